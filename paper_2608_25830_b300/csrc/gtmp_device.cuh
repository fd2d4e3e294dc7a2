// Device-side building blocks of the layered-graph planner (sm_103a).
//
// * Philox4x32-10 counter-based generator (Salmon et al., SC'11) and the
//   sample streams of the planner (Alg. 1 uniform layers; AO-GTMP informed /
//   heuristic expansion).
// * Forward kinematics of a DH serial arm into link collision spheres and the
//   sphere/box obstacle predicate of one configuration (membership in C_free,
//   Sec. III).
// * Packed (value, index) keys for the min/argmin of the value iteration
//   (Sec. IV-B): costs are non-negative floats, so their IEEE bit patterns
//   order like unsigned integers and a 64-bit unsigned min over
//   (bits(value) << 32 | index) is the lexicographic (value, first index)
//   minimum, independent of the order in which candidates arrive.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace gtmp {

constexpr int kMaxDof = 16;
constexpr int kMaxSpl = 8;
constexpr uint32_t kTagUniform = 1u;
constexpr uint32_t kTagInformed = 2u;
constexpr uint32_t kTagCoin = 3u;
constexpr uint32_t kTagFree = 5u;  // rejection attempts of the free-space sampler
constexpr unsigned long long kEmptyKey = ~0ull;
constexpr unsigned kFull = 0xffffffffu;

// Error bits written to the context's device error word.
constexpr int kErrSamplerExhausted = 1;
constexpr int kErrWaitTimeout = 2;

// ----------------------------------------------------------------------------
// Robot description passed by value (kernel parameter space, i.e. constant
// bank): with compile-time link and sphere counts every access below is an
// immediate constant-bank operand.
// ----------------------------------------------------------------------------
struct RobotDev {
  int kind;          // 0 = point robot, 1 = DH serial arm
  int dof;
  int spl;           // spheres per link (arm)
  int uniform_r;     // all robot spheres share radius r_uniform
  float r_uniform;
  float point_radius;
  float d[kMaxDof], a[kMaxDof], ca[kMaxDof], sa[kMaxDof], toff[kMaxDof];
  float4 sph[kMaxDof * kMaxSpl];  // x, y, z, r in the link frame
  float4 lb[kMaxDof];              // per link: centre (link frame) and radius of a ball holding all its spheres
};

// ----------------------------------------------------------------------------
// Philox4x32-10
// ----------------------------------------------------------------------------
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k) {
  constexpr uint32_t m0 = 0xD2511F53u, m1 = 0xCD9E8D57u;
  constexpr uint32_t w0 = 0x9E3779B9u, w1 = 0xBB67AE85u;
#pragma unroll
  for (int round = 0; round < 10; ++round) {
    if (round > 0) {
      k.x += w0;
      k.y += w1;
    }
    const uint32_t hi0 = __umulhi(m0, c.x), lo0 = m0 * c.x;
    const uint32_t hi1 = __umulhi(m1, c.z), lo1 = m1 * c.z;
    c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
  }
  return c;
}

__device__ __forceinline__ uint2 seed_key(unsigned long long seed) {
  return make_uint2(static_cast<uint32_t>(seed), static_cast<uint32_t>(seed >> 32));
}

__device__ __forceinline__ uint32_t word_of(const uint4& w, int k) {
  switch (k & 3) {
    case 0: return w.x;
    case 1: return w.y;
    case 2: return w.z;
    default: return w.w;
  }
}

// top 24 bits of a Philox word times 2^-24: exact float in [0, 1)
__device__ __forceinline__ float word_to_unit(uint32_t w) {
  return __fmul_rn(__uint2float_rn(w >> 8), 5.9604644775390625e-08f);
}

// ----------------------------------------------------------------------------
// Packed keys
// ----------------------------------------------------------------------------
__device__ __forceinline__ unsigned long long make_key(float value, uint32_t index) {
  return (static_cast<unsigned long long>(__float_as_uint(value)) << 32) | index;
}
__device__ __forceinline__ float key_value(unsigned long long k) {
  return k == kEmptyKey ? __int_as_float(0x7f800000) : __uint_as_float(static_cast<uint32_t>(k >> 32));
}
__device__ __forceinline__ int key_index(unsigned long long k) {
  return k == kEmptyKey ? -1 : static_cast<int>(static_cast<uint32_t>(k));
}

__device__ __forceinline__ unsigned long long warp_min_u64(unsigned long long v) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    const unsigned long long o = __shfl_xor_sync(kFull, v, off);
    v = o < v ? o : v;
  }
  return v;
}

// ----------------------------------------------------------------------------
// Obstacle predicate for a group of robot spheres.
//
// Sphere obstacles live in shared memory as float4 (cx, cy, cz, w):
//   uniform robot radius r:  w = (r_obs + r)^2   (inflated squared threshold)
//   otherwise:               w = r_obs
// Boxes as two float4: (cx, cy, cz, hx), (hy, hz, -, -) (centre, half extents).
// A robot sphere (c, r) collides with a sphere obstacle iff |c - o|^2 < (r+r_o)^2,
// with a box iff the squared distance from c to the box is below r^2, or c is
// strictly inside the box (only decisive for a zero-radius point robot).
// ----------------------------------------------------------------------------
template <int NS, bool UNIF, bool INSIDE_TEST>
__device__ __forceinline__ bool spheres_hit(const float (&cx)[NS], const float (&cy)[NS], const float (&cz)[NS],
                                            const float (&rad)[NS], int ns_active,
                                            const float4* __restrict__ sph, int n_s,
                                            const float4* __restrict__ box, int n_b, float r2_box_uniform) {
  bool hit = false;
#pragma unroll 2
  for (int o = 0; o < n_s; ++o) {
    const float4 ob = sph[o];
#pragma unroll
    for (int k = 0; k < NS; ++k) {
      if (NS > 1 && k >= ns_active) break;
      const float dx = __fsub_rn(cx[k], ob.x);
      const float dy = __fsub_rn(cy[k], ob.y);
      const float dz = __fsub_rn(cz[k], ob.z);
      const float d2 = __fmaf_rn(dz, dz, __fmaf_rn(dy, dy, __fmul_rn(dx, dx)));
      float thr;
      if (UNIF) {
        thr = ob.w;
      } else {
        const float rs = __fadd_rn(rad[k], ob.w);
        thr = __fmul_rn(rs, rs);
      }
      hit |= d2 < thr;
    }
  }
#pragma unroll 1
  for (int o = 0; o < n_b; ++o) {
    const float4 b0 = box[2 * o];
    const float4 b1 = box[2 * o + 1];
#pragma unroll
    for (int k = 0; k < NS; ++k) {
      if (NS > 1 && k >= ns_active) break;
      const float ex = __fsub_rn(fabsf(__fsub_rn(cx[k], b0.x)), b0.w);
      const float ey = __fsub_rn(fabsf(__fsub_rn(cy[k], b0.y)), b1.x);
      const float ez = __fsub_rn(fabsf(__fsub_rn(cz[k], b0.z)), b1.y);
      const float px = fmaxf(ex, 0.0f), py = fmaxf(ey, 0.0f), pz = fmaxf(ez, 0.0f);
      const float d2 = __fmaf_rn(pz, pz, __fmaf_rn(py, py, __fmul_rn(px, px)));
      const float r2 = UNIF ? r2_box_uniform : __fmul_rn(rad[k], rad[k]);
      hit |= d2 < r2;
      if (INSIDE_TEST) hit |= fmaxf(ex, fmaxf(ey, ez)) < 0.0f;
    }
  }
  return hit;
}

// ----------------------------------------------------------------------------
// Conservative prefilter (uniform robot-sphere radius r).  Every obstacle o is
// enclosed in a ball (centre o, radius R_o = r_obs + r for a sphere,
// |half extents| + r for a box) and stored in pairs as float4
//   (ax_a, ax_b, ay_a, ay_b), (az_a, az_b, k_a, k_b),  a = -2 o,
//   k = |o|^2 - R_o^2 - margin,
// so that t = |c|^2 + a.c + k = |c - o|^2 - R_o^2 - margin takes three
// packed FMAs per pair of obstacles.  A robot sphere may touch o only if
// t < 0; margin (set on the host) exceeds the float32 rounding error of this
// expanded form by two orders of magnitude, so a pair the prefilter clears is
// also cleared by the exact test, and the exact test is run whenever any lane
// is not cleared.  The labels are therefore those of the exact test alone.
// ----------------------------------------------------------------------------
// Joint angles the arm kernels accept: |q| <= kMaxJointAngle for joint
// limits (so for every sample, endpoint and goal, which lie in the joint box)
// and |theta_offset| <= kMaxThetaOffset, so that every argument of
// joint_sincos stays within 6144 rad.  gtmp_create and gtmp_batch_create
// refuse arms outside these bounds; gtmp_label_configs labels a configuration
// with a larger coordinate as colliding.
constexpr float kMaxJointAngle = 4096.0f;
constexpr float kMaxThetaOffset = 2048.0f;

// Sine and cosine of a joint angle for the forward kinematics: Cody-Waite
// reduction by pi/2 (pi/2 split into three float32 parts, the first two with
// significands of at most 12 bits, so that k times each is exact for
// |k| < 2^12, i.e. |x| < 6434), then the Taylor series of sin and cos about 0
// on |r| <= pi/4 (through r^9 and r^10; the first omitted terms are below
// 2e-9 there), then the quadrant's swap and signs.  Within 1.5 ulp of the
// exact values for |x| <= 6144 (float32 emulation against FP64, and a GPU
// test against FP64).  No branch: the fused kernels keep their registers.
__device__ __forceinline__ void joint_sincos(float x, float* s_out, float* c_out) {
  const float t = __fmaf_rn(x, 0.636619772f, 12582912.0f);  // 1.5 * 2^23 + rint(x * 2 / pi)
  const float kf = __fsub_rn(t, 12582912.0f);
  const int q = __float_as_int(t) & 3;                        // rint(x * 2 / pi) mod 4
  float r = __fmaf_rn(-kf, 1.5703125f, x);
  r = __fmaf_rn(-kf, 4.837512969970703e-4f, r);
  r = __fmaf_rn(-kf, 7.549790126404332e-8f, r);
  const float r2 = __fmul_rn(r, r);
  // 1/9!, -1/7!, 1/5!, -1/3!
  float ps = __fmaf_rn(r2, 2.75573192e-6f, -1.98412698e-4f);
  ps = __fmaf_rn(r2, ps, 8.33333333e-3f);
  ps = __fmaf_rn(r2, ps, -1.66666667e-1f);
  const float sn = __fmaf_rn(__fmul_rn(r, r2), ps, r);
  // -1/10!, 1/8!, -1/6!, 1/4!, -1/2!
  float pc = __fmaf_rn(r2, -2.75573192e-7f, 2.48015873e-5f);
  pc = __fmaf_rn(r2, pc, -1.38888889e-3f);
  pc = __fmaf_rn(r2, pc, 4.16666667e-2f);
  pc = __fmaf_rn(r2, pc, -0.5f);
  const float cs = __fmaf_rn(r2, pc, 1.0f);
  const float a = (q & 1) ? cs : sn;
  const float b = (q & 1) ? sn : cs;
  *s_out = __int_as_float(__float_as_int(a) ^ ((q & 2) << 30));
  *c_out = __int_as_float(__float_as_int(b) ^ (((q + 1) & 2) << 30));
}

__device__ __forceinline__ float fmin3(float a, float b, float c) {
  float r;
  asm("min.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
  return r;
}

template <int NS>
__device__ __forceinline__ bool prefilter_maybe(const float (&cx)[NS], const float (&cy)[NS], const float (&cz)[NS],
                                                const float4* __restrict__ pre, int n_pairs) {
  float2 x2[NS], y2[NS], z2[NS];
  float m[NS], c2[NS];
#pragma unroll
  for (int k = 0; k < NS; ++k) {
    x2[k] = make_float2(cx[k], cx[k]);
    y2[k] = make_float2(cy[k], cy[k]);
    z2[k] = make_float2(cz[k], cz[k]);
    c2[k] = __fmaf_rn(cz[k], cz[k], __fmaf_rn(cy[k], cy[k], __fmul_rn(cx[k], cx[k])));
    m[k] = __int_as_float(0x7f800000);
  }
#pragma unroll 2
  for (int p = 0; p < n_pairs; ++p) {
    const float4 P0 = pre[2 * p];
    const float4 P1 = pre[2 * p + 1];
    const float2 ax = make_float2(P0.x, P0.y), ay = make_float2(P0.z, P0.w);
    const float2 az = make_float2(P1.x, P1.y), kk = make_float2(P1.z, P1.w);
#pragma unroll
    for (int k = 0; k < NS; ++k) {
      const float2 t = __ffma2_rn(z2[k], az, __ffma2_rn(y2[k], ay, __ffma2_rn(x2[k], ax, kk)));
      m[k] = fmin3(m[k], t.x, t.y);
    }
  }
  bool maybe = false;
#pragma unroll
  for (int k = 0; k < NS; ++k) maybe |= m[k] < -c2[k];
  return maybe;
}

// ----------------------------------------------------------------------------
// Link cull of the early-exit mode: which obstacles can come within the
// link's bounding ball (centre c, radius R) plus a margin?  Table pairs (three
// float4), sphere obstacles' pairs first, then box obstacles' pairs (the
// pairing of the exact tables): (-2ox_a, -2ox_b, -2oy_a, -2oy_b),
// (-2oz_a, -2oz_b, K_a, K_b), (-2r_a, -2r_b, 0, 0) with K = |o|^2 - r_o^2 -
// margin (boxes: their enclosing ball).  Obstacle o may reach the ball iff
// |c|^2 - 2 o.c + K - 2 r_o R - R^2 < 0.  Returns bit p set when pair p may
// (pairs past 64 are all reported near); a cleared obstacle cannot touch any
// of the link's spheres, which all lie inside the ball.
// ----------------------------------------------------------------------------
// Uniform grid over the obstacles (see build_cull_grid): the cell holding a
// link ball's centre gives the cull pairs that can reach the ball, a superset
// of what link_cull_mask finds; points outside the grid reach no obstacle.
struct CullGrid {
  const unsigned* cells = nullptr;  // null: no grid
  float lx = 0.0f, ly = 0.0f, lz = 0.0f, inv = 0.0f;
  int nx = 0, ny = 0, nz = 0;
  float fnx = 0.0f, fny = 0.0f, fnz = 0.0f;  // nx, ny, nz as floats
};

// The cell's mask of obstacle pairs (0 outside the grid).  The cell index takes floor(f) for
// 0 <= f < 2^23 as the bits of f + 2^23 rounded down (an FP32 add, where a float-to-int conversion
// would go to the slower conversion pipe), the grid extents as floats.
__device__ __forceinline__ unsigned grid_cell_mask(const CullGrid& gv, float x, float y, float z) {
  const float fx = __fmul_rn(__fsub_rn(x, gv.lx), gv.inv);
  const float fy = __fmul_rn(__fsub_rn(y, gv.ly), gv.inv);
  const float fz = __fmul_rn(__fsub_rn(z, gv.lz), gv.inv);
  if (!(fx >= 0.0f && fy >= 0.0f && fz >= 0.0f && fx < gv.fnx && fy < gv.fny && fz < gv.fnz)) return 0u;
  const int ix = min(__float_as_int(__fadd_rd(fx, 8388608.0f)) - 0x4B000000, gv.nx - 1);
  const int iy = min(__float_as_int(__fadd_rd(fy, 8388608.0f)) - 0x4B000000, gv.ny - 1);
  const int iz = min(__float_as_int(__fadd_rd(fz, 8388608.0f)) - 0x4B000000, gv.nz - 1);
  return gv.cells[(iz * gv.ny + iy) * gv.nx + ix];
}

// link_cull_mask restricted to the pairs set in sel (at most 32 pairs)
__device__ __forceinline__ unsigned link_cull_mask_sel(float cx, float cy, float cz, float R,
                                                       const float4* __restrict__ cull, unsigned sel) {
  const float2 x2 = make_float2(cx, cx), y2 = make_float2(cy, cy), z2 = make_float2(cz, cz);
  const float2 r2 = make_float2(R, R);
  const float c2 = __fmaf_rn(cz, cz, __fmaf_rn(cy, cy, __fmul_rn(cx, cx)));
  const float thr = __fmaf_rn(R, R, -c2);
  unsigned mask = 0u;
  while (sel) {
    const int p = __ffs(sel) - 1;
    sel &= sel - 1u;
    const float4 A = cull[3 * p], B = cull[3 * p + 1], C = cull[3 * p + 2];
    float2 t = __ffma2_rn(z2, make_float2(B.x, B.y),
                          __ffma2_rn(y2, make_float2(A.z, A.w), __ffma2_rn(x2, make_float2(A.x, A.y), make_float2(B.z, B.w))));
    t = __ffma2_rn(make_float2(C.x, C.y), r2, t);
    if (fminf(t.x, t.y) < thr) mask |= 1u << p;
  }
  return mask;
}

__device__ __forceinline__ unsigned long long link_cull_mask(float cx, float cy, float cz, float R,
                                                             const float4* __restrict__ cull, int n_pairs) {
  const float2 x2 = make_float2(cx, cx), y2 = make_float2(cy, cy), z2 = make_float2(cz, cz);
  const float2 r2 = make_float2(R, R);
  const float c2 = __fmaf_rn(cz, cz, __fmaf_rn(cy, cy, __fmul_rn(cx, cx)));
  const float thr = __fmaf_rn(R, R, -c2);
  if (n_pairs <= 32) {
    // one 32-bit word and a running bit: no 64-bit shifts in the loop
    unsigned mask = 0u, bit = 1u;
#pragma unroll 2
    for (int p = 0; p < n_pairs; ++p, bit <<= 1) {
      const float4 A = cull[3 * p], B = cull[3 * p + 1], C = cull[3 * p + 2];
      float2 t = __ffma2_rn(z2, make_float2(B.x, B.y),
                            __ffma2_rn(y2, make_float2(A.z, A.w), __ffma2_rn(x2, make_float2(A.x, A.y), make_float2(B.z, B.w))));
      t = __ffma2_rn(make_float2(C.x, C.y), r2, t);
      if (fminf(t.x, t.y) < thr) mask |= bit;
    }
    return mask;
  }
  unsigned long long mask = n_pairs > 64 ? ~0ull : 0ull;
  const int n = n_pairs < 64 ? n_pairs : 64;
#pragma unroll 2
  for (int p = 0; p < n; ++p) {
    const float4 A = cull[3 * p], B = cull[3 * p + 1], C = cull[3 * p + 2];
    float2 t = __ffma2_rn(z2, make_float2(B.x, B.y),
                          __ffma2_rn(y2, make_float2(A.z, A.w), __ffma2_rn(x2, make_float2(A.x, A.y), make_float2(B.z, B.w))));
    t = __ffma2_rn(make_float2(C.x, C.y), r2, t);
    if (fminf(t.x, t.y) < thr) mask |= 1ull << p;
  }
  return mask;
}

// ----------------------------------------------------------------------------
// Exact test of the uniform-radius arm kernels, two obstacles per packed
// float32x2 instruction.  Tables (negated positions, radius r of the robot
// spheres folded into the thresholds):
//   sphere pair: (-ox_a, -ox_b, -oy_a, -oy_b), (-oz_a, -oz_b, -T_a, -T_b),
//                T = (r_obs + r)^2;
//   box pair:    (-bx_a, -bx_b, -by_a, -by_b), (-bz_a, -bz_b, -hx_a, -hx_b),
//                (-hy_a, -hy_b, -hz_a, -hz_b)   (centre b, half extents h).
// A sphere hits iff dx^2 + dy^2 + dz^2 - T < 0 and a box iff
// sum_k max(|c_k - b_k| - h_k, 0)^2 - r^2 < 0, each sum taken as one fma chain
// starting from the negated threshold (each box gap clamped as box_gap
// states).  Odd counts are padded with obstacles at 1e18 that never hit.
// ----------------------------------------------------------------------------
// Gap of a box test along one axis, max(|u| - h, 0) for u the offset from the
// box centre and neg_h = -h, clamped to at most 1 by the same instruction (a
// saturating add, one rounding as __fadd_rn).  The clamp changes no decision
// while the robot sphere radius r is below 1: the test is gx^2 + gy^2 + gz^2
// - r^2 < 0, and one clamped gap alone already makes the sum at least 1 - r^2
// > 0, as the unclamped gap does.  The packed arm kernels are therefore chosen
// only for radii below 1 (arm_kernel_variant).
__device__ __forceinline__ float box_gap(float u, float neg_h) {
  float g;
  asm("{\n\t.reg .f32 a;\n\tabs.f32 a, %1;\n\tadd.rn.sat.f32 %0, a, %2;\n\t}" : "=f"(g) : "f"(u), "f"(neg_h));
  return g;
}

template <int NS>
__device__ __forceinline__ bool exact_packed_hit(const float (&cx)[NS], const float (&cy)[NS], const float (&cz)[NS],
                                                 const float4* __restrict__ sphp, int n_sp,
                                                 const float4* __restrict__ boxp, int n_bp, float neg_r2) {
  float2 x2[NS], y2[NS], z2[NS];
  float m[NS];
#pragma unroll
  for (int k = 0; k < NS; ++k) {
    x2[k] = make_float2(cx[k], cx[k]);
    y2[k] = make_float2(cy[k], cy[k]);
    z2[k] = make_float2(cz[k], cz[k]);
    m[k] = __int_as_float(0x7f800000);
  }
#pragma unroll 1
  for (int p = 0; p < n_sp; ++p) {
    const float4 P0 = sphp[2 * p];
    const float4 P1 = sphp[2 * p + 1];
    const float2 nx = make_float2(P0.x, P0.y), ny = make_float2(P0.z, P0.w);
    const float2 nz = make_float2(P1.x, P1.y), nt = make_float2(P1.z, P1.w);
#pragma unroll
    for (int k = 0; k < NS; ++k) {
      const float2 dx = __fadd2_rn(x2[k], nx);
      const float2 dy = __fadd2_rn(y2[k], ny);
      const float2 dz = __fadd2_rn(z2[k], nz);
      const float2 t = __ffma2_rn(dz, dz, __ffma2_rn(dy, dy, __ffma2_rn(dx, dx, nt)));
      m[k] = fmin3(m[k], t.x, t.y);
    }
  }
  const float2 nr2 = make_float2(neg_r2, neg_r2);
#pragma unroll 1
  for (int p = 0; p < n_bp; ++p) {
    const float4 B0 = boxp[3 * p];
    const float4 B1 = boxp[3 * p + 1];
    const float4 B2 = boxp[3 * p + 2];
    const float2 nbx = make_float2(B0.x, B0.y), nby = make_float2(B0.z, B0.w), nbz = make_float2(B1.x, B1.y);
#pragma unroll
    for (int k = 0; k < NS; ++k) {
      const float2 ux = __fadd2_rn(x2[k], nbx);
      const float2 uy = __fadd2_rn(y2[k], nby);
      const float2 uz = __fadd2_rn(z2[k], nbz);
      const float2 px = make_float2(box_gap(ux.x, B1.z), box_gap(ux.y, B1.w));
      const float2 py = make_float2(box_gap(uy.x, B2.x), box_gap(uy.y, B2.y));
      const float2 pz = make_float2(box_gap(uz.x, B2.z), box_gap(uz.y, B2.w));
      const float2 t = __ffma2_rn(pz, pz, __ffma2_rn(py, py, __ffma2_rn(px, px, nr2)));
      m[k] = fmin3(m[k], t.x, t.y);
    }
  }
  bool hit = false;
#pragma unroll
  for (int k = 0; k < NS; ++k) hit |= m[k] < 0.0f;
  return hit;
}

// The exact test restricted to the sphere pairs set in smask and the box pairs
// set in bmask (pairs a link cull could not clear); same arithmetic per pair.
template <int NS>
__device__ __forceinline__ bool exact_packed_hit_masked(const float (&cx)[NS], const float (&cy)[NS],
                                                        const float (&cz)[NS], const float4* __restrict__ sphp,
                                                        const float4* __restrict__ boxp, float neg_r2,
                                                        unsigned smask, unsigned bmask) {
  float2 x2[NS], y2[NS], z2[NS];
  float m[NS];
#pragma unroll
  for (int k = 0; k < NS; ++k) {
    x2[k] = make_float2(cx[k], cx[k]);
    y2[k] = make_float2(cy[k], cy[k]);
    z2[k] = make_float2(cz[k], cz[k]);
    m[k] = __int_as_float(0x7f800000);
  }
  for (unsigned sm = smask; sm; sm &= sm - 1) {
    const int p = __ffs(sm) - 1;
    const float4 P0 = sphp[2 * p];
    const float4 P1 = sphp[2 * p + 1];
    const float2 nx = make_float2(P0.x, P0.y), ny = make_float2(P0.z, P0.w);
    const float2 nz = make_float2(P1.x, P1.y), nt = make_float2(P1.z, P1.w);
#pragma unroll
    for (int k = 0; k < NS; ++k) {
      const float2 dx = __fadd2_rn(x2[k], nx);
      const float2 dy = __fadd2_rn(y2[k], ny);
      const float2 dz = __fadd2_rn(z2[k], nz);
      const float2 t = __ffma2_rn(dz, dz, __ffma2_rn(dy, dy, __ffma2_rn(dx, dx, nt)));
      m[k] = fmin3(m[k], t.x, t.y);
    }
  }
  const float2 nr2 = make_float2(neg_r2, neg_r2);
  for (unsigned bm = bmask; bm; bm &= bm - 1) {
    const int p = __ffs(bm) - 1;
    const float4 B0 = boxp[3 * p];
    const float4 B1 = boxp[3 * p + 1];
    const float4 B2 = boxp[3 * p + 2];
    const float2 nbx = make_float2(B0.x, B0.y), nby = make_float2(B0.z, B0.w), nbz = make_float2(B1.x, B1.y);
#pragma unroll
    for (int k = 0; k < NS; ++k) {
      const float2 ux = __fadd2_rn(x2[k], nbx);
      const float2 uy = __fadd2_rn(y2[k], nby);
      const float2 uz = __fadd2_rn(z2[k], nbz);
      const float2 px = make_float2(box_gap(ux.x, B1.z), box_gap(ux.y, B1.w));
      const float2 py = make_float2(box_gap(uy.x, B2.x), box_gap(uy.y, B2.y));
      const float2 pz = make_float2(box_gap(uz.x, B2.z), box_gap(uz.y, B2.w));
      const float2 t = __ffma2_rn(pz, pz, __ffma2_rn(py, py, __ffma2_rn(px, px, nr2)));
      m[k] = fmin3(m[k], t.x, t.y);
    }
  }
  bool hit = false;
#pragma unroll
  for (int k = 0; k < NS; ++k) hit |= m[k] < 0.0f;
  return hit;
}

// ----------------------------------------------------------------------------
// One configuration against the scene.
//
// WARP_EXIT: the caller is a whole warp evaluating waypoints of the same
// edge; after each link the warp stops as soon as any active lane has found a
// collision (early exit).  Otherwise each thread stops at its own first hit.
// FULL: no early exit at all (data-independent work), result unchanged.
// Returns, for WARP_EXIT, the warp-uniform "some active lane collides"; else
// the lane's own label.
// ----------------------------------------------------------------------------
// PACKED (uniform-radius arms): sph/box are the packed pair tables of
// exact_packed_hit with n_s/n_b pair counts, pre the prefilter table; the
// prefilter is used only when FULL is false.  Otherwise sph/box are the
// scalar tables of spheres_hit.
template <int DOF_T, int SPL_T, bool UNIF, bool WARP_EXIT, bool FULL, bool PACKED = false>
__device__ __forceinline__ bool arm_config_collides(const float* q, bool active, const RobotDev& rb,
                                                    const float4* __restrict__ sph, int n_s,
                                                    const float4* __restrict__ box, int n_b,
                                                    const float4* __restrict__ pre = nullptr, int n_pairs = 0,
                                                    const float4* __restrict__ cull = nullptr, int n_cull = 0,
                                                    const CullGrid& grid = CullGrid()) {
  constexpr int NS = SPL_T > 0 ? SPL_T : kMaxSpl;
  constexpr int NQ = DOF_T > 0 ? DOF_T : kMaxDof;
  const int dof = DOF_T > 0 ? DOF_T : rb.dof;
  const int spl = SPL_T > 0 ? SPL_T : rb.spl;
  const float r2u = __fmul_rn(rb.r_uniform, rb.r_uniform);
  // joint angles rotate through a register array so that the link loop stays
  // rolled (one copy of the link body: small code, no instruction-cache misses)
  float ang[NQ];
#pragma unroll
  for (int k = 0; k < NQ; ++k) ang[k] = (DOF_T > 0 || k < dof) ? q[k] : 0.0f;
  // running frame of link i: rotation columns X, Y, Z and origin T
  float X0 = 1.f, X1 = 0.f, X2 = 0.f, Y0 = 0.f, Y1 = 1.f, Y2 = 0.f, Z0 = 0.f, Z1 = 0.f, Z2 = 1.f;
  float T0 = 0.f, T1 = 0.f, T2 = 0.f;
  bool hit = false;
  // without FULL, the next joint's sine and cosine are computed a link ahead, a chain independent of
  // the current link's (more independent work per warp; wasted only on the link where a warp exits;
  // measured slower in FULL, where nothing exits)
  float s_nx = 0.0f, c_nx = 1.0f;
  if constexpr (!FULL) joint_sincos(__fadd_rn(ang[0], rb.toff[0]), &s_nx, &c_nx);
  // FULL unrolls the link loop (no exits: the straight-line code schedules better, 45.6 against 46.7
  // ms per full-evaluation solve of a 7-joint arm); the other modes keep one copy of the body, since
  // their branches and exits made an unrolled loop slower (instruction-cache misses)
#pragma unroll(FULL ? 8 : 1)
  for (int i = 0; i < dof; ++i) {
    const float qi = ang[0];
#pragma unroll
    for (int k = 0; k + 1 < NQ; ++k) ang[k] = ang[k + 1];
    float s, c;
    if constexpr (FULL) {
      joint_sincos(__fadd_rn(qi, rb.toff[i]), &s, &c);
    } else {
      s = s_nx;
      c = c_nx;
      // joint i + 1 (past the last joint the result goes unused; the index stays inside toff)
      joint_sincos(__fadd_rn(ang[0], rb.toff[i + 1 < kMaxDof ? i + 1 : i]), &s_nx, &c_nx);
    }
    // A_i = Rz(theta) Tz(d) Tx(a) Rx(alpha): new x axis u = c X + s Y,
    // v = -s X + c Y, new y = ca v + sa Z, new z = -sa v + ca Z,
    // new origin = T + a u + d Z.
    const float u0 = __fmaf_rn(s, Y0, __fmul_rn(c, X0));
    const float u1 = __fmaf_rn(s, Y1, __fmul_rn(c, X1));
    const float u2 = __fmaf_rn(s, Y2, __fmul_rn(c, X2));
    const float v0 = __fmaf_rn(c, Y0, __fmul_rn(-s, X0));
    const float v1 = __fmaf_rn(c, Y1, __fmul_rn(-s, X1));
    const float v2 = __fmaf_rn(c, Y2, __fmul_rn(-s, X2));
    const float ca = rb.ca[i], sa = rb.sa[i];
    T0 = __fmaf_rn(rb.d[i], Z0, __fmaf_rn(rb.a[i], u0, T0));
    T1 = __fmaf_rn(rb.d[i], Z1, __fmaf_rn(rb.a[i], u1, T1));
    T2 = __fmaf_rn(rb.d[i], Z2, __fmaf_rn(rb.a[i], u2, T2));
    const float y0 = __fmaf_rn(sa, Z0, __fmul_rn(ca, v0));
    const float y1 = __fmaf_rn(sa, Z1, __fmul_rn(ca, v1));
    const float y2 = __fmaf_rn(sa, Z2, __fmul_rn(ca, v2));
    const float z0 = __fmaf_rn(ca, Z0, __fmul_rn(-sa, v0));
    const float z1 = __fmaf_rn(ca, Z1, __fmul_rn(-sa, v1));
    const float z2 = __fmaf_rn(ca, Z2, __fmul_rn(-sa, v2));
    X0 = u0; X1 = u1; X2 = u2;
    Y0 = y0; Y1 = y1; Y2 = y2;
    Z0 = z0; Z1 = z1; Z2 = z2;
    // obstacle pairs a link cull could not clear (sphere pairs, box pairs)
    unsigned near_s = 0xffffffffu, near_b = 0xffffffffu;
    if constexpr (PACKED && !FULL) {
      // skip the link when its bounding ball is clear of every obstacle (for
      // every active lane), else test only the obstacles near the ball
      if (n_cull > 0) {
        const float4 lb = rb.lb[i];
        const float lx = __fmaf_rn(lb.z, Z0, __fmaf_rn(lb.y, Y0, __fmaf_rn(lb.x, X0, T0)));
        const float ly = __fmaf_rn(lb.z, Z1, __fmaf_rn(lb.y, Y1, __fmaf_rn(lb.x, X1, T1)));
        const float lz = __fmaf_rn(lb.z, Z2, __fmaf_rn(lb.y, Y2, __fmaf_rn(lb.x, X2, T2)));
        unsigned long long near;
        if (grid.cells != nullptr) {
          // the grid cell first (one lookup), then the ball test on the pairs it keeps
          unsigned sel = active ? grid_cell_mask(grid, lx, ly, lz) : 0u;
          if (WARP_EXIT) sel = __reduce_or_sync(kFull, sel);
          if (sel == 0u) continue;
          unsigned m = active ? link_cull_mask_sel(lx, ly, lz, lb.w, cull, sel) : 0u;
          if (WARP_EXIT) m = __reduce_or_sync(kFull, m);
          near = m;
        } else {
          near = active ? link_cull_mask(lx, ly, lz, lb.w, cull, n_cull) : 0ull;
          if (WARP_EXIT) {
            const unsigned lo = __reduce_or_sync(kFull, static_cast<unsigned>(near));
            const unsigned hi = n_cull > 32 ? __reduce_or_sync(kFull, static_cast<unsigned>(near >> 32)) : 0u;
            near = (static_cast<unsigned long long>(hi) << 32) | lo;
          }
        }
        if (near == 0ull) continue;
        if (n_cull <= 64 && n_s <= 32 && n_b <= 32) {
          near_s = static_cast<unsigned>(near & (n_s >= 32 ? 0xffffffffull : (1ull << n_s) - 1ull));
          near_b = static_cast<unsigned>(near >> n_s);
        }
      }
    }
    float cx[NS], cy[NS], cz[NS], rad[NS];
#pragma unroll
    for (int k = 0; k < NS; ++k) {
      if (SPL_T == 0 && k >= spl) break;
      const float4 p = rb.sph[i * (SPL_T > 0 ? SPL_T : kMaxSpl) + k];
      cx[k] = __fmaf_rn(p.z, Z0, __fmaf_rn(p.y, Y0, __fmaf_rn(p.x, X0, T0)));
      cy[k] = __fmaf_rn(p.z, Z1, __fmaf_rn(p.y, Y1, __fmaf_rn(p.x, X1, T1)));
      cz[k] = __fmaf_rn(p.z, Z2, __fmaf_rn(p.y, Y2, __fmaf_rn(p.x, X2, T2)));
      rad[k] = p.w;
    }
    if constexpr (PACKED && FULL) {
      hit |= exact_packed_hit<NS>(cx, cy, cz, sph, n_s, box, n_b, -r2u);
    } else if constexpr (PACKED) {
      if (n_cull > 0 && n_cull <= 64 && n_s <= 32 && n_b <= 32) {
        // exact tests against the obstacles the link cull kept
        hit |= exact_packed_hit_masked<NS>(cx, cy, cz, sph, box, -r2u, near_s, near_b);
      } else {
        // exact tests only where the prefilter could not clear the link
        const bool maybe = prefilter_maybe<NS>(cx, cy, cz, pre, n_pairs);
        bool run_exact;
        if constexpr (WARP_EXIT)
          run_exact = __any_sync(kFull, active && maybe);
        else
          run_exact = maybe;
        if (run_exact) hit |= exact_packed_hit<NS>(cx, cy, cz, sph, n_s, box, n_b, -r2u);
      }
    } else {
      hit |= spheres_hit<NS, UNIF, false>(cx, cy, cz, rad, spl, sph, n_s, box, n_b, r2u);
    }
    if (!FULL) {
      if (WARP_EXIT) {
        if (__any_sync(kFull, active && hit)) return true;
      } else if (hit) {
        return true;
      }
    }
  }
  if (WARP_EXIT) return __any_sync(kFull, active && hit);
  return hit;
}

template <bool WARP_EXIT>
__device__ __forceinline__ bool point_config_collides(const float* q, bool active, const RobotDev& rb,
                                                      const float4* __restrict__ sph, int n_s,
                                                      const float4* __restrict__ box, int n_b) {
  const float cx[1] = {q[0]};
  const float cy[1] = {rb.dof > 1 ? q[1] : 0.0f};
  const float cz[1] = {rb.dof > 2 ? q[2] : 0.0f};
  const float rad[1] = {rb.point_radius};
  const float r2u = __fmul_rn(rb.point_radius, rb.point_radius);
  const bool hit = spheres_hit<1, true, true>(cx, cy, cz, rad, 1, sph, n_s, box, n_b, r2u);
  if (WARP_EXIT) return __any_sync(kFull, active && hit);
  return hit;
}

}  // namespace gtmp
