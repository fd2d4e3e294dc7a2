// Device-side pieces shared by the single-problem kernels (gtmp_kernels.cu)
// and the batched persistent solver (gtmp_batch.cu): launch constants, the
// bounded TMA staging of obstacle tables, robot-variant traits, the per-
// configuration collision test and the per-row chunk of the fused edge +
// min-plus step.  Everything here has internal linkage.
#pragma once

#include "gtmp_kernels.cuh"

namespace gtmp {

namespace {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
// resident blocks per SM the edge kernels are compiled for (2 -> register budget 128)
#ifndef GTMP_FUSED_MIN_BLOCKS
#define GTMP_FUSED_MIN_BLOCKS 2
#endif
constexpr int kFusedMinBlocks = GTMP_FUSED_MIN_BLOCKS;
#define kInf __int_as_float(0x7f800000)

struct Box16 {
  float lo[kMaxDof], hi[kMaxDof];
};

// ---------------------------------------------------------------------------
// Bulk (TMA) staging of the obstacle list into shared memory, completed on an
// mbarrier.  Every wait is bounded; on timeout the error word is set and the
// block skips its work after one more bounded wait for the copy in flight.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ bool mbar_wait_bounded(uint32_t mbar, uint32_t parity, int limit) {
  for (int it = 0; it < limit; ++it) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(mbar), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}

// Returns false (on all threads) if the copy did not complete in time.
__device__ bool stage_obstacles(float4* s_obs, const float4* g_obs, int n4, uint64_t* mbar_storage, int* err) {
  const uint32_t bytes = static_cast<uint32_t>(n4) * 16u;
  const uint32_t mbar = smem_addr(mbar_storage);
  if (bytes == 0) return __syncthreads_and(1) != 0;
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(mbar) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(mbar), "r"(bytes) : "memory");
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_addr(s_obs)),
        "l"(g_obs), "r"(bytes), "r"(mbar)
        : "memory");
  }
  bool ok = mbar_wait_bounded(mbar, 0, 1 << 22);
  if (!ok) {
    atomicOr(err, kErrWaitTimeout);
    mbar_wait_bounded(mbar, 0, 1 << 22);  // let a late copy land before the block exits
  }
  return __syncthreads_and(ok) != 0;
}

// Plain cooperative staging (used where a kernel also writes other shared data).
__device__ void stage_obstacles_plain(float4* s_obs, const float4* g_obs, int n4) {
  for (int k = threadIdx.x; k < n4; k += blockDim.x) s_obs[k] = g_obs[k];
}

template <int VAR>
struct Var;
template <>
struct Var<kVarPoint> {
  static constexpr bool kArm = false;
  static constexpr int kDof = 0, kSpl = 1, kDp = 4;
  static constexpr bool kUnif = true;
};
template <>
struct Var<kVarArm6x4> {
  static constexpr bool kArm = true;
  static constexpr int kDof = 6, kSpl = 4, kDp = 8;
  static constexpr bool kUnif = true;
};
template <>
struct Var<kVarArm7x4> {
  static constexpr bool kArm = true;
  static constexpr int kDof = 7, kSpl = 4, kDp = 8;
  static constexpr bool kUnif = true;
};
template <>
struct Var<kVarArmGeneric> {
  static constexpr bool kArm = true;
  static constexpr int kDof = 0, kSpl = 0, kDp = kMaxDof;
  static constexpr bool kUnif = false;
};

template <int VAR, bool WARP_EXIT, bool FULL>
__device__ __forceinline__ bool config_collides(const float* q, bool active, const RobotDev& rb, const float4* s_obs,
                                                const SceneDev& sc) {
  using V = Var<VAR>;
  if constexpr (V::kArm && V::kUnif) {
    // uniform-radius arms: packed pair tables, then the prefilter table
    const float4* boxp = s_obs + 2 * sc.n_sp;
    const float4* pre = boxp + 3 * sc.n_bp;
    const float4* cull = pre + 2 * sc.n_pairs;
    CullGrid grid;
    if (sc.gnx > 0) {
      grid.cells = reinterpret_cast<const unsigned*>(s_obs + sc.g_off);
      grid.lx = sc.glx;
      grid.ly = sc.gly;
      grid.lz = sc.glz;
      grid.inv = sc.ginv;
      grid.nx = sc.gnx;
      grid.ny = sc.gny;
      grid.nz = sc.gnz;
      grid.fnx = static_cast<float>(sc.gnx);
      grid.fny = static_cast<float>(sc.gny);
      grid.fnz = static_cast<float>(sc.gnz);
    }
    return arm_config_collides<V::kDof, V::kSpl, V::kUnif, WARP_EXIT, FULL, true>(
        q, active, rb, s_obs, sc.n_sp, boxp, sc.n_bp, pre, sc.n_pairs, cull, sc.n_cull, grid);
  } else if constexpr (V::kArm) {
    return arm_config_collides<V::kDof, V::kSpl, V::kUnif, WARP_EXIT, FULL>(q, active, rb, s_obs, sc.n_s,
                                                                            s_obs + sc.n_s, sc.n_b);
  } else {
    return point_config_collides<WARP_EXIT>(q, active, rb, s_obs, sc.n_s, s_obs + sc.n_s, sc.n_b);
  }
}

// load a padded vertex (dp floats; dp == V::kDp for the specialised variants)
template <int DP>
__device__ __forceinline__ void load_vertex(float (&q)[DP], const float* p, int dp) {
  if (DP == 4 || DP == 8) {
#pragma unroll
    for (int d = 0; d < DP; d += 4) {
      const float4 v = __ldg(reinterpret_cast<const float4*>(p + d));
      q[d] = v.x;
      q[d + 1] = v.y;
      q[d + 2] = v.z;
      q[d + 3] = v.w;
    }
  } else {
#pragma unroll
    for (int d = 0; d < DP; ++d) q[d] = d < dp ? __ldg(p + d) : 0.0f;
  }
}

// ---------------------------------------------------------------------------
// Weighted length (App. "General Costs"): w(q) = 1 + sum_b a_b max(0, 1 -
// |q - c_b|^2 / s_b^2) (1 <= w <= 1 + sum a_b, Lipschitz).  The cost of a
// free edge is the trapezoid rule of w on its H waypoints,
//   |v - u| / (H - 1) * (w_0 / 2 + w_1 + ... + w_{H-2} + w_{H-1} / 2),
// summed in waypoint order in float32, so the lane-per-waypoint and the
// lane-per-edge forms below give the same bits.  Waypoints are the checked
// ones: the endpoints themselves, fma(t_k, v - u, u) in between.
// ---------------------------------------------------------------------------
template <int DP>
__device__ __forceinline__ float weight_at(const float (&q)[DP], const float4* wb, int n_wb) {
  constexpr int kStride = DP / 4 + 1;
  float w = 1.0f;
  for (int b = 0; b < n_wb; ++b) {
    const float4* p = wb + b * kStride;
    float d2 = 0.0f;
#pragma unroll
    for (int d = 0; d < DP; d += 4) {
      const float4 c = __ldg(p + d / 4);
      float e = __fsub_rn(q[d], c.x);
      d2 = __fmaf_rn(e, e, d2);
      e = __fsub_rn(q[d + 1], c.y);
      d2 = __fmaf_rn(e, e, d2);
      e = __fsub_rn(q[d + 2], c.z);
      d2 = __fmaf_rn(e, e, d2);
      e = __fsub_rn(q[d + 3], c.w);
      d2 = __fmaf_rn(e, e, d2);
    }
    const float4 par = __ldg(p + DP / 4);
    w = __fmaf_rn(par.y, fmaxf(__fmaf_rn(-d2, par.x, 1.0f), 0.0f), w);
  }
  return w;
}

// The edge kernels take the weighted cost as a template parameter, so the
// collision loops of the plain-length kernels keep their register allocation.

// one thread, one edge qi -> qj of length len
template <int DP>
__device__ __forceinline__ float weighted_cost_thread(const float (&qi)[DP], const float (&qj)[DP], float len,
                                                      const GraphDev& g) {
  float dq[DP];
#pragma unroll
  for (int d = 0; d < DP; ++d) dq[d] = __fsub_rn(qj[d], qi[d]);
  const float steps = static_cast<float>(g.H - 1);
  float sum = __fmul_rn(0.5f, weight_at<DP>(qi, g.wb, g.n_wb));
  for (int k = 1; k <= g.H - 2; ++k) {
    const float t = __fdiv_rn(static_cast<float>(k), steps);
    float q[DP];
#pragma unroll
    for (int d = 0; d < DP; ++d) q[d] = __fmaf_rn(t, dq[d], qi[d]);
    sum = __fadd_rn(sum, weight_at<DP>(q, g.wb, g.n_wb));
  }
  sum = __fadd_rn(sum, __fmul_rn(0.5f, weight_at<DP>(qj, g.wb, g.n_wb)));
  return __fmul_rn(len, __fdiv_rn(sum, steps));
}

// one warp, one edge: lane k evaluates interior waypoint kb + k, every lane
// then adds the values in waypoint order (all 32 lanes must be converged);
// dq = qj - qi as the collision loop computed it, qj read back from qj_ptr
template <int DP>
__device__ __forceinline__ float weighted_cost_warp(const float (&qi)[DP], const float* qj_ptr, int dp,
                                                    const float (&dq)[DP], float len, const GraphDev& g, int lane) {
  const float steps = static_cast<float>(g.H - 1);
  float sum = __fmul_rn(0.5f, weight_at<DP>(qi, g.wb, g.n_wb));
  for (int kb = 1; kb <= g.H - 2; kb += 32) {
    const int k = kb + lane;
    float w = 0.0f;
    if (k <= g.H - 2) {
      const float t = __fdiv_rn(static_cast<float>(k), steps);
      float q[DP];
#pragma unroll
      for (int d = 0; d < DP; ++d) q[d] = __fmaf_rn(t, dq[d], qi[d]);
      w = weight_at<DP>(q, g.wb, g.n_wb);
    }
    const int n = min(32, g.H - 1 - kb);
    for (int m = 0; m < n; ++m) sum = __fadd_rn(sum, __shfl_sync(kFull, w, m));
  }
  float qj[DP];
  load_vertex<DP>(qj, qj_ptr, dp);
  sum = __fadd_rn(sum, __fmul_rn(0.5f, weight_at<DP>(qj, g.wb, g.n_wb)));
  return __fmul_rn(len, __fdiv_rn(sum, steps));
}

// ---------------------------------------------------------------------------
// One warp, one row i of the transition layer -> layer + 1 of graph r, columns
// [j0, j1): the 32 lanes carry the H-2 interior waypoints of one edge at a
// time (endpoint labels are the vertex flags), the warp leaves an edge at its
// first colliding link unless FULL, and the best (value, column) key of the
// chunk is returned on every lane (kEmptyKey if no edge is realised).
// s_V holds the column layer's cost-to-go, +inf where the vertex collides or
// reaches no goal.
// ---------------------------------------------------------------------------
// Point robots: one waypoint test is a handful of flops, so the 32 lanes take
// 32 columns (edges) at a time and each lane walks its own edge's waypoints.
template <bool FULL, bool WEIGHTED = false>
__device__ __forceinline__ unsigned long long point_row_chunk_best(const GraphDev& g, int r, int layer, int i,
                                                                   int j0, int j1, const float* s_V,
                                                                   const RobotDev& rb, const float4* s_obs,
                                                                   const SceneDev& sc, int lane) {
  constexpr int DP = Var<kVarPoint>::kDp;
  const size_t vi = vidx(g, r, layer, i);
  const bool row_hit = g.vflag[vi] != 0;
  unsigned long long best = kEmptyKey;
  if (!FULL && row_hit) return best;
  const int H = g.H;
  const float steps = static_cast<float>(H - 1);
  float qi[DP];
  load_vertex<DP>(qi, g.Q + vi * g.dp, g.dp);
  for (int jb = j0; jb < j1; jb += 32) {
    const int j = jb + lane;
    unsigned long long key = kEmptyKey;
    if (j < j1) {
      const float Vj = s_V[j];
      float qj[DP];
      load_vertex<DP>(qj, g.Q + vidx(g, r, layer + 1, j) * g.dp, g.dp);
      float dq[DP];
      float s2 = 0.0f;
#pragma unroll
      for (int d = 0; d < DP; ++d) {
        dq[d] = __fsub_rn(qj[d], qi[d]);
        s2 = __fmaf_rn(dq[d], dq[d], s2);
      }
      const float len = __fsqrt_rn(s2);
      const bool skip = !(Vj < kInf) || len > g.max_edge_len || row_hit ||
                        (g.prune && g.prune[static_cast<size_t>(i) * layer_size(g, layer + 1) + j]);
      bool hit = false;
      if (FULL || !skip) {
        for (int k = 1; k <= H - 2; ++k) {
          const float t = __fdiv_rn(static_cast<float>(k), steps);
          float q[DP];
#pragma unroll
          for (int d = 0; d < DP; ++d) q[d] = __fmaf_rn(t, dq[d], qi[d]);
          hit |= point_config_collides<false>(q, true, rb, s_obs, sc.n_s, s_obs + sc.n_s, sc.n_b);
          if (!FULL && hit) break;
        }
      }
      if (!hit && !skip) {
        float cost = len;
        if constexpr (WEIGHTED) cost = weighted_cost_thread<DP>(qi, qj, len, g);
        key = make_key(__fadd_rn(cost, Vj), static_cast<uint32_t>(j));
      }
    }
    key = warp_min_u64(key);
    best = key < best ? key : best;
  }
  return best;
}

template <int VAR, bool FULL, bool WEIGHTED = false>
__device__ __forceinline__ unsigned long long row_chunk_best(const GraphDev& g, int r, int layer, int i, int j0,
                                                             int j1, const float* s_V, const RobotDev& rb,
                                                             const float4* s_obs, const SceneDev& sc, int lane) {
  if constexpr (VAR == kVarPoint) {
    return point_row_chunk_best<FULL, WEIGHTED>(g, r, layer, i, j0, j1, s_V, rb, s_obs, sc, lane);
  }
  using V = Var<VAR>;
  constexpr int DP = V::kDp;
  const size_t vi = vidx(g, r, layer, i);
  const bool row_hit = g.vflag[vi] != 0;
  unsigned long long best = kEmptyKey;
  if (!FULL && row_hit) return best;
  const int H = g.H;
  const float steps = static_cast<float>(H - 1);
  float qi[DP];
  load_vertex<DP>(qi, g.Q + vi * g.dp, g.dp);
  const int n_cols = layer_size(g, layer + 1);
  if constexpr (FULL) {
    // Full evaluation has no early exit, so the warp need not stay on one
    // edge: the (edge, waypoint) items of up to 32 columns are dealt to the
    // lanes in order (no lane idles when H - 2 is not a multiple of 32), each
    // lane's label is OR-ed into its edge's bit, then lane e keys edge e.
    const int nw = H - 2;
    for (int jb = j0; jb < j1; jb += 32) {
      const int n_edges = min(32, j1 - jb);
      const int n_items = n_edges * nw;
      unsigned hit_mask = 0u;
      for (int t0 = 0; t0 < n_items; t0 += 32) {
        const int t = t0 + lane;
        const bool active = t < n_items;
        const int e = active ? t / nw : 0;
        const int k = active ? t - e * nw + 1 : 1;
        float qj[DP];
        load_vertex<DP>(qj, g.Q + vidx(g, r, layer + 1, jb + e) * g.dp, g.dp);
        const float tt = __fdiv_rn(static_cast<float>(k), steps);
        float q[DP];
#pragma unroll
        for (int d = 0; d < DP; ++d) q[d] = __fmaf_rn(tt, __fsub_rn(qj[d], qi[d]), qi[d]);
        const bool h = config_collides<VAR, false, true>(q, active, rb, s_obs, sc) && active;
        hit_mask |= __reduce_or_sync(kFull, h ? (1u << e) : 0u);
      }
      unsigned long long key = kEmptyKey;
      if (lane < n_edges) {
        const int j = jb + lane;
        const float Vj = s_V[j];
        float qj[DP];
        load_vertex<DP>(qj, g.Q + vidx(g, r, layer + 1, j) * g.dp, g.dp);
        float s2 = 0.0f;
#pragma unroll
        for (int d = 0; d < DP; ++d) {
          const float e = __fsub_rn(qj[d], qi[d]);
          s2 = __fmaf_rn(e, e, s2);
        }
        const float len = __fsqrt_rn(s2);
        const bool pruned = g.prune && g.prune[static_cast<size_t>(i) * n_cols + j];
        if (!((hit_mask >> lane) & 1u) && !(len > g.max_edge_len) && !row_hit && Vj < kInf && !pruned) {
          float cost = len;
          if constexpr (WEIGHTED) cost = weighted_cost_thread<DP>(qi, qj, len, g);
          key = make_key(__fadd_rn(cost, Vj), static_cast<uint32_t>(j));
        }
      }
      key = warp_min_u64(key);
      best = key < best ? key : best;
    }
    return best;
  } else {
    // early exit: the warp's lanes carry the interior waypoints of one edge
    for (int j = j0; j < j1; ++j) {
      const float Vj = s_V[j];
      if (!(Vj < kInf)) continue;
      if (g.prune && g.prune[static_cast<size_t>(i) * n_cols + j]) continue;  // dropped by the surrogate
      float qj[DP];
      load_vertex<DP>(qj, g.Q + vidx(g, r, layer + 1, j) * g.dp, g.dp);
      float dq[DP];
      float s2 = 0.0f;
#pragma unroll
      for (int d = 0; d < DP; ++d) {
        dq[d] = __fsub_rn(qj[d], qi[d]);
        s2 = __fmaf_rn(dq[d], dq[d], s2);
      }
      const float len = __fsqrt_rn(s2);
      if (len > g.max_edge_len) continue;
      bool hit = false;
      for (int kb = 1; kb <= H - 2; kb += 32) {
        const int k = kb + lane;
        const bool active = k <= H - 2;
        const float t = __fdiv_rn(static_cast<float>(k), steps);
        float q[DP];
#pragma unroll
        for (int d = 0; d < DP; ++d) q[d] = __fmaf_rn(t, dq[d], qi[d]);
        hit |= config_collides<VAR, true, false>(q, active, rb, s_obs, sc);
        if (hit) break;
      }
      if (!hit) {
        float cost = len;
        if constexpr (WEIGHTED)
          cost = weighted_cost_warp<DP>(qi, g.Q + vidx(g, r, layer + 1, j) * g.dp, g.dp, dq, len, g, lane);
        const unsigned long long key = make_key(__fadd_rn(cost, Vj), static_cast<uint32_t>(j));
        best = key < best ? key : best;
      }
    }
    return best;
  }
}

// ---------------------------------------------------------------------------
// Lazy realisation (exact).  The best key of row i is the smallest
// (c(i,j) + J_{l+1}(j), j) over realised edges; an edge whose key is not below
// a key already found for the row cannot change the row's minimum, so it is
// never checked.  The unit of work is one block of (up to) 32 columns
// [j0, min(j0 + 32, j_end)) of one row:
// the warp scores the block's candidates (lane = column), drops those at or
// above the row's current best (the row's key word in global memory, which
// every unit of the row lowers with atomicMin), sorts the rest (bitonic,
// 64-bit keys, one per lane) and checks them in ascending order, re-reading
// the row's best before each check, until the first free edge (published at
// once) or the first key at or above the best.  Units are handed out block-
// major (block 0 of every row, then block 1, ...), so later blocks of a row
// usually start with a bound from its earlier ones.  The final key word is
// the one the exhaustive modes compute, bit for bit: the row's minimal free
// edge is skipped only if its own key has already been published.
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned long long warp_sort32_u64(unsigned long long key, int lane) {
#pragma unroll
  for (int k = 2; k <= 32; k <<= 1) {
#pragma unroll
    for (int j = k >> 1; j > 0; j >>= 1) {
      const unsigned long long other = __shfl_xor_sync(kFull, key, j);
      const bool up = (lane & k) == 0;
      const bool low = (lane & j) == 0;
      key = (low == up) ? (other < key ? other : key) : (other > key ? other : key);
    }
  }
  return key;
}

template <int VAR, bool WEIGHTED = false>
__device__ __forceinline__ void lazy_block(const GraphDev& g, int r, int layer, int i, int j0, int j_end,
                                           const float* s_V, const RobotDev& rb, const float4* s_obs,
                                           const SceneDev& sc, int lane) {
  using V = Var<VAR>;
  constexpr int DP = V::kDp;
  const size_t vi = vidx(g, r, layer, i);
  if (g.vflag[vi] != 0) return;
  unsigned long long* row_key = g.keys + vi;
  unsigned long long bound = __ldcg(row_key);
  const int H = g.H;
  const float steps = static_cast<float>(H - 1);
  const int n_cols = layer_size(g, layer + 1);
  float qi[DP];
  load_vertex<DP>(qi, g.Q + vi * g.dp, g.dp);
  const int jl = j0 + lane;
  unsigned long long key = kEmptyKey;
  if (jl < j_end) {
    const float Vj = s_V[jl];
    if (Vj < kInf && !(g.prune && g.prune[static_cast<size_t>(i) * n_cols + jl])) {
      float qj[DP];
      load_vertex<DP>(qj, g.Q + vidx(g, r, layer + 1, jl) * g.dp, g.dp);
      float s2 = 0.0f;
#pragma unroll
      for (int d = 0; d < DP; ++d) {
        const float e = __fsub_rn(qj[d], qi[d]);
        s2 = __fmaf_rn(e, e, s2);
      }
      const float len = __fsqrt_rn(s2);
      if (!(len > g.max_edge_len)) {
        float cost = len;
        if constexpr (WEIGHTED) cost = weighted_cost_thread<DP>(qi, qj, len, g);
        key = make_key(__fadd_rn(cost, Vj), static_cast<uint32_t>(jl));
      }
    }
  }
  if (key >= bound) key = kEmptyKey;
  const unsigned live = __ballot_sync(kFull, key != kEmptyKey);
  if (live == 0) return;
  if (live & (live - 1)) key = warp_sort32_u64(key, lane);
  else key = __shfl_sync(kFull, key, __ffs(live) - 1);  // a single candidate: move it to slot 0
  const int n_live = __popc(live);
  for (int t = 0; t < n_live; ++t) {
    const unsigned long long kt = __shfl_sync(kFull, key, t);
    if (t > 0) {
      unsigned long long b = 0;
      if (lane == 0) b = __ldcg(row_key);
      b = __shfl_sync(kFull, b, 0);
      bound = b < bound ? b : bound;
    }
    if (kt >= bound) break;
    const int j = static_cast<int>(static_cast<uint32_t>(kt));
    float qj[DP];
    load_vertex<DP>(qj, g.Q + vidx(g, r, layer + 1, j) * g.dp, g.dp);
    float dq[DP];
#pragma unroll
    for (int d = 0; d < DP; ++d) dq[d] = __fsub_rn(qj[d], qi[d]);
    bool hit = false;
    if constexpr (VAR == kVarPoint) {
      // lanes take waypoints here as well
      for (int kb = 1; kb <= H - 2 && !hit; kb += 32) {
        const int k = kb + lane;
        const float tt = __fdiv_rn(static_cast<float>(k), steps);
        float q[DP];
#pragma unroll
        for (int d = 0; d < DP; ++d) q[d] = __fmaf_rn(tt, dq[d], qi[d]);
        hit = point_config_collides<true>(q, k <= H - 2, rb, s_obs, sc.n_s, s_obs + sc.n_s, sc.n_b);
      }
    } else {
      for (int kb = 1; kb <= H - 2; kb += 32) {
        const int k = kb + lane;
        const float tt = __fdiv_rn(static_cast<float>(k), steps);
        float q[DP];
#pragma unroll
        for (int d = 0; d < DP; ++d) q[d] = __fmaf_rn(tt, dq[d], qi[d]);
        hit |= config_collides<VAR, true, false>(q, k <= H - 2, rb, s_obs, sc);
        if (hit) break;
      }
    }
    if (!hit) {
      // the smallest remaining key of the block is free: nothing later in it can win
      if (lane == 0) atomicMin(row_key, kt);
      return;
    }
  }
}

}  // namespace
}  // namespace gtmp
