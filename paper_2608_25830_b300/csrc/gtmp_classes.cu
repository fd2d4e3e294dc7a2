// Class-augmented value iteration for planar point robots (Prop. 1; the
// class-indexed archive of Alg. 1 anytime-gtmp).
//
// Label of a start-to-goal chain: the winding numbers of the closed loop
// (chain, then the straight segment qg -> q0) about every obstacle's centre,
// a homology invariant like the h-signature.  It is additive over edges: edge
// (u, v) contributes the winding numbers of the triangle u -> v -> qg -> u,
// 0 or +-1 per obstacle, because the triangles' extra sides cancel in pairs.
// The triangle test uses orientation predicates in float64, which are exact
// for float32 coordinates (exact differences and products, one correctly
// rounded subtraction), so every side agrees on every label bit for bit.
//
//   J_{L+1}(qg, 0) = 0,
//   J_l(u, chi) = min over (v, chi') with kappa(u, v) + chi' = chi of c(u, v) + J_{l+1}(v, chi').
//
// A label is 16 signed bytes (one per obstacle, at most 16 obstacles); the
// entries of a chain of L + 1 edges stay within [-L, L].  Each vertex keeps a
// list of (label, key) pairs, key = bits(cost) << 32 | v << 16 | slot (the
// successor vertex and its list slot), so one 64-bit minimum keeps the least
// cost and, among equal costs, the lowest successor index.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <vector>

#include "gtmp_ctx.h"

using namespace gtmp;

namespace gtmp_classes_impl {

constexpr int kMaxClassObstacles = 16;
constexpr int kClassThreads = 256;
constexpr int kErrLabelTable = 4;           // a vertex had more labels than the table holds
constexpr long long kPublishSpin = 1 << 22;  // bounded wait for a slot's label to be published

struct Centres {
  double x[kMaxClassObstacles], y[kMaxClassObstacles];
  int n;
};

// per-layer arrays of the class tables: entries of vertex i of layer l at
// (l * M_stride + i) * K
struct ClassTables {
  uint4* lab;
  unsigned long long* key;
  int* count;
  int K;
};

__device__ __forceinline__ double orient2d(double ax, double ay, double bx, double by, double cx, double cy) {
  return __dsub_rn(__dmul_rn(__dsub_rn(bx, ax), __dsub_rn(cy, ay)), __dmul_rn(__dsub_rn(by, ay), __dsub_rn(cx, ax)));
}

// winding number of the triangle a -> b -> c -> a about p: the sign of its
// orientation when p lies strictly inside, else 0
__device__ __forceinline__ int triangle_winding(double ax, double ay, double bx, double by, double cx, double cy,
                                                double px, double py) {
  const double o = orient2d(ax, ay, bx, by, cx, cy);
  if (o == 0.0) return 0;
  const double d1 = orient2d(ax, ay, bx, by, px, py);
  const double d2 = orient2d(bx, by, cx, cy, px, py);
  const double d3 = orient2d(cx, cy, ax, ay, px, py);
  if (o > 0.0 && d1 > 0.0 && d2 > 0.0 && d3 > 0.0) return 1;
  if (o < 0.0 && d1 < 0.0 && d2 < 0.0 && d3 < 0.0) return -1;
  return 0;
}

__device__ __forceinline__ uint4 label_add(uint4 a, uint4 b) {
  return make_uint4(__vadd4(a.x, b.x), __vadd4(a.y, b.y), __vadd4(a.z, b.z), __vadd4(a.w, b.w));
}

__device__ __forceinline__ bool label_eq(uint4 a, uint4 b) {
  return a.x == b.x && a.y == b.y && a.z == b.z && a.w == b.w;
}

__device__ __forceinline__ uint32_t label_hash(uint4 a) {
  uint32_t h = a.x * 0x9E3779B1u;
  h ^= a.y + 0x7F4A7C15u + (h << 6) + (h >> 2);
  h ^= a.z + 0x85EBCA77u + (h << 6) + (h >> 2);
  h ^= a.w + 0xC2B2AE3Du + (h << 6) + (h >> 2);
  return h ^ (h >> 15);
}

__global__ void class_init_kernel(GraphDev g, ClassTables t) {
  const long long n = static_cast<long long>(g.L + 2) * g.M_stride;
  for (long long k = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x; k < n;
       k += static_cast<long long>(gridDim.x) * blockDim.x)
    t.count[k] = 0;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    // the goal: the empty label at cost 0, no successor
    const size_t gi = static_cast<size_t>(g.L + 1) * g.M_stride;
    t.count[gi] = 1;
    t.lab[gi * t.K] = make_uint4(0, 0, 0, 0);
    t.key[gi * t.K] = make_key(0.0f, 0xffffffffu);
  }
}

// Insert (chi, key) into the block's open-addressing table: the slot of chi
// keeps the minimum key.  A slot is claimed (state 1), its label written, then
// published (state 2); others wait (bounded) for the publication before
// comparing labels.  Returns false when the table is full or a wait ran out.
__device__ bool table_insert(uint4 chi, unsigned long long key, uint4* s_lab, unsigned long long* s_key, int* s_state,
                             int K) {
  uint32_t h = label_hash(chi) & static_cast<uint32_t>(K - 1);
  for (int probe = 0; probe < K; ++probe) {
    const int st = atomicCAS(&s_state[h], 0, 1);
    if (st == 0) {
      s_lab[h] = chi;
      __threadfence_block();
      atomicExch(&s_state[h], 2);
      atomicMin(&s_key[h], key);
      return true;
    }
    long long spins = 0;
    while (*reinterpret_cast<volatile int*>(&s_state[h]) != 2) {
      if (++spins > kPublishSpin) return false;
    }
    __threadfence_block();
    const volatile uint4* vl = reinterpret_cast<const volatile uint4*>(&s_lab[h]);
    const uint4 here = make_uint4(vl->x, vl->y, vl->z, vl->w);
    if (label_eq(here, chi)) {
      atomicMin(&s_key[h], key);
      return true;
    }
    h = (h + 1) & static_cast<uint32_t>(K - 1);
  }
  return false;
}

// One CTA per vertex u of `layer`: all (label, key) pairs of u from the free
// edges to layer + 1 and the label lists there.  Dynamic shared memory: K
// labels (16 B), K keys (8 B), K states (4 B).
__global__ void __launch_bounds__(kClassThreads) class_sweep_kernel(GraphDev g, int layer, const float* __restrict__ C,
                                                                    int cs, Centres ctr, ClassTables t, int* err) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int K = t.K;
  uint4* s_lab = reinterpret_cast<uint4*>(smem);
  unsigned long long* s_key = reinterpret_cast<unsigned long long*>(smem + static_cast<size_t>(K) * 16);
  int* s_state = reinterpret_cast<int*>(smem + static_cast<size_t>(K) * 24);
  __shared__ int s_count, s_fail;
  const int u = blockIdx.x;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int k = threadIdx.x; k < K; k += blockDim.x) {
    s_state[k] = 0;
    s_key[k] = kEmptyKey;
  }
  if (threadIdx.x == 0) {
    s_count = 0;
    s_fail = 0;
  }
  __syncthreads();
  const size_t vu = vidx(g, 0, layer, u);
  const int n_cols = layer_size(g, layer + 1);
  if (g.vflag[vu] == 0) {
    const float* qu = g.Q + vu * g.dp;
    const float* qg = g.Q + vidx(g, 0, g.L + 1, 0) * g.dp;
    const double ux = qu[0], uy = qu[1], gx = qg[0], gy = qg[1];
    for (int v = warp; v < n_cols; v += kClassThreads / 32) {
      const float c_uv = C[static_cast<size_t>(u) * cs + v];
      if (!(c_uv < __int_as_float(0x7f800000))) continue;  // +inf = no edge
      const size_t vv = vidx(g, 0, layer + 1, v);
      const int n_v = t.count[vv];
      if (n_v == 0) continue;
      // kappa(u, v): lane o computes obstacle o, the warp packs the 16 bytes
      const float* qv = g.Q + vv * g.dp;
      int w = 0;
      if (lane < ctr.n) w = triangle_winding(ux, uy, double(qv[0]), double(qv[1]), gx, gy, ctr.x[lane], ctr.y[lane]);
      uint32_t words[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        uint32_t word = 0;
#pragma unroll
        for (int b = 0; b < 4; ++b) word |= (static_cast<uint32_t>(__shfl_sync(kFull, w, 4 * q + b)) & 0xffu) << (8 * b);
        words[q] = word;
      }
      const uint4 kap = make_uint4(words[0], words[1], words[2], words[3]);
      const uint4* lab_v = t.lab + vv * K;
      const unsigned long long* key_v = t.key + vv * K;
      for (int s = lane; s < n_v; s += 32) {
        const uint4 chi = label_add(kap, lab_v[s]);
        const float cost = __fadd_rn(c_uv, key_value(key_v[s]));
        const unsigned long long key = make_key(cost, (static_cast<uint32_t>(v) << 16) | static_cast<uint32_t>(s));
        if (!table_insert(chi, key, s_lab, s_key, s_state, K)) s_fail = 1;
      }
    }
  }
  __syncthreads();
  // compact the table into the vertex's list
  uint4* lab_u = t.lab + vu * K;
  unsigned long long* key_u = t.key + vu * K;
  for (int k = threadIdx.x; k < K; k += blockDim.x) {
    if (s_state[k] == 2) {
      const int idx = atomicAdd(&s_count, 1);
      lab_u[idx] = s_lab[k];
      key_u[idx] = s_key[k];
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    t.count[vu] = s_count;
    if (s_fail) atomicOr(err, kErrLabelTable);
  }
}

// One thread per label of the start vertex: follow the successors to the goal.
__global__ void class_extract_kernel(GraphDev g, ClassTables t, int max_classes, int32_t* paths, float* costs,
                                     int8_t* labels) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  const size_t v0 = vidx(g, 0, 0, 0);
  const int n = min(t.count[v0], max_classes);
  if (c >= n) return;
  unsigned long long key = t.key[v0 * t.K + c];
  const uint4 lab = t.lab[v0 * t.K + c];
  costs[c] = key_value(key);
  const uint32_t words[4] = {lab.x, lab.y, lab.z, lab.w};
  for (int o = 0; o < kMaxClassObstacles; ++o) labels[static_cast<size_t>(c) * kMaxClassObstacles + o] =
      static_cast<int8_t>((words[o >> 2] >> (8 * (o & 3))) & 0xffu);
  int32_t* out = paths + static_cast<size_t>(c) * g.L;
  for (int l = 1; l <= g.L; ++l) {
    const uint32_t succ = static_cast<uint32_t>(key);
    const int v = static_cast<int>(succ >> 16), slot = static_cast<int>(succ & 0xffffu);
    out[l - 1] = v;
    key = t.key[vidx(g, 0, l, v) * t.K + slot];
  }
}

gtmp_status cfail(gtmp_ctx* c, gtmp_status s, const char* fmt, ...) {
  if (c) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    c->last_error = buf;
  }
  return s;
}

#define CLS_TRY(ctx, expr)                                                                                \
  do {                                                                                                    \
    cudaError_t e_ = (expr);                                                                              \
    if (e_ != cudaSuccess)                                                                                \
      return cfail((ctx), e_ == cudaErrorMemoryAllocation ? GTMP_ERR_OOM : GTMP_ERR_CUDA, "%s: %s", #expr, \
                   cudaGetErrorString(e_));                                                               \
  } while (0)

}  // namespace gtmp_classes_impl

using namespace gtmp_classes_impl;

extern "C" GTMP_API gtmp_status gtmp_solve_classes(gtmp_ctx* c, int32_t max_labels, int32_t max_classes,
                                                   int32_t* dev_paths, float* dev_costs, int8_t* dev_labels,
                                                   int32_t* n_classes) {
  GtmpNvtxRange nvtx_("gtmp_solve_classes");
  if (!c || !dev_paths || !dev_costs || !dev_labels || !n_classes || max_classes < 1 || max_labels < 32 ||
      max_labels > 4096 || (max_labels & (max_labels - 1)) != 0)
    return cfail(c, GTMP_ERR_INVALID_ARG, "bad class request (max_labels a power of two in [32, 4096])");
  if (c->rb.kind != GTMP_ROBOT_POINT || c->dof != 2)
    return cfail(c, GTMP_ERR_UNSUPPORTED, "class labels are defined for planar point robots (dof 2)");
  if (static_cast<int>(c->centres.size()) > kMaxClassObstacles)
    return cfail(c, GTMP_ERR_UNSUPPORTED, "class labels support at most %d obstacles", kMaxClassObstacles);
  if (!c->have_endpoints || c->M_active < 1)
    return cfail(c, GTMP_ERR_NOT_READY, "endpoints or samples missing");
  if (c->G != 1) return cfail(c, GTMP_ERR_UNSUPPORTED, "class labels are defined for a single goal");
  gtmp_status s = gtmp_internal_edge_costs(c);
  if (s != GTMP_OK) return s;
  const int L = c->p.L, K = max_labels;
  const size_t n_vert = static_cast<size_t>(L + 2) * c->p.M;
  const size_t bytes = n_vert * K * (sizeof(uint4) + sizeof(unsigned long long)) + n_vert * sizeof(int);
  if (c->cls_bytes < bytes) {
    cudaFree(c->cls);
    c->cls = nullptr;
    c->cls_bytes = 0;
    CLS_TRY(c, cudaMalloc(&c->cls, bytes));
    c->cls_bytes = bytes;
  }
  ClassTables t;
  t.K = K;
  t.lab = static_cast<uint4*>(c->cls);
  t.key = reinterpret_cast<unsigned long long*>(t.lab + n_vert * K);
  t.count = reinterpret_cast<int*>(t.key + n_vert * K);
  Centres ctr{};
  ctr.n = static_cast<int>(c->centres.size());
  for (int o = 0; o < ctr.n; ++o) {
    ctr.x[o] = c->centres[o].first;
    ctr.y[o] = c->centres[o].second;
  }
  GraphDev g;
  g.Q = c->Q;
  g.vflag = c->vflag;
  g.keys = c->keys;
  g.R = 1;
  g.L = L;
  g.M = c->M_active;
  g.dp = c->dp;
  g.H = c->p.H;
  g.M_stride = c->p.M;
  g.max_edge_len = c->p.max_edge_len;
  cudaStream_t st = c->stream;
  class_init_kernel<<<64, 256, 0, st>>>(g, t);
  CLS_TRY(c, cudaGetLastError());
  const size_t smem = static_cast<size_t>(K) * (16 + 8 + 4);
  CLS_TRY(c, cudaFuncSetAttribute(class_sweep_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  static_cast<int>(smem)));
  for (int layer = L; layer >= 0; --layer) {
    const int rows = layer_size(g, layer);
    class_sweep_kernel<<<rows, kClassThreads, smem, st>>>(g, layer, c->C + c->c_off[layer], c->c_cs[layer], ctr, t,
                                                          c->err);
    CLS_TRY(c, cudaGetLastError());
  }
  const int ext = std::min(max_classes, K);
  class_extract_kernel<<<(ext + 127) / 128, 128, 0, st>>>(g, t, max_classes, dev_paths, dev_costs, dev_labels);
  CLS_TRY(c, cudaGetLastError());
  c->launches += L + 3;
  int count = 0, err = 0;
  CLS_TRY(c, cudaMemcpyAsync(&count, t.count, sizeof(int), cudaMemcpyDeviceToHost, st));
  CLS_TRY(c, cudaMemcpyAsync(&err, c->err, sizeof(int), cudaMemcpyDeviceToHost, st));
  CLS_TRY(c, cudaStreamSynchronize(st));
  if (err & kErrLabelTable) {
    CLS_TRY(c, cudaMemset(c->err, 0, sizeof(int)));
    return cfail(c, GTMP_ERR_OOM, "a vertex has more than max_labels = %d labels", K);
  }
  *n_classes = count;
  return GTMP_OK;
}
