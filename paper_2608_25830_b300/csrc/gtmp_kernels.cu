// Kernels of the layered-graph planner (sm_103a).
//
//   sample_uniform      Alg. 1 "uniformly sample Q" (Philox4x32-10 stream)
//   vertex_labels       C_free membership of every vertex (start, samples, goal)
//   label_configs       the same exact checker on caller-supplied configurations
//   fused_transition    straight-line edge realisation (Sec. VI SEV planner:
//                       H waypoints -> FK -> sphere/box tests) fused with the
//                       min-plus step J_l(u) = min_v c(u,v) + J_{l+1}(v)
//                       (Sec. IV-B); the cost matrix is never stored
//   edge_costs          unfused variant: writes C_l (FP32, +inf = absent)
//   minplus             unfused variant: J_l from a stored C_l (HBM-bound)
//   extract_paths       follow the minimisers from q0 (Alg. 1 path extraction)
//   expand              expand-samples of Alg. 1 (AO-GTMP, Sec. IV-D)
#include <algorithm>
#include <cfloat>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <vector>

#include "gtmp_edge.cuh"

namespace gtmp {

namespace {

// ---------------------------------------------------------------------------
// Uniform layer sampling: thread per (r, layer 1..L, i).  Word k & 3 of
// Philox block (i, layer - 1, restart, TAG_UNIFORM << 24 | k >> 2).
// ---------------------------------------------------------------------------
__global__ void sample_uniform_kernel(GraphDev g, Box16 box, int dof, unsigned long long seed, int restart0) {
  const long long tid = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x;
  const long long total = static_cast<long long>(g.R) * g.L * g.M;
  if (tid >= total) return;
  const int i = static_cast<int>(tid % g.M);
  const int l = static_cast<int>((tid / g.M) % g.L);
  const int r = static_cast<int>(tid / (static_cast<long long>(g.M) * g.L));
  float* out = g.Q + vidx(g, r, l + 1, i) * g.dp;
  const uint2 key = seed_key(seed);
  uint4 w = make_uint4(0, 0, 0, 0);
  for (int k = 0; k < g.dp; ++k) {
    if (k >= dof) {
      out[k] = 0.0f;
      continue;
    }
    if ((k & 3) == 0)
      w = philox4x32_10(make_uint4(static_cast<uint32_t>(i), static_cast<uint32_t>(l),
                                   static_cast<uint32_t>(restart0 + r), (kTagUniform << 24) | (k >> 2)),
                        key);
    const float u = word_to_unit(word_of(w, k));
    out[k] = __fmaf_rn(u, __fsub_rn(box.hi[k], box.lo[k]), box.lo[k]);
  }
}

// ---------------------------------------------------------------------------
// Layer sampling on C_free by rejection (Sec. III: pi_m is a measure on
// C_m and C_free): thread per (r, layer 1..L, i); attempt 0 is the uniform
// sample above, attempt a >= 1 takes word k & 3 of Philox block
// (i, layer - 1, restart, TAG_FREE << 24 | a << 2 | k >> 2); the first
// attempt the exact checker finds free is kept, else the last (its edges then
// collide through their endpoint, as with uniform sampling).
// ---------------------------------------------------------------------------
template <int VAR>
__global__ void __launch_bounds__(kThreads) sample_free_kernel(GraphDev g, RobotDev rb, SceneDev sc, Box16 box,
                                                               int dof, unsigned long long seed, int restart0,
                                                               int max_attempts) {
  extern __shared__ float4 s_obs[];
  stage_obstacles_plain(s_obs, sc.obs, scene_float4s(sc));
  __syncthreads();
  const long long tid = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x;
  const long long total = static_cast<long long>(g.R) * g.L * g.M;
  if (tid >= total) return;
  const int i = static_cast<int>(tid % g.M);
  const int l = static_cast<int>((tid / g.M) % g.L);
  const int r = static_cast<int>(tid / (static_cast<long long>(g.M) * g.L));
  const uint2 key = seed_key(seed);
  constexpr int DP = Var<VAR>::kDp;
  float q[DP];
  for (int a = 0; a < max_attempts; ++a) {
    uint4 w = make_uint4(0, 0, 0, 0);
#pragma unroll
    for (int k = 0; k < DP; ++k) {
      if (k >= dof) {
        q[k] = 0.0f;
        continue;
      }
      if ((k & 3) == 0) {
        const uint32_t word3 = a == 0 ? (kTagUniform << 24) | static_cast<uint32_t>(k >> 2)
                                      : (kTagFree << 24) | (static_cast<uint32_t>(a) << 2) | static_cast<uint32_t>(k >> 2);
        w = philox4x32_10(make_uint4(static_cast<uint32_t>(i), static_cast<uint32_t>(l),
                                     static_cast<uint32_t>(restart0 + r), word3),
                          key);
      }
      q[k] = __fmaf_rn(word_to_unit(word_of(w, k)), __fsub_rn(box.hi[k], box.lo[k]), box.lo[k]);
    }
    if (!config_collides<VAR, false, false>(q, true, rb, s_obs, sc)) break;
  }
  float* out = g.Q + vidx(g, r, l + 1, i) * g.dp;
#pragma unroll
  for (int k = 0; k < DP; ++k) out[k] = q[k];
}

__global__ void init_keys_kernel(GraphDev g, int* counters, int n_counters) {
  const long long tid = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x;
  const long long per_r = static_cast<long long>(g.L + 2) * g.M_stride;
  if (tid < n_counters) counters[tid] = 0;
  if (tid >= per_r * g.R) return;
  const int layer = static_cast<int>((tid % per_r) / g.M_stride);
  const int i = static_cast<int>(tid % g.M_stride);
  // goal vertex i starts at its terminal value V_g[i] (Alg. 1: V_h[M-1] <- min(C_l + V_g))
  g.keys[tid] = (layer == g.L + 1 && i < g.G) ? make_key(g.gval ? g.gval[i] : 0.0f, static_cast<uint32_t>(i))
                                               : kEmptyKey;
}

// ---------------------------------------------------------------------------
// Vertex labels: thread per vertex of every layer (0..L+1).
// ---------------------------------------------------------------------------
template <int VAR>
__global__ void __launch_bounds__(kThreads) vertex_labels_kernel(GraphDev g, RobotDev rb, SceneDev sc) {
  extern __shared__ float4 s_obs[];
  stage_obstacles_plain(s_obs, sc.obs, scene_float4s(sc));
  __syncthreads();
  const long long tid = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x;
  const long long per_r = static_cast<long long>(g.L + 2) * g.M_stride;
  if (tid >= per_r * g.R) return;
  const int r = static_cast<int>(tid / per_r);
  const int layer = static_cast<int>((tid % per_r) / g.M_stride);
  const int i = static_cast<int>(tid % g.M_stride);
  if (i >= layer_size(g, layer)) return;
  constexpr int DP = Var<VAR>::kDp;
  float q[DP];
  load_vertex<DP>(q, g.Q + vidx(g, r, layer, i) * g.dp, g.dp);
  g.vflag[vidx(g, r, layer, i)] = config_collides<VAR, false, false>(q, true, rb, s_obs, sc) ? 1 : 0;
}

template <int VAR>
__global__ void __launch_bounds__(kThreads) label_configs_kernel(const float* q_in, int n, int dof, RobotDev rb,
                                                                 SceneDev sc, uint8_t* out) {
  extern __shared__ float4 s_obs[];
  stage_obstacles_plain(s_obs, sc.obs, scene_float4s(sc));
  __syncthreads();
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n) return;
  constexpr int DP = Var<VAR>::kDp;
  float q[DP];
#pragma unroll
  for (int d = 0; d < DP; ++d) q[d] = d < dof ? q_in[static_cast<size_t>(t) * dof + d] : 0.0f;
  // arms: a coordinate beyond the accepted joint range (or NaN) is labelled colliding
  bool in_range = true;
  if constexpr (VAR != kVarPoint) {
#pragma unroll
    for (int d = 0; d < DP; ++d) in_range = in_range && fabsf(q[d]) <= kMaxJointAngle;
  }
  out[t] = (!in_range || config_collides<VAR, false, false>(q, true, rb, s_obs, sc)) ? 1 : 0;
}

// ---------------------------------------------------------------------------
// Fused edge realisation + min-plus for transition layer -> layer + 1.
//
// grid = (persistent blocks, R).  Each warp repeatedly takes a chunk of edges
// (one row i, up to `chunk` consecutive columns) from the restart's counter;
// the 32 lanes evaluate the H-2 interior waypoints of one edge at a time
// (endpoint labels come from vertex_labels), the warp leaves the edge at the
// first colliding link unless MODE == kEvalFull, and the row's best
// (value, column) key is merged with one 64-bit atomicMin per chunk.
// Shared memory: obstacles (bulk copy) and the column layer's cost-to-go,
// +inf where that vertex collides or reaches no goal.
// ---------------------------------------------------------------------------
template <int VAR, int MODE, bool WEIGHTED>
__global__ void __launch_bounds__(kThreads, kFusedMinBlocks) fused_transition_kernel(GraphDev g, int layer, RobotDev rb, SceneDev sc,
                                                                    int* counters, int chunk, int* err) {
  constexpr bool FULL = MODE == kEvalFull;
  extern __shared__ __align__(128) float4 smem[];
  __shared__ __align__(8) uint64_t mbar;
  const int n4 = scene_float4s(sc);
  float4* s_obs = smem;
  float* s_V = reinterpret_cast<float*>(smem + n4);
  const int r = blockIdx.y;
  const int n_rows = layer_size(g, layer), n_cols = layer_size(g, layer + 1);

  // launched as a programmatic dependent of the previous transition (except the
  // first): the obstacle table stages while that grid finishes, and only the
  // cost-to-go J_{l+1}, its output, waits for it
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  if (!stage_obstacles(s_obs, sc.obs, n4, &mbar, err)) return;  // also a block barrier
  asm volatile("griddepcontrol.wait;" ::: "memory");
  for (int j = threadIdx.x; j < n_cols; j += blockDim.x) {
    const size_t v = vidx(g, r, layer + 1, j);
    s_V[j] = g.vflag[v] ? kInf : key_value(g.keys[v]);
  }
  __syncthreads();

  const int lane = threadIdx.x & 31;
  const int cpr = (n_cols + chunk - 1) / chunk;
  const int n_chunks = n_rows * cpr;
  int* counter = counters + r;
  if constexpr (MODE == kEvalLazy) {
    // units = (32-column block, row), block-major, so a row's later blocks see its earlier results
    const int n_blk = (n_cols + 31) / 32;
    const int n_units = n_rows * n_blk;
    while (true) {
      int c = 0;
      if (lane == 0) c = atomicAdd(counter, 1);
      c = __shfl_sync(kFull, c, 0);
      if (c >= n_units) break;
      const int b = c / n_rows;
      lazy_block<VAR, WEIGHTED>(g, r, layer, c - b * n_rows, b * 32, n_cols, s_V, rb, s_obs, sc, lane);
    }
  } else {
    while (true) {
      int c = 0;
      if (lane == 0) c = atomicAdd(counter, 1);
      c = __shfl_sync(kFull, c, 0);
      if (c >= n_chunks) break;
      const int i = c / cpr;
      const int j0 = (c - i * cpr) * chunk;
      const int j1 = min(j0 + chunk, n_cols);
      const size_t vi = vidx(g, r, layer, i);
      const unsigned long long best =
          row_chunk_best<VAR, FULL, WEIGHTED>(g, r, layer, i, j0, j1, s_V, rb, s_obs, sc, lane);
      if (lane == 0 && best != kEmptyKey) atomicMin(&g.keys[vi], best);
    }
  }
}

// ---------------------------------------------------------------------------
// Unfused variant, step 1: C[i][j] (row stride cs) = ||q_j - q_i|| or +inf.
// ---------------------------------------------------------------------------
template <int VAR, bool WEIGHTED>
__global__ void __launch_bounds__(kThreads, kFusedMinBlocks) edge_costs_kernel(GraphDev g, int layer, RobotDev rb, SceneDev sc,
                                                              float* C, int cs, int* counter, int chunk, int* err) {
  using V = Var<VAR>;
  constexpr int DP = V::kDp;
  extern __shared__ __align__(128) float4 smem[];
  __shared__ __align__(8) uint64_t mbar;
  const int n4 = scene_float4s(sc);
  float4* s_obs = smem;
  if (!stage_obstacles(s_obs, sc.obs, n4, &mbar, err)) return;
  const int r = 0;
  const int n_rows = layer_size(g, layer), n_cols = layer_size(g, layer + 1);
  const int lane = threadIdx.x & 31;
  const int cpr = (n_cols + chunk - 1) / chunk;
  const int n_chunks = n_rows * cpr;
  const int H = g.H;
  while (true) {
    int c = 0;
    if (lane == 0) c = atomicAdd(counter, 1);
    c = __shfl_sync(kFull, c, 0);
    if (c >= n_chunks) break;
    const int i = c / cpr;
    const int j0 = (c - i * cpr) * chunk;
    const int j1 = min(j0 + chunk, n_cols);
    const size_t vi = vidx(g, r, layer, i);
    const bool row_hit = g.vflag[vi] != 0;
    float qi[DP];
    load_vertex<DP>(qi, g.Q + vi * g.dp, g.dp);
    for (int j = j0; j < j1; ++j) {
      const size_t vj = vidx(g, r, layer + 1, j);
      float out = kInf;
      if (!row_hit && !g.vflag[vj]) {
        float qj[DP];
        load_vertex<DP>(qj, g.Q + vj * g.dp, g.dp);
        float dq[DP];
        float s2 = 0.0f;
#pragma unroll
        for (int d = 0; d < DP; ++d) {
          dq[d] = __fsub_rn(qj[d], qi[d]);
          s2 = __fmaf_rn(dq[d], dq[d], s2);
        }
        const float len = __fsqrt_rn(s2);
        if (!(len > g.max_edge_len)) {
          bool hit = false;
          for (int kb = 1; kb <= H - 2; kb += 32) {
            const int k = kb + lane;
            const float t = __fdiv_rn(static_cast<float>(k), static_cast<float>(H - 1));
            float q[DP];
#pragma unroll
            for (int d = 0; d < DP; ++d) q[d] = __fmaf_rn(t, dq[d], qi[d]);
            hit |= config_collides<VAR, true, false>(q, k <= H - 2, rb, s_obs, sc);
            if (hit) break;
          }
          if (!hit) {
            out = len;
            if constexpr (WEIGHTED) out = weighted_cost_warp<DP>(qi, g.Q + vj * g.dp, g.dp, dq, len, g, lane);
          }
        }
      }
      if (lane == 0) C[static_cast<size_t>(i) * cs + j] = out;
    }
  }
}

// ---------------------------------------------------------------------------
// Unfused variant, step 2: one warp per row, J_l(i) = min_j C[i][j] + J_{l+1}(j)
// with first-index ties.  HBM-bound: the row streams through 16-byte
// streaming loads in batches of kMpBatch per lane, and the first batch of the
// warp's first row is issued before J_{l+1} is staged in shared memory, so the
// prologue overlaps the first DRAM round trip.  J_{l+1} is read from shared
// memory as float4 (conflict-free).  Each lane keeps a float minimum and the
// first column reaching it (its columns are visited in increasing order, so a
// strict comparison keeps the first); the warp then reduces (value, index)
// keys, which keeps the smallest index among equal values.
// ---------------------------------------------------------------------------
constexpr int kMpBatch = 8;

__device__ __forceinline__ void minplus_take(const float4 c, const float4 v, int j, float& bv, int& bj) {
  const float x0 = __fadd_rn(c.x, v.x), x1 = __fadd_rn(c.y, v.y), x2 = __fadd_rn(c.z, v.z), x3 = __fadd_rn(c.w, v.w);
  if (x0 < bv) { bv = x0; bj = j; }
  if (x1 < bv) { bv = x1; bj = j + 1; }
  if (x2 < bv) { bv = x2; bj = j + 2; }
  if (x3 < bv) { bv = x3; bj = j + 3; }
}

__device__ __forceinline__ void minplus_load(float4 (&c)[kMpBatch], const float4* row, int q0, int n4) {
#pragma unroll
  for (int k = 0; k < kMpBatch; ++k) {
    const int q = q0 + 32 * k;
    if (q < n4) c[k] = __ldcs(row + q);
  }
}

// Launched as a programmatic dependent of the previous transition's sweep
// (except the first): the next launch may start as soon as this one is
// running, its first row of C (written by kernels that completed before the
// first sweep began) loads while this one finishes, and only the cost-to-go
// J_{l+1} waits for the previous grid (griddepcontrol.wait).
__global__ void __launch_bounds__(kThreads) minplus_kernel(GraphDev g, int layer, const float* __restrict__ C, int cs) {
  extern __shared__ __align__(16) float s_Vm[];
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  const int n_rows = layer_size(g, layer), n_cols = layer_size(g, layer + 1);
  const int lane = threadIdx.x & 31;
  const int warps_total = gridDim.x * kWarps;
  const int n4 = cs / 4;
  int i = blockIdx.x * kWarps + (threadIdx.x >> 5);
  float4 c[kMpBatch];
  if (i < n_rows) minplus_load(c, reinterpret_cast<const float4*>(C + static_cast<size_t>(i) * cs), lane, n4);
  asm volatile("griddepcontrol.wait;" ::: "memory");  // J_{l+1} is the previous sweep's output
  // stage J_{l+1}: all of a thread's key loads are issued before the first is used
  constexpr int kFill = 8;
  const unsigned long long* knext = g.keys + vidx(g, 0, layer + 1, 0);
  for (int j0 = threadIdx.x; j0 < cs; j0 += kThreads * kFill) {
    float v[kFill];
#pragma unroll
    for (int u = 0; u < kFill; ++u) {
      const int j = j0 + u * kThreads;
      v[u] = j < n_cols ? key_value(__ldcg(knext + j)) : kInf;
    }
#pragma unroll
    for (int u = 0; u < kFill; ++u) {
      const int j = j0 + u * kThreads;
      if (j < cs) s_Vm[j] = v[u];
    }
  }
  __syncthreads();
  const float4* s_V4 = reinterpret_cast<const float4*>(s_Vm);
  for (; i < n_rows; i += warps_total) {
    const float4* row = reinterpret_cast<const float4*>(C + static_cast<size_t>(i) * cs);
    float bv = kInf;
    int bj = 0;
    for (int q0 = lane; q0 < n4; q0 += 32 * kMpBatch) {
      if (q0 != lane) minplus_load(c, row, q0, n4);
#pragma unroll
      for (int k = 0; k < kMpBatch; ++k) {
        const int q = q0 + 32 * k;
        if (q < n4) minplus_take(c[k], s_V4[q], 4 * q, bv, bj);
      }
    }
    unsigned long long best = bv < kInf ? make_key(bv, static_cast<uint32_t>(bj)) : kEmptyKey;
    best = warp_min_u64(best);
    if (lane == 0) g.keys[vidx(g, 0, layer, i)] = best;
    // first batch of the next row
    if (i + warps_total < n_rows)
      minplus_load(c, reinterpret_cast<const float4*>(C + static_cast<size_t>(i + warps_total) * cs), lane, n4);
  }
}

// ---------------------------------------------------------------------------
// Path extraction (one thread per restart) and best-restart selection.
// ---------------------------------------------------------------------------
__global__ void extract_paths_kernel(GraphDev g, int32_t* path, float* cost, int32_t* best) {
  __shared__ unsigned long long s_best;
  if (threadIdx.x == 0) s_best = kEmptyKey;
  __syncthreads();
  for (int r = threadIdx.x; r < g.R; r += blockDim.x) {
    const unsigned long long k0 = g.keys[vidx(g, r, 0, 0)];
    int32_t* p = path + static_cast<size_t>(r) * g.L;
    if (k0 == kEmptyKey) {
      for (int l = 0; l < g.L; ++l) p[l] = -1;
      cost[r] = kInf;
      continue;
    }
    cost[r] = key_value(k0);
    int i = key_index(k0);
    for (int l = 1; l <= g.L; ++l) {
      p[l - 1] = i;
      if (l < g.L) i = key_index(g.keys[vidx(g, r, l, i)]);
    }
    atomicMin(&s_best, (static_cast<unsigned long long>(__float_as_uint(key_value(k0))) << 32) | r);
  }
  __syncthreads();
  if (threadIdx.x == 0 && best) *best = s_best == kEmptyKey ? -1 : static_cast<int32_t>(s_best & 0xffffffffu);
}

// ---------------------------------------------------------------------------
// Path-level lazy evaluation (a lazy variant of the kind Sec. VII names): the
// min-plus step over optimistic edge costs -- each edge's cost as the exact
// kernels compute it, with no collision check -- leaving out the edges found
// colliding so far, and the exact check of the chain that step returns.
// bad holds a bit per (row, column) of each transition: bit i * M_stride + j
// of transition `layer` at word offset layer * words.
// ---------------------------------------------------------------------------
template <int VAR, bool WEIGHTED>
__global__ void __launch_bounds__(kThreads) optimistic_transition_kernel(GraphDev g, int layer, const uint32_t* bad,
                                                                       const int* state) {
  using V = Var<VAR>;
  constexpr int DP = V::kDp;
  // a finished solve, or a transition above the highest one that lost an edge: nothing changes
  if (state[kLazyDone] != 0 || layer > state[kLazyStart]) return;
  const int lane = threadIdx.x & 31;
  const int i = static_cast<int>((static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5);
  if (i >= layer_size(g, layer)) return;
  const size_t vi = vidx(g, 0, layer, i);
  if (g.vflag[vi] != 0) return;
  const int cols = layer_size(g, layer + 1);
  float qi[DP];
  load_vertex<DP>(qi, g.Q + vi * g.dp, g.dp);
  unsigned long long best = kEmptyKey;
  for (int j = lane; j < cols; j += 32) {
    const size_t vj = vidx(g, 0, layer + 1, j);
    if (g.vflag[vj] != 0) continue;
    const unsigned long long kj = __ldcg(g.keys + vj);
    if (kj == kEmptyKey) continue;
    const size_t bit = static_cast<size_t>(i) * g.M_stride + j;
    if ((bad[bit >> 5] >> (bit & 31)) & 1u) continue;
    float qj[DP];
    load_vertex<DP>(qj, g.Q + vj * g.dp, g.dp);
    float s2 = 0.0f;
#pragma unroll
    for (int d = 0; d < DP; ++d) {
      const float e = __fsub_rn(qj[d], qi[d]);
      s2 = __fmaf_rn(e, e, s2);
    }
    const float len = __fsqrt_rn(s2);
    if (len > g.max_edge_len) continue;
    float cost = len;
    if constexpr (WEIGHTED) cost = weighted_cost_thread<DP>(qi, qj, len, g);
    const unsigned long long key = make_key(__fadd_rn(cost, key_value(kj)), static_cast<uint32_t>(j));
    best = key < best ? key : best;
  }
  best = warp_min_u64(best);
  if (lane == 0) g.keys[vi] = best;  // every free row rewritten: a later sweep needs no re-initialisation
}

// The exact check of the chain extract_paths wrote (start, path[0..L-1], the
// goal its last key names): one warp per edge, lanes over the interior
// waypoints as the early-exit kernel takes them; a colliding edge sets its bit
// in bad, counts in state[kLazyFound] and raises state[kLazyHigh] to its
// transition.  An infeasible chain (no start key) is not checked.
template <int VAR>
__global__ void __launch_bounds__(kThreads) check_chain_kernel(GraphDev g, const int32_t* path, RobotDev rb,
                                                               SceneDev sc, uint32_t* bad, size_t words,
                                                               int* state) {
  extern __shared__ __align__(16) float4 s_obs[];
  using V = Var<VAR>;
  constexpr int DP = V::kDp;
  if (state[kLazyDone] != 0 || g.keys[vidx(g, 0, 0, 0)] == kEmptyKey) return;
  stage_obstacles_plain(s_obs, sc.obs, scene_float4s(sc));
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const float steps = static_cast<float>(g.H - 1);
  for (int e = static_cast<int>(threadIdx.x >> 5); e <= g.L; e += static_cast<int>(blockDim.x >> 5)) {
    const int a = e == 0 ? 0 : path[e - 1];
    const int b = e < g.L ? path[e] : key_index(g.keys[vidx(g, 0, g.L, path[g.L - 1])]);
    float qa[DP], qb[DP];
    load_vertex<DP>(qa, g.Q + vidx(g, 0, e, a) * g.dp, g.dp);
    load_vertex<DP>(qb, g.Q + vidx(g, 0, e + 1, b) * g.dp, g.dp);
    float dq[DP];
#pragma unroll
    for (int d = 0; d < DP; ++d) dq[d] = __fsub_rn(qb[d], qa[d]);
    bool hit = false;
    for (int kb = 1; kb <= g.H - 2 && !hit; kb += 32) {
      const int k = kb + lane;
      const float tt = __fdiv_rn(static_cast<float>(k), steps);
      float q[DP];
#pragma unroll
      for (int d = 0; d < DP; ++d) q[d] = __fmaf_rn(tt, dq[d], qa[d]);
      hit = config_collides<VAR, true, false>(q, k <= g.H - 2, rb, s_obs, sc);
    }
    if (hit && lane == 0) {
      const size_t bit = static_cast<size_t>(a) * g.M_stride + b;
      atomicOr(bad + static_cast<size_t>(e) * words + (bit >> 5), 1u << (bit & 31));
      atomicAdd(state + kLazyFound, 1);
      atomicMax(state + kLazyHigh, e);
    }
  }
}

// one thread: open an iteration's chain check (unless the solve has finished)
__global__ void lazy_iteration_begin_kernel(int* state) {
  if (state[kLazyDone] == 0) {
    state[kLazyFound] = 0;
    state[kLazyHigh] = -1;
  }
}

// one thread: close an iteration: a chain with no colliding edge (or none at
// all) finishes the solve, so does the iteration cap; otherwise the next sweep
// starts at the highest transition that lost an edge
__global__ void lazy_iteration_end_kernel(int* state, int max_iterations) {
  if (state[kLazyDone] != 0) return;
  state[kLazyIters] += 1;
  state[kLazyEdges] += state[kLazyFound];
  if (state[kLazyFound] == 0 || state[kLazyIters] >= max_iterations)
    state[kLazyDone] = 1;
  else
    state[kLazyStart] = state[kLazyHigh];
}

__global__ void get_values_kernel(GraphDev g, float* V, int32_t* sigma) {
  const long long tid = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x;
  const long long per_r = static_cast<long long>(g.L + 2) * g.M;
  if (tid >= per_r * g.R) return;
  const int r = static_cast<int>(tid / per_r);
  const int layer = static_cast<int>((tid % per_r) / g.M);
  const int i = static_cast<int>(tid % g.M);
  if (i >= layer_size(g, layer)) {
    V[tid] = kInf;
    sigma[tid] = -1;
    return;
  }
  const unsigned long long k = g.keys[vidx(g, r, layer, i)];
  V[tid] = key_value(k);
  sigma[tid] = layer == g.L + 1 ? -1 : key_index(k);
}

// copy between caller layout [R][L][M][dof] and internal padded layout
__global__ void pack_layers_kernel(GraphDev g, float* user, int dof, int to_internal) {
  const long long tid = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x;
  const long long total = static_cast<long long>(g.R) * g.L * g.M;
  if (tid >= total) return;
  const int i = static_cast<int>(tid % g.M);
  const int l = static_cast<int>((tid / g.M) % g.L);
  const int r = static_cast<int>(tid / (static_cast<long long>(g.M) * g.L));
  float* in = g.Q + vidx(g, r, l + 1, i) * g.dp;
  float* u = user + static_cast<size_t>(tid) * dof;
  for (int k = 0; k < g.dp; ++k) {
    if (to_internal)
      in[k] = k < dof ? u[k] : 0.0f;
    else if (k < dof)
      u[k] = in[k];
  }
}

// ---------------------------------------------------------------------------
// expand-samples (Alg. 1, AO-GTMP).  Thread per new slot (layer, i), i in
// [M_old, M_new).  The rule (FP32, fixed operation order):
//   c_best = +inf      -> box-uniform from the plain stream (restart 0);
//   coin heads / a neighbour layer empty -> uniform in X_f(c_best) ∩ box by
//                        rejection from [-1,1]^d (attempt a: block
//                        (i, l, a, TAG_INFORMED << 24 | k >> 2));
//   otherwise          -> midpoint of u = layer l-1 sample (word 1 of the coin
//                        block mod |layer l-1|) and its nearest layer l+1
//                        sample (first index on ties).
// Coin = bit 0 of word 0 of block (i, l, 0, TAG_COIN << 24).  All draws see
// only the samples present on entry (indices < M_old).
// ---------------------------------------------------------------------------
struct EllipsoidDev {
  float centre[kMaxDof], axis[kMaxDof];
  float r1, r2;
};

__device__ void informed_params(const float* q0, const float* qg, int dof, float c, EllipsoidDev& e) {
  float s = 0.0f;
  for (int k = 0; k < dof; ++k) {
    const float dq = __fsub_rn(qg[k], q0[k]);
    s = __fmaf_rn(dq, dq, s);
  }
  const float cmin = __fsqrt_rn(s);
  for (int k = 0; k < dof; ++k) {
    e.centre[k] = __fmul_rn(0.5f, __fadd_rn(q0[k], qg[k]));
    e.axis[k] = cmin > 0.0f ? __fdiv_rn(__fsub_rn(qg[k], q0[k]), cmin) : (k == 0 ? 1.0f : 0.0f);
  }
  e.r1 = __fmul_rn(0.5f, c);
  float diff = __fsub_rn(__fmul_rn(c, c), __fmul_rn(cmin, cmin));
  if (diff < 0.0f) diff = 0.0f;
  e.r2 = __fmul_rn(0.5f, __fsqrt_rn(diff));
}

__global__ void expand_kernel(GraphDev g, int dof, Box16 box, unsigned long long seed, int M_old, int M_new,
                              const float* c_best_ptr, int max_attempts, int* err) {
  const int n_new = M_new - M_old;
  const long long tid = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (tid >= static_cast<long long>(g.L) * n_new) return;
  const int l = static_cast<int>(tid / n_new);  // 0-based sample layer (internal layer l + 1)
  const int i = M_old + static_cast<int>(tid % n_new);
  const uint2 key = seed_key(seed);
  float* x = g.Q + vidx(g, 0, l + 1, i) * g.dp;
  for (int k = dof; k < g.dp; ++k) x[k] = 0.0f;
  const float c_best = *c_best_ptr;
  if (!(c_best < kInf)) {
    uint4 w = make_uint4(0, 0, 0, 0);
    for (int k = 0; k < dof; ++k) {
      if ((k & 3) == 0)
        w = philox4x32_10(make_uint4(i, l, 0u, (kTagUniform << 24) | (k >> 2)), key);
      x[k] = __fmaf_rn(word_to_unit(word_of(w, k)), __fsub_rn(box.hi[k], box.lo[k]), box.lo[k]);
    }
    return;
  }
  const uint4 coin = philox4x32_10(make_uint4(i, l, 0u, kTagCoin << 24), key);
  const bool heuristic = (coin.x & 1u) != 0u;
  const int n_prev = l == 0 ? 1 : M_old;
  const int n_next = l == g.L - 1 ? 1 : M_old;
  const float* q0 = g.Q + vidx(g, 0, 0, 0) * g.dp;
  const float* qg = g.Q + vidx(g, 0, g.L + 1, 0) * g.dp;
  if (!heuristic || n_prev == 0 || n_next == 0) {
    EllipsoidDev e;
    informed_params(q0, qg, dof, c_best, e);
    const float rdiff = __fsub_rn(e.r1, e.r2);
    for (int a = 0; a < max_attempts; ++a) {
      float z[kMaxDof];
      uint4 w = make_uint4(0, 0, 0, 0);
      for (int k = 0; k < dof; ++k) {
        if ((k & 3) == 0)
          w = philox4x32_10(make_uint4(i, l, static_cast<uint32_t>(a), (kTagInformed << 24) | (k >> 2)), key);
        z[k] = __fsub_rn(__fmul_rn(2.0f, word_to_unit(word_of(w, k))), 1.0f);
      }
      float ss = 0.0f;
      for (int k = 0; k < dof; ++k) ss = __fmaf_rn(z[k], z[k], ss);
      if (!(ss <= 1.0f)) continue;
      float dot = 0.0f;
      for (int k = 0; k < dof; ++k) dot = __fmaf_rn(e.axis[k], z[k], dot);
      const float coef = __fmul_rn(rdiff, dot);
      bool inside = true;
      float y[kMaxDof];
      for (int k = 0; k < dof; ++k) {
        y[k] = __fmaf_rn(coef, e.axis[k], __fmaf_rn(e.r2, z[k], e.centre[k]));
        inside = inside && (y[k] >= box.lo[k] && y[k] <= box.hi[k]);
      }
      if (inside) {
        for (int k = 0; k < dof; ++k) x[k] = y[k];
        return;
      }
    }
    atomicOr(err, kErrSamplerExhausted);
    for (int k = 0; k < dof; ++k) x[k] = __int_as_float(0x7fc00000);
    return;
  }
  const uint32_t pick = coin.y % static_cast<uint32_t>(n_prev);
  const float* u = l == 0 ? q0 : g.Q + vidx(g, 0, l, pick) * g.dp;
  const float* v = qg;
  if (l != g.L - 1) {
    float best = kInf;
    int bi = 0;
    for (int j = 0; j < n_next; ++j) {
      const float* c = g.Q + vidx(g, 0, l + 2, j) * g.dp;
      float d2 = 0.0f;
      for (int k = 0; k < dof; ++k) {
        const float dd = __fsub_rn(c[k], u[k]);
        d2 = __fmaf_rn(dd, dd, d2);
      }
      if (d2 < best) {
        best = d2;
        bi = j;
      }
    }
    v = g.Q + vidx(g, 0, l + 2, bi) * g.dp;
  }
  for (int k = 0; k < dof; ++k) x[k] = __fmul_rn(0.5f, __fadd_rn(u[k], v[k]));
}

__global__ void update_best_kernel(int L, const int32_t* cand_path, const float* cand_cost, int32_t* best_path,
                                   float* best_cost) {
  const float c = *cand_cost;
  const float b = *best_cost;
  __syncthreads();
  if (c < b) {
    for (int l = threadIdx.x; l < L; l += blockDim.x) best_path[l] = cand_path[l];
    __syncthreads();
    if (threadIdx.x == 0) *best_cost = c;
  }
}

// The chain q0, Q[1][path[0]], ..., Q[L][path[L-1]], qg of graph 0 as
// configurations: chain[row][dof], rows = L_cap + 2, rows past qg (and any
// row of an infeasible path) NaN.
__global__ void gather_chain_kernel(GraphDev g, const int32_t* path, float* chain, int dof, int rows) {
  const int row = blockIdx.x, k = threadIdx.x;
  if (row >= rows || k >= dof) return;
  float v = __int_as_float(0x7fc00000);
  if (row == 0) {
    v = g.Q[vidx(g, 0, 0, 0) * g.dp + k];
  } else if (row <= g.L) {
    const int i = path[row - 1];
    if (i >= 0 && i < g.M) v = g.Q[vidx(g, 0, row, i) * g.dp + k];
  } else if (row == g.L + 1) {
    v = g.Q[vidx(g, 0, g.L + 1, 0) * g.dp + k];
  }
  chain[static_cast<size_t>(row) * dof + k] = v;
}

inline int blocks_for(long long n, int threads) { return static_cast<int>((n + threads - 1) / threads); }

Box16 make_box(const float* lo, const float* hi, int dof) {
  Box16 b{};
  for (int k = 0; k < dof; ++k) {
    b.lo[k] = lo[k];
    b.hi[k] = hi[k];
  }
  return b;
}

template <int VAR, int MODE>
cudaError_t fused_dispatch_mode(const GraphDev& g, int layer, const RobotDev& rb, const SceneDev& sc, int* counters,
                                int grid_x, int chunk, int* err, bool dependent, cudaStream_t st) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid_x, g.R);
  cfg.blockDim = dim3(kThreads);
  cfg.dynamicSmemBytes = static_cast<size_t>(scene_float4s(sc)) * 16 + static_cast<size_t>(g.M_stride) * 4;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = dependent ? 1 : 0;
  if (g.n_wb > 0)
    return cudaLaunchKernelEx(&cfg, fused_transition_kernel<VAR, MODE, true>, g, layer, rb, sc, counters, chunk, err);
  return cudaLaunchKernelEx(&cfg, fused_transition_kernel<VAR, MODE, false>, g, layer, rb, sc, counters, chunk, err);
}

template <int VAR>
cudaError_t fused_dispatch(const GraphDev& g, int layer, const RobotDev& rb, const SceneDev& sc, int mode,
                           int* counters, int grid_x, int chunk, int* err, bool dependent, cudaStream_t st) {
  if (mode == kEvalFull)
    return fused_dispatch_mode<VAR, kEvalFull>(g, layer, rb, sc, counters, grid_x, chunk, err, dependent, st);
  if (mode == kEvalLazy)
    return fused_dispatch_mode<VAR, kEvalLazy>(g, layer, rb, sc, counters, grid_x, chunk, err, dependent, st);
  return fused_dispatch_mode<VAR, kEvalEarlyExit>(g, layer, rb, sc, counters, grid_x, chunk, err, dependent, st);
}

template <template <int> class F, typename... Args>
cudaError_t by_variant(int variant, Args&&... args) {
  switch (variant) {
    case kVarPoint: return F<kVarPoint>::run(args...);
    case kVarArm6x4: return F<kVarArm6x4>::run(args...);
    case kVarArm7x4: return F<kVarArm7x4>::run(args...);
    default: return F<kVarArmGeneric>::run(args...);
  }
}

template <int VAR>
struct SampleFreeRun {
  static cudaError_t run(const GraphDev& g, const RobotDev& rb, const SceneDev& sc, const Box16& box, int dof,
                         unsigned long long seed, int restart0, int max_attempts, cudaStream_t st) {
    const long long n = static_cast<long long>(g.R) * g.L * g.M;
    if (n == 0) return cudaSuccess;
    const size_t smem = static_cast<size_t>(scene_float4s(sc)) * 16;
    sample_free_kernel<VAR><<<blocks_for(n, kThreads), kThreads, smem, st>>>(g, rb, sc, box, dof, seed, restart0,
                                                                             max_attempts);
    return cudaGetLastError();
  }
};

template <int VAR>
struct VertexLabelsRun {
  static cudaError_t run(const GraphDev& g, const RobotDev& rb, const SceneDev& sc, cudaStream_t st) {
    const long long n = static_cast<long long>(g.R) * (g.L + 2) * g.M_stride;
    const size_t smem = static_cast<size_t>(scene_float4s(sc)) * 16;
    vertex_labels_kernel<VAR><<<blocks_for(n, kThreads), kThreads, smem, st>>>(g, rb, sc);
    return cudaGetLastError();
  }
};

template <int VAR>
struct LabelConfigsRun {
  static cudaError_t run(const float* q, int n, int dof, const RobotDev& rb, const SceneDev& sc, uint8_t* out,
                         cudaStream_t st) {
    const size_t smem = static_cast<size_t>(scene_float4s(sc)) * 16;
    label_configs_kernel<VAR><<<blocks_for(n, kThreads), kThreads, smem, st>>>(q, n, dof, rb, sc, out);
    return cudaGetLastError();
  }
};

template <int VAR>
struct OptimisticRun {
  static cudaError_t run(const GraphDev& g, int layer, const uint32_t* bad, const int* state, cudaStream_t st) {
    const int rows = layer_size(g, layer);
    const int blocks = (rows + kWarps - 1) / kWarps;
    if (g.n_wb > 0)
      optimistic_transition_kernel<VAR, true><<<blocks, kThreads, 0, st>>>(g, layer, bad, state);
    else
      optimistic_transition_kernel<VAR, false><<<blocks, kThreads, 0, st>>>(g, layer, bad, state);
    return cudaGetLastError();
  }
};

template <int VAR>
struct CheckChainRun {
  static cudaError_t run(const GraphDev& g, const int32_t* path, const RobotDev& rb, const SceneDev& sc,
                         uint32_t* bad, size_t words, int* state, cudaStream_t st) {
    const size_t smem = static_cast<size_t>(scene_float4s(sc)) * 16;
    check_chain_kernel<VAR><<<1, kThreads, smem, st>>>(g, path, rb, sc, bad, words, state);
    return cudaGetLastError();
  }
};

template <int VAR>
struct FusedRun {
  static cudaError_t run(const GraphDev& g, int layer, const RobotDev& rb, const SceneDev& sc, int mode,
                         int* counters, int grid_x, int chunk, int* err, bool dependent, cudaStream_t st) {
    return fused_dispatch<VAR>(g, layer, rb, sc, mode, counters, grid_x, chunk, err, dependent, st);
  }
};

template <int VAR>
struct EdgeCostsRun {
  static cudaError_t run(const GraphDev& g, int layer, const RobotDev& rb, const SceneDev& sc, float* C, int cs,
                         int* counter, int grid_x, int chunk, int* err, cudaStream_t st) {
    const size_t smem = static_cast<size_t>(scene_float4s(sc)) * 16;
    if (g.n_wb > 0)
      edge_costs_kernel<VAR, true><<<grid_x, kThreads, smem, st>>>(g, layer, rb, sc, C, cs, counter, chunk, err);
    else
      edge_costs_kernel<VAR, false><<<grid_x, kThreads, smem, st>>>(g, layer, rb, sc, C, cs, counter, chunk, err);
    return cudaGetLastError();
  }
};

template <int VAR>
struct OccupancyRun {
  static cudaError_t run(int mode, int* out) {
    if (mode == kEvalFull)
      return cudaOccupancyMaxActiveBlocksPerMultiprocessor(out, fused_transition_kernel<VAR, kEvalFull, false>,
                                                           kThreads, 16 * 1024);
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(out, fused_transition_kernel<VAR, kEvalEarlyExit, false>,
                                                         kThreads, 16 * 1024);
  }
};

template <int VAR>
struct ConfigureRun {
  static cudaError_t run(int smem_max) {
    cudaError_t e;
    const void* fns[] = {
        reinterpret_cast<const void*>(fused_transition_kernel<VAR, kEvalFull, false>),
        reinterpret_cast<const void*>(fused_transition_kernel<VAR, kEvalEarlyExit, false>),
        reinterpret_cast<const void*>(fused_transition_kernel<VAR, kEvalLazy, false>),
        reinterpret_cast<const void*>(fused_transition_kernel<VAR, kEvalFull, true>),
        reinterpret_cast<const void*>(fused_transition_kernel<VAR, kEvalEarlyExit, true>),
        reinterpret_cast<const void*>(fused_transition_kernel<VAR, kEvalLazy, true>),
        reinterpret_cast<const void*>(edge_costs_kernel<VAR, false>),
        reinterpret_cast<const void*>(edge_costs_kernel<VAR, true>)};
    for (const void* f : fns)
      if ((e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_max)) != cudaSuccess) return e;
    if ((e = cudaFuncSetAttribute(vertex_labels_kernel<VAR>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  smem_max)) != cudaSuccess)
      return e;
    if ((e = cudaFuncSetAttribute(sample_free_kernel<VAR>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_max)) !=
        cudaSuccess)
      return e;
    if ((e = cudaFuncSetAttribute(check_chain_kernel<VAR>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_max)) !=
        cudaSuccess)
      return e;
    return cudaFuncSetAttribute(label_configs_kernel<VAR>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_max);
  }
};

}  // namespace

double arm_reach_bound(const RobotDev& rb) {
  double reach = 0.0, offset = 0.0;
  for (int i = 0; i < rb.dof; ++i) {
    reach += std::fabs(static_cast<double>(rb.a[i])) + std::fabs(static_cast<double>(rb.d[i]));
    const int stride = rb.spl > 4 || rb.uniform_r == 0 ? kMaxSpl : 4;
    for (int k = 0; k < rb.spl; ++k) {
      const float4 p = rb.sph[i * stride + k];
      offset = std::fmax(offset, std::sqrt(double(p.x) * p.x + double(p.y) * p.y + double(p.z) * p.z));
    }
  }
  return reach + offset;
}

int build_prefilter_table(const float* spheres, int n_s, const float* boxes, int n_b, float r, double reach,
                          float4* out) {
  const int n = n_s + n_b;
  if (n == 0) return 0;
  // bound of the obstacle centres and radii, for the rounding-error margin
  double bo = 0.0, rmax = 0.0;
  std::vector<double> cx(n), cy(n), cz(n), R(n);
  for (int o = 0; o < n_s; ++o) {
    const float* s = spheres + 4 * o;
    cx[o] = s[0];
    cy[o] = s[1];
    cz[o] = s[2];
    R[o] = double(s[3]) + double(r);
  }
  for (int o = 0; o < n_b; ++o) {
    const float* b = boxes + 6 * o;
    const float c0 = 0.5f * (b[0] + b[3]), c1 = 0.5f * (b[1] + b[4]), c2 = 0.5f * (b[2] + b[5]);
    const float h0 = 0.5f * (b[3] - b[0]), h1 = 0.5f * (b[4] - b[1]), h2 = 0.5f * (b[5] - b[2]);
    cx[n_s + o] = c0;
    cy[n_s + o] = c1;
    cz[n_s + o] = c2;
    // enclosing ball of the box as the kernel sees it (float centre and half extents), enlarged by a hair
    R[n_s + o] = std::sqrt(double(h0) * h0 + double(h1) * h1 + double(h2) * h2) * (1.0 + 1e-6) + 1e-7 + double(r);
  }
  for (int o = 0; o < n; ++o) {
    bo = std::fmax(bo, std::sqrt(cx[o] * cx[o] + cy[o] * cy[o] + cz[o] * cz[o]));
    rmax = std::fmax(rmax, R[o]);
  }
  // float32 error of |c|^2 + a.c + k is below 8 * 2^-24 * ((|c| + |o|)^2 + R^2); keep 100x of it
  const double err = 8.0 * std::ldexp(1.0, -24) * ((reach + bo) * (reach + bo) + rmax * rmax + reach * reach);
  const double margin = std::fmax(1e-3, 100.0 * err);
  const int pairs = (n + 1) / 2;
  for (int p = 0; p < pairs; ++p) {
    float ax[2], ay[2], az[2], kk[2];
    for (int h = 0; h < 2; ++h) {
      const int o = 2 * p + h;
      if (o < n) {
        ax[h] = static_cast<float>(-2.0 * cx[o]);
        ay[h] = static_cast<float>(-2.0 * cy[o]);
        az[h] = static_cast<float>(-2.0 * cz[o]);
        kk[h] = static_cast<float>(cx[o] * cx[o] + cy[o] * cy[o] + cz[o] * cz[o] - R[o] * R[o] - margin);
      } else {  // padding: never flags
        ax[h] = ay[h] = az[h] = 0.0f;
        kk[h] = 1e30f;
      }
    }
    out[2 * p] = make_float4(ax[0], ax[1], ay[0], ay[1]);
    out[2 * p + 1] = make_float4(az[0], az[1], kk[0], kk[1]);
  }
  return pairs;
}

// Link-cull table (three float4 per obstacle pair, layout of link_cull_mask):
// the sphere obstacles' pairs, then the box obstacles' pairs, paired like the
// exact tables so that pair p's bit selects the same obstacles there; per
// obstacle -2o, |o|^2 - r_o^2 - margin and -2 r_o, boxes by their enclosing
// ball; the margin covers the float32 error of the test as the prefilter's
// does, with link balls of radius up to 1 m.
int build_cull_table(const float* spheres, int n_s, const float* boxes, int n_b, double reach, float4* out) {
  const int n = n_s + n_b;
  if (n == 0) return 0;
  std::vector<double> cx(n), cy(n), cz(n), R(n);
  for (int o = 0; o < n_s; ++o) {
    const float* s = spheres + 4 * o;
    cx[o] = s[0];
    cy[o] = s[1];
    cz[o] = s[2];
    R[o] = s[3];
  }
  for (int o = 0; o < n_b; ++o) {
    const float* b = boxes + 6 * o;
    const float c0 = 0.5f * (b[0] + b[3]), c1 = 0.5f * (b[1] + b[4]), c2 = 0.5f * (b[2] + b[5]);
    const float h0 = 0.5f * (b[3] - b[0]), h1 = 0.5f * (b[4] - b[1]), h2 = 0.5f * (b[5] - b[2]);
    cx[n_s + o] = c0;
    cy[n_s + o] = c1;
    cz[n_s + o] = c2;
    R[n_s + o] = std::sqrt(double(h0) * h0 + double(h1) * h1 + double(h2) * h2) * (1.0 + 1e-6) + 1e-7;
  }
  double bo = 0.0, rmax = 0.0;
  for (int o = 0; o < n; ++o) {
    bo = std::fmax(bo, std::sqrt(cx[o] * cx[o] + cy[o] * cy[o] + cz[o] * cz[o]));
    rmax = std::fmax(rmax, R[o]);
  }
  const double err = 8.0 * std::ldexp(1.0, -24) * ((reach + bo) * (reach + bo) + (rmax + 1.0) * (rmax + 1.0) + reach * reach);
  const double margin = std::fmax(1e-3, 100.0 * err);
  const int n_sp = (n_s + 1) / 2, n_bp = (n_b + 1) / 2;
  for (int p = 0; p < n_sp + n_bp; ++p) {
    // pair p: spheres 2p, 2p+1, or boxes 2(p - n_sp), 2(p - n_sp)+1
    const bool sph = p < n_sp;
    const int first = sph ? 2 * p : n_s + 2 * (p - n_sp);
    const int end = sph ? n_s : n;
    float ax[2], ay[2], az[2], kk[2], rr[2];
    for (int h = 0; h < 2; ++h) {
      const int o = first + h;
      if (o < end) {
        ax[h] = static_cast<float>(-2.0 * cx[o]);
        ay[h] = static_cast<float>(-2.0 * cy[o]);
        az[h] = static_cast<float>(-2.0 * cz[o]);
        kk[h] = static_cast<float>(cx[o] * cx[o] + cy[o] * cy[o] + cz[o] * cz[o] - R[o] * R[o] - margin);
        rr[h] = static_cast<float>(-2.0 * R[o]);
      } else {  // padding: never near
        ax[h] = ay[h] = az[h] = rr[h] = 0.0f;
        kk[h] = 1e30f;
      }
    }
    out[3 * p] = make_float4(ax[0], ax[1], ay[0], ay[1]);
    out[3 * p + 1] = make_float4(az[0], az[1], kk[0], kk[1]);
    out[3 * p + 2] = make_float4(rr[0], rr[1], 0.0f, 0.0f);
  }
  return n_sp + n_bp;
}

int build_packed_tables(const float* spheres, int n_s, const float* boxes, int n_b, float r, double reach,
                        float4* out, SceneDev* sc) {
  const int n_sp = (n_s + 1) / 2, n_bp = (n_b + 1) / 2;
  const float far = 1e18f;
  for (int p = 0; p < n_sp; ++p) {
    float v[2][4];
    for (int h = 0; h < 2; ++h) {
      const int o = 2 * p + h;
      if (o < n_s) {
        const float* q = spheres + 4 * o;
        const float rr = q[3] + r;
        v[h][0] = -q[0];
        v[h][1] = -q[1];
        v[h][2] = -q[2];
        v[h][3] = -(rr * rr);
      } else {
        v[h][0] = v[h][1] = v[h][2] = -far;
        v[h][3] = 0.0f;
      }
    }
    out[2 * p] = make_float4(v[0][0], v[1][0], v[0][1], v[1][1]);
    out[2 * p + 1] = make_float4(v[0][2], v[1][2], v[0][3], v[1][3]);
  }
  float4* bo = out + 2 * n_sp;
  for (int p = 0; p < n_bp; ++p) {
    float v[2][6];
    for (int h = 0; h < 2; ++h) {
      const int o = 2 * p + h;
      if (o < n_b) {
        const float* b = boxes + 6 * o;
        v[h][0] = -(0.5f * (b[0] + b[3]));
        v[h][1] = -(0.5f * (b[1] + b[4]));
        v[h][2] = -(0.5f * (b[2] + b[5]));
        v[h][3] = -(0.5f * (b[3] - b[0]));
        v[h][4] = -(0.5f * (b[4] - b[1]));
        v[h][5] = -(0.5f * (b[5] - b[2]));
      } else {
        v[h][0] = v[h][1] = v[h][2] = -far;
        v[h][3] = v[h][4] = v[h][5] = 0.0f;
      }
    }
    bo[3 * p] = make_float4(v[0][0], v[1][0], v[0][1], v[1][1]);
    bo[3 * p + 1] = make_float4(v[0][2], v[1][2], v[0][3], v[1][3]);
    bo[3 * p + 2] = make_float4(v[0][4], v[1][4], v[0][5], v[1][5]);
  }
  const int n_pp = build_prefilter_table(spheres, n_s, boxes, n_b, r, reach, bo + 3 * n_bp);
  int n_cull = 0;
  const int base = 2 * n_sp + 3 * n_bp + 2 * n_pp;
  if (base + 3 * (n_sp + n_bp) <= kMaxTableFloat4s)
    n_cull = build_cull_table(spheres, n_s, boxes, n_b, reach, bo + 3 * n_bp + 2 * n_pp);
  sc->n_s = n_s;
  sc->n_b = n_b;
  sc->packed = 1;
  sc->n_sp = n_sp;
  sc->n_bp = n_bp;
  sc->n_pairs = n_pp;
  sc->n_cull = n_cull;
  return base + 3 * n_cull;
}

int build_cull_grid(const float* spheres, int n_s, const float* boxes, int n_b, double R_link, int max_cells,
                    float4* out, SceneDev* sc) {
  sc->gnx = sc->gny = sc->gnz = 0;
  const int n_sp = (n_s + 1) / 2, n_pairs = n_sp + (n_b + 1) / 2;
  if (n_s + n_b == 0 || n_pairs > 32 || sc->n_cull != n_pairs || max_cells < 64) return 0;
  // each obstacle as (lo, hi, reach): a sphere is its centre with reach
  // R_link + r_obs, a box its extent with reach R_link; margin over float32
  // rounding of the lookup (cell index of a point within ~1e-6 m of a face)
  const double margin = 2e-3;
  const int n = n_s + n_b;
  std::vector<double> lo(3 * n), hi(3 * n), reach(n);
  std::vector<int> bit(n);
  for (int o = 0; o < n_s; ++o) {
    for (int k = 0; k < 3; ++k) lo[3 * o + k] = hi[3 * o + k] = spheres[4 * o + k];
    reach[o] = R_link + spheres[4 * o + 3] + margin;
    bit[o] = o / 2;
  }
  for (int o = 0; o < n_b; ++o) {
    for (int k = 0; k < 3; ++k) {
      lo[3 * (n_s + o) + k] = boxes[6 * o + k];
      hi[3 * (n_s + o) + k] = boxes[6 * o + 3 + k];
    }
    reach[n_s + o] = R_link + margin;
    bit[n_s + o] = n_sp + o / 2;
  }
  double glo[3], ghi[3];
  for (int k = 0; k < 3; ++k) {
    glo[k] = 1e300;
    ghi[k] = -1e300;
    for (int o = 0; o < n; ++o) {
      glo[k] = std::fmin(glo[k], lo[3 * o + k] - reach[o] - margin);
      ghi[k] = std::fmax(ghi[k], hi[3 * o + k] + reach[o] + margin);
    }
  }
  const double ex = ghi[0] - glo[0], ey = ghi[1] - glo[1], ez = ghi[2] - glo[2];
  double h = std::cbrt(ex * ey * ez / max_cells);
  int nx, ny, nz;
  for (;;) {
    nx = std::max(1, static_cast<int>(std::ceil(ex / h)));
    ny = std::max(1, static_cast<int>(std::ceil(ey / h)));
    nz = std::max(1, static_cast<int>(std::ceil(ez / h)));
    if (static_cast<long long>(nx) * ny * nz <= max_cells) break;
    h *= 1.02;
  }
  // the lookup uses 1 / h in float32: take h as the float it implies
  const float inv = static_cast<float>(1.0 / h);
  h = 1.0 / static_cast<double>(inv);
  const int cells = nx * ny * nz;
  std::vector<uint32_t> mask(static_cast<size_t>(cells) + 3, 0u);
  // the squared distance between a cell and an obstacle's extent separates by
  // axis: per obstacle, the squared gap of every cell row along each axis
  std::vector<double> g2[3];
  for (int k = 0; k < 3; ++k) g2[k].resize(k == 0 ? nx : k == 1 ? ny : nz);
  for (int o = 0; o < n; ++o) {
    int c0[3], c1[3];
    for (int k = 0; k < 3; ++k) {
      const int nk = k == 0 ? nx : k == 1 ? ny : nz;
      c0[k] = std::max(0, static_cast<int>(std::floor((lo[3 * o + k] - reach[o] - glo[k]) / h)) - 1);
      c1[k] = std::min(nk - 1, static_cast<int>(std::floor((hi[3 * o + k] + reach[o] - glo[k]) / h)) + 1);
      for (int i = c0[k]; i <= c1[k]; ++i) {
        const double a = glo[k] + i * h, b = a + h;
        const double gap = std::fmax(std::fmax(lo[3 * o + k] - b, a - hi[3 * o + k]), 0.0);
        g2[k][i] = gap * gap;
      }
    }
    const double r2 = reach[o] * reach[o];
    const uint32_t b = 1u << bit[o];
    for (int iz = c0[2]; iz <= c1[2]; ++iz)
      for (int iy = c0[1]; iy <= c1[1]; ++iy) {
        const double dyz = g2[2][iz] + g2[1][iy];
        if (dyz >= r2) continue;
        uint32_t* row = mask.data() + (static_cast<size_t>(iz) * ny + iy) * nx;
        for (int ix = c0[0]; ix <= c1[0]; ++ix)
          if (dyz + g2[0][ix] < r2) row[ix] |= b;
      }
  }
  std::memcpy(out, mask.data(), static_cast<size_t>((cells + 3) / 4) * sizeof(float4));
  sc->gnx = nx;
  sc->gny = ny;
  sc->gnz = nz;
  sc->glx = static_cast<float>(glo[0]);
  sc->gly = static_cast<float>(glo[1]);
  sc->glz = static_cast<float>(glo[2]);
  sc->ginv = inv;
  sc->g_off = 2 * sc->n_sp + 3 * sc->n_bp + 2 * sc->n_pairs + 3 * sc->n_cull;
  return (cells + 3) / 4;
}

void fill_link_bounds(RobotDev* rb) {
  const int stride = rb->spl > 4 || rb->uniform_r == 0 ? kMaxSpl : 4;
  for (int i = 0; i < rb->dof; ++i) {
    double c[3] = {0.0, 0.0, 0.0};
    for (int k = 0; k < rb->spl; ++k) {
      const float4 p = rb->sph[i * stride + k];
      c[0] += p.x;
      c[1] += p.y;
      c[2] += p.z;
    }
    for (double& v : c) v /= rb->spl;
    const float cx = static_cast<float>(c[0]), cy = static_cast<float>(c[1]), cz = static_cast<float>(c[2]);
    double R = 0.0;
    for (int k = 0; k < rb->spl; ++k) {
      const float4 p = rb->sph[i * stride + k];
      const double dx = double(p.x) - cx, dy = double(p.y) - cy, dz = double(p.z) - cz;
      R = std::fmax(R, std::sqrt(dx * dx + dy * dy + dz * dz) + double(p.w));
    }
    // enlarged by a hair, like the enclosing balls of boxes
    rb->lb[i] = make_float4(cx, cy, cz, static_cast<float>(R * (1.0 + 1e-6) + 1e-7));
  }
}

cudaError_t configure_kernels(int smem_max) {
  cudaError_t e;
  for (int v = 0; v < 4; ++v)
    if ((e = by_variant<ConfigureRun>(v, smem_max)) != cudaSuccess) return e;
  return cudaFuncSetAttribute(minplus_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_max);
}

// ------------------------------------------------------------------------------------------------
// launch wrappers
// ------------------------------------------------------------------------------------------------
cudaError_t launch_sample_uniform(const GraphDev& g, const float* lo, const float* hi, int dof,
                                  unsigned long long seed, int restart0, cudaStream_t st) {
  const long long n = static_cast<long long>(g.R) * g.L * g.M;
  if (n == 0) return cudaSuccess;
  sample_uniform_kernel<<<blocks_for(n, kThreads), kThreads, 0, st>>>(g, make_box(lo, hi, dof), dof, seed, restart0);
  return cudaGetLastError();
}

cudaError_t launch_sample_free(const GraphDev& g, const RobotDev& rb, int variant, const SceneDev& sc, const float* lo,
                               const float* hi, int dof, unsigned long long seed, int restart0, int max_attempts,
                               cudaStream_t st) {
  return by_variant<SampleFreeRun>(variant, g, rb, sc, make_box(lo, hi, dof), dof, seed, restart0, max_attempts, st);
}

cudaError_t launch_init_keys(const GraphDev& g, int* counters, int n_counters, cudaStream_t st) {
  long long n = static_cast<long long>(g.R) * (g.L + 2) * g.M_stride;
  if (n < n_counters) n = n_counters;
  init_keys_kernel<<<blocks_for(n, kThreads), kThreads, 0, st>>>(g, counters, n_counters);
  return cudaGetLastError();
}

cudaError_t launch_vertex_labels(const GraphDev& g, const RobotDev& rb, int variant, const SceneDev& sc,
                                 cudaStream_t st) {
  return by_variant<VertexLabelsRun>(variant, g, rb, sc, st);
}

namespace {
__global__ void joint_sincos_kernel(const float* x, int n, float* s, float* c) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < n) joint_sincos(x[t], s + t, c + t);
}
}  // namespace

cudaError_t launch_joint_sincos(const float* x, int n, float* s, float* c, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  joint_sincos_kernel<<<(n + 255) / 256, 256, 0, st>>>(x, n, s, c);
  return cudaGetLastError();
}

cudaError_t launch_label_configs(const float* q, int n, int dof, const RobotDev& rb, int variant, const SceneDev& sc,
                                 uint8_t* out, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  return by_variant<LabelConfigsRun>(variant, q, n, dof, rb, sc, out, st);
}

cudaError_t launch_lazy_iteration(const GraphDev& g, int variant, const RobotDev& rb, const SceneDev& sc,
                                  uint32_t* bad, size_t words, int32_t* path, float* cost, int* state,
                                  int max_iterations, cudaStream_t st) {
  cudaError_t e;
  for (int layer = g.L; layer >= 0; --layer)
    if ((e = by_variant<OptimisticRun>(variant, g, layer, bad + static_cast<size_t>(layer) * words,
                                       static_cast<const int*>(state), st)) != cudaSuccess)
      return e;
  if ((e = launch_extract_paths(g, path, cost, nullptr, st)) != cudaSuccess) return e;
  lazy_iteration_begin_kernel<<<1, 1, 0, st>>>(state);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if ((e = by_variant<CheckChainRun>(variant, g, path, rb, sc, bad, words, state, st)) != cudaSuccess) return e;
  lazy_iteration_end_kernel<<<1, 1, 0, st>>>(state, max_iterations);
  return cudaGetLastError();
}

cudaError_t launch_fused_transition(const GraphDev& g, int layer, const RobotDev& rb, int variant, const SceneDev& sc,
                                    int mode, int* counters, int grid_x, int chunk, int* err, cudaStream_t st,
                                    bool dependent) {
  return by_variant<FusedRun>(variant, g, layer, rb, sc, mode, counters, grid_x, chunk, err, dependent, st);
}

int fused_max_blocks_per_sm(int variant, int mode) {
  int out = 1;
  if (by_variant<OccupancyRun>(variant, mode, &out) != cudaSuccess || out < 1) out = 1;
  return out;
}

cudaError_t launch_extract_paths(const GraphDev& g, int32_t* path, float* cost, int32_t* best, cudaStream_t st) {
  extract_paths_kernel<<<1, 256, 0, st>>>(g, path, cost, best);
  return cudaGetLastError();
}

cudaError_t launch_get_values(const GraphDev& g, float* V, int32_t* sigma, cudaStream_t st) {
  const long long n = static_cast<long long>(g.R) * (g.L + 2) * g.M;
  get_values_kernel<<<blocks_for(n, kThreads), kThreads, 0, st>>>(g, V, sigma);
  return cudaGetLastError();
}

cudaError_t launch_pack_layers(const GraphDev& g, float* user, int dof, int to_internal, cudaStream_t st) {
  const long long n = static_cast<long long>(g.R) * g.L * g.M;
  if (n == 0) return cudaSuccess;
  pack_layers_kernel<<<blocks_for(n, kThreads), kThreads, 0, st>>>(g, user, dof, to_internal);
  return cudaGetLastError();
}

cudaError_t launch_edge_costs(const GraphDev& g, int layer, const RobotDev& rb, int variant, const SceneDev& sc,
                              float* C, int cs, int* counter, int grid_x, int chunk, int* err, cudaStream_t st) {
  return by_variant<EdgeCostsRun>(variant, g, layer, rb, sc, C, cs, counter, grid_x, chunk, err, st);
}

cudaError_t launch_minplus(const GraphDev& g, int layer, const float* C, int cs, int grid, bool dependent,
                           cudaStream_t st) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(kThreads);
  cfg.dynamicSmemBytes = static_cast<size_t>(cs) * 4;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = dependent ? 1 : 0;
  return cudaLaunchKernelEx(&cfg, minplus_kernel, g, layer, C, cs);
}

// goal vertex reached by graph gi's best chain (-1 if infeasible)
__global__ void goal_reached_kernel(GraphDev g, int gi, int32_t* goal) {
  unsigned long long k = g.keys[vidx(g, gi, 0, 0)];
  if (k == kEmptyKey) {
    *goal = -1;
    return;
  }
  for (int l = 1; l <= g.L; ++l) k = g.keys[vidx(g, gi, l, key_index(k))];
  *goal = static_cast<int32_t>(key_index(k));
}

cudaError_t launch_goal_reached(const GraphDev& g, int gi, int32_t* goal, cudaStream_t st) {
  goal_reached_kernel<<<1, 1, 0, st>>>(g, gi, goal);
  return cudaGetLastError();
}

cudaError_t launch_expand(const GraphDev& g, int dof, const float* lo, const float* hi, unsigned long long seed,
                          int M_old, int M_new, const float* c_best, int max_attempts, int* err, cudaStream_t st) {
  const long long n = static_cast<long long>(g.L) * (M_new - M_old);
  if (n <= 0) return cudaSuccess;
  expand_kernel<<<blocks_for(n, 128), 128, 0, st>>>(g, dof, make_box(lo, hi, dof), seed, M_old, M_new, c_best,
                                                    max_attempts, err);
  return cudaGetLastError();
}

cudaError_t launch_gather_chain(const GraphDev& g, const int32_t* path, float* chain, int dof, int rows,
                                cudaStream_t st) {
  gather_chain_kernel<<<rows, 32, 0, st>>>(g, path, chain, dof, rows);
  return cudaGetLastError();
}

cudaError_t launch_update_best(int L, const int32_t* cand_path, const float* cand_cost, int32_t* best_path,
                               float* best_cost, cudaStream_t st) {
  update_best_kernel<<<1, 32, 0, st>>>(L, cand_path, cand_cost, best_path, best_cost);
  return cudaGetLastError();
}

}  // namespace gtmp
