// Batched planning: many independent layered graphs (different robots, M, L,
// obstacle sets) solved by one persistent launch.
//
// Each problem is Alg. 1 gtmp with the straight-line planner, exactly as
// gtmp_solve runs it (same samples for the same seed, same per-edge device
// code, same tie rule), so every problem's result equals its single-problem
// solve.  The persistent kernel serves a work list of (problem, depth,
// block of rows) items ordered by depth (depth 0 = the transition into the
// goal, depth L_p = the start row); a CTA takes the next item from a global
// counter, waits until every item of the previous depth of the same problem
// has finished, and realises its rows with the warp-per-edge fused step.
// Because items are handed out in depth order, an item only ever waits for
// items that were handed out before it to CTAs that are already running, so
// the queue cannot deadlock; every wait is nevertheless bounded in time and
// sets the error word when it gives up.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <string>
#include <vector>

#include "../../include/gtmp.h"
#include "gtmp_edge.cuh"

using namespace gtmp;

namespace gtmp_batch_impl {

struct ProblemDev {
  GraphDev g;          // R = 1, M_stride = M
  SceneDev sc;         // obs points into the batch obstacle buffer
  int variant;
  int robot;           // index into the robot array
  int dof;
  int need_base;       // offset of this problem's per-depth item counts / done counters
  unsigned long long seed;
  float lo[kMaxDof], hi[kMaxDof];
};

struct WorkItem {
  int p, depth, row0, rows, col0, cols;
};

constexpr int kBoundaryItemEdges = 256;          // item size cap for the start row and the goal column
constexpr long long kWaitCycles = 4000000000LL;  // ~2 s at 2 GHz without progress

__device__ __forceinline__ int ld_acquire(const int* p) {
  int v;
  asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// ---------------------------------------------------------------------------
// per-problem set-up kernels: grid.y = problem
// ---------------------------------------------------------------------------
__global__ void batch_init_kernel(const ProblemDev* probs) {
  const ProblemDev& P = probs[blockIdx.y];
  const GraphDev& g = P.g;
  const long long n = static_cast<long long>(g.L + 2) * g.M_stride;
  for (long long t = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x; t < n;
       t += static_cast<long long>(gridDim.x) * blockDim.x) {
    const int layer = static_cast<int>(t / g.M_stride);
    const int i = static_cast<int>(t % g.M_stride);
    g.keys[t] = (layer == g.L + 1 && i == 0) ? make_key(0.0f, 0u) : kEmptyKey;
  }
}

// Alg. 1 uniform sampling, the rule of gtmp_sample_layers (restart 0)
__global__ void batch_sample_kernel(const ProblemDev* probs) {
  const ProblemDev& P = probs[blockIdx.y];
  const GraphDev& g = P.g;
  const long long n = static_cast<long long>(g.L) * g.M;
  const uint2 key = seed_key(P.seed);
  for (long long t = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x; t < n;
       t += static_cast<long long>(gridDim.x) * blockDim.x) {
    const int i = static_cast<int>(t % g.M);
    const int l = static_cast<int>(t / g.M);
    float* out = g.Q + vidx(g, 0, l + 1, i) * g.dp;
    uint4 w = make_uint4(0, 0, 0, 0);
    for (int k = 0; k < g.dp; ++k) {
      if (k >= P.dof) {
        out[k] = 0.0f;
        continue;
      }
      if ((k & 3) == 0)
        w = philox4x32_10(make_uint4(static_cast<uint32_t>(i), static_cast<uint32_t>(l), 0u,
                                     (kTagUniform << 24) | (k >> 2)),
                          key);
      out[k] = __fmaf_rn(word_to_unit(word_of(w, k)), __fsub_rn(P.hi[k], P.lo[k]), P.lo[k]);
    }
  }
}

template <int VAR>
__device__ __forceinline__ bool vertex_collides(const float* p, int dp, const RobotDev& rb, const float4* s_obs,
                                                const SceneDev& sc) {
  constexpr int DP = Var<VAR>::kDp;
  float q[DP];
  load_vertex<DP>(q, p, dp);
  return config_collides<VAR, false, false>(q, true, rb, s_obs, sc);
}

__global__ void __launch_bounds__(kThreads) batch_labels_kernel(const ProblemDev* probs, const RobotDev* robots) {
  __shared__ RobotDev s_rb;
  extern __shared__ __align__(16) float4 s_obs[];
  const ProblemDev& P = probs[blockIdx.y];
  const GraphDev& g = P.g;
  {
    const int* src = reinterpret_cast<const int*>(robots + P.robot);
    int* dst = reinterpret_cast<int*>(&s_rb);
    for (int k = threadIdx.x; k < static_cast<int>(sizeof(RobotDev) / 4); k += blockDim.x) dst[k] = src[k];
  }
  stage_obstacles_plain(s_obs, P.sc.obs, scene_float4s(P.sc));
  __syncthreads();
  const long long n = static_cast<long long>(g.L + 2) * g.M_stride;
  for (long long t = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x; t < n;
       t += static_cast<long long>(gridDim.x) * blockDim.x) {
    const int layer = static_cast<int>(t / g.M_stride);
    const int i = static_cast<int>(t % g.M_stride);
    if (i >= layer_size(g, layer)) continue;
    const float* q = g.Q + vidx(g, 0, layer, i) * g.dp;
    bool hit;
    switch (P.variant) {
      case kVarPoint: hit = vertex_collides<kVarPoint>(q, g.dp, s_rb, s_obs, P.sc); break;
      case kVarArm6x4: hit = vertex_collides<kVarArm6x4>(q, g.dp, s_rb, s_obs, P.sc); break;
      case kVarArm7x4: hit = vertex_collides<kVarArm7x4>(q, g.dp, s_rb, s_obs, P.sc); break;
      default: hit = vertex_collides<kVarArmGeneric>(q, g.dp, s_rb, s_obs, P.sc); break;
    }
    g.vflag[vidx(g, 0, layer, i)] = hit ? 1 : 0;
  }
}

// ---------------------------------------------------------------------------
// the persistent kernel
// ---------------------------------------------------------------------------
template <int VAR, bool LAZY>
__device__ __forceinline__ void item_rows(const GraphDev& g, const SceneDev& sc, int layer, int row0, int rows,
                                          int col0, int cols, int chunk, const float* s_V, const RobotDev& rb,
                                          const float4* s_obs, int* s_next) {
  const int lane = threadIdx.x & 31;
  if constexpr (LAZY) {
    // (32-column block, row) units, block-major, as the single-problem lazy kernel
    const int n_blk = (cols + 31) / 32;
    const int n_units = rows * n_blk;
    while (true) {
      int c = 0;
      if (lane == 0) c = atomicAdd(s_next, 1);
      c = __shfl_sync(kFull, c, 0);
      if (c >= n_units) break;
      const int b = c / rows;
      lazy_block<VAR>(g, 0, layer, row0 + c - b * rows, col0 + b * 32, col0 + cols, s_V, rb, s_obs, sc, lane);
    }
  } else {
    if (VAR == kVarPoint) chunk = chunk < 32 ? 32 : chunk;  // one edge per lane
    const int cpr = (cols + chunk - 1) / chunk;
    const int n_chunks = rows * cpr;
    while (true) {
      int c = 0;
      if (lane == 0) c = atomicAdd(s_next, 1);
      c = __shfl_sync(kFull, c, 0);
      if (c >= n_chunks) break;
      const int i = row0 + c / cpr;
      const int j0 = col0 + (c % cpr) * chunk;
      const int j1 = min(j0 + chunk, col0 + cols);
      const unsigned long long best = row_chunk_best<VAR, false>(g, 0, layer, i, j0, j1, s_V, rb, s_obs, sc, lane);
      if (lane == 0 && best != kEmptyKey) atomicMin(&g.keys[vidx(g, 0, layer, i)], best);
    }
  }
}

// One persistent kernel per robot variant and mode, launched one after another
// on the batch stream over that variant's share of the work list: each keeps
// its edge code inlined, as the single-problem kernel does (one kernel for
// all variants needed out-of-line bodies, which cost ~12 % per edge, or
// spilled); the problem's graph and scene descriptors are read from shared
// memory, the robot constants too (a batch holds a robot per problem).
template <int VAR, bool LAZY>
__global__ void __launch_bounds__(kThreads, kFusedMinBlocks)
    batch_persistent_kernel(const ProblemDev* __restrict__ probs, const RobotDev* __restrict__ robots,
                            const WorkItem* __restrict__ items, int n_items, const int* __restrict__ need,
                            int* done, int* next_item, int chunk, int* err) {
  __shared__ RobotDev s_rb;
  // raw storage: the descriptor types have default member initialisers
  __shared__ __align__(16) unsigned char s_g_raw[sizeof(GraphDev)];
  __shared__ __align__(16) unsigned char s_sc_raw[sizeof(SceneDev)];
  GraphDev& s_g = *reinterpret_cast<GraphDev*>(s_g_raw);
  SceneDev& s_sc = *reinterpret_cast<SceneDev*>(s_sc_raw);
  __shared__ int s_item, s_next, s_ok;
  extern __shared__ __align__(16) float4 smem[];
  // the next variant's persistent launch (independent problems) may start on the SMs this one leaves
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  while (true) {
    if (threadIdx.x == 0) {
      s_item = atomicAdd(next_item, 1);
      s_next = 0;
    }
    __syncthreads();
    const int it = s_item;
    if (it >= n_items) break;
    const WorkItem w = items[it];
    const ProblemDev& P = probs[w.p];
    const int layer = P.g.L - w.depth;
    // dependency: every item of depth - 1 of this problem has finished
    if (threadIdx.x == 0) {
      int ok = 1;
      if (w.depth > 0) {
        const int* cnt = done + P.need_base + w.depth - 1;
        const int want = need[P.need_base + w.depth - 1];
        // the limit applies to time without progress: it restarts whenever
        // another item of the awaited depth finishes
        long long t0 = clock64();
        int seen = -1;
        for (int v = ld_acquire(cnt); v < want; v = ld_acquire(cnt)) {
          if (v != seen) {
            seen = v;
            t0 = clock64();
          }
          if (*reinterpret_cast<volatile int*>(err) != 0 || clock64() - t0 > kWaitCycles) {
            atomicOr(err, kErrWaitTimeout);
            ok = 0;
            break;
          }
          __nanosleep(256);
        }
      }
      s_ok = ok;
    }
    __syncthreads();
    if (!s_ok) continue;  // the item is abandoned; the error word reports it
    // stage the robot, the problem's descriptors, the obstacles and the column layer's cost-to-go
    {
      const int* src = reinterpret_cast<const int*>(robots + P.robot);
      int* dst = reinterpret_cast<int*>(&s_rb);
      for (int k = threadIdx.x; k < static_cast<int>(sizeof(RobotDev) / 4); k += blockDim.x) dst[k] = src[k];
      if (threadIdx.x == 0) {
        s_g = P.g;
        s_sc = P.sc;
      }
    }
    const int n4 = scene_float4s(P.sc);
    stage_obstacles_plain(smem, P.sc.obs, n4);
    float* s_V = reinterpret_cast<float*>(smem + n4);
    for (int j = w.col0 + threadIdx.x; j < w.col0 + w.cols; j += blockDim.x) {
      const size_t v = vidx(P.g, 0, layer + 1, j);
      s_V[j] = P.g.vflag[v] ? kInf : key_value(__ldcg(P.g.keys + v));
    }
    __syncthreads();
    if constexpr (VAR == kVarPoint) {
      item_rows<VAR, LAZY>(s_g, s_sc, layer, w.row0, w.rows, w.col0, w.cols, chunk, s_V, s_rb, smem, &s_next);
    } else {
      // the arms' edge loop with the problem's descriptors in registers (measured 2.4 % faster per edge;
      // the point robot's is faster reading them from shared memory); the robot stays in shared memory
      const GraphDev g = s_g;
      const SceneDev sc = s_sc;
      item_rows<VAR, LAZY>(g, sc, layer, w.row0, w.rows, w.col0, w.cols, chunk, s_V, s_rb, smem, &s_next);
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) atomicAdd(done + P.need_base + w.depth, 1);
  }
  // launched as a dependent of the previous variant's kernel: finish only after it has, so that the
  // path kernel behind this one sees every variant's results
  asm volatile("griddepcontrol.wait;" ::: "memory");
}

__global__ void batch_paths_kernel(const ProblemDev* probs, int n, int L_max, int32_t* paths, float* costs) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= n) return;
  const GraphDev& g = probs[p].g;
  int32_t* out = paths + static_cast<size_t>(p) * L_max;
  for (int l = 0; l < L_max; ++l) out[l] = -1;
  const unsigned long long k0 = g.keys[vidx(g, 0, 0, 0)];
  if (k0 == kEmptyKey) {
    costs[p] = kInf;
    return;
  }
  costs[p] = key_value(k0);
  int i = key_index(k0);
  for (int l = 1; l <= g.L; ++l) {
    out[l - 1] = i;
    if (l < g.L) i = key_index(g.keys[vidx(g, 0, l, i)]);
  }
}

// robot kind of a kernel variant: 0 = point robot, 1 = DH arm
inline int robot_kind(int variant) { return variant == kVarPoint ? GTMP_ROBOT_POINT : GTMP_ROBOT_DH_ARM; }

bool finite_all(const float* v, size_t n) {
  for (size_t k = 0; k < n; ++k)
    if (!std::isfinite(v[k])) return false;
  return true;
}

}  // namespace gtmp_batch_impl

using namespace gtmp_batch_impl;

struct gtmp_batch {
  int n = 0, H = 0, L_max = 0, M_max = 0, obs4_max = 0;
  int num_sms = 148;
  int bps[4][2] = {};                    // persistent blocks per SM per variant and mode (early exit, lazy)
  size_t smem[4] = {};                   // dynamic shared memory of variant v's persistent launch: its largest
                                         // obstacle table and cost-to-go row
  int item_begin[5] = {};                // the work list holds variant v's items in [item_begin[v], item_begin[v + 1])
  cudaStream_t stream = nullptr;
  // host copies
  std::vector<ProblemDev> probs;
  std::vector<RobotDev> robots;
  std::vector<int> need;  // items per (problem, depth)
  double nominal_checks = 0.0;
  // tiling per robot kind (GTMP_ROBOT_POINT, GTMP_ROBOT_DH_ARM), autotuned
  int target_edges[2] = {16384, 16384};
  int chunk[2] = {32, 16};
  int eval_mode = GTMP_EVAL_EARLY_EXIT;
  int n_items = 0;
  // device memory
  ProblemDev* d_probs = nullptr;
  RobotDev* d_robots = nullptr;
  WorkItem* d_items = nullptr;
  int* d_need = nullptr;
  int* d_done = nullptr;  // [need.size()] done counters followed by one item counter per variant
  int* d_err = nullptr;
  float4* d_obs = nullptr;
  float* d_Q = nullptr;
  uint8_t* d_vflag = nullptr;
  unsigned long long* d_keys = nullptr;
  std::string last_error;
};

namespace gtmp_batch_impl {

gtmp_status bfail(gtmp_batch* b, gtmp_status s, const char* fmt, ...) {
  if (b) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    b->last_error = buf;
  }
  return s;
}

#define BATCH_TRY(b, expr)                                                                               \
  do {                                                                                                   \
    cudaError_t e_ = (expr);                                                                             \
    if (e_ != cudaSuccess)                                                                               \
      return bfail((b), e_ == cudaErrorMemoryAllocation ? GTMP_ERR_OOM : GTMP_ERR_CUDA, "%s: %s", #expr, \
                   cudaGetErrorString(e_));                                                              \
  } while (0)

// robot constants and kernel variant, as gtmp_create chooses them
bool make_robot(const gtmp_robot& r, RobotDev* rb, int* variant, int* dp) {
  *rb = RobotDev{};
  rb->kind = r.kind;
  rb->dof = r.dof;
  rb->point_radius = r.point_radius;
  if (r.kind == GTMP_ROBOT_POINT) {
    if (r.dof < 1 || r.dof > 3 || !(r.point_radius >= 0.0f) || !std::isfinite(r.point_radius)) return false;
    rb->spl = 1;
    rb->uniform_r = 1;
    rb->r_uniform = r.point_radius;
    *variant = kVarPoint;
    *dp = 4;
    return true;
  }
  if (r.kind != GTMP_ROBOT_DH_ARM || r.dof < 1 || r.dof > kMaxDof || !r.dh || !r.link_spheres ||
      r.spheres_per_link < 1 || r.spheres_per_link > kMaxSpl)
    return false;
  const int spl = r.spheres_per_link;
  if (!finite_all(r.dh, static_cast<size_t>(r.dof) * 4) ||
      !finite_all(r.link_spheres, static_cast<size_t>(r.dof) * spl * 4) || !r.q_lo || !r.q_hi ||
      !arm_angles_in_range(r.q_lo, r.q_hi, r.dh, r.dof))
    return false;
  bool uniform = true;
  const float r0 = r.link_spheres[3];
  for (int s = 0; s < r.dof * spl; ++s) {
    if (!(r.link_spheres[s * 4 + 3] > 0.0f)) return false;
    if (r.link_spheres[s * 4 + 3] != r0) uniform = false;
  }
  *variant = arm_kernel_variant(uniform, spl, r.dof, r0);
  const int stride = *variant == kVarArmGeneric ? kMaxSpl : 4;
  *dp = *variant == kVarArmGeneric ? kMaxDof : 8;
  rb->spl = spl;
  rb->uniform_r = *variant == kVarArmGeneric ? 0 : 1;
  rb->r_uniform = r0;
  for (int i = 0; i < r.dof; ++i) {
    rb->d[i] = r.dh[i * 4 + 0];
    rb->a[i] = r.dh[i * 4 + 1];
    rb->ca[i] = cosf(r.dh[i * 4 + 2]);
    rb->sa[i] = sinf(r.dh[i * 4 + 2]);
    rb->toff[i] = r.dh[i * 4 + 3];
    for (int s = 0; s < spl; ++s) {
      const float* ls = r.link_spheres + (static_cast<size_t>(i) * spl + s) * 4;
      rb->sph[i * stride + s] = make_float4(ls[0], ls[1], ls[2], ls[3]);
    }
  }
  fill_link_bounds(rb);
  return true;
}

constexpr int kBatchGridCells = 16384;
constexpr size_t kBatchSmemMax = 200 * 1024;  // dynamic shared memory the batch kernels opt in to

// scalar or packed obstacle table of one problem (the layout gtmp_set_obstacles writes)
int obstacle_table(const gtmp_problem& q, const RobotDev& rb, int variant, std::vector<float4>& out, SceneDev* sc) {
  *sc = SceneDev{};
  if (variant == kVarArm6x4 || variant == kVarArm7x4) {
    out.resize(packed_table_capacity(q.n_s + q.n_b) + kBatchGridCells / 4 + 1);
    int n4 = build_packed_tables(q.spheres, q.n_s, q.boxes, q.n_b, rb.r_uniform, arm_reach_bound(rb), out.data(),
                                 sc);
    // the single-problem solver's cull grid (16384 cells, 64 KB of masks), when the table has room for it
    double R_link = 0.0;
    for (int i = 0; i < rb.dof; ++i) R_link = std::fmax(R_link, static_cast<double>(rb.lb[i].w));
    if (n4 + kBatchGridCells / 4 + 1 <= kMaxTableFloat4s)
      n4 += build_cull_grid(q.spheres, q.n_s, q.boxes, q.n_b, R_link, kBatchGridCells, out.data() + n4, sc);
    out.resize(n4);
    return n4;
  }
  out.resize(static_cast<size_t>(q.n_s) + 2 * static_cast<size_t>(q.n_b));
  for (int o = 0; o < q.n_s; ++o) {
    const float* s = q.spheres + 4 * o;
    float w = s[3];
    if (rb.uniform_r) {
      const float rr = s[3] + rb.r_uniform;
      w = rr * rr;
    }
    out[o] = make_float4(s[0], s[1], s[2], w);
  }
  for (int o = 0; o < q.n_b; ++o) {
    const float* bx = q.boxes + 6 * o;
    out[q.n_s + 2 * o] = make_float4(0.5f * (bx[0] + bx[3]), 0.5f * (bx[1] + bx[4]), 0.5f * (bx[2] + bx[5]),
                                     0.5f * (bx[3] - bx[0]));
    out[q.n_s + 2 * o + 1] = make_float4(0.5f * (bx[4] - bx[1]), 0.5f * (bx[5] - bx[2]), 0.0f, 0.0f);
  }
  sc->n_s = q.n_s;
  sc->n_b = q.n_b;
  return static_cast<int>(out.size());
}

// work list for the current tiling: items sorted by depth, then problem
gtmp_status build_items(gtmp_batch* b) {
  std::vector<WorkItem> items;
  std::fill(b->need.begin(), b->need.end(), 0);
  for (int v = 0; v < 4; ++v) {
   b->item_begin[v] = static_cast<int>(items.size());
   for (int d = 0; d <= b->L_max; ++d)
    for (int p = 0; p < b->n; ++p) {
      const ProblemDev& P = b->probs[p];
      if (P.variant != v || d > P.g.L) continue;
      const int layer = P.g.L - d;
      const int rows = layer_size(P.g, layer), cols = layer_size(P.g, layer + 1);
      // boundary transitions (start row, goal column) sit at the two ends of
      // every problem's dependency chain: cut them into small items
      // each robot kind has its own item size (a point-robot edge costs about 1/20 of an arm edge)
      const long long target = b->target_edges[robot_kind(P.variant)];
      const int edges_per_item = static_cast<int>(
          (rows == 1 || cols == 1) ? std::min<long long>(target, kBoundaryItemEdges) : std::min<long long>(target, 1 << 30));
      if (rows == 1) {
        for (int c0 = 0; c0 < cols; c0 += edges_per_item) {
          items.push_back(WorkItem{p, d, 0, 1, c0, std::min(edges_per_item, cols - c0)});
          b->need[P.need_base + d] += 1;
        }
        continue;
      }
      if (edges_per_item < cols) {
        // items smaller than a row: column pieces of one row (keeps a depth's
        // items many and short, so its last wave leaves few CTAs idle)
        for (int r0 = 0; r0 < rows; ++r0)
          for (int c0 = 0; c0 < cols; c0 += edges_per_item) {
            items.push_back(WorkItem{p, d, r0, 1, c0, std::min(edges_per_item, cols - c0)});
            b->need[P.need_base + d] += 1;
          }
        continue;
      }
      int per = edges_per_item / std::max(cols, 1);
      per = std::max(1, std::min(per, rows));
      for (int r0 = 0; r0 < rows; r0 += per) {
        items.push_back(WorkItem{p, d, r0, std::min(per, rows - r0), 0, cols});
        b->need[P.need_base + d] += 1;
      }
    }
  }
  b->item_begin[4] = static_cast<int>(items.size());
  b->n_items = static_cast<int>(items.size());
  cudaFree(b->d_items);
  b->d_items = nullptr;
  BATCH_TRY(b, cudaMalloc(&b->d_items, items.size() * sizeof(WorkItem)));
  BATCH_TRY(b, cudaMemcpy(b->d_items, items.data(), items.size() * sizeof(WorkItem), cudaMemcpyHostToDevice));
  BATCH_TRY(b, cudaMemcpy(b->d_need, b->need.data(), b->need.size() * sizeof(int), cudaMemcpyHostToDevice));
  return GTMP_OK;
}

// one variant's persistent launch; dependent: a programmatic dependent of the previous kernel on the stream
template <int VAR, bool LAZY>
cudaError_t launch_persistent(dim3 grid, size_t smem, cudaStream_t st, bool dependent, const ProblemDev* probs,
                              const RobotDev* robots, const WorkItem* items, int n_items, const int* need,
                              int* done, int* next_item, int chunk, int* err) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = dim3(kThreads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = dependent ? 1 : 0;
  return cudaLaunchKernelEx(&cfg, batch_persistent_kernel<VAR, LAZY>, probs, robots, items, n_items, need, done,
                            next_item, chunk, err);
}

// ev (optional): events 2 v and 2 v + 1 are recorded around variant v's persistent launch
gtmp_status enqueue_solve(gtmp_batch* b, int32_t* dev_paths, float* dev_costs, cudaEvent_t* ev = nullptr) {
  cudaStream_t st = b->stream;
  const size_t n_done = b->need.size() + 4;
  BATCH_TRY(b, cudaMemsetAsync(b->d_done, 0, n_done * sizeof(int), st));
  const int per_problem_blocks = std::max(1, std::min(64, ((b->L_max + 2) * b->M_max + kThreads - 1) / kThreads));
  batch_init_kernel<<<dim3(per_problem_blocks, b->n), kThreads, 0, st>>>(b->d_probs);
  BATCH_TRY(b, cudaGetLastError());
  batch_sample_kernel<<<dim3(per_problem_blocks, b->n), kThreads, 0, st>>>(b->d_probs);
  BATCH_TRY(b, cudaGetLastError());
  batch_labels_kernel<<<dim3(per_problem_blocks, b->n), kThreads, b->obs4_max * sizeof(float4), st>>>(b->d_probs,
                                                                                                    b->d_robots);
  BATCH_TRY(b, cudaGetLastError());
  const int lazy = b->eval_mode == GTMP_EVAL_LAZY ? 1 : 0;
  // the arms first, the point robots last: their short items fill the SMs the arm kernel's last items leave
  // (each later variant is a programmatic dependent of the one before; timed runs launch them plainly)
  static const int kOrder[4] = {kVarArm7x4, kVarArm6x4, kVarArmGeneric, kVarPoint};
  bool first = true;
  for (int v : kOrder) {
    const int n_items = b->item_begin[v + 1] - b->item_begin[v];
    if (n_items == 0) continue;
    const dim3 grid(b->num_sms * b->bps[v][lazy]);
    const size_t smem = b->smem[v];
    const WorkItem* items = b->d_items + b->item_begin[v];
    int* counter = b->d_done + b->need.size() + v;
    const int chunk = b->chunk[robot_kind(v)];
    const bool dependent = !first && ev == nullptr;
    first = false;
    if (ev) BATCH_TRY(b, cudaEventRecord(ev[2 * v], st));
    cudaError_t le = cudaSuccess;
#define GTMP_BATCH_LAUNCH(VAR)                                                                                 \
  le = lazy ? launch_persistent<VAR, true>(grid, smem, st, dependent, b->d_probs, b->d_robots, items, n_items,  \
                                           b->d_need, b->d_done, counter, chunk, b->d_err)                      \
            : launch_persistent<VAR, false>(grid, smem, st, dependent, b->d_probs, b->d_robots, items, n_items, \
                                            b->d_need, b->d_done, counter, chunk, b->d_err)
    switch (v) {
      case kVarPoint: GTMP_BATCH_LAUNCH(kVarPoint); break;
      case kVarArm6x4: GTMP_BATCH_LAUNCH(kVarArm6x4); break;
      case kVarArm7x4: GTMP_BATCH_LAUNCH(kVarArm7x4); break;
      default: GTMP_BATCH_LAUNCH(kVarArmGeneric); break;
    }
#undef GTMP_BATCH_LAUNCH
    BATCH_TRY(b, le);
    if (ev) BATCH_TRY(b, cudaEventRecord(ev[2 * v + 1], st));
  }
  batch_paths_kernel<<<(b->n + 127) / 128, 128, 0, st>>>(b->d_probs, b->n, b->L_max, dev_paths, dev_costs);
  BATCH_TRY(b, cudaGetLastError());
  return GTMP_OK;
}

}  // namespace gtmp_batch_impl

extern "C" {

GTMP_API gtmp_status gtmp_batch_create(const gtmp_problem* problems, int32_t n, int32_t H, void* cuda_stream,
                                       gtmp_batch** out) {
  if (!out || !problems || n < 1 || n > (1 << 20) || H < 2 || H > 1024) return GTMP_ERR_INVALID_ARG;
  *out = nullptr;
  gtmp_batch* b = new gtmp_batch();
  b->n = n;
  b->H = H;
  b->stream = static_cast<cudaStream_t>(cuda_stream);
  b->probs.resize(n);
  b->robots.resize(n);
  std::vector<std::vector<float4>> tables(n);
  size_t q_floats = 0, verts = 0, obs4 = 0;
  int need_total = 0;
  for (int p = 0; p < n; ++p) {
    const gtmp_problem& q = problems[p];
    RobotDev rb;
    int variant = 0, dp = 0;
    if (!make_robot(q.robot, &rb, &variant, &dp) || q.M < 1 || q.M > 16384 || q.L < 1 || q.L > 64 || q.n_s < 0 ||
        q.n_b < 0 || q.n_s + q.n_b > 4096 || (q.n_s > 0 && !q.spheres) || (q.n_b > 0 && !q.boxes) ||
        !q.q_start || !q.q_goal || !q.robot.q_lo || !q.robot.q_hi) {
      delete b;
      return GTMP_ERR_INVALID_ARG;
    }
    const int dof = q.robot.dof;
    bool ok = finite_all(q.robot.q_lo, dof) && finite_all(q.robot.q_hi, dof) &&
              (q.n_s == 0 || finite_all(q.spheres, static_cast<size_t>(q.n_s) * 4)) &&
              (q.n_b == 0 || finite_all(q.boxes, static_cast<size_t>(q.n_b) * 6));
    for (int k = 0; ok && k < dof; ++k)
      ok = q.robot.q_hi[k] > q.robot.q_lo[k] && std::isfinite(q.q_start[k]) && std::isfinite(q.q_goal[k]) &&
           q.q_start[k] >= q.robot.q_lo[k] && q.q_start[k] <= q.robot.q_hi[k] && q.q_goal[k] >= q.robot.q_lo[k] &&
           q.q_goal[k] <= q.robot.q_hi[k];
    for (int o = 0; ok && o < q.n_s; ++o) ok = q.spheres[4 * o + 3] >= 0.0f;
    for (int o = 0; ok && o < q.n_b; ++o)
      for (int k = 0; k < 3; ++k) ok = ok && q.boxes[6 * o + 3 + k] >= q.boxes[6 * o + k];
    if (!ok) {
      delete b;
      return GTMP_ERR_INVALID_ARG;
    }
    b->robots[p] = rb;
    ProblemDev& P = b->probs[p];
    P = ProblemDev{};
    P.variant = variant;
    P.robot = p;
    P.dof = dof;
    P.seed = q.seed;
    for (int k = 0; k < dof; ++k) {
      P.lo[k] = q.robot.q_lo[k];
      P.hi[k] = q.robot.q_hi[k];
    }
    P.g.R = 1;
    P.g.L = q.L;
    P.g.M = q.M;
    P.g.M_stride = q.M;
    P.g.dp = dp;
    P.g.H = H;
    P.g.max_edge_len = INFINITY;
    const int n4 = obstacle_table(q, rb, variant, tables[p], &P.sc);
    // offsets (converted to pointers once the buffers exist)
    P.g.Q = reinterpret_cast<float*>(q_floats);
    P.g.vflag = reinterpret_cast<uint8_t*>(verts);
    P.g.keys = reinterpret_cast<unsigned long long*>(verts);
    P.sc.obs = reinterpret_cast<const float4*>(obs4);
    const size_t v = static_cast<size_t>(q.L + 2) * q.M;
    q_floats += v * dp;
    verts += v;
    obs4 += n4;
    P.need_base = need_total;
    need_total += q.L + 1;
    b->L_max = std::max(b->L_max, q.L);
    b->M_max = std::max(b->M_max, q.M);
    b->obs4_max = std::max(b->obs4_max, n4);
    b->smem[variant] = std::max(b->smem[variant], n4 * sizeof(float4) + static_cast<size_t>(q.M) * sizeof(float));
    b->nominal_checks += static_cast<double>(H) * (2.0 * q.M + (q.L - 1.0) * q.M * q.M);
  }
  b->need.assign(need_total, 0);
  // every item stages its problem's obstacle table and cost-to-go row in shared memory
  if (static_cast<size_t>(b->obs4_max) * sizeof(float4) > kBatchSmemMax ||
      *std::max_element(b->smem, b->smem + 4) > kBatchSmemMax) {
    delete b;
    return GTMP_ERR_UNSUPPORTED;
  }
  auto fail_create = [&](cudaError_t e) {
    gtmp_batch_destroy(b);
    return e == cudaErrorMemoryAllocation ? GTMP_ERR_OOM : GTMP_ERR_CUDA;
  };
  cudaError_t e = cudaSuccess;
  int dev = 0;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return fail_create(e);
  if ((e = cudaDeviceGetAttribute(&b->num_sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess)
    return fail_create(e);
  if ((e = cudaFuncSetAttribute(batch_labels_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  static_cast<int>(kBatchSmemMax))) !=
      cudaSuccess)
    return fail_create(e);
  {
    const void* kernels[4][2] = {
        {reinterpret_cast<const void*>(batch_persistent_kernel<kVarPoint, false>),
         reinterpret_cast<const void*>(batch_persistent_kernel<kVarPoint, true>)},
        {reinterpret_cast<const void*>(batch_persistent_kernel<kVarArm6x4, false>),
         reinterpret_cast<const void*>(batch_persistent_kernel<kVarArm6x4, true>)},
        {reinterpret_cast<const void*>(batch_persistent_kernel<kVarArm7x4, false>),
         reinterpret_cast<const void*>(batch_persistent_kernel<kVarArm7x4, true>)},
        {reinterpret_cast<const void*>(batch_persistent_kernel<kVarArmGeneric, false>),
         reinterpret_cast<const void*>(batch_persistent_kernel<kVarArmGeneric, true>)}};
    for (int v = 0; v < 4; ++v)
      for (int m = 0; m < 2; ++m) {
        if ((e = cudaFuncSetAttribute(kernels[v][m], cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  static_cast<int>(kBatchSmemMax))) !=
            cudaSuccess)
          return fail_create(e);
        if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b->bps[v][m], kernels[v][m], kThreads,
                                                               b->smem[v])) !=
            cudaSuccess)
          return fail_create(e);
        if (b->bps[v][m] < 1) b->bps[v][m] = 1;
      }
  }
  if ((e = cudaMalloc(&b->d_Q, std::max<size_t>(q_floats, 1) * sizeof(float))) != cudaSuccess ||
      (e = cudaMalloc(&b->d_vflag, std::max<size_t>(verts, 1))) != cudaSuccess ||
      (e = cudaMalloc(&b->d_keys, std::max<size_t>(verts, 1) * sizeof(unsigned long long))) != cudaSuccess ||
      (e = cudaMalloc(&b->d_obs, std::max<size_t>(obs4, 1) * sizeof(float4))) != cudaSuccess ||
      (e = cudaMalloc(&b->d_probs, n * sizeof(ProblemDev))) != cudaSuccess ||
      (e = cudaMalloc(&b->d_robots, n * sizeof(RobotDev))) != cudaSuccess ||
      (e = cudaMalloc(&b->d_need, (need_total + 1) * sizeof(int))) != cudaSuccess ||
      (e = cudaMalloc(&b->d_done, (need_total + 4) * sizeof(int))) != cudaSuccess ||
      (e = cudaMalloc(&b->d_err, sizeof(int))) != cudaSuccess)
    return fail_create(e);
  // rebase offsets to device pointers; write endpoints and obstacle tables
  std::vector<float4> all_obs(obs4);
  std::vector<float> ends;
  for (int p = 0; p < n; ++p) {
    ProblemDev& P = b->probs[p];
    const size_t qo = reinterpret_cast<size_t>(P.g.Q), vo = reinterpret_cast<size_t>(P.g.vflag);
    const size_t oo = reinterpret_cast<size_t>(P.sc.obs);
    std::copy(tables[p].begin(), tables[p].end(), all_obs.begin() + oo);
    P.g.Q = b->d_Q + qo;
    P.g.vflag = b->d_vflag + vo;
    P.g.keys = b->d_keys + vo;
    P.sc.obs = b->d_obs + oo;
    ends.assign(P.g.dp, 0.0f);
    for (int k = 0; k < P.dof; ++k) ends[k] = problems[p].q_start[k];
    if ((e = cudaMemcpy(P.g.Q, ends.data(), P.g.dp * sizeof(float), cudaMemcpyHostToDevice)) != cudaSuccess)
      return fail_create(e);
    for (int k = 0; k < P.dof; ++k) ends[k] = problems[p].q_goal[k];
    if ((e = cudaMemcpy(P.g.Q + static_cast<size_t>(P.g.L + 1) * P.g.M * P.g.dp, ends.data(), P.g.dp * sizeof(float),
                        cudaMemcpyHostToDevice)) != cudaSuccess)
      return fail_create(e);
  }
  if ((obs4 > 0 && (e = cudaMemcpy(b->d_obs, all_obs.data(), obs4 * sizeof(float4), cudaMemcpyHostToDevice)) !=
                       cudaSuccess) ||
      (e = cudaMemcpy(b->d_probs, b->probs.data(), n * sizeof(ProblemDev), cudaMemcpyHostToDevice)) != cudaSuccess ||
      (e = cudaMemcpy(b->d_robots, b->robots.data(), n * sizeof(RobotDev), cudaMemcpyHostToDevice)) != cudaSuccess ||
      (e = cudaMemset(b->d_err, 0, sizeof(int))) != cudaSuccess)
    return fail_create(e);
  gtmp_status s = build_items(b);
  if (s != GTMP_OK) {
    gtmp_batch_destroy(b);
    return s;
  }
  *out = b;
  return GTMP_OK;
}

GTMP_API gtmp_status gtmp_batch_destroy(gtmp_batch* b) {
  if (!b) return GTMP_OK;
  cudaStreamSynchronize(b->stream);
  cudaFree(b->d_probs);
  cudaFree(b->d_robots);
  cudaFree(b->d_items);
  cudaFree(b->d_need);
  cudaFree(b->d_done);
  cudaFree(b->d_err);
  cudaFree(b->d_obs);
  cudaFree(b->d_Q);
  cudaFree(b->d_vflag);
  cudaFree(b->d_keys);
  delete b;
  return GTMP_OK;
}

GTMP_API const char* gtmp_batch_last_error(const gtmp_batch* b) { return b ? b->last_error.c_str() : "null batch"; }

GTMP_API gtmp_status gtmp_batch_set_stream(gtmp_batch* b, void* cuda_stream) {
  if (!b) return GTMP_ERR_INVALID_ARG;
  b->stream = static_cast<cudaStream_t>(cuda_stream);
  return GTMP_OK;
}

GTMP_API gtmp_status gtmp_batch_info(const gtmp_batch* b, int32_t* L_max, double* nominal_checks,
                                     int32_t* work_items, int32_t* kernels) {
  if (!b) return GTMP_ERR_INVALID_ARG;
  if (L_max) *L_max = b->L_max;
  if (nominal_checks) *nominal_checks = b->nominal_checks;
  if (work_items) *work_items = b->n_items;
  if (kernels) {
    // init, sample, labels, one persistent launch per variant present, paths
    int k = 4;
    for (int v = 0; v < 4; ++v) k += b->item_begin[v + 1] > b->item_begin[v] ? 1 : 0;
    *kernels = k;
  }
  return GTMP_OK;
}

GTMP_API gtmp_status gtmp_batch_solve(gtmp_batch* b, int32_t* dev_paths, float* dev_costs) {
  GtmpNvtxRange nvtx_("gtmp_batch_solve");
  if (!b || !dev_paths || !dev_costs) return bfail(b, GTMP_ERR_INVALID_ARG, "NULL output");
  return enqueue_solve(b, dev_paths, dev_costs);
}

GTMP_API gtmp_status gtmp_batch_synchronize(gtmp_batch* b) {
  if (!b) return GTMP_ERR_INVALID_ARG;
  BATCH_TRY(b, cudaStreamSynchronize(b->stream));
  int err = 0;
  BATCH_TRY(b, cudaMemcpy(&err, b->d_err, sizeof(int), cudaMemcpyDeviceToHost));
  if (err) {
    BATCH_TRY(b, cudaMemset(b->d_err, 0, sizeof(int)));
    return bfail(b, GTMP_ERR_TIMEOUT, "device error flags 0x%x (2 = a dependency wait timed out)", err);
  }
  return GTMP_OK;
}

GTMP_API gtmp_status gtmp_batch_set_kind_tiling(gtmp_batch* b, int32_t kind, int32_t target_edges, int32_t chunk) {
  if (!b || (kind != GTMP_ROBOT_POINT && kind != GTMP_ROBOT_DH_ARM) || target_edges < 1 || chunk < 1 || chunk > 4096)
    return bfail(b, GTMP_ERR_INVALID_ARG, "bad tiling");
  BATCH_TRY(b, cudaStreamSynchronize(b->stream));
  b->target_edges[kind] = target_edges;
  b->chunk[kind] = chunk;
  return build_items(b);
}

GTMP_API gtmp_status gtmp_batch_set_tiling(gtmp_batch* b, int32_t target_edges, int32_t chunk) {
  if (!b || target_edges < 1 || chunk < 1 || chunk > 4096) return bfail(b, GTMP_ERR_INVALID_ARG, "bad tiling");
  BATCH_TRY(b, cudaStreamSynchronize(b->stream));
  for (int k = 0; k < 2; ++k) {
    b->target_edges[k] = target_edges;
    b->chunk[k] = chunk;
  }
  return build_items(b);
}

GTMP_API gtmp_status gtmp_batch_autotune(gtmp_batch* b, int32_t repeats, int32_t* dev_paths, float* dev_costs,
                                         float* best_ms) {
  if (!b || repeats < 1 || !dev_paths || !dev_costs) return bfail(b, GTMP_ERR_INVALID_ARG, "bad autotune request");
  // candidate item sizes per kind (a point-robot edge is ~20 times cheaper), then chunks at the best size
  static const int kTargets[2][4] = {{4096, 16384, 65536, 262144}, {1024, 4096, 16384, 65536}};
  static const int kChunks[] = {4, 8, 16, 32};
  cudaEvent_t ev[10] = {};
  gtmp_status s = GTMP_OK;
  for (int k = 0; k < 10 && s == GTMP_OK; ++k)
    if (cudaEventCreate(&ev[k]) != cudaSuccess) s = bfail(b, GTMP_ERR_CUDA, "cudaEventCreate failed");
  int best_t[2] = {b->target_edges[0], b->target_edges[1]}, best_c[2] = {b->chunk[0], b->chunk[1]};
  float best[2] = {1e30f, 1e30f};
  // time every kind's persistent launches under tiling (t[k], c[k]); keep each kind's fastest
  auto trial = [&](const int* t, const int* c) -> gtmp_status {
    for (int k = 0; k < 2; ++k) {
      b->target_edges[k] = t[k];
      b->chunk[k] = c[k];
    }
    gtmp_status r = build_items(b);
    float ms[2] = {0.0f, 0.0f};
    for (int rep = 0; rep < repeats && r == GTMP_OK; ++rep) {
      if ((r = enqueue_solve(b, dev_paths, dev_costs, ev)) != GTMP_OK) break;
      if ((r = gtmp_batch_synchronize(b)) != GTMP_OK) break;
      for (int v = 0; v < 4; ++v) {
        if (b->item_begin[v + 1] == b->item_begin[v]) continue;
        float m = 0.0f;
        cudaEventElapsedTime(&m, ev[2 * v], ev[2 * v + 1]);
        ms[robot_kind(v)] += m / repeats;
      }
    }
    for (int k = 0; k < 2 && r == GTMP_OK; ++k)
      if (ms[k] < best[k]) {
        best[k] = ms[k];
        best_t[k] = t[k];
        best_c[k] = c[k];
      }
    return r;
  };
  if (s == GTMP_OK) s = build_items(b);
  if (s == GTMP_OK) s = enqueue_solve(b, dev_paths, dev_costs);  // warm-up
  if (s == GTMP_OK) s = gtmp_batch_synchronize(b);
  const int c0[2] = {best_c[0], best_c[1]};
  for (int i = 0; i < 4 && s == GTMP_OK; ++i) {
    const int t[2] = {kTargets[0][i], kTargets[1][i]};
    s = trial(t, c0);
  }
  const int t1[2] = {best_t[0], best_t[1]};
  for (int c : kChunks) {
    if (s != GTMP_OK) break;
    const int cc[2] = {c, c};
    s = trial(t1, cc);
  }
  if (s == GTMP_OK) {
    for (int k = 0; k < 2; ++k) {
      b->target_edges[k] = best_t[k];
      b->chunk[k] = best_c[k];
    }
    s = build_items(b);
  }
  if (s == GTMP_OK && best_ms) {
    // one timed pass of the whole solve under the tilings kept
    cudaEventRecord(ev[8], b->stream);
    for (int rep = 0; rep < repeats && s == GTMP_OK; ++rep) s = enqueue_solve(b, dev_paths, dev_costs);
    cudaEventRecord(ev[9], b->stream);
    if (s == GTMP_OK) s = gtmp_batch_synchronize(b);
    float ms = 0.0f;
    if (s == GTMP_OK) cudaEventElapsedTime(&ms, ev[8], ev[9]);
    *best_ms = ms / repeats;
  }
  for (cudaEvent_t e : ev)
    if (e) cudaEventDestroy(e);
  return s;
}

GTMP_API gtmp_status gtmp_batch_set_eval_mode(gtmp_batch* b, int32_t eval_mode) {
  if (!b || (eval_mode != GTMP_EVAL_EARLY_EXIT && eval_mode != GTMP_EVAL_LAZY))
    return bfail(b, GTMP_ERR_INVALID_ARG, "batch eval mode must be GTMP_EVAL_EARLY_EXIT or GTMP_EVAL_LAZY");
  b->eval_mode = eval_mode;
  return GTMP_OK;
}

GTMP_API gtmp_status gtmp_batch_inject_stall(gtmp_batch* b, int32_t problem, int32_t depth) {
  if (!b) return GTMP_ERR_INVALID_ARG;
  BATCH_TRY(b, cudaStreamSynchronize(b->stream));
  if (problem < 0) {
    BATCH_TRY(b, cudaMemcpy(b->d_need, b->need.data(), b->need.size() * sizeof(int), cudaMemcpyHostToDevice));
    return GTMP_OK;
  }
  if (problem >= b->n || depth < 0 || depth >= b->probs[problem].g.L)
    return bfail(b, GTMP_ERR_INVALID_ARG, "stall at problem %d depth %d: outside the batch", problem, depth);
  const int unreachable = 0x7fffffff;
  BATCH_TRY(b, cudaMemcpy(b->d_need + b->probs[problem].need_base + depth, &unreachable, sizeof(int),
                          cudaMemcpyHostToDevice));
  return GTMP_OK;
}

GTMP_API gtmp_status gtmp_batch_get_tiling(const gtmp_batch* b, int32_t kind, int32_t* target_edges, int32_t* chunk) {
  if (!b || (kind != GTMP_ROBOT_POINT && kind != GTMP_ROBOT_DH_ARM)) return GTMP_ERR_INVALID_ARG;
  if (target_edges) *target_edges = b->target_edges[kind];
  if (chunk) *chunk = b->chunk[kind];
  return GTMP_OK;
}

}  // extern "C"
