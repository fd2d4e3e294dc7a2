// Kernel launch interface shared by the C-ABI layer and the kernel sources.
#pragma once

#include <cmath>
#include <cstdint>
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include "gtmp_device.cuh"

// Scoped NVTX range around an ABI call, so Nsight timelines show the
// planner's stages (a no-op unless a tool is attached).
struct GtmpNvtxRange {
  explicit GtmpNvtxRange(const char* name) { nvtxRangePushA(name); }
  ~GtmpNvtxRange() { nvtxRangePop(); }
  GtmpNvtxRange(const GtmpNvtxRange&) = delete;
  GtmpNvtxRange& operator=(const GtmpNvtxRange&) = delete;
};

namespace gtmp {

// Geometry of one batch of same-shaped layered graphs (R restarts or copies).
// Vertex (r, layer, i) lives at Q[((r * (L + 2) + layer) * M + i) * dp]; layer 0
// holds q0 at i = 0, layers 1..L the samples, layer L+1 holds qg at i = 0.
struct GraphDev {
  float* Q;                      // [R][L+2][M][dp]
  uint8_t* vflag;                // [R][L+2][M]   1 = vertex in collision
  unsigned long long* keys;      // [R][L+2][M]   packed (V, sigma)
  int R, L, M, dp, H;            // M = active samples per layer, M_stride = allocated
  int M_stride;
  float max_edge_len;
  const uint8_t* prune = nullptr;  // [rows][cols] of the transition being run; 1 = edge dropped before checking
  int G = 1;                       // goal vertices (layer L+1)
  const float* gval = nullptr;     // [G] terminal values V_g (null: all 0)
  // weighted-length edge cost: n_wb bumps of dp / 4 + 1 float4 each, the
  // centre (dp floats, zero-padded), then (1 / s^2, a, 0, 0); n_wb = 0: length
  const float4* wb = nullptr;
  int n_wb = 0;
};

__host__ __device__ inline size_t vidx(const GraphDev& g, int r, int layer, int i) {
  return (static_cast<size_t>(r) * (g.L + 2) + layer) * g.M_stride + i;
}
__host__ __device__ inline int layer_size(const GraphDev& g, int layer) {
  return layer == 0 ? 1 : layer == g.L + 1 ? g.G : g.M;
}

// Obstacle table in device memory (staged whole into shared memory).
//  scalar layout (point robot, generic arm): n_s sphere float4, then 2 n_b box float4;
//  packed layout (uniform-radius 6/7-joint arms): 2 n_sp sphere-pair float4,
//  3 n_bp box-pair float4, 2 n_pairs prefilter float4 (see gtmp_device.cuh).
struct SceneDev {
  const float4* obs;
  int n_s, n_b;        // obstacle counts
  int packed;          // 1 = packed layout
  int n_sp, n_bp;      // packed: sphere pairs, box pairs
  int n_pairs;         // packed: prefilter pairs
  int n_cull = 0;      // packed: link-cull pairs (0: no cull)
  // packed, at most 32 cull pairs: uniform grid over the obstacles, per cell
  // the 32-bit mask of the cull pairs that can reach a link ball centred in
  // it (nx = 0: no grid); cells stored as uint32 from float4 offset g_off
  int g_off = 0;
  int gnx = 0, gny = 0, gnz = 0;
  float glx = 0.0f, gly = 0.0f, glz = 0.0f, ginv = 0.0f;  // lower corner, 1 / cell size
};

__host__ __device__ inline int scene_float4s(const SceneDev& s) {
  return s.packed ? 2 * s.n_sp + 3 * s.n_bp + 2 * s.n_pairs + 3 * s.n_cull + (s.gnx * s.gny * s.gnz + 3) / 4
                  : s.n_s + 2 * s.n_b;
}

// largest cull grid (cells; 64 KB of masks)
constexpr int kMaxGridCells = 16384;

// float4 capacity a packed obstacle table of n obstacles needs
inline size_t packed_table_capacity(int n) { return 5 * static_cast<size_t>(n) + 16; }

// largest obstacle table (float4s) the kernels stage into shared memory
constexpr int kMaxTableFloat4s = 12800;

enum EvalMode { kEvalEarlyExit = 0, kEvalFull = 1, kEvalLazy = 2 };

// Variant selector for the robot-specialised kernels.
enum RobotVariant { kVarPoint = 0, kVarArm6x4 = 1, kVarArm7x4 = 2, kVarArmGeneric = 3 };

// Kernel variant of a DH arm: the packed 6- and 7-joint kernels take four
// spheres per link of one radius r < 1 (their box test clamps each axis gap
// at 1, which decides nothing differently only while r < 1); every other arm
// takes the generic kernel.
inline int arm_kernel_variant(bool uniform, int spheres_per_link, int dof, float r) {
  if (!uniform || spheres_per_link != 4 || !(r < 1.0f)) return kVarArmGeneric;
  return dof == 6 ? kVarArm6x4 : dof == 7 ? kVarArm7x4 : kVarArmGeneric;
}

// Host: an arm's joint box (hence every sample, endpoint and goal) and theta
// offsets lie within the ranges the kinematics' joint_sincos serves
// (|q| <= kMaxJointAngle, |theta_offset| <= kMaxThetaOffset); dh is [dof][4].
inline bool arm_angles_in_range(const float* q_lo, const float* q_hi, const float* dh, int dof) {
  for (int k = 0; k < dof; ++k)
    if (!(std::fabs(q_lo[k]) <= kMaxJointAngle && std::fabs(q_hi[k]) <= kMaxJointAngle &&
          std::fabs(dh[4 * k + 3]) <= kMaxThetaOffset))
      return false;
  return true;
}

// Host: tables of the uniform-radius arm kernels (see gtmp_device.cuh).
// Prefilter: out receives 2 * pairs float4 (pairs = ceil((n_s + n_b) / 2));
// `reach` bounds |c| for every robot-sphere centre.  Returns the pair count.
int build_prefilter_table(const float* spheres, int n_s, const float* boxes, int n_b, float r, double reach,
                          float4* out);
// Packed exact + prefilter tables; fills sc's counts (not sc.obs) and returns
// the float4 count written to out (capacity 3 * (n_s + n_b) + 8 float4).
int build_packed_tables(const float* spheres, int n_s, const float* boxes, int n_b, float r, double reach,
                        float4* out, SceneDev* sc);
// Host: the cull grid appended after the packed tables (sc's counts set by
// build_packed_tables, at most 32 cull pairs): cells of the obstacles' region
// dilated by R_link, at most max_cells of them; cell mask bit p set when
// pair p's sphere comes within R_link + r_obs (box: R_link) of the cell, plus
// a margin.  Writes the float4s at out and the grid fields of sc; returns
// their count (0: no grid).
int build_cull_grid(const float* spheres, int n_s, const float* boxes, int n_b, double R_link, int max_cells,
                    float4* out, SceneDev* sc);
// Host: a bound on |c| over all robot-sphere centres of a DH arm.
double arm_reach_bound(const RobotDev& rb);
// per link, the centre and radius of a ball holding all its spheres (RobotDev::lb)
void fill_link_bounds(RobotDev* rb);

cudaError_t configure_kernels(int smem_max);
cudaError_t launch_sample_free(const GraphDev& g, const RobotDev& rb, int variant, const SceneDev& sc, const float* lo,
                               const float* hi, int dof, unsigned long long seed, int restart0, int max_attempts,
                               cudaStream_t st);
cudaError_t launch_sample_uniform(const GraphDev& g, const float* lo, const float* hi, int dof,
                                  unsigned long long seed, int restart0, cudaStream_t st);
cudaError_t launch_init_keys(const GraphDev& g, int* counters, int n_counters, cudaStream_t st);
cudaError_t launch_vertex_labels(const GraphDev& g, const RobotDev& rb, int variant, const SceneDev& sc,
                                 cudaStream_t st);
// the kinematics' joint_sincos on n arguments (device pointers)
cudaError_t launch_joint_sincos(const float* x, int n, float* s, float* c, cudaStream_t st);
cudaError_t launch_label_configs(const float* q, int n, int dof, const RobotDev& rb, int variant,
                                 const SceneDev& sc, uint8_t* out, cudaStream_t st);
// dependent: launch as a programmatic dependent of the previous kernel on the
// stream (that kernel must be the previous transition of the same sweep)
cudaError_t launch_fused_transition(const GraphDev& g, int layer, const RobotDev& rb, int variant,
                                    const SceneDev& sc, int mode, int* counters, int grid_x, int chunk, int* err,
                                    cudaStream_t st, bool dependent = false);
int fused_max_blocks_per_sm(int variant, int mode);
// Path-level lazy evaluation, one iteration on the stream: the min-plus sweep over optimistic
// costs (no collision check) without the edges marked in bad (words 32-bit words per transition),
// from transition state[kLazyStart] down, the chain extracted into path / cost, its exact check
// (colliding edges marked in bad) and the iteration's bookkeeping in state; every kernel returns
// at once when state[kLazyDone] is set, so iterations can be enqueued ahead of the host.
enum LazyState { kLazyFound = 0, kLazyHigh = 1, kLazyStart = 2, kLazyDone = 3, kLazyIters = 4, kLazyEdges = 5,
                 kLazyStateInts = 6 };
cudaError_t launch_lazy_iteration(const GraphDev& g, int variant, const RobotDev& rb, const SceneDev& sc,
                                  uint32_t* bad, size_t words, int32_t* path, float* cost, int* state,
                                  int max_iterations, cudaStream_t st);
cudaError_t launch_extract_paths(const GraphDev& g, int32_t* path, float* cost, int32_t* best, cudaStream_t st);
cudaError_t launch_goal_reached(const GraphDev& g, int gi, int32_t* goal, cudaStream_t st);
cudaError_t launch_get_values(const GraphDev& g, float* V, int32_t* sigma, cudaStream_t st);
cudaError_t launch_pack_layers(const GraphDev& g, float* user, int dof, int to_internal, cudaStream_t st);
cudaError_t launch_edge_costs(const GraphDev& g, int layer, const RobotDev& rb, int variant, const SceneDev& sc,
                              float* C, int cs, int* counter, int grid_x, int chunk, int* err, cudaStream_t st);
cudaError_t launch_minplus(const GraphDev& g, int layer, const float* C, int cs, int grid, bool dependent,
                           cudaStream_t st);
cudaError_t launch_expand(const GraphDev& g, int dof, const float* lo, const float* hi, unsigned long long seed,
                          int M_old, int M_new, const float* c_best, int max_attempts, int* err, cudaStream_t st);
cudaError_t launch_gather_chain(const GraphDev& g, const int32_t* path, float* chain, int dof, int rows,
                                cudaStream_t st);
cudaError_t launch_update_best(int L, const int32_t* cand_path, const float* cand_cost, int32_t* best_path,
                               float* best_cost, cudaStream_t st);

}  // namespace gtmp
