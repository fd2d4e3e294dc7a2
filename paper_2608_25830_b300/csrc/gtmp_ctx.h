// Context of the C ABI (private to the library's host code).
#pragma once

#include <string>
#include <utility>
#include <vector>

#include "../../include/gtmp.h"
#include "gtmp_kernels.cuh"

namespace gtmp {
struct SurrogateState;  // gtmp_surrogate.cu
void surrogate_free(SurrogateState* s);
}  // namespace gtmp

using gtmp::RobotDev;
using gtmp::SceneDev;
using gtmp::kMaxDof;
using gtmp::kVarArmGeneric;

struct gtmp_ctx {
  int device = 0;
  int num_sms = 148;
  cudaStream_t stream = nullptr;
  gtmp_params p{};
  RobotDev rb{};
  int variant = kVarArmGeneric;
  int dof = 0, dp = 0;
  float q_lo[kMaxDof] = {}, q_hi[kMaxDof] = {};
  // device memory
  float* Q = nullptr;
  uint8_t* vflag = nullptr;
  unsigned long long* keys = nullptr;
  int* counters = nullptr;
  int n_counters = 0;
  float4* obs = nullptr;
  SceneDev sc{};  // counts and layout of the obstacle table at obs
  int* err = nullptr;
  float* C = nullptr;
  std::vector<size_t> c_off;
  std::vector<int> c_cs;
  // goal set (Alg. 1's G with terminal values V_g); gtmp_set_endpoints resets it to its single goal
  int G = 1;
  float* gval = nullptr;  // [p.M] device, valid when goal_values is set
  bool goal_values = false;
  // layer capacity (gtmp_create's L); p.L is the active layer count (gtmp_set_num_layers)
  int L_cap = 0;
  // host copies of the start and the goal set, re-uploaded when the layer count changes
  std::vector<float> host_start, host_goals;
  // aogtmp_run scratch (device): stage path, best path [L_cap] int32, stage cost, best cost
  int32_t* ao_scratch = nullptr;
  // weighted-length edge cost: n_wb bumps in the GraphDev layout (null/0: plain length)
  float4* wb = nullptr;
  int n_wb = 0;
  // layer sampler: GTMP_SAMPLER_UNIFORM or GTMP_SAMPLER_FREE (rejection on C_free, bounded attempts)
  int sampler = 0;
  int sampler_attempts = 64;
  // state
  bool have_endpoints = false;
  int M_active = 0;
  int fused_bps[2] = {1, 1};
  std::string last_error;
  // instrumentation
  long long launches = 0;
  bool timing = false;
  std::vector<cudaEvent_t> ev_pool;
  std::vector<std::pair<int, int>> ev_used;  // (start, end) indices into ev_pool
  double timed_edges = 0.0;
  std::vector<std::pair<int, int>> ev_minplus;  // (start, end) indices into ev_pool
  double minplus_bytes = 0.0;
  int64_t minplus_launches = 0;
  int64_t fused_timed_launches = 0;             // fused launches timed (the sweeps in ev_used)                 // min-plus launches timed (the sweeps in ev_minplus)
  // learned collision surrogate (allocated by gtmp_surrogate_train)
  gtmp::SurrogateState* sur = nullptr;
  float sur_protect = 0.0f;  // protection band of the pruned solve (gtmp_surrogate_set_protect); 0 = off
  uint8_t* prune = nullptr;  // per-transition prune mask, M x M
  uint32_t* lazy_bad = nullptr;  // path-level lazy evaluation: per transition a bit per (row, column) found colliding
  size_t lazy_words = 0;         // 32-bit words per transition of lazy_bad
  int* lazy_count = nullptr;     // the iteration state of gtmp_solve_lazy_path (LazyState)
  // class-augmented sweep (allocated by gtmp_solve_classes)
  void* cls = nullptr;
  size_t cls_bytes = 0;
  std::vector<std::pair<double, double>> centres;  // obstacle centres in the plane (host)
};

// vertex labels and every transition's stored cost matrix (step 1 of gtmp_solve_unfused)
gtmp_status gtmp_internal_edge_costs(gtmp_ctx* c);
