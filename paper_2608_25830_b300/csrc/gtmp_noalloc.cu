// gtmp_solve_noalloc: the fused solve of gtmp_solve without any device
// allocation, for callers that are not allowed to allocate device memory
// (see the declaration in include/gtmp.h).  All per-solve scratch lives in one
// file-scope device array of fixed size; this file only arranges that scratch
// and enqueues the same kernels gtmp_solve uses.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>

#include "../../include/gtmp.h"
#include "gtmp_kernels.cuh"

using namespace gtmp;

namespace {

// Scratch shared by every call on a device; every GPU that loads this library
// holds these bytes until the process exits.
constexpr size_t kNoallocScratchBytes = size_t(1) << 20;  // 1 MiB
constexpr int kNoallocMaxObstacles = 256;                 // spheres + boxes
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocScratchBytes];

// The call's host inputs (obstacle table, endpoints), carried to the device
// inside the kernel parameters of one staging launch: nothing is read from
// the caller's or this call's host memory after the call returns, and the
// call does not wait for earlier work on the stream (a pageable
// cudaMemcpyAsync would).  Kernel parameters may hold up to 32 764 bytes.
constexpr int kNoallocTableCap = 5 * kNoallocMaxObstacles + 16;  // packed_table_capacity(256)
struct NoallocStage {
  float4 obs[kNoallocTableCap];
  float ends[2][kMaxDof];  // start, goal; zero beyond dof
  int n4;                  // float4s of obs in use
  int dp;                  // padded coordinates per sample
  long long goal_offset;   // float offset of the goal vertex in Q
};
static_assert(sizeof(NoallocStage) <= 32000, "staging parameters exceed the kernel-parameter limit");

// error word = 0, obstacle table, both endpoints into Q (one block)
__global__ void noalloc_stage_kernel(const __grid_constant__ NoallocStage s, int* err, float4* obs, float* Q) {
  if (threadIdx.x == 0) *err = 0;
  for (int k = threadIdx.x; k < s.n4; k += blockDim.x) obs[k] = s.obs[k];
  if (threadIdx.x < s.dp) {
    Q[threadIdx.x] = s.ends[0][threadIdx.x];
    Q[s.goal_offset + threadIdx.x] = s.ends[1][threadIdx.x];
  }
}

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
unsigned char* g_scratch_dev[kMaxDevices] = {};  // device address of g_noalloc_scratch per device
int g_num_sms[kMaxDevices] = {};
int g_bps[kMaxDevices][4] = {};                  // fused blocks per SM per robot variant (early-exit mode)

gtmp_status report(char* msg, int32_t len, gtmp_status s, const char* fmt, ...) {
  if (msg && len > 0) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(msg, static_cast<size_t>(len), fmt, ap);
    va_end(ap);
  }
  return s;
}

// One-time set-up per device (with that device current): resolve the device
// address of the scratch array and query launch limits.
cudaError_t setup_device(int dev) {
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (g_scratch_dev[dev]) return cudaSuccess;
  void* ptr = nullptr;
  cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
  if (e != cudaSuccess) return e;
  int sms = 0;
  if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
  if ((e = configure_kernels(200 * 1024)) != cudaSuccess) return e;
  for (int v = 0; v < 4; ++v) g_bps[dev][v] = fused_max_blocks_per_sm(v, kEvalEarlyExit);
  g_num_sms[dev] = sms;
  g_scratch_dev[dev] = static_cast<unsigned char*>(ptr);
  return cudaSuccess;
}

size_t align256(size_t x) { return (x + 255) & ~static_cast<size_t>(255); }

bool all_finite(const float* v, size_t n) {
  for (size_t k = 0; k < n; ++k)
    if (!std::isfinite(v[k])) return false;
  return true;
}

}  // namespace

extern "C" GTMP_API gtmp_status gtmp_solve_noalloc(const gtmp_robot* robot, const float* spheres, int32_t n_s,
                                                   const float* boxes, int32_t n_b, const float* q_start,
                                                   const float* q_goal, const float* dev_Q, int32_t M, int32_t L,
                                                   int32_t H, float max_edge_len, void* cuda_stream,
                                                   int32_t* dev_path, float* dev_cost, int32_t* dev_status,
                                                   char* err_msg, int32_t err_msg_len) {
  if (err_msg && err_msg_len > 0) err_msg[0] = '\0';
  const gtmp_status bad = GTMP_ERR_INVALID_ARG;
  // ---- arguments (checked before any device call)
  if (!robot || !q_start || !q_goal || !dev_Q || !dev_path || !dev_cost)
    return report(err_msg, err_msg_len, bad, "NULL argument");
  if (robot->kind != GTMP_ROBOT_POINT && robot->kind != GTMP_ROBOT_DH_ARM)
    return report(err_msg, err_msg_len, bad, "unknown robot kind");
  const int dof = robot->dof;
  if (dof < 1 || dof > kMaxDof || (robot->kind == GTMP_ROBOT_POINT && dof > 3))
    return report(err_msg, err_msg_len, bad, "dof %d out of range", dof);
  if (!robot->q_lo || !robot->q_hi || !all_finite(robot->q_lo, dof) || !all_finite(robot->q_hi, dof))
    return report(err_msg, err_msg_len, bad, "bad joint box");
  for (int k = 0; k < dof; ++k)
    if (!(robot->q_hi[k] > robot->q_lo[k])) return report(err_msg, err_msg_len, bad, "joint box hi <= lo");
  if (M < 1 || L < 1 || L > 64 || H < 2 || H > 1024 || std::isnan(max_edge_len) || !(max_edge_len > 0.0f))
    return report(err_msg, err_msg_len, bad, "M, L, H or max_edge_len out of range");
  if (n_s < 0 || n_b < 0 || n_s + n_b > kNoallocMaxObstacles)
    return report(err_msg, err_msg_len, bad, "%d obstacles exceed the no-allocation limit of %d", n_s + n_b,
                  kNoallocMaxObstacles);
  if ((n_s > 0 && (!spheres || !all_finite(spheres, static_cast<size_t>(n_s) * 4))) ||
      (n_b > 0 && (!boxes || !all_finite(boxes, static_cast<size_t>(n_b) * 6))))
    return report(err_msg, err_msg_len, bad, "bad obstacle data");
  for (int k = 0; k < dof; ++k)
    if (!std::isfinite(q_start[k]) || !std::isfinite(q_goal[k]) || q_start[k] < robot->q_lo[k] ||
        q_start[k] > robot->q_hi[k] || q_goal[k] < robot->q_lo[k] || q_goal[k] > robot->q_hi[k])
      return report(err_msg, err_msg_len, bad, "endpoint outside the joint box");

  // ---- robot constants (kernel parameters) and kernel variant
  RobotDev rb{};
  rb.kind = robot->kind;
  rb.dof = dof;
  rb.point_radius = robot->point_radius;
  int variant = kVarPoint;
  int dp = 4;
  if (robot->kind == GTMP_ROBOT_DH_ARM) {
    const int spl = robot->spheres_per_link;
    if (!robot->dh || !robot->link_spheres || spl < 1 || spl > kMaxSpl ||
        !all_finite(robot->dh, static_cast<size_t>(dof) * 4) ||
        !all_finite(robot->link_spheres, static_cast<size_t>(dof) * spl * 4))
      return report(err_msg, err_msg_len, bad, "bad arm description");
    if (!arm_angles_in_range(robot->q_lo, robot->q_hi, robot->dh, dof))
      return report(err_msg, err_msg_len, bad, "joint limits beyond +-4096 rad or theta offset beyond +-2048 rad");
    bool uniform = true;
    const float r0 = robot->link_spheres[3];
    for (int s = 0; s < dof * spl; ++s) {
      if (!(robot->link_spheres[s * 4 + 3] > 0.0f)) return report(err_msg, err_msg_len, bad, "sphere radius <= 0");
      if (robot->link_spheres[s * 4 + 3] != r0) uniform = false;
    }
    variant = arm_kernel_variant(uniform, spl, dof, r0);
    const int stride = variant == kVarArmGeneric ? kMaxSpl : 4;
    dp = variant == kVarArmGeneric ? kMaxDof : 8;
    rb.spl = spl;
    rb.uniform_r = variant == kVarArmGeneric ? 0 : 1;
    rb.r_uniform = r0;
    for (int i = 0; i < dof; ++i) {
      rb.d[i] = robot->dh[i * 4 + 0];
      rb.a[i] = robot->dh[i * 4 + 1];
      rb.ca[i] = cosf(robot->dh[i * 4 + 2]);
      rb.sa[i] = sinf(robot->dh[i * 4 + 2]);
      rb.toff[i] = robot->dh[i * 4 + 3];
      for (int s = 0; s < spl; ++s) {
        const float* ls = robot->link_spheres + (static_cast<size_t>(i) * spl + s) * 4;
        rb.sph[i * stride + s] = make_float4(ls[0], ls[1], ls[2], ls[3]);
      }
    }
    fill_link_bounds(&rb);
  } else {
    if (!(robot->point_radius >= 0.0f) || !std::isfinite(robot->point_radius))
      return report(err_msg, err_msg_len, bad, "bad point radius");
    rb.spl = 1;
    rb.uniform_r = 1;
    rb.r_uniform = robot->point_radius;
  }

  // ---- host inputs for the staging launch (kernel parameters; no heap, no device allocation)
  for (int o = 0; o < n_s; ++o)
    if (!(spheres[4 * o + 3] >= 0.0f)) return report(err_msg, err_msg_len, bad, "negative sphere radius");
  for (int o = 0; o < n_b; ++o)
    for (int k = 0; k < 3; ++k)
      if (!(boxes[6 * o + 3 + k] >= boxes[6 * o + k])) return report(err_msg, err_msg_len, bad, "box with hi < lo");
  const bool packed = variant == kVarArm6x4 || variant == kVarArm7x4;
  NoallocStage stage;
  SceneDev sc{};
  int n4 = 0;  // float4 count of the obstacle table, as its builder reports it
  if (packed) {
    n4 = build_packed_tables(spheres, n_s, boxes, n_b, rb.r_uniform, arm_reach_bound(rb), stage.obs, &sc);
  } else {
    for (int o = 0; o < n_s; ++o) {
      const float* s = spheres + 4 * o;
      float w = s[3];
      if (rb.uniform_r) {
        const float rr = s[3] + rb.r_uniform;
        w = rr * rr;
      }
      stage.obs[o] = make_float4(s[0], s[1], s[2], w);
    }
    for (int o = 0; o < n_b; ++o) {
      const float* b = boxes + 6 * o;
      stage.obs[n_s + 2 * o] = make_float4(0.5f * (b[0] + b[3]), 0.5f * (b[1] + b[4]), 0.5f * (b[2] + b[5]),
                                           0.5f * (b[3] - b[0]));
      stage.obs[n_s + 2 * o + 1] = make_float4(0.5f * (b[4] - b[1]), 0.5f * (b[5] - b[2]), 0.0f, 0.0f);
    }
    sc.n_s = n_s;
    sc.n_b = n_b;
    n4 = n_s + 2 * n_b;
  }
  if (n4 < 0 || n4 > kNoallocTableCap)
    return report(err_msg, err_msg_len, GTMP_ERR_UNSUPPORTED, "obstacle table of %d float4 exceeds %d", n4,
                  kNoallocTableCap);
  stage.n4 = n4;
  stage.dp = dp;
  for (int k = 0; k < kMaxDof; ++k) {
    stage.ends[0][k] = k < dof ? q_start[k] : 0.0f;
    stage.ends[1][k] = k < dof ? q_goal[k] : 0.0f;
  }

  // ---- scratch layout and the size limit
  const size_t verts = static_cast<size_t>(L + 2) * M;
  size_t off = 0;
  const size_t off_err = off;
  off = align256(off + sizeof(int));
  const size_t off_counters = off;
  off = align256(off + static_cast<size_t>(L + 1) * sizeof(int));
  const size_t off_obs = off;
  off = align256(off + static_cast<size_t>(n4) * sizeof(float4));
  const size_t off_Q = off;
  off = align256(off + verts * dp * sizeof(float));
  const size_t off_keys = off;
  off = align256(off + verts * sizeof(unsigned long long));
  const size_t off_flags = off;
  off = align256(off + verts);
  if (off > kNoallocScratchBytes)
    return report(err_msg, err_msg_len, bad,
                  "M=%d, L=%d, dof=%d need %zu bytes of scratch; the no-allocation entry point has %zu",
                  M, L, dof, off, kNoallocScratchBytes);
  stage.goal_offset = static_cast<long long>(L + 1) * M * dp;

  // ---- device set-up (first call on this device) and launches
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return report(err_msg, err_msg_len, GTMP_ERR_CUDA, "cudaGetDevice: %s", cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices) return report(err_msg, err_msg_len, GTMP_ERR_UNSUPPORTED, "device %d", dev);
  if ((e = setup_device(dev)) != cudaSuccess)
    return report(err_msg, err_msg_len, GTMP_ERR_CUDA, "scratch set-up: %s", cudaGetErrorString(e));
  unsigned char* base = g_scratch_dev[dev];
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  int* err = reinterpret_cast<int*>(base + off_err);
  int* counters = reinterpret_cast<int*>(base + off_counters);
  float4* d_obs = reinterpret_cast<float4*>(base + off_obs);

  GraphDev g;
  g.Q = reinterpret_cast<float*>(base + off_Q);
  g.keys = reinterpret_cast<unsigned long long*>(base + off_keys);
  g.vflag = base + off_flags;
  g.R = 1;
  g.L = L;
  g.M = M;
  g.M_stride = M;
  g.dp = dp;
  g.H = H;
  g.max_edge_len = max_edge_len;
  sc.obs = d_obs;

#define NA_TRY(expr)                                                                                     \
  do {                                                                                                   \
    cudaError_t e_ = (expr);                                                                             \
    if (e_ != cudaSuccess)                                                                               \
      return report(err_msg, err_msg_len, GTMP_ERR_CUDA, "%s: %s", #expr, cudaGetErrorString(e_));      \
  } while (0)

  // error word (the one value that must start at zero), obstacle table and endpoints; everything
  // else in the scratch is written before it is read
  noalloc_stage_kernel<<<1, 256, 0, st>>>(stage, err, d_obs, g.Q);
  NA_TRY(cudaGetLastError());
  NA_TRY(launch_pack_layers(g, const_cast<float*>(dev_Q), dof, 1, st));
  NA_TRY(launch_init_keys(g, counters, L + 1, st));
  NA_TRY(launch_vertex_labels(g, rb, variant, sc, st));
  const int resident = g_num_sms[dev] * (g_bps[dev][variant] > 0 ? g_bps[dev][variant] : 1);
  for (int layer = L; layer >= 0; --layer) {
    const int rows = layer_size(g, layer), cols = layer_size(g, layer + 1);
    const long long edges = static_cast<long long>(rows) * cols;
    int grid_x = resident;
    long long chunk = edges / (static_cast<long long>(grid_x) * 8 * 8);
    if (chunk < 1) chunk = 1;
    if (chunk > 32) chunk = 32;
    if (variant == kVarPoint) chunk = 32;  // one edge per lane
    if (chunk > cols) chunk = cols;
    const long long n_chunks = rows * ((cols + chunk - 1) / chunk);
    if (grid_x > (n_chunks + 7) / 8) grid_x = static_cast<int>((n_chunks + 7) / 8);
    NA_TRY(launch_fused_transition(g, layer, rb, variant, sc, kEvalEarlyExit, counters + layer, grid_x,
                                   static_cast<int>(chunk), err, st));
  }
  NA_TRY(launch_extract_paths(g, dev_path, dev_cost, nullptr, st));
  if (dev_status) NA_TRY(cudaMemcpyAsync(dev_status, err, sizeof(int), cudaMemcpyDeviceToDevice, st));
#undef NA_TRY
  return GTMP_OK;
}
