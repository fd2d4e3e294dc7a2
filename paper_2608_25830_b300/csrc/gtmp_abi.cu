// C ABI of the layered-graph planner: argument checking, context memory, and
// the launch sequences of gtmp / anytime-gtmp / ao-gtmp (Alg. 1).
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <limits>
#include <string>
#include <vector>

#include "gtmp_ctx.h"

using namespace gtmp;


namespace {

gtmp_status fail(gtmp_ctx* c, gtmp_status s, const char* fmt, ...) {
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

#define CUDA_TRY(ctx, expr)                                                                              \
  do {                                                                                                   \
    cudaError_t e_ = (expr);                                                                             \
    if (e_ != cudaSuccess)                                                                               \
      return fail((ctx), e_ == cudaErrorMemoryAllocation ? GTMP_ERR_OOM : GTMP_ERR_CUDA, "%s: %s", #expr, \
                  cudaGetErrorString(e_));                                                               \
  } while (0)

bool finite_all(const float* v, size_t n) {
  for (size_t k = 0; k < n; ++k)
    if (!std::isfinite(v[k])) return false;
  return true;
}

GraphDev graph(gtmp_ctx* c, int R, int M) {
  GraphDev g;
  g.Q = c->Q;
  g.vflag = c->vflag;
  g.keys = c->keys;
  g.R = R;
  g.L = c->p.L;
  g.M = M;
  g.dp = c->dp;
  g.H = c->p.H;
  g.M_stride = c->p.M;
  g.max_edge_len = c->p.max_edge_len;
  g.G = c->G;
  g.gval = c->goal_values ? c->gval : nullptr;
  g.wb = c->wb;
  g.n_wb = c->n_wb;
  return g;
}

SceneDev scene(gtmp_ctx* c) {
  SceneDev s = c->sc;
  s.obs = c->obs;
  return s;
}

// q0 into layer 0 and the goal set into layer L + 1 of every graph, from the
// host copies (called again when the layer count changes)
gtmp_status upload_terminals(gtmp_ctx* c) {
  const int G = c->G;
  std::vector<float> s(static_cast<size_t>(c->p.R) * c->dp, 0.0f), g(static_cast<size_t>(c->p.R) * G * c->dp, 0.0f);
  for (int r = 0; r < c->p.R; ++r) {
    for (int k = 0; k < c->dof; ++k) s[static_cast<size_t>(r) * c->dp + k] = c->host_start[k];
    for (int i = 0; i < G; ++i)
      for (int k = 0; k < c->dof; ++k)
        g[(static_cast<size_t>(r) * G + i) * c->dp + k] = c->host_goals[static_cast<size_t>(i) * c->dof + k];
  }
  const size_t graph_stride = static_cast<size_t>(c->p.L + 2) * c->p.M * c->dp * sizeof(float);
  const size_t row = c->dp * sizeof(float), width = static_cast<size_t>(G) * row;
  CUDA_TRY(c, cudaMemcpy2DAsync(c->Q, graph_stride, s.data(), row, row, c->p.R, cudaMemcpyHostToDevice, c->stream));
  float* dst = c->Q + static_cast<size_t>(c->p.L + 1) * c->p.M * c->dp;
  CUDA_TRY(c, cudaMemcpy2DAsync(dst, graph_stride, g.data(), width, width, c->p.R, cudaMemcpyHostToDevice, c->stream));
  CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  return GTMP_OK;
}

bool uses_prefilter(int variant) { return variant == kVarArm6x4 || variant == kVarArm7x4; }

// layer sizes and chunking of one transition
void transition_shape(const GraphDev& g, int layer, int* rows, int* cols) {
  *rows = layer_size(g, layer);
  *cols = layer_size(g, layer + 1);
}

// count one enqueued kernel
#define LAUNCHED(ctx, n) ((ctx)->launches += (n))

cudaError_t event_at(gtmp_ctx* c, size_t slot, cudaEvent_t* out) {
  while (c->ev_pool.size() <= slot) {
    cudaEvent_t e;
    cudaError_t r = cudaEventCreate(&e);
    if (r != cudaSuccess) return r;
    c->ev_pool.push_back(e);
  }
  *out = c->ev_pool[slot];
  return cudaSuccess;
}

// The L + 1 fused transitions of a sweep, each after the first a programmatic
// dependent of the one before (it stages its obstacle table while that one
// finishes).  Timing covers the whole sweep with one event pair: events
// between the launches would serialise them.
gtmp_status run_fused(gtmp_ctx* c, const GraphDev& g, int mode) {
  const int bps = c->fused_bps[mode == GTMP_EVAL_FULL ? 1 : 0];
  const int resident = c->num_sms * bps;
  CUDA_TRY(c, launch_init_keys(g, c->counters, (g.L + 1) * g.R, c->stream));
  CUDA_TRY(c, launch_vertex_labels(g, c->rb, c->variant, scene(c), c->stream));
  LAUNCHED(c, 2);
  size_t slot = 0;
  if (c->timing) {
    slot = (c->ev_used.size() + c->ev_minplus.size()) * 2;
    cudaEvent_t e0 = nullptr;
    CUDA_TRY(c, event_at(c, slot, &e0));
    CUDA_TRY(c, cudaEventRecord(e0, c->stream));
  }
  for (int layer = g.L; layer >= 0; --layer) {
    int rows, cols;
    transition_shape(g, layer, &rows, &cols);
    const long long edges = static_cast<long long>(rows) * cols;
    int grid_x, chunk;
    if (mode == GTMP_EVAL_LAZY) {
      // a warp per (32-column block, row) unit: enough blocks for every unit, at most the resident count
      const long long units = static_cast<long long>(rows) * ((cols + 31) / 32);
      grid_x = static_cast<int>(std::max(1LL, std::min<long long>(resident / g.R, (units + 7) / 8)));
      chunk = 32;
    } else {
      grid_x = std::max(1, resident / g.R);
      const long long warps = static_cast<long long>(grid_x) * 8;
      long long ch = edges / (warps * 8);
      if (ch < 1) ch = 1;
      if (ch > 32) ch = 32;
      if (c->variant == kVarPoint) ch = 32;  // one edge per lane
      if (ch > cols) ch = cols;
      const long long n_chunks = rows * ((cols + ch - 1) / ch);
      const long long useful_blocks = (n_chunks + 7) / 8;
      if (grid_x > useful_blocks) grid_x = static_cast<int>(useful_blocks);
      chunk = static_cast<int>(ch);
    }
    CUDA_TRY(c, launch_fused_transition(g, layer, c->rb, c->variant, scene(c), mode, c->counters + layer * g.R,
                                        grid_x, chunk, c->err, c->stream, layer < g.L));
    LAUNCHED(c, 1);
    if (c->timing) {
      c->fused_timed_launches += 1;
      c->timed_edges += static_cast<double>(edges) * g.R;
    }
  }
  if (c->timing) {
    cudaEvent_t e1 = nullptr;
    CUDA_TRY(c, event_at(c, slot + 1, &e1));
    CUDA_TRY(c, cudaEventRecord(e1, c->stream));
    c->ev_used.emplace_back(static_cast<int>(slot), static_cast<int>(slot + 1));
  }
  return GTMP_OK;
}

// the context's layer sampler (uniform in the joint box, or on C_free by rejection)
cudaError_t sample_layers_of(gtmp_ctx* c, const GraphDev& g, uint64_t seed) {
  if (c->sampler == GTMP_SAMPLER_FREE)
    return launch_sample_free(g, c->rb, c->variant, scene(c), c->q_lo, c->q_hi, c->dof, seed, 0, c->sampler_attempts,
                              c->stream);
  return launch_sample_uniform(g, c->q_lo, c->q_hi, c->dof, seed, 0, c->stream);
}

gtmp_status check_ready(gtmp_ctx* c) {
  if (!c->have_endpoints) return fail(c, GTMP_ERR_NOT_READY, "endpoints not set (gtmp_set_endpoints)");
  if (c->M_active < 1) return fail(c, GTMP_ERR_NOT_READY, "no samples (gtmp_sample_layers / gtmp_set_layers)");
  return GTMP_OK;
}

}  // namespace

// Step 1 of the unfused variant, shared with the class-augmented sweep: vertex
// labels and every transition's cost matrix C_l (C_L first, so that, when the
// matrices outgrow L2, the sweep that follows reads each from HBM).
gtmp_status gtmp_internal_edge_costs(gtmp_ctx* c) {
  const int L = c->p.L;
  if (!c->C) {
    GraphDev cap = graph(c, 1, c->p.M);
    size_t total = 0;
    c->c_off.assign(L + 2, 0);
    c->c_cs.assign(L + 1, 0);
    for (int layer = 0; layer <= L; ++layer) {
      int rows, cols;
      transition_shape(cap, layer, &rows, &cols);
      c->c_cs[layer] = ((cols + 3) / 4) * 4;
      c->c_off[layer] = total;
      total += static_cast<size_t>(rows) * c->c_cs[layer];
    }
    c->c_off[L + 1] = total;
    CUDA_TRY(c, cudaMalloc(&c->C, total * sizeof(float)));
  }
  GraphDev g = graph(c, 1, c->M_active);
  CUDA_TRY(c, launch_init_keys(g, c->counters, (L + 1), c->stream));
  CUDA_TRY(c, launch_vertex_labels(g, c->rb, c->variant, scene(c), c->stream));
  LAUNCHED(c, 2);
  const int resident = c->num_sms * c->fused_bps[0];
  for (int layer = L; layer >= 0; --layer) {
    int rows, cols;
    transition_shape(g, layer, &rows, &cols);
    // the unfused step recomputes its own row stride for the active M
    const int cs = ((cols + 3) / 4) * 4;
    c->c_cs[layer] = cs;
    const long long edges = static_cast<long long>(rows) * cols;
    long long chunk = edges / (static_cast<long long>(resident) * 64);
    if (chunk < 1) chunk = 1;
    if (chunk > 32) chunk = 32;
    if (chunk > cols) chunk = cols;
    const long long n_chunks = rows * ((cols + chunk - 1) / chunk);
    int grid = resident;
    if (grid > (n_chunks + 7) / 8) grid = static_cast<int>((n_chunks + 7) / 8);
    CUDA_TRY(c, launch_edge_costs(g, layer, c->rb, c->variant, scene(c), c->C + c->c_off[layer], cs,
                                  c->counters + layer, grid, static_cast<int>(chunk), c->err, c->stream));
    LAUNCHED(c, 1);
  }
  return GTMP_OK;
}

extern "C" {

const char* gtmp_status_string(gtmp_status s) {
  switch (s) {
    case GTMP_OK: return "GTMP_OK";
    case GTMP_ERR_INVALID_ARG: return "GTMP_ERR_INVALID_ARG";
    case GTMP_ERR_CUDA: return "GTMP_ERR_CUDA";
    case GTMP_ERR_OOM: return "GTMP_ERR_OOM";
    case GTMP_ERR_TIMEOUT: return "GTMP_ERR_TIMEOUT";
    case GTMP_ERR_UNSUPPORTED: return "GTMP_ERR_UNSUPPORTED";
    case GTMP_ERR_NOT_READY: return "GTMP_ERR_NOT_READY";
  }
  return "GTMP_ERR_UNKNOWN";
}

const char* gtmp_last_error(const gtmp_ctx* ctx) { return ctx ? ctx->last_error.c_str() : "null context"; }

gtmp_status gtmp_create(const gtmp_robot* robot, const gtmp_params* params, void* cuda_stream, gtmp_ctx** out) {
  if (!out || !robot || !params) return GTMP_ERR_INVALID_ARG;
  *out = nullptr;
  // --- validate everything before touching the GPU
  const gtmp_params& p = *params;
  if (robot->kind != GTMP_ROBOT_POINT && robot->kind != GTMP_ROBOT_DH_ARM) return GTMP_ERR_INVALID_ARG;
  if (robot->dof < 1 || robot->dof > kMaxDof) return GTMP_ERR_INVALID_ARG;
  if (robot->kind == GTMP_ROBOT_POINT && robot->dof > 3) return GTMP_ERR_INVALID_ARG;
  if (!robot->q_lo || !robot->q_hi) return GTMP_ERR_INVALID_ARG;
  if (!finite_all(robot->q_lo, robot->dof) || !finite_all(robot->q_hi, robot->dof)) return GTMP_ERR_INVALID_ARG;
  for (int k = 0; k < robot->dof; ++k)
    if (!(robot->q_hi[k] > robot->q_lo[k])) return GTMP_ERR_INVALID_ARG;
  if (robot->kind == GTMP_ROBOT_DH_ARM) {
    if (!robot->dh || !robot->link_spheres) return GTMP_ERR_INVALID_ARG;
    if (robot->spheres_per_link < 1 || robot->spheres_per_link > kMaxSpl) return GTMP_ERR_INVALID_ARG;
    if (!finite_all(robot->dh, static_cast<size_t>(robot->dof) * 4)) return GTMP_ERR_INVALID_ARG;
    if (!arm_angles_in_range(robot->q_lo, robot->q_hi, robot->dh, robot->dof)) return GTMP_ERR_INVALID_ARG;
    const size_t ns = static_cast<size_t>(robot->dof) * robot->spheres_per_link;
    if (!finite_all(robot->link_spheres, ns * 4)) return GTMP_ERR_INVALID_ARG;
    for (size_t s = 0; s < ns; ++s)
      if (!(robot->link_spheres[s * 4 + 3] > 0.0f)) return GTMP_ERR_INVALID_ARG;
  } else if (!(robot->point_radius >= 0.0f) || !std::isfinite(robot->point_radius)) {
    return GTMP_ERR_INVALID_ARG;
  }
  if (p.M < 1 || p.M > 16384 || p.L < 1 || p.L > 64 || p.H < 2 || p.H > 1024 || p.R < 1 || p.R > 4096 ||
      p.max_obstacles < 0 || p.max_obstacles > 4096 ||
      (p.eval_mode != GTMP_EVAL_EARLY_EXIT && p.eval_mode != GTMP_EVAL_FULL && p.eval_mode != GTMP_EVAL_LAZY) ||
      std::isnan(p.max_edge_len) ||
      !(p.max_edge_len > 0.0f))
    return GTMP_ERR_INVALID_ARG;
  const size_t graph_vertices = static_cast<size_t>(p.R) * (p.L + 2) * p.M;
  if (graph_vertices > (size_t(1) << 31)) return GTMP_ERR_INVALID_ARG;

  gtmp_ctx* c = new gtmp_ctx();
  c->p = p;
  c->L_cap = p.L;
  c->stream = static_cast<cudaStream_t>(cuda_stream);
  c->dof = robot->dof;
  // --- robot constants
  RobotDev& rb = c->rb;
  rb.kind = robot->kind;
  rb.dof = robot->dof;
  rb.point_radius = robot->point_radius;
  for (int k = 0; k < robot->dof; ++k) {
    c->q_lo[k] = robot->q_lo[k];
    c->q_hi[k] = robot->q_hi[k];
  }
  if (robot->kind == GTMP_ROBOT_DH_ARM) {
    rb.spl = robot->spheres_per_link;
    bool uniform = true;
    const float r0 = robot->link_spheres[3];
    for (int i = 0; i < robot->dof; ++i) {
      rb.d[i] = robot->dh[i * 4 + 0];
      rb.a[i] = robot->dh[i * 4 + 1];
      rb.ca[i] = cosf(robot->dh[i * 4 + 2]);
      rb.sa[i] = sinf(robot->dh[i * 4 + 2]);
      rb.toff[i] = robot->dh[i * 4 + 3];
    }
    // sphere table laid out [link][stride] with stride = 4 for the 4-sphere
    // variants and kMaxSpl for the generic one
    for (int i = 0; i < robot->dof; ++i)
      for (int s = 0; s < robot->spheres_per_link; ++s) {
        const float* ls = robot->link_spheres + (static_cast<size_t>(i) * robot->spheres_per_link + s) * 4;
        if (ls[3] != r0) uniform = false;
      }
    rb.r_uniform = r0;
    c->variant = arm_kernel_variant(uniform, robot->spheres_per_link, robot->dof, r0);
    // the specialised kernels read inflated squared thresholds (r_obs + r)^2,
    // the generic kernel reads plain obstacle radii
    rb.uniform_r = (c->variant == kVarArmGeneric) ? 0 : 1;
    const int stride = (c->variant == kVarArmGeneric) ? kMaxSpl : 4;
    for (int i = 0; i < robot->dof; ++i)
      for (int s = 0; s < robot->spheres_per_link; ++s) {
        const float* ls = robot->link_spheres + (static_cast<size_t>(i) * robot->spheres_per_link + s) * 4;
        rb.sph[i * stride + s] = make_float4(ls[0], ls[1], ls[2], ls[3]);
      }
    fill_link_bounds(&rb);
    c->dp = 8;
  } else {
    rb.spl = 1;
    rb.uniform_r = 1;
    rb.r_uniform = robot->point_radius;
    c->variant = kVarPoint;
    c->dp = 4;
  }
  if (c->variant == kVarArmGeneric) c->dp = kMaxDof;  // generic kernels read kMaxDof padded floats
  // --- device memory
  cudaError_t e = cudaGetDevice(&c->device);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, c->device);
  auto alloc = [&](void** ptr, size_t bytes) {
    if (e == cudaSuccess) e = cudaMalloc(ptr, bytes > 0 ? bytes : 16);
  };
  alloc(reinterpret_cast<void**>(&c->Q), graph_vertices * c->dp * sizeof(float));
  alloc(reinterpret_cast<void**>(&c->vflag), graph_vertices);
  alloc(reinterpret_cast<void**>(&c->keys), graph_vertices * sizeof(unsigned long long));
  c->n_counters = (p.L + 1) * p.R;
  alloc(reinterpret_cast<void**>(&c->counters), static_cast<size_t>(c->n_counters) * sizeof(int));
  // scalar table (<= 2 float4 per obstacle) or packed tables (<= 3 (n_s + n_b) + 8 float4)
  alloc(reinterpret_cast<void**>(&c->obs), (packed_table_capacity(p.max_obstacles) + kMaxGridCells / 4) * sizeof(float4));
  alloc(reinterpret_cast<void**>(&c->err), sizeof(int));
  if (e == cudaSuccess) e = cudaMemsetAsync(c->Q, 0, graph_vertices * c->dp * sizeof(float), c->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(c->err, 0, sizeof(int), c->stream);
  if (e == cudaSuccess) e = configure_kernels(200 * 1024);
  if (e == cudaSuccess) {
    c->fused_bps[0] = fused_max_blocks_per_sm(c->variant, GTMP_EVAL_EARLY_EXIT);
    c->fused_bps[1] = fused_max_blocks_per_sm(c->variant, GTMP_EVAL_FULL);
    e = cudaStreamSynchronize(c->stream);
  }
  if (e != cudaSuccess) {
    gtmp_status s = e == cudaErrorMemoryAllocation ? GTMP_ERR_OOM : GTMP_ERR_CUDA;
    gtmp_destroy(c);
    return s;
  }
  *out = c;
  return GTMP_OK;
}

gtmp_status gtmp_destroy(gtmp_ctx* c) {
  if (!c) return GTMP_OK;
  cudaStreamSynchronize(c->stream);
  cudaFree(c->Q);
  cudaFree(c->vflag);
  cudaFree(c->keys);
  cudaFree(c->counters);
  cudaFree(c->obs);
  cudaFree(c->err);
  cudaFree(c->C);
  cudaFree(c->cls);
  cudaFree(c->gval);
  cudaFree(c->wb);
  cudaFree(c->ao_scratch);
  cudaFree(c->prune);
  cudaFree(c->lazy_bad);
  cudaFree(c->lazy_count);
  surrogate_free(c->sur);
  for (cudaEvent_t e : c->ev_pool) cudaEventDestroy(e);
  delete c;
  return GTMP_OK;
}

gtmp_status gtmp_set_stream(gtmp_ctx* c, void* cuda_stream) {
  if (!c) return GTMP_ERR_INVALID_ARG;
  c->stream = static_cast<cudaStream_t>(cuda_stream);
  return GTMP_OK;
}

gtmp_status gtmp_synchronize(gtmp_ctx* c) {
  if (!c) return GTMP_ERR_INVALID_ARG;
  CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  int err = 0;
  CUDA_TRY(c, cudaMemcpy(&err, c->err, sizeof(int), cudaMemcpyDeviceToHost));
  if (err) {
    CUDA_TRY(c, cudaMemset(c->err, 0, sizeof(int)));
    return fail(c, GTMP_ERR_TIMEOUT, "device error flags 0x%x (1 = sampler exhausted, 2 = wait timed out)", err);
  }
  return GTMP_OK;
}

gtmp_status gtmp_set_obstacles(gtmp_ctx* c, const float* spheres, int32_t n_s, const float* boxes, int32_t n_b) {
  GtmpNvtxRange nvtx_("gtmp_set_obstacles");
  if (!c) return GTMP_ERR_INVALID_ARG;
  if (n_s < 0 || n_b < 0 || n_s + n_b > c->p.max_obstacles)
    return fail(c, GTMP_ERR_INVALID_ARG, "obstacle count %d + %d exceeds capacity %d", n_s, n_b, c->p.max_obstacles);
  if ((n_s > 0 && !spheres) || (n_b > 0 && !boxes)) return fail(c, GTMP_ERR_INVALID_ARG, "NULL obstacle array");
  if ((n_s > 0 && !finite_all(spheres, static_cast<size_t>(n_s) * 4)) ||
      (n_b > 0 && !finite_all(boxes, static_cast<size_t>(n_b) * 6)))
    return fail(c, GTMP_ERR_INVALID_ARG, "non-finite obstacle data");
  SceneDev sc{};
  std::vector<float4> host;
  if (uses_prefilter(c->variant)) {
    for (int o = 0; o < n_s; ++o)
      if (!(spheres[4 * o + 3] >= 0.0f)) return fail(c, GTMP_ERR_INVALID_ARG, "negative sphere radius");
    for (int o = 0; o < n_b; ++o)
      for (int k = 0; k < 3; ++k)
        if (!(boxes[6 * o + 3 + k] >= boxes[6 * o + k])) return fail(c, GTMP_ERR_INVALID_ARG, "box with hi < lo");
    host.resize(packed_table_capacity(n_s + n_b) + kMaxGridCells / 4);
    int n4 = build_packed_tables(spheres, n_s, boxes, n_b, c->rb.r_uniform, arm_reach_bound(c->rb), host.data(),
                                 &sc);
    // cull grid within the shared memory that keeps two edge-kernel blocks per SM
    // (table + grid + the column layer's cost-to-go <= ~110 KB per block)
    double R_link = 0.0;
    for (int i = 0; i < c->dof; ++i) R_link = std::fmax(R_link, static_cast<double>(c->rb.lb[i].w));
    const long long budget = (110LL * 1024 - 4LL * c->p.M - 16LL * n4 - 2048) / 4;
    const int max_cells = static_cast<int>(std::min<long long>(kMaxGridCells, std::max<long long>(budget, 0)));
    if (n4 + max_cells / 4 + 1 <= kMaxTableFloat4s)
      n4 += build_cull_grid(spheres, n_s, boxes, n_b, R_link, max_cells, host.data() + n4, &sc);
    host.resize(n4);
  } else {
    host.resize(static_cast<size_t>(n_s) + 2 * static_cast<size_t>(n_b));
    for (int o = 0; o < n_s; ++o) {
      const float* s = spheres + 4 * o;
      if (!(s[3] >= 0.0f)) return fail(c, GTMP_ERR_INVALID_ARG, "negative sphere radius");
      float w = s[3];
      if (c->rb.uniform_r) {
        const float rr = s[3] + c->rb.r_uniform;
        w = rr * rr;  // inflated squared threshold
      }
      host[o] = make_float4(s[0], s[1], s[2], w);
    }
    for (int o = 0; o < n_b; ++o) {
      const float* b = boxes + 6 * o;
      for (int k = 0; k < 3; ++k)
        if (!(b[3 + k] >= b[k])) return fail(c, GTMP_ERR_INVALID_ARG, "box with hi < lo");
      const float cx = 0.5f * (b[0] + b[3]), cy = 0.5f * (b[1] + b[4]), cz = 0.5f * (b[2] + b[5]);
      const float hx = 0.5f * (b[3] - b[0]), hy = 0.5f * (b[4] - b[1]), hz = 0.5f * (b[5] - b[2]);
      host[n_s + 2 * o] = make_float4(cx, cy, cz, hx);
      host[n_s + 2 * o + 1] = make_float4(hy, hz, 0.0f, 0.0f);
    }
    sc.n_s = n_s;
    sc.n_b = n_b;
  }
  if (!host.empty())
    CUDA_TRY(c, cudaMemcpyAsync(c->obs, host.data(), host.size() * sizeof(float4), cudaMemcpyHostToDevice, c->stream));
  CUDA_TRY(c, cudaStreamSynchronize(c->stream));  // the host vector goes out of scope
  c->sc = sc;
  // obstacle centres in the plane, kept for the class-augmented sweep (its labels
  // wind about these points; float64 sums of float32 inputs are exact)
  c->centres.clear();
  for (int o = 0; o < n_s; ++o) c->centres.emplace_back(double(spheres[4 * o]), double(spheres[4 * o + 1]));
  for (int o = 0; o < n_b; ++o) {
    const float* b = boxes + 6 * o;
    c->centres.emplace_back(0.5 * (double(b[0]) + double(b[3])), 0.5 * (double(b[1]) + double(b[4])));
  }
  return GTMP_OK;
}

gtmp_status gtmp_set_endpoints(gtmp_ctx* c, const float* q_start, const float* q_goal) {
  if (!c || !q_start || !q_goal) return fail(c, GTMP_ERR_INVALID_ARG, "NULL endpoint");
  for (int k = 0; k < c->dof; ++k) {
    if (!std::isfinite(q_start[k]) || !std::isfinite(q_goal[k]))
      return fail(c, GTMP_ERR_INVALID_ARG, "non-finite endpoint");
    if (q_start[k] < c->q_lo[k] || q_start[k] > c->q_hi[k] || q_goal[k] < c->q_lo[k] || q_goal[k] > c->q_hi[k])
      return fail(c, GTMP_ERR_INVALID_ARG, "endpoint outside the joint box (coordinate %d)", k);
  }
  c->host_start.assign(q_start, q_start + c->dof);
  c->host_goals.assign(q_goal, q_goal + c->dof);
  c->G = 1;
  c->goal_values = false;
  gtmp_status st = upload_terminals(c);
  if (st == GTMP_OK) c->have_endpoints = true;
  return st;
}

gtmp_status gtmp_set_goals(gtmp_ctx* c, const float* goals, const float* values, int32_t G) {
  if (!c || !goals) return fail(c, GTMP_ERR_INVALID_ARG, "NULL goal array");
  if (!c->have_endpoints) return fail(c, GTMP_ERR_NOT_READY, "set the start with gtmp_set_endpoints first");
  if (G < 1 || G > c->p.M) return fail(c, GTMP_ERR_INVALID_ARG, "goal count %d outside [1, M = %d]", G, c->p.M);
  for (int i = 0; i < G; ++i) {
    for (int k = 0; k < c->dof; ++k) {
      const float q = goals[static_cast<size_t>(i) * c->dof + k];
      if (!std::isfinite(q) || q < c->q_lo[k] || q > c->q_hi[k])
        return fail(c, GTMP_ERR_INVALID_ARG, "goal %d non-finite or outside the joint box", i);
    }
    if (values && !(std::isfinite(values[i]) && values[i] >= 0.0f))
      return fail(c, GTMP_ERR_INVALID_ARG, "goal value %d must be finite and >= 0", i);
  }
  if (values) {
    if (!c->gval) CUDA_TRY(c, cudaMalloc(&c->gval, static_cast<size_t>(c->p.M) * sizeof(float)));
    CUDA_TRY(c, cudaMemcpyAsync(c->gval, values, G * sizeof(float), cudaMemcpyHostToDevice, c->stream));
  }
  c->host_goals.assign(goals, goals + static_cast<size_t>(G) * c->dof);
  c->G = G;
  c->goal_values = values != nullptr;
  return upload_terminals(c);
}

gtmp_status gtmp_set_num_layers(gtmp_ctx* c, int32_t L) {
  if (!c) return GTMP_ERR_INVALID_ARG;
  if (L < 1 || L > c->L_cap) return fail(c, GTMP_ERR_INVALID_ARG, "layer count %d outside [1, %d]", L, c->L_cap);
  CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  c->p.L = L;
  c->M_active = 0;  // the samples of the old layout are gone
  cudaFree(c->C);   // stored cost matrices are laid out per transition
  c->C = nullptr;
  c->c_off.clear();
  c->c_cs.clear();
  return c->have_endpoints ? upload_terminals(c) : GTMP_OK;
}

gtmp_status gtmp_set_max_edge_len(gtmp_ctx* c, float max_edge_len) {
  if (!c) return GTMP_ERR_INVALID_ARG;
  if (std::isnan(max_edge_len) || !(max_edge_len > 0.0f))
    return fail(c, GTMP_ERR_INVALID_ARG, "edge-length limit must be > 0 (+inf: none)");
  c->p.max_edge_len = max_edge_len;
  return GTMP_OK;
}

gtmp_status gtmp_set_cost_weight(gtmp_ctx* c, const float* bumps, int32_t K) {
  GtmpNvtxRange nvtx_("gtmp_set_cost_weight");
  if (!c) return GTMP_ERR_INVALID_ARG;
  if (K < 0 || K > GTMP_MAX_WEIGHT_BUMPS || (K > 0 && !bumps))
    return fail(c, GTMP_ERR_INVALID_ARG, "bump count %d outside [0, %d] or NULL bumps", K, GTMP_MAX_WEIGHT_BUMPS);
  const int stride = c->dp / 4 + 1;  // float4 per bump: centre (dp floats), then (1 / s^2, a, 0, 0)
  std::vector<float4> img(static_cast<size_t>(K) * stride, make_float4(0.0f, 0.0f, 0.0f, 0.0f));
  double w_max = 1.0;
  for (int b = 0; b < K; ++b) {
    const float* p = bumps + static_cast<size_t>(b) * (c->dof + 2);
    if (!finite_all(p, c->dof + 2)) return fail(c, GTMP_ERR_INVALID_ARG, "bump %d has a non-finite value", b);
    const double s = p[c->dof], a = p[c->dof + 1];
    const float inv_s2 = static_cast<float>(1.0 / (s * s));
    if (!(s > 0.0) || !std::isfinite(inv_s2) || !(a >= 0.0))
      return fail(c, GTMP_ERR_INVALID_ARG, "bump %d needs radius > 0 (1/s^2 finite) and amplitude >= 0", b);
    w_max += a;
    float* cen = reinterpret_cast<float*>(&img[static_cast<size_t>(b) * stride]);
    for (int k = 0; k < c->dof; ++k) cen[k] = p[k];
    img[static_cast<size_t>(b) * stride + stride - 1] = make_float4(inv_s2, static_cast<float>(a), 0.0f, 0.0f);
  }
  if (!std::isfinite(static_cast<float>(w_max)))
    return fail(c, GTMP_ERR_INVALID_ARG, "the weight's maximum 1 + sum a_b overflows float32");
  if (K > 0) {
    if (!c->wb)
      CUDA_TRY(c, cudaMalloc(&c->wb, static_cast<size_t>(GTMP_MAX_WEIGHT_BUMPS) * stride * sizeof(float4)));
    CUDA_TRY(c, cudaMemcpyAsync(c->wb, img.data(), img.size() * sizeof(float4), cudaMemcpyHostToDevice, c->stream));
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  }
  c->n_wb = K;
  return GTMP_OK;
}

gtmp_status gtmp_cull_grid(const float* spheres, int32_t n_s, const float* boxes, int32_t n_b, float R_link,
                           int32_t max_cells, uint32_t* masks, int32_t* dims, float* origin_inv) {
  if (n_s < 0 || n_b < 0 || (n_s > 0 && !spheres) || (n_b > 0 && !boxes) || !masks || !dims || !origin_inv ||
      !(R_link > 0.0f) || !std::isfinite(R_link) || max_cells < 0 || max_cells > kMaxGridCells || n_s + n_b > 4096)
    return GTMP_ERR_INVALID_ARG;
  if ((n_s > 0 && !finite_all(spheres, static_cast<size_t>(n_s) * 4)) ||
      (n_b > 0 && !finite_all(boxes, static_cast<size_t>(n_b) * 6)))
    return GTMP_ERR_INVALID_ARG;
  SceneDev sc{};
  std::vector<float4> host(packed_table_capacity(n_s + n_b) + kMaxGridCells / 4 + 1);
  const int n4 = build_packed_tables(spheres, n_s, boxes, n_b, 0.0f, 4.0, host.data(), &sc);
  const int g4 = build_cull_grid(spheres, n_s, boxes, n_b, R_link, max_cells, host.data() + n4, &sc);
  dims[0] = sc.gnx;
  dims[1] = sc.gny;
  dims[2] = sc.gnz;
  origin_inv[0] = sc.glx;
  origin_inv[1] = sc.gly;
  origin_inv[2] = sc.glz;
  origin_inv[3] = sc.ginv;
  if (g4 > 0)
    std::memcpy(masks, host.data() + n4, static_cast<size_t>(sc.gnx) * sc.gny * sc.gnz * sizeof(uint32_t));
  return GTMP_OK;
}

gtmp_status gtmp_set_sampler(gtmp_ctx* c, int32_t sampler, int32_t max_attempts) {
  if (!c || (sampler != GTMP_SAMPLER_UNIFORM && sampler != GTMP_SAMPLER_FREE) || max_attempts < 1 ||
      max_attempts > (1 << 20))
    return fail(c, GTMP_ERR_INVALID_ARG, "sampler must be GTMP_SAMPLER_UNIFORM or _FREE, attempts in [1, 2^20]");
  c->sampler = sampler;
  c->sampler_attempts = max_attempts;
  return GTMP_OK;
}

gtmp_status gtmp_get_goal_reached(gtmp_ctx* c, int32_t gi, int32_t* dev_goal) {
  if (!c || !dev_goal || gi < 0 || gi >= c->p.R) return fail(c, GTMP_ERR_INVALID_ARG, "bad request");
  if (c->M_active < 1) return fail(c, GTMP_ERR_NOT_READY, "no samples");
  GraphDev g = graph(c, c->p.R, c->M_active);
  CUDA_TRY(c, launch_goal_reached(g, gi, dev_goal, c->stream));
  LAUNCHED(c, 1);
  return GTMP_OK;
}

gtmp_status gtmp_sample_layers(gtmp_ctx* c, uint64_t seed, int32_t M) {
  GtmpNvtxRange nvtx_("gtmp_sample_layers");
  if (!c) return GTMP_ERR_INVALID_ARG;
  if (M < 1 || M > c->p.M) return fail(c, GTMP_ERR_INVALID_ARG, "M=%d outside 1..%d", M, c->p.M);
  GraphDev g = graph(c, 1, M);
  CUDA_TRY(c, sample_layers_of(c, g, seed));
  LAUNCHED(c, 1);
  c->M_active = M;
  return GTMP_OK;
}

gtmp_status gtmp_set_layers(gtmp_ctx* c, const float* dev_Q, int32_t M) {
  if (!c || !dev_Q) return fail(c, GTMP_ERR_INVALID_ARG, "NULL samples");
  if (M < 1 || M > c->p.M) return fail(c, GTMP_ERR_INVALID_ARG, "M=%d outside 1..%d", M, c->p.M);
  GraphDev g = graph(c, 1, M);
  CUDA_TRY(c, launch_pack_layers(g, const_cast<float*>(dev_Q), c->dof, 1, c->stream));
  LAUNCHED(c, 1);
  c->M_active = M;
  return GTMP_OK;
}

gtmp_status gtmp_get_layers(gtmp_ctx* c, float* dev_Q) {
  if (!c || !dev_Q) return fail(c, GTMP_ERR_INVALID_ARG, "NULL output");
  if (c->M_active < 1) return fail(c, GTMP_ERR_NOT_READY, "no samples");
  GraphDev g = graph(c, 1, c->M_active);
  CUDA_TRY(c, launch_pack_layers(g, dev_Q, c->dof, 0, c->stream));
  LAUNCHED(c, 1);
  return GTMP_OK;
}

gtmp_status gtmp_profile_enable(gtmp_ctx* c, int32_t enable) {
  if (!c) return GTMP_ERR_INVALID_ARG;
  c->timing = enable != 0;
  return GTMP_OK;
}

gtmp_status gtmp_profile_read(gtmp_ctx* c, gtmp_profile* out) {
  if (!c || !out) return fail(c, GTMP_ERR_INVALID_ARG, "NULL output");
  CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  double ms = 0.0;
  for (const auto& pr : c->ev_used) {
    float t = 0.0f;
    CUDA_TRY(c, cudaEventElapsedTime(&t, c->ev_pool[pr.first], c->ev_pool[pr.second]));
    ms += t;
  }
  out->launches = c->launches;
  out->fused_launches = c->fused_timed_launches;
  out->fused_ms = ms;
  out->fused_edges = c->timed_edges;
  double mp = 0.0;
  for (const auto& pr : c->ev_minplus) {
    float t = 0.0f;
    CUDA_TRY(c, cudaEventElapsedTime(&t, c->ev_pool[pr.first], c->ev_pool[pr.second]));
    mp += t;
  }
  out->minplus_launches = c->minplus_launches;
  out->minplus_ms = mp;
  out->minplus_bytes = c->minplus_bytes;
  c->launches = 0;
  c->fused_timed_launches = 0;
  c->ev_used.clear();
  c->timed_edges = 0.0;
  c->ev_minplus.clear();
  c->minplus_bytes = 0.0;
  c->minplus_launches = 0;
  return GTMP_OK;
}

gtmp_status gtmp_get_M(const gtmp_ctx* c, int32_t* M) {
  if (!c || !M) return GTMP_ERR_INVALID_ARG;
  *M = c->M_active;
  return GTMP_OK;
}

gtmp_status gtmp_joint_sincos(const float* dev_x, int32_t n, float* dev_s, float* dev_c, void* cuda_stream) {
  if (n < 0 || (n > 0 && (!dev_x || !dev_s || !dev_c))) return GTMP_ERR_INVALID_ARG;
  return launch_joint_sincos(dev_x, n, dev_s, dev_c, static_cast<cudaStream_t>(cuda_stream)) == cudaSuccess
             ? GTMP_OK
             : GTMP_ERR_CUDA;
}

gtmp_status gtmp_label_configs(gtmp_ctx* c, const float* dev_q, int32_t n, uint8_t* dev_labels) {
  if (!c || n < 0 || (n > 0 && (!dev_q || !dev_labels))) return fail(c, GTMP_ERR_INVALID_ARG, "bad label request");
  CUDA_TRY(c, launch_label_configs(dev_q, n, c->dof, c->rb, c->variant, scene(c), dev_labels, c->stream));
  if (n > 0) LAUNCHED(c, 1);
  return GTMP_OK;
}

gtmp_status gtmp_solve(gtmp_ctx* c, int32_t* dev_path, float* dev_cost) {
  GtmpNvtxRange nvtx_("gtmp_solve");
  if (!c || !dev_path || !dev_cost) return fail(c, GTMP_ERR_INVALID_ARG, "NULL output");
  gtmp_status s = check_ready(c);
  if (s != GTMP_OK) return s;
  GraphDev g = graph(c, 1, c->M_active);
  if ((s = run_fused(c, g, c->p.eval_mode)) != GTMP_OK) return s;
  CUDA_TRY(c, launch_extract_paths(g, dev_path, dev_cost, nullptr, c->stream));
  LAUNCHED(c, 1);
  return GTMP_OK;
}

gtmp_status gtmp_solve_lazy_path(gtmp_ctx* c, int32_t max_iterations, int32_t* dev_path, float* dev_cost,
                                 gtmp_lazy_stats* stats) {
  GtmpNvtxRange nvtx_("gtmp_solve_lazy_path");
  if (!c || !dev_path || !dev_cost || max_iterations < 1) return fail(c, GTMP_ERR_INVALID_ARG, "bad lazy request");
  gtmp_status s = check_ready(c);
  if (s != GTMP_OK) return s;
  const GraphDev g = graph(c, 1, c->M_active);
  const size_t words = (static_cast<size_t>(c->p.M) * c->p.M + 31) / 32;
  if (c->lazy_words != words || !c->lazy_bad) {
    cudaFree(c->lazy_bad);
    c->lazy_bad = nullptr;
    c->lazy_words = 0;
    // (L_cap + 1) transitions of M x M bits
    CUDA_TRY(c, cudaMalloc(&c->lazy_bad, (static_cast<size_t>(c->L_cap) + 1) * words * sizeof(uint32_t)));
    c->lazy_words = words;
  }
  if (!c->lazy_count) CUDA_TRY(c, cudaMalloc(&c->lazy_count, kLazyStateInts * sizeof(int)));
  cudaStream_t st = c->stream;
  CUDA_TRY(c, cudaMemsetAsync(c->lazy_bad, 0, (static_cast<size_t>(g.L) + 1) * words * sizeof(uint32_t), st));
  int state[kLazyStateInts] = {0, -1, g.L, 0, 0, 0};  // the first sweep covers every transition
  CUDA_TRY(c, cudaMemcpyAsync(c->lazy_count, state, sizeof(state), cudaMemcpyHostToDevice, st));
  CUDA_TRY(c, launch_init_keys(g, c->counters, g.L + 1, st));
  CUDA_TRY(c, launch_vertex_labels(g, c->rb, c->variant, scene(c), st));
  LAUNCHED(c, 2);
  // iterations are enqueued eight at a time and the state read back after each group: the kernels of
  // the iterations after the last one return at once, and the cap bounds the loop on the device too
  for (;;) {
    for (int k = 0; k < 8; ++k) {
      CUDA_TRY(c, launch_lazy_iteration(g, c->variant, c->rb, scene(c), c->lazy_bad, words, dev_path, dev_cost,
                                        c->lazy_count, max_iterations, st));
      LAUNCHED(c, g.L + 5);
    }
    CUDA_TRY(c, cudaMemcpyAsync(state, c->lazy_count, sizeof(state), cudaMemcpyDeviceToHost, st));
    CUDA_TRY(c, cudaStreamSynchronize(st));
    if (state[kLazyDone] != 0) break;
  }
  if (stats) {
    stats->iterations = state[kLazyIters];
    stats->colliding_edges = state[kLazyEdges];
  }
  // a chain with no colliding edge (or no chain at all) is the optimum: every other chain's optimistic
  // cost, a lower bound of its true cost, is at least this chain's true cost
  if (state[kLazyFound] != 0)
    return fail(c, GTMP_ERR_TIMEOUT, "lazy evaluation: %d iterations without a verified chain", state[kLazyIters]);
  return GTMP_OK;
}

gtmp_status gtmp_get_values(gtmp_ctx* c, int32_t gi, float* dev_V, int32_t* dev_sigma) {
  if (!c || !dev_V || !dev_sigma || gi < 0 || gi >= c->p.R) return fail(c, GTMP_ERR_INVALID_ARG, "bad request");
  GraphDev g = graph(c, 1, c->M_active);
  // view graph gi as a one-graph batch
  const size_t off = static_cast<size_t>(gi) * (c->p.L + 2) * c->p.M;
  g.Q += off * c->dp;
  g.vflag += off;
  g.keys += off;
  CUDA_TRY(c, launch_get_values(g, dev_V, dev_sigma, c->stream));
  LAUNCHED(c, 1);
  return GTMP_OK;
}

gtmp_status gtmp_solve_unfused(gtmp_ctx* c, int32_t* dev_path, float* dev_cost) {
  GtmpNvtxRange nvtx_("gtmp_solve_unfused");
  if (!c || !dev_path || !dev_cost) return fail(c, GTMP_ERR_INVALID_ARG, "NULL output");
  gtmp_status s = check_ready(c);
  if (s != GTMP_OK) return s;
  if ((s = gtmp_internal_edge_costs(c)) != GTMP_OK) return s;
  const int L = c->p.L;
  GraphDev g = graph(c, 1, c->M_active);
  // step 2: the min-plus sweep over the stored matrices, each transition a
  // programmatic dependent of the previous one (timed as one sweep: events
  // between the launches would serialise them)
  size_t slot = 0;
  if (c->timing) {
    slot = (c->ev_used.size() + c->ev_minplus.size()) * 2;
    cudaEvent_t e0 = nullptr;
    CUDA_TRY(c, event_at(c, slot, &e0));
    CUDA_TRY(c, cudaEventRecord(e0, c->stream));
  }
  for (int layer = L; layer >= 0; --layer) {
    int rows, cols;
    transition_shape(g, layer, &rows, &cols);
    int grid = (rows + 7) / 8;
    if (grid > c->num_sms * 8) grid = c->num_sms * 8;
    CUDA_TRY(c, launch_minplus(g, layer, c->C + c->c_off[layer], c->c_cs[layer], grid, layer < L, c->stream));
    LAUNCHED(c, 1);
    if (c->timing) {
      c->minplus_launches += 1;
      c->minplus_bytes += 4.0 * rows * cols + 8.0 * cols + 8.0 * rows;
    }
  }
  if (c->timing) {
    cudaEvent_t e1 = nullptr;
    CUDA_TRY(c, event_at(c, slot + 1, &e1));
    CUDA_TRY(c, cudaEventRecord(e1, c->stream));
    c->ev_minplus.emplace_back(static_cast<int>(slot), static_cast<int>(slot + 1));
  }
  CUDA_TRY(c, launch_extract_paths(g, dev_path, dev_cost, nullptr, c->stream));
  LAUNCHED(c, 1);
  return GTMP_OK;
}

gtmp_status gtmp_get_edge_costs(gtmp_ctx* c, int32_t l, float* dev_C) {
  if (!c || !dev_C || l < 0 || l > c->p.L) return fail(c, GTMP_ERR_INVALID_ARG, "bad request");
  if (!c->C) return fail(c, GTMP_ERR_NOT_READY, "no unfused solve yet");
  GraphDev g = graph(c, 1, c->M_active);
  int rows, cols;
  transition_shape(g, l, &rows, &cols);
  CUDA_TRY(c, cudaMemcpy2DAsync(dev_C, cols * sizeof(float), c->C + c->c_off[l], c->c_cs[l] * sizeof(float),
                                cols * sizeof(float), rows, cudaMemcpyDeviceToDevice, c->stream));
  return GTMP_OK;
}

gtmp_status gtmp_anytime(gtmp_ctx* c, uint64_t seed, int32_t restarts, int32_t* dev_paths, float* dev_costs,
                         int32_t* dev_best) {
  GtmpNvtxRange nvtx_("gtmp_anytime");
  if (!c || !dev_paths || !dev_costs || !dev_best) return fail(c, GTMP_ERR_INVALID_ARG, "NULL output");
  if (restarts < 1 || restarts > c->p.R)
    return fail(c, GTMP_ERR_INVALID_ARG, "restarts=%d outside 1..%d", restarts, c->p.R);
  if (!c->have_endpoints) return fail(c, GTMP_ERR_NOT_READY, "endpoints not set");
  GraphDev g = graph(c, restarts, c->p.M);
  CUDA_TRY(c, sample_layers_of(c, g, seed));
  LAUNCHED(c, 1);
  c->M_active = c->p.M;
  gtmp_status s = run_fused(c, g, c->p.eval_mode);
  if (s != GTMP_OK) return s;
  CUDA_TRY(c, launch_extract_paths(g, dev_paths, dev_costs, dev_best, c->stream));
  LAUNCHED(c, 1);
  return GTMP_OK;
}

gtmp_status aogtmp_expand(gtmp_ctx* c, uint64_t seed, int32_t M_new, int32_t* dev_stage_path, float* dev_stage_cost,
                          int32_t* dev_best_path, float* dev_best_cost) {
  GtmpNvtxRange nvtx_("aogtmp_expand");
  if (!c || !dev_stage_path || !dev_stage_cost || !dev_best_path || !dev_best_cost)
    return fail(c, GTMP_ERR_INVALID_ARG, "NULL output");
  if (!c->have_endpoints) return fail(c, GTMP_ERR_NOT_READY, "endpoints not set");
  if (c->G != 1)
    return fail(c, GTMP_ERR_UNSUPPORTED, "informed expansion is defined for a single goal (the ellipsoid's focus)");
  const int M_old = c->M_active;
  if (M_new < M_old || M_new < 1 || M_new > c->p.M)
    return fail(c, GTMP_ERR_INVALID_ARG, "M_new=%d outside %d..%d", M_new, M_old, c->p.M);
  GraphDev g = graph(c, 1, M_new);
  CUDA_TRY(c, launch_expand(g, c->dof, c->q_lo, c->q_hi, seed, M_old, M_new, dev_best_cost, 1 << 16, c->err,
                            c->stream));
  if (M_new > M_old) LAUNCHED(c, 1);
  c->M_active = M_new;
  gtmp_status s = run_fused(c, g, c->p.eval_mode);
  if (s != GTMP_OK) return s;
  CUDA_TRY(c, launch_extract_paths(g, dev_stage_path, dev_stage_cost, nullptr, c->stream));
  CUDA_TRY(c, launch_update_best(c->p.L, dev_stage_path, dev_stage_cost, dev_best_path, dev_best_cost, c->stream));
  LAUNCHED(c, 2);
  return GTMP_OK;
}

gtmp_status aogtmp_run(gtmp_ctx* c, uint64_t seed, const gtmp_ao_schedule* sch, float* dev_best_chain,
                       float* dev_best_cost, gtmp_ao_stage* log, int32_t* best_layers) {
  GtmpNvtxRange nvtx_("aogtmp_run");
  if (!c || !sch || !dev_best_chain || !dev_best_cost || !log || !best_layers)
    return fail(c, GTMP_ERR_INVALID_ARG, "NULL argument");
  const gtmp_ao_schedule S = *sch;
  const double margin = 2.0 * static_cast<double>(S.r) + static_cast<double>(S.varsigma);
  if (S.L0 < 1 || S.L0 > c->L_cap || S.M0 < 1 || S.M_max < S.M0 || S.M_max > c->p.M || S.stages < 1 ||
      std::isnan(S.reach) || !(S.r >= 0.0f) || !(S.varsigma >= 0.0f) || !std::isfinite(S.r) ||
      !std::isfinite(S.varsigma) || !(static_cast<double>(S.reach) > margin))
    return fail(c, GTMP_ERR_INVALID_ARG, "schedule outside its ranges (L0 1..%d, M0 <= M_max <= %d, reach > 2r + "
                "varsigma)", c->L_cap, c->p.M);
  if (!c->have_endpoints) return fail(c, GTMP_ERR_NOT_READY, "endpoints not set");
  if (c->G != 1) return fail(c, GTMP_ERR_UNSUPPORTED, "informed expansion is defined for a single goal");
  if (!c->ao_scratch) CUDA_TRY(c, cudaMalloc(&c->ao_scratch, (2 * static_cast<size_t>(c->L_cap) + 2) * sizeof(int32_t)));
  int32_t* stage_path = c->ao_scratch;
  int32_t* best_path = c->ao_scratch + c->L_cap;
  float* stage_cost = reinterpret_cast<float*>(c->ao_scratch + 2 * c->L_cap);
  const float inf = std::numeric_limits<float>::infinity();
  const float limit0 = c->p.max_edge_len;
  const int rows = c->L_cap + 2;
  CUDA_TRY(c, cudaMemcpyAsync(dev_best_cost, &inf, sizeof(float), cudaMemcpyHostToDevice, c->stream));
  *best_layers = 0;
  double best = std::numeric_limits<double>::infinity();
  int epoch = 0, L = S.L0, M = S.M0;
  gtmp_status st = gtmp_set_num_layers(c, L);
  for (int stage = 0; st == GTMP_OK && stage < S.stages; ++stage) {
    float limit = limit0;
    if (S.limit_edges && std::isfinite(best)) {
      const float l = static_cast<float>(best / (L + 1) + margin);
      limit = l < limit0 ? l : limit0;
    }
    c->p.max_edge_len = limit;
    st = aogtmp_expand(c, seed + static_cast<uint64_t>(epoch), M, stage_path, stage_cost, best_path, dev_best_cost);
    if (st != GTMP_OK) break;
    float h[2];
    if (cudaMemcpyAsync(&h[0], stage_cost, sizeof(float), cudaMemcpyDeviceToHost, c->stream) != cudaSuccess ||
        cudaMemcpyAsync(&h[1], dev_best_cost, sizeof(float), cudaMemcpyDeviceToHost, c->stream) != cudaSuccess ||
        cudaStreamSynchronize(c->stream) != cudaSuccess) {
      st = fail(c, GTMP_ERR_CUDA, "reading the stage cost back failed");
      break;
    }
    if (static_cast<double>(h[0]) < best) {  // this stage found the new best chain: keep its configurations
      GraphDev g = graph(c, 1, M);
      if (launch_gather_chain(g, stage_path, dev_best_chain, c->dof, rows, c->stream) != cudaSuccess) {
        st = fail(c, GTMP_ERR_CUDA, "chain gather launch failed");
        break;
      }
      LAUNCHED(c, 1);
      *best_layers = L;
    }
    best = h[1];
    log[stage] = gtmp_ao_stage{epoch, L, M, limit, h[0], h[1]};
    // next stage: the layer rule, then saturation, else double the samples
    int L_next = L;
    bool new_epoch = false;
    if (std::isfinite(S.reach) && std::isfinite(best) && L < c->L_cap) {
      const double need = std::ceil(best / (static_cast<double>(S.reach) - margin)) - 1.0;
      if (need > L) {
        L_next = need > L + 1 ? (need < c->L_cap ? static_cast<int>(need) : c->L_cap) : L + 1;
        new_epoch = true;
      }
    }
    if (!new_epoch && M >= S.M_max) {
      L_next = L + 1;
      new_epoch = true;
    }
    if (new_epoch) {
      L = L_next < c->L_cap ? L_next : c->L_cap;
      M = S.M0;
      ++epoch;
      if (stage + 1 < S.stages) st = gtmp_set_num_layers(c, L);
    } else {
      M = 2 * M < S.M_max ? 2 * M : S.M_max;
    }
  }
  c->p.max_edge_len = limit0;
  if (st == GTMP_OK && *best_layers == 0) {
    // no feasible chain: every row NaN
    std::vector<float> nan(static_cast<size_t>(rows) * c->dof, std::numeric_limits<float>::quiet_NaN());
    CUDA_TRY(c, cudaMemcpyAsync(dev_best_chain, nan.data(), nan.size() * sizeof(float), cudaMemcpyHostToDevice,
                                c->stream));
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  }
  return st;
}

}  // extern "C"
