// Learned collision surrogate on the tcgen05 tensor cores, and the
// surrogate-pruned solve.  The paper has no surrogate; it names lazy edge
// realisation as future work (Sec. VII).  Model (BF16 weights, FP32
// accumulation):
//   phi(q) = [sin(B q), cos(B q)]      B: 64 x d Fourier frequencies (fixed)
//   h1 = relu(W1 phi + b1)   h2 = relu(W2 h1 + b2)   h3 = relu(W3 h2 + b3)
//   logit = w4 . h3 + b4                (256 hidden units per layer)
// Hidden activations are rounded to BF16 between layers; the head reads the
// FP32 h3.  Training: binary cross-entropy against the exact checker's labels,
// Adam, FP32 master weights.  Pruning: an edge is dropped before exact
// checking when the surrogate calls any of its waypoints t = 1/4, 1/2, 3/4 a
// collision with probability above the threshold; every edge that survives
// is still realised by the exact checker, which therefore judges every
// returned path.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <random>
#include <vector>

#include "../../include/gtmp.h"
#include "gtmp_edge.cuh"
#include "gtmp_umma.cuh"

namespace gtmp {
namespace umma_impl {

constexpr int kMbarLimit = 1 << 24;

__device__ __forceinline__ uint32_t s_u32(const void* p) { return static_cast<uint32_t>(__cvta_generic_to_shared(p)); }

// UMMA shared-memory descriptor: start, leading (K-direction) and stride
// (8-row-group) byte offsets >> 4, descriptor version 1, no swizzle.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  return static_cast<uint64_t>((addr >> 4) & 0x3FFF) | (static_cast<uint64_t>((lbo >> 4) & 0x3FFF) << 16) |
         (static_cast<uint64_t>((sbo >> 4) & 0x3FFF) << 32) | (1ull << 46);
}

__device__ __forceinline__ void cp_async16(uint32_t dst, const void* src, uint32_t bytes) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool mbar_wait_parity(uint32_t mbar, uint32_t parity, int limit) {
  for (int it = 0; it < limit; ++it) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(mbar), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}

template <int BN, int EPI>
__global__ void __launch_bounds__(kUmmaThreads, 1) umma_gemm_kernel(UmmaArgs a) {
  constexpr int kA = kUmmaBM * kUmmaBK * 2;
  constexpr int kB = BN * kUmmaBK * 2;
  constexpr int kStage = kA + kB;
  extern __shared__ __align__(1024) uint8_t smem[];
  __shared__ __align__(8) uint64_t mbar;
  __shared__ uint32_t tmem_base;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int m0 = blockIdx.y * kUmmaBM, n0 = blockIdx.x * BN;
  const int nk = (a.K + kUmmaBK - 1) / kUmmaBK;
  const uint32_t mb = s_u32(&mbar);

  auto load_stage = [&](int kt, int s) {
    const int k0 = kt * kUmmaBK;
    const uint32_t sA = s_u32(smem + s * kStage), sB = sA + kA;
    for (int c = tid; c < kUmmaBM * 8; c += kUmmaThreads) {
      const int r = c >> 3, kc = c & 7;
      const int gm = m0 + r, gk = k0 + kc * 8;
      const bool ok = gm < a.M && gk < a.K;
      const __nv_bfloat16* src = ok ? a.A + static_cast<size_t>(gm) * a.lda + gk : a.A;
      cp_async16(sA + ((r >> 3) * 8 + kc) * 128 + (r & 7) * 16, src, ok ? 16u : 0u);
    }
    for (int c = tid; c < BN * 8; c += kUmmaThreads) {
      const int r = c >> 3, kc = c & 7;
      const int gn = n0 + r, gk = k0 + kc * 8;
      const bool ok = gn < a.N && gk < a.K;
      const __nv_bfloat16* src = ok ? a.B + static_cast<size_t>(gn) * a.ldb + gk : a.B;
      cp_async16(sB + ((r >> 3) * 8 + kc) * 128 + (r & 7) * 16, src, ok ? 16u : 0u);
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
  };

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(s_u32(&tmem_base)),
                 "r"(BN)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(mb) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  load_stage(0, 0);
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_base;
  // kind::f16 instruction descriptor: D f32, A/B bf16, both K-major, N >> 3, M >> 4
  const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | (static_cast<uint32_t>(BN >> 3) << 17) |
                         (static_cast<uint32_t>(kUmmaBM >> 4) << 24);
  bool ok = true;
  for (int kt = 0; kt < nk; ++kt) {
    const int s = kt & 1;
    asm volatile("cp.async.wait_all;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    if (kt + 1 < nk) load_stage(kt + 1, s ^ 1);  // that buffer's MMAs completed in the previous iteration
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t sA = s_u32(smem + s * kStage), sB = sA + kA;
#pragma unroll
      for (int kk = 0; kk < kUmmaBK / 16; ++kk) {
        const uint64_t da = smem_desc(sA + kk * 256, 128, 1024);
        const uint64_t db = smem_desc(sB + kk * 256, 128, 1024);
        const uint32_t acc = (kt > 0 || kk > 0) ? 1u : 0u;
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem),
            "l"(da), "l"(db), "r"(idesc), "r"(acc)
            : "memory");
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mb)
                   : "memory");
    }
    const bool done = mbar_wait_parity(mb, static_cast<uint32_t>(kt & 1), kMbarLimit);
    ok = __syncthreads_and(done) != 0;
    if (!ok) {
      if (tid == 0) atomicOr(a.err, kErrWaitTimeout);
      mbar_wait_parity(mb, static_cast<uint32_t>(kt & 1), kMbarLimit);  // let the MMAs drain
      break;
    }
  }
  asm volatile("cp.async.wait_all;" ::: "memory");
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (ok) {
    const int row = m0 + warp * 32 + lane;
    const bool row_ok = row < a.M;
    float dot = 0.0f;
#pragma unroll 1
    for (int c0 = 0; c0 < BN; c0 += 32) {
      uint32_t v[32];
      const uint32_t taddr = tmem + (static_cast<uint32_t>(warp * 32) << 16) + c0;
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
          "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
          : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
            "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]),
            "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]),
            "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
          : "r"(taddr));
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
      if (!row_ok) continue;
#pragma unroll
      for (int j = 0; j < 32; ++j) {
        const int n = n0 + c0 + j;
        if (n >= a.N) break;
        float x = __uint_as_float(v[j]);
        if constexpr (EPI == kEpiF32) {
          a.outf[static_cast<size_t>(row) * a.ldf + n] = x;
          continue;
        } else if constexpr (EPI == kEpiMaskBf16) {
          x = __bfloat162float(a.mask[static_cast<size_t>(row) * a.ldm + n]) > 0.0f ? x : 0.0f;
        } else {
          x = fmaxf(x + a.bias[n], 0.0f);
          if constexpr (EPI == kEpiHead) dot = __fmaf_rn(x, a.w4[n], dot);
        }
        const __nv_bfloat16 hx = __float2bfloat16_rn(x);
        if (a.out) a.out[static_cast<size_t>(row) * a.ldo + n] = hx;
        if (a.outT) a.outT[static_cast<size_t>(n) * a.ldoT + row] = hx;
      }
    }
    if constexpr (EPI == kEpiHead) {
      if (row_ok) a.logits[row] = dot + *a.b4;
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(BN) : "memory");
}

// ---------------------------------------------------------------------------
// Fourier features of configurations, and of edge waypoints for scoring
// ---------------------------------------------------------------------------
struct FourierDev {
  float B[64 * kMaxDof];  // [64][dof]
  int dof;
};

// The features of one configuration, computed exactly as the fused scoring
// kernel computes them (same FMA order, the fast __sincosf), so that training,
// prediction and scoring evaluate one and the same model.
__device__ __forceinline__ void fourier_row(const float* q, const FourierDev& f, __nv_bfloat16* out) {
  for (int k = 0; k < 64; ++k) {
    float z = 0.0f;
    for (int d = 0; d < f.dof; ++d) z = __fmaf_rn(f.B[k * f.dof + d], q[d], z);
    float s, c;
    __sincosf(z, &s, &c);
    out[k] = __float2bfloat16_rn(s);
    out[64 + k] = __float2bfloat16_rn(c);
  }
}

// q [n][dof] -> X [n][128] and XT [128][ldT] (column offset 0)
__global__ void features_kernel(const float* q, int n, FourierDev f, __nv_bfloat16* X, __nv_bfloat16* XT, int ldT) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  __nv_bfloat16 row[128];
  fourier_row(q + static_cast<size_t>(i) * f.dof, f, row);
  for (int k = 0; k < 128; ++k) {
    X[static_cast<size_t>(i) * 128 + k] = row[k];
    if (XT) XT[static_cast<size_t>(k) * ldT + i] = row[k];
  }
}

// ---------------------------------------------------------------------------
// training pieces
// ---------------------------------------------------------------------------
// training configurations: uniform in the joint box, Philox block (i, 0, 0, 4<<24 | k>>2)
__global__ void train_configs_kernel(int n, int dof, FourierDev f, unsigned long long seed, const float* lo,
                                     const float* hi, float* q) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const uint2 key = seed_key(seed);
  uint4 w = make_uint4(0, 0, 0, 0);
  for (int k = 0; k < dof; ++k) {
    if ((k & 3) == 0) w = philox4x32_10(make_uint4(static_cast<uint32_t>(i), 0u, 0u, (4u << 24) | (k >> 2)), key);
    q[static_cast<size_t>(i) * dof + k] = __fmaf_rn(word_to_unit(word_of(w, k)), __fsub_rn(hi[k], lo[k]), lo[k]);
  }
}

// dz = (sigmoid(z) - y) / B; loss += BCE; dA3 = dz * w4 * (h3 > 0) (+ transposed)
__global__ void head_backward_kernel(const float* logits, const uint8_t* labels, int b0, int B, const float* w4,
                                     const __nv_bfloat16* H3, __nv_bfloat16* dA3, __nv_bfloat16* dA3T, int ldT,
                                     float* dz, double* loss) {
  const int i = blockIdx.x;  // row of the batch
  const float z = logits[i];
  const float y = labels[b0 + i] ? 1.0f : 0.0f;
  const float p = 1.0f / (1.0f + __expf(-z));
  const float g = (p - y) / static_cast<float>(B);
  if (threadIdx.x == 0) {
    dz[i] = g;
    // numerically stable BCE with logits
    const float l = fmaxf(z, 0.0f) - z * y + log1pf(__expf(-fabsf(z)));
    atomicAdd(loss, static_cast<double>(l));
  }
  for (int n = threadIdx.x; n < 256; n += blockDim.x) {
    const float h = __bfloat162float(H3[static_cast<size_t>(i) * 256 + n]);
    const __nv_bfloat16 d = __float2bfloat16_rn(h > 0.0f ? g * w4[n] : 0.0f);
    dA3[static_cast<size_t>(i) * 256 + n] = d;
    dA3T[static_cast<size_t>(n) * ldT + i] = d;
  }
}

// gw4[n] = sum_i dz[i] h3[i][n] (h3T rows), gb4 = sum dz; bias grads = row sums of dAT
__global__ void colsum_kernel(const __nv_bfloat16* T, int ld, int B, const float* weights, float* out) {
  const int n = blockIdx.x;
  float s = 0.0f;
  for (int i = threadIdx.x; i < B; i += blockDim.x) {
    const float x = __bfloat162float(T[static_cast<size_t>(n) * ld + i]);
    s += weights ? x * weights[i] : x;
  }
  for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(kFull, s, off);
  __shared__ float part[32];
  if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    float t = 0.0f;
    for (int w = 0; w < (blockDim.x + 31) / 32; ++w) t += part[w];
    out[n] = t;
  }
}

__global__ void sum_kernel(const float* x, int n, float* out) {
  float s = 0.0f;
  for (int i = threadIdx.x; i < n; i += blockDim.x) s += x[i];
  for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(kFull, s, off);
  __shared__ float part[32];
  if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    float t = 0.0f;
    for (int w = 0; w < (blockDim.x + 31) / 32; ++w) t += part[w];
    *out = t;
  }
}

// Adam on a flat fp32 parameter vector; also writes bf16 copies (row-major and transposed) of weight matrices
__global__ void adam_kernel(float* w, const float* g, float* m, float* v, int n, float lr, float b1, float b2,
                            float eps, float c1, float c2, __nv_bfloat16* wb, __nv_bfloat16* wbT, int rows, int cols) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float gi = g[i];
  const float mi = b1 * m[i] + (1.0f - b1) * gi;
  const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
  m[i] = mi;
  v[i] = vi;
  const float wi = w[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
  w[i] = wi;
  if (wb) {
    const __nv_bfloat16 h = __float2bfloat16_rn(wi);
    wb[i] = h;
    const int r = i / cols, c = i % cols;
    wbT[static_cast<size_t>(c) * rows + r] = h;
  }
}

__global__ void f32_to_bf16_kernel(const float* w, int rows, int cols, __nv_bfloat16* wb, __nv_bfloat16* wbT) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= rows * cols) return;
  const __nv_bfloat16 h = __float2bfloat16_rn(w[i]);
  wb[i] = h;
  if (wbT) wbT[static_cast<size_t>(i % cols) * rows + i / cols] = h;
}

inline int nblk(long long n, int t) { return static_cast<int>((n + t - 1) / t); }

}  // namespace umma_impl

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
using namespace umma_impl;

cudaError_t umma_gemm(const UmmaArgs& a, int epi, cudaStream_t st) {
  const int bn = a.N > 128 ? 256 : 128;
  const dim3 grid((a.N + bn - 1) / bn, (a.M + kUmmaBM - 1) / kUmmaBM);
  const size_t smem = 2 * static_cast<size_t>(kUmmaBM * kUmmaBK * 2 + bn * kUmmaBK * 2);
  if (epi == kEpiHead && a.N > 256) return cudaErrorInvalidValue;
#define UMMA_LAUNCH(BN, EPI)                                                                                    \
  do {                                                                                                          \
    cudaError_t e = cudaFuncSetAttribute(umma_gemm_kernel<BN, EPI>, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                                         static_cast<int>(smem));                                               \
    if (e != cudaSuccess) return e;                                                                             \
    umma_gemm_kernel<BN, EPI><<<grid, kUmmaThreads, smem, st>>>(a);                                             \
    return cudaGetLastError();                                                                                  \
  } while (0)
  if (bn == 256) {
    switch (epi) {
      case kEpiBiasReluBf16: UMMA_LAUNCH(256, kEpiBiasReluBf16);
      case kEpiF32: UMMA_LAUNCH(256, kEpiF32);
      case kEpiMaskBf16: UMMA_LAUNCH(256, kEpiMaskBf16);
      default: UMMA_LAUNCH(256, kEpiHead);
    }
  } else {
    switch (epi) {
      case kEpiBiasReluBf16: UMMA_LAUNCH(128, kEpiBiasReluBf16);
      case kEpiF32: UMMA_LAUNCH(128, kEpiF32);
      case kEpiMaskBf16: UMMA_LAUNCH(128, kEpiMaskBf16);
      default: UMMA_LAUNCH(128, kEpiHead);
    }
  }
#undef UMMA_LAUNCH
}

}  // namespace gtmp

// ===========================================================================
// C ABI: training, prediction and the pruned solve
// ===========================================================================
#include "gtmp_ctx.h"

namespace gtmp {

// Parameter tensors, in the order of gtmp_surrogate_get_params.
constexpr int kHid = 256, kFeat = 128;
constexpr int kNW1 = kHid * kFeat, kNW2 = kHid * kHid, kNW3 = kHid * kHid;
constexpr int kParamCount = kNW1 + kHid + kNW2 + kHid + kNW3 + kHid + kHid + 1;


// ---------------------------------------------------------------------------
// Fused surrogate scoring of edges: features -> 3 layers -> head -> prune mask
// in one persistent kernel (one CTA per SM: eight epilogue warps and one MMA
// warp).  Shared memory (canonical K-major no-swizzle layouts): W1 [256 x 128]
// resident (64 K, one bulk copy per CTA); the features X [128 x 128] (32 K),
// layer 1's A operand; three 32 K buffers for the 256 x 64 K-chunks of W2 and
// W3, pre-arranged in global memory as images of their shared-memory tiles;
// the epilogues' biases.  Every epilogue thread copies its 128 bytes of a
// chunk with cp.async two chunks ahead of the MMAs (chunk numbers run on
// across a CTA's tiles, so the next tile's first chunks load during this
// tile's head); measured on B300, cp.async from all threads moves ~49 B per
// cycle per SM and one bulk copy engine ~16 (a bulk copy per chunk from the
// MMA thread measured 25.4 ms of scoring per solve against 23.9).  TMEM: two
// 128 x 256 fp32 accumulators (all 512 columns).  Each layer's epilogue runs
// in four 64-column chunks; a warp's 32 columns of a chunk go back into the
// first 16 of those columns as bf16 pairs, where they are the next layer's A
// operand (tcgen05.mma reads A from tensor memory: no shared-memory
// activations, stores or proxy fences), and the chunk's four MMAs (K-slice c
// of layer l + 1, into the other accumulator) run under the epilogue of chunk
// c + 1.  An MMA issue blocks its thread for about the MMA's own duration, so
// one warp does nothing else; its chunk g queues behind chunk g - 1, and the
// buffer of chunk g - 1 is reloaded only after that (the tensor pipe does not
// drain between chunks).  A tile is 128 queries: Q = 128 / kw edges with kw
// waypoints each (t = 1/2 for kw = 1; 1/4, 1/2, 3/4 for kw = 3); an edge is
// pruned when its largest logit exceeds `cut`.  Only live edges are scored
// (compacted row and column lists).
// ---------------------------------------------------------------------------
// Live rows (vertex free) and live columns (vertex free, finite cost-to-go)
// of a transition, in increasing order: one block, ballot + prefix per warp.
__global__ void __launch_bounds__(1024) live_lists_kernel(GraphDev g, int layer, int cap, int* live) {
  __shared__ int s_warp[32];
  __shared__ int s_base;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int side = 0; side < 2; ++side) {
    const int lay = layer + side;
    const int n = layer_size(g, lay);
    int* out = live + 2 + side * cap;
    if (threadIdx.x == 0) s_base = 0;
    __syncthreads();
    for (int i0 = 0; i0 < n; i0 += blockDim.x) {
      const int i = i0 + threadIdx.x;
      bool on = false;
      if (i < n) {
        const size_t v = vidx(g, 0, lay, i);
        on = g.vflag[v] == 0 && (side == 0 || g.keys[v] != kEmptyKey);
      }
      const unsigned b = __ballot_sync(kFull, on);
      if (lane == 0) s_warp[warp] = __popc(b);
      __syncthreads();
      int before = 0;
      for (int w = 0; w < warp; ++w) before += s_warp[w];
      if (on) out[s_base + before + __popc(b & ((1u << lane) - 1u))] = i;
      __syncthreads();
      if (threadIdx.x == 0) {
        int tot = 0;
        for (int w = 0; w < static_cast<int>(blockDim.x >> 5); ++w) tot += s_warp[w];
        s_base += tot;
      }
      __syncthreads();
    }
    if (threadIdx.x == 0) live[side] = s_base;
    __syncthreads();
  }
}

// The protection band of a transition: per live row (one warp), the smallest
// edge bound |v - u| + J(v) over the live columns (edges longer than the edge
// limit left out; float32 as the exact kernels compute the length), then
// every live edge of the row marked in the prune mask: kPruneProtected when
// its bound is at most factor times that minimum, else 0.  The scoring
// kernel then writes every live edge's decision, never pruning a marked one.
constexpr uint8_t kPruneProtected = 3;

__device__ __forceinline__ float edge_bound(const GraphDev& g, int layer, const float* u, int j) {
  const size_t vj = vidx(g, 0, layer + 1, j);
  const float* v = g.Q + vj * g.dp;
  float s2 = 0.0f;
  for (int d = 0; d < g.dp; ++d) {
    const float e = __fsub_rn(v[d], u[d]);
    s2 = __fmaf_rn(e, e, s2);
  }
  const float len = __fsqrt_rn(s2);
  return len > g.max_edge_len ? kInf : __fadd_rn(len, key_value(__ldcg(g.keys + vj)));
}

__global__ void __launch_bounds__(256) protect_band_kernel(GraphDev g, int layer, const int* live, int cap,
                                                           float factor, uint8_t* prune) {
  const int nr = live[0], nc = live[1];
  const int* rows_live = live + 2;
  const int* cols_live = live + 2 + cap;
  const int lane = threadIdx.x & 31;
  const int r = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (r >= nr) return;
  const int i = rows_live[r];
  const int cols = layer_size(g, layer + 1);
  const float* u = g.Q + vidx(g, 0, layer, i) * g.dp;
  // four columns per lane and trip: four independent chains of dependent loads in flight
  float best = kInf;
  for (int c0 = lane; c0 < nc; c0 += 128) {
#pragma unroll
    for (int k = 0; k < 4; ++k)
      if (c0 + 32 * k < nc) best = fminf(best, edge_bound(g, layer, u, cols_live[c0 + 32 * k]));
  }
  for (int o = 16; o > 0; o >>= 1) best = fminf(best, __shfl_xor_sync(kFull, best, o));
  const float lim = __fmul_rn(factor, best);
  uint8_t* row = prune + static_cast<size_t>(i) * cols;
  for (int c0 = lane; c0 < nc; c0 += 128) {
#pragma unroll
    for (int k = 0; k < 4; ++k)
      if (c0 + 32 * k < nc) {
        const int j = cols_live[c0 + 32 * k];
        row[j] = edge_bound(g, layer, u, j) <= lim ? kPruneProtected : 0;
      }
  }
}

// eight epilogue warps (two per TMEM lane quarter), one MMA warp, whose lane 0 issues every MMA (an
// issue blocks for about the MMA's own duration, so it has a warp of its own), and one load warp, whose
// lane 0 streams the weight chunks; the first nine synchronise on named barrier 2
constexpr int kEpiThreads = 256, kMmaThread = kEpiThreads, kMainThreads = kEpiThreads + 32;
constexpr int kLoadThread = kMainThreads, kScoreThreads = kMainThreads + 32;

// barrier 2 over the epilogue and MMA warps; the _and form returns whether p held in every thread
__device__ __forceinline__ void bar_sync_main() { asm volatile("bar.sync 2, %0;" ::"n"(kMainThreads) : "memory"); }
__device__ __forceinline__ bool bar_and_main(bool p) {
  uint32_t r;
  asm volatile(
      "{\n\t.reg .pred p, q;\n\tsetp.ne.u32 p, %1, 0;\n\tbar.red.and.pred q, 2, %2, p;\n\tselp.u32 %0, 1, 0, q;\n\t}"
      : "=r"(r)
      : "r"(static_cast<uint32_t>(p)), "n"(kMainThreads)
      : "memory");
  return r != 0;
}
constexpr int kSmemW1 = 256 * 128 * 2, kSmemX = 128 * 128 * 2, kSmemS = 256 * 64 * 2, kSmemP = 4 * 256 * 4;
constexpr int kChunkBufs = 3;                      // stream buffers: one being read, two loading
constexpr int kSmemF = 64 * kMaxDof * 4;           // the Fourier matrix, one padded row per frequency
constexpr int kScoreSmem = kSmemW1 + kSmemX + kChunkBufs * kSmemS + kSmemP + kSmemF;

struct ScoreArgs {
  GraphDev g;
  int layer;
  const int* live;         // [0]: live rows nr, [1]: live columns nc, then nr row and nc column indices
  int cap;                 // capacity of each index list (>= rows, cols)
  int kw;                  // waypoints per edge (1 or 3)
  float cut;               // logit threshold
  const __nv_bfloat16* W1b;
  const __nv_bfloat16* W2b;
  const __nv_bfloat16* W3b;
  const uint8_t* Wimg;     // W1 (64 KB) then the eight 256 x 64 chunks of W2, W3 (32 KB each), in shared-memory layout
  const float* P;          // fp32 parameters (biases, w4, b4)
  uint8_t* prune;
  unsigned long long* n_pruned;
  int* err;
  // protection band on: live entries of prune hold kPruneProtected (never pruned) or 0 on entry
  int protect;
};

// byte offset of element (r, k) in a canonical K-major tile whose rows hold kdim elements
__device__ __forceinline__ uint32_t canon(int r, int k, int kdim) {
  return static_cast<uint32_t>(((r >> 3) * (kdim >> 3) + (k >> 3)) * 128 + (r & 7) * 16 + (k & 7) * 2);
}

// the same with A read from tensor memory (columns ta.., 128 lanes, two bf16 per 32-bit column)
__device__ __forceinline__ void issue_mma_ts(uint32_t tmem, uint32_t ta, uint64_t db, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n\t}\n" ::"r"(tmem),
      "r"(ta), "l"(db), "r"(idesc), "r"(acc)
      : "memory");
}

__device__ __forceinline__ void issue_mma(uint32_t tmem, uint64_t da, uint64_t db, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem),
      "l"(da), "l"(db), "r"(idesc), "r"(acc)
      : "memory");
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&v)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
        "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]),
        "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]),
        "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// 16 TMEM columns of this warp's 32 lanes, waited for
__device__ __forceinline__ void tmem_st16(uint32_t taddr, const uint32_t (&w)[16]) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16};" ::"r"(
          taddr),
      "r"(w[0]), "r"(w[1]), "r"(w[2]), "r"(w[3]), "r"(w[4]), "r"(w[5]), "r"(w[6]), "r"(w[7]), "r"(w[8]), "r"(w[9]),
      "r"(w[10]), "r"(w[11]), "r"(w[12]), "r"(w[13]), "r"(w[14]), "r"(w[15])
      : "memory");
  asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
}

// 64 TMEM columns of this warp's 32 lanes in one load
__device__ __forceinline__ void tmem_ld64(uint32_t taddr, uint32_t (&v)[64]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x64.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31,%32,%33,%34,%35,%36,%37,%38,%39,"
      "%40,%41,%42,%43,%44,%45,%46,%47,%48,%49,%50,%51,%52,%53,%54,%55,%56,%57,%58,%59,%60,%61,%62,%63}, [%64];"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
        "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]),
        "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]),
        "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31]),
        "=r"(v[32]), "=r"(v[33]), "=r"(v[34]), "=r"(v[35]), "=r"(v[36]), "=r"(v[37]), "=r"(v[38]), "=r"(v[39]),
        "=r"(v[40]), "=r"(v[41]), "=r"(v[42]), "=r"(v[43]), "=r"(v[44]), "=r"(v[45]), "=r"(v[46]), "=r"(v[47]),
        "=r"(v[48]), "=r"(v[49]), "=r"(v[50]), "=r"(v[51]), "=r"(v[52]), "=r"(v[53]), "=r"(v[54]), "=r"(v[55]),
        "=r"(v[56]), "=r"(v[57]), "=r"(v[58]), "=r"(v[59]), "=r"(v[60]), "=r"(v[61]), "=r"(v[62]), "=r"(v[63])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// Weight images for the scoring kernel: W1 [256 x 128] and the chunks
// c = 0..7 (W2 then W3, input columns [64 (c & 3), + 64)) laid out in global
// memory exactly as their shared-memory tiles (canonical K-major), so that one
// bulk copy moves each.  Thread per 16-byte segment.
__global__ void weight_images_kernel(const __nv_bfloat16* W1b, const __nv_bfloat16* W2b, const __nv_bfloat16* W3b,
                                     uint8_t* img) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < 256 * 16) {
    const int n = t >> 4, kc = t & 15;
    *reinterpret_cast<uint4*>(img + canon(n, kc * 8, 128)) =
        *reinterpret_cast<const uint4*>(W1b + static_cast<size_t>(n) * kFeat + kc * 8);
    return;
  }
  const int u = t - 256 * 16;
  if (u >= 8 * 256 * 8) return;
  const int c = u >> 11, n = (u >> 3) & 255, kc = u & 7;
  const __nv_bfloat16* W = c < 4 ? W2b : W3b;
  *reinterpret_cast<uint4*>(img + kSmemW1 + c * kSmemS + canon(n, kc * 8, 64)) =
      *reinterpret_cast<const uint4*>(W + static_cast<size_t>(n) * kHid + (c & 3) * 64 + kc * 8);
}

// eight features of one query: frequencies [k0, k0 + 8) of the waypoint q, the Fourier matrix rows
// from shared memory (row k at sF + k kMaxDof; one address per warp, a broadcast): sine and cosine
// rounded to bf16, packed in pairs (the lower frequency in the low half).  z = B_k q sums over the
// joints in order, one FMA each, as the feature routine of training and prediction does.
template <int DOF>
__device__ __forceinline__ void score_features_part(const float (&q)[DOF > 0 ? DOF : kMaxDof], const float* sF,
                                                    int dof_rt, int k0, uint32_t (&sw)[4], uint32_t (&cw)[4]) {
  constexpr int ND = DOF > 0 ? DOF : kMaxDof;
  constexpr int ND4 = (ND + 3) / 4;
  const int dof = DOF > 0 ? DOF : dof_rt;
#pragma unroll
  for (int k2 = 0; k2 < 4; ++k2) {
    float sn[2], cs[2];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const float4* row = reinterpret_cast<const float4*>(sF + (k0 + 2 * k2 + h) * kMaxDof);
      float b[4 * ND4];
#pragma unroll
      for (int i = 0; i < ND4; ++i) {
        const float4 r4 = row[i];
        b[4 * i] = r4.x;
        b[4 * i + 1] = r4.y;
        b[4 * i + 2] = r4.z;
        b[4 * i + 3] = r4.w;
      }
      float z = 0.0f;
#pragma unroll
      for (int d = 0; d < ND; ++d)
        if (d < dof) z = __fmaf_rn(b[d], q[d], z);
      __sincosf(z, &sn[h], &cs[h]);
    }
    const __nv_bfloat162 s2 = __floats2bfloat162_rn(sn[0], sn[1]);
    const __nv_bfloat162 c2 = __floats2bfloat162_rn(cs[0], cs[1]);
    sw[k2] = *reinterpret_cast<const uint32_t*>(&s2);
    cw[k2] = *reinterpret_cast<const uint32_t*>(&c2);
  }
}

template <int DOF>
__global__ void __launch_bounds__(kScoreThreads, 1) score_edges_kernel(ScoreArgs a, FourierDev f) {
  extern __shared__ __align__(1024) uint8_t smem[];
  __shared__ __align__(8) uint64_t mbar_layer;            // one arrival per layer's MMAs: three per tile
  __shared__ __align__(8) uint64_t mbar_buf[kChunkBufs];  // chunk g's MMAs done: buffer g % kChunkBufs is free
  __shared__ __align__(8) uint64_t mbar_full[kChunkBufs]; // chunk g's weights have landed in its buffer
  __shared__ __align__(8) uint64_t mbar_w1;               // the resident W1
  __shared__ __align__(8) uint64_t mbar_fin;              // every MMA of the CTA done (teardown)
  __shared__ int s_abort;
  __shared__ uint32_t tmem_base;
  __shared__ float s_part[2][128];
  __shared__ float s_logit[128];
  uint8_t* sW1 = smem;
  uint8_t* sX = sW1 + kSmemW1;                     // the tile's features (layer 1's A operand)
  uint8_t* sS = sX + kSmemX;                       // stream buffers
  float* sP = reinterpret_cast<float*>(sS + kChunkBufs * kSmemS);  // b1, b2, b3, w4
  float* sF = sP + 4 * kHid;                                        // B [64][kMaxDof], zero padded
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const bool epi = tid < kEpiThreads;  // an epilogue thread (else the MMA or the load warp)
  const uint32_t mbl = s_u32(&mbar_layer);
  {
    const float* P1 = a.P + kNW1;
    const float* P2 = P1 + kHid + kNW2;
    const float* P3 = P2 + kHid + kNW3;
    if (tid < kHid) {
      sP[tid] = P1[tid];
      sP[kHid + tid] = P2[tid];
      sP[2 * kHid + tid] = P3[tid];
      sP[3 * kHid + tid] = P3[kHid + tid];
    }
    for (int i = tid; i < 64 * kMaxDof; i += kScoreThreads) {
      const int k = i / kMaxDof, d = i % kMaxDof;
      sF[i] = d < f.dof ? f.B[k * f.dof + d] : 0.0f;
    }
  }
  const float* b1 = sP;
  const float* b2 = sP + kHid;
  const float* b3 = sP + 2 * kHid;
  const float* w4 = sP + 3 * kHid;
  const float b4 = a.P[kNW1 + kHid + kNW2 + kHid + kNW3 + kHid + kHid];

  uint32_t ph_layer = 0;
  // every thread waits for the next layer completion; the CTA agrees on the outcome (and on an earlier
  // wait's, passed in)
  auto wait_layer = [&](bool earlier_ok = true) -> bool {
    const bool w = mbar_wait_parity(mbl, ph_layer, kMbarLimit);
    ph_layer ^= 1u;
    return bar_and_main(earlier_ok && w && s_abort == 0);
  };

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(s_u32(&tmem_base)),
                 "r"(512)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) {
    s_abort = 0;
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(mbl) : "memory");
    for (int k = 0; k < kChunkBufs; ++k) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(s_u32(&mbar_buf[k])) : "memory");
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(s_u32(&mbar_full[k])) : "memory");
    }
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(s_u32(&mbar_w1)) : "memory");
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(s_u32(&mbar_fin)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    // resident W1: one bulk copy of its image
    const uint32_t bar = s_u32(&mbar_w1);
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(kSmemW1) : "memory");
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     s_u32(sW1)),
                 "l"(a.Wimg), "r"(kSmemW1), "r"(bar)
                 : "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  bool w1_ready = false, any_mma = false;  // the MMA thread's state
  bool released = false;                   // the MMA thread has released the layer barrier by hand
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_base;
  const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | (256u >> 3 << 17) | (128u >> 4 << 24);
  const int q_per_tile = 128 / a.kw * a.kw, e_per_tile = 128 / a.kw;
  // only live edges are scored: a row whose vertex collides, or a column with
  // no path to the goal, is skipped by the exact solve whatever its mask says
  const int nr = a.live[0], nc = a.live[1];
  const int* rows_live = a.live + 2;
  const int* cols_live = a.live + 2 + a.cap;
  const long long n_live = static_cast<long long>(nr) * nc;
  const long long n_tiles = (n_live + e_per_tile - 1) / e_per_tile;
  const int cols = layer_size(a.g, a.layer + 1);
  const int quarter = warp & 3, half = warp >> 2;
  const int row = quarter * 32 + lane;  // TMEM lane = tile row this thread reads
  const uint32_t lane_addr = tmem + (static_cast<uint32_t>(quarter * 32) << 16);
  bool ok = true;
  const long long my_tiles = blockIdx.x < n_tiles ? (n_tiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;
  const long long total_chunks = my_tiles * 8;
  long long chunks_issued = 0;

  // Features of a tile's queries -> X, in stages spread over the tiles before so that their loads and
  // arithmetic run under their layers: the query's vertex indices (two tiles ahead), its end points
  // (one tile ahead), then the features in four parts, one per step of layer 1's epilogue, each stored
  // to X (free once the current tile's layer 1 has read it).  Two threads per query, 32 frequencies
  // each; the fast __sincosf is ample here (|Bq| < 10, absolute error ~1e-6, the features are rounded
  // to bf16 right after).
  constexpr int ND = DOF > 0 ? DOF : kMaxDof;
  const int qidx = tid & 127, hf = tid >> 7;
  const bool small = n_live <= 0x7fffffffLL;
  // live edge e -> (row list index, column list index)
  auto split_edge = [&](long long e, int& r, int& cidx) {
    if (small) {
      const int ei = static_cast<int>(e);
      r = ei / nc;
      cidx = ei - r * nc;
    } else {
      r = static_cast<int>(e / nc);
      cidx = static_cast<int>(e - static_cast<long long>(r) * nc);
    }
  };
  int fi = 0, fj = 0;
  bool fvalid = false;
  float fu[ND], fv[ND], fq[ND];
  auto feat_index = [&](long long tile_f) {
    const long long e = tile_f * e_per_tile + qidx / a.kw;
    fvalid = epi && qidx < q_per_tile && e < n_live;
    if (fvalid) {
      int r, cidx;
      split_edge(e, r, cidx);
      fi = rows_live[r];
      fj = cols_live[cidx];
    }
  };
  auto feat_points = [&]() {
    if (fvalid) {
      const int dof = DOF > 0 ? DOF : f.dof;
      const float* u = a.g.Q + vidx(a.g, 0, a.layer, fi) * a.g.dp;
      const float* v = a.g.Q + vidx(a.g, 0, a.layer + 1, fj) * a.g.dp;
#pragma unroll
      for (int d = 0; d < ND; ++d) {
        fu[d] = d < dof ? u[d] : 0.0f;
        fv[d] = d < dof ? v[d] : 0.0f;
      }
    }
  };
  // the query's waypoint q = u + t (v - u) from its end points
  auto feat_waypoint = [&]() {
    if (fvalid) {
      const int dof = DOF > 0 ? DOF : f.dof;
      const float t = a.kw == 1 ? 0.5f : 0.25f * static_cast<float>(qidx % a.kw + 1);
#pragma unroll
      for (int d = 0; d < ND; ++d) fq[d] = d < dof ? __fmaf_rn(t, __fsub_rn(fv[d], fu[d]), fu[d]) : 0.0f;
    }
  };
  // part p of 4 of the features (8 of this thread's 32 frequencies) -> X; part 3 fences X for the MMAs
  auto feat_part = [&](int p) {
    if (!epi) return;
    uint32_t sw[4] = {0u, 0u, 0u, 0u}, cw[4] = {0u, 0u, 0u, 0u};
    if (fvalid) {
      score_features_part<DOF>(fq, sF, f.dof, hf * 32 + p * 8, sw, cw);
    }
    *reinterpret_cast<uint4*>(sX + canon(qidx, hf * 32 + p * 8, 128)) = make_uint4(sw[0], sw[1], sw[2], sw[3]);
    *reinterpret_cast<uint4*>(sX + canon(qidx, 64 + hf * 32 + p * 8, 128)) = make_uint4(cw[0], cw[1], cw[2], cw[3]);
    if (p == 3) asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // X (generic writes) -> MMA reads
  };
  // layer 1 (D = X W1^T) into the accumulator at TMEM column acc, committed to the layer barrier; on a W1
  // timeout the barrier is released by hand and the abort flag set
  auto issue_l1 = [&](uint32_t acc) {
    if (tid != kMmaThread) return;
    bool go = true;
    if (!w1_ready) {
      go = mbar_wait_parity(s_u32(&mbar_w1), 0u, kMbarLimit);
      w1_ready = true;
      if (!go) {
        s_abort = 1;
        asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(mbl) : "memory");
        released = true;
      }
    }
    if (go) {
      any_mma = true;
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      for (int kk = 0; kk < 8; ++kk)
        issue_mma(tmem + acc, smem_desc(s_u32(sX) + kk * 256, 128, 2048), smem_desc(s_u32(sW1) + kk * 256, 128, 2048),
                  idesc, kk > 0);
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbl)
                   : "memory");
    }
  };

  // Per tile: the layer-1 accumulator A (TMEM columns 0 or 256, alternating by tile) also takes layer 3,
  // the other one, B, layer 2.  Each epilogue runs in four 64-column chunks; chunk c of layer l's
  // output, written back to tensor memory as bf16, is K-slice c of layer l + 1's A operand, whose four
  // MMAs are issued at once and run under the epilogue of chunk c + 1.  The next tile's end points are
  // loaded before this tile's layer-1 wait, and its features computed and stored to X (free once this
  // tile's layer 1 is done) a quarter per step of layer 1's epilogue; its layer-1 MMAs (into B) run
  // under this tile's head (which reads A).
  if (tid >= kMainThreads) {
    // The load warp: lane 0 streams chunk g into buffer g % kChunkBufs as one bulk copy completing on
    // mbar_full, once chunk g - kChunkBufs's MMAs have freed the buffer.  It runs ahead of the MMAs by
    // the buffers; it stops on the CTA's abort flag (polled between slices of each bounded wait).
    if (tid == kLoadThread) {
      auto wait_or_abort = [&](uint32_t bar, uint32_t parity) -> bool {
        for (int slice = 0; slice < 64; ++slice) {
          if (mbar_wait_parity(bar, parity, kMbarLimit / 64)) return true;
          if (*static_cast<volatile int*>(&s_abort)) return false;
        }
        return false;
      };
      long long g = 0;
      for (; g < total_chunks; ++g) {
        const int b = static_cast<int>(g % kChunkBufs);
        if (g >= kChunkBufs) {
          const long long h = g - kChunkBufs;
          if (!wait_or_abort(s_u32(&mbar_buf[b]), static_cast<uint32_t>((h / kChunkBufs) & 1))) {
            s_abort = 1;
            break;
          }
        }
        const uint8_t* src = a.Wimg + kSmemW1 + static_cast<size_t>(g % 8) * kSmemS;
        const uint32_t bar = s_u32(&mbar_full[b]);
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(kSmemS) : "memory");
        asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                         s_u32(sS + b * kSmemS)),
                     "l"(src), "r"(kSmemS), "r"(bar)
                     : "memory");
      }
      // the last copy issued into each buffer has landed before the shared memory is released (bounded)
      for (long long h = g > kChunkBufs ? g - kChunkBufs : 0; h < g; ++h)
        mbar_wait_parity(s_u32(&mbar_full[h % kChunkBufs]), static_cast<uint32_t>((h / kChunkBufs) & 1), kMbarLimit);
    }
  } else {
    long long tile = blockIdx.x;
    uint32_t par = 0;
    if (tile < n_tiles) {
      feat_index(tile);
      feat_points();
      feat_waypoint();
      for (int p = 0; p < 4; ++p) feat_part(p);
      bar_sync_main();
      issue_l1(0u);
      if (tile + gridDim.x < n_tiles) feat_index(tile + gridDim.x);
    }
    for (; tile < n_tiles && ok; tile += gridDim.x, par ^= 1u) {
      const uint32_t accA = par ? 256u : 0u, accB = par ? 0u : 256u;
      const long long next = tile + gridDim.x;
      // this thread's edge of the head (threads 0..127) and the next tile's query: their index loads
      // are issued now and used a layer later
      size_t pidx = 0;
      bool prot = false;
      const long long e_mine = tile * e_per_tile + tid;
      const bool mine = tid < e_per_tile && e_mine < n_live;
      int hr = 0, hc = 0;
      if (mine) {
        int r, cidx;
        split_edge(e_mine, r, cidx);
        hr = rows_live[r];
        hc = cols_live[cidx];
      }
      // the next tile's end points (its indices were loaded a tile earlier), used under layer 1's epilogue
      if (next < n_tiles) feat_points();
      // layer 1, issued under the previous tile's head, is long done: each thread waits for it on its
      // own (the barrier's completion orders the accumulator for this thread's tensor-memory reads),
      // and a timeout joins the CTA's decision at the layer-2 wait
      const bool l1_ok = mbar_wait_parity(mbl, ph_layer, kMbarLimit);
      ph_layer ^= 1u;
      if (next < n_tiles) feat_waypoint();
      for (int l = 0; l < 2 && ok; ++l) {
        if (l == 1) {
          // the indices of the tile after next, and this edge's protection mark, under layer 2
          if (next + gridDim.x < n_tiles) feat_index(next + gridDim.x);
          if (mine) {
            pidx = static_cast<size_t>(hr) * cols + hc;
            if (a.protect) prot = a.prune[pidx] == kPruneProtected;
          }
          ok = wait_layer(l1_ok);  // layer 2 (and layer 1's outcome)
          if (!ok) break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t acc_in = l == 0 ? accA : accB, acc_out = l == 0 ? accB : accA;
        const float* bias = l == 0 ? b1 : b2;
        for (int c = 0; c < 4; ++c) {
          // epilogue chunk c: this warp's 32 columns [n0, n0 + 32) of acc_in -> relu(acc + b) -> bf16 pairs,
          // written back over the first 16 of those columns (read by this warp alone, and already read):
          // there they are K-slice [n0, n0 + 32) of layer l + 1's A operand
          if (epi) {
            const int n0 = c * 64 + half * 32;
            uint32_t v[32];
            tmem_ld32(lane_addr + acc_in + n0, v);
            uint32_t w[16];
#pragma unroll
            for (int g4 = 0; g4 < 8; ++g4) {
              const float4 bb = *reinterpret_cast<const float4*>(bias + n0 + g4 * 4);
              // relu and the bf16 rounding in one conversion (the high half takes the first operand); it
              // differs from max-then-round only in the sign of a zero, which no product sees, and in
              // passing a NaN on (a model with NaN weights then prunes nothing: z > cut fails)
              const float2 a0 = __fadd2_rn(make_float2(__uint_as_float(v[4 * g4]), __uint_as_float(v[4 * g4 + 1])),
                                           make_float2(bb.x, bb.y));
              const float2 a1 = __fadd2_rn(make_float2(__uint_as_float(v[4 * g4 + 2]), __uint_as_float(v[4 * g4 + 3])),
                                           make_float2(bb.z, bb.w));
              asm("cvt.rn.relu.bf16x2.f32 %0, %1, %2;" : "=r"(w[2 * g4]) : "f"(a0.y), "f"(a0.x));
              asm("cvt.rn.relu.bf16x2.f32 %0, %1, %2;" : "=r"(w[2 * g4 + 1]) : "f"(a1.y), "f"(a1.x));
            }
            tmem_st16(lane_addr + acc_in + n0, w);
          }
          // a quarter of the next tile's features to X (layer 1 has read this tile's), while the MMAs of
          // chunk c - 1 run
          if (l == 0 && next < n_tiles) feat_part(c);
          // chunk g = chunks_issued goes to the MMAs once every epilogue chunk is in place (its tensor-memory
          // stores completed in tmem_st16) and its weights have landed.  A plain barrier (a reducing one
          // measured 8 % of the kernel): the abort flag, which the MMA or load thread may set at any time,
          // is taken at the next layer wait, which combines every thread's reading of it
          const long long g = chunks_issued;
          asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
          bar_sync_main();
          if (tid == kMmaThread) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t sb = s_u32(sS + static_cast<int>(g % kChunkBufs) * kSmemS);
            // after its own abort the MMA thread waits for nothing more (a load-thread abort shows here as
            // a chunk that never lands, the bounded wait's timeout)
            const bool go = !released && mbar_wait_parity(s_u32(&mbar_full[g % kChunkBufs]),
                                                          static_cast<uint32_t>((g / kChunkBufs) & 1), kMbarLimit);
            // K-step kk of chunk c: A columns 16 kk .. + 16 of the chunk, i.e. half kk / 2's packed
            // columns, 8 columns per 16 K
            if (go) {
              for (int kk = 0; kk < 4; ++kk)
                issue_mma_ts(tmem + acc_out, tmem + acc_in + c * 64 + (kk >> 1) * 32 + (kk & 1) * 8,
                             smem_desc(sb + kk * 256, 128, 1024), idesc, (c > 0 || kk > 0) ? 1u : 0u);
              // chunk g's MMAs free its buffer for chunk g + kChunkBufs (the load thread waits on this)
              asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                               s_u32(&mbar_buf[g % kChunkBufs]))
                           : "memory");
              if (c == 3)
                asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbl)
                             : "memory");
            } else if (!released) {
              // a timeout (here or in the load thread): the CTA stops at its next layer wait, whose
              // barrier is released once by hand
              s_abort = 1;
              asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(mbl) : "memory");
              released = true;
            }
          }
          ++chunks_issued;
        }
      }
      if (!ok) break;
      ok = wait_layer();  // layer 3 (accumulator A)
      if (!ok) break;
      // the next tile's layer-1 MMAs into B (its X was stored under layer 1's epilogue, before this
      // tile's chunk barriers), under this head; the MMA thread issues after the barrier (issuing
      // before it would hold every warp's head back by the ~1 k cycles the issue blocks)
      if (next < n_tiles) issue_l1(accB);
      // head: relu(acc + b3) . w4 + b4, per query; then the edge's max against the cut
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      float dot = 0.0f;
      for (int cp = 0; cp < 2 && epi; ++cp) {
        uint32_t v[64];
        tmem_ld64(lane_addr + accA + half * 128 + cp * 64, v);
#pragma unroll
        for (int c2 = 0; c2 < 2; ++c2) {
          const int n0 = half * 128 + (2 * cp + c2) * 32;
          // four partial sums: a short dependency chain
          float part[4] = {0.0f, 0.0f, 0.0f, 0.0f};
#pragma unroll
          for (int j4 = 0; j4 < 8; ++j4) {
            const float4 bb = *reinterpret_cast<const float4*>(b3 + n0 + 4 * j4);
            const float4 ww = *reinterpret_cast<const float4*>(w4 + n0 + 4 * j4);
            const uint32_t* vv = v + 32 * c2 + 4 * j4;
            const float2 s0 = __fadd2_rn(make_float2(__uint_as_float(vv[0]), __uint_as_float(vv[1])),
                                         make_float2(bb.x, bb.y));
            const float2 s1 = __fadd2_rn(make_float2(__uint_as_float(vv[2]), __uint_as_float(vv[3])),
                                         make_float2(bb.z, bb.w));
            const float2 p01 = __ffma2_rn(make_float2(fmaxf(s0.x, 0.0f), fmaxf(s0.y, 0.0f)), make_float2(ww.x, ww.y),
                                          make_float2(part[0], part[1]));
            const float2 p23 = __ffma2_rn(make_float2(fmaxf(s1.x, 0.0f), fmaxf(s1.y, 0.0f)), make_float2(ww.z, ww.w),
                                          make_float2(part[2], part[3]));
            part[0] = p01.x;
            part[1] = p01.y;
            part[2] = p23.x;
            part[3] = p23.y;
          }
          dot += (part[0] + part[1]) + (part[2] + part[3]);
        }
      }
      if (epi) s_part[half][row] = dot;
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      bar_sync_main();
      if (tid < 128) {  // warps 0..3, full warps for the ballot, under a barrier of their own
        s_logit[tid] = s_part[0][tid] + s_part[1][tid] + b4;
        asm volatile("bar.sync 1, 128;" ::: "memory");
        bool pr = false;
        if (mine) {
          float z = s_logit[tid * a.kw];
          for (int w = 1; w < a.kw; ++w) z = fmaxf(z, s_logit[tid * a.kw + w]);
          pr = z > a.cut && !prot;
          a.prune[pidx] = pr ? 1 : 0;
        }
        const unsigned b = __ballot_sync(kFull, pr);
        if (lane == 0 && b) atomicAdd(a.n_pruned, static_cast<unsigned long long>(__popc(b)));
      }
      // s_part and s_logit are next written after the next tile's first CTA barrier
    }
    if (!ok) s_abort = 1;  // the load thread stops streaming
    if (tid == kMmaThread) {
      // every MMA this CTA issued has completed before TMEM is freed (bounded)
      bool drained = true;
      if (any_mma) {
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                         s_u32(&mbar_fin))
                     : "memory");
        drained = mbar_wait_parity(s_u32(&mbar_fin), 0u, kMbarLimit);
      }
      if (!ok || !drained) atomicOr(a.err, kErrWaitTimeout);
      // the W1 copy has landed before the shared memory is released, also in a CTA that got no tile
      // (the grid is sized by all edges, the tiles by the live ones) or stopped early (bounded)
      if (!w1_ready) mbar_wait_parity(s_u32(&mbar_w1), 0u, kMbarLimit);
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512) : "memory");
}

struct SurrogateState {
  int dof = 0;
  FourierDev four{};
  float* P = nullptr;  // fp32 master parameters [kParamCount]: W1 b1 W2 b2 W3 b3 w4 b4
  float* G = nullptr;  // gradients, same layout
  float* Mm = nullptr;
  float* Vv = nullptr;
  __nv_bfloat16 *W1b = nullptr, *W1bT = nullptr, *W2b = nullptr, *W2bT = nullptr, *W3b = nullptr, *W3bT = nullptr;
  int cap = 0;  // rows of the activation buffers
  __nv_bfloat16 *X = nullptr, *XT = nullptr, *H1 = nullptr, *H1T = nullptr, *H2 = nullptr, *H2T = nullptr,
                *H3 = nullptr, *H3T = nullptr, *dA = nullptr, *dAT = nullptr, *dB = nullptr, *dBT = nullptr;
  float *logits = nullptr, *dz = nullptr;
  double* loss = nullptr;
  unsigned long long* counter = nullptr;
  int* live = nullptr;  // live rows / columns of the transition being scored: [2 + 2 * live_cap]
  uint8_t* wimg = nullptr;  // weight images of the scoring kernel (W1, then 8 chunks of W2 / W3)
  int live_cap = 0;
  bool trained = false;
  long long steps = 0;
};

void surrogate_free(SurrogateState* s) {
  if (!s) return;
  void* bufs[] = {s->P,   s->G,   s->Mm,  s->Vv,  s->W1b, s->W1bT,   s->W2b,     s->W2bT, s->W3b,
                  s->W3bT, s->X,  s->XT,  s->H1,  s->H1T, s->H2,     s->H2T,     s->H3,   s->H3T,
                  s->dA,  s->dAT, s->dB,  s->dBT, s->logits, s->dz, s->loss, s->counter, s->live, s->wimg};
  for (void* b : bufs) cudaFree(b);
  delete s;
}

namespace {

float* pW1(SurrogateState* s, float* base) { return base; }
float* pb1(SurrogateState* s, float* base) { return base + kNW1; }
float* pW2(SurrogateState* s, float* base) { return base + kNW1 + kHid; }
float* pb2(SurrogateState* s, float* base) { return pW2(s, base) + kNW2; }
float* pW3(SurrogateState* s, float* base) { return pb2(s, base) + kHid; }
float* pb3(SurrogateState* s, float* base) { return pW3(s, base) + kNW3; }
float* pw4(SurrogateState* s, float* base) { return pb3(s, base) + kHid; }
float* pb4(SurrogateState* s, float* base) { return pw4(s, base) + kHid; }

cudaError_t ensure_buffers(SurrogateState* s, int cap) {
  if (s->cap >= cap) return cudaSuccess;
  __nv_bfloat16** bufs[] = {&s->X, &s->XT, &s->H1, &s->H1T, &s->H2, &s->H2T, &s->H3, &s->H3T,
                            &s->dA, &s->dAT, &s->dB, &s->dBT};
  for (auto b : bufs) {
    cudaFree(*b);
    *b = nullptr;
  }
  cudaFree(s->logits);
  cudaFree(s->dz);
  s->logits = s->dz = nullptr;
  s->cap = 0;
  cudaError_t e = cudaSuccess;
  for (auto b : bufs)
    if (e == cudaSuccess) e = cudaMalloc(b, static_cast<size_t>(cap) * kHid * sizeof(__nv_bfloat16));
  if (e == cudaSuccess) e = cudaMalloc(&s->logits, static_cast<size_t>(cap) * sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc(&s->dz, static_cast<size_t>(cap) * sizeof(float));
  if (e == cudaSuccess) s->cap = cap;
  return e;
}

UmmaArgs gemm_args(const __nv_bfloat16* A, int lda, const __nv_bfloat16* B, int ldb, int M, int N, int K, int* err) {
  UmmaArgs a{};
  a.A = A;
  a.lda = lda;
  a.B = B;
  a.ldb = ldb;
  a.M = M;
  a.N = N;
  a.K = K;
  a.err = err;
  return a;
}

// forward of rows [X] (bf16 [n][128]) -> logits; training also keeps H and H^T
cudaError_t forward(SurrogateState* s, const __nv_bfloat16* X, int n, bool keep, int ldT, int* err,
                    cudaStream_t st) {
  cudaError_t e;
  UmmaArgs a = gemm_args(X, kFeat, s->W1b, kFeat, n, kHid, kFeat, err);
  a.bias = pb1(s, s->P);
  a.out = s->H1;
  a.ldo = kHid;
  a.outT = keep ? s->H1T : nullptr;
  a.ldoT = ldT;
  if ((e = umma_gemm(a, kEpiBiasReluBf16, st)) != cudaSuccess) return e;
  a = gemm_args(s->H1, kHid, s->W2b, kHid, n, kHid, kHid, err);
  a.bias = pb2(s, s->P);
  a.out = s->H2;
  a.ldo = kHid;
  a.outT = keep ? s->H2T : nullptr;
  a.ldoT = ldT;
  if ((e = umma_gemm(a, kEpiBiasReluBf16, st)) != cudaSuccess) return e;
  a = gemm_args(s->H2, kHid, s->W3b, kHid, n, kHid, kHid, err);
  a.bias = pb3(s, s->P);
  a.w4 = pw4(s, s->P);
  a.b4 = pb4(s, s->P);
  a.out = keep ? s->H3 : nullptr;
  a.ldo = kHid;
  a.outT = keep ? s->H3T : nullptr;
  a.ldoT = ldT;
  a.logits = s->logits;
  return umma_gemm(a, kEpiHead, st);
}

// Forward and backward of one batch: gradients of the mean binary
// cross-entropy into s->G, summed loss added to *s->loss.  X: bf16 [batch][128]
// features; XT: the same features transposed, rows of stride ldXT.
cudaError_t batch_gradients(SurrogateState* s, const __nv_bfloat16* X, const __nv_bfloat16* XT, int ldXT,
                            const uint8_t* labels, int batch, int* err, cudaStream_t st) {
  cudaError_t e;
  if ((e = forward(s, X, batch, true, batch, err, st)) != cudaSuccess) return e;
  head_backward_kernel<<<batch, 256, 0, st>>>(s->logits, labels, 0, batch, pw4(s, s->P), s->H3, s->dA, s->dAT,
                                              batch, s->dz, s->loss);
  colsum_kernel<<<kHid, 256, 0, st>>>(s->H3T, batch, batch, s->dz, pw4(s, s->G));
  sum_kernel<<<1, 256, 0, st>>>(s->dz, batch, pb4(s, s->G));
  // layer 3: dW3 = dA3^T H2, db3, dA2 = (dA3 W3) * (H2 > 0)
  UmmaArgs a = gemm_args(s->dAT, batch, s->H2T, batch, kHid, kHid, batch, err);
  a.outf = pW3(s, s->G);
  a.ldf = kHid;
  if ((e = umma_gemm(a, kEpiF32, st)) != cudaSuccess) return e;
  colsum_kernel<<<kHid, 256, 0, st>>>(s->dAT, batch, batch, nullptr, pb3(s, s->G));
  a = gemm_args(s->dA, kHid, s->W3bT, kHid, batch, kHid, kHid, err);
  a.mask = s->H2;
  a.ldm = kHid;
  a.out = s->dB;
  a.ldo = kHid;
  a.outT = s->dBT;
  a.ldoT = batch;
  if ((e = umma_gemm(a, kEpiMaskBf16, st)) != cudaSuccess) return e;
  // layer 2
  a = gemm_args(s->dBT, batch, s->H1T, batch, kHid, kHid, batch, err);
  a.outf = pW2(s, s->G);
  a.ldf = kHid;
  if ((e = umma_gemm(a, kEpiF32, st)) != cudaSuccess) return e;
  colsum_kernel<<<kHid, 256, 0, st>>>(s->dBT, batch, batch, nullptr, pb2(s, s->G));
  a = gemm_args(s->dB, kHid, s->W2bT, kHid, batch, kHid, kHid, err);
  a.mask = s->H1;
  a.ldm = kHid;
  a.out = s->dA;
  a.ldo = kHid;
  a.outT = s->dAT;
  a.ldoT = batch;
  if ((e = umma_gemm(a, kEpiMaskBf16, st)) != cudaSuccess) return e;
  // layer 1: dW1 = dA1^T X
  a = gemm_args(s->dAT, batch, XT, ldXT, kHid, kFeat, batch, err);
  a.outf = pW1(s, s->G);
  a.ldf = kFeat;
  if ((e = umma_gemm(a, kEpiF32, st)) != cudaSuccess) return e;
  colsum_kernel<<<kHid, 256, 0, st>>>(s->dAT, batch, batch, nullptr, pb1(s, s->G));
  return cudaGetLastError();
}

}  // namespace
}  // namespace gtmp

using namespace gtmp;

namespace {

gtmp_status sfail(gtmp_ctx* c, gtmp_status s, const char* msg, cudaError_t e = cudaSuccess) {
  if (c) {
    c->last_error = msg;
    if (e != cudaSuccess) c->last_error += std::string(": ") + cudaGetErrorString(e);
  }
  return s;
}

#define SUR_TRY(ctx, expr)                                                                                  \
  do {                                                                                                      \
    cudaError_t e_ = (expr);                                                                                \
    if (e_ != cudaSuccess)                                                                                  \
      return sfail((ctx), e_ == cudaErrorMemoryAllocation ? GTMP_ERR_OOM : GTMP_ERR_CUDA, #expr, e_);       \
  } while (0)

SceneDev ctx_scene(gtmp_ctx* c) {
  SceneDev s = c->sc;
  s.obs = c->obs;
  return s;
}

}  // namespace

extern "C" {

GTMP_API gtmp_status gtmp_surrogate_train(gtmp_ctx* c, const gtmp_surrogate_config* cfg, gtmp_surrogate_stats* out) {
  GtmpNvtxRange nvtx_("gtmp_surrogate_train");
  if (!c || !cfg) return GTMP_ERR_INVALID_ARG;
  const int n_train = cfg->n_train, n_hold = cfg->n_holdout, batch = cfg->batch, epochs = cfg->epochs;
  if (n_train < 64 || n_train % 64 != 0 || n_hold < 0 || batch < 64 || batch % 64 != 0 || batch > n_train ||
      epochs < 1 ||
      !(cfg->lr > 0.0f) || n_train > (1 << 26) || n_hold > (1 << 26) || c->dof > kMaxDof)
    return sfail(c, GTMP_ERR_INVALID_ARG,
                 "bad surrogate configuration (n_train and batch multiples of 64, batch <= n_train)");
  cudaStream_t st = c->stream;
  if (!c->sur) c->sur = new SurrogateState();
  SurrogateState* s = c->sur;
  s->dof = c->dof;
  // ---- parameters: Fourier frequencies B ~ N(0, 1) per rad, Kaiming-uniform weights, zero biases
  std::mt19937_64 rng(cfg->seed ^ 0x5eed5u);
  std::normal_distribution<float> nd(0.0f, cfg->fourier_sigma > 0.0f ? cfg->fourier_sigma : 1.0f);
  s->four.dof = c->dof;
  for (int k = 0; k < 64 * c->dof; ++k) s->four.B[k] = nd(rng);
  std::vector<float> host(kParamCount, 0.0f);
  auto init = [&](float* w, int n, int fan_in) {
    std::uniform_real_distribution<float> ud(-1.0f / std::sqrt(float(fan_in)), 1.0f / std::sqrt(float(fan_in)));
    for (int i = 0; i < n; ++i) w[i] = ud(rng);
  };
  init(pW1(s, host.data()), kNW1, kFeat);
  init(pW2(s, host.data()), kNW2, kHid);
  init(pW3(s, host.data()), kNW3, kHid);
  init(pw4(s, host.data()), kHid, kHid);
  if (!s->P) {
    SUR_TRY(c, cudaMalloc(&s->P, kParamCount * sizeof(float)));
    SUR_TRY(c, cudaMalloc(&s->G, kParamCount * sizeof(float)));
    SUR_TRY(c, cudaMalloc(&s->Mm, kParamCount * sizeof(float)));
    SUR_TRY(c, cudaMalloc(&s->Vv, kParamCount * sizeof(float)));
    SUR_TRY(c, cudaMalloc(&s->W1b, kNW1 * sizeof(__nv_bfloat16)));
    SUR_TRY(c, cudaMalloc(&s->W1bT, kNW1 * sizeof(__nv_bfloat16)));
    SUR_TRY(c, cudaMalloc(&s->W2b, kNW2 * sizeof(__nv_bfloat16)));
    SUR_TRY(c, cudaMalloc(&s->W2bT, kNW2 * sizeof(__nv_bfloat16)));
    SUR_TRY(c, cudaMalloc(&s->W3b, kNW3 * sizeof(__nv_bfloat16)));
    SUR_TRY(c, cudaMalloc(&s->W3bT, kNW3 * sizeof(__nv_bfloat16)));
    SUR_TRY(c, cudaMalloc(&s->loss, sizeof(double)));
    SUR_TRY(c, cudaMalloc(&s->counter, sizeof(unsigned long long)));
  }
  SUR_TRY(c, cudaMemcpyAsync(s->P, host.data(), kParamCount * sizeof(float), cudaMemcpyHostToDevice, st));
  SUR_TRY(c, cudaMemsetAsync(s->Mm, 0, kParamCount * sizeof(float), st));
  SUR_TRY(c, cudaMemsetAsync(s->Vv, 0, kParamCount * sizeof(float), st));
  f32_to_bf16_kernel<<<nblk(kNW1, 256), 256, 0, st>>>(pW1(s, s->P), kHid, kFeat, s->W1b, s->W1bT);
  f32_to_bf16_kernel<<<nblk(kNW2, 256), 256, 0, st>>>(pW2(s, s->P), kHid, kHid, s->W2b, s->W2bT);
  f32_to_bf16_kernel<<<nblk(kNW3, 256), 256, 0, st>>>(pW3(s, s->P), kHid, kHid, s->W3b, s->W3bT);
  SUR_TRY(c, cudaGetLastError());
  SUR_TRY(c, ensure_buffers(s, batch));
  // ---- data: configurations uniform in the joint box, labelled by the exact checker
  const int n_all = n_train + n_hold;
  float *q = nullptr, *lo = nullptr, *hi = nullptr;
  uint8_t* y = nullptr;
  __nv_bfloat16 *F = nullptr, *FT = nullptr;
  auto release = [&]() {
    cudaFree(q);
    cudaFree(lo);
    cudaFree(hi);
    cudaFree(y);
    cudaFree(F);
    cudaFree(FT);
  };
  cudaError_t e = cudaSuccess;
  if (e == cudaSuccess) e = cudaMalloc(&q, static_cast<size_t>(n_all) * c->dof * sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc(&lo, kMaxDof * sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc(&hi, kMaxDof * sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc(&y, n_all);
  if (e == cudaSuccess) e = cudaMalloc(&F, static_cast<size_t>(n_all) * kFeat * sizeof(__nv_bfloat16));
  if (e == cudaSuccess) e = cudaMalloc(&FT, static_cast<size_t>(n_train) * kFeat * sizeof(__nv_bfloat16));
  if (e == cudaSuccess) e = cudaMemcpyAsync(lo, c->q_lo, kMaxDof * sizeof(float), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(hi, c->q_hi, kMaxDof * sizeof(float), cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) {
    release();
    return sfail(c, e == cudaErrorMemoryAllocation ? GTMP_ERR_OOM : GTMP_ERR_CUDA, "surrogate data buffers", e);
  }
  cudaEvent_t t0, t1;
  cudaEventCreate(&t0);
  cudaEventCreate(&t1);
  cudaEventRecord(t0, st);
  train_configs_kernel<<<nblk(n_all, 256), 256, 0, st>>>(n_all, c->dof, s->four, cfg->seed, lo, hi, q);
  e = launch_label_configs(q, n_all, c->dof, c->rb, c->variant, ctx_scene(c), y, st);
  if (e == cudaSuccess) {
    features_kernel<<<nblk(n_train, 128), 128, 0, st>>>(q, n_train, s->four, F, FT, n_train);
    features_kernel<<<nblk(n_hold, 128), 128, 0, st>>>(q + static_cast<size_t>(n_train) * c->dof, n_hold, s->four,
                                                         F + static_cast<size_t>(n_train) * kFeat, nullptr, 0);
    e = cudaGetLastError();
  }
  // ---- epochs of mini-batch Adam on binary cross-entropy
  const int steps_per_epoch = n_train / batch;
  double last_loss = 0.0;
  for (int ep = 0; ep < epochs && e == cudaSuccess; ++ep) {
    cudaMemsetAsync(s->loss, 0, sizeof(double), st);
    for (int b = 0; b < steps_per_epoch && e == cudaSuccess; ++b) {
      const int b0 = b * batch;
      const __nv_bfloat16* X = F + static_cast<size_t>(b0) * kFeat;
      const __nv_bfloat16* XT = FT + b0;  // rows of FT have stride n_train
      if ((e = batch_gradients(s, X, XT, n_train, y + b0, batch, c->err, st)) != cudaSuccess) break;
      // Adam
      s->steps += 1;
      const float b1 = 0.9f, b2 = 0.999f;
      const float c1 = 1.0f - std::pow(b1, float(s->steps)), c2 = 1.0f - std::pow(b2, float(s->steps));
      struct T {
        float* (*at)(SurrogateState*, float*);
        int n, rows, cols;
        __nv_bfloat16 *wb, *wbT;
      } tensors[] = {{pW1, kNW1, kHid, kFeat, s->W1b, s->W1bT}, {pb1, kHid, 1, kHid, nullptr, nullptr},
                     {pW2, kNW2, kHid, kHid, s->W2b, s->W2bT},  {pb2, kHid, 1, kHid, nullptr, nullptr},
                     {pW3, kNW3, kHid, kHid, s->W3b, s->W3bT},  {pb3, kHid, 1, kHid, nullptr, nullptr},
                     {pw4, kHid, 1, kHid, nullptr, nullptr},    {pb4, 1, 1, 1, nullptr, nullptr}};
      for (const T& t : tensors)
        adam_kernel<<<nblk(t.n, 256), 256, 0, st>>>(t.at(s, s->P), t.at(s, s->G), t.at(s, s->Mm), t.at(s, s->Vv),
                                                    t.n, cfg->lr, b1, b2, 1e-8f, c1, c2, t.wb, t.wbT, t.rows, t.cols);
      e = cudaGetLastError();
    }
    if (e == cudaSuccess) {
      double l = 0.0;
      e = cudaMemcpyAsync(&l, s->loss, sizeof(double), cudaMemcpyDeviceToHost, st);
      if (e == cudaSuccess) e = cudaStreamSynchronize(st);
      last_loss = l / (static_cast<double>(steps_per_epoch) * batch);
    }
  }
  cudaEventRecord(t1, st);
  // ---- held-out statistics
  float acc = 0.0f, fn = 0.0f, fp = 0.0f;
  if (e == cudaSuccess && n_hold > 0) {
    std::vector<float> z(n_hold);
    std::vector<uint8_t> yl(n_hold);
    for (int r0 = 0; r0 < n_hold && e == cudaSuccess; r0 += batch) {
      const int nr = std::min(batch, n_hold - r0);
      e = forward(s, F + static_cast<size_t>(n_train + r0) * kFeat, nr, false, 0, c->err, st);
      if (e == cudaSuccess)
        e = cudaMemcpyAsync(z.data() + r0, s->logits, nr * sizeof(float), cudaMemcpyDeviceToHost, st);
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(yl.data(), y + n_train, n_hold, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    long long n_pos = 0, n_neg = 0, ok = 0, miss = 0, false_alarm = 0;
    for (int i = 0; i < n_hold; ++i) {
      const bool pred = z[i] > 0.0f;  // p > 1/2
      const bool lab = yl[i] != 0;
      ok += pred == lab;
      if (lab) {
        ++n_pos;
        miss += !pred;
      } else {
        ++n_neg;
        false_alarm += pred;
      }
    }
    acc = float(ok) / n_hold;
    fn = n_pos ? float(miss) / n_pos : 0.0f;
    fp = n_neg ? float(false_alarm) / n_neg : 0.0f;
  }
  float ms = 0.0f;
  if (e == cudaSuccess) {
    cudaEventSynchronize(t1);
    cudaEventElapsedTime(&ms, t0, t1);
  }
  cudaEventDestroy(t0);
  cudaEventDestroy(t1);
  release();
  if (e != cudaSuccess) return sfail(c, GTMP_ERR_CUDA, "surrogate training", e);
  s->trained = true;
  if (out) {
    out->final_loss = static_cast<float>(last_loss);
    out->holdout_accuracy = acc;
    out->holdout_fn_rate = fn;
    out->holdout_fp_rate = fp;
    out->train_ms = ms;
  }
  return GTMP_OK;
}

GTMP_API gtmp_status gtmp_surrogate_predict(gtmp_ctx* c, const float* dev_q, int32_t n, float* dev_logits) {
  if (!c || n < 0 || (n > 0 && (!dev_q || !dev_logits))) return GTMP_ERR_INVALID_ARG;
  if (!c->sur || !c->sur->trained) return sfail(c, GTMP_ERR_NOT_READY, "surrogate not trained");
  SurrogateState* s = c->sur;
  cudaStream_t st = c->stream;
  const int chunk = 1 << 16;
  SUR_TRY(c, ensure_buffers(s, std::min(std::max(n, 128), chunk)));
  for (int r0 = 0; r0 < n; r0 += s->cap) {
    const int nr = std::min(s->cap, n - r0);
    features_kernel<<<nblk(nr, 128), 128, 0, st>>>(dev_q + static_cast<size_t>(r0) * c->dof, nr, s->four, s->X,
                                                   nullptr, 0);
    SUR_TRY(c, cudaGetLastError());
    SUR_TRY(c, forward(s, s->X, nr, false, 0, c->err, st));
    SUR_TRY(c, cudaMemcpyAsync(dev_logits + r0, s->logits, nr * sizeof(float), cudaMemcpyDeviceToDevice, st));
  }
  return GTMP_OK;
}

GTMP_API gtmp_status gtmp_surrogate_get_params(gtmp_ctx* c, float* host_params, int64_t n, float* host_fourier,
                                               int64_t n_fourier) {
  if (!c || !host_params || n != kParamCount || !host_fourier || n_fourier != 64 * c->dof)
    return sfail(c, GTMP_ERR_INVALID_ARG, "parameter buffer sizes must match gtmp_surrogate_param_count");
  if (!c->sur || !c->sur->trained) return sfail(c, GTMP_ERR_NOT_READY, "surrogate not trained");
  SUR_TRY(c, cudaMemcpyAsync(host_params, c->sur->P, kParamCount * sizeof(float), cudaMemcpyDeviceToHost, c->stream));
  SUR_TRY(c, cudaStreamSynchronize(c->stream));
  for (int k = 0; k < 64 * c->dof; ++k) host_fourier[k] = c->sur->four.B[k];
  return GTMP_OK;
}

GTMP_API int64_t gtmp_surrogate_param_count(void) { return kParamCount; }

}  // extern "C"

namespace {

// Buffers, kernel attributes and the weight images the scoring kernel needs
// (the images are rebuilt from the current weights on every call).
gtmp_status prepare_scoring(gtmp_ctx* c) {
  SurrogateState* s = c->sur;
  cudaStream_t st = c->stream;
  if (s->live_cap < c->p.M) {
    cudaFree(s->live);
    s->live = nullptr;
    s->live_cap = 0;
    SUR_TRY(c, cudaMalloc(&s->live, (2 + 2 * static_cast<size_t>(c->p.M)) * sizeof(int)));
    s->live_cap = c->p.M;
  }
  SUR_TRY(c, cudaFuncSetAttribute(score_edges_kernel<7>, cudaFuncAttributeMaxDynamicSharedMemorySize, kScoreSmem));
  SUR_TRY(c, cudaFuncSetAttribute(score_edges_kernel<6>, cudaFuncAttributeMaxDynamicSharedMemorySize, kScoreSmem));
  SUR_TRY(c, cudaFuncSetAttribute(score_edges_kernel<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, kScoreSmem));
  if (!s->wimg) SUR_TRY(c, cudaMalloc(&s->wimg, static_cast<size_t>(kSmemW1) + 8 * static_cast<size_t>(kSmemS)));
  weight_images_kernel<<<(256 * 16 + 8 * 256 * 8 + 255) / 256, 256, 0, st>>>(s->W1b, s->W2b, s->W3b, s->wimg);
  SUR_TRY(c, cudaGetLastError());
  SUR_TRY(c, cudaMemsetAsync(s->counter, 0, sizeof(unsigned long long), st));
  return GTMP_OK;
}

GraphDev pruned_graph(gtmp_ctx* c) {
  GraphDev g;
  g.Q = c->Q;
  g.vflag = c->vflag;
  g.keys = c->keys;
  g.R = 1;
  g.L = c->p.L;
  g.M = c->M_active;
  g.dp = c->dp;
  g.H = c->p.H;
  g.M_stride = c->p.M;
  g.max_edge_len = c->p.max_edge_len;
  g.G = c->G;
  g.gval = c->goal_values ? c->gval : nullptr;
  return g;
}

// Score the live edges of transition `layer` (rows = its live vertices, columns
// = the next layer's free vertices with a finite cost-to-go in the keys) into
// prune[i * cols + j]: 1 = pruned, 0 = kept; other entries are not written.
// band_start, band_done (optional): recorded after the live lists and after the protection-band pass,
// before the scoring kernel
gtmp_status launch_score_transition(gtmp_ctx* c, const GraphDev& g, int layer, float cut, int kw, uint8_t* prune,
                                    cudaEvent_t band_start = nullptr, cudaEvent_t band_done = nullptr) {
  SurrogateState* s = c->sur;
  cudaStream_t st = c->stream;
  const long long ne = static_cast<long long>(layer_size(g, layer)) * layer_size(g, layer + 1);
  ScoreArgs sa{};
  sa.g = g;
  sa.layer = layer;
  sa.live = s->live;
  sa.cap = s->live_cap;
  sa.kw = kw;
  sa.cut = cut;
  sa.W1b = s->W1b;
  sa.W2b = s->W2b;
  sa.W3b = s->W3b;
  sa.Wimg = s->wimg;
  sa.P = s->P;
  sa.prune = prune;
  sa.n_pruned = s->counter;
  sa.err = c->err;
  sa.protect = c->sur_protect > 0.0f ? 1 : 0;
  // the live count stays on the device: a persistent grid reads it
  live_lists_kernel<<<1, 1024, 0, st>>>(g, layer, s->live_cap, s->live);
  SUR_TRY(c, cudaGetLastError());
  if (band_start) cudaEventRecord(band_start, st);
  if (sa.protect) {
    protect_band_kernel<<<(layer_size(g, layer) * 32 + 255) / 256, 256, 0, st>>>(g, layer, s->live, s->live_cap,
                                                                              1.0f + c->sur_protect, prune);
    SUR_TRY(c, cudaGetLastError());
  }
  if (band_done) cudaEventRecord(band_done, st);
  const long long tiles = (ne + 128 / kw - 1) / (128 / kw);
  const int score_grid = static_cast<int>(std::min<long long>(tiles, c->num_sms));
  if (s->four.dof == 7)
    score_edges_kernel<7><<<score_grid, kScoreThreads, kScoreSmem, st>>>(sa, s->four);
  else if (s->four.dof == 6)
    score_edges_kernel<6><<<score_grid, kScoreThreads, kScoreSmem, st>>>(sa, s->four);
  else
    score_edges_kernel<0><<<score_grid, kScoreThreads, kScoreSmem, st>>>(sa, s->four);
  SUR_TRY(c, cudaGetLastError());
  return GTMP_OK;
}

}  // namespace

extern "C" {

GTMP_API gtmp_status gtmp_surrogate_set_protect(gtmp_ctx* c, float band) {
  if (!c || !(band >= 0.0f && band <= 16.0f)) return sfail(c, GTMP_ERR_INVALID_ARG, "protection band must be in [0, 16]");
  c->sur_protect = band;
  return GTMP_OK;
}

GTMP_API gtmp_status gtmp_surrogate_score(gtmp_ctx* c, int32_t layer, float threshold, int32_t score_waypoints,
                                          uint8_t* dev_mask, int64_t* host_scored) {
  GtmpNvtxRange nvtx_("gtmp_surrogate_score");
  if (!c || !dev_mask || !(threshold > 0.0f && threshold < 1.0f) || (score_waypoints != 1 && score_waypoints != 3))
    return sfail(c, GTMP_ERR_INVALID_ARG, "bad scoring request (threshold in (0, 1), 1 or 3 waypoints)");
  if (!c->sur || !c->sur->trained) return sfail(c, GTMP_ERR_NOT_READY, "surrogate not trained");
  if (!c->have_endpoints || c->M_active < 1) return sfail(c, GTMP_ERR_NOT_READY, "endpoints or samples missing");
  if (layer < 0 || layer > c->p.L) return sfail(c, GTMP_ERR_INVALID_ARG, "layer outside 0..L");
  gtmp_status r = prepare_scoring(c);
  if (r != GTMP_OK) return r;
  const GraphDev g = pruned_graph(c);
  const size_t n = static_cast<size_t>(layer_size(g, layer)) * layer_size(g, layer + 1);
  SUR_TRY(c, cudaMemsetAsync(dev_mask, 2, n, c->stream));
  r = launch_score_transition(c, g, layer, std::log(threshold / (1.0f - threshold)), score_waypoints, dev_mask);
  if (r != GTMP_OK) return r;
  int live_n[2] = {0, 0};
  SUR_TRY(c, cudaMemcpyAsync(live_n, c->sur->live, sizeof(live_n), cudaMemcpyDeviceToHost, c->stream));
  SUR_TRY(c, cudaStreamSynchronize(c->stream));
  if (host_scored) *host_scored = static_cast<int64_t>(live_n[0]) * live_n[1];
  return GTMP_OK;
}

GTMP_API gtmp_status gtmp_solve_pruned(gtmp_ctx* c, float threshold, int32_t score_waypoints, int32_t* dev_path,
                                       float* dev_cost, gtmp_prune_stats* stats) {
  GtmpNvtxRange nvtx_("gtmp_solve_pruned");
  if (!c || !dev_path || !dev_cost || !(threshold > 0.0f && threshold < 1.0f) ||
      (score_waypoints != 1 && score_waypoints != 3))
    return sfail(c, GTMP_ERR_INVALID_ARG, "bad pruned-solve request (threshold in (0, 1), 1 or 3 waypoints)");
  if (!c->sur || !c->sur->trained) return sfail(c, GTMP_ERR_NOT_READY, "surrogate not trained");
  if (!c->have_endpoints || c->M_active < 1) return sfail(c, GTMP_ERR_NOT_READY, "endpoints or samples missing");
  SurrogateState* s = c->sur;
  cudaStream_t st = c->stream;
  const int L = c->p.L;
  if (!c->prune) SUR_TRY(c, cudaMalloc(&c->prune, static_cast<size_t>(c->p.M) * c->p.M));
  gtmp_status r = prepare_scoring(c);
  if (r != GTMP_OK) return r;
  const float cut = std::log(threshold / (1.0f - threshold));  // logit of the threshold
  const GraphDev g = pruned_graph(c);
  cudaEvent_t e0, e1, e2, eb0, eb1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  cudaEventCreate(&e2);
  cudaEventCreate(&eb0);
  cudaEventCreate(&eb1);
  float score_ms = 0.0f, solve_ms = 0.0f, band_ms = 0.0f, lists_ms = 0.0f;
  SUR_TRY(c, launch_init_keys(g, c->counters, L + 1, st));
  SUR_TRY(c, launch_vertex_labels(g, c->rb, c->variant, ctx_scene(c), st));
  const int resident = c->num_sms * c->fused_bps[0];
  double edges_total = 0.0, scored_total = 0.0;
  for (int layer = L; layer >= 0; --layer) {
    const int rows = layer_size(g, layer), cols = layer_size(g, layer + 1);
    const long long ne = static_cast<long long>(rows) * cols;
    edges_total += static_cast<double>(ne);
    cudaEventRecord(e0, st);
    // score the live edges of the transition with the fused tensor-core kernel
    r = launch_score_transition(c, g, layer, cut, score_waypoints, c->prune, eb0, eb1);
    if (r != GTMP_OK) return r;
    cudaEventRecord(e1, st);
    // exact realisation of the surviving edges, fused with the min-plus step
    GraphDev gp = g;
    gp.prune = c->prune;
    if (c->p.eval_mode == GTMP_EVAL_LAZY) {
      // bound-ordered realisation of the surviving edges (one warp per 32-column block of a row)
      const long long units = static_cast<long long>(rows) * ((cols + 31) / 32);
      const int lgrid = static_cast<int>(std::max(1LL, std::min<long long>(resident, (units + 7) / 8)));
      SUR_TRY(c, launch_fused_transition(gp, layer, c->rb, c->variant, ctx_scene(c), GTMP_EVAL_LAZY,
                                         c->counters + layer, lgrid, 32, c->err, st));
    } else {
      long long chunk = ne / (static_cast<long long>(resident) * 64);
      if (chunk < 1) chunk = 1;
      if (chunk > 32) chunk = 32;
      if (c->variant == kVarPoint) chunk = 32;
      if (chunk > cols) chunk = cols;
      const long long n_chunks = rows * ((cols + chunk - 1) / chunk);
      int grid = resident;
      if (grid > (n_chunks + 7) / 8) grid = static_cast<int>((n_chunks + 7) / 8);
      SUR_TRY(c, launch_fused_transition(gp, layer, c->rb, c->variant, ctx_scene(c), GTMP_EVAL_EARLY_EXIT,
                                         c->counters + layer, grid, static_cast<int>(chunk), c->err, st));
    }
    int live_n[2] = {0, 0};
    SUR_TRY(c, cudaMemcpyAsync(live_n, s->live, sizeof(live_n), cudaMemcpyDeviceToHost, st));
    cudaEventRecord(e2, st);
    SUR_TRY(c, cudaEventSynchronize(e2));
    scored_total += static_cast<double>(live_n[0]) * live_n[1];
    // e0 | live lists | eb0 | protection band | eb1 | scoring kernel | e1 | exact transition | e2
    float a = 0.0f, b = 0.0f, bb = 0.0f, ll = 0.0f;
    cudaEventElapsedTime(&a, eb1, e1);
    cudaEventElapsedTime(&b, e1, e2);
    cudaEventElapsedTime(&bb, eb0, eb1);
    cudaEventElapsedTime(&ll, e0, eb0);
    score_ms += a;
    solve_ms += b;
    band_ms += bb;
    lists_ms += ll;
  }
  SUR_TRY(c, launch_extract_paths(g, dev_path, dev_cost, nullptr, st));
  unsigned long long pruned = 0;
  SUR_TRY(c, cudaMemcpyAsync(&pruned, s->counter, sizeof(pruned), cudaMemcpyDeviceToHost, st));
  SUR_TRY(c, cudaStreamSynchronize(st));
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaEventDestroy(e2);
  cudaEventDestroy(eb0);
  cudaEventDestroy(eb1);
  if (stats) {
    stats->edges = edges_total;
    stats->pruned = static_cast<double>(pruned);
    stats->score_ms = score_ms;
    stats->solve_ms = solve_ms;
    stats->scored = scored_total;
    stats->band_ms = band_ms;
    stats->lists_ms = lists_ms;
  }
  return GTMP_OK;
}

}  // extern "C"

extern "C" GTMP_API gtmp_status gtmp_umma_gemm_f32(const void* dev_A, int32_t lda, const void* dev_B, int32_t ldb,
                                                   int32_t M, int32_t N, int32_t K, float* dev_C, int32_t ldc,
                                                   void* cuda_stream, int32_t* dev_err) {
  if (!dev_A || !dev_B || !dev_C || !dev_err || M < 1 || N < 16 || N % 16 != 0 || K < 8 || K % 8 != 0 || lda < K ||
      ldb < K || lda % 8 != 0 || ldb % 8 != 0 || ldc < N)
    return GTMP_ERR_INVALID_ARG;
  if ((reinterpret_cast<uintptr_t>(dev_A) | reinterpret_cast<uintptr_t>(dev_B)) & 15) return GTMP_ERR_INVALID_ARG;
  UmmaArgs a{};
  a.A = static_cast<const __nv_bfloat16*>(dev_A);
  a.lda = lda;
  a.B = static_cast<const __nv_bfloat16*>(dev_B);
  a.ldb = ldb;
  a.M = M;
  a.N = N;
  a.K = K;
  a.outf = dev_C;
  a.ldf = ldc;
  a.err = dev_err;
  return gtmp::umma_gemm(a, gtmp::kEpiF32, static_cast<cudaStream_t>(cuda_stream)) == cudaSuccess ? GTMP_OK
                                                                                                 : GTMP_ERR_CUDA;
}


// ---------------------------------------------------------------------------
// parameter injection and one-batch gradients (training diagnostics)
// ---------------------------------------------------------------------------
extern "C" GTMP_API gtmp_status gtmp_surrogate_set_params(gtmp_ctx* c, const float* host_params, int64_t n,
                                                          const float* host_fourier, int64_t n_fourier) {
  if (!c || !host_params || n != kParamCount || !host_fourier || n_fourier != 64 * c->dof || c->dof > kMaxDof)
    return sfail(c, GTMP_ERR_INVALID_ARG, "parameter buffer sizes must match gtmp_surrogate_param_count");
  if (!c->sur) c->sur = new SurrogateState();
  SurrogateState* s = c->sur;
  cudaStream_t st = c->stream;
  if (!s->P) {
    SUR_TRY(c, cudaMalloc(&s->P, kParamCount * sizeof(float)));
    SUR_TRY(c, cudaMalloc(&s->G, kParamCount * sizeof(float)));
    SUR_TRY(c, cudaMalloc(&s->Mm, kParamCount * sizeof(float)));
    SUR_TRY(c, cudaMalloc(&s->Vv, kParamCount * sizeof(float)));
    SUR_TRY(c, cudaMalloc(&s->W1b, kNW1 * sizeof(__nv_bfloat16)));
    SUR_TRY(c, cudaMalloc(&s->W1bT, kNW1 * sizeof(__nv_bfloat16)));
    SUR_TRY(c, cudaMalloc(&s->W2b, kNW2 * sizeof(__nv_bfloat16)));
    SUR_TRY(c, cudaMalloc(&s->W2bT, kNW2 * sizeof(__nv_bfloat16)));
    SUR_TRY(c, cudaMalloc(&s->W3b, kNW3 * sizeof(__nv_bfloat16)));
    SUR_TRY(c, cudaMalloc(&s->W3bT, kNW3 * sizeof(__nv_bfloat16)));
    SUR_TRY(c, cudaMalloc(&s->loss, sizeof(double)));
    SUR_TRY(c, cudaMalloc(&s->counter, sizeof(unsigned long long)));
  }
  s->dof = c->dof;
  s->four.dof = c->dof;
  for (int k = 0; k < 64 * c->dof; ++k) s->four.B[k] = host_fourier[k];
  SUR_TRY(c, cudaMemcpyAsync(s->P, host_params, kParamCount * sizeof(float), cudaMemcpyHostToDevice, st));
  f32_to_bf16_kernel<<<nblk(kNW1, 256), 256, 0, st>>>(pW1(s, s->P), kHid, kFeat, s->W1b, s->W1bT);
  f32_to_bf16_kernel<<<nblk(kNW2, 256), 256, 0, st>>>(pW2(s, s->P), kHid, kHid, s->W2b, s->W2bT);
  f32_to_bf16_kernel<<<nblk(kNW3, 256), 256, 0, st>>>(pW3(s, s->P), kHid, kHid, s->W3b, s->W3bT);
  SUR_TRY(c, cudaGetLastError());
  SUR_TRY(c, cudaStreamSynchronize(st));
  s->trained = true;
  return GTMP_OK;
}

extern "C" GTMP_API gtmp_status gtmp_surrogate_loss_grad(gtmp_ctx* c, const float* dev_q, const uint8_t* dev_labels,
                                                         int32_t n, double* host_loss, float* host_grad,
                                                         int64_t n_grad) {
  if (!c || !dev_q || !dev_labels || n < 64 || n % 64 != 0 || n > (1 << 16) || !host_loss || !host_grad ||
      n_grad != kParamCount)
    return sfail(c, GTMP_ERR_INVALID_ARG, "bad gradient request (n a multiple of 64, at most 65536)");
  if (!c->sur || !c->sur->trained) return sfail(c, GTMP_ERR_NOT_READY, "surrogate has no parameters");
  SurrogateState* s = c->sur;
  cudaStream_t st = c->stream;
  SUR_TRY(c, ensure_buffers(s, n));
  SUR_TRY(c, cudaMemsetAsync(s->loss, 0, sizeof(double), st));
  features_kernel<<<nblk(n, 128), 128, 0, st>>>(dev_q, n, s->four, s->X, s->XT, n);
  SUR_TRY(c, cudaGetLastError());
  SUR_TRY(c, batch_gradients(s, s->X, s->XT, n, dev_labels, n, c->err, st));
  SUR_TRY(c, cudaMemcpyAsync(host_grad, s->G, kParamCount * sizeof(float), cudaMemcpyDeviceToHost, st));
  SUR_TRY(c, cudaMemcpyAsync(host_loss, s->loss, sizeof(double), cudaMemcpyDeviceToHost, st));
  SUR_TRY(c, cudaStreamSynchronize(st));
  *host_loss /= n;
  return GTMP_OK;
}
