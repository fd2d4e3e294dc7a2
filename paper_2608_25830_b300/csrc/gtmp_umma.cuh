// Fifth-generation tensor cores (tcgen05) for the collision surrogate: a
// BF16 x BF16 -> FP32 GEMM with the accumulator in tensor memory (TMEM).
//
//   C[m][n] = sum_k A[m][k] * B[n][k]        (A: M x K, B: N x K, both with K
//                                             contiguous in global memory)
//
// One CTA (4 warps) owns a 128 x BN tile of C.  Operand tiles of 64 K-columns
// are copied with cp.async straight into the canonical no-swizzle K-major
// layout of the UMMA shared-memory descriptor (core matrices of 8 rows x 16
// bytes: element (r, k) of a tile at ((r/8)*8 + k/8)*128 + (r%8)*16 + (k%8)*2
// bytes), double-buffered; one elected thread issues four
// tcgen05.mma.cta_group::1.kind::f16 (K = 16 each) per tile and commits them
// to an mbarrier; the epilogue reads the accumulator rows with tcgen05.ld
// (warp w owns TMEM lanes 32w..32w+31 = tile rows) and applies one of the
// epilogues below.  Every mbarrier wait is bounded; on timeout the kernel
// sets the error word, waits (bounded) for its MMAs and frees its TMEM.
#pragma once

#include <cuda_bf16.h>
#include <cstdint>

namespace gtmp {

enum UmmaEpilogue {
  kEpiBiasReluBf16 = 0,  // out = bf16(relu(acc + bias[n])), optional transposed copy
  kEpiF32 = 1,           // outf = acc (fp32)
  kEpiMaskBf16 = 2,      // out = bf16(acc * (mask[m][n] > 0)), optional transposed copy
  kEpiHead = 3,          // h = relu(acc + bias[n]); logit[m] = sum_n h[n] w4[n] + b4;
                         // optional bf16 h and transposed copy (training)
};

struct UmmaArgs {
  const __nv_bfloat16* A;
  int lda;  // elements between rows of A
  const __nv_bfloat16* B;
  int ldb;
  int M, N, K;
  // epilogue
  const float* bias;            // [N]
  __nv_bfloat16* out;           // [M][ldo]
  int ldo;
  __nv_bfloat16* outT;          // [N][ldoT] or null
  int ldoT;
  float* outf;                  // [M][ldf]
  int ldf;
  const __nv_bfloat16* mask;    // [M][ldm]
  int ldm;
  const float* w4;              // head weights [N]
  const float* b4;              // head bias [1] (device)
  float* logits;                // [M]
  int* err;
};

constexpr int kUmmaBM = 128;
constexpr int kUmmaBK = 64;
constexpr int kUmmaThreads = 128;

}  // namespace gtmp
