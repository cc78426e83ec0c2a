// Batched tensor-core GEMM C = alpha A B^T (both K-major, BF16 or TF32 operands), internal.
#pragma once

#include <cuda_bf16.h>

#include "attn_internal.h"

namespace attn {

// A K-major operand viewed as [batches][rows][K] with row stride ld and batch stride
// bstride (elements; 16-byte multiples, base 16-byte aligned): BF16, or FP32 values
// rounded to TF32 when tf is set.
struct TnOperand {
  const void* p = nullptr;
  bool tf = false;
  int K = 0, rows = 0, batches = 1;
  long ld = 0, bstride = 0;
};

struct TnParams {
  int M = 0, N = 0, K = 0;
  int Bhi = 1, Blo = 1;                 // batch entries b = bhi * Blo + blo
  int a_bhi = 0, a_blo = 0;             // batch coordinate of A = bhi * a_bhi + blo * a_blo
  int b_bhi = 0, b_blo = 0;
  void* C = nullptr;
  int c_type = 0;                       // 0 FP32, 1 BF16, 2 FP64, 3 FP32 rounded to TF32
  long c_rs = 0, c_cs = 1, c_bhi = 0, c_blo = 0;  // element strides of C
  float alpha = 1.0f;
  int accumulate = 0;                   // C += alpha * AB^T instead of C = ...
  long batch_offset = 0;                // set by the launcher
  int* err = nullptr;                   // set by the launcher
};

// A and B must have the same operand type.
void tn_gemm(attn_ctx* ctx, const TnOperand& A, const TnOperand& B, TnParams p, DevBuf& err);

}  // namespace attn
