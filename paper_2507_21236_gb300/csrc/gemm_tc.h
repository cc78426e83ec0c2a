// Batched BF16 tensor-core GEMM C = alpha A B^T (both K-major), internal.
#pragma once

#include <cuda_bf16.h>

#include "attn_internal.h"

namespace attn {

// A K-major BF16 operand viewed as [batches][rows][K] with row stride ld and
// batch stride bstride (elements; both multiples of 8, base 16-byte aligned).
struct TnOperand {
  const __nv_bfloat16* p = nullptr;
  int K = 0, rows = 0, batches = 1;
  long ld = 0, bstride = 0;
};

struct TnParams {
  int M = 0, N = 0, K = 0;
  int Bhi = 1, Blo = 1;                 // batch entries b = bhi * Blo + blo
  int a_bhi = 0, a_blo = 0;             // batch coordinate of A = bhi * a_bhi + blo * a_blo
  int b_bhi = 0, b_blo = 0;
  void* C = nullptr;
  int c_type = 0;                       // 0 FP32, 1 BF16, 2 FP64
  long c_rs = 0, c_cs = 1, c_bhi = 0, c_blo = 0;  // element strides of C
  float alpha = 1.0f;
  int accumulate = 0;                   // C += alpha * AB^T instead of C = ...
  long batch_offset = 0;                // set by the launcher
  int* err = nullptr;                   // set by the launcher
};

void tn_gemm_bf16(attn_ctx* ctx, const TnOperand& A, const TnOperand& B, TnParams p, DevBuf& err);

}  // namespace attn
