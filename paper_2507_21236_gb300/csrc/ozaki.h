// FP64-accurate GEMM from exact BF16 slice products on the tensor cores (internal).
#pragma once

#include <cuda_bf16.h>

#include "attn_internal.h"

namespace attn {

// A strided FP64 operand seen as [batches][rows][K'] with K' = G K: entry
// (bh, bl, r, g K + k) at p + bh sBhi + bl sBlo + r sR + g sG + k sK.
struct OzView {
  const double* p = nullptr;
  long sR = 0, sK = 0, sG = 0, sBhi = 0, sBlo = 0;
  int rows = 0, K = 0, G = 1;
  int nbhi = 1, nblo = 1;  // distinct batch entries of this operand
};

// Row exponents E (|entry| < 2^E per row; -2000 for a zero row) and six BF16 slices
// of 2^-E times each row (Kpad >= K G, a multiple of 64), stored tiled: per batch entry,
// tile of tile_rows rows and 64-wide K block, the six [tile_rows][64] slice blocks.
void ozaki_slice(attn_ctx* ctx, const OzView& v, long Kpad, int tile_rows, DevBuf& slices, DevBuf& exps);

// The GemmF64 contraction C = alpha sum_g A_g B_g + beta C, computed from the
// slices' exact BF16 products (normwise error about (K + 2) 2^-46 of the row scales).
void gemm_f64_ozaki(attn_ctx* ctx, const GemmF64& g);

// Read and clear the split GEMM's device error word (0 = ok).
int ozaki_error(attn_ctx* ctx);

}  // namespace attn
