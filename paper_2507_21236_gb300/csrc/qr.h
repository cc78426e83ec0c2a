// FP64 QR and tensor<->column-matrix permutations (internal).
#pragma once

#include "attn_internal.h"

namespace attn {

struct QRWork {
  DevBuf part, part2, nrm0, defic;
};

// In-place QR of the column-stored matrix At[k][M] (column j contiguous):
// on return At holds Q's columns and R (k x k, row-major, device) the
// upper-triangular factor with diag(R) >= 0.
void qr_columns(attn_ctx* ctx, double* At, long M, int k, double* R, QRWork& w);

// At[j][row] = T with the `slot` index as column j, the other two (in order) as row.
void tensor_to_columns(attn_ctx* ctx, const double* T, const int d[3], int slot, double* At);
void columns_to_tensor(attn_ctx* ctx, const double* At, const int d[3], int slot, double* T);

}  // namespace attn
