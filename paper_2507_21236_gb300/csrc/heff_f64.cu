// H_eff x in FP64 on the CUDA cores (Sec. 3.3.2 last paragraph; Sec. 4.4.2).
//
// y = sum_l H_l x_l x + sum_kinds sum_r A_r x_p B_r x_q x + sum_r (O0 (x) O1 (x) O2)_r x
//
// Each product group is two (three for triples) strided GEMM stages: stage 1
// applies the second operator of every product of a chunk to x, writing one
// intermediate per product; stage 2 is a single GEMM whose reduction runs over
// (product, link index), accumulating straight into y.
#include <algorithm>

#include "heff.h"

using namespace attn;

double attn_heff::flops() const {
  double f = 0.0;
  for (int s = 0; s < 3; ++s)
    if (has_hint[s]) f += 2.0 * m[s] * V;
  for (int k = 0; k < 3; ++k) f += (double)npair[k] * 2.0 * (m[kPairP[k]] + m[kPairQ[k]]) * V;
  f += (double)ntrip * 2.0 * (m[0] + m[1] + m[2]) * V;
  return f;
}

attn_heff::~attn_heff() {
  delete eg;
  attn::tc_release(this);
}

namespace attn {

// y += sum_{r<R} A_r x_p W_r with W_r = per-product tensors (stride V).
void accumulate_slot_f64(attn_ctx* ctx, const int d[3], int p, const double* A, int R, const double* W, double* y) {
  const long V = (long)d[0] * d[1] * d[2];
  GemmF64 g;
  g.split_ok = true;
  g.beta = 1.0;
  g.G = R;
  if (p == 0) {
    g.M = d[0]; g.N = d[1] * d[2]; g.K = d[0];
    g.A = A; g.aM = d[0]; g.aK = 1; g.aG = (long)d[0] * d[0];
    g.B = W; g.bK = (long)d[1] * d[2]; g.bN = 1; g.bG = V;
    g.C = y; g.cM = (long)d[1] * d[2]; g.cN = 1;
  } else if (p == 1) {
    g.M = d[1]; g.N = d[2]; g.K = d[1];
    g.A = A; g.aM = d[1]; g.aK = 1; g.aG = (long)d[1] * d[1];
    g.B = W; g.bK = d[2]; g.bN = 1; g.bG = V; g.bBlo = (long)d[1] * d[2];
    g.C = y; g.cM = d[2]; g.cN = 1; g.cBlo = (long)d[1] * d[2];
    g.Blo = d[0];
  } else {
    g.M = d[0] * d[1]; g.N = d[2]; g.K = d[2];
    g.A = W; g.aM = d[2]; g.aK = 1; g.aG = V;
    g.B = A; g.bK = 1; g.bN = d[2]; g.bG = (long)d[2] * d[2];
    g.C = y; g.cM = d[2]; g.cN = 1;
  }
  gemm_f64(ctx, g);
}

}  // namespace attn

void attn_heff::apply_f64(const double* x, double* y) {
  const int d[3] = {m[0], m[1], m[2]};
  fill_f64(ctx, y, (size_t)V, 0.0);
  for (int s = 0; s < 3; ++s)
    if (has_hint[s]) mode_product_f64(ctx, d, s, hint[s].as<double>(), 1, x, 0, y, 1.0);
  // chunk so that the intermediates stay below ~1 GiB
  const long budget = 1L << 27;  // doubles
  const int chunk = (int)std::max<long>(1, std::min<long>(4096, budget / std::max<long>(V, 1)));
  for (int k = 0; k < 3; ++k) {
    const int p = kPairP[k], q = kPairQ[k];
    for (int r0 = 0; r0 < npair[k]; r0 += chunk) {
      const int R = std::min(chunk, npair[k] - r0);
      ctx->ws[0].reserve(sizeof(double) * (size_t)R * V);
      double* W = ctx->ws[0].as<double>();
      mode_product_f64(ctx, d, q, pb[k].as<double>() + (long)r0 * m[q] * m[q], R, x, 0, W, 0.0);
      accumulate_slot_f64(ctx, d, p, pa[k].as<double>() + (long)r0 * m[p] * m[p], R, W, y);
    }
  }
  for (int r0 = 0; r0 < ntrip; r0 += chunk) {
    const int R = std::min(chunk, ntrip - r0);
    ctx->ws[0].reserve(sizeof(double) * (size_t)R * V);
    ctx->ws[1].reserve(sizeof(double) * (size_t)R * V);
    double* W1 = ctx->ws[0].as<double>();
    double* W2 = ctx->ws[1].as<double>();
    mode_product_f64(ctx, d, 2, tr[2].as<double>() + (long)r0 * m[2] * m[2], R, x, 0, W1, 0.0);
    mode_product_f64(ctx, d, 1, tr[1].as<double>() + (long)r0 * m[1] * m[1], R, W1, V, W2, 0.0);
    accumulate_slot_f64(ctx, d, 0, tr[0].as<double>() + (long)r0 * m[0] * m[0], R, W2, y);
  }
}
