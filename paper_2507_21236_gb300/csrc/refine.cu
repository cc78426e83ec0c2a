// Mixed-precision refinement of the lowest eigenpair of the local eigenproblem
// (Sec. 4.4.2) after a low-precision Lanczos solve.
//
// Outer loop in FP64: Rayleigh-Ritz on an orthonormal subspace V (starting from
// the low-precision Ritz vector), with W = H V computed by FP64 matvecs, one
// per new basis vector; Ritz pair (theta, u), residual r = H u - theta u, all
// from exact FP64 data. Each correction t approximately solves the
// Jacobi-Davidson equation
//     (I - u u^T)(H - theta)(I - u u^T) t = -r,   t _|_ u
// by conjugate gradients whose matvecs use the low-precision H_eff: their
// errors are relative to |t|, which shrinks with |r|, so every outer step gains
// the low-precision accuracy again (iterative refinement). With inner = 0 the
// correction is r itself, and k outer steps are the k FP64 residual-correction
// steps (a Rayleigh-Ritz on span{v, r, ...}). Stops when ||r|| < tol |theta| or
// when a correction lowers theta by no more than tol |theta|.
#include <algorithm>
#include <cmath>
#include <vector>

#include "attn_internal.h"
#include "lanczos.h"

namespace attn {

namespace {

constexpr int RT = 256;
// device scalar slots
constexpr int C_PQ = 0, C_RR = 1, C_RRN = 2, C_BETA = 3, C_STOP = 4, C_UQ = 5, C_THETA = 6, C_Y = 16, C_SIZE = 64;

int rgrid(long V) { return (int)std::max<long>(1, std::min<long>((V + RT - 1) / RT, 1024)); }

// q -= theta p
__global__ void shift_kernel(double* q, const double* p, const double* theta, long V) {
  const double th = *theta;
  for (long e = blockIdx.x * (long)RT + threadIdx.x; e < V; e += (long)gridDim.x * RT) q[e] = fma(-th, p[e], q[e]);
}

// alpha = rr / pq (0 once stopped or when the operator is not positive on p); t += alpha p, res -= alpha q
__global__ void cg_update(double* t, double* res, const double* p, const double* q, const double* C, long V) {
  const double pq = C[C_PQ], rr = C[C_RR];
  const double a = (C[C_STOP] != 0.0 || !(pq > 0.0)) ? 0.0 : rr / pq;
  if (a == 0.0) return;
  for (long e = blockIdx.x * (long)RT + threadIdx.x; e < V; e += (long)gridDim.x * RT) {
    t[e] = fma(a, p[e], t[e]);
    res[e] = fma(-a, q[e], res[e]);
  }
}

// beta = rr_new / rr; stop when the operator lost positivity or the residual vanished
__global__ void cg_scalars(double* C) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  if (C[C_STOP] != 0.0) return;
  if (!(C[C_PQ] > 0.0) || !(C[C_RR] > 0.0)) {
    C[C_STOP] = 1.0;
    return;
  }
  C[C_BETA] = C[C_RRN] / C[C_RR];
  C[C_RR] = C[C_RRN];
  if (!(C[C_RRN] > 0.0)) C[C_STOP] = 1.0;
}

// p = res + beta p (skipped once stopped)
__global__ void cg_direction(double* p, const double* res, const double* C, long V) {
  if (C[C_STOP] != 0.0) return;
  const double b = C[C_BETA];
  for (long e = blockIdx.x * (long)RT + threadIdx.x; e < V; e += (long)gridDim.x * RT) p[e] = fma(b, p[e], res[e]);
}

// r = hu - theta u
__global__ void resid_kernel(double* r, const double* hu, const double* u, const double* theta, long V) {
  const double th = *theta;
  for (long e = blockIdx.x * (long)RT + threadIdx.x; e < V; e += (long)gridDim.x * RT) r[e] = fma(-th, u[e], hu[e]);
}

// out = -in
__global__ void neg_kernel(double* out, const double* in, long V) {
  for (long e = blockIdx.x * (long)RT + threadIdx.x; e < V; e += (long)gridDim.x * RT) out[e] = -in[e];
}

// Lowest eigenpair of a small dense symmetric matrix (cyclic Jacobi, host).
void small_lowest(std::vector<double> a, int n, double& theta, std::vector<double>& y) {
  std::vector<double> v((size_t)n * n, 0.0);
  for (int i = 0; i < n; ++i) v[(size_t)i * n + i] = 1.0;
  for (int sweep = 0; sweep < 60; ++sweep) {
    double off = 0.0;
    for (int i = 0; i < n; ++i)
      for (int j = i + 1; j < n; ++j) off += a[(size_t)i * n + j] * a[(size_t)i * n + j];
    if (off < 1e-300) break;
    for (int p = 0; p < n; ++p)
      for (int q = p + 1; q < n; ++q) {
        const double apq = a[(size_t)p * n + q];
        if (std::fabs(apq) < 1e-300) continue;
        const double tau = (a[(size_t)q * n + q] - a[(size_t)p * n + p]) / (2.0 * apq);
        const double t = (tau >= 0 ? 1.0 : -1.0) / (std::fabs(tau) + std::sqrt(1.0 + tau * tau));
        const double c = 1.0 / std::sqrt(1.0 + t * t), s = t * c;
        for (int k = 0; k < n; ++k) {
          const double akp = a[(size_t)k * n + p], akq = a[(size_t)k * n + q];
          a[(size_t)k * n + p] = c * akp - s * akq;
          a[(size_t)k * n + q] = s * akp + c * akq;
        }
        for (int k = 0; k < n; ++k) {
          const double apk = a[(size_t)p * n + k], aqk = a[(size_t)q * n + k];
          a[(size_t)p * n + k] = c * apk - s * aqk;
          a[(size_t)q * n + k] = s * apk + c * aqk;
        }
        for (int k = 0; k < n; ++k) {
          const double vkp = v[(size_t)k * n + p], vkq = v[(size_t)k * n + q];
          v[(size_t)k * n + p] = c * vkp - s * vkq;
          v[(size_t)k * n + q] = s * vkp + c * vkq;
        }
      }
  }
  int imin = 0;
  for (int i = 1; i < n; ++i)
    if (a[(size_t)i * n + i] < a[(size_t)imin * n + imin]) imin = i;
  theta = a[(size_t)imin * n + imin];
  y.assign(n, 0.0);
  for (int k = 0; k < n; ++k) y[k] = v[(size_t)k * n + imin];
}

}  // namespace

RefineResult refine_eig(attn_ctx* ctx, const MatVec& h64, const MatVec& hlo, double* x, long V, int max_outer,
                        int inner, double tol, RefineWork& w) {
  ATTN_REQUIRE(max_outer >= 1 && max_outer <= 32, ATTN_EINVAL, "refinement steps must be in 1..32");
  const int kmax = max_outer + 1;
  cudaStream_t s = ctx->stream;
  w.Vb.reserve(sizeof(double) * (size_t)kmax * V);
  w.Wb.reserve(sizeof(double) * (size_t)kmax * V);
  for (DevBuf* b : {&w.u, &w.hu, &w.r, &w.t, &w.res, &w.p, &w.q}) b->reserve(sizeof(double) * V);
  w.C.reserve(sizeof(double) * (C_SIZE + (size_t)kmax * kmax));
  double* Vb = w.Vb.as<double>();
  double* Wb = w.Wb.as<double>();
  double* C = w.C.as<double>();
  double* G = C + C_SIZE;  // column j of V^T W at G + j * kmax
  RefineResult out{0.0, 0.0, 0, 0, 0, false};

  // V_0 = x / |x|, W_0 = H V_0
  normalise_dev(ctx, Vb, x, V, C + C_RRN);
  h64(Vb, Wb);
  out.fp64_matvecs = 1;
  std::vector<double> g((size_t)kmax * kmax, 0.0), y;
  double theta = 0.0;
  for (int k = 1;; ++k) {
    // new column of the projected matrix, then the Ritz pair on the host
    multi_dot(ctx, Vb, k, V, Wb + (long)(k - 1) * V, G + (long)(k - 1) * kmax, nullptr);
    std::vector<double> col(k);
    ATTN_CHECK_CUDA(cudaMemcpyAsync(col.data(), G + (long)(k - 1) * kmax, sizeof(double) * k, cudaMemcpyDeviceToHost, s));
    ATTN_CHECK_CUDA(cudaStreamSynchronize(s));
    for (int i = 0; i < k; ++i) {
      ATTN_REQUIRE(std::isfinite(col[i]), ATTN_ENONFINITE, "non-finite value in the refinement");
      g[(size_t)i * kmax + (k - 1)] = g[(size_t)(k - 1) * kmax + i] = col[i];
    }
    std::vector<double> a((size_t)k * k);
    for (int i = 0; i < k; ++i)
      for (int j = 0; j < k; ++j) a[(size_t)i * k + j] = g[(size_t)i * kmax + j];
    small_lowest(a, k, theta, y);
    double hy[40];
    hy[0] = theta;
    for (int i = 0; i < k; ++i) hy[1 + i] = y[i];
    ATTN_CHECK_CUDA(cudaMemcpyAsync(C + C_THETA, hy, sizeof(double), cudaMemcpyHostToDevice, s));
    ATTN_CHECK_CUDA(cudaMemcpyAsync(C + C_Y, hy + 1, sizeof(double) * k, cudaMemcpyHostToDevice, s));
    // u = V y, Hu = W y, r = Hu - theta u
    combine_dev(ctx, w.u.as<double>(), Vb, C + C_Y, k, V);
    combine_dev(ctx, w.hu.as<double>(), Wb, C + C_Y, k, V);
    resid_kernel<<<rgrid(V), RT, 0, s>>>(w.r.as<double>(), w.hu.as<double>(), w.u.as<double>(), C + C_THETA, V);
    ctx->launches++;
    multi_dot(ctx, w.r.as<double>(), 1, V, w.r.as<double>(), C + C_RRN, nullptr);
    double rr = 0.0;
    ATTN_CHECK_CUDA(cudaMemcpyAsync(&rr, C + C_RRN, sizeof(double), cudaMemcpyDeviceToHost, s));
    ATTN_CHECK_CUDA(cudaStreamSynchronize(s));
    const double scale = std::max(std::fabs(theta), 1e-300);
    // Rayleigh-Ritz on nested subspaces never raises theta; a correction that lowers it
    // by at most tol |theta| leaves an eigenvalue error of that order (the residual
    // bound is much stricter: the eigenvalue error goes as ||r||^2 / gap)
    const bool settled = k > 1 && out.theta - theta <= tol * scale;
    out.theta = theta;
    out.resid = std::sqrt(std::max(rr, 0.0));
    out.outer = k - 1;
    if (out.resid < tol * scale || settled) {
      out.converged = true;
      break;
    }
    if (k == kmax) break;
    // correction t
    double* t = w.t.as<double>();
    if (inner <= 0) {
      copy_f64(ctx, t, w.r.as<double>(), V);
    } else {
      double* res = w.res.as<double>();
      double* p = w.p.as<double>();
      double* q = w.q.as<double>();
      const double* u = w.u.as<double>();
      fill_f64(ctx, t, V, 0.0);
      neg_kernel<<<rgrid(V), RT, 0, s>>>(res, w.r.as<double>(), V);
      copy_f64(ctx, p, res, V);
      ctx->launches++;
      ATTN_CHECK_CUDA(cudaMemsetAsync(C + C_STOP, 0, sizeof(double), s));
      ATTN_CHECK_CUDA(cudaMemcpyAsync(C + C_RR, &rr, sizeof(double), cudaMemcpyHostToDevice, s));
      for (int it = 0; it < inner; ++it) {
        // q = P (H_lo - theta) p: p stays orthogonal to u, so only the output is projected
        hlo(p, q);
        shift_kernel<<<rgrid(V), RT, 0, s>>>(q, p, C + C_THETA, V);
        multi_dot(ctx, u, 1, V, q, C + C_UQ, nullptr);
        multi_axpy_dev(ctx, q, u, C + C_UQ, 1, V, 1.0);
        multi_dot(ctx, p, 1, V, q, C + C_PQ, nullptr);
        cg_update<<<rgrid(V), RT, 0, s>>>(t, res, p, q, C, V);
        multi_dot(ctx, res, 1, V, res, C + C_RRN, nullptr);
        cg_scalars<<<1, 1, 0, s>>>(C);
        cg_direction<<<rgrid(V), RT, 0, s>>>(p, res, C, V);
        ctx->launches += 4;
      }
      out.lo_matvecs += inner;
    }
    // V_k = t orthonormalised against V (twice), W_k = H V_k
    double* vk = Vb + (long)k * V;
    multi_dot(ctx, Vb, k, V, t, C + C_Y, nullptr);
    multi_axpy_dev(ctx, t, Vb, C + C_Y, k, V, 1.0);
    multi_dot(ctx, Vb, k, V, t, C + C_Y, nullptr);
    multi_axpy_dev(ctx, t, Vb, C + C_Y, k, V, 1.0);
    normalise_dev(ctx, vk, t, V, C + C_RRN);
    double tn = 0.0;
    ATTN_CHECK_CUDA(cudaMemcpyAsync(&tn, C + C_RRN, sizeof(double), cudaMemcpyDeviceToHost, s));
    ATTN_CHECK_CUDA(cudaStreamSynchronize(s));
    if (!(tn > 1e-28 * std::max(rr, 1e-300))) break;  // no new direction
    h64(vk, Wb + (long)k * V);
    out.fp64_matvecs++;
  }
  copy_f64(ctx, x, w.u.as<double>(), V);
  return out;
}

}  // namespace attn
