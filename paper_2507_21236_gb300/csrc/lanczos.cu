// Lanczos local eigensolver in FP64 on the GPU (Sec. 4.4.2: the local
// eigenproblem is solved with Lanczos; the matrix-vector product is H_eff).
//
// Krylov recurrence from the current centre tensor, full reorthogonalisation
// (classical Gram-Schmidt against the whole basis, twice), and the lowest
// eigenpair of the tridiagonal projection computed on the device: bisection
// with Sturm counts for the eigenvalue, inverse iteration (tridiagonal
// Gaussian elimination with partial pivoting) for the eigenvector. Stops when
// the Ritz residual beta_k |y_k| < tol |theta|, on breakdown, or at `depth`.
#include <algorithm>
#include <cmath>

#include "attn_internal.h"
#include "lanczos.h"

namespace attn {

namespace {

constexpr int LT = 256;
constexpr int LB = 512;  // blocks for the vector reductions

__device__ __forceinline__ double warp_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

// part[b][i] = partial of <basis_i, w> over block b's grid-stride elements.
__global__ void multi_dot_partial(const double* basis, int nvec, long V, const double* w, double* part) {
  __shared__ double sh[LT / 32];
  for (int i = 0; i < nvec; ++i) {
    const double* v = basis + (long)i * V;
    double s = 0.0;
    for (long e = blockIdx.x * (long)LT + threadIdx.x; e < V; e += (long)gridDim.x * LT) s = fma(v[e], w[e], s);
    s = warp_sum(s);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
      double t = 0;
      for (int k = 0; k < LT / 32; ++k) t += sh[k];
      part[(long)blockIdx.x * nvec + i] = t;
    }
    __syncthreads();
  }
}

// out[i] = sum_b part[b][i] (fixed order); optionally out2[i] += out[i].
__global__ void multi_dot_reduce(const double* part, int nb, int nvec, double* out, double* accum) {
  int i = blockIdx.x;
  __shared__ double sh[LT / 32];
  double s = 0.0;
  for (int b = threadIdx.x; b < nb; b += LT) s += part[(long)b * nvec + i];
  s = warp_sum(s);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0;
    for (int k = 0; k < LT / 32; ++k) t += sh[k];
    out[i] = t;
    if (accum) accum[i] += t;
  }
}

// w -= sum_i coef[i] * basis_i
__global__ void multi_axpy(double* w, const double* basis, const double* coef, int nvec, long V, double sign) {
  for (long e = blockIdx.x * (long)LT + threadIdx.x; e < V; e += (long)gridDim.x * LT) {
    double v = w[e];
    for (int i = 0; i < nvec; ++i) v = fma(-sign * coef[i], basis[(long)i * V + e], v);
    w[e] = v;
  }
}

// out = sum_i coef[i] * basis_i
__global__ void combine(double* out, const double* basis, const double* coef, int nvec, long V) {
  for (long e = blockIdx.x * (long)LT + threadIdx.x; e < V; e += (long)gridDim.x * LT) {
    double v = 0.0;
    for (int i = 0; i < nvec; ++i) v = fma(coef[i], basis[(long)i * V + e], v);
    out[e] = v;
  }
}

// dst = src * (1 / *nrm) where *nrm is a device norm (sqrt applied here if squared)
__global__ void scale_by_norm(double* dst, const double* src, const double* nrm_sq, long V) {
  double n = sqrt(*nrm_sq);
  double inv = n > 0.0 ? 1.0 / n : 0.0;
  for (long e = blockIdx.x * (long)LT + threadIdx.x; e < V; e += (long)gridDim.x * LT) dst[e] = src[e] * inv;
}

// Number of eigenvalues of the tridiagonal (a, b) smaller than x.
__device__ int sturm_count(const double* a, const double* b, int n, double x) {
  int c = 0;
  double d = 1.0;
  for (int i = 0; i < n; ++i) {
    double bb = (i > 0) ? b[i - 1] * b[i - 1] : 0.0;
    d = (a[i] - x) - (i > 0 ? bb / d : 0.0);
    if (d == 0.0) d = -1e-300;
    if (d < 0.0) ++c;
  }
  return c;
}

// Lowest eigenpair of the n x n symmetric tridiagonal (alpha, beta) -> theta, y, resid = beta_n |y_{n-1}|.
__global__ void tridiag_lowest(const double* alpha, const double* beta, int n, double beta_next, double* out) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  // out layout: [0] theta, [1] resid, [2 .. 2+n) y
  double lo = 1e300, hi = -1e300;
  for (int i = 0; i < n; ++i) {
    double r = (i > 0 ? fabs(beta[i - 1]) : 0.0) + (i < n - 1 ? fabs(beta[i]) : 0.0);
    lo = fmin(lo, alpha[i] - r);
    hi = fmax(hi, alpha[i] + r);
  }
  for (int it = 0; it < 200; ++it) {
    double mid = 0.5 * (lo + hi);
    if (mid <= lo || mid >= hi) break;
    if (sturm_count(alpha, beta, n, mid) >= 1) hi = mid; else lo = mid;
  }
  const double theta = 0.5 * (lo + hi);
  // inverse iteration with partial pivoting (up to n = 64)
  double y[64], z[64];
  double dl[64], dd[64], du[64], du2[64];
  int piv[64];
  for (int i = 0; i < n; ++i) y[i] = 1.0 / sqrt((double)n);
  const double scale = fmax(fabs(lo), fabs(hi)) + 1e-300;
  for (int iter = 0; iter < 4; ++iter) {
    for (int i = 0; i < n; ++i) {
      dd[i] = alpha[i] - theta;
      du[i] = (i < n - 1) ? beta[i] : 0.0;
      dl[i] = (i < n - 1) ? beta[i] : 0.0;
      du2[i] = 0.0;
      z[i] = y[i];
    }
    // factor (LAPACK-style gttrf without the library): rows i and i+1
    for (int i = 0; i < n - 1; ++i) {
      if (fabs(dd[i]) >= fabs(dl[i])) {
        piv[i] = 0;
        double pv = dd[i] == 0.0 ? 1e-300 * scale : dd[i];
        dd[i] = pv;
        double f = dl[i] / pv;
        dl[i] = f;
        dd[i + 1] -= f * du[i];
      } else {
        piv[i] = 1;
        double f = dd[i] / dl[i];
        dd[i] = dl[i];
        dl[i] = f;
        double t = du[i];
        du[i] = dd[i + 1];
        dd[i + 1] = t - f * dd[i + 1];
        if (i < n - 2) {
          du2[i] = du[i + 1];
          du[i + 1] = -f * du[i + 1];
        }
      }
    }
    if (dd[n - 1] == 0.0) dd[n - 1] = 1e-300 * scale;
    if (fabs(dd[n - 1]) < 1e-18 * scale) dd[n - 1] = (dd[n - 1] < 0 ? -1.0 : 1.0) * 1e-18 * scale;
    // solve L U z = y (apply row swaps while eliminating)
    for (int i = 0; i < n - 1; ++i) {
      if (piv[i] == 0) {
        z[i + 1] -= dl[i] * z[i];
      } else {
        double t = z[i];
        z[i] = z[i + 1];
        z[i + 1] = t - dl[i] * z[i];
      }
    }
    z[n - 1] /= dd[n - 1];
    if (n > 1) z[n - 2] = (z[n - 2] - du[n - 2] * z[n - 1]) / dd[n - 2];
    for (int i = n - 3; i >= 0; --i) z[i] = (z[i] - du[i] * z[i + 1] - du2[i] * z[i + 2]) / dd[i];
    double nrm = 0.0;
    for (int i = 0; i < n; ++i) nrm += z[i] * z[i];
    nrm = sqrt(nrm);
    if (!(nrm > 0.0) || !isfinite(nrm)) break;
    for (int i = 0; i < n; ++i) y[i] = z[i] / nrm;
  }
  // fix the sign: largest-magnitude component positive
  int imax = 0;
  for (int i = 1; i < n; ++i)
    if (fabs(y[i]) > fabs(y[imax])) imax = i;
  double sg = y[imax] < 0 ? -1.0 : 1.0;
  out[0] = theta;
  out[1] = fabs(beta_next * y[n - 1]);
  for (int i = 0; i < n; ++i) out[2 + i] = sg * y[i];
}

inline int vgrid(long V) { return (int)std::max<long>(1, std::min<long>((V + LT - 1) / LT, LB)); }

}  // namespace

void multi_dot(attn_ctx* ctx, const double* basis, int nvec, long V, const double* w, double* out, double* accum) {
  const int nb = vgrid(V);
  ctx->partials.reserve(sizeof(double) * (size_t)nb * std::max(nvec, 1));
  multi_dot_partial<<<nb, LT, 0, ctx->stream>>>(basis, nvec, V, w, ctx->partials.as<double>());
  multi_dot_reduce<<<nvec, LT, 0, ctx->stream>>>(ctx->partials.as<double>(), nb, nvec, out, accum);
  ctx->launches += 2;
  ATTN_CHECK_CUDA(cudaGetLastError());
}

void multi_axpy_dev(attn_ctx* ctx, double* w, const double* basis, const double* coef, int nvec, long V,
                    double sign) {
  multi_axpy<<<vgrid(V), LT, 0, ctx->stream>>>(w, basis, coef, nvec, V, sign);
  ctx->launches++;
  ATTN_CHECK_CUDA(cudaGetLastError());
}

void combine_dev(attn_ctx* ctx, double* out, const double* basis, const double* coef, int nvec, long V) {
  combine<<<vgrid(V), LT, 0, ctx->stream>>>(out, basis, coef, nvec, V);
  ctx->launches++;
  ATTN_CHECK_CUDA(cudaGetLastError());
}

void normalise_dev(attn_ctx* ctx, double* dst, const double* src, long V, double* nrm_sq_dev) {
  multi_dot(ctx, src, 1, V, src, nrm_sq_dev, nullptr);
  scale_by_norm<<<vgrid(V), LT, 0, ctx->stream>>>(dst, src, nrm_sq_dev, V);
  ctx->launches++;
  ATTN_CHECK_CUDA(cudaGetLastError());
}

LanczosResult lanczos_lowest(attn_ctx* ctx, const MatVec& apply, double* x, long V, int depth, double tol,
                             LanczosWork& w) {
  ATTN_REQUIRE(depth >= 1 && depth <= 60, ATTN_EINVAL, "Lanczos depth must be in 1..60");
  w.basis.reserve(sizeof(double) * (size_t)(depth + 1) * V);
  w.wvec.reserve(sizeof(double) * (size_t)V);
  w.scal.reserve(sizeof(double) * 512);
  double* B = w.basis.as<double>();
  double* W = w.wvec.as<double>();
  double* S = w.scal.as<double>();
  // S layout: [0..64) alpha, [64..128) beta, [128] tmp, [192..) tridiag out, [320..) h
  double* alpha = S;
  double* beta = S + 64;
  double* tmp = S + 128;
  double* tri = S + 192;
  double* h = S + 320;
  cudaStream_t s = ctx->stream;
  normalise_dev(ctx, B, x, V, tmp);
  std::vector<double> ha(depth), hb(depth);
  double host_tri[2 + 64];
  LanczosResult res{0.0, 0, 0.0, false};
  int nk = 0;
  for (int k = 0; k < depth; ++k) {
    double* vk = B + (long)k * V;
    apply(vk, W);
    multi_dot(ctx, vk, 1, V, W, alpha + k, nullptr);
    // W -= alpha_k v_k + beta_{k-1} v_{k-1}  (coefficients from device)
    multi_axpy_dev(ctx, W, vk, alpha + k, 1, V, 1.0);
    if (k > 0) multi_axpy_dev(ctx, W, B + (long)(k - 1) * V, beta + (k - 1), 1, V, 1.0);
    for (int pass = 0; pass < 2; ++pass) {
      multi_dot(ctx, B, k + 1, V, W, h, nullptr);
      multi_axpy_dev(ctx, W, B, h, k + 1, V, 1.0);
    }
    multi_dot(ctx, W, 1, V, W, tmp, nullptr);
    ATTN_CHECK_CUDA(cudaMemcpyAsync(&hb[k], tmp, sizeof(double), cudaMemcpyDeviceToHost, s));
    ATTN_CHECK_CUDA(cudaStreamSynchronize(s));
    const double b = std::sqrt(std::max(hb[k], 0.0));
    nk = k + 1;
    tridiag_lowest<<<1, 1, 0, s>>>(alpha, beta, nk, b, tri);
    ctx->launches++;
    ATTN_CHECK_CUDA(cudaMemcpyAsync(host_tri, tri, sizeof(double) * 2, cudaMemcpyDeviceToHost, s));
    ATTN_CHECK_CUDA(cudaStreamSynchronize(s));
    res.theta = host_tri[0];
    res.resid = host_tri[1];
    res.iters = nk;
    const double sc = std::max(std::fabs(res.theta), 1e-300);
    ATTN_REQUIRE(std::isfinite(res.theta) && std::isfinite(b), ATTN_ENONFINITE, "non-finite value in Lanczos");
    if (res.resid < tol * sc || b < 1e-14 * sc) {
      res.converged = true;
      break;
    }
    if (k == depth - 1) break;
    // beta_k and v_{k+1} = W / beta_k
    ATTN_CHECK_CUDA(cudaMemcpyAsync(beta + k, &b, sizeof(double), cudaMemcpyHostToDevice, s));
    scale_by_norm<<<vgrid(V), LT, 0, s>>>(B + (long)(k + 1) * V, W, tmp, V);
    ctx->launches++;
  }
  // Ritz vector x = sum_i y_i v_i, normalised
  combine_dev(ctx, W, B, tri + 2, nk, V);
  normalise_dev(ctx, x, W, V, tmp);
  ATTN_CHECK_CUDA(cudaGetLastError());
  return res;
}

}  // namespace attn
