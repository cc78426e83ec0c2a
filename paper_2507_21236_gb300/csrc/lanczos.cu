// Lanczos local eigensolver in FP64 on the GPU (Sec. 4.4.2: the local
// eigenproblem is solved with Lanczos; the matrix-vector product is H_eff).
//
// Krylov recurrence from the current centre tensor, full reorthogonalisation
// (classical Gram-Schmidt against the whole basis, twice, as three fused
// streaming passes), and the lowest
// eigenpair of the tridiagonal projection computed on the device: bisection
// with Sturm counts for the eigenvalue, inverse iteration (tridiagonal
// Gaussian elimination with partial pivoting) for the eigenvector. Stops when
// the Ritz residual beta_k |y_k| < tol |theta|, on breakdown, or at `depth`.
//
// The Krylov basis is stored block-interleaved: for every chunk of 256 elements the
// chunks of all basis vectors lie next to each other, so each Gram-Schmidt pass over
// the basis reads one contiguous stream (vectors 16.8 MB apart at m = 128 made one
// stream per vector); a contiguous copy of the newest vector feeds the matvec.
//
// The whole recurrence is device-resident: beta_k, the Ritz solve and the
// stop decision are taken by a one-thread kernel after every step and kept in
// device memory; kernels after the stop see the flag and return, and the
// final Ritz vector is assembled with the device-side basis size. The host
// enqueues a fixed sequence of launches (capturable in a CUDA graph) and reads
// the result once.
#include <algorithm>
#include <cmath>
#include <type_traits>

#include "attn_internal.h"
#include "lanczos.h"

namespace attn {

namespace {

constexpr int LT = 256;
constexpr int LB = 512;  // blocks for the vector reductions

// scalar slots in the work buffer (doubles)
constexpr int S_ALPHA = 0, S_BETA = 64, S_TMP = 128, S_DONE = 129, S_NK = 130, S_THETA = 131, S_RESID = 132,
              S_Y = 192, S_H = 320, S_H2 = 400, S_SIZE = 512;

// Element e of basis vector i: block-interleaved with capacity D (chunks of LT = 256
// elements, chunk c of vector i at (c D + i) LT), or contiguous (D = 0: vector i at i V).
__device__ __forceinline__ long bidx(int i, long e, long V, int D) {
  return D ? (((e >> 8) * D + i) << 8) + (e & 255) : (long)i * V + e;
}

__device__ __forceinline__ double warp_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}
// fused multiply-add in the operands' own precision (never promoted)
__device__ __forceinline__ double fma_t(double a, double b, double c) { return __fma_rn(a, b, c); }
__device__ __forceinline__ float fma_t(float a, float b, float c) { return __fmaf_rn(a, b, c); }

__device__ __forceinline__ float warp_sum(float v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

// part[b][i] = partial of <basis_i, w> over block b's grid-stride elements.
__global__ void multi_dot_partial(const double* basis, int nvec, long V, int D, const double* w, double* part,
                                  const double* done) {
  if (done && *done != 0.0) return;
  __shared__ double sh[LT / 32];
  for (int i = 0; i < nvec; ++i) {
    double s = 0.0;
    for (long e = blockIdx.x * (long)LT + threadIdx.x; e < V; e += (long)gridDim.x * LT)
      s = fma(basis[bidx(i, e, V, D)], w[e], s);
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

// out[i] = sum_b part[b][i] (fixed order); optionally accum[i] += out[i].
__global__ void multi_dot_reduce(const double* part, int nb, int nvec, double* out, double* accum, const double* done) {
  if (done && *done != 0.0) return;
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
__global__ void multi_axpy(double* w, const double* basis, const double* coef, int nvec, long V, int D, double sign,
                           const double* done) {
  if (done && *done != 0.0) return;
  for (long e = blockIdx.x * (long)LT + threadIdx.x; e < V; e += (long)gridDim.x * LT) {
    double v = w[e];
    for (int i = 0; i < nvec; ++i) v = fma(-sign * coef[i], basis[bidx(i, e, V, D)], v);
    w[e] = v;
  }
}

// ---- fused classical Gram-Schmidt passes (up to kFusedMax basis vectors).
// One CGS2 step as three streaming passes over the basis instead of five:
//   (A) h_i = <v_i, w>;  (B) w -= sum h_i v_i and h2_i = <v_i, w>;
//   (C) w -= sum h2_i v_i and ||w||^2.
// Each pass reads every basis vector once; block partials are summed in a fixed
// order by multi_dot_reduce, so results are deterministic. The kernels are
// instantiated for NV vectors at most with U elements per thread and step
// (fewer vectors -> more elements), so that every thread keeps NV * U loads in
// flight: a streaming pass over HBM needs about 40 KB outstanding per SM.
constexpr int kFusedMax = 24;

// Sum the per-thread values acc[0..n) over the block and write them to out[0..n).
// (warp sums in the accumulator's type, the rest in FP64)
template <int NV, class A>
__device__ __forceinline__ void block_sum_store(A (&acc)[NV], int n, double* out) {
  __shared__ double sh[LT / 32][NV];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
  for (int i = 0; i < NV; ++i) {
    if (i < n) {
      const double s = (double)warp_sum(acc[i]);
      if (lane == 0) sh[warp][i] = s;
    }
  }
  __syncthreads();
  if (threadIdx.x < n) {
    double t = 0.0;
    for (int q = 0; q < LT / 32; ++q) t += sh[q][threadIdx.x];
    out[threadIdx.x] = t;
  }
}

// The passes are instantiated for an FP64 basis and for an FP32 one (the basis of a
// Lanczos whose matvecs run in BF16 or TF32: its vectors carry no more than FP32 accuracy);
// they compute in the basis' type T, with w (FP64 storage) rounded to T on load.

// (A) part[b][i] = block b's share of <basis_i, w>
template <int NV, int U, class T>
__global__ void __launch_bounds__(LT, 2) cgs_dot(const T* __restrict__ basis, int n, long V, int D,
                                              const double* __restrict__ w, double* part, const double* done) {
  if (done && *done != 0.0) return;
  T acc[NV];
#pragma unroll
  for (int i = 0; i < NV; ++i) acc[i] = 0;
  const long stride = (long)gridDim.x * LT;
  for (long e0 = blockIdx.x * (long)LT + threadIdx.x; e0 < V; e0 += stride * U) {
    T we[U];
#pragma unroll
    for (int u = 0; u < U; ++u) we[u] = (e0 + u * stride < V) ? (T)w[e0 + u * stride] : (T)0;
#pragma unroll
    for (int i = 0; i < NV; ++i)
      if (i < n) {
#pragma unroll
        for (int u = 0; u < U; ++u)
          if (e0 + u * stride < V) acc[i] = fma_t(basis[bidx(i, e0 + u * stride, V, D)], we[u], acc[i]);
      }
  }
  block_sum_store<NV>(acc, n, part + (long)blockIdx.x * n);
}

// (B) w -= sum_i h_i basis_i, then part[b][i] = block share of <basis_i, w_new>
template <int NV, int U, class T>
__global__ void __launch_bounds__(LT, 2) cgs_axpy_dot(double* __restrict__ w, const T* __restrict__ basis,
                                                   const double* h, int n, long V, int D, double* part,
                                                   const double* done) {
  if (done && *done != 0.0) return;
  __shared__ T c[NV];
  if (threadIdx.x < NV) c[threadIdx.x] = threadIdx.x < n ? (T)h[threadIdx.x] : (T)0;
  __syncthreads();
  T acc[NV];
#pragma unroll
  for (int i = 0; i < NV; ++i) acc[i] = 0;
  const long stride = (long)gridDim.x * LT;
  if constexpr (NV == 16 || NV == 20) {
    // wide bases: each thread parks the basis elements it loads for the update of w in
    // its own column of shared memory and reads them back for the dot products, so that
    // only the accumulators stay in registers and two blocks fit on an SM
    static_assert(U == 1, "the shared-memory form handles one element per thread and pass");
    __shared__ T sb[NV][LT];
    for (long e = blockIdx.x * (long)LT + threadIdx.x; e < V; e += stride) {
      T v = (T)w[e];
#pragma unroll
      for (int i = 0; i < NV; ++i)
        if (i < n) {
          const T bi = basis[bidx(i, e, V, D)];
          sb[i][threadIdx.x] = bi;
          v = fma_t(-c[i], bi, v);
        }
      w[e] = (double)v;
#pragma unroll
      for (int i = 0; i < NV; ++i)
        if (i < n) acc[i] = fma_t(sb[i][threadIdx.x], v, acc[i]);
    }
    block_sum_store<NV>(acc, n, part + (long)blockIdx.x * n);
    return;
  }
  for (long e0 = blockIdx.x * (long)LT + threadIdx.x; e0 < V; e0 += stride * U) {
    T b[U][NV], v[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const long e = e0 + u * stride;
      v[u] = e < V ? (T)w[e] : (T)0;
#pragma unroll
      for (int i = 0; i < NV; ++i) b[u][i] = (i < n && e < V) ? basis[bidx(i, e, V, D)] : (T)0;
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
#pragma unroll
      for (int i = 0; i < NV; ++i)
        if (i < n) v[u] = fma_t(-c[i], b[u][i], v[u]);
      const long e = e0 + u * stride;
      if (e < V) w[e] = (double)v[u];
#pragma unroll
      for (int i = 0; i < NV; ++i)
        if (i < n) acc[i] = fma_t(b[u][i], v[u], acc[i]);
    }
  }
  block_sum_store<NV>(acc, n, part + (long)blockIdx.x * n);
}

// (C) w -= sum_i h_i basis_i, then part[b] = block share of ||w_new||^2
template <int NV, int U, class T>
__global__ void __launch_bounds__(LT, 2) cgs_axpy_norm(double* __restrict__ w, const T* __restrict__ basis,
                                                    const double* h, int n, long V, int D, double* part,
                                                    const double* done) {
  if (done && *done != 0.0) return;
  __shared__ T c[NV];
  if (threadIdx.x < NV) c[threadIdx.x] = threadIdx.x < n ? (T)h[threadIdx.x] : (T)0;
  __syncthreads();
  T acc[1] = {0};
  const long stride = (long)gridDim.x * LT;
  for (long e0 = blockIdx.x * (long)LT + threadIdx.x; e0 < V; e0 += stride * U) {
    T v[U];
#pragma unroll
    for (int u = 0; u < U; ++u) v[u] = (e0 + u * stride < V) ? (T)w[e0 + u * stride] : (T)0;
#pragma unroll
    for (int i = 0; i < NV; ++i)
      if (i < n) {
#pragma unroll
        for (int u = 0; u < U; ++u)
          if (e0 + u * stride < V) v[u] = fma_t(-c[i], basis[bidx(i, e0 + u * stride, V, D)], v[u]);
      }
#pragma unroll
    for (int u = 0; u < U; ++u)
      if (e0 + u * stride < V) {
        w[e0 + u * stride] = (double)v[u];
        acc[0] = fma_t(v[u], v[u], acc[0]);
      }
  }
  block_sum_store<1>(acc, 1, part + blockIdx.x);
}

// out = sum_{i < n} coef[i] * basis_i with n = nvec, or (int)*nvec_dev if given; an FP32
// basis (at most 61 vectors) is summed in FP32, since it gives the vector no more accuracy
template <class T>
__global__ void combine(double* out, const T* basis, const double* coef, int nvec, const double* nvec_dev,
                        long V, int D) {
  const int n = nvec_dev ? (int)(*nvec_dev) : nvec;
  if constexpr (std::is_same<T, float>::value) {
    __shared__ float c[64];
    for (int i = threadIdx.x; i < 64; i += blockDim.x) c[i] = i < n ? (float)coef[i] : 0.0f;
    __syncthreads();
    for (long e = blockIdx.x * (long)LT + threadIdx.x; e < V; e += (long)gridDim.x * LT) {
      float v = 0.0f;
      for (int i = 0; i < n && i < 64; ++i) v = fma_t(c[i], basis[bidx(i, e, V, D)], v);
      out[e] = (double)v;
    }
  } else {
    for (long e = blockIdx.x * (long)LT + threadIdx.x; e < V; e += (long)gridDim.x * LT) {
      double v = 0.0;
      for (int i = 0; i < n; ++i) v = fma_t(coef[i], basis[bidx(i, e, V, D)], v);
      out[e] = v;
    }
  }
}

// dst = src / sqrt(*nrm_sq) (skipped when *done != 0)
__global__ void scale_by_norm(double* dst, const double* src, const double* nrm_sq, long V, const double* done) {
  if (done && *done != 0.0) return;
  double n = sqrt(*nrm_sq);
  double inv = n > 0.0 ? 1.0 / n : 0.0;
  for (long e = blockIdx.x * (long)LT + threadIdx.x; e < V; e += (long)gridDim.x * LT) dst[e] = src[e] * inv;
}

// The same into slot i of the interleaved basis (capacity D) and into the contiguous vk.
// basis_i = src / ||src|| (in the basis' type) and vk = the same vector in FP64, so that the
// next matvec sees exactly the stored basis vector.
template <class T>
__global__ void scale_into_basis(T* basis, int i, int D, double* vk, const double* src, const double* nrm_sq,
                                 long V, const double* done) {
  if (done && *done != 0.0) return;
  double n = sqrt(*nrm_sq);
  double inv = n > 0.0 ? 1.0 / n : 0.0;
  for (long e = blockIdx.x * (long)LT + threadIdx.x; e < V; e += (long)gridDim.x * LT) {
    const T v = (T)(src[e] * inv);
    basis[bidx(i, e, V, D)] = v;
    vk[e] = (double)v;
  }
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

// Lowest eigenpair of the n x n symmetric tridiagonal (alpha, beta): theta and unit y.
// Called by all 32 lanes of one warp: each bisection round evaluates 32 Sturm
// counts at once and shrinks the bracket 33-fold; lane 0 then runs the
// inverse iteration and writes the results.
__device__ void tridiag_lowest(const double* alpha, const double* beta, int n, double* theta_out, double* yout) {
  const int lane = threadIdx.x & 31;
  double lo = 1e300, hi = -1e300;
  for (int i = 0; i < n; ++i) {
    double r = (i > 0 ? fabs(beta[i - 1]) : 0.0) + (i < n - 1 ? fabs(beta[i]) : 0.0);
    lo = fmin(lo, alpha[i] - r);
    hi = fmax(hi, alpha[i] + r);
  }
  for (int round = 0; round < 40; ++round) {
    const double w = hi - lo;
    if (!(w > 4e-16 * fmax(fabs(lo), fabs(hi)))) break;
    const double x = lo + w * (double)(lane + 1) / 33.0;
    const unsigned mask = __ballot_sync(0xffffffffu, sturm_count(alpha, beta, n, x) >= 1);
    const int first = mask ? __ffs(mask) - 1 : 32;  // smallest point above lambda_min
    const double nhi = (first < 32) ? lo + w * (double)(first + 1) / 33.0 : hi;
    const double nlo = (first > 0) ? lo + w * (double)first / 33.0 : lo;
    if (nhi >= hi && nlo <= lo) break;
    lo = nlo;
    hi = nhi;
  }
  if (lane != 0) return;
  const double theta = 0.5 * (lo + hi);
  // inverse iteration with partial pivoting (n <= 64)
  double y[64], z[64];
  double dl[64], dd[64], du[64], du2[64];
  int piv[64];
  for (int i = 0; i < n; ++i) y[i] = 1.0 / sqrt((double)n);
  const double scale = fmax(fabs(lo), fabs(hi)) + 1e-300;
  for (int iter = 0; iter < 3; ++iter) {
    for (int i = 0; i < n; ++i) {
      dd[i] = alpha[i] - theta;
      du[i] = (i < n - 1) ? beta[i] : 0.0;
      dl[i] = (i < n - 1) ? beta[i] : 0.0;
      du2[i] = 0.0;
      z[i] = y[i];
    }
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
  int imax = 0;
  for (int i = 1; i < n; ++i)
    if (fabs(y[i]) > fabs(y[imax])) imax = i;
  double sg = y[imax] < 0 ? -1.0 : 1.0;
  *theta_out = theta;
  for (int i = 0; i < n; ++i) yout[i] = sg * y[i];
}

// After step k (one warp): alpha_k from the two Gram-Schmidt passes, beta_k =
// ||w||, Ritz pair of T_{k+1} and the stop decision, all on the device. With
// tol <= 0 (fixed depth) the Ritz solve runs only at the last step or on breakdown.
__global__ void lz_step(double* S, int k, int depth, double tol) {
  if (blockIdx.x != 0) return;
  const int lane = threadIdx.x & 31;
  if (S[S_DONE] != 0.0) return;
  const double a = S[S_H + k] + S[S_H2 + k];
  const double b = sqrt(fmax(S[S_TMP], 0.0));
  __syncwarp();
  if (lane == 0) {
    S[S_ALPHA + k] = a;
    S[S_BETA + k] = b;
  }
  __syncwarp();
  const double prev = k > 0 ? S[S_BETA + k - 1] : 0.0;
  const bool breakdown = b < 1e-14 * (fabs(a) + prev + 1e-300) || !isfinite(b);
  if (tol <= 0.0 && k < depth - 1 && !breakdown) return;
  const int n = k + 1;
  double theta, y[64];
  tridiag_lowest(S + S_ALPHA, S + S_BETA, n, &theta, y);
  if (lane != 0) return;
  const double resid = fabs(b * y[n - 1]);
  const double sc = fmax(fabs(theta), 1e-300);
  const bool stop = resid < tol * sc || b < 1e-14 * sc || breakdown || k == depth - 1 || !isfinite(theta);
  S[S_THETA] = theta;
  S[S_RESID] = resid;
  S[S_NK] = (double)n;
  for (int i = 0; i < n; ++i) S[S_Y + i] = y[i];
  if (stop) S[S_DONE] = 1.0;
}

__global__ void lz_init(double* S) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    S[S_DONE] = 0.0;
    S[S_NK] = 1.0;
    S[S_Y] = 1.0;
    S[S_THETA] = 0.0;
    S[S_RESID] = 0.0;
  }
}

inline int vgrid(long V) { return (int)std::max<long>(1, std::min<long>((V + LT - 1) / LT, LB)); }

template <int NV, int U, class T>
void cgs2_launch(cudaStream_t s, const T* B, int D, double* W, double* S, int n, long V, int nb, double* part,
                 const double* done) {
  cgs_dot<NV, U, T><<<nb, LT, 0, s>>>(B, n, V, D, W, part, done);
  multi_dot_reduce<<<n, LT, 0, s>>>(part, nb, n, S + S_H, nullptr, done);
  cgs_axpy_dot<NV, U, T><<<nb, LT, 0, s>>>(W, B, S + S_H, n, V, D, part, done);
  multi_dot_reduce<<<n, LT, 0, s>>>(part, nb, n, S + S_H2, nullptr, done);
  cgs_axpy_norm<NV, U, T><<<nb, LT, 0, s>>>(W, B, S + S_H2, n, V, D, part, done);
  multi_dot_reduce<<<1, LT, 0, s>>>(part, nb, 1, S + S_TMP, nullptr, done);
}

// One CGS2 step against n <= kFusedMax basis vectors (six launches).
template <class T>
void cgs2_fused(cudaStream_t s, const T* B, int D, double* W, double* S, int n, long V, int nb, double* part,
                const double* done) {
  if (n <= 4) cgs2_launch<4, 4, T>(s, B, D, W, S, n, V, nb, part, done);
  else if (n <= 8) cgs2_launch<8, 2, T>(s, B, D, W, S, n, V, nb, part, done);
  else if (n <= 12) cgs2_launch<12, 2, T>(s, B, D, W, S, n, V, nb, part, done);
  else if (n <= 16) cgs2_launch<16, 1, T>(s, B, D, W, S, n, V, nb, part, done);
  else if (n <= 20) cgs2_launch<20, 1, T>(s, B, D, W, S, n, V, nb, part, done);
  else cgs2_launch<24, 1, T>(s, B, D, W, S, n, V, nb, part, done);
}

// Blocks for the fused streaming passes: enough resident warps on every SM to
// keep HBM busy, never more blocks than elements / LT.
int fused_grid(long V) {
  static int sms = 0;
  if (sms == 0) {
    int dev = 0;
    ATTN_CHECK_CUDA(cudaGetDevice(&dev));
    ATTN_CHECK_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  }
  return (int)std::max<long>(1, std::min<long>((V + LT - 1) / LT, 4L * sms));
}

void multi_dot_g(attn_ctx* ctx, const double* basis, int nvec, long V, int D, const double* w, double* out,
                 double* accum, const double* done) {
  const int nb = vgrid(V);
  ctx->partials.reserve(sizeof(double) * (size_t)nb * std::max(nvec, 1));
  multi_dot_partial<<<nb, LT, 0, ctx->stream>>>(basis, nvec, V, D, w, ctx->partials.as<double>(), done);
  multi_dot_reduce<<<nvec, LT, 0, ctx->stream>>>(ctx->partials.as<double>(), nb, nvec, out, accum, done);
  ctx->launches += 2;
  ATTN_CHECK_CUDA(cudaGetLastError());
}

}  // namespace

void multi_dot(attn_ctx* ctx, const double* basis, int nvec, long V, const double* w, double* out, double* accum) {
  multi_dot_g(ctx, basis, nvec, V, 0, w, out, accum, nullptr);
}

void multi_axpy_dev(attn_ctx* ctx, double* w, const double* basis, const double* coef, int nvec, long V,
                    double sign) {
  multi_axpy<<<vgrid(V), LT, 0, ctx->stream>>>(w, basis, coef, nvec, V, 0, sign, nullptr);
  ctx->launches++;
  ATTN_CHECK_CUDA(cudaGetLastError());
}

void combine_dev(attn_ctx* ctx, double* out, const double* basis, const double* coef, int nvec, long V) {
  combine<double><<<vgrid(V), LT, 0, ctx->stream>>>(out, basis, coef, nvec, nullptr, V, 0);
  ctx->launches++;
  ATTN_CHECK_CUDA(cudaGetLastError());
}

void normalise_dev(attn_ctx* ctx, double* dst, const double* src, long V, double* nrm_sq_dev) {
  multi_dot(ctx, src, 1, V, src, nrm_sq_dev, nullptr);
  scale_by_norm<<<vgrid(V), LT, 0, ctx->stream>>>(dst, src, nrm_sq_dev, V, nullptr);
  ctx->launches++;
  ATTN_CHECK_CUDA(cudaGetLastError());
}

template <class T>
void lanczos_enqueue_t(attn_ctx* ctx, const MatVec& apply, double* x, long V, int depth, double tol, LanczosWork& w,
                       int host_check_every) {
  ATTN_REQUIRE(depth >= 1 && depth <= 60, ATTN_EINVAL, "Lanczos depth must be in 1..60");
  const int D = depth + 1;                 // basis capacity
  const long chunks = (V + LT - 1) / LT;   // interleaving granule: LT elements
  w.basis.reserve(sizeof(T) * (size_t)D * chunks * LT);
  w.wvec.reserve(sizeof(double) * (size_t)V);
  w.vk.reserve(sizeof(double) * (size_t)V);
  w.scal.reserve(sizeof(double) * S_SIZE);
  T* B = w.basis.as<T>();
  double* W = w.wvec.as<double>();
  double* vk = w.vk.as<double>();
  double* S = w.scal.as<double>();
  double* done = S + S_DONE;
  cudaStream_t s = ctx->stream;
  lz_init<<<1, 1, 0, s>>>(S);
  ctx->launches++;
  // v_0 = x / |x| into basis slot 0 and the contiguous matvec input
  multi_dot_g(ctx, x, 1, V, 0, x, S + S_TMP, nullptr, nullptr);
  scale_into_basis<T><<<vgrid(V), LT, 0, s>>>(B, 0, D, vk, x, S + S_TMP, V, nullptr);
  ctx->launches++;
  for (int k = 0; k < depth; ++k) {
    apply(vk, W);
    // w -= sum_i <v_i, w> v_i over the whole basis, twice; the coefficient of
    // v_k is alpha_k and those of v_{k-1} and older vectors take the place of
    // the three-term recurrence (equal in exact arithmetic)
    const int n = k + 1;
    if (n <= kFusedMax) {
      const int nb = fused_grid(V);
      ctx->partials.reserve(sizeof(double) * (size_t)nb * n);
      cgs2_fused<T>(s, B, D, W, S, n, V, nb, ctx->partials.as<double>(), done);
      ctx->launches += 6;
    } else if constexpr (std::is_same<T, double>::value) {
      multi_dot_g(ctx, B, n, V, D, W, S + S_H, nullptr, done);
      multi_axpy<<<vgrid(V), LT, 0, s>>>(W, B, S + S_H, n, V, D, 1.0, done);
      multi_dot_g(ctx, B, n, V, D, W, S + S_H2, nullptr, done);
      multi_axpy<<<vgrid(V), LT, 0, s>>>(W, B, S + S_H2, n, V, D, 1.0, done);
      ctx->launches += 2;
      multi_dot_g(ctx, W, 1, V, 0, W, S + S_TMP, nullptr, done);
    }
    lz_step<<<1, 32, 0, s>>>(S, k, depth, tol);
    ctx->launches++;
    if (k + 1 < depth) {
      scale_into_basis<T><<<vgrid(V), LT, 0, s>>>(B, k + 1, D, vk, W, S + S_TMP, V, done);
      ctx->launches++;
    }
    if (host_check_every > 0 && (k + 1) % host_check_every == 0 && k + 1 < depth) {
      double hd = 0;
      ATTN_CHECK_CUDA(cudaMemcpyAsync(&hd, done, sizeof(double), cudaMemcpyDeviceToHost, s));
      ATTN_CHECK_CUDA(cudaStreamSynchronize(s));
      if (hd != 0.0) break;
    }
  }
  combine<T><<<vgrid(V), LT, 0, s>>>(W, B, S + S_Y, 0, S + S_NK, V, D);
  ctx->launches++;
  normalise_dev(ctx, x, W, V, S + S_TMP);
  ATTN_CHECK_CUDA(cudaGetLastError());
}

void lanczos_enqueue(attn_ctx* ctx, const MatVec& apply, double* x, long V, int depth, double tol, LanczosWork& w,
                     int host_check_every, bool f32_basis) {
  // the FP32 basis keeps every step in the fused passes
  if (f32_basis && depth <= kFusedMax) lanczos_enqueue_t<float>(ctx, apply, x, V, depth, tol, w, host_check_every);
  else lanczos_enqueue_t<double>(ctx, apply, x, V, depth, tol, w, host_check_every);
}

LanczosResult lanczos_read(attn_ctx* ctx, LanczosWork& w) {
  double h[8];
  ATTN_CHECK_CUDA(cudaMemcpyAsync(h, w.scal.as<double>() + S_DONE, sizeof(h), cudaMemcpyDeviceToHost, ctx->stream));
  ATTN_CHECK_CUDA(cudaStreamSynchronize(ctx->stream));
  // h[0] done, h[1] nk, h[2] theta, h[3] resid
  LanczosResult r{h[2], (int)h[1], h[3], false};
  ATTN_REQUIRE(std::isfinite(r.theta), ATTN_ENONFINITE, "non-finite value in Lanczos");
  return r;
}

LanczosResult lanczos_lowest(attn_ctx* ctx, const MatVec& apply, double* x, long V, int depth, double tol,
                             LanczosWork& w, bool f32_basis) {
  lanczos_enqueue(ctx, apply, x, V, depth, tol, w, tol > 0.0 ? 5 : 0, f32_basis);
  LanczosResult r = lanczos_read(ctx, w);
  r.converged = r.resid < tol * std::max(std::fabs(r.theta), 1e-300);
  return r;
}

}  // namespace attn
