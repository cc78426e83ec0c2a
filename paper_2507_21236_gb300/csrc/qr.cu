// FP64 QR re-isometrisation on the GPU (Sec. 3.1, Fig. iso).
//
// A node tensor is viewed as the matrix A (M x k) whose column index is the
// link towards the next isometry centre; A = Q R with Q^T Q = 1 and
// R upper triangular, diag(R) >= 0. Columns are orthogonalised one after the
// other by classical Gram-Schmidt applied twice ("CGS2", numerically as
// orthogonal as Householder for full-rank A). A column whose remaining norm
// falls below 1e-13 of its original norm is rank-deficient: its R diagonal is
// set to 0 and, after the sweep over columns, it is replaced by a unit vector
// orthogonalised against all other columns (A = Q R still holds because every
// later column was orthogonalised against the zero column).
//
// Storage: At[j][row] = A[row][j] (each column contiguous).
// Per column: [dots] -> [update + dots] -> [update + norm] -> [finalise]
// with every block reducing the partials itself (no extra reduce launches).
#include <algorithm>
#include <cmath>

#include "attn_internal.h"
#include "qr.h"

namespace attn {

namespace {

constexpr int QT = 256;   // threads per block
constexpr int QROWS = 256;   // rows per block (one per thread)

__device__ __forceinline__ double warp_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

// part[b][i] = sum_{rows of block b} At[i][row] * At[j][row], i < j
__device__ void partial_dots(const double* At, long M, int j, double* part, int nblk_stride) {
  const long r0 = (long)blockIdx.x * QROWS;
  const long r1 = min(M, r0 + QROWS);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const double* a = At + (long)j * M;
  for (int i = warp; i < j; i += QT / 32) {
    const double* q = At + (long)i * M;
    double s = 0.0;
    for (long r = r0 + lane; r < r1; r += 32) s = fma(q[r], a[r], s);
    s = warp_sum(s);
    if (lane == 0) part[(long)blockIdx.x * nblk_stride + i] = s;
  }
}

// h[i] = sum_b part[b][i] for i < j (into shared), R[i][j] += h[i] by block 0.
__device__ void reduce_h(const double* part, int nb, int j, int stride, double* h, double* R, int k, bool accum_R) {
  for (int i = threadIdx.x; i < j; i += QT) {
    double s = 0.0;
    for (int b = 0; b < nb; ++b) s += part[(long)b * stride + i];
    h[i] = s;
    if (accum_R && blockIdx.x == 0) R[(long)i * k + j] += s;
  }
  __syncthreads();
}

__global__ void qr_init_kernel(const double* At, long M, int k, double* nrm0, double* R) {
  // nrm0[j] = ||a_j|| (one block per column), R zeroed
  int j = blockIdx.x;
  __shared__ double sh[QT / 32];
  const double* a = At + (long)j * M;
  double s = 0.0;
  for (long r = threadIdx.x; r < M; r += QT) s = fma(a[r], a[r], s);
  s = warp_sum(s);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0;
    for (int w = 0; w < QT / 32; ++w) t += sh[w];
    nrm0[j] = sqrt(t);
  }
  for (int c = threadIdx.x; c < k; c += QT) R[(long)j * k + c] = 0.0;
}

__global__ void qr_dots_kernel(const double* At, long M, int j, double* part, int stride) {
  partial_dots(At, M, j, part, stride);
}

// a_j -= Q h (h from partials); then either the next dots or the norm partial.
__global__ void qr_update_kernel(double* At, long M, int j, int k, double* part, int nb, int stride, double* R,
                                 int next_is_norm, double* part2) {
  extern __shared__ double h[];
  reduce_h(part, nb, j, stride, h, R, k, true);
  const long r0 = (long)blockIdx.x * QROWS;
  const long r1 = min(M, r0 + QROWS);
  double* a = At + (long)j * M;
  for (long r = r0 + threadIdx.x; r < r1; r += QT) {
    double v = a[r];
    for (int i = 0; i < j; ++i) v = fma(-h[i], At[(long)i * M + r], v);
    a[r] = v;
  }
  __syncthreads();
  if (!next_is_norm) {
    partial_dots(At, M, j, part2, stride);
  } else {
    __shared__ double sh[QT / 32];
    double s = 0.0;
    for (long r = r0 + threadIdx.x; r < r1; r += QT) s = fma(a[r], a[r], s);
    s = warp_sum(s);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
      double t = 0;
      for (int w = 0; w < QT / 32; ++w) t += sh[w];
      part2[blockIdx.x] = t;
    }
  }
}

__global__ void qr_norm_partial_kernel(const double* At, long M, int j, double* part) {
  __shared__ double sh[QT / 32];
  const long r0 = (long)blockIdx.x * QROWS;
  const long r1 = min(M, r0 + QROWS);
  const double* a = At + (long)j * M;
  double s = 0.0;
  for (long r = r0 + threadIdx.x; r < r1; r += QT) s = fma(a[r], a[r], s);
  s = warp_sum(s);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0;
    for (int w = 0; w < QT / 32; ++w) t += sh[w];
    part[blockIdx.x] = t;
  }
}

__global__ void qr_finalise_kernel(double* At, long M, int j, int k, const double* part, int nb, const double* nrm0,
                                   double* R, int* deficient) {
  __shared__ double rj;
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int b = 0; b < nb; ++b) s += part[b];
    double r = sqrt(s);
    if (!(r > 1e-13 * nrm0[j]) || !(r > 1e-300)) {
      r = 0.0;
      if (blockIdx.x == 0) deficient[j] = 1;
    } else if (blockIdx.x == 0) {
      deficient[j] = 0;
    }
    rj = r;
    if (blockIdx.x == 0) R[(long)j * k + j] = r;
  }
  __syncthreads();
  const double inv = rj > 0.0 ? 1.0 / rj : 0.0;
  const long r0 = (long)blockIdx.x * QROWS;
  const long r1 = min(M, r0 + QROWS);
  double* a = At + (long)j * M;
  for (long r = r0 + threadIdx.x; r < r1; r += QT) a[r] *= inv;
}

// Replacement of deficient column j: a_j = e_t, then CGS2 against all other columns.
__global__ void qr_set_unit_kernel(double* At, long M, int j, long t) {
  double* a = At + (long)j * M;
  for (long r = blockIdx.x * (long)blockDim.x + threadIdx.x; r < M; r += (long)gridDim.x * blockDim.x)
    a[r] = (r == t) ? 1.0 : 0.0;
}

// single-block: a_j -= sum_{i != j} <q_i, a_j> q_i (all other columns), twice, then normalise; writes norm
__global__ void qr_fix_column_kernel(double* At, long M, int j, int k, double* out_norm) {
  extern __shared__ double h[];
  __shared__ double sh[QT / 32];
  double* a = At + (long)j * M;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int pass = 0; pass < 2; ++pass) {
    for (int i = warp; i < k; i += QT / 32) {
      double s = 0.0;
      if (i != j) {
        const double* q = At + (long)i * M;
        for (long r = lane; r < M; r += 32) s = fma(q[r], a[r], s);
      }
      s = warp_sum(s);
      if (lane == 0) h[i] = s;
    }
    __syncthreads();
    for (long r = threadIdx.x; r < M; r += QT) {
      double v = a[r];
      for (int i = 0; i < k; ++i)
        if (i != j) v = fma(-h[i], At[(long)i * M + r], v);
      a[r] = v;
    }
    __syncthreads();
  }
  double s = 0.0;
  for (long r = threadIdx.x; r < M; r += QT) s = fma(a[r], a[r], s);
  s = warp_sum(s);
  if (lane == 0) sh[warp] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0;
    for (int w = 0; w < QT / 32; ++w) t += sh[w];
    sh[0] = sqrt(t);
    *out_norm = sh[0];
  }
  __syncthreads();
  double inv = sh[0] > 0.5 ? 1.0 / sh[0] : 0.0;
  for (long r = threadIdx.x; r < M; r += QT) a[r] *= inv;
}

// Permute T[d0][d1][d2] into At[k = d_slot][M] (other two indices in order) and back.
__global__ void to_columns_kernel(const double* T, int d0, int d1, int d2, int slot, double* At) {
  long V = (long)d0 * d1 * d2;
  for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < V; e += (long)gridDim.x * blockDim.x) {
    int c = e % d2;
    long t = e / d2;
    int b = t % d1;
    int a = t / d1;
    long col, row;
    if (slot == 0) { col = a; row = (long)b * d2 + c; }
    else if (slot == 1) { col = b; row = (long)a * d2 + c; }
    else { col = c; row = (long)a * d1 + b; }
    long M = V / (slot == 0 ? d0 : slot == 1 ? d1 : d2);
    At[col * M + row] = T[e];
  }
}

__global__ void from_columns_kernel(const double* At, int d0, int d1, int d2, int slot, double* T) {
  long V = (long)d0 * d1 * d2;
  for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < V; e += (long)gridDim.x * blockDim.x) {
    int c = e % d2;
    long t = e / d2;
    int b = t % d1;
    int a = t / d1;
    long col, row;
    if (slot == 0) { col = a; row = (long)b * d2 + c; }
    else if (slot == 1) { col = b; row = (long)a * d2 + c; }
    else { col = c; row = (long)a * d1 + b; }
    long M = V / (slot == 0 ? d0 : slot == 1 ? d1 : d2);
    T[e] = At[col * M + row];
  }
}

int grid1(long n) { return (int)std::max<long>(1, std::min<long>((n + 255) / 256, 4096)); }

}  // namespace

void qr_columns(attn_ctx* ctx, double* At, long M, int k, double* R, QRWork& w) {
  ATTN_REQUIRE(k >= 1 && M >= k, ATTN_EINVAL, "QR needs M >= k >= 1 (link wider than its other side)");
  const int nb = (int)((M + QROWS - 1) / QROWS);
  const int stride = k;
  w.part.reserve(sizeof(double) * ((size_t)nb * k + 16));
  w.part2.reserve(sizeof(double) * ((size_t)nb * k + 16));
  w.nrm0.reserve(sizeof(double) * k);
  w.defic.reserve(sizeof(int) * k);
  double* part = w.part.as<double>();
  double* part2 = w.part2.as<double>();
  double* nrm0 = w.nrm0.as<double>();
  int* def = w.defic.as<int>();
  cudaStream_t s = ctx->stream;
  qr_init_kernel<<<k, QT, 0, s>>>(At, M, k, nrm0, R);
  ctx->launches++;
  const size_t hsh = sizeof(double) * k;
  for (int j = 0; j < k; ++j) {
    if (j > 0) {
      qr_dots_kernel<<<nb, QT, 0, s>>>(At, M, j, part, stride);
      qr_update_kernel<<<nb, QT, hsh, s>>>(At, M, j, k, part, nb, stride, R, 0, part2);
      qr_update_kernel<<<nb, QT, hsh, s>>>(At, M, j, k, part2, nb, stride, R, 1, part);
      ctx->launches += 3;
    } else {
      qr_norm_partial_kernel<<<nb, QT, 0, s>>>(At, M, j, part);
      ctx->launches++;
    }
    qr_finalise_kernel<<<nb, QT, 0, s>>>(At, M, j, k, part, nb, nrm0, R, def);
    ctx->launches++;
  }
  ATTN_CHECK_CUDA(cudaGetLastError());
  // rank-deficient columns (rare): host check, one small sync
  std::vector<int> hdef(k);
  ATTN_CHECK_CUDA(cudaMemcpyAsync(hdef.data(), def, sizeof(int) * k, cudaMemcpyDeviceToHost, s));
  ATTN_CHECK_CUDA(cudaStreamSynchronize(s));
  for (int j = 0; j < k; ++j) {
    if (!hdef[j]) continue;
    bool ok = false;
    for (long trial = 0; trial < std::min<long>(M, 64) && !ok; ++trial) {
      long t = ((long)j * 7919 + trial * 104729) % M;
      qr_set_unit_kernel<<<grid1(M), 256, 0, s>>>(At, M, j, t);
      qr_fix_column_kernel<<<1, QT, hsh, s>>>(At, M, j, k, part);
      ctx->launches += 2;
      double nrm = 0;
      ATTN_CHECK_CUDA(cudaMemcpyAsync(&nrm, part, sizeof(double), cudaMemcpyDeviceToHost, s));
      ATTN_CHECK_CUDA(cudaStreamSynchronize(s));
      ok = nrm > 0.5;
    }
    ATTN_REQUIRE(ok, ATTN_ENOTISOMETRIC, "QR could not complete a rank-deficient column");
  }
}

void tensor_to_columns(attn_ctx* ctx, const double* T, const int d[3], int slot, double* At) {
  long V = (long)d[0] * d[1] * d[2];
  to_columns_kernel<<<grid1(V), 256, 0, ctx->stream>>>(T, d[0], d[1], d[2], slot, At);
  ctx->launches++;
  ATTN_CHECK_CUDA(cudaGetLastError());
}

void columns_to_tensor(attn_ctx* ctx, const double* At, const int d[3], int slot, double* T) {
  long V = (long)d[0] * d[1] * d[2];
  from_columns_kernel<<<grid1(V), 256, 0, ctx->stream>>>(At, d[0], d[1], d[2], slot, T);
  ctx->launches++;
  ATTN_CHECK_CUDA(cudaGetLastError());
}

}  // namespace attn
