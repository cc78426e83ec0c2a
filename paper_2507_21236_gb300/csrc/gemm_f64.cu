// FP64 CUDA-core contraction kernels.
//
// One generic batched, grouped, fully strided GEMM covers every FP64
// contraction of the method: the two stages of each H_eff product
// (Sec. 4.4.2, Fig. eff-op-cost), the renormalisation T^T (O (x) O) T
// (Fig. eff-op) and the Gram/projection products of QR. GB300's FP64 rate is
// low (FMA-bound at about 1.2 TFLOP/s), so the kernel is a plain
// shared-memory-tiled register-blocked GEMM: a BM x BN output tile per
// 256-thread CTA (16 x 16 threads, BM/16 x BN/16 accumulators each), K tile 16;
// loads pick the coalesced mapping from the unit stride of each operand. The
// tile is 32 or 64 wide in each direction, chosen from M and N: the mode
// products of link dimension 32 are batches of 32 x 32 GEMMs, which a 64 x 64
// tile would compute at a quarter of its width. A GEMM whose output tiles do not
// fill one wave of resident CTAs (the product-summing stage at m = 64 has 64)
// splits its G reduction over CTA groups; the partial outputs are summed in a
// fixed order by a second kernel, so results do not depend on scheduling.
#include <cuda_runtime.h>

#include <algorithm>

#include "attn_internal.h"
#include "ozaki.h"

namespace attn {

namespace {

constexpr int BK = 16, NT = 256;

template <int BM, int BN>
__global__ void __launch_bounds__(NT) gemm_f64_kernel(GemmF64 g) {
  constexpr int TM = BM / 16, TN = BN / 16;  // accumulators per thread
  __shared__ double As[BK][BM + 1];
  __shared__ double Bs[BK][BN + 1];
  const int tid = threadIdx.x;
  const int tx = tid % 16, ty = tid / 16;
  const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
  const long nb = (long)g.Bhi * g.Blo;
  const bool a_kfast = (g.aK == 1);
  const bool b_nfast = (g.bN == 1);
  for (long bz = blockIdx.z; bz < nb * g.gsplit; bz += gridDim.z) {
    const long sp = bz / nb, bb = bz % nb;
    const long bh = bb / g.Blo, bl = bb % g.Blo;
    const double* Ab = g.A + bh * g.aBhi + bl * g.aBlo;
    const double* Bb = g.B + bh * g.bBhi + bl * g.bBlo;
    double* Cb = g.C + sp * g.cS + bh * g.cBhi + bl * g.cBlo;
    const int ga = (int)(sp * g.G / g.gsplit), gb = (int)((sp + 1) * g.G / g.gsplit);
    double acc[TM][TN];
#pragma unroll
    for (int i = 0; i < TM; ++i)
#pragma unroll
      for (int j = 0; j < TN; ++j) acc[i][j] = 0.0;
    for (int gg = ga; gg < gb; ++gg) {
      const double* Ag = Ab + gg * g.aG;
      const double* Bg = Bb + gg * g.bG;
      for (int k0 = 0; k0 < g.K; k0 += BK) {
#pragma unroll
        for (int q = 0; q < (BM * BK) / NT; ++q) {
          int e = tid + q * NT;
          int i, k;
          if (a_kfast) { k = e % BK; i = e / BK; } else { i = e % BM; k = e / BM; }
          int gi = m0 + i, gk = k0 + k;
          As[k][i] = (gi < g.M && gk < g.K) ? Ag[gi * g.aM + gk * g.aK] : 0.0;
        }
#pragma unroll
        for (int q = 0; q < (BN * BK) / NT; ++q) {
          int e = tid + q * NT;
          int j, k;
          if (b_nfast) { j = e % BN; k = e / BN; } else { k = e % BK; j = e / BK; }
          int gj = n0 + j, gk = k0 + k;
          Bs[k][j] = (gj < g.N && gk < g.K) ? Bg[gk * g.bK + gj * g.bN] : 0.0;
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < BK; ++k) {
          double a[TM], b[TN];
#pragma unroll
          for (int i = 0; i < TM; ++i) a[i] = As[k][ty + 16 * i];
#pragma unroll
          for (int j = 0; j < TN; ++j) b[j] = Bs[k][tx + 16 * j];
#pragma unroll
          for (int i = 0; i < TM; ++i)
#pragma unroll
            for (int j = 0; j < TN; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
        }
        __syncthreads();
      }
    }
#pragma unroll
    for (int i = 0; i < TM; ++i) {
      int gi = m0 + ty + 16 * i;
      if (gi >= g.M) continue;
#pragma unroll
      for (int j = 0; j < TN; ++j) {
        int gj = n0 + tx + 16 * j;
        if (gj >= g.N) continue;
        double* c = Cb + gi * g.cM + gj * g.cN;
        double v = g.alpha * acc[i][j];
        *c = (g.beta == 0.0) ? v : fma(g.beta, *c, v);
      }
    }
  }
}

// C = beta C + alpha sum_s P[s] over the dense partials P[gsplit][batch][M][N].
__global__ void split_reduce_kernel(GemmF64 g, const double* __restrict__ P) {
  const long mn = (long)g.M * g.N, per = (long)g.Bhi * g.Blo * mn;
  for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < per; e += (long)gridDim.x * blockDim.x) {
    const long b = e / mn, r = e % mn;
    const long i = r / g.N, j = r % g.N;
    double s = 0.0;
    for (int sp = 0; sp < g.gsplit; ++sp) s += P[sp * per + e];
    double* c = g.C + (b / g.Blo) * g.cBhi + (b % g.Blo) * g.cBlo + i * g.cM + j * g.cN;
    const double v = g.alpha * s;
    *c = (g.beta == 0.0) ? v : fma(g.beta, *c, v);
  }
}

__global__ void fill_kernel(double* p, size_t n, double v) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) p[i] = v;
}

__global__ void axpy_kernel(double* y, const double* x, size_t n, double a) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    y[i] = fma(a, x[i], y[i]);
}

__global__ void copy_kernel(double* d, const double* s, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) d[i] = s[i];
}

__global__ void gather_kernel(double* dst, const double* src, const int* idx, int R, long len) {
  long total = (long)R * len;
  for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < total; e += (long)gridDim.x * blockDim.x) {
    long r = e / len, o = e % len;
    dst[e] = src[(long)idx[r] * len + o];
  }
}

__global__ void identity_kernel(double* dst, int R, int m) {
  long total = (long)R * m * m;
  for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < total; e += (long)gridDim.x * blockDim.x) {
    long o = e % ((long)m * m);
    dst[e] = (o / m == o % m) ? 1.0 : 0.0;
  }
}

// Deterministic two-pass dot product: per-block partials then one block sums them.
__global__ void dot_partial_kernel(const double* x, const double* y, size_t n, double* part) {
  __shared__ double sh[32];
  double s = 0.0;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    s = fma(x[i], y[i], s);
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x < 32) {
    s = (threadIdx.x < (blockDim.x >> 5)) ? sh[threadIdx.x] : 0.0;
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if (threadIdx.x == 0) part[blockIdx.x] = s;
  }
}

__global__ void sum_partials_kernel(const double* part, int n, double* out) {
  __shared__ double sh[32];
  double s = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) s += part[i];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x < 32) {
    s = (threadIdx.x < (blockDim.x >> 5)) ? sh[threadIdx.x] : 0.0;
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if (threadIdx.x == 0) *out = s;
  }
}

inline int grid_for(size_t n, int threads = 256, int cap = 4096) {
  size_t b = (n + threads - 1) / threads;
  return (int)std::max<size_t>(1, std::min<size_t>(b, (size_t)cap));
}

}  // namespace

// Launch with the tile shape that wastes least of M and N (grid.y > 65535 is rejected).
cudaError_t launch_gemm(cudaStream_t stream, const GemmF64& g) {
  const bool sm = g.M <= 32, sn = g.N <= 32;
  const int bm = sm ? 32 : 64, bn = sn ? 32 : 64;
  dim3 grid((g.N + bn - 1) / bn, (g.M + bm - 1) / bm, (unsigned)std::min<long>((long)g.Bhi * g.Blo * g.gsplit, 65535));
  if (grid.y > 65535) return cudaErrorInvalidValue;
  if (sm && sn) gemm_f64_kernel<32, 32><<<grid, NT, 0, stream>>>(g);
  else if (sm) gemm_f64_kernel<32, 64><<<grid, NT, 0, stream>>>(g);
  else if (sn) gemm_f64_kernel<64, 32><<<grid, NT, 0, stream>>>(g);
  else gemm_f64_kernel<64, 64><<<grid, NT, 0, stream>>>(g);
  return cudaGetLastError();
}

// Resident CTAs per SM of the tile shape launch_gemm picks for g (queried once per shape).
static int resident_ctas(const GemmF64& g) {
  static int occ[4] = {0, 0, 0, 0};
  const int v = (g.M <= 32 ? 2 : 0) + (g.N <= 32 ? 1 : 0);
  if (!occ[v]) {
    cudaError_t e;
    if (v == 3) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ[v], gemm_f64_kernel<32, 32>, NT, 0);
    else if (v == 2) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ[v], gemm_f64_kernel<32, 64>, NT, 0);
    else if (v == 1) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ[v], gemm_f64_kernel<64, 32>, NT, 0);
    else e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ[v], gemm_f64_kernel<64, 64>, NT, 0);
    ATTN_CHECK_CUDA(e);
    occ[v] = std::max(occ[v], 1);
  }
  return occ[v];
}

void gemm_f64(attn_ctx* ctx, const GemmF64& g) {
  if (g.M <= 0 || g.N <= 0 || g.Bhi <= 0 || g.Blo <= 0) return;
  ATTN_REQUIRE((g.M + 31) / 32 <= 65535, ATTN_EUNSUPPORTED, "GEMM M too large");
  const double fl = 2.0 * g.M * g.N * (double)g.K * g.G * g.Bhi * g.Blo;
  // marked contractions of at least ~1e8 FLOP run as exact BF16 slice products when
  // enabled: GB300's FP64 FMA rate is a small fraction of its tensor-core rate. The
  // slicing grid takes at most 65535 distinct batch entries per operand.
  const long nbA = (g.aBhi ? (long)g.Bhi : 1L) * (g.aBlo ? (long)g.Blo : 1L);
  const long nbB = (g.bBhi ? (long)g.Bhi : 1L) * (g.bBlo ? (long)g.Blo : 1L);
  if (ctx->cfg.f64_split && g.split_ok && fl >= 1e8 && std::max(g.M, g.N) >= 32 && nbA <= 65535 &&
      nbB <= 65535) {
    gemm_f64_ozaki(ctx, g);
    return;
  }
  const int bm = g.M <= 32 ? 32 : 64, bn = g.N <= 32 ? 32 : 64;
  const long nb = (long)g.Bhi * g.Blo;
  const long tiles = (long)((g.N + bn - 1) / bn) * ((g.M + bm - 1) / bm) * nb;
  const long slots = (long)std::max(ctx->num_sms, 1) * resident_ctas(g);
  // split the G reduction when the output tiles fill less than half a wave: as many
  // groups as keep the whole grid within one wave of resident CTAs
  const int ks = (g.G >= 2 && 2 * tiles <= slots) ? (int)std::min<long>(g.G, slots / tiles) : 1;
  ctx->prof_begin(1);
  if (ks > 1) {
    const long per = nb * g.M * g.N;
    ctx->gsplit_ws.reserve(sizeof(double) * (size_t)ks * per);
    GemmF64 p = g;
    p.C = ctx->gsplit_ws.as<double>();
    p.cN = 1;
    p.cM = g.N;
    p.cBlo = (long)g.M * g.N;
    p.cBhi = (long)g.Blo * g.M * g.N;
    p.cS = per;
    p.gsplit = ks;
    p.alpha = 1.0;
    p.beta = 0.0;
    ATTN_CHECK_CUDA(launch_gemm(ctx->stream, p));
    GemmF64 r = g;
    r.gsplit = ks;
    split_reduce_kernel<<<grid_for((size_t)per), 256, 0, ctx->stream>>>(r, p.C);
    ctx->launches += 2;
  } else {
    ATTN_CHECK_CUDA(launch_gemm(ctx->stream, g));
    ctx->launches++;
  }
  ctx->prof_end(1, fl);
  ATTN_CHECK_CUDA(cudaGetLastError());
}

cudaError_t gemm_f64_stream(cudaStream_t stream, const GemmF64& g) {
  if (g.M <= 0 || g.N <= 0 || g.Bhi <= 0 || g.Blo <= 0) return cudaSuccess;
  return launch_gemm(stream, g);
}

cudaError_t fill_f64_stream(cudaStream_t stream, double* p, size_t n, double v) {
  if (!n) return cudaSuccess;
  fill_kernel<<<grid_for(n), 256, 0, stream>>>(p, n, v);
  return cudaGetLastError();
}

void mode_product_f64(attn_ctx* ctx, const int d[3], int slot, const double* mats, int R, const double* in,
                      long in_stride, double* out, double beta) {
  const long V = (long)d[0] * d[1] * d[2];
  const long ms = (long)d[slot] * d[slot];
  GemmF64 g;
  g.split_ok = true;
  g.beta = beta;
  if (slot == 0) {
    // out_r[i, (bc)] = sum_j M_r[i, j] in_r[j, (bc)]
    g.M = d[0]; g.N = d[1] * d[2]; g.K = d[0];
    g.A = mats; g.aM = d[0]; g.aK = 1; g.aBhi = ms;
    g.B = in; g.bK = (long)d[1] * d[2]; g.bN = 1; g.bBhi = in_stride;
    g.C = out; g.cM = (long)d[1] * d[2]; g.cN = 1; g.cBhi = V;
    g.Bhi = R; g.Blo = 1;
  } else if (slot == 1) {
    // out_r[a][i, c] = sum_j M_r[i, j] in_r[a][j, c]
    g.M = d[1]; g.N = d[2]; g.K = d[1];
    g.A = mats; g.aM = d[1]; g.aK = 1; g.aBhi = ms; g.aBlo = 0;
    g.B = in; g.bK = d[2]; g.bN = 1; g.bBhi = in_stride; g.bBlo = (long)d[1] * d[2];
    g.C = out; g.cM = d[2]; g.cN = 1; g.cBhi = V; g.cBlo = (long)d[1] * d[2];
    g.Bhi = R; g.Blo = d[0];
  } else {
    // out_r[(ab), i] = sum_j in_r[(ab), j] M_r[i, j]
    g.M = d[0] * d[1]; g.N = d[2]; g.K = d[2];
    g.A = in; g.aM = d[2]; g.aK = 1; g.aBhi = in_stride;
    g.B = mats; g.bK = 1; g.bN = d[2]; g.bBhi = ms;
    g.C = out; g.cM = d[2]; g.cN = 1; g.cBhi = V;
    g.Bhi = R; g.Blo = 1;
  }
  gemm_f64(ctx, g);
}

void fill_f64(attn_ctx* ctx, double* p, size_t n, double v) {
  if (!n) return;
  fill_kernel<<<grid_for(n), 256, 0, ctx->stream>>>(p, n, v);
  ctx->launches++;
  ATTN_CHECK_CUDA(cudaGetLastError());
}

void copy_f64(attn_ctx* ctx, double* d, const double* s, size_t n) {
  if (!n) return;
  copy_kernel<<<grid_for(n), 256, 0, ctx->stream>>>(d, s, n);
  ctx->launches++;
  ATTN_CHECK_CUDA(cudaGetLastError());
}

void axpy_f64(attn_ctx* ctx, double* y, const double* x, size_t n, double a) {
  if (!n) return;
  axpy_kernel<<<grid_for(n), 256, 0, ctx->stream>>>(y, x, n, a);
  ctx->launches++;
  ATTN_CHECK_CUDA(cudaGetLastError());
}

void gather_rows_f64(attn_ctx* ctx, double* dst, const double* src, const int* idx, int R, long len) {
  if (R <= 0 || len <= 0) return;
  gather_kernel<<<grid_for((size_t)R * len), 256, 0, ctx->stream>>>(dst, src, idx, R, len);
  ctx->launches++;
  ATTN_CHECK_CUDA(cudaGetLastError());
}

void identity_stack_f64(attn_ctx* ctx, double* dst, int R, int m) {
  if (R <= 0) return;
  identity_kernel<<<grid_for((size_t)R * m * m), 256, 0, ctx->stream>>>(dst, R, m);
  ctx->launches++;
  ATTN_CHECK_CUDA(cudaGetLastError());
}

void dot_f64(attn_ctx* ctx, const double* x, const double* y, size_t n, double* out_dev) {
  const int blocks = 256;
  ctx->partials.reserve(sizeof(double) * blocks);
  double* part = ctx->partials.as<double>();
  dot_partial_kernel<<<blocks, 256, 0, ctx->stream>>>(x, y, n, part);
  sum_partials_kernel<<<1, 256, 0, ctx->stream>>>(part, blocks, out_dev);
  ctx->launches += 2;
  ATTN_CHECK_CUDA(cudaGetLastError());
}

}  // namespace attn
