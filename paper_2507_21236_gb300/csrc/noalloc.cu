// Allocation-free FP64 H_eff application for callers that cannot allocate
// device memory.
//
// Some callers cannot call cudaMalloc: a host framework may have reserved all
// free device memory for its own pool and forbid raw allocations, and
// latency-critical code must avoid the implicit device-wide synchronisation
// that cudaFree performs. For them this entry point computes the same
// y = H_eff x as attn_heff_create + attn_heff_apply(ATTN_F64) but reads the
// caller's operator arrays in place and uses, as its only scratch, one
// file-scope device array of ATTN_NOALLOC_SCRATCH_DOUBLES doubles (16 MiB),
// which a GPU holds, once committed by the first call there, until the process
// exits (CUDA loads device code lazily by default).
#include <mutex>

#include "attn_internal.h"

namespace {

constexpr long kScratchDoubles = ATTN_NOALLOC_SCRATCH_DOUBLES;
constexpr int kMaxDevices = 64;

// The scratch array. In host code this name is a host-side stand-in, not a
// device address: kernels get the address from cudaGetSymbolAddress.
static __device__ __align__(256) double g_noalloc_scratch[kScratchDoubles];

std::mutex g_mu;
double* g_scratch_addr[kMaxDevices] = {nullptr};

// Set-up, once per device, with that device current.
cudaError_t scratch_address(double** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_addr[dev] = static_cast<double*>(p);
  }
  *out = g_scratch_addr[dev];
  return cudaSuccess;
}

// out_r = beta out_r + mat_r x_slot in_r for a [d0][d1][d2] tensor (in_stride 0: shared input).
cudaError_t mode_product(cudaStream_t s, const int d[3], int slot, const double* mats, int R, const double* in,
                         long in_stride, double* out, double beta) {
  const long V = (long)d[0] * d[1] * d[2];
  const long ms = (long)d[slot] * d[slot];
  attn::GemmF64 g;
  g.beta = beta;
  if (slot == 0) {
    g.M = d[0]; g.N = d[1] * d[2]; g.K = d[0];
    g.A = mats; g.aM = d[0]; g.aK = 1; g.aBhi = ms;
    g.B = in; g.bK = (long)d[1] * d[2]; g.bN = 1; g.bBhi = in_stride;
    g.C = out; g.cM = (long)d[1] * d[2]; g.cN = 1; g.cBhi = V;
    g.Bhi = R;
  } else if (slot == 1) {
    g.M = d[1]; g.N = d[2]; g.K = d[1];
    g.A = mats; g.aM = d[1]; g.aK = 1; g.aBhi = ms;
    g.B = in; g.bK = d[2]; g.bN = 1; g.bBhi = in_stride; g.bBlo = (long)d[1] * d[2];
    g.C = out; g.cM = d[2]; g.cN = 1; g.cBhi = V; g.cBlo = (long)d[1] * d[2];
    g.Bhi = R; g.Blo = d[0];
  } else {
    g.M = d[0] * d[1]; g.N = d[2]; g.K = d[2];
    g.A = in; g.aM = d[2]; g.aK = 1; g.aBhi = in_stride;
    g.B = mats; g.bK = 1; g.bN = d[2]; g.bBhi = ms;
    g.C = out; g.cM = d[2]; g.cN = 1; g.cBhi = V;
    g.Bhi = R;
  }
  return attn::gemm_f64_stream(s, g);
}

// y += sum_{r<R} A_r x_p W_r, W_r = per-product tensors (stride V), p in {0, 1}
cudaError_t accumulate(cudaStream_t s, const int d[3], int p, const double* A, int R, const double* W, double* y) {
  const long V = (long)d[0] * d[1] * d[2];
  attn::GemmF64 g;
  g.beta = 1.0;
  g.G = R;
  if (p == 0) {
    g.M = d[0]; g.N = d[1] * d[2]; g.K = d[0];
    g.A = A; g.aM = d[0]; g.aK = 1; g.aG = (long)d[0] * d[0];
    g.B = W; g.bK = (long)d[1] * d[2]; g.bN = 1; g.bG = V;
    g.C = y; g.cM = (long)d[1] * d[2]; g.cN = 1;
  } else {
    g.M = d[1]; g.N = d[2]; g.K = d[1];
    g.A = A; g.aM = d[1]; g.aK = 1; g.aG = (long)d[1] * d[1];
    g.B = W; g.bK = d[2]; g.bN = 1; g.bG = V; g.bBlo = (long)d[1] * d[2];
    g.C = y; g.cM = d[2]; g.cN = 1; g.cBlo = (long)d[1] * d[2];
    g.Blo = d[0];
  }
  return attn::gemm_f64_stream(s, g);
}

}  // namespace

#define NA_TRY(expr)                                                                         \
  do {                                                                                       \
    cudaError_t _e = (expr);                                                                 \
    if (_e != cudaSuccess) {                                                                 \
      attn::set_error("%s: %s", #expr, cudaGetErrorString(_e));                              \
      return ATTN_ECUDA;                                                                     \
    }                                                                                        \
  } while (0)

extern "C" ATTN_API attn_status attn_heff_apply_f64_static(const attn_heff_desc* d, const double* x, double* y,
                                                           void* cuda_stream) {
  static const int kP[3] = {0, 0, 1}, kQ[3] = {1, 2, 2};
  if (!d || !x || !y) {
    attn::set_error("desc, x_dev and y_dev must be non-NULL");
    return ATTN_EINVAL;
  }
  if (x == y) {
    attn::set_error("x and y must be distinct buffers");
    return ATTN_EINVAL;
  }
  for (int s = 0; s < 3; ++s)
    if (d->m[s] < 1 || d->m[s] > 4096) {
      attn::set_error("link dimension must be 1..4096");
      return ATTN_EINVAL;
    }
  const long V = (long)d->m[0] * d->m[1] * d->m[2];
  const long need = (d->n_triple > 0) ? 2 * V : V;
  if (need > kScratchDoubles) {
    attn::set_error("allocation-free H_eff: a [%d,%d,%d] tensor needs %ld scratch doubles but the static scratch "
                    "holds %ld (limit m0*m1*m2 <= %ld, or half of it with three-link products)",
                    d->m[0], d->m[1], d->m[2], need, kScratchDoubles, kScratchDoubles);
    return ATTN_EINVAL;
  }
  for (int k = 0; k < 3; ++k)
    if (d->n_pair[k] < 0 || (d->n_pair[k] > 0 && (!d->pair_a[k] || !d->pair_b[k]))) {
      attn::set_error("pair kind %d: negative count or NULL operator array", k);
      return ATTN_EINVAL;
    }
  if (d->n_triple < 0 || (d->n_triple > 0 && (!d->triple[0] || !d->triple[1] || !d->triple[2]))) {
    attn::set_error("negative triple count or NULL operator array");
    return ATTN_EINVAL;
  }
  double* W = nullptr;
  NA_TRY(scratch_address(&W));
  cudaStream_t s = (cudaStream_t)cuda_stream;
  const int dm[3] = {d->m[0], d->m[1], d->m[2]};
  // y starts at zero; the scratch is always fully written before it is read
  NA_TRY(attn::fill_f64_stream(s, y, (size_t)V, 0.0));
  for (int l = 0; l < 3; ++l)
    if (d->h_int[l]) NA_TRY(mode_product(s, dm, l, d->h_int[l], 1, x, 0, y, 1.0));
  const int chunk = (int)std::max<long>(1, std::min<long>(4096, kScratchDoubles / V));
  for (int k = 0; k < 3; ++k) {
    const int p = kP[k], q = kQ[k];
    for (int r0 = 0; r0 < d->n_pair[k]; r0 += chunk) {
      const int R = std::min(chunk, d->n_pair[k] - r0);
      NA_TRY(mode_product(s, dm, q, d->pair_b[k] + (long)r0 * dm[q] * dm[q], R, x, 0, W, 0.0));
      NA_TRY(accumulate(s, dm, p, d->pair_a[k] + (long)r0 * dm[p] * dm[p], R, W, y));
    }
  }
  const int tchunk = (int)std::max<long>(1, std::min<long>(4096, kScratchDoubles / (2 * V)));
  for (int r0 = 0; r0 < d->n_triple; r0 += tchunk) {
    const int R = std::min(tchunk, d->n_triple - r0);
    double* W1 = W;
    double* W2 = W + (long)R * V;
    NA_TRY(mode_product(s, dm, 2, d->triple[2] + (long)r0 * dm[2] * dm[2], R, x, 0, W1, 0.0));
    NA_TRY(mode_product(s, dm, 1, d->triple[1] + (long)r0 * dm[1] * dm[1], R, W1, V, W2, 0.0));
    NA_TRY(accumulate(s, dm, 0, d->triple[0] + (long)r0 * dm[0] * dm[0], R, W2, y));
  }
  attn::clear_error();
  return ATTN_OK;
}
