// Lanczos and vector kernels (internal).
#pragma once

#include <functional>

#include "attn_internal.h"

namespace attn {

using MatVec = std::function<void(const double* x, double* y)>;

struct LanczosWork {
  DevBuf basis;  // block-interleaved Krylov basis (chunks of 256 elements, capacity depth + 1)
  DevBuf wvec, vk, scal;  // residual vector, contiguous copy of the newest basis vector, scalars
};

struct LanczosResult {
  double theta;
  int iters;
  double resid;
  bool converged;
};

// Lowest Ritz pair of the symmetric operator `apply` starting from x (device,
// length V). On return x holds the unit-norm Ritz vector. f32_basis: keep the Krylov
// basis and its reorthogonalisation in FP32 (for a low-precision `apply`, whose
// vectors carry no more; depth <= 24, else FP64 is used); the recurrence scalars,
// the matvec input and output and the Ritz vector stay FP64.
LanczosResult lanczos_lowest(attn_ctx* ctx, const MatVec& apply, double* x, long V, int depth, double tol,
                             LanczosWork& w, bool f32_basis = false);
// The same as a fixed launch sequence with no host synchronisation when
// host_check_every == 0 (capturable); lanczos_read waits and returns the result.
void lanczos_enqueue(attn_ctx* ctx, const MatVec& apply, double* x, long V, int depth, double tol, LanczosWork& w,
                     int host_check_every, bool f32_basis = false);
LanczosResult lanczos_read(attn_ctx* ctx, LanczosWork& w);

// Mixed-precision refinement of the lowest eigenpair after a low-precision
// Lanczos: FP64 Rayleigh-Ritz on a subspace grown by corrections from an
// approximate Jacobi-Davidson solve with `inner` conjugate-gradient steps of the
// low-precision operator (inner = 0: the residual itself). At most max_outer
// corrections (one FP64 matvec each); stops when ||H u - theta u|| < tol |theta|
// or when the last correction lowered theta by at most tol |theta|.
// On return x holds the unit Ritz vector u.
struct RefineResult {
  double theta;
  double resid;
  int outer;         // corrections made
  int fp64_matvecs;
  int lo_matvecs;
  bool converged;
};
struct RefineWork {
  DevBuf Vb, Wb, u, hu, r, t, res, p, q, C;
};
RefineResult refine_eig(attn_ctx* ctx, const MatVec& h64, const MatVec& hlo, double* x, long V, int max_outer,
                        int inner, double tol, RefineWork& w);

// out[i] = <basis_i, w> for i < nvec (deterministic two-pass reduction); accum[i] += out[i] if given.
void multi_dot(attn_ctx* ctx, const double* basis, int nvec, long V, const double* w, double* out, double* accum);
void multi_axpy_dev(attn_ctx* ctx, double* w, const double* basis, const double* coef, int nvec, long V, double sign);
void combine_dev(attn_ctx* ctx, double* out, const double* basis, const double* coef, int nvec, long V);
// dst = src / ||src||; nrm_sq_dev receives ||src||^2.
void normalise_dev(attn_ctx* ctx, double* dst, const double* src, long V, double* nrm_sq_dev);

}  // namespace attn
