// Effective-Hamiltonian object (internal).
#pragma once

#include "attn_internal.h"
#include "lanczos.h"

// A captured CUDA graph of one eigensolve (Lanczos + optional FP64 refinement)
// on a fixed start-vector buffer; the buffers it uses are owned here.
struct EigGraph {
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  const double* x = nullptr;
  int depth = 0, dtype = 0, refine = 0, f64_split = 0, tc_schedule = 0, basis = 0;
  double tol = 0.0, rtol = 0.0;
  bool prof = false;
  uint64_t epoch = ~0ull;         // the context's scratch_epoch the graph was captured under
  uint64_t epoch_before = ~0ull;  // the same, read before the capture began
  uint64_t launches = 0;
  attn::LanczosWork w;
  attn::RefineWork rw;
  std::vector<attn_ctx::GraphEv> evs;
  ~EigGraph() {
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    for (auto& e : evs) {
      cudaEventDestroy(e.a);
      cudaEventDestroy(e.b);
    }
  }
};

// Pair kinds: 0 = slots (0,1) with slice slot 2; 1 = (0,2) slice 1; 2 = (1,2) slice 0.
static const int kPairP[3] = {0, 0, 1};
static const int kPairQ[3] = {1, 2, 2};
static const int kPairS[3] = {2, 1, 0};

struct attn_heff {
  attn_ctx* ctx = nullptr;
  int m[3] = {0, 0, 0};
  long V = 0;
  bool has_hint[3] = {false, false, false};
  attn::DevBuf hint[3];   // [m_l][m_l] FP64
  int npair[3] = {0, 0, 0};
  attn::DevBuf pa[3], pb[3];  // FP64 stacks [n][m_p][m_p], [n][m_q][m_q]
  int ntrip = 0;
  attn::DevBuf tr[3];     // FP64 stacks [n][m_l][m_l]
  // Low-precision tensor-core copies, built at the first application in that type:
  // tc[0] BF16 operands, tc[1] TF32 operands (opaque, owned by heff_tc.cu).
  void* tc[2] = {nullptr, nullptr};
  EigGraph* eg = nullptr; // cached eigensolve graph (use_graphs)
  attn::DevBuf host_x;    // device copy of the tensor of attn_eigsolve_host
  double flops() const;
  void apply_f64(const double* x, double* y);
  void apply_bf16(const double* x, double* y);
  void apply_tf32(const double* x, double* y);
  void apply_tc(const double* x, double* y, bool tf32);
  // contractions in `dt` (ATTN_F64, ATTN_BF16 or ATTN_TF32)
  void apply(const double* x, double* y, attn_dtype dt) {
    if (dt == ATTN_BF16) apply_bf16(x, y);
    else if (dt == ATTN_TF32) apply_tf32(x, y);
    else apply_f64(x, y);
  }
  ~attn_heff();
};

namespace attn {
void tc_release(attn_heff* h);
// Marks the tensor-core copies stale after the H_eff's operators were replaced: the
// next low-precision application rebuilds them into the same device buffers.
void tc_invalidate(attn_heff* h);
bool tc_supported(const attn_heff* h);
int tc_error(attn_heff* h);
// Throws ATTN_ETIMEOUT when a bounded wait in a tensor-core kernel gave up (the
// H_eff's tensor-core error word, if h is given, and the split FP64 GEMM's).
void check_device_errors(attn_ctx* ctx, attn_heff* h);
// Runs f(); if it throws, a device-side timeout recorded meanwhile is reported in
// its place (a kernel that gave up leaves its outputs unwritten, which the host
// may then see as non-finite values).
template <class F>
auto timeout_first(attn_ctx* ctx, attn_heff* h, F&& f) -> decltype(f()) {
  try {
    return f();
  } catch (const Error&) {
    check_device_errors(ctx, h);
    throw;
  }
}
// y += sum_{r<R} A_r x_p W_r with W_r per-product tensors (stride V), FP64.
void accumulate_slot_f64(attn_ctx* ctx, const int d[3], int p, const double* A, int R, const double* W, double* y);
}  // namespace attn
