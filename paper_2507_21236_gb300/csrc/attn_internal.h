// Internal declarations of libattn (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <cstdio>
#include <string>
#include <array>
#include <map>
#include <vector>

#include "attn.h"

namespace attn {

// ------------------------------------------------------------------ errors
void set_error(const char* fmt, ...);
void clear_error();
const char* last_error();

struct Error {
  attn_status status;
  std::string msg;
};

#define ATTN_CHECK_CUDA(expr)                                                                  \
  do {                                                                                         \
    cudaError_t _e = (expr);                                                                   \
    if (_e != cudaSuccess) {                                                                   \
      throw ::attn::Error{ATTN_ECUDA, std::string(#expr) + ": " + cudaGetErrorString(_e)};     \
    }                                                                                          \
  } while (0)

#define ATTN_REQUIRE(cond, status, msg)                                                        \
  do {                                                                                         \
    if (!(cond)) throw ::attn::Error{status, std::string(msg)};                                \
  } while (0)

// ------------------------------------------------------------ device memory
// Owning device buffer (cudaMalloc / cudaFree). A buffer that captured CUDA graphs
// may reference carries an epoch counter, bumped whenever the buffer is
// reallocated, so that graphs built on the old address can be detected.
// Device memory comes from cudaMalloc, or from the caller's allocator installed with
// attn_set_allocator; a buffer remembers which one served it and returns it there.
struct Allocator {
  attn_alloc_fn alloc = nullptr;
  attn_free_fn free = nullptr;
  void* user = nullptr;
};
const Allocator* current_allocator();  // nullptr: cudaMalloc / cudaFree
void set_allocator(attn_alloc_fn alloc, attn_free_fn free_fn, void* user);

struct DevBuf {
  void* p = nullptr;
  size_t bytes = 0;
  uint64_t* epoch = nullptr;  // not owned; bumped on every reallocation
  const Allocator* from = nullptr;  // allocator that served p (nullptr: cudaMalloc)
  DevBuf() = default;
  DevBuf(const DevBuf&) = delete;
  DevBuf& operator=(const DevBuf&) = delete;
  DevBuf(DevBuf&& o) noexcept : p(o.p), bytes(o.bytes), from(o.from) { o.p = nullptr; o.bytes = 0; }
  DevBuf& operator=(DevBuf&& o) noexcept {
    if (this != &o) {
      release();
      p = o.p; bytes = o.bytes; from = o.from;
      o.p = nullptr; o.bytes = 0;
    }
    return *this;
  }
  ~DevBuf() { release(); }
  void release();
  // Ensure capacity >= n bytes (contents not preserved on growth).
  void reserve(size_t n);
  template <class T> T* as() const { return static_cast<T*>(p); }
};

}  // namespace attn

// ------------------------------------------------------------------ context
struct attn_ctx {
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  attn_config cfg{};
  uint64_t launches = 0;
  int device = 0;
  int num_sms = 0;
  // Scratch areas reused across calls (grow only). Every reallocation of one of
  // them bumps scratch_epoch: a captured eigensolve graph records the epoch it was
  // built under and is rebuilt when it differs (its kernels hold the old addresses).
  uint64_t scratch_epoch = 0;
  attn::DevBuf ws[4];
  attn::DevBuf scal;      // small device scalars
  attn::DevBuf partials;  // reduction partials (fixed size, allocated at creation)
  attn::DevBuf gsplit_ws; // partial outputs of FP64 GEMMs whose reduction is split over CTA groups
  attn::DevBuf oz_ws[4];  // split-GEMM operand slices and row exponents (P slices, P exps, Q slices, Q exps)
  attn::DevBuf oz_err;    // split-GEMM device error word
  bool oz_err_init = false;
  // Optional per-kernel timing (attn_profile_enable): event pairs around launches.
  bool prof_on = false;
  struct ProfRec {
    std::vector<cudaEvent_t> ev;  // start/stop interleaved
    size_t used = 0;              // events in use (pairs * 2)
    double flops = 0.0;           // algorithmic FLOPs of the recorded launches
    int launches = 0;
    double acc_ms = 0.0;          // harvested from graph replays
    double acc_flops = 0.0;
    int acc_launches = 0;
  } prof[9];  // ids as documented at attn_profile_enable
  // While a CUDA graph is being captured, launch events go to this list
  // (kernel id, start, stop, FLOPs) instead of the pool above.
  struct GraphEv {
    int kid;
    cudaEvent_t a, b;
    double flops;
  };
  std::vector<GraphEv>* capture_events = nullptr;
  // Product split chosen for the tensor-core H_eff, by shape, products per kind and
  // operand type (m0, m1, m2, R0, R1, R2, tf32): sweeps rebuild H_eff at every local step.
  std::map<std::array<int, 7>, int> tc_split_cache;
  void prof_begin(int kid);
  void prof_end(int kid, double flops);
  ~attn_ctx();
};

namespace attn {

// ------------------------------------------------------- generic FP64 GEMM
// C[bh,bl][i][j] = beta*C + alpha * sum_{g<G} sum_{k<K} A[..][i][k] * B[..][k][j]
// with arbitrary element strides (all in elements).
struct GemmF64 {
  int M = 0, N = 0, K = 0, G = 1, Bhi = 1, Blo = 1;
  const double* A = nullptr;
  long aM = 0, aK = 0, aG = 0, aBhi = 0, aBlo = 0;
  const double* B = nullptr;
  long bK = 0, bN = 0, bG = 0, bBhi = 0, bBlo = 0;
  double* C = nullptr;
  long cM = 0, cN = 0, cBhi = 0, cBlo = 0;
  double alpha = 1.0, beta = 0.0;
  // split of the G reduction over gsplit CTA groups: group s sums its share of G
  // into C + s * cS (set by gemm_f64 when the output tiles alone underfill the GPU)
  int gsplit = 1;
  long cS = 0;
  // the contraction may run as exact BF16 slice products when attn_config.f64_split is set
  bool split_ok = false;
};
void gemm_f64(attn_ctx* ctx, const GemmF64& g);
// The same kernels launched on a bare stream (no context, no allocation).
cudaError_t gemm_f64_stream(cudaStream_t stream, const GemmF64& g);
cudaError_t fill_f64_stream(cudaStream_t stream, double* p, size_t n, double v);

// out[r] = mat_r x_slot in[r or shared] for a [m0][m1][m2] tensor; mats is a
// stack [R][m_s][m_s]; in_stride 0 shares one input, V for per-r inputs.
void mode_product_f64(attn_ctx* ctx, const int dims[3], int slot, const double* mats, int R,
                      const double* in, long in_stride, double* out, double beta);

// Small helper kernels.
void fill_f64(attn_ctx* ctx, double* p, size_t n, double v);
void copy_f64(attn_ctx* ctx, double* dst, const double* src, size_t n);
void axpy_f64(attn_ctx* ctx, double* y, const double* x, size_t n, double a);
// dst[i] = src_ptrs gathered: dst[r] = src + idx[r]*stride (each of len elements), idx on device
void gather_rows_f64(attn_ctx* ctx, double* dst, const double* src, const int* idx_dev, int R, long len);
void identity_stack_f64(attn_ctx* ctx, double* dst, int R, int m);
// Reductions.
void dot_f64(attn_ctx* ctx, const double* x, const double* y, size_t n, double* out_dev);

// ------------------------------------------------------------- host model
struct Term {
  int n = 0;
  int site[3] = {0, 0, 0};
  std::vector<double> op;  // (2^n)^2 row-major, first site most significant
};

// One rank-1 product of a mapped term: sum over these products equals H'.
struct Prod {
  int term = 0;
  int n = 0;
  int site[3] = {0, 0, 0};
  double op[3][4];  // one 2x2 matrix per site, row-major
};

struct Model {
  int n_sites = 0;
  std::vector<Term> terms;
  std::vector<std::pair<int, int>> bonds;  // candidate disentangler pairs (two-site terms)
};

struct Tree {
  int n_sites = 0, m = 0, nL = 0, n_nodes = 0;
  std::vector<int> layer, index, lo, hi;  // hi exclusive
  // neighbour of (node, slot): kind 0 = site, 1 = node
  struct Nbr { int kind, idx, back; };
  std::vector<Nbr> nbr;  // [node*3 + slot]
  std::vector<int> shape;  // [node*3 + slot]
  void build(int n_sites, int m);
  int id(int l, int j) const;
  int top0() const { return id(nL, 0); }
  int top1() const { return id(nL, 1); }
  int slot_towards(int n, int nb) const;
  std::vector<int> path(int a, int b) const;
  std::vector<int> post_order() const;
  int lca_layer(int i, int j) const;
  // is site s behind link (n, slot) as seen from n?
  bool behind(int n, int slot, int s) const;
};

void build_tfim(Model& M, int L, double h);
void build_tri_heisenberg(Model& M, int L, double J);
void build_generic(Model& M, int n_sites, int n_terms, const int* nsites, const int* sites, const double* ops);
void hilbert_d2xy(int n, int d, int* x, int* y);

std::vector<std::pair<int, int>> place_disentanglers(const Tree& T, const Model& M, int max_de);
std::vector<Term> map_terms(const Model& M, const std::vector<std::pair<int, int>>& des,
                            const std::vector<std::vector<double>>& us);
std::vector<Prod> split_products(const std::vector<Term>& terms);
// One term per distinct site set: the operators of terms on the same sites summed
// (same linear map, fewer rank-1 products after the split).
std::vector<Term> compress_terms(const std::vector<Term>& terms);

}  // namespace attn
