/*
 * attn.h -- C ABI of the GB300 aTTN ground-state-search library (libattn.so).
 *
 * The library implements the hot path of the augmented tree tensor network
 * (aTTN) ground-state search of "The Augmented Tree Tensor Network Cookbook"
 * (Reinic, Pavesic, Jaschke, Montangero, arXiv:2507.21236):
 *   - effective Hamiltonian H_eff of one binary-TTN tensor as a sum over
 *     tensor-product-operator (TPO) terms (Sec. 3.3.2, Fig. eff-op) and its
 *     application to the order-3 tensor inside Lanczos (Sec. 4.4.2,
 *     Fig. eff-op-cost);
 *   - renormalisation T^T (O (x) O) T of link operators (Fig. eff-op);
 *   - Lanczos local eigensolver, QR re-isometrisation (Sec. 3.1, Fig. iso);
 *   - disentangler placement (Sec. 6.1), the mapping H' = D^T H D
 *     (Sec. 4.3, Algorithm 1) and the MERA-like update (Sec. 4.1.1);
 *   - the sweep schedule (Sec. 4).
 * Every compute step runs in the library's own CUDA kernels for sm_103a on
 * one GPU. There is no CPU fallback: without a usable GPU every compute call
 * returns ATTN_ECUDA.
 *
 * Conventions (all entry points):
 *  - Status: every call returns attn_status; ATTN_OK == 0. On failure a
 *    thread-local message is available from attn_last_error(). No C++
 *    exception crosses this boundary.
 *  - Streams: a context owns one CUDA stream (given at creation, or its own).
 *    Device work is enqueued on it. Calls that return host scalars
 *    (eigenvalues, energies) or copy to host synchronise that stream only.
 *  - Ownership: handles (attn_ctx, attn_model, attn_state, attn_heff) are
 *    created and destroyed by the library; all device memory they hold is
 *    allocated with cudaMalloc and freed by the matching destroy call.
 *    Pointers passed in (x_dev, y_dev, host arrays) stay owned by the caller
 *    and are never freed or retained after the call returns.
 *  - Layout: a node tensor is a C-contiguous FP64 array T[m0][m1][m2] with
 *    slot 0 = left child link, slot 1 = right child link, slot 2 = parent
 *    link (the top link for the two top tensors). Link operators are
 *    row-major FP64 m x m matrices O[out][in] acting on a link index.
 *  - Sites are numbered along the Hilbert curve (Sec. 6); a node of layer l
 *    covers 2^l consecutive sites.
 */
#ifndef ATTN_H
#define ATTN_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define ATTN_API __attribute__((visibility("default")))

typedef enum {
  ATTN_OK = 0,
  ATTN_EINVAL = 1,         /* bad argument, shape or state (message says which) */
  ATTN_ENOMEM = 2,         /* device or host allocation failed */
  ATTN_ECUDA = 3,          /* CUDA runtime error, or no usable GPU */
  ATTN_ENONFINITE = 4,     /* NaN/Inf found in an input or a result */
  ATTN_ENOTISOMETRIC = 5,  /* a tensor that must be an isometry is not */
  ATTN_ENOTCONVERGED = 6,  /* an iteration stopped before its tolerance; best result kept */
  ATTN_ETIMEOUT = 7,       /* a bounded device-side wait gave up */
  ATTN_EUNSUPPORTED = 8    /* shape/dtype combination not implemented */
} attn_status;

typedef enum {
  ATTN_F64 = 0,  /* FP64 contractions (CUDA cores, or exact BF16 slice products with f64_split) */
  ATTN_F32 = 1,  /* reserved */
  ATTN_TF32 = 2, /* TF32 operands (FP32 rounded to 10 mantissa bits), FP32 accumulation on the tcgen05 tensor cores */
  ATTN_BF16 = 3  /* BF16 operands, FP32 accumulation on the tcgen05 tensor cores */
} attn_dtype;

typedef struct attn_ctx attn_ctx;
typedef struct attn_model attn_model;
typedef struct attn_state attn_state;
typedef struct attn_heff attn_heff;
typedef struct attn_mlp attn_mlp;

/* Run parameters. attn_config_default fills the paper's/our defaults. */
typedef struct {
  int lanczos_depth;        /* Krylov depth of the local eigensolver (20) */
  double lanczos_tol;       /* stop when beta_k |y_k| < tol |theta| (1e-13) */
  int de_max_iter;          /* MERA-like update iterations, Sec. 4.1.1 (20) */
  double de_rel_dev;        /* relative energy change that stops them (1e-12) */
  int s_ttn;                /* sweeps without disentangler optimisation, Sec. 6.3 (1) */
  attn_dtype matvec_dtype;  /* precision of the H_eff contractions in Lanczos: ATTN_F64, ATTN_TF32 or ATTN_BF16;
                               nodes with a link the tensor-core tiles cannot take use FP64 (ATTN_F64) */
  int refine_steps;         /* FP64 corrections (one FP64 matvec each) after a low-precision Lanczos (3) */
  double refine_tol;        /* stop refining when ||H v - theta v|| < tol |theta| or a correction
                               lowers theta by at most tol |theta| (1e-10) */
  int use_graphs;           /* attn_eigsolve replays a captured CUDA graph of the low-precision Lanczos (0) */
  int refine_inner;         /* conjugate-gradient steps of the low-precision H_eff per correction, solving the
                               Jacobi-Davidson correction equation; 0 = the residual itself (16) */
  int f64_split;            /* FP64 contractions of H_eff applications, renormalisation and disentangler
                               environments as exact BF16 slice products on the tensor cores (Ozaki
                               scheme, 47-bit operand slices): normwise error about (K + 2) 2^-46 of the
                               operands' row scales, K the contraction length; QR stays on FP64 FMAs (0) */
  int report_unconverged;   /* attn_eigsolve returns ATTN_ENOTCONVERGED (results still written) when the
                               Lanczos residual or the refinement stopped above its tolerance (0) */
  int wait_limit_log2;      /* consumer-side wait limit of the tensor-core H_eff kernel, 2^k clock cycles;
                               0 = the default of about 2 s. A short limit makes the kernel give up,
                               drain its copies and report ATTN_ETIMEOUT: for testing failure handling (0) */
  int compress_terms;       /* sum the mapped terms of H' that act on the same sites into one term before the
                               rank-1 split (the compression of Sec. 6.2.2: the xx, yy and zz terms of a bond
                               mapped through one disentangler give one term of bond dimension <= d^2 instead of
                               three); the same linear map with fewer products (0) */
  int de_method;            /* disentangler optimisation: 0 = MERA-like self-consistent update (Sec. 4.1.1),
                               1 = Riemannian conjugate gradients of the true E_k on O(4) (Sec. 4.1.2) (0) */
  int tc_schedule;          /* grid of the tensor-core H_eff kernel: 0 = chosen by timing at the first
                               application (the split grid or the persistent form, whichever is faster), 1 =
                               split grid (one CTA per slice pair and product range), 2 = persistent (one CTA per
                               SM over a cost-balanced cut of the node's products). Results agree to FP32
                               rounding either way (0) */
  int lanczos_basis;        /* Krylov basis and CGS2 reorthogonalisation of a Lanczos with BF16 or TF32 matvecs:
                               0 = FP64 (the Lanczos recurrence, its reorthogonalisation and the Ritz solve all
                               in FP64), 1 = FP32 basis and FP32 reorthogonalisation (recurrence scalars, matvec
                               vectors and Ritz vector stay FP64; depth <= 24; a faster option whose vectors
                               carry FP32 accuracy, which the FP64 refinement then lifts) (0) */
} attn_config;

ATTN_API attn_status attn_config_default(attn_config* cfg);

/* Last error message of the calling thread ("" if none). Valid until the next call. */
ATTN_API const char* attn_last_error(void);

/* Library version string. */
ATTN_API const char* attn_version(void);

/* ----------------------------------------------------------------- context */

/* Create a context on the current CUDA device. cuda_stream is a cudaStream_t
 * on which all of the context's work is enqueued (NULL: the legacy default
 * stream, which is also what PyTorch's default stream reports). cfg may be
 * NULL (defaults). */
ATTN_API attn_status attn_create(const attn_config* cfg, void* cuda_stream, attn_ctx** out);
ATTN_API attn_status attn_destroy(attn_ctx* ctx);
ATTN_API attn_status attn_set_config(attn_ctx* ctx, const attn_config* cfg);
ATTN_API attn_status attn_get_config(attn_ctx* ctx, attn_config* cfg);
/* Block until all work enqueued by the context has finished; ATTN_ETIMEOUT if a
 * bounded wait in the split FP64 GEMM gave up meanwhile (its error word is then cleared). */
ATTN_API attn_status attn_sync(attn_ctx* ctx);
/* Device memory from the caller (e.g. a framework's caching allocator). After
 * attn_set_allocator(alloc, free, user) every device buffer the library allocates
 * -- handle storage and the contexts' scratch -- comes from alloc(bytes, device,
 * user), which must return a 256-byte aligned block of at least `bytes` on the
 * current device (or NULL: the call fails with ATTN_ENOMEM), and goes back through
 * free(ptr, bytes, device, user) of the allocator that served it, after the library
 * has synchronised the device (as cudaFree would). (NULL, NULL, NULL) restores
 * cudaMalloc/cudaFree. The setting is process-wide and applies to allocations made
 * after the call; buffers allocated before it are returned to where they came
 * from. Install it before creating contexts; the callbacks may be called from any
 * library call until every handle is destroyed. The allocation-free entry point
 * attn_heff_apply_f64_static never allocates and is unaffected. No counterpart in
 * the paper: ownership of device memory is the host framework's. */
typedef void* (*attn_alloc_fn)(size_t bytes, int device, void* user);
typedef void (*attn_free_fn)(void* ptr, size_t bytes, int device, void* user);
ATTN_API attn_status attn_set_allocator(attn_alloc_fn alloc, attn_free_fn free_fn, void* user);

/* Number of library kernels launched by this context so far. */
ATTN_API attn_status attn_kernel_launches(attn_ctx* ctx, uint64_t* count);
/* Timing for measurement tools. enable != 0 clears the records and makes the
 * library bracket each launch of its main kernels, and each phase of a local
 * step, with a CUDA event pair on the context stream. kernel_id: 0 = tensor-core
 * H_eff kernel, 1 = FP64 contraction kernel, 2 = tensor-core GEMM kernel,
 * 3 = split FP64 GEMM (slicing and products); phases: 4 = centre moves (QR),
 * 5 = H_eff builds (renormalisation of the node's link operators, operator
 * stacks), 6 = Lanczos, 7 = FP64 energy and refinement, 8 = disentangler updates.
 * attn_profile_read waits for the last recorded event and returns the summed
 * stream time (ms, for a phase including any idle gaps between its launches),
 * the number of recorded launches or phases and, for kernels, their algorithmic
 * FLOPs (Sec. 4.4.2 counting: 2 m_l V per operator applied on link l of a tensor
 * of V entries). */
ATTN_API attn_status attn_profile_enable(attn_ctx* ctx, int enable);
ATTN_API attn_status attn_profile_read(attn_ctx* ctx, int kernel_id, double* total_ms, int* launches, double* flops);

/* ------------------------------------------------------------------ models */

/* L x L open square lattice, H = -sum_<ij> Z_i Z_j - h sum_i X_i
 * (Sec. 6, Eq. qising, in the coupling-on-Z form; same spectrum). L a power of two. */
ATTN_API attn_status attn_model_tfim(attn_ctx* ctx, int L, double h, attn_model** out);
/* L x L open triangular lattice (square plus (+1,+1) bonds),
 * H = J sum_<ij> (Sx Sx + Sy Sy + Sz Sz) with S = sigma/2 (Sec. 6, Eq. xxz);
 * three separate terms per bond. */
ATTN_API attn_status attn_model_tri_heisenberg(attn_ctx* ctx, int L, double J, attn_model** out);
/* Generic Hamiltonian on n_sites spin-1/2 sites (n_sites a power of two >= 4):
 * term t acts on term_nsites[t] in {1,2,3} ascending sites
 * term_sites[3t .. 3t+nsites-1] with the real operator
 * term_ops[64t ...] stored row-major as a (2^k x 2^k) matrix, first site most
 * significant. One-site terms on the same site are summed (Sec. 3.3).
 * n_bonds/bond_sites list the candidate disentangler pairs (NULL: the
 * two-site terms). */
ATTN_API attn_status attn_model_terms(attn_ctx* ctx, int n_sites, int n_terms, const int* term_nsites,
                                      const int* term_sites, const double* term_ops, attn_model** out);
ATTN_API attn_status attn_model_destroy(attn_model* model);
ATTN_API attn_status attn_model_info(const attn_model* model, int* n_sites, int* n_terms);

/* ------------------------------------------------------------------- state */

/* Build a TTN with bond dimension m for the model's sites (Sec. 3.1): nodes
 * numbered layer by layer from the bottom, tensors [c0][c1][parent] with link
 * above a layer-l node of dimension min(2^(2^l), m). raw_host[n] points to
 * the raw FP64 entries of node n (shape from attn_node_shape, C order); each
 * non-centre tensor is replaced by the Q factor of its (c0 c1) x parent QR
 * (R's diagonal >= 0) and the centre (left top node) is normalised -- on the
 * GPU. Disentanglers start empty (none placed). */
ATTN_API attn_status attn_state_create(attn_ctx* ctx, const attn_model* model, int m,
                                       const double* const* raw_host, attn_state** out);
ATTN_API attn_status attn_state_destroy(attn_state* st);
/* n_nodes, centre node, number of layers nL. Any pointer may be NULL. */
ATTN_API attn_status attn_state_info(attn_state* st, int* n_nodes, int* centre, int* n_layers);
ATTN_API attn_status attn_node_shape(attn_state* st, int node, int shape[3]);
/* Neighbour of (node, slot): *kind = 0 site (index in *idx), 1 node (*idx, *back slot there). */
ATTN_API attn_status attn_node_neighbour(attn_state* st, int node, int slot, int* kind, int* idx, int* back);
/* Copy node tensor to/from host (synchronous). Setting a tensor invalidates
 * the effective operators that depend on it. */
ATTN_API attn_status attn_node_get(attn_state* st, int node, double* host_out);
ATTN_API attn_status attn_node_set(attn_state* st, int node, const double* host_in);
/* Device pointer of a node tensor, for reading (valid until the state is destroyed or
 * the centre moves through the node). Change a tensor with attn_node_set, which
 * invalidates the effective operators and the cached state energy that depend on it. */
ATTN_API attn_status attn_node_device_ptr(attn_state* st, int node, double** dev_ptr);
/* Move the isometry centre along the tree path with one QR per link (Fig. iso). */
ATTN_API attn_status attn_move_centre(attn_state* st, int node);
/* max ||T^T T - 1|| over non-centre tensors (towards the centre). */
ATTN_API attn_status attn_isometry_error(attn_state* st, double* err);

/* Renormalise the effective operators across the link `slot` of `node` (Fig.
 * eff-op, Fig. iso): the isometry centre moves to the neighbour n' on that link
 * (one QR per link crossed; node must not be a lowest-layer tensor's site link),
 * and the operators of every rank-1 product of H' with sites behind node, as seen
 * from n', are built from node's two other links by O_out = T^T (O_x (x) O_y) T:
 * products that lie entirely behind the link are summed into one internal
 * operator, the others stay open (one operator each). *n_open (may be NULL)
 * receives the number of open products. Requires attn_map_hamiltonian. */
ATTN_API attn_status attn_renormalise(attn_state* st, int node, int slot, int* n_open);
/* Effective operators of link (node, slot) as seen from node (computed if stale;
 * the isometry centre must not lie behind that link): *dim the link dimension,
 * *n_open the number of open products, *has_internal whether an internal operator
 * exists; h_int (may be NULL) receives the internal operator (dim x dim row-major,
 * zeros if none). Synchronous. */
ATTN_API attn_status attn_link_operators(attn_state* st, int node, int slot, int* dim, int* n_open,
                                         int* has_internal, double* h_int);

/* --------------------------------------------------------------- persistence */

/* Write / read everything a run resumes from: tensors, isometry centre,
 * disentangler placement and matrices, sweep count, the known FP64 energy and the
 * learned-start records (binary file, FP64 little-endian; the model is not stored,
 * only a fingerprint of its terms). attn_state_load reads into a state of the same
 * model and bond dimension (ATTN_EINVAL on any mismatch); effective operators are
 * rebuilt on demand, so a resumed run repeats the original one's arithmetic. */
ATTN_API attn_status attn_state_save(attn_state* st, const char* path);
ATTN_API attn_status attn_state_load(attn_state* st, const char* path);

/* ------------------------------------------------------------ disentanglers */

/* Greedy placement of Sec. 6.1.2 under the restrictions of Sec. 6.1.1, up to
 * max_de pairs; *n_placed receives the number actually placed. Replaces any
 * previous placement; all disentanglers start as the identity (Sec. 6). */
ATTN_API attn_status attn_de_place(attn_state* st, int max_de, int* n_placed);
/* Sites (i < j) of every placed disentangler, 2 ints each. */
ATTN_API attn_status attn_de_sites(attn_state* st, int* pairs_out);
/* Set / get the 4x4 orthogonal matrix u_k (row-major, site i most significant). */
ATTN_API attn_status attn_de_set(attn_state* st, int k, const double* u16);
ATTN_API attn_status attn_de_get(attn_state* st, int k, double* u16);
/* Map the Hamiltonian through the disentangler layer, H' = D^T H D
 * (Sec. 4.3, Algorithm 1), and split the mapped terms into rank-1 products.
 * All effective operators are invalidated; they are rebuilt on the GPU on
 * demand (Sec. 3.3.2) by the calls that need them. */
ATTN_API attn_status attn_map_hamiltonian(attn_state* st);
/* Number of mapped terms and rank-1 products of the current H'. */
ATTN_API attn_status attn_hamiltonian_info(attn_state* st, int* n_terms, int* n_products);
/* Structure of H_eff at `node` (host bookkeeping only, no device work): the
 * number of rank-1 products of H' spanning link pairs (0,1), (0,2), (1,2),
 * all three links, and lying behind a single link (summed into that link's
 * internal operator), in counts[0..4]. Requires attn_map_hamiltonian. */
ATTN_API attn_status attn_heff_counts(attn_state* st, int node, int counts[5]);

/* -------------------------------------------------------------------- H_eff */

/* Explicit description of a node's effective Hamiltonian (the summed-link
 * form of Sec. 3.3.2): with x[a][b][c] of shape (m[0], m[1], m[2]),
 *   y = sum_l H_l x_l x                                  (h_int[l], may be NULL)
 *     + sum_{k} sum_r (A_r on slot p_k)(B_r on slot q_k) x   (pair kinds k:
 *                                     0 = slots (0,1), 1 = (0,2), 2 = (1,2))
 *     + sum_r (O0_r (x) O1_r (x) O2_r) x                 (three-link products).
 * All operator arrays are DEVICE FP64, row-major; pair_a[k] is [n_pair[k]][m_p][m_p],
 * pair_b[k] is [n_pair[k]][m_q][m_q], triple[l] is [n_triple][m_l][m_l]. The
 * library copies them at creation (the caller may free them afterwards). */
typedef struct {
  int m[3];
  const double* h_int[3];
  int n_pair[3];
  const double* pair_a[3];
  const double* pair_b[3];
  int n_triple;
  const double* triple[3];
} attn_heff_desc;

ATTN_API attn_status attn_heff_create(attn_ctx* ctx, const attn_heff_desc* desc, attn_heff** out);
/* H_eff of `node` built from the state's effective operators (Sec. 3.3.2):
 * the isometry centre must be at `node` (ATTN_EINVAL otherwise). */
ATTN_API attn_status attn_heff_build(attn_state* st, int node, attn_heff** out);
ATTN_API attn_status attn_heff_destroy(attn_heff* h);
/* Counts: n_pair[3], n_triple, and the algorithmic FLOPs of one apply. */
ATTN_API attn_status attn_heff_info(attn_heff* h, int n_pair[3], int* n_triple, double* flops);
/* y_dev = H_eff x_dev (both DEVICE FP64 [m0][m1][m2], distinct buffers),
 * contractions in `dtype`: ATTN_F64 (its larger contractions as exact BF16 slice
 * products when the context's f64_split is set), or ATTN_BF16 / ATTN_TF32 operands
 * with FP32 accumulation on the tensor cores, which need every link dimension in
 * {16, 32, ..., 128} (ATTN_EUNSUPPORTED otherwise). Asynchronous on the context
 * stream. */
ATTN_API attn_status attn_heff_apply(attn_heff* h, const double* x_dev, double* y_dev, attn_dtype dtype);
/* Same with host buffers: copies x in, applies, copies y out (synchronous). */
ATTN_API attn_status attn_heff_apply_host(attn_heff* h, const double* x_host, double* y_host, attn_dtype dtype);

/* Allocation-free variant of attn_heff_create + attn_heff_apply(ATTN_F64).
 * The paper has no counterpart: this is for callers that cannot allocate
 * device memory -- a host framework may have reserved all free device memory
 * for its own pool and forbid raw cudaMalloc, or latency-critical code must
 * not pay the device-wide synchronisation of cudaFree. y_dev = H_eff x_dev
 * with the operators read in place from the DEVICE arrays of `desc`
 * (same layout as attn_heff_create), enqueued on cuda_stream (NULL: legacy
 * default stream). It calls no cudaMalloc or cudaFree; its only scratch is a
 * file-scope device array of ATTN_NOALLOC_SCRATCH_DOUBLES doubles (16 MiB) that
 * a GPU holds, once committed, until the process exits. Limits: m0*m1*m2 <=
 * ATTN_NOALLOC_SCRATCH_DOUBLES, or half of it when n_triple > 0; larger sizes
 * return ATTN_EINVAL with a message. The first call on each device looks up
 * the scratch array's device address (with that device current). CUDA loads a
 * library's device code lazily by default, so that first call is also when the
 * 16 MiB are committed on the device: make it before the framework reserves
 * its memory pool (or run with CUDA_MODULE_LOADING=EAGER, which commits the
 * array when the library is loaded), and before any stream capture. Every
 * call shares the one array, which keeps the last call's contents: calls
 * whose work overlaps on the GPU (other streams, other threads on the same
 * device) race and must be serialised by the caller. */
#define ATTN_NOALLOC_SCRATCH_DOUBLES (1L << 21)
ATTN_API attn_status attn_heff_apply_f64_static(const attn_heff_desc* desc, const double* x_dev, double* y_dev,
                                                void* cuda_stream);

/* Lowest eigenpair of H_eff by Lanczos (Sec. 4.4.2) started from T_dev
 * (device [m0][m1][m2]); on return T_dev holds the unit-norm Ritz vector and
 * *theta the Ritz value. Matvecs in the context's matvec_dtype; when that is
 * not FP64, refine_steps FP64 residual corrections follow. *iters may be NULL. */
ATTN_API attn_status attn_eigsolve(attn_heff* h, double* T_dev, double* theta, int* iters);
/* attn_eigsolve on a HOST tensor: T_host [m0][m1][m2] is copied to a device buffer
 * owned by h, solved there, and the Ritz vector copied back into T_host
 * (synchronous). */
ATTN_API attn_status attn_eigsolve_host(attn_heff* h, double* T_host, double* theta, int* iters);

/* ----------------------------------------------------------- sweep drivers */

/* Local optimisation at `node`: move the centre there, build H_eff, Lanczos,
 * write the tensor back if the Ritz value does not exceed the current energy. */
ATTN_API attn_status attn_local_step(attn_state* st, int node, double* energy);
/* One TTN sweep under the current H' (post-order, Sec. 4 step 3). */
ATTN_API attn_status attn_ttn_sweep(attn_state* st, double* energy);
/* Energy <T|H_eff|T> at the centre (FP64). */
ATTN_API attn_status attn_energy(attn_state* st, double* energy);

/* Update of every placed disentangler for the current TTN. The environments (the
 * TTN's reduced density matrices on each disentangler's terms, Sec. 4.2) are
 * contracted once on the GPU; all disentanglers are independent given the TTN
 * (restriction 1) and are updated in one batch, each by:
 *  - de_method 0 (default), the MERA-like update (Sec. 4.1.1, Eqs. contracted
 *    and cost function): Gamma_k with u^T fixed, u = -V W^T from the SVD
 *    Gamma_k = W sigma V^T, accepted while the true E_k does not increase; terms
 *    are shifted by their spectral norm (reading: the paper gives no shift);
 *  - de_method 1, Riemannian conjugate gradients of the true E_k(u) on O(4)
 *    (Sec. 4.1.2): Polak-Ribiere+ directions, QR retraction, Armijo steps;
 * up to de_max_iter steps or a relative change below de_rel_dev. *dE (may be
 * NULL) receives sum_k [E_k(new) - E_k(old)]. The mapped Hamiltonian is marked
 * stale. */
ATTN_API attn_status attn_de_update(attn_state* st, double* dE);
/* E_k before and after the last attn_de_update, 2 doubles per disentangler. */
ATTN_API attn_status attn_de_energies(attn_state* st, double* e_out);
/* The same update for disentangler k alone: its environments only, the others
 * unchanged (restriction 1 makes the updates independent). */
ATTN_API attn_status attn_de_update_one(attn_state* st, int k, double* dE);
/* Environment of disentangler k at a given orthogonal u (row-major 4 x 4): gamma16
 * receives Gamma_k with E = Tr(u Gamma_k) for u^T fixed at u (Eq. contracted, terms
 * shifted by their spectral norm), *e_k the true E_k(u) (Sec. 4.1.1). */
ATTN_API attn_status attn_de_environment(attn_state* st, int k, const double* u16, double* gamma16, double* e_k);
/* Two-site reduced density matrix of the TTN on disentangler k's sites (i, j),
 * row-major 4 x 4 with site i most significant: the environment the update and
 * the learned start read. */
ATTN_API attn_status attn_rdm2(attn_state* st, int k, double* rho16);

/* ------------------------------------------------------------- observables */

/* Expectation values <psi_aTTN| o |psi_aTTN> (Sec. 5, Eq. obs) of products of
 * one-site operators: observable q acts on nsites[q] in 1..4 distinct sites
 * sites[4q .. 4q+nsites[q]-1] with the real 2 x 2 operators ops[16q + 4a ..]
 * (row-major) on site a. Each is mapped through the disentangler layer (o' =
 * D^T o D, the Hamiltonian's convention: an observable on n sites spans at most
 * 2n after the mapping) and measured on the TTN. values receives n_obs doubles.
 * Synchronous. */
ATTN_API attn_status attn_measure(attn_state* st, int n_obs, const int* nsites, const int* sites, const double* ops,
                                  double* values);
/* Two-body correlation matrix of Eq. corrmat: C[i][j] = <o^a_i o^b_j> over all
 * sites (Hilbert order), the diagonal being <(o^a o^b)_i>; oa, ob are 2 x 2
 * row-major, C receives N x N doubles row-major. */
ATTN_API attn_status attn_correlation_matrix(attn_state* st, const double* oa, const double* ob, double* C);
/* One aTTN sweep (Sec. 4): if s_ttn sweeps have been done and disentanglers
 * are placed, update all disentanglers; map H -> H' if needed; then one TTN
 * sweep under H'. *energy receives the last local energy (= E of the state). */
ATTN_API attn_status attn_sweep(attn_state* st, double* energy);

/* ------------------------------------------------- learned disentangler start
 * Not in the paper (which starts every disentangler at the identity, Sec. 6):
 * an FP32 MLP 16 -> 128 -> 128 -> 16 (tanh) maps the two-site reduced density
 * matrix rho_ij of a disentangler (row-major 4 x 4, first site most
 * significant) to M; u = expm((M - M^T)/2). Parameters are one FP32 array:
 * W1[128][16] b1[128] W2[128][128] b2[128] W3[16][128] b3[16]. Training
 * minimises mean ||u - u_target||_F^2 with Adam; gradients pass through expm
 * by its Frechet derivative. */
ATTN_API attn_status attn_mlp_param_count(int* n);
ATTN_API attn_status attn_mlp_create(attn_ctx* ctx, const float* params_host, attn_mlp** out);
ATTN_API attn_status attn_mlp_destroy(attn_mlp* m);
ATTN_API attn_status attn_mlp_get_params(attn_mlp* m, float* params_out);
/* u_host[n][16] = expm(generator(rho_host[n][16])) */
ATTN_API attn_status attn_mlp_predict(attn_mlp* m, int n, const double* rho_host, double* u_host);
/* Loss and its gradient with respect to the parameters (grad_host may be NULL). */
ATTN_API attn_status attn_mlp_loss_grad(attn_mlp* m, int n, const double* rho_host, const double* u_target_host,
                                        double* loss, float* grad_host);
/* `steps` full-batch Adam steps (beta1 0.9, beta2 0.999, eps 1e-8) with rate lr. */
ATTN_API attn_status attn_mlp_train(attn_mlp* m, int n, const double* rho_host, const double* u_target_host,
                                    int steps, double lr, double* final_loss);
/* Attach a model (NULL detaches): the first disentangler update of the state
 * starts each u_k from the prediction, falling back to the plain start when
 * the prediction is non-finite or raises E_k (the plain method judges it).
 * The model must outlive its use by the state. */
ATTN_API attn_status attn_set_learned_init(attn_state* st, attn_mlp* m);
/* Training pairs of this run: rho_ij recorded at the first disentangler update
 * (16 doubles per disentangler) and the current u_k, with det(u) = -1 targets
 * replaced by u diag(1, 1, 1, -1) (unreachable by expm otherwise). */
ATTN_API attn_status attn_de_training_pairs(attn_state* st, double* rho_out, double* u_out);
/* How many disentanglers started from the prediction / fell back at the first update. */
ATTN_API attn_status attn_learned_init_report(attn_state* st, int* used, int* fallback);

#ifdef __cplusplus
}
#endif
#endif /* ATTN_H */
