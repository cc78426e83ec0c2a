// extern "C" entry points of libattn (see include/attn.h for the contract).
// Every entry point converts internal exceptions into an attn_status and a
// thread-local message; nothing throws across the boundary.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdarg>
#include <cstring>
#include <memory>

#include "heff.h"
#include "state.h"

namespace attn {

static thread_local std::string g_err;

void set_error(const char* fmt, ...) {
  char buf[1024];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_err = buf;
}
void clear_error() { g_err.clear(); }
const char* last_error() { return g_err.c_str(); }

// The allocator installed by attn_set_allocator. Records are never freed: a buffer
// keeps a pointer to the one that served it until the buffer is released.
static std::atomic<const Allocator*> g_allocator{nullptr};
const Allocator* current_allocator() { return g_allocator.load(); }
void set_allocator(attn_alloc_fn alloc, attn_free_fn free_fn, void* user) {
  if (!alloc) {
    g_allocator.store(nullptr);
    return;
  }
  g_allocator.store(new Allocator{alloc, free_fn, user});
}

void DevBuf::release() {
  if (p) {
    if (from) {
      // cudaFree waits for the device before it returns memory; a caller's allocator
      // may hand the block out again at once, so wait here for kernels still using it
      int dev = 0;
      cudaGetDevice(&dev);
      cudaDeviceSynchronize();
      from->free(p, bytes, dev, from->user);
    } else {
      cudaFree(p);
    }
  }
  p = nullptr;
  bytes = 0;
  from = nullptr;
}

void DevBuf::reserve(size_t n) {
  if (n <= bytes && p) return;
  release();
  if (epoch) ++*epoch;
  size_t want = std::max<size_t>(n, 256);
  const Allocator* a = current_allocator();
  if (a) {
    int dev = 0;
    ATTN_CHECK_CUDA(cudaGetDevice(&dev));
    p = a->alloc(want, dev, a->user);
    ATTN_REQUIRE(p != nullptr, ATTN_ENOMEM,
                 "the caller's allocator returned NULL for " + std::to_string(want) + " bytes");
    ATTN_REQUIRE(((uintptr_t)p & 255) == 0, ATTN_EINVAL, "the caller's allocator must return 256-byte aligned blocks");
    from = a;
  } else {
    cudaError_t e = cudaMalloc(&p, want);
    if (e != cudaSuccess) {
      p = nullptr;
      (void)cudaGetLastError();
      throw Error{ATTN_ENOMEM, std::string("cudaMalloc of ") + std::to_string(want) + " bytes failed: " +
                                   cudaGetErrorString(e)};
    }
  }
  bytes = want;
}

}  // namespace attn

void attn_ctx::prof_begin(int kid) {
  if (!prof_on) return;
  if (capture_events) {
    GraphEv g{kid, nullptr, nullptr, 0.0};
    ATTN_CHECK_CUDA(cudaEventCreate(&g.a));
    ATTN_CHECK_CUDA(cudaEventCreate(&g.b));
    // an external record becomes an event-record node that fires on every replay
    ATTN_CHECK_CUDA(cudaEventRecordWithFlags(g.a, stream, cudaEventRecordExternal));
    capture_events->push_back(g);
    return;
  }
  ProfRec& p = prof[kid];
  if (p.used + 2 > p.ev.size()) {
    cudaEvent_t a, b;
    ATTN_CHECK_CUDA(cudaEventCreate(&a));
    ATTN_CHECK_CUDA(cudaEventCreate(&b));
    p.ev.push_back(a);
    p.ev.push_back(b);
  }
  ATTN_CHECK_CUDA(cudaEventRecord(p.ev[p.used], stream));
}

void attn_ctx::prof_end(int kid, double flops) {
  if (!prof_on) return;
  if (capture_events) {
    GraphEv& g = capture_events->back();
    ATTN_CHECK_CUDA(cudaEventRecordWithFlags(g.b, stream, cudaEventRecordExternal));
    g.flops = flops;
    return;
  }
  ProfRec& p = prof[kid];
  ATTN_CHECK_CUDA(cudaEventRecord(p.ev[p.used + 1], stream));
  p.used += 2;
  p.flops += flops;
  p.launches += 1;
}

attn_ctx::~attn_ctx() {
  for (auto& p : prof)
    for (auto e : p.ev) cudaEventDestroy(e);
}

using namespace attn;

#define ATTN_TRY try {
#define ATTN_CATCH                                           \
  }                                                          \
  catch (const Error& e) {                                   \
    set_error("%s", e.msg.c_str());                          \
    return e.status;                                         \
  }                                                          \
  catch (const std::bad_alloc&) {                            \
    set_error("host allocation failed");                     \
    return ATTN_ENOMEM;                                      \
  }                                                          \
  catch (const std::exception& e) {                          \
    set_error("%s", e.what());                               \
    return ATTN_EINVAL;                                      \
  }                                                          \
  clear_error();                                             \
  return ATTN_OK;

#define NEED(p, what) ATTN_REQUIRE((p) != nullptr, ATTN_EINVAL, what " is NULL")

struct attn_model {
  attn_ctx* ctx;
  Model M;
};

extern "C" {

ATTN_API const char* attn_last_error(void) { return last_error(); }
ATTN_API const char* attn_version(void) { return "attn-gb300 0.1 (sm_103a)"; }

ATTN_API attn_status attn_config_default(attn_config* cfg) {
  ATTN_TRY
  NEED(cfg, "cfg");
  std::memset(cfg, 0, sizeof(*cfg));
  cfg->lanczos_depth = 20;
  cfg->lanczos_tol = 1e-13;
  cfg->de_max_iter = 20;
  cfg->de_rel_dev = 1e-12;
  cfg->s_ttn = 1;
  cfg->matvec_dtype = ATTN_F64;
  cfg->refine_steps = 3;
  cfg->refine_tol = 1e-10;
  cfg->refine_inner = 16;
  ATTN_CATCH
}

ATTN_API attn_status attn_create(const attn_config* cfg, void* stream, attn_ctx** out) {
  ATTN_TRY
  NEED(out, "out");
  *out = nullptr;
  int ndev = 0;
  cudaError_t e = cudaGetDeviceCount(&ndev);
  if (e != cudaSuccess || ndev == 0) {
    (void)cudaGetLastError();
    throw Error{ATTN_ECUDA, "no CUDA device available: the library has no CPU fallback"};
  }
  auto ctx = std::make_unique<attn_ctx>();
  if (cfg) ctx->cfg = *cfg; else attn_config_default(&ctx->cfg);
  ATTN_CHECK_CUDA(cudaGetDevice(&ctx->device));
  cudaDeviceProp prop;
  ATTN_CHECK_CUDA(cudaGetDeviceProperties(&prop, ctx->device));
  ATTN_REQUIRE(prop.major == 10 && prop.minor == 3, ATTN_ECUDA,
               std::string("libattn is built for sm_103a only; device is ") + prop.name);
  ctx->num_sms = prop.multiProcessorCount;
  // NULL selects the legacy default stream (what torch's default stream reports as 0)
  ctx->stream = stream ? (cudaStream_t)stream : (cudaStream_t)0;
  ctx->own_stream = false;
  for (DevBuf* b : {&ctx->ws[0], &ctx->ws[1], &ctx->ws[2], &ctx->ws[3], &ctx->scal, &ctx->partials,
                    &ctx->gsplit_ws, &ctx->oz_ws[0], &ctx->oz_ws[1], &ctx->oz_ws[2], &ctx->oz_ws[3], &ctx->oz_err})
    b->epoch = &ctx->scratch_epoch;
  ctx->partials.reserve(sizeof(double) * 512 * 64);
  ctx->scal.reserve(sizeof(double) * 64);
  *out = ctx.release();
  ATTN_CATCH
}

ATTN_API attn_status attn_destroy(attn_ctx* ctx) {
  ATTN_TRY
  if (!ctx) return ATTN_OK;
  cudaStreamSynchronize(ctx->stream);
  if (ctx->own_stream) cudaStreamDestroy(ctx->stream);
  delete ctx;
  ATTN_CATCH
}

ATTN_API attn_status attn_set_config(attn_ctx* ctx, const attn_config* cfg) {
  ATTN_TRY
  NEED(ctx, "ctx");
  NEED(cfg, "cfg");
  ATTN_REQUIRE(cfg->lanczos_depth >= 1 && cfg->lanczos_depth <= 60, ATTN_EINVAL, "lanczos_depth must be 1..60");
  ATTN_REQUIRE(cfg->matvec_dtype == ATTN_F64 || cfg->matvec_dtype == ATTN_BF16 || cfg->matvec_dtype == ATTN_TF32,
               ATTN_EUNSUPPORTED, "matvec_dtype must be ATTN_F64, ATTN_TF32 or ATTN_BF16");
  ATTN_REQUIRE(cfg->wait_limit_log2 >= 0 && cfg->wait_limit_log2 <= 62, ATTN_EINVAL, "wait_limit_log2 must be 0..62");
  ATTN_REQUIRE(cfg->de_method == 0 || cfg->de_method == 1, ATTN_EINVAL, "de_method must be 0 or 1");
  ATTN_REQUIRE(cfg->tc_schedule >= 0 && cfg->tc_schedule <= 2, ATTN_EINVAL, "tc_schedule must be 0, 1 or 2");
  ATTN_REQUIRE(cfg->lanczos_basis == 0 || cfg->lanczos_basis == 1, ATTN_EINVAL, "lanczos_basis must be 0 or 1");
  ctx->cfg = *cfg;
  ATTN_CATCH
}

ATTN_API attn_status attn_get_config(attn_ctx* ctx, attn_config* cfg) {
  ATTN_TRY
  NEED(ctx, "ctx");
  NEED(cfg, "cfg");
  *cfg = ctx->cfg;
  ATTN_CATCH
}

ATTN_API attn_status attn_sync(attn_ctx* ctx) {
  ATTN_TRY
  NEED(ctx, "ctx");
  ATTN_CHECK_CUDA(cudaStreamSynchronize(ctx->stream));
  check_device_errors(ctx, nullptr);
  ATTN_CATCH
}

ATTN_API attn_status attn_profile_enable(attn_ctx* ctx, int enable) {
  ATTN_TRY
  NEED(ctx, "ctx");
  ctx->prof_on = enable != 0;
  for (auto& p : ctx->prof) {
    p.used = 0;
    p.flops = 0.0;
    p.launches = 0;
    p.acc_ms = p.acc_flops = 0.0;
    p.acc_launches = 0;
  }
  ATTN_CATCH
}

ATTN_API attn_status attn_profile_read(attn_ctx* ctx, int kernel_id, double* total_ms, int* launches, double* flops) {
  ATTN_TRY
  NEED(ctx, "ctx");
  ATTN_REQUIRE(kernel_id >= 0 && kernel_id < 9, ATTN_EINVAL, "kernel_id must be 0..8");
  attn_ctx::ProfRec& p = ctx->prof[kernel_id];
  double tot = 0.0;
  if (p.used) ATTN_CHECK_CUDA(cudaEventSynchronize(p.ev[p.used - 1]));
  for (size_t i = 0; i + 1 < p.used; i += 2) {
    float ms = 0.f;
    ATTN_CHECK_CUDA(cudaEventElapsedTime(&ms, p.ev[i], p.ev[i + 1]));
    tot += ms;
  }
  if (total_ms) *total_ms = tot + p.acc_ms;
  if (launches) *launches = p.launches + p.acc_launches;
  if (flops) *flops = p.flops + p.acc_flops;
  ATTN_CATCH
}

ATTN_API attn_status attn_kernel_launches(attn_ctx* ctx, uint64_t* count) {
  ATTN_TRY
  NEED(ctx, "ctx");
  NEED(count, "count");
  *count = ctx->launches;
  ATTN_CATCH
}

// ------------------------------------------------------------------ models
ATTN_API attn_status attn_model_tfim(attn_ctx* ctx, int L, double h, attn_model** out) {
  ATTN_TRY
  NEED(ctx, "ctx");
  NEED(out, "out");
  auto m = std::make_unique<attn_model>();
  m->ctx = ctx;
  build_tfim(m->M, L, h);
  *out = m.release();
  ATTN_CATCH
}

ATTN_API attn_status attn_model_tri_heisenberg(attn_ctx* ctx, int L, double J, attn_model** out) {
  ATTN_TRY
  NEED(ctx, "ctx");
  NEED(out, "out");
  auto m = std::make_unique<attn_model>();
  m->ctx = ctx;
  build_tri_heisenberg(m->M, L, J);
  *out = m.release();
  ATTN_CATCH
}

ATTN_API attn_status attn_model_terms(attn_ctx* ctx, int n_sites, int n_terms, const int* nsites, const int* sites,
                                      const double* ops, attn_model** out) {
  ATTN_TRY
  NEED(ctx, "ctx");
  NEED(out, "out");
  ATTN_REQUIRE(n_terms >= 0, ATTN_EINVAL, "n_terms < 0");
  if (n_terms) {
    NEED(nsites, "term_nsites");
    NEED(sites, "term_sites");
    NEED(ops, "term_ops");
  }
  auto m = std::make_unique<attn_model>();
  m->ctx = ctx;
  build_generic(m->M, n_sites, n_terms, nsites, sites, ops);
  *out = m.release();
  ATTN_CATCH
}

ATTN_API attn_status attn_model_destroy(attn_model* model) {
  ATTN_TRY
  delete model;
  ATTN_CATCH
}

ATTN_API attn_status attn_model_info(const attn_model* model, int* n_sites, int* n_terms) {
  ATTN_TRY
  NEED(model, "model");
  if (n_sites) *n_sites = model->M.n_sites;
  if (n_terms) *n_terms = (int)model->M.terms.size();
  ATTN_CATCH
}

// ------------------------------------------------------------------- state
ATTN_API attn_status attn_state_create(attn_ctx* ctx, const attn_model* model, int m, const double* const* raw,
                                       attn_state** out) {
  ATTN_TRY
  NEED(ctx, "ctx");
  NEED(model, "model");
  NEED(raw, "raw_host");
  NEED(out, "out");
  auto st = std::make_unique<attn_state>();
  st->ctx = ctx;
  st->model = model->M;
  st->tree.build(model->M.n_sites, m);
  for (int n = 0; n < st->tree.n_nodes; ++n) {
    NEED(raw[n], "raw_host[node]");
    for (long i = 0; i < st->vol(n); ++i)
      ATTN_REQUIRE(std::isfinite(raw[n][i]), ATTN_ENONFINITE, "non-finite initial tensor entry");
  }
  st->init_from_raw(raw);
  ATTN_CHECK_CUDA(cudaStreamSynchronize(ctx->stream));
  *out = st.release();
  ATTN_CATCH
}

ATTN_API attn_status attn_state_destroy(attn_state* st) {
  ATTN_TRY
  if (!st) return ATTN_OK;
  cudaStreamSynchronize(st->ctx->stream);
  delete st;
  ATTN_CATCH
}

ATTN_API attn_status attn_state_info(attn_state* st, int* n_nodes, int* centre, int* n_layers) {
  ATTN_TRY
  NEED(st, "state");
  if (n_nodes) *n_nodes = st->tree.n_nodes;
  if (centre) *centre = st->centre;
  if (n_layers) *n_layers = st->tree.nL;
  ATTN_CATCH
}

ATTN_API attn_status attn_node_shape(attn_state* st, int node, int shape[3]) {
  ATTN_TRY
  NEED(st, "state");
  NEED(shape, "shape");
  ATTN_REQUIRE(node >= 0 && node < st->tree.n_nodes, ATTN_EINVAL, "node out of range");
  for (int s = 0; s < 3; ++s) shape[s] = st->dim(node, s);
  ATTN_CATCH
}

ATTN_API attn_status attn_node_neighbour(attn_state* st, int node, int slot, int* kind, int* idx, int* back) {
  ATTN_TRY
  NEED(st, "state");
  ATTN_REQUIRE(node >= 0 && node < st->tree.n_nodes && slot >= 0 && slot < 3, ATTN_EINVAL, "node/slot out of range");
  const Tree::Nbr& nb = st->tree.nbr[3 * node + slot];
  if (kind) *kind = nb.kind;
  if (idx) *idx = nb.idx;
  if (back) *back = nb.back;
  ATTN_CATCH
}

ATTN_API attn_status attn_node_get(attn_state* st, int node, double* host_out) {
  ATTN_TRY
  NEED(st, "state");
  NEED(host_out, "host_out");
  ATTN_REQUIRE(node >= 0 && node < st->tree.n_nodes, ATTN_EINVAL, "node out of range");
  ATTN_CHECK_CUDA(cudaMemcpyAsync(host_out, st->tensor(node), sizeof(double) * st->vol(node), cudaMemcpyDeviceToHost,
                                  st->ctx->stream));
  ATTN_CHECK_CUDA(cudaStreamSynchronize(st->ctx->stream));
  ATTN_CATCH
}

ATTN_API attn_status attn_node_set(attn_state* st, int node, const double* host_in) {
  ATTN_TRY
  NEED(st, "state");
  NEED(host_in, "host_in");
  ATTN_REQUIRE(node >= 0 && node < st->tree.n_nodes, ATTN_EINVAL, "node out of range");
  for (long i = 0; i < st->vol(node); ++i)
    ATTN_REQUIRE(std::isfinite(host_in[i]), ATTN_ENONFINITE, "non-finite tensor entry");
  ATTN_CHECK_CUDA(cudaMemcpyAsync(st->tensor(node), host_in, sizeof(double) * st->vol(node), cudaMemcpyHostToDevice,
                                  st->ctx->stream));
  ATTN_CHECK_CUDA(cudaStreamSynchronize(st->ctx->stream));
  st->invalidate_from(node);
  st->energy_known = std::nan("");
  ATTN_CATCH
}

ATTN_API attn_status attn_node_device_ptr(attn_state* st, int node, double** dev_ptr) {
  ATTN_TRY
  NEED(st, "state");
  NEED(dev_ptr, "dev_ptr");
  ATTN_REQUIRE(node >= 0 && node < st->tree.n_nodes, ATTN_EINVAL, "node out of range");
  *dev_ptr = st->tensor(node);
  ATTN_CATCH
}

ATTN_API attn_status attn_move_centre(attn_state* st, int node) {
  ATTN_TRY
  NEED(st, "state");
  st->move_centre(node);
  ATTN_CHECK_CUDA(cudaStreamSynchronize(st->ctx->stream));
  ATTN_CATCH
}

ATTN_API attn_status attn_isometry_error(attn_state* st, double* err) {
  ATTN_TRY
  NEED(st, "state");
  NEED(err, "err");
  *err = st->isometry_error();
  ATTN_CATCH
}

// ------------------------------------------------------------ disentanglers
ATTN_API attn_status attn_de_place(attn_state* st, int max_de, int* n_placed) {
  ATTN_TRY
  NEED(st, "state");
  ATTN_REQUIRE(max_de >= 0, ATTN_EINVAL, "max_de < 0");
  st->des = place_disentanglers(st->tree, st->model, max_de);
  st->us.assign(st->des.size(), std::vector<double>(16, 0.0));
  for (auto& u : st->us)
    for (int i = 0; i < 4; ++i) u[i * 5] = 1.0;
  st->mapped_ready = false;
  if (n_placed) *n_placed = (int)st->des.size();
  ATTN_CATCH
}

ATTN_API attn_status attn_de_sites(attn_state* st, int* pairs) {
  ATTN_TRY
  NEED(st, "state");
  NEED(pairs, "pairs_out");
  for (size_t k = 0; k < st->des.size(); ++k) {
    pairs[2 * k] = st->des[k].first;
    pairs[2 * k + 1] = st->des[k].second;
  }
  ATTN_CATCH
}

ATTN_API attn_status attn_de_set(attn_state* st, int k, const double* u16) {
  ATTN_TRY
  NEED(st, "state");
  NEED(u16, "u16");
  ATTN_REQUIRE(k >= 0 && k < (int)st->des.size(), ATTN_EINVAL, "disentangler index out of range");
  double err = 0;
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 4; ++j) {
      double s = 0;
      for (int q = 0; q < 4; ++q) s += u16[q * 4 + i] * u16[q * 4 + j];
      err = std::max(err, std::fabs(s - (i == j ? 1.0 : 0.0)));
    }
  ATTN_REQUIRE(err < 1e-10, ATTN_ENOTISOMETRIC, "disentangler is not orthogonal (|u^T u - 1| >= 1e-10)");
  st->us[k].assign(u16, u16 + 16);
  st->mapped_ready = false;
  ATTN_CATCH
}

ATTN_API attn_status attn_de_get(attn_state* st, int k, double* u16) {
  ATTN_TRY
  NEED(st, "state");
  NEED(u16, "u16");
  ATTN_REQUIRE(k >= 0 && k < (int)st->des.size(), ATTN_EINVAL, "disentangler index out of range");
  std::memcpy(u16, st->us[k].data(), 16 * sizeof(double));
  ATTN_CATCH
}

ATTN_API attn_status attn_map_hamiltonian(attn_state* st) {
  ATTN_TRY
  NEED(st, "state");
  st->set_products();
  ATTN_CATCH
}

ATTN_API attn_status attn_heff_counts(attn_state* st, int node, int counts[5]) {
  ATTN_TRY
  NEED(st, "state");
  NEED(counts, "counts");
  ATTN_REQUIRE(node >= 0 && node < st->tree.n_nodes, ATTN_EINVAL, "node out of range");
  ATTN_REQUIRE(st->mapped_ready, ATTN_EINVAL, "Hamiltonian not mapped yet (call attn_map_hamiltonian)");
  for (int i = 0; i < 5; ++i) counts[i] = 0;
  for (const Prod& p : st->prods) {
    int mask = 0;
    for (int a = 0; a < p.n; ++a)
      for (int s = 0; s < 3; ++s)
        if (st->tree.behind(node, s, p.site[a])) mask |= 1 << s;
    if (mask == 3) counts[0]++;
    else if (mask == 5) counts[1]++;
    else if (mask == 6) counts[2]++;
    else if (mask == 7) counts[3]++;
    else counts[4]++;
  }
  ATTN_CATCH
}

ATTN_API attn_status attn_hamiltonian_info(attn_state* st, int* n_terms, int* n_products) {
  ATTN_TRY
  NEED(st, "state");
  if (n_terms) *n_terms = (int)st->mapped.size();
  if (n_products) *n_products = (int)st->prods.size();
  ATTN_CATCH
}

// -------------------------------------------------------------------- H_eff
ATTN_API attn_status attn_heff_create(attn_ctx* ctx, const attn_heff_desc* d, attn_heff** out) {
  ATTN_TRY
  NEED(ctx, "ctx");
  NEED(d, "desc");
  NEED(out, "out");
  auto h = std::make_unique<attn_heff>();
  h->ctx = ctx;
  for (int s = 0; s < 3; ++s) {
    ATTN_REQUIRE(d->m[s] >= 1 && d->m[s] <= 4096, ATTN_EINVAL, "link dimension must be 1..4096");
    h->m[s] = d->m[s];
  }
  h->V = (long)d->m[0] * d->m[1] * d->m[2];
  for (int s = 0; s < 3; ++s) {
    if (!d->h_int[s]) continue;
    const long sz = (long)d->m[s] * d->m[s];
    h->has_hint[s] = true;
    h->hint[s].reserve(sizeof(double) * sz);
    copy_f64(ctx, h->hint[s].as<double>(), d->h_int[s], sz);
  }
  for (int k = 0; k < 3; ++k) {
    ATTN_REQUIRE(d->n_pair[k] >= 0, ATTN_EINVAL, "n_pair < 0");
    h->npair[k] = d->n_pair[k];
    if (!d->n_pair[k]) continue;
    NEED(d->pair_a[k], "pair_a");
    NEED(d->pair_b[k], "pair_b");
    const int p = kPairP[k], q = kPairQ[k];
    const long na = (long)d->n_pair[k] * d->m[p] * d->m[p], nb = (long)d->n_pair[k] * d->m[q] * d->m[q];
    h->pa[k].reserve(sizeof(double) * na);
    h->pb[k].reserve(sizeof(double) * nb);
    copy_f64(ctx, h->pa[k].as<double>(), d->pair_a[k], na);
    copy_f64(ctx, h->pb[k].as<double>(), d->pair_b[k], nb);
  }
  ATTN_REQUIRE(d->n_triple >= 0, ATTN_EINVAL, "n_triple < 0");
  h->ntrip = d->n_triple;
  if (h->ntrip) {
    for (int s = 0; s < 3; ++s) {
      NEED(d->triple[s], "triple");
      const long n = (long)h->ntrip * d->m[s] * d->m[s];
      h->tr[s].reserve(sizeof(double) * n);
      copy_f64(ctx, h->tr[s].as<double>(), d->triple[s], n);
    }
  }
  *out = h.release();
  ATTN_CATCH
}

ATTN_API attn_status attn_heff_build(attn_state* st, int node, attn_heff** out) {
  ATTN_TRY
  NEED(st, "state");
  NEED(out, "out");
  ATTN_REQUIRE(node >= 0 && node < st->tree.n_nodes, ATTN_EINVAL, "node out of range");
  *out = st->build_heff(node);
  ATTN_CATCH
}

ATTN_API attn_status attn_heff_destroy(attn_heff* h) {
  ATTN_TRY
  if (!h) return ATTN_OK;
  cudaStreamSynchronize(h->ctx->stream);
  delete h;
  ATTN_CATCH
}

ATTN_API attn_status attn_heff_info(attn_heff* h, int n_pair[3], int* n_triple, double* flops) {
  ATTN_TRY
  NEED(h, "heff");
  if (n_pair)
    for (int k = 0; k < 3; ++k) n_pair[k] = h->npair[k];
  if (n_triple) *n_triple = h->ntrip;
  if (flops) *flops = h->flops();
  ATTN_CATCH
}

ATTN_API attn_status attn_heff_apply(attn_heff* h, const double* x, double* y, attn_dtype dtype) {
  ATTN_TRY
  NEED(h, "heff");
  NEED(x, "x_dev");
  NEED(y, "y_dev");
  ATTN_REQUIRE(x != y, ATTN_EINVAL, "x and y must be distinct buffers");
  ATTN_REQUIRE(dtype == ATTN_F64 || dtype == ATTN_BF16 || dtype == ATTN_TF32, ATTN_EUNSUPPORTED,
               "dtype must be ATTN_F64, ATTN_TF32 or ATTN_BF16");
  h->apply(x, y, dtype);
  ATTN_CATCH
}

ATTN_API attn_status attn_heff_apply_host(attn_heff* h, const double* xh, double* yh, attn_dtype dtype) {
  ATTN_TRY
  NEED(h, "heff");
  NEED(xh, "x_host");
  NEED(yh, "y_host");
  attn_ctx* ctx = h->ctx;
  ctx->ws[2].reserve(sizeof(double) * 2 * h->V);
  double* xd = ctx->ws[2].as<double>();
  double* yd = xd + h->V;
  ATTN_CHECK_CUDA(cudaMemcpyAsync(xd, xh, sizeof(double) * h->V, cudaMemcpyHostToDevice, ctx->stream));
  ATTN_REQUIRE(dtype == ATTN_F64 || dtype == ATTN_BF16 || dtype == ATTN_TF32, ATTN_EUNSUPPORTED,
               "dtype must be ATTN_F64, ATTN_TF32 or ATTN_BF16");
  h->apply(xd, yd, dtype);
  ATTN_CHECK_CUDA(cudaMemcpyAsync(yh, yd, sizeof(double) * h->V, cudaMemcpyDeviceToHost, ctx->stream));
  ATTN_CHECK_CUDA(cudaStreamSynchronize(ctx->stream));
  ATTN_CATCH
}

}  // extern "C"

// Lowest eigenpair of H_eff from the device tensor T_dev (the body of attn_eigsolve).
static void eigsolve_dev(attn_heff* h, double* T_dev, double* theta, int* iters) {
  attn_ctx* ctx = h->ctx;
  const attn_config& cfg = ctx->cfg;
  // shapes the tensor-core tiles cannot take run their matvecs in FP64 (on the GPU)
  const attn_dtype dt = (cfg.matvec_dtype != ATTN_F64 && tc_supported(h)) ? cfg.matvec_dtype : ATTN_F64;
  MatVec lo = [&](const double* a, double* b) { h->apply(a, b, dt); };
  MatVec hi = [&](const double* a, double* b) { h->apply_f64(a, b); };
  const int rsteps = (dt != ATTN_F64) ? cfg.refine_steps : 0;
  if (cfg.use_graphs) {
    EigGraph* g = h->eg;
    // a graph holds the addresses of the context's scratch buffers at capture time:
    // any reallocation since (scratch_epoch) or a change of the FP64 contraction path
    // (f64_split) or of the tensor-core grid (tc_schedule) makes it stale
    if (!g || g->x != T_dev || g->depth != cfg.lanczos_depth || g->tol != cfg.lanczos_tol || g->dtype != dt ||
        g->refine != rsteps || g->rtol != cfg.refine_tol || g->prof != ctx->prof_on ||
        g->f64_split != cfg.f64_split || g->tc_schedule != cfg.tc_schedule || g->basis != cfg.lanczos_basis ||
        g->epoch != ctx->scratch_epoch) {
      delete g;
      g = h->eg = new EigGraph();
      g->x = T_dev;
      g->depth = cfg.lanczos_depth;
      g->tol = cfg.lanczos_tol;
      g->dtype = dt;
      g->refine = rsteps;
      g->rtol = cfg.refine_tol;
      g->prof = ctx->prof_on;
      g->f64_split = cfg.f64_split;
      g->tc_schedule = cfg.tc_schedule;
      g->basis = cfg.lanczos_basis;
      // warm-up on a scratch copy: every buffer the solve needs is allocated before capture
      ctx->ws[3].reserve(sizeof(double) * h->V);
      copy_f64(ctx, ctx->ws[3].as<double>(), T_dev, h->V);
      const bool prof_was = ctx->prof_on;
      ctx->prof_on = false;
      lanczos_enqueue(ctx, lo, ctx->ws[3].as<double>(), h->V, cfg.lanczos_depth, cfg.lanczos_tol, g->w, 0,
                      dt != ATTN_F64 && cfg.lanczos_basis == 1);
      ctx->prof_on = prof_was;
      ATTN_CHECK_CUDA(cudaStreamSynchronize(ctx->stream));
      g->epoch_before = ctx->scratch_epoch;
      cudaStream_t user = ctx->stream, cs;
      ATTN_CHECK_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
      const uint64_t l0 = ctx->launches;
      ctx->stream = cs;
      ctx->capture_events = &g->evs;
      cudaError_t ce = cudaStreamBeginCapture(cs, cudaStreamCaptureModeRelaxed);
      try {
        ATTN_CHECK_CUDA(ce);
        lanczos_enqueue(ctx, lo, T_dev, h->V, cfg.lanczos_depth, cfg.lanczos_tol, g->w, 0,
                        dt != ATTN_F64 && cfg.lanczos_basis == 1);
      } catch (...) {
        cudaGraph_t tmp = nullptr;
        cudaStreamEndCapture(cs, &tmp);
        if (tmp) cudaGraphDestroy(tmp);
        ctx->stream = user;
        ctx->capture_events = nullptr;
        cudaStreamDestroy(cs);
        delete g;
        h->eg = nullptr;
        throw;
      }
      ATTN_CHECK_CUDA(cudaStreamEndCapture(cs, &g->graph));
      ctx->stream = user;
      ctx->capture_events = nullptr;
      ATTN_CHECK_CUDA(cudaStreamDestroy(cs));
      g->launches = ctx->launches - l0;
      ctx->launches = l0;
      // the warm-up sized every scratch buffer, so none may have moved during the capture
      ATTN_REQUIRE(ctx->scratch_epoch == g->epoch_before, ATTN_ECUDA,
                   "a scratch buffer was reallocated while the eigensolve graph was captured");
      g->epoch = ctx->scratch_epoch;
      ATTN_CHECK_CUDA(cudaGraphInstantiate(&g->exec, g->graph, 0));
    }
    ATTN_CHECK_CUDA(cudaGraphLaunch(g->exec, ctx->stream));
    ctx->launches += g->launches;
    LanczosResult r = timeout_first(ctx, h, [&] { return lanczos_read(ctx, g->w); });
    r.converged = r.resid < cfg.lanczos_tol * std::max(std::fabs(r.theta), 1e-300);
    for (auto& e : g->evs) {
      float ms = 0.f;
      ATTN_CHECK_CUDA(cudaEventElapsedTime(&ms, e.a, e.b));
      ctx->prof[e.kid].acc_ms += ms;
      ctx->prof[e.kid].acc_flops += e.flops;
      ctx->prof[e.kid].acc_launches += 1;
    }
    *theta = r.theta;
    int it = r.iters;
    bool conv = r.converged;
    if (rsteps > 0) {
      RefineResult f = timeout_first(ctx, h, [&] {
        return refine_eig(ctx, hi, lo, T_dev, h->V, rsteps, cfg.refine_inner, cfg.refine_tol, g->rw);
      });
      *theta = f.theta;
      it += f.fp64_matvecs + f.lo_matvecs;
      conv = f.converged;
    }
    check_device_errors(ctx, h);
    if (iters) *iters = it;
    ATTN_REQUIRE(!(cfg.report_unconverged && !conv), ATTN_ENOTCONVERGED,
                 "the eigensolve stopped above its tolerance (best Ritz pair written)");
    return;
  }
  LanczosWork w;
  LanczosResult r = timeout_first(ctx, h, [&] {
    return lanczos_lowest(ctx, lo, T_dev, h->V, cfg.lanczos_depth, cfg.lanczos_tol, w,
                          dt != ATTN_F64 && cfg.lanczos_basis == 1);
  });
  double th = r.theta;
  int it = r.iters;
  bool conv = r.converged;
  if (rsteps > 0) {
    RefineWork rw;
    RefineResult f = timeout_first(ctx, h, [&] {
      return refine_eig(ctx, hi, lo, T_dev, h->V, rsteps, cfg.refine_inner, cfg.refine_tol, rw);
    });
    th = f.theta;
    it += f.fp64_matvecs + f.lo_matvecs;
    conv = f.converged;
  }
  ATTN_CHECK_CUDA(cudaStreamSynchronize(ctx->stream));
  check_device_errors(ctx, h);
  *theta = th;
  if (iters) *iters = it;
  ATTN_REQUIRE(!(cfg.report_unconverged && !conv), ATTN_ENOTCONVERGED,
               "the eigensolve stopped above its tolerance (best Ritz pair written)");
}

extern "C" {

ATTN_API attn_status attn_eigsolve(attn_heff* h, double* T_dev, double* theta, int* iters) {
  ATTN_TRY
  NEED(h, "heff");
  NEED(T_dev, "T_dev");
  NEED(theta, "theta");
  eigsolve_dev(h, T_dev, theta, iters);
  ATTN_CATCH
}

ATTN_API attn_status attn_eigsolve_host(attn_heff* h, double* T_host, double* theta, int* iters) {
  ATTN_TRY
  NEED(h, "heff");
  NEED(T_host, "T_host");
  NEED(theta, "theta");
  attn_ctx* ctx = h->ctx;
  h->host_x.reserve(sizeof(double) * h->V);  // owned by h: a stable address for graph replays
  double* xd = h->host_x.as<double>();
  ATTN_CHECK_CUDA(cudaMemcpyAsync(xd, T_host, sizeof(double) * h->V, cudaMemcpyHostToDevice, ctx->stream));
  eigsolve_dev(h, xd, theta, iters);
  ATTN_CHECK_CUDA(cudaMemcpyAsync(T_host, xd, sizeof(double) * h->V, cudaMemcpyDeviceToHost, ctx->stream));
  ATTN_CHECK_CUDA(cudaStreamSynchronize(ctx->stream));
  ATTN_CATCH
}

// ----------------------------------------------------------- sweep drivers
ATTN_API attn_status attn_local_step(attn_state* st, int node, double* energy) {
  ATTN_TRY
  NEED(st, "state");
  double e = st->local_step(node);
  ATTN_CHECK_CUDA(cudaStreamSynchronize(st->ctx->stream));
  if (energy) *energy = e;
  ATTN_CATCH
}

ATTN_API attn_status attn_ttn_sweep(attn_state* st, double* energy) {
  ATTN_TRY
  NEED(st, "state");
  double e = 0;
  for (int n : st->tree.post_order()) e = st->local_step(n);
  ATTN_CHECK_CUDA(cudaStreamSynchronize(st->ctx->stream));
  if (energy) *energy = e;
  ATTN_CATCH
}

ATTN_API attn_status attn_de_update(attn_state* st, double* dE) {
  ATTN_TRY
  NEED(st, "state");
  st->ctx->prof_begin(8);
  double d = st->de_update(nullptr);
  st->ctx->prof_end(8, 0.0);
  if (dE) *dE = d;
  ATTN_CATCH
}

ATTN_API attn_status attn_de_energies(attn_state* st, double* e_out) {
  ATTN_TRY
  NEED(st, "state");
  NEED(e_out, "e_out");
  std::copy(st->last_de_energy.begin(), st->last_de_energy.end(), e_out);
  ATTN_CATCH
}

ATTN_API attn_status attn_sweep(attn_state* st, double* energy) {
  ATTN_TRY
  NEED(st, "state");
  const attn_config& cfg = st->ctx->cfg;
  if (st->sweep_count >= cfg.s_ttn && !st->des.empty()) {
    st->ctx->prof_begin(8);
    st->de_update(nullptr);
    st->ctx->prof_end(8, 0.0);
  }
  if (!st->mapped_ready) st->set_products();
  double e = 0;
  for (int n : st->tree.post_order()) e = st->local_step(n);
  ATTN_CHECK_CUDA(cudaStreamSynchronize(st->ctx->stream));
  st->sweep_count++;
  if (energy) *energy = e;
  ATTN_CATCH
}

// ------------------------------------------------------ learned initialiser
ATTN_API attn_status attn_mlp_param_count(int* n) {
  ATTN_TRY
  NEED(n, "n");
  *n = (int)mlp_param_count();
  ATTN_CATCH
}

ATTN_API attn_status attn_mlp_create(attn_ctx* ctx, const float* params, attn_mlp** out) {
  ATTN_TRY
  NEED(ctx, "ctx");
  NEED(params, "params_host");
  NEED(out, "out");
  for (size_t i = 0; i < mlp_param_count(); ++i)
    ATTN_REQUIRE(std::isfinite(params[i]), ATTN_ENONFINITE, "non-finite MLP parameter");
  auto m = std::make_unique<attn_mlp>();
  m->net.init(ctx, params);
  ATTN_CHECK_CUDA(cudaStreamSynchronize(ctx->stream));
  *out = m.release();
  ATTN_CATCH
}

ATTN_API attn_status attn_mlp_destroy(attn_mlp* m) {
  ATTN_TRY
  if (!m) return ATTN_OK;
  cudaStreamSynchronize(m->net.ctx->stream);
  delete m;
  ATTN_CATCH
}

ATTN_API attn_status attn_mlp_get_params(attn_mlp* m, float* out) {
  ATTN_TRY
  NEED(m, "mlp");
  NEED(out, "params_out");
  ATTN_CHECK_CUDA(cudaMemcpyAsync(out, m->net.params.p, sizeof(float) * mlp_param_count(), cudaMemcpyDeviceToHost,
                                  m->net.ctx->stream));
  ATTN_CHECK_CUDA(cudaStreamSynchronize(m->net.ctx->stream));
  ATTN_CATCH
}

ATTN_API attn_status attn_mlp_predict(attn_mlp* m, int n, const double* rho, double* u) {
  ATTN_TRY
  NEED(m, "mlp");
  ATTN_REQUIRE(n >= 1, ATTN_EINVAL, "n must be >= 1");
  NEED(rho, "rho_host");
  NEED(u, "u_host");
  m->net.predict(n, rho, u);
  ATTN_CATCH
}

ATTN_API attn_status attn_mlp_loss_grad(attn_mlp* m, int n, const double* rho, const double* ut, double* loss,
                                        float* grad) {
  ATTN_TRY
  NEED(m, "mlp");
  ATTN_REQUIRE(n >= 1, ATTN_EINVAL, "n must be >= 1");
  NEED(rho, "rho_host");
  NEED(ut, "u_target_host");
  m->net.upload_inputs(n, rho, ut);
  const float l = m->net.loss_grad(n);
  if (loss) *loss = l;
  if (grad) {
    ATTN_CHECK_CUDA(cudaMemcpyAsync(grad, m->net.grad.p, sizeof(float) * mlp_param_count(), cudaMemcpyDeviceToHost,
                                    m->net.ctx->stream));
    ATTN_CHECK_CUDA(cudaStreamSynchronize(m->net.ctx->stream));
  }
  ATTN_CATCH
}

ATTN_API attn_status attn_mlp_train(attn_mlp* m, int n, const double* rho, const double* ut, int steps, double lr,
                                    double* final_loss) {
  ATTN_TRY
  NEED(m, "mlp");
  ATTN_REQUIRE(n >= 1 && steps >= 0 && lr > 0, ATTN_EINVAL, "need n >= 1, steps >= 0, lr > 0");
  NEED(rho, "rho_host");
  NEED(ut, "u_target_host");
  m->net.upload_inputs(n, rho, ut);
  float l = 0.f;
  for (int s = 0; s < steps; ++s) {
    l = m->net.loss_grad(n);
    ATTN_REQUIRE(std::isfinite(l), ATTN_ENONFINITE, "non-finite training loss");
    m->net.adam_step((float)lr);
  }
  if (final_loss) *final_loss = steps ? l : m->net.loss_grad(n);
  ATTN_CATCH
}

ATTN_API attn_status attn_set_learned_init(attn_state* st, attn_mlp* m) {
  ATTN_TRY
  NEED(st, "state");
  st->learned = m;
  ATTN_CATCH
}

ATTN_API attn_status attn_de_training_pairs(attn_state* st, double* rho_out, double* u_out) {
  ATTN_TRY
  NEED(st, "state");
  ATTN_REQUIRE(st->first_de_done, ATTN_EINVAL, "no disentangler update has run on this state");
  const int n = (int)st->des.size();
  if (rho_out) std::copy(st->rho_first.begin(), st->rho_first.end(), rho_out);
  if (u_out) {
    for (int k = 0; k < n; ++k) {
      double u[16];
      std::copy(st->us[k].begin(), st->us[k].end(), u);
      // det(u) < 0 cannot be reached by expm of an antisymmetric generator:
      // use u diag(1, 1, 1, -1) as the target (reading)
      double M[16];
      std::copy(u, u + 16, M);
      double det = 1.0;
      for (int c = 0; c < 4; ++c) {  // Gaussian elimination with partial pivoting
        int p = c;
        for (int r = c + 1; r < 4; ++r)
          if (std::fabs(M[r * 4 + c]) > std::fabs(M[p * 4 + c])) p = r;
        if (M[p * 4 + c] == 0.0) { det = 0.0; break; }
        if (p != c) {
          for (int q = 0; q < 4; ++q) std::swap(M[c * 4 + q], M[p * 4 + q]);
          det = -det;
        }
        det *= M[c * 4 + c];
        for (int r = c + 1; r < 4; ++r) {
          const double f = M[r * 4 + c] / M[c * 4 + c];
          for (int q = c; q < 4; ++q) M[r * 4 + q] -= f * M[c * 4 + q];
        }
      }
      if (det < 0)
        for (int r = 0; r < 4; ++r) u[r * 4 + 3] = -u[r * 4 + 3];
      std::copy(u, u + 16, u_out + 16L * k);
    }
  }
  ATTN_CATCH
}

ATTN_API attn_status attn_learned_init_report(attn_state* st, int* used, int* fallback) {
  ATTN_TRY
  NEED(st, "state");
  if (used) *used = st->learned_used;
  if (fallback) *fallback = st->learned_fallback;
  ATTN_CATCH
}

ATTN_API attn_status attn_energy(attn_state* st, double* energy) {
  ATTN_TRY
  NEED(st, "state");
  NEED(energy, "energy");
  *energy = st->energy();
  ATTN_CATCH
}


// ----------------------------------------------------- boundary additions
ATTN_API attn_status attn_set_allocator(attn_alloc_fn alloc, attn_free_fn free_fn, void* user) {
  ATTN_TRY
  ATTN_REQUIRE((alloc == nullptr) == (free_fn == nullptr), ATTN_EINVAL, "give both alloc and free, or neither");
  set_allocator(alloc, free_fn, user);
  ATTN_CATCH
}

ATTN_API attn_status attn_renormalise(attn_state* st, int node, int slot, int* n_open) {
  ATTN_TRY
  NEED(st, "state");
  ATTN_REQUIRE(node >= 0 && node < st->tree.n_nodes && slot >= 0 && slot < 3, ATTN_EINVAL, "node/slot out of range");
  ATTN_REQUIRE(st->mapped_ready, ATTN_EINVAL, "Hamiltonian not mapped yet (call attn_map_hamiltonian)");
  const Tree::Nbr& nb = st->tree.nbr[3 * node + slot];
  ATTN_REQUIRE(nb.kind == 1, ATTN_EINVAL, "the link leads to a physical site, not to a tensor");
  st->move_centre(nb.idx);
  const Env& e = st->get_env(nb.idx, nb.back);
  ATTN_CHECK_CUDA(cudaStreamSynchronize(st->ctx->stream));
  if (n_open) *n_open = (int)e.open.size();
  ATTN_CATCH
}

ATTN_API attn_status attn_link_operators(attn_state* st, int node, int slot, int* dim, int* n_open, int* has_internal,
                                         double* h_int) {
  ATTN_TRY
  NEED(st, "state");
  ATTN_REQUIRE(node >= 0 && node < st->tree.n_nodes && slot >= 0 && slot < 3, ATTN_EINVAL, "node/slot out of range");
  const Env& e = st->get_env(node, slot);
  if (dim) *dim = e.dim;
  if (n_open) *n_open = (int)e.open.size();
  if (has_internal) *has_internal = e.has_hint ? 1 : 0;
  if (h_int) {
    const size_t n = (size_t)e.dim * e.dim;
    if (e.has_hint)
      ATTN_CHECK_CUDA(cudaMemcpyAsync(h_int, e.hint.p, sizeof(double) * n, cudaMemcpyDeviceToHost, st->ctx->stream));
    else
      std::fill(h_int, h_int + n, 0.0);
  }
  ATTN_CHECK_CUDA(cudaStreamSynchronize(st->ctx->stream));
  ATTN_CATCH
}

ATTN_API attn_status attn_state_save(attn_state* st, const char* path) {
  ATTN_TRY
  NEED(st, "state");
  NEED(path, "path");
  st->save(path);
  ATTN_CATCH
}

ATTN_API attn_status attn_state_load(attn_state* st, const char* path) {
  ATTN_TRY
  NEED(st, "state");
  NEED(path, "path");
  st->load(path);
  ATTN_CATCH
}

ATTN_API attn_status attn_de_update_one(attn_state* st, int k, double* dE) {
  ATTN_TRY
  NEED(st, "state");
  ATTN_REQUIRE(k >= 0 && k < (int)st->des.size(), ATTN_EINVAL, "disentangler index out of range");
  const std::vector<int> one = {k};
  st->ctx->prof_begin(8);
  const double d = st->de_update(&one);
  st->ctx->prof_end(8, 0.0);
  if (dE) *dE = d;
  ATTN_CATCH
}

ATTN_API attn_status attn_de_environment(attn_state* st, int k, const double* u16, double* gamma16, double* e_k) {
  ATTN_TRY
  NEED(st, "state");
  NEED(u16, "u16");
  ATTN_REQUIRE(k >= 0 && k < (int)st->des.size(), ATTN_EINVAL, "disentangler index out of range");
  double g[16], e = 0.0;
  st->de_environment(k, u16, g, &e);
  if (gamma16) std::copy(g, g + 16, gamma16);
  if (e_k) *e_k = e;
  ATTN_CATCH
}

ATTN_API attn_status attn_rdm2(attn_state* st, int k, double* rho16) {
  ATTN_TRY
  NEED(st, "state");
  NEED(rho16, "rho16");
  ATTN_REQUIRE(k >= 0 && k < (int)st->des.size(), ATTN_EINVAL, "disentangler index out of range");
  const std::vector<double> r = st->de_rdms({k});
  std::copy(r.begin(), r.end(), rho16);
  ATTN_CATCH
}

ATTN_API attn_status attn_measure(attn_state* st, int n_obs, const int* nsites, const int* sites, const double* ops,
                                  double* values) {
  ATTN_TRY
  NEED(st, "state");
  ATTN_REQUIRE(n_obs >= 0, ATTN_EINVAL, "n_obs < 0");
  if (!n_obs) return ATTN_OK;
  NEED(nsites, "nsites");
  NEED(sites, "sites");
  NEED(ops, "ops");
  NEED(values, "values");
  const std::vector<double> v = st->measure(n_obs, nsites, sites, ops);
  std::copy(v.begin(), v.end(), values);
  ATTN_CATCH
}

ATTN_API attn_status attn_correlation_matrix(attn_state* st, const double* oa, const double* ob, double* C) {
  ATTN_TRY
  NEED(st, "state");
  NEED(oa, "oa");
  NEED(ob, "ob");
  NEED(C, "C");
  const int N = st->model.n_sites;
  std::vector<int> ns((size_t)N * N), sites(4L * N * N, 0);
  std::vector<double> ops(16L * N * N, 0.0);
  double ab[4];  // o^a o^b on one site
  for (int r = 0; r < 2; ++r)
    for (int c = 0; c < 2; ++c) ab[r * 2 + c] = oa[r * 2] * ob[c] + oa[r * 2 + 1] * ob[2 + c];
  for (int i = 0; i < N; ++i)
    for (int j = 0; j < N; ++j) {
      const long q = (long)i * N + j;
      if (i == j) {
        ns[q] = 1;
        sites[4 * q] = i;
        std::copy(ab, ab + 4, ops.begin() + 16 * q);
      } else {
        ns[q] = 2;
        sites[4 * q] = i;
        sites[4 * q + 1] = j;
        std::copy(oa, oa + 4, ops.begin() + 16 * q);
        std::copy(ob, ob + 4, ops.begin() + 16 * q + 4);
      }
    }
  const std::vector<double> v = st->measure(N * N, ns.data(), sites.data(), ops.data());
  std::copy(v.begin(), v.end(), C);
  ATTN_CATCH
}

}  // extern "C"
