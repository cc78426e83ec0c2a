// TTN state, effective operators, renormalisation and the sweep (Secs. 3.1,
// 3.3.2, 4, 4.4.2).
//
// Each directed link (n, slot) keeps the operators of the rank-1 products of
// H' as seen from n: the sum of all products lying entirely behind the link
// (one m x m "internal" operator) and one renormalised operator per product
// with sites on both sides. Moving across node c towards n renormalises them
// with O_out = T_c^T (O_x (x) O_y) T_c over c's two other links (Fig. eff-op);
// products that become entirely internal are summed into the new internal
// operator. H_eff of the centre then reads the three links' operators: a
// product present on two links is a pair term, on all three a triple term.
// Link operators are recomputed lazily after a tensor on their far side
// changes, so they always point at the current isometry centre.
#include <algorithm>
#include <cmath>
#include <climits>
#include <cstring>

#include "state.h"

using namespace attn;

namespace attn {

int Env::find(int q) const {
  auto it = std::lower_bound(pos.begin(), pos.end(), std::make_pair(q, -1));
  if (it != pos.end() && it->first == q) return it->second;
  return -1;
}

// y += sum_r A_r x_p W_r  (W_r per-product tensors, stride V) -- defined in heff_f64.cu
void accumulate_slot_f64(attn_ctx* ctx, const int d[3], int p, const double* A, int R, const double* W, double* y);

namespace {

__global__ void gram_err_kernel(const double* G, int k, double* out) {
  __shared__ double sh[256];
  double m = 0.0;
  for (long e = threadIdx.x; e < (long)k * k; e += blockDim.x) {
    long i = e / k, j = e % k;
    double v = fabs(G[e] - (i == j ? 1.0 : 0.0));
    m = fmax(m, v);
  }
  sh[threadIdx.x] = m;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) sh[threadIdx.x] = fmax(sh[threadIdx.x], sh[threadIdx.x + s]);
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = sh[0];
}

// out[r][i][j] = sum over the two other slots of T[.. i at t ..] * W_r[.. j at t ..]
void contract_tt(attn_ctx* ctx, const double* T, const int d[3], int t, const double* W, int R, double* out) {
  const long V = (long)d[0] * d[1] * d[2];
  GemmF64 g;
  g.split_ok = true;
  g.M = g.N = d[t];
  g.Bhi = R;
  g.C = out; g.cM = d[t]; g.cN = 1; g.cBhi = (long)d[t] * d[t];
  if (t == 2) {
    g.K = d[0] * d[1];
    g.A = T; g.aM = 1; g.aK = d[2];
    g.B = W; g.bK = d[2]; g.bN = 1; g.bBhi = V;
  } else if (t == 0) {
    g.K = d[1] * d[2];
    g.A = T; g.aM = (long)d[1] * d[2]; g.aK = 1;
    g.B = W; g.bK = 1; g.bN = (long)d[1] * d[2]; g.bBhi = V;
  } else {
    g.K = d[2];
    g.G = d[0];
    g.A = T; g.aM = d[2]; g.aK = 1; g.aG = (long)d[1] * d[2];
    g.B = W; g.bK = 1; g.bN = d[2]; g.bG = (long)d[1] * d[2]; g.bBhi = V;
  }
  gemm_f64(ctx, g);
}

void upload_idx(attn_ctx* ctx, DevBuf& buf, const std::vector<int>& idx) {
  buf.reserve(sizeof(int) * std::max<size_t>(idx.size(), 1));
  if (!idx.empty())
    ATTN_CHECK_CUDA(cudaMemcpyAsync(buf.p, idx.data(), sizeof(int) * idx.size(), cudaMemcpyHostToDevice, ctx->stream));
}

}  // namespace
}  // namespace attn

// ----------------------------------------------------------------- basics
void attn_state::init_from_raw(const double* const* raw) {
  const int N = tree.n_nodes;
  T.clear();
  T.resize(N);
  for (int n = 0; n < N; ++n) {
    const long V = vol(n);
    T[n].reserve(sizeof(double) * V);
    ATTN_CHECK_CUDA(cudaMemcpyAsync(T[n].p, raw[n], sizeof(double) * V, cudaMemcpyHostToDevice, ctx->stream));
  }
  ctx->scal.reserve(sizeof(double) * 64);
  for (int n = 0; n < N; ++n) {
    const int d[3] = {dim(n, 0), dim(n, 1), dim(n, 2)};
    if (n == tree.top0()) {
      normalise_dev(ctx, tensor(n), tensor(n), vol(n), ctx->scal.as<double>());
      continue;
    }
    const long M = (long)d[0] * d[1];
    colbuf.reserve(sizeof(double) * vol(n));
    rbuf.reserve(sizeof(double) * d[2] * d[2]);
    tensor_to_columns(ctx, tensor(n), d, 2, colbuf.as<double>());
    qr_columns(ctx, colbuf.as<double>(), M, d[2], rbuf.as<double>(), qrw);
    columns_to_tensor(ctx, colbuf.as<double>(), d, 2, tensor(n));
  }
  centre = tree.top0();
  env.clear();
  env.resize(3 * N);
  for (int n = 0; n < N; ++n)
    for (int s = 0; s < 3; ++s) env[3 * n + s].dim = dim(n, s);
  mapped_ready = false;
  energy_known = std::nan("");
}

void attn_state::invalidate_from(int c) {
  for (int n = 0; n < tree.n_nodes; ++n)
    for (int s = 0; s < 3; ++s) {
      Env& e = env[3 * n + s];
      if (!e.valid) continue;
      const Tree::Nbr& nb = tree.nbr[3 * n + s];
      if (nb.kind == 0) continue;
      bool far;
      if (s < 2) {
        const int ch = nb.idx;
        far = tree.lo[ch] <= tree.lo[c] && tree.hi[c] <= tree.hi[ch];
      } else {
        far = !(tree.lo[n] <= tree.lo[c] && tree.hi[c] <= tree.hi[n]);
      }
      if (far) e.valid = false;
    }
}

void attn_state::move_centre(int target) {
  ATTN_REQUIRE(target >= 0 && target < tree.n_nodes, ATTN_EINVAL, "node out of range");
  std::vector<int> p = tree.path(centre, target);
  for (size_t h = 0; h + 1 < p.size(); ++h) {
    const int a = p[h], b = p[h + 1];
    const int s = tree.slot_towards(a, b), back = tree.slot_towards(b, a);
    const int da[3] = {dim(a, 0), dim(a, 1), dim(a, 2)};
    const int db[3] = {dim(b, 0), dim(b, 1), dim(b, 2)};
    const int k = da[s];
    const long M = vol(a) / k;
    colbuf.reserve(sizeof(double) * vol(a));
    rbuf.reserve(sizeof(double) * k * k);
    tensor_to_columns(ctx, tensor(a), da, s, colbuf.as<double>());
    qr_columns(ctx, colbuf.as<double>(), M, k, rbuf.as<double>(), qrw);
    columns_to_tensor(ctx, colbuf.as<double>(), da, s, tensor(a));
    tmpT.reserve(sizeof(double) * vol(b));
    mode_product_f64(ctx, db, back, rbuf.as<double>(), 1, tensor(b), 0, tmpT.as<double>(), 0.0);
    std::swap(T[b], tmpT);
    invalidate_from(a);
    invalidate_from(b);
    centre = b;
  }
}

void attn_state::set_products() {
  mapped = map_terms(model, des, us);
  if (ctx->cfg.compress_terms) mapped = compress_terms(mapped);
  prods = split_products(mapped);
  for (auto& e : env) e.valid = false;
  mapped_ready = true;
  energy_known = std::nan("");
}

// ------------------------------------------------------- link operators
Env& attn_state::get_env(int n, int slot) {
  ATTN_REQUIRE(mapped_ready, ATTN_EINVAL, "Hamiltonian not mapped yet (call attn_map_hamiltonian)");
  Env& e = env[3 * n + slot];
  if (e.valid) return e;
  const Tree::Nbr& nb = tree.nbr[3 * n + slot];
  if (nb.kind == 0) {
    build_physical_env(n, slot);
  } else {
    const int c = nb.idx, t = nb.back;
    // the centre must not lie on the far side of this link
    const bool centre_far = (slot < 2) ? (tree.lo[c] <= tree.lo[centre] && tree.hi[centre] <= tree.hi[c])
                                       : !(tree.lo[n] <= tree.lo[centre] && tree.hi[centre] <= tree.hi[n]);
    ATTN_REQUIRE(!centre_far, ATTN_EINVAL, "link operators requested away from the isometry centre");
    for (int s = 0; s < 3; ++s)
      if (s != t) get_env(c, s);
    renormalise_into(n, slot);
  }
  e.valid = true;
  return e;
}

void attn_state::build_physical_env(int n, int slot) {
  Env& e = env[3 * n + slot];
  const int site = tree.nbr[3 * n + slot].idx;
  double hint[4] = {0, 0, 0, 0};
  bool has = false;
  std::vector<double> ops;
  e.open.clear();
  e.pos.clear();
  for (size_t q = 0; q < prods.size(); ++q) {
    const Prod& p = prods[q];
    int k = -1;
    for (int a = 0; a < p.n; ++a)
      if (p.site[a] == site) k = a;
    if (k < 0) continue;
    if (p.n == 1) {
      for (int i = 0; i < 4; ++i) hint[i] += p.op[0][i];
      has = true;
    } else {
      e.pos.push_back({(int)q, (int)e.open.size()});
      e.open.push_back((int)q);
      ops.insert(ops.end(), p.op[k], p.op[k] + 4);
    }
  }
  e.dim = 2;
  e.has_hint = has;
  e.hint.reserve(sizeof(double) * 4);
  ATTN_CHECK_CUDA(cudaMemcpyAsync(e.hint.p, hint, sizeof(hint), cudaMemcpyHostToDevice, ctx->stream));
  if (!ops.empty()) {
    e.ops.reserve(sizeof(double) * ops.size());
    ATTN_CHECK_CUDA(cudaMemcpyAsync(e.ops.p, ops.data(), sizeof(double) * ops.size(), cudaMemcpyHostToDevice,
                                    ctx->stream));
  }
}

void attn_state::renormalise_into(int n, int slot) {
  Env& out = env[3 * n + slot];
  const Tree::Nbr& nb = tree.nbr[3 * n + slot];
  const int c = nb.idx, t = nb.back;
  int xs[2], ni = 0;
  for (int s = 0; s < 3; ++s)
    if (s != t) xs[ni++] = s;
  const int x = xs[0], y = xs[1];
  const Env& Ex = env[3 * c + x];
  const Env& Ey = env[3 * c + y];
  const int d[3] = {dim(c, 0), dim(c, 1), dim(c, 2)};
  const long V = vol(c);
  const int dt = d[t];
  const double* Tc = tensor(c);

  // classify products
  std::vector<int> both, xonly, yonly, closed;
  std::vector<int> bx, by, cx, cy, xi, yi;
  {
    size_t i = 0, j = 0;
    auto outside = [&](int q) {
      const Prod& p = prods[q];
      for (int a = 0; a < p.n; ++a)
        if (tree.behind(c, t, p.site[a])) return true;
      return false;
    };
    while (i < Ex.pos.size() || j < Ey.pos.size()) {
      int qx = i < Ex.pos.size() ? Ex.pos[i].first : INT32_MAX;
      int qy = j < Ey.pos.size() ? Ey.pos[j].first : INT32_MAX;
      if (qx == qy) {
        if (outside(qx)) { both.push_back(qx); bx.push_back(Ex.pos[i].second); by.push_back(Ey.pos[j].second); }
        else { closed.push_back(qx); cx.push_back(Ex.pos[i].second); cy.push_back(Ey.pos[j].second); }
        ++i; ++j;
      } else if (qx < qy) {
        xonly.push_back(qx); xi.push_back(Ex.pos[i].second); ++i;
      } else {
        yonly.push_back(qy); yi.push_back(Ey.pos[j].second); ++j;
      }
    }
  }
  out.open.clear();
  out.open.insert(out.open.end(), both.begin(), both.end());
  out.open.insert(out.open.end(), xonly.begin(), xonly.end());
  out.open.insert(out.open.end(), yonly.begin(), yonly.end());
  out.pos.clear();
  for (size_t k = 0; k < out.open.size(); ++k) out.pos.push_back({out.open[k], (int)k});
  std::sort(out.pos.begin(), out.pos.end());
  out.dim = dt;
  const long osz = (long)dt * dt;
  if (!out.open.empty()) out.ops.reserve(sizeof(double) * out.open.size() * osz);

  const long budget = 1L << 26;  // doubles per intermediate
  const int chunk = (int)std::max<long>(1, std::min<long>(1024, budget / std::max<long>(V, 1)));
  renorm_batch(Tc, d, t, x, y, Ex.ops.as<double>(), bx, Ey.ops.as<double>(), by, out.ops.as<double>());
  renorm_batch(Tc, d, t, x, y, Ex.ops.as<double>(), xi, nullptr, {}, out.ops.as<double>() + (long)both.size() * osz);
  renorm_batch(Tc, d, t, x, y, nullptr, {}, Ey.ops.as<double>(), yi,
               out.ops.as<double>() + (long)(both.size() + xonly.size()) * osz);

  // internal operator: T^T (H_x (x) 1 + 1 (x) H_y + sum_closed A (x) B) T
  out.has_hint = Ex.has_hint || Ey.has_hint || !closed.empty();
  out.hint.reserve(sizeof(double) * osz);
  if (!out.has_hint) return;
  rw1.reserve(sizeof(double) * V);
  double* Wsum = rw1.as<double>();
  fill_f64(ctx, Wsum, V, 0.0);
  if (Ex.has_hint) mode_product_f64(ctx, d, x, Ex.hint.as<double>(), 1, Tc, 0, Wsum, 1.0);
  if (Ey.has_hint) mode_product_f64(ctx, d, y, Ey.hint.as<double>(), 1, Tc, 0, Wsum, 1.0);
  for (size_t r0 = 0; r0 < closed.size(); r0 += chunk) {
    const int Rc = (int)std::min<size_t>(chunk, closed.size() - r0);
    rw2.reserve(sizeof(double) * (size_t)Rc * V);
    double* W1 = rw2.as<double>();
    std::vector<int> sy(cy.begin() + r0, cy.begin() + r0 + Rc), sx(cx.begin() + r0, cx.begin() + r0 + Rc);
    upload_idx(ctx, idxbuf, sy);
    opsB.reserve(sizeof(double) * (size_t)Rc * d[y] * d[y]);
    gather_rows_f64(ctx, opsB.as<double>(), Ey.ops.as<double>(), idxbuf.as<int>(), Rc, (long)d[y] * d[y]);
    mode_product_f64(ctx, d, y, opsB.as<double>(), Rc, Tc, 0, W1, 0.0);
    upload_idx(ctx, idxbuf, sx);
    opsA.reserve(sizeof(double) * (size_t)Rc * d[x] * d[x]);
    gather_rows_f64(ctx, opsA.as<double>(), Ex.ops.as<double>(), idxbuf.as<int>(), Rc, (long)d[x] * d[x]);
    accumulate_slot_f64(ctx, d, x, opsA.as<double>(), Rc, W1, Wsum);
  }
  contract_tt(ctx, Tc, d, t, Wsum, 1, out.hint.as<double>());
}

// out[r] = T^T (A[ia[r]] on slot x (x) B[ib[r]] on slot y) T over slots x, y
// (open slot t); an empty index list means the identity on that slot.
void attn_state::renorm_batch(const double* Tc, const int d[3], int t, int x, int y, const double* Aops,
                              const std::vector<int>& ia, const double* Bops, const std::vector<int>& ib,
                              double* out) {
  const long V = (long)d[0] * d[1] * d[2];
  const long osz = (long)d[t] * d[t];
  const long budget = 1L << 26;  // doubles per intermediate
  const int chunk = (int)std::max<long>(1, std::min<long>(1024, budget / std::max<long>(V, 1)));
  const int R = (int)std::max(ia.size(), ib.size());
  for (int r0 = 0; r0 < R; r0 += chunk) {
    const int Rc = std::min(chunk, R - r0);
    rw1.reserve(sizeof(double) * (size_t)Rc * V);
    rw2.reserve(sizeof(double) * (size_t)Rc * V);
    double* W1 = rw1.as<double>();
    double* W2 = rw2.as<double>();
    const double* cur = Tc;
    long cur_stride = 0;
    if (!ib.empty()) {
      std::vector<int> sub(ib.begin() + r0, ib.begin() + r0 + Rc);
      upload_idx(ctx, idxbuf, sub);
      opsB.reserve(sizeof(double) * (size_t)Rc * d[y] * d[y]);
      gather_rows_f64(ctx, opsB.as<double>(), Bops, idxbuf.as<int>(), Rc, (long)d[y] * d[y]);
      mode_product_f64(ctx, d, y, opsB.as<double>(), Rc, cur, cur_stride, W1, 0.0);
      cur = W1;
      cur_stride = V;
    }
    if (!ia.empty()) {
      std::vector<int> sub(ia.begin() + r0, ia.begin() + r0 + Rc);
      upload_idx(ctx, idxbuf, sub);
      opsA.reserve(sizeof(double) * (size_t)Rc * d[x] * d[x]);
      gather_rows_f64(ctx, opsA.as<double>(), Aops, idxbuf.as<int>(), Rc, (long)d[x] * d[x]);
      double* dst = (cur == W1) ? W2 : W1;
      mode_product_f64(ctx, d, x, opsA.as<double>(), Rc, cur, cur_stride, dst, 0.0);
      cur = dst;
    }
    contract_tt(ctx, Tc, d, t, cur, Rc, out + (long)r0 * osz);
  }
}

// ------------------------------------------------------------------ H_eff
void attn_state::recycle(attn_heff* h) {
  if (!h) return;
  if (spare_heff) {
    delete h;
    return;
  }
  delete h->eg;  // a captured graph holds the old operators' launch parameters
  h->eg = nullptr;
  attn::tc_invalidate(h);
  spare_heff = h;
}

attn_heff* attn_state::build_heff(int n) {
  ATTN_REQUIRE(n == centre, ATTN_EINVAL, "H_eff requested away from the isometry centre");
  Env* E[3];
  for (int s = 0; s < 3; ++s) E[s] = &get_env(n, s);
  attn_heff* h = spare_heff ? spare_heff : new attn_heff();
  spare_heff = nullptr;
  h->ctx = ctx;
  for (int s = 0; s < 3; ++s) h->m[s] = dim(n, s);
  h->V = vol(n);
  for (int s = 0; s < 3; ++s) {
    h->has_hint[s] = E[s]->has_hint;
    if (E[s]->has_hint) {
      const long sz = (long)h->m[s] * h->m[s];
      h->hint[s].reserve(sizeof(double) * sz);
      copy_f64(ctx, h->hint[s].as<double>(), E[s]->hint.as<double>(), sz);
    }
  }
  // merge the three sorted product lists
  std::vector<int> ia[3], ib[3], it[3];
  {
    size_t i[3] = {0, 0, 0};
    while (true) {
      int q = INT32_MAX;
      for (int s = 0; s < 3; ++s)
        if (i[s] < E[s]->pos.size()) q = std::min(q, E[s]->pos[i[s]].first);
      if (q == INT32_MAX) break;
      int idx[3] = {-1, -1, -1};
      int mask = 0;
      for (int s = 0; s < 3; ++s)
        if (i[s] < E[s]->pos.size() && E[s]->pos[i[s]].first == q) {
          idx[s] = E[s]->pos[i[s]].second;
          mask |= 1 << s;
          ++i[s];
        }
      if (mask == 7) {
        for (int s = 0; s < 3; ++s) it[s].push_back(idx[s]);
      } else {
        int k = (mask == 3) ? 0 : (mask == 5) ? 1 : (mask == 6) ? 2 : -1;
        ATTN_REQUIRE(k >= 0, ATTN_EINVAL, "inconsistent link operators (product open on one link only)");
        ia[k].push_back(idx[kPairP[k]]);
        ib[k].push_back(idx[kPairQ[k]]);
      }
    }
  }
  for (int k = 0; k < 3; ++k) {
    const int p = kPairP[k], q = kPairQ[k];
    const int R = (int)ia[k].size();
    h->npair[k] = R;
    if (!R) continue;
    h->pa[k].reserve(sizeof(double) * (size_t)R * h->m[p] * h->m[p]);
    h->pb[k].reserve(sizeof(double) * (size_t)R * h->m[q] * h->m[q]);
    upload_idx(ctx, idxbuf, ia[k]);
    gather_rows_f64(ctx, h->pa[k].as<double>(), E[p]->ops.as<double>(), idxbuf.as<int>(), R, (long)h->m[p] * h->m[p]);
    upload_idx(ctx, idxbuf, ib[k]);
    gather_rows_f64(ctx, h->pb[k].as<double>(), E[q]->ops.as<double>(), idxbuf.as<int>(), R, (long)h->m[q] * h->m[q]);
  }
  h->ntrip = (int)it[0].size();
  if (h->ntrip) {
    for (int s = 0; s < 3; ++s) {
      h->tr[s].reserve(sizeof(double) * (size_t)h->ntrip * h->m[s] * h->m[s]);
      upload_idx(ctx, idxbuf, it[s]);
      gather_rows_f64(ctx, h->tr[s].as<double>(), E[s]->ops.as<double>(), idxbuf.as<int>(), h->ntrip,
                      (long)h->m[s] * h->m[s]);
    }
  }
  return h;
}

double attn_state::energy() {
  attn_heff* h = build_heff(centre);
  const long V = vol(centre);
  lw.wvec.reserve(sizeof(double) * V);
  ctx->scal.reserve(sizeof(double) * 64);
  double* y = lw.wvec.as<double>();
  double* s = ctx->scal.as<double>();
  try {
    h->apply_f64(tensor(centre), y);
  } catch (...) {
    delete h;
    throw;
  }
  recycle(h);
  multi_dot(ctx, tensor(centre), 1, V, y, s, nullptr);
  multi_dot(ctx, tensor(centre), 1, V, tensor(centre), s + 1, nullptr);
  double hv[2];
  ATTN_CHECK_CUDA(cudaMemcpyAsync(hv, s, sizeof(hv), cudaMemcpyDeviceToHost, ctx->stream));
  ATTN_CHECK_CUDA(cudaStreamSynchronize(ctx->stream));
  return hv[0] / hv[1];
}

double attn_state::local_step(int n) {
  ctx->prof_begin(4);
  move_centre(n);
  ctx->prof_end(4, 0.0);
  ctx->prof_begin(5);
  attn_heff* h = build_heff(n);
  ctx->prof_end(5, 0.0);
  const long V = vol(n);
  double result = 0.0;
  try {
    const attn_config& cfg = ctx->cfg;
    tmpT.reserve(sizeof(double) * V);
    double* v = tmpT.as<double>();
    copy_f64(ctx, v, tensor(n), V);
    // nodes whose links are too small for the tensor-core tiles use FP64 matvecs
    const attn_dtype dt = (cfg.matvec_dtype != ATTN_F64 && tc_supported(h)) ? cfg.matvec_dtype : ATTN_F64;
    MatVec mv_lo = [&](const double* a, double* b) { h->apply(a, b, dt); };
    MatVec mv64 = [&](const double* a, double* b) { h->apply_f64(a, b); };
    // current energy (FP64): known from the last local step unless H' or a tensor changed since
    double e_cur = energy_known;
    if (!std::isfinite(e_cur)) {
      ctx->prof_begin(7);
      lw2.wvec.reserve(sizeof(double) * V);
      ctx->scal.reserve(sizeof(double) * 64);
      double* s = ctx->scal.as<double>();
      h->apply_f64(tensor(n), lw2.wvec.as<double>());
      multi_dot(ctx, tensor(n), 1, V, lw2.wvec.as<double>(), s, nullptr);
      multi_dot(ctx, tensor(n), 1, V, tensor(n), s + 1, nullptr);
      double hv[2];
      ATTN_CHECK_CUDA(cudaMemcpyAsync(hv, s, sizeof(hv), cudaMemcpyDeviceToHost, ctx->stream));
      ATTN_CHECK_CUDA(cudaStreamSynchronize(ctx->stream));
      e_cur = hv[0] / hv[1];
      ctx->prof_end(7, 0.0);
    }
    ctx->prof_begin(6);
    LanczosResult r =
        timeout_first(ctx, h, [&] {
          return lanczos_lowest(ctx, mv_lo, v, V, cfg.lanczos_depth, cfg.lanczos_tol, lw,
                                dt != ATTN_F64 && cfg.lanczos_basis == 1);
        });
    ctx->prof_end(6, 0.0);
    double theta = r.theta;
    bool exact = (dt == ATTN_F64);
    if (dt != ATTN_F64 && cfg.refine_steps > 0) {
      // FP64 Rayleigh-Ritz with low-precision corrections: theta and v are FP64-exact for this H_eff
      ctx->prof_begin(7);
      theta = timeout_first(ctx, h, [&] {
                return refine_eig(ctx, mv64, mv_lo, v, V, cfg.refine_steps, cfg.refine_inner, cfg.refine_tol, rfw);
              }).theta;
      ctx->prof_end(7, 0.0);
      exact = true;
    }
    check_device_errors(ctx, h);
    if (theta <= e_cur + 1e-14 * std::fabs(e_cur)) {
      std::swap(T[n], tmpT);
      invalidate_from(n);
      result = theta;
      energy_known = exact ? theta : std::nan("");
    } else {
      result = e_cur;
      energy_known = e_cur;
    }
  } catch (...) {
    delete h;
    throw;
  }
  recycle(h);
  return result;
}

double attn_state::isometry_error() {
  double err = 0.0;
  ctx->scal.reserve(sizeof(double) * 64);
  for (int n = 0; n < tree.n_nodes; ++n) {
    if (n == centre) continue;
    std::vector<int> p = tree.path(n, centre);
    const int s = tree.slot_towards(n, p[1]);
    const int d[3] = {dim(n, 0), dim(n, 1), dim(n, 2)};
    const int k = d[s];
    const long M = vol(n) / k;
    colbuf.reserve(sizeof(double) * vol(n));
    rbuf.reserve(sizeof(double) * k * k);
    tensor_to_columns(ctx, tensor(n), d, s, colbuf.as<double>());
    GemmF64 g;
    g.M = g.N = k;
    g.K = (int)M;
    g.A = colbuf.as<double>(); g.aM = M; g.aK = 1;
    g.B = colbuf.as<double>(); g.bK = 1; g.bN = M;
    g.C = rbuf.as<double>(); g.cM = k; g.cN = 1;
    gemm_f64(ctx, g);
    gram_err_kernel<<<1, 256, 0, ctx->stream>>>(rbuf.as<double>(), k, ctx->scal.as<double>());
    ctx->launches++;
    double e = 0;
    ATTN_CHECK_CUDA(cudaMemcpyAsync(&e, ctx->scal.p, sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    ATTN_CHECK_CUDA(cudaStreamSynchronize(ctx->stream));
    err = std::max(err, e);
  }
  return err;
}
