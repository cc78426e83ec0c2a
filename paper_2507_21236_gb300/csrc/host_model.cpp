// Host-side geometry and Hamiltonian bookkeeping of the aTTN (no device code).
//
//  - Site order: classic Hilbert-curve d2xy mapping (Sec. 6).
//  - Models: square-lattice TFIM H = -sum Z Z - h sum X (Eq. qising, coupling
//    on Z) and triangular-lattice Heisenberg with S = sigma/2 (Eq. xxz).
//    One-site terms on the same site are summed (Sec. 3.3).
//  - Tree: layers 1..nL = log2(N)-1, a layer-l node covers 2^l consecutive
//    sites, the two top nodes share the top link, the link above a layer-l
//    node has dimension min(2^(2^l), m) (Sec. 3.1).
//  - Disentangler placement: greedy over interaction bonds, highest supported
//    link first, under restrictions (1) one disentangler per term and (2) no
//    untruncated supported link (Secs. 6.1.1-6.1.2).
//  - Mapping H' = D^T H D per term (Sec. 4.3, Algorithm 1): case (a)/(b) by
//    embedding the term and u on the union of sites.
//  - Rank-1 split of each mapped term by successive SVDs (one-sided Jacobi),
//    at most d^2 = 4 products for a two-site term (Sec. 4.3); optionally terms on
//    the same sites are summed first (the compression suggested in Sec. 6.2.2).
#include <algorithm>
#include <array>
#include <cmath>
#include <cstring>
#include <map>
#include <set>

#include "attn_internal.h"

namespace attn {

void hilbert_d2xy(int n, int d, int* xo, int* yo) {
  int x = 0, y = 0, t = d;
  for (int s = 1; s < n; s *= 2) {
    int rx = 1 & (t / 2);
    int ry = 1 & (t ^ rx);
    if (ry == 0) {
      if (rx == 1) { x = s - 1 - x; y = s - 1 - y; }
      std::swap(x, y);
    }
    x += s * rx;
    y += s * ry;
    t /= 4;
  }
  *xo = x;
  *yo = y;
}

static const double kX[4] = {0, 1, 1, 0};
static const double kZ[4] = {1, 0, 0, -1};
static const double kIY[4] = {0, 1, -1, 0};

static std::vector<double> kron2(const double* a, const double* b) {
  std::vector<double> out(16);
  for (int i = 0; i < 2; ++i)
    for (int j = 0; j < 2; ++j)
      for (int k = 0; k < 2; ++k)
        for (int l = 0; l < 2; ++l) out[(i * 2 + k) * 4 + (j * 2 + l)] = a[i * 2 + j] * b[k * 2 + l];
  return out;
}

static void lattice_bonds(int L, bool tri, std::vector<std::pair<int, int>>& bonds) {
  ATTN_REQUIRE(L >= 2 && (L & (L - 1)) == 0, ATTN_EINVAL, "L must be a power of two >= 2");
  std::vector<int> idx(L * L);
  for (int d = 0; d < L * L; ++d) {
    int x, y;
    hilbert_d2xy(L, d, &x, &y);
    idx[x * L + y] = d;
  }
  int steps[3][2] = {{1, 0}, {0, 1}, {1, 1}};
  int ns = tri ? 3 : 2;
  for (int x = 0; x < L; ++x)
    for (int y = 0; y < L; ++y)
      for (int k = 0; k < ns; ++k) {
        int x2 = x + steps[k][0], y2 = y + steps[k][1];
        if (x2 >= L || y2 >= L) continue;
        int a = idx[x * L + y], b = idx[x2 * L + y2];
        bonds.emplace_back(std::min(a, b), std::max(a, b));
      }
  std::sort(bonds.begin(), bonds.end());
}

static void sum_local(Model& M) {
  std::map<int, std::vector<double>> local;
  std::vector<Term> rest;
  for (auto& t : M.terms) {
    if (t.n == 1) {
      auto& acc = local[t.site[0]];
      if (acc.empty()) acc.assign(4, 0.0);
      for (int i = 0; i < 4; ++i) acc[i] += t.op[i];
    } else {
      rest.push_back(t);
    }
  }
  for (auto& kv : local) {
    Term t;
    t.n = 1;
    t.site[0] = kv.first;
    t.op = kv.second;
    rest.push_back(t);
  }
  M.terms.swap(rest);
}

void build_tfim(Model& M, int L, double h) {
  M = Model();
  M.n_sites = L * L;
  lattice_bonds(L, false, M.bonds);
  for (auto& b : M.bonds) {
    Term t;
    t.n = 2;
    t.site[0] = b.first;
    t.site[1] = b.second;
    t.op = kron2(kZ, kZ);
    for (auto& v : t.op) v = -v;
    M.terms.push_back(t);
  }
  for (int s = 0; s < M.n_sites; ++s) {
    Term t;
    t.n = 1;
    t.site[0] = s;
    t.op.assign(kX, kX + 4);
    for (auto& v : t.op) v *= -h;
    M.terms.push_back(t);
  }
  sum_local(M);
}

void build_tri_heisenberg(Model& M, int L, double J) {
  M = Model();
  M.n_sites = L * L;
  lattice_bonds(L, true, M.bonds);
  for (auto& b : M.bonds) {
    const double* ops[3] = {kX, kIY, kZ};
    const double sg[3] = {0.25 * J, -0.25 * J, 0.25 * J};
    for (int a = 0; a < 3; ++a) {
      Term t;
      t.n = 2;
      t.site[0] = b.first;
      t.site[1] = b.second;
      t.op = kron2(ops[a], ops[a]);
      for (auto& v : t.op) v *= sg[a];
      M.terms.push_back(t);
    }
  }
}

void build_generic(Model& M, int n_sites, int n_terms, const int* nsites, const int* sites, const double* ops) {
  M = Model();
  ATTN_REQUIRE(n_sites >= 4 && (n_sites & (n_sites - 1)) == 0, ATTN_EINVAL, "n_sites must be a power of two >= 4");
  M.n_sites = n_sites;
  std::set<std::pair<int, int>> bonds;
  for (int t = 0; t < n_terms; ++t) {
    Term term;
    term.n = nsites[t];
    ATTN_REQUIRE(term.n >= 1 && term.n <= 3, ATTN_EINVAL, "term sites must be 1..3");
    for (int k = 0; k < term.n; ++k) {
      term.site[k] = sites[3 * t + k];
      ATTN_REQUIRE(term.site[k] >= 0 && term.site[k] < n_sites, ATTN_EINVAL, "term site out of range");
      if (k) ATTN_REQUIRE(term.site[k] > term.site[k - 1], ATTN_EINVAL, "term sites must ascend");
    }
    int D = 1 << term.n;
    term.op.assign(ops + 64L * t, ops + 64L * t + D * D);
    for (double v : term.op) ATTN_REQUIRE(std::isfinite(v), ATTN_ENONFINITE, "non-finite term operator");
    if (term.n == 2) bonds.insert({term.site[0], term.site[1]});
    M.terms.push_back(term);
  }
  M.bonds.assign(bonds.begin(), bonds.end());
  sum_local(M);
}

// ------------------------------------------------------------------- tree
static int cap_dim(int exp2, int m) {  // min(2^(2^exp2), m)
  if (exp2 >= 5) return m;
  long v = 1L << (1 << exp2);
  return (int)std::min<long>(v, m);
}

void Tree::build(int N, int m_) {
  ATTN_REQUIRE(N >= 4 && (N & (N - 1)) == 0, ATTN_EINVAL, "number of sites must be a power of two >= 4");
  ATTN_REQUIRE(m_ >= 2, ATTN_EINVAL, "bond dimension must be >= 2");
  n_sites = N;
  m = m_;
  nL = 0;
  while ((2 << nL) < N) ++nL;  // 2^(nL+1) == N
  layer.clear(); index.clear(); lo.clear(); hi.clear();
  for (int l = 1; l <= nL; ++l)
    for (int j = 0; j < (N >> l); ++j) {
      layer.push_back(l);
      index.push_back(j);
      lo.push_back(j << l);
      hi.push_back((j + 1) << l);
    }
  n_nodes = (int)layer.size();
  nbr.assign(3 * n_nodes, Nbr{0, 0, 0});
  shape.assign(3 * n_nodes, 0);
  for (int n = 0; n < n_nodes; ++n) {
    int l = layer[n], j = index[n];
    if (l == 1) {
      nbr[3 * n + 0] = {0, 2 * j, -1};
      nbr[3 * n + 1] = {0, 2 * j + 1, -1};
      shape[3 * n] = shape[3 * n + 1] = 2;
    } else {
      nbr[3 * n + 0] = {1, id(l - 1, 2 * j), 2};
      nbr[3 * n + 1] = {1, id(l - 1, 2 * j + 1), 2};
      shape[3 * n] = shape[3 * n + 1] = cap_dim(l - 1, m);
    }
    if (l < nL) {
      nbr[3 * n + 2] = {1, id(l + 1, j / 2), j % 2};
      shape[3 * n + 2] = cap_dim(l, m);
    } else {
      nbr[3 * n + 2] = {1, id(l, 1 - j), 2};
      shape[3 * n + 2] = cap_dim(nL, m);
    }
  }
}

int Tree::id(int l, int j) const {
  int base = 0;
  for (int k = 1; k < l; ++k) base += n_sites >> k;
  return base + j;
}

int Tree::slot_towards(int n, int nb) const {
  for (int s = 0; s < 3; ++s)
    if (nbr[3 * n + s].kind == 1 && nbr[3 * n + s].idx == nb) return s;
  throw Error{ATTN_EINVAL, "nodes are not adjacent"};
}

std::vector<int> Tree::path(int a, int b) const {
  if (a == b) return {a};
  auto up = [&](int n) {
    std::vector<int> c{n};
    while (layer[c.back()] < nL) c.push_back(nbr[3 * c.back() + 2].idx);
    return c;
  };
  std::vector<int> ua = up(a), ub = up(b);
  std::vector<int> out;
  if (ua.back() != ub.back()) {
    out = ua;
    out.insert(out.end(), ub.rbegin(), ub.rend());
    return out;
  }
  std::set<int> sb(ub.begin(), ub.end());
  size_t i = 0;
  while (!sb.count(ua[i])) ++i;
  int lca = ua[i];
  out.assign(ua.begin(), ua.begin() + i + 1);
  size_t k = std::find(ub.begin(), ub.end(), lca) - ub.begin();
  for (size_t q = k; q-- > 0;) out.push_back(ub[q]);
  return out;
}

std::vector<int> Tree::post_order() const {
  std::vector<int> order;
  std::vector<std::pair<int, int>> st;  // node, state
  for (int top : {top0(), top1()}) {
    st.push_back({top, 0});
    while (!st.empty()) {
      auto [n, s] = st.back();
      st.pop_back();
      if (layer[n] == 1 || s == 2) {
        order.push_back(n);
        continue;
      }
      st.push_back({n, s + 1});
      st.push_back({nbr[3 * n + s].idx, 0});
    }
  }
  return order;
}

int Tree::lca_layer(int i, int j) const {
  for (int l = 1; l <= nL; ++l)
    if ((i >> l) == (j >> l)) return l;
  return nL + 1;
}

bool Tree::behind(int n, int slot, int s) const {
  const Nbr& nb = nbr[3 * n + slot];
  if (nb.kind == 0) return s == nb.idx;
  if (slot < 2) return s >= lo[nb.idx] && s < hi[nb.idx];
  return !(s >= lo[n] && s < hi[n]);
}

// ------------------------------------------------------------- placement
std::vector<std::pair<int, int>> place_disentanglers(const Tree& T, const Model& M, int max_de) {
  std::vector<std::pair<int, int>> cands = M.bonds;
  std::stable_sort(cands.begin(), cands.end(), [&](const std::pair<int, int>& a, const std::pair<int, int>& b) {
    int la = T.lca_layer(a.first, a.second), lb = T.lca_layer(b.first, b.second);
    if (la != lb) return la > lb;
    return a < b;
  });
  std::vector<std::vector<int>> site_terms(M.n_sites);
  for (size_t t = 0; t < M.terms.size(); ++t)
    for (int k = 0; k < M.terms[t].n; ++k) site_terms[M.terms[t].site[k]].push_back((int)t);
  std::vector<int> owner(M.n_sites, -1);
  std::vector<std::pair<int, int>> placed;
  for (auto& c : cands) {
    if ((int)placed.size() >= max_de) break;
    int i = c.first, j = c.second;
    if (owner[i] >= 0 || owner[j] >= 0) continue;
    int l = T.lca_layer(i, j);
    int e = l - 1;  // supported link has max dim 2^(2^e)
    bool trunc = e >= 5 || (long)T.m < (1L << (1 << e));
    if (!trunc) continue;
    bool ok = true;
    for (int s : {i, j}) {
      for (int t : site_terms[s]) {
        const Term& tm = M.terms[t];
        for (int k = 0; k < tm.n; ++k)
          if (owner[tm.site[k]] >= 0) ok = false;
      }
    }
    if (!ok) continue;
    owner[i] = owner[j] = (int)placed.size();
    placed.push_back(c);
  }
  return placed;
}

// ---------------------------------------------------------------- mapping
// Embed operator on ascending `sites` (k) into ascending `target` (kt).
static std::vector<double> embed(const std::vector<double>& op, const std::vector<int>& sites,
                                 const std::vector<int>& target) {
  int k = (int)sites.size(), kt = (int)target.size();
  int D = 1 << kt;
  std::vector<int> pos(k);
  for (int a = 0; a < k; ++a) pos[a] = (int)(std::find(target.begin(), target.end(), sites[a]) - target.begin());
  std::vector<double> out((size_t)D * D, 0.0);
  for (int r = 0; r < D; ++r)
    for (int c = 0; c < D; ++c) {
      // spins of target (first most significant)
      bool same_rest = true;
      int ri = 0, ci = 0;
      for (int b = 0; b < kt; ++b) {
        int rb = (r >> (kt - 1 - b)) & 1, cb = (c >> (kt - 1 - b)) & 1;
        int a = -1;
        for (int q = 0; q < k; ++q)
          if (pos[q] == b) a = q;
        if (a < 0) {
          if (rb != cb) same_rest = false;
        } else {
          ri |= rb << (k - 1 - a);
          ci |= cb << (k - 1 - a);
        }
      }
      if (same_rest) out[(size_t)r * D + c] = op[(size_t)ri * (1 << k) + ci];
    }
  return out;
}

std::vector<Term> map_terms(const Model& M, const std::vector<std::pair<int, int>>& des,
                            const std::vector<std::vector<double>>& us) {
  std::vector<int> owner(M.n_sites, -1);
  for (size_t k = 0; k < des.size(); ++k) owner[des[k].first] = owner[des[k].second] = (int)k;
  std::vector<Term> out;
  out.reserve(M.terms.size());
  for (const Term& t : M.terms) {
    int k = -1;
    for (int a = 0; a < t.n; ++a) {
      int o = owner[t.site[a]];
      if (o >= 0) {
        ATTN_REQUIRE(k < 0 || k == o, ATTN_EINVAL, "a term touches two disentanglers (restriction 1)");
        k = o;
      }
    }
    if (k < 0) {
      out.push_back(t);
      continue;
    }
    std::vector<int> sites(t.site, t.site + t.n);
    std::set<int> ts(sites.begin(), sites.end());
    ts.insert(des[k].first);
    ts.insert(des[k].second);
    std::vector<int> target(ts.begin(), ts.end());
    std::vector<double> h = embed(t.op, sites, target);
    std::vector<double> u = embed(us[k], {des[k].first, des[k].second}, target);
    int D = 1 << target.size();
    // h' = u^T h u
    std::vector<double> hu((size_t)D * D, 0.0), res((size_t)D * D, 0.0);
    for (int i = 0; i < D; ++i)
      for (int j = 0; j < D; ++j) {
        double s = 0;
        for (int q = 0; q < D; ++q) s += h[i * D + q] * u[q * D + j];
        hu[i * D + j] = s;
      }
    for (int i = 0; i < D; ++i)
      for (int j = 0; j < D; ++j) {
        double s = 0;
        for (int q = 0; q < D; ++q) s += u[q * D + i] * hu[q * D + j];
        res[i * D + j] = s;
      }
    Term nt;
    nt.n = (int)target.size();
    for (int a = 0; a < nt.n; ++a) nt.site[a] = target[a];
    nt.op = res;
    out.push_back(nt);
  }
  return out;
}

std::vector<Term> compress_terms(const std::vector<Term>& terms) {
  std::map<std::vector<int>, size_t> at;
  std::vector<Term> out;
  for (const Term& t : terms) {
    std::vector<int> key(t.site, t.site + t.n);
    auto it = at.find(key);
    if (it == at.end()) {
      at[key] = out.size();
      out.push_back(t);
    } else {
      std::vector<double>& op = out[it->second].op;
      for (size_t i = 0; i < op.size(); ++i) op[i] += t.op[i];
    }
  }
  return out;
}

// One-sided Jacobi: orthogonalise the `nc` columns of B (rows x nc, row-major),
// accumulating the rotations into J (nc x nc, row-major). Columns of B become
// B_orig J with mutually orthogonal columns.
static void jacobi_cols(std::vector<double>& B, int rows, int nc, std::vector<double>& J) {
  J.assign((size_t)nc * nc, 0.0);
  for (int i = 0; i < nc; ++i) J[i * nc + i] = 1.0;
  for (int sweep = 0; sweep < 60; ++sweep) {
    double off = 0.0;
    for (int p = 0; p < nc; ++p)
      for (int q = p + 1; q < nc; ++q) {
        double a = 0, b = 0, c = 0;
        for (int r = 0; r < rows; ++r) {
          double x = B[r * nc + p], y = B[r * nc + q];
          a += x * x;
          b += y * y;
          c += x * y;
        }
        if (c == 0.0) continue;
        double ratio = std::fabs(c) / std::sqrt(a * b);
        if (!(ratio > 1e-16)) continue;
        off = std::max(off, ratio);
        double zeta = (b - a) / (2.0 * c);
        double t = (zeta >= 0 ? 1.0 : -1.0) / (std::fabs(zeta) + std::sqrt(1.0 + zeta * zeta));
        double cs = 1.0 / std::sqrt(1.0 + t * t), sn = cs * t;
        for (int r = 0; r < rows; ++r) {
          double x = B[r * nc + p], y = B[r * nc + q];
          B[r * nc + p] = cs * x - sn * y;
          B[r * nc + q] = sn * x + cs * y;
        }
        for (int r = 0; r < nc; ++r) {
          double x = J[r * nc + p], y = J[r * nc + q];
          J[r * nc + p] = cs * x - sn * y;
          J[r * nc + q] = sn * x + cs * y;
        }
      }
    if (off < 1e-15) break;
  }
}

// Split a tensor t with first index of size 4 (current site's (s, s') pair)
// and `rest` trailing entries into sum_k head_k (x) tail_k.
static void split_rec(const std::vector<double>& t, int nsite, std::vector<std::vector<std::array<double, 4>>>& out,
                      std::vector<std::array<double, 4>>& prefix) {
  if (nsite == 1) {
    std::array<double, 4> h;
    for (int i = 0; i < 4; ++i) h[i] = t[i];
    prefix.push_back(h);
    out.push_back(prefix);
    prefix.pop_back();
    return;
  }
  int rest = (int)t.size() / 4;
  // B = t^T : rest x 4
  std::vector<double> B((size_t)rest * 4);
  for (int i = 0; i < 4; ++i)
    for (int r = 0; r < rest; ++r) B[r * 4 + i] = t[(size_t)i * rest + r];
  std::vector<double> J;
  jacobi_cols(B, rest, 4, J);
  double sig[4], smax = 0;
  for (int k = 0; k < 4; ++k) {
    double s = 0;
    for (int r = 0; r < rest; ++r) s += B[r * 4 + k] * B[r * 4 + k];
    sig[k] = std::sqrt(s);
    smax = std::max(smax, sig[k]);
  }
  if (smax == 0.0) return;
  for (int k = 0; k < 4; ++k) {
    if (!(sig[k] > 1e-14 * smax)) continue;
    std::array<double, 4> h;
    for (int i = 0; i < 4; ++i) h[i] = J[i * 4 + k] * sig[k];
    std::vector<double> tail(rest);
    for (int r = 0; r < rest; ++r) tail[r] = B[r * 4 + k] / sig[k];
    prefix.push_back(h);
    split_rec(tail, nsite - 1, out, prefix);
    prefix.pop_back();
  }
}

std::vector<Prod> split_products(const std::vector<Term>& terms) {
  std::vector<Prod> out;
  for (size_t ti = 0; ti < terms.size(); ++ti) {
    const Term& t = terms[ti];
    int k = t.n, D = 1 << k;
    // reorder op[(s1..sk),(s1'..sk')] into (s1 s1')(s2 s2')...
    std::vector<double> r((size_t)D * D);
    for (int a = 0; a < D; ++a)
      for (int b = 0; b < D; ++b) {
        int idx = 0;
        for (int q = 0; q < k; ++q) {
          int sa = (a >> (k - 1 - q)) & 1, sb = (b >> (k - 1 - q)) & 1;
          idx = idx * 4 + sa * 2 + sb;
        }
        r[idx] = t.op[(size_t)a * D + b];
      }
    std::vector<std::vector<std::array<double, 4>>> parts;
    std::vector<std::array<double, 4>> prefix;
    split_rec(r, k, parts, prefix);
    for (auto& p : parts) {
      Prod pr;
      pr.term = (int)ti;
      pr.n = k;
      for (int q = 0; q < k; ++q) {
        pr.site[q] = t.site[q];
        for (int i = 0; i < 4; ++i) pr.op[q][i] = p[q][i];
      }
      out.push_back(pr);
    }
  }
  return out;
}

}  // namespace attn
