// Measurement of observables of the aTTN (Sec. 5, Eq. obs, Eq. corrmat).
//
// An observable o = o_1 (x) ... (x) o_n of one-site operators on distinct sites
// is measured on the aTTN as <psi_TTN| D^T o D |psi_TTN> (Eq. obs with the
// convention |psi_aTTN> = D |psi_TTN> of the Hamiltonian mapping): every
// disentangler u_k touching the observable's sites conjugates the part of o on
// its pair (i_k, j_k), O'_k = u_k^T (o_i (x) o_j) u_k (a missing factor is the
// identity), which is split exactly into rank-1 products a_r (x) b_r across the
// pair (Sec. 4.3); factors on sites outside the disentangler layer stay as they
// are. The mapped observable is thus a sum of products of one-site factors (a
// two-body correlator touching two disentanglers spans four sites, Fig.
// de-contr-scenarios; an observable on n <= 4 sites at most 2n), and each
// product is an expectation value of the TTN: its
// factors are renormalised link by link towards the isometry centre and
// contracted there -- only the links on the paths from the factors' sites to the
// centre are touched (the sub-tree of Sec. 5.1), and partial products shared by
// several probes are computed once.
#include <algorithm>
#include <array>
#include <cmath>
#include <map>

#include "state.h"

using namespace attn;

namespace attn {
namespace {

// R = U diag(s) V^T of a 4 x 4 matrix by one-sided Jacobi on the columns.
void svd4(const double* A, double* U, double* s, double* V) {
  double B[16];
  for (int i = 0; i < 16; ++i) {
    B[i] = A[i];
    V[i] = (i % 5 == 0) ? 1.0 : 0.0;
  }
  for (int sweep = 0; sweep < 60; ++sweep) {
    double off = 0.0;
    for (int p = 0; p < 4; ++p)
      for (int q = p + 1; q < 4; ++q) {
        double a = 0, b = 0, c = 0;
        for (int r = 0; r < 4; ++r) {
          a += B[r * 4 + p] * B[r * 4 + p];
          b += B[r * 4 + q] * B[r * 4 + q];
          c += B[r * 4 + p] * B[r * 4 + q];
        }
        if (c == 0.0 || a == 0.0 || b == 0.0) continue;
        const double ratio = std::fabs(c) / std::sqrt(a * b);
        if (!(ratio > 1e-16)) continue;
        off = std::max(off, ratio);
        const double zeta = (b - a) / (2.0 * c);
        const double t = (zeta >= 0 ? 1.0 : -1.0) / (std::fabs(zeta) + std::sqrt(1.0 + zeta * zeta));
        const double cs = 1.0 / std::sqrt(1.0 + t * t), sn = cs * t;
        for (int r = 0; r < 4; ++r) {
          double x = B[r * 4 + p], y = B[r * 4 + q];
          B[r * 4 + p] = cs * x - sn * y;
          B[r * 4 + q] = sn * x + cs * y;
          x = V[r * 4 + p];
          y = V[r * 4 + q];
          V[r * 4 + p] = cs * x - sn * y;
          V[r * 4 + q] = sn * x + cs * y;
        }
      }
    if (off < 1e-15) break;
  }
  for (int k = 0; k < 4; ++k) {
    double n = 0;
    for (int r = 0; r < 4; ++r) n += B[r * 4 + k] * B[r * 4 + k];
    s[k] = std::sqrt(n);
    for (int r = 0; r < 4; ++r) U[r * 4 + k] = s[k] > 0 ? B[r * 4 + k] / s[k] : 0.0;
  }
}

// One-site factor lists of a mapped observable: one list of alternatives per block
// (a disentangler pair contributes up to four rank-1 products, a free site one).
struct Block {
  std::vector<std::vector<ProbeFactor>> alts;  // alternatives, each 1 or 2 factors
};

}  // namespace
}  // namespace attn

std::vector<double> attn_state::measure(int n_obs, const int* nsites, const int* sites, const double* ops) {
  std::vector<int> owner(model.n_sites, -1);
  for (size_t k = 0; k < des.size(); ++k) owner[des[k].first] = owner[des[k].second] = (int)k;
  std::vector<ProbeFactor> F;
  std::vector<Probe> P;
  std::vector<int> obs_of;  // probe -> observable
  // identical factors share one id, so that their renormalised partial products
  // (e.g. o^a_i of a whole row of the correlation matrix) are computed once
  std::map<std::array<double, 5>, int> fids;
  auto factor_id = [&](const ProbeFactor& f) {
    const std::array<double, 5> key = {(double)f.site, f.op[0], f.op[1], f.op[2], f.op[3]};
    auto it = fids.find(key);
    if (it != fids.end()) return it->second;
    F.push_back(f);
    return fids[key] = (int)F.size() - 1;
  };
  for (int o = 0; o < n_obs; ++o) {
    const int n = nsites[o];
    ATTN_REQUIRE(n >= 1 && n <= 4, ATTN_EINVAL, "an observable acts on 1..4 sites");
    const int* S = sites + 4L * o;
    const double* Op = ops + 16L * o;
    for (int a = 0; a < n; ++a) {
      ATTN_REQUIRE(S[a] >= 0 && S[a] < model.n_sites, ATTN_EINVAL, "observable site out of range");
      for (int b = 0; b < a; ++b) ATTN_REQUIRE(S[a] != S[b], ATTN_EINVAL, "observable sites must be distinct");
      for (int e = 0; e < 4; ++e) ATTN_REQUIRE(std::isfinite(Op[4 * a + e]), ATTN_ENONFINITE, "non-finite observable");
    }
    std::vector<Block> blocks;
    std::vector<int> done_de;
    int support = 0;
    for (int a = 0; a < n; ++a) {
      const int k = owner[S[a]];
      if (k < 0) {
        Block b;
        ProbeFactor f;
        f.site = S[a];
        std::copy(Op + 4 * a, Op + 4 * a + 4, f.op);
        b.alts.push_back({f});
        blocks.push_back(b);
        support += 1;
        continue;
      }
      if (std::find(done_de.begin(), done_de.end(), k) != done_de.end()) continue;
      done_de.push_back(k);
      const int i = des[k].first, j = des[k].second;
      double oi[4] = {1, 0, 0, 1}, oj[4] = {1, 0, 0, 1};
      for (int c = 0; c < n; ++c) {
        if (S[c] == i) std::copy(Op + 4 * c, Op + 4 * c + 4, oi);
        if (S[c] == j) std::copy(Op + 4 * c, Op + 4 * c + 4, oj);
      }
      // O = oi (x) oj on (i, j), i most significant; O' = u^T O u
      double O[16], W[16], Om[16];
      for (int r = 0; r < 4; ++r)
        for (int c = 0; c < 4; ++c) O[r * 4 + c] = oi[(r >> 1) * 2 + (c >> 1)] * oj[(r & 1) * 2 + (c & 1)];
      const double* u = us[k].data();
      for (int r = 0; r < 4; ++r)
        for (int c = 0; c < 4; ++c) {
          double acc = 0;
          for (int q = 0; q < 4; ++q) acc += O[r * 4 + q] * u[q * 4 + c];
          W[r * 4 + c] = acc;
        }
      for (int r = 0; r < 4; ++r)
        for (int c = 0; c < 4; ++c) {
          double acc = 0;
          for (int q = 0; q < 4; ++q) acc += u[q * 4 + r] * W[q * 4 + c];
          Om[r * 4 + c] = acc;
        }
      // R[(a_i b_i)][(a_j b_j)] = O'[(a_i a_j)][(b_i b_j)], split R = sum_r s_r U_r V_r^T
      double R[16], U[16], sv[4], V[16];
      for (int ai = 0; ai < 2; ++ai)
        for (int aj = 0; aj < 2; ++aj)
          for (int bi = 0; bi < 2; ++bi)
            for (int bj = 0; bj < 2; ++bj) R[(ai * 2 + bi) * 4 + aj * 2 + bj] = Om[(ai * 2 + aj) * 4 + bi * 2 + bj];
      svd4(R, U, sv, V);
      const double smax = std::max(std::max(sv[0], sv[1]), std::max(sv[2], sv[3]));
      Block b;
      for (int r = 0; r < 4; ++r) {
        if (!(sv[r] > 1e-14 * smax)) continue;
        ProbeFactor fi, fj;
        fi.site = i;
        fj.site = j;
        for (int e = 0; e < 4; ++e) {
          fi.op[e] = sv[r] * U[e * 4 + r];
          fj.op[e] = V[e * 4 + r];
        }
        b.alts.push_back({fi, fj});
      }
      blocks.push_back(b);
      support += 2;
    }
    ATTN_REQUIRE(support <= 8, ATTN_EINVAL, "observable support above eight sites");
    // every combination of one alternative per block is one probe
    bool zero = false;
    for (const Block& b : blocks) zero = zero || b.alts.empty();
    if (zero) continue;  // the mapped observable vanishes
    std::vector<int> pick(blocks.size(), 0);
    while (true) {
      Probe p;
      p.n = 0;
      for (int& f : p.f) f = -1;
      for (size_t bi = 0; bi < blocks.size(); ++bi)
        for (const ProbeFactor& f : blocks[bi].alts[pick[bi]]) p.f[p.n++] = factor_id(f);
      P.push_back(p);
      obs_of.push_back(o);
      size_t bi = 0;
      for (; bi < blocks.size(); ++bi) {
        if (++pick[bi] < (int)blocks[bi].alts.size()) break;
        pick[bi] = 0;
      }
      if (bi == blocks.size()) break;
    }
  }
  std::vector<double> out(n_obs, 0.0);
  if (P.empty()) return out;
  DevBuf vals;
  probe_expectations(F, P, vals);
  std::vector<double> pv(P.size());
  ATTN_CHECK_CUDA(cudaMemcpyAsync(pv.data(), vals.p, sizeof(double) * pv.size(), cudaMemcpyDeviceToHost, ctx->stream));
  ATTN_CHECK_CUDA(cudaStreamSynchronize(ctx->stream));
  for (size_t q = 0; q < P.size(); ++q) out[obs_of[q]] += pv[q];
  for (double v : out) ATTN_REQUIRE(std::isfinite(v), ATTN_ENONFINITE, "non-finite expectation value");
  return out;
}
