// Disentangler update on the GPU (Sec. 4.1: Eqs. energy, contracted, cost
// function; Sec. 4.2: environments of a disentangler).
//
// With restriction (1) the energy splits as E = sum_k E_k(u_k) + const. For a
// disentangler u on sites (i, j) and an original term h_p touching i or j:
//  - if h_p lives on {i, j} only, with C_p its 4x4 form on (i, j):
//        E_p(u) = Tr(rho_ij u^T C_p u);
//  - if h_p also touches a third site e, write h_p = sum_r C_r (x) f_r across
//    (ij)|e (exact SVD split, r <= 4) and M_r = Tr_e[rho_ije (1 (x) f_r)]:
//        E_p(u) = sum_r Tr(M_r u^T C_r u).
// Fixing the transposed factor at u_old makes the energy linear in u,
// E = Tr(u Gamma) (Eq. contracted) with
//        Gamma = sum_p sum_r M_r u_old^T C_r - (sum_p lambda_p) rho_ij u_old^T,
// where every term is shifted by lambda_p = ||h_p||_2 (negative semidefinite
// h~_p; a u-independent constant). The minimiser is u = -V W^T for
// Gamma = W sigma V^T (Eq. cost function); steps are accepted while the true
// E_k does not increase, at most de_max_iter of them, stopping when the
// relative change falls below de_rel_dev.
//
// rho_ij and the M_r are expectation values of products of one-site factors
// (matrix units on i and j, f_r on e). They are computed by renormalising the
// factors from their sites to the isometry centre along the tree (the path
// contraction of Sec. 4.2.1 for all disentanglers at once, with identical
// partial products shared), then contracting with the centre tensor. The
// 4x4 iterations of all disentanglers run in one kernel, one thread each,
// with a one-sided Jacobi SVD.
#include <algorithm>
#include <array>
#include <cmath>
#include <map>
#include <set>

#include "lanczos.h"
#include "state.h"

using namespace attn;

namespace attn {

// mode product and contraction helpers from state.cu / gemm_f64.cu
void gather_rows_f64(attn_ctx* ctx, double* dst, const double* src, const int* idx_dev, int R, long len);

namespace {

constexpr int kMaxEnt = 48;  // entries per disentangler handled by the kernel

__device__ void mm4(const double* a, const double* b, double* c) {  // c = a b
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 4; ++j) {
      double s = 0;
      for (int q = 0; q < 4; ++q) s += a[i * 4 + q] * b[q * 4 + j];
      c[i * 4 + j] = s;
    }
}
__device__ void mtm4(const double* a, const double* b, double* c) {  // c = a^T b
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 4; ++j) {
      double s = 0;
      for (int q = 0; q < 4; ++q) s += a[q * 4 + i] * b[q * 4 + j];
      c[i * 4 + j] = s;
    }
}

struct DEArgs {
  int n_de;
  const int* ent_begin;   // [n_de + 1]
  const int* ent_midx;    // [n_ent][16] indices into vals (M[a][b])
  const double* ent_C;    // [n_ent][16]
  const double* lambda;   // [n_de]
  const int* rho_idx;     // [n_de][16]
  const double* vals;     // probe expectation values
  const double* u_in;     // [n_de][16]
  double* u_out;          // [n_de][16]
  double* e_out;          // [n_de][2]: E_k(u_in), E_k(u_out)
  int max_iter;
  double rel_dev;
};

__device__ double de_energy(const DEArgs& a, int b0, int b1, const double* u) {
  double e = 0.0;
  double uc[16], w[16];
  for (int q = b0; q < b1; ++q) {
    const double* C = a.ent_C + 16L * q;
    mm4(C, u, w);      // C u
    mtm4(u, w, uc);    // u^T C u
    for (int al = 0; al < 4; ++al)
      for (int be = 0; be < 4; ++be) e += a.vals[a.ent_midx[16L * q + al * 4 + be]] * uc[be * 4 + al];
  }
  return e;
}

__device__ void de_gamma(const DEArgs& a, int k, int b0, int b1, const double* u, double* g) {
  double M[16], utc[16], t[16];
  for (int i = 0; i < 16; ++i) g[i] = 0.0;
  for (int q = b0; q < b1; ++q) {
    const double* C = a.ent_C + 16L * q;
    for (int i = 0; i < 16; ++i) M[i] = a.vals[a.ent_midx[16L * q + i]];
    mtm4(u, C, utc);  // u^T C
    mm4(M, utc, t);
    for (int i = 0; i < 16; ++i) g[i] += t[i];
  }
  double rho[16], ut[16];
  for (int i = 0; i < 16; ++i) rho[i] = a.vals[a.rho_idx[16L * k + i]];
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 4; ++j) ut[i * 4 + j] = u[j * 4 + i];
  mm4(rho, ut, t);
  for (int i = 0; i < 16; ++i) g[i] -= a.lambda[k] * t[i];
}

// u = -V W^T for G = W diag(s) V^T (one-sided Jacobi on the columns of G).
__device__ void mera_solve(const double* G, double* u) {
  double B[16], J[16];
  for (int i = 0; i < 16; ++i) { B[i] = G[i]; J[i] = (i % 5 == 0) ? 1.0 : 0.0; }
  for (int sweep = 0; sweep < 40; ++sweep) {
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
        double ratio = fabs(c) / sqrt(a * b);
        if (!(ratio > 1e-16)) continue;
        off = fmax(off, ratio);
        double zeta = (b - a) / (2.0 * c);
        double t = (zeta >= 0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
        double cs = 1.0 / sqrt(1.0 + t * t), sn = cs * t;
        for (int r = 0; r < 4; ++r) {
          double x = B[r * 4 + p], y = B[r * 4 + q];
          B[r * 4 + p] = cs * x - sn * y;
          B[r * 4 + q] = sn * x + cs * y;
          x = J[r * 4 + p];
          y = J[r * 4 + q];
          J[r * 4 + p] = cs * x - sn * y;
          J[r * 4 + q] = sn * x + cs * y;
        }
      }
    if (off < 1e-15) break;
  }
  double W[16], s[4], smax = 0.0;
  for (int k = 0; k < 4; ++k) {
    double n = 0;
    for (int r = 0; r < 4; ++r) n += B[r * 4 + k] * B[r * 4 + k];
    s[k] = sqrt(n);
    smax = fmax(smax, s[k]);
  }
  bool done[4];
  for (int k = 0; k < 4; ++k) {
    done[k] = s[k] > 1e-13 * smax && s[k] > 0.0;
    for (int r = 0; r < 4; ++r) W[r * 4 + k] = done[k] ? B[r * 4 + k] / s[k] : 0.0;
  }
  // complete rank-deficient columns with unit vectors orthogonalised against the others
  for (int k = 0; k < 4; ++k) {
    if (done[k]) continue;
    for (int tr = 0; tr < 4; ++tr) {
      double v[4] = {0, 0, 0, 0};
      v[tr] = 1.0;
      for (int pass = 0; pass < 2; ++pass)
        for (int o = 0; o < 4; ++o) {
          if (!done[o]) continue;
          double d = 0;
          for (int r = 0; r < 4; ++r) d += W[r * 4 + o] * v[r];
          for (int r = 0; r < 4; ++r) v[r] -= d * W[r * 4 + o];
        }
      double n = sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2] + v[3] * v[3]);
      if (n > 0.5) {
        for (int r = 0; r < 4; ++r) W[r * 4 + k] = v[r] / n;
        done[k] = true;
        break;
      }
    }
  }
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 4; ++j) {
      double acc = 0;
      for (int q = 0; q < 4; ++q) acc += J[i * 4 + q] * W[j * 4 + q];
      u[i * 4 + j] = -acc;
    }
}

__global__ void de_mera_kernel(DEArgs a) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= a.n_de) return;
  const int b0 = a.ent_begin[k], b1 = a.ent_begin[k + 1];
  double u[16], g[16], un[16];
  for (int i = 0; i < 16; ++i) u[i] = a.u_in[16L * k + i];
  double e = de_energy(a, b0, b1, u);
  a.e_out[2 * k] = e;
  for (int it = 0; it < a.max_iter; ++it) {
    de_gamma(a, k, b0, b1, u, g);
    mera_solve(g, un);
    const double en = de_energy(a, b0, b1, un);
    if (!(en <= e + 1e-14 * fmax(1.0, fabs(e)))) break;
    const bool done = fabs(en - e) <= a.rel_dev * fmax(fabs(e), 1e-300);
    for (int i = 0; i < 16; ++i) u[i] = un[i];
    e = en;
    if (done) break;
  }
  for (int i = 0; i < 16; ++i) a.u_out[16L * k + i] = u[i];
  a.e_out[2 * k + 1] = e;
}

// ---- Riemannian conjugate gradients on O(4) (Sec. 4.1.2): the true E_k(u) with u
// and u^T varying together. With E = sum_q Tr(M_q u^T C_q u), the Euclidean gradient
// is sum_q (C_q u M_q + C_q^T u M_q^T); it is projected onto the tangent space
// u skew(u^T G); Polak-Ribiere+ directions are carried to the new point by the same
// projection; the retraction is the Q factor (positive diagonal of R) of u + xi; the
// step is found by Armijo backtracking (c1 = 1e-4, halving) from a Frobenius step
// of 0.25, doubled after an accepted step up to 1. Stops like the MERA-like update.
__device__ void de_egrad(const DEArgs& a, int b0, int b1, const double* u, double* g) {
  double M[16], t1[16], t2[16];
  for (int i = 0; i < 16; ++i) g[i] = 0.0;
  for (int q = b0; q < b1; ++q) {
    const double* C = a.ent_C + 16L * q;
    for (int i = 0; i < 16; ++i) M[i] = a.vals[a.ent_midx[16L * q + i]];
    mm4(C, u, t1);   // C u
    mm4(t1, M, t2);  // C u M
    for (int i = 0; i < 16; ++i) g[i] += t2[i];
    mtm4(C, u, t1);  // C^T u
    for (int r = 0; r < 4; ++r)  // (C^T u) M^T
      for (int c = 0; c < 4; ++c) {
        double acc = 0.0;
        for (int k = 0; k < 4; ++k) acc += t1[r * 4 + k] * M[c * 4 + k];
        g[r * 4 + c] += acc;
      }
  }
}

// u skew(u^T z)
__device__ void de_tangent(const double* u, const double* z, double* out) {
  double a[16], sk[16];
  mtm4(u, z, a);
  for (int r = 0; r < 4; ++r)
    for (int c = 0; c < 4; ++c) sk[r * 4 + c] = 0.5 * (a[r * 4 + c] - a[c * 4 + r]);
  mm4(u, sk, out);
}

// Q of u + xi by Gram-Schmidt on the columns, applied twice (R's diagonal > 0)
__device__ void de_retract(const double* u, const double* xi, double* q) {
  for (int i = 0; i < 16; ++i) q[i] = u[i] + xi[i];
  for (int c = 0; c < 4; ++c) {
    for (int pass = 0; pass < 2; ++pass)
      for (int o = 0; o < c; ++o) {
        double d = 0.0;
        for (int r = 0; r < 4; ++r) d += q[r * 4 + o] * q[r * 4 + c];
        for (int r = 0; r < 4; ++r) q[r * 4 + c] -= d * q[r * 4 + o];
      }
    double n = 0.0;
    for (int r = 0; r < 4; ++r) n += q[r * 4 + c] * q[r * 4 + c];
    n = sqrt(n);
    for (int r = 0; r < 4; ++r) q[r * 4 + c] /= n;
  }
}

__device__ double dot16(const double* x, const double* y) {
  double s = 0.0;
  for (int i = 0; i < 16; ++i) s += x[i] * y[i];
  return s;
}

__global__ void de_rgd_kernel(DEArgs a) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= a.n_de) return;
  const int b0 = a.ent_begin[k], b1 = a.ent_begin[k + 1];
  double u[16], g[16], d[16], un[16], gn[16], go[16], dn[16], z[16], xi[16];
  for (int i = 0; i < 16; ++i) u[i] = a.u_in[16L * k + i];
  double e = de_energy(a, b0, b1, u);
  a.e_out[2 * k] = e;
  de_egrad(a, b0, b1, u, z);
  de_tangent(u, z, g);
  for (int i = 0; i < 16; ++i) d[i] = -g[i];
  double step = 0.25;
  for (int it = 0; it < a.max_iter; ++it) {
    double gd = dot16(g, d);
    if (!(gd < 0.0)) {
      for (int i = 0; i < 16; ++i) d[i] = -g[i];
      gd = -dot16(g, g);
    }
    const double dnorm = sqrt(dot16(d, d));
    if (dnorm == 0.0) break;
    double t = step / dnorm, en = 0.0;
    bool accepted = false;
    for (int ls = 0; ls < 40; ++ls) {
      for (int i = 0; i < 16; ++i) xi[i] = t * d[i];
      de_retract(u, xi, un);
      en = de_energy(a, b0, b1, un);
      if (en <= e + 1e-4 * t * gd) {
        accepted = true;
        break;
      }
      t *= 0.5;
    }
    if (!accepted) break;
    step = fmin(1.0, 2.0 * t * dnorm);
    de_egrad(a, b0, b1, un, z);
    de_tangent(un, z, gn);
    de_tangent(un, g, go);
    de_tangent(un, d, dn);
    double gg = dot16(g, g);
    double beta = fmax(0.0, (dot16(gn, gn) - dot16(gn, go)) / fmax(gg, 1e-300));
    const bool done = fabs(en - e) <= a.rel_dev * fmax(fabs(e), 1e-300);
    for (int i = 0; i < 16; ++i) {
      u[i] = un[i];
      g[i] = gn[i];
      d[i] = -gn[i] + beta * dn[i];
    }
    e = en;
    if (done) break;
  }
  for (int i = 0; i < 16; ++i) a.u_out[16L * k + i] = u[i];
  a.e_out[2 * k + 1] = e;
}

// E_k of candidate disentanglers (one thread per disentangler)
__global__ void de_energy_kernel(DEArgs a, const double* u_cand, double* e_out) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= a.n_de) return;
  e_out[k] = de_energy(a, a.ent_begin[k], a.ent_begin[k + 1], u_cand + 16L * k);
}

__global__ void scale_vals(double* v, int n, const double* nrm_sq) {
  const double inv = 1.0 / *nrm_sq;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) v[i] *= inv;
}

void upload(attn_ctx* ctx, DevBuf& b, const void* src, size_t bytes) {
  b.reserve(std::max<size_t>(bytes, 16));
  if (bytes) ATTN_CHECK_CUDA(cudaMemcpyAsync(b.p, src, bytes, cudaMemcpyHostToDevice, ctx->stream));
}

// Embed an operator on `sites` (ascending) into the ordered site list `target` (any order).
std::vector<double> embed_any(const std::vector<double>& op, const std::vector<int>& sites,
                              const std::vector<int>& target) {
  const int k = (int)sites.size(), kt = (int)target.size(), D = 1 << kt;
  std::vector<int> pos(k);
  for (int a = 0; a < k; ++a) pos[a] = (int)(std::find(target.begin(), target.end(), sites[a]) - target.begin());
  std::vector<double> out((size_t)D * D, 0.0);
  for (int r = 0; r < D; ++r)
    for (int c = 0; c < D; ++c) {
      bool same = true;
      int ri = 0, ci = 0;
      for (int b = 0; b < kt; ++b) {
        const int rb = (r >> (kt - 1 - b)) & 1, cb = (c >> (kt - 1 - b)) & 1;
        int a = -1;
        for (int q = 0; q < k; ++q)
          if (pos[q] == b) a = q;
        if (a < 0) {
          if (rb != cb) same = false;
        } else {
          ri |= rb << (k - 1 - a);
          ci |= cb << (k - 1 - a);
        }
      }
      if (same) out[(size_t)r * D + c] = op[(size_t)ri * (1 << k) + ci];
    }
  return out;
}

// Singular triplets of a small dense matrix (rows x cols, row-major) by one-sided Jacobi.
void small_svd(const std::vector<double>& A, int rows, int cols, std::vector<double>& U, std::vector<double>& s,
               std::vector<double>& V) {
  // B = A (rows x cols); rotate columns
  std::vector<double> B = A;
  V.assign((size_t)cols * cols, 0.0);
  for (int i = 0; i < cols; ++i) V[i * cols + i] = 1.0;
  for (int sweep = 0; sweep < 60; ++sweep) {
    double off = 0.0;
    for (int p = 0; p < cols; ++p)
      for (int q = p + 1; q < cols; ++q) {
        double a = 0, b = 0, c = 0;
        for (int r = 0; r < rows; ++r) {
          a += B[r * cols + p] * B[r * cols + p];
          b += B[r * cols + q] * B[r * cols + q];
          c += B[r * cols + p] * B[r * cols + q];
        }
        if (c == 0.0 || a == 0.0 || b == 0.0) continue;
        double ratio = std::fabs(c) / std::sqrt(a * b);
        if (!(ratio > 1e-16)) continue;
        off = std::max(off, ratio);
        double zeta = (b - a) / (2.0 * c);
        double t = (zeta >= 0 ? 1.0 : -1.0) / (std::fabs(zeta) + std::sqrt(1.0 + zeta * zeta));
        double cs = 1.0 / std::sqrt(1.0 + t * t), sn = cs * t;
        for (int r = 0; r < rows; ++r) {
          double x = B[r * cols + p], y = B[r * cols + q];
          B[r * cols + p] = cs * x - sn * y;
          B[r * cols + q] = sn * x + cs * y;
        }
        for (int r = 0; r < cols; ++r) {
          double x = V[r * cols + p], y = V[r * cols + q];
          V[r * cols + p] = cs * x - sn * y;
          V[r * cols + q] = sn * x + cs * y;
        }
      }
    if (off < 1e-15) break;
  }
  s.assign(cols, 0.0);
  U.assign((size_t)rows * cols, 0.0);
  for (int k = 0; k < cols; ++k) {
    double n = 0;
    for (int r = 0; r < rows; ++r) n += B[r * cols + k] * B[r * cols + k];
    s[k] = std::sqrt(n);
    for (int r = 0; r < rows; ++r) U[r * cols + k] = s[k] > 0 ? B[r * cols + k] / s[k] : 0.0;
  }
}

}  // namespace
}  // namespace attn

// ----------------------------------------------------- probe expectations
void attn_state::probe_expectations(const std::vector<ProbeFactor>& F, const std::vector<Probe>& P, DevBuf& vals) {
  using Key = std::vector<int>;
  const int c0 = centre;
  const int NP = (int)P.size();
  auto slot_of = [&](int n, int site) {
    for (int s = 0; s < 3; ++s)
      if (tree.behind(n, s, site)) return s;
    throw Error{ATTN_EINVAL, "site not behind any link"};
  };
  std::vector<std::array<Key, 3>> pk(NP);
  std::map<int, std::set<Key>> need;
  for (int q = 0; q < NP; ++q) {
    for (int a = 0; a < P[q].n; ++a) pk[q][slot_of(c0, F[P[q].f[a]].site)].push_back(P[q].f[a]);
    for (int s = 0; s < 3; ++s) {
      std::sort(pk[q][s].begin(), pk[q][s].end());
      if (!pk[q][s].empty()) need[3 * c0 + s].insert(pk[q][s]);
    }
  }
  std::vector<int> order;
  std::vector<int> queue;
  for (int s = 0; s < 3; ++s)
    if (need.count(3 * c0 + s)) queue.push_back(3 * c0 + s);
  std::set<int> seen(queue.begin(), queue.end());
  for (size_t qi = 0; qi < queue.size(); ++qi) {
    const int L = queue[qi];
    order.push_back(L);
    const Tree::Nbr& nb = tree.nbr[L];
    if (nb.kind == 0) continue;
    const int c = nb.idx, t = nb.back;
    int xs[2], ni = 0;
    for (int s = 0; s < 3; ++s)
      if (s != t) xs[ni++] = s;
    for (const Key& K : need[L]) {
      // kx holds the factors behind c's slot xs[0], ky those behind xs[1]
      Key kx, ky;
      for (int f : K) {
        const int s = slot_of(c, F[f].site);
        ATTN_REQUIRE(s != t, ATTN_EINVAL, "probe bookkeeping error");
        (s == xs[0] ? kx : ky).push_back(f);
      }
      if (!kx.empty()) need[3 * c + xs[0]].insert(kx);
      if (!ky.empty()) need[3 * c + xs[1]].insert(ky);
    }
    for (int s = 0; s < 3; ++s) {
      if (s == t) continue;
      const int L2 = 3 * c + s;
      if (need.count(L2) && !seen.count(L2)) {
        seen.insert(L2);
        queue.push_back(L2);
      }
    }
  }
  struct PL {
    std::vector<Key> keys;
    std::map<Key, int> idx;
    DevBuf ops;
  };
  std::map<int, PL> pl;
  for (auto it = order.rbegin(); it != order.rend(); ++it) {
    const int L = *it;
    const int n = L / 3, slot = L % 3;
    PL& o = pl[L];
    const Tree::Nbr& nb = tree.nbr[L];
    const int dimL = dim(n, slot);
    const long osz = (long)dimL * dimL;
    if (nb.kind == 0) {
      std::vector<double> h;
      for (const Key& K : need[L]) {
        ATTN_REQUIRE(K.size() == 1 && F[K[0]].site == nb.idx, ATTN_EINVAL, "probe bookkeeping error (site)");
        o.idx[K] = (int)o.keys.size();
        o.keys.push_back(K);
        h.insert(h.end(), F[K[0]].op, F[K[0]].op + 4);
      }
      upload(ctx, o.ops, h.data(), sizeof(double) * h.size());
      continue;
    }
    const int c = nb.idx, t = nb.back;
    int xs[2], ni = 0;
    for (int s = 0; s < 3; ++s)
      if (s != t) xs[ni++] = s;
    const PL& Px = pl[3 * c + xs[0]];
    const PL& Py = pl[3 * c + xs[1]];
    std::vector<Key> gb, gx, gy;
    std::vector<int> bx, by, xi, yi;
    for (const Key& K : need[L]) {
      Key kx, ky;
      for (int f : K) (slot_of(c, F[f].site) == xs[0] ? kx : ky).push_back(f);
      if (!kx.empty() && !ky.empty()) {
        gb.push_back(K);
        bx.push_back(Px.idx.at(kx));
        by.push_back(Py.idx.at(ky));
      } else if (!kx.empty()) {
        gx.push_back(K);
        xi.push_back(Px.idx.at(kx));
      } else {
        gy.push_back(K);
        yi.push_back(Py.idx.at(ky));
      }
    }
    for (auto* g : {&gb, &gx, &gy})
      for (const Key& K : *g) {
        o.idx[K] = (int)o.keys.size();
        o.keys.push_back(K);
      }
    o.ops.reserve(sizeof(double) * std::max<size_t>(1, o.keys.size()) * osz);
    const int d[3] = {dim(c, 0), dim(c, 1), dim(c, 2)};
    const double* Tc = tensor(c);
    const double* Ax = Px.ops.as<double>();
    const double* By = Py.ops.as<double>();
    double* out = o.ops.as<double>();
    if (!gb.empty()) renorm_batch(Tc, d, t, xs[0], xs[1], Ax, bx, By, by, out);
    if (!gx.empty()) renorm_batch(Tc, d, t, xs[0], xs[1], Ax, xi, nullptr, {}, out + (long)gb.size() * osz);
    if (!gy.empty())
      renorm_batch(Tc, d, t, xs[0], xs[1], nullptr, {}, By, yi, out + (long)(gb.size() + gx.size()) * osz);
  }
  // contract at the centre: <T| (x)_s O_s |T> / <T|T>, grouped by slot pattern
  const int d[3] = {dim(c0, 0), dim(c0, 1), dim(c0, 2)};
  const long V = vol(c0);
  vals.reserve(sizeof(double) * std::max(NP, 1) + 64);
  double* dv = vals.as<double>();
  std::vector<std::vector<int>> by_pat(8);
  for (int q = 0; q < NP; ++q) {
    int mask = 0;
    for (int s = 0; s < 3; ++s)
      if (!pk[q][s].empty()) mask |= 1 << s;
    by_pat[mask].push_back(q);
  }
  std::vector<int> pos(NP, -1);
  int filled = 0;
  const long budget = 1L << 26;
  const int chunk = (int)std::max<long>(1, std::min<long>(512, budget / std::max<long>(V, 1)));
  std::vector<int> out_order;
  for (int mask = 1; mask < 8; ++mask) {
    const std::vector<int>& qs = by_pat[mask];
    for (size_t r0 = 0; r0 < qs.size(); r0 += chunk) {
      const int Rc = (int)std::min<size_t>(chunk, qs.size() - r0);
      rw1.reserve(sizeof(double) * (size_t)Rc * V);
      rw2.reserve(sizeof(double) * (size_t)Rc * V);
      double* W[2] = {rw1.as<double>(), rw2.as<double>()};
      const double* cur = tensor(c0);
      long cur_stride = 0;
      int wi = 0;
      for (int s = 2; s >= 0; --s) {
        if (!(mask & (1 << s))) continue;
        const PL& Ps = pl[3 * c0 + s];
        std::vector<int> ix(Rc);
        for (int r = 0; r < Rc; ++r) ix[r] = Ps.idx.at(pk[qs[r0 + r]][s]);
        upload(ctx, idxbuf, ix.data(), sizeof(int) * ix.size());
        opsA.reserve(sizeof(double) * (size_t)Rc * d[s] * d[s]);
        gather_rows_f64(ctx, opsA.as<double>(), Ps.ops.as<double>(), idxbuf.as<int>(), Rc, (long)d[s] * d[s]);
        mode_product_f64(ctx, d, s, opsA.as<double>(), Rc, cur, cur_stride, W[wi], 0.0);
        cur = W[wi];
        cur_stride = V;
        wi ^= 1;
      }
      multi_dot(ctx, cur, Rc, V, tensor(c0), dv + filled, nullptr);
      for (int r = 0; r < Rc; ++r) pos[qs[r0 + r]] = filled + r;
      filled += Rc;
    }
  }
  // normalise by <T|T> and put the values in probe order
  ctx->scal.reserve(sizeof(double) * 64);
  multi_dot(ctx, tensor(c0), 1, V, tensor(c0), ctx->scal.as<double>(), nullptr);
  scale_vals<<<std::max(1, std::min(1024, (NP + 255) / 256)), 256, 0, ctx->stream>>>(dv, NP, ctx->scal.as<double>());
  ctx->launches++;
  idxbuf.reserve(sizeof(int) * std::max(NP, 1));
  upload(ctx, idxbuf, pos.data(), sizeof(int) * pos.size());
  rw2.reserve(sizeof(double) * std::max(NP, 1));
  gather_rows_f64(ctx, rw2.as<double>(), dv, idxbuf.as<int>(), NP, 1);
  copy_f64(ctx, dv, rw2.as<double>(), NP);
  ATTN_CHECK_CUDA(cudaGetLastError());
}

// ------------------------------------------------------ disentangler update
// Probes and 4x4 coefficient blocks of the selected disentanglers (Sec. 4.1.1):
// position q of `sel` owns entries ent_begin[q] .. ent_begin[q+1] and the matrix
// units rho_idx[16 q ..] of its two-site density matrix.
void attn_state::de_setup(const std::vector<int>& sel, DESetup& S) {
  const int nDE = (int)des.size();
  const int nS = (int)sel.size();
  S.sel = sel;
  S.F.clear();
  S.P.clear();
  std::vector<int> owner(model.n_sites, -1);
  for (int q = 0; q < nS; ++q) {
    ATTN_REQUIRE(sel[q] >= 0 && sel[q] < nDE, ATTN_EINVAL, "disentangler index out of range");
    owner[des[sel[q]].first] = owner[des[sel[q]].second] = q;
  }
  std::vector<ProbeFactor>& F = S.F;
  std::vector<Probe>& P = S.P;
  // matrix units on every selected disentangler site: fid[q][side][x], x = a*2+b for |a><b|
  std::vector<std::array<std::array<int, 4>, 2>> fid(nS);
  for (int q = 0; q < nS; ++q)
    for (int side = 0; side < 2; ++side)
      for (int x = 0; x < 4; ++x) {
        ProbeFactor f;
        f.site = side ? des[sel[q]].second : des[sel[q]].first;
        for (int i = 0; i < 4; ++i) f.op[i] = (i == x) ? 1.0 : 0.0;
        fid[q][side][x] = (int)F.size();
        F.push_back(f);
      }
  // M[alpha][beta] = < |beta><alpha| (x) extra >: the probe for (alpha, beta) has
  // |b_i><a_i| on i and |b_j><a_j| on j (x = b*2 + a), and `extra` (factor id or -1).
  auto add_block = [&](int q, int extra, std::vector<int>& midx) {
    midx.resize(16);
    for (int al = 0; al < 4; ++al)
      for (int be = 0; be < 4; ++be) {
        const int ai = al >> 1, aj = al & 1, bi = be >> 1, bj = be & 1;
        Probe p;
        p.n = extra >= 0 ? 3 : 2;
        p.f[0] = fid[q][0][bi * 2 + ai];
        p.f[1] = fid[q][1][bj * 2 + aj];
        p.f[2] = extra;
        for (int e = 3; e < 8; ++e) p.f[e] = -1;
        midx[al * 4 + be] = (int)P.size();
        P.push_back(p);
      }
  };
  S.rho_idx.assign(16L * nS, 0);
  S.ent_begin.assign(nS + 1, 0);
  S.ent_midx.clear();
  S.ent_C.clear();
  S.lambda.assign(nS, 0.0);
  std::vector<std::vector<std::pair<std::vector<int>, std::vector<double>>>> ents(nS);
  for (int q = 0; q < nS; ++q) {
    std::vector<int> m;
    add_block(q, -1, m);
    std::copy(m.begin(), m.end(), S.rho_idx.begin() + 16L * q);
  }
  for (const Term& tm : model.terms) {
    int q = -1;
    for (int a = 0; a < tm.n; ++a)
      if (owner[tm.site[a]] >= 0) q = owner[tm.site[a]];
    if (q < 0) continue;
    const int i = des[sel[q]].first, j = des[sel[q]].second;
    std::vector<int> sites(tm.site, tm.site + tm.n), extra;
    for (int s : sites)
      if (s != i && s != j) extra.push_back(s);
    ATTN_REQUIRE(extra.size() <= 1, ATTN_EUNSUPPORTED, "disentangler update supports terms with <= 1 extra site");
    {  // spectral norm of the term
      std::vector<double> U, sv, V;
      const int D = 1 << tm.n;
      small_svd(tm.op, D, D, U, sv, V);
      S.lambda[q] += *std::max_element(sv.begin(), sv.end());
    }
    if (extra.empty()) {
      ents[q].push_back({std::vector<int>(S.rho_idx.begin() + 16L * q, S.rho_idx.begin() + 16L * q + 16),
                         embed_any(tm.op, sites, {i, j})});
      continue;
    }
    const int e = extra[0];
    std::vector<double> h3 = embed_any(tm.op, sites, {i, j, e});  // order (i, j, e)
    // R[(al,be)][(ep,ep')] = h3[(al ep)][(be ep')]
    std::vector<double> R(16 * 4);
    for (int al = 0; al < 4; ++al)
      for (int be = 0; be < 4; ++be)
        for (int ep = 0; ep < 2; ++ep)
          for (int eq = 0; eq < 2; ++eq) R[(al * 4 + be) * 4 + ep * 2 + eq] = h3[(al * 2 + ep) * 8 + be * 2 + eq];
    std::vector<double> U, sv, Vv;
    small_svd(R, 16, 4, U, sv, Vv);
    const double smax = *std::max_element(sv.begin(), sv.end());
    for (int r = 0; r < 4; ++r) {
      if (!(sv[r] > 1e-14 * smax)) continue;
      ProbeFactor f;
      f.site = e;
      for (int c = 0; c < 4; ++c) f.op[c] = Vv[c * 4 + r];
      const int fidx = (int)F.size();
      F.push_back(f);
      std::vector<int> m;
      add_block(q, fidx, m);
      std::vector<double> C(16);
      for (int c = 0; c < 16; ++c) C[c] = U[c * 4 + r] * sv[r];
      ents[q].push_back({m, C});
    }
  }
  for (int q = 0; q < nS; ++q) {
    ATTN_REQUIRE((int)ents[q].size() <= kMaxEnt, ATTN_EUNSUPPORTED, "too many terms on one disentangler");
    S.ent_begin[q + 1] = S.ent_begin[q] + (int)ents[q].size();
    for (auto& pr : ents[q]) {
      S.ent_midx.insert(S.ent_midx.end(), pr.first.begin(), pr.first.end());
      S.ent_C.insert(S.ent_C.end(), pr.second.begin(), pr.second.end());
    }
  }
}

namespace attn {
namespace {
// Device copies of a DESetup's tables, and the kernel arguments pointing at them.
struct DEDev {
  DevBuf eb, em, ec, lam, rho, vals;
};
DEArgs de_upload(attn_ctx* ctx, const DESetup& S, DEDev& d) {
  upload(ctx, d.eb, S.ent_begin.data(), sizeof(int) * S.ent_begin.size());
  upload(ctx, d.em, S.ent_midx.data(), sizeof(int) * S.ent_midx.size());
  upload(ctx, d.ec, S.ent_C.data(), sizeof(double) * S.ent_C.size());
  upload(ctx, d.lam, S.lambda.data(), sizeof(double) * S.lambda.size());
  upload(ctx, d.rho, S.rho_idx.data(), sizeof(int) * S.rho_idx.size());
  DEArgs a;
  a.n_de = (int)S.sel.size();
  a.ent_begin = d.eb.as<int>();
  a.ent_midx = d.em.as<int>();
  a.ent_C = d.ec.as<double>();
  a.lambda = d.lam.as<double>();
  a.rho_idx = d.rho.as<int>();
  a.vals = d.vals.as<double>();
  a.u_in = a.u_out = nullptr;
  a.e_out = nullptr;
  a.max_iter = ctx->cfg.de_max_iter;
  a.rel_dev = ctx->cfg.de_rel_dev;
  return a;
}

// Gamma_k (shifted terms, Eq. contracted) and E_k at given disentanglers, one thread each.
__global__ void de_gamma_kernel(DEArgs a, const double* u, double* g_out, double* e_out) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= a.n_de) return;
  const int b0 = a.ent_begin[k], b1 = a.ent_begin[k + 1];
  de_gamma(a, k, b0, b1, u + 16L * k, g_out + 16L * k);
  e_out[k] = de_energy(a, b0, b1, u + 16L * k);
}
}  // namespace
}  // namespace attn

std::vector<double> attn_state::de_rdms(const std::vector<int>& sel) {
  DESetup S;
  de_setup(sel, S);
  DevBuf vals;
  probe_expectations(S.F, S.P, vals);
  std::vector<double> pv(S.P.size());
  ATTN_CHECK_CUDA(cudaMemcpyAsync(pv.data(), vals.p, sizeof(double) * pv.size(), cudaMemcpyDeviceToHost, ctx->stream));
  ATTN_CHECK_CUDA(cudaStreamSynchronize(ctx->stream));
  std::vector<double> rho(16L * sel.size());
  for (size_t q = 0; q < rho.size(); ++q) rho[q] = pv[S.rho_idx[q]];
  return rho;
}

void attn_state::de_environment(int k, const double* u16, double* gamma16, double* e_k) {
  DESetup S;
  de_setup({k}, S);
  DEDev d;
  probe_expectations(S.F, S.P, d.vals);
  DEArgs a = de_upload(ctx, S, d);
  DevBuf du, dg, de;
  upload(ctx, du, u16, sizeof(double) * 16);
  dg.reserve(sizeof(double) * 16);
  de.reserve(sizeof(double));
  de_gamma_kernel<<<1, 32, 0, ctx->stream>>>(a, du.as<double>(), dg.as<double>(), de.as<double>());
  ctx->launches++;
  ATTN_CHECK_CUDA(cudaGetLastError());
  ATTN_CHECK_CUDA(cudaMemcpyAsync(gamma16, dg.p, sizeof(double) * 16, cudaMemcpyDeviceToHost, ctx->stream));
  ATTN_CHECK_CUDA(cudaMemcpyAsync(e_k, de.p, sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
  ATTN_CHECK_CUDA(cudaStreamSynchronize(ctx->stream));
}

double attn_state::de_update(const std::vector<int>* only) {
  const int nDE = (int)des.size();
  if (!nDE) return 0.0;
  std::vector<int> sel;
  if (only) sel = *only;
  else for (int k = 0; k < nDE; ++k) sel.push_back(k);
  const int nS = (int)sel.size();
  if (!nS) return 0.0;
  const bool all = (nS == nDE);
  DESetup S;
  de_setup(sel, S);
  DEDev d;
  probe_expectations(S.F, S.P, d.vals);
  DEArgs a = de_upload(ctx, S, d);
  DevBuf d_uin, d_uout, d_e;
  std::vector<double> uin(16L * nS);
  for (int q = 0; q < nS; ++q) std::copy(us[sel[q]].begin(), us[sel[q]].end(), uin.begin() + 16L * q);
  upload(ctx, d_uin, uin.data(), sizeof(double) * uin.size());
  d_uout.reserve(sizeof(double) * uin.size());
  d_e.reserve(sizeof(double) * 2 * nS);
  // reduced density matrices on the disentangler sites (recorded at the first full update)
  const bool first = all && !first_de_done;
  std::vector<double> rho_h;
  if (first) {
    std::vector<double> pv(S.P.size());
    ATTN_CHECK_CUDA(cudaMemcpyAsync(pv.data(), d.vals.p, sizeof(double) * pv.size(), cudaMemcpyDeviceToHost,
                                    ctx->stream));
    ATTN_CHECK_CUDA(cudaStreamSynchronize(ctx->stream));
    rho_h.assign(16L * nS, 0.0);
    for (long q = 0; q < 16L * nS; ++q) rho_h[q] = pv[S.rho_idx[q]];
    rho_first = rho_h;
    first_de_done = true;
  }
  a.u_in = d_uin.as<double>();
  a.u_out = d_uout.as<double>();
  a.e_out = d_e.as<double>();
  if (first && learned) {
    // learned start: keep the prediction where it is finite and does not raise E_k
    std::vector<double> up(16L * nS);
    learned->net.predict(nS, rho_h.data(), up.data());
    DevBuf d_up, d_ep, d_e0;
    upload(ctx, d_up, up.data(), sizeof(double) * up.size());
    d_ep.reserve(sizeof(double) * nS);
    d_e0.reserve(sizeof(double) * nS);
    de_energy_kernel<<<(nS + 63) / 64, 64, 0, ctx->stream>>>(a, d_up.as<double>(), d_ep.as<double>());
    de_energy_kernel<<<(nS + 63) / 64, 64, 0, ctx->stream>>>(a, d_uin.as<double>(), d_e0.as<double>());
    ctx->launches += 2;
    std::vector<double> ep(nS), e0(nS);
    ATTN_CHECK_CUDA(cudaMemcpyAsync(ep.data(), d_ep.p, sizeof(double) * nS, cudaMemcpyDeviceToHost, ctx->stream));
    ATTN_CHECK_CUDA(cudaMemcpyAsync(e0.data(), d_e0.p, sizeof(double) * nS, cudaMemcpyDeviceToHost, ctx->stream));
    ATTN_CHECK_CUDA(cudaStreamSynchronize(ctx->stream));
    learned_used = learned_fallback = 0;
    for (int q = 0; q < nS; ++q) {
      bool ok = std::isfinite(ep[q]);
      for (int i = 0; i < 16; ++i) ok = ok && std::isfinite(up[16L * q + i]);
      if (ok && ep[q] <= e0[q]) {
        std::copy(up.begin() + 16L * q, up.begin() + 16L * q + 16, uin.begin() + 16L * q);
        ++learned_used;
      } else {
        ++learned_fallback;
      }
    }
    upload(ctx, d_uin, uin.data(), sizeof(double) * uin.size());
    a.u_in = d_uin.as<double>();
  }
  if (ctx->cfg.de_method == 1) de_rgd_kernel<<<(nS + 63) / 64, 64, 0, ctx->stream>>>(a);
  else de_mera_kernel<<<(nS + 63) / 64, 64, 0, ctx->stream>>>(a);
  ctx->launches++;
  ATTN_CHECK_CUDA(cudaGetLastError());
  std::vector<double> uout(uin.size()), eo(2L * nS);
  ATTN_CHECK_CUDA(cudaMemcpyAsync(uout.data(), d_uout.p, sizeof(double) * uout.size(), cudaMemcpyDeviceToHost, ctx->stream));
  ATTN_CHECK_CUDA(cudaMemcpyAsync(eo.data(), d_e.p, sizeof(double) * eo.size(), cudaMemcpyDeviceToHost, ctx->stream));
  ATTN_CHECK_CUDA(cudaStreamSynchronize(ctx->stream));
  if ((int)last_de_energy.size() != 2 * nDE) last_de_energy.assign(2L * nDE, std::nan(""));
  double dE = 0.0;
  for (int q = 0; q < nS; ++q) {
    ATTN_REQUIRE(std::isfinite(eo[2 * q + 1]), ATTN_ENONFINITE, "non-finite disentangler energy");
    us[sel[q]].assign(uout.begin() + 16L * q, uout.begin() + 16L * q + 16);
    dE += eo[2 * q + 1] - eo[2 * q];
    last_de_energy[2 * sel[q]] = eo[2 * q];
    last_de_energy[2 * sel[q] + 1] = eo[2 * q + 1];
  }
  mapped_ready = false;
  return dE;
}
