// TTN state with per-link effective operators (internal).
#pragma once

#include <cmath>

#include <utility>
#include <vector>

#include "attn_internal.h"
#include "heff.h"
#include "lanczos.h"
#include "mlp.h"
#include "qr.h"

namespace attn {

// Operators on link (n, slot) as seen from node n (Sec. 3.3.2): the summed
// operator of every product lying entirely behind the link (hint) and one
// renormalised operator per product with sites on both sides (open).
struct Env {
  int dim = 0;
  bool valid = false;
  bool has_hint = false;
  DevBuf hint;                         // dim x dim
  std::vector<int> open;               // product ids, in stacking order
  std::vector<std::pair<int, int>> pos;  // (product id, index in ops), sorted by id
  DevBuf ops;                          // [open.size()][dim][dim]
  int find(int q) const;               // index in ops or -1
};

// One-site factor of a probe product and a probe (up to three factors on distinct sites).
struct ProbeFactor {
  int site;
  double op[4];
};
struct Probe {
  int n;
  int f[8];
};

// Probes and coefficient tables of the MERA-like update of a set of disentanglers.
struct DESetup {
  std::vector<int> sel;              // disentangler indices, by position
  std::vector<ProbeFactor> F;
  std::vector<Probe> P;
  std::vector<int> rho_idx;          // [pos][16] probe index of each rho_ij entry
  std::vector<int> ent_begin;        // [pos + 1] entry ranges
  std::vector<int> ent_midx;         // [entry][16] probe index of each M entry
  std::vector<double> ent_C;         // [entry][16]
  std::vector<double> lambda;        // [pos] summed spectral-norm shifts
};

}  // namespace attn

struct attn_state {
  attn_ctx* ctx = nullptr;
  attn::Model model;
  attn::Tree tree;
  std::vector<attn::DevBuf> T;  // node tensors [d0][d1][d2] FP64
  int centre = 0;
  std::vector<std::pair<int, int>> des;
  std::vector<std::vector<double>> us;
  std::vector<attn::Term> mapped;
  std::vector<attn::Prod> prods;
  std::vector<attn::Env> env;  // [node*3 + slot]
  bool mapped_ready = false;
  // FP64 energy <psi|H'|psi> of the current state when known exactly (after a local
  // step with an FP64-exact Ritz value; centre moves are gauge changes and keep it),
  // NaN otherwise. Saves the FP64 matvec that prices the current tensor.
  double energy_known = std::nan("");
  int sweep_count = 0;
  std::vector<double> last_de_energy;  // [k][2]: E_k before / after the last update
  bool first_de_done = false;          // the first disentangler update of this state ran
  std::vector<double> rho_first;       // rho_ij of every disentangler at that first update
  attn_mlp* learned = nullptr;         // optional learned start for the first update (not owned)
  int learned_used = 0, learned_fallback = 0;
  attn::QRWork qrw;
  attn::LanczosWork lw, lw2;
  attn::RefineWork rfw;
  attn::DevBuf colbuf, rbuf, tmpT, idxbuf, opsA, opsB, rw1, rw2;
  // The H_eff of the last local step, kept with its device buffers so that the next
  // build reuses them (its operator stacks and their tensor-core copies take hundreds
  // of MB at m = 128; allocating and freeing them every step cost milliseconds and a
  // device synchronisation each).
  attn_heff* spare_heff = nullptr;
  attn_state() = default;
  attn_state(const attn_state&) = delete;
  attn_state& operator=(const attn_state&) = delete;
  ~attn_state() { delete spare_heff; }
  void recycle(attn_heff* h);

  int dim(int n, int s) const { return tree.shape[3 * n + s]; }
  long vol(int n) const { return (long)dim(n, 0) * dim(n, 1) * dim(n, 2); }
  double* tensor(int n) { return T[n].as<double>(); }

  void init_from_raw(const double* const* raw);
  void invalidate_from(int changed_node);
  void move_centre(int target);
  void set_products();         // map terms through the disentanglers and split
  attn::Env& get_env(int n, int slot);
  void build_physical_env(int n, int slot);
  void renormalise_into(int n, int slot);
  void renorm_batch(const double* Tc, const int d[3], int t, int x, int y, const double* Aops,
                    const std::vector<int>& ia, const double* Bops, const std::vector<int>& ib, double* out);
  // <psi| prod_s f_s |psi> for rank-1 probes of one-site factors (device results)
  void probe_expectations(const std::vector<attn::ProbeFactor>& F, const std::vector<attn::Probe>& P,
                          attn::DevBuf& vals);
  // MERA-like update of the listed disentanglers (all when `only` is null), Sec. 4.1.1;
  // returns the sum of their dE_k
  void de_setup(const std::vector<int>& sel, attn::DESetup& S);
  double de_update(const std::vector<int>* only);
  // two-site density matrices of the TTN on the listed disentanglers' sites ([pos][16])
  std::vector<double> de_rdms(const std::vector<int>& sel);
  // Gamma_k at u (shifted terms, Eq. contracted) and the true E_k(u)
  void de_environment(int k, const double* u16, double* gamma16, double* e_k);
  // <psi_aTTN| o |psi_aTTN> of products of one-site operators (Eq. obs): nsites[o] in
  // 1..4, sites[4 o ..], ops[16 o ..] (2 x 2 row-major per site); mapped through the
  // disentanglers an observable spans at most eight sites
  std::vector<double> measure(int n_obs, const int* nsites, const int* sites, const double* ops);
  attn_heff* build_heff(int n);
  double energy();
  double local_step(int n);
  double isometry_error();
  void save(const char* path);
  void load(const char* path);
};
