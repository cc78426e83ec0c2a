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
  int f[3];
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
  // MERA-like update of every disentangler (Sec. 4.1.1); returns sum of dE_k
  double de_update(const std::vector<std::vector<double>>* u_start, std::vector<double>* rho_out);
  attn_heff* build_heff(int n);
  double energy();
  double local_step(int n);
  double isometry_error();
};
