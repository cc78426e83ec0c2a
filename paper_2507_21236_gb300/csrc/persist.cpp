// Save and resume a ground-state search (host code).
//
// The file holds everything the next sweep reads besides the model: every node
// tensor, the isometry centre, the disentangler placement and matrices, the sweep
// count, the FP64 energy known for the current state, and the learned-start
// records. Effective operators are not stored: they are rebuilt on demand from
// the tensors by the same deterministic kernels, so a resumed FP64 run repeats the
// original run's arithmetic bit for bit.
//
// Layout (little-endian): "ATTNST01", int32 version, n_sites, m, n_nodes, centre,
// n_de, sweep_count, first_de_done, learned_used, learned_fallback, mapped_ready;
// uint64 fingerprint of the model's terms; double energy_known; per node int32
// shape[3] and its FP64 entries; int32 pairs[2 n_de]; double u[16 n_de]; int64
// count and doubles of rho_first; int64 count and doubles of last_de_energy.
#include <cstdio>
#include <cstring>
#include <memory>

#include "state.h"

using namespace attn;

namespace {

constexpr char kMagic[8] = {'A', 'T', 'T', 'N', 'S', 'T', '0', '1'};
constexpr int32_t kVersion = 1;

uint64_t fnv1a(uint64_t h, const void* p, size_t n) {
  const unsigned char* c = static_cast<const unsigned char*>(p);
  for (size_t i = 0; i < n; ++i) {
    h ^= c[i];
    h *= 1099511628211ull;
  }
  return h;
}

uint64_t model_fingerprint(const Model& M) {
  uint64_t h = 1469598103934665603ull;
  h = fnv1a(h, &M.n_sites, sizeof(M.n_sites));
  for (const Term& t : M.terms) {
    h = fnv1a(h, &t.n, sizeof(t.n));
    h = fnv1a(h, t.site, sizeof(int) * t.n);
    h = fnv1a(h, t.op.data(), sizeof(double) * t.op.size());
  }
  return h;
}

struct File {
  FILE* f = nullptr;
  std::string path;
  File(const char* p, const char* mode) : f(std::fopen(p, mode)), path(p) {
    ATTN_REQUIRE(f != nullptr, ATTN_EINVAL, "cannot open " + path);
  }
  ~File() {
    if (f) std::fclose(f);
  }
  void put(const void* p, size_t n) {
    ATTN_REQUIRE(std::fwrite(p, 1, n, f) == n, ATTN_EINVAL, "write failed: " + path);
  }
  void get(void* p, size_t n) {
    ATTN_REQUIRE(std::fread(p, 1, n, f) == n, ATTN_EINVAL, "truncated state file: " + path);
  }
  template <class T> void put(const T& v) { put(&v, sizeof(T)); }
  template <class T> T get() {
    T v;
    get(&v, sizeof(T));
    return v;
  }
};

}  // namespace

void attn_state::save(const char* path) {
  ATTN_CHECK_CUDA(cudaStreamSynchronize(ctx->stream));
  File f(path, "wb");
  f.put(kMagic, sizeof(kMagic));
  const int32_t hdr[11] = {kVersion,         model.n_sites,    tree.m,           tree.n_nodes,
                           centre,           (int32_t)des.size(), sweep_count,   first_de_done ? 1 : 0,
                           learned_used,     learned_fallback, mapped_ready ? 1 : 0};
  f.put(hdr, sizeof(hdr));
  f.put<uint64_t>(model_fingerprint(model));
  f.put<double>(energy_known);
  std::vector<double> buf;
  for (int n = 0; n < tree.n_nodes; ++n) {
    const int32_t sh[3] = {dim(n, 0), dim(n, 1), dim(n, 2)};
    f.put(sh, sizeof(sh));
    buf.resize(vol(n));
    ATTN_CHECK_CUDA(cudaMemcpy(buf.data(), tensor(n), sizeof(double) * buf.size(), cudaMemcpyDeviceToHost));
    f.put(buf.data(), sizeof(double) * buf.size());
  }
  for (const auto& d : des) {
    const int32_t pr[2] = {d.first, d.second};
    f.put(pr, sizeof(pr));
  }
  for (const auto& u : us) f.put(u.data(), sizeof(double) * 16);
  for (const std::vector<double>* v : {&rho_first, &last_de_energy}) {
    f.put<int64_t>((int64_t)v->size());
    if (!v->empty()) f.put(v->data(), sizeof(double) * v->size());
  }
}

void attn_state::load(const char* path) {
  File f(path, "rb");
  char magic[8];
  f.get(magic, sizeof(magic));
  ATTN_REQUIRE(std::memcmp(magic, kMagic, sizeof(kMagic)) == 0, ATTN_EINVAL, "not an aTTN state file");
  int32_t hdr[11];
  f.get(hdr, sizeof(hdr));
  ATTN_REQUIRE(hdr[0] == kVersion, ATTN_EINVAL, "unsupported state file version");
  ATTN_REQUIRE(hdr[1] == model.n_sites && hdr[2] == tree.m && hdr[3] == tree.n_nodes, ATTN_EINVAL,
               "state file was written for another lattice size or bond dimension");
  ATTN_REQUIRE(f.get<uint64_t>() == model_fingerprint(model), ATTN_EINVAL,
               "state file was written for another Hamiltonian");
  const int new_centre = hdr[4], n_de = hdr[5];
  ATTN_REQUIRE(new_centre >= 0 && new_centre < tree.n_nodes && n_de >= 0 && n_de <= model.n_sites / 2, ATTN_EINVAL,
               "corrupt state file header");
  const double e_known = f.get<double>();
  std::vector<std::vector<double>> tensors(tree.n_nodes);
  for (int n = 0; n < tree.n_nodes; ++n) {
    int32_t sh[3];
    f.get(sh, sizeof(sh));
    ATTN_REQUIRE(sh[0] == dim(n, 0) && sh[1] == dim(n, 1) && sh[2] == dim(n, 2), ATTN_EINVAL,
                 "state file tensor shape does not match the tree");
    tensors[n].resize(vol(n));
    f.get(tensors[n].data(), sizeof(double) * tensors[n].size());
    for (double v : tensors[n]) ATTN_REQUIRE(std::isfinite(v), ATTN_ENONFINITE, "non-finite tensor in state file");
  }
  std::vector<std::pair<int, int>> d(n_de);
  for (auto& pr : d) {
    int32_t p2[2];
    f.get(p2, sizeof(p2));
    ATTN_REQUIRE(p2[0] >= 0 && p2[0] < p2[1] && p2[1] < model.n_sites, ATTN_EINVAL, "corrupt disentangler sites");
    pr = {p2[0], p2[1]};
  }
  std::vector<std::vector<double>> u(n_de, std::vector<double>(16));
  for (auto& x : u) f.get(x.data(), sizeof(double) * 16);
  std::vector<double> recs[2];
  for (auto& v : recs) {
    const int64_t n = f.get<int64_t>();
    ATTN_REQUIRE(n >= 0 && n <= 16L * model.n_sites, ATTN_EINVAL, "corrupt state file record");
    v.resize(n);
    if (n) f.get(v.data(), sizeof(double) * n);
  }
  // commit: nothing above touched the state
  ATTN_CHECK_CUDA(cudaStreamSynchronize(ctx->stream));
  for (int n = 0; n < tree.n_nodes; ++n)
    ATTN_CHECK_CUDA(cudaMemcpy(tensor(n), tensors[n].data(), sizeof(double) * tensors[n].size(),
                               cudaMemcpyHostToDevice));
  centre = new_centre;
  des = d;
  us = u;
  sweep_count = hdr[6];
  first_de_done = hdr[7] != 0;
  learned_used = hdr[8];
  learned_fallback = hdr[9];
  rho_first = recs[0];
  last_de_energy = recs[1];
  for (auto& e : env) e.valid = false;
  mapped_ready = false;
  if (hdr[10]) set_products();  // H' of the saved disentanglers, as the saved run had it
  energy_known = e_known;
}
