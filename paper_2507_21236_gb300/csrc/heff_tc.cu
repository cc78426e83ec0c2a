// BF16 H_eff on the 5th-generation tensor cores (tcgen05 + TMEM + TMA), FP32
// accumulation (Sec. 3.3.2 last paragraph, Sec. 4.4.2, Fig. eff-op-cost).
//
// For a pair kind (p, q) with slice slot s, every slice X_s (P x Q, the
// tensor with slot s fixed) gets
//     Y_s = sum_r A_r X_s B_r^T      (A_r: P x P on slot p, B_r: Q x Q on slot q)
// computed per product as two chained MMAs:
//   stage 1:  D1[j][i'] = sum_j' B_r[j][j'] X_s[i'][j']     (A = B_r, B = X_s, both in shared memory)
//   convert:  D1 (FP32) -> BF16 Z^T[j][i'], packed in place in tensor memory
//   stage 2:  D2[j][i] += sum_i' Z^T[j][i'] A_r[i][i']       (A = Z^T from tensor memory, B = A_r)
// so D2 = Y_s^T stays in TMEM across all products. Taking the stage-2 A
// operand from TMEM keeps the stage-1 result out of shared memory, whose
// bandwidth bounds a 128 x 128 MMA fed from shared memory alone.
//
// One CTA owns two slices of the same pair kind: every operator tile it loads
// serves both, which halves the TMA traffic per product. TMEM holds
// D1 and D2 for each slice (4 x 128 columns). The MMA order is
//   S1(r, 0), S1(r, 1), S2(r, 0), S2(r, 1), S1(r+1, 0), ...
// so that converting slice 0 overlaps stage 1 of slice 1 and converting slice 1
// overlaps stage 2 of slice 0; each 64-column half of Z^T is handed to stage 2
// as soon as it is packed. At N = 128 one MMA (K = 16) takes 64 cycles, which
// one issuing thread cannot sustain between its waits and commits: the two
// stages are issued by two threads, with descriptors precomputed and each K
// block unrolled. Operator tiles stream through one ring of 16 KB
// K-block stages in consumption order (B_r, A_r, B_{r+1}, ...). A slice pair's
// product list may be split over several CTAs (`rsplit`, chosen by an
// autotuner at the first application) whose partial Y_s meet by FP32 atomics.
//
// Warp roles (640 threads): warp 0 = TMA producer, warp 1 = TMEM allocation
// and stage-1 MMA issue, warp 2 = stage-2 MMA issue, warps 4-19 = conversion
// and epilogue, eight per slice in two
// column halves (warp w reads TMEM lanes 32*(w%4) .. +31). Internal
// (single-link) operators enter as products with an identity partner.
//
// A three-link product A_r (x) B_r (x) C_r (slots 0, 1, 2) is applied in two
// steps: a batched TN GEMM contracts slot 2 with C_r, giving per product the
// slice stack W_r[c] = (x x_2 C_r)[:, :, c] in the layout of the pair kind (0, 1);
// the same kernel then runs in per-product mode (kPP), where each product brings
// its own X slices through the ring (B_r, X_{r,s0}, X_{r,s0+1}, A_r) and the
// result adds onto the kind-(0, 1) output. Every mbarrier wait is
// bounded (about 2 s of clock); on timeout the kernel records an error code,
// stops issuing work, waits (bounded) for its in-flight copies, frees TMEM and
// returns.
#include <algorithm>
#include <cstring>

#include "gemm_tc.h"
#include "heff.h"
#include "ozaki.h"
#include "tc_ptx.h"

namespace attn {

// cuTensorMapEncodeTiled through the runtime's driver entry point, so that the
// library does not link libcuda directly (it loads on machines without a driver).
PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q);
    ATTN_REQUIRE(e == cudaSuccess && q == cudaDriverEntryPointSuccess && p, ATTN_ECUDA,
                 "cuTensorMapEncodeTiled is not available from the driver");
    fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  }
  return fn;
}

namespace {

using namespace tc;

constexpr int kThreads = 640;         // 4 role warps + 16 conversion/epilogue warps
constexpr int kHalfWarps = 4;         // conversion warps per slice half (one Z-full arrival each)
constexpr int kTileBytes = 128 * 128 * 2;  // one 128 x 128 BF16 tile (two 64-wide K blocks)
constexpr int kKBlockBytes = 128 * 128;    // 128 rows x 128 bytes
constexpr int kStages = 10;                // operator ring depth (K blocks), BF16
constexpr int kStagesTF = 6;               // the same for TF32: the two FP32 X slices take twice the room
constexpr int kStagesPP = 14;              // ring depth when every product brings its own slices
constexpr uint32_t kTmemCols = 512;

struct KindParams {
  int P, Q, S, R;     // slice rows/cols, slices, products
  int rsplit;         // CTAs per slice pair, each owning a contiguous range of products
  int cta_begin;      // first CTA index of this kind
  float* Y;           // [S][P][Q] fp32 output (written, or accumulated when rsplit > 1)
  int accumulate;     // add to Y instead of writing it
};

struct TcParams {
  KindParams kind[3];
  int nkinds;
  int* err;           // device error word (0 = ok)
  long long wait;     // wait limit (cycles) of the MMA-issue, conversion and epilogue threads
  // Persistent form (segs != null): CTA b walks segments seg_start[b] .. seg_start[b + 1] - 1
  // of a cost-balanced cut of the node's (kind, slice pair, product) list; otherwise each
  // CTA owns one (kind, slice pair, product range) given by its index and the kinds' splits.
  const int4* segs;   // {kind, slice pair, first product, products | 1 << 30 when added atomically}
  const int* seg_start;
};

// One CTA's share of the work: products r0 .. r0 + n - 1 of slice pair `pair` of a kind.
struct Seg {
  int kind, pair, r0, n;
  bool atomic;  // the pair's output is shared with other CTAs (or adds onto an earlier result)
};

struct TcMaps {
  CUtensorMap x[3], a[3], b[3];
};

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
  __nv_bfloat162 h = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<uint32_t*>(&h);
}

// ------------------------------------------------------------------ kernel
// kPP = false: the CTA's two X slices are loaded once and serve every product.
// kPP = true: product r has its own slices (slice z = r S + s of the X map),
// streamed through the ring between B_r and A_r.
// kTF = false: BF16 operands (kind::f16), the stage-1 result packed to BF16 in TMEM
// by the conversion warps; kTF = true: TF32 operands (kind::tf32, FP32 storage
// rounded to TF32), and stage 2 reads the FP32 stage-1 result from TMEM as it is
// (the MMA uses its TF32 part), so there is no conversion pass.
template <bool kPP, bool kTF>
__global__ void __launch_bounds__(kThreads, 1) sandwich_tc_kernel(const __grid_constant__ TcMaps maps, TcParams prm) {
  constexpr int NS = kPP ? kStagesPP : (kTF ? kStagesTF : kStages);
  constexpr int KB = kTF ? 32 : 64;  // elements per 128-byte K block
  constexpr int KS = kTF ? 8 : 16;   // elements per MMA K step (32 bytes)
  constexpr int kXBytes = (kTF ? 4 : 2) * kTileBytes;  // X of both slices: up to 4 (TF32) or 2 K blocks
  extern __shared__ uint8_t smem_raw[];
  // 1024-aligned regions: X of both slices (K block kb of slice u at
  // 32 KB kb + 16 KB u; absent when kPP), operator ring, barriers.
  const uint32_t raw = smem_u32(smem_raw);
  const uint32_t base = (raw + 1023u) & ~1023u;
  uint8_t* gbase = smem_raw + (base - raw);
  const uint32_t sX = base;
  const uint32_t sRing = kPP ? base : base + kXBytes;
  const uint32_t sBar = sRing + NS * kKBlockBytes;
  enum {
    XFULL = 0,
    FULL = 1,
    EMPTY = 1 + NS,
    D1FULL = 1 + 2 * NS,  // [slice]: stage 1 done
    ZFULL = 3 + 2 * NS,   // [slice][half]: that half of Z^T packed in TMEM
    S2DONE = 7 + 2 * NS,  // [slice]: stage 2 done, D1 free for the next product
    D2FULL = 9 + 2 * NS,  // a segment's stage 2 complete
    S1END = 10 + 2 * NS,  // [issuer]: every MMA of that issuer complete (TMEM may be freed)
    XEMPTY = 12 + 2 * NS, // a segment's stage-1 MMAs complete: its X may be replaced
    D2EMPTY = 13 + 2 * NS,  // the epilogue has read a segment's D2
    NBAR = 14 + 2 * NS
  };
  uint64_t* bars = reinterpret_cast<uint64_t*>(gbase + (sBar - base));
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + NBAR);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
  auto bar = [&](int i) { return sBar + 8u * (uint32_t)i; };

  // the CTA's segments: one per CTA (split grid), or a cost-balanced run of them (persistent)
  const int nseg = prm.segs ? prm.seg_start[blockIdx.x + 1] - prm.seg_start[blockIdx.x] : 1;
  auto seg_at = [&](int j) {
    Seg g;
    if (prm.segs) {
      const int4 v = prm.segs[prm.seg_start[blockIdx.x] + j];
      g.kind = v.x;
      g.pair = v.y;
      g.r0 = v.z;
      g.n = v.w & 0x3FFFFFFF;
      g.atomic = (v.w >> 30) & 1;
      return g;
    }
    g.kind = 0;
    if (prm.nkinds > 1 && (int)blockIdx.x >= prm.kind[1].cta_begin) g.kind = 1;
    if (prm.nkinds > 2 && (int)blockIdx.x >= prm.kind[2].cta_begin) g.kind = 2;
    const KindParams& k = g.kind == 0 ? prm.kind[0] : (g.kind == 1 ? prm.kind[1] : prm.kind[2]);
    const int local = blockIdx.x - k.cta_begin;
    const int part = local % k.rsplit;
    g.pair = local / k.rsplit;
    g.r0 = (int)((long)k.R * part / k.rsplit);
    g.n = (int)((long)k.R * (part + 1) / k.rsplit) - g.r0;
    g.atomic = k.rsplit > 1 || k.accumulate;
    return g;
  };
  // (static indices only: a runtime index into the parameter struct would copy it to local memory)
  auto kind_of = [&](int k) -> KindParams {
    if (k == 1) return prm.kind[1];
    if (k == 2) return prm.kind[2];
    return prm.kind[0];
  };
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  if (threadIdx.x == 0) {
    mbar_init(bar(XFULL), 1);
    mbar_init(bar(XEMPTY), 1);
    for (int i = 0; i < NS; ++i) {
      mbar_init(bar(FULL + i), 1);
      mbar_init(bar(EMPTY + i), 1);
    }
    for (int u = 0; u < 2; ++u) {
      mbar_init(bar(D1FULL + u), 1);
      mbar_init(bar(S2DONE + u), 1);
    }
    for (int i = 0; i < 4; ++i) mbar_init(bar(ZFULL + i), kHalfWarps);
    mbar_init(bar(D2FULL), 1);
    mbar_init(bar(D2EMPTY), 16);
    mbar_init(bar(S1END), 1);
    mbar_init(bar(S1END + 1), 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(kTmemCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = *tmem_slot;
  // TMEM: D1 of slice u in columns 128u .. 128u+P-1 (Z^T packed in place), D2 of slice u at 256 + 128u
  auto tD1 = [&](int u) { return tmem + 128u * (uint32_t)u; };
  auto tD2 = [&](int u) { return tmem + 256u + 128u * (uint32_t)u; };

  if (warp == 0 && lane == 0) {
    // ---- producer: per segment X of both slices (or per product when kPP), then the
    // operator K blocks in consumption order; X of a segment is loaded once the stage-1
    // MMAs of the previous one have read theirs
    int issued = 0, xissued = 0;
    int st = 0;       // ring stage of the next load
    uint32_t ph = 0;  // parity of that stage's current fill
    bool ok = true;
    for (int j = 0; ok && j < nseg; ++j) {
      const Seg g = seg_at(j);
      const KindParams kp = kind_of(g.kind);
      const int P = kp.P, Q = kp.Q, s0 = 2 * g.pair, nsl = (s0 + 1 < kp.S) ? 2 : 1;
      const int nkbQ = (Q + KB - 1) / KB, nkbP = (P + KB - 1) / KB;
      const CUtensorMap* mX = &maps.x[g.kind];
      const CUtensorMap* mA = &maps.a[g.kind];
      const CUtensorMap* mB = &maps.b[g.kind];
      if (!kPP) {
        if (j > 0 && !mbar_wait(bar(XEMPTY), (j - 1) & 1, prm.err, 12, abort_flag)) {
          ok = false;
          break;
        }
        mbar_expect_tx(bar(XFULL), (uint32_t)(nsl * nkbQ * P * 128));
        for (int u = 0; u < nsl; ++u)
          for (int kb = 0; kb < nkbQ; ++kb)
            tma_load_3d(sX + kb * kTileBytes + u * (kTileBytes / 2), mX, KB * kb, 0, s0 + u, bar(XFULL));
        ++xissued;
      }
      const int nparts = kPP ? 2 + nsl : 2;  // B_r, [X_{r,s0}, X_{r,s0+1}], A_r
      for (int r = 0; ok && r < g.n; ++r) {
        for (int part = 0; ok && part < nparts; ++part) {
          const bool isB = part == 0, isA = part == nparts - 1;
          const CUtensorMap* mp = isB ? mB : (isA ? mA : mX);
          const int nkb = isA ? nkbP : nkbQ;
          const int z = isB || isA ? g.r0 + r : (g.r0 + r) * kp.S + s0 + (part - 1);
          const uint32_t bytes = isB || isA ? (uint32_t)kKBlockBytes : (uint32_t)(P * 128);
          for (int kb = 0; kb < nkb; ++kb) {
            // the stage's previous contents (fill ph - 1) must have been consumed
            if (issued >= NS && !mbar_wait(bar(EMPTY + st), ph ^ 1u, prm.err, 11, abort_flag)) {
              ok = false;
              break;
            }
            mbar_expect_tx(bar(FULL + st), bytes);
            tma_load_3d(sRing + st * kKBlockBytes, mp, KB * kb, 0, z, bar(FULL + st));
            ++issued;
            if (++st == NS) { st = 0; ph ^= 1u; }
          }
        }
      }
    }
    // drain: wait (bounded) until every issued load has landed
    if (xissued > 0) {
      long long t0 = clock64();
      while (!mbar_try_wait(bar(XFULL), (xissued - 1) & 1) && clock64() - t0 < kWaitCycles) {}
    }
    for (int q = (issued > NS ? issued - NS : 0); q < issued; ++q) {
      long long t0 = clock64();
      while (!mbar_try_wait(bar(FULL + q % NS), (q / NS) & 1) && clock64() - t0 < kWaitCycles) {}
    }
  } else if ((warp == 1 || warp == 2) && lane == 0) {
    // ---- MMA issue, split over two threads on different SM sub-partitions: a
    // single thread cannot issue N = 128 MMAs (64 cycles each) back to back once
    // waits and commits are interleaved. Warp 1 issues stage 1, warp 2 stage 2;
    // the pipe sees S1(r,0), S1(r,1), S2(r,0), S2(r,1), S1(r+1,0), ...
    // Barrier phases count products per slice across segments (cnt[u]).
    const uint64_t dRing0 = sw128_desc(sRing);  // ring stage st: + st * (kKBlockBytes >> 4)
    const uint32_t barFull = bar(FULL), barEmpty = bar(EMPTY);
    int st = 0;        // ring stage of the product's first K block
    uint32_t ph = 0;   // its phase parity
    auto advance = [&](int n) {
      for (int i = 0; i < n; ++i)
        if (++st == NS) { st = 0; ph ^= 1u; }
    };
    int cnt[2] = {0, 0};
    bool ok = true;
    if (warp == 1) {
      const uint64_t dX0 = sw128_desc(sX);  // X block kb of slice u: + (32 KB kb + 16 KB u) >> 4
      for (int j = 0; ok && j < nseg; ++j) {
        const Seg g = seg_at(j);
        const KindParams kp = kind_of(g.kind);
        const int P = kp.P, Q = kp.Q, nsl = (2 * g.pair + 1 < kp.S) ? 2 : 1;
        const int nkbQ = (Q + KB - 1) / KB, nkbP = (P + KB - 1) / KB;
        const int nkbX = kPP ? nsl * nkbQ : 0;  // ring K blocks of X per product
        const uint32_t id = idesc_of<kTF>(128, P);  // both stages: M = 128 TMEM lanes, N = P
        const int nk16Q = Q / KS;
        if (!kPP && !mbar_wait(bar(XFULL), j & 1, prm.err, 31, abort_flag, prm.wait)) { ok = false; break; }
        for (int r = 0; ok && r < g.n; ++r) {
          // stage 1 per slice: D1_u = B_r X_u^T (the B_r blocks serve both slices)
          for (int u = 0; ok && u < nsl; ++u) {
            // D1_u holds Z_u of the previous product until its stage 2 has completed
            if (cnt[u] > 0 && !mbar_wait(bar(S2DONE + u), (cnt[u] - 1) & 1, prm.err, 35, abort_flag, prm.wait)) {
              ok = false;
              break;
            }
            fence_after();
            int s1 = st;
            uint32_t p1 = ph;
            int sx = st + nkbQ * (1 + u);  // ring stage of this slice's first X block (kPP)
            uint32_t px = ph;
            while (sx >= NS) { sx -= NS; px ^= 1u; }
            for (int kb = 0; kb < nkbQ; ++kb) {
              if (u == 0 && !mbar_wait(barFull + 8 * s1, p1, prm.err, 32, abort_flag, prm.wait)) { ok = false; break; }
              if (kPP && !mbar_wait(barFull + 8 * sx, px, prm.err, 36, abort_flag, prm.wait)) { ok = false; break; }
              const uint64_t dB = dRing0 + (uint64_t)(s1 * (kKBlockBytes >> 4));
              const uint64_t dX = kPP ? dRing0 + (uint64_t)(sx * (kKBlockBytes >> 4))
                                      : dX0 + (uint64_t)((kb * kTileBytes + u * (kTileBytes / 2)) >> 4);
              const int n4 = nk16Q - 4 * kb;
              if (n4 >= 4) {
                mma4_ss_t<kTF>(tD1(u), dB, dX, id, kb > 0 ? 1u : 0u);
              } else {
                for (int k4 = 0; k4 < n4; ++k4)
                  mma_ss<kTF>(tD1(u), dB + 2 * k4, dX + 2 * k4, id, (kb > 0 || k4 > 0) ? 1u : 0u);
              }
              if (u == nsl - 1) mma_commit(barEmpty + 8 * s1);
              if (kPP) mma_commit(barEmpty + 8 * sx);
              if (++s1 == NS) { s1 = 0; p1 ^= 1u; }
              if (++sx == NS) { sx = 0; px ^= 1u; }
            }
            if (!ok) break;
            mma_commit(bar(D1FULL + u));
            ++cnt[u];
          }
          advance(nkbQ + nkbX + nkbP);
        }
        // once these MMAs complete, the segment's X is no longer read
        if (ok && !kPP) mma_commit(bar(XEMPTY));
      }
      mma_commit(bar(S1END));
      long long t0 = clock64();
      while (!mbar_try_wait(bar(S1END), 0) && clock64() - t0 < kWaitCycles) {}
    } else {
      int done = 0;  // segments whose stage-2 MMAs were committed to D2FULL
      uint32_t zpar = 0;  // bit 2 u + h: parity of the products consumed from [slice u][half h] (ZFULL)
      for (int j = 0; ok && j < nseg; ++j) {
        const Seg g = seg_at(j);
        const KindParams kp = kind_of(g.kind);
        const int P = kp.P, Q = kp.Q, nsl = (2 * g.pair + 1 < kp.S) ? 2 : 1;
        const int nkbQ = (Q + KB - 1) / KB, nkbP = (P + KB - 1) / KB;
        const int nkbX = kPP ? nsl * nkbQ : 0;
        const uint32_t id = idesc_of<kTF>(128, P);
        const int nk16P = P / KS;
        for (int r = 0; ok && r < g.n; ++r) {
          advance(nkbQ + nkbX);
          // stage 2 per slice: D2_u += Z_u^T A_r^T, Z_u read from TMEM half by half
          for (int u = 0; ok && u < nsl; ++u) {
            int s2 = st;
            uint32_t p2 = ph;
            for (int kb = 0; kb < nkbP; ++kb) {
              // BF16: each 64-column half of Z^T once the conversion warps packed it;
              // TF32: the whole stage-1 result once its MMAs are complete
              if (kTF ? (kb == 0 && !mbar_wait(bar(D1FULL + u), cnt[u] & 1, prm.err, 34, abort_flag, prm.wait))
                      : !mbar_wait(bar(ZFULL + 2 * u + kb), (zpar >> (2 * u + kb)) & 1u, prm.err, 34, abort_flag,
                                   prm.wait)) {
                ok = false;
                break;
              }
              if (!kTF) zpar ^= 1u << (2 * u + kb);
              // the segment's first MMA restarts D2: the epilogue must have read the last one's
              if (j > 0 && r == 0 && u == 0 && kb == 0 &&
                  !mbar_wait(bar(D2EMPTY), (j - 1) & 1, prm.err, 37, abort_flag, prm.wait)) {
                ok = false;
                break;
              }
              if (u == 0 && !mbar_wait(barFull + 8 * s2, p2, prm.err, 33, abort_flag, prm.wait)) { ok = false; break; }
              fence_after();  // Z was written by tcgen05.st in other threads (BF16) or by MMAs
              const uint64_t dA = dRing0 + (uint64_t)(s2 * (kKBlockBytes >> 4));
              const uint32_t aZ = tD1(u) + (kTF ? 32u : 64u) * (uint32_t)kb;
              const int n4 = nk16P - 4 * kb;
              if (n4 >= 4) {
                mma4_ts_t<kTF>(tD2(u), aZ, dA, id, (r > 0 || kb > 0) ? 1u : 0u);
              } else {
                for (int k4 = 0; k4 < n4; ++k4)
                  mma_ts<kTF>(tD2(u), aZ + 8 * k4, dA + 2 * k4, id, (r > 0 || kb > 0 || k4 > 0) ? 1u : 0u);
              }
              if (u == nsl - 1) mma_commit(barEmpty + 8 * s2);
              if (++s2 == NS) { s2 = 0; p2 ^= 1u; }
            }
            if (!ok) break;
            mma_commit(bar(S2DONE + u));
            ++cnt[u];
          }
          advance(nkbP);
        }
        if (!ok) break;
        mma_commit(bar(D2FULL));
        ++done;
      }
      // every MMA this thread issued must finish before TMEM can be freed
      if (done > 0) {
        long long t0 = clock64();
        while (!mbar_try_wait(bar(D2FULL), (done - 1) & 1) && clock64() - t0 < kWaitCycles) {}
      }
      mma_commit(bar(S1END + 1));
      long long t0 = clock64();
      while (!mbar_try_wait(bar(S1END + 1), 0) && clock64() - t0 < kWaitCycles) {}
    }
  } else if (warp >= 4) {
    // ---- conversion D1 -> packed BF16 Z^T and the epilogue. Slice u has warps
    // 4+8u .. 11+8u; warps of half hh own the 64 columns from 64 hh of the slice's
    // D1 and pack them into the first 32 of those columns (nothing else reads them).
    const int cw = warp - 4;
    const int u = cw >> 3, hh = (cw >> 2) & 1;
    const int q4 = warp & 3;
    const int jl = q4 * 32 + lane;  // TMEM lane == row jl of D1 and of D2 = Y^T
    const uint32_t lane_off = (uint32_t)(q4 * 32) << 16;
    const int c0 = 64 * hh;
    const uint32_t tz = tD1(u) + lane_off + (uint32_t)c0;
    int cnt = 0;  // stage-1 results of this warp's slice so far (D1FULL phases), converted or not
    bool ok = true;
    for (int j = 0; ok && j < nseg; ++j) {
      const Seg g = seg_at(j);
      const KindParams kp = kind_of(g.kind);
      const int P = kp.P, Q = kp.Q, s0 = 2 * g.pair, nsl = (s0 + 1 < kp.S) ? 2 : 1;
      const bool mine = u < nsl && c0 < P;  // this warp's columns exist in this segment
      for (int r = 0; !kTF && mine && r < g.n; ++r) {
        // warp-uniform: the TMEM accesses below are .sync.aligned
        if (!__all_sync(0xffffffffu, mbar_wait(bar(D1FULL + u), cnt & 1, prm.err, 41, abort_flag, prm.wait))) {
          ok = false;
          break;
        }
        fence_after();
        uint32_t w[32];  // packed BF16 pairs of this thread's 64 columns
#pragma unroll
        for (int t = 0; t < 2; ++t) {
          float v[32];
          tmem_ld32(tz + 32 * t, v);
#pragma unroll
          for (int h = 0; h < 16; ++h) w[16 * t + h] = pack_bf16(v[2 * h], v[2 * h + 1]);
        }
        tmem_st32(tz, w);
        fence_before();
        // one arrival per warp: 256 arrivals on one barrier would serialise on its word
        __syncwarp();
        if (lane == 0) mbar_arrive(bar(ZFULL + 2 * u + hh));
        ++cnt;
      }
      if (!ok) break;
      // a slice whose columns lie outside this warp's half still advanced D1FULL
      if (!kTF && !mine && u < nsl) cnt += g.n;
      // the segment's result; every warp takes part in the phases, whether it has columns or not
      if (!__all_sync(0xffffffffu, mbar_wait(bar(D2FULL), j & 1, prm.err, 43, abort_flag, prm.wait))) {
        ok = false;
        break;
      }
      fence_after();
      if (mine && g.n > 0) {
        float* yp = kp.Y + ((long)(s0 + u) * P + c0) * Q + jl;  // walks down column jl of Y_s
        // partial sums of a shared product list meet here, and per-product results add onto the pair result
        for (int cc = c0; cc < c0 + 64 && cc < P; cc += 32) {
          float v[32];
          tmem_ld32(tD2(u) + lane_off + cc, v);  // v[c] = Y_s[cc + c][jl]
          if (jl < Q) {
#pragma unroll
            for (int c = 0; c < 32; ++c) {
              if (cc + c < P) {
                if (g.atomic) atomicAdd(yp, v[c]);
                else *yp = v[c];
              }
              yp += Q;
            }
          }
        }
      }
      fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(bar(D2EMPTY));
    }
  }
  fence_before();
  __syncthreads();
  if (warp == 1) {
    fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols));
  }
}

// ------------------------------------------------------------ prep kernels
// Operand element of the tensor-core path: BF16, or FP32 rounded to TF32.
template <class T> __device__ __forceinline__ T to_operand(double v);
template <> __device__ __forceinline__ __nv_bfloat16 to_operand<__nv_bfloat16>(double v) { return __double2bfloat16(v); }
template <> __device__ __forceinline__ float to_operand<float>(double v) { return tc::round_tf32(__double2float_rn(v)); }

// x (fp64 [m0][m1][m2]) -> slice-major operand copies for the three pair kinds:
// X01[c][a][b], X02[b][a][c], X12[a][b][c]. One block handles a 32 x 32 tile of
// the (b, c) plane of one a: X02 and X12 rows are contiguous in c like x, and
// the b <-> c transpose for X01 goes through shared memory, so every global
// access is coalesced.
constexpr int kTile = 32;

template <class T>
__global__ void prep_x_kernel(const double* __restrict__ x, int m0, int m1, int m2, T* x01, T* x02, T* x12) {
  __shared__ T t[kTile][kTile + 2];
  const int a = blockIdx.z, b0 = blockIdx.y * kTile, c0 = blockIdx.x * kTile;
  for (int bb = threadIdx.y; bb < kTile; bb += blockDim.y) {
    const int b = b0 + bb, c = c0 + threadIdx.x;
    if (b < m1 && c < m2) {
      const T v = to_operand<T>(x[((long)a * m1 + b) * m2 + c]);
      t[bb][threadIdx.x] = v;
      if (x02) x02[((long)b * m0 + a) * m2 + c] = v;
      if (x12) x12[((long)a * m1 + b) * m2 + c] = v;
    }
  }
  if (!x01) return;
  __syncthreads();
  for (int cc = threadIdx.y; cc < kTile; cc += blockDim.y) {
    const int c = c0 + cc, b = b0 + threadIdx.x;
    if (b < m1 && c < m2) x01[((long)c * m0 + a) * m1 + b] = t[threadIdx.x][cc];
  }
}

// y = Y01^T + Y02^T + Y12 (fp32 -> fp64), the same tiling as prep_x_kernel.
__global__ void combine_kernel(double* __restrict__ y, int m0, int m1, int m2, const float* y01, const float* y02,
                               const float* y12) {
  __shared__ float t[kTile][kTile + 1];
  const int a = blockIdx.z, b0 = blockIdx.y * kTile, c0 = blockIdx.x * kTile;
  if (y01) {
    for (int cc = threadIdx.y; cc < kTile; cc += blockDim.y) {
      const int c = c0 + cc, b = b0 + threadIdx.x;
      if (b < m1 && c < m2) t[threadIdx.x][cc] = y01[((long)c * m0 + a) * m1 + b];
    }
    __syncthreads();
  }
  for (int bb = threadIdx.y; bb < kTile; bb += blockDim.y) {
    const int b = b0 + bb, c = c0 + threadIdx.x;
    if (b < m1 && c < m2) {
      double v = y01 ? (double)t[bb][threadIdx.x] : 0.0;
      if (y02) v += (double)y02[((long)b * m0 + a) * m2 + c];
      if (y12) v += (double)y12[((long)a * m1 + b) * m2 + c];
      y[((long)a * m1 + b) * m2 + c] = v;
    }
  }
}

dim3 tile_grid(const int* m) { return dim3((m[2] + kTile - 1) / kTile, (m[1] + kTile - 1) / kTile, m[0]); }

template <class T>
__global__ void to_operand_kernel(T* dst, const double* src, long n) {
  for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < n; e += (long)gridDim.x * blockDim.x)
    dst[e] = to_operand<T>(src[e]);
}

template <class T>
__global__ void identity_operand_kernel(T* dst, int m) {
  for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < (long)m * m; e += (long)gridDim.x * blockDim.x)
    dst[e] = to_operand<T>((e / m == e % m) ? 1.0 : 0.0);
}

int vgrid(long n) { return (int)std::max<long>(1, std::min<long>((n + 255) / 256, 4096)); }

// Host: 3-D tiled tensor map over a [D2][D1][D0] operand array (BF16, or FP32 holding
// TF32) with a {128 bytes, rows, 1} box and the 128B swizzle.
void encode_map(CUtensorMap* map, const void* ptr, int d0, int d1, int d2, int box_rows, bool tf) {
  const int es = tf ? 4 : 2;
  cuuint64_t dims[3] = {(cuuint64_t)d0, (cuuint64_t)d1, (cuuint64_t)d2};
  cuuint64_t strides[2] = {(cuuint64_t)d0 * es, (cuuint64_t)d0 * d1 * es};
  cuuint32_t box[3] = {(cuuint32_t)(128 / es), (cuuint32_t)box_rows, 1};
  cuuint32_t estr[3] = {1, 1, 1};
  CUresult res = tensor_map_encoder()(map, tf ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3,
                                      const_cast<void*>(ptr), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                                      CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                                      CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  ATTN_REQUIRE(res == CUDA_SUCCESS, ATTN_ECUDA, "cuTensorMapEncodeTiled failed (" + std::to_string((int)res) + ")");
}

}  // namespace

// Per-H_eff tensor-core state of one operand type.
struct TcState {
  bool tf = false;       // TF32 operands (FP32 storage) instead of BF16
  DevBuf a[3], b[3];     // operator stacks per kind [R'][P][P], [R'][Q][Q]
  int R[3] = {0, 0, 0};  // products per kind (incl. internal operators)
  DevBuf x[3];           // slice-major input per kind
  DevBuf y[3];           // fp32 output per kind
  DevBuf err;
  TcMaps maps;
  TcParams prm;
  int grid = 0;
  size_t smem = 0;
  int rsplit = 1;        // products of a slice split over this many CTAs (autotuned)
  bool tuned = false;
  bool stale = false;    // the H_eff's operators changed since the copies were made
  // persistent form: one CTA per SM over a cost-balanced cut of the work list
  bool persistent = false, seg_atomic = false;
  int pgrid = 0;
  std::vector<int4> hsegs;
  std::vector<int> hstart;
  DevBuf segs, seg_start;
  // three-link products: factors per slot, the slot-2 contraction of one chunk
  // of products ([tchunk][m2][m0][m1]) and the per-product kernel's maps and parameters
  int nt = 0, tchunk = 0;
  DevBuf t0, t1, t2, w;
  TcMaps tmaps;
  TcParams tprm;
  size_t es() const { return tf ? 4 : 2; }
  // Split every kind's product list f ways (at least 8 products per CTA) and lay out
  // the grid: one CTA per slice pair and product range.
  // f >= 1: split grid (products of a slice pair over f CTAs); f = 0: persistent form
  void set_split(int f) {
    persistent = f == 0;
    rsplit = f;
    if (persistent) {
      prm.segs = segs.as<int4>();
      prm.seg_start = seg_start.as<int>();
      grid = pgrid;
      return;
    }
    prm.segs = nullptr;
    prm.seg_start = nullptr;
    int cta = 0;
    for (int k = 0; k < prm.nkinds; ++k) {
      KindParams& kp = prm.kind[k];
      kp.rsplit = std::max(1, std::min(f, kp.R / 8));
      kp.cta_begin = cta;
      cta += (kp.S + 1) / 2 * kp.rsplit;
    }
    grid = cta;
    rsplit = f;
  }
  bool split_any() const {
    if (persistent) return seg_atomic;
    for (int k = 0; k < prm.nkinds; ++k)
      if (prm.kind[k].rsplit > 1) return true;
    return false;
  }
  // Cut the work list (kind, slice pair, product), each product weighted by its MMA work
  // P + Q, into G runs of equal cost, one per CTA; a slice pair whose products land in
  // more than one run is summed atomically.
  void build_segments(int G, cudaStream_t st) {
    double total = 0.0;
    for (int k = 0; k < prm.nkinds; ++k)
      total += (double)((prm.kind[k].S + 1) / 2) * prm.kind[k].R * (prm.kind[k].P + prm.kind[k].Q);
    hsegs.clear();
    hstart.assign(G + 1, 0);
    const double per = total / G;
    double pos = 0.0;
    int cur = -1;  // CTA of the last segment
    seg_atomic = false;
    for (int k = 0; k < prm.nkinds; ++k) {
      const KindParams& kp = prm.kind[k];
      const double w = kp.P + kp.Q;
      for (int pair = 0; pair < (kp.S + 1) / 2; ++pair) {
        const size_t first = hsegs.size();
        for (int r = 0; r < kp.R; ++r, pos += w) {
          const int c = std::min(G - 1, (int)(pos / per));
          if (hsegs.size() > first && c == cur && hsegs.back().x == k && hsegs.back().y == pair) {
            ++hsegs.back().w;
          } else {
            for (int cc = cur + 1; cc <= c; ++cc) hstart[cc] = (int)hsegs.size();
            hsegs.push_back(make_int4(k, pair, r, 1));
            cur = c;
          }
        }
        const bool shared = hsegs.size() - first > 1;
        for (size_t i = first; i < hsegs.size(); ++i)
          if (shared || kp.accumulate) {
            hsegs[i].w |= 1 << 30;
            seg_atomic = true;
          }
      }
    }
    for (int cc = cur + 1; cc <= G; ++cc) hstart[cc] = (int)hsegs.size();
    segs.reserve(sizeof(int4) * std::max<size_t>(hsegs.size(), 1));
    seg_start.reserve(sizeof(int) * (size_t)(G + 1));
    ATTN_CHECK_CUDA(cudaMemcpyAsync(segs.p, hsegs.data(), sizeof(int4) * hsegs.size(), cudaMemcpyHostToDevice, st));
    ATTN_CHECK_CUDA(cudaMemcpyAsync(seg_start.p, hstart.data(), sizeof(int) * (size_t)(G + 1), cudaMemcpyHostToDevice, st));
    pgrid = G;
  }
};

bool tc_supported(const attn_heff* h) {
  for (int s = 0; s < 3; ++s)
    if (h->m[s] % 16 != 0 || h->m[s] > 128 || h->m[s] < 16) return false;
  return true;
}

void tc_invalidate(attn_heff* h) {
  for (int i = 0; i < 2; ++i)
    if (h->tc[i]) static_cast<TcState*>(h->tc[i])->stale = true;
}

void tc_release(attn_heff* h) {
  for (int i = 0; i < 2; ++i) {
    delete static_cast<TcState*>(h->tc[i]);
    h->tc[i] = nullptr;
  }
}

namespace {

// Launch the pair-product kernel (or its per-product form) for the state's operand type.
void launch_sandwich(bool pp, const TcState* t, int grid, const TcMaps& maps, const TcParams& prm, cudaStream_t st) {
  if (t->tf) {
    if (pp) sandwich_tc_kernel<true, true><<<grid, kThreads, t->smem, st>>>(maps, prm);
    else sandwich_tc_kernel<false, true><<<grid, kThreads, t->smem, st>>>(maps, prm);
  } else {
    if (pp) sandwich_tc_kernel<true, false><<<grid, kThreads, t->smem, st>>>(maps, prm);
    else sandwich_tc_kernel<false, false><<<grid, kThreads, t->smem, st>>>(maps, prm);
  }
}

template <class T>
void to_operand(const TcState* t, cudaStream_t st, void* dst, const double* src, long n) {
  to_operand_kernel<T><<<vgrid(n), 256, 0, st>>>(static_cast<T*>(dst), src, n);
}

void convert(const TcState* t, cudaStream_t st, void* dst, const double* src, long n) {
  if (t->tf) to_operand<float>(t, st, dst, src, n);
  else to_operand<__nv_bfloat16>(t, st, dst, src, n);
}

void identity(const TcState* t, cudaStream_t st, void* dst, int m) {
  if (t->tf) identity_operand_kernel<float><<<vgrid((long)m * m), 256, 0, st>>>(static_cast<float*>(dst), m);
  else identity_operand_kernel<__nv_bfloat16><<<vgrid((long)m * m), 256, 0, st>>>(static_cast<__nv_bfloat16*>(dst), m);
}

}  // namespace

static TcState* tc_build(attn_heff* h, bool tf) {
  attn_ctx* ctx = h->ctx;
  auto* t = new TcState();
  t->tf = tf;
  // a stale state of a recycled H_eff hands its device buffers over (they only grow)
  if (auto* old = static_cast<TcState*>(h->tc[tf ? 1 : 0])) {
    for (int k = 0; k < 3; ++k) {
      t->a[k] = std::move(old->a[k]);
      t->b[k] = std::move(old->b[k]);
      t->x[k] = std::move(old->x[k]);
      t->y[k] = std::move(old->y[k]);
    }
    t->err = std::move(old->err);
    t->segs = std::move(old->segs);
    t->seg_start = std::move(old->seg_start);
    t->t0 = std::move(old->t0);
    t->t1 = std::move(old->t1);
    t->t2 = std::move(old->t2);
    t->w = std::move(old->w);
    delete old;
  }
  h->tc[tf ? 1 : 0] = t;
  cudaStream_t st = ctx->stream;
  const int* m = h->m;
  const size_t es = t->es();
  int cta = 0, nk = 0;
  for (int k = 0; k < 3; ++k) {
    const int p = kPairP[k], q = kPairQ[k], sl = kPairS[k];
    const int P = m[p], Q = m[q];
    // internal operators fold in as products with an identity partner:
    // H_0 -> kind 0 (H_0, 1), H_1 -> kind 0 (1, H_1), H_2 -> kind 1 (1, H_2)
    int extra = 0;
    const double* ea[2] = {nullptr, nullptr};
    const double* eb[2] = {nullptr, nullptr};
    if (k == 0) {
      if (h->has_hint[0]) { ea[extra] = h->hint[0].as<double>(); eb[extra] = nullptr; ++extra; }
      if (h->has_hint[1]) { ea[extra] = nullptr; eb[extra] = h->hint[1].as<double>(); ++extra; }
    } else if (k == 1) {
      if (h->has_hint[2]) { ea[extra] = nullptr; eb[extra] = h->hint[2].as<double>(); ++extra; }
    }
    const int R = h->npair[k] + extra;
    t->R[k] = R;
    if (R == 0) continue;
    t->a[k].reserve(es * (size_t)R * P * P);
    t->b[k].reserve(es * (size_t)R * Q * Q);
    uint8_t* A = t->a[k].as<uint8_t>();
    uint8_t* B = t->b[k].as<uint8_t>();
    if (h->npair[k]) {
      convert(t, st, A, h->pa[k].as<double>(), (long)h->npair[k] * P * P);
      convert(t, st, B, h->pb[k].as<double>(), (long)h->npair[k] * Q * Q);
      ctx->launches += 2;
    }
    for (int e = 0; e < extra; ++e) {
      uint8_t* Ae = A + es * (size_t)(h->npair[k] + e) * P * P;
      uint8_t* Be = B + es * (size_t)(h->npair[k] + e) * Q * Q;
      if (ea[e]) convert(t, st, Ae, ea[e], (long)P * P);
      else identity(t, st, Ae, P);
      if (eb[e]) convert(t, st, Be, eb[e], (long)Q * Q);
      else identity(t, st, Be, Q);
      ctx->launches += 2;
    }
    const int S = m[sl];
    t->x[k].reserve(es * (size_t)h->V);
    t->y[k].reserve(sizeof(float) * (size_t)h->V);
    encode_map(&t->maps.x[nk], t->x[k].p, Q, P, S, P, tf);
    encode_map(&t->maps.a[nk], t->a[k].p, P, P, R, 128, tf);
    encode_map(&t->maps.b[nk], t->b[k].p, Q, Q, R, 128, tf);
    KindParams& kp = t->prm.kind[nk];
    kp.P = P; kp.Q = Q; kp.S = S; kp.R = R; kp.cta_begin = cta; kp.Y = t->y[k].as<float>();
    kp.rsplit = 1;
    kp.accumulate = 0;
    cta += (S + 1) / 2;
    ++nk;
  }
  t->prm.nkinds = nk;
  t->grid = cta;
  t->prm.segs = nullptr;
  t->prm.seg_start = nullptr;
  t->tprm.segs = nullptr;
  t->tprm.seg_start = nullptr;
  if (nk > 0) t->build_segments(std::max(ctx->num_sms, 1), st);
  t->err.reserve(sizeof(int));
  ATTN_CHECK_CUDA(cudaMemsetAsync(t->err.p, 0, sizeof(int), st));
  t->prm.err = t->err.as<int>();
  if (h->ntrip > 0) {
    // three-link products: W_r = x x_2 C_r lands in the kind-(0, 1) slice layout
    // [c][a][b] and the per-product kernel adds A_r W_r[c] B_r^T onto Y01
    const int nt = h->ntrip, P = m[0], Q = m[1], S = m[2];
    t->nt = nt;
    t->t0.reserve(es * (size_t)nt * P * P);
    t->t1.reserve(es * (size_t)nt * Q * Q);
    t->t2.reserve(es * (size_t)nt * S * S);
    convert(t, st, t->t0.p, h->tr[0].as<double>(), (long)nt * P * P);
    convert(t, st, t->t1.p, h->tr[1].as<double>(), (long)nt * Q * Q);
    convert(t, st, t->t2.p, h->tr[2].as<double>(), (long)nt * S * S);
    ctx->launches += 3;
    // products per chunk: W of one chunk stays under 1 GiB
    t->tchunk = (int)std::min<long>(nt, std::max<long>(8, (1L << 30) / (long)es / std::max<long>(h->V, 1)));
    t->w.reserve(es * (size_t)t->tchunk * h->V);
    if (!t->R[0]) t->y[0].reserve(sizeof(float) * (size_t)h->V);
    if (!t->R[2]) t->x[2].reserve(es * (size_t)h->V);
    encode_map(&t->tmaps.x[0], t->w.p, Q, P, t->tchunk * S, P, tf);
    encode_map(&t->tmaps.a[0], t->t0.p, P, P, nt, 128, tf);
    encode_map(&t->tmaps.b[0], t->t1.p, Q, Q, nt, 128, tf);
    KindParams& kp = t->tprm.kind[0];
    kp.P = P; kp.Q = Q; kp.S = S; kp.R = 0; kp.rsplit = 1; kp.cta_begin = 0;
    kp.Y = t->y[0].as<float>();
    kp.accumulate = 1;
    t->tprm.nkinds = 1;
    t->tprm.err = t->err.as<int>();
  }
  t->smem = 1024 + 2 * (size_t)kTileBytes + (size_t)kStages * kKBlockBytes + 512;
  static_assert(2 * kTileBytes + kStages * kKBlockBytes == kStagesPP * kKBlockBytes,
                "both kernel modes use the same shared-memory size");
  static_assert(4 * kTileBytes + kStagesTF * kKBlockBytes == kStagesPP * kKBlockBytes,
                "the TF32 kernel uses the same shared-memory size");
  if (tf) {
    ATTN_CHECK_CUDA(cudaFuncSetAttribute(sandwich_tc_kernel<false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)t->smem));
    ATTN_CHECK_CUDA(cudaFuncSetAttribute(sandwich_tc_kernel<true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)t->smem));
  } else {
    ATTN_CHECK_CUDA(cudaFuncSetAttribute(sandwich_tc_kernel<false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)t->smem));
    ATTN_CHECK_CUDA(cudaFuncSetAttribute(sandwich_tc_kernel<true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)t->smem));
  }
  ATTN_CHECK_CUDA(cudaGetLastError());
  return t;
}

// Read and clear the tensor-core error words of an H_eff (0 = ok).
int tc_error(attn_heff* h) {
  int out = 0;
  for (int i = 0; i < 2; ++i) {
    TcState* t = static_cast<TcState*>(h->tc[i]);
    if (!t) continue;
    int e = 0;
    ATTN_CHECK_CUDA(cudaMemcpyAsync(&e, t->err.p, sizeof(int), cudaMemcpyDeviceToHost, h->ctx->stream));
    ATTN_CHECK_CUDA(cudaStreamSynchronize(h->ctx->stream));
    if (e) ATTN_CHECK_CUDA(cudaMemsetAsync(t->err.p, 0, sizeof(int), h->ctx->stream));
    if (!out) out = e;
  }
  return out;
}

void check_device_errors(attn_ctx* ctx, attn_heff* h) {
  const int et = h ? tc_error(h) : 0;
  const int eo = ozaki_error(ctx);
  ATTN_REQUIRE(et == 0 && eo == 0, ATTN_ETIMEOUT,
               "a bounded wait in a tensor-core kernel gave up (code " + std::to_string(et ? et : eo) + ")");
}

}  // namespace attn

using namespace attn;

void attn_heff::apply_tc(const double* x, double* y, bool tf) {
  ATTN_REQUIRE(tc_supported(this), ATTN_EUNSUPPORTED,
               "the tensor-core path needs every link dimension in {16, 32, ..., 128}");
  TcState* t = static_cast<TcState*>(tc[tf ? 1 : 0]);
  if (!t || t->stale) t = tc_build(this, tf);
  cudaStream_t st = ctx->stream;
  // consumer-side wait limit (a short one is how tests make the kernel give up)
  const int wl = ctx->cfg.wait_limit_log2;
  t->prm.wait = t->tprm.wait = (wl > 0) ? (1LL << std::min(wl, 62)) : attn::tc::kWaitCycles;
  // the kind buffers are indexed by pair kind k (0,1,2); kinds with no products pass null
  void* xk[3];
  for (int k = 0; k < 3; ++k) xk[k] = (t->R[k] || (k == 2 && t->nt)) ? t->x[k].p : nullptr;
  if (tf)
    prep_x_kernel<float><<<tile_grid(m), dim3(kTile, 8), 0, st>>>(x, m[0], m[1], m[2], static_cast<float*>(xk[0]),
                                                                   static_cast<float*>(xk[1]), static_cast<float*>(xk[2]));
  else
    prep_x_kernel<__nv_bfloat16><<<tile_grid(m), dim3(kTile, 8), 0, st>>>(
        x, m[0], m[1], m[2], static_cast<__nv_bfloat16*>(xk[0]), static_cast<__nv_bfloat16*>(xk[1]),
        static_cast<__nv_bfloat16*>(xk[2]));
  ctx->launches++;
  auto zero_split_outputs = [&]() {
    for (int k = 0; k < 3; ++k)
      if (t->R[k]) ATTN_CHECK_CUDA(cudaMemsetAsync(t->y[k].p, 0, sizeof(float) * (size_t)V, st));
  };
  const std::array<int, 7> key = {m[0], m[1], m[2], t->R[0], t->R[1], t->R[2], tf ? 1 : 0};
  const int sched = ctx->cfg.tc_schedule;
  if (t->grid > 0 && sched == 2) {
    // persistent form requested
    if (!t->persistent || !t->tuned) t->set_split(0);
    t->tuned = true;
  } else if (t->grid > 0 && sched == 1 && (t->persistent || !t->tuned)) {
    // split grid requested: the smallest split that gives every SM a CTA (no timing)
    int f = 1;
    for (int c : {1, 2, 3, 4, 6, 8}) {
      t->set_split(c);
      f = c;
      if (t->grid >= ctx->num_sms) break;
    }
    t->set_split(f);
    t->tuned = true;
  }
  if (t->grid > 0 && !t->tuned) {
    auto hit = ctx->tc_split_cache.find(key);
    double fl_all = 0.0;
    for (int k = 0; k < 3; ++k) fl_all += (double)t->R[k] * 2.0 * (m[kPairP[k]] + m[kPairQ[k]]) * V;
    if (hit != ctx->tc_split_cache.end()) {
      t->set_split(hit->second);
      t->tuned = true;
    } else if (fl_all < 4e10) {
      // small operator: no timing, the smallest split that gives every SM a CTA
      int f = 1;
      for (int c : {1, 2, 3, 4, 6, 8}) {
        t->set_split(c);
        f = c;
        if (t->grid >= ctx->num_sms) break;
      }
      t->set_split(f);
      t->tuned = true;
      ctx->tc_split_cache[key] = f;
    }
  }
  if (t->grid > 0 && !t->tuned) {
    // Autotuner: time the candidate product splits on this H_eff's real input and
    // keep the fastest (one-off per shape, product counts and operand type, at the
    // first tensor-core application).
    cudaEvent_t e0, e1;
    ATTN_CHECK_CUDA(cudaEventCreate(&e0));
    ATTN_CHECK_CUDA(cudaEventCreate(&e1));
    float best = 1e30f;
    int best_f = 1;
    for (int f : {0, 1, 2, 3, 4, 5, 6, 8, 10, 12}) {
      t->set_split(f);
      if (f > 1 && !t->split_any()) continue;
      float tot = 0.f;
      for (int rep = 0; rep < 3; ++rep) {
        if (t->split_any()) zero_split_outputs();
        ATTN_CHECK_CUDA(cudaEventRecord(e0, st));
        launch_sandwich(false, t, t->grid, t->maps, t->prm, st);
        ATTN_CHECK_CUDA(cudaEventRecord(e1, st));
        ATTN_CHECK_CUDA(cudaEventSynchronize(e1));
        float ms = 0.f;
        ATTN_CHECK_CUDA(cudaEventElapsedTime(&ms, e0, e1));
        if (rep > 0) tot += ms;
        ctx->launches++;
      }
      if (tot < best) {
        best = tot;
        best_f = f;
      }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    t->set_split(best_f);
    t->tuned = true;
    ctx->tc_split_cache[key] = best_f;
  }
  if (t->grid > 0) {
    // algorithmic FLOPs of this launch: the pair products and the internal operators
    double fl = 0.0;
    for (int k = 0; k < 3; ++k) fl += (double)npair[k] * 2.0 * (m[kPairP[k]] + m[kPairQ[k]]) * V;
    for (int s = 0; s < 3; ++s)
      if (has_hint[s]) fl += 2.0 * m[s] * V;
    if (t->split_any()) zero_split_outputs();
    ctx->prof_begin(0);
    launch_sandwich(false, t, t->grid, t->maps, t->prm, st);
    ctx->prof_end(0, fl);
    ctx->launches++;
  }
  if (t->nt > 0) {
    // three-link products, one chunk of products at a time: W = x x_2 C_r on the
    // TN GEMM, then Y01[c] += A_r W_r[c] B_r^T on the per-product kernel
    const int P = m[0], Q = m[1], S = m[2];
    const size_t es = t->es();
    if (!t->R[0]) ATTN_CHECK_CUDA(cudaMemsetAsync(t->y[0].p, 0, sizeof(float) * (size_t)V, st));
    for (int r0 = 0; r0 < t->nt; r0 += t->tchunk) {
      const int Rc = std::min(t->tchunk, t->nt - r0);
      TnOperand A;  // x as [a b][c]: rows P Q, K = S
      A.p = t->x[2].p; A.tf = tf; A.K = S; A.rows = P * Q; A.batches = 1; A.ld = S; A.bstride = 0;
      TnOperand B;  // C_r as [r][c][c']
      B.p = t->t2.as<uint8_t>() + es * (size_t)r0 * S * S; B.tf = tf; B.K = S; B.rows = S; B.batches = Rc;
      B.ld = S; B.bstride = (long)S * S;
      TnParams g;
      g.M = P * Q; g.N = S; g.K = S; g.Bhi = Rc; g.Blo = 1; g.a_bhi = 0; g.b_bhi = 1;
      g.C = t->w.p; g.c_type = tf ? 3 : 1; g.c_rs = 1; g.c_cs = (long)P * Q; g.c_bhi = V;
      tn_gemm(ctx, A, B, g, t->err);
      KindParams& kp = t->tprm.kind[0];
      kp.R = Rc;
      const int pairs = (S + 1) / 2;
      const int f = std::max(1, std::min((ctx->num_sms + pairs - 1) / pairs, Rc / 8));
      kp.rsplit = f;
      const int grid = pairs * f;
      TcMaps mp = t->tmaps;
      encode_map(&mp.a[0], t->t0.as<uint8_t>() + es * (size_t)r0 * P * P, P, P, Rc, 128, tf);
      encode_map(&mp.b[0], t->t1.as<uint8_t>() + es * (size_t)r0 * Q * Q, Q, Q, Rc, 128, tf);
      ctx->prof_begin(0);
      launch_sandwich(true, t, grid, mp, t->tprm, st);
      ctx->prof_end(0, (double)Rc * 2.0 * (P + Q) * V);
      ctx->launches++;
    }
  }
  combine_kernel<<<tile_grid(m), dim3(kTile, 8), 0, st>>>(y, m[0], m[1], m[2],
                                           (t->R[0] || t->nt) ? t->y[0].as<float>() : nullptr,
                                           t->R[1] ? t->y[1].as<float>() : nullptr,
                                           t->R[2] ? t->y[2].as<float>() : nullptr);
  ctx->launches++;
  ATTN_CHECK_CUDA(cudaGetLastError());
}

void attn_heff::apply_bf16(const double* x, double* y) { apply_tc(x, y, false); }
void attn_heff::apply_tf32(const double* x, double* y) { apply_tc(x, y, true); }
