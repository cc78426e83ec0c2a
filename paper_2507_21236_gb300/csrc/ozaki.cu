// FP64-accurate GEMM on the BF16 tensor cores by operand splitting (the Ozaki
// scheme: K. Ozaki, T. Ogita, S. Oishi, S. M. Rump, "Error-free transformations
// of matrix multiplication by using fast routines of matrix multiplication and
// its applications", Numer. Algorithms 59 (2012)).
//
// GB300 executes FP64 FMAs at about 1.2 TFLOP/s, three orders of magnitude
// below its BF16 tensor rate, so the FP64 contractions of the method (the
// renormalisation T^T (O (x) O) T of Fig. eff-op and the FP64 H_eff
// applications of the residual corrections) can run faster as many exact BF16
// products than as FP64 FMAs. For C = P Q^T (P: M x K, Q: N x K, FP64):
//
//  * every row of P (and of Q) is scaled by a power of two 2^-E so that its
//    entries lie in (-1, 1), then written as six BF16 integers,
//        p = 2^E sum_{s=1..6} n_s 2^(1-8s),  |n_s| <= 128,
//    i.e. 7 + 5 x 8 = 47 significant bits (relative residual <= 2^-48);
//  * the slice pairs (s, t) with s + t <= 7 (21 of 36; the rest lie below
//    2^-46 of the row scales) are multiplied on the tensor cores. Pairs on
//    one diagonal c = s + t share the scale 2^(2-8c) and accumulate into one
//    TMEM accumulator. Every product is an integer of magnitude at most 2^14;
//  * diagonal d (0-based, d = s + t - 2) sums d + 1 slice pairs, so over F K
//    blocks of 64 its partial sums stay below (d + 1) 2^14 64 F, exact in FP32
//    while (d + 1) F <= 16. Diagonals 0-3 accumulate over windows of 4 K blocks,
//    diagonals 4 and 5 over windows of 2. At the end of each window the epilogue
//    folds the diagonals into an int64 fixed-point sum per output element (unit
//    2^-46 of the row scales; the finest diagonal is rounded to that unit), and
//    the sum is converted to FP64 once.
//
// The error is normwise: |C - C~|_ij <= about (K + 2) 2^-46 2^(E_i + E_j),
// with 2^E_i and 2^E_j at most twice the largest |entry| of row i of P and of
// row j of Q. K per launch is limited to 65536 so the int64 sum cannot overflow.
//
// Kernel: persistent, one CTA per SM walking the 128 x 64 output tiles of every
// batch entry (tile t = blockIdx.x + i gridDim.x, column tiles fastest so that CTAs
// running at the same time share the P tile in L2); barriers and tensor memory are
// set up once, and the copies and MMAs of the next tile overlap the epilogue of the
// current one. Warp 0 is the TMA producer, warps 1 and 2 issue the MMAs, warps
// 3-18 read the accumulators (four warps per 32-lane quarter w % 4, 16 columns
// each).
//
// Wide MMAs. A thread can issue a tcgen05.mma only about every 70-110 cycles
// whatever its N, while an M = 128, K = 16 MMA runs N / 2 cycles, so pair-by-pair
// N = 64 products would leave the tensor pipe idle more than half of the time. The
// six Q slices of a K block sit one after another in shared memory and the six
// diagonal accumulators one after another in tensor memory, so one MMA of width
// 64 n multiplies P slice s with Q slices t .. t + n - 1 into diagonals s + t ..
// s + t + n - 1 at once: warp 1 covers diagonals 0-3 with one MMA per P slice
// s <= 3 (N = 256 - 64 s), warp 2 diagonals 4-5 with one per P slice (N = 128,
// and 64 for s = 5): 10 MMAs per K step instead of 21. Each issuer owns its
// diagonals, so the MMA that restarts a window precedes every other write to them.
// Diagonals 4-5 have two accumulator buffers (6 x 64 + 2 x 64 = 512 columns) and
// alternate between them from window to window, so the epilogue reads one while
// the MMAs fill the other; diagonals 0-3 are handed back as soon as they are read.
// The six Q slices of a K block (48 KB) are double-buffered; the P slices stream
// through a ring of eight 16 KB stages. All waits are bounded; on a timeout the CTA
// records an error code, stops issuing, drains its copies and frees TMEM.
#include <algorithm>
#include <cmath>

#include "ozaki.h"
#include "tc_ptx.h"

namespace attn {

namespace {

using namespace tc;

constexpr int kSlices = 6;
constexpr int kDiags = 6;               // c = s + t = 2 .. 7
constexpr int kOzThreads = 608;         // 3 role warps + 16 epilogue warps
constexpr int kQRows = 64;              // output tile columns (rows of Q)
constexpr int kPBytes = 128 * 128;      // one 128-row x 64-wide BF16 K block of one P slice
constexpr int kQBytes = kQRows * 128;   // one 64-row K block of one Q slice
constexpr int kPStages = 8;
constexpr int kQBufBytes = kSlices * kQBytes;
constexpr int kEmptyRow = -2000;        // exponent of an all-zero row
constexpr int kUnitExp = 46;            // fixed-point unit 2^-46 of the row scales
// K blocks per accumulation window: diagonals 0-3 (one TMEM buffer, columns 64 d)
// and diagonals 4-5 (two buffers, columns 256 + 128 b + 64 (d - 4))
constexpr int kFoldA = 4, kFoldB = 2;

struct OzParams {
  int M, N, nkb;           // rows of P, rows of Q, 64-wide K blocks
  int nrtP, nrtQ;          // row tiles (of 128 and 64 rows) per operand batch entry
  int Bhi, Blo;            // batch entries b = bhi * Blo + blo
  int p_hi, p_lo, q_hi, q_lo;  // sliced-operand batch index = bhi * x_hi + blo * x_lo
  const int* EP;           // [batches of P][M] row exponents
  const int* EQ;           // [batches of Q][N]
  double* C;
  long c_rs, c_cs, c_bhi, c_blo;
  double alpha_rest, beta;  // alpha = alpha_rest 2^alpha_exp (alpha_rest = 1 for a power of two)
  int alpha_exp;
  long tiles;              // column tiles x row tiles x batch entries
  int* err;
};

// Slices are stored tiled: per operand batch entry, row tile, 64-wide K block and slice
// one contiguous [tile rows][64] BF16 block, so that every TMA box is one contiguous
// 16 KB (P) or 8 KB (Q) read rather than 128 or 64 strided 128-byte segments.
struct OzMaps {
  CUtensorMap p, q;  // [((batch * nrt + tile) * nkb + kb) * 6 + s][tile rows][64], boxes {64, 128 / 64, 1}
};

// a 2^e as a double for an int64 a, rounded to nearest even like ldexp((double)a, e),
// from integer instructions alone (this GPU issues about two FP64 operations per SM
// and cycle, which made the FP64 conversion the epilogue's bottleneck); the rare
// results outside the normal range take the FP64 route.
__device__ __forceinline__ double scaled_i64(long long a, int e) {
  if (a == 0) return 0.0;
  const unsigned long long sign = a < 0 ? 0x8000000000000000ull : 0ull;
  const unsigned long long u = a < 0 ? 0ull - (unsigned long long)a : (unsigned long long)a;
  int top = 63 - __clzll(u);  // u in [2^top, 2^(top + 1))
  unsigned long long m;
  if (top > 52) {
    const int sh = top - 52;
    const unsigned long long rem = u & ((1ull << sh) - 1ull), half = 1ull << (sh - 1);
    m = u >> sh;
    if (rem > half || (rem == half && (m & 1ull))) {
      if (++m == (1ull << 53)) {
        m >>= 1;
        ++top;
      }
    }
  } else {
    m = u << (52 - top);
  }
  const int be = top + e + 1023;
  if (be < 1 || be > 2046) return ldexp((double)a, e);
  return __longlong_as_double((long long)(sign | ((unsigned long long)be << 52) | (m & 0xFFFFFFFFFFFFFull)));
}

__device__ __forceinline__ bool window_end(int fold, int kb, int nkb) {
  return (kb + 1) % fold == 0 || kb == nkb - 1;
}

__global__ void __launch_bounds__(kOzThreads, 1) ozaki_gemm_kernel(const __grid_constant__ OzMaps maps, OzParams p) {
  extern __shared__ uint8_t smem_raw[];
  const uint32_t raw = smem_u32(smem_raw);
  const uint32_t base = (raw + 1023u) & ~1023u;
  uint8_t* gbase = smem_raw + (base - raw);
  const uint32_t sQ = base;                     // two buffers of six Q slices
  const uint32_t sP = base + 2 * kQBufBytes;    // ring of P slice K blocks
  const uint32_t sBar = sP + kPStages * kPBytes;
  enum {
    QFULL = 0,
    QEMPTY = 2,                 // both issuers release a Q buffer
    PFULL = 4,
    PEMPTY = 4 + kPStages,      // both issuers release a P stage
    AFULL = 4 + 2 * kPStages,   // a window of diagonals 0-3 is complete in TMEM
    AEMPTY = AFULL + 1,         // the epilogue has read it
    BFULL = AEMPTY + 1,         // [b]: a window of diagonals 4-5 is complete in buffer b
    BEMPTY = BFULL + 2,         // [b]: the epilogue has read buffer b
    MDONE = BEMPTY + 2,         // [issuer]: every MMA of that issuer has completed
    NBAR = MDONE + 2
  };
  uint64_t* bars = reinterpret_cast<uint64_t*>(gbase + (sBar - base));
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + NBAR);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
  auto bar = [&](int i) { return sBar + 8u * (uint32_t)i; };
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nkb = p.nkb;
  const int ntn = (p.N + kQRows - 1) / kQRows, ntm = (p.M + 127) / 128;
  // tile t: column tile, row tile, batch entry (bhi, blo) and the operands' batch indices
  struct Tile {
    int nt, mt, bhi, blo, bp, bq;
  };
  auto tile = [&](long t) {
    Tile r;
    r.nt = (int)(t % ntn);
    const long rest = t / ntn;
    r.mt = (int)(rest % ntm);
    const long b = rest / ntm;
    r.bhi = (int)(b / p.Blo);
    r.blo = (int)(b % p.Blo);
    r.bp = r.bhi * p.p_hi + r.blo * p.p_lo;
    r.bq = r.bhi * p.q_hi + r.blo * p.q_lo;
    return r;
  };

  if (threadIdx.x == 0) {
    for (int i = 0; i < 2; ++i) {
      mbar_init(bar(QFULL + i), 1);
      mbar_init(bar(QEMPTY + i), 2);
      mbar_init(bar(MDONE + i), 1);
    }
    for (int i = 0; i < kPStages; ++i) {
      mbar_init(bar(PFULL + i), 1);
      mbar_init(bar(PEMPTY + i), 2);
    }
    mbar_init(bar(AFULL), 1);
    mbar_init(bar(AEMPTY), 16);
    for (int i = 0; i < 2; ++i) {
      mbar_init(bar(BFULL + i), 1);
      mbar_init(bar(BEMPTY + i), 16);
    }
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(512));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = *tmem_slot;  // diagonals 0-3 at columns 64 d, 4-5 at 256 + 128 b + 64 (d - 4)

  if (warp == 0 && lane == 0) {
    // ---- producer: per K block the six Q slices, then the six P slices; g counts the
    // K blocks of all tiles of this CTA
    int pst = 0, pissued = 0;
    uint32_t pph = 0;
    int qissued = 0, g = 0;
    bool ok = true;
    for (long t = blockIdx.x; ok && t < p.tiles; t += gridDim.x) {
      const Tile tl = tile(t);
      const int zP = (tl.bp * p.nrtP + tl.mt) * nkb * kSlices;
      const int zQ = (tl.bq * p.nrtQ + tl.nt) * nkb * kSlices;
      for (int kb = 0; ok && kb < nkb; ++kb, ++g) {
        const int qb = g & 1;
        if (g >= 2 && !mbar_wait(bar(QEMPTY + qb), ((g >> 1) - 1) & 1, p.err, 61, abort_flag)) {
          ok = false;
          break;
        }
        mbar_expect_tx(bar(QFULL + qb), (uint32_t)kQBufBytes);
        for (int s = 0; s < kSlices; ++s)
          tma_load_3d(sQ + qb * kQBufBytes + s * kQBytes, &maps.q, 0, 0, zQ + kb * kSlices + s, bar(QFULL + qb));
        qissued = g + 1;
        for (int s = 0; s < kSlices; ++s) {
          if (pissued >= kPStages && !mbar_wait(bar(PEMPTY + pst), pph ^ 1u, p.err, 62, abort_flag)) {
            ok = false;
            break;
          }
          mbar_expect_tx(bar(PFULL + pst), (uint32_t)kPBytes);
          tma_load_3d(sP + pst * kPBytes, &maps.p, 0, 0, zP + kb * kSlices + s, bar(PFULL + pst));
          ++pissued;
          if (++pst == kPStages) { pst = 0; pph ^= 1u; }
        }
      }
    }
    // drain: every issued copy must land before the CTA exits
    for (int q = (qissued > 2 ? qissued - 2 : 0); q < qissued; ++q) {
      long long t0 = clock64();
      while (!mbar_try_wait(bar(QFULL + (q & 1)), (q >> 1) & 1) && clock64() - t0 < kWaitCycles) {}
    }
    for (int q = (pissued > kPStages ? pissued - kPStages : 0); q < pissued; ++q) {
      long long t0 = clock64();
      while (!mbar_try_wait(bar(PFULL + q % kPStages), (q / kPStages) & 1) && clock64() - t0 < kWaitCycles) {}
    }
  } else if ((warp == 1 || warp == 2) && lane == 0) {
    // ---- MMA issue, one thread per diagonal set: diagonal d accumulates the pairs
    // (s, t) with s + t = d (0-based slices) over a window of kFold[d] K blocks
    const int me = warp - 1;
    const uint64_t dP0 = sw128_desc(sP), dQ0 = sw128_desc(sQ);
    const int fold = me == 0 ? kFoldA : kFoldB;
    int pst = 0, g = 0;
    uint32_t pph = 0;
    int win = 0;  // windows of this issuer's diagonals begun so far (all tiles)
    bool ok = true;
    for (long tt = blockIdx.x; ok && tt < p.tiles; tt += gridDim.x) {
      for (int kb = 0; ok && kb < nkb; ++kb, ++g) {
        const int qb = g & 1;
        if (!mbar_wait(bar(QFULL + qb), (g >> 1) & 1, p.err, 64, abort_flag)) {
          ok = false;
          break;
        }
        fence_after();
        const bool first = kb % fold == 0;
        // a window refills its accumulator once the epilogue has read what the last
        // window left there: window win - 1 (diagonals 0-3) or win - 2 (4-5, two buffers)
        if (first && me == 0 && win > 0 && !mbar_wait(bar(AEMPTY), (win - 1) & 1, p.err, 63, abort_flag)) {
          ok = false;
          break;
        }
        if (first && me == 1 && win > 1 &&
            !mbar_wait(bar(BEMPTY + (win & 1)), ((win >> 1) - 1) & 1, p.err, 63, abort_flag)) {
          ok = false;
          break;
        }
        fence_after();
        const uint32_t accB = tmem + 256u + 128u * (uint32_t)(win & 1);
        for (int s = 0; s < kSlices; ++s) {
          if (!mbar_wait(bar(PFULL + pst), pph, p.err, 65, abort_flag)) { ok = false; break; }
          fence_after();
          const uint64_t dP = dP0 + (uint64_t)(pst * (kPBytes >> 4));
          const uint32_t restart = (first && s == 0) ? 0u : 1u;
          if (me == 0) {
            // diagonals s .. 3 from Q slices 0 .. 3 - s
            if (s < 4)
              mma4_ss(tmem + 64u * (uint32_t)s, dP, dQ0 + (uint64_t)((qb * kQBufBytes) >> 4),
                      idesc_bf16(128, 64 * (4 - s)), restart);
          } else {
            // diagonals 4-5 from Q slices 4 - s, 5 - s (s <= 4); diagonal 5 from Q slice 0 (s = 5)
            const int t0 = s < 5 ? 4 - s : 0;
            mma4_ss(s < 5 ? accB : accB + 64u, dP, dQ0 + (uint64_t)((qb * kQBufBytes + t0 * kQBytes) >> 4),
                    idesc_bf16(128, s < 5 ? 128 : 64), restart);
          }
          mma_commit(bar(PEMPTY + pst));
          if (++pst == kPStages) { pst = 0; pph ^= 1u; }
        }
        mma_commit(bar(QEMPTY + qb));
        if (!ok) break;
        if (window_end(fold, kb, nkb)) {
          mma_commit(bar(me == 0 ? AFULL : BFULL + (win & 1)));
          ++win;
        }
      }
    }
    mma_commit(bar(MDONE + me));
    long long t0 = clock64();
    while (!mbar_try_wait(bar(MDONE + me), 0) && clock64() - t0 < kWaitCycles) {}
  } else if (warp >= 3) {
    // ---- epilogue: lane quarter q4, columns 16 h .. 16 h + 15 of the tile; every
    // finished window of a diagonal is folded into an int64 fixed-point sum
    const int q4 = warp & 3, h = (warp - 3) >> 2;
    const uint32_t lane_off = (uint32_t)(q4 * 32) << 16;
    int winA = 0, winB = 0;  // windows read so far (all tiles)
    bool ok = true;
    for (long tt = blockIdx.x; ok && tt < p.tiles; tt += gridDim.x) {
      long long acc[16];
#pragma unroll
      for (int c = 0; c < 16; ++c) acc[c] = 0;
      for (int kb = 0; ok && kb < nkb; ++kb) {
        if (window_end(kFoldA, kb, nkb)) {
          // warp-uniform: the TMEM loads below are .sync.aligned
          if (!__all_sync(0xffffffffu, mbar_wait(bar(AFULL), winA & 1, p.err, 66, abort_flag))) {
            ok = false;
            break;
          }
          ++winA;
          fence_after();
#pragma unroll
          for (int d = 0; d < 4; ++d) {
            float v[16];
            tmem_ld16(tmem + lane_off + 64u * (uint32_t)d + 16u * (uint32_t)h, v);
            if (d == 3) {
              fence_before();
              __syncwarp();
              if (lane == 0) mbar_arrive(bar(AEMPTY));
            }
#pragma unroll
            for (int c = 0; c < 16; ++c)  // exact: |v| <= 2^24
              acc[c] += (long long)__float2int_rn(v[c]) << (8 * (kDiags - 2 - d));
          }
        }
        if (window_end(kFoldB, kb, nkb)) {
          const int b = winB & 1;
          if (!__all_sync(0xffffffffu, mbar_wait(bar(BFULL + b), (winB >> 1) & 1, p.err, 67, abort_flag))) {
            ok = false;
            break;
          }
          ++winB;
          fence_after();
#pragma unroll
          for (int e = 0; e < 2; ++e) {
            float v[16];
            tmem_ld16(tmem + lane_off + 256u + 128u * (uint32_t)b + 64u * (uint32_t)e + 16u * (uint32_t)h, v);
            if (e == 1) {
              fence_before();
              __syncwarp();
              if (lane == 0) mbar_arrive(bar(BEMPTY + b));
            }
#pragma unroll
            for (int c = 0; c < 16; ++c) {
              const long long x = (long long)__float2int_rn(v[c]);
              acc[c] += e == 0 ? x : (x + 128) >> 8;  // diagonal 4 is the unit; 5, the finest, rounded to it
            }
          }
        }
      }
      const Tile tl = tile(tt);
      const int i = tl.mt * 128 + q4 * 32 + lane;
      if (ok && i < p.M) {
        const int ep = p.EP[(long)tl.bp * p.M + i];
        const long cbase = (long)tl.bhi * p.c_bhi + (long)tl.blo * p.c_blo + (long)i * p.c_rs;
#pragma unroll
        for (int c = 0; c < 16; ++c) {
          const int j = tl.nt * kQRows + 16 * h + c;
          if (j < p.N) {
            const int e = ep + p.EQ[(long)tl.bq * p.N + j] - kUnitExp + p.alpha_exp;
            double v = scaled_i64(acc[c], e);
            if (p.alpha_rest != 1.0) v *= p.alpha_rest;
            double* cp = p.C + cbase + (long)j * p.c_cs;
            if (p.beta == 0.0) *cp = v;
            else if (p.beta == 1.0) *cp += v;
            else *cp = fma(p.beta, *cp, v);
          }
        }
      }
    }
  }
  fence_before();
  __syncthreads();
  if (warp == 1) {
    fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512));
  }
}

// ------------------------------------------------------------ slicing kernels
// Operand element (batch bh, bl; row r; k' = g K + k) of a strided FP64 view.
__device__ __forceinline__ long oz_offset(const OzView& v, int bh, int bl, long r, long kk) {
  const long g = kk / v.K, k = kk - g * v.K;
  return (long)bh * v.sBhi + (long)bl * v.sBlo + r * v.sR + g * v.sG + k * v.sK;
}

constexpr int kT = 32;  // 32 rows x 32 k per tile, 32 x 8 threads

__global__ void fill_int_kernel(int* p, long n, int v) {
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) p[i] = v;
}

// Binary exponent e of a finite nonzero double (|x| = f 2^e, f in [0.5, 1)) from its
// bits: integer instructions only (the FP64 pipe is the scarce unit on this GPU).
__device__ __forceinline__ int exp_bits(long long b) {
  const int ef = (int)((b >> 52) & 0x7FF);
  if (ef) return ef - 1022;
  const unsigned long long m = (unsigned long long)b & 0xFFFFFFFFFFFFFull;  // subnormal
  return -1022 - (__clzll(m) - 12);
}

// E[batch][row] = max over k' of the binary exponent of |entry| (|entry| < 2^E).
// Lanes walk k when k is the unit stride (each warp then owns four rows of the
// tile), rows otherwise; every shuffle runs on the whole warp.
__global__ void oz_exponent_kernel(OzView v, int* E) {
  __shared__ int sh[8][kT + 1];
  const int tx = threadIdx.x, ty = threadIdx.y;
  const long r0 = (long)blockIdx.y * kT;
  const int batch = blockIdx.z, bh = batch / v.nblo, bl = batch % v.nblo;
  const long Kt = (long)v.K * v.G;
  const bool kfast = (v.sK == 1 && v.sR != 1);
  int em[kT / 8];
#pragma unroll
  for (int j = 0; j < kT / 8; ++j) em[j] = kEmptyRow;
  for (long k0 = (long)blockIdx.x * kT; k0 < Kt; k0 += (long)gridDim.x * kT) {
#pragma unroll
    for (int j = 0; j < kT / 8; ++j) {
      const int i = ty + 8 * j;
      const long r = kfast ? r0 + i : r0 + tx, k = kfast ? k0 + tx : k0 + i;
      if (r < v.rows && k < Kt) {
        const long long b = __double_as_longlong(v.p[oz_offset(v, bh, bl, r, k)]);
        if (b & 0x7FFFFFFFFFFFFFFFll) em[j] = max(em[j], exp_bits(b));
      }
    }
  }
  if (kfast) {
#pragma unroll
    for (int j = 0; j < kT / 8; ++j) {
      int m = em[j];
      for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
      const long r = r0 + ty + 8 * j;
      if (tx == 0 && r < v.rows && m > kEmptyRow) atomicMax(&E[(long)batch * v.rows + r], m);
    }
    return;
  }
  int m = em[0];
#pragma unroll
  for (int j = 1; j < kT / 8; ++j) m = max(m, em[j]);
  sh[ty][tx] = m;
  __syncthreads();
  if (ty == 0) {
    for (int i = 1; i < 8; ++i) m = max(m, sh[i][tx]);
    const long r = r0 + tx;
    if (r < v.rows && m > kEmptyRow) atomicMax(&E[(long)batch * v.rows + r], m);
  }
}

// The same for views whose rows are contiguous (row stride 1): one thread per row,
// 256 consecutive rows per block, so every K index reads 2 KB of consecutive memory
// (the tiled kernel above reads 256 bytes per K index there, which wastes DRAM pages
// when K is strided). Blocks split K into chunks; loads are unrolled four deep.
constexpr int kER = 256;
__global__ void __launch_bounds__(kER) oz_exponent_rows_kernel(OzView v, int* E, long kchunk) {
  const long r = (long)blockIdx.y * kER + threadIdx.x;
  const int batch = blockIdx.z, bh = batch / v.nblo, bl = batch % v.nblo;
  const long Kt = (long)v.K * v.G;
  const long k0 = (long)blockIdx.x * kchunk, k1 = k0 + kchunk < Kt ? k0 + kchunk : Kt;
  if (r >= v.rows) return;
  int em = kEmptyRow;
  long k = k0;
  for (; k + 4 <= k1; k += 4) {
    long long b[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) b[u] = __double_as_longlong(v.p[oz_offset(v, bh, bl, r, k + u)]);
#pragma unroll
    for (int u = 0; u < 4; ++u)
      if (b[u] & 0x7FFFFFFFFFFFFFFFll) em = max(em, exp_bits(b[u]));
  }
  for (; k < k1; ++k) {
    const long long b = __double_as_longlong(v.p[oz_offset(v, bh, bl, r, k)]);
    if (b & 0x7FFFFFFFFFFFFFFFll) em = max(em, exp_bits(b));
  }
  if (em > kEmptyRow) atomicMax(&E[(long)batch * v.rows + r], em);
}

// Slice s of 2^-E[row] entry, written tiled: element (batch, row, k) of slice s at
// ((((batch nrt + row / TR) nkb + k / 64) 6 + s) TR + row % TR) 64 + k % 64, zero for
// k >= K G and for the padding rows of the last tile. The entry becomes the integer
// F = round(|x| 2^(47-E)) (|F| < 2^47, from the bits of x, rounding half up), signed,
// then balanced base-256 digits from the bottom: n_6 .. n_2 in [-128, 127], n_1 = the
// rest (|n_1| <= 128), F = sum_s n_s 2^(8(6-s)).
// One block per 64 x 64 tile (64 rows, one 64-wide K block), 64 x 4 threads: the
// operand is read along its unit-stride direction (512 bytes per warp pair) and every
// output row of every slice is written as one full 128-byte line.
constexpr int kST = 64;
__global__ void __launch_bounds__(256) oz_slice_kernel(OzView v, const int* E, __nv_bfloat16* S, long Kpad, int TR,
                                                       int nrt) {
  __shared__ long long t[kST][kST + 1];  // [row][k]
  const int tx = threadIdx.x, ty = threadIdx.y;
  const bool kfast = (v.sK == 1 && v.sR != 1);
  // blockIdx.x walks the operand's unit-stride direction, so that neighbouring blocks
  // read neighbouring memory
  const long r0 = (long)(kfast ? blockIdx.y : blockIdx.x) * kST, k0 = (long)(kfast ? blockIdx.x : blockIdx.y) * kST;
  const int batch = blockIdx.z, bh = batch / v.nblo, bl = batch % v.nblo;
  const long Kt = (long)v.K * v.G;
  const long nkb = Kpad / 64;
#pragma unroll 4
  for (int j = 0; j < kST / 4; ++j) {
    const int i = ty + 4 * j;
    const long r = kfast ? r0 + i : r0 + tx, k = kfast ? k0 + tx : k0 + i;
    long long b = 0;
    if (r < v.rows && k < Kt) b = __double_as_longlong(v.p[oz_offset(v, bh, bl, r, k)]);
    if (kfast) t[i][tx] = b;
    else t[tx][i] = b;
  }
  __syncthreads();
  // each thread: one row and 8 consecutive k, every slice written as one 16-byte store
  // (8 threads fill the 128-byte row of a slice block)
  const int lin = ty * kST + tx;
  const long sstride = (long)TR * 64;
#pragma unroll 1
  for (int rep = 0; rep < 2; ++rep) {
    const int idx = lin + 256 * rep, i = idx >> 3, kq = (idx & 7) * 8;
    const long r = r0 + i, k = k0 + kq;
    if (r >= (long)nrt * TR || k >= Kpad) continue;
    const int e = r < v.rows ? E[(long)batch * v.rows + r] : kEmptyRow;
    uint32_t w[kSlices][4];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const long long b = t[i][kq + u];
      long long F = 0;
      if ((b & 0x7FFFFFFFFFFFFFFFll) && e != kEmptyRow) {
        const int ef = (int)((b >> 52) & 0x7FF);
        const long long mant = (b & 0xFFFFFFFFFFFFFll) | (ef ? (1ll << 52) : 0ll);
        const int sh = (ef ? ef - 1075 : -1074) + 47 - e;  // |x| = mant 2^(ef - 1075)
        if (sh >= 0) F = mant << sh;                       // < 2^47 since |x| < 2^e
        else if (sh > -64) F = (sh == -63 ? 0ll : (mant + (1ll << (-sh - 1))) >> (-sh));
        if (b < 0) F = -F;
      }
      // Balanced base-256 digits: the bytes of G = F + 128 (1 + 2^8 + ... + 2^32) minus
      // 128 are the digits n_6 .. n_2 in [-128, 127], and G >> 40 is n_1 (|n_1| <= 128),
      // the same digits as peeling F from the bottom. A digit g - 128 becomes a float
      // exactly as (2^23 + g) - (2^23 + 128), and a BF16 as the float's upper half.
      const long long G = F + 0x8080808080ll;
      const uint32_t lo = (uint32_t)G, hi = (uint32_t)(G >> 32);
      const uint32_t g[kSlices] = {(uint32_t)(((int)hi >> 8) + 128), hi & 255u, lo >> 24, (lo >> 16) & 255u,
                                   (lo >> 8) & 255u, lo & 255u};
#pragma unroll
      for (int sl = 0; sl < kSlices; ++sl) {
        const uint32_t f = __float_as_uint(__uint_as_float(0x4B000000u + g[sl]) - 8388736.0f);
        if (u & 1) w[sl][u >> 1] = __byte_perm(w[sl][u >> 1], f, 0x7610);
        else w[sl][u >> 1] = f >> 16;
      }
    }
    uint4* out = reinterpret_cast<uint4*>(
        S + ((((long)batch * nrt + r / TR) * nkb + (k >> 6)) * kSlices * TR + r % TR) * 64 + (k & 63));
#pragma unroll
    for (int sl = 0; sl < kSlices; ++sl)
      out[(long)sl * sstride / 8] = make_uint4(w[sl][0], w[sl][1], w[sl][2], w[sl][3]);
  }
}

// Map over tiled slices: [nz][tile rows][64] BF16 with a {64, tile rows, 1} box.
void encode_slices(CUtensorMap* map, const __nv_bfloat16* p, int tile_rows, long nz) {
  cuuint64_t dims[3] = {64, (cuuint64_t)tile_rows, (cuuint64_t)nz};
  cuuint64_t strides[2] = {128, (cuuint64_t)tile_rows * 128};
  cuuint32_t box[3] = {64, (cuuint32_t)tile_rows, 1};
  cuuint32_t estr[3] = {1, 1, 1};
  CUresult r = tensor_map_encoder()(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<__nv_bfloat16*>(p), dims,
                                    strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                                    CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  ATTN_REQUIRE(r == CUDA_SUCCESS, ATTN_ECUDA, "cuTensorMapEncodeTiled failed for Ozaki slices");
}


}  // namespace

void ozaki_slice(attn_ctx* ctx, const OzView& v, long Kpad, int tile_rows, DevBuf& slices, DevBuf& exps) {
  const long nb = (long)v.nbhi * v.nblo;
  ATTN_REQUIRE(nb <= 65535, ATTN_EUNSUPPORTED, "too many operand batches for the split GEMM");
  const int nrt = (v.rows + tile_rows - 1) / tile_rows;
  const long padded = (long)nrt * tile_rows;
  ATTN_REQUIRE(nb * nrt * (Kpad / 64) * kSlices < (1L << 31), ATTN_EUNSUPPORTED, "operand too large for the split GEMM");
  slices.reserve(sizeof(__nv_bfloat16) * (size_t)(nb * kSlices * padded * Kpad));
  exps.reserve(sizeof(int) * (size_t)(nb * v.rows));
  cudaStream_t st = ctx->stream;
  const long ne = nb * v.rows;
  fill_int_kernel<<<(int)std::min<long>((ne + 255) / 256, 4096), 256, 0, st>>>(exps.as<int>(), ne, kEmptyRow);
  const long Kt = (long)v.K * v.G;
  const long rt = (v.rows + kT - 1) / kT;
  ATTN_REQUIRE(rt <= 65535, ATTN_EUNSUPPORTED, "too many rows for the split GEMM");
  dim3 blk(kT, 8);
  if (v.sR == 1) {
    // rows contiguous: one thread per row, K split into chunks for about 2048 blocks
    const long rb = (v.rows + kER - 1) / kER;
    const long nchunk = std::max<long>(1, std::min<long>((Kt + 63) / 64, 2048 / std::max<long>(rb * nb, 1)));
    const long kchunk = (Kt + nchunk - 1) / nchunk;
    dim3 ge((unsigned)((Kt + kchunk - 1) / kchunk), (unsigned)rb, (unsigned)nb);
    oz_exponent_rows_kernel<<<ge, kER, 0, st>>>(v, exps.as<int>(), kchunk);
  } else {
    // exponent pass: k tiles folded so that the grid stays modest
    const long kt = (Kt + kT - 1) / kT;
    dim3 ge((unsigned)std::min<long>(kt, std::max<long>(1, 8192 / std::max<long>(rt * nb, 1))), (unsigned)rt,
            (unsigned)nb);
    oz_exponent_kernel<<<ge, blk, 0, st>>>(v, exps.as<int>());
  }
  const bool kfast = (v.sK == 1 && v.sR != 1);
  const unsigned nkt = (unsigned)(Kpad / kST), nrb = (unsigned)((padded + kST - 1) / kST);
  dim3 gs(kfast ? nkt : nrb, kfast ? nrb : nkt, (unsigned)nb);
  ATTN_REQUIRE(gs.y <= 65535, ATTN_EUNSUPPORTED, "operand too large for the split GEMM");
  oz_slice_kernel<<<gs, dim3(kST, 4), 0, st>>>(v, exps.as<int>(), slices.as<__nv_bfloat16>(), Kpad, tile_rows, nrt);
  ctx->launches += 3;
  ATTN_CHECK_CUDA(cudaGetLastError());
}

// C = alpha sum_g A_g B_g + beta C of a GemmF64 through the split BF16 products.
void gemm_f64_ozaki(attn_ctx* ctx, const GemmF64& g0) {
  if (g0.M <= 0 || g0.N <= 0 || g0.Bhi <= 0 || g0.Blo <= 0) return;
  // orientation: TMEM lanes are output rows, so the side whose C stride is 1 goes on
  // the 128-row side (coalesced stores) unless it is much shorter than the other
  bool swap = g0.N > g0.M;
  if (std::min(g0.M, g0.N) >= 64) {
    if (g0.cN == 1 && g0.cM != 1) swap = true;
    else if (g0.cM == 1 && g0.cN != 1) swap = false;
  }
  OzView P, Q;
  int M, N;
  long c_rs, c_cs;
  if (!swap) {
    M = g0.M; N = g0.N;
    P.p = g0.A; P.sR = g0.aM; P.sK = g0.aK; P.sG = g0.aG; P.sBhi = g0.aBhi; P.sBlo = g0.aBlo;
    Q.p = g0.B; Q.sR = g0.bN; Q.sK = g0.bK; Q.sG = g0.bG; Q.sBhi = g0.bBhi; Q.sBlo = g0.bBlo;
    c_rs = g0.cM; c_cs = g0.cN;
  } else {
    M = g0.N; N = g0.M;
    P.p = g0.B; P.sR = g0.bN; P.sK = g0.bK; P.sG = g0.bG; P.sBhi = g0.bBhi; P.sBlo = g0.bBlo;
    Q.p = g0.A; Q.sR = g0.aM; Q.sK = g0.aK; Q.sG = g0.aG; Q.sBhi = g0.aBhi; Q.sBlo = g0.aBlo;
    c_rs = g0.cN; c_cs = g0.cM;
  }
  P.rows = M; Q.rows = N;
  P.K = Q.K = g0.K;
  P.nbhi = P.sBhi ? g0.Bhi : 1; P.nblo = P.sBlo ? g0.Blo : 1;
  Q.nbhi = Q.sBhi ? g0.Bhi : 1; Q.nblo = Q.sBlo ? g0.Blo : 1;
  // K per launch <= 65536 (int64 headroom): groups of G
  const int gstep = std::max(1, (int)std::min<long>(g0.G, 65536L / std::max(g0.K, 1)));
  ATTN_REQUIRE(g0.K <= 65536, ATTN_EUNSUPPORTED, "K above 65536 for the split GEMM");
  const size_t smem = 1024 + 2 * (size_t)kQBufBytes + (size_t)kPStages * kPBytes + 256;
  static bool attr = false;
  if (!attr) {
    ATTN_CHECK_CUDA(cudaFuncSetAttribute(ozaki_gemm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    attr = true;
  }
  ctx->oz_err.reserve(sizeof(int));
  if (!ctx->oz_err_init) {
    ATTN_CHECK_CUDA(cudaMemsetAsync(ctx->oz_err.p, 0, sizeof(int), ctx->stream));
    ctx->oz_err_init = true;
  }
  const double fl = 2.0 * g0.M * g0.N * (double)g0.K * g0.G * g0.Bhi * g0.Blo;
  ctx->prof_begin(3);
  for (int ga = 0; ga < g0.G; ga += gstep) {
    const int gn = std::min(gstep, g0.G - ga);
    OzView p = P, q = Q;
    p.p = P.p + (long)ga * P.sG;
    q.p = Q.p + (long)ga * Q.sG;
    p.G = q.G = gn;
    const long Kt = (long)g0.K * gn;
    const long Kpad = (Kt + 63) / 64 * 64;
    ozaki_slice(ctx, p, Kpad, 128, ctx->oz_ws[0], ctx->oz_ws[1]);
    ozaki_slice(ctx, q, Kpad, kQRows, ctx->oz_ws[2], ctx->oz_ws[3]);
    const int nrtP = (M + 127) / 128, nrtQ = (N + kQRows - 1) / kQRows;
    const long nkb = Kpad / 64;
    OzMaps maps;
    encode_slices(&maps.p, ctx->oz_ws[0].as<__nv_bfloat16>(), 128, (long)p.nbhi * p.nblo * nrtP * nkb * kSlices);
    encode_slices(&maps.q, ctx->oz_ws[2].as<__nv_bfloat16>(), kQRows, (long)q.nbhi * q.nblo * nrtQ * nkb * kSlices);
    OzParams prm;
    prm.M = M; prm.N = N; prm.nkb = (int)nkb;
    prm.nrtP = nrtP; prm.nrtQ = nrtQ;
    prm.Bhi = g0.Bhi; prm.Blo = g0.Blo;
    prm.p_hi = P.sBhi ? p.nblo : 0; prm.p_lo = P.sBlo ? 1 : 0;
    prm.q_hi = Q.sBhi ? q.nblo : 0; prm.q_lo = Q.sBlo ? 1 : 0;
    prm.EP = ctx->oz_ws[1].as<int>();
    prm.EQ = ctx->oz_ws[3].as<int>();
    prm.C = g0.C; prm.c_rs = c_rs; prm.c_cs = c_cs; prm.c_bhi = g0.cBhi; prm.c_blo = g0.cBlo;
    {
      int ex = 0;
      const double fr = std::frexp(g0.alpha, &ex);  // alpha = fr 2^ex, fr in [0.5, 1)
      const bool pow2 = std::isfinite(g0.alpha) && std::fabs(fr) == 0.5;
      prm.alpha_exp = pow2 ? ex - 1 : 0;
      prm.alpha_rest = pow2 ? (fr < 0 ? -1.0 : 1.0) : g0.alpha;
    }
    prm.beta = ga == 0 ? g0.beta : 1.0;
    prm.err = ctx->oz_err.as<int>();
    // persistent: one CTA per SM (the shared-memory ring allows one), at most one per tile
    prm.tiles = (long)((N + kQRows - 1) / kQRows) * ((M + 127) / 128) * g0.Bhi * g0.Blo;
    const int grid = (int)std::min<long>(prm.tiles, std::max(ctx->num_sms, 1));
    ozaki_gemm_kernel<<<grid, kOzThreads, smem, ctx->stream>>>(maps, prm);
    ctx->launches++;
  }
  ctx->prof_end(3, fl);
  ATTN_CHECK_CUDA(cudaGetLastError());
}

int ozaki_error(attn_ctx* ctx) {
  if (!ctx->oz_err_init) return 0;
  int e = 0;
  ATTN_CHECK_CUDA(cudaMemcpyAsync(&e, ctx->oz_err.p, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
  ATTN_CHECK_CUDA(cudaStreamSynchronize(ctx->stream));
  if (e) ATTN_CHECK_CUDA(cudaMemsetAsync(ctx->oz_err.p, 0, sizeof(int), ctx->stream));
  return e;
}

}  // namespace attn
