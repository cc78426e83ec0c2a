// BF16 H_eff on the 5th-generation tensor cores (tcgen05 + TMEM + TMA), FP32
// accumulation (Sec. 3.3.2 last paragraph, Sec. 4.4.2, Fig. eff-op-cost).
//
// For a pair kind (p, q) with slice slot s, every slice X_s (P x Q, the
// tensor with slot s fixed) gets
//     Y_s = sum_r A_r X_s B_r^T      (A_r: P x P on slot p, B_r: Q x Q on slot q)
// computed per product as two chained MMAs in one CTA:
//   stage 1:  D1[j][i'] = sum_j' B_r[j][j'] X_s[i'][j']          (M = j, N = i', K = j')
//   convert:  D1 (FP32, TMEM) -> BF16 Z^T[j][i'] in shared memory (128B swizzle)
//   stage 2:  D2[i][j] += sum_i' A_r[i][i'] Z^T[j][i']           (M = i, N = j, K = i')
// D2 = Y_s stays in TMEM across all products of the slice. All operands are
// K-major with the 128-byte swizzle; TMA brings X_s once and streams A_r, B_r
// through two-deep rings (separate producer threads for the A and B rings).
// The stage-1 accumulator is double-buffered in TMEM so that the conversion of
// product r overlaps stage 1 of product r+1.
//
// Warp roles (256 threads): warp 0 = B/X producer, warp 2 = A producer,
// warp 1 = TMEM allocation + MMA issue, warps 4-7 = conversion and epilogue
// (warp w reads TMEM lanes 32*(w%4) .. +31). Internal (single-link)
// operators enter as products with an identity partner; three-link products
// go through the FP64 path. Every mbarrier wait is bounded (about 2 s of
// clock); on timeout the kernel records an error code, stops issuing work,
// waits (bounded) for its in-flight copies, frees TMEM and returns.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>

#include "heff.h"

namespace attn {

namespace {

constexpr int kThreads = 256;
constexpr int kTileBytes = 128 * 128 * 2;  // one 128 x 128 BF16 operand tile (two 64-wide K blocks)
constexpr int kKBlockBytes = 128 * 128;    // 128 rows x 128 bytes
constexpr uint32_t kTmemCols = 512;
constexpr long long kWaitCycles = 4000000000LL;  // ~2 s at 2 GHz

struct KindParams {
  int P, Q, S, R;     // slice rows/cols, slices, products
  int cta_begin;      // first CTA index of this kind
  float* Y;           // [S][P][Q] fp32 output (written)
};

struct TcParams {
  KindParams kind[3];
  int nkinds;
  int* err;           // device error word (0 = ok)
};

struct TcMaps {
  CUtensorMap x[3], a[3], b[3];
};

// ------------------------------------------------------------- PTX helpers
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count));
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}

// Bounded wait: returns false (and records `code`) after ~kWaitCycles.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, int* err, int code, volatile int* abort_flag) {
  long long t0 = clock64();
  while (!mbar_try_wait(bar, parity)) {
    if (*abort_flag) return false;
    if (clock64() - t0 > kWaitCycles) {
      atomicCAS(err, 0, code);
      *abort_flag = 1;
      return false;
    }
  }
  return true;
}

__device__ __forceinline__ void tma_load_3d(uint32_t dst, const CUtensorMap* map, int c0, int c1, int c2,
                                            uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(
          dst),
      "l"((uint64_t)map), "r"(c0), "r"(c1), "r"(c2), "r"(bar)
      : "memory");
}

__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);  // start address
  d |= (uint64_t)1 << 16;                     // leading byte offset (unused for swizzled K-major)
  d |= (uint64_t)(1024 >> 4) << 32;           // stride byte offset: 8 rows x 128 B
  d |= (uint64_t)1 << 46;                     // descriptor version
  d |= (uint64_t)2 << 61;                     // 128-byte swizzle
  return d;
}

// kind::f16 instruction descriptor: D = F32, A = B = BF16, both K-major.
__device__ __forceinline__ uint32_t idesc_bf16(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(
          d_tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(acc)
      : "memory");
}

__device__ __forceinline__ void mma_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,%18,%19,"
      "%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]),
        "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
        "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
  __nv_bfloat162 h = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<uint32_t*>(&h);
}

// ------------------------------------------------------------------ kernel
__global__ void __launch_bounds__(kThreads, 1) sandwich_tc_kernel(const __grid_constant__ TcMaps maps, TcParams prm) {
  extern __shared__ uint8_t smem_raw[];
  // carve 1024-aligned regions
  const uint32_t raw = smem_u32(smem_raw);
  const uint32_t base = (raw + 1023u) & ~1023u;
  uint8_t* gbase = smem_raw + (base - raw);
  const uint32_t sX = base;                       // 32 KB
  const uint32_t sB = sX + kTileBytes;            // 2 x 32 KB
  const uint32_t sA = sB + 2 * kTileBytes;        // 2 x 32 KB
  const uint32_t sZ = sA + 2 * kTileBytes;        // 32 KB
  uint8_t* gZ = gbase + (sZ - base);
  const uint32_t sBar = sZ + kTileBytes;          // barriers
  uint64_t* bars = reinterpret_cast<uint64_t*>(gbase + (sBar - base));
  // barrier indices
  enum { XFULL = 0, BFULL = 1, BEMPTY = 3, AFULL = 5, AEMPTY = 7, D1FULL = 9, ZFULL = 11, ZEMPTY = 12, D2FULL = 13,
         NBAR = 14 };
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + NBAR);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
  auto bar = [&](int i) { return sBar + 8u * (uint32_t)i; };

  // which kind / slice does this CTA own?
  int kind = 0;
  for (int k = 1; k < prm.nkinds; ++k)
    if ((int)blockIdx.x >= prm.kind[k].cta_begin) kind = k;
  const KindParams kp = prm.kind[kind];
  const int s = blockIdx.x - kp.cta_begin;
  const int P = kp.P, Q = kp.Q, R = kp.R;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  if (threadIdx.x == 0) {
    mbar_init(bar(XFULL), 1);
    for (int i = 0; i < 2; ++i) {
      mbar_init(bar(BFULL + i), 1);
      mbar_init(bar(BEMPTY + i), 1);
      mbar_init(bar(AFULL + i), 1);
      mbar_init(bar(AEMPTY + i), 1);
      mbar_init(bar(D1FULL + i), 1);
    }
    mbar_init(bar(ZFULL), 128);
    mbar_init(bar(ZEMPTY), 1);
    mbar_init(bar(D2FULL), 1);
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
  const uint32_t tD1[2] = {tmem, tmem + 128};
  const uint32_t tD2 = tmem + 256;
  const int nkbQ = (Q + 63) / 64, nkbP = (P + 63) / 64;
  const CUtensorMap* mX = &maps.x[kind];
  const CUtensorMap* mA = &maps.a[kind];
  const CUtensorMap* mB = &maps.b[kind];

  if (warp == 0 && lane == 0) {
    // ---- X and B producer
    mbar_expect_tx(bar(XFULL), (uint32_t)(nkbQ * P * 128));
    for (int kb = 0; kb < nkbQ; ++kb) tma_load_3d(sX + kb * (P * 128), mX, 64 * kb, 0, s, bar(XFULL));
    int issued = 0;
    for (int r = 0; r < R; ++r) {
      const int slot = r & 1;
      if (r >= 2 && !mbar_wait(bar(BEMPTY + slot), ((r >> 1) - 1) & 1, prm.err, 11, abort_flag)) break;
      mbar_expect_tx(bar(BFULL + slot), (uint32_t)(nkbQ * kKBlockBytes));
      for (int kb = 0; kb < nkbQ; ++kb)
        tma_load_3d(sB + slot * kTileBytes + kb * kKBlockBytes, mB, 64 * kb, 0, r, bar(BFULL + slot));
      issued = r + 1;
    }
    // drain: wait (bounded) until every issued load has landed
    mbar_wait(bar(XFULL), 0, prm.err, 12, abort_flag);
    for (int r = (issued >= 2 ? issued - 2 : 0); r < issued; ++r) {
      long long t0 = clock64();
      while (!mbar_try_wait(bar(BFULL + (r & 1)), (r >> 1) & 1) && clock64() - t0 < kWaitCycles) {}
    }
  } else if (warp == 2 && lane == 0) {
    // ---- A producer
    int issued = 0;
    for (int r = 0; r < R; ++r) {
      const int slot = r & 1;
      if (r >= 2 && !mbar_wait(bar(AEMPTY + slot), ((r >> 1) - 1) & 1, prm.err, 21, abort_flag)) break;
      mbar_expect_tx(bar(AFULL + slot), (uint32_t)(nkbP * kKBlockBytes));
      for (int kb = 0; kb < nkbP; ++kb)
        tma_load_3d(sA + slot * kTileBytes + kb * kKBlockBytes, mA, 64 * kb, 0, r, bar(AFULL + slot));
      issued = r + 1;
    }
    for (int r = (issued >= 2 ? issued - 2 : 0); r < issued; ++r) {
      long long t0 = clock64();
      while (!mbar_try_wait(bar(AFULL + (r & 1)), (r >> 1) & 1) && clock64() - t0 < kWaitCycles) {}
    }
  } else if (warp == 1 && lane == 0) {
    // ---- MMA issuer
    const uint32_t id1 = idesc_bf16(128, P);
    const uint32_t id2 = idesc_bf16(128, Q);
    bool ok = mbar_wait(bar(XFULL), 0, prm.err, 31, abort_flag);
    for (int r = 0; ok && r <= R; ++r) {
      if (r < R) {
        const int slot = r & 1;
        if (!mbar_wait(bar(BFULL + slot), (r >> 1) & 1, prm.err, 32, abort_flag)) break;
        fence_after();
        const uint32_t aB = sB + slot * kTileBytes;
        for (int k = 0; k < Q / 16; ++k) {
          const uint32_t off = (k >> 2) * kKBlockBytes + (k & 3) * 32;
          const uint32_t offX = (k >> 2) * (P * 128) + (k & 3) * 32;
          mma_bf16(tD1[r & 1], sw128_desc(aB + off), sw128_desc(sX + offX), id1, k > 0);
        }
        mma_commit(bar(BEMPTY + slot));
        mma_commit(bar(D1FULL + (r & 1)));
      }
      if (r >= 1) {
        const int rr = r - 1, slot = rr & 1;
        if (!mbar_wait(bar(AFULL + slot), (rr >> 1) & 1, prm.err, 33, abort_flag)) break;
        if (!mbar_wait(bar(ZFULL), rr & 1, prm.err, 34, abort_flag)) break;
        fence_after();
        const uint32_t aA = sA + slot * kTileBytes;
        for (int k = 0; k < P / 16; ++k) {
          const uint32_t off = (k >> 2) * kKBlockBytes + (k & 3) * 32;
          const uint32_t offZ = (k >> 2) * (Q * 128) + (k & 3) * 32;
          mma_bf16(tD2, sw128_desc(aA + off), sw128_desc(sZ + offZ), id2, (rr > 0 || k > 0) ? 1u : 0u);
        }
        mma_commit(bar(AEMPTY + slot));
        mma_commit(bar(ZEMPTY));
      }
    }
    mma_commit(bar(D2FULL));
    // every MMA this thread issued must finish before TMEM can be freed
    {
      long long t0 = clock64();
      while (!mbar_try_wait(bar(D2FULL), 0) && clock64() - t0 < kWaitCycles) {}
    }
  } else if (warp >= 4) {
    // ---- conversion D1 -> Z^T (bf16, swizzled) and the epilogue
    const int q4 = warp & 3;
    const int j = q4 * 32 + lane;  // TMEM lane == row of D1 (j) and of D2 (i)
    const uint32_t lane_off = (uint32_t)(q4 * 32) << 16;
    bool ok = true;
    for (int r = 0; r < R && ok; ++r) {
      if (!mbar_wait(bar(D1FULL + (r & 1)), (r >> 1) & 1, prm.err, 41, abort_flag)) { ok = false; break; }
      if (r >= 1 && !mbar_wait(bar(ZEMPTY), (r - 1) & 1, prm.err, 42, abort_flag)) { ok = false; break; }
      fence_after();
      for (int c0 = 0; c0 < P; c0 += 32) {
        float v[32];
        tmem_ld32(tD1[r & 1] + lane_off + c0, v);
        if (j < Q) {
#pragma unroll
          for (int h = 0; h < 4; ++h) {  // four 16-byte chunks of 8 elements
            const int i0 = c0 + 8 * h;   // column index i'
            const int kb = i0 >> 6, chunk = (i0 & 63) >> 3;
            uint4 w;
            w.x = pack_bf16(v[8 * h + 0], v[8 * h + 1]);
            w.y = pack_bf16(v[8 * h + 2], v[8 * h + 3]);
            w.z = pack_bf16(v[8 * h + 4], v[8 * h + 5]);
            w.w = pack_bf16(v[8 * h + 6], v[8 * h + 7]);
            const uint32_t off = kb * (Q * 128) + (j >> 3) * 1024 + (j & 7) * 128 + ((chunk ^ (j & 7)) << 4);
            *reinterpret_cast<uint4*>(gZ + off) = w;
          }
        }
      }
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      fence_before();
      mbar_arrive(bar(ZFULL));
    }
    if (ok && mbar_wait(bar(D2FULL), 0, prm.err, 43, abort_flag)) {
      fence_after();
      const int i = j;
      float* yrow = kp.Y + ((long)s * P + i) * Q;
      for (int c0 = 0; c0 < Q; c0 += 32) {
        float v[32];
        tmem_ld32(tD2 + lane_off + c0, v);
        if (i < P) {
#pragma unroll
          for (int h = 0; h < 8; ++h)
            if (c0 + 4 * h < Q)
              *reinterpret_cast<float4*>(yrow + c0 + 4 * h) =
                  make_float4(v[4 * h], v[4 * h + 1], v[4 * h + 2], v[4 * h + 3]);
        }
      }
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
// x (fp64 [m0][m1][m2]) -> bf16 slice-major copies for the three pair kinds:
// X01[c][a][b], X02[b][a][c], X12[a][b][c].
__global__ void prep_x_kernel(const double* x, int m0, int m1, int m2, __nv_bfloat16* x01, __nv_bfloat16* x02,
                              __nv_bfloat16* x12) {
  const long V = (long)m0 * m1 * m2;
  for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < V; e += (long)gridDim.x * blockDim.x) {
    const int c = e % m2;
    const long t = e / m2;
    const int b = t % m1, a = t / m1;
    const __nv_bfloat16 v = __double2bfloat16(x[e]);
    if (x01) x01[((long)c * m0 + a) * m1 + b] = v;
    if (x02) x02[((long)b * m0 + a) * m2 + c] = v;
    if (x12) x12[e] = v;
  }
}

// y = Y01^T + Y02^T + Y12 (fp32 -> fp64)
__global__ void combine_kernel(double* y, int m0, int m1, int m2, const float* y01, const float* y02,
                               const float* y12) {
  const long V = (long)m0 * m1 * m2;
  for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < V; e += (long)gridDim.x * blockDim.x) {
    const int c = e % m2;
    const long t = e / m2;
    const int b = t % m1, a = t / m1;
    double v = 0.0;
    if (y01) v += (double)y01[((long)c * m0 + a) * m1 + b];
    if (y02) v += (double)y02[((long)b * m0 + a) * m2 + c];
    if (y12) v += (double)y12[e];
    y[e] = v;
  }
}

// dst[r] = bf16(src[r]) for r < R (stack of m x m), plus optional extra slices:
// identity (mode 1) or a given matrix (mode 2) appended.
__global__ void to_bf16_kernel(__nv_bfloat16* dst, const double* src, long n) {
  for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < n; e += (long)gridDim.x * blockDim.x)
    dst[e] = __double2bfloat16(src[e]);
}

__global__ void identity_bf16_kernel(__nv_bfloat16* dst, int m) {
  for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < (long)m * m; e += (long)gridDim.x * blockDim.x)
    dst[e] = __float2bfloat16((e / m == e % m) ? 1.0f : 0.0f);
}

int vgrid(long n) { return (int)std::max<long>(1, std::min<long>((n + 255) / 256, 4096)); }

}  // namespace

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

// Host: 3-D tiled tensor map over a [D2][D1][D0] bf16 array with a {64, rows, 1} box, 128B swizzle.
void encode_map(CUtensorMap* map, const void* ptr, int d0, int d1, int d2, int box_rows) {
  cuuint64_t dims[3] = {(cuuint64_t)d0, (cuuint64_t)d1, (cuuint64_t)d2};
  cuuint64_t strides[2] = {(cuuint64_t)d0 * 2, (cuuint64_t)d0 * d1 * 2};
  cuuint32_t box[3] = {64, (cuuint32_t)box_rows, 1};
  cuuint32_t estr[3] = {1, 1, 1};
  CUresult res = tensor_map_encoder()(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<void*>(ptr), dims,
                                        strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                                        CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  ATTN_REQUIRE(res == CUDA_SUCCESS, ATTN_ECUDA, "cuTensorMapEncodeTiled failed (" + std::to_string((int)res) + ")");
}

}  // namespace

// Per-H_eff tensor-core state.
struct TcState {
  DevBuf a[3], b[3];     // bf16 operator stacks per kind [R'][P][P], [R'][Q][Q]
  int R[3] = {0, 0, 0};  // products per kind (incl. internal operators)
  DevBuf x[3];           // bf16 slice-major input per kind
  DevBuf y[3];           // fp32 output per kind
  DevBuf err;
  TcMaps maps;
  TcParams prm;
  int grid = 0;
  size_t smem = 0;
  bool fp64_triples = false;
};

bool tc_supported(const attn_heff* h) {
  for (int s = 0; s < 3; ++s)
    if (h->m[s] % 16 != 0 || h->m[s] > 128 || h->m[s] < 16) return false;
  return true;
}

void tc_release(attn_heff* h) {
  delete static_cast<TcState*>(h->tc);
  h->tc = nullptr;
  h->tc_ready = false;
}

static void tc_build(attn_heff* h) {
  attn_ctx* ctx = h->ctx;
  auto* t = new TcState();
  h->tc = t;
  cudaStream_t st = ctx->stream;
  const int* m = h->m;
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
    t->a[k].reserve(sizeof(__nv_bfloat16) * (size_t)R * P * P);
    t->b[k].reserve(sizeof(__nv_bfloat16) * (size_t)R * Q * Q);
    auto* A = t->a[k].as<__nv_bfloat16>();
    auto* B = t->b[k].as<__nv_bfloat16>();
    if (h->npair[k]) {
      to_bf16_kernel<<<vgrid((long)h->npair[k] * P * P), 256, 0, st>>>(A, h->pa[k].as<double>(), (long)h->npair[k] * P * P);
      to_bf16_kernel<<<vgrid((long)h->npair[k] * Q * Q), 256, 0, st>>>(B, h->pb[k].as<double>(), (long)h->npair[k] * Q * Q);
      ctx->launches += 2;
    }
    for (int e = 0; e < extra; ++e) {
      __nv_bfloat16* Ae = A + (long)(h->npair[k] + e) * P * P;
      __nv_bfloat16* Be = B + (long)(h->npair[k] + e) * Q * Q;
      if (ea[e]) to_bf16_kernel<<<vgrid((long)P * P), 256, 0, st>>>(Ae, ea[e], (long)P * P);
      else identity_bf16_kernel<<<vgrid((long)P * P), 256, 0, st>>>(Ae, P);
      if (eb[e]) to_bf16_kernel<<<vgrid((long)Q * Q), 256, 0, st>>>(Be, eb[e], (long)Q * Q);
      else identity_bf16_kernel<<<vgrid((long)Q * Q), 256, 0, st>>>(Be, Q);
      ctx->launches += 2;
    }
    const int S = m[sl];
    t->x[k].reserve(sizeof(__nv_bfloat16) * (size_t)h->V);
    t->y[k].reserve(sizeof(float) * (size_t)h->V);
    encode_map(&t->maps.x[k], t->x[k].p, Q, P, S, P);
    encode_map(&t->maps.a[k], t->a[k].p, P, P, R, 128);
    encode_map(&t->maps.b[k], t->b[k].p, Q, Q, R, 128);
    KindParams& kp = t->prm.kind[nk];
    kp.P = P; kp.Q = Q; kp.S = S; kp.R = R; kp.cta_begin = cta; kp.Y = t->y[k].as<float>();
    if (nk != k) {
      t->maps.x[nk] = t->maps.x[k];
      t->maps.a[nk] = t->maps.a[k];
      t->maps.b[nk] = t->maps.b[k];
    }
    cta += S;
    ++nk;
  }
  t->prm.nkinds = nk;
  t->grid = cta;
  t->err.reserve(sizeof(int));
  ATTN_CHECK_CUDA(cudaMemsetAsync(t->err.p, 0, sizeof(int), st));
  t->prm.err = t->err.as<int>();
  t->smem = 1024 + 6 * (size_t)kTileBytes + 256;
  ATTN_CHECK_CUDA(cudaFuncSetAttribute(sandwich_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)t->smem));
  ATTN_CHECK_CUDA(cudaGetLastError());
  h->tc_ready = true;
}

}  // namespace attn

using namespace attn;

void attn_heff::apply_bf16(const double* x, double* y) {
  ATTN_REQUIRE(tc_supported(this), ATTN_EUNSUPPORTED,
               "BF16 tensor-core path needs every link dimension in {16, 32, ..., 128}");
  if (!tc_ready) tc_build(this);
  TcState* t = static_cast<TcState*>(tc);
  cudaStream_t st = ctx->stream;
  // the kind buffers are indexed by pair kind k (0,1,2); kinds with no products pass null
  prep_x_kernel<<<vgrid(V), 256, 0, st>>>(x, m[0], m[1], m[2], t->R[0] ? t->x[0].as<__nv_bfloat16>() : nullptr,
                                          t->R[1] ? t->x[1].as<__nv_bfloat16>() : nullptr,
                                          t->R[2] ? t->x[2].as<__nv_bfloat16>() : nullptr);
  ctx->launches++;
  if (t->grid > 0) {
    // algorithmic FLOPs of this launch: the pair products and the internal operators
    double fl = 0.0;
    for (int k = 0; k < 3; ++k) fl += (double)npair[k] * 2.0 * (m[kPairP[k]] + m[kPairQ[k]]) * V;
    for (int s = 0; s < 3; ++s)
      if (has_hint[s]) fl += 2.0 * m[s] * V;
    ctx->prof_begin(0);
    sandwich_tc_kernel<<<t->grid, kThreads, t->smem, st>>>(t->maps, t->prm);
    ctx->prof_end(0, fl);
    ctx->launches++;
  }
  combine_kernel<<<vgrid(V), 256, 0, st>>>(y, m[0], m[1], m[2], t->R[0] ? t->y[0].as<float>() : nullptr,
                                           t->R[1] ? t->y[1].as<float>() : nullptr,
                                           t->R[2] ? t->y[2].as<float>() : nullptr);
  ctx->launches++;
  ATTN_CHECK_CUDA(cudaGetLastError());
  if (ntrip > 0) {
    // three-link products in FP64 on top of the tensor-core result
    const int d[3] = {m[0], m[1], m[2]};
    const long budget = 1L << 27;
    const int chunk = (int)std::max<long>(1, std::min<long>(4096, budget / std::max<long>(V, 1)));
    for (int r0 = 0; r0 < ntrip; r0 += chunk) {
      const int R = std::min(chunk, ntrip - r0);
      ctx->ws[0].reserve(sizeof(double) * (size_t)R * V);
      ctx->ws[1].reserve(sizeof(double) * (size_t)R * V);
      double* W1 = ctx->ws[0].as<double>();
      double* W2 = ctx->ws[1].as<double>();
      mode_product_f64(ctx, d, 2, tr[2].as<double>() + (long)r0 * m[2] * m[2], R, x, 0, W1, 0.0);
      mode_product_f64(ctx, d, 1, tr[1].as<double>() + (long)r0 * m[1] * m[1], R, W1, V, W2, 0.0);
      accumulate_slot_f64(ctx, d, 0, tr[0].as<double>() + (long)r0 * m[0] * m[0], R, W2, y);
    }
  }
}

namespace attn {
// Read and clear the tensor-core error word of an H_eff (0 = ok).
int tc_error(attn_heff* h) {
  if (!h->tc_ready) return 0;
  TcState* t = static_cast<TcState*>(h->tc);
  int e = 0;
  ATTN_CHECK_CUDA(cudaMemcpyAsync(&e, t->err.p, sizeof(int), cudaMemcpyDeviceToHost, h->ctx->stream));
  ATTN_CHECK_CUDA(cudaStreamSynchronize(h->ctx->stream));
  if (e) ATTN_CHECK_CUDA(cudaMemsetAsync(t->err.p, 0, sizeof(int), h->ctx->stream));
  return e;
}
}  // namespace attn
