// Batched GEMM on the tcgen05 tensor cores, FP32 accumulation in TMEM:
//     C[b][i][j] (+)= alpha * sum_k A[bA(b)][i][k] * B[bB(b)][j][k]
// with BF16 operands (kind::f16) or TF32 ones (kind::tf32, FP32 storage).
// Both operands are K-major (a row of A or B is contiguous along k) and come in
// through TMA as 128-row x 128-byte tiles (64 BF16 or 32 TF32 values of k) with the
// 128-byte swizzle, three stages deep.
// One CTA computes one 128 x 128 output tile of one batch entry; the epilogue
// writes FP32, BF16 or FP64 with arbitrary row/column/batch strides (so a
// transposed or permuted output layout costs nothing extra). Used for the
// tensor-core renormalisation T^T (A (x) B) T of Fig. eff-op and for the
// three-link products of H_eff.
//
// Warp roles (192 threads): warp 0 = TMA producer, warp 1 = TMEM allocation
// and MMA issue, warps 2-5 = epilogue (warp w reads TMEM lanes 32*(w%4)+..).
// All waits are bounded; a timeout records an error code and the CTA drains
// and frees TMEM before returning.
#include <algorithm>

#include "gemm_tc.h"
#include "tc_ptx.h"

namespace attn {

namespace {

using namespace tc;

constexpr int kStages = 3;
constexpr int kStageBytes = 2 * 128 * 128;  // A and B tiles of 128 rows x 128 bytes
constexpr int kTnThreads = 192;

struct TnMaps {
  CUtensorMap a, b;
};

template <bool kTF>
__global__ void __launch_bounds__(kTnThreads, 2) tn_gemm_kernel(const __grid_constant__ TnMaps maps, TnParams p) {
  constexpr int KB = kTF ? 32 : 64;  // k values per 128-byte K block
  extern __shared__ uint8_t smem_raw[];
  const uint32_t raw = smem_u32(smem_raw);
  const uint32_t base = (raw + 1023u) & ~1023u;
  uint8_t* gbase = smem_raw + (base - raw);
  const uint32_t sBar = base + kStages * kStageBytes;
  enum { FULL = 0, EMPTY = kStages, DONE = 2 * kStages, NBAR = 2 * kStages + 1 };
  uint64_t* bars = reinterpret_cast<uint64_t*>(gbase + (sBar - base));
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + NBAR);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
  auto bar = [&](int i) { return sBar + 8u * (uint32_t)i; };
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const long b = (long)blockIdx.z + p.batch_offset;
  const int bhi = (int)(b / p.Blo), blo = (int)(b % p.Blo);
  const int m0 = blockIdx.y * 128, n0 = blockIdx.x * 128;
  const int nk = (p.K + KB - 1) / KB;

  if (threadIdx.x == 0) {
    for (int s = 0; s < kStages; ++s) {
      mbar_init(bar(FULL + s), 1);
      mbar_init(bar(EMPTY + s), 1);
    }
    mbar_init(bar(DONE), 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(128));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == 0 && lane == 0) {
    const int ca = bhi * p.a_bhi + blo * p.a_blo, cb = bhi * p.b_bhi + blo * p.b_blo;
    int issued = 0;
    for (int kb = 0; kb < nk; ++kb) {
      const int s = kb % kStages;
      if (kb >= kStages && !mbar_wait(bar(EMPTY + s), ((kb / kStages) - 1) & 1, p.err, 51, abort_flag)) break;
      mbar_expect_tx(bar(FULL + s), (uint32_t)kStageBytes);
      const uint32_t dst = base + s * kStageBytes;
      tma_load_3d(dst, &maps.a, KB * kb, m0, ca, bar(FULL + s));
      tma_load_3d(dst + kStageBytes / 2, &maps.b, KB * kb, n0, cb, bar(FULL + s));
      issued = kb + 1;
    }
    for (int kb = (issued > kStages ? issued - kStages : 0); kb < issued; ++kb) {
      long long t0 = clock64();
      while (!mbar_try_wait(bar(FULL + kb % kStages), (kb / kStages) & 1) && clock64() - t0 < kWaitCycles) {}
    }
  } else if (warp == 1 && lane == 0) {
    const uint32_t id = idesc_of<kTF>(128, 128);
    for (int kb = 0; kb < nk; ++kb) {
      const int s = kb % kStages;
      if (!mbar_wait(bar(FULL + s), (kb / kStages) & 1, p.err, 52, abort_flag)) break;
      fence_after();
      const uint32_t a = base + s * kStageBytes, bb = a + kStageBytes / 2;
#pragma unroll
      for (int k = 0; k < 4; ++k)
        mma_ss<kTF>(tmem, sw128_desc(a + 32 * k), sw128_desc(bb + 32 * k), id, (kb > 0 || k > 0) ? 1u : 0u);
      mma_commit(bar(EMPTY + s));
    }
    mma_commit(bar(DONE));
    long long t0 = clock64();
    while (!mbar_try_wait(bar(DONE), 0) && clock64() - t0 < kWaitCycles) {}
  } else if (warp >= 2) {
    const int q4 = warp & 3;
    const int i = m0 + q4 * 32 + lane;
    const uint32_t lane_off = (uint32_t)(q4 * 32) << 16;
    // warp-uniform: the TMEM loads below are .sync.aligned
    if (nk > 0 && __all_sync(0xffffffffu, mbar_wait(bar(DONE), 0, p.err, 53, abort_flag))) {
      fence_after();
      const long cbase = (long)bhi * p.c_bhi + (long)blo * p.c_blo + (long)i * p.c_rs;
      for (int c0 = 0; c0 < 128; c0 += 32) {
        float v[32];
        tmem_ld32(tmem + lane_off + c0, v);
        if (i >= p.M) continue;
#pragma unroll
        for (int h = 0; h < 32; ++h) {
          const int j = n0 + c0 + h;
          if (j >= p.N) continue;
          const long o = cbase + (long)j * p.c_cs;
          const float val = p.alpha * v[h];
          if (p.c_type == 0) {
            float* C = static_cast<float*>(p.C);
            C[o] = p.accumulate ? C[o] + val : val;
          } else if (p.c_type == 1) {
            __nv_bfloat16* C = static_cast<__nv_bfloat16*>(p.C);
            C[o] = __float2bfloat16(p.accumulate ? __bfloat162float(C[o]) + val : val);
          } else if (p.c_type == 2) {
            double* C = static_cast<double*>(p.C);
            C[o] = p.accumulate ? C[o] + (double)val : (double)val;
          } else {
            float* C = static_cast<float*>(p.C);
            C[o] = round_tf32(p.accumulate ? C[o] + val : val);
          }
        }
      }
    }
  }
  fence_before();
  __syncthreads();
  if (warp == 1) {
    fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(128));
  }
}

void encode(CUtensorMap* map, const TnOperand& o) {
  const int es = o.tf ? 4 : 2;
  cuuint64_t dims[3] = {(cuuint64_t)o.K, (cuuint64_t)o.rows, (cuuint64_t)std::max(o.batches, 1)};
  cuuint64_t strides[2] = {(cuuint64_t)o.ld * es, (cuuint64_t)std::max<long>(o.bstride, o.ld * o.rows) * es};
  cuuint32_t box[3] = {(cuuint32_t)(128 / es), 128, 1};
  cuuint32_t estr[3] = {1, 1, 1};
  ATTN_REQUIRE((o.ld * es) % 16 == 0 && ((o.bstride * es) % 16 == 0) && ((uintptr_t)o.p % 16 == 0), ATTN_EINVAL,
               "tensor-core GEMM operands need 16-byte aligned rows");
  CUresult r = tensor_map_encoder()(map, o.tf ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3,
                                    const_cast<void*>(o.p), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                                    CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  ATTN_REQUIRE(r == CUDA_SUCCESS, ATTN_ECUDA, "cuTensorMapEncodeTiled failed for a GEMM operand");
}

}  // namespace

void tn_gemm(attn_ctx* ctx, const TnOperand& A, const TnOperand& B, TnParams p, DevBuf& err) {
  if (p.M <= 0 || p.N <= 0 || p.Bhi <= 0 || p.Blo <= 0) return;
  ATTN_REQUIRE(A.tf == B.tf, ATTN_EINVAL, "tensor-core GEMM operands must have the same type");
  TnMaps maps;
  encode(&maps.a, A);
  encode(&maps.b, B);
  err.reserve(sizeof(int));
  p.err = err.as<int>();
  const size_t smem = 1024 + (size_t)kStages * kStageBytes + 256;
  static bool attr = false;
  if (!attr) {
    ATTN_CHECK_CUDA(cudaFuncSetAttribute(tn_gemm_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    ATTN_CHECK_CUDA(cudaFuncSetAttribute(tn_gemm_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    attr = true;
  }
  const long total = (long)p.Bhi * p.Blo;
  dim3 grid((p.N + 127) / 128, (p.M + 127) / 128, 1);
  ATTN_REQUIRE(grid.y <= 65535, ATTN_EUNSUPPORTED, "GEMM M too large");
  double fl = 2.0 * p.M * (double)p.N * p.K * (double)total;
  ctx->prof_begin(2);
  for (long off = 0; off < total; off += 65535) {
    grid.z = (unsigned)std::min<long>(65535, total - off);
    p.batch_offset = off;
    if (A.tf) tn_gemm_kernel<true><<<grid, kTnThreads, smem, ctx->stream>>>(maps, p);
    else tn_gemm_kernel<false><<<grid, kTnThreads, smem, ctx->stream>>>(maps, p);
    ctx->launches++;
  }
  ctx->prof_end(2, fl);
  ATTN_CHECK_CUDA(cudaGetLastError());
}

}  // namespace attn
