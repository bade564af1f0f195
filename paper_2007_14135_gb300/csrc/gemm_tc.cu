// BF16 GEMM on the tensor cores for the learned-proposal network: D[M x N] = A[M x K] B[N x K]^T
// (both operands K-contiguous, "NT"), FP32 accumulation in TMEM, fused epilogues.
//
// Tile 128 x BN (BN <= 256, multiple of 16) x 64 (one 128-byte swizzle atom of BF16). TMA loads
// both operand tiles with the 128B swizzle straight into the layout tcgen05 reads, through a
// 4-stage ring: warp 0 (one lane) produces (waits "empty", expect_tx, two cp.async.bulk.tensor),
// warp 1 (one lane) consumes (waits "full", four MMAs of K = 16, commit to "empty"); a final
// commit releases the epilogue, where each of the 4 warps reads its 32 TMEM lanes (rows) with
// tcgen05.ld and applies one of:
//   EPI_F32      : D stored as FP32 (row-major, ldd)
//   EPI_BIAS_F32 : D + bias[col] stored as FP32
//   EPI_BIAS_RELU: relu(D + bias[col]) stored as BF16 row-major and, if given, transposed
//                  (the transposed copy is the K-contiguous operand of the weight gradients)
// Out-of-range rows, columns and K are zero-filled by TMA and masked at the store, so any M, N,
// K work as long as the row pitches are multiples of 8 elements (16-byte TMA strides).
#include <cuda.h>
#include <cudaTypedefs.h>

#include "doa_internal.cuh"
#include "tc_common.cuh"

namespace doa {
namespace {

using namespace tc;

constexpr int kGmThreads = 128;
constexpr int kStages = 4;

__device__ __forceinline__ void tma_2d(uint32_t dst, const CUtensorMap *map, int x, int y, uint32_t mbar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
          dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(mbar)
      : "memory");
}
__device__ __forceinline__ void expect_tx(uint32_t mbar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(mbar), "r"(bytes) : "memory");
}

struct GemmArgs {
  int M, N, K, BN;
  int epi;
  const float *bias;
  void *D;              // FP32 or BF16 output
  int ldd;
  __nv_bfloat16 *DT;    // optional transposed BF16 output (N x M, ld lddt)
  int lddt;
  int *err;             // set to 1 if a bounded wait ran out
};

__global__ void __launch_bounds__(kGmThreads, 1) gemm_tc_kernel(const __grid_constant__ CUtensorMap amap,
                                                                const __grid_constant__ CUtensorMap bmap, GemmArgs g) {
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  uint8_t *sm = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  __shared__ __align__(8) uint64_t full_bar[kStages], empty_bar[kStages], done_bar;
  __shared__ uint32_t tmem_base;
  __shared__ int s_ok, s_issued, s_consumed;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int abytes = kTcRows * 128, bbytes = g.BN * 128;
  const int stage_bytes = abytes + (bbytes + 1023) / 1024 * 1024;
  const int m0 = blockIdx.x * kTcRows, n0 = blockIdx.y * g.BN;
  const int KT = (g.K + 63) / 64;
  int cols = 32;
  while (cols < g.BN) cols <<= 1;

  if (tid == 0) {
    for (int s = 0; s < kStages; ++s) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&full_bar[s])));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&empty_bar[s])));
    }
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&done_bar)));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    s_ok = 1;
    s_issued = 0;
    s_consumed = 0;
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                 "r"(cols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_base;

  if (warp == 0 && lane == 0) {
    // producer
    for (int kt = 0; kt < KT; ++kt) {
      const int s = kt % kStages;
      if (kt >= kStages && !mbar_wait(smem_u32(&empty_bar[s]), (uint32_t)(((kt / kStages) - 1) & 1))) {
        s_ok = 0;
        break;
      }
      uint8_t *st = sm + s * stage_bytes;
      expect_tx(smem_u32(&full_bar[s]), (uint32_t)(abytes + bbytes));
      tma_2d(smem_u32(st), &amap, kt * 64, m0, smem_u32(&full_bar[s]));
      tma_2d(smem_u32(st + abytes), &bmap, kt * 64, n0, smem_u32(&full_bar[s]));
      s_issued = kt + 1;
    }
  } else if (warp == 1 && lane == 0) {
    // MMA issuer
    const uint32_t idesc = inst_desc(1, g.BN);
    for (int kt = 0; kt < KT; ++kt) {
      const int s = kt % kStages;
      if (!mbar_wait(smem_u32(&full_bar[s]), (uint32_t)((kt / kStages) & 1))) {
        s_ok = 0;
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t pa = smem_u32(sm + s * stage_bytes), pb = pa + abytes;
      for (int kk = 0; kk < 4; ++kk)
        mma(tmem, smem_desc(pa + kk * 32), smem_desc(pb + kk * 32), idesc, (kt > 0 || kk > 0) ? 1u : 0u);
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                       smem_u32(&empty_bar[s]))
                   : "memory");
      s_consumed = kt + 1;
    }
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                     smem_u32(&done_bar))
                 : "memory");
  }
  // epilogue
  bool ok = mbar_wait(smem_u32(&done_bar), 0u);
  ok = __syncthreads_and(ok && s_ok) != 0;
  if (!ok && tid == 0) {
    if (g.err) atomicExch(g.err, 1);
    // let the copies still in flight land before the CTA exits (bounded waits)
    for (int kt = s_consumed; kt < s_issued; ++kt)
      mbar_wait(smem_u32(&full_bar[kt % kStages]), (uint32_t)((kt / kStages) & 1));
  }
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const int row = m0 + warp * 32 + lane;
  if (ok) {
    for (int c0 = 0; c0 < g.BN; c0 += 8) {
      float v[8];
      tmem_ld8(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, v);
      const int col0 = n0 + c0;
      if (g.epi != 0 && g.bias) {
#pragma unroll
        for (int j = 0; j < 8; ++j)
          if (col0 + j < g.N) v[j] += g.bias[col0 + j];
      }
      if (g.epi == 2) {
#pragma unroll
        for (int j = 0; j < 8; ++j) v[j] = fmaxf(v[j], 0.f);
      }
      if (row < g.M) {
        if (g.epi == 2) {
          __nv_bfloat16 *D = reinterpret_cast<__nv_bfloat16 *>(g.D) + (size_t)row * g.ldd;
#pragma unroll
          for (int j = 0; j < 8; ++j)
            if (col0 + j < g.N) D[col0 + j] = __float2bfloat16_rn(v[j]);
          if (g.DT) {
#pragma unroll
            for (int j = 0; j < 8; ++j)
              if (col0 + j < g.N) g.DT[(size_t)(col0 + j) * g.lddt + row] = __float2bfloat16_rn(v[j]);
          }
        } else {
          float *D = reinterpret_cast<float *>(g.D) + (size_t)row * g.ldd;
#pragma unroll
          for (int j = 0; j < 8; ++j)
            if (col0 + j < g.N) D[col0 + j] = v[j];
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(cols));
}

PFN_cuTensorMapEncodeTiled_v12000 g_encode_g = nullptr;

cudaError_t encode_bf16(CUtensorMap *map, const void *base, int rows, int cols, int ld, int box_rows) {
  if (!g_encode_g) {
    cudaDriverEntryPointQueryResult q;
    void *fn = nullptr;
    cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q);
    if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !fn) return cudaErrorNotSupported;
    g_encode_g = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
  }
  cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)ld * 2};
  cuuint32_t box[2] = {64, (cuuint32_t)box_rows};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = g_encode_g(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void *>(base), dims, strides, box, estr,
                          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                          CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

}  // namespace

// D = A B^T with A (M x K, ld lda) and B (N x K, ld ldb) BF16, K contiguous.
cudaError_t launch_gemm_tc(const __nv_bfloat16 *A, int lda, const __nv_bfloat16 *B, int ldb, int M, int N, int K,
                           int epi, const float *bias, void *D, int ldd, __nv_bfloat16 *DT, int lddt, int *err,
                           cudaStream_t s) {
  const int BN = N >= 256 ? 256 : (N + 15) / 16 * 16;
  CUtensorMap amap, bmap;
  cudaError_t e = encode_bf16(&amap, A, M, K, lda, kTcRows);
  if (e != cudaSuccess) return e;
  if ((e = encode_bf16(&bmap, B, N, K, ldb, BN)) != cudaSuccess) return e;
  const int stage = kTcRows * 128 + (BN * 128 + 1023) / 1024 * 1024;
  const int smem = kStages * stage + 1024;
  if ((e = cudaFuncSetAttribute(gemm_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem)) != cudaSuccess)
    return e;
  GemmArgs g{M, N, K, BN, epi, bias, D, ldd, DT, lddt, err};
  dim3 grid((M + kTcRows - 1) / kTcRows, (N + BN - 1) / BN);
  gemm_tc_kernel<<<grid, kGmThreads, smem, s>>>(amap, bmap, g);
  return cudaGetLastError();
}

}  // namespace doa
