// Step-1 (Sec. 3.1, Eq. 3) on the tensor cores, fed by TMA: R = X X^H / N as one real GEMM.
//
// With Y = X viewed as M x 2N reals (each snapshot's (re, im) pair adjacent, exactly the complex64
// bytes in HBM) and Z the same rows with every pair mapped (re, im) -> (im, -re),
//     [Y; Z] Y^T = [Re(X X^H); Im(X X^H)],
// so a UMMA with M = 128 rows ([Y; Z], 2M <= 128, zero rows below) and N = M (rounded up to 16)
// columns produces the whole covariance in TMEM.
//
// Per CTA: TMA (cp.async.bulk.tensor, FP32, no swizzle) brings 32 snapshots of all M rows
// (M x 64 floats) into a two-stage staging ring guarded by mbarriers; all threads split the FP32
// values into hi/lo 16-bit parts (BF16, or FP16 with the lo part scaled by 2^11) and write the
// three operand views (Y and Z rows of A, Y rows of B) in the 128B-swizzled K-major layout; one
// thread issues the MMAs (one product for DOA_BF16, hi*hi + hi*lo + lo*hi for the x3 forms, the
// FP16 cross terms into a second accumulator) and commits them to an mbarrier that releases the
// operand buffer two stages later. A cluster of up to 8 CTAs splits the snapshots; each CTA reads
// its accumulator with tcgen05.ld into shared memory and CTA rank 0 adds the partials in FP64
// through distributed shared memory, keeps the upper triangle and mirrors it (Hermitian).
// Accuracy: the split forms carry ~16 (BF16x3) or ~22 (FP16x3) significant bits per operand and
// accumulate in FP32; this is the reduced-precision covariance of the large-array configuration.
#include <cooperative_groups.h>
#include <cuda.h>
#include <cudaTypedefs.h>

#include "doa_internal.cuh"
#include "tc_common.cuh"

namespace cg = cooperative_groups;

namespace doa {
namespace {

using namespace tc;

constexpr int kCtThreads = 128;
constexpr int kCtCluster = 8;
constexpr int kAtomSnap = 32;   // snapshots per K atom (64 reals = one 128-byte swizzle row)

struct CtLayout {
  int NP;        // N dimension of the MMA: M rounded up to 16
  int tmem_cols;
  int stage_bytes;                          // M x 64 floats
  int off_stage[2], off_ahi[2], off_alo[2], off_bhi[2], off_blo[2], total;
};

__host__ __device__ inline CtLayout ct_layout(int M, int prec) {
  CtLayout t;
  t.NP = (M + 15) / 16 * 16;
  const int cols = prec == DOA_FP16X3 ? 2 * t.NP : t.NP;
  int p2 = 32;
  while (p2 < cols) p2 <<= 1;
  t.tmem_cols = p2;
  t.stage_bytes = M * 64 * 4;
  const int abytes = kTcRows * 128, bbytes = t.NP * 128;
  int at = 0;
  for (int s = 0; s < 2; ++s) {
    t.off_ahi[s] = at;
    at += abytes;
    t.off_alo[s] = at;
    at += abytes;
  }
  for (int s = 0; s < 2; ++s) {       // B blocks are multiples of 2 KB; keep 1 KB alignment
    t.off_bhi[s] = at;
    at += (bbytes + 1023) / 1024 * 1024;
    t.off_blo[s] = at;
    at += (bbytes + 1023) / 1024 * 1024;
  }
  for (int s = 0; s < 2; ++s) {
    t.off_stage[s] = at;
    at += (t.stage_bytes + 1023) / 1024 * 1024;
  }
  const int part = kTcRows * t.NP * 4;   // FP32 partial of R, aliases the operand buffers
  t.total = (at > part ? at : part) + 1024;
  return t;
}

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap *map, int x, int y, uint32_t mbar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
          dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(mbar)
      : "memory");
}
__device__ __forceinline__ void mbar_expect(uint32_t mbar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(mbar), "r"(bytes) : "memory");
}

__global__ void __launch_bounds__(kCtThreads, 1) covariance_tc_kernel(const __grid_constant__ CUtensorMap xmap,
                                                                      int M, int N, int prec, int per_cta,
                                                                      float2 *R, double2 *R64) {
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  uint8_t *sm = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  __shared__ __align__(8) uint64_t full_bar[2], mma_bar[2];
  __shared__ uint32_t tmem_base;
  __shared__ int s_ok;
  cg::cluster_group cluster = cg::this_cluster();
  const int rank = (int)cluster.block_rank(), nranks = (int)cluster.num_blocks();
  const CtLayout lay = ct_layout(M, prec);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int atoms_total = (N + kAtomSnap - 1) / kAtomSnap;
  const int a0 = rank * per_cta, a1 = min(atoms_total, a0 + per_cta);
  const int natoms = max(0, a1 - a0);

  // zero both operand buffers once (padding rows 2M..127 of A, M..NP-1 of B stay zero)
  for (int e = tid * 16; e < lay.off_stage[0]; e += kCtThreads * 16)
    *reinterpret_cast<uint4 *>(sm + e) = make_uint4(0, 0, 0, 0);
  if (tid == 0) {
    for (int s = 0; s < 2; ++s) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&full_bar[s])));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mma_bar[s])));
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    s_ok = 1;
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                 "r"(lay.tmem_cols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_base;
  const uint32_t idesc = inst_desc(prec == DOA_FP16X3 ? 0 : 1, lay.NP);
  const bool split = prec != DOA_BF16;

  // prologue: the first two atoms in flight (issued / consumed: bookkeeping of thread 0)
  int issued = 0, consumed = 0;
  if (tid == 0)
    for (int s = 0; s < 2 && s < natoms; ++s, ++issued) {
      mbar_expect(smem_u32(&full_bar[s]), (uint32_t)lay.stage_bytes);
      tma_load_2d(smem_u32(sm + lay.off_stage[s]), &xmap, (a0 + s) * 2 * kAtomSnap, 0, smem_u32(&full_bar[s]));
    }
  bool ok = true;
  for (int i = 0; i < natoms; ++i) {
    const int s = i & 1;
    // the operand buffer s was last read by the MMAs of atom i - 2
    bool good = ok;
    if (good && i >= 2) good = mbar_wait(smem_u32(&mma_bar[s]), (uint32_t)(((i - 2) >> 1) & 1));
    if (good) good = mbar_wait(smem_u32(&full_bar[s]), (uint32_t)((i >> 1) & 1));
    ok = __syncthreads_and(good);
    if (!ok) break;
    consumed = i + 1;
    // split the staged FP32 atom (M rows x 32 complex) into the three operand views
    const float *stg = reinterpret_cast<const float *>(sm + lay.off_stage[s]);
    uint8_t *ahi = sm + lay.off_ahi[s], *alo = sm + lay.off_alo[s];
    uint8_t *bhi = sm + lay.off_bhi[s], *blo = sm + lay.off_blo[s];
    for (int task = tid; task < M * 8; task += kCtThreads) {
      const int r = task >> 3, ch = task & 7;        // row, chunk of 4 complex (8 reals)
      const float4 u = *reinterpret_cast<const float4 *>(stg + r * 64 + ch * 8);
      const float4 v = *reinterpret_cast<const float4 *>(stg + r * 64 + ch * 8 + 4);
      const float y[8] = {u.x, u.y, u.z, u.w, v.x, v.y, v.z, v.w};
      const float z[8] = {u.y, -u.x, u.w, -u.z, v.y, -v.x, v.w, -v.z};   // (re, im) -> (im, -re)
      uint16_t yh[8], yl[8], zh[8], zl[8];
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        split16(y[j], prec, yh[j], yl[j]);
        split16(z[j], prec, zh[j], zl[j]);
      }
      auto pack = [](const uint16_t (&h)[8]) {
        return make_uint4(h[0] | ((uint32_t)h[1] << 16), h[2] | ((uint32_t)h[3] << 16), h[4] | ((uint32_t)h[5] << 16),
                          h[6] | ((uint32_t)h[7] << 16));
      };
      const uint32_t offy = sw128(r, ch * 8), offz = sw128(M + r, ch * 8);
      *reinterpret_cast<uint4 *>(ahi + offy) = pack(yh);
      *reinterpret_cast<uint4 *>(ahi + offz) = pack(zh);
      *reinterpret_cast<uint4 *>(bhi + offy) = pack(yh);
      if (split) {
        *reinterpret_cast<uint4 *>(alo + offy) = pack(yl);
        *reinterpret_cast<uint4 *>(alo + offz) = pack(zl);
        *reinterpret_cast<uint4 *>(blo + offy) = pack(yl);
      }
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    if (tid == 0) {
      // staging slot s is free again: fetch atom i + 2
      if (i + 2 < natoms) {
        mbar_expect(smem_u32(&full_bar[s]), (uint32_t)lay.stage_bytes);
        tma_load_2d(smem_u32(sm + lay.off_stage[s]), &xmap, (a0 + i + 2) * 2 * kAtomSnap, 0, smem_u32(&full_bar[s]));
        ++issued;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t pa = smem_u32(ahi), pal = smem_u32(alo), pb = smem_u32(bhi), pbl = smem_u32(blo);
      for (int kk = 0; kk < 4; ++kk) {
        const uint32_t off = kk * 32;
        const uint32_t acc = (i > 0 || kk > 0) ? 1u : 0u;
        mma(tmem, smem_desc(pa + off), smem_desc(pb + off), idesc, acc);
        if (prec == DOA_BF16X3) {
          mma(tmem, smem_desc(pa + off), smem_desc(pbl + off), idesc, 1u);
          mma(tmem, smem_desc(pal + off), smem_desc(pb + off), idesc, 1u);
        } else if (prec == DOA_FP16X3) {
          mma(tmem + lay.NP, smem_desc(pa + off), smem_desc(pbl + off), idesc, acc);
          mma(tmem + lay.NP, smem_desc(pal + off), smem_desc(pb + off), idesc, 1u);
        }
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                       smem_u32(&mma_bar[s]))
                   : "memory");
    }
  }
  // after a timed-out wait, let the copies still in flight land before the CTA exits (bounded)
  if (!ok && tid == 0)
    for (int a = consumed; a < issued; ++a) mbar_wait(smem_u32(&full_bar[a & 1]), (uint32_t)((a >> 1) & 1));
  // drain: the last commit covers every earlier MMA of this thread
  if (natoms > 0 && ok) {
    const int il = natoms - 1;
    ok = mbar_wait(smem_u32(&mma_bar[il & 1]), (uint32_t)((il >> 1) & 1));
  }
  ok = __syncthreads_and(ok);
  if (tid == 0 && !ok) s_ok = 0;
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  // accumulator -> FP32 partial [128 rows][NP] in shared memory (aliases the operand buffers)
  float *part = reinterpret_cast<float *>(sm);
  const int row = warp * 32 + lane;
  for (int c0 = 0; c0 < lay.NP; c0 += 8) {
    float v[8];
    if (natoms > 0 && ok) {
      tmem_ld8(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, v);
      if (prec == DOA_FP16X3) {
        float w[8];
        tmem_ld8(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(lay.NP + c0), w);
#pragma unroll
        for (int j = 0; j < 8; ++j) v[j] = fmaf(w[j], 4.8828125e-4f, v[j]);
      }
    } else {
#pragma unroll
      for (int j = 0; j < 8; ++j) v[j] = 0.f;
    }
#pragma unroll
    for (int j = 0; j < 8; ++j) part[row * lay.NP + c0 + j] = v[j];
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  cluster.sync();
  if (rank == 0) {
    const double inv_n = 1.0 / (double)N;
    bool all_ok = true;
    for (int r = 0; r < nranks; ++r) all_ok = all_ok && *cluster.map_shared_rank(&s_ok, r);
    for (int e = tid; e < M * M; e += kCtThreads) {
      const int a = e / M, b = e % M;
      if (a > b) continue;
      double re = 0.0, im = 0.0;
      for (int r = 0; r < nranks; ++r) {
        const float *rp = cluster.map_shared_rank(part, r);
        re += (double)rp[a * lay.NP + b];
        im += (double)rp[(M + a) * lay.NP + b];
      }
      re *= inv_n;
      im = a == b ? 0.0 : im * inv_n;
      if (!all_ok) re = im = __longlong_as_double(0x7ff8000000000000ll);   // timed out: NaN marks R
      if (R64) {
        R64[a * M + b] = make_double2(re, im);
        R64[b * M + a] = make_double2(re, -im);
      }
      if (R) {
        R[a * M + b] = make_float2((float)re, (float)im);
        R[b * M + a] = make_float2((float)re, (float)-im);
      }
    }
  }
  cluster.sync();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(lay.tmem_cols));
}

PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;

}  // namespace

cudaError_t launch_covariance_tc_single(const float2 *X, int M, int N, int ldx, int prec, float2 *R, double2 *R64,
                                        cudaStream_t s) {
  if (!g_encode) {
    cudaDriverEntryPointQueryResult q;
    void *fn = nullptr;
    cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q);
    if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !fn) return cudaErrorNotSupported;
    g_encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
  }
  // X as an (M rows) x (2N floats) FP32 matrix, row pitch ldx*8 bytes; box = 64 floats x M rows
  CUtensorMap map;
  cuuint64_t dims[2] = {(cuuint64_t)(2 * N), (cuuint64_t)M};
  cuuint64_t strides[1] = {(cuuint64_t)ldx * 8};
  cuuint32_t box[2] = {64, (cuuint32_t)M};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = g_encode(&map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float2 *>(X), dims, strides, box, estr,
                        CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return cudaErrorInvalidValue;
  const CtLayout lay = ct_layout(M, prec);
  cudaError_t e = cudaFuncSetAttribute(covariance_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, lay.total);
  if (e != cudaSuccess) return e;
  const int atoms = (N + kAtomSnap - 1) / kAtomSnap;
  const int nc = atoms < kCtCluster ? atoms : kCtCluster;
  const int per = (atoms + nc - 1) / nc;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(nc);
  cfg.blockDim = dim3(kCtThreads);
  cfg.dynamicSmemBytes = lay.total;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = nc;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, covariance_tc_kernel, map, M, N, prec, per, R, R64);
}

}  // namespace doa
