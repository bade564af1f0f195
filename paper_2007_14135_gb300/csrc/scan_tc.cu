// Step-5 on the 5th-generation tensor cores (tcgen05): the pseudospectrum as a real GEMM of the
// generated steering block against the real embedding of the noise factor B, with FP32
// accumulation in tensor memory (TMEM) and a per-row norm in the epilogue.
//
// Real embedding: a steering row [Re a_0, Im a_0, ..., Re a_{M-1}, Im a_{M-1}] (K-dim 2M) times
// W (2M x 2K) with W[2m][2k] = Re b_mk, W[2m+1][2k] = Im b_mk, W[2m][2k+1] = -Im b_mk,
// W[2m+1][2k+1] = Re b_mk gives [Re y_0, Im y_0, ...] with y = B^H a, so den = sum of squares of
// the row. One tile = 128 grid points (UMMA M = 128); N = 2K rounded up to 32; K-dim = 2M
// rounded up to 64 (whole 128-byte swizzle atoms; the padding of W is zero).
//
// Operand precision (doa_prec):
//   BF16   : one product A_hi W_hi (8-bit significands; shows why splitting is needed)
//   BF16X3 : A = A_hi + A_lo, W = W_hi + W_lo in BF16; A_hi W_hi + A_hi W_lo + A_lo W_hi
//   FP16X3 : the same in FP16 with the lo parts scaled by 2^11 (kept normal) and accumulated in
//            a second TMEM accumulator that the epilogue scales back by 2^-11
// For the split forms, accuracy near the spectral nulls is won back: every point whose tensor
// denominator falls below c_prec * sum_k ||b_k||^2 (c from the split's per-term error, target
// 1e-3 relative) is re-evaluated by a whole warp in FP32 (exact integer phases), and those
// still below the FP32 threshold in FP64, exactly as the FP32 path does.
//
// Structure: one persistent CTA of 512 threads per SM. Four threads generate the phasors of
// one grid point (exact 32-bit integer phases, phasor_q32), split them into hi/lo and store
// them straight into the 128B-swizzled K-major shared-memory layout the tensor core reads;
// one thread issues the MMAs and commits to an mbarrier (bounded wait); the 16 warps read the
// accumulator back with tcgen05.ld (warp w: TMEM lanes 32(w%4).., column slice w/4).
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <float.h>

#include "doa_internal.cuh"
#include "tc_common.cuh"

namespace doa {
namespace {

using namespace tc;
constexpr int kTcThreads = 512;   // 4 threads per point
constexpr int kTcWarps = kTcThreads / 32;

struct TcLayout {
  int MP;      // M rounded up to 16
  int KD;      // K-dim (bf16 elements per row): 2*MP rounded up to 64
  int N;       // 2K rounded up to 32
  int atoms;   // KD / 64
  int tmem_cols;
  // byte offsets in the 1024-aligned dynamic shared memory
  int off_whi, off_wlo, off_ahi, off_alo, off_b32, off_ph, off_red, total;
};

__host__ __device__ inline TcLayout tc_layout(int M, int K, int prec) {
  TcLayout t;
  t.MP = (M + 15) / 16 * 16;
  t.KD = (2 * t.MP + 63) / 64 * 64;
  t.N = (2 * K + 31) / 32 * 32;
  t.atoms = t.KD / 64;
  int cols = prec == DOA_FP16X3 ? 2 * t.N : t.N;
  int p2 = 32;
  while (p2 < cols) p2 <<= 1;
  t.tmem_cols = p2;
  const int wbytes = t.atoms * t.N * 128, abytes = t.atoms * kTcRows * 128;
  t.off_whi = 0;
  t.off_wlo = t.off_whi + wbytes;
  t.off_ahi = t.off_wlo + wbytes;
  t.off_alo = t.off_ahi + abytes;
  t.off_b32 = t.off_alo + abytes;
  t.off_ph = t.off_b32 + ((K * t.MP * 8 + 15) / 16) * 16;
  t.off_red = t.off_ph + kTcWarps * kMaxM * 16;
  t.total = t.off_red + kTcRows * 4 * 4 + 1024;
  return t;
}

struct TcArgs {
  const double2 *B;     // FP64 factor, column-major, ld M
  int M, K, L, prec;
  double lo, step;
  const uint32_t *S;    // phase table (may alias P)
  float *P;
};

// FP32 re-evaluation of point k by one warp (phasors m = lane, lane+32; columns col = lane, lane+32).
__device__ float den32_warp(const float2 *B32, int MP, int M, int K, uint32_t Sk, float2 *ph) {
  const int lane = threadIdx.x & 31;
  for (int m = lane; m < M; m += 32) ph[m] = phasor_q32((uint32_t)m * Sk);
  __syncwarp();
  float den = 0.f;
  for (int col = lane; col < K; col += 32) {
    float yr = 0.f, yi = 0.f;
    const float2 *b = B32 + col * MP;
    for (int m = 0; m < M; ++m) {
      const float2 bb = b[m], a = ph[m];
      yr = fmaf(bb.x, a.x, fmaf(bb.y, a.y, yr));
      yi = fmaf(bb.x, a.y, fmaf(-bb.y, a.x, yi));
    }
    den = fmaf(yr, yr, fmaf(yi, yi, den));
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) den += __shfl_xor_sync(0xffffffffu, den, off);
  __syncwarp();
  return den;
}

// FP64 re-evaluation of point k by one warp, from the grid angle.
__device__ double den64_warp(const TcArgs &a, int k, double2 *ph) {
  const int lane = threadIdx.x & 31;
  const double theta = __dadd_rn(a.lo, __dmul_rn((double)k, a.step));
  const double s = sin(theta * 0.017453292519943295);
  for (int m = lane; m < a.M; m += 32) {
    double sn, cs;
    sincospi((double)m * s, &sn, &cs);
    ph[m] = make_double2(cs, sn);
  }
  __syncwarp();
  double den = 0.0;
  for (int col = lane; col < a.K; col += 32) {
    double yr = 0.0, yi = 0.0;
    const double2 *b = a.B + (size_t)col * a.M;
    for (int m = 0; m < a.M; ++m) {
      const double2 bb = b[m], p = ph[m];
      yr = fma(bb.x, p.x, fma(bb.y, p.y, yr));
      yi = fma(bb.x, p.y, fma(-bb.y, p.x, yi));
    }
    den = fma(yr, yr, fma(yi, yi, den));
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) den += __shfl_xor_sync(0xffffffffu, den, off);
  __syncwarp();
  return den;
}

__global__ void __launch_bounds__(kTcThreads, 1) scan_tc_kernel(TcArgs a, int ntiles) {
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  uint8_t *sm = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  __shared__ __align__(8) uint64_t mbar;
  __shared__ uint32_t tmem_base;
  __shared__ float s_scale2, s_thr_tc, s_thr32;
  __shared__ int s_flags[kTcRows];
  __shared__ uint32_t s_sk[kTcRows];
  __shared__ int s_nflag;
  __shared__ float s_red_max, s_red_e, s_red_n2;

  const TcLayout lay = tc_layout(a.M, a.K, a.prec);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  uint8_t *whi = sm + lay.off_whi, *wlo = sm + lay.off_wlo, *ahi = sm + lay.off_ahi, *alo = sm + lay.off_alo;
  float2 *B32 = reinterpret_cast<float2 *>(sm + lay.off_b32);
  float *red = reinterpret_cast<float *>(sm + lay.off_red);
  double2 *ph64 = reinterpret_cast<double2 *>(sm + lay.off_ph) + warp * kMaxM;
  float2 *ph32 = reinterpret_cast<float2 *>(ph64);

  // ---- factor: FP32 copy, max |component|, E = sum_k (sum_m |b|)^2 and sum ||b_k||^2
  if (tid == 0) {
    s_red_max = 0.f;
    s_red_e = 0.f;
    s_red_n2 = 0.f;
    s_nflag = 0;
  }
  __syncthreads();
  float mx = 0.f;
  for (int e = tid; e < a.K * lay.MP; e += kTcThreads) {
    int k = e / lay.MP, m = e % lay.MP;
    float2 v = make_float2(0.f, 0.f);
    if (m < a.M) {
      double2 b = a.B[(size_t)k * a.M + m];
      v = make_float2((float)b.x, (float)b.y);
    }
    B32[e] = v;
    mx = fmaxf(mx, fmaxf(fabsf(v.x), fabsf(v.y)));
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, off));
  if (lane == 0) atomicMax(reinterpret_cast<int *>(&s_red_max), __float_as_int(mx));
  __syncthreads();
  if (warp == 0) {
    float e = 0.f, n2 = 0.f;
    for (int k = lane; k < a.K; k += 32) {
      float n1 = 0.f, q = 0.f;
      for (int m = 0; m < a.M; ++m) {
        float2 b = B32[k * lay.MP + m];
        q += b.x * b.x + b.y * b.y;
        n1 += sqrtf(b.x * b.x + b.y * b.y);
      }
      e += n1 * n1;
      n2 += q;
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
      e += __shfl_xor_sync(0xffffffffu, e, off);
      n2 += __shfl_xor_sync(0xffffffffu, n2, off);
    }
    if (lane == 0) {
      s_red_e = e;
      s_red_n2 = n2;
    }
  }
  __syncthreads();
  // scale W by 2^-e so its entries are at most 1; den_true = den_scaled * 2^(2e)
  int ex = 0;
  frexpf(fmaxf(s_red_max, FLT_MIN), &ex);
  const float wscale = ldexpf(1.f, -ex);
  if (tid == 0) {
    s_scale2 = ldexpf(1.f, 2 * ex);
    // per-term relative error of the split product: BF16x3 ~ 8e-6 (16 significant bits),
    // FP16x3 ~ 1e-6 (22 bits); both set so the unrefined points stay within ~1e-3 relative
    const float gam = a.prec == DOA_FP16X3 ? 1.0e-6f : 8.0e-6f;
    const float c = (2.8f * gam / 1.0e-3f);
    s_thr_tc = a.prec == DOA_BF16 ? 0.f : c * c * s_red_n2;
    s_thr32 = 3.7e-6f * s_red_e;
  }
  // ---- W = real embedding of B (B operand, N rows x KD, K-major, 128B swizzle), hi and lo
  for (int e = tid; e < lay.N * lay.KD; e += kTcThreads) {
    const int n = e / lay.KD, kap = e % lay.KD;
    const int col = n >> 1, m = kap >> 1;
    float w = 0.f;
    if (col < a.K && m < a.M) {
      const float2 b = B32[col * lay.MP + m];
      const bool re_out = (n & 1) == 0, re_in = (kap & 1) == 0;
      w = re_out ? (re_in ? b.x : b.y) : (re_in ? -b.y : b.x);
      w *= wscale;
    }
    uint16_t h, l;
    split16(w, a.prec, h, l);
    const uint32_t off = (uint32_t)(kap >> 6) * lay.N * 128 + sw128(n, kap & 63);
    *reinterpret_cast<uint16_t *>(whi + off) = h;
    *reinterpret_cast<uint16_t *>(wlo + off) = l;
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar)));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                 "r"(lay.tmem_cols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_base;
  const int fmt = a.prec == DOA_FP16X3 ? 0 : 1;
  const uint32_t idesc = inst_desc(fmt, lay.N);
  const float thr_tc = s_thr_tc, thr32 = s_thr32, scale2 = s_scale2;
  const int pt = tid >> 2, part = tid & 3;        // point within the tile, quarter of its elements
  const int q = warp & 3, cs = warp >> 2;         // TMEM lane quarter, column slice (epilogue)
  const int ncs = lay.N / 4;                      // columns per slice (multiple of 8)
  bool ok = true;
  uint32_t iter = 0;

  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++iter) {
    const int k0 = tile * kTcRows;
    // ---- steering block: row pt, elements m in [part*MP/4, (part+1)*MP/4), 4 per 16-byte chunk
    {
      const int k = k0 + pt;
      const uint32_t Sk = k < a.L ? a.S[k] : 0u;
      if (part == 0) s_sk[pt] = Sk;   // P (which may hold S) is overwritten below
      const int mq = lay.MP / 4;
      const int m0 = part * mq;
      uint32_t phi = (uint32_t)m0 * Sk;
      for (int c = 0; c < mq; c += 4) {
        uint16_t hs[8], ls[8];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const float2 v = phasor_q32(phi);
          phi += Sk;
          split16(v.x, a.prec, hs[2 * j], ls[2 * j]);
          split16(v.y, a.prec, hs[2 * j + 1], ls[2 * j + 1]);
        }
        const int kap = 2 * (m0 + c);   // first K index of this 8-element chunk
        const uint32_t off = (uint32_t)(kap >> 6) * kTcRows * 128 + sw128(pt, kap & 63);
        uint4 vh, vl;
        vh.x = hs[0] | ((uint32_t)hs[1] << 16);
        vh.y = hs[2] | ((uint32_t)hs[3] << 16);
        vh.z = hs[4] | ((uint32_t)hs[5] << 16);
        vh.w = hs[6] | ((uint32_t)hs[7] << 16);
        vl.x = ls[0] | ((uint32_t)ls[1] << 16);
        vl.y = ls[2] | ((uint32_t)ls[3] << 16);
        vl.z = ls[4] | ((uint32_t)ls[5] << 16);
        vl.w = ls[6] | ((uint32_t)ls[7] << 16);
        *reinterpret_cast<uint4 *>(ahi + off) = vh;
        *reinterpret_cast<uint4 *>(alo + off) = vl;
      }
      // K padding beyond 2*MP (only when 2*MP is not a multiple of 64): zero chunks
      for (int kap = 2 * lay.MP + part * 8; kap < lay.KD; kap += 32) {
        const uint32_t off = (uint32_t)(kap >> 6) * kTcRows * 128 + sw128(pt, kap & 63);
        *reinterpret_cast<uint4 *>(ahi + off) = make_uint4(0, 0, 0, 0);
        *reinterpret_cast<uint4 *>(alo + off) = make_uint4(0, 0, 0, 0);
      }
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    // ---- MMAs (one thread)
    if (tid == 0 && ok) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t b_ahi = smem_u32(ahi), b_alo = smem_u32(alo), b_whi = smem_u32(whi), b_wlo = smem_u32(wlo);
      const int ksteps = lay.KD / 16;
      for (int kk = 0; kk < ksteps; ++kk) {
        const uint32_t offa = (uint32_t)(kk >> 2) * kTcRows * 128 + (kk & 3) * 32;
        const uint32_t offw = (uint32_t)(kk >> 2) * lay.N * 128 + (kk & 3) * 32;
        const uint32_t acc = kk > 0 ? 1u : 0u;
        mma(tmem, smem_desc(b_ahi + offa), smem_desc(b_whi + offw), idesc, acc);
        if (a.prec == DOA_BF16X3) {
          mma(tmem, smem_desc(b_ahi + offa), smem_desc(b_wlo + offw), idesc, 1u);
          mma(tmem, smem_desc(b_alo + offa), smem_desc(b_whi + offw), idesc, 1u);
        } else if (a.prec == DOA_FP16X3) {
          mma(tmem + lay.N, smem_desc(b_ahi + offa), smem_desc(b_wlo + offw), idesc, acc);
          mma(tmem + lay.N, smem_desc(b_alo + offa), smem_desc(b_whi + offw), idesc, 1u);
        }
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                       smem_u32(&mbar))
                   : "memory");
    }
    const bool done = ok && mbar_wait(smem_u32(&mbar), iter & 1u);
    ok = __syncthreads_and(done);
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    // ---- epilogue: den of each row from its column slice
    const int row = q * 32 + lane;
    float part_den = 0.f;
    if (ok) {
      for (int c0 = cs * ncs; c0 < (cs + 1) * ncs; c0 += 8) {
        float v[8];
        tmem_ld8(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)c0, v);
        if (a.prec == DOA_FP16X3) {
          float w[8];
          tmem_ld8(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(lay.N + c0), w);
#pragma unroll
          for (int j = 0; j < 8; ++j) v[j] = fmaf(w[j], 4.8828125e-4f, v[j]);
        }
#pragma unroll
        for (int j = 0; j < 8; ++j) part_den = fmaf(v[j], v[j], part_den);
      }
    }
    red[row * 4 + cs] = part_den;
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (tid < kTcRows) {
      const int k = k0 + tid;
      if (k < a.L) {
        const float den = (red[tid * 4] + red[tid * 4 + 1] + red[tid * 4 + 2] + red[tid * 4 + 3]);
        if (!ok) {
          a.P[k] = __int_as_float(0x7fc00000);   // timed-out tile: NaN marks it
        } else {
          a.P[k] = 1.0f / fmaxf(den * scale2, FLT_MIN);
          if (den * scale2 < thr_tc) {
            int pos = atomicAdd(&s_nflag, 1);
            s_flags[pos] = k;
          }
        }
      }
    }
    __syncthreads();
    // ---- null-adaptive refinement: FP32 warp re-evaluation, then FP64 below the FP32 threshold
    const int nf = s_nflag;
    for (int i = warp; i < nf; i += kTcWarps) {
      const int k = s_flags[i];
      const float d32 = den32_warp(B32, lay.MP, a.M, a.K, s_sk[k - k0], ph32);
      if (d32 < thr32) {
        const double d64 = den64_warp(a, k, ph64);
        if (lane == 0) a.P[k] = (float)(1.0 / fmax(d64, (double)FLT_MIN));
      } else if (lane == 0) {
        a.P[k] = 1.0f / fmaxf(d32, FLT_MIN);
      }
    }
    __syncthreads();
    if (tid == 0) s_nflag = 0;
    __syncthreads();
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(lay.tmem_cols));
}

}  // namespace

cudaError_t launch_scan_tc_single(const double2 *B, int M, int K, int L, double lo, double step, int prec,
                                  const uint32_t *S, float *P, cudaStream_t s) {
  const TcLayout lay = tc_layout(M, K, prec);
  cudaError_t e = cudaFuncSetAttribute(scan_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, lay.total);
  if (e != cudaSuccess) return e;
  const int sms = device_sm_count();
  const int ntiles = (L + kTcRows - 1) / kTcRows;
  const int grid = ntiles < sms ? ntiles : sms;
  TcArgs a{B, M, K, L, prec, lo, step, S, P};
  scan_tc_kernel<<<grid, kTcThreads, lay.total, s>>>(a, ntiles);
  return cudaGetLastError();
}

}  // namespace doa
