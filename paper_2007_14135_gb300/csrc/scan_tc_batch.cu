// Step-5 of the batch on the tensor cores (problems with doa_problem.prec = DOA_FP16X3 or
// DOA_BF16X3, M <= 32): the shared-contraction scan of scan_common.cuh (one steering block per
// tile of 128 grid points against the problem's whole factor F, readouts MUSIC / EV / PHD / MN)
// done as the real GEMM of scan_tc.cu:
//   A (128 x KD): rows = grid points, [Re a_0, Im a_0, Re a_1, ...] split into hi + lo halves;
//   W (N x KD):   real embedding of F (rows 2c, 2c+1 give Re y_c, Im y_c), scaled by a power of two
//                 so that its entries are at most 1, split into hi + lo;
//   D (128 x N) in TMEM, FP32: hi*hi (+ hi*lo + lo*hi; FP16: the cross terms, scaled by 2^11, in a
//   second accumulator).
// KD = 64 (2 M rounded up to one 128-byte swizzle atom), N = 2 Kf rounded up to 32.
//
// Per CTA (256 threads, two per grid point; two CTAs per SM while their TMEM fits): a software
// pipeline over consecutive tiles of one problem with two steering buffers and two accumulator
// sets — the threads write tile i+1's steering block into the swizzled K-major layout and one
// thread issues its MMAs (committed to that buffer's mbarrier, bounded wait) while the 8 warps
// read tile i's accumulator rows back (warp w: TMEM lanes 32 (w % 4).., half w / 4 of the
// columns) and form the readouts.
// Accuracy: a readout below c^2 sum_k w_k ||f_k||^2 (c from the split's per-term error, so that
// the others stay within 1e-3 relative) is re-evaluated by a warp in FP32 with exact integer
// phases, and where the FP32 value is below the FP32 path's threshold, in FP64
// (refine_point_warp), exactly as the CUDA-core scan does.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <float.h>

#include "doa_internal.cuh"
#include "scan_common.cuh"
#include "tc_common.cuh"

namespace doa {
namespace {

using namespace tc;
using namespace scanc;

constexpr int kTbThreads = 256;
constexpr int kTbWarps = kTbThreads / 32;
constexpr int kTbKD = 64;                          // K extent (one swizzle atom)
constexpr int kTbMaxCols = kTcBatchMaxM + 1;       // Kf <= M + 1
constexpr int kTbMaxN = (2 * kTbMaxCols + 31) / 32 * 32;
constexpr int kTbRun = 16;                         // consecutive tiles per run

// dynamic shared memory layout (bytes from a 1024-aligned base)
constexpr int kABytes = kTcRows * 128;                                 // one 128 x 64 16-bit operand
constexpr int kOffA = 0;                                                // [buffer][hi, lo]
constexpr int kOffWhi = kOffA + 4 * kABytes;
constexpr int kOffWlo = kOffWhi + kTbMaxN * 128;
constexpr int kOffB32 = kOffWlo + kTbMaxN * 128;                        // Kf x 32 float2
constexpr int kOffPh64 = kOffB32 + kTbMaxCols * kTcBatchMaxM * 8;        // per warp 32 double2
constexpr int kYbCols = kTbMaxCols + 1;
constexpr int kOffYb = kOffPh64 + kTbWarps * kTcBatchMaxM * 16;          // per warp kYbCols float2
constexpr int kOffPh32 = kOffYb + kTbWarps * kYbCols * 8;                // per warp 32 float2
constexpr int kOffRed = kOffPh32 + kTbWarps * kTcBatchMaxM * 8;          // 128 x 2 float4
constexpr int kTbSmem = kOffRed + kTcRows * 2 * 16 + 1024;
static_assert(2 * (kTbSmem + 2048) <= 228 * 1024, "two CTAs per SM");

struct TbShared {
  uint64_t mbar[2];
  uint32_t tmem;
  int nflag;
  int flags[kTcRows];
  uint32_t sk[2 * kTcRows];
  float w32[kTcBatchMaxM];
  float thr32[4], thrtc[4];
  float scale2;
  int maxbits;
};

// FP32 re-evaluation of all readouts of one point by a warp (lanes: phasors, then columns).
__device__ __forceinline__ void readouts32_warp(const float2 *B32, int MPs, int M, const ScanJob &j, const float *w32,
                                                uint32_t Sk, float2 *ph, float (&d)[4]) {
  const int lane = threadIdx.x & 31;
  for (int m = lane; m < M; m += 32) ph[m] = phasor_q32((uint32_t)m * Sk);
  __syncwarp();
  float dm = 0.f, de = 0.f, dp = 0.f, dn = 0.f;
  for (int col = lane; col < j.Kf; col += 32) {
    float yr = 0.f, yi = 0.f;
    const float2 *b = B32 + col * MPs;
    for (int m = 0; m < M; ++m) {
      const float2 bb = b[m], a = ph[m];
      yr = fmaf(bb.x, a.x, fmaf(bb.y, a.y, yr));
      yi = fmaf(bb.x, a.y, fmaf(-bb.y, a.x, yi));
    }
    const float n = fmaf(yr, yr, yi * yi);
    if (col < j.Kn) {
      dm += n;
      de = fmaf(w32[col], n, de);
    }
    if (col == j.kphd) dp = n;
    if (col == j.kmn) dn = n;
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    dm += __shfl_xor_sync(0xffffffffu, dm, off);
    de += __shfl_xor_sync(0xffffffffu, de, off);
    dp += __shfl_xor_sync(0xffffffffu, dp, off);
    dn += __shfl_xor_sync(0xffffffffu, dn, off);
  }
  d[kRoPhd] = dp;
  d[kRoMusic] = dm;
  d[kRoEv] = de;
  d[kRoMn] = dn;
  __syncwarp();
}

__global__ void __launch_bounds__(kTbThreads, 2) scan_tc_batch_kernel(const uint8_t *plan, uint8_t *ws, int *status) {
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  uint8_t *sm = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  __shared__ TbShared sh;
  const PlanHeader *h = reinterpret_cast<const PlanHeader *>(plan);
  const int nunits = h->tc_jobs;
  const int64_t ntiles = h->tc_tiles;
  const int32_t *list = reinterpret_cast<const int32_t *>(plan + h->off_tc);
  const PlanProblem *probs = reinterpret_cast<const PlanProblem *>(plan + h->off_prob);
  const PlanGrid *grids = reinterpret_cast<const PlanGrid *>(plan + h->off_grid);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  uint8_t *whi = sm + kOffWhi, *wlo = sm + kOffWlo;
  float2 *B32 = reinterpret_cast<float2 *>(sm + kOffB32);
  double2 *ph64 = reinterpret_cast<double2 *>(sm + kOffPh64) + warp * kTcBatchMaxM;
  float2 *yb = reinterpret_cast<float2 *>(sm + kOffYb) + warp * kYbCols;
  float2 *ph32 = reinterpret_cast<float2 *>(sm + kOffPh32) + warp * kTcBatchMaxM;
  float4 *red = reinterpret_cast<float4 *>(sm + kOffRed);
  auto a_hi = [&](int b) { return sm + kOffA + (2 * b) * kABytes; };
  auto a_lo = [&](int b) { return sm + kOffA + (2 * b + 1) * kABytes; };

  if (tid == 0) {
    for (int b = 0; b < 2; ++b) asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&sh.mbar[b])));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    sh.nflag = 0;
  }
  const int cols = h->tc_cols;
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&sh.tmem)),
                 "r"(cols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = sh.tmem;

  bool ok = true;
  uint32_t phase[2] = {0u, 0u};   // next parity to wait for, per mbarrier
  int pending = -1;               // mbarrier whose wait ran out (its commit may still land)
  uint32_t pending_parity = 0u;
  int cur = -1;
  ScanJob j{};
  const PlanProblem *pp = nullptr;
  const PlanGrid *g = nullptr;
  int prec = DOA_FP16X3, MPs = 16, N = 32;
  uint32_t idesc = 0;

  // steering block of tile t into buffer b (row pt, elements [part * MPs / 2, (part + 1) * MPs / 2),
  // 4 per 16-byte chunk: the chunk's first phasor from its exact phase, the others as its products
  // with a_1, a_2, a_3; (re, im) pairs split with packed conversions into the swizzled row)
  auto gen = [&](int b, int64_t t) {
    const int L = g->L;
    const int k0 = (int)(t - pp->tile_start) * kTcRows;
    const uint32_t *S = reinterpret_cast<const uint32_t *>(ws + g->S_off);
    uint8_t *ahi = a_hi(b), *alo = a_lo(b);
    const int pt = tid >> 1, part = tid & 1;
    const int k = k0 + pt;
    const uint32_t Sk = k < L ? S[k] : 0u;
    if (part == 0) sh.sk[b * kTcRows + pt] = Sk;
    const int mh = MPs / 2, m0 = part * mh;
    const float2 z1 = phasor_q32(Sk), z2 = phasor_q32(2u * Sk), z3 = phasor_q32(3u * Sk);
    for (int c = 0; c < mh; c += 4) {
      const float2 a0 = (m0 + c) == 0 ? make_float2(1.f, 0.f) : phasor_q32((uint32_t)(m0 + c) * Sk);
      float2 v[4];
      v[0] = a0;
      v[1] = make_float2(fmaf(a0.x, z1.x, -a0.y * z1.y), fmaf(a0.x, z1.y, a0.y * z1.x));
      v[2] = make_float2(fmaf(a0.x, z2.x, -a0.y * z2.y), fmaf(a0.x, z2.y, a0.y * z2.x));
      v[3] = make_float2(fmaf(a0.x, z3.x, -a0.y * z3.y), fmaf(a0.x, z3.y, a0.y * z3.x));
      uint32_t hw[4], lw[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        if (prec == DOA_FP16X3) {
          const __half2 h2 = __floats2half2_rn(v[q].x, v[q].y);
          const float2 bk = __half22float2(h2);
          const __half2 l2 = __floats2half2_rn((v[q].x - bk.x) * 2048.0f, (v[q].y - bk.y) * 2048.0f);
          hw[q] = *reinterpret_cast<const uint32_t *>(&h2);
          lw[q] = *reinterpret_cast<const uint32_t *>(&l2);
        } else {
          const __nv_bfloat162 h2 = __floats2bfloat162_rn(v[q].x, v[q].y);
          const float2 bk = __bfloat1622float2(h2);
          const __nv_bfloat162 l2 = __floats2bfloat162_rn(v[q].x - bk.x, v[q].y - bk.y);
          hw[q] = *reinterpret_cast<const uint32_t *>(&h2);
          lw[q] = *reinterpret_cast<const uint32_t *>(&l2);
        }
      }
      const uint32_t off = sw128(pt, 2 * (m0 + c));
      *reinterpret_cast<uint4 *>(ahi + off) = make_uint4(hw[0], hw[1], hw[2], hw[3]);
      *reinterpret_cast<uint4 *>(alo + off) = make_uint4(lw[0], lw[1], lw[2], lw[3]);
    }
    for (int kap = 2 * MPs + part * 8; kap < kTbKD; kap += 16) {   // K padding
      const uint32_t off = sw128(pt, kap);
      *reinterpret_cast<uint4 *>(ahi + off) = make_uint4(0, 0, 0, 0);
      *reinterpret_cast<uint4 *>(alo + off) = make_uint4(0, 0, 0, 0);
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  };
  // MMAs of buffer b into accumulator set b (thread 0; after a barrier that follows gen(b))
  auto issue = [&](int b) {
    if (tid != 0 || !ok) return;
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t b_ahi = smem_u32(a_hi(b)), b_alo = smem_u32(a_lo(b)), b_whi = smem_u32(whi), b_wlo = smem_u32(wlo);
    const uint32_t acc0 = tmem + (uint32_t)(b * 2 * N);
    for (int kk = 0; kk < kTbKD / 16; ++kk) {
      const uint32_t off = (uint32_t)kk * 32;
      const uint32_t acc = kk > 0 ? 1u : 0u;
      mma(acc0, smem_desc(b_ahi + off), smem_desc(b_whi + off), idesc, acc);
      if (prec == DOA_BF16X3) {
        mma(acc0, smem_desc(b_ahi + off), smem_desc(b_wlo + off), idesc, 1u);
        mma(acc0, smem_desc(b_alo + off), smem_desc(b_whi + off), idesc, 1u);
      } else {
        mma(acc0 + (uint32_t)N, smem_desc(b_ahi + off), smem_desc(b_wlo + off), idesc, acc);
        mma(acc0 + (uint32_t)N, smem_desc(b_alo + off), smem_desc(b_whi + off), idesc, 1u);
      }
    }
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                     smem_u32(&sh.mbar[b]))
                 : "memory");
  };

  for (int64_t run = blockIdx.x; run * kTbRun < ntiles; run += gridDim.x) {
    const int64_t t_begin = run * kTbRun, t_end = min(ntiles, t_begin + kTbRun);
    int u = 0, hi = nunits - 1;
    while (u < hi) {  // last problem with tile_start <= t_begin
      int mid = (u + hi + 1) >> 1;
      if (probs[list[mid]].tile_start <= t_begin) u = mid; else hi = mid - 1;
    }
    for (int64_t t = t_begin; t < t_end;) {
      while (u + 1 < nunits && probs[list[u + 1]].tile_start <= t) ++u;
      const int64_t seg_end = (u + 1 < nunits) ? min(t_end, probs[list[u + 1]].tile_start) : t_end;
      if (u != cur) {
        // ---- problem setup (no MMA in flight here): FP32 factor, weights, thresholds, split W
        pp = &probs[list[u]];
        g = &grids[pp->grid_id];
        j.F = reinterpret_cast<const double2 *>(ws + pp->fac_off);
        j.w = pp->Kn > 0 && pp->slot[DOA_EV] >= 0
                  ? reinterpret_cast<const double *>(ws + pp->fac_off) + 2 * pp->p.M * (pp->p.M + 1)
                  : nullptr;
        j.S64 = reinterpret_cast<const uint64_t *>(ws + g->S64_off);
        for (int r = 0; r < 4; ++r) j.P[r] = pp->slot[r] >= 0 ? pp->p.P + (size_t)pp->slot[r] * g->L : nullptr;
        j.lo = g->lo;
        j.step = g->step;
        j.M = pp->p.M;
        j.Kf = pp->Kf;
        j.Kn = pp->Kn;
        j.kphd = pp->kphd;
        j.kmn = pp->kmn;
        j.kofs = 0;
        prec = pp->p.prec;
        MPs = (j.M + 15) / 16 * 16;
        N = (2 * j.Kf + 31) / 32 * 32;
        idesc = inst_desc(prec == DOA_FP16X3 ? 0 : 1, N);
        __syncthreads();
        if (tid == 0) sh.maxbits = 0;
        __syncthreads();
        float mx = 0.f;
        for (int e = tid; e < j.Kf * MPs; e += kTbThreads) {
          const int k = e / MPs, m = e % MPs;
          float2 v = make_float2(0.f, 0.f);
          if (m < j.M) {
            const double2 bb = j.F[(size_t)k * j.M + m];
            v = make_float2((float)bb.x, (float)bb.y);
          }
          B32[e] = v;
          mx = fmaxf(mx, fmaxf(fabsf(v.x), fabsf(v.y)));
        }
        for (int k = tid; k < j.Kn; k += kTbThreads) sh.w32[k] = j.w ? (float)j.w[k] : 1.f;
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, off));
        if (lane == 0) atomicMax(&sh.maxbits, __float_as_int(mx));
        __syncthreads();
        if (warp == 0) {
          // E_r from s_k = sum_m |f_mk| (FP32 threshold), N2_r from ||f_k||^2 (tensor threshold)
          const float gam = prec == DOA_FP16X3 ? 1.0e-6f : 8.0e-6f;
          const float c = 2.8f * gam / 1.0e-3f;
          float em = 0.f, ee = 0.f, nm = 0.f, ne = 0.f;
          for (int k = lane; k < j.Kf; k += 32) {
            float n1 = 0.f, q2 = 0.f;
            for (int m = 0; m < j.M; ++m) {
              const float2 bb = B32[k * MPs + m];
              const float a2 = bb.x * bb.x + bb.y * bb.y;
              q2 += a2;
              n1 += sqrtf(a2);
            }
            const float e = n1 * n1;
            if (k < j.Kn) {
              em += e;
              ee += sh.w32[k] * e;
              nm += q2;
              ne += sh.w32[k] * q2;
            }
            if (k == j.kphd) {
              sh.thr32[kRoPhd] = kRefineC * e;
              sh.thrtc[kRoPhd] = c * c * q2;
            }
            if (k == j.kmn) {
              sh.thr32[kRoMn] = kRefineC * e;
              sh.thrtc[kRoMn] = c * c * q2;
            }
          }
#pragma unroll
          for (int off = 16; off > 0; off >>= 1) {
            em += __shfl_xor_sync(0xffffffffu, em, off);
            ee += __shfl_xor_sync(0xffffffffu, ee, off);
            nm += __shfl_xor_sync(0xffffffffu, nm, off);
            ne += __shfl_xor_sync(0xffffffffu, ne, off);
          }
          if (lane == 0) {
            sh.thr32[kRoMusic] = kRefineC * em;
            sh.thr32[kRoEv] = kRefineC * ee;
            sh.thrtc[kRoMusic] = c * c * nm;
            sh.thrtc[kRoEv] = c * c * ne;
          }
        }
        int ex = 0;
        frexpf(fmaxf(__int_as_float(sh.maxbits), FLT_MIN), &ex);
        const float wscale = ldexpf(1.f, -ex);
        if (tid == 0) sh.scale2 = ldexpf(1.f, 2 * ex);
        for (int e = tid; e < N * kTbKD; e += kTbThreads) {
          const int n = e / kTbKD, kap = e % kTbKD;
          const int col = n >> 1, m = kap >> 1;
          float w = 0.f;
          if (col < j.Kf && m < j.M) {
            const float2 bb = B32[col * MPs + m];
            const bool re_out = (n & 1) == 0, re_in = (kap & 1) == 0;
            w = (re_out ? (re_in ? bb.x : bb.y) : (re_in ? -bb.y : bb.x)) * wscale;
          }
          uint16_t hv, lv;
          split16(w, prec, hv, lv);
          const uint32_t off = sw128(n, kap);
          *reinterpret_cast<uint16_t *>(whi + off) = hv;
          *reinterpret_cast<uint16_t *>(wlo + off) = lv;
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        cur = u;
      }
      // ---- software pipeline over the segment's tiles: the steering block of tile i+1 is built
      // and its MMAs issued while tile i's accumulator is read back and its readouts formed
      gen(0, t);
      __syncthreads();
      issue(0);
      for (int64_t i = 0; t + i < seg_end; ++i) {
        const int b = (int)(i & 1);
        const bool has_next = t + i + 1 < seg_end;
        if (has_next) gen(b ^ 1, t + i + 1);
        const bool was_ok = ok;
        const bool done = tid != 0 || (ok && mbar_wait(smem_u32(&sh.mbar[b]), phase[b]));
        ok = __syncthreads_and(done && ok);
        if (was_ok && !ok) {
          pending = b;
          pending_parity = phase[b];
        }
        phase[b] ^= 1u;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        if (has_next) issue(b ^ 1);
        // epilogue of tile t + i: readout partial sums of each row over this warp's column half
        const int L = g->L;
        const int k0 = (int)(t + i - pp->tile_start) * kTcRows;
        const int q = warp & 3, cs = warp >> 2;
        const int row = q * 32 + lane;
        float4 part = make_float4(0.f, 0.f, 0.f, 0.f);   // (MUSIC, EV, PHD, MN)
        if (ok) {
          const int half = N / 2;
          const uint32_t acc0 = tmem + (uint32_t)(b * 2 * N) + ((uint32_t)(q * 32) << 16);
          for (int c0 = cs * half; c0 < (cs + 1) * half; c0 += 8) {
            float v[8];
            tmem_ld8(acc0 + (uint32_t)c0, v);
            if (prec == DOA_FP16X3) {
              float w[8];
              tmem_ld8(acc0 + (uint32_t)(N + c0), w);
#pragma unroll
              for (int x = 0; x < 8; ++x) v[x] = fmaf(w[x], 4.8828125e-4f, v[x]);
            }
#pragma unroll
            for (int x = 0; x < 4; ++x) {
              const int col = c0 / 2 + x;
              const float n = fmaf(v[2 * x], v[2 * x], v[2 * x + 1] * v[2 * x + 1]);
              if (col < j.Kn) {
                part.x += n;
                part.y = fmaf(sh.w32[col], n, part.y);
              }
              if (col == j.kphd) part.z = n;
              if (col == j.kmn) part.w = n;
            }
          }
        }
        red[row * 2 + cs] = part;
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();
        if (tid < kTcRows) {
          const int k = k0 + tid;
          if (k < L) {
            if (!ok) {
              const float nan = __int_as_float(0x7fc00000);   // timed-out tile: NaN marks it
              for (int r = 0; r < 4; ++r)
                if (j.P[r]) j.P[r][k] = nan;
            } else {
              const float4 a = red[tid * 2], c2 = red[tid * 2 + 1];
              const float s2 = sh.scale2;
              float den[4];
              den[kRoMusic] = (a.x + c2.x) * s2;
              den[kRoEv] = (a.y + c2.y) * s2;
              den[kRoPhd] = (a.z + c2.z) * s2;
              den[kRoMn] = (a.w + c2.w) * s2;
              bool flag = false;
              for (int r = 0; r < 4; ++r)
                if (j.P[r]) {
                  j.P[r][k] = recip_out(den[r]);
                  flag = flag || den[r] < sh.thrtc[r];
                }
              if (flag) sh.flags[atomicAdd(&sh.nflag, 1)] = k;
            }
          }
        }
        __syncthreads();
        // re-evaluation of the flagged points: FP32 by a warp, FP64 below the FP32 threshold
        const int nf = sh.nflag;
        for (int f = warp; f < nf; f += kTbWarps) {
          const int k = sh.flags[f];
          float d[4];
          readouts32_warp(B32, MPs, j.M, j, sh.w32, sh.sk[b * kTcRows + (k - k0)], ph32, d);
          bool need64 = false;
          for (int r = 0; r < 4; ++r) need64 = need64 || (j.P[r] && d[r] < sh.thr32[r]);
          if (need64) {
            refine_point_warp(j, k, sh.w32, ph64, yb);
          } else if (lane == 0) {
            for (int r = 0; r < 4; ++r)
              if (j.P[r]) j.P[r][k] = recip_out(d[r]);
          }
        }
        __syncthreads();
        if (tid == 0) {
          sh.nflag = 0;
          if (!ok && status) status[list[u]] = DOA_ETIMEOUT;
        }
      }
      t = seg_end;
    }
  }
  // a commit whose wait ran out may still land: one more bounded wait before TMEM is freed
  if (pending >= 0) mbar_wait(smem_u32(&sh.mbar[pending]), pending_parity);
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(cols));
}

}  // namespace

cudaError_t launch_scan_tc_batch(const uint8_t *plan_dev, const PlanHeader &h, uint8_t *ws, int *status,
                                 cudaStream_t s) {
  if (h.tc_jobs == 0 || h.tc_tiles == 0) return cudaSuccess;
  cudaError_t e = ensure_smem_attr(reinterpret_cast<const void *>(scan_tc_batch_kernel), kTbSmem);
  if (e != cudaSuccess) return e;
  const int sms = device_sm_count();
  const int64_t runs = (h.tc_tiles + kTbRun - 1) / kTbRun;
  int64_t grid = (int64_t)sms * (h.tc_cols <= 256 ? 2 : 1);   // TMEM: 512 columns per SM
  if (grid > runs) grid = runs;
  scan_tc_batch_kernel<<<(unsigned)grid, kTbThreads, kTbSmem, s>>>(plan_dev, ws, status);
  return cudaGetLastError();
}

}  // namespace doa
