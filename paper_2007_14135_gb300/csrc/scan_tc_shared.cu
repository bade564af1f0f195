// Step-5 on the tensor cores for split-precision ULA problems that share a grid (Table 2, Step-5:
// P(theta) = 1 / (a^H C a), C = B W B^H of Table 3), as the batched complex GEMM of one steering
// block against the stacked factors of many problems:
//   A (128 x 64):  rows = the 128 grid points of a tile, [Re a_0, Im a_0, Re a_1, ...] split into
//                  hi + lo (generated once per tile and shared by every group of the unit);
//   W (NG x 64):   a group's stacked real embeddings of B (each problem's 2 Kf rows, rounded up to
//                  16, scaled by its own power of two so that its entries are at most 1), split into
//                  hi + lo, prepared once per solve by tcg_prep_kernel and copied per group into
//                  shared memory by TMA (cp.async.bulk);
//   D (128 x NG):  TMEM, FP32: hi*hi (+ hi*lo + lo*hi; FP16: the cross terms, scaled by 2^11, in a
//                  second accumulator 128 columns on).
// A unit is one tile of the grid for a chunk of up to kTcgChunk groups of the same grid, M bucket
// and precision. Per unit the 256 threads write the steering block; then, group by group, one
// thread issues the TMA copy of the next groups' W (two buffers) and the UMMAs of the next group
// into the other TMEM buffer, while the 8 warps read the current group's accumulator back (warp w:
// TMEM lanes 32 (w % 4).., the problems of parity w / 4) and form each problem's readouts
// (MUSIC sum |y_c|^2, EV sum w_c |y_c|^2, PHD |y_kphd|^2, MN |y_kmn|^2).
// Accuracy: as the per-problem tensor-core scan — a readout below its threshold c^2 sum w ||f||^2
// is queued and re-evaluated by a warp in FP32 with exact integer phases, and in FP64 where the
// FP32 value is below the FP32 path's threshold.
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

constexpr int kTgThreads = 256;
constexpr int kTgWarps = kTgThreads / 32;
constexpr int kTgKD = 64;                        // K extent (one swizzle atom)
constexpr int kTgFlagCap = 2048;                 // queued (problem, point) pairs per drain
constexpr int kTgMaxM = kTcBatchMaxM;

// dynamic shared memory (bytes from a 1024-aligned base)
constexpr int kTgABytes = kTcRows * 128;                       // one 128 x 64 16-bit operand
constexpr int kTgOffAhi = 0;
constexpr int kTgOffAlo = kTgOffAhi + kTgABytes;
constexpr int kTgOffW = kTgOffAlo + kTgABytes;                 // [buffer][hi, lo], kTcgWBytes each
constexpr int kTgOffFlags = kTgOffW + 4 * (int)kTcgWBytes;     // int2 (group * 16 + problem, point)
constexpr int kTgOffPh64 = kTgOffFlags + kTgFlagCap * 8;       // per warp kTgMaxM double2
constexpr int kTgYbCols = kTgMaxM + 2;
constexpr int kTgOffYb = kTgOffPh64 + kTgWarps * kTgMaxM * 16;  // per warp kTgYbCols float2
constexpr int kTgOffPh32 = kTgOffYb + kTgWarps * kTgYbCols * 8; // per warp kTgMaxM float2
constexpr int kTgSmem = kTgOffPh32 + kTgWarps * kTgMaxM * 8 + 1024;
static_assert(kTgSmem + 2048 <= 227 * 1024, "one CTA per SM");

struct TgShared {
  uint64_t tma[2];        // W buffer b landed
  uint64_t mma[2];        // accumulator b written
  uint32_t tmem;
  int nflag;
  uint32_t sk[kTcRows];   // the tile's 32-bit phase steps
  int maxbits;
  float thr[8];           // prep: thr32[4], thrtc[4]
};

__device__ __forceinline__ void tg_bulk_copy(uint32_t dst, const void *src, uint32_t bytes, uint32_t mbar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
               "l"(src), "r"(bytes), "r"(mbar)
               : "memory");
}
__device__ __forceinline__ void tg_arrive_tx(uint32_t mbar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(mbar), "r"(bytes) : "memory");
}
__device__ __forceinline__ void tg_commit(uint32_t mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar) : "memory");
}

// 16 consecutive TMEM columns of this warp's 32 lanes, without waiting (tg_wait_ld waits for all).
__device__ __forceinline__ void tg_ld16(uint32_t addr, uint32_t (&r)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(addr));
}
__device__ __forceinline__ void tg_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// One CTA per group: each problem's FP32 factor (float2 [Kf][MPs] at fac32_off(M) of its factor
// area) and EV weights (after (M + 1) MPs float2), its thresholds and scale, and its rows of the
// group's split operand W (the rows of a problem's column padding and past the last problem are
// zero).
__global__ void __launch_bounds__(kTgThreads) tcg_prep_kernel(const uint8_t *plan, uint8_t *ws) {
  __shared__ TgShared sh;
  const PlanHeader *h = reinterpret_cast<const PlanHeader *>(plan);
  const PlanTcGroup &gr = reinterpret_cast<const PlanTcGroup *>(plan + h->off_tcg)[blockIdx.x];
  const int32_t *list = reinterpret_cast<const int32_t *>(plan + h->off_tcgl);
  const PlanProblem *probs = reinterpret_cast<const PlanProblem *>(plan + h->off_prob);
  const PlanGrid *grids = reinterpret_cast<const PlanGrid *>(plan + h->off_grid);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  uint8_t *rec = ws + gr.rec_off;
  uint8_t *whi = rec, *wlo = rec + kTcgWBytes;
  TcgProb *tab = reinterpret_cast<TcgProb *>(rec + 2 * kTcgWBytes);
  for (int e = tid; e < gr.NG * 128 / 16; e += kTgThreads) {
    reinterpret_cast<uint4 *>(whi)[e] = make_uint4(0, 0, 0, 0);
    reinterpret_cast<uint4 *>(wlo)[e] = make_uint4(0, 0, 0, 0);
  }
  int col = 0;
  for (int i = 0; i < gr.count; ++i) {
    const int prob = list[gr.first + i];
    const PlanProblem &pp = probs[prob];
    const PlanGrid &g = grids[pp.grid_id];
    const int M = pp.p.M, Kf = pp.Kf, Kn = pp.Kn, MPs = (M + 15) / 16 * 16;
    const double2 *F = reinterpret_cast<const double2 *>(ws + pp.fac_off);
    const double *w = Kn > 0 && pp.slot[DOA_EV] >= 0 ? reinterpret_cast<const double *>(F + (size_t)M * (M + 1)) : nullptr;
    float2 *B32 = reinterpret_cast<float2 *>(ws + pp.fac_off + fac32_off(M));
    float *w32 = reinterpret_cast<float *>(ws + pp.fac_off + fac32_off(M) + (size_t)(M + 1) * MPs * 8);
    __syncthreads();   // the zeroed rows and the previous problem's table entry are done
    if (tid == 0) sh.maxbits = 0;
    if (tid < 8) sh.thr[tid] = 0.f;
    __syncthreads();
    float mx = 0.f;
    for (int e = tid; e < Kf * MPs; e += kTgThreads) {
      const int k = e / MPs, m = e % MPs;
      float2 v = make_float2(0.f, 0.f);
      if (m < M) {
        const double2 bb = F[(size_t)k * M + m];
        v = make_float2((float)bb.x, (float)bb.y);
      }
      B32[e] = v;
      mx = fmaxf(mx, fmaxf(fabsf(v.x), fabsf(v.y)));
    }
    for (int k = tid; k < Kn; k += kTgThreads) w32[k] = w ? (float)w[k] : 1.f;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, off));
    if (lane == 0) atomicMax(&sh.maxbits, __float_as_int(mx));
    __syncthreads();   // B32, w32 written (global, same CTA) and the maximum known
    if (warp == 0) {
      // thr32 from s_k = sum_m |f_mk| (FP32 path), thrtc from ||f_k||^2 (the split's error)
      const float gam = pp.p.prec == DOA_FP16X3 ? 1.0e-6f : 8.0e-6f;
      const float c = 2.8f * gam / 1.0e-3f;
      float em = 0.f, ee = 0.f, nm = 0.f, ne = 0.f;
      for (int k = lane; k < Kf; k += 32) {
        float n1 = 0.f, q2 = 0.f;
        for (int m = 0; m < M; ++m) {
          const float2 bb = B32[k * MPs + m];
          const float a2 = bb.x * bb.x + bb.y * bb.y;
          q2 += a2;
          n1 += sqrtf(a2);
        }
        const float e = n1 * n1;
        if (k < Kn) {
          em += e;
          ee += w32[k] * e;
          nm += q2;
          ne += w32[k] * q2;
        }
        if (k == pp.kphd) {
          sh.thr[kRoPhd] = kRefineC * e;
          sh.thr[4 + kRoPhd] = c * c * q2;
        }
        if (k == pp.kmn) {
          sh.thr[kRoMn] = kRefineC * e;
          sh.thr[4 + kRoMn] = c * c * q2;
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
        sh.thr[kRoMusic] = kRefineC * em;
        sh.thr[kRoEv] = kRefineC * ee;
        sh.thr[4 + kRoMusic] = c * c * nm;
        sh.thr[4 + kRoEv] = c * c * ne;
      }
    }
    int ex = 0;
    frexpf(fmaxf(__int_as_float(sh.maxbits), FLT_MIN), &ex);
    const float wscale = ldexpf(1.f, -ex);
    // rows col .. col + 2 Kf - 1: row 2c + 0 gives Re y_c, 2c + 1 gives Im y_c (y = B^H a)
    for (int e = tid; e < 2 * Kf * kTgKD; e += kTgThreads) {
      const int n = e / kTgKD, kap = e % kTgKD;
      const int fc = n >> 1, m = kap >> 1;
      float v = 0.f;
      if (m < M) {
        const float2 bb = B32[fc * MPs + m];
        const bool re_out = (n & 1) == 0, re_in = (kap & 1) == 0;
        v = (re_out ? (re_in ? bb.x : bb.y) : (re_in ? -bb.y : bb.x)) * wscale;
      }
      uint16_t hv, lv;
      split16(v, pp.p.prec, hv, lv);
      const uint32_t off = sw128(col + n, kap);
      *reinterpret_cast<uint16_t *>(whi + off) = hv;
      *reinterpret_cast<uint16_t *>(wlo + off) = lv;
    }
    __syncthreads();   // thresholds written by warp 0
    if (tid == 0) {
      TcgProb t{};
      for (int r = 0; r < 4; ++r) t.P[r] = pp.slot[r] >= 0 ? pp.p.P + (size_t)pp.slot[r] * g.L : nullptr;
      t.B32 = B32;
      t.w32 = w32;
      t.prob = prob;
      t.col = col;
      t.Kf = Kf;
      t.Kn = Kn;
      t.kphd = pp.kphd;
      t.kmn = pp.kmn;
      t.M = M;
      t.MPs = MPs;
      t.scale2 = ldexpf(1.f, 2 * ex);
      for (int r = 0; r < 4; ++r) {
        t.thr32[r] = sh.thr[r];
        t.thrtc[r] = sh.thr[4 + r];
      }
      tab[i] = t;
    }
    col += (2 * Kf + 15) / 16 * 16;
  }
}

// FP32 re-evaluation of all readouts of one point by a warp (lanes: phasors, then columns).
__device__ __forceinline__ void tg_readouts32(const float2 *B32, int MPs, int M, const ScanJob &j, const float *w32,
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

// Persistent: units (tile, chunk) dealt round robin. Roles inside a unit: every thread writes the
// steering block; thread 0 issues the TMA copies and the UMMAs; the 8 warps read back. Every wait
// is bounded; a CTA whose wait ran out stops issuing, writes NaN into the readouts of the points
// it still owns, reports DOA_ETIMEOUT for their problems and waits (bounded) for its copies and
// MMAs in flight before it frees TMEM.
__global__ void __launch_bounds__(kTgThreads, 1) tcg_scan_kernel(const uint8_t *plan, uint8_t *ws, int *status) {
  extern __shared__ __align__(1024) uint8_t tg_smem_raw[];
  uint8_t *sm = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(tg_smem_raw) + 1023) & ~uintptr_t(1023));
  __shared__ TgShared sh;
  const PlanHeader *h = reinterpret_cast<const PlanHeader *>(plan);
  const PlanTcGroup *groups = reinterpret_cast<const PlanTcGroup *>(plan + h->off_tcg);
  const PlanTcChunk *chunks = reinterpret_cast<const PlanTcChunk *>(plan + h->off_tcc);
  const PlanProblem *probs = reinterpret_cast<const PlanProblem *>(plan + h->off_prob);
  const PlanGrid *grids = reinterpret_cast<const PlanGrid *>(plan + h->off_grid);
  const int nchunks = h->tcg_chunks;
  const int64_t nunits = h->tcg_units;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  uint8_t *ahi = sm + kTgOffAhi, *alo = sm + kTgOffAlo;
  auto wbuf = [&](int b, int lohalf) { return sm + kTgOffW + (2 * b + lohalf) * (int)kTcgWBytes; };
  int2 *flags = reinterpret_cast<int2 *>(sm + kTgOffFlags);
  double2 *ph64 = reinterpret_cast<double2 *>(sm + kTgOffPh64) + warp * kTgMaxM;
  float2 *yb = reinterpret_cast<float2 *>(sm + kTgOffYb) + warp * kTgYbCols;
  float2 *ph32 = reinterpret_cast<float2 *>(sm + kTgOffPh32) + warp * kTgMaxM;

  if (tid == 0) {
    for (int b = 0; b < 2; ++b) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&sh.tma[b])));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&sh.mma[b])));
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    sh.nflag = 0;
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&sh.tmem)),
                 "r"(512));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = sh.tmem;

  bool ok = true;
  // thread 0's barrier bookkeeping: next parity per barrier, and operations issued but not waited
  uint32_t tph[2] = {0u, 0u}, mph[2] = {0u, 0u};
  bool tpend[2] = {false, false}, mpend[2] = {false, false};

  // units are taken from a counter in the workspace (zeroed at the start of the solve), so the
  // CTAs whose units re-evaluate many points take fewer of them
  __shared__ unsigned s_unit;
  unsigned *next_unit = reinterpret_cast<unsigned *>(ws) + kCtrTcg;
  for (;;) {
    if (tid == 0) s_unit = atomicAdd(next_unit, 1u);
    __syncthreads();   // the previous unit ended with a barrier, so s_unit is not read while rewritten
    const int64_t u = s_unit;
    if (u >= nunits) break;
    int ci = 0, hi = nchunks - 1;
    while (ci < hi) {   // last chunk with unit_start <= u
      const int mid = (ci + hi + 1) >> 1;
      if (chunks[mid].unit_start <= u) ci = mid; else hi = mid - 1;
    }
    const PlanTcChunk ch = chunks[ci];
    const PlanGrid &g = grids[ch.grid_id];
    const int L = g.L;
    const int k0 = (int)(u - ch.unit_start) * kTcRows;
    const int ng = ch.ngroups;
    const int prec = groups[ch.first_group].prec;

    // ---- steering block of the tile: two threads per point, chunks of 4 phasors (the chunk's
    // first from its exact integer phase, the others as its products with a_1, a_2, a_3)
    {
      const uint32_t *S = reinterpret_cast<const uint32_t *>(ws + g.S_off);
      const int pt = tid >> 1, part = tid & 1;
      const int k = k0 + pt;
      const uint32_t Sk = k < L ? S[k] : 0u;
      if (part == 0) sh.sk[pt] = Sk;
      const int mh = ch.Mg / 2, m0 = part * mh;
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
      for (int kap = 2 * ch.Mg + part * 8; kap < kTgKD; kap += 16) {   // K padding
        const uint32_t off = sw128(pt, kap);
        *reinterpret_cast<uint4 *>(ahi + off) = make_uint4(0, 0, 0, 0);
        *reinterpret_cast<uint4 *>(alo + off) = make_uint4(0, 0, 0, 0);
      }
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    __syncthreads();

    // ---- thread 0: TMA copies of a group's W into buffer i & 1, UMMAs into accumulator i & 1
    auto issue_tma = [&](int i) {
      const int b = i & 1;
      const PlanTcGroup &G = groups[ch.first_group + i];
      const uint8_t *rec = ws + G.rec_off;
      const uint32_t bytes = (uint32_t)G.NG * 128u;
      const uint32_t mb = smem_u32(&sh.tma[b]);
      tg_arrive_tx(mb, 2u * bytes);
      tg_bulk_copy(smem_u32(wbuf(b, 0)), rec, bytes, mb);
      tg_bulk_copy(smem_u32(wbuf(b, 1)), rec + kTcgWBytes, bytes, mb);
      tpend[b] = true;
    };
    auto wait_tma = [&](int b) {
      const bool d = mbar_wait(smem_u32(&sh.tma[b]), tph[b]);
      if (d) {
        tph[b] ^= 1u;
        tpend[b] = false;
      }
      return d;
    };
    auto issue_mma = [&](int i) {
      const int b = i & 1;
      const int NG = groups[ch.first_group + i].NG;
      const uint32_t id = inst_desc(prec == DOA_FP16X3 ? 0 : 1, NG);
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t b_ahi = smem_u32(ahi), b_alo = smem_u32(alo);
      const uint32_t b_whi = smem_u32(wbuf(b, 0)), b_wlo = smem_u32(wbuf(b, 1));
      const uint32_t acc0 = tmem + (uint32_t)(b * 256);
      for (int kk = 0; kk < kTgKD / 16; ++kk) {
        const uint32_t off = (uint32_t)kk * 32;
        const uint32_t acc = kk > 0 ? 1u : 0u;
        mma(acc0, smem_desc(b_ahi + off), smem_desc(b_whi + off), id, acc);
        if (prec == DOA_BF16X3) {
          mma(acc0, smem_desc(b_ahi + off), smem_desc(b_wlo + off), id, 1u);
          mma(acc0, smem_desc(b_alo + off), smem_desc(b_whi + off), id, 1u);
        } else {
          mma(acc0 + 128u, smem_desc(b_ahi + off), smem_desc(b_wlo + off), id, acc);
          mma(acc0 + 128u, smem_desc(b_alo + off), smem_desc(b_whi + off), id, 1u);
        }
      }
      tg_commit(smem_u32(&sh.mma[b]));
      mpend[b] = true;
    };
    auto wait_mma = [&](int b) {
      const bool d = mbar_wait(smem_u32(&sh.mma[b]), mph[b]);
      if (d) {
        mph[b] ^= 1u;
        mpend[b] = false;
      }
      return d;
    };

    if (tid == 0 && ok) {
      issue_tma(0);
      if (ng > 1) issue_tma(1);
      if (wait_tma(0)) issue_mma(0); else ok = false;
    }
    for (int i = 0; i < ng; ++i) {
      const int b = i & 1;
      if (tid == 0 && ok) {
        // the next group's UMMAs go to the other accumulator while this one is read back
        if (i + 1 < ng) {
          if (wait_tma(b ^ 1)) issue_mma(i + 1); else ok = false;
        }
        if (ok && !wait_mma(b)) ok = false;
        if (ok && i + 2 < ng) issue_tma(i + 2);   // buffer b: group i's UMMAs are done with it
      }
      ok = __syncthreads_and(tid != 0 || ok) != 0;
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      // ---- epilogue of group i: thread (row, parity) forms the readouts of its problems
      const PlanTcGroup &G = groups[ch.first_group + i];
      const TcgProb *tab = reinterpret_cast<const TcgProb *>(ws + G.rec_off + 2 * kTcgWBytes);
      const int q = warp & 3, cs = warp >> 2;
      const int row = q * 32 + lane, k = k0 + row;
      for (int pi = cs; pi < G.count; pi += 2) {
        // the problem's table entry in registers (the TMEM waits below are compiler barriers)
        const TcgProb &tp = tab[pi];
        float *P[4];
        float thc[4];
        for (int r = 0; r < 4; ++r) {
          P[r] = tp.P[r];
          thc[r] = tp.thrtc[r];
        }
        const float *w32 = tp.w32;
        const int col = tp.col, Kf = tp.Kf, Kn = tp.Kn, kphd = tp.kphd, kmn = tp.kmn, prob = tp.prob;
        const float scale2 = tp.scale2;
        float dm = 0.f, de = 0.f, dp = 0.f, dn = 0.f;
        auto add_cols = [&](const uint32_t (&r)[16], const uint32_t (&rc)[16], int c0) {
#pragma unroll
          for (int x = 0; x < 8; ++x) {
            const int c = c0 / 2 + x;
            float re = __uint_as_float(r[2 * x]), im = __uint_as_float(r[2 * x + 1]);
            if (prec == DOA_FP16X3) {
              re = fmaf(__uint_as_float(rc[2 * x]), 4.8828125e-4f, re);
              im = fmaf(__uint_as_float(rc[2 * x + 1]), 4.8828125e-4f, im);
            }
            if (c < Kf) {
              const float n = fmaf(re, re, im * im);
              if (c < Kn) {
                dm += n;
                de = fmaf(w32[c], n, de);
              }
              if (c == kphd) dp = n;
              if (c == kmn) dn = n;
            }
          }
        };
        if (ok) {
          // 32 columns (two loads of 16, plus the FP16 cross terms) per wait; a problem's block of
          // columns is a multiple of 16, so no load reaches past it
          const uint32_t acc0 = tmem + (uint32_t)(b * 256 + col) + ((uint32_t)(q * 32) << 16);
          for (int c0 = 0; c0 < 2 * Kf; c0 += 32) {
            const bool two = c0 + 16 < 2 * Kf;
            uint32_t r0[16], r1[16], q0[16], q1[16];
            tg_ld16(acc0 + (uint32_t)c0, r0);
            if (prec == DOA_FP16X3) tg_ld16(acc0 + 128u + (uint32_t)c0, q0);
            if (two) {
              tg_ld16(acc0 + (uint32_t)(c0 + 16), r1);
              if (prec == DOA_FP16X3) tg_ld16(acc0 + 128u + (uint32_t)(c0 + 16), q1);
            }
            tg_wait_ld();
            add_cols(r0, q0, c0);
            if (two) add_cols(r1, q1, c0 + 16);
          }
        }
        if (k < L) {
          if (!ok) {
            const float nan = __int_as_float(0x7fc00000);   // timed-out unit: NaN marks the points
            for (int r = 0; r < 4; ++r)
              if (P[r]) P[r][k] = nan;
          } else {
            float den[4];
            den[kRoPhd] = dp * scale2;
            den[kRoMusic] = dm * scale2;
            den[kRoEv] = de * scale2;
            den[kRoMn] = dn * scale2;
            bool flag = false;
            for (int r = 0; r < 4; ++r)
              if (P[r]) {
                P[r][k] = recip_out(den[r]);
                flag = flag || den[r] < thc[r];
              }
            if (flag) {
              const int pos = atomicAdd(&sh.nflag, 1);
              if (pos < kTgFlagCap) flags[pos] = make_int2(pi, k);   // a group adds at most 16 x 128
            }
          }
        }
        if (!ok && k == k0 && status) status[prob] = DOA_ETIMEOUT;
      }
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncthreads();
      // ---- re-evaluation of the group's queued points: FP32 by a warp, FP64 below the FP32 threshold
      const int nf = min(sh.nflag, kTgFlagCap);
      for (int f = warp; f < nf; f += kTgWarps) {
        const int2 e = flags[f];
        const TcgProb &t = tab[e.x];
        const PlanProblem &pp = probs[t.prob];
        ScanJob j{};
        j.F = reinterpret_cast<const double2 *>(ws + pp.fac_off);
        j.w = t.Kn > 0 && pp.slot[DOA_EV] >= 0
                  ? reinterpret_cast<const double *>(ws + pp.fac_off) + 2 * t.M * (t.M + 1)
                  : nullptr;
        j.S64 = reinterpret_cast<const uint64_t *>(ws + g.S64_off);
        for (int r = 0; r < 4; ++r) j.P[r] = t.P[r];
        j.lo = g.lo;
        j.step = g.step;
        j.M = t.M;
        j.Kf = t.Kf;
        j.Kn = t.Kn;
        j.kphd = t.kphd;
        j.kmn = t.kmn;
        j.kofs = 0;
        float d[4];
        tg_readouts32(t.B32, t.MPs, t.M, j, t.w32, sh.sk[e.y - k0], ph32, d);
        bool need64 = false;
        for (int r = 0; r < 4; ++r) need64 = need64 || (t.P[r] && d[r] < t.thr32[r]);
        if (need64) {
          refine_point_warp(j, e.y, t.w32, ph64, yb);
        } else if (lane == 0) {
          for (int r = 0; r < 4; ++r)
            if (t.P[r]) t.P[r][e.y] = recip_out(d[r]);
        }
      }
      __syncthreads();
      if (tid == 0) sh.nflag = 0;
    }
    __syncthreads();   // the steering block is rewritten by the next unit
  }
  // copies and UMMAs whose wait ran out may still land: one more bounded wait before TMEM is freed
  if (tid == 0) {
    for (int b = 0; b < 2; ++b) {
      if (tpend[b]) mbar_wait(smem_u32(&sh.tma[b]), tph[b]);
      if (mpend[b]) mbar_wait(smem_u32(&sh.mma[b]), mph[b]);
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512));
}

}  // namespace

cudaError_t launch_scan_tc_shared(const uint8_t *plan_dev, const PlanHeader &h, uint8_t *ws, int *status,
                                  cudaStream_t s) {
  if (h.tcg_groups == 0 || h.tcg_units == 0) return cudaSuccess;
  tcg_prep_kernel<<<h.tcg_groups, kTgThreads, 0, s>>>(plan_dev, ws);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  if ((e = ensure_smem_attr((const void *)tcg_scan_kernel, kTgSmem)) != cudaSuccess) return e;
  const int64_t grid = std::min<int64_t>(h.tcg_units, device_sm_count());   // TMEM: 512 columns per SM
  tcg_scan_kernel<<<(unsigned)grid, kTgThreads, kTgSmem, s>>>(plan_dev, ws, status);
  return cudaGetLastError();
}

}  // namespace doa
