// Device pieces of the CUDA-core FP32 scan shared by the full-grid, batched and windowed scans.
//
// One scan job contracts the steering vectors with the Kf columns f_k of a factor F and turns the
// column outputs y_k = f_k^H a into up to four pseudospectra ("readouts", Table 3):
//   MUSIC  den = sum_{k<Kn} |y_k|^2                 (F[:, :Kn] = E_n)
//   EV     den = sum_{k<Kn} w_k |y_k|^2, w_k = 1/lambda_k   (E_n Lambda_n^-1 E_n^H)
//   PHD    den = |y_kphd|^2                         (column kphd = v_min)
//   MN     den = |y_kmn|^2                          (column kmn = valph = P_n e1 / (e1^H P_n e1))
// so a problem that asks for several algorithms generates its steering vectors once and
// contracts the noise eigenvectors once. A single-factor scan (doa_scan) is the MUSIC readout
// with F = B, Kn = K.
#pragma once

#include <float.h>

#include "doa_internal.cuh"

namespace doa {
namespace scanc {

constexpr float kRefineC = 3.7e-6f;   // (4 * 4 eps32 / 5e-4)^2, direct sum (4 eps per term)
constexpr float kRefineCH = 2.05e-6f; // (4 * 3 eps32 / 5e-4)^2, blocked Horner ULA form (3 eps per term)

// ULA scans use the blocked Horner form (below) up to MP = 16; larger factors keep the direct sum
// (the outer Horner chain in w4 would grow beyond three steps).
template <int MP>
__host__ __device__ constexpr bool ula_horner_form() { return MP <= 16; }
// Refinement constant of a scan: the Horner bound for ULA jobs evaluated in that form.
template <int MP, bool kUla>
__host__ __device__ constexpr float refine_c() { return kUla && ula_horner_form<MP>() ? kRefineCH : kRefineC; }
constexpr int kFlagCap = 1024;         // queued refinements per drain (overflow: refined in place)
constexpr int kScanWarps = kScanThreads / 32;
constexpr int kMaxCols = kMaxM + 1;    // E_n (up to M columns when d = 0) plus valph

// Readout slots, in doa_alg order.
constexpr int kRoPhd = 0, kRoMusic = 1, kRoEv = 2, kRoMn = 3;

struct ScanJob {
  const double2 *F;      // FP64 factor, column-major, ld M, Kf columns
  const double *w;       // FP64 EV weights (Kn entries); null when EV is absent
  const uint64_t *S64;   // 64-bit phase steps per local point, or null (computed from lo, step)
  float *P[4];           // output row of each readout (local point index); null = absent
  double lo, step;
  int M, Kf, Kn, kphd, kmn;
  int kofs;              // grid index of local point 0 (windowed scans)
};

struct ScanShared {
  double2 ph[kScanWarps][kMaxM];      // per-warp FP64 phasors for refinement
  float2 yb[kScanWarps][kMaxCols];    // per-warp column outputs of refinement (rounded once)
  float w32[kMaxM];                   // FP32 EV weights
  // Refinement queue: points whose FP32 value of MUSIC or EV (or any readout, for M > 32) is
  // below its threshold fill flags[] from the front and are re-evaluated for every readout;
  // points flagged only for PHD and / or MN fill it from the back, with fmask[] naming the
  // readouts (bit r = readout r), and are re-evaluated for those columns alone. nflag counts both:
  // front entries in its low 16 bits, back entries in its high 16 bits.
  int flags[kFlagCap];
  uint8_t fmask[kFlagCap];
  unsigned nflag;
  float thr[4];                       // per-readout refinement thresholds (-1: readout absent)
};
__device__ __forceinline__ int queue_front(unsigned n) { return (int)(n & 0xffffu); }
__device__ __forceinline__ int queue_back(unsigned n) { return (int)(n >> 16); }

// F (M x Kf complex128, column-major, ld M) -> Bs[k][m] (FP32, rows m >= M zero-padded to MP);
// EV weights -> sh.w32.
template <int MP>
__device__ __forceinline__ void load_job(const ScanJob &j, float2 *Bs, ScanShared &sh) {
  for (int e = threadIdx.x; e < j.Kf * MP; e += blockDim.x) {
    int k = e / MP, m = e % MP;
    float2 v = make_float2(0.f, 0.f);
    if (m < j.M) {
      double2 b = j.F[(size_t)k * j.M + m];
      v = make_float2((float)b.x, (float)b.y);
    }
    Bs[e] = v;
  }
  for (int k = threadIdx.x; k < j.Kn; k += blockDim.x) sh.w32[k] = j.w ? (float)j.w[k] : 1.f;
}

// Threshold of readout r = C * E_r (C = refine_c) with s_k = sum_m |f_mk| (FP32 factor):
// E_MUSIC = sum_{k<Kn} s_k^2, E_EV = sum_{k<Kn} w_k s_k^2, E_PHD = s_kphd^2, E_MN = s_kmn^2.
// (A bound of ~4 eps per term on y_k gives den a relative error below ~5e-4 above it.)
// Computed by the 32 lanes of one warp (every lane returns the same values); thr[r] of an absent
// readout is left as it was.
template <int MP, bool kUla = false>
__device__ __forceinline__ void job_thresholds(const float2 *F32, const float *w32, int Kf, int Kn, int kphd, int kmn,
                                               float (&thr)[4]) {
  const int lane = threadIdx.x & 31;
  float em = 0.f, ee = 0.f, ep = -1.f, en = -1.f;
  for (int k = lane; k < Kf; k += 32) {
    float n1 = 0.f;
    for (int m = 0; m < MP; ++m) {
      const float2 b = F32[k * MP + m];
      n1 = __fadd_rn(n1, __fsqrt_rn(__fmaf_rn(b.x, b.x, __fmul_rn(b.y, b.y))));
    }
    const float e = __fmul_rn(n1, n1);
    if (k < Kn) {
      em = __fadd_rn(em, e);
      ee = __fmaf_rn(w32[k], e, ee);
    }
    if (k == kphd) ep = e;
    if (k == kmn) en = e;
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    em = __fadd_rn(em, __shfl_xor_sync(0xffffffffu, em, off));
    ee = __fadd_rn(ee, __shfl_xor_sync(0xffffffffu, ee, off));
    ep = fmaxf(ep, __shfl_xor_sync(0xffffffffu, ep, off));
    en = fmaxf(en, __shfl_xor_sync(0xffffffffu, en, off));
  }
  constexpr float C = refine_c<MP, kUla>();
  thr[kRoMusic] = __fmul_rn(C, em);
  thr[kRoEv] = __fmul_rn(C, ee);
  if (kphd >= 0) thr[kRoPhd] = __fmul_rn(C, ep);
  if (kmn >= 0) thr[kRoMn] = __fmul_rn(C, en);
}

template <int MP, bool kUla = false>
__device__ __forceinline__ void set_threshold(const float2 *Bs, const ScanJob &j, ScanShared &sh) {
  if (threadIdx.x < 32) {
    float thr[4] = {0.f, 0.f, 0.f, 0.f};
    job_thresholds<MP, kUla>(Bs, sh.w32, j.Kf, j.Kn, j.kphd, j.kmn, thr);
    if (threadIdx.x == 0) {
#pragma unroll
      for (int r = 0; r < 4; ++r) sh.thr[r] = thr[r];
      sh.nflag = 0;
    }
  }
}

// Paired-FMA form of the FP32 scan (fma.rn.f32x2: two FP32 FMAs per instruction, one for each of
// two grid points): the factor is held in shared memory as Bd[k][m] = (bx, bx, by, by), so one
// 16-byte load gives both operand pairs of an element.
template <int MP>
__device__ __forceinline__ void load_job2(const ScanJob &j, float4 *Bd, ScanShared &sh) {
  for (int e = threadIdx.x; e < j.Kf * MP; e += blockDim.x) {
    const int k = e / MP, m = e % MP;
    float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
    if (m < j.M) {
      const double2 b = j.F[(size_t)k * j.M + m];
      const float bx = (float)b.x, by = (float)b.y;
      v = make_float4(bx, bx, by, by);
    }
    Bd[e] = v;
  }
  for (int k = threadIdx.x; k < j.Kn; k += blockDim.x) sh.w32[k] = j.w ? (float)j.w[k] : 1.f;
}

// job_thresholds on the duplicated layout (the same FP32 values, the same arithmetic).
template <int MP, bool kUla = false>
__device__ __forceinline__ void job_thresholds2(const float4 *Bd, const float *w32, int Kf, int Kn, int kphd, int kmn,
                                                float (&thr)[4]) {
  const int lane = threadIdx.x & 31;
  float em = 0.f, ee = 0.f, ep = -1.f, en = -1.f;
  for (int k = lane; k < Kf; k += 32) {
    float n1 = 0.f;
    for (int m = 0; m < MP; ++m) {
      const float4 b = Bd[k * MP + m];
      n1 = __fadd_rn(n1, __fsqrt_rn(__fmaf_rn(b.x, b.x, __fmul_rn(b.z, b.z))));
    }
    const float e = __fmul_rn(n1, n1);
    if (k < Kn) {
      em = __fadd_rn(em, e);
      ee = __fmaf_rn(w32[k], e, ee);
    }
    if (k == kphd) ep = e;
    if (k == kmn) en = e;
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    em = __fadd_rn(em, __shfl_xor_sync(0xffffffffu, em, off));
    ee = __fadd_rn(ee, __shfl_xor_sync(0xffffffffu, ee, off));
    ep = fmaxf(ep, __shfl_xor_sync(0xffffffffu, ep, off));
    en = fmaxf(en, __shfl_xor_sync(0xffffffffu, en, off));
  }
  constexpr float C = refine_c<MP, kUla>();
  thr[kRoMusic] = __fmul_rn(C, em);
  thr[kRoEv] = __fmul_rn(C, ee);
  if (kphd >= 0) thr[kRoPhd] = __fmul_rn(C, ep);
  if (kmn >= 0) thr[kRoMn] = __fmul_rn(C, en);
}

template <int MP, bool kUla = false>
__device__ __forceinline__ void set_threshold2(const float4 *Bd, const ScanJob &j, ScanShared &sh) {
  if (threadIdx.x < 32) {
    float thr[4] = {0.f, 0.f, 0.f, 0.f};
    job_thresholds2<MP, kUla>(Bd, sh.w32, j.Kf, j.Kn, j.kphd, j.kmn, thr);
    if (threadIdx.x == 0) {
#pragma unroll
      for (int r = 0; r < 4; ++r) sh.thr[r] = thr[r];
      sh.nflag = 0;
    }
  }
}

__device__ __forceinline__ uint64_t phase64_of_point(const ScanJob &j, int k) {
  if (j.S64) return j.S64[k];
  const double theta = __dadd_rn(j.lo, __dmul_rn((double)(k + j.kofs), j.step));
  return phase_step64_of_sin(sin(theta * 0.017453292519943295));
}

__device__ __forceinline__ float recip_out(float den) { return __frcp_rn(fmaxf(den, FLT_MIN)); }

// FP64 steering source of the ULA scans: the exact 64-bit phase m * S64_k of element m.
struct UlaSource {
  const ScanJob *j;
  __device__ __forceinline__ uint64_t prep(int k) const { return phase64_of_point(*j, k); }
  __device__ __forceinline__ double2 phasor(uint64_t step, int m) const { return phasor_q64((uint64_t)m * step); }
};

// Re-evaluation of local point k by one whole warp with the steering vector and the contraction
// in FP64: phasors from the source (lane m), then y_c = f_c^H a with LPC lanes per column (LPC =
// the largest power of two with Kf * LPC <= 32, so one pass covers the columns when it can), each
// lane summing a contiguous run of elements and the LPC partial sums combined by shuffles. The
// cancellation that makes the FP32 result inaccurate happens inside y_c; the readouts sum
// |y_c|^2 >= 0 and are formed from y_c rounded once to FP32.
template <class Src>
inline __device__ void refine_point_warp_src(const ScanJob &j, int k, const Src &src, const float *w32, double2 *ph,
                                             float2 *yb) {
  const int lane = threadIdx.x & 31;
  const auto st = src.prep(k);
  const int M = j.M, Kf = j.Kf;
  for (int m = lane; m < M; m += 32) ph[m] = src.phasor(st, m);
  __syncwarp();
  int lpc = 1;
  while (lpc < 32 && Kf * lpc * 2 <= 32 && lpc < M) lpc <<= 1;
  const int epl = (M + lpc - 1) / lpc;     // elements per lane
  const int sub = lane % lpc, cpp = 32 / lpc;
  for (int c0 = 0; c0 < Kf; c0 += cpp) {
    const int col = c0 + lane / lpc;
    double yr = 0.0, yi = 0.0;
    if (col < Kf) {
      const double2 *f = j.F + (size_t)col * M;
      const int m1 = min(M, (sub + 1) * epl);
      for (int m = sub * epl; m < m1; ++m) {
        const double2 b = f[m], a = ph[m];     // conj(b) * a
        yr = fma(b.x, a.x, fma(b.y, a.y, yr));
        yi = fma(b.x, a.y, fma(-b.y, a.x, yi));
      }
    }
    for (int off = lpc >> 1; off > 0; off >>= 1) {
      yr += __shfl_xor_sync(0xffffffffu, yr, off);
      yi += __shfl_xor_sync(0xffffffffu, yi, off);
    }
    if (sub == 0 && col < Kf) yb[col] = make_float2((float)yr, (float)yi);
  }
  __syncwarp();
  float dm = 0.f, de = 0.f;
  for (int c = lane; c < j.Kn; c += 32) {
    const float2 y = yb[c];
    const float n = fmaf(y.x, y.x, y.y * y.y);
    dm += n;
    de = fmaf(w32[c], n, de);
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    dm += __shfl_xor_sync(0xffffffffu, dm, off);
    de += __shfl_xor_sync(0xffffffffu, de, off);
  }
  if (lane == 0) {
    if (j.P[kRoMusic]) j.P[kRoMusic][k] = recip_out(dm);
    if (j.P[kRoEv]) j.P[kRoEv][k] = recip_out(de);
    if (j.P[kRoPhd]) {
      const float2 y = yb[j.kphd];
      j.P[kRoPhd][k] = recip_out(fmaf(y.x, y.x, y.y * y.y));
    }
    if (j.P[kRoMn]) {
      const float2 y = yb[j.kmn];
      j.P[kRoMn][k] = recip_out(fmaf(y.x, y.x, y.y * y.y));
    }
  }
  __syncwarp();
}

inline __device__ void refine_point_warp(const ScanJob &j, int k, const float *w32, double2 *ph, float2 *yb) {
  refine_point_warp_src(j, k, UlaSource{&j}, w32, ph, yb);
}

// Same computation by a single thread (only when a tile's queue overflows).
template <class Src>
inline __device__ void refine_point_thread_src(const ScanJob &j, int k, const Src &src, const float *w32) {
  const auto st = src.prep(k);
  float dm = 0.f, de = 0.f, dp = 0.f, dn = 0.f;
  for (int col = 0; col < j.Kf; ++col) {
    double yr = 0.0, yi = 0.0;
    for (int m = 0; m < j.M; ++m) {
      const double2 a = src.phasor(st, m);
      const double2 b = j.F[(size_t)col * j.M + m];
      yr = fma(b.x, a.x, fma(b.y, a.y, yr));
      yi = fma(b.x, a.y, fma(-b.y, a.x, yi));
    }
    const float fr = (float)yr, fi = (float)yi;
    const float n = fmaf(fr, fr, fi * fi);
    if (col < j.Kn) {
      dm += n;
      de = fmaf(w32[col], n, de);
    }
    if (col == j.kphd) dp = n;
    if (col == j.kmn) dn = n;
  }
  if (j.P[kRoMusic]) j.P[kRoMusic][k] = recip_out(dm);
  if (j.P[kRoEv]) j.P[kRoEv][k] = recip_out(de);
  if (j.P[kRoPhd]) j.P[kRoPhd][k] = recip_out(dp);
  if (j.P[kRoMn]) j.P[kRoMn][k] = recip_out(dn);
}

// Re-evaluation of several points per warp for small factors: a sub-warp of W lanes per point
// (W = 8 or 16, 32 / W points at once; needs M <= W and Kf <= W). Lanes own the phasors a_m
// (m = lane in the sub-warp), then one factor column each (y_c = f_c^H a over all M elements in
// FP64), and the readouts are sums over the sub-warp of |y_c|^2 from y_c rounded once to FP32,
// as in refine_point_warp_src. Every lane of the warp runs the same number of steps (a sub-warp
// without a point works on a copy of the first and does not store).
template <int W, class Src>
inline __device__ void refine_points_subwarp(const ScanJob &j, const int *ks, int cnt, const Src &src,
                                             const float *w32, double2 *ph) {
  const int lane = threadIdx.x & 31, sub = lane % W, grp = lane / W;
  const bool live = grp < cnt;
  const int k = ks[live ? grp : 0];
  const auto st = src.prep(k);
  double2 *mine = ph + grp * W;
  if (sub < j.M) mine[sub] = src.phasor(st, sub);
  __syncwarp();
  float n = 0.f;
  if (sub < j.Kf) {
    const double2 *f = j.F + (size_t)sub * j.M;
    double yr = 0.0, yi = 0.0;
    for (int m = 0; m < j.M; ++m) {
      const double2 b = f[m], a = mine[m];     // conj(b) * a
      yr = fma(b.x, a.x, fma(b.y, a.y, yr));
      yi = fma(b.x, a.y, fma(-b.y, a.x, yi));
    }
    const float fr = (float)yr, fi = (float)yi;
    n = fmaf(fr, fr, fi * fi);
  }
  float dm = sub < j.Kn ? n : 0.f;
  float de = sub < j.Kn ? w32[sub] * n : 0.f;
#pragma unroll
  for (int off = W / 2; off > 0; off >>= 1) {
    dm += __shfl_xor_sync(0xffffffffu, dm, off);
    de += __shfl_xor_sync(0xffffffffu, de, off);
  }
  const int base = grp * W;
  const float dp = __shfl_sync(0xffffffffu, n, base + (j.kphd >= 0 ? j.kphd : 0));
  const float dn = __shfl_sync(0xffffffffu, n, base + (j.kmn >= 0 ? j.kmn : 0));
  if (live && sub == 0) {
    if (j.P[kRoMusic]) j.P[kRoMusic][k] = recip_out(dm);
    if (j.P[kRoEv]) j.P[kRoEv][k] = recip_out(de);
    if (j.P[kRoPhd]) j.P[kRoPhd][k] = recip_out(dp);
    if (j.P[kRoMn]) j.P[kRoMn][k] = recip_out(dn);
  }
  __syncwarp();
}

// Re-evaluation of the PHD and / or MN readouts alone (the others were above their thresholds):
// a sub-warp of W lanes per point (W = 8, 16 or 32; M <= W), lane m the product conj(f_mc) a_m in
// FP64 for the flagged column c (v_min, valph), the sum over the sub-warp by shuffles, y rounded
// once to FP32 and P = 1 / |y|^2 as in refine_point_warp_src. Every lane runs the same steps (a
// sub-warp without a point or without the readout sums zeros and does not store).
template <int W, class Src>
inline __device__ void refine_points_single(const ScanJob &j, const int *ks, const uint8_t *masks, int cnt,
                                            const Src &src) {
  const int lane = threadIdx.x & 31, sub = lane % W, grp = lane / W;
  const bool live = grp < cnt;
  const int k = ks[live ? grp : 0];
  const unsigned mk = live ? masks[grp] : 0u;
  const auto st = src.prep(k);
  double2 a = make_double2(0.0, 0.0);
  if (sub < j.M) a = src.phasor(st, sub);
#pragma unroll
  for (int r = 0; r < 2; ++r) {
    const int R = r == 0 ? kRoPhd : kRoMn, col = r == 0 ? j.kphd : j.kmn;
    const bool want = ((mk >> R) & 1u) && col >= 0;
    double yr = 0.0, yi = 0.0;
    if (want && sub < j.M) {
      const double2 b = j.F[(size_t)col * j.M + sub];   // conj(b) * a
      yr = fma(b.x, a.x, b.y * a.y);
      yi = fma(b.x, a.y, -b.y * a.x);
    }
#pragma unroll
    for (int off = W / 2; off > 0; off >>= 1) {
      yr += __shfl_xor_sync(0xffffffffu, yr, off);
      yi += __shfl_xor_sync(0xffffffffu, yi, off);
    }
    if (want && sub == 0) {
      const float fr = (float)yr, fi = (float)yi;
      j.P[R][k] = recip_out(fmaf(fr, fr, fi * fi));
    }
  }
}

// The back of the queue (points flagged for PHD / MN alone): 4, 2 or 1 points per warp pass.
template <class Src>
__device__ __forceinline__ void refine_single_run(const ScanJob &j, const int *ks, const uint8_t *masks, int n,
                                                  const Src &src) {
  if (j.M <= 8) {
    for (int c = 0; c < n; c += 4) refine_points_single<8>(j, ks + c, masks + c, min(4, n - c), src);
  } else if (j.M <= 16) {
    for (int c = 0; c < n; c += 2) refine_points_single<16>(j, ks + c, masks + c, min(2, n - c), src);
  } else {
    for (int c = 0; c < n; ++c) refine_points_single<32>(j, ks + c, masks + c, 1, src);
  }
}

// Drains the tile's refinement queue (all threads of the CTA call this): several points per warp
// when the factor is small enough, else one point per warp.
template <class Src>
__device__ __forceinline__ void drain_refinements_src(const ScanJob &j, const Src &src, ScanShared &sh) {
  __syncthreads();
  const int n = queue_front(sh.nflag), nb = queue_back(sh.nflag);
  const int warp = threadIdx.x >> 5;
  if (j.M <= 8 && j.Kf <= 8) {
    for (int i = warp * 4; i < n; i += kScanWarps * 4)
      refine_points_subwarp<8>(j, sh.flags + i, min(4, n - i), src, sh.w32, sh.ph[warp]);
  } else if (j.M <= 16 && j.Kf <= 16) {
    for (int i = warp * 2; i < n; i += kScanWarps * 2)
      refine_points_subwarp<16>(j, sh.flags + i, min(2, n - i), src, sh.w32, sh.ph[warp]);
  } else {
    for (int i = warp; i < n; i += kScanWarps)
      refine_point_warp_src(j, sh.flags[i], src, sh.w32, sh.ph[warp], sh.yb[warp]);
  }
  // back entries, kFlagCap - nb .. kFlagCap - 1, in chunks of 4 per warp
  for (int i = kFlagCap - nb + warp * 4; i < kFlagCap; i += kScanWarps * 4)
    refine_single_run(j, sh.flags + i, sh.fmask + i, min(4, kFlagCap - i), src);
  __syncthreads();
  if (threadIdx.x == 0) sh.nflag = 0;
  __syncthreads();
}

__device__ __forceinline__ void drain_refinements(const ScanJob &j, ScanShared &sh) {
  drain_refinements_src(j, UlaSource{&j}, sh);
}

template <int PT>
__device__ __forceinline__ void store_row(float *P, int L, int k0, const float (&out)[PT]) {
  if (PT == 4 && k0 + 3 < L && ((reinterpret_cast<uintptr_t>(P + k0) & 15u) == 0)) {
    *reinterpret_cast<float4 *>(P + k0) = make_float4(out[0], out[1 % PT], out[2 % PT], out[3 % PT]);
  } else if (PT == 2 && k0 + 1 < L && ((reinterpret_cast<uintptr_t>(P + k0) & 7u) == 0)) {
    *reinterpret_cast<float2 *>(P + k0) = make_float2(out[0], out[1 % PT]);
  } else {
#pragma unroll
    for (int q = 0; q < PT; ++q)
      if (k0 + q < L) P[k0 + q] = out[q];
  }
}

// Readouts of the PT points k0 .. k0+PT-1 (those < L) from their denominators: P = 1 / den stored per
// present readout, and every point where some readout's den is below its refinement threshold
// queued for drain_refinements_src (or, on queue overflow, re-evaluated in place from src). With
// kExt every queued point also records `tag` in tags[] (the grid-shared scan queues the points of
// several problems).
template <int PT, class Src, bool kExt>
__device__ __forceinline__ void finish_points(const ScanJob &j, const float (&dp)[PT], const float (&dm)[PT],
                                              const float (&de)[PT], const float (&dn)[PT], int L, int k0,
                                              ScanShared &sh, const Src &src, const float *w32, const float *thr_,
                                              uint8_t *tags, int tag) {
  unsigned mk[PT];   // bit r: readout r below its threshold
#pragma unroll
  for (int q = 0; q < PT; ++q) mk[q] = 0u;
  float out[PT];
#define DOA_READOUT(R, DEN)                                                   \
  if (j.P[R]) {                                                               \
    const float thr = thr_[R];                                                \
    _Pragma("unroll") for (int q = 0; q < PT; ++q) {                          \
      out[q] = __frcp_rn(fmaxf(DEN[q], FLT_MIN));                              \
      mk[q] |= (DEN[q] < thr ? 1u : 0u) << R;                                 \
    }                                                                         \
    store_row<PT>(j.P[R], L, k0, out);                                        \
  }
  DOA_READOUT(kRoPhd, dp)
  DOA_READOUT(kRoMusic, dm)
  DOA_READOUT(kRoEv, de)
  DOA_READOUT(kRoMn, dn)
#undef DOA_READOUT
  bool over[PT];
#pragma unroll
  for (int q = 0; q < PT; ++q) {
    over[q] = false;
    if (k0 + q < L && mk[q]) {
      // whole re-evaluation for MUSIC / EV (every E_n column) and for M > 32; PHD / MN alone
      // need their own column only
      const bool whole = (mk[q] & ((1u << kRoMusic) | (1u << kRoEv))) || j.M > 32;
      const unsigned inc = whole ? 1u : 0x10000u;
      const unsigned old = atomicAdd(&sh.nflag, inc);
      const int f = queue_front(old), b = queue_back(old);
      if (f + b < kFlagCap) {
        const int slot = whole ? f : kFlagCap - 1 - b;
        sh.flags[slot] = k0 + q;
        sh.fmask[slot] = (uint8_t)mk[q];
        if (kExt) tags[slot] = (uint8_t)tag;
      } else {
        atomicSub(&sh.nflag, inc);   // not queued (the queue is full): the count stays that of the entries
        over[q] = true;
      }
    }
  }
  // queue overflow (more than kFlagCap small denominators before a drain): refine in place
#pragma unroll
  for (int q = 0; q < PT; ++q)
    if (over[q]) refine_point_thread_src(j, k0 + q, src, w32);
}

// Contracts the PT x MP phasor block a (points k0 .. k0+PT-1 of a job, those < L) with the factor
// and writes the readouts. Points where any readout falls below its refinement threshold are
// queued for drain_refinements_src (or, on queue overflow, re-evaluated in place from src).
// kExt: the EV weights and thresholds come from w32x / thrx instead of sh, and every queued point
// also records `tag` in tags[] (the grid-shared scan queues the points of several problems).
template <int MP, int PT, class Src, bool kExt = false>
__device__ __forceinline__ void contract_points(const float2 *Bs, const ScanJob &j, const float2 (&a)[PT][MP], int L,
                                                int k0, ScanShared &sh, const Src &src, const float *w32x = nullptr,
                                                const float *thrx = nullptr, uint8_t *tags = nullptr, int tag = 0) {
  const float *w32 = kExt ? w32x : sh.w32;
  const float *thr_ = kExt ? thrx : sh.thr;
  float dm[PT], de[PT], dp[PT], dn[PT], n[PT];
#pragma unroll
  for (int q = 0; q < PT; ++q) dm[q] = de[q] = dp[q] = dn[q] = n[q] = 0.f;
  // n = |f_k^H a|^2 for the PT points; factor rows read two elements (16 bytes) at a time.
  // conj(b) * a = (br ar + bi ai) + j (br ai - bi ar): the imaginary part as two sums subtracted at
  // the end of the column, the operations (and their order) of contract_points2, so every launch
  // shape gives the same bits.
  auto column = [&](int k) {
    float yr[PT], ya[PT], yb[PT];
#pragma unroll
    for (int q = 0; q < PT; ++q) yr[q] = ya[q] = yb[q] = 0.f;
    const float4 *b2 = reinterpret_cast<const float4 *>(Bs + k * MP);
#pragma unroll
    for (int m2 = 0; m2 < MP / 2; ++m2) {
      const float4 bb = b2[m2];
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const float bx = h ? bb.z : bb.x, by = h ? bb.w : bb.y;
        const int m = 2 * m2 + h;
#pragma unroll
        for (int q = 0; q < PT; ++q) {
          yr[q] = __fmaf_rn(bx, a[q][m].x, __fmaf_rn(by, a[q][m].y, yr[q]));
          ya[q] = __fmaf_rn(bx, a[q][m].y, ya[q]);
          yb[q] = __fmaf_rn(by, a[q][m].x, yb[q]);
        }
      }
    }
#pragma unroll
    for (int q = 0; q < PT; ++q) {
      const float yi = __fsub_rn(ya[q], yb[q]);
      n[q] = __fmaf_rn(yr[q], yr[q], __fmul_rn(yi, yi));
    }
  };
  const int Kf = j.Kf, Kn = j.Kn, kphd = j.kphd, kmn = j.kmn;
  // E_n columns: MUSIC and EV sums (PHD, when present, reads the last of them)
  for (int k = 0; k < Kn; ++k) {
    column(k);
    const float w = w32[k];
#pragma unroll
    for (int q = 0; q < PT; ++q) {
      dm[q] = __fadd_rn(dm[q], n[q]);
      de[q] = __fmaf_rn(w, n[q], de[q]);
    }
  }
  if (Kn > 0 && kphd == Kn - 1) {
#pragma unroll
    for (int q = 0; q < PT; ++q) dp[q] = n[q];
  }
  // remaining single columns: v_min without E_n, valph
  for (int k = Kn; k < Kf; ++k) {
    column(k);
    if (k == kphd) {
#pragma unroll
      for (int q = 0; q < PT; ++q) dp[q] = n[q];
    }
    if (k == kmn) {
#pragma unroll
      for (int q = 0; q < PT; ++q) dn[q] = n[q];
    }
  }
  finish_points<PT, Src, kExt>(j, dp, dm, de, dn, L, k0, sh, src, w32, thr_, tags, tag);
}

// Paired FP32 arithmetic on two values in one 64-bit register pair (lo, hi).
__device__ __forceinline__ uint64_t f2pack(float lo, float hi) {
  return (uint64_t)__float_as_uint(lo) | ((uint64_t)__float_as_uint(hi) << 32);
}
__device__ __forceinline__ float f2lo(uint64_t v) { return __uint_as_float((uint32_t)v); }
__device__ __forceinline__ float f2hi(uint64_t v) { return __uint_as_float((uint32_t)(v >> 32)); }
__device__ __forceinline__ uint64_t f2fma(uint64_t a, uint64_t b, uint64_t c) {
  uint64_t d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
  return d;
}
__device__ __forceinline__ uint64_t f2mul(uint64_t a, uint64_t b) {
  uint64_t d;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ uint64_t f2add(uint64_t a, uint64_t b) {
  uint64_t d;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ uint64_t f2sub(uint64_t a, uint64_t b) {
  uint64_t d;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}

// contract_points in the paired form: the PT points (PT even) are taken two at a time, ax[p][m] /
// ay[p][m] holding Re / Im of a_m at points k0 + 2p and k0 + 2p + 1. Per element and pair, four
// paired FMAs: yr += bx ax + by ay, yi_a += bx ay, yi_b += by ax (yi = yi_a - yi_b at the end of the
// column), so every FMA of the contraction is half an instruction. Readouts, thresholds and the
// refinement queue are those of contract_points.
template <int MP, int PT, class Src, bool kExt = false>
__device__ __forceinline__ void contract_points2(const float4 *Bd, const ScanJob &j, const uint64_t (&ax)[PT / 2][MP],
                                                 const uint64_t (&ay)[PT / 2][MP], int L, int k0, ScanShared &sh,
                                                 const Src &src, const float *w32x = nullptr,
                                                 const float *thrx = nullptr, uint8_t *tags = nullptr, int tag = 0) {
  static_assert(PT % 2 == 0, "points are paired");
  constexpr int HP = PT / 2;
  const float *w32 = kExt ? w32x : sh.w32;
  const float *thr_ = kExt ? thrx : sh.thr;
  uint64_t dm[HP], de[HP], dp[HP], dn[HP], n[HP];
#pragma unroll
  for (int q = 0; q < HP; ++q) dm[q] = de[q] = dp[q] = dn[q] = n[q] = 0ull;
  auto column = [&](int k) {
    uint64_t yr[HP], ya[HP], yb[HP];
#pragma unroll
    for (int q = 0; q < HP; ++q) yr[q] = ya[q] = yb[q] = 0ull;
    const float4 *b4 = Bd + k * MP;
#pragma unroll
    for (int m = 0; m < MP; ++m) {
      const float4 bb = b4[m];
      const uint64_t bxx = f2pack(bb.x, bb.y), byy = f2pack(bb.z, bb.w);
#pragma unroll
      for (int q = 0; q < HP; ++q) {
        yr[q] = f2fma(bxx, ax[q][m], f2fma(byy, ay[q][m], yr[q]));
        ya[q] = f2fma(bxx, ay[q][m], ya[q]);
        yb[q] = f2fma(byy, ax[q][m], yb[q]);
      }
    }
#pragma unroll
    for (int q = 0; q < HP; ++q) {
      const uint64_t yi = f2sub(ya[q], yb[q]);
      n[q] = f2fma(yr[q], yr[q], f2mul(yi, yi));
    }
  };
  const int Kf = j.Kf, Kn = j.Kn, kphd = j.kphd, kmn = j.kmn;
  for (int k = 0; k < Kn; ++k) {
    column(k);
    const float w = w32[k];
    const uint64_t ww = f2pack(w, w);
#pragma unroll
    for (int q = 0; q < HP; ++q) {
      dm[q] = f2add(dm[q], n[q]);
      de[q] = f2fma(ww, n[q], de[q]);
    }
  }
  if (Kn > 0 && kphd == Kn - 1) {
#pragma unroll
    for (int q = 0; q < HP; ++q) dp[q] = n[q];
  }
  for (int k = Kn; k < Kf; ++k) {
    column(k);
    if (k == kphd) {
#pragma unroll
      for (int q = 0; q < HP; ++q) dp[q] = n[q];
    }
    if (k == kmn) {
#pragma unroll
      for (int q = 0; q < HP; ++q) dn[q] = n[q];
    }
  }
  float fp[PT], fm[PT], fe[PT], fn[PT];
#pragma unroll
  for (int q = 0; q < HP; ++q) {
    fp[2 * q] = f2lo(dp[q]), fp[2 * q + 1] = f2hi(dp[q]);
    fm[2 * q] = f2lo(dm[q]), fm[2 * q + 1] = f2hi(dm[q]);
    fe[2 * q] = f2lo(de[q]), fe[2 * q + 1] = f2hi(de[q]);
    fn[2 * q] = f2lo(dn[q]), fn[2 * q + 1] = f2hi(dn[q]);
  }
  finish_points<PT, Src, kExt>(j, fp, fm, fe, fn, L, k0, sh, src, w32, thr_, tags, tag);
}

// ---------------------------------------------------------------------------------------------
// ULA scan by blocked Horner evaluation (MP <= 16). For a ULA the steering phasors are powers of
// z = e^{j pi sin theta}, so y_k = sum_m conj(f_mk) z^m is a polynomial in z, and
//     conj(y_k) = sum_m f_mk w^m,  w = conj(z),
// evaluated in blocks of four elements: Q_i = ((f_{4i+3} w + f_{4i+2}) w + f_{4i+1}) w + f_{4i}, then
// conj(y_k) = (((Q_{NB-1} w4 + Q_{NB-2}) w4 + ...) w4 + Q_0 with w4 = conj(z^4). Both w and w4 come
// from exact integer phases (phasor_q32 of S_k and 4 S_k), so a thread needs two phasors per point
// instead of M, and 15 complex multiply-adds per column at M = 16 (the direct sum takes 16). The
// Horner chains are three steps long, which keeps the rounding error within the ~4 eps per term
// on which the refinement threshold rests (an FP32 emulation over 18001-point grids and M = 16
// noise subspaces gave at most 2.6 eps sum_m |f_mk|, the direct sum 4.3). |conj(y)|^2 = |y|^2, so
// the readouts and the refinement are those of the direct form.
// One step u <- u w + c: Re = ur wr - ui wi + cr, Im = ur wi + ui wr + ci, with wn = -wi held so
// that no negation is needed: four FMAs, two per component.
struct HornerW1 {
  float r1, i1, n1, r4, i4, n4;   // Re w, Im w, -Im w; the same for w4
};
struct HornerW2 {
  uint64_t r1, i1, n1, r4, i4, n4;   // HornerW1 of two points, paired
};

__device__ __forceinline__ void hstep1(float &ur, float &ui, float wr, float wi, float wn, float cr, float ci) {
  const float r = __fmaf_rn(ur, wr, __fmaf_rn(ui, wn, cr));
  ui = __fmaf_rn(ur, wi, __fmaf_rn(ui, wr, ci));
  ur = r;
}
__device__ __forceinline__ void hstep2(uint64_t &ur, uint64_t &ui, uint64_t wr, uint64_t wi, uint64_t wn, uint64_t cr,
                                       uint64_t ci) {
  const uint64_t r = f2fma(ur, wr, f2fma(ui, wn, cr));
  ui = f2fma(ur, wi, f2fma(ui, wr, ci));
  ur = r;
}

// w and w4 of the points k0 .. k0+PT-1 (those < L; the others get phase 0).
template <int PT>
__device__ __forceinline__ void ula_horner(const uint32_t *S, int L, int k0, HornerW1 (&w)[PT]) {
#pragma unroll
  for (int q = 0; q < PT; ++q) {
    const uint32_t step = (k0 + q < L) ? S[k0 + q] : 0u;
    const float2 z1 = phasor_q32(step), z4 = phasor_q32(4u * step);
    w[q] = HornerW1{z1.x, -z1.y, z1.y, z4.x, -z4.y, z4.y};
  }
}
template <int PT>
__device__ __forceinline__ void ula_horner2(const uint32_t *S, int L, int k0, HornerW2 (&w)[PT / 2]) {
  HornerW1 v[PT];
  ula_horner<PT>(S, L, k0, v);
#pragma unroll
  for (int q = 0; q < PT / 2; ++q) {
    const HornerW1 &a = v[2 * q], &b = v[2 * q + 1];
    w[q] = HornerW2{f2pack(a.r1, b.r1), f2pack(a.i1, b.i1), f2pack(a.n1, b.n1),
                    f2pack(a.r4, b.r4), f2pack(a.i4, b.i4), f2pack(a.n4, b.n4)};
  }
}

// n = |y_k|^2 of column k for PT points (factor Bs[k][m] = (bx, by), read two elements at a time).
template <int MP, int PT>
__device__ __forceinline__ void horner_column1(const float2 *Bs, int k, const HornerW1 (&w)[PT], float (&n)[PT]) {
  static_assert(MP % 4 == 0, "blocks of four elements");
  constexpr int NB = MP / 4;
  const float4 *b2 = reinterpret_cast<const float4 *>(Bs + k * MP);
  float ur[PT], ui[PT];
#pragma unroll
  for (int i = NB - 1; i >= 0; --i) {
    const float4 c23 = b2[2 * i + 1], c01 = b2[2 * i];   // (f_{4i+2}, f_{4i+3}), (f_{4i}, f_{4i+1})
    float qr[PT], qi[PT];
#pragma unroll
    for (int q = 0; q < PT; ++q) {
      qr[q] = c23.z, qi[q] = c23.w;
      hstep1(qr[q], qi[q], w[q].r1, w[q].i1, w[q].n1, c23.x, c23.y);
      hstep1(qr[q], qi[q], w[q].r1, w[q].i1, w[q].n1, c01.z, c01.w);
      hstep1(qr[q], qi[q], w[q].r1, w[q].i1, w[q].n1, c01.x, c01.y);
      if (i == NB - 1) {
        ur[q] = qr[q], ui[q] = qi[q];
      } else {
        hstep1(ur[q], ui[q], w[q].r4, w[q].i4, w[q].n4, qr[q], qi[q]);
      }
    }
  }
#pragma unroll
  for (int q = 0; q < PT; ++q) n[q] = __fmaf_rn(ur[q], ur[q], __fmul_rn(ui[q], ui[q]));
}

// The same operations on pairs of points (factor Bd[k][m] = (bx, bx, by, by)).
template <int MP, int HP>
__device__ __forceinline__ void horner_column2(const float4 *Bd, int k, const HornerW2 (&w)[HP], uint64_t (&n)[HP]) {
  static_assert(MP % 4 == 0, "blocks of four elements");
  constexpr int NB = MP / 4;
  // each element as two 64-bit operands (bx, bx) and (by, by), straight from one 16-byte load
  const ulonglong2 *b4 = reinterpret_cast<const ulonglong2 *>(Bd + k * MP);
  uint64_t ur[HP], ui[HP];
#pragma unroll
  for (int i = NB - 1; i >= 0; --i) {
    const ulonglong2 c3 = b4[4 * i + 3], c2 = b4[4 * i + 2], c1 = b4[4 * i + 1], c0 = b4[4 * i];
    uint64_t qr[HP], qi[HP];
#pragma unroll
    for (int q = 0; q < HP; ++q) {
      qr[q] = c3.x, qi[q] = c3.y;
      hstep2(qr[q], qi[q], w[q].r1, w[q].i1, w[q].n1, c2.x, c2.y);
      hstep2(qr[q], qi[q], w[q].r1, w[q].i1, w[q].n1, c1.x, c1.y);
      hstep2(qr[q], qi[q], w[q].r1, w[q].i1, w[q].n1, c0.x, c0.y);
      if (i == NB - 1) {
        ur[q] = qr[q], ui[q] = qi[q];
      } else {
        hstep2(ur[q], ui[q], w[q].r4, w[q].i4, w[q].n4, qr[q], qi[q]);
      }
    }
  }
#pragma unroll
  for (int q = 0; q < HP; ++q) n[q] = f2fma(ur[q], ur[q], f2mul(ui[q], ui[q]));
}

// contract_points with the blocked Horner columns (same readouts, thresholds and queue).
template <int MP, int PT, class Src, bool kExt = false>
__device__ __forceinline__ void contract_horner(const float2 *Bs, const ScanJob &j, const HornerW1 (&w)[PT], int L,
                                                int k0, ScanShared &sh, const Src &src, const float *w32x = nullptr,
                                                const float *thrx = nullptr, uint8_t *tags = nullptr, int tag = 0) {
  const float *w32 = kExt ? w32x : sh.w32;
  const float *thr_ = kExt ? thrx : sh.thr;
  float dm[PT], de[PT], dp[PT], dn[PT], n[PT];
#pragma unroll
  for (int q = 0; q < PT; ++q) dm[q] = de[q] = dp[q] = dn[q] = n[q] = 0.f;
  const int Kf = j.Kf, Kn = j.Kn, kphd = j.kphd, kmn = j.kmn;
  for (int k = 0; k < Kn; ++k) {
    horner_column1<MP, PT>(Bs, k, w, n);
    const float wk = w32[k];
#pragma unroll
    for (int q = 0; q < PT; ++q) {
      dm[q] = __fadd_rn(dm[q], n[q]);
      de[q] = __fmaf_rn(wk, n[q], de[q]);
    }
  }
  if (Kn > 0 && kphd == Kn - 1) {
#pragma unroll
    for (int q = 0; q < PT; ++q) dp[q] = n[q];
  }
  for (int k = Kn; k < Kf; ++k) {
    horner_column1<MP, PT>(Bs, k, w, n);
    if (k == kphd) {
#pragma unroll
      for (int q = 0; q < PT; ++q) dp[q] = n[q];
    }
    if (k == kmn) {
#pragma unroll
      for (int q = 0; q < PT; ++q) dn[q] = n[q];
    }
  }
  finish_points<PT, Src, kExt>(j, dp, dm, de, dn, L, k0, sh, src, w32, thr_, tags, tag);
}

template <int MP, int PT, class Src, bool kExt = false>
__device__ __forceinline__ void contract_horner2(const float4 *Bd, const ScanJob &j, const HornerW2 (&w)[PT / 2], int L,
                                                 int k0, ScanShared &sh, const Src &src, const float *w32x = nullptr,
                                                 const float *thrx = nullptr, uint8_t *tags = nullptr, int tag = 0) {
  static_assert(PT % 2 == 0, "points are paired");
  constexpr int HP = PT / 2;
  const float *w32 = kExt ? w32x : sh.w32;
  const float *thr_ = kExt ? thrx : sh.thr;
  uint64_t dm[HP], de[HP], dp[HP], dn[HP], n[HP];
#pragma unroll
  for (int q = 0; q < HP; ++q) dm[q] = de[q] = dp[q] = dn[q] = n[q] = 0ull;
  const int Kf = j.Kf, Kn = j.Kn, kphd = j.kphd, kmn = j.kmn;
  for (int k = 0; k < Kn; ++k) {
    horner_column2<MP, HP>(Bd, k, w, n);
    const float wk = w32[k];
    const uint64_t ww = f2pack(wk, wk);
#pragma unroll
    for (int q = 0; q < HP; ++q) {
      dm[q] = f2add(dm[q], n[q]);
      de[q] = f2fma(ww, n[q], de[q]);
    }
  }
  if (Kn > 0 && kphd == Kn - 1) {
#pragma unroll
    for (int q = 0; q < HP; ++q) dp[q] = n[q];
  }
  for (int k = Kn; k < Kf; ++k) {
    horner_column2<MP, HP>(Bd, k, w, n);
    if (k == kphd) {
#pragma unroll
      for (int q = 0; q < HP; ++q) dp[q] = n[q];
    }
    if (k == kmn) {
#pragma unroll
      for (int q = 0; q < HP; ++q) dn[q] = n[q];
    }
  }
  float fp[PT], fm[PT], fe[PT], fn[PT];
#pragma unroll
  for (int q = 0; q < HP; ++q) {
    fp[2 * q] = f2lo(dp[q]), fp[2 * q + 1] = f2hi(dp[q]);
    fm[2 * q] = f2lo(dm[q]), fm[2 * q + 1] = f2hi(dm[q]);
    fe[2 * q] = f2lo(de[q]), fe[2 * q + 1] = f2hi(de[q]);
    fn[2 * q] = f2lo(dn[q]), fn[2 * q + 1] = f2hi(dn[q]);
  }
  finish_points<PT, Src, kExt>(j, fp, fm, fe, fn, L, k0, sh, src, w32, thr_, tags, tag);
}

// Steering phasors of the points k0 .. k0+PT-1 (those < L; the others get phase 0) from their
// 32-bit phase steps: a_m, m = 4i + r: a_{4i} and a_r (r = 1..3) from their exact integer phases,
// the rest as the product a_{4i} a_r (one FP32 complex multiply of two polynomial phasors).
template <int MP, int PT>
__device__ __forceinline__ void ula_phasors(const uint32_t *S, int L, int k0, float2 (&a)[PT][MP]) {
  static_assert(MP % 4 == 0, "MP is a multiple of 4");
#pragma unroll
  for (int q = 0; q < PT; ++q) {
    const uint32_t step = (k0 + q < L) ? S[k0 + q] : 0u;
    a[q][0] = make_float2(1.f, 0.f);
#pragma unroll
    for (int r = 1; r < 4; ++r) a[q][r] = phasor_q32((uint32_t)r * step);
#pragma unroll
    for (int i = 1; i < MP / 4; ++i) {
      const float2 A = phasor_q32((uint32_t)(4 * i) * step);
      a[q][4 * i] = A;
#pragma unroll
      for (int r = 1; r < 4; ++r) {
        const float2 z = a[q][r];
        a[q][4 * i + r] = make_float2(fmaf(A.x, z.x, -A.y * z.y), fmaf(A.x, z.y, A.y * z.x));
      }
    }
  }
}

// Evaluates the local points k0 .. k0+PT-1 (those < L) of one job. S may alias a P row of a
// single-readout job: each thread reads its own phase steps before it writes its own outputs.
// Points where any readout falls below its refinement threshold are queued for drain_refinements.
template <int MP, int PT>
__device__ __forceinline__ void scan_points(const float2 *Bs, const ScanJob &j, const uint32_t *S, int L, int k0,
                                            ScanShared &sh) {
  if constexpr (ula_horner_form<MP>()) {
    HornerW1 w[PT];
    ula_horner<PT>(S, L, k0, w);
    contract_horner<MP, PT>(Bs, j, w, L, k0, sh, UlaSource{&j});
  } else {
    float2 a[PT][MP];
    ula_phasors<MP, PT>(S, L, k0, a);
    contract_points<MP, PT>(Bs, j, a, L, k0, sh, UlaSource{&j});
  }
}

// ula_phasors packed for contract_points2 (PT even).
template <int MP, int PT>
__device__ __forceinline__ void ula_phasors2(const uint32_t *S, int L, int k0, uint64_t (&ax)[PT / 2][MP],
                                             uint64_t (&ay)[PT / 2][MP]) {
  float2 a[PT][MP];
  ula_phasors<MP, PT>(S, L, k0, a);
#pragma unroll
  for (int q = 0; q < PT / 2; ++q)
#pragma unroll
    for (int m = 0; m < MP; ++m) {
      ax[q][m] = f2pack(a[2 * q][m].x, a[2 * q + 1][m].x);
      ay[q][m] = f2pack(a[2 * q][m].y, a[2 * q + 1][m].y);
    }
}

template <int MP, int PT>
__device__ __forceinline__ void scan_points2(const float4 *Bd, const ScanJob &j, const uint32_t *S, int L, int k0,
                                             ScanShared &sh) {
  if constexpr (ula_horner_form<MP>()) {
    HornerW2 w[PT / 2];
    ula_horner2<PT>(S, L, k0, w);
    contract_horner2<MP, PT>(Bd, j, w, L, k0, sh, UlaSource{&j});
  } else {
    uint64_t ax[PT / 2][MP], ay[PT / 2][MP];
    ula_phasors2<MP, PT>(S, L, k0, ax, ay);
    contract_points2<MP, PT>(Bd, j, ax, ay, L, k0, sh, UlaSource{&j});
  }
}

}  // namespace scanc
}  // namespace doa
