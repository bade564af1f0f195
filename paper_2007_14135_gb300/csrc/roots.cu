// Root form of the ULA scan (root-MUSIC; beyond the paper, which evaluates the spectrum on a grid).
// On the unit circle, with z = e^{j pi sin theta}, the scan's denominator is a Laurent polynomial:
//   a(theta)^H C a(theta) = sum_{l=-(M-1)}^{M-1} c_l z^l,   c_l = sum_{j-i=l} C_ij,
// and with C = sum_k w_k f_k f_k^H (the readout's factor columns and weights, Table 3),
//   c_l = sum_k w_k sum_n f_nk conj(f_{n+l,k}).
// z^{M-1} D(z) is a polynomial of degree 2M-2 whose roots pair up as z, 1/conj(z); the d roots with
// |z| <= 1 closest to the unit circle give the estimates theta = asin(arg(z) / pi).
//
// Roots by the Aberth-Ehrlich iteration (simultaneous Newton corrections with the repulsion sum
// over the other roots), all corrections computed from the previous iterate, started on the unit
// circle at angles 2 pi i / n + 0.4: first in FP32 on the rounded coefficients (to corrections of
// 1e-6 |z| or the FP32 rounding bound), then in FP64 from there; in FP64 a root counts as converged
// when its correction is below 1e-14 max(1, |z|) or when |p(z)| is within the rounding bound of its
// Horner evaluation,
// 8 n eps sum_t |a_t| |z|^t (clustered roots -- the pairs z, 1/conj(z) near the circle -- cannot be
// resolved further). A converged root keeps its value and takes no further correction; the
// iteration ends when all have converged, 400 iterations at most (else DOA_ENOCONV). One warp per
// (problem, algorithm) job: lanes own coefficients, then roots; the selection runs on lane 0.
#include <math_constants.h>

#include "doa_internal.cuh"

namespace doa {
namespace {

constexpr int kRootWarps = 4;
constexpr int kMaxDeg = 2 * kMaxM - 2;
constexpr int kRootMaxIter = 400;

struct RootShared {
  float2 af[kMaxDeg + 1];   // the coefficients rounded to FP32 (first phase)
  float amf[kMaxDeg + 1];
  float2 zf[kMaxDeg];
  float2 wf[kMaxDeg];
  double2 a[kMaxDeg + 1];   // polynomial coefficients, a[t] multiplies z^t
  double am[kMaxDeg + 1];   // |a_t| (for the rounding bound of the Horner evaluation)
  double2 z[kMaxDeg];       // current roots
  double2 w[kMaxDeg];       // corrections of this iteration
  int conv[kMaxDeg];        // root converged (its correction is no longer computed)
};

__device__ __forceinline__ double2 cadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 fcmul(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ float2 fcadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 fcsub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 fcdiv(float2 a, float2 b) {
  const float inv = __frcp_rn(fmaf(b.x, b.x, b.y * b.y));
  return make_float2(fmaf(a.x, b.x, a.y * b.y) * inv, fmaf(a.y, b.x, -a.x * b.y) * inv);
}
__device__ __forceinline__ double2 csub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ double2 cdiv(double2 a, double2 b) {
  const double inv = __drcp_rn(b.x * b.x + b.y * b.y);
  return make_double2((a.x * b.x + a.y * b.y) * inv, (a.y * b.x - a.x * b.y) * inv);
}
__device__ __forceinline__ double2 crcp(double2 b) {   // 1 / b
  const double inv = __drcp_rn(b.x * b.x + b.y * b.y);
  return make_double2(b.x * inv, -b.y * inv);
}

struct RootJob {
  const double2 *F;   // factor, column-major, ld M
  const double *w;    // EV weights or null
  int M, Kf, Kn, kphd, kmn, alg, d;
};

__device__ __forceinline__ double root_weight(const RootJob &j, int c) {
  switch (j.alg) {
    case DOA_MUSIC: return c < j.Kn ? 1.0 : 0.0;
    case DOA_EV: return c < j.Kn ? (j.w ? j.w[c] : 1.0) : 0.0;
    case DOA_PHD: return c == j.kphd ? 1.0 : 0.0;
    case DOA_MN: return c == j.kmn ? 1.0 : 0.0;
    default: return c < j.Kf ? 1.0 : 0.0;
  }
}

// Writes the d angles (degrees, ascending) of one job to out; returns 0 or DOA_ENOCONV.
__device__ int root_music_warp(const RootJob &j, RootShared &sh, double *out) {
  const int lane = threadIdx.x & 31;
  const int M = j.M, n = 2 * M - 2;
  // coefficients: a[t] = c_{t - (M-1)}
  for (int t = lane; t <= n; t += 32) {
    const int l = t - (M - 1);
    double cr = 0.0, ci = 0.0;
    for (int c = 0; c < j.Kf; ++c) {
      const double wc = root_weight(j, c);
      if (wc == 0.0) continue;
      const double2 *f = j.F + (size_t)c * M;
      double sr = 0.0, si = 0.0;
      for (int q = max(0, -l); q < M && q + l < M; ++q) {   // f_q conj(f_{q+l})
        const double2 x = f[q], y = f[q + l];
        sr = fma(x.x, y.x, fma(x.y, y.y, sr));
        si = fma(x.y, y.x, fma(-x.x, y.y, si));
      }
      cr = fma(wc, sr, cr);
      ci = fma(wc, si, ci);
    }
    sh.a[t] = make_double2(cr, ci);
    sh.am[t] = sqrt(cr * cr + ci * ci);
    sh.af[t] = make_float2((float)cr, (float)ci);
    sh.amf[t] = (float)sh.am[t];
  }
  for (int i = lane; i < n; i += 32) {
    float s, c;
    sincosf(6.283185307179586f * (float)i / (float)n + 0.4f, &s, &c);
    sh.zf[i] = make_float2(c, s);
    sh.wf[i] = make_float2(0.f, 0.f);
    sh.conv[i] = 0;
  }
  __syncwarp();
  int st = DOA_ENOCONV;
  const double2 lead = sh.a[n];
  const bool usable = lead.x * lead.x + lead.y * lead.y > 0.0;
  // first phase, FP32 (the FP64 rate is 1/73 of FP32 here): corrections down to 1e-6 |z| or the
  // FP32 rounding bound of p(z); the FP64 phase then polishes the same roots
  if (usable) {
    for (int it = 0; it < kRootMaxIter; ++it) {
      bool small = true;
      for (int i = lane; i < n; i += 32) {
        if (sh.conv[i]) continue;
        const float2 zi = sh.zf[i];
        const float zm = sqrtf(fmaf(zi.x, zi.x, zi.y * zi.y));
        float2 p = sh.af[n], dp = make_float2(0.f, 0.f);
        float pe = sh.amf[n];
        for (int t = n - 1; t >= 0; --t) {
          dp = fcadd(fcmul(dp, zi), p);
          p = fcadd(fcmul(p, zi), sh.af[t]);
          pe = fmaf(pe, zm, sh.amf[t]);
        }
        float2 rep = make_float2(0.f, 0.f);
        for (int k = 0; k < n; ++k) {
          if (k == i) continue;
          rep = fcadd(rep, fcdiv(make_float2(1.f, 0.f), fcsub(zi, sh.zf[k])));
        }
        const float2 ratio = fcdiv(p, dp);
        const float2 wi = fcdiv(ratio, fcsub(make_float2(1.f, 0.f), fcmul(ratio, rep)));
        sh.wf[i] = wi;
        const float mag = sqrtf(fmaf(wi.x, wi.x, wi.y * wi.y)), res = sqrtf(fmaf(p.x, p.x, p.y * p.y));
        const bool ok = isfinite(mag) && (mag <= 1e-6f * fmaxf(1.f, zm) || res <= 8.f * n * 5.9604645e-08f * pe);
        small = small && ok;
        if (ok) sh.conv[i] = 1;
      }
      __syncwarp();
      for (int i = lane; i < n; i += 32) {
        sh.zf[i] = fcsub(sh.zf[i], sh.wf[i]);
        sh.wf[i] = make_float2(0.f, 0.f);
      }
      __syncwarp();
      if (__all_sync(0xffffffffu, small)) break;
    }
  }
  bool finite_start = true;
  for (int i = lane; i < n; i += 32) finite_start = finite_start && isfinite(sh.zf[i].x) && isfinite(sh.zf[i].y);
  finite_start = __all_sync(0xffffffffu, finite_start);
  for (int i = lane; i < n; i += 32) {
    if (finite_start) {
      sh.z[i] = make_double2((double)sh.zf[i].x, (double)sh.zf[i].y);
    } else {
      double s, c;
      sincos(2.0 * CUDART_PI * (double)i / (double)n + 0.4, &s, &c);
      sh.z[i] = make_double2(c, s);
    }
    sh.w[i] = make_double2(0.0, 0.0);
    sh.conv[i] = 0;
  }
  __syncwarp();
  if (usable) {
    for (int it = 0; it < kRootMaxIter; ++it) {
      bool small = true;
      for (int i = lane; i < n; i += 32) {
        if (sh.conv[i]) continue;                    // converged: no more correction
        const double2 zi = sh.z[i];
        const double zm = sqrt(zi.x * zi.x + zi.y * zi.y);
        double2 p = sh.a[n], dp = make_double2(0.0, 0.0);
        double pe = sh.am[n];
        for (int t = n - 1; t >= 0; --t) {          // Horner for p, p' and the bound sum |a_t| |z|^t
          dp = cadd(cmul(dp, zi), p);
          p = cadd(cmul(p, zi), sh.a[t]);
          pe = fma(pe, zm, sh.am[t]);
        }
        double2 rep = make_double2(0.0, 0.0);       // sum_{k != i} 1 / (z_i - z_k)
        for (int k = 0; k < n; ++k) {
          if (k == i) continue;
          rep = cadd(rep, crcp(csub(zi, sh.z[k])));
        }
        const double2 ratio = cdiv(p, dp);
        const double2 den = csub(make_double2(1.0, 0.0), cmul(ratio, rep));
        const double2 wi = cdiv(ratio, den);
        sh.w[i] = wi;
        const double mag = sqrt(wi.x * wi.x + wi.y * wi.y);
        const double res = sqrt(p.x * p.x + p.y * p.y);
        const bool ok = isfinite(mag) && (mag <= 1e-14 * fmax(1.0, zm) || res <= 8.0 * n * 1.1102230246251565e-16 * pe);
        small = small && ok;
        if (ok) sh.conv[i] = 1;
      }
      __syncwarp();
      for (int i = lane; i < n; i += 32) {
        sh.z[i] = csub(sh.z[i], sh.w[i]);
        sh.w[i] = make_double2(0.0, 0.0);
      }
      __syncwarp();
      if (__all_sync(0xffffffffu, small)) {
        st = 0;
        break;
      }
    }
  }
  if (lane == 0) {
    // the d roots with |z| <= 1 of largest modulus (lower index on a tie), then angles ascending
    double sel[kMaxM];
    int ns = 0;
    if (st == 0) {
      int taken[kMaxM];
      for (int q = 0; q < j.d; ++q) {
        int best = -1;
        double bm = -1.0;
        for (int i = 0; i < n; ++i) {
          const double2 zi = sh.z[i];
          const double m = sqrt(zi.x * zi.x + zi.y * zi.y);
          if (!(m <= 1.0) || !(m > bm)) continue;
          bool used = false;
          for (int r = 0; r < ns; ++r) used = used || taken[r] == i;
          if (used) continue;
          best = i;
          bm = m;
        }
        if (best < 0) break;
        taken[ns] = best;
        const double2 zb = sh.z[best];
        const double sx = fmin(fmax(atan2(zb.y, zb.x) / CUDART_PI, -1.0), 1.0);
        sel[ns++] = asin(sx) * (180.0 / CUDART_PI);
      }
      for (int a = 1; a < ns; ++a) {
        const double v = sel[a];
        int b = a - 1;
        while (b >= 0 && sel[b] > v) {
          sel[b + 1] = sel[b];
          --b;
        }
        sel[b + 1] = v;
      }
      if (ns < j.d) st = DOA_ENOCONV;
    }
    for (int q = 0; q < j.d; ++q) out[q] = q < ns ? sel[q] : CUDART_NAN;
  }
  __syncwarp();
  return st;
}

__global__ void __launch_bounds__(32 * kRootWarps) roots_batch_kernel(const uint8_t *plan, uint8_t *ws, int *status) {
  __shared__ RootShared sh[kRootWarps];
  const PlanHeader *h = reinterpret_cast<const PlanHeader *>(plan);
  const int warp = threadIdx.x >> 5;
  const int job = blockIdx.x * kRootWarps + warp;
  if (job >= h->njobs) return;
  const PlanJob &jb = reinterpret_cast<const PlanJob *>(plan + h->off_job)[job];
  const PlanProblem &pp = reinterpret_cast<const PlanProblem *>(plan + h->off_prob)[jb.prob];
  if (!pp.p.root_angle || pp.p.d < 1) return;
  if (status[jb.prob] != 0) return;     // no decomposition to root
  RootJob j{};
  j.F = reinterpret_cast<const double2 *>(ws + pp.fac_off);
  j.w = pp.Kn > 0 && pp.slot[DOA_EV] >= 0
            ? reinterpret_cast<const double *>(ws + pp.fac_off) + 2 * pp.p.M * (pp.p.M + 1)
            : nullptr;
  j.M = pp.p.M;
  j.Kf = pp.Kf;
  j.Kn = pp.Kn;
  j.kphd = pp.kphd;
  j.kmn = pp.kmn;
  j.alg = jb.alg;
  j.d = pp.p.d;
  const int st = root_music_warp(j, sh[warp], pp.p.root_angle + (size_t)jb.slot * pp.p.d);
  if (st && (threadIdx.x & 31) == 0) atomicCAS(status + jb.prob, 0, st);
}

__global__ void __launch_bounds__(32) roots_single_kernel(RootJob j, double *theta, int *info) {
  __shared__ RootShared sh;
  const int st = root_music_warp(j, sh, theta);
  if (threadIdx.x == 0) *info = st ? -st : 0;
}

}  // namespace

cudaError_t launch_roots_batch(const uint8_t *plan_dev, const PlanHeader &h, uint8_t *ws, int *status, cudaStream_t s) {
  if (h.nroots == 0 || h.njobs == 0) return cudaSuccess;
  roots_batch_kernel<<<(h.njobs + kRootWarps - 1) / kRootWarps, 32 * kRootWarps, 0, s>>>(plan_dev, ws, status);
  return cudaGetLastError();
}

cudaError_t launch_roots_single(const double2 *B, int M, int K, int d, double *theta, int *info, cudaStream_t s) {
  RootJob j{};
  j.F = B;
  j.M = M;
  j.Kf = K;
  j.Kn = K;
  j.kphd = j.kmn = -1;
  j.alg = -1;
  j.d = d;
  roots_single_kernel<<<1, 32, 0, s>>>(j, theta, info);
  return cudaGetLastError();
}

}  // namespace doa
