// Sub-grid refinement of picked peaks (beyond the paper's Step-6, which stops at the grid): the
// local minimiser of a readout's denominator next to each grid peak, in FP64.
//
// den(theta) = sum_c w_c |y_c|^2, y_c = f_c^H a(theta), over the factor columns the readout reads
// (MUSIC: E_n, w = 1; EV: E_n, w = 1/lambda; PHD: v_min; MN: valph; a single-call factor B: all
// columns, w = 1), which equals a^H C a for the weighting matrix C of Table 3. Its derivatives come
// from the steering vector's: with y', y'' = F^H a', F^H a'',
//   den'  = 2 sum_c w_c Re(conj(y_c) y'_c),   den'' = 2 sum_c w_c (Re(conj(y_c) y''_c) + |y'_c|^2).
//
// ULA (steering a_m = exp(j pi m sin theta), phases from the exact 64-bit phase step of sin theta
// as in the scan's refinement): bracketed Newton on den' = 0 inside [theta_{k-1}, theta_{k+1}] --
// the bracket shrinks by the sign of den'; a Newton step shorter than 1e-13 rad (with den'' > 0)
// is taken and ends the iteration; otherwise the Newton point is taken if strictly inside the
// bracket, else the bracket's midpoint; stop below a 1e-13 rad move or after 60 steps.
//
// Geometry (Eq. 2 as printed, positions relative to their centroid -- a common phase that leaves
// den unchanged): damped Newton in (azimuth, elevation) inside the box of one grid step around the
// peak, with gradient g and Hessian H from the first and second derivatives of the element phases
// t_m = p_m . u(theta, phi). A step is -H^-1 g when H is positive definite (taken as it is when
// shorter than 1e-6 rad in both angles), else the steepest-descent direction scaled to the box
// half-width, halved up to 40 times until den does not increase; stop below a 1e-13 rad move, when
// no halving decreases den, or after 60 steps.
//
// One warp per (problem, algorithm) job: lanes own elements for the steering vector and its
// derivatives (shared memory), then factor columns for the contractions, and a shuffle reduction
// gives every lane the same den, gradient and Hessian, so all lanes take the same decisions.
// In the batch the iteration starts from the vertex of the parabola through the FP32 spectrum's
// 1/P at the peak and its neighbours (per axis in 2-D), which leaves Newton one or two steps; the
// local minimiser it converges to does not depend on the start.
#include <float.h>
#include <math_constants.h>

#include "doa_internal.cuh"

namespace doa {
namespace {

constexpr int kRefWarps = 4;
constexpr int kRefMaxIter = 60;
constexpr double kD2R = 3.14159265358979323846 / 180.0;
constexpr double kPi = 3.14159265358979323846;

struct RefineJob {
  const double2 *F;      // factor, column-major, ld M
  const double *w;       // EV weights (Kn) or null
  int M, Kf, Kn, kphd, kmn;
  int alg;               // readout: DOA_PHD .. DOA_MN, or -1 = all columns unweighted (single call)
  // ULA grid
  double lo, step;
  // geometry (pos != null)
  const double *pos;
  double cx, cy, cz;
  double az_lo, az_step, el_lo, el_step;
  int La, Le, wrap;
  const float *P;        // the job's FP32 spectrum (start point), or null: start at the grid point
};

// Offset, in grid steps, of the vertex of the parabola through 1/P at points a, b (the peak), c;
// 0 when the three do not bracket a minimum of 1/P.
__device__ __forceinline__ double vertex_offset(float pa, float pb, float pc) {
  const double da = 1.0 / (double)pa, db = 1.0 / (double)pb, dc = 1.0 / (double)pc;
  const double curv = da - 2.0 * db + dc;
  if (!(curv > 0.0) || !(db <= da) || !(db <= dc)) return 0.0;
  return fmin(fmax(0.5 * (da - dc) / curv, -0.9), 0.9);
}

struct RefShared {
  double2 v[6][kMaxM];   // a and its derivatives (1-D: a, a', a''; 2-D: a, a_t, a_p, a_tt, a_tp, a_pp)
};

__device__ __forceinline__ double2 cmul_j(double s, double2 a) {   // (j s) a
  return make_double2(-s * a.y, s * a.x);
}

__device__ __forceinline__ double col_weight(const RefineJob &j, int c) {
  switch (j.alg) {
    case DOA_MUSIC: return c < j.Kn ? 1.0 : 0.0;
    case DOA_EV: return c < j.Kn ? (j.w ? j.w[c] : 1.0) : 0.0;
    case DOA_PHD: return c == j.kphd ? 1.0 : 0.0;
    case DOA_MN: return c == j.kmn ? 1.0 : 0.0;
    default: return c < j.Kf ? 1.0 : 0.0;
  }
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
  return v;
}

// conj(f_c)^T v for lane-owned column c (v in shared memory).
__device__ __forceinline__ double2 col_dot(const RefineJob &j, int c, const double2 *v) {
  const double2 *f = j.F + (size_t)c * j.M;
  double yr = 0.0, yi = 0.0;
  for (int m = 0; m < j.M; ++m) {
    const double2 b = f[m], a = v[m];
    yr = fma(b.x, a.x, fma(b.y, a.y, yr));
    yi = fma(b.x, a.y, fma(-b.y, a.x, yi));
  }
  return make_double2(yr, yi);
}

// ---- ULA ------------------------------------------------------------------------------------
// den, den', den'' at theta (radians).
__device__ void ula_eval(const RefineJob &j, double th, RefShared &sh, double &f, double &f1, double &f2) {
  const int lane = threadIdx.x & 31;
  double s, c;
  sincos(th, &s, &c);
  const uint64_t step = phase_step64_of_sin(s);
  for (int m = lane; m < j.M; m += 32) {
    const double2 a = phasor_q64((uint64_t)m * step);
    const double pm = kPi * (double)m;
    sh.v[0][m] = a;
    sh.v[1][m] = cmul_j(pm * c, a);
    const double2 ja = cmul_j(-pm * s, a);
    const double q = (pm * c) * (pm * c);
    sh.v[2][m] = make_double2(ja.x - q * a.x, ja.y - q * a.y);
  }
  __syncwarp();
  double pf = 0.0, p1 = 0.0, p2 = 0.0;
  for (int col = lane; col < j.Kf; col += 32) {
    const double wc = col_weight(j, col);
    if (wc == 0.0) continue;
    const double2 y = col_dot(j, col, sh.v[0]), y1 = col_dot(j, col, sh.v[1]), y2 = col_dot(j, col, sh.v[2]);
    pf += wc * (y.x * y.x + y.y * y.y);
    p1 += 2.0 * wc * (y.x * y1.x + y.y * y1.y);
    p2 += 2.0 * wc * ((y.x * y2.x + y.y * y2.y) + (y1.x * y1.x + y1.y * y1.y));
  }
  __syncwarp();
  f = warp_sum(pf);
  f1 = warp_sum(p1);
  f2 = warp_sum(p2);
}

__device__ double refine_ula_warp(const RefineJob &j, int k, RefShared &sh) {
  const double t0 = __dadd_rn(j.lo, __dmul_rn((double)(k - 1), j.step));
  const double t1 = __dadd_rn(j.lo, __dmul_rn((double)k, j.step));
  const double t2 = __dadd_rn(j.lo, __dmul_rn((double)(k + 1), j.step));
  double x_lo = __dmul_rn(fmin(t0, t2), kD2R), x_hi = __dmul_rn(fmax(t0, t2), kD2R), x = __dmul_rn(t1, kD2R);
  if (j.P) x = (t1 + vertex_offset(j.P[k - 1], j.P[k], j.P[k + 1]) * j.step) * kD2R;
  for (int it = 0; it < kRefMaxIter; ++it) {
    double f, f1, f2;
    ula_eval(j, x, sh, f, f1, f2);
    if (f1 > 0.0) x_hi = x; else x_lo = x;
    if (f2 > 0.0 && fabs(f1) < 1e-13 * f2) {
      x -= f1 / f2;
      break;
    }
    double xn = (f2 > 0.0) ? x - f1 / f2 : CUDART_NAN;
    if (!(xn > x_lo && xn < x_hi)) xn = 0.5 * (x_lo + x_hi);
    const double dx = fabs(xn - x);
    x = xn;
    if (dx < 1e-13) break;
  }
  return x / kD2R;
}

// ---- geometry -------------------------------------------------------------------------------
// den and (when deriv) its gradient and Hessian (H[0] = tt, H[1] = tp, H[2] = pp) at (th, ph).
__device__ double geo_eval(const RefineJob &j, double th, double ph, bool deriv, RefShared &sh, double *g,
                           double *H) {
  const int lane = threadIdx.x & 31;
  double st, ct, sp, cp;
  sincos(th, &st, &ct);
  sincos(ph, &sp, &cp);
  const double u0 = st * sp, u1 = ct * sp, u2 = cp;
  const double tp2 = 2.0 * kPi;
  for (int m = lane; m < j.M; m += 32) {
    const double px = j.pos[3 * m] - j.cx, py = j.pos[3 * m + 1] - j.cy, pz = j.pos[3 * m + 2] - j.cz;
    const double t = px * u0 + py * u1 + pz * u2;
    const double fr = t - rint(t);
    const double2 a = phasor_q64((uint64_t)__double2ll_rn(fr * 4611686018427387904.0) << 2);
    sh.v[0][m] = a;
    if (deriv) {
      const double t_t = px * (ct * sp) + py * (-st * sp);
      const double t_p = px * (st * cp) + py * (ct * cp) + pz * (-sp);
      const double t_tt = px * (-st * sp) + py * (-ct * sp);
      const double t_tp = px * (ct * cp) + py * (-st * cp);
      const double t_pp = px * (-st * sp) + py * (-ct * sp) + pz * (-cp);
      sh.v[1][m] = cmul_j(tp2 * t_t, a);
      sh.v[2][m] = cmul_j(tp2 * t_p, a);
      double2 q = cmul_j(tp2 * t_tt, a);
      double r = tp2 * tp2 * t_t * t_t;
      sh.v[3][m] = make_double2(q.x - r * a.x, q.y - r * a.y);
      q = cmul_j(tp2 * t_tp, a);
      r = tp2 * tp2 * t_t * t_p;
      sh.v[4][m] = make_double2(q.x - r * a.x, q.y - r * a.y);
      q = cmul_j(tp2 * t_pp, a);
      r = tp2 * tp2 * t_p * t_p;
      sh.v[5][m] = make_double2(q.x - r * a.x, q.y - r * a.y);
    }
  }
  __syncwarp();
  double pf = 0.0, pg0 = 0.0, pg1 = 0.0, ph0 = 0.0, ph1 = 0.0, ph2 = 0.0;
  for (int col = lane; col < j.Kf; col += 32) {
    const double wc = col_weight(j, col);
    if (wc == 0.0) continue;
    const double2 y = col_dot(j, col, sh.v[0]);
    pf += wc * (y.x * y.x + y.y * y.y);
    if (deriv) {
      const double2 yt = col_dot(j, col, sh.v[1]), yp = col_dot(j, col, sh.v[2]);
      const double2 ytt = col_dot(j, col, sh.v[3]), ytp = col_dot(j, col, sh.v[4]), ypp = col_dot(j, col, sh.v[5]);
      pg0 += 2.0 * wc * (y.x * yt.x + y.y * yt.y);
      pg1 += 2.0 * wc * (y.x * yp.x + y.y * yp.y);
      ph0 += 2.0 * wc * ((y.x * ytt.x + y.y * ytt.y) + (yt.x * yt.x + yt.y * yt.y));
      ph1 += 2.0 * wc * ((y.x * ytp.x + y.y * ytp.y) + (yt.x * yp.x + yt.y * yp.y));
      ph2 += 2.0 * wc * ((y.x * ypp.x + y.y * ypp.y) + (yp.x * yp.x + yp.y * yp.y));
    }
  }
  __syncwarp();
  const double f = warp_sum(pf);
  if (deriv) {
    g[0] = warp_sum(pg0);
    g[1] = warp_sum(pg1);
    H[0] = warp_sum(ph0);
    H[1] = warp_sum(ph1);
    H[2] = warp_sum(ph2);
  }
  return f;
}

__device__ void refine_geo_warp(const RefineJob &j, int flat, RefShared &sh, double *out) {
  const int l = flat / j.La, k = flat - l * j.La;
  double x0 = __dmul_rn(__dadd_rn(j.az_lo, __dmul_rn((double)k, j.az_step)), kD2R);
  double x1 = __dmul_rn(__dadd_rn(j.el_lo, __dmul_rn((double)l, j.el_step)), kD2R);
  const double hw0 = fabs(j.az_step) * kD2R, hw1 = fabs(j.el_step) * kD2R;
  const double bl0 = x0 - hw0, bh0 = x0 + hw0, bl1 = x1 - hw1, bh1 = x1 + hw1;
  if (j.P) {
    const float pc = j.P[flat];
    const int km = k > 0 ? k - 1 : (j.wrap ? j.La - 1 : -1), kp = k + 1 < j.La ? k + 1 : (j.wrap ? 0 : -1);
    if (km >= 0 && kp >= 0 && km != kp)
      x0 += vertex_offset(j.P[(size_t)l * j.La + km], pc, j.P[(size_t)l * j.La + kp]) * j.az_step * kD2R;
    if (l > 0 && l + 1 < j.Le)
      x1 += vertex_offset(j.P[(size_t)(l - 1) * j.La + k], pc, j.P[(size_t)(l + 1) * j.La + k]) * j.el_step * kD2R;
  }
  for (int it = 0; it < kRefMaxIter; ++it) {
    double g[2], H[3];
    const double f = geo_eval(j, x0, x1, true, sh, g, H);
    const double det = H[0] * H[2] - H[1] * H[1];
    double d0, d1;
    if (H[0] > 0.0 && det > 0.0) {
      d0 = -(H[2] * g[0] - H[1] * g[1]) / det;
      d1 = -(H[0] * g[1] - H[1] * g[0]) / det;
      if (fmax(fabs(d0), fabs(d1)) < 1e-6) {
        const double n0 = fmin(fmax(x0 + d0, bl0), bh0), n1 = fmin(fmax(x1 + d1, bl1), bh1);
        const double mv = fmax(fabs(n0 - x0), fabs(n1 - x1));
        x0 = n0;
        x1 = n1;
        if (mv < 1e-13) break;
        continue;
      }
    } else {
      const double gn = sqrt(g[0] * g[0] + g[1] * g[1]);
      const double wdt = fmax(hw0, hw1);
      d0 = gn > 0.0 ? -g[0] / gn * wdt : 0.0;
      d1 = gn > 0.0 ? -g[1] / gn * wdt : 0.0;
    }
    double t = 1.0, n0 = x0, n1 = x1;
    bool accepted = false;
    for (int h = 0; h <= 40; ++h) {
      n0 = fmin(fmax(x0 + t * d0, bl0), bh0);
      n1 = fmin(fmax(x1 + t * d1, bl1), bh1);
      if (geo_eval(j, n0, n1, false, sh, nullptr, nullptr) <= f) {
        accepted = true;
        break;
      }
      t *= 0.5;
    }
    if (!accepted) break;
    const double mv = fmax(fabs(n0 - x0), fabs(n1 - x1));
    x0 = n0;
    x1 = n1;
    if (mv < 1e-13) break;
  }
  out[0] = x0 / kD2R;
  out[1] = x1 / kD2R;
}

// Refines peaks idx[0..n) of one job; out: n angles (ULA) or n (azimuth, elevation) pairs.
__device__ void refine_job_warp(const RefineJob &j, const int *idx, int n, double *out, RefShared &sh) {
  const int lane = threadIdx.x & 31;
  for (int q = 0; q < n; ++q) {
    const int k = idx[q];
    if (j.pos) {
      double r[2];
      refine_geo_warp(j, k, sh, r);
      if (lane == 0) {
        out[2 * q] = r[0];
        out[2 * q + 1] = r[1];
      }
    } else {
      const double th = refine_ula_warp(j, k, sh);
      if (lane == 0) out[q] = th;
    }
    __syncwarp();
  }
}

__device__ void set_centroid(RefineJob &j) {
  double cx = 0.0, cy = 0.0, cz = 0.0;
  for (int m = 0; m < j.M; ++m) {
    cx += j.pos[3 * m];
    cy += j.pos[3 * m + 1];
    cz += j.pos[3 * m + 2];
  }
  j.cx = cx / j.M;
  j.cy = cy / j.M;
  j.cz = cz / j.M;
}

__global__ void __launch_bounds__(32 * kRefWarps) refine_batch_kernel(const uint8_t *plan, uint8_t *ws) {
  __shared__ RefShared sh[kRefWarps];
  const PlanHeader *h = reinterpret_cast<const PlanHeader *>(plan);
  const int warp = threadIdx.x >> 5;
  const int job = blockIdx.x * kRefWarps + warp;
  if (job >= h->njobs) return;
  const PlanJob &jb = reinterpret_cast<const PlanJob *>(plan + h->off_job)[job];
  const PlanProblem &pp = reinterpret_cast<const PlanProblem *>(plan + h->off_prob)[jb.prob];
  if (!pp.p.peak_angle || pp.p.d < 1) return;
  RefineJob j{};
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
  j.lo = pp.p.grid.lo_deg;
  j.step = pp.p.grid.step_deg;
  j.pos = pp.p.geom.pos;
  if (j.pos) {
    set_centroid(j);
    j.az_lo = pp.p.grid.lo_deg;
    j.az_step = pp.p.grid.step_deg;
    j.el_lo = pp.p.geom.el_lo_deg;
    j.el_step = pp.p.geom.el_step_deg;
    j.La = pp.p.grid.L;
    j.Le = pp.p.geom.Le;
    j.wrap = pp.p.geom.wrap_az;
  }
  j.P = pp.p.P + (size_t)jb.slot * pp.npts;
  const int d = pp.p.d;
  const int n = min(pp.p.peak_count[jb.slot], d);
  const int per = j.pos ? 2 : 1;
  refine_job_warp(j, pp.p.peak_idx + (size_t)jb.slot * d, n, pp.p.peak_angle + (size_t)jb.slot * d * per, sh[warp]);
}

__global__ void __launch_bounds__(32) refine_single_kernel(RefineJob j, const int *idx, const int *count, int cap,
                                                           double *out) {
  __shared__ RefShared sh;
  if (j.pos) set_centroid(j);
  const int n = min(*count, cap);
  refine_job_warp(j, idx, n, out, sh);
}

}  // namespace

cudaError_t launch_refine_batch(const uint8_t *plan_dev, const PlanHeader &h, uint8_t *ws, cudaStream_t s) {
  if (h.nrefine == 0 || h.njobs == 0) return cudaSuccess;
  refine_batch_kernel<<<(h.njobs + kRefWarps - 1) / kRefWarps, 32 * kRefWarps, 0, s>>>(plan_dev, ws);
  return cudaGetLastError();
}

cudaError_t launch_refine_single(const double2 *B, int M, int K, double lo, double step, const double *pos,
                                 double el_lo, double el_step, int La, const int *idx, const int *count, int cap,
                                 double *out, cudaStream_t s) {
  RefineJob j{};
  j.F = B;
  j.M = M;
  j.Kf = K;
  j.Kn = K;
  j.kphd = j.kmn = -1;
  j.alg = -1;
  j.lo = lo;
  j.step = step;
  j.pos = pos;
  j.az_lo = lo;
  j.az_step = step;
  j.el_lo = el_lo;
  j.el_step = el_step;
  j.La = La;
  refine_single_kernel<<<1, 32, 0, s>>>(j, idx, count, cap, out);
  return cudaGetLastError();
}

}  // namespace doa
