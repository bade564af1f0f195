// Step-5 (Table 2) for an arbitrary array geometry on an azimuth x elevation grid, with the
// steering vector of Eq. 2 as printed:
//   a_m(theta, phi) = exp{ j 2 pi (x_m u + y_m v + z_m w) },
//   u = sin(theta) sin(phi), v = cos(theta) sin(phi), w = cos(phi),
// positions in wavelengths, theta the azimuth (columns) and phi the elevation angle (rows).
//
// The spectrum is Le x La row-major; a thread evaluates PT consecutive flat points (so a tile can
// span rows) and the contraction and readouts are those of the ULA scan (scan_common.cuh): one
// factor F = [E_n | valph] per problem feeds MUSIC, EV, PHD and MN.
//
// FP32 steering. The direction angles are formed in half turns, h = h0 + k hs with h0 reduced to
// [-1, 1) and h0, hs split into FP32 hi + lo parts (two roundings, relative 2 eps, whatever the
// step), and sincospif reduces them exactly. The element phase t_m = p_m . (u, v, w) (turns) uses the positions relative to their
// centroid: that subtracts a common phase from every element, which leaves ||F^H a|| unchanged and
// keeps |t_m| at most the array's radius. The fraction t_m - rint(t_m) becomes a 32-bit phase and
// phasor_q32 turns it into cos + j sin.
//
// Refinement. The FP32 phasor error is bounded (in units of eps = 2^-24) by
//   eps_a = 2 pi rho (2 pi (x_az + x_el) + 9) + 3,
// where rho = max_m (|x_m| + |y_m| + |z_m|) of the centred positions and x_az, x_el bound the
// half-turn arguments over the grid: each argument is rounded twice (2 eps x), sincospif adds an
// ulp (2 eps), the direction cosines one product, the positions one rounding and the phase three
// fma roundings (each eps rho), and phasor_q32 about 3 eps. With
// the factor's own rounding, eps_a + 3 per term replaces the 4 eps per term of the ULA scan, so the
// refinement thresholds of scan_common.cuh scale by ((eps_a + 3) / 4)^2. Points below them are
// re-evaluated with FP64 angles (sincospi), FP64 phases and the FP64 factor (warp per point).
#include <float.h>

#include "doa_internal.cuh"
#include "scan_common.cuh"

namespace doa {
namespace {

using namespace scanc;

struct GeoParams {
  const double *pos;     // M x 3 FP64 positions (wavelengths)
  double az_lo, az_step, el_lo, el_step;
  int La, Le;
};

struct GeoShared {
  float4 p32[kMaxM];     // centred positions in FP32 (x, y, z, 0); rows >= M zero
  double cen[3];         // centroid (FP64)
  float a0h, a0l, ash, asl;  // azimuth origin and step in half turns, hi + lo
  float e0h, e0l, esh, esl;  // elevation origin and step in half turns, hi + lo
};

// FP64 steering source of the refinement: flat point i -> (u, v, w), then the phase of element m.
struct GeoSource {
  const double *pos;
  double cx, cy, cz;
  double az_lo, az_step, el_lo, el_step;
  int La;
  struct Dir {
    double u, v, w;
  };
  __device__ __forceinline__ Dir prep(int i) const {
    const int l = i / La, k = i - l * La;
    const double th = __dadd_rn(az_lo, __dmul_rn((double)k, az_step));
    const double ph = __dadd_rn(el_lo, __dmul_rn((double)l, el_step));
    double st, ct, sp, cp;
    sincospi(th / 180.0, &st, &ct);
    sincospi(ph / 180.0, &sp, &cp);
    return Dir{st * sp, ct * sp, cp};
  }
  __device__ __forceinline__ double2 phasor(const Dir &d, int m) const {
    const double t = (pos[3 * m] - cx) * d.u + (pos[3 * m + 1] - cy) * d.v + (pos[3 * m + 2] - cz) * d.w;
    const double f = t - rint(t);                                    // [-1/2, 1/2] turn
    return phasor_q64((uint64_t)__double2ll_rn(f * 4611686018427387904.0) << 2);   // f * 2^64
  }
};

__device__ __forceinline__ void split_f(double x, float &hi, float &lo) {
  hi = (float)x;
  lo = (float)(x - (double)hi);
}

// Per-job constants: centroid, FP32 positions, angle splits, and the scaled thresholds. Every
// thread of the CTA calls it after load_job; it ends with a barrier.
template <int MP>
__device__ void geo_setup(const float2 *Bs, const ScanJob &j, const GeoParams &g, GeoShared &gs, ScanShared &sh) {
  if (threadIdx.x == 0) {
    double cx = 0.0, cy = 0.0, cz = 0.0;
    for (int m = 0; m < j.M; ++m) {
      cx += g.pos[3 * m];
      cy += g.pos[3 * m + 1];
      cz += g.pos[3 * m + 2];
    }
    gs.cen[0] = cx / j.M;
    gs.cen[1] = cy / j.M;
    gs.cen[2] = cz / j.M;
    double a0 = g.az_lo / 180.0, e0 = g.el_lo / 180.0;
    a0 -= 2.0 * rint(0.5 * a0);
    e0 -= 2.0 * rint(0.5 * e0);
    const double as = g.az_step / 180.0, es = g.el_step / 180.0;
    split_f(a0, gs.a0h, gs.a0l);
    split_f(as, gs.ash, gs.asl);
    split_f(e0, gs.e0h, gs.e0l);
    split_f(es, gs.esh, gs.esl);
  }
  __syncthreads();
  for (int m = threadIdx.x; m < MP; m += blockDim.x) {
    float4 p = make_float4(0.f, 0.f, 0.f, 0.f);
    if (m < j.M)
      p = make_float4((float)(g.pos[3 * m] - gs.cen[0]), (float)(g.pos[3 * m + 1] - gs.cen[1]),
                      (float)(g.pos[3 * m + 2] - gs.cen[2]), 0.f);
    gs.p32[m] = p;
  }
  set_threshold<MP>(Bs, j, sh);
  __syncthreads();
  if (threadIdx.x == 0) {
    double rho = 0.0;
    for (int m = 0; m < j.M; ++m)
      rho = fmax(rho, fabs(g.pos[3 * m] - gs.cen[0]) + fabs(g.pos[3 * m + 1] - gs.cen[1]) +
                          fabs(g.pos[3 * m + 2] - gs.cen[2]));
    const double xa = fabs(g.az_lo / 180.0 - 2.0 * rint(g.az_lo / 360.0)) + (g.La - 1) * fabs(g.az_step / 180.0);
    const double xe = fabs(g.el_lo / 180.0 - 2.0 * rint(g.el_lo / 360.0)) + (g.Le - 1) * fabs(g.el_step / 180.0);
    const double kPi = 3.141592653589793;
    const double ea = 2.0 * kPi * rho * (2.0 * kPi * (xa + xe) + 9.0) + 3.0;
    double sc = (ea + 3.0) / 4.0;
    sc = fmax(sc * sc, 1.0);
    for (int r = 0; r < 4; ++r) sh.thr[r] = (float)(sh.thr[r] * sc);
  }
  __syncthreads();
}

template <int MP, int PT>
__device__ __forceinline__ void geo_points(const float2 *Bs, const ScanJob &j, const GeoShared &gs, int La, int npts,
                                           int i0, ScanShared &sh, const GeoSource &src) {
  static_assert(MP % 4 == 0, "MP is a multiple of 4");
  float2 a[PT][MP];
  int l = i0 / La, k = i0 - l * La;
#pragma unroll
  for (int q = 0; q < PT; ++q) {
    const float kf = (float)k, lf = (float)l;
    const float ha = fmaf(kf, gs.ash, gs.a0h) + fmaf(kf, gs.asl, gs.a0l);
    const float he = fmaf(lf, gs.esh, gs.e0h) + fmaf(lf, gs.esl, gs.e0l);
    float sa, ca, se, ce;
    sincospif(ha, &sa, &ca);
    sincospif(he, &se, &ce);
    const float u = sa * se, v = ca * se, w = ce;
#pragma unroll
    for (int m = 0; m < MP; ++m) {
      const float4 p = gs.p32[m];
      const float t = fmaf(p.x, u, fmaf(p.y, v, p.z * w));
      const float f = t - rintf(t);                                   // [-1/2, 1/2] turn
      a[q][m] = phasor_q32((uint32_t)__float2int_rn(f * 4294967296.0f));
    }
    if (++k == La) {
      k = 0;
      ++l;
    }
  }
  contract_points<MP, PT>(Bs, j, a, npts, i0, sh, src);
}

__device__ __forceinline__ GeoSource make_source(const GeoParams &g, const GeoShared &gs) {
  GeoSource s;
  s.pos = g.pos;
  s.cx = gs.cen[0];
  s.cy = gs.cen[1];
  s.cz = gs.cen[2];
  s.az_lo = g.az_lo;
  s.az_step = g.az_step;
  s.el_lo = g.el_lo;
  s.el_step = g.el_step;
  s.La = g.La;
  return s;
}

template <int MP, int PT>
__global__ void __launch_bounds__(kScanThreads) scan_geometry_single_kernel(const double2 *B, int M, int K,
                                                                            GeoParams g, float *P) {
  __shared__ __align__(16) float2 Bs[MP * MP];
  __shared__ ScanShared sh;
  __shared__ GeoShared gs;
  ScanJob j{};
  j.F = B;
  j.P[kRoMusic] = P;
  j.M = M;
  j.Kf = K;
  j.Kn = K;
  j.kphd = j.kmn = -1;
  load_job<MP>(j, Bs, sh);
  __syncthreads();
  geo_setup<MP>(Bs, j, g, gs, sh);
  const int npts = g.La * g.Le;
  const GeoSource src = make_source(g, gs);
  const int i0 = (blockIdx.x * kScanThreads + threadIdx.x) * PT;
  geo_points<MP, PT>(Bs, j, gs, g.La, npts, i0, sh, src);
  drain_refinements_src(j, src, sh);
}

// Batched: the tiles of the geometry problems of one M bucket, dealt in runs of kRun tiles like the
// ULA batch scan (run r to CTA r mod gridDim).
constexpr int kRun = 16;

template <int MP, int PT>
__global__ void __launch_bounds__(kScanThreads) scan_geometry_batch_kernel(const uint8_t *plan, uint8_t *ws,
                                                                           int bucket) {
  __shared__ __align__(16) float2 Bs[(MP + 1) * MP];
  __shared__ ScanShared sh;
  __shared__ GeoShared gs;
  const PlanHeader *h = reinterpret_cast<const PlanHeader *>(plan);
  const int nunits = h->geo_jobs[bucket];
  const int64_t ntiles = h->geo_tiles[bucket];
  const int32_t *list = reinterpret_cast<const int32_t *>(plan + h->off_geo[bucket]);
  const PlanProblem *probs = reinterpret_cast<const PlanProblem *>(plan + h->off_prob);
  constexpr int TP = kScanThreads * PT;
  int cur = -1;
  ScanJob j{};
  GeoParams g{};
  GeoSource src{};
  const PlanProblem *pp = nullptr;
  for (int64_t run = blockIdx.x; run * kRun < ntiles; run += gridDim.x) {
    const int64_t t_begin = run * kRun, t_end = min(ntiles, t_begin + kRun);
    int u = 0, hi = nunits - 1;
    while (u < hi) {  // last problem with tile_start <= t_begin
      int mid = (u + hi + 1) >> 1;
      if (probs[list[mid]].tile_start <= t_begin) u = mid; else hi = mid - 1;
    }
    for (int64_t t = t_begin; t < t_end; ++t) {
      while (u + 1 < nunits && probs[list[u + 1]].tile_start <= t) ++u;
      if (u != cur) {
        pp = &probs[list[u]];
        const int npts = pp->npts;
        j.F = reinterpret_cast<const double2 *>(ws + pp->fac_off);
        j.w = pp->Kn > 0 && pp->slot[DOA_EV] >= 0
                  ? reinterpret_cast<const double *>(ws + pp->fac_off) + 2 * pp->p.M * (pp->p.M + 1)
                  : nullptr;
        j.S64 = nullptr;
        for (int r = 0; r < 4; ++r) j.P[r] = pp->slot[r] >= 0 ? pp->p.P + (size_t)pp->slot[r] * npts : nullptr;
        j.M = pp->p.M;
        j.Kf = pp->Kf;
        j.Kn = pp->Kn;
        j.kphd = pp->kphd;
        j.kmn = pp->kmn;
        j.kofs = 0;
        g.pos = pp->p.geom.pos;
        g.az_lo = pp->p.grid.lo_deg;
        g.az_step = pp->p.grid.step_deg;
        g.el_lo = pp->p.geom.el_lo_deg;
        g.el_step = pp->p.geom.el_step_deg;
        g.La = pp->p.grid.L;
        g.Le = pp->p.geom.Le;
        __syncthreads();
        load_job<MP>(j, Bs, sh);
        __syncthreads();
        geo_setup<MP>(Bs, j, g, gs, sh);
        src = make_source(g, gs);
        cur = u;
      }
      const int i0 = (int)(t - pp->tile_start) * TP + threadIdx.x * PT;
      geo_points<MP, PT>(Bs, j, gs, g.La, pp->npts, i0, sh, src);
      drain_refinements_src(j, src, sh);
    }
  }
}

int g_num_sms = 0;

int num_sms() {
  if (g_num_sms == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&g_num_sms, cudaDevAttrMultiProcessorCount, dev);
    if (g_num_sms <= 0) g_num_sms = 1;
  }
  return g_num_sms;
}

template <int MP, int PT>
cudaError_t run_geo_batch(const uint8_t *plan, const PlanHeader &h, uint8_t *ws, int bucket, cudaStream_t s) {
  const int64_t tiles = h.geo_tiles[bucket];
  if (tiles == 0) return cudaSuccess;
  int per_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, scan_geometry_batch_kernel<MP, PT>, kScanThreads, 0);
  if (per_sm < 1) per_sm = 1;
  int64_t grid = (int64_t)num_sms() * per_sm;
  const int64_t runs = (tiles + kRun - 1) / kRun;
  if (grid > runs) grid = runs;
  scan_geometry_batch_kernel<MP, PT><<<(unsigned)grid, kScanThreads, 0, s>>>(plan, ws, bucket);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_scan_geometry_single(const double2 *B, int M, int K, const double *pos, double az_lo,
                                        double az_step, int La, double el_lo, double el_step, int Le, float *P,
                                        cudaStream_t s) {
  GeoParams g{pos, az_lo, az_step, el_lo, el_step, La, Le};
  const int b = m_bucket(M);
  const int pt = scan_pt_default(b);
  const int64_t npts = (int64_t)La * Le;
  const unsigned grid = (unsigned)((npts + kScanThreads * pt - 1) / (kScanThreads * pt));
  switch (b) {
    case 0: scan_geometry_single_kernel<8, 4><<<grid, kScanThreads, 0, s>>>(B, M, K, g, P); break;
    case 1: scan_geometry_single_kernel<16, 2><<<grid, kScanThreads, 0, s>>>(B, M, K, g, P); break;
    case 2: scan_geometry_single_kernel<32, 1><<<grid, kScanThreads, 0, s>>>(B, M, K, g, P); break;
    default: scan_geometry_single_kernel<64, 1><<<grid, kScanThreads, 0, s>>>(B, M, K, g, P); break;
  }
  return cudaGetLastError();
}

cudaError_t launch_scan_geometry_batch(const uint8_t *plan_dev, const PlanHeader &h, uint8_t *ws, cudaStream_t s) {
  cudaError_t e;
  switch (h.scan_pt[0]) {
    case 1: e = run_geo_batch<8, 1>(plan_dev, h, ws, 0, s); break;
    case 2: e = run_geo_batch<8, 2>(plan_dev, h, ws, 0, s); break;
    default: e = run_geo_batch<8, 4>(plan_dev, h, ws, 0, s); break;
  }
  if (e != cudaSuccess) return e;
  switch (h.scan_pt[1]) {
    case 1: e = run_geo_batch<16, 1>(plan_dev, h, ws, 1, s); break;
    case 4: e = run_geo_batch<16, 4>(plan_dev, h, ws, 1, s); break;
    default: e = run_geo_batch<16, 2>(plan_dev, h, ws, 1, s); break;
  }
  if (e != cudaSuccess) return e;
  if (h.scan_pt[2] == 2)
    e = run_geo_batch<32, 2>(plan_dev, h, ws, 2, s);
  else
    e = run_geo_batch<32, 1>(plan_dev, h, ws, 2, s);
  if (e != cudaSuccess) return e;
  return run_geo_batch<64, 1>(plan_dev, h, ws, 3, s);
}

}  // namespace doa
