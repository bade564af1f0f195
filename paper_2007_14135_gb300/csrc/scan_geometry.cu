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
// Trigonometric tables. sin and cos of every azimuth theta_k and elevation angle phi_l of the
// grid are evaluated once per grid in FP64 (rounded multiply and add for the angle, then sincospi
// of angle / 180) and kept as FP64 and as FP32 (rounded once) in the workspace; a point reads
// its row's and column's entries, u = sin(theta) sin(phi), v = cos(theta) sin(phi), w = cos(phi).
//
// FP32 steering. The element phase t_m = p_m . (u, v, w) uses the positions relative to their
// centroid: that subtracts a common phase from every element, which leaves ||F^H a|| unchanged and
// keeps |t_m| at most the array's radius. Positions are held times 4, so the phase comes out in
// quarter turns and phasor_quarter splits it into a quadrant and a remainder without conversions
// (positions up to 2^20 wavelengths from the centroid).
//
// Refinement. The FP32 phasor error is bounded (in units of eps = 2^-24) by
//   eps_a = 2 pi rho (3 + 1 + 3) + 3,
// where rho = max_m (|x_m| + |y_m| + |z_m|) of the centred positions: the direction cosines carry
// 3 eps (two table roundings and the product), the positions one rounding and the phase three fma
// roundings (each eps rho), and phasor_q32 about 3 eps. With the factor's own rounding, eps_a + 3
// per term replaces the 4 eps per term of the ULA scan, so the refinement thresholds of
// scan_common.cuh scale by ((eps_a + 3) / 4)^2. Points below them are re-evaluated with the FP64
// tables, FP64 phases and the FP64 factor (warp per point).
//
// Shared steering tables (batch). Geometry problems that pass the same positions pointer with the
// same grid and M read their phasors from one FP32 table, written once per solve from the FP64
// phases of the refinement (each component rounded once, an error well inside eps_a), instead of
// evaluating them per problem: the phasors are about half of a point's instructions.
#include <float.h>

#include <algorithm>

#include "doa_internal.cuh"
#include "scan_common.cuh"

namespace doa {
namespace {

using namespace scanc;

struct GeoParams {
  const double *pos;     // M x 3 FP64 positions (wavelengths)
  const float2 *t32;     // (sin, cos): La azimuths, then Le elevation angles
  const double2 *t64;
  int La, Le;
};

struct GeoShared {
  float4 p32[kMaxM];     // 4 x centred positions in FP32 (x, y, z, 0); rows >= M zero
  double cen[3];         // centroid (FP64)
};

// (sin, cos) table entry e of a grid: e < La the azimuth theta_e, else the elevation angle
// phi_(e - La), each angle as lo + index * step in FP64 (rounded multiply, rounded add).
__device__ __forceinline__ void geo_table_entry(double az_lo, double az_step, int La, double el_lo, double el_step,
                                                int e, float2 *t32, double2 *t64) {
  const double ang = e < La ? __dadd_rn(az_lo, __dmul_rn((double)e, az_step))
                            : __dadd_rn(el_lo, __dmul_rn((double)(e - La), el_step));
  double sn, cs;
  sincospi(ang / 180.0, &sn, &cs);
  t64[e] = make_double2(sn, cs);
  t32[e] = make_float2((float)sn, (float)cs);
}

__global__ void geo_table_single_kernel(double az_lo, double az_step, int La, double el_lo, double el_step, int Le,
                                        float2 *t32, double2 *t64) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e < La + Le) geo_table_entry(az_lo, az_step, La, el_lo, el_step, e, t32, t64);
}

__global__ void geo_table_batch_kernel(const uint8_t *plan, uint8_t *ws) {
  const PlanHeader *h = reinterpret_cast<const PlanHeader *>(plan);
  const PlanGeoGrid g = reinterpret_cast<const PlanGeoGrid *>(plan + h->off_geo_grid)[blockIdx.y];
  float2 *t32 = reinterpret_cast<float2 *>(ws + g.t32_off);
  double2 *t64 = reinterpret_cast<double2 *>(ws + g.t64_off);
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < g.La + g.Le; e += gridDim.x * blockDim.x)
    geo_table_entry(g.az_lo, g.az_step, g.La, g.el_lo, g.el_step, e, t32, t64);
}

// FP64 steering source of the refinement and of the shared tables: flat point i -> (u, v, w), then
// the phase of element m.
struct GeoSource {
  const double *pos;
  const double2 *t64;
  double cx, cy, cz;
  int La;
  struct Dir {
    double u, v, w;
  };
  __device__ __forceinline__ Dir prep(int i) const {
    const int l = i / La, k = i - l * La;
    const double2 a = t64[k], e = t64[La + l];
    return Dir{a.x * e.x, a.y * e.x, e.y};
  }
  __device__ __forceinline__ double2 phasor(const Dir &d, int m) const {
    const double t = (pos[3 * m] - cx) * d.u + (pos[3 * m + 1] - cy) * d.v + (pos[3 * m + 2] - cz) * d.w;
    const double f = t - rint(t);                                    // [-1/2, 1/2] turn
    return phasor_q64((uint64_t)__double2ll_rn(f * 4611686018427387904.0) << 2);   // f * 2^64
  }
};

// Shared steering table t of the plan (blockIdx.y): tab[m * ldt + i] = a_m at flat point i, the
// FP64 phasor of the refinement rounded to FP32; rows m >= M and points i >= npts are zero.
__global__ void geo_steer_kernel(const uint8_t *plan, uint8_t *ws) {
  const PlanHeader *h = reinterpret_cast<const PlanHeader *>(plan);
  const PlanGeoSteer st = reinterpret_cast<const PlanGeoSteer *>(plan + h->off_geo_steer)[blockIdx.y];
  const PlanGeoGrid g = reinterpret_cast<const PlanGeoGrid *>(plan + h->off_geo_grid)[st.geo_grid];
  __shared__ double cen[3];
  if (threadIdx.x == 0) {
    double cx = 0.0, cy = 0.0, cz = 0.0;
    for (int m = 0; m < st.M; ++m) {
      cx += st.pos[3 * m];
      cy += st.pos[3 * m + 1];
      cz += st.pos[3 * m + 2];
    }
    cen[0] = cx / st.M;
    cen[1] = cy / st.M;
    cen[2] = cz / st.M;
  }
  __syncthreads();
  GeoSource src;
  src.pos = st.pos;
  src.t64 = reinterpret_cast<const double2 *>(ws + g.t64_off);
  src.cx = cen[0];
  src.cy = cen[1];
  src.cz = cen[2];
  src.La = g.La;
  float2 *tab = reinterpret_cast<float2 *>(ws + st.tab_off);
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < st.ldt; i += gridDim.x * blockDim.x) {
    const bool in = i < st.npts;
    GeoSource::Dir d{0.0, 0.0, 0.0};
    if (in) d = src.prep(i);
    for (int m = 0; m < st.MP; ++m) {
      float2 v = make_float2(0.f, 0.f);
      if (in && m < st.M) {
        const double2 a = src.phasor(d, m);
        v = make_float2((float)a.x, (float)a.y);
      }
      tab[(size_t)m * st.ldt + i] = v;
    }
  }
}

// Per-job constants: centroid, FP32 positions and the scaled thresholds. Every thread of the CTA
// calls it after load_job; it ends with a barrier.
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
  }
  __syncthreads();
  for (int m = threadIdx.x; m < MP; m += blockDim.x) {
    float4 p = make_float4(0.f, 0.f, 0.f, 0.f);
    if (m < j.M)
      p = make_float4((float)(4.0 * (g.pos[3 * m] - gs.cen[0])), (float)(4.0 * (g.pos[3 * m + 1] - gs.cen[1])),
                      (float)(4.0 * (g.pos[3 * m + 2] - gs.cen[2])), 0.f);
    gs.p32[m] = p;
  }
  set_threshold<MP>(Bs, j, sh);
  __syncthreads();
  if (threadIdx.x == 0) {
    double rho = 0.0;
    for (int m = 0; m < j.M; ++m)
      rho = fmax(rho, fabs(g.pos[3 * m] - gs.cen[0]) + fabs(g.pos[3 * m + 1] - gs.cen[1]) +
                          fabs(g.pos[3 * m + 2] - gs.cen[2]));
    const double ea = 2.0 * 3.141592653589793 * rho * 7.0 + 3.0;
    double sc = (ea + 3.0) / 4.0;
    sc = fmax(sc * sc, 1.0);
    for (int r = 0; r < 4; ++r) sh.thr[r] = (float)(sh.thr[r] * sc);
  }
  __syncthreads();
}

// tab (nullable): the problem's shared steering table (row stride ldt, a multiple of every tile's
// point count, so the PT points of a thread lie inside each row and start on a 2 * PT float
// boundary); without it the phasors are evaluated here.
template <int MP, int PT>
__device__ __forceinline__ void geo_points(const float2 *Bs, const ScanJob &j, const GeoShared &gs,
                                           const float2 *__restrict__ t32, int La, int Le, int npts, int i0,
                                           ScanShared &sh, const GeoSource &src,
                                           const float2 *__restrict__ tab = nullptr, int ldt = 0) {
  static_assert(MP % 4 == 0, "MP is a multiple of 4");
  float2 a[PT][MP];
  if (tab) {
#pragma unroll
    for (int m = 0; m < MP; ++m) {
      const float2 *row = tab + (size_t)m * ldt + i0;
      if constexpr (PT % 2 == 0) {
#pragma unroll
        for (int q2 = 0; q2 < PT / 2; ++q2) {
          const float4 v = __ldg(reinterpret_cast<const float4 *>(row) + q2);
          a[2 * q2][m] = make_float2(v.x, v.y);
          a[2 * q2 + 1][m] = make_float2(v.z, v.w);
        }
      } else {
#pragma unroll
        for (int q = 0; q < PT; ++q) a[q][m] = __ldg(row + q);
      }
    }
    contract_points<MP, PT>(Bs, j, a, npts, i0, sh, src);
    return;
  }
  int l = i0 / La, k = i0 - l * La;
#pragma unroll
  for (int q = 0; q < PT; ++q) {
    // points past the end (l >= Le) read a valid entry and are never stored
    const float2 ta = __ldg(t32 + k), te = __ldg(t32 + La + min(l, Le - 1));
    const float u = ta.x * te.x, v = ta.y * te.x, w = te.y;
#pragma unroll
    for (int m = 0; m < MP; ++m) {
      const float4 p = gs.p32[m];
      a[q][m] = phasor_quarter(fmaf(p.x, u, fmaf(p.y, v, p.z * w)));   // phase in quarter turns
    }
    if (++k == La) {
      k = 0;
      ++l;
    }
  }
  contract_points<MP, PT>(Bs, j, a, npts, i0, sh, src);
}

// Re-evaluates the queued points of the current job in FP64 (warp per point).
__device__ __forceinline__ void geo_drain(const ScanJob &j, const GeoSource &src, ScanShared &sh) {
  drain_refinements_src(j, src, sh);
}

__device__ __forceinline__ GeoSource make_source(const GeoParams &g, const GeoShared &gs) {
  GeoSource s;
  s.pos = g.pos;
  s.t64 = g.t64;
  s.cx = gs.cen[0];
  s.cy = gs.cen[1];
  s.cz = gs.cen[2];
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
  geo_points<MP, PT>(Bs, j, gs, g.t32, g.La, g.Le, npts, i0, sh, src);
  geo_drain(j, src, sh);
}

// Batched: the tiles of the geometry problems of one M bucket, dealt in runs of kRun tiles like the
// ULA batch scan (run r to CTA r mod gridDim). Flagged points accumulate over a run and are
// re-evaluated when the run ends or its problem changes, so the warps share the FP64 work of
// many tiles and meet at a barrier once per run rather than once per tile.
constexpr int kRun = 16;   // longest run (large batches); small ones use shorter runs so every SM gets one

template <int MP, int PT>
__global__ void __launch_bounds__(kScanThreads) scan_geometry_batch_kernel(const uint8_t *plan, uint8_t *ws,
                                                                           int bucket, int run_len) {
  __shared__ __align__(16) float2 Bs[(MP + 1) * MP];
  __shared__ ScanShared sh;
  __shared__ GeoShared gs;
  const PlanHeader *h = reinterpret_cast<const PlanHeader *>(plan);
  const int nunits = h->geo_jobs[bucket];
  const int64_t ntiles = h->geo_tiles[bucket];
  const int32_t *list = reinterpret_cast<const int32_t *>(plan + h->off_geo[bucket]);
  const PlanProblem *probs = reinterpret_cast<const PlanProblem *>(plan + h->off_prob);
  const PlanGeoGrid *geo_grids = reinterpret_cast<const PlanGeoGrid *>(plan + h->off_geo_grid);
  const PlanGeoSteer *steers = reinterpret_cast<const PlanGeoSteer *>(plan + h->off_geo_steer);
  constexpr int TP = kScanThreads * PT;
  static_assert(kSteerAlign % TP == 0, "a tile's points lie inside one steering-table row");
  int cur = -1;
  ScanJob j{};
  GeoParams g{};
  GeoSource src{};
  const PlanProblem *pp = nullptr;
  const float2 *tab = nullptr;
  int ldt = 0;
  // (runs dealt round-robin: taking them from a counter, as the ULA scans do, measured slower here)
  for (int64_t run = blockIdx.x; run * run_len < ntiles; run += gridDim.x) {
    const int64_t t_begin = run * run_len, t_end = min(ntiles, t_begin + run_len);
    int u = 0, hi = nunits - 1;
    while (u < hi) {  // last problem with tile_start <= t_begin
      int mid = (u + hi + 1) >> 1;
      if (probs[list[mid]].tile_start <= t_begin) u = mid; else hi = mid - 1;
    }
    for (int64_t t = t_begin; t < t_end; ++t) {
      while (u + 1 < nunits && probs[list[u + 1]].tile_start <= t) ++u;
      if (u != cur) {
        if (cur >= 0) geo_drain(j, src, sh);
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
        const PlanGeoGrid &gg = geo_grids[pp->geo_grid];
        g.pos = pp->p.geom.pos;
        g.t32 = reinterpret_cast<const float2 *>(ws + gg.t32_off);
        g.t64 = reinterpret_cast<const double2 *>(ws + gg.t64_off);
        g.La = gg.La;
        g.Le = gg.Le;
        tab = nullptr;
        ldt = 0;
        if (pp->geo_steer >= 0) {
          const PlanGeoSteer &st = steers[pp->geo_steer];
          tab = reinterpret_cast<const float2 *>(ws + st.tab_off);
          ldt = st.ldt;
        }
        __syncthreads();
        load_job<MP>(j, Bs, sh);
        __syncthreads();
        geo_setup<MP>(Bs, j, g, gs, sh);
        src = make_source(g, gs);
        cur = u;
      }
      const int i0 = (int)(t - pp->tile_start) * TP + threadIdx.x * PT;
      geo_points<MP, PT>(Bs, j, gs, g.t32, g.La, g.Le, pp->npts, i0, sh, src, tab, ldt);
    }
    geo_drain(j, src, sh);
  }
}


template <int MP, int PT>
cudaError_t run_geo_batch(const uint8_t *plan, const PlanHeader &h, uint8_t *ws, int bucket, cudaStream_t s) {
  const int64_t tiles = h.geo_tiles[bucket];
  if (tiles == 0) return cudaSuccess;
  int per_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, scan_geometry_batch_kernel<MP, PT>, kScanThreads, 0);
  if (per_sm < 1) per_sm = 1;
  const int64_t cap = (int64_t)device_sm_count() * per_sm;
  const int run_len = (int)std::min<int64_t>(kRun, std::max<int64_t>(1, (tiles + cap - 1) / cap));
  const int64_t grid = std::min<int64_t>(cap, (tiles + run_len - 1) / run_len);
  scan_geometry_batch_kernel<MP, PT><<<(unsigned)grid, kScanThreads, 0, s>>>(plan, ws, bucket, run_len);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_scan_geometry_single(const double2 *B, int M, int K, const double *pos, double az_lo,
                                        double az_step, int La, double el_lo, double el_step, int Le, float *P,
                                        uint8_t *ws, cudaStream_t s) {
  double2 *t64 = reinterpret_cast<double2 *>(ws);
  float2 *t32 = reinterpret_cast<float2 *>(ws + 16 * ((int64_t)La + Le));
  geo_table_single_kernel<<<(La + Le + 255) / 256, 256, 0, s>>>(az_lo, az_step, La, el_lo, el_step, Le, t32, t64);
  GeoParams g{pos, t32, t64, La, Le};
  const int b = m_bucket(M);
  const int pt = scan_pt_default(b);
  const int64_t npts = (int64_t)La * Le;
  const unsigned grid = (unsigned)((npts + kScanThreads * pt - 1) / (kScanThreads * pt));
  switch (b) {
    case 0: scan_geometry_single_kernel<8, 4><<<grid, kScanThreads, 0, s>>>(B, M, K, g, P); break;
    case 1: scan_geometry_single_kernel<16, 4><<<grid, kScanThreads, 0, s>>>(B, M, K, g, P); break;
    case 2: scan_geometry_single_kernel<32, 1><<<grid, kScanThreads, 0, s>>>(B, M, K, g, P); break;
    default: scan_geometry_single_kernel<64, 1><<<grid, kScanThreads, 0, s>>>(B, M, K, g, P); break;
  }
  return cudaGetLastError();
}

cudaError_t launch_geo_tables(const uint8_t *plan_dev, const PlanHeader &h, uint8_t *ws, cudaStream_t s) {
  if (h.ngeo_grids == 0) return cudaSuccess;
  const int bx = (h.geo_grid_points + 255) / 256;
  geo_table_batch_kernel<<<dim3(bx, h.ngeo_grids), 256, 0, s>>>(plan_dev, ws);
  if (h.ngeo_steer > 0) {   // the shared steering tables read the FP64 sin / cos tables just written
    const int sx = std::min(2 * device_sm_count(), (h.steer_max_ldt + 255) / 256);
    geo_steer_kernel<<<dim3(sx, h.ngeo_steer), 256, 0, s>>>(plan_dev, ws);
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
