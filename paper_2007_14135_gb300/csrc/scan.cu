// Step-5 (Table 2; steering vector Eq. 2): pseudospectrum P_k = 1 / ||B^H a(theta_k)||^2, which
// equals 1 / (a^H C a) for the weighting matrix C = B B^H of Table 3 and is never negative.
//
// Fused, on CUDA cores in FP32: every thread evaluates PT consecutive grid points. For each it
// generates the M steering phasors in registers from the grid's 32-bit phase step S_k
// (phase of element m = m*S_k mod 2^32, exact integer arithmetic; phasor_q32 turns a phase into
// cos + j sin), contracts them with the noise factor B (held in shared memory as FP32, read as
// warp-wide broadcasts) one column at a time, accumulates |y_k|^2, and stores 1/den with
// vectorised stores. The whole block of PT x M phasors is reused across the K columns of B.
//
// Near-null refinement: where the FP32 denominator is small its relative error grows (the
// contraction cancels), so every point with den < kRefineC * E, E = sum_k (sum_m |b_mk|)^2, is
// re-evaluated in FP64 from the grid angle (theta_k, sin theta_k and the phasors in FP64) and the
// FP64 factor. Flagged points of a tile are queued in shared memory and each is then handled by a
// whole warp (lanes own phasors, then columns of B), so the FP64 work runs without divergence.
// With per-term FP32 errors below ~4 eps the FP32 result elsewhere stays within ~5e-4 relative.
#include <float.h>

#include "doa_internal.cuh"

namespace doa {
namespace {

__global__ void grid_table_single_kernel(double lo, double step, int L, uint32_t *S) {
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k < L) S[k] = grid_phase_step(lo, step, k);
}

__global__ void grid_table_batch_kernel(const uint8_t *plan, uint8_t *ws) {
  const PlanHeader *h = reinterpret_cast<const PlanHeader *>(plan);
  const PlanGrid g = reinterpret_cast<const PlanGrid *>(plan + h->off_grid)[blockIdx.y];
  uint32_t *S = reinterpret_cast<uint32_t *>(ws + g.S_off);
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < g.L; k += gridDim.x * blockDim.x)
    S[k] = grid_phase_step(g.lo, g.step, k);
}

// B (M x K complex128, column-major, ld M) -> Bs[k][m] (FP32, rows m >= M zero-padded to MP).
template <int MP>
__device__ __forceinline__ void load_factor(const double2 *__restrict__ B, int M, int K, float2 *Bs) {
  for (int e = threadIdx.x; e < K * MP; e += blockDim.x) {
    int k = e / MP, m = e % MP;
    float2 v = make_float2(0.f, 0.f);
    if (m < M) {
      double2 b = B[(size_t)k * M + m];
      v = make_float2((float)b.x, (float)b.y);
    }
    Bs[e] = v;
  }
}

constexpr float kRefineC = 3.7e-6f;   // (4 * 4 eps32 / 5e-4)^2
constexpr int kFlagCap = 256;          // queued refinements per tile (overflow: refined in place)
constexpr int kScanWarps = kScanThreads / 32;

struct RefineCtx {
  const double2 *B;   // FP64 factor, column-major, ld M
  int M, K;
  double lo, step;
};

struct ScanShared {
  double2 ph[kScanWarps][kMaxM];   // per-warp FP64 phasors for refinement
  int flags[kFlagCap];
  int nflag;
  float thr;
};

// E = sum_k (sum_m |b_mk|)^2 over the FP32 factor in shared memory; thr = kRefineC * E.
template <int MP>
__device__ __forceinline__ void set_threshold(const float2 *Bs, int K, ScanShared &sh) {
  if (threadIdx.x < 32) {
    float e = 0.f;
    for (int k = threadIdx.x; k < K; k += 32) {
      float n1 = 0.f;
      for (int m = 0; m < MP; ++m) {
        float2 b = Bs[k * MP + m];
        n1 += sqrtf(b.x * b.x + b.y * b.y);
      }
      e += n1 * n1;
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) e += __shfl_xor_sync(0xffffffffu, e, off);
    if (threadIdx.x == 0) {
      sh.thr = kRefineC * e;
      sh.nflag = 0;
    }
  }
}

// FP64 re-evaluation of grid point k by one whole warp: lanes compute phasors m = lane, lane+32,
// then each lane contracts whole columns k = lane, lane+32 of B; den is a warp sum.
__device__ void refine_point_warp(const RefineCtx &c, int k, float *P, double2 *ph) {
  const int lane = threadIdx.x & 31;
  const double theta = __dadd_rn(c.lo, __dmul_rn((double)k, c.step));
  const double s = sin(theta * 0.017453292519943295);
  for (int m = lane; m < c.M; m += 32) {
    double sn, cs;
    sincospi((double)m * s, &sn, &cs);
    ph[m] = make_double2(cs, sn);
  }
  __syncwarp();
  double den = 0.0;
  for (int col = lane; col < c.K; col += 32) {
    double yr = 0.0, yi = 0.0;
    const double2 *b = c.B + (size_t)col * c.M;
    for (int m = 0; m < c.M; ++m) {
      double2 bb = b[m], a = ph[m];
      yr = fma(bb.x, a.x, fma(bb.y, a.y, yr));
      yi = fma(bb.x, a.y, fma(-bb.y, a.x, yi));
    }
    den = fma(yr, yr, fma(yi, yi, den));
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) den += __shfl_xor_sync(0xffffffffu, den, off);
  if (lane == 0) P[k] = (float)(1.0 / fmax(den, (double)FLT_MIN));
  __syncwarp();
}

// Same computation by a single thread (only when a tile's queue overflows).
__device__ void refine_point_thread(const RefineCtx &c, int k, float *P) {
  const double theta = __dadd_rn(c.lo, __dmul_rn((double)k, c.step));
  const double s = sin(theta * 0.017453292519943295);
  double den = 0.0;
  for (int col = 0; col < c.K; ++col) {
    double yr = 0.0, yi = 0.0;
    for (int m = 0; m < c.M; ++m) {
      double sn, cs;
      sincospi((double)m * s, &sn, &cs);
      double2 bb = c.B[(size_t)col * c.M + m];
      yr = fma(bb.x, cs, fma(bb.y, sn, yr));
      yi = fma(bb.x, sn, fma(-bb.y, cs, yi));
    }
    den = fma(yr, yr, fma(yi, yi, den));
  }
  P[k] = (float)(1.0 / fmax(den, (double)FLT_MIN));
}

// Drains the tile's refinement queue (all threads of the CTA call this).
__device__ __forceinline__ void drain_refinements(const RefineCtx &c, float *P, ScanShared &sh) {
  __syncthreads();
  const int n = min(sh.nflag, kFlagCap);
  const int warp = threadIdx.x >> 5;
  for (int i = warp; i < n; i += kScanWarps) refine_point_warp(c, sh.flags[i], P, sh.ph[warp]);
  __syncthreads();
  if (threadIdx.x == 0) sh.nflag = 0;
  __syncthreads();
}

// Evaluates the PT points k0 .. k0+PT-1 (those < L) of one spectrum. S may alias P: each
// thread reads its own phase steps before it writes its own outputs. Points below the
// refinement threshold are queued for drain_refinements.
template <int MP, int PT>
__device__ __forceinline__ void scan_points(const float2 *Bs, int K, const uint32_t *S, float *P, int L, int k0,
                                            const RefineCtx &rc, ScanShared &sh) {
  float2 a[PT][MP];
#pragma unroll
  for (int j = 0; j < PT; ++j) {
    uint32_t step = (k0 + j < L) ? S[k0 + j] : 0u;
    uint32_t phi = 0u;
#pragma unroll
    for (int m = 0; m < MP; ++m) {
      a[j][m] = phasor_q32(phi);
      phi += step;
    }
  }
  float den[PT];
#pragma unroll
  for (int j = 0; j < PT; ++j) den[j] = 0.f;
  for (int k = 0; k < K; ++k) {
    float yr[PT], yi[PT];
#pragma unroll
    for (int j = 0; j < PT; ++j) yr[j] = yi[j] = 0.f;
#pragma unroll
    for (int m = 0; m < MP; ++m) {
      const float2 b = Bs[k * MP + m];
#pragma unroll
      for (int j = 0; j < PT; ++j) {
        // conj(b) * a = (br ar + bi ai) + j (br ai - bi ar)
        yr[j] = fmaf(b.x, a[j][m].x, fmaf(b.y, a[j][m].y, yr[j]));
        yi[j] = fmaf(b.x, a[j][m].y, fmaf(-b.y, a[j][m].x, yi[j]));
      }
    }
#pragma unroll
    for (int j = 0; j < PT; ++j) den[j] = fmaf(yr[j], yr[j], fmaf(yi[j], yi[j], den[j]));
  }
  float out[PT];
  int pos[PT];
  const float thr = sh.thr;
#pragma unroll
  for (int j = 0; j < PT; ++j) {
    out[j] = 1.0f / fmaxf(den[j], FLT_MIN);
    pos[j] = -1;
    if (k0 + j < L && den[j] < thr) {
      pos[j] = atomicAdd(&sh.nflag, 1);
      if (pos[j] < kFlagCap) sh.flags[pos[j]] = k0 + j;
    }
  }
  // vectorised store when the whole group is in range and aligned
  if (PT == 4 && k0 + 3 < L && ((reinterpret_cast<uintptr_t>(P + k0) & 15u) == 0)) {
    *reinterpret_cast<float4 *>(P + k0) = make_float4(out[0], out[1], out[2 % PT], out[3 % PT]);
  } else if (PT == 2 && k0 + 1 < L && ((reinterpret_cast<uintptr_t>(P + k0) & 7u) == 0)) {
    *reinterpret_cast<float2 *>(P + k0) = make_float2(out[0], out[1 % PT]);
  } else {
#pragma unroll
    for (int j = 0; j < PT; ++j)
      if (k0 + j < L) P[k0 + j] = out[j];
  }
  // queue overflow (more than kFlagCap small denominators in one tile): refine in place
#pragma unroll
  for (int j = 0; j < PT; ++j)
    if (pos[j] >= kFlagCap) refine_point_thread(rc, k0 + j, P);
}

template <int MP, int PT>
__global__ void __launch_bounds__(kScanThreads) scan_single_kernel(const double2 *B, int M, int K, int L, double lo,
                                                                   double step, const uint32_t *S, float *P) {
  __shared__ __align__(16) float2 Bs[MP * MP];
  __shared__ ScanShared sh;
  load_factor<MP>(B, M, K, Bs);
  __syncthreads();
  set_threshold<MP>(Bs, K, sh);
  __syncthreads();
  const RefineCtx rc{B, M, K, lo, step};
  const int k0 = (blockIdx.x * kScanThreads + threadIdx.x) * PT;
  scan_points<MP, PT>(Bs, K, S, P, L, k0, rc, sh);
  drain_refinements(rc, P, sh);
}

// Persistent batched scan over the tiles of the jobs of one M bucket. Tiles are striped over
// the CTAs; the job of a tile is found by binary search on the jobs' first tiles.
template <int MP, int PT>
__global__ void __launch_bounds__(kScanThreads) scan_batch_kernel(const uint8_t *plan, uint8_t *ws, int bucket) {
  __shared__ __align__(16) float2 Bs[MP * MP];
  __shared__ ScanShared sh;
  const PlanHeader *h = reinterpret_cast<const PlanHeader *>(plan);
  const int njobs = h->scan_jobs[bucket];
  const int64_t ntiles = h->scan_tiles[bucket];
  const int32_t *list = reinterpret_cast<const int32_t *>(plan + h->off_scan[bucket]);
  const PlanJob *jobs = reinterpret_cast<const PlanJob *>(plan + h->off_job);
  const PlanProblem *probs = reinterpret_cast<const PlanProblem *>(plan + h->off_prob);
  const PlanGrid *grids = reinterpret_cast<const PlanGrid *>(plan + h->off_grid);
  constexpr int TP = kScanThreads * PT;
  int cur = -1;
  for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
    int lo = 0, hi = njobs - 1;
    while (lo < hi) {  // last job with tile_start <= t
      int mid = (lo + hi + 1) >> 1;
      if (jobs[list[mid]].tile_start <= t) lo = mid; else hi = mid - 1;
    }
    const PlanJob &jb = jobs[list[lo]];
    const PlanProblem &pp = probs[jb.prob];
    const double2 *B64 = reinterpret_cast<const double2 *>(ws + jb.B_off);
    if (lo != cur) {
      __syncthreads();
      load_factor<MP>(B64, pp.p.M, jb.K, Bs);
      __syncthreads();
      set_threshold<MP>(Bs, jb.K, sh);
      __syncthreads();
      cur = lo;
    }
    const PlanGrid &g = grids[pp.grid_id];
    const uint32_t *S = reinterpret_cast<const uint32_t *>(ws + g.S_off);
    float *P = pp.p.P + (size_t)jb.slot * g.L;
    const RefineCtx rc{B64, pp.p.M, jb.K, g.lo, g.step};
    const int k0 = (int)(t - jb.tile_start) * TP + threadIdx.x * PT;
    scan_points<MP, PT>(Bs, jb.K, S, P, g.L, k0, rc, sh);
    drain_refinements(rc, P, sh);
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
cudaError_t run_batch(const uint8_t *plan, const PlanHeader &h, uint8_t *ws, int bucket, cudaStream_t s) {
  const int64_t tiles = h.scan_tiles[bucket];
  if (tiles == 0) return cudaSuccess;
  int per_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, scan_batch_kernel<MP, PT>, kScanThreads, 0);
  if (per_sm < 1) per_sm = 1;
  int64_t grid = (int64_t)num_sms() * per_sm;
  if (grid > tiles) grid = tiles;
  scan_batch_kernel<MP, PT><<<(unsigned)grid, kScanThreads, 0, s>>>(plan, ws, bucket);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_grid_table_single(double lo, double step, int L, uint32_t *S, cudaStream_t s) {
  grid_table_single_kernel<<<(L + 255) / 256, 256, 0, s>>>(lo, step, L, S);
  return cudaGetLastError();
}

cudaError_t launch_grid_tables(const uint8_t *plan_dev, const PlanHeader &h, uint8_t *ws, cudaStream_t s) {
  if (h.ngrids == 0) return cudaSuccess;
  int64_t per = (h.grid_points + h.ngrids - 1) / h.ngrids;
  int bx = (int)((per + 255) / 256);
  if (bx > 4096) bx = 4096;
  if (bx < 1) bx = 1;
  grid_table_batch_kernel<<<dim3(bx, h.ngrids), 256, 0, s>>>(plan_dev, ws);
  return cudaGetLastError();
}

cudaError_t launch_scan_single(const double2 *B, int M, int K, int L, double lo, double step, const uint32_t *S,
                               float *P, cudaStream_t s) {
  const int b = m_bucket(M);
  const int tp = kScanThreads * scan_pt_default(b);
  const unsigned grid = (unsigned)((L + tp - 1) / tp);
  switch (b) {
    case 0: scan_single_kernel<8, 4><<<grid, kScanThreads, 0, s>>>(B, M, K, L, lo, step, S, P); break;
    case 1: scan_single_kernel<16, 2><<<grid, kScanThreads, 0, s>>>(B, M, K, L, lo, step, S, P); break;
    case 2: scan_single_kernel<32, 1><<<grid, kScanThreads, 0, s>>>(B, M, K, L, lo, step, S, P); break;
    default: scan_single_kernel<64, 1><<<grid, kScanThreads, 0, s>>>(B, M, K, L, lo, step, S, P); break;
  }
  return cudaGetLastError();
}

cudaError_t launch_scan_batch(const uint8_t *plan_dev, const PlanHeader &h, uint8_t *ws, cudaStream_t s) {
  cudaError_t e;
  switch (h.scan_pt[0]) {
    case 1: e = run_batch<8, 1>(plan_dev, h, ws, 0, s); break;
    case 2: e = run_batch<8, 2>(plan_dev, h, ws, 0, s); break;
    default: e = run_batch<8, 4>(plan_dev, h, ws, 0, s); break;
  }
  if (e != cudaSuccess) return e;
  switch (h.scan_pt[1]) {
    case 1: e = run_batch<16, 1>(plan_dev, h, ws, 1, s); break;
    case 4: e = run_batch<16, 4>(plan_dev, h, ws, 1, s); break;
    default: e = run_batch<16, 2>(plan_dev, h, ws, 1, s); break;
  }
  if (e != cudaSuccess) return e;
  if (h.scan_pt[2] == 2)
    e = run_batch<32, 2>(plan_dev, h, ws, 2, s);
  else
    e = run_batch<32, 1>(plan_dev, h, ws, 2, s);
  if (e != cudaSuccess) return e;
  return run_batch<64, 1>(plan_dev, h, ws, 3, s);
}

}  // namespace doa
