// Step-5 (Table 2; steering vector Eq. 2): pseudospectrum P_k = 1 / ||B^H a(theta_k)||^2, which
// equals 1 / (a^H C a) for the weighting matrix C = B B^H of Table 3 and is never negative.
//
// Fused, on CUDA cores in FP32: every thread evaluates PT consecutive grid points. For M <= 16
// a ULA's steering vector is the power sequence of z = e^{j pi sin theta_k}, so each column output
// is a polynomial in z, evaluated by the blocked Horner scheme of scan_common.cuh from two phasors
// per point (z and z^4, from the grid's 32-bit phase step S_k by exact integer arithmetic:
// phase of element m = m*S_k mod 2^32; phasor_q32 turns a phase into cos + j sin). Larger arrays
// generate the M phasors of each point in registers and contract them directly. Either way the
// factor is held in shared memory as FP32 and read as warp-wide broadcasts, one column at a
// time, and the readouts of scan_common.cuh are formed.
//
// Batched: one scan job per problem. A problem that asks for MUSIC or EV contracts its noise
// eigenvectors E_n once and reads MUSIC, EV and PHD (v_min is the last column of E_n) from the
// same column outputs, plus one extra column for MN (valph); PHD / MN alone contract one column
// each. All four of Table 3's spectra of one problem therefore share one steering generation.
//
// Near-null refinement: where the FP32 denominator is small its relative error grows (the
// contraction cancels), so every point with den_r < C * E_r for some readout r is
// re-evaluated with FP64 steering and contraction (exact 64-bit phases m * S64_k from a per-grid
// table in the batch, else from sin theta_k recomputed in FP64) and the FP64 factor, for all
// readouts of the job. Flagged points of a
// tile are queued in shared memory and each is then handled by a whole warp (lanes own phasors,
// then elements of columns), so the FP64 work runs without divergence. With per-term FP32
// errors below ~4 eps (direct sum; C = kRefineC) or ~3 eps (blocked Horner; C = kRefineCH) the
// FP32 result elsewhere stays within ~5e-4 relative.
#include <float.h>

#include <algorithm>
#include <math_constants.h>

#include "doa_internal.cuh"
#include "scan_common.cuh"

namespace doa {
namespace {

using namespace scanc;

__global__ void grid_table_single_kernel(double lo, double step, int k0, int n, uint32_t *S) {
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k < n) S[k] = grid_phase_step(lo, step, k0 + k);
}

__global__ void grid_table_batch_kernel(const uint8_t *plan, uint8_t *ws) {
  const PlanHeader *h = reinterpret_cast<const PlanHeader *>(plan);
  const PlanGrid g = reinterpret_cast<const PlanGrid *>(plan + h->off_grid)[blockIdx.y];
  uint32_t *S = reinterpret_cast<uint32_t *>(ws + g.S_off);
  uint64_t *S64 = reinterpret_cast<uint64_t *>(ws + g.S64_off);
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < g.L; k += gridDim.x * blockDim.x) {
    const double theta = __dadd_rn(g.lo, __dmul_rn((double)k, g.step));
    const double s = sin(theta * 0.017453292519943295);
    S[k] = phase_step_of_sin(s);
    S64[k] = phase_step64_of_sin(s);
  }
}

template <int MP, int PT>
__global__ void __launch_bounds__(kScanThreads) scan_single_kernel(const double2 *B, int M, int K, int L, double lo,
                                                                   double step, int kofs, const uint32_t *S,
                                                                   float *P) {
  __shared__ __align__(16) float2 Bs[MP * MP];
  __shared__ ScanShared sh;
  ScanJob j{};
  j.F = B;
  j.P[kRoMusic] = P;
  j.lo = lo;
  j.step = step;
  j.M = M;
  j.Kf = K;
  j.Kn = K;
  j.kphd = j.kmn = -1;
  j.kofs = kofs;
  load_job<MP>(j, Bs, sh);
  __syncthreads();
  set_threshold<MP, true>(Bs, j, sh);
  __syncthreads();
  const int k0 = (blockIdx.x * kScanThreads + threadIdx.x) * PT;
  scan_points<MP, PT>(Bs, j, S, L, k0, sh);
  drain_refinements(j, sh);
}

// Scan job of a ULA problem of the batch on its grid (factor and EV weights in the workspace).
__device__ __forceinline__ ScanJob ula_job(const PlanProblem &pp, const PlanGrid &g, const uint8_t *ws) {
  ScanJob j{};
  j.F = reinterpret_cast<const double2 *>(ws + pp.fac_off);
  j.w = pp.Kn > 0 && pp.slot[DOA_EV] >= 0
            ? reinterpret_cast<const double *>(ws + pp.fac_off) + 2 * pp.p.M * (pp.p.M + 1)
            : nullptr;
  j.S64 = reinterpret_cast<const uint64_t *>(ws + g.S64_off);
  for (int r = 0; r < 4; ++r) j.P[r] = pp.slot[r] >= 0 ? pp.p.P + (size_t)pp.slot[r] * g.L : nullptr;
  j.lo = g.lo;
  j.step = g.step;
  j.M = pp.p.M;
  j.Kf = pp.Kf;
  j.Kn = pp.Kn;
  j.kphd = pp.kphd;
  j.kmn = pp.kmn;
  j.kofs = 0;
  return j;
}

// Persistent batched scan over the tiles of the problems of one M bucket. The tiles are dealt
// to the CTAs in runs of consecutive tiles, run r to CTA r mod gridDim: consecutive tiles
// mostly share a problem (its factor stays in shared memory), while the runs of problems of
// different cost (columns, M) spread evenly over the CTAs. The problem of a run's first tile
// comes from a binary search on the problems' first tiles, the following ones by stepping.
// Flagged points queue up over the run and are re-evaluated when it ends or its problem changes.
constexpr int kRun = 16;   // longest run (large batches); small ones use shorter runs so every SM gets one

template <int MP, int PT>
__global__ void __launch_bounds__(kScanThreads) scan_batch_kernel(const uint8_t *plan, uint8_t *ws, int bucket,
                                                                  int run_len) {
  // factor: (bx, bx, by, by) per element for the paired contraction (PT even), else (bx, by)
  constexpr bool kPair = PT % 2 == 0;
  __shared__ __align__(16) float Fsm[(kPair ? 4 : 2) * (MP + 1) * MP];
  float2 *Bs = reinterpret_cast<float2 *>(Fsm);
  float4 *Bd = reinterpret_cast<float4 *>(Fsm);
  __shared__ ScanShared sh;
  const PlanHeader *h = reinterpret_cast<const PlanHeader *>(plan);
  const int nunits = h->scan_jobs[bucket];
  const int64_t ntiles = h->scan_tiles[bucket];
  const int32_t *list = reinterpret_cast<const int32_t *>(plan + h->off_scan[bucket]);
  const PlanProblem *probs = reinterpret_cast<const PlanProblem *>(plan + h->off_prob);
  const PlanGrid *grids = reinterpret_cast<const PlanGrid *>(plan + h->off_grid);
  constexpr int TP = kScanThreads * PT;
  int cur = -1;
  ScanJob j{};
  const PlanProblem *pp = nullptr;
  const PlanGrid *g = nullptr;
  // runs are taken from a counter in the workspace (zeroed at the start of the solve)
  __shared__ unsigned s_run;
  unsigned *next_run = reinterpret_cast<unsigned *>(ws) + kCtrBatch + bucket;
  for (;;) {
    if (threadIdx.x == 0) s_run = atomicAdd(next_run, 1u);
    __syncthreads();   // the previous run ended with a barrier, so s_run is not read while rewritten
    const int64_t run = s_run;
    if (run * run_len >= ntiles) break;
    const int64_t t_begin = run * run_len, t_end = min(ntiles, t_begin + run_len);
    int u = 0, hi = nunits - 1;
    while (u < hi) {  // last problem with tile_start <= t_begin
      int mid = (u + hi + 1) >> 1;
      if (probs[list[mid]].tile_start <= t_begin) u = mid; else hi = mid - 1;
    }
    for (int64_t t = t_begin; t < t_end; ++t) {
      while (u + 1 < nunits && probs[list[u + 1]].tile_start <= t) ++u;
      if (u != cur) {
        if (cur >= 0) drain_refinements(j, sh);   // the queued points belong to the previous problem
        pp = &probs[list[u]];
        g = &grids[pp->grid_id];
        j = ula_job(*pp, *g, ws);
        __syncthreads();
        if constexpr (kPair) load_job2<MP>(j, Bd, sh); else load_job<MP>(j, Bs, sh);
        __syncthreads();
        if constexpr (kPair) set_threshold2<MP, true>(Bd, j, sh); else set_threshold<MP, true>(Bs, j, sh);
        __syncthreads();
        cur = u;
      }
      const uint32_t *S = reinterpret_cast<const uint32_t *>(ws + g->S_off);
      const int k0 = (int)(t - pp->tile_start) * TP + threadIdx.x * PT;
      if constexpr (kPair)
        scan_points2<MP, PT>(Bd, j, S, g->L, k0, sh);
      else
        scan_points<MP, PT>(Bs, j, S, g->L, k0, sh);
    }
    drain_refinements(j, sh);   // once per run: the warps share the FP64 work of its tiles
  }
}

// Grid-shared scan (problems of one M bucket that share a grid, in groups of up to
// kScanGroupMax). A unit is one tile of the grid for every problem of a group: the CTA generates
// the tile's steering once (w and w^4 per point in the Horner form, the M phasors otherwise), keeps
// it in registers and contracts it with the factor of each problem of the group in turn, so the
// phasor polynomials cost 1 / count of the per-problem scan and nearly every instruction left is
// a contraction FMA. Each problem's FP32 factor, EV
// weights and thresholds were written once per solve by scan_prep_kernel (the same values the
// per-problem scan computes), so every point gets bit for bit the spectrum of the per-problem
// scan. Flagged points of all the group's problems queue up with their problem's position in the
// group and are re-evaluated in FP64 when the unit ends.

// FP32 copy of each grouped problem's factor (one warp per problem): F32 as (bx, bx, by, by) per
// element, w32, thresholds.
template <int MP>
__global__ void __launch_bounds__(kScanThreads) scan_prep_kernel(const uint8_t *plan, uint8_t *ws, int bucket) {
  const PlanHeader *h = reinterpret_cast<const PlanHeader *>(plan);
  const int32_t *list = reinterpret_cast<const int32_t *>(plan + h->off_sgl[bucket]);
  const PlanProblem *probs = reinterpret_cast<const PlanProblem *>(plan + h->off_prob);
  const int i = blockIdx.x * kScanWarps + (threadIdx.x >> 5), lane = threadIdx.x & 31;
  if (i >= h->sg_probs[bucket]) return;
  const PlanProblem &pp = probs[list[i]];
  const int M = pp.p.M, Kf = pp.Kf, Kn = pp.Kn;
  const double2 *F = reinterpret_cast<const double2 *>(ws + pp.fac_off);
  const double *w = pp.Kn > 0 && pp.slot[DOA_EV] >= 0 ? reinterpret_cast<const double *>(F + M * (M + 1)) : nullptr;
  float4 *F32 = reinterpret_cast<float4 *>(ws + pp.fac_off + fac32_off(M));
  float *w32 = reinterpret_cast<float *>(F32 + (M + 1) * MP);
  for (int e = lane; e < Kf * MP; e += 32) {
    const int k = e / MP, m = e % MP;
    float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
    if (m < M) {
      const double2 b = F[(size_t)k * M + m];
      const float bx = (float)b.x, by = (float)b.y;
      v = make_float4(bx, bx, by, by);
    }
    F32[e] = v;
  }
  for (int k = lane; k < Kn; k += 32) w32[k] = w ? (float)w[k] : 1.f;
  __syncwarp();
  float thr[4] = {0.f, 0.f, 0.f, 0.f};
  job_thresholds2<MP, true>(F32, w32, Kf, Kn, pp.kphd, pp.kmn, thr);
  if (lane < 4) w32[MP + lane] = thr[lane];
}

// 16-byte global -> shared copies that complete asynchronously (one group per problem).
__device__ __forceinline__ void cp_async16(void *dst, const void *src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"((uint32_t)__cvta_generic_to_shared(dst)),
               "l"(src)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

// CTAs per SM the register budget of the grid-shared scan is set for: 4 where the steering of a
// thread's points fits in 128 registers without spilling, else 3.
template <int MP, int PT>
__host__ __device__ constexpr int shared_min_blocks() {
  return MP <= 16 || (MP == 32 && PT == 1) ? 4 : 3;
}

template <int MP, int PT>
__global__ void __launch_bounds__(kScanThreads, shared_min_blocks<MP, PT>())
    scan_shared_kernel(const uint8_t *plan, uint8_t *ws, int bucket) {
  constexpr bool kPair = PT % 2 == 0;
  // paired form: two factor buffers; the next problem's factor, EV weights and thresholds are
  // copied asynchronously while the current one is contracted
  constexpr int kBufs = kPair ? 2 : 1;
  __shared__ __align__(16) float Fsm[kBufs][(kPair ? 4 : 2) * (MP + 1) * MP];
  __shared__ __align__(16) float Wsm[kBufs][MP + 4];   // EV weights, then the 4 thresholds
  __shared__ uint8_t tags[kFlagCap];
  __shared__ ScanShared sh;
  __shared__ ScanJob jobs[kScanGroupMax];   // the current group's jobs (read once per group)
  const PlanHeader *h = reinterpret_cast<const PlanHeader *>(plan);
  const PlanScanGroup *groups = reinterpret_cast<const PlanScanGroup *>(plan + h->off_sg[bucket]);
  const int ngroups = h->sg_groups[bucket];
  const int64_t nunits = h->sg_units[bucket];
  const int32_t *list = reinterpret_cast<const int32_t *>(plan + h->off_sgl[bucket]);
  const PlanProblem *probs = reinterpret_cast<const PlanProblem *>(plan + h->off_prob);
  const PlanGrid *grids = reinterpret_cast<const PlanGrid *>(plan + h->off_grid);
  const int tid = threadIdx.x, warp = tid >> 5;
  constexpr int TP = kScanThreads * PT;
  if (tid == 0) sh.nflag = 0;
  int cached = -1;   // group whose jobs are in shared memory (every thread holds the same value)
  // units are taken from a counter in the workspace (zeroed at the start of the solve), so the
  // CTAs that meet cheap units (a grid's short last tile, few near-null points) take more of them
  // and all end together
  __shared__ unsigned s_unit;
  unsigned *next_unit = reinterpret_cast<unsigned *>(ws) + kCtrShared + bucket;
  for (;;) {
    if (tid == 0) s_unit = atomicAdd(next_unit, 1u);
    __syncthreads();   // the previous unit ended with a barrier, so s_unit is not read while rewritten
    const int64_t u = s_unit;
    if (u >= nunits) break;
    int gi = 0, hi = ngroups - 1;
    while (gi < hi) {  // last group with unit_start <= u
      const int mid = (gi + hi + 1) >> 1;
      if (groups[mid].unit_start <= u) gi = mid; else hi = mid - 1;
    }
    const PlanScanGroup gr = groups[gi];
    const PlanGrid &g = grids[gr.grid_id];
    const int L = g.L, k0 = (int)(u - gr.unit_start) * TP + tid * PT;
    const uint32_t *S = reinterpret_cast<const uint32_t *>(ws + g.S_off);
    if (gi != cached) {   // the previous unit's drain has ended (barrier at its end)
      for (int i = tid; i < gr.count; i += kScanThreads) jobs[i] = ula_job(probs[list[gr.first + i]], g, ws);
      __syncthreads();
      cached = gi;
    }
    // the copies of problem i of the group into buffer b (Kf columns of the factor, then the
    // MP EV weights and 4 thresholds, all 16-byte multiples)
    auto issue = [&](int i, int b) {
      const ScanJob &ji = jobs[i];
      const uint8_t *f32 = reinterpret_cast<const uint8_t *>(ji.F) + fac32_off(ji.M);
      const float4 *src = reinterpret_cast<const float4 *>(f32);
      float4 *dst = reinterpret_cast<float4 *>(Fsm[b]);
      for (int e = tid; e < ji.Kf * MP; e += kScanThreads) cp_async16(dst + e, src + e);
      const float4 *wsrc = reinterpret_cast<const float4 *>(f32 + (size_t)(ji.M + 1) * MP * 16);
      for (int e = tid; e < (MP + 4) / 4; e += kScanThreads) cp_async16(reinterpret_cast<float4 *>(Wsm[b]) + e, wsrc + e);
      cp_async_commit();
    };
    if constexpr (kPair) issue(0, 0);
    // steering of the unit's points: w and w4 (Horner form) or the phasor block (direct form)
    constexpr bool kH = ula_horner_form<MP>();
    HornerW1 hw[!kH || kPair ? 1 : PT];
    HornerW2 hw2[kH && kPair ? PT / 2 : 1];
    float2 a[!kH && !kPair ? PT : 1][kH ? 1 : MP];
    uint64_t ax[!kH && kPair ? PT / 2 : 1][kH ? 1 : MP], ay[!kH && kPair ? PT / 2 : 1][kH ? 1 : MP];
    if constexpr (kH && kPair)
      ula_horner2<PT>(S, L, k0, hw2);
    else if constexpr (kH)
      ula_horner<PT>(S, L, k0, hw);
    else if constexpr (kPair)
      ula_phasors2<MP, PT>(S, L, k0, ax, ay);
    else
      ula_phasors<MP, PT>(S, L, k0, a);
    for (int i = 0; i < gr.count; ++i) {
      const ScanJob &j = jobs[i];
      if constexpr (kPair) {
        const int b = i & 1;
        cp_async_wait_all();   // this thread's copies of problem i have landed
        __syncthreads();       // everyone's have; and problem i - 1 is no longer read from buffer b ^ 1
        if (i + 1 < gr.count) issue(i + 1, b ^ 1);
        if constexpr (kH)
          contract_horner2<MP, PT, UlaSource, true>(reinterpret_cast<const float4 *>(Fsm[b]), j, hw2, L, k0, sh,
                                                    UlaSource{&j}, Wsm[b], Wsm[b] + MP, tags, i);
        else
          contract_points2<MP, PT, UlaSource, true>(reinterpret_cast<const float4 *>(Fsm[b]), j, ax, ay, L, k0, sh,
                                                    UlaSource{&j}, Wsm[b], Wsm[b] + MP, tags, i);
      } else {
        const uint8_t *f32 = reinterpret_cast<const uint8_t *>(j.F) + fac32_off(j.M);
        float2 *Bs = reinterpret_cast<float2 *>(Fsm[0]);
        __syncthreads();   // the previous problem's contraction has finished reading Bs
        const float4 *src4 = reinterpret_cast<const float4 *>(f32);
        for (int e = tid; e < j.Kf * MP; e += kScanThreads) {
          const float4 v = src4[e];
          Bs[e] = make_float2(v.x, v.z);
        }
        const float *wg = reinterpret_cast<const float *>(f32 + (size_t)(j.M + 1) * MP * 16);
        for (int k = tid; k < MP + 4; k += kScanThreads) Wsm[0][k] = wg[k];
        __syncthreads();
        if constexpr (kH)
          contract_horner<MP, PT, UlaSource, true>(Bs, j, hw, L, k0, sh, UlaSource{&j}, Wsm[0], Wsm[0] + MP, tags, i);
        else
          contract_points<MP, PT, UlaSource, true>(Bs, j, a, L, k0, sh, UlaSource{&j}, Wsm[0], Wsm[0] + MP, tags, i);
      }
    }
    // FP64 re-evaluation of the unit's flagged points, several per warp for small factors; the
    // queue holds the points of each problem together (problems run one after the other)
    __syncthreads();
    const int n = queue_front(sh.nflag), nb = queue_back(sh.nflag);
    for (int i0 = warp * 4; i0 < n; i0 += kScanWarps * 4) {
      const int end = min(i0 + 4, n);
      for (int c0 = i0; c0 < end;) {
        const int tag = tags[c0];
        int c1 = c0 + 1;
        while (c1 < end && tags[c1] == tag) ++c1;
        const ScanJob &j = jobs[tag];
        const float *wg = reinterpret_cast<const float *>(reinterpret_cast<const uint8_t *>(j.F) + fac32_off(j.M) +
                                                          (size_t)(j.M + 1) * MP * 16);
        const UlaSource src{&j};
        if (j.M <= 8 && j.Kf <= 8) {
          refine_points_subwarp<8>(j, sh.flags + c0, c1 - c0, src, wg, sh.ph[warp]);
        } else if (j.M <= 16 && j.Kf <= 16) {
          for (int c = c0; c < c1; c += 2) refine_points_subwarp<16>(j, sh.flags + c, min(2, c1 - c), src, wg, sh.ph[warp]);
        } else {
          for (int c = c0; c < c1; ++c) refine_point_warp_src(j, sh.flags[c], src, wg, sh.ph[warp], sh.yb[warp]);
        }
        c0 = c1;
      }
    }
    // points flagged for PHD / MN alone (the back of the queue): those columns only
    for (int i0 = kFlagCap - nb + warp * 4; i0 < kFlagCap; i0 += kScanWarps * 4) {
      const int end = min(i0 + 4, kFlagCap);
      for (int c0 = i0; c0 < end;) {
        const int tag = tags[c0];
        int c1 = c0 + 1;
        while (c1 < end && tags[c1] == tag) ++c1;
        const ScanJob &j = jobs[tag];
        refine_single_run(j, sh.flags + c0, sh.fmask + c0, c1 - c0, UlaSource{&j});
        c0 = c1;
      }
    }
    __syncthreads();
    if (tid == 0) sh.nflag = 0;
  }
}

// Peak polish (DOA_FLAG_POLISH_PEAKS): one warp per problem re-evaluates, with the FP64
// steering and contraction of the scan's refinement (two or four points per pass in sub-warps
// for small factors), every readout of the problem at the union of its algorithms' picked peaks
// and their two neighbours on each side (each point once); the
// peaks are then picked again. A peak whose outcome the FP32 values already decide is skipped:
// the FP32 spectrum is within kPolishCertain / 2 (relative) of the FP64 one, so when every pair of
// consecutive points from k-3 to k+3 differs by more than kPolishCertain, and the algorithm's
// weakest selected peak exceeds its best unselected one by more than that, re-evaluating in FP64
// cannot change which points are peaks or which are selected.
constexpr int kPolishWarps = 4;
constexpr int kPolishMax = 4 * kMaxM;
constexpr float kPolishCertain = 2e-3f;   // twice the FP32 path's relative error bound (5e-4), doubled

__device__ __forceinline__ bool order_certain(float a, float b) {
  return fabsf(a - b) > kPolishCertain * fmaxf(a, b);
}

__global__ void __launch_bounds__(32 * kPolishWarps) polish_batch_kernel(const uint8_t *plan, uint8_t *ws) {
  __shared__ double2 ph[kPolishWarps][kMaxM];
  __shared__ float2 yb[kPolishWarps][kMaxCols];
  __shared__ float w32[kPolishWarps][kMaxM];
  __shared__ int pk[kPolishWarps][kPolishMax];
  __shared__ int cand[kPolishWarps][kPolishMax];
  __shared__ int pts[kPolishWarps][4];
  const PlanHeader *h = reinterpret_cast<const PlanHeader *>(plan);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int prob = blockIdx.x * kPolishWarps + warp;
  if (prob >= h->nprob) return;
  const PlanProblem &pp = reinterpret_cast<const PlanProblem *>(plan + h->off_prob)[prob];
  if (!(pp.p.flags & DOA_FLAG_POLISH_PEAKS) || pp.p.d < 1) return;
  const PlanGrid &g = reinterpret_cast<const PlanGrid *>(plan + h->off_grid)[pp.grid_id];
  ScanJob j{};
  j.F = reinterpret_cast<const double2 *>(ws + pp.fac_off);
  j.w = pp.Kn > 0 && pp.slot[DOA_EV] >= 0
            ? reinterpret_cast<const double *>(ws + pp.fac_off) + 2 * pp.p.M * (pp.p.M + 1)
            : nullptr;
  j.S64 = reinterpret_cast<const uint64_t *>(ws + g.S64_off);
  for (int r = 0; r < 4; ++r) j.P[r] = pp.slot[r] >= 0 ? pp.p.P + (size_t)pp.slot[r] * g.L : nullptr;
  j.lo = g.lo;
  j.step = g.step;
  j.M = pp.p.M;
  j.Kf = pp.Kf;
  j.Kn = pp.Kn;
  j.kphd = pp.kphd;
  j.kmn = pp.kmn;
  j.kofs = 0;
  for (int c = lane; c < j.Kn; c += 32) w32[warp][c] = j.w ? (float)j.w[c] : 1.f;
  const int d = pp.p.d, L = g.L;
  const float *next = h->next_val_off >= 0 ? reinterpret_cast<const float *>(ws + h->next_val_off) : nullptr;
  // lane s < njobs: is job s's selection decided by its FP32 values (its weakest selected peak
  // above its best unselected value by more than the FP32 error)?
  bool bnd = true;
  if (lane < pp.njobs) {
    const int cnt = min(pp.p.peak_count[lane], d);
    if (cnt == d && next) {
      float vmin = INFINITY;
      for (int q = 0; q < cnt; ++q) vmin = fminf(vmin, pp.p.peak_val[(size_t)lane * d + q]);
      const float nv = next[pp.first_job + lane];
      bnd = !(nv > -INFINITY) || (vmin > nv && order_certain(vmin, nv));
    }
  }
  const unsigned bmask = __ballot_sync(0xffffffffu, bnd);
  // lane e takes peak e % d of job e / d: undecided peaks go to cand[] (one round of loads for all)
  int ncand = 0;
  for (int e0 = 0; e0 < pp.njobs * d; e0 += 32) {
    const int e = e0 + lane;
    int k = -1;
    if (e < pp.njobs * d) {
      const int sj = e / d, q = e % d;
      if (q < min(pp.p.peak_count[sj], d)) {
        k = pp.p.peak_idx[(size_t)sj * d + q];
        const float *Ps = pp.p.P + (size_t)sj * L;
        const int i0 = max(k - 3, 0), i1 = min(k + 3, L - 1);
        float v[7];
#pragma unroll
        for (int t = 0; t < 7; ++t) v[t] = i0 + t <= i1 ? Ps[i0 + t] : 0.f;
        bool decided = ((bmask >> sj) & 1u) && next;
#pragma unroll
        for (int t = 0; t < 6; ++t) decided = decided && (i0 + t >= i1 || order_certain(v[t], v[t + 1]));
        if (decided) k = -1;
      }
    }
    const unsigned um = __ballot_sync(0xffffffffu, k >= 0);
    if (k >= 0) cand[warp][ncand + __popc(um & ((1u << lane) - 1u))] = k;
    ncand += __popc(um);
  }
  __syncwarp();
  int n = 0;
  if (lane == 0) {   // the undecided peaks, sorted, each once
    for (int c = 0; c < ncand; ++c) {
      const int k = cand[warp][c];
      int a = n;
      while (a > 0 && pk[warp][a - 1] > k) --a;
      if (a > 0 && pk[warp][a - 1] == k) continue;
      for (int b = n; b > a; --b) pk[warp][b] = pk[warp][b - 1];
      pk[warp][a] = k;
      ++n;
    }
  }
  n = __shfl_sync(0xffffffffu, n, 0);
  __syncwarp();
  // mark the problem's jobs for the second pick (a NaN in their next-value slots); the jobs of a
  // problem with nothing to polish keep their first pick
  if (n > 0 && next && lane < pp.njobs) const_cast<float *>(next)[pp.first_job + lane] = CUDART_NAN_F;
  // the points, each once and in increasing order, several per pass for small factors (sub-warps
  // of 8 or 16 lanes per point, as in the scan's refinement), else one per pass
  const bool sub8 = j.M <= 8 && j.Kf <= 8, sub16 = !sub8 && j.M <= 16 && j.Kf <= 16;
  const int per = sub8 ? 4 : (sub16 ? 2 : 1);
  int last = -1, nb = 0;
  auto flush = [&]() {
    __syncwarp();
    if (sub8)
      refine_points_subwarp<8>(j, pts[warp], nb, UlaSource{&j}, w32[warp], ph[warp]);
    else if (sub16)
      refine_points_subwarp<16>(j, pts[warp], nb, UlaSource{&j}, w32[warp], ph[warp]);
    else
      refine_point_warp(j, pts[warp][0], w32[warp], ph[warp], yb[warp]);
    __syncwarp();
    nb = 0;
  };
  for (int i = 0; i < n; ++i) {
    const int k0 = pk[warp][i];
    for (int k = max(max(k0 - 2, last + 1), 0); k <= min(k0 + 2, L - 1); ++k) {
      if (lane == 0) pts[warp][nb] = k;
      ++nb;
      last = k;
      if (nb == per) flush();
    }
  }
  if (nb > 0) flush();
}


template <int MP, int PT>
cudaError_t run_batch(const uint8_t *plan, const PlanHeader &h, uint8_t *ws, int bucket, cudaStream_t s) {
  const int64_t tiles = h.scan_tiles[bucket];
  if (tiles == 0) return cudaSuccess;
  int per_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, scan_batch_kernel<MP, PT>, kScanThreads, 0);
  if (per_sm < 1) per_sm = 1;
  const int64_t cap = (int64_t)device_sm_count() * per_sm;
  const int run_len = (int)std::min<int64_t>(kRun, std::max<int64_t>(1, (tiles + cap - 1) / cap));
  const int64_t grid = std::min<int64_t>(cap, (tiles + run_len - 1) / run_len);
  scan_batch_kernel<MP, PT><<<(unsigned)grid, kScanThreads, 0, s>>>(plan, ws, bucket, run_len);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_grid_table_single(double lo, double step, int k0, int n, uint32_t *S, cudaStream_t s) {
  grid_table_single_kernel<<<(n + 255) / 256, 256, 0, s>>>(lo, step, k0, n, S);
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

cudaError_t launch_scan_single(const double2 *B, int M, int K, int L, double lo, double step, int kofs,
                               const uint32_t *S, float *P, cudaStream_t s) {
  const int b = m_bucket(M);
  const int tp = kScanThreads * scan_pt_default(b);
  const unsigned grid = (unsigned)((L + tp - 1) / tp);
  switch (b) {
    case 0: scan_single_kernel<8, 4><<<grid, kScanThreads, 0, s>>>(B, M, K, L, lo, step, kofs, S, P); break;
    case 1: scan_single_kernel<16, 4><<<grid, kScanThreads, 0, s>>>(B, M, K, L, lo, step, kofs, S, P); break;
    case 2: scan_single_kernel<32, 1><<<grid, kScanThreads, 0, s>>>(B, M, K, L, lo, step, kofs, S, P); break;
    default: scan_single_kernel<64, 1><<<grid, kScanThreads, 0, s>>>(B, M, K, L, lo, step, kofs, S, P); break;
  }
  return cudaGetLastError();
}

cudaError_t launch_polish_batch(const uint8_t *plan_dev, const PlanHeader &h, uint8_t *ws, cudaStream_t s) {
  if (h.nprob == 0) return cudaSuccess;
  polish_batch_kernel<<<(h.nprob + kPolishWarps - 1) / kPolishWarps, 32 * kPolishWarps, 0, s>>>(plan_dev, ws);
  return cudaGetLastError();
}

template <int MP, int PT>
cudaError_t run_shared(const uint8_t *plan, const PlanHeader &h, uint8_t *ws, int bucket, cudaStream_t s) {
  if (h.sg_units[bucket] == 0) return cudaSuccess;
  scan_prep_kernel<MP><<<(h.sg_probs[bucket] + kScanWarps - 1) / kScanWarps, kScanThreads, 0, s>>>(plan, ws, bucket);
  int per_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, scan_shared_kernel<MP, PT>, kScanThreads, 0);
  if (per_sm < 1) per_sm = 1;
  const int64_t grid = std::min<int64_t>((int64_t)device_sm_count() * per_sm, h.sg_units[bucket]);
  scan_shared_kernel<MP, PT><<<(unsigned)grid, kScanThreads, 0, s>>>(plan, ws, bucket);
  return cudaGetLastError();
}

static cudaError_t launch_scan_shared(const uint8_t *plan_dev, const PlanHeader &h, uint8_t *ws, cudaStream_t s) {
  cudaError_t e;
  switch (h.scan_pt[0]) {
    case 1: e = run_shared<8, 1>(plan_dev, h, ws, 0, s); break;
    case 2: e = run_shared<8, 2>(plan_dev, h, ws, 0, s); break;
    default: e = run_shared<8, 4>(plan_dev, h, ws, 0, s); break;
  }
  if (e != cudaSuccess) return e;
  switch (h.scan_pt[1]) {
    case 1: e = run_shared<16, 1>(plan_dev, h, ws, 1, s); break;
    case 4: e = run_shared<16, 4>(plan_dev, h, ws, 1, s); break;
    default: e = run_shared<16, 2>(plan_dev, h, ws, 1, s); break;
  }
  if (e != cudaSuccess) return e;
  if (h.scan_pt[2] == 2)
    e = run_shared<32, 2>(plan_dev, h, ws, 2, s);
  else
    e = run_shared<32, 1>(plan_dev, h, ws, 2, s);
  if (e != cudaSuccess) return e;
  return run_shared<64, 1>(plan_dev, h, ws, 3, s);
}

cudaError_t launch_scan_batch(const uint8_t *plan_dev, const PlanHeader &h, uint8_t *ws, cudaStream_t s) {
  cudaError_t e = launch_scan_shared(plan_dev, h, ws, s);
  if (e != cudaSuccess) return e;
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
