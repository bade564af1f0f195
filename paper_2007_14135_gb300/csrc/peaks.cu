// Step-6 (Table 2): findPeaks + PeakSelection(peakVals, inds, D), one CTA per spectrum.
//
// A peak is the left end i of a maximal run [i..j] of equal values with 1 <= i, j <= L-2,
// P[i-1] < P[i] and P[j+1] < P[j]. The D largest peaks are selected (equal values: lower
// index first) and written in ascending index order.
//
// Thread t owns the aligned quads of four points t, t + 256, ... (16-byte coalesced loads) and
// keeps its best kCache peaks in registers. Each warp picks its D best in D rounds of a warp
// arg-max (the winning lane pops its head and, if its cache runs dry while it still has peaks,
// rescans its quads for the next ones below its last selected peak); one warp then merges the
// warps' lists. This realises the shared-memory max-reduction that the paper names as future work
// for Step-6 (Sec. 6).
#include <climits>

#include "doa_internal.cuh"
#include "peaks_common.cuh"

namespace doa {
namespace {

using namespace pk;

// Writes the nsel selected peaks in ascending index order (thread 0).
__device__ void write_sel(Cand *sel, int nsel, int *idx, float *val, int *count) {
  if (threadIdx.x == 0) {
    for (int a = 1; a < nsel; ++a) {
      Cand c = sel[a];
      int b = a - 1;
      while (b >= 0 && sel[b].i > c.i) {
        sel[b + 1] = sel[b];
        --b;
      }
      sel[b + 1] = c;
    }
    for (int a = 0; a < nsel; ++a) {
      idx[a] = sel[a].i;
      val[a] = sel[a].v;
    }
    *count = nsel;
  }
}

// next (nullable): receives the value of the (d+1)-th best peak (-inf if there is none).
__device__ void peaks_block(const float *__restrict__ P, int L, int d, int *idx, float *val, int *count,
                            float *next = nullptr) {
  __shared__ Cand sel[kMaxM + 1];
  const int want = next ? d + 1 : d;
  int nsel = select_top(P, L, want, sel);
  if (next) {
    if (threadIdx.x == 0) *next = nsel > d ? sel[d].v : -INFINITY;
    nsel = min(nsel, d);
  }
  write_sel(sel, nsel, idx, val, count);
}

__device__ void peaks2d_block(const float *__restrict__ P, int La, int Le, bool wrap, int d, int *idx, float *val,
                              int *count) {
  __shared__ Cand sel[kMaxM];
  const int nsel = select_top2d(P, La, Le, wrap, d, sel);
  write_sel(sel, nsel, idx, val, count);
}

__global__ void __launch_bounds__(kPeakThreads) peaks2d_single_kernel(const float *P, int La, int Le, int wrap, int d,
                                                                      int *idx, float *val, int *count) {
  peaks2d_block(P, La, Le, wrap != 0, d, idx, val, count);
}

__global__ void __launch_bounds__(kPeakThreads) peaks_single_kernel(const float *P, int L, int d, int *idx, float *val,
                                                                    int *count) {
  peaks_block(P, L, d, idx, val, count);
}

// One CTA per (problem, algorithm) job; the 1-D and 2-D rules run as separate kernels (each skips
// the other kind's jobs) so that each keeps its own register budget.
// repick: the pick after the peak polish, only for the jobs the polish marked (NaN next value).
__global__ void __launch_bounds__(kPeakThreads, 5) peaks_batch_kernel(const uint8_t *plan, uint8_t *ws, int repick) {
  const PlanHeader *h = reinterpret_cast<const PlanHeader *>(plan);
  const PlanJob &jb = reinterpret_cast<const PlanJob *>(plan + h->off_job)[blockIdx.x];
  const PlanProblem &pp = reinterpret_cast<const PlanProblem *>(plan + h->off_prob)[jb.prob];
  if (pp.p.geom.pos) return;
  const int L = pp.npts, d = pp.p.d;
  const bool polish = (pp.p.flags & DOA_FLAG_POLISH_PEAKS) && h->next_val_off >= 0;
  float *next = polish ? reinterpret_cast<float *>(ws + h->next_val_off) + blockIdx.x : nullptr;
  if (repick) {
    if (!polish || !isnan(*next)) return;
    next = nullptr;
  }
  peaks_block(pp.p.P + (size_t)jb.slot * L, L, d, pp.p.peak_idx + (size_t)jb.slot * d,
              pp.p.peak_val + (size_t)jb.slot * d, pp.p.peak_count + jb.slot, next);
}

__global__ void __launch_bounds__(kPeakThreads, 5) peaks2d_batch_kernel(const uint8_t *plan) {
  const PlanHeader *h = reinterpret_cast<const PlanHeader *>(plan);
  const PlanJob &jb = reinterpret_cast<const PlanJob *>(plan + h->off_job)[blockIdx.x];
  const PlanProblem &pp = reinterpret_cast<const PlanProblem *>(plan + h->off_prob)[jb.prob];
  if (!pp.p.geom.pos) return;
  const int L = pp.npts, d = pp.p.d;
  peaks2d_block(pp.p.P + (size_t)jb.slot * L, pp.p.grid.L, pp.p.geom.Le, pp.p.geom.wrap_az != 0, d,
                pp.p.peak_idx + (size_t)jb.slot * d, pp.p.peak_val + (size_t)jb.slot * d, pp.p.peak_count + jb.slot);
}

// ---- grid slices ---------------------------------------------------------------------------
// Value at global index k of a slice buffer that starts at global index b0.
struct SliceView {
  const float *buf;
  int b0;
  __device__ float operator()(int k) const { return buf[k - b0]; }
};

// 0: not a peak, 1: decided peak, 2: run still equal at `limit` (< L - 1), undecided.
__device__ __forceinline__ int slice_peak_state(const SliceView &P, int i, float v, int limit, int L) {
  if (!(P(i - 1) < v)) return 0;
  int j = i;
  while (j + 1 <= limit && P(j + 1) == v) ++j;
  if (j + 1 <= limit) return P(j + 1) < v ? 1 : 0;
  return limit < L - 1 ? 2 : 0;
}

// Best decided peaks among the thread's points (i = c0, c0 + T, ... < c1) worse than thr.
__device__ bool slice_fill(const SliceView &P, int c0, int c1, int limit, int L, const Cand &thr,
                           Cand (&cache)[kCache], int &n, int *open_idx, float *open_val) {
  n = 0;
  bool more = false;
  for (int i = c0; i < c1; i += kPeakThreads) {
    const float v = P(i);
    const int st = slice_peak_state(P, i, v, limit, L);
    if (st == 2) {
      *open_idx = i;   // the unique run that reaches the end of the slice's data
      *open_val = v;
    }
    if (st != 1) continue;
    cache_insert(Cand{v, i}, thr, cache, n, more);
  }
  return more;
}

__global__ void __launch_bounds__(kPeakThreads) slice_peaks_kernel(const float *Pbuf, int b0, int k0, int k1, int L,
                                                                    int d, doa_slice_summary *out) {
  __shared__ Cand red[kPeakThreads / 32 + 1];
  __shared__ int s_open_idx;
  __shared__ float s_open_val;
  const SliceView P{Pbuf, b0};
  const int limit = min(k1 + 1, L) - 1;              // last readable global index
  const int c0 = max(k0, 1) + threadIdx.x, c1 = min(k1, L - 1);
  if (threadIdx.x == 0) s_open_idx = -1;
  __syncthreads();
  int oi = -1;
  float ov = 0.f;
  Cand cache[kCache];
  int n = 0, head = 0;
  const Cand none{0.f, INT_MAX};
  bool more = slice_fill(P, c0, c1, limit, L, none, cache, n, &oi, &ov);
  if (oi >= 0) {
    s_open_idx = oi;
    s_open_val = ov;
  }
  int nsel = 0;
  for (int r = 0; r < d; ++r) {
    Cand mine = head < n ? cache[head] : none;
    Cand w = block_best(mine, red);
    if (w.i == INT_MAX) break;
    if (threadIdx.x == 0) {
      out->idx[nsel] = w.i;
      out->val[nsel] = w.v;
    }
    ++nsel;
    if (mine.i == w.i) {
      ++head;
      if (head == n && more) {
        int dummy_i;
        float dummy_v;
        more = slice_fill(P, c0, c1, limit, L, w, cache, n, &dummy_i, &dummy_v);
        head = 0;
      }
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    out->count = nsel;
    out->open_idx = s_open_idx;
    out->open_val = s_open_idx >= 0 ? s_open_val : 0.f;
    const float v0 = P(k0);
    int k = k0;
    while (k + 1 <= limit && P(k + 1) == v0) ++k;
    out->first_val = v0;
    out->first_run_to_end = k + 1 > limit ? 1 : 0;
    out->first_next_val = k + 1 <= limit ? P(k + 1) : 0.f;
  }
}

}  // namespace

cudaError_t launch_slice_peaks(const float *Pbuf, int b0, int k0, int k1, int L, int d, doa_slice_summary *out,
                               cudaStream_t s) {
  slice_peaks_kernel<<<1, kPeakThreads, 0, s>>>(Pbuf, b0, k0, k1, L, d, out);
  return cudaGetLastError();
}

cudaError_t launch_peaks_single(const float *P, int L, int d, int *idx, float *val, int *count, cudaStream_t s) {
  peaks_single_kernel<<<1, kPeakThreads, 0, s>>>(P, L, d, idx, val, count);
  return cudaGetLastError();
}

cudaError_t launch_peaks2d_single(const float *P, int La, int Le, int wrap_az, int d, int *idx, float *val,
                                  int *count, cudaStream_t s) {
  peaks2d_single_kernel<<<1, kPeakThreads, 0, s>>>(P, La, Le, wrap_az, d, idx, val, count);
  return cudaGetLastError();
}

cudaError_t launch_peaks_batch(const uint8_t *plan_dev, const PlanHeader &h, uint8_t *ws, bool ula, bool geo,
                               cudaStream_t s) {
  int ngeo = 0;
  for (int b = 0; b < kNumBuckets; ++b) ngeo += h.geo_jobs[b];
  const int repick = ula && !geo;   // the call after the polish
  if (h.njobs > 0 && ula && ngeo < h.nprob) peaks_batch_kernel<<<h.njobs, kPeakThreads, 0, s>>>(plan_dev, ws, repick);
  if (h.njobs > 0 && geo && ngeo > 0) peaks2d_batch_kernel<<<h.njobs, kPeakThreads, 0, s>>>(plan_dev);
  return cudaGetLastError();
}

}  // namespace doa
