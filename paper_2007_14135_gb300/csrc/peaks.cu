// Step-6 (Table 2): findPeaks + PeakSelection(peakVals, inds, D), one CTA per spectrum.
//
// A peak is the left end i of a maximal run [i..j] of equal values with 1 <= i, j <= L-2,
// P[i-1] < P[i] and P[j+1] < P[j]. The D largest peaks are selected (equal values: lower
// index first) and written in ascending index order.
//
// Each thread owns a contiguous chunk of [1, L-2] and keeps its best kCache peaks in registers.
// Selection runs D rounds of a block-wide arg-max (warp shuffles, then one warp over the warp
// winners); the winning thread pops its head and, if its cache runs dry while it still has
// peaks, rescans its chunk for the next ones below its last selected peak. This realises the
// shared-memory max-reduction that the paper names as future work for Step-6 (Sec. 6).
#include <climits>

#include "doa_internal.cuh"

namespace doa {
namespace {

constexpr int kPeakThreads = 256;
constexpr int kCache = 4;

struct Cand {
  float v;
  int i;  // INT_MAX = none
};

__device__ __forceinline__ bool better(const Cand &a, const Cand &b) {
  if (a.i == INT_MAX) return false;
  if (b.i == INT_MAX) return true;
  return a.v > b.v || (a.v == b.v && a.i < b.i);
}

__device__ __forceinline__ bool is_peak(const float *__restrict__ P, int L, int i, float v) {
  if (!(P[i - 1] < v)) return false;
  int j = i;
  while (j + 1 <= L - 1 && P[j + 1] == v) ++j;
  return j + 1 <= L - 1 && P[j + 1] < v;
}

// Fills cache with the best peaks of [c0, c1) that are worse than thr (thr.i == INT_MAX: any).
// Returns whether more such peaks exist beyond the cache.
__device__ bool fill(const float *__restrict__ P, int L, int c0, int c1, const Cand &thr, Cand (&cache)[kCache],
                     int &n) {
  n = 0;
  bool more = false;
  for (int i = c0; i < c1; ++i) {
    float v = P[i];
    if (!is_peak(P, L, i, v)) continue;
    Cand c{v, i};
    if (thr.i != INT_MAX && !better(thr, c)) continue;
    if (n < kCache) {
      int k = n++;
      while (k > 0 && better(c, cache[k - 1])) {
        cache[k] = cache[k - 1];
        --k;
      }
      cache[k] = c;
    } else if (better(c, cache[kCache - 1])) {
      more = true;
      int k = kCache - 1;
      while (k > 0 && better(c, cache[k - 1])) {
        cache[k] = cache[k - 1];
        --k;
      }
      cache[k] = c;
    } else {
      more = true;
    }
  }
  return more;
}

__device__ Cand block_best(Cand c, Cand *red) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    Cand o;
    o.v = __shfl_down_sync(0xffffffffu, c.v, off);
    o.i = __shfl_down_sync(0xffffffffu, c.i, off);
    if (better(o, c)) c = o;
  }
  if (lane == 0) red[warp] = c;
  __syncthreads();
  if (warp == 0) {
    c = lane < (kPeakThreads / 32) ? red[lane] : Cand{0.f, INT_MAX};
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
      Cand o;
      o.v = __shfl_down_sync(0xffffffffu, c.v, off);
      o.i = __shfl_down_sync(0xffffffffu, c.i, off);
      if (better(o, c)) c = o;
    }
    if (lane == 0) red[kPeakThreads / 32] = c;
  }
  __syncthreads();
  Cand w = red[kPeakThreads / 32];
  __syncthreads();
  return w;
}

__device__ void peaks_block(const float *__restrict__ P, int L, int d, int *idx, float *val, int *count) {
  __shared__ Cand red[kPeakThreads / 32 + 1];
  __shared__ Cand sel[kMaxM];
  const int interior = L - 2;
  const int chunk = (interior + kPeakThreads - 1) / kPeakThreads;
  const int c0 = 1 + threadIdx.x * chunk;
  const int c1 = min(L - 1, c0 + chunk);
  Cand cache[kCache];
  int n = 0, head = 0;
  const Cand none{0.f, INT_MAX};
  bool more = fill(P, L, c0, c1, none, cache, n);
  int nsel = 0;
  for (int r = 0; r < d; ++r) {
    Cand mine = head < n ? cache[head] : none;
    Cand w = block_best(mine, red);
    if (w.i == INT_MAX) break;
    if (threadIdx.x == 0) sel[nsel] = w;
    ++nsel;
    if (mine.i == w.i) {
      ++head;
      if (head == n && more) {
        more = fill(P, L, c0, c1, w, cache, n);
        head = 0;
      }
    }
  }
  __syncthreads();
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

__global__ void __launch_bounds__(kPeakThreads) peaks_single_kernel(const float *P, int L, int d, int *idx, float *val,
                                                                    int *count) {
  peaks_block(P, L, d, idx, val, count);
}

__global__ void __launch_bounds__(kPeakThreads) peaks_batch_kernel(const uint8_t *plan) {
  const PlanHeader *h = reinterpret_cast<const PlanHeader *>(plan);
  const PlanJob &jb = reinterpret_cast<const PlanJob *>(plan + h->off_job)[blockIdx.x];
  const PlanProblem &pp = reinterpret_cast<const PlanProblem *>(plan + h->off_prob)[jb.prob];
  const int L = pp.p.grid.L, d = pp.p.d;
  peaks_block(pp.p.P + (size_t)jb.slot * L, L, d, pp.p.peak_idx + (size_t)jb.slot * d,
              pp.p.peak_val + (size_t)jb.slot * d, pp.p.peak_count + jb.slot);
}

}  // namespace

cudaError_t launch_peaks_single(const float *P, int L, int d, int *idx, float *val, int *count, cudaStream_t s) {
  peaks_single_kernel<<<1, kPeakThreads, 0, s>>>(P, L, d, idx, val, count);
  return cudaGetLastError();
}

cudaError_t launch_peaks_batch(const uint8_t *plan_dev, const PlanHeader &h, cudaStream_t s) {
  if (h.njobs > 0) peaks_batch_kernel<<<h.njobs, kPeakThreads, 0, s>>>(plan_dev);
  return cudaGetLastError();
}

}  // namespace doa
