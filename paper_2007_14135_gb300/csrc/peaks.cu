// Step-6 (Table 2): findPeaks + PeakSelection(peakVals, inds, D), one CTA per spectrum.
//
// A peak is the left end i of a maximal run [i..j] of equal values with 1 <= i, j <= L-2,
// P[i-1] < P[i] and P[j+1] < P[j]. The D largest peaks are selected (equal values: lower
// index first) and written in ascending index order.
//
// Thread t owns the interior points 1 + t, 1 + t + 256, ... (coalesced loads) and keeps its best
// kCache peaks in registers. Selection runs D rounds of a block-wide arg-max (warp shuffles, then
// one warp over the warp winners); the winning thread pops its head and, if its cache runs dry
// while it still has peaks, rescans its points for the next ones below its last selected peak. This realises the
// shared-memory max-reduction that the paper names as future work for Step-6 (Sec. 6).
#include <climits>

#include "doa_internal.cuh"
#include "peaks_common.cuh"

namespace doa {
namespace {

using namespace pk;

__device__ void peaks_block(const float *__restrict__ P, int L, int d, int *idx, float *val, int *count) {
  __shared__ Cand sel[kMaxM];
  const int nsel = select_top(P, L, d, sel);
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
