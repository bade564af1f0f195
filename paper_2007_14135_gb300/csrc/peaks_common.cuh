// Block-wide peak search and top-d selection shared by doa_peaks and the windowed scan.
// A peak is the left end i of a maximal run [i..j] of equal values with 1 <= i, j <= L-2,
// P[i-1] < P[i] and P[j+1] < P[j] (Table 2 Step-6). Each thread owns a contiguous chunk and keeps
// its best kCache peaks in registers; d rounds of a block arg-max pick the winners, a thread
// rescanning its chunk only when its cache runs dry.
#pragma once

#include <climits>

#include "doa_internal.cuh"

namespace doa {
namespace pk {

constexpr int kPeakThreads = 256;
constexpr int kCache = 4;

struct Cand {
  float v;
  int i;  // INT_MAX = none
};

inline __device__ bool better(const Cand &a, const Cand &b) {
  if (a.i == INT_MAX) return false;
  if (b.i == INT_MAX) return true;
  return a.v > b.v || (a.v == b.v && a.i < b.i);
}

inline __device__ bool is_peak(const float *__restrict__ P, int L, int i, float v) {
  if (!(P[i - 1] < v)) return false;
  int j = i;
  while (j + 1 <= L - 1 && P[j + 1] == v) ++j;
  return j + 1 <= L - 1 && P[j + 1] < v;
}

// Fills cache with the best peaks among i = c0, c0 + stride, ... < c1 that are worse than thr
// (thr.i == INT_MAX: any). Returns whether more such peaks exist beyond the cache. Four points
// are examined per step with all their loads (value and both neighbours) issued first; a point
// whose right neighbour is equal goes through the full plateau walk of is_peak.
inline __device__ bool fill(const float *__restrict__ P, int L, int c0, int c1, int stride, const Cand &thr,
                            Cand (&cache)[kCache], int &n) {
  n = 0;
  bool more = false;
  auto consider = [&](int i, float v) {
    Cand c{v, i};
    if (thr.i != INT_MAX && !better(thr, c)) return;
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
  };
  int i = c0;
  for (; i + 3 * stride < c1; i += 4 * stride) {
    float v[4], pv[4], nv[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      v[u] = P[i + u * stride];
      pv[u] = P[i + u * stride - 1];
      nv[u] = P[i + u * stride + 1];
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      if (!(pv[u] < v[u])) continue;
      const int k = i + u * stride;
      bool pk = nv[u] < v[u];
      if (!pk && nv[u] == v[u]) pk = is_peak(P, L, k, v[u]);
      if (pk) consider(k, v[u]);
    }
  }
  for (; i < c1; i += stride) {
    const float v = P[i];
    if (is_peak(P, L, i, v)) consider(i, v);
  }
  return more;
}

inline __device__ Cand block_best(Cand c, Cand *red) {
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

// d rounds of a block arg-max over the threads' caches. fill(thr, cache, n) fills a thread's cache
// with its best peaks worse than thr (thr.i == INT_MAX: any) and returns whether more exist.
// Selected peaks go to sel[0..n) (value descending, index ascending); n is returned in every thread.
template <class Fill>
__device__ __forceinline__ int select_rounds(int d, Cand *sel, Fill fill) {
  __shared__ Cand red[kPeakThreads / 32 + 1];
  Cand cache[kCache];
  int n = 0, head = 0;
  const Cand none{0.f, INT_MAX};
  bool more = fill(none, cache, n);
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
        more = fill(w, cache, n);
        head = 0;
      }
    }
  }
  __syncthreads();
  return nsel;
}

// Selects the d best peaks of P[0..L) (value descending, index ascending) into sel[0..n),
// n returned (identical in every thread). All threads of the block must call it.
__device__ __forceinline__ int select_top(const float *__restrict__ P, int L, int d, Cand *sel) {
  const int c0 = 1 + threadIdx.x, c1 = L - 1;
  return select_rounds(d, sel, [&](const Cand &thr, Cand (&cache)[kCache], int &n) {
    return fill(P, L, c0, c1, kPeakThreads, thr, cache, n);
  });
}

// ---- 2-D (azimuth x elevation) spectra ---------------------------------------------------------
// A point of an Le x La row-major spectrum is a peak when it is strictly larger than each of its
// neighbours (the up to 8 points at row and column distance <= 1; rows outside the grid are absent,
// columns wrap around when wrap) and it has at least one.

// Best 2-D peaks among the flat points i = c0, c0 + stride, ... < La * Le worse than thr. The row
// and column of i advance by the stride's quotient and remainder (no division per point); four
// points per step load their value and row neighbours first, and only the points that beat both
// row neighbours look at the rows above and below.
inline __device__ bool fill2d(const float *__restrict__ P, int La, int Le, bool wrap, int c0, int stride,
                              const Cand &thr, Cand (&cache)[kCache], int &n) {
  n = 0;
  bool more = false;
  const int npts = La * Le;
  const int sl = stride / La, sk = stride - sl * La;
  int l = c0 / La, k = c0 - l * La;
  auto consider = [&](int i, float v) {
    Cand c{v, i};
    if (thr.i != INT_MAX && !better(thr, c)) return;
    if (n < kCache) {
      int q = n++;
      while (q > 0 && better(c, cache[q - 1])) {
        cache[q] = cache[q - 1];
        --q;
      }
      cache[q] = c;
    } else {
      more = true;
      if (better(c, cache[kCache - 1])) {
        int q = kCache - 1;
        while (q > 0 && better(c, cache[q - 1])) {
          cache[q] = cache[q - 1];
          --q;
        }
        cache[q] = c;
      }
    }
  };
  // value of the row neighbour at column kk of row l (kk = -1 or La: wrapped, or absent = -inf)
  auto row_nb = [&](int row, int kk) -> float {
    if (kk < 0 || kk >= La) {
      if (!wrap) return -INFINITY;
      kk = kk < 0 ? kk + La : kk - La;
    }
    return P[(size_t)row * La + kk];
  };
  auto advance = [&](int &ll, int &kk) {
    ll += sl;
    kk += sk;
    if (kk >= La) {
      kk -= La;
      ++ll;
    }
  };
  int i = c0;
  while (i < npts) {
    float v[4], lv[4], rv[4];
    int li[4], ki[4], ii[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      ii[u] = i;
      li[u] = l;
      ki[u] = k;
      const bool in = i < npts;
      v[u] = in ? P[i] : -INFINITY;
      lv[u] = in ? row_nb(l, k - 1) : 0.f;
      rv[u] = in ? row_nb(l, k + 1) : 0.f;
      i += stride;
      advance(l, k);
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      if (ii[u] >= npts || !(lv[u] < v[u]) || !(rv[u] < v[u])) continue;
      // the row neighbours are smaller (or absent); a point with no neighbour at all is no peak
      bool pk = La > 1 || wrap || Le > 1;
      for (int dl = -1; dl <= 1 && pk; dl += 2) {
        const int row = li[u] + dl;
        if (row < 0 || row >= Le) continue;
        if (!(P[(size_t)row * La + ki[u]] < v[u]) || !(row_nb(row, ki[u] - 1) < v[u]) ||
            !(row_nb(row, ki[u] + 1) < v[u]))
          pk = false;
      }
      if (pk) consider(ii[u], v[u]);
    }
  }
  return more;
}

__device__ __forceinline__ int select_top2d(const float *__restrict__ P, int La, int Le, bool wrap, int d, Cand *sel) {
  const int c0 = threadIdx.x;
  return select_rounds(d, sel, [&](const Cand &thr, Cand (&cache)[kCache], int &n) {
    return fill2d(P, La, Le, wrap, c0, kPeakThreads, thr, cache, n);
  });
}

}  // namespace pk
}  // namespace doa
