// Block-wide peak search and top-d selection shared by doa_peaks and the windowed scan.
// A peak is the left end i of a maximal run [i..j] of equal values with 1 <= i, j <= L-2,
// P[i-1] < P[i] and P[j+1] < P[j] (Table 2 Step-6). Each thread owns every kPeakThreads-th aligned
// quad of four points and keeps its best kCache peaks in registers; d rounds of a warp arg-max pick
// each warp's winners (a thread rescanning its quads only when its cache runs dry), and one warp
// merges the warps' lists.
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

// Spectrum points are read as aligned float4 quads: quad q holds P[4q - off .. 4q - off + 3] with
// off = (address of P / 4) mod 4, so each quad inside [0, L) is one 16-byte load; a quad that
// sticks out at either end is read point by point (its points outside [0, L) read as 0: they are
// neither candidates nor neighbours of one). Thread t owns the quads t, t + stride, ...
inline __device__ int quad_off(const float *P) { return (int)((reinterpret_cast<uintptr_t>(P) >> 2) & 3); }

inline __device__ float4 load_quad(const float *__restrict__ P, int n, int i0) {
  if (i0 >= 0 && i0 + 3 < n) return *reinterpret_cast<const float4 *>(P + i0);
  float4 r;
  r.x = (i0 >= 0 && i0 < n) ? P[i0] : 0.f;
  r.y = (i0 + 1 >= 0 && i0 + 1 < n) ? P[i0 + 1] : 0.f;
  r.z = (i0 + 2 >= 0 && i0 + 2 < n) ? P[i0 + 2] : 0.f;
  r.w = (i0 + 3 >= 0 && i0 + 3 < n) ? P[i0 + 3] : 0.f;
  return r;
}

// Inserts c into the thread's sorted cache (best first) if it is worse than thr; sets more when a
// peak worse than thr is left out of the cache.
inline __device__ void cache_insert(const Cand &c, const Cand &thr, Cand (&cache)[kCache], int &n, bool &more) {
  if (thr.i != INT_MAX && !better(thr, c)) return;
  if (n < kCache) {
    int k = n++;
    while (k > 0 && better(c, cache[k - 1])) {
      cache[k] = cache[k - 1];
      --k;
    }
    cache[k] = c;
  } else {
    more = true;
    if (better(c, cache[kCache - 1])) {
      int k = kCache - 1;
      while (k > 0 && better(c, cache[k - 1])) {
        cache[k] = cache[k - 1];
        --k;
      }
      cache[k] = c;
    }
  }
}

// Fills cache with the thread's best peaks (quads t0, t0 + stride, ...) that are worse than thr
// (thr.i == INT_MAX: any). Returns whether more such peaks exist beyond the cache. Four quads are
// in flight per step, each with the point before and the point after it (scalar loads); a point
// whose right neighbour is equal goes through the full plateau walk of is_peak.
inline __device__ bool fill(const float *__restrict__ P, int L, int t0, int stride, const Cand &thr,
                            Cand (&cache)[kCache], int &n) {
  n = 0;
  bool more = false;
  const int off = quad_off(P), nq = (L + off + 3) >> 2;
  auto test = [&](int i0, const float4 &q, float left, float right) {
    const float v[4] = {q.x, q.y, q.z, q.w};
    // candidates: above the point before and not below the point after (NaN: no); most quads of a
    // smooth spectrum have none and cost these four tests and one branch
    bool c[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) c[u] = (u == 0 ? left : v[u - 1]) < v[u] && (u == 3 ? right : v[u + 1]) <= v[u];
    if (!(c[0] || c[1] || c[2] || c[3])) return;
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int i = i0 + u;
      if (!c[u] || i < 1 || i > L - 2) continue;
      // a right neighbour equal to the point: the plateau walk decides
      const bool pk = (u == 3 ? right : v[u + 1]) < v[u] || is_peak(P, L, i, v[u]);
      if (pk) cache_insert(Cand{v[u], i}, thr, cache, n, more);
    }
  };
  constexpr int U = 4;
  int q = t0;
  for (; q + (U - 1) * stride < nq; q += U * stride) {
    float4 v[U];
    float lf[U], rt[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int i0 = 4 * (q + u * stride) - off;
      v[u] = load_quad(P, L, i0);
      lf[u] = i0 >= 1 ? P[i0 - 1] : 0.f;
      rt[u] = i0 + 4 <= L - 1 ? P[i0 + 4] : 0.f;
    }
#pragma unroll
    for (int u = 0; u < U; ++u) test(4 * (q + u * stride) - off, v[u], lf[u], rt[u]);
  }
  for (; q < nq; q += stride) {
    const int i0 = 4 * q - off;
    test(i0, load_quad(P, L, i0), i0 >= 1 ? P[i0 - 1] : 0.f, i0 + 4 <= L - 1 ? P[i0 + 4] : 0.f);
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

// Best candidate of the warp, in every lane.
inline __device__ Cand warp_best(Cand c) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    Cand o;
    o.v = __shfl_xor_sync(0xffffffffu, c.v, off);
    o.i = __shfl_xor_sync(0xffffffffu, c.i, off);
    if (better(o, c)) c = o;
  }
  return c;
}

// Top-d selection over the threads' caches. fill(thr, cache, n) fills a thread's cache with its
// best peaks worse than thr (thr.i == INT_MAX: any) and returns whether more exist. Each warp first
// picks its own d best in d rounds of a warp arg-max (the winning lane pops its head and, when its
// cache runs dry while it still has peaks, rescans for the next ones below the one just taken);
// then warp 0 merges the warps' sorted lists in d rounds (the block's d best are among them).
// Selected peaks go to sel[0..n) (value descending, index ascending); n is returned in every thread.
template <class Fill>
__device__ __forceinline__ int select_rounds(int d, Cand *sel, Fill fill) {
  constexpr int kWarps = kPeakThreads / 32;
  __shared__ Cand wsel[kWarps][kMaxM + 1];
  __shared__ int wcount[kWarps];
  __shared__ int s_nsel;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const Cand none{0.f, INT_MAX};
  Cand cache[kCache];
  int n = 0, head = 0;
  bool more = fill(none, cache, n);
  int nw = 0;
  for (int r = 0; r < d; ++r) {
    const Cand mine = head < n ? cache[head] : none;
    const Cand w = warp_best(mine);
    if (w.i == INT_MAX) break;
    if (lane == 0) wsel[warp][nw] = w;
    ++nw;
    if (mine.i == w.i) {
      ++head;
      if (head == n && more) {
        more = fill(w, cache, n);
        head = 0;
      }
    }
    __syncwarp();
  }
  if (lane == 0) wcount[warp] = nw;
  __syncthreads();
  if (warp == 0) {
    const int cnt = lane < kWarps ? wcount[lane] : 0;
    int pos = 0, nsel = 0;
    for (int r = 0; r < d; ++r) {
      const Cand mine = pos < cnt ? wsel[lane][pos] : none;
      const Cand w = warp_best(mine);
      if (w.i == INT_MAX) break;
      if (lane == 0) sel[nsel] = w;
      ++nsel;
      if (mine.i == w.i) ++pos;
    }
    if (lane == 0) s_nsel = nsel;
  }
  __syncthreads();
  return s_nsel;
}

// Selects the d best peaks of P[0..L) (value descending, index ascending) into sel[0..n),
// n returned (identical in every thread). All threads of the block must call it.
__device__ __forceinline__ int select_top(const float *__restrict__ P, int L, int d, Cand *sel) {
  return select_rounds(d, sel, [&](const Cand &thr, Cand (&cache)[kCache], int &n) {
    return fill(P, L, (int)threadIdx.x, kPeakThreads, thr, cache, n);
  });
}

// ---- 2-D (azimuth x elevation) spectra ---------------------------------------------------------
// A point of an Le x La row-major spectrum is a peak when it is strictly larger than each of its
// neighbours (the up to 8 points at row and column distance <= 1; rows outside the grid are absent,
// columns wrap around when wrap) and it has at least one.

// Best 2-D peaks among the thread's quads of flat points (t0, t0 + stride, ...; as in fill) worse
// than thr. The row and column of a quad's first point advance by the quotient and remainder of
// 4 * stride (no division per point). A point's row neighbours come from its own quad, from the
// points before and after the quad, or (at a row end) from the row's other end; only the points
// that beat both row neighbours look at the rows above and below. With rows of four points or
// more every quad runs the same branch-free test (a row end inside the quad costs two predicated
// loads), so the lanes of a warp stay together until a point beats both row neighbours.
inline __device__ bool fill2d(const float *__restrict__ P, int La, int Le, bool wrap, int t0, int stride,
                              const Cand &thr, Cand (&cache)[kCache], int &n) {
  n = 0;
  bool more = false;
  const int npts = La * Le;
  const int off = quad_off(P), nq = (npts + off + 3) >> 2;
  const int qstep = 4 * stride, sl = qstep / La, sk = qstep - sl * La;
  // row and column of the first point of quad t0 (it may lie before the spectrum: row -1)
  int i0 = 4 * t0 - off;
  int l0 = i0 >= 0 ? i0 / La : -((-i0 + La - 1) / La);
  int k0 = i0 - l0 * La;
  // value at column kk (-1 .. La) of row `row` (kk = -1 or La: wrapped, or absent = -inf)
  auto row_nb = [&](int row, int kk) -> float {
    if (kk < 0 || kk >= La) {
      if (!wrap) return -INFINITY;
      kk = kk < 0 ? kk + La : kk - La;
    }
    return P[(size_t)row * La + kk];
  };
  constexpr int U = 2;
  for (int q = t0; q < nq; q += U * stride) {
    float4 v4[U];
    float lf[U], rt[U];
    int qi[U], ql[U], qk[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      qi[u] = i0;
      ql[u] = l0;
      qk[u] = k0;
      const bool in = q + u * stride < nq;
      v4[u] = in ? load_quad(P, npts, i0) : make_float4(0.f, 0.f, 0.f, 0.f);
      lf[u] = in && i0 >= 1 ? P[i0 - 1] : 0.f;
      rt[u] = in && i0 + 4 <= npts - 1 ? P[i0 + 4] : 0.f;
      i0 += qstep;
      l0 += sl;
      k0 += sk;
      if (k0 >= La) {
        k0 -= La;
        ++l0;
      }
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      if (q + u * stride >= nq) continue;
      const float v[4] = {v4[u].x, v4[u].y, v4[u].z, v4[u].w};
      bool c[4];
      int row[4], col[4];
      if (La >= 4) {
        // at most one row end inside the quad: element eb (if <= 3) starts the next row; the
        // wrapped neighbours of a row's first and last point are two predicated loads
        const int eb = La - qk[u];
        const int e0 = qk[u] == 0 ? 0 : (eb <= 3 ? eb : -1);   // the element at column 0
        const int e1 = eb <= 4 ? eb - 1 : -1;                    // the element at column La - 1
        float wl = -INFINITY, wr = -INFINITY;
        if (wrap && e0 >= 0 && qi[u] + e0 >= 0 && qi[u] + e0 < npts)
          wl = P[(size_t)(ql[u] + (e0 > 0 ? 1 : 0)) * La + (La - 1)];
        if (wrap && e1 >= 0 && qi[u] + e1 >= 0 && qi[u] + e1 < npts) wr = P[(size_t)ql[u] * La];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const int i = qi[u] + e;
          row[e] = ql[u] + (e >= eb ? 1 : 0);
          col[e] = qk[u] + e - (e >= eb ? La : 0);
          const float left = e == e0 ? wl : (e > 0 ? v[e - 1] : lf[u]);
          const float right = e == e1 ? wr : (e < 3 ? v[e + 1] : rt[u]);
          c[e] = i >= 0 && i < npts && left < v[e] && right < v[e];
        }
      } else {
        // rows of fewer than four points: each element's neighbours one by one
        int l = ql[u], k = qk[u];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const int i = qi[u] + e;
          row[e] = l;
          col[e] = k;
          if (++k == La) {
            k = 0;
            ++l;
          }
          c[e] = false;
          if (i < 0 || i >= npts) continue;
          const float left = col[e] > 0 ? (e > 0 ? v[e - 1] : lf[u]) : row_nb(row[e], -1);
          const float right = col[e] < La - 1 ? (e < 3 ? v[e + 1] : rt[u]) : row_nb(row[e], La);
          c[e] = left < v[e] && right < v[e];
        }
      }
      if (!(c[0] || c[1] || c[2] || c[3])) continue;
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        if (!c[e]) continue;
        // the point beats both row neighbours: it is a peak when it also beats its neighbours in
        // the rows above and below (absent rows are skipped) and has a neighbour at all. The
        // checks stop at the first neighbour that is not smaller: in rows that are nearly flat
        // along the azimuth (near the pole) many points beat their row neighbours, and most fail
        // on the first load.
        bool pk = La > 1 || wrap || Le > 1;
        for (int dl = -1; dl <= 1 && pk; dl += 2) {
          const int r = row[e] + dl;
          if (r < 0 || r >= Le) continue;
          pk = P[(size_t)r * La + col[e]] < v[e] && row_nb(r, col[e] - 1) < v[e] && row_nb(r, col[e] + 1) < v[e];
        }
        if (pk) cache_insert(Cand{v[e], qi[u] + e}, thr, cache, n, more);
      }
    }
  }
  return more;
}

__device__ __forceinline__ int select_top2d(const float *__restrict__ P, int La, int Le, bool wrap, int d, Cand *sel) {
  return select_rounds(d, sel, [&](const Cand &thr, Cand (&cache)[kCache], int &n) {
    return fill2d(P, La, Le, wrap, (int)threadIdx.x, kPeakThreads, thr, cache, n);
  });
}

}  // namespace pk
}  // namespace doa
