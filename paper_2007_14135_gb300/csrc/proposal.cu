// Learned-proposal pipeline pieces (not in the paper): GPU snapshot synthesis for training data,
// proposal decoding into fine-grid windows, and the windowed fine scan with its peak merge and
// fallback flags.
//
// Snapshot synthesis follows the signal model of Sec. 3.1 (Eq. 1) for the half-wavelength ULA:
// X = A(theta) S + W with unit-power CN(0,1) sources and CN(0, sigma^2) noise. Random numbers come
// from the counter-based Philox4x32-10 generator (Salmon, Moraes, Dror, Shaw, "Parallel random
// numbers: as easy as 1, 2, 3", SC'11: 10 rounds of the two 32x32->64 multiplies by 0xD2511F53 and
// 0xCD9E8D57, Weyl key increments 0x9E3779B9 and 0xBB67AE85), turned into normals by the
// Box-Muller transform. Counter = (snapshot, instance low, instance high, draw), key = seed.
#include <climits>
#include <float.h>

#include "doa_internal.cuh"
#include "peaks_common.cuh"
#include "scan_common.cuh"

namespace doa {
namespace {

using namespace scanc;

struct Philox {
  uint32_t c[4], k[2];
  __device__ __forceinline__ uint4 next() {
    uint32_t x0 = c[0], x1 = c[1], x2 = c[2], x3 = c[3];
    uint32_t k0 = k[0], k1 = k[1];
#pragma unroll
    for (int r = 0; r < 10; ++r) {
      const uint32_t hi0 = __umulhi(0xD2511F53u, x0), lo0 = 0xD2511F53u * x0;
      const uint32_t hi1 = __umulhi(0xCD9E8D57u, x2), lo1 = 0xCD9E8D57u * x2;
      const uint32_t y0 = hi1 ^ x1 ^ k0, y1 = lo1, y2 = hi0 ^ x3 ^ k1, y3 = lo0;
      x0 = y0; x1 = y1; x2 = y2; x3 = y3;
      k0 += 0x9E3779B9u;
      k1 += 0xBB67AE85u;
    }
    ++c[3];
    return make_uint4(x0, x1, x2, x3);
  }
};

// two standard normals from two uniform words (Box-Muller)
__device__ __forceinline__ float2 box_muller(uint32_t a, uint32_t b) {
  const float u1 = ((float)a + 1.0f) * 2.3283064365386963e-10f;   // (0, 1]
  const float u2 = (float)b * 2.3283064365386963e-10f;            // [0, 1)
  const float r = sqrtf(-2.0f * logf(u1));
  float s, c;
  sincospif(2.0f * u2, &s, &c);
  return make_float2(r * c, r * s);
}

constexpr int kSynthMaxD = 16;

__global__ void synth_kernel(int M, int N, const int32_t *d, const float *angles, int dmax, const float *snr_db,
                             uint64_t seed, uint64_t first, float2 *X) {
  __shared__ float2 A[kMaxM][kSynthMaxD];
  const int b = blockIdx.y;
  const int db = min(d[b], kSynthMaxD);
  for (int e = threadIdx.x; e < M * db; e += blockDim.x) {
    const int m = e / db, i = e % db;
    const float s = sinpif(angles[(size_t)b * dmax + i] / 180.0f);
    float sn, cs;
    sincospif((float)m * s, &sn, &cs);
    A[m][i] = make_float2(cs, sn);
  }
  __syncthreads();
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= N) return;
  const float sigma = sqrtf(exp10f(-snr_db[b] / 10.0f)) * 0.70710678118654752f;
  const uint64_t inst = first + (uint64_t)b;
  Philox rng;
  rng.c[0] = (uint32_t)t;
  rng.c[1] = (uint32_t)inst;
  rng.c[2] = (uint32_t)(inst >> 32);
  rng.c[3] = 0u;
  rng.k[0] = (uint32_t)seed;
  rng.k[1] = (uint32_t)(seed >> 32);
  float2 s[kSynthMaxD];
  for (int i = 0; i < db; i += 2) {
    const uint4 r = rng.next();
    const float2 g0 = box_muller(r.x, r.y), g1 = box_muller(r.z, r.w);
    s[i] = make_float2(g0.x * 0.70710678118654752f, g0.y * 0.70710678118654752f);
    if (i + 1 < db) s[i + 1] = make_float2(g1.x * 0.70710678118654752f, g1.y * 0.70710678118654752f);
  }
  float2 *Xb = X + (size_t)b * M * N;
  for (int m = 0; m < M; m += 2) {
    const uint4 r = rng.next();
    const float2 w0 = box_muller(r.x, r.y), w1 = box_muller(r.z, r.w);
    for (int h = 0; h < 2 && m + h < M; ++h) {
      const float2 w = h == 0 ? w0 : w1;
      float xr = w.x * sigma, xi = w.y * sigma;
      for (int i = 0; i < db; ++i) {
        const float2 a = A[m + h][i];
        xr += a.x * s[i].x - a.y * s[i].y;
        xi += a.x * s[i].y + a.y * s[i].x;
      }
      Xb[(size_t)(m + h) * N + t] = make_float2(xr, xi);
    }
  }
}

// One warp per row: the d + extra highest of 181 bins (at most dmax) with 1-bin suppression
// around each pick; window w starts at the fine-grid index of the bin centre minus width/2
// (clamped into the grid).
__global__ void windows_kernel(const float *probs, const int32_t *d, int batch, int dmax, int extra, double lo,
                               double step, int L, int width, double bin_lo, double bin_step, int32_t *win_first) {
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (warp >= batch) return;
  const float *p = probs + (size_t)warp * DOA_MLP_OUT;
  unsigned taken[6] = {0, 0, 0, 0, 0, 0};   // 181 bins -> 6 words
  const int db = min(d[warp] + extra, dmax);
  for (int w = 0; w < dmax; ++w) {
    float best = -FLT_MAX;
    int bi = INT_MAX;
    if (w < db) {
      for (int i = lane; i < DOA_MLP_OUT; i += 32) {
        if ((taken[i >> 5] >> (i & 31)) & 1u) continue;
        const float v = p[i];
        if (v > best || (v == best && i < bi)) {
          best = v;
          bi = i;
        }
      }
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
      const float ov = __shfl_xor_sync(0xffffffffu, best, off);
      const int oi = __shfl_xor_sync(0xffffffffu, bi, off);
      if (ov > best || (ov == best && oi < bi)) {
        best = ov;
        bi = oi;
      }
    }
    int first = -1;
    if (w < db && bi != INT_MAX) {
      for (int j = bi - 1; j <= bi + 1; ++j)
        if (j >= 0 && j < DOA_MLP_OUT) taken[j >> 5] |= 1u << (j & 31);
      const double centre = bin_lo + bin_step * (double)bi;
      const long long c = llrint((centre - lo) / step);
      long long f = c - width / 2;
      if (f > (long long)L - width) f = (long long)L - width;
      if (f < 0) f = 0;
      first = (int)f;
    }
    if (lane == 0) win_first[(size_t)warp * dmax + w] = first;
  }
}

// Windowed scan: block = (row slot, window, tile of 128 x PT points).
template <int MP, int PT>
__global__ void __launch_bounds__(kScanThreads) scan_windows_kernel(const double2 *B, int M, const int32_t *K,
                                                                    const int32_t *rows, int dmax, double lo,
                                                                    double step, int L, const int32_t *win_first,
                                                                    int width, int full, const uint32_t *S,
                                                                    float *Pwin, int tiles) {
  __shared__ __align__(16) float2 Bs[MP * MP];
  __shared__ ScanShared sh;
  const int nw = full ? 1 : dmax;
  const long long bid = blockIdx.x;
  const int tile = (int)(bid % tiles);
  const int w = (int)((bid / tiles) % nw);
  const int slot = (int)(bid / ((long long)tiles * nw));
  const int r = rows ? rows[slot] : slot;
  const int first = full ? 0 : win_first[(size_t)r * dmax + w];
  if (first < 0) return;
  const int len = full ? L : min(width, L - first);
  ScanJob j{};
  j.F = B + (size_t)r * M * M;
  j.P[kRoMusic] = Pwin + ((size_t)slot * nw + w) * (size_t)(full ? L : width);
  j.lo = lo;
  j.step = step;
  j.M = M;
  j.Kf = j.Kn = K[r];
  j.kphd = j.kmn = -1;
  j.kofs = first;
  load_job<MP>(j, Bs, sh);
  __syncthreads();
  set_threshold<MP, true>(Bs, j, sh);
  __syncthreads();
  const int k0 = (tile * kScanThreads + threadIdx.x) * PT;
  scan_points<MP, PT>(Bs, j, S + first, len, k0, sh);
  drain_refinements(j, sh);
}

// Peaks of one row's windows, merged: the d best peaks of each window (the plateau rule of
// doa_peaks applied to the window's points, so window edges are never peaks), duplicates from
// overlapping windows removed, the d largest kept (ties: lower index) in ascending index order.
// fallback = fewer than d peaks, or a window whose maximum lies on its first or last point with a
// value above the weakest selected peak (the spectrum still rises beyond that edge above the
// d-th peak, so a higher peak may lie outside every window).
__global__ void __launch_bounds__(pk::kPeakThreads) window_peaks_kernel(const float *Pwin, const int32_t *rows,
                                                                       const int32_t *d, int dmax, int L,
                                                                       const int32_t *win_first, int width, int full,
                                                                       int32_t *idx, float *val, int32_t *count,
                                                                       int32_t *fallback) {
  __shared__ pk::Cand sel[kMaxM], merged[6 * kMaxM];
  __shared__ float red_v[pk::kPeakThreads / 32];
  __shared__ int red_p[pk::kPeakThreads / 32];
  __shared__ int nmerged, nedge;
  __shared__ float edge_v[8];
  const int slot = blockIdx.x;
  const int r = rows ? rows[slot] : slot;
  const int nw = full ? 1 : dmax;
  const int db = min(d[r], kMaxM - 1);
  if (threadIdx.x == 0) {
    nmerged = 0;
    nedge = 0;
  }
  __syncthreads();
  for (int w = 0; w < nw; ++w) {
    const int first = full ? 0 : win_first[(size_t)r * dmax + w];
    if (first < 0) continue;
    const int len = full ? L : min(width, L - first);
    const float *P = Pwin + ((size_t)slot * nw + w) * (size_t)(full ? L : width);
    const int ns = pk::select_top(P, len, db, sel);
    if (threadIdx.x == 0)
      for (int a = 0; a < ns && nmerged < 6 * kMaxM; ++a) merged[nmerged++] = pk::Cand{sel[a].v, first + sel[a].i};
    if (!full) {
      // window maximum (value, then lowest index): shuffles, then one thread over the warps
      float bv = -FLT_MAX;
      int bp = INT_MAX;
      for (int k = threadIdx.x; k < len; k += pk::kPeakThreads) {
        const float v = P[k];
        if (v > bv || (v == bv && k < bp)) {
          bv = v;
          bp = k;
        }
      }
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) {
        const float ov = __shfl_xor_sync(0xffffffffu, bv, off);
        const int op = __shfl_xor_sync(0xffffffffu, bp, off);
        if (ov > bv || (ov == bv && op < bp)) {
          bv = ov;
          bp = op;
        }
      }
      if ((threadIdx.x & 31) == 0) {
        red_v[threadIdx.x >> 5] = bv;
        red_p[threadIdx.x >> 5] = bp;
      }
      __syncthreads();
      if (threadIdx.x == 0) {
        float mv = -FLT_MAX;
        int mp = INT_MAX;
        for (int q = 0; q < pk::kPeakThreads / 32; ++q)
          if (red_v[q] > mv || (red_v[q] == mv && red_p[q] < mp)) {
            mv = red_v[q];
            mp = red_p[q];
          }
        if (len > 0 && (mp == 0 || mp == len - 1) && nedge < 8) edge_v[nedge++] = mv;
      }
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const int n = nmerged;
    for (int a = 1; a < n; ++a) {   // value descending, index ascending
      const pk::Cand c = merged[a];
      int b = a - 1;
      while (b >= 0 && pk::better(c, merged[b])) {
        merged[b + 1] = merged[b];
        --b;
      }
      merged[b + 1] = c;
    }
    int sel_i[kMaxM];
    float sel_v[kMaxM];
    int ns = 0;
    for (int a = 0; a < n && ns < db; ++a) {
      bool dup = false;
      for (int q = 0; q < ns; ++q) dup = dup || sel_i[q] == merged[a].i;
      if (dup) continue;
      sel_i[ns] = merged[a].i;
      sel_v[ns] = merged[a].v;
      ++ns;
    }
    for (int a = 1; a < ns; ++a) {
      const int ci = sel_i[a];
      const float cv = sel_v[a];
      int b = a - 1;
      while (b >= 0 && sel_i[b] > ci) {
        sel_i[b + 1] = sel_i[b];
        sel_v[b + 1] = sel_v[b];
        --b;
      }
      sel_i[b + 1] = ci;
      sel_v[b + 1] = cv;
    }
    for (int a = 0; a < ns; ++a) {
      idx[(size_t)r * dmax + a] = sel_i[a];
      val[(size_t)r * dmax + a] = sel_v[a];
    }
    count[r] = ns;
    float vmin = FLT_MAX;
    for (int a = 0; a < ns; ++a) vmin = fminf(vmin, sel_v[a]);
    bool edge = false;
    for (int q = 0; q < nedge; ++q) edge = edge || edge_v[q] > vmin;
    if (fallback) fallback[r] = (ns < d[r] || edge) ? 1 : 0;
  }
}

// Judge of the learned proposal against the plain full-grid method (one warp per row): every
// local maximum of the row's coarse full-grid spectrum (interior: strictly above its left
// neighbour, at least its right one; the ends when they are at least their neighbour) marks where
// a fine-grid peak can lie. One that no learned window covers with a margin of jwidth / 2 fine
// points on each side gets a judge window of jwidth points centred on it (at most kJudgeMax per
// row; more marks the row for the full-grid fallback).
constexpr int kJudgeMax = 16;

__global__ void judge_windows_kernel(const float *Pc, int Lc, double clo, double cstep, double flo, double fstep, int Lf,
                                     const int32_t *win_first, int dmax, int width, int jwidth, int batch,
                                     int32_t *judge_first, int32_t *fallback) {
  const int r = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (r >= batch) return;
  const float *p = Pc + (size_t)r * Lc;
  int n = 0;
  bool over = false;
  for (int k0 = 0; k0 < Lc; k0 += 32) {
    const int k = k0 + lane;
    bool cand = false;
    if (k < Lc) {
      const float v = p[k];
      const bool left = k == 0 || v > p[k - 1];
      const bool right = k == Lc - 1 || v >= p[k + 1];
      cand = (k == 0 ? v >= p[min(1, Lc - 1)] : left) && right;
    }
    bool need = false;
    int first = 0;
    if (cand) {
      const double theta = __dadd_rn(clo, __dmul_rn((double)k, cstep));
      const long long c = llrint((theta - flo) / fstep);
      long long f = c - jwidth / 2;
      if (f > (long long)Lf - jwidth) f = (long long)Lf - jwidth;
      if (f < 0) f = 0;
      first = (int)f;
      need = true;
      for (int w = 0; w < dmax && need; ++w) {
        const int a = win_first[(size_t)r * dmax + w];
        if (a >= 0 && a <= first && first + jwidth <= a + width) need = false;
      }
    }
    const unsigned m = __ballot_sync(0xffffffffu, need);
    const int pos = n + __popc(m & ((1u << lane) - 1u));
    if (need) {
      if (pos < kJudgeMax)
        judge_first[(size_t)r * kJudgeMax + pos] = first;
      else
        over = true;
    }
    n += __popc(m);
  }
  for (int w = n + lane; w < kJudgeMax; w += 32) judge_first[(size_t)r * kJudgeMax + w] = -1;
  if (__any_sync(0xffffffffu, over) && lane == 0) fallback[r] = 1;
}

// One CTA per row: the row falls back to the full grid when it has fewer than d selected peaks, or
// when any point of its judge windows reaches its weakest selected peak (a peak of the full-grid
// spectrum at least that high lies outside every learned window).
__global__ void judge_compare_kernel(const float *Pj, const int32_t *judge_first, int jwidth, int Lf, const float *val,
                                     const int32_t *count, const int32_t *d, int dmax, int32_t *fallback) {
  __shared__ float s_w;
  __shared__ int s_hit;
  const int r = blockIdx.x;
  if (threadIdx.x == 0) {
    const int c = count[r];
    float w = FLT_MAX;
    for (int a = 0; a < c && a < dmax; ++a) w = fminf(w, val[(size_t)r * dmax + a]);
    s_w = w;
    s_hit = c < d[r];
  }
  __syncthreads();
  const float W = s_w;
  bool hit = false;
  for (int w = 0; w < kJudgeMax && !s_hit; ++w) {
    const int first = judge_first[(size_t)r * kJudgeMax + w];
    if (first < 0) break;
    const int len = min(jwidth, Lf - first);
    const float *P = Pj + ((size_t)r * kJudgeMax + w) * (size_t)jwidth;
    for (int k = threadIdx.x; k < len; k += blockDim.x) hit = hit || P[k] >= W;
    if (__syncthreads_or(hit) && threadIdx.x == 0) s_hit = 1;
    __syncthreads();
  }
  if (threadIdx.x == 0 && s_hit) fallback[r] = 1;
}

__global__ void phase_table_kernel(double lo, double step, int L, uint32_t *S) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k < L) S[k] = grid_phase_step(lo, step, k);
}

}  // namespace
}  // namespace doa

using namespace doa;

extern "C" doa_status doa_synth_ula(int batch, int M, int N, const int32_t *d, const float *angles_deg, int dmax,
                                    const float *snr_db, uint64_t seed, uint64_t first_instance, float *X,
                                    void *stream) {
  if (batch < 1 || M < 2 || M > kMaxM || N < 1 || dmax < 1 || dmax > kSynthMaxD || !d || !angles_deg || !snr_db || !X)
    return DOA_EINVAL;
  for (int b0 = 0; b0 < batch; b0 += 65535) {   // grid.y holds at most 65535 instances per launch
    const int nb = batch - b0 < 65535 ? batch - b0 : 65535;
    dim3 grid((N + 255) / 256, nb);
    synth_kernel<<<grid, 256, 0, reinterpret_cast<cudaStream_t>(stream)>>>(
        M, N, d + b0, angles_deg + (size_t)b0 * dmax, dmax, snr_db + b0, seed, first_instance + (uint64_t)b0,
        reinterpret_cast<float2 *>(X) + (size_t)b0 * M * N);
  }
  return cudaGetLastError() == cudaSuccess ? DOA_OK : DOA_ECUDA;
}

extern "C" doa_status doa_proposal_windows(const float *probs, const int32_t *d, int batch, int dmax, int extra,
                                           doa_grid fine, int width, int32_t *win_first, void *stream) {
  if (!probs || !d || !win_first || batch < 1 || dmax < 1 || dmax > 8 || extra < 0 || width < 3 || width > fine.L ||
      fine.L < 3 || !(fine.step_deg > 0.0))
    return DOA_EINVAL;
  const int threads = 256, warps = threads / 32;
  windows_kernel<<<(batch + warps - 1) / warps, threads, 0, reinterpret_cast<cudaStream_t>(stream)>>>(
      probs, d, batch, dmax, extra, fine.lo_deg, fine.step_deg, fine.L, width, -90.0, 1.0, win_first);
  return cudaGetLastError() == cudaSuccess ? DOA_OK : DOA_ECUDA;
}

extern "C" doa_status doa_scan_windows(const double *B, int M, const int32_t *K, const int32_t *d, const int32_t *rows,
                                       int nrows, int dmax, doa_grid fine, const int32_t *win_first, int width,
                                       int full, uint32_t *S, float *Pwin, int32_t *idx, float *val, int32_t *count,
                                       int32_t *fallback, void *stream) {
  if (!B || !K || !d || !S || !Pwin || !idx || !val || !count || nrows < 1 || M < 2 || M > 16 || dmax < 1 ||
      dmax > 64 || fine.L < 3 || !(fine.step_deg > 0.0))
    return DOA_EINVAL;
  if (!full && (!win_first || width < 3 || width > fine.L)) return DOA_EINVAL;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  phase_table_kernel<<<(fine.L + 255) / 256, 256, 0, s>>>(fine.lo_deg, fine.step_deg, fine.L, S);
  const int len = full ? fine.L : width;
  const int tp = kScanThreads * 2;
  const int tiles = (len + tp - 1) / tp;
  const long long blocks = (long long)nrows * (full ? 1 : dmax) * tiles;
  if (blocks > INT_MAX) return DOA_EINVAL;
  if (M <= 8)
    scan_windows_kernel<8, 2><<<(unsigned)blocks, kScanThreads, 0, s>>>(
        reinterpret_cast<const double2 *>(B), M, K, rows, dmax, fine.lo_deg, fine.step_deg, fine.L, win_first, width,
        full, S, Pwin, tiles);
  else
    scan_windows_kernel<16, 2><<<(unsigned)blocks, kScanThreads, 0, s>>>(
        reinterpret_cast<const double2 *>(B), M, K, rows, dmax, fine.lo_deg, fine.step_deg, fine.L, win_first, width,
        full, S, Pwin, tiles);
  window_peaks_kernel<<<nrows, pk::kPeakThreads, 0, s>>>(Pwin, rows, d, dmax, fine.L, win_first, width, full, idx, val,
                                                   count, fallback);
  return cudaGetLastError() == cudaSuccess ? DOA_OK : DOA_ECUDA;
}

extern "C" doa_status doa_proposal_judge(const double *B, int M, const int32_t *K, const int32_t *d, int batch,
                                         const float *Pc, doa_grid coarse, doa_grid fine, const int32_t *win_first,
                                         int dmax, int width, const float *val, const int32_t *count, int jwidth,
                                         int32_t *judge_first, uint32_t *S, float *Pjudge, int32_t *fallback,
                                         void *stream) {
  if (!B || !K || !d || !Pc || !win_first || !val || !count || !judge_first || !S || !Pjudge || !fallback ||
      batch < 1 || M < 2 || M > 16 || dmax < 1 || dmax > 64 || coarse.L < 3 || fine.L < 3 ||
      !(coarse.step_deg > 0.0) || !(fine.step_deg > 0.0) || width < 3 || width > fine.L || jwidth < 3 ||
      jwidth > fine.L)
    return DOA_EINVAL;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const int threads = 256, warps = threads / 32;
  judge_windows_kernel<<<(batch + warps - 1) / warps, threads, 0, s>>>(
      Pc, coarse.L, coarse.lo_deg, coarse.step_deg, fine.lo_deg, fine.step_deg, fine.L, win_first, dmax, width,
      jwidth, batch, judge_first, fallback);
  phase_table_kernel<<<(fine.L + 255) / 256, 256, 0, s>>>(fine.lo_deg, fine.step_deg, fine.L, S);
  const int tp = kScanThreads * 2;
  const int tiles = (jwidth + tp - 1) / tp;
  const long long blocks = (long long)batch * kJudgeMax * tiles;
  if (blocks > INT_MAX) return DOA_EINVAL;
  if (M <= 8)
    scan_windows_kernel<8, 2><<<(unsigned)blocks, kScanThreads, 0, s>>>(
        reinterpret_cast<const double2 *>(B), M, K, nullptr, kJudgeMax, fine.lo_deg, fine.step_deg, fine.L,
        judge_first, jwidth, 0, S, Pjudge, tiles);
  else
    scan_windows_kernel<16, 2><<<(unsigned)blocks, kScanThreads, 0, s>>>(
        reinterpret_cast<const double2 *>(B), M, K, nullptr, kJudgeMax, fine.lo_deg, fine.step_deg, fine.L,
        judge_first, jwidth, 0, S, Pjudge, tiles);
  judge_compare_kernel<<<batch, 256, 0, s>>>(Pjudge, judge_first, jwidth, fine.L, val, count, d, dmax, fallback);
  return cudaGetLastError() == cudaSuccess ? DOA_OK : DOA_ECUDA;
}
