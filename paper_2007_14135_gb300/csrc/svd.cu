// Step-2 of Table 2 taken as an SVD of the snapshot matrix X itself (the paper computes Step-2 with
// a Jacobi SVD, Sec. 4.2): one-sided Jacobi (Hestenes) on the M rows of X, so R = X X^H / N is
// never formed and the small singular values keep their relative accuracy.
//
// GPU form. The rows are rotated in place in an FP64 copy Y of X (workspace). One sweep of the
// cyclic one-sided Jacobi is taken as: one streaming pass over Y that applies the previous sweep's
// accumulated rotation V (Y <- V^H Y) and, on the rotated rows, forms the Gram matrix G = Y Y^H in
// FP64 (partial sums per CTA, summed in a fixed order); then one CTA runs the sweep's row-cyclic
// rotations on G itself (G <- J^H G J for each pair, the Hermitian Jacobi rotation built from
// alpha = G_pp, beta = G_qq, gamma = G_pq), accumulating them into V and into U. Within a sweep the
// pair entries are therefore the rotated Gram entries rather than entries recomputed from the
// rows, but each sweep starts from a Gram matrix formed afresh from the rows, and the iteration
// stops after the first sweep that rotates nothing: then every off-diagonal entry of the fresh
// Gram matrix meets the threshold, exactly the stopping rule of the row-by-row form, and
// S_k^2 = G_kk. Every pass reads X or Y once and writes Y once; the passes are spread over the
// SMs, N split into 32-snapshot chunks.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>

#include "doa.h"
#include "doa_internal.cuh"

namespace doa {
namespace {

constexpr int kSvdThreads = 256;
constexpr int kSvdT = 32;              // snapshots per chunk
constexpr int kSvdMaxBlocks = 256;     // pass CTAs (partial Gram blocks) at most
constexpr int kSvdMaxE = (kMaxM * (kMaxM + 1) / 2 + kSvdThreads - 1) / kSvdThreads;   // Gram entries per thread

struct SvdState {
  int done;     // set once the outputs are written
  int sweeps;   // sweeps taken
  int pad[2];
};

struct SvdLayout {
  int64_t off_state, off_G, off_V, off_U, off_part, off_Y, bytes;
};

inline int64_t align16(int64_t x) { return (x + 15) / 16 * 16; }

SvdLayout svd_layout(int M, int N) {
  SvdLayout l{};
  const int64_t E = (int64_t)M * (M + 1) / 2;
  l.off_state = 0;
  l.off_G = 64;
  l.off_V = l.off_G + align16((int64_t)M * M * 16);
  l.off_U = l.off_V + align16((int64_t)M * M * 16);
  l.off_part = l.off_U + align16((int64_t)M * M * 16);
  l.off_Y = l.off_part + align16((int64_t)kSvdMaxBlocks * E * 16);
  l.bytes = l.off_Y + align16((int64_t)M * N * 16);
  return l;
}

// Row i and column j of the upper-triangle entry e (row-major over i <= j).
__device__ __forceinline__ void tri_index(int e, int M, int &i, int &j) {
  int r = 0, left = e;
  while (left >= M - r) {
    left -= M - r;
    ++r;
  }
  i = r;
  j = r + left;
}

// One pass: Y <- V^H Y (kFirst: Y <- X promoted to FP64) chunk by chunk, and the CTA's partial
// Gram sums G_ij = sum_t y_i(t) conj(y_j(t)), i <= j, over its chunks.
template <bool kFirst, bool kC128>
__global__ void __launch_bounds__(kSvdThreads, 1) svd_pass_kernel(const void *X, int ldx, int M, int N, uint8_t *ws,
                                                               SvdLayout lay) {
  const SvdState *st = reinterpret_cast<const SvdState *>(ws + lay.off_state);
  if (!kFirst && st->done) return;
  extern __shared__ __align__(16) uint8_t svd_smem[];
  double2 *S0 = reinterpret_cast<double2 *>(svd_smem);   // M x kSvdT source chunk
  double2 *S1 = S0 + M * kSvdT;                            // M x kSvdT rotated chunk
  double2 *Vs = S1 + M * kSvdT;                            // M x M rotation (row-major)
  double2 *Y = reinterpret_cast<double2 *>(ws + lay.off_Y);
  const int tid = threadIdx.x;
  if (!kFirst) {
    const double2 *V = reinterpret_cast<const double2 *>(ws + lay.off_V);
    for (int e = tid; e < M * M; e += kSvdThreads) Vs[e] = V[e];
  }
  const int E = M * (M + 1) / 2;
  int ei[kSvdMaxE], ej[kSvdMaxE];
  double2 acc[kSvdMaxE];
#pragma unroll
  for (int k = 0; k < kSvdMaxE; ++k) {
    const int e = tid + k * kSvdThreads;
    ei[k] = ej[k] = 0;
    if (e < E) tri_index(e, M, ei[k], ej[k]);
    acc[k] = make_double2(0.0, 0.0);
  }
  const int nchunks = (N + kSvdT - 1) / kSvdT;
  for (int c = blockIdx.x; c < nchunks; c += gridDim.x) {
    const int64_t t0 = (int64_t)c * kSvdT;
    const int cnt = (int)(N - t0 < kSvdT ? N - t0 : kSvdT);
    __syncthreads();   // the previous chunk's Gram sums have finished reading S1
    for (int e = tid; e < M * kSvdT; e += kSvdThreads) {
      const int i = e / kSvdT, t = e % kSvdT;
      double2 v = make_double2(0.0, 0.0);
      if (t < cnt) {
        if (kFirst) {
          if (kC128) {
            v = reinterpret_cast<const double2 *>(X)[(int64_t)i * ldx + t0 + t];
          } else {
            const float2 a = reinterpret_cast<const float2 *>(X)[(int64_t)i * ldx + t0 + t];
            v = make_double2((double)a.x, (double)a.y);
          }
        } else {
          v = Y[(int64_t)i * N + t0 + t];
        }
      }
      S0[e] = v;
    }
    __syncthreads();
    for (int e = tid; e < M * kSvdT; e += kSvdThreads) {
      const int i = e / kSvdT, t = e % kSvdT;
      double2 y = S0[e];
      if (!kFirst) {
        // (V^H Y)_i = sum_j conj(V_ji) y_j
        double re = 0.0, im = 0.0;
        for (int jj = 0; jj < M; ++jj) {
          const double2 v = Vs[jj * M + i], x = S0[jj * kSvdT + t];
          re = fma(v.x, x.x, fma(v.y, x.y, re));
          im = fma(v.x, x.y, fma(-v.y, x.x, im));
        }
        y = make_double2(re, im);
      }
      S1[e] = y;
      if (t < cnt) Y[(int64_t)i * N + t0 + t] = y;
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < kSvdMaxE; ++k) {
      if (tid + k * kSvdThreads < E) {
        const double2 *yi = S1 + ei[k] * kSvdT, *yj = S1 + ej[k] * kSvdT;
        double re = acc[k].x, im = acc[k].y;
        for (int t = 0; t < kSvdT; ++t) {
          const double2 a = yi[t], b = yj[t];   // a conj(b)
          re = fma(a.x, b.x, fma(a.y, b.y, re));
          im = fma(a.y, b.x, fma(-a.x, b.y, im));
        }
        acc[k] = make_double2(re, im);
      }
    }
  }
  double2 *part = reinterpret_cast<double2 *>(ws + lay.off_part) + (int64_t)blockIdx.x * E;
#pragma unroll
  for (int k = 0; k < kSvdMaxE; ++k) {
    const int e = tid + k * kSvdThreads;
    if (e < E) part[e] = acc[k];
  }
}

// One CTA: sums the partial Gram matrices (block order), then either finishes (no pair of the
// sweep needs a rotation, or the sweep cap is reached) or runs the sweep's rotations on G,
// accumulating them into V (this sweep, applied to Y by the next pass) and U (all sweeps).
__global__ void __launch_bounds__(kSvdThreads) svd_sweep_kernel(int M, int N, int nblk, double tol, int max_sweeps,
                                                                uint8_t *ws, SvdLayout lay, double *evals,
                                                                double2 *Uout, int *info) {
  SvdState *st = reinterpret_cast<SvdState *>(ws + lay.off_state);
  if (st->done) return;
  extern __shared__ __align__(16) uint8_t svd_smem[];
  double2 *G = reinterpret_cast<double2 *>(svd_smem);   // M x M row-major
  double2 *V = G + M * M;
  double2 *U = V + M * M;
  __shared__ double ev[kMaxM];
  __shared__ int order[kMaxM];
  __shared__ int rotated;
  const int tid = threadIdx.x;
  const int E = M * (M + 1) / 2;
  const double2 *part = reinterpret_cast<const double2 *>(ws + lay.off_part);
  for (int e = tid; e < E; e += kSvdThreads) {
    double re = 0.0, im = 0.0;
    for (int b = 0; b < nblk; ++b) {
      const double2 v = part[(int64_t)b * E + e];
      re += v.x;
      im += v.y;
    }
    int i, j;
    tri_index(e, M, i, j);
    if (i == j) im = 0.0;   // y_i y_i^H is real
    G[i * M + j] = make_double2(re, im);
    G[j * M + i] = make_double2(re, -im);
  }
  const int sweeps = st->sweeps;
  const double2 *Ug = reinterpret_cast<const double2 *>(ws + lay.off_U);
  for (int e = tid; e < M * M; e += kSvdThreads) {
    const int r = e / M, c = e % M;
    V[e] = make_double2(r == c ? 1.0 : 0.0, 0.0);
    U[e] = sweeps == 0 ? V[e] : Ug[e];
  }
  if (tid == 0) rotated = 0;
  __syncthreads();
  // rows whose squared norm is below 1e-30 of the largest (fresh Gram diagonal) are numerically
  // zero (a rank-deficient X leaves them at the rounding level, where |gamma| stays comparable to
  // sqrt(alpha beta)): pairs with one are not rotated
  double maxd = 0.0;
  for (int i = 0; i < M; ++i) maxd = fmax(maxd, G[i * M + i].x);
  const double floor_d = 1e-30 * maxd;
  const bool last = sweeps + 1 >= max_sweeps;
  for (int p = 0; p < M - 1; ++p) {
    for (int q = p + 1; q < M; ++q) {
      // every thread takes the same decision from the same shared entries
      const double alpha = G[p * M + p].x, beta = G[q * M + q].x;
      const double2 gamma = G[p * M + q];
      const double mag = hypot(gamma.x, gamma.y);
      if (mag == 0.0 || mag <= tol * sqrt(alpha * beta) || alpha <= floor_d || beta <= floor_d) continue;
      if (tid == 0) rotated = 1;
      if (last) continue;   // the cap is reached: report, do not rotate
      const double2 ph = make_double2(gamma.x / mag, gamma.y / mag);
      const double tau = (beta - alpha) / (2.0 * mag);
      const double tt = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
      const double c = 1.0 / sqrt(1.0 + tt * tt), s = tt * c;
      const double2 sph = make_double2(s * ph.x, s * ph.y), sphc = cconj(sph);
      // rows p, q of G: G <- J^H G
      if (tid < M) {
        const double2 rp = G[p * M + tid], rq = G[q * M + tid];
        const double2 a = cmul(sph, rq), b = cmul(sphc, rp);
        G[p * M + tid] = make_double2(c * rp.x - a.x, c * rp.y - a.y);
        G[q * M + tid] = make_double2(b.x + c * rq.x, b.y + c * rq.y);
      }
      __syncthreads();
      // columns p, q of G, V and U: X <- X J
      if (tid < 3 * kMaxM && (tid & (kMaxM - 1)) < M) {
        double2 *A = tid < kMaxM ? G : (tid < 2 * kMaxM ? V : U);
        const int r = tid & (kMaxM - 1);
        const double2 xp = A[r * M + p], xq = A[r * M + q];
        const double2 a = cmul(sphc, xq), b = cmul(sph, xp);
        A[r * M + p] = make_double2(c * xp.x - a.x, c * xp.y - a.y);
        A[r * M + q] = make_double2(b.x + c * xq.x, b.y + c * xq.y);
      }
      __syncthreads();
    }
  }
  __syncthreads();
  const int nsw = sweeps + 1;
  if (!rotated || last) {
    // S_k^2 = G_kk (the fresh Gram matrix when nothing rotated); eigenvalues of R = S^2 / N
    // descending, equal values in index order
    if (tid < M) ev[tid] = G[tid * M + tid].x / (double)N;
    __syncthreads();
    if (tid == 0) {
      for (int i = 0; i < M; ++i) order[i] = i;
      for (int i = 1; i < M; ++i) {
        const int cur = order[i];
        int j = i - 1;
        while (j >= 0 && ev[order[j]] < ev[cur]) {
          order[j + 1] = order[j];
          --j;
        }
        order[j + 1] = cur;
      }
    }
    __syncthreads();
    if (tid < M) evals[tid] = ev[order[tid]];
    for (int e = tid; e < M * M; e += kSvdThreads) {
      const int col = e / M, r = e % M;
      Uout[e] = U[r * M + order[col]];   // column-major: column col = singular vector col
    }
    if (tid == 0) {
      *info = rotated ? -(int)DOA_ENOCONV : nsw;
      st->sweeps = nsw;
      st->done = 1;
    }
    return;
  }
  double2 *Vg = reinterpret_cast<double2 *>(ws + lay.off_V);
  double2 *Uw = reinterpret_cast<double2 *>(ws + lay.off_U);
  for (int e = tid; e < M * M; e += kSvdThreads) {
    Vg[e] = V[e];
    Uw[e] = U[e];
  }
  if (tid == 0) st->sweeps = nsw;
}

}  // namespace
}  // namespace doa

using namespace doa;

extern "C" {

size_t doa_svd_data_ws_bytes(int M, int N) {
  if (M < 2 || M > kMaxM || N < 1) return 0;
  return (size_t)svd_layout(M, N).bytes;
}

doa_status doa_svd_data(const void *X, int x_c128, int M, int N, int ldx, double tol, int max_sweeps, double *evals,
                        double *U, int *info, void *ws, size_t ws_bytes, void *stream) {
  if (!X || !evals || !U || !info || !ws || M < 2 || M > kMaxM || N < 1 || ldx < N || (x_c128 != 0 && x_c128 != 1))
    return DOA_EINVAL;
  if (!(tol > 0.0) || !std::isfinite(tol) || max_sweeps < 1 || max_sweeps > 1000) return DOA_EINVAL;
  auto aligned = [](const void *p, size_t a) { return reinterpret_cast<uintptr_t>(p) % a == 0; };
  if (!aligned(X, x_c128 ? 16 : 8) || !aligned(evals, 8) || !aligned(U, 16) || !aligned(info, 4) || !aligned(ws, 16))
    return DOA_EINVAL;
  const SvdLayout lay = svd_layout(M, N);
  if (ws_bytes < (size_t)lay.bytes) return DOA_ENOMEM;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const int nchunks = (N + kSvdT - 1) / kSvdT;
  const int nblk = std::min(std::min(nchunks, kSvdMaxBlocks), device_sm_count());
  const size_t pass_smem = (size_t)(2 * M * kSvdT + M * M) * sizeof(double2);
  const size_t sweep_smem = (size_t)3 * M * M * sizeof(double2);
  const void *kernels[] = {(const void *)svd_pass_kernel<true, false>, (const void *)svd_pass_kernel<true, true>,
                           (const void *)svd_pass_kernel<false, false>};
  for (const void *k : kernels)
    if (ensure_smem_attr(k, (int)pass_smem) != cudaSuccess) return DOA_ECUDA;
  if (ensure_smem_attr((const void *)svd_sweep_kernel, (int)sweep_smem) != cudaSuccess) return DOA_ECUDA;
  uint8_t *w = static_cast<uint8_t *>(ws);
  if (cudaMemsetAsync(w + lay.off_state, 0, sizeof(SvdState), s) != cudaSuccess) return DOA_ECUDA;
  auto *U2 = reinterpret_cast<double2 *>(U);
  for (int sw = 0; sw < max_sweeps; ++sw) {
    if (sw == 0) {
      if (x_c128)
        svd_pass_kernel<true, true><<<nblk, kSvdThreads, pass_smem, s>>>(X, ldx, M, N, w, lay);
      else
        svd_pass_kernel<true, false><<<nblk, kSvdThreads, pass_smem, s>>>(X, ldx, M, N, w, lay);
    } else {
      svd_pass_kernel<false, false><<<nblk, kSvdThreads, pass_smem, s>>>(X, ldx, M, N, w, lay);
    }
    svd_sweep_kernel<<<1, kSvdThreads, sweep_smem, s>>>(M, N, nblk, tol, max_sweeps, w, lay, evals, U2, info);
  }
  return cudaGetLastError() == cudaSuccess ? DOA_OK : DOA_ECUDA;
}

}  // extern "C"
