// Device pieces of the CUDA-core FP32 scan shared by the full-grid, batched and windowed scans.
#pragma once

#include <float.h>

#include "doa_internal.cuh"

namespace doa {
namespace scanc {

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
  int kofs;           // grid index of local point 0 (windowed scans)
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
inline __device__ void refine_point_warp(const RefineCtx &c, int k, float *P, double2 *ph) {
  const int lane = threadIdx.x & 31;
  const double theta = __dadd_rn(c.lo, __dmul_rn((double)(k + c.kofs), c.step));
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
inline __device__ void refine_point_thread(const RefineCtx &c, int k, float *P) {
  const double theta = __dadd_rn(c.lo, __dmul_rn((double)(k + c.kofs), c.step));
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

}  // namespace scanc
}  // namespace doa
