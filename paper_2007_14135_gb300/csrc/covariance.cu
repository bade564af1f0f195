// Step-1 (Sec. 3.1, Eq. 3): R = X X^H / N on CUDA cores (FP32 products, FP64 across chunks).
//
// A CTA handles one range of snapshots of one problem. It stages tiles of kTS snapshots of all
// M rows in shared memory (loads coalesced along time); each thread owns a 4 x 4 block of the
// upper triangle of R and a strided subset of each tile's snapshots and accumulates
// x_a conj(x_b) with FP32 FMAs. The per-thread sums are then added across snapshot groups in
// FP32 (a few dozen terms each) and the CTA's partial leaves as FP64.
//
// Batched form: one CTA per work item (problem, chunk of kCovChunk snapshots); multi-chunk
// problems add their chunk partials in chunk order in FP64 (covariance_reduce_batch), so the
// result is deterministic.
// Single-problem form: a thread-block cluster of up to 8 CTAs splits the snapshots; CTA rank 0
// adds the other CTAs' partials through distributed shared memory in rank order.
#include <cooperative_groups.h>

#include "doa_internal.cuh"

namespace cg = cooperative_groups;

namespace doa {
namespace {

constexpr int kCovThreads = 256;
constexpr int kTS = 64;   // snapshots per shared-memory tile
constexpr int kRB = 4;    // register block edge
constexpr int kSmemBytes = 32768;  // max(tile = 64 x 64 float2, group partials = 256 x 32 floats)
constexpr int kMaxCluster = 8;

struct CovLayout {
  int M, MB, nb, groups;
  __device__ CovLayout(int M_) : M(M_) {
    MB = (M + kRB - 1) / kRB;
    nb = MB * (MB + 1) / 2;
    groups = max(1, kCovThreads / nb);
  }
  // block (bi, bj), bi <= bj, of the linear upper-triangle block index b
  __device__ void block_of(int b, int &bi, int &bj) const {
    int i = 0, rem = b;
    while (rem >= MB - i) { rem -= MB - i; ++i; }
    bi = i;
    bj = i + rem;
  }
  __device__ int nout() const { return nb * kRB * kRB; }
};

// Accumulates the snapshots [t0, t1) and leaves the CTA's FP32 sums (nb x 16 complex) at the
// start of `smem`, which it returns.
__device__ float2 *cov_accumulate(const float2 *__restrict__ X, int ldx, int t0, int t1, const CovLayout &lay,
                                  uint8_t *smem) {
  float2 *tile = reinterpret_cast<float2 *>(smem);
  const int tid = threadIdx.x;
  const int blk = tid % lay.nb;
  const int grp = tid / lay.nb;
  const bool active = grp < lay.groups;
  int bi, bj;
  lay.block_of(blk, bi, bj);

  float acc[kRB][kRB][2];
#pragma unroll
  for (int i = 0; i < kRB; ++i)
#pragma unroll
    for (int j = 0; j < kRB; ++j) acc[i][j][0] = acc[i][j][1] = 0.f;

  const int MP = lay.MB * kRB;
  for (int ts = t0; ts < t1; ts += kTS) {
    const int cnt = min(kTS, t1 - ts);
    __syncthreads();
    for (int e = tid; e < MP * kTS; e += kCovThreads) {
      int r = e / kTS, t = e % kTS;
      float2 v = make_float2(0.f, 0.f);
      if (r < lay.M && t < cnt) v = X[(size_t)r * ldx + ts + t];
      tile[r * kTS + t] = v;
    }
    __syncthreads();
    if (active) {
      for (int t = grp; t < cnt; t += lay.groups) {
        float2 xa[kRB], xb[kRB];
#pragma unroll
        for (int i = 0; i < kRB; ++i) {
          xa[i] = tile[(bi * kRB + i) * kTS + t];
          xb[i] = tile[(bj * kRB + i) * kTS + t];
        }
#pragma unroll
        for (int i = 0; i < kRB; ++i)
#pragma unroll
          for (int j = 0; j < kRB; ++j) {
            // x_a * conj(x_b) = (ar br + ai bi) + j (ai br - ar bi)
            acc[i][j][0] = fmaf(xa[i].x, xb[j].x, fmaf(xa[i].y, xb[j].y, acc[i][j][0]));
            acc[i][j][1] = fmaf(xa[i].y, xb[j].x, fmaf(-xa[i].x, xb[j].y, acc[i][j][1]));
          }
      }
    }
  }
  // add across snapshot groups: stage the per-thread sums (tile memory is reused)
  __syncthreads();
  float2 *stage = reinterpret_cast<float2 *>(smem);  // groups x nb x 16
  const int nout = lay.nout();
  if (active) {
#pragma unroll
    for (int i = 0; i < kRB; ++i)
#pragma unroll
      for (int j = 0; j < kRB; ++j)
        stage[(size_t)grp * nout + blk * kRB * kRB + i * kRB + j] = make_float2(acc[i][j][0], acc[i][j][1]);
  }
  __syncthreads();
  // the owner of slot e is the only reader of stage[g * nout + e] for every g, so it may
  // overwrite stage[e] (= out[e]) in place
  for (int e = tid; e < nout; e += kCovThreads) {
    float2 s = make_float2(0.f, 0.f);
    for (int g = 0; g < lay.groups; ++g) {
      float2 v = stage[(size_t)g * nout + e];
      s.x += v.x;
      s.y += v.y;
    }
    stage[e] = s;
  }
  __syncthreads();
  return stage;
}

// Maps output slot e (block-major) to (row, col); returns false outside the upper triangle.
__device__ __forceinline__ bool slot_rc(const CovLayout &lay, int e, int &row, int &col) {
  int b = e / (kRB * kRB), ij = e % (kRB * kRB);
  int bi, bj;
  lay.block_of(b, bi, bj);
  row = bi * kRB + ij / kRB;
  col = bj * kRB + ij % kRB;
  return row < lay.M && col < lay.M && row <= col;
}

__device__ __forceinline__ void store_r(int M, int row, int col, double2 v, double inv_n, float2 *R,
                                        double2 *R64) {
  v.x *= inv_n;
  v.y *= inv_n;
  if (row == col) v.y = 0.0;
  if (R64) {
    R64[row * M + col] = v;
    R64[col * M + row] = make_double2(v.x, -v.y);
  }
  if (R) {
    R[row * M + col] = make_float2((float)v.x, (float)v.y);
    R[col * M + row] = make_float2((float)v.x, (float)-v.y);
  }
}

__global__ void __launch_bounds__(kCovThreads) covariance_cluster_kernel(const float2 *X, int M, int N, int ldx,
                                                                         int per_cta, float2 *R, double2 *R64) {
  __shared__ __align__(16) uint8_t smem[kSmemBytes];
  cg::cluster_group cluster = cg::this_cluster();
  const int rank = (int)cluster.block_rank();
  const int nranks = (int)cluster.num_blocks();
  CovLayout lay(M);
  const int t0 = rank * per_cta;
  const int t1 = min(N, t0 + per_cta);
  float2 *part = cov_accumulate(X, ldx, t0, max(t0, t1), lay, smem);
  cluster.sync();
  if (rank == 0) {
    const double inv_n = 1.0 / (double)N;
    for (int e = threadIdx.x; e < lay.nout(); e += kCovThreads) {
      int row, col;
      if (!slot_rc(lay, e, row, col)) continue;
      double2 s = make_double2(0.0, 0.0);
      for (int r = 0; r < nranks; ++r) {
        const float2 *rp = cluster.map_shared_rank(part, r);
        float2 v = rp[e];
        s.x += (double)v.x;
        s.y += (double)v.y;
      }
      store_r(M, row, col, s, inv_n, R, R64);
    }
  }
  cluster.sync();  // keep every CTA's partial alive until rank 0 has read it
}

// Batch: one CTA per work item (problem, chunk).
__global__ void __launch_bounds__(kCovThreads) covariance_batch_kernel(const uint8_t *plan, uint8_t *ws) {
  __shared__ __align__(16) uint8_t smem[kSmemBytes];
  const PlanHeader *h = reinterpret_cast<const PlanHeader *>(plan);
  const PlanCovItem it = reinterpret_cast<const PlanCovItem *>(plan + h->off_cov)[blockIdx.x];
  const PlanProblem &pp = reinterpret_cast<const PlanProblem *>(plan + h->off_prob)[it.prob];
  const int M = pp.p.M, N = pp.p.N;
  CovLayout lay(M);
  const int t0 = it.chunk * kCovChunk;
  const int t1 = min(N, t0 + kCovChunk);
  const float2 *part = cov_accumulate(reinterpret_cast<const float2 *>(pp.p.X), pp.p.ldx, t0, t1, lay, smem);
  double2 *R64 = reinterpret_cast<double2 *>(ws + pp.r64_off);
  double2 *partial = reinterpret_cast<double2 *>(ws + pp.part_off) + (size_t)it.chunk * M * M;
  const double inv_n = 1.0 / (double)N;
  for (int e = threadIdx.x; e < lay.nout(); e += kCovThreads) {
    int row, col;
    if (!slot_rc(lay, e, row, col)) continue;
    double2 v = make_double2((double)part[e].x, (double)part[e].y);
    if (pp.nchunks == 1)
      store_r(M, row, col, v, inv_n, nullptr, R64);
    else
      partial[row * M + col] = v;
  }
}

// Batch reduce: one CTA per multi-chunk problem, chunk partials added in chunk order.
__global__ void covariance_reduce_batch(const uint8_t *plan, uint8_t *ws) {
  const PlanHeader *h = reinterpret_cast<const PlanHeader *>(plan);
  const int prob = reinterpret_cast<const int32_t *>(plan + h->off_reduce)[blockIdx.x];
  const PlanProblem &pp = reinterpret_cast<const PlanProblem *>(plan + h->off_prob)[prob];
  const int M = pp.p.M;
  const double2 *partials = reinterpret_cast<const double2 *>(ws + pp.part_off);
  double2 *R64 = reinterpret_cast<double2 *>(ws + pp.r64_off);
  const double inv_n = 1.0 / (double)pp.p.N;
  for (int e = threadIdx.x; e < M * M; e += blockDim.x) {
    int row = e / M, col = e % M;
    if (row > col) continue;
    double2 s = make_double2(0.0, 0.0);
    for (int c = 0; c < pp.nchunks; ++c) {
      double2 v = partials[(size_t)c * M * M + row * M + col];
      s.x += v.x;
      s.y += v.y;
    }
    store_r(M, row, col, s, inv_n, nullptr, R64);
  }
}

}  // namespace

cudaError_t launch_covariance_single(const float2 *X, int M, int N, int ldx, float2 *R, double2 *R64,
                                     cudaStream_t s) {
  int chunks = (N + kCovChunk - 1) / kCovChunk;
  int nc = chunks < kMaxCluster ? chunks : kMaxCluster;
  int per = (N + nc - 1) / nc;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(nc);
  cfg.blockDim = dim3(kCovThreads);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = nc;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, covariance_cluster_kernel, X, M, N, ldx, per, R, R64);
}

cudaError_t launch_covariance_batch(const uint8_t *plan_dev, const PlanHeader &h, uint8_t *ws,
                                    cudaStream_t s) {
  if (h.ncov > 0) covariance_batch_kernel<<<h.ncov, kCovThreads, 0, s>>>(plan_dev, ws);
  if (h.nreduce > 0) covariance_reduce_batch<<<h.nreduce, 256, 0, s>>>(plan_dev, ws);
  return cudaGetLastError();
}

}  // namespace doa
