// Step-1 (Sec. 3.1, Eq. 3): R = X X^H / N on CUDA cores.
//
// A CTA handles one range of snapshots of one problem. It stages tiles of kTS snapshots of all
// M rows in shared memory (loads coalesced along time); each thread owns a 4 x 4 block of the
// upper triangle of R and a strided subset of each tile's snapshots.
//
// Two accumulation modes (template kComp):
//  - plain: x_a conj(x_b) accumulated with FP32 FMAs (relative error ~1e-7 of |R|);
//  - compensated: every real product is split exactly into p + e (p = fl(a*b), e = fma(a, b, -p))
//    and added to a double-float accumulator (hi, lo) with TwoSum (Knuth), so the only error is
//    the final rounding of hi + lo (about 2^-44 relative). The block-task kernels (4 < M <= 16)
//    start their accumulators at a power-of-two bias above twice the largest partial sum a lane
//    can reach in its chunk (from the chunk's largest |component|), which makes Dekker's Fast2Sum
//    (3 operations) exact in place of TwoSum (6); the lo word then holds errors of magnitude up to
//    2^-24 of the bias, so a lane's result is exact to ~n^2 2^-48 of the bias (n <= 32 snapshots
//    per lane and chunk), still ~1e-11 of the chunk's largest product sum. The Pisarenko (PHD) spectrum needs it:
//    its minimum eigenvector moves by |dR| / (lambda_{M-2} - lambda_{M-1}), and the noise
//    eigenvalue gaps are tiny, so an FP32-accurate R shifts that spectrum by up to ~1 dB.
// The per-thread sums are added across snapshot groups in double-float and leave as FP64.
//
// Batched form: one CTA per work item (problem, chunk of kCovChunk snapshots); multi-chunk
// problems add their chunk partials in chunk order in FP64 (covariance_reduce_batch), so the
// result is deterministic. Problems that request PHD use the compensated mode.
// Single-problem form: a thread-block cluster of up to 8 CTAs splits the snapshots (always
// compensated); CTA rank 0 adds the other CTAs' partials through distributed shared memory.
#include <cooperative_groups.h>

#include "doa_internal.cuh"

namespace cg = cooperative_groups;

namespace doa {
namespace {

constexpr int kCovThreads = 256;
constexpr int kTS = 64;   // snapshots per shared-memory tile
constexpr int kRB = 4;    // register block edge
// max(tile = 64 x 64 float2, staged group sums = 256 threads x 16 slots x float4)
constexpr int kSmemBytes = 65536;
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

// s + e = a + b exactly (Knuth's TwoSum; no assumption on the magnitudes).
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
  s = __fadd_rn(a, b);
  float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// (h, l) += (h2, l2) in double-float arithmetic, renormalised.
__device__ __forceinline__ void df_add(float &h, float &l, float h2, float l2) {
  float s, e;
  two_sum(h, h2, s, e);
  e = __fadd_rn(e, __fadd_rn(l, l2));
  h = __fadd_rn(s, e);
  l = __fsub_rn(e, __fsub_rn(h, s));
}

// hi + lo += a * b, exactly up to the rounding of lo.
template <bool kComp>
__device__ __forceinline__ void mac(float &hi, float &lo, float a, float b) {
  if (kComp) {
    float p = __fmul_rn(a, b);
    float e = __fmaf_rn(a, b, -p);
    float s, t;
    two_sum(hi, p, s, t);
    hi = s;
    lo = __fadd_rn(lo, __fadd_rn(e, t));
  } else {
    hi = fmaf(a, b, hi);
  }
}

// hi + lo += a * b for an accumulator carrying a bias B (a power of two) with |hi| >= B/2 and
// |a b| <= B/2 throughout: the sum's rounding error is then exact by Fast2Sum (Dekker), three
// operations instead of TwoSum's six; (hi - B) is exact at the end (Sterbenz).
__device__ __forceinline__ void mac_biased(float &hi, float &lo, float a, float b) {
  const float p = __fmul_rn(a, b);
  const float e = __fmaf_rn(a, b, -p);
  const float s = __fadd_rn(hi, p);
  const float t = __fsub_rn(p, __fsub_rn(s, hi));
  hi = s;
  lo = __fadd_rn(lo, __fadd_rn(e, t));
}

// Accumulates the snapshots [t0, t1) and leaves the CTA's sums (nb x 16 slots of float4
// (re_hi, re_lo, im_hi, im_lo)) at the start of `smem`, which it returns.
template <bool kComp>
__device__ float4 *cov_accumulate(const float2 *__restrict__ X, int ldx, int t0, int t1, const CovLayout &lay,
                                  uint8_t *smem) {
  float2 *tile = reinterpret_cast<float2 *>(smem);
  const int tid = threadIdx.x;
  const int blk = tid % lay.nb;
  const int grp = tid / lay.nb;
  const bool active = grp < lay.groups;
  int bi, bj;
  lay.block_of(blk, bi, bj);

  float rh[kRB][kRB], rl[kRB][kRB], ih[kRB][kRB], il[kRB][kRB];
#pragma unroll
  for (int i = 0; i < kRB; ++i)
#pragma unroll
    for (int j = 0; j < kRB; ++j) rh[i][j] = rl[i][j] = ih[i][j] = il[i][j] = 0.f;

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
            mac<kComp>(rh[i][j], rl[i][j], xa[i].x, xb[j].x);
            mac<kComp>(rh[i][j], rl[i][j], xa[i].y, xb[j].y);
            mac<kComp>(ih[i][j], il[i][j], xa[i].y, xb[j].x);
            mac<kComp>(ih[i][j], il[i][j], -xa[i].x, xb[j].y);
          }
      }
    }
  }
  // add across snapshot groups (tile memory is reused for the staged sums)
  __syncthreads();
  float4 *stage = reinterpret_cast<float4 *>(smem);  // groups x nb x 16
  const int nout = lay.nout();
  if (active) {
#pragma unroll
    for (int i = 0; i < kRB; ++i)
#pragma unroll
      for (int j = 0; j < kRB; ++j)
        stage[(size_t)grp * nout + blk * kRB * kRB + i * kRB + j] =
            make_float4(rh[i][j], rl[i][j], ih[i][j], il[i][j]);
  }
  __syncthreads();
  // the owner of slot e is the only reader of stage[g * nout + e] for every g, so it may
  // overwrite stage[e] in place
  for (int e = tid; e < nout; e += kCovThreads) {
    float4 s = stage[e];
    for (int g = 1; g < lay.groups; ++g) {
      float4 v = stage[(size_t)g * nout + e];
      df_add(s.x, s.y, v.x, v.y);
      df_add(s.z, s.w, v.z, v.w);
    }
    stage[e] = s;
  }
  __syncthreads();
  return stage;
}

__device__ __forceinline__ double2 slot_value(const float4 &v) {
  return make_double2((double)v.x + (double)v.y, (double)v.z + (double)v.w);
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
  extern __shared__ __align__(16) uint8_t smem[];
  cg::cluster_group cluster = cg::this_cluster();
  const int rank = (int)cluster.block_rank();
  const int nranks = (int)cluster.num_blocks();
  CovLayout lay(M);
  const int t0 = rank * per_cta;
  const int t1 = min(N, t0 + per_cta);
  float4 *part = cov_accumulate<true>(X, ldx, t0, max(t0, t1), lay, smem);
  cluster.sync();
  if (rank == 0) {
    const double inv_n = 1.0 / (double)N;
    for (int e = threadIdx.x; e < lay.nout(); e += kCovThreads) {
      int row, col;
      if (!slot_rc(lay, e, row, col)) continue;
      double2 s = make_double2(0.0, 0.0);
      for (int r = 0; r < nranks; ++r) {
        const float4 *rp = cluster.map_shared_rank(part, r);
        double2 v = slot_value(rp[e]);
        s.x += v.x;
        s.y += v.y;
      }
      store_r(M, row, col, s, inv_n, R, R64);
    }
  }
  cluster.sync();  // keep every CTA's partial alive until rank 0 has read it
}

// ------------------------------------------------------------------------------------------
// Block-task form for 4 < M <= 16 (MB = ceil(M/4) in {2, 3, 4}). The upper triangle is cut into
// tasks of equal work: every off-diagonal 4x4 block (16 complex entries, 64 real MACs per
// snapshot) and every pair of diagonal blocks (4 real diagonal entries + 6 complex entries each,
// 2 x 32 MACs), so no lane computes a lower-triangle entry or the zero imaginary part of the
// diagonal. A warp owns one task and its lanes take snapshots t = lane, lane + 32, ... of each
// 64-snapshot tile; the next tile streams into a second shared-memory buffer (cp.async) while the
// current one is consumed.
// Every task has 32 real accumulators per lane; at the end the 32 lane partials of each
// accumulator are added in lane order in double-float arithmetic (deterministic).
// ------------------------------------------------------------------------------------------
template <int MB>
struct CovTasks {
  static constexpr int kOff = MB * (MB - 1) / 2;
  static constexpr int kDiag = (MB + 1) / 2;
  static constexpr int kTS = 64;
  static constexpr int kMP = 4 * MB;
};

// One launch per task kind (0: off-diagonal blocks, 1: diagonal-block pairs), so that every SM
// runs a single unrolled instruction stream: the two kinds' bodies together overflow the
// instruction cache when their warps share an SM.
template <int MB, int kKind>
struct CovKind {
  using T = CovTasks<MB>;
  static constexpr int kTasks = kKind == 0 ? T::kOff : T::kDiag;
  static constexpr int kFirst = kKind == 0 ? 0 : T::kOff;       // global index of the kind's first task
  static constexpr int kThreads = 32 * kTasks;
  static constexpr int kMinBlocks = (65536 / 112) / kThreads > 0 ? (65536 / 112) / kThreads : 1;  // <= 112 regs
  static constexpr int kStageBytes = kTasks * 32 * 32 * 8;       // (hi, lo) per lane per accumulator
  static constexpr int kTileBytes = 2 * T::kMP * T::kTS * 8;      // double-buffered tile
  static constexpr int kSmem = kStageBytes > kTileBytes ? kStageBytes : kTileBytes;
};

// Asynchronous 8-byte global -> shared copy; src_bytes = 0 writes zeros (rows >= M, ragged tail).
__device__ __forceinline__ void cp_async8(void *dst, const void *src, int src_bytes) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(d), "l"(src), "r"(src_bytes) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

// Accumulator a (0..31) of task `task` -> (row, col, imaginary?) ; false if outside M.
template <int MB>
__device__ __forceinline__ bool task_slot(int task, int a, int M, int &row, int &col, bool &imag, bool &diag) {
  using T = CovTasks<MB>;
  if (task < T::kOff) {
    int bi = 0, rem = task;
    while (rem >= MB - 1 - bi) { rem -= MB - 1 - bi; ++bi; }
    const int bj = bi + 1 + rem;
    const int e = a >> 1;
    row = bi * 4 + (e >> 2);
    col = bj * 4 + (e & 3);
    imag = a & 1;
    diag = false;
  } else {
    const int b = 2 * (task - T::kOff) + (a >> 4);
    const int s = a & 15;                 // 0..3: diagonal entries; 4..15: (re, im) of the 6 pairs
    if (s < 4) {
      row = col = b * 4 + s;
      imag = false;
      diag = true;
    } else {
      const int pr = (s - 4) >> 1;        // pair index of (i, j), i < j, in row-major order
      constexpr int pi[6] = {0, 0, 0, 1, 1, 2}, pj[6] = {1, 2, 3, 2, 3, 3};
      row = b * 4 + pi[pr];
      col = b * 4 + pj[pr];
      imag = (s - 4) & 1;
      diag = false;
    }
    if (b >= MB) return false;
  }
  return row < M && col < M;
}

// One snapshot's products for a task; compensated accumulators carry the bias of cov_tasks.
template <int MB, bool kComp>
__device__ __forceinline__ void task_mac(float &hi, float &lo, float a, float b) {
  if (kComp)
    mac_biased(hi, lo, a, b);
  else
    hi = fmaf(a, b, hi);
}

template <int MB, bool kComp>
__device__ __forceinline__ void task_macs(int task, const float2 *tile, int t, float (&hi)[32], float (&lo)[32]) {
  using T = CovTasks<MB>;
  if (task < T::kOff) {
    int bi = 0, rem = task;
    while (rem >= MB - 1 - bi) { rem -= MB - 1 - bi; ++bi; }
    const int bj = bi + 1 + rem;
    float2 xa[4], xb[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      xa[i] = tile[(bi * 4 + i) * T::kTS + t];
      xb[i] = tile[(bj * 4 + i) * T::kTS + t];
    }
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int a = 2 * (i * 4 + j);
        // x_a conj(x_b) = (ar br + ai bi) + j (ai br - ar bi)
        task_mac<MB, kComp>(hi[a], lo[a], xa[i].x, xb[j].x);
        task_mac<MB, kComp>(hi[a], lo[a], xa[i].y, xb[j].y);
        task_mac<MB, kComp>(hi[a + 1], lo[a + 1], xa[i].y, xb[j].x);
        task_mac<MB, kComp>(hi[a + 1], lo[a + 1], -xa[i].x, xb[j].y);
      }
  } else {
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int b = 2 * (task - T::kOff) + h;
      if (b >= MB) break;
      float2 x[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) x[i] = tile[(b * 4 + i) * T::kTS + t];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        task_mac<MB, kComp>(hi[16 * h + i], lo[16 * h + i], x[i].x, x[i].x);
        task_mac<MB, kComp>(hi[16 * h + i], lo[16 * h + i], x[i].y, x[i].y);
      }
      int a = 16 * h + 4;
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = i + 1; j < 4; ++j) {
          task_mac<MB, kComp>(hi[a], lo[a], x[i].x, x[j].x);
          task_mac<MB, kComp>(hi[a], lo[a], x[i].y, x[j].y);
          task_mac<MB, kComp>(hi[a + 1], lo[a + 1], x[i].y, x[j].x);
          task_mac<MB, kComp>(hi[a + 1], lo[a + 1], -x[i].x, x[j].y);
          a += 2;
        }
    }
  }
}

template <int MB, int kKind, bool kComp>
__device__ void cov_tasks(const float2 *__restrict__ X, int M, int ldx, int t0, int t1, uint8_t *smem,
                          int nchunks, double inv_n, double2 *R64, double2 *partial) {
  using T = CovTasks<MB>;
  using K = CovKind<MB, kKind>;
  float2 *tiles = reinterpret_cast<float2 *>(smem);   // two tiles of kMP x kTS
  const int tid = threadIdx.x;
  const int warp = tid >> 5, g = tid & 31;
  const int task = K::kFirst + warp;
  // compensated mode: every accumulator starts at the bias B, a power of two with B/2 above both
  // a lane's running sum (at most 2 m^2 per snapshot, m the chunk's largest |component|) and any
  // single product (m^2), so mac_biased's Fast2Sum is exact
  float bias = 0.f;
  if (kComp) {
    __shared__ float red[32];
    float m = 0.f;
    const int cnt = t1 - t0;
    for (int r = 0; r < M; ++r)
      for (int t = tid; t < cnt; t += K::kThreads) {
        const float2 v = X[(size_t)r * ldx + t0 + t];
        m = fmaxf(m, fmaxf(fabsf(v.x), fabsf(v.y)));
      }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, off));
    if (g == 0) red[warp] = m;
    __syncthreads();
    m = 0.f;
    for (int w = 0; w < K::kThreads / 32; ++w) m = fmaxf(m, red[w]);
    const int per_lane = (cnt + 31) / 32;
    const float b = (float)(4 * per_lane + 2) * m * m;
    bias = __int_as_float((__float_as_int(b) & 0x7F800000) + 0x00800000);   // next power of two above b
  }
  float hi[32], lo[32];
#pragma unroll
  for (int a = 0; a < 32; ++a) {
    hi[a] = bias;
    lo[a] = 0.f;
  }
  auto issue = [&](int buf, int ts) {
    const int cnt = min(T::kTS, t1 - ts);
    float2 *dst = tiles + buf * (T::kMP * T::kTS);
    for (int e = tid; e < T::kMP * T::kTS; e += K::kThreads) {
      const int r = e / T::kTS, t = e % T::kTS;
      const bool ok = r < M && t < cnt;
      cp_async8(dst + e, ok ? X + (size_t)r * ldx + ts + t : X, ok ? 8 : 0);
    }
    cp_async_commit();
  };
  if (t0 < t1) issue(0, t0);
  int buf = 0;
  for (int ts = t0; ts < t1; ts += T::kTS, buf ^= 1) {
    const int cnt = min(T::kTS, t1 - ts);
    if (ts + T::kTS < t1) {
      issue(buf ^ 1, ts + T::kTS);
      cp_async_wait<1>();
    } else {
      cp_async_wait<0>();
    }
    __syncthreads();
    const float2 *tile = tiles + buf * (T::kMP * T::kTS);
    for (int t = g; t < cnt; t += 32) task_macs<MB, kComp>(task, tile, t, hi, lo);
    __syncthreads();
  }
  // lane partials -> shared memory, then one thread per (task, accumulator) adds them in order
  __syncthreads();
  float2 *stage = reinterpret_cast<float2 *>(smem);   // [local task][a][lane]
#pragma unroll
  for (int a = 0; a < 32; ++a) stage[((size_t)warp * 32 + a) * 32 + g] = make_float2(__fsub_rn(hi[a], bias), lo[a]);
  __syncthreads();
  for (int item = tid; item < K::kTasks * 32; item += K::kThreads) {
    const int tk = K::kFirst + item / 32, a = item % 32;
    int row, col;
    bool imag, diag;
    if (!task_slot<MB>(tk, a, M, row, col, imag, diag)) continue;
    const float2 *v = stage + (size_t)item * 32;
    float sh = v[0].x, sl = v[0].y;
    for (int q = 1; q < 32; ++q) df_add(sh, sl, v[q].x, v[q].y);
    const double val = (double)sh + (double)sl;
    if (nchunks == 1) {
      const double x = val * inv_n;
      double *up = reinterpret_cast<double *>(R64 + row * M + col), *dn = reinterpret_cast<double *>(R64 + col * M + row);
      if (diag) {
        up[0] = x;
        up[1] = 0.0;
      } else if (imag) {
        up[1] = x;
        dn[1] = -x;
      } else {
        up[0] = x;
        dn[0] = x;
      }
    } else {
      double *pv = reinterpret_cast<double *>(partial + row * M + col);
      if (diag) {
        pv[0] = val;
        pv[1] = 0.0;
      } else {
        pv[imag ? 1 : 0] = val;
      }
    }
  }
}

template <int MB, int kKind>
__global__ void __launch_bounds__(CovKind<MB, kKind>::kThreads, CovKind<MB, kKind>::kMinBlocks) covariance_tasks_kernel(const uint8_t *plan,
                                                                                        uint8_t *ws, int first) {
  extern __shared__ __align__(16) uint8_t smem[];
  const PlanHeader *h = reinterpret_cast<const PlanHeader *>(plan);
  const PlanCovItem it = reinterpret_cast<const PlanCovItem *>(plan + h->off_cov)[first + blockIdx.x];
  const PlanProblem &pp = reinterpret_cast<const PlanProblem *>(plan + h->off_prob)[it.prob];
  const int M = pp.p.M, N = pp.p.N;
  const int t0 = it.chunk * kCovChunk, t1 = min(N, t0 + kCovChunk);
  const float2 *X = reinterpret_cast<const float2 *>(pp.p.X);
  double2 *R64 = reinterpret_cast<double2 *>(ws + pp.r64_off);
  double2 *partial = reinterpret_cast<double2 *>(ws + pp.part_off) + (size_t)it.chunk * M * M;
  const double inv_n = 1.0 / (double)N;
  if (pp.p.alg_mask & (1u << DOA_PHD))
    cov_tasks<MB, kKind, true>(X, M, pp.p.ldx, t0, t1, smem, pp.nchunks, inv_n, R64, partial);
  else
    cov_tasks<MB, kKind, false>(X, M, pp.p.ldx, t0, t1, smem, pp.nchunks, inv_n, R64, partial);
}

// Batch: one CTA per work item (problem, chunk) of the generic class.
__global__ void __launch_bounds__(kCovThreads) covariance_batch_kernel(const uint8_t *plan, uint8_t *ws, int first) {
  extern __shared__ __align__(16) uint8_t smem[];
  const PlanHeader *h = reinterpret_cast<const PlanHeader *>(plan);
  const PlanCovItem it = reinterpret_cast<const PlanCovItem *>(plan + h->off_cov)[first + blockIdx.x];
  const PlanProblem &pp = reinterpret_cast<const PlanProblem *>(plan + h->off_prob)[it.prob];
  const int M = pp.p.M, N = pp.p.N;
  CovLayout lay(M);
  const int t0 = it.chunk * kCovChunk;
  const int t1 = min(N, t0 + kCovChunk);
  const float2 *X = reinterpret_cast<const float2 *>(pp.p.X);
  const float4 *part = (pp.p.alg_mask & (1u << DOA_PHD)) ? cov_accumulate<true>(X, pp.p.ldx, t0, t1, lay, smem)
                                                          : cov_accumulate<false>(X, pp.p.ldx, t0, t1, lay, smem);
  double2 *R64 = reinterpret_cast<double2 *>(ws + pp.r64_off);
  double2 *partial = reinterpret_cast<double2 *>(ws + pp.part_off) + (size_t)it.chunk * M * M;
  const double inv_n = 1.0 / (double)N;
  for (int e = threadIdx.x; e < lay.nout(); e += kCovThreads) {
    int row, col;
    if (!slot_rc(lay, e, row, col)) continue;
    double2 v = slot_value(part[e]);
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

// Batch fixup of the tensor-core covariance (covariance_tc_batch.cu): a listed problem that kernel
// marked (a sample beyond its scaling range, non-finite data, a bounded wait that ran out) is
// recomputed here with the compensated accumulation, one CTA per problem, chunk by chunk, the chunk
// sums added in FP64 in chunk order. Unmarked problems cost one flag read.
constexpr int kFixupSlots = 160;   // output slots of M <= 16 (10 blocks of 4 x 4)

__global__ void __launch_bounds__(kCovThreads) covariance_fixup_kernel(const uint8_t *plan, uint8_t *ws) {
  extern __shared__ __align__(16) uint8_t smem[];
  __shared__ double2 acc[kFixupSlots];
  const PlanHeader *h = reinterpret_cast<const PlanHeader *>(plan);
  const int n0 = h->ncovtc[0], total = n0 + h->ncovtc[1];
  const int32_t *flags = reinterpret_cast<const int32_t *>(ws + h->covtc_flag_off);
  for (int f = blockIdx.x; f < total; f += gridDim.x) {
    if (flags[f] == 0) continue;
    const int prob = f < n0 ? reinterpret_cast<const int32_t *>(plan + h->off_covtc[0])[f]
                            : reinterpret_cast<const int32_t *>(plan + h->off_covtc[1])[f - n0];
    const PlanProblem &pp = reinterpret_cast<const PlanProblem *>(plan + h->off_prob)[prob];
    const int M = pp.p.M, N = pp.p.N;
    const float2 *X = reinterpret_cast<const float2 *>(pp.p.X);
    CovLayout lay(M);
    for (int e = threadIdx.x; e < lay.nout(); e += kCovThreads) acc[e] = make_double2(0.0, 0.0);
    for (int t0 = 0; t0 < N; t0 += kCovChunk) {
      const float4 *part = cov_accumulate<true>(X, pp.p.ldx, t0, min(N, t0 + kCovChunk), lay, smem);
      for (int e = threadIdx.x; e < lay.nout(); e += kCovThreads) {
        const double2 v = slot_value(part[e]);
        acc[e].x += v.x;
        acc[e].y += v.y;
      }
    }
    double2 *R64 = reinterpret_cast<double2 *>(ws + pp.r64_off);
    const double inv_n = 1.0 / (double)N;
    for (int e = threadIdx.x; e < lay.nout(); e += kCovThreads) {
      int row, col;
      if (slot_rc(lay, e, row, col)) store_r(M, row, col, acc[e], inv_n, nullptr, R64);
    }
    __syncthreads();
  }
}

}  // namespace

cudaError_t launch_covariance_fixup(const uint8_t *plan_dev, const PlanHeader &h, uint8_t *ws, cudaStream_t s) {
  const int total = h.ncovtc[0] + h.ncovtc[1];
  if (total == 0) return cudaSuccess;
  static_assert(kCovTcMaxM <= 16, "fixup slots cover M <= 16");
  cudaError_t e = ensure_smem_attr(reinterpret_cast<const void *>(covariance_fixup_kernel), kSmemBytes);
  if (e != cudaSuccess) return e;
  const int grid = total < 2 * device_sm_count() ? total : 2 * device_sm_count();
  covariance_fixup_kernel<<<grid, kCovThreads, kSmemBytes, s>>>(plan_dev, ws);
  return cudaGetLastError();
}

cudaError_t launch_covariance_single(const float2 *X, int M, int N, int ldx, float2 *R, double2 *R64,
                                     cudaStream_t s) {
  cudaError_t e = ensure_smem_attr(reinterpret_cast<const void *>(covariance_cluster_kernel), kSmemBytes);
  if (e != cudaSuccess) return e;
  int chunks = (N + kCovChunk - 1) / kCovChunk;
  int nc = chunks < kMaxCluster ? chunks : kMaxCluster;
  int per = (N + nc - 1) / nc;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(nc);
  cfg.blockDim = dim3(kCovThreads);
  cfg.dynamicSmemBytes = kSmemBytes;
  cfg.stream = s;
  cudaLaunchAttribute attr_[1];
  attr_[0].id = cudaLaunchAttributeClusterDimension;
  attr_[0].val.clusterDim.x = nc;
  attr_[0].val.clusterDim.y = 1;
  attr_[0].val.clusterDim.z = 1;
  cfg.attrs = attr_;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, covariance_cluster_kernel, X, M, N, ldx, per, R, R64);
}

template <int MB, int kKind>
cudaError_t launch_tasks_kind(const uint8_t *plan_dev, int first, int n, uint8_t *ws, cudaStream_t s) {
  using K = CovKind<MB, kKind>;
  cudaError_t e = ensure_smem_attr(reinterpret_cast<const void *>(covariance_tasks_kernel<MB, kKind>), K::kSmem);
  if (e != cudaSuccess) return e;
  covariance_tasks_kernel<MB, kKind><<<n, K::kThreads, K::kSmem, s>>>(plan_dev, ws, first);
  return cudaGetLastError();
}

template <int MB>
cudaError_t launch_tasks(const uint8_t *plan_dev, const PlanHeader &h, uint8_t *ws, cudaStream_t s) {
  const int c = MB - 2, n = h.cov_first[c + 1] - h.cov_first[c];
  if (n == 0) return cudaSuccess;
  cudaError_t e = launch_tasks_kind<MB, 0>(plan_dev, h.cov_first[c], n, ws, s);
  if (e != cudaSuccess) return e;
  return launch_tasks_kind<MB, 1>(plan_dev, h.cov_first[c], n, ws, s);
}

cudaError_t launch_covariance_batch(const uint8_t *plan_dev, const PlanHeader &h, uint8_t *ws,
                                    cudaStream_t s) {
  cudaError_t e = ensure_smem_attr(reinterpret_cast<const void *>(covariance_batch_kernel), kSmemBytes);
  if (e != cudaSuccess) return e;
  if ((e = launch_tasks<2>(plan_dev, h, ws, s)) != cudaSuccess) return e;
  if ((e = launch_tasks<3>(plan_dev, h, ws, s)) != cudaSuccess) return e;
  if ((e = launch_tasks<4>(plan_dev, h, ws, s)) != cudaSuccess) return e;
  const int ngen = h.cov_first[kCovClasses] - h.cov_first[kCovClasses - 1];
  if (ngen > 0)
    covariance_batch_kernel<<<ngen, kCovThreads, kSmemBytes, s>>>(plan_dev, ws, h.cov_first[kCovClasses - 1]);
  if (h.nreduce > 0) covariance_reduce_batch<<<h.nreduce, 256, 0, s>>>(plan_dev, ws);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  // problems with M <= 16: tensor cores, then the recomputation of any it marked
  if ((e = launch_covariance_tc_batch(plan_dev, h, ws, s)) != cudaSuccess) return e;
  return launch_covariance_fixup(plan_dev, h, ws, s);
}

}  // namespace doa

// ------------------------------------------------------------------------------------------
// Covariance that allocates nothing and needs no caller workspace.
//
// Some callers cannot allocate device memory when they call in: a fixed-memory real-time loop
// (cudaMalloc may synchronise the device and take driver locks), a host framework that forbids
// allocation after start-up, or code without an allocator of its own. This entry point keeps
// the per-chunk partial sums of the batched covariance in a library-owned, file-scope device
// array instead of a caller workspace. The paper has no counterpart.
//
// Limits and sharing: the array holds kNoallocScratchBytes (DOA_NOALLOC_SCRATCH_BYTES); a
// problem needs ceil(N / 1024) * M * M * 16 bytes of it and larger ones are rejected with
// DOA_ENOMEM. Every GPU that loads the library keeps the array until the process exits. All
// calls on a device share it, so calls that overlap on that GPU (other streams, other host
// threads) race on its contents; serialise them. Nothing in it has to start at zero: every
// chunk writes every entry it later reads. The first call on each device looks up the array's
// device address (cudaGetSymbolAddress, with that device current) and sets the kernel's shared
// memory limit; make that first call before any stream capture.
// ------------------------------------------------------------------------------------------
#include <mutex>

namespace doa {
namespace {

constexpr size_t kNoallocScratchBytes = DOA_NOALLOC_SCRATCH_BYTES;
constexpr int kNoallocMaxDevices = 64;

static __device__ __align__(256) double2 g_noalloc_scratch[kNoallocScratchBytes / sizeof(double2)];

std::mutex g_noalloc_mutex;
double2 *g_noalloc_ptr[kNoallocMaxDevices] = {};

__global__ void __launch_bounds__(kCovThreads) covariance_noalloc_kernel(const float2 *X, int M, int N, int ldx,
                                                                         double2 *partials, float2 *R, double2 *R64) {
  extern __shared__ __align__(16) uint8_t smem[];
  CovLayout lay(M);
  const int t0 = blockIdx.x * kCovChunk;
  const int t1 = min(N, t0 + kCovChunk);
  const float4 *part = cov_accumulate<true>(X, ldx, t0, t1, lay, smem);
  const double inv_n = 1.0 / (double)N;
  double2 *mine = partials + (size_t)blockIdx.x * M * M;
  for (int e = threadIdx.x; e < lay.nout(); e += kCovThreads) {
    int row, col;
    if (!slot_rc(lay, e, row, col)) continue;
    double2 v = slot_value(part[e]);
    if (gridDim.x == 1)
      store_r(M, row, col, v, inv_n, R, R64);
    else
      mine[row * M + col] = v;
  }
}

__global__ void covariance_noalloc_reduce(const double2 *partials, int nchunks, int M, int N, float2 *R,
                                          double2 *R64) {
  const double inv_n = 1.0 / (double)N;
  for (int e = threadIdx.x; e < M * M; e += blockDim.x) {
    int row = e / M, col = e % M;
    if (row > col) continue;
    double2 s = make_double2(0.0, 0.0);
    for (int c = 0; c < nchunks; ++c) {
      double2 v = partials[(size_t)c * M * M + row * M + col];
      s.x += v.x;
      s.y += v.y;
    }
    store_r(M, row, col, s, inv_n, R, R64);
  }
}

// Device address of the scratch array for the current device (looked up once per device).
cudaError_t noalloc_scratch(double2 **out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kNoallocMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_noalloc_mutex);
  if (!g_noalloc_ptr[dev]) {
    double2 *p = nullptr;
    e = cudaGetSymbolAddress(reinterpret_cast<void **>(&p), g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(covariance_noalloc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemBytes);
    if (e != cudaSuccess) return e;
    g_noalloc_ptr[dev] = p;
  }
  *out = g_noalloc_ptr[dev];
  return cudaSuccess;
}

}  // namespace
}  // namespace doa

extern "C" doa_status doa_covariance_noalloc(const float *X, int M, int N, int ldx, float *R, double *R64,
                                             void *stream) {
  using namespace doa;
  if (!X || M < 2 || M > kMaxM || N < 1 || ldx < N || (!R && !R64)) return DOA_EINVAL;
  if ((reinterpret_cast<uintptr_t>(X) & 7u) || (reinterpret_cast<uintptr_t>(R) & 7u) ||
      (reinterpret_cast<uintptr_t>(R64) & 15u))
    return DOA_EINVAL;
  const int nchunks = (N + kCovChunk - 1) / kCovChunk;
  if ((size_t)nchunks * M * M * sizeof(double2) > kNoallocScratchBytes) return DOA_ENOMEM;
  double2 *scratch = nullptr;
  if (noalloc_scratch(&scratch) != cudaSuccess) return DOA_ECUDA;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  covariance_noalloc_kernel<<<nchunks, kCovThreads, kSmemBytes, s>>>(
      reinterpret_cast<const float2 *>(X), M, N, ldx, scratch, reinterpret_cast<float2 *>(R),
      reinterpret_cast<double2 *>(R64));
  if (nchunks > 1)
    covariance_noalloc_reduce<<<1, 256, 0, s>>>(scratch, nchunks, M, N, reinterpret_cast<float2 *>(R),
                                                reinterpret_cast<double2 *>(R64));
  return cudaGetLastError() == cudaSuccess ? DOA_OK : DOA_ECUDA;
}
