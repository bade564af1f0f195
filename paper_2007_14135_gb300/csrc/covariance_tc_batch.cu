// Step-1 of the batch (Sec. 3.1, Eq. 3) on the tensor cores: R = X X^H / N for every problem with
// M <= 16, exact to about 2^-40 of the largest snapshot magnitude squared.
//
// Exact slices. A problem's samples are scaled by one power of two (from the first stage's largest
// |component|, with one bit of headroom) so that |w| <= 64, and each w is cut into six slices
//     w = s_0 + s_1 + ... + s_5 + r,   s_k = n_k 2^(-7k), n_k integer, |n_k| <= 64, |r| <= 2^-36,
// by rounding to the nearest multiple of 2^(-7k) (one FP32 add and subtract of 1.5 * 2^(23-7k)).
// Every slice is exact in BF16, every slice product exact in FP32, and a window of 960 snapshots
// sums fewer than 960 * 64 * 64 < 2^22 units of 2^(-7(i+j)), so the tensor core's FP32 accumulator
// holds the exact integer sum of slice pair (i, j) over the window. The pairs with i + j <= 5 are
// kept (the dropped ones and r are below 2^-40 of the largest product).
//
// Planar GEMM. Slice k of a problem is a block of 2 MP operand rows (Re plane: elements 0..MP-1,
// then the Im plane), K = snapshots. With D = [slices of A] [slices of B]^T, the four real
// products of a block pair give P_ij = X_i X_j^H:
//     Re P_ij = RR + II,   Im P_ij = IR - RI.
// One UMMA per 16 snapshots covers all 12 unordered pairs {i, j}, i + j <= 5:
//     MP = 16: A = [s4 s0 s1 s2] (128 rows), B = [s0 s1 s2 s3 s5] (N = 160);
//     MP = 8 : A = [s0 .. s5, pad] (128 rows), B = [s0 s1 s2] (N = 48).
// The operand rows are stored once per stage so that A and B are overlapping windows of them.
//
// Combination. Each readout thread owns one A row (slice i, plane p, element a) and adds its
// designated blocks (each unordered pair once, the diagonal pair with weight 1, the others with
// weight 2) to 64-bit integer sums U'(a, b) in units of 2^-28 (level-5 pairs rounded to that
// unit), so the chunk sums combine exactly and in any order; at the end of the problem
//     R = (U' + U'^H) / 2 * 2^-28 * u0^2 / N   (u0 the scaling unit),
// written to the workspace as FP64 (full Hermitian matrix, zero imaginary diagonal).
//
// Roles (one persistent CTA per SM, static round-robin over the problems, longest first):
//   warps 0-7  producers, four groups of two warps: group q slices the operand stages g = q (mod 4)
//              (64 snapshots each) into a five-deep operand ring (128B-swizzled, K-major), so four
//              stages are sliced at once; the group that slices a problem's first stage also fixes
//              its scaling unit and hands it to the others;
//   warps 8-11 TMEM readout (warp w reads lanes 32 (w % 4) ..), int64 sums, per-problem finalize;
//   warp 13    one thread: TMA bulk copies (cp.async.bulk) of 256 snapshots of each of the M rows
//              per staging stage (one copy per row: the copy engine's cost is per request, so few
//              large requests keep enough bytes in flight), rows 2064 bytes apart so that the
//              producers' 16-byte loads hit distinct banks; each staging stage feeds four operand
//              stages;
//   warp 12    one thread: the MMAs, one accumulation window (15 stages) per TMEM buffer (two
//              buffers), committed to the operand ring and to the buffer's mbarrier.
// A sample beyond the scaling unit's range (or a non-finite one) marks the problem; a problem that
// times out in a bounded wait marks every problem of its CTA. Marked problems are recomputed by the
// compensated CUDA-core kernel (covariance_fixup) launched right after this one.
#include <limits.h>

#include "doa_internal.cuh"
#include "tc_common.cuh"

namespace doa {
namespace {

using namespace tc;

constexpr int kCbSnap = 64;          // snapshots per operand stage (64 BF16 = one 128-byte operand row)
constexpr int kCbStgSnap = 256;      // snapshots per staging stage (one bulk copy of 2 KB per row)
constexpr int kCbSub = kCbStgSnap / kCbSnap;
constexpr int kCbStg = 3;            // staging ring depth (99 KB of reads in flight per SM at M = 16)
constexpr int kCbOps = 5;            // operand ring depth (four stages being sliced, one waiting)
constexpr int kCbWin = 15;           // operand stages per exact accumulation window (960 snapshots)
constexpr int kCbRowPitch = 2064;    // staging bytes per element row (2048 + 16)
// Warp w issues from SM sub-partition w % 4. The readout warps take one per sub-partition (warp
// w reads TMEM lanes 32 (w % 4) ..); the MMA issuer shares sub-partition 0 with the readout of
// slice 4 (two blocks), away from the readout of slice 0 (five blocks, sub-partition 1).
constexpr int kCbProdWarps = 8;     // producer warps 0-7
constexpr int kCbGroups = 4;        // producer groups of two warps; group q slices the stages g = q (mod 4)
constexpr int kCbGroupWarps = kCbProdWarps / kCbGroups;
constexpr int kCbTasks = 256 / (32 * kCbGroupWarps);   // tasks per producer thread and stage
constexpr int kCbReadWarp0 = 8;     // readout warps 8-11
constexpr int kCbMmaWarp = 12, kCbTmaWarp = 13;
constexpr int kCbThreads = 32 * 14;
constexpr int kCbRing = 8;           // scaling-unit ring (producers -> readout)
constexpr int kCbAccCols = 256;      // TMEM columns per accumulator buffer

// Slicing constants 1.5 * 2^(23 - 7k): adding and subtracting one rounds to a multiple of 2^(-7k).
__device__ __forceinline__ float slice_magic(int k) {
  return __uint_as_float((uint32_t)(127 + 23 - 7 * k) << 23) * 1.5f;
}

// Paired FP32 arithmetic (two IEEE round-to-nearest operations per instruction), on the values of
// two consecutive snapshots held as one 64-bit register pair.
// max(|a|, |b|), NaN when either is NaN (so a NaN sample cannot hide behind a finite maximum).
__device__ __forceinline__ float max_abs_nan(float a, float b) {
  float d;
  asm("max.NaN.f32 %0, %1, %2;" : "=f"(d) : "f"(fabsf(a)), "f"(fabsf(b)));
  return d;
}

__device__ __forceinline__ uint64_t pack2(float lo, float hi) {
  return (uint64_t)__float_as_uint(lo) | ((uint64_t)__float_as_uint(hi) << 32);
}
__device__ __forceinline__ float lo2(uint64_t v) { return __uint_as_float((uint32_t)v); }
__device__ __forceinline__ float hi2(uint64_t v) { return __uint_as_float((uint32_t)(v >> 32)); }
__device__ __forceinline__ uint64_t add2(uint64_t a, uint64_t b) {
  uint64_t d;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ uint64_t sub2(uint64_t a, uint64_t b) {
  uint64_t d;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ uint64_t mul2(uint64_t a, uint64_t b) {
  uint64_t d;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}

template <int MP>
struct CbShape;

template <>
struct CbShape<16> {
  static constexpr int kRows = 192;                  // storage rows: s4 s0 s1 s2 s3 s5 (32 each)
  static constexpr int kBlock = 32;
  static constexpr int kBStart = 32;                 // B starts at storage row 32 (s0)
  static constexpr int kN = 160;
  static constexpr int kSN = 4;                      // snapshots per producer task
  __host__ __device__ static constexpr int block_of(int k) { return k == 4 ? 0 : (k == 5 ? 5 : k + 1); }
  __host__ __device__ static constexpr int a_slice(int blk) { return blk == 0 ? 4 : blk - 1; }   // A row block
  __host__ __device__ static constexpr int b_slice(int cb) { return cb == 4 ? 5 : cb; }          // B col block
  static constexpr int kBBlocks = 5;
  // each unordered pair {i, j}, i + j <= 5, once: (i, j) with i <= j, and (4, 0), (4, 1)
  __host__ __device__ static constexpr bool designated(int i, int j) {
    return i + j <= 5 && (i <= j || i == 4);
  }
};

template <>
struct CbShape<8> {
  static constexpr int kRows = 128;                  // s0 .. s5 (16 each) then 32 rows of zeros
  static constexpr int kBlock = 16;
  static constexpr int kBStart = 0;
  static constexpr int kN = 48;
  static constexpr int kSN = 2;
  __host__ __device__ static constexpr int block_of(int k) { return k; }
  __host__ __device__ static constexpr int a_slice(int blk) { return blk; }                      // 6, 7: padding
  __host__ __device__ static constexpr int b_slice(int cb) { return cb; }
  static constexpr int kBBlocks = 3;
  __host__ __device__ static constexpr bool designated(int i, int j) { return i <= 5 && i + j <= 5 && i >= j; }
};

template <int MP>
struct CbLayout {
  using S = CbShape<MP>;
  static constexpr int kStgBytes = MP * kCbRowPitch;   // one staging stage (a multiple of 128 bytes)
  static constexpr int kOpBytes = S::kRows * 128;
  static constexpr int kOffOp = 0;                                        // 1024-aligned stages
  static constexpr int kOffStg = kOffOp + kCbOps * kOpBytes;
  static constexpr int kOffU = kOffStg + kCbStg * ((kStgBytes + 127) / 128 * 128);
  static constexpr int kUBytes = MP * MP * 16;                           // int64 (re, im)
  // at least 116 KB, so that no two CTAs share an SM (each allocates all 512 TMEM columns)
  static constexpr int kSmem = (kOffU + kUBytes + 1024) > 118784 ? (kOffU + kUBytes + 1024) : 118784;
};

struct CbShared {
  uint64_t full[kCbStg], empty[kCbStg], opfull[kCbOps], opempty[kCbOps], accfull[2], accempty[2];
  uint64_t efull[kCbRing], eempty[kCbRing], fin;
  uint64_t pred[kCbGroups][2];  // a group's first-stage maximum exchange (count 2 warps)
  uint64_t sfull[kCbRing];     // scaling unit of ring slot fixed (producers -> the other groups)
  uint64_t rb[2];             // readout warps' finalize steps (count 4 warps)
  uint32_t tmem;
  int abort;
  int eexp[kCbRing];          // scaling exponent k of the problem in ring slot (or INT_MIN: marked)
  float escale[kCbRing];      // scaling factor 2^(5 - k) of the problem in ring slot (0: marked)
  float red[kCbGroups][2][kCbGroupWarps];   // a group's first-stage maxima (double-buffered)
};

__device__ __forceinline__ void bulk_copy(uint32_t dst, const void *src, uint32_t bytes, uint32_t mbar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
               "l"(src), "r"(bytes), "r"(mbar)
               : "memory");
}
__device__ __forceinline__ void arrive_tx(uint32_t mbar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(mbar), "r"(bytes) : "memory");
}
__device__ __forceinline__ void arrive(uint32_t mbar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(mbar) : "memory");
}
__device__ __forceinline__ void arrive_cnt(uint32_t mbar, uint32_t cnt) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0], %1;" ::"r"(mbar), "r"(cnt) : "memory");
}
__device__ __forceinline__ void commit(uint32_t mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar) : "memory");
}

// Bounded wait that also gives up as soon as another role has given up. The waiting thread is
// suspended for up to kCbSuspendNs per try (it resumes as soon as the phase completes), so a
// role that waits most of the time (the MMA issuer, the readout, the copies) takes few issue
// slots from the producers; at most kCbWaitTries tries (about a second).
constexpr uint32_t kCbSuspendNs = 10000;
constexpr int kCbWaitTries = 1 << 17;
__device__ __forceinline__ bool cb_wait(uint32_t mbar, uint32_t parity, volatile int *abort) {
  uint32_t done = 0;
  for (int it = 0; it < kCbWaitTries && !done; ++it) {
    asm volatile(
        "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\nselp.b32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(mbar), "r"(parity), "r"(kCbSuspendNs)
        : "memory");
    if (!done && (it & 15) == 15 && *abort) break;
  }
  if (!done) *abort = 1;
  return done != 0;
}

// Wait of a whole warp: every lane waits (bounded) and the outcome is made warp-uniform, so a lane
// that gave up never diverges from the others into a warp-collective instruction.
// Lane 0 polls; once the phase has completed every lane tests it once (non-blocking) for its own
// acquire of the data the phase guards. The phase cannot move on meanwhile: its next completion
// needs an arrival from this warp.
__device__ __forceinline__ bool warp_wait(uint32_t mbar, uint32_t parity, volatile int *abort) {
  int ok = 1;
  if ((threadIdx.x & 31) == 0) ok = cb_wait(mbar, parity, abort) ? 1 : 0;
  ok = __shfl_sync(0xffffffffu, ok, 0);
  if (!ok) return false;
  uint32_t done = 0;
  asm volatile(
      "{\n.reg .pred p;\nmbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.b32 %0, 1, 0, p;\n}\n"
      : "=r"(done)
      : "r"(mbar), "r"(parity)
      : "memory");
  return __all_sync(0xffffffffu, done != 0);
}

// Warp-granular barrier on an mbarrier with one arrival per participating warp, bounded like every wait.
__device__ __forceinline__ bool warp_bar(uint64_t *bar, uint32_t parity, volatile int *abort) {
  __syncwarp();
  if ((threadIdx.x & 31) == 0) arrive(smem_u32(bar));
  return warp_wait(smem_u32(bar), parity, abort);
}

template <int N>
__device__ __forceinline__ void tmem_ld(uint32_t addr, uint32_t (&r)[N]);
template <>
__device__ __forceinline__ void tmem_ld<16>(uint32_t addr, uint32_t (&r)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(addr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}
template <>
__device__ __forceinline__ void tmem_ld<32>(uint32_t addr, uint32_t (&r)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,%18,%19,"
      "%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];\n"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]),
        "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
        "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(addr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// One designated block (i, j) of this thread's accumulator row, columns [MP Re | MP Im] of the
// B slice: each value is n 2^(-7L), L = i + j, |n| < 2^22, so adding 1.5 * 2^23 to n leaves it in
// the low mantissa bits; it enters U' in units of 2^-28 of w^2, doubled for an off-diagonal pair
// (shift 28 - 7L + off; level 5 is rounded to that unit). mul = 2^(7L), or 0 for a lane that does
// not need the block (its n is then 0). Re row: Re += RR, Im -= RI; Im row: Re += II, Im += IR.
template <int MP>
__device__ __forceinline__ void add_block(const uint32_t (&v)[2 * MP], float mul, int sh, bool im_row,
                                          long long (&ure)[MP], long long (&uim)[MP]) {
  const int rsh = sh < 0 ? -sh : 0, lsh = sh > 0 ? sh : 0;
  const int half = rsh > 0 ? 1 << (rsh - 1) : 0;
#pragma unroll
  for (int b = 0; b < MP; ++b) {
    const int nr = (int)(__float_as_uint(__fmaf_rn(__uint_as_float(v[b]), mul, 12582912.0f)) - 0x4B400000u);
    const int ni = (int)(__float_as_uint(__fmaf_rn(__uint_as_float(v[MP + b]), mul, 12582912.0f)) - 0x4B400000u);
    const long long xr = (long long)((nr + half) >> rsh) << lsh;   // (row plane) x Re b
    const long long xi = (long long)((ni + half) >> rsh) << lsh;   // (row plane) x Im b
    ure[b] += im_row ? xi : xr;
    uim[b] += im_row ? xr : -xi;
  }
}

// Adds one window of this thread's accumulator row to U'. The thread's A slice i comes from its
// TMEM lane; the B slices are walked at run time (one copy of the unrolled block code) and loaded
// with one warp-collective tcgen05.ld when any lane of the warp needs the block.
template <int MP>
__device__ __forceinline__ void read_window(uint32_t taddr, int quarter, int lane, long long (&ure)[MP],
                                            long long (&uim)[MP]) {
  using S = CbShape<MP>;
  const int blk = (32 * quarter + lane) / S::kBlock;        // A row block of this lane
  const int i = S::a_slice(blk);                            // MP = 8: blocks 6, 7 are padding (i > 5)
  const bool im_row = (lane % S::kBlock) >= MP;
  for (int cb = 0; cb < CbShape<MP>::kBBlocks; ++cb) {
    const int j = S::b_slice(cb);
    const bool need = i <= 5 && S::designated(i, j);
    if (!__any_sync(0xffffffffu, need)) continue;
    uint32_t v[2 * MP];
    tmem_ld<2 * MP>(taddr + (uint32_t)(cb * S::kBlock), v);
    const int L = need ? i + j : 0;   // a lane without the block adds n = 0
    const float mul = need ? __uint_as_float((uint32_t)(127 + 7 * L) << 23) : 0.f;
    add_block<MP>(v, mul, 28 - 7 * L + (need && i != j ? 1 : 0), im_row, ure, uim);
  }
}

template <int MP>
__global__ void __launch_bounds__(kCbThreads, 1) covariance_tc_batch_kernel(const uint8_t *plan, uint8_t *ws, int cls) {
  using S = CbShape<MP>;
  using Lay = CbLayout<MP>;
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  uint8_t *sm = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  __shared__ CbShared sh;
  const PlanHeader *h = reinterpret_cast<const PlanHeader *>(plan);
  const PlanProblem *probs = reinterpret_cast<const PlanProblem *>(plan + h->off_prob);
  const int32_t *list = reinterpret_cast<const int32_t *>(plan + h->off_covtc[cls]);
  const int count = h->ncovtc[cls];
  int32_t *flags = reinterpret_cast<int32_t *>(ws + h->covtc_flag_off) + (cls == 0 ? 0 : h->ncovtc[0]);
  long long *U = reinterpret_cast<long long *>(sm + Lay::kOffU);   // [MP][MP][re, im]
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  volatile int *abort = &sh.abort;

  // zero the operand ring (MP = 8: its padding rows are read by the MMAs) and U
  for (int e = tid * 16; e < Lay::kOffStg; e += kCbThreads * 16) *reinterpret_cast<uint4 *>(sm + e) = make_uint4(0, 0, 0, 0);
  for (int e = tid; e < MP * MP * 2; e += kCbThreads) U[e] = 0;
  if (tid == 0) {
    auto init = [](uint64_t *b, int n, int cnt) {
      for (int i = 0; i < n; ++i) asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(b + i)), "r"(cnt));
    };
    init(sh.full, kCbStg, 1);
    init(sh.empty, kCbStg, kCbProdWarps);
    init(sh.opfull, kCbOps, kCbGroupWarps);
    init(sh.opempty, kCbOps, 1);
    init(sh.accfull, 2, 1);
    init(sh.accempty, 2, 4);
    init(sh.efull, kCbRing, 1);
    init(sh.eempty, kCbRing, 4);
    init(&sh.fin, 1, 1);
    for (int q = 0; q < kCbGroups; ++q) init(sh.pred[q], 2, kCbGroupWarps);
    init(sh.sfull, kCbRing, 1);
    init(sh.rb, 2, 4);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    sh.abort = 0;
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&sh.tmem)), "r"(512));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = sh.tmem;

  if (warp < kCbProdWarps) {
    // ---------------------------------------------------------------- producers
    // Four groups of two warps: group q slices the operand stages g = q (mod 4) of the CTA's stage
    // sequence, so four stages are sliced at once and a group has four stages' time for one. A
    // thread takes kCbTasks of the stage's 256 tasks (MP rows x (64 / SN) chunks of SN
    // snapshots); its task j is virtual thread vt = lt + 64 j of a 256-thread layout in which a
    // quarter-warp takes 8 consecutive rows of one chunk (its 16-byte staging loads then fall on
    // distinct banks, the rows being 2064 bytes apart) and the two quarter-warps of a half-warp
    // take two neighbouring chunks (its 8-byte operand stores fill both halves of each swizzled
    // 16-byte slot); every warp instruction covers one such virtual warp.
    constexpr int SN = S::kSN;
    const int grp = warp / kCbGroupWarps, lt = tid % (32 * kCbGroupWarps);
    int mt[kCbTasks], ct[kCbTasks];   // the tasks' row and chunk
    uint32_t so[kCbTasks];            // swizzled byte offset of the task's Re row in slice block 0
#pragma unroll
    for (int j = 0; j < kCbTasks; ++j) {
      const int vt = lt + 32 * kCbGroupWarps * j, qw = vt >> 3, r8 = vt & 7;
      mt[j] = MP == 16 ? r8 + 8 * ((qw >> 1) & 1) : r8;
      ct[j] = MP == 16 ? (qw & 1) + 2 * (qw >> 2) : qw;
      so[j] = sw128(mt[j], SN * ct[j]);
    }
    // rows block * kBlock + m and that + MP (Im plane): multiples of 8 rows apart, so the swizzle
    // pattern of row m carries over and the offsets differ by whole 1024-byte row groups
    constexpr uint32_t kImOff = (uint32_t)(MP / 8) * 1024u;
    uint32_t g0 = 0, gs0 = 0;   // CTA operand / staging stage of the current problem's first stage
    uint32_t own = 0;           // problems whose scaling unit this group has fixed
    int kth = 0;                // problem counter of this CTA
    bool live = true;
    for (int pi = blockIdx.x; pi < count && live && !*abort; pi += gridDim.x, ++kth) {
      const PlanProblem &pp = probs[list[pi]];
      const int M = pp.p.M, N = pp.p.N, ldx = pp.p.ldx;
      const float2 *X = reinterpret_cast<const float2 *>(pp.p.X);
      const int nst = (N + kCbSnap - 1) / kCbSnap, nstg = (N + kCbStgSnap - 1) / kCbStgSnap;
      const int r = kth % kCbRing;
      float scale = 0.f;
      bool bad = false, have = false;
      for (int s = (grp - (int)(g0 % kCbGroups) + kCbGroups) % kCbGroups; s < nst; s += kCbGroups) {
        const uint32_t g = g0 + (uint32_t)s, gs = gs0 + (uint32_t)(s / kCbSub);
        const int sub = s % kCbSub, ss = gs % kCbStg, os = g % kCbOps;
        if (!warp_wait(smem_u32(&sh.full[ss]), (gs / kCbStg) & 1u, abort)) {
          live = false;
          break;
        }
        // the tasks' SN snapshots of row m (zeros past N and for rows >= M); t counts snapshots
        // from the start of the staging stage, whose first cb arrived by bulk copy
        float re[kCbTasks][SN], im[kCbTasks][SN];
        const int t0 = (s - sub) * kCbSnap, cnt = min(kCbStgSnap, N - t0), cb = cnt & ~1;
        const uint8_t *stg = sm + Lay::kOffStg + ss * Lay::kStgBytes;
#pragma unroll
        for (int j = 0; j < kCbTasks; ++j) {
          const int m = mt[j], c = ct[j];
#pragma unroll
          for (int q = 0; q < SN / 2; ++q) {
            const int t = sub * kCbSnap + c * SN + 2 * q;
            float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
            if (m < M) {
              if (t + 1 < cb) {
                v = *reinterpret_cast<const float4 *>(stg + m * kCbRowPitch + 8 * t);
              } else if (t < cnt) {   // t >= cb: the odd last snapshot, outside the bulk copy
                const float2 a = X[(size_t)m * ldx + t0 + t];
                v.x = a.x;
                v.y = a.y;
              }
            }
            re[j][2 * q] = v.x;
            im[j][2 * q] = v.y;
            re[j][2 * q + 1] = v.z;
            im[j][2 * q + 1] = v.w;
          }
        }
        // this sub-stage of the staging stage has been read. A staging stage takes 8 arrivals (four
        // sub-stages x two warps); the last sub-stage of a short one stands in for the missing ones.
        {
          const int nsub = min(kCbSub, nst - (s - sub));
          __syncwarp();
          if (lane == 0) arrive_cnt(smem_u32(&sh.empty[ss]), sub == nsub - 1 ? (uint32_t)(1 + kCbSub - nsub) : 1u);
        }
        if (s == 0) {
          // this group fixes the scaling unit from the problem's first stage: 2^(k-1) <= mx < 2^k,
          // u0 = 2^(k-5), so |w| = |x| / u0 <= 64 for |x| <= 2^(k+1) (one bit of headroom)
          float mx = 0.f;
#pragma unroll
          for (int j = 0; j < kCbTasks; ++j)
#pragma unroll
            for (int q = 0; q < SN; ++q) mx = fmaxf(mx, fmaxf(fabsf(re[j][q]), fabsf(im[j][q])));
#pragma unroll
          for (int off = 16; off > 0; off >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, off));
          const int slot = own & 1;
          if (lane == 0) sh.red[grp][slot][warp % kCbGroupWarps] = mx;
          if (!warp_bar(&sh.pred[grp][slot], (own >> 1) & 1u, abort)) {
            live = false;
            break;
          }
          mx = 0.f;
#pragma unroll
          for (int w = 0; w < kCbGroupWarps; ++w) mx = fmaxf(mx, sh.red[grp][slot][w]);
          ++own;
          const int eb = (int)((__float_as_uint(mx) >> 23) & 0xffu);
          bad = eb < 4 || eb > 254;                       // zero, subnormal, tiny or non-finite
          const int k = eb - 126;
          scale = bad ? 0.f : __uint_as_float((uint32_t)(258 - eb) << 23);   // 2^(5 - k)
          if (lt == 0) {
            if (kth >= kCbRing) cb_wait(smem_u32(&sh.eempty[r]), (uint32_t)((kth / kCbRing - 1) & 1), abort);
            sh.eexp[r] = bad ? INT_MIN : k;
            sh.escale[r] = scale;
            arrive(smem_u32(&sh.efull[r]));
            arrive(smem_u32(&sh.sfull[r]));
          }
          have = true;
        } else if (!have) {
          // the scaling unit fixed by the group that sliced the problem's first stage
          if (!warp_wait(smem_u32(&sh.sfull[r]), (uint32_t)((kth / kCbRing) & 1), abort)) {
            live = false;
            break;
          }
          scale = sh.escale[r];
          have = true;
        }
        // operand slot free (the MMAs of its previous stage are done)
        if (g >= (uint32_t)kCbOps && !warp_wait(smem_u32(&sh.opempty[os]), (g / kCbOps - 1) & 1u, abort)) {
          live = false;
          break;
        }
        uint8_t *op = sm + Lay::kOffOp + os * Lay::kOpBytes;
        // w = x * scale, pairs of consecutive snapshots in 64-bit registers
        const uint64_t sc2 = pack2(scale, scale);
        uint64_t wr[kCbTasks][SN / 2], wi[kCbTasks][SN / 2];
        float amax = 0.f;   // largest |w| of the thread's samples, NaN if any is NaN
#pragma unroll
        for (int j = 0; j < kCbTasks; ++j)
#pragma unroll
          for (int q = 0; q < SN / 2; ++q) {
            wr[j][q] = mul2(pack2(re[j][2 * q], re[j][2 * q + 1]), sc2);
            wi[j][q] = mul2(pack2(im[j][2 * q], im[j][2 * q + 1]), sc2);
            amax = max_abs_nan(amax, max_abs_nan(max_abs_nan(lo2(wr[j][q]), hi2(wr[j][q])),
                                                 max_abs_nan(lo2(wi[j][q]), hi2(wi[j][q]))));
          }
        bad |= !(amax <= 64.f);
#pragma unroll
        for (int k = 0; k < 6; ++k) {
          const float Cf = slice_magic(k);
          const uint64_t C = pack2(Cf, Cf);
          const uint32_t blk = (uint32_t)(S::block_of(k) * S::kBlock / 8) * 1024u;
#pragma unroll
          for (int j = 0; j < kCbTasks; ++j) {
            uint32_t pr[SN / 2], pim[SN / 2];
#pragma unroll
            for (int q = 0; q < SN / 2; ++q) {
              const uint64_t sr = sub2(add2(wr[j][q], C), C), si = sub2(add2(wi[j][q], C), C);
              if (k < 5) {
                wr[j][q] = sub2(wr[j][q], sr);
                wi[j][q] = sub2(wi[j][q], si);
              }
              const __nv_bfloat162 a = __floats2bfloat162_rn(lo2(sr), hi2(sr)),
                                   b = __floats2bfloat162_rn(lo2(si), hi2(si));
              pr[q] = *reinterpret_cast<const uint32_t *>(&a);
              pim[q] = *reinterpret_cast<const uint32_t *>(&b);
            }
            if constexpr (SN == 4) {
              *reinterpret_cast<uint2 *>(op + so[j] + blk) = make_uint2(pr[0], pr[1]);
              *reinterpret_cast<uint2 *>(op + so[j] + blk + kImOff) = make_uint2(pim[0], pim[1]);
            } else {
              *reinterpret_cast<uint32_t *>(op + so[j] + blk) = pr[0];
              *reinterpret_cast<uint32_t *>(op + so[j] + blk + kImOff) = pim[0];
            }
          }
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncwarp();
        if (lane == 0) arrive(smem_u32(&sh.opfull[os]));
      }
      // a sample outside the unit's range (or a non-finite one): recompute the problem elsewhere
      if (live && __any_sync(0xffffffffu, bad) && lane == 0) atomicOr(&flags[pi], 1);
      g0 += (uint32_t)nst;
      gs0 += (uint32_t)nstg;
    }
  } else if (warp == kCbTmaWarp) {
    // ---------------------------------------------------------------- TMA: staging copies
    if (lane == 0) {
      uint32_t g = 0;   // staging stages issued
      for (int pi = blockIdx.x; pi < count && !*abort; pi += gridDim.x) {
        const PlanProblem &pp = probs[list[pi]];
        const int M = pp.p.M, N = pp.p.N, ldx = pp.p.ldx;
        const float2 *X = reinterpret_cast<const float2 *>(pp.p.X);
        const int nstg = (N + kCbStgSnap - 1) / kCbStgSnap;
        flags[pi] = 0;   // ordered before the producers' marks by the first stage's mbarrier
        for (int st = 0; st < nstg; ++st, ++g) {
          const int ss = g % kCbStg;
          if (g >= (uint32_t)kCbStg && !cb_wait(smem_u32(&sh.empty[ss]), (g / kCbStg - 1) & 1u, abort)) break;
          const int t0 = st * kCbStgSnap, cb = min(kCbStgSnap, N - t0) & ~1;
          const uint32_t dst = smem_u32(sm + Lay::kOffStg + ss * Lay::kStgBytes);
          arrive_tx(smem_u32(&sh.full[ss]), (uint32_t)(M * cb * 8));
          if (cb > 0)
            for (int m = 0; m < M; ++m)
              bulk_copy(dst + m * kCbRowPitch, X + (size_t)m * ldx + t0, (uint32_t)(cb * 8), smem_u32(&sh.full[ss]));
        }
      }
      // let every copy in flight land before the CTA can exit
      if (*abort)
        for (uint32_t q = g > (uint32_t)kCbStg ? g - kCbStg : 0u; q < g; ++q)
          mbar_wait(smem_u32(&sh.full[q % kCbStg]), (q / kCbStg) & 1u);
    }
    __syncwarp();
  } else if (warp == kCbMmaWarp) {
    // ---------------------------------------------------------------- MMA issuer
    if (lane == 0) {
      const uint32_t idesc = inst_desc(1, S::kN);
      uint32_t g = 0, gw = 0;
      for (int pi = blockIdx.x; pi < count && !*abort; pi += gridDim.x) {
        const int N = probs[list[pi]].p.N;
        const int nst = (N + kCbSnap - 1) / kCbSnap, nwin = (nst + kCbWin - 1) / kCbWin;
        for (int w = 0; w < nwin && !*abort; ++w, ++gw) {
          const int buf = gw & 1;
          if (gw >= 2u && !cb_wait(smem_u32(&sh.accempty[buf]), ((gw >> 1) - 1) & 1u, abort)) break;
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          const int s1 = min(nst, (w + 1) * kCbWin);
          for (int s = w * kCbWin; s < s1; ++s, ++g) {
            const int os = g % kCbOps;
            if (!cb_wait(smem_u32(&sh.opfull[os]), (g / kCbOps) & 1u, abort)) break;
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t pa = smem_u32(sm + Lay::kOffOp + os * Lay::kOpBytes), pb = pa + S::kBStart * 128;
#pragma unroll
            for (int kk = 0; kk < 4; ++kk)
              mma(tmem + (uint32_t)(buf * kCbAccCols), smem_desc(pa + kk * 32), smem_desc(pb + kk * 32), idesc,
                  (s > w * kCbWin || kk > 0) ? 1u : 0u);
            commit(smem_u32(&sh.opempty[os]));
          }
          commit(smem_u32(&sh.accfull[buf]));
        }
      }
      // every MMA of this thread done before the CTA releases TMEM and shared memory
      commit(smem_u32(&sh.fin));
      mbar_wait(smem_u32(&sh.fin), 0u);
    }
    __syncwarp();
  } else {
    // ---------------------------------------------------------------- TMEM readout and finalize
    const int q = warp & 3;                                    // TMEM lane quarter
    const int rt = tid - 32 * kCbReadWarp0;                    // 0..127
    uint32_t gw = 0;
    int kth = 0;
    for (int pi = blockIdx.x; pi < count && !*abort; pi += gridDim.x, ++kth) {
      const PlanProblem &pp = probs[list[pi]];
      const int M = pp.p.M, N = pp.p.N;
      const int nst = (N + kCbSnap - 1) / kCbSnap, nwin = (nst + kCbWin - 1) / kCbWin;
      long long ure[MP], uim[MP];
#pragma unroll
      for (int b = 0; b < MP; ++b) ure[b] = uim[b] = 0;
      bool ok = true;
      for (int w = 0; w < nwin; ++w, ++gw) {
        const int buf = gw & 1;
        if (!warp_wait(smem_u32(&sh.accfull[buf]), (gw >> 1) & 1u, abort)) {
          ok = false;
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        read_window<MP>(tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(buf * kCbAccCols), q, lane, ure, uim);
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncwarp();
        if (lane == 0) arrive(smem_u32(&sh.accempty[buf]));
      }
      if (!ok) break;
      // finalize: U' = sum over this problem's rows, R = (U' + U'^H) / 2 scaled
      const int r = kth % kCbRing;
      if (!warp_wait(smem_u32(&sh.efull[r]), (uint32_t)((kth / kCbRing) & 1), abort)) break;
      const int kexp = sh.eexp[r];
      // every thread has zeroed its entries of U (previous problem) before anyone adds to it
      if (!warp_bar(&sh.rb[0], (uint32_t)(kth & 1), abort)) break;
      // my row: element a (lanes within the slice block); padding rows add nothing
      const int a = MP == 16 ? (lane & 15) : (lane & 7);
#pragma unroll
      for (int b = 0; b < MP; ++b) {
        if (ure[b] != 0) atomicAdd(reinterpret_cast<unsigned long long *>(&U[(a * MP + b) * 2]), (unsigned long long)ure[b]);
        if (uim[b] != 0) atomicAdd(reinterpret_cast<unsigned long long *>(&U[(a * MP + b) * 2 + 1]), (unsigned long long)uim[b]);
      }
      if (!warp_bar(&sh.rb[1], (uint32_t)(kth & 1), abort)) break;
      if (lane == 0) arrive(smem_u32(&sh.eempty[r]));
      // one thread per pair (ea <= eb): both entries of R from U'(ea, eb) and U'(eb, ea), then zeroed
      double2 *R64 = reinterpret_cast<double2 *>(ws + pp.r64_off);
      const double sc = kexp == INT_MIN ? 0.0 : ldexp(1.0, 2 * kexp - 10 - 29) / (double)N;
      for (int e = rt; e < M * M; e += 128) {
        const int ea = e / M, eb = e % M;
        if (ea > eb) continue;
        long long *u1 = &U[(ea * MP + eb) * 2], *u2 = &U[(eb * MP + ea) * 2];
        const long long re = u1[0] + u2[0], im = u1[1] - u2[1];
        if (kexp != INT_MIN) {   // a marked problem is rewritten by the fixup kernel
          R64[ea * M + eb] = make_double2((double)re * sc, ea == eb ? 0.0 : (double)im * sc);
          R64[eb * M + ea] = make_double2((double)re * sc, ea == eb ? 0.0 : -(double)im * sc);
        }
        u1[0] = u1[1] = u2[0] = u2[1] = 0;
      }
    }
  }

  // -------------------------------------------------------------------- teardown
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (*abort && tid == 0)   // every problem of this CTA goes to the fixup kernel
    for (int pi = blockIdx.x; pi < count; pi += gridDim.x) flags[pi] = 2;
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512));
}

template <int MP>
cudaError_t launch_class(const uint8_t *plan_dev, const PlanHeader &h, uint8_t *ws, int cls, cudaStream_t s) {
  const int n = h.ncovtc[cls];
  if (n == 0) return cudaSuccess;
  cudaError_t e = ensure_smem_attr(reinterpret_cast<const void *>(covariance_tc_batch_kernel<MP>), CbLayout<MP>::kSmem);
  if (e != cudaSuccess) return e;
  const int grid = n < device_sm_count() ? n : device_sm_count();   // one CTA per SM (512 TMEM columns)
  covariance_tc_batch_kernel<MP><<<grid, kCbThreads, CbLayout<MP>::kSmem, s>>>(plan_dev, ws, cls);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_covariance_tc_batch(const uint8_t *plan_dev, const PlanHeader &h, uint8_t *ws, cudaStream_t s) {
  cudaError_t e = launch_class<8>(plan_dev, h, ws, 0, s);
  if (e != cudaSuccess) return e;
  return launch_class<16>(plan_dev, h, ws, 1, s);
}

}  // namespace doa
