// Internal declarations shared by the CUDA translation units of libdoa.so.
// Device helpers here are header-only (inline) so that every kernel file compiles on its own.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "doa.h"

namespace doa {

constexpr int kMaxM = 64;
constexpr int kCovChunk = 1024;    // snapshots per covariance work item
constexpr int kMaxSweeps = 60;     // Jacobi sweep cap (ENOCONV beyond)
constexpr double kJacobiTol = 1e-15;

// ------------------------------------------------------------------------------------------
// Complex helpers
// ------------------------------------------------------------------------------------------
__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double2 cconj(double2 a) { return make_double2(a.x, -a.y); }

// ------------------------------------------------------------------------------------------
// Grid phase table. theta_k = lo + k*step in FP64 (rounded multiply, rounded add), and the
// phase increment of the half-wavelength ULA, s_k = sin(theta_k), stored as a 32-bit fixed
// point fraction of a half turn: S_k = round(s_k * 2^31) mod 2^32. Then for element m the
// phase m*pi*s_k equals pi * (m*S_k mod 2^32) * 2^-31 exactly in integer arithmetic
// (the wrap of 2^32 is a whole number of turns), so the phase error is that of one rounding
// of s_k (<= 2^-32 half turns), independent of m.
// ------------------------------------------------------------------------------------------
__device__ __forceinline__ uint32_t phase_step_of_sin(double s) {
  long long q = __double2ll_rn(s * 2147483648.0);
  return (uint32_t)q;
}
__device__ __forceinline__ uint32_t grid_phase_step(double lo, double step, int k) {
  double theta = __dadd_rn(lo, __dmul_rn((double)k, step));
  return phase_step_of_sin(sin(theta * 0.017453292519943295));  // pi/180
}

// 64-bit form of the same phase step, S64 = round(2^63 sin theta) mod 2^64 (computed as twice
// round(2^62 s) so that s = +-1 stays in range; both map to 2^63, a half turn, as they must).
__device__ __forceinline__ uint64_t phase_step64_of_sin(double s) {
  return (uint64_t)__double2ll_rn(s * 4611686018427387904.0) << 1;   // 2^62
}

// exp(j (pi/2) (quad + f)) for a quarter-turn count quad (mod 4) and a remainder f in [-1/2, 1/2]
// of a quarter turn: the Taylor series of sin and cos about 0 in x = (pi/2) f, |x| <= pi/4, through
// x^9 and x^10 (Lagrange remainders below 2e-9 and 2e-10), then a rotation by quad quarter turns.
// Coefficients are (pi/2)^n / n! folded so that the polynomials take f directly.
__device__ __forceinline__ float2 phasor_quarter_core(float f, uint32_t quad) {
  float f2 = f * f;
  // sin((pi/2) f) = f*(s1 + f2*(s3 + f2*(s5 + f2*(s7 + f2*s9))))
  const float s1 = 1.5707963267948966f, s3 = -0.6459640975062462f, s5 = 0.07969262624616704f,
              s7 = -0.004681754135318687f, s9 = 0.00016044118478735982f;
  // cos((pi/2) f) = 1 + f2*(c2 + f2*(c4 + f2*(c6 + f2*(c8 + f2*c10))))
  const float c2 = -1.2337005501361697f, c4 = 0.25366950790104797f, c6 = -0.020863480763352958f,
              c8 = 0.0009192602748394263f, c10 = -2.5202042373060603e-05f;
  float sp = fmaf(f2, s9, s7);
  sp = fmaf(f2, sp, s5);
  sp = fmaf(f2, sp, s3);
  sp = fmaf(f2, sp, s1);
  float sn = f * sp;
  float cp = fmaf(f2, c10, c8);
  cp = fmaf(f2, cp, c6);
  cp = fmaf(f2, cp, c4);
  cp = fmaf(f2, cp, c2);
  float cs = fmaf(f2, cp, 1.0f);
  // rotate by quad quarter turns: (c, s) -> quad 1: (-s, c), 2: (-c, -s), 3: (s, -c)
  float re = (quad & 1u) ? sn : cs;
  float im = (quad & 1u) ? cs : sn;
  if ((quad + 1u) & 2u) re = -re;   // quad 1 or 2
  if (quad & 2u) im = -im;          // quad 2 or 3
  return make_float2(re, im);
}

// exp(j*pi*phi*2^-31) for a 32-bit phase phi (a fraction of a full turn: 2^32 = 2 pi).
// The top two bits (rounded) select the quadrant; the signed remainder f in [-1/2, 1/2) of a
// quarter turn goes to phasor_quarter_core.
__device__ __forceinline__ float2 phasor_q32(uint32_t phi) {
  uint32_t quad = (phi + 0x20000000u) >> 30;             // nearest quarter turn, 0..3
  int32_t rem = (int32_t)(phi - (quad << 30));            // [-2^29, 2^29)
  float f = (float)rem * 9.31322574615478515625e-10f;     // * 2^-30 -> [-0.5, 0.5)
  return phasor_quarter_core(f, quad);
}

// exp(j (pi/2) t4) for a phase t4 in quarter turns, |t4| < 2^22. Adding 1.5 * 2^23 rounds t4 to
// the nearest integer q (ties to even) and leaves q mod 2^22 in the low mantissa bits, so the
// quadrant is those bits mod 4 and the remainder t4 - q in [-1/2, 1/2] is exact: no conversion
// instructions.
__device__ __forceinline__ float2 phasor_quarter(float t4) {
  const float big = 12582912.0f;                          // 1.5 * 2^23
  const float y = __fadd_rn(t4, big);
  const float q = __fsub_rn(y, big);
  return phasor_quarter_core(__fsub_rn(t4, q), __float_as_uint(y) & 3u);
}

// FP64 counterpart for refinement: exp(j 2 pi phi 2^-64) for a 64-bit phase phi (fraction of a
// full turn). Quadrant from the top two bits (rounded), remainder f in [-1/2, 1/2) of a quarter
// turn, then the Taylor series of sin and cos of x = (pi/2) f (|x| <= pi/4) through x^17 and
// x^16: the first omitted terms are below 1e-19 and 3e-18. The coefficients (pi/2)^n / n! are
// formed at compile time from pi/2.
__host__ __device__ constexpr double half_pi_taylor(int n) {
  double c = 1.0;
  for (int k = 1; k <= n; ++k) c *= 1.5707963267948966 / k;
  return c;
}
__device__ __forceinline__ double2 phasor_q64(uint64_t phi) {
  const uint64_t quad = (phi + (1ull << 61)) >> 62;
  const int64_t rem = (int64_t)(phi - (quad << 62));                 // [-2^61, 2^61)
  const double f = (double)rem * 2.168404344971009e-19;              // * 2^-62
  const double f2 = f * f;
  constexpr double s1 = half_pi_taylor(1), s3 = -half_pi_taylor(3), s5 = half_pi_taylor(5),
                   s7 = -half_pi_taylor(7), s9 = half_pi_taylor(9), s11 = -half_pi_taylor(11),
                   s13 = half_pi_taylor(13), s15 = -half_pi_taylor(15), s17 = half_pi_taylor(17);
  constexpr double c2 = -half_pi_taylor(2), c4 = half_pi_taylor(4), c6 = -half_pi_taylor(6),
                   c8 = half_pi_taylor(8), c10 = -half_pi_taylor(10), c12 = half_pi_taylor(12),
                   c14 = -half_pi_taylor(14), c16 = half_pi_taylor(16);
  double sp = fma(f2, s17, s15);
  sp = fma(f2, sp, s13);
  sp = fma(f2, sp, s11);
  sp = fma(f2, sp, s9);
  sp = fma(f2, sp, s7);
  sp = fma(f2, sp, s5);
  sp = fma(f2, sp, s3);
  sp = fma(f2, sp, s1);
  const double sn = f * sp;
  double cp = fma(f2, c16, c14);
  cp = fma(f2, cp, c12);
  cp = fma(f2, cp, c10);
  cp = fma(f2, cp, c8);
  cp = fma(f2, cp, c6);
  cp = fma(f2, cp, c4);
  cp = fma(f2, cp, c2);
  const double cs = fma(f2, cp, 1.0);
  double re = (quad & 1u) ? sn : cs;
  double im = (quad & 1u) ? cs : sn;
  if ((quad + 1u) & 2u) re = -re;   // quad 1 or 2
  if (quad & 2u) im = -im;          // quad 2 or 3
  return make_double2(re, im);
}

// ------------------------------------------------------------------------------------------
// Batch plan. The same bytes live on the host (for launch sizes) and on the device.
// ------------------------------------------------------------------------------------------
constexpr uint32_t kPlanMagic = 0x444f4131u;  // "DOA1"
constexpr int kNumBuckets = 4;                // M <= 8, <= 16, <= 32, <= 64
// Covariance work-item classes: 4x4 register blocks per row, MB = ceil(M / 4) in {2, 3, 4} use
// the block-task kernel (one launch per class, CTA shape fixed by MB); every other M the
// generic kernel.
constexpr int kCovClasses = 4;
__host__ __device__ inline int cov_class(int M) {
  const int mb = (M + 3) / 4;
  return (mb >= 2 && mb <= 4) ? mb - 2 : 3;
}

struct PlanProblem {
  doa_problem p;          // the caller's descriptor
  int64_t r64_off;        // byte offset of R (M x M complex128) in the workspace
  int64_t part_off;       // byte offset of the covariance partials (nchunks x M x M complex128)
  int64_t fac_off;        // byte offset of the scan factor F (M x (M+1) complex128 capacity,
                          // column-major) followed by the EV weights (M doubles)
  int64_t tile_start;     // first scan tile of this problem within its bucket's tile range
  int32_t nchunks;        // covariance work items of this problem
  int32_t first_job;      // first (problem, algorithm) job
  int32_t njobs;
  int32_t grid_id;        // index of the problem's phase table
  int32_t Kf, Kn;         // factor columns; columns read by MUSIC / EV (E_n), 0 if neither
  int32_t kphd, kmn;      // columns read by PHD (v_min) and MN (valph), -1 if absent
  int32_t slot[4];        // output row of each algorithm (doa_alg order), -1 if not requested
  int32_t npts;           // points of one spectrum: L, or La x Le for a geometry problem
  int32_t geo_grid;       // geometry problems: index of the azimuth x elevation grid's tables
  int32_t geo_steer;      // geometry problems: index of the shared FP32 steering table, or -1
};

// The Python binding reads problem i's R offset (r64_off) from the plan record at
// off_prob + i * sizeof(PlanProblem).
static_assert(offsetof(PlanProblem, r64_off) == sizeof(doa_problem), "PlanProblem layout changed");
static_assert(sizeof(PlanProblem) == sizeof(doa_problem) + 96, "PlanProblem layout changed");

__host__ __device__ inline int m_bucket(int M) { return M <= 8 ? 0 : (M <= 16 ? 1 : (M <= 32 ? 2 : 3)); }
__host__ __device__ inline int scan_mp(int M) { return 8 << m_bucket(M); }   // padded rows of the FP32 scan

// A problem's scan factor area: F (M x (M+1) complex128, column-major) and the EV weights (M
// doubles), then at fac32_off(M) the FP32 copy the grid-shared scan reads: F32 (M+1 columns of
// scan_mp(M) elements (bx, bx, by, by), rows >= M zero), w32 (scan_mp(M) floats) and the four
// readout thresholds.
__host__ __device__ inline int64_t fac32_off(int M) { return ((int64_t)M * (M + 1) * 16 + (int64_t)M * 8 + 15) / 16 * 16; }
__host__ __device__ inline int64_t factor_bytes(int M) {
  return fac32_off(M) + (int64_t)(M + 1) * scan_mp(M) * 16 + (int64_t)scan_mp(M) * 4 + 16;
}

struct PlanJob {          // one (problem, algorithm) pair: a spectrum and its peaks
  int32_t prob;
  int32_t alg;
  int32_t slot;           // position of the algorithm among the problem's algorithms
  int32_t pad;
};

struct PlanGrid {
  double lo, step;
  int32_t L;
  int32_t pad;
  int64_t S_off;          // byte offset of the phase table (L x uint32) in the workspace
  int64_t S64_off;        // byte offset of the 64-bit phase table (L x uint64) in the workspace
};

// Azimuth x elevation grid of geometry problems, with its trigonometric tables in the workspace:
// (sin, cos) of theta_k = az_lo + k az_step (k < La) followed by those of phi_l = el_lo + l el_step
// (l < Le), evaluated in FP64 (rounded multiply, rounded add, then sincospi of the angle / 180).
struct PlanGeoGrid {
  double az_lo, az_step, el_lo, el_step;
  int32_t La, Le;
  int64_t t32_off;        // float2[La + Le], the FP64 values rounded once
  int64_t t64_off;        // double2[La + Le]
};

// FP32 steering table of the geometry problems that pass the same positions pointer, grid and M:
// a_m at every point of the grid, rows m < MP (rows >= M zero), written once per solve from the
// FP64 phases and read by the scan instead of evaluating the phasors for each problem.
struct PlanGeoSteer {
  const double *pos;      // the problems' element positions (M x 3, FP64, wavelengths)
  int32_t geo_grid;       // their azimuth x elevation grid
  int32_t M, MP;          // elements; table rows (the M bucket's padded size)
  int32_t npts, ldt;      // points of the grid; row stride (npts rounded up to kSteerAlign)
  int32_t pad;
  int64_t tab_off;        // workspace byte offset of float2[MP][ldt]
};
constexpr int kSteerAlign = 1024;   // row stride multiple: every scan tile's points lie inside a row

// Grid-shared FP32 scan: ULA problems of one M bucket that share a grid are scanned in groups; a
// unit is one tile of the grid for every problem of a group (the tile's steering phasors are
// generated once and contracted with each problem's factor in turn). Units are numbered group by
// group from unit_start.
struct PlanScanGroup {
  int32_t grid_id;
  int32_t first;          // first entry of the group in the bucket's problem list
  int32_t count;          // problems in the group (<= kScanGroupMax)
  int32_t tiles;          // tiles of kScanThreads x scan_pt points covering the grid
  int64_t unit_start;
};
// Grid-shared tensor-core scan: a group's stacked factor columns (each problem's 2 Kf real
// columns rounded up to 16) form one UMMA N <= kTcgMaxCols; its record in the workspace holds the
// split operand W (hi, lo: kTcgMaxCols rows of 128 bytes, 128B-swizzled K-major) and a TcgProb per
// problem.
constexpr int kTcgMaxCols = 128;
constexpr int kTcgTile = 128;          // grid points per tile (UMMA M)
constexpr int kTcgMaxProbs = 16;
constexpr int kTcgChunk = 8;           // groups per unit (one steering block serves all of them)
struct PlanTcGroup {
  int32_t first;          // first entry of the group in the tcg problem list
  int32_t count;
  int32_t NG;             // stacked columns (multiple of 16, <= kTcgMaxCols)
  int32_t prec;           // DOA_BF16X3 or DOA_FP16X3
  int64_t rec_off;        // workspace byte offset of the group record (1024-aligned)
};
struct PlanTcChunk {
  int32_t grid_id;
  int32_t first_group;
  int32_t ngroups;
  int32_t Mg;             // phasors per point the steering block holds (max M of its groups, to 8)
  int32_t tiles;          // 128-point tiles of the grid
  int32_t pad;
  int64_t unit_start;
};
struct TcgProb {
  float *P[4];            // output row per readout (null: absent)
  const float2 *B32;      // FP32 factor [Kf][MPs] (re-evaluation)
  const float *w32;       // FP32 EV weights
  int32_t prob, col, Kf, Kn, kphd, kmn, M, MPs;
  float scale2;           // the W scale's square inverse (den = accumulator sum * scale2)
  float thr32[4];         // FP32 re-evaluation threshold per readout
  float thrtc[4];         // tensor-product threshold per readout
  int32_t pad[3];
};
static_assert(sizeof(TcgProb) == 128, "TcgProb layout");
constexpr int64_t kTcgWBytes = (int64_t)kTcgMaxCols * 128;
constexpr int64_t kTcgRecBytes = 2 * kTcgWBytes + kTcgMaxProbs * (int64_t)sizeof(TcgProb);

constexpr int kScanGroupMax = 32;       // problems per group (their jobs are staged in shared memory)
constexpr int kScanGroupDefault = 32;
__host__ __device__ inline bool scan_group_allowed(int g) { return g >= 1 && g <= kScanGroupMax && (g & (g - 1)) == 0; }

struct PlanCovItem {
  int32_t prob;
  int32_t chunk;
};

struct PlanHeader {
  uint32_t magic;
  int32_t nprob, njobs, ngrids, ncov;
  int32_t nreduce;                       // problems with more than one covariance chunk
  int32_t eig_count[kNumBuckets];        // problems per M bucket
  int32_t scan_jobs[kNumBuckets];        // scan jobs (problems) per M bucket
  int64_t scan_tiles[kNumBuckets];       // scan tiles per M bucket
  int32_t scan_pt[kNumBuckets];          // grid points per scan thread, per M bucket
  int64_t grid_points;                   // sum of L over distinct grids
  int64_t ws_bytes;
  // byte offsets of the arrays inside the plan
  int64_t off_prob, off_job, off_grid, off_cov, off_reduce, off_eig[kNumBuckets],
      off_scan[kNumBuckets], off_grid_pts;
  int32_t eig_mats[kNumBuckets];         // matrices per Jacobi warp, per M bucket
  int32_t cov_first[kCovClasses + 1];    // covariance items sorted by class: class c owns
                                         // items [cov_first[c], cov_first[c + 1])
  // problems scanned on the tensor cores (prec BF16X3 / FP16X3, M <= 32), in their own list
  int32_t tc_jobs;
  int32_t tc_cols;                       // TMEM columns a CTA allocates (covers every tc problem)
  int64_t tc_tiles;                      // 128-point tiles over all tc problems
  int64_t off_tc;                        // byte offset of the tc problem list
  int32_t npolish;                       // problems with DOA_FLAG_POLISH_PEAKS
  int32_t pad2;
  // problems with an explicit geometry (2-D azimuth x elevation scans), per M bucket
  int32_t geo_jobs[kNumBuckets];
  int64_t geo_tiles[kNumBuckets];
  int64_t off_geo[kNumBuckets];
  int32_t ngeo_grids;                    // distinct azimuth x elevation grids
  int32_t geo_grid_points;               // largest La + Le among them
  int64_t off_geo_grid;
  int32_t nrefine;                       // problems with a peak_angle output (sub-grid refinement)
  int32_t nroots;                        // problems with a root_angle output (root form of the scan)
  int64_t next_val_off;                  // workspace byte offset of one float per job: the value of
                                         // the best peak below the d selected (peak polish), or -1
  int32_t ngeo_steer;                    // shared FP32 steering tables of geometry problems
  int32_t steer_max_ldt;                 // largest row stride among them
  int64_t off_geo_steer;
  // problems whose covariance runs on the tensor cores (exact BF16 slices), M <= 8 and 8 < M <= 16;
  // their lists hold problem indices, longest N first
  int32_t ncovtc[2];
  int64_t off_covtc[2];
  int64_t covtc_flag_off;                // workspace byte offset of one int32 per listed problem
                                         // (class 0 then class 1): 0 done, else recomputed by
                                         // the compensated CUDA-core fixup kernel
  // grid-shared FP32 scan, per M bucket (problems in these groups are not in the per-problem lists)
  int32_t sg_size[kNumBuckets];          // problems per group (1: every problem scanned alone)
  int32_t sg_groups[kNumBuckets];
  int64_t sg_units[kNumBuckets];
  int64_t off_sg[kNumBuckets];           // PlanScanGroup arrays
  int64_t off_sgl[kNumBuckets];          // their problem lists
  int32_t sg_probs[kNumBuckets];         // problems in the groups
  // grid-shared tensor-core scan: split-operand ULA problems that share a grid, M bucket and
  // precision, stacked into groups of at most kTcgMaxCols factor columns (not in the tc list)
  int32_t tcg_groups;
  int32_t tcg_chunks;                    // runs of up to kTcgChunk groups of one grid and key
  int32_t tcg_probs;
  int32_t tcg_pad;
  int64_t tcg_units;                     // (tile, chunk) units
  int64_t off_tcg, off_tcc, off_tcgl;    // PlanTcGroup, PlanTcChunk arrays and the problem list
};

// The Python binding reads these header fields by position (int32 index 22 = scan_pt, 58 = eig_mats,
// 62 = cov_first, 67 = tc_jobs, 74 = npolish, 76 = geo_jobs, 96 = ngeo_grids, 100 = nrefine,
// 101 = nroots, 104 = ngeo_steer, 108 = ncovtc, 114 = covtc_flag_off (int64), 116 = sg_size,
// 120 = sg_groups, 124 = sg_units (int64), 148 = sg_probs, 152 = tcg_groups, 156 = tcg_units (int64)).
static_assert(offsetof(PlanHeader, scan_pt) == 88, "PlanHeader layout changed");
static_assert(offsetof(PlanHeader, scan_tiles) == 56, "PlanHeader layout changed");
static_assert(offsetof(PlanHeader, eig_mats) == 232, "PlanHeader layout changed");
static_assert(offsetof(PlanHeader, cov_first) == 248, "PlanHeader layout changed");
static_assert(offsetof(PlanHeader, tc_jobs) == 268, "PlanHeader layout changed");
static_assert(offsetof(PlanHeader, npolish) == 296, "PlanHeader layout changed");
static_assert(offsetof(PlanHeader, geo_jobs) == 304, "PlanHeader layout changed");
static_assert(offsetof(PlanHeader, ngeo_grids) == 384, "PlanHeader layout changed");
static_assert(offsetof(PlanHeader, nrefine) == 400, "PlanHeader layout changed");
static_assert(offsetof(PlanHeader, nroots) == 404, "PlanHeader layout changed");
static_assert(offsetof(PlanHeader, ngeo_steer) == 416, "PlanHeader layout changed");
static_assert(offsetof(PlanHeader, off_prob) == 120, "PlanHeader layout changed");
static_assert(offsetof(PlanHeader, ncovtc) == 432, "PlanHeader layout changed");
static_assert(offsetof(PlanHeader, covtc_flag_off) == 456, "PlanHeader layout changed");
static_assert(offsetof(PlanHeader, sg_size) == 464 && offsetof(PlanHeader, sg_units) == 496 &&
                  offsetof(PlanHeader, sg_probs) == 592,
              "PlanHeader layout changed");
static_assert(offsetof(PlanHeader, tcg_groups) == 608 && offsetof(PlanHeader, tcg_units) == 624 &&
                  sizeof(PlanHeader) == 656,
              "PlanHeader layout changed");

// Scan tiles: kScanThreads threads, each evaluating PT consecutive grid points (tile shape
// 128 x PT). PT is chosen per M bucket (the autotuner's knob); the register budget limits it
// to {1,2,4} for M <= 16, {1,2} for M <= 32 and 1 for M <= 64.
constexpr int kScanThreads = 128;
__host__ __device__ constexpr int scan_pt_default(int bucket) { return bucket <= 1 ? 4 : 1; }
__host__ __device__ inline bool scan_pt_allowed(int bucket, int pt) {
  return pt == 1 || (pt == 2 && bucket <= 2) || (pt == 4 && bucket <= 1);
}

// Jacobi packing: a warp holds G matrices of one bucket with G x (NP / 2) <= 32 rotation pairs
// (one lane each); the M <= 64 bucket runs one matrix per 256-thread CTA.
__host__ __device__ constexpr int eig_mats_max(int bucket) { return bucket == 0 ? 8 : (bucket == 1 ? 4 : (bucket == 2 ? 2 : 1)); }
__host__ __device__ inline bool eig_mats_allowed(int bucket, int g) {
  return g >= 1 && g <= eig_mats_max(bucket) && (g & (g - 1)) == 0;
}
// Default: the largest packing that still leaves ~24 warps per SM (152 SMs) of work, else 1.
__host__ __device__ inline int eig_mats_default(int bucket, int count) {
  int g = eig_mats_max(bucket);
  while (g > 1 && (count + g - 1) / g < 152 * 24) g >>= 1;
  return g;
}

// Tensor-core batch covariance: problems with M <= kCovTcMaxM, a 16-byte aligned X and an even
// row stride (whole-row bulk copies), and N <= kCovTcMaxN (range of its 64-bit sums).
constexpr int kCovTcMaxM = 16;
constexpr int kCovTcMaxN = 1 << 21;

// ------------------------------------------------------------------------------------------
// Per-device host state (device_cache.cu): the dynamic shared-memory limit of a kernel, raised
// once per device, and the device's SM count.
// ------------------------------------------------------------------------------------------
cudaError_t ensure_smem_attr(const void *func, int bytes);
int device_sm_count();
// The first bytes of a batch workspace hold per-solve counters (uint32, zeroed at the start of
// every doa_solve_batch): the next unit of the grid-shared FP32 scan (slot bucket), the next run
// of the per-problem FP32 scan (slot 4 + bucket) and the next unit of the grid-shared
// tensor-core scan (slot 8).
constexpr int64_t kWsCounterBytes = 256;
constexpr int kCtrShared = 0, kCtrBatch = 4, kCtrTcg = 8;
// Shared memory of the current device: per SM, per block (opt-in maximum), reserved per block.
struct SmemLimits {
  int per_sm, per_block, reserve;
};
SmemLimits device_smem_limits();

// ------------------------------------------------------------------------------------------
// Host launchers (one translation unit each). They return cudaError_t of the launch.
// ------------------------------------------------------------------------------------------
cudaError_t launch_grid_table_single(double lo, double step, int k0, int n, uint32_t *S, cudaStream_t s);
cudaError_t launch_grid_tables(const uint8_t *plan_dev, const PlanHeader &h, uint8_t *ws, cudaStream_t s);

cudaError_t launch_covariance_single(const float2 *X, int M, int N, int ldx, float2 *R, double2 *R64,
                                     cudaStream_t s);
cudaError_t launch_covariance_batch(const uint8_t *plan_dev, const PlanHeader &h, uint8_t *ws,
                                    cudaStream_t s);
cudaError_t launch_covariance_tc_batch(const uint8_t *plan_dev, const PlanHeader &h, uint8_t *ws, cudaStream_t s);
// Recomputes, with the compensated CUDA-core accumulation, the listed problems the tensor-core
// kernel marked (sample beyond its scaling range, non-finite data, or a bounded wait that ran out).
cudaError_t launch_covariance_fixup(const uint8_t *plan_dev, const PlanHeader &h, uint8_t *ws, cudaStream_t s);
cudaError_t launch_covariance_tc_single(const float2 *X, int M, int N, int ldx, int prec, float2 *R, double2 *R64,
                                        cudaStream_t s);

cudaError_t launch_eig_single(const double2 *R64, int M, int d, int alg, int prec, double *evals, double2 *B,
                              int *K_out, int *info, cudaStream_t s);
cudaError_t launch_model_order_single(const double *evals, int M, int N, int *mdl, int *aic, cudaStream_t s);
cudaError_t launch_eig_batch(const uint8_t *plan_dev, const PlanHeader &h, uint8_t *ws, int *status,
                             cudaStream_t s);

cudaError_t launch_scan_single(const double2 *B, int M, int K, int L, double lo, double step, int kofs,
                               const uint32_t *S, float *P, cudaStream_t s);
cudaError_t launch_scan_batch(const uint8_t *plan_dev, const PlanHeader &h, uint8_t *ws, cudaStream_t s);
cudaError_t launch_scan_tc_batch(const uint8_t *plan_dev, const PlanHeader &h, uint8_t *ws, int *status,
                                 cudaStream_t s);
cudaError_t launch_scan_tc_shared(const uint8_t *plan_dev, const PlanHeader &h, uint8_t *ws, int *status,
                                  cudaStream_t s);
// Tensor-core batch scan: tiles of 128 points; problems with M <= 32 only.
constexpr int kTcBatchMaxM = 32;
__host__ __device__ inline int tc_batch_cols(int Kf) {   // TMEM columns: 2 buffers x 2 accumulators of N
  const int N = (2 * Kf + 31) / 32 * 32;
  int p2 = 32;
  while (p2 < 4 * N) p2 <<= 1;
  return p2;
}
cudaError_t launch_scan_tc_single(const double2 *B, int M, int K, int L, double lo, double step, int prec,
                                  const uint32_t *S, float *P, cudaStream_t s);

// Bytes of the trigonometric tables of an La x Le geometry grid (float2 and double2 per angle).
__host__ __device__ inline int64_t geo_table_bytes(int64_t La, int64_t Le) { return 24 * (La + Le); }
cudaError_t launch_scan_geometry_single(const double2 *B, int M, int K, const double *pos, double az_lo,
                                        double az_step, int La, double el_lo, double el_step, int Le, float *P,
                                        uint8_t *ws, cudaStream_t s);
cudaError_t launch_geo_tables(const uint8_t *plan_dev, const PlanHeader &h, uint8_t *ws, cudaStream_t s);
cudaError_t launch_scan_geometry_batch(const uint8_t *plan_dev, const PlanHeader &h, uint8_t *ws, cudaStream_t s);

cudaError_t launch_peaks_single(const float *P, int L, int d, int *idx, float *val, int *count,
                                cudaStream_t s);
cudaError_t launch_peaks2d_single(const float *P, int La, int Le, int wrap_az, int d, int *idx, float *val,
                                  int *count, cudaStream_t s);
// ula / geo: launch the 1-D and / or the 2-D peak kernel (each only when the plan has such jobs);
// ula without geo is the pick after the peak polish (only the jobs the polish marked).
cudaError_t launch_peaks_batch(const uint8_t *plan_dev, const PlanHeader &h, uint8_t *ws, bool ula, bool geo,
                               cudaStream_t s);
cudaError_t launch_polish_batch(const uint8_t *plan_dev, const PlanHeader &h, uint8_t *ws, cudaStream_t s);
cudaError_t launch_roots_batch(const uint8_t *plan_dev, const PlanHeader &h, uint8_t *ws, int *status, cudaStream_t s);
cudaError_t launch_roots_single(const double2 *B, int M, int K, int d, double *theta, int *info, cudaStream_t s);
cudaError_t launch_refine_batch(const uint8_t *plan_dev, const PlanHeader &h, uint8_t *ws, cudaStream_t s);
// pos == null: ULA grid (lo, step); else geometry with azimuth (lo, step, La) and elevation (el_lo, el_step).
cudaError_t launch_refine_single(const double2 *B, int M, int K, double lo, double step, const double *pos,
                                 double el_lo, double el_step, int La, const int *idx, const int *count, int cap,
                                 double *out, cudaStream_t s);
cudaError_t launch_slice_peaks(const float *Pbuf, int b0, int k0, int k1, int L, int d, doa_slice_summary *out,
                               cudaStream_t s);

}  // namespace doa
