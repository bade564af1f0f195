/*
 * doa.h -- C ABI of libdoa.so: noise-subspace narrowband DOA estimation (PHD, MUSIC, EV, MN)
 * on one NVIDIA GB300 (sm_103a).
 *
 * The method is the one of Eray & Temizel, "Performance Analysis of Noise Subspace-based
 * Narrowband DOA Estimation Algorithms on CPU and GPU" (arXiv 2007.14135):
 *   Step-1  R = X X^H / N                                   (Sec. 3.1, Eq. 3; Table 2)
 *   Step-2  eigendecomposition of the Hermitian R           (Table 2; SVD == EVD for PSD R)
 *   Step-3/4 noise subspace and weighting                   (Table 3)
 *   Step-5  P(theta) = 1 / (a(theta)^H C a(theta))          (Table 2; steering vector Eq. 2)
 *   Step-6  peak finding and selection of D peaks           (Table 2)
 *
 * Conventions shared by every entry point:
 *   - All data pointers are DEVICE pointers unless stated otherwise; the caller owns every
 *     buffer. No entry point allocates device or pinned memory, and none synchronises the
 *     stream: each call only enqueues work on `stream` (a cudaStream_t passed as void*; NULL =
 *     legacy default stream).
 *   - Complex numbers are interleaved (re, im): complex64 = 2 floats, complex128 = 2 doubles.
 *   - The array is a half-wavelength uniform linear array (Eq. 2 with x_m = m*lambda/2,
 *     y = z = 0, phi = 90 deg): a_m(theta) = exp(+j*pi*m*sin(theta)), m = 0..M-1, theta in
 *     degrees from broadside. Element 0 is the reference element of MN.
 *   - The scan grid is theta_k = lo_deg + k*step_deg, k = 0..L-1, evaluated in FP64.
 *   - Other geometries (any element positions; Eq. 2 as printed) are scanned over an
 *     azimuth x elevation grid by doa_scan_geometry / doa_peaks2d and by batch problems that
 *     carry a doa_geometry (see below).
 *   - Argument errors are reported synchronously by the return value and enqueue nothing.
 *     Launch failures return DOA_ECUDA. Numerical problems found on the device (no
 *     convergence, rank loss, non-finite data) are written to the caller's `info`/`status`
 *     words; kernels never trap.
 *   - Sizes: 2 <= M <= 64, 0 <= d < M, N >= 1, 3 <= L <= 2^30.
 */
#ifndef DOA_H
#define DOA_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  DOA_OK = 0,
  DOA_EINVAL = 1,      /* bad argument (size, null or misaligned pointer, unknown enum)     */
  DOA_ENOMEM = 2,      /* caller-provided workspace, or the library's own scratch, too small */
  DOA_ECUDA = 3,       /* a CUDA launch or runtime call failed                               */
  DOA_ENOCONV = 4,     /* Jacobi sweep cap reached                                           */
  DOA_ERANK = 5,       /* EV with a non-positive noise eigenvalue, MN with e1^H P_n e1 == 0 */
  DOA_ENONFINITE = 6,  /* NaN or Inf in the covariance                                       */
  DOA_ETIMEOUT = 7     /* reserved: a bounded device wait ran out                            */
} doa_status;

typedef enum { DOA_PHD = 0, DOA_MUSIC = 1, DOA_EV = 2, DOA_MN = 3 } doa_alg;

/* Arithmetic of the Jacobi eigensolver (the batch's eig_prec; doa_noise_subspace_prec). GB300
 * issues FP64 at about 1/64 of its FP32 rate, so DOA_EIG_DOUBLE_FLOAT runs the same rotations in
 * double-float arithmetic (pairs of FP32 numbers, ~48 significant bits) on the FP32 pipe;
 * DOA_EIG_FP64 runs them in FP64. In the batch the noise eigenvectors are then checked for
 * orthonormality in FP64 (max |E_n^H E_n - I| <= 1e-10, else the problem's status is
 * DOA_ENOCONV). */
typedef enum { DOA_EIG_DOUBLE_FLOAT = 0, DOA_EIG_FP64 = 1 } doa_eig_prec;

/* Arithmetic of the covariance and scan contractions. */
typedef enum {
  DOA_FP32 = 0,    /* FP32 operands, FP32 FMA on CUDA cores                                   */
  DOA_BF16 = 1,    /* one BF16 tensor-core product, FP32 accumulation                        */
  DOA_BF16X3 = 2,  /* BF16 hi+lo split operands, three tensor-core products, FP32 accumulation */
  DOA_FP16X3 = 3   /* FP16 hi+lo split operands, three tensor-core products, FP32 accumulation */
} doa_prec;

/* Scan grid theta_k = lo_deg + k*step_deg (degrees, FP64), k = 0..L-1. */
typedef struct {
  double lo_deg;
  double step_deg;
  int32_t L;
  int32_t reserved;
} doa_grid;

/*
 * Array geometry and elevation grid of a 2-D (azimuth x elevation) scan with the steering vector
 * of Eq. 2 as printed:
 *   a_m(theta, phi) = exp{ j 2 pi (x_m sin(theta) sin(phi) + y_m cos(theta) sin(phi) + z_m cos(phi)) }
 * theta = azimuth (the columns: a doa_grid of La points), phi = the elevation angle of Eq. 2 (the
 * rows: phi_l = el_lo_deg + l * el_step_deg, l < Le; phi = 90 deg is the plane z = 0, where
 * Sec. 5.1 takes its accuracy scans). Positions (x_m, y_m, z_m) are in wavelengths. The spectrum
 * is Le x La row-major (flat index l * La + k); peaks are reported as flat indices.
 *   pos      : DEVICE pointer to M x 3 finite doubles (x_m, y_m, z_m), element by element; NULL in
 *              a batch problem means the 1-D half-wavelength ULA scan. 8-byte aligned.
 *   wrap_az  : 1 if the azimuth grid closes the circle (its first and last columns are
 *              neighbours for peak finding), else 0.
 *   Sizes    : 1 <= La, Le <= 2^24, La * Le <= 2^30.
 */
typedef struct {
  const double *pos;
  double el_lo_deg;
  double el_step_deg;
  int32_t Le;
  int32_t wrap_az;
} doa_geometry;

/* Human-readable name of a status code (static string, never NULL). */
const char *doa_status_str(int status);

/*
 * Step-1 (Eq. 3): R = (1/N) * sum_t X(t_t) X(t_t)^H.
 *   X    : M x N complex64, row-major: row m is the time series of element m; row stride
 *          ldx >= N complex elements. 8-byte aligned.
 *   R    : M x M complex64 row-major (nullable).
 *   R64  : M x M complex128 row-major (nullable). At least one of R, R64 is non-NULL.
 *   prec : DOA_FP32: exact FP32 products (FMA) accumulated in double-float within ranges of
 *          snapshots, ranges combined in FP64 (a cluster of up to 8 CTAs, reduced through
 *          distributed shared memory); about 2^-44 relative error.
 *          DOA_BF16 / DOA_BF16X3 / DOA_FP16X3: one real tcgen05 GEMM [Y; Z] Y^T fed by TMA
 *          (Y = X as reals, Z = pairs (re, im) -> (im, -re)) with BF16 or split hi+lo operands
 *          and FP32 accumulation (about 2^-8, 2^-16, 2^-22 relative per product); these need a
 *          16-byte aligned X and an even ldx.
 * Errors: DOA_EINVAL for M outside [2, 64], N < 1, ldx < N, NULL X, both outputs NULL.
 */
doa_status doa_covariance(const float *X, int M, int N, int ldx, float *R, double *R64, int prec,
                          void *stream);

/*
 * Covariance for callers that cannot allocate: the accuracy of doa_covariance with DOA_FP32 (exact
 * FP32 products accumulated in compensated double-float, FP64 sums, about 2^-44 relative), with no
 * allocation and no caller workspace. It splits the snapshots into 1024-snapshot chunks added in
 * chunk order by a second kernel, where doa_covariance splits them over up to 8 cluster CTAs, so
 * the two agree to that accuracy, not bit for bit. The paper has no counterpart.
 *   Who needs it: code that must not call cudaMalloc once running -- a fixed-memory real-time
 *   processing loop (cudaMalloc can synchronise the device and take driver locks), a host
 *   framework that forbids allocation after start-up, or a caller without its own allocator.
 *   Scratch: a library-owned device array of DOA_NOALLOC_SCRATCH_BYTES (4 MiB), resident on
 *   every GPU that loads the library until the process exits. A call needs
 *   ceil(N / 1024) * M * M * 16 bytes of it (M = 64: N <= 65536); larger problems return
 *   DOA_ENOMEM and enqueue nothing. Nothing in it needs to start at zero.
 *   Sharing: all calls on a device use the same array, so calls that overlap on one GPU (other
 *   streams or host threads) race on it; the caller must serialise them.
 *   First call per device: looks up the array's device address (cudaGetSymbolAddress, with that
 *   device current) and sets the kernel's shared-memory limit. Make that first call before any
 *   stream capture.
 *   Arguments and other errors: as doa_covariance (no prec argument: always DOA_FP32).
 */
#define DOA_NOALLOC_SCRATCH_BYTES (4u << 20)
doa_status doa_covariance_noalloc(const float *X, int M, int N, int ldx, float *R, double *R64,
                                  void *stream);

/*
 * Steps 2-4: Hermitian eigendecomposition of R by FP64 cyclic Jacobi (one warp per matrix,
 * parallel round-robin ordering), eigenvalues sorted descending (equal values keep their
 * index order), then the noise-subspace factor B of the weighting matrix, C = B B^H (Table 3):
 *   PHD   : B = e_min (last eigenvector),                K = 1
 *   MUSIC : B = E_n = eigenvectors d..M-1,               K = M - d
 *   EV    : B = E_n diag(lambda_i^{-1/2}),               K = M - d
 *   MN    : B = valph = P_n e1 / (e1^H P_n e1),          K = 1
 *   R64   : M x M complex128 row-major (Hermitian; only the upper triangle is read).
 *   evals : M doubles, descending (nullable).
 *   B     : M x K complex128, column-major with leading dimension M (capacity M*M).
 *   K_out : one int32 receiving K (nullable).
 *   info  : one int32: > 0 number of sweeps; < 0 minus a doa_status (ENOCONV, ERANK,
 *           ENONFINITE). Never NULL.
 */
doa_status doa_noise_subspace(const double *R64, int M, int d, int alg, double *evals, double *B,
                              int *K_out, int *info, void *stream);

/* doa_noise_subspace with the Jacobi's arithmetic chosen (doa_eig_prec): doa_noise_subspace is
 * this call with DOA_EIG_FP64. With DOA_EIG_DOUBLE_FLOAT the rotations run until no pair has
 * |a_pq| > 1e-12 sqrt(|a_pp a_qq|), the converged A and V are rounded to FP64 and sorted, and the
 * factor is formed in FP64 as for the FP64 form. For M > 32 the FP64 form runs one 512-thread CTA
 * per matrix (the element updates of every round spread over all its threads); the double-float
 * form runs a cluster of four 512-thread CTAs (about 200 KB of shared memory each, one per SM),
 * each owning 16 rows of A and V, with results identical to the one-CTA form. DOA_EINVAL also for
 * an unknown eig_prec. */
doa_status doa_noise_subspace_prec(const double *R64, int M, int d, int alg, int eig_prec, double *evals,
                                   double *B, int *K_out, int *info, void *stream);

/*
 * Step-5: P_k = 1 / ||B^H a(theta_k)||^2 for k = 0..L-1 (equal to 1/(a^H C a) with C = B B^H).
 *   B    : M x K complex128 column-major, leading dimension M (as written by
 *          doa_noise_subspace). 1 <= K <= M.
 *   grid : scan grid; L >= 3.
 *   prec : DOA_FP32: CUDA-core FFMA; phases exact to 2^-31 of a half turn; points whose
 *          denominator is small are re-evaluated in FP64 (warp per point).
 *          DOA_BF16 / DOA_BF16X3 / DOA_FP16X3: tcgen05 GEMM of the generated steering block
 *          against the real embedding of B (one BF16 product, or split hi+lo operands with three
 *          products); for the split forms the points below the split's error threshold are
 *          re-evaluated in FP32 and then FP64, so they meet the FP32 tolerance.
 *   P    : L floats, 4-byte aligned. The call first writes the grid's phase table into P and
 *          then overwrites it with the spectrum, so P needs no companion buffer.
 */
doa_status doa_scan(const double *B, int M, int K, doa_grid grid, int prec, float *P, void *stream);

/*
 * Step-6: peaks of P (left end of each strict local-maximum plateau, end points excluded),
 * the d largest (equal values: lower index first), written in ascending index order.
 *   idx, val : d entries each (entries past *count are left untouched); count: one int32.
 */
doa_status doa_peaks(const float *P, int L, int d, int *idx, float *val, int *count, void *stream);

/*
 * Step-5 for an arbitrary geometry on an azimuth x elevation grid (Eq. 2 as printed):
 * P[l * La + k] = 1 / ||B^H a(theta_k, phi_l)||^2.
 *   B     : M x K complex128 column-major, ld M, as for doa_scan. 1 <= K <= M.
 *   az    : azimuth grid (La = az.L >= 1 columns); geom: positions and elevation rows (pos != NULL).
 *   P     : La * Le floats, 4-byte aligned.
 *   ws    : device scratch of doa_scan_geometry_ws_bytes(La, Le) bytes (24 per azimuth and per
 *           elevation row), 16-byte aligned; it receives the grid's sin / cos tables (DOA_ENOMEM if
 *           ws_bytes is smaller).
 * FP32 on CUDA cores: sin and cos of every grid angle evaluated once in FP64 and rounded, phases
 * t_m = p_m . u in turns from the positions relative to their centroid (a common phase, which
 * leaves ||B^H a|| unchanged), phasors from the fraction of t_m as a 32-bit phase. Points whose
 * denominator falls below a threshold derived from the geometry's phase-error bound are
 * re-evaluated in FP64 (warp per point).
 */
size_t doa_scan_geometry_ws_bytes(int La, int Le);
doa_status doa_scan_geometry(const double *B, int M, int K, doa_grid az, doa_geometry geom, float *P, void *ws,
                             size_t ws_bytes, void *stream);

/*
 * Step-6 on an Le x La azimuth x elevation spectrum: a peak is a point strictly larger than each
 * of its (up to 8) neighbours, rows outside the grid absent, columns wrapping when wrap_az; the d
 * largest (equal values: lower flat index first), written as flat indices in ascending order.
 *   idx, val : d entries each; count: one int32. 0 <= d < 64.
 */
doa_status doa_peaks2d(const float *P, int La, int Le, int wrap_az, int d, int *idx, float *val, int *count,
                       void *stream);

/*
 * Model-order estimation (Table 2 takes D as given; these are Wax and Kailath's information
 * criteria for complex data): for k = 0..M-1 assumed sources, with a and g the arithmetic and
 * geometric means of the M-k smallest eigenvalues,
 *   L(k) = N (M-k) log(a/g)  (+inf when one of them is not positive),
 *   MDL(k) = L(k) + k (2M-k) log(N) / 2,   AIC(k) = 2 L(k) + 2 k (2M-k);
 * *mdl and *aic receive the argmin (the smaller k on a tie), in FP64.
 *   evals : M device doubles, descending (as written by doa_noise_subspace); N: snapshots.
 *   mdl, aic : device int32 (either may be NULL).
 */
doa_status doa_model_order(const double *evals, int M, int N, int *mdl, int *aic, void *stream);

/*
 * Step-2 of Table 2 as an SVD of the snapshot matrix X itself (the paper's Step-2 is a Jacobi SVD,
 * Sec. 4.2), R = X X^H / N never formed: one-sided Jacobi (Hestenes) on the M rows of X. Rows
 * y_p, y_q are rotated, Y <- J^H Y and U <- U J, by the Hermitian Jacobi rotation of
 * doa_noise_subspace built from alpha = ||y_p||^2, beta = ||y_q||^2, gamma = y_p y_q^H; pairs in
 * row-cyclic order; a pair is rotated when |gamma| > tol sqrt(alpha beta) and neither row is
 * numerically zero (squared norm above 1e-30 of the largest: rank-deficient X, N < M); the
 * iteration stops after the first sweep that rotates nothing. Then X = U S V^H, and the eigenvalues of R are
 * S_k^2 / N with eigenvectors the columns of U. Small singular values keep their relative
 * accuracy (R's eigenvalues below ~1e-16 of the largest do not).
 * GPU form: the rows live in an FP64 copy Y of X in ws; each sweep is one pass over Y on all SMs
 * that applies the previous sweep's rotations and forms the Gram matrix Y Y^H in FP64, then the
 * sweep's rotations run on that Gram matrix in one CTA (its pair entries are the rotated Gram
 * entries, formed afresh from the rows once per sweep).
 *   X          : M x N snapshots, row-major with row stride ldx (>= N) elements: complex64
 *                (x_c128 = 0, 8-byte aligned) or complex128 (x_c128 = 1, 16-byte aligned).
 *   tol        : rotation threshold (> 0; 1e-15 is the usual choice). max_sweeps: 1..1000.
 *   evals      : M device doubles, descending (equal values in index order).
 *   U          : M x M complex128, column-major (ld M): column k is the singular vector of evals[k].
 *   info       : one device int32: the sweep count, or -DOA_ENOCONV when max_sweeps sweeps still
 *                rotated (outputs then hold the last sweep's Gram diagonal and rotations).
 *   ws         : device scratch of doa_svd_data_ws_bytes(M, N) bytes, 16-byte aligned (about
 *                16 M N bytes: the FP64 rows, plus the partial Gram matrices); DOA_ENOMEM if
 *                ws_bytes is smaller. The call enqueues 2 * max_sweeps kernels; those after
 *                convergence return at once.
 * Errors: DOA_EINVAL for M outside [2, 64], N < 1, ldx < N, a NULL or misaligned pointer, or a
 * bad tol / max_sweeps.
 */
size_t doa_svd_data_ws_bytes(int M, int N);
doa_status doa_svd_data(const void *X, int x_c128, int M, int N, int ldx, double tol, int max_sweeps,
                        double *evals, double *U, int *info, void *ws, size_t ws_bytes, void *stream);

/*
 * Root form of the ULA scan (root-MUSIC for the MUSIC factor; any factor B works the same way): on
 * |z| = 1, z = e^{j pi sin theta}, ||B^H a||^2 = sum_{l=-(M-1)}^{M-1} c_l z^l with
 * c_l = sum_k sum_n B_nk conj(B_{n+l,k}); the roots of the degree-(2M-2) polynomial z^{M-1} D(z)
 * pair up as z, 1/conj(z), and the d roots with |z| <= 1 closest to the unit circle give
 * theta = asin(arg(z) / pi). Roots by the Aberth-Ehrlich iteration in FP64 (converged when every
 * correction is below 1e-14 max(1, |z|), 400 iterations at most).
 *   B, M, K : as for doa_scan.  d: 1 <= d < M.  theta: d device doubles (ascending, degrees; NaN
 *   when the iteration fails).  info: device int32, 0 or -DOA_ENOCONV.
 */
doa_status doa_root_music(const double *B, int M, int K, int d, double *theta, int *info, void *stream);

/*
 * Sub-grid refinement of picked peaks (beyond Step-6, which stops at the grid): for each peak the
 * local minimiser, in FP64, of den = ||B^H a||^2 (= a^H C a) next to it.
 *   ULA: bracketed Newton on den'(theta) = 0 inside [theta_{k-1}, theta_{k+1}] (steps shrink the
 *        bracket by the sign of den'; Newton point inside the bracket, else its midpoint; stop
 *        below a 1e-13 rad move, 60 steps at most). theta: count angles in degrees.
 *   2-D (doa_refine_peaks2d, Eq. 2 as printed): damped Newton in (azimuth, elevation) inside the
 *        box of one grid step around the peak (Newton step when the Hessian is positive definite,
 *        else steepest descent scaled to the box; halving until den does not increase; Newton
 *        steps below 1e-6 rad taken as they are). out: count (azimuth, elevation) pairs, degrees.
 *   B, M, K : factor as for doa_scan / doa_scan_geometry (all K columns, unweighted).
 *   idx     : device peak indices (as written by doa_peaks / doa_peaks2d); count: device int32
 *             number of peaks; cap: capacity of idx / the output (min(*count, cap) are refined).
 * Batch problems get the same per algorithm (its readout's columns and weights) through
 * doa_problem.peak_angle.
 */
doa_status doa_refine_peaks(const double *B, int M, int K, doa_grid grid, const int *idx, const int *count,
                            int cap, double *theta, void *stream);
doa_status doa_refine_peaks2d(const double *B, int M, int K, doa_grid az, doa_geometry geom, const int *idx,
                              const int *count, int cap, double *out, void *stream);

/* ----------------------------------------------------------------------------------------- */
/* Measurement utility (not in the paper)                                                      */
/* ----------------------------------------------------------------------------------------- */

/*
 * FMA issue-rate probe: `blocks` CTAs of 256 threads, each thread 8 independent chains of `iters`
 * dependent FMAs: mode (fp64) 0 = FP32 FFMA, 1 = FP64 DFMA, 2 = paired FP32 (fma.rn.f32x2, two FMAs
 * per instruction); *flops (host) receives the flop count of the launch (2 per FMA). out: device
 * buffer of blocks x 256 floats (doubles for mode 1), the chain sums. The caller times the launch
 * (events on `stream`) to get FLOP/s.
 */
doa_status doa_probe_fma(int fp64, int blocks, int iters, void *out, double *flops, void *stream);

/* ----------------------------------------------------------------------------------------- */
/* Grid slices (not in the paper): one spectrum split into contiguous slices of the angle grid, */
/* e.g. one slice per GPU, with B replicated. The slice scan computes exactly the points the    */
/* full scan computes; the slice peak summary plus a host merge of the summaries of all slices  */
/* reproduces doa_peaks on the whole spectrum bit for bit.                                     */
/* ----------------------------------------------------------------------------------------- */

/*
 * Step-5 on the global grid points k0 .. k0+n-1 of `grid` (0 <= k0, n >= 1, k0 + n <= L): P[i]
 * receives the value doa_scan would write at k0 + i (same phases, same FP64 re-evaluation).
 * DOA_FP32 only. P: n floats; as with doa_scan the phase table is staged in P first.
 */
doa_status doa_scan_slice(const double *B, int M, int K, doa_grid grid, int k0, int n, float *P, void *stream);

/* Peak summary of one slice of a spectrum (written by doa_slice_peaks, read by the host merge). */
#define DOA_SLICE_MAXD 64
typedef struct {
  int32_t count;                  /* decided peaks of the slice in idx/val (<= d)                 */
  int32_t open_idx;               /* left end of a run that reaches the end of the slice's data   */
                                  /* with equal values (undecided), or -1                         */
  float open_val;
  float first_val;                /* P[k0]                                                          */
  int32_t first_run_to_end;       /* 1 if P[k0] .. P[last readable] are all equal                  */
  float first_next_val;           /* otherwise the first value after that run                      */
  int32_t idx[DOA_SLICE_MAXD];    /* global indices, best first (value descending, index ascending) */
  float val[DOA_SLICE_MAXD];
} doa_slice_summary;

/*
 * Step-6 on one slice. The slice owns global points [k0, k1) of a spectrum of L points; Pbuf holds
 * the points [b0, b1) with b0 = max(k0 - 1, 0) and b1 = min(k1 + 1, L) (one halo point on each
 * side that exists), Pbuf[0] being global index b0. A peak is decided with the rule of doa_peaks
 * (left end i of a maximal run of equal values, strictly lower on both sides, 1 <= i and run
 * end <= L-2) using only those points; a run that starts at an owned point and is still equal at
 * b1 - 1 < L - 1 is reported as the open candidate, to be decided by the merge from the next
 * slices' first_* fields. The d best decided peaks are kept (0 <= d <= DOA_SLICE_MAXD).
 *   out: one doa_slice_summary in device memory.
 */
doa_status doa_slice_peaks(const float *Pbuf, int b0, int k0, int k1, int L, int d, doa_slice_summary *out,
                           void *stream);

/*
 * Host-only merge of the summaries of all slices of one spectrum, given in slice order (for
 * slices split across GPUs: after an all-gather of the summaries). Decides every open candidate
 * from the first_* fields of the following slices (the run ends with a strict descent: peak; it
 * rises or reaches the last point: no peak), then keeps the d best peaks (value descending,
 * index ascending) and writes them in ascending index order, exactly as doa_peaks would.
 *   sums: nslices host summaries; idx, val: d host entries each; count: one host int32.
 * Errors: DOA_EINVAL for bad arguments or summaries that do not chain (an open run whose value
 * differs from the next slice's first value).
 */
doa_status doa_merge_slices(const doa_slice_summary *sums, int nslices, int d, int32_t *idx, float *val,
                            int32_t *count);

/* ----------------------------------------------------------------------------------------- */
/* Batched solve (not in the paper): many independent problems with uneven M, d, N, L and    */
/* algorithms in one plan, executed as a fixed sequence of kernels on one stream that a       */
/* caller may capture into a CUDA graph.                                                      */
/* ----------------------------------------------------------------------------------------- */

/* One problem of a batch. All pointers are device pointers owned by the caller. */
typedef struct {
  const float *X;        /* M x N complex64 row-major, row stride ldx                        */
  float *P;              /* nalg x L spectra (nalg = popcount(alg_mask), in bit order)       */
  int32_t *peak_idx;     /* nalg x d peak indices (ascending per algorithm)                  */
  float *peak_val;       /* nalg x d peak values                                             */
  int32_t *peak_count;   /* nalg counts                                                      */
  double *evals;         /* M eigenvalues, descending (nullable)                             */
  doa_grid grid;
  int32_t M, N, ldx, d;
  uint32_t alg_mask;     /* bit a set => algorithm a (DOA_PHD=bit 0 ... DOA_MN=bit 3)        */
  int32_t prec;          /* doa_prec of the covariance and scan                              */
  float *features;       /* nullable: M(M+1) floats, the upper triangle (row by row, i <= j)  */
                         /* of R / tr(R) as (re, im) pairs (the proposal network's input)     */
  double *B_out;         /* nullable: copy of the factor B of the first algorithm in          */
                         /* alg_mask (M x K complex128, column-major, ld M)                   */
  int32_t eig_prec;      /* doa_eig_prec of the batch's Jacobi                                */
  int32_t flags;         /* DOA_FLAG_* bits                                                   */
  doa_geometry geom;     /* geom.pos == NULL: the 1-D ULA scan over `grid`. Otherwise a 2-D   */
                         /* scan, `grid` the azimuth columns: P holds nalg x (Le x La) floats, */
                         /* peaks are flat indices, prec must be DOA_FP32 and flags 0.         */
                         /* Problems that pass the same geom.pos pointer with the same grid    */
                         /* and M share one FP32 steering table in the workspace (written once */
                         /* per solve; pass one pointer for one physical array)                */
  double *peak_angle;    /* nullable: sub-grid refined peak angles in degrees (see            */
                         /* doa_refine_peaks): nalg x d (ULA) or nalg x d x 2 (geometry:       */
                         /* azimuth, elevation), entries past peak_count untouched             */
  int32_t *order_est;    /* nullable: 2 int32, the MDL and AIC source-count estimates from     */
                         /* the eigenvalues (see doa_model_order); d itself stays as given     */
  double *root_angle;    /* nullable, ULA problems only: nalg x d angles (degrees, ascending)   */
                         /* from the roots of the scan's polynomial (see doa_root_music);      */
                         /* status DOA_ENOCONV (angles NaN) if the root iteration fails        */
} doa_problem;

/* Peak polish: after Step-6 the spectrum is re-evaluated in FP64 (steering and contraction) at
 * the picked peaks and their two neighbours on each side, and the peaks are picked again, so a
 * near tie between neighbouring grid points is decided as the FP64 spectrum decides it. A peak
 * whose outcome the FP32 values already decide (every consecutive pair from k-3 to k+3 differs by
 * more than 2e-3 relative, four times the FP32 path's error bound, and so does the algorithm's
 * weakest selected peak from its best unselected one) is left as computed. */
#define DOA_FLAG_POLISH_PEAKS 1

/* Covariance arithmetic of a batch problem. Problems with M <= 16, a 16-byte aligned X, an even
 * ldx and N <= 2^21 compute R on the tensor cores by default: every sample is scaled by one power
 * of two and cut into six 7-bit slices (exact in BF16), every slice product and every window of
 * 960 snapshots of their sums is exact in the FP32 accumulators, and the windows are added in
 * 64-bit integers, so R is exact to about 2^-40 of the largest sample magnitude squared and does
 * not depend on the order of the additions. This flag selects the compensated CUDA-core
 * accumulation instead (the form every other problem uses). */
#define DOA_FLAG_COV_CUDA_CORE 2

/* Launch-shape knobs of a plan, per M bucket (M <= 8, <= 16, <= 32, <= 64); 0 = default. */
typedef struct {
  int32_t scan_pt[4];    /* grid points per scan thread (tile = 128 threads x scan_pt points).  */
                         /* Allowed {1, 2, 4}, {1, 2, 4}, {1, 2}, {1} (the register budget of   */
                         /* the in-register phasors); default (4, 2, 1, 1).                     */
  int32_t eig_mats[4];   /* matrices per Jacobi warp. Allowed {1, 2, 4, 8}, {1, 2, 4}, {1, 2},   */
                         /* {1} (a lane per rotation pair); default: 1 unless the bucket holds   */
                         /* enough problems to keep ~24 packed warps per SM busy.               */
  int32_t scan_group[4]; /* FP32 ULA problems that share a grid are scanned together in groups  */
                         /* of this many (one steering generation per tile of the grid for the   */
                         /* whole group, each problem's factor contracted in turn); 1 scans every */
                         /* problem alone. Allowed powers of two 1..32; default 32.              */
} doa_tuning;

/*
 * Host-only planning. doa_batch_plan_bytes returns the plan size for these problems (0 if one
 * is invalid). doa_batch_plan packs the problems into `plan` (caller host memory of at least
 * that size) and returns the device workspace size in *ws_bytes.
 * tuning: NULL (defaults) or the launch shapes above; these are the autotuner's knobs and do
 * not change any result bit.
 * The caller copies the same plan bytes to device memory (16-byte aligned) before
 * doa_solve_batch. Errors: DOA_EINVAL for an invalid problem (its index in *bad_index if
 * bad_index is not NULL) or a tuning value outside the allowed sets, DOA_ENOMEM if plan_bytes
 * is too small.
 */
size_t doa_batch_plan_bytes(const doa_problem *probs, int nprob);
doa_status doa_batch_plan(const doa_problem *probs, int nprob, const doa_tuning *tuning, void *plan,
                          size_t plan_bytes, size_t *ws_bytes, int *bad_index);

/* Stages of doa_solve_batch, in launch order (for per-stage timing). */
#define DOA_BATCH_STAGES 5 /* 0 phase tables, 1 covariance, 2 eig + noise subspace, 3 scan, 4 peaks */

/*
 * Executes a plan: covariance, eigendecomposition + noise subspace, scan and peaks for every
 * problem and algorithm. Only prec == DOA_FP32 problems are accepted by this version.
 *   plan_host, plan_dev : the same plan bytes on the host and in device memory (16-byte aligned).
 *   ws      : device memory of at least the planned size, 256-byte aligned. Its contents need
 *             no initialisation and are overwritten.
 *   status  : one int32 per problem: 0, or a doa_status found on the device.
 *   stage_events : NULL, or DOA_BATCH_STAGES + 1 cudaEvent_t handles; event i is recorded on
 *             `stream` before stage i and the last one after the final stage (the per-stage time
 *             breakdown of the method, cf. the paper's Fig. 2).
 * The call reads only plan_host on the host and enqueues a fixed sequence of kernels, so a
 * stream capture of it replays as a CUDA graph.
 */
doa_status doa_solve_batch(const void *plan_host, const void *plan_dev, void *ws, size_t ws_bytes,
                           int *status, void *const *stage_events, void *stream);

/* ----------------------------------------------------------------------------------------- */
/* Learned angle proposal (not in the paper): a multilayer perceptron that maps the             */
/* trace-normalised upper triangle of R (136 complex = 272 reals, doa_problem.features) to a     */
/* 181-bin (1 degree, -90..90) occupancy map, so the fine scan runs only in windows around the   */
/* proposed angles. Layers 272 -> 256 -> 256 -> 256 -> 181, ReLU hidden, sigmoid output,        */
/* binary cross-entropy on logits, Adam. FP32 master weights; the products run as BF16 tcgen05  */
/* GEMMs (TMA-fed) with FP32 accumulation.                                                       */
/* ----------------------------------------------------------------------------------------- */
#define DOA_MLP_IN 272
#define DOA_MLP_HIDDEN 256
#define DOA_MLP_OUT 181

/* Device buffers of the network, layer l = 0..3 with (in, out) = (272,256), (256,256),
 * (256,256), (256,181). W[l] is out x in row-major FP32, b[l] out FP32; mW/vW/mb/vb are the Adam
 * moments and gW/gb the gradients (same shapes; only needed for training). Wh[l] is the BF16
 * copy of W[l] (row pitch in), WhT[l] its transpose (in x out, row pitch out rounded up to 8). */
typedef struct {
  float *W[4], *b[4];
  float *mW[4], *vW[4], *mb[4], *vb[4];
  float *gW[4], *gb[4];
  void *Wh[4], *WhT[4];
} doa_mlp;

/* Workspace of a forward/backward pass on `batch` rows (a multiple of 8); 0 if invalid. */
size_t doa_mlp_workspace_bytes(int batch);

/* Writes the BF16 copies Wh/WhT from the FP32 masters W (after initialisation). */
doa_status doa_mlp_refresh(const doa_mlp *net, void *stream);

/* features: batch x 272 FP32. probs (nullable): batch x 181 sigmoid outputs; logits (nullable):
 * batch x 181. ws: doa_mlp_workspace_bytes(batch) bytes, 256-byte aligned. */
doa_status doa_mlp_forward(const doa_mlp *net, const float *features, int batch, float *probs,
                           float *logits, void *ws, size_t ws_bytes, void *stream);

/* Forward + backward on one minibatch: fills gW/gb with the gradient of the mean (over rows)
 * summed binary cross-entropy against labels (batch x 181, in [0, 1]); loss (nullable device
 * float) receives that mean. */
doa_status doa_mlp_backward(const doa_mlp *net, const float *features, const float *labels,
                            int batch, float *loss, void *ws, size_t ws_bytes, void *stream);

/* One Adam step (Kingma & Ba) on every parameter with bias corrections for step t >= 1, then
 * refreshes the BF16 copies. */
doa_status doa_mlp_adam(const doa_mlp *net, float lr, float beta1, float beta2, float eps, int t,
                        void *stream);

/*
 * Seeded ULA snapshots generated on the GPU (training data of the proposal network; the signal
 * model of Sec. 3.1, Eq. 1): X_b = A(theta_b) S_b + W_b with unit-power CN(0,1) sources and white
 * CN(0, sigma_b^2) noise, sigma_b^2 = 10^(-snr_db[b]/10). Random numbers: Philox4x32-10 (Salmon et
 * al., SC'11) with key = seed and counter = (snapshot, instance, instance >> 32, draw), instance =
 * first_instance + b; normals by Box-Muller. The per-instance source count d[b] <= 16, angles
 * (degrees, row b holds d[b] of dmax entries) and SNR are device inputs.
 *   X: batch x M x N complex64 (row-major per instance). M <= 64.
 */
doa_status doa_synth_ula(int batch, int M, int N, const int32_t *d, const float *angles_deg, int dmax,
                         const float *snr_db, uint64_t seed, uint64_t first_instance, float *X,
                         void *stream);

/*
 * Proposal decoding: for each row b of probs (batch x 181 sigmoid outputs of 1-degree bins centred
 * at -90, -89, ..., 90 deg), the min(d[b] + extra, dmax) highest bins (ties: lower bin) with the
 * two neighbours of every pick suppressed; pick w becomes a window of `width` points of the fine
 * grid starting at win_first[b*dmax + w] (the grid index of the bin centre minus width/2, clamped
 * into the grid); unused entries are -1. dmax <= 8.
 */
doa_status doa_proposal_windows(const float *probs, const int32_t *d, int batch, int dmax, int extra,
                                doa_grid fine, int width, int32_t *win_first, void *stream);

/*
 * Windowed fine scan (FP32 path with FP64 near-null refinement, M <= 16) and merged peaks.
 *   B: batch x (M*M) complex128 factors (row b: M x K[b], column-major, ld M), e.g. from
 *      doa_problem.B_out. rows: NULL (rows 0..nrows-1) or nrows row indices.
 *   full = 0: row b scans its windows [win_first[b*dmax+w], +width) of `fine`; full = 1: row b
 *      scans the whole grid (the fallback and the plain full-grid method).
 *   S: L uint32 scratch (phase table); Pwin: nrows x (full ? 1 : dmax) x (full ? L : width) floats
 *      scratch (the window spectra, readable afterwards).
 *   Peaks: interior local maxima of each window (the plateau rule of doa_peaks inside the window),
 *      duplicates from overlapping windows merged, the d[b] largest (ties: lower index) written to
 *      idx/val[b*dmax ..] as fine-grid indices in ascending order, count[b]. fallback[b]
 *      (nullable) = 1 when fewer than d[b] peaks were found, or a window's maximum lies on its
 *      first or last point with a value above the weakest selected peak (the spectrum rises
 *      beyond the window above the d-th peak); the caller then rescans row b with full = 1.
 */
doa_status doa_scan_windows(const double *B, int M, const int32_t *K, const int32_t *d, const int32_t *rows,
                            int nrows, int dmax, doa_grid fine, const int32_t *win_first, int width, int full,
                            uint32_t *S, float *Pwin, int32_t *idx, float *val, int32_t *count,
                            int32_t *fallback, void *stream);

/*
 * Judge of the learned proposal against the plain full-grid method. Every local maximum of the
 * row's coarse full-grid spectrum Pc (the plain MUSIC scan on `coarse`, e.g. 0.1 deg, computed for
 * the whole batch) marks where a fine-grid peak can lie; where no learned window covers the fine
 * points within jwidth / 2 of it, a judge window of jwidth fine points centred on it is scanned
 * (the same points, bit for bit, as the full fine-grid scan). fallback[b] is set to 1 (never
 * cleared) when the row has fewer than d[b] selected peaks, more than 16 uncovered maxima, or a
 * judge-window point at least as high as its weakest selected peak: then a full-grid peak at least
 * that high lies outside every learned window and the row must be rescanned on the full grid.
 *   B, M, K, d : factors as for doa_scan_windows (M <= 16), batch rows.
 *   Pc         : batch x coarse.L floats.  win_first, dmax, width: the learned windows.
 *   val, count : the windowed peaks (batch x dmax values, batch counts) from doa_scan_windows.
 *   judge_first: batch x 16 int32 (written: judge window starts, -1 unused).
 *   S          : fine.L uint32 scratch;  Pjudge: batch x 16 x jwidth float scratch.
 */
doa_status doa_proposal_judge(const double *B, int M, const int32_t *K, const int32_t *d, int batch,
                              const float *Pc, doa_grid coarse, doa_grid fine, const int32_t *win_first,
                              int dmax, int width, const float *val, const int32_t *count, int jwidth,
                              int32_t *judge_first, uint32_t *S, float *Pjudge, int32_t *fallback,
                              void *stream);

#ifdef __cplusplus
}
#endif

#endif /* DOA_H */
