/*
 * FP64 CPU oracle for noise-subspace narrowband DOA estimation (PHD, MUSIC, EV, MN).
 *
 * TEST INFRASTRUCTURE ONLY. This file is the plain, slow, obviously-correct statement of what
 * the GPU path computes. Only the test suite, the smoke check and the benchmark's CPU-baseline
 * leg may load it. It shares no code, header, table or constant with the CUDA library; the two
 * are written independently from the paper (Eray & Temizel, "Performance Analysis of Noise
 * Subspace-based Narrowband DOA Estimation Algorithms on CPU and GPU").
 *
 * Every step follows the paper in its own order and notation:
 *   Step-1  sample covariance                      Sec. 3.1, Eq. 3; Table 2 Step-1
 *   Step-2  Hermitian eigendecomposition of R      Table 2 Step-2 (SVD of a Hermitian PSD matrix
 *           = its eigendecomposition; singular values = eigenvalues, sorted descending)
 *   Step-3  noise subspace selection               Table 3 (Step-3 rows)
 *   Step-4  weighting matrix C (explicit M x M)    Table 3 (Step-4 rows)
 *   Step-5  pseudospectrum P = 1 / (a^H C a)       Table 2 Step-5, steering vector Eq. 2
 *   Step-6  peak finding and selection of D peaks  Table 2 Step-6
 *   Step-2 as an SVD of X itself (one-sided Jacobi on its rows, R never formed): oracle_svd_data
 *
 * Readings where the paper is silent (each one is listed in the design notes):
 *   - steering vector: Eq. 2 for a uniform linear array on the x axis with half-wavelength
 *     spacing, phi = 90 deg: a_m(theta) = exp(+j * pi * m * sin(theta)), m = 0..M-1,
 *     theta in degrees measured from broadside;
 *   - grid: theta_k = lo + k * step (one rounded multiply, one rounded add, no FMA);
 *   - PHD takes the last column after the descending sort (the minimum eigenvalue);
 *   - a peak is the left end i of a maximal plateau [i..j] with P[i-1] < P[i] and
 *     P[j+1] < P[j]; the end points 0 and L-1 are never peaks; the D largest are kept
 *     (ties to the lower index) and returned in ascending index order;
 *   - invP <= 0 gives P = +inf (exact-covariance self-tests only).
 *
 * Numbers are FP64 throughout; complex values use C99 `double complex`.
 * Compile with -ffp-contract=off so that every product and sum is rounded as written.
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORACLE_PI 3.14159265358979323846

enum { ORACLE_PHD = 0, ORACLE_MUSIC = 1, ORACLE_EV = 2, ORACLE_MN = 3 };
enum { ORACLE_OK = 0, ORACLE_EINVAL = 1, ORACLE_ENOCONV = 4, ORACLE_ERANK = 5 };

/* ---------------------------------------------------------------------------------------------
 * Step-1, Eq. 3:  R = (1/N) * sum_{k=1..N} X(t_k) X(t_k)^H.
 * X: M x N complex64, row-major, interleaved (re, im), row stride ldx complex elements.
 * R: M x M complex128, row-major, interleaved. Each float is promoted exactly to double.
 * ------------------------------------------------------------------------------------------- */
void oracle_covariance(const float *X, int M, int N, int ldx, double *R) {
  for (int a = 0; a < M; ++a) {
    for (int b = 0; b < M; ++b) {
      double complex acc = 0.0;
      for (int t = 0; t < N; ++t) {
        const float *xa = X + 2 * ((size_t)a * ldx + t);
        const float *xb = X + 2 * ((size_t)b * ldx + t);
        double complex va = (double)xa[0] + I * (double)xa[1];
        double complex vb = (double)xb[0] + I * (double)xb[1];
        acc += va * conj(vb);
      }
      acc /= (double)N;
      R[2 * (a * M + b)] = creal(acc);
      R[2 * (a * M + b) + 1] = cimag(acc);
    }
  }
}

/* ---------------------------------------------------------------------------------------------
 * Step-2: eigendecomposition of the Hermitian matrix R by the cyclic Jacobi method
 * (Jacobi 1846; Golub & Van Loan, Matrix Computations, Sec. 8.5, extended to complex
 * Hermitian matrices by a phase factor). Pairs are visited row by row, (0,1), (0,2), ...,
 * (M-2, M-1). A pair is rotated when |a_pq| > tol * sqrt(|a_pp a_qq|) (and a_pq != 0);
 * the iteration stops after the first sweep that rotates nothing.
 *
 * For the pair (p, q) with a_pq = |a_pq| e^{j phi}, the unitary rotation
 *     J = [[ c,            s e^{j phi} ],
 *          [ -s e^{-j phi}, c          ]]      (acting on coordinates p, q)
 * with tau = (a_qq - a_pp) / (2 |a_pq|), t = sgn(tau) / (|tau| + sqrt(1 + tau^2)),
 * c = 1 / sqrt(1 + t^2), s = t c, makes (J^H A J)_pq = 0.  A <- J^H A J, V <- V J.
 *
 * Output: evals[M] descending (stable: equal values keep their original order),
 * V: M x M complex128, column-major (column i = eigenvector of evals[i]), interleaved.
 * Returns the number of sweeps (>= 1), or -ORACLE_ENOCONV when max_sweeps is reached.
 * ------------------------------------------------------------------------------------------- */
int oracle_eigh(const double *R, int M, double tol, int max_sweeps, double *evals, double *V) {
  double complex *A = (double complex *)malloc(sizeof(double complex) * M * M);
  double complex *W = (double complex *)malloc(sizeof(double complex) * M * M);
  for (int i = 0; i < M; ++i)
    for (int j = 0; j < M; ++j) {
      A[i * M + j] = R[2 * (i * M + j)] + I * R[2 * (i * M + j) + 1];
      W[i * M + j] = (i == j) ? 1.0 : 0.0; /* W is row-major here: W[i*M + j] = V(i, j) */
    }
  int sweeps = 0, converged = 0;
  while (sweeps < max_sweeps) {
    ++sweeps;
    int rotations = 0;
    for (int p = 0; p < M - 1; ++p) {
      for (int q = p + 1; q < M; ++q) {
        double complex apq = A[p * M + q];
        double mag = cabs(apq);
        double app = creal(A[p * M + p]), aqq = creal(A[q * M + q]);
        if (mag == 0.0 || mag <= tol * sqrt(fabs(app * aqq))) continue;
        ++rotations;
        double complex ph = apq / mag; /* e^{j phi} */
        double tau = (aqq - app) / (2.0 * mag);
        double t = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
        double c = 1.0 / sqrt(1.0 + t * t);
        double s = t * c;
        /* A <- A J : columns p and q */
        for (int r = 0; r < M; ++r) {
          double complex xp = A[r * M + p], xq = A[r * M + q];
          A[r * M + p] = c * xp - s * conj(ph) * xq;
          A[r * M + q] = s * ph * xp + c * xq;
        }
        /* A <- J^H A : rows p and q */
        for (int k = 0; k < M; ++k) {
          double complex xp = A[p * M + k], xq = A[q * M + k];
          A[p * M + k] = c * xp - s * ph * xq;
          A[q * M + k] = s * conj(ph) * xp + c * xq;
        }
        /* the rotation annihilates a_pq; the diagonal of a Hermitian matrix is real */
        A[p * M + q] = 0.0;
        A[q * M + p] = 0.0;
        A[p * M + p] = creal(A[p * M + p]);
        A[q * M + q] = creal(A[q * M + q]);
        /* V <- V J */
        for (int r = 0; r < M; ++r) {
          double complex xp = W[r * M + p], xq = W[r * M + q];
          W[r * M + p] = c * xp - s * conj(ph) * xq;
          W[r * M + q] = s * ph * xp + c * xq;
        }
      }
    }
    if (rotations == 0) {
      converged = 1;
      break;
    }
  }
  /* stable descending sort of the eigenvalues (insertion sort on an index permutation) */
  int *order = (int *)malloc(sizeof(int) * M);
  for (int i = 0; i < M; ++i) order[i] = i;
  for (int i = 1; i < M; ++i) {
    int cur = order[i];
    double v = creal(A[cur * M + cur]);
    int j = i - 1;
    while (j >= 0 && creal(A[order[j] * M + order[j]]) < v) {
      order[j + 1] = order[j];
      --j;
    }
    order[j + 1] = cur;
  }
  for (int i = 0; i < M; ++i) {
    int src = order[i];
    evals[i] = creal(A[src * M + src]);
    for (int r = 0; r < M; ++r) {
      V[2 * (i * M + r)] = creal(W[r * M + src]);
      V[2 * (i * M + r) + 1] = cimag(W[r * M + src]);
    }
  }
  free(order);
  free(W);
  free(A);
  return converged ? sweeps : -ORACLE_ENOCONV;
}

/* ---------------------------------------------------------------------------------------------
 * Steps 3 and 4 (Table 3): noise subspace selection and the explicit weighting matrix C.
 * evals[M] descending, V column-major (as returned by oracle_eigh); D = number of sources.
 *   PHD   : e_min = column of the minimum eigenvalue;      C = e_min e_min^H
 *   MUSIC : E_n = columns D..M-1 (0-based);                C = E_n E_n^H
 *   EV    : E_{n,w} = E_n with column i scaled by 1/lambda_i;  C = E_{n,w} E_n^H
 *   MN    : P_n = E_n E_n^H, u = [1, 0, ..., 0]^T, lambda = (u^H P_n u)^{-1},
 *           valph = P_n lambda u;                          C = valph valph^H
 * C: M x M complex128 row-major interleaved. Returns ORACLE_OK, ORACLE_EINVAL or ORACLE_ERANK
 * (EV with a non-positive noise eigenvalue; MN with u^H P_n u == 0).
 * ------------------------------------------------------------------------------------------- */
int oracle_weighting(const double *evals, const double *V, int M, int D, int alg, double *C) {
  if (M < 1 || D < 0 || D >= M) return ORACLE_EINVAL;
  double complex *Vc = (double complex *)malloc(sizeof(double complex) * M * M);
  double complex *Cm = (double complex *)calloc((size_t)M * M, sizeof(double complex));
  for (int col = 0; col < M; ++col)
    for (int r = 0; r < M; ++r) Vc[col * M + r] = V[2 * (col * M + r)] + I * V[2 * (col * M + r) + 1];
#define VCOL(col, r) Vc[(col) * M + (r)]
  int status = ORACLE_OK;
  if (alg == ORACLE_PHD) {
    /* minIdx <- min(d.diag): the eigenvalues are sorted descending, so the minimum is last */
    int minIdx = M - 1;
    for (int i = 0; i < M; ++i)
      for (int k = 0; k < M; ++k) Cm[i * M + k] = VCOL(minIdx, i) * conj(VCOL(minIdx, k));
  } else if (alg == ORACLE_MUSIC) {
    for (int i = 0; i < M; ++i)
      for (int k = 0; k < M; ++k) {
        double complex acc = 0.0;
        for (int col = D; col < M; ++col) acc += VCOL(col, i) * conj(VCOL(col, k));
        Cm[i * M + k] = acc;
      }
  } else if (alg == ORACLE_EV) {
    for (int col = D; col < M; ++col)
      if (!(evals[col] > 0.0)) status = ORACLE_ERANK;
    if (status == ORACLE_OK)
      for (int i = 0; i < M; ++i)
        for (int k = 0; k < M; ++k) {
          double complex acc = 0.0;
          for (int col = D; col < M; ++col) acc += (VCOL(col, i) * (1.0 / evals[col])) * conj(VCOL(col, k));
          Cm[i * M + k] = acc;
        }
  } else if (alg == ORACLE_MN) {
    double complex *Pn = (double complex *)calloc((size_t)M * M, sizeof(double complex));
    for (int i = 0; i < M; ++i)
      for (int k = 0; k < M; ++k) {
        double complex acc = 0.0;
        for (int col = D; col < M; ++col) acc += VCOL(col, i) * conj(VCOL(col, k));
        Pn[i * M + k] = acc;
      }
    double uPu = creal(Pn[0]); /* u^H P_n u with u = e_1 */
    if (!(uPu > 0.0)) {
      status = ORACLE_ERANK;
    } else {
      double lambda = 1.0 / uPu;
      double complex *valph = (double complex *)malloc(sizeof(double complex) * M);
      for (int i = 0; i < M; ++i) valph[i] = Pn[i * M + 0] * lambda; /* P_n * lambda * u */
      for (int i = 0; i < M; ++i)
        for (int k = 0; k < M; ++k) Cm[i * M + k] = valph[i] * conj(valph[k]);
      free(valph);
    }
    free(Pn);
  } else {
    status = ORACLE_EINVAL;
  }
#undef VCOL
  for (int i = 0; i < M * M; ++i) {
    C[2 * i] = creal(Cm[i]);
    C[2 * i + 1] = cimag(Cm[i]);
  }
  free(Cm);
  free(Vc);
  return status;
}

/* Eq. 2 for the half-wavelength uniform linear array: a_m = exp(j pi m sin(theta)). */
static void oracle_steering(int M, double theta_deg, double complex *a) {
  double s = sin(theta_deg * (ORACLE_PI / 180.0));
  for (int m = 0; m < M; ++m) {
    double phase = ORACLE_PI * (double)m * s;
    a[m] = cos(phase) + I * sin(phase);
  }
}

/* ---------------------------------------------------------------------------------------------
 * Step-5 (Table 2): for every grid angle theta_k = lo + k*step, k = 0..L-1,
 *   invP_k = a_k^H C a_k,  P_k = 1 / invP_k.
 * C: M x M complex128 row-major interleaved. P: L doubles. The imaginary part of invP is
 * returned through max_rel_imag (max over k of |Im invP| / |Re invP|), which is zero up to
 * rounding for a Hermitian C. invP <= 0 gives P = +inf.
 * ------------------------------------------------------------------------------------------- */
void oracle_scan(const double *C, int M, double lo, double step, int L, double *P, double *max_rel_imag) {
  double complex *Cm = (double complex *)malloc(sizeof(double complex) * M * M);
  double complex *a = (double complex *)malloc(sizeof(double complex) * M);
  for (int i = 0; i < M * M; ++i) Cm[i] = C[2 * i] + I * C[2 * i + 1];
  double worst = 0.0;
  for (int k = 0; k < L; ++k) {
    double kstep = (double)k * step;
    double theta = lo + kstep;
    oracle_steering(M, theta, a);
    double complex invP = 0.0;
    for (int i = 0; i < M; ++i) {
      double complex row = 0.0;
      for (int j = 0; j < M; ++j) row += Cm[i * M + j] * a[j];
      invP += conj(a[i]) * row;
    }
    double re = creal(invP);
    if (re != 0.0) {
      double r = fabs(cimag(invP)) / fabs(re);
      if (r > worst) worst = r;
    }
    P[k] = (re > 0.0) ? 1.0 / re : INFINITY;
  }
  if (max_rel_imag) *max_rel_imag = worst;
  free(a);
  free(Cm);
}

/* ---------------------------------------------------------------------------------------------
 * Step-6 (Table 2): findPeaks then PeakSelection(peakVals, inds, D).
 * A peak is the left end i of a maximal run [i..j] of equal values with 1 <= i, j <= L-2,
 * P[i-1] < P[i] and P[j+1] < P[j]. The D largest values are selected (equal values: lower
 * index first) and written to idx/val in ascending index order. Returns the count (<= D).
 * ------------------------------------------------------------------------------------------- */
int oracle_peaks(const double *P, int L, int D, int *idx, double *val) {
  int cap = 0, n = 0;
  int *cand = NULL;
  for (int i = 1; i <= L - 2; ++i) {
    if (!(P[i - 1] < P[i])) continue;
    int j = i;
    while (j + 1 <= L - 1 && P[j + 1] == P[i]) ++j;
    if (j + 1 <= L - 1 && P[j + 1] < P[j]) {
      if (n == cap) {
        cap = cap ? 2 * cap : 64;
        cand = (int *)realloc(cand, sizeof(int) * cap);
      }
      cand[n++] = i;
    }
  }
  /* order candidates by (value descending, index ascending): insertion sort, stable on index */
  for (int a = 1; a < n; ++a) {
    int cur = cand[a];
    int b = a - 1;
    while (b >= 0 && (P[cand[b]] < P[cur])) {
      cand[b + 1] = cand[b];
      --b;
    }
    cand[b + 1] = cur;
  }
  int count = n < D ? n : D;
  /* ascending index order for the selected ones */
  for (int a = 1; a < count; ++a) {
    int cur = cand[a];
    int b = a - 1;
    while (b >= 0 && cand[b] > cur) {
      cand[b + 1] = cand[b];
      --b;
    }
    cand[b + 1] = cur;
  }
  for (int a = 0; a < count; ++a) {
    idx[a] = cand[a];
    val[a] = P[cand[a]];
  }
  free(cand);
  return count;
}

/* ---------------------------------------------------------------------------------------------
 * Whole method for one snapshot matrix and one algorithm (Table 2, Steps 1-6).
 * Outputs: P[L], evals[M], C[M*M*2], idx/val[D]; returns count of peaks (>= 0) or -status.
 * ------------------------------------------------------------------------------------------- */
int oracle_solve(const float *X, int M, int N, int ldx, int D, int alg, double lo, double step, int L,
                 double *P, double *evals, double *C, int *idx, double *val) {
  if (M < 2 || N < 1 || L < 3 || D < 0 || D >= M) return -ORACLE_EINVAL;
  double *R = (double *)malloc(sizeof(double) * 2 * M * M);
  double *V = (double *)malloc(sizeof(double) * 2 * M * M);
  oracle_covariance(X, M, N, ldx, R);
  int sweeps = oracle_eigh(R, M, 1e-15, 100, evals, V);
  int status = 0;
  if (sweeps < 0) {
    status = -sweeps;
  } else {
    int st = oracle_weighting(evals, V, M, D, alg, C);
    if (st != ORACLE_OK) status = st;
  }
  int count = 0;
  if (status == 0) {
    double rel_imag = 0.0;
    oracle_scan(C, M, lo, step, L, P, &rel_imag);
    count = oracle_peaks(P, L, D, idx, val);
  }
  free(V);
  free(R);
  return status ? -status : count;
}

/* ---------------------------------------------------------------------------------------------
 * Step-5 for an arbitrary array geometry on an azimuth x elevation grid (Eq. 2 as printed):
 *   a_m(theta, phi) = exp{ j 2 pi / lambda (x_m sin theta sin phi + y_m cos theta sin phi
 *                                           + z_m cos phi) },
 * theta = azimuth, phi = elevation, both in degrees; pos holds (x_m, y_m, z_m) in wavelengths.
 * Grid: theta_k = az_lo + k az_step (k < La), phi_l = el_lo + l el_step (l < Le); P is Le x La
 * row-major (row l = one azimuth sweep at elevation phi_l). invP = a^H C a with the explicit C.
 * ------------------------------------------------------------------------------------------- */
void oracle_scan_geometry(const double *C, int M, const double *pos, double az_lo, double az_step, int La,
                          double el_lo, double el_step, int Le, double *P) {
  double complex *Cm = (double complex *)malloc(sizeof(double complex) * M * M);
  double complex *a = (double complex *)malloc(sizeof(double complex) * M);
  for (int i = 0; i < M * M; ++i) Cm[i] = C[2 * i] + I * C[2 * i + 1];
  for (int l = 0; l < Le; ++l) {
    double lstep = (double)l * el_step;
    double phi = (el_lo + lstep) * (ORACLE_PI / 180.0);
    for (int k = 0; k < La; ++k) {
      double kstep = (double)k * az_step;
      double theta = (az_lo + kstep) * (ORACLE_PI / 180.0);
      double u = sin(theta) * sin(phi), v = cos(theta) * sin(phi), w = cos(phi);
      for (int m = 0; m < M; ++m) {
        double t = pos[3 * m] * u + pos[3 * m + 1] * v + pos[3 * m + 2] * w;
        double phase = 2.0 * ORACLE_PI * t;
        a[m] = cos(phase) + I * sin(phase);
      }
      double complex invP = 0.0;
      for (int i = 0; i < M; ++i) {
        double complex row = 0.0;
        for (int j = 0; j < M; ++j) row += Cm[i * M + j] * a[j];
        invP += conj(a[i]) * row;
      }
      double re = creal(invP);
      P[(size_t)l * La + k] = (re > 0.0) ? 1.0 / re : INFINITY;
    }
  }
  free(a);
  free(Cm);
}

/* ---------------------------------------------------------------------------------------------
 * Step-6 on an Le x La azimuth-elevation spectrum (row-major, row = elevation). A peak is a point
 * strictly larger than every one of its 8 neighbours; in azimuth the neighbours wrap around when
 * wrap_az != 0 (the azimuth grid closes the circle), in elevation rows outside the grid do not
 * exist. The D largest (equal values: lower flat index l*La + k first) are returned as flat
 * indices in ascending order. Returns the count (<= D).
 * ------------------------------------------------------------------------------------------- */
int oracle_peaks2d(const double *P, int La, int Le, int wrap_az, int D, int *idx, double *val) {
  int cap = 0, n = 0;
  int *cand = NULL;
  for (int l = 0; l < Le; ++l)
    for (int k = 0; k < La; ++k) {
      double v = P[(size_t)l * La + k];
      int peak = 1, nbrs = 0;
      for (int dl = -1; dl <= 1 && peak; ++dl)
        for (int dk = -1; dk <= 1 && peak; ++dk) {
          if (dl == 0 && dk == 0) continue;
          int ll = l + dl, kk = k + dk;
          if (ll < 0 || ll >= Le) continue;
          if (kk < 0 || kk >= La) {
            if (!wrap_az) continue;
            kk = (kk + La) % La;
          }
          ++nbrs;
          if (!(P[(size_t)ll * La + kk] < v)) peak = 0;
        }
      if (peak && nbrs > 0) {
        if (n == cap) {
          cap = cap ? 2 * cap : 64;
          cand = (int *)realloc(cand, sizeof(int) * cap);
        }
        cand[n++] = l * La + k;
      }
    }
  for (int a = 1; a < n; ++a) {   /* value descending, flat index ascending */
    int cur = cand[a];
    int b = a - 1;
    while (b >= 0 && (P[cand[b]] < P[cur])) {
      cand[b + 1] = cand[b];
      --b;
    }
    cand[b + 1] = cur;
  }
  int count = n < D ? n : D;
  for (int a = 1; a < count; ++a) {
    int cur = cand[a];
    int b = a - 1;
    while (b >= 0 && cand[b] > cur) {
      cand[b + 1] = cand[b];
      --b;
    }
    cand[b + 1] = cur;
  }
  for (int a = 0; a < count; ++a) {
    idx[a] = cand[a];
    val[a] = P[cand[a]];
  }
  free(cand);
  return count;
}

/* ---------------------------------------------------------------------------------------------
 * Sub-grid refinement of a Step-6 peak (beyond the paper, which stops at grid resolution): the
 * local minimiser of den(theta) = a(theta)^H C a(theta) next to grid peak k of the ULA scan,
 * found by Newton's method on den'(theta) = 0 (theta in radians), kept inside the bracket
 * [theta_{k-1}, theta_{k+1}]: each step first shrinks the bracket by the sign of den' (den' > 0:
 * the minimiser lies to the left); when den'' > 0 and the Newton step -den'/den'' is shorter than
 * 1e-13 rad it takes it and stops; otherwise it moves to the Newton point if that lies strictly
 * inside the bracket, else to the bracket's midpoint, and stops when that move is shorter than
 * 1e-13 rad or after 60 steps. With a_m = exp(j pi m sin theta):
 *   a'_m  = j pi m cos(theta) a_m,
 *   a''_m = (-j pi m sin(theta) - (pi m cos(theta))^2) a_m,
 *   den'  = 2 Re(a'^H C a),   den'' = 2 Re(a''^H C a) + 2 a'^H C a'.
 * Returns the refined angle in degrees; *iters receives the steps taken.
 * ------------------------------------------------------------------------------------------- */
static void oracle_den_derivs(const double complex *Cm, int M, double th, double *f, double *f1, double *f2) {
  double complex *a = (double complex *)malloc(sizeof(double complex) * 3 * M);
  double complex *a1 = a + M, *a2 = a + 2 * M;
  double s = sin(th), c = cos(th);
  for (int m = 0; m < M; ++m) {
    double phase = ORACLE_PI * (double)m * s;
    a[m] = cos(phase) + I * sin(phase);
    double pm = ORACLE_PI * (double)m;
    a1[m] = (I * pm * c) * a[m];
    a2[m] = (-I * pm * s - (pm * c) * (pm * c)) * a[m];
  }
  double complex q0 = 0.0, q1 = 0.0, q2 = 0.0, q11 = 0.0;
  for (int i = 0; i < M; ++i) {
    double complex row0 = 0.0, row1 = 0.0;
    for (int j = 0; j < M; ++j) {
      row0 += Cm[i * M + j] * a[j];
      row1 += Cm[i * M + j] * a1[j];
    }
    q0 += conj(a[i]) * row0;
    q1 += conj(a1[i]) * row0;
    q2 += conj(a2[i]) * row0;
    q11 += conj(a1[i]) * row1;
  }
  *f = creal(q0);
  *f1 = 2.0 * creal(q1);
  *f2 = 2.0 * creal(q2) + 2.0 * creal(q11);
  free(a);
}

double oracle_refine_peak(const double *C, int M, double lo, double step, int k, int *iters) {
  double complex *Cm = (double complex *)malloc(sizeof(double complex) * M * M);
  for (int i = 0; i < M * M; ++i) Cm[i] = C[2 * i] + I * C[2 * i + 1];
  const double d2r = ORACLE_PI / 180.0;
  double t0 = lo + (double)(k - 1) * step, t1 = lo + (double)k * step, t2 = lo + (double)(k + 1) * step;
  double x_lo = fmin(t0, t2) * d2r, x_hi = fmax(t0, t2) * d2r, x = t1 * d2r;
  int it = 0;
  for (; it < 60; ++it) {
    double f, f1, f2;
    oracle_den_derivs(Cm, M, x, &f, &f1, &f2);
    if (f1 > 0.0) x_hi = x; else x_lo = x;
    if (f2 > 0.0 && fabs(f1) < 1e-13 * f2) {
      x -= f1 / f2;
      ++it;
      break;
    }
    double xn = (f2 > 0.0) ? x - f1 / f2 : NAN;
    if (!(xn > x_lo && xn < x_hi)) xn = 0.5 * (x_lo + x_hi);
    double dx = fabs(xn - x);
    x = xn;
    if (dx < 1e-13) {
      ++it;
      break;
    }
  }
  if (iters) *iters = it;
  free(Cm);
  return x / d2r;
}

/* ---------------------------------------------------------------------------------------------
 * Sub-grid refinement of a 2-D peak (flat index l * La + k of the azimuth x elevation scan, Eq. 2
 * as printed): the local minimiser of den(theta, phi) = a^H C a inside the box theta_k +- |az step|,
 * phi_l +- |el step|, by damped Newton. With t_m = p_m . u(theta, phi) (turns),
 *   a_m = exp(j 2 pi t_m),  a_i = j 2 pi t_i a,  a_ij = (j 2 pi t_ij - 4 pi^2 t_i t_j) a,
 *   g_i = 2 Re(a_i^H C a),  H_ij = 2 Re(a_ij^H C a) + 2 Re(a_i^H C a_j),
 * where t_i, t_ij are t's derivatives through u = (sin th sin ph, cos th sin ph, cos ph). A step
 * is d = -H^-1 g when H is positive definite, else the steepest-descent direction scaled to the box
 * half-width. A Newton step shorter than 1e-6 rad in both angles is taken as it is (the quadratic
 * end game, where den itself is below its rounding noise); any other step is halved (up to 40
 * times) until den does not increase. The point is clamped into the box; the iteration stops when
 * a step moves both angles by less than 1e-13 rad, when no halving decreases den, or after 60
 * steps. out[0] = azimuth, out[1] = elevation (degrees).
 * ------------------------------------------------------------------------------------------- */
static double oracle_den2d(const double complex *Cm, int M, const double *pos, double th, double ph, double g[2],
                           double H[3]) {
  double complex *a = (double complex *)malloc(sizeof(double complex) * 6 * M);
  double complex *at = a + M, *ap = a + 2 * M, *att = a + 3 * M, *atp = a + 4 * M, *app = a + 5 * M;
  const double st = sin(th), ct = cos(th), sp = sin(ph), cp = cos(ph);
  const double u[3] = {st * sp, ct * sp, cp};
  const double ut[3] = {ct * sp, -st * sp, 0.0};
  const double up[3] = {st * cp, ct * cp, -sp};
  const double utt[3] = {-st * sp, -ct * sp, 0.0};
  const double utp[3] = {ct * cp, -st * cp, 0.0};
  const double upp[3] = {-st * sp, -ct * sp, -cp};
  const double tp = 2.0 * ORACLE_PI;
  for (int m = 0; m < M; ++m) {
    const double *p = pos + 3 * m;
    double t = p[0] * u[0] + p[1] * u[1] + p[2] * u[2];
    double t_t = p[0] * ut[0] + p[1] * ut[1] + p[2] * ut[2];
    double t_p = p[0] * up[0] + p[1] * up[1] + p[2] * up[2];
    double t_tt = p[0] * utt[0] + p[1] * utt[1] + p[2] * utt[2];
    double t_tp = p[0] * utp[0] + p[1] * utp[1] + p[2] * utp[2];
    double t_pp = p[0] * upp[0] + p[1] * upp[1] + p[2] * upp[2];
    a[m] = cos(tp * t) + I * sin(tp * t);
    at[m] = (I * tp * t_t) * a[m];
    ap[m] = (I * tp * t_p) * a[m];
    att[m] = (I * tp * t_tt - tp * tp * t_t * t_t) * a[m];
    atp[m] = (I * tp * t_tp - tp * tp * t_t * t_p) * a[m];
    app[m] = (I * tp * t_pp - tp * tp * t_p * t_p) * a[m];
  }
  double complex q0 = 0, qt = 0, qp = 0, qtt = 0, qtp = 0, qpp = 0, rtt = 0, rtp = 0, rpp = 0;
  for (int i = 0; i < M; ++i) {
    double complex r0 = 0, rt = 0, rp = 0;
    for (int j = 0; j < M; ++j) {
      r0 += Cm[i * M + j] * a[j];
      rt += Cm[i * M + j] * at[j];
      rp += Cm[i * M + j] * ap[j];
    }
    q0 += conj(a[i]) * r0;
    qt += conj(at[i]) * r0;
    qp += conj(ap[i]) * r0;
    qtt += conj(att[i]) * r0;
    qtp += conj(atp[i]) * r0;
    qpp += conj(app[i]) * r0;
    rtt += conj(at[i]) * rt;
    rtp += conj(at[i]) * rp;
    rpp += conj(ap[i]) * rp;
  }
  if (g) {
    g[0] = 2.0 * creal(qt);
    g[1] = 2.0 * creal(qp);
    H[0] = 2.0 * creal(qtt) + 2.0 * creal(rtt);
    H[1] = 2.0 * creal(qtp) + 2.0 * creal(rtp);
    H[2] = 2.0 * creal(qpp) + 2.0 * creal(rpp);
  }
  free(a);
  return creal(q0);
}

void oracle_refine_peak2d(const double *C, int M, const double *pos, double az_lo, double az_step, int La,
                          double el_lo, double el_step, int flat, double *out, int *iters) {
  double complex *Cm = (double complex *)malloc(sizeof(double complex) * M * M);
  for (int i = 0; i < M * M; ++i) Cm[i] = C[2 * i] + I * C[2 * i + 1];
  const double d2r = ORACLE_PI / 180.0;
  const int l = flat / La, k = flat - l * La;
  double x[2] = {(az_lo + (double)k * az_step) * d2r, (el_lo + (double)l * el_step) * d2r};
  const double hw[2] = {fabs(az_step) * d2r, fabs(el_step) * d2r};
  const double bl[2] = {x[0] - hw[0], x[1] - hw[1]}, bh[2] = {x[0] + hw[0], x[1] + hw[1]};
  int it = 0;
  for (; it < 60; ++it) {
    double g[2], H[3];
    double f = oracle_den2d(Cm, M, pos, x[0], x[1], g, H);
    double det = H[0] * H[2] - H[1] * H[1];
    double d[2];
    if (H[0] > 0.0 && det > 0.0) {
      d[0] = -(H[2] * g[0] - H[1] * g[1]) / det;
      d[1] = -(H[0] * g[1] - H[1] * g[0]) / det;
      if (fmax(fabs(d[0]), fabs(d[1])) < 1e-6) {
        double xn0 = fmin(fmax(x[0] + d[0], bl[0]), bh[0]), xn1 = fmin(fmax(x[1] + d[1], bl[1]), bh[1]);
        double mv = fmax(fabs(xn0 - x[0]), fabs(xn1 - x[1]));
        x[0] = xn0;
        x[1] = xn1;
        if (mv < 1e-13) {
          ++it;
          break;
        }
        continue;
      }
    } else {
      double gn = sqrt(g[0] * g[0] + g[1] * g[1]);
      double w = fmax(hw[0], hw[1]);
      d[0] = gn > 0.0 ? -g[0] / gn * w : 0.0;
      d[1] = gn > 0.0 ? -g[1] / gn * w : 0.0;
    }
    double t = 1.0, xn[2] = {x[0], x[1]};
    int accepted = 0;
    for (int h = 0; h <= 40; ++h) {
      xn[0] = fmin(fmax(x[0] + t * d[0], bl[0]), bh[0]);
      xn[1] = fmin(fmax(x[1] + t * d[1], bl[1]), bh[1]);
      if (oracle_den2d(Cm, M, pos, xn[0], xn[1], NULL, NULL) <= f) {
        accepted = 1;
        break;
      }
      t *= 0.5;
    }
    if (!accepted) {
      ++it;
      break;
    }
    double mv = fmax(fabs(xn[0] - x[0]), fabs(xn[1] - x[1]));
    x[0] = xn[0];
    x[1] = xn[1];
    if (mv < 1e-13) {
      ++it;
      break;
    }
  }
  if (iters) *iters = it;
  out[0] = x[0] / d2r;
  out[1] = x[1] / d2r;
  free(Cm);
}

/* ---------------------------------------------------------------------------------------------
 * Model-order estimation (beyond the paper, whose Table 2 takes D as given): the information
 * criteria of Wax and Kailath (1985) for complex data from the sample eigenvalues lambda_0 >= ...
 * >= lambda_{M-1} of R and the snapshot count N. For k assumed sources the M - k smallest
 * eigenvalues are the noise ones; with their arithmetic mean a(k) and geometric mean g(k),
 *   L(k)   = N (M - k) log(a(k) / g(k))           (>= 0, zero when they are all equal),
 *   MDL(k) = L(k) + k (2M - k) log(N) / 2,
 *   AIC(k) = 2 L(k) + 2 k (2M - k),
 * for k = 0 .. M-1; the estimates are the k of the smallest value (the smaller k on a tie). A
 * non-positive noise eigenvalue makes L(k) = +inf. mdl_val / aic_val (nullable) receive the M
 * criterion values.
 * ------------------------------------------------------------------------------------------- */
void oracle_model_order(const double *evals, int M, int N, int *mdl, int *aic, double *mdl_val, double *aic_val) {
  int best_m = 0, best_a = 0;
  double vm = INFINITY, va = INFINITY;
  for (int k = 0; k < M; ++k) {
    int n = M - k;
    double s = 0.0, ls = 0.0;
    int bad = 0;
    for (int i = k; i < M; ++i) {
      s += evals[i];
      if (evals[i] > 0.0) ls += log(evals[i]); else bad = 1;
    }
    double L = bad ? INFINITY : (double)N * (double)n * (log(s / (double)n) - ls / (double)n);
    double pen = (double)k * (double)(2 * M - k);
    double m = L + 0.5 * pen * log((double)N);
    double a = 2.0 * L + 2.0 * pen;
    if (mdl_val) mdl_val[k] = m;
    if (aic_val) aic_val[k] = a;
    if (m < vm) {
      vm = m;
      best_m = k;
    }
    if (a < va) {
      va = a;
      best_a = k;
    }
  }
  *mdl = best_m;
  *aic = best_a;
}

/* ---------------------------------------------------------------------------------------------
 * Step-2 taken as an SVD of the data (the paper computes Step-2 as an SVD; here of X itself, not
 * of R): one-sided Jacobi (Hestenes 1958) on the M rows of X. Rows y_p, y_q of Y (initially X)
 * are rotated, Y <- J^H Y and U <- U J, with the Hermitian Jacobi rotation of oracle_eigh built
 * from the Gram entries alpha = ||y_p||^2, beta = ||y_q||^2, gamma = y_p y_q^H, each recomputed
 * from the rows in FP64 (R is never formed). Pairs row by row; a pair is rotated when
 * |gamma| > tol * sqrt(alpha beta) (and gamma != 0) and neither row is numerically zero (squared
 * norm above 1e-30 of the largest at the sweep's start: the threshold relative to the largest
 * entry that the Jacobi SVD of Sec. 4.2 uses to stop on rank-deficient data); the iteration stops
 * after the first sweep that rotates nothing. Then X = U S V^H with S_k = ||y_k||, and the eigenvalues of R = X X^H / N
 * (Eq. 3) are S_k^2 / N with eigenvectors the columns of U.
 *
 * X: M x N complex128, row-major, interleaved, row stride ldx complex elements (callers with
 * complex64 snapshots promote them exactly). Output as oracle_eigh: evals[M] descending (stable),
 * U column-major interleaved. Returns the number of sweeps, or -ORACLE_ENOCONV.
 * ------------------------------------------------------------------------------------------- */
int oracle_svd_data(const double *X, int M, int N, int ldx, double tol, int max_sweeps, double *evals, double *U) {
  double complex *Y = (double complex *)malloc(sizeof(double complex) * (size_t)M * N);
  double complex *W = (double complex *)malloc(sizeof(double complex) * M * M);
  for (int i = 0; i < M; ++i) {
    for (int t = 0; t < N; ++t)
      Y[(size_t)i * N + t] = X[2 * ((size_t)i * ldx + t)] + I * X[2 * ((size_t)i * ldx + t) + 1];
    for (int j = 0; j < M; ++j) W[i * M + j] = (i == j) ? 1.0 : 0.0; /* row-major: W[i*M+j] = U(i,j) */
  }
  int sweeps = 0, converged = 0;
  while (sweeps < max_sweeps) {
    ++sweeps;
    int rotations = 0;
    /* rows whose squared norm is below 1e-30 of the largest (at the sweep's start) are numerically
       zero: a rank-deficient X (N < M) leaves such rows at the rounding level, where |gamma| is
       comparable to sqrt(alpha beta) whatever is done, so pairs with one are not rotated */
    double maxd = 0.0;
    for (int i = 0; i < M; ++i) {
      double a = 0.0;
      for (int t = 0; t < N; ++t) a += creal(Y[(size_t)i * N + t] * conj(Y[(size_t)i * N + t]));
      if (a > maxd) maxd = a;
    }
    const double floor_d = 1e-30 * maxd;
    for (int p = 0; p < M - 1; ++p) {
      for (int q = p + 1; q < M; ++q) {
        const double complex *yp = Y + (size_t)p * N, *yq = Y + (size_t)q * N;
        double alpha = 0.0, beta = 0.0;
        double complex gamma = 0.0;
        for (int t = 0; t < N; ++t) {
          alpha += creal(yp[t] * conj(yp[t]));
          beta += creal(yq[t] * conj(yq[t]));
          gamma += yp[t] * conj(yq[t]);
        }
        double mag = cabs(gamma);
        if (mag == 0.0 || mag <= tol * sqrt(alpha * beta) || alpha <= floor_d || beta <= floor_d) continue;
        ++rotations;
        double complex ph = gamma / mag;
        double tau = (beta - alpha) / (2.0 * mag);
        double tt = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
        double c = 1.0 / sqrt(1.0 + tt * tt);
        double s = tt * c;
        /* Y <- J^H Y : rows p and q */
        for (int t = 0; t < N; ++t) {
          double complex xp = Y[(size_t)p * N + t], xq = Y[(size_t)q * N + t];
          Y[(size_t)p * N + t] = c * xp - s * ph * xq;
          Y[(size_t)q * N + t] = s * conj(ph) * xp + c * xq;
        }
        /* U <- U J : columns p and q */
        for (int r = 0; r < M; ++r) {
          double complex xp = W[r * M + p], xq = W[r * M + q];
          W[r * M + p] = c * xp - s * conj(ph) * xq;
          W[r * M + q] = s * ph * xp + c * xq;
        }
      }
    }
    if (rotations == 0) {
      converged = 1;
      break;
    }
  }
  double *nrm = (double *)malloc(sizeof(double) * M);
  for (int i = 0; i < M; ++i) {
    double a = 0.0;
    for (int t = 0; t < N; ++t) a += creal(Y[(size_t)i * N + t] * conj(Y[(size_t)i * N + t]));
    nrm[i] = a / (double)N;
  }
  int *order = (int *)malloc(sizeof(int) * M);
  for (int i = 0; i < M; ++i) order[i] = i;
  for (int i = 1; i < M; ++i) {
    int cur = order[i];
    int j = i - 1;
    while (j >= 0 && nrm[order[j]] < nrm[cur]) {
      order[j + 1] = order[j];
      --j;
    }
    order[j + 1] = cur;
  }
  for (int i = 0; i < M; ++i) {
    int src = order[i];
    evals[i] = nrm[src];
    for (int r = 0; r < M; ++r) {
      U[2 * (i * M + r)] = creal(W[r * M + src]);
      U[2 * (i * M + r) + 1] = cimag(W[r * M + src]);
    }
  }
  free(order);
  free(nrm);
  free(W);
  free(Y);
  return converged ? sweeps : -ORACLE_ENOCONV;
}
