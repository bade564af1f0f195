// Steps 2-4 (Table 2 Step-2, Table 3): Hermitian eigendecomposition of R by FP64 cyclic Jacobi,
// followed by the noise-subspace factor B of each algorithm's weighting matrix C = B B^H (one
// call), or, in the batch, one scan factor per problem from which every requested algorithm's
// spectrum is read (E_n with EV weights 1/lambda, v_min, valph).
//
// Jacobi (Golub & Van Loan, Sec. 8.5, with a phase factor for complex Hermitian matrices):
// for a pair (p, q) with a_pq = |a_pq| e^{j phi}, tau = (a_qq - a_pp) / (2 |a_pq|),
// t = sgn(tau) / (|tau| + sqrt(1 + tau^2)), c = 1/sqrt(1 + t^2), s = t c, sigma = s e^{j phi};
// J = [[c, sigma], [-conj(sigma), c]] on coordinates (p, q) zeroes (J^H A J)_pq.
// Each rotation's parameters use reciprocal square roots and one reciprocal (no divisions,
// hypot or sqrt), so c^2 + |sigma|^2 = 1 holds to FP64 rounding.
//
// Parallel ordering: n/2 disjoint rotations per round (round-robin "circle" ordering over
// n = M rounded up to even; pairs that touch the padding index are skipped): the row update
// A <- J^H A for all rotated pairs, then the column updates A <- A J and V <- V J. A pair is
// rotated when |a_pq|^2 > tol^2 |a_pp a_qq|; a matrix has converged after a sweep that rotates
// nothing. A warp holds 32 / (NP/2) matrices so that every lane owns one pair's rotation
// (8 matrices of M <= 8, 4 of M <= 16, 2 of M <= 32); a matrix of M <= 64 gets a whole CTA in
// FP64, or in double-float a cluster of four CTAs that split its rows (jacobi_cluster_df).
// The element updates of each matrix are spread over all threads of its group. A and V live in shared memory with a padded row stride
// (NP + 1 complex128) so that column accesses by consecutive lanes hit distinct banks.
#include <cooperative_groups.h>
#include <math_constants.h>

#include "doa_internal.cuh"

namespace doa {
namespace {

namespace cg = cooperative_groups;

struct Rot {
  double c, sr, si;  // cosine and sigma = s e^{j phi}
};

template <int NP>
struct EigSmem {
  // A and V row-major without padding; element (i, k) sits in column slot k ^ (i & 7), so that
  // both row walks (fixed i) and column walks (fixed k, consecutive rows) touch distinct banks
  double2 A[NP][NP];
  double2 V[NP][NP];
  Rot rot[NP / 2];      // the sweeps' rotations; after the sweeps the same bytes hold lam, order
  int2 pq[NP / 2];
  unsigned mask;        // rotation mask broadcast when a group spans several warps
  __device__ __forceinline__ double2 &a(int i, int k) { return A[i][k ^ (i & 7)]; }
  __device__ __forceinline__ double2 &v(int i, int k) { return V[i][k ^ (i & 7)]; }
  __device__ __forceinline__ double *lam() { return reinterpret_cast<double *>(rot); }
  __device__ __forceinline__ int *order() { return reinterpret_cast<int *>(reinterpret_cast<double *>(rot) + NP); }
  static_assert(sizeof(Rot) * (NP / 2) >= NP * (sizeof(double) + sizeof(int)), "lam and order fit in rot");
};

// A group of T threads works on G matrices: one warp on 8, 4 or 2 matrices of M <= 8, 16, 32
// (every lane owns one pair), or a whole 16-warp CTA on one matrix of M <= 64 (the 32 pairs
// are owned by warp 0's lanes; the element updates are spread over all 512 threads).
template <int NP>
__host__ __device__ constexpr int grp_threads() { return NP <= 32 ? 32 : 512; }
template <int NP>
__host__ __device__ constexpr int mats_per_warp() { return NP <= 32 ? 64 / NP : 1; }
// Warps per CTA of the batch kernel, at most (the launch picks the count for the resident total).
template <int NP>
__host__ __device__ constexpr int eig_warps() { return NP <= 8 ? 4 : (NP <= 16 ? 9 : (NP <= 32 ? 1 : 16)); }
// CTAs per SM the batch kernel's register budget is set for: three nine-warp CTAs at M <= 16,
// elsewhere 64 registers a thread.
template <int NP>
__host__ __device__ constexpr int eig_min_ctas() { return NP > 8 && NP <= 16 ? 3 : 1024 / (32 * eig_warps<NP>()); }

template <int T>
struct Grp {
  __device__ static int id() { return (int)(threadIdx.x % T); }
  __device__ static void sync() {
    if (T == 32) __syncwarp(); else __syncthreads();
  }
  __device__ static bool all(bool p) { return T == 32 ? __all_sync(0xffffffffu, p) : __syncthreads_and(p) != 0; }
  __device__ static bool any(bool p) { return T == 32 ? __any_sync(0xffffffffu, p) : __syncthreads_or(p) != 0; }
};

__device__ __forceinline__ int rr_player(int pos, int r, int n) {
  return pos == 0 ? 0 : ((pos - 1 + r) % (n - 1)) + 1;
}

// Rotation of pair (p, q) of A; returns false if the pair is below threshold.
template <int NP>
__device__ __forceinline__ bool rotation(EigSmem<NP> &s, int p, int q, Rot &ro) {
  const double app = s.a(p, p).x, aqq = s.a(q, q).x;
  const double2 apq = s.a(p, q);
  const double n2 = apq.x * apq.x + apq.y * apq.y;
  if (!(n2 > 0.0) || !(n2 > kJacobiTol * kJacobiTol * fabs(app * aqq))) return false;
  const double r = rsqrt(n2);                         // 1 / |a_pq|
  const double tau = (aqq - app) * (0.5 * r);
  double t;
  if (fabs(tau) > 1e18) {
    t = 0.5 * __drcp_rn(tau);                         // t = 1/(2 tau) to within tau^-2
  } else {
    const double u = fma(tau, tau, 1.0);
    const double h = u * rsqrt(u);                    // sqrt(1 + tau^2)
    t = copysign(__drcp_rn(fabs(tau) + h), tau);
  }
  const double c = rsqrt(fma(t, t, 1.0));
  const double sn = t * c * r;
  ro = Rot{c, sn * apq.x, sn * apq.y};
  return true;
}

// Runs Jacobi on the G matrices of a warp (matrix j has size Ms[j] <= NP, 0 = unused), all
// loaded from Rs[j] (upper triangle). res[j] receives sweeps (> 0) or -status.
template <int NP, int G>
__device__ void jacobi_group(EigSmem<NP> *mats, const int *Ms, const double2 *const *Rs, int *res) {
  constexpr int HP = NP / 2;
  constexpr int T = grp_threads<NP>();
  using g = Grp<T>;
  const int lane = g::id();
  unsigned live = 0u;  // matrices still iterating
  for (int j = 0; j < G; ++j) {
    const int M = Ms[j];
    res[j] = 0;
    if (M <= 0) continue;
    EigSmem<NP> &s = mats[j];
    const double2 *R = Rs[j];
    bool finite = true;
    for (int e = lane; e < M * M; e += T) {
      int i = e / M, k = e % M;
      double2 v;
      if (i <= k) {
        v = R[i * M + k];
      } else {
        v = R[k * M + i];
        v.y = -v.y;
      }
      if (i == k) v.y = 0.0;
      finite = finite && isfinite(v.x) && isfinite(v.y);
      s.a(i, k) = v;
      s.v(i, k) = make_double2(i == k ? 1.0 : 0.0, 0.0);
    }
    if (g::all(finite))
      live |= 1u << j;
    else
      res[j] = -DOA_ENONFINITE;
  }
  g::sync();
  int maxn = 0;
  for (int j = 0; j < G; ++j)
    if ((live >> j) & 1u) maxn = max(maxn, (Ms[j] + 1) & ~1);
  // lane -> (matrix, pair) for the rotation parameters
  const int lj = lane < 32 ? lane / HP : G, li = lane % HP;
  for (int sweep = 1; sweep <= kMaxSweeps && live; ++sweep) {
    unsigned rotated = 0u;
    for (int r = 0; r < maxn - 1; ++r) {
      bool act = false;
      if (lj < G && ((live >> lj) & 1u)) {
        const int M = Ms[lj], n = (M + 1) & ~1;
        if (r < n - 1 && li < n / 2) {
          const int a = rr_player(li, r, n), b = rr_player(n - 1 - li, r, n);
          const int p = min(a, b), q = max(a, b);
          if (q < M) {
            Rot ro;
            if (rotation<NP>(mats[lj], p, q, ro)) {
              act = true;
              mats[lj].rot[li] = ro;
              mats[lj].pq[li] = make_int2(p, q);
            }
          }
        }
      }
      unsigned mask;
      if (T == 32) {
        mask = __ballot_sync(0xffffffffu, act);
      } else {
        const unsigned m0 = __ballot_sync(0xffffffffu, act);
        if (threadIdx.x == 0) mats[0].mask = m0;    // only warp 0 owns pairs
        __syncthreads();
        mask = mats[0].mask;
        __syncthreads();
      }
      if (mask == 0u) continue;
      g::sync();
      // rows: A <- J^H A. new row p = c x_p - sigma x_q; new row q = conj(sigma) x_p + c x_q
      for (int j = 0; j < G; ++j) {
        const unsigned seg = (mask >> (j * HP)) & ((HP == 32) ? 0xffffffffu : ((1u << HP) - 1u));
        if (!seg) continue;
        rotated |= 1u << j;
        EigSmem<NP> &s = mats[j];
        const int M = Ms[j];
        for (int it = lane; it < HP * M; it += T) {
          const int i = it / M, k = it % M;
          if (!((seg >> i) & 1u)) continue;
          const Rot ro = s.rot[i];
          const int2 pq = s.pq[i];
          const double2 xp = s.a(pq.x, k), xq = s.a(pq.y, k);
          s.a(pq.x, k) = make_double2(ro.c * xp.x - (ro.sr * xq.x - ro.si * xq.y),
                                      ro.c * xp.y - (ro.sr * xq.y + ro.si * xq.x));
          s.a(pq.y, k) = make_double2(ro.c * xq.x + (ro.sr * xp.x + ro.si * xp.y),
                                      ro.c * xq.y + (ro.sr * xp.y - ro.si * xp.x));
        }
      }
      g::sync();
      // columns: A <- A J, V <- V J. new col p = c x_p - conj(sigma) x_q; new col q = sigma x_p + c x_q
      for (int j = 0; j < G; ++j) {
        const unsigned seg = (mask >> (j * HP)) & ((HP == 32) ? 0xffffffffu : ((1u << HP) - 1u));
        if (!seg) continue;
        EigSmem<NP> &s = mats[j];
        const int M = Ms[j];
        for (int it = lane; it < HP * M; it += T) {
          const int i = it / M, k = it % M;
          if (!((seg >> i) & 1u)) continue;
          const Rot ro = s.rot[i];
          const int2 pq = s.pq[i];
          const double2 xp = s.a(k, pq.x), xq = s.a(k, pq.y);
          s.a(k, pq.x) = make_double2(ro.c * xp.x - (ro.sr * xq.x + ro.si * xq.y),
                                      ro.c * xp.y - (ro.sr * xq.y - ro.si * xq.x));
          s.a(k, pq.y) = make_double2(ro.c * xq.x + (ro.sr * xp.x - ro.si * xp.y),
                                      ro.c * xq.y + (ro.sr * xp.y + ro.si * xp.x));
          const double2 vp = s.v(k, pq.x), vq = s.v(k, pq.y);
          s.v(k, pq.x) = make_double2(ro.c * vp.x - (ro.sr * vq.x + ro.si * vq.y),
                                      ro.c * vp.y - (ro.sr * vq.y - ro.si * vq.x));
          s.v(k, pq.y) = make_double2(ro.c * vq.x + (ro.sr * vp.x - ro.si * vp.y),
                                      ro.c * vq.y + (ro.sr * vp.y + ro.si * vp.x));
        }
      }
      g::sync();
      if (act) {
        EigSmem<NP> &s = mats[lj];
        const int2 pq = s.pq[li];
        s.a(pq.x, pq.y) = make_double2(0.0, 0.0);
        s.a(pq.y, pq.x) = make_double2(0.0, 0.0);
        s.a(pq.x, pq.x).y = 0.0;
        s.a(pq.y, pq.y).y = 0.0;
      }
      g::sync();
    }
    // matrices without a rotation in this sweep have converged
    for (int j = 0; j < G; ++j)
      if (((live >> j) & 1u) && !((rotated >> j) & 1u)) {
        res[j] = sweep;
        live &= ~(1u << j);
      }
  }
  for (int j = 0; j < G; ++j)
    if ((live >> j) & 1u) res[j] = -DOA_ENOCONV;
}

// ------------------------------------------------------------------------------------------
// Double-float Jacobi for the batch. GB300 issues FP64 at ~1/64 of its FP32 rate, so the batch
// runs the same cyclic Jacobi with A and V held as unevaluated sums hi + lo of two FP32 numbers
// (about 48 significant bits) and every element update done on the FP32 pipe: each new real part
// is a three-term dot product of double-float numbers, formed with exact FMA products and
// TwoSum (a compensated dot product, relative error a few 2^-48 of the sum of |terms|).
// The rotation angle only needs to be good to FP32: tau, t and (c, sigma) are computed in FP32
// from the hi parts (the diagonal difference from hi and lo), then (c, sigma) is scaled by
// 1/sqrt(c^2 + |sigma|^2) to double-float accuracy, so every applied rotation is unitary to
// ~1e-15; a_pq is left at its computed residual (about 1e-7 of its old value) instead of being
// set to zero, and the next sweep removes it. Converged when a sweep rotates no pair with
// |a_pq| > kJacobiTolDF sqrt(|a_pp a_qq|). A and V are converted to FP64 in place at the end.
// ------------------------------------------------------------------------------------------
constexpr float kJacobiTolDF = 1e-12f;

struct F2 {
  float h, l;
};

__device__ __forceinline__ void two_sum_f(float a, float b, float &s, float &e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// u1 v1 + u2 v2 + u3 v3 in double-float.
__device__ __forceinline__ F2 dot3(F2 u1, F2 v1, F2 u2, F2 v2, F2 u3, F2 v3) {
  const float p1 = __fmul_rn(u1.h, v1.h), p2 = __fmul_rn(u2.h, v2.h), p3 = __fmul_rn(u3.h, v3.h);
  float low = __fmaf_rn(u1.h, v1.h, -p1);
  low = __fadd_rn(low, __fmaf_rn(u2.h, v2.h, -p2));
  low = __fadd_rn(low, __fmaf_rn(u3.h, v3.h, -p3));
  low = __fadd_rn(low, __fmaf_rn(u1.h, v1.l, __fmul_rn(u1.l, v1.h)));
  low = __fadd_rn(low, __fmaf_rn(u2.h, v2.l, __fmul_rn(u2.l, v2.h)));
  low = __fadd_rn(low, __fmaf_rn(u3.h, v3.l, __fmul_rn(u3.l, v3.h)));
  float s, e1, e2;
  two_sum_f(p1, p2, s, e1);
  two_sum_f(s, p3, s, e2);
  low = __fadd_rn(low, __fadd_rn(e1, e2));
  F2 r;
  two_sum_f(s, low, r.h, r.l);
  return r;
}

__device__ __forceinline__ F2 neg(F2 a) { return F2{-a.h, -a.l}; }
__device__ __forceinline__ F2 re_of(float4 v) { return F2{v.x, v.y}; }
__device__ __forceinline__ F2 im_of(float4 v) { return F2{v.z, v.w}; }
__device__ __forceinline__ float4 cplx(F2 re, F2 im) { return make_float4(re.h, re.l, im.h, im.l); }
__device__ __forceinline__ float4 df_of(double2 v) {
  const float rh = (float)v.x, ih = (float)v.y;
  return make_float4(rh, (float)(v.x - (double)rh), ih, (float)(v.y - (double)ih));
}

struct RotDF {
  F2 c, sr, si;   // cosine and sigma = s e^{j phi}, each hi + lo
};

template <int NP>
struct EigSmemDF {   // the same bytes as EigSmem<NP>, viewed as double-float
  float4 A[NP][NP];
  float4 V[NP][NP];
  RotDF rot[NP / 2];
  __device__ __forceinline__ float4 &a(int i, int k) { return A[i][k ^ (i & 7)]; }
  __device__ __forceinline__ float4 &v(int i, int k) { return V[i][k ^ (i & 7)]; }
};
static_assert(sizeof(RotDF) == sizeof(Rot), "rotation records share storage");

// Rotation of a pair from its entries a_pp, a_qq, a_pq; returns false below threshold.
__device__ __forceinline__ bool rotation_df_of(const float4 app, const float4 aqq, const float4 apq, RotDF &ro) {
  const float n2 = apq.x * apq.x + apq.z * apq.z;
  if (!(n2 > 0.f) || !(n2 > kJacobiTolDF * kJacobiTolDF * fabsf(app.x * aqq.x))) return false;
  const float r = rsqrtf(n2);                                   // 1 / |a_pq|
  const float diff = __fadd_rn(__fsub_rn(aqq.x, app.x), __fsub_rn(aqq.y, app.y));
  const float tau = diff * (0.5f * r);
  float t;
  if (fabsf(tau) > 1e4f) {
    t = 0.5f / tau;                                             // 1/(2 tau), relative error < tau^-2 / 4
  } else {
    t = copysignf(1.f / (fabsf(tau) + sqrtf(fmaf(tau, tau, 1.f))), tau);
  }
  const float c0 = rsqrtf(fmaf(t, t, 1.f));
  const float sn = t * c0 * r;
  const float sr0 = sn * apq.x, si0 = sn * apq.z;
  // n = c0^2 + sr0^2 + si0^2 exactly to double-float; scale all three by 1/sqrt(n) = 1 + eps
  const float q1 = __fmul_rn(c0, c0), q2 = __fmul_rn(sr0, sr0), q3 = __fmul_rn(si0, si0);
  float low = __fadd_rn(__fadd_rn(__fmaf_rn(c0, c0, -q1), __fmaf_rn(sr0, sr0, -q2)), __fmaf_rn(si0, si0, -q3));
  float sum, e1, e2;
  two_sum_f(q1, q2, sum, e1);
  two_sum_f(sum, q3, sum, e2);
  const float delta = __fadd_rn(__fsub_rn(sum, 1.f), __fadd_rn(low, __fadd_rn(e1, e2)));
  const float eps = delta * fmaf(0.375f, delta, -0.5f);        // (1 + delta)^(-1/2) - 1 to O(delta^3)
  ro = RotDF{F2{c0, c0 * eps}, F2{sr0, sr0 * eps}, F2{si0, si0 * eps}};
  return true;
}

template <int NP>
__device__ __forceinline__ bool rotation_df(EigSmemDF<NP> &s, int p, int q, RotDF &ro) {
  return rotation_df_of(s.a(p, p), s.a(q, q), s.a(p, q), ro);
}

// Same contract as jacobi_group, in double-float arithmetic; on return A and V hold FP64.
template <int NP, int G>
__device__ void jacobi_group_df(EigSmem<NP> *mats64, const int *Ms, const double2 *const *Rs, int *res) {
  constexpr int HP = NP / 2;
  constexpr int T = grp_threads<NP>();
  using g = Grp<T>;
  static_assert(sizeof(EigSmemDF<NP>) <= sizeof(EigSmem<NP>), "double-float view fits");
  // matrix j's double-float view starts where its EigSmem record starts (the records are laid out
  // with the EigSmem stride, so the view is formed per matrix, never by indexing a view array)
  auto df = [&](int j) -> EigSmemDF<NP> & { return *reinterpret_cast<EigSmemDF<NP> *>(&mats64[j]); };
  const int lane = g::id();
  unsigned live = 0u;
  for (int j = 0; j < G; ++j) {
    const int M = Ms[j];
    res[j] = 0;
    if (M <= 0) continue;
    EigSmemDF<NP> &s = df(j);
    const double2 *R = Rs[j];
    bool finite = true;
    for (int e = lane; e < M * M; e += T) {
      int i = e / M, k = e % M;
      double2 v;
      if (i <= k) {
        v = R[i * M + k];
      } else {
        v = R[k * M + i];
        v.y = -v.y;
      }
      if (i == k) v.y = 0.0;
      finite = finite && isfinite(v.x) && isfinite(v.y);
      s.a(i, k) = df_of(v);
      s.v(i, k) = make_float4(i == k ? 1.f : 0.f, 0.f, 0.f, 0.f);
    }
    if (g::all(finite))
      live |= 1u << j;
    else
      res[j] = -DOA_ENONFINITE;
  }
  g::sync();
  int maxn = 0;
  for (int j = 0; j < G; ++j)
    if ((live >> j) & 1u) maxn = max(maxn, (Ms[j] + 1) & ~1);
  const int lj = lane < 32 ? lane / HP : G, li = lane % HP;
  for (int sweep = 1; sweep <= kMaxSweeps && live; ++sweep) {
    unsigned rotated = 0u;
    for (int r = 0; r < maxn - 1; ++r) {
      bool act = false;
      if (lj < G && ((live >> lj) & 1u)) {
        const int M = Ms[lj], n = (M + 1) & ~1;
        if (r < n - 1 && li < n / 2) {
          const int a = rr_player(li, r, n), b = rr_player(n - 1 - li, r, n);
          const int p = min(a, b), q = max(a, b);
          if (q < M) {
            RotDF ro;
            if (rotation_df<NP>(df(lj), p, q, ro)) {
              act = true;
              df(lj).rot[li] = ro;
              mats64[lj].pq[li] = make_int2(p, q);
            }
          }
        }
      }
      unsigned mask;
      if (T == 32) {
        mask = __ballot_sync(0xffffffffu, act);
      } else {
        const unsigned m0 = __ballot_sync(0xffffffffu, act);
        if (threadIdx.x == 0) mats64[0].mask = m0;
        __syncthreads();
        mask = mats64[0].mask;
        __syncthreads();
      }
      if (mask == 0u) continue;
      g::sync();
      // rows: A <- J^H A. new row p = c x_p - sigma x_q; new row q = conj(sigma) x_p + c x_q
      for (int j = 0; j < G; ++j) {
        const unsigned seg = (mask >> (j * HP)) & ((HP == 32) ? 0xffffffffu : ((1u << HP) - 1u));
        if (!seg) continue;
        rotated |= 1u << j;
        EigSmemDF<NP> &s = df(j);
        const int M = Ms[j];
        for (int it = lane; it < HP * M; it += T) {
          const int i = it / M, k = it % M;
          if (!((seg >> i) & 1u)) continue;
          const RotDF ro = s.rot[i];
          const int2 pq = mats64[j].pq[i];
          const float4 xp = s.a(pq.x, k), xq = s.a(pq.y, k);
          s.a(pq.x, k) = cplx(dot3(ro.c, re_of(xp), neg(ro.sr), re_of(xq), ro.si, im_of(xq)),
                              dot3(ro.c, im_of(xp), neg(ro.sr), im_of(xq), neg(ro.si), re_of(xq)));
          s.a(pq.y, k) = cplx(dot3(ro.c, re_of(xq), ro.sr, re_of(xp), ro.si, im_of(xp)),
                              dot3(ro.c, im_of(xq), ro.sr, im_of(xp), neg(ro.si), re_of(xp)));
        }
      }
      g::sync();
      // columns: A <- A J, V <- V J. new col p = c x_p - conj(sigma) x_q; new col q = sigma x_p + c x_q
      for (int j = 0; j < G; ++j) {
        const unsigned seg = (mask >> (j * HP)) & ((HP == 32) ? 0xffffffffu : ((1u << HP) - 1u));
        if (!seg) continue;
        EigSmemDF<NP> &s = df(j);
        const int M = Ms[j];
        for (int it = lane; it < HP * M; it += T) {
          const int i = it / M, k = it % M;
          if (!((seg >> i) & 1u)) continue;
          const RotDF ro = s.rot[i];
          const int2 pq = mats64[j].pq[i];
          const float4 xp = s.a(k, pq.x), xq = s.a(k, pq.y);
          s.a(k, pq.x) = cplx(dot3(ro.c, re_of(xp), neg(ro.sr), re_of(xq), neg(ro.si), im_of(xq)),
                              dot3(ro.c, im_of(xp), neg(ro.sr), im_of(xq), ro.si, re_of(xq)));
          s.a(k, pq.y) = cplx(dot3(ro.c, re_of(xq), ro.sr, re_of(xp), neg(ro.si), im_of(xp)),
                              dot3(ro.c, im_of(xq), ro.sr, im_of(xp), ro.si, re_of(xp)));
          const float4 vp = s.v(k, pq.x), vq = s.v(k, pq.y);
          s.v(k, pq.x) = cplx(dot3(ro.c, re_of(vp), neg(ro.sr), re_of(vq), neg(ro.si), im_of(vq)),
                              dot3(ro.c, im_of(vp), neg(ro.sr), im_of(vq), ro.si, re_of(vq)));
          s.v(k, pq.y) = cplx(dot3(ro.c, re_of(vq), ro.sr, re_of(vp), neg(ro.si), im_of(vp)),
                              dot3(ro.c, im_of(vq), ro.sr, im_of(vp), ro.si, re_of(vp)));
        }
      }
      g::sync();
      if (act) {   // the diagonal of a Hermitian matrix is real
        EigSmemDF<NP> &s = df(lj);
        const int2 pq = mats64[lj].pq[li];
        s.a(pq.x, pq.x).z = s.a(pq.x, pq.x).w = 0.f;
        s.a(pq.y, pq.y).z = s.a(pq.y, pq.y).w = 0.f;
      }
      g::sync();
    }
    for (int j = 0; j < G; ++j)
      if (((live >> j) & 1u) && !((rotated >> j) & 1u)) {
        res[j] = sweep;
        live &= ~(1u << j);
      }
  }
  for (int j = 0; j < G; ++j)
    if ((live >> j) & 1u) res[j] = -DOA_ENOCONV;
  // double-float -> FP64 in place (same bytes per element; every element has one owner lane)
  for (int j = 0; j < G; ++j) {
    const int M = Ms[j];
    if (M <= 0) continue;
    EigSmemDF<NP> &s = df(j);
    for (int e = lane; e < M * M; e += T) {
      const int i = e / M, k = e % M;
      const float4 a = s.a(i, k), v = s.v(i, k);
      mats64[j].a(i, k) = make_double2((double)a.x + (double)a.y, (double)a.z + (double)a.w);
      mats64[j].v(i, k) = make_double2((double)v.x + (double)v.y, (double)v.z + (double)v.w);
    }
  }
  g::sync();
}

// ---- One matrix of 33 <= M <= 64 on a cluster of four CTAs (double-float) ----
// The same rounds as jacobi_group_df with the rows of A and V spread over the cluster: CTA c owns
// rows 16c .. 16c+15 (one per warp). For a round's rotation J (n/2 disjoint pairs) the element
// (i, col) of J^H A J needs only rows i and partner(i) at the columns of col's pair, so warp w
// forms row i's new values pair by pair (lane j: columns p_j, q_j): first the row mix with the
// partner row (read through distributed shared memory when another CTA owns it), then the column
// mix, in the same double-float operations and order as the row and column passes of
// jacobi_group_df; V's rows take the column mix in place. A is double-buffered, so one cluster
// barrier per round orders every CTA's reads of the current buffer before the writes that reuse
// it. Warp 0 of every CTA forms the round's rotations from the same bytes with the same code, so
// every CTA takes the same decisions (rounds to skip, sweeps, convergence) and meets the same
// barriers.
constexpr int kClRanks = 4;                 // CTAs per matrix
constexpr int kClRows = 64 / kClRanks;      // rows of A and V owned by a CTA (one per warp)
constexpr int kClThreads = 32 * kClRows;
static_assert(kClThreads == grp_threads<64>(), "the cluster's rank 0 runs the M <= 64 finishing code");

struct ClusterDF {
  float4 A[2][kClRows][64];    // double-float (hi, lo) re, (hi, lo) im
  float4 V[kClRows][64];
  RotDF rot[2][32];            // the round's rotations, by round parity
  int2 pq[2][32];
  unsigned mask[2];
};

// Shared memory of a cluster kernel: the FP64 record that rank 0 finishes in, then the rows.
constexpr int kClFinBytes = (int)((sizeof(EigSmem<64>) + 15) / 16 * 16);
constexpr int kClSmemBytes = kClFinBytes + (int)sizeof(ClusterDF);

// Row mixes of A <- J^H A: row p of the pair becomes c x_p - sigma x_q, row q conj(sigma) x_p + c x_q.
__device__ __forceinline__ float4 mix_row_p(const RotDF &ro, float4 xp, float4 xq) {
  return cplx(dot3(ro.c, re_of(xp), neg(ro.sr), re_of(xq), ro.si, im_of(xq)),
              dot3(ro.c, im_of(xp), neg(ro.sr), im_of(xq), neg(ro.si), re_of(xq)));
}
__device__ __forceinline__ float4 mix_row_q(const RotDF &ro, float4 xp, float4 xq) {
  return cplx(dot3(ro.c, re_of(xq), ro.sr, re_of(xp), ro.si, im_of(xp)),
              dot3(ro.c, im_of(xq), ro.sr, im_of(xp), neg(ro.si), re_of(xp)));
}
// Column mix of A <- A J (and V <- V J): column p becomes c x_p - conj(sigma) x_q, column q
// sigma x_p + c x_q.
__device__ __forceinline__ void mix_cols(const RotDF &ro, float4 &xp, float4 &xq) {
  const float4 np = cplx(dot3(ro.c, re_of(xp), neg(ro.sr), re_of(xq), neg(ro.si), im_of(xq)),
                         dot3(ro.c, im_of(xp), neg(ro.sr), im_of(xq), ro.si, re_of(xq)));
  const float4 nq = cplx(dot3(ro.c, re_of(xq), ro.sr, re_of(xp), neg(ro.si), im_of(xp)),
                         dot3(ro.c, im_of(xq), ro.sr, im_of(xp), ro.si, re_of(xp)));
  xp = np;
  xq = nq;
}

// Cyclic Jacobi of the Hermitian M x M matrix R (FP64, row-major; the upper triangle is read) in
// double-float over the calling cluster. Returns the sweep count (> 0), -DOA_ENONFINITE or
// -DOA_ENOCONV, the same in every CTA; on a positive return rank 0's fin holds V and the diagonal
// of A in FP64 (the finishing code reads nothing else of A).
__device__ int jacobi_cluster_df(ClusterDF &w, EigSmem<64> &fin, int M, const double2 *__restrict__ R) {
  cg::cluster_group cl = cg::this_cluster();
  const int rank = (int)cl.block_rank();
  const int tid = threadIdx.x, wp = tid >> 5, lane = tid & 31;
  const int row = rank * kClRows + wp;
  // every CTA checks the whole upper triangle, so all reach the same verdict
  bool finite = true;
  for (int e = tid; e < M * M; e += kClThreads) {
    const int i = e / M, k = e % M;
    if (i > k) continue;
    const double2 v = R[e];
    finite = finite && isfinite(v.x) && (i == k || isfinite(v.y));
  }
  for (int e = tid; e < kClRows * 64; e += kClThreads) {
    const int li = e / 64, k = e % 64, i = rank * kClRows + li;
    float4 a = make_float4(0.f, 0.f, 0.f, 0.f), v = a;
    if (i < M && k < M) {
      double2 x;
      if (i <= k) {
        x = R[i * M + k];
      } else {
        x = R[k * M + i];
        x.y = -x.y;
      }
      if (i == k) x.y = 0.0;
      a = df_of(x);
      v.x = i == k ? 1.f : 0.f;
    }
    w.A[0][li][k] = a;
    w.A[1][li][k] = make_float4(0.f, 0.f, 0.f, 0.f);
    w.V[li][k] = v;
  }
  const bool ok = __syncthreads_and(finite) != 0;
  cl.sync();   // every CTA's rows are in place before the first remote read
  if (!ok) return -DOA_ENONFINITE;
  const int n = (M + 1) & ~1;
  int cur = 0, res = -DOA_ENOCONV;
  unsigned t = 0;   // rounds so far: the parity selects the rotation record
  for (int sweep = 1; sweep <= kMaxSweeps; ++sweep) {
    bool rotated = false;
    for (int r = 0; r < n - 1; ++r, ++t) {
      const int sl = (int)(t & 1u);
      if (wp == 0) {
        bool act = false;
        if (lane < n / 2) {
          const int a = rr_player(lane, r, n), b = rr_player(n - 1 - lane, r, n);
          const int p = min(a, b), q = max(a, b);
          w.pq[sl][lane] = make_int2(p, q);
          if (q < M) {
            const float4 *Ap = cl.map_shared_rank(&w.A[cur][p % kClRows][0], p / kClRows);
            const float4 *Aq = cl.map_shared_rank(&w.A[cur][q % kClRows][0], q / kClRows);
            RotDF ro;
            act = rotation_df_of(Ap[p], Aq[q], Ap[q], ro);
            if (act) w.rot[sl][lane] = ro;
          }
        }
        const unsigned m = __ballot_sync(0xffffffffu, act);
        if (lane == 0) w.mask[sl] = m;
      }
      __syncthreads();
      const unsigned mask = w.mask[sl];
      if (mask == 0u) continue;   // nothing written: the buffers stay as they are
      rotated = true;
      const int nxt = cur ^ 1;
      if (row < M && lane < n / 2) {
        const int2 pj = w.pq[sl][lane];
        float4 xp = w.A[cur][wp][pj.x], xq = w.A[cur][wp][pj.y];
        // the pair that holds this row: its position in the round-robin order, folded
        const int pos = row == 0 ? 0 : ((row - 1 - r) % (n - 1) + (n - 1)) % (n - 1) + 1;
        const int k = min(pos, n - 1 - pos);
        if ((mask >> k) & 1u) {
          const RotDF rk = w.rot[sl][k];
          const int2 pk = w.pq[sl][k];
          const int other = pk.x + pk.y - row;
          const float4 *Ao = cl.map_shared_rank(&w.A[cur][other % kClRows][0], other / kClRows);
          const float4 yp = Ao[pj.x], yq = Ao[pj.y];
          if (row == pk.x) {
            xp = mix_row_p(rk, xp, yp);
            xq = mix_row_p(rk, xq, yq);
          } else {
            xp = mix_row_q(rk, yp, xp);
            xq = mix_row_q(rk, yq, xq);
          }
        }
        if ((mask >> lane) & 1u) {
          const RotDF rj = w.rot[sl][lane];
          mix_cols(rj, xp, xq);
          float4 vp = w.V[wp][pj.x], vq = w.V[wp][pj.y];
          mix_cols(rj, vp, vq);
          w.V[wp][pj.x] = vp;
          w.V[wp][pj.y] = vq;
        }
        if (row == pj.x) xp.z = xp.w = 0.f;   // the diagonal of a Hermitian matrix is real
        if (row == pj.y) xq.z = xq.w = 0.f;
        w.A[nxt][wp][pj.x] = xp;
        w.A[nxt][wp][pj.y] = xq;
      }
      cl.sync();   // this round's writes are visible, and nobody still reads the old buffer
      cur = nxt;
    }
    if (!rotated) {
      res = sweep;
      break;
    }
  }
  if (res > 0 && rank == 0) {
    for (int e = tid; e < M * M; e += kClThreads) {
      const int i = e / M, k = e % M;
      const float4 v = cl.map_shared_rank(&w.V[i % kClRows][0], i / kClRows)[k];
      fin.v(i, k) = make_double2((double)v.x + (double)v.y, (double)v.z + (double)v.w);
      if (i == k) {
        const float4 a = cl.map_shared_rank(&w.A[cur][i % kClRows][0], i / kClRows)[i];
        fin.a(i, i) = make_double2((double)a.x + (double)a.y, (double)a.z + (double)a.w);
      }
    }
  }
  cl.sync();   // the other CTAs' rows stay in place until rank 0 has read them
  return res;
}

// Stable descending order of the eigenvalues (equal values keep index order).
template <int NP>
__device__ void sort_desc(int M, EigSmem<NP> &s) {
  constexpr int T = grp_threads<NP>();
  using g = Grp<T>;
  const int lane = g::id();
  for (int i = lane; i < M; i += T) s.lam()[i] = s.a(i, i).x;
  g::sync();
  // ranks form a permutation even for non-finite values (NaN ranks below every number)
  for (int i = lane; i < M; i += T) {
    const double li = isnan(s.lam()[i]) ? -INFINITY : s.lam()[i];
    int rank = 0;
    for (int j = 0; j < M; ++j) {
      const double lj = isnan(s.lam()[j]) ? -INFINITY : s.lam()[j];
      rank += (lj > li) || (lj == li && j < i);
    }
    s.order()[rank] = i;
  }
  g::sync();
}

// Writes B (column-major, ld M) of algorithm alg; returns 0 or a doa_status.
template <int NP>
__device__ int build_factor(int M, int d, int alg, EigSmem<NP> &s, double2 *__restrict__ B) {
  constexpr int T = grp_threads<NP>();
  using g = Grp<T>;
  const int lane = g::id();
  const int Kn = M - d;  // noise subspace dimension
  if (alg == DOA_PHD) {
    int col = s.order()[M - 1];
    for (int r = lane; r < M; r += T) B[r] = s.v(r, col);
    return 0;
  }
  if (alg == DOA_MUSIC || alg == DOA_EV) {
    bool bad = false;
    for (int e = lane; e < M * Kn; e += T) {
      int c = e / M, r = e % M;
      int col = s.order()[d + c];
      double2 v = s.v(r, col);
      if (alg == DOA_EV) {
        double l = s.lam()[col];
        if (!(l > 0.0)) {
          bad = true;
          v = make_double2(0.0, 0.0);
        } else {
          double w = 1.0 / sqrt(l);
          v.x *= w;
          v.y *= w;
        }
      }
      B[c * M + r] = v;
    }
    bad = g::any(bad);
    return bad ? DOA_ERANK : 0;
  }
  // MN: valph = P_n e1 / (e1^H P_n e1); (P_n e1)_r = sum_c V[r][c] conj(V[0][c]) over noise c
  double nrm = 0.0;
  for (int c = 0; c < Kn; ++c) {
    double2 g = s.v(0, s.order()[d + c]);
    nrm += g.x * g.x + g.y * g.y;
  }
  if (!(nrm > 0.0)) {
    for (int r = lane; r < M; r += T) B[r] = make_double2(0.0, 0.0);
    return DOA_ERANK;
  }
  const double inv = 1.0 / nrm;
  for (int r = lane; r < M; r += T) {
    double2 acc = make_double2(0.0, 0.0);
    for (int c = 0; c < Kn; ++c) {
      int col = s.order()[d + c];
      double2 v = s.v(r, col), g = s.v(0, col);
      // v * conj(g)
      acc.x += v.x * g.x + v.y * g.y;
      acc.y += v.y * g.x - v.x * g.y;
    }
    B[r] = make_double2(acc.x * inv, acc.y * inv);
  }
  return 0;
}

// FP64 check that the noise eigenvectors are orthonormal: max |E_n^H E_n - I| <= kOrthoTol.
constexpr double kOrthoTol = 1e-10;

template <int NP>
__device__ bool noise_orthonormal(int M, int d, EigSmem<NP> &s) {
  constexpr int T = grp_threads<NP>();
  using g = Grp<T>;
  const int lane = g::id();
  const int Kn = M - d;
  bool ok = true;
  for (int e = lane; e < Kn * Kn; e += T) {
    const int a = e / Kn, b = e % Kn;
    if (a > b) continue;
    const int ca = s.order()[d + a], cb = s.order()[d + b];
    double gr = 0.0, gi = 0.0;
    for (int r = 0; r < M; ++r) {   // conj(V[r][ca]) * V[r][cb]
      const double2 x = s.v(r, ca), y = s.v(r, cb);
      gr = fma(x.x, y.x, fma(x.y, y.y, gr));
      gi = fma(x.x, y.y, fma(-x.y, y.x, gi));
    }
    if (a == b) gr -= 1.0;
    ok = ok && fabs(gr) <= kOrthoTol && fabs(gi) <= kOrthoTol;
  }
  return g::all(ok);
}

// Model-order estimates (Wax and Kailath's criteria for complex data) from the sorted eigenvalues:
// for k assumed sources, L(k) = N (M-k) log(a/g) over the M-k smallest eigenvalues (arithmetic and
// geometric means; +inf when one is not positive), MDL(k) = L + k(2M-k) log(N)/2, AIC(k) = 2L +
// 2k(2M-k); out[0] = argmin MDL, out[1] = argmin AIC (the smaller k on a tie). The group's lanes
// take one k each; the criterion values go to the A matrix's first row (no longer needed here).
template <int NP>
__device__ void model_order(int M, int N, EigSmem<NP> &s, int32_t *out) {
  constexpr int T = grp_threads<NP>();
  using g = Grp<T>;
  const int lane = g::id();
  const double logN = log((double)N);
  for (int k = lane; k < M; k += T) {
    const int n = M - k;
    double sum = 0.0, ls = 0.0;
    bool bad = false;
    for (int i = k; i < M; ++i) {
      const double l = s.lam()[s.order()[i]];
      sum += l;
      if (l > 0.0) ls += log(l); else bad = true;
    }
    const double L = bad ? CUDART_INF : (double)N * (double)n * (log(sum / (double)n) - ls / (double)n);
    const double pen = (double)k * (double)(2 * M - k);
    s.a(0, k) = make_double2(L + 0.5 * pen * logN, 2.0 * L + 2.0 * pen);
  }
  g::sync();
  if (lane == 0) {
    int bm = 0, ba = 0;
    double vm = CUDART_INF, va = CUDART_INF;
    for (int k = 0; k < M; ++k) {
      const double2 v = s.a(0, k);
      if (v.x < vm) {
        vm = v.x;
        bm = k;
      }
      if (v.y < va) {
        va = v.y;
        ba = k;
      }
    }
    out[0] = bm;
    out[1] = ba;
  }
  g::sync();
}

// Writes a batch problem's scan factor F (columns as laid out by the plan: E_n, or v_min; then
// valph) and the EV weights w_c = 1 / lambda_{d+c}; returns 0 or a doa_status.
template <int NP>
__device__ int build_scan_factor(const PlanProblem &pp, EigSmem<NP> &s, double2 *__restrict__ F,
                                 double *__restrict__ w) {
  constexpr int T = grp_threads<NP>();
  using g = Grp<T>;
  const int lane = g::id();
  const int M = pp.p.M, d = pp.p.d;
  int st = 0;
  if (pp.Kn > 0) {
    build_factor<NP>(M, d, DOA_MUSIC, s, F);
    if (pp.slot[DOA_EV] >= 0) {
      bool bad = false;
      for (int c = lane; c < pp.Kn; c += T) {
        const double l = s.lam()[s.order()[d + c]];
        bad = bad || !(l > 0.0);
        w[c] = l > 0.0 ? 1.0 / l : 0.0;
      }
      if (g::any(bad)) st = DOA_ERANK;
    }
  } else if (pp.kphd >= 0) {
    build_factor<NP>(M, d, DOA_PHD, s, F + (size_t)pp.kphd * M);
  }
  if (pp.kmn >= 0) {
    const int e = build_factor<NP>(M, d, DOA_MN, s, F + (size_t)pp.kmn * M);
    if (e && !st) st = e;
  }
  return st;
}

// The eigenvalues, B and the status of a single call from a finished decomposition (res: the
// sweep count, or minus a doa_status).
template <int NP>
__device__ void finish_single(int M, int d, int alg, EigSmem<NP> &s, int res, double *evals, double2 *B, int *K_out,
                              int *info) {
  constexpr int T = grp_threads<NP>();
  const int lane = Grp<T>::id();
  int st = 0;
  if (res > 0) {
    sort_desc<NP>(M, s);
    if (evals)
      for (int i = lane; i < M; i += T) evals[i] = s.lam()[s.order()[i]];
    st = build_factor<NP>(M, d, alg, s, B);
  } else {
    st = -res;
  }
  if (lane == 0) {
    *info = st ? -st : res;
    if (K_out) *K_out = (alg == DOA_PHD || alg == DOA_MN) ? 1 : M - d;
  }
}

template <int NP, bool kDF>
__global__ void __launch_bounds__(grp_threads<NP>()) eig_single_kernel(const double2 *R64, int M, int d, int alg, double *evals,
                                                       double2 *B, int *K_out, int *info) {
  extern __shared__ __align__(16) uint8_t smem[];
  constexpr int G = mats_per_warp<NP>();
  EigSmem<NP> *mats = reinterpret_cast<EigSmem<NP> *>(smem);
  int Ms[G];
  const double2 *Rs[G];
  int res[G];
  for (int j = 0; j < G; ++j) {
    Ms[j] = j == 0 ? M : 0;
    Rs[j] = R64;
  }
  if (kDF)
    jacobi_group_df<NP, G>(mats, Ms, Rs, res);
  else
    jacobi_group<NP, G>(mats, Ms, Rs, res);
  finish_single<NP>(M, d, alg, mats[0], res[0], evals, B, K_out, info);
}

// Single call, 33 <= M <= 64, double-float: one four-CTA cluster; rank 0 finishes.
__global__ void __cluster_dims__(kClRanks, 1, 1) __launch_bounds__(kClThreads, 1)
    eig_cluster_single_kernel(const double2 *R64, int M, int d, int alg, double *evals, double2 *B, int *K_out,
                              int *info) {
  extern __shared__ __align__(16) uint8_t smem[];
  EigSmem<64> &s = *reinterpret_cast<EigSmem<64> *>(smem);
  ClusterDF &w = *reinterpret_cast<ClusterDF *>(smem + kClFinBytes);
  const int res = jacobi_cluster_df(w, s, M, R64);
  if (cg::this_cluster().block_rank() != 0) return;
  finish_single<64>(M, d, alg, s, res, evals, B, K_out, info);
}

// A batch problem's outputs from its finished decomposition (res: the sweep count, or minus a
// doa_status): evals, the scan factor and EV weights, the optional B, order estimates and
// proposal features, and the status.
template <int NP>
__device__ void finish_batch(const PlanProblem &pp, const PlanJob *jobs, EigSmem<NP> &s, int res, uint8_t *ws,
                             int *status) {
  constexpr int T = grp_threads<NP>();
  const int lane = Grp<T>::id();
  const int M = pp.p.M, d = pp.p.d;
  int st = 0;
  if (pp.p.features) {
    // proposal-network input: upper triangle of R / tr(R), (re, im) pairs row by row
    const double2 *R = reinterpret_cast<const double2 *>(ws + pp.r64_off);
    double tr = 0.0;
    for (int i = 0; i < M; ++i) tr += R[i * M + i].x;
    const double inv = tr > 0.0 ? 1.0 / tr : 0.0;
    for (int e = lane; e < M * (M + 1) / 2; e += T) {
      int i = 0, rem = e;
      while (rem >= M - i) { rem -= M - i; ++i; }
      const double2 v = R[i * M + i + rem];
      pp.p.features[2 * e] = (float)(v.x * inv);
      pp.p.features[2 * e + 1] = (float)(v.y * inv);
    }
  }
  double2 *F = reinterpret_cast<double2 *>(ws + pp.fac_off);
  double *w = reinterpret_cast<double *>(F + (size_t)M * (M + 1));
  if (res > 0) {
    sort_desc<NP>(M, s);
    if (pp.p.evals)
      for (int i = lane; i < M; i += T) pp.p.evals[i] = s.lam()[s.order()[i]];
    st = build_scan_factor<NP>(pp, s, F, w);
    if (!noise_orthonormal<NP>(M, d, s) && !st) st = DOA_ENOCONV;
    if (pp.p.B_out) build_factor<NP>(M, d, jobs[pp.first_job].alg, s, reinterpret_cast<double2 *>(pp.p.B_out));
    if (pp.p.order_est) {
      Grp<T>::sync();
      model_order<NP>(M, pp.p.N, s, pp.p.order_est);
    }
  } else {
    st = -res;
    // a failed decomposition leaves a zero factor, so the scan writes the 1/FLT_MIN sentinel
    for (int e = lane; e < M * pp.Kf; e += T) F[e] = make_double2(0.0, 0.0);
    for (int e = lane; e < pp.Kn; e += T) w[e] = 0.0;
  }
  if (lane == 0) *status = st;
  Grp<T>::sync();
}

template <int NP, int G>
__global__ void __launch_bounds__(32 * eig_warps<NP>(), eig_min_ctas<NP>()) eig_batch_kernel(const uint8_t *plan, uint8_t *ws, int bucket,
                                                                         int *status) {
  extern __shared__ __align__(16) uint8_t smem[];
  constexpr int T = grp_threads<NP>();
  const int grp = threadIdx.x / T, lane = Grp<T>::id();
  EigSmem<NP> *mats = reinterpret_cast<EigSmem<NP> *>(smem) + grp * G;
  const PlanHeader *h = reinterpret_cast<const PlanHeader *>(plan);
  const int base = (blockIdx.x * (int)(blockDim.x / T) + grp) * G;
  const int count = h->eig_count[bucket];
  if (base >= count) return;
  const int32_t *list = reinterpret_cast<const int32_t *>(plan + h->off_eig[bucket]);
  const PlanProblem *probs = reinterpret_cast<const PlanProblem *>(plan + h->off_prob);
  const PlanJob *jobs = reinterpret_cast<const PlanJob *>(plan + h->off_job);
  int Ms[G], prob[G], res[G];
  const double2 *Rs[G];
  for (int j = 0; j < G; ++j) {
    prob[j] = base + j < count ? list[base + j] : -1;
    Ms[j] = prob[j] >= 0 ? probs[prob[j]].p.M : 0;
    Rs[j] = prob[j] >= 0 ? reinterpret_cast<const double2 *>(ws + probs[prob[j]].r64_off) : nullptr;
  }
  bool fp64 = false;   // a group runs FP64 when any of its problems asks for it
  for (int j = 0; j < G; ++j) fp64 = fp64 || (prob[j] >= 0 && probs[prob[j]].p.eig_prec == DOA_EIG_FP64);
  if (fp64)
    jacobi_group<NP, G>(mats, Ms, Rs, res);
  else
    jacobi_group_df<NP, G>(mats, Ms, Rs, res);
  for (int j = 0; j < G; ++j) {
    if (prob[j] < 0) continue;
    finish_batch<NP>(probs[prob[j]], jobs, mats[j], res[j], ws, status + prob[j]);
  }
}

// Bucket M <= 64 of the batch in double-float: one four-CTA cluster per problem; rank 0 finishes.
// A problem that asks for the FP64 Jacobi runs it in rank 0 alone (the other CTAs leave at once).
__global__ void __cluster_dims__(kClRanks, 1, 1) __launch_bounds__(kClThreads, 1)
    eig_cluster_batch_kernel(const uint8_t *plan, uint8_t *ws, int bucket, int *status) {
  extern __shared__ __align__(16) uint8_t smem[];
  EigSmem<64> &s = *reinterpret_cast<EigSmem<64> *>(smem);
  ClusterDF &w = *reinterpret_cast<ClusterDF *>(smem + kClFinBytes);
  const PlanHeader *h = reinterpret_cast<const PlanHeader *>(plan);
  const int idx = (int)(blockIdx.x / kClRanks);   // the same for every CTA of the cluster
  if (idx >= h->eig_count[bucket]) return;
  const int32_t *list = reinterpret_cast<const int32_t *>(plan + h->off_eig[bucket]);
  const PlanProblem *probs = reinterpret_cast<const PlanProblem *>(plan + h->off_prob);
  const PlanJob *jobs = reinterpret_cast<const PlanJob *>(plan + h->off_job);
  const int prob = list[idx];
  const PlanProblem &pp = probs[prob];
  const double2 *R = reinterpret_cast<const double2 *>(ws + pp.r64_off);
  const bool rank0 = cg::this_cluster().block_rank() == 0;
  int res;
  if (pp.p.eig_prec == DOA_EIG_FP64) {
    if (!rank0) return;
    int Ms[1] = {pp.p.M}, r1[1];
    const double2 *Rs[1] = {R};
    jacobi_group<64, 1>(&s, Ms, Rs, r1);
    res = r1[0];
  } else {
    res = jacobi_cluster_df(w, s, pp.p.M, R);
    if (!rank0) return;
  }
  finish_batch<64>(pp, jobs, s, res, ws, status + prob);
}


template <int NP, bool kDF>
cudaError_t run_single_p(const double2 *R64, int M, int d, int alg, double *evals, double2 *B, int *K_out,
                         int *info, cudaStream_t st) {
  const int smem = (int)sizeof(EigSmem<NP>) * mats_per_warp<NP>();
  cudaError_t e = ensure_smem_attr((const void *)eig_single_kernel<NP, kDF>, smem);
  if (e != cudaSuccess) return e;
  eig_single_kernel<NP, kDF><<<1, grp_threads<NP>(), smem, st>>>(R64, M, d, alg, evals, B, K_out, info);
  return cudaGetLastError();
}

cudaError_t run_single_cluster(const double2 *R64, int M, int d, int alg, double *evals, double2 *B, int *K_out,
                               int *info, cudaStream_t st) {
  cudaError_t e = ensure_smem_attr(reinterpret_cast<const void *>(eig_cluster_single_kernel), kClSmemBytes);
  if (e != cudaSuccess) return e;
  eig_cluster_single_kernel<<<kClRanks, kClThreads, kClSmemBytes, st>>>(R64, M, d, alg, evals, B, K_out, info);
  return cudaGetLastError();
}

template <int NP>
cudaError_t run_single(const double2 *R64, int M, int d, int alg, int prec, double *evals, double2 *B, int *K_out,
                       int *info, cudaStream_t st) {
  if (prec == DOA_EIG_FP64) return run_single_p<NP, false>(R64, M, d, alg, evals, B, K_out, info, st);
  if constexpr (NP == 64)
    return run_single_cluster(R64, M, d, alg, evals, B, K_out, info, st);
  else
    return run_single_p<NP, true>(R64, M, d, alg, evals, B, K_out, info, st);
}

// Warps per CTA: the count (up to eig_warps) that keeps the most matrices resident per SM, the
// larger count on a tie. Shared memory is the limit (each CTA also costs the driver's reserve),
// so for M <= 16, nine one-matrix warps per CTA hold 27 matrices per SM where two held 24: a
// 4096-matrix batch then runs in one wave instead of 1.12.
template <int NP, int G>
int eig_cta_warps() {
  if (NP > 32) return 1;
  const SmemLimits lim = device_smem_limits();
  const int per_mat = (int)sizeof(EigSmem<NP>);
  int best = 1, best_res = -1;
  for (int w = 1; w <= eig_warps<NP>(); ++w) {
    const int bytes = w * G * per_mat;
    if (bytes > lim.per_block) break;
    const int ctas = lim.per_sm / (bytes + lim.reserve);
    if (ctas * w * G >= best_res) {
      best_res = ctas * w * G;
      best = w;
    }
  }
  return best;
}

template <int NP, int G>
cudaError_t run_batch_g(const uint8_t *plan, int count, uint8_t *ws, int *status, int bucket, cudaStream_t st) {
  const int W = NP <= 32 ? eig_cta_warps<NP, G>() : eig_warps<NP>();
  const int per_cta = (NP <= 32 ? W : 1) * G;
  const int smem = (int)sizeof(EigSmem<NP>) * per_cta;
  cudaError_t e = ensure_smem_attr(reinterpret_cast<const void *>(eig_batch_kernel<NP, G>), smem);
  if (e != cudaSuccess) return e;
  eig_batch_kernel<NP, G><<<(count + per_cta - 1) / per_cta, 32 * W, smem, st>>>(plan, ws, bucket, status);
  return cudaGetLastError();
}

// Matrices per warp from the plan (G in {1, 2, 4, 8} up to the bucket's maximum).
template <int NP>
cudaError_t run_batch(const uint8_t *plan, const PlanHeader &h, uint8_t *ws, int *status, int bucket,
                      cudaStream_t st) {
  const int count = h.eig_count[bucket];
  if (count == 0) return cudaSuccess;
  const int g = h.eig_mats[bucket];
  if (g >= 8 && mats_per_warp<NP>() >= 8) return run_batch_g<NP, (mats_per_warp<NP>() >= 8 ? 8 : 1)>(plan, count, ws, status, bucket, st);
  if (g >= 4 && mats_per_warp<NP>() >= 4) return run_batch_g<NP, (mats_per_warp<NP>() >= 4 ? 4 : 1)>(plan, count, ws, status, bucket, st);
  if (g >= 2 && mats_per_warp<NP>() >= 2) return run_batch_g<NP, (mats_per_warp<NP>() >= 2 ? 2 : 1)>(plan, count, ws, status, bucket, st);
  return run_batch_g<NP, 1>(plan, count, ws, status, bucket, st);
}

// Bucket M <= 64: one four-CTA cluster per problem.
cudaError_t run_batch_cluster(const uint8_t *plan, const PlanHeader &h, uint8_t *ws, int *status, int bucket,
                              cudaStream_t st) {
  const int count = h.eig_count[bucket];
  if (count == 0) return cudaSuccess;
  cudaError_t e = ensure_smem_attr(reinterpret_cast<const void *>(eig_cluster_batch_kernel), kClSmemBytes);
  if (e != cudaSuccess) return e;
  eig_cluster_batch_kernel<<<(unsigned)count * kClRanks, kClThreads, kClSmemBytes, st>>>(plan, ws, bucket, status);
  return cudaGetLastError();
}

}  // namespace

namespace {
__global__ void __launch_bounds__(32) model_order_single_kernel(const double *evals, int M, int N, int *mdl, int *aic) {
  __shared__ double2 v[kMaxM];
  const int lane = threadIdx.x;
  const double logN = log((double)N);
  for (int k = lane; k < M; k += 32) {
    const int n = M - k;
    double sum = 0.0, ls = 0.0;
    bool bad = false;
    for (int i = k; i < M; ++i) {
      const double l = evals[i];
      sum += l;
      if (l > 0.0) ls += log(l); else bad = true;
    }
    const double L = bad ? CUDART_INF : (double)N * (double)n * (log(sum / (double)n) - ls / (double)n);
    const double pen = (double)k * (double)(2 * M - k);
    v[k] = make_double2(L + 0.5 * pen * logN, 2.0 * L + 2.0 * pen);
  }
  __syncwarp();
  if (lane == 0) {
    int bm = 0, ba = 0;
    double vm = CUDART_INF, va = CUDART_INF;
    for (int k = 0; k < M; ++k) {
      if (v[k].x < vm) {
        vm = v[k].x;
        bm = k;
      }
      if (v[k].y < va) {
        va = v[k].y;
        ba = k;
      }
    }
    if (mdl) *mdl = bm;
    if (aic) *aic = ba;
  }
}
}  // namespace

cudaError_t launch_model_order_single(const double *evals, int M, int N, int *mdl, int *aic, cudaStream_t s) {
  model_order_single_kernel<<<1, 32, 0, s>>>(evals, M, N, mdl, aic);
  return cudaGetLastError();
}

cudaError_t launch_eig_single(const double2 *R64, int M, int d, int alg, int prec, double *evals, double2 *B,
                              int *K_out, int *info, cudaStream_t s) {
  switch (m_bucket(M)) {
    case 0: return run_single<8>(R64, M, d, alg, prec, evals, B, K_out, info, s);
    case 1: return run_single<16>(R64, M, d, alg, prec, evals, B, K_out, info, s);
    case 2: return run_single<32>(R64, M, d, alg, prec, evals, B, K_out, info, s);
    default: return run_single<64>(R64, M, d, alg, prec, evals, B, K_out, info, s);
  }
}

cudaError_t launch_eig_batch(const uint8_t *plan_dev, const PlanHeader &h, uint8_t *ws, int *status,
                             cudaStream_t s) {
  cudaError_t e;
  if ((e = run_batch<8>(plan_dev, h, ws, status, 0, s)) != cudaSuccess) return e;
  if ((e = run_batch<16>(plan_dev, h, ws, status, 1, s)) != cudaSuccess) return e;
  if ((e = run_batch<32>(plan_dev, h, ws, status, 2, s)) != cudaSuccess) return e;
  return run_batch_cluster(plan_dev, h, ws, status, 3, s);
}

}  // namespace doa
