// C ABI of libdoa.so (declarations and contracts in include/doa.h): argument checks, batch
// planning on the host, and the launch sequences. No entry point allocates memory or
// synchronises; every launch goes to the caller's stream.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <functional>
#include <unordered_map>
#include <vector>

#include "doa_internal.cuh"

using namespace doa;

namespace {

inline cudaStream_t as_stream(void *s) { return reinterpret_cast<cudaStream_t>(s); }
inline bool aligned(const void *p, size_t a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; }
inline int64_t round_up(int64_t x, int64_t a) { return (x + a - 1) / a * a; }
inline doa_status cuda_status(cudaError_t e) { return e == cudaSuccess ? DOA_OK : DOA_ECUDA; }

// Columns of a problem's scan factor F (see PlanProblem): E_n when MUSIC or EV is requested (PHD
// then reads its last column), else v_min for PHD; plus valph for MN.
void factor_layout(const doa_problem &p, PlanProblem &q) {
  const unsigned m = p.alg_mask;
  const bool en = (m >> DOA_MUSIC) & 1u || (m >> DOA_EV) & 1u;
  int k = 0;
  q.Kn = 0;
  q.kphd = q.kmn = -1;
  if (en) {
    q.Kn = p.M - p.d;
    k = q.Kn;
    if ((m >> DOA_PHD) & 1u) q.kphd = q.Kn - 1;
  } else if ((m >> DOA_PHD) & 1u) {
    q.kphd = k++;
  }
  if ((m >> DOA_MN) & 1u) q.kmn = k++;
  q.Kf = k;
}

bool grid_ok(const doa_grid &g) {
  return g.L >= 3 && g.L <= (1 << 30) && std::isfinite(g.lo_deg) && std::isfinite(g.step_deg) &&
         g.step_deg != 0.0;
}

// Azimuth columns and geometry of a 2-D scan (doa_geometry): sizes, finite angles, positions.
bool geometry_ok(const doa_grid &az, const doa_geometry &g) {
  const int64_t La = az.L, Le = g.Le;
  if (!g.pos || !aligned(g.pos, 8) || La < 1 || Le < 1 || La > (1 << 24) || Le > (1 << 24) || La * Le > (1 << 30))
    return false;
  if (!std::isfinite(az.lo_deg) || !std::isfinite(az.step_deg) || !std::isfinite(g.el_lo_deg) ||
      !std::isfinite(g.el_step_deg))
    return false;
  return g.wrap_az == 0 || g.wrap_az == 1;
}

bool problem_ok(const doa_problem &p) {
  if (p.M < 2 || p.M > kMaxM || p.d < 0 || p.d >= p.M || p.N < 1 || p.ldx < p.N) return false;
  if (!p.X || !aligned(p.X, 8) || !p.P || !aligned(p.P, 4)) return false;
  if (p.alg_mask == 0u || p.alg_mask > 15u) return false;
  if (p.eig_prec != DOA_EIG_DOUBLE_FLOAT && p.eig_prec != DOA_EIG_FP64) return false;
  if (p.flags & ~(DOA_FLAG_POLISH_PEAKS | DOA_FLAG_COV_CUDA_CORE)) return false;
  if (p.d > 0 && (!p.peak_idx || !p.peak_val)) return false;
  if (p.peak_angle && !aligned(p.peak_angle, 8)) return false;
  if (p.order_est && !aligned(p.order_est, 4)) return false;
  if (p.root_angle && (!aligned(p.root_angle, 8) || p.geom.pos || p.d < 1)) return false;
  if (!p.peak_count) return false;
  if (p.geom.pos)   // 2-D scan: FP32 on CUDA cores, no peak polish
    return p.prec == DOA_FP32 && (p.flags & DOA_FLAG_POLISH_PEAKS) == 0 && geometry_ok(p.grid, p.geom);
  // scan form: FP32 (CUDA cores) or split operands on the tensor cores (M <= 32)
  if (p.prec != DOA_FP32 && !((p.prec == DOA_BF16X3 || p.prec == DOA_FP16X3) && p.M <= kTcBatchMaxM)) return false;
  return grid_ok(p.grid);
}

// Covariance on the tensor cores (exact BF16 slices, covariance_tc_batch.cu): M <= 16, whole-row
// bulk copies (16-byte aligned X, even row stride), N within the range of its 64-bit sums.
bool cov_tc_ok(const doa_problem &p) {
  return p.M <= kCovTcMaxM && !(p.flags & DOA_FLAG_COV_CUDA_CORE) && aligned(p.X, 16) && (p.ldx & 1) == 0 &&
         p.N <= kCovTcMaxN;
}
int cov_tc_class(int M) { return M <= 8 ? 0 : 1; }

int64_t spectrum_points(const doa_problem &p) {
  return p.geom.pos ? (int64_t)p.grid.L * p.geom.Le : (int64_t)p.grid.L;
}

struct PlanSizes {
  int nprob = 0, njobs = 0, ngrids = 0, ncov = 0, nreduce = 0;
  int cov_class[kCovClasses] = {0, 0, 0, 0};
  int covtc[2] = {0, 0};
  int tc = 0;
  int eig[kNumBuckets] = {0, 0, 0, 0};
  int scan[kNumBuckets] = {0, 0, 0, 0};
  int geo[kNumBuckets] = {0, 0, 0, 0};
  int ngeo_grids = 0;
  int ngeo_steer = 0;
};

// A geometry problem's azimuth x elevation grid (the key of its trigonometric tables).
struct GeoGridKey {
  doa_grid az;
  double el_lo, el_step;
  int32_t Le;
};

// Bit-exact key of a grid (azimuth or ULA grid, plus the elevation rows of a 2-D grid): two grids
// share their tables only when every double matches bit for bit.
struct GridHash {
  uint64_t lo, step, el_lo, el_step;
  int32_t L, Le;
  bool operator==(const GridHash &o) const {
    return lo == o.lo && step == o.step && el_lo == o.el_lo && el_step == o.el_step && L == o.L && Le == o.Le;
  }
  struct Hasher {
    size_t operator()(const GridHash &k) const {
      uint64_t h = 0x9e3779b97f4a7c15ull;
      for (uint64_t v : {k.lo, k.step, k.el_lo, k.el_step, ((uint64_t)(uint32_t)k.L << 32) | (uint32_t)k.Le})
        h = (h ^ v) * 0x100000001b3ull + (h >> 29);
      return (size_t)h;
    }
  };
};

GridHash grid_hash(const doa_grid &g, double el_lo, double el_step, int32_t Le) {
  GridHash k{};
  std::memcpy(&k.lo, &g.lo_deg, 8);
  std::memcpy(&k.step, &g.step_deg, 8);
  std::memcpy(&k.el_lo, &el_lo, 8);
  std::memcpy(&k.el_step, &el_step, 8);
  k.L = g.L;
  k.Le = Le;
  return k;
}

// Geometry problems that pass the same positions pointer with the same grid and M share one FP32
// steering table (when at least two do, and the table is at most kSteerMaxBytes).
struct SteerKey {
  const double *pos;
  int geo_grid, M, count;
};
constexpr int64_t kSteerMaxBytes = int64_t(1) << 28;

struct SteerHash {
  uintptr_t pos;
  int geo_grid, M;
  bool operator==(const SteerHash &o) const { return pos == o.pos && geo_grid == o.geo_grid && M == o.M; }
  struct Hasher {
    size_t operator()(const SteerHash &k) const {
      return std::hash<uintptr_t>()(k.pos) ^ (std::hash<int64_t>()(((int64_t)k.geo_grid << 8) | k.M) * 0x9e3779b97f4a7c15ull);
    }
  };
};

int64_t steer_ldt(const GeoGridKey &g) { return round_up((int64_t)g.az.L * g.Le, kSteerAlign); }
int steer_rows(int M) { return 8 << m_bucket(M); }

// Counts the plan's arrays; returns false on an invalid problem. steer_of[i]: the shared steering
// table of geometry problem i, or -1.
bool count_plan(const doa_problem *probs, int nprob, PlanSizes &sz, std::vector<doa_grid> &grids,
                std::vector<int> &grid_of, std::vector<GeoGridKey> &geo_grids, std::vector<SteerKey> &steers,
                std::vector<int> &steer_of, int *bad_index) {
  sz.nprob = nprob;
  grid_of.resize(nprob);
  steer_of.assign(nprob, -1);
  std::unordered_map<SteerHash, int, SteerHash::Hasher> steer_index;
  std::unordered_map<GridHash, int, GridHash::Hasher> grid_index, geo_index;
  for (int i = 0; i < nprob; ++i) {
    const doa_problem &p = probs[i];
    if (!problem_ok(p)) {
      if (bad_index) *bad_index = i;
      return false;
    }
    if (cov_tc_ok(p)) {
      sz.covtc[cov_tc_class(p.M)] += 1;
    } else {
      int chunks = (p.N + kCovChunk - 1) / kCovChunk;
      sz.ncov += chunks;
      sz.cov_class[cov_class(p.M)] += chunks;
      sz.nreduce += chunks > 1;
    }
    sz.eig[m_bucket(p.M)] += 1;
    sz.njobs += __builtin_popcount(p.alg_mask);
    if (p.geom.pos) {   // 2-D scan: trigonometric tables of its azimuth x elevation grid
      sz.geo[m_bucket(p.M)] += 1;
      const GridHash gkey = grid_hash(p.grid, p.geom.el_lo_deg, p.geom.el_step_deg, p.geom.Le);
      auto git = geo_index.find(gkey);
      int g;
      if (git == geo_index.end()) {
        g = (int)geo_grids.size();
        geo_grids.push_back(GeoGridKey{p.grid, p.geom.el_lo_deg, p.geom.el_step_deg, p.geom.Le});
        geo_index.emplace(gkey, g);
      } else {
        g = git->second;
      }
      grid_of[i] = g;
      // (pointer, grid, M) -> key index; a hash map, since every problem may bring its own pointer
      const SteerHash key{reinterpret_cast<uintptr_t>(p.geom.pos), g, p.M};
      auto it = steer_index.find(key);
      int st;
      if (it == steer_index.end()) {
        st = (int)steers.size();
        steers.push_back(SteerKey{p.geom.pos, g, p.M, 0});
        steer_index.emplace(key, st);
      } else {
        st = it->second;
      }
      ++steers[st].count;
      steer_of[i] = st;
      continue;
    }
    if (p.prec == DOA_FP32)
      sz.scan[m_bucket(p.M)] += 1;
    else
      sz.tc += 1;
    const GridHash ukey = grid_hash(p.grid, 0.0, 0.0, 0);
    auto uit = grid_index.find(ukey);
    int g;
    if (uit == grid_index.end()) {
      g = (int)grids.size();
      grids.push_back(p.grid);
      grid_index.emplace(ukey, g);
    } else {
      g = uit->second;
    }
    grid_of[i] = g;
  }
  sz.ngrids = (int)grids.size();
  sz.ngeo_grids = (int)geo_grids.size();
  // keep the tables that two or more problems read; renumber them in order of first use
  std::vector<int> keep(steers.size(), -1);
  std::vector<SteerKey> kept;
  for (size_t k = 0; k < steers.size(); ++k) {
    const SteerKey &t = steers[k];
    if (t.count >= 2 && 8 * steer_rows(t.M) * steer_ldt(geo_grids[t.geo_grid]) <= kSteerMaxBytes &&
        kept.size() < 65535) {   // one grid row of the table kernel per table
      keep[k] = (int)kept.size();
      kept.push_back(t);
    }
  }
  for (int i = 0; i < nprob; ++i)
    if (steer_of[i] >= 0) steer_of[i] = keep[steer_of[i]];
  steers.swap(kept);
  sz.ngeo_steer = (int)steers.size();
  return true;
}

struct PlanOffsets {
  int64_t prob, job, grid, cov, reduce, eig[kNumBuckets], scan[kNumBuckets], tc, geo[kNumBuckets], geo_grid,
      geo_steer, covtc[2], sg[kNumBuckets], sgl[kNumBuckets], tcg, tcc, tcgl, total;
};

PlanOffsets plan_offsets(const PlanSizes &sz) {
  PlanOffsets o;
  int64_t at = round_up(sizeof(PlanHeader), 16);
  o.prob = at;
  at = round_up(at + (int64_t)sz.nprob * sizeof(PlanProblem), 16);
  o.job = at;
  at = round_up(at + (int64_t)sz.njobs * sizeof(PlanJob), 16);
  o.grid = at;
  at = round_up(at + (int64_t)sz.ngrids * sizeof(PlanGrid), 16);
  o.cov = at;
  at = round_up(at + (int64_t)sz.ncov * sizeof(PlanCovItem), 16);
  o.reduce = at;
  at = round_up(at + (int64_t)sz.nreduce * 4, 16);
  for (int b = 0; b < kNumBuckets; ++b) {
    o.eig[b] = at;
    at = round_up(at + (int64_t)sz.eig[b] * 4, 16);
  }
  for (int b = 0; b < kNumBuckets; ++b) {
    o.scan[b] = at;
    at = round_up(at + (int64_t)sz.scan[b] * 4, 16);
  }
  o.tc = at;
  at = round_up(at + (int64_t)sz.tc * 4, 16);
  for (int b = 0; b < kNumBuckets; ++b) {
    o.geo[b] = at;
    at = round_up(at + (int64_t)sz.geo[b] * 4, 16);
  }
  o.geo_grid = at;
  at = round_up(at + (int64_t)sz.ngeo_grids * sizeof(PlanGeoGrid), 16);
  o.geo_steer = at;
  at = round_up(at + (int64_t)sz.ngeo_steer * sizeof(PlanGeoSteer), 16);
  for (int c = 0; c < 2; ++c) {
    o.covtc[c] = at;
    at = round_up(at + (int64_t)sz.covtc[c] * 4, 16);
  }
  // grid-shared scan groups and lists: room for every FP32 ULA problem of the bucket (the grouping
  // depends on the tuning, the plan size must not)
  for (int b = 0; b < kNumBuckets; ++b) {
    o.sg[b] = at;
    at = round_up(at + (int64_t)sz.scan[b] * sizeof(PlanScanGroup), 16);
    o.sgl[b] = at;
    at = round_up(at + (int64_t)sz.scan[b] * 4, 16);
  }
  // grid-shared tensor-core scan: room for every split-precision ULA problem
  o.tcg = at;
  at = round_up(at + (int64_t)sz.tc * sizeof(PlanTcGroup), 16);
  o.tcc = at;
  at = round_up(at + (int64_t)sz.tc * sizeof(PlanTcChunk), 16);
  o.tcgl = at;
  at = round_up(at + (int64_t)sz.tc * 4, 16);
  o.total = at;
  return o;
}

}  // namespace

extern "C" {

const char *doa_status_str(int status) {
  switch (status) {
    case DOA_OK: return "ok";
    case DOA_EINVAL: return "invalid argument";
    case DOA_ENOMEM: return "workspace or plan buffer too small";
    case DOA_ECUDA: return "CUDA launch or runtime error";
    case DOA_ENOCONV: return "Jacobi sweep cap reached";
    case DOA_ERANK: return "noise subspace rank failure";
    case DOA_ENONFINITE: return "non-finite covariance";
    case DOA_ETIMEOUT: return "bounded device wait ran out";
    default: return "unknown status";
  }
}

doa_status doa_covariance(const float *X, int M, int N, int ldx, float *R, double *R64, int prec, void *stream) {
  if (!X || M < 2 || M > kMaxM || N < 1 || ldx < N || (!R && !R64) || prec < DOA_FP32 || prec > DOA_FP16X3)
    return DOA_EINVAL;
  if (!aligned(X, 8) || (R && !aligned(R, 8)) || (R64 && !aligned(R64, 16))) return DOA_EINVAL;
  const float2 *X2 = reinterpret_cast<const float2 *>(X);
  if (prec == DOA_FP32)
    return cuda_status(launch_covariance_single(X2, M, N, ldx, reinterpret_cast<float2 *>(R),
                                                reinterpret_cast<double2 *>(R64), as_stream(stream)));
  // tensor-core forms read X with TMA: 16-byte aligned base and row pitch
  if (!aligned(X, 16) || (ldx & 1)) return DOA_EINVAL;
  return cuda_status(launch_covariance_tc_single(X2, M, N, ldx, prec, reinterpret_cast<float2 *>(R),
                                                 reinterpret_cast<double2 *>(R64), as_stream(stream)));
}

doa_status doa_noise_subspace(const double *R64, int M, int d, int alg, double *evals, double *B, int *K_out,
                              int *info, void *stream) {
  return doa_noise_subspace_prec(R64, M, d, alg, DOA_EIG_FP64, evals, B, K_out, info, stream);
}

doa_status doa_noise_subspace_prec(const double *R64, int M, int d, int alg, int eig_prec, double *evals, double *B,
                                   int *K_out, int *info, void *stream) {
  if (!R64 || !B || !info || M < 2 || M > kMaxM || d < 0 || d >= M || alg < DOA_PHD || alg > DOA_MN ||
      (eig_prec != DOA_EIG_DOUBLE_FLOAT && eig_prec != DOA_EIG_FP64))
    return DOA_EINVAL;
  if (!aligned(R64, 16) || !aligned(B, 16) || (evals && !aligned(evals, 8))) return DOA_EINVAL;
  return cuda_status(launch_eig_single(reinterpret_cast<const double2 *>(R64), M, d, alg, eig_prec, evals,
                                       reinterpret_cast<double2 *>(B), K_out, info, as_stream(stream)));
}

doa_status doa_scan(const double *B, int M, int K, doa_grid grid, int prec, float *P, void *stream) {
  if (!B || !P || M < 2 || M > kMaxM || K < 1 || K > M || !grid_ok(grid) || prec < DOA_FP32 || prec > DOA_FP16X3)
    return DOA_EINVAL;
  if (!aligned(B, 16) || !aligned(P, 4)) return DOA_EINVAL;
  cudaStream_t s = as_stream(stream);
  uint32_t *S = reinterpret_cast<uint32_t *>(P);  // phase table first, spectrum over it
  cudaError_t e = launch_grid_table_single(grid.lo_deg, grid.step_deg, 0, grid.L, S, s);
  if (e != cudaSuccess) return DOA_ECUDA;
  const double2 *B2 = reinterpret_cast<const double2 *>(B);
  if (prec == DOA_FP32)
    return cuda_status(launch_scan_single(B2, M, K, grid.L, grid.lo_deg, grid.step_deg, 0, S, P, s));
  return cuda_status(launch_scan_tc_single(B2, M, K, grid.L, grid.lo_deg, grid.step_deg, prec, S, P, s));
}

doa_status doa_scan_slice(const double *B, int M, int K, doa_grid grid, int k0, int n, float *P, void *stream) {
  if (!B || !P || M < 2 || M > kMaxM || K < 1 || K > M || !grid_ok(grid) || k0 < 0 || n < 1 ||
      (int64_t)k0 + n > grid.L)
    return DOA_EINVAL;
  if (!aligned(B, 16) || !aligned(P, 4)) return DOA_EINVAL;
  cudaStream_t s = as_stream(stream);
  uint32_t *S = reinterpret_cast<uint32_t *>(P);
  if (launch_grid_table_single(grid.lo_deg, grid.step_deg, k0, n, S, s) != cudaSuccess) return DOA_ECUDA;
  return cuda_status(launch_scan_single(reinterpret_cast<const double2 *>(B), M, K, n, grid.lo_deg, grid.step_deg,
                                        k0, S, P, s));
}

doa_status doa_slice_peaks(const float *Pbuf, int b0, int k0, int k1, int L, int d, doa_slice_summary *out,
                           void *stream) {
  if (!Pbuf || !out || L < 3 || k0 < 0 || k1 <= k0 || k1 > L || b0 != (k0 > 0 ? k0 - 1 : 0) || d < 0 ||
      d > DOA_SLICE_MAXD)
    return DOA_EINVAL;
  if (!aligned(Pbuf, 4) || !aligned(out, 4)) return DOA_EINVAL;
  return cuda_status(launch_slice_peaks(Pbuf, b0, k0, k1, L, d, out, as_stream(stream)));
}

doa_status doa_merge_slices(const doa_slice_summary *sums, int nslices, int d, int32_t *idx, float *val,
                            int32_t *count) {
  if (!sums || nslices < 1 || d < 0 || d > DOA_SLICE_MAXD || !count || (d > 0 && (!idx || !val))) return DOA_EINVAL;
  struct C {
    float v;
    int32_t i;
  };
  std::vector<C> cands;
  for (int t = 0; t < nslices; ++t) {
    const doa_slice_summary &a = sums[t];
    if (a.count < 0 || a.count > DOA_SLICE_MAXD) return DOA_EINVAL;
    for (int q = 0; q < a.count; ++q) cands.push_back(C{a.val[q], a.idx[q]});
    if (a.open_idx < 0) continue;
    const float v = a.open_val;
    bool peak = false;
    for (int u = t + 1; u < nslices; ++u) {   // the run covers the first point of slice u
      if (!(sums[u].first_val == v)) return DOA_EINVAL;
      if (!sums[u].first_run_to_end) {
        peak = sums[u].first_next_val < v;
        break;
      }
    }
    if (peak) cands.push_back(C{v, a.open_idx});
  }
  std::sort(cands.begin(), cands.end(), [](const C &x, const C &y) { return x.v > y.v || (x.v == y.v && x.i < y.i); });
  const int n = std::min<int>(d, (int)cands.size());
  std::sort(cands.begin(), cands.begin() + n, [](const C &x, const C &y) { return x.i < y.i; });
  for (int q = 0; q < n; ++q) {
    idx[q] = cands[q].i;
    val[q] = cands[q].v;
  }
  *count = n;
  return DOA_OK;
}

doa_status doa_peaks(const float *P, int L, int d, int *idx, float *val, int *count, void *stream) {
  if (!P || !count || L < 3 || d < 0 || d >= kMaxM || (d > 0 && (!idx || !val))) return DOA_EINVAL;
  return cuda_status(launch_peaks_single(P, L, d, idx, val, count, as_stream(stream)));
}

size_t doa_scan_geometry_ws_bytes(int La, int Le) {
  if (La < 1 || Le < 1) return 0;
  return (size_t)geo_table_bytes(La, Le);
}

doa_status doa_scan_geometry(const double *B, int M, int K, doa_grid az, doa_geometry geom, float *P, void *ws,
                             size_t ws_bytes, void *stream) {
  if (!B || !P || !ws || M < 2 || M > kMaxM || K < 1 || K > M || !geometry_ok(az, geom)) return DOA_EINVAL;
  if (!aligned(B, 16) || !aligned(P, 4) || !aligned(ws, 16)) return DOA_EINVAL;
  if (ws_bytes < (size_t)geo_table_bytes(az.L, geom.Le)) return DOA_ENOMEM;
  return cuda_status(launch_scan_geometry_single(reinterpret_cast<const double2 *>(B), M, K, geom.pos, az.lo_deg,
                                                 az.step_deg, az.L, geom.el_lo_deg, geom.el_step_deg, geom.Le, P,
                                                 static_cast<uint8_t *>(ws), as_stream(stream)));
}

doa_status doa_peaks2d(const float *P, int La, int Le, int wrap_az, int d, int *idx, float *val, int *count,
                       void *stream) {
  if (!P || !count || La < 1 || Le < 1 || La > (1 << 24) || Le > (1 << 24) || (int64_t)La * Le > (1 << 30) ||
      (wrap_az != 0 && wrap_az != 1) || d < 0 || d >= kMaxM || (d > 0 && (!idx || !val)))
    return DOA_EINVAL;
  if (!aligned(P, 4)) return DOA_EINVAL;
  return cuda_status(launch_peaks2d_single(P, La, Le, wrap_az, d, idx, val, count, as_stream(stream)));
}

doa_status doa_root_music(const double *B, int M, int K, int d, double *theta, int *info, void *stream) {
  if (!B || !theta || !info || M < 2 || M > kMaxM || K < 1 || K > M || d < 1 || d >= M) return DOA_EINVAL;
  if (!aligned(B, 16) || !aligned(theta, 8) || !aligned(info, 4)) return DOA_EINVAL;
  return cuda_status(launch_roots_single(reinterpret_cast<const double2 *>(B), M, K, d, theta, info,
                                         as_stream(stream)));
}

doa_status doa_model_order(const double *evals, int M, int N, int *mdl, int *aic, void *stream) {
  if (!evals || M < 1 || M > kMaxM || N < 1 || (!mdl && !aic)) return DOA_EINVAL;
  if (!aligned(evals, 8) || (mdl && !aligned(mdl, 4)) || (aic && !aligned(aic, 4))) return DOA_EINVAL;
  return cuda_status(launch_model_order_single(evals, M, N, mdl, aic, as_stream(stream)));
}

doa_status doa_refine_peaks(const double *B, int M, int K, doa_grid grid, const int *idx, const int *count,
                            int cap, double *theta, void *stream) {
  if (!B || !idx || !count || !theta || M < 2 || M > kMaxM || K < 1 || K > M || !grid_ok(grid) || cap < 1)
    return DOA_EINVAL;
  if (!aligned(B, 16) || !aligned(idx, 4) || !aligned(count, 4) || !aligned(theta, 8)) return DOA_EINVAL;
  return cuda_status(launch_refine_single(reinterpret_cast<const double2 *>(B), M, K, grid.lo_deg, grid.step_deg,
                                          nullptr, 0.0, 0.0, grid.L, idx, count, cap, theta, as_stream(stream)));
}

doa_status doa_refine_peaks2d(const double *B, int M, int K, doa_grid az, doa_geometry geom, const int *idx,
                              const int *count, int cap, double *out, void *stream) {
  if (!B || !idx || !count || !out || M < 2 || M > kMaxM || K < 1 || K > M || !geometry_ok(az, geom) || cap < 1)
    return DOA_EINVAL;
  if (!aligned(B, 16) || !aligned(idx, 4) || !aligned(count, 4) || !aligned(out, 8)) return DOA_EINVAL;
  return cuda_status(launch_refine_single(reinterpret_cast<const double2 *>(B), M, K, az.lo_deg, az.step_deg,
                                          geom.pos, geom.el_lo_deg, geom.el_step_deg, az.L, idx, count, cap, out,
                                          as_stream(stream)));
}

size_t doa_batch_plan_bytes(const doa_problem *probs, int nprob) {
  if (!probs || nprob < 1) return 0;
  PlanSizes sz;
  std::vector<doa_grid> grids;
  std::vector<int> grid_of;
  std::vector<GeoGridKey> geo_grids;
  std::vector<SteerKey> steers;
  std::vector<int> steer_of;
  if (!count_plan(probs, nprob, sz, grids, grid_of, geo_grids, steers, steer_of, nullptr)) return 0;
  return (size_t)plan_offsets(sz).total;
}

doa_status doa_batch_plan(const doa_problem *probs, int nprob, const doa_tuning *tuning, void *plan,
                          size_t plan_bytes, size_t *ws_bytes, int *bad_index) {
  if (bad_index) *bad_index = -1;
  if (!probs || nprob < 1 || !ws_bytes) return DOA_EINVAL;
  int pt[kNumBuckets];
  for (int b = 0; b < kNumBuckets; ++b) {
    pt[b] = (tuning && tuning->scan_pt[b] != 0) ? tuning->scan_pt[b] : scan_pt_default(b);
    if (!scan_pt_allowed(b, pt[b])) return DOA_EINVAL;
    if (tuning && tuning->eig_mats[b] != 0 && !eig_mats_allowed(b, tuning->eig_mats[b])) return DOA_EINVAL;
    if (tuning && tuning->scan_group[b] != 0 && !scan_group_allowed(tuning->scan_group[b])) return DOA_EINVAL;
  }
  PlanSizes sz;
  std::vector<doa_grid> grids;
  std::vector<int> grid_of;
  std::vector<GeoGridKey> geo_grids;
  std::vector<SteerKey> steers;
  std::vector<int> steer_of;
  if (!count_plan(probs, nprob, sz, grids, grid_of, geo_grids, steers, steer_of, bad_index)) return DOA_EINVAL;
  const PlanOffsets o = plan_offsets(sz);
  if (!plan || plan_bytes < (size_t)o.total) return DOA_ENOMEM;
  uint8_t *base = static_cast<uint8_t *>(plan);
  std::memset(base, 0, (size_t)o.total);
  PlanHeader &h = *reinterpret_cast<PlanHeader *>(base);
  PlanProblem *pp = reinterpret_cast<PlanProblem *>(base + o.prob);
  PlanJob *jobs = reinterpret_cast<PlanJob *>(base + o.job);
  PlanGrid *pg = reinterpret_cast<PlanGrid *>(base + o.grid);
  PlanCovItem *cov = reinterpret_cast<PlanCovItem *>(base + o.cov);
  int32_t *reduce = reinterpret_cast<int32_t *>(base + o.reduce);
  int32_t *eig[kNumBuckets], *scan[kNumBuckets];
  for (int b = 0; b < kNumBuckets; ++b) {
    eig[b] = reinterpret_cast<int32_t *>(base + o.eig[b]);
    scan[b] = reinterpret_cast<int32_t *>(base + o.scan[b]);
  }
  int32_t *tcl = reinterpret_cast<int32_t *>(base + o.tc);
  h.off_tc = o.tc;
  int32_t *geo[kNumBuckets];
  for (int b = 0; b < kNumBuckets; ++b) {
    geo[b] = reinterpret_cast<int32_t *>(base + o.geo[b]);
    h.off_geo[b] = o.geo[b];
  }
  h.magic = kPlanMagic;
  for (int b = 0; b < kNumBuckets; ++b) h.scan_pt[b] = pt[b];
  h.nprob = sz.nprob;
  h.njobs = sz.njobs;
  h.ngrids = sz.ngrids;
  h.ncov = sz.ncov;
  h.nreduce = sz.nreduce;
  h.off_prob = o.prob;
  h.off_job = o.job;
  h.off_grid = o.grid;
  h.off_cov = o.cov;
  h.off_reduce = o.reduce;
  for (int b = 0; b < kNumBuckets; ++b) {
    h.off_eig[b] = o.eig[b];
    h.off_scan[b] = o.scan[b];
  }
  // workspace: per-solve counters, per-grid 32- and 64-bit phase tables, then per problem R,
  // partials and scan factor
  int64_t ws = kWsCounterBytes;
  for (int g = 0; g < sz.ngrids; ++g) {
    pg[g].lo = grids[g].lo_deg;
    pg[g].step = grids[g].step_deg;
    pg[g].L = grids[g].L;
    pg[g].S_off = ws;
    ws = round_up(ws + (int64_t)grids[g].L * 4, 256);
    pg[g].S64_off = ws;
    ws = round_up(ws + (int64_t)grids[g].L * 8, 256);
    h.grid_points += grids[g].L;
  }
  // workspace: trigonometric tables of the geometry grids (FP64 then FP32 entries)
  PlanGeoGrid *pgg = reinterpret_cast<PlanGeoGrid *>(base + o.geo_grid);
  h.off_geo_grid = o.geo_grid;
  h.ngeo_grids = sz.ngeo_grids;
  for (int g = 0; g < sz.ngeo_grids; ++g) {
    const GeoGridKey &k = geo_grids[g];
    PlanGeoGrid &e = pgg[g];
    e.az_lo = k.az.lo_deg;
    e.az_step = k.az.step_deg;
    e.el_lo = k.el_lo;
    e.el_step = k.el_step;
    e.La = k.az.L;
    e.Le = k.Le;
    e.t64_off = ws;
    ws = round_up(ws + 16 * ((int64_t)e.La + e.Le), 256);
    e.t32_off = ws;
    ws = round_up(ws + 8 * ((int64_t)e.La + e.Le), 256);
    h.geo_grid_points = std::max(h.geo_grid_points, e.La + e.Le);
  }
  // workspace: shared FP32 steering tables (float2[MP][ldt] each)
  PlanGeoSteer *pst = reinterpret_cast<PlanGeoSteer *>(base + o.geo_steer);
  h.off_geo_steer = o.geo_steer;
  h.ngeo_steer = sz.ngeo_steer;
  for (int t = 0; t < sz.ngeo_steer; ++t) {
    const SteerKey &k = steers[t];
    PlanGeoSteer &e = pst[t];
    e.pos = k.pos;
    e.geo_grid = k.geo_grid;
    e.M = k.M;
    e.MP = steer_rows(k.M);
    e.npts = geo_grids[k.geo_grid].az.L * geo_grids[k.geo_grid].Le;
    e.ldt = (int32_t)steer_ldt(geo_grids[k.geo_grid]);
    e.tab_off = ws;
    ws = round_up(ws + 8 * (int64_t)e.MP * e.ldt, 256);
    h.steer_max_ldt = std::max(h.steer_max_ldt, e.ldt);
  }
  // tensor-core covariance lists and their per-problem marks in the workspace
  int32_t *covtc[2];
  int icovtc[2] = {0, 0};
  for (int c = 0; c < 2; ++c) {
    covtc[c] = reinterpret_cast<int32_t *>(base + o.covtc[c]);
    h.off_covtc[c] = o.covtc[c];
    h.ncovtc[c] = sz.covtc[c];
  }
  h.covtc_flag_off = ws;
  ws = round_up(ws + 4 * (int64_t)(sz.covtc[0] + sz.covtc[1]), 256);
  int icov[kCovClasses], ired = 0, ijob = 0;
  h.cov_first[0] = 0;
  for (int c = 0; c < kCovClasses; ++c) {
    h.cov_first[c + 1] = h.cov_first[c] + sz.cov_class[c];
    icov[c] = h.cov_first[c];
  }
  int ie[kNumBuckets] = {0, 0, 0, 0}, is[kNumBuckets] = {0, 0, 0, 0};
  int64_t tiles[kNumBuckets] = {0, 0, 0, 0};
  // grid-shared scan: FP32 ULA problems of a bucket whose grid at least one other such problem
  // shares go to groups of sg_size[b]; sharers[g * kNumBuckets + b] lists them in problem order
  int sgsize[kNumBuckets];
  for (int b = 0; b < kNumBuckets; ++b) {
    sgsize[b] = (tuning && tuning->scan_group[b] != 0) ? tuning->scan_group[b] : kScanGroupDefault;
    h.sg_size[b] = sgsize[b];
  }
  auto ula_fp32 = [](const doa_problem &p) { return !p.geom.pos && p.prec == DOA_FP32; };
  std::vector<std::vector<int32_t>> sharers((size_t)sz.ngrids * kNumBuckets);
  for (int i = 0; i < nprob; ++i)
    if (ula_fp32(probs[i])) sharers[(size_t)grid_of[i] * kNumBuckets + m_bucket(probs[i].M)].push_back(i);
  auto grouped = [&](int i) {
    const int b = m_bucket(probs[i].M);
    return ula_fp32(probs[i]) && sgsize[b] > 1 && sharers[(size_t)grid_of[i] * kNumBuckets + b].size() >= 2;
  };
  // grid-shared tensor-core scan: split-precision ULA problems sharing (grid, M bucket, precision)
  auto ula_tc = [](const doa_problem &p) { return !p.geom.pos && p.prec != DOA_FP32; };
  auto tc_key = [&](int i) { return ((size_t)grid_of[i] * kNumBuckets + m_bucket(probs[i].M)) * 4 + probs[i].prec; };
  std::vector<std::vector<int32_t>> tc_sharers((size_t)sz.ngrids * kNumBuckets * 4);
  for (int i = 0; i < nprob; ++i)
    if (ula_tc(probs[i])) tc_sharers[tc_key(i)].push_back(i);
  auto tc_grouped = [&](int i) {
    return ula_tc(probs[i]) && sgsize[m_bucket(probs[i].M)] > 1 && tc_sharers[tc_key(i)].size() >= 2;
  };
  for (int i = 0; i < nprob; ++i) {
    const doa_problem &p = probs[i];
    PlanProblem &q = pp[i];
    q.p = p;
    const int M = p.M, b = m_bucket(M);
    const int64_t mm = (int64_t)M * M * 16;
    q.r64_off = ws;
    ws = round_up(ws + mm, 256);
    q.npts = (int32_t)spectrum_points(p);
    q.part_off = ws;
    if (cov_tc_ok(p)) {
      q.nchunks = 0;
      covtc[cov_tc_class(M)][icovtc[cov_tc_class(M)]++] = i;
    } else {
      q.nchunks = (p.N + kCovChunk - 1) / kCovChunk;
      if (q.nchunks > 1) {
        ws = round_up(ws + mm * q.nchunks, 256);
        reduce[ired++] = i;
      }
      for (int c = 0; c < q.nchunks; ++c) cov[icov[cov_class(M)]++] = PlanCovItem{i, c};
    }
    eig[b][ie[b]++] = i;
    q.grid_id = p.geom.pos ? -1 : grid_of[i];
    q.geo_grid = p.geom.pos ? grid_of[i] : -1;
    q.geo_steer = p.geom.pos ? steer_of[i] : -1;
    q.first_job = ijob;
    int slot = 0;
    for (int a = 0; a < 4; ++a) {
      q.slot[a] = -1;
      if (!((p.alg_mask >> a) & 1u)) continue;
      PlanJob &j = jobs[ijob++];
      j.prob = i;
      j.alg = a;
      j.slot = q.slot[a] = slot++;
    }
    q.njobs = slot;
    factor_layout(p, q);
    if (p.flags & DOA_FLAG_POLISH_PEAKS) ++h.npolish;
    if (p.peak_angle) ++h.nrefine;
    if (p.root_angle) ++h.nroots;
    q.fac_off = ws;
    ws = round_up(ws + factor_bytes(M), 256);
    if (p.geom.pos) {
      const int tp = kScanThreads * pt[b];
      q.tile_start = h.geo_tiles[b];
      h.geo_tiles[b] += (q.npts + tp - 1) / tp;
      geo[b][h.geo_jobs[b]++] = i;
    } else if (grouped(i) || tc_grouped(i)) {
      q.tile_start = 0;   // scanned by its group (grid-shared scan)
    } else if (p.prec == DOA_FP32) {
      const int tp = kScanThreads * pt[b];
      q.tile_start = tiles[b];
      tiles[b] += (p.grid.L + tp - 1) / tp;
      scan[b][is[b]++] = i;
    } else {
      q.tile_start = h.tc_tiles;
      h.tc_tiles += (p.grid.L + 127) / 128;
      tcl[h.tc_jobs++] = i;
      h.tc_cols = std::max(h.tc_cols, tc_batch_cols(q.Kf));
    }
  }
  // longest problems first, so the static round-robin over SMs ends evenly (stable: equal N keep order)
  for (int c = 0; c < 2; ++c)
    std::stable_sort(covtc[c], covtc[c] + sz.covtc[c], [&](int32_t a, int32_t b) { return probs[a].N > probs[b].N; });
  for (int b = 0; b < kNumBuckets; ++b) {
    h.eig_mats[b] = (tuning && tuning->eig_mats[b] != 0) ? tuning->eig_mats[b] : eig_mats_default(b, sz.eig[b]);
    h.eig_count[b] = sz.eig[b];
    h.scan_jobs[b] = is[b];
    h.scan_tiles[b] = tiles[b];
  }
  // the groups, grid by grid, sg_size problems each (the last one of a grid may be smaller)
  for (int b = 0; b < kNumBuckets; ++b) {
    PlanScanGroup *grp = reinterpret_cast<PlanScanGroup *>(base + o.sg[b]);
    int32_t *sgl = reinterpret_cast<int32_t *>(base + o.sgl[b]);
    h.off_sg[b] = o.sg[b];
    h.off_sgl[b] = o.sgl[b];
    const int tp = kScanThreads * pt[b];
    for (int g = 0; g < sz.ngrids; ++g) {
      const std::vector<int32_t> &v = sharers[(size_t)g * kNumBuckets + b];
      if (sgsize[b] <= 1 || v.size() < 2) continue;
      for (size_t f = 0; f < v.size(); f += (size_t)sgsize[b]) {
        PlanScanGroup &e = grp[h.sg_groups[b]++];
        e.grid_id = g;
        e.first = h.sg_probs[b];
        e.count = (int32_t)std::min<size_t>((size_t)sgsize[b], v.size() - f);
        e.tiles = (grids[g].L + tp - 1) / tp;
        e.unit_start = h.sg_units[b];
        h.sg_units[b] += e.tiles;
        for (int q = 0; q < e.count; ++q) sgl[h.sg_probs[b]++] = v[f + q];
      }
    }
  }
  // tensor-core groups: each key's problems in order, packed while their columns (2 Kf rounded
  // up to 16) fit kTcgMaxCols and their count the bucket's group size; runs of up to kTcgChunk
  // groups of one key form the chunks; one record per group in the workspace
  {
    PlanTcGroup *tg = reinterpret_cast<PlanTcGroup *>(base + o.tcg);
    PlanTcChunk *tcc = reinterpret_cast<PlanTcChunk *>(base + o.tcc);
    int32_t *tgl = reinterpret_cast<int32_t *>(base + o.tcgl);
    h.off_tcg = o.tcg;
    h.off_tcc = o.tcc;
    h.off_tcgl = o.tcgl;
    for (size_t key = 0; key < tc_sharers.size(); ++key) {
      const std::vector<int32_t> &v = tc_sharers[key];
      if (v.size() < 2) continue;
      const int b = (int)((key / 4) % kNumBuckets), g = (int)(key / 4 / kNumBuckets);
      if (sgsize[b] <= 1) continue;
      const int maxp = std::min(kTcgMaxProbs, sgsize[b]);
      int chunk = -1;
      size_t f = 0;
      while (f < v.size()) {
        PlanTcGroup &e = tg[h.tcg_groups];
        e.first = h.tcg_probs;
        e.count = 0;
        e.prec = probs[v[f]].prec;
        int cols = 0, Mmax = 0;
        while (f < v.size() && e.count < maxp) {
          const int c = (2 * pp[v[f]].Kf + 15) / 16 * 16;
          if (cols + c > kTcgMaxCols) break;
          cols += c;
          Mmax = std::max(Mmax, probs[v[f]].M);
          tgl[h.tcg_probs++] = v[f++];
          ++e.count;
        }
        e.NG = std::max(16, (cols + 15) / 16 * 16);
        ws = round_up(ws, 1024);
        e.rec_off = ws;
        ws = round_up(ws + kTcgRecBytes, 1024);
        if (chunk < 0 || tcc[chunk].ngroups == kTcgChunk) {
          chunk = h.tcg_chunks++;
          PlanTcChunk &c = tcc[chunk];
          c.grid_id = g;
          c.first_group = h.tcg_groups;
          c.ngroups = 0;
          c.Mg = 8;
          c.tiles = (grids[g].L + kTcgTile - 1) / kTcgTile;
          c.unit_start = h.tcg_units;
          h.tcg_units += c.tiles;
        }
        tcc[chunk].ngroups += 1;
        tcc[chunk].Mg = std::max(tcc[chunk].Mg, (Mmax + 7) / 8 * 8);
        ++h.tcg_groups;
      }
    }
  }
  h.next_val_off = -1;
  if (h.npolish > 0) {   // the polish reads, per job, the best peak value below the selection
    h.next_val_off = ws;
    ws = round_up(ws + 4 * (int64_t)sz.njobs, 256);
  }
  h.ws_bytes = ws;
  *ws_bytes = (size_t)ws;
  return DOA_OK;
}

doa_status doa_solve_batch(const void *plan_host, const void *plan_dev, void *ws, size_t ws_bytes, int *status,
                           void *const *stage_events, void *stream) {
  if (!plan_host || !plan_dev || !ws || !status) return DOA_EINVAL;
  const PlanHeader &h = *static_cast<const PlanHeader *>(plan_host);
  if (h.magic != kPlanMagic || h.nprob < 1) return DOA_EINVAL;
  if (!aligned(plan_dev, 16) || !aligned(ws, 256) || !aligned(status, 4)) return DOA_EINVAL;
  if (ws_bytes < (size_t)h.ws_bytes) return DOA_ENOMEM;
  cudaStream_t s = as_stream(stream);
  const uint8_t *pd = static_cast<const uint8_t *>(plan_dev);
  uint8_t *w = static_cast<uint8_t *>(ws);
  auto mark = [&](int i) -> bool {
    return !stage_events || cudaEventRecord(static_cast<cudaEvent_t>(stage_events[i]), s) == cudaSuccess;
  };
  // the per-solve counters at the start of the workspace (the persistent scans' next unit / run)
  if (!mark(0) || cudaMemsetAsync(w, 0, (size_t)kWsCounterBytes, s) != cudaSuccess ||
      launch_grid_tables(pd, h, w, s) != cudaSuccess || launch_geo_tables(pd, h, w, s) != cudaSuccess)
    return DOA_ECUDA;
  if (!mark(1) || launch_covariance_batch(pd, h, w, s) != cudaSuccess) return DOA_ECUDA;
  if (!mark(2) || launch_eig_batch(pd, h, w, status, s) != cudaSuccess) return DOA_ECUDA;
  if (!mark(3) || launch_scan_batch(pd, h, w, s) != cudaSuccess) return DOA_ECUDA;
  if (h.tc_jobs > 0 && launch_scan_tc_batch(pd, h, w, status, s) != cudaSuccess) return DOA_ECUDA;
  if (h.tcg_groups > 0 && launch_scan_tc_shared(pd, h, w, status, s) != cudaSuccess) return DOA_ECUDA;
  if (launch_scan_geometry_batch(pd, h, w, s) != cudaSuccess) return DOA_ECUDA;
  if (!mark(4) || launch_peaks_batch(pd, h, w, true, true, s) != cudaSuccess) return DOA_ECUDA;
  // peak polish applies to ULA problems only (geometry problems reject the flag)
  if (h.npolish > 0 &&
      (launch_polish_batch(pd, h, w, s) != cudaSuccess || launch_peaks_batch(pd, h, w, true, false, s) != cudaSuccess))
    return DOA_ECUDA;
  if (launch_refine_batch(pd, h, w, s) != cudaSuccess) return DOA_ECUDA;
  if (launch_roots_batch(pd, h, w, status, s) != cudaSuccess) return DOA_ECUDA;
  if (!mark(5)) return DOA_ECUDA;
  return DOA_OK;
}

}  // extern "C"
