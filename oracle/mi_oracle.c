/*
 * mi_oracle.c — plain CPU oracle for the voxelized-feature MI cost (arXiv 1709.06948).
 *
 * TEST INFRASTRUCTURE ONLY: loaded by the test suite, the smoke check and the
 * benchmark's CPU-baseline leg, never by the library it checks.  Built with
 * -O2 -ffp-contract=off so that every floating-point operation is the one written.
 *
 * Nothing here is blocked, fused or reordered: per pose it fills dense per-voxel
 * arrays for B, scans every voxel of the overlap box, and evaluates Eqs. 2-5 in FP64.
 */
#include "mi_oracle.h"

#include <math.h>
#include <pthread.h>
#include <stdlib.h>
#include <string.h>

static int64_t grid_voxels(const orc_grid* g) {
  return (int64_t)g->dims[0] * g->dims[1] * g->dims[2];
}

int orc_grid_init(orc_grid* g, const float origin[3], float res_m, const int32_t dims[3],
                  int32_t feature, int32_t count_levels, int32_t var_levels,
                  const uint32_t* count_thresh, const int64_t* var_thresh) {
  memset(g, 0, sizeof(*g));
  for (int i = 0; i < 3; ++i) {
    g->origin[i] = origin[i];
    g->dims[i] = dims[i];
    if (dims[i] <= 0) return -1;
  }
  if (!(res_m > 0.0f)) return -1;
  g->res_m = res_m;
  g->feature = feature;
  g->count_levels = count_levels;
  g->var_levels = var_levels;
  /* Voxel edge in whole millimetres: z-heights are integers in mm (design reading). */
  double mm = (double)res_m * 1000.0;
  g->res_mm = (int32_t)llround(mm);
  if (g->res_mm < 1 || fabs(mm - (double)g->res_mm) > 1e-3) return -1;
  g->inv_res = (float)(1.0 / (double)res_m);

  int use_count = (feature == ORC_FEAT_COUNT || feature == ORC_FEAT_COUNT_ZVAR);
  int use_var = (feature == ORC_FEAT_ZVAR || feature == ORC_FEAT_COUNT_ZVAR);
  if (!use_count && !use_var) return -1;
  if (use_count) {
    if (count_levels < 1 || count_levels > ORC_MAX_LEVELS) return -1;
    for (int j = 0; j < count_levels - 1; ++j) {
      /* default: level boundaries at n = 2, 4, 8, ... (level = floor(log2 n), capped);
         boundaries past 2^31 saturate at the largest 32-bit count */
      g->count_thresh[j] = count_thresh ? count_thresh[j] : (j + 1 < 32 ? (uint32_t)1u << (j + 1) : UINT32_MAX);
      if (j > 0 && g->count_thresh[j] < g->count_thresh[j - 1]) return -1;
    }
  }
  if (use_var) {
    if (var_levels < 1 || var_levels > ORC_MAX_LEVELS) return -1;
    int64_t r2 = (int64_t)g->res_mm * g->res_mm;
    for (int j = 0; j < var_levels - 1; ++j) {
      /* default: tau_j = floor((res_mm^2 / 4) * 2^-(L_v - 1 - j)), log-spaced below the
         largest variance a voxel can hold (all points on its two z faces: res^2/4). */
      int shift = 2 + (var_levels - 1 - j);
      g->var_thresh[j] = var_thresh ? var_thresh[j] : (shift >= 63 ? 0 : (r2 >> shift));
      if (g->var_thresh[j] < 0) return -1;
      if (j > 0 && g->var_thresh[j] < g->var_thresh[j - 1]) return -1;
    }
  }
  if (feature == ORC_FEAT_COUNT) g->n_symbols = 1 + count_levels;
  else if (feature == ORC_FEAT_ZVAR) g->n_symbols = 1 + var_levels;
  else g->n_symbols = 1 + count_levels * var_levels;
  if (g->n_symbols > ORC_MAX_SYMBOLS) return -1;
  return 0;
}

/* Pose: p_A = R p_B + t with R = Rz(thz) Ry(thy) Rx(thx), evaluated in FP64 and rounded
   once to FP32; the translation is stored relative to the grid origin. */
void orc_round_pose(const orc_grid* g, const double eta[6], float pose12[12]) {
  double cx = cos(eta[3]), sx = sin(eta[3]);
  double cy = cos(eta[4]), sy = sin(eta[4]);
  double cz = cos(eta[5]), sz = sin(eta[5]);
  double R[9];
  R[0] = cz * cy;
  R[1] = cz * sy * sx - sz * cx;
  R[2] = cz * sy * cx + sz * sx;
  R[3] = sz * cy;
  R[4] = sz * sy * sx + cz * cx;
  R[5] = sz * sy * cx - cz * sx;
  R[6] = -sy;
  R[7] = cy * sx;
  R[8] = cy * cx;
  for (int i = 0; i < 9; ++i) pose12[i] = (float)R[i];
  for (int i = 0; i < 3; ++i) pose12[9 + i] = (float)(eta[i] - (double)g->origin[i]);
}

/* Voxel-point map for one point (Algorithm 1, "extract associated voxel ids"):
   u_i = fma(r_i0, x, fma(r_i1, y, r_i2 * z)), g_i = u_i + t'_i  (FP32),
   k_i = floor(g_i * inv_res), inside iff 0 <= k_i < dims_i,
   key = (k_z * Y + k_y) * X + k_x,
   z in mm: zq = round-half-even(g_z * 1000), dz = zq - k_z * res_mm. */
int64_t orc_point_key(const orc_grid* g, const float pose12[12], const float p[3], int32_t* dz) {
  float gx = fmaf(pose12[0], p[0], fmaf(pose12[1], p[1], pose12[2] * p[2])) + pose12[9];
  float gy = fmaf(pose12[3], p[0], fmaf(pose12[4], p[1], pose12[5] * p[2])) + pose12[10];
  float gz = fmaf(pose12[6], p[0], fmaf(pose12[7], p[1], pose12[8] * p[2])) + pose12[11];
  float fx = floorf(gx * g->inv_res);
  float fy = floorf(gy * g->inv_res);
  float fz = floorf(gz * g->inv_res);
  if (!(fx >= 0.0f && fx < (float)g->dims[0])) return -1;
  if (!(fy >= 0.0f && fy < (float)g->dims[1])) return -1;
  if (!(fz >= 0.0f && fz < (float)g->dims[2])) return -1;
  int64_t kx = (int64_t)fx, ky = (int64_t)fy, kz = (int64_t)fz;
  float zmm = gz * 1000.0f;
  int64_t zq = (int64_t)nearbyintf(zmm); /* default rounding mode: to nearest, ties to even */
  if (dz) *dz = (int32_t)(zq - kz * g->res_mm);
  return (kz * g->dims[1] + ky) * g->dims[0] + kx;
}

static void box_empty(int32_t box[6]) {
  box[0] = box[1] = box[2] = INT32_MAX;
  box[3] = box[4] = box[5] = INT32_MIN;
}

int64_t orc_accumulate(const orc_grid* g, const float* xyz, int64_t n, const float pose12[12],
                       int64_t* cnt, int64_t* s1, int64_t* s2, int32_t box[6]) {
  int64_t V = grid_voxels(g);
  memset(cnt, 0, (size_t)V * sizeof(int64_t));
  memset(s1, 0, (size_t)V * sizeof(int64_t));
  memset(s2, 0, (size_t)V * sizeof(int64_t));
  int64_t inside = 0;
  for (int64_t i = 0; i < n; ++i) {
    int32_t dz = 0;
    int64_t key = orc_point_key(g, pose12, xyz + 3 * i, &dz);
    if (key < 0) continue;
    cnt[key] += 1;
    s1[key] += dz;
    s2[key] += (int64_t)dz * dz;
    inside += 1;
  }
  /* bbox of the occupied voxels, found by visiting every voxel */
  box_empty(box);
  int64_t X = g->dims[0], Y = g->dims[1];
  for (int64_t v = 0; v < V; ++v) {
    if (cnt[v] == 0) continue;
    int32_t kx = (int32_t)(v % X), ky = (int32_t)((v / X) % Y), kz = (int32_t)(v / (X * Y));
    if (kx < box[0]) box[0] = kx;
    if (ky < box[1]) box[1] = ky;
    if (kz < box[2]) box[2] = kz;
    if (kx > box[3]) box[3] = kx;
    if (ky > box[4]) box[4] = ky;
    if (kz > box[5]) box[5] = kz;
  }
  return inside;
}

/* Feature levels.  Count: 1 + #{thresholds <= n}.  z-variance: population variance of the
   voxel's dz values, compared without division as n*S2 - S1^2 >= tau * n^2 (exact in
   128-bit integers).  Joint: count level major, variance level minor. */
static int32_t count_level(const orc_grid* g, int64_t n) {
  int32_t lvl = 0;
  for (int j = 0; j < g->count_levels - 1; ++j)
    if (n >= (int64_t)g->count_thresh[j]) lvl += 1;
  return lvl;
}

static int32_t var_level(const orc_grid* g, int64_t n, int64_t s1, int64_t s2) {
  __int128 spread = (__int128)n * s2 - (__int128)s1 * s1; /* = n^2 * variance */
  __int128 n2 = (__int128)n * n;
  int32_t lvl = 0;
  for (int j = 0; j < g->var_levels - 1; ++j)
    if (spread >= (__int128)g->var_thresh[j] * n2) lvl += 1;
  return lvl;
}

int32_t orc_symbol(const orc_grid* g, int64_t n, int64_t s1, int64_t s2) {
  if (n == 0) return 0; /* phi: no feature */
  if (g->feature == ORC_FEAT_COUNT) return 1 + count_level(g, n);
  if (g->feature == ORC_FEAT_ZVAR) return 1 + var_level(g, n, s1, s2);
  return 1 + count_level(g, n) * g->var_levels + var_level(g, n, s1, s2);
}

void orc_reference(const orc_grid* g, const float* xyzA, int64_t nA, uint8_t* symA, int32_t boxA[6]) {
  int64_t V = grid_voxels(g);
  int64_t* cnt = (int64_t*)malloc((size_t)V * sizeof(int64_t));
  int64_t* s1 = (int64_t*)malloc((size_t)V * sizeof(int64_t));
  int64_t* s2 = (int64_t*)malloc((size_t)V * sizeof(int64_t));
  /* A is never moved: identity rotation, translation 0 (so t' = -origin). */
  const double eta0[6] = {0, 0, 0, 0, 0, 0};
  float pose[12];
  orc_round_pose(g, eta0, pose);
  orc_accumulate(g, xyzA, nA, pose, cnt, s1, s2, boxA);
  for (int64_t v = 0; v < V; ++v) symA[v] = (uint8_t)orc_symbol(g, cnt[v], s1[v], s2[v]);
  free(cnt);
  free(s1);
  free(s2);
}

int64_t orc_joint_hist(const orc_grid* g, const uint8_t* symA, const int32_t boxA[6],
                       const float* xyzB, int64_t nB, const float pose12[12],
                       uint64_t* h, int32_t box_out[6]) {
  int64_t V = grid_voxels(g);
  int32_t K = g->n_symbols;
  memset(h, 0, (size_t)K * K * sizeof(uint64_t));
  int64_t* cnt = (int64_t*)malloc((size_t)V * sizeof(int64_t));
  int64_t* s1 = (int64_t*)malloc((size_t)V * sizeof(int64_t));
  int64_t* s2 = (int64_t*)malloc((size_t)V * sizeof(int64_t));
  int32_t boxB[6];
  orc_accumulate(g, xyzB, nB, pose12, cnt, s1, s2, boxB);
  /* Algorithm 1, overlapping bounding region: max of the minima, min of the maxima. */
  int32_t box[6];
  for (int i = 0; i < 3; ++i) {
    box[i] = boxA[i] > boxB[i] ? boxA[i] : boxB[i];
    box[3 + i] = boxA[3 + i] < boxB[3 + i] ? boxA[3 + i] : boxB[3 + i];
  }
  if (box_out) memcpy(box_out, box, sizeof(box));
  int64_t N = 0;
  if (box[0] <= box[3] && box[1] <= box[4] && box[2] <= box[5]) {
    int64_t X = g->dims[0], Y = g->dims[1];
    for (int64_t z = box[2]; z <= box[5]; ++z)
      for (int64_t y = box[1]; y <= box[4]; ++y)
        for (int64_t x = box[0]; x <= box[3]; ++x) {
          int64_t v = (z * Y + y) * X + x;
          int32_t a = symA[v];
          int32_t b = orc_symbol(g, cnt[v], s1[v], s2[v]);
          h[a * K + b] += 1;
          N += 1;
        }
  }
  free(cnt);
  free(s1);
  free(s2);
  return N;
}

static double plogp(uint64_t c, int64_t N) {
  if (c == 0) return 0.0; /* 0 log 0 = 0 */
  double p = (double)c / (double)N;
  return p * log(p);
}

double orc_entropy_rows(const uint64_t* h, int32_t K, int64_t N) {
  if (N <= 0) return 0.0;
  double H = 0.0;
  for (int a = 0; a < K; ++a) {
    uint64_t r = 0;
    for (int b = 0; b < K; ++b) r += h[a * K + b];
    H -= plogp(r, N);
  }
  return H;
}

double orc_entropy_cols(const uint64_t* h, int32_t K, int64_t N) {
  if (N <= 0) return 0.0;
  double H = 0.0;
  for (int b = 0; b < K; ++b) {
    uint64_t c = 0;
    for (int a = 0; a < K; ++a) c += h[a * K + b];
    H -= plogp(c, N);
  }
  return H;
}

double orc_entropy_joint(const uint64_t* h, int32_t K, int64_t N) {
  if (N <= 0) return 0.0;
  double H = 0.0;
  for (int i = 0; i < K * K; ++i) H -= plogp(h[i], N);
  return H;
}

double orc_mi_from_hist(const uint64_t* h, int32_t K, int64_t N) {
  if (N <= 0) return 0.0; /* empty overlap: no information */
  return orc_entropy_rows(h, K, N) + orc_entropy_cols(h, K, N) - orc_entropy_joint(h, K, N);
}

void orc_eval_mi(const orc_grid* g, const uint8_t* symA, const int32_t boxA[6],
                 const float* xyzB, int64_t nB, const float* poses12, int64_t p0, int64_t p1,
                 double* mi, uint32_t* hist, int64_t* n_overlap) {
  int32_t K = g->n_symbols;
  uint64_t* h = (uint64_t*)malloc((size_t)K * K * sizeof(uint64_t));
  for (int64_t p = p0; p < p1; ++p) {
    int64_t N = orc_joint_hist(g, symA, boxA, xyzB, nB, poses12 + 12 * p, h, NULL);
    mi[p] = orc_mi_from_hist(h, K, N);
    if (hist)
      for (int i = 0; i < K * K; ++i) hist[p * K * K + i] = (uint32_t)h[i];
    if (n_overlap) n_overlap[p] = N;
  }
  free(h);
}

typedef struct {
  const orc_grid* g;
  const uint8_t* symA;
  const int32_t* boxA;
  const float* xyzB;
  int64_t nB;
  const float* poses12;
  int64_t p0, p1;
  double* mi;
  uint32_t* hist;
  int64_t* n_overlap;
} orc_job;

static void* orc_job_run(void* arg) {
  orc_job* j = (orc_job*)arg;
  orc_eval_mi(j->g, j->symA, j->boxA, j->xyzB, j->nB, j->poses12, j->p0, j->p1, j->mi, j->hist,
              j->n_overlap);
  return NULL;
}

void orc_eval_mi_threads(const orc_grid* g, const uint8_t* symA, const int32_t boxA[6],
                         const float* xyzB, int64_t nB, const float* poses12, int64_t P,
                         double* mi, uint32_t* hist, int64_t* n_overlap, int32_t nthreads) {
  if (nthreads < 1) nthreads = 1;
  if (nthreads > P) nthreads = (int32_t)(P > 0 ? P : 1);
  pthread_t* th = (pthread_t*)malloc(sizeof(pthread_t) * (size_t)nthreads);
  orc_job* jobs = (orc_job*)malloc(sizeof(orc_job) * (size_t)nthreads);
  for (int t = 0; t < nthreads; ++t) {
    orc_job j = {g, symA, boxA, xyzB, nB, poses12, P * t / nthreads, P * (t + 1) / nthreads,
                 mi, hist, n_overlap};
    jobs[t] = j;
  }
  for (int t = 1; t < nthreads; ++t) pthread_create(&th[t], NULL, orc_job_run, &jobs[t]);
  orc_job_run(&jobs[0]);
  for (int t = 1; t < nthreads; ++t) pthread_join(th[t], NULL);
  free(th);
  free(jobs);
}

int64_t orc_argmax(const double* mi, int64_t P) {
  int64_t best = -1;
  for (int64_t p = 0; p < P; ++p)
    if (best < 0 || mi[p] > mi[best]) best = p; /* strict: ties keep the lower index */
  return best;
}

/* Lattice offsets along one axis: counts samples evenly spread over [-range, +range]
   (a single sample sits at the centre). */
static double lattice_offset(double range, int32_t count, int32_t i) {
  if (count <= 1) return 0.0;
  return (range * (double)(2 * i - (count - 1))) / (double)(count - 1);
}

void orc_lattice(const double center[6], const double range[6], const int32_t counts[6], double* eta_out) {
  /* index = ((((i_rx*m_ry + i_ry)*m_rz + i_rz)*m_tx + i_tx)*m_ty + i_ty)*m_tz + i_tz */
  int64_t idx = 0;
  for (int32_t irx = 0; irx < counts[3]; ++irx)
    for (int32_t iry = 0; iry < counts[4]; ++iry)
      for (int32_t irz = 0; irz < counts[5]; ++irz)
        for (int32_t itx = 0; itx < counts[0]; ++itx)
          for (int32_t ity = 0; ity < counts[1]; ++ity)
            for (int32_t itz = 0; itz < counts[2]; ++itz) {
              double* e = eta_out + 6 * idx;
              e[0] = center[0] + lattice_offset(range[0], counts[0], itx);
              e[1] = center[1] + lattice_offset(range[1], counts[1], ity);
              e[2] = center[2] + lattice_offset(range[2], counts[2], itz);
              e[3] = center[3] + lattice_offset(range[3], counts[3], irx);
              e[4] = center[4] + lattice_offset(range[4], counts[4], iry);
              e[5] = center[5] + lattice_offset(range[5], counts[5], irz);
              idx += 1;
            }
}

void orc_search(const orc_grid* g, const uint8_t* symA, const int32_t boxA[6],
                const float* xyzB, int64_t nB, const double init[6], const double range[6],
                const int32_t counts[6], int32_t levels, int32_t nthreads,
                double T_out[6], double* mi_out, int64_t* level_best) {
  int64_t P = 1;
  for (int a = 0; a < 6; ++a) P *= (counts[a] > 0 ? counts[a] : 1);
  double* eta = (double*)malloc(sizeof(double) * 6 * (size_t)P);
  float* poses = (float*)malloc(sizeof(float) * 12 * (size_t)P);
  double* mi = (double*)malloc(sizeof(double) * (size_t)P);
  double c[6], r[6];
  memcpy(c, init, sizeof(c));
  memcpy(r, range, sizeof(r));
  double best_mi = 0.0;
  for (int32_t l = 0; l < levels; ++l) {
    orc_lattice(c, r, counts, eta);
    for (int64_t p = 0; p < P; ++p) orc_round_pose(g, eta + 6 * p, poses + 12 * p);
    orc_eval_mi_threads(g, symA, boxA, xyzB, nB, poses, P, mi, NULL, NULL, nthreads);
    int64_t b = orc_argmax(mi, P);
    if (level_best) level_best[l] = b;
    memcpy(c, eta + 6 * b, sizeof(c));
    best_mi = mi[b];
    for (int a = 0; a < 6; ++a) r[a] = r[a] * 0.5;
  }
  memcpy(T_out, c, sizeof(c));
  if (mi_out) *mi_out = best_mi;
  free(eta);
  free(poses);
  free(mi);
}


/* ------------------------------------------------------------------------------------
   Nelder-Mead (Nelder and Mead 1965), six parameters, standard coefficients.
   ------------------------------------------------------------------------------------ */
#define NM_N 6

/* Reorder vertices by f, stable (insertion sort keeps equal values in their order). */
static void nm_sort(double sim[NM_N + 1][NM_N], double fsim[NM_N + 1]) {
  for (int i = 1; i <= NM_N; ++i) {
    double fx = fsim[i];
    double x[NM_N];
    memcpy(x, sim[i], sizeof(x));
    int j = i - 1;
    while (j >= 0 && fsim[j] > fx) {
      fsim[j + 1] = fsim[j];
      memcpy(sim[j + 1], sim[j], sizeof(x));
      --j;
    }
    fsim[j + 1] = fx;
    memcpy(sim[j + 1], x, sizeof(x));
  }
}

int32_t orc_nm(orc_objective f, void* ctx, const double x0[6], const double step[6], int32_t max_iter,
               double ftol, double x_out[6], double* f_out) {
  const double rho = 1.0, chi = 2.0, psi = 0.5, sigma = 0.5;
  double sim[NM_N + 1][NM_N], fsim[NM_N + 1];
  for (int i = 0; i <= NM_N; ++i) {
    memcpy(sim[i], x0, sizeof(sim[i]));
    if (i > 0) sim[i][i - 1] = x0[i - 1] + step[i - 1];
    fsim[i] = f(sim[i], ctx);
  }
  nm_sort(sim, fsim);
  int32_t it = 0;
  while (it < max_iter) {
    if (ftol > 0.0) {
      double spread = 0.0;
      for (int i = 1; i <= NM_N; ++i) {
        const double d = fabs(fsim[i] - fsim[0]);
        if (d > spread) spread = d;
      }
      if (spread <= ftol) break;
    }
    double xbar[NM_N];
    for (int j = 0; j < NM_N; ++j) {
      double acc = 0.0;
      for (int i = 0; i < NM_N; ++i) acc += sim[i][j];  /* all vertices but the worst */
      xbar[j] = acc / (double)NM_N;
    }
    double xr[NM_N], xe[NM_N], xc[NM_N];
    for (int j = 0; j < NM_N; ++j) xr[j] = (1.0 + rho) * xbar[j] - rho * sim[NM_N][j];
    const double fr = f(xr, ctx);
    int shrink = 0;
    if (fr < fsim[0]) {
      for (int j = 0; j < NM_N; ++j) xe[j] = (1.0 + rho * chi) * xbar[j] - rho * chi * sim[NM_N][j];
      const double fe = f(xe, ctx);
      if (fe < fr) {
        memcpy(sim[NM_N], xe, sizeof(xe));
        fsim[NM_N] = fe;
      } else {
        memcpy(sim[NM_N], xr, sizeof(xr));
        fsim[NM_N] = fr;
      }
    } else if (fr < fsim[NM_N - 1]) {
      memcpy(sim[NM_N], xr, sizeof(xr));
      fsim[NM_N] = fr;
    } else if (fr < fsim[NM_N]) {  /* outside contraction */
      for (int j = 0; j < NM_N; ++j) xc[j] = (1.0 + psi * rho) * xbar[j] - psi * rho * sim[NM_N][j];
      const double fc = f(xc, ctx);
      if (fc <= fr) {
        memcpy(sim[NM_N], xc, sizeof(xc));
        fsim[NM_N] = fc;
      } else {
        shrink = 1;
      }
    } else {  /* inside contraction */
      for (int j = 0; j < NM_N; ++j) xc[j] = (1.0 - psi) * xbar[j] + psi * sim[NM_N][j];
      const double fc = f(xc, ctx);
      if (fc < fsim[NM_N]) {
        memcpy(sim[NM_N], xc, sizeof(xc));
        fsim[NM_N] = fc;
      } else {
        shrink = 1;
      }
    }
    if (shrink) {
      for (int i = 1; i <= NM_N; ++i) {
        for (int j = 0; j < NM_N; ++j) sim[i][j] = sim[0][j] + sigma * (sim[i][j] - sim[0][j]);
        fsim[i] = f(sim[i], ctx);
      }
    }
    nm_sort(sim, fsim);
    ++it;
  }
  memcpy(x_out, sim[0], sizeof(sim[0]));
  if (f_out) *f_out = fsim[0];
  return it;
}

typedef struct {
  const orc_grid* g;
  const uint8_t* symA;
  const int32_t* boxA;
  const float* xyzB;
  int64_t nB;
} nm_mi_ctx;

static double nm_neg_mi(const double x[6], void* vctx) {
  const nm_mi_ctx* c = (const nm_mi_ctx*)vctx;
  float pose[12];
  double mi = 0.0;
  orc_round_pose(c->g, x, pose);
  orc_eval_mi(c->g, c->symA, c->boxA, c->xyzB, c->nB, pose, 0, 1, &mi, NULL, NULL);
  return -mi;
}

int32_t orc_nm_mi(const orc_grid* g, const uint8_t* symA, const int32_t boxA[6], const float* xyzB,
                  int64_t nB, const double x0[6], const double step[6], int32_t max_iter, double ftol,
                  double T_out[6], double* mi_out) {
  nm_mi_ctx ctx = {g, symA, boxA, xyzB, nB};
  double f = 0.0;
  const int32_t it = orc_nm(nm_neg_mi, &ctx, x0, step, max_iter, ftol, T_out, &f);
  if (mi_out) *mi_out = -f;
  return it;
}

typedef struct {
  const double* w;
  const double* c;
} nm_quad_ctx;

static double nm_quad(const double x[6], void* vctx) {
  const nm_quad_ctx* q = (const nm_quad_ctx*)vctx;
  double s = 0.0;
  for (int i = 0; i < 6; ++i) s += q->w[i] * (x[i] - q->c[i]) * (x[i] - q->c[i]);
  return s;
}

int32_t orc_nm_quadratic(const double w[6], const double c[6], const double x0[6], const double step[6],
                         int32_t max_iter, double ftol, double x_out[6], double* f_out) {
  nm_quad_ctx q = {w, c};
  return orc_nm(nm_quad, &q, x0, step, max_iter, ftol, x_out, f_out);
}
