/*
 * mi_oracle.h — plain, slow, single-threaded CPU oracle for the voxelized-feature
 * mutual-information (MI) cost of Mehta, McBride & Pandey, "Robust and Fast 3D
 * Scan Alignment using Mutual Information" (arXiv 1709.06948).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg may load this library.  It shares no code,
 * header, table or constant with the CUDA library and never calls it.
 *
 * Every step follows the paper's definitions directly, in the paper's order:
 *   - Sec. III-A: a 3-D grid of resolution R_v covering both scans; a voxel
 *     per point (voxel-point map); per-voxel features "variance of z-height"
 *     and "number of points"; unoccupied voxels keep a no-feature value phi.
 *   - Algorithm 1: voxelize A once; per pose transform B, voxelize, build the
 *     feature map, take the overlapping bounding region (max of mins, min of
 *     maxes), treat the two feature maps over that region as X and Y.
 *   - Eqs. 2-5: MI(X,Y) = H(X) + H(Y) - H(X,Y) with plug-in probabilities.
 *   - Eq. 1: the pose of highest MI.
 * Readings where the paper is silent (Euler order, bin edges, integer z in mm,
 * tie-breaking, the lattice search standing in for Nelder-Mead) are fixed in
 * the repository's design notes and restated beside each function below.
 */
#ifndef MI_ORACLE_H
#define MI_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum { ORC_FEAT_COUNT = 0, ORC_FEAT_ZVAR = 1, ORC_FEAT_COUNT_ZVAR = 2 };
enum { ORC_MAX_SYMBOLS = 64, ORC_MAX_LEVELS = 63 };

typedef struct {
  float origin[3];          /* grid corner in A's frame, metres */
  float res_m;              /* voxel edge R_v, metres (whole millimetres) */
  int32_t dims[3];          /* X, Y, Z voxels */
  int32_t feature;          /* ORC_FEAT_* */
  int32_t count_levels;     /* L_c: occupied count levels */
  int32_t var_levels;       /* L_v: occupied z-variance levels */
  uint32_t count_thresh[ORC_MAX_LEVELS]; /* L_c-1 ascending thresholds on n */
  int64_t var_thresh[ORC_MAX_LEVELS];    /* L_v-1 ascending thresholds, mm^2 */
  /* derived */
  float inv_res;            /* fp32(1/R_v) */
  int32_t res_mm;           /* R_v in whole millimetres */
  int32_t n_symbols;        /* K, including the empty symbol 0 */
} orc_grid;

/* Fill a grid; NULL thresholds take the defaults.  Returns 0, or -1 on bad input. */
int orc_grid_init(orc_grid* g, const float origin[3], float res_m, const int32_t dims[3],
                  int32_t feature, int32_t count_levels, int32_t var_levels,
                  const uint32_t* count_thresh, const int64_t* var_thresh);

/* eta = [tx,ty,tz,thx,thy,thz] (m, rad) -> fp32 [r00..r22, t'x,t'y,t'z], t' = t - origin. */
void orc_round_pose(const orc_grid* g, const double eta[6], float pose12[12]);

/* Map one point; returns the linear voxel key (or -1 when outside the grid) and dz (mm). */
int64_t orc_point_key(const orc_grid* g, const float pose12[12], const float p[3], int32_t* dz);

/* Dense per-voxel accumulation of (n, sum dz, sum dz^2) for all points under one pose.
   cnt/s1/s2 have V entries and are overwritten.  box = inclusive voxel-index bbox of the
   occupied voxels [xmin,ymin,zmin,xmax,ymax,zmax] (xmin > xmax when nothing is in the grid).
   Returns the number of in-grid points. */
int64_t orc_accumulate(const orc_grid* g, const float* xyz, int64_t n, const float pose12[12],
                       int64_t* cnt, int64_t* s1, int64_t* s2, int32_t box[6]);

/* Feature symbol of one voxel from its integer sums (0 = no feature). */
int32_t orc_symbol(const orc_grid* g, int64_t n, int64_t s1, int64_t s2);

/* Algorithm 1 initialisation: A's symbol per voxel (V bytes) and A's bbox. */
void orc_reference(const orc_grid* g, const float* xyzA, int64_t nA, uint8_t* symA, int32_t boxA[6]);

/* Joint histogram h[K][K] (row = A symbol, column = B symbol) over the overlap box for one
   pose.  Returns N_o (voxels in the box, 0 when empty).  box_out may be NULL. */
int64_t orc_joint_hist(const orc_grid* g, const uint8_t* symA, const int32_t boxA[6],
                       const float* xyzB, int64_t nB, const float pose12[12],
                       uint64_t* h, int32_t box_out[6]);

/* Eqs. 2-5 on a K x K count table with total N (FP64, natural log, 0 log 0 = 0). */
double orc_mi_from_hist(const uint64_t* h, int32_t K, int64_t N);
double orc_entropy_rows(const uint64_t* h, int32_t K, int64_t N);   /* H(X) */
double orc_entropy_cols(const uint64_t* h, int32_t K, int64_t N);   /* H(Y) */
double orc_entropy_joint(const uint64_t* h, int32_t K, int64_t N);  /* H(X,Y) */

/* MI for poses [p0, p1) of a pose batch.  mi has P entries (only [p0,p1) written);
   hist (optional, P*K*K uint32) and n_overlap (optional, P) likewise. */
void orc_eval_mi(const orc_grid* g, const uint8_t* symA, const int32_t boxA[6],
                 const float* xyzB, int64_t nB, const float* poses12, int64_t p0, int64_t p1,
                 double* mi, uint32_t* hist, int64_t* n_overlap);

/* The same over all P poses, split into nthreads disjoint pose ranges. */
void orc_eval_mi_threads(const orc_grid* g, const uint8_t* symA, const int32_t boxA[6],
                         const float* xyzB, int64_t nB, const float* poses12, int64_t P,
                         double* mi, uint32_t* hist, int64_t* n_overlap, int32_t nthreads);

/* Eq. 1: index of the largest MI; ties go to the lowest index. */
int64_t orc_argmax(const double* mi, int64_t P);

/* Coarse-to-fine lattice search (stand-in for the Nelder-Mead loop of Algorithm 1):
   per level, counts[a] samples per axis around the centre, best pose becomes the centre,
   ranges halve.  Returns the final centre in T_out and its MI in *mi_out.
   level_best (optional, levels entries) receives each level's argmax index. */
void orc_search(const orc_grid* g, const uint8_t* symA, const int32_t boxA[6],
                const float* xyzB, int64_t nB, const double init[6], const double range[6],
                const int32_t counts[6], int32_t levels, int32_t nthreads,
                double T_out[6], double* mi_out, int64_t* level_best);

/* The lattice of one search level: P = prod(counts) poses (eta, FP64), rotation axes outer. */
void orc_lattice(const double center[6], const double range[6], const int32_t counts[6], double* eta_out);

/* Nelder-Mead minimisation over R^6 (the optimiser of Algorithm 1, "Update T_c using
   Nelder-Mead optimization"; Nelder and Mead 1965, cited in Sec. III-C).  Initial simplex:
   x0 and x0 + step[i] e_i (Sec. IV gives the step sizes).  Coefficients: reflection 1,
   expansion 2, contraction 1/2, shrink 1/2.  Each iteration orders the vertices by f
   (equal values keep their previous order), reflects the worst through the centroid of the
   others, and expands, contracts or shrinks.  Stops after max_iter iterations, or earlier
   when ftol > 0 and every vertex is within ftol of the best.  Returns the iterations run;
   x_out / f_out: the best vertex.  f(x, ctx) is the objective. */
typedef double (*orc_objective)(const double x[6], void* ctx);
int32_t orc_nm(orc_objective f, void* ctx, const double x0[6], const double step[6], int32_t max_iter,
               double ftol, double x_out[6], double* f_out);

/* Nelder-Mead on f(eta) = -MI(round(eta)) with the FP64 MI of orc_eval_mi. */
int32_t orc_nm_mi(const orc_grid* g, const uint8_t* symA, const int32_t boxA[6], const float* xyzB,
                  int64_t nB, const double x0[6], const double step[6], int32_t max_iter, double ftol,
                  double T_out[6], double* mi_out);

/* Nelder-Mead on the quadratic f(x) = sum_i w_i (x_i - c_i)^2 (test objective). */
int32_t orc_nm_quadratic(const double w[6], const double c[6], const double x0[6], const double step[6],
                         int32_t max_iter, double ftol, double x_out[6], double* f_out);

#ifdef __cplusplus
}
#endif
#endif
