/*
 * align.h — C ABI of the GB300 library for the voxelized-feature mutual-information
 * (MI) scan-alignment cost of Mehta, McBride & Pandey, "Robust and Fast 3D Scan
 * Alignment using Mutual Information" (arXiv 1709.06948).
 *
 * The library evaluates, for large batches of candidate 6-DOF poses of scan B, the
 * MI between the voxel feature maps of scan A and of the transformed scan B over
 * their overlapping bounding region (Sec. III-A, Algorithm 1, Eqs. 1-5), and the
 * pose of maximum MI.  All compute runs in hand-written CUDA kernels on one GPU;
 * there is no CPU fallback: without a usable GPU every call fails with
 * ALIGN_E_CUDA.
 *
 * Conventions (fixed here because the paper leaves them open):
 *  - A pose eta = [tx, ty, tz, thx, thy, thz] (metres, radians) maps B's frame into
 *    A's frame: p_A = R p_B + t with R = Rz(thz) Ry(thy) Rx(thx) (Sec. I, Eq. 1).
 *    R is evaluated in FP64 on the host and rounded once to FP32; the translation is
 *    stored relative to the grid origin: pose12 = [r00 r01 r02 r10 r11 r12 r20 r21
 *    r22 t'x t'y t'z] with t' = fp32(t - origin).
 *  - Voxel of a point (Sec. III-A, Algorithm 1 "extract voxel ids"), in FP32:
 *      u_i = fma(r_i0, x, fma(r_i1, y, r_i2 * z));  g_i = u_i + t'_i;
 *      k_i = floor(g_i * fp32(1/res));  inside iff 0 <= k_i < dims_i;
 *      key = (k_z * Y + k_y) * X + k_x.
 *    Points outside the grid are dropped.
 *  - z-height in whole millimetres: zq = round-half-even(g_z * 1000),
 *    dz = zq - k_z * res_mm.  Per voxel the exact integer sums n, S1 = sum dz and
 *    S2 = sum dz^2 are kept.
 *  - Features (Sec. III-A: "number of points in voxel", "variance of z-height";
 *    unoccupied voxels keep the no-feature value phi = symbol 0):
 *      count level    = #{ j : n >= count_thresh[j] }            (0 .. L_c-1)
 *      variance level = #{ j : n*S2 - S1^2 >= var_thresh[j] * n^2 } (0 .. L_v-1)
 *      symbol = 0 if n == 0, else
 *        ALIGN_FEAT_COUNT:      1 + count level              (K = 1 + L_c)
 *        ALIGN_FEAT_ZVAR:       1 + variance level           (K = 1 + L_v)
 *        ALIGN_FEAT_COUNT_ZVAR: 1 + count level * L_v + variance level (K = 1 + L_c*L_v)
 *    Defaults: count_thresh[j] = 2^(j+1); var_thresh[j] = floor(res_mm^2 / 2^(2 + L_v-1-j)).
 *  - Overlap region (Algorithm 1): the inclusive voxel-index bounding boxes of the
 *    occupied voxels of A and of transformed B, intersected (max of minima, min of
 *    maxima).  Every voxel of the region counts, phi voxels included (Sec. III-A).
 *    An empty region gives MI = 0.
 *  - MI = H(X) + H(Y) - H(X,Y) (Eqs. 2-5) with p = count / N_o over the region's
 *    N_o voxels, natural log, 0 log 0 = 0; evaluated in FP32 on the GPU.
 *  - argmax (Eq. 1): the largest MI; ties go to the lowest pose index.
 *
 * Limits: dims_i in [1, 2^20], X*Y*Z < 2^31, res in whole millimetres in [1, 8000]
 * mm, L_c, L_v >= 1 with K <= 64, point counts < 2^31, poses per call < 2^31.
 *
 * Threading: a grid and everything enqueued on it belong to one host thread at a
 * time.  Errors are return codes; align_last_error() describes the last failure of
 * the calling thread.  No function aborts or throws.
 */
#ifndef ALIGN_H
#define ALIGN_H
#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* 2: align_batch_stats fills 9 counters (poses per CTA added), align_eval_stats 6 (sweep
   kind added); align_batch_set_poses_per_cta, align_eval_redo_poses, align_set_sweep,
   align_set_spill and align_microbench added. */
#define ALIGN_API_VERSION 2

typedef enum {
  ALIGN_OK = 0,
  ALIGN_NOT_READY = 1,     /* align_poll: request still running */
  ALIGN_E_INVALID = -1,    /* bad argument (message in align_last_error) */
  ALIGN_E_OOM = -2,        /* device or pinned host allocation failed */
  ALIGN_E_CUDA = -3,       /* CUDA runtime error, or no usable GPU */
  ALIGN_E_BUSY = -4,       /* server admission refused (queue full / over budget) */
  ALIGN_E_TIMEOUT = -5,    /* a bounded wait gave up (align_wait) */
  ALIGN_E_NOREF = -6,      /* align_set_reference has not been called on this grid */
  ALIGN_E_INTERNAL = -7    /* a kernel reported a violated internal bound */
} align_status;

typedef enum { ALIGN_FEAT_COUNT = 0, ALIGN_FEAT_ZVAR = 1, ALIGN_FEAT_COUNT_ZVAR = 2 } align_feature;

/* Where the buffers of a call live (bit flags).  Without ALIGN_XYZ_DEVICE the points
   are host memory and are copied before the call returns.  With ALIGN_OUT_DEVICE the
   outputs are device pointers and the call returns without waiting for the GPU: the
   results are ready when the grid's stream reaches that point. */
enum {
  ALIGN_XYZ_DEVICE = 1,
  ALIGN_POSES_DEVICE = 2,
  ALIGN_OUT_DEVICE = 4
};

typedef struct {
  float origin[3];               /* grid corner (min x, y, z) in A's frame, metres */
  float res_m;                   /* voxel edge R_v, metres, whole millimetres */
  int32_t dims[3];               /* X, Y, Z */
  int32_t feature;               /* align_feature */
  int32_t count_levels;          /* L_c (count levels of an occupied voxel) */
  int32_t var_levels;            /* L_v (z-variance levels of an occupied voxel) */
  const uint32_t* count_thresh;  /* L_c-1 ascending thresholds on n, or NULL */
  const int64_t* var_thresh;     /* L_v-1 ascending thresholds in mm^2, or NULL */
} align_grid_desc;

typedef struct align_grid align_grid;     /* opaque; owns its device state */

/* Create a grid (Sec. III-A: one grid of resolution R_v covering both scans).
   cuda_stream: a cudaStream_t to enqueue all of this grid's work on (NULL = legacy
   default stream).  The desc and its threshold arrays are copied. */
align_status align_create_grid(const align_grid_desc* desc, void* cuda_stream, align_grid** out);
align_status align_destroy_grid(align_grid* grid);

/* K (symbols, empty included) and V (voxels) of a grid. */
align_status align_grid_info(const align_grid* grid, int32_t* n_symbols, int64_t* n_voxels);

/* Algorithm 1 initialisation: voxelize scan A (never moved), build A's feature map,
   A's bounding box and per-symbol 3-D prefix counts.  xyzA: nA x 3 fp32 (host, or
   device with ALIGN_XYZ_DEVICE).  The state stays resident until the next call or
   align_destroy_grid.  nA may be 0 (every overlap is then empty and MI = 0). */
align_status align_set_reference(align_grid* grid, const float* xyzA, int64_t nA, int flags);

/* Copy A's feature map (V bytes, host) and bbox [xmin,ymin,zmin,xmax,ymax,zmax]
   (xmin > xmax when A has no point in the grid) to the caller.  Either may be NULL. */
align_status align_get_reference(align_grid* grid, uint8_t* symA, int32_t boxA[6]);

/* Host-side pose rounding (the convention above) for a grid whose corner is `origin`:
   eta6 P x 6 FP64 -> poses12 P x 12 FP32.  Pure host code; needs no GPU. */
align_status align_round_poses(const float origin[3], const double* eta6, int64_t P, float* poses12);

/* MI for a batch of P poses of scan B (Algorithm 1 loop body for every pose; Eqs. 1-5).
   xyzB: nB x 3 fp32.  Poses: either poses12 (P x 12 FP32, host or device with
   ALIGN_POSES_DEVICE) or eta6 (P x 6 FP64, host); exactly one non-NULL.
   mi_out: P floats.  argmax_out: one int64 (may be NULL).  hist_out (may be NULL):
   P x K x K uint32 joint histograms, row = A symbol, column = B symbol.
   P may be 0 (nothing is written; *argmax_out = -1).  Host poses must be finite
   (ALIGN_E_INVALID otherwise); points may hold NaN or infinities, which fall outside
   the grid under every pose. */
align_status align_eval_mi(align_grid* grid, const float* xyzB, int64_t nB, int flags,
                           const float* poses12, const double* eta6, int64_t P,
                           float* mi_out, int64_t* argmax_out, uint32_t* hist_out);

/* Per-voxel integer sums of B under one pose, from the same kernel that serves
   align_eval_mi: acc_out (host) V x 3 int64 rows (n, S1, S2), zero for empty voxels
   (S1, S2 are produced for every feature here); box_out: B's occupied bbox as above.
   For parity checks of the voxel map. */
align_status align_accumulate(align_grid* grid, const float* xyzB, int64_t nB, int flags,
                              const float pose12[12], int64_t* acc_out, int32_t box_out[6]);

/* Coarse-to-fine lattice search standing in for Algorithm 1's Nelder-Mead loop:
   per level, counts[a] evenly spaced samples of each axis over centre +- range
   (a single sample sits at the centre), poses ordered rotation axes outermost
   (rx, ry, rz, tx, ty, tz; the last fastest); the best pose becomes the next
   centre and every range halves.  T_out: final centre (eta); mi_out: its MI.
   align_search uses counts = {8, 8, 2, 2, 2, 8} (4,096 poses per level).
   level_best (may be NULL): each level's argmax index. */
align_status align_search(align_grid* grid, const float* xyzB, int64_t nB, int flags,
                          const double init[6], const double range[6], int32_t levels,
                          double T_out[6], float* mi_out);
align_status align_search_ex(align_grid* grid, const float* xyzB, int64_t nB, int flags,
                             const double init[6], const double range[6], const int32_t counts[6],
                             int32_t levels, double T_out[6], float* mi_out, int64_t* level_best);

/* Nelder-Mead refinement, the optimiser of Algorithm 1 ("Update T_c using Nelder-Mead
   optimization"; Nelder and Mead 1965, cited in Sec. III-C), maximising MI over eta.
   S simplices run in lockstep, each from its start (starts: S x 6 FP64, host): initial
   vertices x0 and x0 + step[i] e_i (Sec. IV uses step = {8, 8, 1, 0.1, 0.1, 0.8});
   coefficients reflection 1, expansion 2, contraction 1/2, shrink 1/2; vertices ordered by
   -MI with equal values keeping their order.  Every phase of an iteration evaluates the
   points of all simplices that need one in one batched evaluation (align_eval_mi's path).
   A simplex stops after max_iter iterations, or earlier when ftol > 0 and all its vertices'
   MI lie within ftol of its best.  T_out: S x 6 best vertices; mi_out (may be NULL): their
   MI; iters_out (may be NULL): iterations run.  xyzB as for align_eval_mi. */
align_status align_refine_nm(align_grid* grid, const float* xyzB, int64_t nB, int flags, const double* starts,
                             int32_t S, const double step[6], int32_t max_iter, double ftol, double* T_out,
                             float* mi_out, int32_t* iters_out);

/* Counters of the last synchronising evaluation on this grid (host ints):
   [0] key-partition passes of the hardest pose so far, [1] voxels that needed the
   wide (64-bit) side sums, [2] hash-table slots per CTA, [3] CTAs of the last eval
   launch, [4] kernels launched by this grid since creation, [5] how the last eval launch
   swept its poses: 0 one pose per CTA, 1 pose pairs (two poses per CTA that share their
   rotation, t_y and t_z), 2 one pose per 2-CTA cluster sharing a table split between the
   two CTAs' shared memories (grids whose single poses need 8 or more key partitions).
   Each way learns its own key-partition count; results are the same whichever runs. */
align_status align_eval_stats(align_grid* grid, int64_t out[6]);

/* How this grid's launches sweep their poses (the kinds of align_eval_stats [5]): -1
   automatic (the default: pairs while their tables need no more key partitions than
   single poses', or, with spill queues and both partitioned, no more than twice as many up
   to 8; the cluster while single poses need 8 or more key partitions), 0 one pose per CTA, 1 pose
   pairs wherever the poses form pairs (single poses elsewhere), 2 one pose per 2-CTA
   cluster for single-pose launches (never for align_accumulate's dumps nor inside a batch,
   which sweeps pairs or single poses).  Results are the same for every kind; the choice
   serves measurement and tests.  Errors: ALIGN_E_INVALID for another value. */
align_status align_set_sweep(align_grid* grid, int32_t kind);

/* Whether poses (or pose pairs) that need key partitions sweep B once (on = 1, the default)
   or once per partition (0).  Swept once, the sweep appends every run of B's points to a
   per-CTA queue of its key partition in device memory, and each pass inserts one queue into
   the shared-memory table.  queue_runs: runs each queue holds (16 bytes each, rounded up to
   a multiple of 32); 0 (the default) sizes them for half the points of B (all of them for
   pose pairs), so that the grid holds about CTAs x 8 x n_B / 2 x 16 bytes at 8 partitions
   of single poses.  A pose
   whose runs overflow a queue is finished by the exact path.  Results are the same either
   way.  Errors: ALIGN_E_INVALID for another on, or queue_runs outside 0 .. 2^31. */
align_status align_set_spill(align_grid* grid, int32_t on, int64_t queue_runs);

/* Poses of the last evaluation on this grid (align_eval_mi, align_accumulate or the last
   level of a search) that the exact path finished: poses whose voxels did not fit the
   shared-memory table at the partition count in use, or whose per-voxel sums could exceed
   the table's 32-bit words.  Their results are the same as every other pose's; this
   listing serves parity checks.  Waits for the grid's stream.  *n_out: how many there were;
   out (host, may be NULL when cap is 0): the first min(cap, *n_out) pose indices, ascending. */
align_status align_eval_redo_poses(align_grid* grid, int64_t* out, int64_t cap, int64_t* n_out);

/* Kernel timing with CUDA events recorded on the grid's stream around every eval
   kernel and every compose+argmax pair.  mode 1: enable and reset the totals;
   mode 0: disable; mode 2: only read.  out (may be NULL): [0] total eval-kernel ms,
   [1] total compose+argmax ms, [2] eval launches timed.  Every call of this function
   first waits for the launches recorded so far and adds them to the totals. */
align_status align_profile(align_grid* grid, int32_t mode, double out[3]);

/* Micro-benchmarks of this GPU's throughputs that bound the MI evaluation (the measured
   denominators of its roofline; not part of the method).  kind:
     0  FP32 FFMA lane operations          1  INT32 add/xor lane operations
     2  the voxel map's own per-point mix (FADD, FMUL, float-to-int floor, compares, IMAD)
     3  shared 32-bit red.add, one bank per lane      4  the same with atom.add (returns)
     5  shared 32-bit red.add, random words of 32 KiB 6  the same with atom.add
     7  L2 32-bit atomic adds on random words of an L2-resident region (up to 16 MiB)
   dev_buf: a device buffer of buf_bytes >= 1 MiB the kernels may overwrite (caller-owned).
   The work runs on cuda_stream (NULL = legacy default stream) `reps` times after one
   warm-up; out[0] = operations per second of the fastest run, out[1] = its milliseconds,
   out[2] = operations per run.  Synchronises the stream. */
align_status align_microbench(int32_t kind, void* dev_buf, int64_t buf_bytes, int32_t reps, void* cuda_stream,
                              double out[3]);

/* align_reference_noalloc — A's feature map and bbox without allocating anything.
   The paper has no counterpart; this is a library convenience.  align_set_reference
   allocates working arrays (kept by the grid between calls), which some callers cannot
   do at all: processes whose
   device memory belongs to another allocator under a fixed budget, and latency-bound
   loops in which a device allocation (it may synchronise the device) is not allowed.
   This entry point computes the same symbols and bbox as align_set_reference followed
   by align_get_reference, using a fixed working area that is a static array in the
   library's device memory (10 MiB, held by every GPU that loads the library until the
   process exits).  It calls no cudaMalloc, cudaFree or other allocating routine.
     desc:   as for align_create_grid; X*Y*Z must be at most 2^19 (524,288) voxels,
             larger grids are refused with ALIGN_E_INVALID.
     xyzA:   nA x 3 fp32, device memory.
     symA:   V bytes, device memory (written).   boxA: 6 int32, device memory (written).
     cuda_stream: stream to enqueue on (NULL = legacy default stream).
   The call is asynchronous: outputs are ready when the stream reaches this point.  The
   first call on a device looks up the working area's device address (once per device,
   with that device current); make that first call before any stream capture.  The address
   belongs to the device's CUDA context: after a cudaDeviceReset the next call looks it up
   again (so that call, too, should come before any stream capture).  All calls
   on a device share the working area (each clears what it uses first), so calls whose
   work overlaps on the GPU race; issue them one after another. */
align_status align_reference_noalloc(const align_grid_desc* desc, const float* xyzA, int64_t nA,
                                     uint8_t* symA, int32_t* boxA, void* cuda_stream);

/* ---------------------------------------------------------------------------------
   Batching: many scan pairs, each with its own grid (reference scan A resident) and its
   own pose batch, evaluated in one launch sequence on the batch's stream, capturable as
   one CUDA graph (Algorithm 1's MI evaluation for every pair and pose; Eqs. 1-5).  Results
   are identical to align_eval_mi on each pair.
   --------------------------------------------------------------------------------- */
typedef struct align_pair {
  align_grid* grid;        /* reference set; every grid of a batch on the batch's device */
  const float* xyzB;       /* nB x 3 fp32 (device with ALIGN_XYZ_DEVICE) */
  int64_t nB;
  const float* poses12;    /* P x 12 fp32 (device with ALIGN_POSES_DEVICE), or NULL */
  const double* eta6;      /* P x 6 FP64 host, or NULL; exactly one of the two when P > 0 */
  int64_t P;
  float* mi_out;           /* P (device with ALIGN_OUT_DEVICE) */
  int64_t* argmax_out;     /* 1 or NULL: index of the largest MI, lowest on ties, -1 if P == 0 */
} align_pair;

typedef struct align_batch align_batch;

/* Extra flags of align_eval_batch. */
enum {
  ALIGN_BATCH_GRAPH = 8,   /* capture the launch sequence as a CUDA graph; replay it while
                              the batch keeps its shape (pairs, sizes, grids) */
  ALIGN_BATCH_TUNE = 16    /* pick the kernel shape by timing the candidates on this batch;
                              the choice is cached per batch class (and in the file named by
                              the environment variable ALIGN_TUNE_CACHE, if set) */
};

/* A batch owns its device workspace, a CUDA stream of its own (graphs cannot be captured
   on the legacy default stream) and its graph.  Work queued on cuda_stream before a call
   (e.g. the producer of device inputs) is ordered before the batch's work. */
align_status align_batch_create(void* cuda_stream, align_batch** out);
align_status align_batch_destroy(align_batch* b);

/* Evaluate every pair's poses in one launch sequence: one packing launch for all pairs,
   then per pair the persistent eval kernel (and its exact-path kernel) with the pair's own
   table layout, then one composition and one argmax launch for all pairs.  Inputs are
   copied into the batch's workspace first, so the caller's
   buffers may be reused when the call returns; the call waits for the results.  Pairs
   with P == 0 get argmax -1.  ALIGN_E_INVALID for bad arguments, ALIGN_E_NOREF if a grid
   has no reference, ALIGN_E_OOM / ALIGN_E_CUDA as usual. */
align_status align_eval_batch(align_batch* b, const align_pair* pairs, int32_t n_pairs, int flags);

/* Fix the kernel shape (0..2, see align_batch_stats) or return to the default (-1). */
align_status align_batch_set_shape(align_batch* b, int32_t shape);

/* Fix the poses a CTA sweeps together: 1 (one pose per sweep) or 2 (pose pairs: two poses of
   a pair with the same rotation, t_y and t_z share one pass over the points and one
   shared-memory table), or return to the default (-1: pairs where the poses form them).
   Pairs need pre-rotated tiles (host poses whose rotations repeat); results are the same
   either way. */
align_status align_batch_set_poses_per_cta(align_batch* b, int32_t poses_per_cta);

/* Counters: [0] batch launches, [1] graph captures, [2] graph replays, [3] kernel shape of
   the last launch (0: 1024 threads x 1 point per tile, 1: 1024 x 2, 2: 512 x 1 with two
   CTAs per SM), [4] largest table slots per CTA of the last launch, [5] kernels launched by
   the library, [6] device time of the last launch in microseconds (pack to argmax), [7]
   tuner trials run, [8] poses per CTA of the last launch (2 when any pair used pose pairs).
   The tuner (ALIGN_BATCH_TUNE) times every kernel shape x poses-per-CTA candidate. */
align_status align_batch_stats(const align_batch* b, int64_t out[9]);

/* ---------------------------------------------------------------------------------
   Serving: alignment requests (a lattice search of scan B against a resident reference
   scan A, as align_search_ex) submitted at any time.  The server has max_slots slots, each
   a worker thread with its own CUDA stream and evaluation workspace.  A free slot admits the
   request at the head of the queue (first come, first served) as soon as the device memory
   budget allows and runs its whole search on the slot's stream, every level built on the
   device from the previous level's argmax.  Requests arriving while others run are admitted
   as slots and memory free up, and the launches of all active requests interleave on the
   device.  A request's result is the same as align_search_ex on its grid alone.
   --------------------------------------------------------------------------------- */
typedef struct align_server align_server;

typedef struct align_request {
  int32_t ref_id;          /* from align_server_add_reference */
  const float* xyzB;       /* nB x 3 fp32, host memory, copied by align_submit */
  int64_t nB;
  double init[6];          /* lattice centre of level 0 (eta) */
  double range[6];         /* half-widths of level 0 (they halve every level) */
  int32_t counts[6];       /* samples per axis (tx, ty, tz, rx, ry, rz); {0} = {8,8,2,2,2,8} */
  int32_t levels;
} align_request;

typedef struct align_result {
  double T[6];             /* final centre (eta) */
  float mi;                /* its MI */
  int32_t status;          /* ALIGN_OK or the failure of the step that ran the request */
  double t_submit, t_start, t_done;  /* seconds on the server's monotonic clock */
} align_result;

/* hbm_budget_bytes: device memory the server may hold for the references and the slots'
   workspaces (a workspace keeps the buffers of the largest request it has run; estimated
   per request from its sizes, its grid and the device, including the spill queues of
   align_set_spill when the request's grid has already needed key partitions; a request
   on a grid that has not sweeps B once per partition); max_slots (1..256): most requests
   active at once.  When the request at the head of the queue fits the budget only without
   them and no request runs, idle slots release their workspaces. */
align_status align_server_create(size_t hbm_budget_bytes, int32_t max_slots, align_server** out);
/* Keep scan A (host, nA x 3 fp32) resident as a reference under `desc`; *ref_id names it. */
align_status align_server_add_reference(align_server* s, const align_grid_desc* desc, const float* xyzA,
                                        int64_t nA, int32_t* ref_id);
/* Queue a request; *ticket identifies it.  ALIGN_E_OOM if it could never fit the budget. */
align_status align_submit(align_server* s, const align_request* req, uint64_t* ticket);
/* ALIGN_NOT_READY while the request runs; ALIGN_OK with *out filled (once) when done. */
align_status align_poll(align_server* s, uint64_t ticket, align_result* out);
/* Block until done or timeout_ms elapses (ALIGN_E_TIMEOUT); timeout_ms < 0 waits forever. */
align_status align_wait(align_server* s, uint64_t ticket, int64_t timeout_ms, align_result* out);
/* Seconds on the server's monotonic clock (the clock of align_result's times). */
double align_server_now(const align_server* s);
/* [0] lattice levels evaluated (all slots), [1] requests admitted, [2] requests done, [3] most
   requests active at once, [4] pose evaluations, [5] device bytes held now (estimate: the
   references and the slots' workspaces), [6] peak of [5], [7] requests waiting in the queue. */
align_status align_server_stats(align_server* s, int64_t out[8]);
/* Stops the workers after their current requests; queued requests are dropped.  No call on
   the server (align_wait included) may be in progress or follow. */
align_status align_server_destroy(align_server* s);

/* Message of the calling thread's last failure ("" if none). */
const char* align_last_error(void);

#ifdef __cplusplus
}
#endif
#endif
