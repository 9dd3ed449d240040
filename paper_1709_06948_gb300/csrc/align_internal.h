// align_internal.h — device-side conventions and launch interfaces shared by the
// library's translation units (never by the CPU oracle).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "align.h"

namespace mialign {

constexpr int kMaxSymbols = 64;
constexpr int kMaxLevels = 63;
constexpr uint32_t kEmptyKey = 0xFFFFFFFFu;

// Error bits written by kernels into the grid's error word.
enum : uint32_t {
  kErrDzBound = 1u,       // |dz| above the bound the 32-bit sums were sized for
  // 2u: unused (an earlier bounded-wait bit)
  kErrPassLimit = 4u,     // key partitioning could not make the table fit
  kErrLattice = 8u,       // a device-built lattice level found its previous argmax out of range
};

// Grid constants passed by value to every kernel (Sec. III-A grid + feature definition).
struct GridConst {
  float inv_res;          // fp32(1/res)
  int32_t res_mm;         // voxel edge in whole millimetres
  int32_t X, Y, Z;
  int32_t K;              // symbols including phi (0)
  int32_t feature;        // 0 count, 1 z-variance, 2 joint
  int32_t Lc, Lv;         // occupied levels
  int32_t dz_bound;       // |dz| <= dz_bound for every in-grid point
  int32_t dz_shift;       // smallest m with 2^m > 2 * dz_bound (the sweep checks dz + dz_bound < 2^m)
  uint32_t nlim;          // largest n whose S1, S2 fit the 32-bit table sums for |dz| < 2^m - dz_bound
  uint32_t nlim_pack;     // largest n of the packed word n * 2^ns + sum(dz + dz_bound) (and of S2)
  uint32_t nlim3c;        // three-word layout: largest n whose sums of dz - res_mm / 2 and of its
                          // square fit 32 bits (below 2^16 when sym32)
  int32_t ns_shift;       // ns, the shift of n in the packed word
  int32_t wide_shift;     // ns + b, b the largest with 2^(b+1) - 2 <= nlim_pack: two n fields
                          // below 2^b sum to at most nlim_pack
  int32_t sym32;          // nlim < 2^16 and every var_thresh < 2^32 (the table scan's symbol
                          // test then multiplies 32-bit values)
  int32_t boxA[6];        // A's occupied bbox (xmin > xmax when empty)
  uint64_t div_x, div_y;  // floor((2^64 - 1) / X) + 1 (0 when X == 1): k / X = umulhi64(div_x, k) for k < 2^32
  uint32_t count_thresh[kMaxLevels];
  int64_t var_thresh[kMaxLevels];
};

// Pose-batched evaluation over one or more scan pairs ("items").  Per pose: per-voxel sums
// in a shared-memory hash table, then the partial joint histogram c[a][b>=1] of the
// occupied B voxels inside boxA and B's occupied bbox; then the overlap, MI and argmax.
struct EvalItem {
  GridConst gc;               // the pair's grid, feature and A bbox
  const uint8_t* symA;        // V
  const int32_t* sat;         // (K-1) x (Z+1) x (Y+1) x (X+1)
  const float4* src;          // point tiles: copies of n_tiles * tile float4 each (raw xyz, or
                              // pre-rotated by one rotation); see pack_points_kernel
  uint64_t src_stride;        // float4 entries per copy
  const int32_t* pose_src;    // P: copy of each pose (nullptr: copy 0)
  const float* poses;         // P x 12
  int32_t n_tiles;            // tiles per copy (>= 3)
  int32_t P;                  // poses of this item
  int32_t pose_base;          // global index of the item's pose 0
  int32_t passes0;            // initial key partitions of this item's poses (power of two; 0: the launch's)
  uint32_t* out_c;            // P x K x K
  int32_t* out_box;           // P x 6
  float* mi;                  // P
  uint32_t* hist;             // optional P x K x K full joint histograms
  unsigned long long* best;   // packed (MI, ~index) running maximum (zeroed before the launch)
  int64_t* argmax;            // one
  int64_t* dump;              // optional: V x 3 (n, S1, S2) of pose 0 (parity checks; S1, S2
                              // are accumulated whenever dump is set, whatever the feature)
  uint32_t* item_passes;      // optional: running max of the partitions this item's poses used
};

struct EvalArgs {
  EvalItem one;               // a copy of items[0] when n_items == 1 (read from the parameter bank)
  const EvalItem* items;
  const int32_t* item_start;  // n_items + 1 ascending global pose offsets (nullptr: one item)
  int32_t n_items;
  int32_t P;                  // poses over all items
  int32_t K;                  // largest symbol count over the items
  int32_t table_slots;
  int32_t passes0;            // initial key-partition passes (power of two)
  int32_t n_buckets;          // table_slots / 4
  uint32_t* err;              // error bits
  uint32_t* max_passes;       // running max of key-partition passes (seed for the next launch)
  uint32_t* wide_count;       // voxels that needed the 64-bit side sums
  uint32_t* wide_poses;       // passes of packed-layout poses sent to the exact path by a wide
                              // voxel (nullptr: not counted)
  unsigned long long* wide;   // per CTA: table_slots x 2 (S1 as two's complement, S2)
  uint32_t* redo_list;        // P: poses whose table overflowed, finished by the redo kernel
  uint32_t* redo_count;       // entries in redo_list (zeroed before every launch)
  uint4* ovf;                 // per CTA: ovf_cap runs (key, n, S1, S2) whose home bucket was full
  int32_t ovf_cap;
  int32_t p_begin;            // eval_kernel: first global pose of this launch (poses p_begin..P-1)
  // Pose pairs (one item, pre-rotated tiles): n_units units of two pose indices each, the
  // second -1 for a single pose.  nullptr: one pose per CTA step (eval_kernel).
  const int32_t* units;
  int32_t n_units;
  // One item, one pose per 2-CTA cluster sharing a table split between the pair's shared
  // memories (eval_cluster_kernel; an even number of CTAs).
  int32_t cluster;
  // eval_kernel, poses with 2 .. spill_np key partitions: B is swept once and its runs are
  // queued here by key partition (per CTA: spill_np queues of spill_cap runs), each pass
  // inserting one queue.  nullptr: every pass sweeps B.
  uint4* spill;
  int64_t spill_cap;
  int32_t spill_np;
};

// One point-tile PackCopy of a batch: scan xyz (n points) -> out (n_out float4), raw
// (rotate == 0) or pre-rotated by R.
struct PackCopy {
  const float* xyz;
  int64_t n;
  int64_t n_out;
  float4* out;
  float R[9];
  int32_t rotate;
  int32_t pad0;
};

// One compiled shape of the eval path.  eval.cu is compiled once per shape (threads per
// CTA, points per thread per tile, resident CTAs per SM); the tile layout of the packed
// points belongs to the shape, so a launch packs and evaluates with the same one.
struct EvalKernels {
  const char* name;
  int threads;      // threads per CTA: one stream of scan points each
  int ppt;          // points per thread per tile
  int ctas_per_sm;  // resident CTAs per SM, each evaluating one pose at a time with its own table
  int (*tile_points)();
  int (*ovf_cap)();  // overflow-list entries per CTA (EvalArgs::ovf holds CTAs x this many)
  int (*min_tiles)();
  // vw: table value words per slot (eval_layout); np: poses swept together (2 for pairs)
  size_t (*smem_bytes)(int K, int table_slots, int vw, int np);
  int (*table_slots_for)(int K, int vw, size_t smem_budget, int np);
  // Raise the kernels' dynamic shared-memory limit on the current device (once per device,
  // before any launch or stream capture).
  cudaError_t (*setup)();
  // vw: table layout (eval_layout); rotate: tiles hold raw xyz (the kernel applies each
  // pose's rotation) instead of pre-rotated copies.  Launches the eval and redo kernels.  A
  // launch with item_start == nullptr is a single-item launch (its item is read from `one`);
  // one with units != nullptr evaluates pose pairs (single item, pre-rotated tiles only).
  cudaError_t (*launch_eval)(const EvalArgs& a, int n_ctas, int vw, bool rotate, cudaStream_t s);
  // xyz (n x 3 fp32) -> n_out float4 with NaN padding; with rots (n_rot x 9), one
  // pre-rotated copy u = R p per rotation (same FMA order as the voxel map).
  cudaError_t (*launch_pack_points)(const float* xyz, int64_t n, int64_t n_out, const float* rots, int n_rot,
                                    float4* out, cudaStream_t s);
  cudaError_t (*launch_pack_batch)(const PackCopy* copies, int n_copies, int64_t max_out, cudaStream_t s);
  // Overlap box, phi column, MI and the running argmax of every pose.
  cudaError_t (*launch_compose)(const EvalArgs& a, cudaStream_t s);
  // Each item's argmax from its packed running maximum.
  cudaError_t (*launch_argmax_finalize)(const EvalItem* items, int n_items, cudaStream_t s);
};
constexpr int kEvalShapes = 3;
// Table value words per slot for a launch over grids with constants gc: 1 without z sums
// (count feature), 2 (n and the biased z sum packed in one word, then S2) when the packed
// word holds at least kPackMinN points per voxel, else 3 (n, S1, S2).
constexpr uint32_t kPackMinN = 2000;
inline int eval_layout(const GridConst& gc, bool var) {
  if (!var) return 1;
  return gc.nlim_pack >= kPackMinN ? 2 : 3;
}
// 0: 1024 threads x 1 point, one CTA per SM; 1: 1024 x 2; 2: 512 x 1, two CTAs per SM.
const EvalKernels& eval_shape(int i);

// One level of a lattice search built on the device (lattice.cu).  Centre: c_prev, moved
// to the previous level's argmax sample when am_prev is set (else c_prev itself).  Pose p:
// rotation cand[opt][p / n_trans] (opt = the previous argmax's rotation sample, 0 without
// one), translation t' = fp32(centre_t + offset_t - origin_t) in FP64.
constexpr int kLatticeMaxAxis = 32;  // samples per pose component of a device-built level
struct LatticeLevel {
  // offset_i = range * (2i - (m - 1)) / (m - 1) of every sample (0 for one sample), computed
  // by the host with the same FP64 operations as its own lattice construction
  double off[6][kLatticeMaxAxis];       // this level's offsets
  double off_prev[6][kLatticeMaxAxis];  // the previous level's offsets
  int32_t m[6];             // samples per pose component (tx, ty, tz, rx, ry, rz; the same every level)
  float origin[3];
  int32_t n_rot;            // rotation samples m[3] * m[4] * m[5]
  int32_t P;                // poses per level
  const double* c_prev;     // 6: the previous level's centre (or the initial centre)
  const int64_t* am_prev;   // the previous level's argmax (nullptr at level 0)
  const float* cand;        // rotations: (options) x n_rot x 9
  double* c_out;            // 6: this level's centre
  float* poses;             // P x 12
  int32_t* pose_src;        // P: rotation sample of each pose (its pre-rotated copy)
  float* rots;              // n_rot x 9
  uint32_t* err;            // error bits
};
cudaError_t launch_lattice_level(const LatticeLevel& L, cudaStream_t s);

cudaError_t launch_ref_accumulate(const GridConst& gc, const float* xyz, int64_t n, const float* pose12,
                                  uint32_t* cnt, unsigned long long* s1, unsigned long long* s2,
                                  cudaStream_t s);
cudaError_t launch_ref_symbols(const GridConst& gc, const uint32_t* cnt, const unsigned long long* s1,
                               const unsigned long long* s2, uint8_t* symA, int32_t* box, cudaStream_t s);
cudaError_t launch_ref_sat(const GridConst& gc, const uint8_t* symA, int32_t* sat, cudaStream_t s);

// Host helpers shared by the C-ABI translation units (defined in runtime.cu).
align_status check_grid_desc(const align_grid_desc* desc, GridConst* gc);
align_status report_error(align_status st, const char* msg);
align_status report_cuda_error(cudaError_t e, const char* what);
void round_pose_host(const float origin[3], const double* eta6, float* pose12);
// P poses; equal consecutive angles reuse the previous rotation (identical results).
void round_poses_host(const float origin[3], const double* eta6, int64_t P, float* poses12);

}  // namespace mialign
