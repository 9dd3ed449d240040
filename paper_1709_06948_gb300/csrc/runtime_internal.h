// runtime_internal.h — host-side state shared by the library's C-ABI translation units
// (grids, device buffers, error reporting).  Not part of the public interface.
#pragma once
#include <cuda_runtime.h>

#include <algorithm>
#include <array>
#include <cstdint>
#include <vector>

#include "align.h"
#include "align_internal.h"

namespace mialign {

// A growable device allocation (cudaMalloc; contents undefined after growth).
struct DevBuf {
  void* p = nullptr;
  size_t cap = 0;
  cudaError_t ensure(size_t bytes) {
    if (bytes <= cap && p != nullptr) return cudaSuccess;
    if (p) cudaFree(p);
    p = nullptr;
    cap = 0;
    size_t want = std::max<size_t>(bytes, 256);
    cudaError_t e = cudaMalloc(&p, want);
    if (e == cudaSuccess) cap = want;
    return e;
  }
  void release() {
    if (p) cudaFree(p);
    p = nullptr;
    cap = 0;
  }
  template <class T>
  T* as() const {
    return static_cast<T*>(p);
  }
};

// A growable page-locked host allocation (asynchronous copies from and to it).
struct HostBuf {
  void* p = nullptr;
  size_t cap = 0;
  cudaError_t ensure(size_t bytes) {
    if (bytes <= cap && p != nullptr) return cudaSuccess;
    if (p) cudaFreeHost(p);
    p = nullptr;
    cap = 0;
    size_t want = std::max<size_t>(bytes, 256);
    cudaError_t e = cudaMallocHost(&p, want);
    if (e == cudaSuccess) cap = want;
    return e;
  }
  void release() {
    if (p) cudaFreeHost(p);
    p = nullptr;
    cap = 0;
  }
  template <class T>
  T* as() const {
    return static_cast<T*>(p);
  }
};

// Error reporting into the thread-local message of align_last_error.
align_status report_errorf(align_status st, const char* fmt, ...);
// Distinct rotations (bitwise-equal 3x3 blocks) of a host pose batch and each pose's
// group; -1 when there are more than max_groups.
int group_pose_rotations(const float* poses12, int64_t P, std::vector<float>& rots, std::vector<int32_t>& idx,
                         int max_groups);
align_status check_grid_device(align_grid* g);
// Pose pairs of a host pose batch for the pair kernel: poses with the same tile copy
// (src, or all one copy when NULL) and bitwise equal t'_y, t'_z, two per unit in order of
// their first pose (local indices; the second -1 for a single pose).  Returns the units.
int pair_units(const float* poses12, const int32_t* src, int64_t P, std::vector<int32_t>& units);
// Whether pose pairs are the automatic choice for a grid with these learned key-partition
// counts (pairs, single poses).
bool pairs_fit(const align_grid* g, int32_t seed_pair, int32_t seed_single);
// One level of the coarse-to-fine lattice: FP64 poses around centre c (ranges r, m samples
// per axis; order rx, ry, rz, tx, ty, tz with tz fastest) and their rounded FP32 form.
void lattice_poses(const float origin[3], const double c[6], const double r[6], const int32_t m[6],
                   std::vector<double>& eta, std::vector<float>& poses);

}  // namespace mialign

// A grid: its voxel map, the resident reference state of scan A, and the workspace of its
// own evaluations.
struct align_grid {
  mialign::GridConst gc{};
  float origin[3];
  float res_m;
  int64_t V = 0;
  cudaStream_t stream = nullptr;
  int device = 0;
  int n_sm = 0;
  int table_slots = 0;  // of the last launch (it depends on the table layout)
  size_t smem_optin = 0;
  bool has_ref = false;
  int32_t boxA[6];
  mialign::DevBuf symA, sat;
  // evaluation workspace
  mialign::DevBuf xyz, poses, out_c, out_box, mi, hist, best, argmax, err, max_passes, wide_count, wide, dump;
  mialign::DevBuf pts4, pose_src, rots, redo_list, redo_count, items, ovf;
  // device-built lattice levels (align_search_ex): centres, rotation tables, read-backs
  mialign::DevBuf lat_c, lat_cand;
  // reference-build working buffers (align_set_reference)
  mialign::DevBuf ref_pts, ref_pose, ref_cnt, ref_s1, ref_s2, ref_box;
  mialign::HostBuf ref_box_h;
  bool ref_pose_set = false;
  mialign::HostBuf lat_cand_h, lat_rec_h, lat_c_h;
  std::vector<cudaEvent_t> lat_ev;
  bool lat_pending = false;  // a search's copies may still be reading the pinned buffers
  int64_t n_points = 0;  // points staged in `xyz`
  // key partitions the next launch starts with, per kernel shape (its table size), and for
  // the pose-pair kernel (shape 0)
  int32_t passes_seed[mialign::kEvalShapes] = {1, 1, 1};
  int32_t passes_seed_pair[mialign::kEvalShapes] = {1, 1, 1};
  int32_t passes_seed_cluster = 1;  // the 2-CTA cluster kernel (shape 0)
  int32_t sweep_mode = -1;  // -1 automatic, else the sweep kind every launch takes (align_set_sweep)
  bool last_pairs = false;    // the last eval launch evaluated pose pairs
  bool last_cluster = false;  // ... or ran one pose per 2-CTA cluster
  mialign::DevBuf units;    // pose pairs of the last pair launch with host poses
  mialign::DevBuf spill;    // runs queued for the later key partitions (EvalArgs::spill)
  int32_t spill_on = 1;     // align_set_spill
  int32_t layout_min = 1;   // smallest table layout (value words) of this grid's z-sum launches:
                            // 3 once packed-layout poses went to the exact path for a wide voxel
  int32_t last_vw = 0;      // the layout of the last eval launch
  int64_t spill_runs = 0;   // runs per queue and CTA (0: half the padded points of B)
  int32_t spill_np_max = 8; // most key partitions the spill queues serve (a server's workspace: its request's)
  mialign::DevBuf lat_units;           // pose pairs of a device-built lattice level (by index)
  std::vector<int32_t> lattice_units;  // ... on the host
  int32_t lattice_units_m[6] = {0, 0, 0, 0, 0, 0};
  int64_t stats[6] = {0, 0, 0, 0, 0, 0};
  // event timing (align_profile): one (before eval, after eval, after argmax) triple per
  // launch, drained into the totals at the next synchronising call or profile read
  bool profiling = false;
  std::vector<std::array<cudaEvent_t, 3>> ev_pending, ev_pool;
  double prof[3] = {0.0, 0.0, 0.0};
};
