// runtime.cu — the C ABI of include/align.h: grids with resident reference state,
// pose-batched MI evaluation, per-voxel sum export, lattice search, errors.
// Host code is compiled with -ffp-contract=off so that the FP64 pose rounding and the
// lattice offsets are evaluated exactly as written.
#include <cuda_runtime.h>

#include <algorithm>
#include <array>
#include <climits>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <unordered_map>
#include <vector>

#include "align.h"
#include "align_internal.h"
#include "runtime_internal.h"

using namespace mialign;

namespace {

thread_local std::string g_last_error;

align_status fail(align_status st, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_last_error = buf;
  return st;
}

align_status cuda_fail(cudaError_t e, const char* what) {
  (void)cudaGetLastError();  // clear a sticky non-fatal error
  if (e == cudaErrorMemoryAllocation) return fail(ALIGN_E_OOM, "%s: %s", what, cudaGetErrorString(e));
  return fail(ALIGN_E_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

#define CU(call, what)                                    \
  do {                                                    \
    cudaError_t e_ = (call);                              \
    if (e_ != cudaSuccess) return cuda_fail(e_, (what));  \
  } while (0)


}  // namespace


namespace {

// --------------------------------------------------------------------------------------
// Host-side conventions (the library's own implementation of the stated convention).
// --------------------------------------------------------------------------------------
// R = Rz(thz) Ry(thy) Rx(thx) from the cosines and sines of the three angles, FP64, rounded
// once to FP32.
void rotation_fp32(double cx, double sx, double cy, double sy, double cz, double sz, float* out9) {
  const double czsy = cz * sy;
  const double szsy = sz * sy;
  const double R[9] = {cz * cy, czsy * sx - sz * cx, czsy * cx + sz * sx,
                       sz * cy, szsy * sx + cz * cx, szsy * cx - cz * sx,
                       -sy,     cy * sx,             cy * cx};
  for (int i = 0; i < 9; ++i) out9[i] = (float)R[i];
}

void pose_to_fp32(const float origin[3], const double* eta, float* out12);

// Many poses, each as pose_to_fp32; a pose whose three angles equal the previous pose's
// (bit for bit) takes the previous pose's rotation, so lattices listed rotation-major pay
// the cosines and sines once per rotation.
void poses_to_fp32(const float origin[3], const double* eta6, int64_t P, float* poses12) {
  for (int64_t p = 0; p < P; ++p) {
    const double* e = eta6 + 6 * p;
    float* out = poses12 + 12 * p;
    if (p > 0 && std::memcmp(e + 3, e - 3, 3 * sizeof(double)) == 0) {
      std::memcpy(out, out - 12, 9 * sizeof(float));
      for (int i = 0; i < 3; ++i) out[9 + i] = (float)(e[i] - (double)origin[i]);
    } else {
      pose_to_fp32(origin, e, out);
    }
  }
}

void pose_to_fp32(const float origin[3], const double* eta, float* out12) {
  // R = Rz(thz) Ry(thy) Rx(thx), FP64, rounded once; t' = t - origin.
  const double cx = std::cos(eta[3]), sx = std::sin(eta[3]);
  const double cy = std::cos(eta[4]), sy = std::sin(eta[4]);
  const double cz = std::cos(eta[5]), sz = std::sin(eta[5]);
  const double czsy = cz * sy;
  const double szsy = sz * sy;
  const double R[9] = {cz * cy, czsy * sx - sz * cx, czsy * cx + sz * sx,
                       sz * cy, szsy * sx + cz * cx, szsy * cx - cz * sx,
                       -sy,     cy * sx,             cy * cx};
  for (int i = 0; i < 9; ++i) out12[i] = (float)R[i];
  for (int i = 0; i < 3; ++i) out12[9 + i] = (float)(eta[i] - (double)origin[i]);
}

// Evenly spread samples over centre +- range (one sample: the centre itself).
double lattice_step(double range, int32_t count, int32_t i) {
  if (count < 2) return 0.0;
  const double num = range * (double)(2 * i - (count - 1));
  return num / (double)(count - 1);
}

// Rounded poses of a lattice: the FP64 rotation of each distinct (rx, ry, rz) sample is
// evaluated once (same operations as pose_to_fp32, so the bits are identical).
void round_lattice(const float origin[3], const std::vector<double>& eta, const int32_t m[6],
                   std::vector<float>& poses) {
  const int64_t P = (int64_t)(eta.size() / 6);
  const int64_t n_trans = (int64_t)m[0] * m[1] * m[2];
  poses.resize((size_t)P * 12);
  for (int64_t p = 0; p < P; ++p) {
    float* out = &poses[(size_t)p * 12];
    if (p % n_trans == 0) {
      pose_to_fp32(origin, &eta[(size_t)p * 6], out);
    } else {
      const float* first = &poses[(size_t)(p - p % n_trans) * 12];
      for (int i = 0; i < 9; ++i) out[i] = first[i];
      for (int i = 0; i < 3; ++i) out[9 + i] = (float)(eta[(size_t)p * 6 + i] - (double)origin[i]);
    }
  }
}

void build_lattice(const double c[6], const double r[6], const int32_t m[6], std::vector<double>& eta) {
  // order: rx, ry, rz, tx, ty, tz (last fastest)
  const int64_t P = (int64_t)m[0] * m[1] * m[2] * m[3] * m[4] * m[5];
  eta.resize((size_t)P * 6);
  for (int64_t idx = 0; idx < P; ++idx) {
    int64_t rem = idx;
    const int32_t itz = (int32_t)(rem % m[2]); rem /= m[2];
    const int32_t ity = (int32_t)(rem % m[1]); rem /= m[1];
    const int32_t itx = (int32_t)(rem % m[0]); rem /= m[0];
    const int32_t irz = (int32_t)(rem % m[5]); rem /= m[5];
    const int32_t iry = (int32_t)(rem % m[4]); rem /= m[4];
    const int32_t irx = (int32_t)rem;
    double* e = &eta[(size_t)idx * 6];
    e[0] = c[0] + lattice_step(r[0], m[0], itx);
    e[1] = c[1] + lattice_step(r[1], m[1], ity);
    e[2] = c[2] + lattice_step(r[2], m[2], itz);
    e[3] = c[3] + lattice_step(r[3], m[3], irx);
    e[4] = c[4] + lattice_step(r[4], m[4], iry);
    e[5] = c[5] + lattice_step(r[5], m[5], irz);
  }
}

align_status validate_desc(const align_grid_desc* d, GridConst* gc) {
  if (!d) return fail(ALIGN_E_INVALID, "desc is NULL");
  for (int i = 0; i < 3; ++i)
    if (d->dims[i] < 1 || d->dims[i] > (1 << 20)) return fail(ALIGN_E_INVALID, "dims[%d] out of [1, 2^20]", i);
  const int64_t V = (int64_t)d->dims[0] * d->dims[1] * d->dims[2];
  if (V >= INT32_MAX) return fail(ALIGN_E_INVALID, "X*Y*Z must be below 2^31");
  for (int i = 0; i < 3; ++i)
    if (!std::isfinite(d->origin[i])) return fail(ALIGN_E_INVALID, "origin not finite");
  if (!(d->res_m > 0.0f) || !std::isfinite(d->res_m)) return fail(ALIGN_E_INVALID, "res_m must be > 0");
  const double mm = (double)d->res_m * 1000.0;
  const int64_t res_mm = (int64_t)std::llround(mm);
  if (res_mm < 1 || res_mm > 8000 || std::fabs(mm - (double)res_mm) > 1e-3)
    return fail(ALIGN_E_INVALID, "res_m must be a whole number of millimetres in [1, 8000]");
  if (d->feature < ALIGN_FEAT_COUNT || d->feature > ALIGN_FEAT_COUNT_ZVAR)
    return fail(ALIGN_E_INVALID, "unknown feature %d", d->feature);
  const bool use_c = d->feature != ALIGN_FEAT_ZVAR;
  const bool use_v = d->feature != ALIGN_FEAT_COUNT;
  const int Lc = use_c ? d->count_levels : 1;
  const int Lv = use_v ? d->var_levels : 1;
  if (use_c && (Lc < 1 || Lc > kMaxLevels)) return fail(ALIGN_E_INVALID, "count_levels out of [1, 63]");
  if (use_v && (Lv < 1 || Lv > kMaxLevels)) return fail(ALIGN_E_INVALID, "var_levels out of [1, 63]");
  int K = d->feature == ALIGN_FEAT_COUNT ? 1 + Lc : d->feature == ALIGN_FEAT_ZVAR ? 1 + Lv : 1 + Lc * Lv;
  if (K > kMaxSymbols) return fail(ALIGN_E_INVALID, "too many symbols (%d > 64)", K);

  std::memset(gc, 0, sizeof(*gc));
  gc->inv_res = (float)(1.0 / (double)d->res_m);
  gc->res_mm = (int32_t)res_mm;
  gc->X = d->dims[0];
  gc->Y = d->dims[1];
  gc->Z = d->dims[2];
  gc->K = K;
  gc->feature = d->feature;
  gc->Lc = Lc;
  gc->Lv = Lv;
  for (int j = 0; j < kMaxLevels; ++j) {
    gc->count_thresh[j] = 0xFFFFFFFFu;
    gc->var_thresh[j] = INT64_MAX;
  }
  for (int j = 0; j + 1 < Lc; ++j) {
    gc->count_thresh[j] = d->count_thresh ? d->count_thresh[j] : (j + 1 < 32 ? (1u << (j + 1)) : 0xFFFFFFFFu);
    if (j > 0 && gc->count_thresh[j] < gc->count_thresh[j - 1])
      return fail(ALIGN_E_INVALID, "count_thresh must be ascending");
  }
  const int64_t r2 = res_mm * res_mm;
  for (int j = 0; j + 1 < Lv; ++j) {
    const int shift = 2 + (Lv - 1 - j);
    gc->var_thresh[j] = d->var_thresh ? d->var_thresh[j] : (shift >= 63 ? 0 : (r2 >> shift));
    if (gc->var_thresh[j] < 0) return fail(ALIGN_E_INVALID, "var_thresh must be >= 0");
    if (j > 0 && gc->var_thresh[j] < gc->var_thresh[j - 1])
      return fail(ALIGN_E_INVALID, "var_thresh must be ascending");
  }
  // z offsets: for a point inside the grid (0 <= fl(g_z * inv_res) < Z), the FP32 errors of
  // inv_res = fl(1/res), fl(g_z * inv_res) and fl(g_z * 1000) together with the drift of
  // k_z * res_mm against 1000 * k_z * res move 1000 * g_z by at most
  // Z * res_mm * 2.2 * 2^-24 + Z * |1000 res - res_mm| + 2^-24 * (Z * res_mm + 1) < 1/2 mm
  // under the two limits below, so zq = round(g_z * 1000) lies in [k_z, k_z + 1] * res_mm
  // and 0 <= dz <= res_mm: the sweep needs no per-point check.
  if ((int64_t)gc->Z * res_mm >= (int64_t(1) << 20))
    return fail(ALIGN_E_INVALID, "the grid is too tall: Z * res must stay below 1,048 m");
  const double drift = std::fabs(mm - (double)res_mm) * (double)gc->Z;
  if (drift >= 0.25) return fail(ALIGN_E_INVALID, "res_m is too far from a whole number of mm for Z layers");
  gc->dz_bound = (int32_t)(res_mm + 4 + (int64_t)std::ceil(drift));
  int m = 0;
  while ((1 << m) <= 2 * gc->dz_bound) ++m;
  gc->dz_shift = m;
  // the sweep's check accepts dz in [-dz_bound, 2^m - 1 - dz_bound], i.e. dz + dz_bound in
  // [0, 2^m - 1].  The table packs n and the biased sum S1' = sum(dz + dz_bound) into one
  // word n * 2^ns + S1': exact while n < 2^(32 - ns) and n * (2^m - 1) < 2^ns; ns is chosen
  // for the largest such n, and S2 = sum(dz^2) must also fit 32 bits.
  const uint64_t D = (uint64_t)((1 << m) - 1 - gc->dz_bound);  // largest |dz|
  uint64_t best = 0;
  int best_ns = m;
  for (int ns = m; ns <= 31; ++ns) {
    const uint64_t lim = std::min<uint64_t>((1ull << (32 - ns)) - 1, ((1ull << ns) - 1) / ((1ull << m) - 1));
    if (lim > best) best = lim, best_ns = ns;
  }
  gc->ns_shift = best_ns;
  gc->nlim = (uint32_t)std::min<uint64_t>(0xFFFFFFFFull / (D * D), 0x7FFFFFFFull / D);
  gc->nlim_pack = (uint32_t)std::min<uint64_t>(best, gc->nlim);
  // The three-word table layout sums dz - c with c = res_mm / 2: shifting every dz of a voxel
  // by c leaves n * S2 - S1^2 (all the feature symbols read) unchanged, and |dz - c| is at
  // most res_mm - c for in-grid points (0 <= dz <= res_mm, above), a quarter of the squares
  // (plus the same margin as dz_bound).
  const uint64_t Dc = (uint64_t)(res_mm - res_mm / 2 + 4 + (int64_t)std::ceil(drift));
  gc->nlim3c = (uint32_t)std::min<uint64_t>(0xFFFFFFFFull / (Dc * Dc), 0x7FFFFFFFull / Dc);
  int b = 0;
  while (b < 30 && (2ull << (b + 1)) - 2ull <= (uint64_t)gc->nlim_pack) ++b;
  gc->wide_shift = std::min(31, best_ns + b);
  gc->sym32 = gc->nlim < 65536u ? 1 : 0;
  for (int j = 0; j + 1 < Lv; ++j)
    if (gc->var_thresh[j] >= (int64_t(1) << 32)) gc->sym32 = 0;
  // the 32-bit symbol test needs n < 2^16 (nlim3c >= nlim either way: |dz - c| <= |dz|)
  if (gc->sym32) gc->nlim3c = std::min(gc->nlim3c, 65535u);
  for (int i = 0; i < 3; ++i) gc->boxA[i] = INT_MAX, gc->boxA[3 + i] = INT_MIN;
  // division of 32-bit keys by X and Y as a 64-bit multiply-high (Lemire, Kaser and Kurz,
  // "Faster remainder by direct computation", 2019: exact for every 32-bit dividend)
  gc->div_x = gc->X > 1 ? UINT64_MAX / (uint64_t)gc->X + 1 : 0;
  gc->div_y = gc->Y > 1 ? UINT64_MAX / (uint64_t)gc->Y + 1 : 0;
  return ALIGN_OK;
}

align_status check_grid(align_grid* g) {
  if (!g) return fail(ALIGN_E_INVALID, "grid is NULL");
  cudaError_t e = cudaSetDevice(g->device);
  if (e != cudaSuccess) return cuda_fail(e, "cudaSetDevice");
  return ALIGN_OK;
}

// Stage scan B (n x 3 fp32) in device memory; every evaluation packs it into tiles.
align_status upload_points(align_grid* g, const float* xyz, int64_t n, int flags, int32_t* n_tiles_out) {
  if (n < 0 || n >= INT32_MAX) return fail(ALIGN_E_INVALID, "point count out of range");
  if (n > 0 && !xyz) return fail(ALIGN_E_INVALID, "xyz is NULL");
  const EvalKernels& ek = eval_shape(0);
  const int tile = ek.tile_points();
  const int64_t n_tiles = std::max<int64_t>(ek.min_tiles(), (n + tile - 1) / tile);
  CU(g->xyz.ensure(std::max<size_t>(1, (size_t)n) * 3 * sizeof(float)), "allocate point buffer");
  if (n > 0) {
    const cudaMemcpyKind kind = (flags & ALIGN_XYZ_DEVICE) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    CU(cudaMemcpyAsync(g->xyz.p, xyz, (size_t)n * 3 * sizeof(float), kind, g->stream), "copy points");
  }
  g->n_points = n;
  *n_tiles_out = (int32_t)n_tiles;
  return ALIGN_OK;
}

// Distinct rotations of a host pose batch (bitwise equal 3x3 blocks), and each pose's index.
struct RotKey {
  uint32_t w[9];
  bool operator==(const RotKey& o) const { return std::memcmp(w, o.w, sizeof(w)) == 0; }
};
struct RotHash {
  size_t operator()(const RotKey& k) const {
    uint64_t h = 1469598103934665603ull;
    for (uint32_t v : k.w) h = (h ^ v) * 1099511628211ull;
    return (size_t)h;
  }
};

int group_rotations(const float* poses12, int64_t P, std::vector<float>& rots, std::vector<int32_t>& idx,
                    int max_groups) {
  std::unordered_map<RotKey, int32_t, RotHash> seen;
  rots.clear();
  idx.resize((size_t)P);
  for (int64_t p = 0; p < P; ++p) {
    // lattices list poses rotation-major: most poses share the previous pose's rotation
    if (p > 0 && std::memcmp(poses12 + 12 * p, poses12 + 12 * (p - 1), 9 * sizeof(float)) == 0) {
      idx[(size_t)p] = idx[(size_t)(p - 1)];
      continue;
    }
    RotKey k;
    std::memcpy(k.w, poses12 + 12 * p, sizeof(k.w));
    auto it = seen.find(k);
    if (it == seen.end()) {
      if ((int)seen.size() >= max_groups) return -1;
      it = seen.emplace(k, (int32_t)seen.size()).first;
      rots.insert(rots.end(), poses12 + 12 * p, poses12 + 12 * p + 9);
    }
    idx[(size_t)p] = it->second;
  }
  return (int)seen.size();
}

// Error word and counters: allocated once per grid and zeroed (cudaMalloc memory is not).
align_status ensure_status_words(align_grid* g) {
  if (g->err.p && g->max_passes.p && g->wide_count.p) return ALIGN_OK;
  CU(g->err.ensure(16), "allocate error word");
  CU(g->max_passes.ensure(16), "allocate counters");
  CU(g->wide_count.ensure(16), "allocate counters");
  CU(cudaMemsetAsync(g->err.p, 0, 16, g->stream), "clear error word");
  CU(cudaMemsetAsync(g->max_passes.p, 0, 16, g->stream), "clear counters");
  CU(cudaMemsetAsync(g->wide_count.p, 0, 16, g->stream), "clear counters");
  return ALIGN_OK;
}

struct EvalOut {
  float* mi;          // device
  uint32_t* hist;     // device or null
  int64_t* argmax;    // device
  int64_t* dump;      // device or null
};

// Whether a batch of P poses with n_rot distinct rotations gets one pre-rotated tile copy
// per rotation (else one raw copy, rotated per pose by the kernel).
int max_rotation_copies(int64_t P, int32_t n_tiles) {
  const EvalKernels& ek = eval_shape(0);
  const int64_t n_pad = (int64_t)n_tiles * ek.tile_points();
  const int max_groups = (int)std::max<int64_t>(1, P / 4);
  const size_t budget = (size_t)512 << 20;
  const int cap_mem = (int)std::max<int64_t>(0, (int64_t)(budget / ((size_t)n_pad * 16)));
  return std::min(max_groups, cap_mem);
}

// Pose pairs for the pair kernel: poses that read the same pre-rotated tile copy (group
// index `src`) and whose t'_y and t'_z are equal bit for bit, two at a time in order of
// their first pose; a group's odd pose is a unit of its own.  Two entries per unit (the
// second -1 for a single pose).  Returns the unit count.
int pair_units_impl(const float* poses12, const int32_t* src, int64_t P, std::vector<int32_t>& units) {
  struct Key {
    int32_t src;
    uint32_t ty, tz;
    bool operator==(const Key& o) const { return src == o.src && ty == o.ty && tz == o.tz; }
  };
  struct KeyHash {
    size_t operator()(const Key& k) const {
      return (size_t)(((uint64_t)(uint32_t)k.src * 0x9E3779B97F4A7C15ull) ^ ((uint64_t)k.ty << 32 | k.tz));
    }
  };
  std::unordered_map<Key, int64_t, KeyHash> open;  // pose waiting for a partner, per key
  std::vector<int64_t> partner((size_t)P, -2);     // -2: not yet placed
  units.clear();
  std::vector<std::pair<int64_t, int64_t>> pairs;
  for (int64_t p = 0; p < P; ++p) {
    Key k;
    k.src = src ? src[p] : 0;
    std::memcpy(&k.ty, poses12 + 12 * p + 10, 4);
    std::memcpy(&k.tz, poses12 + 12 * p + 11, 4);
    auto it = open.find(k);
    if (it == open.end()) {
      open.emplace(k, p);
    } else {
      pairs.emplace_back(it->second, p);
      open.erase(it);
    }
  }
  for (const auto& kv : open) pairs.emplace_back(kv.second, -1);
  std::sort(pairs.begin(), pairs.end());
  for (const auto& q : pairs) {
    units.push_back((int32_t)q.first);
    units.push_back((int32_t)q.second);
  }
  return (int)pairs.size();
}

// Whether the next pre-rotated launch on this grid evaluates pose pairs (automatic choice,
// from the key-partition counts learned per grid, which only grow): while pairs have needed
// no more partitions than single poses, one pair sweep does the work of two single sweeps;
// and where both need partitions, the spill queues sweep the points once whatever the count,
// so pairs pay only their extra passes' table scans: measured per 4,096 poses 2.44 against
// 2.51 ms (0.25 m LiDAR grid, 4 against 2 partitions), and even on the 6.4M-voxel grid (8
// against 4; 6.6-6.8 against 6.6-7.0 ms over three runs).
}  // namespace
bool mialign::pairs_fit(const align_grid* g, int32_t seed_pair, int32_t seed_single) {
  if (seed_pair <= seed_single) return true;
  return g->spill_on && seed_single >= 2 && seed_pair <= 2 * seed_single && seed_pair <= g->spill_np_max;
}
namespace {
bool use_pairs(const align_grid* g) {
  return g->sweep_mode < 0 ? pairs_fit(g, g->passes_seed_pair[0], g->passes_seed[0]) : g->sweep_mode == 1;
}

// Whether a launch of single poses runs one pose per 2-CTA cluster: while the grid's single
// poses need at least 8 key partitions and the cluster's twice-as-large table has needed
// fewer.  Half of a cluster's table inserts go to the peer CTA's shared memory and wait
// several times as long as a local insert; measured per 4,096 poses, halving 2 partitions
// to 1 loses (4.01 against 2.81 ms, 0.25 m LiDAR grid) and halving 4 to 2 breaks even
// (10.14 against 10.04 ms, 0.2 m 6.4M-voxel grid).
bool use_cluster(const align_grid* g) {
  if (g->sweep_mode >= 0) return g->sweep_mode == 2 && g->n_sm >= 2;
  return g->n_sm >= 2 && g->passes_seed[0] >= 8 && g->passes_seed_cluster < g->passes_seed[0];
}

align_status enqueue_eval_core(align_grid* g, int32_t n_tiles, const float* d_poses, int64_t P, bool rotate,
                               int n_rot, const EvalOut& out, const int32_t* d_units = nullptr,
                               int32_t n_units = 0, bool cluster = false);

// Enqueue pack + eval + redo + compose + argmax for poses already on the device.
// h_poses (may be NULL): the same poses on the host, used to find shared rotations (and
// pose pairs).
align_status enqueue_eval(align_grid* g, int32_t n_tiles, const float* d_poses, const float* h_poses, int64_t P,
                          const EvalOut& out) {
  bool rotate = true;
  int n_rot = 0;
  if (h_poses != nullptr) {
    std::vector<float> rots;
    std::vector<int32_t> idx;
    const int groups = group_rotations(h_poses, P, rots, idx, max_rotation_copies(P, n_tiles));
    if (groups > 0 && out.dump == nullptr && P >= 2 && use_pairs(g)) {
      std::vector<int32_t> units;
      const int n_units = pair_units_impl(h_poses, idx.data(), P, units);
      if (n_units < P) {  // at least one pair
        CU(g->rots.ensure(rots.size() * 4), "allocate rotations");
        CU(cudaMemcpyAsync(g->rots.p, rots.data(), rots.size() * 4, cudaMemcpyHostToDevice, g->stream),
           "copy rotations");
        CU(g->pose_src.ensure((size_t)P * 4), "allocate pose sources");
        CU(cudaMemcpyAsync(g->pose_src.p, idx.data(), (size_t)P * 4, cudaMemcpyHostToDevice, g->stream),
           "copy pose sources");
        CU(g->units.ensure(units.size() * 4), "allocate pose pairs");
        CU(cudaMemcpyAsync(g->units.p, units.data(), units.size() * 4, cudaMemcpyHostToDevice, g->stream),
           "copy pose pairs");
        // the copies read pageable host memory: they complete before this call returns
        return enqueue_eval_core(g, n_tiles, d_poses, P, false, groups, out, g->units.as<int32_t>(), n_units);
      }
    }
    if (groups > 0) {
      CU(g->rots.ensure(rots.size() * 4), "allocate rotations");
      CU(cudaMemcpyAsync(g->rots.p, rots.data(), rots.size() * 4, cudaMemcpyHostToDevice, g->stream),
         "copy rotations");
      CU(g->pose_src.ensure((size_t)P * 4), "allocate pose sources");
      CU(cudaMemcpyAsync(g->pose_src.p, idx.data(), (size_t)P * 4, cudaMemcpyHostToDevice, g->stream),
         "copy pose sources");
      rotate = false;
      n_rot = groups;
    }
  }
  return enqueue_eval_core(g, n_tiles, d_poses, P, rotate, n_rot, out, nullptr, 0,
                           out.dump == nullptr && use_cluster(g));
}

// The launches of one evaluation.  Unless `rotate`, g->rots holds n_rot rotations and
// g->pose_src each pose's rotation (on the device, in stream order).
align_status enqueue_eval_core(align_grid* g, int32_t n_tiles, const float* d_poses, int64_t P, bool rotate,
                               int n_rot, const EvalOut& out, const int32_t* d_units, int32_t n_units,
                               bool cluster) {
  const int K = g->gc.K;
  const size_t KK = (size_t)K * K;
  CU(g->out_c.ensure((size_t)P * KK * sizeof(uint32_t)), "allocate histograms");
  CU(g->out_box.ensure((size_t)P * 6 * sizeof(int32_t)), "allocate boxes");
  CU(g->best.ensure(sizeof(unsigned long long)), "allocate argmax");
  align_status st0 = ensure_status_words(g);
  if (st0 != ALIGN_OK) return st0;
  const bool pairs = d_units != nullptr && n_units > 0 && !rotate;
  cluster = cluster && !pairs;
  const int n_ctas = cluster ? 2 * (int)std::min<int64_t>(P, g->n_sm / 2)
                             : (int)std::min<int64_t>(pairs ? n_units : P, g->n_sm);
  const bool var = g->gc.feature != ALIGN_FEAT_COUNT || out.dump != nullptr;
  const int vw = var ? std::max(eval_layout(g->gc, var), g->layout_min) : eval_layout(g->gc, var);
  g->last_vw = vw;
  g->table_slots = eval_shape(0).table_slots_for(K, vw, g->smem_optin, pairs ? 2 : 1);
  g->last_pairs = pairs;
  g->last_cluster = cluster;
  const size_t wide_bytes = (size_t)n_ctas * 2 * g->table_slots * sizeof(unsigned long long);
  if (g->wide.cap < wide_bytes || g->wide.p == nullptr) {
    CU(g->wide.ensure(wide_bytes), "allocate wide sums");
    CU(cudaMemsetAsync(g->wide.p, 0, g->wide.cap, g->stream), "clear wide sums");
  }
  CU(cudaMemsetAsync(g->best.p, 0, sizeof(unsigned long long), g->stream), "reset argmax");
  CU(g->redo_list.ensure((size_t)P * 4), "allocate redo list");
  CU(g->redo_count.ensure(16), "allocate redo count");
  CU(cudaMemsetAsync(g->redo_count.p, 0, 4, g->stream), "reset redo count");

  // Pack B into float4 tiles; when many poses share a rotation, one pre-rotated copy per
  // distinct rotation (the kernel then only translates).
  const EvalKernels& ek = eval_shape(0);
  const int64_t n_pad = (int64_t)n_tiles * ek.tile_points();
  CU(g->pts4.ensure((size_t)std::max(n_rot, 1) * (size_t)n_pad * 16), "allocate tiles");
  CU(ek.launch_pack_points(g->xyz.as<float>(), g->n_points, n_pad, rotate ? nullptr : g->rots.as<float>(), n_rot,
                        g->pts4.as<float4>(), g->stream),
     "launch pack");

  EvalItem item{};
  item.gc = g->gc;
  item.symA = g->symA.as<uint8_t>();
  item.sat = g->sat.as<int32_t>();
  item.src = g->pts4.as<float4>();
  item.src_stride = (uint64_t)n_pad;
  item.pose_src = rotate ? nullptr : g->pose_src.as<int32_t>();
  item.poses = d_poses;
  item.n_tiles = n_tiles;
  item.P = (int32_t)P;
  item.pose_base = 0;
  // a cluster's table holds twice a CTA's keys: it starts from half the single-pose count
  item.passes0 = pairs     ? g->passes_seed_pair[0]
                 : cluster ? std::max(g->passes_seed_cluster, g->passes_seed[0] / 2)
                           : g->passes_seed[0];
  item.item_passes = nullptr;
  item.out_c = g->out_c.as<uint32_t>();
  item.out_box = g->out_box.as<int32_t>();
  item.mi = out.mi;
  item.hist = out.hist;
  item.best = g->best.as<unsigned long long>();
  item.argmax = out.argmax;
  item.dump = out.dump;
  CU(g->items.ensure(sizeof(EvalItem)), "allocate item table");
  CU(cudaMemcpyAsync(g->items.p, &item, sizeof(EvalItem), cudaMemcpyHostToDevice, g->stream), "copy item table");

  EvalArgs a{};
  a.one = item;
  a.items = g->items.as<EvalItem>();
  a.item_start = nullptr;
  a.n_items = 1;
  a.P = (int32_t)P;
  a.K = K;
  a.table_slots = g->table_slots;
  a.n_buckets = g->table_slots / 4;
  a.passes0 = item.passes0;
  a.units = pairs ? d_units : nullptr;
  a.n_units = pairs ? n_units : 0;
  a.cluster = cluster ? 1 : 0;
  a.err = g->err.as<uint32_t>();
  a.max_passes = g->max_passes.as<uint32_t>();
  a.wide_count = g->wide_count.as<uint32_t>();
  a.wide_poses = g->wide_count.as<uint32_t>() + 1;  // the counter buffer's second word
  a.wide = g->wide.as<unsigned long long>();
  a.redo_list = g->redo_list.as<uint32_t>();
  a.redo_count = g->redo_count.as<uint32_t>();
  CU(g->ovf.ensure((size_t)n_ctas * ek.ovf_cap() * 16), "allocate overflow lists");
  a.ovf = g->ovf.as<uint4>();
  a.ovf_cap = ek.ovf_cap();
  // single poses or pose pairs that need key partitions: B swept once, its runs queued by
  // partition (room for one doubling of the seed, at most 8 partitions; half a run per padded
  // point and queue, a whole one for pairs: a queue that fills sends its pose to the exact
  // path)
  if (g->spill_on && !cluster && out.dump == nullptr && item.passes0 >= 2 && item.passes0 <= g->spill_np_max) {
    const int32_t np = std::min(g->spill_np_max, 2 * item.passes0);
    const int64_t cap = ((g->spill_runs > 0 ? g->spill_runs : pairs ? n_pad : n_pad / 2) + 31) / 32 * 32;
    CU(g->spill.ensure((size_t)n_ctas * (size_t)np * (size_t)cap * 16), "allocate spill queues");
    a.spill = g->spill.as<uint4>();
    a.spill_cap = cap;
    a.spill_np = np;
  }
  std::array<cudaEvent_t, 3> evs{};
  if (g->profiling) {
    if (g->ev_pool.empty()) {
      for (cudaEvent_t& e : evs) CU(cudaEventCreate(&e), "create event");
    } else {
      evs = g->ev_pool.back();
      g->ev_pool.pop_back();
    }
    CU(cudaEventRecord(evs[0], g->stream), "record event");
  }
  CU(ek.launch_eval(a, n_ctas, vw, rotate, g->stream), "launch eval kernel");
  if (g->profiling) CU(cudaEventRecord(evs[1], g->stream), "record event");
  CU(ek.launch_compose(a, g->stream), "launch compose kernel");
  CU(ek.launch_argmax_finalize(a.items, 1, g->stream), "launch argmax");
  if (g->profiling) {
    CU(cudaEventRecord(evs[2], g->stream), "record event");
    g->ev_pending.push_back(evs);
  }
  g->stats[2] = g->table_slots;
  g->stats[3] = n_ctas;
  g->stats[5] = pairs ? 1 : cluster ? 2 : 0;
  g->stats[4] += 5;  // pack, eval, redo, compose, argmax
  return ALIGN_OK;
}

// Add the elapsed times of all recorded event triples to the profile totals.
align_status drain_events(align_grid* g) {
  for (auto& evs : g->ev_pending) {
    CU(cudaEventSynchronize(evs[2]), "synchronize event");
    float t0 = 0.0f, t1 = 0.0f;
    CU(cudaEventElapsedTime(&t0, evs[0], evs[1]), "event time");
    CU(cudaEventElapsedTime(&t1, evs[1], evs[2]), "event time");
    g->prof[0] += t0;
    g->prof[1] += t1;
    g->prof[2] += 1.0;
    g->ev_pool.push_back(evs);
  }
  g->ev_pending.clear();
  return ALIGN_OK;
}

// Key partitions the last launch's hardest pose needed: the seed of the next launch of the
// same kind.
void learn_passes(align_grid* g, uint32_t used) {
  if (used == 0 || used > (1u << 16) || (used & (used - 1)) != 0) return;
  int32_t& seed = g->last_pairs ? g->passes_seed_pair[0] : g->last_cluster ? g->passes_seed_cluster : g->passes_seed[0];
  if (used > (uint32_t)seed) seed = (int32_t)used;
}

// Read back the kernels' error word and counters (synchronises the stream).
align_status collect_status(align_grid* g) {
  uint32_t vals[4] = {0, 0, 0, 0};
  CU(cudaMemcpyAsync(&vals[0], g->err.p, 4, cudaMemcpyDeviceToHost, g->stream), "read error word");
  CU(cudaMemcpyAsync(&vals[1], g->max_passes.p, 4, cudaMemcpyDeviceToHost, g->stream), "read counters");
  CU(cudaMemcpyAsync(&vals[2], g->wide_count.p, 8, cudaMemcpyDeviceToHost, g->stream), "read counters");
  CU(cudaStreamSynchronize(g->stream), "synchronize");
  {
    align_status stp = drain_events(g);
    if (stp != ALIGN_OK) return stp;
  }
  CU(cudaMemsetAsync(g->err.p, 0, 4, g->stream), "reset error word");
  CU(cudaMemsetAsync(g->wide_count.p, 0, 8, g->stream), "reset counters");
  CU(cudaMemsetAsync(g->max_passes.p, 0, 4, g->stream), "reset counters");  // a per-launch maximum
  // seed the next launch of the same kind (pairs or single poses) with the largest
  // partition count a pose needed (a power of two)
  learn_passes(g, vals[1]);
  // packed-layout poses that a voxel past nlim_pack sent to the exact path: the grid's scans
  // are dense enough for the three-word layout (a limit several times larger, fewer slots)
  if (vals[3] > 0 && g->last_vw == 2) g->layout_min = 3;
  g->stats[0] = vals[1];
  g->stats[1] = vals[2];
  if (vals[0] & kErrDzBound) return fail(ALIGN_E_INTERNAL, "a z offset exceeded its proven bound");
  if (vals[0] & kErrPassLimit) return fail(ALIGN_E_INTERNAL, "key partitioning limit reached");
  if (vals[0] & kErrLattice) return fail(ALIGN_E_INTERNAL, "a lattice level found its argmax out of range");
  return ALIGN_OK;
}

// Largest rotation table (rotation samples squared) of a search whose levels are built on
// the device; larger rotation lattices take the synchronous path.
constexpr int64_t kMaxLatticeCand = 16384;
constexpr int kMaxAxisSamples = 32;  // rotation samples per axis of a device-built search

// Centre of the next level: the sample `am` of the lattice around c with ranges r (the same
// FP64 operations as build_lattice).
void lattice_sample(const double c[6], const double r[6], const int32_t m[6], int64_t am, double out[6]) {
  int64_t rem = am;
  int32_t i[6];
  i[2] = (int32_t)(rem % m[2]); rem /= m[2];
  i[1] = (int32_t)(rem % m[1]); rem /= m[1];
  i[0] = (int32_t)(rem % m[0]); rem /= m[0];
  i[5] = (int32_t)(rem % m[5]); rem /= m[5];
  i[4] = (int32_t)(rem % m[4]); rem /= m[4];
  i[3] = (int32_t)rem;
  for (int a = 0; a < 6; ++a) out[a] = c[a] + lattice_step(r[a], m[a], i[a]);
}

// Coarse-to-fine lattice search with every level built on the device from the previous
// level's argmax (lattice.cu), so that the levels follow each other on the stream.  Only
// the rotations need the host (FP64 cos/sin, as every other pose rounding): for level l it
// prepares the rotation of every (rotation sample of level l-1, rotation sample of level l)
// pair, which needs level l-1's centre, i.e. level l-2's argmax.  The host therefore waits
// for level l-2 while level l-1 runs, and the device always has the next level queued.
// Results are identical to the level-by-level search: the same poses, bit for bit.
align_status search_pipelined(align_grid* g, int32_t n_tiles, const double c0[6], const double r0[6],
                              const int32_t m[6], int64_t P, int32_t n_rot, int32_t levels, double T_out[6],
                              float* mi_out, int64_t* level_best) {
  const size_t slot = (size_t)n_rot * n_rot * 9;  // floats of one level's rotation table
  struct Rec {
    int64_t am;
    unsigned long long best;
    uint32_t max_passes;
    uint32_t pad;
  };
  CU(g->lat_c.ensure((size_t)(levels + 1) * 6 * sizeof(double)), "allocate lattice centres");
  CU(g->lat_cand.ensure(2 * slot * sizeof(float)), "allocate rotation tables");
  CU(g->poses.ensure((size_t)P * 48), "allocate poses");
  CU(g->rots.ensure((size_t)n_rot * 36), "allocate rotations");
  CU(g->pose_src.ensure((size_t)P * 4), "allocate pose sources");
  CU(g->mi.ensure((size_t)P * 4), "allocate MI");
  CU(g->argmax.ensure(8), "allocate argmax");
  CU(g->lat_cand_h.ensure(2 * slot * sizeof(float)), "allocate pinned rotation tables");
  CU(g->lat_rec_h.ensure((size_t)levels * sizeof(Rec)), "allocate pinned read-back");
  CU(g->lat_c_h.ensure(6 * sizeof(double)), "allocate pinned centre");
  while ((int32_t)g->lat_ev.size() < levels) {
    cudaEvent_t e;
    CU(cudaEventCreateWithFlags(&e, cudaEventDisableTiming), "create event");
    g->lat_ev.push_back(e);
  }
  // copies out of the pinned buffers left by a search that stopped early must be done
  // before the buffers change (a search that finished has synchronised the stream)
  if (g->lat_pending) CU(cudaStreamSynchronize(g->stream), "synchronize");
  g->lat_pending = true;
  // pose pairs of every level (the lattice's index structure: t_x samples 2i and 2i+1 of the
  // same rotation, t_y and t_z), decided once for the whole search
  const bool pairs = P >= 2 && m[0] >= 2 && use_pairs(g);
  const bool cluster = !pairs && use_cluster(g);  // likewise decided once for the search
  int32_t n_units = 0;
  if (pairs) {
    if (!std::equal(m, m + 6, g->lattice_units_m) || g->lat_units.p == nullptr) {
      std::vector<int32_t>& u = g->lattice_units;
      u.clear();
      const int64_t n_yz = (int64_t)m[1] * m[2], n_trans = (int64_t)m[0] * n_yz;
      for (int64_t p = 0; p < P; ++p) {
        const int64_t itx = (p % n_trans) / n_yz;
        if (itx % 2 != 0) continue;
        u.push_back((int32_t)p);
        u.push_back(itx + 1 < m[0] ? (int32_t)(p + n_yz) : -1);
      }
      CU(g->lat_units.ensure(u.size() * 4), "allocate pose pairs");
      // a pageable source: staged before the call returns
      CU(cudaMemcpyAsync(g->lat_units.p, u.data(), u.size() * 4, cudaMemcpyHostToDevice, g->stream),
         "copy pose pairs");
      std::copy(m, m + 6, g->lattice_units_m);
    }
    n_units = (int32_t)(g->lattice_units.size() / 2);
  }
  Rec* rec = g->lat_rec_h.as<Rec>();
  std::vector<std::array<double, 6>> c((size_t)levels + 1), r((size_t)levels);
  for (int a = 0; a < 6; ++a) c[0][a] = c0[a], r[0][a] = r0[a];
  for (int32_t l = 1; l < levels; ++l)
    for (int a = 0; a < 6; ++a) r[(size_t)l][a] = r[(size_t)l - 1][a] * 0.5;
  std::memcpy(g->lat_c_h.p, c0, 6 * sizeof(double));
  CU(cudaMemcpyAsync(g->lat_c.p, g->lat_c_h.p, 6 * sizeof(double), cudaMemcpyHostToDevice, g->stream),
     "copy centre");
  double* d_c = g->lat_c.as<double>();
  uint32_t passes_used = 0;
  for (int32_t l = 0; l < levels; ++l) {
    if (l >= 2) {  // level l-1's centre, from level l-2's argmax
      CU(cudaEventSynchronize(g->lat_ev[(size_t)l - 2]), "wait for a lattice level");
      const Rec& q = rec[l - 2];
      if (q.am < 0 || q.am >= P) return fail(ALIGN_E_INTERNAL, "argmax out of range");
      lattice_sample(c[(size_t)l - 2].data(), r[(size_t)l - 2].data(), m, q.am, c[(size_t)l - 1].data());
      passes_used = std::max(passes_used, q.max_passes);
      learn_passes(g, q.max_passes);
    }
    // rotation table of level l: options = rotation samples of level l-1 (one at level 0).
    // Per axis the angle of (option sample i, sample j) is centre + offset_i + offset_j; its
    // cosine and sine are taken once (the same values pose_to_fp32 would compute).
    float* tab = g->lat_cand_h.as<float>() + (size_t)(l % 2) * slot;
    const int32_t n_opt = l == 0 ? 1 : n_rot;
    double cs[3][2][kMaxAxisSamples * kMaxAxisSamples];
    for (int ax = 0; ax < 3; ++ax) {
      const int a = 3 + ax, ma = m[a];
      for (int32_t io = 0; io < (l == 0 ? 1 : ma); ++io)
        for (int32_t j = 0; j < ma; ++j) {
          const double centre = l == 0 ? c[0][a] : c[(size_t)l - 1][a] + lattice_step(r[(size_t)l - 1][a], ma, io);
          const double ang = centre + lattice_step(r[(size_t)l][a], ma, j);
          cs[ax][0][io * ma + j] = std::cos(ang);
          cs[ax][1][io * ma + j] = std::sin(ang);
        }
    }
    for (int32_t opt = 0; opt < n_opt; ++opt) {
      const int32_t oz = opt % m[5], oy = (opt / m[5]) % m[4], ox = opt / (m[5] * m[4]);
      for (int32_t jr = 0; jr < n_rot; ++jr) {
        const int32_t jz = jr % m[5], jy = (jr / m[5]) % m[4], jx = jr / (m[5] * m[4]);
        const int ix = ox * m[3] + jx, iy = oy * m[4] + jy, iz = oz * m[5] + jz;
        rotation_fp32(cs[0][0][ix], cs[0][1][ix], cs[1][0][iy], cs[1][1][iy], cs[2][0][iz], cs[2][1][iz],
                      tab + ((size_t)opt * n_rot + jr) * 9);
      }
    }
    float* d_tab = g->lat_cand.as<float>() + (size_t)(l % 2) * slot;
    CU(cudaMemcpyAsync(d_tab, tab, (size_t)n_opt * n_rot * 36, cudaMemcpyHostToDevice, g->stream),
       "copy rotation table");
    LatticeLevel L{};
    for (int a = 0; a < 6; ++a) {
      L.m[a] = m[a];
      for (int32_t i = 0; i < m[a]; ++i) {
        L.off[a][i] = lattice_step(r[(size_t)l][a], m[a], i);
        L.off_prev[a][i] = l > 0 ? lattice_step(r[(size_t)l - 1][a], m[a], i) : 0.0;
      }
    }
    for (int a = 0; a < 3; ++a) L.origin[a] = g->origin[a];
    L.n_rot = n_rot;
    L.P = (int32_t)P;
    L.c_prev = d_c + 6 * (size_t)l;
    L.am_prev = l > 0 ? g->argmax.as<int64_t>() : nullptr;
    L.cand = d_tab;
    L.c_out = d_c + 6 * ((size_t)l + 1);
    L.poses = g->poses.as<float>();
    L.pose_src = g->pose_src.as<int32_t>();
    L.rots = g->rots.as<float>();
    L.err = g->err.as<uint32_t>();
    CU(launch_lattice_level(L, g->stream), "launch lattice level");
    g->stats[4] += 1;
    EvalOut o{};
    o.mi = g->mi.as<float>();
    o.argmax = g->argmax.as<int64_t>();
    align_status st = enqueue_eval_core(g, n_tiles, g->poses.as<float>(), P, false, n_rot, o,
                                        pairs ? g->lat_units.as<int32_t>() : nullptr, n_units,
                                        !pairs && cluster);
    if (st != ALIGN_OK) return st;
    CU(cudaMemcpyAsync(&rec[l].am, g->argmax.p, 8, cudaMemcpyDeviceToHost, g->stream), "read argmax");
    CU(cudaMemcpyAsync(&rec[l].best, g->best.p, 8, cudaMemcpyDeviceToHost, g->stream), "read best");
    CU(cudaMemcpyAsync(&rec[l].max_passes, g->max_passes.p, 4, cudaMemcpyDeviceToHost, g->stream),
       "read counters");
    CU(cudaMemsetAsync(g->max_passes.p, 0, 4, g->stream), "reset counters");
    CU(cudaEventRecord(g->lat_ev[(size_t)l], g->stream), "record event");
  }
  align_status st = collect_status(g);  // synchronises the stream
  if (st != ALIGN_OK) return st;
  g->lat_pending = false;
  for (int32_t l = std::max(0, levels - 2); l < levels; ++l) {
    if (rec[l].am < 0 || rec[l].am >= P) return fail(ALIGN_E_INTERNAL, "argmax out of range");
    lattice_sample(c[(size_t)l].data(), r[(size_t)l].data(), m, rec[l].am, c[(size_t)l + 1].data());
  }
  for (int32_t l = 0; l < levels; ++l) {
    passes_used = std::max(passes_used, rec[l].max_passes);
    if (level_best) level_best[l] = rec[l].am;
  }
  g->stats[0] = passes_used;
  std::memcpy(T_out, c[(size_t)levels].data(), 6 * sizeof(double));
  if (mi_out) {  // the MI of the last level's argmax, from its packed running maximum
    const uint32_t ord = (uint32_t)(rec[levels - 1].best >> 32);
    const uint32_t u = (ord & 0x80000000u) ? (ord & 0x7FFFFFFFu) : ~ord;
    std::memcpy(mi_out, &u, 4);
  }
  return ALIGN_OK;
}



}  // namespace

extern "C" {

const char* align_last_error(void) { return g_last_error.c_str(); }

align_status align_create_grid(const align_grid_desc* desc, void* cuda_stream, align_grid** out) {
  if (!out) return fail(ALIGN_E_INVALID, "out is NULL");
  *out = nullptr;
  GridConst gc;
  align_status st = validate_desc(desc, &gc);
  if (st != ALIGN_OK) return st;
  int n_dev = 0;
  cudaError_t e = cudaGetDeviceCount(&n_dev);
  if (e != cudaSuccess || n_dev < 1) {
    (void)cudaGetLastError();
    return fail(ALIGN_E_CUDA, "no usable CUDA device");
  }
  int dev = 0;
  CU(cudaGetDevice(&dev), "cudaGetDevice");
  cudaDeviceProp prop;
  CU(cudaGetDeviceProperties(&prop, dev), "cudaGetDeviceProperties");
  if (prop.major < 10) return fail(ALIGN_E_CUDA, "this library is built for sm_103a (found sm_%d%d)", prop.major, prop.minor);
  for (int i = 0; i < kEvalShapes; ++i) CU(eval_shape(i).setup(), "set up eval kernels");
  align_grid* g = new (std::nothrow) align_grid();
  if (!g) return fail(ALIGN_E_OOM, "host allocation failed");
  g->gc = gc;
  for (int i = 0; i < 3; ++i) g->origin[i] = desc->origin[i];
  g->res_m = desc->res_m;
  g->V = (int64_t)gc.X * gc.Y * gc.Z;
  g->stream = (cudaStream_t)cuda_stream;
  g->device = dev;
  g->n_sm = prop.multiProcessorCount;
  g->smem_optin = prop.sharedMemPerBlockOptin;
  g->table_slots = eval_shape(0).table_slots_for(gc.K, eval_layout(gc, gc.feature != ALIGN_FEAT_COUNT), g->smem_optin, 1);
  for (int i = 0; i < 6; ++i) g->boxA[i] = i < 3 ? INT_MAX : INT_MIN;
  *out = g;
  return ALIGN_OK;
}

align_status align_destroy_grid(align_grid* g) {
  if (!g) return ALIGN_OK;
  cudaSetDevice(g->device);
  cudaStreamSynchronize(g->stream);
  for (DevBuf* b : {&g->symA, &g->sat, &g->xyz, &g->poses, &g->out_c, &g->out_box, &g->mi, &g->hist, &g->best,
                    &g->argmax, &g->err, &g->max_passes, &g->wide_count, &g->wide, &g->dump, &g->pts4,
                    &g->pose_src, &g->rots, &g->redo_list, &g->redo_count, &g->items, &g->ovf, &g->lat_c,
                    &g->lat_cand, &g->ref_pts, &g->ref_pose, &g->ref_cnt, &g->ref_s1, &g->ref_s2, &g->ref_box,
                    &g->units, &g->lat_units})
    b->release();
  for (HostBuf* b : {&g->lat_cand_h, &g->lat_rec_h, &g->lat_c_h, &g->ref_box_h}) b->release();
  for (cudaEvent_t e : g->lat_ev) cudaEventDestroy(e);
  for (auto* v : {&g->ev_pending, &g->ev_pool})
    for (auto& evs : *v)
      for (cudaEvent_t e : evs) cudaEventDestroy(e);
  delete g;
  return ALIGN_OK;
}

align_status align_grid_info(const align_grid* g, int32_t* n_symbols, int64_t* n_voxels) {
  if (!g) return fail(ALIGN_E_INVALID, "grid is NULL");
  if (n_symbols) *n_symbols = g->gc.K;
  if (n_voxels) *n_voxels = g->V;
  return ALIGN_OK;
}

align_status align_round_poses(const float origin[3], const double* eta6, int64_t P, float* poses12) {
  if (!origin) return fail(ALIGN_E_INVALID, "origin is NULL");
  if (P < 0 || (P > 0 && (!eta6 || !poses12))) return fail(ALIGN_E_INVALID, "bad pose arrays");
  poses_to_fp32(origin, eta6, P, poses12);
  return ALIGN_OK;
}

align_status align_set_reference(align_grid* g, const float* xyzA, int64_t nA, int flags) {
  align_status st = check_grid(g);
  if (st != ALIGN_OK) return st;
  if (nA < 0 || nA >= INT32_MAX) return fail(ALIGN_E_INVALID, "nA out of range");
  if (nA > 0 && !xyzA) return fail(ALIGN_E_INVALID, "xyzA is NULL");
  g->has_ref = false;
  st = ensure_status_words(g);
  if (st != ALIGN_OK) return st;
  const GridConst& gc = g->gc;
  const size_t V = (size_t)g->V;
  // working buffers, kept by the grid between calls (a free would synchronise the device)
  DevBuf &pts = g->ref_pts, &pose = g->ref_pose, &cnt = g->ref_cnt, &s1 = g->ref_s1, &s2 = g->ref_s2,
         &box = g->ref_box;
  align_status result = ALIGN_OK;
  do {
    cudaError_t e;
#define TRY(call, what)                 \
  if ((e = (call)) != cudaSuccess) {    \
    result = cuda_fail(e, (what));      \
    break;                              \
  }
    TRY(pts.ensure(std::max<size_t>(1, (size_t)nA) * 12), "allocate A points");
    if (nA > 0)
      TRY(cudaMemcpyAsync(pts.p, xyzA, (size_t)nA * 12,
                          (flags & ALIGN_XYZ_DEVICE) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, g->stream),
          "copy A points");
    if (!g->ref_pose_set) {  // the identity pose, rounded like every other pose
      float ident[12];
      const double eta0[6] = {0, 0, 0, 0, 0, 0};
      pose_to_fp32(g->origin, eta0, ident);
      TRY(pose.ensure(sizeof(ident)), "allocate pose");
      TRY(cudaMemcpyAsync(pose.p, ident, sizeof(ident), cudaMemcpyHostToDevice, g->stream), "copy pose");
      TRY(cudaStreamSynchronize(g->stream), "synchronize");
      g->ref_pose_set = true;
    }
    TRY(cnt.ensure(V * 4), "allocate A counts");
    TRY(s1.ensure(V * 8), "allocate A sums");
    TRY(s2.ensure(V * 8), "allocate A sums");
    TRY(cudaMemsetAsync(cnt.p, 0, V * 4, g->stream), "clear");
    TRY(cudaMemsetAsync(s1.p, 0, V * 8, g->stream), "clear");
    TRY(cudaMemsetAsync(s2.p, 0, V * 8, g->stream), "clear");
    TRY(launch_ref_accumulate(gc, pts.as<float>(), nA, pose.as<float>(), cnt.as<uint32_t>(),
                              s1.as<unsigned long long>(), s2.as<unsigned long long>(), g->stream),
        "launch reference accumulate");
    TRY(g->symA.ensure(V), "allocate A symbols");
    TRY(box.ensure(sizeof(int32_t) * 6), "allocate box");
    TRY(g->ref_box_h.ensure(sizeof(int32_t) * 12), "allocate pinned box");
    int32_t* box_h = g->ref_box_h.as<int32_t>();
    for (int i = 0; i < 6; ++i) box_h[i] = i < 3 ? INT_MAX : INT_MIN;
    TRY(cudaMemcpyAsync(box.p, box_h, sizeof(int32_t) * 6, cudaMemcpyHostToDevice, g->stream), "init box");
    TRY(launch_ref_symbols(gc, cnt.as<uint32_t>(), s1.as<unsigned long long>(), s2.as<unsigned long long>(),
                           g->symA.as<uint8_t>(), box.as<int32_t>(), g->stream),
        "launch reference symbols");
    const size_t sat_elems = (size_t)(gc.K - 1) * (gc.Z + 1) * (gc.Y + 1) * (gc.X + 1);
    TRY(g->sat.ensure(std::max<size_t>(1, sat_elems) * 4), "allocate prefix sums");
    TRY(cudaMemsetAsync(g->sat.p, 0, std::max<size_t>(1, sat_elems) * 4, g->stream), "clear prefix sums");
    TRY(launch_ref_sat(gc, g->symA.as<uint8_t>(), g->sat.as<int32_t>(), g->stream), "launch prefix sums");
    int32_t* hb = box_h + 6;
    TRY(cudaMemcpyAsync(hb, box.p, sizeof(int32_t) * 6, cudaMemcpyDeviceToHost, g->stream), "read box");
    TRY(cudaStreamSynchronize(g->stream), "synchronize");
    for (int i = 0; i < 6; ++i) g->boxA[i] = g->gc.boxA[i] = hb[i];
    g->stats[4] += (nA > 0 ? 1 : 0) + 1 + (gc.K > 1 ? 3 : 0);
#undef TRY
  } while (0);
  if (result != ALIGN_OK) return result;
  g->has_ref = true;
  return ALIGN_OK;
}

align_status align_get_reference(align_grid* g, uint8_t* symA, int32_t boxA[6]) {
  align_status st = check_grid(g);
  if (st != ALIGN_OK) return st;
  if (!g->has_ref) return fail(ALIGN_E_NOREF, "no reference scan set");
  if (symA) {
    CU(cudaMemcpyAsync(symA, g->symA.p, (size_t)g->V, cudaMemcpyDeviceToHost, g->stream), "read symbols");
    CU(cudaStreamSynchronize(g->stream), "synchronize");
  }
  if (boxA) std::memcpy(boxA, g->boxA, sizeof(g->boxA));
  return ALIGN_OK;
}

static align_status eval_common(align_grid* g, const float* xyzB, int64_t nB, int flags, const float* poses12,
                                const double* eta6, int64_t P, float* mi_out, int64_t* argmax_out,
                                uint32_t* hist_out, int64_t* dump_dev, bool points_ready, int32_t n_tiles_ready) {
  const bool out_dev = (flags & ALIGN_OUT_DEVICE) != 0;
  int32_t n_tiles = n_tiles_ready;
  if (!points_ready) {
    align_status st = upload_points(g, xyzB, nB, flags, &n_tiles);
    if (st != ALIGN_OK) return st;
  }
  // poses -> device fp32 (and a host copy, to find shared rotations)
  const float* d_poses = nullptr;
  const float* h_poses = nullptr;
  std::vector<float> tmp;
  if (poses12 && (flags & ALIGN_POSES_DEVICE)) {
    d_poses = poses12;
  } else {
    CU(g->poses.ensure((size_t)P * 12 * sizeof(float)), "allocate poses");
    if (poses12) {
      h_poses = poses12;
    } else {
      tmp.resize((size_t)P * 12);
      poses_to_fp32(g->origin, eta6, P, tmp.data());
      h_poses = tmp.data();
    }
    for (int64_t i = 0; i < P * 12; ++i)
      if (!std::isfinite(h_poses[i])) return fail(ALIGN_E_INVALID, "pose %lld is not finite", (long long)(i / 12));
    // a pageable source is staged before the call returns
    CU(cudaMemcpyAsync(g->poses.p, h_poses, (size_t)P * 48, cudaMemcpyHostToDevice, g->stream), "copy poses");
    d_poses = g->poses.as<float>();
  }
  const size_t KK = (size_t)g->gc.K * g->gc.K;
  EvalOut o{};
  if (out_dev) {
    o.mi = mi_out;
    o.hist = hist_out;
    if (argmax_out) {
      o.argmax = argmax_out;
    } else {
      CU(g->argmax.ensure(8), "allocate argmax");
      o.argmax = g->argmax.as<int64_t>();
    }
  } else {
    CU(g->mi.ensure((size_t)P * 4), "allocate MI");
    CU(g->argmax.ensure(8), "allocate argmax");
    o.mi = g->mi.as<float>();
    o.argmax = g->argmax.as<int64_t>();
    if (hist_out) {
      CU(g->hist.ensure((size_t)P * KK * 4), "allocate histograms");
      o.hist = g->hist.as<uint32_t>();
    }
  }
  o.dump = dump_dev;
  align_status st = enqueue_eval(g, n_tiles, d_poses, h_poses, P, o);
  if (st != ALIGN_OK) return st;
  if (out_dev) return ALIGN_OK;
  if (mi_out) CU(cudaMemcpyAsync(mi_out, o.mi, (size_t)P * 4, cudaMemcpyDeviceToHost, g->stream), "read MI");
  if (argmax_out) CU(cudaMemcpyAsync(argmax_out, o.argmax, 8, cudaMemcpyDeviceToHost, g->stream), "read argmax");
  if (hist_out)
    CU(cudaMemcpyAsync(hist_out, o.hist, (size_t)P * KK * 4, cudaMemcpyDeviceToHost, g->stream), "read histograms");
  return collect_status(g);
}

align_status align_eval_mi(align_grid* g, const float* xyzB, int64_t nB, int flags, const float* poses12,
                           const double* eta6, int64_t P, float* mi_out, int64_t* argmax_out, uint32_t* hist_out) {
  align_status st = check_grid(g);
  if (st != ALIGN_OK) return st;
  if (!g->has_ref) return fail(ALIGN_E_NOREF, "no reference scan set");
  if (P < 0 || P >= INT32_MAX) return fail(ALIGN_E_INVALID, "P out of range");
  if ((poses12 == nullptr) == (eta6 == nullptr) && P > 0)
    return fail(ALIGN_E_INVALID, "give exactly one of poses12 and eta6");
  if (eta6 && (flags & ALIGN_POSES_DEVICE)) return fail(ALIGN_E_INVALID, "eta6 must be host memory");
  if (P > 0 && !mi_out) return fail(ALIGN_E_INVALID, "mi_out is NULL");
  if (nB < 0 || nB >= INT32_MAX) return fail(ALIGN_E_INVALID, "nB out of range");
  if (P == 0) {
    if (argmax_out) {
      const int64_t none = -1;
      if (flags & ALIGN_OUT_DEVICE)
        CU(cudaMemcpyAsync(argmax_out, &none, 8, cudaMemcpyHostToDevice, g->stream), "write argmax");
      else
        *argmax_out = -1;
      if (flags & ALIGN_OUT_DEVICE) CU(cudaStreamSynchronize(g->stream), "synchronize");
    }
    return ALIGN_OK;
  }
  st = ensure_status_words(g);
  if (st != ALIGN_OK) return st;
  return eval_common(g, xyzB, nB, flags, poses12, eta6, P, mi_out, argmax_out, hist_out, nullptr, false, 0);
}

align_status align_accumulate(align_grid* g, const float* xyzB, int64_t nB, int flags, const float pose12[12],
                              int64_t* acc_out, int32_t box_out[6]) {
  align_status st = check_grid(g);
  if (st != ALIGN_OK) return st;
  if (!g->has_ref) return fail(ALIGN_E_NOREF, "no reference scan set");
  if (!pose12) return fail(ALIGN_E_INVALID, "pose12 is NULL");
  st = ensure_status_words(g);
  if (st != ALIGN_OK) return st;
  const size_t bytes = (size_t)g->V * 3 * sizeof(int64_t);
  CU(g->dump.ensure(bytes), "allocate sums");
  CU(cudaMemsetAsync(g->dump.p, 0, bytes, g->stream), "clear sums");
  float mi = 0.0f;
  int64_t am = 0;
  st = eval_common(g, xyzB, nB, flags & ~(ALIGN_OUT_DEVICE | ALIGN_POSES_DEVICE), pose12, nullptr, 1, &mi, &am,
                   nullptr, g->dump.as<int64_t>(), false, 0);
  if (st != ALIGN_OK) return st;
  if (acc_out) CU(cudaMemcpy(acc_out, g->dump.p, bytes, cudaMemcpyDeviceToHost), "read sums");
  if (box_out) CU(cudaMemcpy(box_out, g->out_box.p, 6 * sizeof(int32_t), cudaMemcpyDeviceToHost), "read box");
  return ALIGN_OK;
}

align_status align_search_ex(align_grid* g, const float* xyzB, int64_t nB, int flags, const double init[6],
                             const double range[6], const int32_t counts[6], int32_t levels, double T_out[6],
                             float* mi_out, int64_t* level_best) {
  align_status st = check_grid(g);
  if (st != ALIGN_OK) return st;
  if (!g->has_ref) return fail(ALIGN_E_NOREF, "no reference scan set");
  if (!init || !range || !counts || !T_out) return fail(ALIGN_E_INVALID, "NULL argument");
  if (levels < 0) return fail(ALIGN_E_INVALID, "levels < 0");
  int64_t P = 1;
  for (int a = 0; a < 6; ++a) {
    if (counts[a] < 1) return fail(ALIGN_E_INVALID, "counts must be >= 1");
    P *= counts[a];
    if (P >= (1 << 26)) return fail(ALIGN_E_INVALID, "lattice too large");
  }
  st = ensure_status_words(g);
  if (st != ALIGN_OK) return st;
  int32_t n_tiles = 0;
  st = upload_points(g, xyzB, nB, flags, &n_tiles);
  if (st != ALIGN_OK) return st;
  double c[6], r[6];
  std::memcpy(c, init, sizeof(c));
  std::memcpy(r, range, sizeof(r));
  const int32_t n_rot = counts[3] * counts[4] * counts[5];
  if (levels >= 1 && (int64_t)n_rot * n_rot <= kMaxLatticeCand && n_rot <= max_rotation_copies(P, n_tiles) &&
      *std::max_element(counts, counts + 6) <= std::min(kMaxAxisSamples, kLatticeMaxAxis))
    return search_pipelined(g, n_tiles, c, r, counts, P, n_rot, levels, T_out, mi_out, level_best);
  std::vector<double> eta;
  std::vector<float> poses;
  float best_mi = 0.0f;
  CU(g->mi.ensure((size_t)P * 4), "allocate MI");
  for (int32_t l = 0; l < levels; ++l) {
    build_lattice(c, r, counts, eta);
    round_lattice(g->origin, eta, counts, poses);
    int64_t am = -1;
    // MI stays on the device; only the argmax (and its MI) come back each level
    st = eval_common(g, xyzB, nB, ALIGN_OUT_DEVICE, poses.data(), nullptr, P, g->mi.as<float>(), nullptr,
                     nullptr, nullptr, true, n_tiles);
    if (st != ALIGN_OK) return st;
    CU(cudaMemcpyAsync(&am, g->argmax.p, 8, cudaMemcpyDeviceToHost, g->stream), "read argmax");
    st = collect_status(g);
    if (st != ALIGN_OK) return st;
    if (am < 0 || am >= P) return fail(ALIGN_E_INTERNAL, "argmax out of range");
    CU(cudaMemcpy(&best_mi, g->mi.as<float>() + am, 4, cudaMemcpyDeviceToHost), "read MI");
    if (level_best) level_best[l] = am;
    std::memcpy(c, &eta[(size_t)am * 6], sizeof(c));
    for (int a = 0; a < 6; ++a) r[a] = r[a] * 0.5;
  }
  std::memcpy(T_out, c, sizeof(c));
  if (mi_out) *mi_out = best_mi;
  return ALIGN_OK;
}

// ---------------------------------------------------------------------------------------
// Nelder-Mead refinement (Algorithm 1's optimiser), S simplices in lockstep: every phase of
// an iteration (reflections; expansions or contractions; shrinks) evaluates the points of
// all simplices that need one in a single batched evaluation.
// ---------------------------------------------------------------------------------------
namespace {

struct NmSimplex {
  double x[7][6];
  double f[7];   // -MI
  int32_t it = 0;
  bool done = false;
  double xbar[6], xr[6], x2[6];
  double fr = 0.0;
  int stage = 0;  // 0 accept reflection, 1 expansion, 2 outside contraction, 3 inside contraction
  bool shrink = false;
};

// Order the vertices by f; equal values keep their order.
void nm_sort(NmSimplex& s) {
  for (int i = 1; i < 7; ++i) {
    double xi[6];
    std::memcpy(xi, s.x[i], sizeof(xi));
    const double fi = s.f[i];
    int j = i - 1;
    while (j >= 0 && s.f[j] > fi) {
      s.f[j + 1] = s.f[j];
      std::memcpy(s.x[j + 1], s.x[j], sizeof(xi));
      --j;
    }
    s.f[j + 1] = fi;
    std::memcpy(s.x[j + 1], xi, sizeof(xi));
  }
}

// -MI of a list of points (FP64 eta) through one batched evaluation.
align_status nm_eval(align_grid* g, int32_t n_tiles, const std::vector<const double*>& pts, std::vector<double>& f) {
  const int64_t P = (int64_t)pts.size();
  f.assign((size_t)P, 0.0);
  if (P == 0) return ALIGN_OK;
  std::vector<float> poses((size_t)P * 12), mi((size_t)P);
  for (int64_t p = 0; p < P; ++p) pose_to_fp32(g->origin, pts[(size_t)p], &poses[(size_t)p * 12]);
  int64_t am = 0;
  align_status st = eval_common(g, nullptr, g->n_points, 0, poses.data(), nullptr, P, mi.data(), &am, nullptr,
                                nullptr, true, n_tiles);
  if (st != ALIGN_OK) return st;
  for (int64_t p = 0; p < P; ++p) f[(size_t)p] = -(double)mi[(size_t)p];
  return ALIGN_OK;
}

}  // namespace

align_status align_refine_nm(align_grid* g, const float* xyzB, int64_t nB, int flags, const double* starts,
                             int32_t S, const double step[6], int32_t max_iter, double ftol, double* T_out,
                             float* mi_out, int32_t* iters_out) {
  align_status st = check_grid(g);
  if (st != ALIGN_OK) return st;
  if (!g->has_ref) return fail(ALIGN_E_NOREF, "no reference scan set");
  if (S < 0 || (S > 0 && (!starts || !T_out))) return fail(ALIGN_E_INVALID, "bad simplex arrays");
  if (!step || max_iter < 0) return fail(ALIGN_E_INVALID, "bad step or max_iter");
  for (int32_t i = 0; i < S * 6; ++i)
    if (!std::isfinite(starts[i])) return fail(ALIGN_E_INVALID, "start %d is not finite", i / 6);
  for (int a = 0; a < 6; ++a)
    if (!std::isfinite(step[a])) return fail(ALIGN_E_INVALID, "step not finite");
  if (S == 0) return ALIGN_OK;
  st = ensure_status_words(g);
  if (st != ALIGN_OK) return st;
  int32_t n_tiles = 0;
  st = upload_points(g, xyzB, nB, flags, &n_tiles);
  if (st != ALIGN_OK) return st;
  const double rho = 1.0, chi = 2.0, psi = 0.5, sigma = 0.5;
  std::vector<NmSimplex> sx((size_t)S);
  std::vector<const double*> pts;
  std::vector<double> f;
  // initial simplices: x0 and x0 + step[i] e_i
  for (int32_t k = 0; k < S; ++k)
    for (int i = 0; i < 7; ++i) {
      std::memcpy(sx[(size_t)k].x[i], starts + 6 * k, 6 * sizeof(double));
      if (i > 0) sx[(size_t)k].x[i][i - 1] = starts[6 * k + i - 1] + step[i - 1];
      pts.push_back(sx[(size_t)k].x[i]);
    }
  st = nm_eval(g, n_tiles, pts, f);
  if (st != ALIGN_OK) return st;
  for (int32_t k = 0; k < S; ++k) {
    for (int i = 0; i < 7; ++i) sx[(size_t)k].f[i] = f[(size_t)(7 * k + i)];
    nm_sort(sx[(size_t)k]);
    sx[(size_t)k].done = max_iter == 0;
  }
  for (;;) {
    // convergence test, centroid and reflection of every active simplex
    pts.clear();
    std::vector<NmSimplex*> act;
    for (NmSimplex& s : sx) {
      if (s.done) continue;
      if (ftol > 0.0) {
        double spread = 0.0;
        for (int i = 1; i < 7; ++i) spread = std::max(spread, std::fabs(s.f[i] - s.f[0]));
        if (spread <= ftol) {
          s.done = true;
          continue;
        }
      }
      for (int j = 0; j < 6; ++j) {
        double acc = 0.0;
        for (int i = 0; i < 6; ++i) acc += s.x[i][j];
        s.xbar[j] = acc / 6.0;
        s.xr[j] = (1.0 + rho) * s.xbar[j] - rho * s.x[6][j];
      }
      act.push_back(&s);
      pts.push_back(s.xr);
    }
    if (act.empty()) break;
    st = nm_eval(g, n_tiles, pts, f);
    if (st != ALIGN_OK) return st;
    // second point: expansion or contraction
    pts.clear();
    std::vector<NmSimplex*> second;
    for (size_t q = 0; q < act.size(); ++q) {
      NmSimplex& s = *act[q];
      s.fr = f[q];
      s.shrink = false;
      if (s.fr < s.f[0]) {
        s.stage = 1;
        for (int j = 0; j < 6; ++j) s.x2[j] = (1.0 + rho * chi) * s.xbar[j] - rho * chi * s.x[6][j];
      } else if (s.fr < s.f[5]) {
        s.stage = 0;
      } else if (s.fr < s.f[6]) {
        s.stage = 2;
        for (int j = 0; j < 6; ++j) s.x2[j] = (1.0 + psi * rho) * s.xbar[j] - psi * rho * s.x[6][j];
      } else {
        s.stage = 3;
        for (int j = 0; j < 6; ++j) s.x2[j] = (1.0 - psi) * s.xbar[j] + psi * s.x[6][j];
      }
      if (s.stage != 0) {
        second.push_back(&s);
        pts.push_back(s.x2);
      } else {
        std::memcpy(s.x[6], s.xr, sizeof(s.xr));
        s.f[6] = s.fr;
      }
    }
    st = nm_eval(g, n_tiles, pts, f);
    if (st != ALIGN_OK) return st;
    pts.clear();
    std::vector<NmSimplex*> shrinking;
    for (size_t q = 0; q < second.size(); ++q) {
      NmSimplex& s = *second[q];
      const double f2 = f[q];
      if (s.stage == 1) {
        if (f2 < s.fr) {
          std::memcpy(s.x[6], s.x2, sizeof(s.x2));
          s.f[6] = f2;
        } else {
          std::memcpy(s.x[6], s.xr, sizeof(s.xr));
          s.f[6] = s.fr;
        }
      } else if ((s.stage == 2 && f2 <= s.fr) || (s.stage == 3 && f2 < s.f[6])) {
        std::memcpy(s.x[6], s.x2, sizeof(s.x2));
        s.f[6] = f2;
      } else {
        s.shrink = true;
        for (int i = 1; i < 7; ++i) {
          for (int j = 0; j < 6; ++j) s.x[i][j] = s.x[0][j] + sigma * (s.x[i][j] - s.x[0][j]);
          pts.push_back(s.x[i]);
        }
        shrinking.push_back(&s);
      }
    }
    st = nm_eval(g, n_tiles, pts, f);
    if (st != ALIGN_OK) return st;
    for (size_t q = 0; q < shrinking.size(); ++q)
      for (int i = 1; i < 7; ++i) shrinking[q]->f[i] = f[q * 6 + (size_t)(i - 1)];
    for (NmSimplex* s : act) {
      nm_sort(*s);
      if (++s->it >= max_iter) s->done = true;
    }
  }
  for (int32_t k = 0; k < S; ++k) {
    std::memcpy(T_out + 6 * k, sx[(size_t)k].x[0], 6 * sizeof(double));
    if (mi_out) mi_out[k] = (float)(-sx[(size_t)k].f[0]);
    if (iters_out) iters_out[k] = sx[(size_t)k].it;
  }
  return ALIGN_OK;
}

align_status align_search(align_grid* g, const float* xyzB, int64_t nB, int flags, const double init[6],
                          const double range[6], int32_t levels, double T_out[6], float* mi_out) {
  const int32_t counts[6] = {8, 8, 2, 2, 2, 8};
  return align_search_ex(g, xyzB, nB, flags, init, range, counts, levels, T_out, mi_out, nullptr);
}

align_status align_eval_stats(align_grid* g, int64_t out[6]) {
  if (!g || !out) return fail(ALIGN_E_INVALID, "NULL argument");
  for (int i = 0; i < 6; ++i) out[i] = g->stats[i];
  // batched launches feed back through the seed of the way the last launch swept its poses
  const int32_t seed = g->last_pairs ? g->passes_seed_pair[0] : g->last_cluster ? g->passes_seed_cluster
                                                                                 : g->passes_seed[0];
  out[0] = std::max<int64_t>(out[0], seed);
  return ALIGN_OK;
}

align_status align_set_sweep(align_grid* g, int32_t kind) {
  if (!g) return fail(ALIGN_E_INVALID, "NULL grid");
  if (kind < -1 || kind > 2) return fail(ALIGN_E_INVALID, "sweep kind must be -1, 0, 1 or 2");
  g->sweep_mode = kind;
  return ALIGN_OK;
}

align_status align_set_spill(align_grid* g, int32_t on, int64_t queue_runs) {
  if (!g) return fail(ALIGN_E_INVALID, "NULL grid");
  if (on != 0 && on != 1) return fail(ALIGN_E_INVALID, "spill must be 0 or 1");
  if (queue_runs < 0 || queue_runs > (int64_t)1 << 31) return fail(ALIGN_E_INVALID, "queue_runs out of range");
  g->spill_on = on;
  g->spill_runs = queue_runs;
  return ALIGN_OK;
}

align_status align_eval_redo_poses(align_grid* g, int64_t* out, int64_t cap, int64_t* n_out) {
  align_status st = check_grid(g);
  if (st != ALIGN_OK) return st;
  if (!n_out || cap < 0 || (cap > 0 && !out)) return fail(ALIGN_E_INVALID, "bad output arguments");
  *n_out = 0;
  if (g->redo_count.p == nullptr || g->redo_list.p == nullptr) return ALIGN_OK;  // nothing evaluated yet
  uint32_t n = 0;
  CU(cudaMemcpyAsync(&n, g->redo_count.p, 4, cudaMemcpyDeviceToHost, g->stream), "read redo count");
  CU(cudaStreamSynchronize(g->stream), "synchronize");
  *n_out = n;
  const int64_t k = std::min<int64_t>(cap, n);
  if (k > 0) {
    std::vector<uint32_t> idx((size_t)k);
    CU(cudaMemcpy(idx.data(), g->redo_list.p, (size_t)k * 4, cudaMemcpyDeviceToHost), "read redo list");
    std::sort(idx.begin(), idx.end());
    for (int64_t i = 0; i < k; ++i) out[i] = idx[(size_t)i];
  }
  return ALIGN_OK;
}

align_status align_profile(align_grid* g, int32_t mode, double out[3]) {
  align_status st = check_grid(g);
  if (st != ALIGN_OK) return st;
  if (mode != 0 && mode != 1 && mode != 2) return fail(ALIGN_E_INVALID, "mode must be 0, 1 or 2");
  st = drain_events(g);  // waits for the recorded launches
  if (st != ALIGN_OK) return st;
  if (mode == 1) {
    g->profiling = true;
    g->prof[0] = g->prof[1] = g->prof[2] = 0.0;
  } else if (mode == 0) {
    g->profiling = false;
  }
  if (out)
    for (int i = 0; i < 3; ++i) out[i] = g->prof[i];
  return ALIGN_OK;
}

}  // extern "C"

// Helpers for other translation units of the library (validation, messages, pose rounding).
namespace mialign {
const EvalKernels& eval_shape_1024x1();
const EvalKernels& eval_shape_1024x2();
const EvalKernels& eval_shape_512x1();
const EvalKernels& eval_shape(int i) {
  switch (i) {
    case 1:
      return eval_shape_1024x2();
    case 2:
      return eval_shape_512x1();
    default:
      return eval_shape_1024x1();
  }
}
align_status report_errorf(align_status st, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  return fail(st, "%s", buf);
}
int group_pose_rotations(const float* poses12, int64_t P, std::vector<float>& rots, std::vector<int32_t>& idx,
                         int max_groups) {
  return group_rotations(poses12, P, rots, idx, max_groups);
}
align_status check_grid_device(align_grid* g) { return check_grid(g); }
int pair_units(const float* poses12, const int32_t* src, int64_t P, std::vector<int32_t>& units) {
  return pair_units_impl(poses12, src, P, units);
}
void lattice_poses(const float origin[3], const double c[6], const double r[6], const int32_t m[6],
                   std::vector<double>& eta, std::vector<float>& poses) {
  build_lattice(c, r, m, eta);
  round_lattice(origin, eta, m, poses);
}
align_status check_grid_desc(const align_grid_desc* desc, GridConst* gc) { return validate_desc(desc, gc); }
align_status report_error(align_status st, const char* msg) { return fail(st, "%s", msg); }
align_status report_cuda_error(cudaError_t e, const char* what) { return cuda_fail(e, what); }
void round_pose_host(const float origin[3], const double* eta6, float* pose12) { pose_to_fp32(origin, eta6, pose12); }
void round_poses_host(const float origin[3], const double* eta6, int64_t P, float* poses12) {
  poses_to_fp32(origin, eta6, P, poses12);
}
}  // namespace mialign
