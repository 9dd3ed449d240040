// device_common.cuh — device-side steps of the method shared by the library's kernels:
// the voxel-point map of one point under one pose and the feature symbol of one voxel.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "align_internal.h"

namespace mialign {

// ---------------------------------------------------------------------------------
// Voxel-point map (Sec. III-A; Algorithm 1 "transform scan B", "extract voxel ids").
// The FP32 operation order is fixed so that every implementation of the convention
// gets the same voxel for every point:
//   u_i = fma(r_i0, x, fma(r_i1, y, r_i2 * z)),  g_i = u_i + t'_i,
//   k_i = floor(g_i * inv_res),  inside iff 0 <= k_i < dims_i,
//   zq = round-half-even(g_z * 1000),  dz = zq - k_z * res_mm.
// Intrinsics with explicit rounding keep the compiler from contracting or reordering.
// Returns the linear key, or kEmptyKey outside the grid.
// ---------------------------------------------------------------------------------
struct Pose12 {
  float r[9];
  float t[3];
};

// u = R p with the fixed FMA order (shared by every rotation of every pose).
__device__ __forceinline__ void rotate_point(const float* r, float x, float y, float z, float& ux, float& uy,
                                             float& uz) {
  ux = __fmaf_rn(r[0], x, __fmaf_rn(r[1], y, __fmul_rn(r[2], z)));
  uy = __fmaf_rn(r[3], x, __fmaf_rn(r[4], y, __fmul_rn(r[5], z)));
  uz = __fmaf_rn(r[6], x, __fmaf_rn(r[7], y, __fmul_rn(r[8], z)));
}

// Key and dz of a transformed point g = u + t'.
__device__ __forceinline__ uint32_t voxel_key_g(float gx, float gy, float gz, float inv_res, int X, int Y, int Z,
                                                int res_mm, int* dz) {
  const float fx = __fmul_rn(gx, inv_res);
  const float fy = __fmul_rn(gy, inv_res);
  const float fz = __fmul_rn(gz, inv_res);
  // floor(f) in [0, D)  <=>  f in [0, D)  (NaN fails both compares)
  const bool in = (fx >= 0.0f) & (fx < (float)X) & (fy >= 0.0f) & (fy < (float)Y) & (fz >= 0.0f) &
                  (fz < (float)Z);
  if (!in) return kEmptyKey;
  const int kx = __float2int_rd(fx);
  const int ky = __float2int_rd(fy);
  const int kz = __float2int_rd(fz);
  const int zq = __float2int_rn(__fmul_rn(gz, 1000.0f));
  *dz = zq - kz * res_mm;
  return (uint32_t)((kz * Y + ky) * X + kx);
}

__device__ __forceinline__ uint32_t voxel_key(const Pose12& P, float x, float y, float z, float inv_res,
                                              int X, int Y, int Z, int res_mm, int* dz) {
  float ux, uy, uz;
  rotate_point(P.r, x, y, z, ux, uy, uz);
  return voxel_key_g(__fadd_rn(ux, P.t[0]), __fadd_rn(uy, P.t[1]), __fadd_rn(uz, P.t[2]), inv_res, X, Y, Z, res_mm,
                     dz);
}

// ---------------------------------------------------------------------------------
// Feature symbol of one voxel from its exact integer sums (Sec. III-A features; phi = 0).
// count level    = #{ j : n >= ct[j] }                     (ct ascending)
// variance level = #{ j : n*S2 - S1^2 >= vt[j] * n^2 }      (vt ascending; exact in 128 bits)
// Both sets are prefixes of the ascending thresholds, so a binary search finds the count.
// ---------------------------------------------------------------------------------
__device__ __forceinline__ int count_level(const uint32_t* ct, int Lc, uint64_t n) {
  int lo = 0, hi = Lc - 1;  // answer in [0, Lc-1]
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (n >= (uint64_t)ct[mid]) lo = mid + 1;
    else hi = mid;
  }
  return lo;
}

__device__ __forceinline__ int var_level(const int64_t* vt, int Lv, uint64_t n, int64_t s1, uint64_t s2) {
  const __int128 spread = (__int128)n * (__int128)s2 - (__int128)s1 * (__int128)s1;  // n^2 * var
  const __int128 n2 = (__int128)n * (__int128)n;
  int lo = 0, hi = Lv - 1;
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (spread >= (__int128)vt[mid] * n2) lo = mid + 1;
    else hi = mid;
  }
  return lo;
}

__device__ __forceinline__ int feature_symbol(int feature, int Lc, int Lv, const uint32_t* ct, const int64_t* vt,
                                              uint64_t n, int64_t s1, uint64_t s2) {
  if (n == 0) return 0;
  if (feature == 0) return 1 + count_level(ct, Lc, n);
  if (feature == 1) return 1 + var_level(vt, Lv, n, s1, s2);
  return 1 + count_level(ct, Lc, n) * Lv + var_level(vt, Lv, n, s1, s2);
}

}  // namespace mialign
