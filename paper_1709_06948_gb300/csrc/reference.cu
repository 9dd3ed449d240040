// reference.cu — Algorithm 1 initialisation for scan A (cold path, once per reference):
// voxelize A with the identity pose, its feature symbol per voxel, its occupied bbox,
// and per-symbol 3-D prefix sums used to count A's symbols over any overlap box.
#include <climits>

#include "align_internal.h"
#include "device_common.cuh"

namespace mialign {

namespace {

__global__ void ref_accumulate_kernel(const GridConst gc, const float* __restrict__ xyz, int64_t n,
                                      const float* __restrict__ pose12, uint32_t* cnt, unsigned long long* s1,
                                      unsigned long long* s2) {
  Pose12 P;
#pragma unroll
  for (int i = 0; i < 9; ++i) P.r[i] = pose12[i];
#pragma unroll
  for (int i = 0; i < 3; ++i) P.t[i] = pose12[9 + i];
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    int dz = 0;
    const uint32_t key =
        voxel_key(P, xyz[3 * i], xyz[3 * i + 1], xyz[3 * i + 2], gc.inv_res, gc.X, gc.Y, gc.Z, gc.res_mm, &dz);
    if (key == kEmptyKey) continue;
    atomicAdd(&cnt[key], 1u);
    atomicAdd(&s1[key], (unsigned long long)(long long)dz);
    atomicAdd(&s2[key], (unsigned long long)((long long)dz * dz));
  }
}

__global__ void ref_symbols_kernel(const GridConst gc, const uint32_t* __restrict__ cnt,
                                   const unsigned long long* __restrict__ s1, const unsigned long long* __restrict__ s2,
                                   uint8_t* symA, int32_t* box) {
  __shared__ uint32_t ct[kMaxLevels];
  __shared__ int64_t vt[kMaxLevels];
  for (int i = threadIdx.x; i < kMaxLevels; i += blockDim.x) {
    ct[i] = gc.count_thresh[i];
    vt[i] = gc.var_thresh[i];
  }
  __syncthreads();
  const int64_t V = (int64_t)gc.X * gc.Y * gc.Z;
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < V; v += (int64_t)gridDim.x * blockDim.x) {
    const uint64_t n = cnt[v];
    const int sym = feature_symbol(gc.feature, gc.Lc, gc.Lv, ct, vt, n, (int64_t)s1[v], s2[v]);
    symA[v] = (uint8_t)sym;
    if (n > 0) {
      const int kx = (int)(v % gc.X), ky = (int)((v / gc.X) % gc.Y), kz = (int)(v / ((int64_t)gc.X * gc.Y));
      atomicMin(&box[0], kx);
      atomicMin(&box[1], ky);
      atomicMin(&box[2], kz);
      atomicMax(&box[3], kx);
      atomicMax(&box[4], ky);
      atomicMax(&box[5], kz);
    }
  }
}

// sat[a-1][z][y][x] = #{ voxels (x', y', z') with x' < x, y' < y, z' < z and symA == a }.
// Pass 0: running sums along x per (a, z, y) row (a warp per row: inclusive warp scans over
// 32-voxel chunks, coalesced); pass 1 along y and pass 2 along z (a thread per column, rows
// read kChunk at a time so that the loads of a chunk are in flight together).
constexpr int kChunk = 8;

__global__ void ref_sat_x_kernel(const GridConst gc, const uint8_t* __restrict__ symA, int32_t* __restrict__ sat) {
  const int X = gc.X, Y = gc.Y, Z = gc.Z, X1 = X + 1, Y1 = Y + 1, Z1 = Z + 1;
  const int64_t rows = (int64_t)(gc.K - 1) * Z * Y;
  const int lane = threadIdx.x & 31;
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t r = blockIdx.x * (int64_t)(blockDim.x >> 5) + (threadIdx.x >> 5); r < rows; r += warps) {
    const int y = (int)(r % Y);
    const int z = (int)((r / Y) % Z);
    const int a = (int)(r / ((int64_t)Y * Z)) + 1;
    int32_t* out = sat + (((size_t)(a - 1) * Z1 + (z + 1)) * Y1 + (y + 1)) * X1;
    const uint8_t* in = symA + ((size_t)z * Y + y) * X;
    if (lane == 0) out[0] = 0;
    int32_t carry = 0;
    for (int x0 = 0; x0 < X; x0 += 32) {
      const int x = x0 + lane;
      int32_t v = (x < X && in[x] == a) ? 1 : 0;
#pragma unroll
      for (int d = 1; d < 32; d <<= 1) {
        const int32_t u = __shfl_up_sync(0xFFFFFFFFu, v, d);
        if (lane >= d) v += u;
      }
      if (x < X) out[x + 1] = carry + v;
      carry += __shfl_sync(0xFFFFFFFFu, v, 31);
    }
  }
}

// Running sums down a column of n entries `stride` apart (entry 0 stays as it is).
__device__ __forceinline__ void column_scan(int32_t* __restrict__ base, int n, size_t stride) {
  int32_t acc = 0;
  for (int i0 = 1; i0 < n; i0 += kChunk) {
    int32_t v[kChunk];
#pragma unroll
    for (int k = 0; k < kChunk; ++k) v[k] = (i0 + k < n) ? base[(size_t)(i0 + k) * stride] : 0;
#pragma unroll
    for (int k = 0; k < kChunk; ++k) {
      acc += v[k];
      if (i0 + k < n) base[(size_t)(i0 + k) * stride] = acc;
    }
  }
}

__global__ void ref_sat_y_kernel(const GridConst gc, int32_t* sat) {
  const int X1 = gc.X + 1, Y1 = gc.Y + 1, Z1 = gc.Z + 1;
  const int64_t cols = (int64_t)(gc.K - 1) * gc.Z * X1;
  for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < cols; c += (int64_t)gridDim.x * blockDim.x) {
    const int x = (int)(c % X1);
    const int z = (int)((c / X1) % gc.Z) + 1;
    const int a = (int)(c / ((int64_t)X1 * gc.Z));
    column_scan(sat + ((size_t)a * Z1 + z) * Y1 * X1 + x, Y1, (size_t)X1);
  }
}

__global__ void ref_sat_z_kernel(const GridConst gc, int32_t* sat) {
  const int X1 = gc.X + 1, Y1 = gc.Y + 1, Z1 = gc.Z + 1;
  const int64_t cols = (int64_t)(gc.K - 1) * Y1 * X1;
  const size_t plane = (size_t)Y1 * X1;
  for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < cols; c += (int64_t)gridDim.x * blockDim.x) {
    const int64_t xy = c % ((int64_t)Y1 * X1);
    const int a = (int)(c / ((int64_t)Y1 * X1));
    column_scan(sat + (size_t)a * Z1 * plane + xy, Z1, plane);
  }
}

int blocks_for(int64_t work, int threads) {
  int64_t b = (work + threads - 1) / threads;
  if (b < 1) b = 1;
  if (b > 65535LL * 16) b = 65535LL * 16;
  return (int)b;
}

}  // namespace

cudaError_t launch_ref_accumulate(const GridConst& gc, const float* xyz, int64_t n, const float* pose12, uint32_t* cnt,
                                  unsigned long long* s1, unsigned long long* s2, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  ref_accumulate_kernel<<<blocks_for(n, 256), 256, 0, s>>>(gc, xyz, n, pose12, cnt, s1, s2);
  return cudaGetLastError();
}

cudaError_t launch_ref_symbols(const GridConst& gc, const uint32_t* cnt, const unsigned long long* s1,
                               const unsigned long long* s2, uint8_t* symA, int32_t* box, cudaStream_t s) {
  const int64_t V = (int64_t)gc.X * gc.Y * gc.Z;
  ref_symbols_kernel<<<blocks_for(V, 256), 256, 0, s>>>(gc, cnt, s1, s2, symA, box);
  return cudaGetLastError();
}

cudaError_t launch_ref_sat(const GridConst& gc, const uint8_t* symA, int32_t* sat, cudaStream_t s) {
  if (gc.K <= 1) return cudaSuccess;
  const int64_t rows = (int64_t)(gc.K - 1) * gc.Z * gc.Y;
  ref_sat_x_kernel<<<blocks_for(rows * 32, 256), 256, 0, s>>>(gc, symA, sat);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const int64_t cy = (int64_t)(gc.K - 1) * gc.Z * (gc.X + 1);
  ref_sat_y_kernel<<<blocks_for(cy, 128), 128, 0, s>>>(gc, sat);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const int64_t cz = (int64_t)(gc.K - 1) * (gc.Y + 1) * (gc.X + 1);
  ref_sat_z_kernel<<<blocks_for(cz, 128), 128, 0, s>>>(gc, sat);
  return cudaGetLastError();
}

}  // namespace mialign
