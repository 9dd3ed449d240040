// lattice.cu — one level of the coarse-to-fine lattice search built on the device, so that
// the levels of a search follow each other on the stream without a host round trip.
//
// A level's centre is the pose the previous level chose (its argmax, read here from device
// memory); its samples are centre + offset per axis, offset_i = range*(2i - (m-1))/(m-1)
// (one sample: the centre); pose index order rx, ry, rz, tx, ty, tz with tz fastest.  The
// offsets come from the host (its own FP64 values), and the sums and the rounding
// t' = fp32(eta_t - origin) are the same IEEE operations, in the same order, as the host's
// lattice construction and pose rounding; the rotations, which need cos/sin, arrive from the
// host as a table of FP32 matrices, one per (rotation sample of the previous level, rotation
// sample of this level).
#include <algorithm>

#include "align_internal.h"

namespace mialign {

namespace {

// Lattice index -> sample index of each pose component (i[0..5] for tx, ty, tz, rx, ry, rz;
// index order rx, ry, rz, tx, ty, tz with tz fastest).
__device__ __forceinline__ void lattice_indices(int64_t idx, const int32_t m[6], int32_t i[6]) {
  int64_t rem = idx;
  i[2] = (int32_t)(rem % m[2]); rem /= m[2];
  i[1] = (int32_t)(rem % m[1]); rem /= m[1];
  i[0] = (int32_t)(rem % m[0]); rem /= m[0];
  i[5] = (int32_t)(rem % m[5]); rem /= m[5];
  i[4] = (int32_t)(rem % m[4]); rem /= m[4];
  i[3] = (int32_t)rem;
}

__global__ void lattice_level_kernel(const __grid_constant__ LatticeLevel L) {
  const int32_t n_trans = L.m[0] * L.m[1] * L.m[2];
  double c[6];
  int32_t opt = 0;
  if (L.am_prev != nullptr) {
    int64_t am = *L.am_prev;
    if (am < 0 || am >= L.P) {  // never produced by the argmax; reported by the host
      if (blockIdx.x == 0 && threadIdx.x == 0) atomicOr(L.err, kErrLattice);
      am = 0;
    }
    int32_t i[6];
    lattice_indices(am, L.m, i);
    for (int a = 0; a < 6; ++a) c[a] = __dadd_rn(L.c_prev[a], L.off_prev[a][i[a]]);
    opt = (int32_t)(am / n_trans);
  } else {
    for (int a = 0; a < 6; ++a) c[a] = L.c_prev[a];
  }
  if (blockIdx.x == 0 && threadIdx.x < 6) L.c_out[threadIdx.x] = c[threadIdx.x];
  const float* cand = L.cand + (size_t)opt * L.n_rot * 9;
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < L.P; p += (int64_t)gridDim.x * blockDim.x) {
    int32_t j[6];
    lattice_indices(p, L.m, j);
    const int32_t jr = (int32_t)(p / n_trans);
    float* out = L.poses + 12 * p;
    for (int k = 0; k < 9; ++k) out[k] = cand[9 * jr + k];
    for (int a = 0; a < 3; ++a) {
      const double e = __dadd_rn(c[a], L.off[a][j[a]]);
      out[9 + a] = __double2float_rn(__dsub_rn(e, (double)L.origin[a]));
    }
    L.pose_src[p] = jr;
    if (p % n_trans == 0)
      for (int k = 0; k < 9; ++k) L.rots[9 * jr + k] = cand[9 * jr + k];
  }
}

}  // namespace

cudaError_t launch_lattice_level(const LatticeLevel& L, cudaStream_t s) {
  const int threads = 256;
  const int64_t blocks = std::max<int64_t>(1, std::min<int64_t>((L.P + threads - 1) / threads, 1024));
  lattice_level_kernel<<<(unsigned)blocks, threads, 0, s>>>(L);
  return cudaGetLastError();
}

}  // namespace mialign
