// peaks.cu — micro-benchmarks of the throughputs that bound the MI evaluation on this GPU:
// 32-bit lane-operation issue (FP32 and INT32 arithmetic, and the voxel map's own mix),
// shared-memory 32-bit atomics (the per-CTA hash table and histograms) and L2 atomics (the
// alternative of per-pose accumulators in global memory).  They give the measured
// denominators of the roofline that the benchmark reports; none of them is on the hot path.
//
// Every kernel runs a fixed amount of independent work per thread with all SMs busy; the
// rate is operations (lane operations or atomics) over the fastest of `reps` launches timed
// with CUDA events on the caller's stream.
#include <algorithm>
#include <cfloat>
#include <vector>

#include "align_internal.h"

namespace mialign {
namespace {

constexpr int kThreads = 1024;

// FP32: 8 independent FFMA chains per thread (one lane operation each).
__global__ void __launch_bounds__(kThreads) mb_ffma(float* out, int iters, float a, float b) {
  float x[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) x[i] = (float)(threadIdx.x + i);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int i = 0; i < 8; ++i) x[i] = fmaf(x[i], a, b);
  }
  float s = 0.0f;
#pragma unroll
  for (int i = 0; i < 8; ++i) s += x[i];
  if (s == 1.2345f) out[blockIdx.x] = s;  // keeps the chains alive
}

// INT32: 8 independent chains of add and xor (one lane operation each).
__global__ void __launch_bounds__(kThreads) mb_iadd(uint32_t* out, int iters, uint32_t a, uint32_t b) {
  uint32_t x[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) x[i] = threadIdx.x * (i + 3);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      asm("add.u32 %0, %0, %1;" : "+r"(x[i]) : "r"(a));
      asm("xor.b32 %0, %0, %1;" : "+r"(x[i]) : "r"(b));
    }
  }
  uint32_t s = 0;
#pragma unroll
  for (int i = 0; i < 8; ++i) s ^= x[i];
  if (s == 0x9E3779B9u) out[blockIdx.x] = s;
}

// The voxel map's own mix per point (translation add, scale multiply, floor conversion,
// range compare, key multiply-add, mm rounding): 4 independent points per thread, 16 lane
// operations each: 3 FADD, 4 FMUL, 4 F2I, 3 ISETP/SELP, 2 IMAD.
__global__ void __launch_bounds__(kThreads) mb_keymix(uint32_t* out, int iters, float t, float inv) {
  float gx[4], gy[4], gz[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    gx[i] = (float)((threadIdx.x * 7 + i) & 255) * 0.37f;
    gy[i] = (float)((threadIdx.x * 5 + i) & 255) * 0.29f;
    gz[i] = (float)((threadIdx.x * 3 + i) & 15) * 0.31f;
  }
  uint32_t acc = 0;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      gx[i] = __fadd_rn(gx[i], t);
      gy[i] = __fadd_rn(gy[i], t);
      gz[i] = __fadd_rn(gz[i], t);
      const uint32_t kx = (uint32_t)__float2int_rd(__fmul_rn(gx[i], inv));
      const uint32_t ky = (uint32_t)__float2int_rd(__fmul_rn(gy[i], inv));
      const uint32_t kz = (uint32_t)__float2int_rd(__fmul_rn(gz[i], inv));
      const uint32_t zq = (uint32_t)__float2int_rn(__fmul_rn(gz[i], 1000.0f));
      const bool in = (kx < 160u) & (ky < 160u) & (kz < 16u);
      const uint32_t key = (kz * 160u + ky) * 160u + kx;
      acc += in ? key : zq;
    }
  }
  if (acc == 0x12345u) out[blockIdx.x] = acc;
}

// Shared-memory atomics: every lane hits its own bank (pattern 0) or a pseudo-random word of
// a 32 KiB region (pattern 1, like hash-table slots); `ret` selects atom (returns the old
// value) instead of red.  8 independent atomics per iteration.
template <bool kRet, int kPattern>
__global__ void __launch_bounds__(kThreads) mb_smem_atomic(uint32_t* out, int iters) {
  __shared__ uint32_t buf[8192];
  for (int i = threadIdx.x; i < 8192; i += kThreads) buf[i] = 0u;
  __syncthreads();
  const uint32_t base = (uint32_t)__cvta_generic_to_shared(buf);
  uint32_t h = threadIdx.x * 0x9E3779B1u + blockIdx.x;
  uint32_t acc = 0;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      uint32_t w;
      if (kPattern == 0) {
        w = (uint32_t)((threadIdx.x & 31) + 32 * ((threadIdx.x >> 5) + 32 * i)) & 8191u;
      } else {
        h = h * 1664525u + 1013904223u;
        w = h >> 19;  // 13 bits: 0 .. 8191
      }
      if (kRet) {
        uint32_t old;
        asm volatile("atom.shared.add.u32 %0, [%1], 1;" : "=r"(old) : "r"(base + 4u * w) : "memory");
        acc += old;
      } else {
        asm volatile("red.shared.add.u32 [%0], 1;" ::"r"(base + 4u * w) : "memory");
      }
    }
  }
  __syncthreads();
  if (acc == 0x7FFFFFFFu || (threadIdx.x == 0 && buf[0] == 0xFFFFFFFFu)) out[blockIdx.x] = acc;
}

// L2 atomics on a buffer of `words` 32-bit words (sized to stay L2-resident): pseudo-random
// words, 8 independent atomics per iteration.
template <bool kRet>
__global__ void __launch_bounds__(kThreads) mb_l2_atomic(uint32_t* buf, uint32_t words_mask, int iters,
                                                         uint32_t* out) {
  uint32_t h = (blockIdx.x * kThreads + threadIdx.x) * 0x9E3779B1u;
  uint32_t acc = 0;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      h = h * 1664525u + 1013904223u;
      uint32_t* p = buf + ((h >> 7) & words_mask);
      if (kRet) acc += atomicAdd(p, 1u);
      else atomicAdd(p, 1u);  // result unused: compiled to a reduction
    }
  }
  if (acc == 0x7FFFFFFFu) out[blockIdx.x] = acc;
}

}  // namespace
}  // namespace mialign

using namespace mialign;

extern "C" align_status align_microbench(int32_t kind, void* dev_buf, int64_t buf_bytes, int32_t reps,
                                         void* cuda_stream, double out[3]) {
  if (!out || reps < 1 || reps > 1000) return report_error(ALIGN_E_INVALID, "align_microbench: bad arguments");
  if (kind < 0 || kind > 7) return report_error(ALIGN_E_INVALID, "align_microbench: kind must be 0..7");
  if (!dev_buf || buf_bytes < (int64_t)(1 << 20))
    return report_error(ALIGN_E_INVALID, "align_microbench: needs a device buffer of at least 1 MiB");
  int dev = 0, n_sm = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return report_cuda_error(e, "device query");
  cudaStream_t s = (cudaStream_t)cuda_stream;
  uint32_t* sink = static_cast<uint32_t*>(dev_buf);
  // words of the L2 target: a power of two within the buffer and at most 16 MiB (L2-resident)
  uint64_t words = 1;
  while (words * 2 * 4 <= (uint64_t)std::min<int64_t>(buf_bytes - 65536, 16 << 20)) words *= 2;
  uint32_t* l2buf = sink + 16384;
  const int blocks = 2 * n_sm;  // two 1,024-thread CTAs per SM: every warp slot busy
  const double threads = (double)blocks * kThreads;
  int iters = 0;
  double ops_per_iter = 0.0;  // per thread
  switch (kind) {
    case 0: iters = 16384; ops_per_iter = 8; break;   // FFMA lane operations
    case 1: iters = 8192; ops_per_iter = 16; break;   // IADD + XOR lane operations
    case 2: iters = 2048; ops_per_iter = 64; break;   // voxel-map mix lane operations
    case 3: case 4: case 5: case 6: iters = 1024; ops_per_iter = 8; break;  // shared atomics
    default: iters = 64; ops_per_iter = 8; break;     // L2 atomics
  }
  auto launch = [&]() {
    switch (kind) {
      case 0: mb_ffma<<<blocks, kThreads, 0, s>>>(reinterpret_cast<float*>(sink), iters, 0.999f, 1e-3f); break;
      case 1: mb_iadd<<<blocks, kThreads, 0, s>>>(sink, iters, 0x9E3779B9u, 0x7F4A7C15u); break;
      case 2: mb_keymix<<<blocks, kThreads, 0, s>>>(sink, iters, 1e-4f, 2.0f); break;
      case 3: mb_smem_atomic<false, 0><<<blocks, kThreads, 0, s>>>(sink, iters); break;
      case 4: mb_smem_atomic<true, 0><<<blocks, kThreads, 0, s>>>(sink, iters); break;
      case 5: mb_smem_atomic<false, 1><<<blocks, kThreads, 0, s>>>(sink, iters); break;
      case 6: mb_smem_atomic<true, 1><<<blocks, kThreads, 0, s>>>(sink, iters); break;
      default: mb_l2_atomic<false><<<blocks, kThreads, 0, s>>>(l2buf, (uint32_t)(words - 1), iters, sink); break;
    }
  };
  cudaEvent_t e0, e1;
  if ((e = cudaEventCreate(&e0)) != cudaSuccess) return report_cuda_error(e, "cudaEventCreate");
  if ((e = cudaEventCreate(&e1)) != cudaSuccess) {
    cudaEventDestroy(e0);
    return report_cuda_error(e, "cudaEventCreate");
  }
  float best = FLT_MAX;
  launch();  // warm-up
  e = cudaGetLastError();
  for (int r = 0; r < reps && e == cudaSuccess; ++r) {
    cudaEventRecord(e0, s);
    launch();
    cudaEventRecord(e1, s);
    e = cudaEventSynchronize(e1);
    float ms = 0.0f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e == cudaSuccess) best = std::min(best, ms);
  }
  if (e == cudaSuccess) e = cudaGetLastError();
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (e != cudaSuccess) return report_cuda_error(e, "micro-benchmark");
  const double ops = threads * iters * ops_per_iter;
  out[0] = ops / (best * 1e-3);
  out[1] = best;
  out[2] = ops;
  return ALIGN_OK;
}
