// noalloc.cu — reference-scan voxelization without any device allocation.
//
// align_set_reference allocates its working arrays (per-voxel counts and z sums) with
// cudaMalloc, and a grid keeps them between calls.  Some callers cannot allocate at all: a
// process whose device memory is handed out by another framework's allocator under a fixed
// budget, or a latency-bound loop in which an allocation (cudaMalloc may synchronise the
// device and take milliseconds) is not allowed.  align_reference_noalloc gives them the same
// A-side result (feature symbol per voxel and occupied bounding box) using a working
// area that is a fixed array in the library's own device memory.
//
// The working area: kNoallocMaxVoxels voxels x (uint32 count + two uint64 sums) = 10 MiB,
// a file-scope __device__ array.  Every GPU that loads the library holds it until the
// process exits.  All calls on a device share it and it keeps the last call's contents,
// so each call clears the part it uses first, and calls whose work overlaps on the GPU
// (different streams, or different host threads) race and must not be issued.
#include <cuda.h>  // driver types for the context lookups (entry points via the runtime)

#include <algorithm>
#include <climits>
#include <mutex>

#include "align_internal.h"
#include "device_common.cuh"

namespace mialign {

namespace {

constexpr int64_t kNoallocMaxVoxels = int64_t(1) << 19;  // covers 160 x 160 x 16

// counts (uint32) | S1 (uint64, two's complement) | S2 (uint64) | identity pose (12 floats)
constexpr size_t kCntBytes = (size_t)kNoallocMaxVoxels * 4;
constexpr size_t kSumBytes = (size_t)kNoallocMaxVoxels * 8;
constexpr size_t kScratchBytes = kCntBytes + 2 * kSumBytes + 64;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

// Device address of g_noalloc_scratch per device, looked up once (with that device
// current).  In host code the symbol itself is only a host-side stand-in.  The address
// belongs to the device's current context: a cudaDeviceReset destroys that context and the
// next one may place the array elsewhere, so the lookup is keyed by the context's unique id
// (cuCtxGetId, never reused within a process) and repeated when the id changes.
constexpr int kMaxDevices = 64;
struct ScratchSlot {
  unsigned long long ctx_id = 0;
  void* addr = nullptr;
};
std::mutex g_addr_mutex;
ScratchSlot g_slot[kMaxDevices];

typedef CUresult (*CtxGetCurrentFn)(CUcontext*);
typedef CUresult (*CtxGetIdFn)(CUcontext, unsigned long long*);
CtxGetCurrentFn g_ctx_get_current = nullptr;
CtxGetIdFn g_ctx_get_id = nullptr;

// Unique id of the calling thread's current context on device `dev` (the runtime's primary
// context, made current first if no context is).  Driver entry points come through the
// runtime, so the library needs no link against the driver library.
align_status current_context_id(int dev, unsigned long long* id) {
  if (g_ctx_get_current == nullptr || g_ctx_get_id == nullptr) {
    void* f0 = nullptr;
    void* f1 = nullptr;
    cudaDriverEntryPointQueryResult q0, q1;
    cudaError_t e = cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f0, 12000, cudaEnableDefault, &q0);
    if (e == cudaSuccess) e = cudaGetDriverEntryPointByVersion("cuCtxGetId", &f1, 12000, cudaEnableDefault, &q1);
    if (e != cudaSuccess) return report_cuda_error(e, "cudaGetDriverEntryPointByVersion");
    if (q0 != cudaDriverEntryPointSuccess || q1 != cudaDriverEntryPointSuccess || !f0 || !f1)
      return report_error(ALIGN_E_CUDA, "driver entry points cuCtxGetCurrent/cuCtxGetId not found");
    g_ctx_get_current = reinterpret_cast<CtxGetCurrentFn>(f0);
    g_ctx_get_id = reinterpret_cast<CtxGetIdFn>(f1);
  }
  CUcontext ctx = nullptr;
  if (g_ctx_get_current(&ctx) != CUDA_SUCCESS) return report_error(ALIGN_E_CUDA, "cuCtxGetCurrent failed");
  if (ctx == nullptr) {  // no context current yet: cudaSetDevice initialises the primary context
    cudaError_t e = cudaSetDevice(dev);
    if (e != cudaSuccess) return report_cuda_error(e, "cudaSetDevice");
    if (g_ctx_get_current(&ctx) != CUDA_SUCCESS || ctx == nullptr)
      return report_error(ALIGN_E_CUDA, "no current CUDA context");
  }
  if (g_ctx_get_id(ctx, id) != CUDA_SUCCESS) return report_error(ALIGN_E_CUDA, "cuCtxGetId failed");
  return ALIGN_OK;
}

__global__ void noalloc_clear_kernel(unsigned char* base, int64_t V, Pose12 pose, int32_t* box) {
  uint32_t* cnt = reinterpret_cast<uint32_t*>(base);
  unsigned long long* s1 = reinterpret_cast<unsigned long long*>(base + kCntBytes);
  unsigned long long* s2 = reinterpret_cast<unsigned long long*>(base + kCntBytes + kSumBytes);
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < V; v += (int64_t)gridDim.x * blockDim.x) {
    cnt[v] = 0u;
    s1[v] = 0ull;
    s2[v] = 0ull;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    float* p = reinterpret_cast<float*>(base + kCntBytes + 2 * kSumBytes);
    for (int i = 0; i < 9; ++i) p[i] = pose.r[i];
    for (int i = 0; i < 3; ++i) p[9 + i] = pose.t[i];
    box[0] = box[1] = box[2] = INT_MAX;
    box[3] = box[4] = box[5] = INT_MIN;
  }
}

align_status scratch_address(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return report_cuda_error(e, "cudaGetDevice");
  if (dev < 0 || dev >= kMaxDevices) return report_error(ALIGN_E_INVALID, "device index beyond 63");
  std::lock_guard<std::mutex> lock(g_addr_mutex);
  unsigned long long ctx_id = 0;
  align_status st = current_context_id(dev, &ctx_id);
  if (st != ALIGN_OK) return st;
  ScratchSlot& slot = g_slot[dev];
  if (slot.addr == nullptr || slot.ctx_id != ctx_id) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return report_cuda_error(e, "cudaGetSymbolAddress(noalloc scratch)");
    slot.addr = p;
    slot.ctx_id = ctx_id;
  }
  *out = slot.addr;
  return ALIGN_OK;
}

}  // namespace

}  // namespace mialign

using namespace mialign;

extern "C" align_status align_reference_noalloc(const align_grid_desc* desc, const float* xyzA, int64_t nA,
                                                uint8_t* symA, int32_t* boxA, void* cuda_stream) {
  GridConst gc;
  align_status st = check_grid_desc(desc, &gc);
  if (st != ALIGN_OK) return st;
  const int64_t V = (int64_t)gc.X * gc.Y * gc.Z;
  if (V > kNoallocMaxVoxels)
    return report_error(ALIGN_E_INVALID, "align_reference_noalloc: grid has more than 2^19 voxels");
  if (nA < 0 || nA >= INT32_MAX) return report_error(ALIGN_E_INVALID, "nA out of range");
  if ((nA > 0 && !xyzA) || !symA || !boxA) return report_error(ALIGN_E_INVALID, "NULL buffer");
  void* base = nullptr;
  st = scratch_address(&base);
  if (st != ALIGN_OK) return st;
  cudaStream_t s = (cudaStream_t)cuda_stream;
  unsigned char* b = static_cast<unsigned char*>(base);
  uint32_t* cnt = reinterpret_cast<uint32_t*>(b);
  unsigned long long* s1 = reinterpret_cast<unsigned long long*>(b + kCntBytes);
  unsigned long long* s2 = reinterpret_cast<unsigned long long*>(b + kCntBytes + kSumBytes);
  const float* pose_dev = reinterpret_cast<const float*>(b + kCntBytes + 2 * kSumBytes);

  // A is never moved: the identity pose, rounded by the same host convention.
  float ident[12];
  const double eta0[6] = {0, 0, 0, 0, 0, 0};
  round_pose_host(desc->origin, eta0, ident);
  Pose12 pose;
  for (int i = 0; i < 9; ++i) pose.r[i] = ident[i];
  for (int i = 0; i < 3; ++i) pose.t[i] = ident[9 + i];

  int blocks = (int)std::min<int64_t>((V + 255) / 256, 4096);
  noalloc_clear_kernel<<<blocks < 1 ? 1 : blocks, 256, 0, s>>>(b, V, pose, boxA);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return report_cuda_error(e, "launch clear");
  e = launch_ref_accumulate(gc, xyzA, nA, pose_dev, cnt, s1, s2, s);
  if (e != cudaSuccess) return report_cuda_error(e, "launch accumulate");
  e = launch_ref_symbols(gc, cnt, s1, s2, symA, boxA, s);
  if (e != cudaSuccess) return report_cuda_error(e, "launch symbols");
  return ALIGN_OK;
}
