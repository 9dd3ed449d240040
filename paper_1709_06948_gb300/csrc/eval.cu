// eval.cu — the pose-batched MI hot path (arXiv 1709.06948, Algorithm 1 loop body for
// a whole batch of candidate poses; Sec. III-A features; Eqs. 1-5).
//
// pack_points_kernel: scan B as float4 tiles (NaN padding), either raw xyz or one
// pre-rotated copy u = R p per distinct rotation of the batch (a search lattice has 32
// rotations for 4,096 poses, so the 9-FMA rotation leaves the per-pose loop).  The tiles
// are laid out as kThreads streams: thread s of a CTA reads, tile after tile, the points
// s*L, s*L+1, ... of B's given order (L = kPPT * tiles), so each thread walks a stretch
// of consecutive scan points.
//
// eval_kernel: persistent, one CTA per SM, one pose at a time per CTA.  The tiles of the
// pose's source array arrive by 1-D bulk (TMA) copies on a cyclic mbarrier ring whose
// schedule already knows the CTA's next pose, so the copies never stall at pose
// boundaries.  Per point and pose: voxel key and dz (device_common.cuh).  Each thread
// keeps the run of equal keys it is walking in registers (n, S1, S2); when the key
// changes, the finished run is added into a shared-memory open-addressing hash table
// with 32-bit shared atomics.  After the sweep one pass over the table gives the feature
// symbols, B's occupied bbox and the partial joint histogram c[a][b >= 1] of the occupied
// voxels inside A's bbox.
//  - A pose with more occupied voxels than fit the table is handed to redo_kernel (which
//    splits the keys into 2, 4, ... hash partitions, one sweep each); a crowded table
//    makes the CTA sweep its following poses in twice as many partitions.
//  - A voxel with more points than the 32-bit sums allow diverts its later runs to 64-bit
//    side sums in global memory (per CTA, indexed by table slot).
//
// compose_kernel: per pose, the overlap box (Algorithm 1), A's symbol counts over it from
// per-symbol prefix sums, the phi column h[a][0], then Eqs. 2-5 in FP32 with a fixed
// reduction order, and the packed (MI, index) maximum for Eq. 1.
#include <climits>

#include "align_internal.h"
#include "device_common.cuh"

namespace mialign {

namespace {

constexpr int kThreads = 1024;
constexpr int kWarps = kThreads / 32;
constexpr int kPPT = 1;                       // points per thread per tile
constexpr int kTile = kThreads * kPPT;        // points per tile
constexpr uint32_t kTileBytes = kTile * 16u;  // float4 per point
constexpr int kStages = 3;
// Tile delivery: true = bulk (TMA) copies into a shared-memory ring; false = every thread
// loads its own stream's points from L2 into registers, three tiles ahead.
constexpr bool kTmaTiles = false;
constexpr uint32_t kQueue = 64;               // finished runs buffered per warp
constexpr int kMaxPasses = 1 << 16;
constexpr uint32_t kFull = 0xFFFFFFFFu;

__host__ __device__ constexpr int round4(int x) { return (x + 3) & ~3; }

struct EvalSmem {
  float4* tiles;
  uint4* queue;         // per warp: a ring of kQueue finished runs (key, n, S1, S2)
  uint32_t* tkey;
  uint32_t* tcnt;
  int32_t* ts1;
  uint32_t* ts2;
  uint32_t* hist;
  uint32_t* ct;
  int64_t* vt;
  uint64_t* mbar;       // [0, kStages): full, [kStages, 2 kStages): empty
  uint32_t* issue_cnt;  // kStages
  uint32_t* sched;      // q_start, n_consume, src_cur, src_next
  int32_t* box;         // 6
  uint32_t* flags;      // occupied count, table full, abort, sums need the exact path
};

__host__ __device__ inline size_t eval_smem_layout(int K, int T, EvalSmem* s, uint8_t* base) {
  size_t off = 0;
  auto take = [&](size_t bytes, size_t align) {
    off = (off + align - 1) / align * align;
    size_t o = off;
    off += bytes;
    return o;
  };
  size_t o_tiles = take(kTmaTiles ? (size_t)kStages * kTileBytes : 16, 128);
  size_t o_queue = take((size_t)kWarps * kQueue * 16, 16);
  size_t o_key = take((size_t)T * 4, 16);
  size_t o_cnt = take((size_t)T * 4, 16);
  size_t o_s1 = take((size_t)T * 4, 16);
  size_t o_s2 = take((size_t)T * 4, 16);
  size_t o_hist = take((size_t)round4(K * K) * 4, 16);
  size_t o_ct = take(kMaxLevels * 4 + 4, 16);
  size_t o_vt = take(kMaxLevels * 8 + 8, 16);
  size_t o_mbar = take(2 * kStages * 8, 8);
  size_t o_issue = take(kStages * 4, 4);
  size_t o_sched = take(4 * 4, 4);
  size_t o_box = take(6 * 4, 4);
  size_t o_flags = take(4 * 4, 4);
  if (s) {
    s->tiles = (float4*)(base + o_tiles);
    s->queue = (uint4*)(base + o_queue);
    s->tkey = (uint32_t*)(base + o_key);
    s->tcnt = (uint32_t*)(base + o_cnt);
    s->ts1 = (int32_t*)(base + o_s1);
    s->ts2 = (uint32_t*)(base + o_s2);
    s->hist = (uint32_t*)(base + o_hist);
    s->ct = (uint32_t*)(base + o_ct);
    s->vt = (int64_t*)(base + o_vt);
    s->mbar = (uint64_t*)(base + o_mbar);
    s->issue_cnt = (uint32_t*)(base + o_issue);
    s->sched = (uint32_t*)(base + o_sched);
    s->box = (int32_t*)(base + o_box);
    s->flags = (uint32_t*)(base + o_flags);
  }
  return off;
}

__device__ __forceinline__ uint32_t pose_source(const EvalArgs& a, int p) {
  return a.pose_src ? (uint32_t)a.pose_src[p] : 0u;
}

// Issue the bulk copy for consumption index q: within the current pose's sweeps it is a
// tile of the current source array, past them a tile of the next pose's array.
__device__ __forceinline__ void issue_tile(const EvalSmem& S, const EvalArgs& a, uint32_t q) {
  const uint32_t b = q % kStages;
  const uint32_t rel = q - S.sched[0];
  uint32_t src, tile;
  if (rel < S.sched[1]) {
    src = S.sched[2];
    tile = rel % (uint32_t)a.n_tiles;
  } else {
    src = S.sched[3];
    tile = (rel - S.sched[1]) % (uint32_t)a.n_tiles;
  }
  const uint32_t full = smem_addr(&S.mbar[b]);
  mbar_arrive_expect_tx(full, kTileBytes);
  bulk_copy_g2s(smem_addr(S.tiles + (size_t)b * kTile), a.src + (size_t)src * a.src_stride + (size_t)tile * kTile,
                kTileBytes, full);
}

// Find or insert `key` in the open-addressing table: buckets of 4 key slots read with one
// 16-byte load, probed linearly; slots of a bucket fill in order, so a bucket with a free
// slot ends the search.  Returns -1 when the probe budget is spent (table full).
__device__ __forceinline__ int table_slot(const EvalSmem& S, uint32_t key, int T) {
  const uint32_t nb = (uint32_t)T >> 2;
  uint32_t b = __umulhi(key * 0x9E3779B1u, nb);
  for (uint32_t i = 0; i < nb + 4; ++i) {
    uint4 k4;
    asm volatile("ld.volatile.shared.v4.u32 {%0, %1, %2, %3}, [%4];"
                 : "=r"(k4.x), "=r"(k4.y), "=r"(k4.z), "=r"(k4.w)
                 : "r"(smem_addr(S.tkey + 4 * b)));
    if (k4.x == key) return (int)(4 * b);
    if (k4.y == key) return (int)(4 * b + 1);
    if (k4.z == key) return (int)(4 * b + 2);
    if (k4.w == key) return (int)(4 * b + 3);
    const int e = (k4.x == kEmptyKey) ? 0 : (k4.y == kEmptyKey) ? 1 : (k4.z == kEmptyKey) ? 2 : (k4.w == kEmptyKey) ? 3 : -1;
    if (e >= 0) {
      const uint32_t old = atomicCAS(&S.tkey[4 * b + e], kEmptyKey, key);
      if (old == kEmptyKey || old == key) return (int)(4 * b + e);
      continue;  // another lane took that slot: read the bucket again
    }
    b = (b + 1 == nb) ? 0u : b + 1;
  }
  return -1;
}

// Add one finished run (n points of one voxel, sums s1, s2) to the table.
template <bool kVar>
__device__ __forceinline__ void add_run(const EvalSmem& S, const GridConst& gc, unsigned long long* wide, uint32_t key,
                                        uint32_t n, int s1, uint32_t s2, int T) {
  if (*(volatile uint32_t*)&S.flags[1]) return;  // table already full: the pose is redone
  const int slot = table_slot(S, key, T);
  if (slot < 0) {
    S.flags[1] = 1u;
    return;
  }
  if (kVar) {
    const uint32_t old = atomicAdd(&S.tcnt[slot], n);
    if (old + n <= gc.nlim) {
      atomicAdd(&S.ts1[slot], s1);
      atomicAdd(&S.ts2[slot], s2);
    } else {
      atomicAdd(&wide[2 * slot], (unsigned long long)(long long)s1);
      atomicAdd(&wide[2 * slot + 1], (unsigned long long)s2);
      S.flags[3] = 1u;
    }
  } else {
    atomicAdd(&S.tcnt[slot], n);
  }
}

// Fast path: add a finished run with fire-and-forget 32-bit shared atomics.  A voxel whose
// count ends above nlim may have wrapped its sums; the table scan sends such a pose to the
// exact path (redo_kernel).
template <bool kVar>
__device__ __forceinline__ void fast_add(const EvalSmem& S, const uint4& e, int T) {
  if (*(volatile uint32_t*)&S.flags[1]) return;
  const int slot = table_slot(S, e.x, T);
  if (slot < 0) {
    S.flags[1] = 1u;
    return;
  }
  atomicAdd(&S.tcnt[slot], e.y);
  if (kVar) {
    atomicAdd(&S.ts1[slot], (int)e.z);
    atomicAdd(&S.ts2[slot], e.w);
  }
}

// Per-warp ring of finished runs: lanes append what they finished at this step; once 32
// are waiting, the whole warp adds 32 of them to the table at once.
struct WarpQueue {
  uint32_t head;
  uint32_t fill;
};

template <bool kVar>
__device__ __forceinline__ void queue_drain(const EvalSmem& S, uint4* ring, WarpQueue& wq, int lane, int T,
                                            uint32_t count) {
  __syncwarp();
  if ((uint32_t)lane < count) fast_add<kVar>(S, ring[(wq.head + (uint32_t)lane) & (kQueue - 1)], T);
  __syncwarp();
  wq.head = (wq.head + count) & (kQueue - 1);
  wq.fill -= count;
}

template <bool kVar>
__device__ __forceinline__ void queue_push(const EvalSmem& S, uint4* ring, WarpQueue& wq, int lane, bool has,
                                           const uint4& e, int T) {
  const uint32_t m = __ballot_sync(kFull, has);
  if (m == 0u) return;
  if (has) ring[(wq.head + wq.fill + (uint32_t)__popc(m & ((1u << lane) - 1u))) & (kQueue - 1)] = e;
  wq.fill += (uint32_t)__popc(m);
  if (wq.fill >= 32u) queue_drain<kVar>(S, ring, wq, lane, T, 32u);
}

// The run of equal keys a thread is walking.  Keys outside the current partition (and
// points outside the grid) are skipped without ending the run.
struct Run {
  uint32_t key;
  uint32_t n;
  int s1;
  uint32_t s2;
};

// Advance a run by one point; returns true (and the finished run in `fin`) when the key
// changes.  A run stays below nlim points so that its 32-bit sums cannot overflow.
template <bool kVar>
__device__ __forceinline__ bool advance_run(const GridConst& gc, Run& r, uint32_t key, int dz, uint4& fin) {
  if (key == kEmptyKey) return false;
  if (key == r.key && (!kVar || r.n < gc.nlim)) {
    r.n += 1u;
    if (kVar) {
      r.s1 += dz;
      r.s2 += (uint32_t)(dz * dz);
    }
    return false;
  }
  const bool done = r.n != 0u;
  fin = make_uint4(r.key, r.n, (uint32_t)r.s1, r.s2);
  r.key = key;
  r.n = 1u;
  r.s1 = dz;
  r.s2 = (uint32_t)(dz * dz);
  return done;
}

// Exact path (redo_kernel): the run goes straight to the table, with 64-bit side sums
// for voxels beyond nlim points.
template <bool kVar>
__device__ __forceinline__ void step_run(const EvalSmem& S, const GridConst& gc, unsigned long long* wide, Run& r,
                                         uint32_t key, int dz, int T) {
  if (key == kEmptyKey) return;
  // a run stays below nlim points so that its 32-bit sums cannot overflow
  if (key == r.key && (!kVar || r.n < gc.nlim)) {
    r.n += 1u;
    if (kVar) {
      r.s1 += dz;
      r.s2 += (uint32_t)(dz * dz);
    }
    return;
  }
  if (r.n != 0u) add_run<kVar>(S, gc, wide, r.key, r.n, r.s1, r.s2, T);
  r.key = key;
  r.n = 1u;
  r.s1 = dz;
  r.s2 = (uint32_t)(dz * dz);
}

struct PoseRegs {
  float r[9];
  float t[3];
};

// Keys of this thread's kPPT points (in registers) under the pose (key partition `part`
// of 2^lg).
template <bool kRot>
__device__ __forceinline__ void regs_keys(const GridConst& gc, const PoseRegs& P, const float4* pts, int lg,
                                          uint32_t part, uint32_t* key, int* dz) {
#pragma unroll
  for (int j = 0; j < kPPT; ++j) {
    const float4 p = pts[j];
    float gx, gy, gz;
    dz[j] = 0;
    if (kRot) {
      float ux, uy, uz;
      rotate_point(P.r, p.x, p.y, p.z, ux, uy, uz);
      gx = __fadd_rn(ux, P.t[0]);
      gy = __fadd_rn(uy, P.t[1]);
      gz = __fadd_rn(uz, P.t[2]);
      key[j] = voxel_key_g(gx, gy, gz, gc.inv_res, gc.X, gc.Y, gc.Z, gc.res_mm, &dz[j]);
    } else {
      // Pre-rotated copies hold finite values or +inf (pack_points_kernel), and host poses
      // are finite, so g is never NaN: a saturating floor and unsigned compares decide
      // "inside" exactly as the float compares would.
      gx = __fadd_rn(p.x, P.t[0]);
      gy = __fadd_rn(p.y, P.t[1]);
      gz = __fadd_rn(p.z, P.t[2]);
      const int kx = __float2int_rd(__fmul_rn(gx, gc.inv_res));
      const int ky = __float2int_rd(__fmul_rn(gy, gc.inv_res));
      const int kz = __float2int_rd(__fmul_rn(gz, gc.inv_res));
      const bool in = ((uint32_t)kx < (uint32_t)gc.X) & ((uint32_t)ky < (uint32_t)gc.Y) & ((uint32_t)kz < (uint32_t)gc.Z);
      dz[j] = __float2int_rn(__fmul_rn(gz, 1000.0f)) - kz * gc.res_mm;
      key[j] = in ? (uint32_t)((kz * gc.Y + ky) * gc.X + kx) : kEmptyKey;
    }
    if (lg > 0 && key[j] != kEmptyKey && ((key[j] * 0x85EBCA77u) >> (32 - lg)) != part) key[j] = kEmptyKey;
  }
}

// The same for this thread's points of one tile (`pts`: the tile plus the thread index;
// the thread's points are kThreads apart).
template <bool kRot>
__device__ __forceinline__ void tile_keys(const GridConst& gc, const PoseRegs& P, const float4* pts, int lg,
                                          uint32_t part, uint32_t* key, int* dz) {
  float4 v[kPPT];
#pragma unroll
  for (int j = 0; j < kPPT; ++j) v[j] = pts[j * kThreads];
  regs_keys<kRot>(gc, P, v, lg, part, key, dz);
}

__device__ __forceinline__ void load_pose(const EvalArgs& a, int p, PoseRegs& P) {
#pragma unroll
  for (int i = 0; i < 9; ++i) P.r[i] = __ldg(a.poses + 12 * (size_t)p + i);
#pragma unroll
  for (int i = 0; i < 3; ++i) P.t[i] = __ldg(a.poses + 12 * (size_t)p + 9 + i);
}

// Read (and clear) the table after a sweep: symbols, bbox and histogram unless `discard`.
// The CTA-wide occupied count is added to S.flags[0].
template <bool kVar, bool kExact>
__device__ __forceinline__ void scan_table(const EvalSmem& S, const GridConst& gc, const EvalArgs& a,
                                           unsigned long long* wide, int T, int K, int p, bool discard) {
  const int tid = threadIdx.x, lane = tid & 31;
  int mn0 = INT_MAX, mn1 = INT_MAX, mn2 = INT_MAX, mx0 = INT_MIN, mx1 = INT_MIN, mx2 = INT_MIN;
  uint32_t occupied = 0;
  for (int s = tid; s < T; s += kThreads) {
    const uint32_t k = S.tkey[s];
    if (k == kEmptyKey) continue;
    ++occupied;
    const uint64_t n = S.tcnt[s];
    int64_t s1 = S.ts1[s];
    uint64_t s2 = S.ts2[s];
    if (!kExact && kVar && n > gc.nlim) S.flags[3] = 1u;  // sums may have wrapped: exact path
    if (kExact && kVar && n > gc.nlim) {
      s1 += (int64_t)wide[2 * s];
      s2 += wide[2 * s + 1];
      wide[2 * s] = 0ull;
      wide[2 * s + 1] = 0ull;
      if (!discard) atomicAdd(a.wide_count, 1u);
    }
    S.tkey[s] = kEmptyKey;
    S.tcnt[s] = 0u;
    S.ts1[s] = 0;
    S.ts2[s] = 0u;
    if (discard) continue;
    const int kx = (int)(k % (uint32_t)gc.X);
    const uint32_t r = k / (uint32_t)gc.X;
    const int ky = (int)(r % (uint32_t)gc.Y);
    const int kz = (int)(r / (uint32_t)gc.Y);
    mn0 = min(mn0, kx); mn1 = min(mn1, ky); mn2 = min(mn2, kz);
    mx0 = max(mx0, kx); mx1 = max(mx1, ky); mx2 = max(mx2, kz);
    const int sB = feature_symbol(gc.feature, gc.Lc, gc.Lv, S.ct, S.vt, n, s1, s2);
    if (kx >= gc.boxA[0] && kx <= gc.boxA[3] && ky >= gc.boxA[1] && ky <= gc.boxA[4] && kz >= gc.boxA[2] &&
        kz <= gc.boxA[5])
      atomicAdd(&S.hist[(int)__ldg(a.symA + k) * K + sB], 1u);
    if (a.dump != nullptr && p == 0) {
      a.dump[3 * (size_t)k] = (int64_t)n;
      a.dump[3 * (size_t)k + 1] = s1;
      a.dump[3 * (size_t)k + 2] = (int64_t)s2;
    }
  }
  occupied = __reduce_add_sync(kFull, occupied);
  if (lane == 0 && occupied) atomicAdd(&S.flags[0], occupied);
  mn0 = __reduce_min_sync(kFull, mn0); mn1 = __reduce_min_sync(kFull, mn1);
  mn2 = __reduce_min_sync(kFull, mn2); mx0 = __reduce_max_sync(kFull, mx0);
  mx1 = __reduce_max_sync(kFull, mx1); mx2 = __reduce_max_sync(kFull, mx2);
  if (lane == 0 && !discard && mn0 != INT_MAX) {
    atomicMin(&S.box[0], mn0); atomicMin(&S.box[1], mn1); atomicMin(&S.box[2], mn2);
    atomicMax(&S.box[3], mx0); atomicMax(&S.box[4], mx1); atomicMax(&S.box[5], mx2);
  }
}

__device__ __forceinline__ void init_smem(const EvalSmem& S, const GridConst& gc, int T, int KK) {
  const int tid = threadIdx.x;
  for (int i = tid; i < T; i += kThreads) {
    S.tkey[i] = kEmptyKey;
    S.tcnt[i] = 0u;
    S.ts1[i] = 0;
    S.ts2[i] = 0u;
  }
  for (int i = tid; i < KK; i += kThreads) S.hist[i] = 0u;
  if (tid < kMaxLevels) {
    S.ct[tid] = gc.count_thresh[tid];
    S.vt[tid] = gc.var_thresh[tid];
  }
  if (tid == 0) {
    S.box[0] = S.box[1] = S.box[2] = INT_MAX;
    S.box[3] = S.box[4] = S.box[5] = INT_MIN;
    S.flags[0] = S.flags[1] = S.flags[2] = S.flags[3] = 0u;
  }
}

// Store the pose's partial histogram and bbox, then reset them for the next pose.
__device__ __forceinline__ void emit_pose(const EvalSmem& S, const EvalArgs& a, int KK, int p) {
  const int tid = threadIdx.x;
  uint32_t* oc = a.out_c + (size_t)p * KK;
  for (int i = tid; i < KK; i += kThreads) {
    oc[i] = S.hist[i];
    S.hist[i] = 0u;
  }
  if (tid < 6) a.out_box[6 * (size_t)p + tid] = S.box[tid];
  __syncthreads();
  if (tid < 6) S.box[tid] = tid < 3 ? INT_MAX : INT_MIN;
}

__device__ __forceinline__ void reset_pose(const EvalSmem& S, int KK) {
  const int tid = threadIdx.x;
  for (int i = tid; i < KK; i += kThreads) S.hist[i] = 0u;
  if (tid < 6) S.box[tid] = tid < 3 ? INT_MAX : INT_MIN;
}

__device__ __forceinline__ void load_tile(const float4* src, int t, float4* v) {
#pragma unroll
  for (int j = 0; j < kPPT; ++j) v[j] = __ldg(src + (size_t)t * kTile + j * kThreads);
}

// One tile of this thread's stream: keys, run stepping, queueing of finished runs.  A dz
// outside its proven bound is remembered in `bad` (reported once per sweep).
template <bool kVar, bool kRot>
__device__ __forceinline__ void sweep_tile(const EvalSmem& S, const GridConst& gc, const PoseRegs& P,
                                           const float4* pts, int lg, int pass, Run& run, WarpQueue& wq, uint4* ring,
                                           int lane, int T, uint32_t& bad) {
  uint32_t key[kPPT];
  int dz[kPPT];
  regs_keys<kRot>(gc, P, pts, lg, (uint32_t)pass, key, dz);
#pragma unroll
  for (int j = 0; j < kPPT; ++j) {
    bad |= (uint32_t)(key[j] != kEmptyKey) & (uint32_t)((uint32_t)(dz[j] + gc.dz_bound) > (uint32_t)(2 * gc.dz_bound));
    uint4 fin;
    const bool has = advance_run<kVar>(gc, run, key[j], dz[j], fin);
    queue_push<kVar>(S, ring, wq, lane, has, fin, T);
  }
}

template <bool kVar, bool kRot>
__global__ void __launch_bounds__(kThreads, 1) eval_kernel(const GridConst gc, const EvalArgs a) {
  extern __shared__ __align__(128) uint8_t smem_raw[];
  EvalSmem S;
  const int T = a.table_slots;
  const int K = gc.K, KK = K * K;
  eval_smem_layout(K, T, &S, smem_raw);
  const int tid = threadIdx.x, lane = tid & 31;
  const uint32_t cap = (uint32_t)T - (uint32_t)T / 10u;  // above 90% full the table counts as crowded
  uint4* ring = S.queue + (size_t)(tid >> 5) * kQueue;
  unsigned long long* wide = a.wide + (size_t)blockIdx.x * 2u * (size_t)T;
  const int G = gridDim.x;

  init_smem(S, gc, T, KK);
  int passes = a.passes0;
  if (kTmaTiles && tid == 0) {
    for (int b = 0; b < kStages; ++b) {
      mbar_init(smem_addr(&S.mbar[b]), 1u);
      mbar_init(smem_addr(&S.mbar[kStages + b]), (uint32_t)kWarps);
      S.issue_cnt[b] = 0u;
    }
    const int p0 = blockIdx.x;
    S.sched[0] = 0u;
    S.sched[1] = (uint32_t)passes * (uint32_t)a.n_tiles;
    S.sched[2] = pose_source(a, p0);
    S.sched[3] = pose_source(a, p0 + G < a.P ? p0 + G : p0);
    fence_mbar_init();
  }
  __syncthreads();
  if (kTmaTiles && tid == 0)
    for (int b = 0; b < kStages; ++b) issue_tile(S, a, (uint32_t)b);

  uint32_t q = 0;  // consumption counter, identical in every warp
  bool aborted = false;

  for (int p = blockIdx.x; p < a.P && !aborted; p += G) {
    if (kTmaTiles && p != (int)blockIdx.x) {
      if (tid == 0) {  // the pose's sweeps start at q; every warp is past the previous pose
        S.sched[0] = q;
        S.sched[1] = (uint32_t)passes * (uint32_t)a.n_tiles;
        S.sched[2] = pose_source(a, p);
        S.sched[3] = pose_source(a, p + G < a.P ? p + G : p);
      }
      __syncthreads();
    }
    PoseRegs P;
    load_pose(a, p, P);
    const int pose_passes = passes;
    const int lg = __ffs(pose_passes) - 1;
    uint32_t max_occupied = 0;
    bool full = false;
    for (int pass = 0; pass < pose_passes; ++pass) {
      Run run{kEmptyKey, 0u, 0, 0u};
      WarpQueue wq{0u, 0u};
      // ---- sweep all tiles of the pose's source array ----
      if constexpr (kTmaTiles) {
        for (int t = 0; t < a.n_tiles; ++t, ++q) {
          const uint32_t b = q % kStages;
          const uint32_t par = (q / kStages) & 1u;
          if (*(volatile uint32_t*)&S.flags[2]) continue;  // aborting: no more waits
          if (!mbar_wait_bounded(smem_addr(&S.mbar[b]), par, kWaitLimitNs)) {
            atomicOr(a.err, kErrWaitTimeout);
            S.flags[2] = 1u;
            continue;
          }
          if (!full) {
            uint32_t key[kPPT];
            int dz[kPPT];
            tile_keys<kRot>(gc, P, S.tiles + (size_t)b * kTile + tid, lg, (uint32_t)pass, key, dz);
  #pragma unroll
            for (int j = 0; j < kPPT; ++j) {
              if (key[j] != kEmptyKey && (uint32_t)(dz[j] + gc.dz_bound) > (uint32_t)(2 * gc.dz_bound))
                atomicOr(a.err, kErrDzBound);
              uint4 fin;
              const bool has = advance_run<kVar>(gc, run, key[j], dz[j], fin);
              queue_push<kVar>(S, ring, wq, lane, has, fin, T);
            }
          }
          __syncwarp();
          if (lane == 0) {
            mbar_arrive(smem_addr(&S.mbar[kStages + b]));
            const uint32_t c = atomicAdd(&S.issue_cnt[b], 1u);
            if (c == (uint32_t)kWarps - 1u) {  // the last warp done with this buffer refills it
              S.issue_cnt[b] = 0u;
              if (mbar_wait_bounded(smem_addr(&S.mbar[kStages + b]), par, kWaitLimitNs)) {
                issue_tile(S, a, q + kStages);
              } else {
                atomicOr(a.err, kErrWaitTimeout);
                S.flags[2] = 1u;
              }
            }
          }
        }
      } else {
        // every thread streams its own points straight from L2, three tiles ahead
        const float4* src = a.src + (size_t)pose_source(a, p) * a.src_stride + tid;
        float4 b0[kPPT], b1[kPPT], b2[kPPT];
        load_tile(src, 0, b0);
        load_tile(src, 1, b1);
        load_tile(src, 2, b2);
        uint32_t bad = 0u;
        const int nt = a.n_tiles;
        for (int t = 0; t < nt && !full; t += 3) {
          sweep_tile<kVar, kRot>(S, gc, P, b0, lg, pass, run, wq, ring, lane, T, bad);
          if (t + 3 < nt) load_tile(src, t + 3, b0);
          if (t + 1 < nt) {
            sweep_tile<kVar, kRot>(S, gc, P, b1, lg, pass, run, wq, ring, lane, T, bad);
            if (t + 4 < nt) load_tile(src, t + 4, b1);
          }
          if (t + 2 < nt) {
            sweep_tile<kVar, kRot>(S, gc, P, b2, lg, pass, run, wq, ring, lane, T, bad);
            if (t + 5 < nt) load_tile(src, t + 5, b2);
          }
        }
        if (bad) atomicOr(a.err, kErrDzBound);
      }
      if (!full) {
        queue_push<kVar>(S, ring, wq, lane, run.n != 0u, make_uint4(run.key, run.n, (uint32_t)run.s1, run.s2), T);
        while (wq.fill > 0u) queue_drain<kVar>(S, ring, wq, lane, T, min(wq.fill, 32u));
      }
      __syncthreads();
      if (S.flags[2]) {
        aborted = true;
        break;
      }
      full = full || S.flags[1] != 0u;
      scan_table<kVar, false>(S, gc, a, wide, T, K, p, full);
      __syncthreads();
      max_occupied = max(max_occupied, S.flags[0]);
      full = full || S.flags[3] != 0u;
      __syncthreads();
      if (tid == 0) {
        S.flags[0] = 0u;
        S.flags[3] = 0u;
      }
    }
    if (aborted) break;
    if (full) {
      // the remaining sweeps of this pose were consumed without work; finish it later
      reset_pose(S, KK);
      if (tid == 0) {
        S.flags[1] = 0u;
        a.redo_list[atomicAdd(a.redo_count, 1u)] = (uint32_t)p;
      }
      if (passes < kMaxPasses) passes *= 2;
      __syncthreads();
      continue;
    }
    emit_pose(S, a, KK, p);
    if (max_occupied > cap && passes < kMaxPasses) passes *= 2;  // crowded: more partitions next
  }

  // Drain the prefetched tiles still in flight before the CTA's shared memory is released.
  __syncthreads();
  if (tid == 0) {
    if (!aborted) atomicMax(a.max_passes, (uint32_t)passes);
    for (int i = 0; kTmaTiles && i < kStages; ++i) {
      const uint32_t qq = q + (uint32_t)i;
      if (!mbar_wait_bounded(smem_addr(&S.mbar[qq % kStages]), (qq / kStages) & 1u, kWaitLimitNs))
        atomicOr(a.err, kErrWaitTimeout);
    }
  }
}

// Poses whose table filled up in eval_kernel: plain loads (no prefetch ring), and on a full
// table the pose simply restarts with twice the key partitions.
template <bool kVar, bool kRot>
__global__ void __launch_bounds__(kThreads, 1) redo_kernel(const GridConst gc, const EvalArgs a) {
  extern __shared__ __align__(128) uint8_t smem_raw[];
  EvalSmem S;
  const int T = a.table_slots;
  const int K = gc.K, KK = K * K;
  eval_smem_layout(K, T, &S, smem_raw);
  const int tid = threadIdx.x;
  unsigned long long* wide = a.wide + (size_t)blockIdx.x * 2u * (size_t)T;
  const uint32_t n_redo = *(volatile const uint32_t*)a.redo_count;
  if (blockIdx.x >= n_redo) return;
  init_smem(S, gc, T, KK);
  __syncthreads();
  int passes = 2 * (int)*(volatile const uint32_t*)a.max_passes;
  if (passes < 2) passes = 2;
  if (passes > kMaxPasses) passes = kMaxPasses;
  for (uint32_t i = blockIdx.x; i < n_redo; i += gridDim.x) {
    const int p = (int)a.redo_list[i];
    PoseRegs P;
    load_pose(a, p, P);
    const float4* src = a.src + (size_t)pose_source(a, p) * a.src_stride;
    int pass = 0;
    while (pass < passes) {
      const int lg = __ffs(passes) - 1;
      Run run{kEmptyKey, 0u, 0, 0u};
      for (int t = 0; t < a.n_tiles; ++t) {
        uint32_t key[kPPT];
        int dz[kPPT];
        tile_keys<kRot>(gc, P, src + (size_t)t * kTile + tid, lg, (uint32_t)pass, key, dz);
#pragma unroll
        for (int j = 0; j < kPPT; ++j) {
          if (key[j] != kEmptyKey && (uint32_t)(dz[j] + gc.dz_bound) > (uint32_t)(2 * gc.dz_bound))
            atomicOr(a.err, kErrDzBound);
          step_run<kVar>(S, gc, wide, run, key[j], dz[j], T);
        }
      }
      if (run.n != 0u) add_run<kVar>(S, gc, wide, run.key, run.n, run.s1, run.s2, T);
      __syncthreads();
      const bool full = S.flags[1] != 0u;
      scan_table<kVar, true>(S, gc, a, wide, T, K, p, full);
      __syncthreads();
      if (tid == 0) S.flags[0] = 0u;
      if (full) {
        reset_pose(S, KK);
        if (tid == 0) S.flags[1] = 0u;
        if (passes >= kMaxPasses) {
          if (tid == 0) atomicOr(a.err, kErrPassLimit);
          return;
        }
        passes *= 2;
        pass = 0;
        __syncthreads();
        continue;
      }
      ++pass;
      __syncthreads();
    }
    emit_pose(S, a, KK, p);
    __syncthreads();
  }
  if (tid == 0) atomicMax(a.max_passes, (uint32_t)passes);
}

// xyz -> float4 tiles (NaN padding), optionally one rotated copy per rotation.  Tile t,
// position j*kThreads + s holds point s*L + kPPT*t + j of B (L = kPPT * tiles): stream s
// visits consecutive points of B, kPPT per tile.
__global__ void pack_points_kernel(const float* __restrict__ xyz, int64_t n, int64_t n_out,
                                   const float* __restrict__ rots, float4* out) {
  const int r = blockIdx.y;
  const float nan = __int_as_float(0x7fc00000);
  float R[9];
  if (rots != nullptr)
    for (int i = 0; i < 9; ++i) R[i] = rots[9 * r + i];
  float4* o = out + (size_t)r * n_out;
  const int64_t L = n_out / kThreads;  // points per stream
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n_out; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t t = i / kTile;
    const int pos = (int)(i - t * kTile);
    const int j = pos / kThreads;
    const int sidx = pos - j * kThreads;
    const int64_t src = (int64_t)sidx * L + (int64_t)kPPT * t + j;
    // padding: NaN for raw tiles (the in-kernel rotation keeps NaN), +inf for rotated copies
    const float pad = rots != nullptr ? __int_as_float(0x7f800000) : nan;
    float4 v = make_float4(pad, pad, pad, 0.0f);
    if (src < n) {
      const float x = xyz[3 * src], y = xyz[3 * src + 1], z = xyz[3 * src + 2];
      if (rots != nullptr) {
        rotate_point(R, x, y, z, v.x, v.y, v.z);
        // a non-finite coordinate can only come from a non-finite point (or an overflow),
        // which the voxel map drops under every pose; +inf keeps it dropped
        if (!(isfinite(v.x) && isfinite(v.y) && isfinite(v.z))) v = make_float4(__int_as_float(0x7f800000),
                                                                               __int_as_float(0x7f800000),
                                                                               __int_as_float(0x7f800000), 0.0f);
      } else {
        v.x = x;
        v.y = y;
        v.z = z;
      }
    }
    o[i] = v;
  }
}

// -----------------------------------------------------------------------------------
// Compose: overlap box, A's counts over it, phi column, Eqs. 2-5, Eq. 1 key.
// -----------------------------------------------------------------------------------
constexpr int kComposeThreads = 256;

__device__ __forceinline__ long long sat_at(const int32_t* sat, int X1, int Y1, int x, int y, int z) {
  return (long long)sat[((size_t)z * Y1 + y) * X1 + x];
}

__device__ __forceinline__ float block_sum_fixed(float v, float* red) {
  // xor butterfly: every lane ends with the same value; warps combined in index order
  for (int m = 16; m >= 1; m >>= 1) v += __shfl_xor_sync(kFull, v, m);
  const int w = threadIdx.x >> 5;
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[w] = v;
  __syncthreads();
  float s = 0.0f;
  for (int i = 0; i < kComposeThreads / 32; ++i) s += red[i];
  return s;
}

__device__ __forceinline__ float neg_plogp(uint64_t c, float N) {
  if (c == 0) return 0.0f;
  const float q = __fdiv_rn((float)c, N);
  return -q * logf(q);
}

__global__ void __launch_bounds__(kComposeThreads) compose_kernel(const GridConst gc, const ComposeArgs a) {
  __shared__ uint32_t h[kMaxSymbols * kMaxSymbols];
  __shared__ long long cntA[kMaxSymbols];
  __shared__ float red[kComposeThreads / 32];
  const int p = blockIdx.x;
  const int tid = threadIdx.x;
  const int K = gc.K, KK = K * K;
  const int32_t* bb = a.boxB + 6 * (size_t)p;
  int lo[3], hi[3];
  bool empty = false;
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    lo[i] = max(gc.boxA[i], bb[i]);
    hi[i] = min(gc.boxA[3 + i], bb[3 + i]);
    empty |= lo[i] > hi[i];
  }
  const long long N = empty ? 0 : (long long)(hi[0] - lo[0] + 1) * (hi[1] - lo[1] + 1) * (hi[2] - lo[2] + 1);
  for (int i = tid; i < KK; i += kComposeThreads) h[i] = empty ? 0u : a.c[(size_t)p * KK + i];
  if (!empty && tid >= 1 && tid < K) {
    // count of A symbol `tid` over the box from its 3-D prefix sums (8 corners)
    const int X1 = gc.X + 1, Y1 = gc.Y + 1;
    const int32_t* S = a.sat + (size_t)(tid - 1) * (size_t)(gc.Z + 1) * Y1 * X1;
    const int x0 = lo[0], y0 = lo[1], z0 = lo[2], x1 = hi[0] + 1, y1 = hi[1] + 1, z1 = hi[2] + 1;
    cntA[tid] = sat_at(S, X1, Y1, x1, y1, z1) - sat_at(S, X1, Y1, x0, y1, z1) - sat_at(S, X1, Y1, x1, y0, z1) -
                sat_at(S, X1, Y1, x1, y1, z0) + sat_at(S, X1, Y1, x0, y0, z1) + sat_at(S, X1, Y1, x0, y1, z0) +
                sat_at(S, X1, Y1, x1, y0, z0) - sat_at(S, X1, Y1, x0, y0, z0);
  }
  __syncthreads();
  if (!empty && tid == 0) {
    long long s = 0;
    for (int i = 1; i < K; ++i) s += cntA[i];
    cntA[0] = N - s;
  }
  __syncthreads();
  if (!empty && tid < K) {
    uint32_t occ = 0;
    for (int b = 1; b < K; ++b) occ += h[tid * K + b];
    h[tid * K] = (uint32_t)(cntA[tid] - (long long)occ);  // A symbol tid, B phi
  }
  __syncthreads();
  float hxy = 0.0f, hx = 0.0f, hy = 0.0f;
  if (!empty) {
    const float Nf = (float)N;
    for (int i = tid; i < KK; i += kComposeThreads) hxy += neg_plogp(h[i], Nf);
    if (tid < K) {
      hx = neg_plogp((uint64_t)cntA[tid], Nf);
      uint64_t col = 0;
      for (int r = 0; r < K; ++r) col += h[r * K + tid];
      hy = neg_plogp(col, Nf);
    }
  }
  hxy = block_sum_fixed(hxy, red);
  hx = block_sum_fixed(hx, red);
  hy = block_sum_fixed(hy, red);
  const float mi = empty ? 0.0f : (hx + hy) - hxy;
  if (tid == 0) {
    a.mi[p] = mi;
    const uint32_t u = __float_as_uint(mi);
    const uint32_t ord = (u & 0x80000000u) ? ~u : (u | 0x80000000u);
    atomicMax(a.best, ((unsigned long long)ord << 32) | (unsigned long long)(0xFFFFFFFFu - (uint32_t)p));
  }
  if (a.hist != nullptr)
    for (int i = tid; i < KK; i += kComposeThreads) a.hist[(size_t)p * KK + i] = h[i];
}

__global__ void argmax_finalize_kernel(const unsigned long long* best, int64_t* out) {
  const unsigned long long b = *best;
  *out = (b == 0ull) ? -1 : (int64_t)(0xFFFFFFFFu - (uint32_t)(b & 0xFFFFFFFFull));
}

template <bool kVar, bool kRot>
cudaError_t launch_eval_t(const GridConst& gc, const EvalArgs& a, int n_ctas, size_t smem, cudaStream_t s) {
  cudaError_t e =
      cudaFuncSetAttribute(eval_kernel<kVar, kRot>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(redo_kernel<kVar, kRot>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  eval_kernel<kVar, kRot><<<n_ctas, kThreads, smem, s>>>(gc, a);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  redo_kernel<kVar, kRot><<<n_ctas, kThreads, smem, s>>>(gc, a);
  return cudaGetLastError();
}

}  // namespace

int eval_tile_points() { return kTile; }
int eval_min_tiles() { return kStages; }

size_t eval_smem_bytes(int K, int table_slots) { return eval_smem_layout(K, table_slots, nullptr, nullptr); }

int eval_table_slots_for(int K, size_t smem_budget) {
  int lo = 32;
  while (eval_smem_bytes(K, lo + 32) <= smem_budget && lo < (1 << 16)) lo += 32;
  return lo;
}

cudaError_t launch_eval(const GridConst& gc, const EvalArgs& a, int n_ctas, bool rotate, cudaStream_t s) {
  const size_t smem = eval_smem_bytes(gc.K, a.table_slots);
  const bool var = !(gc.feature == 0 && a.dump == nullptr);  // the count feature needs no z sums
  if (var)
    return rotate ? launch_eval_t<true, true>(gc, a, n_ctas, smem, s)
                  : launch_eval_t<true, false>(gc, a, n_ctas, smem, s);
  return rotate ? launch_eval_t<false, true>(gc, a, n_ctas, smem, s)
                : launch_eval_t<false, false>(gc, a, n_ctas, smem, s);
}

cudaError_t launch_pack_points(const float* xyz, int64_t n, int64_t n_out, const float* rots, int n_rot, float4* out,
                               cudaStream_t s) {
  const int threads = 256;
  int64_t bx = (n_out + threads - 1) / threads;
  if (bx > 2048) bx = 2048;
  if (bx < 1) bx = 1;
  dim3 grid((unsigned)bx, (unsigned)(rots != nullptr && n_rot > 0 ? n_rot : 1));
  pack_points_kernel<<<grid, threads, 0, s>>>(xyz, n, n_out, rots, out);
  return cudaGetLastError();
}

cudaError_t launch_compose(const GridConst& gc, const ComposeArgs& a, cudaStream_t s) {
  if (a.P <= 0) return cudaSuccess;
  compose_kernel<<<a.P, kComposeThreads, 0, s>>>(gc, a);
  return cudaGetLastError();
}

cudaError_t launch_argmax_finalize(const unsigned long long* best, int64_t* out, cudaStream_t s) {
  argmax_finalize_kernel<<<1, 1, 0, s>>>(best, out);
  return cudaGetLastError();
}

}  // namespace mialign
