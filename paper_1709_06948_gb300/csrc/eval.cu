// eval.cu — the pose-batched MI hot path (arXiv 1709.06948, Algorithm 1 loop body for
// a whole batch of candidate poses; Sec. III-A features; Eqs. 1-5).
//
// eval_kernel: persistent, one CTA per SM, one pose at a time per CTA.  Scan B is
// streamed through shared memory in tiles by 1-D bulk (TMA) copies on a cyclic
// multi-stage mbarrier pipeline.  For every point and the CTA's current pose the warp
// computes the voxel key and dz (device_common.cuh), collapses runs of equal keys
// among its 32 consecutive points with a segmented shuffle scan, and the run's last
// lane adds (n, S1, S2) into a shared-memory open-addressing hash table with 32-bit
// shared atomics.  After the sweep the table holds the pose's occupied B voxels; one
// pass over it yields the feature symbols, B's occupied bbox and the partial joint
// histogram c[a][b >= 1] of the occupied voxels inside A's bbox.
//  - If a pose occupies more voxels than the table holds, the pose restarts with the
//    keys split into 2, 4, ... disjoint hash partitions swept one after another.
//  - A voxel holding more points than the 32-bit sums allow diverts its later runs to
//    64-bit side sums in global memory (per CTA, indexed by table slot).
// compose_kernel: per pose, the overlap box (Algorithm 1), A's symbol counts over it
// from per-symbol prefix sums, the phi column h[a][0], then Eqs. 2-5 in FP32 with a
// fixed reduction order, and the packed (MI, index) maximum for Eq. 1.
#include <climits>

#include "align_internal.h"
#include "device_common.cuh"

namespace mialign {

namespace {

constexpr int kThreads = 512;
constexpr int kWarps = kThreads / 32;
constexpr int kPPT = 2;                       // points per thread per tile
constexpr int kTile = kThreads * kPPT;        // points per tile
constexpr uint32_t kTileBytes = kTile * 12u;  // fp32 xyz
constexpr int kStages = 4;
constexpr int kMaxPasses = 1 << 16;
constexpr uint32_t kFull = 0xFFFFFFFFu;

__host__ __device__ constexpr int round4(int x) { return (x + 3) & ~3; }

struct EvalSmem {
  float* tiles;
  uint32_t* tkey;
  uint32_t* tcnt;
  int32_t* ts1;
  uint32_t* ts2;
  uint32_t* hist;
  uint32_t* ct;
  int64_t* vt;
  uint64_t* mbar;      // [0, kStages): full, [kStages, 2 kStages): empty
  uint32_t* issue_cnt; // kStages
  int32_t* box;        // 6
  uint32_t* flags;     // fill, overflow, abort, wide
};

__host__ __device__ inline size_t eval_smem_layout(int K, int T, EvalSmem* s, uint8_t* base) {
  size_t off = 0;
  auto take = [&](size_t bytes, size_t align) {
    off = (off + align - 1) / align * align;
    size_t o = off;
    off += bytes;
    return o;
  };
  size_t o_tiles = take((size_t)kStages * kTileBytes, 128);
  size_t o_key = take((size_t)T * 4, 16);
  size_t o_cnt = take((size_t)T * 4, 16);
  size_t o_s1 = take((size_t)T * 4, 16);
  size_t o_s2 = take((size_t)T * 4, 16);
  size_t o_hist = take((size_t)round4(K * K) * 4, 16);
  size_t o_ct = take(kMaxLevels * 4 + 4, 16);
  size_t o_vt = take(kMaxLevels * 8 + 8, 16);
  size_t o_mbar = take(2 * kStages * 8, 8);
  size_t o_issue = take(kStages * 4, 4);
  size_t o_box = take(6 * 4, 4);
  size_t o_flags = take(4 * 4, 4);
  if (s) {
    s->tiles = (float*)(base + o_tiles);
    s->tkey = (uint32_t*)(base + o_key);
    s->tcnt = (uint32_t*)(base + o_cnt);
    s->ts1 = (int32_t*)(base + o_s1);
    s->ts2 = (uint32_t*)(base + o_s2);
    s->hist = (uint32_t*)(base + o_hist);
    s->ct = (uint32_t*)(base + o_ct);
    s->vt = (int64_t*)(base + o_vt);
    s->mbar = (uint64_t*)(base + o_mbar);
    s->issue_cnt = (uint32_t*)(base + o_issue);
    s->box = (int32_t*)(base + o_box);
    s->flags = (uint32_t*)(base + o_flags);
  }
  return off;
}

// Issue the bulk copy of consumption slot q (cyclic over the tiles).
__device__ __forceinline__ void issue_tile(const EvalSmem& S, const EvalArgs& a, uint32_t q) {
  const uint32_t b = q % kStages;
  const uint32_t tile = q % (uint32_t)a.n_tiles;
  const uint32_t full = smem_addr(&S.mbar[b]);
  mbar_arrive_expect_tx(full, kTileBytes);
  bulk_copy_g2s(smem_addr(S.tiles + (size_t)b * kTile * 3), a.xyz + (size_t)tile * kTile * 3, kTileBytes, full);
}

// Find or insert `key` in the open-addressing table (linear probing, bounded by T probes).
// A full table flags the pose for a restart with more key partitions.
__device__ __forceinline__ int table_slot(const EvalSmem& S, uint32_t key, int T) {
  uint32_t h = __umulhi(key * 0x9E3779B1u, (uint32_t)T);
  volatile uint32_t* vkey = S.tkey;
  for (int i = 0; i < T; ++i) {
    const uint32_t k = vkey[h];
    if (k == key) return (int)h;
    if (k == kEmptyKey) {
      const uint32_t old = atomicCAS(&S.tkey[h], kEmptyKey, key);
      if (old == kEmptyKey || old == key) return (int)h;
    }
    h = (h + 1 == (uint32_t)T) ? 0u : h + 1;
  }
  S.flags[1] = 1u;
  return -1;
}

// One warp row of 32 consecutive points: collapse runs of equal keys, then the run's
// last lane adds the run's (n, S1, S2) into the table.
template <bool kVar>
__device__ __forceinline__ void commit_row(const EvalSmem& S, const GridConst& gc, const EvalArgs& a,
                                           unsigned long long* wide, uint32_t key, int dz, int lane, int T) {
  const uint32_t valid = __ballot_sync(kFull, key != kEmptyKey);
  if (valid == 0u) return;
  const uint32_t prev = __shfl_up_sync(kFull, key, 1);
  const bool head = (lane == 0) || (key != prev);
  const uint32_t hm = __ballot_sync(kFull, head);
  const bool tail = ((((hm >> 1) | 0x80000000u) >> lane) & 1u) != 0u;
  const int hl = 31 - __clz(hm & (kFull >> (31 - lane)));
  const int d = lane - hl;
  int a1 = dz;
  uint32_t a2 = (uint32_t)(dz * dz);
  if (kVar) {
    const int maxd = (int)__reduce_max_sync(kFull, (uint32_t)d);
    for (int off = 1; off <= maxd; off <<= 1) {
      const int t1 = __shfl_up_sync(kFull, a1, off);
      const uint32_t t2 = __shfl_up_sync(kFull, a2, off);
      if (d >= off) {
        a1 += t1;
        a2 += t2;
      }
    }
  }
  if (tail && key != kEmptyKey) {
    if (*(volatile uint32_t*)&S.flags[1]) return;  // pose restarts anyway
    const int slot = table_slot(S, key, T);
    if (slot < 0) return;
    const uint32_t n = (uint32_t)(d + 1);
    if (kVar) {
      const uint32_t old = atomicAdd(&S.tcnt[slot], n);
      if (old + n <= gc.nlim) {
        atomicAdd(&S.ts1[slot], a1);
        atomicAdd(&S.ts2[slot], a2);
      } else {
        atomicAdd(&wide[2 * slot], (unsigned long long)(long long)a1);
        atomicAdd(&wide[2 * slot + 1], (unsigned long long)a2);
        S.flags[3] = 1u;
      }
    } else {
      atomicAdd(&S.tcnt[slot], n);
    }
  }
}

template <bool kVar>
__global__ void __launch_bounds__(kThreads, 1) eval_kernel(const GridConst gc, const EvalArgs a) {
  extern __shared__ __align__(128) uint8_t smem_raw[];
  EvalSmem S;
  const int T = a.table_slots;
  const int K = gc.K, KK = K * K;
  eval_smem_layout(K, T, &S, smem_raw);
  const int tid = threadIdx.x, lane = tid & 31;
  const uint32_t cap = (uint32_t)T - (uint32_t)T / 4u;  // 75% load factor
  unsigned long long* wide = a.wide + (size_t)blockIdx.x * 2u * (size_t)T;

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
    for (int b = 0; b < kStages; ++b) {
      mbar_init(smem_addr(&S.mbar[b]), 1u);
      mbar_init(smem_addr(&S.mbar[kStages + b]), (uint32_t)kWarps);
      S.issue_cnt[b] = 0u;
    }
    S.box[0] = S.box[1] = S.box[2] = INT_MAX;
    S.box[3] = S.box[4] = S.box[5] = INT_MIN;
    S.flags[0] = S.flags[1] = S.flags[2] = S.flags[3] = 0u;
    fence_mbar_init();
  }
  __syncthreads();
  if (tid == 0)
    for (int b = 0; b < kStages; ++b) issue_tile(S, a, (uint32_t)b);

  uint32_t q = 0;  // consumption counter, identical in every warp
  int passes = a.passes0;
  bool aborted = false;

  for (int p = blockIdx.x; p < a.P && !aborted; p += gridDim.x) {
    Pose12 P;
#pragma unroll
    for (int i = 0; i < 9; ++i) P.r[i] = __ldg(a.poses + 12 * (size_t)p + i);
#pragma unroll
    for (int i = 0; i < 3; ++i) P.t[i] = __ldg(a.poses + 12 * (size_t)p + 9 + i);

    int pass = 0;
    while (pass < passes) {
      const int lg = __ffs(passes) - 1;
      // ---- sweep all tiles of B for this pose (and key partition) ----
      for (int t = 0; t < a.n_tiles; ++t, ++q) {
        const uint32_t b = q % kStages;
        const uint32_t par = (q / kStages) & 1u;
        if (*(volatile uint32_t*)&S.flags[2]) continue;  // aborting: no more waits
        if (!mbar_wait_bounded(smem_addr(&S.mbar[b]), par, kWaitLimitNs)) {
          atomicOr(a.err, kErrWaitTimeout);
          S.flags[2] = 1u;
          continue;
        }
        const float* tile = S.tiles + (size_t)b * kTile * 3;
        const int base = t * kTile;
#pragma unroll
        for (int j = 0; j < kPPT; ++j) {
          const int li = j * kThreads + tid;
          uint32_t key = kEmptyKey;
          int dz = 0;
          if (base + li < a.n_points) {
            key = voxel_key(P, tile[3 * li], tile[3 * li + 1], tile[3 * li + 2], gc.inv_res, gc.X, gc.Y, gc.Z,
                            gc.res_mm, &dz);
            if (key != kEmptyKey) {
              if ((uint32_t)(dz + gc.dz_bound) > (uint32_t)(2 * gc.dz_bound)) atomicOr(a.err, kErrDzBound);
              if (lg > 0 && ((key * 0x85EBCA77u) >> (32 - lg)) != (uint32_t)pass) key = kEmptyKey;
            }
          }
          commit_row<kVar>(S, gc, a, wide, key, dz, lane, T);
        }
        __syncwarp();
        if (lane == 0) {
          mbar_arrive(smem_addr(&S.mbar[kStages + b]));
          const uint32_t c = atomicAdd(&S.issue_cnt[b], 1u);
          if (c == (uint32_t)kWarps - 1u) {  // last warp done with this buffer refills it
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
      __syncthreads();
      if (S.flags[2]) {
        aborted = true;
        break;
      }
      const bool overflow = S.flags[1] != 0u;
      // ---- read (and clear) the table ----
      int mn0 = INT_MAX, mn1 = INT_MAX, mn2 = INT_MAX, mx0 = INT_MIN, mx1 = INT_MIN, mx2 = INT_MIN;
      uint32_t occupied = 0;
      for (int s = tid; s < T; s += kThreads) {
        const uint32_t k = S.tkey[s];
        if (k == kEmptyKey) continue;
        ++occupied;
        const uint64_t n = S.tcnt[s];
        int64_t s1 = S.ts1[s];
        uint64_t s2 = S.ts2[s];
        if (kVar && n > gc.nlim) {
          s1 += (int64_t)wide[2 * s];
          s2 += wide[2 * s + 1];
          wide[2 * s] = 0ull;
          wide[2 * s + 1] = 0ull;
          if (!overflow) atomicAdd(a.wide_count, 1u);
        }
        S.tkey[s] = kEmptyKey;
        S.tcnt[s] = 0u;
        S.ts1[s] = 0;
        S.ts2[s] = 0u;
        if (overflow) continue;
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
      if (lane == 0 && !overflow && mn0 != INT_MAX) {
        atomicMin(&S.box[0], mn0); atomicMin(&S.box[1], mn1); atomicMin(&S.box[2], mn2);
        atomicMax(&S.box[3], mx0); atomicMax(&S.box[4], mx1); atomicMax(&S.box[5], mx2);
      }
      __syncthreads();
      if (overflow) {
        // restart this pose with twice as many key partitions
        for (int i = tid; i < KK; i += kThreads) S.hist[i] = 0u;
        if (tid == 0) {
          S.box[0] = S.box[1] = S.box[2] = INT_MAX;
          S.box[3] = S.box[4] = S.box[5] = INT_MIN;
          S.flags[0] = 0u;
          S.flags[1] = 0u;
        }
        if (passes >= kMaxPasses) {
          if (tid == 0) atomicOr(a.err, kErrPassLimit);
          aborted = true;
          __syncthreads();
          break;
        }
        passes *= 2;
        pass = 0;
        __syncthreads();
        continue;
      }
      // a table filled beyond 3/4 probes slowly: sweep the following poses in more partitions
      const bool crowded = S.flags[0] > cap;
      __syncthreads();
      if (tid == 0) S.flags[0] = 0u;
      if (crowded && passes < kMaxPasses) {
        passes *= 2;
        pass = 2 * pass + 2;  // the partitions already swept are split in two; continue after them
      } else {
        ++pass;
      }
      __syncthreads();
    }
    if (aborted) break;
    // ---- this pose's partial histogram and B bbox ----
    uint32_t* oc = a.out_c + (size_t)p * KK;
    for (int i = tid; i < KK; i += kThreads) {
      oc[i] = S.hist[i];
      S.hist[i] = 0u;
    }
    if (tid < 6) a.out_box[6 * (size_t)p + tid] = S.box[tid];
    __syncthreads();
    if (tid < 6) S.box[tid] = tid < 3 ? INT_MAX : INT_MIN;
  }

  // Drain the prefetched tiles still in flight before the CTA's shared memory is released.
  __syncthreads();
  if (tid == 0) {
    if (!aborted) atomicMax(a.max_passes, (uint32_t)passes);
    for (int i = 0; i < kStages; ++i) {
      const uint32_t qq = q + (uint32_t)i;
      if (!mbar_wait_bounded(smem_addr(&S.mbar[qq % kStages]), (qq / kStages) & 1u, kWaitLimitNs))
        atomicOr(a.err, kErrWaitTimeout);
    }
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

}  // namespace

int eval_tile_points() { return kTile; }

size_t eval_smem_bytes(int K, int table_slots) { return eval_smem_layout(K, table_slots, nullptr, nullptr); }

int eval_table_slots_for(int K, size_t smem_budget) {
  // largest multiple of 32 slots that fits the budget
  int lo = 32, hi = 1 << 16;
  while (lo < hi) {
    int mid = ((lo + hi + 1) / 2) & ~31;
    if (mid <= lo) break;
    if (eval_smem_bytes(K, mid) <= smem_budget) lo = mid;
    else hi = mid - 1;
  }
  while (eval_smem_bytes(K, lo) > smem_budget && lo > 32) lo -= 32;
  return lo;
}

cudaError_t launch_eval(const GridConst& gc, const EvalArgs& a, int n_ctas, cudaStream_t s) {
  const size_t smem = eval_smem_bytes(gc.K, a.table_slots);
  cudaError_t e;
  if (gc.feature == 0 && a.dump == nullptr) {  // the count feature needs no z sums
    e = cudaFuncSetAttribute(eval_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    eval_kernel<false><<<n_ctas, kThreads, smem, s>>>(gc, a);
  } else {
    e = cudaFuncSetAttribute(eval_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    eval_kernel<true><<<n_ctas, kThreads, smem, s>>>(gc, a);
  }
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
