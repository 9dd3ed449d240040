// eval.cu — the pose-batched MI hot path (arXiv 1709.06948, Algorithm 1 loop body for
// whole batches of candidate poses of one or more scan pairs; Sec. III-A features; Eqs. 1-5).
//
// pack_points_kernel: scan B as float4 tiles, either raw xyz (NaN padding) or one
// pre-rotated copy u = R p per distinct rotation of the batch (+inf padding; a search
// lattice has 32 rotations for 4,096 poses, so the 9-FMA rotation leaves the per-pose
// loop).  The tiles are laid out as kThreads streams: thread s of a CTA reads, tile after
// tile, the points s*L, s*L+1, ... of B's given order (L = kPPT * tiles), so each thread
// walks a stretch of consecutive scan points (stream_of: which stream a thread walks).
//
// eval_kernel: persistent, one CTA per SM, one pose at a time per CTA; a launch covers the
// poses of one scan pair (grid constants in the kernel parameters) or, in the multi-pair
// mode, of several pairs, each pose bringing its pair's constants.  Every thread streams
// its own points straight from L2, four tiles ahead, computes the voxel keys and z
// offsets of the buffered tiles, then keeps the run of equal keys it is walking in
// registers (the table layout's value words: n and the z sums).  Finished runs go to a
// per-warp ring in shared memory; 32 at a time the whole warp adds them into a
// shared-memory open-addressing hash table (buckets of 4 keys, 32-bit shared atomics).
// After the sweep one pass over the table gives the feature symbols, B's occupied bbox
// and the partial joint histogram c[a][b >= 1] of the occupied voxels inside A's bbox.
//  - A pose with more occupied voxels than fit the table, or with a voxel so full that
//    its table sums may have wrapped, is finished by redo_kernel: plain sweeps with the
//    keys split into 2, 4, ... hash partitions, each run added at once, the plain count in
//    the table and S1, S2 in 64-bit sums in global memory.  A crowded table makes the CTA
//    sweep its following poses in twice as many partitions.
//  - Key partitions: a pose whose voxels do not fit the table keeps the keys of one hash
//    partition per pass.  With spill queues (eval_kernel<..., kSp>) B is swept once, every
//    run is appended to its partition's queue in device memory, and each pass inserts one
//    queue; otherwise every pass sweeps B and drops the other partitions' keys.
//
// eval_pair_kernel: two poses that read the same tile copy and differ only in t'_x, swept
// together over one table (one point load and one y/z half of the voxel map for both).
// eval_cluster_kernel: one pose per 2-CTA cluster, its table split between the two CTAs'
// shared memories (distributed shared memory).
//
// compose_kernel: per pose, the overlap box (Algorithm 1), A's symbol counts over it from
// per-symbol prefix sums, the phi column h[a][0], then Eqs. 2-5 in FP32 with a fixed
// reduction order, and the packed (MI, index) maximum for Eq. 1.
#include <algorithm>
#include <climits>
#include <mutex>

#include "align_internal.h"
#include "device_common.cuh"

// The shape this translation unit is compiled for (see EvalKernels).
#ifndef MI_EVAL_THREADS
#define MI_EVAL_THREADS 1024
#endif
#ifndef MI_EVAL_PPT
#define MI_EVAL_PPT 1
#endif
#ifndef MI_EVAL_CTAS_PER_SM
#define MI_EVAL_CTAS_PER_SM 1
#endif
#ifndef MI_EVAL_SHAPE_FN
#define MI_EVAL_SHAPE_FN eval_shape_1024x1
#endif
#define MI_STR2(x) #x
#define MI_STR(x) MI_STR2(x)

namespace mialign {

namespace {

constexpr int kThreads = MI_EVAL_THREADS;
constexpr int kCtasPerSm = MI_EVAL_CTAS_PER_SM;
constexpr int kWarps = kThreads / 32;
constexpr int kPPT = MI_EVAL_PPT;       // points per thread per tile
constexpr int kTile = kThreads * kPPT;  // points per tile
#ifndef MI_EVAL_DEPTH
#define MI_EVAL_DEPTH 4
#endif
constexpr int kDepth = MI_EVAL_DEPTH;   // tiles loaded ahead into registers
#ifndef MI_EVAL_PAIR_DEPTH
#define MI_EVAL_PAIR_DEPTH (MI_EVAL_PPT >= 2 ? 1 : 2)
#endif
constexpr int kPairDepth = MI_EVAL_PAIR_DEPTH;  // the same for the pose-pair sweep (two runs per thread)
constexpr int kMinTiles = 3;
constexpr uint32_t kQueue = 64;         // finished runs buffered per warp (32 drained at a time)
constexpr int kProbeBuckets = 1024;     // probe budget per key (buckets of 4 slots)
constexpr int kOvfCap = 16384;          // overflow list entries per CTA
constexpr int kMaxPasses = 1 << 16;
constexpr uint32_t kFull = 0xFFFFFFFFu;
constexpr int kGcWords = (int)(sizeof(GridConst) / 4);

__host__ __device__ constexpr int round4(int x) { return (x + 3) & ~3; }

// ---------------------------------------------------------------------------------
// Shared memory by 32-bit shared-window address (explicit ld/st/red/atom.shared).
// ---------------------------------------------------------------------------------
__device__ __forceinline__ uint32_t lds32(uint32_t a) {
  uint32_t v;
  asm volatile("ld.shared.u32 %0, [%1];" : "=r"(v) : "r"(a) : "memory");
  return v;
}
__device__ __forceinline__ void sts32(uint32_t a, uint32_t v) {
  asm volatile("st.shared.u32 [%0], %1;" ::"r"(a), "r"(v) : "memory");
}
__device__ __forceinline__ uint4 lds128(uint32_t a) {
  uint4 v;
  asm volatile("ld.shared.v4.u32 {%0, %1, %2, %3}, [%4];"
               : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
               : "r"(a)
               : "memory");
  return v;
}
__device__ __forceinline__ void sts128(uint32_t a, uint4 v) {
  asm volatile("st.shared.v4.u32 [%0], {%1, %2, %3, %4};" ::"r"(a), "r"(v.x), "r"(v.y), "r"(v.z), "r"(v.w)
               : "memory");
}
// st.shared.v4 under a predicate (no branch around the store).
__device__ __forceinline__ void sts128_if(bool p, uint32_t a, uint4 v) {
  asm volatile(
      "{\n\t.reg .pred q;\n\tsetp.ne.u32 q, %0, 0;\n\t@q st.shared.v4.u32 [%1], {%2, %3, %4, %5};\n\t}" ::"r"(
          (uint32_t)p),
      "r"(a), "r"(v.x), "r"(v.y), "r"(v.z), "r"(v.w)
      : "memory");
}
__device__ __forceinline__ void sts32_if(bool p, uint32_t a, uint32_t v) {
  asm volatile("{\n\t.reg .pred q;\n\tsetp.ne.u32 q, %0, 0;\n\t@q st.shared.u32 [%1], %2;\n\t}" ::"r"((uint32_t)p),
               "r"(a), "r"(v)
               : "memory");
}
__device__ __forceinline__ void red_add_if(bool p, uint32_t a, uint32_t v) {
  asm volatile("{\n\t.reg .pred q;\n\tsetp.ne.u32 q, %0, 0;\n\t@q red.shared.add.u32 [%1], %2;\n\t}" ::"r"(
                   (uint32_t)p),
               "r"(a), "r"(v)
               : "memory");
}
// Shared atomic add under a predicate; returns 0 when not executed.
__device__ __forceinline__ uint32_t atom_add_if(bool p, uint32_t a, uint32_t v) {
  uint32_t old;
  asm volatile(
      "{\n\t.reg .pred q;\n\tsetp.ne.u32 q, %1, 0;\n\tmov.u32 %0, 0;\n\t@q atom.shared.add.u32 %0, [%2], %3;\n\t}"
      : "=r"(old)
      : "r"((uint32_t)p), "r"(a), "r"(v)
      : "memory");
  return old;
}
// 16-byte global store under a predicate.
__device__ __forceinline__ void stg128_if(bool p, uint4* g, uint4 v) {
  asm volatile("{\n\t.reg .pred q;\n\tsetp.ne.u32 q, %0, 0;\n\t@q st.global.v4.u32 [%1], {%2, %3, %4, %5};\n\t}" ::"r"(
                   (uint32_t)p),
               "l"(g), "r"(v.x), "r"(v.y), "r"(v.z), "r"(v.w)
               : "memory");
}
// CAS under a predicate; returns `cmp` when not executed.
__device__ __forceinline__ uint32_t atom_cas_if(bool p, uint32_t a, uint32_t cmp, uint32_t v) {
  uint32_t old;
  asm volatile(
      "{\n\t.reg .pred q;\n\tsetp.ne.u32 q, %1, 0;\n\tmov.u32 %0, %3;\n\t@q atom.shared.cas.b32 %0, [%2], %3, %4;\n\t}"
      : "=r"(old)
      : "r"((uint32_t)p), "r"(a), "r"(cmp), "r"(v)
      : "memory");
  return old;
}
__device__ __forceinline__ void red_add(uint32_t a, uint32_t v) {
  asm volatile("red.shared.add.u32 [%0], %1;" ::"r"(a), "r"(v) : "memory");
}
__device__ __forceinline__ uint32_t atom_add(uint32_t a, uint32_t v) {
  uint32_t old;
  asm volatile("atom.shared.add.u32 %0, [%1], %2;" : "=r"(old) : "r"(a), "r"(v) : "memory");
  return old;
}
__device__ __forceinline__ uint32_t atom_cas(uint32_t a, uint32_t cmp, uint32_t v) {
  uint32_t old;
  asm volatile("atom.shared.cas.b32 %0, [%1], %2, %3;" : "=r"(old) : "r"(a), "r"(cmp), "r"(v) : "memory");
  return old;
}
__device__ __forceinline__ void red_min_s32(uint32_t a, int v) {
  asm volatile("red.shared.min.s32 [%0], %1;" ::"r"(a), "r"(v) : "memory");
}
__device__ __forceinline__ void red_max_s32(uint32_t a, int v) {
  asm volatile("red.shared.max.s32 [%0], %1;" ::"r"(a), "r"(v) : "memory");
}
__device__ __forceinline__ uint32_t lane_mask_lt() {
  uint32_t m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

// ---------------------------------------------------------------------------------
// Thread-block clusters (the cluster kernel): rank, the distributed shared-memory window
// (.shared::cluster addresses of either CTA's shared memory) and the cluster barrier.
// ---------------------------------------------------------------------------------
__device__ __forceinline__ uint32_t cluster_rank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
// All threads of every CTA of the cluster; release/acquire: shared-memory writes before it
// are visible to the other CTA after it.
__device__ __forceinline__ void cluster_sync() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}
// The .shared::cluster address of shared-window address `a` of CTA `rank` of the cluster.
__device__ __forceinline__ uint32_t map_cluster(uint32_t a, uint32_t rank) {
  uint32_t d;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(d) : "r"(a), "r"(rank));
  return d;
}
__device__ __forceinline__ uint32_t ldc32(uint32_t a) {
  uint32_t v;
  asm volatile("ld.shared::cluster.u32 %0, [%1];" : "=r"(v) : "r"(a) : "memory");
  return v;
}
__device__ __forceinline__ uint4 ldc128(uint32_t a) {
  uint4 v;
  asm volatile("ld.shared::cluster.v4.u32 {%0, %1, %2, %3}, [%4];"
               : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
               : "r"(a)
               : "memory");
  return v;
}
__device__ __forceinline__ uint32_t atomc_cas(uint32_t a, uint32_t cmp, uint32_t v) {
  uint32_t old;
  asm volatile("atom.shared::cluster.cas.b32 %0, [%1], %2, %3;" : "=r"(old) : "r"(a), "r"(cmp), "r"(v) : "memory");
  return old;
}
__device__ __forceinline__ uint32_t atomc_add(uint32_t a, uint32_t v) {
  uint32_t old;
  asm volatile("atom.shared::cluster.add.u32 %0, [%1], %2;" : "=r"(old) : "r"(a), "r"(v) : "memory");
  return old;
}
__device__ __forceinline__ void redc_add(uint32_t a, uint32_t v) {
  asm volatile("red.shared::cluster.add.u32 [%0], %1;" ::"r"(a), "r"(v) : "memory");
}
__device__ __forceinline__ void redc_min_s32(uint32_t a, int v) {
  asm volatile("red.shared::cluster.min.s32 [%0], %1;" ::"r"(a), "r"(v) : "memory");
}
__device__ __forceinline__ void redc_max_s32(uint32_t a, int v) {
  asm volatile("red.shared::cluster.max.s32 [%0], %1;" ::"r"(a), "r"(v) : "memory");
}
__device__ __forceinline__ uint32_t atomc_cas_if(bool p, uint32_t a, uint32_t cmp, uint32_t v) {
  uint32_t old;
  asm volatile(
      "{\n\t.reg .pred q;\n\tsetp.ne.u32 q, %1, 0;\n\tmov.u32 %0, %3;\n\t@q atom.shared::cluster.cas.b32 %0, [%2], "
      "%3, %4;\n\t}"
      : "=r"(old)
      : "r"((uint32_t)p), "r"(a), "r"(cmp), "r"(v)
      : "memory");
  return old;
}
__device__ __forceinline__ uint32_t atomc_add_if(bool p, uint32_t a, uint32_t v) {
  uint32_t old;
  asm volatile(
      "{\n\t.reg .pred q;\n\tsetp.ne.u32 q, %1, 0;\n\tmov.u32 %0, 0;\n\t@q atom.shared::cluster.add.u32 %0, [%2], "
      "%3;\n\t}"
      : "=r"(old)
      : "r"((uint32_t)p), "r"(a), "r"(v)
      : "memory");
  return old;
}
__device__ __forceinline__ void redc_add_if(bool p, uint32_t a, uint32_t v) {
  asm volatile("{\n\t.reg .pred q;\n\tsetp.ne.u32 q, %0, 0;\n\t@q red.shared::cluster.add.u32 [%1], %2;\n\t}" ::"r"(
                   (uint32_t)p),
               "r"(a), "r"(v)
               : "memory");
}

// Layout: per-warp rings | flags (16 B) | table keys (T x 4 B) | table values (T x kVW
// words) | histogram | grid constants | bbox | current item.  The flags sit just below the
// keys so that the hot loop reaches them at a fixed offset from the key base.
//
// Table values, kVW words per slot (chosen per launch, see eval_layout):
//   1: n (no z sums: count feature);
//   2: W = n * 2^ns + S1' and S2, where S1' = sum(dz + dz_bound) >= 0 is the biased z sum
//      (S1 = S1' - n * dz_bound) and ns = GridConst::ns_shift.  While n <= nlim_pack the
//      biased sum stays below 2^ns, so W holds both exactly; a voxel that may pass nlim_pack
//      sends the pose to the exact path.  A third more slots than layout 3 in the same memory;
//   3: n, S1 (two's complement), S2; a voxel above nlim (the 32-bit sums may have wrapped)
//      sends the pose to the exact path.
// The exact path (redo_kernel) keeps the plain count in word 0 and S1, S2 in 64-bit sums in
// global memory.
struct EvalSmem {
  uint4* queue;       // per warp: kQueue finished runs (key, and the run's value words), a ring
  uint32_t* flags;    // occupied count, table full, overflow entries, sums need the exact path
  uint32_t* spill_cnt;  // runs spilled to each key partition's queue (eval_kernel, 8 words)
  uint32_t* tkey;
  uint32_t* tval;     // kVW words per slot
  uint32_t* hist;     // np partial histograms of hist_stride words
  GridConst* gc;      // the current item's grid constants
  int32_t* box;       // np x 6
  int32_t* item;      // the item whose constants are loaded
  uint32_t hist_stride;
  // shared-window addresses
  uint32_t a_queue, a_key, a_vals, a_hist, a_box, a_spill;
  // the cluster kernel: this CTA's rank and the .shared::cluster address of a_key in each
  // CTA of the pair (both CTAs have the same layout, so any table address maps by offset)
  uint32_t rank, c_key[2];
};
// The CTA of a 2-CTA cluster whose half of the distributed table holds `key`.
__device__ __forceinline__ uint32_t key_owner(uint32_t key) { return (key * 0xD6E8FEB9u) >> 31; }
constexpr uint32_t kFlagOccupied = 16u;  // byte offsets of the flags below a_key
constexpr uint32_t kFlagFull = 12u;
constexpr uint32_t kFlagOvf = 8u;        // entries in the CTA's overflow list
constexpr uint32_t kFlagWide = 4u;

// np: poses swept together (1, or 2 for a pose pair): one partial histogram and one bbox each.
__host__ __device__ inline size_t eval_smem_layout(int K, int T, int vw, int np, EvalSmem* s, uint8_t* base) {
  size_t off = 0;
  auto take = [&](size_t bytes, size_t align) {
    off = (off + align - 1) / align * align;
    size_t o = off;
    off += bytes;
    return o;
  };
  size_t o_queue = take((size_t)kWarps * kQueue * 16, 16);
  size_t o_spill = take(32, 16);
  size_t o_flags = take(16, 16);  // directly below the keys: addressed as a_key - kFlag*
  size_t o_key = take((size_t)T * 4, 16);
  size_t o_vals = take((size_t)T * 4 * vw, 16);
  size_t o_hist = take((size_t)np * round4(K * K) * 4, 16);
  size_t o_gc = take(sizeof(GridConst), 16);
  size_t o_box = take((size_t)np * 6 * 4, 4);
  size_t o_item = take(4, 4);
  if (s) {
    s->queue = (uint4*)(base + o_queue);
    s->flags = (uint32_t*)(base + o_flags);
    s->spill_cnt = (uint32_t*)(base + o_spill);
    s->tkey = (uint32_t*)(base + o_key);
    s->tval = (uint32_t*)(base + o_vals);
    s->hist = (uint32_t*)(base + o_hist);
    s->gc = (GridConst*)(base + o_gc);
    s->box = (int32_t*)(base + o_box);
    s->item = (int32_t*)(base + o_item);
    s->hist_stride = (uint32_t)round4(K * K);
#ifdef __CUDA_ARCH__
    const uint32_t a0 = (uint32_t)__cvta_generic_to_shared(base);
    s->a_queue = a0 + (uint32_t)o_queue;
    s->a_key = a0 + (uint32_t)o_key;
    s->a_vals = a0 + (uint32_t)o_vals;
    s->a_hist = a0 + (uint32_t)o_hist;
    s->a_box = a0 + (uint32_t)o_box;
    s->a_spill = a0 + (uint32_t)o_spill;
#endif
  }
  return off;
}

// Per-pose constants of the voxel map, kept in registers.
struct VoxelConst {
  float inv_res;
  int X, Y, Z, res_mm, dz_bound;
  uint32_t nlim;        // largest n per voxel of the layout's table sums
  uint32_t winc;        // layout 2, per point: 2^ns + dz_bound (plus dz)
  uint32_t wide_shift;  // layout 2: ns + b with 2^(b+1) - 2 <= nlim_pack (the drains' bound)
  int zc;               // layout 3 sums dz - zc (zc = res_mm / 2; 0 in the other layouts)
};

template <int kVW>
__device__ __forceinline__ VoxelConst voxel_const(const GridConst& g) {
  const uint32_t nlim = kVW == 2 ? g.nlim_pack : kVW == 3 ? g.nlim3c : 0x7FFFFFFFu;
  return VoxelConst{g.inv_res, g.X, g.Y, g.Z, g.res_mm, g.dz_bound, nlim,
                    (1u << g.ns_shift) + (uint32_t)g.dz_bound, (uint32_t)g.wide_shift,
                    kVW == 3 ? g.res_mm / 2 : 0};
}

// The table: buckets of 4 key slots (one 16-byte load each).  With kTwo (the pair kernel,
// whose table holds two poses' voxels) it is two-choice ("d-left"): a key's
// candidate buckets are b1 in the left half and b2 in the right half of the table, and a new
// key goes to the one with fewer keys (b1 on a tie).  Slots of a bucket fill in order and
// never empty during a sweep, so a bucket's key count is the index of its first free slot,
// and two inserters of the same key can never settle in different buckets: an inserter
// places the key only in a slot that was empty when it read both buckets without finding
// the key, and it reads both before it chooses.  A key whose two buckets are full (or whose
// insert lost a race) goes to the overflow list; table_slot then places it by a linear probe
// that starts after b2, the same sequence for every inserter of that key.
__device__ __forceinline__ void table_buckets(uint32_t key, uint32_t nb, uint32_t& b1, uint32_t& b2) {
  const uint32_t half = nb >> 1;
  b1 = __umulhi(key * 0x9E3779B1u, half);
  b2 = half + __umulhi(key * 0xC2B2AE35u, nb - half);
}
// Lowest slot of bucket k4 holding `key` (-1: none), and the bucket's key count.
__device__ __forceinline__ int bucket_hit(const uint4& k4, uint32_t key) {
  return (k4.x == key) ? 0 : (k4.y == key) ? 1 : (k4.z == key) ? 2 : (k4.w == key) ? 3 : -1;
}
__device__ __forceinline__ uint32_t bucket_fill(const uint4& k4) {
  return (uint32_t)(k4.x != kEmptyKey) + (uint32_t)(k4.y != kEmptyKey) + (uint32_t)(k4.z != kEmptyKey) +
         (uint32_t)(k4.w != kEmptyKey);
}

// Find or insert `key` (any thread, after the sweep's drains): returns the slot, or -1 when
// kProbeBuckets buckets past b2 were searched in vain (the pose then counts as overflowing).
// kTwo == false: one candidate bucket per key over the whole table (the single-pose kernel,
// whose table is about a third full), linear probing from it when it is full.
__device__ __noinline__ int table_slot_slow(uint32_t a_key, uint32_t key, uint32_t nb, uint32_t b);
template <bool kTwo>
__device__ __forceinline__ int table_slot(const EvalSmem& S, uint32_t key, uint32_t nb) {
  if constexpr (!kTwo) {
    const uint32_t b = __umulhi(key * 0x9E3779B1u, nb);
    const uint4 k4 = lds128(S.a_key + 16u * b);
    const int h = bucket_hit(k4, key);
    if (h >= 0) return (int)(4 * b) + h;
    const uint32_t f = bucket_fill(k4);
    if (f < 4u) {
      const uint32_t s = 4 * b + f;
      const uint32_t old = atom_cas(S.a_key + 4u * s, kEmptyKey, key);
      if (old == kEmptyKey || old == key) return (int)s;
    }
    return table_slot_slow(S.a_key, key, nb, b);
  }
  uint32_t b1, b2;
  table_buckets(key, nb, b1, b2);
#pragma unroll 1
  for (int tries = 0; tries < 9; ++tries) {  // each lost race means one more key in b1 or b2
    const uint4 ka = lds128(S.a_key + 16u * b1);
    const uint4 kb = lds128(S.a_key + 16u * b2);
    const int ha = bucket_hit(ka, key), hb = bucket_hit(kb, key);
    if (ha >= 0) return (int)(4 * b1) + ha;
    if (hb >= 0) return (int)(4 * b2) + hb;
    const uint32_t fa = bucket_fill(ka), fb = bucket_fill(kb);
    if (fa == 4u && fb == 4u) break;  // both full: the key can never enter b1 or b2
    const uint32_t s = fa <= fb ? 4 * b1 + fa : 4 * b2 + fb;
    const uint32_t old = atom_cas(S.a_key + 4u * s, kEmptyKey, key);
    if (old == kEmptyKey || old == key) return (int)s;
  }
  return table_slot_slow(S.a_key, key, nb, b2 + 1 == nb ? 0u : b2 + 1);
}
__device__ __noinline__ int table_slot_slow(uint32_t a_key, uint32_t key, uint32_t nb, uint32_t b) {
#pragma unroll 1
  for (int i = 0; i < kProbeBuckets; ++i) {
    const uint4 k4 = lds128(a_key + 16u * b);
    const int h = bucket_hit(k4, key);
    if (h >= 0) return (int)(4 * b) + h;
    const uint32_t f = bucket_fill(k4);
    if (f < 4u) {
      const uint32_t s = 4 * b + f;
      const uint32_t old = atom_cas(a_key + 4u * s, kEmptyKey, key);
      if (old == kEmptyKey || old == key) return (int)s;
      continue;  // another thread took that slot: read the bucket again
    }
    b = (b + 1 == nb) ? 0u : b + 1;
  }
  return -1;
}

// Add one finished run (ring entry: key and the run's value words) to the table.  In the
// packed layout the packed word is added with an atomic that returns the old value, so that
// an add taking the voxel above nlim_pack flags the pose for the exact path.
template <int kVW>
__device__ __forceinline__ void table_add_slot(const EvalSmem& S, const uint4& e, int slot, const GridConst& gc) {
  const uint32_t v = S.a_vals + 4u * kVW * (uint32_t)slot;
  if (kVW == 2) {
    const uint32_t ns = (uint32_t)gc.ns_shift;
    const uint32_t old = atom_add(v, e.y);
    if ((old >> ns) + (e.y >> ns) > gc.nlim_pack) sts32(S.a_key - kFlagWide, 1u);
    red_add(v + 4u, e.z);
  } else {
    red_add(v, e.y);
    if (kVW == 3) {
      red_add(v + 4u, e.z);
      red_add(v + 8u, e.w);
    }
  }
}

// After a sweep: insert the overflow list with the full probe (all threads of the CTA).
template <int kVW, bool kTwo>
__device__ __forceinline__ void insert_overflow(const EvalSmem& S, const EvalArgs& a, const GridConst& gc) {
  const uint32_t n = min(*(volatile uint32_t*)&S.flags[2], (uint32_t)kOvfCap);
  const uint4* ovf = a.ovf + (size_t)blockIdx.x * kOvfCap;
  for (uint32_t i = threadIdx.x; i < n; i += kThreads) {
    const uint4 e = ovf[i];
    const int slot = table_slot<kTwo>(S, e.x, (uint32_t)a.n_buckets);
    if (slot < 0) sts32(S.a_key - kFlagFull, 1u);
    else table_add_slot<kVW>(S, e, slot, gc);
  }
}

// The same find-or-insert for the cluster kernel's distributed table (two-choice buckets in
// the owning CTA's half, addressed through the cluster window).  tb: the owner's key base.
__device__ __noinline__ int table_slot_slow_cl(uint32_t tb, uint32_t key, uint32_t nb, uint32_t b) {
#pragma unroll 1
  for (int i = 0; i < kProbeBuckets; ++i) {
    const uint4 k4 = ldc128(tb + 16u * b);
    const int h = bucket_hit(k4, key);
    if (h >= 0) return (int)(4 * b) + h;
    const uint32_t f = bucket_fill(k4);
    if (f < 4u) {
      const uint32_t s = 4 * b + f;
      const uint32_t old = atomc_cas(tb + 4u * s, kEmptyKey, key);
      if (old == kEmptyKey || old == key) return (int)s;
      continue;  // another thread took that slot: read the bucket again
    }
    b = (b + 1 == nb) ? 0u : b + 1;
  }
  return -1;
}
__device__ __forceinline__ int table_slot_cl(uint32_t tb, uint32_t key, uint32_t nb) {
  uint32_t b1, b2;
  table_buckets(key, nb, b1, b2);
#pragma unroll 1
  for (int tries = 0; tries < 9; ++tries) {  // each lost race means one more key in b1 or b2
    const uint4 ka = ldc128(tb + 16u * b1);
    const uint4 kb = ldc128(tb + 16u * b2);
    const int ha = bucket_hit(ka, key), hb = bucket_hit(kb, key);
    if (ha >= 0) return (int)(4 * b1) + ha;
    if (hb >= 0) return (int)(4 * b2) + hb;
    const uint32_t fa = bucket_fill(ka), fb = bucket_fill(kb);
    if (fa == 4u && fb == 4u) break;  // both full: the key can never enter b1 or b2
    const uint32_t s = fa <= fb ? 4 * b1 + fa : 4 * b2 + fb;
    const uint32_t old = atomc_cas(tb + 4u * s, kEmptyKey, key);
    if (old == kEmptyKey || old == key) return (int)s;
  }
  return table_slot_slow_cl(tb, key, nb, b2 + 1 == nb ? 0u : b2 + 1);
}

// Cluster kernel, after a sweep: insert this CTA's overflow list into the distributed table.
template <int kVW>
__device__ __forceinline__ void insert_overflow_cl(const EvalSmem& S, const EvalArgs& a, const GridConst& gc) {
  const uint32_t n = min(*(volatile uint32_t*)&S.flags[2], (uint32_t)kOvfCap);
  const uint4* ovf = a.ovf + (size_t)blockIdx.x * kOvfCap;
  for (uint32_t i = threadIdx.x; i < n; i += kThreads) {
    const uint4 e = ovf[i];
    const uint32_t tb = S.c_key[key_owner(e.x)];
    const int slot = table_slot_cl(tb, e.x, (uint32_t)a.n_buckets);
    if (slot < 0) {
      sts32(S.a_key - kFlagFull, 1u);
      continue;
    }
    const uint32_t v = tb + (S.a_vals - S.a_key) + 4u * kVW * (uint32_t)slot;
    if (kVW == 2) {
      const uint32_t ns = (uint32_t)gc.ns_shift;
      const uint32_t old = atomc_add(v, e.y);
      if ((old >> ns) + (e.y >> ns) > gc.nlim_pack) sts32(S.a_key - kFlagWide, 1u);
      redc_add(v + 4u, e.z);
    } else {
      redc_add(v, e.y);
      if (kVW == 3) {
        redc_add(v + 4u, e.z);
        redc_add(v + 8u, e.w);
      }
    }
  }
}

// Exact path (redo_kernel): add one run; the table keeps the plain count, S1 and S2 go to
// the CTA's 64-bit sums in global memory.
template <int kVW>
__device__ __forceinline__ void add_run(const EvalSmem& S, unsigned long long* wide, uint32_t key, uint32_t n,
                                        int s1, uint32_t s2, uint32_t nb) {
  if (lds32(S.a_key - kFlagFull)) return;  // table already full: the pose restarts
  const int slot = table_slot<false>(S, key, nb);
  if (slot < 0) {
    sts32(S.a_key - kFlagFull, 1u);
    return;
  }
  red_add(S.a_vals + 4u * kVW * (uint32_t)slot, n);
  if (kVW > 1) {
    atomicAdd(&wide[2 * slot], (unsigned long long)(long long)s1);
    atomicAdd(&wide[2 * slot + 1], (unsigned long long)s2);
  }
}

// The run of equal keys a thread is walking: w is the packed word (layout 2) or n, s1 and
// s2 the z sums (s1 only in layout 3).  Points outside the grid (or outside the current key
// partition) carry kEmptyKey and form runs of their own, which are dropped.
struct Run {
  uint32_t key;
  uint32_t w;
  uint32_t s1;  // two's complement
  uint32_t s2;
};

// The ring entry of a run: key, then the table's value words.
template <int kVW>
__device__ __forceinline__ uint4 run_entry(const Run& r) {
  return kVW == 3 ? make_uint4(r.key, r.w, r.s1, r.s2) : make_uint4(r.key, r.w, r.s2, 0u);
}

// Per-warp ring of finished runs in shared memory: lanes append what they finished at
// this step (compacted by a ballot); once 32 are waiting the whole warp adds entries
// 0..31 to the table and moves the rest down, so the ring never wraps.  The insert is
// written with predicated shared-memory operations so that the drain is one straight
// sequence; a run whose home bucket is full goes to the overflow list.
//
// Packed-word bound: `acc` ORs every old table word and every run word the lane added.
// While no n field in it reaches 2^b (2^(b+1) - 2 <= nlim), every add kept the voxel at or
// below nlim; the sweep's end tests acc once (the exact path takes the pose otherwise).
// kCount32: a drain of 32 entries (during the sweep); otherwise `count` (the last drain).
// One entry per lane (e.x == kEmptyKey: none) into the table; all 32 lanes take part.
template <int kVW, bool kTwo, bool kCl = false>
__device__ __forceinline__ void insert_entry(const EvalSmem& S, const EvalArgs& a, const uint4& e, uint32_t& acc) {
  const bool valid = e.x != kEmptyKey;
  // the table holding e.x: this CTA's, or (cluster kernel) the owning CTA's half of the
  // distributed table, addressed through the cluster window
  const uint32_t tb = kCl ? S.c_key[key_owner(e.x)] : S.a_key;  // keys
  const uint32_t vb = tb + (S.a_vals - S.a_key);                 // values
  int slot;
  uint32_t s_new;
  bool ins;
  if constexpr (kTwo) {
    uint32_t b1, b2;
    table_buckets(e.x, (uint32_t)a.n_buckets, b1, b2);
    const uint4 ka = kCl ? ldc128(tb + 16u * b1) : lds128(tb + 16u * b1);
    const uint4 kb = kCl ? ldc128(tb + 16u * b2) : lds128(tb + 16u * b2);
    const int ha = bucket_hit(ka, e.x), hb = bucket_hit(kb, e.x);
    const uint32_t fa = bucket_fill(ka), fb = bucket_fill(kb);
    slot = ha >= 0 ? (int)(4 * b1) + ha : hb >= 0 ? (int)(4 * b2) + hb : -1;
    // a new key: the emptier bucket's first free slot
    s_new = fa <= fb ? 4 * b1 + fa : 4 * b2 + fb;
    ins = valid && slot < 0 && (fa < 4u || fb < 4u);
  } else {
    const uint32_t b = __umulhi(e.x * 0x9E3779B1u, (uint32_t)a.n_buckets);
    const uint4 k4 = kCl ? ldc128(tb + 16u * b) : lds128(tb + 16u * b);
    const int h = bucket_hit(k4, e.x);
    const uint32_t f = bucket_fill(k4);
    slot = h >= 0 ? (int)(4 * b) + h : -1;
    s_new = 4 * b + f;
    ins = valid && slot < 0 && f < 4u;
  }
  const uint32_t old = kCl ? atomc_cas_if(ins, tb + 4u * s_new, kEmptyKey, e.x)
                           : atom_cas_if(ins, tb + 4u * s_new, kEmptyKey, e.x);
  if (ins && (old == kEmptyKey || old == e.x)) slot = (int)s_new;
  const bool ok = valid && slot >= 0;
  const uint32_t v = vb + 4u * kVW * (uint32_t)slot;
  if (kVW == 2) {
    const uint32_t old = kCl ? atomc_add_if(ok, v, e.y) : atom_add_if(ok, v, e.y);
    acc |= ok ? (old | e.y) : 0u;
    if (kCl) redc_add_if(ok, v + 4u, e.z);
    else red_add_if(ok, v + 4u, e.z);
  } else if (kCl) {
    redc_add_if(ok, v, e.y);
    if (kVW == 3) {
      redc_add_if(ok, v + 4u, e.z);
      redc_add_if(ok, v + 8u, e.w);
    }
  } else {
    red_add_if(ok, v, e.y);
    if (kVW == 3) {
      red_add_if(ok, v + 4u, e.z);
      red_add_if(ok, v + 8u, e.w);
    }
  }
  // both buckets full (or insert race lost): the run goes to this CTA's overflow list (rare
  // at the table's load: the warp skips this unless one of its lanes needs it)
  const bool ov = valid && slot < 0;
  if (__any_sync(kFull, ov)) {
    const uint32_t i = atom_add_if(ov, S.a_key - kFlagOvf, 1u);
    const bool ov_ok = ov && i < (uint32_t)kOvfCap;
    stg128_if(ov_ok, a.ovf + ((size_t)blockIdx.x * kOvfCap + (ov_ok ? i : 0u)), e);
    sts32_if(ov && !ov_ok, S.a_key - kFlagFull, 1u);
  }
}

// Two entries per lane into this CTA's single-bucket table, the steps of the two inserts
// interleaved so that their shared-memory round trips overlap (insert_entry's steps, twice).
// Two entries of one lane compete for a slot like entries of two lanes: the same new key
// aimed at one free slot is placed by the first CAS and found by the second; a different
// key loses the slot and goes to the overflow list.
template <int kVW>
__device__ __forceinline__ void insert_entry2(const EvalSmem& S, const EvalArgs& a, const uint4& e0, const uint4& e1,
                                              uint32_t& acc) {
  const bool v0 = e0.x != kEmptyKey, v1 = e1.x != kEmptyKey;
  const uint32_t nb = (uint32_t)a.n_buckets;
  const uint32_t b0 = __umulhi(e0.x * 0x9E3779B1u, nb), b1 = __umulhi(e1.x * 0x9E3779B1u, nb);
  const uint4 k0 = lds128(S.a_key + 16u * b0);
  const uint4 k1 = lds128(S.a_key + 16u * b1);
  const int h0 = bucket_hit(k0, e0.x), h1 = bucket_hit(k1, e1.x);
  const uint32_t f0 = bucket_fill(k0), f1 = bucket_fill(k1);
  int slot0 = h0 >= 0 ? (int)(4 * b0) + h0 : -1;
  int slot1 = h1 >= 0 ? (int)(4 * b1) + h1 : -1;
  const uint32_t s0 = 4 * b0 + f0, s1 = 4 * b1 + f1;
  const bool ins0 = v0 && slot0 < 0 && f0 < 4u, ins1 = v1 && slot1 < 0 && f1 < 4u;
  const uint32_t o0 = atom_cas_if(ins0, S.a_key + 4u * s0, kEmptyKey, e0.x);
  const uint32_t o1 = atom_cas_if(ins1, S.a_key + 4u * s1, kEmptyKey, e1.x);
  if (ins0 && (o0 == kEmptyKey || o0 == e0.x)) slot0 = (int)s0;
  if (ins1 && (o1 == kEmptyKey || o1 == e1.x)) slot1 = (int)s1;
  const bool ok0 = v0 && slot0 >= 0, ok1 = v1 && slot1 >= 0;
  const uint32_t w0 = S.a_vals + 4u * kVW * (uint32_t)slot0, w1 = S.a_vals + 4u * kVW * (uint32_t)slot1;
  if (kVW == 2) {
    const uint32_t old0 = atom_add_if(ok0, w0, e0.y);
    const uint32_t old1 = atom_add_if(ok1, w1, e1.y);
    red_add_if(ok0, w0 + 4u, e0.z);
    red_add_if(ok1, w1 + 4u, e1.z);
    acc |= (ok0 ? (old0 | e0.y) : 0u) | (ok1 ? (old1 | e1.y) : 0u);
  } else {
    red_add_if(ok0, w0, e0.y);
    red_add_if(ok1, w1, e1.y);
    if (kVW == 3) {
      red_add_if(ok0, w0 + 4u, e0.z);
      red_add_if(ok1, w1 + 4u, e1.z);
      red_add_if(ok0, w0 + 8u, e0.w);
      red_add_if(ok1, w1 + 8u, e1.w);
    }
  }
  const bool ov0 = v0 && slot0 < 0, ov1 = v1 && slot1 < 0;
  if (__any_sync(kFull, ov0 || ov1)) {
    uint4* ovf = a.ovf + (size_t)blockIdx.x * kOvfCap;
    const uint32_t i0 = atom_add_if(ov0, S.a_key - kFlagOvf, 1u);
    const uint32_t i1 = atom_add_if(ov1, S.a_key - kFlagOvf, 1u);
    const bool ok_i0 = ov0 && i0 < (uint32_t)kOvfCap, ok_i1 = ov1 && i1 < (uint32_t)kOvfCap;
    stg128_if(ok_i0, ovf + (ok_i0 ? i0 : 0u), e0);
    stg128_if(ok_i1, ovf + (ok_i1 ? i1 : 0u), e1);
    sts32_if((ov0 && !ok_i0) || (ov1 && !ok_i1), S.a_key - kFlagFull, 1u);
  }
}

// A pose swept once for all its key partitions (eval_kernel<..., kSp>): every entry is
// appended to this CTA's queue of its key partition p (of 2^lg) in global memory, and each
// pass then inserts one queue into the table, 32 entries per warp at a time (inserting
// partition 0's entries during the sweep would run the insert for every lane of a drain
// with only a 2^-lg share of them valid).  Lanes of one partition take consecutive queue
// places (one shared atomic per partition and warp).  A full queue sends the pose to the
// exact path.
__device__ __forceinline__ void spill_entry(const EvalSmem& S, const EvalArgs& a, const uint4& e, uint32_t lg) {
  const bool sp = e.x != kEmptyKey;
  const uint32_t part = sp ? (e.x * 0x85EBCA77u) >> (32 - lg) : 0u;
  const uint32_t lane = threadIdx.x & 31u;
  const uint32_t grp = __match_any_sync(kFull, sp ? part : 0xFFFFFFFFu);
  const uint32_t leader = (uint32_t)__ffs(grp) - 1u;
  uint32_t base = 0u;
  if (sp && lane == leader) base = atom_add(S.a_spill + 4u * part, (uint32_t)__popc(grp));
  base = __shfl_sync(kFull, base, (int)leader);
  const uint32_t idx = base + (uint32_t)__popc(grp & lane_mask_lt());
  const bool ok = sp && idx < (uint32_t)a.spill_cap;
  uint4* q = a.spill + ((size_t)blockIdx.x * (size_t)a.spill_np + part) * (size_t)a.spill_cap;
  stg128_if(ok, q + (ok ? idx : 0u), e);
  sts32_if(sp && !ok, S.a_key - kFlagFull, 1u);
}

template <int kVW, bool kCount32, bool kTwo, bool kCl = false, bool kSpill = false>
__device__ __forceinline__ void ring_drain(const EvalSmem& S, uint32_t ring, uint32_t& fill, uint32_t count_arg,
                                           const EvalArgs& a, uint32_t& acc, uint32_t lg = 0u) {
  const uint32_t count = kCount32 ? 32u : count_arg;
  const uint32_t lane = threadIdx.x & 31u;
  __syncwarp();
  uint4 e = lds128(ring + 16u * lane);  // the ring holds 64 entries: always in bounds
  if (!kCount32 && lane >= count) e.x = kEmptyKey;
  if constexpr (kSpill) spill_entry(S, a, e, lg);
  else insert_entry<kVW, kTwo, kCl>(S, a, e, acc);
  // move the entries beyond `count` down (lane l reads entry l + count and writes entry l,
  // which only it has read; entry l + count < 64 for count <= 32)
  const bool mv = lane + count < fill;
  const uint32_t dst = ring + 16u * lane;
  const uint4 moved = lds128(dst + 16u * count);
  sts128_if(mv, dst, moved);
  __syncwarp();
  fill -= count;
}

// Append the finished runs of the lanes with `done` set, then drain if 32 are waiting.
template <int kVW, bool kTwo, bool kCl = false, bool kSpill = false>
__device__ __forceinline__ void ring_push(const EvalSmem& S, uint32_t ring, uint32_t lane_lt, bool done,
                                          const Run& r, uint32_t& fill, const EvalArgs& a, uint32_t& acc,
                                          uint32_t lg = 0u) {
  const uint32_t m = __ballot_sync(kFull, done);
  sts128_if(done, ring + 16u * (fill + (uint32_t)__popc(m & lane_lt)), run_entry<kVW>(r));
  fill += (uint32_t)__popc(m);
  // fill is the same in every lane; the vote lets the compiler know the branch is uniform
  if (__any_sync(kFull, fill >= 32u)) ring_drain<kVW, true, kTwo, kCl, kSpill>(S, ring, fill, 32u, a, acc, lg);
}

struct PoseRegs {
  float r[9];
  float t[3];
};

// Key and dz of one point under the pose; key = kEmptyKey (and dz = 0) outside the grid.
template <bool kRot>
__device__ __forceinline__ void point_key(const VoxelConst& vc, const PoseRegs& P, const float4& p, uint32_t& key,
                                          int& dz) {
  if (kRot) {
    float ux, uy, uz;
    rotate_point(P.r, p.x, p.y, p.z, ux, uy, uz);
    dz = 0;
    key = voxel_key_g(__fadd_rn(ux, P.t[0]), __fadd_rn(uy, P.t[1]), __fadd_rn(uz, P.t[2]), vc.inv_res, vc.X, vc.Y,
                      vc.Z, vc.res_mm, &dz);
  } else {
    // Pre-rotated copies hold finite values or +inf (pack_points_kernel), and host poses
    // are finite, so g is never NaN: a saturating floor and unsigned compares decide
    // "inside" exactly as the float compares would.  dz is meaningful only inside the grid
    // (outside, the point's run has kEmptyKey and is dropped with its sums).
    const float gx = __fadd_rn(p.x, P.t[0]);
    const float gy = __fadd_rn(p.y, P.t[1]);
    const float gz = __fadd_rn(p.z, P.t[2]);
    const uint32_t kx = (uint32_t)__float2int_rd(__fmul_rn(gx, vc.inv_res));
    const uint32_t ky = (uint32_t)__float2int_rd(__fmul_rn(gy, vc.inv_res));
    const uint32_t kz = (uint32_t)__float2int_rd(__fmul_rn(gz, vc.inv_res));
    const bool in = (kx < (uint32_t)vc.X) & (ky < (uint32_t)vc.Y) & (kz < (uint32_t)vc.Z);
    const uint32_t zq = (uint32_t)__float2int_rn(__fmul_rn(gz, 1000.0f));
    dz = (int)(zq - kz * (uint32_t)vc.res_mm);
    key = in ? (kz * (uint32_t)vc.Y + ky) * (uint32_t)vc.X + kx : kEmptyKey;
  }
}

__device__ __forceinline__ void load_pose(const float* poses, PoseRegs& P) {
#pragma unroll
  for (int i = 0; i < 9; ++i) P.r[i] = __ldg(poses + i);
#pragma unroll
  for (int i = 0; i < 3; ++i) P.t[i] = __ldg(poses + 9 + i);
}

// Tile layout (kTile float4 slots of storage per tile): x,y of the tile's points as float2
// in the first half, z as float in the next quarter (12 bytes read per point).  `src` is
// the copy's base plus this thread's index.
__device__ __forceinline__ void load_tile(const float4* src, int t, float4* v) {
  const float4* tile = src - threadIdx.x + (size_t)t * kTile;
  const float2* xy = reinterpret_cast<const float2*>(tile);
  const float* z = reinterpret_cast<const float*>(tile) + 2 * kTile;
#pragma unroll
  for (int j = 0; j < kPPT; ++j) {
    const float2 p = __ldg(xy + threadIdx.x + j * kThreads);
    v[j].x = p.x;
    v[j].y = p.y;
    v[j].z = __ldg(z + threadIdx.x + j * kThreads);
  }
}

// The same load from per-thread pointers into a tile: xy at xy[j*kThreads], z at
// z[j*kThreads].  The sweep advances the pointers from tile to tile, so that the
// addresses of the tiles it prefetches are constant offsets from them.
__device__ __forceinline__ void load_tile_at(const float2* xy, const float* z, float4* v) {
#pragma unroll
  for (int j = 0; j < kPPT; ++j) {
    const float2 p = __ldg(xy + j * kThreads);
    v[j].x = p.x;
    v[j].y = p.y;
    v[j].z = __ldg(z + j * kThreads);
  }
}
constexpr int kTileXY = 2 * kTile;  // tile stride in float2 (kTile float4 slots)
constexpr int kTileZ = 4 * kTile;   // tile stride in float

// Store point `i` (position within its tile copy) in the tile layout above.
__device__ __forceinline__ void store_point(float4* out, int64_t i, float x, float y, float z) {
  const int64_t t = i / kTile;
  const int pos = (int)(i - t * kTile);
  float4* tile = out + t * kTile;
  reinterpret_cast<float2*>(tile)[pos] = make_float2(x, y);
  (reinterpret_cast<float*>(tile) + 2 * kTile)[pos] = z;
}

// Make `it` the current item: its grid constants into shared memory.  Called by all
// threads at a pose boundary.
__device__ __forceinline__ void select_item(const EvalSmem& S, const EvalArgs& a, int it) {
  if (*(volatile int32_t*)S.item == it) return;
  __syncthreads();
  const uint32_t* src = reinterpret_cast<const uint32_t*>(&a.items[it].gc);
  uint32_t* dst = reinterpret_cast<uint32_t*>(S.gc);
  for (int i = threadIdx.x; i < kGcWords; i += blockDim.x) dst[i] = __ldg(src + i);
  __syncthreads();
  if (threadIdx.x == 0) *S.item = it;
  __syncthreads();
}

// Feature symbol of a voxel whose sums fit the 32-bit table (n <= nlim, so n*S2 < 2^64 and
// S1^2 < 2^62): the same integer tests as feature_symbol, in 64-bit arithmetic.  The variance
// test n*S2 - S1^2 >= t*n^2 compares the 128-bit product t*n^2 by its high and low words.
__device__ __forceinline__ int feature_symbol_small(const GridConst& gc, uint32_t n, int32_t s1, uint32_t s2) {
  if (n == 0u) return 0;
  int lc = 0, lv = 0;
  if (gc.feature != 1) {  // count level: #{j : n >= ct[j]}, a prefix of the ascending thresholds
    int lo = 0, hi = gc.Lc - 1;
    while (lo < hi) {
      const int mid = (lo + hi) >> 1;
      if (n >= gc.count_thresh[mid]) lo = mid + 1;
      else hi = mid;
    }
    lc = lo;
  }
  if (gc.feature != 0) {  // variance level: #{j : n*S2 - S1^2 >= vt[j] * n^2}
    const uint64_t spread = (uint64_t)n * s2 - (uint64_t)((int64_t)s1 * s1);  // >= 0 (Cauchy-Schwarz)
    int lo = 0, hi = gc.Lv - 1;
    if (gc.sym32) {  // n < 2^16 and every threshold < 2^32: t * n^2 is one 32 x 32-bit product
      const uint32_t n2 = n * n;
      while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if ((uint64_t)(uint32_t)gc.var_thresh[mid] * n2 <= spread) lo = mid + 1;
        else hi = mid;
      }
    } else {
      const uint64_t n2 = (uint64_t)n * n;
      while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        const uint64_t t = (uint64_t)gc.var_thresh[mid];  // thresholds are >= 0
        const bool reached = __umul64hi(t, n2) == 0ull && t * n2 <= spread;
        if (reached) lo = mid + 1;
        else hi = mid;
      }
    }
    lv = lo;
  }
  if (gc.feature == 0) return 1 + lc;
  if (gc.feature == 1) return 1 + lv;
  return 1 + lc * gc.Lv + lv;
}

// Bbox accumulators of a warp's share of the table scan, one box per pose of the sweep.
template <int kNP>
struct ScanBox {
  int mn[kNP][3], mx[kNP][3];
  __device__ ScanBox() {
#pragma unroll
    for (int a = 0; a < kNP; ++a)
#pragma unroll
      for (int i = 0; i < 3; ++i) mn[a][i] = INT_MAX, mx[a][i] = INT_MIN;
  }
  // add voxel (kx, ky, kz) to the box of pose pa (branch-free for two poses)
  __device__ __forceinline__ void add(uint32_t pa, int kx, int ky, int kz) {
    const int k[3] = {kx, ky, kz};
#pragma unroll
    for (int a = 0; a < kNP; ++a) {
      const bool mine = kNP == 1 || pa == (uint32_t)a;
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        mn[a][i] = mine ? min(mn[a][i], k[i]) : mn[a][i];
        mx[a][i] = mine ? max(mx[a][i], k[i]) : mx[a][i];
      }
    }
  }
};

// One occupied slot: read and clear it, then (unless `discard`) its voxel's coordinates,
// feature symbol and joint-histogram entry.  With kNP == 2 the key's top bit names the pose
// of the pair (the keys of the second pose carry bit 31).
template <int kVW, bool kExact, int kNP>
__device__ __forceinline__ void scan_entry(const EvalSmem& S, const GridConst& gc, const EvalItem& I,
                                           unsigned long long* wide, uint32_t* wide_count, uint32_t s, int lp,
                                           bool discard, ScanBox<kNP>& bx) {
  const uint32_t kk = lds32(S.a_key + 4u * s);
  const uint32_t pa = kNP == 2 ? kk >> 31 : 0u;
  const uint32_t k = kNP == 2 ? kk & 0x7FFFFFFFu : kk;
  // A's symbol of the voxel, requested first: its L2 latency overlaps the work below
  const int sA = discard ? 0 : (int)__ldg(I.symA + k);
  const uint32_t v = S.a_vals + 4u * kVW * s;
  const uint32_t w = lds32(v);
  uint64_t n = w;
  int64_t s1 = 0;
  uint64_t s2 = 0;
  if (kExact) {  // plain count in the table, S1 and S2 in the 64-bit sums
    if (kVW > 1) {
      s1 = (int64_t)wide[2 * s];
      s2 = wide[2 * s + 1];
      wide[2 * s] = 0ull;
      wide[2 * s + 1] = 0ull;
      if (!discard && n > gc.nlim) atomicAdd(wide_count, 1u);
    }
  } else if (kVW == 2) {  // packed: W = n * 2^ns + sum(dz + dz_bound)
    n = w >> gc.ns_shift;
    s1 = (int64_t)(w & ((1u << gc.ns_shift) - 1u)) - (int64_t)n * gc.dz_bound;
    s2 = lds32(v + 4u);
  } else if (kVW == 3) {  // sums of dz - res_mm / 2 (the feature symbols are shift-invariant)
    s1 = (int32_t)lds32(v + 4u);
    s2 = lds32(v + 8u);
    if (n > gc.nlim3c) sts32(S.a_key - kFlagWide, 1u);  // the sums may have wrapped: exact path
  }
  sts32(S.a_key + 4u * s, kEmptyKey);
#pragma unroll
  for (int i = 0; i < kVW; ++i) sts32(v + 4u * i, 0u);
  if (discard) return;
  const uint32_t r = gc.div_x ? (uint32_t)__umul64hi(gc.div_x, k) : k;  // k / X
  const uint32_t q = gc.div_y ? (uint32_t)__umul64hi(gc.div_y, r) : r;  // r / Y
  const int kx = (int)(k - r * (uint32_t)gc.X);
  const int ky = (int)(r - q * (uint32_t)gc.Y);
  const int kz = (int)q;
  bx.add(pa, kx, ky, kz);
  // The fast path redoes any pose with a voxel above nlim (flag above), so its symbols only
  // need the 64-bit test; the exact path takes the 128-bit one where needed.
  const int sB = (kExact && n > gc.nlim)
                     ? feature_symbol(gc.feature, gc.Lc, gc.Lv, gc.count_thresh, gc.var_thresh, n, s1, s2)
                     : feature_symbol_small(gc, (uint32_t)n, (int32_t)s1, (uint32_t)s2);
  if (kx >= gc.boxA[0] && kx <= gc.boxA[3] && ky >= gc.boxA[1] && ky <= gc.boxA[4] && kz >= gc.boxA[2] &&
      kz <= gc.boxA[5])
    red_add(S.a_hist + 4u * (pa * S.hist_stride + (uint32_t)(sA * gc.K + sB)), 1u);
  if (I.dump != nullptr && lp == 0 && pa == 0u) {
    if (kVW == 3 && !kExact) {  // back to sums of dz: S1 + n c and S2 + 2 c S1 + n c^2
      const int64_t c = gc.res_mm / 2;
      s2 = (uint64_t)((int64_t)s2 + 2 * c * s1 + (int64_t)n * c * c);
      s1 += (int64_t)n * c;
    }
    I.dump[3 * (size_t)k] = (int64_t)n;
    I.dump[3 * (size_t)k + 1] = s1;
    I.dump[3 * (size_t)k + 2] = (int64_t)s2;
  }
}

// Read (and clear) the table after a sweep: symbols, bboxes and histograms unless `discard`.
// Every warp scans a contiguous share of the slots and compacts the occupied ones into a
// list (in its run ring, empty after the sweep), so that the per-voxel work runs with all
// 32 lanes busy.  The CTA-wide occupied count is added to the occupied flag word.
template <int kVW, bool kExact, int kNP>
__device__ __forceinline__ void scan_table(const EvalSmem& S, const GridConst& gc, const EvalItem& I,
                                           unsigned long long* wide, uint32_t* wide_count, int T, int lp,
                                           bool discard) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const uint32_t lane_lt = lane_mask_lt();
  const uint32_t list = S.a_queue + (uint32_t)warp * kQueue * 16u;
  const int per = (T + kWarps * 32 - 1) / (kWarps * 32) * 32;
  const int beg = warp * per, end = min(T, beg + per);
  ScanBox<kNP> bx;
  uint32_t cnt = 0, occupied = 0;
  for (int base = beg; base < end; base += 32) {
    const int s = base + lane;
    const bool occ = s < end && lds32(S.a_key + 4u * (uint32_t)s) != kEmptyKey;
    const uint32_t m = __ballot_sync(kFull, occ);
    if (occ) sts32(list + 4u * (cnt + (uint32_t)__popc(m & lane_lt)), (uint32_t)s);
    cnt += (uint32_t)__popc(m);
    occupied += (uint32_t)__popc(m);
    if (cnt >= 32u) {
      __syncwarp();
      scan_entry<kVW, kExact, kNP>(S, gc, I, wide, wide_count, lds32(list + 4u * (uint32_t)lane), lp, discard, bx);
      // move the rest down (lane l reads entry l + 32 and writes entry l, which only it read)
      if ((uint32_t)lane + 32u < cnt) sts32(list + 4u * (uint32_t)lane, lds32(list + 4u * ((uint32_t)lane + 32u)));
      __syncwarp();
      cnt -= 32u;
    }
  }
  __syncwarp();
  if ((uint32_t)lane < cnt)
    scan_entry<kVW, kExact, kNP>(S, gc, I, wide, wide_count, lds32(list + 4u * (uint32_t)lane), lp, discard, bx);
  if (lane == 0 && occupied) red_add(S.a_key - kFlagOccupied, occupied);
#pragma unroll
  for (int a = 0; a < kNP; ++a) {
    const int mn0 = __reduce_min_sync(kFull, bx.mn[a][0]), mn1 = __reduce_min_sync(kFull, bx.mn[a][1]);
    const int mn2 = __reduce_min_sync(kFull, bx.mn[a][2]), mx0 = __reduce_max_sync(kFull, bx.mx[a][0]);
    const int mx1 = __reduce_max_sync(kFull, bx.mx[a][1]), mx2 = __reduce_max_sync(kFull, bx.mx[a][2]);
    if (lane == 0 && !discard && mn0 != INT_MAX) {
      const uint32_t b = S.a_box + 24u * (uint32_t)a;
      red_min_s32(b, mn0); red_min_s32(b + 4, mn1); red_min_s32(b + 8, mn2);
      red_max_s32(b + 12, mx0); red_max_s32(b + 16, mx1); red_max_s32(b + 20, mx2);
    }
  }
}

template <int kVW>
__device__ __forceinline__ void init_smem(const EvalSmem& S, int T, int KK, int np) {
  const int tid = threadIdx.x;
  for (int i = tid; i < T; i += kThreads) {
    S.tkey[i] = kEmptyKey;
#pragma unroll
    for (int j = 0; j < kVW; ++j) S.tval[kVW * i + j] = 0u;
  }
  for (int i = tid; i < np * (int)S.hist_stride; i += kThreads) S.hist[i] = 0u;
  if (tid == 0) {
    for (int a = 0; a < np; ++a) {
      S.box[6 * a + 0] = S.box[6 * a + 1] = S.box[6 * a + 2] = INT_MAX;
      S.box[6 * a + 3] = S.box[6 * a + 4] = S.box[6 * a + 5] = INT_MIN;
    }
    S.flags[0] = S.flags[1] = S.flags[2] = S.flags[3] = 0u;
    for (int q = 0; q < 8; ++q) S.spill_cnt[q] = 0u;
    *S.item = -1;
  }
  (void)KK;
}

// After a pass's table scan (flags final): in the packed layout a set wide flag means that a
// voxel may have passed nlim_pack, which sends the pose to the exact path; such passes are
// counted for the host, which then gives the grid the three-word layout (a larger limit).
template <int kVW>
__device__ __forceinline__ void note_wide(const EvalSmem& S, const EvalArgs& a) {
  if (kVW == 2 && threadIdx.x == 0 && a.wide_poses != nullptr && *(volatile uint32_t*)&S.flags[3] != 0u)
    atomicAdd(a.wide_poses, 1u);
}

// Store the partial histogram and bbox of pose `a` of the sweep as pose lp of item I, then
// reset them for the next sweep.  Called by all threads.
__device__ __forceinline__ void emit_pose(const EvalSmem& S, const EvalItem& I, int lp, int a = 0) {
  const int tid = threadIdx.x;
  const int KK = S.gc->K * S.gc->K;
  uint32_t* oc = I.out_c + (size_t)lp * KK;
  uint32_t* h = S.hist + (size_t)a * S.hist_stride;
  int32_t* bx = S.box + 6 * a;
  for (int i = tid; i < KK; i += kThreads) {
    oc[i] = h[i];
    h[i] = 0u;
  }
  if (tid < 6) I.out_box[6 * (size_t)lp + tid] = bx[tid];
  __syncthreads();
  if (tid < 6) bx[tid] = tid < 3 ? INT_MAX : INT_MIN;
  __syncthreads();
}

__device__ __forceinline__ void reset_pose(const EvalSmem& S, int a = 0) {
  const int tid = threadIdx.x;
  const int KK = S.gc->K * S.gc->K;
  uint32_t* h = S.hist + (size_t)a * S.hist_stride;
  for (int i = tid; i < KK; i += kThreads) h[i] = 0u;
  if (tid < 6) S.box[6 * a + tid] = tid < 3 ? INT_MAX : INT_MIN;
}

// Item of global pose gp: the last item whose start is <= gp (binary search).
__device__ __forceinline__ int item_of(const EvalArgs& a, int gp) {
  if (a.item_start == nullptr) return 0;
  int lo = 0, hi = a.n_items - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (__ldg(a.item_start + mid) <= gp) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

// The item of a pose.  With a single item its fields (and the voxel map constants of the
// sweep) are read straight from the kernel parameters, which costs no registers.
template <bool kOne>
__device__ __forceinline__ const EvalItem& item_at(const EvalArgs& a, int it) {
  if constexpr (kOne) {
    return a.one;
  } else {
    return a.items[it];
  }
}

__device__ __forceinline__ const float4* pose_tiles(const EvalItem& I, int lp) {
  const int src = I.pose_src ? __ldg(I.pose_src + lp) : 0;
  return I.src + (size_t)src * I.src_stride;
}

// One tile of this thread's stream: key, run step, ring append of the finished run.  No
// per-point check of dz: the grid constants guarantee 0 <= dz <= res_mm for every point
// inside the grid (validate_desc).
template <int kVW, bool kRot, bool kPart, bool kTwo = false, bool kCl = false, bool kSpill = false>
__device__ __forceinline__ void sweep_tile(const EvalSmem& S, const EvalArgs& a, const VoxelConst& vc,
                                           const PoseRegs& P, const float4* pts, int lg, uint32_t part, Run& run,
                                           uint32_t ring, uint32_t lane_lt, uint32_t& fill, uint32_t& acc) {
#pragma unroll
  for (int j = 0; j < kPPT; ++j) {
    uint32_t key;
    int dz;
    point_key<kRot>(vc, P, pts[j], key, dz);
    if (kPart && key != kEmptyKey && ((key * 0x85EBCA77u) >> (32 - lg)) != part) key = kEmptyKey;
    const bool done = key != run.key;
    ring_push<kVW, kTwo, kCl, kSpill>(S, ring, lane_lt, done && run.key != kEmptyKey, run, fill, a, acc,
                                      (uint32_t)lg);
    const int dzr = kVW == 3 ? dz - vc.zc : dz;  // layout 3 sums offsets from the voxel's middle
    if (kVW == 2) {
      run.w = (done ? 0u : run.w) + ((uint32_t)dz + vc.winc);
    } else {
      run.w = (done ? 0u : run.w) + 1u;
      if (kVW == 3) run.s1 = (done ? 0u : run.s1) + (uint32_t)dzr;
    }
    if (kVW > 1) run.s2 = (done ? 0u : run.s2) + (uint32_t)(dzr * dzr);
    run.key = key;
  }
}

// The run step of one point whose key and dz are known: append the finished run, extend or
// restart the run.
template <int kVW, bool kTwo, bool kCl = false, bool kSpill = false>
__device__ __forceinline__ void run_step(const EvalSmem& S, const EvalArgs& a, const VoxelConst& vc, uint32_t key,
                                         int dz, Run& run, uint32_t ring, uint32_t lane_lt, uint32_t& fill,
                                         uint32_t& acc, uint32_t lg = 0u) {
  const bool done = key != run.key;
  // a finished run of points outside the grid (or outside the key partition) is dropped
  ring_push<kVW, kTwo, kCl, kSpill>(S, ring, lane_lt, done && run.key != kEmptyKey, run, fill, a, acc, lg);
  const int dzr = kVW == 3 ? dz - vc.zc : dz;  // layout 3 sums offsets from the voxel's middle
  if (kVW == 2) {
    run.w = (done ? 0u : run.w) + ((uint32_t)dz + vc.winc);
  } else {
    run.w = (done ? 0u : run.w) + 1u;
    if (kVW == 3) run.s1 = (done ? 0u : run.s1) + (uint32_t)dzr;
  }
  if (kVW > 1) run.s2 = (done ? 0u : run.s2) + (uint32_t)(dzr * dzr);
  run.key = key;
}

// One pass over all tiles of the pose: every thread streams its own points straight from
// L2, kDepth tiles ahead.  A run is cut every `cut` tiles so that its 32-bit sums stay
// below nlim points.
template <int kVW, bool kRot, bool kPart, bool kTwo = false, bool kCl = false, int kD = kDepth,
          bool kSpill = false>
__device__ __forceinline__ void sweep_pose(const EvalSmem& S, const EvalArgs& a, const VoxelConst& vc,
                                               const PoseRegs& P, const float4* src, int nt, int lg, uint32_t part,
                                               uint32_t ring, uint32_t lane_lt, int cut) {
  Run run{kEmptyKey, 0u, 0u, 0u};
  uint32_t fill = 0u, acc = 0u;
  float4 buf[kD][kPPT];  // register ring of the next kD tiles
  // this thread's slot of tile 0 (x,y and z); tile t is kTileXY / kTileZ further on
  const float2* xy = reinterpret_cast<const float2*>(src - threadIdx.x) + threadIdx.x;
  const float* zz = reinterpret_cast<const float*>(src - threadIdx.x) + 2 * kTile + threadIdx.x;
#pragma unroll
  for (int d = 0; d < kD; ++d)
    if (d < nt) load_tile_at(xy + d * kTileXY, zz + d * kTileZ, buf[d]);
  xy += kD * kTileXY;  // the next tile to load: t + kD
  zz += kD * kTileZ;
  int next_cut = cut;
  int t = 0;
  for (; t + 2 * kD <= nt; t += kD) {  // every prefetch in range: no guards
    if (t >= next_cut) {  // uniform; only when a stream is longer than nlim points
      ring_push<kVW, kTwo, kCl, kSpill>(S, ring, lane_lt, run.key != kEmptyKey, run, fill, a, acc, (uint32_t)lg);
      run = Run{kEmptyKey, 0u, 0u, 0u};
      next_cut += cut;
    }
    // the keys of the kD buffered tiles first (independent of one another), then the
    // next loads into the freed buffers, then the run steps in stream order
    uint32_t keys[kD][kPPT];
    int dzs[kD][kPPT];
#pragma unroll
    for (int d = 0; d < kD; ++d)
#pragma unroll
      for (int j = 0; j < kPPT; ++j) {
        point_key<kRot>(vc, P, buf[d][j], keys[d][j], dzs[d][j]);
        if (kPart && keys[d][j] != kEmptyKey && ((keys[d][j] * 0x85EBCA77u) >> (32 - lg)) != part)
          keys[d][j] = kEmptyKey;
      }
#pragma unroll
    for (int d = 0; d < kD; ++d) load_tile_at(xy + d * kTileXY, zz + d * kTileZ, buf[d]);
#pragma unroll
    for (int d = 0; d < kD; ++d)
#pragma unroll
      for (int j = 0; j < kPPT; ++j)
        run_step<kVW, kTwo, kCl, kSpill>(S, a, vc, keys[d][j], dzs[d][j], run, ring, lane_lt, fill, acc,
                                         (uint32_t)lg);
    xy += kD * kTileXY;
    zz += kD * kTileZ;
  }
  for (; t < nt; t += kD) {
    if (t >= next_cut) {
      ring_push<kVW, kTwo, kCl, kSpill>(S, ring, lane_lt, run.key != kEmptyKey, run, fill, a, acc, (uint32_t)lg);
      run = Run{kEmptyKey, 0u, 0u, 0u};
      next_cut += cut;
    }
#pragma unroll
    for (int d = 0; d < kD; ++d) {
      if (t + d < nt) {
        sweep_tile<kVW, kRot, kPart, kTwo, kCl, kSpill>(S, a, vc, P, buf[d], lg, part, run, ring, lane_lt, fill, acc);
        if (t + kD + d < nt) load_tile_at(xy + d * kTileXY, zz + d * kTileZ, buf[d]);
      }
    }
    xy += kD * kTileXY;
    zz += kD * kTileZ;
  }
  ring_push<kVW, kTwo, kCl, kSpill>(S, ring, lane_lt, run.key != kEmptyKey, run, fill, a, acc, (uint32_t)lg);
  while (fill > 0u)
    ring_drain<kVW, false, kTwo, kCl, kSpill>(S, ring, fill, min(fill, 32u), a, acc, (uint32_t)lg);
  if (kVW == 2 && (acc >> vc.wide_shift) != 0u) sts32(S.a_key - kFlagWide, 1u);  // may pass nlim_pack
}

// Plain 16-byte global load (not the read-only path: the data were written in this launch).
__device__ __forceinline__ uint4 ldg128_plain(const uint4* g) {
  uint4 v;
  asm volatile("ld.global.v4.u32 {%0, %1, %2, %3}, [%4];"
               : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
               : "l"(g)
               : "memory");
  return v;
}

// Pass `part` of a pose (or pose pair) swept once (eval_kernel<..., kSp>, eval_pair_kernel<...,
// kSp>): insert the runs that the sweep queued for this partition.  kTwo: the pair kernel's
// two-choice table, one batch per warp at a time with the next loading meanwhile.
template <int kVW, bool kTwo = false>
__device__ __forceinline__ void drain_spilled(const EvalSmem& S, const EvalArgs& a, const VoxelConst& vc,
                                              uint32_t part) {
  const uint32_t n = min(*(volatile uint32_t*)&S.spill_cnt[part], (uint32_t)a.spill_cap);
  const uint4* q = a.spill + ((size_t)blockIdx.x * (size_t)a.spill_np + part) * (size_t)a.spill_cap;
  const uint32_t lane = threadIdx.x & 31u;
  const uint4 none = make_uint4(kEmptyKey, 0u, 0u, 0u);
  uint32_t acc = 0u;
  constexpr uint32_t kStep = 32u * kWarps;
  uint32_t i = (threadIdx.x >> 5) * 32u;
  if constexpr (kTwo) {
    uint4 e = i + lane < n ? ldg128_plain(q + i + lane) : none;
    for (; i < n; i += kStep) {  // the same trip count in every lane of a warp
      const uint32_t j = i + kStep;
      const uint4 nx = j + lane < n ? ldg128_plain(q + j + lane) : none;
      insert_entry<kVW, true>(S, a, e, acc);
      e = nx;
    }
    if (kVW == 2 && (acc >> vc.wide_shift) != 0u) sts32(S.a_key - kFlagWide, 1u);  // may pass nlim_pack
    return;
  }
  // each warp takes two batches of 32 at a time (the two inserts interleaved), the next two
  // loading meanwhile
  uint4 e0 = i + lane < n ? ldg128_plain(q + i + lane) : none;
  uint4 e1 = i + kStep + lane < n ? ldg128_plain(q + i + kStep + lane) : none;
  for (; i < n; i += 2u * kStep) {  // the same trip count in every lane of a warp
    const uint32_t j = i + 2u * kStep;
    const uint4 n0 = j + lane < n ? ldg128_plain(q + j + lane) : none;
    const uint4 n1 = j + kStep + lane < n ? ldg128_plain(q + j + kStep + lane) : none;
    insert_entry2<kVW>(S, a, e0, e1, acc);
    e0 = n0;
    e1 = n1;
  }
  if (kVW == 2 && (acc >> vc.wide_shift) != 0u) sts32(S.a_key - kFlagWide, 1u);  // may pass nlim_pack
}

// Keys and dz of one pre-rotated point under the two poses of a pair, which differ only in
// t'_x: the y and z halves of the voxel map (k_y, k_z, the mm rounding and dz) are computed
// once.  The same FP32 operations as point_key, so each key is bit-identical to a single
// sweep's; the second pose's keys carry bit 31 (keys are below 2^31).
__device__ __forceinline__ void pair_key(const VoxelConst& vc, float tx0, float tx1, float ty, float tz,
                                         const float4& p, uint32_t& k0, uint32_t& k1, int& dz) {
  const float gy = __fadd_rn(p.y, ty);
  const float gz = __fadd_rn(p.z, tz);
  const uint32_t ky = (uint32_t)__float2int_rd(__fmul_rn(gy, vc.inv_res));
  const uint32_t kz = (uint32_t)__float2int_rd(__fmul_rn(gz, vc.inv_res));
  const bool in_yz = (ky < (uint32_t)vc.Y) & (kz < (uint32_t)vc.Z);
  const uint32_t zq = (uint32_t)__float2int_rn(__fmul_rn(gz, 1000.0f));
  dz = (int)(zq - kz * (uint32_t)vc.res_mm);
  const uint32_t kyz = (kz * (uint32_t)vc.Y + ky) * (uint32_t)vc.X;
  const uint32_t kx0 = (uint32_t)__float2int_rd(__fmul_rn(__fadd_rn(p.x, tx0), vc.inv_res));
  const uint32_t kx1 = (uint32_t)__float2int_rd(__fmul_rn(__fadd_rn(p.x, tx1), vc.inv_res));
  k0 = (in_yz & (kx0 < (uint32_t)vc.X)) ? kyz + kx0 : kEmptyKey;
  k1 = (in_yz & (kx1 < (uint32_t)vc.X)) ? (kyz + kx1) | 0x80000000u : kEmptyKey;
}

// One pass over all tiles for a pose pair (pre-rotated tiles): as sweep_pose, with one run
// per pose; both poses' runs go to the same ring and table.
template <int kVW, bool kPart, bool kSpill = false>
__device__ __forceinline__ void sweep_pair(const EvalSmem& S, const EvalArgs& a, const VoxelConst& vc, float tx0,
                                           float tx1, float ty, float tz, const float4* src, int nt, int lg,
                                           uint32_t part, uint32_t ring, uint32_t lane_lt, int cut) {
  Run r0{kEmptyKey, 0u, 0u, 0u}, r1{kEmptyKey, 0u, 0u, 0u};
  uint32_t fill = 0u, acc = 0u;
  float4 buf[kPairDepth][kPPT];
  const float2* xy = reinterpret_cast<const float2*>(src - threadIdx.x) + threadIdx.x;
  const float* zz = reinterpret_cast<const float*>(src - threadIdx.x) + 2 * kTile + threadIdx.x;
#pragma unroll
  for (int d = 0; d < kPairDepth; ++d)
    if (d < nt) load_tile_at(xy + d * kTileXY, zz + d * kTileZ, buf[d]);
  xy += kPairDepth * kTileXY;
  zz += kPairDepth * kTileZ;
  int next_cut = cut;
  int t = 0;
  for (; t + 2 * kPairDepth <= nt; t += kPairDepth) {
    if (t >= next_cut) {
      ring_push<kVW, true, false, kSpill>(S, ring, lane_lt, r0.key != kEmptyKey, r0, fill, a, acc, (uint32_t)lg);
      ring_push<kVW, true, false, kSpill>(S, ring, lane_lt, r1.key != kEmptyKey, r1, fill, a, acc, (uint32_t)lg);
      r0 = Run{kEmptyKey, 0u, 0u, 0u};
      r1 = Run{kEmptyKey, 0u, 0u, 0u};
      next_cut += cut;
    }
    uint32_t k0[kPairDepth][kPPT], k1[kPairDepth][kPPT];
    int dzs[kPairDepth][kPPT];
#pragma unroll
    for (int d = 0; d < kPairDepth; ++d)
#pragma unroll
      for (int j = 0; j < kPPT; ++j) {
        pair_key(vc, tx0, tx1, ty, tz, buf[d][j], k0[d][j], k1[d][j], dzs[d][j]);
        if (kPart) {
          if (k0[d][j] != kEmptyKey && ((k0[d][j] * 0x85EBCA77u) >> (32 - lg)) != part) k0[d][j] = kEmptyKey;
          if (k1[d][j] != kEmptyKey && ((k1[d][j] * 0x85EBCA77u) >> (32 - lg)) != part) k1[d][j] = kEmptyKey;
        }
      }
#pragma unroll
    for (int d = 0; d < kPairDepth; ++d) load_tile_at(xy + d * kTileXY, zz + d * kTileZ, buf[d]);
#pragma unroll
    for (int d = 0; d < kPairDepth; ++d)
#pragma unroll
      for (int j = 0; j < kPPT; ++j) {
        run_step<kVW, true, false, kSpill>(S, a, vc, k0[d][j], dzs[d][j], r0, ring, lane_lt, fill, acc, (uint32_t)lg);
        run_step<kVW, true, false, kSpill>(S, a, vc, k1[d][j], dzs[d][j], r1, ring, lane_lt, fill, acc, (uint32_t)lg);
      }
    xy += kPairDepth * kTileXY;
    zz += kPairDepth * kTileZ;
  }
  for (; t < nt; t += kPairDepth) {
    if (t >= next_cut) {
      ring_push<kVW, true, false, kSpill>(S, ring, lane_lt, r0.key != kEmptyKey, r0, fill, a, acc, (uint32_t)lg);
      ring_push<kVW, true, false, kSpill>(S, ring, lane_lt, r1.key != kEmptyKey, r1, fill, a, acc, (uint32_t)lg);
      r0 = Run{kEmptyKey, 0u, 0u, 0u};
      r1 = Run{kEmptyKey, 0u, 0u, 0u};
      next_cut += cut;
    }
#pragma unroll
    for (int d = 0; d < kPairDepth; ++d) {
      if (t + d < nt) {
#pragma unroll
        for (int j = 0; j < kPPT; ++j) {
          uint32_t q0, q1;
          int dz;
          pair_key(vc, tx0, tx1, ty, tz, buf[d][j], q0, q1, dz);
          if (kPart) {
            if (q0 != kEmptyKey && ((q0 * 0x85EBCA77u) >> (32 - lg)) != part) q0 = kEmptyKey;
            if (q1 != kEmptyKey && ((q1 * 0x85EBCA77u) >> (32 - lg)) != part) q1 = kEmptyKey;
          }
          run_step<kVW, true, false, kSpill>(S, a, vc, q0, dz, r0, ring, lane_lt, fill, acc, (uint32_t)lg);
          run_step<kVW, true, false, kSpill>(S, a, vc, q1, dz, r1, ring, lane_lt, fill, acc, (uint32_t)lg);
        }
        if (t + kPairDepth + d < nt) load_tile_at(xy + d * kTileXY, zz + d * kTileZ, buf[d]);
      }
    }
    xy += kPairDepth * kTileXY;
    zz += kPairDepth * kTileZ;
  }
  ring_push<kVW, true, false, kSpill>(S, ring, lane_lt, r0.key != kEmptyKey, r0, fill, a, acc, (uint32_t)lg);
  ring_push<kVW, true, false, kSpill>(S, ring, lane_lt, r1.key != kEmptyKey, r1, fill, a, acc, (uint32_t)lg);
  while (fill > 0u) ring_drain<kVW, false, true, false, kSpill>(S, ring, fill, min(fill, 32u), a, acc, (uint32_t)lg);
  if (kVW == 2 && (acc >> vc.wide_shift) != 0u) sts32(S.a_key - kFlagWide, 1u);  // may pass nlim_pack
}

// kSp (one item, a.spill set): every pose in 2 .. a.spill_np key partitions with B swept once
// (the first pass queues the runs of the later partitions, which the later passes insert); a
// pose whose table overflows at a.spill_np partitions goes to the exact path.
template <int kVW, bool kRot, bool kOne, bool kSp = false>
__global__ void __launch_bounds__(kThreads, kCtasPerSm) eval_kernel(const __grid_constant__ EvalArgs a) {
  extern __shared__ __align__(128) uint8_t smem_raw[];
  EvalSmem S;
  const int T = a.table_slots;
  eval_smem_layout(a.K, T, kVW, 1, &S, smem_raw);
  const int tid = threadIdx.x;
  const uint32_t cap = (uint32_t)T - (uint32_t)T / 10u;  // above 90% full the table counts as crowded
  const uint32_t ring = S.a_queue + (uint32_t)(tid >> 5) * kQueue * 16u;
  const uint32_t lane_lt = lane_mask_lt();
  unsigned long long* wide = a.wide + (size_t)blockIdx.x * 2u * (size_t)T;

  init_smem<kVW>(S, T, a.K * a.K, 1);
  __syncthreads();
  int passes = a.passes0;
  int cur = -1;  // item of the previous pose: key partitions are learned per item

  for (int gp = a.p_begin + blockIdx.x; gp < a.P; gp += gridDim.x) {
    const int it = kOne ? 0 : item_of(a, gp);
    select_item(S, a, it);
    const EvalItem& I = item_at<kOne>(a, it);
    if (it != cur) {
      if (cur >= 0 && tid == 0 && item_at<kOne>(a, cur).item_passes)
        atomicMax(item_at<kOne>(a, cur).item_passes, (uint32_t)passes);
      cur = it;
      if (I.passes0 > 0) passes = I.passes0;
      if (kSp) passes = min(max(passes, 2), a.spill_np);
    }
    const int lp = gp - I.pose_base;
    const VoxelConst vc = voxel_const<kVW>(kOne ? a.one.gc : *S.gc);
    const int nt = I.n_tiles;
    // runs are cut every `cut` tiles (a multiple of the prefetch depth, where the sweep checks)
    const int cut = max(kPairDepth, (int)min(vc.nlim / (uint32_t)kPPT, (uint32_t)INT_MAX) / kPairDepth * kPairDepth);
    PoseRegs P;
    load_pose(I.poses + 12 * (size_t)lp, P);
    const float4* src = pose_tiles(I, lp) + tid;
    const int pose_passes = passes;
    const int lg = __ffs(pose_passes) - 1;
    uint32_t max_occupied = 0;
    bool full = false;        // pose handed to the exact path
    bool overflowed = false;  // ... because its keys did not fit: more partitions help
    for (int pass = 0; pass < pose_passes; ++pass) {
      if (!full) {
        if constexpr (kSp) {
          // B swept once in the first pass, every run queued by key partition; each pass
          // inserts its partition's queue
          if (pass == 0) {
            sweep_pose<kVW, kRot, false, false, false, kDepth, true>(S, a, vc, P, src, nt, lg, 0u, ring, lane_lt,
                                                                     cut);
            __syncthreads();  // every queue complete (full is the same in every thread)
          }
          drain_spilled<kVW>(S, a, vc, (uint32_t)pass);
        } else if (lg == 0) {
          sweep_pose<kVW, kRot, false>(S, a, vc, P, src, nt, 0, 0u, ring, lane_lt, cut);
        } else {
          sweep_pose<kVW, kRot, true>(S, a, vc, P, src, nt, lg, (uint32_t)pass, ring, lane_lt, cut);
        }
      }
      __syncthreads();
      if (!full && *(volatile uint32_t*)&S.flags[2] != 0u) {  // runs whose home bucket was full
        insert_overflow<kVW, false>(S, a, kOne ? a.one.gc : *S.gc);
        __syncthreads();
      }
      overflowed = overflowed || S.flags[1] != 0u;
      full = full || overflowed;
      scan_table<kVW, false, 1>(S, kOne ? a.one.gc : *S.gc, I, wide, a.wide_count, T, lp, full);
      __syncthreads();
      max_occupied = max(max_occupied, S.flags[0]);
      note_wide<kVW>(S, a);
      full = full || S.flags[3] != 0u;  // a voxel beyond the table sums: wide sums, not partitions
      __syncthreads();
      if (tid == 0) {
        S.flags[0] = 0u;
        S.flags[2] = 0u;
        S.flags[3] = 0u;
        if (kSp && pass == pose_passes - 1)
          for (int q = 0; q < 8; ++q) S.spill_cnt[q] = 0u;
      }
      __syncthreads();  // the resets before the next pass's drains count again
    }
    if (full) {
      // finished later by the exact path
      reset_pose(S);
      if (tid == 0) {
        S.flags[1] = 0u;
        a.redo_list[atomicAdd(a.redo_count, 1u)] = (uint32_t)gp;
      }
      if (overflowed && passes < (kSp ? a.spill_np : kMaxPasses)) passes *= 2;
      __syncthreads();
      continue;
    }
    emit_pose(S, I, lp);
    if (max_occupied > cap && passes < (kSp ? a.spill_np : kMaxPasses)) passes *= 2;  // crowded: more next
  }
  if (tid == 0) {
    atomicMax(a.max_passes, (uint32_t)passes);
    if (cur >= 0 && item_at<kOne>(a, cur).item_passes) atomicMax(item_at<kOne>(a, cur).item_passes, (uint32_t)passes);
  }
}

// One sweep set of the pair kernel: the poses lp0 and, with kNP == 2, lp1 (a pair that shares
// its tile copy and t'_y, t'_z) swept together over the same table, key partitions as
// needed; then their histograms and boxes, or both poses to the exact path.
template <int kVW, bool kSp = false>
__device__ __forceinline__ void pair_sweep_set(const EvalSmem& S, const EvalArgs& a, const VoxelConst& vc, int lp0,
                                               int lp1, bool two, int T, int cut, uint32_t cap, uint32_t ring,
                                               uint32_t lane_lt, unsigned long long* wide, int& passes) {
  constexpr int kNP = 2;
  const EvalItem& I = a.one;
  const int tid = threadIdx.x;
  PoseRegs P;
  load_pose(I.poses + 12 * (size_t)lp0, P);
  // without a second pose, t'_x = +inf puts every point of the second run outside the grid
  const float tx1 = two ? __ldg(I.poses + 12 * (size_t)lp1 + 9) : __int_as_float(0x7f800000);
  const float4* src = pose_tiles(I, lp0) + tid;
  const int nt = I.n_tiles;
  const int pose_passes = passes;
  const int lg = __ffs(pose_passes) - 1;
  uint32_t max_occupied = 0;
  bool full = false, overflowed = false;
  for (int pass = 0; pass < pose_passes; ++pass) {
    if (!full) {
      if constexpr (kSp) {
        // the pair's points swept once in the first pass, every run queued by key partition;
        // each pass inserts its partition's queue
        if (pass == 0) {
          sweep_pair<kVW, false, true>(S, a, vc, P.t[0], tx1, P.t[1], P.t[2], src, nt, lg, 0u, ring, lane_lt, cut);
          __syncthreads();  // every queue complete (full is the same in every thread)
        }
        drain_spilled<kVW, true>(S, a, vc, (uint32_t)pass);
      } else if (lg == 0) {
        sweep_pair<kVW, false>(S, a, vc, P.t[0], tx1, P.t[1], P.t[2], src, nt, 0, 0u, ring, lane_lt, cut);
      } else {
        sweep_pair<kVW, true>(S, a, vc, P.t[0], tx1, P.t[1], P.t[2], src, nt, lg, (uint32_t)pass, ring, lane_lt, cut);
      }
    }
    __syncthreads();
    if (!full && *(volatile uint32_t*)&S.flags[2] != 0u) {  // runs whose home bucket was full
      insert_overflow<kVW, true>(S, a, I.gc);
      __syncthreads();
    }
    overflowed = overflowed || S.flags[1] != 0u;
    full = full || overflowed;
    scan_table<kVW, false, kNP>(S, I.gc, I, wide, a.wide_count, T, lp0, full);
    __syncthreads();
    max_occupied = max(max_occupied, S.flags[0]);
    note_wide<kVW>(S, a);
    full = full || S.flags[3] != 0u;  // a voxel beyond the table sums: wide sums, not partitions
    __syncthreads();
    if (tid == 0) {
      S.flags[0] = 0u;
      S.flags[2] = 0u;
      S.flags[3] = 0u;
      if (kSp && pass == pose_passes - 1)
        for (int q = 0; q < 8; ++q) S.spill_cnt[q] = 0u;
    }
    __syncthreads();  // the resets before the next pass's drains count again
  }
  if (full) {  // both poses are finished later by the exact path
    reset_pose(S, 0);
    reset_pose(S, 1);
    if (tid == 0) {  // the redo list holds global pose indices (item pose base + local index)
      S.flags[1] = 0u;
      a.redo_list[atomicAdd(a.redo_count, 1u)] = (uint32_t)(I.pose_base + lp0);
      if (two) a.redo_list[atomicAdd(a.redo_count, 1u)] = (uint32_t)(I.pose_base + lp1);
    }
    if (overflowed && passes < (kSp ? a.spill_np : kMaxPasses)) passes *= 2;
    __syncthreads();
    return;
  }
  emit_pose(S, I, lp0, 0);
  if (two) emit_pose(S, I, lp1, 1);
  else reset_pose(S, 1);
  if (max_occupied > cap && passes < (kSp ? a.spill_np : kMaxPasses)) passes *= 2;  // crowded: more next
}

// Pose pairs (pre-rotated tiles, one item): unit u of a.units is (pose, pose or -1), local
// pose indices of the item (a.one).  Two
// poses that read the same tile copy and whose t'_y and t'_z are equal bit for bit are swept
// together (sweep_pair: one point load and one y/z voxel-map half for both); any other unit
// is swept one pose at a time.  The results are those of the single-pose kernel.
// kSp (a.spill set): every pair in 2 .. a.spill_np key partitions with its points swept once
// and the runs queued by partition (as eval_kernel<..., kSp>).
template <int kVW, bool kSp = false>
__global__ void __launch_bounds__(kThreads, kCtasPerSm) eval_pair_kernel(const __grid_constant__ EvalArgs a) {
  extern __shared__ __align__(128) uint8_t smem_raw[];
  EvalSmem S;
  const int T = a.table_slots;
  eval_smem_layout(a.K, T, kVW, 2, &S, smem_raw);
  const int tid = threadIdx.x;
  const uint32_t cap = (uint32_t)T - (uint32_t)T / 10u;  // above 90% full the table counts as crowded
  const uint32_t ring = S.a_queue + (uint32_t)(tid >> 5) * kQueue * 16u;
  const uint32_t lane_lt = lane_mask_lt();
  unsigned long long* wide = a.wide + (size_t)blockIdx.x * 2u * (size_t)T;
  init_smem<kVW>(S, T, a.K * a.K, 2);
  __syncthreads();
  select_item(S, a, 0);
  const EvalItem& I = a.one;
  int passes = I.passes0 > 0 ? I.passes0 : a.passes0;
  if (kSp) passes = min(max(passes, 2), a.spill_np);
  const VoxelConst vc = voxel_const<kVW>(I.gc);
  // runs are cut every `cut` tiles (a multiple of the prefetch depth, where the sweep checks)
  const int cut = max(kDepth, (int)min(vc.nlim / (uint32_t)kPPT, (uint32_t)INT_MAX) / kDepth * kDepth);
  static_assert(kDepth % kPairDepth == 0, "the pair sweep checks cuts at multiples of its depth");
  for (int u = blockIdx.x; u < a.n_units; u += gridDim.x) {
    const int p0 = __ldg(a.units + 2 * u), p1 = __ldg(a.units + 2 * u + 1);
    bool two = false;
    if (p1 >= 0) {
      const float* q0 = I.poses + 12 * (size_t)p0;
      const float* q1 = I.poses + 12 * (size_t)p1;
      const int s0 = I.pose_src ? __ldg(I.pose_src + p0) : 0, s1 = I.pose_src ? __ldg(I.pose_src + p1) : 0;
      two = s0 == s1 && __float_as_uint(__ldg(q0 + 10)) == __float_as_uint(__ldg(q1 + 10)) &&
            __float_as_uint(__ldg(q0 + 11)) == __float_as_uint(__ldg(q1 + 11));
    }
    if (two || p1 < 0) {
      // a single pose is swept as a pair whose second pose has no point inside the grid
      pair_sweep_set<kVW, kSp>(S, a, vc, p0, p1, two, T, cut, cap, ring, lane_lt, wide, passes);
    } else if (tid == 0) {  // not a pair after all: both poses go to the exact path (single sweeps)
      a.redo_list[atomicAdd(a.redo_count, 1u)] = (uint32_t)(I.pose_base + p0);
      a.redo_list[atomicAdd(a.redo_count, 1u)] = (uint32_t)(I.pose_base + p1);
    }
  }
  if (tid == 0) {
    atomicMax(a.max_passes, (uint32_t)passes);
    if (I.item_passes) atomicMax(I.item_passes, (uint32_t)passes);
  }
}

// One pose at a time per 2-CTA cluster, for grids whose single-pose table needs key
// partitions (the large grid).  The two CTAs sweep the two halves of every thread's stream
// of points and share one table split between their shared memories: a key lives in the
// half its owner bit names (key_owner), reached through the cluster window, so the pair
// holds twice the keys of one CTA's table (half the key partitions) and every point is swept
// once per pass, by one of the two CTAs.  Each CTA then scans its own half; the second CTA
// adds its partial histogram and box into the first's, which emits them.  Every cluster
// barrier is reached by both CTAs with the same decisions, taken from both halves' flags,
// and neither CTA leaves while the other may still address its shared memory.
template <int kVW, bool kRot>
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(kThreads, 1)
    eval_cluster_kernel(const __grid_constant__ EvalArgs a) {
  extern __shared__ __align__(128) uint8_t smem_raw[];
  EvalSmem S;
  const int T = a.table_slots;
  eval_smem_layout(a.K, T, kVW, 1, &S, smem_raw);
  const int tid = threadIdx.x;
  const uint32_t rank = cluster_rank();
  const uint32_t peer = rank ^ 1u;
  S.rank = rank;
  S.c_key[0] = map_cluster(S.a_key, 0u);
  S.c_key[1] = map_cluster(S.a_key, 1u);
  const uint32_t cap = (uint32_t)T - (uint32_t)T / 10u;  // above 90% full a half counts as crowded
  const uint32_t ring = S.a_queue + (uint32_t)(tid >> 5) * kQueue * 16u;
  const uint32_t lane_lt = lane_mask_lt();
  unsigned long long* wide = a.wide + (size_t)blockIdx.x * 2u * (size_t)T;
  init_smem<kVW>(S, T, a.K * a.K, 1);
  __syncthreads();
  select_item(S, a, 0);
  cluster_sync();  // both halves are empty before any insert crosses over
  const EvalItem& I = a.one;
  int passes = I.passes0 > 0 ? I.passes0 : a.passes0;
  const VoxelConst vc = voxel_const<kVW>(I.gc);
  const int cut = max(kDepth, (int)min(vc.nlim / (uint32_t)kPPT, (uint32_t)INT_MAX) / kDepth * kDepth);
  const int nt = I.n_tiles;
  const int half = (nt + 1) / 2;  // tiles [0, half) for rank 0, [half, nt) for rank 1
  const int t0 = rank == 0u ? 0 : half;
  const int nt_mine = rank == 0u ? half : nt - half;
  const int n_cl = (int)(gridDim.x / 2), cid = (int)(blockIdx.x / 2);
  const uint32_t c_peer = S.c_key[peer];
  for (int gp = cid; gp < a.P; gp += n_cl) {
    const int lp = gp - I.pose_base;
    PoseRegs P;
    load_pose(I.poses + 12 * (size_t)lp, P);
    const float4* src = pose_tiles(I, lp) + tid + (size_t)t0 * kTile;
    const int pose_passes = passes;
    const int lg = __ffs(pose_passes) - 1;
    uint32_t max_occupied = 0;
    bool full = false, overflowed = false;
    for (int pass = 0; pass < pose_passes; ++pass) {
      if (!full && nt_mine > 0) {
        if (lg == 0) sweep_pose<kVW, kRot, false, true, true, 2>(S, a, vc, P, src, nt_mine, 0, 0u, ring, lane_lt, cut);
        else sweep_pose<kVW, kRot, true, true, true, 2>(S, a, vc, P, src, nt_mine, lg, (uint32_t)pass, ring, lane_lt, cut);
      }
      cluster_sync();  // every run of both CTAs is in the table or in an overflow list
      if (!full && *(volatile uint32_t*)&S.flags[2] != 0u) insert_overflow_cl<kVW>(S, a, I.gc);
      cluster_sync();  // the overflow inserts of both CTAs are done
      overflowed = overflowed || S.flags[1] != 0u || ldc32(c_peer - kFlagFull) != 0u;
      full = full || overflowed;
      scan_table<kVW, false, 1>(S, I.gc, I, wide, a.wide_count, T, lp, full);  // this CTA's half
      __syncthreads();
      cluster_sync();  // both scans are done: the occupied counts and wide flags are final
      max_occupied = max(max_occupied, max(S.flags[0], ldc32(c_peer - kFlagOccupied)));
      note_wide<kVW>(S, a);
      full = full || S.flags[3] != 0u || ldc32(c_peer - kFlagWide) != 0u;
      cluster_sync();  // both have read the other's flags before they are reset
      if (tid == 0) {
        S.flags[0] = 0u;
        S.flags[2] = 0u;
        S.flags[3] = 0u;
      }
      __syncthreads();  // the resets before the next pass's drains count again
    }
    if (full) {  // finished later by the exact path
      reset_pose(S);
      if (tid == 0) {
        S.flags[1] = 0u;
        if (rank == 0u) a.redo_list[atomicAdd(a.redo_count, 1u)] = (uint32_t)gp;
      }
      if (overflowed && passes < kMaxPasses) passes *= 2;
      __syncthreads();
      cluster_sync();  // the full flags are reset before either CTA sweeps the next pose
      continue;
    }
    // the pose's histogram and box: the second CTA adds its partial ones into the first's
    if (rank == 1u) {
      const int KK = S.gc->K * S.gc->K;
      const uint32_t h0 = c_peer + (S.a_hist - S.a_key);
      for (int i = tid; i < KK; i += kThreads) {
        const uint32_t v = S.hist[i];
        if (v != 0u) redc_add(h0 + 4u * (uint32_t)i, v);
        S.hist[i] = 0u;
      }
      if (tid < 6) {
        const uint32_t b0 = c_peer + (S.a_box - S.a_key) + 4u * (uint32_t)tid;
        if (tid < 3) redc_min_s32(b0, S.box[tid]);
        else redc_max_s32(b0, S.box[tid]);
        S.box[tid] = tid < 3 ? INT_MAX : INT_MIN;
      }
    }
    cluster_sync();  // the first CTA holds the pose's histogram and box
    if (rank == 0u) emit_pose(S, I, lp);
    if (max_occupied > cap && passes < kMaxPasses) passes *= 2;  // crowded: more partitions next
  }
  if (tid == 0 && rank == 0u) {
    atomicMax(a.max_passes, (uint32_t)passes);
    if (I.item_passes) atomicMax(I.item_passes, (uint32_t)passes);
  }
  cluster_sync();  // neither CTA leaves while the other may still address its shared memory
}

// Poses that eval_kernel could not finish: plain sweeps; each run goes straight into the
// table with 64-bit side sums for voxels beyond the 32-bit bound; a full table restarts
// the pose with twice the key partitions.
template <int kVW, bool kRot>
__global__ void __launch_bounds__(kThreads, kCtasPerSm) redo_kernel(const __grid_constant__ EvalArgs a) {
  constexpr bool kVar = kVW > 1;
  extern __shared__ __align__(128) uint8_t smem_raw[];
  EvalSmem S;
  const int T = a.table_slots;
  eval_smem_layout(a.K, T, kVW, a.units != nullptr ? 2 : 1, &S, smem_raw);
  const int tid = threadIdx.x;
  const uint32_t nb = (uint32_t)T >> 2;
  unsigned long long* wide = a.wide + (size_t)blockIdx.x * 2u * (size_t)T;
  const uint32_t n_redo = *(volatile const uint32_t*)a.redo_count;
  if (blockIdx.x >= n_redo) return;
  init_smem<kVW>(S, T, a.K * a.K, 1);
  __syncthreads();
  int passes_used = 1;
  for (uint32_t i = blockIdx.x; i < n_redo; i += gridDim.x) {
    const int gp = (int)a.redo_list[i];
    const int it = item_of(a, gp);
    select_item(S, a, it);
    const EvalItem& I = a.items[it];
    const int lp = gp - I.pose_base;
    const VoxelConst vc = voxel_const<3>(*S.gc);
    const uint32_t run_lim = S.gc->nlim;  // runs with 32-bit sums of dz and dz^2, cut at nlim
    PoseRegs P;
    load_pose(I.poses + 12 * (size_t)lp, P);
    const float4* src = pose_tiles(I, lp) + tid;
    // Start from the item's partition count: a pose redone for its wide sums needs no more,
    // one redone for a full table doubles below until its partitions fit.
    int passes = max(1, min(I.passes0 > 0 ? I.passes0 : a.passes0, kMaxPasses));
    int pass = 0;
    while (pass < passes) {
      const int lg = __ffs(passes) - 1;
      // plain runs: count n, S1 (two's complement) and S2, cut at nlim points
      uint32_t rkey = kEmptyKey, rn = 0u, rs1 = 0u, rs2 = 0u;
      uint32_t bad = 0u;
      for (int t = 0; t < I.n_tiles; ++t) {
        float4 v[kPPT];
        load_tile(src, t, v);
#pragma unroll
        for (int j = 0; j < kPPT; ++j) {
          uint32_t key;
          int dz;
          point_key<kRot>(vc, P, v[j], key, dz);
          if (lg > 0 && key != kEmptyKey && ((key * 0x85EBCA77u) >> (32 - lg)) != (uint32_t)pass) key = kEmptyKey;
          // dz is meaningful inside the grid only (the bound holds there; a cheap assertion)
          bad |= (uint32_t)(key != kEmptyKey && (uint32_t)(dz + vc.dz_bound) > (uint32_t)(2 * vc.dz_bound));
          if (key != rkey || (kVar && rn >= run_lim)) {
            if (rkey != kEmptyKey && rn != 0u) add_run<kVW>(S, wide, rkey, rn, (int)rs1, rs2, nb);
            rkey = key;
            rn = rs1 = rs2 = 0u;
          }
          rn += 1u;
          rs1 += (uint32_t)dz;
          rs2 += (uint32_t)(dz * dz);
        }
      }
      if (bad) atomicOr(a.err, kErrDzBound);
      if (rkey != kEmptyKey && rn != 0u) add_run<kVW>(S, wide, rkey, rn, (int)rs1, rs2, nb);
      __syncthreads();
      const bool full = S.flags[1] != 0u;
      scan_table<kVW, true, 1>(S, *S.gc, I, wide, a.wide_count, T, lp, full);
      __syncthreads();
      if (tid == 0) S.flags[0] = 0u;
      if (full) {
        reset_pose(S);
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
    passes_used = max(passes_used, passes);
    emit_pose(S, I, lp);
  }
  if (tid == 0) atomicMax(a.max_passes, (uint32_t)passes_used);
}

// Stream (stretch of consecutive scan points) walked by thread `tid`: lane l of warp w takes
// stream l * kWarps + w, so every warp samples the whole scan and the warps of a CTA finish
// their sweeps (and drains) at about the same time.
__device__ __forceinline__ int stream_of(int tid) { return (tid & 31) * kWarps + (tid >> 5); }

// xyz -> float4 tiles, optionally one rotated copy per rotation.  Tile t, position
// j*kThreads + s holds point s*L + kPPT*t + j of B (L = kPPT * tiles): stream s visits
// consecutive points of B, kPPT per tile.  Block (t, g) writes tile t of the copies of
// rotations g*kPackRot ... : each point is gathered once and rotated for all of them, and
// every copy's tile is written with coalesced stores.
constexpr int kPackRot = 8;
constexpr int kPackThreads = 256;

__global__ void __launch_bounds__(kPackThreads) pack_points_kernel(const float* __restrict__ xyz, int64_t n,
                                                                   int64_t n_out, const float* __restrict__ rots,
                                                                   int n_rot, float4* out) {
  const float nan = __int_as_float(0x7fc00000);
  const float inf = __int_as_float(0x7f800000);
  const int64_t L = n_out / kThreads;  // points per stream
  const int64_t t = blockIdx.x;
  const int r0 = (int)blockIdx.y * kPackRot;
  const int r1 = rots != nullptr ? min(n_rot, r0 + kPackRot) : 1;
  for (int slot = threadIdx.x; slot < kTile; slot += blockDim.x) {
    const int j = slot / kThreads;
    const int64_t src = (int64_t)stream_of(slot - j * kThreads) * L + (int64_t)kPPT * t + j;
    const bool have = src < n;
    const float x = have ? xyz[3 * src] : 0.0f, y = have ? xyz[3 * src + 1] : 0.0f, z = have ? xyz[3 * src + 2] : 0.0f;
    const int64_t i = t * kTile + slot;
    for (int r = r0; r < r1; ++r) {
      // padding: NaN for raw tiles (the in-kernel rotation keeps NaN), +inf for rotated copies
      float4 v = rots != nullptr ? make_float4(inf, inf, inf, 0.0f) : make_float4(nan, nan, nan, 0.0f);
      if (have) {
        if (rots != nullptr) {
          float R[9];
#pragma unroll
          for (int k = 0; k < 9; ++k) R[k] = __ldg(rots + 9 * r + k);
          rotate_point(R, x, y, z, v.x, v.y, v.z);
          // a non-finite coordinate can only come from a non-finite point (or an overflow),
          // which the voxel map drops under every pose; +inf keeps it dropped
          if (!(isfinite(v.x) && isfinite(v.y) && isfinite(v.z))) v = make_float4(inf, inf, inf, 0.0f);
        } else {
          v.x = x;
          v.y = y;
          v.z = z;
        }
      }
      store_point(out + (size_t)r * n_out, i, v.x, v.y, v.z);
    }
  }
}

// The same packing for every tile copy of a batch (one copy per blockIdx.y).
__global__ void pack_batch_kernel(const PackCopy* __restrict__ copies) {
  const PackCopy& c = copies[blockIdx.y];
  const float nan = __int_as_float(0x7fc00000);
  const float inf = __int_as_float(0x7f800000);
  const bool rot = c.rotate != 0;
  float R[9];
  for (int i = 0; i < 9; ++i) R[i] = c.R[i];
  const int64_t L = c.n_out / kThreads;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < c.n_out; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t t = i / kTile;
    const int pos = (int)(i - t * kTile);
    const int j = pos / kThreads;
    const int64_t src = (int64_t)stream_of(pos - j * kThreads) * L + (int64_t)kPPT * t + j;
    const float pad = rot ? inf : nan;
    float4 v = make_float4(pad, pad, pad, 0.0f);
    if (src < c.n) {
      const float x = c.xyz[3 * src], y = c.xyz[3 * src + 1], z = c.xyz[3 * src + 2];
      if (rot) {
        rotate_point(R, x, y, z, v.x, v.y, v.z);
        if (!(isfinite(v.x) && isfinite(v.y) && isfinite(v.z))) v = make_float4(inf, inf, inf, 0.0f);
      } else {
        v.x = x;
        v.y = y;
        v.z = z;
      }
    }
    store_point(c.out, i, v.x, v.y, v.z);
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

__global__ void __launch_bounds__(kComposeThreads) compose_kernel(const __grid_constant__ EvalArgs a) {
  __shared__ uint32_t h[kMaxSymbols * kMaxSymbols];
  __shared__ long long cntA[kMaxSymbols];
  __shared__ float red[kComposeThreads / 32];
  const int gp = blockIdx.x;
  const int tid = threadIdx.x;
  const EvalItem& I = a.items[item_of(a, gp)];
  const GridConst& gc = I.gc;
  const int lp = gp - I.pose_base;
  const int K = gc.K, KK = K * K;
  const int32_t* bb = I.out_box + 6 * (size_t)lp;
  int lo[3], hi[3];
  bool empty = false;
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    lo[i] = max(gc.boxA[i], bb[i]);
    hi[i] = min(gc.boxA[3 + i], bb[3 + i]);
    empty |= lo[i] > hi[i];
  }
  const long long N = empty ? 0 : (long long)(hi[0] - lo[0] + 1) * (hi[1] - lo[1] + 1) * (hi[2] - lo[2] + 1);
  for (int i = tid; i < KK; i += kComposeThreads) h[i] = empty ? 0u : I.out_c[(size_t)lp * KK + i];
  if (!empty && tid >= 1 && tid < K) {
    // count of A symbol `tid` over the box from its 3-D prefix sums (8 corners)
    const int X1 = gc.X + 1, Y1 = gc.Y + 1;
    const int32_t* S = I.sat + (size_t)(tid - 1) * (size_t)(gc.Z + 1) * Y1 * X1;
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
    I.mi[lp] = mi;
    const uint32_t u = __float_as_uint(mi);
    const uint32_t ord = (u & 0x80000000u) ? ~u : (u | 0x80000000u);
    atomicMax(I.best, ((unsigned long long)ord << 32) | (unsigned long long)(0xFFFFFFFFu - (uint32_t)lp));
  }
  if (I.hist != nullptr)
    for (int i = tid; i < KK; i += kComposeThreads) I.hist[(size_t)lp * KK + i] = h[i];
}

__global__ void argmax_finalize_kernel(const EvalItem* items, int n_items) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n_items) return;
  const unsigned long long b = *items[i].best;
  *items[i].argmax = (b == 0ull) ? -1 : (int64_t)(0xFFFFFFFFu - (uint32_t)(b & 0xFFFFFFFFull));
}

template <int kVW, bool kRot>
cudaError_t setup_t(int smem) {
  cudaError_t e = cudaFuncSetAttribute(eval_kernel<kVW, kRot, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(eval_kernel<kVW, kRot, true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(eval_kernel<kVW, kRot, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(redo_kernel<kVW, kRot>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e == cudaSuccess && !kRot)
    e = cudaFuncSetAttribute(eval_pair_kernel<kVW>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e == cudaSuccess && !kRot)
    e = cudaFuncSetAttribute(eval_pair_kernel<kVW, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(eval_cluster_kernel<kVW, kRot>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  return e;
}

template <int kVW, bool kRot>
cudaError_t launch_eval_t(const EvalArgs& a, int n_ctas, size_t smem, cudaStream_t s) {
  if (a.cluster) {  // 2-CTA clusters: an even grid, one item
    if (a.item_start != nullptr || n_ctas < 2 || (n_ctas & 1)) return cudaErrorInvalidValue;
    eval_cluster_kernel<kVW, kRot><<<n_ctas, kThreads, smem, s>>>(a);
  } else {
    auto* k = a.item_start != nullptr ? eval_kernel<kVW, kRot, false>
              : a.spill != nullptr      ? eval_kernel<kVW, kRot, true, true>
                                        : eval_kernel<kVW, kRot, true>;
    k<<<n_ctas, kThreads, smem, s>>>(a);
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  redo_kernel<kVW, kRot><<<n_ctas, kThreads, smem, s>>>(a);
  return cudaGetLastError();
}

int eval_tile_points() { return kTile; }
int eval_ovf_cap() { return kOvfCap; }
int eval_min_tiles() { return kMinTiles; }

size_t eval_smem_bytes(int K, int table_slots, int vw, int np) {
  return eval_smem_layout(K, table_slots, vw, np, nullptr, nullptr);
}

int eval_table_slots_for(int K, int vw, size_t smem_budget, int np) {
  if (kCtasPerSm > 1) {  // share the SM's shared memory between its resident CTAs
    int dev = 0, per_sm = 0, reserved = 0;
    if (cudaGetDevice(&dev) == cudaSuccess &&
        cudaDeviceGetAttribute(&per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev) == cudaSuccess &&
        cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, dev) == cudaSuccess)
      smem_budget = std::min(smem_budget, (size_t)(per_sm / kCtasPerSm - reserved));
  }
  int lo = 32;
  while (eval_smem_bytes(K, lo + 32, vw, np) <= smem_budget && lo < (1 << 16)) lo += 32;
  return lo;
}

template <int kVW>
cudaError_t launch_pair_t(const EvalArgs& a, int n_ctas, size_t smem, cudaStream_t s) {
  if (a.spill != nullptr) eval_pair_kernel<kVW, true><<<n_ctas, kThreads, smem, s>>>(a);
  else eval_pair_kernel<kVW><<<n_ctas, kThreads, smem, s>>>(a);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  redo_kernel<kVW, false><<<n_ctas, kThreads, smem, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_eval(const EvalArgs& a, int n_ctas, int vw, bool rotate, cudaStream_t s) {
  const size_t smem = eval_smem_bytes(a.K, a.table_slots, vw, a.units != nullptr ? 2 : 1);
  if (a.units != nullptr) {  // pose pairs: pre-rotated tiles of one item only
    if (rotate || a.item_start != nullptr) return cudaErrorInvalidValue;
    switch (vw) {
      case 1: return launch_pair_t<1>(a, n_ctas, smem, s);
      case 2: return launch_pair_t<2>(a, n_ctas, smem, s);
      case 3: return launch_pair_t<3>(a, n_ctas, smem, s);
      default: return cudaErrorInvalidValue;
    }
  }
  switch (vw) {
    case 1: return rotate ? launch_eval_t<1, true>(a, n_ctas, smem, s) : launch_eval_t<1, false>(a, n_ctas, smem, s);
    case 2: return rotate ? launch_eval_t<2, true>(a, n_ctas, smem, s) : launch_eval_t<2, false>(a, n_ctas, smem, s);
    case 3: return rotate ? launch_eval_t<3, true>(a, n_ctas, smem, s) : launch_eval_t<3, false>(a, n_ctas, smem, s);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t eval_setup() {
  static std::mutex mu;
  static bool done[64] = {};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(mu);
  if (done[dev]) return cudaSuccess;
  int smem = 0;
  e = cudaDeviceGetAttribute(&smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (e != cudaSuccess) return e;
  if ((e = setup_t<1, true>(smem)) != cudaSuccess) return e;
  if ((e = setup_t<1, false>(smem)) != cudaSuccess) return e;
  if ((e = setup_t<2, true>(smem)) != cudaSuccess) return e;
  if ((e = setup_t<2, false>(smem)) != cudaSuccess) return e;
  if ((e = setup_t<3, true>(smem)) != cudaSuccess) return e;
  if ((e = setup_t<3, false>(smem)) != cudaSuccess) return e;
  done[dev] = true;
  return cudaSuccess;
}

cudaError_t launch_pack_batch(const PackCopy* copies, int n_copies, int64_t max_out, cudaStream_t s) {
  if (n_copies <= 0) return cudaSuccess;
  const int threads = 256;
  int64_t bx = (max_out + threads - 1) / threads;
  if (bx > 1024) bx = 1024;
  if (bx < 1) bx = 1;
  pack_batch_kernel<<<dim3((unsigned)bx, (unsigned)n_copies), threads, 0, s>>>(copies);
  return cudaGetLastError();
}

cudaError_t launch_pack_points(const float* xyz, int64_t n, int64_t n_out, const float* rots, int n_rot, float4* out,
                               cudaStream_t s) {
  const int64_t n_tiles = n_out / kTile;
  const int groups = rots != nullptr && n_rot > 0 ? (n_rot + kPackRot - 1) / kPackRot : 1;
  if (n_tiles < 1 || n_tiles > INT_MAX || groups > 65535) return cudaErrorInvalidValue;
  pack_points_kernel<<<dim3((unsigned)n_tiles, (unsigned)groups), kPackThreads, 0, s>>>(xyz, n, n_out, rots,
                                                                                         n_rot, out);
  return cudaGetLastError();
}

cudaError_t launch_compose(const EvalArgs& a, cudaStream_t s) {
  if (a.P <= 0) return cudaSuccess;
  compose_kernel<<<a.P, kComposeThreads, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_argmax_finalize(const EvalItem* items, int n_items, cudaStream_t s) {
  if (n_items <= 0) return cudaSuccess;
  argmax_finalize_kernel<<<(n_items + 127) / 128, 128, 0, s>>>(items, n_items);
  return cudaGetLastError();
}

}  // namespace

const EvalKernels& MI_EVAL_SHAPE_FN() {
  static const EvalKernels k{MI_STR(MI_EVAL_SHAPE_FN), kThreads, kPPT, kCtasPerSm, eval_tile_points, eval_ovf_cap, eval_min_tiles,
                             eval_smem_bytes, eval_table_slots_for, eval_setup, launch_eval, launch_pack_points,
                             launch_pack_batch, launch_compose, launch_argmax_finalize};
  return k;
}

}  // namespace mialign
