// Device lowering engine: Celerity-style tasks -> per-node instruction graphs.
//
// One warp owns one virtual node of one program (each node generates only its
// own instruction graph, paper Sec. 2.4). The node's region maps live in HBM
// as structure-of-arrays box tables, scanned coalesced 32 entries at a time;
// variable numbers of boxes, instructions and edges are emitted with warp
// ballot / prefix-sum compaction. The warp's control flow is uniform: every
// lane follows the same path and holds the same scalars.
//
// Steps (paper passages):
//   a1 chunk split + device assignment ... Sec. 3.1
//   a2 range mappers ..................... Sec. 2.1, Listing 1, Listing 2
//   a3 push / await push ................. Sec. 2.4, Sec. 3.4
//   a4 allocation + lookahead merge ...... Sec. 3.2, Sec. 4.3
//   a5 coherence copies .................. Sec. 3.3 (producer x consumer split)
//   a6 sends, a7 receives ................ Sec. 3.4
//   a8 dependencies ...................... Fig. 5 legend, Sec. 3.5, Sec. 4.2
//   a9 horizon / epoch compaction ........ Sec. 3.5
//   a10 emission ......................... Sec. 4.1 (topological emission order)
//   debug checks ......................... Sec. 4.4
#include <cuda_runtime.h>

#include "igs_internal.h"

namespace igs {
namespace {

constexpr uint32_t FULL = 0xffffffffu;

// scratch table slots
enum : int {
  S_CH = 0, S_MP = 1, S_CH2 = 2, S_MP2 = 3, S_T0 = 4, S_T1 = 5, S_T2 = 6, S_T3 = 7, S_T4 = 8, S_T5 = 9,
  S_CL = 10, S_DEP = 11, S_CAN = 12, S_RG = 13
};

struct Bx {
  uint32_t lo[3], hi[3];
};

// This thread's lane (a register read; the copy in Ctx would be a memory load).
__device__ __forceinline__ uint32_t laneid() {
  uint32_t l;
  asm("mov.u32 %0, %%laneid;" : "=r"(l));
  return l;
}
__device__ __forceinline__ uint32_t lanemask_lt() {
  uint32_t m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

__device__ __forceinline__ bool bx_empty(const Bx& b) {
  return b.lo[0] >= b.hi[0] || b.lo[1] >= b.hi[1] || b.lo[2] >= b.hi[2];
}
__device__ __forceinline__ Bx bx_isect(const Bx& a, const Bx& b) {
  Bx r;
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    r.lo[d] = max(a.lo[d], b.lo[d]);
    r.hi[d] = min(a.hi[d], b.hi[d]);
  }
  return r;
}
__device__ __forceinline__ bool bx_overlap(const Bx& a, const Bx& b) {
#pragma unroll
  for (int d = 0; d < 3; ++d)
    if (max(a.lo[d], b.lo[d]) >= min(a.hi[d], b.hi[d])) return false;
  return true;
}
__device__ __forceinline__ bool bx_contains(const Bx& o, const Bx& i) {
#pragma unroll
  for (int d = 0; d < 3; ++d)
    if (i.lo[d] < o.lo[d] || i.hi[d] > o.hi[d]) return false;
  return true;
}
__device__ __forceinline__ Bx bx_union(const Bx& a, const Bx& b) {
  Bx r;
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    r.lo[d] = min(a.lo[d], b.lo[d]);
    r.hi[d] = max(a.hi[d], b.hi[d]);
  }
  return r;
}
__device__ __forceinline__ bool bx_less(const Bx& a, const Bx& b) {
#pragma unroll
  for (int d = 0; d < 3; ++d)
    if (a.lo[d] != b.lo[d]) return a.lo[d] < b.lo[d];
#pragma unroll
  for (int d = 0; d < 3; ++d)
    if (a.hi[d] != b.hi[d]) return a.hi[d] < b.hi[d];
  return false;
}
__device__ __forceinline__ uint64_t bx_volume(const Bx& b) {
  if (bx_empty(b)) return 0;
  return (uint64_t)(b.hi[0] - b.lo[0]) * (b.hi[1] - b.lo[1]) * (b.hi[2] - b.lo[2]);
}
// a \ b: up to six disjoint pieces; a itself when they do not overlap.
__device__ __forceinline__ int bx_minus(const Bx& a, const Bx& b, Bx* out) {
  if (!bx_overlap(a, b)) {
    out[0] = a;
    return 1;
  }
  int k = 0;
  Bx rem = a;
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    if (rem.lo[d] < b.lo[d]) {
      out[k] = rem;
      out[k].hi[d] = b.lo[d];
      ++k;
      rem.lo[d] = b.lo[d];
    }
    if (rem.hi[d] > b.hi[d]) {
      out[k] = rem;
      out[k].lo[d] = b.hi[d];
      ++k;
      rem.hi[d] = b.hi[d];
    }
  }
  return k;
}
// The pieces of a \ b for overlapping a and b, in bx_minus's order: their
// number, and each piece handed to f(index, piece) as it is formed (no array
// of pieces, which would live in local memory).
__device__ __forceinline__ int bx_minus_count(const Bx& a, const Bx& b) {
  int k = 0;
#pragma unroll
  for (int d = 0; d < 3; ++d) k += (a.lo[d] < b.lo[d]) + (a.hi[d] > b.hi[d]);
  return k;
}
template <class F>
__device__ __forceinline__ void bx_minus_each(const Bx& a, const Bx& b, F f) {
  int k = 0;
  Bx rem = a;
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    if (rem.lo[d] < b.lo[d]) {
      Bx o = rem;
      o.hi[d] = b.lo[d];
      f(k++, o);
      rem.lo[d] = b.lo[d];
    }
    if (rem.hi[d] > b.hi[d]) {
      Bx o = rem;
      o.lo[d] = b.hi[d];
      f(k++, o);
      rem.hi[d] = b.hi[d];
    }
  }
}
// Two boxes whose union is a box (adjacent along one dimension, equal in the others).
__device__ __forceinline__ bool bx_mergeable(const Bx& a, const Bx& b) {
  int adj = -1;
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    if (a.lo[d] == b.lo[d] && a.hi[d] == b.hi[d]) continue;
    if (adj >= 0) return false;
    if (a.hi[d] == b.lo[d] || b.hi[d] == a.lo[d]) adj = d;
    else return false;
  }
  return adj >= 0;
}

// ---- tables ----------------------------------------------------------------

__device__ __forceinline__ uint32_t& FLD(const Table& t, int f, uint32_t i) { return t.base[(size_t)i * F_COUNT + f]; }
__device__ __forceinline__ uint32_t t_key(const Table& t, uint32_t i) { return FLD(t, F_KEY, i); }
__device__ __forceinline__ uint32_t t_v(const Table& t, int k, uint32_t i) { return FLD(t, F_V + k, i); }
__device__ __forceinline__ Bx t_box(const Table& t, uint32_t i) {
  const uint4* e = reinterpret_cast<const uint4*>(t.base + (size_t)i * F_COUNT);
  const uint4 a = e[0], b = e[1];
  Bx r;
  r.lo[0] = a.y;
  r.lo[1] = a.z;
  r.lo[2] = a.w;
  r.hi[0] = b.x;
  r.hi[1] = b.y;
  r.hi[2] = b.z;
  return r;
}
__device__ __forceinline__ void t_put(const Table& t, uint32_t i, uint32_t key, const Bx& b, uint32_t v0, uint32_t v1,
                                      uint32_t v2) {
  uint4* e = reinterpret_cast<uint4*>(t.base + (size_t)i * F_COUNT);
  e[0] = make_uint4(key, b.lo[0], b.lo[1], b.lo[2]);
  e[1] = make_uint4(b.hi[0], b.hi[1], b.hi[2], v0);
  e[2] = make_uint4(v1, v2, 0u, 0u);
}
__device__ __forceinline__ void t_kill(const Table& t, uint32_t i) { FLD(t, F_KEY, i) = DEAD; }

// A whole entry, read with three independent 16-byte loads (one round trip
// instead of a chain of dependent word loads).
struct Ent {
  uint32_t key;
  Bx b;
  uint32_t v0, v1, v2;
};
__device__ __forceinline__ Ent t_ent(const Table& t, uint32_t i) {
  const uint4* e = reinterpret_cast<const uint4*>(t.base + (size_t)i * F_COUNT);
  const uint4 a = e[0], b = e[1], c = e[2];
  Ent r;
  r.key = a.x;
  r.b.lo[0] = a.y;
  r.b.lo[1] = a.z;
  r.b.lo[2] = a.w;
  r.b.hi[0] = b.x;
  r.b.hi[1] = b.y;
  r.b.hi[2] = b.z;
  r.v0 = b.w;
  r.v1 = c.x;
  r.v2 = c.y;
  return r;
}

struct Acc {
  const Table* t;
  uint32_t from, to, alloc, mode;
};

struct Ctx {
  NodeDev* nd;
  const ProgDev* pg;
  uint32_t lane, err, err_info;
  uint32_t node, N, D;
  uint32_t epoch, last_horizon, last_sync, next_msg, n_alloc, n_free, n_live, heap_top;
  uint32_t n_instr, n_edge, n_box, n_bind, n_diag, n_rej;
  uint32_t lookahead, q_head, q_count, q_hzn;
  Table qr;
  Table s[14];
  uint64_t map_reads, map_writes;
  int* lock;  // block's heap lock (shared memory) when several warps of the block lower, else null
  void* block;       // the block's shared control (BlockShared) when it has helper warps, else null
  uint32_t workers;  // warps sharing the kernel phase (1 = warp 0 alone)
  struct Stage* stage;  // emit into this staging area with provisional ids (coherence workers), else null
  bool helper;          // a helper warp (keeps off the node's profile counters)
  // item compiled straight from delivery: its chunks and mapped boxes are
  // still in S_CH / S_MP and it is known not to allocate (NONE otherwise)
  uint32_t fresh;
  struct Pipe* pipe;  // the block's pipeline with a front warp (warp 0 only), else null
  // dependencies on allocation snap_alloc come from copies of its writer /
  // reader tables (snap_tab, snap_n entries) instead (NONE: no copies)
  uint32_t snap_alloc;
  const uint32_t* snap_tab[2];
  uint32_t snap_n[2];
};

// Instructions a coherence worker emits before their final ids are known:
// provisional id = PROV | worker << 24 | index. Records carry their edges'
// range in bind_off / bind_cnt (staged instructions have no bindings).
constexpr uint32_t PROV = 0x80000000u;
struct Stage {
  igs_instruction* instrs;
  igs_edge* edges;
  igs_box* boxes;
  uint32_t* map;  // index -> final id (filled when warp 0 appends the records)
  uint32_t n_instr, n_edge, n_box, cap_instr, cap_edge, cap_box, id_base;
};

__device__ __forceinline__ void fail(Ctx& c, uint32_t code) {
  if (c.err == ST_OK) c.err = code;
}
// An internal failure records which check failed (err_info = site).
__device__ __forceinline__ void fail_internal(Ctx& c, uint32_t site) {
  if (c.err == ST_OK) {
    c.err = ST_INTERNAL;
    c.err_info = site;
  }
}
// A capacity failure records what ran out and its capacity for the host.
__device__ __forceinline__ void fail_cap(Ctx& c, CapKind what, uint32_t cap) {
  if (c.err == ST_OK) {
    c.err = ST_CAPACITY;
    c.err_info = ((uint32_t)what << 24) | (cap < 0xFFFFFFu ? cap : 0xFFFFFFu);
  }
}

// Phase cycle accounting (lane 0 adds to the node's counters).
enum Phase : int {
  PH_SPLIT = 0, PH_OVERLAP = 1, PH_A3 = 2, PH_ALLOCATING = 3, PH_P1 = 4, PH_P2 = 5, PH_P3 = 6, PH_P4 = 7,
  PH_P5 = 8, PH_REMOTE = 9, PH_SYNC = 10, PH_APPLY = 11, PH_TOTAL = 12, PH_EMIT = 13, PH_CANON = 14, PH_FIND = 15
};
struct PhaseTimer {
  long long t0;
};
__device__ __forceinline__ PhaseTimer pt_start() {
  PhaseTimer p;
  p.t0 = clock64();
  return p;
}

// Detail counters (cycles inside region-map primitives and parts of
// emission, call counts), compiled in with IGS_PROFILE_DETAIL only.
enum Detail : int {
  D_MERGE = 16, D_SUBTRACT = 17, D_QUERY = 18, D_COMPACT = 19, D_PROBE = 20, D_DEDUP = 21, D_RECORD = 22,
  D_APPLY = 23, N_MERGE = 24, N_MERGE_PROBE = 25, N_SUBTRACT = 26, N_EMIT = 27, N_PROBE_ENTRIES = 28, N_TIDY = 29,
  N_GROW = 30
};
#ifdef IGS_PROFILE_DETAIL
#define DT_START(v) PhaseTimer v = pt_start()
#define DT_LAP(v, ph) pt_lap(v, c, ph)
#define DT_COUNT(k, x)                          \
  do {                                          \
    if (laneid() == 0) c.nd->prof[k] += (x);      \
  } while (0)
#else
#define DT_START(v) \
  do {              \
  } while (0)
#define DT_LAP(v, ph) \
  do {                \
  } while (0)
#define DT_COUNT(k, x) \
  do {                 \
  } while (0)
#endif

// ---- the node's entry heap ---------------------------------------------------

__device__ __forceinline__ int heap_class(uint32_t entries) {
  int k = 0;
  while ((32u << k) < entries && k < kHeapClasses - 1) ++k;
  return k;
}

// A slab of at least `entries` entries (uniform); NONE when the heap is full.
// With several warps lowering one node, the heap (free lists and top, then
// kept in NodeDev) is shared: a warp takes the block's lock around every heap
// operation. The wait is bounded; a lock not obtained fails the node.
__device__ bool heap_lock(Ctx& c) {
  if (!c.lock) return true;
  uint32_t ok = 1;
  if (laneid() == 0) {
    uint32_t spins = 0;
    while (atomicCAS(c.lock, 0, 1) != 0) {
      if (++spins > (1u << 20)) {
        ok = 0;
        break;
      }
      __nanosleep(64);
    }
    __threadfence_block();
  }
  ok = __shfl_sync(FULL, ok, 0);
  if (!ok) fail(c, ST_TIMEOUT);
  return ok != 0;
}
__device__ void heap_unlock(Ctx& c) {
  if (!c.lock) return;
  __syncwarp();
  if (laneid() == 0) {
    __threadfence_block();
    atomicExch(c.lock, 0);
  }
  __syncwarp();
}

__device__ __noinline__ uint32_t heap_alloc(Ctx& c, uint32_t entries, uint32_t& cap) {
  const int k = heap_class(entries);
  cap = 32u << k;
  NodeDev* nd = c.nd;
  if (!heap_lock(c)) return NONE;
  volatile uint32_t* fh = nd->free_head;
  __syncwarp();
  const uint32_t head = fh[k];
  if (head != NONE) {
    const uint32_t next = reinterpret_cast<volatile uint32_t*>(nd->heap)[(size_t)head * F_COUNT];
    __syncwarp();
    if (laneid() == 0) fh[k] = next;
    heap_unlock(c);
    return head;
  }
  volatile uint32_t* vtop = &nd->heap_top;
  const uint32_t top = c.lock ? *vtop : c.heap_top;
  if ((uint64_t)top + cap > nd->cap_heap) {
    heap_unlock(c);
    fail_cap(c, CAP_HEAP, nd->cap_heap);
    return NONE;
  }
  if (c.lock) {
    __syncwarp();
    if (laneid() == 0) *vtop = top + cap;
  } else {
    c.heap_top = top + cap;
  }
  heap_unlock(c);
  return top;
}

__device__ void heap_free(Ctx& c, uint32_t off, uint32_t cap) {
  const int k = heap_class(cap);
  NodeDev* nd = c.nd;
  if (!heap_lock(c)) return;
  volatile uint32_t* fh = nd->free_head;
  __syncwarp();
  if (laneid() == 0) {
    reinterpret_cast<volatile uint32_t*>(nd->heap)[(size_t)off * F_COUNT] = fh[k];
    fh[k] = off;
  }
  heap_unlock(c);
}

__device__ __forceinline__ void t_publish(Ctx& c, Table& t) {
  if (t.dp && laneid() == 0) {
    t.dp[2] = t.n;
    t.dp[3] = t.live;
  }
}

// Grows a heap table (descriptor dp, n entries used of cap at base) to hold
// `need` entries: the entries move to a bigger slab at the same indices (a
// scan in progress stays valid). Returns the new slab; base is null on failure.
// Scalars in and out, so that callers keep their table header in registers.
struct Slab {
  uint32_t* base;
  uint32_t cap;
};
__device__ __noinline__ Slab t_grow_to(Ctx& c, uint32_t* dp, const uint32_t* base, uint32_t n, uint32_t cap,
                                       uint32_t need) {
  Slab r{nullptr, cap};
  if (!dp) {
    fail_cap(c, CAP_TABLE, cap);
    return r;
  }
  uint32_t ncap = 0;
  const uint32_t off = heap_alloc(c, need > 2 * cap ? need : 2 * cap, ncap);
  if (off == NONE) return r;
  DT_COUNT(N_GROW, 1);
  uint4* dst = reinterpret_cast<uint4*>(c.nd->heap + (size_t)off * F_COUNT);
  const uint4* src = reinterpret_cast<const uint4*>(base);
  const uint32_t words4 = n * (F_COUNT / 4);
  for (uint32_t i = laneid(); i < words4; i += 32) dst[i] = src[i];
  __syncwarp();
  heap_free(c, dp[0], cap);
  if (laneid() == 0) {
    dp[0] = off;
    dp[1] = ncap;
  }
  __syncwarp();
  r.base = c.nd->heap + (size_t)off * F_COUNT;
  r.cap = ncap;
  return r;
}
__device__ __forceinline__ bool t_grow(Ctx& c, Table& t, uint32_t need) {
  const Slab g = t_grow_to(c, t.dp, t.base, t.n, t.cap, need);
  if (!g.base) return false;
  t.base = g.base;
  t.cap = g.cap;
  return true;
}

// Claims one slot per predicated lane (all lanes call). NONE on overflow.
__device__ __forceinline__ uint32_t t_claim(Ctx& c, Table& t, bool pred) {
  const uint32_t m = __ballot_sync(FULL, pred);
  const uint32_t slot = t.n + __popc(m & lanemask_lt());
  const uint32_t nn = t.n + __popc(m);
  if (nn > t.cap && !t_grow(c, t, nn)) return NONE;
  t.n = nn;
  t.live += __popc(m);
  c.map_writes += __popc(m);
  t_publish(c, t);
  return pred ? slot : NONE;
}
// Claims one slot per predicated lane (all lanes call); false (every lane)
// when the table could not grow.
__device__ __forceinline__ bool t_claim_ok(Ctx& c, Table& t, bool pred, uint32_t& slot) {
  const uint32_t m = __ballot_sync(FULL, pred);
  slot = t.n + __popc(m & lanemask_lt());
  const uint32_t nn = t.n + __popc(m);
  if (nn > t.cap && !t_grow(c, t, nn)) return false;
  t.n = nn;
  t.live += __popc(m);
  c.map_writes += __popc(m);
  t_publish(c, t);
  return true;
}
// Claims k consecutive slots per lane; returns this lane's first slot.
__device__ __forceinline__ uint32_t t_claim_n(Ctx& c, Table& t, uint32_t k) {
  uint32_t excl, total;
  if (!__any_sync(FULL, k >= 8u)) {
    // counts below 8 (box pieces): prefix sums from three bit-plane ballots
    const uint32_t lt = lanemask_lt();
    const uint32_t b0 = __ballot_sync(FULL, k & 1u), b1 = __ballot_sync(FULL, k & 2u),
                   b2 = __ballot_sync(FULL, k & 4u);
    excl = __popc(b0 & lt) + 2 * __popc(b1 & lt) + 4 * __popc(b2 & lt);
    total = __popc(b0) + 2 * __popc(b1) + 4 * __popc(b2);
  } else {
    uint32_t x = k;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(FULL, x, o);
      if ((int)laneid() >= o) x += y;
    }
    total = __shfl_sync(FULL, x, 31);
    excl = x - k;
  }
  const uint32_t first = t.n + excl;
  if (t.n + total > t.cap && !t_grow(c, t, t.n + total)) return NONE;
  t.n += total;
  t.live += total;
  c.map_writes += total;
  t_publish(c, t);
  return first;
}

__device__ __forceinline__ void t_reset(Table& t) {
  t.n = 0;
  t.live = 0;
}

// k entries of t were marked dead.
__device__ __forceinline__ void t_dead(Ctx& c, Table& t, uint32_t k) {
  t.live -= k;
  t_publish(c, t);
}

template <class P>
__device__ __forceinline__ uint32_t warp_find_first(const Ctx& c, uint32_t n, P pred) {
  for (uint32_t base = 0; base < n; base += 32) {
    const uint32_t i = base + laneid();
    const bool h = i < n && pred(i);
    const uint32_t m = __ballot_sync(FULL, h);
    if (m) return base + __ffs(m) - 1;
  }
  return NONE;
}

__device__ __forceinline__ uint64_t warp_min64(uint64_t v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const uint64_t y = __shfl_xor_sync(FULL, v, o);
    v = y < v ? y : v;
  }
  return v;
}
__device__ __forceinline__ uint32_t warp_or(uint32_t v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v |= __shfl_xor_sync(FULL, v, o);
  return v;
}
__device__ __forceinline__ uint32_t warp_sum(uint32_t v) { return __reduce_add_sync(FULL, v); }
__device__ __forceinline__ uint64_t warp_sum64(uint64_t v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
  return v;
}
// Exclusive prefix sum over the lanes; total: the sum over all lanes.
__device__ __forceinline__ uint32_t warp_excl_scan(uint32_t v, uint32_t& total) {
  uint32_t x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(FULL, x, o);
    if ((int)laneid() >= o) x += y;
  }
  total = __shfl_sync(FULL, x, 31);
  return x - v;
}
__device__ __forceinline__ Bx warp_bbox(Bx b, bool valid) {
  Bx r;
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    uint32_t lo = valid ? b.lo[d] : 0xFFFFFFFFu, hi = valid ? b.hi[d] : 0u;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      lo = min(lo, __shfl_xor_sync(FULL, lo, o));
      hi = max(hi, __shfl_xor_sync(FULL, hi, o));
    }
    r.lo[d] = lo;
    r.hi[d] = hi;
  }
  return r;
}

__device__ void pt_lap(PhaseTimer& p, Ctx& c, int ph) {
  const long long t1 = clock64();
  if (laneid() == 0 && !c.helper) c.nd->prof[ph] += (uint64_t)(t1 - p.t0);
  p.t0 = t1;
}

// Stable in-place removal of dead entries of n entries at base; returns the
// number kept.
__device__ __noinline__ uint32_t t_compact_n(Ctx& c, uint32_t* tbase, uint32_t n) {
  DT_START(dt);
  Table t;
  t.base = tbase;
  t.n = n;
  uint32_t w = 0;
  for (uint32_t base = 0; base < t.n; base += 32) {
    const uint32_t i = base + laneid();
    const bool in = i < t.n;
    uint32_t key = DEAD, v0 = 0, v1 = 0, v2 = 0;
    Bx b{};
    if (in) {
      const Ent x = t_ent(t, i);
      key = x.key;
      b = x.b;
      v0 = x.v0;
      v1 = x.v1;
      v2 = x.v2;
    }
    __syncwarp();
    const bool live = in && key != DEAD;
    const uint32_t m = __ballot_sync(FULL, live);
    if (live) t_put(t, w + __popc(m & lanemask_lt()), key, b, v0, v1, v2);
    w += __popc(m);
    __syncwarp();
  }
  DT_LAP(dt, D_COMPACT);
  return w;
}
__device__ __forceinline__ void t_compact(Ctx& c, Table& t) {
  const uint32_t w = t_compact_n(c, t.base, t.n);
  t.n = w;
  t.live = w;
  t_publish(c, t);
  __syncwarp();
}

// Compacts a table once dead entries make up a fifth of it (scans cost the
// table's length, dead entries included; compaction keeps the entries' order).
__device__ __forceinline__ void t_tidy(Ctx& c, Table& t) {
  const uint32_t dead = t.n - t.live;
  if (dead > 4 && 4 * dead > t.live) {
    DT_COUNT(N_TIDY, 1);
    t_compact(c, t);
  }
}

__device__ Bx t_bbox(const Ctx& c, const Table& t, uint32_t from, uint32_t to) {
  Bx acc;
  acc.lo[0] = acc.lo[1] = acc.lo[2] = 0xFFFFFFFFu;
  acc.hi[0] = acc.hi[1] = acc.hi[2] = 0;
  for (uint32_t base = from; base < to; base += 32) {
    const uint32_t i = base + laneid();
    const bool in = i < to && t_key(t, i) != DEAD;
    Bx b{};
    if (in) b = t_box(t, i);
    Bx r = warp_bbox(b, in);
    acc = bx_union(acc, r);
  }
  return acc;
}

// Appends (entry n q) with the entry's values for every entry of `key`
// (NONE = any) that overlaps q and satisfies pred(values).
template <class P>
__device__ void t_query(Ctx& c, const Table& src, uint32_t key, const Bx& q, Table& out_ref, P pred) {
  DT_START(dt);
  Table out = out_ref;  // header in registers while scanning
  const uint32_t n = src.n;
  c.map_reads += n;
  for (uint32_t base = 0; base < n; base += 32) {
    const uint32_t i = base + laneid();
    bool hit = false;
    Bx is{};
    uint32_t v0 = 0, v1 = 0, v2 = 0;
    if (i < n) {
      const Ent e = t_ent(src, i);
      if (e.key != DEAD && (key == NONE || e.key == key)) {
        is = bx_isect(e.b, q);
        if (!bx_empty(is)) {
          v0 = e.v0;
          v1 = e.v1;
          v2 = e.v2;
          hit = pred(v0, v1, v2);
        }
      }
    }
    if (!__any_sync(FULL, hit)) continue;
    uint32_t s;
    if (!t_claim_ok(c, out, hit, s)) break;
    if (hit) t_put(out, s, 0, is, v0, v1, v2);
  }
  __syncwarp();
  out_ref = out;
  DT_LAP(dt, D_QUERY);
}

// Removes box r from every entry of `key` (NONE = any) that matches the
// optional value filter; the remainders keep their values.
__device__ __forceinline__ void t_subtract(Ctx& c, Table& t_ref, uint32_t key, const Bx& r, uint32_t vfilter = NONE) {
  DT_START(dt);
  DT_COUNT(N_SUBTRACT, 1);
  Table t = t_ref;  // header in registers while scanning
  t_tidy(c, t);
  const uint32_t n0 = t.n;
  for (uint32_t base = 0; base < n0; base += 32) {
    const uint32_t i = base + laneid();
    bool hit = false;
    uint32_t k = DEAD, v0 = 0, v1 = 0, v2 = 0;
    Bx e{};
    if (i < n0) {
      const Ent x = t_ent(t, i);
      k = x.key;
      if (k != DEAD && (key == NONE || k == key)) {
        e = x.b;
        v0 = x.v0;
        v1 = x.v1;
        v2 = x.v2;
        hit = bx_overlap(e, r) && (vfilter == NONE || v0 == vfilter);
      }
    }
    const uint32_t hits = __ballot_sync(FULL, hit);
    if (!hits) continue;  // nothing to remove in these 32 entries
    const int np = hit ? bx_minus_count(e, r) : 0;
    t_dead(c, t, __popc(hits));
    const uint32_t first = t_claim_n(c, t, (uint32_t)np);
    if (first == NONE) break;  // the table could not grow (status set)
    if (hit) {
      t_kill(t, i);
      bx_minus_each(e, r, [&](int j, const Bx& pb) { t_put(t, first + j, k, pb, v0, v1, v2); });
    }
  }
  __syncwarp();
  t_ref = t;
  DT_LAP(dt, D_SUBTRACT);
}

// value[vidx] |= bits on box r for entries of `key` (the table's header in
// and out by value).
__device__ __noinline__ Table t_or_v(Ctx& c, Table t, uint32_t key, const Bx& r, int vidx, uint32_t bits) {
  t_tidy(c, t);
  const uint32_t n0 = t.n;
  for (uint32_t base = 0; base < n0; base += 32) {
    const uint32_t i = base + laneid();
    bool hit = false;
    uint32_t v[3] = {0, 0, 0};
    Bx e{};
    uint32_t k = DEAD;
    if (i < n0) {
      const Ent x = t_ent(t, i);
      k = x.key;
      if (k != DEAD && (key == NONE || k == key)) {
        e = x.b;
        v[0] = x.v0;
        v[1] = x.v1;
        v[2] = x.v2;
        hit = bx_overlap(e, r) && (v[vidx] & bits) != bits;
      }
    }
    const uint32_t hits = __ballot_sync(FULL, hit);
    if (!hits) continue;
    const int np = hit ? bx_minus_count(e, r) : 0;
    t_dead(c, t, __popc(hits));
    const uint32_t first = t_claim_n(c, t, hit ? (uint32_t)np + 1 : 0u);
    if (first == NONE) break;  // the table could not grow (status set)
    if (hit) {
      t_kill(t, i);
      bx_minus_each(e, r, [&](int j, const Bx& pb) { t_put(t, first + j, k, pb, v[0], v[1], v[2]); });
      v[vidx] |= bits;
      t_put(t, first + np, k, bx_isect(e, r), v[0], v[1], v[2]);
    }
  }
  __syncwarp();
  return t;
}
__device__ __forceinline__ void t_or(Ctx& c, Table& t, uint32_t key, const Bx& r, int vidx, uint32_t bits) {
  t = t_or_v(c, t, key, r, vidx, bits);
}

// Sets the values of box r for `key`.
__device__ __forceinline__ void t_set(Ctx& c, Table& t_ref, uint32_t key, const Bx& r, uint32_t v0, uint32_t v1, uint32_t v2) {
  Table t = t_ref;
  t_subtract(c, t, key, r);
  uint32_t s;
  if (!c.err && t_claim_ok(c, t, laneid() == 0, s) && laneid() == 0) t_put(t, s, key == NONE ? 0u : key, r, v0, v1, v2);
  __syncwarp();
  t_ref = t;
}

// Merges entries from index `from` on with equal key and values into
// adjacent entries whose union is a box (keeps the tables small).
__device__ __noinline__ Table t_merge_from_v(Ctx& c, Table t, uint32_t from) {
  DT_START(dt);
  DT_COUNT(N_MERGE, 1);
  for (uint32_t i = from; i < t.n; ++i) {
    uint32_t cand = i;
    for (int guard = 0; guard < 4096; ++guard) {
      DT_COUNT(N_MERGE_PROBE, 1);
      const Ent ce = t_ent(t, cand);
      const uint32_t k = ce.key;
      if (k == DEAD) break;
      const Bx e = ce.b;
      const uint32_t v0 = ce.v0, v1 = ce.v1, v2 = ce.v2;
      Bx jb{};
      const uint32_t j = warp_find_first(c, t.n, [&](uint32_t x) {
        const Ent f = t_ent(t, x);
        const bool m = x != cand && f.key == k && f.v0 == v0 && f.v1 == v1 && f.v2 == v2 && bx_mergeable(e, f.b);
        if (m) jb = f.b;
        return m;
      });
      if (j == NONE) break;
      const uint32_t src_lane = (j & 31u);
      Bx jbb;
      for (int d = 0; d < 3; ++d) {
        jbb.lo[d] = __shfl_sync(FULL, jb.lo[d], src_lane);
        jbb.hi[d] = __shfl_sync(FULL, jb.hi[d], src_lane);
      }
      const Bx u = bx_union(e, jbb);
      __syncwarp();
      if (laneid() == 0) {
        t_put(t, j, k, u, v0, v1, v2);
        t_kill(t, cand);
      }
      t_dead(c, t, 1);
      __syncwarp();
      cand = j;
    }
  }
  DT_LAP(dt, D_MERGE);
  return t;
}
__device__ __forceinline__ void t_merge_from(Ctx& c, Table& t, uint32_t from) { t = t_merge_from_v(c, t, from); }

// Live entries above which an allocation's writer / reader table is
// re-merged after an access (tunable at compile time).
#ifndef IGS_MERGE_FLOOR
#define IGS_MERGE_FLOOR 48
#endif

// Re-merges a heap table once its live entries exceed max(floor, twice the
// count after its previous re-merge): fragmentation stays bounded while the
// quadratic merge runs a logarithmic number of times as a table grows.
__device__ __forceinline__ void t_set_mark(Ctx& c, Table& t) {
  __syncwarp();
  if (t.dp && laneid() == 0) t.dp[4] = t.live;
  __syncwarp();
}
__device__ __forceinline__ void t_maybe_merge(Ctx& c, Table& t, uint32_t floor) {
  const uint32_t mark = t.dp ? t.dp[4] : 0;
  if (t.live <= floor || t.live <= 2 * mark) return;
  t_merge_from(c, t, 0);
  t_set_mark(c, t);
}

// Makes the live entries with value v0 == val (NONE = all) of each key
// pairwise disjoint by subtracting earlier entries from later ones.
__device__ __noinline__ Table t_make_disjoint_v(Ctx& c, Table t, uint32_t val) {
  for (uint32_t i = 0; i < t.n; ++i) {
    const uint32_t k = t_key(t, i);
    if (k == DEAD) continue;
    if (val != NONE && t_v(t, 0, i) != val) continue;
    const Bx e = t_box(t, i);
    const uint32_t n0 = t.n;
    for (uint32_t base = i + 1; base < n0; base += 32) {
      const uint32_t j = base + laneid();
      bool hit = false;
      Bx f{};
      uint32_t w0 = 0, w1 = 0, w2 = 0;
      if (j < n0 && t_key(t, j) == k && (val == NONE || t_v(t, 0, j) == val)) {
        f = t_box(t, j);
        hit = bx_overlap(e, f);
        if (hit) {
          w0 = t_v(t, 0, j);
          w1 = t_v(t, 1, j);
          w2 = t_v(t, 2, j);
        }
      }
      const uint32_t hits = __ballot_sync(FULL, hit);
      if (!hits) continue;
      const int np = hit ? bx_minus_count(f, e) : 0;
      t_dead(c, t, __popc(hits));
      const uint32_t first = t_claim_n(c, t, (uint32_t)np);
      if (first == NONE) return t;  // the table could not grow (status set)
      if (hit) {
        t_kill(t, j);
        bx_minus_each(f, e, [&](int q, const Bx& pb) { t_put(t, first + q, k, pb, w0, w1, w2); });
      }
    }
    __syncwarp();
  }
  return t;
}
__device__ __forceinline__ void t_make_disjoint(Ctx& c, Table& t, uint32_t val = NONE) { t = t_make_disjoint_v(c, t, val); }

// Canonical form (row-major maximal decomposition) of the live boxes of
// in[from, to), which must be pairwise disjoint; appended to `out` sorted by
// (lo, hi). Three rewrite phases on a work table: make intervals along the
// fastest dimension maximal (splitting partially overlapping neighbours),
// then merge identical intervals over the middle dimension, then identical
// rectangles over the slowest dimension.
__device__ __noinline__ uint32_t canonical_impl(Ctx& c, const Table& in, uint32_t from, uint32_t to, Table& out);
__device__ uint32_t canonical(Ctx& c, const Table& in, uint32_t from, uint32_t to, Table& out) {
  PhaseTimer pt = pt_start();
  if (to == from + 1) {
    // one box is its own canonical form (none if it is dead or empty)
    const Ent e = t_ent(in, from);
    if (e.key == DEAD || bx_empty(e.b)) return 0;
    uint32_t s;
    if (!t_claim_ok(c, out, laneid() == 0, s)) return 0;
    if (laneid() == 0) t_put(out, s, 0, e.b, 0, 0, 0);
    __syncwarp();
    pt_lap(pt, c, PH_CANON);
    return 1;
  }
  const uint32_t r = canonical_impl(c, in, from, to, out);
  pt_lap(pt, c, PH_CANON);
  return r;
}
__device__ __noinline__ uint32_t canonical_impl(Ctx& c, const Table& in, uint32_t from, uint32_t to, Table& out) {
  Table& W = c.s[S_CAN];
  t_reset(W);
  for (uint32_t base = from; base < to; base += 32) {
    const uint32_t i = base + laneid();
    bool live = false;
    Bx b{};
    if (i < to && t_key(in, i) != DEAD) {
      b = t_box(in, i);
      live = !bx_empty(b);
    }
    const uint32_t s = t_claim(c, W, live);
    if (c.err) return 0;
    if (live) t_put(W, s, 0, b, 0, 0, 0);
  }
  __syncwarp();
  // A region whose boxes fill their bounding box exactly (the boxes are
  // disjoint, so equal volumes suffice) is that one box.
  if (W.n > 1) {
    uint64_t vol = 0;
    for (uint32_t base = 0; base < W.n; base += 32) {
      const uint32_t i = base + laneid();
      uint64_t v = i < W.n ? bx_volume(t_box(W, i)) : 0;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
      vol += v;
    }
    const Bx bb = t_bbox(c, W, 0, W.n);
    if (vol == bx_volume(bb)) {
      __syncwarp();
      if (laneid() == 0) t_put(W, 0, 0, bb, 0, 0, 0);
      W.n = 1;
      W.live = 1;
      __syncwarp();
    }
  }
  // Phase md rewrites until no box a has a neighbour b with a.hi[md] ==
  // b.lo[md], equal extents in the faster dimensions and overlapping extents
  // in the slower ones. One pass finds, for every box, its successor with
  // equal extents in all other dimensions (unique: the boxes are disjoint)
  // and the first pair that needs a split; whole successor chains merge at
  // once, else one pair is split so that its slower extents coincide. The
  // fixpoint of each phase is unique, so the order of rewrites does not
  // change the result.
  if (W.n > 1) {
    for (int phase = 0; phase < 3; ++phase) {
      const int md = 2 - phase;  // dimension merged in this phase
      for (uint32_t guard = 0;; ++guard) {
        if (guard > 64u * W.cap) {  // every round merges or splits: unreachable for valid input
          fail_internal(c, 1);
          return 0;
        }
        const uint32_t n = W.n;  // compacted: every entry is live
        uint64_t split = ~0ull;
        bool any_succ = false;
        for (uint32_t base = 0; base < n; base += 32) {
          const uint32_t i = base + laneid();
          uint32_t succ = NONE;
          uint64_t sp = ~0ull;
          if (i < n) {
            const Bx a = t_box(W, i);
            for (uint32_t j = 0; j < n; ++j) {
              if (j == i) continue;
              const Bx b = t_box(W, j);
              if (a.hi[md] != b.lo[md]) continue;
              bool faster_eq = true, slower_ov = true, slower_eq = true;
              for (int d = 0; d < 3; ++d) {
                if (d == md) continue;
                const bool eq = a.lo[d] == b.lo[d] && a.hi[d] == b.hi[d];
                if (d > md) {
                  faster_eq = faster_eq && eq;
                } else {
                  slower_ov = slower_ov && max(a.lo[d], b.lo[d]) < min(a.hi[d], b.hi[d]);
                  slower_eq = slower_eq && eq;
                }
              }
              if (!faster_eq || !slower_ov) continue;
              if (slower_eq) succ = j;
              else if (sp == ~0ull) sp = (uint64_t)i * n + j;
            }
            FLD(W, F_V, i) = succ;
            FLD(W, F_V + 1, i) = 0;
          }
          any_succ = any_succ || __any_sync(FULL, succ != NONE);
          sp = warp_min64(sp);
          split = sp < split ? sp : split;
        }
        __syncwarp();
        if (any_succ) {
          // mark boxes that have a predecessor; each chain head absorbs its chain
          for (uint32_t base = 0; base < n; base += 32) {
            const uint32_t i = base + laneid();
            if (i < n) {
              const uint32_t sc = t_v(W, 0, i);
              if (sc != NONE) FLD(W, F_V + 1, sc) = 1;
            }
          }
          __syncwarp();
          for (uint32_t base = 0; base < n; base += 32) {
            const uint32_t i = base + laneid();
            if (i < n && t_v(W, 0, i) != NONE && t_v(W, 1, i) == 0) {
              uint32_t cur = i, hi = 0;
              while (t_v(W, 0, cur) != NONE) {
                cur = t_v(W, 0, cur);
                hi = t_box(W, cur).hi[md];
                t_kill(W, cur);
              }
              FLD(W, F_HI + md, i) = hi;
            }
          }
          __syncwarp();
          t_compact(c, W);
          continue;
        }
        if (split == ~0ull) break;
        const uint32_t i = (uint32_t)(split / n), j = (uint32_t)(split % n);
        const Bx a = t_box(W, i), b = t_box(W, j);
        // split a and b so that their slower-dimension extents coincide
        Bx ia = a, ib = b;
        for (int d = 0; d < md; ++d) {
          ia.lo[d] = ib.lo[d] = max(a.lo[d], b.lo[d]);
          ia.hi[d] = ib.hi[d] = min(a.hi[d], b.hi[d]);
        }
        Bx pa[6], pb[6];
        const int na = bx_minus(a, ia, pa), nb = bx_minus(b, ib, pb);
        const uint32_t first = t_claim_n(c, W, laneid() == 0 ? (uint32_t)(na + nb + 2) : 0u);
        if (c.err) return 0;
        if (laneid() == 0) {
          t_kill(W, i);
          t_kill(W, j);
          uint32_t q = first;
          t_put(W, q++, 0, ia, 0, 0, 0);
          t_put(W, q++, 0, ib, 0, 0, 0);
          for (int x = 0; x < na; ++x) t_put(W, q++, 0, pa[x], 0, 0, 0);
          for (int x = 0; x < nb; ++x) t_put(W, q++, 0, pb[x], 0, 0, 0);
        }
        __syncwarp();
        t_compact(c, W);
      }
    }
  }
  // rank sort into out
  const uint32_t n = W.n;
  if (out.n + n > out.cap) {
    fail_cap(c, CAP_TABLE, out.cap);
    return 0;
  }
  for (uint32_t base = 0; base < n; base += 32) {
    const uint32_t i = base + laneid();
    if (i < n) {
      const Bx b = t_box(W, i);
      uint32_t rank = 0;
      for (uint32_t j = 0; j < n; ++j)
        if (j != i && bx_less(t_box(W, j), b)) ++rank;
      t_put(out, out.n + rank, 0, b, 0, 0, 0);
    }
  }
  out.n += n;
  __syncwarp();
  return n;
}

// ---- node state helpers ----------------------------------------------------

// A heap table from its descriptor {offset, cap, n, live} (no warp sync: safe
// in divergent code).
__device__ __forceinline__ Table heap_table(const NodeDev* nd, uint32_t* d) {
  Table t;
  t.base = nd->heap + (size_t)d[0] * F_COUNT;
  t.cap = d[1];
  t.n = d[2];
  t.live = d[3];
  t.dp = d;
  return t;
}
__device__ __forceinline__ Table slab(const Ctx& c, uint32_t* d) {
  __syncwarp();
  return heap_table(c.nd, d);
}
// Node-level ownership map of a buffer (owner node, replication mask).
__device__ __forceinline__ Table own_t(const Ctx& c, uint32_t b) { return slab(c, c.nd->own_d + kDesc * b); }
// Local state of a buffer (original producer, its memory, up-to-date memories).
__device__ __forceinline__ Table bst_t(const Ctx& c, uint32_t b) { return slab(c, c.nd->bst_d + kDesc * b); }
// Last writers / readers since the last write of an allocation.
__device__ __forceinline__ Table wr_t(const Ctx& c, uint32_t aid) {
  return slab(c, c.nd->wr_d + kDesc * c.nd->allocs[aid].slot);
}
__device__ __forceinline__ Table rd_t(const Ctx& c, uint32_t aid) {
  return slab(c, c.nd->rd_d + kDesc * c.nd->allocs[aid].slot);
}

// A fresh empty heap table behind descriptor d.
__device__ bool table_new(Ctx& c, uint32_t* d, uint32_t entries) {
  uint32_t cap = 0;
  const uint32_t off = heap_alloc(c, entries, cap);
  if (off == NONE) return false;
  __syncwarp();
  if (laneid() == 0) {
    d[0] = off;
    d[1] = cap;
    d[2] = 0;
    d[3] = 0;
    d[4] = 0;
  }
  __syncwarp();
  return true;
}
__device__ void table_free(Ctx& c, uint32_t* d) {
  __syncwarp();
  const uint32_t off = d[0], cap = d[1];
  if (cap) heap_free(c, off, cap);
  if (laneid() == 0) d[1] = 0;
  __syncwarp();
}

// Registers a new allocation record with an empty writer / reader slab.
__device__ bool new_alloc(Ctx& c, uint32_t aid, uint32_t b, uint32_t m, const Bx& bb, uint32_t user) {
  if (aid >= c.nd->cap_alloc || c.n_free == 0) {
    fail_cap(c, CAP_ALLOC, c.n_free == 0 ? c.nd->cap_slots : c.nd->cap_alloc);
    return false;
  }
  c.n_free -= 1;
  const uint32_t slot = c.nd->free_slots[c.n_free];
  if (!table_new(c, c.nd->wr_d + kDesc * slot, 32) || !table_new(c, c.nd->rd_d + kDesc * slot, 32)) return false;
  if (laneid() == 0) {
    AllocRec rec;
    rec.buffer = b;
    rec.mem = m;
    rec.live = 1;
    rec.user = user;
    for (int d = 0; d < 3; ++d) {
      rec.lo[d] = bb.lo[d];
      rec.hi[d] = bb.hi[d];
    }
    rec.mark = NONE;
    rec.slot = slot;
    c.nd->allocs[aid] = rec;
    c.nd->live[c.n_live] = aid;  // ids grow: the list stays sorted
  }
  c.n_live += 1;
  __syncwarp();
  return true;
}

// Drops an allocation: its slab goes back to the free list.
__device__ void drop_alloc(Ctx& c, uint32_t aid) {
  const uint32_t slot = c.nd->allocs[aid].slot;
  table_free(c, c.nd->wr_d + kDesc * slot);
  table_free(c, c.nd->rd_d + kDesc * slot);
  __syncwarp();
  if (laneid() == 0) {
    c.nd->allocs[aid].live = 0;
    c.nd->free_slots[c.n_free] = slot;
    uint32_t* L = c.nd->live;
    uint32_t k = 0;
    while (k < c.n_live && L[k] != aid) ++k;
    for (; k + 1 < c.n_live; ++k) L[k] = L[k + 1];
  }
  c.n_free += 1;
  c.n_live -= 1;
  __syncwarp();
}

__device__ __forceinline__ Bx alloc_box(const AllocRec& a) {
  Bx b;
  for (int d = 0; d < 3; ++d) {
    b.lo[d] = a.lo[d];
    b.hi[d] = a.hi[d];
  }
  return b;
}

// The live allocation of (buffer, memory) containing box, or NONE.
__device__ uint32_t find_alloc(Ctx& c, uint32_t buf, uint32_t mem, const Bx& b) {
  PhaseTimer pt = pt_start();
  const AllocRec* A = c.nd->allocs;
  const uint32_t* L = c.nd->live;
  const uint32_t k = warp_find_first(c, c.n_live, [&](uint32_t i) {
    const AllocRec& a = A[L[i]];
    return a.buffer == buf && a.mem == mem && bx_contains(alloc_box(a), b);
  });
  pt_lap(pt, c, PH_FIND);
  return k == NONE ? NONE : L[k];
}

// Per-lane variant (no warp collectives).
__device__ bool covered_by_alloc(const Ctx& c, uint32_t buf, uint32_t mem, const Bx& b) {
  const AllocRec* A = c.nd->allocs;
  const uint32_t* L = c.nd->live;
  for (uint32_t i = 0; i < c.n_live; ++i) {
    const AllocRec& a = A[L[i]];
    if (a.buffer == buf && a.mem == mem && bx_contains(alloc_box(a), b)) return true;
  }
  return false;
}

__device__ __forceinline__ const igs_task& task_of(const Ctx& c, uint32_t item) {
  return c.pg->tasks[c.pg->items[item].task];
}
__device__ __forceinline__ const BufDesc& buf_of(const Ctx& c, uint32_t b) { return c.pg->bufs[b]; }

__device__ Bx buffer_box(const BufDesc& b) {
  Bx x;
  for (int d = 0; d < 3; ++d) {
    x.lo[d] = 0;
    x.hi[d] = d < (int)b.dims ? b.extent[d] : 1;
  }
  return x;
}

// a1: chunks of a task: key = chunk index, v0 = node, v1 = memory (Sec. 3.1).
__device__ __noinline__ void task_chunks(Ctx& c, const igs_task& t, Table& CH) {
  t_reset(CH);
  const uint32_t Cx = t.num_chunks >> 16;
  if (Cx) {
    // split along dims 0 and 1: a Cy x Cx grid; grid row iy goes to node
    // floor(iy*N/Cy), a node's K chunks (row-major, j) to its device
    // floor(j*D/K); chunk index iy*Cx + ix
    const uint64_t Cy = t.num_chunks & 0xFFFFu, N = c.N, D = c.D, E0 = t.range[0], E1 = t.range[1];
    const uint32_t total = (uint32_t)(Cy * Cx);
    for (uint32_t base = 0; base < total; base += 32) {
      const uint32_t i = base + laneid();
      bool ok = false;
      Bx b{};
      uint32_t node = 0, mem = 0;
      if (i < total) {
        const uint64_t iy = i / Cx, ix = i % Cx;
        const uint64_t nd = iy * N / Cy;
        const uint64_t r0n = (nd * Cy + N - 1) / N, r1n = ((nd + 1) * Cy + N - 1) / N;
        const uint64_t K = (r1n - r0n) * Cx, j = (iy - r0n) * Cx + ix;
        node = (uint32_t)nd;
        mem = 2 + (uint32_t)(j * D / K);
        b.lo[0] = (uint32_t)(iy * E0 / Cy);
        b.hi[0] = (uint32_t)((iy + 1) * E0 / Cy);
        b.lo[1] = (uint32_t)(ix * E1 / Cx);
        b.hi[1] = (uint32_t)((ix + 1) * E1 / Cx);
        b.lo[2] = 0;
        b.hi[2] = t.range[2];
        ok = b.lo[0] < b.hi[0] && b.lo[1] < b.hi[1];
      }
      const uint32_t s = t_claim(c, CH, ok);
      if (c.err) return;
      if (ok) t_put(CH, s, i, b, node, mem, 0);
    }
    __syncwarp();
    return;
  }
  const uint64_t E0 = t.range[0], C = t.num_chunks, M = (uint64_t)c.N * c.D;
  for (uint32_t base = 0; base < t.num_chunks; base += 32) {
    const uint32_t i = base + laneid();
    bool ok = false;
    Bx b{};
    uint32_t node = 0, mem = 0;
    if (i < t.num_chunks) {
      const uint32_t r0 = (uint32_t)((uint64_t)i * E0 / C), r1 = (uint32_t)((uint64_t)(i + 1) * E0 / C);
      ok = r0 < r1;
      const uint32_t g = (uint32_t)((uint64_t)i * M / C);
      node = g / c.D;
      mem = 2 + g % c.D;
      b.lo[0] = r0;
      b.hi[0] = r1;
      for (int d = 1; d < 3; ++d) {
        b.lo[d] = 0;
        b.hi[d] = t.range[d];
      }
    }
    const uint32_t s = t_claim(c, CH, ok);
    if (c.err) return;
    if (ok) t_put(CH, s, i, b, node, mem, 0);
  }
  __syncwarp();
}

// a2: mapped box of accessor a for a chunk box, clamped to the buffer.
__device__ Bx map_box(const igs_accessor& a, const Bx& ch, const BufDesc& buf) {
  Bx r;
  for (int d = 0; d < 3; ++d) {
    const uint32_t ext = d < (int)buf.dims ? buf.extent[d] : 1;
    int64_t lo, hi;
    const igs_map_dim& m = a.dim[d];
    if (d >= (int)buf.dims) {
      lo = 0;
      hi = 1;
    } else if (m.kind == IGS_MAP_ALL) {
      lo = 0;
      hi = ext;
    } else if (m.kind == IGS_MAP_FIXED) {
      lo = m.a;
      hi = m.b;
    } else {
      const uint32_t k = m.a;
      lo = (int64_t)ch.lo[k] + (int32_t)m.b - (int64_t)m.c;
      hi = (int64_t)ch.hi[k] + (int32_t)m.b + (int64_t)m.c;
    }
    lo = lo < 0 ? 0 : lo;
    hi = hi > (int64_t)ext ? (int64_t)ext : hi;
    if (lo >= hi) {
      lo = 0;
      hi = 0;
    }
    r.lo[d] = (uint32_t)lo;
    r.hi[d] = (uint32_t)hi;
  }
  return r;
}

// Mapped boxes for every (chunk slot, accessor): MP[slot * nacc + a].
__device__ __noinline__ void task_mapped(Ctx& c, const igs_task& t, const Table& CH, Table& MP) {
  const uint32_t na = t.num_accessors, total = CH.n * na;
  if (total > MP.cap) {
    fail_cap(c, CAP_TABLE, MP.cap);
    return;
  }
  for (uint32_t base = 0; base < total; base += 32) {
    const uint32_t i = base + laneid();
    if (i < total) {
      const uint32_t slot = i / na, a = i % na;
      const Bx b = map_box(t.acc[a], t_box(CH, slot), buf_of(c, t.acc[a].buffer));
      t_put(MP, i, 0, b, 0, 0, 0);
    }
  }
  MP.n = total;
  __syncwarp();
}

// Chunks are disjoint along kernel dimension 0; an accessor that maps that
// dimension one to one (radius 0) onto some buffer dimension gives them
// disjoint images there, so one accessor's chunks cannot overlap each other.
__device__ __forceinline__ bool split_dim_injective(const igs_accessor& acc, uint32_t dims) {
  for (uint32_t d = 0; d < dims; ++d)
    if (acc.dim[d].kind == IGS_MAP_AFFINE && acc.dim[d].a == 0 && acc.dim[d].c == 0) return true;
  return false;
}

// Sec. 4.4: chunks of one task writing overlapping regions.
__device__ __noinline__ bool overlapping_writes(Ctx& c, const igs_task& t, const Table& CH, const Table& MP) {
  const uint32_t na = t.num_accessors;
  for (uint32_t a = 0; a < na; ++a) {
    if (!(t.acc[a].mode & IGS_WRITE)) continue;
    for (uint32_t b = a; b < na; ++b) {
      if (!(t.acc[b].mode & IGS_WRITE) || t.acc[b].buffer != t.acc[a].buffer) continue;
      if (a == b && split_dim_injective(t.acc[a], buf_of(c, t.acc[a].buffer).dims)) continue;
      // chunk x's accessor a against every later chunk y's accessor b (and a
      // against b within the pair of accessors when a != b)
      for (uint32_t x = 0; x < CH.n; ++x) {
        const Bx bx = t_box(MP, x * na + a);
        if (bx_empty(bx)) continue;
        for (uint32_t base = 0; base < CH.n; base += 32) {
          const uint32_t y = base + laneid();
          bool bad = false;
          if (y < CH.n && y != x && (a != b || y > x)) bad = bx_overlap(bx, t_box(MP, y * na + b));
          if (__ballot_sync(FULL, bad)) return true;
        }
      }
    }
  }
  return false;
}

// ---- emission with dependency tracking (a8, a10) --------------------------


// Emits one instruction. Dependencies: extra edges already in S_DEP (when
// keep_dep) plus, per access, the last writers (RAW dataflow; WAW anti; a
// fresh allocation's own alloc instruction: allocation lifetime) and, for
// writes, the readers since the last write (WAR anti); no predecessor at all
// means an edge to the last epoch. Then reads, then writes are applied to
// the per-allocation tracking tables.
__device__ __noinline__ uint32_t emit_impl(Ctx& c, uint32_t type, uint32_t seq, uint32_t fa, uint32_t fb, uint32_t fc, uint32_t fd,
                              const Table* bt, uint32_t bfrom, uint32_t bto, const Acc* acc, int nacc, bool keep_dep,
                              const Table* bindt, uint32_t bind_from, uint32_t bind_n);
__device__ uint32_t emit(Ctx& c, uint32_t type, uint32_t seq, uint32_t fa, uint32_t fb, uint32_t fc, uint32_t fd,
                         const Table* bt, uint32_t bfrom, uint32_t bto, const Acc* acc, int nacc, bool keep_dep,
                         const Table* bindt = nullptr, uint32_t bind_from = 0, uint32_t bind_n = 0) {
  PhaseTimer pt = pt_start();
  const uint32_t r = emit_impl(c, type, seq, fa, fb, fc, fd, bt, bfrom, bto, acc, nacc, keep_dep, bindt, bind_from, bind_n);
  pt_lap(pt, c, PH_EMIT);
  return r;
}
// Dependencies of the next instruction into S_DEP (after the extra edges
// already there when keep_dep): per access the last writers (RAW dataflow;
// WAW anti; a fresh allocation's own alloc instruction: allocation
// lifetime) and, for writes, the readers since the last write (WAR anti); no
// predecessor at all means an edge to the last epoch.
__device__ __forceinline__ bool emit_deps(Ctx& c, const Acc* acc, int nacc, bool keep_dep) {
  if (c.err) return false;
  NodeDev* nd = c.nd;
  Table D = c.s[S_DEP];  // header in registers; written back below
  if (!keep_dep) t_reset(D);
  // One pass per (access, table): each lane tests one entry against every
  // box of the access region (broadcast loads) and records one dependency
  // per overlapping entry (its kind depends on the entry and the access
  // mode only; duplicates are merged when the edges are emitted).
  for (int k = 0; k < nacc; ++k) {
    const Acc& A = acc[k];
    const uint32_t slot = nd->allocs[A.alloc].slot;
    const bool snap = A.alloc == c.snap_alloc;
    const int ntab = (A.mode & IGS_WRITE) ? 2 : 1;
    for (int tab = 0; tab < ntab; ++tab) {
      const uint32_t* dsc = (tab == 0 ? nd->wr_d : nd->rd_d) + kDesc * slot;
      const uint32_t n = snap ? c.snap_n[tab] : dsc[2];
      if (n == 0) continue;
      const uint32_t* tb = snap ? c.snap_tab[tab] : nd->heap + (size_t)dsc[0] * F_COUNT;
      c.map_reads += n;
      DT_COUNT(N_PROBE_ENTRIES, n);
      for (uint32_t base = 0; base < n; base += 32) {
        const uint32_t f = base + laneid();
        bool hit = false;
        uint32_t w = 0, kind = 0;
        if (f < n) {
          const uint4* e = reinterpret_cast<const uint4*>(tb + (size_t)f * F_COUNT);
          const uint4 e0 = e[0], e1 = e[1], e2 = e[2];
          if (e0.x != DEAD) {
            Bx eb;
            eb.lo[0] = e0.y;
            eb.lo[1] = e0.z;
            eb.lo[2] = e0.w;
            eb.hi[0] = e1.x;
            eb.hi[1] = e1.y;
            eb.hi[2] = e1.z;
            for (uint32_t r = A.from; r < A.to && !hit; ++r) {
              const Ent q = t_ent(*A.t, r);
              hit = q.key != DEAD && bx_overlap(eb, q.b);
            }
            if (hit) {
              w = e1.w;  // v0
              if (tab == 1) kind = IGS_DEP_ANTI;
              else if (e2.x == 1) kind = IGS_DEP_ALLOC;  // v1: an allocation writer
              else kind = ((A.mode & IGS_READ) ? IGS_DEP_DATAFLOW : 0u) | ((A.mode & IGS_WRITE) ? IGS_DEP_ANTI : 0u);
            }
          }
        }
        if (!__any_sync(FULL, hit)) continue;
        uint32_t s;
        if (!t_claim_ok(c, D, hit, s)) {
          c.s[S_DEP] = D;
          return false;
        }
        if (hit) {
          FLD(D, F_V, s) = w;
          FLD(D, F_V + 1, s) = kind;
        }
      }
    }
  }
  __syncwarp();
  if (D.n == 0) {
    if (laneid() == 0) {
      FLD(D, F_V, 0) = c.epoch;
      FLD(D, F_V + 1, 0) = IGS_DEP_EPOCH;
    }
    D.n = 1;
    __syncwarp();
  }
  c.s[S_DEP] = D;
  return true;
}

// The unique predecessors in S_DEP, ascending, kinds OR-ed, as edges into
// instruction id, written to out[0, count) (at most cap of them, else a
// capacity failure of kind cap_kind); marks each predecessor as having a
// successor. Returns the count (NONE on failure).
__device__ __forceinline__ uint32_t emit_edges(Ctx& c, uint32_t id, igs_edge* out, uint32_t cap, CapKind cap_kind,
                                            uint32_t cap_report) {
  if (c.err) return NONE;
  NodeDev* nd = c.nd;
  const Table& D = c.s[S_DEP];
  // unique predecessors in ascending order, kinds OR-ed
  const uint32_t nd0 = D.n;
  uint32_t n_unique = 0;
  if (nd0 <= 32) {
    // one entry per lane: the first lane of each group of equal predecessors
    // leads it; a leader's kind ORs its group's kinds and its rank counts the
    // leaders with smaller ids (one pass over the entries)
    const bool in = laneid() < nd0;
    const uint32_t p = in ? FLD(D, F_V, laneid()) : 0xFFFFFFFFu;
    const uint32_t k = in ? FLD(D, F_V + 1, laneid()) : 0u;
    const uint32_t grp = __match_any_sync(FULL, p);
    const bool lead = in && (uint32_t)(__ffs(grp) - 1) == laneid();
    const uint32_t leaders = __ballot_sync(FULL, lead);
    uint32_t kind = 0, rank = 0;
    for (uint32_t j = 0; j < nd0; ++j) {
      const uint32_t pj = __shfl_sync(FULL, p, j), kj = __shfl_sync(FULL, k, j);
      if (pj == p) kind |= kj;
      else if (((leaders >> j) & 1u) && pj < p) ++rank;
    }
    n_unique = __popc(leaders);
    if (n_unique > cap) {
      fail_cap(c, cap_kind, cap_report);
      return NONE;
    }
    if (lead) {
      igs_edge e;
      e.from = p;
      e.to = id;
      e.kind = kind;
      out[rank] = e;
      if (!(p & PROV)) nd->has_succ[p] = 1;
    }
  } else {
    // pass 1: mark each entry that is the first of its predecessor id (the
    // mark lives in the entry's third value word)
    for (uint32_t base = 0; base < nd0; base += 32) {
      const uint32_t i = base + laneid();
      bool first = false;
      if (i < nd0) {
        const uint32_t p = FLD(D, F_V, i);
        first = true;
        for (uint32_t j = 0; j < i; ++j)
          if (FLD(D, F_V, j) == p) {
            first = false;
            break;
          }
        FLD(D, F_V + 2, i) = first ? 1u : 0u;
      }
      n_unique += __popc(__ballot_sync(FULL, first));
    }
    __syncwarp();
    if (n_unique > cap) {
      fail_cap(c, cap_kind, cap_report);
      return NONE;
    }
    // pass 2: a first entry's rank is the number of first entries with a
    // smaller id; its kind ORs the kinds of every entry with its id
    for (uint32_t base = 0; base < nd0; base += 32) {
      const uint32_t i = base + laneid();
      if (i < nd0) {
        const uint32_t p = FLD(D, F_V, i);
        const bool first = FLD(D, F_V + 2, i) != 0;
        uint32_t kind = 0, rank = 0;
        if (first)
          for (uint32_t j = 0; j < nd0; ++j) {
            const uint32_t q = FLD(D, F_V, j);
            if (q == p) kind |= FLD(D, F_V + 1, j);
            else if (q < p && FLD(D, F_V + 2, j)) ++rank;
          }
        if (first) {
          igs_edge e;
          e.from = p;
          e.to = id;
          e.kind = kind;
          out[rank] = e;
          if (!(p & PROV)) nd->has_succ[p] = 1;
        }
      }
    }
  }
  __syncwarp();
  return n_unique;
}

// The record of instruction c.n_instr with its boxes (bt[bfrom, bto)) and
// bindings (bindt[bind_from, +bind_n)). clear_succ: mark it as having no
// successor yet (callers that emitted its successors' edges already pass false).
__device__ __forceinline__ bool emit_record(Ctx& c, uint32_t type, uint32_t seq, uint32_t fa, uint32_t fb, uint32_t fc,
                                         uint32_t fd, const Table* bt, uint32_t bfrom, uint32_t bto, const Table* bindt,
                                         uint32_t bind_from, uint32_t bind_n, bool clear_succ) {
  if (c.err) return false;
  NodeDev* nd = c.nd;
  const uint32_t id = c.n_instr;
  if (c.n_instr + 1 > nd->cap_instr) {
    fail_cap(c, CAP_EDGE, nd->cap_edge);
    return false;
  }
  // instruction record, its boxes and bindings
  uint32_t nb = 0;
  if (bt) {
    for (uint32_t base = bfrom; base < bto; base += 32) {
      const uint32_t i = base + laneid();
      const bool live = i < bto && t_key(*bt, i) != DEAD;
      const uint32_t m = __ballot_sync(FULL, live);
      if (c.n_box + nb + __popc(m) > nd->cap_box) {
        fail_cap(c, CAP_BOX, nd->cap_box);
        return false;
      }
      if (live) {
        const Bx b = t_box(*bt, i);
        igs_box o;
        for (int d = 0; d < 3; ++d) {
          o.lo[d] = b.lo[d];
          o.hi[d] = b.hi[d];
        }
        nd->boxes[c.n_box + nb + __popc(m & lanemask_lt())] = o;
      }
      nb += __popc(m);
    }
  }
  if (c.n_bind + bind_n > nd->cap_bind) {
    fail_cap(c, CAP_BIND, nd->cap_bind);
    return false;
  }
  if (bindt && laneid() < bind_n) {
    const uint32_t i = bind_from + laneid();
    const Bx b = t_box(*bindt, i);
    igs_binding o;
    o.alloc = t_v(*bindt, 0, i);
    for (int d = 0; d < 3; ++d) {
      o.lo[d] = b.lo[d];
      o.hi[d] = b.hi[d];
    }
    nd->binds[c.n_bind + laneid()] = o;
  }
  if (laneid() == 0) {
    igs_instruction r;
    r.id = id;
    r.type = type;
    r.seq = seq;
    r.a = fa;
    r.b = fb;
    r.c = fc;
    r.d = fd;
    r.box_off = c.n_box;
    r.box_cnt = nb;
    r.bind_off = c.n_bind;
    r.bind_cnt = bind_n;
    nd->instrs[id] = r;
    if (clear_succ) nd->has_succ[id] = 0;
  }
  c.n_box += nb;
  c.n_bind += bind_n;
  c.n_instr += 1;
  __syncwarp();
  return true;
}

// A read of instruction id over the boxes box(r) (r < n; box returns false
// for a dead one) joins allocation aid's readers; again: the instruction
// already read there through another accessor (its earlier entries over the
// boxes are replaced).
template <class G>
__device__ __forceinline__ bool apply_read(Ctx& c, uint32_t aid, uint32_t n, G box, uint32_t id, bool again) {
  Table RD = rd_t(c, aid);
  t_tidy(c, RD);
  for (uint32_t r = 0; r < n; ++r) {
    Bx q;
    if (!box(r, q)) continue;
    if (again) t_subtract(c, RD, NONE, q, id);
    const uint32_t s = t_claim(c, RD, laneid() == 0);
    if (c.err) return false;
    if (laneid() == 0) t_put(RD, s, 0, q, id, 0, 0);
    __syncwarp();
  }
  // re-merge only a table that has grown: keeps hot paths short and bounds
  // fragmentation between horizons
  t_maybe_merge(c, RD, IGS_MERGE_FLOOR);
  return true;
}
// A write of instruction id over the boxes box(r) replaces allocation aid's
// writers there and clears its readers.
template <class G>
__device__ __forceinline__ bool apply_write(Ctx& c, uint32_t aid, uint32_t n, G box, uint32_t id) {
  Table RD = rd_t(c, aid);
  Table WR = wr_t(c, aid);
  t_tidy(c, WR);
  for (uint32_t r = 0; r < n; ++r) {
    Bx q;
    if (!box(r, q)) continue;
    t_subtract(c, RD, NONE, q);
    t_set(c, WR, NONE, q, id, 0, 0);
    if (c.err) return false;
  }
  t_maybe_merge(c, WR, IGS_MERGE_FLOOR);
  t_maybe_merge(c, RD, IGS_MERGE_FLOOR);
  return true;
}

// Applies an instruction's accesses to the per-allocation tables: reads
// join the readers, writes replace the writers and clear the readers.
__device__ __forceinline__ bool emit_apply(Ctx& c, const Acc* acc, int nacc, uint32_t id) {
  if (c.err) return false;
  // apply reads, then writes
  for (int k = 0; k < nacc; ++k) {
    const Acc& A = acc[k];
    if (!(A.mode & IGS_READ)) continue;
    bool again = false;
    for (int j = 0; j < k; ++j)
      if (acc[j].alloc == A.alloc && (acc[j].mode & IGS_READ)) again = true;
    auto box = [&](uint32_t r, Bx& q) {
      const Ent e = t_ent(*A.t, A.from + r);
      q = e.b;
      return e.key != DEAD;
    };
    if (!apply_read(c, A.alloc, A.to - A.from, box, id, again)) return false;
  }
  for (int k = 0; k < nacc; ++k) {
    const Acc& A = acc[k];
    if (!(A.mode & IGS_WRITE)) continue;
    auto box = [&](uint32_t r, Bx& q) {
      const Ent e = t_ent(*A.t, A.from + r);
      q = e.b;
      return e.key != DEAD;
    };
    if (!apply_write(c, A.alloc, A.to - A.from, box, id)) return false;
  }
  return true;
}

__device__ __noinline__ uint32_t emit_impl(Ctx& c, uint32_t type, uint32_t seq, uint32_t fa, uint32_t fb, uint32_t fc, uint32_t fd,
                              const Table* bt, uint32_t bfrom, uint32_t bto, const Acc* acc, int nacc, bool keep_dep,
                              const Table* bindt, uint32_t bind_from, uint32_t bind_n) {
  if (c.err) return NONE;
  NodeDev* nd = c.nd;
  if (c.stage) {
    // a coherence worker: record, edges and boxes into its stage; the tables
    // stay as they are
    Stage& st = *c.stage;
    if (bind_n || st.n_instr + 1 > st.cap_instr) {
      fail_cap(c, CAP_TABLE, st.cap_instr);
      return NONE;
    }
    const uint32_t pid = st.id_base | st.n_instr;
    if (!emit_deps(c, acc, nacc, keep_dep)) return NONE;
    const uint32_t ne = emit_edges(c, pid, st.edges + st.n_edge, st.cap_edge - st.n_edge, CAP_TABLE, st.cap_edge);
    if (ne == NONE) return NONE;
    uint32_t nb = 0;
    if (bt) {
      for (uint32_t base = bfrom; base < bto; base += 32) {
        const uint32_t i = base + laneid();
        const bool live = i < bto && t_key(*bt, i) != DEAD;
        const uint32_t m = __ballot_sync(FULL, live);
        if (st.n_box + nb + __popc(m) > st.cap_box) {
          fail_cap(c, CAP_TABLE, st.cap_box);
          return NONE;
        }
        if (live) {
          const Bx b = t_box(*bt, i);
          igs_box o;
          for (int d = 0; d < 3; ++d) {
            o.lo[d] = b.lo[d];
            o.hi[d] = b.hi[d];
          }
          st.boxes[st.n_box + nb + __popc(m & lanemask_lt())] = o;
        }
        nb += __popc(m);
      }
    }
    if (laneid() == 0) {
      igs_instruction r;
      r.id = pid;
      r.type = type;
      r.seq = seq;
      r.a = fa;
      r.b = fb;
      r.c = fc;
      r.d = fd;
      r.box_off = st.n_box;
      r.box_cnt = nb;
      r.bind_off = st.n_edge;
      r.bind_cnt = ne;
      st.instrs[st.n_instr] = r;
    }
    __syncwarp();
    st.n_edge += ne;
    st.n_box += nb;
    st.n_instr += 1;
    // the accesses are applied to the tables once every worker has planned
    // (p4_apply), in the order of the single-warp path
    return pid;
  }
  const uint32_t id = c.n_instr;
  DT_START(dt);
  DT_COUNT(N_EMIT, 1);
  if (!emit_deps(c, acc, nacc, keep_dep)) return NONE;
  DT_LAP(dt, D_PROBE);
  const uint32_t ne = emit_edges(c, id, nd->edges + c.n_edge, nd->cap_edge - c.n_edge, CAP_EDGE, nd->cap_edge);
  if (ne == NONE) return NONE;
  c.n_edge += ne;
  DT_LAP(dt, D_DEDUP);
  if (!emit_record(c, type, seq, fa, fb, fc, fd, bt, bfrom, bto, bindt, bind_from, bind_n, true)) return NONE;
  DT_LAP(dt, D_RECORD);
  if (!emit_apply(c, acc, nacc, id)) return NONE;
  DT_LAP(dt, D_APPLY);
  return id;
}

// Replace every tracked instruction id older than h by h and re-merge (a9).
// In writer tables (writers = true) v1 marks allocation writers; a replaced
// writer is the horizon, which is not one. Returns whether any id changed.
__device__ __noinline__ bool map_ids(Ctx& c, Table& T, uint32_t h, bool writers = false) {
  bool any = false;
  for (uint32_t base = 0; base < T.n; base += 32) {
    const uint32_t i = base + laneid();
    bool ch = false;
    if (i < T.n && t_key(T, i) != DEAD) {
      const uint32_t v = t_v(T, 0, i);
      if (v < h) {
        FLD(T, F_V, i) = h;
        if (writers) FLD(T, F_V + 1, i) = 0;
        ch = true;
      }
    }
    any = any || __any_sync(FULL, ch);
  }
  __syncwarp();
  return any;
}

// Live entries above which a table whose ids changed is re-merged when a
// horizon is applied (smaller tables are only compacted: merging is a matter
// of table size, not of content, and costs a scan per entry).
#ifndef IGS_EPOCH_MERGE_FLOOR
#define IGS_EPOCH_MERGE_FLOOR 16
#endif

// Worker w of `workers` takes the live allocations li and the buffers b with
// li, b = w mod workers (the tables are independent of one another).
__device__ __noinline__ void epoch_share(Ctx& c, uint32_t h, uint32_t w, uint32_t workers) {
  for (uint32_t li = w; li < c.n_live; li += workers) {
    const uint32_t aid = c.nd->live[li];
    // tables whose ids all stay are left as they are; the others are
    // compacted and, above the floor, re-merged
    Table WR = wr_t(c, aid);
    if (map_ids(c, WR, h, true)) {
      t_compact(c, WR);
      if (WR.live > IGS_EPOCH_MERGE_FLOOR) {
        t_merge_from(c, WR, 0);
        t_compact(c, WR);
      }
      t_set_mark(c, WR);
    }
    Table RD = rd_t(c, aid);
    if (map_ids(c, RD, h)) {
      t_make_disjoint(c, RD, h);
      t_compact(c, RD);
      if (RD.live > IGS_EPOCH_MERGE_FLOOR) {
        t_merge_from(c, RD, 0);
        t_compact(c, RD);
      }
      t_set_mark(c, RD);
    }
    if (c.err) return;
  }
  const uint32_t nb = c.nd->cap_buffers;
  for (uint32_t b = w; b < nb && !c.err; b += workers) {
    if (c.nd->bst_d[kDesc * b + 1] == 0) continue;  // no table (never created or destroyed)
    Table B = bst_t(c, b);
    if (B.n == 0) continue;
    if (!map_ids(c, B, h)) continue;
    t_compact(c, B);
    t_merge_from(c, B, 0);
    t_compact(c, B);
    t_set_mark(c, B);
  }
}

// Free of an allocation: depends on every writer and reader (allocation lifetime).
__device__ __noinline__ void emit_free(Ctx& c, uint32_t seq, uint32_t aid) {
  Table& D = c.s[S_DEP];
  t_reset(D);
  for (int k = 0; k < 2; ++k) {
    const Table T = k == 0 ? wr_t(c, aid) : rd_t(c, aid);
    for (uint32_t base = 0; base < T.n; base += 32) {
      const uint32_t i = base + laneid();
      const bool hit = i < T.n && t_key(T, i) != DEAD;
      const uint32_t s = t_claim(c, D, hit);
      if (c.err) return;
      if (hit) {
        FLD(D, F_V, s) = t_v(T, 0, i);
        FLD(D, F_V + 1, s) = IGS_DEP_ALLOC;
      }
    }
  }
  __syncwarp();
  const AllocRec a = c.nd->allocs[aid];
  emit(c, IGS_FREE, seq, aid, a.mem, a.buffer, NONE, nullptr, 0, 0, nullptr, 0, true);
  drop_alloc(c, aid);
}

// a5: coherence copies making need = T[from, to) (disjoint boxes) up to date
// in memory m, allocation dst: stale parts split by original producer, then
// by source allocation, one copy per (producer, source allocation).
// Planned by a coherence worker (c.stage set): the copies go to its stage and
// neither the buffer state nor the allocation tables change; the regions its
// earlier copies of b into memory m cover count as up to date, as they would
// after those copies' buffer-state update.
__device__ __noinline__ void coherence(Ctx& c, uint32_t seq, uint32_t b, uint32_t m, uint32_t dst, const Table& T, uint32_t from,
                          uint32_t to) {
  Table& Q = c.s[S_T0];
  Table& G = c.s[S_T1];
  Table& P = c.s[S_T2];
  Table& CP = c.s[S_T3];
  Table& CN = c.s[S_T5];
  t_reset(Q);
  t_reset(CP);
  {
    const Table B = bst_t(c, b);
    for (uint32_t r = from; r < to; ++r) {
      if (t_key(T, r) == DEAD) continue;
      const Bx q = t_box(T, r);
      t_query(c, B, NONE, q, Q, [m](uint32_t prod, uint32_t, uint32_t mask) {
        return !((mask >> m) & 1u) && prod != NONE;
      });
      if (c.err) return;
    }
  }
  const Stage* plan = c.stage;
  if (plan) {
    if (c.nd->stage_d2d) {  // host-staged copies allocate: never planned
      fail_internal(c, 10);
      return;
    }
    for (uint32_t q = 0; q < plan->n_instr && Q.n; ++q) {
      const igs_instruction r = plan->instrs[q];
      if (r.c != b || c.nd->allocs[r.b].mem != m) continue;
      for (uint32_t i = 0; i < r.box_cnt; ++i) {
        const igs_box o = plan->boxes[r.box_off + i];
        Bx x;
        for (int d = 0; d < 3; ++d) {
          x.lo[d] = o.lo[d];
          x.hi[d] = o.hi[d];
        }
        t_subtract(c, Q, NONE, x);
        if (c.err) return;
      }
    }
    if (Q.live != Q.n) t_compact(c, Q);  // the scans below take every entry as live
  }
  uint64_t last = 0;
  bool first_round = true;
  for (;;) {
    uint64_t best = ~0ull;
    for (uint32_t base = 0; base < Q.n; base += 32) {
      const uint32_t i = base + laneid();
      uint64_t k = ~0ull;
      if (i < Q.n) {
        k = ((uint64_t)t_v(Q, 0, i) << 32) | t_v(Q, 1, i);
        if (!first_round && k <= last) k = ~0ull;
      }
      k = warp_min64(k);
      best = k < best ? k : best;
    }
    if (best == ~0ull) break;
    first_round = false;
    last = best;
    const uint32_t prod = (uint32_t)(best >> 32), pmem = (uint32_t)best;
    if (prod == REMOTE) {
      fail_internal(c, 2);
      return;
    }
    t_reset(G);
    for (uint32_t base = 0; base < Q.n; base += 32) {
      const uint32_t i = base + laneid();
      const bool hit = i < Q.n && t_v(Q, 0, i) == prod && t_v(Q, 1, i) == pmem;
      const uint32_t s = t_claim(c, G, hit);
      if (c.err) return;
      if (hit) t_put(G, s, 0, t_box(Q, i), 0, 0, 0);
    }
    __syncwarp();
    // one copy per source allocation of (b, pmem), in live (ascending id) order
    auto copy_from = [&](uint32_t src) -> bool {
      const AllocRec a = c.nd->allocs[src];
      t_reset(P);
      const Bx ab = alloc_box(a);
      for (uint32_t base = 0; base < G.n; base += 32) {
        const uint32_t i = base + laneid();
        Bx is{};
        bool hit = false;
        if (i < G.n) {
          is = bx_isect(t_box(G, i), ab);
          hit = !bx_empty(is);
        }
        const uint32_t s = t_claim(c, P, hit);
        if (c.err) return false;
        if (hit) t_put(P, s, 0, is, 0, 0, 0);
      }
      __syncwarp();
      if (P.n == 0) return true;
      t_reset(CN);
      canonical(c, P, 0, P.n, CN);
      if (c.err) return false;
      if (c.nd->stage_d2d && a.mem >= 2 && m >= 2) {
        // staged in host memory (Sec. 3.3): a fresh allocation in M1 over
        // the region's bounding box, a copy into it, a copy out of it, its free
        Bx bb;
        for (int d = 0; d < 3; ++d) {
          bb.lo[d] = 0xFFFFFFFFu;
          bb.hi[d] = 0;
        }
        for (uint32_t i = 0; i < CN.n; ++i) {
          if (t_key(CN, i) == DEAD) continue;
          const Bx x = t_box(CN, i);
          for (int d = 0; d < 3; ++d) {
            bb.lo[d] = min(bb.lo[d], x.lo[d]);
            bb.hi[d] = max(bb.hi[d], x.hi[d]);
          }
        }
        if (c.n_alloc >= c.nd->cap_alloc) {
          fail_cap(c, CAP_ALLOC, c.nd->cap_alloc);
          return false;
        }
        t_reset(P);  // P now holds the allocation's box
        const uint32_t s0 = t_claim(c, P, laneid() == 0);
        if (c.err) return false;
        if (laneid() == 0) t_put(P, s0, 0, bb, 0, 0, 0);
        __syncwarp();
        const uint32_t hid = c.n_alloc;
        const uint32_t iid = emit(c, IGS_ALLOC, seq, hid, 1, b, NONE, &P, 0, 1, nullptr, 0, false);
        if (c.err) return false;
        if (!new_alloc(c, hid, b, 1, bb, 0)) return false;
        c.n_alloc += 1;
        {
          Table WR = wr_t(c, hid);
          const uint32_t s1 = t_claim(c, WR, laneid() == 0);
          if (c.err) return false;
          if (laneid() == 0) t_put(WR, s1, 0, bb, iid, 1, 0);  // v1 = 1: the writer is an allocation
          __syncwarp();
        }
        Acc in[2] = {{&CN, 0, CN.n, src, IGS_READ}, {&CN, 0, CN.n, hid, IGS_WRITE}};
        emit(c, IGS_COPY, seq, src, hid, b, 0, &CN, 0, CN.n, in, 2, false);
        if (c.err) return false;
        Acc out[2] = {{&CN, 0, CN.n, hid, IGS_READ}, {&CN, 0, CN.n, dst, IGS_WRITE}};
        emit(c, IGS_COPY, seq, hid, dst, b, 0, &CN, 0, CN.n, out, 2, false);
        if (c.err) return false;
        emit_free(c, seq, hid);
        if (c.err) return false;
      } else {
        Acc acc[2] = {{&CN, 0, CN.n, src, IGS_READ}, {&CN, 0, CN.n, dst, IGS_WRITE}};
        emit(c, IGS_COPY, seq, src, dst, b, 0, &CN, 0, CN.n, acc, 2, false);
        if (c.err) return false;
      }
      // remember the copied region (a planned copy's boxes are in its record)
      for (uint32_t base = 0; base < (plan ? 0u : CN.n); base += 32) {
        const uint32_t i = base + laneid();
        const bool in = i < CN.n;
        const uint32_t s = t_claim(c, CP, in);
        if (c.err) return false;
        if (in) t_put(CP, s, 0, t_box(CN, i), 0, 0, 0);
      }
      __syncwarp();
      return true;
    };
    for (uint32_t lb = 0; lb < c.n_live; lb += 32) {
      const uint32_t li = lb + laneid();
      uint32_t mine = NONE;
      if (li < c.n_live) {
        mine = c.nd->live[li];
        const AllocRec& r = c.nd->allocs[mine];
        if (r.buffer != b || r.mem != pmem) mine = NONE;
      }
      for (uint32_t set = __ballot_sync(FULL, mine != NONE); set; set &= set - 1)
        if (!copy_from(__shfl_sync(FULL, mine, __ffs(set) - 1))) return;
    }
  }
  if (plan) return;  // the buffer state is updated by p4_apply
  Table B = bst_t(c, b);
  t_tidy(c, B);
  const uint32_t from_bst = B.n;
  for (uint32_t i = 0; i < CP.n; ++i) {
    t_or(c, B, NONE, t_box(CP, i), 2, 1u << m);
    if (c.err) return;
  }
  t_merge_from(c, B, from_bst);
}

// ---- a3: push / await push (node level) ------------------------------------

// NB[m] = bounding box of node m's chunks (key DEAD if it has none). The
// chunks of a node are consecutive along the split dimension, so this box is
// exactly their union.
__device__ __noinline__ void node_bboxes(Ctx& c, const Table& CH, Table& NB) {
  for (uint32_t m = 0; m < c.N; ++m) {
    Bx acc;
    acc.lo[0] = acc.lo[1] = acc.lo[2] = 0xFFFFFFFFu;
    acc.hi[0] = acc.hi[1] = acc.hi[2] = 0;
    bool any = false;
    for (uint32_t base = 0; base < CH.n; base += 32) {
      const uint32_t i = base + laneid();
      const bool in = i < CH.n && t_v(CH, 0, i) == m;
      Bx b{};
      if (in) b = t_box(CH, i);
      acc = bx_union(acc, warp_bbox(b, in));
      any = any || __ballot_sync(FULL, in) != 0;
    }
    if (laneid() == 0) t_put(NB, m, any ? 0u : DEAD, acc, 0, 0, 0);
  }
  NB.n = c.N;
  __syncwarp();
}

// The union over a node's chunks of an accessor's mapped boxes is the mapped
// box of the node's chunk range when at most one buffer dimension follows
// each split kernel dimension (dimension 0, and 1 for a split along it): the
// chunks of a node form a full grid, so the per-chunk images are products of
// consecutive intervals.
__device__ __forceinline__ bool union_is_image(const igs_task& t, uint32_t acc, const BufDesc& buf) {
  const igs_accessor& a = t.acc[acc];
  int k0 = 0, k1 = 0;
  for (int d = 0; d < (int)buf.dims; ++d)
    if (a.dim[d].kind == IGS_MAP_AFFINE) {
      if (a.dim[d].a == 0) ++k0;
      if (a.dim[d].a == 1) ++k1;
    }
  return k0 <= 1 && ((t.num_chunks >> 16) == 0 || k1 <= 1);
}

// ---- several warps per node ---------------------------------------------------

// Warp 0 of a block lowers its node; in blocks with helper warps, phases whose
// parts touch disjoint tables and emit nothing whose id depends on another
// part are shared: warp 0 posts a job, every worker does its share, warp 0
// then appends the parts' results in the order of the single-warp path.
enum BlockCmd : uint32_t {
  CMD_NONE = 0, CMD_P5 = 1, CMD_A3 = 2, CMD_P4 = 3, CMD_P4_APPLY = 4, CMD_EXIT = 5, CMD_P5_PLAN = 6, CMD_P5_FINISH = 7,
  CMD_EPOCH = 8, CMD_P3 = 9
};
__device__ void load_ctx(Ctx& c, NodeDev* nd, const ProgDev* pg);

struct WorkJob {
  NodeDev* nd;
  const ProgDev* pg;
  const igs_task* task;
  Table CH, MP, AL, NB;  // warp 0's tables (AL[slot * na]: v0 kernel id, v1/v2 staged edges)
  uint32_t na, epoch, node, workers, stage_cap, seq;
  igs_edge* stage0;  // worker 0's staged edges (warp 0's scratch)
  Table out0;        // worker 0's staged push / await entries (warp 0's scratch)
  uint32_t nbuf;     // push / await, coherence: buffers in ascending order, their staged entries
  uint32_t buf[IGS_MAX_ACCESSORS], buf_off[IGS_MAX_ACCESSORS], buf_cnt[IGS_MAX_ACCESSORS];
  Table PC;          // coherence: the consumers (flags, box, v0 = chunk slot * na + accessor,
                     // v1 / v2 = first staged copy and count)
  uint32_t n_live;   // coherence: live allocations (NodeDev's count is stale during a launch)
  uint32_t devices;  // coherence and kernel phase: devices per node
  uint32_t horizon;  // a9: the instruction older ids are replaced by
  uint32_t p4_states_later;  // coherence: some up-to-date bits are set in the planned kernel phase
  uint32_t p4_split;         // coherence: copies whose up-to-date bits the apply phase sets (in order)
  Table qr;                  // pushes and awaits: warp 0's push / await table
  uint32_t p3_n;             // awaits planned beside the pushes (group gi by helper gi + 1):
  uint32_t p3_g0[kMaxWorkers], p3_g1[kMaxWorkers], p3_dst[kMaxWorkers];  // qr range, host allocation,
  uint32_t p3_nw[kMaxWorkers], p3_nr[kMaxWorkers], p3_cnt[kMaxWorkers];  // copied table sizes, planned count
};

// Pipelined lowering of one node (a launch with several items): a front
// warp (warp kFrontWarp, its own scratch set) runs the node-level step of
// each task ahead of warp 0 — chunks, the overlapping-write check and push /
// await push (a3), which read and update only the node's ownership tables —
// and stages the task's push / await regions in one of kPipeDepth slots;
// warp 0 (the back) takes a slot when it delivers that item. Instruction-
// level state is warp 0's alone, so the lowered graph is unchanged.
constexpr uint32_t kPipeDepth = 4;
constexpr uint32_t kPipeMinItems = 4;  // fewer items per launch: no front warp
constexpr uint32_t kFrontWarp = kMaxWorkers;
struct Pipe {
  volatile uint32_t front_done;  // items the front warp has finished (absolute index)
  volatile uint32_t back_done;   // items warp 0 has delivered
  volatile uint32_t abort;       // set by either side when it stops early
  volatile uint32_t err, err_info;
  volatile uint32_t rejected[kPipeDepth];  // the slot's task had overlapping writes
  volatile uint32_t n[kPipeDepth];         // push / await entries staged in the slot
  uint32_t begin, end;                     // the items this launch lowers
};

struct BlockShared {
  int lock;
  volatile uint32_t cmd, err, err_info;
  WorkJob job;
  uint32_t piped;
  Pipe pipe;
};

__device__ __forceinline__ void worker_bar(uint32_t workers) {
  asm volatile("bar.sync 1, %0;" ::"r"(workers * 32) : "memory");
}

// Worker w's scratch table k (kHelperTables per worker; worker 0 = warp 0
// uses only its staging tables 8-11).
__device__ __forceinline__ uint32_t* helper_table(const NodeDev* nd, uint32_t w, uint32_t k) {
  return nd->helper_scratch + ((size_t)w * kHelperTables + k) * nd->cap_scratch * F_COUNT;
}

__device__ __forceinline__ igs_edge* stage_of(const WorkJob& j, uint32_t w) {
  return w == 0 ? j.stage0 : reinterpret_cast<igs_edge*>(helper_table(j.nd, w, 2));
}

__device__ __forceinline__ Table scratch_table(uint32_t* base, uint32_t cap) {
  Table t;
  t.base = base;
  t.n = 0;
  t.cap = cap;
  t.live = 0;
  t.dp = nullptr;
  return t;
}

// Posts a job (lane 0 has filled sh.job) and runs warp 0's share between the
// start and end barriers; returns false on a failure of any worker.
template <class F>
__device__ bool run_shared(Ctx& c, BlockShared& sh, uint32_t cmd, F share0) {
  __syncwarp();
  if (laneid() == 0) {
    c.nd->prof[31] += 1;  // shared phases run (profile counter)
    sh.err = ST_OK;
    sh.cmd = cmd;
    __threadfence_block();
  }
  __syncwarp();
  worker_bar(c.workers);  // helpers start
  share0();
  worker_bar(c.workers);  // every share done
  if (sh.err != ST_OK && c.err == ST_OK) {
    c.err = sh.err;
    c.err_info = sh.err_info;
  }
  return c.err == ST_OK;
}

// Per buffer: missing_m = reads of node m's chunks not replicated on m; this
// node awaits missing_node and pushes missing_m n owned(node) to every m.
// Results go to the QR table under key seq: v0 = 0 push boxes, 1 await boxes,
// 2 push bbox, 3 await bbox; v1 = buffer; v2 = target node.
// Push / await of one buffer b; the QR entries go to OUT.
__device__ __noinline__ void a3_buffer(Ctx& c, const igs_task& t, uint32_t seq, const Table& CH, const Table& MP,
                                       const Table& NB, uint32_t b, Table& OUT) {
  const uint32_t na = t.num_accessors;
  Table& TMP = c.s[S_T0];
  Table& MISS = c.s[S_T1];
  Table& PT = c.s[S_T2];
  Table& CN = c.s[S_T3];
  t_reset(MISS);
  const BufDesc& bd = buf_of(c, b);
  for (uint32_t m = 0; m < c.N; ++m) {
    t_reset(TMP);
    if (t_key(NB, m) == DEAD) continue;
    const Table O = own_t(c, b);
    auto lacking = [m](uint32_t, uint32_t repl, uint32_t) { return !((repl >> m) & 1u); };
    for (uint32_t a = 0; a < na; ++a) {
      if (t.acc[a].buffer != b || !(t.acc[a].mode & IGS_READ)) continue;
      if (union_is_image(t, a, bd)) {
        const Bx x = map_box(t.acc[a], t_box(NB, m), bd);
        if (!bx_empty(x)) t_query(c, O, NONE, x, TMP, lacking);
      } else {
        for (uint32_t slot = 0; slot < CH.n; ++slot) {
          if (t_v(CH, 0, slot) != m) continue;
          const Bx x = t_box(MP, slot * na + a);
          if (!bx_empty(x)) t_query(c, O, NONE, x, TMP, lacking);
        }
      }
      if (c.err) return;
    }
    t_make_disjoint(c, TMP);
    if (c.err) return;
    for (uint32_t base = 0; base < TMP.n; base += 32) {
      const uint32_t i = base + laneid();
      const bool live = i < TMP.n && t_key(TMP, i) != DEAD;
      const uint32_t s = t_claim(c, MISS, live);
      if (c.err) return;
      if (live) t_put(MISS, s, 0, t_box(TMP, i), m, 0, 0);
    }
    __syncwarp();
  }
  // this node's await (canonical) and bbox
  {
    Table& sel = TMP;
    t_reset(sel);
    for (uint32_t base = 0; base < MISS.n; base += 32) {
      const uint32_t i = base + laneid();
      const bool hit = i < MISS.n && t_v(MISS, 0, i) == c.node;
      const uint32_t s = t_claim(c, sel, hit);
      if (c.err) return;
      if (hit) t_put(sel, s, 0, t_box(MISS, i), 0, 0, 0);
    }
    __syncwarp();
    if (sel.n) {
      t_reset(CN);
      canonical(c, sel, 0, sel.n, CN);
      if (c.err) return;
      const Bx bb = t_bbox(c, CN, 0, CN.n);
      for (uint32_t base = 0; base < CN.n + 1; base += 32) {
        const uint32_t i = base + laneid();
        const bool in = i < CN.n + 1;
        const uint32_t s = t_claim(c, OUT, in);
        if (c.err) return;
        if (in) {
          if (i < CN.n) t_put(OUT, s, seq, t_box(CN, i), 1, b, NONE);
          else t_put(OUT, s, seq, bb, 3, b, NONE);
        }
      }
      __syncwarp();
    }
  }
  // this node's pushes to every other node
  for (uint32_t m = 0; m < c.N; ++m) {
    if (m == c.node) continue;
    t_reset(PT);
    for (uint32_t i = 0; i < MISS.n; ++i) {
      if (t_v(MISS, 0, i) != m) continue;
      const uint32_t me = c.node;
      t_query(c, own_t(c, b), NONE, t_box(MISS, i), PT, [me](uint32_t owner, uint32_t, uint32_t) { return owner == me; });
      if (c.err) return;
    }
    if (PT.n == 0) continue;
    t_reset(CN);
    canonical(c, PT, 0, PT.n, CN);
    if (c.err) return;
    const Bx bb = t_bbox(c, CN, 0, CN.n);
    for (uint32_t base = 0; base < CN.n + 1; base += 32) {
      const uint32_t i = base + laneid();
      const bool in = i < CN.n + 1;
      const uint32_t s = t_claim(c, OUT, in);
      if (c.err) return;
      if (in) {
        if (i < CN.n) t_put(OUT, s, seq, t_box(CN, i), 0, b, m);
        else t_put(OUT, s, seq, bb, 2, b, m);
      }
    }
    __syncwarp();
  }
  // replication: every node now holds what it awaited
  Table O = own_t(c, b);
  t_tidy(c, O);
  const uint32_t from = O.n;
  for (uint32_t i = 0; i < MISS.n; ++i) {
    t_or(c, O, NONE, t_box(MISS, i), 1, 1u << t_v(MISS, 0, i));
    if (c.err) return;
  }
  // writes: owner = writing node, replicated there only
  for (uint32_t a = 0; a < na; ++a) {
    if (t.acc[a].buffer != b || !(t.acc[a].mode & IGS_WRITE)) continue;
    if (union_is_image(t, a, bd)) {
      for (uint32_t wn = 0; wn < c.N; ++wn) {
        if (t_key(NB, wn) == DEAD) continue;
        const Bx x = map_box(t.acc[a], t_box(NB, wn), bd);
        if (!bx_empty(x)) t_set(c, O, NONE, x, wn, 1u << wn, 0);
      }
    } else {
      for (uint32_t slot = 0; slot < CH.n; ++slot) {
        const uint32_t wn = t_v(CH, 0, slot);
        const Bx x = t_box(MP, slot * na + a);
        if (!bx_empty(x)) t_set(c, O, NONE, x, wn, 1u << wn, 0);
      }
    }
    if (c.err) return;
  }
  t_merge_from(c, O, from);
}

// Worker w's buffers of a push / await job: i mod workers == w.
__device__ __noinline__ void a3_share(Ctx& c, WorkJob& j, uint32_t w, Table& OUT) {
  for (uint32_t i = w; i < j.nbuf && !c.err; i += j.workers) {
    const uint32_t from = OUT.n;
    a3_buffer(c, *j.task, j.seq, j.CH, j.MP, j.NB, j.buf[i], OUT);
    __syncwarp();
    if (laneid() == 0) {
      j.buf_off[i] = from;
      j.buf_cnt[i] = OUT.n - from;
    }
    __syncwarp();
  }
}

__device__ __noinline__ void a3_task(Ctx& c, const igs_task& t, uint32_t seq, const Table& CH, const Table& MP) {
  const uint32_t na = t.num_accessors;
  Table& NB = c.s[S_T4];
  node_bboxes(c, CH, NB);
  // the task's buffers, ascending
  uint32_t bufs[IGS_MAX_ACCESSORS], nbuf = 0;
  for (uint32_t done = 0;;) {
    uint32_t b = NONE;
    for (uint32_t a = 0; a < na; ++a)
      if (!(done >> a & 1u) && (b == NONE || t.acc[a].buffer < b)) b = t.acc[a].buffer;
    if (b == NONE) break;
    for (uint32_t a = 0; a < na; ++a)
      if (t.acc[a].buffer == b) done |= 1u << a;
    bufs[nbuf++] = b;
  }
  if (c.block && c.workers > 1 && c.nd->helper_scratch && nbuf > 1) {
    BlockShared& sh = *static_cast<BlockShared*>(c.block);
    WorkJob& j = sh.job;
    Table& OUT0 = c.s[S_T5];
    t_reset(OUT0);
    __syncwarp();
    if (laneid() == 0) {
      j.nd = c.nd;
      j.pg = c.pg;
      j.task = &t;
      j.CH = CH;
      j.MP = MP;
      j.NB = NB;
      j.seq = seq;
      j.epoch = c.epoch;
      j.node = c.node;
      j.workers = c.workers;
      j.nbuf = nbuf;
      for (uint32_t i = 0; i < nbuf; ++i) j.buf[i] = bufs[i];
    }
    if (!run_shared(c, sh, CMD_A3, [&]() { a3_share(c, j, 0, OUT0); })) return;
    // the QR entries in buffer order, as the single-warp path appends them
    for (uint32_t i = 0; i < nbuf; ++i) {
      const uint32_t w = i % c.workers, off = j.buf_off[i], cnt = j.buf_cnt[i];
      const uint32_t* src = w == 0 ? OUT0.base : helper_table(c.nd, w, 5);
      const uint32_t first = __shfl_sync(FULL, t_claim_n(c, c.qr, laneid() == 0 ? cnt : 0u), 0);  // lane 0's slot
      if (c.err) return;
      const uint4* s4 = reinterpret_cast<const uint4*>(src + (size_t)off * F_COUNT);
      uint4* d4 = reinterpret_cast<uint4*>(c.qr.base + (size_t)first * F_COUNT);
      for (uint32_t k = laneid(); k < cnt * (F_COUNT / 4); k += 32) d4[k] = s4[k];
      __syncwarp();
    }
    return;
  }
  for (uint32_t i = 0; i < nbuf; ++i) {
    a3_buffer(c, t, seq, CH, MP, NB, bufs[i], c.qr);
    if (c.err) return;
  }
}

// ---- requirements, allocation planning (a4) --------------------------------

// QR block [qs, qe) of a task (entries of key seq are contiguous).
__device__ void qr_block(const Ctx& c, uint32_t seq, uint32_t& qs, uint32_t& qe) {
  qs = warp_find_first(c, c.qr.n, [&](uint32_t i) { return t_key(c.qr, i) == seq; });
  if (qs == NONE) {
    qs = qe = 0;
    return;
  }
  qe = qs;
  while (qe < c.qr.n && t_key(c.qr, qe) == seq) ++qe;
}

// Appends the requirements (key = buffer * 32 + memory, box) of a task on this
// node: every non-empty mapped box of a local chunk, plus the staging bboxes.
__device__ __noinline__ void requirements(Ctx& c, const igs_task& t, uint32_t seq, const Table& CH, const Table& MP, Table& RQ,
                             uint32_t only_key, uint32_t own_flag) {
  const uint32_t na = t.num_accessors, total = CH.n * na;
  for (uint32_t base = 0; base < total; base += 32) {
    const uint32_t i = base + laneid();
    bool hit = false;
    Bx x{};
    uint32_t key = 0;
    if (i < total) {
      const uint32_t slot = i / na, a = i % na;
      if (t_v(CH, 0, slot) == c.node) {
        x = t_box(MP, i);
        key = t.acc[a].buffer * 32 + t_v(CH, 1, slot);
        hit = !bx_empty(x) && (only_key == NONE || key == only_key);
      }
    }
    const uint32_t s = t_claim(c, RQ, hit);
    if (c.err) return;
    if (hit) t_put(RQ, s, key, x, own_flag, 0, 0);
  }
  uint32_t qs, qe;
  qr_block(c, seq, qs, qe);
  for (uint32_t base = qs; base < qe; base += 32) {
    const uint32_t i = base + laneid();
    bool hit = false;
    uint32_t key = 0;
    if (i < qe) {
      const uint32_t kind = t_v(c.qr, 0, i);
      key = t_v(c.qr, 1, i) * 32 + 1;
      hit = (kind == 2 || kind == 3) && (only_key == NONE || key == only_key);
    }
    const uint32_t s = t_claim(c, RQ, hit);
    if (c.err) return;
    if (hit) t_put(RQ, s, key, t_box(c.qr, i), own_flag, 0, 0);
  }
  __syncwarp();
}

__device__ __noinline__ bool allocating(Ctx& c, const igs_task& t, uint32_t seq, const Table& CH, const Table& MP) {
  Table& RQ = c.s[S_CL];
  t_reset(RQ);
  requirements(c, t, seq, CH, MP, RQ, NONE, 1);
  if (c.err) return false;
  for (uint32_t base = 0; base < RQ.n; base += 32) {
    const uint32_t i = base + laneid();
    bool need = false;
    if (i < RQ.n) {
      const uint32_t key = t_key(RQ, i);
      need = !covered_by_alloc(c, key >> 5, key & 31u, t_box(RQ, i));
    }
    if (__ballot_sync(FULL, need)) return true;
  }
  return false;
}

__device__ __noinline__ void alloc_phase(Ctx& c, const igs_task& t, uint32_t seq, const Table& CH, const Table& MP) {
  Table& RQ = c.s[S_T4];
  Table& CL = c.s[S_CL];
  Table& CH2 = c.s[S_CH2];
  Table& MP2 = c.s[S_MP2];
  Table& Q = c.s[S_T0];
  Table& CN = c.s[S_T5];
  t_reset(RQ);
  requirements(c, t, seq, CH, MP, RQ, NONE, 1);
  if (c.err) return;
  uint32_t last_key = NONE;
  bool first_key = true;
  for (;;) {
    uint64_t best = ~0ull;
    for (uint32_t base = 0; base < RQ.n; base += 32) {
      const uint32_t i = base + laneid();
      uint64_t k = ~0ull;
      if (i < RQ.n) {
        const uint32_t key = t_key(RQ, i);
        if (first_key || key > last_key) k = key;
      }
      k = warp_min64(k);
      best = k < best ? k : best;
    }
    if (best == ~0ull) break;
    first_key = false;
    const uint32_t key = (uint32_t)best;
    last_key = key;
    const uint32_t b = key >> 5, m = key & 31u;
    t_reset(CL);
    for (uint32_t base = 0; base < RQ.n; base += 32) {
      const uint32_t i = base + laneid();
      bool hit = false;
      Bx x{};
      if (i < RQ.n && t_key(RQ, i) == key) {
        x = t_box(RQ, i);
        hit = !covered_by_alloc(c, b, m, x);
      }
      const uint32_t s = t_claim(c, CL, hit);
      if (c.err) return;
      if (hit) t_put(CL, s, 0, x, 1, 0, 0);
    }
    __syncwarp();
    if (CL.n == 0) continue;
    // lookahead: requirements of every task still queued (Sec. 4.3)
    for (uint32_t q = 0; q < c.q_count; ++q) {
      const uint32_t item = c.nd->queue[(c.q_head + q) % c.nd->cap_queue];
      const Item it = c.pg->items[item];
      if (it.kind != IT_TASK) continue;
      const igs_task& qt = c.pg->tasks[it.task];
      task_chunks(c, qt, CH2);
      task_mapped(c, qt, CH2, MP2);
      const uint32_t from = CL.n;
      requirements(c, qt, it.seq, CH2, MP2, CL, key, 0);
      if (c.err) return;
      // drop the ones already inside an allocation
      for (uint32_t base = from; base < CL.n; base += 32) {
        const uint32_t i = base + laneid();
        if (i < CL.n && covered_by_alloc(c, b, m, t_box(CL, i))) t_kill(CL, i);
      }
      __syncwarp();
      for (uint32_t base = from; base < CL.n; base += 32) {
        const uint32_t i = base + laneid();
        if (i < CL.n && t_key(CL, i) != DEAD) FLD(CL, F_KEY, i) = 0;
      }
      __syncwarp();
    }
    // clusters: fixed point of merging positively overlapping bounding boxes
    // and absorbing every overlapping live allocation of (b, m) [positive
    // volume, merely touching boxes stay apart]
    AllocRec* A = c.nd->allocs;
    const uint32_t* L = c.nd->live;
    for (uint32_t base = 0; base < c.n_live; base += 32) {
      const uint32_t i = base + laneid();
      if (i < c.n_live) A[L[i]].mark = NONE;
    }
    __syncwarp();
    for (int guard = 0;; ++guard) {
      if (guard > 1 << 20) {
        fail_internal(c, 3);
        return;
      }
      const uint32_t n = CL.n;
      const uint64_t pairs = (uint64_t)n * n;
      uint32_t found = NONE;
      for (uint64_t base = 0; base < pairs; base += 32) {
        const uint64_t p = base + laneid();
        bool h = false;
        if (p < pairs) {
          const uint32_t i = (uint32_t)(p / n), j = (uint32_t)(p % n);
          h = i < j && t_key(CL, i) != DEAD && t_key(CL, j) != DEAD && bx_overlap(t_box(CL, i), t_box(CL, j));
        }
        const uint32_t mm = __ballot_sync(FULL, h);
        if (mm) {
          found = (uint32_t)(base + __ffs(mm) - 1);
          break;
        }
      }
      if (found != NONE) {
        const uint32_t i = found / n, j = found % n;
        const Bx u = bx_union(t_box(CL, i), t_box(CL, j));
        const uint32_t own = t_v(CL, 0, i) | t_v(CL, 0, j);
        __syncwarp();
        if (laneid() == 0) {
          t_put(CL, i, 0, u, own, 0, 0);
          t_kill(CL, j);
        }
        for (uint32_t base = 0; base < c.n_live; base += 32) {
          const uint32_t x = base + laneid();
          if (x < c.n_live && A[L[x]].mark == j) A[L[x]].mark = i;
        }
        __syncwarp();
        continue;
      }
      // a cluster overlapping an unabsorbed allocation
      const uint32_t nl = c.n_live;
      const uint64_t cp = (uint64_t)n * nl;
      found = NONE;
      for (uint64_t base = 0; base < cp; base += 32) {
        const uint64_t p = base + laneid();
        bool h = false;
        if (p < cp) {
          const uint32_t i = (uint32_t)(p / nl), x = L[(uint32_t)(p % nl)];
          const AllocRec& a = A[x];
          h = t_key(CL, i) != DEAD && a.buffer == b && a.mem == m && a.mark == NONE &&
              bx_overlap(t_box(CL, i), alloc_box(a));
        }
        const uint32_t mm = __ballot_sync(FULL, h);
        if (mm) {
          found = (uint32_t)(base + __ffs(mm) - 1);
          break;
        }
      }
      if (found == NONE) break;
      {
        const uint32_t i = found / nl, x = L[found % nl];
        const Bx u = bx_union(t_box(CL, i), alloc_box(A[x]));
        const uint32_t own = t_v(CL, 0, i);
        __syncwarp();
        if (laneid() == 0) {
          t_put(CL, i, 0, u, own, 0, 0);
          A[x].mark = i;
        }
        __syncwarp();
      }
    }
    // emit one allocation per cluster holding a requirement of this task, in
    // box order; resize: copy the live part of every absorbed allocation, free it
    const uint32_t n = CL.n;
    for (uint32_t base = 0; base < n; base += 32) {
      const uint32_t i = base + laneid();
      if (i < n && t_key(CL, i) != DEAD && t_v(CL, 0, i) == 1) {
        const Bx bi = t_box(CL, i);
        uint32_t rank = 0;
        for (uint32_t j = 0; j < n; ++j)
          if (j != i && t_key(CL, j) != DEAD && t_v(CL, 0, j) == 1 && bx_less(t_box(CL, j), bi)) ++rank;
        FLD(CL, F_V + 1, i) = rank;
      }
    }
    __syncwarp();
    for (uint32_t r = 0;; ++r) {
      const uint32_t ci = warp_find_first(c, n, [&](uint32_t i) {
        return t_key(CL, i) != DEAD && t_v(CL, 0, i) == 1 && t_v(CL, 1, i) == r;
      });
      if (ci == NONE) break;
      const Bx bb = t_box(CL, ci);
      if (c.n_alloc >= c.nd->cap_alloc) {
        fail_cap(c, CAP_ALLOC, c.nd->cap_alloc);
        return;
      }
      const uint32_t aid = c.n_alloc;
      const uint32_t iid = emit(c, IGS_ALLOC, seq, aid, m, b, NONE, &CL, ci, ci + 1, nullptr, 0, false);
      if (c.err) return;
      if (!new_alloc(c, aid, b, m, bb, 0)) return;
      c.n_alloc += 1;
      {
        Table WR = wr_t(c, aid);
        const uint32_t s = t_claim(c, WR, laneid() == 0);
        if (c.err) return;
        if (laneid() == 0) t_put(WR, s, 0, bb, iid, 1, 0);  // v1 = 1: the writer is an allocation
        __syncwarp();
      }
      // the absorbed allocations, ascending (the live list changes as they are freed)
      Table& AB = c.s[S_T3];
      t_reset(AB);
      for (uint32_t base = 0; base < c.n_live; base += 32) {
        const uint32_t x = base + laneid();
        const bool hit = x < c.n_live && L[x] != aid && A[L[x]].mark == ci;
        const uint32_t s = t_claim(c, AB, hit);
        if (c.err) return;
        if (hit) FLD(AB, F_V, s) = L[x];
      }
      __syncwarp();
      for (uint32_t ai = 0; ai < AB.n; ++ai) {
        const uint32_t old = FLD(AB, F_V, ai);
        t_reset(Q);
        t_query(c, bst_t(c, b), NONE, alloc_box(A[old]), Q,
                [m](uint32_t, uint32_t, uint32_t mask) { return ((mask >> m) & 1u) != 0; });
        if (c.err) return;
        t_reset(CN);
        canonical(c, Q, 0, Q.n, CN);
        if (c.err) return;
        if (CN.n) {
          Acc acc[2] = {{&CN, 0, CN.n, old, IGS_READ}, {&CN, 0, CN.n, aid, IGS_WRITE}};
          emit(c, IGS_COPY, seq, old, aid, b, 1, &CN, 0, CN.n, acc, 2, false);
          if (c.err) return;
        }
        emit_free(c, seq, old);
        if (c.err) return;
      }
    }
  }
}

// ---- kernel phase shared by several warps ----------------------------------

// Kernels of different devices touch disjoint allocation tables and depend on
// nothing the others emit in the same phase; their ids are known in advance
// (one per local chunk, in chunk order). So each worker warp takes the chunks
// of the devices d with d mod workers == its index: their dependencies (edges
// staged per worker) and their table updates. Warp 0 then writes edges,
// boxes, bindings and records in chunk order, exactly as the single-warp path.
// The kernel's bindings / accesses of local chunk `slot` into BT and acc.
__device__ bool p5_accesses(Ctx& c, const igs_task& t, const Table& MP, const Table& AL, uint32_t slot, uint32_t na,
                            Table& BT, Acc* acc, int& nacc) {
  t_reset(BT);
  nacc = 0;
  for (uint32_t a = 0; a < na; ++a) {
    const Bx x = t_box(MP, slot * na + a);
    const uint32_t al = FLD(AL, F_KEY, slot * na + a);
    if (al == NONE - 1) {
      fail_internal(c, 4);
      return false;
    }
    if (laneid() == 0) {
      Bx z{};
      t_put(BT, a, 0, bx_empty(x) ? z : x, al, 0, 0);
    }
    if (al != NONE) acc[nacc++] = Acc{&BT, a, a + 1, al, t.acc[a].mode};
  }
  BT.n = na;
  __syncwarp();
  return true;
}

__device__ __noinline__ void p5_share(Ctx& c, const WorkJob& j, uint32_t w) {
  const Table& CH = j.CH;
  const Table& MP = j.MP;
  const Table& AL = j.AL;
  const uint32_t na = j.na;
  Table& BT = c.s[S_T4];
  igs_edge* stage = stage_of(j, w);
  uint32_t off = 0;
  for (uint32_t slot = 0; slot < CH.n && !c.err; ++slot) {
    if (t_v(CH, 0, slot) != j.node) continue;
    const uint32_t mem = t_v(CH, 1, slot);
    if ((mem - 2) % j.workers != w) continue;
    const uint32_t kid = FLD(AL, F_V, slot * na);
    __syncwarp();
    if (laneid() == 0) c.nd->has_succ[kid] = 0;  // before a later kernel of this worker marks it
    Acc acc[IGS_MAX_ACCESSORS];
    int nacc = 0;
    if (!p5_accesses(c, *j.task, MP, AL, slot, na, BT, acc, nacc)) break;
    if (!emit_deps(c, acc, nacc, false)) break;
    const uint32_t ne = emit_edges(c, kid, stage + off, j.stage_cap - off, CAP_TABLE, j.stage_cap);
    if (ne == NONE) break;
    __syncwarp();
    if (laneid() == 0) {
      FLD(AL, F_V + 1, slot * na) = off;
      FLD(AL, F_V + 2, slot * na) = ne;
    }
    off += ne;
    if (!emit_apply(c, acc, nacc, kid)) break;
  }
  __syncwarp();
}

// ---- coherence shared by several warps ---------------------------------------

// One consumer of the coherence phase: PC entry k (flags bit 0 uninitialized
// read, bit 1 stale data). diag: write its warning here (single-warp path).
__device__ bool p4_consumer(Ctx& c, const igs_task& t, uint32_t seq, const Table& CH, const Table& PC, uint32_t k,
                            uint32_t na, bool diag) {
  const uint32_t flags = t_key(PC, k), i = t_v(PC, 0, k);
  const uint32_t slot = i / na, a = i % na;
  const uint32_t mem = t_v(CH, 1, slot), b = t.acc[a].buffer;
  const Bx x = t_box(PC, k);
  if (diag && (flags & 1u)) {  // uninitialized read warning (Sec. 4.4)
    if (c.n_diag >= c.nd->cap_diag) {
      fail_cap(c, CAP_DIAG, c.nd->cap_diag);
      return false;
    }
    if (laneid() == 0) {
      igs_diag dg;
      dg.seq = seq;
      dg.chunk = t_key(CH, slot);
      dg.accessor = a;
      c.nd->diags[c.n_diag] = dg;
    }
    c.n_diag += 1;
    __syncwarp();
  }
  if (!(flags & 2u)) return true;
  const uint32_t dst = find_alloc(c, b, mem, x);
  if (dst == NONE) {
    fail_internal(c, 9);
    return false;
  }
  Table& RG = c.s[S_RG];
  t_reset(RG);
  const uint32_t s = t_claim(c, RG, laneid() == 0);
  if (c.err) return false;
  if (laneid() == 0) t_put(RG, s, 0, x, 0, 0, 0);
  __syncwarp();
  coherence(c, seq, b, mem, dst, RG, 0, 1);
  return c.err == ST_OK;
}

// Coherence with several warps (Sec. 3.3, a5), in two shared phases.
// Plan: worker p4_worker(b, m) takes, in consumer order, the stale consumers
// of buffer b on memory m whose regions meet another one of that pair (the
// others go to the workers in turn) and stages their copies (records, boxes,
// edges) without changing any table. Planning against the tables as they were
// before the phase gives the single-warp path's copies and edges: a copy
// reads a region that is up to date at its producer's memory and writes one
// that is stale at its own, so no copy of the phase reads or writes what
// another one writes; consumers of the same (b, m) see their predecessors'
// copies through the exclusion in coherence().
// Apply: warp 0 appends the staged copies in consumer order (their ids were
// fixed before the phase) while the helpers apply them to the tables: the
// owner of an allocation applies every read and write of it, the owner of a
// buffer's state its up-to-date bits, each in consumer and copy order, so
// every table sees the single-warp path's updates in its order. When the
// kernel phase that follows is planned, the up-to-date bits are set by the
// last worker while the others plan it (nothing in between reads them).
__device__ __forceinline__ uint32_t p4_worker(uint32_t b, uint32_t m, uint32_t devices, uint32_t workers) {
  return (b * devices + m) % workers;
}
// Apply-phase owners among the helpers 1 .. workers-1: with three or more
// workers and the buffer states in this phase, the last one keeps the
// states, the others the allocations.
__device__ __forceinline__ uint32_t p4_alloc_owner(uint32_t aid, uint32_t workers, bool states) {
  if (workers <= 2) return 1u;
  const uint32_t n = states ? workers - 2 : workers - 1;
  return 1u + aid % n;
}
__device__ __forceinline__ uint32_t p4_state_owner(uint32_t workers) { return workers - 1; }

__device__ Stage make_stage(const NodeDev* nd, uint32_t w) {
  Stage st;
  const uint32_t words = nd->cap_scratch * F_COUNT;  // words per table
  st.instrs = reinterpret_cast<igs_instruction*>(helper_table(nd, w, 8));
  st.edges = reinterpret_cast<igs_edge*>(helper_table(nd, w, 9));
  st.boxes = reinterpret_cast<igs_box*>(helper_table(nd, w, 10));
  st.map = helper_table(nd, w, 11);
  st.cap_instr = words * 4 / (uint32_t)sizeof(igs_instruction);
  st.cap_edge = words * 4 / (uint32_t)sizeof(igs_edge);
  st.cap_box = words * 4 / (uint32_t)sizeof(igs_box);
  st.n_instr = st.n_edge = st.n_box = 0;
  st.id_base = PROV | (w << 24);
  return st;
}

// The stale consumer in PC entry k: its buffer, memory and planning worker
// (v3 = worker | memory << 8, v4 = buffer, set when the phase is chosen).
constexpr int F_P4_WM = F_V + 3, F_P4_BUF = F_V + 4;
struct P4Consumer {
  uint32_t b, m, w;
};
__device__ __forceinline__ P4Consumer p4_of(const Table& PC, uint32_t k) {
  const uint32_t wm = FLD(PC, F_P4_WM, k);
  P4Consumer r;
  r.b = FLD(PC, F_P4_BUF, k);
  r.m = wm >> 8;
  r.w = wm & 0xFFu;
  return r;
}
// Calls f(k) in consumer order for the PC entries whose flags meet `want`
// (and, unless w is NONE, that worker w plans), until f returns false.
template <class F>
__device__ __forceinline__ void p4_each(const Table& PC, uint32_t want, uint32_t w, F f) {
  for (uint32_t base = 0; base < PC.n; base += 32) {
    const uint32_t k = base + laneid();
    const bool hit = k < PC.n && (t_key(PC, k) & want) && (w == NONE || (FLD(PC, F_P4_WM, k) & 0xFFu) == w);
    for (uint32_t m = __ballot_sync(FULL, hit); m; m &= m - 1)
      if (!f(base + __ffs(m) - 1)) return;
  }
}

__device__ __noinline__ void p4_share(Ctx& c, WorkJob& j, uint32_t w) {
  Stage st = make_stage(c.nd, w);
  c.stage = &st;
  const Table& PC = j.PC;
  const igs_task& t = *j.task;
  p4_each(PC, 2u, w, [&](uint32_t k) -> bool {
    const uint32_t first = st.n_instr;
    if (!p4_consumer(c, t, j.seq, j.CH, PC, k, j.na, false)) return false;
    __syncwarp();
    if (laneid() == 0) {
      FLD(PC, F_V + 1, k) = first;
      FLD(PC, F_V + 2, k) = st.n_instr - first;
    }
    __syncwarp();
    return true;
  });
  c.stage = nullptr;
}

// The up-to-date bits of the planned copies, in consumer and copy order:
// part 0 the consumers before the one whose copies reach j.p4_split copies,
// part 1 the others.
__device__ __noinline__ void p4_states(Ctx& c, const WorkJob& j, int part) {
  const Table& PC = j.PC;
  uint32_t before = 0;  // copies of the earlier consumers
  p4_each(PC, 2u, NONE, [&](uint32_t k) -> bool {
    const P4Consumer pc = p4_of(PC, k);
    const Stage st = make_stage(c.nd, pc.w);
    const uint32_t first = FLD(PC, F_V + 1, k), cnt = FLD(PC, F_V + 2, k);
    const bool in_part0 = before < j.p4_split;
    before += cnt;
    if (in_part0 != (part == 0)) return true;
    Table B = bst_t(c, pc.b);
    t_tidy(c, B);
    const uint32_t from_bst = B.n;
    for (uint32_t q = first; q < first + cnt; ++q) {
      const igs_instruction r = st.instrs[q];
      for (uint32_t e = 0; e < r.box_cnt; ++e) {
        const igs_box o = st.boxes[r.box_off + e];
        Bx x;
        for (int d = 0; d < 3; ++d) {
          x.lo[d] = o.lo[d];
          x.hi[d] = o.hi[d];
        }
        t_or(c, B, NONE, x, 2, 1u << pc.m);
        if (c.err) return false;
      }
    }
    t_merge_from(c, B, from_bst);
    return c.err == ST_OK;
  });
}

// Helper w's part of the apply phase (the final ids are in the stages' maps).
__device__ __noinline__ void p4_apply(Ctx& c, const WorkJob& j, uint32_t w) {
  const Table& PC = j.PC;
  const bool states = j.p4_split != 0;  // some up-to-date bits are set in this phase
  if (states && p4_state_owner(j.workers) == w && j.workers > 2) {
    p4_states(c, j, 0);
    return;
  }
  p4_each(PC, 2u, NONE, [&](uint32_t k) -> bool {
    const Stage st = make_stage(c.nd, p4_of(PC, k).w);
    const uint32_t first = FLD(PC, F_V + 1, k), cnt = FLD(PC, F_V + 2, k);
    for (uint32_t q = first; q < first + cnt; ++q) {
      const igs_instruction r = st.instrs[q];
      const uint32_t id = st.map[q];
      auto box = [&](uint32_t e, Bx& x) {
        const igs_box o = st.boxes[r.box_off + e];
        for (int d = 0; d < 3; ++d) {
          x.lo[d] = o.lo[d];
          x.hi[d] = o.hi[d];
        }
        return true;
      };
      // a copy reads allocation r.a and writes r.b (reads first, as emit_apply)
      if (p4_alloc_owner(r.a, j.workers, states) == w && !apply_read(c, r.a, r.box_cnt, box, id, false)) return false;
      if (p4_alloc_owner(r.b, j.workers, states) == w && !apply_write(c, r.b, r.box_cnt, box, id)) return false;
    }
    return true;
  });
  if (states && j.workers <= 2 && !c.err) p4_states(c, j, 0);
}

// Warp 0: plan with the helpers; then, in consumer order, the warnings of
// uninitialized reads, the copies' final ids and the capacity checks; then
// the append (warp 0) beside the table updates (helpers).
__device__ __noinline__ void p4_parallel(Ctx& c, const igs_task& t, uint32_t seq, const Table& CH, Table& PC,
                                         uint32_t na, bool states_later) {
  BlockShared& sh = *static_cast<BlockShared*>(c.block);
  WorkJob& j = sh.job;
  __syncwarp();
  if (laneid() == 0) {
    j.nd = c.nd;
    j.pg = c.pg;
    j.task = &t;
    j.CH = CH;
    j.PC = PC;
    j.na = na;
    j.seq = seq;
    j.epoch = c.epoch;
    j.node = c.node;
    j.workers = c.workers;
    j.devices = c.D;
    j.n_live = c.n_live;
    j.p4_states_later = states_later ? 1u : 0u;
  }
  if (!run_shared(c, sh, CMD_P4, [&]() { p4_share(c, j, 0); })) return;
  NodeDev* nd = c.nd;
  uint32_t next = c.n_instr, n_edge = 0, n_box = 0;
  p4_each(PC, 3u, NONE, [&](uint32_t k) -> bool {
    const uint32_t flags = t_key(PC, k);
    if (flags & 1u) {
      const uint32_t i = t_v(PC, 0, k), slot = i / na, a = i % na;
      if (c.n_diag >= nd->cap_diag) {
        fail_cap(c, CAP_DIAG, nd->cap_diag);
        return false;
      }
      if (laneid() == 0) {
        igs_diag dg;
        dg.seq = seq;
        dg.chunk = t_key(CH, slot);
        dg.accessor = a;
        nd->diags[c.n_diag] = dg;
      }
      c.n_diag += 1;
      __syncwarp();
    }
    if (!(flags & 2u)) return true;
    const Stage st = make_stage(nd, p4_of(PC, k).w);
    const uint32_t first = FLD(PC, F_V + 1, k), cnt = FLD(PC, F_V + 2, k);
    for (uint32_t q = first + laneid(); q < first + cnt; q += 32) {
      st.map[q] = next + (q - first);
      n_edge += st.instrs[q].bind_cnt;
      n_box += st.instrs[q].box_cnt;
    }
    next += cnt;
    return true;
  });
  if (c.err) return;
  n_edge = warp_sum(n_edge);
  n_box = warp_sum(n_box);
  if (next > nd->cap_instr || c.n_edge + n_edge > nd->cap_edge) {
    fail_cap(c, CAP_EDGE, nd->cap_edge);
    return;
  }
  if (c.n_box + n_box > nd->cap_box) {
    fail_cap(c, CAP_BOX, nd->cap_box);
    return;
  }
  __syncwarp();
  // with a planned kernel phase to follow, about half of the up-to-date bits
  // wait for it (its last worker plans no kernels)
  if (laneid() == 0) j.p4_split = states_later ? (next - c.n_instr + 1) / 2 : NONE;
  __syncwarp();
  run_shared(c, sh, CMD_P4_APPLY, [&]() {
    p4_each(PC, 2u, NONE, [&](uint32_t k) -> bool {
      const Stage st = make_stage(nd, p4_of(PC, k).w);
      const uint32_t first = FLD(PC, F_V + 1, k), cnt = FLD(PC, F_V + 2, k);
      for (uint32_t q = first; q < first + cnt; ++q) {
        const igs_instruction r = st.instrs[q];
        const uint32_t id = c.n_instr;
        if (laneid() == 0) nd->has_succ[id] = 0;
        // the predecessors were marked when the edges were staged
        for (uint32_t e = laneid(); e < r.bind_cnt; e += 32) {
          igs_edge ed = st.edges[r.bind_off + e];
          ed.to = id;
          nd->edges[c.n_edge + e] = ed;
        }
        for (uint32_t e = laneid(); e < r.box_cnt; e += 32) nd->boxes[c.n_box + e] = st.boxes[r.box_off + e];
        if (laneid() == 0) {
          igs_instruction o = r;
          o.id = id;
          o.box_off = c.n_box;
          o.bind_off = c.n_bind;
          o.bind_cnt = 0;
          nd->instrs[id] = o;
        }
        c.n_edge += r.bind_cnt;
        c.n_box += r.box_cnt;
        c.n_instr += 1;
        __syncwarp();
      }
      return true;
    });
  });
}

// a9 over every table: with helper warps, shared by the workers.
__device__ __noinline__ void apply_epoch(Ctx& c, uint32_t h) {
  if (c.block && c.workers > 1) {
    BlockShared& sh = *static_cast<BlockShared*>(c.block);
    __syncwarp();
    if (laneid() == 0) {
      WorkJob& j = sh.job;
      j.nd = c.nd;
      j.pg = c.pg;
      j.epoch = c.epoch;
      j.node = c.node;
      j.workers = c.workers;
      j.n_live = c.n_live;
      j.horizon = h;
    }
    if (!run_shared(c, sh, CMD_EPOCH, [&]() { epoch_share(c, h, 0, c.workers); })) return;
  } else {
    epoch_share(c, h, 0, 1);
    if (c.err) return;
  }
  c.epoch = h;
}

__device__ __noinline__ void p5_plan(Ctx& c, const WorkJob& j, uint32_t w);
__device__ __noinline__ void p5_finish(Ctx& c, const WorkJob& j, uint32_t w);
__device__ __noinline__ void p3_plan(Ctx& c, WorkJob& j, uint32_t w);

// Helper warp w: waits for work from warp 0, does its share, reports.
__device__ void helper_loop(BlockShared& sh, uint32_t w, uint32_t workers) {
  for (;;) {
    worker_bar(workers);
    const uint32_t cmd = sh.cmd;
    if (cmd == CMD_EXIT) break;
    if (cmd != CMD_NONE) {
      WorkJob& j = sh.job;
      Ctx hc;
      load_ctx(hc, j.nd, j.pg);
      hc.err = ST_OK;
      hc.epoch = j.epoch;
      hc.node = j.node;
      hc.lock = &sh.lock;
      hc.helper = true;
      if (cmd == CMD_P4 || cmd == CMD_P4_APPLY) {
        hc.n_live = j.n_live;
        const int tabs[8] = {S_T0, S_T1, S_T2, S_T3, S_T5, S_RG, S_CAN, S_DEP};
        for (int k = 0; k < 8; ++k) hc.s[tabs[k]].base = helper_table(j.nd, w, k);
        if (cmd == CMD_P4) p4_share(hc, j, w);
        else p4_apply(hc, j, w);
      } else if (cmd == CMD_P3) {
        const int tabs[7] = {S_T1, S_T5, S_RG, S_CAN, S_DEP, S_T4, S_CL};
        for (int k = 0; k < 7; ++k) hc.s[tabs[k]].base = helper_table(j.nd, w, k);
        p3_plan(hc, j, w);
      } else if (cmd == CMD_EPOCH) {
        hc.n_live = j.n_live;
        epoch_share(hc, j.horizon, w, j.workers);
      } else if (cmd == CMD_P5 || cmd == CMD_P5_PLAN || cmd == CMD_P5_FINISH) {
        hc.s[S_DEP].base = helper_table(j.nd, w, 0);
        hc.s[S_T4].base = helper_table(j.nd, w, 1);
        hc.s[S_T3].base = helper_table(j.nd, w, 3);
        if (cmd == CMD_P5) p5_share(hc, j, w);
        else if (cmd == CMD_P5_PLAN) p5_plan(hc, j, w);
        else p5_finish(hc, j, w);
      } else {
        hc.s[S_T0].base = helper_table(j.nd, w, 0);
        hc.s[S_T1].base = helper_table(j.nd, w, 1);
        hc.s[S_T2].base = helper_table(j.nd, w, 2);
        hc.s[S_T3].base = helper_table(j.nd, w, 3);
        hc.s[S_CAN].base = helper_table(j.nd, w, 4);
        Table out = scratch_table(helper_table(j.nd, w, 5), j.nd->cap_scratch);
        a3_share(hc, j, w, out);
      }
      if (laneid() == 0) {
        atomicAdd(reinterpret_cast<unsigned long long*>(&j.nd->map_reads), (unsigned long long)hc.map_reads);
        atomicAdd(reinterpret_cast<unsigned long long*>(&j.nd->map_writes), (unsigned long long)hc.map_writes);
        if (hc.err != ST_OK) {
          sh.err_info = hc.err_info;
          sh.err = hc.err;
        }
      }
      __syncwarp();
    }
    worker_bar(workers);
  }
}

// Warp 0: the kernel phase with the helpers, then the records in chunk order.
__device__ __noinline__ void p5_parallel(Ctx& c, const igs_task& t, uint32_t seq, const Table& CH, const Table& MP,
                                         Table& AL, uint32_t na) {
  BlockShared& sh = *static_cast<BlockShared*>(c.block);
  uint32_t next = c.n_instr;
  for (uint32_t slot = 0; slot < CH.n; ++slot) {
    if (t_v(CH, 0, slot) != c.node) continue;
    if (laneid() == 0) FLD(AL, F_V, slot * na) = next;
    ++next;
  }
  __syncwarp();
  if (laneid() == 0) {
    WorkJob& j = sh.job;
    j.nd = c.nd;
    j.pg = c.pg;
    j.task = &t;
    j.CH = CH;
    j.MP = MP;
    j.AL = AL;
    j.na = na;
    j.epoch = c.epoch;
    j.node = c.node;
    j.workers = c.workers;
    j.stage_cap = c.nd->cap_scratch * (F_COUNT * 4 / (uint32_t)sizeof(igs_edge));
    j.stage0 = reinterpret_cast<igs_edge*>(c.s[S_T0].base);
  }
  if (!run_shared(c, sh, CMD_P5, [&]() { p5_share(c, sh.job, 0); })) return;
  const WorkJob& j = sh.job;
  Table& BT = c.s[S_T4];
  NodeDev* nd = c.nd;
  for (uint32_t slot = 0; slot < CH.n; ++slot) {
    if (t_v(CH, 0, slot) != c.node) continue;
    const uint32_t mem = t_v(CH, 1, slot);
    const uint32_t kid = FLD(AL, F_V, slot * na), off = FLD(AL, F_V + 1, slot * na), ne = FLD(AL, F_V + 2, slot * na);
    if (kid != c.n_instr) {
      fail_internal(c, 5);
      return;
    }
    if (c.n_edge + ne > nd->cap_edge) {
      fail_cap(c, CAP_EDGE, nd->cap_edge);
      return;
    }
    const igs_edge* stage = stage_of(j, (mem - 2) % j.workers);
    for (uint32_t i = laneid(); i < ne; i += 32) nd->edges[c.n_edge + i] = stage[off + i];
    c.n_edge += ne;
    Acc acc[IGS_MAX_ACCESSORS];
    int nacc = 0;
    if (!p5_accesses(c, t, MP, AL, slot, na, BT, acc, nacc)) return;
    if (!emit_record(c, IGS_KERNEL, seq, t_key(CH, slot), mem, t.kernel_id, NONE, &CH, slot, slot + 1, &BT, 0, na,
                     false))
      return;
  }
}

// The buffer state of every region task t writes (AL[slot * na].v0: the
// chunk's kernel); NB: scratch for the nodes' bounding boxes.
__device__ __noinline__ void p5_state(Ctx& c, const igs_task& t, const Table& CH, const Table& MP, const Table& AL,
                                      Table& NB) {
  const uint32_t na = t.num_accessors;
  // buffer state of every written region: a local chunk's kernel is its
  // original producer in the chunk's memory; writes of other nodes make the
  // local copies stale. The written regions of one accessor are disjoint
  // (overlapping writes were rejected), so the order of these updates does
  // not matter.
  node_bboxes(c, CH, NB);
  for (uint32_t a = 0; a < na; ++a) {
    if (!(t.acc[a].mode & IGS_WRITE)) continue;
    const BufDesc& bd = buf_of(c, t.acc[a].buffer);
    Table B = bst_t(c, t.acc[a].buffer);
    t_tidy(c, B);
    const uint32_t from = B.n;
    if (union_is_image(t, a, bd)) {
      // all chunks' writes form the image of the task's range: one subtraction
      Bx all;
      all.lo[0] = all.lo[1] = all.lo[2] = 0xFFFFFFFFu;
      all.hi[0] = all.hi[1] = all.hi[2] = 0;
      for (uint32_t m = 0; m < c.N; ++m)
        if (t_key(NB, m) != DEAD) all = bx_union(all, t_box(NB, m));
      const Bx U = map_box(t.acc[a], all, bd);
      if (!bx_empty(U)) t_subtract(c, B, NONE, U);
      for (uint32_t base = 0; base < CH.n; base += 32) {
        const uint32_t slot = base + laneid();
        bool hit = false;
        Bx x{};
        uint32_t kid = 0, mem = 0;
        if (slot < CH.n && t_v(CH, 0, slot) == c.node) {
          x = t_box(MP, slot * na + a);
          hit = !bx_empty(x);
          kid = FLD(AL, F_V, slot * na);
          mem = t_v(CH, 1, slot);
        }
        const uint32_t s = t_claim(c, B, hit);
        if (c.err) return;
        if (hit) t_put(B, s, 0, x, kid, mem, 1u << mem);
      }
      for (uint32_t m = 0; m < c.N; ++m) {
        if (m == c.node || t_key(NB, m) == DEAD) continue;
        const Bx x = map_box(t.acc[a], t_box(NB, m), bd);
        if (bx_empty(x)) continue;
        const uint32_t s = t_claim(c, B, laneid() == 0);
        if (c.err) return;
        if (laneid() == 0) t_put(B, s, 0, x, REMOTE, 0, 0);
        __syncwarp();
      }
    } else {
      for (uint32_t slot = 0; slot < CH.n; ++slot) {
        const Bx x = t_box(MP, slot * na + a);
        if (bx_empty(x)) continue;
        if (t_v(CH, 0, slot) == c.node) {
          const uint32_t mem = t_v(CH, 1, slot);
          t_set(c, B, NONE, x, FLD(AL, F_V, slot * na), mem, 1u << mem);
        } else {
          t_set(c, B, NONE, x, REMOTE, 0, 0);
        }
        if (c.err) return;
      }
    }
    __syncwarp();
    t_merge_from(c, B, from);
    t_maybe_merge(c, B, 4 * CH.n + 64);
  }
}

// Kernel phase planned per chunk (P5). When no buffer the task writes is
// accessed through a second accessor, no two kernels of the task touch an
// overlapping region of one allocation unless both only read it (the written
// regions of an accessor are disjoint), so no kernel of the task depends on
// another and their dependencies can be found against the tables as they
// were before the phase. Plan: planner li mod planners (every worker but
// the last) takes the li-th local chunk and stages its edges. Finish: every
// planner writes the records of the chunks it planned at offsets fixed in
// between, and the owner of an allocation (a planner) applies every access
// to it in chunk and accessor order (reads, then writes, as emit_apply); the
// last worker updates the buffer state meanwhile. Every table sees the
// single-warp path's updates in its order.
__device__ __forceinline__ bool p5_plannable(const igs_task& t) {
  for (uint32_t a = 0; a < t.num_accessors; ++a) {
    if (!(t.acc[a].mode & IGS_WRITE)) continue;
    for (uint32_t o = 0; o < t.num_accessors; ++o)
      if (o != a && t.acc[o].buffer == t.acc[a].buffer) return false;
  }
  return true;
}
__device__ __forceinline__ uint32_t p5_planners(uint32_t workers) { return workers - 1; }

// AL entries of a local chunk (index slot * na): v0 kernel id, v1 / v2 staged
// edges (offset in the planner's stage, count), v3 / v4 first edge / box in
// the graph, lo[0] first binding in the graph, lo[1] planner. Every entry
// slot * na + a: lo[2] the worker that applies its access (NONE: none).
constexpr int F_EDGE_AT = F_V + 3, F_BOX_AT = F_V + 4, F_BIND_AT = F_LO, F_PLANNER = F_LO + 1, F_OWNER = F_LO + 2;

// Calls f(slot) in chunk order for the local chunks planner w plans, until f
// returns false.
template <class F>
__device__ __forceinline__ void p5_each_planned(const WorkJob& j, uint32_t w, F f) {
  for (uint32_t base = 0; base < j.CH.n; base += 32) {
    const uint32_t slot = base + laneid();
    const bool mine = slot < j.CH.n && t_v(j.CH, 0, slot) == j.node && FLD(j.AL, F_PLANNER, slot * j.na) == w;
    for (uint32_t m = __ballot_sync(FULL, mine); m; m &= m - 1)
      if (!f(base + __ffs(m) - 1)) return;
  }
}

__device__ __noinline__ void p5_plan(Ctx& c, const WorkJob& j, uint32_t w) {
  if (w == p5_planners(j.workers)) {  // plans nothing: the coherence phase's up-to-date bits
    if (j.p4_states_later) p4_states(c, j, 1);
    return;
  }
  const Table& AL = j.AL;
  const uint32_t na = j.na;
  Table& BT = c.s[S_T4];
  igs_edge* stage = stage_of(j, w);
  uint32_t off = 0;
  p5_each_planned(j, w, [&](uint32_t slot) -> bool {
    const uint32_t kid = FLD(AL, F_V, slot * na);
    __syncwarp();
    if (laneid() == 0) c.nd->has_succ[kid] = 0;
    Acc acc[IGS_MAX_ACCESSORS];
    int nacc = 0;
    if (!p5_accesses(c, *j.task, j.MP, AL, slot, na, BT, acc, nacc)) return false;
    if (!emit_deps(c, acc, nacc, false)) return false;
    const uint32_t ne = emit_edges(c, kid, stage + off, j.stage_cap - off, CAP_TABLE, j.stage_cap);
    if (ne == NONE) return false;
    __syncwarp();
    if (laneid() == 0) {
      FLD(AL, F_V + 1, slot * na) = off;
      FLD(AL, F_V + 2, slot * na) = ne;
    }
    off += ne;
    return true;
  });
  __syncwarp();
}

__device__ __noinline__ void p5_finish(Ctx& c, const WorkJob& j, uint32_t w) {
  const Table& CH = j.CH;
  const Table& MP = j.MP;
  const Table& AL = j.AL;
  const igs_task& t = *j.task;
  const uint32_t na = j.na;
  NodeDev* nd = c.nd;
  if (w == p5_planners(j.workers)) {
    p5_state(c, t, CH, MP, AL, c.s[S_T3]);
    return;
  }
  Table& BT = c.s[S_T4];
  const igs_edge* stage = stage_of(j, w);
  // the records of the chunks this worker planned
  p5_each_planned(j, w, [&](uint32_t slot) -> bool {
    const uint32_t i0 = slot * na;
    const uint32_t kid = FLD(AL, F_V, i0), off = FLD(AL, F_V + 1, i0), ne = FLD(AL, F_V + 2, i0);
    const uint32_t e_at = FLD(AL, F_EDGE_AT, i0), b_at = FLD(AL, F_BOX_AT, i0), d_at = FLD(AL, F_BIND_AT, i0);
    for (uint32_t e = laneid(); e < ne; e += 32) nd->edges[e_at + e] = stage[off + e];
    Acc acc[IGS_MAX_ACCESSORS];
    int nacc = 0;
    if (!p5_accesses(c, t, MP, AL, slot, na, BT, acc, nacc)) return false;
    const Ent ch = t_ent(CH, slot);
    const uint32_t nb = ch.key != DEAD ? 1u : 0u;
    if (laneid() < na) {
      const Ent bi = t_ent(BT, laneid());
      igs_binding o;
      o.alloc = bi.v0;
      for (int d = 0; d < 3; ++d) {
        o.lo[d] = bi.b.lo[d];
        o.hi[d] = bi.b.hi[d];
      }
      nd->binds[d_at + laneid()] = o;
    }
    if (laneid() == 0) {
      if (nb) {
        igs_box o;
        for (int d = 0; d < 3; ++d) {
          o.lo[d] = ch.b.lo[d];
          o.hi[d] = ch.b.hi[d];
        }
        nd->boxes[b_at] = o;
      }
      igs_instruction r;
      r.id = kid;
      r.type = IGS_KERNEL;
      r.seq = j.seq;
      r.a = ch.key;
      r.b = ch.v1;  // the chunk's memory
      r.c = t.kernel_id;
      r.d = NONE;
      r.box_off = b_at;
      r.box_cnt = nb;
      r.bind_off = d_at;
      r.bind_cnt = na;
      nd->instrs[kid] = r;
    }
    __syncwarp();
    return true;
  });
  // the accesses this worker applies, in chunk and accessor order: an
  // allocation of a written buffer serves one accessor (its read, then its
  // write), one of a read-only buffer only reads, so each allocation sees
  // emit_apply's order
  const uint32_t total = CH.n * na;
  for (uint32_t base = 0; base < total && !c.err; base += 32) {
    const uint32_t i = base + laneid();
    const bool mine = i < total && FLD(AL, F_OWNER, i) == w;
    for (uint32_t m = __ballot_sync(FULL, mine); m; m &= m - 1) {
      const uint32_t e = base + __ffs(m) - 1, slot = e / na, a = e % na;
      const uint32_t al = FLD(AL, F_KEY, e), kid = FLD(AL, F_V, slot * na), mode = t.acc[a].mode;
      const Bx x = t_box(MP, e);
      auto box = [&](uint32_t, Bx& q) {
        q = x;
        return true;
      };
      if (mode & IGS_READ) {
        bool again = false;
        for (uint32_t o = 0; o < a; ++o)
          if ((t.acc[o].mode & IGS_READ) && FLD(AL, F_KEY, slot * na + o) == al) again = true;
        if (!apply_read(c, al, 1, box, kid, again)) return;
      }
      if ((mode & IGS_WRITE) && !apply_write(c, al, 1, box, kid)) return;
    }
  }
}

// Warp 0: kernel ids, planners and owners; plan with the helpers; every
// local kernel's place in the graph; finish with the helpers.
__device__ __noinline__ void p5_planned(Ctx& c, const igs_task& t, uint32_t seq, const Table& CH, const Table& MP,
                                        Table& AL, uint32_t na, bool p4_states_pending) {
  BlockShared& sh = *static_cast<BlockShared*>(c.block);
  NodeDev* nd = c.nd;
  const uint32_t planners = p5_planners(c.workers);
  {
    uint32_t k = 0;
    for (uint32_t base = 0; base < CH.n; base += 32) {
      const uint32_t slot = base + laneid();
      const bool local = slot < CH.n && t_v(CH, 0, slot) == c.node;
      const uint32_t mask = __ballot_sync(FULL, local), r = k + __popc(mask & lanemask_lt());
      if (local) {
        FLD(AL, F_V, slot * na) = c.n_instr + r;
        FLD(AL, F_PLANNER, slot * na) = r % planners;
      }
      k += __popc(mask);
    }
    // an allocation's owner is one function of (buffer, memory): the
    // accessor that first names the buffer and the chunk's memory
    const uint32_t total = CH.n * na;
    for (uint32_t base = 0; base < total; base += 32) {
      const uint32_t i = base + laneid();
      if (i < total) {
        const uint32_t slot = i / na, a = i % na;
        uint32_t owner = NONE;
        if (FLD(AL, F_KEY, i) != NONE && t_v(CH, 0, slot) == c.node) {
          uint32_t first = a;
          for (uint32_t o = 0; o < a; ++o)
            if (t.acc[o].buffer == t.acc[a].buffer) {
              first = o;
              break;
            }
          owner = (first * c.D + t_v(CH, 1, slot)) % planners;
        }
        FLD(AL, F_OWNER, i) = owner;
      }
    }
  }
  __syncwarp();
  if (laneid() == 0) {
    WorkJob& j = sh.job;
    j.nd = nd;
    j.pg = c.pg;
    j.task = &t;
    j.CH = CH;
    j.MP = MP;
    j.AL = AL;
    j.na = na;
    j.seq = seq;
    j.epoch = c.epoch;
    j.node = c.node;
    j.workers = c.workers;
    j.devices = c.D;
    j.stage_cap = nd->cap_scratch * (F_COUNT * 4 / (uint32_t)sizeof(igs_edge));
    j.stage0 = reinterpret_cast<igs_edge*>(c.s[S_T0].base);
    j.p4_states_later = p4_states_pending ? 1u : 0u;  // j.PC still holds the coherence consumers
  }
  if (!run_shared(c, sh, CMD_P5_PLAN, [&]() { p5_plan(c, sh.job, 0); })) return;
  // places in chunk order; the first kernel that would overflow a capacity
  // fails as in the single-warp path (edges and records, then boxes, then
  // bindings)
  uint32_t n_edge = c.n_edge, n_box = c.n_box, n_bind = c.n_bind, n_k = 0, bad = NONE, bad_kind = 0;
  for (uint32_t base = 0; base < CH.n; base += 32) {
    const uint32_t slot = base + laneid();
    const bool local = slot < CH.n && t_v(CH, 0, slot) == c.node;
    const uint32_t ne = local ? FLD(AL, F_V + 2, slot * na) : 0u;
    const uint32_t nb = local && t_key(CH, slot) != DEAD ? 1u : 0u;
    uint32_t te, tb, tk;
    const uint32_t xe = warp_excl_scan(ne, te), xb = warp_excl_scan(nb, tb), xk = warp_excl_scan(local ? 1u : 0u, tk);
    uint32_t kind = 0;
    if (local) {
      FLD(AL, F_EDGE_AT, slot * na) = n_edge + xe;
      FLD(AL, F_BOX_AT, slot * na) = n_box + xb;
      FLD(AL, F_BIND_AT, slot * na) = n_bind + xk * na;
      if (n_edge + xe + ne > nd->cap_edge || c.n_instr + n_k + xk + 1 > nd->cap_instr) kind = 1;
      else if (n_box + xb + nb > nd->cap_box) kind = 2;
      else if (n_bind + (xk + 1) * na > nd->cap_bind) kind = 3;
    }
    const uint32_t fails = __ballot_sync(FULL, kind != 0);
    if (fails && bad == NONE) {
      bad = base + __ffs(fails) - 1;
      bad_kind = __shfl_sync(FULL, kind, __ffs(fails) - 1);
    }
    n_edge += te;
    n_box += tb;
    n_bind += tk * na;
    n_k += tk;
  }
  if (bad != NONE) {
    if (bad_kind == 1) fail_cap(c, CAP_EDGE, nd->cap_edge);
    else if (bad_kind == 2) fail_cap(c, CAP_BOX, nd->cap_box);
    else fail_cap(c, CAP_BIND, nd->cap_bind);
    return;
  }
  __syncwarp();
  if (!run_shared(c, sh, CMD_P5_FINISH, [&]() { p5_finish(c, sh.job, 0); })) return;
  c.n_instr += n_k;
  c.n_edge = n_edge;
  c.n_box = n_box;
  c.n_bind = n_bind;
}

// P2 of task item (qr entries [qs, qe)): per (buffer, target) in ascending
// order, coherence copies into host memory and one send per (original
// producer, canonical box).
__device__ __noinline__ void p2_pushes(Ctx& c, uint32_t seq, uint32_t qs, uint32_t qe) {
  Table& Q = c.s[S_T0];
  Table& G = c.s[S_T1];
  Table& CN = c.s[S_T5];
  Table& RG = c.s[S_RG];
  for (uint32_t g0 = qs; g0 < qe;) {
    uint32_t g1 = g0;
    while (g1 < qe && t_v(c.qr, 0, g1) == t_v(c.qr, 0, g0)) ++g1;  // boxes, then one bbox entry
    const uint32_t kind = t_v(c.qr, 0, g0);
    if (kind != 0) {
      g0 = g1 + (kind == 1 ? 1 : 0);
      continue;
    }
    const uint32_t b = t_v(c.qr, 1, g0), target = t_v(c.qr, 2, g0);
    const Bx bb = t_box(c.qr, g1);  // the bbox entry follows the boxes
    const uint32_t dst = find_alloc(c, b, 1, bb);
    if (dst == NONE) {
      fail_internal(c, 6);
      return;
    }
    // copy the push region into RG (coherence uses the scratch tables)
    t_reset(RG);
    for (uint32_t base = g0; base < g1; base += 32) {
      const uint32_t i = base + laneid();
      const bool in = i < g1;
      const uint32_t s = t_claim(c, RG, in);
      if (c.err) return;
      if (in) t_put(RG, s, 0, t_box(c.qr, i), 0, 0, 0);
    }
    __syncwarp();
    coherence(c, seq, b, 1, dst, RG, 0, RG.n);
    if (c.err) return;
    // sends: one per (original producer, canonical box)
    t_reset(Q);
    {
      const Table B = bst_t(c, b);
      for (uint32_t r = 0; r < RG.n; ++r) {
        t_query(c, B, NONE, t_box(RG, r), Q, [](uint32_t, uint32_t, uint32_t) { return true; });
        if (c.err) return;
      }
    }
    uint64_t last = 0;
    bool first_round = true;
    for (;;) {
      uint64_t best = ~0ull;
      for (uint32_t base = 0; base < Q.n; base += 32) {
        const uint32_t i = base + laneid();
        uint64_t k = ~0ull;
        if (i < Q.n) {
          k = ((uint64_t)t_v(Q, 0, i) << 32) | t_v(Q, 1, i);
          if (!first_round && k <= last) k = ~0ull;
        }
        k = warp_min64(k);
        best = k < best ? k : best;
      }
      if (best == ~0ull) break;
      first_round = false;
      last = best;
      t_reset(G);
      for (uint32_t base = 0; base < Q.n; base += 32) {
        const uint32_t i = base + laneid();
        const bool hit = i < Q.n && (((uint64_t)t_v(Q, 0, i) << 32) | t_v(Q, 1, i)) == best;
        const uint32_t s = t_claim(c, G, hit);
        if (c.err) return;
        if (hit) t_put(G, s, 0, t_box(Q, i), 0, 0, 0);
      }
      __syncwarp();
      t_reset(CN);
      canonical(c, G, 0, G.n, CN);
      if (c.err) return;
      for (uint32_t i = 0; i < CN.n; ++i) {
        Acc acc[1] = {{&CN, i, i + 1, dst, IGS_READ}};
        emit(c, IGS_SEND, seq, dst, target, b, c.next_msg, &CN, i, i + 1, acc, 1, false);
        if (c.err) return;
        c.next_msg += 1;
      }
    }
    g0 = g1 + 1;
  }
}

// P3 for one await group qr[g0, g1) (its bounding-box entry at g1) into
// host allocation dst: one receive, or a split receive and one await receive
// per consumer part. Planned by a helper (c.stage set): the instructions go
// to its stage and no table changes (p3_finish applies them afterwards).
__device__ __noinline__ void p3_group(Ctx& c, const igs_task& t, uint32_t seq, const Table& CH, const Table& MP,
                                      const Table& qr, uint32_t g0, uint32_t g1, uint32_t dst) {
  const uint32_t na = t.num_accessors;
  const bool plan = c.stage != nullptr;
  const uint32_t b = t_v(qr, 1, g0);
  Table& CONS = c.s[S_T4];
  Table& COV = c.s[S_CL];
  Table& G = c.s[S_T1];
  Table& CN = c.s[S_T5];
  Table& RG = c.s[S_RG];
  t_reset(RG);
  uint64_t wvol = 0;
  for (uint32_t base = g0; base < g1; base += 32) {
    const uint32_t i = base + laneid();
    const bool in = i < g1;
    const uint32_t s = t_claim(c, RG, in);
    if (c.err) return;
    if (in) t_put(RG, s, 0, t_box(qr, i), 0, 0, 0);
  }
  __syncwarp();
  for (uint32_t i = laneid(); i < RG.n; i += 32) wvol += bx_volume(t_box(RG, i));
  wvol = warp_sum64(wvol);
  const Bx rg_bb = t_bbox(c, RG, 0, RG.n);
  // consumers in (chunk, accessor) order: v0 = consumer index
  t_reset(CONS);
  uint32_t ncons = 0;
  bool whole = true;
  const uint32_t total = CH.n * na;
  for (uint32_t eb = 0; eb < total; eb += 32) {
    bool cand = false;
    if (eb + laneid() < total) {
      const uint32_t e = eb + laneid(), slot = e / na, a = e % na;
      if (t_v(CH, 0, slot) == c.node && t.acc[a].buffer == b && (t.acc[a].mode & IGS_READ)) {
        const Bx x = t_box(MP, e);
        cand = !bx_empty(x) && bx_overlap(x, rg_bb);  // else it reads nothing awaited
      }
    }
    for (uint32_t cm = __ballot_sync(FULL, cand); cm; cm &= cm - 1) {
      const Bx x = t_box(MP, eb + __ffs(cm) - 1);
      uint64_t vol = 0;
      const uint32_t from = CONS.n;
      for (uint32_t base = 0; base < RG.n; base += 32) {
        const uint32_t i = base + laneid();
        Bx is{};
        bool hit = false;
        if (i < RG.n) {
          is = bx_isect(t_box(RG, i), x);
          hit = !bx_empty(is);
        }
        const uint32_t s = t_claim(c, CONS, hit);
        if (c.err) return;
        if (hit) t_put(CONS, s, 0, is, ncons, 0, 0);
      }
      __syncwarp();
      if (CONS.n == from) continue;
      for (uint32_t i = from + laneid(); i < CONS.n; i += 32) vol += bx_volume(t_box(CONS, i));
      if (warp_sum64(vol) != wvol) whole = false;
      ++ncons;
    }
  }
  if (ncons <= 1) whole = true;
  if (whole) {
    Acc acc[1] = {{&RG, 0, RG.n, dst, IGS_WRITE}};
    const uint32_t id = emit(c, IGS_RECEIVE, seq, dst, NONE, b, NONE, &RG, 0, RG.n, acc, 1, false);
    if (c.err || plan) return;
    Table B = bst_t(c, b);
    t_tidy(c, B);
    const uint32_t from = B.n;
    for (uint32_t i = 0; i < RG.n; ++i) {
      t_set(c, B, NONE, t_box(RG, i), id, 1, 1u << 1);
      if (c.err) return;
    }
    t_merge_from(c, B, from);
  } else {
    Acc acc[1] = {{&RG, 0, RG.n, dst, IGS_WRITE}};
    const uint32_t sid = emit(c, IGS_SPLIT_RECEIVE, seq, dst, NONE, b, NONE, &RG, 0, RG.n, acc, 1, false);
    if (c.err) return;
    t_reset(COV);
    for (uint32_t k = 0; k < ncons; ++k) {
      // part = consumer k's region minus what earlier await receives cover
      t_reset(G);
      for (uint32_t base = 0; base < CONS.n; base += 32) {
        const uint32_t i = base + laneid();
        const bool hit = i < CONS.n && t_v(CONS, 0, i) == k;
        const uint32_t s = t_claim(c, G, hit);
        if (c.err) return;
        if (hit) t_put(G, s, 0, t_box(CONS, i), 0, 0, 0);
      }
      __syncwarp();
      for (uint32_t i = 0; i < COV.n; ++i) {
        t_subtract(c, G, NONE, t_box(COV, i));
        if (c.err) return;
      }
      t_reset(CN);
      canonical(c, G, 0, G.n, CN);
      if (c.err) return;
      if (CN.n == 0) continue;
      Table& D = c.s[S_DEP];
      t_reset(D);
      if (laneid() == 0) {
        FLD(D, F_V, 0) = sid;
        FLD(D, F_V + 1, 0) = IGS_DEP_DATAFLOW;
      }
      D.n = 1;
      __syncwarp();
      const uint32_t aid = emit(c, IGS_AWAIT_RECEIVE, seq, dst, sid, b, NONE, &CN, 0, CN.n, nullptr, 0, true);
      if (c.err) return;
      if (!plan) {
        Table WR = wr_t(c, dst);
        Table B = bst_t(c, b);
        t_tidy(c, WR);
        t_tidy(c, B);
        const uint32_t fw = WR.n, fb = B.n;
        for (uint32_t i = 0; i < CN.n; ++i) {
          const Bx x = t_box(CN, i);
          t_set(c, WR, NONE, x, aid, 0, 0);
          t_set(c, B, NONE, x, aid, 1, 1u << 1);
          if (c.err) return;
        }
        t_merge_from(c, WR, fw);
        t_merge_from(c, B, fb);
      }
      for (uint32_t base = 0; base < CN.n; base += 32) {
        const uint32_t i = base + laneid();
        const bool in = i < CN.n;
        const uint32_t s = t_claim(c, COV, in);
        if (c.err) return;
        if (in) t_put(COV, s, 0, t_box(CN, i), 0, 0, 0);
      }
      __syncwarp();
    }
  }
}

// P2 with P3 beside it (helper warps): the await groups' receives are planned
// by helpers 1, 2, ... (one group each) while warp 0 emits the pushes. A
// receive writes host memory the node awaits; a push reads and sends what
// the node owns, so the two phases touch disjoint regions of a host
// allocation and never depend on one another. The planner finds a receive's
// dependencies in a copy of its allocation's tables taken before the pushes.
// Afterwards warp 0 appends the planned instructions in group order and
// applies their table updates as the single-warp path does. Returns false
// (nothing done) when the phases stay sequential.
__device__ __noinline__ void p3_plan(Ctx& c, WorkJob& j, uint32_t w) {
  const uint32_t gi = w - 1;
  if (w == 0 || gi >= j.p3_n) return;
  Stage st = make_stage(c.nd, w);
  c.stage = &st;
  const uint32_t nw = j.p3_nw[gi];
  c.snap_alloc = j.p3_dst[gi];
  c.snap_tab[0] = helper_table(c.nd, w, 7);
  c.snap_n[0] = nw;
  c.snap_tab[1] = c.snap_tab[0] + (size_t)nw * F_COUNT;
  c.snap_n[1] = j.p3_nr[gi];
  p3_group(c, *j.task, j.seq, j.CH, j.MP, j.qr, j.p3_g0[gi], j.p3_g1[gi], j.p3_dst[gi]);
  __syncwarp();
  if (laneid() == 0) j.p3_cnt[gi] = st.n_instr;
  c.stage = nullptr;
  c.snap_alloc = NONE;
}

__device__ __noinline__ bool p23_parallel(Ctx& c, const igs_task& t, uint32_t seq, const Table& CH, const Table& MP,
                                          uint32_t qs, uint32_t qe) {
  if (!c.block || c.workers < 2 || !c.nd->helper_scratch || c.nd->stage_d2d) return false;
  NodeDev* nd = c.nd;
  BlockShared& sh = *static_cast<BlockShared*>(c.block);
  WorkJob& j = sh.job;
  // the groups: pushes to overlap with, awaits that fit one helper each
  uint32_t n = 0, pushes = 0;
  uint32_t g0s[kMaxWorkers], g1s[kMaxWorkers], dsts[kMaxWorkers];
  for (uint32_t g0 = qs; g0 < qe;) {
    uint32_t g1 = g0;
    while (g1 < qe && t_v(c.qr, 0, g1) == t_v(c.qr, 0, g0)) ++g1;
    const uint32_t kind = t_v(c.qr, 0, g0);
    if (kind == 0) ++pushes;
    if (kind != 1) {
      g0 = g1 + (kind == 0 ? 1 : 0);
      continue;
    }
    if (n + 1 >= c.workers) return false;
    const uint32_t dst = find_alloc(c, t_v(c.qr, 1, g0), 1, t_box(c.qr, g1));
    if (dst == NONE) {
      fail_internal(c, 7);
      return false;
    }
    const Table WR = wr_t(c, dst), RD = rd_t(c, dst);
    if (WR.n + RD.n > nd->cap_scratch) return false;
    g0s[n] = g0;
    g1s[n] = g1;
    dsts[n] = dst;
    ++n;
    g0 = g1 + 1;
  }
  if (n == 0 || pushes == 0) return false;
  // the copies of the receiving allocations' tables (writers, then readers)
  for (uint32_t gi = 0; gi < n; ++gi) {
    const Table WR = wr_t(c, dsts[gi]), RD = rd_t(c, dsts[gi]);
    uint4* out = reinterpret_cast<uint4*>(helper_table(nd, gi + 1, 7));
    const uint32_t q = F_COUNT / 4;  // 16-byte words per entry
    const uint4* w4 = reinterpret_cast<const uint4*>(WR.base);
    const uint4* r4 = reinterpret_cast<const uint4*>(RD.base);
    for (uint32_t k = laneid(); k < WR.n * q; k += 32) out[k] = w4[k];
    for (uint32_t k = laneid(); k < RD.n * q; k += 32) out[WR.n * q + k] = r4[k];
    if (laneid() == 0) {
      j.p3_g0[gi] = g0s[gi];
      j.p3_g1[gi] = g1s[gi];
      j.p3_dst[gi] = dsts[gi];
      j.p3_nw[gi] = WR.n;
      j.p3_nr[gi] = RD.n;
    }
  }
  __syncwarp();
  if (laneid() == 0) {
    j.nd = nd;
    j.pg = c.pg;
    j.task = &t;
    j.CH = CH;
    j.MP = MP;
    j.qr = c.qr;
    j.na = t.num_accessors;
    j.seq = seq;
    j.epoch = c.epoch;
    j.node = c.node;
    j.workers = c.workers;
    j.p3_n = n;
  }
  if (!run_shared(c, sh, CMD_P3, [&]() { p2_pushes(c, seq, qs, qe); })) return true;
  // the planned instructions in group order, each with the single-warp
  // path's table updates
  for (uint32_t gi = 0; gi < n && !c.err; ++gi) {
    const Stage st = make_stage(nd, gi + 1);
    const uint32_t dst = j.p3_dst[gi], b = t_v(c.qr, 1, j.p3_g0[gi]), cnt = j.p3_cnt[gi];
    for (uint32_t q = 0; q < cnt; ++q) {
      const igs_instruction r = st.instrs[q];
      const uint32_t id = c.n_instr;
      if (c.n_instr + 1 > nd->cap_instr || c.n_edge + r.bind_cnt > nd->cap_edge) {
        fail_cap(c, CAP_EDGE, nd->cap_edge);
        return true;
      }
      if (c.n_box + r.box_cnt > nd->cap_box) {
        fail_cap(c, CAP_BOX, nd->cap_box);
        return true;
      }
      __syncwarp();
      if (laneid() == 0) {
        st.map[q] = id;
        nd->has_succ[id] = 0;
      }
      __syncwarp();
      for (uint32_t e = laneid(); e < r.bind_cnt; e += 32) {
        igs_edge ed = st.edges[r.bind_off + e];
        if (ed.from & PROV) {  // the split receive of this group
          ed.from = st.map[ed.from & 0xFFFFFFu];
          nd->has_succ[ed.from] = 1;
        }
        ed.to = id;
        nd->edges[c.n_edge + e] = ed;
      }
      for (uint32_t e = laneid(); e < r.box_cnt; e += 32) nd->boxes[c.n_box + e] = st.boxes[r.box_off + e];
      if (laneid() == 0) {
        igs_instruction o = r;
        o.id = id;
        if (o.b != NONE && (o.b & PROV)) o.b = st.map[o.b & 0xFFFFFFu];  // an await receive's split receive
        o.box_off = c.n_box;
        o.bind_off = c.n_bind;
        o.bind_cnt = 0;
        nd->instrs[id] = o;
      }
      c.n_edge += r.bind_cnt;
      c.n_box += r.box_cnt;
      c.n_instr += 1;
      __syncwarp();
      auto box = [&](uint32_t e, Bx& x) {
        const igs_box o = st.boxes[r.box_off + e];
        for (int d = 0; d < 3; ++d) {
          x.lo[d] = o.lo[d];
          x.hi[d] = o.hi[d];
        }
        return true;
      };
      if (r.type == IGS_RECEIVE || r.type == IGS_SPLIT_RECEIVE) {
        if (!apply_write(c, dst, r.box_cnt, box, id)) return true;
        if (r.type == IGS_SPLIT_RECEIVE) continue;
        Table B = bst_t(c, b);
        t_tidy(c, B);
        const uint32_t from = B.n;
        for (uint32_t e = 0; e < r.box_cnt; ++e) {
          Bx x;
          box(e, x);
          t_set(c, B, NONE, x, id, 1, 1u << 1);
          if (c.err) return true;
        }
        t_merge_from(c, B, from);
      } else {  // an await receive
        Table WR = wr_t(c, dst);
        Table B = bst_t(c, b);
        t_tidy(c, WR);
        t_tidy(c, B);
        const uint32_t fw = WR.n, fb = B.n;
        for (uint32_t e = 0; e < r.box_cnt; ++e) {
          Bx x;
          box(e, x);
          t_set(c, WR, NONE, x, id, 0, 0);
          t_set(c, B, NONE, x, id, 1, 1u << 1);
          if (c.err) return true;
        }
        t_merge_from(c, WR, fw);
        t_merge_from(c, B, fb);
      }
    }
  }
  return true;
}

// ---- compile one task (P1..P5) ----------------------------------------------

__device__ __noinline__ void compile_task(Ctx& c, uint32_t item) {
  const Item it = c.pg->items[item];
  const igs_task& t = c.pg->tasks[it.task];
  const uint32_t seq = it.seq, na = t.num_accessors;
  Table& CH = c.s[S_CH];
  Table& MP = c.s[S_MP];
  PhaseTimer pt = pt_start();
  // delivered and compiled at once: chunks and mapped boxes are still in
  // place and the task was found not to allocate
  const bool fresh = c.fresh == item;
  if (!fresh) {
    task_chunks(c, t, CH);
    task_mapped(c, t, CH, MP);
  }
  if (c.err) return;
  pt_lap(pt, c, PH_SPLIT);
  // P1 (nothing to do unless some requirement lies outside every allocation)
  if (!fresh && allocating(c, t, seq, CH, MP)) alloc_phase(c, t, seq, CH, MP);
  if (c.err) return;
  pt_lap(pt, c, PH_P1);
  uint32_t qs, qe;
  qr_block(c, seq, qs, qe);
  // P2: pushes; P3: awaits (with helper warps, P3 is planned beside P2)
  if (!p23_parallel(c, t, seq, CH, MP, qs, qe)) {
    if (c.err) return;
    p2_pushes(c, seq, qs, qe);
    if (c.err) return;
    pt_lap(pt, c, PH_P2);
    for (uint32_t g0 = qs; g0 < qe;) {
      uint32_t g1 = g0;
      while (g1 < qe && t_v(c.qr, 0, g1) == t_v(c.qr, 0, g0)) ++g1;
      const uint32_t kind = t_v(c.qr, 0, g0);
      if (kind != 1) {
        g0 = g1 + (kind == 0 ? 1 : 0);
        continue;
      }
      const uint32_t dst = find_alloc(c, t_v(c.qr, 1, g0), 1, t_box(c.qr, g1));
      if (dst == NONE) {
        fail_internal(c, 7);
        return;
      }
      p3_group(c, t, seq, CH, MP, c.qr, g0, g1, dst);
      if (c.err) return;
      g0 = g1 + 1;
    }
  }
  if (c.err) return;
  pt_lap(pt, c, PH_P3);
  // P4: coherence for every reading accessor, (chunk, accessor) order.
  // Pre-check, one lane per consumer: does its box overlap never-written data
  // (bit 0) or data not up to date in its memory (bit 1)? Copies emitted in
  // this phase only add up-to-date memories and leave producers unchanged, so
  // a consumer with nothing stale now has nothing stale when its turn comes.
  Table& PC = c.s[S_CL];
  t_reset(PC);
  {
    const uint32_t total = CH.n * na;
    for (uint32_t base = 0; base < total; base += 32) {
      const uint32_t i = base + laneid();
      bool hit = false;
      uint32_t flags = 0;
      Bx x{};
      if (i < total) {
        const uint32_t slot = i / na, a = i % na;
        if (t_v(CH, 0, slot) == c.node && (t.acc[a].mode & IGS_READ)) {
          x = t_box(MP, i);
          hit = !bx_empty(x);
          if (hit) {
            const uint32_t b = t.acc[a].buffer, m = t_v(CH, 1, slot);
            const Table B = heap_table(c.nd, c.nd->bst_d + kDesc * b);
            for (uint32_t j = 0; j < B.n; ++j) {
              if (t_key(B, j) == DEAD || !bx_overlap(t_box(B, j), x)) continue;
              const uint32_t prod = t_v(B, 0, j), mask = t_v(B, 2, j);
              if (prod == NONE) flags |= 1u;
              else if (!((mask >> m) & 1u)) flags |= 2u;
            }
          }
        }
      }
      const uint32_t s = t_claim(c, PC, hit);
      if (c.err) return;
      if (hit) t_put(PC, s, flags, x, i, 0, 0);
    }
    __syncwarp();
  }
  // stale consumers that more than one worker would plan: shared by the
  // helper warps. A consumer whose region meets no other stale consumer of
  // its (buffer, memory) sees none of their copies, so it goes to the next
  // worker in turn; the others are planned in order by their pair's worker.
  bool multi = false;
  if (c.block && c.workers > 1 && c.nd->helper_scratch && !c.nd->stage_d2d) {
    for (uint32_t base = 0; base < PC.n; base += 32) {
      const uint32_t k = base + laneid();
      if (k < PC.n && (t_key(PC, k) & 2u)) {
        const uint32_t i = t_v(PC, 0, k);
        FLD(PC, F_P4_WM, k) = t_v(CH, 1, i / na) << 8;
        FLD(PC, F_P4_BUF, k) = t.acc[i % na].buffer;
      }
    }
    __syncwarp();
    uint32_t used = 0, turn = 0;
    for (uint32_t base = 0; base < PC.n; base += 32) {
      const uint32_t k = base + laneid();
      const bool stale = k < PC.n && (t_key(PC, k) & 2u);
      const uint32_t mask = __ballot_sync(FULL, stale);
      if (stale) {
        const uint32_t b = FLD(PC, F_P4_BUF, k), m = FLD(PC, F_P4_WM, k) >> 8;
        const Bx x = t_box(PC, k);
        bool alone = true;
        for (uint32_t o = 0; o < PC.n && alone; ++o)
          if (o != k && (t_key(PC, o) & 2u) && FLD(PC, F_P4_BUF, o) == b && (FLD(PC, F_P4_WM, o) >> 8) == m &&
              bx_overlap(t_box(PC, o), x))
            alone = false;
        const uint32_t w = alone ? (turn + __popc(mask & lanemask_lt())) % c.workers : p4_worker(b, m, c.D, c.workers);
        FLD(PC, F_P4_WM, k) = w | (m << 8);
        used |= 1u << w;
      }
      turn += __popc(mask);
    }
    multi = __popc(warp_or(used)) >= 2;
  }
  // a planned kernel phase sets the coherence copies' up-to-date bits
  const bool p5_shared = c.block && c.workers > 2 && c.nd->helper_scratch && p5_plannable(t);
  if (multi) {
    p4_parallel(c, t, seq, CH, PC, na, p5_shared);
    if (c.err) return;
  } else {
    for (uint32_t k = 0; k < PC.n; ++k) {
      if (!t_key(PC, k)) continue;
      if (!p4_consumer(c, t, seq, CH, PC, k, na, true)) return;
    }
  }
  pt_lap(pt, c, PH_P4);
  // P5: one device kernel per local chunk; every accessor's allocation is
  // looked up first, one lane per (chunk, accessor)
  Table& BT = c.s[S_T4];
  Table& AL = c.s[S_T5];
  {
    const uint32_t total = CH.n * na;
    if (total > AL.cap) {
      fail_cap(c, CAP_TABLE, AL.cap);
      return;
    }
    const AllocRec* A = c.nd->allocs;
    const uint32_t* L = c.nd->live;
    for (uint32_t base = 0; base < total; base += 32) {
      const uint32_t i = base + laneid();
      if (i < total) {
        const uint32_t slot = i / na, a = i % na;
        uint32_t al = NONE;
        if (t_v(CH, 0, slot) == c.node) {
          const Bx x = t_box(MP, i);
          if (!bx_empty(x)) {
            const uint32_t buf = t.acc[a].buffer, mem = t_v(CH, 1, slot);
            for (uint32_t k = 0; k < c.n_live && al == NONE; ++k) {
              const AllocRec& r = A[L[k]];
              if (r.buffer == buf && r.mem == mem && bx_contains(alloc_box(r), x)) al = L[k];
            }
            if (al == NONE) al = NONE - 1;  // missing: an internal error
          }
        }
        FLD(AL, F_KEY, i) = al;
      }
    }
    AL.n = total;
    __syncwarp();
  }
  bool planned = false;
  if (c.block && c.workers > 1 && c.nd->helper_scratch) {
    planned = p5_plannable(t);
    if (planned) p5_planned(c, t, seq, CH, MP, AL, na, multi && p5_shared);
    else p5_parallel(c, t, seq, CH, MP, AL, na);
    if (c.err) return;
  } else {
    for (uint32_t slot = 0; slot < CH.n; ++slot) {
      if (t_v(CH, 0, slot) != c.node) continue;
      const uint32_t mem = t_v(CH, 1, slot);
      Acc acc[IGS_MAX_ACCESSORS];
      int nacc = 0;
      if (!p5_accesses(c, t, MP, AL, slot, na, BT, acc, nacc)) return;
      const uint32_t kid = emit(c, IGS_KERNEL, seq, t_key(CH, slot), mem, t.kernel_id, NONE, &CH, slot, slot + 1, acc,
                                nacc, false, &BT, 0, na);
      if (c.err) return;
      __syncwarp();
      if (laneid() == 0) FLD(AL, F_V, slot * na) = kid;  // the chunk's kernel, for the buffer state below
      __syncwarp();
    }
  }
  pt_lap(pt, c, PH_P5);
  if (!planned) p5_state(c, t, CH, MP, AL, c.s[S_T3]);
  if (c.err) return;
  // the task's push / await regions are consumed
  for (uint32_t base = qs; base < qe; base += 32) {
    const uint32_t i = base + laneid();
    if (i < qe) t_kill(c.qr, i);
  }
  t_dead(c, c.qr, qe - qs);
  __syncwarp();
  pt_lap(pt, c, PH_REMOTE);
}

// ---- items ---------------------------------------------------------------------

__device__ __noinline__ void process(Ctx& c, uint32_t item) {
  const Item it = c.pg->items[item];
  switch (it.kind) {
    case IT_CREATE: {
      const BufDesc& bd = buf_of(c, it.arg);
      const Bx dom = buffer_box(bd);
      if (it.arg >= c.nd->cap_buffers) {
        fail_cap(c, CAP_BUFFERS, c.nd->cap_buffers);
        return;
      }
      if (!table_new(c, c.nd->bst_d + kDesc * it.arg, 32)) return;
      Table B = bst_t(c, it.arg);
      if (bd.init) {
        const uint32_t aid = c.n_alloc;
        if (!new_alloc(c, aid, it.arg, 0, dom, 1)) return;
        c.n_alloc += 1;
        Table WR = wr_t(c, aid);
        const uint32_t s = t_claim(c, WR, laneid() == 0);
        if (c.err) return;
        if (laneid() == 0) t_put(WR, s, 0, dom, c.epoch, 0, 0);
        const uint32_t s2 = t_claim(c, B, laneid() == 0);
        if (c.err) return;
        if (laneid() == 0) t_put(B, s2, 0, dom, c.epoch, 0, 1u);
      } else {
        const uint32_t s2 = t_claim(c, B, laneid() == 0);
        if (c.err) return;
        if (laneid() == 0) t_put(B, s2, 0, dom, NONE, 0, 0);
      }
      __syncwarp();
      break;
    }
    case IT_TASK:
      compile_task(c, item);
      break;
    case IT_HORIZON:
    case IT_EPOCH: {
      Table& D = c.s[S_DEP];
      t_reset(D);
      for (uint32_t base = c.last_sync; base < c.n_instr; base += 32) {
        const uint32_t i = base + laneid();
        const bool f = i < c.n_instr && !c.nd->has_succ[i];
        const uint32_t s = t_claim(c, D, f);
        if (c.err) return;
        if (f) {
          FLD(D, F_V, s) = i;
          FLD(D, F_V + 1, s) = IGS_DEP_FRONT;
        }
      }
      __syncwarp();
      PhaseTimer pt = pt_start();
      const uint32_t id = emit(c, it.kind == IT_EPOCH ? IGS_EPOCH : IGS_HORIZON, it.seq, NONE, NONE, NONE, NONE,
                               nullptr, 0, 0, nullptr, 0, true);
      if (c.err) return;
      pt_lap(pt, c, PH_SYNC);
      c.last_sync = id;
      if (it.kind == IT_EPOCH) {
        apply_epoch(c, id);
        c.last_horizon = NONE;
      } else {
        if (c.last_horizon != NONE) apply_epoch(c, c.last_horizon);
        c.last_horizon = id;
      }
      pt_lap(pt, c, PH_APPLY);
      break;
    }
    case IT_DESTROY: {
      const uint32_t b = it.arg;
      Table& AB = c.s[S_T3];
      t_reset(AB);
      for (uint32_t base = 0; base < c.n_live; base += 32) {
        const uint32_t x = base + laneid();
        const bool hit = x < c.n_live && c.nd->allocs[c.nd->live[x]].buffer == b;
        const uint32_t s = t_claim(c, AB, hit);
        if (c.err) return;
        if (hit) FLD(AB, F_V, s) = c.nd->live[x];
      }
      __syncwarp();
      for (uint32_t m = 0; m < 2 + c.D; ++m)
        for (uint32_t ai = 0; ai < AB.n; ++ai) {
          const uint32_t aid = FLD(AB, F_V, ai);
          const AllocRec a = c.nd->allocs[aid];
          if (a.mem != m) continue;
          if (!a.user) {
            emit_free(c, it.seq, aid);
            if (c.err) return;
          } else {
            drop_alloc(c, aid);
          }
        }
      table_free(c, c.nd->bst_d + kDesc * b);
      break;
    }
    default:
      break;
  }
}

__device__ uint32_t queued_tasks(const Ctx& c) {
  uint32_t k = 0;
  for (uint32_t q = 0; q < c.q_count; ++q)
    if (c.pg->items[c.nd->queue[(c.q_head + q) % c.nd->cap_queue]].kind == IT_TASK) ++k;
  return k;
}

__device__ void flush_queue(Ctx& c) {
  while (c.q_count > 0 && !c.err) {
    const uint32_t item = c.nd->queue[c.q_head];
    c.q_head = (c.q_head + 1) % c.nd->cap_queue;
    c.q_count -= 1;
    process(c, item);
  }
}

__device__ void enqueue(Ctx& c, uint32_t item) {
  if (c.q_count >= c.nd->cap_queue) {
    fail_cap(c, CAP_QUEUE, c.nd->cap_queue);
    return;
  }
  if (laneid() == 0) c.nd->queue[(c.q_head + c.q_count) % c.nd->cap_queue] = item;
  c.q_count += 1;
  __syncwarp();
}

__device__ void maintain(Ctx& c) { t_tidy(c, c.qr); }

// Horizon-count lookahead (Sec. 4.3 "Lookahead Heuristic"). The requirement
// boxes of every task queued in this mode are kept in the QR table (kind 4,
// v1 = buffer * 32 + memory) until the task is compiled. A task is allocating
// while the queue is non-empty when one of its requirement boxes lies neither
// inside a live allocation nor inside a queued requirement box of the same
// (buffer, memory).
constexpr uint32_t QR_QUEUED_REQ = 4;

__device__ bool covered_by_queued(const Ctx& c, uint32_t key, const Bx& b) {
  for (uint32_t i = 0; i < c.qr.n; ++i)
    if (t_key(c.qr, i) != DEAD && t_v(c.qr, 0, i) == QR_QUEUED_REQ && t_v(c.qr, 1, i) == key &&
        bx_contains(t_box(c.qr, i), b))
      return true;
  return false;
}

__device__ __noinline__ bool allocating_queued(Ctx& c, const igs_task& t, uint32_t seq, const Table& CH,
                                                const Table& MP) {
  Table& RQ = c.s[S_CL];
  t_reset(RQ);
  requirements(c, t, seq, CH, MP, RQ, NONE, 1);
  if (c.err) return false;
  for (uint32_t base = 0; base < RQ.n; base += 32) {
    const uint32_t i = base + laneid();
    bool need = false;
    if (i < RQ.n) {
      const uint32_t key = t_key(RQ, i);
      const Bx x = t_box(RQ, i);
      need = !covered_by_alloc(c, key >> 5, key & 31u, x) && !covered_by_queued(c, key, x);
    }
    if (__ballot_sync(FULL, need)) return true;
  }
  return false;
}

// Appends a queued task's requirement boxes to its QR block.
__device__ __noinline__ void record_queued_reqs(Ctx& c, const igs_task& t, uint32_t seq, const Table& CH,
                                                 const Table& MP) {
  Table& RQ = c.s[S_CL];
  t_reset(RQ);
  requirements(c, t, seq, CH, MP, RQ, NONE, 1);
  for (uint32_t base = 0; base < RQ.n && !c.err; base += 32) {
    const uint32_t i = base + laneid();
    const bool in = i < RQ.n;
    const uint32_t s = t_claim(c, c.qr, in);
    if (c.err) return;
    if (in) t_put(c.qr, s, seq, t_box(RQ, i), QR_QUEUED_REQ, t_key(RQ, i), 0);
  }
  __syncwarp();
}

// Scheduler lookahead (Sec. 4.3): a task is queued while an allocating task
// is queued; the queue is compiled when it holds more than `lookahead` tasks,
// at an epoch, or when a buffer is destroyed.
// The node-level ownership table of a new buffer: the whole buffer owned by
// user memory (host data) or by no one, replicated on every node.
__device__ void own_create(Ctx& c, const Item& it) {
  if (it.arg >= c.nd->cap_buffers) {
    fail_cap(c, CAP_BUFFERS, c.nd->cap_buffers);
    return;
  }
  const BufDesc& bd = buf_of(c, it.arg);
  if (!table_new(c, c.nd->own_d + kDesc * it.arg, 32)) return;
  Table O = own_t(c, it.arg);
  const uint32_t s = t_claim(c, O, laneid() == 0);
  if (c.err) return;
  if (laneid() == 0) t_put(O, s, 0, buffer_box(bd), bd.init ? HOST : NONE, 0xFFFFFFFFu, 0);
  __syncwarp();
}

// Warp 0 of a pipelined launch: the push / await regions the front warp
// staged for this item are appended to the QR table (as a3_task appends its
// own).
__device__ void pipe_take(Ctx& c, uint32_t item) {
  const uint32_t slot = item % kPipeDepth, cnt = c.pipe->n[slot];
  if (cnt == 0) return;
  const uint32_t* src = helper_table(c.nd, kFrontWarp, 8 + slot);
  const uint32_t first = __shfl_sync(FULL, t_claim_n(c, c.qr, laneid() == 0 ? cnt : 0u), 0);  // lane 0's slot
  if (c.err) return;
  const uint4* s4 = reinterpret_cast<const uint4*>(src);
  uint4* d4 = reinterpret_cast<uint4*>(c.qr.base + (size_t)first * F_COUNT);
  for (uint32_t k = laneid(); k < cnt * (F_COUNT / 4); k += 32) d4[k] = s4[k];
  __syncwarp();
}

__device__ __noinline__ void deliver(Ctx& c, uint32_t item) {
  const Item it = c.pg->items[item];
  maintain(c);
  if (c.err) return;
  if (it.kind == IT_LOOKAHEAD) {
    // switching to the horizon count compiles the queue first
    if (it.arg == IGS_LOOKAHEAD_HORIZONS && c.q_count > 0) flush_queue(c);
    c.lookahead = it.arg;
    c.q_hzn = 0;
    if (c.q_count > 0 && queued_tasks(c) > c.lookahead) flush_queue(c);
    return;
  }
  if (it.kind == IT_CREATE && !c.pipe) {  // pipelined: the front warp creates it
    own_create(c, it);
    if (c.err) return;
  }
  bool alloc_now = false;
  if (it.kind == IT_TASK) {
    const igs_task& t = c.pg->tasks[it.task];
    Table& CH = c.s[S_CH];
    Table& MP = c.s[S_MP];
    PhaseTimer pt = pt_start();
    task_chunks(c, t, CH);
    task_mapped(c, t, CH, MP);
    if (c.err) return;
    pt_lap(pt, c, PH_SPLIT);
    // pipelined: the front warp has checked the task and staged its push /
    // await regions
    const bool bad = c.pipe ? c.pipe->rejected[item % kPipeDepth] != 0 : overlapping_writes(c, t, CH, MP);
    pt_lap(pt, c, PH_OVERLAP);
    if (bad) {
      if (c.n_rej < c.nd->cap_rej) {
        if (laneid() == 0) c.nd->rejected[c.n_rej] = it.seq;
        c.n_rej += 1;
        __syncwarp();
      }
      return;
    }
    if (c.pipe) pipe_take(c, item);
    else a3_task(c, t, it.seq, CH, MP);
    if (c.err) return;
    pt_lap(pt, c, PH_A3);
    if (c.q_count == 0) alloc_now = allocating(c, t, it.seq, CH, MP);
    else if (c.lookahead == IGS_LOOKAHEAD_HORIZONS) alloc_now = allocating_queued(c, t, it.seq, CH, MP);
    if (c.err) return;
    pt_lap(pt, c, PH_ALLOCATING);
  }
  const bool horizons = c.lookahead == IGS_LOOKAHEAD_HORIZONS;
  if (c.q_count == 0) {
    if (alloc_now) {
      enqueue(c, item);
      c.q_hzn = 0;
      if (horizons) record_queued_reqs(c, c.pg->tasks[it.task], it.seq, c.s[S_CH], c.s[S_MP]);
      else if (queued_tasks(c) > c.lookahead) flush_queue(c);
    } else {
      if (it.kind == IT_TASK) c.fresh = item;  // nothing changes the allocations before it compiles
      process(c, item);
      c.fresh = NONE;
    }
  } else if (horizons) {
    // compile once two horizons follow the last task the queue would not make room for
    enqueue(c, item);
    if (it.kind == IT_TASK) {
      record_queued_reqs(c, c.pg->tasks[it.task], it.seq, c.s[S_CH], c.s[S_MP]);
      if (alloc_now) c.q_hzn = 0;
    }
    if (it.kind == IT_HORIZON) c.q_hzn += 1;
    if (it.kind == IT_EPOCH || it.kind == IT_DESTROY || c.q_hzn >= 2) flush_queue(c);
  } else {
    enqueue(c, item);
    if (it.kind == IT_EPOCH || it.kind == IT_DESTROY || queued_tasks(c) > c.lookahead) flush_queue(c);
  }
  if (c.err) return;
  if (it.kind == IT_DESTROY && !c.pipe) table_free(c, c.nd->own_d + kDesc * it.arg);
}

__device__ void load_ctx(Ctx& c, NodeDev* nd, const ProgDev* pg) {
  c.nd = nd;
  c.pg = pg;
  c.lane = threadIdx.x & 31u;
  c.err = nd->status;
  c.err_info = nd->err_info;
  c.node = nd->node;
  c.N = nd->N;
  c.D = nd->D;
  c.epoch = nd->epoch;
  c.last_horizon = nd->last_horizon;
  c.last_sync = nd->last_sync;
  c.next_msg = nd->next_msg;
  c.n_alloc = nd->n_alloc;
  c.n_free = nd->n_free;
  c.n_live = nd->n_live;
  c.heap_top = nd->heap_top;
  c.n_instr = nd->n_instr;
  c.n_edge = nd->n_edge;
  c.n_box = nd->n_box;
  c.n_bind = nd->n_bind;
  c.n_diag = nd->n_diag;
  c.n_rej = nd->n_rej;
  c.lookahead = nd->lookahead;
  c.q_head = nd->q_head;
  c.q_count = nd->q_count;
  c.q_hzn = nd->q_hzn;
  c.qr.base = nd->qr_base;
  c.qr.n = nd->qr_n;
  c.qr.cap = nd->cap_qr;
  c.qr.live = nd->qr_live;
  c.qr.dp = nullptr;
  for (int k = 0; k < 14; ++k) {
    c.s[k].base = nd->scratch_base + (size_t)k * nd->cap_scratch * F_COUNT;
    c.s[k].n = 0;
    c.s[k].cap = nd->cap_scratch;
    c.s[k].live = 0;
    c.s[k].dp = nullptr;
  }
  c.map_reads = 0;
  c.map_writes = 0;
  c.lock = nullptr;
  c.block = nullptr;
  c.workers = 1;
  c.stage = nullptr;
  c.snap_alloc = NONE;
  c.helper = false;
  c.fresh = NONE;
  c.pipe = nullptr;
}

__device__ void store_ctx(Ctx& c, uint32_t cursor) {
  __syncwarp();
  if (laneid() != 0) return;
  NodeDev* nd = c.nd;
  nd->status = c.err;
  nd->err_info = c.err_info;
  nd->cursor = cursor;
  nd->epoch = c.epoch;
  nd->last_horizon = c.last_horizon;
  nd->last_sync = c.last_sync;
  nd->next_msg = c.next_msg;
  nd->n_alloc = c.n_alloc;
  nd->n_free = c.n_free;
  nd->n_live = c.n_live;
  if (!c.lock) nd->heap_top = c.heap_top;  // with a lock, NodeDev holds the top throughout
  nd->n_instr = c.n_instr;
  nd->n_edge = c.n_edge;
  nd->n_box = c.n_box;
  nd->n_bind = c.n_bind;
  nd->n_diag = c.n_diag;
  nd->n_rej = c.n_rej;
  nd->lookahead = c.lookahead;
  nd->q_head = c.q_head;
  nd->q_count = c.q_count;
  nd->q_hzn = c.q_hzn;
  nd->qr_n = c.qr.n;
  nd->qr_live = c.qr.live;
  nd->map_reads += c.map_reads;
  nd->map_writes += c.map_writes;
  nd->launches += 1;
}

// One warp per unit; each lowers the unit's pending items (at most max_items).
// Publishes a node's progress to host-mapped memory: every record it counts
// is written (and fenced) before the counts.
__device__ __noinline__ void publish_progress(const Ctx& c, volatile uint32_t* pr, uint32_t cursor) {
  __syncwarp();
  if (laneid() == 0) {
    __threadfence_system();
    pr[PR_INSTR] = c.n_instr;
    pr[PR_EDGE] = c.n_edge;
    pr[PR_BOX] = c.n_box;
    pr[PR_BIND] = c.n_bind;
    pr[PR_STATUS] = c.err;
    __threadfence_system();
    pr[PR_CURSOR] = cursor;  // last: the host reads it first
  }
  __syncwarp();
}

// Waits (every lane polls) until ready() holds; false when the other side
// of the pipeline stopped (taking its error, if any) or after 30 s of device
// time (ST_TIMEOUT, and the other side is told to stop). Polls back off from
// min_ns to 2 us between looks (the front warp, usually ahead, mostly sleeps).
template <class F>
__device__ bool pipe_wait(Ctx& c, Pipe& P, F ready, uint32_t min_ns) {
  uint64_t t0;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t0));
  uint32_t ns = min_ns;
  for (;;) {
    if (__any_sync(FULL, P.abort != 0)) {
      if (P.err != ST_OK && c.err == ST_OK) {
        c.err = P.err;
        c.err_info = P.err_info;
      }
      return false;
    }
    if (__all_sync(FULL, ready())) break;
    uint64_t t1;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t1));
    if (__shfl_sync(FULL, t1 - t0, 0) > 30000000000ull) {
      fail(c, ST_TIMEOUT);
      __syncwarp();
      if (laneid() == 0) {
        P.err = ST_TIMEOUT;
        __threadfence_block();
        P.abort = 1;
      }
      __syncwarp();
      return false;
    }
    __nanosleep(ns);
    ns = ns < 2048u ? 2 * ns : 2048u;
  }
  __threadfence_block();
  return true;
}

// The front warp of a pipelined launch (see Pipe): items [begin, end) of one
// node, at most kPipeDepth ahead of warp 0.
__device__ void front_loop(BlockShared& sh, const Unit u) {
  Pipe& P = sh.pipe;
  Ctx f;
  load_ctx(f, u.node, u.prog);
  f.err = ST_OK;
  f.lock = &sh.lock;
  f.helper = true;
  const uint32_t cap = u.node->cap_scratch;
  const int used[8] = {S_CH, S_MP, S_T0, S_T1, S_T2, S_T3, S_T4, S_CAN};
  for (int k = 0; k < 14; ++k) f.s[k] = scratch_table(nullptr, 0);  // tables the front never uses
  for (int k = 0; k < 8; ++k) f.s[used[k]] = scratch_table(helper_table(u.node, kFrontWarp, k), cap);
  for (uint32_t i = P.begin; i < P.end && f.err == ST_OK; ++i) {
    if (!pipe_wait(f, P, [&]() { return i - P.back_done < kPipeDepth; }, 256)) break;
    const uint32_t slot = i % kPipeDepth;
    f.qr = scratch_table(helper_table(u.node, kFrontWarp, 8 + slot), cap);
    uint32_t rejected = 0;
    const Item it = f.pg->items[i];
    if (it.kind == IT_CREATE) {
      own_create(f, it);
    } else if (it.kind == IT_TASK) {
      const igs_task& t = f.pg->tasks[it.task];
      task_chunks(f, t, f.s[S_CH]);
      task_mapped(f, t, f.s[S_CH], f.s[S_MP]);
      if (f.err == ST_OK) {
        if (overlapping_writes(f, t, f.s[S_CH], f.s[S_MP])) rejected = 1;
        else a3_task(f, t, it.seq, f.s[S_CH], f.s[S_MP]);
      }
    } else if (it.kind == IT_DESTROY) {
      table_free(f, f.nd->own_d + kDesc * it.arg);
    }
    if (f.err != ST_OK) break;
    __syncwarp();
    if (laneid() == 0) {
      P.rejected[slot] = rejected;
      P.n[slot] = f.qr.n;
      __threadfence_block();
      P.front_done = i + 1;
    }
    __syncwarp();
  }
  if (laneid() == 0) {
    if (f.err != ST_OK) {
      P.err_info = f.err_info;
      P.err = f.err;
      __threadfence_block();
      P.abort = 1;
    }
    atomicAdd(reinterpret_cast<unsigned long long*>(&u.node->map_reads), (unsigned long long)f.map_reads);
    atomicAdd(reinterpret_cast<unsigned long long*>(&u.node->map_writes), (unsigned long long)f.map_writes);
  }
  __syncwarp();
}

__device__ void lower_unit(const Unit* units, uint32_t n_units, uint32_t max_items, uint32_t w,
                           volatile uint32_t* progress, BlockShared* sh, uint32_t workers, Pipe* pipe = nullptr) {
  if (w >= n_units) return;
  const Unit u = units[w];
  Ctx c;
  load_ctx(c, u.node, u.prog);
  if (sh && c.nd->helper_scratch) {  // nodes without helper scratch lower alone
    c.lock = &sh->lock;
    c.block = sh;
    c.workers = workers;
  }
  uint32_t cursor = u.node->cursor;
  const uint32_t avail = *u.prog->n_items;
  uint32_t end = avail;
  if (max_items != NONE && cursor + max_items < end) end = cursor + max_items;
  if (pipe) {  // the same items as the front warp
    c.pipe = pipe;
    cursor = pipe->begin;
    end = pipe->end;
  }
  volatile uint32_t* pr = progress ? progress + (size_t)w * PR_WORDS : nullptr;
  PhaseTimer pt = pt_start();
  uint64_t* const item_ts = u.node->item_ts;
  while (cursor < end && c.err == ST_OK) {
    if (pipe && !pipe_wait(c, *pipe, [&]() { return pipe->front_done > cursor; }, 32)) break;
    deliver(c, cursor);
    if (item_ts && laneid() == 0) {
      uint64_t t;
      asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
      item_ts[cursor] = t;
    }
    ++cursor;
    if (pipe) {
      __syncwarp();
      if (laneid() == 0) {
        __threadfence_block();
        pipe->back_done = cursor;  // the item's slot is free again
      }
      __syncwarp();
    }
    if (pr) publish_progress(c, pr, cursor);
  }
  if (pipe) {  // the front warp leaves any wait
    __syncwarp();
    if (laneid() == 0) {
      if (c.err != ST_OK && pipe->err == ST_OK) {
        pipe->err_info = c.err_info;
        pipe->err = c.err;
      }
      __threadfence_block();
      pipe->abort = 1;
    }
    __syncwarp();
  }
  pt_lap(pt, c, PH_TOTAL);
  store_ctx(c, cursor);
  if (pr) publish_progress(c, pr, cursor);
}

// Block b lowers unit b with its first warp. Blocks launched with more warps
// (kReserveThreads) park the others at the barrier: they hold most of the
// SM's registers, so no block of another kernel (the executor's copies and
// kernels running concurrently) shares the SM, its issue slots or its L1.
constexpr uint32_t kReserveThreads = 512;
__global__ void __launch_bounds__(kReserveThreads) lower_kernel(const Unit* units, uint32_t n_units, uint32_t max_items,
                                                               volatile uint32_t* progress) {
  __shared__ BlockShared sh;
  const uint32_t warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const uint32_t workers = nw < kMaxWorkers ? nw : kMaxWorkers;
  if (threadIdx.x == 0) {
    sh.lock = 0;
    sh.cmd = CMD_NONE;
    sh.err = ST_OK;
    sh.piped = 0;
    // a front warp when the block has one, the node has its scratch set and
    // the launch lowers several items
    if (nw > kFrontWarp && blockIdx.x < n_units) {
      const Unit u = units[blockIdx.x];
      const NodeDev* nd = u.node;
      if (nd->helper_scratch && nd->status == ST_OK) {
        const uint32_t cur = nd->cursor, avail = *u.prog->n_items;
        uint32_t end = avail;
        if (max_items != NONE && cur + max_items < end) end = cur + max_items;
        if (end > cur && end - cur >= kPipeMinItems) {
          sh.piped = 1;
          sh.pipe.begin = cur;
          sh.pipe.end = end;
          sh.pipe.front_done = cur;
          sh.pipe.back_done = cur;
          sh.pipe.abort = 0;
          sh.pipe.err = ST_OK;
          sh.pipe.err_info = 0;
        }
      }
    }
  }
  __syncthreads();
  if (warp == 0) {
    lower_unit(units, n_units, max_items, blockIdx.x, progress, workers > 1 ? &sh : nullptr, workers,
               sh.piped ? &sh.pipe : nullptr);
    if (workers > 1) {
      if ((threadIdx.x & 31u) == 0) {
        sh.cmd = CMD_EXIT;
        __threadfence_block();
      }
      __syncwarp();
      worker_bar(workers);  // the helpers leave their loop
    }
  } else if (warp < workers) {
    helper_loop(sh, warp, workers);
  } else if (warp == kFrontWarp && sh.piped) {
    front_loop(sh, units[blockIdx.x]);
  }
  __syncthreads();
}

// Batched lowering with a device work queue: the first warp of each
// persistent block takes the next unit (a node of one program) from *head, in
// the order `order` gives (longest estimated work first, say), until every
// unit is lowered. The block's other warps (if any) help with the shared
// phases of units whose node has helper scratch, and wait at the block
// barrier otherwise.
__global__ void __launch_bounds__(32 * kMaxWorkers) lower_queue_kernel(const Unit* units, uint32_t n_units,
                                                                      const uint32_t* order, uint32_t* head) {
  __shared__ BlockShared sh;
  const uint32_t warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const uint32_t workers = nw < kMaxWorkers ? nw : kMaxWorkers;
  if (threadIdx.x == 0) {
    sh.lock = 0;
    sh.cmd = CMD_NONE;
    sh.err = ST_OK;
  }
  __syncthreads();
  if (warp == 0) {
    for (;;) {
      uint32_t u = 0;
      __syncwarp();
      if ((threadIdx.x & 31u) == 0) u = atomicAdd(head, 1u);
      u = __shfl_sync(FULL, u, 0);
      if (u >= n_units) break;
      lower_unit(units, n_units, NONE, order ? order[u] : u, nullptr, workers > 1 ? &sh : nullptr, workers);
    }
    if (workers > 1) {
      if ((threadIdx.x & 31u) == 0) {
        sh.cmd = CMD_EXIT;
        __threadfence_block();
      }
      __syncwarp();
      worker_bar(workers);
    }
  } else if (warp < workers) {
    helper_loop(sh, warp, workers);
  }
  __syncthreads();
}

// Copies submissions [from, to) and their tasks from the host-mapped arrays
// into the program's device arrays (16-byte words, all lanes). Every node warp
// of a program stages the same records; the copies write equal bytes.
__device__ __noinline__ void stage_submissions(const ProgDev* pg, uint32_t from, uint32_t to) {
  // host-written records are read with cache-volatile loads (never from a
  // line cached before the host wrote it)
  static_assert(sizeof(Item) == 16, "an item is one 16-byte word");
  const uint4* src = reinterpret_cast<const uint4*>(pg->src_items);
  uint4* dst = reinterpret_cast<uint4*>(const_cast<Item*>(pg->items));
  const uint32_t lane = threadIdx.x & 31u;
  for (uint32_t i = from + lane; i < to; i += 32) dst[i] = __ldcv(src + i);
  __syncwarp();
  static_assert(sizeof(igs_task) % 4 == 0, "task record is a whole number of words");
  constexpr uint32_t words = sizeof(igs_task) / 4;
  for (uint32_t i = from; i < to; ++i) {
    const Item it = pg->items[i];
    if (it.kind != IT_TASK) continue;
    const uint32_t* s = reinterpret_cast<const uint32_t*>(pg->src_tasks + it.task);
    uint32_t* d = reinterpret_cast<uint32_t*>(const_cast<igs_task*>(pg->tasks + it.task));
    for (uint32_t w = lane; w < words; w += 32) d[w] = __ldcv(s + w);
  }
  __threadfence_block();
  __syncwarp();
}

// Serving loop: warp w serves slot w; it takes every submission published so
// far, then publishes its progress. Waits are bounded: after idle_polls empty
// polls (about 2 us each) the warp leaves with EXIT_IDLE; a set stop flag ends
// it with EXIT_STOPPED.
__global__ void __launch_bounds__(32) serve_kernel(ServeSlot* slots, uint32_t n_slots, volatile uint32_t* stop,
                                                    uint64_t idle_polls) {
  const uint32_t w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (w >= n_slots) return;
  ServeSlot& S = slots[w];
  uint64_t idle = 0;
  uint32_t exit_code = EXIT_IDLE;
  const bool leader = (threadIdx.x & 31u) == 0;
  for (;;) {
    // host-written words are read once by lane 0 and broadcast, so every lane
    // takes the same path
    uint32_t st = 0, stp = 0;
    if (leader) {
      st = S.state;
      stp = *stop;
    }
    st = __shfl_sync(FULL, st, 0);
    stp = __shfl_sync(FULL, stp, 0);
    if (stp) {
      exit_code = EXIT_STOPPED;
      break;
    }
    bool worked = false;
    if (st == SLOT_ACTIVE) {
      // mark the slot busy, then confirm it is still active: the host clears
      // the state first and then waits for busy == 0
      if (leader) S.busy = 1;
      __threadfence_system();
      uint32_t st2 = 0;
      if (leader) st2 = S.state;
      st2 = __shfl_sync(FULL, st2, 0);
      const Unit u = S.unit;
      uint32_t avail = 0;
      if (leader && st2 == SLOT_ACTIVE) avail = *u.prog->n_items;
      avail = __shfl_sync(FULL, avail, 0);
      __threadfence_system();
      if (st2 == SLOT_ACTIVE && u.node->cursor < avail && u.node->status == ST_OK) {
        uint32_t cursor = u.node->cursor;
        stage_submissions(u.prog, cursor, avail);
        Ctx c;
        load_ctx(c, u.node, u.prog);
        while (cursor < avail && c.err == ST_OK) {
          deliver(c, cursor);
          ++cursor;
        }
        store_ctx(c, cursor);
        __threadfence_system();
        if (leader) {
          S.status = c.err;
          S.done = cursor;
        }
        __threadfence_system();
        worked = true;
      }
      __threadfence_system();
      if (leader) S.busy = 0;
    }
    __syncwarp();
    if (worked) {
      idle = 0;
      continue;
    }
    if (++idle > idle_polls) break;
    __nanosleep(2000);
  }
  if (leader) S.exit = exit_code;
  __threadfence_system();
}

}  // namespace
}  // namespace igs

int igs_launch_serve(igs::ServeSlot* slots, uint32_t n_slots, volatile uint32_t* stop, uint64_t idle_polls, void* stream) {
  if (n_slots == 0) return 0;
  // one warp per block: each slot's warp gets an SM (and its L1) to itself
  // while there are fewer slots than SMs
  static bool carveout = false;
  if (!carveout) {
    cudaFuncSetAttribute(igs::serve_kernel, cudaFuncAttributePreferredSharedMemoryCarveout, 0);
    carveout = true;
  }
  igs::serve_kernel<<<n_slots, 32, 0, (cudaStream_t)stream>>>(slots, n_slots, stop, idle_polls);
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

int igs_launch_lower_queue(const igs::Unit* units_dev, uint32_t n_units, const uint32_t* order_dev, uint32_t* head_dev,
                           uint32_t blocks, uint32_t warps, void* stream) {
  if (warps < 1 || warps > igs::kMaxWorkers) return -1;
  if (n_units == 0) return 0;
  static bool carveout = false;
  if (!carveout) {
    cudaFuncSetAttribute(igs::lower_queue_kernel, cudaFuncAttributePreferredSharedMemoryCarveout, 0);
    carveout = true;
  }
  igs::lower_queue_kernel<<<blocks, 32 * warps, 0, (cudaStream_t)stream>>>(units_dev, n_units, order_dev, head_dev);
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

int igs_launch_lower(const igs::Unit* units_dev, uint32_t n_units, uint32_t max_items, void* stream, bool reserve,
                     volatile uint32_t* progress, bool workers) {
  if (n_units == 0) return 0;
  // one unit per block, so that units spread over the SMs (each node's
  // tables then share an L1 with as few other units as possible)
  static bool carveout = false;
  if (!carveout) {
    cudaFuncSetAttribute(igs::lower_kernel, cudaFuncAttributePreferredSharedMemoryCarveout, 0);
    carveout = true;
  }
  // with workers: kMaxWorkers warps plus the front warp of pipelined launches
  const uint32_t threads = reserve ? igs::kReserveThreads : (workers ? 32 * (igs::kMaxWorkers + 1) : 32);
  igs::lower_kernel<<<n_units, threads, 0, (cudaStream_t)stream>>>(units_dev, n_units, max_items, progress);
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}
