// Instruction-graph lowering oracle — TEST INFRASTRUCTURE ONLY.
//
// A plain, slow, single-threaded CPU restatement of the instruction-graph
// generator of "Concurrent Scheduling of High-Level Parallel Programs on
// Multi-GPU Systems" (Knorr et al.), used by the tests, by smoke() and by the
// bench's CPU-baseline leg to check the CUDA lowering engine. Nothing in the
// product library may link, import or call this file.
//
// Every region operation is recomputed from scratch on plain std::vector box
// lists; after every update a region map is re-normalised (entries grouped by
// value, each group put in canonical form). No incremental structure, no
// blocking, no reordering beyond what the rules below state.
//
// Paper passages followed (section / table / listing of the paper):
//   a1 chunk split + assignment ........ Sec. 3.1 (hierarchical work assignment)
//   a2 range mappers ................... Sec. 2.1, Listing 1; Listing 2
//   a3 node-level push / await push .... Sec. 2.4, Sec. 3.4 (first paragraphs)
//   a4 allocations + lookahead ......... Sec. 3.2, Fig. 4 caption; Sec. 4.3
//   a5 coherence copies ................ Sec. 3.3 (producer split x consumer split)
//   a6 outbound sends .................. Sec. 3.4 "Outbound Transfers"
//   a7 inbound receive / split / await . Sec. 3.4 "Inbound Transfers"
//   a8 dependencies, edge kinds ........ Fig. 5 legend; Sec. 3.6; Sec. 4.2
//   a9 horizons / epochs ............... Sec. 3.5; Sec. 2.4
//   debug checks ....................... Sec. 4.4 (uninitialized read, overlapping write)
// Where the paper is silent the rules take a fixed reading; each is marked
// [R<n>] and stated in words where it is applied.
//
// Parity status: pinned against a per-element brute-force generator, graph
// invariants, sequential execution and the paper's worked examples (tests/).
#include <algorithm>
#include <cstdint>
#include <cstring>
#include <deque>
#include <map>
#include <set>
#include <vector>

namespace orc {

constexpr uint32_t NONE = 0xFFFFFFFFu;
constexpr uint32_t REMOTE = 0xFFFFFFFEu;  // producer / owner sentinel
constexpr uint32_t HOST = 0xFFFFFFFEu;    // owner: user host memory, every node has it

enum Type : uint32_t {
  EPOCH = 0, HORIZON = 1, ALLOC = 2, FREE = 3, COPY = 4, SEND = 5,
  RECEIVE = 6, SPLIT_RECEIVE = 7, AWAIT_RECEIVE = 8, KERNEL = 9
};
enum Kind : uint32_t { K_DATAFLOW = 1, K_ANTI = 2, K_ALLOC = 4, K_EPOCH = 8, K_FRONT = 16 };
enum Mode : uint32_t { M_READ = 1, M_WRITE = 2 };

struct Box {
  uint32_t lo[3], hi[3];
};

static bool empty(const Box& b) {
  for (int d = 0; d < 3; ++d)
    if (b.lo[d] >= b.hi[d]) return true;
  return false;
}
static Box isect(const Box& a, const Box& b) {
  Box r;
  for (int d = 0; d < 3; ++d) {
    r.lo[d] = std::max(a.lo[d], b.lo[d]);
    r.hi[d] = std::min(a.hi[d], b.hi[d]);
  }
  return r;
}
static bool overlap(const Box& a, const Box& b) { return !empty(isect(a, b)); }
static bool contains(const Box& outer, const Box& inner) {
  for (int d = 0; d < 3; ++d)
    if (inner.lo[d] < outer.lo[d] || inner.hi[d] > outer.hi[d]) return false;
  return true;
}
static Box bbox2(const Box& a, const Box& b) {
  Box r;
  for (int d = 0; d < 3; ++d) {
    r.lo[d] = std::min(a.lo[d], b.lo[d]);
    r.hi[d] = std::max(a.hi[d], b.hi[d]);
  }
  return r;
}
static bool box_less(const Box& a, const Box& b) {
  for (int d = 0; d < 3; ++d)
    if (a.lo[d] != b.lo[d]) return a.lo[d] < b.lo[d];
  for (int d = 0; d < 3; ++d)
    if (a.hi[d] != b.hi[d]) return a.hi[d] < b.hi[d];
  return false;
}
static bool box_eq(const Box& a, const Box& b) {
  for (int d = 0; d < 3; ++d)
    if (a.lo[d] != b.lo[d] || a.hi[d] != b.hi[d]) return false;
  return true;
}

using Region = std::vector<Box>;  // pairwise disjoint boxes

// a \ b as at most six disjoint pieces.
static void box_minus(const Box& a, const Box& b, Region& out) {
  if (!overlap(a, b)) {
    out.push_back(a);
    return;
  }
  Box rem = a;
  for (int d = 0; d < 3; ++d) {
    if (rem.lo[d] < b.lo[d]) {
      Box p = rem;
      p.hi[d] = b.lo[d];
      out.push_back(p);
      rem.lo[d] = b.lo[d];
    }
    if (rem.hi[d] > b.hi[d]) {
      Box p = rem;
      p.lo[d] = b.hi[d];
      out.push_back(p);
      rem.hi[d] = b.hi[d];
    }
  }
}

static Region region_minus(const Region& a, const Region& b) {
  Region cur = a;
  for (const Box& r : b) {
    Region nxt;
    for (const Box& x : cur) box_minus(x, r, nxt);
    cur.swap(nxt);
  }
  return cur;
}
static Region region_isect(const Region& a, const Region& b) {
  Region out;
  for (const Box& x : a)
    for (const Box& y : b) {
      Box i = isect(x, y);
      if (!empty(i)) out.push_back(i);
    }
  return out;
}
static Region region_isect_box(const Region& a, const Box& b) {
  Region out;
  for (const Box& x : a) {
    Box i = isect(x, b);
    if (!empty(i)) out.push_back(i);
  }
  return out;
}

// Canonical form [R4]: row-major maximal decomposition. For every line along
// the fastest dimension take the maximal intervals; merge identical intervals
// over maximal runs of consecutive lines of the middle dimension; merge
// identical rectangles over maximal runs of the slowest dimension; sort
// lexicographically by (lo, hi). Computed plainly on the grid of elementary
// cells spanned by all box corners.
static Region canonical(const Region& in) {
  Region r;
  for (const Box& b : in)
    if (!empty(b)) r.push_back(b);
  if (r.size() <= 1) return r;
  std::vector<uint32_t> br[3];
  for (int d = 0; d < 3; ++d) {
    for (const Box& b : r) {
      br[d].push_back(b.lo[d]);
      br[d].push_back(b.hi[d]);
    }
    std::sort(br[d].begin(), br[d].end());
    br[d].erase(std::unique(br[d].begin(), br[d].end()), br[d].end());
  }
  const size_t n0 = br[0].size() - 1, n1 = br[1].size() - 1, n2 = br[2].size() - 1;
  std::vector<uint8_t> cell(n0 * n1 * n2, 0);
  for (size_t i = 0; i < n0; ++i)
    for (size_t j = 0; j < n1; ++j)
      for (size_t k = 0; k < n2; ++k) {
        const uint32_t p[3] = {br[0][i], br[1][j], br[2][k]};
        for (const Box& b : r) {
          bool in_b = true;
          for (int d = 0; d < 3; ++d)
            if (p[d] < b.lo[d] || p[d] >= b.hi[d]) in_b = false;
          if (in_b) {
            cell[(i * n1 + j) * n2 + k] = 1;
            break;
          }
        }
      }
  struct Run { size_t a, b; bool operator==(const Run& o) const { return a == o.a && b == o.b; } };
  struct Rect { size_t j0, j1, k0, k1; bool operator==(const Rect& o) const { return j0 == o.j0 && j1 == o.j1 && k0 == o.k0 && k1 == o.k1; } };
  auto runs_of = [&](size_t i, size_t j) {
    std::vector<Run> out;
    size_t k = 0;
    while (k < n2) {
      if (!cell[(i * n1 + j) * n2 + k]) { ++k; continue; }
      size_t s = k;
      while (k < n2 && cell[(i * n1 + j) * n2 + k]) ++k;
      out.push_back({s, k});
    }
    return out;
  };
  auto has = [](const std::vector<Run>& v, const Run& x) { return std::find(v.begin(), v.end(), x) != v.end(); };
  std::vector<std::vector<Rect>> rects(n0);
  for (size_t i = 0; i < n0; ++i) {
    std::vector<std::vector<Run>> rows(n1);
    for (size_t j = 0; j < n1; ++j) rows[j] = runs_of(i, j);
    for (size_t j = 0; j < n1; ++j)
      for (const Run& x : rows[j]) {
        if (j > 0 && has(rows[j - 1], x)) continue;  // continues a run started above
        size_t e = j;
        while (e + 1 < n1 && has(rows[e + 1], x)) ++e;
        rects[i].push_back({j, e + 1, x.a, x.b});
      }
  }
  auto hasr = [](const std::vector<Rect>& v, const Rect& x) { return std::find(v.begin(), v.end(), x) != v.end(); };
  Region out;
  for (size_t i = 0; i < n0; ++i)
    for (const Rect& x : rects[i]) {
      if (i > 0 && hasr(rects[i - 1], x)) continue;
      size_t e = i;
      while (e + 1 < n0 && hasr(rects[e + 1], x)) ++e;
      Box b;
      b.lo[0] = br[0][i]; b.hi[0] = br[0][e + 1];
      b.lo[1] = br[1][x.j0]; b.hi[1] = br[1][x.j1];
      b.lo[2] = br[2][x.k0]; b.hi[2] = br[2][x.k1];
      out.push_back(b);
    }
  std::sort(out.begin(), out.end(), box_less);
  return out;
}

static Box bbox_of(const Region& r) {
  Box b = r[0];
  for (const Box& x : r) b = bbox2(b, x);
  return b;
}

// A total region map over a domain box: (box, value) entries, pairwise
// disjoint, covering the domain. Re-normalised after every update.
template <class V>
struct RMap {
  std::vector<std::pair<Box, V>> e;

  void init(const Box& dom, const V& v) { e.assign(1, {dom, v}); }

  std::vector<std::pair<Box, V>> query(const Box& q) const {
    std::vector<std::pair<Box, V>> out;
    for (const auto& x : e) {
      Box i = isect(x.first, q);
      if (!empty(i)) out.push_back({i, x.second});
    }
    return out;
  }
  std::vector<std::pair<Box, V>> query(const Region& q) const {
    std::vector<std::pair<Box, V>> out;
    for (const Box& b : q) {
      auto part = query(b);
      out.insert(out.end(), part.begin(), part.end());
    }
    return out;
  }

  // value := f(value) on every point of R.
  template <class F>
  void update(const Region& R, F f) {
    if (R.empty()) return;
    std::vector<std::pair<Box, V>> nxt;
    for (const auto& x : e) {
      Region outside = region_minus({x.first}, R);
      for (const Box& b : outside) nxt.push_back({b, x.second});
      for (const Box& r : R) {
        Box i = isect(x.first, r);
        if (!empty(i)) nxt.push_back({i, f(x.second)});
      }
    }
    e.swap(nxt);
    normalize();
  }
  template <class F>
  void map_values(F f) {
    for (auto& x : e) x.second = f(x.second);
    normalize();
  }
  void normalize() {
    std::vector<V> vals;
    for (const auto& x : e)
      if (std::find(vals.begin(), vals.end(), x.second) == vals.end()) vals.push_back(x.second);
    std::vector<std::pair<Box, V>> nxt;
    for (const V& v : vals) {
      Region g;
      for (const auto& x : e)
        if (x.second == v) g.push_back(x.first);
      for (const Box& b : canonical(g)) nxt.push_back({b, v});
    }
    e.swap(nxt);
  }
};

// ---- program description ---------------------------------------------------

struct MapDim { uint32_t kind, a, b, c; };  // kind 0 = affine(k, offset, radius), 1 = all, 2 = fixed[lo,hi)
struct Acc { uint32_t buffer, mode; MapDim m[3]; };
struct TaskDesc {
  uint32_t dims, range[3], chunks, kernel, nacc, params[4];
  Acc acc[8];
};
struct BufDesc { uint32_t dims, extent[3], elem; bool init; bool live; };

struct BState {  // per-buffer local state: original producer, its memory, up-to-date memories
  uint32_t prod, pmem, mask;
  bool operator==(const BState& o) const { return prod == o.prod && pmem == o.pmem && mask == o.mask; }
};
struct Own {  // node-level: last writer node, nodes holding the newest version
  uint32_t owner, repl;
  bool operator==(const Own& o) const { return owner == o.owner && repl == o.repl; }
};

struct Chunk { uint32_t index, node, mem; Box box; };

// Per-node view of one task, fixed when the task is submitted.
struct NodeTask {
  uint32_t seq;
  const TaskDesc* t;
  std::vector<Chunk> chunks;               // chunks on this node
  std::vector<std::vector<Box>> mapped;    // [local chunk][acc] mapped box (maybe empty)
  std::vector<std::pair<Chunk, std::vector<Box>>> remote;  // chunks of other nodes + mapped boxes
  std::map<std::pair<uint32_t, uint32_t>, Region> push;    // (buffer, target) -> region
  std::map<uint32_t, Region> await_;                       // buffer -> region
};

enum ItemKind { I_CREATE, I_TASK, I_HORIZON, I_EPOCH, I_DESTROY, I_LOOKAHEAD };
struct Item {
  ItemKind kind;
  uint32_t seq, arg;
  NodeTask nt;
};

struct Alloc {
  uint32_t id, buffer, mem;
  Box box;
  bool live, user;
  RMap<uint32_t> writers;
  RMap<std::vector<uint32_t>> readers;
};

struct Instr { uint32_t id, type, seq, a, b, c, d, box_off, box_cnt, bind_off, bind_cnt; };
struct Edge { uint32_t from, to, kind; };
struct Bind { uint32_t alloc; Box box; };
struct Diag { uint32_t seq, chunk, acc; };

struct Access { uint32_t alloc; Region r; uint32_t mode; };

struct Node {
  uint32_t id;
  std::vector<Instr> instrs;
  std::vector<Edge> edges;
  std::vector<Box> boxes;
  std::vector<Bind> binds;
  std::vector<Diag> diags;
  std::vector<Alloc> allocs;                 // index = alloc id
  std::map<uint32_t, RMap<BState>> bstate;   // buffer -> map
  std::set<uint32_t> front;
  uint32_t epoch = 0, last_horizon = NONE, next_msg = 0;
  uint32_t lookahead = 0;
  std::deque<Item> queue;
  uint32_t horizons_after_alloc = 0;  // horizon-count heuristic: horizons queued since the last allocating task
  bool stage_d2d = false;             // device-to-device copies staged in host memory [R27]
};

struct Ctx {
  uint32_t N, D, hstep;
  // critical-path horizon cadence [R29]: per buffer the boxes each task last
  // wrote and the boxes tasks read since; per task its depth in the task graph
  bool horizon_cp = false;
  std::map<uint32_t, std::vector<std::pair<Box, uint32_t>>> t_writers, t_readers;
  std::vector<uint32_t> depth;
  uint32_t cpl = 0, cpl_at_horizon = 0;
  std::vector<BufDesc> bufs;
  std::map<uint32_t, RMap<Own>> own;  // buffer -> node-level map
  std::vector<Node> nodes;
  std::deque<TaskDesc> tasks;         // stable addresses
  std::vector<uint32_t> rejected;     // seq of rejected tasks
  uint32_t seq = 0, ntasks = 0;
};

static Box buffer_box(const BufDesc& b) {
  Box x;
  for (int d = 0; d < 3; ++d) { x.lo[d] = 0; x.hi[d] = d < (int)b.dims ? b.extent[d] : 1; }
  return x;
}

// a2: range-mapper evaluation of one accessor for one chunk box, clamped [R3].
static Box map_box(const Acc& a, const Box& chunk, const BufDesc& buf) {
  Box r;
  for (int d = 0; d < 3; ++d) {
    const uint32_t ext = d < (int)buf.dims ? buf.extent[d] : 1;
    int64_t lo, hi;
    const MapDim& m = a.m[d];
    if (d >= (int)buf.dims) { lo = 0; hi = 1; }
    else if (m.kind == 1) { lo = 0; hi = ext; }
    else if (m.kind == 2) { lo = m.a; hi = m.b; }
    else {
      const uint32_t k = m.a;
      const int64_t off = (int32_t)m.b, rad = m.c;
      lo = (int64_t)chunk.lo[k] + off - rad;
      hi = (int64_t)chunk.hi[k] + off + rad;
    }
    lo = std::max<int64_t>(lo, 0);
    hi = std::min<int64_t>(hi, ext);
    if (lo >= hi) { lo = 0; hi = 0; }
    r.lo[d] = (uint32_t)lo;
    r.hi[d] = (uint32_t)hi;
  }
  return r;
}

// a1 with a split along dims 0 and 1 [R28] (Sec. 3.1: the node split, then
// the same scheme again among a node's devices): a Cy x Cx grid of chunks,
// chunk (iy, ix) = rows [floor(iy*E0/Cy), floor((iy+1)*E0/Cy)) x columns
// [floor(ix*E1/Cx), floor((ix+1)*E1/Cx)), index iy*Cx + ix. Grid row iy goes
// to node floor(iy*N/Cy); a node's K chunks, numbered j in row-major order,
// go to its device floor(j*D/K). Empty chunks are dropped after assignment.
static std::vector<Chunk> split_2d(const Ctx& c, const TaskDesc& t, uint64_t Cy, uint64_t Cx) {
  std::vector<Chunk> out;
  const uint64_t E0 = t.range[0], E1 = t.range[1], N = c.N, D = c.D;
  auto first_row = [&](uint64_t n) { return (n * Cy + N - 1) / N; };  // smallest iy with floor(iy*N/Cy) >= n
  for (uint64_t iy = 0; iy < Cy; ++iy) {
    const uint64_t node = iy * N / Cy;
    const uint64_t r0n = first_row(node), K = (first_row(node + 1) - r0n) * Cx;
    for (uint64_t ix = 0; ix < Cx; ++ix) {
      const uint64_t j = (iy - r0n) * Cx + ix;
      const uint32_t y0 = (uint32_t)(iy * E0 / Cy), y1 = (uint32_t)((iy + 1) * E0 / Cy);
      const uint32_t x0 = (uint32_t)(ix * E1 / Cx), x1 = (uint32_t)((ix + 1) * E1 / Cx);
      if (y0 >= y1 || x0 >= x1) continue;
      Chunk ch;
      ch.index = (uint32_t)(iy * Cx + ix);
      ch.node = (uint32_t)node;
      ch.mem = 2 + (uint32_t)(j * D / K);
      ch.box.lo[0] = y0; ch.box.hi[0] = y1;
      ch.box.lo[1] = x0; ch.box.hi[1] = x1;
      ch.box.lo[2] = 0; ch.box.hi[2] = t.range[2];
      out.push_back(ch);
    }
  }
  return out;
}

// a1: split along dim 0 into C chunks, drop empty ones, assign chunk c to the
// global device floor(c*M/C) [R1, R2]; num_chunks' high 16 bits, if set, give
// a split along dim 1 too (split_2d).
static std::vector<Chunk> split(const Ctx& c, const TaskDesc& t) {
  if (t.chunks >> 16) return split_2d(c, t, t.chunks & 0xFFFFu, t.chunks >> 16);
  std::vector<Chunk> out;
  const uint64_t E0 = t.range[0], C = t.chunks, M = (uint64_t)c.N * c.D;
  for (uint64_t i = 0; i < C; ++i) {
    const uint32_t r0 = (uint32_t)(i * E0 / C), r1 = (uint32_t)((i + 1) * E0 / C);
    if (r0 >= r1) continue;
    Chunk ch;
    ch.index = (uint32_t)i;
    const uint32_t g = (uint32_t)(i * M / C);
    ch.node = g / c.D;
    ch.mem = 2 + g % c.D;
    ch.box.lo[0] = r0; ch.box.hi[0] = r1;
    for (int d = 1; d < 3; ++d) { ch.box.lo[d] = 0; ch.box.hi[d] = t.range[d]; }
    out.push_back(ch);
  }
  return out;
}

// ---- emission with dependency tracking (a8) -------------------------------

static uint32_t push_boxes(Node& n, const Region& r) {
  const uint32_t off = (uint32_t)n.boxes.size();
  n.boxes.insert(n.boxes.end(), r.begin(), r.end());
  return off;
}

static std::vector<uint32_t> add_reader(const std::vector<uint32_t>& s, uint32_t id) {
  std::vector<uint32_t> r = s;
  if (std::find(r.begin(), r.end(), id) == r.end()) r.push_back(id);
  std::sort(r.begin(), r.end());
  return r;
}

// Emits one instruction: its dependencies come from the per-allocation
// last-writer and reader maps of every access (RAW -> dataflow, WAR/WAW ->
// anti, first use of an allocation -> allocation lifetime), plus explicit
// extra edges; an instruction without any predecessor depends on the last
// epoch [R15]. Then the accesses are applied: reads first, then writes.
static uint32_t emit(Node& n, Instr rec, const Region& boxes, const std::vector<Access>& acc,
                     const std::map<uint32_t, uint32_t>& extra, const std::vector<Bind>* binds = nullptr) {
  const uint32_t id = (uint32_t)n.instrs.size();
  std::map<uint32_t, uint32_t> deps = extra;
  for (const Access& a : acc) {
    const Alloc& al = n.allocs[a.alloc];
    if (a.mode & M_READ)
      for (const auto& w : al.writers.query(a.r))
        deps[w.second] |= n.instrs[w.second].type == ALLOC ? K_ALLOC : K_DATAFLOW;
    if (a.mode & M_WRITE) {
      for (const auto& w : al.writers.query(a.r))
        deps[w.second] |= n.instrs[w.second].type == ALLOC ? K_ALLOC : K_ANTI;
      for (const auto& rd : al.readers.query(a.r))
        for (uint32_t x : rd.second) deps[x] |= K_ANTI;
    }
  }
  if (deps.empty()) deps[n.epoch] = K_EPOCH;
  for (const auto& d : deps) {
    n.edges.push_back({d.first, id, d.second});
    n.front.erase(d.first);
  }
  n.front.insert(id);
  rec.id = id;
  rec.box_off = push_boxes(n, boxes);
  rec.box_cnt = (uint32_t)boxes.size();
  rec.bind_off = (uint32_t)n.binds.size();
  rec.bind_cnt = 0;
  if (binds) {
    n.binds.insert(n.binds.end(), binds->begin(), binds->end());
    rec.bind_cnt = (uint32_t)binds->size();
  }
  n.instrs.push_back(rec);
  for (const Access& a : acc)
    if (a.mode & M_READ)
      n.allocs[a.alloc].readers.update(a.r, [id](const std::vector<uint32_t>& s) { return add_reader(s, id); });
  for (const Access& a : acc)
    if (a.mode & M_WRITE) {
      n.allocs[a.alloc].writers.update(a.r, [id](uint32_t) { return id; });
      n.allocs[a.alloc].readers.update(a.r, [](const std::vector<uint32_t>&) { return std::vector<uint32_t>(); });
    }
  return id;
}

static Instr rec0(uint32_t type, uint32_t seq) { return Instr{0, type, seq, NONE, NONE, NONE, NONE, 0, 0, 0, 0}; }

// The single live allocation of (buffer, memory) that contains box, or NONE.
static uint32_t find_alloc(const Node& n, uint32_t buf, uint32_t mem, const Box& b) {
  for (const Alloc& a : n.allocs)
    if (a.live && a.buffer == buf && a.mem == mem && contains(a.box, b)) return a.id;
  return NONE;
}

// Replace every tracked instruction id older than h by h and re-merge (a9).
static void apply_epoch(Node& n, uint32_t h) {
  auto f = [h](uint32_t v) { return v < h ? h : v; };
  for (Alloc& a : n.allocs) {
    if (!a.live) continue;
    a.writers.map_values(f);
    a.readers.map_values([h](const std::vector<uint32_t>& s) {
      std::vector<uint32_t> r;
      for (uint32_t x : s) r.push_back(x < h ? h : x);
      std::sort(r.begin(), r.end());
      r.erase(std::unique(r.begin(), r.end()), r.end());
      return r;
    });
  }
  for (auto& b : n.bstate)
    b.second.map_values([h](const BState& s) {
      BState r = s;
      if (r.prod != NONE && r.prod != REMOTE && r.prod < h) r.prod = h;
      return r;
    });
  n.epoch = h;
}

// ---- requirements and allocation planning (a4) ----------------------------

struct Req { uint32_t buffer, mem; Box box; };

static std::vector<Req> requirements(const NodeTask& nt) {
  std::vector<Req> out;
  for (size_t i = 0; i < nt.chunks.size(); ++i)
    for (uint32_t a = 0; a < nt.t->nacc; ++a)
      if (!empty(nt.mapped[i][a])) out.push_back({nt.t->acc[a].buffer, nt.chunks[i].mem, nt.mapped[i][a]});
  for (const auto& p : nt.push) out.push_back({p.first.first, 1, bbox_of(p.second)});
  for (const auto& w : nt.await_) out.push_back({w.first, 1, bbox_of(w.second)});
  return out;
}

static bool allocating(const Node& n, const NodeTask& nt) {
  for (const Req& r : requirements(nt))
    if (find_alloc(n, r.buffer, r.mem, r.box) == NONE) return true;
  return false;
}

// [R24] With the queue non-empty (horizon-count heuristic), a task is
// allocating when one of its requirement boxes lies neither inside a live
// allocation nor inside a requirement box of a queued task of the same
// (buffer, memory): compiling the queue would not make room for it.
static bool allocating_queued(const Node& n, const NodeTask& nt) {
  for (const Req& r : requirements(nt)) {
    if (find_alloc(n, r.buffer, r.mem, r.box) != NONE) continue;
    bool covered = false;
    for (const Item& q : n.queue) {
      if (q.kind != I_TASK) continue;
      for (const Req& x : requirements(q.nt))
        if (x.buffer == r.buffer && x.mem == r.mem && contains(x.box, r.box)) covered = true;
    }
    if (!covered) return true;
  }
  return false;
}

static void resize_and_alloc(Node& n, const Item& it, const std::vector<const NodeTask*>& look) {
  const NodeTask& nt = it.nt;
  std::vector<Req> reqs = requirements(nt);
  std::set<std::pair<uint32_t, uint32_t>> keys;
  for (const Req& r : reqs) keys.insert({r.buffer, r.mem});
  for (const auto& key : keys) {
    const uint32_t b = key.first, m = key.second;
    struct Cl { Box bb; bool own; std::vector<uint32_t> absorbed; };
    std::vector<Cl> cl;
    for (const Req& r : reqs)
      if (r.buffer == b && r.mem == m && find_alloc(n, b, m, r.box) == NONE) cl.push_back({r.box, true, {}});
    if (cl.empty()) continue;
    for (const NodeTask* q : look)
      for (const Req& r : requirements(*q))
        if (r.buffer == b && r.mem == m && find_alloc(n, b, m, r.box) == NONE) cl.push_back({r.box, false, {}});
    // Fixed point of merging clusters whose bounding boxes overlap with
    // positive volume, absorbing every overlapping live allocation [R5].
    bool changed = true;
    while (changed) {
      changed = false;
      for (size_t i = 0; i < cl.size() && !changed; ++i)
        for (size_t j = i + 1; j < cl.size() && !changed; ++j)
          if (overlap(cl[i].bb, cl[j].bb)) {
            cl[i].bb = bbox2(cl[i].bb, cl[j].bb);
            cl[i].own = cl[i].own || cl[j].own;
            cl[i].absorbed.insert(cl[i].absorbed.end(), cl[j].absorbed.begin(), cl[j].absorbed.end());
            cl.erase(cl.begin() + j);
            changed = true;
          }
      for (size_t i = 0; i < cl.size() && !changed; ++i)
        for (const Alloc& a : n.allocs) {
          if (!a.live || a.buffer != b || a.mem != m) continue;
          bool taken = false;
          for (const Cl& c : cl)
            if (std::find(c.absorbed.begin(), c.absorbed.end(), a.id) != c.absorbed.end()) taken = true;
          if (!taken && overlap(cl[i].bb, a.box)) {
            cl[i].bb = bbox2(cl[i].bb, a.box);
            cl[i].absorbed.push_back(a.id);
            changed = true;
            break;
          }
        }
    }
    std::vector<Cl> mine;
    for (const Cl& c : cl)
      if (c.own) mine.push_back(c);
    std::sort(mine.begin(), mine.end(), [](const Cl& x, const Cl& y) { return box_less(x.bb, y.bb); });
    for (Cl& c : mine) {
      const uint32_t aid = (uint32_t)n.allocs.size();
      Instr r = rec0(ALLOC, it.seq);
      r.a = aid; r.b = m; r.c = b;
      const uint32_t iid = emit(n, r, {c.bb}, {}, {});
      Alloc al;
      al.id = aid; al.buffer = b; al.mem = m; al.box = c.bb; al.live = true; al.user = false;
      al.writers.init(c.bb, iid);
      al.readers.init(c.bb, {});
      n.allocs.push_back(al);
      std::sort(c.absorbed.begin(), c.absorbed.end());
      for (uint32_t old : c.absorbed) {
        // Resize: copy the part of the old allocation that is up to date in
        // this memory, then free it [R6].
        Region live;
        for (const auto& s : n.bstate[b].query(n.allocs[old].box))
          if (s.second.mask >> m & 1u) live.push_back(s.first);
        live = canonical(live);
        if (!live.empty()) {
          Instr cp = rec0(COPY, it.seq);
          cp.a = old; cp.b = aid; cp.c = b; cp.d = 1;
          emit(n, cp, live, {{old, live, M_READ}, {aid, live, M_WRITE}}, {});
        }
        Instr fr = rec0(FREE, it.seq);
        fr.a = old; fr.b = m; fr.c = b;
        std::map<uint32_t, uint32_t> fd;
        for (const auto& w : n.allocs[old].writers.e) fd[w.second] |= K_ALLOC;
        for (const auto& rd : n.allocs[old].readers.e)
          for (uint32_t x : rd.second) fd[x] |= K_ALLOC;
        emit(n, fr, {}, {}, fd);
        n.allocs[old].live = false;
      }
    }
  }
}

// A copy of `part` from allocation src to allocation dst; with host staging
// of device-to-device copies [R27] (Sec. 3.3, last paragraph), a copy between
// two device memories becomes: a fresh allocation in the node's host memory M1
// over the bounding box of the region, a copy into it, a copy out of it, and
// its free.
static void emit_copy(Node& n, uint32_t seq, uint32_t b, uint32_t src, uint32_t dst, const Region& part) {
  const uint32_t sm = n.allocs[src].mem, dm = n.allocs[dst].mem;
  if (!(n.stage_d2d && sm >= 2 && dm >= 2)) {
    Instr cp = rec0(COPY, seq);
    cp.a = src; cp.b = dst; cp.c = b; cp.d = 0;
    emit(n, cp, part, {{src, part, M_READ}, {dst, part, M_WRITE}}, {});
    return;
  }
  Box bb = part[0];
  for (const Box& x : part) bb = bbox2(bb, x);
  const uint32_t hid = (uint32_t)n.allocs.size();
  Instr al = rec0(ALLOC, seq);
  al.a = hid; al.b = 1; al.c = b;
  const uint32_t iid = emit(n, al, {bb}, {}, {});
  Alloc h;
  h.id = hid; h.buffer = b; h.mem = 1; h.box = bb; h.live = true; h.user = false;
  h.writers.init(bb, iid);
  h.readers.init(bb, {});
  n.allocs.push_back(h);
  Instr in = rec0(COPY, seq);
  in.a = src; in.b = hid; in.c = b; in.d = 0;
  emit(n, in, part, {{src, part, M_READ}, {hid, part, M_WRITE}}, {});
  Instr out = rec0(COPY, seq);
  out.a = hid; out.b = dst; out.c = b; out.d = 0;
  emit(n, out, part, {{hid, part, M_READ}, {dst, part, M_WRITE}}, {});
  Instr fr = rec0(FREE, seq);
  fr.a = hid; fr.b = 1; fr.c = b;
  std::map<uint32_t, uint32_t> fd;
  for (const auto& w : n.allocs[hid].writers.e) fd[w.second] |= K_ALLOC;
  for (const auto& rd : n.allocs[hid].readers.e)
    for (uint32_t x : rd.second) fd[x] |= K_ALLOC;
  emit(n, fr, {}, {}, fd);
  n.allocs[hid].live = false;
}

// Coherence copies of `need` into allocation dst (memory m), split by
// original producer, then by source allocation [R7, R8].
static void coherence(Node& n, uint32_t seq, uint32_t b, uint32_t m, uint32_t dst, const Region& need) {
  std::vector<std::pair<Box, BState>> stale;
  for (const auto& s : n.bstate[b].query(need))
    if (!(s.second.mask >> m & 1u) && s.second.prod != NONE) stale.push_back(s);
  std::vector<std::pair<uint32_t, uint32_t>> producers;
  for (const auto& s : stale) producers.push_back({s.second.prod, s.second.pmem});
  std::sort(producers.begin(), producers.end());
  producers.erase(std::unique(producers.begin(), producers.end()), producers.end());
  Region copied;
  for (const auto& p : producers) {
    Region g;
    for (const auto& s : stale)
      if (s.second.prod == p.first && s.second.pmem == p.second) g.push_back(s.first);
    const size_t n_alloc = n.allocs.size();  // staging allocations are appended below
    for (size_t ai = 0; ai < n_alloc; ++ai) {   // ascending allocation id
      const Alloc src = n.allocs[ai];
      if (!src.live || src.buffer != b || src.mem != p.second) continue;
      Region part = canonical(region_isect_box(g, src.box));
      if (part.empty()) continue;
      emit_copy(n, seq, b, src.id, dst, part);
      copied.insert(copied.end(), part.begin(), part.end());
    }
  }
  n.bstate[b].update(copied, [m](const BState& s) { BState r = s; r.mask |= 1u << m; return r; });
}

static void compile_task(Ctx& c, Node& n, const Item& it, const std::vector<const NodeTask*>& look) {
  const NodeTask& nt = it.nt;
  const TaskDesc& t = *nt.t;
  // P1: allocations and resizes.
  resize_and_alloc(n, it, look);
  // P2: pushes — coherence copy into staging memory M1, then one send per
  // (original producer, canonical box).
  for (const auto& p : nt.push) {
    const uint32_t b = p.first.first, target = p.first.second;
    const Region& P = p.second;
    const uint32_t dst = find_alloc(n, b, 1, bbox_of(P));
    coherence(n, it.seq, b, 1, dst, P);
    auto parts = n.bstate[b].query(P);
    std::vector<std::pair<uint32_t, uint32_t>> producers;
    for (const auto& s : parts) producers.push_back({s.second.prod, s.second.pmem});
    std::sort(producers.begin(), producers.end());
    producers.erase(std::unique(producers.begin(), producers.end()), producers.end());
    for (const auto& pr : producers) {
      Region g;
      for (const auto& s : parts)
        if (s.second.prod == pr.first && s.second.pmem == pr.second) g.push_back(s.first);
      for (const Box& bx : canonical(g)) {
        Instr s = rec0(SEND, it.seq);
        s.a = dst; s.b = target; s.c = b; s.d = n.next_msg++;
        emit(n, s, {bx}, {{dst, {bx}, M_READ}}, {});
      }
    }
  }
  // P3: await push — one receive, or a split receive plus one await receive
  // per consumer (disjoint remainders in consumer order) [R10].
  for (const auto& w : nt.await_) {
    const uint32_t b = w.first;
    const Region& W = w.second;
    const uint32_t dst = find_alloc(n, b, 1, bbox_of(W));
    std::vector<Region> cons;
    for (size_t i = 0; i < nt.chunks.size(); ++i)
      for (uint32_t a = 0; a < t.nacc; ++a) {
        if (t.acc[a].buffer != b || !(t.acc[a].mode & M_READ) || empty(nt.mapped[i][a])) continue;
        Region r = canonical(region_isect_box(W, nt.mapped[i][a]));
        if (!r.empty()) cons.push_back(r);
      }
    bool whole = cons.size() <= 1;
    if (!whole) {
      whole = true;
      for (const Region& r : cons)
        if (!region_minus(W, r).empty()) whole = false;
    }
    if (whole) {
      Instr r = rec0(RECEIVE, it.seq);
      r.a = dst; r.c = b;
      const uint32_t id = emit(n, r, W, {{dst, W, M_WRITE}}, {});
      n.bstate[b].update(W, [id](const BState&) { return BState{id, 1, 1u << 1}; });
    } else {
      Instr r = rec0(SPLIT_RECEIVE, it.seq);
      r.a = dst; r.c = b;
      const uint32_t sid = emit(n, r, W, {{dst, W, M_WRITE}}, {});
      Region covered;
      for (const Region& cr : cons) {
        Region part = canonical(region_minus(cr, covered));
        if (part.empty()) continue;
        Instr aw = rec0(AWAIT_RECEIVE, it.seq);
        aw.a = dst; aw.b = sid; aw.c = b;
        const uint32_t aid = emit(n, aw, part, {}, {{sid, K_DATAFLOW}});
        n.allocs[dst].writers.update(part, [aid](uint32_t) { return aid; });
        n.bstate[b].update(part, [aid](const BState&) { return BState{aid, 1, 1u << 1}; });
        covered.insert(covered.end(), part.begin(), part.end());
      }
    }
  }
  // P4: coherence copies for every reading accessor, consumer split in
  // (chunk, accessor) order [R9]; uninitialized reads are warnings [R18].
  for (size_t i = 0; i < nt.chunks.size(); ++i)
    for (uint32_t a = 0; a < t.nacc; ++a) {
      const Acc& ac = t.acc[a];
      const Box& bx = nt.mapped[i][a];
      if (!(ac.mode & M_READ) || empty(bx)) continue;
      bool uninit = false;
      for (const auto& s : n.bstate[ac.buffer].query(bx))
        if (s.second.prod == NONE) uninit = true;
      if (uninit) n.diags.push_back({it.seq, nt.chunks[i].index, a});
      const uint32_t dst = find_alloc(n, ac.buffer, nt.chunks[i].mem, bx);
      coherence(n, it.seq, ac.buffer, nt.chunks[i].mem, dst, {bx});
    }
  // P5: one device kernel per chunk.
  for (size_t i = 0; i < nt.chunks.size(); ++i) {
    const Chunk& ch = nt.chunks[i];
    std::vector<Access> acc;
    std::vector<Bind> binds;
    for (uint32_t a = 0; a < t.nacc; ++a) {
      const Box& bx = nt.mapped[i][a];
      if (empty(bx)) {
        Box z{};
        binds.push_back({NONE, z});
        continue;
      }
      const uint32_t al = find_alloc(n, t.acc[a].buffer, ch.mem, bx);
      binds.push_back({al, bx});
      acc.push_back({al, {bx}, t.acc[a].mode});
    }
    Instr k = rec0(KERNEL, it.seq);
    k.a = ch.index; k.b = ch.mem; k.c = t.kernel;
    const uint32_t kid = emit(n, k, {ch.box}, acc, {}, &binds);
    for (uint32_t a = 0; a < t.nacc; ++a) {
      const Box& bx = nt.mapped[i][a];
      if (!(t.acc[a].mode & M_WRITE) || empty(bx)) continue;
      const uint32_t mem = ch.mem;
      n.bstate[t.acc[a].buffer].update({bx}, [kid, mem](const BState&) { return BState{kid, mem, 1u << mem}; });
    }
  }
  // Writes of other nodes make the local copies stale.
  for (const auto& rc : nt.remote)
    for (uint32_t a = 0; a < t.nacc; ++a) {
      const Box& bx = rc.second[a];
      if (!(t.acc[a].mode & M_WRITE) || empty(bx)) continue;
      n.bstate[t.acc[a].buffer].update({bx}, [](const BState&) { return BState{REMOTE, 0, 0}; });
    }
  (void)c;
}

static void process(Ctx& c, Node& n, const Item& it, const std::vector<const NodeTask*>& look) {
  switch (it.kind) {
    case I_CREATE: {
      const BufDesc& bd = c.bufs[it.arg];
      const Box dom = buffer_box(bd);
      RMap<BState> st;
      if (bd.init) {
        Alloc al;
        al.id = (uint32_t)n.allocs.size(); al.buffer = it.arg; al.mem = 0; al.box = dom;
        al.live = true; al.user = true;
        al.writers.init(dom, n.epoch);
        al.readers.init(dom, {});
        n.allocs.push_back(al);
        st.init(dom, BState{n.epoch, 0, 1u});
      } else {
        st.init(dom, BState{NONE, 0, 0});
      }
      n.bstate[it.arg] = st;
      break;
    }
    case I_TASK: compile_task(c, n, it, look); break;
    case I_HORIZON:
    case I_EPOCH: {
      std::map<uint32_t, uint32_t> fd;
      for (uint32_t f : n.front) fd[f] = K_FRONT;
      const uint32_t id = emit(n, rec0(it.kind == I_EPOCH ? EPOCH : HORIZON, it.seq), {}, {}, fd);
      n.front.clear();
      n.front.insert(id);
      if (it.kind == I_EPOCH) {
        apply_epoch(n, id);
        n.last_horizon = NONE;
      } else {
        if (n.last_horizon != NONE) apply_epoch(n, n.last_horizon);
        n.last_horizon = id;
      }
      break;
    }
    case I_DESTROY: {
      std::vector<uint32_t> ids;
      for (const Alloc& a : n.allocs)
        if (a.live && a.buffer == it.arg) ids.push_back(a.id);
      std::sort(ids.begin(), ids.end(), [&](uint32_t x, uint32_t y) {
        if (n.allocs[x].mem != n.allocs[y].mem) return n.allocs[x].mem < n.allocs[y].mem;
        return x < y;
      });
      for (uint32_t id : ids) {
        Alloc& a = n.allocs[id];
        if (!a.user) {
          Instr fr = rec0(FREE, it.seq);
          fr.a = id; fr.b = a.mem; fr.c = a.buffer;
          std::map<uint32_t, uint32_t> fd;
          for (const auto& w : a.writers.e) fd[w.second] |= K_ALLOC;
          for (const auto& rd : a.readers.e)
            for (uint32_t x : rd.second) fd[x] |= K_ALLOC;
          emit(n, fr, {}, {}, fd);
        }
        n.allocs[id].live = false;
      }
      n.bstate.erase(it.arg);
      break;
    }
    case I_LOOKAHEAD: break;
  }
}

static uint32_t queued_tasks(const Node& n) {
  uint32_t k = 0;
  for (const Item& x : n.queue)
    if (x.kind == I_TASK) ++k;
  return k;
}

static void flush_queue(Ctx& c, Node& n) {
  while (!n.queue.empty()) {
    Item it = n.queue.front();
    n.queue.pop_front();
    std::vector<const NodeTask*> look;
    for (const Item& q : n.queue)
      if (q.kind == I_TASK) look.push_back(&q.nt);
    process(c, n, it, look);
  }
}

// Scheduler lookahead [R17]: a task is queued while any queued task is
// allocating; the queue is compiled once it holds more than L tasks, or on an
// epoch or a buffer destruction.
// The horizon-count heuristic (Sec. 4.3 "Lookahead Heuristic") [R24], L =
// LOOKAHEAD_HORIZONS: the queue is compiled once two horizons have been
// queued after the last allocating task (allocating_queued), or on an epoch
// or a destruction. Switching to it compiles a non-empty queue first.
constexpr uint32_t LOOKAHEAD_HORIZONS = 0xFFFFFFFEu;

static void deliver(Ctx& c, Node& n, Item it) {
  if (it.kind == I_LOOKAHEAD) {
    if (it.arg == LOOKAHEAD_HORIZONS && !n.queue.empty()) flush_queue(c, n);
    n.lookahead = it.arg;
    n.horizons_after_alloc = 0;
    if (!n.queue.empty() && queued_tasks(n) > n.lookahead) flush_queue(c, n);
    return;
  }
  const bool horizons = n.lookahead == LOOKAHEAD_HORIZONS;
  if (n.queue.empty()) {
    if (it.kind == I_TASK && allocating(n, it.nt)) {
      n.queue.push_back(it);
      n.horizons_after_alloc = 0;
      if (!horizons && queued_tasks(n) > n.lookahead) flush_queue(c, n);
    } else {
      process(c, n, it, {});
    }
    return;
  }
  const bool force = it.kind == I_EPOCH || it.kind == I_DESTROY;
  if (horizons) {
    if (it.kind == I_TASK && allocating_queued(n, it.nt)) n.horizons_after_alloc = 0;
    n.queue.push_back(it);
    if (it.kind == I_HORIZON) n.horizons_after_alloc += 1;
    if (force || n.horizons_after_alloc >= 2) flush_queue(c, n);
    return;
  }
  n.queue.push_back(it);
  if (force || queued_tasks(n) > n.lookahead) flush_queue(c, n);
}

static void broadcast(Ctx& c, ItemKind k, uint32_t arg) {
  const uint32_t s = c.seq++;
  for (Node& n : c.nodes) {
    Item it;
    it.kind = k; it.seq = s; it.arg = arg;
    deliver(c, n, it);
  }
}

// a3: node-level push / await-push [R12, R19]; returns false if the task has
// overlapping writes (rejected, no state change).
// Task-graph bookkeeping for the critical-path horizon cadence [R29] (Sec.
// 3.5): a task's region per accessor is its range mapper over the task's
// whole range; it depends on the last writers of every region it accesses
// and, for writes, on the tasks that read the region since; its depth is one
// more than its deepest predecessor's. True when the critical path (the
// largest depth so far) has grown by horizon_step since the last horizon.
static bool critical_path_step(Ctx& c, const TaskDesc& t) {
  Box whole;
  for (int d = 0; d < 3; ++d) { whole.lo[d] = 0; whole.hi[d] = t.range[d]; }
  std::vector<std::pair<uint32_t, Box>> acc(t.nacc);
  uint32_t deepest = 0;
  for (uint32_t a = 0; a < t.nacc; ++a) {
    const uint32_t b = t.acc[a].buffer;
    acc[a] = {b, map_box(t.acc[a], whole, c.bufs[b])};
    if (empty(acc[a].second)) continue;
    for (const auto& e : c.t_writers[b])
      if (overlap(e.first, acc[a].second)) deepest = std::max(deepest, c.depth[e.second]);
    if (t.acc[a].mode & M_WRITE)
      for (const auto& e : c.t_readers[b])
        if (overlap(e.first, acc[a].second)) deepest = std::max(deepest, c.depth[e.second]);
  }
  const uint32_t me = (uint32_t)c.depth.size();
  c.depth.push_back(deepest + 1);
  for (uint32_t a = 0; a < t.nacc; ++a)
    if ((t.acc[a].mode & M_READ) && !empty(acc[a].second)) c.t_readers[acc[a].first].push_back({acc[a].second, me});
  for (uint32_t a = 0; a < t.nacc; ++a) {
    if (!(t.acc[a].mode & M_WRITE) || empty(acc[a].second)) continue;
    const Box& w = acc[a].second;
    for (auto* list : {&c.t_writers[acc[a].first], &c.t_readers[acc[a].first]}) {
      std::vector<std::pair<Box, uint32_t>> kept;
      for (const auto& e : *list)
        for (const Box& rest : region_minus({e.first}, {w})) kept.push_back({rest, e.second});
      *list = kept;
    }
    c.t_writers[acc[a].first].push_back({w, me});
  }
  c.cpl = std::max(c.cpl, deepest + 1);
  if (c.hstep && c.cpl >= c.cpl_at_horizon + c.hstep) {
    c.cpl_at_horizon = c.cpl;
    return true;
  }
  return false;
}

static bool submit(Ctx& c, const TaskDesc& td) {
  c.tasks.push_back(td);
  const TaskDesc& t = c.tasks.back();
  const uint32_t seq = c.seq++;
  const std::vector<Chunk> ch = split(c, t);
  std::vector<std::vector<Box>> mapped(ch.size());
  for (size_t i = 0; i < ch.size(); ++i)
    for (uint32_t a = 0; a < t.nacc; ++a) mapped[i].push_back(map_box(t.acc[a], ch[i].box, c.bufs[t.acc[a].buffer]));
  bool bad = false;
  for (size_t i = 0; i < ch.size(); ++i)
    for (size_t j = i + 1; j < ch.size(); ++j)
      for (uint32_t a = 0; a < t.nacc; ++a)
        for (uint32_t b = 0; b < t.nacc; ++b) {
          if (!(t.acc[a].mode & M_WRITE) || !(t.acc[b].mode & M_WRITE)) continue;
          if (t.acc[a].buffer != t.acc[b].buffer) continue;
          if (!empty(mapped[i][a]) && !empty(mapped[j][b]) && overlap(mapped[i][a], mapped[j][b])) bad = true;
        }
  std::vector<NodeTask> per(c.N);
  for (uint32_t n = 0; n < c.N; ++n) {
    per[n].seq = seq;
    per[n].t = &t;
    for (size_t i = 0; i < ch.size(); ++i) {
      if (ch[i].node == n) {
        per[n].chunks.push_back(ch[i]);
        per[n].mapped.push_back(mapped[i]);
      } else {
        per[n].remote.push_back({ch[i], mapped[i]});
      }
    }
  }
  if (!bad) {
    std::set<uint32_t> bufs;
    for (uint32_t a = 0; a < t.nacc; ++a) bufs.insert(t.acc[a].buffer);
    for (uint32_t b : bufs) {
      RMap<Own>& own = c.own[b];
      std::vector<Region> missing(c.N);
      for (uint32_t m = 0; m < c.N; ++m) {
        Region R;
        for (size_t i = 0; i < ch.size(); ++i)
          for (uint32_t a = 0; a < t.nacc; ++a)
            if (ch[i].node == m && t.acc[a].buffer == b && (t.acc[a].mode & M_READ) && !empty(mapped[i][a]))
              R.push_back(mapped[i][a]);
        // union of the chunk boxes as a disjoint region
        Region U;
        for (const Box& x : R) {
          Region add = region_minus({x}, U);
          U.insert(U.end(), add.begin(), add.end());
        }
        Region miss;
        for (const auto& e : own.query(U))
          if (!(e.second.repl >> m & 1u)) miss.push_back(e.first);
        missing[m] = canonical(miss);
      }
      for (uint32_t m = 0; m < c.N; ++m) {
        if (missing[m].empty()) continue;
        per[m].await_[b] = missing[m];
        auto parts = own.query(missing[m]);
        for (uint32_t o = 0; o < c.N; ++o) {
          Region g;
          for (const auto& e : parts)
            if (e.second.owner == o) g.push_back(e.first);
          g = canonical(g);
          if (!g.empty()) per[o].push[{b, m}] = g;
        }
      }
      for (uint32_t m = 0; m < c.N; ++m)
        own.update(missing[m], [m](const Own& v) { return Own{v.owner, v.repl | (1u << m)}; });
      for (size_t i = 0; i < ch.size(); ++i)
        for (uint32_t a = 0; a < t.nacc; ++a)
          if (t.acc[a].buffer == b && (t.acc[a].mode & M_WRITE) && !empty(mapped[i][a])) {
            const uint32_t o = ch[i].node;
            own.update({mapped[i][a]}, [o](const Own&) { return Own{o, 1u << o}; });
          }
    }
    for (uint32_t n = 0; n < c.N; ++n) {
      Item it;
      it.kind = I_TASK; it.seq = seq; it.arg = 0; it.nt = per[n];
      deliver(c, c.nodes[n], it);
    }
  } else {
    c.rejected.push_back(seq);
  }
  const bool cp_horizon = critical_path_step(c, t);  // every task counts, rejected or not [R29]
  ++c.ntasks;
  if (c.horizon_cp ? cp_horizon : (c.hstep && c.ntasks % c.hstep == 0)) broadcast(c, I_HORIZON, 0);
  return !bad;
}

}  // namespace orc

// ---- C interface used by the tests (ctypes) ---------------------------------

using namespace orc;

extern "C" {

void* orc_create(uint32_t nodes, uint32_t devs, uint32_t horizon_step, uint32_t lookahead) {
  if (nodes == 0 || devs == 0 || nodes > 32 || devs > 29) return nullptr;
  Ctx* c = new Ctx();
  c->N = nodes; c->D = devs; c->hstep = horizon_step;
  c->nodes.resize(nodes);
  for (uint32_t n = 0; n < nodes; ++n) {
    Node& nd = c->nodes[n];
    nd.id = n;
    nd.lookahead = lookahead;
    Instr e = rec0(EPOCH, NONE);
    e.id = 0;
    nd.instrs.push_back(e);
    nd.front.insert(0);
    nd.epoch = 0;
  }
  return c;
}

void orc_destroy(void* p) { delete static_cast<Ctx*>(p); }

int orc_create_buffer(void* p, uint32_t dims, const uint32_t* extent, uint32_t elem, int init) {
  Ctx* c = static_cast<Ctx*>(p);
  if (dims < 1 || dims > 3) return -1;
  BufDesc b{};
  b.dims = dims;
  for (int d = 0; d < 3; ++d) b.extent[d] = d < (int)dims ? extent[d] : 1;
  for (int d = 0; d < (int)dims; ++d)
    if (b.extent[d] == 0) return -1;
  b.elem = elem; b.init = init != 0; b.live = true;
  const uint32_t id = (uint32_t)c->bufs.size();
  c->bufs.push_back(b);
  RMap<Own> own;
  own.init(buffer_box(b), Own{init ? HOST : NONE, 0xFFFFFFFFu});
  c->own[id] = own;
  broadcast(*c, I_CREATE, id);
  return (int)id;
}

int orc_destroy_buffer(void* p, uint32_t b) {
  Ctx* c = static_cast<Ctx*>(p);
  if (b >= c->bufs.size() || !c->bufs[b].live) return -1;
  c->bufs[b].live = false;
  broadcast(*c, I_DESTROY, b);
  c->own.erase(b);
  return 0;
}

// Flat task layout: dims, range[3], chunks, kernel, nacc, params[4], then per
// accessor: buffer, mode, 3 x (kind, a, b, c).
int orc_submit_task(void* p, const uint32_t* w) {
  Ctx* c = static_cast<Ctx*>(p);
  TaskDesc t{};
  t.dims = w[0];
  for (int d = 0; d < 3; ++d) t.range[d] = w[1 + d];
  t.chunks = w[4]; t.kernel = w[5]; t.nacc = w[6];
  for (int i = 0; i < 4; ++i) t.params[i] = w[7 + i];
  if (t.nacc > 8 || t.chunks == 0 || t.dims < 1 || t.dims > 3) return -1;
  if ((t.chunks >> 16) && ((t.chunks & 0xFFFFu) == 0 || t.dims < 2)) return -1;  // a 2D split needs rows and dims >= 2
  for (uint32_t a = 0; a < t.nacc; ++a) {
    const uint32_t* x = w + 11 + 14 * a;
    t.acc[a].buffer = x[0]; t.acc[a].mode = x[1];
    if (x[0] >= c->bufs.size() || !c->bufs[x[0]].live || x[1] < 1 || x[1] > 3) return -1;
    for (int d = 0; d < 3; ++d) {
      t.acc[a].m[d] = MapDim{x[2 + 4 * d], x[3 + 4 * d], x[4 + 4 * d], x[5 + 4 * d]};
      if (t.acc[a].m[d].kind > 2 || (t.acc[a].m[d].kind == 0 && t.acc[a].m[d].a > 2)) return -1;
    }
  }
  return submit(*c, t) ? 0 : -2;
}

int orc_set_horizon_cp(void* p, int on) {
  static_cast<Ctx*>(p)->horizon_cp = on != 0;
  return 0;
}

int orc_set_stage_d2d(void* p, int on) {
  Ctx* c = static_cast<Ctx*>(p);
  for (Node& n : c->nodes) n.stage_d2d = on != 0;
  return 0;
}

int orc_set_lookahead(void* p, uint32_t L) {
  Ctx* c = static_cast<Ctx*>(p);
  const uint32_t s = c->seq;  // a control item consumes no sequence number
  for (Node& n : c->nodes) {
    Item it;
    it.kind = I_LOOKAHEAD; it.seq = s; it.arg = L;
    deliver(*c, n, it);
  }
  return 0;
}

int orc_flush(void* p) {
  broadcast(*static_cast<Ctx*>(p), I_EPOCH, 0);
  return 0;
}

// what: 0 instructions (11 u32), 1 edges (3), 2 boxes (6), 3 bindings (7),
// 4 diagnostics (3), 5 rejected task sequence numbers (1, node ignored).
uint32_t orc_count(void* p, uint32_t node, int what) {
  Ctx* c = static_cast<Ctx*>(p);
  if (what == 5) return (uint32_t)c->rejected.size();
  const Node& n = c->nodes[node];
  switch (what) {
    case 0: return (uint32_t)n.instrs.size();
    case 1: return (uint32_t)n.edges.size();
    case 2: return (uint32_t)n.boxes.size();
    case 3: return (uint32_t)n.binds.size();
    case 4: return (uint32_t)n.diags.size();
  }
  return 0;
}

int orc_copy_out(void* p, uint32_t node, int what, uint32_t* dst) {
  Ctx* c = static_cast<Ctx*>(p);
  if (what == 5) {
    for (size_t i = 0; i < c->rejected.size(); ++i) dst[i] = c->rejected[i];
    return 0;
  }
  const Node& n = c->nodes[node];
  size_t k = 0;
  switch (what) {
    case 0:
      for (const Instr& x : n.instrs) {
        const uint32_t v[11] = {x.id, x.type, x.seq, x.a, x.b, x.c, x.d, x.box_off, x.box_cnt, x.bind_off, x.bind_cnt};
        std::memcpy(dst + k, v, sizeof v); k += 11;
      }
      break;
    case 1:
      for (const Edge& e : n.edges) { dst[k++] = e.from; dst[k++] = e.to; dst[k++] = e.kind; }
      break;
    case 2:
      for (const Box& b : n.boxes)
        for (int d = 0; d < 6; ++d) dst[k++] = d < 3 ? b.lo[d] : b.hi[d - 3];
      break;
    case 3:
      for (const Bind& b : n.binds) {
        dst[k++] = b.alloc;
        for (int d = 0; d < 6; ++d) dst[k++] = d < 3 ? b.box.lo[d] : b.box.hi[d - 3];
      }
      break;
    case 4:
      for (const Diag& d : n.diags) { dst[k++] = d.seq; dst[k++] = d.chunk; dst[k++] = d.acc; }
      break;
  }
  return 0;
}

// Canonical form of a box list (6 u32 per box), for the box-algebra pins.
uint32_t orc_canonical(const uint32_t* in, uint32_t n, uint32_t* out) {
  Region r;
  for (uint32_t i = 0; i < n; ++i) {
    Box b;
    for (int d = 0; d < 3; ++d) { b.lo[d] = in[6 * i + d]; b.hi[d] = in[6 * i + 3 + d]; }
    r.push_back(b);
  }
  Region c = canonical(r);
  for (size_t i = 0; i < c.size(); ++i)
    for (int d = 0; d < 3; ++d) { out[6 * i + d] = c[i].lo[d]; out[6 * i + 3 + d] = c[i].hi[d]; }
  return (uint32_t)c.size();
}

// a \ b over box lists (for the box-algebra pins).
uint32_t orc_minus(const uint32_t* a, uint32_t na, const uint32_t* b, uint32_t nb, uint32_t* out, uint32_t cap) {
  Region A, B;
  for (uint32_t i = 0; i < na; ++i) {
    Box x;
    for (int d = 0; d < 3; ++d) { x.lo[d] = a[6 * i + d]; x.hi[d] = a[6 * i + 3 + d]; }
    A.push_back(x);
  }
  for (uint32_t i = 0; i < nb; ++i) {
    Box x;
    for (int d = 0; d < 3; ++d) { x.lo[d] = b[6 * i + d]; x.hi[d] = b[6 * i + 3 + d]; }
    B.push_back(x);
  }
  Region c = region_minus(A, B);
  if (c.size() > cap) return 0xFFFFFFFFu;
  for (size_t i = 0; i < c.size(); ++i)
    for (int d = 0; d < 3; ++d) { out[6 * i + d] = c[i].lo[d]; out[6 * i + 3 + d] = c[i].hi[d]; }
  return (uint32_t)c.size();
}

}  // extern "C"
