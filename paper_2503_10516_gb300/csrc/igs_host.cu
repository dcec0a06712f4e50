// Host front-end of libigs: the C ABI of include/igs.h.
//
// The host side only validates descriptors, appends submissions to the
// device-visible item stream, launches the lowering kernel, and drives the
// executor; chunking, range mappers, region maps, allocation planning,
// coherence, transfers and dependencies all run in the CUDA lowering engine.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cstdio>
#include <thread>
#include <cstring>
#include <deque>
#include <map>
#include <unordered_map>
#include <string>
#include <vector>

#include "igs_check.h"
#include "igs_exec.h"
#include "igs_internal.h"
#include "igs_tdag.h"

using namespace igs;

namespace {

struct ExecAlloc {
  uint8_t* ptr = nullptr;
  uint32_t buffer = 0, mem = 0;
  uint32_t lo[3] = {0, 0, 0}, hi[3] = {1, 1, 1};
  bool live = false, user = false;
};

// A send the executor has carried out: its data sits in a mailbox (device
// memory of its own) until the matching receive copies it out.
struct SendRec {
  uint32_t node, level;
  uint32_t fid = 0;  // its dataflow node (execute call `call`)
  uint64_t call;  // execute call that copied the data into the mailbox
  igs_box box;
  uint8_t* mail;
};

struct NodeHost {
  // fetched graph (everything so far) for execution
  std::vector<igs_instruction> instrs;
  std::vector<igs_edge> edges;
  std::vector<igs_box> boxes;
  std::vector<igs_binding> binds;
  std::vector<uint32_t> first_edge;  // per instruction: index of its first edge
  uint32_t executed = 1;             // instruction 0 is the initial epoch
  std::map<uint32_t, ExecAlloc> allocs;
  std::vector<uint32_t> level;       // topological level per instruction (current execute call)
  std::vector<uint32_t> fid;         // dataflow node per instruction (current execute call)
};

// Which kernel instruction an out-of-bounds record slot belongs to.
struct OobMeta {
  uint32_t seq, node, chunk, nacc;
};

// A call's out-of-bounds records, kept until they have been read back.
struct OobKeep {
  uint32_t* rec;
  uint32_t first, count;  // slots [first, first + count)
};

// A dataflow launch kept until its node timestamps have been read back.
struct FlowKeep {
  void* arena;
  size_t off_nodes;
  uint32_t n_nodes;
};

}  // namespace

struct igs_ctx {
  igs_config cfg{};
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  std::string err;
  uint32_t N = 0, D = 0;
  std::vector<BufDesc> bufs;
  std::vector<uint8_t*> init_dev;  // per buffer: device copy of host_init (user memory M0), or null
  std::vector<bool> buf_live;
  std::vector<Item> items;
  std::vector<igs_task> tasks;
  std::vector<uint32_t> seq_task;  // submission sequence number -> task index (NONE if not a task)
  uint32_t items_up = 0, tasks_up = 0, bufs_up = 0;
  uint32_t seq = 0, ntasks = 0;
  CriticalPath cpath;  // task-graph depth (IGS_FLAG_HORIZON_CP)
  // device
  Item* d_items = nullptr;
  uint32_t cap_items = 0;
  igs_task* d_tasks = nullptr;
  uint32_t cap_tasks = 0;
  BufDesc* d_bufs = nullptr;
  uint32_t cap_bufs = 0;
  uint32_t* d_nitems = nullptr;
  ProgDev* d_prog = nullptr;
  NodeDev* d_nodes = nullptr;
  Unit* d_units = nullptr;
  void* d_arena = nullptr;
  std::vector<NodeDev> nodes_host;  // layout templates (pointers), refreshed by downloads
  // executor
  std::vector<NodeHost> nh;
  cudaStream_t xstream = nullptr;  // executor stream of pipelined runs (own, created on first use)
  cudaStream_t cstream = nullptr;  // copies of graph records to the host during pipelined runs
  volatile uint32_t* m_progress = nullptr;  // host-mapped progress records (PR_WORDS per node)
  uint32_t* d_progress = nullptr;
  uint32_t* d_helpers = nullptr;  // helper warps' scratch of every node (pipelined runs)
  bool pipelined = false;          // a pipelined run is in progress: launches go to xstream
  std::multimap<uint64_t, SendRec> sends;  // (seq, buffer, receiver) -> sends not yet received
  uint64_t exec_call = 0;
  // job arrays: two sets, used alternately; a set is reused once the event
  // recorded after its last launch has completed
  CopyJob* d_cjobs[2] = {nullptr, nullptr};
  uint32_t cap_cjobs[2] = {0, 0};
  KernelJob* d_kjobs[2] = {nullptr, nullptr};
  uint32_t cap_kjobs[2] = {0, 0};
  CopyJob* h_cjobs[2] = {nullptr, nullptr};  // pinned staging of the job arrays
  KernelJob* h_kjobs[2] = {nullptr, nullptr};
  uint32_t hcap_cjobs[2] = {0, 0}, hcap_kjobs[2] = {0, 0};
  cudaEvent_t jobs_done[2] = {nullptr, nullptr};
  int jobs_set = 0;
  // dataflow executor: pinned staging of each launch's arrays (two sets, as
  // the job arrays), launches kept for timestamp read-back, statistics
  uint32_t executor = IGS_EXEC_LEVELS;
  uint8_t* h_flow[2] = {nullptr, nullptr};
  size_t hcap_flow[2] = {0, 0};
  std::vector<FlowKeep> flow_keep;
  // outgrown pinned staging, freed with the context: freeing page-locked
  // memory waits for the whole device, which would stall the host loop of a
  // pipelined run behind the lowering launch
  std::vector<void*> retired_pinned;
  // accessor bounds checking: one slot per kernel job, read back at sync points
  std::vector<OobMeta> oob_meta;
  std::vector<OobKeep> oob_keep;
  std::vector<igs_bounds_error> bounds;
  bool oob_pending = false;  // violations found since the last execute / run returned
  double flow_stats[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  uint64_t launches = 0;
  size_t arena_bytes = 0;
  // serving: submissions live in host-mapped memory the loop polls
  igs_server* server = nullptr;
  // waiting in the server's admission queue: submissions are kept on the host
  // (not published, not lowered) until a detach makes room
  bool serve_pending = false;
  // per-item completion timestamps (igs_set_item_times): nodes x cap_item_ts
  bool item_times = false;
  uint64_t* d_item_ts = nullptr;
  uint32_t cap_item_ts = 0;
  std::vector<uint32_t> slot_ids;
  Item* m_items = nullptr;
  igs_task* m_tasks = nullptr;
  uint32_t* m_nitems = nullptr;
  uint32_t serve_cap = 0;
  uint32_t m_cap = 0;  // entries of m_items / m_tasks
  // device-time accounting
  bool timing = false;
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev_pool;
  size_t ev_used = 0;
  std::vector<std::pair<int, size_t>> ev_pending;  // (class, index into ev_pool)
  double ms[3] = {0, 0, 0};
  double last_lower_ms = 0;
  uint64_t n_launch[3] = {0, 0, 0};
  double copy_bytes = 0;
};

struct igs_server {
  igs_serve_config cfg{};
  cudaStream_t stream = nullptr;
  ServeSlot* slots = nullptr;  // host-mapped
  ServeSlot* d_slots = nullptr;
  uint32_t* stop = nullptr;    // host-mapped
  uint32_t* d_stop = nullptr;
  cudaEvent_t done_ev = nullptr;
  bool launched = false;
  std::vector<uint32_t> free_slots;
  double used = 0;
  std::vector<std::pair<igs_ctx*, double>> attached;
  // admission queue (FIFO): contexts that did not fit when enqueued, with
  // their submission capacity
  std::deque<std::pair<igs_ctx*, uint32_t>> waiting;
  uint64_t n_admitted = 0, n_admitted_queued = 0, peak_waiting = 0;
};

namespace {

int fail_ctx(igs_ctx* c, int code, const std::string& msg) {
  if (c) c->err = msg;
  return code;
}

#define CK(x)                                                                               \
  do {                                                                                      \
    cudaError_t e_ = (x);                                                                   \
    if (e_ != cudaSuccess) return fail_ctx(c, IGS_ERR_CUDA, std::string(#x ": ") + cudaGetErrorString(e_)); \
  } while (0)

template <class T>
int grow_device(igs_ctx* c, T*& ptr, uint32_t& cap, uint32_t need, uint32_t used) {
  if (need <= cap) return IGS_OK;
  uint32_t ncap = std::max<uint32_t>(need, std::max<uint32_t>(64, cap * 2));
  T* np = nullptr;
  CK(cudaStreamSynchronize(c->stream));
  CK(cudaMalloc(&np, sizeof(T) * (size_t)ncap));
  if (ptr && used) CK(cudaMemcpy(np, ptr, sizeof(T) * (size_t)used, cudaMemcpyDeviceToDevice));
  if (ptr) CK(cudaFree(ptr));
  ptr = np;
  cap = ncap;
  return IGS_OK;
}

int upload_prog(igs_ctx* c) {
  int r;
  if ((r = grow_device(c, c->d_items, c->cap_items, (uint32_t)c->items.size(), c->items_up))) return r;
  if ((r = grow_device(c, c->d_tasks, c->cap_tasks, (uint32_t)c->tasks.size(), c->tasks_up))) return r;
  if ((r = grow_device(c, c->d_bufs, c->cap_bufs, (uint32_t)c->bufs.size(), c->bufs_up))) return r;
  if (c->tasks.size() > c->tasks_up)
    CK(cudaMemcpyAsync(c->d_tasks + c->tasks_up, c->tasks.data() + c->tasks_up,
                       sizeof(igs_task) * (c->tasks.size() - c->tasks_up), cudaMemcpyHostToDevice, c->stream));
  if (c->bufs.size() > c->bufs_up)
    CK(cudaMemcpyAsync(c->d_bufs + c->bufs_up, c->bufs.data() + c->bufs_up,
                       sizeof(BufDesc) * (c->bufs.size() - c->bufs_up), cudaMemcpyHostToDevice, c->stream));
  if (c->items.size() > c->items_up)
    CK(cudaMemcpyAsync(c->d_items + c->items_up, c->items.data() + c->items_up,
                       sizeof(Item) * (c->items.size() - c->items_up), cudaMemcpyHostToDevice, c->stream));
  c->tasks_up = (uint32_t)c->tasks.size();
  c->bufs_up = (uint32_t)c->bufs.size();
  c->items_up = (uint32_t)c->items.size();
  ProgDev p;
  p.items = c->d_items;
  p.tasks = c->d_tasks;
  p.bufs = c->d_bufs;
  p.n_items = c->d_nitems;
  p.src_items = nullptr;
  p.src_tasks = nullptr;
  CK(cudaMemcpyAsync(c->d_prog, &p, sizeof p, cudaMemcpyHostToDevice, c->stream));
  const uint32_t n = (uint32_t)c->items.size();
  CK(cudaMemcpyAsync(c->d_nitems, &n, sizeof n, cudaMemcpyHostToDevice, c->stream));
  return IGS_OK;
}

// Event pair around one launch of class k (0 lowering, 1 box copy, 2 workload).
size_t ev_begin(igs_ctx* c, cudaStream_t s = nullptr) {
  if (c->ev_used == c->ev_pool.size()) {
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    c->ev_pool.push_back({a, b});
  }
  cudaEventRecord(c->ev_pool[c->ev_used].first, s ? s : c->stream);
  return c->ev_used++;
}
void ev_end(igs_ctx* c, int k, size_t i, cudaStream_t s = nullptr) {
  cudaEventRecord(c->ev_pool[i].second, s ? s : c->stream);
  c->ev_pending.push_back({k, i});
}
// Folds completed event pairs into the totals (after a stream sync; held
// back while a pipelined run still has executor work in flight).
void ev_collect(igs_ctx* c) {
  if (c->pipelined) return;
  for (auto& p : c->ev_pending) {
    float t = 0;
    cudaEventElapsedTime(&t, c->ev_pool[p.second].first, c->ev_pool[p.second].second);
    c->ms[p.first] += t;
    if (p.first == 0) c->last_lower_ms = t;
  }
  c->ev_pending.clear();
  c->ev_used = 0;
}

// Scratch for the helper warps that share each node's kernel phase (nodes
// with more than one device only).
int ensure_helpers(igs_ctx* c) {
  if (c->d_helpers || c->D < 2) return IGS_OK;
  const size_t per = (size_t)kScratchSets * kHelperTables * c->nodes_host[0].cap_scratch * F_COUNT;
  CK(cudaStreamSynchronize(c->stream));
  CK(cudaMalloc((void**)&c->d_helpers, sizeof(uint32_t) * per * c->N));
  for (uint32_t n = 0; n < c->N; ++n) {
    uint32_t* p = c->d_helpers + per * n;
    CK(cudaMemcpy(&c->d_nodes[n].helper_scratch, &p, sizeof p, cudaMemcpyHostToDevice));
    c->nodes_host[n].helper_scratch = p;
  }
  return IGS_OK;
}

// Timestamp array of at least the context's item count per node (item timing on).
int ensure_item_ts(igs_ctx* c) {
  const uint32_t need = (uint32_t)c->items.size();
  if (need <= c->cap_item_ts) return IGS_OK;
  const uint32_t cap = std::max<uint32_t>(need, std::max<uint32_t>(1024, 2 * c->cap_item_ts));
  uint64_t* p = nullptr;
  CK(cudaStreamSynchronize(c->stream));
  CK(cudaMalloc(&p, sizeof(uint64_t) * (size_t)cap * c->N));
  CK(cudaMemset(p, 0, sizeof(uint64_t) * (size_t)cap * c->N));
  for (uint32_t n = 0; n < c->N; ++n) {
    if (c->d_item_ts)
      CK(cudaMemcpy(p + (size_t)cap * n, c->d_item_ts + (size_t)c->cap_item_ts * n, sizeof(uint64_t) * c->cap_item_ts,
                    cudaMemcpyDeviceToDevice));
    uint64_t* q = p + (size_t)cap * n;
    CK(cudaMemcpy(&c->d_nodes[n].item_ts, &q, sizeof q, cudaMemcpyHostToDevice));
    c->nodes_host[n].item_ts = q;
  }
  if (c->d_item_ts) CK(cudaFree(c->d_item_ts));
  c->d_item_ts = p;
  c->cap_item_ts = cap;
  return IGS_OK;
}

int launch_lower(igs_ctx* c, uint32_t max_items = IGS_NONE, bool reserve = false, uint32_t* progress = nullptr) {
  if (c->server) return IGS_OK;  // the serving loop lowers it
  int r = upload_prog(c);
  if (r) return r;
  if (c->item_times && (r = ensure_item_ts(c))) return r;
  // one context's launch has few units (its nodes): helper warps share
  // parts of each node's lowering (nodes with several devices)
  const bool workers = c->D > 1;
  if (workers && (r = ensure_helpers(c))) return r;
  const size_t ev = c->timing ? ev_begin(c) : 0;
  if (igs_launch_lower(c->d_units, c->N, max_items, c->stream, reserve, progress, workers))
    return fail_ctx(c, IGS_ERR_CUDA, "lowering launch failed");
  if (c->timing) ev_end(c, 0, ev);
  c->launches++;
  c->n_launch[0]++;
  return IGS_OK;
}

int download_nodes(igs_ctx* c) {
  CK(cudaStreamSynchronize(c->stream));
  ev_collect(c);
  CK(cudaMemcpy(c->nodes_host.data(), c->d_nodes, sizeof(NodeDev) * c->N, cudaMemcpyDeviceToHost));
  return IGS_OK;
}

int check_status(igs_ctx* c) {
  int r = download_nodes(c);
  if (r) return r;
  for (uint32_t n = 0; n < c->N; ++n) {
    const NodeDev& nd = c->nodes_host[n];
    if (nd.status == ST_CAPACITY) {
      static const char* kinds[] = {"?", "scratch table (scratch_capacity)", "region-map heap (map_heap)",
                                    "allocations (max_allocations / max_live_allocs)", "instructions / edges",
                                    "boxes (max_boxes)", "bindings", "diagnostics", "buffers (max_buffers)",
                                    "lookahead queue (max_queue)"};
      const uint32_t k = nd.err_info >> 24;
      return fail_ctx(c, IGS_ERR_CAPACITY, std::string("capacity exceeded on node ") + std::to_string(n) + ": " +
                                               kinds[k < 10 ? k : 0] + ", capacity " +
                                               std::to_string(nd.err_info & 0xFFFFFFu));
    }
    if (nd.status == ST_TIMEOUT) return fail_ctx(c, IGS_ERR_TIMEOUT, "device wait timed out");
    if (nd.status != ST_OK)
      return fail_ctx(c, IGS_ERR_CUDA, "lowering engine internal error on node " + std::to_string(n) + " (status " +
                                           std::to_string(nd.status) + ", check " + std::to_string(nd.err_info) + ")");
  }
  if (c->nodes_host[0].n_rej) return fail_ctx(c, IGS_ERR_OVERLAPPING_WRITE, "a task with overlapping writes was rejected");
  return IGS_OK;
}

int push_item(igs_ctx* c, uint32_t kind, uint32_t arg, uint32_t task) {
  Item it;
  it.kind = kind;
  if (c->server && c->items.size() >= c->serve_cap) return fail_ctx(c, IGS_ERR_CAPACITY, "serving capacity of this context exceeded");
  if (kind != IT_LOOKAHEAD) c->seq_task.push_back(kind == IT_TASK ? task : NONE);
  it.seq = kind == IT_LOOKAHEAD ? c->seq : c->seq++;
  it.arg = arg;
  it.task = task;
  c->items.push_back(it);
  if (c->server && !c->serve_pending) {
    // the record, then (after a release fence) the count the loop polls
    if (kind == IT_TASK) c->m_tasks[task] = c->tasks[task];
    c->m_items[c->items.size() - 1] = it;
    std::atomic_thread_fence(std::memory_order_seq_cst);
    *reinterpret_cast<volatile uint32_t*>(c->m_nitems) = (uint32_t)c->items.size();
    std::atomic_thread_fence(std::memory_order_seq_cst);
    c->items_up = (uint32_t)c->items.size();
    c->tasks_up = (uint32_t)c->tasks.size();
  }
  return IGS_OK;
}

size_t table_bytes(uint32_t cap) { return (size_t)F_COUNT * cap * sizeof(uint32_t); }

}  // namespace

namespace {
int flow_collect(igs_ctx* c);
int oob_collect(igs_ctx* c);
int oob_status(igs_ctx* c);
}  // namespace

extern "C" {

int igs_create(const igs_config* cfg, igs_ctx** out) {
  if (!out) return IGS_ERR_INVALID_ARG;
  *out = nullptr;
  if (!cfg || cfg->num_nodes < 1 || cfg->num_nodes > 32 || cfg->devices_per_node < 1 || cfg->devices_per_node > 29)
    return IGS_ERR_INVALID_ARG;
  if (cfg->mode > IGS_MODE_BATCHED) return IGS_ERR_INVALID_ARG;
  if (!config_flags_ok(cfg->flags)) return IGS_ERR_INVALID_ARG;
  // scratch tables hold one entry per node (up to 32) or per accessor without a claim
  if (cfg->scratch_capacity && cfg->scratch_capacity < 32) return IGS_ERR_INVALID_ARG;
  igs_ctx* c = new igs_ctx();
  c->cfg = *cfg;
  c->N = cfg->num_nodes;
  c->D = cfg->devices_per_node;
  const uint32_t cap_instr = cfg->max_instructions ? cfg->max_instructions : (1u << 18);
  const uint32_t cap_edge = cfg->max_edges ? cfg->max_edges : 4 * cap_instr;
  const uint32_t cap_box = cfg->max_boxes ? cfg->max_boxes : 4 * cap_instr;
  const uint32_t cap_bind = 2 * cap_instr;
  const uint32_t cap_heap = cfg->map_heap ? cfg->map_heap : (1u << 20);
  const uint32_t cap_scr = cfg->scratch_capacity ? cfg->scratch_capacity : 4096;
  const uint32_t cap_buffers = cfg->max_buffers ? cfg->max_buffers : 64;
  const uint32_t cap_slots = cfg->max_live_allocs ? cfg->max_live_allocs : 1024;
  const uint32_t cap_alloc = cfg->max_allocations ? cfg->max_allocations : (1u << 16);
  const uint32_t cap_queue = cfg->max_queue ? cfg->max_queue : (1u << 16);
  const uint32_t cap_qr = std::max<uint32_t>(4096, std::min<uint32_t>(1u << 16, 4 * cap_queue));
  const uint32_t cap_diag = std::min<uint32_t>(1u << 16, cap_instr), cap_rej = 1024;
  cudaError_t e = cudaSetDevice(cfg->device);
  if (e != cudaSuccess) {
    delete c;
    return IGS_ERR_CUDA;
  }
  // kernels load on first use otherwise, and loading one while the lowering
  // launch runs would hold up the first pipelined run until that launch ends
  igs_exec_preload();
  if (cfg->stream) {
    c->stream = (cudaStream_t)cfg->stream;
  } else {
    if (cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking) != cudaSuccess) {
      delete c;
      return IGS_ERR_CUDA;
    }
    c->own_stream = true;
  }
  // per-node arena
  size_t per = 0;
  auto take = [&](size_t bytes) {
    size_t off = per;
    per += (bytes + 255) & ~(size_t)255;
    return off;
  };
  const size_t o_heap = take(table_bytes(cap_heap));
  const size_t o_desc = take(sizeof(uint32_t) * kDesc * (2 * cap_buffers + 2 * cap_slots));
  const size_t o_free = take(sizeof(uint32_t) * cap_slots);
  const size_t o_live = take(sizeof(uint32_t) * cap_slots);
  const size_t o_qr = take(table_bytes(cap_qr));
  const size_t o_alloc = take(sizeof(AllocRec) * cap_alloc);
  const size_t o_queue = take(sizeof(uint32_t) * cap_queue);
  const size_t o_succ = take(cap_instr);
  const size_t o_instr = take(sizeof(igs_instruction) * cap_instr);
  const size_t o_edge = take(sizeof(igs_edge) * cap_edge);
  const size_t o_box = take(sizeof(igs_box) * cap_box);
  const size_t o_bind = take(sizeof(igs_binding) * cap_bind);
  const size_t o_diag = take(sizeof(igs_diag) * cap_diag);
  const size_t o_rej = take(sizeof(uint32_t) * cap_rej);
  const size_t o_scr = take(table_bytes(cap_scr) * 14);
  c->arena_bytes = per * c->N;
  if (cudaMalloc(&c->d_arena, per * c->N) != cudaSuccess || cudaMalloc(&c->d_nodes, sizeof(NodeDev) * c->N) != cudaSuccess ||
      cudaMalloc(&c->d_units, sizeof(Unit) * c->N) != cudaSuccess || cudaMalloc(&c->d_prog, sizeof(ProgDev)) != cudaSuccess ||
      cudaMalloc(&c->d_nitems, sizeof(uint32_t)) != cudaSuccess) {
    igs_destroy(c);
    return IGS_ERR_CUDA;
  }
  c->nodes_host.resize(c->N);
  std::vector<Unit> units(c->N);
  std::vector<uint32_t> slots(cap_slots);
  for (uint32_t i = 0; i < cap_slots; ++i) slots[i] = cap_slots - 1 - i;  // pops 0, 1, 2, ...
  for (uint32_t n = 0; n < c->N; ++n) {
    uint8_t* base = static_cast<uint8_t*>(c->d_arena) + per * n;
    NodeDev nd;
    std::memset(&nd, 0, sizeof nd);
    nd.node = n;
    nd.N = c->N;
    nd.D = c->D;
    nd.status = ST_OK;
    nd.cursor = 0;
    nd.lookahead = cfg->lookahead;
    nd.stage_d2d = (cfg->flags & IGS_FLAG_STAGE_D2D) ? 1u : 0u;
    nd.epoch = 0;
    nd.last_horizon = NONE;
    nd.last_sync = 0;
    nd.n_instr = 1;
    nd.n_free = cap_slots;
    nd.cap_instr = cap_instr;
    nd.cap_edge = cap_edge;
    nd.cap_box = cap_box;
    nd.cap_bind = cap_bind;
    nd.cap_diag = cap_diag;
    nd.cap_rej = cap_rej;
    nd.cap_alloc = cap_alloc;
    nd.cap_queue = cap_queue;
    nd.cap_buffers = cap_buffers;
    nd.cap_slots = cap_slots;
    nd.cap_qr = cap_qr;
    nd.cap_scratch = cap_scr;
    nd.heap = reinterpret_cast<uint32_t*>(base + o_heap);
    nd.cap_heap = cap_heap;
    nd.heap_top = 0;
    for (int k = 0; k < kHeapClasses; ++k) nd.free_head[k] = NONE;
    nd.own_d = reinterpret_cast<uint32_t*>(base + o_desc);
    nd.bst_d = nd.own_d + kDesc * cap_buffers;
    nd.wr_d = nd.bst_d + kDesc * cap_buffers;
    nd.rd_d = nd.wr_d + kDesc * cap_slots;
    nd.free_slots = reinterpret_cast<uint32_t*>(base + o_free);
    nd.live = reinterpret_cast<uint32_t*>(base + o_live);
    nd.qr_base = reinterpret_cast<uint32_t*>(base + o_qr);
    nd.allocs = reinterpret_cast<AllocRec*>(base + o_alloc);
    nd.queue = reinterpret_cast<uint32_t*>(base + o_queue);
    nd.has_succ = base + o_succ;
    nd.instrs = reinterpret_cast<igs_instruction*>(base + o_instr);
    nd.edges = reinterpret_cast<igs_edge*>(base + o_edge);
    nd.boxes = reinterpret_cast<igs_box*>(base + o_box);
    nd.binds = reinterpret_cast<igs_binding*>(base + o_bind);
    nd.diags = reinterpret_cast<igs_diag*>(base + o_diag);
    nd.rejected = reinterpret_cast<uint32_t*>(base + o_rej);
    nd.scratch_base = reinterpret_cast<uint32_t*>(base + o_scr);
    c->nodes_host[n] = nd;
    units[n].node = c->d_nodes + n;
    units[n].prog = c->d_prog;
    // initial epoch I0, empty tables, the slab free list
    igs_instruction i0{0, IGS_EPOCH, NONE, NONE, NONE, NONE, NONE, 0, 0, 0, 0};
    if (cudaMemcpy(nd.instrs, &i0, sizeof i0, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemset(nd.has_succ, 0, 1) != cudaSuccess ||
        cudaMemset(nd.own_d, 0, sizeof(uint32_t) * kDesc * (2 * cap_buffers + 2 * cap_slots)) != cudaSuccess ||
        cudaMemcpy(nd.free_slots, slots.data(), sizeof(uint32_t) * cap_slots, cudaMemcpyHostToDevice) != cudaSuccess) {
      igs_destroy(c);
      return IGS_ERR_CUDA;
    }
  }
  uint32_t zero = 0;
  if (cudaMemcpy(c->d_nodes, c->nodes_host.data(), sizeof(NodeDev) * c->N, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(c->d_units, units.data(), sizeof(Unit) * c->N, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(c->d_nitems, &zero, sizeof zero, cudaMemcpyHostToDevice) != cudaSuccess) {
    igs_destroy(c);
    return IGS_ERR_CUDA;
  }
  c->nh.resize(c->N);
  *out = c;
  return IGS_OK;
}

void igs_destroy(igs_ctx* c) {
  if (!c) return;
  if (c->stream) cudaStreamSynchronize(c->stream);
  if (c->xstream) cudaStreamSynchronize(c->xstream);
  for (auto& sr : c->sends)
    if (sr.second.mail) cudaFree(sr.second.mail);
  for (auto& f : c->flow_keep) cudaFree(f.arena);
  if (c->d_item_ts) cudaFree(c->d_item_ts);
  for (auto& o : c->oob_keep) cudaFree(o.rec);
  for (void* p : c->retired_pinned) cudaFreeHost(p);
  for (int k = 0; k < 2; ++k) {
    if (c->h_flow[k]) cudaFreeHost(c->h_flow[k]);
    if (c->d_cjobs[k]) cudaFreeAsync(c->d_cjobs[k], c->stream);
    if (c->d_kjobs[k]) cudaFreeAsync(c->d_kjobs[k], c->stream);
    if (c->h_cjobs[k]) cudaFreeHost(c->h_cjobs[k]);
    if (c->h_kjobs[k]) cudaFreeHost(c->h_kjobs[k]);
    if (c->jobs_done[k]) cudaEventDestroy(c->jobs_done[k]);
  }
  if (c->xstream) cudaStreamDestroy(c->xstream);
  if (c->cstream) cudaStreamDestroy(c->cstream);
  if (c->d_helpers) cudaFree(c->d_helpers);
  if (c->m_progress) cudaFreeHost((void*)c->m_progress);
  for (auto& e : c->ev_pool) {
    cudaEventDestroy(e.first);
    cudaEventDestroy(e.second);
  }
  for (auto& n : c->nh)
    for (auto& a : n.allocs)
      if (a.second.live && !a.second.user && a.second.ptr) cudaFree(a.second.ptr);
  for (uint8_t* p : c->init_dev)
    if (p) cudaFree(p);
  cudaFree(c->d_items);
  cudaFree(c->d_tasks);
  cudaFree(c->d_bufs);
  cudaFree(c->d_nitems);
  cudaFree(c->d_prog);
  cudaFree(c->d_nodes);
  cudaFree(c->d_units);
  cudaFree(c->d_arena);
  if (c->m_items) cudaFreeHost(c->m_items);
  if (c->m_tasks) cudaFreeHost(c->m_tasks);
  if (c->m_nitems) cudaFreeHost(c->m_nitems);
  if (c->own_stream) cudaStreamDestroy(c->stream);
  delete c;
}

const char* igs_last_error(const igs_ctx* c) { return c ? c->err.c_str() : "null context"; }

int igs_profile(igs_ctx* c, uint64_t out[32]) {
  if (!c || !out) return IGS_ERR_INVALID_ARG;
  int r = download_nodes(c);
  if (r) return r;
  std::memset(out, 0, sizeof(uint64_t) * 32);
  for (const NodeDev& nd : c->nodes_host)
    for (int k = 0; k < 32; ++k) out[k] += nd.prof[k];
  return IGS_OK;
}

int igs_bounds_errors(igs_ctx* c, igs_bounds_error* out, uint32_t cap, uint32_t* count) {
  if (!c || !count || (cap && !out)) return IGS_ERR_INVALID_ARG;
  CK(cudaStreamSynchronize(c->stream));
  if (c->xstream) CK(cudaStreamSynchronize(c->xstream));
  int r = oob_collect(c);
  if (r) return r;
  *count = (uint32_t)c->bounds.size();
  for (uint32_t i = 0; i < cap && i < c->bounds.size(); ++i) out[i] = c->bounds[i];
  return IGS_OK;
}

int igs_set_executor(igs_ctx* c, uint32_t executor) {
  if (!c || executor > IGS_EXEC_DATAFLOW) return IGS_ERR_INVALID_ARG;
  if (c->pipelined) return fail_ctx(c, IGS_ERR_STATE, "a pipelined run is in progress");
  c->executor = executor;
  return IGS_OK;
}

int igs_exec_stats(igs_ctx* c, double out[8]) {
  if (!c || !out) return IGS_ERR_INVALID_ARG;
  CK(cudaStreamSynchronize(c->stream));
  if (c->xstream) CK(cudaStreamSynchronize(c->xstream));
  int r = flow_collect(c);
  if (r) return r;
  for (int k = 0; k < 8; ++k) out[k] = c->flow_stats[k];
  return IGS_OK;
}

int igs_selftest_flow_wait(uint32_t wait_ms) {
  if (wait_ms < 1 || wait_ms > 10000) return IGS_ERR_INVALID_ARG;
  // layout: control block, two nodes, successor list {1, 0}, pending {1, 1},
  // claimed, finished, ready (both empty)
  const size_t o_nodes = 64, o_succ = o_nodes + 2 * sizeof(FlowNode), o_pend = o_succ + 16, o_claim = o_pend + 16,
               o_fin = o_claim + 16, o_ready = o_fin + 16, total = o_ready + 16;
  std::vector<uint8_t> H(total, 0);
  FlowNode* nodes = reinterpret_cast<FlowNode*>(H.data() + o_nodes);
  for (int i = 0; i < 2; ++i) {
    nodes[i].kind = FK_NONE;
    nodes[i].tiles = 1;
    nodes[i].succ_off = (uint32_t)i;
    nodes[i].succ_cnt = 1;
  }
  uint32_t* succ = reinterpret_cast<uint32_t*>(H.data() + o_succ);
  succ[0] = 1;
  succ[1] = 0;
  uint32_t* pend = reinterpret_cast<uint32_t*>(H.data() + o_pend);
  pend[0] = pend[1] = 1;
  uint32_t* ready = reinterpret_cast<uint32_t*>(H.data() + o_ready);
  ready[0] = ready[1] = 0xFFFFFFFFu;
  uint8_t* D = nullptr;
  cudaStream_t s = nullptr;
  if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) return IGS_ERR_CUDA;
  int r = IGS_ERR_CUDA;
  if (cudaMalloc((void**)&D, total) == cudaSuccess &&
      cudaMemcpy(D, H.data(), total, cudaMemcpyHostToDevice) == cudaSuccess &&
      igs_launch_flow(reinterpret_cast<FlowCtl*>(D), reinterpret_cast<FlowNode*>(D + o_nodes), 2,
                      reinterpret_cast<uint32_t*>(D + o_succ), reinterpret_cast<uint32_t*>(D + o_pend),
                      reinterpret_cast<uint32_t*>(D + o_claim), reinterpret_cast<uint32_t*>(D + o_fin),
                      reinterpret_cast<uint32_t*>(D + o_ready), nullptr, nullptr, (uint64_t)wait_ms * 1000000ull,
                      s) == 0 &&
      cudaStreamSynchronize(s) == cudaSuccess) {
    FlowCtl ctl;
    if (cudaMemcpy(&ctl, D, sizeof ctl, cudaMemcpyDeviceToHost) == cudaSuccess) {
      const int e = igs_exec_error(true);
      r = (ctl.error && e >= 0 && (e & 2)) ? IGS_ERR_TIMEOUT : IGS_OK;
    }
  }
  if (D) cudaFree(D);
  cudaStreamDestroy(s);
  return r;
}

int igs_set_timing(igs_ctx* c, int on) {
  if (!c) return IGS_ERR_INVALID_ARG;
  c->timing = on != 0;
  return IGS_OK;
}

int igs_set_item_times(igs_ctx* c, int on) {
  if (!c) return IGS_ERR_INVALID_ARG;
  if (c->server || c->pipelined) return fail_ctx(c, IGS_ERR_STATE, "the context is served or running");
  c->item_times = on != 0;
  if (!c->item_times && c->d_item_ts) {  // later launches record nothing
    CK(cudaStreamSynchronize(c->stream));
    for (uint32_t n = 0; n < c->N; ++n) {
      uint64_t* q = nullptr;
      CK(cudaMemcpy(&c->d_nodes[n].item_ts, &q, sizeof q, cudaMemcpyHostToDevice));
      c->nodes_host[n].item_ts = nullptr;
    }
    CK(cudaFree(c->d_item_ts));
    c->d_item_ts = nullptr;
    c->cap_item_ts = 0;
  }
  return IGS_OK;
}

int igs_item_times(igs_ctx* c, uint64_t* out, uint32_t cap, uint32_t* count) {
  if (!c || !count || (cap && !out)) return IGS_ERR_INVALID_ARG;
  const uint32_t n = (uint32_t)c->items.size();
  *count = n;
  if (!out || !c->d_item_ts) return IGS_OK;
  CK(cudaStreamSynchronize(c->stream));
  const uint32_t m = std::min<uint32_t>(std::min(n, cap), c->cap_item_ts);
  std::vector<uint64_t> ts((size_t)c->cap_item_ts * c->N);
  CK(cudaMemcpy(ts.data(), c->d_item_ts, sizeof(uint64_t) * ts.size(), cudaMemcpyDeviceToHost));
  for (uint32_t i = 0; i < m; ++i) {
    uint64_t t = 0;
    for (uint32_t k = 0; k < c->N; ++k) {
      const uint64_t v = ts[(size_t)c->cap_item_ts * k + i];
      if (v == 0) {  // not lowered on some node yet
        t = 0;
        break;
      }
      t = std::max(t, v);
    }
    out[2 * i] = c->items[i].kind;
    out[2 * i + 1] = t;
  }
  return IGS_OK;
}

int igs_stats(igs_ctx* c, double out[8]) {
  if (!c || !out) return IGS_ERR_INVALID_ARG;
  CK(cudaStreamSynchronize(c->stream));
  ev_collect(c);
  out[0] = c->ms[0];
  out[1] = c->ms[1];
  out[2] = c->ms[2];
  out[3] = c->copy_bytes;
  out[4] = (double)c->n_launch[0];
  out[5] = (double)c->n_launch[1];
  out[6] = (double)c->n_launch[2];
  out[7] = c->last_lower_ms;
  return IGS_OK;
}

int igs_create_buffer(igs_ctx* c, uint32_t dims, const uint32_t extent[3], uint32_t elem_size, const void* host_init,
                      uint32_t* out_buffer) {
  if (!c || !extent || !out_buffer) return fail_ctx(c, IGS_ERR_INVALID_ARG, "null argument");
  if (!buffer_shape_ok(dims, extent, elem_size)) return fail_ctx(c, IGS_ERR_INVALID_ARG, "bad buffer shape");
  BufDesc b{};
  b.dims = dims;
  uint64_t count = 1;
  for (int d = 0; d < 3; ++d) {
    b.extent[d] = d < (int)dims ? extent[d] : 1;
    if (b.extent[d] == 0) return fail_ctx(c, IGS_ERR_INVALID_ARG, "zero extent");
    count *= b.extent[d];
  }
  b.elem = elem_size;
  b.init = host_init ? 1 : 0;
  if (c->bufs.size() >= c->nodes_host[0].cap_buffers)
    return fail_ctx(c, IGS_ERR_CAPACITY, "too many buffers for this context");
  uint8_t* dev = nullptr;
  if (host_init) {
    CK(cudaMalloc(&dev, count * elem_size));
    CK(cudaMemcpy(dev, host_init, count * elem_size, cudaMemcpyHostToDevice));
  }
  if (c->server) return fail_ctx(c, IGS_ERR_STATE, "create buffers before attaching the context to a server");
  const uint32_t id = (uint32_t)c->bufs.size();
  c->bufs.push_back(b);
  c->init_dev.push_back(dev);
  c->buf_live.push_back(true);
  push_item(c, IT_CREATE, id, 0);
  *out_buffer = id;
  if (c->cfg.mode == IGS_MODE_PLAIN) return launch_lower(c);
  return IGS_OK;
}

int igs_destroy_buffer(igs_ctx* c, uint32_t b) {
  if (!c || b >= c->bufs.size() || !c->buf_live[b]) return fail_ctx(c, IGS_ERR_INVALID_ARG, "unknown buffer");
  c->buf_live[b] = false;
  if (int r = push_item(c, IT_DESTROY, b, 0)) return r;
  if (c->cfg.mode == IGS_MODE_PLAIN) return launch_lower(c);
  return IGS_OK;
}

int igs_submit_task(igs_ctx* c, const igs_task* t, uint64_t* out_seq) {
  if (!c || !t) return fail_ctx(c, IGS_ERR_INVALID_ARG, "null argument");
  if (const char* why = task_problem(*t, [c](uint32_t b) { return b < c->bufs.size() && c->buf_live[b]; }))
    return fail_ctx(c, IGS_ERR_INVALID_ARG, why);
  if (c->server && c->items.size() + 2 > c->serve_cap)
    return fail_ctx(c, IGS_ERR_CAPACITY, "serving capacity of this context exceeded");
  const uint32_t ti = (uint32_t)c->tasks.size();
  c->tasks.push_back(*t);
  const uint32_t s = c->seq;
  push_item(c, IT_TASK, 0, ti);
  const bool by_cp = (c->cfg.flags & IGS_FLAG_HORIZON_CP) != 0;
  const bool cp_horizon =
      by_cp && c->cpath.add(
                   *t, [c](uint32_t b) { return c->bufs[b].dims; }, [c](uint32_t b) { return c->bufs[b].extent; },
                   c->cfg.horizon_step);
  c->ntasks++;
  const bool horizon = by_cp ? cp_horizon : (c->cfg.horizon_step && c->ntasks % c->cfg.horizon_step == 0);
  if (horizon) push_item(c, IT_HORIZON, 0, 0);
  if (out_seq) *out_seq = s;
  if (c->cfg.mode == IGS_MODE_PLAIN) return launch_lower(c);
  return IGS_OK;
}

int igs_set_lookahead(igs_ctx* c, uint32_t L) {
  if (!c) return IGS_ERR_INVALID_ARG;
  if (int r = push_item(c, IT_LOOKAHEAD, L, 0)) return r;
  if (c->cfg.mode == IGS_MODE_PLAIN) return launch_lower(c);
  return IGS_OK;
}

int igs_sync(igs_ctx* c) {
  if (!c) return IGS_ERR_INVALID_ARG;
  if (c->server) return fail_ctx(c, IGS_ERR_STATE, "the context is served");
  if (c->items_up < c->items.size() || c->cfg.mode == IGS_MODE_BATCHED) {
    int r = launch_lower(c);
    if (r) return r;
  }
  return check_status(c);
}

int igs_submit_epoch(igs_ctx* c) {
  if (!c) return IGS_ERR_INVALID_ARG;
  if (int r = push_item(c, IT_EPOCH, 0, 0)) return r;
  if (c->cfg.mode == IGS_MODE_PLAIN) return launch_lower(c);
  return IGS_OK;
}

int igs_flush(igs_ctx* c) {
  if (!c) return IGS_ERR_INVALID_ARG;
  if (c->server) return fail_ctx(c, IGS_ERR_STATE, "the context is served: use igs_submit_epoch");
  push_item(c, IT_EPOCH, 0, 0);
  int r = launch_lower(c);
  if (r) return r;
  return check_status(c);
}

int igs_lower_batch(igs_ctx* const* ctxs, uint32_t n) { return igs_lower_batch_shaped(ctxs, n, nullptr); }

int igs_lower_batch_shaped(igs_ctx* const* ctxs, uint32_t n, const igs_batch_shape* shape) {
  if (!ctxs || n == 0) return IGS_ERR_INVALID_ARG;
  igs_ctx* c = ctxs[0];
  if (shape && (shape->order > IGS_ORDER_LONGEST_FIRST || shape->warps > kMaxWorkers))
    return fail_ctx(c, IGS_ERR_INVALID_ARG, "bad batch shape");
  const bool queue = shape && shape->persistent_blocks;
  const uint32_t warps = queue && shape->warps > 1 ? shape->warps : 1;
  std::vector<Unit> units;
  std::vector<double> work;  // estimated work per unit: pending items plus chunk-accessor pairs per node
  std::vector<std::pair<double, uint32_t>> heavy;  // (work, context) of contexts with several devices
  for (uint32_t i = 0; i < n; ++i)
    if (!ctxs[i] || ctxs[i]->server) return fail_ctx(ctxs[i], IGS_ERR_STATE, "a served context cannot be batch-lowered");
  for (uint32_t i = 0; i < n; ++i) {
    igs_ctx* x = ctxs[i];
    int r = upload_prog(x);
    if (r) return r;
    if (cudaStreamSynchronize(x->stream) != cudaSuccess) return IGS_ERR_CUDA;
    double w = 0;
    for (size_t k = x->nodes_host[0].cursor; k < x->items.size(); ++k) {
      w += 1;
      if (x->items[k].kind == IT_TASK) {
        const igs_task& t = x->tasks[x->items[k].task];
        const double chunks = (double)(t.num_chunks & 0xFFFFu) * std::max(1u, t.num_chunks >> 16);
        w += chunks * t.num_accessors / x->N;
      }
    }
    for (uint32_t k = 0; k < x->N; ++k) {
      units.push_back(Unit{x->d_nodes + k, x->d_prog});
      work.push_back(w);
    }
    if (x->D > 1) heavy.push_back({w, i});
  }
  if (warps > 1 && shape->helped) {
    std::stable_sort(heavy.begin(), heavy.end(), [](const auto& a, const auto& b) { return a.first > b.first; });
    for (size_t h = 0; h < heavy.size() && h < shape->helped; ++h) {
      int r = ensure_helpers(ctxs[heavy[h].second]);
      if (r) return r;
    }
  }
  static thread_local Unit* d_units = nullptr;
  static thread_local uint32_t* d_order = nullptr;  // followed by the queue head
  static thread_local size_t cap_units = 0;
  if (units.size() > cap_units) {
    if (d_units) cudaFree(d_units);
    if (d_order) cudaFree(d_order);
    d_units = nullptr;
    d_order = nullptr;
    cap_units = units.size() * 2;
    if (cudaMalloc(&d_units, sizeof(Unit) * cap_units) != cudaSuccess ||
        cudaMalloc(&d_order, sizeof(uint32_t) * (cap_units + 1)) != cudaSuccess)
      return fail_ctx(c, IGS_ERR_CUDA, "alloc units");
  }
  CK(cudaMemcpyAsync(d_units, units.data(), sizeof(Unit) * units.size(), cudaMemcpyHostToDevice, c->stream));
  const uint32_t nu = (uint32_t)units.size();
  if (queue) {
    // the device work queue: unit order, then the head the blocks advance
    std::vector<uint32_t> order(nu + 1);
    for (uint32_t u = 0; u < nu; ++u) order[u] = u;
    if (shape->order == IGS_ORDER_LONGEST_FIRST)
      std::stable_sort(order.begin(), order.begin() + nu, [&](uint32_t a, uint32_t b) { return work[a] > work[b]; });
    order[nu] = 0;
    CK(cudaMemcpyAsync(d_order, order.data(), sizeof(uint32_t) * (nu + 1), cudaMemcpyHostToDevice, c->stream));
    const uint32_t blocks = std::min(shape->persistent_blocks, nu);
    if (igs_launch_lower_queue(d_units, nu, d_order, d_order + nu, blocks, warps, c->stream))
      return fail_ctx(c, IGS_ERR_CUDA, "batch launch");
  } else if (igs_launch_lower(d_units, nu, IGS_NONE, c->stream)) {
    return fail_ctx(c, IGS_ERR_CUDA, "batch launch");
  }
  CK(cudaStreamSynchronize(c->stream));
  for (uint32_t i = 0; i < n; ++i) {
    ctxs[i]->launches++;
    int r = check_status(ctxs[i]);
    if (r && r != IGS_ERR_OVERLAPPING_WRITE) return fail_ctx(c, r, "context " + std::to_string(i) + ": " + ctxs[i]->err);
  }
  return IGS_OK;
}

int igs_rejected_tasks(igs_ctx* c, uint64_t* seqs, uint32_t cap, uint32_t* count) {
  if (!c || !count) return IGS_ERR_INVALID_ARG;
  int r = download_nodes(c);
  if (r) return r;
  const NodeDev& nd = c->nodes_host[0];
  *count = nd.n_rej;
  std::vector<uint32_t> tmp(nd.n_rej);
  if (nd.n_rej) CK(cudaMemcpy(tmp.data(), nd.rejected, sizeof(uint32_t) * nd.n_rej, cudaMemcpyDeviceToHost));
  for (uint32_t i = 0; i < nd.n_rej && i < cap; ++i) seqs[i] = tmp[i];
  return IGS_OK;
}

int igs_fetch_instructions(igs_ctx* c, igs_graph_view* v) {
  if (!c || !v || v->node >= c->N) return fail_ctx(c, IGS_ERR_INVALID_ARG, "bad view");
  if (c->server) return fail_ctx(c, IGS_ERR_STATE, "detach the context from its server first");
  int r = download_nodes(c);
  if (r) return r;
  const NodeDev& nd = c->nodes_host[v->node];
  v->num_instrs = nd.n_instr;
  v->num_edges = nd.n_edge;
  v->num_boxes = nd.n_box;
  v->num_binds = nd.n_bind;
  v->num_diags = nd.n_diag;
  if (v->instr_cap < nd.n_instr || v->edge_cap < nd.n_edge || v->box_cap < nd.n_box || v->bind_cap < nd.n_bind ||
      v->diag_cap < nd.n_diag)
    return IGS_ERR_TRUNCATED;
  if (nd.n_instr) CK(cudaMemcpyAsync(v->instrs, nd.instrs, sizeof(igs_instruction) * nd.n_instr, cudaMemcpyDeviceToHost, c->stream));
  if (nd.n_edge) CK(cudaMemcpyAsync(v->edges, nd.edges, sizeof(igs_edge) * nd.n_edge, cudaMemcpyDeviceToHost, c->stream));
  if (nd.n_box) CK(cudaMemcpyAsync(v->boxes, nd.boxes, sizeof(igs_box) * nd.n_box, cudaMemcpyDeviceToHost, c->stream));
  if (nd.n_bind) CK(cudaMemcpyAsync(v->binds, nd.binds, sizeof(igs_binding) * nd.n_bind, cudaMemcpyDeviceToHost, c->stream));
  if (nd.n_diag) CK(cudaMemcpyAsync(v->diags, nd.diags, sizeof(igs_diag) * nd.n_diag, cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  return IGS_OK;
}

int igs_counters(igs_ctx* c, uint64_t out[8]) {
  if (!c || !out) return IGS_ERR_INVALID_ARG;
  int r = download_nodes(c);
  if (r) return r;
  std::memset(out, 0, sizeof(uint64_t) * 8);
  for (const NodeDev& nd : c->nodes_host) {
    out[0] += nd.n_instr;
    out[1] += nd.n_edge;
    out[2] += nd.n_box;
    out[3] += nd.map_reads;
    out[4] += nd.map_writes;
  }
  out[5] = c->launches;
  return IGS_OK;
}

}  // extern "C"

// ---- executor ----------------------------------------------------------------

namespace {

// Work of one execute call, by topological level: an instruction's level is
// one more than the highest level among its predecessors if it launches work
// (copies, receives, kernels), equal to it otherwise (allocs, sends, horizons,
// epochs). Instructions of one level are mutually independent, so every level
// costs at most one box-copy launch, one stencil launch and one workload
// launch; frees follow the launches of their level.
struct LevelWork {
  std::vector<CopyJob> copies;
  std::vector<KernelJob> kernels, stencils;
  std::vector<void*> frees;
  uint64_t copy_units = 0, kernel_items = 0, stencil_max = 0;
};

// The dataflow graph of one execute call: a node per walked instruction, its
// copy or kernel jobs, (predecessor, successor) pairs, deferred frees.
struct FlowBuild {
  uint32_t oob_first = 0;  // first out-of-bounds slot of this call
  std::vector<FlowNode> nodes;
  std::vector<std::pair<uint32_t, uint32_t>> edges;
  std::vector<CopyJob> copies;
  std::vector<KernelJob> kernels;
  std::vector<void*> frees;
  uint32_t add_node(uint32_t kind) {
    FlowNode f{};
    f.kind = kind;
    f.first = (uint32_t)(kind == FK_COPY ? copies.size() : kernels.size());
    nodes.push_back(f);
    return (uint32_t)nodes.size() - 1;
  }
  // appends a copy job to node F (the last node added); tiles counts units so far
  void add_copy(uint32_t F, CopyJob J) {
    FlowNode& f = nodes[F];
    J.unit_begin = f.tiles;
    const uint64_t segs = (J.extent[2] + J.seg_bytes - 1) / J.seg_bytes;
    f.tiles += (uint32_t)((uint64_t)J.extent[0] * J.extent[1] * segs);
    copies.push_back(J);
    f.count++;
  }
};

struct Pending {
  FlowBuild* flow = nullptr;  // set: build the dataflow graph instead of levels
  uint32_t oob_first = 0;     // first out-of-bounds slot of this call
  std::vector<LevelWork> levels;
  LevelWork& at(uint32_t L) {
    if (levels.size() <= L) levels.resize(L + 1);
    return levels[L];
  }
};

// Collapses a box copy between two row-major allocations into rows of
// contiguous bytes.
bool make_copy_job(const uint8_t* src, const uint32_t slo[3], const uint32_t shi[3], uint8_t* dst, const uint32_t dlo[3],
                   const uint32_t dhi[3], const igs_box& b, uint32_t elem, CopyJob& J) {
  uint64_t e[3], ss[3], ds[3];
  for (int d = 0; d < 3; ++d) {
    if (b.lo[d] >= b.hi[d]) return false;
    // the box must lie inside both allocations
    if (b.lo[d] < slo[d] || b.hi[d] > shi[d] || b.lo[d] < dlo[d] || b.hi[d] > dhi[d]) return false;
    e[d] = b.hi[d] - b.lo[d];
  }
  ss[2] = elem;
  ds[2] = elem;
  ss[1] = ss[2] * (shi[2] - slo[2]);
  ds[1] = ds[2] * (dhi[2] - dlo[2]);
  ss[0] = ss[1] * (shi[1] - slo[1]);
  ds[0] = ds[1] * (dhi[1] - dlo[1]);
  const uint64_t soff = (b.lo[0] - slo[0]) * ss[0] + (b.lo[1] - slo[1]) * ss[1] + (b.lo[2] - slo[2]) * ss[2];
  const uint64_t doff = (b.lo[0] - dlo[0]) * ds[0] + (b.lo[1] - dlo[1]) * ds[1] + (b.lo[2] - dlo[2]) * ds[2];
  // contiguous run: innermost dims while the box spans both allocations fully
  uint64_t run = e[2] * elem;
  int outer = 1;  // dims [0, outer] remain as rows
  if (e[2] == shi[2] - slo[2] && e[2] == dhi[2] - dlo[2]) {
    run *= e[1];
    outer = 0;
    if (e[1] == shi[1] - slo[1] && e[1] == dhi[1] - dlo[1]) {
      run *= e[0];
      outer = -1;
    }
  }
  J.src = src + soff;
  J.dst = dst + doff;
  if (outer == 1) {
    J.extent[0] = (uint32_t)e[0];
    J.extent[1] = (uint32_t)e[1];
    J.src_stride[0] = ss[0];
    J.src_stride[1] = ss[1];
    J.dst_stride[0] = ds[0];
    J.dst_stride[1] = ds[1];
  } else if (outer == 0) {
    J.extent[0] = (uint32_t)e[0];
    J.extent[1] = 1;
    J.src_stride[0] = ss[0];
    J.dst_stride[0] = ds[0];
    J.src_stride[1] = J.dst_stride[1] = 0;
  } else {
    J.extent[0] = J.extent[1] = 1;
    J.src_stride[0] = J.dst_stride[0] = J.src_stride[1] = J.dst_stride[1] = 0;
  }
  // very long runs are split into rows of at most 1 GiB to keep 32-bit lengths
  J.extent[2] = (uint32_t)std::min<uint64_t>(run, 1ull << 30);
  if (run > (1ull << 30)) return false;
  J.seg_bytes = 64 * 1024;
  return true;
}

// Appends a copy job to level L's box-copy launch (its work units follow the level's earlier jobs).
void add_copy(Pending& p, uint32_t L, const CopyJob& J) {
  LevelWork& w = p.at(L);
  CopyJob j = J;
  j.unit_begin = w.copy_units;
  const uint64_t segs = (j.extent[2] + j.seg_bytes - 1) / j.seg_bytes;
  w.copy_units += (uint64_t)j.extent[0] * j.extent[1] * segs;
  w.copies.push_back(j);
}

void add_kernel(Pending& p, uint32_t L, KernelJob J, uint64_t items, bool stencil) {
  LevelWork& w = p.at(L);
  if (stencil) {
    w.stencils.push_back(J);
    w.stencil_max = std::max(w.stencil_max, items);
    return;
  }
  J.item_begin = w.kernel_items;
  w.kernel_items += items;
  w.kernels.push_back(J);
}

// Stream-ordered growth of a device array whose contents need not survive
// (no device-wide synchronization, unlike cudaFree).
template <class T>
int grow_device_async(igs_ctx* c, T*& ptr, uint32_t& cap, size_t need, cudaStream_t s) {
  if (need <= cap) return IGS_OK;
  const uint32_t ncap = (uint32_t)std::max<size_t>(need, std::max<size_t>(4096, (size_t)cap * 2));
  if (ptr) CK(cudaFreeAsync(ptr, s));
  ptr = nullptr;
  CK(cudaMallocAsync((void**)&ptr, sizeof(T) * (size_t)ncap, s));
  cap = ncap;
  return IGS_OK;
}

template <class T>
int grow_pinned(igs_ctx* c, T*& ptr, uint32_t& cap, size_t need) {
  if (need <= cap) return IGS_OK;
  const uint32_t ncap = (uint32_t)std::max<size_t>(need, std::max<size_t>(4096, (size_t)cap * 2));
  if (ptr) c->retired_pinned.push_back(ptr);
  ptr = nullptr;
  CK(cudaHostAlloc((void**)&ptr, sizeof(T) * (size_t)ncap, cudaHostAllocDefault));
  cap = ncap;
  return IGS_OK;
}

// Allocates (zeroed, on stream s) the out-of-bounds records of kernel job
// slots [first, c->oob_meta.size()) and points every accessor of the given
// jobs at its record.
int oob_prepare(igs_ctx* c, KernelJob* jobs, size_t n, uint32_t first, cudaStream_t s) {
  const uint32_t count = (uint32_t)c->oob_meta.size() - first;
  if (count == 0 || n == 0) return IGS_OK;
  const size_t words = (size_t)count * IGS_MAX_ACCESSORS * kOobWords;
  uint32_t* rec = nullptr;
  CK(cudaMallocAsync((void**)&rec, words * sizeof(uint32_t), s));
  CK(cudaMemsetAsync(rec, 0, words * sizeof(uint32_t), s));
  for (size_t j = 0; j < n; ++j)
    for (uint32_t a = 0; a < IGS_MAX_ACCESSORS; ++a)
      jobs[j].acc[a].oob = rec + ((size_t)(jobs[j].oob_slot - first) * IGS_MAX_ACCESSORS + a) * kOobWords;
  c->oob_keep.push_back(OobKeep{rec, first, count});
  return IGS_OK;
}

// Reads back the out-of-bounds records of completed calls into c->bounds.
int oob_collect(igs_ctx* c) {
  for (const OobKeep& k : c->oob_keep) {
    std::vector<uint32_t> h((size_t)k.count * IGS_MAX_ACCESSORS * kOobWords);
    CK(cudaMemcpy(h.data(), k.rec, h.size() * sizeof(uint32_t), cudaMemcpyDeviceToHost));
    CK(cudaFree(k.rec));
    for (uint32_t i = 0; i < k.count; ++i) {
      const OobMeta& m = c->oob_meta[k.first + i];
      for (uint32_t a = 0; a < m.nacc && a < IGS_MAX_ACCESSORS; ++a) {
        const uint32_t* w = h.data() + ((size_t)i * IGS_MAX_ACCESSORS + a) * kOobWords;
        if (!w[3]) continue;
        igs_bounds_error e{};
        e.seq = m.seq;
        e.node = m.node;
        e.chunk = m.chunk;
        e.accessor = a;
        for (int d = 0; d < 3; ++d) {
          e.lo[d] = ~w[d];
          e.hi[d] = w[3 + d];
        }
        c->bounds.push_back(e);
        c->oob_pending = true;
      }
    }
  }
  c->oob_keep.clear();
  return IGS_OK;
}

// IGS_ERR_OUT_OF_BOUNDS once per execute / run that met accessor violations.
int oob_status(igs_ctx* c) {
  if (!c->oob_pending) return IGS_OK;
  c->oob_pending = false;
  return fail_ctx(c, IGS_ERR_OUT_OF_BOUNDS,
                  "a kernel accessed elements outside its accessor's range-mapper box (igs_bounds_errors lists them)");
}

// Reads and clears the execution error flags (after the stream has completed).
int exec_error_status(igs_ctx* c) {
  const int ro = oob_collect(c);
  if (ro) return ro;
  const int e = igs_exec_error(true);
  if (e < 0) return fail_ctx(c, IGS_ERR_CUDA, "reading the execution error flags");
  if (e & 2) return fail_ctx(c, IGS_ERR_TIMEOUT, "the dataflow executor saw no tile finish for 2 s and gave up");
  if (e & 1) return fail_ctx(c, IGS_ERR_STATE, "a workload kernel accessed outside its allocation");
  return IGS_OK;
}

// Uploads every job once and launches level by level on stream s. The job
// arrays alternate between two sets; with wait == false the call returns
// once everything is enqueued.
int run_pending(igs_ctx* c, Pending& p, cudaStream_t s, bool wait) {
  const int k = c->jobs_set;
  c->jobs_set ^= 1;
  if (!c->jobs_done[k]) CK(cudaEventCreateWithFlags(&c->jobs_done[k], cudaEventDisableTiming));
  CK(cudaEventSynchronize(c->jobs_done[k]));  // the set's previous launches are done
  size_t ncj = 0, nkj = 0;
  for (const LevelWork& w : p.levels) {
    ncj += w.copies.size();
    nkj += w.kernels.size() + w.stencils.size();
  }
  std::vector<size_t> co(p.levels.size()), ko(p.levels.size()), so(p.levels.size());
  int r;
  if ((r = grow_pinned(c, c->h_cjobs[k], c->hcap_cjobs[k], std::max<size_t>(ncj, 1)))) return r;
  if ((r = grow_pinned(c, c->h_kjobs[k], c->hcap_kjobs[k], std::max<size_t>(nkj, 1)))) return r;
  size_t nc = 0, nk = 0;
  for (size_t L = 0; L < p.levels.size(); ++L) {
    const LevelWork& w = p.levels[L];
    co[L] = nc;
    std::copy(w.copies.begin(), w.copies.end(), c->h_cjobs[k] + nc);
    nc += w.copies.size();
    ko[L] = nk;
    std::copy(w.kernels.begin(), w.kernels.end(), c->h_kjobs[k] + nk);
    nk += w.kernels.size();
    so[L] = nk;
    std::copy(w.stencils.begin(), w.stencils.end(), c->h_kjobs[k] + nk);
    nk += w.stencils.size();
  }
  if ((r = oob_prepare(c, c->h_kjobs[k], nk, p.oob_first, s))) return r;
  if (nc) {
    if ((r = grow_device_async(c, c->d_cjobs[k], c->cap_cjobs[k], nc, s))) return r;
    CK(cudaMemcpyAsync(c->d_cjobs[k], c->h_cjobs[k], sizeof(CopyJob) * nc, cudaMemcpyHostToDevice, s));
  }
  if (nk) {
    if ((r = grow_device_async(c, c->d_kjobs[k], c->cap_kjobs[k], nk, s))) return r;
    CK(cudaMemcpyAsync(c->d_kjobs[k], c->h_kjobs[k], sizeof(KernelJob) * nk, cudaMemcpyHostToDevice, s));
  }
  for (size_t L = 0; L < p.levels.size(); ++L) {
    LevelWork& w = p.levels[L];
    // a level with both copies and stencil jobs runs as one launch (its
    // instructions are independent of one another); its time counts as
    // workload time and its copy bytes are not in copy_bytes
    if (!w.copies.empty() && !w.stencils.empty() && w.stencils.size() + 2048 <= 65535) {
      const size_t ev = c->timing ? ev_begin(c, s) : 0;
      if (igs_launch_level(c->d_kjobs[k] + so[L], (uint32_t)w.stencils.size(), w.stencil_max, c->d_cjobs[k] + co[L],
                           (uint32_t)w.copies.size(), w.copy_units, s))
        return fail_ctx(c, IGS_ERR_CUDA, "level launch");
      if (c->timing) ev_end(c, 2, ev, s);
      c->n_launch[2]++;
    } else {
      if (!w.copies.empty()) {
        const size_t ev = c->timing ? ev_begin(c, s) : 0;
        if (igs_launch_copies(c->d_cjobs[k] + co[L], (uint32_t)w.copies.size(), w.copy_units, s))
          return fail_ctx(c, IGS_ERR_CUDA, "box copy launch");
        if (c->timing) ev_end(c, 1, ev, s);
        c->n_launch[1]++;
        for (const CopyJob& j : w.copies) c->copy_bytes += 2.0 * j.extent[0] * j.extent[1] * j.extent[2];
      }
      for (size_t first = 0; first < w.stencils.size(); first += 65535) {
        const uint32_t n = (uint32_t)std::min<size_t>(65535, w.stencils.size() - first);
        const size_t ev = c->timing ? ev_begin(c, s) : 0;
        if (igs_launch_stencil(c->d_kjobs[k] + so[L] + first, n, w.stencil_max, s))
          return fail_ctx(c, IGS_ERR_CUDA, "stencil launch");
        if (c->timing) ev_end(c, 2, ev, s);
        c->n_launch[2]++;
      }
    }
    if (!w.kernels.empty()) {
      const size_t ev = c->timing ? ev_begin(c, s) : 0;
      if (igs_launch_workload(c->d_kjobs[k] + ko[L], (uint32_t)w.kernels.size(), w.kernel_items, s))
        return fail_ctx(c, IGS_ERR_CUDA, "workload launch");
      if (c->timing) ev_end(c, 2, ev, s);
      c->n_launch[2]++;
    }
    for (void* f : w.frees) CK(cudaFreeAsync(f, s));
  }
  CK(cudaEventRecord(c->jobs_done[k], s));
  p.levels.clear();
  if (!wait) return IGS_OK;
  CK(cudaStreamSynchronize(s));
  ev_collect(c);
  return exec_error_status(c);
}

int run_flow(igs_ctx* c, FlowBuild& g, cudaStream_t s, bool wait);

// Runs what the walk collected, on the executor the context uses.
int run_walk(igs_ctx* c, Pending& p, cudaStream_t s, bool wait) {
  return p.flow ? run_flow(c, *p.flow, s, wait) : run_pending(c, p, s, wait);
}

// Length of the union of intervals (sorted in place).
double union_ns(std::vector<std::pair<uint64_t, uint64_t>>& v) {
  std::sort(v.begin(), v.end());
  double total = 0;
  uint64_t lo = 0, hi = 0;
  bool open = false;
  for (const auto& x : v) {
    if (!open || x.first > hi) {
      if (open) total += (double)(hi - lo);
      lo = x.first;
      hi = x.second;
      open = true;
    } else {
      hi = std::max(hi, x.second);
    }
  }
  if (open) total += (double)(hi - lo);
  return total;
}

// Reads back the node timestamps of kept dataflow launches (their streams
// have completed) and adds span, copy-busy, kernel-busy and overlap times.
int flow_collect(igs_ctx* c) {
  for (const FlowKeep& f : c->flow_keep) {
    std::vector<FlowNode> nodes(f.n_nodes);
    CK(cudaMemcpy(nodes.data(), (uint8_t*)f.arena + f.off_nodes, sizeof(FlowNode) * f.n_nodes, cudaMemcpyDeviceToHost));
    CK(cudaFree(f.arena));
    std::vector<std::pair<uint64_t, uint64_t>> cp, kn, all;
    uint64_t t0 = ~0ull, t1 = 0;
    for (const FlowNode& n : nodes) {
      if (n.kind == FK_NONE || n.t_end < n.t_start) continue;
      (n.kind == FK_COPY ? cp : kn).push_back({n.t_start, n.t_end});
      all.push_back({n.t_start, n.t_end});
      t0 = std::min<uint64_t>(t0, n.t_start);
      t1 = std::max<uint64_t>(t1, n.t_end);
    }
    const double uc = union_ns(cp), uk = union_ns(kn), ua = union_ns(all);
    if (t1 > t0) c->flow_stats[4] += (double)(t1 - t0) * 1e-6;
    c->flow_stats[5] += uc * 1e-6;
    c->flow_stats[6] += uk * 1e-6;
    c->flow_stats[7] += (uc + uk - ua) * 1e-6;
  }
  c->flow_keep.clear();
  return IGS_OK;
}

// Lays the dataflow graph out in one device arena (control block, nodes,
// successor CSR, predecessor counts, claim / finish counters, ready queue,
// jobs), uploads it and launches it on stream s; frees follow the launch.
int run_flow(igs_ctx* c, FlowBuild& g, cudaStream_t s, bool wait) {
  const uint32_t n = (uint32_t)g.nodes.size();
  if (n == 0) {
    for (void* f : g.frees) CK(cudaFreeAsync(f, s));
    return IGS_OK;
  }
  std::vector<uint32_t> pend(n, 0), off(n + 1, 0);
  for (const auto& e : g.edges) {
    off[e.first + 1]++;
    pend[e.second]++;
  }
  for (uint32_t i = 0; i < n; ++i) off[i + 1] += off[i];
  uint64_t tiles = 0;
  for (uint32_t i = 0; i < n; ++i) {
    FlowNode& f = g.nodes[i];
    f.succ_off = off[i];
    f.succ_cnt = off[i + 1] - off[i];
    if (f.kind == FK_COPY && f.count == 0) f.kind = FK_NONE;
    if (f.kind == FK_STENCIL) {
      const KernelJob& J = g.kernels[f.first];
      const uint32_t strips = ((J.hi[1] - J.lo[1] + 3) / 4 + kFlowThreads - 1) / kFlowThreads;
      f.tiles = strips * ((J.hi[0] - J.lo[0] + kFlowStencilRows - 1) / kFlowStencilRows);
    } else if (f.kind == FK_WORKLOAD) {
      const KernelJob& J = g.kernels[f.first];
      const uint64_t items = (uint64_t)(J.hi[0] - J.lo[0]) * (J.hi[1] - J.lo[1]) * (J.hi[2] - J.lo[2]);
      f.tiles = J.kernel == K_NBODY_STEP ? (J.hi[0] - J.lo[0] + kFlowBodies - 1) / kFlowBodies
                                         : (uint32_t)((items + kFlowItems - 1) / kFlowItems);
    } else if (f.kind == FK_NONE) {
      f.tiles = 1;
    }
    if (f.tiles == 0) {
      f.kind = FK_NONE;
      f.tiles = 1;
    }
    f.t_start = f.t_end = 0;
    tiles += f.tiles;
  }
  const uint32_t m = (uint32_t)g.edges.size();
  auto al = [](size_t x) { return (x + 15) & ~size_t(15); };
  const size_t o_ctl = 0, o_nodes = al(sizeof(FlowCtl)), o_succ = al(o_nodes + sizeof(FlowNode) * n),
               o_pend = al(o_succ + 4ull * std::max(m, 1u)), o_claim = al(o_pend + 4ull * n),
               o_fin = al(o_claim + 4ull * n), o_ready = al(o_fin + 4ull * n), o_cj = al(o_ready + 4ull * n),
               o_kj = al(o_cj + sizeof(CopyJob) * g.copies.size()), total = al(o_kj + sizeof(KernelJob) * g.kernels.size());
  const int k = c->jobs_set;
  c->jobs_set ^= 1;
  if (!c->jobs_done[k]) CK(cudaEventCreateWithFlags(&c->jobs_done[k], cudaEventDisableTiming));
  CK(cudaEventSynchronize(c->jobs_done[k]));  // the set's staging is free again
  if (c->hcap_flow[k] < total) {
    if (c->h_flow[k]) c->retired_pinned.push_back(c->h_flow[k]);
    c->h_flow[k] = nullptr;
    c->hcap_flow[k] = std::max(total, std::max<size_t>(2 * c->hcap_flow[k], 4u << 20));
    CK(cudaHostAlloc((void**)&c->h_flow[k], c->hcap_flow[k], cudaHostAllocDefault));
  }
  uint8_t* H = c->h_flow[k];
  std::memset(H, 0, o_succ);
  FlowCtl* ctl = reinterpret_cast<FlowCtl*>(H + o_ctl);
  std::memcpy(H + o_nodes, g.nodes.data(), sizeof(FlowNode) * n);
  uint32_t* succ = reinterpret_cast<uint32_t*>(H + o_succ);
  {
    std::vector<uint32_t> pos(off.begin(), off.end() - 1);
    for (const auto& e : g.edges) succ[pos[e.first]++] = e.second;
  }
  std::memcpy(H + o_pend, pend.data(), 4ull * n);
  std::memset(H + o_claim, 0, o_ready - o_claim);
  uint32_t* ready = reinterpret_cast<uint32_t*>(H + o_ready);
  uint32_t nready = 0;
  for (uint32_t i = 0; i < n; ++i)
    if (pend[i] == 0) ready[nready++] = i;
  for (uint32_t i = nready; i < n; ++i) ready[i] = 0xFFFFFFFFu;
  if (nready == 0) return fail_ctx(c, IGS_ERR_STATE, "dataflow graph without a ready node");
  ctl->tail = nready;
  if (!g.copies.empty()) std::memcpy(H + o_cj, g.copies.data(), sizeof(CopyJob) * g.copies.size());
  int ro = oob_prepare(c, g.kernels.data(), g.kernels.size(), g.oob_first, s);
  if (ro) return ro;
  if (!g.kernels.empty()) std::memcpy(H + o_kj, g.kernels.data(), sizeof(KernelJob) * g.kernels.size());
  uint8_t* D = nullptr;
  CK(cudaMallocAsync((void**)&D, total, s));
  CK(cudaMemcpyAsync(D, H, total, cudaMemcpyHostToDevice, s));
  CK(cudaEventRecord(c->jobs_done[k], s));
  const size_t ev = c->timing ? ev_begin(c, s) : 0;
  if (igs_launch_flow(reinterpret_cast<FlowCtl*>(D + o_ctl), reinterpret_cast<FlowNode*>(D + o_nodes), n,
                      reinterpret_cast<uint32_t*>(D + o_succ), reinterpret_cast<uint32_t*>(D + o_pend),
                      reinterpret_cast<uint32_t*>(D + o_claim), reinterpret_cast<uint32_t*>(D + o_fin),
                      reinterpret_cast<uint32_t*>(D + o_ready), reinterpret_cast<CopyJob*>(D + o_cj),
                      reinterpret_cast<KernelJob*>(D + o_kj), 2000000000ull, s))
    return fail_ctx(c, IGS_ERR_CUDA, "dataflow launch");
  if (c->timing) ev_end(c, 2, ev, s);
  c->n_launch[2]++;
  for (const CopyJob& j : g.copies) c->copy_bytes += 2.0 * j.extent[0] * j.extent[1] * j.extent[2];
  c->flow_stats[0] += 1;
  c->flow_stats[1] += n;
  c->flow_stats[2] += (double)tiles;
  c->flow_stats[3] += m;
  if (c->timing) c->flow_keep.push_back(FlowKeep{D, o_nodes, n});
  else CK(cudaFreeAsync(D, s));
  for (void* f : g.frees) CK(cudaFreeAsync(f, s));
  if (!wait) return IGS_OK;
  CK(cudaStreamSynchronize(s));
  ev_collect(c);
  int r = flow_collect(c);
  if (r) return r;
  return exec_error_status(c);
}

ExecAlloc* get_alloc(igs_ctx* c, uint32_t node, uint32_t aid, uint32_t buffer_hint) {
  auto& m = c->nh[node].allocs;
  auto it = m.find(aid);
  if (it != m.end()) return &it->second;
  // a user allocation (M0): host data of the buffer
  if (buffer_hint >= c->bufs.size() || !c->init_dev[buffer_hint]) return nullptr;
  ExecAlloc a;
  a.ptr = c->init_dev[buffer_hint];
  a.buffer = buffer_hint;
  a.mem = 0;
  for (int d = 0; d < 3; ++d) {
    a.lo[d] = 0;
    a.hi[d] = c->bufs[buffer_hint].extent[d];
  }
  a.live = true;
  a.user = true;
  return &(m[aid] = a);
}

// Brings node n's records up to the given counts to the host (on stream s,
// which is then synchronized).
int fetch_node(igs_ctx* c, uint32_t n, uint32_t ni, uint32_t ne, uint32_t nbx, uint32_t nbd, cudaStream_t s) {
  const NodeDev& nd = c->nodes_host[n];
  NodeHost& h = c->nh[n];
  const size_t oi = h.instrs.size(), oe = h.edges.size(), ob = h.boxes.size(), ok = h.binds.size();
  if (ni < oi || ne < oe || nbx < ob || nbd < ok) return fail_ctx(c, IGS_ERR_STATE, "graph counts went back");
  h.instrs.resize(ni);
  h.edges.resize(ne);
  h.boxes.resize(nbx);
  h.binds.resize(nbd);
  if (ni > oi)
    CK(cudaMemcpyAsync(h.instrs.data() + oi, nd.instrs + oi, sizeof(igs_instruction) * (ni - oi), cudaMemcpyDeviceToHost, s));
  if (ne > oe)
    CK(cudaMemcpyAsync(h.edges.data() + oe, nd.edges + oe, sizeof(igs_edge) * (ne - oe), cudaMemcpyDeviceToHost, s));
  if (nbx > ob)
    CK(cudaMemcpyAsync(h.boxes.data() + ob, nd.boxes + ob, sizeof(igs_box) * (nbx - ob), cudaMemcpyDeviceToHost, s));
  if (nbd > ok)
    CK(cudaMemcpyAsync(h.binds.data() + ok, nd.binds + ok, sizeof(igs_binding) * (nbd - ok), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  h.first_edge.resize(ni + 1, 0);
  h.level.resize(ni, 0);
  // edges are grouped by successor in emission order
  size_t e = oe;
  for (uint32_t i = (uint32_t)oi; i < ni; ++i) {
    while (e < h.edges.size() && h.edges[e].to < i) ++e;
    h.first_edge[i] = (uint32_t)e;
  }
  h.first_edge[ni] = (uint32_t)h.edges.size();
  return IGS_OK;
}

int fetch_for_exec(igs_ctx* c) {
  int r = download_nodes(c);
  if (r) return r;
  for (uint32_t n = 0; n < c->N; ++n) {
    const NodeDev& nd = c->nodes_host[n];
    if ((r = fetch_node(c, n, nd.n_instr, nd.n_edge, nd.n_box, nd.n_bind, c->stream))) return r;
  }
  return IGS_OK;
}

uint32_t pred_level(const NodeHost& h, uint32_t id) {
  uint32_t L = 0;
  for (uint32_t e = h.first_edge[id]; e < h.first_edge[id + 1]; ++e) L = std::max(L, h.level[h.edges[e].from]);
  return L;
}

bool box_in(const uint32_t lo[3], const uint32_t hi[3], const uint32_t blo[3], const uint32_t bhi[3]) {
  for (int d = 0; d < 3; ++d)
    if (blo[d] < lo[d] || bhi[d] > hi[d]) return false;
  return true;
}

// A Jacobi / wave chunk whose allocations cover what the stencil touches can
// run on the vectorized stencil kernel.
bool stencil_ok(const igs_ctx* c, const KernelJob& J) {
  if (J.kernel != K_JACOBI && J.kernel != K_WAVE) return false;
  const uint32_t nu = J.kernel == K_WAVE ? 1 : 0, no = J.kernel == K_WAVE ? 2 : 1;
  if (J.nacc != no + 1) return false;
  for (uint32_t a = 0; a < J.nacc; ++a)
    if (!J.acc[a].valid || J.acc[a].elem != 4 || J.acc[a].dims != 2) return false;
  const KAcc& U = J.acc[nu];
  uint32_t lo[3], hi[3];
  for (int d = 0; d < 3; ++d) {
    lo[d] = J.lo[d];
    hi[d] = J.hi[d];
  }
  // the fast kernels do not check single accesses: the allocations AND the
  // boxes the range mappers permit must cover everything they touch
  if (!box_in(J.acc[no].lo, J.acc[no].hi, lo, hi) || !box_in(J.acc[no].plo, J.acc[no].phi, lo, hi)) return false;
  if (J.kernel == K_WAVE && (!box_in(J.acc[0].lo, J.acc[0].hi, lo, hi) || !box_in(J.acc[0].plo, J.acc[0].phi, lo, hi)))
    return false;
  for (int d = 0; d < 2; ++d) {
    lo[d] = lo[d] > 0 ? lo[d] - 1 : 0;
    hi[d] = std::min(hi[d] + 1, U.ext[d]);
  }
  return box_in(U.lo, U.hi, lo, hi) && box_in(U.plo, U.phi, lo, hi);
}

// One walk over the fetched, not yet executed instructions of every node,
// by submission sequence; within one, every node's part up to its first
// receive, then the rest (sends precede the matching receives). A receive
// whose sends have not all been carried out stops its node for this walk.
// Sets *halted_any when some node stopped early.
int exec_walk(igs_ctx* c, Pending& p, cudaStream_t xs, bool* halted_any, bool* progress) {
  c->exec_call += 1;
  FlowBuild* g = p.flow;
  p.oob_first = (uint32_t)c->oob_meta.size();
  if (g) g->oob_first = p.oob_first;
  std::vector<uint32_t> walk_start(c->N);
  for (uint32_t n = 0; n < c->N; ++n) {
    walk_start[n] = c->nh[n].executed;
    if (g) c->nh[n].fid.resize(c->nh[n].instrs.size());
  }
  // per split receive of this call: (send box, its copy node)
  std::unordered_map<uint64_t, std::vector<std::pair<igs_box, uint32_t>>> split_parts;
  // the dataflow node of instruction i of node n; its predecessors walked in
  // this call become its predecessor nodes (earlier ones have completed)
  auto flow_node = [&](uint32_t n, uint32_t i, uint32_t kind) -> uint32_t {
    NodeHost& h = c->nh[n];
    const uint32_t F = g->add_node(kind);
    for (uint32_t e = h.first_edge[i]; e < h.first_edge[i + 1]; ++e) {
      const uint32_t from = h.edges[e].from;
      if (from >= walk_start[n]) g->edges.push_back({h.fid[from], F});
    }
    h.fid[i] = F;
    return F;
  };
  std::map<uint32_t, std::vector<std::pair<uint32_t, std::pair<uint32_t, uint32_t>>>> order;
  std::vector<bool> halted(c->N, false);
  std::vector<uint32_t> stop_at(c->N, 0);
  for (uint32_t n = 0; n < c->N; ++n) {
    NodeHost& h = c->nh[n];
    std::fill(h.level.begin(), h.level.end(), 0u);  // earlier calls: complete (stream order)
    uint32_t i = h.executed;
    while (i < h.instrs.size()) {
      const uint32_t sq = h.instrs[i].seq;
      uint32_t j = i;
      while (j < h.instrs.size() && h.instrs[j].seq == sq) ++j;
      order[sq].push_back({n, {i, j}});
      i = j;
    }
  }
  auto key_of = [](uint32_t seq, uint32_t buf, uint32_t recv) { return ((uint64_t)seq << 32) | ((uint64_t)buf << 8) | recv; };
  for (auto& so : order) {
    for (int half = 0; half < 2; ++half) {
      for (auto& part : so.second) {
        const uint32_t n = part.first;
        if (halted[n]) continue;
        NodeHost& h = c->nh[n];
        uint32_t i0 = part.second.first, i1 = part.second.second, cut = i1;
        for (uint32_t i = i0; i < i1; ++i)
          if (h.instrs[i].type == IGS_RECEIVE || h.instrs[i].type == IGS_SPLIT_RECEIVE) {
            cut = i;
            break;
          }
        const uint32_t a0 = half == 0 ? i0 : cut, a1 = half == 0 ? cut : i1;
        for (uint32_t i = a0; i < a1 && !halted[n]; ++i) {
          const igs_instruction& in = h.instrs[i];
          const uint32_t L = pred_level(h, i);
          h.level[i] = L;
          switch (in.type) {
            case IGS_ALLOC: {
              const igs_box& b = h.boxes[in.box_off];
              ExecAlloc a;
              a.buffer = in.c;
              a.mem = in.b;
              uint64_t cnt = c->bufs[in.c].elem;
              for (int d = 0; d < 3; ++d) {
                a.lo[d] = b.lo[d];
                a.hi[d] = b.hi[d];
                cnt *= (b.hi[d] - b.lo[d]);
              }
              CK(cudaMallocAsync((void**)&a.ptr, cnt ? cnt : 1, xs));
              a.live = true;
              h.allocs[in.a] = a;
              if (g) flow_node(n, i, FK_NONE);
              break;
            }
            case IGS_FREE: {
              auto it = h.allocs.find(in.a);
              if (it != h.allocs.end()) {
                if (!it->second.user) {
                  if (g) g->frees.push_back(it->second.ptr);  // after the launch
                  else p.at(L).frees.push_back(it->second.ptr);
                }
                h.allocs.erase(it);
              }
              if (g) flow_node(n, i, FK_NONE);
              break;
            }
            case IGS_COPY: {
              ExecAlloc* s = get_alloc(c, n, in.a, in.c);
              ExecAlloc* d = get_alloc(c, n, in.b, in.c);
              if (!s || !d) return fail_ctx(c, IGS_ERR_STATE, "copy between unknown allocations");
              const uint32_t F = g ? flow_node(n, i, FK_COPY) : 0;
              for (uint32_t k = 0; k < in.box_cnt; ++k) {
                CopyJob J{};
                if (!make_copy_job(s->ptr, s->lo, s->hi, d->ptr, d->lo, d->hi, h.boxes[in.box_off + k], c->bufs[in.c].elem, J))
                  return fail_ctx(c, IGS_ERR_STATE, "bad copy box");
                if (g) g->add_copy(F, J);
                else add_copy(p, L + 1, J);
              }
              h.level[i] = L + 1;
              break;
            }
            case IGS_SEND: {
              // the data moves at the send: into a mailbox of its own, one
              // level after the send's predecessors
              ExecAlloc* sa = get_alloc(c, n, in.a, in.c);
              if (!sa) return fail_ctx(c, IGS_ERR_STATE, "send from unknown allocation");
              SendRec sr;
              sr.node = n;
              sr.box = h.boxes[in.box_off];
              sr.level = L + 1;
              sr.call = c->exec_call;
              const uint32_t elem = c->bufs[in.c].elem;
              uint64_t bytes = elem;
              for (int d = 0; d < 3; ++d) bytes *= sr.box.hi[d] - sr.box.lo[d];
              CK(cudaMallocAsync((void**)&sr.mail, bytes ? bytes : 1, xs));
              CopyJob J{};
              if (!make_copy_job(sa->ptr, sa->lo, sa->hi, sr.mail, sr.box.lo, sr.box.hi, sr.box, elem, J))
                return fail_ctx(c, IGS_ERR_STATE, "bad send box");
              if (g) {
                sr.fid = flow_node(n, i, FK_COPY);
                g->add_copy(sr.fid, J);
              } else {
                add_copy(p, L + 1, J);
              }
              c->sends.insert({key_of(in.seq, in.c, in.b), sr});
              h.level[i] = L + 1;
              break;
            }
            case IGS_RECEIVE:
            case IGS_SPLIT_RECEIVE: {
              // every send of this (task, buffer) to this node must have been
              // carried out; otherwise the node stops here until a later call
              auto range = c->sends.equal_range(key_of(in.seq, in.c, n));
              uint64_t need = 0, have = 0;
              for (uint32_t k = 0; k < in.box_cnt; ++k) {
                const igs_box& b = h.boxes[in.box_off + k];
                need += (uint64_t)(b.hi[0] - b.lo[0]) * (b.hi[1] - b.lo[1]) * (b.hi[2] - b.lo[2]);
              }
              for (auto it = range.first; it != range.second; ++it) {
                const igs_box& b = it->second.box;
                have += (uint64_t)(b.hi[0] - b.lo[0]) * (b.hi[1] - b.lo[1]) * (b.hi[2] - b.lo[2]);
              }
              if (have < need) {
                halted[n] = true;
                stop_at[n] = i;
                break;
              }
              uint32_t Lr = L;
              for (auto it = range.first; it != range.second; ++it)
                if (it->second.call == c->exec_call) Lr = std::max(Lr, it->second.level);
              ExecAlloc* d = get_alloc(c, n, in.a, in.c);
              if (!d) return fail_ctx(c, IGS_ERR_STATE, "receive into unknown allocation");
              uint32_t F = 0;
              if (g && in.type == IGS_SPLIT_RECEIVE) {
                // receive arbitration (Sec. 3.4 "Inbound Transfers", cases a
                // and c): one copy node per incoming send, gated by the split
                // receive's own predecessors and by that send; the split
                // receive completes with the last of them, and each await
                // receive as soon as the sends meeting its region have landed
                const uint32_t gate = flow_node(n, i, FK_NONE);  // carries the split receive's predecessors
                const uint32_t sid = g->add_node(FK_NONE);       // the split receive itself
                h.fid[i] = sid;
                auto& parts = split_parts[((uint64_t)n << 32) | i];
                for (auto it = range.first; it != range.second; ++it) {
                  const igs_box& b = it->second.box;
                  CopyJob J{};
                  if (!make_copy_job(it->second.mail, b.lo, b.hi, d->ptr, d->lo, d->hi, b, c->bufs[in.c].elem, J))
                    return fail_ctx(c, IGS_ERR_STATE, "bad receive box");
                  const uint32_t cf = g->add_node(FK_COPY);
                  g->add_copy(cf, J);
                  g->edges.push_back({gate, cf});
                  if (it->second.call == c->exec_call) g->edges.push_back({it->second.fid, cf});
                  g->edges.push_back({cf, sid});
                  g->frees.push_back(it->second.mail);
                  parts.push_back({b, cf});
                }
                c->sends.erase(range.first, range.second);
                h.level[i] = Lr + 1;
                break;
              }
              if (g) {
                F = flow_node(n, i, FK_COPY);
                for (auto it = range.first; it != range.second; ++it)
                  if (it->second.call == c->exec_call) g->edges.push_back({it->second.fid, F});
              }
              for (auto it = range.first; it != range.second; ++it) {
                const igs_box& b = it->second.box;
                CopyJob J{};
                if (!make_copy_job(it->second.mail, b.lo, b.hi, d->ptr, d->lo, d->hi, b, c->bufs[in.c].elem, J))
                  return fail_ctx(c, IGS_ERR_STATE, "bad receive box");
                if (g) {
                  g->add_copy(F, J);
                  g->frees.push_back(it->second.mail);
                } else {
                  add_copy(p, Lr + 1, J);
                  p.at(Lr + 1).frees.push_back(it->second.mail);
                }
              }
              c->sends.erase(range.first, range.second);
              h.level[i] = Lr + 1;
              break;
            }
            case IGS_KERNEL: {
              if (in.seq >= c->seq_task.size() || c->seq_task[in.seq] == NONE)
                return fail_ctx(c, IGS_ERR_STATE, "kernel of unknown task");
              const igs_task& t = c->tasks[c->seq_task[in.seq]];
              KernelJob J{};
              J.kernel = t.kernel_id;
              J.seq = in.seq;
              J.nacc = t.num_accessors;
              const igs_box& cb = h.boxes[in.box_off];
              uint64_t items = 1;
              for (int d = 0; d < 3; ++d) {
                J.lo[d] = cb.lo[d];
                J.hi[d] = cb.hi[d];
                items *= (cb.hi[d] - cb.lo[d]);
              }
              for (int k = 0; k < 4; ++k) J.params[k] = t.params[k];
              for (uint32_t a = 0; a < t.num_accessors; ++a) {
                const igs_binding& bd = h.binds[in.bind_off + a];
                KAcc& A = J.acc[a];
                const BufDesc& bf = c->bufs[t.acc[a].buffer];
                A.dims = bf.dims;
                A.elem = bf.elem;
                A.mode = t.acc[a].mode;
                for (int d = 0; d < 3; ++d) {
                  A.ext[d] = bf.extent[d];
                  A.map[d] = t.acc[a].dim[d];
                }
                A.valid = 0;
                for (int d = 0; d < 3; ++d) {
                  A.plo[d] = bd.lo[d];
                  A.phi[d] = bd.hi[d];
                }
                if (bd.alloc != IGS_NONE) {
                  ExecAlloc* al = get_alloc(c, n, bd.alloc, t.acc[a].buffer);
                  if (!al) return fail_ctx(c, IGS_ERR_STATE, "kernel on unknown allocation");
                  A.ptr = al->ptr;
                  for (int d = 0; d < 3; ++d) {
                    A.lo[d] = al->lo[d];
                    A.hi[d] = al->hi[d];
                  }
                  A.valid = 1;
                }
              }
              if (J.kernel != K_NOP && items) {
                J.oob_slot = (uint32_t)c->oob_meta.size();
                c->oob_meta.push_back(OobMeta{in.seq, n, in.a, J.nacc});
              }
              if (g) {
                const bool work = J.kernel != K_NOP && items;
                flow_node(n, i, !work ? FK_NONE : stencil_ok(c, J) ? FK_STENCIL : FK_WORKLOAD);
                if (work) {
                  g->kernels.push_back(J);
                  g->nodes.back().count = 1;
                }
              } else if (J.kernel != K_NOP && items) {
                add_kernel(p, L + 1, J, items, stencil_ok(c, J));
              }
              h.level[i] = L + 1;
              break;
            }
            case IGS_AWAIT_RECEIVE: {
              if (!g) break;
              // completes once the received copies meeting its region are in
              // (instead of waiting for the whole split receive)
              const auto sp = split_parts.find(((uint64_t)n << 32) | in.b);
              if (sp == split_parts.end()) {  // split receive of an earlier call: complete
                flow_node(n, i, FK_NONE);
                break;
              }
              const uint32_t F = g->add_node(FK_NONE);
              for (uint32_t e = h.first_edge[i]; e < h.first_edge[i + 1]; ++e) {
                const uint32_t from = h.edges[e].from;
                if (from >= walk_start[n] && from != in.b) g->edges.push_back({h.fid[from], F});
              }
              bool any = false;
              for (const auto& part : sp->second)
                for (uint32_t k = 0; k < in.box_cnt; ++k) {
                  const igs_box& a = h.boxes[in.box_off + k];
                  bool meet = true;
                  for (int dd = 0; dd < 3; ++dd)
                    if (std::max(a.lo[dd], part.first.lo[dd]) >= std::min(a.hi[dd], part.first.hi[dd])) meet = false;
                  if (meet) {
                    g->edges.push_back({part.second, F});
                    any = true;
                    break;
                  }
                }
              if (!any) g->edges.push_back({h.fid[in.b], F});
              h.fid[i] = F;
              break;
            }
            default:  // horizon, epoch: no work of their own
              if (g) flow_node(n, i, FK_NONE);
              break;
          }
        }
      }
    }
  }
  *halted_any = false;
  *progress = false;
  for (uint32_t n = 0; n < c->N; ++n) {
    NodeHost& h = c->nh[n];
    const uint32_t upto = halted[n] ? stop_at[n] : (uint32_t)h.instrs.size();
    if (upto > h.executed) *progress = true;
    h.executed = upto;
    if (halted[n]) *halted_any = true;
  }
  return IGS_OK;
}

}  // namespace

extern "C" int igs_execute(igs_ctx* c, uint32_t flags) {
  if (!c) return IGS_ERR_INVALID_ARG;
  if (c->server) return fail_ctx(c, IGS_ERR_STATE, "detach the context from its server first");
  int r = fetch_for_exec(c);
  if (r) return r;
  for (;;) {
    Pending p;
    FlowBuild g;
    if (c->executor == IGS_EXEC_DATAFLOW) p.flow = &g;
    bool halted = false, progress = false;
    if ((r = exec_walk(c, p, c->stream, &halted, &progress))) return r;
    if ((r = run_walk(c, p, c->stream, true))) return r;
    if (!halted) break;
    if (!progress) break;  // a receive waits for sends not lowered yet: a later call executes it
  }
  (void)flags;
  return oob_status(c);
}

extern "C" int igs_run(igs_ctx* c, uint32_t window) {
  if (!c || window == 0) return IGS_ERR_INVALID_ARG;
  if (c->server) return fail_ctx(c, IGS_ERR_STATE, "detach the context from its server first");
  if (c->cfg.mode != IGS_MODE_BATCHED) return igs_execute(c, 0);  // already lowered at submission
  if (!c->xstream) CK(cudaStreamCreateWithFlags(&c->xstream, cudaStreamNonBlocking));
  if (!c->cstream) CK(cudaStreamCreateWithFlags(&c->cstream, cudaStreamNonBlocking));
  if (!c->m_progress) {
    CK(cudaHostAlloc((void**)&c->m_progress, sizeof(uint32_t) * PR_WORDS * c->N, cudaHostAllocMapped));
    CK(cudaHostGetDevicePointer((void**)&c->d_progress, (void*)c->m_progress, 0));
  }
  int r = download_nodes(c);
  if (r) return r;
  if ((r = ensure_helpers(c))) return r;
  for (uint32_t n = 0; n < c->N; ++n) {
    const NodeDev& nd = c->nodes_host[n];
    volatile uint32_t* pr = c->m_progress + (size_t)n * PR_WORDS;
    pr[PR_INSTR] = nd.n_instr;
    pr[PR_EDGE] = nd.n_edge;
    pr[PR_BOX] = nd.n_box;
    pr[PR_BIND] = nd.n_bind;
    pr[PR_STATUS] = nd.status;
    pr[PR_CURSOR] = nd.cursor;
  }
  std::atomic_thread_fence(std::memory_order_seq_cst);
  // the executor stream starts after everything already enqueued on the context's stream
  cudaEvent_t ready;
  CK(cudaEventCreateWithFlags(&ready, cudaEventDisableTiming));
  CK(cudaEventRecord(ready, c->stream));
  CK(cudaStreamWaitEvent(c->xstream, ready, 0));
  CK(cudaEventDestroy(ready));
  c->pipelined = true;
  auto finish = [&](int code) {
    cudaStreamSynchronize(c->xstream);
    cudaStreamSynchronize(c->stream);
    c->pipelined = false;
    ev_collect(c);
    const int fr = flow_collect(c);
    const int er = exec_error_status(c);
    const int orr = oob_status(c);
    return code != IGS_OK ? code : fr != IGS_OK ? fr : er != IGS_OK ? er : orr;
  };
  // one launch lowers every pending submission; each node's warp publishes
  // its progress, and the executor follows behind on its own stream
  if ((r = launch_lower(c, IGS_NONE, true, c->d_progress))) return finish(r);
  const uint32_t total = (uint32_t)c->items.size();
  std::vector<uint32_t> cur(c->N), cnt(4 * c->N);
  uint32_t executed_upto = 0;
  for (;;) {
    bool done = true, failed = false;
    uint32_t low = 0xFFFFFFFFu;
    for (uint32_t n = 0; n < c->N; ++n) {
      volatile uint32_t* pr = c->m_progress + (size_t)n * PR_WORDS;
      cur[n] = pr[PR_CURSOR];
      std::atomic_thread_fence(std::memory_order_acquire);
      cnt[4 * n] = pr[PR_INSTR];
      cnt[4 * n + 1] = pr[PR_EDGE];
      cnt[4 * n + 2] = pr[PR_BOX];
      cnt[4 * n + 3] = pr[PR_BIND];
      if (pr[PR_STATUS] != ST_OK) failed = true;
      if (cur[n] < total) done = false;
      low = std::min(low, cur[n]);
    }
    if (failed) break;  // the status check below reports it
    if (!done && cudaStreamQuery(c->stream) != cudaErrorNotReady) break;  // the launch ended early
    if (!done && low < executed_upto + window) {
      std::this_thread::sleep_for(std::chrono::microseconds(20));
      continue;
    }
    executed_upto = low;
    for (uint32_t n = 0; n < c->N; ++n)
      if ((r = fetch_node(c, n, cnt[4 * n], cnt[4 * n + 1], cnt[4 * n + 2], cnt[4 * n + 3], c->cstream)))
        return finish(r);
    Pending p;
    FlowBuild g;
    if (c->executor == IGS_EXEC_DATAFLOW) p.flow = &g;
    bool halted = false, progress = false;
    if ((r = exec_walk(c, p, c->xstream, &halted, &progress))) return finish(r);
    if ((r = run_walk(c, p, c->xstream, false))) return finish(r);
    if (done) break;
  }
  // the lowering launch has ended (or failed): its final state, then the rest
  r = check_status(c);
  if (r && r != IGS_ERR_OVERLAPPING_WRITE) return finish(r);
  const int rejected = r;
  if ((r = fetch_for_exec(c))) return finish(r);
  for (;;) {
    Pending p;
    FlowBuild g;
    if (c->executor == IGS_EXEC_DATAFLOW) p.flow = &g;
    bool halted = false, progress = false;
    if ((r = exec_walk(c, p, c->xstream, &halted, &progress))) return finish(r);
    if ((r = run_walk(c, p, c->xstream, false))) return finish(r);
    if (!halted || !progress) break;
  }
  return finish(rejected);
}

namespace {

// Host-side view of one node table (read back for igs_read_buffer).
struct HEntry {
  uint32_t key, lo[3], hi[3], v[3];
};

// Reads the heap table behind descriptor `desc` {offset, cap, n, live} of a
// node from the device.
int read_slab(igs_ctx* c, const NodeDev& nd, const uint32_t* desc, std::vector<HEntry>& out) {
  out.clear();
  uint32_t d[4];
  CK(cudaMemcpy(d, desc, sizeof d, cudaMemcpyDeviceToHost));
  const uint32_t n = d[2];
  if (d[1] == 0 || n == 0) return IGS_OK;
  std::vector<uint32_t> raw((size_t)F_COUNT * n);
  const uint32_t* t = nd.heap + (size_t)d[0] * F_COUNT;
  CK(cudaMemcpy(raw.data(), t, sizeof(uint32_t) * F_COUNT * n, cudaMemcpyDeviceToHost));
  for (uint32_t i = 0; i < n; ++i) {
    const uint32_t* w = raw.data() + (size_t)i * F_COUNT;
    HEntry e;
    e.key = w[F_KEY];
    for (int d = 0; d < 3; ++d) {
      e.lo[d] = w[F_LO + d];
      e.hi[d] = w[F_HI + d];
    }
    for (int k = 0; k < 3; ++k) e.v[k] = w[F_V + k];
    if (e.key != DEAD) out.push_back(e);
  }
  return IGS_OK;
}

bool isect(const uint32_t alo[3], const uint32_t ahi[3], const uint32_t blo[3], const uint32_t bhi[3], igs_box& o) {
  for (int d = 0; d < 3; ++d) {
    o.lo[d] = std::max(alo[d], blo[d]);
    o.hi[d] = std::min(ahi[d], bhi[d]);
    if (o.lo[d] >= o.hi[d]) return false;
  }
  return true;
}

}  // namespace

extern "C" int igs_read_buffer(igs_ctx* c, uint32_t b, const uint32_t lo[3], const uint32_t hi[3], void* host_dst) {
  if (!c || b >= c->bufs.size() || !lo || !hi || !host_dst) return fail_ctx(c, IGS_ERR_INVALID_ARG, "bad read");
  if (!c->buf_live[b]) return fail_ctx(c, IGS_ERR_INVALID_ARG, "buffer was destroyed");
  const BufDesc& bf = c->bufs[b];
  uint64_t cnt = bf.elem;
  uint32_t rl[3], rh[3];
  for (int d = 0; d < 3; ++d) {
    rl[d] = lo[d];
    rh[d] = hi[d];
    if (rl[d] >= rh[d] || rh[d] > bf.extent[d]) return fail_ctx(c, IGS_ERR_INVALID_ARG, "read box outside buffer");
    cnt *= rh[d] - rl[d];
  }
  int r = download_nodes(c);
  if (r) return r;
  uint8_t* stage = nullptr;
  CK(cudaMalloc(&stage, cnt));
  CK(cudaMemsetAsync(stage, 0, cnt, c->stream));
  std::vector<HEntry> own, bst;
  {
    const NodeDev& n0 = c->nodes_host[0];
    r = read_slab(c, n0, n0.own_d + kDesc * b, own);
    if (r) return r;
  }
  Pending p;
  for (const HEntry& e : own) {
    igs_box piece;
    if (!isect(e.lo, e.hi, rl, rh, piece)) continue;
    if (e.v[0] == HOST) {
      CopyJob J{};
      uint32_t blo[3] = {0, 0, 0}, bhi[3] = {bf.extent[0], bf.extent[1], bf.extent[2]};
      if (make_copy_job(c->init_dev[b], blo, bhi, stage, rl, rh, piece, bf.elem, J)) add_copy(p, 1, J);
      continue;
    }
    if (e.v[0] >= c->N) continue;  // never written
    const uint32_t o = e.v[0];
    {
      const NodeDev& no = c->nodes_host[o];
      r = read_slab(c, no, no.bst_d + kDesc * b, bst);
      if (r) return r;
    }
    for (const HEntry& f : bst) {
      igs_box q;
      if (!isect(f.lo, f.hi, piece.lo, piece.hi, q)) continue;
      const uint32_t pmem = f.v[1];
      for (auto& al : c->nh[o].allocs) {
        const ExecAlloc& A = al.second;
        if (!A.live || A.buffer != b || A.mem != pmem) continue;
        igs_box z;
        if (!isect(A.lo, A.hi, q.lo, q.hi, z)) continue;
        CopyJob J{};
        if (make_copy_job(A.ptr, A.lo, A.hi, stage, rl, rh, z, bf.elem, J)) add_copy(p, 1, J);
      }
    }
  }
  r = run_pending(c, p, c->stream, true);
  if (r) return r;
  CK(cudaMemcpyAsync(host_dst, stage, cnt, cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  CK(cudaFree(stage));
  return IGS_OK;
}

extern "C" int igs_box_copy(const igs_copy_job* jobs, uint32_t n, void* stream) {
  igs_ctx* c = nullptr;
  if (!jobs && n) return IGS_ERR_INVALID_ARG;
  std::vector<CopyJob> v;
  uint64_t units = 0;
  for (uint32_t i = 0; i < n; ++i) {
    const igs_copy_job& j = jobs[i];
    CopyJob J{};
    for (int d = 0; d < 3; ++d)
      if (j.box.lo[d] < j.src_box.lo[d] || j.box.hi[d] > j.src_box.hi[d] || j.box.lo[d] < j.dst_box.lo[d] ||
          j.box.hi[d] > j.dst_box.hi[d])
        return IGS_ERR_INVALID_ARG;
    if (!make_copy_job(static_cast<const uint8_t*>(j.src), j.src_box.lo, j.src_box.hi, static_cast<uint8_t*>(j.dst),
                       j.dst_box.lo, j.dst_box.hi, j.box, j.elem_size, J))
      continue;
    J.unit_begin = units;
    units += (uint64_t)J.extent[0] * J.extent[1] * ((J.extent[2] + J.seg_bytes - 1) / J.seg_bytes);
    v.push_back(J);
  }
  if (v.empty()) return IGS_OK;
  static thread_local CopyJob* d_jobs = nullptr;
  static thread_local size_t cap = 0;
  if (v.size() > cap) {
    if (d_jobs) cudaFree(d_jobs);
    cap = v.size() * 2;
    CK(cudaMalloc(&d_jobs, sizeof(CopyJob) * cap));
  }
  CK(cudaMemcpyAsync(d_jobs, v.data(), sizeof(CopyJob) * v.size(), cudaMemcpyHostToDevice, (cudaStream_t)stream));
  if (igs_launch_copies(d_jobs, (uint32_t)v.size(), units, stream)) return IGS_ERR_CUDA;
  CK(cudaStreamSynchronize((cudaStream_t)stream));
  return IGS_OK;
}

// ---- served lowering ----------------------------------------------------------

extern "C" int igs_serve_create(const igs_serve_config* cfg, igs_server** out) {
  if (!cfg || !out || cfg->max_slots == 0) return IGS_ERR_INVALID_ARG;
  *out = nullptr;
  if (cudaSetDevice(cfg->device) != cudaSuccess) return IGS_ERR_CUDA;
  igs_server* s = new igs_server();
  s->cfg = *cfg;
  if (s->cfg.idle_timeout_ms == 0) s->cfg.idle_timeout_ms = 10000;
  if (cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking) != cudaSuccess ||
      cudaHostAlloc(&s->slots, sizeof(ServeSlot) * cfg->max_slots, cudaHostAllocMapped) != cudaSuccess ||
      cudaHostAlloc(&s->stop, sizeof(uint32_t), cudaHostAllocMapped) != cudaSuccess ||
      cudaHostGetDevicePointer((void**)&s->d_slots, s->slots, 0) != cudaSuccess ||
      cudaHostGetDevicePointer((void**)&s->d_stop, s->stop, 0) != cudaSuccess ||
      cudaEventCreateWithFlags(&s->done_ev, cudaEventDisableTiming) != cudaSuccess) {
    igs_serve_destroy(s);
    return IGS_ERR_CUDA;
  }
  std::memset((void*)s->slots, 0, sizeof(ServeSlot) * cfg->max_slots);
  *s->stop = 0;
  for (uint32_t i = cfg->max_slots; i > 0; --i) s->free_slots.push_back(i - 1);
  *out = s;
  return IGS_OK;
}

extern "C" int igs_serve_stop(igs_server* s) {
  if (!s) return IGS_ERR_INVALID_ARG;
  *reinterpret_cast<volatile uint32_t*>(s->stop) = 1;
  std::atomic_thread_fence(std::memory_order_seq_cst);
  if (s->launched) {
    if (cudaStreamSynchronize(s->stream) != cudaSuccess) return IGS_ERR_CUDA;
    s->launched = false;
  }
  *reinterpret_cast<volatile uint32_t*>(s->stop) = 0;
  return IGS_OK;
}

extern "C" void igs_serve_destroy(igs_server* s) {
  if (!s) return;
  igs_serve_stop(s);
  for (auto& a : s->attached) a.first->server = nullptr;
  for (auto& w : s->waiting) {
    w.first->server = nullptr;
    w.first->serve_pending = false;
  }
  if (s->slots) cudaFreeHost((void*)s->slots);
  if (s->stop) cudaFreeHost(s->stop);
  if (s->done_ev) cudaEventDestroy(s->done_ev);
  if (s->stream) cudaStreamDestroy(s->stream);
  delete s;
}

extern "C" int igs_serve_start(igs_server* s) {
  if (!s) return IGS_ERR_INVALID_ARG;
  if (s->launched) {
    if (cudaEventQuery(s->done_ev) == cudaErrorNotReady) return IGS_OK;  // still running
    s->launched = false;
  }
  const uint64_t idle = (uint64_t)s->cfg.idle_timeout_ms * 500;  // polls of about 2 us
  if (igs_launch_serve(s->d_slots, s->cfg.max_slots, s->d_stop, idle, s->stream)) return IGS_ERR_CUDA;
  if (cudaEventRecord(s->done_ev, s->stream) != cudaSuccess) return IGS_ERR_CUDA;
  s->launched = true;
  return IGS_OK;
}

namespace {
// Footprint a served context is charged against the budget: its device arena
// plus every buffer's bytes on every memory of every node plus its host data.
double serve_footprint(const igs_ctx* c) {
  double foot = (double)c->arena_bytes;
  for (size_t b = 0; b < c->bufs.size(); ++b) {
    double bytes = c->bufs[b].elem;
    for (int d = 0; d < 3; ++d) bytes *= c->bufs[b].extent[d];
    foot += bytes * c->N * (c->D + 1) + (c->init_dev[b] ? bytes : 0.0);
  }
  return foot;
}

bool serve_fits(const igs_server* s, const igs_ctx* c) {
  if (s->free_slots.size() < c->N) return false;
  return !s->cfg.hbm_budget_bytes || s->used + serve_footprint(c) <= (double)s->cfg.hbm_budget_bytes;
}

// Attaches c (not served, or leaving the admission queue) when it fits.
int serve_attach_impl(igs_server* s, igs_ctx* c, uint32_t max_items) {
  const double foot = serve_footprint(c);
  if (s->free_slots.size() < c->N) return fail_ctx(c, IGS_ERR_BUDGET, "no free serving slots");
  if (s->cfg.hbm_budget_bytes && s->used + foot > (double)s->cfg.hbm_budget_bytes)
    return fail_ctx(c, IGS_ERR_BUDGET, "HBM budget exceeded");
  // everything submitted so far must be lowered before the loop takes over
  if (c->items_up < c->items.size() || c->cfg.mode == IGS_MODE_BATCHED) {
    int r = launch_lower(c);
    if (r) return r;
  }
  if (int r = check_status(c)) {
    if (r != IGS_ERR_OVERLAPPING_WRITE) return r;
  }
  const uint32_t cap = max_items;
  // device arrays for every submission the context can take while served
  // (the loop stages new ones into them), host-mapped arrays the host
  // publishes into
  if (int r = grow_device(c, c->d_items, c->cap_items, cap, c->items_up)) return r;
  if (int r = grow_device(c, c->d_tasks, c->cap_tasks, cap, c->tasks_up)) return r;
  if (c->m_items && cap > c->m_cap) {  // an earlier attach's arrays are too small
    cudaFreeHost(c->m_items);
    cudaFreeHost(c->m_tasks);
    c->m_items = nullptr;
    c->m_tasks = nullptr;
  }
  if (!c->m_items) {
    CK(cudaHostAlloc(&c->m_items, sizeof(Item) * cap, cudaHostAllocMapped));
    CK(cudaHostAlloc(&c->m_tasks, sizeof(igs_task) * cap, cudaHostAllocMapped));
    c->m_cap = cap;
  }
  if (!c->m_nitems) CK(cudaHostAlloc(&c->m_nitems, sizeof(uint32_t), cudaHostAllocMapped));
  std::memcpy(c->m_items, c->items.data(), sizeof(Item) * c->items.size());
  std::memcpy(c->m_tasks, c->tasks.data(), sizeof(igs_task) * c->tasks.size());
  *reinterpret_cast<volatile uint32_t*>(c->m_nitems) = (uint32_t)c->items.size();
  ProgDev p;
  p.items = c->d_items;
  p.tasks = c->d_tasks;
  p.bufs = c->d_bufs;
  CK(cudaHostGetDevicePointer((void**)&p.src_items, c->m_items, 0));
  CK(cudaHostGetDevicePointer((void**)&p.src_tasks, c->m_tasks, 0));
  uint32_t* dn = nullptr;
  CK(cudaHostGetDevicePointer((void**)&dn, c->m_nitems, 0));
  p.n_items = dn;
  CK(cudaMemcpy(c->d_prog, &p, sizeof p, cudaMemcpyHostToDevice));
  c->serve_cap = cap;
  c->items_up = (uint32_t)c->items.size();
  c->tasks_up = (uint32_t)c->tasks.size();
  c->slot_ids.clear();
  for (uint32_t n = 0; n < c->N; ++n) {
    const uint32_t id = s->free_slots.back();
    s->free_slots.pop_back();
    c->slot_ids.push_back(id);
    ServeSlot& S = s->slots[id];
    S.unit.node = c->d_nodes + n;
    S.unit.prog = c->d_prog;
    S.done = (uint32_t)c->items.size();
    S.status = 0;
    S.exit = 0;
    S.busy = 0;
    std::atomic_thread_fence(std::memory_order_seq_cst);
    S.state = SLOT_ACTIVE;
  }
  std::atomic_thread_fence(std::memory_order_seq_cst);
  c->server = s;
  s->used += foot;
  s->attached.push_back({c, foot});
  s->n_admitted += 1;
  return IGS_OK;
}

// Admits waiting contexts in arrival order while the head of the queue fits.
// A context whose admission fails leaves the queue unserved (its error is in
// igs_last_error; later submissions take the launch path).
void serve_admit_waiting(igs_server* s) {
  while (!s->waiting.empty()) {
    igs_ctx* c = s->waiting.front().first;
    const uint32_t cap = s->waiting.front().second;
    if (!serve_fits(s, c)) break;
    s->waiting.pop_front();
    c->server = nullptr;
    c->serve_pending = false;
    if (serve_attach_impl(s, c, cap) == IGS_OK) s->n_admitted_queued += 1;
  }
}
}  // namespace

extern "C" int igs_serve_attach(igs_server* s, igs_ctx* c, uint32_t max_items) {
  if (!s || !c || c->server || max_items < c->items.size() + 1) return IGS_ERR_INVALID_ARG;
  return serve_attach_impl(s, c, max_items);
}

extern "C" int igs_serve_enqueue(igs_server* s, igs_ctx* c, uint32_t max_items, uint32_t* admitted) {
  if (!s || !c || c->server || max_items < c->items.size() + 1) return IGS_ERR_INVALID_ARG;
  if (admitted) *admitted = 0;
  // a context that could never fit is refused rather than queued forever
  if (c->N > s->cfg.max_slots) return fail_ctx(c, IGS_ERR_BUDGET, "more nodes than serving slots");
  if (s->cfg.hbm_budget_bytes && serve_footprint(c) > (double)s->cfg.hbm_budget_bytes)
    return fail_ctx(c, IGS_ERR_BUDGET, "footprint exceeds the whole HBM budget");
  if (s->waiting.empty() && serve_fits(s, c)) {
    const int r = serve_attach_impl(s, c, max_items);
    if (r == IGS_OK && admitted) *admitted = 1;
    return r;
  }
  // the device and host-mapped submission arrays are sized now, so that the
  // admission (during a detach, with the loop running) allocates nothing
  if (int r = grow_device(c, c->d_items, c->cap_items, max_items, c->items_up)) return r;
  if (int r = grow_device(c, c->d_tasks, c->cap_tasks, max_items, c->tasks_up)) return r;
  if (c->m_items && max_items > c->m_cap) {
    cudaFreeHost(c->m_items);
    cudaFreeHost(c->m_tasks);
    c->m_items = nullptr;
    c->m_tasks = nullptr;
  }
  if (!c->m_items) {
    CK(cudaHostAlloc(&c->m_items, sizeof(Item) * max_items, cudaHostAllocMapped));
    CK(cudaHostAlloc(&c->m_tasks, sizeof(igs_task) * max_items, cudaHostAllocMapped));
    c->m_cap = max_items;
  }
  if (!c->m_nitems) CK(cudaHostAlloc(&c->m_nitems, sizeof(uint32_t), cudaHostAllocMapped));
  c->server = s;
  c->serve_pending = true;
  c->serve_cap = max_items;
  s->waiting.push_back({c, max_items});
  s->peak_waiting = std::max<uint64_t>(s->peak_waiting, s->waiting.size());
  return IGS_OK;
}

extern "C" int igs_serve_stats(const igs_server* s, uint64_t out[8]) {
  if (!s || !out) return IGS_ERR_INVALID_ARG;
  std::memset(out, 0, sizeof(uint64_t) * 8);
  out[0] = s->n_admitted;
  out[1] = s->n_admitted_queued;
  out[2] = s->waiting.size();
  out[3] = s->peak_waiting;
  out[4] = s->cfg.max_slots - s->free_slots.size();
  out[5] = (uint64_t)s->used;
  return IGS_OK;
}


extern "C" int igs_serve_progress(const igs_ctx* c, uint32_t* submitted, uint32_t* taken) {
  if (!c || !c->server) return IGS_ERR_INVALID_ARG;
  if (c->serve_pending) {  // waiting for admission: nothing taken yet
    if (submitted) *submitted = (uint32_t)c->items.size();
    if (taken) *taken = 0;
    return IGS_OK;
  }
  uint32_t t = 0xFFFFFFFFu, st = 0;
  for (uint32_t id : c->slot_ids) {
    const ServeSlot& S = c->server->slots[id];
    const uint32_t d = S.done, e = S.status;
    t = std::min(t, d);
    st |= e;
  }
  if (submitted) *submitted = (uint32_t)c->items.size();
  if (taken) *taken = t;
  return st ? IGS_ERR_CAPACITY : IGS_OK;
}

extern "C" int igs_serve_replay_ex(igs_server* s, igs_ctx* const* ctxs, uint32_t n_ctx, const igs_replay_item* items,
                                   uint32_t n, uint32_t timeout_ms, uint32_t flags, uint64_t* latency_ns,
                                   uint64_t* wall_ns) {
  if (!s || !ctxs || (n && (!items || !latency_ns))) return IGS_ERR_INVALID_ARG;
  for (uint32_t i = 0; i < n_ctx; ++i)
    if (!ctxs[i] || ctxs[i]->server != s) return IGS_ERR_INVALID_ARG;
  for (uint32_t k = 0; k < n; ++k)
    if (items[k].ctx >= n_ctx || (!items[k].epoch && !items[k].task) || (k && items[k].arrival_ns < items[k - 1].arrival_ns))
      return IGS_ERR_INVALID_ARG;
  using clock = std::chrono::steady_clock;
  const auto t0 = clock::now();
  auto now_ns = [&]() { return (uint64_t)std::chrono::duration_cast<std::chrono::nanoseconds>(clock::now() - t0).count(); };
  // per context: (submission count that completes the item, item index), in order
  std::vector<std::vector<std::pair<uint32_t, uint32_t>>> fifo(n_ctx);
  std::vector<size_t> head(n_ctx, 0);
  std::vector<uint32_t> busy;  // contexts with items in flight
  // with IGS_REPLAY_DETACH: a context is detached once its last item of the
  // trace is taken, which admits contexts waiting in the admission queue
  const bool detach_at_end = (flags & IGS_REPLAY_DETACH) != 0;
  std::vector<uint32_t> last_item(n_ctx, 0xFFFFFFFFu);
  for (uint32_t k = 0; k < n; ++k) last_item[items[k].ctx] = k;
  uint32_t next = 0, done = 0;
  uint64_t last = 0;
  const uint64_t limit = (n ? items[n - 1].arrival_ns : 0) + (uint64_t)timeout_ms * 1000000ull;
  for (;;) {
    uint64_t t = now_ns();
    while (next < n && items[next].arrival_ns <= t) {
      const igs_replay_item& it = items[next];
      igs_ctx* c = ctxs[it.ctx];
      uint64_t seq = 0;
      const int r = it.epoch ? igs_submit_epoch(c) : igs_submit_task(c, it.task, &seq);
      if (r && r != IGS_ERR_OVERLAPPING_WRITE) return r;
      if (head[it.ctx] == fifo[it.ctx].size()) busy.push_back(it.ctx);
      fifo[it.ctx].push_back({(uint32_t)c->items.size(), next});
      ++next;
    }
    t = now_ns();
    for (size_t b = 0; b < busy.size();) {
      const uint32_t ci = busy[b];
      uint32_t sub = 0, taken = 0;
      if (igs_serve_progress(ctxs[ci], &sub, &taken)) return fail_ctx(ctxs[ci], IGS_ERR_CAPACITY, "a serving slot failed");
      auto& q = fifo[ci];
      while (head[ci] < q.size() && q[head[ci]].first <= taken) {
        const uint32_t k = q[head[ci]].second;
        latency_ns[k] = t > items[k].arrival_ns ? t - items[k].arrival_ns : 0;
        last = t;
        ++head[ci];
        ++done;
      }
      if (head[ci] == q.size()) {
        busy[b] = busy.back();
        busy.pop_back();
        if (detach_at_end && last_item[ci] != 0xFFFFFFFFu && last_item[ci] < next) {
          last_item[ci] = 0xFFFFFFFFu;
          if (int e = igs_serve_detach(s, ctxs[ci], timeout_ms)) return e;
          t = now_ns();
        }
      } else {
        ++b;
      }
    }
    if (done == n) break;
    if (t > limit) return IGS_ERR_TIMEOUT;
    if (s->launched && cudaEventQuery(s->done_ev) == cudaSuccess) {
      s->launched = false;  // the loop went idle: restart it
      if (int e = igs_serve_start(s)) return e;
    }
  }
  if (wall_ns) *wall_ns = last;
  return IGS_OK;
}

extern "C" int igs_serve_replay(igs_server* s, igs_ctx* const* ctxs, uint32_t n_ctx, const igs_replay_item* items,
                                uint32_t n, uint32_t timeout_ms, uint64_t* latency_ns, uint64_t* wall_ns) {
  return igs_serve_replay_ex(s, ctxs, n_ctx, items, n, timeout_ms, 0, latency_ns, wall_ns);
}

extern "C" int igs_replay_plain(igs_ctx* const* ctxs, uint32_t n_ctx, const igs_replay_item* items, uint32_t n,
                                uint32_t timeout_ms, uint64_t* latency_ns, uint64_t* wall_ns) {
  if (!ctxs || (n && (!items || !latency_ns))) return IGS_ERR_INVALID_ARG;
  for (uint32_t i = 0; i < n_ctx; ++i)
    if (!ctxs[i] || ctxs[i]->server || ctxs[i]->cfg.mode != IGS_MODE_PLAIN || ctxs[i]->pipelined)
      return IGS_ERR_INVALID_ARG;
  for (uint32_t k = 0; k < n; ++k)
    if (items[k].ctx >= n_ctx || (!items[k].epoch && !items[k].task) || (k && items[k].arrival_ns < items[k - 1].arrival_ns))
      return IGS_ERR_INVALID_ARG;
  using clock = std::chrono::steady_clock;
  const auto t0 = clock::now();
  auto now_ns = [&]() { return (uint64_t)std::chrono::duration_cast<std::chrono::nanoseconds>(clock::now() - t0).count(); };
  // per context, in submission order: (completion event, item index)
  std::vector<std::deque<std::pair<cudaEvent_t, uint32_t>>> inflight(n_ctx);
  std::vector<cudaEvent_t> pool;
  auto release = [&]() {
    for (auto& q : inflight)
      for (auto& e : q) cudaEventDestroy(e.first);
    for (cudaEvent_t e : pool) cudaEventDestroy(e);
  };
  uint32_t next = 0, done = 0;
  uint64_t last = 0;
  const uint64_t limit = (n ? items[n - 1].arrival_ns : 0) + (uint64_t)timeout_ms * 1000000ull;
  while (done < n) {
    uint64_t t = now_ns();
    while (next < n && items[next].arrival_ns <= t) {
      const igs_replay_item& it = items[next];
      igs_ctx* c = ctxs[it.ctx];
      uint64_t seq = 0;
      const int r = it.epoch ? igs_submit_epoch(c) : igs_submit_task(c, it.task, &seq);  // one launch
      if (r && r != IGS_ERR_OVERLAPPING_WRITE) {
        release();
        return r;
      }
      cudaEvent_t ev = nullptr;
      if (!pool.empty()) {
        ev = pool.back();
        pool.pop_back();
      } else if (cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess) {
        release();
        return fail_ctx(c, IGS_ERR_CUDA, "event creation failed");
      }
      if (cudaEventRecord(ev, c->stream) != cudaSuccess) {
        pool.push_back(ev);
        release();
        return fail_ctx(c, IGS_ERR_CUDA, "event record failed");
      }
      inflight[it.ctx].push_back({ev, next});
      ++next;
    }
    t = now_ns();
    for (uint32_t ci = 0; ci < n_ctx; ++ci) {
      auto& q = inflight[ci];
      while (!q.empty()) {
        const cudaError_t e = cudaEventQuery(q.front().first);
        if (e == cudaErrorNotReady) break;
        if (e != cudaSuccess) {
          release();
          return fail_ctx(ctxs[ci], IGS_ERR_CUDA, "lowering launch failed");
        }
        const uint32_t k = q.front().second;
        latency_ns[k] = t > items[k].arrival_ns ? t - items[k].arrival_ns : 0;
        last = t;
        pool.push_back(q.front().first);
        q.pop_front();
        ++done;
      }
    }
    if (done < n && t > limit) {
      release();
      return IGS_ERR_TIMEOUT;
    }
  }
  release();
  for (uint32_t i = 0; i < n_ctx; ++i) {
    const int r = check_status(ctxs[i]);
    if (r && r != IGS_ERR_OVERLAPPING_WRITE) return r;
  }
  if (wall_ns) *wall_ns = last;
  return IGS_OK;
}

extern "C" int igs_serve_detach(igs_server* s, igs_ctx* c, uint32_t timeout_ms) {
  if (!s || !c || c->server != s) return IGS_ERR_INVALID_ARG;
  if (c->serve_pending) {  // still queued: it leaves the queue unserved
    for (auto it = s->waiting.begin(); it != s->waiting.end(); ++it)
      if (it->first == c) {
        s->waiting.erase(it);
        break;
      }
    c->server = nullptr;
    c->serve_pending = false;
    return IGS_OK;
  }
  const auto t0 = std::chrono::steady_clock::now();
  for (;;) {
    uint32_t sub = 0, tk = 0;
    const int r = igs_serve_progress(c, &sub, &tk);
    if (r) break;
    if (tk >= sub) break;
    if (std::chrono::steady_clock::now() - t0 > std::chrono::milliseconds(timeout_ms))
      return fail_ctx(c, IGS_ERR_TIMEOUT, "serving loop did not take every submission in time");
    if (s->launched && cudaEventQuery(s->done_ev) == cudaSuccess) {
      s->launched = false;  // the loop left (idle or error): restart it
      if (int e = igs_serve_start(s)) return e;
    }
    std::this_thread::sleep_for(std::chrono::microseconds(50));
  }
  for (uint32_t id : c->slot_ids) s->slots[id].state = SLOT_EMPTY;
  std::atomic_thread_fence(std::memory_order_seq_cst);
  // a warp marks its slot busy before it re-reads the state and processes;
  // once busy reads 0 after the state was cleared, no warp touches the context
  for (uint32_t id : c->slot_ids) {
    const auto t1 = std::chrono::steady_clock::now();
    while (s->slots[id].busy) {
      if (std::chrono::steady_clock::now() - t1 > std::chrono::milliseconds(timeout_ms))
        return fail_ctx(c, IGS_ERR_TIMEOUT, "serving warp did not leave its slot");
      std::this_thread::yield();
    }
    s->free_slots.push_back(id);
  }
  for (size_t i = 0; i < s->attached.size(); ++i)
    if (s->attached[i].first == c) {
      s->used -= s->attached[i].second;
      s->attached.erase(s->attached.begin() + i);
      break;
    }
  c->server = nullptr;
  c->slot_ids.clear();
  // the freed slots and budget go to the contexts waiting for admission
  serve_admit_waiting(s);
  // later submissions go through the launch path again
  const int r = check_status(c);
  return r == IGS_ERR_OVERLAPPING_WRITE ? IGS_OK : r;
}
