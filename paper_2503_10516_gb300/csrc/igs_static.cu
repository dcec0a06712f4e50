// Lowering without allocation: the whole node state, the scratch tables and
// the staged inputs live in one file-scope device array, so this entry point
// never calls cudaMalloc, cudaFree or any allocating routine. It is meant for
// callers that cannot allocate device memory on their own: a host runtime
// whose device memory all comes from its own pool and must not be bypassed,
// or a latency-critical loop that must not enter the driver's allocator
// (which can block on, or synchronize with, other work on the device). The
// caller passes host inputs and device output arrays that it owns.
#include <cuda_runtime.h>

#include <cstring>
#include <mutex>
#include <vector>

#include "igs_check.h"
#include "igs_internal.h"
#include "igs_tdag.h"

namespace {

// The scratch every call shares: 32 MiB per device that loads the library,
// held until the process exits. Calls that overlap on the GPU race on it.
constexpr size_t kStaticBytes = 32u << 20;
__device__ __align__(256) uint8_t g_static_scratch[kStaticBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
uint8_t* g_base[kMaxDevices] = {};

// Per-node capacities of this variant (modest, fixed).
constexpr uint32_t kBuffers = 16, kHeap = 1u << 15, kSlots = 128, kQr = 2048, kScratch = 1024;
constexpr uint32_t kAlloc = 4096, kQueue = 4096, kRej = 256;

size_t tbytes(uint32_t cap) { return (size_t)igs::F_COUNT * cap * sizeof(uint32_t); }

struct Layout {
  size_t per_node, o_heap, o_desc, o_free, o_live, o_qr, o_alloc, o_queue, o_succ, o_rej, o_scr;
};

Layout layout(uint32_t cap_instr) {
  Layout L{};
  size_t p = 0;
  auto take = [&](size_t b) {
    const size_t o = p;
    p += (b + 255) & ~(size_t)255;
    return o;
  };
  L.o_heap = take(tbytes(kHeap));
  L.o_desc = take(4 * igs::kDesc * (2 * kBuffers + 2 * kSlots));
  L.o_free = take(4 * kSlots);
  L.o_live = take(4 * kSlots);
  L.o_qr = take(tbytes(kQr));
  L.o_alloc = take(sizeof(igs::AllocRec) * kAlloc);
  L.o_queue = take(4 * kQueue);
  L.o_succ = take(cap_instr);
  L.o_rej = take(4 * kRej);
  L.o_scr = take(tbytes(kScratch) * 14);
  L.per_node = p;
  return L;
}

}  // namespace

extern "C" int igs_horizon_plan(const igs_static_buffer* bufs, uint32_t num_buffers, const igs_task* tasks,
                                uint32_t num_tasks, uint32_t horizon_step, uint32_t flags, uint8_t* horizon_after) {
  if ((num_buffers && !bufs) || (num_tasks && (!tasks || !horizon_after))) return IGS_ERR_INVALID_ARG;
  igs::CriticalPath cpath;
  for (uint32_t i = 0; i < num_tasks; ++i) {
    const igs_task& t = tasks[i];
    if (t.num_accessors > IGS_MAX_ACCESSORS) return IGS_ERR_INVALID_ARG;
    for (uint32_t a = 0; a < t.num_accessors; ++a)
      if (t.acc[a].buffer >= num_buffers) return IGS_ERR_INVALID_ARG;
    const bool cp = cpath.add(
        t, [&](uint32_t b) { return bufs[b].dims; }, [&](uint32_t b) { return bufs[b].extent; }, horizon_step);
    horizon_after[i] = (flags & IGS_FLAG_HORIZON_CP) ? cp : (horizon_step && (i + 1) % horizon_step == 0);
  }
  return IGS_OK;
}

extern "C" int igs_lower_static(const igs_config* cfg, const igs_static_buffer* bufs, uint32_t num_buffers,
                                const igs_task* tasks, uint32_t num_tasks, const igs_static_op* ops,
                                uint32_t num_ops, igs_static_output* outs, void* stream_ptr) {
  using namespace igs;
  if (!cfg || !outs || (num_buffers && !bufs) || (num_tasks && !tasks) || (num_ops && !ops)) return IGS_ERR_INVALID_ARG;
  const uint32_t N = cfg->num_nodes, D = cfg->devices_per_node;
  if (N < 1 || N > 32 || D < 1 || D > 29 || num_buffers > kBuffers) return IGS_ERR_INVALID_ARG;
  if (!config_flags_ok(cfg->flags)) return IGS_ERR_INVALID_ARG;
  cudaStream_t stream = (cudaStream_t)stream_ptr;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return IGS_ERR_CUDA;
  uint8_t* base = nullptr;
  {
    // set-up, once per device, with that device current: the array's device
    // address (the symbol itself is only a host-side stand-in)
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_base[dev]) {
      void* p = nullptr;
      if (cudaGetSymbolAddress(&p, g_static_scratch) != cudaSuccess || !p) return IGS_ERR_CUDA;
      g_base[dev] = static_cast<uint8_t*>(p);
    }
    base = g_base[dev];
  }
  uint32_t cap_instr = 0xFFFFFFFFu;
  for (uint32_t n = 0; n < N; ++n) {
    const igs_static_output& o = outs[n];
    if (!o.instrs || !o.edges || !o.boxes || !o.binds || !o.diags || !o.counts) return IGS_ERR_INVALID_ARG;
    if (o.instr_cap == 0) return IGS_ERR_INVALID_ARG;
    cap_instr = o.instr_cap < cap_instr ? o.instr_cap : cap_instr;
  }
  // the submission stream, as the lowering warps see it
  std::vector<Item> items;
  std::vector<BufDesc> bd(num_buffers);
  for (uint32_t b = 0; b < num_buffers; ++b) {
    bd[b].dims = bufs[b].dims;
    for (int d = 0; d < 3; ++d) bd[b].extent[d] = d < (int)bufs[b].dims ? bufs[b].extent[d] : 1;
    bd[b].elem = bufs[b].elem_size;
    bd[b].init = bufs[b].has_init ? 1 : 0;
    if (!buffer_shape_ok(bufs[b].dims, bufs[b].extent, bufs[b].elem_size)) return IGS_ERR_INVALID_ARG;
  }
  uint32_t seq = 0, ntask = 0, created = 0;
  bool live[kBuffers] = {};  // created and not destroyed (the same checks as the context API)
  CriticalPath cpath;  // task-graph depth (IGS_FLAG_HORIZON_CP)
  for (uint32_t i = 0; i < num_ops; ++i) {
    const igs_static_op& op = ops[i];
    Item it{};
    switch (op.kind) {
      case IGS_OP_CREATE_BUFFER:
        if (op.arg != created || op.arg >= num_buffers) return IGS_ERR_INVALID_ARG;
        it = Item{IT_CREATE, seq++, op.arg, 0};
        live[op.arg] = true;
        ++created;
        items.push_back(it);
        break;
      case IGS_OP_TASK: {
        if (op.arg >= num_tasks) return IGS_ERR_INVALID_ARG;
        const igs_task& t = tasks[op.arg];
        if (task_problem(t, [&](uint32_t b) { return b < created && live[b]; })) return IGS_ERR_INVALID_ARG;
        items.push_back(Item{IT_TASK, seq++, 0, op.arg});
        const bool cp_horizon =
            (cfg->flags & IGS_FLAG_HORIZON_CP) &&
            cpath.add(
                t, [&](uint32_t b) { return bufs[b].dims; }, [&](uint32_t b) { return bufs[b].extent; },
                cfg->horizon_step);
        ++ntask;
        if ((cfg->flags & IGS_FLAG_HORIZON_CP) ? cp_horizon : (cfg->horizon_step && ntask % cfg->horizon_step == 0))
          items.push_back(Item{IT_HORIZON, seq++, 0, 0});
        break;
      }
      case IGS_OP_FLUSH:
        items.push_back(Item{IT_EPOCH, seq++, 0, 0});
        break;
      case IGS_OP_DESTROY_BUFFER:
        if (op.arg >= created || !live[op.arg]) return IGS_ERR_INVALID_ARG;  // unknown, or destroyed already
        live[op.arg] = false;
        items.push_back(Item{IT_DESTROY, seq++, op.arg, 0});
        break;
      case IGS_OP_LOOKAHEAD:
        items.push_back(Item{IT_LOOKAHEAD, seq, op.arg, 0});
        break;
      default:
        return IGS_ERR_INVALID_ARG;
    }
  }
  // carve the array: nodes, units, program, inputs
  const Layout L = layout(cap_instr);
  size_t off = 0;
  auto take = [&](size_t b) {
    const size_t o = off;
    off += (b + 255) & ~(size_t)255;
    return o;
  };
  const size_t o_nodes = take(sizeof(NodeDev) * N);
  const size_t o_units = take(sizeof(Unit) * N);
  const size_t o_prog = take(sizeof(ProgDev));
  const size_t o_nitems = take(sizeof(uint32_t));
  const size_t o_items = take(sizeof(Item) * (items.size() + 1));
  const size_t o_tasks = take(sizeof(igs_task) * (num_tasks + 1));
  const size_t o_bufs = take(sizeof(BufDesc) * (num_buffers + 1));
  const size_t o_state = take(L.per_node * N);
  if (off > kStaticBytes) return IGS_ERR_CAPACITY;  // program or instruction capacity too large for the array
  std::vector<NodeDev> nodes(N);
  std::vector<Unit> units(N);
  std::vector<uint32_t> slots(kSlots);
  for (uint32_t i = 0; i < kSlots; ++i) slots[i] = kSlots - 1 - i;
  for (uint32_t n = 0; n < N; ++n) {
    uint8_t* nb = base + o_state + L.per_node * n;
    NodeDev& nd = nodes[n];
    std::memset(&nd, 0, sizeof nd);
    const igs_static_output& o = outs[n];
    nd.node = n;
    nd.N = N;
    nd.D = D;
    nd.status = ST_OK;
    nd.lookahead = cfg->lookahead;
    nd.stage_d2d = (cfg->flags & IGS_FLAG_STAGE_D2D) ? 1u : 0u;
    nd.last_horizon = NONE;
    nd.n_instr = 1;
    nd.n_free = kSlots;
    nd.cap_instr = cap_instr;
    nd.cap_edge = o.edge_cap;
    nd.cap_box = o.box_cap;
    nd.cap_bind = o.bind_cap;
    nd.cap_diag = o.diag_cap;
    nd.cap_rej = kRej;
    nd.cap_alloc = kAlloc;
    nd.cap_queue = kQueue;
    nd.cap_buffers = kBuffers;
    nd.cap_slots = kSlots;
    nd.cap_qr = kQr;
    nd.cap_scratch = kScratch;
    nd.heap = reinterpret_cast<uint32_t*>(nb + L.o_heap);
    nd.cap_heap = kHeap;
    nd.heap_top = 0;
    for (int k = 0; k < igs::kHeapClasses; ++k) nd.free_head[k] = NONE;
    nd.own_d = reinterpret_cast<uint32_t*>(nb + L.o_desc);
    nd.bst_d = nd.own_d + igs::kDesc * kBuffers;
    nd.wr_d = nd.bst_d + igs::kDesc * kBuffers;
    nd.rd_d = nd.wr_d + igs::kDesc * kSlots;
    nd.free_slots = reinterpret_cast<uint32_t*>(nb + L.o_free);
    nd.live = reinterpret_cast<uint32_t*>(nb + L.o_live);
    nd.qr_base = reinterpret_cast<uint32_t*>(nb + L.o_qr);
    nd.allocs = reinterpret_cast<AllocRec*>(nb + L.o_alloc);
    nd.queue = reinterpret_cast<uint32_t*>(nb + L.o_queue);
    nd.has_succ = nb + L.o_succ;
    nd.rejected = reinterpret_cast<uint32_t*>(nb + L.o_rej);
    nd.scratch_base = reinterpret_cast<uint32_t*>(nb + L.o_scr);
    nd.instrs = o.instrs;
    nd.edges = o.edges;
    nd.boxes = o.boxes;
    nd.binds = o.binds;
    nd.diags = o.diags;
    units[n].node = reinterpret_cast<NodeDev*>(base + o_nodes) + n;
    units[n].prog = reinterpret_cast<ProgDev*>(base + o_prog);
  }
  ProgDev pg;
  pg.items = reinterpret_cast<const Item*>(base + o_items);
  pg.tasks = reinterpret_cast<const igs_task*>(base + o_tasks);
  pg.bufs = reinterpret_cast<const BufDesc*>(base + o_bufs);
  pg.n_items = reinterpret_cast<volatile uint32_t*>(base + o_nitems);
  const uint32_t n_items = (uint32_t)items.size();
  const igs_instruction i0{0, IGS_EPOCH, NONE, NONE, NONE, NONE, NONE, 0, 0, 0, 0};
  // the array keeps the previous call's contents: reset what must start at zero
#define CKS(x)                          \
  do {                                  \
    if ((x) != cudaSuccess) return IGS_ERR_CUDA; \
  } while (0)
  CKS(cudaMemcpyAsync(base + o_nodes, nodes.data(), sizeof(NodeDev) * N, cudaMemcpyHostToDevice, stream));
  CKS(cudaMemcpyAsync(base + o_units, units.data(), sizeof(Unit) * N, cudaMemcpyHostToDevice, stream));
  CKS(cudaMemcpyAsync(base + o_prog, &pg, sizeof pg, cudaMemcpyHostToDevice, stream));
  CKS(cudaMemcpyAsync(base + o_nitems, &n_items, sizeof n_items, cudaMemcpyHostToDevice, stream));
  if (n_items) CKS(cudaMemcpyAsync(base + o_items, items.data(), sizeof(Item) * n_items, cudaMemcpyHostToDevice, stream));
  if (num_tasks) CKS(cudaMemcpyAsync(base + o_tasks, tasks, sizeof(igs_task) * num_tasks, cudaMemcpyHostToDevice, stream));
  if (num_buffers) CKS(cudaMemcpyAsync(base + o_bufs, bd.data(), sizeof(BufDesc) * num_buffers, cudaMemcpyHostToDevice, stream));
  for (uint32_t n = 0; n < N; ++n) {
    uint8_t* nb = base + o_state + L.per_node * n;
    CKS(cudaMemsetAsync(nb + L.o_desc, 0, 4 * igs::kDesc * (2 * kBuffers + 2 * kSlots), stream));
    CKS(cudaMemsetAsync(nb + L.o_succ, 0, 1, stream));
    CKS(cudaMemcpyAsync(nb + L.o_free, slots.data(), 4 * kSlots, cudaMemcpyHostToDevice, stream));
    CKS(cudaMemcpyAsync(outs[n].instrs, &i0, sizeof i0, cudaMemcpyHostToDevice, stream));
  }
  if (igs_launch_lower(reinterpret_cast<const Unit*>(base + o_units), N, NONE, stream)) return IGS_ERR_CUDA;
  // counts and status of every node into the caller's device words
  for (uint32_t n = 0; n < N; ++n) {
    const NodeDev* nd = reinterpret_cast<const NodeDev*>(base + o_nodes) + n;
    uint32_t* cnt = outs[n].counts;
    CKS(cudaMemcpyAsync(cnt + 0, &nd->n_instr, 4, cudaMemcpyDeviceToDevice, stream));
    CKS(cudaMemcpyAsync(cnt + 1, &nd->n_edge, 4, cudaMemcpyDeviceToDevice, stream));
    CKS(cudaMemcpyAsync(cnt + 2, &nd->n_box, 4, cudaMemcpyDeviceToDevice, stream));
    CKS(cudaMemcpyAsync(cnt + 3, &nd->n_bind, 4, cudaMemcpyDeviceToDevice, stream));
    CKS(cudaMemcpyAsync(cnt + 4, &nd->n_diag, 4, cudaMemcpyDeviceToDevice, stream));
    CKS(cudaMemcpyAsync(cnt + 5, &nd->status, 4, cudaMemcpyDeviceToDevice, stream));
  }
  // tasks rejected for overlapping writes (Sec. 4.4), counted per node
  uint32_t rej[32];
  for (uint32_t n = 0; n < N; ++n)
    CKS(cudaMemcpyAsync(&rej[n], &(reinterpret_cast<const NodeDev*>(base + o_nodes) + n)->n_rej, 4,
                        cudaMemcpyDeviceToHost, stream));
  CKS(cudaStreamSynchronize(stream));
#undef CKS
  for (uint32_t n = 0; n < N; ++n)
    if (rej[n]) return IGS_ERR_OVERLAPPING_WRITE;
  return IGS_OK;
}
