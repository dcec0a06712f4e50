/* igs.h — GB300-native instruction-graph lowering and box copies (C ABI).
 *
 * Implements the data-parallel hot path of the instruction-graph scheduler of
 * "Concurrent Scheduling of High-Level Parallel Programs on Multi-GPU
 * Systems" (Knorr, Salzmann, Thoman, Fahringer): a stream of Celerity-style
 * tasks (a kernel over an index range split into chunks, with range-mapped
 * buffer accesses; Sec. 2.1, Listing 1) is lowered into per-node instruction
 * graphs — alloc, free, copy, send, receive, split receive, await receive,
 * device kernel, horizon, epoch instructions and dependency edges (Sec. 3,
 * Table 1) — with scheduler lookahead merging allocations (Sec. 4.3). The
 * emitted graph can then be executed on one GPU, virtual nodes and devices
 * being disjoint HBM partitions, box copies running as CUDA kernels.
 *
 * All lowering runs in CUDA kernels on the device (region maps stay in HBM
 * between calls); this header holds plain C types only.
 *
 * Conventions
 *   Return codes: IGS_OK (0) or a negative IGS_ERR_* code. No C++ exception
 *   crosses this boundary. igs_last_error() gives a message for the last
 *   failing call on a context.
 *   Ownership: the library owns every igs_ctx and all device state; the
 *   caller owns every pointer it passes (host_init is read during the call
 *   only; fetch/read destinations are written before the call returns).
 *   Threading: one context must not be used from two threads at once;
 *   different contexts are independent.
 *   Ids: buffer ids are dense per context in creation order. Instruction,
 *   allocation and message ids are dense per virtual node (each node builds
 *   its own instruction graph, Sec. 2.4); instruction 0 of every node is the
 *   initial epoch.
 *   Memory ids (Sec. 3.2): 0 = user host memory (host_init data, shared by
 *   all nodes), 1 = the node's pinned staging memory, 2 + d = device d of the
 *   node.
 *   Boxes: half-open [lo, hi) in three dimensions, dim 0 slowest; a
 *   1- or 2-dimensional buffer has extent 1 in its unused trailing dims.
 */
#ifndef IGS_H
#define IGS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- return codes -------------------------------------------------------- */
#define IGS_OK 0
#define IGS_ERR_INVALID_ARG -1      /* malformed descriptor, unknown buffer, bad config */
#define IGS_ERR_OVERLAPPING_WRITE -2 /* chunks of one task write overlapping regions (Sec. 4.4) */
#define IGS_ERR_CAPACITY -3         /* a device-side table or output array is full */
#define IGS_ERR_TRUNCATED -4        /* caller's fetch arrays too small; counts hold the sizes needed */
#define IGS_ERR_TIMEOUT -5          /* a bounded device-side wait gave up */
#define IGS_ERR_CUDA -6             /* a CUDA runtime call failed */
#define IGS_ERR_BUDGET -7           /* HBM admission budget exceeded (serving) */
#define IGS_ERR_STATE -8            /* call not valid in the context's current state */
#define IGS_ERR_OUT_OF_BOUNDS -9    /* a kernel accessed outside its accessor's range (Sec. 4.4) */

/* ---- instruction types (Table 1) and dependency kinds (Fig. 5 legend) ---- */
enum igs_instruction_type {
  IGS_EPOCH = 0, IGS_HORIZON = 1, IGS_ALLOC = 2, IGS_FREE = 3, IGS_COPY = 4, IGS_SEND = 5,
  IGS_RECEIVE = 6, IGS_SPLIT_RECEIVE = 7, IGS_AWAIT_RECEIVE = 8, IGS_KERNEL = 9
};
enum igs_dependency_kind {
  IGS_DEP_DATAFLOW = 1,  /* read after write */
  IGS_DEP_ANTI = 2,      /* write after read or write (anti- and output dependencies) */
  IGS_DEP_ALLOC = 4,     /* allocation lifetime: alloc -> first use, uses -> free */
  IGS_DEP_EPOCH = 8,     /* no other predecessor: depends on the last epoch / applied horizon */
  IGS_DEP_FRONT = 16     /* horizon or epoch on the execution front */
};

/* access modes (Sec. 2.1; WRITE is write_only with no_init) */
#define IGS_READ 1u
#define IGS_WRITE 2u
#define IGS_READ_WRITE 3u

/* range-mapper dimension kinds (Sec. 2.1 one_to_one / all / neighborhood; Listing 2) */
#define IGS_MAP_AFFINE 0u /* [klo[a] + (int32)b - c, khi[a] + (int32)b + c): kernel dim a, offset b, radius c */
#define IGS_MAP_ALL 1u    /* [0, extent) */
#define IGS_MAP_FIXED 2u  /* [a, b) */

#define IGS_MAX_ACCESSORS 8
#define IGS_LOOKAHEAD_INFINITE 0xFFFFFFFFu
/* lookahead value selecting the paper's horizon-count heuristic (Sec. 4.3):
 * the queue of tasks held back by an allocating task is compiled once two
 * horizons have been queued after the last task whose requirements neither a
 * live allocation nor a queued task's requirement box covers (or at an epoch
 * or a buffer destruction) */
#define IGS_LOOKAHEAD_HORIZONS 0xFFFFFFFEu
#define IGS_NONE 0xFFFFFFFFu

/* lowering modes */
#define IGS_MODE_PLAIN 0u   /* every submit lowers that task in its own launch */
#define IGS_MODE_BATCHED 1u /* submits accumulate; igs_flush / igs_lower_batch lower them in one launch */

typedef struct igs_config {
  uint32_t num_nodes;        /* virtual nodes, 1..32 */
  uint32_t devices_per_node; /* virtual devices per node, 1..29 */
  uint32_t horizon_step;     /* a horizon after every k submitted tasks; 0 = none (Sec. 3.5) */
  uint32_t lookahead;        /* scheduler lookahead window in tasks (Sec. 4.3); IGS_LOOKAHEAD_INFINITE or
                                IGS_LOOKAHEAD_HORIZONS */
  uint32_t mode;             /* IGS_MODE_PLAIN or IGS_MODE_BATCHED */
  uint32_t max_instructions; /* per node output capacity; 0 = default (1 << 18) */
  uint32_t max_edges;        /* per node; 0 = default (4 x max_instructions) */
  uint32_t max_boxes;        /* per node; 0 = default (4 x max_instructions) */
  uint32_t map_heap;         /* entries (48 bytes each) of each node's region-map heap, which holds every
                                buffer's and allocation's box tables; a table grows on demand by moving to a
                                larger slab of the heap; 0 = default (1 << 20) */
  uint32_t scratch_capacity; /* boxes per device-side scratch table, at least 32; 0 = default (4096) */
  uint32_t max_buffers;      /* buffers per context; 0 = default (64) */
  uint32_t max_live_allocs;  /* live allocations per node; 0 = default (1024) */
  uint32_t max_allocations;  /* allocation ids per node over the context's life; 0 = default (65536) */
  uint32_t max_queue;        /* submissions held by the lookahead queue; 0 = default (65536) */
  int device;                /* CUDA device ordinal */
  void* stream;              /* cudaStream_t to launch on; NULL = the library's own stream */
  uint32_t flags;            /* IGS_FLAG_* */
} igs_config;

/* Stage every device-to-device coherence copy in host memory (Sec. 3.3, for
 * devices without peer copies): a copy of region R from one device memory to
 * another of the node becomes an allocation in the node's host memory M1
 * over R's bounding box, a copy into it, a copy out of it (both carrying R's
 * canonical box list) and its free, emitted in that order in place of the
 * direct copy. */
#define IGS_FLAG_STAGE_D2D 1u
/* Horizons by the task graph's critical path (Sec. 3.5) instead of after
 * every horizon_step tasks: a task depends on the tasks that last wrote any
 * part of a region it accesses and, where it writes, on the tasks that read
 * that region since (each accessor's region = its range mapper over the
 * task's whole range); its depth is one more than its deepest
 * predecessor's; a horizon follows the task after which the largest depth
 * so far has grown by horizon_step since the previous horizon. */
#define IGS_FLAG_HORIZON_CP 2u

typedef struct igs_map_dim { uint32_t kind, a, b, c; } igs_map_dim;

typedef struct igs_accessor {
  uint32_t buffer;        /* buffer id */
  uint32_t mode;          /* IGS_READ / IGS_WRITE / IGS_READ_WRITE */
  igs_map_dim dim[3];     /* range mapper, one descriptor per buffer dimension */
} igs_accessor;

/* A task: a kernel over `range` (dims 1..3, trailing extents 1), split along
 * dim 0 into num_chunks chunks (Sec. 3.1): chunk c = rows [c*E0/C, (c+1)*E0/C)
 * on global device floor(c*M/C). If num_chunks' high 16 bits Cx are non-zero
 * (dims >= 2), the range is split along dims 0 and 1 into a Cy x Cx grid (Cy
 * = the low 16 bits): grid row iy goes to node floor(iy*N/Cy), and a node's K
 * chunks, numbered j in row-major order, to its device floor(j*D/K) (the
 * node split applied a second time among the node's devices); chunk index
 * iy*Cx + ix. Same layout as 11 + 14 * 8 uint32 words. */
typedef struct igs_task {
  uint32_t dims;
  uint32_t range[3];
  uint32_t num_chunks;    /* >= 1; bits 16-31: chunks along dim 1 (a 2D split, see above) */
  uint32_t kernel_id;     /* workload kernel run by execute: 0 none, 1 Jacobi (read 0, write 1),
                             2 wave (u_prev 0, u 1, u_next 2), 3 N-body step (positions 0, velocities 1),
                             4 N-body update (velocities 0, positions 1), 5 growing rows, 6 generic
                             integer (every accessor), 7 shifted read: accessor 1 at item := accessor 0
                             at item + (int32) params[0..2] (for bounds-checking tests) */
  uint32_t num_accessors; /* 0..8 */
  uint32_t params[4];     /* workload kernel parameters */
  igs_accessor acc[IGS_MAX_ACCESSORS];
} igs_task;

/* Output records (all uint32). Field meaning by type:
 *   ALLOC  a=allocation id, b=memory, c=buffer; boxes = [allocation box]
 *   FREE   a=allocation id, b=memory, c=buffer
 *   COPY   a=source allocation, b=destination allocation, c=buffer,
 *          d=0 coherence copy / 1 resize copy; boxes = canonical region
 *   SEND   a=staging allocation, b=target node, c=buffer, d=message id; boxes = [box]
 *   RECEIVE / SPLIT_RECEIVE  a=staging allocation, c=buffer; boxes = awaited region
 *   AWAIT_RECEIVE  a=staging allocation, b=split receive id, c=buffer; boxes = region
 *   KERNEL a=chunk index, b=memory, c=kernel id; boxes = [chunk box];
 *          bindings = one per accessor (allocation or IGS_NONE, accessed box)
 *   EPOCH / HORIZON  no fields
 * Unused fields are IGS_NONE. seq is the submission sequence number of the
 * buffer / task / horizon / epoch / destroy that emitted the instruction. */
typedef struct igs_instruction {
  uint32_t id, type, seq, a, b, c, d, box_off, box_cnt, bind_off, bind_cnt;
} igs_instruction;
typedef struct igs_edge { uint32_t from, to, kind; } igs_edge;       /* from = predecessor */
typedef struct igs_box { uint32_t lo[3], hi[3]; } igs_box;
typedef struct igs_binding { uint32_t alloc; uint32_t lo[3], hi[3]; } igs_binding;
typedef struct igs_diag { uint32_t seq, chunk, accessor; } igs_diag; /* uninitialized read (Sec. 4.4) */

/* Caller-owned destination arrays for igs_fetch_instructions. On entry the
 * *_cap fields give capacities; on return the num_* fields give the counts of
 * the whole graph of `node` so far. */
typedef struct igs_graph_view {
  uint32_t node;
  igs_instruction* instrs; uint32_t instr_cap, num_instrs;
  igs_edge* edges;         uint32_t edge_cap, num_edges;
  igs_box* boxes;          uint32_t box_cap, num_boxes;
  igs_binding* binds;      uint32_t bind_cap, num_binds;
  igs_diag* diags;         uint32_t diag_cap, num_diags;
} igs_graph_view;

typedef struct igs_ctx igs_ctx;

/* Creates a lowering context on cfg->device (Sec. 3: one instruction graph per
 * virtual node; initial epoch I0 emitted on every node). Allocates the
 * device-resident region maps and output arrays. *out is NULL on error. */
int igs_create(const igs_config* cfg, igs_ctx** out);
void igs_destroy(igs_ctx* ctx);

/* Creates a virtual buffer (Sec. 2.2, Sec. 3.2). host_init (nullable): extent
 * product x elem_size bytes, row-major, copied during the call into user
 * memory M0; NULL leaves the buffer uninitialized (reads warn, Sec. 4.4). */
int igs_create_buffer(igs_ctx* ctx, uint32_t dims, const uint32_t extent[3], uint32_t elem_size,
                      const void* host_init, uint32_t* out_buffer);

/* Drops the user's buffer: emits the frees of its backing allocations once
 * every queued task has been lowered (Sec. 3.2, last paragraph). */
int igs_destroy_buffer(igs_ctx* ctx, uint32_t buffer);

/* Submits one task (Sec. 2.1). Validates the descriptor on the host; the
 * lowering itself (chunking, mappers, push / await push, allocations,
 * coherence, transfers, dependencies) runs on the device — immediately in
 * IGS_MODE_PLAIN, at the next flush in IGS_MODE_BATCHED. A task whose chunks
 * write overlapping regions is rejected by the device (no instructions, no
 * state change) and reported by the next igs_flush / igs_sync as
 * IGS_ERR_OVERLAPPING_WRITE. *out_seq receives the task's sequence number. */
int igs_submit_task(igs_ctx* ctx, const igs_task* task, uint64_t* out_seq);

/* Sets the scheduler lookahead window (Sec. 4.3): tasks queue while an
 * allocating task is queued and are compiled once more than `window_tasks`
 * tasks are queued, or at an epoch / buffer destruction. */
int igs_set_lookahead(igs_ctx* ctx, uint32_t window_tasks);

/* Submits an epoch (Sec. 2.4): compiles every queued task, then emits an epoch
 * instruction on every node that depends on the execution front. Lowers all
 * pending submissions and waits for the device. Returns the first rejected
 * task's error, if any. */
int igs_flush(igs_ctx* ctx);

/* Lowers pending submissions (no epoch) and waits for the device. */
int igs_sync(igs_ctx* ctx);

/* Submits an epoch like igs_flush but, in IGS_MODE_BATCHED, only stages it:
 * the next igs_sync / igs_flush / igs_lower_batch lowers it. In
 * IGS_MODE_PLAIN it is lowered at once (without waiting). */
int igs_submit_epoch(igs_ctx* ctx);

/* Copies node view->node's graph (everything emitted so far) into the
 * caller's arrays. IGS_ERR_TRUNCATED if a capacity is too small (counts are
 * still filled in). */
int igs_fetch_instructions(igs_ctx* ctx, igs_graph_view* view);

/* Sequence numbers of rejected tasks: writes up to cap of them; *count = total. */
int igs_rejected_tasks(igs_ctx* ctx, uint64_t* seqs, uint32_t cap, uint32_t* count);

/* Executes every instruction emitted and not yet executed, on the device, in
 * an order that respects the graph (Sec. 3.7; by topological level or out of
 * order, see igs_set_executor): allocations from a
 * stream-ordered pool, coherence copies as box-copy kernels, device kernels
 * as the workload kernels. A send copies its box into a mailbox (device
 * memory of its own) when it executes; the receive matched to it by (task,
 * buffer, receiver) copies the mailbox into its allocation and frees it. A
 * receive whose sends have not all been lowered yet stops its node; a later
 * call continues from there. Returns when the work has completed (flags:
 * IGS_EXEC_SYNC, accepted for compatibility; execution is always complete on
 * return). */
#define IGS_EXEC_SYNC 1u
int igs_execute(igs_ctx* ctx, uint32_t flags);

/* Which executor igs_execute and igs_run use (default IGS_EXEC_LEVELS).
 * IGS_EXEC_LEVELS: the instructions of one call are grouped by topological
 * level; each level costs at most one box-copy, one stencil and one workload
 * launch, in stream order. IGS_EXEC_DATAFLOW: out-of-order execution (Sec.
 * 3.7 / 4.1: an instruction becomes ready once its predecessors have
 * completed) in ONE persistent launch per call: every instruction is a node
 * with a predecessor count and a successor list (its graph edges within the
 * call, plus send -> matching receive), its work is split into tiles (64 KiB
 * copy segments, stencil tiles of 16 rows x 1024 columns, 1024-item workload tiles, 256
 * N-body bodies) and blocks take tiles of whichever nodes are ready, so
 * copies, kernels and transfers of different devices, nodes and tasks run
 * concurrently. A split receive becomes one copy per incoming send, and
 * each await receive completes once the sends meeting its region have landed
 * (Sec. 3.4 "Inbound Transfers", receive arbitration). Frees of the call run
 * after the launch. Results are identical. A launch in which no tile finishes for 2 s (a broken graph)
 * returns IGS_ERR_TIMEOUT. IGS_ERR_STATE during a pipelined run. */
#define IGS_EXEC_LEVELS 0u
#define IGS_EXEC_DATAFLOW 1u
int igs_set_executor(igs_ctx* ctx, uint32_t executor);

/* Dataflow executor statistics since the context was created: [0] launches,
 * [1] nodes, [2] tiles, [3] edges; with igs_set_timing on, from node
 * timestamps (global timer) of each launch: [4] span ms (first tile claimed to
 * last node completed), [5] ms during which some copy node was running,
 * [6] the same for kernel nodes, [7] ms during which both were (copy / kernel
 * overlap). Waits for the context's streams. */
int igs_exec_stats(igs_ctx* ctx, double out[8]);

/* Accessor bounds checking (Sec. 4.4): every element a workload kernel
 * reads or writes through an accessor is checked against the box the
 * accessor's range mapper grants the kernel's chunk (the binding box of its
 * instruction). Indices outside it are collected per (kernel instruction,
 * accessor) into a bounding box; the access itself is carried out when it lies
 * inside the allocation, skipped otherwise. After an igs_execute / igs_run
 * whose kernels produced such indices, that call returns
 * IGS_ERR_OUT_OF_BOUNDS once all work has run, and igs_bounds_errors lists
 * every record so far (the stencil fast path is only taken where the
 * permitted boxes cover everything it touches). Writes up to cap records;
 * *count = total. */
typedef struct igs_bounds_error {
  uint32_t seq;       /* submission sequence number of the task */
  uint32_t node;      /* virtual node of the kernel instruction */
  uint32_t chunk;     /* chunk index */
  uint32_t accessor;  /* accessor index within the task */
  uint32_t lo[3], hi[3];  /* bounding box of the out-of-range indices */
} igs_bounds_error;
int igs_bounds_errors(igs_ctx* ctx, igs_bounds_error* out, uint32_t cap, uint32_t* count);

/* Self-test of the dataflow executor's bounded wait on the current device:
 * launches it over a two-node cycle (a graph no lowering emits, so no node
 * ever becomes ready) with a wait limit of wait_ms (1..10000). Returns
 * IGS_ERR_TIMEOUT when every block gave up waiting and the launch ended, as
 * designed (the device stays usable), IGS_OK if the launch ended without
 * giving up (a defect), IGS_ERR_INVALID_ARG / IGS_ERR_CUDA otherwise. */
int igs_selftest_flow_wait(uint32_t wait_ms);

/* Lowers every pending submission and executes the whole graph with the
 * scheduler running ahead of the executor (Sec. 4: instruction generation
 * runs concurrently with execution, off the critical path): one launch on the
 * context's stream lowers all pending submissions, each node publishing its
 * progress after every submission to host-mapped memory; meanwhile the
 * executor fetches what has been emitted whenever every node has advanced by
 * `window` submissions and executes it on a second stream of the library's
 * own. The lowering blocks keep the executor's kernels off their SMs. The
 * emitted graph is the same as for igs_flush + igs_execute. For
 * IGS_MODE_BATCHED contexts (plain contexts lower at submission: this then
 * equals igs_execute). Returns when execution has completed;
 * IGS_ERR_OVERLAPPING_WRITE if a task was rejected (the rest ran). */
int igs_run(igs_ctx* ctx, uint32_t window);

/* Reads box [lo, hi) of a buffer, after execute, from the memory holding the
 * newest version of each element, into host_dst (row-major, elem_size each). */
int igs_read_buffer(igs_ctx* ctx, uint32_t buffer, const uint32_t lo[3], const uint32_t hi[3], void* host_dst);

/* Lowers the pending submissions of n contexts in ONE persistent launch (all
 * contexts must share a device). Waits for completion. */
int igs_lower_batch(igs_ctx* const* ctxs, uint32_t n);

/* Batched lowering shapes. persistent_blocks = 0: one block per (program,
 * node) unit, as igs_lower_batch (the other fields are ignored). Otherwise
 * that many persistent blocks of `warps` warps (1..8; 0 counts as 1) take
 * units from a device work queue, in the order `order` gives:
 * IGS_ORDER_SUBMISSION (contexts, then nodes) or IGS_ORDER_LONGEST_FIRST
 * (estimated pending work, descending; the host estimates it as pending
 * submissions plus chunk-accessor pairs per node). With warps > 1 the
 * `helped` heaviest contexts that have several devices per node get helper
 * scratch (about 4.5 KiB per scratch entry of every node, kept until the
 * context is destroyed), and the block's other warps share the per-device
 * and per-buffer phases of those contexts' nodes; other nodes are lowered by
 * the first warp alone. The graphs do not depend on the shape; the binding's
 * tune_lower_batch picks a shape by timing candidates on copies of a batch.
 * IGS_ERR_INVALID_ARG for an unknown order or more than 8 warps. Waits for
 * completion. */
#define IGS_ORDER_SUBMISSION 0u
#define IGS_ORDER_LONGEST_FIRST 1u
typedef struct igs_batch_shape {
  uint32_t persistent_blocks;
  uint32_t order;
  uint32_t warps;
  uint32_t helped;
} igs_batch_shape;
int igs_lower_batch_shaped(igs_ctx* const* ctxs, uint32_t n, const igs_batch_shape* shape);

/* ---- served lowering ------------------------------------------------------
 * A device-resident request loop (one persistent kernel, one warp per slot =
 * one node of one attached context) lowers submissions of many concurrent
 * program streams as they arrive: region maps stay on the device between
 * requests, and no launch happens per request. Contexts are admitted while the
 * slots and the HBM budget allow (footprint = the context's device arena plus
 * every buffer's bytes on every memory of every node plus its host data).
 * After igs_serve_attach, igs_submit_task / igs_submit_epoch / igs_destroy_buffer
 * on that context only publish the submission (host-mapped memory); create
 * the context's buffers before attaching. Every device wait is bounded: the
 * loop exits after idle_timeout_ms without work (restart it with
 * igs_serve_start) or when stopped. */
typedef struct igs_serve_config {
  uint32_t max_slots;         /* warps of the loop (node units), e.g. 256 */
  uint32_t idle_timeout_ms;   /* loop exits after this long without work; 0 = 10000 */
  uint64_t hbm_budget_bytes;  /* admission budget; 0 = unlimited */
  int device;
} igs_serve_config;
typedef struct igs_server igs_server;
int igs_serve_create(const igs_serve_config* cfg, igs_server** out);
void igs_serve_destroy(igs_server* srv);
/* Admits ctx (up to max_items submissions in all): IGS_ERR_BUDGET if its
 * footprint does not fit the remaining budget or too few slots are free. */
int igs_serve_attach(igs_server* srv, igs_ctx* ctx, uint32_t max_items);
/* Continuous batching (Sec. 4: the scheduler admits work while execution
 * proceeds). Admits ctx exactly like igs_serve_attach when the free slots and
 * the budget allow and no context is waiting (*admitted = 1); otherwise ctx
 * joins the server's admission queue (FIFO, *admitted = 0, IGS_OK). While it
 * waits, its submissions are kept on the host (igs_serve_progress reports
 * none taken); when a detach frees enough slots and budget, contexts are
 * admitted from the head of the queue in arrival order, their waiting
 * submissions lowered by one launch before the loop takes over. Detaching a
 * waiting context removes it from the queue (its submissions stay unlowered
 * until the next flush / sync). The submission arrays for max_items are
 * allocated here. IGS_ERR_BUDGET if ctx could never fit (more nodes than
 * slots, or a footprint above the whole budget); IGS_ERR_INVALID_ARG as for
 * igs_serve_attach. admitted may be null. */
int igs_serve_enqueue(igs_server* srv, igs_ctx* ctx, uint32_t max_items, uint32_t* admitted);
/* Server counters: [0] contexts admitted (directly or from the queue), [1]
 * admitted from the queue after a detach, [2] contexts waiting now, [3] the
 * most that waited at once, [4] slots in use, [5] budget bytes in use. */
int igs_serve_stats(const igs_server* srv, uint64_t out[8]);
/* Launches the loop if it is not running. */
int igs_serve_start(igs_server* srv);
/* Submissions published by ctx, and the number taken by every node (min over
 * its nodes). Reads host-mapped words only. */
int igs_serve_progress(const igs_ctx* ctx, uint32_t* submitted, uint32_t* taken);
/* Waits (bounded by timeout_ms) until every submission of ctx is taken, then
 * releases its slots and budget. IGS_ERR_TIMEOUT if the wait gave up. */
int igs_serve_detach(igs_server* srv, igs_ctx* ctx, uint32_t timeout_ms);
/* Stops the loop and waits for it. */
int igs_serve_stop(igs_server* srv);

/* Replays a timed trace of submissions against the served loop from a host
 * loop in the library, so that a trace is not limited by the caller's
 * submission rate: item k is submitted (igs_submit_task, or igs_submit_epoch
 * when `epoch` is 1) to ctxs[item.ctx] once arrival_ns nanoseconds have passed
 * since the call began (or at once if later), items in array order
 * (arrival_ns non-decreasing); latency_ns[k] receives the time from item k's
 * arrival until every node of its context has taken it (igs_serve_progress),
 * polled continuously. Restarts the loop if it went idle. Every context must
 * be attached to srv. IGS_ERR_TIMEOUT if the trace has not completed
 * timeout_ms after its last arrival; IGS_ERR_CAPACITY if a slot failed.
 * *wall_ns receives the time from the call's start until the last item was
 * taken. */
typedef struct igs_replay_item {
  uint32_t ctx;         /* index into ctxs */
  uint32_t epoch;       /* 1: an epoch, 0: the task `task` */
  const igs_task* task; /* caller-owned for the duration of the call */
  uint64_t arrival_ns;  /* since the start of the call */
} igs_replay_item;
int igs_serve_replay(igs_server* srv, igs_ctx* const* ctxs, uint32_t n_ctx, const igs_replay_item* items, uint32_t n,
                     uint32_t timeout_ms, uint64_t* latency_ns, uint64_t* wall_ns);
/* igs_serve_replay with flags. IGS_REPLAY_DETACH: once every item of a
 * context in the trace has been taken, the context is detached
 * (igs_serve_detach), which admits contexts waiting for admission; the
 * contexts may have been enqueued (igs_serve_enqueue) rather than attached.
 * A waiting context's items count their wait for admission in latency_ns. */
#define IGS_REPLAY_DETACH 1u
int igs_serve_replay_ex(igs_server* srv, igs_ctx* const* ctxs, uint32_t n_ctx, const igs_replay_item* items,
                        uint32_t n, uint32_t timeout_ms, uint32_t flags, uint64_t* latency_ns, uint64_t* wall_ns);

/* The comparator of the served loop, driven like igs_serve_replay: item k
 * is submitted to ctxs[item.ctx] (contexts in IGS_MODE_PLAIN, not served) at
 * its arrival time, which is one lowering launch on that context's stream;
 * latency_ns[k] = time from arrival until that launch completed (an event
 * polled continuously; contexts run concurrently, each in submission order).
 * IGS_ERR_INVALID_ARG for a served or non-plain context, IGS_ERR_TIMEOUT if
 * the trace has not completed timeout_ms after its last arrival; lowering
 * failures as igs_sync reports them. *wall_ns as for igs_serve_replay. */
int igs_replay_plain(igs_ctx* const* ctxs, uint32_t n_ctx, const igs_replay_item* items, uint32_t n,
                     uint32_t timeout_ms, uint64_t* latency_ns, uint64_t* wall_ns);

/* Per-item lowering times, off by default. While on, every lowering launch
 * records on the device when each node finished each submitted item (a
 * buffer creation, task, horizon, epoch, ...: the items in submission order,
 * horizons included). igs_item_times writes, for items [0, min(count, cap)),
 * out[2i] = the item's kind (0 buffer creation, 1 task, 2 horizon, 3 epoch,
 * 4 buffer destruction, 5 lookahead change) and out[2i + 1] = the time
 * (device clock, ns) the last node finished it, 0 if some node has not; it
 * waits for the context's stream. *count = items submitted. out may be null
 * (count only). IGS_ERR_STATE for a served or running context. */
int igs_set_item_times(igs_ctx* ctx, int on);
int igs_item_times(igs_ctx* ctx, uint64_t* out, uint32_t cap, uint32_t* count);

/* Counters: [0] instructions, [1] edges, [2] boxes, [3] map entries read,
 * [4] map entries written, [5] launches of the lowering kernel, summed over
 * nodes. */
int igs_counters(igs_ctx* ctx, uint64_t out[8]);

/* Device-time accounting (CUDA events on the context's stream around every
 * lowering launch, box-copy wave and workload-kernel wave), off by default.
 * igs_stats: [0] lowering ms, [1] box-copy ms, [2] workload ms, [3] box-copy
 * bytes (read + written), [4] lowering launches, [5] box-copy launches,
 * [6] workload launches, [7] per-launch lowering ms of the last launch. */
int igs_set_timing(igs_ctx* ctx, int on);
int igs_stats(igs_ctx* ctx, double out[8]);

/* Lowering-engine clock cycles summed over nodes, by phase: [0] chunking and
 * range mappers, [1] overlapping-write check, [2] push / await push,
 * [3] allocating test, [4] allocations, [5] pushes and sends, [6] receives,
 * [7] coherence copies, [8] kernels, [9] remote-write bookkeeping,
 * [10] horizon / epoch emission, [11] horizon / epoch compaction, [12] total
 * inside the lowering kernel; cycles spent inside [13] instruction emission,
 * [14] canonical-form computation, [15] allocation lookup (these overlap the
 * phases above). [16..30] are detail counters (region-map primitives, parts
 * of emission, call counts); they stay zero unless the library was compiled
 * with IGS_PROFILE_DETAIL. [31] counts the phases that helper warps shared
 * with a node's first warp. */
int igs_profile(igs_ctx* ctx, uint64_t out[32]);

const char* igs_last_error(const igs_ctx* ctx);

/* ---- box copies (Table 1 "copy"; a11) ------------------------------------ */
/* One strided box copy job: copy box [lo, hi) (buffer coordinates) from an
 * allocation holding box src_box at src to one holding dst_box at dst,
 * elem_size bytes per element. Both allocations are row-major over their box.
 * Pointers are device pointers. */
typedef struct igs_copy_job {
  const void* src; void* dst;
  igs_box src_box, dst_box, box;
  uint32_t elem_size;
} igs_copy_job;

/* Runs n box-copy jobs in one launch on `stream` (cudaStream_t, NULL =
 * default stream). jobs is a HOST array; the library stages it on the
 * device. Jobs must not overlap in their destinations. */
int igs_box_copy(const igs_copy_job* jobs, uint32_t n, void* stream);

/* ---- lowering without allocation ------------------------------------------
 * The paper has no counterpart to this entry point. It exists for callers that
 * cannot allocate device memory themselves: a runtime whose device memory all
 * comes from its own pool, or a latency-critical loop that must not enter the
 * driver's allocator (which can block on or synchronize with other work on the
 * device). igs_lower_static lowers a whole program (buffers, tasks, flushes,
 * buffer destructions, lookahead changes, in `ops` order) on every node into
 * caller-owned DEVICE output arrays, using a 32 MiB file-scope device array as
 * its only scratch: it calls no cudaMalloc, cudaFree or other allocating
 * routine. Every GPU that loads the library holds that array until exit.
 *   Limits: at most 16 buffers; per node at most 128 live allocations and a
 *   region-map heap of 32768 entries shared by all its box tables; the
 *   program's staged inputs plus per-node state (about 2.6 MiB + instr_cap
 *   bytes per node) must fit the array, else IGS_ERR_CAPACITY before anything
 *   runs. A capacity that runs out during the lowering (the heap, an output
 *   array) shows only in that node's status word (counts[5] = 1); the call
 *   still returns IGS_OK.
 *   Checks: the same programs as the context API are accepted (buffer shapes,
 *   task headers, accessors, config flags); a task that accesses a destroyed
 *   buffer, or a second destruction of a buffer, is IGS_ERR_INVALID_ARG.
 *   A task whose chunks write overlapping regions (Sec. 4.4) is left out of
 *   the graph, as igs_submit_task does, and the call then returns
 *   IGS_ERR_OVERLAPPING_WRITE (the outputs and counts are still written).
 *   Sharing: every call uses the same array and leaves its last contents there
 *   (each call resets what must start at zero); calls that overlap on the GPU
 *   race, so serialize them. The call synchronizes `stream` (cudaStream_t,
 *   NULL = default stream): it returns after the lowering has finished.
 *   Set-up: the first call on each device looks up the array's device address
 *   (cudaGetSymbolAddress) with that device current; make that first call
 *   before any stream capture.
 *   Outputs: outs[n] for node n; counts (device, 6 words) receives the numbers
 *   of instructions, edges, boxes, bindings, diagnostics, and the node's status
 *   (0 = ok, 1 = a capacity was exceeded, 2 = internal error). */
#define IGS_OP_CREATE_BUFFER 0u /* arg = buffer index (in creation order) */
#define IGS_OP_TASK 1u          /* arg = index into tasks */
#define IGS_OP_FLUSH 2u         /* an epoch */
#define IGS_OP_DESTROY_BUFFER 3u
#define IGS_OP_LOOKAHEAD 4u     /* arg = window */
typedef struct igs_static_buffer { uint32_t dims, extent[3], elem_size, has_init; } igs_static_buffer;
typedef struct igs_static_op { uint32_t kind, arg; } igs_static_op;
typedef struct igs_static_output {
  igs_instruction* instrs; uint32_t instr_cap;
  igs_edge* edges;         uint32_t edge_cap;
  igs_box* boxes;          uint32_t box_cap;
  igs_binding* binds;      uint32_t bind_cap;
  igs_diag* diags;         uint32_t diag_cap;
  uint32_t* counts;
} igs_static_output;
/* Where horizons go in a task sequence (host only; no device is touched):
 * horizon_after[i] = 1 when a horizon follows tasks[i], under horizon_step
 * and IGS_FLAG_HORIZON_CP in flags (else every horizon_step tasks), exactly
 * as igs_submit_task and igs_lower_static place them. Task validity is not
 * checked beyond buffer ids (IGS_ERR_INVALID_ARG). */
int igs_horizon_plan(const igs_static_buffer* bufs, uint32_t num_buffers, const igs_task* tasks, uint32_t num_tasks,
                     uint32_t horizon_step, uint32_t flags, uint8_t* horizon_after);

int igs_lower_static(const igs_config* cfg, const igs_static_buffer* bufs, uint32_t num_buffers,
                     const igs_task* tasks, uint32_t num_tasks, const igs_static_op* ops, uint32_t num_ops,
                     igs_static_output* outs, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* IGS_H */
