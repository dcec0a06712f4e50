// Internal structures shared by the lowering engine, the executor and the
// host front-end of libigs. Not part of the public C ABI (include/igs.h).
#pragma once
#include <cstddef>
#include <cstdint>

#include "igs.h"

namespace igs {

constexpr uint32_t NONE = 0xFFFFFFFFu;
constexpr uint32_t REMOTE = 0xFFFFFFFEu;  // producer: written by another node
constexpr uint32_t HOST = 0xFFFFFFFEu;    // owner: user host memory, present on every node
constexpr uint32_t DEAD = 0xFFFFFFFFu;    // table key of a removed entry

enum ItemKind : uint32_t { IT_CREATE = 0, IT_TASK = 1, IT_HORIZON = 2, IT_EPOCH = 3, IT_DESTROY = 4, IT_LOOKAHEAD = 5 };

// One submission as seen by every node's lowering warp.
struct Item {
  uint32_t kind, seq, arg, task;  // arg: buffer id / lookahead; task: index into the task array
};

struct BufDesc {
  uint32_t dims, extent[3], elem, init;
};

enum Status : uint32_t { ST_OK = 0, ST_CAPACITY = 1, ST_INTERNAL = 2, ST_TIMEOUT = 3 };

// What ran out on ST_CAPACITY: NodeDev::err_info = kind << 24 | capacity.
enum CapKind : uint32_t {
  CAP_TABLE = 1, CAP_HEAP = 2, CAP_ALLOC = 3, CAP_EDGE = 4, CAP_BOX = 5, CAP_BIND = 6, CAP_DIAG = 7,
  CAP_BUFFERS = 8, CAP_QUEUE = 9
};

// Field layout of a box-table entry: 12 words (48 bytes, 16-byte aligned) so
// an entry loads with three 16-byte vector loads; F_COUNT is the stride.
enum TableField : int { F_KEY = 0, F_LO = 1, F_HI = 4, F_V = 7, F_COUNT = 12 };

struct Table {
  uint32_t* base;  // cap entries of F_COUNT words
  uint32_t n, cap;
  uint32_t live;   // entries not marked dead
  uint32_t* dp;    // heap table descriptor {offset, cap, n, live, merge mark}; nullptr for scratch tables
};

// Warps that share parts of a node's lowering (warp 0 and up to 7 helpers),
// and the scratch tables of each helper.
constexpr uint32_t kMaxWorkers = 8;
constexpr uint32_t kHelperTables = 12;
// Scratch sets in a node's helper scratch: one per worker, plus one for the
// front warp that runs push / await push ahead of warp 0 (pipelined launches).
constexpr uint32_t kScratchSets = kMaxWorkers + 1;

// Size classes of the per-node entry heap: 32 << k entries.
constexpr int kHeapClasses = 24;
// Words per heap-table descriptor: {offset, cap, n, live, merge mark, 3 spare}.
constexpr uint32_t kDesc = 8;

struct AllocRec {
  uint32_t buffer, mem, live, user;
  uint32_t lo[3], hi[3];
  uint32_t mark;  // scratch: cluster index during allocation planning
  uint32_t slot;  // slab of its writer / reader tables
};

// Persistent device state of one virtual node's lowering (one warp owns it).
struct NodeDev {
  // configuration
  uint32_t node, N, D, prog;
  // scalars (owned by the warp; written back after every item)
  uint32_t status, err_info, cursor, lookahead, epoch, last_horizon, last_sync, next_msg, n_alloc;
  uint32_t n_instr, n_edge, n_box, n_bind, n_diag, n_rej;
  uint32_t q_head, q_count, qr_n, n_free, n_live, qr_live;
  uint32_t q_hzn;  // horizon-count lookahead: horizons queued since the last allocating task
  uint32_t stage_d2d;  // device-to-device copies staged in host memory (IGS_FLAG_STAGE_D2D)
  uint64_t map_reads, map_writes, launches;
  uint64_t prof[32];   // clock cycles per lowering phase and detail counters (see the engine)
  // capacities
  uint32_t cap_instr, cap_edge, cap_box, cap_bind, cap_diag, cap_rej, cap_alloc, cap_queue;
  uint32_t cap_buffers, cap_slots, cap_qr, cap_scratch;
  // entry heap holding every region-map table of the node (size classes,
  // free lists threaded through the first word of a free slab)
  uint32_t* heap;      // cap_heap entries of F_COUNT words
  uint32_t cap_heap, heap_top;
  uint32_t free_head[kHeapClasses];
  // table descriptors (kDesc words, {offset, cap, n, live, merge mark}): per buffer the node-level
  // ownership map and the local buffer state; per allocation slot its last
  // writers and readers since the last write
  uint32_t* own_d;
  uint32_t* bst_d;
  uint32_t* wr_d;
  uint32_t* rd_d;
  uint32_t* free_slots;
  uint32_t* live;      // ids of live allocations, ascending
  // per-task push and await regions (key = task sequence number)
  uint32_t* qr_base;
  AllocRec* allocs;
  uint32_t* queue;     // item indices (ring of cap_queue)
  uint8_t* has_succ;   // per instruction: has a successor
  // outputs (same record layouts as the public structs)
  igs_instruction* instrs;
  igs_edge* edges;
  igs_box* boxes;
  igs_binding* binds;
  igs_diag* diags;
  uint32_t* rejected;
  // scratch tables for the warp
  uint32_t* scratch_base;  // 14 tables of cap_scratch entries
  // scratch of the warps that share parts of the lowering when a node is
  // lowered by several warps (kScratchSets x kHelperTables tables of
  // cap_scratch entries), or null
  uint32_t* helper_scratch;
  // completion time (%globaltimer, ns) of each item, by item index, written
  // by the lowering warp when item timing is on; null otherwise
  uint64_t* item_ts;
};

// Program-level inputs shared by all node warps of one context.
struct ProgDev {
  const Item* items;
  const igs_task* tasks;
  const BufDesc* bufs;
  volatile uint32_t* n_items;  // number of valid items (host-mapped in serving)
  // serving: submissions arrive in host-mapped memory; a warp copies each
  // new item and its task into `items` / `tasks` (device memory) once and
  // lowers from there. nullptr when not served.
  const Item* src_items;
  const igs_task* src_tasks;
};

// A unit of lowering work: one node of one program.
struct Unit {
  NodeDev* node;
  ProgDev* prog;
};

// Progress record of one lowering unit (host-mapped): written by the unit's
// warp after each submission, cursor last.
enum ProgressWord : uint32_t { PR_CURSOR = 0, PR_INSTR = 1, PR_EDGE = 2, PR_BOX = 3, PR_BIND = 4, PR_STATUS = 5, PR_WORDS = 8 };

// One slot of the serving loop (host-mapped memory): a warp serves the unit
// while `state` is SLOT_ACTIVE and publishes how many submissions it has
// taken in `done`.
enum SlotState : uint32_t { SLOT_EMPTY = 0, SLOT_ACTIVE = 1 };
enum SlotExit : uint32_t { EXIT_NONE = 0, EXIT_STOPPED = 1, EXIT_IDLE = 2, EXIT_ERROR = 3 };
struct ServeSlot {
  Unit unit;
  volatile uint32_t state, done, status, exit, busy, pad;
};

// Box-copy work descriptor (device side).
struct CopyJob {
  const uint8_t* src;
  uint8_t* dst;
  uint64_t src_stride[2], dst_stride[2];  // bytes per step of dim 0 / dim 1 (after collapsing)
  uint32_t extent[3];                     // rows0, rows1, contiguous bytes per row
  uint32_t seg_bytes;                     // bytes per work unit along the row
  uint64_t unit_begin;                    // prefix of work units
};

}  // namespace igs

// Device entry points implemented in the .cu translation units.
// Persistent blocks of `warps` warps (1..kMaxWorkers) pulling units from a
// device work queue (*head, zero before the launch) in the order order_dev
// (null = index order); extra warps help nodes that have helper scratch.
int igs_launch_lower_queue(const igs::Unit* units_dev, uint32_t n_units, const uint32_t* order_dev, uint32_t* head_dev,
                           uint32_t blocks, uint32_t warps, void* stream);
// One block per unit.
// reserve: each unit's block also holds most of its SM's registers, keeping
// other kernels off the SMs that lower (used while the executor runs concurrently).
// progress (host-mapped, PR_WORDS per unit, or null): each unit publishes its
// cursor and output counts after every submission it lowers.
// workers: blocks of kMaxWorkers warps, so that helper warps share each
// node's kernel phase (when the node has helper scratch).
int igs_launch_lower(const igs::Unit* units_dev, uint32_t n_units, uint32_t max_items, void* stream,
                     bool reserve = false, volatile uint32_t* progress = nullptr, bool workers = false);
// Persistent serving loop over n_slots slots; exits when *stop is set or a
// warp stays idle for idle_polls polls (about 2 us each).
int igs_launch_serve(igs::ServeSlot* slots, uint32_t n_slots, volatile uint32_t* stop, uint64_t idle_polls, void* stream);
int igs_launch_copies(const igs::CopyJob* jobs_dev, uint32_t n_jobs, uint64_t n_units, void* stream);
