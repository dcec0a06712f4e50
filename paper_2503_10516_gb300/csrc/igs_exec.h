// Execution-side descriptors shared by the executor (host) and its kernels.
#pragma once
#include <cstdint>

#include "igs_internal.h"

namespace igs {

// Workload kernels run by device-kernel instructions.
enum WorkloadKernel : uint32_t {
  K_NOP = 0, K_JACOBI = 1, K_WAVE = 2, K_NBODY_STEP = 3, K_NBODY_UPDATE = 4, K_GROW = 5, K_GENERIC = 6,
  K_SHIFT = 7  // reads accessor 0 at item + offset (params 0-2, int32), writes it to accessor 1 at item
};

// Words of one accessor's out-of-bounds record: ~lo[3] then hi[3], both
// combined with atomicMax from zero (so the record is the bounding box of
// every index outside the accessor's permitted box; all zero = none).
constexpr uint32_t kOobWords = 6;

struct KAcc {
  uint8_t* ptr;            // allocation base
  uint32_t lo[3], hi[3];   // allocation box
  uint32_t plo[3], phi[3]; // permitted box: what the range mapper grants this chunk
  uint32_t* oob;           // out-of-bounds record (kOobWords), or null
  uint32_t ext[3];         // buffer extent
  uint32_t dims, mode, elem, valid;
  igs_map_dim map[3];
};

struct KernelJob {
  uint32_t kernel, seq, nacc;
  uint32_t oob_slot;  // index of the job's out-of-bounds records (IGS_MAX_ACCESSORS of them)
  uint32_t lo[3], hi[3];  // chunk box (kernel index space)
  uint32_t params[4];
  uint64_t item_begin;
  KAcc acc[IGS_MAX_ACCESSORS];
};

// ---- dataflow executor ---------------------------------------------------
// One node per instruction of an execute call; a node's work is split into
// tiles that any block may run once every predecessor node has finished.
enum FlowKind : uint32_t { FK_NONE = 0, FK_COPY = 1, FK_STENCIL = 2, FK_WORKLOAD = 3 };

// Tile sizes: a stencil tile is kFlowStencilRows rows of a strip of
// kFlowThreads groups of four columns; workload items; N-body bodies.
constexpr uint32_t kFlowThreads = 256;
constexpr uint32_t kFlowStencilRows = 16;
constexpr uint32_t kFlowItems = 1024;
constexpr uint32_t kFlowBodies = kFlowThreads;

struct FlowNode {
  uint32_t kind, first, count;  // jobs [first, first + count) of the copy or kernel job array
  uint32_t tiles;               // >= 1 (a node without work has one empty tile)
  uint32_t succ_off, succ_cnt;  // successors in the CSR array
  uint32_t pad[2];
  unsigned long long t_start, t_end;  // global timer at the first claim and at completion
};

// Queue state of one launch: ready[] receives node ids in the order they
// become ready (slots reserved at tail, filled once); blocks take tiles of
// ready[head] and move head on once all its tiles are claimed.
struct FlowCtl {
  uint32_t tail, head, abort, error;
  unsigned long long tiles_done;
  uint32_t pad[10];
};

}  // namespace igs

// Runs a dataflow graph in one persistent launch (arrays in device memory,
// laid out by the host; pending = predecessor counts, claimed / finished zero,
// ready = the initially ready nodes then 0xFFFFFFFF). A block that finds no
// ready tile waits; if no tile finishes anywhere for wait_ns the launch sets
// bit 1 of the execution error flag and every block returns.
int igs_launch_flow(igs::FlowCtl* ctl, igs::FlowNode* nodes, uint32_t n_nodes, const uint32_t* succ, uint32_t* pending,
                    uint32_t* claimed, uint32_t* finished, uint32_t* ready, const igs::CopyJob* cjobs,
                    const igs::KernelJob* kjobs, uint64_t wait_ns, void* stream);
// Loads the execution kernels' code now (once per process).
void igs_exec_preload();
int igs_launch_workload(const igs::KernelJob* jobs_dev, uint32_t n_jobs, uint64_t n_items, void* stream);
// 5-point stencil jobs (Jacobi / wave), pre-validated by the host; n_jobs <= 65535.
int igs_launch_stencil(const igs::KernelJob* jobs_dev, uint32_t n_jobs, uint64_t max_items, void* stream);
// One level's stencil jobs and box-copy units in one launch (they are
// independent by construction of the levels). -1 when the grid would exceed
// 65535 rows (the caller then launches them separately).
int igs_launch_level(const igs::KernelJob* sjobs_dev, uint32_t n_sjobs, uint64_t max_items,
                     const igs::CopyJob* cjobs_dev, uint32_t n_cjobs, uint64_t n_units, void* stream);
// Execution error flags (0 = none; bit 0: a workload kernel met an index
// outside its allocation, bit 1: a dataflow launch gave up waiting);
// optionally clears them.
int igs_exec_error(bool clear);
