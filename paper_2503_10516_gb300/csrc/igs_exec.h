// Execution-side descriptors shared by the executor (host) and its kernels.
#pragma once
#include <cstdint>

#include "igs_internal.h"

namespace igs {

// Workload kernels run by device-kernel instructions.
enum WorkloadKernel : uint32_t { K_NOP = 0, K_JACOBI = 1, K_WAVE = 2, K_NBODY_STEP = 3, K_NBODY_UPDATE = 4, K_GROW = 5, K_GENERIC = 6 };

struct KAcc {
  uint8_t* ptr;            // allocation base
  uint32_t lo[3], hi[3];   // allocation box
  uint32_t ext[3];         // buffer extent
  uint32_t dims, mode, elem, valid;
  igs_map_dim map[3];
};

struct KernelJob {
  uint32_t kernel, seq, nacc, pad;
  uint32_t lo[3], hi[3];  // chunk box (kernel index space)
  uint32_t params[4];
  uint64_t item_begin;
  KAcc acc[IGS_MAX_ACCESSORS];
};

}  // namespace igs

int igs_launch_workload(const igs::KernelJob* jobs_dev, uint32_t n_jobs, uint64_t n_items, void* stream);
// 5-point stencil jobs (Jacobi / wave), pre-validated by the host; n_jobs <= 65535.
int igs_launch_stencil(const igs::KernelJob* jobs_dev, uint32_t n_jobs, uint64_t max_items, void* stream);
// Workload out-of-allocation flag (0 = none); optionally clears it.
int igs_exec_error(bool clear);
