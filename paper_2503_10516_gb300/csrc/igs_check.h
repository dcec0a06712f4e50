// Argument checks shared by every entry point that takes program
// descriptions (the context API and the allocation-free lowering), so that
// both accept exactly the same programs. Host code only.
#pragma once
#include <cstdint>

#include "igs.h"

namespace igs {

// igs_config.flags: only the documented variant bits.
inline bool config_flags_ok(uint32_t flags) { return (flags & ~(IGS_FLAG_STAGE_D2D | IGS_FLAG_HORIZON_CP)) == 0; }

// A buffer of 1-3 dimensions with nonzero extents (unused dimensions are
// ignored) and a nonzero element size.
inline bool buffer_shape_ok(uint32_t dims, const uint32_t extent[3], uint32_t elem_size) {
  if (dims < 1 || dims > 3 || elem_size == 0 || !extent) return false;
  for (uint32_t d = 0; d < dims; ++d)
    if (extent[d] == 0) return false;
  return true;
}

// nullptr if the task is well formed, else what is wrong with it.
// buffer_live(b): whether accessor buffer b exists and has not been destroyed.
template <class F>
inline const char* task_problem(const igs_task& t, F buffer_live) {
  if ((t.num_chunks >> 16) && ((t.num_chunks & 0xFFFFu) == 0 || t.dims < 2)) return "bad 2D split";
  if (t.dims < 1 || t.dims > 3 || t.num_chunks == 0 || t.num_accessors > IGS_MAX_ACCESSORS) return "bad task header";
  for (int d = 0; d < 3; ++d)
    if (d >= (int)t.dims && t.range[d] != 1) return "unused range dims must be 1";
  for (uint32_t a = 0; a < t.num_accessors; ++a) {
    const igs_accessor& ac = t.acc[a];
    if (!buffer_live(ac.buffer)) return "unknown buffer";
    if (ac.mode < 1 || ac.mode > 3) return "bad access mode";
    for (int d = 0; d < 3; ++d)
      if (ac.dim[d].kind > IGS_MAP_FIXED || (ac.dim[d].kind == IGS_MAP_AFFINE && ac.dim[d].a > 2))
        return "bad range mapper";
  }
  return nullptr;
}

}  // namespace igs
