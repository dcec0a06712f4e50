// Task-graph depth for the critical-path horizon cadence (Sec. 3.5: horizons
// are placed by the task graph's critical path). Host side: horizons are
// items of the submission stream, so the decision is taken where tasks are
// appended. A task's region per accessor is its range mapper applied to the
// task's whole range; the task depends on the tasks that last wrote any part
// of a region it accesses and, for a region it writes, on the tasks that read
// it since; its depth is one more than its deepest predecessor's. A horizon
// follows a task when the longest path has grown by horizon_step since the
// previous horizon. Every submitted task counts, including ones the lowering
// later rejects for overlapping writes (the decision precedes lowering).
#pragma once
#include <algorithm>
#include <cstdint>
#include <map>
#include <utility>
#include <vector>

#include "igs.h"

namespace igs {

struct TBox {
  uint32_t lo[3], hi[3];
};

inline bool tbox_empty(const TBox& b) { return b.lo[0] >= b.hi[0] || b.lo[1] >= b.hi[1] || b.lo[2] >= b.hi[2]; }

inline bool tbox_meet(const TBox& a, const TBox& b) {
  for (int d = 0; d < 3; ++d)
    if (std::max(a.lo[d], b.lo[d]) >= std::min(a.hi[d], b.hi[d])) return false;
  return true;
}

// a minus b as disjoint boxes (slabs below and above b along each dimension in turn).
inline void tbox_minus(const TBox& a, const TBox& b, std::vector<TBox>& out) {
  if (!tbox_meet(a, b)) {
    out.push_back(a);
    return;
  }
  TBox rest = a;
  for (int d = 0; d < 3; ++d) {
    if (rest.lo[d] < b.lo[d]) {
      TBox s = rest;
      s.hi[d] = b.lo[d];
      out.push_back(s);
      rest.lo[d] = b.lo[d];
    }
    if (rest.hi[d] > b.hi[d]) {
      TBox s = rest;
      s.lo[d] = b.hi[d];
      out.push_back(s);
      rest.hi[d] = b.hi[d];
    }
  }
}

// The range mapper of one accessor over the whole task range, clamped to the
// buffer (dims, extent); empty when the clamp leaves nothing.
inline TBox mapped_over_range(const igs_accessor& a, const uint32_t range[3], uint32_t dims, const uint32_t ext[3]) {
  TBox r;
  for (int d = 0; d < 3; ++d) {
    int64_t lo, hi;
    const igs_map_dim& m = a.dim[d];
    if (d >= (int)dims) {
      lo = 0;
      hi = 1;
    } else if (m.kind == IGS_MAP_ALL) {
      lo = 0;
      hi = ext[d];
    } else if (m.kind == IGS_MAP_FIXED) {
      lo = m.a;
      hi = m.b;
    } else {
      lo = (int64_t)(int32_t)m.b - (int64_t)m.c;
      hi = (int64_t)range[m.a] + (int32_t)m.b + (int64_t)m.c;
    }
    lo = std::max<int64_t>(lo, 0);
    hi = std::min<int64_t>(hi, d < (int)dims ? (int64_t)ext[d] : 1);
    if (lo >= hi) lo = hi = 0;
    r.lo[d] = (uint32_t)lo;
    r.hi[d] = (uint32_t)hi;
  }
  return r;
}

class CriticalPath {
 public:
  // Adds a task; buffer b has dims[b] dimensions and extent ext[b]. True when
  // a horizon is to follow it.
  template <class DimsOf, class ExtOf>
  bool add(const igs_task& t, DimsOf dims_of, ExtOf ext_of, uint32_t step) {
    std::vector<TBox> box(t.num_accessors);
    uint32_t deepest = 0;
    for (uint32_t a = 0; a < t.num_accessors; ++a) {
      const uint32_t b = t.acc[a].buffer;
      box[a] = mapped_over_range(t.acc[a], t.range, dims_of(b), ext_of(b));
      if (tbox_empty(box[a])) continue;
      for (const auto& e : writers_[b])
        if (tbox_meet(e.first, box[a])) deepest = std::max(deepest, depth_[e.second]);
      if (t.acc[a].mode & IGS_WRITE)
        for (const auto& e : readers_[b])
          if (tbox_meet(e.first, box[a])) deepest = std::max(deepest, depth_[e.second]);
    }
    const uint32_t me = (uint32_t)depth_.size();
    depth_.push_back(deepest + 1);
    for (uint32_t a = 0; a < t.num_accessors; ++a)
      if ((t.acc[a].mode & IGS_READ) && !tbox_empty(box[a])) readers_[t.acc[a].buffer].push_back({box[a], me});
    for (uint32_t a = 0; a < t.num_accessors; ++a) {
      if (!(t.acc[a].mode & IGS_WRITE) || tbox_empty(box[a])) continue;
      for (auto* list : {&writers_[t.acc[a].buffer], &readers_[t.acc[a].buffer]}) {
        std::vector<std::pair<TBox, uint32_t>> kept;
        std::vector<TBox> parts;
        for (const auto& e : *list) {
          parts.clear();
          tbox_minus(e.first, box[a], parts);
          for (const TBox& p : parts) kept.push_back({p, e.second});
        }
        list->swap(kept);
      }
      writers_[t.acc[a].buffer].push_back({box[a], me});
    }
    longest_ = std::max(longest_, deepest + 1);
    if (step && longest_ >= at_horizon_ + step) {
      at_horizon_ = longest_;
      return true;
    }
    return false;
  }

 private:
  std::map<uint32_t, std::vector<std::pair<TBox, uint32_t>>> writers_, readers_;
  std::vector<uint32_t> depth_;
  uint32_t longest_ = 0, at_horizon_ = 0;
};

}  // namespace igs
