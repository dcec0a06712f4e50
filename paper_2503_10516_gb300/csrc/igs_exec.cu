// Execution kernels: strided box copies (copy / send-receive instructions,
// paper Table 1) and the workload kernels launched by device-kernel
// instructions. Compiled with -fmad=false so the float workload kernels round
// after every operation, in the order written.
#include <cuda_runtime.h>

#include "igs_exec.h"

namespace igs {

// Set when a workload kernel meets an index outside its allocation (the
// access is skipped); read and cleared by the executor after every call.
__device__ uint32_t g_exec_error = 0;

namespace {

constexpr unsigned FULL_MASK = 0xFFFFFFFFu;

// Load policies. Kernels of the level executor read through L1 (plain) or
// with streaming hints; the dataflow executor's blocks read data that other
// blocks of the same launch wrote, so every data load there goes to L2
// (L1 is not coherent between SMs within a launch).
struct LdPlain {
  template <class T>
  __device__ __forceinline__ static T ld(const T* p) { return *p; }
};
struct LdStream {
  template <class T>
  __device__ __forceinline__ static T ld(const T* p) { return __ldcs(p); }
};
struct LdL2 {
  template <class T>
  __device__ __forceinline__ static T ld(const T* p) { return __ldcg(p); }
};

// ---- box copy ---------------------------------------------------------------
//
// A job is a 3-level strided copy: rows0 x rows1 rows of `run` contiguous
// bytes. Work units are (job, row0, row1, segment of seg_bytes); a CTA copies
// one unit at a time with 16-byte vectors when every address and the length
// allow it. The grid is persistent (a multiple of the SM count).

__device__ __forceinline__ uint32_t find_job(const CopyJob* jobs, uint32_t n, uint64_t u) {
  uint32_t lo = 0, hi = n;  // last job with unit_begin <= u
  while (hi - lo > 1) {
    const uint32_t mid = (lo + hi) >> 1;
    if (jobs[mid].unit_begin <= u) lo = mid;
    else hi = mid;
  }
  return lo;
}

// One work unit (row segment) of a copy job, by the whole block.
template <class Ld>
__device__ __forceinline__ void copy_unit(const CopyJob& J, uint64_t local) {
  {
    const uint32_t segs = (J.extent[2] + J.seg_bytes - 1) / J.seg_bytes;
    const uint64_t row = local / segs;
    const uint32_t seg = (uint32_t)(local % segs);
    const uint32_t r0 = (uint32_t)(row / J.extent[1]), r1 = (uint32_t)(row % J.extent[1]);
    const uint32_t off = seg * J.seg_bytes;
    const uint32_t len = min(J.seg_bytes, J.extent[2] - off);
    const uint8_t* s = J.src + r0 * J.src_stride[0] + r1 * J.src_stride[1] + off;
    uint8_t* d = J.dst + r0 * J.dst_stride[0] + r1 * J.dst_stride[1] + off;
    if ((((uintptr_t)s | (uintptr_t)d | len) & 15u) == 0) {
      // four independent 16-byte loads in flight per thread before the stores
      const uint4* s4 = reinterpret_cast<const uint4*>(s);
      uint4* d4 = reinterpret_cast<uint4*>(d);
      const uint32_t n4 = len >> 4, bd = blockDim.x;
      uint32_t i = threadIdx.x;
      for (; i + 3 * bd < n4; i += 4 * bd) {
        const uint4 a = Ld::ld(s4 + i), b = Ld::ld(s4 + i + bd), c = Ld::ld(s4 + i + 2 * bd),
                    e = Ld::ld(s4 + i + 3 * bd);
        __stcs(d4 + i, a);
        __stcs(d4 + i + bd, b);
        __stcs(d4 + i + 2 * bd, c);
        __stcs(d4 + i + 3 * bd, e);
      }
      for (; i < n4; i += bd) __stcs(d4 + i, Ld::ld(s4 + i));
    } else if ((((uintptr_t)s | (uintptr_t)d | len) & 3u) == 0) {
      const uint32_t* s1 = reinterpret_cast<const uint32_t*>(s);
      uint32_t* d1 = reinterpret_cast<uint32_t*>(d);
      const uint32_t n1 = len >> 2;
      for (uint32_t i = threadIdx.x; i < n1; i += blockDim.x) d1[i] = Ld::ld(s1 + i);
    } else {
      for (uint32_t i = threadIdx.x; i < len; i += blockDim.x) d[i] = Ld::ld(s + i);
    }
  }
}

__global__ void __launch_bounds__(256) box_copy_kernel(const CopyJob* __restrict__ jobs, uint32_t n_jobs,
                                                       uint64_t n_units) {
  for (uint64_t u = blockIdx.x; u < n_units; u += gridDim.x) {
    const uint32_t j = find_job(jobs, n_jobs, u);
    const CopyJob& J = jobs[j];
    copy_unit<LdStream>(J, u - J.unit_begin);
  }
}

// ---- workload kernels ---------------------------------------------------------

// Address of element p in an allocation. An index outside the accessor's
// permitted box (its range mapper's box for this chunk; Sec. 4.4 accessor
// bounds checking) is added to the accessor's out-of-bounds record. An index
// outside the allocation is skipped (nullptr); if it was permitted, that is
// an executor defect and sets the error flag.
__device__ __forceinline__ uint8_t* elem_ptr(const KAcc& a, uint32_t p0, uint32_t p1, uint32_t p2) {
  const bool permitted = a.valid && p0 >= a.plo[0] && p0 < a.phi[0] && p1 >= a.plo[1] && p1 < a.phi[1] &&
                         p2 >= a.plo[2] && p2 < a.phi[2];
  if (!permitted && a.oob) {
    atomicMax(a.oob + 0, ~p0);
    atomicMax(a.oob + 1, ~p1);
    atomicMax(a.oob + 2, ~p2);
    atomicMax(a.oob + 3, p0 + 1);
    atomicMax(a.oob + 4, p1 + 1);
    atomicMax(a.oob + 5, p2 + 1);
  }
  if (!a.valid || p0 < a.lo[0] || p0 >= a.hi[0] || p1 < a.lo[1] || p1 >= a.hi[1] || p2 < a.lo[2] || p2 >= a.hi[2]) {
    if (permitted) atomicOr(&g_exec_error, 1u);
    return nullptr;
  }
  const uint64_t w1 = a.hi[1] - a.lo[1], w2 = a.hi[2] - a.lo[2];
  return a.ptr + ((((uint64_t)(p0 - a.lo[0]) * w1) + (p1 - a.lo[1])) * w2 + (p2 - a.lo[2])) * a.elem;
}

// Low corner of the mapped box of one kernel item, false if clamped empty.
__device__ bool item_lo(const KAcc& a, const uint32_t item[3], uint32_t p[3]) {
  for (int d = 0; d < 3; ++d) {
    int64_t l, h;
    const uint32_t ext = a.ext[d];
    if (d >= (int)a.dims) {
      l = 0;
      h = 1;
    } else if (a.map[d].kind == IGS_MAP_ALL) {
      l = 0;
      h = ext;
    } else if (a.map[d].kind == IGS_MAP_FIXED) {
      l = a.map[d].a;
      h = a.map[d].b;
    } else {
      const int64_t off = (int32_t)a.map[d].b;
      l = (int64_t)item[a.map[d].a] + off - a.map[d].c;
      h = (int64_t)item[a.map[d].a] + off + a.map[d].c + 1;
    }
    l = l < 0 ? 0 : l;
    h = h > (int64_t)ext ? (int64_t)ext : h;
    if (l >= h) return false;
    p[d] = (uint32_t)l;
  }
  return true;
}

__device__ __forceinline__ uint32_t mix(uint32_t seq, uint32_t w, uint32_t lin) {
  uint32_t h = seq * 0x9E3779B1u + (w + 1u) * 0x85EBCA77u + lin * 0xC2B2AE3Du;
  h ^= h >> 15;
  h *= 0x2C1B3C6Du;
  h ^= h >> 12;
  return h;
}

template <class Ld>
__device__ __forceinline__ float ldf(const KAcc& a, uint32_t y, uint32_t x) {
  const uint8_t* p = elem_ptr(a, y, x, 0);
  return p ? Ld::ld(reinterpret_cast<const float*>(p)) : 0.0f;
}
__device__ __forceinline__ void stf(const KAcc& a, uint32_t y, uint32_t x, float v) {
  uint8_t* p = elem_ptr(a, y, x, 0);
  if (p) *reinterpret_cast<float*>(p) = v;
}
template <class Ld>
__device__ __forceinline__ float4 ld4(const KAcc& a, uint32_t i) {
  const uint8_t* p = elem_ptr(a, i, 0, 0);
  return p ? Ld::ld(reinterpret_cast<const float4*>(p)) : make_float4(0.f, 0.f, 0.f, 0.f);
}
__device__ __forceinline__ void st4(const KAcc& a, uint32_t i, float4 v) {
  uint8_t* p = elem_ptr(a, i, 0, 0);
  if (p) *reinterpret_cast<float4*>(p) = v;
}

// The N-body step's update of body y from the accelerations (same order of
// operations everywhere it is used).
__device__ __forceinline__ float4 nbody_kick(float4 v, float ax, float ay, float az) {
  v.x = v.x + ax * 0.01f;
  v.y = v.y + ay * 0.01f;
  v.z = v.z + az * 0.01f;
  return v;
}

// Adds body pj's pull on pi to the running sums (one term of the sequential
// j-sum).
__device__ __forceinline__ void nbody_term(const float4 pi, const float4 pj, float& ax, float& ay, float& az) {
  const float dx = pj.x - pi.x, dy = pj.y - pi.y, dz = pj.z - pi.z;
  const float r2 = ((dx * dx + dy * dy) + dz * dz) + 1e-6f;
  const float s = sqrtf(r2);
  const float inv = 1.0f / (r2 * s);
  const float wgt = pj.w * inv;
  ax = ax + dx * wgt;
  ay = ay + dy * wgt;
  az = az + dz * wgt;
}

template <class Ld>
__device__ void run_item(const KernelJob& J, uint32_t y, uint32_t x, uint32_t z) {
  switch (J.kernel) {
    case K_JACOBI:
    case K_WAVE: {
      const bool wave = J.kernel == K_WAVE;
      const KAcc& U = J.acc[wave ? 1 : 0];
      const KAcc& O = J.acc[wave ? 2 : 1];
      const uint32_t H = U.ext[0], W = U.ext[1];
      const float c = ldf<Ld>(U, y, x);
      float v = c;
      if (y > 0 && y + 1 < H && x > 0 && x + 1 < W) {
        const float n = ldf<Ld>(U, y - 1, x), s = ldf<Ld>(U, y + 1, x), w = ldf<Ld>(U, y, x - 1), e = ldf<Ld>(U, y, x + 1);
        if (!wave) {
          v = ((n + s) + (w + e)) * 0.25f;
        } else {
          const float pv = ldf<Ld>(J.acc[0], y, x);
          const float t2 = (2.0f * c) - pv;
          const float t5 = (n + s) + (w + e);
          const float t8 = 0.25f * (t5 - 4.0f * c);
          v = t2 + t8;
        }
      }
      stf(O, y, x, v);
      break;
    }
    case K_NBODY_STEP: {
      const KAcc& P = J.acc[0];
      const KAcc& V = J.acc[1];
      const uint32_t n = P.ext[0];
      const float4 pi = ld4<Ld>(P, y);
      float ax = 0.f, ay = 0.f, az = 0.f;
      // rows [0, n) inside both the permitted box and the allocation (one
      // row per body): no per-body check is needed
      const bool whole = P.valid && n > 0 && P.plo[0] == 0 && P.phi[0] >= n && P.lo[0] == 0 && P.hi[0] >= n &&
                         P.plo[1] == 0 && P.phi[1] >= 1 && P.plo[2] == 0 && P.phi[2] >= 1 && P.lo[1] == 0 &&
                         P.hi[1] == 1 && P.lo[2] == 0 && P.hi[2] == 1 && P.elem == 16;
      if (whole) {
        const float4* pb = reinterpret_cast<const float4*>(P.ptr);
        for (uint32_t j = 0; j < n; ++j) nbody_term(pi, Ld::ld(pb + j), ax, ay, az);
      } else {
        for (uint32_t j = 0; j < n; ++j) nbody_term(pi, ld4<Ld>(P, j), ax, ay, az);
      }
      st4(V, y, nbody_kick(ld4<Ld>(V, y), ax, ay, az));
      break;
    }
    case K_NBODY_UPDATE: {
      const float4 v = ld4<Ld>(J.acc[0], y);
      float4 p = ld4<Ld>(J.acc[1], y);
      p.x = p.x + v.x * 0.01f;
      p.y = p.y + v.y * 0.01f;
      p.z = p.z + v.z * 0.01f;
      st4(J.acc[1], y, p);
      break;
    }
    case K_GROW: {
      if (J.nacc == 1) {
        const float v = (float)((y * 131u + x * 7u) & 1023u) * 0.5f;
        stf(J.acc[0], y, x, v);
      } else {
        const uint32_t r = J.params[0];
        const uint32_t yy = y + r;
        const float last = ldf<Ld>(J.acc[0], r - 1, x);
        const float v = last * 0.5f + (float)(yy & 255u);
        stf(J.acc[1], yy, x, v);
      }
      break;
    }
    case K_SHIFT: {
      // a test kernel that may reach past its accessor's range on purpose
      const int64_t q0 = (int64_t)y + (int32_t)J.params[0], q1 = (int64_t)x + (int32_t)J.params[1],
                    q2 = (int64_t)z + (int32_t)J.params[2];
      const KAcc& A = J.acc[0];
      float v = 0.0f;
      if (q0 >= 0 && q1 >= 0 && q2 >= 0 && q0 < A.ext[0] && q1 < A.ext[1] && q2 < A.ext[2]) {
        const uint8_t* p = elem_ptr(A, (uint32_t)q0, (uint32_t)q1, (uint32_t)q2);
        if (p) v = Ld::ld(reinterpret_cast<const float*>(p));
      }
      uint8_t* d = elem_ptr(J.acc[1], y, x, z);
      if (d) *reinterpret_cast<float*>(d) = v;
      break;
    }
    case K_GENERIC: {
      const uint32_t item[3] = {y, x, z};
      uint32_t s = 0;
      for (uint32_t a = 0; a < J.nacc; ++a) {
        const KAcc& A = J.acc[a];
        if (!A.valid || !(A.mode & IGS_READ)) continue;
        uint32_t p[3];
        if (!item_lo(A, item, p)) continue;
        const uint8_t* q = elem_ptr(A, p[0], p[1], p[2]);
        if (q) s += Ld::ld(reinterpret_cast<const uint32_t*>(q));
      }
      for (uint32_t a = 0; a < J.nacc; ++a) {
        const KAcc& A = J.acc[a];
        if (!A.valid || !(A.mode & IGS_WRITE)) continue;
        uint32_t p[3];
        if (!item_lo(A, item, p)) continue;
        const uint32_t lin = (p[0] * A.ext[1] + p[1]) * A.ext[2] + p[2];
        uint8_t* q = elem_ptr(A, p[0], p[1], p[2]);
        if (q) *reinterpret_cast<uint32_t*>(q) = mix(J.seq, a, lin) + s;
      }
      break;
    }
    default:
      break;
  }
}

__device__ __forceinline__ uint32_t find_kjob(const KernelJob* jobs, uint32_t n, uint64_t u) {
  uint32_t lo = 0, hi = n;
  while (hi - lo > 1) {
    const uint32_t mid = (lo + hi) >> 1;
    if (jobs[mid].item_begin <= u) lo = mid;
    else hi = mid;
  }
  return lo;
}

// One thread per kernel item over all jobs of a wave (independent chunks).
// GENERIC reads its inputs before any write of the same item; items of one
// chunk never write a location another item of the chunk reads.
__global__ void __launch_bounds__(256) workload_kernel(const KernelJob* __restrict__ jobs, uint32_t n_jobs,
                                                       uint64_t n_items) {
  for (uint64_t u = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; u < n_items; u += (uint64_t)gridDim.x * blockDim.x) {
    const uint32_t j = find_kjob(jobs, n_jobs, u);
    const KernelJob& J = jobs[j];
    uint64_t local = u - J.item_begin;
    const uint32_t e1 = J.hi[1] - J.lo[1], e2 = J.hi[2] - J.lo[2];
    const uint32_t z = J.lo[2] + (uint32_t)(local % e2);
    local /= e2;
    const uint32_t x = J.lo[1] + (uint32_t)(local % e1);
    const uint32_t y = J.lo[0] + (uint32_t)(local / e1);
    run_item<LdPlain>(J, y, x, z);
  }
}

// 5-point stencils (Jacobi, wave) over whole chunks: one job per block row
// (blockIdx.y), four consecutive columns per thread with 16-byte loads and
// stores; the host has checked that the read allocation covers the chunk plus
// its one-element halo (clamped to the buffer) and the others cover the chunk.
__device__ __forceinline__ uint64_t stencil_groups(const KernelJob& J) {
  return (uint64_t)(J.hi[0] - J.lo[0]) * ((J.hi[1] - J.lo[1] + 3) / 4);
}

// Groups g0, g0 + stride, ... below g1 of one stencil job (a group is four
// consecutive columns of one row).
template <class Ld>
__device__ __forceinline__ void stencil_range(const KernelJob& J, uint64_t g0, uint64_t g1, uint64_t stride) {
  const bool wave = J.kernel == K_WAVE;
  const KAcc& U = J.acc[wave ? 1 : 0];
  const KAcc& O = J.acc[wave ? 2 : 1];
  const KAcc& P = J.acc[0];
  const uint32_t H = U.ext[0], W = U.ext[1];
  const uint32_t y0 = J.lo[0], x0 = J.lo[1], x1 = J.hi[1];
  const uint32_t uw = U.hi[1] - U.lo[1], ow = O.hi[1] - O.lo[1], pw = P.hi[1] - P.lo[1];
  const float* u = reinterpret_cast<const float*>(U.ptr);
  const float* pv = reinterpret_cast<const float*>(P.ptr);
  float* o = reinterpret_cast<float*>(O.ptr);
  const uint32_t groups = (x1 - x0 + 3) / 4;
  // 16-byte loads of the four columns when every row of every allocation
  // starts on a 16-byte boundary at x0
  const bool vec = ((x0 - U.lo[1]) % 4 == 0) && uw % 4 == 0 && ((x0 - O.lo[1]) % 4 == 0) && ow % 4 == 0 &&
                   (!wave || (((x0 - P.lo[1]) % 4 == 0) && pw % 4 == 0)) &&
                   ((reinterpret_cast<uintptr_t>(u) | reinterpret_cast<uintptr_t>(o) |
                     (wave ? reinterpret_cast<uintptr_t>(pv) : 0u)) & 15u) == 0;
  for (uint64_t g = g0; g < g1; g += stride) {
    const uint32_t y = y0 + (uint32_t)(g / groups);
    const uint32_t xs = x0 + 4 * (uint32_t)(g % groups);
    const float* ur = u + (size_t)(y - U.lo[0]) * uw - U.lo[1];
    const float* urn = y > 0 ? u + (size_t)(y - 1 - U.lo[0]) * uw - U.lo[1] : ur;
    const float* urs = y + 1 < H ? u + (size_t)(y + 1 - U.lo[0]) * uw - U.lo[1] : ur;
    const float* pr = wave ? pv + (size_t)(y - P.lo[0]) * pw - P.lo[1] : nullptr;
    float* orow = o + (size_t)(y - O.lo[0]) * ow - O.lo[1];
    float out[4];
    if (vec && xs + 4 <= x1) {
      // the same arithmetic, in the same order, on registers
      const float4 c4 = Ld::ld(reinterpret_cast<const float4*>(ur + xs));
      const float4 n4 = Ld::ld(reinterpret_cast<const float4*>(urn + xs));
      const float4 s4 = Ld::ld(reinterpret_cast<const float4*>(urs + xs));
      const float4 p4 = wave ? Ld::ld(reinterpret_cast<const float4*>(pr + xs)) : make_float4(0.f, 0.f, 0.f, 0.f);
      const float cs[6] = {xs > 0 ? Ld::ld(ur + xs - 1) : 0.f, c4.x, c4.y, c4.z, c4.w,
                           xs + 4 < W ? Ld::ld(ur + xs + 4) : 0.f};
      const float ns[4] = {n4.x, n4.y, n4.z, n4.w}, ss[4] = {s4.x, s4.y, s4.z, s4.w},
                  ps[4] = {p4.x, p4.y, p4.z, p4.w};
      const bool row_in = y > 0 && y + 1 < H;
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const uint32_t x = xs + k;
        const float c = cs[k + 1];
        float v = c;
        if (row_in && x > 0 && x + 1 < W) {
          const float n = ns[k], s = ss[k], w = cs[k], e = cs[k + 2];
          if (!wave) {
            v = ((n + s) + (w + e)) * 0.25f;
          } else {
            const float t2 = (2.0f * c) - ps[k];
            const float t5 = (n + s) + (w + e);
            const float t8 = 0.25f * (t5 - 4.0f * c);
            v = t2 + t8;
          }
        }
        out[k] = v;
      }
      __stcs(reinterpret_cast<float4*>(orow + xs), make_float4(out[0], out[1], out[2], out[3]));
      continue;
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const uint32_t x = xs + k;
      if (x >= x1) break;
      // streaming (evict-first) loads and stores: the stencil's data passes
      // through L2 once per step and should not displace other kernels' lines
      const float c = Ld::ld(ur + x);
      float v = c;
      if (y > 0 && y + 1 < H && x > 0 && x + 1 < W) {
        const float n = Ld::ld(urn + x), s = Ld::ld(urs + x), w = Ld::ld(ur + x - 1), e = Ld::ld(ur + x + 1);
        if (!wave) {
          v = ((n + s) + (w + e)) * 0.25f;
        } else {
          const float t2 = (2.0f * c) - Ld::ld(pr + x);
          const float t5 = (n + s) + (w + e);
          const float t8 = 0.25f * (t5 - 4.0f * c);
          v = t2 + t8;
        }
      }
      out[k] = v;
    }
    if (xs + 4 <= x1 && ((reinterpret_cast<uintptr_t>(orow + xs) & 15u) == 0)) {
      __stcs(reinterpret_cast<float4*>(orow + xs), make_float4(out[0], out[1], out[2], out[3]));
    } else {
      for (int k = 0; k < 4 && xs + k < x1; ++k) __stcs(orow + xs + k, out[k]);
    }
  }
}

// One dataflow tile of a stencil job: rows [ya, ya + kFlowStencilRows) of a
// strip of kFlowThreads groups. Each thread walks down its four columns,
// keeping the north and centre rows in registers, and takes the west and east
// neighbours from the adjacent lanes, so u is read about once per element;
// the arithmetic and its order are those of stencil_range. Warps whose groups
// are not all full 16-byte vectors take stencil_range row by row.
template <class Ld>
__device__ __forceinline__ void stencil_tile(const KernelJob& J, uint32_t t) {
  const bool wave = J.kernel == K_WAVE;
  const KAcc& U = J.acc[wave ? 1 : 0];
  const KAcc& O = J.acc[wave ? 2 : 1];
  const KAcc& P = J.acc[0];
  const uint32_t H = U.ext[0], W = U.ext[1];
  const uint32_t y0 = J.lo[0], y1 = J.hi[0], x0 = J.lo[1], x1 = J.hi[1];
  const uint32_t groups = (x1 - x0 + 3) / 4;
  const uint32_t strips = (groups + kFlowThreads - 1) / kFlowThreads;
  const uint32_t ya = y0 + (t / strips) * kFlowStencilRows, yb = min(ya + kFlowStencilRows, y1);
  const uint32_t gi = (t % strips) * kFlowThreads + threadIdx.x;
  const uint32_t glast = (t % strips) * kFlowThreads + (threadIdx.x | 31u);  // this warp's last group
  const uint32_t uw = U.hi[1] - U.lo[1], ow = O.hi[1] - O.lo[1], pw = P.hi[1] - P.lo[1];
  const float* u = reinterpret_cast<const float*>(U.ptr);
  const float* pv = reinterpret_cast<const float*>(P.ptr);
  float* o = reinterpret_cast<float*>(O.ptr);
  const bool vec = ((x0 - U.lo[1]) % 4 == 0) && uw % 4 == 0 && ((x0 - O.lo[1]) % 4 == 0) && ow % 4 == 0 &&
                   (!wave || (((x0 - P.lo[1]) % 4 == 0) && pw % 4 == 0)) &&
                   ((reinterpret_cast<uintptr_t>(u) | reinterpret_cast<uintptr_t>(o) |
                     (wave ? reinterpret_cast<uintptr_t>(pv) : 0u)) & 15u) == 0;
  if (!(vec && x0 + 4 * glast + 4 <= x1)) {
    for (uint32_t y = ya; y < yb; ++y)
      if (gi < groups) {
        const uint64_t g = (uint64_t)(y - y0) * groups + gi;
        stencil_range<Ld>(J, g, g + 1, 1);
      }
    return;
  }
  const uint32_t xs = x0 + 4 * gi, lane = threadIdx.x & 31u;
  const float* ubase = u - U.lo[1] + xs;
  const float* pbase = pv - P.lo[1] + xs;
  float4 c4 = Ld::ld(reinterpret_cast<const float4*>(ubase + (size_t)(ya - U.lo[0]) * uw));
  float4 n4 = ya > 0 ? Ld::ld(reinterpret_cast<const float4*>(ubase + (size_t)(ya - 1 - U.lo[0]) * uw)) : c4;
  // rows in batches of kRows: every load of a batch is issued before the
  // first row of the batch is computed (more bytes in flight per thread)
  constexpr uint32_t kRows = 4;
  const float4 zero = make_float4(0.f, 0.f, 0.f, 0.f);
  for (uint32_t y = ya; y < yb; y += kRows) {
    float4 sx[kRows], px[kRows];
#pragma unroll
    for (uint32_t r = 0; r < kRows; ++r) {
      const uint32_t yr = y + r;
      sx[r] = yr < yb && yr + 1 < H ? Ld::ld(reinterpret_cast<const float4*>(ubase + (size_t)(yr + 1 - U.lo[0]) * uw))
                                    : zero;
      px[r] = wave && yr < yb ? Ld::ld(reinterpret_cast<const float4*>(pbase + (size_t)(yr - P.lo[0]) * pw)) : zero;
    }
#pragma unroll
    for (uint32_t r = 0; r < kRows; ++r) {
      const uint32_t yr = y + r;
      if (yr >= yb) break;
      const float4 s4 = yr + 1 < H ? sx[r] : c4;
      const float* ur = ubase + (size_t)(yr - U.lo[0]) * uw;  // column xs of row yr
      float west = __shfl_up_sync(FULL_MASK, c4.w, 1), east = __shfl_down_sync(FULL_MASK, c4.x, 1);
      if (lane == 0) west = xs > 0 ? Ld::ld(ur - 1) : 0.f;
      if (lane == 31) east = xs + 4 < W ? Ld::ld(ur + 4) : 0.f;
      const float cs[6] = {west, c4.x, c4.y, c4.z, c4.w, east};
      const float ns[4] = {n4.x, n4.y, n4.z, n4.w}, ss[4] = {s4.x, s4.y, s4.z, s4.w},
                  ps[4] = {px[r].x, px[r].y, px[r].z, px[r].w};
      const bool row_in = yr > 0 && yr + 1 < H;
      float out[4];
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const uint32_t x = xs + k;
        const float c = cs[k + 1];
        float v = c;
        if (row_in && x > 0 && x + 1 < W) {
          const float n = ns[k], s = ss[k], w = cs[k], e = cs[k + 2];
          if (!wave) {
            v = ((n + s) + (w + e)) * 0.25f;
          } else {
            const float t2 = (2.0f * c) - ps[k];
            const float t5 = (n + s) + (w + e);
            const float t8 = 0.25f * (t5 - 4.0f * c);
            v = t2 + t8;
          }
        }
        out[k] = v;
      }
      float* orow = o + (size_t)(yr - O.lo[0]) * ow - O.lo[1];
      __stcs(reinterpret_cast<float4*>(orow + xs), make_float4(out[0], out[1], out[2], out[3]));
      n4 = c4;
      c4 = s4;
    }
  }
}

__global__ void __launch_bounds__(256) stencil_kernel(const KernelJob* __restrict__ jobs) {
  const KernelJob& J = jobs[blockIdx.y];
  stencil_range<LdStream>(J, (uint64_t)blockIdx.x * blockDim.x + threadIdx.x, stencil_groups(J),
                          (uint64_t)gridDim.x * blockDim.x);
}

// One level of the level executor in one launch: the level's stencil jobs
// (grid rows 0 .. n_sjobs-1, as stencil_kernel) and its box-copy units (the
// grid rows after them, walked as box_copy_kernel walks its units). The
// instructions of one level never depend on one another (a dependency puts
// its successor on a later level), so copies and stencils may run together.
__global__ void __launch_bounds__(256) level_kernel(const KernelJob* __restrict__ sjobs, uint32_t n_sjobs,
                                                    const CopyJob* __restrict__ cjobs, uint32_t n_cjobs,
                                                    uint64_t n_units) {
  if (blockIdx.y < n_sjobs) {
    const KernelJob& J = sjobs[blockIdx.y];
    stencil_range<LdStream>(J, (uint64_t)blockIdx.x * blockDim.x + threadIdx.x, stencil_groups(J),
                            (uint64_t)gridDim.x * blockDim.x);
    return;
  }
  const uint64_t nb = (uint64_t)(gridDim.y - n_sjobs) * gridDim.x;
  for (uint64_t u = (uint64_t)(blockIdx.y - n_sjobs) * gridDim.x + blockIdx.x; u < n_units; u += nb) {
    const uint32_t j = find_job(cjobs, n_cjobs, u);
    copy_unit<LdStream>(cjobs[j], u - cjobs[j].unit_begin);
  }
}

// ---- dataflow executor -----------------------------------------------------
//
// Out-of-order execution of an instruction graph (Sec. 3.7 / 4.1: an
// instruction may run once its predecessors have completed) inside one
// persistent launch: ready instructions are handed out tile by tile to
// whichever block asks next, so copies, kernels and transfers of different
// nodes, devices and tasks overlap without level barriers or host round trips.
// A block only ever waits when nothing is ready; every claimed tile runs to
// completion without waiting, so the launch progresses whether or not all of
// its blocks are resident.

__device__ __forceinline__ unsigned long long gtimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// N-body step over one tile of up to kFlowBodies bodies: the block stages
// kFlowBodies bodies of P at a time in shared memory (loaded from L2); each
// thread sums the terms in the same sequential j order as run_item.
__device__ __forceinline__ void nbody_tile(const KernelJob& J, uint32_t y_first, uint32_t y_end, float4* s_body) {
  const KAcc& P = J.acc[0];
  const KAcc& V = J.acc[1];
  const uint32_t n = P.ext[0];
  const uint32_t y = y_first + threadIdx.x;
  const bool mine = y < y_end;
  const float4 pi = mine ? ld4<LdL2>(P, y) : make_float4(0.f, 0.f, 0.f, 0.f);
  float ax = 0.f, ay = 0.f, az = 0.f;
  for (uint32_t j0 = 0; j0 < n; j0 += kFlowBodies) {
    const uint32_t cnt = min(kFlowBodies, n - j0);
    __syncthreads();
    if (threadIdx.x < cnt) s_body[threadIdx.x] = ld4<LdL2>(P, j0 + threadIdx.x);
    __syncthreads();
    if (mine)
      for (uint32_t k = 0; k < cnt; ++k) nbody_term(pi, s_body[k], ax, ay, az);
  }
  if (mine) st4(V, y, nbody_kick(ld4<LdL2>(V, y), ax, ay, az));
}

// Tile t of node F, by the whole block.
__device__ void run_tile(const FlowNode& F, uint32_t t, const CopyJob* __restrict__ cjobs,
                         const KernelJob* __restrict__ kjobs, float4* s_body) {
  if (F.kind == FK_COPY) {
    const uint32_t j = F.first + find_job(cjobs + F.first, F.count, t);
    copy_unit<LdL2>(cjobs[j], t - cjobs[j].unit_begin);
  } else if (F.kind == FK_STENCIL) {
    stencil_tile<LdL2>(kjobs[F.first], t);
  } else if (F.kind == FK_WORKLOAD) {
    const KernelJob& J = kjobs[F.first];
    const uint32_t e1 = J.hi[1] - J.lo[1], e2 = J.hi[2] - J.lo[2];
    const uint64_t items = (uint64_t)(J.hi[0] - J.lo[0]) * e1 * e2;
    if (J.kernel == K_NBODY_STEP) {
      // one item per body (the range is 1D)
      const uint32_t y0 = J.lo[0] + t * kFlowBodies;
      nbody_tile(J, y0, min(y0 + kFlowBodies, J.hi[0]), s_body);
      return;
    }
    const uint64_t i0 = (uint64_t)t * kFlowItems, i1 = min(i0 + kFlowItems, items);
    for (uint64_t local = i0 + threadIdx.x; local < i1; local += blockDim.x) {
      uint64_t l = local;
      const uint32_t z = J.lo[2] + (uint32_t)(l % e2);
      l /= e2;
      const uint32_t x = J.lo[1] + (uint32_t)(l % e1);
      const uint32_t y = J.lo[0] + (uint32_t)(l / e1);
      run_item<LdL2>(J, y, x, z);
    }
  }
}

__global__ void __launch_bounds__(kFlowThreads, 3) flow_kernel(FlowCtl* ctl, FlowNode* nodes, uint32_t n_nodes,
                                                            const uint32_t* __restrict__ succ, uint32_t* pending,
                                                            uint32_t* claimed, uint32_t* finished,
                                                            volatile uint32_t* ready,
                                                            const CopyJob* __restrict__ cjobs,
                                                            const KernelJob* __restrict__ kjobs, uint64_t wait_ns) {
  __shared__ uint32_t s_node, s_tile, s_cnt, s_stop;
  __shared__ float4 s_body[kFlowBodies];
  volatile FlowCtl* vc = ctl;
  for (;;) {
    if (threadIdx.x == 0) {
      uint32_t stop = 0, node = 0, tile = 0, cnt = 0, polls = 0, nap = 32;
      unsigned long long seen = vc->tiles_done, since = gtimer();
      for (;;) {
        const uint32_t h = vc->head;
        if (h >= n_nodes) {
          stop = 1;
          break;
        }
        const uint32_t q = ready[h];
        if (q != 0xFFFFFFFFu) {
          __threadfence();  // the tile's loads come after its predecessors' stores
          const uint32_t tiles = nodes[q].tiles;
          // several consecutive tiles per claim on large nodes (fewer round
          // trips per byte); a plain look first, so that blocks arriving late
          // at a node whose tiles are all taken do not pile atomics onto it
          const uint32_t k = tiles >= 64 ? 4u : tiles >= 16 ? 2u : 1u;
          const uint32_t t = *(volatile uint32_t*)&claimed[q] < tiles ? atomicAdd(&claimed[q], k) : tiles;
          if (t < tiles) {
            node = q;
            tile = t;
            cnt = min(k, tiles - t);
            if (t == 0) nodes[q].t_start = gtimer();
            break;
          }
          atomicCAS(&ctl->head, h, h + 1);  // every tile of q is taken
          nap = 32;
          continue;
        }
        // nothing ready: back off (up to about 4 us between looks, so that
        // waiting blocks do not crowd the queue's cache lines), and give up
        // if no tile finishes anywhere for wait_ns
        if ((++polls & 15u) == 0) {
          if (vc->abort) {
            stop = 1;
            break;
          }
          const unsigned long long d = vc->tiles_done, now = gtimer();
          if (d != seen) {
            seen = d;
            since = now;
          } else if (now - since > wait_ns) {
            atomicExch(&ctl->error, 1u);
            atomicExch(&ctl->abort, 1u);
            atomicOr(&g_exec_error, 2u);
            stop = 1;
            break;
          }
        }
        __nanosleep(nap);
        nap = nap < 4096 ? 2 * nap : 4096;
      }
      s_stop = stop;
      s_node = node;
      s_tile = tile;
      s_cnt = cnt;
    }
    __syncthreads();
    if (s_stop) break;
    const uint32_t q = s_node, n_run = s_cnt;
    for (uint32_t i = 0; i < n_run; ++i) run_tile(nodes[q], s_tile + i, cjobs, kjobs, s_body);
    __syncthreads();
    if (threadIdx.x == 0) {
      __threadfence();  // these tiles' stores before their count
      const uint32_t f = atomicAdd(&finished[q], n_run) + n_run;
      atomicAdd(&ctl->tiles_done, (unsigned long long)n_run);
      const FlowNode& F = nodes[q];
      if (f == F.tiles) {
        nodes[q].t_end = gtimer();
        __threadfence();
        for (uint32_t k = 0; k < F.succ_cnt; ++k) {
          const uint32_t sn = succ[F.succ_off + k];
          if (atomicSub(&pending[sn], 1u) == 1u) {
            const uint32_t pos = atomicAdd(&ctl->tail, 1u);
            ready[pos] = sn;
          }
        }
      }
    }
  }
}

}  // namespace
}  // namespace igs

int igs_launch_stencil(const igs::KernelJob* jobs_dev, uint32_t n_jobs, uint64_t max_items, void* stream) {
  if (n_jobs == 0) return 0;
  const uint64_t per_job_blocks = (max_items / 4 + 255) / 256;
  const uint32_t gx = (uint32_t)(per_job_blocks < 64 ? (per_job_blocks ? per_job_blocks : 1) : 64);
  dim3 grid(gx, n_jobs);
  igs::stencil_kernel<<<grid, 256, 0, (cudaStream_t)stream>>>(jobs_dev);
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

int igs_launch_level(const igs::KernelJob* sjobs_dev, uint32_t n_sjobs, uint64_t max_items,
                     const igs::CopyJob* cjobs_dev, uint32_t n_cjobs, uint64_t n_units, void* stream) {
  if (n_sjobs == 0 && n_units == 0) return 0;
  const uint64_t per_job_blocks = (max_items / 4 + 255) / 256;
  const uint32_t gx = (uint32_t)(per_job_blocks < 64 ? (per_job_blocks ? per_job_blocks : 1) : 64);
  int dev = 0, sms = 152;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const uint64_t want = (uint64_t)sms * 8;  // copy blocks, as igs_launch_copies
  const uint64_t cb = n_units < want ? n_units : want;
  const uint64_t crows = (cb + gx - 1) / gx;
  if (n_sjobs + crows > 65535) return -1;
  dim3 grid(gx, (uint32_t)(n_sjobs + crows));
  igs::level_kernel<<<grid, 256, 0, (cudaStream_t)stream>>>(sjobs_dev, n_sjobs, cjobs_dev, n_cjobs, n_units);
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}
int igs_launch_copies(const igs::CopyJob* jobs_dev, uint32_t n_jobs, uint64_t n_units, void* stream) {
  if (n_units == 0) return 0;
  int dev = 0, sms = 152;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const uint64_t want = (uint64_t)sms * 8;
  const uint32_t grid = (uint32_t)(n_units < want ? n_units : want);
  igs::box_copy_kernel<<<grid, 256, 0, (cudaStream_t)stream>>>(jobs_dev, n_jobs, n_units);
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

int igs_exec_error(bool clear) {
  uint32_t v = 0;
  if (cudaMemcpyFromSymbol(&v, igs::g_exec_error, sizeof v) != cudaSuccess) return -1;
  if (clear && v) {
    const uint32_t z = 0;
    cudaMemcpyToSymbol(igs::g_exec_error, &z, sizeof z);
  }
  return (int)v;
}

int igs_launch_workload(const igs::KernelJob* jobs_dev, uint32_t n_jobs, uint64_t n_items, void* stream) {
  if (n_items == 0) return 0;
  int dev = 0, sms = 152;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const uint64_t blocks = (n_items + 255) / 256;
  const uint64_t cap = (uint64_t)sms * 16;
  const uint32_t grid = (uint32_t)(blocks < cap ? blocks : cap);
  igs::workload_kernel<<<grid, 256, 0, (cudaStream_t)stream>>>(jobs_dev, n_jobs, n_items);
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

int igs_launch_flow(igs::FlowCtl* ctl, igs::FlowNode* nodes, uint32_t n_nodes, const uint32_t* succ, uint32_t* pending,
                    uint32_t* claimed, uint32_t* finished, uint32_t* ready, const igs::CopyJob* cjobs,
                    const igs::KernelJob* kjobs, uint64_t wait_ns, void* stream) {
  if (n_nodes == 0) return 0;
  static int grid = 0;
  if (!grid) {
    int dev = 0, sms = 152, per = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, igs::flow_kernel, igs::kFlowThreads, 0);
    grid = sms * (per > 0 ? per : 1);
  }
  igs::flow_kernel<<<grid, igs::kFlowThreads, 0, (cudaStream_t)stream>>>(ctl, nodes, n_nodes, succ, pending, claimed,
                                                                        finished, ready, cjobs, kjobs, wait_ns);
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

void igs_exec_preload() {
  static bool done = false;
  if (done) return;
  cudaFuncAttributes a;
  cudaFuncGetAttributes(&a, igs::box_copy_kernel);
  cudaFuncGetAttributes(&a, igs::stencil_kernel);
  cudaFuncGetAttributes(&a, igs::workload_kernel);
  cudaFuncGetAttributes(&a, igs::flow_kernel);
  done = true;
}
