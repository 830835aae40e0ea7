// fsb_reduce.cuh -- per-thread accumulators and warp reductions shared by the
// library's kernels.  All reductions run in a fixed order (xor-shuffle trees,
// fixed thread-to-data assignment), so every result is deterministic.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "fsb_internal.h"

namespace fsb {

constexpr unsigned kFullMask = 0xFFFFFFFFu;

// A binary32 value with its rounding error carried alongside (hi + lo).
struct F2 {
  float hi, lo;
};

// Knuth's TwoSum: s = fl(a + b) and the exact error e, a + b = s + e.
__device__ __forceinline__ F2 two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return {s, e};
}

// Merge operators of the three per-step partial types: binary32 (plain
// sums), compensated binary32 pairs, binary64.  Reductions run on these so
// the per-step path of the on-chip kernels issues no binary64 arithmetic in
// the binary32 modes (binary64 runs at a small fraction of the binary32
// rate on this GPU).
__device__ __forceinline__ float merge(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ double merge(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ F2 merge(F2 a, F2 b) {
  const F2 t = two_sum(a.hi, b.hi);
  return {t.hi, __fadd_rn(__fadd_rn(a.lo, b.lo), t.lo)};
}
__device__ __forceinline__ float shfl_xor(float v, int off) {
  return __shfl_xor_sync(0xFFFFFFFFu, v, off);
}
__device__ __forceinline__ double shfl_xor(double v, int off) {
  return __shfl_xor_sync(0xFFFFFFFFu, v, off);
}
__device__ __forceinline__ F2 shfl_xor(F2 v, int off) {
  return {__shfl_xor_sync(0xFFFFFFFFu, v.hi, off), __shfl_xor_sync(0xFFFFFFFFu, v.lo, off)};
}
template <typename T>
__device__ __forceinline__ T warp_merge(T v) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) v = merge(v, shfl_xor(v, off));
  return v;
}
// Intra-warp reduction of per-thread partials: compensated pairs are summed
// as two independent binary32 trees (hi and lo; five roundings each, so the
// error stays near 5 ulps of the warp's magnitudes), the exact TwoSum merge
// being kept for the cross-warp level (warp_merge).
__device__ __forceinline__ float warp_tree(float v) { return warp_merge(v); }
__device__ __forceinline__ double warp_tree(double v) { return warp_merge(v); }
__device__ __forceinline__ F2 warp_tree(F2 v) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    v.hi = __fadd_rn(v.hi, __shfl_xor_sync(0xFFFFFFFFu, v.hi, off));
    v.lo = __fadd_rn(v.lo, __shfl_xor_sync(0xFFFFFFFFu, v.lo, off));
  }
  return v;
}

__device__ __forceinline__ double to_double(float v) { return static_cast<double>(v); }
__device__ __forceinline__ double to_double(double v) { return v; }
__device__ __forceinline__ double to_double(F2 v) {
  return static_cast<double>(v.hi) + static_cast<double>(v.lo);
}
template <typename T>
__device__ __forceinline__ T part_zero();
template <>
__device__ __forceinline__ float part_zero<float>() { return 0.f; }
template <>
__device__ __forceinline__ double part_zero<double>() { return 0.0; }
template <>
__device__ __forceinline__ F2 part_zero<F2>() { return {0.f, 0.f}; }

template <int ACC>
struct SumAcc;

// Plain binary32 sums (the precision study's baseline).
template <>
struct SumAcc<kAccPlain32> {
  using Sum = float;
  using Part = float;
  float w = 0.f, x = 0.f, y = 0.f;
  __device__ __forceinline__ void add(float wi, float xi, float yi) {
    w = __fadd_rn(w, wi);
    x = __fadd_rn(x, __fmul_rn(wi, xi));
    y = __fadd_rn(y, __fmul_rn(wi, yi));
  }
  __device__ __forceinline__ void add4(const float (&wi)[4], const float (&xi)[4],
                                       const float (&yi)[4]) {
#pragma unroll
    for (int q = 0; q < 4; ++q) add(wi[q], xi[q], yi[q]);
  }
  __device__ __forceinline__ float rw() const { return w; }
  __device__ __forceinline__ float rx() const { return x; }
  __device__ __forceinline__ float ry() const { return y; }
  __device__ __forceinline__ Part pw() const { return w; }
  __device__ __forceinline__ Part px() const { return x; }
  __device__ __forceinline__ Part py() const { return y; }
};

// Kahan-compensated binary32 per thread; combined in binary64 above.
template <>
struct SumAcc<kAccKahan32> {
  using Sum = double;
  using Part = F2;
  float sw = 0.f, cw = 0.f, sx = 0.f, cx = 0.f, sy = 0.f, cy = 0.f;
  __device__ __forceinline__ static void kadd(float& s, float& c, float v) {
    const float yv = __fsub_rn(v, c);
    const float t = __fadd_rn(s, yv);
    c = __fsub_rn(__fsub_rn(t, s), yv);
    s = t;
  }
  __device__ __forceinline__ void add(float wi, float xi, float yi) {
    kadd(sw, cw, wi);
    kadd(sx, cx, __fmul_rn(wi, xi));
    kadd(sy, cy, __fmul_rn(wi, yi));
  }
  // Four fish of one vector: pairwise binary32 partial (error <= 2 ulps of
  // the four magnitudes), then one compensated add per quantity.
  __device__ __forceinline__ void add4(const float (&wi)[4], const float (&xi)[4],
                                       const float (&yi)[4]) {
    const float pw = __fadd_rn(__fadd_rn(wi[0], wi[1]), __fadd_rn(wi[2], wi[3]));
    const float px = __fadd_rn(__fadd_rn(__fmul_rn(wi[0], xi[0]), __fmul_rn(wi[1], xi[1])),
                               __fadd_rn(__fmul_rn(wi[2], xi[2]), __fmul_rn(wi[3], xi[3])));
    const float py = __fadd_rn(__fadd_rn(__fmul_rn(wi[0], yi[0]), __fmul_rn(wi[1], yi[1])),
                               __fadd_rn(__fmul_rn(wi[2], yi[2]), __fmul_rn(wi[3], yi[3])));
    kadd(sw, cw, pw);
    kadd(sx, cx, px);
    kadd(sy, cy, py);
  }
  __device__ __forceinline__ double rw() const { return double(sw) - double(cw); }
  __device__ __forceinline__ double rx() const { return double(sx) - double(cx); }
  __device__ __forceinline__ double ry() const { return double(sy) - double(cy); }
  // Kahan keeps the negated error in c: the value is s - c
  __device__ __forceinline__ Part pw() const { return {sw, -cw}; }
  __device__ __forceinline__ Part px() const { return {sx, -cx}; }
  __device__ __forceinline__ Part py() const { return {sy, -cy}; }
};

// Binary64 accumulation (products of binary32 operands are exact).
template <>
struct SumAcc<kAccF64> {
  using Sum = double;
  using Part = double;
  double w = 0.0, x = 0.0, y = 0.0;
  template <typename Real>
  __device__ __forceinline__ void add(Real wi, Real xi, Real yi) {
    const double dw = static_cast<double>(wi);
    w = __dadd_rn(w, dw);
    x = __dadd_rn(x, __dmul_rn(dw, static_cast<double>(xi)));
    y = __dadd_rn(y, __dmul_rn(dw, static_cast<double>(yi)));
  }
  template <typename Real>
  __device__ __forceinline__ void add4(const Real (&wi)[4], const Real (&xi)[4],
                                       const Real (&yi)[4]) {
#pragma unroll
    for (int q = 0; q < 4; ++q) add(wi[q], xi[q], yi[q]);
  }
  __device__ __forceinline__ double rw() const { return w; }
  __device__ __forceinline__ double rx() const { return x; }
  __device__ __forceinline__ double ry() const { return y; }
  __device__ __forceinline__ Part pw() const { return w; }
  __device__ __forceinline__ Part px() const { return x; }
  __device__ __forceinline__ Part py() const { return y; }
};

__device__ __forceinline__ float sum2(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ double sum2(double a, double b) { return __dadd_rn(a, b); }

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) v = sum2(v, __shfl_xor_sync(kFullMask, v, off));
  return v;
}

__device__ __forceinline__ uint32_t warp_max(uint32_t v) {
  return __reduce_max_sync(kFullMask, v);
}
__device__ __forceinline__ unsigned long long warp_max(unsigned long long v) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    const unsigned long long o = __shfl_xor_sync(kFullMask, v, off);
    v = o > v ? o : v;
  }
  return v;
}

// ------------------------------------------------- bounded device waits --
__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ unsigned ld_acquire_gpu(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ int ld_relaxed_gpu(const int* p) {
  int v;
  asm volatile("ld.relaxed.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Spin (one thread) until *count >= target.  Gives up, latching
// FSB_ERR_TIMEOUT into *status, after timeout_ns, and returns early when
// another block has already latched an error.  Returns true on success.
__device__ __forceinline__ bool bounded_wait_geq(const unsigned* count, unsigned target,
                                                 int* status, unsigned* site, unsigned site_id,
                                                 unsigned long long timeout_ns) {
  const unsigned long long t0 = global_ns();
  for (unsigned spins = 0;; ++spins) {
    if (ld_acquire_gpu(count) >= target) return true;
    // back off so the spinning warp does not take issue slots from the
    // block's other warps
    if (spins > 4) __nanosleep(64);
    if ((spins & 15u) == 15u) {
      if (ld_relaxed_gpu(status) != 0) return false;
      if (global_ns() - t0 > timeout_ns) {
        if (atomicCAS(status, 0, static_cast<int>(FSB_ERR_TIMEOUT)) == 0) atomicExch(site, site_id);
        return false;
      }
    }
  }
}

}  // namespace fsb
