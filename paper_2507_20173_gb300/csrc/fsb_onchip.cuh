// fsb_onchip.cuh -- the per-pair pass of the on-chip kernels (batched
// schools, resident single school): a block's fish live in shared memory as
// float2 pairs (fish 2e and 2e + 1 of the block's slice share element e, the
// two fish one swim draw moves), and one compact loop per pass walks this
// thread's pairs.  The code of a pass stays small, so the instruction cache
// holds it and a school of a few hundred fish costs little more than its own
// pairs.
#pragma once

#include <cstdint>

#include "fsb_device.cuh"
#include "fsb_reduce.cuh"

namespace fsb {

// ------------------------------------------------- raw per-step partials --
// A partial in the bits of one binary64 word, unconverted: binary32 in the
// low word; a compensated pair with hi in the low word and lo in the high
// word; binary64 as is.  raw_to_sum completes one (binary64 arithmetic,
// slow on this GPU) where its cost is off the per-step path.
__device__ __forceinline__ double raw_sum(float v) {
  return __longlong_as_double(static_cast<long long>(__float_as_uint(v)));
}
__device__ __forceinline__ double raw_sum(double v) { return v; }
__device__ __forceinline__ double raw_sum(F2 v) {
  return __longlong_as_double(static_cast<long long>(
      (static_cast<unsigned long long>(__float_as_uint(v.lo)) << 32) | __float_as_uint(v.hi)));
}
__device__ __forceinline__ void raw_parts(double r, float& hi, float& lo) {
  const unsigned long long b = static_cast<unsigned long long>(__double_as_longlong(r));
  hi = __uint_as_float(static_cast<uint32_t>(b));
  lo = __uint_as_float(static_cast<uint32_t>(b >> 32));
}

// The value of a raw partial of accumulation mode ACC, in that mode's Sum
// type (the compensated pair as hi + lo in binary64).
template <int ACC>
__device__ __forceinline__ typename SumAcc<ACC>::Sum raw_to_sum(double r);
template <>
__device__ __forceinline__ float raw_to_sum<kAccPlain32>(double r) {
  float hi, lo;
  raw_parts(r, hi, lo);
  return hi;
}
template <>
__device__ __forceinline__ double raw_to_sum<kAccKahan32>(double r) {
  float hi, lo;
  raw_parts(r, hi, lo);
  return to_double(F2{hi, lo});
}
template <>
__device__ __forceinline__ double raw_to_sum<kAccF64>(double r) { return r; }

// ----------------------------------------------- barycentre terms of a pair --
// The two fish of one swim pair into the accumulator: plain binary32 and
// binary64 add them one by one; compensated binary32 forms the pair's
// binary32 sums (one rounding each, exact when one weight is zero) and adds
// each with one compensated step.
__device__ __forceinline__ void add_pair(SumAcc<kAccPlain32>& acc, float w0, float x0, float y0,
                                         float w1, float x1, float y1) {
  acc.add(w0, x0, y0);
  acc.add(w1, x1, y1);
}
__device__ __forceinline__ void add_pair(SumAcc<kAccF64>& acc, float w0, float x0, float y0,
                                         float w1, float x1, float y1) {
  acc.add(w0, x0, y0);
  acc.add(w1, x1, y1);
}
__device__ __forceinline__ void add_pair(SumAcc<kAccKahan32>& acc, float w0, float x0, float y0,
                                         float w1, float x1, float y1) {
  using K = SumAcc<kAccKahan32>;
  K::kadd(acc.sw, acc.cw, __fadd_rn(w0, w1));
  K::kadd(acc.sx, acc.cx, __fadd_rn(__fmul_rn(w0, x0), __fmul_rn(w1, x1)));
  K::kadd(acc.sy, acc.cy, __fadd_rn(__fmul_rn(w0, y0), __fmul_rn(w1, y1)));
}

__device__ __forceinline__ unsigned ld_relaxed_u32(const unsigned* p) {
  unsigned v;
  asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// A block's fish.  Positions and the feeding input are read from the source
// arrays and written to the destination arrays (the same arrays for an
// in-place pass; a double-buffered pass keeps step u's positions and input
// for the eat of step u while the swim of step u + 1 writes the others).
// D holds a step's feeding input (delta, or prev - cur when feeding follows
// the paper's eat() value) -- except after the school's last swim, when it
// holds that swim's starting objective (the state's prevObjective) and the
// final eat forms the input from F and D.
struct PairState {
  const float2* Xs;
  const float2* Ys;
  const float2* Ds;
  float2* Xd;
  float2* Yd;
  float2* Dd;
  float2* F;  // currentObjective
  float2* W;
};

// Per-pass context of one block.
struct PassCtx {
  Key key;
  uint32_t school;
  uint32_t pair0;  // in-school pair index of element 0
  uint32_t t;      // step counter of the pass's swim
  float N;         // feeding normaliser of the pass's eat (no feeding if <= 0)
};

// One fish pair of a pass: the eat of step p and its barycentre terms (EAT),
// then the swim of step p + 1 with its objective and maxima (SWIM).
// LAST_SWIM: D keeps the swim's starting objectives; LAST_EAT: the feeding
// input comes from F and D.  `two`: the pair's second fish is in the school
// (a half pair's second fish is computed but neither summed nor maximised).
template <bool EAT, bool SWIM, bool LAST_SWIM, bool LAST_EAT, typename Acc>
__device__ __forceinline__ void pair_pass(const PairState& B, uint32_t e, bool two,
                                          const PassCtx& c, const Physics<float>& ph, Acc& acc,
                                          uint32_t& mb, uint32_t& ek) {
  float2 xv = B.Xs[e], yv = B.Ys[e], fv = B.F[e];
  float2 wv = (EAT || ph.swim_mode) ? B.W[e] : make_float2(0.f, 0.f);
  if (EAT) {
    const float2 dv = B.Ds[e];
    float g0 = dv.x, g1 = dv.y;
    if (LAST_EAT) {
      g0 = ph.feed_mode ? __fsub_rn(dv.x, fv.x) : __fsub_rn(fv.x, dv.x);
      g1 = ph.feed_mode ? __fsub_rn(dv.y, fv.y) : __fsub_rn(fv.y, dv.y);
    }
    if (c.N > 0.f) {
      wv.x = eat(wv.x, g0, c.N, ph);
      wv.y = eat(wv.y, g1, c.N, ph);
    }
    add_pair(acc, wv.x, xv.x, yv.x, two ? wv.y : 0.f, xv.y, yv.y);
    B.W[e] = wv;
  }
  if (SWIM) {
    const Words4 r = pair_draw(c.key, c.school, c.pair0 + e, c.t);
    const float o0 = fv.x, o1 = fv.y;
    swim(xv.x, yv.x, r.v[0], r.v[1], swim_width(ph, wv.x), ph);
    swim(xv.y, yv.y, r.v[2], r.v[3], swim_width(ph, wv.y), ph);
    fv.x = objective(xv.x, yv.x);
    fv.y = objective(xv.y, yv.y);
    const float i0 = __fsub_rn(o0, fv.x), i1 = __fsub_rn(o1, fv.y);  // prev - cur
    const float d0 = __fsub_rn(fv.x, o0), d1 = __fsub_rn(fv.y, o1);  // delta
    const uint32_t m0 = abs_bits(d0), q0 = order_key(i0);
    const uint32_t m1 = two ? abs_bits(d1) : 0u, q1 = two ? order_key(i1) : 0u;
    mb = max(mb, max(m0, m1));
    ek = max(ek, max(q0, q1));
    B.Xd[e] = xv;
    B.Yd[e] = yv;
    B.F[e] = fv;
    B.Dd[e] = LAST_SWIM ? make_float2(o0, o1)
                        : (ph.feed_mode ? make_float2(i0, i1) : make_float2(d0, d1));
  }
}

// All of this thread's pairs in one pass: elements threadIdx.x,
// threadIdx.x + step, ... below np (nf fish), where step is the number of
// threads that share the pass (threads 0 .. step - 1), two per iteration so
// that two independent draws overlap.
template <bool EAT, bool SWIM, bool LAST_SWIM, bool LAST_EAT, typename Acc>
__device__ __forceinline__ void block_pass(const PairState& B, uint32_t np, uint32_t nf,
                                           const PassCtx& c, const Physics<float>& ph, Acc& acc,
                                           uint32_t& mb, uint32_t& ek, uint32_t step) {
  uint32_t e = threadIdx.x;
  for (; e + step < np; e += 2 * step) {
    pair_pass<EAT, SWIM, LAST_SWIM, LAST_EAT>(B, e, true, c, ph, acc, mb, ek);
    const uint32_t e2 = e + step;
    pair_pass<EAT, SWIM, LAST_SWIM, LAST_EAT>(B, e2, 2 * e2 + 1 < nf, c, ph, acc, mb, ek);
  }
  if (e < np) pair_pass<EAT, SWIM, LAST_SWIM, LAST_EAT>(B, e, 2 * e + 1 < nf, c, ph, acc, mb, ek);
}

}  // namespace fsb
