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
// The accumulator of the on-chip passes.  Plain binary32 and binary64 add
// the two fish of a swim pair one by one (SumAcc).  In compensated binary32
// a thread holds at most eleven pairs per step (a block's slice is at most
// 22 fish per thread), so it keeps one plain binary32 sum per fish of its
// pairs (the two lanes of a float2: w, w x, w y; one rounding per addition,
// so an error below 10 * 2^-24 of the lane's sum of magnitudes) and hands the
// warp the exact compensated pair TwoSum(lane 0, lane 1); compensation then
// runs from the warp level up (warp_tree, merge).  This takes 7 instructions
// per pair against 19 for a Kahan step per quantity.
template <int ACC>
struct OnchipAcc : SumAcc<ACC> {};

template <>
struct OnchipAcc<kAccKahan32> {
  using Sum = double;
  using Part = F2;
  float2 w = make_float2(0.f, 0.f), x = make_float2(0.f, 0.f), y = make_float2(0.f, 0.f);
  __device__ __forceinline__ Part pw() const { return two_sum(w.x, w.y); }
  __device__ __forceinline__ Part px() const { return two_sum(x.x, x.y); }
  __device__ __forceinline__ Part py() const { return two_sum(y.x, y.y); }
};

__device__ __forceinline__ float2 add_x2(float2 a, float2 b);

__device__ __forceinline__ void acc_pair(OnchipAcc<kAccPlain32>& acc, float2 wv, float2 xv,
                                         float2 yv) {
  acc.add(wv.x, xv.x, yv.x);
  acc.add(wv.y, xv.y, yv.y);
}
__device__ __forceinline__ void acc_pair(OnchipAcc<kAccF64>& acc, float2 wv, float2 xv,
                                         float2 yv) {
  acc.add(wv.x, xv.x, yv.x);
  acc.add(wv.y, xv.y, yv.y);
}
__device__ __forceinline__ void acc_pair(OnchipAcc<kAccKahan32>& acc, float2 wv, float2 xv,
                                         float2 yv) {
  acc.w = add_x2(acc.w, wv);
  acc.x = add_x2(acc.x, make_float2(__fmul_rn(wv.x, xv.x), __fmul_rn(wv.y, xv.y)));
  acc.y = add_x2(acc.y, make_float2(__fmul_rn(wv.x, yv.x), __fmul_rn(wv.y, yv.y)));
}

__device__ __forceinline__ unsigned ld_relaxed_u32(const unsigned* p) {
  unsigned v;
  asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// ------------------------------------------------ paired binary32 arithmetic --
// One instruction for the same addition or subtraction on both fish of a
// pair: each lane is rounded to nearest even on its own, subnormals kept,
// exactly as the scalar __fadd_rn / __fsub_rn (the f32x2 forms of sm_100
// and later).  Products stay scalar (__fmul_rn): a paired multiply may be
// fused by the code generator with a dependent paired add into one fused
// multiply-add, which rounds once, so it is never used.
__device__ __forceinline__ float2 add_x2(float2 a, float2 b) {
  float2 r;
  asm("{\n\t.reg .b64 pa, pb, pr;\n\t"
      "mov.b64 pa, {%2, %3};\n\tmov.b64 pb, {%4, %5};\n\t"
      "add.rn.f32x2 pr, pa, pb;\n\tmov.b64 {%0, %1}, pr;\n\t}"
      : "=f"(r.x), "=f"(r.y)
      : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
  return r;
}
__device__ __forceinline__ float2 sub_x2(float2 a, float2 b) {
  float2 r;
  asm("{\n\t.reg .b64 pa, pb, pr;\n\t"
      "mov.b64 pa, {%2, %3};\n\tmov.b64 pb, {%4, %5};\n\t"
      "sub.rn.f32x2 pr, pa, pb;\n\tmov.b64 {%0, %1}, pr;\n\t}"
      : "=f"(r.x), "=f"(r.y)
      : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
  return r;
}
__device__ __forceinline__ float2 clamp_x2(float2 v, float lo, float hi) {
  return make_float2(fminf(fmaxf(v.x, lo), hi), fminf(fmaxf(v.y, lo), hi));
}

// The swim (Sec. 2.1.2) of a fish pair: fish 0 moves by draw words 0 and 1,
// fish 1 by words 2 and 3, each coordinate by (2u - 1) * width, clamped to
// [-P, P] -- the per-fish swim() of fsb_device.cuh for two fish.
// (2u - 1) * width is formed as v * (width * 2^-23) with the integer
// v = (r >> 8) - 2^23, which equals the two-rounding form
// (v * 2^-23) * width bit for bit whenever width * 2^-23 is exact: v * 2^-23
// is exact, so both are one rounding of the same real product.  `scaled` is
// that exact width * 2^-23 for the default swim (both fish share the width),
// or 0 to use the two-rounding form with the per-fish widths `width`.
__device__ __forceinline__ void swim_pair(float2& xv, float2& yv, const Words4& r, float scaled,
                                          float2 width, float P) {
  const float vx0 = __int2float_rn(static_cast<int>(r.v[0] >> 8) - (1 << 23));
  const float vy0 = __int2float_rn(static_cast<int>(r.v[1] >> 8) - (1 << 23));
  const float vx1 = __int2float_rn(static_cast<int>(r.v[2] >> 8) - (1 << 23));
  const float vy1 = __int2float_rn(static_cast<int>(r.v[3] >> 8) - (1 << 23));
  float2 dx, dy;
  if (scaled != 0.f) {
    dx = make_float2(__fmul_rn(vx0, scaled), __fmul_rn(vx1, scaled));
    dy = make_float2(__fmul_rn(vy0, scaled), __fmul_rn(vy1, scaled));
  } else {
    dx = make_float2(__fmul_rn(__fmul_rn(vx0, 0x1p-23f), width.x),
                     __fmul_rn(__fmul_rn(vx1, 0x1p-23f), width.y));
    dy = make_float2(__fmul_rn(__fmul_rn(vy0, 0x1p-23f), width.x),
                     __fmul_rn(__fmul_rn(vy1, 0x1p-23f), width.y));
  }
  xv = clamp_x2(add_x2(xv, dx), -P, P);
  yv = clamp_x2(add_x2(yv, dy), -P, P);
}

// The default swim of a pair with the width folded into the exact scale
// `scaled` (nonzero, or the width 0): swim_pair's first form without its
// run-time choice, which measured several per cent in the per-pair loop.
__device__ __forceinline__ void swim_pair_scaled(float2& xv, float2& yv, const Words4& r,
                                                 float scaled, float P) {
  const float vx0 = __int2float_rn(static_cast<int>(r.v[0] >> 8) - (1 << 23));
  const float vy0 = __int2float_rn(static_cast<int>(r.v[1] >> 8) - (1 << 23));
  const float vx1 = __int2float_rn(static_cast<int>(r.v[2] >> 8) - (1 << 23));
  const float vy1 = __int2float_rn(static_cast<int>(r.v[3] >> 8) - (1 << 23));
  const float2 dx = make_float2(__fmul_rn(vx0, scaled), __fmul_rn(vx1, scaled));
  const float2 dy = make_float2(__fmul_rn(vy0, scaled), __fmul_rn(vy1, scaled));
  xv = clamp_x2(add_x2(xv, dx), -P, P);
  yv = clamp_x2(add_x2(yv, dy), -P, P);
}

// width * 2^-23 is exact (and nonzero unless width is 0) for width 0 or
// |width| >= 2^-103: then the scaled form of the default swim applies.
__host__ __device__ __forceinline__ bool swim_scale_exact(float width) {
  return width == 0.f || fabsf(width) >= 0x1p-103f;
}

// Objective (Sec. 2.1.1) of both fish of a pair: sqrt((x * x) + (y * y)).
__device__ __forceinline__ float2 objective_pair(float2 xv, float2 yv) {
  const float2 xx = make_float2(__fmul_rn(xv.x, xv.x), __fmul_rn(xv.y, xv.y));
  const float2 yy = make_float2(__fmul_rn(yv.x, yv.x), __fmul_rn(yv.y, yv.y));
  const float2 s = add_x2(xx, yy);
  return make_float2(__fsqrt_rn(s.x), __fsqrt_rn(s.y));
}

// width * 2^-23 when exact (width = 0, or |width| >= 2^-103 so the product
// is normal), else 0: the swim then keeps the two-rounding form.
__device__ __forceinline__ float exact_scaled_width(float width) {
  const float a = fabsf(width);
  return (a >= 0x1p-103f) ? __fmul_rn(width, 0x1p-23f) : 0.f;
}

// A block's fish.  The positions of a swim pair are one float4 (x of fish
// 0 and 1, then y of fish 0 and 1), so a pass moves them with one 16-byte
// shared-memory access.  The eat of a pass reads positions XYe and the
// feeding input De; the swim reads positions XYs and writes XYd and the next
// feeding input Dd.  An in-place pass uses one set of arrays for all; the
// resident kernel's pipelined pass eats step u from one buffer while the
// swim of step u + 2 reads the other (step u + 1's positions) and
// overwrites the first, pair by pair after its eat.  D holds a step's
// feeding input (delta, or prev - cur when feeding follows the paper's
// eat() value) -- except after the school's last swim, when it holds that
// swim's starting objective (the state's prevObjective) and the final eat
// forms the input from F and D.
struct PairState {
  const float4* XYe;
  const float2* De;
  const float4* XYs;
  float4* XYd;
  float2* Dd;
  float2* F;  // currentObjective
  float2* W;
};

// The same arrays for the eat and the swim (an in-place or one-buffer pass).
__device__ __forceinline__ PairState pair_state(const float4* XYs, const float2* Ds, float4* XYd,
                                                float2* Dd, float2* F, float2* W) {
  return PairState{XYs, Ds, XYs, XYd, Dd, F, W};
}

// ------------------------------------------------ warp barycentre partials --
// The warp's sums of eight binary32 values held by every lane, reduced and
// scattered at once: each xor level hands half of the values a lane still
// holds to its partner and adds the half it keeps, so after the levels 16,
// 8 and 4 a lane holds one value, and levels 2 and 1 finish it.  Lane L ends
// with the warp's sum of value (L >> 2) & 7 (32 terms, a fixed tree), in 32
// instructions where six separate trees take 60.
__device__ __forceinline__ float warp_scatter8(const float (&v)[8]) {
  const int lane = threadIdx.x & 31;
  const bool b16 = lane & 16, b8 = lane & 8, b4 = lane & 4;
  float k[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const float keep = b16 ? v[i + 4] : v[i];
    const float give = b16 ? v[i] : v[i + 4];
    k[i] = __fadd_rn(keep, __shfl_xor_sync(kFullMask, give, 16));
  }
  float h[2];
#pragma unroll
  for (int i = 0; i < 2; ++i) {
    const float keep = b8 ? k[i + 2] : k[i];
    const float give = b8 ? k[i] : k[i + 2];
    h[i] = __fadd_rn(keep, __shfl_xor_sync(kFullMask, give, 8));
  }
  float r = __fadd_rn(b4 ? h[1] : h[0], __shfl_xor_sync(kFullMask, b4 ? h[0] : h[1], 4));
  r = __fadd_rn(r, __shfl_xor_sync(kFullMask, r, 2));
  r = __fadd_rn(r, __shfl_xor_sync(kFullMask, r, 1));
  return r;
}

// A warp's barycentre partials (w, w x, w y) of one step into *dst, a struct
// of three Parts.  Compensated pairs: the hi and lo words are summed over the
// warp as six binary32 values (as warp_tree does, one tree each) by
// warp_scatter8, and lanes 0, 4, .., 20 write them; other types by warp_tree,
// written by lane 0.
template <typename P3, typename Part>
__device__ __forceinline__ void warp_partials(P3* dst, Part w, Part x, Part y) {
  P3 r;
  r.w = warp_tree(w);
  r.x = warp_tree(x);
  r.y = warp_tree(y);
  if ((threadIdx.x & 31) == 0) *dst = r;
}
template <typename P3>
__device__ __forceinline__ void warp_partials(P3* dst, F2 w, F2 x, F2 y) {
  static_assert(sizeof(P3) == 6 * sizeof(float), "three compensated pairs");
  const float v[8] = {w.hi, w.lo, x.hi, x.lo, y.hi, y.lo, 0.f, 0.f};
  const float s = warp_scatter8(v);
  const int lane = threadIdx.x & 31;
  if ((lane & 3) == 0 && lane < 24) reinterpret_cast<float*>(dst)[lane >> 2] = s;
}

// Per-pass context of one block.
struct PassCtx {
  Key key;
  uint32_t school;
  uint32_t pair0;  // in-school pair index of element 0
  uint32_t t;      // step counter of the pass's swim
  float N;         // feeding normaliser of the pass's eat (no feeding if <= 0)
  float scaled;    // exact s * 2^-23 for the default swim, else 0 (swim_pair)
};

// One fish pair of a pass: the eat of step p and its barycentre terms (EAT),
// then the swim of step p + 1 with its objective and maxima (SWIM).
// SCALED: the default swim with c.scaled exact (the kernel's host checks it),
// no run-time choice of the swim's form.
// LAST_SWIM: D keeps the swim's starting objectives; LAST_EAT: the feeding
// input comes from F and D.  `two`: the pair's second fish is in the school
// (a half pair's second fish is computed but neither summed nor maximised).
// AHEAD: the eat reads its own positions (Xe, Ye), else the swim's.
template <bool EAT, bool SWIM, bool LAST_SWIM, bool LAST_EAT, bool AHEAD, bool SCALED = false,
          typename Acc>
__device__ __forceinline__ void pair_pass(const PairState& B, uint32_t e, bool two,
                                          const PassCtx& c, const Physics<float>& ph, Acc& acc,
                                          float& ihi, float& ilo) {
  const float4 ps = B.XYs[e];
  float2 xv = make_float2(ps.x, ps.y), yv = make_float2(ps.z, ps.w), fv = B.F[e];
  float2 wv = (EAT || (!SCALED && ph.swim_mode)) ? B.W[e] : make_float2(0.f, 0.f);
  if (EAT) {
    const float2 dv = B.De[e];
    const float4 pe = AHEAD ? B.XYe[e] : ps;
    const float2 xe = make_float2(pe.x, pe.y), ye = make_float2(pe.z, pe.w);
    float2 g = dv;
    if (LAST_EAT) g = ph.feed_mode ? sub_x2(dv, fv) : sub_x2(fv, dv);
    {
      // w <- clamp(w + g / N, w_min, w_max), one rounding per operation, for
      // N > 0; w unchanged otherwise (selected, not branched on: a branch
      // per pair keeps the pairs of an iteration from interleaving)
      const bool feed = c.N > 0.f;
      const float Nd = feed ? c.N : 1.f;
      const float2 q = make_float2(__fdiv_rn(g.x, Nd), __fdiv_rn(g.y, Nd));
      const float2 wn = clamp_x2(add_x2(wv, q), ph.w_min, ph.w_max);
      wv = feed ? wn : wv;
    }
    if (!two) wv.y = 0.f;  // a half pair's absent fish carries no weight
    acc_pair(acc, wv, xe, ye);
    B.W[e] = wv;
  }
  if (SWIM) {
    const Words4 r = pair_draw(c.key, c.school, c.pair0 + e, c.t);
    const float2 o = fv;
    if (SCALED) {
      swim_pair_scaled(xv, yv, r, c.scaled, ph.pond_half);
    } else {
      const float2 width = ph.swim_mode
                               ? make_float2(swim_width(ph, wv.x), swim_width(ph, wv.y))
                               : make_float2(ph.step, ph.step);
      swim_pair(xv, yv, r, ph.swim_mode ? 0.f : c.scaled, width, ph.pond_half);
    }
    fv = objective_pair(xv, yv);
    const float2 i = sub_x2(o, fv);  // prev - cur
    const float2 d = sub_x2(fv, o);  // delta
    // the largest and smallest prev - cur (a half pair's absent fish
    // repeats fish 0): max |delta| = max(ihi, -ilo), max(prev - cur) = ihi
    const float i1 = two ? i.y : i.x;
    ihi = fmaxf(ihi, fmaxf(i.x, i1));
    ilo = fminf(ilo, fminf(i.x, i1));
    B.XYd[e] = make_float4(xv.x, xv.y, yv.x, yv.y);
    B.F[e] = fv;
    B.Dd[e] = LAST_SWIM ? o : (ph.feed_mode ? i : d);
  }
}

// All of this thread's pairs in one pass: elements first, first + step,
// ... below np (nf fish), where step is the number of threads that share
// the pass and first this thread's rank among them, ITER per iteration
// so that independent draws overlap (measured on GB300 over 1 to 4: the
// resident kernel runs fastest at 2, 3 within 1%; the batch kernel at 1).
// The thread's maxima of the pass's swim go into mb (bits of max |delta|)
// and ek (order key of max(prev - cur)): prev - cur is never -0 (x - x is
// +0), so the float extremes order like the keys.
template <bool EAT, bool SWIM, bool LAST_SWIM, bool LAST_EAT, bool AHEAD = false, int ITER = 2,
          bool SCALED = false, typename Acc>
__device__ __forceinline__ void block_pass_from(const PairState& B, uint32_t np, uint32_t nf,
                                                const PassCtx& c, const Physics<float>& ph,
                                                Acc& acc, uint32_t& mb, uint32_t& ek,
                                                uint32_t first, uint32_t step) {
  float ihi = -__int_as_float(0x7f800000), ilo = __int_as_float(0x7f800000);
  static_assert(ITER >= 1 && ITER <= 4, "1 to 4 pairs per iteration");
  constexpr uint32_t kIter = ITER;
  uint32_t e = first;
  for (; e + (kIter - 1) * step < np; e += kIter * step) {
#pragma unroll
    for (uint32_t k = 0; k < kIter; ++k) {
      const uint32_t ek2 = e + k * step;  // only the group's last pair can be the half pair
      pair_pass<EAT, SWIM, LAST_SWIM, LAST_EAT, AHEAD, SCALED>(
          B, ek2, k + 1 < kIter || 2 * ek2 + 1 < nf, c, ph, acc, ihi, ilo);
    }
  }
  for (; e < np; e += step)
    pair_pass<EAT, SWIM, LAST_SWIM, LAST_EAT, AHEAD, SCALED>(B, e, 2 * e + 1 < nf, c, ph, acc,
                                                             ihi, ilo);
  if (SWIM && ihi >= ilo) {  // at least one fish swum
    mb = max(mb, abs_bits(fmaxf(ihi, -ilo)));
    ek = max(ek, order_key(ihi));
  }
}

// The same pass shared by threads 0 .. step - 1 of the block.
template <bool EAT, bool SWIM, bool LAST_SWIM, bool LAST_EAT, bool AHEAD = false, int ITER = 2,
          bool SCALED = false, typename Acc>
__device__ __forceinline__ void block_pass(const PairState& B, uint32_t np, uint32_t nf,
                                           const PassCtx& c, const Physics<float>& ph, Acc& acc,
                                           uint32_t& mb, uint32_t& ek, uint32_t step) {
  block_pass_from<EAT, SWIM, LAST_SWIM, LAST_EAT, AHEAD, ITER, SCALED>(B, np, nf, c, ph, acc, mb,
                                                                       ek, threadIdx.x, step);
}

}  // namespace fsb
