// fsb_collective.cu -- the streaming step with the collective movements of
// fish-school search (collective_mode 1, a variant beyond the paper).
//
// Each step t adds two moves after the eat: every fish moves by the school's
// instinctive vector I_t (the improvement-weighted mean of the improving
// fish's swim displacements), then along the line through the school's
// barycentre B_t, toward it if the school's weight grew in the step and away
// from it otherwise, by s_vol u with its own draw u.  I_t needs sums over the
// swim of step t; B_t needs sums over the positions after the instinctive
// move, so a step takes two passes over the school:
//
//   swim0   (once per call) swim of the first step; its maxima, its
//           instinctive sums, and the school's weight on the grid before
//           the first eat
//   eat t   eat of step t and the barycentre sums the step reports, then the
//           instinctive move, then the exact barycentre sums
//   move t  volitive move of step t, then (unless t is the call's last step)
//           the swim of step t + 1 with its maxima and instinctive sums
//
// School sums that feed back into positions are exact: each term is rounded
// once onto a fixed grid (v * 2^k to the nearest integer, ties to even) and
// the 64-bit integers add exactly in any order, so every block, warp and
// fold order gives the same vector and barycentre as the one-fish-at-a-time
// CPU definition.  The grid exponents come from the school's configuration
// (the host's collective_grids).  Each thread runs fish pairs, so one swim
// draw and one volitive draw (Philox domain 2) serve two fish.
#include <cstdint>

#include "fsb_device.cuh"
#include "fsb_internal.h"
#include "fsb_reduce.cuh"

namespace fsb {
namespace {

constexpr uint32_t kDomainVolitive = 2u;
constexpr int kCollBlock = 256;

template <typename Real>
struct CollArgs {
  Real* __restrict__ x;
  Real* __restrict__ y;
  Real* __restrict__ w;
  Real* __restrict__ pv;
  uint64_t n;
  Key key;
  uint32_t school;
  Physics<Real> ph;
  Real s_vol;
  Real g_p, g_g, g_w;  // grid scales 2^kp, 2^kg, 2^kw (exact)
  int kp, kg;
  Ctl* ctl;
  CollPartial* partials;
  fsb_step_stats* ring;
  CollRec* coll;
  uint32_t n_steps;
  int vec2;            // every array aligned to 2 elements: pair loads
};

// One fish pair's state as loaded: fish 2p (and 2p + 1 when nf = 2).
template <typename Real>
struct PairIn {
  Real x[2], y[2], w[2], pv[2];
  int nf;
};

template <typename Real>
struct Vec2;
template <>
struct Vec2<float> {
  using type = float2;
};
template <>
struct Vec2<double> {
  using type = double2;
};

// Loads the fields a pass reads for pair p: one two-element vector per
// field when the arrays allow it, else element by element.
template <typename Real, int PASS>
__device__ __forceinline__ PairIn<Real> load_pair(const CollArgs<Real>& a, uint64_t p) {
  using V = typename Vec2<Real>::type;
  PairIn<Real> d;
  const uint64_t i0 = 2 * p;
  d.nf = i0 + 1 < a.n ? 2 : 1;
  const bool need_w = PASS == kCSwim0 || PASS == kCEat || a.ph.swim_mode != 0;
  const bool need_pv = PASS == kCEat;
  if (a.vec2 && d.nf == 2) {
    const V xv = reinterpret_cast<const V*>(a.x)[p];
    const V yv = reinterpret_cast<const V*>(a.y)[p];
    d.x[0] = xv.x;
    d.x[1] = xv.y;
    d.y[0] = yv.x;
    d.y[1] = yv.y;
    if (need_w) {
      const V wv = reinterpret_cast<const V*>(a.w)[p];
      d.w[0] = wv.x;
      d.w[1] = wv.y;
    } else {
      d.w[0] = d.w[1] = Real(0);
    }
    if (need_pv) {
      const V pvv = reinterpret_cast<const V*>(a.pv)[p];
      d.pv[0] = pvv.x;
      d.pv[1] = pvv.y;
    } else {
      d.pv[0] = d.pv[1] = Real(0);
    }
    return d;
  }
#pragma unroll
  for (int f = 0; f < 2; ++f) {
    if (f < d.nf) {
      d.x[f] = a.x[i0 + f];
      d.y[f] = a.y[i0 + f];
      d.w[f] = need_w ? a.w[i0 + f] : Real(0);
      d.pv[f] = need_pv ? a.pv[i0 + f] : Real(0);
    } else {
      d.x[f] = d.y[f] = d.w[f] = d.pv[f] = Real(0);
    }
  }
  return d;
}

// One term of an exact school sum: v * 2^k rounded to the nearest integer,
// ties to even, without a 64-bit float-to-integer conversion (that runs on
// this GPU's slow binary64 pipe).  Binary64 terms: from the bits of v with
// integer operations; v is sig * 2^(exp - bias - mantissa bits), so v * 2^k
// is sig shifted by (exp - bias - mantissa bits + k), and a right shift
// rounds on the bits it drops.
__device__ __forceinline__ long long round_shifted(uint64_t sig, int s, bool neg) {
  uint64_t q;
  if (s >= 0) {
    q = sig << s;
  } else if (s <= -64) {
    q = 0;
  } else {
    const int r = -s;
    q = sig >> r;
    const uint64_t rem = sig & ((1ull << r) - 1ull);
    const uint64_t half = 1ull << (r - 1);
    if (rem > half || (rem == half && (q & 1ull))) ++q;
  }
  const long long sq = static_cast<long long>(q);
  return neg ? -sq : sq;
}

// Binary32 terms round on the FMA pipe instead.  x = v * 2^k is exact (a
// power-of-two scaling), and the grid bounds the whole sum, so |x| <= 2^62 / N.
// When |x| <= 2^43 (every school of at least 2^19 fish):
//  - adding and removing C = 1.5 * 2^45 rounds x to a multiple of 2^22
//    (x + C lies in [2^45, 2^46), where the spacing is 2^22), to nearest,
//    ties to even: x_hi;
//  - x_lo = x - x_hi is exact and |x_lo| <= 2^21;
//  - adding M = 1.5 * 2^23 to x_lo (or to x_hi / 2^22, also within 2^21)
//    lands in [2^23, 2^24), where the spacing is 1, so the sum is rounded to
//    an integer, ties to even, and its bits minus M's bits are that integer.
// x_hi is a multiple of 2^22 (even), so round(x) = x_hi + round(x_lo).
// Smaller schools (`wide`: the kernel copy compiled for them) can have
// terms up to 2^62.  A binary32 value of magnitude 2^23 or more is already an integer:
// its 24-bit significand shifted left by (biased exponent - 150), at most 39
// places.  Below 2^23 the FMA-pipe rounding above applies.
__device__ __forceinline__ long long grid_term(float v, float scale, bool wide) {
  const float x = __fmul_rn(v, scale);
  const float c = 0x1.8p45f;
  const float m = 0x1.8p23f;
  const float x_hi = __fsub_rn(__fadd_rn(x, c), c);
  const float x_lo = __fsub_rn(x, x_hi);
  const int lo = __float_as_int(__fadd_rn(x_lo, m)) - __float_as_int(m);
  const int hi = __float_as_int(__fadd_rn(__fmul_rn(x_hi, 0x1p-22f), m)) - __float_as_int(m);
  long long r = static_cast<long long>(hi) * (1ll << 22) + lo;
  if (wide) {
    const uint32_t b = __float_as_uint(x);
    const int e = static_cast<int>((b >> 23) & 0xFFu);
    if (e >= 150) {
      const long long mag = static_cast<long long>((b & 0x7FFFFFu) | 0x800000u) << (e - 150);
      r = (b >> 31) ? -mag : mag;
    }
  }
  return r;
}

__device__ __forceinline__ long long grid_term(double v, double scale, bool) {
  // scale = 2^k, a normal power of two (|k| <= 100): k from its exponent bits
  const int k =
      static_cast<int>((static_cast<uint64_t>(__double_as_longlong(scale)) >> 52) & 0x7FFull) -
      1023;
  const uint64_t b = static_cast<uint64_t>(__double_as_longlong(v));
  const int e = static_cast<int>((b >> 52) & 0x7FFull);
  const uint64_t m = b & 0xFFFFFFFFFFFFFull;
  return e ? round_shifted(m | (1ull << 52), e - 1075 + k, (b >> 63) != 0ull)
           : round_shifted(m, k - 1074, (b >> 63) != 0ull);
}

__device__ __forceinline__ long long warp_sum_ll(long long v) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(kFullMask, v, off);
  return v;
}

// Pass index j of a call: 0 = swim0, 2t - 1 = eat t, 2t = move t.
template <int PASS>
__device__ __forceinline__ bool coll_prologue(Ctl* ctl, uint32_t n_steps, uint32_t& j,
                                              uint64_t& base) {
  if (__syncthreads_or(ld_relaxed_gpu(&ctl->status) != 0)) return false;
  j = ctl->pass;
  base = ctl->base_step;
  bool ok;
  if (PASS == kCSwim0)
    ok = j == 0;
  else if (PASS == kCEat)
    ok = (j & 1u) == 1u && j < 2 * n_steps;
  else if (PASS == kCMove)
    ok = j >= 2 && (j & 1u) == 0u && j < 2 * n_steps;
  else
    ok = j == 2 * n_steps;
  if (!ok) {
    if (threadIdx.x == 0) atomicCAS(&ctl->status, 0, static_cast<int>(FSB_ERR_STATE));
    return false;
  }
  return true;
}

// Swim of one fish at step t with draw words (r0, r1): the maxima keys, and
// (when it improved) its instinctive terms dx g, dy g and g on the grid.
template <bool WIDE, typename Real, typename B>
__device__ __forceinline__ void swim_fish(Real& x, Real& y, Real& cur, Real w, uint32_t r0,
                                          uint32_t r1, const CollArgs<Real>& a, B& maxb,
                                          B& ekey, long long (&q)[4]) {
  using A = Arith<Real>;
  const Real x0 = x, y0 = y;
  swim(x, y, r0, r1, swim_width(a.ph, w), a.ph);
  const Real ncur = objective(x, y);
  const Real d = A::sub(ncur, cur);
  const Real g = A::sub(cur, ncur);
  const B mb = abs_bits(d);
  const B ek = order_key(g);
  maxb = mb > maxb ? mb : maxb;
  ekey = ek > ekey ? ek : ekey;
  if (g > Real(0)) {
    q[0] += grid_term(A::mul(A::sub(x, x0), g), a.g_p, WIDE);
    q[1] += grid_term(A::mul(A::sub(y, y0), g), a.g_p, WIDE);
    q[2] += grid_term(g, a.g_g, WIDE);
  }
  cur = ncur;
}

// WIDE: terms may exceed 2^43 (schools below 2^19 fish; see grid_term),
// a separate copy so that larger schools carry no test for it.
template <typename Real, int PASS, int ACC, bool WIDE>
__global__ void __launch_bounds__(kCollBlock, 4) coll_kernel(CollArgs<Real> a) {
  using A = Arith<Real>;
  using Bt = typename Bits<Real>::type;
  using Acc = SumAcc<ACC>;
  using Sum = typename Acc::Sum;
  constexpr int kWarps = kCollBlock / 32;
  __shared__ Bt s_max[kWarps], s_ekey[kWarps];
  __shared__ Sum s_w[kWarps], s_x[kWarps], s_y[kWarps];
  __shared__ long long s_q[kWarps][4];
  __shared__ bool s_last;

  uint32_t j;
  uint64_t base;
  if (!coll_prologue<PASS>(a.ctl, a.n_steps, j, base)) return;
  // step whose eat (kCEat) or volitive move (kCMove*) this pass runs
  const uint32_t t = PASS == kCEat ? (j + 1) / 2 : j / 2;
  const uint32_t t_abs = static_cast<uint32_t>(base + t);          // absolute step
  const uint32_t t_swim = static_cast<uint32_t>(base + t + 1);     // step swum here

  Real N = Real(0), ix = Real(0), iy = Real(0), bx = Real(0), by = Real(0);
  bool has_b = false, contract = false;
  if (PASS == kCEat) {
    const fsb_step_stats& rec = a.ring[t - 1];
    N = static_cast<Real>(a.ph.feed_mode ? rec.eat_max_diff : rec.max_abs_delta);
    ix = static_cast<Real>(a.coll[t - 1].ix);
    iy = static_cast<Real>(a.coll[t - 1].iy);
  }
  if (PASS == kCMove || PASS == kCMoveLast) {
    const CollRec& c = a.coll[t - 1];
    bx = static_cast<Real>(c.bx);
    by = static_cast<Real>(c.by);
    has_b = c.has_b != 0;
    contract = c.contract != 0;
  }

  Acc acc;
  Bt maxb = 0, ekey = 0;
  long long q[4] = {0, 0, 0, 0};
  const uint64_t n_pairs = (a.n + 1) / 2;
  const uint64_t stride = static_cast<uint64_t>(gridDim.x) * kCollBlock;
  // the work on one loaded pair (its stores included)
  auto run_pair = [&](uint64_t p, PairIn<Real>& d) {
    const uint64_t i0 = 2 * p;
    const int nf = d.nf;
    Real* x = d.x;
    Real* y = d.y;
    Real* w = d.w;
    Real* pv = d.pv;
    if (PASS == kCSwim0) {
      const Words4 r = pair_draw(a.key, a.school, p, t_swim);
#pragma unroll
      for (int f = 0; f < 2; ++f) {
        if (f < nf) {
          q[3] += grid_term(w[f], a.g_w, WIDE);  // the school's weight before the first eat
          Real cur = objective(x[f], y[f]);
          pv[f] = cur;                     // prevObjective after this swim
          swim_fish<WIDE>(x[f], y[f], cur, w[f], r.v[2 * f], r.v[2 * f + 1], a, maxb, ekey, q);
        }
      }
    } else if (PASS == kCEat) {
#pragma unroll
      for (int f = 0; f < 2; ++f) {
        if (f < nf) {
          const Real cur = objective(x[f], y[f]);
          if (N > Real(0))
            w[f] = eat(w[f], a.ph.feed_mode ? A::sub(pv[f], cur) : A::sub(cur, pv[f]), N, a.ph);
          acc.add(w[f], x[f], y[f]);
          x[f] = A::clamp(A::add(x[f], ix), -a.ph.pond_half, a.ph.pond_half);
          y[f] = A::clamp(A::add(y[f], iy), -a.ph.pond_half, a.ph.pond_half);
          q[0] += grid_term(w[f], a.g_w, WIDE);
          q[1] += grid_term(A::mul(w[f], x[f]), a.g_w, WIDE);
          q[2] += grid_term(A::mul(w[f], y[f]), a.g_w, WIDE);
        }
      }
    } else {
      if (has_b) {
        const Words4 rv = fish_draw(a.key, a.school, p, t_abs, kDomainVolitive);
#pragma unroll
        for (int f = 0; f < 2; ++f) {
          if (f < nf) {
            const Real u = A::unit(rv.v[f]);
            const Real dx = A::sub(x[f], bx);
            const Real dy = A::sub(y[f], by);
            const Real dist = A::sqrt(A::add(A::mul(dx, dx), A::mul(dy, dy)));
            if (dist > Real(0)) {
              const Real m = A::div(A::mul(a.s_vol, u), dist);
              const Real mx = A::mul(m, dx), my = A::mul(m, dy);
              x[f] = A::clamp(contract ? A::sub(x[f], mx) : A::add(x[f], mx), -a.ph.pond_half,
                              a.ph.pond_half);
              y[f] = A::clamp(contract ? A::sub(y[f], my) : A::add(y[f], my), -a.ph.pond_half,
                              a.ph.pond_half);
            }
          }
        }
      }
      if (PASS == kCMove) {
        const Words4 r = pair_draw(a.key, a.school, p, t_swim);
#pragma unroll
        for (int f = 0; f < 2; ++f) {
          if (f < nf) {
            Real cur = objective(x[f], y[f]);
            pv[f] = cur;  // prevObjective after this swim
            swim_fish<WIDE>(x[f], y[f], cur, w[f], r.v[2 * f], r.v[2 * f + 1], a, maxb, ekey, q);
          }
        }
      }
    }
    // stores: positions always; the weights after an eat; prevObjective
    // after a swim
    const bool put_w = PASS == kCEat;
    const bool put_pv = PASS == kCSwim0 || PASS == kCMove;
    if (a.vec2 && nf == 2) {
      using V = typename Vec2<Real>::type;
      reinterpret_cast<V*>(a.x)[p] = V{x[0], x[1]};
      reinterpret_cast<V*>(a.y)[p] = V{y[0], y[1]};
      if (put_w) reinterpret_cast<V*>(a.w)[p] = V{w[0], w[1]};
      if (put_pv) reinterpret_cast<V*>(a.pv)[p] = V{pv[0], pv[1]};
    } else {
#pragma unroll
      for (int f = 0; f < 2; ++f) {
        if (f < nf) {
          a.x[i0 + f] = x[f];
          a.y[i0 + f] = y[f];
          if (put_w) a.w[i0 + f] = w[f];
          if (put_pv) a.pv[i0 + f] = pv[f];
        }
      }
    }
  };
  // binary32: two pairs per iteration, both loaded before either is worked
  // on, so twice the bytes are in flight (binary64 state keeps one: its
  // registers would spill)
  const uint64_t first = static_cast<uint64_t>(blockIdx.x) * kCollBlock + threadIdx.x;
  if (sizeof(Real) == 4) {
    for (uint64_t p = first; p < n_pairs; p += 2 * stride) {
      const uint64_t p2 = p + stride;
      PairIn<Real> d1 = load_pair<Real, PASS>(a, p);
      PairIn<Real> d2;
      if (p2 < n_pairs) d2 = load_pair<Real, PASS>(a, p2);
      run_pair(p, d1);
      if (p2 < n_pairs) run_pair(p2, d2);
    }
  } else {
    for (uint64_t p = first; p < n_pairs; p += stride) {
      PairIn<Real> d = load_pair<Real, PASS>(a, p);
      run_pair(p, d);
    }
  }

  // ---- block reduction, one partial per block; the last block folds them
  // in block order (the integer sums are exact in any order)
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  maxb = warp_max(maxb);
  ekey = warp_max(ekey);
  Sum sw = Sum(acc.rw()), sx = Sum(acc.rx()), sy = Sum(acc.ry());
  sw = warp_sum(sw);
  sx = warp_sum(sx);
  sy = warp_sum(sy);
  long long qs[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) qs[k] = warp_sum_ll(q[k]);
  if (lane == 0) {
    s_max[warp] = maxb;
    s_ekey[warp] = ekey;
    s_w[warp] = sw;
    s_x[warp] = sx;
    s_y[warp] = sy;
#pragma unroll
    for (int k = 0; k < 4; ++k) s_q[warp][k] = qs[k];
  }
  __syncthreads();
  if (warp == 0) {
    Bt m = lane < kWarps ? s_max[lane] : Bt(0);
    Bt e = lane < kWarps ? s_ekey[lane] : Bt(0);
    Sum bw = lane < kWarps ? s_w[lane] : Sum(0);
    Sum bxs = lane < kWarps ? s_x[lane] : Sum(0);
    Sum bys = lane < kWarps ? s_y[lane] : Sum(0);
    long long bq[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) bq[k] = warp_sum_ll(lane < kWarps ? s_q[lane][k] : 0ll);
    m = warp_max(m);
    e = warp_max(e);
    bw = warp_sum(bw);
    bxs = warp_sum(bxs);
    bys = warp_sum(bys);
    if (lane == 0) {
      CollPartial cp;
      cp.max_bits = static_cast<unsigned long long>(m);
      cp.e_key = static_cast<unsigned long long>(e);
      cp.sum_w = static_cast<double>(bw);
      cp.sum_wx = static_cast<double>(bxs);
      cp.sum_wy = static_cast<double>(bys);
#pragma unroll
      for (int k = 0; k < 4; ++k) cp.q[k] = bq[k];
      a.partials[blockIdx.x] = cp;
      __threadfence();
      const unsigned prev = atomicAdd(&a.ctl->arrive, 1u);
      s_last = prev == gridDim.x - 1;
    }
  }
  __syncthreads();
  if (!s_last) return;

  __threadfence();
  Bt m = 0, e = 0;
  Sum fw = Sum(0), fx = Sum(0), fy = Sum(0);
  long long fq[4] = {0, 0, 0, 0};
  for (uint32_t b = threadIdx.x; b < gridDim.x; b += kCollBlock) {
    const CollPartial* cp = a.partials + b;
    const Bt mb = static_cast<Bt>(__ldcg(&cp->max_bits));
    const Bt eb = static_cast<Bt>(__ldcg(&cp->e_key));
    m = mb > m ? mb : m;
    e = eb > e ? eb : e;
    fw = sum2(fw, Sum(__ldcg(&cp->sum_w)));
    fx = sum2(fx, Sum(__ldcg(&cp->sum_wx)));
    fy = sum2(fy, Sum(__ldcg(&cp->sum_wy)));
#pragma unroll
    for (int k = 0; k < 4; ++k) fq[k] += __ldcg(&cp->q[k]);
  }
  m = warp_max(m);
  e = warp_max(e);
  fw = warp_sum(fw);
  fx = warp_sum(fx);
  fy = warp_sum(fy);
#pragma unroll
  for (int k = 0; k < 4; ++k) fq[k] = warp_sum_ll(fq[k]);
  __syncthreads();  // shared arrays are reused
  if (lane == 0) {
    s_max[warp] = m;
    s_ekey[warp] = e;
    s_w[warp] = fw;
    s_x[warp] = fx;
    s_y[warp] = fy;
#pragma unroll
    for (int k = 0; k < 4; ++k) s_q[warp][k] = fq[k];
  }
  __syncthreads();
  if (warp != 0) return;
  m = lane < kWarps ? s_max[lane] : Bt(0);
  e = lane < kWarps ? s_ekey[lane] : Bt(0);
  fw = warp_sum(lane < kWarps ? s_w[lane] : Sum(0));
  fx = warp_sum(lane < kWarps ? s_x[lane] : Sum(0));
  fy = warp_sum(lane < kWarps ? s_y[lane] : Sum(0));
#pragma unroll
  for (int k = 0; k < 4; ++k) fq[k] = warp_sum_ll(lane < kWarps ? s_q[lane][k] : 0ll);
  m = warp_max(m);
  e = warp_max(e);
  if (lane != 0) return;

  if (PASS == kCSwim0 || PASS == kCMove) {
    // maxima and instinctive vector of the step swum here (index t)
    fsb_step_stats* rec = a.ring + t;
    Real mv;
    if (sizeof(Real) == 4)
      mv = static_cast<Real>(__uint_as_float(static_cast<uint32_t>(m)));
    else
      mv = static_cast<Real>(__longlong_as_double(static_cast<long long>(m)));
    rec->max_abs_delta = static_cast<double>(mv);
    rec->eat_max_diff = static_cast<double>(key_to_value(e, Real(0)));
    CollRec* c = a.coll + t;
    double vx = 0.0, vy = 0.0;
    if (fq[2] != 0) {
      const double den = __ll2double_rn(fq[2]);
      vx = scalbn(__ddiv_rn(__ll2double_rn(fq[0]), den), a.kg - a.kp);
      vy = scalbn(__ddiv_rn(__ll2double_rn(fq[1]), den), a.kg - a.kp);
    }
    c->ix = static_cast<double>(static_cast<Real>(vx));
    c->iy = static_cast<double>(static_cast<Real>(vy));
    if (PASS == kCSwim0) c->w_before = fq[3];
  }
  if (PASS == kCEat) {
    fsb_step_stats* rec = a.ring + (t - 1);
    rec->sum_w = static_cast<double>(fw);
    rec->sum_wx = static_cast<double>(fx);
    rec->sum_wy = static_cast<double>(fy);
    CollRec* c = a.coll + (t - 1);
    c->sw = fq[0];
    c->has_b = fq[0] != 0 ? 1 : 0;
    c->contract = fq[0] > c->w_before ? 1 : 0;
    double vbx = 0.0, vby = 0.0;
    if (fq[0] != 0) {
      const double sw_d = __ll2double_rn(fq[0]);
      vbx = __ddiv_rn(__ll2double_rn(fq[1]), sw_d);
      vby = __ddiv_rn(__ll2double_rn(fq[2]), sw_d);
    }
    c->bx = static_cast<double>(static_cast<Real>(vbx));
    c->by = static_cast<double>(static_cast<Real>(vby));
    if (t < a.n_steps) a.coll[t].w_before = fq[0];
  }
  a.ctl->arrive = 0u;
  if (PASS == kCMoveLast) {
    a.ctl->base_step = base + a.n_steps;
    a.ctl->pass = 0u;
  } else {
    a.ctl->pass = j + 1;
  }
  __threadfence();
}

template <typename Real, int PASS, bool WIDE>
const void* pick_acc(int acc) {
  if (sizeof(Real) == 8)
    return reinterpret_cast<const void*>(&coll_kernel<Real, PASS, kAccF64, false>);
  switch (acc) {
    case kAccPlain32:
      return reinterpret_cast<const void*>(&coll_kernel<Real, PASS, kAccPlain32, WIDE>);
    case kAccKahan32:
      return reinterpret_cast<const void*>(&coll_kernel<Real, PASS, kAccKahan32, WIDE>);
    case kAccF64: return reinterpret_cast<const void*>(&coll_kernel<Real, PASS, kAccF64, WIDE>);
    default: return nullptr;
  }
}

template <typename Real, int PASS>
const void* pick_wide(int acc, bool wide) {
  return wide ? pick_acc<Real, PASS, true>(acc) : pick_acc<Real, PASS, false>(acc);
}

template <typename Real>
const void* pick_pass(int pass, int acc, bool wide) {
  switch (pass) {
    case kCSwim0: return pick_wide<Real, kCSwim0>(acc, wide);
    case kCEat: return pick_wide<Real, kCEat>(acc, wide);
    case kCMove: return pick_wide<Real, kCMove>(acc, wide);
    case kCMoveLast: return pick_wide<Real, kCMoveLast>(acc, wide);
    default: return nullptr;
  }
}

template <typename Real>
CollArgs<Real> make_args(const CollLaunch& L, uint32_t n_steps) {
  CollArgs<Real> a;
  a.x = static_cast<Real*>(L.x);
  a.y = static_cast<Real*>(L.y);
  a.w = static_cast<Real*>(L.w);
  a.pv = static_cast<Real*>(L.pv);
  a.n = L.n;
  a.key.k0 = static_cast<uint32_t>(L.seed);
  a.key.k1 = static_cast<uint32_t>(L.seed >> 32);
  a.school = L.school;
  a.ph.pond_half = static_cast<Real>(L.pond_half);
  a.ph.step = static_cast<Real>(L.step);
  a.ph.w0 = static_cast<Real>(L.w0);
  a.ph.w_min = static_cast<Real>(L.w_min);
  a.ph.w_max = static_cast<Real>(L.w_max);
  a.ph.swim_mode = L.swim_mode;
  a.ph.feed_mode = L.feed_mode;
  a.s_vol = static_cast<Real>(L.step_vol);
  a.g_p = static_cast<Real>(ldexp(1.0, L.kp));
  a.g_g = static_cast<Real>(ldexp(1.0, L.kg));
  a.g_w = static_cast<Real>(ldexp(1.0, L.kw));
  a.kp = L.kp;
  a.kg = L.kg;
  a.ctl = L.ctl;
  a.partials = L.partials;
  a.ring = L.ring;
  a.coll = L.coll;
  a.n_steps = n_steps;
  const uintptr_t align = 2 * sizeof(Real);
  a.vec2 = (reinterpret_cast<uintptr_t>(L.x) % align == 0 &&
            reinterpret_cast<uintptr_t>(L.y) % align == 0 &&
            reinterpret_cast<uintptr_t>(L.w) % align == 0 &&
            reinterpret_cast<uintptr_t>(L.pv) % align == 0) ? 1 : 0;
  return a;
}

}  // namespace

int coll_grid(const CollLaunch& L, int sms) {
  const uint64_t pairs = (L.n + 1) / 2;
  const uint64_t want = (pairs + kCollBlock - 1) / kCollBlock;
  const uint64_t full = static_cast<uint64_t>(sms) * 4;
  return static_cast<int>(want < 1 ? 1 : (want < full ? want : full));
}

cudaError_t launch_coll_pass(const CollLaunch& L, int pass_kind, uint32_t n_steps,
                             cudaStream_t s) {
  // every sum of N terms is within 2^62, so a term exceeds 2^43 only when
  // N < 2^19
  const bool wide = L.n < (1ull << 19);
  const void* fn = L.real_is_double ? pick_pass<double>(pass_kind, L.acc, wide)
                                    : pick_pass<float>(pass_kind, L.acc, wide);
  if (!fn || L.grid <= 0) return cudaErrorInvalidValue;
  if (L.real_is_double) {
    CollArgs<double> a = make_args<double>(L, n_steps);
    void* args[] = {&a};
    return cudaLaunchKernel(fn, dim3(L.grid), dim3(kCollBlock), args, 0, s);
  }
  CollArgs<float> a = make_args<float>(L, n_steps);
  void* args[] = {&a};
  return cudaLaunchKernel(fn, dim3(L.grid), dim3(kCollBlock), args, 0, s);
}

}  // namespace fsb
