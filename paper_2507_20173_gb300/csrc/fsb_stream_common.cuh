// fsb_stream_common.cuh -- pieces shared by the two streaming-pass kernels
// (plain vector loads in fsb_stream.cu, bulk asynchronous copies in
// fsb_stream_tma.cu): kernel arguments, the per-fish body of one pass and the
// pass epilogue (block reduction, last-block fold into the statistics ring).
#pragma once

#include <cstdint>

#include "fsb_device.cuh"
#include "fsb_internal.h"
#include "fsb_reduce.cuh"

namespace fsb {

template <typename Real>
struct StreamArgs {
  Real* __restrict__ x;
  Real* __restrict__ y;
  Real* __restrict__ w;
  Real* __restrict__ pv;
  uint64_t n;
  Key key;
  uint32_t school;
  Physics<Real> ph;
  Ctl* ctl;
  BlockPartial* partials;
  fsb_step_stats* ring;
  uint32_t ring_cap;
  unsigned long long timeout_ns;  // bound of every wait in the copy rings
  int inject_block;               // test hook: this block withholds the first copy
  uint32_t inject_pass;           //   of its ring in this pass of a call (-1: none)
};

template <typename Real>
StreamArgs<Real> make_stream_args(const StreamLaunch& L) {
  StreamArgs<Real> a;
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
  a.ctl = L.ctl;
  a.partials = L.partials;
  a.ring = L.ring;
  a.ring_cap = L.ring_cap;
  a.timeout_ns = L.timeout_ns ? L.timeout_ns : 1000000000ull;
  a.inject_block = L.inject_block;
  a.inject_pass = L.inject_pass;
  return a;
}

// Pass index j and step counter of this launch; false (status latched) if
// the control word does not fit this call's sequence.
template <int PASS>
__device__ __forceinline__ bool pass_prologue(const Ctl* ctl, Ctl* wctl, uint32_t ring_cap,
                                              uint32_t& j, uint64_t& base) {
  // a pass of a call that already failed does nothing.  The status word can
  // be latched by another block while this one starts, so the block takes
  // one decision for all its threads (every thread calls the prologue).
  if (__syncthreads_or(ld_relaxed_gpu(&ctl->status) != 0)) return false;
  j = ctl->pass;
  base = ctl->base_step;
  if ((PASS != kSwimOnly && (j == 0 || j > ring_cap)) || (PASS != kSettle && j >= ring_cap)) {
    if (threadIdx.x == 0) atomicCAS(&wctl->status, 0, static_cast<int>(FSB_ERR_STATE));
    return false;
  }
  return true;
}

// The feeding normaliser of step j from its statistics record: M_j, or the
// paper's eat() value E_j when feeding follows it.
template <typename Real>
__device__ __forceinline__ Real feed_normaliser(const fsb_step_stats& rec,
                                                const Physics<Real>& ph) {
  return static_cast<Real>(ph.feed_mode ? rec.eat_max_diff : rec.max_abs_delta);
}

// One fish through one pass, without the barycentre accumulation: eat of
// step j (kinds kFused / kSettle, with N = its feeding normaliser), then
// swim + objective + delta of the step `t` (kinds kSwimOnly / kFused).  The
// caller adds (w, x, y) of step j to its sums between the two halves; see
// fish_pass below.
template <typename Real, int PASS>
__device__ __forceinline__ Real fish_eat(Real x, Real y, Real& w, Real pv, Real N,
                                         const Physics<Real>& ph) {
  using A = Arith<Real>;
  const Real cur = objective(x, y);
  if (PASS != kSwimOnly && N > Real(0))
    w = eat(w, ph.feed_mode ? A::sub(pv, cur) : A::sub(cur, pv), N, ph);
  return cur;
}

template <typename Real, int PASS, typename B>
__device__ __forceinline__ void fish_swim(Real& x, Real& y, Real w, Real& pv, Real cur,
                                          uint32_t r0, uint32_t r1, const Physics<Real>& ph,
                                          B& maxb, B& ekey) {
  using A = Arith<Real>;
  if (PASS != kSettle) {
    swim(x, y, r0, r1, swim_width(ph, w), ph);
    const Real ncur = objective(x, y);
    const B mb = abs_bits(A::sub(ncur, cur));
    const B ek = order_key(A::sub(cur, ncur));
    maxb = mb > maxb ? mb : maxb;
    ekey = ek > ekey ? ek : ekey;
    pv = cur;
  }
}

// One fish through one pass.  `M` is M_j (pass kinds kFused / kSettle),
// `t` the absolute step of the swim (kSwimOnly / kFused).
template <typename Real, int PASS, typename Acc, typename B>
__device__ __forceinline__ void fish_pass(Real& x, Real& y, Real& w, Real& pv, uint64_t i, Real M,
                                          uint32_t t, Key key, uint32_t school,
                                          const Physics<Real>& ph, Acc& acc, B& maxb, B& ekey) {
  const Real cur = fish_eat<Real, PASS>(x, y, w, pv, M, ph);
  if (PASS != kSwimOnly) acc.add(w, x, y);
  Words2 r{0u, 0u};
  if (PASS != kSettle) r = fish_swim_words(key, school, i, t);
  fish_swim<Real, PASS>(x, y, w, pv, cur, r.r0, r.r1, ph, maxb, ekey);
}

// Two fish of one pair (i0 even) through one pass: one swim block moves both.
template <typename Real, int PASS, typename Acc, typename B>
__device__ __forceinline__ void fish_pass2(Real (&x)[2], Real (&y)[2], Real (&w)[2],
                                           Real (&pv)[2], uint64_t i0, Real M, uint32_t t,
                                           Key key, uint32_t school, const Physics<Real>& ph,
                                           Acc& acc, B& maxb, B& ekey) {
  Real cur[2];
#pragma unroll
  for (int q = 0; q < 2; ++q) {
    cur[q] = fish_eat<Real, PASS>(x[q], y[q], w[q], pv[q], M, ph);
    if (PASS != kSwimOnly) acc.add(w[q], x[q], y[q]);
  }
  Words4 r{};
  if (PASS != kSettle) r = pair_draw(key, school, i0 >> 1, t);
#pragma unroll
  for (int q = 0; q < 2; ++q)
    fish_swim<Real, PASS>(x[q], y[q], w[q], pv[q], cur[q], r.v[2 * q], r.v[2 * q + 1], ph, maxb,
                          ekey);
}

// Four consecutive fish (one 16-byte vector of each array, i0 a multiple of
// four) through one pass, with their barycentre contributions added as one
// group; two swim blocks move the two pairs.
template <typename Real, int PASS, typename Acc, typename B>
__device__ __forceinline__ void fish_pass4(Real (&x)[4], Real (&y)[4], Real (&w)[4],
                                           Real (&pv)[4], uint64_t i0, Real M, uint32_t t,
                                           Key key, uint32_t school, const Physics<Real>& ph,
                                           Acc& acc, B& maxb, B& ekey) {
  Real cur[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) cur[q] = fish_eat<Real, PASS>(x[q], y[q], w[q], pv[q], M, ph);
  if (PASS != kSwimOnly) acc.add4(w, x, y);
  Words4 r[2] = {};
  if (PASS != kSettle) {
    r[0] = pair_draw(key, school, i0 >> 1, t);
    r[1] = pair_draw(key, school, (i0 >> 1) + 1, t);
  }
#pragma unroll
  for (int q = 0; q < 4; ++q)
    fish_swim<Real, PASS>(x[q], y[q], w[q], pv[q], cur[q], r[q >> 1].v[2 * (q & 1)],
                          r[q >> 1].v[2 * (q & 1) + 1], ph, maxb, ekey);
}

// Block reduction of the pass's maxima and sums into one partial per block;
// the last block to arrive folds all partials in a fixed order, writes the
// statistics ring and advances the control word.  Every thread of the block
// must call it.
template <typename Real, int PASS, int ACC, int BLOCK>
__device__ __forceinline__ void pass_epilogue(const StreamArgs<Real>& a, const SumAcc<ACC>& acc,
                                              typename Bits<Real>::type maxb,
                                              typename Bits<Real>::type ekey, uint32_t j,
                                              uint64_t base) {
  using B = typename Bits<Real>::type;
  using Sum = typename SumAcc<ACC>::Sum;
  constexpr int kWarps = BLOCK / 32;
  __shared__ B s_max[kWarps], s_ekey[kWarps];
  __shared__ Sum s_w[kWarps], s_x[kWarps], s_y[kWarps];
  __shared__ bool s_last;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  maxb = warp_max(maxb);
  ekey = warp_max(ekey);
  Sum sw = Sum(acc.rw()), sx = Sum(acc.rx()), sy = Sum(acc.ry());
  if (PASS != kSwimOnly) {
    sw = warp_sum(sw);
    sx = warp_sum(sx);
    sy = warp_sum(sy);
  }
  if (lane == 0) {
    s_max[warp] = maxb;
    s_ekey[warp] = ekey;
    s_w[warp] = sw;
    s_x[warp] = sx;
    s_y[warp] = sy;
  }
  __syncthreads();
  if (warp == 0) {
    B m = lane < kWarps ? s_max[lane] : B(0);
    B e = lane < kWarps ? s_ekey[lane] : B(0);
    Sum bw = lane < kWarps ? s_w[lane] : Sum(0);
    Sum bx = lane < kWarps ? s_x[lane] : Sum(0);
    Sum by = lane < kWarps ? s_y[lane] : Sum(0);
    m = warp_max(m);
    e = warp_max(e);
    if (PASS != kSwimOnly) {
      bw = warp_sum(bw);
      bx = warp_sum(bx);
      by = warp_sum(by);
    }
    if (lane == 0) {
      BlockPartial bp;
      bp.max_bits = static_cast<unsigned long long>(m);
      bp.e_key = static_cast<unsigned long long>(e);
      bp.sum_w = static_cast<double>(bw);
      bp.sum_wx = static_cast<double>(bx);
      bp.sum_wy = static_cast<double>(by);
      bp.spare = 0.0;
      a.partials[blockIdx.x] = bp;
      __threadfence();
      const unsigned prev = atomicAdd(&a.ctl->arrive, 1u);
      s_last = (prev == gridDim.x - 1);
    }
  }
  __syncthreads();
  if (!s_last) return;

  // ---- last block: fold all partials in a fixed order
  __threadfence();
  B m = 0, e = 0;
  Sum fw = Sum(0), fx = Sum(0), fy = Sum(0);
  for (uint32_t b = threadIdx.x; b < gridDim.x; b += BLOCK) {
    const BlockPartial* bp = a.partials + b;
    const B mb = static_cast<B>(__ldcg(&bp->max_bits));
    const B eb = static_cast<B>(__ldcg(&bp->e_key));
    m = mb > m ? mb : m;
    e = eb > e ? eb : e;
    if (PASS != kSwimOnly) {
      fw = sum2(fw, Sum(__ldcg(&bp->sum_w)));
      fx = sum2(fx, Sum(__ldcg(&bp->sum_wx)));
      fy = sum2(fy, Sum(__ldcg(&bp->sum_wy)));
    }
  }
  m = warp_max(m);
  e = warp_max(e);
  if (PASS != kSwimOnly) {
    fw = warp_sum(fw);
    fx = warp_sum(fx);
    fy = warp_sum(fy);
  }
  __syncthreads();  // shared arrays are reused
  if (lane == 0) {
    s_max[warp] = m;
    s_ekey[warp] = e;
    s_w[warp] = fw;
    s_x[warp] = fx;
    s_y[warp] = fy;
  }
  __syncthreads();
  if (warp == 0) {
    m = lane < kWarps ? s_max[lane] : B(0);
    e = lane < kWarps ? s_ekey[lane] : B(0);
    fw = lane < kWarps ? s_w[lane] : Sum(0);
    fx = lane < kWarps ? s_x[lane] : Sum(0);
    fy = lane < kWarps ? s_y[lane] : Sum(0);
    m = warp_max(m);
    e = warp_max(e);
    if (PASS != kSwimOnly) {
      fw = warp_sum(fw);
      fx = warp_sum(fx);
      fy = warp_sum(fy);
    }
    if (lane == 0) {
      if (PASS != kSwimOnly) {
        fsb_step_stats* rec = a.ring + (j - 1);
        rec->sum_w = static_cast<double>(fw);
        rec->sum_wx = static_cast<double>(fx);
        rec->sum_wy = static_cast<double>(fy);
      }
      if (PASS != kSettle) {
        fsb_step_stats* rec = a.ring + j;
        Real mv;
        if (sizeof(Real) == 4)
          mv = static_cast<Real>(__uint_as_float(static_cast<uint32_t>(m)));
        else
          mv = static_cast<Real>(__longlong_as_double(static_cast<long long>(m)));
        rec->max_abs_delta = static_cast<double>(mv);
        rec->eat_max_diff = static_cast<double>(key_to_value(e, Real(0)));
      }
      a.ctl->arrive = 0u;
      if (PASS == kSettle) {
        a.ctl->base_step = base + j;
        a.ctl->pass = 0u;
      } else {
        a.ctl->pass = j + 1;
      }
      __threadfence();
    }
  }
}

}  // namespace fsb
