// fsb_stream_blocked.cu -- the streaming step blocked over k steps (stream
// kernels 4 and 5; kernel 5 with k = 8 is the library's streaming kernel for
// a large school).
//
// A school's positions do not depend on its weights (the default swim), and
// the draws are counter-based, so the steps j + 1 .. j + k of a school can be
// swum twice from the same state: once to find their maxima, once to eat and
// swim for real.  A pair of passes then advances k steps with one read of
// the positions and one read and write of the state, instead of one read and
// write per step:
//
//   maxima pass  (state "swum j, not eaten"): reads x, y; swims steps
//                j + 1 .. j + k in registers and reduces, per step, max |delta|
//                and the paper's eat() value max(prev - cur) (Sec. 2.3.2) into
//                the statistics records of those steps.  Writes no fish
//                (kernel 4).
//   step pass    reads x, y, w, prevObjective; for each of the k steps eats
//                (normaliser from the statistics record: M_j from the pass
//                before, the others from the maxima pass), adds the step's
//                barycentre terms and swims the next step; writes the state
//                "swum j + k, not eaten" and the k steps' barycentre sums.
//
// Stream kernel 5 trades memory for instructions: its maxima pass also
// stores the positions of steps j + 1 .. j + k (8 B per fish and step, in
// slots beside the state), and its step pass loads them instead of drawing
// and swimming again, so each fish-step's draw and swim run once (21 B of
// traffic per fish-step at k = 8, against 32 for one pass per step).  Its
// maxima pass has a second copy for whole pairs (k = K), without the
// per-step test of k.
//
// Per fish the arithmetic is fsb_stream.cu's, operation for operation, so
// the state is bit-identical to the one-pass-per-step kernels'; only the
// rounding order of the barycentre sums differs.  The pass sequence of a
// call is the swim-only pass of fsb_stream.cu, then pairs of these passes,
// then fsb_stream.cu's settle pass.  Both passes read the next group's state
// before working on the current one (the loads of one group are in flight
// while the previous one computes).  Binary32 state in 16-byte aligned
// arrays and the default swim only (the host enforces it).
#include <cstdint>

#include "fsb_bulk_copy.cuh"
#include "fsb_stream_common.cuh"

namespace fsb {
namespace {

constexpr int kBlkThreads = 256;
constexpr int kBlkWarps = kBlkThreads / 32;
// Kernel 5's step pass: each thread's positions of the next kLead steps are
// in flight through its own ring of kLead + 1 shared-memory entries, filled
// by asynchronous 16-byte copies (no registers held for them).  Measured at
// N = 2^28, k = 8: a lead of 2 steps 2.46e11 fish-steps/s, 3: 2.45e11, 4:
// 2.43e11, 6: 2.41e11; one step held in registers instead: 2.07e11.  The
// paired (f32x2) arithmetic of the on-chip passes measured slower in both
// passes here (2.43e11; kernel 4 at k = 8: 1.97e11 against 2.04e11).
constexpr int kLead = 2;
constexpr int kRing = kLead + 1;

// 16 bytes into shared memory, of which the first src_bytes (0 or 16) come
// from src and the rest are zero.
__device__ __forceinline__ void cp_async16(void* smem_dst, const void* src, uint32_t src_bytes) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(smem_u32(smem_dst)),
               "l"(src), "r"(src_bytes)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() {
  asm volatile("cp.async.commit_group;" ::: "memory");
}
// Waits until at most N of this thread's copy groups are still pending.
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// Pass index j of the pair and its step count k; false (status latched) if
// they do not fit the call: the maxima pass writes records j .. j + k - 1,
// the step pass reads records j - 1 .. j + k - 2.  A copy for whole pairs
// (FULL) takes k = K only.
template <int K, bool FULL>
__device__ __forceinline__ bool blocked_prologue(Ctl* ctl, uint32_t ring_cap, uint32_t k,
                                                 uint32_t& j, uint64_t& base) {
  if (__syncthreads_or(ld_relaxed_gpu(&ctl->status) != 0)) return false;
  j = ctl->pass;
  base = ctl->base_step;
  if (j == 0 || k == 0 || k > static_cast<uint32_t>(K) || (FULL && k != K) ||
      j + k > ring_cap) {
    if (threadIdx.x == 0) atomicCAS(&ctl->status, 0, static_cast<int>(FSB_ERR_STATE));
    return false;
  }
  return true;
}

// The block's arrival at the end of a pass; true in every thread of the
// last block to arrive (its partials are then all visible).
__device__ __forceinline__ bool arrive_last(Ctl* ctl) {
  __shared__ bool s_last;
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    const unsigned prev = atomicAdd(&ctl->arrive, 1u);
    s_last = prev == gridDim.x - 1;
  }
  __syncthreads();
  if (s_last) __threadfence();
  return s_last;
}

// The swim's move (2u - 1) * width (Sec. 2.1.2) as v * (width * 2^-23) with
// the integer v = (r >> 8) - 2^23: one rounding of the same real product as
// swim()'s (v * 2^-23) * width, since width * 2^-23 is exact (the host runs
// these kernels only for width 0 or |width| >= 2^-103), so bit-identical, with one
// product less per coordinate (measured: 1.2% faster; the same with a
// fallback branch to swim() per fish, 4% slower).
__device__ __forceinline__ float scaled_width(float width) {
  return __fmul_rn(width, 0x1p-23f);
}
__device__ __forceinline__ void swim_scaled(float& x, float& y, uint32_t r0, uint32_t r1,
                                            float scaled, const Physics<float>& ph) {
  const float vx = __int2float_rn(static_cast<int>(r0 >> 8) - (1 << 23));
  const float vy = __int2float_rn(static_cast<int>(r1 >> 8) - (1 << 23));
  x = fminf(fmaxf(__fadd_rn(x, __fmul_rn(vx, scaled)), -ph.pond_half), ph.pond_half);
  y = fminf(fmaxf(__fadd_rn(y, __fmul_rn(vy, scaled)), -ph.pond_half), ph.pond_half);
}

// One fish's swim of one step and its prev - cur into the extremes.
__device__ __forceinline__ void swim_extremes(float& x, float& y, float& cur, uint32_t r0,
                                              uint32_t r1, float scaled,
                                              const Physics<float>& ph, float& hi, float& lo) {
  swim_scaled(x, y, r0, r1, scaled, ph);
  const float n = objective(x, y);
  const float i = __fsub_rn(cur, n);
  hi = fmaxf(hi, i);
  lo = fminf(lo, i);
  cur = n;
}

// ------------------------------------------------------- maxima pass --
// Slot t (the positions after the swim of step j + 1 + t): x, then y.
__device__ __forceinline__ float* slot_x(float* slots, uint64_t ss, int t) {
  return slots + static_cast<uint64_t>(2 * t) * ss;
}
__device__ __forceinline__ float* slot_y(float* slots, uint64_t ss, int t) {
  return slots + static_cast<uint64_t>(2 * t + 1) * ss;
}

template <int K, bool STORE, bool FULL>
__global__ void __launch_bounds__(kBlkThreads, 2)
    blocked_maxima_kernel(StreamArgs<float> a, uint32_t k, BlockPartial* bp, float* slots,
                          uint64_t ss) {
  uint32_t j;
  uint64_t base;
  if (!blocked_prologue<K, FULL>(a.ctl, a.ring_cap, k, j, base)) return;
  const Physics<float> ph = a.ph;
  const float scaled = scaled_width(ph.step);
  const uint32_t t1 = static_cast<uint32_t>(base + j + 1);  // first step swum here
  float hi[K], lo[K];
#pragma unroll
  for (int t = 0; t < K; ++t) {
    hi[t] = -__int_as_float(0x7f800000);
    lo[t] = __int_as_float(0x7f800000);
  }
  const float4* const X = reinterpret_cast<const float4*>(a.x);
  const float4* const Y = reinterpret_cast<const float4*>(a.y);
  const uint64_t ngroups = a.n / 4;
  const uint64_t stride = static_cast<uint64_t>(gridDim.x) * kBlkThreads;
  const uint64_t tid = static_cast<uint64_t>(blockIdx.x) * kBlkThreads + threadIdx.x;
  float4 xn = make_float4(0.f, 0.f, 0.f, 0.f), yn = xn;
  if (tid < ngroups) {
    xn = X[tid];
    yn = Y[tid];
  }
  for (uint64_t g = tid; g < ngroups; g += stride) {
    float x[4] = {xn.x, xn.y, xn.z, xn.w}, y[4] = {yn.x, yn.y, yn.z, yn.w};
    if (g + stride < ngroups) {
      xn = X[g + stride];
      yn = Y[g + stride];
    }
    float cur[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) cur[q] = objective(x[q], y[q]);
#pragma unroll
    for (int t = 0; t < K; ++t) {
      if (FULL || static_cast<uint32_t>(t) < k) {
        const Words4 r0 = pair_draw(a.key, a.school, 2 * g, t1 + t);
        const Words4 r1 = pair_draw(a.key, a.school, 2 * g + 1, t1 + t);
        swim_extremes(x[0], y[0], cur[0], r0.v[0], r0.v[1], scaled, ph, hi[t], lo[t]);
        swim_extremes(x[1], y[1], cur[1], r0.v[2], r0.v[3], scaled, ph, hi[t], lo[t]);
        swim_extremes(x[2], y[2], cur[2], r1.v[0], r1.v[1], scaled, ph, hi[t], lo[t]);
        swim_extremes(x[3], y[3], cur[3], r1.v[2], r1.v[3], scaled, ph, hi[t], lo[t]);
        if (STORE) {
          reinterpret_cast<float4*>(slot_x(slots, ss, t))[g] = make_float4(x[0], x[1], x[2], x[3]);
          reinterpret_cast<float4*>(slot_y(slots, ss, t))[g] = make_float4(y[0], y[1], y[2], y[3]);
        }
      }
    }
  }
  {  // ragged tail: the last n % 4 fish, one per thread
    const uint64_t i = ngroups * 4 + tid;
    if (i < a.n) {
      float x = a.x[i], y = a.y[i];
      float cur = objective(x, y);
#pragma unroll
      for (int t = 0; t < K; ++t) {
        if (FULL || static_cast<uint32_t>(t) < k) {
          const Words2 r = fish_swim_words(a.key, a.school, i, t1 + t);
          swim_extremes(x, y, cur, r.r0, r.r1, scaled, ph, hi[t], lo[t]);
          if (STORE) {
            slot_x(slots, ss, t)[i] = x;
            slot_y(slots, ss, t)[i] = y;
          }
        }
      }
    }
  }

  // ---- per step: the block's maxima into its partial, the last block folds
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  __shared__ uint32_t s_m[K][kBlkWarps], s_e[K][kBlkWarps];
#pragma unroll
  for (int t = 0; t < K; ++t) {
    // prev - cur is never -0 (x - x is +0), so the float extremes order
    // like the keys of fsb_stream.cu
    uint32_t m = 0u, e = 0u;
    if (hi[t] >= lo[t]) {
      m = abs_bits(fmaxf(hi[t], -lo[t]));
      e = order_key(hi[t]);
    }
    m = warp_max(m);
    e = warp_max(e);
    if (lane == 0) {
      s_m[t][warp] = m;
      s_e[t][warp] = e;
    }
  }
  __syncthreads();
  if (warp == 0) {
#pragma unroll
    for (int t = 0; t < K; ++t) {
      if (FULL || static_cast<uint32_t>(t) < k) {
        const uint32_t m = warp_max(lane < kBlkWarps ? s_m[t][lane] : 0u);
        const uint32_t e = warp_max(lane < kBlkWarps ? s_e[t][lane] : 0u);
        if (lane == 0) {
          BlockPartial p{};
          p.max_bits = m;
          p.e_key = e;
          bp[static_cast<uint64_t>(t) * gridDim.x + blockIdx.x] = p;
        }
      }
    }
  }
  if (!arrive_last(a.ctl)) return;
#pragma unroll
  for (int t = 0; t < K; ++t) {
    if (!FULL && static_cast<uint32_t>(t) >= k) continue;
    uint32_t m = 0u, e = 0u;
    for (uint32_t b = threadIdx.x; b < gridDim.x; b += kBlkThreads) {
      const BlockPartial* p = bp + static_cast<uint64_t>(t) * gridDim.x + b;
      const uint32_t pm = static_cast<uint32_t>(__ldcg(&p->max_bits));
      const uint32_t pe = static_cast<uint32_t>(__ldcg(&p->e_key));
      m = pm > m ? pm : m;
      e = pe > e ? pe : e;
    }
    m = warp_max(m);
    e = warp_max(e);
    if (lane == 0) {
      s_m[t][warp] = m;
      s_e[t][warp] = e;
    }
  }
  __syncthreads();
  if (warp == 0) {
#pragma unroll
    for (int t = 0; t < K; ++t) {
      if (!FULL && static_cast<uint32_t>(t) >= k) continue;
      const uint32_t m = warp_max(lane < kBlkWarps ? s_m[t][lane] : 0u);
      const uint32_t e = warp_max(lane < kBlkWarps ? s_e[t][lane] : 0u);
      if (lane == 0) {
        fsb_step_stats* rec = a.ring + (j + t);
        rec->max_abs_delta = static_cast<double>(__uint_as_float(m));
        rec->eat_max_diff = static_cast<double>(key_to_value(e, 0.f));
      }
    }
    if (lane == 0) {
      a.ctl->arrive = 0u;  // the pass index stays: the step pass follows
      __threadfence();
    }
  }
}

// --------------------------------------------------------- step pass --
// One fish through the k steps of a pair: eat of step j + t (normaliser
// N[t]), its barycentre terms, then the swim of step j + t + 1 (STORE: its
// positions from slot t).  `cur` is the objective of the position in hand,
// `pv` the one before its swim; the last swim's objective is not needed.
template <int K, bool STORE, typename Acc>
__device__ __forceinline__ void fish_steps(float& x, float& y, float& w, float& pv, uint64_t i,
                                           const float (&N)[K], uint32_t k, uint32_t t1, Key key,
                                           uint32_t school, const Physics<float>& ph,
                                           Acc (&acc)[K], float* slots, uint64_t ss) {
  float cur = objective(x, y);
#pragma unroll
  for (int t = 0; t < K; ++t) {
    if (static_cast<uint32_t>(t) < k) {
      if (N[t] > 0.f)
        w = eat(w, ph.feed_mode ? __fsub_rn(pv, cur) : __fsub_rn(cur, pv), N[t], ph);
      acc[t].add(w, x, y);
      if (STORE) {
        x = slot_x(slots, ss, t)[i];
        y = slot_y(slots, ss, t)[i];
      } else {
        const Words2 r = fish_swim_words(key, school, i, t1 + t);
        swim_scaled(x, y, r.r0, r.r1, scaled_width(ph.step), ph);
      }
      pv = cur;
      if (static_cast<uint32_t>(t) + 1 < k) cur = objective(x, y);
    }
  }
}

template <int K, int ACC, bool VAR, bool STORE>
__global__ void __launch_bounds__(kBlkThreads, 2)
    blocked_step_kernel(StreamArgs<float> a, uint32_t k, BlockPartial* bp, float* slots,
                        uint64_t ss) {
  using Acc = SumAcc<ACC>;
  using Sum = typename Acc::Sum;
  uint32_t j;
  uint64_t base;
  if (!blocked_prologue<K, false>(a.ctl, a.ring_cap, k, j, base)) return;
  const Physics<float> ph = kernel_physics<VAR>(a.ph);
  const float scaled = scaled_width(ph.step);
  const uint32_t t1 = static_cast<uint32_t>(base + j + 1);
  float N[K];
#pragma unroll
  for (int t = 0; t < K; ++t)
    N[t] = static_cast<uint32_t>(t) < k ? feed_normaliser(a.ring[j - 1 + t], ph) : 0.f;
  Acc acc[K];
  float4* const X = reinterpret_cast<float4*>(a.x);
  float4* const Y = reinterpret_cast<float4*>(a.y);
  float4* const W = reinterpret_cast<float4*>(a.w);
  float4* const PV = reinterpret_cast<float4*>(a.pv);
  const uint64_t ngroups = a.n / 4;
  const uint64_t stride = static_cast<uint64_t>(gridDim.x) * kBlkThreads;
  const uint64_t tid = static_cast<uint64_t>(blockIdx.x) * kBlkThreads + threadIdx.x;
  // kernel 5: the copy cursor runs kLead steps (of this thread's groups in
  // order, k steps each) ahead of the consumer; a step past the thread's
  // last group commits an empty copy group, so that every step commits one
  __shared__ __align__(16) float4 ring[STORE ? kRing : 1][2][kBlkThreads];
  uint64_t pg = tid;
  uint32_t pt = 0, pw = 0, rc = 0;
  // (selects, not branches: past the last group a copy of 0 source bytes
  // from the first group's address zero-fills an entry nobody reads)
  auto issue = [&]() {
    const bool live = pg < ngroups;
    const uint64_t gg = live ? pg : 0u;
    const uint32_t bytes = live ? 16u : 0u;
    cp_async16(&ring[pw][0][threadIdx.x], slot_x(slots, ss, static_cast<int>(pt)) + 4 * gg, bytes);
    cp_async16(&ring[pw][1][threadIdx.x], slot_y(slots, ss, static_cast<int>(pt)) + 4 * gg, bytes);
    const bool wrap = live && pt + 1 == k;
    pg = wrap ? pg + stride : pg;
    pt = wrap ? 0u : (live ? pt + 1 : pt);
    cp_async_commit();
    pw = pw + 1 == kRing ? 0u : pw + 1;
  };
  if (STORE) {
#pragma unroll
    for (int d = 0; d < kLead; ++d) issue();
  }
  // the next group's state is loaded while this one computes
  float4 xn = make_float4(0.f, 0.f, 0.f, 0.f), yn = xn, wn = xn, pn = xn;
  if (tid < ngroups) {
    xn = X[tid];
    yn = Y[tid];
    wn = W[tid];
    pn = PV[tid];
  }
  for (uint64_t g = tid; g < ngroups; g += stride) {
    float x[4] = {xn.x, xn.y, xn.z, xn.w}, y[4] = {yn.x, yn.y, yn.z, yn.w};
    float w[4] = {wn.x, wn.y, wn.z, wn.w}, pv[4] = {pn.x, pn.y, pn.z, pn.w};
    if (g + stride < ngroups) {
      xn = X[g + stride];
      yn = Y[g + stride];
      wn = W[g + stride];
      pn = PV[g + stride];
    }
    float cur[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) cur[q] = objective(x[q], y[q]);
#pragma unroll
    for (int t = 0; t < K; ++t) {
      if (static_cast<uint32_t>(t) < k) {
        {
          // eat for N > 0, else w unchanged: selected, not branched on
          const bool feed = N[t] > 0.f;
          const float Nd = feed ? N[t] : 1.f;
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            const float wn = eat(w[q], ph.feed_mode ? __fsub_rn(pv[q], cur[q])
                                                    : __fsub_rn(cur[q], pv[q]), Nd, ph);
            w[q] = feed ? wn : w[q];
          }
        }
        acc[t].add4(w, x, y);
        if (STORE) {
          cp_async_wait<kLead - 1>();  // this step's copies have landed
          const float4 sx = ring[rc][0][threadIdx.x], sy = ring[rc][1][threadIdx.x];
          rc = rc + 1 == kRing ? 0u : rc + 1;
          x[0] = sx.x; x[1] = sx.y; x[2] = sx.z; x[3] = sx.w;
          y[0] = sy.x; y[1] = sy.y; y[2] = sy.z; y[3] = sy.w;
          issue();  // into the entry read one step before this one
        } else {
          const Words4 r0 = pair_draw(a.key, a.school, 2 * g, t1 + t);
          const Words4 r1 = pair_draw(a.key, a.school, 2 * g + 1, t1 + t);
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            const Words4& r = q < 2 ? r0 : r1;
            swim_scaled(x[q], y[q], r.v[2 * (q & 1)], r.v[2 * (q & 1) + 1], scaled, ph);
          }
        }
        // the objective of the last swim's position is not needed
        const bool more = static_cast<uint32_t>(t) + 1 < k;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          pv[q] = cur[q];
          if (more) cur[q] = objective(x[q], y[q]);
        }
      }
    }
    X[g] = make_float4(x[0], x[1], x[2], x[3]);
    Y[g] = make_float4(y[0], y[1], y[2], y[3]);
    W[g] = make_float4(w[0], w[1], w[2], w[3]);
    PV[g] = make_float4(pv[0], pv[1], pv[2], pv[3]);
  }
  if (STORE) cp_async_wait<0>();  // (every copy issued was consumed)
  {  // ragged tail: the last n % 4 fish, one per thread
    const uint64_t i = ngroups * 4 + tid;
    if (i < a.n) {
      float x = a.x[i], y = a.y[i], w = a.w[i], pv = a.pv[i];
      fish_steps<K, STORE>(x, y, w, pv, i, N, k, t1, a.key, a.school, ph, acc, slots, ss);
      a.x[i] = x;
      a.y[i] = y;
      a.w[i] = w;
      a.pv[i] = pv;
    }
  }

  // ---- per step: the block's sums into its partial, the last block folds
  // them in block order
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  __shared__ Sum s_w[K][kBlkWarps], s_x[K][kBlkWarps], s_y[K][kBlkWarps];
#pragma unroll
  for (int t = 0; t < K; ++t) {
    if (static_cast<uint32_t>(t) >= k) continue;
    const Sum sw = warp_sum(Sum(acc[t].rw())), sx = warp_sum(Sum(acc[t].rx())),
              sy = warp_sum(Sum(acc[t].ry()));
    if (lane == 0) {
      s_w[t][warp] = sw;
      s_x[t][warp] = sx;
      s_y[t][warp] = sy;
    }
  }
  __syncthreads();
  if (warp == 0) {
#pragma unroll
    for (int t = 0; t < K; ++t) {
      if (static_cast<uint32_t>(t) >= k) continue;
      const Sum bw = warp_sum(lane < kBlkWarps ? s_w[t][lane] : Sum(0));
      const Sum bx = warp_sum(lane < kBlkWarps ? s_x[t][lane] : Sum(0));
      const Sum by = warp_sum(lane < kBlkWarps ? s_y[t][lane] : Sum(0));
      if (lane == 0) {
        BlockPartial p{};
        p.sum_w = static_cast<double>(bw);
        p.sum_wx = static_cast<double>(bx);
        p.sum_wy = static_cast<double>(by);
        bp[static_cast<uint64_t>(t) * gridDim.x + blockIdx.x] = p;
      }
    }
  }
  if (!arrive_last(a.ctl)) return;
#pragma unroll
  for (int t = 0; t < K; ++t) {
    if (static_cast<uint32_t>(t) >= k) continue;
    Sum fw = Sum(0), fx = Sum(0), fy = Sum(0);
    for (uint32_t b = threadIdx.x; b < gridDim.x; b += kBlkThreads) {
      const BlockPartial* p = bp + static_cast<uint64_t>(t) * gridDim.x + b;
      fw = sum2(fw, Sum(__ldcg(&p->sum_w)));
      fx = sum2(fx, Sum(__ldcg(&p->sum_wx)));
      fy = sum2(fy, Sum(__ldcg(&p->sum_wy)));
    }
    fw = warp_sum(fw);
    fx = warp_sum(fx);
    fy = warp_sum(fy);
    if (lane == 0) {
      s_w[t][warp] = fw;
      s_x[t][warp] = fx;
      s_y[t][warp] = fy;
    }
  }
  __syncthreads();
  if (warp == 0) {
#pragma unroll
    for (int t = 0; t < K; ++t) {
      if (static_cast<uint32_t>(t) >= k) continue;
      const Sum fw = warp_sum(lane < kBlkWarps ? s_w[t][lane] : Sum(0));
      const Sum fx = warp_sum(lane < kBlkWarps ? s_x[t][lane] : Sum(0));
      const Sum fy = warp_sum(lane < kBlkWarps ? s_y[t][lane] : Sum(0));
      if (lane == 0) {
        fsb_step_stats* rec = a.ring + (j - 1 + t);
        rec->sum_w = static_cast<double>(fw);
        rec->sum_wx = static_cast<double>(fx);
        rec->sum_wy = static_cast<double>(fy);
      }
    }
    if (lane == 0) {
      a.ctl->arrive = 0u;
      a.ctl->pass = j + k;
      __threadfence();
    }
  }
}

template <int K, int ACC, bool STORE>
const void* step_ptr(bool var) {
  return var ? reinterpret_cast<const void*>(&blocked_step_kernel<K, ACC, true, STORE>)
             : reinterpret_cast<const void*>(&blocked_step_kernel<K, ACC, false, STORE>);
}

template <int K, bool STORE>
const void* pick_step(int acc, bool var) {
  switch (acc) {
    case kAccPlain32: return step_ptr<K, kAccPlain32, STORE>(var);
    case kAccKahan32: return step_ptr<K, kAccKahan32, STORE>(var);
    case kAccF64: return step_ptr<K, kAccF64, STORE>(var);
    default: return nullptr;
  }
}

template <int K, bool STORE, bool FULL>
void pick_k(int acc, bool var, const void** maxima, const void** step) {
  *maxima = reinterpret_cast<const void*>(&blocked_maxima_kernel<K, STORE, FULL>);
  *step = pick_step<K, STORE>(acc, var);
}

// The kernels of a pair of up to k_max steps: the maxima pass and the step
// pass (kernel 5 when the slots are set).  Kernel 5's maxima pass has a copy
// for a whole pair (full: k = k_max) without the per-step test of k, which
// the compiler does not take out of the unrolled step loop.  (The step pass
// keeps one copy: knowing k = k_max there, the compiler holds more in
// registers than it has, and spills.)
bool pick_pair(const StreamLaunch& L, bool full, const void** maxima, const void** step) {
  const bool var = L.feed_mode != 0;
  const bool store = L.slots != nullptr;
  switch (L.blocked_k) {
    case 2: store ? (full ? pick_k<2, true, true>(L.acc, var, maxima, step)
                          : pick_k<2, true, false>(L.acc, var, maxima, step))
                  : pick_k<2, false, false>(L.acc, var, maxima, step); break;
    case 4: store ? (full ? pick_k<4, true, true>(L.acc, var, maxima, step)
                          : pick_k<4, true, false>(L.acc, var, maxima, step))
                  : pick_k<4, false, false>(L.acc, var, maxima, step); break;
    case 8: store ? (full ? pick_k<8, true, true>(L.acc, var, maxima, step)
                          : pick_k<8, true, false>(L.acc, var, maxima, step))
                  : pick_k<8, false, false>(L.acc, var, maxima, step); break;
    default: return false;
  }
  return *step != nullptr;
}

}  // namespace

bool stream_blocked_supported(const StreamLaunch& L) {
  // step 0 or |step| >= 2^-103: its product with 2^-23 is exact
  const float step = static_cast<float>(L.step);
  return !L.real_is_double && L.vec == 4 && L.swim_mode == 0 &&
         (step == 0.f || fabsf(step) >= 0x1p-103f);
}

int stream_blocked_blocks_per_sm(const StreamLaunch& L) {
  int best = 0;
  for (bool full : {false, true}) {  // both copies of a pair run on the one grid
    const void* fa = nullptr;
    const void* fb = nullptr;
    if (!pick_pair(L, full, &fa, &fb)) return 0;
    int na = 0, nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&na, fa, kBlkThreads, 0) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, fb, kBlkThreads, 0) != cudaSuccess)
      return 0;
    const int m = na < nb ? na : nb;
    best = full ? (m < best ? m : best) : m;
  }
  return best;
}

cudaError_t launch_blocked_pair(const StreamLaunch& L, uint32_t k, cudaStream_t s) {
  const void* fa = nullptr;
  const void* fb = nullptr;
  if (!pick_pair(L, k == static_cast<uint32_t>(L.blocked_k), &fa, &fb) || L.bgrid <= 0 ||
      !L.bpartials || k == 0 || k > static_cast<uint32_t>(L.blocked_k))
    return cudaErrorInvalidValue;
  if (L.slots && L.slot_stride % 4 != 0) return cudaErrorInvalidValue;
  StreamArgs<float> a = make_stream_args<float>(L);
  BlockPartial* bp = L.bpartials;
  float* slots = L.slots;
  uint64_t ss = L.slot_stride;
  void* args[] = {&a, &k, &bp, &slots, &ss};
  cudaError_t e = cudaLaunchKernel(fa, dim3(L.bgrid), dim3(kBlkThreads), args, 0, s);
  if (e != cudaSuccess) return e;
  return cudaLaunchKernel(fb, dim3(L.bgrid), dim3(kBlkThreads), args, 0, s);
}

}  // namespace fsb
