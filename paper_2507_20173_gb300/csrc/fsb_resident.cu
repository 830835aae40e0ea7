// fsb_resident.cu -- the on-chip ("resident") single-school kernel.
//
// One cooperative launch advances a school by all n_steps of an fsb_step call.
// Each thread keeps FPT fish (x, y, weight, currentObjective and
// prevObjective) in registers for the whole call; HBM is read once at the
// start and written once at the end.  Each step follows the paper's order
// (Sec. 2.1.2 swim, Sec. 2.1.1 objective, delta, the Sec. 2.3.2 max
// reduction, feeding, barycentre), with the phases of consecutive steps
// overlapped:
//   A. swim + objective + delta of step u+1 for every fish (positions do not
//      depend on weights), while the grid is still agreeing on M_u;
//   B. thread 0 waits for barrier u (one arrival per block on a monotonic
//      counter; the wait is bounded by a %globaltimer deadline and gives up
//      with FSB_ERR_TIMEOUT, so a missing block can never hang the GPU) and
//      reads M_u and the eat() value max(prev - cur) from a rotating slot
//      that every block fed with one atomicMax (exact, order-free);
//   C. eat of step u from the parked (delta, x, y) of step u, barycentre
//      partials of step u;
//   D. one block reduction for the maxima of step u+1 and the sums of step u;
//      thread 0 writes the sums, feeds the slot of step u+1 and arrives.
// After the last step the state is written back, a final barrier is taken
// and the per-step partials are folded in a fixed order into the statistics
// ring.  If any wait gives up, every block leaves without writing state, so
// a failed call leaves the school as it was.
#include <cstdint>

#include "fsb_device.cuh"
#include "fsb_internal.h"
#include "fsb_reduce.cuh"

namespace fsb {
namespace {

struct ResidentArgs {
  float* __restrict__ x;
  float* __restrict__ y;
  float* __restrict__ w;
  float* __restrict__ pv;
  uint64_t n;
  uint64_t slice;
  Key key;
  uint32_t school;
  Physics<float> ph;
  uint64_t base_step;
  uint32_t n_steps;
  Ctl* ctl;
  ResCtl* rctl;
  double* sums;
  fsb_step_stats* ring;
  unsigned long long timeout_ns;
  int inject_cta;
  uint32_t inject_step;
};

// Split-phase grid barrier.  Arrival: one release-ordered increment of a
// monotonic counter per block (the block's prior writes -- max slots,
// barycentre partials -- become visible first).  Wait: thread 0 spins until
// barrier k has all arrivals, bounded by a %globaltimer deadline.
__device__ __forceinline__ void grid_arrive(const ResidentArgs& a) {
  asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(&a.rctl->bar_count), "r"(1u)
               : "memory");
}

__device__ __forceinline__ bool grid_wait(const ResidentArgs& a, unsigned k) {
  return bounded_wait_geq(&a.rctl->bar_count, k * gridDim.x, &a.ctl->status,
                          &a.ctl->timeout_site, k, a.timeout_ns);
}

// The resident loop is software-pipelined so the barrier's latency hides
// behind arithmetic: while the grid agrees on M_u, every block already swims
// step u + 1 (positions do not depend on weights).  Eating step u then needs
// that step's delta and post-swim position, which wait in a double-buffered
// shared-memory slab `pend[buffer][delta | x | y][fish slot][thread]`.
// WSWIM: the weight-scaled swim (each fish's half-width is (w / w0) s with
// its weight after the previous step's eat).  The swim of step u + 1 then
// waits for the eat of step u, so it runs after it instead of beside the
// barrier.
template <int FPT, int MAXB, int ACC, bool WSWIM>
__global__ void __launch_bounds__(MAXB, 1) resident_kernel(ResidentArgs a) {
  using Acc = SumAcc<ACC>;
  using Sum = typename Acc::Sum;
  using Part = typename Acc::Part;
  extern __shared__ float pend[];
  __shared__ uint32_t s_max[32], s_ekey[32];
  __shared__ Part s_w[32], s_x[32], s_y[32];
  __shared__ uint32_t s_M, s_E;
  __shared__ int s_abort;

  const int B = blockDim.x;
  const int nw = (B + 31) >> 5;
  const int tid = threadIdx.x;
  const int lane = tid & 31, warp = tid >> 5;
  const bool multi = gridDim.x > 1;
  // a resident school holds at most ~2.5 million fish, so indices fit 32
  // bits.  The thread owns fish pairs (one swim block moves a pair): slot k
  // is fish lo + 2 (tid + (k / 2) B) + k % 2, and slots k < nk are in the
  // school (the slice, hence lo, is even)
  const uint32_t lo = static_cast<uint32_t>(blockIdx.x * a.slice);
  const uint32_t hi = static_cast<uint32_t>(lo + a.slice < a.n ? lo + a.slice : a.n);
  auto fish = [&](int k) -> uint32_t {
    return lo + 2u * (static_cast<uint32_t>(tid) + static_cast<uint32_t>(k >> 1) * B) +
           static_cast<uint32_t>(k & 1);
  };
  int nk = 0;
#pragma unroll
  for (int k = 0; k < FPT; ++k)
    if (fish(k) < hi) nk = k + 1;
  auto P = [&](uint32_t buf, int q, int k) -> float& {
    return pend[((buf * 3 + q) * FPT + k) * B + tid];
  };

  float x[FPT], y[FPT], w[FPT], f[FPT], pv[FPT];
#pragma unroll
  for (int k = 0; k < FPT; ++k) {
    const uint32_t i = fish(k);
    if (k < nk) {
      x[k] = a.x[i];
      y[k] = a.y[i];
      w[k] = a.w[i];
      f[k] = objective(x[k], y[k]);
    } else {
      x[k] = y[k] = w[k] = f[k] = 0.f;
    }
    pv[k] = f[k];
  }
  if (tid == 0) s_abort = 0;

  // swim of step u for every fish of this thread; parks (delta, x, y) in
  // pend[u & 1] and returns the thread's maxima
  auto swim_all = [&](uint32_t u, uint32_t& mb, uint32_t& ek) {
    const uint32_t t = static_cast<uint32_t>(a.base_step + u);
    mb = 0;
    ek = 0;
    Words4 r{};
#pragma unroll
    for (int k = 0; k < FPT; ++k) {
      if (k < nk) {
        pv[k] = f[k];
        if ((k & 1) == 0) r = pair_draw(a.key, a.school, fish(k) >> 1, t);
        swim(x[k], y[k], r.v[2 * (k & 1)], r.v[2 * (k & 1) + 1],
             WSWIM ? swim_width(a.ph, w[k]) : a.ph.step, a.ph);
        f[k] = objective(x[k], y[k]);
        const float d = __fsub_rn(f[k], pv[k]);
        const uint32_t m = abs_bits(d);
        const uint32_t e = order_key(__fsub_rn(pv[k], f[k]));
        mb = m > mb ? m : mb;
        ek = e > ek ? e : ek;
        P(u & 1u, 0, k) = d;
        P(u & 1u, 1, k) = x[k];
        P(u & 1u, 2, k) = y[k];
      }
    }
  };

  // thread 0: hand the block's maxima of step u to the grid (one atomicMax
  // per slot, then the arrival at barrier u), or keep them for a lone block
  auto publish = [&](uint32_t u, uint32_t m, uint32_t e) {
    if (multi) {
      atomicMax(&a.rctl->max_slot[u % 3], m);
      atomicMax(&a.rctl->ekey_slot[u % 3], e);
      const bool skip = static_cast<int>(blockIdx.x) == a.inject_cta && u - 1 == a.inject_step;
      if (!skip) grid_arrive(a);
    } else {
      s_M = m;
      s_E = e;
    }
  };

  // ---- prologue: swim of step 1
  {
    uint32_t mb, ek;
    swim_all(1, mb, ek);
    mb = warp_max(mb);
    ek = warp_max(ek);
    if (lane == 0) {
      s_max[warp] = mb;
      s_ekey[warp] = ek;
    }
    __syncthreads();
    if (warp == 0) {
      uint32_t m = lane < nw ? s_max[lane] : 0u;
      uint32_t e = lane < nw ? s_ekey[lane] : 0u;
      m = warp_max(m);
      e = warp_max(e);
      if (lane == 0) publish(1, m, e);
    }
  }

  for (uint32_t u = 1; u <= a.n_steps; ++u) {
    const bool has_next = u < a.n_steps;
    // ---- A: swim of step u + 1 while the grid settles M_u
    uint32_t mb = 0, ek = 0;
    if (!WSWIM && has_next) swim_all(u + 1, mb, ek);

    // ---- B: M_u
    if (tid == 0) {
      if (multi) {
        if (grid_wait(a, u)) {
          s_M = atomicAdd(&a.rctl->max_slot[u % 3], 0u);
          s_E = atomicAdd(&a.rctl->ekey_slot[u % 3], 0u);
          // slot (u + 2) % 3 was last read before barrier u and is next
          // written after barrier u + 1
          if (blockIdx.x == 0) {
            a.rctl->max_slot[(u + 2) % 3] = 0u;
            a.rctl->ekey_slot[(u + 2) % 3] = 0u;
          }
        } else {
          s_abort = 1;
        }
      }
      if (blockIdx.x == 0 && !s_abort) {
        a.ring[u - 1].max_abs_delta = static_cast<double>(__uint_as_float(s_M));
        a.ring[u - 1].eat_max_diff = static_cast<double>(key_to_value(s_E, 0.f));
      }
    }
    __syncthreads();
    if (s_abort) return;
    // feeding normaliser: M_u, or the paper's eat() value E_u (then the
    // numerator is prev - cur = -delta, exactly, and a zero delta gives the
    // same weight either sign)
    const float M = a.ph.feed_mode ? key_to_value(s_E, 0.f) : __uint_as_float(s_M);

    // ---- C: eat of step u and its barycentre partials
    Acc acc;
#pragma unroll
    for (int k = 0; k < FPT; ++k) {
      if (k < nk) {
        if (M > 0.f) {
          const float d = P(u & 1u, 0, k);
          w[k] = eat(w[k], a.ph.feed_mode ? -d : d, M, a.ph);
        }
        acc.add(w[k], P(u & 1u, 1, k), P(u & 1u, 2, k));
      }
    }
    // ---- A (weight-scaled swim): swim of step u + 1 with the eaten weights
    if (WSWIM && has_next) swim_all(u + 1, mb, ek);

    // ---- D: one block reduction for M_{u+1}, E_{u+1} and the sums of u
    mb = warp_max(mb);
    ek = warp_max(ek);
    Part sw = warp_tree(acc.pw()), sx = warp_tree(acc.px()), sy = warp_tree(acc.py());
    if (lane == 0) {
      s_max[warp] = mb;
      s_ekey[warp] = ek;
      s_w[warp] = sw;
      s_x[warp] = sx;
      s_y[warp] = sy;
    }
    __syncthreads();
    if (warp == 0) {
      uint32_t m = lane < nw ? s_max[lane] : 0u;
      uint32_t e = lane < nw ? s_ekey[lane] : 0u;
      sw = lane < nw ? s_w[lane] : part_zero<Part>();
      sx = lane < nw ? s_x[lane] : part_zero<Part>();
      sy = lane < nw ? s_y[lane] : part_zero<Part>();
      m = warp_max(m);
      e = warp_max(e);
      sw = warp_merge(sw);
      sx = warp_merge(sx);
      sy = warp_merge(sy);
      if (lane == 0) {
        double* p = a.sums + (static_cast<uint64_t>(u - 1) * gridDim.x + blockIdx.x) * 3;
        p[0] = to_double(sw);
        p[1] = to_double(sx);
        p[2] = to_double(sy);
        if (has_next)
          publish(u + 1, m, e);
        else if (multi)
          grid_arrive(a);  // final barrier: every block's partials are out
      }
    }
    // the next iteration's first __syncthreads orders reuse of the arrays
  }

  // ---- write the state back
#pragma unroll
  for (int k = 0; k < FPT; ++k) {
    const uint32_t i = fish(k);
    if (k < nk) {
      a.x[i] = x[k];
      a.y[i] = y[k];
      a.w[i] = w[k];
      a.pv[i] = pv[k];
    }
  }

  // ---- final barrier, then fold the barycentre partials step by step
  __syncthreads();
  if (tid == 0 && multi && !grid_wait(a, a.n_steps + 1)) s_abort = 1;
  __syncthreads();
  if (s_abort) return;
  __shared__ Sum f_w[32], f_x[32], f_y[32];
  for (uint32_t s = blockIdx.x; s < a.n_steps; s += gridDim.x) {
    Sum fw = Sum(0), fx = Sum(0), fy = Sum(0);
    for (uint32_t b = tid; b < gridDim.x; b += B) {
      const double* p = a.sums + (static_cast<uint64_t>(s) * gridDim.x + b) * 3;
      fw = sum2(fw, Sum(__ldcg(p + 0)));
      fx = sum2(fx, Sum(__ldcg(p + 1)));
      fy = sum2(fy, Sum(__ldcg(p + 2)));
    }
    fw = warp_sum(fw);
    fx = warp_sum(fx);
    fy = warp_sum(fy);
    __syncthreads();
    if (lane == 0) {
      f_w[warp] = fw;
      f_x[warp] = fx;
      f_y[warp] = fy;
    }
    __syncthreads();
    if (warp == 0) {
      fw = lane < nw ? f_w[lane] : Sum(0);
      fx = lane < nw ? f_x[lane] : Sum(0);
      fy = lane < nw ? f_y[lane] : Sum(0);
      fw = warp_sum(fw);
      fx = warp_sum(fx);
      fy = warp_sum(fy);
      if (lane == 0) {
        a.ring[s].sum_w = static_cast<double>(fw);
        a.ring[s].sum_wx = static_cast<double>(fx);
        a.ring[s].sum_wy = static_cast<double>(fy);
      }
    }
  }
}

// Largest block each fish-per-thread variant is compiled for (registers:
// five per fish plus the Philox and reduction temporaries).
template <int FPT>
struct MaxBlock;
template <>
struct MaxBlock<4> {
  static constexpr int value = 1024;
};
template <>
struct MaxBlock<8> {
  static constexpr int value = 896;
};
template <>
struct MaxBlock<12> {
  static constexpr int value = 640;
};
template <>
struct MaxBlock<16> {
  static constexpr int value = 512;
};

template <int FPT, int ACC>
const void* kernel_ptr(bool wswim) {
  constexpr int MB = MaxBlock<FPT>::value;
  if (wswim) return reinterpret_cast<const void*>(&resident_kernel<FPT, MB, ACC, true>);
  return reinterpret_cast<const void*>(&resident_kernel<FPT, MB, ACC, false>);
}

template <int FPT>
const void* pick_acc(int acc, bool wswim) {
  switch (acc) {
    case kAccPlain32: return kernel_ptr<FPT, kAccPlain32>(wswim);
    case kAccKahan32: return kernel_ptr<FPT, kAccKahan32>(wswim);
    case kAccF64: return kernel_ptr<FPT, kAccF64>(wswim);
    default: return nullptr;
  }
}

const void* pick(int fpt, int acc, bool wswim) {
  switch (fpt) {
    case 4: return pick_acc<4>(acc, wswim);
    case 8: return pick_acc<8>(acc, wswim);
    case 12: return pick_acc<12>(acc, wswim);
    case 16: return pick_acc<16>(acc, wswim);
    default: return nullptr;
  }
}

}  // namespace

int resident_max_block(int fpt) {
  switch (fpt) {
    case 4: return MaxBlock<4>::value;
    case 8: return MaxBlock<8>::value;
    case 12: return MaxBlock<12>::value;
    case 16: return MaxBlock<16>::value;
    default: return 0;
  }
}

size_t resident_smem_bytes(int fpt, int block) {
  return static_cast<size_t>(2) * 3 * fpt * block * sizeof(float);
}

int resident_blocks_per_sm(int fpt, int acc, int block, int swim_mode) {
  const void* fn = pick(fpt, acc, swim_mode != 0);
  if (!fn) return 0;
  const size_t smem = resident_smem_bytes(fpt, block);
  // the attribute is per kernel, shared by every handle: always the largest
  // slab this variant can ask for, so no handle lowers it under another
  const size_t most = resident_smem_bytes(fpt, resident_max_block(fpt));
  if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           static_cast<int>(most)) != cudaSuccess)
    return 0;
  int nb = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, fn, block, smem) != cudaSuccess) return 0;
  return nb;
}

cudaError_t launch_resident(const ResidentLaunch& L, cudaStream_t s) {
  const void* fn = pick(L.fpt, L.acc, L.swim_mode != 0);
  if (!fn || L.grid < 1 || L.block < 32 || L.block > resident_max_block(L.fpt))
    return cudaErrorInvalidValue;
  ResidentArgs a;
  a.x = static_cast<float*>(L.x);
  a.y = static_cast<float*>(L.y);
  a.w = static_cast<float*>(L.w);
  a.pv = static_cast<float*>(L.pv);
  a.n = L.n;
  a.slice = L.slice;
  a.key.k0 = static_cast<uint32_t>(L.seed);
  a.key.k1 = static_cast<uint32_t>(L.seed >> 32);
  a.school = L.school;
  a.ph.pond_half = static_cast<float>(L.pond_half);
  a.ph.step = static_cast<float>(L.step);
  a.ph.w0 = static_cast<float>(L.w0);
  a.ph.w_min = static_cast<float>(L.w_min);
  a.ph.w_max = static_cast<float>(L.w_max);
  a.ph.swim_mode = L.swim_mode;
  a.ph.feed_mode = L.feed_mode;
  a.base_step = L.base_step;
  a.n_steps = L.n_steps;
  a.ctl = L.ctl;
  a.rctl = L.rctl;
  a.sums = L.sums;
  a.ring = L.ring;
  a.timeout_ns = L.timeout_ns;
  a.inject_cta = L.inject_cta;
  a.inject_step = L.inject_step;
  void* args[] = {&a};
  cudaError_t e = cudaMemsetAsync(L.rctl, 0, sizeof(ResCtl), s);
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(L.grid);
  cfg.blockDim = dim3(L.block);
  cfg.dynamicSmemBytes = resident_smem_bytes(L.fpt, L.block);
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = L.grid > 1 ? 1 : 0;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelExC(&cfg, fn, args);
}

}  // namespace fsb
