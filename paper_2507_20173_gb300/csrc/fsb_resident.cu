// fsb_resident.cu -- the on-chip ("resident") single-school kernel.
//
// One cooperative launch advances a school by all n_steps of an fsb_step call.
// Each block keeps its slice of the school in shared memory for the whole
// call (HBM is read once at the start and written once at the end) and walks
// it with the compact per-pair passes of fsb_onchip.cuh.  Each step follows
// the paper's order (Sec. 2.1.2 swim, Sec. 2.1.1 objective, delta, the
// Sec. 2.3.2 max reduction, feeding, barycentre), with the phases of
// consecutive steps overlapped.  Positions do not depend on weights, so the
// swims run two steps ahead of the eats: one pass over a block's fish eats
// step u (reading step u's positions and feeding input from one half of
// double-buffered arrays) and swims step u + 2 (from step u + 1's positions
// in the other half, written back over step u's pair by pair), and the
// warps' maxima of step u + 2 meet in shared memory by atomics.  One
// synchronisation warp per block does all the grid-wide work beside them:
// it waits for barrier u (one arrival per block on a monotonic counter; the
// wait is bounded by a %globaltimer deadline and gives up with
// FSB_ERR_TIMEOUT, so a missing block can never hang the GPU), reads M_u and
// the eat() value max(prev - cur) from a rotating slot that every block fed
// with one atomicMax (exact, order-free), hands the block's maxima of step
// u + 1 to the grid, arrives at barrier u + 1 and folds the block's
// barycentre partials -- so M_{u+1} has a whole pass to cross the grid.
// The weight-scaled swim (its width depends on the eaten weight) cannot run
// ahead; its passes eat step u and swim step u + 1.
// After the last step the state is written back, a final barrier is taken
// and the per-step partials are folded in a fixed order into the statistics
// ring.  If any wait gives up, every block leaves without writing state, so
// a failed call leaves the school as it was.
#include <cstdint>

#include "fsb_check.cuh"
#include "fsb_device.cuh"
#include "fsb_internal.h"
#include "fsb_onchip.cuh"
#include "fsb_reduce.cuh"

namespace fsb {
namespace {

#ifndef FSB_RESIDENT_FISH_THREADS
#define FSB_RESIDENT_FISH_THREADS 512
#endif
// most fish threads per block (one more warp synchronises)
constexpr int kResThreads = FSB_RESIDENT_FISH_THREADS;
static_assert(kResThreads % 32 == 0 && kResThreads <= 992, "fish threads: whole warps, <= 31");
// shared memory per fish: x and y (two buffers), feeding input (two
// buffers), currentObjective and weight, binary32 each
constexpr size_t kResSmemPerFish = 8 * sizeof(float);
// largest slice a block holds (its arrays fill the opt-in shared memory)
constexpr uint64_t kResMaxSlice = 7168;

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

template <typename Part>
struct ResPart3 {
  Part w, x, y;
};

// Named hardware barriers between the fish warps and the synchronisation
// warp (id 0 is __syncthreads).  Each handover alternates between two ids by
// step parity, so an arrival for step u + 2 can never join a phase of step u.
__device__ __forceinline__ void named_arrive(int id, int threads) {
  asm volatile("bar.arrive %0, %1;" ::"r"(id), "r"(threads) : "memory");
}
__device__ __forceinline__ void named_sync(int id, int threads) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(threads) : "memory");
}
constexpr int kBarM = 1;    // ids 1, 2: "M_u is in s_M[u & 1]" (sync warp -> fish warps)
constexpr int kBarMax = 3;  // ids 3, 4: "the block's maxima of step u are in s_bmax[u & 1]
                            //            and every warp's partials of step u - 2 are out"

// The block is blockDim.x - 32 fish threads (warps 0 .. nw - 1) and one
// synchronisation warp (the last).  The fish warps only swim, eat and meet
// the synchronisation warp at the two named handovers per step; the
// synchronisation warp does all the grid-wide work: it waits for barrier u,
// reads M_u, hands the block's maxima of step u + 1 to the grid, arrives at
// barrier u + 1 and folds the block's barycentre partials, while the fish
// warps swim.
// WSWIM: the weight-scaled swim (each fish's half-width is (w / w0) s with
// its weight after the previous step's eat).  The swim of step u + 1 then
// waits for the eat of step u, so it runs fused with it, after M_u.
template <int ACC, bool WSWIM>
__global__ void __launch_bounds__(kResThreads + 32, 1) resident_kernel(ResidentArgs a) {
  using Acc = OnchipAcc<ACC>;
  using Sum = typename Acc::Sum;
  using Part = typename Acc::Part;
  extern __shared__ __align__(16) float2 res_smem[];
  __shared__ uint32_t s_bmax[2], s_bkey[2];  // the block's maxima of a step, by parity
  __shared__ ResPart3<Part> s_wpart[2][32];  // the warps' barycentre partials, by parity
  __shared__ uint32_t s_M[2], s_E[2];        // M_u and E_u, by parity
  __shared__ int s_abort;

  const int tid = threadIdx.x;
  const int nthreads = blockDim.x;             // fish threads + the sync warp
  const int fish_threads = nthreads - 32;
  const int nw = fish_threads >> 5;            // fish warps
  const int lane = tid & 31, warp = tid >> 5;
  const bool sync_warp = warp == nw;
  const bool multi = gridDim.x > 1;
  // a resident school holds at most ~1.1 million fish, so indices fit 32
  // bits; the slice (hence lo) is even, so no swim pair straddles two blocks
  const uint32_t lo = static_cast<uint32_t>(blockIdx.x * a.slice);
  const uint32_t hi = static_cast<uint32_t>(lo + a.slice < a.n ? lo + a.slice : a.n);
  const uint32_t cap = static_cast<uint32_t>(a.slice / 2);  // pairs per array
  // the slice fits the arrays, and the grid covers the school (host-checked)
  const uint32_t nf0 = hi > lo ? hi - lo : 0u;
  const bool fits = fsb_check(nf0 <= 2 * cap && static_cast<uint64_t>(gridDim.x) * a.slice >= a.n,
                              &a.ctl->status, &a.ctl->timeout_site, 0xB0u);
  const uint32_t nf = fits ? nf0 : (nf0 < 2 * cap ? nf0 : 2 * cap);
  const uint32_t np = (nf + 1) / 2;
  float4* const XY0 = reinterpret_cast<float4*>(res_smem);
  float4* const XY1 = reinterpret_cast<float4*>(res_smem + 2 * cap);
  float2* const D0 = res_smem + 4 * cap;
  float2* const D1 = res_smem + 5 * cap;
  float2* const F = res_smem + 6 * cap;
  float2* const W = res_smem + 7 * cap;
  // buffer k holds the positions after (and the feeding input of) the steps
  // of parity k
  auto state = [&](uint32_t from, uint32_t to) -> PairState {
    return pair_state(from & 1u ? XY1 : XY0, from & 1u ? D1 : D0, to & 1u ? XY1 : XY0,
                      to & 1u ? D1 : D0, F, W);
  };
  // the pipelined pass of step u: eat step u from buffer u & 1 while the
  // swim of step u + 2 reads buffer (u + 1) & 1 and overwrites buffer u & 1
  auto ahead_state = [&](uint32_t u) -> PairState {
    float4* const XYu = u & 1u ? XY1 : XY0;
    float2* const Du = u & 1u ? D1 : D0;
    return PairState{XYu, Du, u & 1u ? XY0 : XY1, XYu, Du, F, W};
  };
  const Physics<float> ph = a.ph;
  const uint32_t T = a.n_steps;
  if (T == 0) return;  // calls advance by at least one step

  for (uint32_t e = tid; e < np; e += nthreads) {
    float xv[2] = {0.f, 0.f}, yv[2] = {0.f, 0.f}, wv[2] = {0.f, 0.f}, fv[2] = {0.f, 0.f};
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      if (2 * e + h < nf) {
        const uint32_t i = lo + 2 * e + h;
        xv[h] = a.x[i];
        yv[h] = a.y[i];
        wv[h] = a.w[i];
        fv[h] = objective(xv[h], yv[h]);
      }
    }
    XY0[e] = make_float4(xv[0], xv[1], yv[0], yv[1]);
    W[e] = make_float2(wv[0], wv[1]);
    F[e] = make_float2(fv[0], fv[1]);
  }
  if (tid == 0) {
    s_abort = 0;
    s_bmax[0] = s_bmax[1] = 0u;
    s_bkey[0] = s_bkey[1] = 0u;
  }
  __syncthreads();

  if (sync_warp) {
    // ---- the synchronisation warp
    // fold of the block's barycentre partial of step u, raw, into a.sums
    auto fold_sums = [&](uint32_t u) {
      const ResPart3<Part>* wp = s_wpart[u & 1u];
      Part w = lane < nw ? wp[lane].w : part_zero<Part>();
      Part x = lane < nw ? wp[lane].x : part_zero<Part>();
      Part y = lane < nw ? wp[lane].y : part_zero<Part>();
      w = warp_merge(w);
      x = warp_merge(x);
      y = warp_merge(y);
      if (lane == 0) {
        double* p = a.sums + (static_cast<uint64_t>(u - 1) * gridDim.x + blockIdx.x) * 3;
        p[0] = raw_sum(w);
        p[1] = raw_sum(x);
        p[2] = raw_sum(y);
      }
    };
    // the block's maxima of step u to the grid (one atomicMax per slot,
    // then the arrival at barrier u); a lone block passes them on directly
    auto publish = [&](uint32_t u) {
      if (lane == 0 && multi) {
        atomicMax(&a.rctl->max_slot[u % 3], s_bmax[u & 1u]);
        atomicMax(&a.rctl->ekey_slot[u % 3], s_bkey[u & 1u]);
        s_bmax[u & 1u] = 0u;
        s_bkey[u & 1u] = 0u;
        const bool skip = static_cast<int>(blockIdx.x) == a.inject_cta && u - 1 == a.inject_step;
        if (!skip) grid_arrive(a);
      }
    };
    named_sync(kBarMax + 1, nthreads);  // maxima of step 1
    publish(1);
    for (uint32_t u = 1; u <= T; ++u) {
      if (lane == 0) {
        bool ok = true;
        uint32_t m, e;
        if (multi) {
          ok = grid_wait(a, u);
          m = ld_relaxed_u32(&a.rctl->max_slot[u % 3]);
          e = ld_relaxed_u32(&a.rctl->ekey_slot[u % 3]);
          // slot (u + 2) % 3 was last read before barrier u and is next
          // written after barrier u + 1
          if (ok && blockIdx.x == 0) {
            a.rctl->max_slot[(u + 2) % 3] = 0u;
            a.rctl->ekey_slot[(u + 2) % 3] = 0u;
          }
        } else {
          m = s_bmax[u & 1u];
          e = s_bkey[u & 1u];
          s_bmax[u & 1u] = 0u;
          s_bkey[u & 1u] = 0u;
        }
        if (!ok) s_abort = 1;
        s_M[u & 1u] = m;
        s_E[u & 1u] = e;
        if (ok && blockIdx.x == 0) {
          a.ring[u - 1].max_abs_delta = static_cast<double>(__uint_as_float(m));
          a.ring[u - 1].eat_max_diff = static_cast<double>(key_to_value(e, 0.f));
        }
      }
      __syncwarp();
      named_arrive(kBarM + (u & 1u), nthreads);
      if (s_abort) return;
      if (u < T) {
        // the fish warps' maxima of step u + 1 (and, with them, their
        // partials of step u - 1)
        named_sync(kBarMax + ((u + 1) & 1u), nthreads);
        publish(u + 1);
        if (u > 1) fold_sums(u - 1);
      }
    }
  } else {
    // ---- the fish warps
    PassCtx c{a.key, a.school, lo / 2, 0u, 0.f, exact_scaled_width(ph.step)};
    // swim of step u from buffer (u - 1) & 1 into buffer u & 1 (fused with
    // the eat of step u - 1 when eat_too); the warps' maxima into
    // s_bmax[u & 1], then the handover to the synchronisation warp
    auto swim_pass = [&](uint32_t u, bool eat_too, Acc& acc) {
      uint32_t mb = 0, ek = 0;
      c.t = static_cast<uint32_t>(a.base_step + u);
      const PairState B = state(u - 1, u);
      if (!eat_too) {
        if (u == T)
          block_pass<false, true, true, false, false, 2, !WSWIM>(B, np, nf, c, ph, acc, mb, ek,
                                                               fish_threads);
        else
          block_pass<false, true, false, false, false, 2, !WSWIM>(B, np, nf, c, ph, acc, mb, ek,
                                                                fish_threads);
      } else {
        if (u == T)
          block_pass<true, true, true, false, false, 2, !WSWIM>(B, np, nf, c, ph, acc, mb, ek,
                                                              fish_threads);
        else
          block_pass<true, true, false, false, false, 2, !WSWIM>(B, np, nf, c, ph, acc, mb, ek,
                                                               fish_threads);
      }
      mb = warp_max(mb);
      ek = warp_max(ek);
      if (lane == 0) {
        atomicMax(&s_bmax[u & 1u], mb);
        atomicMax(&s_bkey[u & 1u], ek);
      }
    };
    auto put_partial = [&](uint32_t u, const Acc& acc) {
      warp_partials(&s_wpart[u & 1u][warp], acc.pw(), acc.px(), acc.py());
    };
    {
      Acc unused;
      swim_pass(1, false, unused);
      named_arrive(kBarMax + 1, nthreads);
      if (!WSWIM && T >= 2) {
        swim_pass(2, false, unused);
        named_arrive(kBarMax + 0, nthreads);
      }
    }
    for (uint32_t u = 1; u <= T; ++u) {
      // ---- M_u from the synchronisation warp
      named_sync(kBarM + (u & 1u), nthreads);
      if (s_abort) return;
      c.N = ph.feed_mode ? key_to_value(s_E[u & 1u], 0.f) : __uint_as_float(s_M[u & 1u]);
      Acc acc;
      if (WSWIM && u < T) {
        // eat of step u fused with the swim of step u + 1 (the swim needs
        // the eaten weights)
        swim_pass(u + 1, true, acc);
        put_partial(u, acc);
        named_arrive(kBarMax + ((u + 1) & 1u), nthreads);
      } else if (!WSWIM && u + 2 <= T) {
        // eat of step u fused with the swim of step u + 2: positions do not
        // depend on weights, so the swims run two steps ahead and M_{u+2}
        // has a whole pass to cross the grid
        uint32_t mb = 0, ek = 0;
        c.t = static_cast<uint32_t>(a.base_step + u + 2);
        const PairState B = ahead_state(u);
        if (u + 2 == T)
          block_pass<true, true, true, false, true, 2, !WSWIM>(B, np, nf, c, ph, acc, mb, ek,
                                                             fish_threads);
        else
          block_pass<true, true, false, false, true, 2, !WSWIM>(B, np, nf, c, ph, acc, mb, ek,
                                                              fish_threads);
        mb = warp_max(mb);
        ek = warp_max(ek);
        if (lane == 0) {
          atomicMax(&s_bmax[u & 1u], mb);  // step u + 2 has the parity of u
          atomicMax(&s_bkey[u & 1u], ek);
        }
        put_partial(u, acc);
        named_arrive(kBarMax + (u & 1u), nthreads);
      } else {
        // eat of step u alone
        uint32_t mb = 0, ek = 0;
        const PairState B = state(u, u);
        if (u == T)
          block_pass<true, false, false, true>(B, np, nf, c, ph, acc, mb, ek, fish_threads);
        else
          block_pass<true, false, false, false>(B, np, nf, c, ph, acc, mb, ek, fish_threads);
        put_partial(u, acc);
      }
    }
  }

  // ---- the last partials, then write the state back
  __syncthreads();
  if (sync_warp) {
    // steps T - 1 (if not folded in the loop) and T
    for (uint32_t u = T > 1 ? T - 1 : 1; u <= T; ++u) {
      const ResPart3<Part>* wp = s_wpart[u & 1u];
      Part w = lane < nw ? wp[lane].w : part_zero<Part>();
      Part x = lane < nw ? wp[lane].x : part_zero<Part>();
      Part y = lane < nw ? wp[lane].y : part_zero<Part>();
      w = warp_merge(w);
      x = warp_merge(x);
      y = warp_merge(y);
      if (lane == 0) {
        double* p = a.sums + (static_cast<uint64_t>(u - 1) * gridDim.x + blockIdx.x) * 3;
        p[0] = raw_sum(w);
        p[1] = raw_sum(x);
        p[2] = raw_sum(y);
      }
    }
  }
  for (uint32_t e = tid; e < np; e += nthreads) {
    const float4 p = (T & 1u ? XY1 : XY0)[e];
    const float2 xv = make_float2(p.x, p.y), yv = make_float2(p.z, p.w), wv = W[e];
    const float2 pv = T ? (T & 1u ? D1 : D0)[e] : F[e];
    const uint32_t i = lo + 2 * e;
    a.x[i] = xv.x;
    a.y[i] = yv.x;
    a.w[i] = wv.x;
    a.pv[i] = pv.x;
    if (2 * e + 1 < nf) {
      a.x[i + 1] = xv.y;
      a.y[i + 1] = yv.y;
      a.w[i + 1] = wv.y;
      a.pv[i + 1] = pv.y;
    }
  }

  // ---- final barrier (every block's partials are out), then fold the
  // barycentre partials step by step
  __syncthreads();
  if (tid == nthreads - 32 && multi) {  // the lane that wrote the partials
    grid_arrive(a);
    if (!grid_wait(a, T + 1)) s_abort = 1;
  }
  __syncthreads();
  if (s_abort) return;
  const int nw_all = nthreads >> 5;
  __shared__ Sum f_w[32], f_x[32], f_y[32];
  for (uint32_t s = blockIdx.x; s < T; s += gridDim.x) {
    Sum fw = Sum(0), fx = Sum(0), fy = Sum(0);
    for (uint32_t b = tid; b < gridDim.x; b += nthreads) {
      const double* p = a.sums + (static_cast<uint64_t>(s) * gridDim.x + b) * 3;
      fw = sum2(fw, raw_to_sum<ACC>(__ldcg(p + 0)));
      fx = sum2(fx, raw_to_sum<ACC>(__ldcg(p + 1)));
      fy = sum2(fy, raw_to_sum<ACC>(__ldcg(p + 2)));
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
      fw = lane < nw_all ? f_w[lane] : Sum(0);
      fx = lane < nw_all ? f_x[lane] : Sum(0);
      fy = lane < nw_all ? f_y[lane] : Sum(0);
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

template <int ACC>
const void* kernel_ptr(bool wswim) {
  if (wswim) return reinterpret_cast<const void*>(&resident_kernel<ACC, true>);
  return reinterpret_cast<const void*>(&resident_kernel<ACC, false>);
}

const void* pick(int acc, bool wswim) {
  switch (acc) {
    case kAccPlain32: return kernel_ptr<kAccPlain32>(wswim);
    case kAccKahan32: return kernel_ptr<kAccKahan32>(wswim);
    case kAccF64: return kernel_ptr<kAccF64>(wswim);
    default: return nullptr;
  }
}

}  // namespace

// Largest block (fish threads) for `fpt`: every variant runs up to
// kResThreads fish threads.
int resident_max_block(int fpt) {
  if (fpt != 4 && fpt != 8 && fpt != 12 && fpt != 16) return 0;
  return kResThreads;
}

// Largest slice of a block of `block` fish threads holding at most `fpt`
// fish per thread, within the shared memory.
uint64_t resident_max_slice(int fpt, int block) {
  const uint64_t by_threads = static_cast<uint64_t>(fpt) * block;
  return by_threads < kResMaxSlice ? by_threads : kResMaxSlice;
}

size_t resident_smem_bytes(uint64_t slice) { return kResSmemPerFish * slice; }

// The kernel copy for a launch: the weight-scaled swim's copy also serves
// the default swim when its width's scaled form is not exact (a step below
// 2^-103 but not 0), for the default copy takes that form without checking.
static bool wswim_copy(int swim_mode, double step) {
  return swim_mode != 0 || !swim_scale_exact(static_cast<float>(step));
}

int resident_blocks_per_sm(int fpt, int acc, int block, int swim_mode, double step) {
  const void* fn = pick(acc, wswim_copy(swim_mode, step));
  if (!fn || block < 32 || block > resident_max_block(fpt)) return 0;
  // the attribute is per kernel, shared by every handle: always the largest
  // slice, so no handle lowers it under another
  if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           static_cast<int>(resident_smem_bytes(kResMaxSlice))) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  int nb = 0;
  const size_t smem = resident_smem_bytes(resident_max_slice(fpt, block));
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, fn, block + 32, smem) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return nb;
}

cudaError_t launch_resident(const ResidentLaunch& L, cudaStream_t s) {
  const void* fn = pick(L.acc, wswim_copy(L.swim_mode, L.step));
  if (!fn || L.grid < 1 || L.block < 32 || L.block % 32 || L.block > resident_max_block(L.fpt) ||
      L.slice < 2 || L.slice % 2 || L.slice > resident_max_slice(L.fpt, L.block) ||
      static_cast<uint64_t>(L.grid) * L.slice < L.n)
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
  cfg.blockDim = dim3(L.block + 32);  // the fish threads and the synchronisation warp
  cfg.dynamicSmemBytes = resident_smem_bytes(L.slice);
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = L.grid > 1 ? 1 : 0;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelExC(&cfg, fn, args);
}

}  // namespace fsb
