// fsb_batch_kernel.cuh -- the batched-schools kernel (fsb_batch.cu has the
// design notes and the host side).  Included by the translation units that
// instantiate it for the cluster sizes 1-4 (fsb_batch.cu) and 5-8
// (fsb_batch_wide.cu), so the two halves compile in parallel.
#pragma once

#include <cstdint>
#include <cstring>

#include <cooperative_groups.h>

#include "fsb_check.cuh"
#include "fsb_device.cuh"
#include "fsb_internal.h"
#include "fsb_onchip.cuh"
#include "fsb_reduce.cuh"

namespace fsb {
namespace {

namespace cg = cooperative_groups;

struct BatchArgs {
  float* __restrict__ x;
  float* __restrict__ y;
  float* __restrict__ w;
  float* __restrict__ pv;
  const unsigned long long* __restrict__ offsets;  // n_schools + 1
  const unsigned long long* __restrict__ seeds;    // n_schools
  const uint32_t* __restrict__ order;              // queues 0..7, each largest first
  uint32_t queue_lo[kBatchQueues + 1];             // queue t: order[queue_lo[t] .. queue_lo[t+1])
  int first_queue;                                 // whole-cluster queue this launch starts at
  uint32_t n_schools;
  Physics<float> ph;
  int init;                                        // initialise each school before stepping
  int weight_mode;
  const unsigned long long* base_step_ptr;
  uint32_t n_steps;
  BatchCtl* bctl;
  fsb_step_stats* stats;                           // n_schools * n_steps, school-major
};

// Barycentre partials of one step: a warp's, a block's.
template <typename Part>
struct Part3 {
  Part w, x, y;
};

#ifndef FSB_BATCH_FISH_THREADS
#define FSB_BATCH_FISH_THREADS 512
#endif
constexpr int kBatchThreads = FSB_BATCH_FISH_THREADS;  // fish threads
static_assert(kBatchThreads % 32 == 0 && kBatchThreads <= 992, "fish threads: whole warps, <= 31");
constexpr int kBatchWarps = kBatchThreads / 32;
constexpr int kBlockThreads = kBatchThreads + 32;  // and one helper warp
// Fish one block holds: 11 pairs per fish thread, 20 B each (220 KB of the
// 227 KB of shared memory a block may have).  Measured on GB300 against
// 8192 (8 pairs per thread): 4.7% faster per SM on single blocks, 6% on
// clusters (fewer and longer passes per fish, narrower clusters), 6.6% on
// the log-uniform ensemble.
constexpr int kBlockFish = 11264;
#ifndef FSB_BATCH_PAIRS_PER_ITER
#define FSB_BATCH_PAIRS_PER_ITER 1
#endif
// fish pairs per thread per iteration of a pass (a build-time constant)
constexpr int kBatchPairsPerIter = FSB_BATCH_PAIRS_PER_ITER;
constexpr int kBlockPairs = kBlockFish / 2;
constexpr int kMaxCluster = 8;
// Packed schools: with 16 fish warps, a block runs schools of up to 8, 4, 2
// or 1 times kTeamFish (704) fish on teams of 8, 4, 2 or 1 warps, each team
// on its own share of the block's fish and its own barrier.
constexpr bool kPacked = kBatchWarps == 16;
constexpr int kTeamFish = kPacked ? kBlockFish / kBatchWarps : 0;
constexpr int kTeamPairs = kTeamFish / 2;
static_assert(!kPacked || (kBatchWarps >> kBatchPackLevels) == 1,
              "packed teams of 8, 4, 2 and 1 warps");
// The block's fish in shared memory: five arrays of kBlockPairs float2
// (fish 2p and 2p + 1 of the block's slice share element p).
constexpr size_t kStateSmem = 5 * sizeof(float2) * kBlockPairs;

// Shared-memory exchange of one block.  The step maxima go into the slots
// of the school's team by atomics (row 0 of rank 0 for a school on whole
// blocks, the row of its first warp for a packed team; three slots rotate
// by step: a slot is read after the barrier that ends its step's swim, and
// zeroed three steps ahead of its next use).  Barycentre partials are
// double-buffered by step parity: the warps' partials of step p are folded
// into the team's after the barrier that ends step p's eat, and, on a
// cluster, the blocks' partials in rank 0 one barrier later.
template <int ACC>
struct BatchShared {
  using Part = typename SumAcc<ACC>::Part;
  uint32_t slot_max[kBatchWarps][3], slot_ekey[kBatchWarps][3];
  uint32_t pick[kBatchWarps];  // a packed team's pick, by its first warp
  Part3<Part> warp_part[2][kBatchWarps];
  Part3<Part> block_part[2][kMaxCluster];
};

// The threads that run one school in a block.  A whole block (WHOLE, a
// compile-time choice, so that its pass keeps its constants): its fish
// warps and the helper warp, synchronised block- or cluster-wide.  A
// packed team: `warps` fish warps from warp0, synchronised by the named
// barrier `bar` (1 .. 14; 0 for a team of one warp, which uses
// __syncwarp), with no helper warp: the team's first warp does the helper's
// work after each barrier.
struct Team {
  int warp0, warps, bar;
};

template <bool WHOLE>
__device__ __forceinline__ void team_sync(const Team& t, cg::cluster_group& cluster, int nb) {
  if (WHOLE) {
    if (nb > 1)
      cluster.sync();
    else
      __syncthreads();
  } else if (t.bar == 0) {
    __syncwarp();
  } else {
    asm volatile("bar.sync %0, %1;" ::"r"(t.bar), "r"(t.warps * 32) : "memory");
  }
}

// Fold of WARPS warps' partials by one warp, a fixed xor tree; the result
// is valid in every lane.  A power-of-two count folds over WARPS lanes
// (lanes beyond them repeat them); any other count over 32 lanes, those
// beyond the warps holding zeros.  The count is a compile-time constant:
// the fold is on the helper's path between two barriers, and a run-time
// count measured several per cent slower for short passes.
template <int WARPS, typename Part>
__device__ __forceinline__ Part3<Part> fold_warps(const Part3<Part>* wp) {
  static_assert(WARPS >= 1 && WARPS <= 31, "at most 31 fish warps");
  constexpr int kLanes = (WARPS & (WARPS - 1)) == 0 ? WARPS : 32;
  const int lane = threadIdx.x & 31;
  Part3<Part> r;
  if (kLanes == WARPS) {
    r = wp[lane & (WARPS - 1)];
  } else if (lane < WARPS) {
    r = wp[lane];
  } else {
    r.w = r.x = r.y = part_zero<Part>();
  }
#pragma unroll
  for (int off = kLanes / 2; off > 0; off >>= 1) {
    r.w = merge(r.w, shfl_xor(r.w, off));
    r.x = merge(r.x, shfl_xor(r.x, off));
    r.y = merge(r.y, shfl_xor(r.y, off));
  }
  return r;
}

// The same for a packed team of 8, 4, 2 or 1 warps.
template <typename Part>
__device__ __forceinline__ Part3<Part> fold_team(const Part3<Part>* wp, int warps) {
  switch (warps) {
    case 8: return fold_warps<8>(wp);
    case 4: return fold_warps<4>(wp);
    case 2: return fold_warps<2>(wp);
    default: return fold_warps<1>(wp);
  }
}

// A step's barycentre sums go out as raw partials (raw_sum) and the host
// converts them after the copy-out (batch_finish_stats), which keeps
// binary64 arithmetic, slow on this GPU, off the per-step critical path.
template <typename Part>
__device__ __forceinline__ void put_sums(fsb_step_stats* st, Part w, Part x, Part y) {
  st->sum_w = raw_sum(w);
  st->sum_wx = raw_sum(x);
  st->sum_wy = raw_sum(y);
}

// Runs one school on `nb` blocks (this block is rank `rank`), or on a
// packed team of warps (nb = 1): load or initialise, all steps, write back.
// For nb > 1 the caller's cluster must contain exactly nb blocks that all
// call this with the same school, and the team's slots (rank 0's) must be
// zero (they are again on return).  B is the team's share of the block's
// fish.
//
// Pass p = 0 .. T over the team's fish pairs (the fish warps): the eat of
// step p with normaliser N_p and its barycentre terms (p >= 1), then the
// swim of step p + 1 with its objective and maxima (p < T).  One barrier
// follows each pass (a cluster barrier for nb > 1):
//   before it: each fish warp's maxima of step p + 1 into the team's slots
//              (atomics) and its barycentre partial of step p;
//   after it:  the fish warps read M_{p+1} and E_{p+1} and start the next
//              pass, while the block's helper warp (a packed team's first
//              warp, before its next pass) zeroes the slots of step p + 3
//              (rank 0), folds the team's partial of step p (nb = 1: the
//              step's sums; else into rank 0's block_part), folds the
//              blocks' partials of step p - 1 (rank 0) and writes the step's
//              maxima -- work that would otherwise hold one fish warp back
//              at every barrier of a whole block.
template <int ACC, bool VAR, bool WHOLE>
__device__ __forceinline__ void run_school(const BatchArgs& a, uint32_t k, int rank, int nb,
                                           BatchShared<ACC>& S, const PairState& B,
                                           const Team& team) {
  using Acc = OnchipAcc<ACC>;
  using Part = typename Acc::Part;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const bool helper = WHOLE && warp == kBatchWarps;
  const bool folds = WHOLE ? helper : warp == team.warp0;
  // this thread's rank in the team, the team's fish threads, and the
  // threads that load and store the fish (a whole block's helper too)
  const uint32_t first = WHOLE ? static_cast<uint32_t>(tid)
                               : static_cast<uint32_t>(tid - team.warp0 * 32);
  const uint32_t fish_threads =
      WHOLE ? static_cast<uint32_t>(kBatchThreads) : static_cast<uint32_t>(team.warps) * 32u;
  const uint32_t io_threads = WHOLE ? static_cast<uint32_t>(kBlockThreads) : fish_threads;
  const uint32_t cap = WHOLE ? static_cast<uint32_t>(kBlockFish)
                             : static_cast<uint32_t>(team.warps) * kTeamFish;
  const uint64_t s_lo = a.offsets[k];
  // in-school fish indices fit 32 bits (schools hold at most C * kBlockFish fish)
  const uint32_t n = static_cast<uint32_t>(a.offsets[k + 1] - s_lo);
  // an even slice keeps each fish pair (one swim block) in one block
  const uint32_t slice = ((n + nb - 1) / nb + 1) & ~1u;
  const uint32_t lo = static_cast<uint32_t>(rank) * slice;
  const uint32_t hi = lo + slice < n ? lo + slice : n;
  // this block's fish (at most what the team holds: the plan gives a school
  // a cluster or a team that holds it) and pairs, the last possibly half
  const uint32_t nf0 = hi > lo ? hi - lo : 0u;
  const uint32_t nf = fsb_check(nf0 <= cap, &a.bctl->status, &a.bctl->site, 1u) ? nf0 : cap;
  const uint32_t np = (nf + 1) / 2;
  const uint32_t pair0 = lo / 2;                  // in-school pair index of element 0
  const Key key{static_cast<uint32_t>(a.seeds[k]), static_cast<uint32_t>(a.seeds[k] >> 32)};
  const uint32_t school = k;
  const Physics<float> ph = kernel_physics<VAR>(a.ph);
  cg::cluster_group cluster = cg::this_cluster();
  // rank 0's exchange (this block's own for nb = 1) and the team's slots
  BatchShared<ACC>* S0 = nb > 1 ? cluster.map_shared_rank(&S, 0) : &S;
  // the team's slots (formed at each use: fewer registers held over the passes)
  const int row = WHOLE ? 0 : team.warp0;
#define FSB_SLOT_MAX(i) (S0->slot_max[row][(i)])
#define FSB_SLOT_EKEY(i) (S0->slot_ekey[row][(i)])
  fsb_step_stats* const st = a.stats + static_cast<uint64_t>(k) * a.n_steps;
  const uint32_t T = a.n_steps;

  // load (or initialise) the slice; the second fish of a half pair is zero
  for (uint32_t e = first; e < np; e += io_threads) {
    float xv[2] = {0.f, 0.f}, yv[2] = {0.f, 0.f}, wv[2] = {0.f, 0.f}, fv[2] = {0.f, 0.f};
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const uint32_t i = lo + 2 * e + h;  // index in school
      if (2 * e + h < nf) {
        if (a.init) {
          init_fish(key, school, i, a.weight_mode, ph, xv[h], yv[h], wv[h]);
        } else {
          xv[h] = a.x[s_lo + i];
          yv[h] = a.y[s_lo + i];
          wv[h] = a.w[s_lo + i];
        }
        fv[h] = objective(xv[h], yv[h]);
      }
    }
    B.XYd[e] = make_float4(xv[0], xv[1], yv[0], yv[1]);
    B.W[e] = make_float2(wv[0], wv[1]);
    B.F[e] = make_float2(fv[0], fv[1]);
  }
  team_sync<WHOLE>(team, cluster, 1);  // the passes take the pairs in another thread order

  const uint32_t last = T + (nb > 1 ? 1u : 0u);  // a cluster's last fold needs one more barrier
  const uint64_t t0 = *a.base_step_ptr;
  const float scaled = exact_scaled_width(ph.step);
  float N = 0.f;  // feeding normaliser of the pass's eat
  for (uint32_t p = 0; p <= last; ++p) {
    const bool do_eat = p >= 1 && p <= T;
    const bool do_swim = p < T;
    if (!helper) {
      PassCtx c{key, school, pair0, static_cast<uint32_t>(t0 + p + 1), N, scaled};
      uint32_t mb = 0, ek = 0;
      Acc acc;
      if (p == 0 && T > 1)
        block_pass_from<false, true, false, false, false, kBatchPairsPerIter, !VAR>(
            B, np, nf, c, ph, acc, mb, ek, first, fish_threads);
      else if (p == 0 && T == 1)
        block_pass_from<false, true, true, false, false, kBatchPairsPerIter, !VAR>(
            B, np, nf, c, ph, acc, mb, ek, first, fish_threads);
      else if (p + 1 < T)
        block_pass_from<true, true, false, false, false, kBatchPairsPerIter, !VAR>(
            B, np, nf, c, ph, acc, mb, ek, first, fish_threads);
      else if (p + 1 == T)
        block_pass_from<true, true, true, false, false, kBatchPairsPerIter, !VAR>(
            B, np, nf, c, ph, acc, mb, ek, first, fish_threads);
      else if (p == T)
        block_pass_from<true, false, false, true, false, kBatchPairsPerIter, !VAR>(
            B, np, nf, c, ph, acc, mb, ek, first, fish_threads);
      if (do_swim) {
        mb = warp_max(mb);
        ek = warp_max(ek);
        if (lane == 0) {
          atomicMax(&FSB_SLOT_MAX((p + 1) % 3), mb);
          atomicMax(&FSB_SLOT_EKEY((p + 1) % 3), ek);
        }
      }
      if (do_eat) {
        warp_partials(&S.warp_part[p & 1][warp], acc.pw(), acc.px(), acc.py());
      }
    }
    team_sync<WHOLE>(team, cluster, nb);
    if (folds) {
      if (rank == 0 && lane == 0) {
        FSB_SLOT_MAX(p % 3) = 0u;
        FSB_SLOT_EKEY(p % 3) = 0u;
      }
      if (do_eat) {
        const Part3<Part> bp = WHOLE ? fold_warps<kBatchWarps>(S.warp_part[p & 1])
                                     : fold_team(S.warp_part[p & 1] + team.warp0, team.warps);
        if (lane == 0) {
          if (nb == 1)
            put_sums(st + (p - 1), bp.w, bp.x, bp.y);
          else
            S0->block_part[p & 1][rank] = bp;
        }
      }
      // the blocks' partials of step p - 1, in rank order
      if (nb > 1 && rank == 0 && lane == 0 && p >= 2) {
        const Part3<Part>* src = S.block_part[(p - 1) & 1];
        Part fw = part_zero<Part>(), fx = part_zero<Part>(), fy = part_zero<Part>();
        for (int r = 0; r < nb; ++r) {
          fw = merge(fw, src[r].w);
          fx = merge(fx, src[r].x);
          fy = merge(fy, src[r].y);
        }
        put_sums(st + (p - 2), fw, fx, fy);
      }
      if (do_swim && rank == 0 && lane == 0) {
        st[p].max_abs_delta = static_cast<double>(__uint_as_float(FSB_SLOT_MAX((p + 1) % 3)));
        st[p].eat_max_diff = static_cast<double>(key_to_value(FSB_SLOT_EKEY((p + 1) % 3), 0.f));
      }
    }
    if (!helper && do_swim) {
      // feeding normaliser of the next pass: M, or the paper's eat() value E
      N = ph.feed_mode ? key_to_value(FSB_SLOT_EKEY((p + 1) % 3), 0.f)
                       : __uint_as_float(FSB_SLOT_MAX((p + 1) % 3));
    }
  }
#undef FSB_SLOT_MAX
#undef FSB_SLOT_EKEY
  // rank 0 has read every block's partials, and its slots are zero, before
  // any block leaves for the next school
  if (nb > 1) cluster.sync();

  for (uint32_t e = first; e < np; e += io_threads) {
    const float4 p = B.XYs[e];
    const float2 xv = make_float2(p.x, p.y), yv = make_float2(p.z, p.w), wv = B.W[e];
    const float2 pv = T ? B.De[e] : B.F[e];
    const uint64_t g = s_lo + lo + 2 * e;
    a.x[g] = xv.x;
    a.y[g] = yv.x;
    a.w[g] = wv.x;
    a.pv[g] = pv.x;
    if (2 * e + 1 < nf) {
      a.x[g + 1] = xv.y;
      a.y[g + 1] = yv.y;
      a.w[g + 1] = wv.y;
      a.pv[g + 1] = pv.y;
    }
  }
  team_sync<WHOLE>(team, cluster, 1);  // the team's shared state is free for the next school
}

// Phase 3 of the batch kernel, for the block's fish warps (the helper warp
// is done: no block-wide barrier follows).  They split into two teams of
// 8, each popping schools of up to 8 * kTeamFish fish; a team whose queue
// is empty splits into two teams of half its warps for the next queue,
// down to single warps.  Team g of w warps owns warps g * w .. g * w + w - 1,
// their share of the block's fish, and named barrier 16 / w - 1 + g.  Not
// inlined, so that the registers of its own copy of the per-school loop do
// not weigh on the whole-block loop.
template <int ACC, bool VAR>
__device__ __noinline__ void run_packed(const BatchArgs& a, BatchShared<ACC>& S,
                                        float2* state_smem) {
  float4* const XY = reinterpret_cast<float4*>(state_smem);
  float2* const D = state_smem + 4 * kBlockPairs;
  cg::cluster_group cluster = cg::this_cluster();
  const int warp = threadIdx.x >> 5;
  for (int level = 0; level < kBatchPackLevels; ++level) {
    const int w = (kBatchWarps / 2) >> level;
    const int g = warp / w;
    const Team team{g * w, w, w == 1 ? 0 : kBatchWarps / w - 1 + g};
    const uint32_t base = static_cast<uint32_t>(team.warp0) * kTeamPairs;
    const PairState Bt = pair_state(XY + base, D + base, XY + base, D + base,
                                    state_smem + 3 * kBlockPairs + base,
                                    state_smem + 2 * kBlockPairs + base);
    const int q = kBatchPackQueue0 + level;
    for (;;) {
      if (threadIdx.x == team.warp0 * 32) S.pick[team.warp0] = atomicAdd(&a.bctl->next[q], 1u);
      team_sync<false>(team, cluster, 1);
      const uint32_t idx = S.pick[team.warp0];
      team_sync<false>(team, cluster, 1);  // every warp has read the pick
      if (idx >= a.queue_lo[q + 1] - a.queue_lo[q]) break;
      run_school<ACC, VAR, false>(a, a.order[a.queue_lo[q] + idx], 0, 1, S, Bt, team);
    }
  }
}

template <int CLUSTER, int ACC, bool VAR>
__global__ void __launch_bounds__(kBlockThreads, 1) batch_kernel(BatchArgs a) {
  __shared__ BatchShared<ACC> S;
  __shared__ uint32_t s_pick;
  extern __shared__ __align__(16) float2 state_smem[];
  float4* const XY = reinterpret_cast<float4*>(state_smem);  // two float2 arrays' room
  float2* const D = state_smem + 4 * kBlockPairs;
  const PairState B = pair_state(XY, D, XY, D, state_smem + 3 * kBlockPairs,
                                 state_smem + 2 * kBlockPairs);
  cg::cluster_group cluster = cg::this_cluster();
  const int rank = static_cast<int>(cluster.block_rank());
  for (int i = threadIdx.x; i < 3 * kBatchWarps; i += kBlockThreads) {
    // visible to the cluster after the first pick's barriers
    S.slot_max[i / 3][i % 3] = 0u;
    S.slot_ekey[i / 3][i % 3] = 0u;
  }

  // Phase 1 (whole cluster per school) through the multi-block queues from
  // this launch's own on, then phase 2 (each block on its own) through the
  // single-block queue, then phase 3 (each packed team on its own) through
  // the packed queues (run_packed).  The queue index is uniform across the
  // cluster (every pick is broadcast from rank 0).  One call site keeps one
  // inlined copy of the whole-block loop.
  constexpr int kSingle = kBatchSingleQueue;
  const Team whole{0, kBatchWarps, 0};
  int t = CLUSTER > 1 ? a.first_queue : kSingle;
  for (;;) {
    const bool whole_cluster = t < kSingle;
    uint32_t idx;
    if (whole_cluster) {
      if (rank == 0 && threadIdx.x == 0) s_pick = atomicAdd(&a.bctl->next[t], 1u);
      cluster.sync();
      idx = *cluster.map_shared_rank(&s_pick, 0);
      cluster.sync();  // every block has read rank 0's pick
    } else {
      if (threadIdx.x == 0) s_pick = atomicAdd(&a.bctl->next[kSingle], 1u);
      __syncthreads();
      idx = s_pick;
      __syncthreads();
    }
    if (idx >= a.queue_lo[t + 1] - a.queue_lo[t]) {
      if (t == kSingle) break;
      ++t;
      continue;
    }
    run_school<ACC, VAR, true>(a, a.order[a.queue_lo[t] + idx], whole_cluster ? rank : 0,
                               whole_cluster ? CLUSTER : 1, S, B, whole);
  }
  if (!kPacked || threadIdx.x >= kBatchThreads) return;  // the helper warp is done
  run_packed<ACC, VAR>(a, S, state_smem);
}

template <int CLUSTER, int ACC>
const void* kernel_ptr(bool var) {
  if (var) return reinterpret_cast<const void*>(&batch_kernel<CLUSTER, ACC, true>);
  return reinterpret_cast<const void*>(&batch_kernel<CLUSTER, ACC, false>);
}

template <int CLUSTER>
const void* pick_acc(int acc, bool var) {
  switch (acc) {
    case kAccPlain32: return kernel_ptr<CLUSTER, kAccPlain32>(var);
    case kAccKahan32: return kernel_ptr<CLUSTER, kAccKahan32>(var);
    case kAccF64: return kernel_ptr<CLUSTER, kAccF64>(var);
    default: return nullptr;
  }
}

}  // namespace
}  // namespace fsb
