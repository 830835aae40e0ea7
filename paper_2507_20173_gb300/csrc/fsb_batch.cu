// fsb_batch.cu -- many independent fish schools of uneven size in one
// persistent launch.
//
// Thread-block clusters of C blocks pop schools from work queues sorted by
// size, largest first (longest-processing-time order), through atomic
// counters over a ragged offset table, and run all n_steps of a school on
// chip: each thread keeps FPT fish (x, y, weight, currentObjective,
// prevObjective) in registers.  A school goes to the queue of the smallest
// cluster that holds it (8, 4, 2 or 1 blocks):
//   - a cluster first takes schools from the queue of its own size, then
//     from the queues of smaller multi-block clusters; the per-step maxima
//     and barycentre partials of its C blocks meet in rank 0's shared memory
//     through distributed shared memory, with one cluster barrier per step
//     (partials double-buffered by step parity);
//   - when those run out, every block pops single-block schools on its own
//     and reduces with __syncthreads only.
// The per-step order within a school is the paper's (Sec. 2.1.2 swim,
// Sec. 2.1.1 objective, delta, the Sec. 2.3.2 max, feeding, barycentre).
// School k uses key seeds[k] and school id k, so it reproduces the
// single-school path bit for bit.  Waits are hardware barriers on uniform
// control flow (every decision a cluster takes is broadcast from rank 0),
// so no block can be left waiting for another.
//
// One persistent launch per cluster size in use runs concurrently with the
// others, each on a share of the SMs in proportion to its queue's fish (a
// launch of single blocks takes the SMs the clusters leave over); all of
// them share the queues, so the launches that finish first help the rest.
#include <cstdint>

#include <cooperative_groups.h>

#include "fsb_device.cuh"
#include "fsb_internal.h"
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
  const uint32_t* __restrict__ order;              // queues 0..3, each largest first
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

// Per-block partial of one step exchanged across the cluster (the sums in
// the accumulation mode's partial type, so the exchange stays in binary32
// in the binary32 modes).
template <typename Part>
struct ClusterPartial {
  uint32_t max_bits, e_key;
  Part sum_w, sum_wx, sum_wy;
};

constexpr int kBatchThreads = 512;
constexpr int kBatchFpt = 16;
constexpr int kMaxCluster = 8;

template <int ACC>
struct BlockReduce {
  using Part = typename SumAcc<ACC>::Part;
  uint32_t s_max[32], s_ekey[32];
  Part s_w[32], s_x[32], s_y[32];
};

// Block reduction of (max, key, three sums); the result is valid in thread 0.
template <int ACC>
__device__ __forceinline__ void block_reduce(BlockReduce<ACC>& R, uint32_t& m, uint32_t& e,
                                             typename SumAcc<ACC>::Part& sw,
                                             typename SumAcc<ACC>::Part& sx,
                                             typename SumAcc<ACC>::Part& sy) {
  using Part = typename SumAcc<ACC>::Part;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  constexpr int nw = kBatchThreads / 32;
  m = warp_max(m);
  e = warp_max(e);
  sw = warp_tree(sw);
  sx = warp_tree(sx);
  sy = warp_tree(sy);
  __syncthreads();  // previous use of R is finished
  if (lane == 0) {
    R.s_max[warp] = m;
    R.s_ekey[warp] = e;
    R.s_w[warp] = sw;
    R.s_x[warp] = sx;
    R.s_y[warp] = sy;
  }
  __syncthreads();
  if (warp == 0) {
    m = lane < nw ? R.s_max[lane] : 0u;
    e = lane < nw ? R.s_ekey[lane] : 0u;
    sw = lane < nw ? R.s_w[lane] : part_zero<Part>();
    sx = lane < nw ? R.s_x[lane] : part_zero<Part>();
    sy = lane < nw ? R.s_y[lane] : part_zero<Part>();
    m = warp_max(m);
    e = warp_max(e);
    sw = warp_merge(sw);
    sx = warp_merge(sx);
    sy = warp_merge(sy);
  }
}

// Runs one school on `nb` blocks (this block is rank `rank`): load or
// initialise, all steps, write back.  For nb > 1 the caller's cluster must
// contain exactly nb blocks that all call this with the same school.
template <int ACC, bool VAR>
__device__ __forceinline__ void run_school(const BatchArgs& a, uint32_t k, int rank, int nb,
                                           BlockReduce<ACC>& R,
                                           ClusterPartial<typename SumAcc<ACC>::Part> (*xchg)[kMaxCluster],
                                           uint32_t* s_M,
                                           uint32_t* s_E, float (*spv)[kBatchThreads]) {
  using Acc = SumAcc<ACC>;
  using Part = typename Acc::Part;
  const int tid = threadIdx.x;
  const uint64_t s_lo = a.offsets[k];
  // in-school fish indices fit 32 bits (schools hold at most C * 8192 fish)
  const uint32_t n = static_cast<uint32_t>(a.offsets[k + 1] - s_lo);
  // an even slice keeps each fish pair (one swim block) in one thread
  const uint32_t slice = ((n + nb - 1) / nb + 1) & ~1u;
  const uint32_t lo = static_cast<uint32_t>(rank) * slice;
  const uint32_t hi = lo + slice < n ? lo + slice : n;
  // slot q of this thread is fish lo + 2 (tid + (q / 2) kBatchThreads) + q % 2
  // (in-school index); slots q < nq are in the school
  auto fish = [&](int q) -> uint32_t {
    return lo + 2u * (static_cast<uint32_t>(tid) + static_cast<uint32_t>(q >> 1) * kBatchThreads) +
           static_cast<uint32_t>(q & 1);
  };
  int nq = 0;
#pragma unroll
  for (int q = 0; q < kBatchFpt; ++q)
    if (fish(q) < hi) nq = q + 1;
  const Key key{static_cast<uint32_t>(a.seeds[k]), static_cast<uint32_t>(a.seeds[k] >> 32)};
  const uint32_t school = k;
  const Physics<float> ph = kernel_physics<VAR>(a.ph);
  cg::cluster_group cluster = cg::this_cluster();

  // prevObjective of each fish waits in shared memory (spv[q][tid]); the
  // other four fields stay in registers
  float x[kBatchFpt], y[kBatchFpt], w[kBatchFpt], f[kBatchFpt];
#pragma unroll
  for (int q = 0; q < kBatchFpt; ++q) {
    const uint32_t i = fish(q);  // index in school
    if (q < nq) {
      if (a.init) {
        init_fish(key, school, i, a.weight_mode, ph, x[q], y[q], w[q]);
      } else {
        x[q] = a.x[s_lo + i];
        y[q] = a.y[s_lo + i];
        w[q] = a.w[s_lo + i];
      }
      f[q] = objective(x[q], y[q]);
    } else {
      x[q] = y[q] = w[q] = f[q] = 0.f;
    }
  }

  // Each step: swim -> local maxima (+ the previous step's sums) -> one
  // exchange -> eat.  The exchange of step u carries the sums of step u - 1;
  // one extra exchange after the last step carries the last sums.
  Part sw = part_zero<Part>(), sx = part_zero<Part>(), sy = part_zero<Part>();
  for (uint32_t u = 1; u <= a.n_steps + 1; ++u) {
    const bool swim_step = u <= a.n_steps;
    uint32_t mb = 0, ek = 0;
    if (swim_step) {
      const uint32_t t = static_cast<uint32_t>(*a.base_step_ptr + u);
      Words4 r{};
#pragma unroll
      for (int q = 0; q < kBatchFpt; ++q) {
        if (q < nq) {
          const float old = f[q];
          spv[q][tid] = old;
          if ((q & 1) == 0) r = pair_draw(key, school, fish(q) >> 1, t);
          swim(x[q], y[q], r.v[2 * (q & 1)], r.v[2 * (q & 1) + 1], swim_width(ph, w[q]), ph);
          f[q] = objective(x[q], y[q]);
          const uint32_t mm = abs_bits(__fsub_rn(f[q], old));
          const uint32_t ee = order_key(__fsub_rn(old, f[q]));
          mb = mm > mb ? mm : mb;
          ek = ee > ek ? ee : ek;
        }
      }
    }
    block_reduce<ACC>(R, mb, ek, sw, sx, sy);
    if (nb == 1) {
      if (tid == 0) {
        *s_M = mb;
        *s_E = ek;
        if (u > 1) {
          fsb_step_stats* st = a.stats + static_cast<uint64_t>(k) * a.n_steps + (u - 2);
          st->sum_w = to_double(sw);
          st->sum_wx = to_double(sx);
          st->sum_wy = to_double(sy);
        }
      }
      __syncthreads();
    } else {
      // every block writes its partial into rank 0's slot for this parity
      if (tid == 0) {
        ClusterPartial<Part>* dst = cluster.map_shared_rank(&xchg[u & 1][rank], 0);
        ClusterPartial<Part> p;
        p.max_bits = mb;
        p.e_key = ek;
        p.sum_w = sw;
        p.sum_wx = sx;
        p.sum_wy = sy;
        *dst = p;
      }
      cluster.sync();
      // fold the nb partials in rank order (identical in every block)
      if (tid == 0) {
        const ClusterPartial<Part>* src = cluster.map_shared_rank(&xchg[u & 1][0], 0);
        uint32_t m = 0, e = 0;
        Part fw = part_zero<Part>(), fx = part_zero<Part>(), fy = part_zero<Part>();
        for (int r = 0; r < nb; ++r) {
          const ClusterPartial<Part> p = src[r];
          m = p.max_bits > m ? p.max_bits : m;
          e = p.e_key > e ? p.e_key : e;
          fw = merge(fw, p.sum_w);
          fx = merge(fx, p.sum_wx);
          fy = merge(fy, p.sum_wy);
        }
        *s_M = m;
        *s_E = e;
        if (rank == 0 && u > 1) {
          fsb_step_stats* st = a.stats + static_cast<uint64_t>(k) * a.n_steps + (u - 2);
          st->sum_w = to_double(fw);
          st->sum_wx = to_double(fx);
          st->sum_wy = to_double(fy);
        }
      }
      __syncthreads();
    }
    if (!swim_step) break;
    const float M = __uint_as_float(*s_M);
    // feeding normaliser: M_u, or the paper's eat() value E_u
    const float N = ph.feed_mode ? key_to_value(*s_E, 0.f) : M;
    if (rank == 0 && tid == 0) {
      fsb_step_stats* st = a.stats + static_cast<uint64_t>(k) * a.n_steps + (u - 1);
      st->max_abs_delta = static_cast<double>(M);
      st->eat_max_diff = static_cast<double>(key_to_value(*s_E, 0.f));
    }
    // eat of step u and its barycentre partials
    Acc acc;
#pragma unroll
    for (int q = 0; q < kBatchFpt; ++q) {
      if (q < nq) {
        if (N > 0.f)
          w[q] = eat(w[q],
                     ph.feed_mode ? __fsub_rn(spv[q][tid], f[q]) : __fsub_rn(f[q], spv[q][tid]),
                     N, ph);
        acc.add(w[q], x[q], y[q]);
      }
    }
    sw = acc.pw();
    sx = acc.px();
    sy = acc.py();
  }
  if (nb > 1) cluster.sync();  // rank 0's slots are free again for the next school

#pragma unroll
  for (int q = 0; q < kBatchFpt; ++q) {
    const uint32_t i = fish(q);
    if (q < nq) {
      a.x[s_lo + i] = x[q];
      a.y[s_lo + i] = y[q];
      a.w[s_lo + i] = w[q];
      a.pv[s_lo + i] = a.n_steps ? spv[q][tid] : f[q];
    }
  }
}

template <int CLUSTER, int ACC, bool VAR>
__global__ void __launch_bounds__(kBatchThreads, 1) batch_kernel(BatchArgs a) {
  __shared__ BlockReduce<ACC> R;
  __shared__ ClusterPartial<typename SumAcc<ACC>::Part> xchg[2][kMaxCluster];
  __shared__ float spv[kBatchFpt][kBatchThreads];
  __shared__ uint32_t s_M, s_E, s_pick;
  cg::cluster_group cluster = cg::this_cluster();
  const int rank = static_cast<int>(cluster.block_rank());

  // Phase 1 (whole cluster per school) through the multi-block queues from
  // this launch's own on, then phase 2 (each block on its own) through the
  // single-block queue.  The queue index is uniform across the cluster
  // (every pick is broadcast from rank 0).  One call site keeps one inlined
  // copy of the per-school loop.
  constexpr int kSingle = kBatchQueues - 1;
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
    run_school<ACC, VAR>(a, a.order[a.queue_lo[t] + idx], whole_cluster ? rank : 0,
                         whole_cluster ? CLUSTER : 1, R, xchg, &s_M, &s_E, spv);
  }
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

// The variant kernels (var) share the default ones' block, register bound
// and shared memory, hence their occupancy.
const void* pick(int cluster, int acc, bool var = false) {
  switch (cluster) {
    case 1: return pick_acc<1>(acc, var);
    case 2: return pick_acc<2>(acc, var);
    case 4: return pick_acc<4>(acc, var);
    case 8: return pick_acc<8>(acc, var);
    default: return nullptr;
  }
}

cudaLaunchConfig_t make_config(int cluster, int grid, cudaStream_t s, cudaLaunchAttribute* attr) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(kBatchThreads);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = s;
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = cluster;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cfg;
}

__global__ void bump_step_kernel(unsigned long long* base_step, uint32_t n) { *base_step += n; }

}  // namespace

cudaError_t launch_bump_step(unsigned long long* base_step, uint32_t n, cudaStream_t s) {
  bump_step_kernel<<<1, 1, 0, s>>>(base_step, n);
  return cudaGetLastError();
}

uint64_t batch_block_capacity() { return static_cast<uint64_t>(kBatchThreads) * kBatchFpt; }
int batch_threads() { return kBatchThreads; }

// Clusters of `cluster` blocks that can be resident at once (0: cannot run).
int batch_max_clusters(int cluster, int acc) {
  const void* fn = pick(cluster, acc);
  if (!fn) return 0;
  cudaLaunchAttribute attr[1];
  cudaLaunchConfig_t cfg = make_config(cluster, cluster, nullptr, attr);
  int n = 0;
  if (cudaOccupancyMaxActiveClusters(&n, fn, &cfg) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return n;
}

cudaError_t launch_batch(const BatchLaunch& L, cudaStream_t s, const cudaStream_t* side,
                         cudaEvent_t fork, const cudaEvent_t* join) {
  const bool var = L.swim_mode != 0 || L.feed_mode != 0;
  if (L.n_launches < 1 || L.n_launches > kBatchMaxLaunches) return cudaErrorInvalidValue;
  if (L.n_launches > 1 && (!side || !fork || !join)) return cudaErrorInvalidValue;
  const void* fn[kBatchMaxLaunches];
  for (int i = 0; i < L.n_launches; ++i) {
    fn[i] = pick(L.cluster[i], L.acc, var);
    if (!fn[i] || L.blocks[i] < L.cluster[i] || L.blocks[i] % L.cluster[i])
      return cudaErrorInvalidValue;
  }
  BatchArgs a;
  a.x = static_cast<float*>(L.x);
  a.y = static_cast<float*>(L.y);
  a.w = static_cast<float*>(L.w);
  a.pv = static_cast<float*>(L.pv);
  a.offsets = L.offsets;
  a.seeds = L.seeds;
  a.order = L.order;
  for (int t = 0; t <= kBatchQueues; ++t) a.queue_lo[t] = L.queue_lo[t];
  a.n_schools = L.n_schools;
  a.ph.pond_half = static_cast<float>(L.pond_half);
  a.ph.step = static_cast<float>(L.step);
  a.ph.w0 = static_cast<float>(L.w0);
  a.ph.w_min = static_cast<float>(L.w_min);
  a.ph.w_max = static_cast<float>(L.w_max);
  a.ph.swim_mode = L.swim_mode;
  a.ph.feed_mode = L.feed_mode;
  a.init = L.init;
  a.weight_mode = L.weight_mode;
  a.base_step_ptr = L.base_step;
  a.n_steps = L.n_steps;
  a.bctl = L.bctl;
  a.stats = L.stats;
  cudaError_t e = cudaMemsetAsync(L.bctl, 0, sizeof(BatchCtl), s);
  if (e != cudaSuccess) return e;
  if (L.n_launches > 1) {
    if ((e = cudaEventRecord(fork, s)) != cudaSuccess) return e;
    for (int i = 1; i < L.n_launches; ++i)
      if ((e = cudaStreamWaitEvent(side[i - 1], fork, 0)) != cudaSuccess) return e;
  }
  // largest clusters first, so they are placed before the smaller launches
  for (int i = 0; i < L.n_launches; ++i) {
    BatchArgs ai = a;
    ai.first_queue = batch_queue_of(L.cluster[i]);
    void* args[] = {&ai};
    cudaLaunchAttribute attr[1];
    cudaLaunchConfig_t cfg = make_config(L.cluster[i], L.blocks[i], i == 0 ? s : side[i - 1], attr);
    if ((e = cudaLaunchKernelExC(&cfg, fn[i], args)) != cudaSuccess) return e;
  }
  for (int i = 1; i < L.n_launches; ++i) {
    if ((e = cudaEventRecord(join[i - 1], side[i - 1])) != cudaSuccess) return e;
    if ((e = cudaStreamWaitEvent(s, join[i - 1], 0)) != cudaSuccess) return e;
  }
  return cudaSuccess;
}

}  // namespace fsb
