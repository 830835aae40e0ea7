// fsb_batch.cu -- many independent fish schools of uneven size in one
// persistent launch.
//
// Thread-block clusters of C blocks pop schools from work queues sorted by
// size, largest first (longest-processing-time order), through atomic
// counters over a ragged offset table, and run all n_steps of a school on
// chip: each block keeps up to 11264 fish (x, y, weight, currentObjective and
// the feeding input) in shared memory and runs one compact pass over them
// per step -- the eat of step p fused with the swim of step p + 1, as in the
// streaming kernel -- so the step's code stays small and a school of a few
// hundred fish costs little more than its own pairs.  A school goes to the
// queue of the narrowest cluster that holds it (ceil(n / 11264) blocks, 1 to
// 8, so every block is at least half full):
//   - a cluster first takes schools from the queue of its own size, then
//     from the queues of smaller multi-block clusters; the warps of its C
//     blocks combine the per-step maxima by atomics in rank 0's shared
//     memory (distributed shared memory), with one cluster barrier per step,
//     and the barycentre partials follow one and two barriers behind, folded
//     in a fixed order;
//   - when those run out, every block pops single-block schools on its own
//     and synchronises with __syncthreads only;
//   - then schools of at most half a block are packed: the block's fish
//     warps split into teams (8, then 4, 2 and 1 warps), each with its own
//     share of the shared memory and its own named barrier (a single warp
//     needs none), popping schools that fill at least half of it.  A small
//     school thus runs beside others instead of leaving most of a block's
//     warps idle at every step's barrier (on one block, a school of 256
//     fish runs at a sixth of the rate per fish of a full one).
// The per-step order within a school is the paper's (Sec. 2.1.2 swim,
// Sec. 2.1.1 objective, delta, the Sec. 2.3.2 max, feeding, barycentre).
// School k uses key seeds[k] and school id k, so it reproduces the
// single-school path bit for bit.  Waits are hardware barriers on uniform
// control flow (every decision a cluster takes is broadcast from rank 0),
// so no block can be left waiting for another.
//
// One persistent launch per cluster size in use runs concurrently with the
// others, each on a share of the SMs in proportion to its queue's weighted
// fish (a launch of single blocks takes the SMs the clusters leave over);
// all of them share the queues, so the launches that finish first help the
// rest.  The kernel itself is in fsb_batch_kernel.cuh: this file
// instantiates it for clusters of 1 to 4 blocks, fsb_batch_wide.cu for 5 to
// 8, so the halves compile in parallel.
#include <cstdint>
#include <cstring>

#include "fsb_batch_kernel.cuh"

namespace fsb {
namespace {

// The variant kernels (var) share the default ones' block, register bound
// and shared memory, hence their occupancy.
const void* pick(int cluster, int acc, bool var = false) {
  switch (cluster) {
    case 1: return pick_acc<1>(acc, var);
    case 2: return pick_acc<2>(acc, var);
    case 3: return pick_acc<3>(acc, var);
    case 4: return pick_acc<4>(acc, var);
    case 5:
    case 6:
    case 7:
    case 8: return batch_kernel_wide(cluster, acc, var);
    default: return nullptr;
  }
}

cudaLaunchConfig_t make_config(int cluster, int grid, cudaStream_t s, cudaLaunchAttribute* attr) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(kBlockThreads);
  cfg.dynamicSmemBytes = kStateSmem;
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

uint64_t batch_block_capacity() { return kBlockFish; }
uint64_t batch_team_fish() { return kTeamFish; }

void batch_finish_stats(fsb_step_stats* st, size_t count, int acc) {
  if (acc == kAccF64) return;
  auto conv = [acc](double& v) {
    uint64_t bits;
    std::memcpy(&bits, &v, sizeof(bits));
    const uint32_t hb = static_cast<uint32_t>(bits), lb = static_cast<uint32_t>(bits >> 32);
    float hi, lo;
    std::memcpy(&hi, &hb, sizeof(hi));
    std::memcpy(&lo, &lb, sizeof(lo));
    v = acc == kAccKahan32 ? static_cast<double>(hi) + static_cast<double>(lo)
                           : static_cast<double>(hi);
  };
  for (size_t i = 0; i < count; ++i) {
    conv(st[i].sum_w);
    conv(st[i].sum_wx);
    conv(st[i].sum_wy);
  }
}
int batch_threads() { return kBatchThreads; }

// Clusters of `cluster` blocks that can be resident at once (0: cannot run).
// Also lets the cluster size's kernels (default and variant model) use the
// shared memory that holds a block's fish, so it runs before any launch.
int batch_max_clusters(int cluster, int acc) {
  const void* fn = pick(cluster, acc);
  if (!fn) return 0;
  for (const void* f : {fn, pick(cluster, acc, true)}) {
    if (cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             static_cast<int>(kStateSmem)) != cudaSuccess) {
      cudaGetLastError();
      return 0;
    }
  }
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
  // the variant copy also serves a default swim whose width's scaled form is
  // not exact (a step below 2^-103 but not 0): the default copy takes that
  // form without checking
  const bool var = L.swim_mode != 0 || L.feed_mode != 0 ||
                   !swim_scale_exact(static_cast<float>(L.step));
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
