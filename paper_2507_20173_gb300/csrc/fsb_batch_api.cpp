// fsb_batch_api.cpp -- C ABI of the batched (many schools) path: the batch
// handle (work list, device copies of the offset table and keys, statistics
// buffer, cached CUDA graph per call length) and the one-shot fsb_run_batch.
// All arithmetic runs in fsb_batch.cu.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <numeric>
#include <vector>

#include <cuda_runtime.h>

#include "fsb_internal.h"

namespace {

int bfail(int status, const char* fmt, ...) {
  char buf[400];
  va_list ap;
  va_start(ap, fmt);
  std::vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  return fsb::record_error(status, buf);
}

#define BCUDA(call)                                                                        \
  do {                                                                                     \
    cudaError_t e_ = (call);                                                               \
    if (e_ != cudaSuccess)                                                                 \
      return bfail(e_ == cudaErrorMemoryAllocation ? FSB_ERR_OOM : FSB_ERR_CUDA,           \
                   "%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__,      \
                   __LINE__);                                                              \
  } while (0)

struct BatchGraph {
  uint32_t n_steps;
  int init;
  cudaGraphExec_t exec;
};

}  // namespace

struct fsb_batch {
  fsb_config tmpl{};
  uint32_t n_schools = 0;
  uint64_t max_school = 0;
  cudaStream_t stream = nullptr;
  cudaStream_t cap_stream = nullptr;
  cudaStream_t side_stream[fsb::kBatchMaxLaunches - 1] = {};
  cudaEvent_t ev_fork = nullptr;
  cudaEvent_t ev_join[fsb::kBatchMaxLaunches - 1] = {};
  int forced_cluster = 0;              // 0: each school on the smallest cluster that holds it
  int sms = 0;
  unsigned long long* d_offsets = nullptr;
  unsigned long long* d_seeds = nullptr;
  uint32_t* d_order = nullptr;
  unsigned long long* d_base = nullptr;
  fsb::BatchCtl* d_bctl = nullptr;
  fsb_step_stats* d_stats = nullptr;
  size_t stats_cap = 0;
  std::vector<uint32_t> sizes_sorted;  // school index by size, largest first
  std::vector<uint64_t> offsets;       // host copy of the offset table
  int pending_init = 0;
  uint64_t step = 0;
  uint32_t last_n = 0;
  fsb::BatchLaunch L{};
  std::vector<BatchGraph> graphs;
  bool timing = false;
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev;
  double kernel_ms = 0.0;
  uint64_t launches = 0;
};

namespace {

// Work queues and launches of a batch.  A school of at most half a block
// goes to the packed queue of the smallest team of warps that holds it
// (with a forced cluster size of 1: to the single-block queue), another
// school one block holds to the single-block queue, a larger one to the
// queue of the smallest cluster that holds it (or, with a forced cluster
// size, to that size's queue).
// Each queue is largest first (longest-processing-time order).  One
// persistent launch per multi-block cluster size in use gets a share of the
// SMs in proportion to its queue's fish (with a forced size: every SM it
// can hold), largest cluster first; a launch of single blocks takes the SMs
// left over.
int plan_batch(fsb_batch* b, int forced) {
  const uint64_t cap = fsb::batch_block_capacity();
  if (forced < 0 || forced > fsb::kMaxBatchCluster)
    return bfail(FSB_ERR_INVALID_ARG, "batch cluster size must be 0 to %d", fsb::kMaxBatchCluster);
  const int widest = forced ? forced : fsb::kMaxBatchCluster;
  if (static_cast<uint64_t>(widest) * cap < b->max_school)
    return bfail(FSB_ERR_UNSUPPORTED,
                 "largest school (%llu fish) exceeds a cluster of %d blocks (%llu fish)",
                 static_cast<unsigned long long>(b->max_school), widest,
                 static_cast<unsigned long long>(widest * cap));
  // the narrowest resident width at least c (0: none up to the widest)
  int width_for[fsb::kMaxBatchCluster + 1] = {};
  for (int c = fsb::kMaxBatchCluster, next = 0; c >= 1; --c) {
    if (c == 1 || fsb::batch_max_clusters(c, b->L.acc) >= 1) next = c;
    width_for[c] = next;
  }
  std::vector<uint32_t> queue[fsb::kBatchQueues];
  uint64_t fish[fsb::kBatchQueues] = {};
  // schools of at most half a block are packed on teams of warps, unless
  // every school is to run on a block of its own (forced cluster size 1)
  const uint64_t team = forced == 1 ? 0 : fsb::batch_team_fish();
  for (uint32_t k : b->sizes_sorted) {
    const uint64_t n = b->offsets[k + 1] - b->offsets[k];
    const int need = static_cast<int>((n + cap - 1) / cap);  // blocks that hold it
    const int c = need <= 1 ? 1 : (forced ? forced : width_for[need]);
    if (c < 1) return bfail(FSB_ERR_UNSUPPORTED, "no resident cluster holds %d blocks", need);
    int t = fsb::batch_queue_of(c);
    if (c == 1 && team > 0 && 2 * n <= cap) {
      int warps = 1;  // the smallest team that holds it
      while (static_cast<uint64_t>(warps) * team < n) warps *= 2;
      t = fsb::batch_pack_queue_of(warps);
    }
    queue[t].push_back(k);
    fish[t] += n;
  }
  std::vector<uint32_t> order;
  order.reserve(b->n_schools);
  fsb::BatchLaunch& L = b->L;
  for (int t = 0; t < fsb::kBatchQueues; ++t) {
    L.queue_lo[t] = static_cast<uint32_t>(order.size());
    order.insert(order.end(), queue[t].begin(), queue[t].end());
  }
  L.queue_lo[fsb::kBatchQueues] = static_cast<uint32_t>(order.size());

  const int slots = fsb::batch_max_clusters(1, L.acc);  // resident single blocks
  if (slots < 1) return bfail(FSB_ERR_UNSUPPORTED, "batch kernel cannot be resident");
  // Work of a queue: its fish times a weight per cluster width, fitted on
  // GB300 to the best of a sweep of explicit plans over a log-uniform
  // ensemble (every launch helps the narrower queues once its own is empty,
  // so the single-block queue needs less than its share; index: cluster
  // size).
  const double cost[fsb::kMaxBatchCluster + 1] = {0.0, 0.8, 1.0, 1.1, 1.1, 1.1, 1.0, 0.9, 1.0};
  double work[fsb::kBatchQueues], total = 0.0;
  for (int t = 0; t < fsb::kBatchQueues; ++t) {
    // packed schools count as single-block ones
    const int c = t >= fsb::kBatchSingleQueue ? 1 : fsb::kMaxBatchCluster - t;
    work[t] = cost[c] * static_cast<double>(fish[t]);
    total += work[t];
  }
  int n = 0, used = 0;
  for (int c = fsb::kMaxBatchCluster; c >= 2; --c) {
    const int t = fsb::batch_queue_of(c);
    if (queue[t].empty()) continue;
    const int max_clusters = fsb::batch_max_clusters(c, L.acc);
    if (max_clusters < 1)
      return bfail(FSB_ERR_UNSUPPORTED, "clusters of %d blocks cannot be resident", c);
    int clusters = max_clusters;
    if (!forced) {
      // the widest launch rounds up: no other launch can take its schools,
      // while the narrower ones hand their spare time down to smaller queues
      const double share = static_cast<double>(slots) * work[t] / total / c;
      clusters = n == 0 ? static_cast<int>(std::ceil(share)) : static_cast<int>(share);
      clusters = clusters < 1 ? 1 : (clusters > max_clusters ? max_clusters : clusters);
      // never more blocks than the SMs left
      while (clusters > 1 && used + clusters * c > slots) --clusters;
    }
    if (used + clusters * c > slots && n > 0) continue;  // no room: a wider launch serves it
    L.cluster[n] = c;
    L.blocks[n] = clusters * c;
    used += L.blocks[n];
    ++n;
  }
  if (n == 0) {
    L.cluster[n] = 1;
    L.blocks[n] = slots;
    ++n;
  } else if (used < slots) {
    L.cluster[n] = 1;  // the SMs the clusters leave over
    L.blocks[n] = slots - used;
    ++n;
  }
  L.n_launches = n;
  BCUDA(cudaMemcpy(b->d_order, order.data(), sizeof(uint32_t) * order.size(),
                   cudaMemcpyHostToDevice));
  b->forced_cluster = forced;
  for (auto& g : b->graphs) cudaGraphExecDestroy(g.exec);
  b->graphs.clear();
  return FSB_OK;
}

int ensure_stats(fsb_batch* b, uint32_t n_steps) {
  const size_t need = static_cast<size_t>(b->n_schools) * (n_steps ? n_steps : 1);
  if (b->stats_cap >= need) return FSB_OK;
  BCUDA(cudaStreamSynchronize(b->stream));
  fsb_step_stats* p = nullptr;
  BCUDA(cudaMalloc(&p, sizeof(fsb_step_stats) * need));
  if (b->d_stats) cudaFree(b->d_stats);
  b->d_stats = p;
  b->stats_cap = need;
  for (auto& g : b->graphs) cudaGraphExecDestroy(g.exec);
  b->graphs.clear();
  return FSB_OK;
}

int enqueue(fsb_batch* b, uint32_t n_steps, int init, cudaStream_t s) {
  fsb::BatchLaunch L = b->L;
  L.n_steps = n_steps;
  L.init = init;
  L.stats = b->d_stats;
  BCUDA(fsb::launch_batch(L, s, b->side_stream, b->ev_fork, b->ev_join));
  if (n_steps) BCUDA(fsb::launch_bump_step(b->d_base, n_steps, s));
  return FSB_OK;
}

int get_graph(fsb_batch* b, uint32_t n_steps, int init, cudaGraphExec_t* out) {
  for (auto& g : b->graphs)
    if (g.n_steps == n_steps && g.init == init) {
      *out = g.exec;
      return FSB_OK;
    }
  BCUDA(cudaStreamBeginCapture(b->cap_stream, cudaStreamCaptureModeThreadLocal));
  const int rc = enqueue(b, n_steps, init, b->cap_stream);
  cudaGraph_t graph = nullptr;
  cudaError_t e = cudaStreamEndCapture(b->cap_stream, &graph);
  if (rc != FSB_OK) {
    if (graph) cudaGraphDestroy(graph);
    return rc;
  }
  BCUDA(e);
  cudaGraphExec_t exec = nullptr;
  e = cudaGraphInstantiate(&exec, graph, 0);
  cudaGraphDestroy(graph);
  BCUDA(e);
  if (b->graphs.size() >= 8) {
    cudaGraphExecDestroy(b->graphs.front().exec);
    b->graphs.erase(b->graphs.begin());
  }
  b->graphs.push_back({n_steps, init, exec});
  *out = exec;
  return FSB_OK;
}

void release(fsb_batch* b) {
  if (!b) return;
  cudaStreamSynchronize(b->stream);
  for (auto& g : b->graphs) cudaGraphExecDestroy(g.exec);
  for (auto& p : b->ev) {
    cudaEventDestroy(p.first);
    cudaEventDestroy(p.second);
  }
  cudaFree(b->d_offsets);
  cudaFree(b->d_seeds);
  cudaFree(b->d_order);
  cudaFree(b->d_base);
  cudaFree(b->d_bctl);
  cudaFree(b->d_stats);
  if (b->cap_stream) cudaStreamDestroy(b->cap_stream);
  for (int i = 0; i < fsb::kBatchMaxLaunches - 1; ++i) {
    if (b->side_stream[i]) cudaStreamDestroy(b->side_stream[i]);
    if (b->ev_join[i]) cudaEventDestroy(b->ev_join[i]);
  }
  if (b->ev_fork) cudaEventDestroy(b->ev_fork);
  delete b;
}

}  // namespace

extern "C" {

int fsb_batch_create(const fsb_config* tmpl, uint32_t n_schools, const uint64_t* offsets,
                     const uint64_t* seeds, const fsb_state_dev* state, int init,
                     uint64_t start_step, void* cuda_stream, fsb_batch_handle* out) {
  if (!out) return bfail(FSB_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (!tmpl || !offsets || !seeds || !state)
    return bfail(FSB_ERR_INVALID_ARG, "NULL argument");
  if (n_schools == 0) return bfail(FSB_ERR_INVALID_ARG, "n_schools must be >= 1");
  if (tmpl->precision == FSB_FP64_STATE)
    return bfail(FSB_ERR_UNSUPPORTED, "the batched path holds binary32 state only");
  if (tmpl->collective_mode != 0)
    return bfail(FSB_ERR_UNSUPPORTED, "the batched path runs no collective movements");
  if (tmpl->precision < FSB_FP32 || tmpl->precision > FSB_FP64_STATE)
    return bfail(FSB_ERR_INVALID_ARG, "unknown precision");
  if (!(tmpl->pond_half > 0.0) || !(tmpl->step >= 0.0) || !(tmpl->w_min <= tmpl->w_max) ||
      (tmpl->init_weight_mode != 0 && tmpl->init_weight_mode != 1) ||
      (tmpl->swim_mode != 0 && tmpl->swim_mode != 1) ||
      (tmpl->feed_mode != 0 && tmpl->feed_mode != 1) ||
      (tmpl->swim_mode == 1 && !(tmpl->w0 > 0.0)))
    return bfail(FSB_ERR_INVALID_ARG, "invalid physics in the template configuration");
  if (offsets[0] != 0) return bfail(FSB_ERR_INVALID_ARG, "offsets[0] must be 0");
  uint64_t max_school = 0;
  for (uint32_t k = 0; k < n_schools; ++k) {
    if (offsets[k + 1] <= offsets[k])
      return bfail(FSB_ERR_INVALID_ARG, "school %u is empty or offsets decrease", k);
    max_school = std::max<uint64_t>(max_school, offsets[k + 1] - offsets[k]);
  }
  if (init && start_step != 0)
    return bfail(FSB_ERR_INVALID_ARG, "initialising schools requires start_step 0");
  if (start_step >= 0xFFFFFFFFull) return bfail(FSB_ERR_INVALID_ARG, "start_step too large");
  const void* p[4] = {state->x, state->y, state->w, state->prev_objective};
  for (const void* q : p)
    if (!q || (reinterpret_cast<uintptr_t>(q) % 4) != 0)
      return bfail(FSB_ERR_INVALID_ARG, "state array NULL or not 4-byte aligned");

  fsb_batch* b = new (std::nothrow) fsb_batch();
  if (!b) return bfail(FSB_ERR_OOM, "host allocation failed");
  b->tmpl = *tmpl;
  b->n_schools = n_schools;
  b->max_school = max_school;
  b->stream = static_cast<cudaStream_t>(cuda_stream);
  b->pending_init = init ? 1 : 0;
  b->step = start_step;
  b->offsets.assign(offsets, offsets + n_schools + 1);
  b->sizes_sorted.resize(n_schools);
  std::iota(b->sizes_sorted.begin(), b->sizes_sorted.end(), 0u);
  std::stable_sort(b->sizes_sorted.begin(), b->sizes_sorted.end(), [&](uint32_t a, uint32_t c) {
    return offsets[a + 1] - offsets[a] > offsets[c + 1] - offsets[c];
  });
  auto body = [&]() -> int {
    BCUDA(cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking));
    for (int i = 0; i < fsb::kBatchMaxLaunches - 1; ++i) {
      BCUDA(cudaStreamCreateWithFlags(&b->side_stream[i], cudaStreamNonBlocking));
      BCUDA(cudaEventCreateWithFlags(&b->ev_join[i], cudaEventDisableTiming));
    }
    BCUDA(cudaEventCreateWithFlags(&b->ev_fork, cudaEventDisableTiming));
    int dev = 0;
    BCUDA(cudaGetDevice(&dev));
    BCUDA(cudaDeviceGetAttribute(&b->sms, cudaDevAttrMultiProcessorCount, dev));
    BCUDA(cudaMalloc(&b->d_offsets, sizeof(unsigned long long) * (n_schools + 1)));
    BCUDA(cudaMalloc(&b->d_seeds, sizeof(unsigned long long) * n_schools));
    BCUDA(cudaMalloc(&b->d_order, sizeof(uint32_t) * n_schools));
    BCUDA(cudaMalloc(&b->d_base, sizeof(unsigned long long)));
    BCUDA(cudaMalloc(&b->d_bctl, sizeof(fsb::BatchCtl)));
    BCUDA(cudaMemcpy(b->d_offsets, offsets, sizeof(unsigned long long) * (n_schools + 1),
                     cudaMemcpyHostToDevice));
    BCUDA(cudaMemcpy(b->d_seeds, seeds, sizeof(unsigned long long) * n_schools,
                     cudaMemcpyHostToDevice));
    const unsigned long long base = start_step;
    BCUDA(cudaMemcpy(b->d_base, &base, sizeof(base), cudaMemcpyHostToDevice));
    fsb::BatchLaunch& L = b->L;
    L.x = state->x;
    L.y = state->y;
    L.w = state->w;
    L.pv = state->prev_objective;
    L.offsets = b->d_offsets;
    L.seeds = b->d_seeds;
    L.order = b->d_order;
    L.n_schools = n_schools;
    L.pond_half = tmpl->pond_half;
    L.step = tmpl->step;
    L.w0 = tmpl->w0;
    L.w_min = tmpl->w_min;
    L.w_max = tmpl->w_max;
    L.swim_mode = tmpl->swim_mode;
    L.feed_mode = tmpl->feed_mode;
    L.acc = tmpl->precision == FSB_FP32 ? fsb::kAccPlain32
            : tmpl->precision == FSB_FP32_KAHAN ? fsb::kAccKahan32 : fsb::kAccF64;
    L.weight_mode = tmpl->init_weight_mode;
    L.base_step = b->d_base;
    L.bctl = b->d_bctl;
    int rc = plan_batch(b, 0);
    if (rc != FSB_OK) return rc;
    return ensure_stats(b, 1);
  };
  const int rc = body();
  if (rc != FSB_OK) {
    release(b);
    return rc;
  }
  *out = b;
  return FSB_OK;
}

int fsb_batch_step(fsb_batch_handle b, uint32_t n_steps, fsb_step_stats* host_stats) {
  if (!b) return bfail(FSB_ERR_INVALID_ARG, "batch handle is NULL");
  if (n_steps == 0 && !b->pending_init)
    return bfail(FSB_ERR_INVALID_ARG, "n_steps must be >= 1 (0 only to initialise)");
  if (b->step + n_steps > 0xFFFFFFFFull)
    return bfail(FSB_ERR_INVALID_ARG, "step counter would pass 2^32 - 1");
  int rc = ensure_stats(b, n_steps);
  if (rc != FSB_OK) return rc;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (b->timing) {
    BCUDA(cudaEventCreate(&e0));
    BCUDA(cudaEventCreate(&e1));
    BCUDA(cudaEventRecord(e0, b->stream));
  }
  cudaGraphExec_t exec = nullptr;
  rc = get_graph(b, n_steps, b->pending_init, &exec);
  if (rc != FSB_OK) return rc;
  BCUDA(cudaGraphLaunch(exec, b->stream));
  if (b->timing) {
    BCUDA(cudaEventRecord(e1, b->stream));
    b->ev.emplace_back(e0, e1);
  }
  b->pending_init = 0;
  b->step += n_steps;
  b->last_n = n_steps;
  if (host_stats && n_steps) {
    const size_t count = static_cast<size_t>(b->n_schools) * n_steps;
    BCUDA(cudaMemcpyAsync(host_stats, b->d_stats, sizeof(fsb_step_stats) * count,
                          cudaMemcpyDeviceToHost, b->stream));
    BCUDA(cudaStreamSynchronize(b->stream));
    fsb::batch_finish_stats(host_stats, count, b->L.acc);
    // the debug build's invariant checks (always 0 in the release build)
    int status = 0;
    BCUDA(cudaMemcpy(&status, &b->d_bctl->status, sizeof(int), cudaMemcpyDeviceToHost));
    if (status != 0) return bfail(FSB_ERR_STATE, "batch kernel invariant check failed");
  }
  return FSB_OK;
}

int fsb_batch_limits(uint64_t* block_fish, uint64_t* team_fish, int* max_cluster) {
  if (block_fish) *block_fish = fsb::batch_block_capacity();
  if (team_fish) *team_fish = fsb::batch_team_fish();
  if (max_cluster) *max_cluster = fsb::kMaxBatchCluster;
  return FSB_OK;
}

int fsb_batch_set_cluster(fsb_batch_handle b, int cluster) {
  if (!b) return bfail(FSB_ERR_INVALID_ARG, "batch handle is NULL");
  BCUDA(cudaStreamSynchronize(b->stream));
  const int saved = b->forced_cluster;
  const int rc = plan_batch(b, cluster);
  if (rc != FSB_OK) plan_batch(b, saved);
  return rc;
}

int fsb_batch_info(fsb_batch_handle b, int* cluster, int* n_clusters, int* filler_blocks,
                   uint32_t* n_big, uint64_t* step) {
  if (!b) return bfail(FSB_ERR_INVALID_ARG, "batch handle is NULL");
  const fsb::BatchLaunch& L = b->L;
  const bool single_only = L.n_launches == 1 && L.cluster[0] == 1;
  if (cluster) *cluster = L.cluster[0];
  if (n_clusters) *n_clusters = L.blocks[0] / L.cluster[0];
  if (filler_blocks)
    *filler_blocks = !single_only && L.cluster[L.n_launches - 1] == 1 ? L.blocks[L.n_launches - 1] : 0;
  if (n_big) *n_big = L.queue_lo[fsb::kBatchSingleQueue];
  if (step) *step = b->step;
  return FSB_OK;
}

int fsb_batch_set_plan(fsb_batch_handle b, int n_launches, const int* cluster,
                       const int* blocks) {
  if (!b || !cluster || !blocks) return bfail(FSB_ERR_INVALID_ARG, "NULL argument");
  if (n_launches < 1 || n_launches > fsb::kBatchMaxLaunches)
    return bfail(FSB_ERR_INVALID_ARG, "n_launches must be 1 to %d", fsb::kBatchMaxLaunches);
  fsb::BatchLaunch& L = b->L;
  for (int i = 0; i < n_launches; ++i) {
    const int c = cluster[i];
    if (c < 1 || c > fsb::kMaxBatchCluster)
      return bfail(FSB_ERR_INVALID_ARG, "launch %d: cluster size must be 1 to %d", i,
                   fsb::kMaxBatchCluster);
    if (i > 0 && c >= cluster[i - 1])
      return bfail(FSB_ERR_INVALID_ARG, "launches must be in decreasing cluster size");
    if (blocks[i] < c || blocks[i] % c)
      return bfail(FSB_ERR_INVALID_ARG, "launch %d: blocks must be a positive multiple of %d",
                   i, c);
    if (c > 1 && fsb::batch_max_clusters(c, L.acc) < 1)
      return bfail(FSB_ERR_UNSUPPORTED, "clusters of %d blocks cannot be resident", c);
  }
  // every multi-block queue needs a launch of at least its cluster size (a
  // launch serves its own queue, then the smaller ones)
  for (int t = 0; t < fsb::kBatchSingleQueue; ++t)
    if (L.queue_lo[t + 1] > L.queue_lo[t] && cluster[0] < fsb::kMaxBatchCluster - t)
      return bfail(FSB_ERR_INVALID_ARG, "schools need clusters of %d blocks; the widest launch "
                   "has %d", fsb::kMaxBatchCluster - t, cluster[0]);
  BCUDA(cudaStreamSynchronize(b->stream));
  L.n_launches = n_launches;
  for (int i = 0; i < n_launches; ++i) {
    L.cluster[i] = cluster[i];
    L.blocks[i] = blocks[i];
  }
  for (auto& g : b->graphs) cudaGraphExecDestroy(g.exec);
  b->graphs.clear();
  return FSB_OK;
}

int fsb_batch_plan(fsb_batch_handle b, int* n_launches, int* cluster, int* blocks,
                   uint32_t* queue_schools) {
  if (!b) return bfail(FSB_ERR_INVALID_ARG, "batch handle is NULL");
  const fsb::BatchLaunch& L = b->L;
  if (n_launches) *n_launches = L.n_launches;
  for (int i = 0; i < fsb::kBatchMaxLaunches; ++i) {
    if (cluster) cluster[i] = i < L.n_launches ? L.cluster[i] : 0;
    if (blocks) blocks[i] = i < L.n_launches ? L.blocks[i] : 0;
  }
  if (queue_schools)
    for (int t = 0; t < fsb::kBatchQueues; ++t) queue_schools[t] = L.queue_lo[t + 1] - L.queue_lo[t];
  return FSB_OK;
}

int fsb_batch_set_timing(fsb_batch_handle b, int enable) {
  if (!b) return bfail(FSB_ERR_INVALID_ARG, "batch handle is NULL");
  b->timing = enable != 0;
  return FSB_OK;
}

int fsb_batch_kernel_time(fsb_batch_handle b, double* ms, uint64_t* launches) {
  if (!b) return bfail(FSB_ERR_INVALID_ARG, "batch handle is NULL");
  BCUDA(cudaStreamSynchronize(b->stream));
  for (auto& p : b->ev) {
    float t = 0.f;
    BCUDA(cudaEventElapsedTime(&t, p.first, p.second));
    b->kernel_ms += t;
    b->launches += 1;
    cudaEventDestroy(p.first);
    cudaEventDestroy(p.second);
  }
  b->ev.clear();
  if (ms) *ms = b->kernel_ms;
  if (launches) *launches = b->launches;
  return FSB_OK;
}

int fsb_batch_destroy(fsb_batch_handle b) {
  if (!b) return FSB_OK;
  cudaError_t e = cudaStreamSynchronize(b->stream);
  release(b);
  if (e != cudaSuccess)
    return bfail(FSB_ERR_CUDA, "sync at batch destroy: %s", cudaGetErrorString(e));
  return FSB_OK;
}

int fsb_run_batch(const fsb_config* tmpl, uint32_t n_schools, const uint64_t* offsets,
                  const uint64_t* seeds, const fsb_state_dev* state, int init,
                  uint64_t start_step, uint32_t n_steps, fsb_step_stats* stats,
                  void* cuda_stream) {
  fsb_batch_handle b = nullptr;
  int rc = fsb_batch_create(tmpl, n_schools, offsets, seeds, state, init, start_step,
                            cuda_stream, &b);
  if (rc != FSB_OK) return rc;
  rc = fsb_batch_step(b, n_steps, stats);
  const int rc2 = fsb_batch_destroy(b);
  return rc != FSB_OK ? rc : rc2;
}

}  // extern "C"
