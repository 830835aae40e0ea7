// fsb_api.cpp -- the C ABI of libfsb.so (declared in include/fsb.h).
//
// Handle lifecycle, argument validation, path selection, the statistics
// ring, CUDA-graph capture of the per-call pass sequence, kernel timing and
// the device status word.  All arithmetic of the method runs in the CUDA
// kernels (fsb_stream.cu, fsb_resident.cu, fsb_batch.cu); this file only
// orchestrates.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include <cuda_runtime.h>

#include "fsb_internal.h"

using fsb::BlockPartial;
using fsb::Ctl;
using fsb::StreamLaunch;

namespace {

thread_local char g_last_error[512] = "";

int fail(int status, const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  std::vsnprintf(g_last_error, sizeof(g_last_error), fmt, ap);
  va_end(ap);
  return status;
}

#define FSB_CUDA(call)                                                                  \
  do {                                                                                  \
    cudaError_t e_ = (call);                                                            \
    if (e_ != cudaSuccess) {                                                            \
      return fail(e_ == cudaErrorMemoryAllocation ? FSB_ERR_OOM : FSB_ERR_CUDA,         \
                  "%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, \
                  __LINE__);                                                            \
    }                                                                                   \
  } while (0)

constexpr uint32_t kGraphMaxSteps = 2048;  // whole-call graphs up to this size
constexpr uint32_t kChunk = 512;           // fused passes per chunk graph beyond it
constexpr int kMaxGraphs = 8;

bool aligned(const void* p, size_t a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; }

int validate_config(const fsb_config* c) {
  if (!c) return fail(FSB_ERR_INVALID_ARG, "config is NULL");
  if (c->n_fish == 0) return fail(FSB_ERR_INVALID_ARG, "n_fish must be >= 1");
  if (!(c->pond_half > 0.0)) return fail(FSB_ERR_INVALID_ARG, "pond_half must be > 0");
  if (!(c->step >= 0.0)) return fail(FSB_ERR_INVALID_ARG, "step must be >= 0");
  if (!(c->w_min <= c->w_max)) return fail(FSB_ERR_INVALID_ARG, "w_min must be <= w_max");
  if (c->init_weight_mode != 0 && c->init_weight_mode != 1)
    return fail(FSB_ERR_INVALID_ARG, "init_weight_mode must be 0 or 1");
  if (c->precision < FSB_FP32 || c->precision > FSB_FP64_STATE)
    return fail(FSB_ERR_INVALID_ARG, "unknown precision %d", c->precision);
  if (c->path < FSB_PATH_AUTO || c->path > FSB_PATH_RESIDENT)
    return fail(FSB_ERR_INVALID_ARG, "unknown path %d", c->path);
  if (c->swim_mode != 0 && c->swim_mode != 1)
    return fail(FSB_ERR_INVALID_ARG, "swim_mode must be 0 or 1");
  if (c->feed_mode != 0 && c->feed_mode != 1)
    return fail(FSB_ERR_INVALID_ARG, "feed_mode must be 0 or 1");
  if (c->swim_mode == 1 && !(c->w0 > 0.0))
    return fail(FSB_ERR_INVALID_ARG, "the weight-scaled swim needs w0 > 0");
  if (c->collective_mode != 0 && c->collective_mode != 1)
    return fail(FSB_ERR_INVALID_ARG, "collective_mode must be 0 or 1");
  if (c->collective_mode == 1 && !(c->step_vol >= 0.0))
    return fail(FSB_ERR_INVALID_ARG, "step_vol must be >= 0");
  return FSB_OK;
}

// Largest k in [-100, 100] with n * bound * 2^k <= 2^62: the grid of an
// exact school sum of n terms bounded by `bound` (collective movements); the
// sum stays below 2^62.
int grid_exponent(uint64_t n, double bound) {
  const double lim = 4611686018427387904.0;  // 2^62
  double t = static_cast<double>(n) * bound;
  int k = 0;
  if (t > lim) {
    while (t > lim && k > -100) {
      t *= 0.5;
      --k;
    }
    return k;
  }
  while (2.0 * t <= lim && k < 100) {
    t *= 2.0;
    ++k;
  }
  return k;
}

// Grid exponents of the collective sums from bounds that hold for every
// value the school can take: swim products dx * g, improvements g, and the
// weight sums w, w x, w y.
void collective_grids(const fsb_config* c, int* kp, int* kg, int* kw) {
  const double a =
      std::fmax(std::fmax(std::fabs(c->w_min), std::fabs(c->w_max)), 1.5 * std::fabs(c->w0));
  const double sm = c->swim_mode == 1 ? 2.0 * c->step * std::fmax(1.0, a / c->w0) : 2.0 * c->step;
  const double e = std::ldexp(1.0, -20) * std::fmax(c->pond_half, 1.0);
  const double bd = sm + e;
  *kp = grid_exponent(c->n_fish, 2.0 * bd * bd);
  *kg = grid_exponent(c->n_fish, 2.0 * bd);
  *kw = grid_exponent(c->n_fish, 2.0 * a * std::fmax(c->pond_half, 1.0));
}

int acc_mode(int precision) {
  switch (precision) {
    case FSB_FP32: return fsb::kAccPlain32;
    case FSB_FP32_KAHAN: return fsb::kAccKahan32;
    default: return fsb::kAccF64;
  }
}

}  // namespace

namespace fsb {
// Lets other translation units report through fsb_last_error().
int record_error(int status, const char* msg) { return fail(status, "%s", msg); }
}  // namespace fsb

struct GraphEntry {
  uint32_t key;  // n_steps, or (1u << 31) | chunk for a fused-only chunk graph
  cudaGraphExec_t exec;
};

struct fsb_school {
  fsb_config cfg{};
  int device = 0;
  cudaStream_t stream = nullptr;       // caller's stream (not owned)
  cudaStream_t cap_stream = nullptr;   // owned, used only to capture graphs
  bool owns_state = false;
  size_t elem = 4;
  void* x = nullptr;
  void* y = nullptr;
  void* w = nullptr;
  void* pv = nullptr;
  uint64_t step = 0;
  uint32_t last_n = 0;
  int path = FSB_PATH_STREAM;
  Ctl* ctl = nullptr;
  BlockPartial* partials = nullptr;
  fsb_step_stats* ring = nullptr;
  uint32_t ring_cap = 0;
  int sms = 0;
  fsb_tuning tuning{};
  StreamLaunch launch{};
  fsb::ResidentLaunch res{};
  fsb::ResCtl* rctl = nullptr;
  double* sums = nullptr;
  size_t sums_cap = 0;             // doubles
  std::vector<GraphEntry> graphs;
  bool timing = false;
  std::vector<cudaEvent_t> ev_free;
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev_pending;
  double fused_ms = 0.0;
  uint64_t fused_launches = 0;
  void* cur_stage = nullptr;       // two chunks of currentObjective for fsb_read_state
  uint64_t cur_chunk = 0;          // fish per chunk
  BlockPartial* bpartials = nullptr;  // stream kernels 4, 5: per-step partials of a pair
  float* slots = nullptr;          // stream kernel 5: positions of a pair's steps
  size_t slot_bytes = 0;
  bool collective = false;         // collective_mode 1: two passes per step
  fsb::CollLaunch coll{};
  uint32_t coll_cap = 0;           // steps the collective record ring holds
};

namespace {

int check_status_word(fsb_school* h) {
  int status = 0;
  FSB_CUDA(cudaMemcpyAsync(&status, &h->ctl->status, sizeof(int), cudaMemcpyDeviceToHost,
                           h->stream));
  FSB_CUDA(cudaStreamSynchronize(h->stream));
  if (status != 0)
    return fail(status, "device status word latched %d (%s)", status, fsb_strerror(status));
  return FSB_OK;
}

// The collective records of a call of n steps (one per step).
int ensure_coll(fsb_school* h, uint32_t n) {
  if (!h->collective || h->coll_cap >= n) return FSB_OK;
  uint32_t cap = h->coll_cap ? h->coll_cap : 1024;
  while (cap < n) cap = cap > 0x7FFFFFFFu ? n : cap * 2;
  FSB_CUDA(cudaStreamSynchronize(h->stream));
  fsb::CollRec* recs = nullptr;
  FSB_CUDA(cudaMalloc(&recs, sizeof(fsb::CollRec) * cap));
  FSB_CUDA(cudaMemset(recs, 0, sizeof(fsb::CollRec) * cap));
  if (h->coll.coll) cudaFree(h->coll.coll);
  h->coll.coll = recs;
  h->coll_cap = cap;
  for (auto& g : h->graphs) cudaGraphExecDestroy(g.exec);
  h->graphs.clear();
  return FSB_OK;
}

int ensure_ring(fsb_school* h, uint32_t n) {
  if (h->ring_cap >= n) return FSB_OK;
  uint32_t cap = h->ring_cap ? h->ring_cap : 1024;
  while (cap < n) cap = cap > 0x7FFFFFFFu ? n : cap * 2;
  FSB_CUDA(cudaStreamSynchronize(h->stream));
  fsb_step_stats* ring = nullptr;
  FSB_CUDA(cudaMalloc(&ring, sizeof(fsb_step_stats) * cap));
  FSB_CUDA(cudaMemset(ring, 0, sizeof(fsb_step_stats) * cap));
  if (h->ring) cudaFree(h->ring);
  h->ring = ring;
  h->ring_cap = cap;
  h->launch.ring = ring;
  h->launch.ring_cap = cap;
  // graphs captured the old ring address
  for (auto& g : h->graphs) cudaGraphExecDestroy(g.exec);
  h->graphs.clear();
  return FSB_OK;
}

int launch_pass(fsb_school* h, int kind, cudaStream_t s) {
  if (h->launch.tma == 2)
    FSB_CUDA(fsb::launch_stream_pass_ws(h->launch, kind, s));
  else if (h->launch.tma)
    FSB_CUDA(fsb::launch_stream_pass_tma(h->launch, kind, s));
  else
    FSB_CUDA(fsb::launch_stream_pass(h->launch, kind, s));
  return FSB_OK;
}

cudaEvent_t take_event(fsb_school* h);

// The collective call (collective_mode 1): swim0, then eat t and move t for
// every step t; the last move closes the call.
int enqueue_collective(fsb_school* h, uint32_t n, cudaStream_t s, bool timed) {
  fsb::CollLaunch& C = h->coll;
  C.ring = h->ring;
  FSB_CUDA(fsb::launch_coll_pass(C, fsb::kCSwim0, n, s));
  for (uint32_t t = 1; t <= n; ++t) {
    cudaEvent_t a = nullptr, b = nullptr;
    if (timed) {
      a = take_event(h);
      b = take_event(h);
      if (!a || !b) return fail(FSB_ERR_CUDA, "cudaEventCreate failed");
      FSB_CUDA(cudaEventRecord(a, s));
    }
    FSB_CUDA(fsb::launch_coll_pass(C, fsb::kCEat, n, s));
    FSB_CUDA(fsb::launch_coll_pass(C, t == n ? fsb::kCMoveLast : fsb::kCMove, n, s));
    if (timed) {
      FSB_CUDA(cudaEventRecord(b, s));
      h->ev_pending.emplace_back(a, b);
    }
  }
  return FSB_OK;
}

// Enqueue the pass sequence of one call on stream s (capturable).
// Stream kernel 4: the pairs of blocked passes between the call's first
// swim and its last eat, each advancing up to blocked_k steps (timed pairs
// bracketed by events when `timed`).
int enqueue_blocked(fsb_school* h, uint32_t n, cudaStream_t s, bool timed) {
  int rc = launch_pass(h, fsb::kSwimOnly, s);
  const uint32_t K = static_cast<uint32_t>(h->launch.blocked_k);
  for (uint32_t j = 1; rc == FSB_OK && j < n; j += K) {
    const uint32_t k = n - j < K ? n - j : K;
    cudaEvent_t a = nullptr, b = nullptr;
    if (timed) {
      a = take_event(h);
      b = take_event(h);
      if (!a || !b) return fail(FSB_ERR_CUDA, "cudaEventCreate failed");
      FSB_CUDA(cudaEventRecord(a, s));
    }
    FSB_CUDA(fsb::launch_blocked_pair(h->launch, k, s));
    if (timed) {
      FSB_CUDA(cudaEventRecord(b, s));
      h->ev_pending.emplace_back(a, b);
    }
  }
  if (rc == FSB_OK) rc = launch_pass(h, fsb::kSettle, s);
  return rc;
}

int enqueue_call(fsb_school* h, uint32_t n, cudaStream_t s) {
  if (h->collective) return enqueue_collective(h, n, s, false);
  if (h->launch.blocked_k) return enqueue_blocked(h, n, s, false);
  int rc = launch_pass(h, fsb::kSwimOnly, s);
  for (uint32_t k = 1; rc == FSB_OK && k < n; ++k) rc = launch_pass(h, fsb::kFused, s);
  if (rc == FSB_OK) rc = launch_pass(h, fsb::kSettle, s);
  return rc;
}

int get_graph(fsb_school* h, uint32_t key, cudaGraphExec_t* out) {
  for (auto& g : h->graphs)
    if (g.key == key) {
      *out = g.exec;
      return FSB_OK;
    }
  cudaGraph_t graph = nullptr;
  FSB_CUDA(cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeThreadLocal));
  int rc;
  if (key & (1u << 31)) {
    rc = FSB_OK;
    for (uint32_t k = 0; rc == FSB_OK && k < (key & 0x7FFFFFFFu); ++k)
      rc = launch_pass(h, fsb::kFused, h->cap_stream);
  } else {
    rc = enqueue_call(h, key, h->cap_stream);
  }
  cudaError_t e = cudaStreamEndCapture(h->cap_stream, &graph);
  if (rc != FSB_OK) {
    if (graph) cudaGraphDestroy(graph);
    return rc;
  }
  FSB_CUDA(e);
  cudaGraphExec_t exec = nullptr;
  e = cudaGraphInstantiate(&exec, graph, 0);
  cudaGraphDestroy(graph);
  FSB_CUDA(e);
  if (static_cast<int>(h->graphs.size()) >= kMaxGraphs) {
    cudaGraphExecDestroy(h->graphs.front().exec);
    h->graphs.erase(h->graphs.begin());
  }
  h->graphs.push_back({key, exec});
  *out = exec;
  return FSB_OK;
}

cudaEvent_t take_event(fsb_school* h) {
  if (!h->ev_free.empty()) {
    cudaEvent_t e = h->ev_free.back();
    h->ev_free.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
  return e;
}

int collect_timing(fsb_school* h) {
  if (h->ev_pending.empty()) return FSB_OK;
  FSB_CUDA(cudaStreamSynchronize(h->stream));
  for (auto& pr : h->ev_pending) {
    float ms = 0.f;
    FSB_CUDA(cudaEventElapsedTime(&ms, pr.first, pr.second));
    h->fused_ms += ms;
    h->fused_launches += 1;
    h->ev_free.push_back(pr.first);
    h->ev_free.push_back(pr.second);
  }
  h->ev_pending.clear();
  return FSB_OK;
}

int run_timed(fsb_school* h, uint32_t n) {
  int rc = launch_pass(h, fsb::kSwimOnly, h->stream);
  for (uint32_t k = 1; rc == FSB_OK && k < n; ++k) {
    cudaEvent_t a = take_event(h), b = take_event(h);
    if (!a || !b) return fail(FSB_ERR_CUDA, "cudaEventCreate failed");
    FSB_CUDA(cudaEventRecord(a, h->stream));
    rc = launch_pass(h, fsb::kFused, h->stream);
    FSB_CUDA(cudaEventRecord(b, h->stream));
    h->ev_pending.emplace_back(a, b);
  }
  if (rc == FSB_OK) rc = launch_pass(h, fsb::kSettle, h->stream);
  return rc;
}

int run_stream(fsb_school* h, uint32_t n) {
  if (h->collective) {
    if (h->timing || n > kGraphMaxSteps) return enqueue_collective(h, n, h->stream, h->timing);
    cudaGraphExec_t exec = nullptr;
    int rc = get_graph(h, n, &exec);
    if (rc != FSB_OK) return rc;
    FSB_CUDA(cudaGraphLaunch(exec, h->stream));
    return FSB_OK;
  }
  if (h->launch.blocked_k) {
    if (h->timing || n > kGraphMaxSteps) return enqueue_blocked(h, n, h->stream, h->timing);
    cudaGraphExec_t exec = nullptr;
    int rc = get_graph(h, n, &exec);
    if (rc != FSB_OK) return rc;
    FSB_CUDA(cudaGraphLaunch(exec, h->stream));
    return FSB_OK;
  }
  if (h->timing) return run_timed(h, n);
  cudaGraphExec_t exec = nullptr;
  if (n <= kGraphMaxSteps) {
    int rc = get_graph(h, n, &exec);
    if (rc != FSB_OK) return rc;
    FSB_CUDA(cudaGraphLaunch(exec, h->stream));
    return FSB_OK;
  }
  int rc = launch_pass(h, fsb::kSwimOnly, h->stream);
  uint32_t rem = n - 1;
  if (rc == FSB_OK && rem >= kChunk) rc = get_graph(h, (1u << 31) | kChunk, &exec);
  while (rc == FSB_OK && rem >= kChunk) {
    FSB_CUDA(cudaGraphLaunch(exec, h->stream));
    rem -= kChunk;
  }
  while (rc == FSB_OK && rem > 0) {
    rc = launch_pass(h, fsb::kFused, h->stream);
    --rem;
  }
  if (rc == FSB_OK) rc = launch_pass(h, fsb::kSettle, h->stream);
  return rc;
}

// Pick (fish per thread, block, grid) so a school of n fish sits in
// registers across at most one block per SM.  Returns false if it does not
// fit on chip.
bool resident_config(int sms, int acc, int swim_mode, double step, uint64_t n,
                     fsb::ResidentLaunch* R, int want_fpt = 0, int want_block = 0) {
  const int fpts[] = {4, 8, 12, 16};
  for (int fpt : fpts) {
    if (want_fpt && fpt != want_fpt) continue;
    const int maxb = fsb::resident_max_block(fpt);
    if (want_block && (want_block % 32 || want_block > maxb)) return false;
    // Four fish per thread without a requested block: the smallest block
    // (a multiple of 32 threads) that holds the school on at most one block
    // per SM.  A step costs the slowest block's pass plus the grid barrier,
    // and on GB300 it shrinks with the blocks: 10^4 fish took 1.6 us per
    // step on 79 blocks of 32 fish threads against 1.9-2.1 us on 10 blocks
    // of 512, 10^3 fish 1.6 us on 8 blocks of 32 against 5.0 us on one of
    // 512.  A school too large for that falls through to the rule below.
    int small_block = 0;
    if (fpt == 4 && !want_block) {
      const uint64_t per_sm = (n + static_cast<uint64_t>(sms) - 1) / static_cast<uint64_t>(sms);
      const uint64_t threads = ((per_sm + fpt - 1) / fpt + 31) / 32 * 32;
      if (threads <= static_cast<uint64_t>(maxb)) small_block = threads < 32 ? 32 : static_cast<int>(threads);
    }
    // a block holds at most fpt fish per thread of its largest block (or of
    // the requested one), within the shared memory
    const int cap_block = want_block ? want_block : (small_block ? small_block : maxb);
    const uint64_t per_block = fsb::resident_max_slice(fpt, cap_block);
    uint64_t grid = (n + per_block - 1) / per_block;
    if (grid > static_cast<uint64_t>(sms)) continue;
    if (grid < 1) grid = 1;
    // spread over more SMs while every block keeps at least fpt * 256 fish
    // (a block's step is latency-bound below some slice; the fish-per-thread
    // setting picks that floor, 1024 to 4096, so the autotuner can trade a
    // cheaper grid barrier against more work per block)
    const uint64_t floor_fish = static_cast<uint64_t>(fpt) * 256;
    const uint64_t spread = (n + floor_fish - 1) / floor_fish;
    const uint64_t most = spread < static_cast<uint64_t>(sms) ? spread : sms;
    if (!small_block && grid < most) grid = most;
    // even, so no fish pair (one swim block) straddles two blocks
    const uint64_t slice = ((n + grid - 1) / grid + 1) & ~1ull;
    // the requested block, the small block, else the largest one with a
    // pair for every thread
    const uint64_t pairs32 = ((slice / 2 + 31) / 32) * 32;
    const int block = want_block ? want_block
                      : small_block ? small_block
                                    : static_cast<int>(pairs32 < static_cast<uint64_t>(maxb) ? pairs32 : maxb);
    if (slice > fsb::resident_max_slice(fpt, block)) continue;
    if (fsb::resident_blocks_per_sm(fpt, acc, block, swim_mode, step) < 1) continue;
    R->fpt = fpt;
    R->block = block;
    R->grid = static_cast<int>((n + slice - 1) / slice);
    R->slice = slice;
    return true;
  }
  return false;
}

constexpr int kMaxPartialsPerSm = 8;
// fsb_read_state computes currentObjective in chunks of this many fish
constexpr uint64_t kCurChunk = 1ull << 22;

// Streaming launch shape: kernel variant, block, grid.  Invalidates graphs.
constexpr int kMaxBlockSteps = 8;
// The library's streaming kernel for a school of at least this many fish
// (binary32, aligned state, default swim): kernel 5 with 8 steps per pair.
// Measured on GB300 against kernel 1: 2^20 fish (in L2) 2.50e11 against
// 2.51e11 fish-steps/s, 2^22 1.45e11 against 1.24e11, 2^24 2.13e11 against
// 1.76e11, 2^26 2.39e11 against 1.98e11, 2^28 2.46e11 against 2.01e11.
constexpr uint64_t kBlockedMinFish = 1ull << 22;

int configure_stream(fsb_school* h, int kernel, int block, int blocks_per_sm, int stages,
                     int block_steps) {
  StreamLaunch L = h->launch;
  const bool tma_ok = !L.real_is_double && L.vec == 4;
  // the library's choice: kernel 5 (k = 8) for a large streaming school
  // whose position slots (64 B per fish) take at most half of the free
  // device memory, else kernel 1
  if (kernel == 0 && block == 0 && blocks_per_sm == 0 && stages == 0 && block_steps == 0 &&
      h->path == FSB_PATH_STREAM && !h->collective && h->cfg.n_fish >= kBlockedMinFish &&
      fsb::stream_blocked_supported(L)) {
    size_t free_b = 0, total_b = 0;
    const size_t slots = 64 * static_cast<size_t>(h->cfg.n_fish);
    if (cudaMemGetInfo(&free_b, &total_b) == cudaSuccess && slots <= free_b / 2 &&
        configure_stream(h, 5, 0, 0, 0, 8) == FSB_OK)
      return FSB_OK;
    cudaGetLastError();
  }
  // stream kernels 4 and 5 run the call's first swim and last eat on kernel
  // 1 in its default shape, and the pairs of blocked passes in between;
  // kernel 5 keeps 2 k position arrays of the school's size (8 k B per fish)
  if (kernel == 4 || kernel == 5) {
    if (!fsb::stream_blocked_supported(L) || h->collective)
      return fail(FSB_ERR_INVALID_ARG, "stream kernels 4 and 5 need binary32, 16-byte aligned "
                  "state, the default swim and a swim step of 0 or at least 2^-103");
    if (block != 0 && block != 256)
      return fail(FSB_ERR_INVALID_ARG, "stream kernels 4 and 5 run 256-thread blocks");
    const int k = block_steps ? block_steps : (kernel == 5 ? 8 : 4);
    if (k != 2 && k != 4 && k != 8)
      return fail(FSB_ERR_INVALID_ARG, "stream_block_steps must be 2, 4 or 8");
    const uint64_t ss = (h->cfg.n_fish + 3) / 4 * 4;
    const size_t need_slots = kernel == 5 ? sizeof(float) * 2 * static_cast<size_t>(k) * ss : 0;
    if (need_slots > h->slot_bytes) {
      // before the handle changes, so that a failure leaves it as it was
      float* p = nullptr;
      const cudaError_t e = cudaMalloc(&p, need_slots);
      if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(e == cudaErrorMemoryAllocation ? FSB_ERR_OOM : FSB_ERR_CUDA,
                    "stream kernel 5: %zu bytes of position slots: %s", need_slots,
                    cudaGetErrorString(e));
      }
      cudaFree(h->slots);
      h->slots = p;
      h->slot_bytes = need_slots;
    }
    int rc = configure_stream(h, 1, 256, 4, 0, 0);
    if (rc != FSB_OK) return rc;
    L = h->launch;
    L.blocked_k = k;
    L.slots = kernel == 5 ? h->slots : nullptr;
    L.slot_stride = kernel == 5 ? ss : 0;
    const int per_sm = fsb::stream_blocked_blocks_per_sm(L);
    if (per_sm < 1) return fail(FSB_ERR_INVALID_ARG, "stream kernel 4 cannot be resident");
    const uint64_t need = (h->cfg.n_fish / 4 + 255) / 256;
    const uint64_t full = static_cast<uint64_t>(h->sms) * per_sm;
    L.bgrid = static_cast<int>(need < 1 ? 1 : (need < full ? need : full));
    if (!h->bpartials) {
      BlockPartial* bp = nullptr;
      FSB_CUDA(cudaMalloc(&bp, sizeof(BlockPartial) * kMaxBlockSteps * full));
      h->bpartials = bp;
    }
    L.bpartials = h->bpartials;
    h->launch = L;
    h->tuning.stream_kernel = kernel;
    h->tuning.stream_block_steps = k;
    return FSB_OK;
  }
  L.blocked_k = 0;
  L.slots = nullptr;
  L.slot_stride = 0;
  h->tuning.stream_block_steps = 0;
  // default measured on GB300 at N = 2^28: vector loads, 256 threads, 4
  // blocks per SM (0.96 of the copy peak, against 0.91 for the bulk-copy
  // ring and 0.90 for its warp-specialised form, timed back to back)
  if (kernel == 0) kernel = 1;
  if (stages == 0) stages = 2;
  if (stages < 2 || stages > 4) return fail(FSB_ERR_INVALID_ARG, "stream stages must be 2..4");
  if ((kernel == 2 || kernel == 3) && !tma_ok)
    return fail(FSB_ERR_INVALID_ARG, "bulk-copy kernels need binary32, 16-byte aligned state");
  if (kernel < 1 || kernel > 5) return fail(FSB_ERR_INVALID_ARG, "unknown stream kernel");
  if (kernel == 3 && stages > 3)
    return fail(FSB_ERR_INVALID_ARG, "warp-specialised ring: stages must be 2 or 3");
  if (block == 0) block = kernel == 1 ? 256 : 512;
  if (blocks_per_sm == 0 && kernel == 1 && block == 256) blocks_per_sm = 4;
  if (block != 256 && block != 512) return fail(FSB_ERR_INVALID_ARG, "stream block must be 256/512");
  L.tma = kernel - 1;
  L.block = block;
  L.stages = stages;
  // the vector kernel is compiled for 1, 3 or 4 guaranteed blocks per SM
  // (register budgets of 255, 80 and 64 per thread at 256 threads)
  L.min_blocks = 1;
  if (!L.tma && block == 256 && !L.real_is_double && L.vec == 4 &&
      (blocks_per_sm == 3 || blocks_per_sm == 4))
    L.min_blocks = blocks_per_sm;
  int per_sm = 0;
  if (L.tma == 2) {
    FSB_CUDA(fsb::stream_ws_prepare(L));
    per_sm = fsb::stream_ws_blocks_per_sm(L);
  } else if (L.tma) {
    FSB_CUDA(fsb::stream_tma_prepare(L));
    per_sm = fsb::stream_tma_blocks_per_sm(L);
  } else {
    per_sm = fsb::stream_blocks_per_sm(L);
  }
  if (per_sm < 1) return fail(FSB_ERR_INVALID_ARG, "stream kernel cannot be resident");
  if (blocks_per_sm > 0 && blocks_per_sm < per_sm) per_sm = blocks_per_sm;
  if (per_sm > kMaxPartialsPerSm) per_sm = kMaxPartialsPerSm;
  const uint64_t unit = L.tma ? static_cast<uint64_t>(block) * 4 : static_cast<uint64_t>(block) * L.vec;
  const uint64_t need = (h->cfg.n_fish + unit - 1) / unit;
  const uint64_t full = static_cast<uint64_t>(h->sms) * per_sm;
  L.grid = static_cast<int>(need < full ? need : full);
  if (L.grid < 1) L.grid = 1;
  h->launch = L;
  h->tuning.stream_kernel = kernel;
  h->tuning.stream_block = block;
  h->tuning.stream_blocks_per_sm = per_sm;
  h->tuning.stream_stages = L.tma ? stages : 0;
  for (auto& g : h->graphs) cudaGraphExecDestroy(g.exec);
  h->graphs.clear();
  return FSB_OK;
}

int ensure_sums(fsb_school* h, uint32_t n) {
  const size_t need = static_cast<size_t>(n) * h->res.grid * 3;
  if (h->sums_cap >= need) return FSB_OK;
  FSB_CUDA(cudaStreamSynchronize(h->stream));
  double* p = nullptr;
  FSB_CUDA(cudaMalloc(&p, need * sizeof(double)));
  if (h->sums) cudaFree(h->sums);
  h->sums = p;
  h->sums_cap = need;
  return FSB_OK;
}

int run_resident(fsb_school* h, uint32_t n) {
  int rc = ensure_sums(h, n);
  if (rc != FSB_OK) return rc;
  fsb::ResidentLaunch& R = h->res;
  R.base_step = h->step;
  R.n_steps = n;
  R.sums = h->sums;
  R.ring = h->ring;
  cudaEvent_t a = nullptr, b = nullptr;
  if (h->timing) {
    a = take_event(h);
    b = take_event(h);
    if (!a || !b) return fail(FSB_ERR_CUDA, "cudaEventCreate failed");
    FSB_CUDA(cudaEventRecord(a, h->stream));
  }
  FSB_CUDA(fsb::launch_resident(R, h->stream));
  if (h->timing) {
    FSB_CUDA(cudaEventRecord(b, h->stream));
    h->ev_pending.emplace_back(a, b);
  }
  R.inject_cta = -1;  // a fault injection applies to one call only
  return FSB_OK;
}

void release(fsb_school* h) {
  if (!h) return;
  if (h->stream || h->cap_stream) cudaStreamSynchronize(h->stream);
  for (auto& g : h->graphs) cudaGraphExecDestroy(g.exec);
  for (auto& pr : h->ev_pending) {
    cudaEventDestroy(pr.first);
    cudaEventDestroy(pr.second);
  }
  for (auto e : h->ev_free) cudaEventDestroy(e);
  if (h->owns_state) {
    cudaFree(h->x);
    cudaFree(h->y);
    cudaFree(h->w);
    cudaFree(h->pv);
  }
  cudaFree(h->ctl);
  cudaFree(h->rctl);
  cudaFree(h->sums);
  cudaFree(h->partials);
  cudaFree(h->bpartials);
  cudaFree(h->slots);
  cudaFree(h->ring);
  cudaFree(h->cur_stage);
  cudaFree(h->coll.partials);
  cudaFree(h->coll.coll);
  if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
  delete h;
}

}  // namespace

extern "C" {

int fsb_config_init(fsb_config* cfg, uint64_t n_fish, uint64_t seed) {
  if (!cfg) return fail(FSB_ERR_INVALID_ARG, "config is NULL");
  std::memset(cfg, 0, sizeof(*cfg));
  cfg->n_fish = n_fish;
  cfg->seed = seed;
  cfg->school_id = 0;
  cfg->init_weight_mode = 0;
  cfg->pond_half = 100.0;
  cfg->step = 0.1;
  cfg->w0 = 1.0;
  cfg->w_min = 0.0;
  cfg->w_max = 2.0;
  cfg->precision = FSB_FP32_KAHAN;
  cfg->path = FSB_PATH_AUTO;
  cfg->collective_mode = 0;
  cfg->step_vol = 0.1;
  return FSB_OK;
}

int fsb_create(const fsb_config* cfg, const fsb_state_dev* buffers, const fsb_state_host* init,
               uint64_t start_step, void* cuda_stream, fsb_handle* out) {
  if (!out) return fail(FSB_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  int rc = validate_config(cfg);
  if (rc != FSB_OK) return rc;
  if (start_step >= 0xFFFFFFFFull)
    return fail(FSB_ERR_INVALID_ARG, "start_step must be below 2^32 - 1");
  if (init && (!init->x || !init->y || !init->w || !init->prev_objective))
    return fail(FSB_ERR_INVALID_ARG, "init has a NULL array");
  const bool dbl = cfg->precision == FSB_FP64_STATE;
  const size_t elem = dbl ? 8 : 4;
  if (buffers) {
    const void* p[4] = {buffers->x, buffers->y, buffers->w, buffers->prev_objective};
    for (const void* q : p)
      if (!q || !aligned(q, elem))
        return fail(FSB_ERR_INVALID_ARG, "state buffer NULL or not %zu-byte aligned", elem);
  }

  fsb_school* h = new (std::nothrow) fsb_school();
  if (!h) return fail(FSB_ERR_OOM, "host allocation failed");
  h->cfg = *cfg;
  h->elem = elem;
  h->stream = static_cast<cudaStream_t>(cuda_stream);
  h->step = start_step;
  h->path = FSB_PATH_STREAM;

#define FSB_TRY(call)        \
  do {                       \
    int r_ = (call);         \
    if (r_ != FSB_OK) {      \
      release(h);            \
      return r_;             \
    }                        \
  } while (0)

  FSB_TRY([&]() -> int {
    FSB_CUDA(cudaGetDevice(&h->device));
    FSB_CUDA(cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking));
    const size_t bytes = elem * cfg->n_fish;
    if (buffers) {
      h->x = buffers->x;
      h->y = buffers->y;
      h->w = buffers->w;
      h->pv = buffers->prev_objective;
    } else {
      h->owns_state = true;
      FSB_CUDA(cudaMalloc(&h->x, bytes));
      FSB_CUDA(cudaMalloc(&h->y, bytes));
      FSB_CUDA(cudaMalloc(&h->w, bytes));
      FSB_CUDA(cudaMalloc(&h->pv, bytes));
    }
    FSB_CUDA(cudaMalloc(&h->ctl, sizeof(Ctl)));
    Ctl c{};
    c.base_step = start_step;
    FSB_CUDA(cudaMemcpyAsync(h->ctl, &c, sizeof(Ctl), cudaMemcpyHostToDevice, h->stream));

    StreamLaunch& L = h->launch;
    L.x = h->x;
    L.y = h->y;
    L.w = h->w;
    L.pv = h->pv;
    L.n = cfg->n_fish;
    L.seed = cfg->seed;
    L.school = cfg->school_id;
    L.real_is_double = dbl ? 1 : 0;
    L.acc = acc_mode(cfg->precision);
    const bool vec_ok = aligned(h->x, 16) && aligned(h->y, 16) && aligned(h->w, 16) &&
                        aligned(h->pv, 16);
    L.vec = vec_ok ? (dbl ? 2 : 4) : 1;
    L.pond_half = cfg->pond_half;
    L.step = cfg->step;
    L.w0 = cfg->w0;
    L.w_min = cfg->w_min;
    L.w_max = cfg->w_max;
    L.swim_mode = cfg->swim_mode;
    L.feed_mode = cfg->feed_mode;
    L.ctl = h->ctl;
    int sms = 0;
    FSB_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, h->device));
    h->sms = sms;
    FSB_CUDA(cudaMalloc(&h->partials, sizeof(BlockPartial) * sms * kMaxPartialsPerSm));
    L.partials = h->partials;
    // kernel 1 until the path is known (the library's choice below)
    int r0 = configure_stream(h, 1, 0, 0, 0, 0);
    if (r0 != FSB_OK) return r0;

    // collective movements: streaming only (two passes per step)
    if (cfg->collective_mode == 1) {
      if (cfg->path == FSB_PATH_RESIDENT)
        return fail(FSB_ERR_UNSUPPORTED, "resident path: the collective movements run streaming");
      h->collective = true;
      fsb::CollLaunch& C = h->coll;
      C.x = h->x;
      C.y = h->y;
      C.w = h->w;
      C.pv = h->pv;
      C.n = cfg->n_fish;
      C.seed = cfg->seed;
      C.school = cfg->school_id;
      C.real_is_double = dbl ? 1 : 0;
      C.acc = L.acc;
      C.pond_half = cfg->pond_half;
      C.step = cfg->step;
      C.w0 = cfg->w0;
      C.w_min = cfg->w_min;
      C.w_max = cfg->w_max;
      C.step_vol = cfg->step_vol;
      C.swim_mode = cfg->swim_mode;
      C.feed_mode = cfg->feed_mode;
      collective_grids(cfg, &C.kp, &C.kg, &C.kw);
      C.ctl = h->ctl;
      C.grid = fsb::coll_grid(C, sms);
      FSB_CUDA(cudaMalloc(&C.partials, sizeof(fsb::CollPartial) * C.grid));
    }

    // resident path: binary32 state that fits in registers across the SMs
    fsb::ResidentLaunch& R = h->res;
    const bool fits = !dbl && !h->collective &&
                      resident_config(sms, h->launch.acc, cfg->swim_mode, cfg->step, cfg->n_fish,
                                      &R);
    if (cfg->path == FSB_PATH_RESIDENT && !fits)
      return fail(FSB_ERR_UNSUPPORTED,
                  "resident path: school of %llu fish does not fit on chip (binary32 only)",
                  static_cast<unsigned long long>(cfg->n_fish));
    h->path = (cfg->path == FSB_PATH_STREAM || !fits) ? FSB_PATH_STREAM : FSB_PATH_RESIDENT;
    if (h->path == FSB_PATH_RESIDENT) {
      R.x = h->x;
      R.y = h->y;
      R.w = h->w;
      R.pv = h->pv;
      R.n = cfg->n_fish;
      R.seed = cfg->seed;
      R.school = cfg->school_id;
      R.pond_half = cfg->pond_half;
      R.step = cfg->step;
      R.w0 = cfg->w0;
      R.w_min = cfg->w_min;
      R.w_max = cfg->w_max;
      R.swim_mode = cfg->swim_mode;
      R.feed_mode = cfg->feed_mode;
      R.acc = h->launch.acc;
      h->tuning.resident_fpt = R.fpt;
      h->tuning.resident_block = R.block;
      R.ctl = h->ctl;
      R.timeout_ns = 1000000000ull;
      R.inject_cta = -1;
      R.inject_step = 0;
      FSB_CUDA(cudaMalloc(&h->rctl, sizeof(fsb::ResCtl)));
      R.rctl = h->rctl;
    }
    if (h->path == FSB_PATH_STREAM && !h->collective) {
      const int rk = configure_stream(h, 0, 0, 0, 0, 0);
      if (rk != FSB_OK) return rk;
    }
    // per-call scratch for calls of up to 1024 steps, so that such a call
    // allocates nothing (a longer one grows it, synchronising once)
    int r = ensure_ring(h, 1024);
    if (r == FSB_OK && h->path == FSB_PATH_RESIDENT) r = ensure_sums(h, 1024);
    if (r != FSB_OK) return r;
    StreamLaunch& L2 = h->launch;

    // pinned host arrays are copied in by the SMs (fsb_transfer.cu), others
    // by the copy engines
    // (no braced lists with commas here: this block is a macro argument)
    const void* in_dev[4] = {};
    bool direct = init != nullptr;
    if (init) {
      in_dev[0] = fsb::host_view(init->x);
      in_dev[1] = fsb::host_view(init->y);
      in_dev[2] = fsb::host_view(init->w);
      in_dev[3] = fsb::host_view(init->prev_objective);
      for (int k = 0; k < 4; ++k)
        if (!in_dev[k]) direct = false;
    }
    if (init && direct) {
      FSB_CUDA(fsb::launch_copy_in(L2, in_dev, h->stream));
    } else if (init) {
      FSB_CUDA(cudaMemcpyAsync(h->x, init->x, bytes, cudaMemcpyHostToDevice, h->stream));
      FSB_CUDA(cudaMemcpyAsync(h->y, init->y, bytes, cudaMemcpyHostToDevice, h->stream));
      FSB_CUDA(cudaMemcpyAsync(h->w, init->w, bytes, cudaMemcpyHostToDevice, h->stream));
      FSB_CUDA(cudaMemcpyAsync(h->pv, init->prev_objective, bytes, cudaMemcpyHostToDevice,
                               h->stream));
    } else {
      FSB_CUDA(fsb::launch_init(L2, cfg->init_weight_mode, h->stream));
    }
    return FSB_OK;
  }());
#undef FSB_TRY
  *out = h;
  return FSB_OK;
}

int fsb_step(fsb_handle h, uint32_t n_steps, fsb_step_stats* host_stats) {
  if (!h) return fail(FSB_ERR_INVALID_ARG, "handle is NULL");
  if (n_steps == 0) return fail(FSB_ERR_INVALID_ARG, "n_steps must be >= 1");
  if (h->step + n_steps > 0xFFFFFFFFull)
    return fail(FSB_ERR_INVALID_ARG, "step counter would pass 2^32 - 1");
  int rc = ensure_ring(h, n_steps);
  if (rc == FSB_OK) rc = ensure_coll(h, n_steps);
  if (rc != FSB_OK) return rc;
  rc = h->path == FSB_PATH_RESIDENT ? run_resident(h, n_steps) : run_stream(h, n_steps);
  if (rc != FSB_OK) return rc;
  h->step += n_steps;
  h->last_n = n_steps;
  if (host_stats) {
    FSB_CUDA(cudaMemcpyAsync(host_stats, h->ring, sizeof(fsb_step_stats) * n_steps,
                             cudaMemcpyDeviceToHost, h->stream));
    return check_status_word(h);
  }
  return FSB_OK;
}

int fsb_last_stats(fsb_handle h, fsb_step_stats* host_stats, uint32_t n_steps) {
  if (!h || !host_stats) return fail(FSB_ERR_INVALID_ARG, "NULL argument");
  if (n_steps == 0 || n_steps > h->last_n)
    return fail(FSB_ERR_INVALID_ARG, "n_steps must be in [1, %u]", h->last_n);
  FSB_CUDA(cudaMemcpyAsync(host_stats, h->ring, sizeof(fsb_step_stats) * n_steps,
                           cudaMemcpyDeviceToHost, h->stream));
  return check_status_word(h);
}

int fsb_read_state(fsb_handle h, void* x, void* y, void* w, void* prev_objective,
                   void* current_objective, uint64_t* step_out) {
  if (!h) return fail(FSB_ERR_INVALID_ARG, "handle is NULL");
  const size_t bytes = h->elem * h->cfg.n_fish;
  // all requested arrays pinned: one kernel writes them (and computes
  // currentObjective on the way, fsb_transfer.cu); else the copy engines
  void* out[5] = {x, y, w, prev_objective, current_objective};
  void* out_dev[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
  bool direct = false;
  for (int k = 0; k < 5; ++k) {
    if (!out[k]) continue;
    out_dev[k] = fsb::host_view(out[k]);
    direct = out_dev[k] != nullptr;
    if (!direct) break;
  }
  if (direct) {
    FSB_CUDA(fsb::launch_read_out(h->launch, out_dev, h->stream));
    if (step_out) *step_out = h->step;
    return check_status_word(h);
  }
  if (x) FSB_CUDA(cudaMemcpyAsync(x, h->x, bytes, cudaMemcpyDeviceToHost, h->stream));
  if (y) FSB_CUDA(cudaMemcpyAsync(y, h->y, bytes, cudaMemcpyDeviceToHost, h->stream));
  if (w) FSB_CUDA(cudaMemcpyAsync(w, h->w, bytes, cudaMemcpyDeviceToHost, h->stream));
  if (prev_objective)
    FSB_CUDA(cudaMemcpyAsync(prev_objective, h->pv, bytes, cudaMemcpyDeviceToHost, h->stream));
  if (current_objective) {
    // computed chunk by chunk into two alternating device buffers, each chunk
    // copied out behind its kernel (stream order keeps a buffer's copy ahead
    // of its next kernel), so the read needs no full-size scratch
    const uint64_t n = h->cfg.n_fish;
    if (!h->cur_stage) {
      h->cur_chunk = n < kCurChunk ? n : kCurChunk;
      FSB_CUDA(cudaMalloc(&h->cur_stage, 2 * h->cur_chunk * h->elem));
    }
    for (uint64_t first = 0, c = 0; first < n; first += h->cur_chunk, ++c) {
      const uint64_t count = n - first < h->cur_chunk ? n - first : h->cur_chunk;
      char* stage = static_cast<char*>(h->cur_stage) + (c & 1) * h->cur_chunk * h->elem;
      FSB_CUDA(fsb::launch_objective(h->launch, first, count, stage, h->stream));
      FSB_CUDA(cudaMemcpyAsync(static_cast<char*>(current_objective) + first * h->elem, stage,
                               count * h->elem, cudaMemcpyDeviceToHost, h->stream));
    }
  }
  if (step_out) *step_out = h->step;
  return check_status_word(h);
}

int fsb_destroy(fsb_handle h) {
  if (!h) return FSB_OK;
  cudaError_t e = cudaStreamSynchronize(h->stream);
  release(h);
  if (e != cudaSuccess) return fail(FSB_ERR_CUDA, "sync at destroy: %s", cudaGetErrorString(e));
  return FSB_OK;
}

int fsb_set_kernel_timing(fsb_handle h, int enable) {
  if (!h) return fail(FSB_ERR_INVALID_ARG, "handle is NULL");
  int rc = collect_timing(h);
  if (rc != FSB_OK) return rc;
  h->timing = enable != 0;
  h->fused_ms = 0.0;
  h->fused_launches = 0;
  return FSB_OK;
}

int fsb_kernel_time(fsb_handle h, double* fused_ms, uint64_t* fused_launches) {
  if (!h) return fail(FSB_ERR_INVALID_ARG, "handle is NULL");
  int rc = collect_timing(h);
  if (rc != FSB_OK) return rc;
  if (fused_ms) *fused_ms = h->fused_ms;
  if (fused_launches) *fused_launches = h->fused_launches;
  return FSB_OK;
}

int fsb_set_tuning(fsb_handle h, const fsb_tuning* t) {
  if (!h || !t) return fail(FSB_ERR_INVALID_ARG, "NULL argument");
  FSB_CUDA(cudaStreamSynchronize(h->stream));
  const StreamLaunch saved = h->launch;
  const fsb_tuning saved_t = h->tuning;
  int rc = configure_stream(h, t->stream_kernel, t->stream_block, t->stream_blocks_per_sm,
                            t->stream_stages, t->stream_block_steps);
  if (rc != FSB_OK) {
    h->launch = saved;
    h->tuning = saved_t;
    return rc;
  }
  if (h->path == FSB_PATH_RESIDENT && (t->resident_fpt || t->resident_block)) {
    fsb::ResidentLaunch R = h->res;
    if (!resident_config(h->sms, R.acc, R.swim_mode, h->cfg.step, h->cfg.n_fish, &R,
                         t->resident_fpt,
                         t->resident_block)) {
      h->launch = saved;
      h->tuning = saved_t;
      return fail(FSB_ERR_INVALID_ARG, "resident tuning does not fit this school");
    }
    h->res = R;
    h->tuning.resident_fpt = R.fpt;
    h->tuning.resident_block = R.block;
  }
  return FSB_OK;
}

int fsb_get_tuning(fsb_handle h, fsb_tuning* t) {
  if (!h || !t) return fail(FSB_ERR_INVALID_ARG, "NULL argument");
  *t = h->tuning;
  return FSB_OK;
}

int fsb_set_fault_injection(fsb_handle h, int block, uint32_t step, uint64_t timeout_ns) {
  if (!h) return fail(FSB_ERR_INVALID_ARG, "handle is NULL");
  if (h->collective)
    return fail(FSB_ERR_UNSUPPORTED, "the collective passes have no waits to make run out");
  if (h->path == FSB_PATH_RESIDENT) {
    if (block >= h->res.grid) return fail(FSB_ERR_INVALID_ARG, "block out of range");
    h->res.inject_cta = block < 0 ? -1 : block;
    h->res.inject_step = step;
    if (timeout_ns) h->res.timeout_ns = timeout_ns;
    return FSB_OK;
  }
  StreamLaunch& L = h->launch;
  if (!L.tma)
    return fail(FSB_ERR_UNSUPPORTED,
                "fault injection needs the resident path or a copy-ring stream kernel");
  if (block >= L.grid) return fail(FSB_ERR_INVALID_ARG, "block out of range");
  FSB_CUDA(cudaStreamSynchronize(h->stream));
  L.inject_block = block < 0 ? -1 : block;
  L.inject_pass = step;
  if (timeout_ns) L.timeout_ns = timeout_ns;
  // launch arguments are baked into the cached graphs
  for (auto& g : h->graphs) cudaGraphExecDestroy(g.exec);
  h->graphs.clear();
  return FSB_OK;
}

int fsb_handle_path(fsb_handle h, int* path_out) {
  if (!h || !path_out) return fail(FSB_ERR_INVALID_ARG, "NULL argument");
  *path_out = h->path;
  return FSB_OK;
}

int fsb_eat_max(const void* prev_objective, const void* current_objective, uint64_t n,
                int construct, double* result, float* device_ms, void* cuda_stream) {
  if (!prev_objective || !current_objective || !result)
    return fail(FSB_ERR_INVALID_ARG, "NULL argument");
  if (n == 0) return fail(FSB_ERR_INVALID_ARG, "n must be >= 1");
  if (construct < FSB_EAT_REDUCTION || construct > FSB_EAT_CRITICAL)
    return fail(FSB_ERR_INVALID_ARG, "unknown reduction construct %d", construct);
  if (!aligned(prev_objective, 16) || !aligned(current_objective, 16))
    return fail(FSB_ERR_INVALID_ARG, "arrays must be 16-byte aligned");
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  int dev = 0, sms = 0;
  FSB_CUDA(cudaGetDevice(&dev));
  FSB_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  // one scratch allocation: the winning order key, then the decoded value
  struct Scratch {
    double value;
    unsigned key;
  };
  Scratch* scratch = nullptr;
  FSB_CUDA(cudaMallocAsync(&scratch, sizeof(Scratch), s));
  cudaEvent_t a = nullptr, b = nullptr;
  cudaError_t e = cudaSuccess;
  if (device_ms) {
    e = cudaEventCreate(&a);
    if (e == cudaSuccess) e = cudaEventCreate(&b);
    if (e == cudaSuccess) e = cudaEventRecord(a, s);
  }
  const uint64_t want = (n / 4 + 255) / 256;
  const uint64_t full = static_cast<uint64_t>(sms) * 8;
  const int grid = static_cast<int>(want < 1 ? 1 : (want < full ? want : full));
  if (e == cudaSuccess)
    e = fsb::launch_eat_max(static_cast<const float*>(prev_objective),
                            static_cast<const float*>(current_objective), n, construct,
                            &scratch->key, &scratch->value, grid, s);
  if (device_ms && e == cudaSuccess) e = cudaEventRecord(b, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(result, &scratch->value, sizeof(double), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (device_ms && e == cudaSuccess) e = cudaEventElapsedTime(device_ms, a, b);
  // released on every path
  if (a) cudaEventDestroy(a);
  if (b) cudaEventDestroy(b);
  cudaFreeAsync(scratch, s);
  FSB_CUDA(e);
  return FSB_OK;
}

const char* fsb_strerror(int status) {
  switch (status) {
    case FSB_OK: return "FSB_OK";
    case FSB_ERR_INVALID_ARG: return "FSB_ERR_INVALID_ARG";
    case FSB_ERR_CUDA: return "FSB_ERR_CUDA";
    case FSB_ERR_OOM: return "FSB_ERR_OOM";
    case FSB_ERR_UNSUPPORTED: return "FSB_ERR_UNSUPPORTED";
    case FSB_ERR_TIMEOUT: return "FSB_ERR_TIMEOUT";
    case FSB_ERR_STATE: return "FSB_ERR_STATE";
    default: return "FSB_ERR_UNKNOWN";
  }
}

const char* fsb_last_error(void) { return g_last_error; }

}  // extern "C"
