// fsb_autotune.cpp -- the library's autotuner: for one school size and
// arithmetic mode it measures every launch shape the library can run and
// reports the fastest.
//
// Candidates:
//   streaming path: vector loads x {256, 512} threads x {occupancy, 3, 4}
//                   guaranteed blocks per SM; bulk-copy ring x {256, 512}
//                   threads x {2, 3, 4} stages
//   resident path:  fish per thread {4, 8, 12, 16} x the block sizes that
//                   keep the school in registers across at most one block
//                   per SM
// The path with the fastest candidate fixes the cutoff between the resident
// and the streaming kernels for that size.  Each candidate runs on a
// scratch school (library-owned state), one warm-up call, then `n_steps`
// steps timed with CUDA events on a private stream.  Results do not depend
// on the launch shape (every shape is parity-tested), so the tuner only
// compares time.
#include <cstdio>
#include <vector>

#include <cuda_runtime.h>

#include "fsb_internal.h"

namespace {

struct Candidate {
  int path;
  fsb_tuning t;
};

int time_candidate(const fsb_config* base, const Candidate& c, uint32_t n_steps,
                   cudaStream_t s, double* ms_out) {
  fsb_config cfg = *base;
  cfg.path = c.path;
  fsb_handle h = nullptr;
  int rc = fsb_create(&cfg, nullptr, nullptr, 0, s, &h);
  if (rc != FSB_OK) return rc;
  rc = fsb_set_tuning(h, &c.t);
  if (rc == FSB_ERR_OOM) rc = FSB_ERR_UNSUPPORTED;  // this shape's scratch does not fit: skip it
  if (rc == FSB_OK) rc = fsb_step(h, n_steps < 8 ? n_steps : 8, nullptr);  // warm-up
  cudaEvent_t a = nullptr, b = nullptr;
  if (rc == FSB_OK && (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess))
    rc = FSB_ERR_CUDA;
  if (rc == FSB_OK && cudaStreamSynchronize(s) != cudaSuccess) rc = FSB_ERR_CUDA;
  if (rc == FSB_OK) {
    cudaEventRecord(a, s);
    rc = fsb_step(h, n_steps, nullptr);
    cudaEventRecord(b, s);
  }
  float ms = 0.f;
  if (rc == FSB_OK && cudaEventSynchronize(b) == cudaSuccess &&
      cudaEventElapsedTime(&ms, a, b) == cudaSuccess)
    *ms_out = ms;
  else if (rc == FSB_OK)
    rc = FSB_ERR_CUDA;
  if (a) cudaEventDestroy(a);
  if (b) cudaEventDestroy(b);
  const int rc2 = fsb_destroy(h);
  return rc != FSB_OK ? rc : rc2;
}

}  // namespace

extern "C" int fsb_autotune(const fsb_config* cfg, uint32_t n_steps, int* best_path,
                            fsb_tuning* best_tuning, double* best_fish_steps_per_s,
                            uint32_t* candidates_tried) {
  if (!cfg || !best_path || !best_tuning) return fsb::record_error(FSB_ERR_INVALID_ARG, "NULL");
  if (n_steps == 0) return fsb::record_error(FSB_ERR_INVALID_ARG, "n_steps must be >= 1");
  if (cfg->collective_mode != 0)
    return fsb::record_error(FSB_ERR_UNSUPPORTED, "the collective passes have one launch shape");
  const bool dbl = cfg->precision == FSB_FP64_STATE;
  std::vector<Candidate> cands;
  const int blocks[] = {256, 512};
  const int minbs[] = {0, 3, 4};
  for (int b : blocks)
    for (int m : minbs) {  // vector-load kernel
      if (m && (b != 256 || dbl)) continue;
      Candidate c{};
      c.path = FSB_PATH_STREAM;
      c.t.stream_kernel = 1;
      c.t.stream_block = b;
      c.t.stream_blocks_per_sm = m;
      cands.push_back(c);
    }
  if (!dbl)
    for (int k = 2; k <= 3; ++k)  // bulk-copy ring, block-synchronised or warp-specialised
      for (int b : blocks)
        for (int st = 2; st <= (k == 2 ? 4 : 3); ++st) {
          Candidate c{};
          c.path = FSB_PATH_STREAM;
          c.t.stream_kernel = k;
          c.t.stream_block = b;
          c.t.stream_stages = st;
          cands.push_back(c);
        }
  if (!dbl && cfg->swim_mode == 0) {
    const int ks[] = {4, 8};
    for (int kernel : {4, 5})  // steps blocked by recompute; 5: positions kept
      for (int k : ks) {
        Candidate c{};
        c.path = FSB_PATH_STREAM;
        c.t.stream_kernel = kernel;
        c.t.stream_block_steps = k;
        cands.push_back(c);
      }
  }
  if (!dbl) {
    const int fpts[] = {4, 8, 12, 16};
    for (int f : fpts) {
      Candidate c{};
      c.path = FSB_PATH_RESIDENT;
      c.t.resident_fpt = f;
      cands.push_back(c);
    }
  }
  cudaStream_t s = nullptr;
  if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess)
    return fsb::record_error(FSB_ERR_CUDA, "fsb_autotune: stream creation failed");
  double best_ms = -1.0;
  uint32_t tried = 0;
  for (const Candidate& c : cands) {
    double ms = 0.0;
    const int rc = time_candidate(cfg, c, n_steps, s, &ms);
    if (rc == FSB_ERR_CUDA || rc == FSB_ERR_OOM) {
      cudaStreamDestroy(s);
      return rc;
    }
    if (rc != FSB_OK) continue;  // shape not available for this size
    ++tried;
    if (best_ms < 0.0 || ms < best_ms) {
      best_ms = ms;
      *best_path = c.path;
      *best_tuning = c.t;
    }
  }
  cudaStreamDestroy(s);
  if (best_ms < 0.0)
    return fsb::record_error(FSB_ERR_UNSUPPORTED, "fsb_autotune: no launch shape could run");
  if (best_fish_steps_per_s)
    *best_fish_steps_per_s = static_cast<double>(cfg->n_fish) * n_steps / (best_ms * 1e-3);
  if (candidates_tried) *candidates_tried = tried;
  return FSB_OK;
}

extern "C" int fsb_autotune_batch(const fsb_config* tmpl, uint32_t n_schools,
                                  const uint64_t* offsets, const uint64_t* seeds,
                                  const fsb_state_dev* state, uint32_t n_steps, int* best_cluster,
                                  double* best_fish_steps_per_s) {
  if (!tmpl || !offsets || !seeds || !state || !best_cluster || n_steps == 0)
    return fsb::record_error(FSB_ERR_INVALID_ARG, "fsb_autotune_batch: bad argument");
  cudaStream_t s = nullptr;
  if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess)
    return fsb::record_error(FSB_ERR_CUDA, "fsb_autotune_batch: stream creation failed");
  double best_ms = -1.0;
  const int clusters[] = {0, 1, 2, 4, 8};  // 0: each school on the smallest cluster that holds it
  for (int c : clusters) {
    fsb_batch_handle b = nullptr;
    int rc = fsb_batch_create(tmpl, n_schools, offsets, seeds, state, 1, 0, s, &b);
    if (rc != FSB_OK) {
      cudaStreamDestroy(s);
      return rc;
    }
    rc = fsb_batch_set_cluster(b, c);
    if (rc == FSB_OK) rc = fsb_batch_step(b, n_steps, nullptr);  // warm-up (+ init)
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    float ms = -1.f;
    if (rc == FSB_OK && cudaEventCreate(&e0) == cudaSuccess &&
        cudaEventCreate(&e1) == cudaSuccess) {
      cudaEventRecord(e0, s);
      rc = fsb_batch_step(b, n_steps, nullptr);
      cudaEventRecord(e1, s);
      if (rc == FSB_OK && cudaEventSynchronize(e1) == cudaSuccess)
        cudaEventElapsedTime(&ms, e0, e1);
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    fsb_batch_destroy(b);
    if (rc == FSB_OK && ms > 0.f && (best_ms < 0.0 || ms < best_ms)) {
      best_ms = ms;
      *best_cluster = c;
    }
  }
  cudaStreamDestroy(s);
  if (best_ms < 0.0)
    return fsb::record_error(FSB_ERR_UNSUPPORTED, "fsb_autotune_batch: no cluster size ran");
  if (best_fish_steps_per_s)
    *best_fish_steps_per_s = static_cast<double>(offsets[n_schools]) * n_steps / (best_ms * 1e-3);
  return FSB_OK;
}
