// fsb_internal.h -- declarations shared by the library's translation units.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/fsb.h"

namespace fsb {

// Device-side control word of one school (or one batch launch).
struct alignas(16) Ctl {
  unsigned long long base_step;  // step counter t at the start of the call
  unsigned int pass;             // pass index within the current call
  unsigned int arrive;           // grid-reduction arrival counter
  int status;                    // latched device error (fsb_status), 0 = ok
  unsigned int timeout_site;     // where a bounded wait gave up (diagnostic)
  unsigned long long spare;
};

// One block's contribution to a step's reductions.
struct alignas(16) BlockPartial {
  unsigned long long max_bits;   // bit pattern of max |delta| (non-negative)
  unsigned long long e_key;      // order key of max (prev - cur)
  double sum_w, sum_wx, sum_wy;
  double spare;
};

enum PassKind : int { kSwimOnly = 0, kFused = 1, kSettle = 2 };
enum AccMode : int { kAccPlain32 = 0, kAccKahan32 = 1, kAccF64 = 2 };

// Launch description for one streaming pass.
struct StreamLaunch {
  void* x;
  void* y;
  void* w;
  void* pv;
  uint64_t n;
  uint64_t seed;
  uint32_t school;
  int real_is_double;
  int acc;          // AccMode
  int vec;          // 1 or vector width
  int block;        // threads per block
  int grid;         // blocks
  double pond_half, step, w0, w_min, w_max;
  Ctl* ctl;
  BlockPartial* partials;
  fsb_step_stats* ring;
  uint32_t ring_cap;
};

cudaError_t launch_stream_pass(const StreamLaunch& L, int pass_kind, cudaStream_t s);
cudaError_t launch_init(const StreamLaunch& L, int weight_mode, cudaStream_t s);
cudaError_t launch_objective(const StreamLaunch& L, void* cur, cudaStream_t s);
// Record `msg` as the calling thread's fsb_last_error() detail; returns status.
int record_error(int status, const char* msg);
// Occupancy-derived blocks per SM for the fused pass of this configuration.
int stream_blocks_per_sm(const StreamLaunch& L);

}  // namespace fsb
