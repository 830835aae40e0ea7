// fsb_noalloc.cu -- fsb_step_static: the streaming step without any device
// allocation.
//
// Some callers cannot let a library allocate device memory at call time: a
// host application that carves all GPU memory into its own arena at start-up
// and forbids later cudaMalloc, or a real-time pipeline in which cudaMalloc /
// cudaFree (which may synchronise the whole device) would stall its other
// streams.  For them this entry point runs the same fused streaming kernels as
// fsb_step, but keeps the kernels' scratch (the control word, one reduction
// partial per block and the per-step statistics ring) in a fixed, file-scope
// __device__ array instead of memory owned by a handle.  The caller passes the
// state arrays and the statistics output; nothing is allocated.
//
// Limits and sharing:
//   - the array is kStaticScratchBytes (about 210 KB) on every GPU that loads
//     the library, held until the process exits;
//   - one call advances at most kStaticMaxSteps steps (statistics ring) and
//     uses at most kStaticMaxBlocks blocks (reduction partials; the grid is
//     capped to that, the grid-stride loop covers any school size);
//   - every call on a device shares the one array, and each call rewrites the
//     control word first, so calls whose kernels overlap on the GPU (two
//     streams, or two host threads) race and give wrong results: serialise
//     them, e.g. on one stream.
//
// Errors found on the device (a status the kernels latch in the control word)
// cannot be returned by an asynchronous call.  The next call's first kernel
// keeps such a status in a carried slot of the array instead of clearing it,
// and the first later call that synchronises (one given host memory for its
// statistics) returns it, together with its own, and clears both.
#include <cstdint>
#include <cstdio>
#include <mutex>

#include <cuda_runtime.h>

#include "fsb_internal.h"

namespace fsb {
namespace {

constexpr uint32_t kStaticMaxSteps = 4096;
constexpr uint32_t kStaticMaxBlocks = 1024;
constexpr size_t kCtlBytes = 256;  // the control word, the carried status, the report slot
constexpr size_t kCarriedOffset = 64;
constexpr size_t kReportOffset = 128;
constexpr size_t kPartialBytes = sizeof(BlockPartial) * kStaticMaxBlocks;
constexpr size_t kRingBytes = sizeof(fsb_step_stats) * kStaticMaxSteps;
constexpr size_t kStaticScratchBytes = kCtlBytes + kPartialBytes + kRingBytes;
constexpr int kMaxDevices = 64;

static_assert(sizeof(Ctl) <= kCarriedOffset, "control word does not fit its slot");
static_assert(kPartialBytes % 256 == 0, "ring must stay 256-byte aligned");

// The shared scratch.  In host code `g_static_scratch` names a host-side
// stand-in, not device memory: host code must use the address returned by
// cudaGetSymbolAddress on the device in question.
__device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

// Resets the control word at the start of every call (the array keeps the
// previous call's contents).  A status the previous call latched is kept in
// the carried slot until a synchronising call reports it.
__global__ void reset_ctl_kernel(Ctl* ctl, int* carried, unsigned long long start_step) {
  if (*carried == 0) *carried = ctl->status;
  Ctl c{};
  c.base_step = start_step;
  *ctl = c;
}

// End of a synchronising call: the first error latched since the last report
// (an earlier call's, else this call's) goes to the report slot, and both
// slots are cleared.
__global__ void take_status_kernel(Ctl* ctl, int* carried, int* report) {
  *report = *carried != 0 ? *carried : ctl->status;
  *carried = 0;
  ctl->status = 0;
}

std::mutex g_setup_mutex;
void* g_scratch_addr[kMaxDevices] = {};

int fail(int status, const char* msg, cudaError_t e = cudaSuccess) {
  char buf[256];
  if (e != cudaSuccess)
    std::snprintf(buf, sizeof(buf), "%s: %s", msg, cudaGetErrorString(e));
  else
    std::snprintf(buf, sizeof(buf), "%s", msg);
  return record_error(status, buf);
}

// Once per device, with that device current: the device address of the
// scratch array.
int scratch_address(int device, void** out) {
  if (device < 0 || device >= kMaxDevices)
    return fail(FSB_ERR_UNSUPPORTED, "fsb_step_static: device ordinal out of range");
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (!g_scratch_addr[device]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
    if (e != cudaSuccess || !p)
      return fail(FSB_ERR_CUDA, "fsb_step_static: cudaGetSymbolAddress failed", e);
    g_scratch_addr[device] = p;
  }
  *out = g_scratch_addr[device];
  return FSB_OK;
}

bool aligned(const void* p, size_t a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; }

}  // namespace
}  // namespace fsb

extern "C" int fsb_step_static(const fsb_config* cfg, const fsb_state_dev* state,
                               uint64_t start_step, uint32_t n_steps,
                               fsb_step_stats* stats_out, void* cuda_stream) {
  using namespace fsb;
  if (!cfg || !state) return fail(FSB_ERR_INVALID_ARG, "fsb_step_static: NULL argument");
  if (cfg->n_fish == 0) return fail(FSB_ERR_INVALID_ARG, "fsb_step_static: n_fish must be >= 1");
  if (!(cfg->pond_half > 0.0) || !(cfg->step >= 0.0) || !(cfg->w_min <= cfg->w_max) ||
      cfg->precision < FSB_FP32 || cfg->precision > FSB_FP64_STATE ||
      (cfg->swim_mode != 0 && cfg->swim_mode != 1) || (cfg->feed_mode != 0 && cfg->feed_mode != 1) ||
      (cfg->swim_mode == 1 && !(cfg->w0 > 0.0)))
    return fail(FSB_ERR_INVALID_ARG, "fsb_step_static: invalid configuration");
  if (n_steps == 0) return fail(FSB_ERR_INVALID_ARG, "fsb_step_static: n_steps must be >= 1");
  if (cfg->collective_mode != 0)
    return fail(FSB_ERR_UNSUPPORTED, "fsb_step_static: the collective movements need fsb_step");
  if (n_steps > kStaticMaxSteps)
    return fail(FSB_ERR_INVALID_ARG,
                "fsb_step_static: n_steps exceeds the static scratch limit of 4096 steps "
                "per call; split the call");
  if (start_step > 0xFFFFFFFFull - n_steps)
    return fail(FSB_ERR_INVALID_ARG, "fsb_step_static: step counter would pass 2^32 - 1");
  const bool dbl = cfg->precision == FSB_FP64_STATE;
  const size_t elem = dbl ? 8 : 4;
  const void* p[4] = {state->x, state->y, state->w, state->prev_objective};
  for (const void* q : p)
    if (!q || !aligned(q, elem))
      return fail(FSB_ERR_INVALID_ARG, "fsb_step_static: state array NULL or misaligned");

  int device = 0;
  cudaError_t e = cudaGetDevice(&device);
  if (e != cudaSuccess) return fail(FSB_ERR_CUDA, "fsb_step_static: cudaGetDevice", e);
  void* base = nullptr;
  int rc = scratch_address(device, &base);
  if (rc != FSB_OK) return rc;
  unsigned char* scratch = static_cast<unsigned char*>(base);

  StreamLaunch L{};
  L.x = state->x;
  L.y = state->y;
  L.w = state->w;
  L.pv = state->prev_objective;
  L.n = cfg->n_fish;
  L.seed = cfg->seed;
  L.school = cfg->school_id;
  L.real_is_double = dbl ? 1 : 0;
  L.acc = cfg->precision == FSB_FP32 ? kAccPlain32
          : cfg->precision == FSB_FP32_KAHAN ? kAccKahan32 : kAccF64;
  const bool vec_ok = aligned(L.x, 16) && aligned(L.y, 16) && aligned(L.w, 16) &&
                      aligned(L.pv, 16);
  L.vec = vec_ok ? (dbl ? 2 : 4) : 1;
  // fsb_step's default streaming shape: 256 threads, and for aligned binary32
  // state the copy compiled for four blocks per SM (64 registers)
  L.block = 256;
  L.min_blocks = (!dbl && L.vec == 4) ? 4 : 1;
  L.pond_half = cfg->pond_half;
  L.step = cfg->step;
  L.w0 = cfg->w0;
  L.w_min = cfg->w_min;
  L.w_max = cfg->w_max;
  L.swim_mode = cfg->swim_mode;
  L.feed_mode = cfg->feed_mode;
  L.ctl = reinterpret_cast<Ctl*>(scratch);
  L.partials = reinterpret_cast<BlockPartial*>(scratch + kCtlBytes);
  L.ring = reinterpret_cast<fsb_step_stats*>(scratch + kCtlBytes + kPartialBytes);
  L.ring_cap = kStaticMaxSteps;

  int sms = 0;
  e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
  if (e != cudaSuccess) return fail(FSB_ERR_CUDA, "fsb_step_static: device attribute", e);
  int per_sm = stream_blocks_per_sm(L);
  if (per_sm < 1) per_sm = 1;
  const uint64_t groups = (cfg->n_fish + L.vec - 1) / L.vec;
  uint64_t grid = (groups + L.block - 1) / L.block;
  const uint64_t full = static_cast<uint64_t>(sms) * per_sm;
  if (grid > full) grid = full;
  if (grid > kStaticMaxBlocks) grid = kStaticMaxBlocks;
  L.grid = static_cast<int>(grid < 1 ? 1 : grid);

  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  int* carried = reinterpret_cast<int*>(scratch + kCarriedOffset);
  int* report = reinterpret_cast<int*>(scratch + kReportOffset);
  // host statistics make the call synchronous, and it then reports the
  // device status (device or managed statistics keep it asynchronous)
  bool host_stats = false;
  if (stats_out) {
    cudaPointerAttributes pa{};
    e = cudaPointerGetAttributes(&pa, stats_out);
    if (e != cudaSuccess) return fail(FSB_ERR_INVALID_ARG, "fsb_step_static: stats_out", e);
    host_stats = pa.type == cudaMemoryTypeHost || pa.type == cudaMemoryTypeUnregistered;
  }
  reset_ctl_kernel<<<1, 1, 0, s>>>(L.ctl, carried, start_step);
  e = cudaGetLastError();
  if (e != cudaSuccess) return fail(FSB_ERR_CUDA, "fsb_step_static: control reset", e);
  e = launch_stream_pass(L, kSwimOnly, s);
  for (uint32_t k = 1; e == cudaSuccess && k < n_steps; ++k) e = launch_stream_pass(L, kFused, s);
  if (e == cudaSuccess) e = launch_stream_pass(L, kSettle, s);
  if (e != cudaSuccess) return fail(FSB_ERR_CUDA, "fsb_step_static: kernel launch", e);
  if (stats_out) {
    e = cudaMemcpyAsync(stats_out, L.ring, sizeof(fsb_step_stats) * n_steps, cudaMemcpyDefault,
                        s);
    if (e != cudaSuccess) return fail(FSB_ERR_CUDA, "fsb_step_static: statistics copy", e);
  }
  if (!host_stats) return FSB_OK;
  take_status_kernel<<<1, 1, 0, s>>>(L.ctl, carried, report);
  e = cudaGetLastError();
  int status = 0;
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(&status, report, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return fail(FSB_ERR_CUDA, "fsb_step_static: status read", e);
  if (status != 0) {
    char buf[128];
    std::snprintf(buf, sizeof(buf), "fsb_step_static: device status word latched %d", status);
    return record_error(status, buf);
  }
  return FSB_OK;
}
