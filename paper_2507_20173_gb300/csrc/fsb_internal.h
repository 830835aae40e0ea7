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

// Control block of one resident launch; zeroed before every launch.
struct alignas(16) ResCtl {
  unsigned bar_count;     // grid-barrier arrivals (monotonic within a launch)
  unsigned max_slot[3];   // rotating per-step slots: bits of max |delta|
  unsigned ekey_slot[3];  // rotating per-step slots: order key of max(prev-cur)
  unsigned spare;
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
  int tma;          // 1: bulk-copy ring (fsb_stream_tma.cu); 2: warp-specialised
                    //    ring (fsb_stream_ws.cu)
  int min_blocks;   // vector kernel: blocks per SM its register budget guarantees
  int stages;       // bulk-copy kernel: tiles in flight per block (2, 3, 4; 0 = 2)
  double pond_half, step, w0, w_min, w_max;
  int swim_mode, feed_mode;
  Ctl* ctl;
  BlockPartial* partials;
  fsb_step_stats* ring;
  uint32_t ring_cap;
  int blocked_k = 0;                   // stream kernels 4, 5: steps per pair of passes (2, 4, 8)
  int bgrid = 0;                       //   their grid
  BlockPartial* bpartials = nullptr;   //   their per-step partials, blocked_k x bgrid
  float* slots = nullptr;              // stream kernel 5: positions of the pair's steps,
  uint64_t slot_stride = 0;            //   x and y of step t at slots + (2t, 2t + 1) * stride
  unsigned long long timeout_ns = 0;  // bound of the copy rings' waits (0: 1 s)
  int inject_block = -1;               // test hook (copy-ring kernels): block that withholds
  uint32_t inject_pass = 0;            //   its first copy in this pass of a call; -1 = none
};

cudaError_t launch_stream_pass(const StreamLaunch& L, int pass_kind, cudaStream_t s);
// Bulk-copy-fed variant (binary32, 16-byte aligned state, block 256 or 512).
bool stream_tma_supported(const StreamLaunch& L);
cudaError_t stream_tma_prepare(const StreamLaunch& L);
int stream_tma_blocks_per_sm(const StreamLaunch& L);
cudaError_t launch_stream_pass_tma(const StreamLaunch& L, int pass_kind, cudaStream_t s);
// Warp-specialised ring (fsb_stream_ws.cu): L.block consumer threads plus one
// producer warp per block; stages 2 or 3.
cudaError_t stream_ws_prepare(const StreamLaunch& L);
int stream_ws_blocks_per_sm(const StreamLaunch& L);
cudaError_t launch_stream_pass_ws(const StreamLaunch& L, int pass_kind, cudaStream_t s);
cudaError_t launch_init(const StreamLaunch& L, int weight_mode, cudaStream_t s);
// Stream kernels 4 and 5 (fsb_stream_blocked.cu): a pair of passes
// advancing k <= L.blocked_k steps, the maxima pass and then the step pass
// (binary32, 16-byte aligned state, default swim); kernel 5 (L.slots set)
// keeps the maxima pass's positions for the step pass.
bool stream_blocked_supported(const StreamLaunch& L);
int stream_blocked_blocks_per_sm(const StreamLaunch& L);
cudaError_t launch_blocked_pair(const StreamLaunch& L, uint32_t k, cudaStream_t s);

// ---- collective movements (collective_mode 1, fsb_collective.cu)
// A call of n steps runs pass 0 (kCSwim0), then for t = 1 .. n the passes
// 2t - 1 (kCEat) and 2t (kCMove, kCMoveLast for t = n).
enum CollPassKind : int { kCSwim0 = 0, kCEat = 1, kCMove = 2, kCMoveLast = 3 };

// One block's contribution to a collective pass's reductions.
struct alignas(16) CollPartial {
  unsigned long long max_bits, e_key;
  double sum_w, sum_wx, sum_wy;
  long long q[4];  // exact grid sums
};

// The collective quantities of one step of a call (index t - 1 for step t).
struct alignas(16) CollRec {
  long long w_before;  // the school's weight on the grid before the step's eat
  long long sw;        // ... after it
  double ix, iy;       // instinctive vector
  double bx, by;       // barycentre of the volitive move
  int has_b;           // sw != 0: a barycentre exists
  int contract;        // sw > w_before: the school moves toward it
};

struct CollLaunch {
  void* x;
  void* y;
  void* w;
  void* pv;
  uint64_t n;
  uint64_t seed;
  uint32_t school;
  int real_is_double;
  int acc;
  int grid;
  double pond_half, step, w0, w_min, w_max, step_vol;
  int swim_mode, feed_mode;
  int kp, kg, kw;      // grid exponents of the exact sums
  Ctl* ctl;
  CollPartial* partials;
  fsb_step_stats* ring;
  CollRec* coll;
};

int coll_grid(const CollLaunch& L, int sms);
cudaError_t launch_coll_pass(const CollLaunch& L, int pass_kind, uint32_t n_steps,
                             cudaStream_t s);
// currentObjective of fish [first, first + count) into cur[0, count).
cudaError_t launch_objective(const StreamLaunch& L, uint64_t first, uint64_t count, void* cur,
                             cudaStream_t s);
// State transfers done by the SMs (fsb_transfer.cu).  host_view: the
// device-visible address of pinned (or registered) host memory, else null.
// launch_read_out: the device state into host arrays out[0..4] (x, y, w,
// prevObjective, currentObjective -- computed on the way; null ones
// skipped), all device-visible.  launch_copy_in: host arrays in[0..3] (x, y,
// w, prevObjective), all device-visible, into the device state.
void* host_view(const void* p);
cudaError_t launch_read_out(const StreamLaunch& L, void* const out[5], cudaStream_t s);
cudaError_t launch_copy_in(const StreamLaunch& L, const void* const in[4], cudaStream_t s);
// Launch description of the resident single-school kernel (binary32 state).
struct ResidentLaunch {
  void* x;
  void* y;
  void* w;
  void* pv;
  uint64_t n;
  uint64_t slice;   // fish per block
  uint64_t seed;
  uint32_t school;
  double pond_half, step, w0, w_min, w_max;
  int swim_mode;    // 1: weight-scaled swim (swims each step after the eat)
  int feed_mode;
  int acc;          // AccMode
  int fpt;          // at most this many fish per thread: 4, 8, 12 or 16
  int block;        // fish threads per block (<= resident_max_block(fpt); one
                    // synchronisation warp more is launched);
                    // slice <= resident_max_slice(fpt, block)
  int grid;         // blocks, all co-resident (cooperative launch)
  uint64_t base_step;
  uint32_t n_steps;
  Ctl* ctl;
  ResCtl* rctl;
  double* sums;     // n_steps * grid * 3 barycentre partials
  fsb_step_stats* ring;
  unsigned long long timeout_ns;
  int inject_cta;   // test hook: this block skips one barrier arrival (-1 none)
  uint32_t inject_step;
};

cudaError_t launch_resident(const ResidentLaunch& L, cudaStream_t s);
int resident_max_block(int fpt);
uint64_t resident_max_slice(int fpt, int block);
int resident_blocks_per_sm(int fpt, int acc, int block, int swim_mode, double step);
size_t resident_smem_bytes(uint64_t slice);

// Work queues of a batch: queue t (t = 0 .. 6) holds the schools run on
// whole clusters of 8 - t blocks, queue 7 the schools one block runs, and
// queues 8 .. 11 the schools packed several to a block, each on a team of
// 8, 4, 2 or 1 fish warps (up to 8, 4, 2 or 1 times batch_team_fish());
// each queue largest first.  One counter per queue, zeroed before every
// call.
constexpr int kMaxBatchCluster = 8;  // widest cluster of a batch (portable limit)
constexpr int kBatchSingleQueue = kMaxBatchCluster - 1;
constexpr int kBatchPackQueue0 = kMaxBatchCluster;  // teams of 8 warps; then 4, 2, 1
constexpr int kBatchPackLevels = 4;
constexpr int kBatchQueues = kMaxBatchCluster + kBatchPackLevels;
constexpr int kBatchMaxLaunches = kMaxBatchCluster;
struct alignas(16) BatchCtl {
  unsigned next[kBatchQueues];
  int status;     // debug build: a failed invariant check (FSB_ERR_STATE)
  unsigned site;  // ... and where
};

// Queue of the schools that need clusters of c blocks (c = 1 .. 8).
inline int batch_queue_of(int c) { return c >= 8 ? 0 : (c <= 1 ? 7 : 8 - c); }
// Queue of the schools packed on teams of `warps` (8, 4, 2, 1) fish warps.
inline int batch_pack_queue_of(int warps) {
  return kBatchPackQueue0 + (warps >= 8 ? 0 : warps >= 4 ? 1 : warps >= 2 ? 2 : 3);
}

// Launch description of the batched (many schools) kernel, binary32 state.
struct BatchLaunch {
  void* x;
  void* y;
  void* w;
  void* pv;
  const unsigned long long* offsets;  // device, n_schools + 1
  const unsigned long long* seeds;    // device, n_schools
  const uint32_t* order;              // device, queues 0..11 back to back
  uint32_t queue_lo[kBatchQueues + 1];  // queue t is order[queue_lo[t] .. queue_lo[t + 1])
  uint32_t n_schools;
  double pond_half, step, w0, w_min, w_max;
  int swim_mode, feed_mode;
  int acc;
  int init;
  int weight_mode;
  const unsigned long long* base_step;  // device: step counter at the start of the launch
  uint32_t n_steps;
  BatchCtl* bctl;
  fsb_step_stats* stats;              // device, n_schools * n_steps
  // Concurrent persistent launches, largest cluster first.  Launch i runs
  // clusters of cluster[i] blocks on a grid of blocks[i]: it takes whole-
  // cluster schools from queue batch_queue_of(cluster[i]) and then from the
  // queues of smaller clusters, then single-block schools one block at a
  // time (queue 7), and finally packed schools, each team of warps on its
  // own (queues 8 .. 11).
  int n_launches;
  int cluster[kBatchMaxLaunches];
  int blocks[kBatchMaxLaunches];
};

// Zeroes the work-list counters, then enqueues launch 0 on `s` and launches
// 1.. on side[0..] (forked from and joined back into `s` through `fork` and
// join[0..]).
cudaError_t launch_batch(const BatchLaunch& L, cudaStream_t s, const cudaStream_t* side,
                         cudaEvent_t fork, const cudaEvent_t* join);
// The batch kernels for clusters of 5 to 8 blocks (fsb_batch_wide.cu).
const void* batch_kernel_wide(int cluster, int acc, bool var);
int batch_max_clusters(int cluster, int acc);
uint64_t batch_block_capacity();
// Fish one fish warp holds when schools are packed on teams of warps (0:
// the batch kernel was built without packing).
uint64_t batch_team_fish();
// Host side: completes the barycentre sums of `count` records copied out of
// the batch kernel's statistics (raw partials of accumulation mode acc).
void batch_finish_stats(fsb_step_stats* st, size_t count, int acc);
int batch_threads();
cudaError_t launch_bump_step(unsigned long long* base_step, uint32_t n, cudaStream_t s);

// Reduction constructs of the stand-alone eat() reduction.
enum EatConstruct : int { kEatHierarchical = 0, kEatPerWarp = 1, kEatPerFish = 2 };
cudaError_t launch_eat_max(const float* prev, const float* cur, uint64_t n, int construct,
                           unsigned* key, double* value, int grid, cudaStream_t s);

// Record `msg` as the calling thread's fsb_last_error() detail; returns status.
int record_error(int status, const char* msg);
// Occupancy-derived blocks per SM for the fused pass of this configuration.
int stream_blocks_per_sm(const StreamLaunch& L);

}  // namespace fsb
