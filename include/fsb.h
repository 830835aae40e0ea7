/*
 * fsb.h -- C ABI of the GB300 Fish School Behaviour library (libfsb.so).
 *
 * The library advances fish schools by the per-step update of the Fish School
 * Behaviour simulation (arxiv 2507.20173): random swim inside the pond
 * (Sec. 2.1.2), objective = Euclidean distance to the pond centre
 * (Sec. 2.1.1), delta of the objective, a max reduction over the school
 * (the eat() reduction of Sec. 2.3.2), feeding normalised by that max and
 * capped, and the school's barycentre sums.  Where the paper leaves a rule
 * unwritten, the reading used is stated at the declaration that relies on it.
 *
 * Conventions for every entry point:
 *   - Return value: FSB_OK (0) or a negative fsb_status.  fsb_strerror()
 *     names a status; fsb_last_error() gives a human-readable detail of the
 *     last failure on the calling thread.
 *   - Device pointers are plain CUDA device addresses (e.g. a torch tensor's
 *     data_ptr()).  Host pointers are plain host addresses; pinned memory is
 *     faster but not required.
 *   - Streams are cudaStream_t passed as void*; NULL means the legacy default
 *     stream.  Calls are asynchronous on the handle's stream unless stated
 *     otherwise.
 *   - No entry point may be called while its stream is being captured into a
 *     CUDA graph by the caller (the library captures its own graphs).
 *   - One GPU: the device current at fsb_create is the device of the handle.
 *   - Nothing here falls back to the CPU: without a usable CUDA device every
 *     call that computes returns FSB_ERR_CUDA.
 */
#ifndef FSB_H
#define FSB_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    FSB_OK = 0,
    FSB_ERR_INVALID_ARG = -1,  /* bad pointer, size, enum or config value   */
    FSB_ERR_CUDA = -2,         /* a CUDA runtime call failed                 */
    FSB_ERR_OOM = -3,          /* device or pinned allocation failed         */
    FSB_ERR_UNSUPPORTED = -4,  /* valid request this library cannot serve    */
    FSB_ERR_TIMEOUT = -5,      /* a bounded device-side wait gave up         */
    FSB_ERR_STATE = -6         /* device status word latched an error        */
} fsb_status;

/* Arithmetic of the state and of the barycentre sums.
 *   FSB_FP32        binary32 state; plain binary32 sums (precision baseline)
 *   FSB_FP32_KAHAN  binary32 state; compensated binary32 sums, combined in
 *                   binary64 (default).  The streaming kernels compensate
 *                   each thread's running sums (Kahan); in the on-chip
 *                   kernels a thread adds at most eight fish pairs per step
 *                   in plain binary32 and compensation starts at the warp
 *   FSB_FP64_ACC    binary32 state; binary64 sums of exact products
 *   FSB_FP64_STATE  binary64 state and arithmetic; binary64 sums
 * In every binary32 mode the per-fish state is bit-identical; only the sums
 * differ. */
typedef enum {
    FSB_FP32 = 0,
    FSB_FP32_KAHAN = 1,
    FSB_FP64_ACC = 2,
    FSB_FP64_STATE = 3
} fsb_precision;

/* Which kernel family advances a single school.
 *   FSB_PATH_STREAM    one fused HBM-streaming pass per step
 *   FSB_PATH_RESIDENT  state held on chip for all steps of a call
 *   FSB_PATH_AUTO      the library picks (autotune table, else size cutoff) */
typedef enum {
    FSB_PATH_AUTO = 0,
    FSB_PATH_STREAM = 1,
    FSB_PATH_RESIDENT = 2
} fsb_path;

/* School configuration: the physics fields of the paper's Config struct
 * (Sec. 2.1.3: fish population, initial weight, pond dimensions) plus the
 * generator key and the arithmetic mode.  Use fsb_config_init() for the
 * defaults below.
 *   n_fish            >= 1
 *   seed              Philox4x32-10 key = (seed lo32, seed hi32)
 *   school_id         XORed into counter word 1 (distinguishes schools)
 *   init_weight_mode  0: w = w0 (default); 1: w = w0 * (0.5 + u), u uniform
 *                     in [0,1) from the init draw (the paper says the weight
 *                     comes from the generator, Sec. 2.1.1, yet Config holds
 *                     one initial weight, Sec. 2.1.3)
 *   pond_half         P: the pond is [-P, P]^2 (200x200 -> 100, Sec. 2.1.2)
 *   step              s: each coordinate moves by (2u - 1) * s per step
 *                     (default 0.1; the paper gives no step size)
 *   w0, w_min, w_max  initial weight 1, floor 0, cap 2 (cap = 2 w0)
 *   precision         fsb_precision
 *   path              fsb_path (ignored by fsb_run_batch)
 *   swim_mode         0 (default): each coordinate moves by (2u - 1) * s;
 *                     1: by (2u - 1) * ((w / w0) * s) with the fish's weight
 *                     before the step's eat -- a reading of the paper's
 *                     weight-dependent mobility (Sec. 2.1.1, 2.1.2); a fish
 *                     of weight 0 stays put.  Every path runs it.
 *   feed_mode         0 (default): w += delta / max|delta|;
 *                     1: w += (prev - cur) / E with E = max(prev - cur), the
 *                     value the paper's eat() reduces (Sec. 2.3.2); nobody
 *                     eats when E <= 0
 *   collective_mode   0 (default); 1: after each step's eat, the two
 *                     collective movements of fish-school search (not in
 *                     the paper): every fish moves by the instinctive vector
 *                     (the improvement-weighted mean swim displacement of
 *                     the fish that improved), then by step_vol * u along
 *                     the line through the school's barycentre, toward it if
 *                     the school's weight grew in the step, away otherwise.
 *                     Those school sums are exact fixed-point sums, so the
 *                     result does not depend on the reduction order.
 *                     Streaming path only (fsb_create with FSB_PATH_RESIDENT,
 *                     fsb_run_batch / fsb_batch_create, fsb_step_static,
 *                     fsb_autotune and fsb_set_fault_injection return
 *                     FSB_ERR_UNSUPPORTED); two passes per step
 *   step_vol          volitive step (default 0.1)                          */
typedef struct {
    uint64_t n_fish;
    uint64_t seed;
    uint32_t school_id;
    int32_t  init_weight_mode;
    double   pond_half;
    double   step;
    double   w0;
    double   w_min;
    double   w_max;
    int32_t  precision;
    int32_t  path;
    int32_t  swim_mode;
    int32_t  feed_mode;
    int32_t  collective_mode;
    double   step_vol;
} fsb_config;

/* Per-fish state arrays on the device, structure of arrays, n_fish elements
 * each, element type float (binary32 modes) or double (FSB_FP64_STATE):
 *   x, y            position (Sec. 2.1.1)
 *   w               weight
 *   prev_objective  prevObjective of the paper's Fish record: the objective
 *                   before the latest swim.  currentObjective is not stored:
 *                   it is sqrt(x*x + y*y) of the stored position, and
 *                   fsb_read_state recomputes it on the device.
 * Base addresses must be aligned to the element size; 16-byte alignment
 * enables the vectorised path. */
typedef struct {
    void* x;
    void* y;
    void* w;
    void* prev_objective;
} fsb_state_dev;

/* The same four arrays in host memory (resume / checkpoint input). */
typedef struct {
    const void* x;
    const void* y;
    const void* w;
    const void* prev_objective;
} fsb_state_host;

/* Statistics of one step t.
 *   max_abs_delta  M_t = max_i |currentObjective_i - prevObjective_i|, the
 *                  normaliser of feeding; exact (it is one fish's |delta|)
 *   eat_max_diff   max_i (prevObjective_i - currentObjective_i): the value
 *                  the paper's eat() reduces (Sec. 2.3.2); exact
 *   sum_w, sum_wx, sum_wy
 *                  barycentre sums over post-swim positions and post-eat
 *                  weights of step t, accumulated as `precision` says;
 *                  barycentre = (sum_wx / sum_w, sum_wy / sum_w)            */
typedef struct {
    double max_abs_delta;
    double eat_max_diff;
    double sum_w;
    double sum_wx;
    double sum_wy;
} fsb_step_stats;

typedef struct fsb_school* fsb_handle;

/* Fill *cfg with the defaults: pond_half 100, step 0.1, w0 1, w_min 0,
 * w_max 2, init_weight_mode 0, precision FSB_FP32_KAHAN, path FSB_PATH_AUTO,
 * school_id 0.  Returns FSB_ERR_INVALID_ARG if cfg is NULL. */
int fsb_config_init(fsb_config* cfg, uint64_t n_fish, uint64_t seed);

/* Create a school on the current device and bind it to `cuda_stream`.
 *   cfg         validated: n_fish >= 1, P > 0, s >= 0, w_min <= w_max,
 *               known enums; else FSB_ERR_INVALID_ARG
 *   buffers     caller-owned device arrays (see fsb_state_dev) that must
 *               outlive the handle; NULL: the library allocates and owns them
 *   init        NULL: initialise by the method's own rule (Sec. 2.1.1: Philox
 *               position uniform over the pond, weight w0, prevObjective =
 *               currentObjective = distance to the centre).  Otherwise a
 *               host checkpoint copied to the device (resume)
 *   start_step  the step counter t of the state (0 for a fresh school; the
 *               value fsb_read_state reported when resuming)
 * On success *out holds the handle.  Library scratch (reduction partials,
 * the per-step statistics ring, the control word) is owned by the handle.
 * Asynchronous on cuda_stream. */
int fsb_create(const fsb_config* cfg, const fsb_state_dev* buffers,
               const fsb_state_host* init, uint64_t start_step,
               void* cuda_stream, fsb_handle* out);

/* Advance the school by n_steps steps (t -> t + n_steps), each step doing
 * swim, objective, delta, max, eat and barycentre in that order (Sec. 2.1.2,
 * Sec. 2.2.1, Sec. 2.3.2).  t + n_steps must stay below 2^32 (the step is a
 * 32-bit Philox counter word).
 *   host_stats  NULL, or room for n_steps records; when given the call
 *               synchronises the stream and fills them in step order
 * Returns FSB_ERR_INVALID_ARG for n_steps == 0 or counter overflow, and
 * FSB_ERR_TIMEOUT / FSB_ERR_STATE if a device-side wait gave up or the
 * device status word is set (checked when the call synchronises).
 * Asynchronous unless host_stats is given. */
int fsb_step(fsb_handle h, uint32_t n_steps, fsb_step_stats* host_stats);

/* Copy the school's state to host memory in the paper's field order
 * (Sec. 2.1.1): x, y, weight, prevObjective, currentObjective, each n_fish
 * elements of the state type; any pointer may be NULL to skip that field.
 * currentObjective is recomputed on the device from the stored position.
 * *step_out (may be NULL) receives the step counter t.  Synchronises the
 * stream; returns the latched device status, if any. */
int fsb_read_state(fsb_handle h, void* x, void* y, void* w,
                   void* prev_objective, void* current_objective,
                   uint64_t* step_out);

/* Copy the statistics of the last fsb_step call (n_steps records) into
 * host memory without running anything.  Synchronises the stream. */
int fsb_last_stats(fsb_handle h, fsb_step_stats* host_stats, uint32_t n_steps);

/* Release the handle and everything it owns (not caller buffers).
 * Synchronises the stream first.  NULL is accepted. */
int fsb_destroy(fsb_handle h);

/* ---- Batched schools (many independent fish schools in one launch) ----
 *
 * Each school is a separate fish school of the paper, advanced by the same
 * per-step update (Sec. 2.1.2 swim, Sec. 2.1.1 objective, delta, the
 * Sec. 2.3.2 max reduction, feeding, barycentre); a batch runs all of them
 * in one persistent launch of thread-block clusters that pop schools from a
 * largest-first work list over a ragged offset table and keep each school's
 * state on chip for all steps of a call.  The launch is captured in a CUDA
 * graph per call length and replayed.
 *
 *   tmpl        physics fields and precision shared by all schools
 *               (n_fish, seed, school_id and path are ignored); binary32
 *               precisions only (FSB_FP64_STATE -> FSB_ERR_UNSUPPORTED)
 *   n_schools   >= 1
 *   offsets     host array of n_schools + 1 increasing fish offsets,
 *               offsets[0] = 0; school k is fish [offsets[k], offsets[k+1])
 *               and holds >= 1 fish and at most 8 * block_fish = 90112 (a
 *               cluster of eight blocks, fsb_batch_limits; larger schools
 *               -> FSB_ERR_UNSUPPORTED, use fsb_create)
 *   seeds       host array of n_schools keys; school k uses key seeds[k] and
 *               school id k, so it reproduces a single-school run created
 *               with that seed and school_id = k
 *   state       device arrays (fsb_state_dev layout, binary32, 4-byte
 *               aligned) of offsets[n_schools] fish: the school states at
 *               step start_step; advanced in place; caller-owned
 *   init        nonzero: initialise every school by the method's rule
 *               (Sec. 2.1.1) at the start of the first fsb_batch_step,
 *               which may then have n_steps = 0; start_step must be 0
 *   stats       NULL, or host room for n_schools * n_steps records,
 *               school-major (record k * n_steps + s is school k, step s)
 * The offset table and keys are copied at creation. */
typedef struct fsb_batch* fsb_batch_handle;

int fsb_batch_create(const fsb_config* tmpl, uint32_t n_schools, const uint64_t* offsets,
                     const uint64_t* seeds, const fsb_state_dev* state, int init,
                     uint64_t start_step, void* cuda_stream, fsb_batch_handle* out);

/* Capacities of the batched kernel (any pointer may be NULL): *block_fish
 * fish one block holds on chip (11264; a school on a cluster of c blocks,
 * c <= *max_cluster = 8, holds up to c times that), and *team_fish fish
 * one warp of a packed team holds (704: schools of at most 8, 4, 2 and 1
 * times that run on teams of 8, 4, 2 and 1 warps, several to a block; 0
 * if the library was built without packing).  Needs no GPU. */
int fsb_batch_limits(uint64_t* block_fish, uint64_t* team_fish, int* max_cluster);

/* Advance every school of the batch by n_steps.  Asynchronous on the
 * batch's stream unless stats is given (then synchronises and fills it). */
int fsb_batch_step(fsb_batch_handle b, uint32_t n_steps, fsb_step_stats* stats);

/* Cluster size of the batch's schools.
 *   0 (default): each school runs on the smallest cluster (1 to 8 blocks of
 *     block_fish fish) that holds it, a school of at most half a block on
 *     the smallest packed team that holds it.  One persistent launch per cluster size in
 *     use runs concurrently with the others, each on a share of the SMs
 *     proportional to its schools' fish times a measured cost per fish of
 *     that width; single-block schools take the SMs left over, and every launch helps with the schools of smaller clusters
 *     once its own are done.
 *   1 to 8: every school larger than one block runs on clusters of this
 *     size (one launch on every SM it can hold, single blocks beside it);
 *     1 also runs every school on a block of its own (no packing).
 * Too small for the largest school -> FSB_ERR_UNSUPPORTED; another value ->
 * FSB_ERR_INVALID_ARG.  Synchronises. */
int fsb_batch_set_cluster(fsb_batch_handle b, int cluster);

/* Launch shape and step counter of a batch (any pointer may be NULL): the
 * largest cluster size in use, its resident clusters, the blocks of the
 * single-block launch beside the clusters (0 if none), the schools that run
 * on clusters of more than one block, the step counter. */
int fsb_batch_info(fsb_batch_handle b, int* cluster, int* n_clusters, int* filler_blocks,
                   uint32_t* n_big, uint64_t* step);

/* The batch's launch plan (any pointer may be NULL): n_launches (1 to 8)
 * concurrent persistent launches, launch i running clusters of cluster[i]
 * blocks on a grid of blocks[i] blocks (arrays of 8; entries past
 * n_launches are 0), and queue_schools[t] (array of 12) schools in the
 * work queue of clusters of 8 - t blocks (t = 0 .. 6), of single blocks
 * (t = 7), and of schools packed several to a block on teams of 8, 4, 2
 * and 1 warps (t = 8 .. 11: at most 8, 4, 2 and 1 times team_fish fish;
 * every school of at most half a block is packed unless the cluster size
 * is forced to 1). */
int fsb_batch_plan(fsb_batch_handle b, int* n_launches, int* cluster, int* blocks,
                   uint32_t* queue_schools);

/* Replace the batch's launches, keeping its work queues (set by
 * fsb_batch_set_cluster): n_launches (1 to 8) launches in decreasing cluster
 * size, launch i running clusters of cluster[i] (1 to 8) blocks on a grid
 * of blocks[i] (a positive multiple of cluster[i]).  The widest launch
 * must be at least as wide as the widest non-empty queue.  Any other
 * combination -> FSB_ERR_INVALID_ARG, handle unchanged.  Synchronises. */
int fsb_batch_set_plan(fsb_batch_handle b, int n_launches, const int* cluster,
                       const int* blocks);

/* Device time of the batch launches since timing was enabled (CUDA events
 * on the batch's stream around each launch). */
int fsb_batch_set_timing(fsb_batch_handle b, int enable);
int fsb_batch_kernel_time(fsb_batch_handle b, double* ms, uint64_t* launches);

int fsb_batch_destroy(fsb_batch_handle b);

/* One-shot form: create, one fsb_batch_step of n_steps, destroy. */
int fsb_run_batch(const fsb_config* tmpl, uint32_t n_schools, const uint64_t* offsets,
                  const uint64_t* seeds, const fsb_state_dev* state, int init,
                  uint64_t start_step, uint32_t n_steps, fsb_step_stats* stats,
                  void* cuda_stream);

/* Kernel timing for one handle, the GPU analogue of the paper's
 * omp_get_wtime() bracketing of eat() (Sec. 2.3.2).  While enabled, every
 * launch of the fused per-step pass is bracketed by CUDA events on the
 * handle's stream; fsb_kernel_time reports the summed device time (ms) and
 * the launch count since it was enabled, synchronising the stream. */
int fsb_set_kernel_timing(fsb_handle h, int enable);
int fsb_kernel_time(fsb_handle h, double* fused_ms, uint64_t* fused_launches);

/* Test hook for failure detection (no counterpart in the paper).
 * Nothing faults on the GPU: the failure is made by withholding one
 * arrival or one copy.  `block` >= 0 arms the hook and -1 clears it.
 * `timeout_ns` (0 keeps the current value, default 1 s) bounds every
 * device-side wait of the handle from then on.
 *   Resident path: on later fsb_step calls, block `block` skips its arrival
 *     at the grid barrier of step index `step` of the call, so every block's
 *     bounded wait runs out.  The school's state is left as it was before
 *     the call.
 *   Streaming path, copy-ring kernels (stream kernel 2 or 3): in pass
 *     `step` of later calls, block `block` withholds the first bulk copy of
 *     its ring, so its wait runs out and the others give up.  Pass 0 swims
 *     only, passes 1 .. n-1 are fused, pass n settles.  The school's state is
 *     then undefined, since passes update it in place.  Any other stream
 *     kernel -> FSB_ERR_UNSUPPORTED.
 * Either way the call reports FSB_ERR_TIMEOUT at its next synchronising
 * point and no block hangs. The status stays latched: later calls and
 * reads on the handle report it, so destroy the handle. */
int fsb_set_fault_injection(fsb_handle h, int block, uint32_t step, uint64_t timeout_ns);

/* Launch shape of a handle's kernels (0 in a field = the library's choice).
 * Set by the autotuner (paper_2507_20173_gb300.autotune) or by hand; the
 * results do not depend on it except for the rounding of the barycentre
 * sums, whose reduction tree follows the grid.
 *   stream_kernel        1: vector loads; 2: bulk asynchronous copies into a
 *                        shared-memory ring (binary32, 16-byte aligned state);
 *                        3: the same ring run by its own producer warp, stages
 *                        released per consumer warp (binary32, aligned state);
 *                        4: steps blocked by recompute -- positions do not
 *                        depend on weights, so a maxima pass swims the next
 *                        stream_block_steps steps from the state to find their
 *                        max |delta| and eat() values, and a step pass then
 *                        eats and swims them all with one read and write of
 *                        the state (binary32, aligned state, swim_mode 0, a
 *                        swim step of 0 or at least 2^-103; the call's first
 *                        swim and last eat take kernel 1);
 *                        5: the same pair of passes, the maxima pass also
 *                        storing the positions of the k steps (8 k B per fish
 *                        in slots the handle allocates), which the step pass
 *                        loads instead of drawing and swimming again.
 *                        The library's choice (0) is kernel 5 with 8 steps
 *                        per pair for a streaming school of at least 2^22
 *                        fish that allows it, when its 64 B per fish of
 *                        slots take at most half of the free device memory;
 *                        kernel 1 otherwise.  A slot allocation that fails
 *                        returns FSB_ERR_OOM
 *   stream_block         threads per block of the streaming pass: 256 or 512
 *                        (kernel 3: consumer threads; the block has 32 more)
 *   stream_blocks_per_sm blocks per SM of the streaming grid (capped by
 *                        occupancy)
 *   resident_fpt         most fish per thread of the resident kernel: 4, 8,
 *                        12, 16 (a block's slice is also bounded by its
 *                        shared memory, 7168 fish)
 *   resident_block       fish threads per block of the resident kernel
 *                        (multiple of 32, at most 512; one synchronisation
 *                        warp is added).  The library's choice: with 4 fish
 *                        per thread, the smallest block that fits the school
 *                        on one block per SM; otherwise the largest block
 *                        with a fish pair for every thread
 *   stream_stages        bulk-copy kernels: shared-memory tiles in flight per
 *                        block, 2, 3 or 4 (kernel 3: 2 or 3)
 *   stream_block_steps   kernels 4 and 5: steps per pair of passes, 2, 4 or
 *                        8 (0: 4 for kernel 4, 8 for kernel 5)
 * A combination that cannot run returns FSB_ERR_INVALID_ARG and leaves the
 * handle unchanged.  Synchronises the handle's stream. */
typedef struct {
    int32_t stream_kernel;
    int32_t stream_block;
    int32_t stream_blocks_per_sm;
    int32_t resident_fpt;
    int32_t resident_block;
    int32_t stream_stages;
    int32_t stream_block_steps;
} fsb_tuning;

int fsb_set_tuning(fsb_handle h, const fsb_tuning* t);
int fsb_get_tuning(fsb_handle h, fsb_tuning* t);

/* Autotuner (no counterpart in the paper's method; the GPU analogue of its
 * thread-count / schedule / chunk study, Sec. 2.2.2).  Measures every launch
 * shape of both single-school paths for a school of cfg->n_fish fish in
 * cfg->precision, on a scratch school (library-owned state, freed before
 * return), n_steps timed steps each, and reports the fastest: *best_path
 * (FSB_PATH_STREAM or FSB_PATH_RESIDENT -- this fixes the cutoff between
 * the two kernels for that size), *best_tuning (apply with fsb_set_tuning
 * to a handle created with that path), its throughput and how many shapes
 * ran.  Synchronous; needs room for one more school of that size. */
int fsb_autotune(const fsb_config* cfg, uint32_t n_steps, int* best_path,
                 fsb_tuning* best_tuning, double* best_fish_steps_per_s,
                 uint32_t* candidates_tried);

/* Batch autotuner: times the batch of fsb_batch_create's arguments with
 * each school on the smallest cluster that holds it (cluster 0, the
 * default) and with every school on clusters of 1, 2, 4 and 8 blocks (those
 * that hold the largest school), and reports the fastest as the value for
 * fsb_batch_set_cluster.  OVERWRITES `state` (every school is initialised
 * and stepped).  Synchronous. */
int fsb_autotune_batch(const fsb_config* tmpl, uint32_t n_schools, const uint64_t* offsets,
                       const uint64_t* seeds, const fsb_state_dev* state, uint32_t n_steps,
                       int* best_cluster, double* best_fish_steps_per_s);

/* The paper's eat() reduction on its own: *result = max over i < n of
 * (prev_objective[i] - current_objective[i]) (binary32 device arrays,
 * 16-byte aligned), computed with the chosen reduction construct -- the GPU
 * analogue of the paper's Experiment 3, which times eat() under OpenMP
 * `reduction(max:)` and under `critical` (Sec. 2.3.2, Sec. 3.4):
 *   FSB_EAT_REDUCTION  hierarchical: warp shuffles, shared memory, one atomic
 *                      per block
 *   FSB_EAT_PER_WARP   one atomic per warp
 *   FSB_EAT_CRITICAL   one atomic per fish on a single word (every update
 *                      serialises on one address)
 * All three are exact (max on order-preserving keys).  *device_ms (may be
 * NULL) receives the device time of the reduction (CUDA events).
 * Synchronises cuda_stream. */
enum { FSB_EAT_REDUCTION = 0, FSB_EAT_PER_WARP = 1, FSB_EAT_CRITICAL = 2 };
int fsb_eat_max(const void* prev_objective, const void* current_objective, uint64_t n,
                int construct, double* result, float* device_ms, void* cuda_stream);

/* Which single-school path a handle runs (fsb_path value), after AUTO is
 * resolved. */
int fsb_handle_path(fsb_handle h, int* path_out);

/* Advance a school held in caller-owned device arrays by n_steps steps
 * WITHOUT ANY DEVICE ALLOCATION.  The paper has no counterpart: this exists
 * for callers that cannot let a library allocate GPU memory at call time --
 * hosts that own all device memory through their own arena and forbid later
 * cudaMalloc, and latency-bound pipelines in which cudaMalloc / cudaFree
 * (which can synchronise the whole device) would stall their other streams.
 * It runs stream kernel 1 (vector loads) in fsb_step's launch shape for that
 * kernel -- not kernel 5, which fsb_step chooses for large schools and whose
 * position slots (64 B per fish) would need an allocation; the kernels'
 * scratch (control word, per-block reduction partials, per-step
 * statistics ring) lives in one fixed file-scope __device__ array of about
 * 210 KB that every GPU loading the library holds until the process exits.
 *   cfg         as for fsb_create (path is ignored: always streaming;
 *               collective_mode 1 -> FSB_ERR_UNSUPPORTED)
 *   state       caller-owned device arrays (fsb_state_dev layout) holding the
 *               school at step start_step; advanced in place
 *   start_step  the state's step counter t; t + n_steps must stay below 2^32
 *   n_steps     1 .. 4096 (the statistics ring's size in the static array);
 *               larger values return FSB_ERR_INVALID_ARG with that reason in
 *               fsb_last_error() -- split longer runs into several calls
 *   stats_out   NULL, or n_steps records.  In device (or managed) memory they
 *               are written in stream order and the call stays asynchronous.
 *               In host memory the call synchronises the stream, fills them
 *               and returns the device status (below)
 * Device-side errors (FSB_ERR_STATE from a pass-sequence or debug-build
 * check) are latched in the static array.  A call that synchronises (host
 * stats_out) returns the first such error latched on that device since the
 * last one it reported -- by an earlier asynchronous call or by itself -- and
 * clears it; an asynchronous call returns only host-side errors.  A call
 * whose passes found an error leaves its school partly advanced.
 * The first call on each device looks up the array's device address (set-up
 * done once per device, with that device current); make that first call
 * before any stream capture.  All calls on a device share the one array and
 * rewrite it: calls whose kernels overlap on the GPU (different streams or
 * threads) race and corrupt each other's results, so serialise them.
 * Allocates nothing (no cudaMalloc, cudaFree, graph or event creation). */
int fsb_step_static(const fsb_config* cfg, const fsb_state_dev* state, uint64_t start_step,
                    uint32_t n_steps, fsb_step_stats* stats_out, void* cuda_stream);

/* Name of a status code (static string). */
const char* fsb_strerror(int status);

/* Detail of the last failure on the calling thread (static per thread). */
const char* fsb_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* FSB_H */
