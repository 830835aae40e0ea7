// fsb_stream_ws.cu -- the streaming pass on a warp-specialised copy ring.
//
// Same pass semantics and shared-memory ring as fsb_stream_tma.cu, but the
// ring is run by its own warp: a block is THREADS consumer threads plus one
// producer warp (the block's last).  One elected producer thread keeps
// STAGES tiles of (x, y, w, prevObjective) in flight with cp.async.bulk
// copies that complete on the stage's "full" mbarrier.  Consumer warps wait
// on "full", take their four fish of each array out of shared memory, and
// hand the stage back through its "empty" mbarrier (one arrival per warp)
// before running the per-fish step; the producer refills a stage once every
// consumer warp has released it.  There is no block-wide barrier per tile,
// so consumer warps drift against each other instead of waiting for the
// slowest one at every tile.
//
// Reads of a stage (generic proxy) must be performed before the refill
// (async proxy) writes it: each consumer thread issues a proxy fence after
// its reads, then its warp converges and one lane arrives (release) on
// "empty", which the producer acquires before the refill.
//
// Every wait is bounded (fsb_bulk_copy.cuh).  A warp whose wait gives up
// leaves its loop (the decision is made warp-wide), the failure is shared
// through the block, the producer waits (bounded) for the copies it still
// has in flight, and the block leaves without its partial; the host sees
// FSB_ERR_TIMEOUT.
#include <cstdint>

#include "fsb_bulk_copy.cuh"
#include "fsb_stream_common.cuh"

namespace fsb {
namespace {

template <int THREADS, int STAGES>
struct WsRing {
  float4 buf[STAGES][4][THREADS];    // per stage: x, y, w, prevObjective tiles
  unsigned long long full[STAGES];   // copies landed (producer's expect_tx)
  unsigned long long empty[STAGES];  // every consumer warp has read the stage
};

// Blocks per SM the register budget is sized for: 2 of 544 or 4 of 288
// threads, about 1100 threads per SM either way.
template <int THREADS>
struct WsMinBlocks {
  static constexpr int value = THREADS == 256 ? 4 : 2;
};

template <int THREADS, int STAGES, int PASS, int ACC, bool VAR>
__global__ void __launch_bounds__(THREADS + 32, WsMinBlocks<THREADS>::value)
    stream_pass_ws_kernel(StreamArgs<float> a) {
  using B = uint32_t;
  using Acc = SumAcc<ACC>;
  using Ring = WsRing<THREADS, STAGES>;
  constexpr int kTile = THREADS * 4;
  constexpr unsigned kTileBytes = kTile * sizeof(float);
  constexpr int kConsumerWarps = THREADS / 32;
  const Physics<float> ph = kernel_physics<VAR>(a.ph);

  extern __shared__ __align__(128) unsigned char smem_raw[];
  Ring& R = *reinterpret_cast<Ring*>(smem_raw);
  __shared__ int s_failed;

  uint32_t j;
  uint64_t base;
  if (!pass_prologue<PASS>(a.ctl, a.ctl, a.ring_cap, j, base)) return;
  float M = 0.f;
  if (PASS != kSwimOnly) M = feed_normaliser(a.ring[j - 1], ph);
  // the swim-only pass needs x, y (and w for the weight-scaled swim)
  const int kArrays = PASS != kSwimOnly ? 4 : (ph.swim_mode != 0 ? 3 : 2);
  const uint32_t t = static_cast<uint32_t>(base + j + 1);

  const uint64_t n_tiles = a.n / kTile;
  const uint64_t my_tiles =
      n_tiles > blockIdx.x ? (n_tiles - blockIdx.x + gridDim.x - 1) / gridDim.x : 0;
  const int lane = threadIdx.x & 31;

  if (threadIdx.x == 0) {
#pragma unroll
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(&R.full[s], 1);
      mbar_init(&R.empty[s], kConsumerWarps);
    }
    fence_mbar_init();
    s_failed = 0;
  }
  __syncthreads();

  Acc acc;
  B maxb = 0, ekey = 0;
  bool ok = true;
  uint64_t issued = 0;  // producer thread: tiles whose copies were issued
  if (threadIdx.x >= THREADS) {
    if (threadIdx.x == THREADS) {
      float* const src[4] = {a.x, a.y, a.w, a.pv};
      for (uint64_t k = 0; k < my_tiles; ++k) {
        const int s = static_cast<int>(k % STAGES);
        // the stage's previous tile (k - STAGES) must be released by every
        // consumer warp: completion number k / STAGES - 1 of empty[s]
        if (k >= static_cast<uint64_t>(STAGES) &&
            !mbar_wait_bounded(&R.empty[s], static_cast<unsigned>((k / STAGES - 1) & 1), a.ctl,
                               a.timeout_ns)) {
          ok = false;
          break;
        }
        issued = k + 1;
        // test hook: this block withholds the first copy of its ring in pass j
        if (k == 0 && static_cast<int>(blockIdx.x) == a.inject_block && j == a.inject_pass)
          continue;
        const uint64_t off = (blockIdx.x + k * gridDim.x) * static_cast<uint64_t>(kTile);
        mbar_expect_tx(&R.full[s], kArrays * kTileBytes);
        for (int q = 0; q < kArrays; ++q)
          bulk_g2s(R.buf[s][q], src[q] + off, kTileBytes, &R.full[s]);
      }
    }
  } else {
    for (uint64_t k = 0; k < my_tiles; ++k) {
      const int s = static_cast<int>(k % STAGES);
      const unsigned parity = static_cast<unsigned>((k / STAGES) & 1);
      const bool mine = mbar_wait_bounded(&R.full[s], parity, a.ctl, a.timeout_ns);
      if (!__all_sync(0xffffffffu, mine)) {
        ok = false;
        break;
      }
      float4 v[4];
#pragma unroll
      for (int q = 0; q < 4; ++q)
        if (q < kArrays) v[q] = R.buf[s][q][threadIdx.x];
      fence_proxy_async_smem();
      __syncwarp();
      if (lane == 0) mbar_arrive(&R.empty[s]);

      const uint64_t tile = blockIdx.x + k * gridDim.x;
      const uint64_t g = tile * THREADS + threadIdx.x;  // float4 index
      float x[4] = {v[0].x, v[0].y, v[0].z, v[0].w};
      float y[4] = {v[1].x, v[1].y, v[1].z, v[1].w};
      float w[4], pv[4];
      if (kArrays >= 3) {
        w[0] = v[2].x; w[1] = v[2].y; w[2] = v[2].z; w[3] = v[2].w;
      }
      if (PASS != kSwimOnly) {
        pv[0] = v[3].x; pv[1] = v[3].y; pv[2] = v[3].z; pv[3] = v[3].w;
      }
      fish_pass4<float, PASS>(x, y, w, pv, g * 4, M, t, a.key, a.school, ph, acc, maxb, ekey);
      if (PASS != kSettle) {
        reinterpret_cast<float4*>(a.x)[g] = make_float4(x[0], x[1], x[2], x[3]);
        reinterpret_cast<float4*>(a.y)[g] = make_float4(y[0], y[1], y[2], y[3]);
        reinterpret_cast<float4*>(a.pv)[g] = make_float4(pv[0], pv[1], pv[2], pv[3]);
      }
      if (PASS != kSwimOnly)
        reinterpret_cast<float4*>(a.w)[g] = make_float4(w[0], w[1], w[2], w[3]);
    }
  }
  if (!ok) s_failed = 1;
  __syncthreads();
  if (s_failed) {
    // leave only after the copies still in flight have landed (bounded)
    if (threadIdx.x == THREADS) {
      const uint64_t first = issued > static_cast<uint64_t>(STAGES) ? issued - STAGES : 0;
      for (uint64_t q = first; q < issued; ++q) {
        const int s = static_cast<int>(q % STAGES);
        const unsigned long long t0 = global_ns();
        while (!mbar_try_wait(&R.full[s], static_cast<unsigned>((q / STAGES) & 1)) &&
               global_ns() - t0 < a.timeout_ns) {
        }
      }
    }
    __syncthreads();
    return;
  }

  // ragged tail: the last n % TILE fish, plain loads, one block's consumers
  if (blockIdx.x == n_tiles % gridDim.x && threadIdx.x < THREADS) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const uint64_t i = n_tiles * kTile + threadIdx.x + static_cast<uint64_t>(q) * THREADS;
      if (i < a.n) {
        float x = a.x[i], y = a.y[i], w = 0.f, pv = 0.f;
        if (kArrays >= 3) w = a.w[i];
        if (PASS != kSwimOnly) pv = a.pv[i];
        fish_pass<float, PASS>(x, y, w, pv, i, M, t, a.key, a.school, ph, acc, maxb, ekey);
        if (PASS != kSettle) {
          a.x[i] = x;
          a.y[i] = y;
          a.pv[i] = pv;
        }
        if (PASS != kSwimOnly) a.w[i] = w;
      }
    }
  }

  // the producer warp joins with empty sums and maxima
  pass_epilogue<float, PASS, ACC, THREADS + 32>(a, acc, maxb, ekey, j, base);
}

template <int THREADS, int STAGES, int PASS, int ACC>
const void* kernel_ptr(bool var) {
  if (var)
    return reinterpret_cast<const void*>(&stream_pass_ws_kernel<THREADS, STAGES, PASS, ACC, true>);
  return reinterpret_cast<const void*>(&stream_pass_ws_kernel<THREADS, STAGES, PASS, ACC, false>);
}

template <int THREADS, int STAGES, int PASS>
const void* pick_acc(int acc, bool var) {
  switch (acc) {
    case kAccPlain32: return kernel_ptr<THREADS, STAGES, PASS, kAccPlain32>(var);
    case kAccKahan32: return kernel_ptr<THREADS, STAGES, PASS, kAccKahan32>(var);
    case kAccF64: return kernel_ptr<THREADS, STAGES, PASS, kAccF64>(var);
    default: return nullptr;
  }
}

template <int THREADS, int STAGES>
const void* pick_pass(int pass, int acc, bool var) {
  switch (pass) {
    case kSwimOnly: return pick_acc<THREADS, STAGES, kSwimOnly>(acc, var);
    case kFused: return pick_acc<THREADS, STAGES, kFused>(acc, var);
    case kSettle: return pick_acc<THREADS, STAGES, kSettle>(acc, var);
    default: return nullptr;
  }
}

template <int THREADS>
const void* pick_stages(int stages, int pass, int acc, bool var, size_t* smem) {
  switch (stages) {
    case 2:
      *smem = sizeof(WsRing<THREADS, 2>);
      return pick_pass<THREADS, 2>(pass, acc, var);
    case 3:
      *smem = sizeof(WsRing<THREADS, 3>);
      return pick_pass<THREADS, 3>(pass, acc, var);
    default:
      return nullptr;
  }
}

const void* pick(const StreamLaunch& L, int pass, size_t* smem) {
  if (L.real_is_double || L.vec != 4) return nullptr;
  const int stages = L.stages ? L.stages : 2;
  const bool var = L.swim_mode != 0 || L.feed_mode != 0;
  switch (L.block) {
    case 256: return pick_stages<256>(stages, pass, L.acc, var, smem);
    case 512: return pick_stages<512>(stages, pass, L.acc, var, smem);
    default: return nullptr;
  }
}

}  // namespace

cudaError_t stream_ws_prepare(const StreamLaunch& L) {
  for (int pass = kSwimOnly; pass <= kSettle; ++pass) {
    size_t smem = 0;
    const void* fn = pick(L, pass, &smem);
    if (!fn) return cudaErrorInvalidValue;
    cudaError_t e =
        cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

int stream_ws_blocks_per_sm(const StreamLaunch& L) {
  size_t smem = 0;
  const void* fn = pick(L, kFused, &smem);
  if (!fn) return 0;
  int nb = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, fn, L.block + 32, smem) != cudaSuccess)
    return 0;
  return nb;
}

cudaError_t launch_stream_pass_ws(const StreamLaunch& L, int pass_kind, cudaStream_t s) {
  size_t smem = 0;
  const void* fn = pick(L, pass_kind, &smem);
  if (!fn || L.grid <= 0) return cudaErrorInvalidValue;
  StreamArgs<float> a = make_stream_args<float>(L);
  void* args[] = {&a};
  return cudaLaunchKernel(fn, dim3(L.grid), dim3(L.block + 32), args, smem, s);
}

}  // namespace fsb
