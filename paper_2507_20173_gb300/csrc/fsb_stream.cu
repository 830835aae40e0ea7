// fsb_stream.cu -- HBM-streaming kernels of the Fish School Behaviour step.
//
// One fused pass per step streams the school's structure-of-arrays state
// (x, y, w, prevObjective) once from HBM and back:
//   pass j of a call (1 <= j < n):  eat + barycentre of step j, using the
//     max M_j that pass j-1 reduced, then swim + objective + delta of step
//     j+1 and the block partials of M_{j+1} and of the paper's eat() value
//     max(prev - cur) (Sec. 2.3.2);
//   pass 0:  swim of step 1 only (the state is settled between calls);
//   pass n:  eat + barycentre of step n only ("settle").
// currentObjective is recomputed from the position in hand instead of being
// stored (bit-identical: same inputs, same correctly rounded operations), so
// a fused pass moves 16 B in and 16 B out per fish in binary32.
//
// Reductions are hierarchical and deterministic: per-thread accumulation in
// a fixed grid-stride order, warp shuffles, shared memory across warps, one
// partial per block in global scratch, and the last block to arrive (atomic
// counter) folds the partials in fixed order and writes the step's record to
// the statistics ring and the control word.
#include <cstdint>

#include "fsb_check.cuh"
#include "fsb_stream_common.cuh"

namespace fsb {
namespace {

// Debug build: every fish a pass reads lies in the pond, |x|, |y| <= P (the
// swim clamps at the bank, and the initial positions are drawn inside it), so
// a state outside it -- or a NaN -- was not produced by the method.  A failed
// check latches FSB_ERR_STATE; the pass still computes (the swim clamps the
// fish back), and the call's later passes do nothing.
template <typename Real>
__device__ __forceinline__ void check_in_pond(Real x, Real y, const Physics<Real>& ph,
                                              Ctl* ctl) {
#ifdef FSB_DEBUG_BOUNDS
  const Real P = ph.pond_half;
  fsb_check(x >= -P && x <= P && y >= -P && y <= P, &ctl->status, &ctl->timeout_site, 10u);
#else
  (void)x;
  (void)y;
  (void)ph;
  (void)ctl;
#endif
}

// ----------------------------------------------------------- vectors --
template <typename Real, int VEC>
struct VecT;
template <>
struct VecT<float, 4> {
  using T = float4;
};
template <>
struct VecT<double, 2> {
  using T = double2;
};
template <>
struct VecT<float, 1> {
  using T = float;
};
template <>
struct VecT<double, 1> {
  using T = double;
};

template <typename Real, int VEC>
__device__ __forceinline__ void vload(Real (&v)[VEC], const Real* p, uint64_t g) {
  using T = typename VecT<Real, VEC>::T;
  *reinterpret_cast<T*>(v) = reinterpret_cast<const T*>(p)[g];
}
template <typename Real, int VEC>
__device__ __forceinline__ void vstore(Real* p, uint64_t g, const Real (&v)[VEC]) {
  using T = typename VecT<Real, VEC>::T;
  reinterpret_cast<T*>(p)[g] = *reinterpret_cast<const T*>(v);
}

template <typename Real, int VEC, int PASS, int ACC, int BLOCK, int MINB, bool VAR>
__global__ void __launch_bounds__(BLOCK, MINB) stream_pass_kernel(StreamArgs<Real> a) {
  using B = typename Bits<Real>::type;
  using Acc = SumAcc<ACC>;
  const Physics<Real> ph = kernel_physics<VAR>(a.ph);

  uint32_t j;
  uint64_t base;
  // The pass index comes from device memory; refuse to index the ring with
  // a value that does not fit this call's sequence.
  if (!pass_prologue<PASS>(a.ctl, a.ctl, a.ring_cap, j, base)) return;
  Real M = Real(0);
  if (PASS != kSwimOnly) M = feed_normaliser(a.ring[j - 1], ph);
  // the weight-scaled swim needs the weights in the swim-only pass too
  const bool load_w = PASS != kSwimOnly || ph.swim_mode != 0;
  const uint32_t t = static_cast<uint32_t>(base + j + 1);

  Acc acc;
  B maxb = 0, ekey = 0;

  const uint64_t ngroups = a.n / VEC;
  const uint64_t stride = static_cast<uint64_t>(gridDim.x) * BLOCK;
  const uint64_t tid = static_cast<uint64_t>(blockIdx.x) * BLOCK + threadIdx.x;
  // consecutive passes sweep the school in opposite directions, so a pass
  // starts on the groups the previous one touched last (still in L2)
  const bool backward = (j & 1u) != 0u;
  for (uint64_t gi = tid; gi < ngroups; gi += stride) {
    const uint64_t g = backward ? ngroups - 1 - gi : gi;
    Real x[VEC], y[VEC], w[VEC], pv[VEC];
    vload<Real, VEC>(x, a.x, g);
    vload<Real, VEC>(y, a.y, g);
    if (load_w) vload<Real, VEC>(w, a.w, g);
    if (PASS != kSwimOnly) vload<Real, VEC>(pv, a.pv, g);
#pragma unroll
    for (int v = 0; v < VEC; ++v) check_in_pond(x[v], y[v], ph, a.ctl);
    if constexpr (VEC == 4) {
      fish_pass4<Real, PASS>(x, y, w, pv, g * VEC, M, t, a.key, a.school, ph, acc, maxb, ekey);
    } else if constexpr (VEC == 2) {
      fish_pass2<Real, PASS>(x, y, w, pv, g * VEC, M, t, a.key, a.school, ph, acc, maxb, ekey);
    } else {
#pragma unroll
      for (int v = 0; v < VEC; ++v)
        fish_pass<Real, PASS>(x[v], y[v], w[v], pv[v], g * VEC + v, M, t, a.key, a.school, ph,
                              acc, maxb, ekey);
    }
    if (PASS != kSettle) {
      vstore<Real, VEC>(a.x, g, x);
      vstore<Real, VEC>(a.y, g, y);
      vstore<Real, VEC>(a.pv, g, pv);
    }
    if (PASS != kSwimOnly) vstore<Real, VEC>(a.w, g, w);
  }
  if (VEC > 1) {  // ragged tail: the last n % VEC fish, one per thread
    const uint64_t i = ngroups * VEC + tid;
    if (i < a.n) {
      Real x = a.x[i], y = a.y[i], w = Real(0), pv = Real(0);
      if (load_w) w = a.w[i];
      if (PASS != kSwimOnly) pv = a.pv[i];
      check_in_pond(x, y, ph, a.ctl);
      fish_pass<Real, PASS>(x, y, w, pv, i, M, t, a.key, a.school, ph, acc, maxb, ekey);
      if (PASS != kSettle) {
        a.x[i] = x;
        a.y[i] = y;
        a.pv[i] = pv;
      }
      if (PASS != kSwimOnly) a.w[i] = w;
    }
  }

  pass_epilogue<Real, PASS, ACC, BLOCK>(a, acc, maxb, ekey, j, base);
}

template <typename Real>
__global__ void init_kernel(Real* __restrict__ x, Real* __restrict__ y, Real* __restrict__ w,
                            Real* __restrict__ pv, uint64_t n, Key key, uint32_t school,
                            int weight_mode, Physics<Real> ph) {
  const uint64_t stride = static_cast<uint64_t>(gridDim.x) * blockDim.x;
  for (uint64_t i = static_cast<uint64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
       i += stride) {
    Real xi, yi, wi;
    init_fish(key, school, i, weight_mode, ph, xi, yi, wi);
    x[i] = xi;
    y[i] = yi;
    w[i] = wi;
    pv[i] = objective(xi, yi);
  }
}

template <typename Real>
__global__ void objective_kernel(const Real* __restrict__ x, const Real* __restrict__ y,
                                 Real* __restrict__ cur, uint64_t n) {
  const uint64_t stride = static_cast<uint64_t>(gridDim.x) * blockDim.x;
  for (uint64_t i = static_cast<uint64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
       i += stride)
    cur[i] = objective(x[i], y[i]);
}

template <typename Real, int VEC, int PASS, int ACC, int BLOCK, int MINB>
const void* kernel_ptr(bool var) {
  if (var)
    return reinterpret_cast<const void*>(&stream_pass_kernel<Real, VEC, PASS, ACC, BLOCK, MINB, true>);
  return reinterpret_cast<const void*>(&stream_pass_kernel<Real, VEC, PASS, ACC, BLOCK, MINB, false>);
}

// Launch shapes: (256 threads, 1 / 3 / 4 blocks per SM guaranteed by the
// register budget) for the binary32 vector kernel, (256 or 512, 1) otherwise.
template <typename Real, int VEC, int PASS, int ACC>
const void* pick_block(int block, int minb, bool var) {
  constexpr bool kHot = sizeof(Real) == 4 && VEC == 4;
  if (block == 256) {
    if (minb <= 1) return kernel_ptr<Real, VEC, PASS, ACC, 256, 1>(var);
    if (kHot && minb == 3) return kernel_ptr<Real, VEC, PASS, ACC, 256, kHot ? 3 : 1>(var);
    if (kHot && minb == 4) return kernel_ptr<Real, VEC, PASS, ACC, 256, kHot ? 4 : 1>(var);
    return nullptr;
  }
  if (block == 512 && minb <= 1) return kernel_ptr<Real, VEC, PASS, ACC, 512, 1>(var);
  return nullptr;
}

template <typename Real, int VEC, int PASS>
const void* pick_acc(int acc, int block, int minb, bool var) {
  if (sizeof(Real) == 8) return pick_block<Real, VEC, PASS, kAccF64>(block, minb, var);
  switch (acc) {
    case kAccPlain32: return pick_block<Real, VEC, PASS, kAccPlain32>(block, minb, var);
    case kAccKahan32: return pick_block<Real, VEC, PASS, kAccKahan32>(block, minb, var);
    case kAccF64: return pick_block<Real, VEC, PASS, kAccF64>(block, minb, var);
    default: return nullptr;
  }
}

template <typename Real, int VEC>
const void* pick_pass(int pass, int acc, int block, int minb, bool var) {
  switch (pass) {
    case kSwimOnly: return pick_acc<Real, VEC, kSwimOnly>(acc, block, minb, var);
    case kFused: return pick_acc<Real, VEC, kFused>(acc, block, minb, var);
    case kSettle: return pick_acc<Real, VEC, kSettle>(acc, block, minb, var);
    default: return nullptr;
  }
}

const void* pick_kernel(const StreamLaunch& L, int pass) {
  const bool var = L.swim_mode != 0 || L.feed_mode != 0;
  if (L.real_is_double) {
    if (L.vec == 2) return pick_pass<double, 2>(pass, L.acc, L.block, L.min_blocks, var);
    if (L.vec == 1) return pick_pass<double, 1>(pass, L.acc, L.block, L.min_blocks, var);
  } else {
    if (L.vec == 4) return pick_pass<float, 4>(pass, L.acc, L.block, L.min_blocks, var);
    if (L.vec == 1) return pick_pass<float, 1>(pass, L.acc, L.block, L.min_blocks, var);
  }
  return nullptr;
}

}  // namespace

cudaError_t launch_stream_pass(const StreamLaunch& L, int pass_kind, cudaStream_t s) {
  const void* fn = pick_kernel(L, pass_kind);
  if (!fn || L.grid <= 0) return cudaErrorInvalidValue;
  if (L.real_is_double) {
    StreamArgs<double> a = make_stream_args<double>(L);
    void* args[] = {&a};
    return cudaLaunchKernel(fn, dim3(L.grid), dim3(L.block), args, 0, s);
  }
  StreamArgs<float> a = make_stream_args<float>(L);
  void* args[] = {&a};
  return cudaLaunchKernel(fn, dim3(L.grid), dim3(L.block), args, 0, s);
}

int stream_blocks_per_sm(const StreamLaunch& L) {
  const void* fn = pick_kernel(L, kFused);
  if (!fn) return 0;
  int nb = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, fn, L.block, 0) != cudaSuccess) return 0;
  return nb;
}

cudaError_t launch_init(const StreamLaunch& L, int weight_mode, cudaStream_t s) {
  const int block = 256;
  const uint64_t want = (L.n + block - 1) / block;
  const int grid = static_cast<int>(want < 4096 ? want : 4096);
  if (L.real_is_double) {
    StreamArgs<double> a = make_stream_args<double>(L);
    init_kernel<double><<<grid, block, 0, s>>>(a.x, a.y, a.w, a.pv, a.n, a.key, a.school,
                                               weight_mode, a.ph);
  } else {
    StreamArgs<float> a = make_stream_args<float>(L);
    init_kernel<float><<<grid, block, 0, s>>>(a.x, a.y, a.w, a.pv, a.n, a.key, a.school,
                                              weight_mode, a.ph);
  }
  return cudaGetLastError();
}

cudaError_t launch_objective(const StreamLaunch& L, uint64_t first, uint64_t count, void* cur,
                             cudaStream_t s) {
  if (count == 0) return cudaSuccess;
  const int block = 256;
  const uint64_t want = (count + block - 1) / block;
  const int grid = static_cast<int>(want < 4096 ? want : 4096);
  if (L.real_is_double)
    objective_kernel<double><<<grid, block, 0, s>>>(static_cast<const double*>(L.x) + first,
                                                    static_cast<const double*>(L.y) + first,
                                                    static_cast<double*>(cur), count);
  else
    objective_kernel<float><<<grid, block, 0, s>>>(static_cast<const float*>(L.x) + first,
                                                   static_cast<const float*>(L.y) + first,
                                                   static_cast<float*>(cur), count);
  return cudaGetLastError();
}

}  // namespace fsb
