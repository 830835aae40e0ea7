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

#include "fsb_device.cuh"
#include "fsb_internal.h"

namespace fsb {
namespace {

constexpr unsigned kFull = 0xFFFFFFFFu;

template <typename Real>
struct StreamArgs {
  Real* __restrict__ x;
  Real* __restrict__ y;
  Real* __restrict__ w;
  Real* __restrict__ pv;
  uint64_t n;
  Key key;
  uint32_t school;
  Physics<Real> ph;
  Ctl* ctl;
  BlockPartial* partials;
  fsb_step_stats* ring;
  uint32_t ring_cap;
};

// ------------------------------------------------------- accumulators --
template <int ACC>
struct SumAcc;

// Plain binary32 sums (the precision study's baseline).
template <>
struct SumAcc<kAccPlain32> {
  using Sum = float;
  float w = 0.f, x = 0.f, y = 0.f;
  __device__ __forceinline__ void add(float wi, float xi, float yi) {
    w = __fadd_rn(w, wi);
    x = __fadd_rn(x, __fmul_rn(wi, xi));
    y = __fadd_rn(y, __fmul_rn(wi, yi));
  }
  __device__ __forceinline__ float rw() const { return w; }
  __device__ __forceinline__ float rx() const { return x; }
  __device__ __forceinline__ float ry() const { return y; }
};

// Kahan-compensated binary32 per thread; combined in binary64 above.
template <>
struct SumAcc<kAccKahan32> {
  using Sum = double;
  float sw = 0.f, cw = 0.f, sx = 0.f, cx = 0.f, sy = 0.f, cy = 0.f;
  __device__ __forceinline__ static void kadd(float& s, float& c, float v) {
    const float yv = __fsub_rn(v, c);
    const float t = __fadd_rn(s, yv);
    c = __fsub_rn(__fsub_rn(t, s), yv);
    s = t;
  }
  __device__ __forceinline__ void add(float wi, float xi, float yi) {
    kadd(sw, cw, wi);
    kadd(sx, cx, __fmul_rn(wi, xi));
    kadd(sy, cy, __fmul_rn(wi, yi));
  }
  __device__ __forceinline__ double rw() const { return double(sw) - double(cw); }
  __device__ __forceinline__ double rx() const { return double(sx) - double(cx); }
  __device__ __forceinline__ double ry() const { return double(sy) - double(cy); }
};

// Binary64 accumulation (products of binary32 operands are exact).
template <>
struct SumAcc<kAccF64> {
  using Sum = double;
  double w = 0.0, x = 0.0, y = 0.0;
  template <typename Real>
  __device__ __forceinline__ void add(Real wi, Real xi, Real yi) {
    const double dw = static_cast<double>(wi);
    w = __dadd_rn(w, dw);
    x = __dadd_rn(x, __dmul_rn(dw, static_cast<double>(xi)));
    y = __dadd_rn(y, __dmul_rn(dw, static_cast<double>(yi)));
  }
  __device__ __forceinline__ double rw() const { return w; }
  __device__ __forceinline__ double rx() const { return x; }
  __device__ __forceinline__ double ry() const { return y; }
};

__device__ __forceinline__ float sum2(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ double sum2(double a, double b) { return __dadd_rn(a, b); }

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) v = sum2(v, __shfl_xor_sync(kFull, v, off));
  return v;
}

__device__ __forceinline__ uint32_t warp_max(uint32_t v) { return __reduce_max_sync(kFull, v); }
__device__ __forceinline__ unsigned long long warp_max(unsigned long long v) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    const unsigned long long o = __shfl_xor_sync(kFull, v, off);
    v = o > v ? o : v;
  }
  return v;
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

// One fish through one pass.  `M` is M_j (pass kinds kFused / kSettle),
// `t` the absolute step of the swim (kSwimOnly / kFused).
template <typename Real, int PASS, typename Acc, typename B>
__device__ __forceinline__ void fish_pass(Real& x, Real& y, Real& w, Real& pv, uint64_t i, Real M,
                                          uint32_t t, Key key, uint32_t school,
                                          const Physics<Real>& ph, Acc& acc, B& maxb, B& ekey) {
  using A = Arith<Real>;
  const Real cur = objective(x, y);
  if (PASS != kSwimOnly) {
    if (M > Real(0)) w = eat(w, A::sub(cur, pv), M, ph);
    acc.add(w, x, y);
  }
  if (PASS != kSettle) {
    const Words4 r = fish_draw(key, school, i, t, kDomainSwim);
    swim(x, y, r.v[0], r.v[1], ph);
    const Real ncur = objective(x, y);
    const B mb = abs_bits(A::sub(ncur, cur));
    const B ek = order_key(A::sub(cur, ncur));
    maxb = mb > maxb ? mb : maxb;
    ekey = ek > ekey ? ek : ekey;
    pv = cur;
  }
}

template <typename Real, int VEC, int PASS, int ACC, int BLOCK>
__global__ void __launch_bounds__(BLOCK) stream_pass_kernel(StreamArgs<Real> a) {
  using B = typename Bits<Real>::type;
  using Acc = SumAcc<ACC>;
  using Sum = typename Acc::Sum;
  constexpr int kWarps = BLOCK / 32;

  const uint32_t j = a.ctl->pass;
  const uint64_t base = a.ctl->base_step;
  // The pass index comes from device memory; refuse to index the ring with
  // a value that does not fit this call's sequence.
  if ((PASS != kSwimOnly && (j == 0 || j > a.ring_cap)) || (PASS != kSettle && j >= a.ring_cap)) {
    if (threadIdx.x == 0) atomicCAS(&a.ctl->status, 0, static_cast<int>(FSB_ERR_STATE));
    return;
  }
  Real M = Real(0);
  if (PASS != kSwimOnly) M = static_cast<Real>(a.ring[j - 1].max_abs_delta);
  const uint32_t t = static_cast<uint32_t>(base + j + 1);

  Acc acc;
  B maxb = 0, ekey = 0;

  const uint64_t ngroups = a.n / VEC;
  const uint64_t stride = static_cast<uint64_t>(gridDim.x) * BLOCK;
  const uint64_t tid = static_cast<uint64_t>(blockIdx.x) * BLOCK + threadIdx.x;
  for (uint64_t g = tid; g < ngroups; g += stride) {
    Real x[VEC], y[VEC], w[VEC], pv[VEC];
    vload<Real, VEC>(x, a.x, g);
    vload<Real, VEC>(y, a.y, g);
    if (PASS != kSwimOnly) {
      vload<Real, VEC>(w, a.w, g);
      vload<Real, VEC>(pv, a.pv, g);
    }
#pragma unroll
    for (int v = 0; v < VEC; ++v)
      fish_pass<Real, PASS>(x[v], y[v], w[v], pv[v], g * VEC + v, M, t, a.key, a.school, a.ph,
                            acc, maxb, ekey);
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
      if (PASS != kSwimOnly) {
        w = a.w[i];
        pv = a.pv[i];
      }
      fish_pass<Real, PASS>(x, y, w, pv, i, M, t, a.key, a.school, a.ph, acc, maxb, ekey);
      if (PASS != kSettle) {
        a.x[i] = x;
        a.y[i] = y;
        a.pv[i] = pv;
      }
      if (PASS != kSwimOnly) a.w[i] = w;
    }
  }

  // ---- block reduction -> one partial per block
  __shared__ B s_max[kWarps], s_ekey[kWarps];
  __shared__ Sum s_w[kWarps], s_x[kWarps], s_y[kWarps];
  __shared__ bool s_last;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  maxb = warp_max(maxb);
  ekey = warp_max(ekey);
  Sum sw = Sum(acc.rw()), sx = Sum(acc.rx()), sy = Sum(acc.ry());
  if (PASS != kSwimOnly) {
    sw = warp_sum(sw);
    sx = warp_sum(sx);
    sy = warp_sum(sy);
  }
  if (lane == 0) {
    s_max[warp] = maxb;
    s_ekey[warp] = ekey;
    s_w[warp] = sw;
    s_x[warp] = sx;
    s_y[warp] = sy;
  }
  __syncthreads();
  if (warp == 0) {
    B m = lane < kWarps ? s_max[lane] : B(0);
    B e = lane < kWarps ? s_ekey[lane] : B(0);
    Sum bw = lane < kWarps ? s_w[lane] : Sum(0);
    Sum bx = lane < kWarps ? s_x[lane] : Sum(0);
    Sum by = lane < kWarps ? s_y[lane] : Sum(0);
    m = warp_max(m);
    e = warp_max(e);
    if (PASS != kSwimOnly) {
      bw = warp_sum(bw);
      bx = warp_sum(bx);
      by = warp_sum(by);
    }
    if (lane == 0) {
      BlockPartial bp;
      bp.max_bits = static_cast<unsigned long long>(m);
      bp.e_key = static_cast<unsigned long long>(e);
      bp.sum_w = static_cast<double>(bw);
      bp.sum_wx = static_cast<double>(bx);
      bp.sum_wy = static_cast<double>(by);
      bp.spare = 0.0;
      a.partials[blockIdx.x] = bp;
      __threadfence();
      const unsigned prev = atomicAdd(&a.ctl->arrive, 1u);
      s_last = (prev == gridDim.x - 1);
    }
  }
  __syncthreads();
  if (!s_last) return;

  // ---- last block: fold all partials in a fixed order
  __threadfence();
  B m = 0, e = 0;
  Sum fw = Sum(0), fx = Sum(0), fy = Sum(0);
  for (uint32_t b = threadIdx.x; b < gridDim.x; b += BLOCK) {
    const BlockPartial* bp = a.partials + b;
    const B mb = static_cast<B>(__ldcg(&bp->max_bits));
    const B eb = static_cast<B>(__ldcg(&bp->e_key));
    m = mb > m ? mb : m;
    e = eb > e ? eb : e;
    if (PASS != kSwimOnly) {
      fw = sum2(fw, Sum(__ldcg(&bp->sum_w)));
      fx = sum2(fx, Sum(__ldcg(&bp->sum_wx)));
      fy = sum2(fy, Sum(__ldcg(&bp->sum_wy)));
    }
  }
  m = warp_max(m);
  e = warp_max(e);
  if (PASS != kSwimOnly) {
    fw = warp_sum(fw);
    fx = warp_sum(fx);
    fy = warp_sum(fy);
  }
  __syncthreads();  // shared arrays are reused
  if (lane == 0) {
    s_max[warp] = m;
    s_ekey[warp] = e;
    s_w[warp] = fw;
    s_x[warp] = fx;
    s_y[warp] = fy;
  }
  __syncthreads();
  if (warp == 0) {
    m = lane < kWarps ? s_max[lane] : B(0);
    e = lane < kWarps ? s_ekey[lane] : B(0);
    fw = lane < kWarps ? s_w[lane] : Sum(0);
    fx = lane < kWarps ? s_x[lane] : Sum(0);
    fy = lane < kWarps ? s_y[lane] : Sum(0);
    m = warp_max(m);
    e = warp_max(e);
    if (PASS != kSwimOnly) {
      fw = warp_sum(fw);
      fx = warp_sum(fx);
      fy = warp_sum(fy);
    }
    if (lane == 0) {
      if (PASS != kSwimOnly) {
        fsb_step_stats* rec = a.ring + (j - 1);
        rec->sum_w = static_cast<double>(fw);
        rec->sum_wx = static_cast<double>(fx);
        rec->sum_wy = static_cast<double>(fy);
      }
      if (PASS != kSettle) {
        fsb_step_stats* rec = a.ring + j;
        Real mv;
        if (sizeof(Real) == 4)
          mv = static_cast<Real>(__uint_as_float(static_cast<uint32_t>(m)));
        else
          mv = static_cast<Real>(__longlong_as_double(static_cast<long long>(m)));
        rec->max_abs_delta = static_cast<double>(mv);
        rec->eat_max_diff = static_cast<double>(key_to_value(e, Real(0)));
      }
      a.ctl->arrive = 0u;
      if (PASS == kSettle) {
        a.ctl->base_step = base + j;
        a.ctl->pass = 0u;
      } else {
        a.ctl->pass = j + 1;
      }
      __threadfence();
    }
  }
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

template <typename Real>
StreamArgs<Real> make_args(const StreamLaunch& L) {
  StreamArgs<Real> a;
  a.x = static_cast<Real*>(L.x);
  a.y = static_cast<Real*>(L.y);
  a.w = static_cast<Real*>(L.w);
  a.pv = static_cast<Real*>(L.pv);
  a.n = L.n;
  a.key.k0 = static_cast<uint32_t>(L.seed);
  a.key.k1 = static_cast<uint32_t>(L.seed >> 32);
  a.school = L.school;
  a.ph.pond_half = static_cast<Real>(L.pond_half);
  a.ph.step = static_cast<Real>(L.step);
  a.ph.w0 = static_cast<Real>(L.w0);
  a.ph.w_min = static_cast<Real>(L.w_min);
  a.ph.w_max = static_cast<Real>(L.w_max);
  a.ctl = L.ctl;
  a.partials = L.partials;
  a.ring = L.ring;
  a.ring_cap = L.ring_cap;
  return a;
}

template <typename Real, int VEC, int PASS, int ACC, int BLOCK>
const void* kernel_ptr() {
  return reinterpret_cast<const void*>(&stream_pass_kernel<Real, VEC, PASS, ACC, BLOCK>);
}

template <typename Real, int VEC, int PASS, int ACC>
const void* pick_block(int block) {
  switch (block) {
    case 256: return kernel_ptr<Real, VEC, PASS, ACC, 256>();
    case 512: return kernel_ptr<Real, VEC, PASS, ACC, 512>();
    default: return nullptr;
  }
}

template <typename Real, int VEC, int PASS>
const void* pick_acc(int acc, int block) {
  if (sizeof(Real) == 8) return pick_block<Real, VEC, PASS, kAccF64>(block);
  switch (acc) {
    case kAccPlain32: return pick_block<Real, VEC, PASS, kAccPlain32>(block);
    case kAccKahan32: return pick_block<Real, VEC, PASS, kAccKahan32>(block);
    case kAccF64: return pick_block<Real, VEC, PASS, kAccF64>(block);
    default: return nullptr;
  }
}

template <typename Real, int VEC>
const void* pick_pass(int pass, int acc, int block) {
  switch (pass) {
    case kSwimOnly: return pick_acc<Real, VEC, kSwimOnly>(acc, block);
    case kFused: return pick_acc<Real, VEC, kFused>(acc, block);
    case kSettle: return pick_acc<Real, VEC, kSettle>(acc, block);
    default: return nullptr;
  }
}

const void* pick_kernel(const StreamLaunch& L, int pass) {
  if (L.real_is_double) {
    if (L.vec == 2) return pick_pass<double, 2>(pass, L.acc, L.block);
    if (L.vec == 1) return pick_pass<double, 1>(pass, L.acc, L.block);
  } else {
    if (L.vec == 4) return pick_pass<float, 4>(pass, L.acc, L.block);
    if (L.vec == 1) return pick_pass<float, 1>(pass, L.acc, L.block);
  }
  return nullptr;
}

}  // namespace

cudaError_t launch_stream_pass(const StreamLaunch& L, int pass_kind, cudaStream_t s) {
  const void* fn = pick_kernel(L, pass_kind);
  if (!fn || L.grid <= 0) return cudaErrorInvalidValue;
  if (L.real_is_double) {
    StreamArgs<double> a = make_args<double>(L);
    void* args[] = {&a};
    return cudaLaunchKernel(fn, dim3(L.grid), dim3(L.block), args, 0, s);
  }
  StreamArgs<float> a = make_args<float>(L);
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
    StreamArgs<double> a = make_args<double>(L);
    init_kernel<double><<<grid, block, 0, s>>>(a.x, a.y, a.w, a.pv, a.n, a.key, a.school,
                                               weight_mode, a.ph);
  } else {
    StreamArgs<float> a = make_args<float>(L);
    init_kernel<float><<<grid, block, 0, s>>>(a.x, a.y, a.w, a.pv, a.n, a.key, a.school,
                                              weight_mode, a.ph);
  }
  return cudaGetLastError();
}

cudaError_t launch_objective(const StreamLaunch& L, void* cur, cudaStream_t s) {
  const int block = 256;
  const uint64_t want = (L.n + block - 1) / block;
  const int grid = static_cast<int>(want < 4096 ? want : 4096);
  if (L.real_is_double)
    objective_kernel<double><<<grid, block, 0, s>>>(static_cast<const double*>(L.x),
                                                    static_cast<const double*>(L.y),
                                                    static_cast<double*>(cur), L.n);
  else
    objective_kernel<float><<<grid, block, 0, s>>>(static_cast<const float*>(L.x),
                                                   static_cast<const float*>(L.y),
                                                   static_cast<float*>(cur), L.n);
  return cudaGetLastError();
}

}  // namespace fsb
