// fsb_transfer.cu -- state transfers between host and device done by the SMs.
//
// Pinned (page-locked, mapped) host memory can be read and written by kernels
// directly over the CPU-GPU link.  On GB300 a grid-stride kernel moves it at
// the copy engines' rate (measured: 211 GB/s host to device, 193 GB/s back,
// whether by cudaMemcpyAsync or by a kernel), but the first copy-engine
// transfer after a long stretch of kernels sometimes stalled: about 110 ms
// more for 4 GiB, on every other call, in either direction; kernel copies
// never did.  So fsb_create (host checkpoint) and fsb_read_state move the
// state with these kernels when every host array is pinned, and the read
// computes currentObjective on the way out, with no device staging buffer.
#include <cstdint>

#include "fsb_device.cuh"
#include "fsb_internal.h"

namespace fsb {
namespace {

constexpr int kXferThreads = 256;

template <typename Real, int VEC>
struct XferVec;
template <>
struct XferVec<float, 4> {
  using T = float4;
};
template <>
struct XferVec<double, 2> {
  using T = double2;
};
template <>
struct XferVec<float, 1> {
  using T = float;
};
template <>
struct XferVec<double, 1> {
  using T = double;
};

template <typename Real, int VEC>
__device__ __forceinline__ void ld(Real (&v)[VEC], const Real* p, uint64_t g) {
  using T = typename XferVec<Real, VEC>::T;
  *reinterpret_cast<T*>(v) = reinterpret_cast<const T*>(p)[g];
}
template <typename Real, int VEC>
__device__ __forceinline__ void st(Real* p, uint64_t g, const Real (&v)[VEC]) {
  using T = typename XferVec<Real, VEC>::T;
  reinterpret_cast<T*>(p)[g] = *reinterpret_cast<const T*>(v);
}

// Device state -> host arrays (any of them null), currentObjective
// recomputed from the position (bit-identical to every kernel's).  Groups of
// VEC fish, then the last n % VEC one per thread.
template <typename Real, int VEC>
__global__ void __launch_bounds__(kXferThreads) read_out_kernel(
    const Real* __restrict__ x, const Real* __restrict__ y, const Real* __restrict__ w,
    const Real* __restrict__ pv, Real* X, Real* Y, Real* W, Real* PV, Real* CUR, uint64_t n) {
  const uint64_t stride = static_cast<uint64_t>(gridDim.x) * kXferThreads;
  const uint64_t tid = static_cast<uint64_t>(blockIdx.x) * kXferThreads + threadIdx.x;
  const bool pos = X || Y || CUR;
  const uint64_t ng = n / VEC;
  for (uint64_t g = tid; g < ng; g += stride) {
    Real a[VEC], b[VEC];
    if (pos) {
      ld<Real, VEC>(a, x, g);
      ld<Real, VEC>(b, y, g);
      if (X) st<Real, VEC>(X, g, a);
      if (Y) st<Real, VEC>(Y, g, b);
      if (CUR) {
        Real c[VEC];
#pragma unroll
        for (int v = 0; v < VEC; ++v) c[v] = objective(a[v], b[v]);
        st<Real, VEC>(CUR, g, c);
      }
    }
    if (W) {
      ld<Real, VEC>(a, w, g);
      st<Real, VEC>(W, g, a);
    }
    if (PV) {
      ld<Real, VEC>(a, pv, g);
      st<Real, VEC>(PV, g, a);
    }
  }
  const uint64_t i = ng * VEC + tid;
  if (VEC > 1 && i < n) {
    if (X) X[i] = x[i];
    if (Y) Y[i] = y[i];
    if (CUR) CUR[i] = objective(x[i], y[i]);
    if (W) W[i] = w[i];
    if (PV) PV[i] = pv[i];
  }
}

// Host arrays -> device state (all four given).
template <typename Real, int VEC>
__global__ void __launch_bounds__(kXferThreads) copy_in_kernel(
    const Real* X, const Real* Y, const Real* W, const Real* PV, Real* __restrict__ x,
    Real* __restrict__ y, Real* __restrict__ w, Real* __restrict__ pv, uint64_t n) {
  const uint64_t stride = static_cast<uint64_t>(gridDim.x) * kXferThreads;
  const uint64_t tid = static_cast<uint64_t>(blockIdx.x) * kXferThreads + threadIdx.x;
  const uint64_t ng = n / VEC;
  for (uint64_t g = tid; g < ng; g += stride) {
    Real a[VEC];
    ld<Real, VEC>(a, X, g);
    st<Real, VEC>(x, g, a);
    ld<Real, VEC>(a, Y, g);
    st<Real, VEC>(y, g, a);
    ld<Real, VEC>(a, W, g);
    st<Real, VEC>(w, g, a);
    ld<Real, VEC>(a, PV, g);
    st<Real, VEC>(pv, g, a);
  }
  const uint64_t i = ng * VEC + tid;
  if (VEC > 1 && i < n) {
    x[i] = X[i];
    y[i] = Y[i];
    w[i] = W[i];
    pv[i] = PV[i];
  }
}

bool all_aligned(const void* const* p, int count, uintptr_t a) {
  for (int k = 0; k < count; ++k)
    if (p[k] && reinterpret_cast<uintptr_t>(p[k]) % a != 0) return false;
  return true;
}

int xfer_grid(uint64_t units) {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    sms = 1;
  const uint64_t want = (units + kXferThreads - 1) / kXferThreads;
  const uint64_t full = static_cast<uint64_t>(sms) * 8;
  return static_cast<int>(want < 1 ? 1 : (want < full ? want : full));
}

template <typename Real>
cudaError_t read_out_typed(const StreamLaunch& L, void* const out[5], cudaStream_t s) {
  const void* all[9] = {L.x, L.y, L.w, L.pv, out[0], out[1], out[2], out[3], out[4]};
  Real* o[5];
  for (int k = 0; k < 5; ++k) o[k] = static_cast<Real*>(out[k]);
  const Real* x = static_cast<const Real*>(L.x);
  const Real* y = static_cast<const Real*>(L.y);
  const Real* w = static_cast<const Real*>(L.w);
  const Real* pv = static_cast<const Real*>(L.pv);
  constexpr int V = sizeof(Real) == 4 ? 4 : 2;
  if (all_aligned(all, 9, 16)) {
    read_out_kernel<Real, V><<<xfer_grid(L.n / V + 1), kXferThreads, 0, s>>>(
        x, y, w, pv, o[0], o[1], o[2], o[3], o[4], L.n);
  } else {
    read_out_kernel<Real, 1><<<xfer_grid(L.n), kXferThreads, 0, s>>>(x, y, w, pv, o[0], o[1],
                                                                       o[2], o[3], o[4], L.n);
  }
  return cudaGetLastError();
}

template <typename Real>
cudaError_t copy_in_typed(const StreamLaunch& L, const void* const in[4], cudaStream_t s) {
  const void* all[8] = {L.x, L.y, L.w, L.pv, in[0], in[1], in[2], in[3]};
  const Real* i[4];
  for (int k = 0; k < 4; ++k) i[k] = static_cast<const Real*>(in[k]);
  Real* x = static_cast<Real*>(L.x);
  Real* y = static_cast<Real*>(L.y);
  Real* w = static_cast<Real*>(L.w);
  Real* pv = static_cast<Real*>(L.pv);
  constexpr int V = sizeof(Real) == 4 ? 4 : 2;
  if (all_aligned(all, 8, 16)) {
    copy_in_kernel<Real, V><<<xfer_grid(L.n / V + 1), kXferThreads, 0, s>>>(
        i[0], i[1], i[2], i[3], x, y, w, pv, L.n);
  } else {
    copy_in_kernel<Real, 1><<<xfer_grid(L.n), kXferThreads, 0, s>>>(i[0], i[1], i[2], i[3], x,
                                                                     y, w, pv, L.n);
  }
  return cudaGetLastError();
}

}  // namespace

void* host_view(const void* p) {
  if (!p) return nullptr;
  cudaPointerAttributes pa{};
  if (cudaPointerGetAttributes(&pa, p) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return pa.type == cudaMemoryTypeHost ? pa.devicePointer : nullptr;
}

cudaError_t launch_read_out(const StreamLaunch& L, void* const out[5], cudaStream_t s) {
  return L.real_is_double ? read_out_typed<double>(L, out, s) : read_out_typed<float>(L, out, s);
}

cudaError_t launch_copy_in(const StreamLaunch& L, const void* const in[4], cudaStream_t s) {
  return L.real_is_double ? copy_in_typed<double>(L, in, s) : copy_in_typed<float>(L, in, s);
}

}  // namespace fsb
