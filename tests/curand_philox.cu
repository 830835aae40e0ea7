// Test helper (not part of the library): cuRAND's device Philox4_32_10,
// called as a library, evaluated for chosen keys and counters so that the
// oracle's own Philox4x32-10 (Salmon et al., SC'11) can be checked against
// an implementation it shares nothing with.
//
// cuRAND's curand_init(seed, subsequence, offset) starts the generator at
// key (seed lo32, seed hi32) and counter (offset / 4 as a 64-bit number in
// words 0-1, subsequence in words 2-3); with offset a multiple of 4 its first
// curand4() is the block at exactly that counter.
#include <cstdint>
#include <cuda_runtime.h>
#include <curand_kernel.h>

namespace {

__global__ void philox_words_kernel(const unsigned long long* seed,
                                    const unsigned long long* ctr_lo,
                                    const unsigned long long* ctr_hi, uint4* out, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  curandStatePhilox4_32_10_t st;
  curand_init(seed[i], ctr_hi[i], ctr_lo[i] * 4ull, &st);
  out[i] = curand4(&st);
}

}  // namespace

// out: 4 words per case.  ctr_lo must be below 2^62 (offset = 4 ctr_lo).
// Returns 0 or a cudaError_t value; every buffer is released on every path.
extern "C" int curand_philox_words(const unsigned long long* seed,
                                   const unsigned long long* ctr_lo,
                                   const unsigned long long* ctr_hi, unsigned int* out, int n) {
  if (n <= 0) return 0;
  const size_t b64 = sizeof(unsigned long long) * static_cast<size_t>(n);
  const size_t bout = sizeof(uint4) * static_cast<size_t>(n);
  unsigned long long *d_seed = nullptr, *d_lo = nullptr, *d_hi = nullptr;
  uint4* d_out = nullptr;
  cudaError_t e = cudaMalloc(&d_seed, b64);
  if (e == cudaSuccess) e = cudaMalloc(&d_lo, b64);
  if (e == cudaSuccess) e = cudaMalloc(&d_hi, b64);
  if (e == cudaSuccess) e = cudaMalloc(&d_out, bout);
  if (e == cudaSuccess) e = cudaMemcpy(d_seed, seed, b64, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(d_lo, ctr_lo, b64, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(d_hi, ctr_hi, b64, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) {
    philox_words_kernel<<<(n + 127) / 128, 128>>>(d_seed, d_lo, d_hi, d_out, n);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpy(out, d_out, bout, cudaMemcpyDeviceToHost);
  cudaFree(d_seed);
  cudaFree(d_lo);
  cudaFree(d_hi);
  cudaFree(d_out);
  return static_cast<int>(e);
}
