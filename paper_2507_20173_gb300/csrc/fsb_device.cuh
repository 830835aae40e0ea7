// fsb_device.cuh -- per-fish device arithmetic of the Fish School Behaviour
// step (arxiv 2507.20173), shared by every kernel of the library.
//
// Every floating-point operation on the per-fish path is an explicit
// round-to-nearest-even intrinsic (__fadd_rn, __fmul_rn, __fdiv_rn,
// __fsqrt_rn and their binary64 forms), which the compiler never contracts
// into FMA, so the state is bit-identical to any IEEE implementation that
// rounds once per operation in the same order.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace fsb {

// ---------------------------------------------------------------- Philox --
// Philox4x32-10, Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as
// easy as 1, 2, 3", SC'11.  A round multiplies counter words 0 and 2 by the
// two published 32-bit constants, keeps both halves of each 64-bit product,
// XORs the high halves with the other two counter words and the round key,
// and permutes; the key advances by the two published Weyl increments.
constexpr uint32_t kPhiloxMulA = 0xD2511F53u;
constexpr uint32_t kPhiloxMulB = 0xCD9E8D57u;
constexpr uint32_t kPhiloxWeyl0 = 0x9E3779B9u;
constexpr uint32_t kPhiloxWeyl1 = 0xBB67AE85u;

struct Words4 {
  uint32_t v[4];
};

__device__ __forceinline__ Words4 philox4x32_10(uint32_t c0, uint32_t c1, uint32_t c2,
                                                uint32_t c3, uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int round = 0; round < 10; ++round) {
    const uint32_t a_hi = __umulhi(kPhiloxMulA, c0);
    const uint32_t a_lo = kPhiloxMulA * c0;
    const uint32_t b_hi = __umulhi(kPhiloxMulB, c2);
    const uint32_t b_lo = kPhiloxMulB * c2;
    c0 = b_hi ^ c1 ^ k0;
    c1 = b_lo;
    c2 = a_hi ^ c3 ^ k1;
    c3 = a_lo;
    k0 += kPhiloxWeyl0;
    k1 += kPhiloxWeyl1;
  }
  Words4 r;
  r.v[0] = c0;
  r.v[1] = c1;
  r.v[2] = c2;
  r.v[3] = c3;
  return r;
}

// Counter layout of the school's draws (reading of the paper's unnamed
// generator, Sec. 2.1.1 / Sec. 2.1.2): word 0 = index low 32 bits, word 1 =
// index high 32 bits XOR school id, word 2 = step t, word 3 = domain (0
// swim, 1 initialisation).  Key = seed.  The initialisation index is the
// fish; the swim index is the fish pair i / 2, whose block of four words
// moves both fish (words 0, 1 for fish 2p, words 2, 3 for fish 2p + 1).
constexpr uint32_t kDomainSwim = 0u;
constexpr uint32_t kDomainInit = 1u;

struct Key {
  uint32_t k0, k1;
};

__device__ __forceinline__ Words4 fish_draw(Key key, uint32_t school, uint64_t i, uint32_t t,
                                            uint32_t domain) {
  return philox4x32_10(static_cast<uint32_t>(i), static_cast<uint32_t>(i >> 32) ^ school, t,
                       domain, key.k0, key.k1);
}

// The swim block of fish pair p at step t.
__device__ __forceinline__ Words4 pair_draw(Key key, uint32_t school, uint64_t p, uint32_t t) {
  return fish_draw(key, school, p, t, kDomainSwim);
}

// The two swim words of one fish, from its pair's block.
struct Words2 {
  uint32_t r0, r1;
};

__device__ __forceinline__ Words2 fish_swim_words(Key key, uint32_t school, uint64_t i,
                                                  uint32_t t) {
  const Words4 r = pair_draw(key, school, i >> 1, t);
  return (i & 1u) ? Words2{r.v[2], r.v[3]} : Words2{r.v[0], r.v[1]};
}

// ------------------------------------------------------- real arithmetic --
// Thin wrappers so one kernel template serves binary32 and binary64 state.
template <typename Real>
struct Arith;

template <>
struct Arith<float> {
  __device__ __forceinline__ static float add(float a, float b) { return __fadd_rn(a, b); }
  __device__ __forceinline__ static float sub(float a, float b) { return __fsub_rn(a, b); }
  __device__ __forceinline__ static float mul(float a, float b) { return __fmul_rn(a, b); }
  __device__ __forceinline__ static float div(float a, float b) { return __fdiv_rn(a, b); }
  __device__ __forceinline__ static float sqrt(float a) { return __fsqrt_rn(a); }
  __device__ __forceinline__ static float clamp(float v, float lo, float hi) {
    return fminf(fmaxf(v, lo), hi);
  }
  // 2u - 1 with u = (r >> 8) * 2^-24; exact: (r >> 8) - 2^23 fits 24 bits.
  __device__ __forceinline__ static float centred(uint32_t r) {
    return __fmul_rn(__int2float_rn(static_cast<int>(r >> 8) - (1 << 23)), 0x1p-23f);
  }
  __device__ __forceinline__ static float unit(uint32_t r) {
    return __fmul_rn(__uint2float_rn(r >> 8), 0x1p-24f);
  }
};

template <>
struct Arith<double> {
  __device__ __forceinline__ static double add(double a, double b) { return __dadd_rn(a, b); }
  __device__ __forceinline__ static double sub(double a, double b) { return __dsub_rn(a, b); }
  __device__ __forceinline__ static double mul(double a, double b) { return __dmul_rn(a, b); }
  __device__ __forceinline__ static double div(double a, double b) { return __ddiv_rn(a, b); }
  __device__ __forceinline__ static double sqrt(double a) { return __dsqrt_rn(a); }
  __device__ __forceinline__ static double clamp(double v, double lo, double hi) {
    return fmin(fmax(v, lo), hi);
  }
  __device__ __forceinline__ static double centred(uint32_t r) {
    return __dmul_rn(static_cast<double>(static_cast<int>(r >> 8) - (1 << 23)), 0x1p-23);
  }
  __device__ __forceinline__ static double unit(uint32_t r) {
    return __dmul_rn(static_cast<double>(r >> 8), 0x1p-24);
  }
};

// Physics constants of one school, rounded once to the state precision.
template <typename Real>
struct Physics {
  Real pond_half;  // P
  Real step;       // s
  Real w0, w_min, w_max;
  int swim_mode;   // 0: half-width s; 1: (w / w0) * s
  int feed_mode;   // 0: delta / max|delta|; 1: (prev - cur) / max(prev - cur)
};

// The physics a kernel runs with.  The model variants (weight-scaled
// swim, feeding normalised by max(prev - cur)) are read from the arguments
// only by the kernels compiled for them (VAR); the default model's kernels
// see constant zero modes, so their per-fish body carries no branch on them.
template <bool VAR, typename Real>
__device__ __forceinline__ Physics<Real> kernel_physics(const Physics<Real>& p) {
  Physics<Real> ph = p;
  if (!VAR) {
    ph.swim_mode = 0;
    ph.feed_mode = 0;
  }
  return ph;
}

// Half-width of one fish's move: s, or (w / w0) * s when the swim is
// weight-scaled (a reading of the paper's weight-dependent movement).
template <typename Real>
__device__ __forceinline__ Real swim_width(const Physics<Real>& ph, Real w) {
  using A = Arith<Real>;
  return ph.swim_mode == 0 ? ph.step : A::mul(A::div(w, ph.w0), ph.step);
}

// Objective (Sec. 2.1.1): Euclidean distance to the pond centre (origin).
template <typename Real>
__device__ __forceinline__ Real objective(Real x, Real y) {
  using A = Arith<Real>;
  return A::sqrt(A::add(A::mul(x, x), A::mul(y, y)));
}

// Swim (Sec. 2.1.2): move each coordinate by (2u - 1) * width, clamp to
// [-P, P].
template <typename Real>
__device__ __forceinline__ void swim(Real& x, Real& y, uint32_t r0, uint32_t r1, Real width,
                                     const Physics<Real>& ph) {
  using A = Arith<Real>;
  x = A::clamp(A::add(x, A::mul(A::centred(r0), width)), -ph.pond_half, ph.pond_half);
  y = A::clamp(A::add(y, A::mul(A::centred(r1), width)), -ph.pond_half, ph.pond_half);
}

// Feeding: w <- clamp(w + g / N, w_min, w_max) for N > 0, with
// (g, N) = (delta, max|delta|) or, when feeding follows the paper's eat()
// value, (prev - cur, max(prev - cur)).
template <typename Real>
__device__ __forceinline__ Real eat(Real w, Real g, Real N, const Physics<Real>& ph) {
  using A = Arith<Real>;
  return A::clamp(A::add(w, A::div(g, N)), ph.w_min, ph.w_max);
}

// Initial fish (Sec. 2.1.1): position uniform over the pond from init draw
// words 0 and 1; weight w0 (mode 0) or w0 * (0.5 + u2) (mode 1).
template <typename Real>
__device__ __forceinline__ void init_fish(Key key, uint32_t school, uint64_t i, int weight_mode,
                                          const Physics<Real>& ph, Real& x, Real& y, Real& w) {
  using A = Arith<Real>;
  const Words4 r = fish_draw(key, school, i, 0u, kDomainInit);
  x = A::mul(A::centred(r.v[0]), ph.pond_half);
  y = A::mul(A::centred(r.v[1]), ph.pond_half);
  w = weight_mode == 0 ? ph.w0 : A::mul(ph.w0, A::add(Real(0.5), A::unit(r.v[2])));
}

// ---------------------------------------------------- order-free maxima --
// |delta| >= 0 orders like its unsigned bit pattern; a signed value is mapped
// to an unsigned key that orders like the value (negative: flip all bits;
// non-negative: flip the sign bit).
__device__ __forceinline__ uint32_t abs_bits(float v) { return __float_as_uint(fabsf(v)); }
__device__ __forceinline__ unsigned long long abs_bits(double v) {
  return static_cast<unsigned long long>(__double_as_longlong(fabs(v)));
}
__device__ __forceinline__ uint32_t order_key(float v) {
  const uint32_t b = __float_as_uint(v);
  return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}
__device__ __forceinline__ unsigned long long order_key(double v) {
  const unsigned long long b = static_cast<unsigned long long>(__double_as_longlong(v));
  return (b & 0x8000000000000000ull) ? ~b : (b | 0x8000000000000000ull);
}
__device__ __forceinline__ float key_to_value(uint32_t k, float) {
  const uint32_t b = (k & 0x80000000u) ? (k & 0x7FFFFFFFu) : ~k;
  return __uint_as_float(b);
}
__device__ __forceinline__ double key_to_value(unsigned long long k, double) {
  const unsigned long long b = (k & 0x8000000000000000ull) ? (k & 0x7FFFFFFFFFFFFFFFull) : ~k;
  return __longlong_as_double(static_cast<long long>(b));
}

template <typename Real>
struct Bits;
template <>
struct Bits<float> {
  using type = uint32_t;
};
template <>
struct Bits<double> {
  using type = unsigned long long;
};

}  // namespace fsb
