// device_math.cuh -- per-element math of GenCD on the GPU.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace gencd {

// Section 1 losses.  t is the fitted value (Xw)_i.
__device__ __forceinline__ double loss_value(int loss, double y, double t) {
  if (loss == 0) {  // squared: (y - t)^2 / 2
    double r = y - t;
    return 0.5 * r * r;
  }
  double m = -y * t;  // logistic: log(1 + e^m), overflow-free on both sides of 0
  return m > 0.0 ? m + log1p(exp(-m)) : log1p(exp(m));
}

// Derivative of the loss in t, u_i = l'(y_i, z_i): t - y (squared),
// -y / (1 + e^{y t}) (logistic).
__device__ __forceinline__ double loss_deriv(int loss, double y, double t) {
  if (loss == 0) return t - y;
  double m = y * t;
  if (m > 0.0) {
    double e = exp(-m);
    return -y * e / (1.0 + e);
  }
  return -y / (1.0 + exp(m));
}

// Convex conjugate of the loss in t, l*(y, v) = sup_t (v t - l(y, t)) (the
// dual of Eq. 1, for the duality gap): squared v y + v^2 / 2; logistic
// p log p + (1 - p) log(1 - p) with p = -y v in [0, 1] (0 log 0 = 0; the
// dual points used here keep p in [0, 1]).
__device__ __forceinline__ double loss_conjugate(int loss, double y, double v) {
  if (loss == 0) return v * y + 0.5 * v * v;
  double p = -y * v;
  p = p < 0.0 ? 0.0 : (p > 1.0 ? 1.0 : p);
  const double a = p > 0.0 ? p * log(p) : 0.0;
  const double b = p < 1.0 ? (1.0 - p) * log1p(-p) : 0.0;
  return a + b;
}

// u_i in the storage precision of u: FP64 mode evaluates l' in FP64; FP32 mode
// evaluates the logistic derivative in FP32 arithmetic (its result is stored
// in FP32 anyway), from the FP64 fitted value.
template <typename U>
__device__ __forceinline__ U u_value(int loss, double y, double t);

template <>
__device__ __forceinline__ double u_value<double>(int loss, double y, double t) {
  return loss_deriv(loss, y, t);
}

template <>
__device__ __forceinline__ float u_value<float>(int loss, double y, double t) {
  if (loss == 0) return (float)(t - y);
  const float yf = (float)y;
  const float m = (float)(y * t);
  if (m > 0.0f) {
    const float e = expf(-m);
    return -yf * e / (1.0f + e);
  }
  return -yf / (1.0f + expf(m));
}

// Eq. 7 step and Eq. 9 proxy for coordinate j from its gradient g, weight
// wj, curvature bound bj = beta_j and ibj = 1/beta_j:
//   delta = -psi(w_j; (g - lam)/b, (g + lam)/b),
//   phi   = b/2 delta^2 + g delta + lam (|w_j + delta| - |w_j|).
// For b > 0 the clip is tested in multiplied form (w b < g - lam, w b > g + lam)
// and the bound is applied with the precomputed 1/b: no FP64 divisions, the
// same step up to rounding.  |w + delta| - |w| is taken as sign(w) delta
// (exact) while w + delta keeps the sign of w, so that a small negative proxy
// is not lost to cancellation near the optimum; the sign tests use the bit
// patterns.  bj == 0 only for a column without non-zeros, whose coordinate
// does not enter F: the step is the minimiser of lam |w_j + delta|.
__device__ __forceinline__ void eq7_step(double g, double wj, double lam, double bj, double ibj, double& d,
                                         double& phi) {
  if (bj > 0.0) {
    const double t = wj * bj;
    const double lo = g - lam, hi = g + lam;
    d = t < lo ? -lo * ibj : (t > hi ? -hi * ibj : -wj);
  } else {
    d = -wj;
  }
  const double x = wj + d;
  const uint64_t sw = (uint64_t)__double_as_longlong(wj), sx = (uint64_t)__double_as_longlong(x);
  const bool keep = (sw << 1) != 0 && (((sw ^ sx) >> 63) == 0 || (sx << 1) == 0);
  const double dabs = keep ? ((sw >> 63) ? -d : d) : fabs(x) - fabs(wj);
  phi = bj > 0.0 ? d * fma(0.5 * bj, d, g) + lam * dabs : -lam * fabs(wj);
}

// Accept candidates.  Only a proxy phi < 0 can be accepted; among negative
// doubles the order of phi is the reverse of the order of |phi|'s bit pattern,
// so "lowest phi, then lowest column" becomes "largest magnitude bits, then
// lowest column" -- integer compares, no FP64 instructions.  mag = 0 means
// "no candidate" (phi >= 0, -0, or NaN).
__device__ __forceinline__ uint64_t candidate_mag(double phi) {
  const uint64_t b = (uint64_t)__double_as_longlong(phi);
  const uint64_t m = b & 0x7fffffffffffffffull;
  return ((b >> 63) && m != 0 && m <= 0x7ff0000000000000ull) ? m : 0ull;
}

// candidate_mag for an FP32 proxy (the same order on FP32 bit patterns)
__device__ __forceinline__ uint32_t candidate_mag32(float phi) {
  const uint32_t b = __float_as_uint(phi);
  const uint32_t m = b & 0x7fffffffu;
  return ((b >> 31) && m != 0 && m <= 0x7f800000u) ? m : 0u;
}

// FP32 copy of a coefficient that is 0 exactly when the coefficient is 0
// (values below the float range keep their sign at the smallest denormal)
__device__ __forceinline__ float w_mirror(double x) {
  const float f = (float)x;
  if (f != 0.0f || x == 0.0) return f;
  return x < 0.0 ? -__int_as_float(1) : __int_as_float(1);
}

// Eq. 7 / Eq. 9 in FP32 (the same steps as eq7_step): the FP32 mode uses it
// to rank the columns of a partition; the accepted column's step is then
// recomputed with eq7_step.
__device__ __forceinline__ void eq7_step_f32(float g, float wj, float lam, float bj, float ibj, float& d,
                                             float& phi) {
  if (bj > 0.0f) {
    const float t = wj * bj;
    const float lo = g - lam, hi = g + lam;
    d = t < lo ? -lo * ibj : (t > hi ? -hi * ibj : -wj);
  } else {
    d = -wj;
  }
  const float x = wj + d;
  const uint32_t sw = __float_as_uint(wj), sx = __float_as_uint(x);
  const bool keep = (sw << 1) != 0 && (((sw ^ sx) >> 31) == 0 || (sx << 1) == 0);
  const float dabs = keep ? ((sw >> 31) ? -d : d) : fabsf(x) - fabsf(wj);
  phi = bj > 0.0f ? d * fmaf(0.5f * bj, d, g) + lam * dabs : -lam * fabsf(wj);
}

__device__ __forceinline__ float kkt_violation_f32(float g, float wj, float lam) {
  const uint32_t sw = __float_as_uint(wj);
  if ((sw << 1) == 0) return fmaxf(fabsf(g) - lam, 0.0f);
  return fabsf(g + ((sw >> 31) ? -lam : lam));
}

// KKT violation of coordinate j: max(|g| - lam, 0) if w_j = 0, else
// |g + lam sign(w_j)|.
__device__ __forceinline__ double kkt_violation(double g, double wj, double lam) {
  const uint64_t sw = (uint64_t)__double_as_longlong(wj);
  if ((sw << 1) == 0) return fmax(fabs(g) - lam, 0.0);
  return fabs(g + ((sw >> 63) ? -lam : lam));
}

// SplitMix64 output i of the stream whose state starts at s
// (Steele, Lea, Flood 2014).
__host__ __device__ __forceinline__ uint64_t splitmix64_at(uint64_t s, uint64_t i) {
  uint64_t x = s + (i + 1ull) * 0x9e3779b97f4a7c15ull;
  x = (x ^ (x >> 30)) * 0xbf58476d1ce4e5b9ull;
  x = (x ^ (x >> 27)) * 0x94d049bb133111ebull;
  return x ^ (x >> 31);
}

// Non-negative doubles order like their bit patterns as unsigned integers.
__device__ __forceinline__ void atomic_max_nonneg(double* addr, double v) {
  atomicMax(reinterpret_cast<unsigned long long*>(addr),
            static_cast<unsigned long long>(__double_as_longlong(v)));
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

}  // namespace gencd
