// FP64 logarithm and reciprocal for the near field and the pair fills.
#pragma once
#include <cstdint>

namespace lmfs {

static __device__ __forceinline__ float fp32_rcp_seed(float x) {
  float y;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// Written from the mathematics, for positive normal arguments:
//  * reciprocal: an FP32 seed refined by two Newton-Raphson steps
//    y <- y + y (1 - a y); each step squares the relative error
//    (2^-22 -> 2^-44 -> below one FP64 rounding);
//  * logarithm: x = 2^e f, f in [1, 2); f = c_k (1 + t) with c_k the centre of
//    the k-th of 64 equal subintervals (c_0 = 1, so t = f - 1 exactly there),
//    |t| <= 1/64; log x = e log 2 + log c_k + log1p(t), log1p(t) from its
//    Taylor series to t^11 (the remainder is below 2^-53 |t|).  The table
//    (c_k, 1/c_k, log c_k) is built per block in shared memory.
constexpr int LOG_TAB = 64;

static __device__ __forceinline__ void log_table_init(double* tab) {
  for (int k = threadIdx.x; k < LOG_TAB; k += blockDim.x) {
    const double c = (k == 0) ? 1.0 : 1.0 + (k + 0.5) / LOG_TAB;
    tab[3 * k] = c;
    tab[3 * k + 1] = 1.0 / c;
    tab[3 * k + 2] = log(c);
  }
}

static __device__ __forceinline__ double log_pos(double x, const double* tab) {
  const long long b = __double_as_longlong(x);
  const int e = (int)(b >> 52) - 1023;
  const int k = (int)((b >> 46) & (LOG_TAB - 1));
  const double f = __longlong_as_double((b & 0x000FFFFFFFFFFFFFLL) | 0x3FF0000000000000LL);
  const double t = (f - tab[3 * k]) * tab[3 * k + 1];
  // log1p(t) = t (1 - t/2 + t^2/3 - ... - t^10/11)
  double p = -1.0 / 11.0;
  p = fma(p, t, 1.0 / 10.0);
  p = fma(p, t, -1.0 / 9.0);
  p = fma(p, t, 1.0 / 8.0);
  p = fma(p, t, -1.0 / 7.0);
  p = fma(p, t, 1.0 / 6.0);
  p = fma(p, t, -1.0 / 5.0);
  p = fma(p, t, 1.0 / 4.0);
  p = fma(p, t, -1.0 / 3.0);
  p = fma(p, t, 1.0 / 2.0);
  p = fma(p, -t, 1.0);
  return fma((double)e, 0.69314718055994530942, fma(t, p, tab[3 * k + 2]));
}

static __device__ __forceinline__ double rcp_pos(double a) {
  double y = (double)fp32_rcp_seed((float)a);
  y = fma(y, fma(-a, y, 1.0), y);
  y = fma(y, fma(-a, y, 1.0), y);
  return y;
}

}  // namespace lmfs
