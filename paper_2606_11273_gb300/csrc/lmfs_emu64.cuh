// FP64-class products on the bf16 tensor cores, exactly, from fixed-point
// digits (the splitting of Ozaki, Ogita, Oishi and Rump, "Error-free
// transformations of matrix multiplication by using fast routines of matrix
// multiplication and its applications", Numer. Algorithms 59, 2012).
//
// Used for the blocked QR's trailing updates and back substitution
// (block_update, backsub) and for the pair precompute's D Z product.
//
// A double x is written against a power-of-two bound 2^E shared by the
// entries that one dot product combines (a column of the trailing matrix, a
// reflector, a column of T^T W, a row of R's block, a row of D, a column of
// Z) as an integer X = round(x 2^(1076 - E)),
// |X| < 2^54, and X as eight balanced base-128 digits d_0..d_7 in [-64, 63]
// (X = sum_i d_i 128^i).  Every digit is an integer that bf16 holds exactly,
// every digit product is below 2^12, and a sum of them below 2^22 is exact in
// the FP32 accumulator of a bf16 mma.  So a dot product of two digit vectors
// is exact, and the dot product of the doubles is the sum, over digit levels,
// of those exact sums shifted by 7 bits a level -- formed here in 64-bit
// integers and rounded once.  Digit pairs of levels 0..8 (level = the sum of
// the two digits' places counted from the most significant) are kept; the
// rest weigh below 2^-56 of the product of the two bounds, so the result is
// as accurate as an FP64 dot product whose error is measured against the
// same bounds.
//
// The scalar steps below compile for the host too, where tests check them
// against exact integer arithmetic.
#pragma once

#include <cstdint>
#include <cstring>
#ifdef __CUDACC__
#include <cuda_bf16.h>
#endif

#ifdef __CUDACC__
#define EMU_HD __host__ __device__ __forceinline__
#else
#define EMU_HD inline
#endif

namespace lmfs {
namespace emu {

constexpr uint64_t DBIAS = 0x0081020408102040ull;   // 64 in each of the eight 7-bit fields
constexpr uint32_t MAGIC_BITS = 0x4B400000u;        // the bits of 1.5 * 2^23
constexpr float MAGIC = 12582912.0f;                 // FP32 accumulators start here: integers
                                                     // below 2^22 in magnitude then sit in
                                                     // the low mantissa bits, exactly

EMU_HD uint64_t dbits(double x) {
#ifdef __CUDA_ARCH__
  return (uint64_t)__double_as_longlong(x);
#else
  uint64_t b; std::memcpy(&b, &x, 8); return b;
#endif
}
EMU_HD double bitsd(uint64_t b) {
#ifdef __CUDA_ARCH__
  return __longlong_as_double((long long)b);
#else
  double x; std::memcpy(&x, &b, 8); return x;
#endif
}
EMU_HD uint32_t fbits(float f) {
#ifdef __CUDA_ARCH__
  return __float_as_uint(f);
#else
  uint32_t u; std::memcpy(&u, &f, 4); return u;
#endif
}
EMU_HD float bitsf(uint32_t u) {
#ifdef __CUDA_ARCH__
  return __uint_as_float(u);
#else
  float f; std::memcpy(&f, &u, 4); return f;
#endif
}
EMU_HD int clz64(uint64_t v) {
#ifdef __CUDA_ARCH__
  return __clzll((long long)v);
#else
  return v ? __builtin_clzll(v) : 64;
#endif
}

// The biased exponent field of x (0 for zero and subnormals).
EMU_HD int bexp(double x) { return (int)((dbits(x) >> 52) & 0x7FF); }

// x against the bound 2^(E - 1023) (E a biased exponent no smaller than
// x's, and at least 64): X = round(x 2^(1076 - E)) with ties away from
// zero, |X| < 2^54, returned as DBIAS + X, whose eight 7-bit fields are the
// digits plus 64.  Zero and subnormals (biased exponent 0) give 0: with
// E >= 64 their shift reaches past all 55 bits.
EMU_HD uint64_t fixpt(double x, int E) {
  const uint64_t b = dbits(x);
  const int ex = (int)((b >> 52) & 0x7FF);
  const uint64_t m4 = ((b & 0x000FFFFFFFFFFFFFull) | 0x0010000000000000ull) << 2;
  int d = E - ex;
  d = d < 0 ? 0 : (d > 63 ? 63 : d);
  const uint64_t mag = ((m4 >> d) + 1ull) >> 1;
  return (b >> 63) ? DBIAS - mag : DBIAS + mag;
}

// Digit (0 = least significant .. 7) of a biased fixed-point value.
EMU_HD int digit(uint64_t y, int i) { return (int)((y >> (7 * i)) & 127u) - 64; }

// The digits at bit offset sh (a multiple of 7, below 56) of two biased
// values as a bf16 pair (y0 in the low half).  On the device: the bits
// 0x4300 | u are the bf16 of 128 + u (exponent 2^7, the 7 digit bits as
// mantissa), so two digits placed in the two halves and one packed bf16
// subtraction of 192 give u - 64 in both halves, exactly.  On the host the
// same integers are formed in FP32 (u - 64 from the bits of 2^23 + u, whose
// upper half is then its bf16).
EMU_HD uint32_t dpair(uint64_t y0, uint64_t y1, int sh) {
#ifdef __CUDA_ARCH__
  const uint32_t a = (uint32_t)(y0 >> sh);
  const uint32_t b = sh >= 16 ? (uint32_t)(y1 >> (sh - 16)) : (uint32_t)(y1 << (16 - sh));
  const uint32_t w = ((a & 0x7Fu) | 0x43004300u) | (b & 0x007F0000u);
  __nv_bfloat162 v;
  std::memcpy(&v, &w, 4);
  const __nv_bfloat162 r = __hsub2(v, __floats2bfloat162_rn(192.0f, 192.0f));
  uint32_t out;
  std::memcpy(&out, &r, 4);
  return out;
#else
  const uint32_t u0 = (uint32_t)(y0 >> sh) & 127u, u1 = (uint32_t)(y1 >> sh) & 127u;
  const float f0 = bitsf(0x4B000000u + u0) - 8388672.0f;
  const float f1 = bitsf(0x4B000000u + u1) - 8388672.0f;
  return (fbits(f0) >> 16) | (fbits(f1) & 0xFFFF0000u);
#endif
}

// The integer held by an accumulator that started at MAGIC.
EMU_HD int32_t acc_int(float a) { return (int32_t)(fbits(a) - MAGIC_BITS); }

// hi * 128 + lo for two accumulators of adjacent levels (hi the heavier),
// from their bits in one wrapped 32-bit step (the true value fits 30 bits).
EMU_HD int32_t acc_pair(float hi, float lo) {
  return (int32_t)(fbits(hi) * 128u + fbits(lo) - 129u * MAGIC_BITS);
}

// v 2^e as the nearest double (ties away from zero); 0 below the normal range.
EMU_HD double i64_ldexp(int64_t v, int e) {
  if (v == 0) return 0.0;
  const uint64_t sgn = v < 0 ? 0x8000000000000000ull : 0ull;
  const uint64_t mag = v < 0 ? 0ull - (uint64_t)v : (uint64_t)v;
  const int lz = clz64(mag);
  const uint64_t nm = mag << lz;                                 // leading one at bit 63
  const uint64_t r = (nm >> 11) + ((nm >> 10) & 1ull);          // 2^52 <= r <= 2^53
  const int eb = 1086 + e - lz;                                  // biased exponent of the leading one
  if (eb < 1) return 0.0;
  if (eb > 2046) return bitsd(sgn | 0x7FF0000000000000ull);
  return bitsd(sgn | (((uint64_t)(eb - 1) << 52) + r));
}

// Level sums of W = V^T C, exactly: accumulator q = 0..8 holds level q from
// the even digits of V and level q + 1 from the odd ones, so acc_pair gives
// their sum in units of level q + 1, weight 128^(13 - q).  W_fix =
// sum_q acc_pair_q 128^(13 - q) is kept as H 2^70 + L 2^35 (two int64 words:
// levels q <= 3 in H, the rest in L; both stay below 2^59 for up to 3072
// rows).  With V against 2^0 (E = 1023) and C against its column bound E,
// W = W_fix 2^(E - 1129).
EMU_HD void w_add(int64_t& H, int64_t& L, int q, int32_t u) {
  // both weights fit 32 bits: one widening multiply-add
  if (q <= 3) H += (int64_t)u * (int32_t)(1 << (21 - 7 * q));
  else L += (int64_t)u * (int32_t)(1 << (56 - 7 * q));
}
EMU_HD double w_value(int64_t H, int64_t L, int E) {
  return i64_ldexp(H, E - 1059) + i64_ldexp(L, E - 1094);
}

// Level sums of P = V W2 (one accumulator per level lambda = 0..8) as
// P_int = (sum_lambda S_lambda 128^(14 - lambda)) / 2^50; with W2 against
// its column bound F, P = P_int 2^(F - 1079).
// The three heaviest levels fit one int32 (a most significant digit is at
// most 33 in magnitude, so over 8 reflectors their sums stay below 2^13.1,
// 2^15.1 and 2^16.1), the rest in pairs; the weights in units of P_int are
// 2^34 (levels 0-2), 2^20 (3-4), 2^6 (5-6) and 2^-8 (7-8).
EMU_HD int64_t comb_p(const float* acc) {
  const int32_t u012 = (int32_t)(fbits(acc[0]) * 16384u + fbits(acc[1]) * 128u + fbits(acc[2]) - 16513u * MAGIC_BITS);
  const int32_t u34 = acc_pair(acc[3], acc[4]), u56 = acc_pair(acc[5], acc[6]), u78 = acc_pair(acc[7], acc[8]);
  int64_t t = (int64_t)u012 * 16384 + u34;
  t = t * 16384 + u56;
  return t * 64 + (u78 >> 8);
}

#ifdef __CUDACC__
__device__ __forceinline__ void prefetch_l1(const void* p) {
  asm volatile("prefetch.global.L1 [%0];\n" ::"l"(p));
}
// (not volatile: a pure function of its operands, so the compiler may
// schedule the digit work around it)
__device__ __forceinline__ void mma16(float* d, uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3,
                                      uint32_t b0, uint32_t b1) {
  asm("mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
               "{%0,%1,%2,%3};\n"
               : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
               : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

// Shared memory (bytes) of block_update inside the caller's work region:
// the digit tiles of one row chunk, then one int per trailing column.
constexpr int UPD_KF = 12;                   // k-steps of 16 rows per accumulator flush (exact sums need <= 14)
constexpr int UPD_KS = 2 * UPD_KF;           // k-steps per staged chunk
constexpr int UPD_CH = 16 * UPD_KS;          // rows per chunk
constexpr int UPD_DG = UPD_CH * 32;          // 32-bit words of digit tiles per chunk
__host__ __device__ constexpr size_t update_smem_bytes(int wld) { return (size_t)UPD_DG * 4 + (size_t)4 * wld; }

// One block's trailing update C <- (I - V T^T V^T) C, rows s..m-1 of the ncol
// columns c0, c0 + 1, ... of A (column-major, leading dimension ld, even),
// with every product formed exactly from digits on the tensor cores:
//   W = V^T C   (GEMM1: per 8-column tile, the V digits of two places share
//                one m16 tile, so each mma serves two digit levels),
//   W2 = T^T W  (FP64, per column),
//   C -= V W2   (GEMM2: per 16-column by 8-row tile, two digit pairs of one
//                level per mma), rounded once into C.
// V (bbe <= 8 reflectors) is read from A: column s + t holds reflector t
// below the diagonal, with its unit diagonal and zeros above implied.  T is
// the RB x RB upper triangular factor (T[u * 8 + t]).  cex[c] (shared) is a
// biased-exponent bound of column c over rows >= s on entry and over rows
// >= s + bbe on return.  Wsc: 16 wld int64 of global scratch; Dg and fcx:
// update_smem_bytes(wld) of shared memory.  s is even, as are ld and the
// column addresses, so that row pairs load as 16-byte words.
template <int NT>
__device__ void block_update(double* __restrict__ A, int ld, int m, int s, int bbe, int c0, int ncol,
                             const double* T, int* cex, int64_t* __restrict__ Wsc, int wld, uint32_t* Dg,
                             int* fcx) {
  constexpr int NW = NT / 32, KS = UPD_KS, KF = UPD_KF, CH = UPD_CH, NR8 = CH / 8;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, g = lane >> 2, t4 = lane & 3;
  const int nch = (m - s + CH - 1) / CH;
  int64_t* WH = Wsc;
  int64_t* WL = Wsc + 8LL * wld;
  auto vval = [&](int t, int i) -> double {
    if (t >= bbe || i >= m || i < s + t) return 0.0;
    return i == s + t ? 1.0 : A[(long long)(s + t) * ld + i];
  };

  // ---- GEMM1, chunk by chunk of rows: the V digits of the chunk staged in
  // the A-fragment order (word (k-step, place, row half, lane)), then each
  // warp's 8-column tiles, their sums added into WH / WL
  const int nt8 = (ncol + 7) >> 3;
  for (int ch = 0; ch < nch; ++ch) {
    const int rb = s + CH * ch;
    __syncthreads();
    for (int u = tid; u < KS * 32; u += NT) {
      const int ks = u >> 5, ln = u & 31, gg = ln >> 2, tt = ln & 3;
      const int r = rb + 16 * ks + 2 * tt;
      const uint64_t y0 = fixpt(vval(gg, r), 1023), y1 = fixpt(vval(gg, r + 1), 1023);
      const uint64_t y2 = fixpt(vval(gg, r + 8), 1023), y3 = fixpt(vval(gg, r + 9), 1023);
      uint32_t* D = Dg + ks * 512 + ln;
#pragma unroll
      for (int sl = 0; sl < 8; ++sl) {
        D[(2 * sl) * 32] = dpair(y0, y1, 7 * (7 - sl));
        D[(2 * sl + 1) * 32] = dpair(y2, y3, 7 * (7 - sl));
      }
    }
    __syncthreads();
    const int kss = min(KS, (m - rb + 15) >> 4);
    for (int j8 = warp; j8 < nt8; j8 += NW) {
      const int lc = 8 * j8 + g;                          // the column this lane loads
      const bool cv = lc < ncol;
      const double* col = A + (long long)(c0 + (cv ? lc : 0)) * ld;
      const int E = cv ? max(cex[c0 + lc], 64) : 64;
      if (cv) {
        // the first three k-steps' lines; each step then asks for the one three ahead
        if (rb + 2 * t4 < m) prefetch_l1(col + rb + 2 * t4);
        if (rb + 16 + 2 * t4 < m) prefetch_l1(col + rb + 16 + 2 * t4);
        if (rb + 32 + 2 * t4 < m) prefetch_l1(col + rb + 32 + 2 * t4);
      }
      // this lane: reflector g, tile columns 2 t4 and 2 t4 + 1
      int64_t h0 = 0, l0 = 0, h1 = 0, l1 = 0;
      for (int k0 = 0; k0 < kss; k0 += KF) {
      float acc[9][4];
#pragma unroll
      for (int q = 0; q < 9; ++q) acc[q][0] = acc[q][1] = acc[q][2] = acc[q][3] = MAGIC;
      const int k1 = min(kss, k0 + KF);
      for (int ks = k0; ks < k1; ++ks) {
        const int r = rb + 16 * ks + 2 * t4;
        if (cv && r + 48 < m) prefetch_l1(col + r + 48);
        double x0 = 0.0, x1 = 0.0, x2 = 0.0, x3 = 0.0;
        if (cv) {
          if (r + 1 < m) { const double2 v = *reinterpret_cast<const double2*>(col + r); x0 = v.x; x1 = v.y; }
          else if (r < m) x0 = col[r];
          if (r + 9 < m) { const double2 v = *reinterpret_cast<const double2*>(col + r + 8); x2 = v.x; x3 = v.y; }
          else if (r + 8 < m) x2 = col[r + 8];
        }
        const uint64_t y0 = fixpt(x0, E), y1 = fixpt(x1, E), y2 = fixpt(x2, E), y3 = fixpt(x3, E);
        uint32_t bl[8], bh[8];
#pragma unroll
        for (int sl = 0; sl < 8; ++sl) {
          bl[sl] = dpair(y0, y1, 7 * (7 - sl));
          bh[sl] = dpair(y2, y3, 7 * (7 - sl));
        }
        const uint32_t* D = Dg + ks * 512 + lane;
#pragma unroll
        for (int p = 0; p < 4; ++p) {
          // rows 0-7: reflectors with V place 2p; rows 8-15: the same with place 2p + 1
          const uint32_t a0 = D[(4 * p) * 32], a1 = D[(4 * p + 2) * 32];
          const uint32_t a2 = D[(4 * p + 1) * 32], a3 = D[(4 * p + 3) * 32];
#pragma unroll
          for (int q = 2 * p; q < 9; ++q)
            if (q - 2 * p <= 7) mma16(acc[q], a0, a1, a2, a3, bl[q - 2 * p], bh[q - 2 * p]);
        }
      }
#pragma unroll
      for (int q = 0; q < 9; ++q) {
        w_add(h0, l0, q, acc_pair(acc[q][0], acc[q][2]));
        w_add(h1, l1, q, acc_pair(acc[q][1], acc[q][3]));
      }
      }
      const int lw = 8 * j8 + 2 * t4;
      if (g < bbe && lw < ncol) {
        int64_t* ph = WH + (long long)g * wld + lw;
        int64_t* pl = WL + (long long)g * wld + lw;
        const bool two = lw + 1 < ncol;
        if (ch) {
          h0 += ph[0]; l0 += pl[0];
          if (two) { h1 += ph[1]; l1 += pl[1]; }
        }
        ph[0] = h0; pl[0] = l0;
        if (two) { ph[1] = h1; pl[1] = l1; }
      }
    }
  }
  __syncthreads();

  // ---- W2 = T^T W per column (FP64), its bound, and the column bound reset
  double* W2 = reinterpret_cast<double*>(Wsc);            // [8][wld] over WH
  for (int lc = tid; lc < ncol; lc += NT) {
    const int c = c0 + lc;
    const int E = cex[c];
    double w[8];
#pragma unroll
    for (int u = 0; u < 8; ++u)
      w[u] = u < bbe ? w_value(WH[(long long)u * wld + lc], WL[(long long)u * wld + lc], E) : 0.0;
    int F = 64;
#pragma unroll
    for (int t = 0; t < 8; ++t) {
      double acc = 0.0;
#pragma unroll
      for (int u = 0; u <= t; ++u) acc = fma(T[u * 8 + t], w[u], acc);
      W2[(long long)t * wld + lc] = acc;                  // zero for t >= bbe
      F = max(F, bexp(acc));
    }
    fcx[lc] = F;
    cex[c] = 0;
  }
  __syncthreads();

  // ---- GEMM2 and the update, chunk by chunk: V digits staged in the
  // B-fragment order (word (8-row tile, place, lane)); each warp's 16-column
  // tiles take the W2 digits of their columns once per chunk
  const int nt16 = (ncol + 15) >> 4;
  const int rlo = s + bbe;
  for (int ch = 0; ch < nch; ++ch) {
    const int rb = s + CH * ch;
    __syncthreads();
    for (int u = tid; u < NR8 * 32; u += NT) {
      const int nt = u >> 5, ln = u & 31, gg = ln >> 2, tt = ln & 3;
      const int r = rb + 8 * nt + gg;
      const uint64_t y0 = fixpt(vval(2 * tt, r), 1023), y1 = fixpt(vval(2 * tt + 1, r), 1023);
      uint32_t* D = Dg + nt * 256 + ln;
#pragma unroll
      for (int sl = 0; sl < 8; ++sl) D[sl * 32] = dpair(y0, y1, 7 * (7 - sl));
    }
    __syncthreads();
    const int nts = min(NR8, (m - rb + 7) >> 3);
    for (int j16 = warp; j16 < nt16; j16 += NW) {
      const int la = 16 * j16 + g, lb = la + 8;
      const bool va = la < ncol, vb = lb < ncol;
      const int fa = va ? fcx[la] : 64, fb = vb ? fcx[lb] : 64;
      const int t0 = 2 * t4;
      uint32_t Ra[8], Rb[8];
      {
        const double wa0 = va ? W2[(long long)t0 * wld + la] : 0.0, wa1 = va ? W2[(long long)(t0 + 1) * wld + la] : 0.0;
        const double wb0 = vb ? W2[(long long)t0 * wld + lb] : 0.0, wb1 = vb ? W2[(long long)(t0 + 1) * wld + lb] : 0.0;
        const uint64_t ya0 = fixpt(wa0, fa), ya1 = fixpt(wa1, fa), yb0 = fixpt(wb0, fb), yb1 = fixpt(wb1, fb);
#pragma unroll
        for (int sl = 0; sl < 8; ++sl) {
          Ra[sl] = dpair(ya0, ya1, 7 * (7 - sl));
          Rb[sl] = dpair(yb0, yb1, 7 * (7 - sl));
        }
      }
      double* cola = A + (long long)(c0 + (va ? la : 0)) * ld;
      double* colb = A + (long long)(c0 + (vb ? lb : 0)) * ld;
      int mxa = 0, mxb = 0;
      if (rb + 2 * t4 < m) {
        if (va) prefetch_l1(cola + rb + 2 * t4);
        if (vb) prefetch_l1(colb + rb + 2 * t4);
      }
      for (int nt = 0; nt < nts; ++nt) {
        const int r = rb + 8 * nt + 2 * t4;
        if (r + 8 < m) {
          if (va) prefetch_l1(cola + r + 8);
          if (vb) prefetch_l1(colb + r + 8);
        }
        // this tile's C before its products, so that the loads overlap them
        double2 xa = make_double2(0.0, 0.0), xb = make_double2(0.0, 0.0);
        if (r + 1 < m) {
          if (va) xa = *reinterpret_cast<const double2*>(cola + r);
          if (vb) xb = *reinterpret_cast<const double2*>(colb + r);
        } else if (r < m) {
          if (va) xa.x = cola[r];
          if (vb) xb.x = colb[r];
        }
        const uint32_t* D = Dg + nt * 256 + lane;
        uint32_t Q[8];
#pragma unroll
        for (int sl = 0; sl < 8; ++sl) Q[sl] = D[sl * 32];
        float acc[9][4];
#pragma unroll
        for (int q = 0; q < 9; ++q) acc[q][0] = acc[q][1] = acc[q][2] = acc[q][3] = MAGIC;
#pragma unroll
        for (int lam = 0; lam < 9; ++lam) {
          const int alo = lam > 7 ? lam - 7 : 0, ahi = lam < 7 ? lam : 7;
#pragma unroll
          for (int a = alo; a <= ahi; a += 2) {
            if (a + 1 <= ahi) mma16(acc[lam], Ra[a], Rb[a], Ra[a + 1], Rb[a + 1], Q[lam - a], Q[lam - a - 1]);
            else mma16(acc[lam], Ra[a], Rb[a], 0u, 0u, Q[lam - a], 0u);
          }
        }
        auto pval = [&](int e, int f) {
          float av[9];
#pragma unroll
          for (int q = 0; q < 9; ++q) av[q] = acc[q][e];
          return i64_ldexp(comb_p(av), f - 1079);
        };
        if (va && r < m) {
          xa.x -= pval(0, fa);
          if (r + 1 < m) {
            xa.y -= pval(1, fa);
            *reinterpret_cast<double2*>(cola + r) = xa;
            if (r + 1 >= rlo) mxa = max(mxa, bexp(xa.y));
          } else {
            cola[r] = xa.x;
          }
          if (r >= rlo) mxa = max(mxa, bexp(xa.x));
        }
        if (vb && r < m) {
          xb.x -= pval(2, fb);
          if (r + 1 < m) {
            xb.y -= pval(3, fb);
            *reinterpret_cast<double2*>(colb + r) = xb;
            if (r + 1 >= rlo) mxb = max(mxb, bexp(xb.y));
          } else {
            colb[r] = xb.x;
          }
          if (r >= rlo) mxb = max(mxb, bexp(xb.x));
        }
      }
      mxa = max(mxa, __shfl_xor_sync(0xffffffffu, mxa, 1));
      mxa = max(mxa, __shfl_xor_sync(0xffffffffu, mxa, 2));
      mxb = max(mxb, __shfl_xor_sync(0xffffffffu, mxb, 1));
      mxb = max(mxb, __shfl_xor_sync(0xffffffffu, mxb, 2));
      if (t4 == 0) {
        if (va) atomicMax(cex + c0 + la, mxa);
        if (vb) atomicMax(cex + c0 + lb, mxb);
      }
    }
  }
  __syncthreads();
}

// Shared memory (bytes) of backsub inside the caller's work region: the
// reciprocal diagonal, one block of solved rows (8 x k), the digit tiles of
// one row chunk, the chunk's row bounds and the block's column bounds.
__host__ __device__ constexpr size_t backsub_smem_bytes(int r, int k) {
  return (size_t)8 * r + (size_t)64 * k + (size_t)UPD_DG * 4 + (size_t)4 * UPD_CH + (size_t)4 * k;
}

// Back substitution R X = Y for the k right-hand sides in columns n .. n+k-1
// of A (rows 0 .. r-1, overwritten by X), R the upper triangle of A's first r
// columns: blocks of 8 rows from the bottom, each solved in FP64 (a thread
// per right-hand side, the reciprocal diagonal), then taken out of the rows
// above, Y[0:j0] -= R[0:j0, j0:j0+8] X_b, as exact digit products on the
// tensor cores like GEMM2 of block_update -- R's digits against the largest
// entry of their row in the block, X_b's against its column's.  smw: the
// work region, backsub_smem_bytes(r, k) bytes.
template <int NT>
__device__ void backsub(double* __restrict__ A, int ld, int r, int n, int k, double* smw) {
  constexpr int NW = NT / 32, CH = UPD_CH, NR8 = CH / 8;
  static_assert((NR8 * 32) % NT == 0, "staging loop: every lane takes the same number of steps");
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, g = lane >> 2, t4 = lane & 3;
  double* rinv = smw;                                     // [r]
  double* Xb = rinv + r;                                  // [8][k]
  uint32_t* Dg = reinterpret_cast<uint32_t*>(Xb + 8 * k); // UPD_DG words
  int* Ei = reinterpret_cast<int*>(Dg + UPD_DG);          // [CH]
  int* fcx = Ei + CH;                                     // [k]
  for (int j = tid; j < r; j += NT) rinv[j] = 1.0 / A[(long long)j * ld + j];
  __syncthreads();
  const int nt16 = (k + 15) >> 4;
  for (int j1 = r; j1 > 0;) {
    const int j0 = max(0, j1 - 8), bw = j1 - j0;
    // the block's rows of X, per right-hand side
    for (int c = tid; c < k; c += NT) {
      double* yc = A + (long long)(n + c) * ld;
      double y[8];
#pragma unroll
      for (int t = 0; t < 8; ++t) y[t] = t < bw ? yc[j0 + t] : 0.0;
#pragma unroll
      for (int t = 7; t >= 0; --t) {
        if (t < bw) {
          const double x = y[t] * rinv[j0 + t];
          y[t] = x;
          const double* rc = A + (long long)(j0 + t) * ld + j0;
#pragma unroll
          for (int u = 0; u < t; ++u) y[u] = fma(-rc[u], x, y[u]);
        }
      }
      int F = 64;
#pragma unroll
      for (int t = 0; t < 8; ++t) {
        Xb[t * k + c] = t < bw ? y[t] : 0.0;
        if (t < bw) {
          yc[j0 + t] = y[t];
          F = max(F, bexp(y[t]));
        }
      }
      fcx[c] = F;
    }
    __syncthreads();
    for (int rb = 0; rb < j0; rb += CH) {
      // R's digits for rows rb .. rb + CH - 1 in the B-fragment order, each
      // row against its largest entry among the block's columns
      for (int u = tid; u < NR8 * 32; u += NT) {
        const int nt = u >> 5, ln = u & 31, gg = ln >> 2, tt = ln & 3;
        const int i = rb + 8 * nt + gg;
        const double v0 = (i < j0 && 2 * tt < bw) ? A[(long long)(j0 + 2 * tt) * ld + i] : 0.0;
        const double v1 = (i < j0 && 2 * tt + 1 < bw) ? A[(long long)(j0 + 2 * tt + 1) * ld + i] : 0.0;
        int e = max(max(bexp(v0), bexp(v1)), 64);
        e = max(e, __shfl_xor_sync(0xffffffffu, e, 1));
        e = max(e, __shfl_xor_sync(0xffffffffu, e, 2));
        if (tt == 0) Ei[8 * nt + gg] = e;
        const uint64_t y0 = fixpt(v0, e), y1 = fixpt(v1, e);
        uint32_t* D = Dg + nt * 256 + ln;
#pragma unroll
        for (int sl = 0; sl < 8; ++sl) D[sl * 32] = dpair(y0, y1, 7 * (7 - sl));
      }
      __syncthreads();
      const int nts = min(NR8, (j0 - rb + 7) >> 3);
      for (int j16 = warp; j16 < nt16; j16 += NW) {
        const int la = 16 * j16 + g, lb = la + 8;
        const bool va = la < k, vb = lb < k;
        const int fa = va ? fcx[la] : 64, fb = vb ? fcx[lb] : 64;
        const int t0 = 2 * t4;
        uint32_t Ra[8], Rb[8];
        {
          const double wa0 = va ? Xb[t0 * k + la] : 0.0, wa1 = va ? Xb[(t0 + 1) * k + la] : 0.0;
          const double wb0 = vb ? Xb[t0 * k + lb] : 0.0, wb1 = vb ? Xb[(t0 + 1) * k + lb] : 0.0;
          const uint64_t ya0 = fixpt(wa0, fa), ya1 = fixpt(wa1, fa), yb0 = fixpt(wb0, fb), yb1 = fixpt(wb1, fb);
#pragma unroll
          for (int sl = 0; sl < 8; ++sl) {
            Ra[sl] = dpair(ya0, ya1, 7 * (7 - sl));
            Rb[sl] = dpair(yb0, yb1, 7 * (7 - sl));
          }
        }
        double* cola = A + (long long)(n + (va ? la : 0)) * ld;
        double* colb = A + (long long)(n + (vb ? lb : 0)) * ld;
        for (int nt = 0; nt < nts; ++nt) {
          const int i = rb + 8 * nt + 2 * t4;             // this lane's rows i, i + 1
          double2 xa = make_double2(0.0, 0.0), xb = make_double2(0.0, 0.0);
          if (i + 1 < j0) {
            if (va) xa = *reinterpret_cast<const double2*>(cola + i);
            if (vb) xb = *reinterpret_cast<const double2*>(colb + i);
          } else if (i < j0) {
            if (va) xa.x = cola[i];
            if (vb) xb.x = colb[i];
          }
          const uint32_t* D = Dg + nt * 256 + lane;
          uint32_t Q[8];
#pragma unroll
          for (int sl = 0; sl < 8; ++sl) Q[sl] = D[sl * 32];
          float acc[9][4];
#pragma unroll
          for (int q = 0; q < 9; ++q) acc[q][0] = acc[q][1] = acc[q][2] = acc[q][3] = MAGIC;
#pragma unroll
          for (int lam = 0; lam < 9; ++lam) {
            const int alo = lam > 7 ? lam - 7 : 0, ahi = lam < 7 ? lam : 7;
#pragma unroll
            for (int a = alo; a <= ahi; a += 2) {
              if (a + 1 <= ahi) mma16(acc[lam], Ra[a], Rb[a], Ra[a + 1], Rb[a + 1], Q[lam - a], Q[lam - a - 1]);
              else mma16(acc[lam], Ra[a], Rb[a], 0u, 0u, Q[lam - a], 0u);
            }
          }
          auto pval = [&](int e, int f) {
            float av[9];
#pragma unroll
            for (int q = 0; q < 9; ++q) av[q] = acc[q][e];
            return i64_ldexp(comb_p(av), f - 2102);
          };
          const int e0 = Ei[i - rb], e1 = Ei[i + 1 - rb];
          if (i < j0) {
            if (va) xa.x -= pval(0, fa + e0);
            if (vb) xb.x -= pval(2, fb + e0);
            if (i + 1 < j0) {
              if (va) { xa.y -= pval(1, fa + e1); *reinterpret_cast<double2*>(cola + i) = xa; }
              if (vb) { xb.y -= pval(3, fb + e1); *reinterpret_cast<double2*>(colb + i) = xb; }
            } else {
              if (va) cola[i] = xa.x;
              if (vb) colb[i] = xb.x;
            }
          }
        }
      }
      __syncthreads();
    }
    j1 = j0;
  }
}
#endif

}  // namespace emu
}  // namespace lmfs
