// Memory-bound kernels of the density-matrix route: forming + slicing, Gershgorin bounds,
// the TRS4 trace reductions and controller, dot products, symmetrisation.
//
// All of them stream n x n FP64 matrices once.  Rows of up to kFusedMaxCols columns map to one
// block each, with every load of the row in flight at once and the row kept in registers for
// the later steps (norm, slices); wider or unaligned rows take the warp-per-row and two-pass
// kernels.  Every global access is coalesced.
#include <cmath>

#include "common.cuh"
#include "gdm_internal.h"

namespace gdm {

namespace {

constexpr int kRowThreads = 256;
constexpr int kRowsPerBlock = 8;  // one warp per row for the reductions

// ------------------------------------------------------------------------------------------
// Y = a X + b X2 + c I, optional FP64 output, optional FP16 integer slices with a power-of-two
// row scale sigma_i >= ||y_i||_2:  y = sigma 2^-11 (m_0 + m_1 2^-b + m_2 2^-2b + m_3 2^-3b ...).
// Slice 0 takes 11 bits (so its row norm is <= 2^11 and |m_0| <= 2048); every later slice takes
// b in 9..12 bits of a residual in [-1/2, 1/2] (|m_s| <= 2^(b-1) <= 2048, exact in FP16).
// Rounding: nearest-even at every slice (rint); each residual is exact in FP64.
// ------------------------------------------------------------------------------------------
__global__ void __launch_bounds__(kRowThreads)
    form_slice_kernel(const double* __restrict__ X, int64_t ldx, const double* __restrict__ X2,
                      int64_t ldx2, int rows, int cols, const double* __restrict__ coef_dev,
                      double ha, double hb, double hc, double* Y, int64_t ldy, __half* out,
                      double* out_scale, int64_t out_ld, int64_t plane, int nslice,
                      const int* skip, double step) {
  __shared__ double red[32];
  if (skip != nullptr && *skip != 0) return;
  const int row = blockIdx.x;
  if (row >= rows) return;
  double a = ha, b = hb, c = hc;
  if (coef_dev != nullptr) {
    a = coef_dev[0];
    b = coef_dev[1];
    c = coef_dev[2];
  }
  const double* xr = X + row * ldx;
  const double* x2r = (X2 != nullptr) ? X2 + row * ldx2 : nullptr;
  double* yr = (Y != nullptr) ? Y + row * ldy : nullptr;
  double ss = 0.0;
  for (int j = threadIdx.x; j < cols; j += blockDim.x) {
    double y = a * xr[j];
    if (x2r != nullptr) y += b * x2r[j];
    if (j == row) y += c;
    ss += y * y;
    if (yr != nullptr) yr[j] = y;
  }
  if (out == nullptr || nslice <= 0) return;
  ss = block_sum(ss, red);
  const double nrm = sqrt(ss);
  int e = 0;
  double scale = 0.0, sigma = 1.0;
  if (nrm > 0.0 && isfinite(nrm)) {
    frexp(nrm, &e);               // nrm = m 2^e, m in [0.5, 1)
    sigma = ldexp(1.0, e);        // sigma >= nrm
    scale = ldexp(1.0, 11 - e);   // y * scale has row norm < 2^11
  }
  if (threadIdx.x == 0) out_scale[row] = sigma;
  __half* orow = out + row * out_ld;
  for (int j = threadIdx.x; j < cols; j += blockDim.x) {
    double y;
    if (yr != nullptr) {
      y = yr[j];
    } else {
      y = a * xr[j];
      if (x2r != nullptr) y += b * x2r[j];
      if (j == row) y += c;
    }
    double x = y * scale;
    for (int s = 0; s < nslice; ++s) {
      const double m = rint(x);
      orow[s * plane + j] = __float2half_rn(static_cast<float>(m));  // exact: |m| <= 2048
      x = (x - m) * step;
    }
  }
}

// ---- FP32 double-float arithmetic: FP64-accurate reductions without the FP64 ALU ----------
// x ~ hi + lo with |x - hi - lo| < 2^-47 |x|, from the FP64 bit pattern (integer operations
// and one int->float conversion).  Magnitudes outside FP32's normal range flush to 0 (inputs
// of this engine are far from 2^-126).
__device__ __forceinline__ void split_double(double x, float& hi, float& lo) {
  const unsigned long long b = static_cast<unsigned long long>(__double_as_longlong(x));
  const int E = static_cast<int>((b >> 52) & 0x7FF);
  const unsigned sign = static_cast<unsigned>(b >> 63) << 31;
  if (E == 0x7FF) {
    hi = __uint_as_float(sign | 0x7F800000u | (((b << 12) != 0) ? 1u : 0u));
    lo = 0.0f;
    return;
  }
  const int ef = E - 1023 + 127;
  if (E == 0 || ef <= 0) {
    hi = 0.0f;
    lo = 0.0f;
    return;
  }
  if (ef >= 255) {
    hi = __uint_as_float(sign | 0x7F800000u);
    lo = 0.0f;
    return;
  }
  hi = __uint_as_float(sign | (static_cast<unsigned>(ef) << 23) |
                       static_cast<unsigned>((b >> 29) & 0x7FFFFF));
  // lo = rem * 2^(E-1075) for the 29 mantissa bits below hi, truncated to 24 bits and built
  // from its bits (no conversion instruction)
  const unsigned rem = static_cast<unsigned>(b & ((1ULL << 29) - 1));
  lo = 0.0f;
  if (rem != 0) {
    const int msb = 31 - __clz(rem);          // 0..28
    const int el = E - 1075 + msb + 127;      // biased exponent of lo
    if (el > 0) {
      const unsigned mant = (msb >= 23) ? (rem >> (msb - 23)) : (rem << (23 - msb));
      lo = __uint_as_float(sign | (static_cast<unsigned>(el) << 23) | (mant & 0x7FFFFFu));
    }
  }
}

// A split of the same kind from the two 32-bit words of the double (lo word first in memory),
// for data that is loaded and kept in integer registers: hi the top 24 significant bits, lo the
// next 23, for |x| in [2^-103, 2^128) (biased FP64 exponent E in [920, 1150]); smaller
// magnitudes, zero included, give hi = lo = 0, and larger ones, Inf and NaN give hi = NaN (a
// non-finite row either way).  Branch-free, about a dozen integer operations:
//  * hi: subtracting 896 from E rebiases the exponent to FP32's (E - 896 in [24, 254] fits the
//    8-bit field), and a funnel shift by 3 moves exponent and mantissa into FP32's places while
//    bringing in the low word's top 3 bits; the sign is put back;
//  * lo: bits 28..6 of the low word, as 2^k (1 + m 2^-23) - 2^k with 2^k (k = E - 1046) the
//    weight of bit 29, whose FP32 pattern is hi's sign and exponent less 23: one exact FP32
//    subtraction (both operands share the exponent).  |x - hi - lo| < 2^-46 |x|.
__device__ __forceinline__ void split_words(unsigned whi, unsigned wlo, float& hi, float& lo) {
  const unsigned E = (whi >> 20) & 0x7FFu;
  const bool in_range = (E - 920u) <= 230u;
  const unsigned hbits =
      (__funnelshift_l(wlo, whi - (896u << 20), 3) & 0x7FFFFFFFu) | (whi & 0x80000000u);
  const unsigned fk = (hbits & 0xFF800000u) - (23u << 23);
  const float l = __fsub_rn(__uint_as_float(fk | ((wlo >> 6) & 0x7FFFFFu)), __uint_as_float(fk));
  hi = __uint_as_float(in_range ? hbits : (E > 1150u ? 0x7FC00000u : 0u));
  lo = in_range ? l : 0.0f;
}

// x truncated to FP32 from the two words of the double (integer operations only): the top 24
// significant bits; 0 below FP32's normal range, +-Inf above it and for Inf, NaN kept.
__device__ __forceinline__ float trunc_words(unsigned whi, unsigned wlo) {
  const int E = static_cast<int>((whi >> 20) & 0x7FF);
  const unsigned sign = whi & 0x80000000u;
  const int ef = E - 1023 + 127;
  const unsigned bits = sign | (static_cast<unsigned>(ef) << 23) | ((whi & 0xFFFFFu) << 3) |
                        (wlo >> 29);
  const unsigned nan_bit = (E == 0x7FF && ((whi & 0xFFFFFu) | wlo) != 0u) ? 1u : 0u;
  const unsigned special = (E == 0x7FF || ef >= 255) ? (sign | 0x7F800000u | nan_bit) : sign;
  return __uint_as_float((E != 0 && E != 0x7FF && ef > 0 && ef < 255) ? bits : special);
}

// Sum of v over the block (FP32, a fixed order); every thread gets the result.  scratch >= 32.
__device__ __forceinline__ float block_sum_f(float v, float* scratch) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  __syncthreads();
  if (lane == 0) scratch[w] = v;
  __syncthreads();
  float t = 0.0f;
  const int nw = (blockDim.x + 31) >> 5;
  for (int j = 0; j < nw; ++j) t += scratch[j];
  return t;
}

// +-2^k x on the two words of x: only the high word changes (exponent and sign); zero and
// subnormal x give 0, results below the normal range 0 (signed), above it Inf, Inf/NaN stay.
__device__ __forceinline__ void pow2_words(unsigned& whi, unsigned& wlo, int k, bool neg) {
  const int E = static_cast<int>((whi >> 20) & 0x7FF);
  const unsigned flip = neg ? 0x80000000u : 0u;
  const unsigned sgn = (whi & 0x80000000u) ^ flip;
  const int En = E + k;
  unsigned h = sgn | (static_cast<unsigned>(En & 0x7FF) << 20) | (whi & 0xFFFFFu);
  unsigned l = wlo;
  const bool under = (E == 0) || (En <= 0);
  h = (En >= 0x7FF) ? (sgn | 0x7FF00000u) : h;
  l = (En >= 0x7FF) ? 0u : l;
  h = under ? ((E == 0) ? 0u : sgn) : h;
  l = under ? 0u : l;
  h = (E == 0x7FF) ? (whi ^ flip) : h;
  l = (E == 0x7FF) ? wlo : l;
  whi = h;
  wlo = l;
}

// Balanced base-2^bits digits of N = round(|y| 2^p) (nearest, ties to even), top digit first,
// with the sign of y applied: |y| 2^p = sum_s d[s] 2^(bits (nslice - 1 - s)), |d[s]| <= 2^(bits-1)
// for s >= 1 and |d[0]| <= 2^11 when |y| < 2^(11 + bits (nslice - 1) - p).  From the bit
// pattern yb with integer operations: the rounding is one 64-bit add and shift, each digit a
// bit field plus a carry.
// NS / BITS fix the slice count and width at compile time (0: taken from the arguments), so
// that the shifts and masks of the common formats are constants.
template <int NS, int BITS>
__device__ __forceinline__ void slice_digits_t(long long yb, int p, int nslice_rt, int bits_rt,
                                               int* d) {
  const int nslice = NS ? NS : nslice_rt;
  const int bits = BITS ? BITS : bits_rt;
  const unsigned long long ub = static_cast<unsigned long long>(yb);
  const int E = static_cast<int>((ub >> 52) & 0x7FF);
  unsigned long long mant = ub & ((1ULL << 52) - 1);
  int Ee = E;
  if (E != 0) mant |= (1ULL << 52); else Ee = 1;
  int r = 1075 - Ee - p;  // >= 6 when |y| is below the row scale (at most 36 digit bits)
  if (r < 1) r = 1;        // not reached for a valid scale; keeps the shifts defined
  unsigned long long N = 0;
  if (r < 64) N = (mant + ((1ULL << (r - 1)) - 1) + ((mant >> r) & 1ULL)) >> r;
  const int H = 1 << (bits - 1);
  const unsigned MASK = (1u << bits) - 1u;
  int carry = 0;
#pragma unroll
  for (int s = 3; s >= 1; --s) {
    if (s < nslice) {
      const int u = static_cast<int>(static_cast<unsigned>(N >> (bits * (nslice - 1 - s))) & MASK) +
                    carry;
      carry = (u >= H) ? 1 : 0;
      d[s] = u - (carry << bits);
    }
  }
  d[0] = static_cast<int>(N >> (bits * (nslice - 1))) + carry;
  if (yb < 0) {
#pragma unroll
    for (int s = 0; s < 4; ++s) d[s] = -d[s];
  }
}

__device__ __forceinline__ void slice_digits(long long yb, int p, int nslice, int bits, int* d) {
  slice_digits_t<0, 0>(yb, p, nslice, bits, d);
}

// Two integers |m| <= 2048 as an FP16 pair (low half = m0): the integers become floats by the
// 1.5 * 2^23 bias trick (an integer add and an FP32 subtract) and are packed by one conversion.
__device__ __forceinline__ uint32_t half_pair(int m0, int m1) {
  const float f0 = __int_as_float(0x4B400000 + m0) - 12582912.0f;
  const float f1 = __int_as_float(0x4B400000 + m1) - 12582912.0f;
  const __half2 h = __floats2half2_rn(f0, f1);
  return *reinterpret_cast<const uint32_t*>(&h);
}

// FP16 bit pattern of an integer |m| <= 2048 (exact), from integer operations only.
__device__ __forceinline__ uint32_t int_to_half_bits(int m) {
  if (m == 0) return 0u;
  const uint32_t sgn = (m < 0) ? 0x8000u : 0u;
  const uint32_t a = static_cast<uint32_t>(m < 0 ? -m : m);
  const int e = 31 - __clz(a);  // 0..11
  const uint32_t mant = (e <= 10) ? (a << (10 - e)) : (a >> (e - 10));
  return sgn | (static_cast<uint32_t>(e + 15) << 10) | (mant & 0x3FFu);
}

// two FP16 integers packed as a half2 word (low half = first)
__device__ __forceinline__ uint32_t pack_half_ints(long long m0, long long m1) {
  return int_to_half_bits(static_cast<int>(m0)) | (int_to_half_bits(static_cast<int>(m1)) << 16);
}

struct DF {
  float hi, lo;
};

__device__ __forceinline__ DF df_add(DF a, DF b) {
  const float s = a.hi + b.hi;
  const float bb = s - a.hi;
  const float e = (a.hi - (s - bb)) + (b.hi - bb) + a.lo + b.lo;
  const float h = s + e;
  return DF{h, e - (h - s)};
}

// acc + x * y, x and y given as (hi, lo) pairs
__device__ __forceinline__ DF df_fma(DF acc, float xh, float xl, float yh, float yl) {
  const float p = xh * yh;
  float pe = fmaf(xh, yh, -p);
  pe = fmaf(xh, yl, fmaf(xl, yh, pe));
  return df_add(acc, DF{p, pe});
}

__device__ __forceinline__ DF df_warp_sum(DF v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    DF w;
    w.hi = __shfl_xor_sync(0xffffffffu, v.hi, o);
    w.lo = __shfl_xor_sync(0xffffffffu, v.lo, o);
    v = df_add(v, w);
  }
  return v;
}

__device__ __forceinline__ double df_to_double(DF v) {
  return static_cast<double>(v.hi) + static_cast<double>(v.lo);
}

// ---- integer slicing helpers: no FP64 arithmetic (GB300 runs FP64 at ~2 DFMA/clk/SM) ----

// y truncated to FP32 from its bit pattern (integer ops only); 0 below FP32's normal range,
// inf/NaN kept.  Used for the row norm, which only has to bound ||y|| from above.
__device__ __forceinline__ float trunc_to_float(double y) {
  const unsigned long long b = static_cast<unsigned long long>(__double_as_longlong(y));
  const int E = static_cast<int>((b >> 52) & 0x7FF);
  const unsigned sign = static_cast<unsigned>(b >> 63) << 31;
  if (E == 0x7FF) return __uint_as_float(sign | 0x7F800000u | (((b << 12) != 0) ? 1u : 0u));
  const int ef = E - 1023 + 127;
  if (E == 0 || ef <= 0) return 0.0f;
  if (ef >= 255) return __uint_as_float(sign | 0x7F800000u);
  return __uint_as_float(sign | (static_cast<unsigned>(ef) << 23) |
                         static_cast<unsigned>((b >> 29) & 0x7FFFFF));
}

// round(y * 2^p) as a signed 64-bit integer (nearest, ties to even), p chosen by the caller so
// that |y * 2^p| < 2^62; exact from the bit pattern b of y.
__device__ __forceinline__ long long fixed_point_bits(long long b, int p) {
  const int E = static_cast<int>((b >> 52) & 0x7FF);
  long long mant = b & ((1LL << 52) - 1);
  int Ee = E;
  if (E != 0) mant |= (1LL << 52); else Ee = 1;
  const int sh = Ee - 1075 + p;
  long long q;
  if (sh >= 0) {
    q = mant << sh;
  } else if (sh > -63) {
    const int r = -sh;
    q = mant >> r;
    const long long rem = mant - (q << r);
    const long long half = 1LL << (r - 1);
    if (rem > half || (rem == half && (q & 1))) ++q;
  } else {
    q = 0;
  }
  return (b < 0) ? -q : q;
}

// Single-pass slicing for rows of up to 2 * 256 * MAXV columns.  The formed row stays in
// registers; loads are 16 B, slice stores 4 B per thread.  The row norm is accumulated in FP32
// from truncated values and enlarged by 0.2% before the power-of-two scale is taken, so the
// scale bounds the true norm; the slices are the balanced base-2^bits digits of
// round(y * 2^(11 - e + bits (nslice - 1))), computed with integer operations.  FP64 arithmetic
// is used only to form y when (a, b, c) is not (1, 0, 0).  Requires an even column count and
// 16-byte aligned rows (checked by the host wrapper).
template <int MAXV>
__global__ void __launch_bounds__(kRowThreads)
    form_slice_vec_kernel(const double* __restrict__ X, int64_t ldx,
                          const double* __restrict__ X2, int64_t ldx2, int rows, int cols,
                          const double* __restrict__ coef_dev, double ha, double hb, double hc,
                          double* Y, int64_t ldy, __half* out, double* out_scale, int64_t out_ld,
                          int64_t plane, int nslice, const int* skip, int bits) {
  __shared__ float redf[32];
  __shared__ int shift_sh;
  if (skip != nullptr && *skip != 0) return;
  const int row = blockIdx.x;
  if (row >= rows) return;
  double a = ha, b = hb, c = hc;
  if (coef_dev != nullptr) {
    a = coef_dev[0];
    b = coef_dev[1];
    c = coef_dev[2];
  }
  const bool plain = (a == 1.0) && (X2 == nullptr || b == 0.0) && (c == 0.0);
  const int npairs = cols >> 1;
  const double2* xr = reinterpret_cast<const double2*>(X + row * ldx);
  const double2* x2r = (X2 != nullptr) ? reinterpret_cast<const double2*>(X2 + row * ldx2)
                                        : nullptr;
  double2* yr = (Y != nullptr) ? reinterpret_cast<double2*>(Y + row * ldy) : nullptr;
  double2 v[MAXV];
  float ss = 0.0f;
#pragma unroll
  for (int i = 0; i < MAXV; ++i) {
    const int p = threadIdx.x + i * kRowThreads;
    v[i] = make_double2(0.0, 0.0);
    if (p < npairs) {
      double2 y = xr[p];
      if (!plain) {
        y.x *= a;
        y.y *= a;
        if (x2r != nullptr) {
          const double2 x2 = x2r[p];
          y.x = fma(b, x2.x, y.x);
          y.y = fma(b, x2.y, y.y);
        }
        if (2 * p == row) y.x += c;
        if (2 * p + 1 == row) y.y += c;
      }
      if (yr != nullptr) yr[p] = y;
      const float f0 = trunc_to_float(y.x), f1 = trunc_to_float(y.y);
      ss = fmaf(f0, f0, fmaf(f1, f1, ss));
      v[i] = y;
    }
  }
  if (out == nullptr || nslice <= 0) return;
  // block sum of ss (fixed order)
  {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) ss += __shfl_xor_sync(0xffffffffu, ss, o);
    if (lane == 0) redf[wid] = ss;
    __syncthreads();
    if (threadIdx.x == 0) {
      float t = 0.0f;
      for (int w = 0; w < kRowThreads / 32; ++w) t += redf[w];
      int e = 0, p = 0;
      if (t > 0.0f && isfinite(t)) {
        frexpf(sqrtf(t * 1.002f) * 1.0001f, &e);  // 2^e > ||y|| with margin
        p = 11 - e + bits * (nslice - 1);
        out_scale[row] = ldexp(1.0, e);
      } else {
        out_scale[row] = isfinite(t) ? 1.0 : __longlong_as_double(0x7FF8000000000000LL);
        p = -100000;  // all-zero slices (zero row, or a NaN/Inf row flagged by the scale)
      }
      shift_sh = p;
    }
    __syncthreads();
  }
  const int p2 = shift_sh;
  const long long H = 1LL << (bits - 1);
  const long long MASK = (1LL << bits) - 1;
  uint32_t* orow = reinterpret_cast<uint32_t*>(out + row * out_ld);
  const int64_t plane2 = plane >> 1;
#pragma unroll
  for (int i = 0; i < MAXV; ++i) {
    const int p = threadIdx.x + i * kRowThreads;
    if (p < npairs) {
      long long n0 = (p2 > -1000) ? fixed_point_bits(__double_as_longlong(v[i].x), p2) : 0;
      long long n1 = (p2 > -1000) ? fixed_point_bits(__double_as_longlong(v[i].y), p2) : 0;
      for (int s = nslice - 1; s >= 1; --s) {
        const long long d0 = ((n0 + H) & MASK) - H, d1 = ((n1 + H) & MASK) - H;
        orow[s * plane2 + p] = pack_half_ints(d0, d1);
        n0 = (n0 - d0) >> bits;
        n1 = (n1 - d1) >> bits;
      }
      orow[p] = pack_half_ints(n0, n1);
    }
  }
}

// a = +-2^k exactly?
__device__ __forceinline__ bool pow2_coef(double a, int& k, bool& neg) {
  const unsigned long long b = static_cast<unsigned long long>(__double_as_longlong(a));
  const int E = static_cast<int>((b >> 52) & 0x7FF);
  if (E == 0 || E == 0x7FF || (b & ((1ULL << 52) - 1)) != 0) return false;
  k = E - 1023;
  neg = (b >> 63) != 0;
  return true;
}

// Row pass of the slicing, one warp per row: forms y = a X + b X2 + c I when (a, b, c) is not
// (1, 0, 0) (FP64, written to Y), and writes the row scale 2^e > ||y|| from an FP32 norm of the
// truncated values enlarged by 0.2% (NaN marks a row with NaN / Inf).  With dot != kDotNone it
// also writes row_dot[row] = sum_j y_j^2 (kDotSelf), sum_j y_j X2_j (kDotX2) or sum_j y_j X_j
// (kDotX) in double-float.
// Diagonal additions are kept out of line (add_on_diagonal_words, minus_one) so that the FP64
// add is a real branch taken once per row, not an if-converted instruction on every element
// (GB300 issues FP64 at about 1/64 of the FP32 rate).

// v - 1, out of line for the same reason (the identity's diagonal in a residual)
__device__ __noinline__ double minus_one(double v) { return v - 1.0; }

enum { kFormPlain = 0, kFormPow2 = 1, kFormGeneral = 2, kFormSplit = 3 };

// kFormSplit: y = a x + b x2 (+ c on the diagonal) in FP32 double-float arithmetic straight to
// y's split (hi, lo) - for passes whose only outputs are slices, norms and row dots (no FP64
// result written, no filtering), which are cut from that split anyway.  Each product is
// Dekker's (the exact hi*hi term by an FMA, the cross terms in FP32), the sum a two-sum
// renormalised by a fast two-sum: y to ~2^-46 of |a x| + |b x2|, far below the slices' last
// digit, and no FP64 instruction (GB300 issues FP64 at ~1/64 of the FP32 rate).
struct DFCoef {
  float ah, al, bh, bl, ch, cl;
};
// The coefficients' FP32 splits from their bit patterns (split_words: 2^-46 relative), with
// integer operations only: these are block-uniform values, and GB300's FP64 pipe would hold up
// every thread of the block at its start.
__device__ __forceinline__ DFCoef df_coef(double a, double b, double c) {
  DFCoef k;
  split_words(static_cast<unsigned>(__double2hiint(a)), static_cast<unsigned>(__double2loint(a)),
              k.ah, k.al);
  split_words(static_cast<unsigned>(__double2hiint(b)), static_cast<unsigned>(__double2loint(b)),
              k.bh, k.bl);
  split_words(static_cast<unsigned>(__double2hiint(c)), static_cast<unsigned>(__double2loint(c)),
              k.ch, k.cl);
  return k;
}

// Block-uniform tests of a coefficient on its bit pattern (no FP64 compare): x == 0 (either
// sign) and x == 1.  A NaN is neither.
__device__ __forceinline__ bool coef_is_zero(double x) {
  return (static_cast<unsigned long long>(__double_as_longlong(x)) << 1) == 0ull;
}
__device__ __forceinline__ bool coef_is_one(double x) {
  return static_cast<unsigned long long>(__double_as_longlong(x)) == 0x3FF0000000000000ull;
}
// (hi, lo) = two_sum(a, b) for any a, b
__device__ __forceinline__ void two_sum_f(float a, float b, float& hi, float& lo) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  lo = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  hi = s;
}
// a x + b x2 (+ c) as a normalised pair from the splits of x and x2
__device__ __forceinline__ void df_axpby(const DFCoef& k, float xh, float xl, float x2h,
                                         float x2l, bool with_x2, bool add_c, float& yh,
                                         float& yl) {
  float p = __fmul_rn(k.ah, xh);
  float pe = __fmaf_rn(k.ah, xh, -p);
  pe = __fmaf_rn(k.ah, xl, __fmaf_rn(k.al, xh, pe));
  float s = p, e = pe;
  if (with_x2) {
    const float q = __fmul_rn(k.bh, x2h);
    float qe = __fmaf_rn(k.bh, x2h, -q);
    qe = __fmaf_rn(k.bh, x2l, __fmaf_rn(k.bl, x2h, qe));
    float t;
    two_sum_f(p, q, s, t);
    e = __fadd_rn(__fadd_rn(pe, qe), t);
  }
  if (add_c) {
    float t;
    const float s0 = s;
    two_sum_f(s0, k.ch, s, t);
    e = __fadd_rn(__fadd_rn(e, k.cl), t);
  }
  yh = __fadd_rn(s, e);
  yl = __fsub_rn(e, __fsub_rn(yh, s));
}

// y_jj + c on the word pair of a diagonal element, out of line (once per row).
__device__ __noinline__ uint2 add_on_diagonal_words(uint2 w, double c) {
  const double v = __hiloint2double(static_cast<int>(w.y), static_cast<int>(w.x)) + c;
  return make_uint2(static_cast<unsigned>(__double2loint(v)), static_cast<unsigned>(__double2hiint(v)));
}

// a x + b x2 on word pairs, the general forming step (two FP64 operations per element; a
// double-float version of it measured 4x slower: its integer reassembly of the FP64 bits costs
// more issue slots than GB300's FP64 pipe).
__device__ __forceinline__ uint2 axpby_words(double a, uint2 x, double b, uint2 x2, bool with_x2) {
  double v = a * __hiloint2double(static_cast<int>(x.y), static_cast<int>(x.x));
  if (with_x2) v = fma(b, __hiloint2double(static_cast<int>(x2.y), static_cast<int>(x2.x)), v);
  return make_uint2(static_cast<unsigned>(__double2loint(v)), static_cast<unsigned>(__double2hiint(v)));
}

// One warp's pass over a row, on integer registers throughout (16-byte loads of two doubles as
// uint4 = {lo0, hi0, lo1, hi1}): form y, write it, accumulate the FP32 norm from the truncated
// values and, for DOT != kDotNone, the double-float row dot product.  MODE picks the forming
// arithmetic: kFormPlain y = x, kFormPow2 y = +-2^k x (exponent shift), kFormGeneral
// y = a x + b x2 (FP64); c I is added out of line on the diagonal element.  Everything that
// is not FP64 arithmetic stays in integer types: on GB300 a double that takes part in integer
// selects can cost FP64-pipe instructions.
// Threshold filtering for the sparse (truncated) purification (TruncArgs, gdm_internal.h).
__device__ __forceinline__ bool filter_words(unsigned& whi, unsigned& wlo,
                                             unsigned long long tau_bits) {
  const unsigned long long mag =
      (static_cast<unsigned long long>(whi & 0x7FFFFFFFu) << 32) | wlo;
  const bool keep = mag >= tau_bits;
  whi = keep ? whi : 0u;
  wlo = keep ? wlo : 0u;
  return keep && mag != 0ull;
}

// One pair of columns (2p, 2p+1) of row `row`, on integer registers (uint4 = {lo0, hi0, lo1,
// hi1}): form y from x (and x2) by MODE, add c on the diagonal element out of line, filter it
// (truncation), write it to yr (if given) and return it in y, accumulate the FP32 norm from the
// truncated values and, for DOT != kDotNone, the double-float row dot product.  Returns whether
// the pair keeps a non-zero element (only meaningful with truncation).
template <int MODE, int DOT>
__device__ __forceinline__ bool form_pair(int p, int row, uint4 x, uint4 x2, bool with_x2,
                                          double a, double b, int ak, bool aneg, bool has_c,
                                          double c, const TruncArgs& tr, uint4* yr, uint4& y,
                                          float& ss, DF& acc, uint4* split = nullptr,
                                          const DFCoef* kc = nullptr) {
  if constexpr (MODE == kFormSplit) {
    // slices-only pass (the host picks this mode only without an FP64 output and filtering)
    const DFCoef k = (kc != nullptr) ? *kc : df_coef(a, b, c);
    float xh0, xl0, xh1, xl1, zh0 = 0.f, zl0 = 0.f, zh1 = 0.f, zl1 = 0.f;
    split_words(x.y, x.x, xh0, xl0);
    split_words(x.w, x.z, xh1, xl1);
    if (with_x2) {
      split_words(x2.y, x2.x, zh0, zl0);
      split_words(x2.w, x2.z, zh1, zl1);
    }
    float h0, l0, h1, l1;
    df_axpby(k, xh0, xl0, zh0, zl0, with_x2, has_c && 2 * p == row, h0, l0);
    df_axpby(k, xh1, xl1, zh1, zl1, with_x2, has_c && 2 * p + 1 == row, h1, l1);
    y = make_uint4(0u, 0u, 0u, 0u);
    ss = fmaf(h0, h0, fmaf(h1, h1, ss));
    if (split != nullptr)
      *split = make_uint4(__float_as_uint(h0), __float_as_uint(l0), __float_as_uint(h1),
                          __float_as_uint(l1));
    if (DOT != kDotNone) {
      float ph0 = h0, pl0 = l0, ph1 = h1, pl1 = l1;
      if (DOT == kDotX2) {
        ph0 = zh0; pl0 = zl0; ph1 = zh1; pl1 = zl1;
      } else if (DOT == kDotX) {
        ph0 = xh0; pl0 = xl0; ph1 = xh1; pl1 = xl1;
      }
      acc = df_fma(acc, h0, l0, ph0, pl0);
      acc = df_fma(acc, h1, l1, ph1, pl1);
    }
    return false;
  }
  y = x;
  if (MODE == kFormPow2) {
    pow2_words(y.y, y.x, ak, aneg);
    pow2_words(y.w, y.z, ak, aneg);
  } else if (MODE == kFormGeneral) {
    const uint2 y0 = axpby_words(a, make_uint2(x.x, x.y), b, make_uint2(x2.x, x2.y), with_x2);
    const uint2 y1 = axpby_words(a, make_uint2(x.z, x.w), b, make_uint2(x2.z, x2.w), with_x2);
    y = make_uint4(y0.x, y0.y, y1.x, y1.y);
  }
  if (has_c && (2 * p == row || 2 * p + 1 == row)) {
    if (2 * p == row) {
      const uint2 d = add_on_diagonal_words(make_uint2(y.x, y.y), c);
      y.x = d.x;
      y.y = d.y;
    } else {
      const uint2 d = add_on_diagonal_words(make_uint2(y.z, y.w), c);
      y.z = d.x;
      y.w = d.y;
    }
  }
  bool nz = false;
  if (tr.tau_bits != 0ull) {
    const bool k0 = filter_words(y.y, y.x, tr.tau_bits);
    const bool k1 = filter_words(y.w, y.z, tr.tau_bits);
    nz = k0 || k1;
  }
  if (yr != nullptr) yr[p] = y;
  float h0, l0, h1, l1;
  split_words(y.y, y.x, h0, l0);
  split_words(y.w, y.z, h1, l1);
  ss = fmaf(h0, h0, fmaf(h1, h1, ss));  // the truncated value bounds |y| from below by 2^-23
  if (split != nullptr)
    *split = make_uint4(__float_as_uint(h0), __float_as_uint(l0), __float_as_uint(h1),
                        __float_as_uint(l1));
  if (DOT != kDotNone) {
    float ph0 = h0, pl0 = l0, ph1 = h1, pl1 = l1;
    if (DOT == kDotX2) {
      split_words(x2.y, x2.x, ph0, pl0);
      split_words(x2.w, x2.z, ph1, pl1);
    } else if (DOT == kDotX) {
      split_words(x.y, x.x, ph0, pl0);
      split_words(x.w, x.z, ph1, pl1);
    }
    acc = df_fma(acc, h0, l0, ph0, pl0);
    acc = df_fma(acc, h1, l1, ph1, pl1);
  }
  return nz;
}

template <int MODE, int DOT>
__device__ __forceinline__ void form_norm_row(const uint4* __restrict__ xr,
                                              const uint4* __restrict__ x2r, uint4* yr,
                                              int npairs, int row, int lane, double a, double b,
                                              int ak, bool aneg, bool has_c, double c,
                                              const TruncArgs& tr, float& ss, DF& acc) {
  constexpr bool kNeedX2 = (MODE == kFormGeneral) || (DOT == kDotX2);
  const bool with_x2 = x2r != nullptr;
  const bool trunc = tr.tau_bits != 0ull;
  auto one = [&](int p, uint4 x, uint4 x2) -> bool {
    uint4 y;
    return form_pair<MODE, DOT>(p, row, x, x2, with_x2, a, b, ak, aneg, has_c, c, tr, yr, y, ss,
                                acc);
  };
  // Warp-uniform loops: full blocks of 32 * U column pairs (U loads in flight per lane), then
  // steps of 32 pairs.  A block of 64 pairs is one 128-column tile.
  constexpr int U = 4;
  uint32_t* mrow = (trunc && tr.mask != nullptr)
                       ? tr.mask + static_cast<int64_t>(row >> 7) * tr.mask_ld : nullptr;
  int base = 0;
  for (; base + 32 * U <= npairs; base += 32 * U) {
    uint4 xv[U], x2v[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      xv[u] = xr[base + lane + 32 * u];
      if (kNeedX2 && with_x2) x2v[u] = x2r[base + lane + 32 * u];
      else x2v[u] = make_uint4(0u, 0u, 0u, 0u);
    }
    bool nz[U];
#pragma unroll
    for (int u = 0; u < U; ++u) nz[u] = one(base + lane + 32 * u, xv[u], x2v[u]);
    if (mrow != nullptr) {
      const bool lo_blk = __any_sync(0xffffffffu, nz[0] || nz[1]);
      const bool hi_blk = __any_sync(0xffffffffu, nz[2] || nz[3]);
      if (lane == 0) {
        if (lo_blk) mrow[base >> 6] = 1u;
        if (hi_blk) mrow[(base >> 6) + 1] = 1u;
      }
    }
  }
  for (; base < npairs; base += 32) {
    const int p = base + lane;
    bool nz = false;
    if (p < npairs) {
      const uint4 x = xr[p];
      const uint4 x2 = (kNeedX2 && with_x2) ? x2r[p] : make_uint4(0u, 0u, 0u, 0u);
      nz = one(p, x, x2);
    }
    if (mrow != nullptr) {
      const bool any = __any_sync(0xffffffffu, nz);
      if (lane == 0 && any) mrow[base >> 6] = 1u;
    }
  }
}

template <int MODE>
__device__ __forceinline__ void form_norm_dispatch(int dot, const uint4* xr, const uint4* x2r,
                                                   uint4* yr, int npairs, int row, int lane,
                                                   double a, double b, int ak, bool aneg,
                                                   bool has_c, double c, const TruncArgs& tr,
                                                   float& ss, DF& acc) {
  switch (dot) {
    case kDotSelf:
      form_norm_row<MODE, kDotSelf>(xr, x2r, yr, npairs, row, lane, a, b, ak, aneg, has_c, c, tr,
                                    ss, acc);
      break;
    case kDotX2:
      form_norm_row<MODE, kDotX2>(xr, x2r, yr, npairs, row, lane, a, b, ak, aneg, has_c, c, tr,
                                  ss, acc);
      break;
    case kDotX:
      form_norm_row<MODE, kDotX>(xr, x2r, yr, npairs, row, lane, a, b, ak, aneg, has_c, c, tr,
                                 ss, acc);
      break;
    default:
      form_norm_row<MODE, kDotNone>(xr, x2r, yr, npairs, row, lane, a, b, ak, aneg, has_c, c, tr,
                                    ss, acc);
  }
}

__global__ void __launch_bounds__(kRowsPerBlock * 32, 4)
    form_norm_kernel(const double* __restrict__ X, int64_t ldx, const double* __restrict__ X2,
                     int64_t ldx2, int rows, int cols, const double* __restrict__ coef_dev,
                     double ha, double hb, double hc, double* Y, int64_t ldy, double* out_scale,
                     const int* skip, int dot, double* row_dot, TruncArgs tr) {
  if (skip != nullptr && *skip != 0) return;
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int row = blockIdx.x * kRowsPerBlock + w;
  if (row >= rows) return;
  double a = ha, b = hb, c = hc;
  if (coef_dev != nullptr) {
    a = coef_dev[0];
    b = coef_dev[1];
    c = coef_dev[2];
  }
  // the forming arithmetic, decided once per warp (uniform)
  int ak = 0;
  bool aneg = false;
  const bool no_x2 = (X2 == nullptr || coef_is_zero(b));
  const bool has_c = !coef_is_zero(c);
  int mode = kFormGeneral;
  if (no_x2 && coef_is_one(a)) mode = kFormPlain;
  else if (no_x2 && pow2_coef(a, ak, aneg)) mode = kFormPow2;
  const uint4* xr = reinterpret_cast<const uint4*>(X + row * ldx);
  const uint4* x2r = (X2 != nullptr) ? reinterpret_cast<const uint4*>(X2 + row * ldx2) : nullptr;
  uint4* yr = (Y != nullptr) ? reinterpret_cast<uint4*>(Y + row * ldy) : nullptr;
  const int npairs = cols >> 1;
  float ss = 0.0f;
  DF acc{0.0f, 0.0f};
  if (mode == kFormPlain)
    form_norm_dispatch<kFormPlain>(dot, xr, x2r, yr, npairs, row, lane, a, b, ak, aneg, has_c, c,
                                   tr, ss, acc);
  else if (mode == kFormPow2)
    form_norm_dispatch<kFormPow2>(dot, xr, x2r, yr, npairs, row, lane, a, b, ak, aneg, has_c, c,
                                  tr, ss, acc);
  else
    form_norm_dispatch<kFormGeneral>(dot, xr, x2r, yr, npairs, row, lane, a, b, ak, aneg, has_c,
                                     c, tr, ss, acc);
  if (dot != kDotNone) {
    acc = df_warp_sum(acc);
    if (lane == 0) row_dot[row] = df_to_double(acc);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) ss += __shfl_xor_sync(0xffffffffu, ss, o);
  if (lane == 0 && out_scale != nullptr) {
    if (ss > 0.0f && isfinite(ss)) {
      int e = 0;
      // the norm from truncated values is low by at most 2^-23 relative: the 0.2% margin covers
      // it and the FP32 accumulation, so 2^e > ||y||
      frexpf(sqrtf(ss * 1.002f) * 1.0001f, &e);
      out_scale[row] = __longlong_as_double(static_cast<long long>(e + 1023) << 52);  // 2^e
    } else {
      out_scale[row] = isfinite(ss) ? 1.0 : __longlong_as_double(0x7FF8000000000000LL);
    }
  }
}

// Element pass of the slicing: block (row, chunk of 2 * 256 column pairs), two pairs per thread
// with both loads issued first; the balanced base-2^bits digits of
// round(y * 2^(11 - e + bits (nslice - 1))), e from the row scale; integer only.
constexpr int kSliceThreads = 256;
constexpr int kSlicePairsPerThread = 2;
__global__ void __launch_bounds__(kSliceThreads)
    slice_pairs_kernel(const double* __restrict__ Yin, int64_t ldy, int rows, int cols,
                       const double* __restrict__ scale, __half* out, int64_t out_ld,
                       int64_t plane, int nslice, int bits, const int* skip) {
  if (skip != nullptr && *skip != 0) return;
  const int row = blockIdx.x;
  if (row >= rows) return;
  const int npairs = cols >> 1;
  const int64_t plane2 = plane >> 1;
  // the row scale and the values are handled as bit patterns: no FP64 instruction here
  const unsigned long long scb =
      static_cast<unsigned long long>(reinterpret_cast<const long long*>(scale)[row]);
  const int Es = static_cast<int>((scb >> 52) & 0x7FF);
  const bool ok = Es != 0x7FF;
  const int e = Es - 1023;
  const int p2 = 11 - e + bits * (nslice - 1);
  const longlong2* yrow = reinterpret_cast<const longlong2*>(Yin + row * ldy);
  uint32_t* orow = reinterpret_cast<uint32_t*>(out + row * out_ld);
  const int pbase = blockIdx.y * (kSliceThreads * kSlicePairsPerThread) + threadIdx.x;
  longlong2 yv[kSlicePairsPerThread];
#pragma unroll
  for (int u = 0; u < kSlicePairsPerThread; ++u) {
    const int p = pbase + u * kSliceThreads;
    yv[u] = make_longlong2(0, 0);
    if (ok && p < npairs) yv[u] = yrow[p];
  }
#pragma unroll
  for (int u = 0; u < kSlicePairsPerThread; ++u) {
    const int p = pbase + u * kSliceThreads;
    if (p >= npairs) break;
    int d0[4] = {0, 0, 0, 0}, d1[4] = {0, 0, 0, 0};
    if (ok) {
      slice_digits(yv[u].x, p2, nslice, bits, d0);
      slice_digits(yv[u].y, p2, nslice, bits, d1);
    }
#pragma unroll
    for (int s = 0; s < 4; ++s)
      if (s < nslice) orow[s * plane2 + p] = half_pair(d0[s], d1[s]);
  }
}

// Forming and slicing in one pass, one block per row: every thread loads its kFusedPPT column
// pairs at once (the whole row is in flight in one round trip), forms them in registers, writes
// Y, reduces the FP32 norm (and the row dot product) over the block in a fixed order, and
// writes the slices from the same registers, so the formed row is never read back.
constexpr int kFusedPPT = 8;
static_assert(kFusedMaxCols == 2 * 512 * kFusedPPT, "fused slicing: up to 512 threads per row");

// x rounded to an integer (nearest, ties to even) on the FP32 pipe, |x| < 2^22: the 1.5 * 2^23
// shift in two additions that the compiler may not contract or reorder.
__device__ __forceinline__ float rint_f(float x) {
  return __fsub_rn(__fadd_rn(x, 12582912.0f), 12582912.0f);
}

// Balanced digits of t = y 2^k (|t| < 2^11) from y's FP32 split y = hi + lo (split_words: hi the
// top 24 bits, lo the next 23, together y to 2^-46), on the FP32 pipe.  What remains of t after
// each digit is kept exactly as an unevaluated pair (r_hi, r_lo) with |r_lo| <= ulp(r_hi) / 2:
//   d_0 = rint(t_hi),                 (r_hi, r_lo) = two_sum(t_hi - d_0, t_lo)
//   d_s = rint(r_hi 2^b),             (r_hi, r_lo) = two_sum(r_hi 2^b - d_s, r_lo 2^b)
//   d_last = rint(r_hi 2^b + r_lo 2^b).
// Each digit is subtracted from the value it rounds, so the subtraction is exact, and the
// two-sum (Dekker's fast form: |first| >= |second| or first = 0 holds here) is exact; the digits
// therefore represent t to half a unit of the last slice (plus the split's 2^-46 |t|).  Deciding
// a digit from r_hi alone leaves at most 1/2 + 2^-13 units, so every later digit stays within
// +-2^(b-1) (2^(b-1) + 1/2 rounds to even) and d_0 within +-2^11: all exact in FP16.
template <int NS, int BITS>
__device__ __forceinline__ void slice_digits_f(float hi, float lo, float scale, int nslice_rt,
                                               int bits_rt, float* d) {
  const int nslice = NS ? NS : nslice_rt;
  const float w = NS ? static_cast<float>(1 << BITS) : __int_as_float((127 + bits_rt) << 23);
  const float th = hi * scale, tl = lo * scale;  // exact: powers of two, in FP32's range
  d[0] = rint_f(th);
  float a = __fsub_rn(th, d[0]);
  float rh = __fadd_rn(a, tl);
  float rl = __fsub_rn(tl, __fsub_rn(rh, a));
#pragma unroll
  for (int sl = 1; sl < 4; ++sl) {
    if (sl < nslice) {
      const float x = rh * w, xl = rl * w;
      if (sl == nslice - 1) {
        d[sl] = rint_f(__fadd_rn(x, xl));
      } else {
        d[sl] = rint_f(x);
        a = __fsub_rn(x, d[sl]);
        rh = __fadd_rn(a, xl);
        rl = __fsub_rn(xl, __fsub_rn(rh, a));
      }
    }
  }
}

// The slices of a row held in registers (kFusedPPT column pairs a thread, each element as its
// FP32 split (hi, lo) in the bits of v: {hi_0, lo_0, hi_1, lo_1}): digits of y 2^k with
// k = p2 - bits (nslice - 1) (p2 <= -1000: an all-zero row), written as FP16 pairs, one plane
// per slice.
template <int NS, int BITS, int THREADS>
__device__ __forceinline__ void write_row_slices(const uint4 (&v)[kFusedPPT], int npairs, int p2,
                                                 uint32_t* orow, int64_t plane2, int nslice,
                                                 int bits) {
  const int ns = NS ? NS : nslice;
  const int b = BITS ? BITS : bits;
  // k is within [-54, 85] for any finite non-zero row (the FP32 norm's range); clamped anyway
  const int k = min(max(p2 - b * (ns - 1), -126), 127);
  const float scale = __int_as_float((k + 127) << 23);
  const bool zero = p2 <= -1000;
#pragma unroll
  for (int i = 0; i < kFusedPPT; ++i) {
    const int p = i * THREADS + threadIdx.x;
    if (p < npairs) {
      float d0[4] = {0.f, 0.f, 0.f, 0.f}, d1[4] = {0.f, 0.f, 0.f, 0.f};
      if (!zero) {
        slice_digits_f<NS, BITS>(__uint_as_float(v[i].x), __uint_as_float(v[i].y), scale, ns, b,
                                 d0);
        slice_digits_f<NS, BITS>(__uint_as_float(v[i].z), __uint_as_float(v[i].w), scale, ns, b,
                                 d1);
      }
#pragma unroll
      for (int sl = 0; sl < 4; ++sl)
        if (sl < ns) {
          const __half2 hh = __floats2half2_rn(d0[sl], d1[sl]);
          orow[sl * plane2 + p] = *reinterpret_cast<const uint32_t*>(&hh);
        }
    }
  }
}

// the route's formats (Newton-Schulz 2 x 12 bits, purification 3 x 12, refinement and
// transforms 4 x 9) with constant shifts; any other format at run time
template <int THREADS>
__device__ __forceinline__ void write_row_slices_any(const uint4 (&v)[kFusedPPT], int npairs,
                                                     int p2, uint32_t* orow, int64_t plane2,
                                                     int nslice, int bits) {
  if (nslice == 3 && bits == 12)
    write_row_slices<3, 12, THREADS>(v, npairs, p2, orow, plane2, nslice, bits);
  else if (nslice == 2 && bits == 12)
    write_row_slices<2, 12, THREADS>(v, npairs, p2, orow, plane2, nslice, bits);
  else if (nslice == 4 && bits == 9)
    write_row_slices<4, 9, THREADS>(v, npairs, p2, orow, plane2, nslice, bits);
  else
    write_row_slices<0, 0, THREADS>(v, npairs, p2, orow, plane2, nslice, bits);
}

template <int MODE, int DOT, int THREADS, bool HAS_X2>
__device__ __forceinline__ void form_slice_row(const uint4* xr, const uint4* x2r, uint4* yr,
                                               int npairs, int row, double a, double b, int ak,
                                               bool aneg, bool has_c, double c,
                                               const TruncArgs& tr, __half* out, int64_t out_ld,
                                               int64_t plane, int nslice, int bits,
                                               double* out_scale, double* row_dot, float* red_ss,
                                               DF* red_dot, int* shift_sh) {
  constexpr bool kNeedX2 =
      HAS_X2 && ((MODE == kFormGeneral) || (MODE == kFormSplit) || (DOT == kDotX2));
  const bool with_x2 = HAS_X2;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  uint4 v[kFusedPPT], v2[kNeedX2 ? kFusedPPT : 1];
#pragma unroll
  for (int i = 0; i < kFusedPPT; ++i) {
    const int p = i * THREADS + threadIdx.x;
    v[i] = make_uint4(0u, 0u, 0u, 0u);
    if (p < npairs) v[i] = xr[p];
    if (kNeedX2) {
      v2[i] = make_uint4(0u, 0u, 0u, 0u);
      if (p < npairs) v2[i] = x2r[p];
    }
  }
  uint32_t* mrow = (tr.tau_bits != 0ull && tr.mask != nullptr)
                       ? tr.mask + static_cast<int64_t>(row >> 7) * tr.mask_ld : nullptr;
  float ss = 0.0f;
  DF acc{0.0f, 0.0f};
  DFCoef kc{0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
  if constexpr (MODE == kFormSplit) kc = df_coef(a, b, c);  // once per thread, not per pair
#pragma unroll
  for (int i = 0; i < kFusedPPT; ++i) {
    const int p0 = i * THREADS + w * 32;  // warp-uniform: the warp's first pair
    if (p0 < npairs) {
      const int p = p0 + lane;
      bool nz = false;
      if (p < npairs) {
        uint4 y, sp;
        nz = form_pair<MODE, DOT>(p, row, v[i], kNeedX2 ? v2[i] : v[i], with_x2, a, b, ak, aneg,
                                  has_c, c, tr, yr, y, ss, acc, &sp, &kc);
        v[i] = sp;  // from here on the row is held as its FP32 splits
      }
      if (mrow != nullptr) {
        // 32 pairs = half a 128-column tile
        const bool any = __any_sync(0xffffffffu, nz);
        if (lane == 0 && any) mrow[p0 >> 6] = 1u;
      }
    }
  }
  // block reductions in a fixed order
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) ss += __shfl_xor_sync(0xffffffffu, ss, o);
  if (DOT != kDotNone) acc = df_warp_sum(acc);
  if (lane == 0) {
    red_ss[w] = ss;
    if (DOT != kDotNone) red_dot[w] = acc;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    float t = 0.0f;
    DF d{0.0f, 0.0f};
    for (int j = 0; j < THREADS / 32; ++j) {
      t += red_ss[j];
      if (DOT != kDotNone) d = df_add(d, red_dot[j]);
    }
    if (DOT != kDotNone) row_dot[row] = df_to_double(d);
    int e = 0;
    unsigned long long scb;
    if (t > 0.0f && isfinite(t)) {
      // the norm from truncated values is low by at most 2^-23 relative: the 0.2% margin covers
      // it and the FP32 accumulation, so 2^e > ||y||
      frexpf(sqrtf(t * 1.002f) * 1.0001f, &e);
      scb = static_cast<unsigned long long>(e + 1023) << 52;  // 2^e
    } else {
      scb = isfinite(t) ? (1023ull << 52) : 0x7FF8000000000000ull;  // 1, or NaN for NaN / Inf
    }
    out_scale[row] = __longlong_as_double(static_cast<long long>(scb));
    // digits of round(y 2^(11 - e + bits (nslice - 1))); a NaN row gets all-zero slices
    shift_sh[0] = (scb >> 52 == 0x7FF) ? -100000 : 11 - e + bits * (nslice - 1);
  }
  __syncthreads();
  const int p2 = shift_sh[0];
  uint32_t* orow = reinterpret_cast<uint32_t*>(out + row * out_ld);
  const int64_t plane2 = plane >> 1;
  write_row_slices_any<THREADS>(v, npairs, p2, orow, plane2, nslice, bits);
}

template <int MODE, int THREADS, bool HAS_X2>
__device__ __forceinline__ void form_slice_dispatch(int dot, const uint4* xr, const uint4* x2r,
                                                    uint4* yr, int npairs, int row, double a,
                                                    double b, int ak, bool aneg, bool has_c,
                                                    double c, const TruncArgs& tr, __half* out,
                                                    int64_t out_ld, int64_t plane, int nslice,
                                                    int bits, double* out_scale,
                                                    double* row_dot, float* red_ss, DF* red_dot,
                                                    int* shift_sh) {
#define GDM_FSR(D)                                                                              \
  form_slice_row<MODE, D, THREADS, HAS_X2>(xr, x2r, yr, npairs, row, a, b, ak, aneg, has_c, c, tr, out, \
                                   out_ld, plane, nslice, bits, out_scale, row_dot, red_ss,     \
                                   red_dot, shift_sh)
  switch (dot) {
    case kDotSelf: GDM_FSR(kDotSelf); break;
    case kDotX2:  // needs X2 (form_and_slice refuses it without)
      if constexpr (HAS_X2) GDM_FSR(kDotX2);
      break;
    case kDotX: GDM_FSR(kDotX); break;
    default: GDM_FSR(kDotNone);
  }
#undef GDM_FSR
}

template <int THREADS, bool HAS_X2>
__global__ void __launch_bounds__(THREADS, HAS_X2 ? 1 : 1024 / THREADS)
    form_slice_fused_kernel(const double* X, int64_t ldx, const double* X2, int64_t ldx2,
                            int rows, int cols, const double* __restrict__ coef_dev, double ha,
                            double hb, double hc, double* Y, int64_t ldy, __half* out,
                            double* out_scale, int64_t out_ld, int64_t plane, int nslice,
                            int bits, const int* skip, int dot, double* row_dot, TruncArgs tr) {
  __shared__ float red_ss[THREADS / 32];
  __shared__ DF red_dot[THREADS / 32];
  __shared__ int shift_sh[1];
  if (skip != nullptr && *skip != 0) return;
  const int row = blockIdx.x;
  if (row >= rows) return;
  double a = ha, b = hb, c = hc;
  if (coef_dev != nullptr) {
    a = coef_dev[0];
    b = coef_dev[1];
    c = coef_dev[2];
  }
  // the forming arithmetic, decided once per block (uniform)
  int ak = 0;
  bool aneg = false;
  const bool no_x2 = (!HAS_X2 || coef_is_zero(b));
  const bool has_c = !coef_is_zero(c);
  int mode = kFormGeneral;
  if (no_x2 && coef_is_one(a)) mode = kFormPlain;
  else if (no_x2 && pow2_coef(a, ak, aneg)) mode = kFormPow2;
  // slices only: form in double-float (no FP64 result to write, no filtering)
  if (mode == kFormGeneral && Y == nullptr && tr.tau_bits == 0ull) mode = kFormSplit;
  const uint4* xr = reinterpret_cast<const uint4*>(X + row * ldx);
  const uint4* x2r = HAS_X2 ? reinterpret_cast<const uint4*>(X2 + row * ldx2) : nullptr;
  uint4* yr = (Y != nullptr) ? reinterpret_cast<uint4*>(Y + row * ldy) : nullptr;
  const int npairs = cols >> 1;
  if (mode == kFormSplit)
    form_slice_dispatch<kFormSplit, THREADS, HAS_X2>(dot, xr, x2r, yr, npairs, row, a, b, ak, aneg,
                                               has_c, c, tr, out, out_ld, plane, nslice, bits,
                                               out_scale, row_dot, red_ss, red_dot, shift_sh);
  else if (mode == kFormPlain)
    form_slice_dispatch<kFormPlain, THREADS, HAS_X2>(dot, xr, x2r, yr, npairs, row, a, b, ak, aneg, has_c,
                                             c, tr, out, out_ld, plane, nslice, bits, out_scale,
                                             row_dot, red_ss, red_dot, shift_sh);
  else if (mode == kFormPow2)
    form_slice_dispatch<kFormPow2, THREADS, HAS_X2>(dot, xr, x2r, yr, npairs, row, a, b, ak, aneg, has_c,
                                            c, tr, out, out_ld, plane, nslice, bits, out_scale,
                                            row_dot, red_ss, red_dot, shift_sh);
  else
    form_slice_dispatch<kFormGeneral, THREADS, HAS_X2>(dot, xr, x2r, yr, npairs, row, a, b, ak, aneg,
                                               has_c, c, tr, out, out_ld, plane, nslice, bits,
                                               out_scale, row_dot, red_ss, red_dot, shift_sh);
}

// The TRS4 trace terms and the slicing of X^2 in one pass, one block per row: X^2's row is
// sliced like form_slice_row (plain forming, no row dot), and the row's trace terms go to
// partials[row * kTraceTerms + k]: X_rr, X2_rr, <X2_r, X_r>, ||X2_r||^2, ||X_r||^2 (double-float
// sums, diagonals exact).  Both rows are read once.
template <int THREADS>
__global__ void __launch_bounds__(THREADS)
    slice_traces_kernel(const double* X2, const double* X, int64_t ld, int n, int cols,
                        __half* out, double* out_scale, int64_t out_ld, int64_t plane, int nslice,
                        int bits, double* partials, const int* skip,
                        const double* __restrict__ x_row_dot) {
  __shared__ float red_ss[THREADS / 32];
  __shared__ DF red_dot[3][THREADS / 32];
  // ||X_r||^2 is X's own row dot product when X's slicing pass left it (x_row_dot != null)
  const bool own_x_dot = (x_row_dot == nullptr);
  __shared__ unsigned long long diag_sh[2];
  __shared__ int shift_sh;
  if (skip != nullptr && *skip != 0) return;
  const int row = blockIdx.x;
  if (row >= n) return;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int npairs = cols >> 1;  // cols = n, or n + 1 over a zero column
  const uint4* yr = reinterpret_cast<const uint4*>(X2 + row * ld);
  const uint4* xr = reinterpret_cast<const uint4*>(X + row * ld);
  uint4 v[kFusedPPT], x[kFusedPPT];
#pragma unroll
  for (int i = 0; i < kFusedPPT; ++i) {
    const int p = i * THREADS + threadIdx.x;
    v[i] = make_uint4(0u, 0u, 0u, 0u);
    x[i] = make_uint4(0u, 0u, 0u, 0u);
    if (p < npairs) {
      v[i] = yr[p];
      x[i] = xr[p];
    }
  }
  float ss = 0.0f;
  DF a3{0.0f, 0.0f}, a4{0.0f, 0.0f}, a5{0.0f, 0.0f};
#pragma unroll
  for (int i = 0; i < kFusedPPT; ++i) {
    const int p = i * THREADS + threadIdx.x;
    if (p < npairs) {
      if (2 * p == row || 2 * p + 1 == row) {  // the diagonal elements, bit for bit
        const bool lo = (2 * p == row);
        diag_sh[0] = lo ? ((static_cast<unsigned long long>(x[i].y) << 32) | x[i].x)
                        : ((static_cast<unsigned long long>(x[i].w) << 32) | x[i].z);
        diag_sh[1] = lo ? ((static_cast<unsigned long long>(v[i].y) << 32) | v[i].x)
                        : ((static_cast<unsigned long long>(v[i].w) << 32) | v[i].z);
      }
      float h0, l0, h1, l1, g0, k0, g1, k1;
      split_words(v[i].y, v[i].x, h0, l0);
      split_words(v[i].w, v[i].z, h1, l1);
      split_words(x[i].y, x[i].x, g0, k0);
      split_words(x[i].w, x[i].z, g1, k1);
      v[i] = make_uint4(__float_as_uint(h0), __float_as_uint(l0), __float_as_uint(h1),
                        __float_as_uint(l1));  // the slices are cut from the FP32 splits
      ss = fmaf(h0, h0, fmaf(h1, h1, ss));
      a3 = df_fma(df_fma(a3, h0, l0, g0, k0), h1, l1, g1, k1);
      a4 = df_fma(df_fma(a4, h0, l0, h0, l0), h1, l1, h1, l1);
      if (own_x_dot) a5 = df_fma(df_fma(a5, g0, k0, g0, k0), g1, k1, g1, k1);
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) ss += __shfl_xor_sync(0xffffffffu, ss, o);
  a3 = df_warp_sum(a3);
  a4 = df_warp_sum(a4);
  if (own_x_dot) a5 = df_warp_sum(a5);
  if (lane == 0) {
    red_ss[w] = ss;
    red_dot[0][w] = a3;
    red_dot[1][w] = a4;
    red_dot[2][w] = a5;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    float t = 0.0f;
    DF d3{0.0f, 0.0f}, d4{0.0f, 0.0f}, d5{0.0f, 0.0f};
    for (int j = 0; j < THREADS / 32; ++j) {
      t += red_ss[j];
      d3 = df_add(d3, red_dot[0][j]);
      d4 = df_add(d4, red_dot[1][j]);
      d5 = df_add(d5, red_dot[2][j]);
    }
    double* pr = partials + static_cast<int64_t>(row) * kTraceTerms;
    pr[0] = __longlong_as_double(static_cast<long long>(diag_sh[0]));
    pr[1] = __longlong_as_double(static_cast<long long>(diag_sh[1]));
    pr[2] = df_to_double(d3);
    pr[3] = df_to_double(d4);
    pr[4] = own_x_dot ? df_to_double(d5) : x_row_dot[row];
    int e = 0;
    unsigned long long scb;
    if (t > 0.0f && isfinite(t)) {
      frexpf(sqrtf(t * 1.002f) * 1.0001f, &e);  // 2^e > ||y|| (see form_slice_row)
      scb = static_cast<unsigned long long>(e + 1023) << 52;
    } else {
      scb = isfinite(t) ? (1023ull << 52) : 0x7FF8000000000000ull;
    }
    out_scale[row] = __longlong_as_double(static_cast<long long>(scb));
    shift_sh = (scb >> 52 == 0x7FF) ? -100000 : 11 - e + bits * (nslice - 1);
  }
  __syncthreads();
  const int p2 = shift_sh;
  uint32_t* orow = reinterpret_cast<uint32_t*>(out + row * out_ld);
  const int64_t plane2 = plane >> 1;
  write_row_slices_any<THREADS>(v, npairs, p2, orow, plane2, nslice, bits);
}

// Row dot products of W = a X + b X^2 + c I with X^2 from the per-row trace terms of
// slice_traces_kernel: <W_i, X2_i> = a <X_i, X2_i> + b ||X2_i||^2 + c (X2)_ii.
__global__ void w_row_dots_kernel(const double* __restrict__ partials, int n,
                                  const double* __restrict__ coef, double* row_dot) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double* p = partials + static_cast<int64_t>(i) * kTraceTerms;
  row_dot[i] = coef[0] * p[2] + coef[1] * p[3] + coef[2] * p[1];
}

// sum_j (A - I)_ij^2 (minus_identity), sum_j A_ij^2 or sum_j A_ij B_ij for one row per block,
// all of the row's loads in flight at once (like the forming/slicing kernels), double-float sums
// (no FP64 instruction) into partials[row].
template <int THREADS, bool HAS_B>
__global__ void __launch_bounds__(THREADS)
    dot_rows_kernel(const double* A, int64_t lda, const double* B, int64_t ldb, int cols,
                    int minus_identity, double* partials, const int* skip) {
  __shared__ DF red[THREADS / 32];
  if (skip != nullptr && *skip != 0) return;
  const int row = blockIdx.x;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int npairs = cols >> 1;
  const uint4* ar = reinterpret_cast<const uint4*>(A + row * lda);
  const uint4* br = HAS_B ? reinterpret_cast<const uint4*>(B + row * ldb) : nullptr;
  uint4 va[kFusedPPT], vb[HAS_B ? kFusedPPT : 1];
#pragma unroll
  for (int i = 0; i < kFusedPPT; ++i) {
    const int p = i * THREADS + threadIdx.x;
    va[i] = make_uint4(0u, 0u, 0u, 0u);
    if (p < npairs) va[i] = ar[p];
    if (HAS_B) {
      vb[i] = make_uint4(0u, 0u, 0u, 0u);
      if (p < npairs) vb[i] = br[p];
    }
  }
  DF acc{0.0f, 0.0f};
#pragma unroll
  for (int i = 0; i < kFusedPPT; ++i) {
    const int p = i * THREADS + threadIdx.x;
    if (p < npairs) {
      uint4 x = va[i];
      if (minus_identity && (2 * p == row || 2 * p + 1 == row)) {
        if (2 * p == row) {
          const uint2 d = add_on_diagonal_words(make_uint2(x.x, x.y), -1.0);
          x.x = d.x;
          x.y = d.y;
        } else {
          const uint2 d = add_on_diagonal_words(make_uint2(x.z, x.w), -1.0);
          x.z = d.x;
          x.w = d.y;
        }
      }
      float h0, l0, h1, l1;
      split_words(x.y, x.x, h0, l0);
      split_words(x.w, x.z, h1, l1);
      if (HAS_B) {
        float g0, k0, g1, k1;
        split_words(vb[i].y, vb[i].x, g0, k0);
        split_words(vb[i].w, vb[i].z, g1, k1);
        acc = df_fma(df_fma(acc, h0, l0, g0, k0), h1, l1, g1, k1);
      } else {
        acc = df_fma(df_fma(acc, h0, l0, h0, l0), h1, l1, h1, l1);
      }
    }
  }
  acc = df_warp_sum(acc);
  if (lane == 0) red[w] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    DF t{0.0f, 0.0f};
    for (int j = 0; j < THREADS / 32; ++j) t = df_add(t, red[j]);
    partials[row] = df_to_double(t);
  }
}

// ------------------------------------------------------------------------------------------
// Gershgorin: lo_i = a_ii - sum_{j != i} |a_ij|, hi_i = a_ii + sum_{j != i} |a_ij|
// ------------------------------------------------------------------------------------------
__global__ void __launch_bounds__(kRowsPerBlock * 32)
    gershgorin_kernel(const double* __restrict__ A, int64_t lda, int n, double* partials) {
  __shared__ double slo[kRowsPerBlock], shi[kRowsPerBlock];
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int row = blockIdx.x * kRowsPerBlock + w;
  double lo = INFINITY, hi = -INFINITY;
  if (row < n) {
    const double* ar = A + row * lda;
    double r = 0.0;
    for (int j = lane; j < n; j += 32)
      if (j != row) r += fabs(ar[j]);
    r = warp_sum(r);
    const double d = ar[row];
    lo = d - r;
    hi = d + r;
  }
  if (lane == 0) {
    slo[w] = lo;
    shi[w] = hi;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double l = slo[0], h = shi[0];
    for (int i = 1; i < kRowsPerBlock; ++i) {
      l = fmin(l, slo[i]);
      h = fmax(h, shi[i]);
    }
    partials[2 * blockIdx.x] = l;
    partials[2 * blockIdx.x + 1] = h;
  }
}

__global__ void minmax_reduce_kernel(const double* partials, int nblocks, double* out) {
  __shared__ double sl[32], sh[32];
  double l = INFINITY, h = -INFINITY;
  for (int i = threadIdx.x; i < nblocks; i += blockDim.x) {
    l = fmin(l, partials[2 * i]);
    h = fmax(h, partials[2 * i + 1]);
  }
  l = warp_min(l);
  h = warp_max(h);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0) {
    sl[w] = l;
    sh[w] = h;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    const int nw = (blockDim.x + 31) >> 5;
    for (int i = 1; i < nw; ++i) {
      l = fmin(l, sl[i]);
      h = fmax(h, sh[i]);
    }
    l = fmin(l, sl[0]);
    h = fmax(h, sh[0]);
    out[0] = l;
    out[1] = h;
  }
}

// ------------------------------------------------------------------------------------------
// TRS4 traces, one warp per row (rows that slice_traces_kernel does not take: odd or wider than
// kFusedMaxCols, or filtered purification)
// ------------------------------------------------------------------------------------------
__global__ void __launch_bounds__(kRowsPerBlock * 32)
    trs4_traces_kernel(const double* __restrict__ X, const double* __restrict__ X2, int64_t ld,
                       int n, double* partials, const int* skip) {
  // <X2, X>, ||X2||^2 and ||X||^2 in FP32 double-float (no FP64 ALU), diagonals exact
  __shared__ double s[kRowsPerBlock][kTraceTerms];
  if (skip != nullptr && *skip != 0) return;
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int row = blockIdx.x * kRowsPerBlock + w;
  double t[kTraceTerms] = {0, 0, 0, 0, 0};
  if (row < n) {
    const double* xr = X + row * ld;
    const double* yr = X2 + row * ld;
    DF a3{0.f, 0.f}, a4{0.f, 0.f}, a5{0.f, 0.f};
    // 4 x 16-byte loads per array in flight per lane when rows are 16-byte aligned
    const bool vec = ((ld & 1) == 0) && ((reinterpret_cast<uintptr_t>(X) |
                                          reinterpret_cast<uintptr_t>(X2)) & 15) == 0;
    const double2* x2p = reinterpret_cast<const double2*>(xr);
    const double2* y2p = reinterpret_cast<const double2*>(yr);
    const int np = vec ? (n >> 1) : 0;
    int p = lane;
    for (; p + 96 < np; p += 128) {
      double2 xv[4], yv[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        xv[u] = x2p[p + 32 * u];
        yv[u] = y2p[p + 32 * u];
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        float xh, xl, yh, yl;
        split_double(xv[u].x, xh, xl);
        split_double(yv[u].x, yh, yl);
        a3 = df_fma(a3, yh, yl, xh, xl);
        a4 = df_fma(a4, yh, yl, yh, yl);
        a5 = df_fma(a5, xh, xl, xh, xl);
        split_double(xv[u].y, xh, xl);
        split_double(yv[u].y, yh, yl);
        a3 = df_fma(a3, yh, yl, xh, xl);
        a4 = df_fma(a4, yh, yl, yh, yl);
        a5 = df_fma(a5, xh, xl, xh, xl);
      }
    }
    const int j0 = vec ? 2 * p : lane, jstep = vec ? 64 : 32, jw = vec ? 2 : 1;
    for (int j = j0; j < n; j += jstep) {  // tail (and unaligned rows) element-wise
      for (int jj = j; jj < j + jw && jj < n; ++jj) {
        float xh, xl, yh, yl;
        split_double(xr[jj], xh, xl);
        split_double(yr[jj], yh, yl);
        a3 = df_fma(a3, yh, yl, xh, xl);
        a4 = df_fma(a4, yh, yl, yh, yl);
        a5 = df_fma(a5, xh, xl, xh, xl);
      }
    }
    a3 = df_warp_sum(a3);
    a4 = df_warp_sum(a4);
    a5 = df_warp_sum(a5);
    if (lane == 0) {
      t[0] = xr[row];
      t[1] = yr[row];
      t[2] = df_to_double(a3);
      t[3] = df_to_double(a4);
      t[4] = df_to_double(a5);
    }
  }
  if (lane == 0)
    for (int k = 0; k < kTraceTerms; ++k) s[w][k] = t[k];
  __syncthreads();
  if (threadIdx.x < kTraceTerms) {
    double acc = 0.0;
    for (int i = 0; i < kRowsPerBlock; ++i) acc += s[i][threadIdx.x];
    partials[blockIdx.x * kTraceTerms + threadIdx.x] = acc;
  }
}

__global__ void __launch_bounds__(kRowsPerBlock * 32)
    dot_kernel(const double* __restrict__ A, int64_t lda, const double* __restrict__ B,
               int64_t ldb, int rows, int cols, int minus_identity, double* partials,
               const int* skip) {
  // FP32 double-float accumulation (no FP64 ALU)
  __shared__ double s[kRowsPerBlock];
  if (skip != nullptr && *skip != 0) return;
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int row = blockIdx.x * kRowsPerBlock + w;
  double r = 0.0;
  if (row < rows) {
    const double* ar = A + row * lda;
    const double* br = (B != nullptr) ? B + row * ldb : nullptr;
    DF acc{0.f, 0.f};
    const bool vec = ((lda & 1) == 0) && (br == nullptr || (ldb & 1) == 0) &&
                     ((reinterpret_cast<uintptr_t>(A) |
                       (br != nullptr ? reinterpret_cast<uintptr_t>(B) : 0)) & 15) == 0;
    int jstart = lane, jstep = 32;
    if (vec) {
      const double2* a2 = reinterpret_cast<const double2*>(ar);
      const double2* b2 = (br != nullptr) ? reinterpret_cast<const double2*>(br) : nullptr;
      const int np = cols >> 1;
      int p = lane;
      for (; p + 96 < np; p += 128) {
        double2 av[4], bv[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          av[u] = a2[p + 32 * u];
          bv[u] = (b2 != nullptr) ? b2[p + 32 * u] : av[u];
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int j = 2 * (p + 32 * u);
          double x0 = av[u].x, x1 = av[u].y;
          if (minus_identity && (j == row || j + 1 == row)) {
            if (j == row) x0 = minus_one(x0);
            else x1 = minus_one(x1);
          }
          double y0 = (b2 != nullptr) ? bv[u].x : x0, y1 = (b2 != nullptr) ? bv[u].y : x1;
          float ah, al, bh, bl;
          split_double(x0, ah, al);
          split_double(y0, bh, bl);
          acc = df_fma(acc, ah, al, bh, bl);
          split_double(x1, ah, al);
          split_double(y1, bh, bl);
          acc = df_fma(acc, ah, al, bh, bl);
        }
      }
      jstart = 2 * p;
      jstep = 64;
    }
    for (int j0 = jstart; j0 < cols; j0 += jstep) {
      for (int j = j0; j < j0 + (vec ? 2 : 1) && j < cols; ++j) {
        float ah, al;
        double av = ar[j];
        if (minus_identity && j == row) av = minus_one(av);
        split_double(av, ah, al);
        if (br != nullptr) {
          float bh, bl;
          split_double(br[j], bh, bl);
          acc = df_fma(acc, ah, al, bh, bl);
        } else {
          acc = df_fma(acc, ah, al, ah, al);
        }
      }
    }
    acc = df_warp_sum(acc);
    r = df_to_double(acc);
  }
  if (lane == 0) s[w] = r;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int i = 0; i < kRowsPerBlock; ++i) t += s[i];
    partials[blockIdx.x] = t;
  }
}

// Deterministic reduction of `nblocks` partial rows of `nterms` doubles (one block).
__device__ void reduce_terms(const double* partials, int nblocks, int nterms, double* out,
                             double* red) {
  for (int k = 0; k < nterms; ++k) {
    double acc = 0.0;
    for (int i = threadIdx.x; i < nblocks; i += blockDim.x) acc += partials[i * nterms + k];
    acc = block_sum(acc, red);
    if (threadIdx.x == 0) out[k] = acc;
  }
}

__global__ void __launch_bounds__(1024) reduce_kernel(const double* partials, int nblocks, int nterms,
                                                    double* out) {
  __shared__ double red[32];
  reduce_terms(partials, nblocks, nterms, out, red);
}

// TRS4 control: F(X) = X^2 (4X - 3X^2), G(X) = X^2 (I - X)^2, Tr F = 4 t3 - 3 t4,
// Tr G = t2 - 2 t3 + t4, gamma = (N - Tr F) / Tr G; branches gamma > 6 -> 2X - X^2,
// gamma < 0 -> X^2, else F + gamma G = X^2 W with W = gamma I + (4 - 2 gamma) X + (gamma - 3) X^2
// (the gamma X^2 term folded into the right factor, so the product needs no addend).
__global__ void trs4_control_kernel(const double* partials, int nblocks, Trs4State* st,
                                    double tol_idem) {
  __shared__ double red[32];
  __shared__ double t[kTraceTerms];
  // A finished problem of a lockstep batch keeps its state and takes no further step.
  if (st->done) {
    if (threadIdx.x == 0) {
      st->skip_gemm = 1;
      st->skip_form_x = 1;
    }
    return;
  }
  reduce_terms(partials, nblocks, kTraceTerms, t, red);
  __syncthreads();
  if (threadIdx.x != 0) return;
  const double N = st->n_occ;
  for (int k = 0; k < kTraceTerms; ++k) st->t[k] = t[k];
  const double trF = 4.0 * t[2] - 3.0 * t[3];
  const double trG = t[1] - 2.0 * t[2] + t[3];
  const double idem = t[0] - t[4];
  st->trG = trG;
  st->idem_prev = (st->iter == 0) ? INFINITY : st->idem;
  st->idem = idem;
  int stop = 0;
  bool finite = true;
  for (int k = 0; k < kTraceTerms; ++k) finite = finite && isfinite(t[k]);
  const double Nf = fmax(N, 1.0);
  if (!finite) {
    stop = 3;
  } else if (fabs(idem) <= tol_idem) {
    stop = 1;
  } else if (fabs(idem) < 1e-4 * Nf && fabs(idem) > 0.5 * fabs(st->idem_prev)) {
    stop = 2;  // the idempotency error no longer falls: the arithmetic's floor is reached
  } else if (st->floor_rule && st->iter > 0 && fabs(st->idem_prev) < 0.01 &&
             (st->branch == 3 || (st->branch == 2 && st->method == kPurifyTrs4)) &&
             fabs(idem) > 20.0 * st->idem_prev * st->idem_prev) {
    // The step that made this iterate was quadratic: with every eigenvalue within
    // e = Tr(X - X^2) < 0.01 of 0 or 1, McWeeny maps a distance d to at most 3 d^2 and the
    // TRS4 map (0 <= gamma <= 6) to at most 6 d^2 + O(d^3), so in exact arithmetic the new
    // error is below 6 e_prev^2.  An error more than 20 e_prev^2 was set by the products'
    // rounding: this iterate is at the floor, and a further step would only confirm it.
    stop = 2;
  }
  if (stop == 0 && st->max_iter > 0 && st->iter >= st->max_iter) stop = 4;
  // Estimated spectral bounds that missed part of the spectrum leave Tr X outside [0, n].
  if (st->check_trace && (!(t[0] > -0.5) || !(t[0] < st->n + 0.5))) {
    stop = 3;
    st->failed = 1;
  }
  st->stop = stop;
  if (stop != 0) {
    // the iterate of this iteration is final, or the previous one if it was better (at the
    // floor a further step only adds rounding); its buffer is the iteration's parity, or the
    // other one
    st->done = 1;
    const int revert = (stop == 2 && st->iter > 0 && fabs(idem) > fabs(st->idem_prev)) ? 1 : 0;
    st->final_buf = (st->iter & 1) ^ revert;
    st->final_idem = revert ? st->idem_prev : idem;
  }
  // Endgame.  Once Tr(X - X^2) < 0.1 every eigenvalue x has x(1-x) < 0.1, i.e. it lies within
  // 0.113 of 0 or 1, and with |Tr X - N| < 0.25 exactly N of them are near 1.  From there the
  // McWeeny map 3X^2 - 2X^3 = X^2 (3I - 2X) takes each to the nearer end (quadratically) and
  // needs no gamma: gamma = (N - Tr F)/Tr G is a ratio of two differences that both vanish at
  // convergence, so its digits go first and a wrong branch would move the trace by Tr(X - X^2).
  const bool endgame = fabs(idem) < 0.1 && fabs(t[0] - N) < 0.25;
  int br;
  if (st->method == kPurifyTrs2 && !endgame) {
    // 2nd-order trace resetting: of X^2 and 2X - X^2, the one whose trace is nearer N
    st->gamma = 0.0;
    if (fabs(t[1] - N) <= fabs(2.0 * t[0] - t[1] - N)) {
      br = 1;
      st->coefX[0] = 0.0;
      st->coefX[1] = 1.0;
    } else {
      br = 0;
      st->coefX[0] = 2.0;
      st->coefX[1] = -1.0;
    }
    st->coefX[2] = 0.0;
    st->branch = br;
    st->skip_gemm = 1;
    st->skip_form_x = (stop != 0) ? 1 : 0;
    st->iter += 1;
    return;
  }
  if (st->method == kPurifyCanonical && !endgame && idem > 1e-12 * Nf) {
    // canonical purification, X <- X W with c = Tr(X^2 - X^3) / Tr(X - X^2) (Tr X is kept):
    // c >= 1/2: W = ((1 + c) X - X^2) / c;  c < 1/2: W = ((1 - 2c) I + (1 + c) X - X^2) / (1 - c)
    const double cc = (t[1] - t[2]) / idem;
    st->gamma = cc;
    if (cc >= 0.5) {
      st->coefW[0] = (1.0 + cc) / cc;
      st->coefW[1] = -1.0 / cc;
      st->coefW[2] = 0.0;
    } else {
      st->coefW[0] = (1.0 + cc) / (1.0 - cc);
      st->coefW[1] = -1.0 / (1.0 - cc);
      st->coefW[2] = (1.0 - 2.0 * cc) / (1.0 - cc);
    }
    st->gemm_coef[0] = 1.0;
    st->gemm_coef[1] = 0.0;
    st->branch = 4;
    st->skip_gemm = (stop != 0) ? 1 : 0;
    st->skip_form_x = 1;
    st->iter += 1;
    return;
  }
  const bool gamma_ok = st->method == kPurifyTrs4 && !endgame && trG > 1e-12 * Nf;
  const double g = gamma_ok ? (N - trF) / trG : 0.0;
  st->gamma = g;
  if (!gamma_ok) {
    br = 3;
    st->coefW[0] = -2.0;
    st->coefW[1] = 0.0;
    st->coefW[2] = 3.0;
    st->gemm_coef[0] = 1.0;
    st->gemm_coef[1] = 0.0;
  } else if (g > 6.0) {
    br = 0;
    st->coefX[0] = 2.0;
    st->coefX[1] = -1.0;
    st->coefX[2] = 0.0;
  } else if (g < 0.0) {
    br = 1;
    st->coefX[0] = 0.0;
    st->coefX[1] = 1.0;
    st->coefX[2] = 0.0;
  } else {
    br = 2;
    st->coefW[0] = 4.0 - 2.0 * g;
    st->coefW[1] = g - 3.0;
    st->coefW[2] = g;
    st->gemm_coef[0] = 1.0;
    st->gemm_coef[1] = 0.0;
  }
  st->branch = br;
  const bool with_product = (br == 2 || br == 3);
  st->skip_gemm = (stop != 0 || !with_product) ? 1 : 0;
  st->skip_form_x = (stop != 0 || with_product) ? 1 : 0;
  st->iter += 1;
}

// Canonical initial guess X0 = (lam/n)(mu I - H~) + (N/n) I: coef = {-lam/n, 0, lam mu/n + N/n}
// with mu = Tr H~ / n (diagonal summed in a fixed order) and
// lam = min(N / (eps_max - mu), (n - N) / (mu - eps_min)).
__global__ void canonical_x0_coef_kernel(const double* bounds, const double* Ht, int64_t ld, int n,
                                         double n_occ, double* coef) {
  __shared__ double red[32];
  double acc = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) acc += Ht[static_cast<int64_t>(i) * (ld + 1)];
  acc = block_sum(acc, red);
  if (threadIdx.x != 0) return;
  const double lo = bounds[0], hi = bounds[1];
  const double nn = static_cast<double>(n);
  const double mu = acc / nn;
  const double lam = fmin(n_occ / (hi - mu), (nn - n_occ) / (mu - lo));
  coef[0] = -lam / nn;
  coef[1] = 0.0;
  coef[2] = lam * mu / nn + n_occ / nn;
}

__global__ void x0_coef_kernel(const double* bounds, double* coef) {
  const double lo = bounds[0], hi = bounds[1];
  const double w = hi - lo;
  coef[0] = -1.0 / w;
  coef[1] = 0.0;
  coef[2] = hi / w;
}

// ---- Lanczos estimates of the extreme eigenvalues of a symmetric matrix ---------------------
// Three-term recurrence without reorthogonalisation (its extreme Ritz values converge first and
// are not disturbed by the loss of orthogonality, which only adds copies of converged values):
//   w = A v_k - beta_{k-1} v_{k-1},  alpha_k = v_k . w,  w -= alpha_k v_k,  beta_k = ||w||,
//   v_{k+1} = w / beta_k.
// The estimates only place the Newton-Schulz scale and the bounds of the initial guess, both
// with margins of several percent, so the recurrence runs in FP32: matrix elements truncated to
// FP32 from their bit patterns (relative error below 2^-23, no FP64 instruction), FP32 vectors
// and sums in a fixed order.  The Ritz values then carry errors of order 1e-6 ||A||, far inside
// the margins.

// v_j = +1 or -1 from an integer hash of (j, seed): a Rademacher probe, E[v v^T] = I.  The
// mixing steps are those of the published 'lowbias32' integer hash (C. Wellons).
__global__ void rademacher_kernel(double* v, int n, unsigned seed) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  unsigned h = static_cast<unsigned>(j) * 2654435761u + seed * 0x9E3779B9u;
  h ^= h >> 16;
  h *= 0x7FEB352Du;
  h ^= h >> 15;
  h *= 0x846CA68Bu;
  h ^= h >> 16;
  v[j] = (h & 0x80000000u) ? 1.0 : -1.0;
}

// Start vector: a fixed pseudo-random vector (integer hash) in [-0.5, 0.5), normalised; the
// previous vector 0.  One block.
__global__ void lanczos_init_kernel(int n, float* x, float* xprev, unsigned* counter) {
  __shared__ float red[32];
  __shared__ float inv_sh;
  if (threadIdx.x == 0 && counter != nullptr) *counter = 0u;
  float acc = 0.0f;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    unsigned h = static_cast<unsigned>(i) * 2654435761u + 0x9E3779B9u;
    h ^= h >> 16;
    h *= 0x85EBCA6Bu;
    h ^= h >> 13;
    const float v = __uint_as_float(0x3F800000u | (h >> 9)) - 1.5f;  // in [-0.5, 0.5)
    x[i] = v;
    acc = fmaf(v, v, acc);
  }
  acc = block_sum_f(acc, red);
  if (threadIdx.x == 0) inv_sh = acc > 0.0f ? rsqrtf(acc) : 0.0f;
  __syncthreads();
  const float inv = inv_sh;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    x[i] *= inv;
    xprev[i] = 0.0f;
  }
}

// y = A x for any n and leading dimension: one warp per row.
__global__ void __launch_bounds__(kRowsPerBlock * 32)
    matvec_f32_kernel(const double* __restrict__ A, int64_t lda, int n,
                      const float* __restrict__ x, float* y) {
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int row = blockIdx.x * kRowsPerBlock + w;
  if (row >= n) return;
  const uint2* ar = reinterpret_cast<const uint2*>(A + row * lda);
  float acc = 0.0f;
  for (int j = lane; j < n; j += 32) {
    const uint2 a = ar[j];
    acc = fmaf(trunc_words(a.y, a.x), x[j], acc);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if (lane == 0) y[row] = acc;
}

// One step after y = A v: alpha_k and beta_k into ab[k] and ab[kmax + k], then the next v.
// A beta at the FP32 rounding level of the step (an invariant subspace) ends the recurrence: the
// next vector is left zero, so every later alpha and beta is zero and the Ritz values stay
// those found.  One block.
__global__ void lanczos_update_kernel(float* y, float* x, float* xprev, int n, double* ab, int k,
                                      int kmax) {
  __shared__ float red[32];
  __shared__ float alpha_sh, inv_sh;
  const float beta_prev = (k > 0) ? static_cast<float>(ab[kmax + k - 1]) : 0.0f;
  float acc = 0.0f;
  for (int i = threadIdx.x; i < n; i += blockDim.x) acc = fmaf(x[i], y[i], acc);
  acc = block_sum_f(acc, red);
  if (threadIdx.x == 0) alpha_sh = acc;
  __syncthreads();
  const float alpha = alpha_sh;
  float ss = 0.0f;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const float wv = y[i] - alpha * x[i] - beta_prev * xprev[i];
    y[i] = wv;
    ss = fmaf(wv, wv, ss);
  }
  ss = block_sum_f(ss, red);
  if (threadIdx.x == 0) {
    const float beta = sqrtf(ss);
    ab[k] = static_cast<double>(alpha);
    // relative to the size of the step's terms (v has unit norm, or is zero once the recurrence
    // has ended): below it the new direction is FP32 rounding noise
    const bool ends = !(beta > 1e-5f * (fabsf(alpha) + beta_prev));
    ab[kmax + k] = ends ? 0.0 : static_cast<double>(beta);
    inv_sh = ends ? 0.0f : 1.0f / beta;
  }
  __syncthreads();
  const float inv = inv_sh;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    xprev[i] = x[i];
    x[i] = y[i] * inv;
  }
}

// One whole Lanczos step in one launch: y = A x with one block per row (rows of even length up
// to kFusedMaxCols), then the last block to finish (a counter in global memory; no block waits
// for another) does the step's vector update as lanczos_update_kernel does, and resets the
// counter for the next launch.  MODE 0 reads the FP64 matrix; MODE 1 reads it and also writes
// its FP32 truncation to a32 (row stride lda32 floats); MODE 2 reads that FP32 copy, half the
// bytes, which stays in L2 between steps for n up to ~5600.
constexpr int kLanczosRead64 = 0, kLanczosCopy32 = 1, kLanczosRead32 = 2;

template <int THREADS, int MODE>
__global__ void __launch_bounds__(THREADS)
    lanczos_step_kernel(const double* A, int64_t lda, float* a32, int64_t lda32, int n,
                        float* y, float* x, float* xprev, unsigned* counter, double* ab, int k,
                        int kmax) {
  __shared__ float red[32];
  __shared__ float alpha_sh, inv_sh;
  __shared__ int last_sh;
  const int row = blockIdx.x;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int npairs = n >> 1;
  const float2* x2 = reinterpret_cast<const float2*>(x);
  float acc = 0.0f;
  if (MODE == kLanczosRead32) {
    const float2* ar = reinterpret_cast<const float2*>(a32 + row * lda32);
    float2 va[kFusedPPT];
#pragma unroll
    for (int i = 0; i < kFusedPPT; ++i) {
      const int p = i * THREADS + threadIdx.x;
      va[i] = make_float2(0.0f, 0.0f);
      if (p < npairs) va[i] = ar[p];
    }
#pragma unroll
    for (int i = 0; i < kFusedPPT; ++i) {
      const int p = i * THREADS + threadIdx.x;
      if (p < npairs) {
        const float2 xv = x2[p];
        acc = fmaf(va[i].x, xv.x, acc);
        acc = fmaf(va[i].y, xv.y, acc);
      }
    }
  } else {
    const uint4* ar = reinterpret_cast<const uint4*>(A + row * lda);
    float2* cr = (MODE == kLanczosCopy32) ? reinterpret_cast<float2*>(a32 + row * lda32) : nullptr;
    uint4 va[kFusedPPT];
#pragma unroll
    for (int i = 0; i < kFusedPPT; ++i) {
      const int p = i * THREADS + threadIdx.x;
      va[i] = make_uint4(0u, 0u, 0u, 0u);
      if (p < npairs) va[i] = ar[p];
    }
#pragma unroll
    for (int i = 0; i < kFusedPPT; ++i) {
      const int p = i * THREADS + threadIdx.x;
      if (p < npairs) {
        const float a0 = trunc_words(va[i].y, va[i].x), a1 = trunc_words(va[i].w, va[i].z);
        if (MODE == kLanczosCopy32) cr[p] = make_float2(a0, a1);
        const float2 xv = x2[p];
        acc = fmaf(a0, xv.x, acc);
        acc = fmaf(a1, xv.y, acc);
      }
    }
  }
  // fixed summation order: per thread, warp butterfly, warps in turn
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if (lane == 0) red[w] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    float t = 0.0f;
    for (int j = 0; j < THREADS / 32; ++j) t += red[j];
    y[row] = t;
    __threadfence();
    const unsigned done = atomicAdd(counter, 1u);
    last_sh = (done + 1u == gridDim.x) ? 1 : 0;
  }
  __syncthreads();
  if (!last_sh) return;
  // the last block: every y[i] is written and visible (fence before each block's count)
  __threadfence();
  if (threadIdx.x == 0) *counter = 0u;
  const float beta_prev = (k > 0) ? static_cast<float>(ab[kmax + k - 1]) : 0.0f;
  float s = 0.0f;
  for (int i = threadIdx.x; i < n; i += THREADS) s = fmaf(x[i], __ldcg(y + i), s);
  s = block_sum_f(s, red);
  if (threadIdx.x == 0) alpha_sh = s;
  __syncthreads();
  const float alpha = alpha_sh;
  float ss = 0.0f;
  for (int i = threadIdx.x; i < n; i += THREADS) {
    const float wv = __ldcg(y + i) - alpha * x[i] - beta_prev * xprev[i];
    ss = fmaf(wv, wv, ss);
  }
  ss = block_sum_f(ss, red);
  if (threadIdx.x == 0) {
    const float beta = sqrtf(ss);
    ab[k] = static_cast<double>(alpha);
    const bool ends = !(beta > 1e-5f * (fabsf(alpha) + beta_prev));
    ab[kmax + k] = ends ? 0.0 : static_cast<double>(beta);
    inv_sh = ends ? 0.0f : 1.0f / beta;
  }
  __syncthreads();
  const float inv = inv_sh;
  for (int i = threadIdx.x; i < n; i += THREADS) {
    const float xi = x[i];
    const float wv = __ldcg(y + i) - alpha * xi - beta_prev * xprev[i];
    xprev[i] = xi;
    x[i] = wv * inv;
  }
}

// Number of eigenvalues below x of the tridiagonal (a, b2 = b^2) (negative pivots of T - x I).
__device__ int sturm_count_f(const float* a, const float* b2, int m, float x) {
  int cnt = 0;
  float q = 1.0f;
  for (int i = 0; i < m; ++i) {
    q = a[i] - x - ((i > 0) ? b2[i - 1] / q : 0.0f);
    if (q == 0.0f) q = -1e-30f;
    if (q < 0.0f) ++cnt;
  }
  return cnt;
}

// Spectral bounds of a matrix from its Lanczos tridiagonal (small + lanczos_at) and
// Gershgorin's interval (small + gersh_at): the extreme Ritz values by multisection on FP32
// Sturm counts, widened by 2% of their span and clamped to Gershgorin's interval, into
// small[bounds_at..+1]; small[bounds_at+2] = 1 when the estimate (not Gershgorin's interval) is
// used.  Two warps, one per end; each round evaluates 32 Sturm counts at once and shrinks the
// bracket 33-fold, down to the FP32 resolution of the counts (about 1e-6 of the tridiagonal's
// norm), which takes five or six rounds.
__global__ void lanczos_bounds_kernel(double* small, int steps, int gersh_at, int lanczos_at,
                                      int bounds_at) {
  __shared__ float af[kMaxLanczos], b2f[kMaxLanczos];
  __shared__ int m_sh, finite_sh;
  __shared__ float glo_sh, ghi_sh, t_sh[2];
  if (blockIdx.x != 0) return;
  const int lane = threadIdx.x & 31, end = threadIdx.x >> 5;
  const double g_lo = small[gersh_at], g_hi = small[gersh_at + 1];
  const double* a = small + lanczos_at;
  const double* b = a + steps;
  if (threadIdx.x == 0) {
    int m = steps;
    for (int k = 0; k < steps; ++k)
      if (!(b[k] > 0.0)) {
        m = k + 1;
        break;
      }
    bool finite = true;
    float glo = INFINITY, ghi = -INFINITY;
    for (int i = 0; i < m; ++i) {
      finite = finite && isfinite(a[i]) && isfinite(b[i]);
      af[i] = static_cast<float>(a[i]);
      b2f[i] = static_cast<float>(b[i] * b[i]);
      const float r = static_cast<float>((i > 0 ? fabs(b[i - 1]) : 0.0) +
                                         (i + 1 < m ? fabs(b[i]) : 0.0));
      glo = fminf(glo, af[i] - r);
      ghi = fmaxf(ghi, af[i] + r);
    }
    m_sh = m;
    finite_sh = finite ? 1 : 0;
    // the tridiagonal's own Gershgorin interval, opened by its FP32 resolution
    const float pad = 1e-6f * fmaxf(fabsf(glo), fabsf(ghi)) + 1e-30f;
    glo_sh = glo - pad;
    ghi_sh = ghi + pad;
  }
  __syncthreads();
  const int m = m_sh;
  if (finite_sh) {
    // end 0: the least x with at least one eigenvalue below it; end 1: with all m below it
    const int want = (end == 0) ? 1 : m;
    float l = glo_sh, u = ghi_sh;
    const float tol = 1e-6f * fmaxf(fabsf(glo_sh), fabsf(ghi_sh));
    for (int it = 0; it < 12 && u - l > tol; ++it) {
      const float x = l + (u - l) * static_cast<float>(lane + 1) * (1.0f / 33.0f);
      const bool above = sturm_count_f(af, b2f, m, x) >= want;
      const unsigned mask = __ballot_sync(0xffffffffu, above);
      // the first point at or above the target bounds it from above, the one before from below
      const int first = mask ? __ffs(mask) - 1 : 32;
      const float nu = (first < 32) ? l + (u - l) * static_cast<float>(first + 1) * (1.0f / 33.0f)
                                    : u;
      const float nl = (first > 0) ? l + (u - l) * static_cast<float>(first) * (1.0f / 33.0f) : l;
      l = nl;
      u = nu;
    }
    if (lane == 0) t_sh[end] = (end == 0) ? l : u;
  }
  __syncthreads();
  if (threadIdx.x != 0) return;
  double lo = g_lo, hi = g_hi;
  double t_raw[2] = {g_lo, g_hi};
  if (finite_sh) {
    const double t0 = t_sh[0], t1 = t_sh[1];
    t_raw[0] = t0;
    t_raw[1] = t1;
    const double margin = 0.02 * (t1 - t0) + 1e-6 * fmax(fabs(t0), fabs(t1));
    const double c_lo = fmax(g_lo, t0 - margin), c_hi = fmin(g_hi, t1 + margin);
    if (isfinite(c_lo) && isfinite(c_hi) && c_hi > c_lo) {
      lo = c_lo;
      hi = c_hi;
    }
  }
  small[bounds_at] = lo;
  small[bounds_at + 1] = hi;
  small[bounds_at + 2] = (lo == g_lo && hi == g_hi) ? 0.0 : 1.0;  // 1: the estimate was used
  small[bounds_at + 3] = finite_sh ? t_raw[0] : g_lo;              // the extreme Ritz values
  small[bounds_at + 4] = finite_sh ? t_raw[1] : g_hi;
}

__global__ void scale_coef_kernel(const double* bounds, int inv_sqrt, double* coef) {
  const double c = bounds[1];
  coef[0] = inv_sqrt ? 1.0 / sqrt(c) : 1.0 / c;
  coef[1] = 0.0;
  coef[2] = 0.0;
}

// A <- (A + A^T)/2 on 32 x 32 tile pairs (I <= J)
__global__ void symmetrise_kernel(double* A, int64_t lda, int n) {
  __shared__ double t1[32][33], t2[32][33];
  const int I = blockIdx.y, J = blockIdx.x;
  if (I > J) return;
  const int tx = threadIdx.x, ty = threadIdx.y;  // 32 x 8
  for (int r = ty; r < 32; r += 8) {
    const int i1 = I * 32 + r, j1 = J * 32 + tx;
    t1[r][tx] = (i1 < n && j1 < n) ? A[i1 * lda + j1] : 0.0;
    const int i2 = J * 32 + r, j2 = I * 32 + tx;
    t2[r][tx] = (i2 < n && j2 < n) ? A[i2 * lda + j2] : 0.0;
  }
  __syncthreads();
  for (int r = ty; r < 32; r += 8) {
    const int i1 = I * 32 + r, j1 = J * 32 + tx;
    const double v1 = 0.5 * (t1[r][tx] + t2[tx][r]);
    const int i2 = J * 32 + r, j2 = I * 32 + tx;
    const double v2 = 0.5 * (t2[r][tx] + t1[tx][r]);
    if (i1 < n && j1 < n) A[i1 * lda + j1] = v1;
    if (I != J && i2 < n && j2 < n) A[i2 * lda + j2] = v2;
  }
}

// C_ii = alpha <a_i, bt_i> + beta D_ii + diag in FP64, one warp per row.  The tensor core
// accumulates in FP32 with truncation; on the diagonal of products whose two factors have
// (nearly) parallel rows, such as X X or X^2 (3I - 2X), the slice-residual terms form a positive
// sum whose truncation error does not average out, so that diagonal is recomputed here.
__global__ void __launch_bounds__(kRowsPerBlock * 32)
    diag_fix_kernel(const double* __restrict__ A, int64_t lda, const double* __restrict__ Bt,
                    int64_t ldb, double* C, int64_t ldc, int n, int K, double alpha, double beta,
                    const double* D, int64_t ldd, double diag, const double* coef,
                    const int* skip) {
  if (skip != nullptr && *skip != 0) return;
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int row = blockIdx.x * kRowsPerBlock + w;
  if (row >= n) return;
  const double* ar = A + row * lda;
  const double* br = Bt + row * ldb;
  DF acc{0.f, 0.f};  // FP32 double-float: ~2^-48 relative, no FP64 ALU in the loop
  const bool vec = ((lda | ldb) & 1) == 0 && ((reinterpret_cast<uintptr_t>(A) |
                                               reinterpret_cast<uintptr_t>(Bt)) & 15) == 0;
  int kstart = lane;
  if (vec) {
    const double2* a2 = reinterpret_cast<const double2*>(ar);
    const double2* b2 = reinterpret_cast<const double2*>(br);
    const int np = K >> 1;
    int p = lane;
    for (; p + 96 < np; p += 128) {
      double2 av[4], bv[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        av[u] = a2[p + 32 * u];
        bv[u] = b2[p + 32 * u];
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        float ah, al, bh, bl;
        split_double(av[u].x, ah, al);
        split_double(bv[u].x, bh, bl);
        acc = df_fma(acc, ah, al, bh, bl);
        split_double(av[u].y, ah, al);
        split_double(bv[u].y, bh, bl);
        acc = df_fma(acc, ah, al, bh, bl);
      }
    }
    kstart = 2 * p;  // continue element-wise from here, stride 64 per lane pair block
    for (int k = kstart; k < K; k += 64) {
      for (int kk = k; kk < k + 2 && kk < K; ++kk) {
        float ah, al, bh, bl;
        split_double(ar[kk], ah, al);
        split_double(br[kk], bh, bl);
        acc = df_fma(acc, ah, al, bh, bl);
      }
    }
  } else {
    for (int k = lane; k < K; k += 32) {
      float ah, al, bh, bl;
      split_double(ar[k], ah, al);
      split_double(br[k], bh, bl);
      acc = df_fma(acc, ah, al, bh, bl);
    }
  }
  acc = df_warp_sum(acc);
  if (lane == 0) {
    double al2 = alpha, be = beta;
    if (coef != nullptr) {
      al2 = coef[0];
      be = coef[1];
    }
    double v = al2 * df_to_double(acc) + diag;
    if (D != nullptr) v += be * D[row * ldd + row];
    C[row * ldc + row] = v;
  }
}

// Trace reset, two launches: trace_factor_kernel (one block) writes sc = target / Tr X to
// out[1] and sc - 1 to out[0]; scale_rows_kernel multiplies X by out[1].
__global__ void trace_factor_kernel(const double* X, int64_t ld, int n, double target,
                                    double* out) {
  __shared__ double red[32];
  double t = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) t += X[i * ld + i];
  t = block_sum(t, red);
  if (threadIdx.x == 0) {
    const double sc = (t != 0.0 && isfinite(t)) ? target / t : 1.0;
    out[0] = sc - 1.0;
    out[1] = sc;
  }
}

__global__ void scale_rows_kernel(double* X, int64_t ld, int n, const double* factor) {
  const double sc = factor[1];
  const int row = blockIdx.x;
  for (int j = threadIdx.x; j < n; j += blockDim.x) X[row * ld + j] *= sc;
}

__global__ void identity_kernel(double* A, int64_t lda, int n) {
  const int row = blockIdx.x;
  for (int j = threadIdx.x; j < n; j += blockDim.x) A[row * lda + j] = (j == row) ? 1.0 : 0.0;
}

}  // namespace

cudaError_t form_and_slice(const double* X, int64_t ldx, const double* X2, int64_t ldx2,
                           int rows, int cols_logical, const double* coef_dev, double ha,
                           double hb, double hc, double* Y, int64_t ldy, SliceBuf* out,
                           int nslice, const int* skip, cudaStream_t stream, int bits, int dot,
                           const TruncArgs* trunc, bool zero_pad) {
  if (rows <= 0) return cudaSuccess;
  // an odd row length with a zero column after it in every buffer is processed as the even one
  // (the paired kernels), and the logical shape stays the caller's
  const int cols = (zero_pad && (cols_logical & 1) && ldx > cols_logical &&
                    (X2 == nullptr || ldx2 > cols_logical) &&
                    (Y == nullptr || ldy > cols_logical) &&
                    (out == nullptr || nslice <= 0 || out->ld > cols_logical))
                       ? cols_logical + 1 : cols_logical;
  if (bits < 9 || bits > 12) return cudaErrorInvalidValue;
  if (dot == kDotX2 && X2 == nullptr) return cudaErrorInvalidValue;
  TruncArgs tr;
  if (out != nullptr) out->mask_valid = false;
  if (trunc != nullptr && trunc->tau_bits != 0ull) {
    tr.tau_bits = trunc->tau_bits;
    // the filtered values must reach memory (the element pass and later steps read them)
    if (Y == nullptr) {
      Y = const_cast<double*>(X);
      ldy = ldx;
    }
    // tile occupancy goes to the output slice buffer when it has storage for it
    if (out != nullptr && nslice > 0 && out->tile_mask != nullptr &&
        out->mask_ld >= (cols + 127) / 128) {
      tr.mask = out->tile_mask;
      tr.mask_ld = out->mask_ld;
      const cudaError_t e = cudaMemsetAsync(
          tr.mask, 0, sizeof(uint32_t) * static_cast<size_t>((rows + 127) / 128) * tr.mask_ld,
          stream);
      if (e != cudaSuccess) return e;
      out->mask_valid = true;
    }
  }
  __half* od = nullptr;
  double* osc = nullptr;
  int64_t old = 0, plane = 0;
  if (out != nullptr && nslice > 0) {
    if (nslice > 4 || out->ld < cols || out->rows_alloc < rows) return cudaErrorInvalidValue;
    od = out->data;
    osc = out->row_scale;
    old = out->ld;
    plane = static_cast<int64_t>(out->ld) * out->rows_alloc;
    out->rows = rows;
    out->cols = cols_logical;
    out->nslice_valid = nslice;
    out->bits = bits;
    out->dot_partner = nullptr;
  } else {
    nslice = 0;
  }
  const double step = ldexp(1.0, bits);
  const bool aligned =
      (cols % 2 == 0) && (ldx % 2 == 0) && (reinterpret_cast<uintptr_t>(X) % 16 == 0) &&
      (X2 == nullptr || ((ldx2 % 2 == 0) && (reinterpret_cast<uintptr_t>(X2) % 16 == 0))) &&
      (Y == nullptr || ((ldy % 2 == 0) && (reinterpret_cast<uintptr_t>(Y) % 16 == 0))) &&
      (od == nullptr || ((old % 2 == 0) && (plane % 2 == 0) &&
                         (reinterpret_cast<uintptr_t>(od) % 4 == 0)));
  const bool host_plain = (coef_dev == nullptr) && ha == 1.0 && (X2 == nullptr || hb == 0.0) &&
                          hc == 0.0;
  if (tr.tau_bits != 0ull && !aligned) return cudaErrorInvalidValue;  // filtering: two passes
  const int npairs = cols / 2;
  if (aligned && od != nullptr && cols <= kFusedMaxCols) {
    // one pass: form, norm, slices (the row stays in registers)
    const bool with_dot = dot != kDotNone && out->row_dot != nullptr;
    const int d = with_dot ? dot : kDotNone;
    double* rd = with_dot ? out->row_dot : nullptr;
    count_launch();
#define GDM_FUSED(T)                                                                             \
  if (X2 != nullptr)                                                                             \
    form_slice_fused_kernel<T, true><<<rows, T, 0, stream>>>(                                    \
        X, ldx, X2, ldx2, rows, cols, coef_dev, ha, hb, hc, Y, ldy, od, osc, old, plane, nslice, \
        bits, skip, d, rd, tr);                                                                  \
  else                                                                                           \
    form_slice_fused_kernel<T, false><<<rows, T, 0, stream>>>(                                   \
        X, ldx, X2, ldx2, rows, cols, coef_dev, ha, hb, hc, Y, ldy, od, osc, old, plane, nslice, \
        bits, skip, d, rd, tr)
    if (npairs <= 128 * kFusedPPT) {
      GDM_FUSED(128);
    } else if (npairs <= 256 * kFusedPPT) {
      GDM_FUSED(256);
    } else {
      GDM_FUSED(512);
    }
#undef GDM_FUSED
    if (with_dot)
      out->dot_partner = (dot == kDotX2) ? X2 : (dot == kDotX ? X : (Y != nullptr ? Y : X));
  } else if (aligned && (host_plain || Y != nullptr || od == nullptr)) {
    // two passes: rows (form + norm) then elements (slices), both fully parallel
    const int nb = (rows + kRowsPerBlock - 1) / kRowsPerBlock;
    const bool with_dot = dot != kDotNone && od != nullptr && out->row_dot != nullptr;
    count_launch();
    form_norm_kernel<<<nb, kRowsPerBlock * 32, 0, stream>>>(
        X, ldx, X2, ldx2, rows, cols, coef_dev, ha, hb, hc, Y, ldy,
        od != nullptr ? osc : nullptr, skip, with_dot ? dot : kDotNone,
        with_dot ? out->row_dot : nullptr, tr);
    if (with_dot)
      out->dot_partner = (dot == kDotX2) ? X2 : (dot == kDotX ? X : (Y != nullptr ? Y : X));
    if (od != nullptr) {
      const double* src = (Y != nullptr) ? Y : X;
      const int64_t lds = (Y != nullptr) ? ldy : ldx;
      const int per_block = kSliceThreads * kSlicePairsPerThread;
      const dim3 grid(static_cast<unsigned>(rows),
                      static_cast<unsigned>((cols / 2 + per_block - 1) / per_block));
      count_launch();
      slice_pairs_kernel<<<grid, kSliceThreads, 0, stream>>>(src, lds, rows, cols, osc, od, old, plane,
                                                     nslice, bits, skip);
    }
  } else if (aligned && cols <= 2 * kRowThreads * 16) {
    count_launch();
    form_slice_vec_kernel<16><<<rows, kRowThreads, 0, stream>>>(
        X, ldx, X2, ldx2, rows, cols, coef_dev, ha, hb, hc, Y, ldy, od, osc, old, plane, nslice,
        skip, bits);
  } else {
    count_launch();
    form_slice_kernel<<<rows, kRowThreads, 0, stream>>>(X, ldx, X2, ldx2, rows, cols, coef_dev,
                                                        ha, hb, hc, Y, ldy, od, osc, old, plane,
                                                        nslice, skip, step);
  }
  return cudaGetLastError();
}

cudaError_t lanczos(const double* A, int64_t lda, int n, int steps, double* work,
                    double* partials, double* ab_dev, cudaStream_t stream, float* a32,
                    int64_t lda32) {
  (void)partials;
  if (n <= 0 || steps <= 0) return cudaSuccess;
  float* x = reinterpret_cast<float*>(work);
  float* xprev = x + n;
  float* y = xprev + n;
  unsigned* counter = reinterpret_cast<unsigned*>(y + n);
  const bool rows_fit = n % 2 == 0 && n <= kFusedMaxCols && lda % 2 == 0 &&
                        (reinterpret_cast<uintptr_t>(A) & 15) == 0;
  const bool copy32 = rows_fit && a32 != nullptr && lda32 >= n && lda32 % 2 == 0 &&
                      (reinterpret_cast<uintptr_t>(a32) & 7) == 0;
  const int nb = (n + kRowsPerBlock - 1) / kRowsPerBlock;
  count_launch();
  lanczos_init_kernel<<<1, 1024, 0, stream>>>(n, x, xprev, counter);
  const int threads = (n / 2 <= 128 * kFusedPPT) ? 128 : (n / 2 <= 256 * kFusedPPT) ? 256 : 512;
  for (int k = 0; k < steps; ++k) {
    count_launch();
    if (!rows_fit) {
      matvec_f32_kernel<<<nb, kRowsPerBlock * 32, 0, stream>>>(A, lda, n, x, y);
      count_launch();
      lanczos_update_kernel<<<1, 1024, 0, stream>>>(y, x, xprev, n, ab_dev, k, steps);
      continue;
    }
    // the first step reads the FP64 matrix and leaves its FP32 copy, the later ones read that
    const int mode = !copy32 ? kLanczosRead64 : (k == 0 ? kLanczosCopy32 : kLanczosRead32);
#define GDM_LZ(T, M)                                                                   \
  lanczos_step_kernel<T, M><<<n, T, 0, stream>>>(A, lda, a32, lda32, n, y, x, xprev, counter, \
                                                 ab_dev, k, steps)
#define GDM_LZT(T)                                     \
  do {                                                 \
    if (mode == kLanczosRead64) GDM_LZ(T, kLanczosRead64);      \
    else if (mode == kLanczosCopy32) GDM_LZ(T, kLanczosCopy32); \
    else GDM_LZ(T, kLanczosRead32);                    \
  } while (0)
    if (threads == 128) GDM_LZT(128);
    else if (threads == 256) GDM_LZT(256);
    else GDM_LZT(512);
#undef GDM_LZT
#undef GDM_LZ
  }
  return cudaGetLastError();
}

cudaError_t lanczos_bounds(double* small, int steps, int gersh_at, int lanczos_at, int bounds_at,
                           cudaStream_t stream) {
  if (steps > kMaxLanczos) return cudaErrorInvalidValue;
  count_launch();
  lanczos_bounds_kernel<<<1, 64, 0, stream>>>(small, steps, gersh_at, lanczos_at, bounds_at);
  return cudaGetLastError();
}

cudaError_t gershgorin(const double* A, int64_t lda, int n, double* partials, double* out_dev,
                       cudaStream_t stream) {
  const int nb = (n + kRowsPerBlock - 1) / kRowsPerBlock;
  count_launch();
  gershgorin_kernel<<<nb, kRowsPerBlock * 32, 0, stream>>>(A, lda, n, partials);
  count_launch();
  minmax_reduce_kernel<<<1, 256, 0, stream>>>(partials, nb, out_dev);
  return cudaGetLastError();
}

cudaError_t trs4_traces(const double* X, const double* X2, int64_t ld, int n, double* partials,
                        int* nblocks, cudaStream_t stream, const int* skip) {
  const int nb = (n + kRowsPerBlock - 1) / kRowsPerBlock;
  count_launch();
  trs4_traces_kernel<<<nb, kRowsPerBlock * 32, 0, stream>>>(X, X2, ld, n, partials, skip);
  *nblocks = nb;
  return cudaGetLastError();
}

cudaError_t slice_traces(const double* X2, const double* X, int64_t ld, int n, SliceBuf* out,
                         int nslice, int bits, double* partials, int* nrows, cudaStream_t stream,
                         const int* skip, bool zero_pad, const double* x_row_dot) {
  *nrows = 0;
  if (n <= 0) return cudaSuccess;
  if (!slice_traces_fits(X2, X, ld, n, out, nslice, zero_pad)) return cudaErrorInvalidValue;
  const int cols = (n & 1) ? n + 1 : n;
  out->mask_valid = false;
  out->rows = n;
  out->cols = n;
  out->nslice_valid = nslice;
  out->bits = bits;
  out->dot_partner = nullptr;
  const int64_t plane = static_cast<int64_t>(out->ld) * out->rows_alloc;
  const int npairs = cols / 2;
  count_launch();
  if (npairs <= 128 * kFusedPPT)
    slice_traces_kernel<128><<<n, 128, 0, stream>>>(X2, X, ld, n, cols, out->data,
                                                   out->row_scale, out->ld, plane, nslice, bits,
                                                   partials, skip, x_row_dot);
  else if (npairs <= 256 * kFusedPPT)
    slice_traces_kernel<256><<<n, 256, 0, stream>>>(X2, X, ld, n, cols, out->data,
                                                   out->row_scale, out->ld, plane, nslice, bits,
                                                   partials, skip, x_row_dot);
  else
    slice_traces_kernel<512><<<n, 512, 0, stream>>>(X2, X, ld, n, cols, out->data,
                                                   out->row_scale, out->ld, plane, nslice, bits,
                                                   partials, skip, x_row_dot);
  *nrows = n;
  return cudaGetLastError();
}

cudaError_t w_row_dots(const double* partials, int n, const double* coef_dev, SliceBuf* w,
                       const double* X2, cudaStream_t stream) {
  if (n <= 0) return cudaSuccess;
  count_launch();
  w_row_dots_kernel<<<(n + 255) / 256, 256, 0, stream>>>(partials, n, coef_dev, w->row_dot);
  w->dot_partner = X2;
  return cudaGetLastError();
}

bool slice_traces_fits(const double* X2, const double* X, int64_t ld, int n, const SliceBuf* out,
                       int nslice, bool zero_pad) {
  // an odd n needs the zero column after the rows (zero_pad) in X, X2 and the slices
  const int cols = (n & 1) ? n + 1 : n;
  return out != nullptr && nslice >= 1 && nslice <= 4 && ((n & 1) == 0 || zero_pad) &&
         ld % 2 == 0 && ld >= cols && cols <= kFusedMaxCols && out->ld >= cols &&
         out->rows_alloc >= n && out->ld % 2 == 0 &&
         ((reinterpret_cast<uintptr_t>(X2) | reinterpret_cast<uintptr_t>(X)) & 15) == 0 &&
         (reinterpret_cast<uintptr_t>(out->data) & 3) == 0;
}

cudaError_t dot_partials(const double* A, int64_t lda, const double* B, int64_t ldb, int rows,
                         int cols_logical, int minus_identity, double* partials, int* nblocks,
                         cudaStream_t stream, const int* skip, bool zero_pad) {
  const int cols = (zero_pad && (cols_logical & 1) && lda > cols_logical &&
                    (B == nullptr || ldb > cols_logical))
                       ? cols_logical + 1 : cols_logical;
  const bool rows_fit =
      cols % 2 == 0 && cols <= kFusedMaxCols && lda % 2 == 0 &&
      ((reinterpret_cast<uintptr_t>(A) & 15) == 0) &&
      (B == nullptr || (ldb % 2 == 0 && (reinterpret_cast<uintptr_t>(B) & 15) == 0));
  if (rows_fit && rows > 0) {
    // one block per row: partials holds one value per row
    const int npairs = cols / 2;
    count_launch();
#define GDM_DOTROWS(T)                                                                         \
  if (B != nullptr)                                                                            \
    dot_rows_kernel<T, true><<<rows, T, 0, stream>>>(A, lda, B, ldb, cols, minus_identity,     \
                                                     partials, skip);                          \
  else                                                                                         \
    dot_rows_kernel<T, false><<<rows, T, 0, stream>>>(A, lda, B, ldb, cols, minus_identity,    \
                                                      partials, skip)
    if (npairs <= 128 * kFusedPPT) {
      GDM_DOTROWS(128);
    } else if (npairs <= 256 * kFusedPPT) {
      GDM_DOTROWS(256);
    } else {
      GDM_DOTROWS(512);
    }
#undef GDM_DOTROWS
    *nblocks = rows;
    return cudaGetLastError();
  }
  const int nb = (rows + kRowsPerBlock - 1) / kRowsPerBlock;
  count_launch();
  dot_kernel<<<nb, kRowsPerBlock * 32, 0, stream>>>(A, lda, B, ldb, rows, cols, minus_identity,
                                                    partials, skip);
  *nblocks = nb;
  return cudaGetLastError();
}

cudaError_t reduce_partials(const double* partials, int nblocks, int nterms, double* out_dev,
                            cudaStream_t stream) {
  count_launch();
  reduce_kernel<<<1, 1024, 0, stream>>>(partials, nblocks, nterms, out_dev);
  return cudaGetLastError();
}

cudaError_t trs4_control(const double* partials, int nblocks, Trs4State* st, double tol_idem,
                         cudaStream_t stream) {
  count_launch();
  trs4_control_kernel<<<1, 256, 0, stream>>>(partials, nblocks, st, tol_idem);
  return cudaGetLastError();
}

cudaError_t x0_coefficients(const double* bounds_dev, double* coef_dev, cudaStream_t stream) {
  count_launch();
  x0_coef_kernel<<<1, 1, 0, stream>>>(bounds_dev, coef_dev);
  return cudaGetLastError();
}

cudaError_t canonical_x0_coefficients(const double* bounds_dev, const double* Ht, int64_t ld, int n,
                                      double n_occ, double* coef_dev, cudaStream_t stream) {
  count_launch();
  canonical_x0_coef_kernel<<<1, 256, 0, stream>>>(bounds_dev, Ht, ld, n, n_occ, coef_dev);
  return cudaGetLastError();
}

cudaError_t scale_coefficients(const double* bounds_dev, int inv_sqrt, double* coef_dev,
                               cudaStream_t stream) {
  count_launch();
  scale_coef_kernel<<<1, 1, 0, stream>>>(bounds_dev, inv_sqrt, coef_dev);
  return cudaGetLastError();
}

cudaError_t symmetrise(double* A, int64_t lda, int n, cudaStream_t stream) {
  const int t = (n + 31) / 32;
  if (t == 0) return cudaSuccess;
  count_launch();
  symmetrise_kernel<<<dim3(t, t), dim3(32, 8), 0, stream>>>(A, lda, n);
  return cudaGetLastError();
}

cudaError_t diag_fix(const double* A, int64_t lda, const double* Bt, int64_t ldb, double* C,
                     int64_t ldc, int n, int K, double alpha, double beta, const double* D,
                     int64_t ldd, double diag, const double* coef, cudaStream_t stream,
                     const int* skip) {
  if (n <= 0) return cudaSuccess;
  const int nb = (n + kRowsPerBlock - 1) / kRowsPerBlock;
  count_launch();
  diag_fix_kernel<<<nb, kRowsPerBlock * 32, 0, stream>>>(A, lda, Bt, ldb, C, ldc, n, K, alpha,
                                                         beta, D, ldd, diag, coef, skip);
  return cudaGetLastError();
}

cudaError_t trace_scale(double* X, int64_t ld, int n, double target, double* fix_out,
                        cudaStream_t stream) {
  if (n <= 0) return cudaSuccess;
  count_launch();
  trace_factor_kernel<<<1, 1024, 0, stream>>>(X, ld, n, target, fix_out);
  count_launch();
  scale_rows_kernel<<<n, 256, 0, stream>>>(X, ld, n, fix_out);
  return cudaGetLastError();
}

__global__ void zero_column_kernel(double* A, int64_t lda, int rows, int col) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < rows; i += gridDim.x * blockDim.x)
    A[i * lda + col] = 0.0;
}

cudaError_t zero_column(double* A, int64_t lda, int rows, int col, cudaStream_t stream) {
  if (rows <= 0 || col >= lda) return cudaSuccess;
  count_launch();
  zero_column_kernel<<<(rows + 255) / 256, 256, 0, stream>>>(A, lda, rows, col);
  return cudaGetLastError();
}

cudaError_t set_identity(double* A, int64_t lda, int n, cudaStream_t stream) {
  if (n <= 0) return cudaSuccess;
  count_launch();
  identity_kernel<<<n, 256, 0, stream>>>(A, lda, n);
  return cudaGetLastError();
}

bool matvec_rows_fit(const double* A, int64_t lda, int n, const double* v) {
  // dot_partials' one-block-per-row path with the vector as every row of B (ldb = 0)
  return n > 0 && n % 2 == 0 && n <= kFusedMaxCols && lda % 2 == 0 &&
         (reinterpret_cast<uintptr_t>(A) & 15) == 0 && (reinterpret_cast<uintptr_t>(v) & 15) == 0;
}

cudaError_t fill_rademacher(double* v, int n, unsigned seed, cudaStream_t stream) {
  if (n <= 0) return cudaSuccess;
  count_launch();
  rademacher_kernel<<<(n + 255) / 256, 256, 0, stream>>>(v, n, seed);
  return cudaGetLastError();
}

}  // namespace gdm
