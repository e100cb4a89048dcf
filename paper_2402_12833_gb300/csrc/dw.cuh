// Double-word ("double-FP32") arithmetic for the FP64-accurate solver on the
// FP32 pipe.
//
// A value is the unevaluated sum hi + lo of two floats with |lo| <= ulp(hi),
// about 48 significant bits (relative rounding ~2^-47 instead of FP64's
// 2^-53), stored in 8 bytes like a double.  GB300 issues FP32 fused
// multiply-adds at 64 times the FP64 rate, so a double-word multiply-add of
// about 15 FP32 operations still runs several times faster than FP64 in the
// ALU-bound block kernels.  Exponent range: that of float (normal numbers
// from 2^-126); the low word of values below about 2^-100 is flushed, which
// only loses precision there.
//
// The building blocks are the error-free transformations TwoSum (Knuth),
// Fast2Sum (Dekker) and the FMA-based TwoProd; addition is the "sloppy"
// double-word sum and multiplication the FMA-based double-word product of
// Joldes, Muller and Popescu, "Tight and rigorous error bounds for basic
// building blocks of double-word arithmetic", ACM TOMS 44 (2017).  Their
// absolute error is a small multiple of 2^-48 (|x| + |y|) (resp. |x y|),
// which is what a sum of products needs: the same normwise bound as FP64
// with a 48-bit significand.  fma(a, b, c) = c + a b folds the product's low
// terms into the sum before one renormalisation.
//
// Conversions to and from double use integer operations only (the FP64
// pipe is the resource being avoided): a double is split by truncation into
// its leading 24 bits and the next (up to 24) bits; a pair is assembled into
// the double nearest below in magnitude (truncation, error < 2^-52 relative).
#pragma once

#include <cuda_runtime.h>
#include <math.h>
#include <string.h>

#include <type_traits>

#ifndef __CUDA_ARCH__
#include <cmath>
#endif

namespace mpcg {

struct dw;
__host__ __device__ inline dw dw_from_double(double d);
__host__ __device__ inline double dw_to_double(float hi, float lo);

struct __align__(8) dw {
  float hi, lo;
  dw() = default;
  __host__ __device__ constexpr dw(float h, float l) : hi(h), lo(l) {}
  __host__ __device__ constexpr dw(int v) : hi((float)v), lo(0.f) {}   // small integers (0, 1) exactly
  __host__ __device__ constexpr dw(float v) : hi(v), lo(0.f) {}
  __host__ __device__ dw(double d);
  __host__ __device__ explicit operator double() const { return dw_to_double(hi, lo); }
  __host__ __device__ explicit operator float() const { return hi + lo; }
};

namespace dwd {

__host__ __device__ inline unsigned long long dbits(double d) {
#ifdef __CUDA_ARCH__
  return (unsigned long long)__double_as_longlong(d);
#else
  unsigned long long u;
  memcpy(&u, &d, 8);
  return u;
#endif
}
__host__ __device__ inline double bits_d(unsigned long long u) {
#ifdef __CUDA_ARCH__
  return __longlong_as_double((long long)u);
#else
  double d;
  memcpy(&d, &u, 8);
  return d;
#endif
}
__host__ __device__ inline unsigned fbits(float f) {
#ifdef __CUDA_ARCH__
  return __float_as_uint(f);
#else
  unsigned u;
  memcpy(&u, &f, 4);
  return u;
#endif
}
__host__ __device__ inline float bits_f(unsigned u) {
#ifdef __CUDA_ARCH__
  return __uint_as_float(u);
#else
  float f;
  memcpy(&f, &u, 4);
  return f;
#endif
}
__host__ __device__ inline int top_bit(unsigned v) {   // v > 0
#ifdef __CUDA_ARCH__
  return 31 - __clz((int)v);
#else
  return 31 - __builtin_clz(v);
#endif
}

// rounded float operations that the compiler may not contract into FMAs
__host__ __device__ inline float add(float a, float b) {
#ifdef __CUDA_ARCH__
  return __fadd_rn(a, b);
#else
  volatile float s = a + b;
  return s;
#endif
}
__host__ __device__ inline float sub(float a, float b) {
#ifdef __CUDA_ARCH__
  return __fsub_rn(a, b);
#else
  volatile float s = a - b;
  return s;
#endif
}
__host__ __device__ inline float mul(float a, float b) {
#ifdef __CUDA_ARCH__
  return __fmul_rn(a, b);
#else
  volatile float s = a * b;
  return s;
#endif
}
__host__ __device__ inline float fmaf_(float a, float b, float c) {
#ifdef __CUDA_ARCH__
  return __fmaf_rn(a, b, c);
#else
  return std::fma(a, b, c);
#endif
}

// s + e = a + b exactly (Knuth's TwoSum, no ordering requirement)
__host__ __device__ inline void two_sum(float a, float b, float& s, float& e) {
  s = add(a, b);
  const float bb = sub(s, a);
  e = add(sub(a, sub(s, bb)), sub(b, bb));
}
// s + e = a + b exactly when |a| >= |b| (Dekker's Fast2Sum)
__host__ __device__ inline void fast_two_sum(float a, float b, float& s, float& e) {
  s = add(a, b);
  e = sub(b, sub(s, a));
}

}  // namespace dwd

__host__ __device__ inline dw dw_from_double(double d) {
  using namespace dwd;
  const unsigned long long u = dbits(d);
  const unsigned sgn = (unsigned)(u >> 63) << 31;
  const int e = (int)((u >> 52) & 0x7FF);
  const unsigned long long m = u & ((1ULL << 52) - 1);
  if (e == 0) return dw(bits_f(sgn), 0.f);   // zero, or a double subnormal: flushed
  if (e == 0x7FF) return dw((float)d, 0.f);   // inf / nan
  const int E = e - 1023;
  if (E < -126) return dw(bits_f(sgn), 0.f);
  if (E > 127) return dw(bits_f(sgn | 0x7F800000u), 0.f);
  const float hi = bits_f(sgn | ((unsigned)(E + 127) << 23) | (unsigned)(m >> 29));
  const unsigned rem = (unsigned)(m & ((1u << 29) - 1));   // value rem * 2^(E - 52)
  if (rem == 0) return dw(hi, 0.f);
  const int k = top_bit(rem);                               // 0 .. 28
  const int el = E - 52 + k;
  if (el < -126) return dw(hi, 0.f);
  const unsigned mant = (k >= 23 ? rem >> (k - 23) : rem << (23 - k)) & 0x7FFFFFu;
  return dw(hi, bits_f(sgn | ((unsigned)(el + 127) << 23) | mant));
}

__host__ __device__ inline double dw_to_double(float hi, float lo) {
  using namespace dwd;
  const unsigned uh = fbits(hi), ul = fbits(lo);
  const unsigned eh = (uh >> 23) & 0xFF;
  const unsigned long long sgn = (unsigned long long)(uh >> 31) << 63;
  if (eh == 0) return bits_d(sgn);   // zero (or a float subnormal, flushed)
  if (eh == 0xFF) return (double)hi;
  int E = (int)eh - 127;
  unsigned long long M = (1ULL << 52) | ((unsigned long long)(uh & 0x7FFFFFu) << 29);
  const unsigned el = (ul >> 23) & 0xFF;
  if (el != 0 && el != 0xFF) {
    const unsigned long long Ml = (1u << 23) | (ul & 0x7FFFFFu);
    const int sh = (int)el - 127 - E + 29;   // lo = Ml * 2^sh units of hi's last bit
    if (sh > 10) return (double)hi + (double)lo;   // not a normalised pair
    const unsigned long long Ma = sh >= 0 ? Ml << sh : (sh > -40 ? Ml >> -sh : 0ULL);
    if (((uh ^ ul) >> 31) == 0) {
      M += Ma;
      if (M >> 53) {
        M >>= 1;
        E += 1;
      }
    } else {
      M -= Ma;
      if (!(M >> 52)) {
        M <<= 1;
        E -= 1;
      }
    }
  }
  return bits_d(sgn | ((unsigned long long)(E + 1023) << 52) | (M & ((1ULL << 52) - 1)));
}

__host__ __device__ inline dw::dw(double d) { *this = dw_from_double(d); }

// Accumulator of a long sum of double-word products with deferred
// renormalisation (the compensated dot product "Dot2" of Ogita, Rump and
// Oishi, SIAM J. Sci. Comput. 26 (2005), with double-word inputs): the
// leading parts of the products are added error-free into s by TwoSum, and
// the exact product errors, the cross terms and the TwoSum errors are summed
// in plain FP32 into e; the pair is renormalised once at the end.  12 FP32
// operations per product instead of 15.
struct dwacc {
  float s, e;
};
__host__ __device__ inline dwacc dwacc_of(dw v) { return {v.hi, v.lo}; }
__host__ __device__ inline void mac(dwacc& c, dw a, dw b) {
  const float p = dwd::mul(a.hi, b.hi);
  float pe = dwd::fmaf_(a.hi, b.hi, -p);
  pe = dwd::fmaf_(a.hi, b.lo, pe);
  pe = dwd::fmaf_(a.lo, b.hi, pe);
  float s, t;
  dwd::two_sum(c.s, p, s, t);
  c.s = s;
  c.e = dwd::add(c.e, dwd::add(t, pe));
}
__host__ __device__ inline dw dwacc_value(dwacc c) {
  float zh, zl;
  dwd::fast_two_sum(c.s, c.e, zh, zl);
  return dw(zh, zl);
}

// The accumulator type of element type T (the element itself for float and
// double, whose mac is one fused multiply-add) and its conversions.
template <typename T>
struct Acc {
  using type = T;
  __host__ __device__ static T of(T v) { return v; }
  __host__ __device__ static T value(T v) { return v; }
};
template <>
struct Acc<dw> {
  using type = dwacc;
  __host__ __device__ static dwacc of(dw v) { return dwacc_of(v); }
  __host__ __device__ static dw value(dwacc v) { return dwacc_value(v); }
};
__host__ __device__ inline void mac(float& c, float a, float b) { c = fmaf(a, b, c); }
__host__ __device__ inline void mac(double& c, double a, double b) { c = fma(a, b, c); }

// true for the double-word element type (its kernels need more registers)
template <typename T>
constexpr bool kIsDw = std::is_same<T, dw>::value;

__host__ __device__ inline dw operator-(dw x) { return dw(-x.hi, -x.lo); }

// sloppy double-word sum (Joldes-Muller-Popescu)
__host__ __device__ inline dw operator+(dw x, dw y) {
  float s, e, zh, zl;
  dwd::two_sum(x.hi, y.hi, s, e);
  const float w = dwd::add(e, dwd::add(x.lo, y.lo));
  dwd::fast_two_sum(s, w, zh, zl);
  return dw(zh, zl);
}
__host__ __device__ inline dw operator-(dw x, dw y) { return x + (-y); }

// double-word product with FMA (Joldes-Muller-Popescu)
__host__ __device__ inline dw operator*(dw x, dw y) {
  const float p = dwd::mul(x.hi, y.hi);
  float e = dwd::fmaf_(x.hi, y.hi, -p);
  e = dwd::fmaf_(x.hi, y.lo, e);
  e = dwd::fmaf_(x.lo, y.hi, e);
  float zh, zl;
  dwd::fast_two_sum(p, e, zh, zl);
  return dw(zh, zl);
}

// double-word quotient: first quotient of the high words, then one
// correction from the double-word remainder x - y q (Joldes-Muller-Popescu,
// DWDivDW1)
__host__ __device__ inline dw operator/(dw x, dw y) {
  const float th = x.hi / y.hi;
  const dw r = x - y * dw(th, 0.f);
  const float tl = r.hi / y.hi;
  float zh, zl;
  dwd::fast_two_sum(th, tl, zh, zl);
  return dw(zh, zl);
}

__host__ __device__ inline dw& operator+=(dw& x, dw y) { return x = x + y; }
__host__ __device__ inline dw& operator-=(dw& x, dw y) { return x = x - y; }
__host__ __device__ inline dw& operator*=(dw& x, dw y) { return x = x * y; }

}  // namespace mpcg

// c + a b with one renormalisation: the product's exact low part and the
// cross terms join the low word of the sum (global scope so that unqualified
// calls in the kernels see it beside the float and double overloads).
__host__ __device__ inline mpcg::dw fma(mpcg::dw a, mpcg::dw b, mpcg::dw c) {
  using namespace mpcg::dwd;
  const float p = mul(a.hi, b.hi);
  float pe = fmaf_(a.hi, b.hi, -p);
  pe = fmaf_(a.hi, b.lo, pe);
  pe = fmaf_(a.lo, b.hi, pe);
  float s, e, zh, zl;
  two_sum(c.hi, p, s, e);
  e = add(e, add(c.lo, pe));
  fast_two_sum(s, e, zh, zl);
  return mpcg::dw(zh, zl);
}

#ifdef __CUDACC__
__device__ inline mpcg::dw __shfl_xor_sync(unsigned mask, mpcg::dw v, int lane, int width = 32) {
  return mpcg::dw(__shfl_xor_sync(mask, v.hi, lane, width), __shfl_xor_sync(mask, v.lo, lane, width));
}
__device__ inline mpcg::dw __shfl_up_sync(unsigned mask, mpcg::dw v, unsigned d, int width = 32) {
  return mpcg::dw(__shfl_up_sync(mask, v.hi, d, width), __shfl_up_sync(mask, v.lo, d, width));
}
__device__ inline mpcg::dw __shfl_down_sync(unsigned mask, mpcg::dw v, unsigned d, int width = 32) {
  return mpcg::dw(__shfl_down_sync(mask, v.hi, d, width), __shfl_down_sync(mask, v.lo, d, width));
}
__device__ inline mpcg::dw __ldcs(const mpcg::dw* p) {
  const float2 q = __ldcs(reinterpret_cast<const float2*>(p));
  return mpcg::dw(q.x, q.y);
}
__device__ inline mpcg::dw __ldg(const mpcg::dw* p) {
  const float2 q = __ldg(reinterpret_cast<const float2*>(p));
  return mpcg::dw(q.x, q.y);
}
__device__ inline mpcg::dw __ldcg(const mpcg::dw* p) {
  const float2 q = __ldcg(reinterpret_cast<const float2*>(p));
  return mpcg::dw(q.x, q.y);
}
#endif
