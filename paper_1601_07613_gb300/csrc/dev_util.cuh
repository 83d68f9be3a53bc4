// Device helpers shared by the kernels.
//
// FP32 <-> FP64 conversions by integer bit manipulation.  On this GPU the
// FP64 pipe runs at 1/64 of the FP32 rate and the hardware conversion
// instructions issue on it, so converting a 40-value element block costs as
// much as 40 FP64 operations; the integer forms below issue on the integer
// pipe only.  Both implement IEEE 754 binary64 <-> binary32 conversion with
// round-to-nearest-even, including zeros, subnormals, overflow, infinities and
// NaNs (quieted).
#pragma once

#include <cfloat>
#include <cstdint>

namespace dgc {

// Programmatic dependent launch.  pdl_wait() blocks until the grid launched
// before this one on the stream has completed and its writes are visible (a
// no-op for a launch without a programmatic dependency).  pdl_trigger() lets
// the next grid's blocks be scheduled once every block of this grid has issued
// it or exited.  A kernel issues pdl_trigger() only after pdl_wait(), so when a
// grid starts, the grid two launches back has completed: it may read that
// grid's output at once and must wait before touching its predecessor's.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// Full conversions (every input class); called out of line for the rare
// inputs the fast paths below do not cover.
static __device__ __noinline__ float d2f_any(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const unsigned sign = (unsigned)(b >> 32) & 0x80000000u;
  const unsigned ed = (unsigned)(b >> 52) & 0x7FFu;
  const unsigned long long mant = b & 0xFFFFFFFFFFFFFull;
  const int e = (int)ed - 896;  // binary32 exponent field of a normal result
  unsigned out;
  if (ed == 0x7FFu) {
    out = 0x7F800000u | (mant ? 0x400000u : 0u);  // infinity, or a quiet NaN
  } else if (e >= 255) {
    out = 0x7F800000u;  // overflow
  } else if (e > 0) {
    const unsigned m = (unsigned)(mant >> 29);       // top 23 fraction bits
    const unsigned rem = (unsigned)mant & 0x1FFFFFFFu;  // the 29 dropped bits
    const unsigned up = (rem > 0x10000000u) | ((rem == 0x10000000u) & (m & 1u));
    out = (((unsigned)e << 23) | m) + up;  // a carry rounds into the exponent (up to infinity)
  } else {
    // binary32 subnormal or zero: the 53-bit significand in units of 2^-149
    const int s = 30 - e;  // right shift, >= 30
    if (ed == 0u || s > 54) {
      out = 0u;
    } else {
      const unsigned long long M = mant | (1ull << 52);
      const unsigned q = (unsigned)(M >> s);
      const unsigned long long r = M & ((1ull << s) - 1ull), h = 1ull << (s - 1);
      out = q + (unsigned)((r > h) | ((r == h) & (q & 1u)));  // may round up to the smallest normal
    }
  }
  return __uint_as_float(out | sign);
}

static __device__ __noinline__ double f2d_any(float f) {
  const unsigned u = __float_as_uint(f);
  const unsigned long long sign = (unsigned long long)(u & 0x80000000u) << 32;
  const unsigned ef = (u >> 23) & 0xFFu;
  const unsigned m = u & 0x7FFFFFu;
  unsigned long long bits;
  if (ef == 0xFFu) {
    bits = 0x7FF0000000000000ull | ((unsigned long long)m << 29);
  } else if (ef != 0u) {
    bits = ((unsigned long long)(ef + 896u) << 52) | ((unsigned long long)m << 29);
  } else if (m == 0u) {
    bits = 0ull;
  } else {
    // binary32 subnormal m 2^-149: normalise around its leading bit k
    const int k = 31 - __clz(m);
    const unsigned long long frac = ((unsigned long long)m << (52 - k)) & 0xFFFFFFFFFFFFFull;
    bits = ((unsigned long long)(k + 874) << 52) | frac;
  }
  return __longlong_as_double((long long)(sign | bits));
}

// Fast paths.  binary64 -> binary32 for results in the normal range: adding
// 0x0FFFFFFF plus the lowest kept bit to the 29 dropped bits rounds to nearest
// even, the carry running into the exponent field (up to infinity); the
// exponent is then rebiased by 1023 - 127.  binary32 -> binary64 for normal
// inputs is a shift and a rebias.  Signed zeros (frequent: uniform regions give
// exact zero increments) are handled inline too.  Anything else goes to the
// calls above.
__device__ __forceinline__ float d2f(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const unsigned ed = (unsigned)(b >> 52) & 0x7FFu;
  if (ed - 897u < 254u) {  // binary32 exponent field 1..254
    const unsigned long long t = b + 0x0FFFFFFFull + ((b >> 29) & 1ull);
    const unsigned mag = (unsigned)((t >> 29) & 0x3FFFFFFFFull) - (896u << 23);
    return __uint_as_float(mag | ((unsigned)(b >> 32) & 0x80000000u));
  }
  if ((b << 1) == 0ull) return __uint_as_float((unsigned)(b >> 32));  // +-0
  return d2f_any(x);
}

__device__ __forceinline__ double f2d(float f) {
  const unsigned u = __float_as_uint(f);
  const unsigned ef = (u >> 23) & 0xFFu;
  if (ef - 1u < 254u) {  // normal
    const unsigned long long bits = ((unsigned long long)(u & 0x7FFFFFFFu) << 29) + (896ull << 52);
    return __longlong_as_double((long long)(bits | ((unsigned long long)(u & 0x80000000u) << 32)));
  }
  if ((u << 1) == 0u) return __longlong_as_double((long long)((unsigned long long)u << 32));  // +-0
  return f2d_any(f);
}

// FP32 pairs (the FP64 lanes' basis contractions): a value x as hi + lo, hi =
// fl32(x), lo = fl32(x - hi), 2^-48 of x.  s += t b runs on the FP32 pipe as
// the error-free product of the high parts (the FMA returns a product's
// rounding error exactly: Dekker's product) plus the two cross terms, added
// into s by Knuth's two-sum (TAOCP vol. 2, 4.2.2): 12 FP32 operations for one
// FP64 FMA.  The intrinsics keep the compiler from contracting the error-free
// steps into FMAs.
struct DF {
  float h, l;
};
__device__ __forceinline__ DF df_split(double x) {
  const float h = d2f(x);
  return DF{h, d2f(x - f2d(h))};
}
__device__ __forceinline__ double df_join(DF a) { return f2d(a.h) + f2d(a.l); }
// a b for two pairs, as a pair (Dekker's product of the high parts plus the
// cross terms; the lo * lo term is below the pairs' precision)
__device__ __forceinline__ DF df_mul(DF a, DF b) {
  const float p = __fmul_rn(a.h, b.h);
  float e = __fmaf_rn(a.h, b.h, -p);
  e = __fmaf_rn(a.h, b.l, e);
  e = __fmaf_rn(a.l, b.h, e);
  const float h = __fadd_rn(p, e);
  return DF{h, __fsub_rn(e, __fsub_rn(h, p))};
}
// s += t b (t a table value as (hi, lo)); the intrinsics keep the compiler from
// contracting the error-free steps into FMAs
__device__ __forceinline__ void df_fma(DF& s, float2 t, DF b) {
  const float p = __fmul_rn(t.x, b.h);
  float e = __fmaf_rn(t.x, b.h, -p);
  e = __fmaf_rn(t.x, b.l, e);
  e = __fmaf_rn(t.y, b.h, e);
  const float u = __fadd_rn(s.h, p);
  const float bp = __fsub_rn(u, s.h);
  const float err = __fadd_rn(__fsub_rn(s.h, __fsub_rn(u, bp)), __fsub_rn(p, bp));
  s.h = u;
  s.l = __fadd_rn(s.l, __fadd_rn(err, e));
}

// Two variables at once (sharing one table value) on the packed FP32 pipe
// (__fmul2_rn, __ffma2_rn, __fadd2_rn): s_k += t b_k for k = 0, 1, with the
// table value t = (hi, hi, lo, lo) and s, b as (hi pair, lo pair); the same
// steps as df_fma, each subtraction an FMA with -1 (one rounding, as a
// subtraction).
__device__ __forceinline__ void df_fma2(float2& sh, float2& sl, float4 t, float2 bh, float2 bl) {
  const float2 th = make_float2(t.x, t.y), tl = make_float2(t.z, t.w), m1 = make_float2(-1.0f, -1.0f);
  const float2 p = __fmul2_rn(th, bh);
  float2 e = __ffma2_rn(th, bh, __fmul2_rn(p, m1));
  e = __ffma2_rn(th, bl, e);
  e = __ffma2_rn(tl, bh, e);
  const float2 u = __fadd2_rn(sh, p);
  const float2 bp = __ffma2_rn(sh, m1, u);   // u - sh
  const float2 ap = __ffma2_rn(bp, m1, u);   // u - bp
  const float2 err = __fadd2_rn(__ffma2_rn(ap, m1, sh), __ffma2_rn(bp, m1, p));
  sh = u;
  sl = __fadd2_rn(sl, __fadd2_rn(err, e));
}

template <typename T>
__device__ __forceinline__ T to(double x);
template <>
__device__ __forceinline__ double to<double>(double x) { return x; }
template <>
__device__ __forceinline__ float to<float>(double x) { return d2f(x); }

__device__ __forceinline__ double widen(float x) { return f2d(x); }
__device__ __forceinline__ double widen(double x) { return x; }
__device__ __forceinline__ float narrow(double x) { return d2f(x); }

// block-wide minimum of non-negative values, combined into *out with one
// atomicMin on the bit pattern (non-negative IEEE values order like their bits).
// The atomic is skipped when the block's minimum is not below the value read
// from L2 first: *out only decreases, so a stale read is never too small, and
// a skipped block could not have lowered it.  Most blocks skip, which keeps
// thousands of same-address atomics from serialising at the end of the pass.
__device__ __forceinline__ void block_min_to(double v, unsigned long long* out) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmin(v, __shfl_xor_sync(0xffffffffu, v, o));
  __shared__ double wmin[32];
  if ((threadIdx.x & 31) == 0) wmin[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double b = wmin[0];
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) b = fmin(b, wmin[w]);
    const unsigned long long bits = (unsigned long long)__double_as_longlong(b);
    if (bits < __ldcg(out)) atomicMin(out, bits);
  }
}

__device__ __forceinline__ void block_min_to(float v, unsigned* out) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fminf(v, __shfl_xor_sync(0xffffffffu, v, o));
  __shared__ float wminf[32];
  if ((threadIdx.x & 31) == 0) wminf[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    float b = wminf[0];
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) b = fminf(b, wminf[w]);
    const unsigned bits = __float_as_uint(b);
    if (bits < __ldcg(out)) atomicMin(out, bits);
  }
}

// The CFL reduction runs in two passes: an FP32 estimate of every element's
// step, then an exact FP64 evaluation of the elements whose estimate lies
// within this relative margin of the smallest estimate.  The FP32 estimate
// of |u| + c has a relative error near 1e-6, far inside the margin, so the
// FP64 minimum is always among the re-evaluated elements.
constexpr float kCflMargin = 1.0f / 1024.0f;

}  // namespace dgc
