// SSP-RK3 in increment form, used by the two FP32 precision forms of the step.
//
// With delta_0 = 0 and b = (1, 1/4, 2/3), stage s = 0, 1, 2 computes
//   delta_{s+1} = b_s (delta_s + dt L(u_s)),   u_{s+1} = u_0 + delta_{s+1},
// which is the Shu-Osher form
//   u1 = u0 + dt L(u0),  u2 = 3/4 u0 + 1/4 (u1 + dt L(u1)),  u3 = 1/3 u0 + 2/3 (u2 + dt L(u2))
// written around u0.  The increments are O(dt) and carry the FP32 flux error
// already, so they are kept in FP32; only the state update is done at full
// precision, once per step:
//  - DGC_FP32_MIXED: FP64 state, u = u0 + delta_3 (one FP64 FMA per value);
//  - DGC_FP32_KAHAN: the state is an FP32 pair (hi, lo) per value and delta_3
//    is added with Kahan's compensated summation (lo = minus the compensation).
// Stages 0 and 1 write the FP32 record of u_{s+1} = u0 + delta_{s+1} read by the
// next stage's fluxes: mean pair (hi, lo) updated by an error-free sum, modes
// j >= 1 by one FP32 addition.
//
// Record layout (floats per element, NF in all, padded to a multiple of 4):
// hi[M], lo[M] of the mean state phi0 c0, then the modes j >= 1 as [M][NP-1].
// Kahan state: the record, then lo of the modes j >= 1 as [M][NP-1], padded.
#pragma once

#include "dev_util.cuh"
#include "device.cuh"

namespace dgc {

__host__ __device__ constexpr int round4(int n) { return (n + 3) / 4 * 4; }

// the FP32 pair nearest to an FP64 value
struct F2 {
  float hi, lo;
};
__device__ __forceinline__ F2 split_f2(double x) {
  F2 r;
  r.hi = d2f(x);
  r.lo = d2f(x - f2d(r.hi));
  return r;
}

// Kahan (compensated) addition of d to the pair value hi + lo
__device__ __forceinline__ void kahan_add(float& hi, float& lo, float d) {
  const float y = d + lo;
  const float t = hi + y;
  lo = y - (t - hi);
  hi = t;
}

// x * (c.hi + c.lo) with the product's low part kept (2 FP32 operations)
__device__ __forceinline__ float mul_f2(float x, F2 c) { return fmaf(x, c.hi, x * c.lo); }

// (hi, lo) <- the pair nearest to hi + lo + x (c.hi + c.lo): the product's
// rounding error from one FMA (two-product), Knuth's two-sum with hi, then a
// renormalisation; about 2^-46 relative, however large x c is against hi.
__device__ __forceinline__ void pair_add_scaled(float& hi, float& lo, float x, F2 c) {
  const float ph = x * c.hi;
  const float pl = fmaf(x, c.hi, -ph) + x * c.lo;
  const float s = hi + ph;
  const float bb = s - hi;
  const float e = (hi - (s - bb)) + (ph - bb);
  const float l = e + (lo + pl);
  hi = s + l;
  lo = l - (hi - s);
}

// element blocks of N floats (16-byte aligned when N % 4 == 0, else 8-byte)
template <int N>
__device__ __forceinline__ void ldv(const float* __restrict__ src, float (&v)[N]) {
  if constexpr (N % 4 == 0) {
    const float4* s = reinterpret_cast<const float4*>(src);
#pragma unroll
    for (int i = 0; i < N / 4; ++i) {
      const float4 x = s[i];
      v[4 * i] = x.x;
      v[4 * i + 1] = x.y;
      v[4 * i + 2] = x.z;
      v[4 * i + 3] = x.w;
    }
  } else {
    static_assert(N % 2 == 0, "even block");
    const float2* s = reinterpret_cast<const float2*>(src);
#pragma unroll
    for (int i = 0; i < N / 2; ++i) {
      const float2 x = s[i];
      v[2 * i] = x.x;
      v[2 * i + 1] = x.y;
    }
  }
}
template <int N>
__device__ __forceinline__ void stv(float* dst, const float (&v)[N]) {
  if constexpr (N % 4 == 0) {
    float4* d = reinterpret_cast<float4*>(dst);
#pragma unroll
    for (int i = 0; i < N / 4; ++i) d[i] = make_float4(v[4 * i], v[4 * i + 1], v[4 * i + 2], v[4 * i + 3]);
  } else {
    static_assert(N % 2 == 0, "even block");
    float2* d = reinterpret_cast<float2*>(dst);
#pragma unroll
    for (int i = 0; i < N / 2; ++i) d[i] = make_float2(v[2 * i], v[2 * i + 1]);
  }
}

template <int N>
__device__ __forceinline__ void ld4(const float* __restrict__ src, float (&v)[N]) {
  static_assert(N % 4 == 0, "float4 blocks");
  const float4* s = reinterpret_cast<const float4*>(src);
#pragma unroll
  for (int i = 0; i < N / 4; ++i) {
    const float4 x = s[i];
    v[4 * i] = x.x;
    v[4 * i + 1] = x.y;
    v[4 * i + 2] = x.z;
    v[4 * i + 3] = x.w;
  }
}
template <int N>
__device__ __forceinline__ void st4(float* dst, const float (&v)[N]) {
  static_assert(N % 4 == 0, "float4 blocks");
  float4* d = reinterpret_cast<float4*>(dst);
#pragma unroll
  for (int i = 0; i < N / 4; ++i) d[i] = make_float4(v[4 * i], v[4 * i + 1], v[4 * i + 2], v[4 * i + 3]);
}

// Epilogue of the last color in increment form for element e, whose complete
// FP32 right-hand side is L.  B holds the record the fluxes used (the record of
// u0 at stage 0).  phi0 = the constant basis function.
// Every branch issues its loads before its stores: the stores may alias what
// is read (the same arrays), so the compiler keeps a load that follows a store
// behind it, and a load-store-load sequence costs one memory round trip each.
template <int M, int NP, typename Blk>
__device__ __forceinline__ void incr_last(const StageArgs& S, int64_t e, const float (&L)[M * NP], const Blk& B,
                                          double phi0) {
  constexpr int NV = M * NP, NM = NP - 1, NF = round4(M * (NP + 1)), LOM = round4(M * NM);
  const double dt = *S.dt;
  const F2 dtp = split_f2(dt);
  float d[NV];
  float* dp = S.delta + e * NV;
  if (S.stage < 2) {
    float r[NF];
    if (S.stage == 0) {
#pragma unroll
      for (int i = 0; i < NV; ++i) d[i] = mul_f2(L[i], dtp);
#pragma unroll
      for (int m = 0; m < M; ++m) {
        r[m] = B.hi[m];
        r[M + m] = B.lo[m];
#pragma unroll
        for (int j = 0; j < NM; ++j) r[2 * M + m * NM + j] = B.cd[m][j];
      }
    } else {
      ldv<NV>(dp, d);
      ld4<NF>(S.rec0 + e * S.rec0_stride, r);
#pragma unroll
      for (int i = 0; i < NV; ++i) d[i] = 0.25f * (d[i] + mul_f2(L[i], dtp));
    }
    const F2 p0 = split_f2(phi0);
#pragma unroll
    for (int m = 0; m < M; ++m) {
      pair_add_scaled(r[m], r[M + m], d[m * NP], p0);
#pragma unroll
      for (int j = 0; j < NM; ++j) r[2 * M + m * NM + j] += d[m * NP + 1 + j];
    }
#pragma unroll
    for (int i = M * (NP + 1); i < NF; ++i) r[i] = 0.0f;
    stv<NV>(dp, d);
    st4<NF>(S.rec_out + e * NF, r);
    return;
  }
  // stage 2: delta_2 + dt L; b_2 = 2/3 is applied by the state update
  ldv<NV>(dp, d);
#pragma unroll
  for (int i = 0; i < NV; ++i) d[i] = d[i] + mul_f2(L[i], dtp);
  if (S.kstate) {
    float* ks = S.kstate + e * S.rec0_stride;
    float r[NF], lo[LOM];
    ld4<NF>(ks, r);
    ld4<LOM>(ks + NF, lo);
    const F2 c23 = split_f2(2.0 / 3.0), k23 = split_f2(2.0 / 3.0 * phi0);
#pragma unroll
    for (int m = 0; m < M; ++m) {
      kahan_add(r[m], r[M + m], mul_f2(d[m * NP], k23));
#pragma unroll
      for (int j = 0; j < NM; ++j) kahan_add(r[2 * M + m * NM + j], lo[m * NM + j], mul_f2(d[m * NP + 1 + j], c23));
    }
    st4<NF>(ks, r);
    st4<LOM>(ks + NF, lo);
  } else {
    // FP64 state: u = u0 + (2/3) f64(d), in chunks of CH value pairs (all of a
    // chunk's loads before its stores; u0 was prefetched into L2)
    constexpr int H = NV / 2, CH = 5;
    const double2* u0 = reinterpret_cast<const double2*>(S.u0 + e * NV);
    double2* u = reinterpret_cast<double2*>(S.uout + e * NV);
#pragma unroll
    for (int c0 = 0; c0 < H; c0 += CH) {
      double2 a[CH];
#pragma unroll
      for (int i = 0; i < CH; ++i)
        if (c0 + i < H) a[i] = u0[c0 + i];
#pragma unroll
      for (int i = 0; i < CH; ++i)
        if (c0 + i < H)
          u[c0 + i] = make_double2(fma(2.0 / 3.0, f2d(d[2 * (c0 + i)]), a[i].x),
                                   fma(2.0 / 3.0, f2d(d[2 * (c0 + i) + 1]), a[i].y));
    }
  }
}

}  // namespace dgc
