// Euler fluxes in perturbation form, for the FP32 kernels.
//
// On a fine mesh the terms of Eq. 2 are much larger than their sum: a
// constant state produces volume and surface integrals of size |F|/h that
// cancel exactly.  FP32 rounding of the state (and of F) leaves an error of
// eps_32 |F| / h in every term, which at h = 1/724, p = 3 is about 1e-5 of the
// right-hand side.  The FP32 kernels therefore work relative to a per-element
// reference state ub (the element mean, phi_0 c_0, split into an FP32 pair
// hi + lo):
//
//   * the trace at a point is ub + d with the deviation d = lo + sum_{j>=1}
//     phi_j c_j, so d is accurate relative to its own (small) size;
//   * F(ub + d) - F(ub) is evaluated with formulas in which every term is
//     proportional to d (no cancellation of O(|F|) quantities);
//   * the constant flux F(ub) is left out of both the volume and the surface
//     integrals of the element: by the divergence theorem its two
//     contributions cancel, and both quadrature rules integrate them exactly
//     (volume integrand of degree p-1, face integrand of degree p).
//
// The result equals Eq. 2 in exact arithmetic; in FP32 the rounding error is
// relative to the deviations instead of to |F|.
#pragma once

namespace dgc {

// Reciprocal and square root of the FP32 flux: the hardware approximations
// (about 1 ulp; arguments are densities and sound speeds of order one, so
// flushing subnormals is harmless), one instruction each instead of the IEEE
// sequences with their correction paths.  Their error is far below the FP32
// flux's own rounding in the right-hand side.
__device__ __forceinline__ float rcp_fast(float x) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
__device__ __forceinline__ float sqrt_fast(float x) {
  float r;
  asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}

// Per-element reference state and the quantities of F(ub) the differences use.
template <int DIM>
struct PertRef {
  static constexpr int M = DIM + 2;
  float u[M];      // ub: rho, momentum, E
  float mb2;       // |m_b|^2
  float pb;        // pressure of ub
  float Hb;        // E_b + p_b
  __device__ __forceinline__ void init(const float (&hi)[M]) {
#pragma unroll
    for (int k = 0; k < M; ++k) u[k] = hi[k];
    mb2 = 0.0f;
#pragma unroll
    for (int a = 0; a < DIM; ++a) mb2 += u[1 + a] * u[1 + a];
    pb = 0.4f * (u[M - 1] - 0.5f * mb2 / u[0]);
    Hb = u[M - 1] + pb;
  }
};

// Shared pieces of F(ub + d) - F(ub) that do not depend on the direction.
template <int DIM>
struct PertState {
  static constexpr int M = DIM + 2;
  float inv;  // 1 / (rho rho_b)
  float dp;   // p - p_b
  float dH;   // H - H_b
  __device__ __forceinline__ void init(const PertRef<DIM>& R, const float* d) {
    const float rb = R.u[0];
    inv = rcp_fast((rb + d[0]) * rb);
    float num = 0.0f;  // rho_b (2 m_b.dm + dm.dm) - drho |m_b|^2, over rho rho_b = d|m|^2/rho
#pragma unroll
    for (int a = 0; a < DIM; ++a) num += d[1 + a] * (2.0f * R.u[1 + a] + d[1 + a]);
    const float dK = (rb * num - d[0] * R.mb2) * inv;
    dp = 0.4f * (d[M - 1] - 0.5f * dK);
    dH = d[M - 1] + dp;
  }
};

// dF = (F(ub + d) - F(ub)).n for direction n (any length); thb = m_b.n.
// Each component a(theta)/rho is differenced as
//   (rho_b (a_b dth + da (th_b + dth)) - drho a_b th_b) / (rho rho_b).
template <int DIM>
__device__ __forceinline__ void pert_flux(const PertRef<DIM>& R, const PertState<DIM>& S, const float* d,
                                          const float* n, float thb, float* dF) {
  constexpr int M = DIM + 2;
  const float rb = R.u[0];
  float dth = 0.0f;
#pragma unroll
  for (int a = 0; a < DIM; ++a) dth += d[1 + a] * n[a];
  const float th = thb + dth;
  dF[0] = dth;
#pragma unroll
  for (int a = 0; a < DIM; ++a)
    dF[1 + a] = (rb * (R.u[1 + a] * dth + d[1 + a] * th) - d[0] * R.u[1 + a] * thb) * S.inv + S.dp * n[a];
  dF[M - 1] = (rb * (R.Hb * dth + S.dH * th) - d[0] * R.Hb * thb) * S.inv;
}

// |u.n| + c of the state ub + d, for a unit normal n
template <int DIM>
__device__ __forceinline__ float pert_wave(const PertRef<DIM>& R, const PertState<DIM>& S, const float* d,
                                           const float* n, float thb) {
  float dth = 0.0f;
#pragma unroll
  for (int a = 0; a < DIM; ++a) dth += d[1 + a] * n[a];
  const float ir = R.u[0] * S.inv;  // 1 / rho
  const float p = R.pb + S.dp;
  return fabsf((thb + dth) * ir) + sqrt_fast(1.4f * p * ir);
}

// Local Lax-Friedrichs flux minus F(ub).n, both traces given as deviations
// from the same reference ub: G = (dF(dL) + dF(dR))/2 - lam (dR - dL)/2.
template <int DIM>
__device__ __forceinline__ void pert_lf(const PertRef<DIM>& R, const float* dL, const float* dR, const float* n,
                                        float thb, float* G) {
  constexpr int M = DIM + 2;
  PertState<DIM> SL, SR;
  SL.init(R, dL);
  SR.init(R, dR);
  float FL[M], FR[M];
  pert_flux<DIM>(R, SL, dL, n, thb, FL);
  pert_flux<DIM>(R, SR, dR, n, thb, FR);
  const float lam = fmaxf(pert_wave<DIM>(R, SL, dL, n, thb), pert_wave<DIM>(R, SR, dR, n, thb));
#pragma unroll
  for (int k = 0; k < M; ++k) G[k] = 0.5f * (FL[k] + FR[k]) - 0.5f * lam * (dR[k] - dL[k]);
}

}  // namespace dgc
