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

// Exchanged-side form of the local Lax-Friedrichs flux for a lane pair (one
// lane per element of an edge or face, each relative to its own element's
// reference).  Per-face constants: the partner's reference relative to ours
// dl = ub' - ub (exchanged), the normal, m_b.n, the references' flux difference
// fb = (F(ub') - F(ub)).n, and sg = +1/2 on side 0 (whose own trace is the left
// one), -1/2 on side 1.  All 32 lanes must call init.
template <int DIM>
struct FaceConst {
  static constexpr int M = DIM + 2;
  float dl[M], n[DIM], thb, fb[M], sg;
  __device__ __forceinline__ void init(const PertRef<DIM>& R, const float (&hi)[M], const float (&nn)[DIM],
                                       int side) {
#pragma unroll
    for (int m = 0; m < M; ++m) dl[m] = __shfl_xor_sync(0xffffffffu, hi[m], 1) - hi[m];
    thb = 0.0f;
#pragma unroll
    for (int a = 0; a < DIM; ++a) {
      n[a] = nn[a];
      thb += R.u[1 + a] * nn[a];
    }
    PertState<DIM> S;
    S.init(R, dl);
    pert_flux<DIM>(R, S, dl, n, thb, fb);
    sg = side ? -0.5f : 0.5f;
  }
};

// The flux minus F(ub).n at one point from the lane's own trace deviation
// t = u - ub and the partner's (relative to the partner's reference): each lane
// evaluates its own side and exchanges one value per variable,
//   A = dF/2 + sg lam t   (the partner's A' = dF'/2 - sg lam t'),
//   G = (dF + dF' + fb)/2 - sg lam (dl + t' - t) = A + A' + fb/2 - sg lam dl,
// lam the larger of the two wave speeds.  All 32 lanes must call it.
template <int DIM>
__device__ __forceinline__ void lf_exchange(const PertRef<DIM>& R, const FaceConst<DIM>& E,
                                            const float (&t)[DIM + 2], float (&G)[DIM + 2]) {
  constexpr int M = DIM + 2;
  PertState<DIM> S;
  S.init(R, t);
  float dF[M];
  pert_flux<DIM>(R, S, t, E.n, E.thb, dF);
  const float w = pert_wave<DIM>(R, S, t, E.n, E.thb);
  const float lam = fmaxf(w, __shfl_xor_sync(0xffffffffu, w, 1));
  const float sl = E.sg * lam;
#pragma unroll
  for (int m = 0; m < M; ++m) {
    const float a = fmaf(sl, t[m], 0.5f * dF[m]);
    G[m] = (a + __shfl_xor_sync(0xffffffffu, a, 1)) + fmaf(-sl, E.dl[m], 0.5f * E.fb[m]);
  }
}

}  // namespace dgc
