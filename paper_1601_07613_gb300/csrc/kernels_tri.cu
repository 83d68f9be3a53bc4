// Triangle kernels: volume integral, colored surface integral (Algorithm 1),
// the atomic / per-edge-buffer comparators and the FP64 CFL reduction.
//
// Eq. 2 with a basis orthonormal on the reference triangle (mass = detJ I):
//   dc_j/dt = sum_q w_q F(U_q).(J^-T grad phi_j)(x_q)
//           - sum_faces |f|/detJ sum_q w_q phi_j(x_q) F*(U-, U+, n).
// Each edge k is handled by a lane pair: the even lane owns the left element,
// the odd lane the right one.  A lane loads its element's modal block with
// 16-byte vector loads, evaluates its trace and the normal flux and wave speed
// of its own side at the edge points, exchanges them with its partner by
// shuffles, forms the Lax-Friedrichs flux, and projects it onto its own
// element.  Within one color no two edges share an element, so the lanes
// update rhs with plain loads and stores (Sec. 1, Algorithm 1): no atomics,
// no scratch buffer.
//
// FP64 kernels evaluate Eq. 2 as written.  FP32 kernels evaluate it in the
// perturbation form of euler_pert.cuh (deviations from the element mean).
#include <cooperative_groups.h>

#include <algorithm>
#include <cfloat>
#include <type_traits>

#include "dev_util.cuh"
#include "device.cuh"
#include "euler_pert.cuh"
#include "incr_form.cuh"

namespace dgc {

// Unrolling of the quadrature-point loops: fully unrolled p = 3 kernels run to
// several thousand instructions and stall on instruction fetch.
#ifndef DGC_QUNROLL
#define DGC_QUNROLL 1
#endif
#define DGC_PRAGMA_(x) _Pragma(#x)
#define DGC_PRAGMA(x) DGC_PRAGMA_(x)
#define DGC_UNROLL_Q DGC_PRAGMA(unroll DGC_QUNROLL)

template <int P>
struct TriDim {
  static constexpr int NP = (P + 1) * (P + 2) / 2;
  static constexpr int NQV = (P + 1) * (P + 1);
  static constexpr int NQE = 2 * P + 1;
  static constexpr int M = 4;
  static constexpr int NV = M * NP;
  // FP32 element record of the mixed-precision step: mean state as hi[M], lo[M],
  // then the modes j >= 1 as [M][NP-1]
  static constexpr int NF = M * (NP + 1);
};

template <typename T, int P>
struct TriTab {
  T phiV[TriDim<P>::NQV][TriDim<P>::NP];  // phi_j at volume points
  T vr[TriDim<P>::NQV][TriDim<P>::NP];    // w_q dphi_j/dr
  T vs[TriDim<P>::NQV][TriDim<P>::NP];    // w_q dphi_j/ds
  // phi_j at the points of local edge f = 0..2, then at those of half h of
  // local edge f as [3 + 2 f + h] (the coarse side of a hanging edge)
  T phiE[9][TriDim<P>::NQE][TriDim<P>::NP];
  T wE[TriDim<P>::NQE];                      // edge weights, sum 1
  T tE[TriDim<P>::NQE];                      // edge points' parameters in [0, 1] from the edge's first vertex
  T phiX[3][TriDim<P>::NP];                  // phi_j at the vertices (0,0), (1,0), (0,1)
};

__constant__ TriTab<double, 1> cTriD1;
__constant__ TriTab<double, 2> cTriD2;
__constant__ TriTab<double, 3> cTriD3;
__constant__ TriTab<float, 1> cTriF1;
__constant__ TriTab<float, 2> cTriF2;
__constant__ TriTab<float, 3> cTriF3;

template <typename T, int P>
__device__ __forceinline__ const TriTab<T, P>& tri_tab();
template <> __device__ __forceinline__ const TriTab<double, 1>& tri_tab<double, 1>() { return cTriD1; }
template <> __device__ __forceinline__ const TriTab<double, 2>& tri_tab<double, 2>() { return cTriD2; }
template <> __device__ __forceinline__ const TriTab<double, 3>& tri_tab<double, 3>() { return cTriD3; }
template <> __device__ __forceinline__ const TriTab<float, 1>& tri_tab<float, 1>() { return cTriF1; }
template <> __device__ __forceinline__ const TriTab<float, 2>& tri_tab<float, 2>() { return cTriF2; }
template <> __device__ __forceinline__ const TriTab<float, 3>& tri_tab<float, 3>() { return cTriF3; }

template <typename T, int P>
static void fill_tab(TriTab<T, P>& K, const RefTables& R) {
  using D = TriDim<P>;
  for (int q = 0; q < D::NQV; ++q)
    for (int j = 0; j < D::NP; ++j) {
      K.phiV[q][j] = (T)R.phiV[q * D::NP + j];
      K.vr[q][j] = (T)(R.vw[q] * R.dphiV[(0 * D::NQV + q) * D::NP + j]);
      K.vs[q][j] = (T)(R.vw[q] * R.dphiV[(1 * D::NQV + q) * D::NP + j]);
    }
  for (int f = 0; f < 3; ++f)
    for (int q = 0; q < D::NQE; ++q)
      for (int j = 0; j < D::NP; ++j) K.phiE[f][q][j] = (T)R.phiF[(f * D::NQE + q) * D::NP + j];
  for (int t = 0; t < 6; ++t)
    for (int q = 0; q < D::NQE; ++q)
      for (int j = 0; j < D::NP; ++j) K.phiE[3 + t][q][j] = (T)R.phiH[(t * D::NQE + q) * D::NP + j];
  for (int q = 0; q < D::NQE; ++q) K.wE[q] = (T)R.fw[q];
  for (int q = 0; q < D::NQE; ++q) K.tE[q] = (T)R.ft[q];
  for (int v = 0; v < 3; ++v)
    for (int j = 0; j < D::NP; ++j) K.phiX[v][j] = (T)R.phiX[v * D::NP + j];
}

template <int P>
static void upload_p(const RefTables& R, const void* symD, const void* symF) {
  static TriTab<double, P> hd;
  static TriTab<float, P> hf;
  fill_tab(hd, R);
  fill_tab(hf, R);
  cudaMemcpyToSymbol(symD, &hd, sizeof hd);
  cudaMemcpyToSymbol(symF, &hf, sizeof hf);
}

// The FP32 volume tables with every entry twice, (v, v): the operand of a packed
// two-lane FP32 FMA (__ffma2_rn, one instruction for two variables).
template <int P>
struct TriPairTab {
  float2 phiV[TriDim<P>::NQV][TriDim<P>::NP];
  float2 vr[TriDim<P>::NQV][TriDim<P>::NP];
  float2 vs[TriDim<P>::NQV][TriDim<P>::NP];
};
__constant__ TriPairTab<1> cTriP1;
__constant__ TriPairTab<2> cTriP2;
__constant__ TriPairTab<3> cTriP3;
template <int P>
__device__ __forceinline__ const TriPairTab<P>& tri_ptab();
template <> __device__ __forceinline__ const TriPairTab<1>& tri_ptab<1>() { return cTriP1; }
template <> __device__ __forceinline__ const TriPairTab<2>& tri_ptab<2>() { return cTriP2; }
template <> __device__ __forceinline__ const TriPairTab<3>& tri_ptab<3>() { return cTriP3; }

template <int P>
static void upload_pairs(const RefTables& R, const void* sym) {
  static TriPairTab<P> h;
  static TriTab<float, P> f;
  fill_tab(f, R);
  for (int q = 0; q < TriDim<P>::NQV; ++q)
    for (int j = 0; j < TriDim<P>::NP; ++j) {
      h.phiV[q][j] = make_float2(f.phiV[q][j], f.phiV[q][j]);
      h.vr[q][j] = make_float2(f.vr[q][j], f.vr[q][j]);
      h.vs[q][j] = make_float2(f.vs[q][j], f.vs[q][j]);
    }
  cudaMemcpyToSymbol(sym, &h, sizeof h);
}



// The FP64 lanes' tables as FP32 pairs (hi, lo) = (fl32(x), fl32(x - hi)): the
// volume tables as (hi, hi, lo, lo), the operand of a packed update of two
// variables (df_fma2), and the edge tables as (hi, lo) (staged into shared
// memory per block as (hi, hi, lo, lo)).
template <int P>
struct TriDfTab {
  float4 phiV[TriDim<P>::NQV][TriDim<P>::NP];
  float4 vr[TriDim<P>::NQV][TriDim<P>::NP];
  float4 vs[TriDim<P>::NQV][TriDim<P>::NP];
  float2 phiE[9][TriDim<P>::NQE][TriDim<P>::NP];
};
__constant__ TriDfTab<1> cTriDF1;
__constant__ TriDfTab<2> cTriDF2;
__constant__ TriDfTab<3> cTriDF3;
template <int P>
__device__ __forceinline__ const TriDfTab<P>& tri_dftab();
template <> __device__ __forceinline__ const TriDfTab<1>& tri_dftab<1>() { return cTriDF1; }
template <> __device__ __forceinline__ const TriDfTab<2>& tri_dftab<2>() { return cTriDF2; }
template <> __device__ __forceinline__ const TriDfTab<3>& tri_dftab<3>() { return cTriDF3; }

static float2 host_df(double x) {
  const float h = (float)x;
  return make_float2(h, (float)(x - (double)h));
}
static float4 host_df4(double x) {
  const float2 v = host_df(x);
  return make_float4(v.x, v.x, v.y, v.y);
}

template <int P>
static void upload_df(const RefTables& R, const void* sym) {
  static TriDfTab<P> h;
  static TriTab<double, P> d;
  fill_tab(d, R);
  for (int q = 0; q < TriDim<P>::NQV; ++q)
    for (int j = 0; j < TriDim<P>::NP; ++j) {
      h.phiV[q][j] = host_df4(d.phiV[q][j]);
      h.vr[q][j] = host_df4(d.vr[q][j]);
      h.vs[q][j] = host_df4(d.vs[q][j]);
    }
  for (int t = 0; t < 9; ++t)
    for (int q = 0; q < TriDim<P>::NQE; ++q)
      for (int j = 0; j < TriDim<P>::NP; ++j) h.phiE[t][q][j] = host_df(d.phiE[t][q][j]);
  cudaMemcpyToSymbol(sym, &h, sizeof h);
}

int tri_record_floats(int p) { return 4 * ((p + 1) * (p + 2) / 2 + 1); }

// ---------------------------------------------------------------------------
// element block loads / stores (M*Np contiguous values, 16-byte vectors)
// ---------------------------------------------------------------------------
template <int N>
__device__ __forceinline__ void load_block(const double* __restrict__ src, double (&v)[N]) {
  static_assert(N % 2 == 0, "even block");
  const double2* s = reinterpret_cast<const double2*>(src);
#pragma unroll
  for (int i = 0; i < N / 2; ++i) {
    double2 x = __ldg(s + i);
    v[2 * i] = x.x;
    v[2 * i + 1] = x.y;
  }
}
template <int N>
__device__ __forceinline__ void load_block(const float* __restrict__ src, float (&v)[N]) {
  static_assert(N % 4 == 0, "block of float4");
  const float4* s = reinterpret_cast<const float4*>(src);
#pragma unroll
  for (int i = 0; i < N / 4; ++i) {
    float4 x = __ldg(s + i);
    v[4 * i] = x.x;
    v[4 * i + 1] = x.y;
    v[4 * i + 2] = x.z;
    v[4 * i + 3] = x.w;
  }
}
// plain (coherent) loads, for blocks an earlier kernel of the stream wrote
template <int N>
__device__ __forceinline__ void load_plain(const double* src, double (&v)[N]) {
  const double2* s = reinterpret_cast<const double2*>(src);
#pragma unroll
  for (int i = 0; i < N / 2; ++i) {
    double2 x = s[i];
    v[2 * i] = x.x;
    v[2 * i + 1] = x.y;
  }
}
template <int N>
__device__ __forceinline__ void load_plain(const float* src, float (&v)[N]) {
  const float4* s = reinterpret_cast<const float4*>(src);
#pragma unroll
  for (int i = 0; i < N / 4; ++i) {
    float4 x = s[i];
    v[4 * i] = x.x;
    v[4 * i + 1] = x.y;
    v[4 * i + 2] = x.z;
    v[4 * i + 3] = x.w;
  }
}
template <int N>
__device__ __forceinline__ void store_block(double* dst, const double (&v)[N]) {
  double2* d = reinterpret_cast<double2*>(dst);
#pragma unroll
  for (int i = 0; i < N / 2; ++i) d[i] = make_double2(v[2 * i], v[2 * i + 1]);
}
template <int N>
__device__ __forceinline__ void store_block(float* dst, const float (&v)[N]) {
  float4* d = reinterpret_cast<float4*>(dst);
#pragma unroll
  for (int i = 0; i < N / 4; ++i) d[i] = make_float4(v[4 * i], v[4 * i + 1], v[4 * i + 2], v[4 * i + 3]);
}

// ---------------------------------------------------------------------------
// FP32 element state in perturbation form: mean hi + lo, deviation modes.
//
// The FP32 buffers of the triangle kernels are mode-major: the M = 4 values of
// mode j of an element form one float4.  Per element:
//   record (NF = 4 (NP + 1) floats): hi of the mean phi0 c0 [4], its lo [4],
//     then mode j = 1 .. NP-1 at 4 (j + 1);
//   Kahan pair state (8 NP floats): the record, then lo of mode j >= 1 at
//     NF + 4 (j - 1);
//   FP32 right-hand side and increment (4 NP floats): mode j at 4 j.
// FP64 blocks (state, FP64 right-hand side) stay [M][NP].
// ---------------------------------------------------------------------------
template <int P>
struct PertBlock {
  using D = TriDim<P>;
  float hi[4], lo[4];
  float cd[4][D::NP - 1];  // modes j >= 1
};

// split the FP64 mean state phi0 c0 into hi + lo (2 FP64 operations per value)
__device__ __forceinline__ void split_mean(double phi0, double c0, float& hi, float& lo) {
  const double u = phi0 * c0;
  hi = d2f(u);
  lo = d2f(u - f2d(hi));
}

template <int P>
__device__ __forceinline__ void load_pert(const double* __restrict__ src, PertBlock<P>& B) {
  using D = TriDim<P>;
  const double phi0 = tri_tab<double, P>().phiV[0][0];
  double v[D::NV];
  load_block(src, v);
#pragma unroll
  for (int m = 0; m < 4; ++m) {
    split_mean(phi0, v[m * D::NP], B.hi[m], B.lo[m]);
#pragma unroll
    for (int j = 1; j < D::NP; ++j) B.cd[m][j - 1] = d2f(v[m * D::NP + j]);
  }
}

template <int P>
__device__ __forceinline__ void load_pert(const float* __restrict__ src, PertBlock<P>& B) {
  using D = TriDim<P>;
  float v[D::NF];
  load_block(src, v);
#pragma unroll
  for (int m = 0; m < 4; ++m) {
    B.hi[m] = v[m];
    B.lo[m] = v[4 + m];
#pragma unroll
    for (int j = 1; j < D::NP; ++j) B.cd[m][j - 1] = v[4 * (j + 1) + m];
  }
}

// FP32 record of an FP64 block (the writers of the mixed-precision step)
template <int P>
__device__ __forceinline__ void record_of(const double (&v)[TriDim<P>::NV], float (&r)[TriDim<P>::NF]) {
  using D = TriDim<P>;
  const double phi0 = tri_tab<double, P>().phiV[0][0];
#pragma unroll
  for (int m = 0; m < 4; ++m) {
    split_mean(phi0, v[m * D::NP], r[m], r[4 + m]);
#pragma unroll
    for (int j = 1; j < D::NP; ++j) r[4 * (j + 1) + m] = d2f(v[m * D::NP + j]);
  }
}

// ---------------------------------------------------------------------------
// FP64 Euler fluxes (gamma = 1.4), Eq. 2 as written
// ---------------------------------------------------------------------------
__device__ __forceinline__ void euler_xy(const double* U, double* F, double* G) {
  const double ir = 1.0 / U[0];
  const double u = U[1] * ir, v = U[2] * ir;
  const double p = 0.4 * (U[3] - 0.5 * (U[1] * u + U[2] * v));
  F[0] = U[1];
  F[1] = U[1] * u + p;
  F[2] = U[2] * u;
  F[3] = (U[3] + p) * u;
  G[0] = U[2];
  G[1] = U[1] * v;
  G[2] = U[2] * v + p;
  G[3] = (U[3] + p) * v;
}

// One side's half of the local Lax-Friedrichs flux at an edge point: its
// normal flux F(U).n and wave speed |u.n| + c.  Each lane of an edge pair
// evaluates its own trace (one division and one square root) and exchanges
// the result with its partner.
__device__ __forceinline__ void lf_side(const double* U, double nx, double ny, double* Fn, double& w) {
  const double ir = 1.0 / U[0];
  const double u = U[1] * ir, v = U[2] * ir;
  const double p = 0.4 * (U[3] - 0.5 * (U[1] * u + U[2] * v));
  const double un = u * nx + v * ny;
  Fn[0] = U[0] * un;
  Fn[1] = U[1] * un + p * nx;
  Fn[2] = U[2] * un + p * ny;
  Fn[3] = (U[3] + p) * un;
  w = fabs(un) + sqrt(1.4 * p * ir);
}


// ---------------------------------------------------------------------------
// FP64 lanes: the basis contractions in FP32 pairs.  On this GPU the FP64 pipe
// runs at 1/64 of the FP32 rate, and the contractions (the traces
// sum_j phi_j c_j and the projections sum_q w_q phi_j F_q) took 60 % of the
// FP64 kernels' time (measured by leaving them out).  A value x is carried as
// a pair hi + lo, hi = fl32(x), lo = fl32(x - hi) (2^-48 of x), and s += t b
// runs on the FP32 pipe as the error-free product of the high parts (the FMA
// returns a product's rounding error exactly, Dekker's product) plus the two
// cross terms, added into s by Knuth's two-sum (TAOCP vol. 2, 4.2.2): 12 FP32
// operations in place of one FP64 FMA.  Fluxes, wave speeds, geometry and the
// stage update stay FP64.  The values projected are the deviations of the
// fluxes from the flux of the element's mean ub: F(u) - F(ub) in the volume,
// F* - F(ub).n on the faces.  For every element the two omitted parts cancel
// (the rules integrate grad phi_j and phi_j exactly, so sum_q w_q grad phi_j .
// F(ub) over the element equals the sum over its faces of sum_q w_q phi_j
// F(ub).n), so the pair arithmetic only carries deviations and its rounding
// stays below the FP64 rounding of the fluxes themselves.
// ---------------------------------------------------------------------------
#ifndef DGC_DF_MIN_P
#define DGC_DF_MIN_P 2
#endif
// doubles per entry of the FP64 lanes' shared-memory edge tables (pair lanes:
// one (hi, hi, lo, lo) float4)
constexpr int kFp64TabWords = 2;
// the FP64 lanes of order P use the pair contractions (at p = 1, with three
// modes, the splits and joins cost more than the FP64 contractions they replace)
template <int P>
__host__ __device__ constexpr bool df_lanes() {
  return P >= DGC_DF_MIN_P;
}

// An FP64 element block split for the pair contractions: the mean ub = phi_0 c_0
// (FP64) and the modes j >= 1 as pairs, two variables per float2 (k: the
// variables 2k and 2k + 1).
template <int P>
struct DfBlock {
  double ub[4];
  float2 ch[2][TriDim<P>::NP - 1], cl[2][TriDim<P>::NP - 1];
  __device__ __forceinline__ void init(const double (&c)[TriDim<P>::NV]) {
    constexpr int NP = TriDim<P>::NP;
    const double phi0 = tri_tab<double, P>().phiV[0][0];
#pragma unroll
    for (int m = 0; m < 4; ++m) ub[m] = phi0 * c[m * NP];
#pragma unroll
    for (int k = 0; k < 2; ++k)
#pragma unroll
      for (int j = 1; j < NP; ++j) {
        const DF a = df_split(c[2 * k * NP + j]), b = df_split(c[(2 * k + 1) * NP + j]);
        ch[k][j - 1] = make_float2(a.h, b.h);
        cl[k][j - 1] = make_float2(a.l, b.l);
      }
  }
};

// Pair accumulators of an element's modes, two variables per float2.
template <int P>
struct DfAcc {
  float2 h[2][TriDim<P>::NP], l[2][TriDim<P>::NP];
  __device__ __forceinline__ void zero() {
#pragma unroll
    for (int k = 0; k < 2; ++k)
#pragma unroll
      for (int j = 0; j < TriDim<P>::NP; ++j) h[k][j] = l[k][j] = make_float2(0.0f, 0.0f);
  }
  // the value of variable m, mode j, in FP64
  __device__ __forceinline__ double get(int m, int j) const {
    const float2 a = h[m >> 1][j], b = l[m >> 1][j];
    return (m & 1) ? df_join(DF{a.y, b.y}) : df_join(DF{a.x, b.x});
  }
};

// split two FP64 values into a (hi pair, lo pair)
__device__ __forceinline__ void df_split2(double x0, double x1, float2& h, float2& l) {
  const DF a = df_split(x0), b = df_split(x1);
  h = make_float2(a.h, b.h);
  l = make_float2(a.l, b.l);
}

// Volume integral sum_q w_q (F(U_q) - F(ub)).(J^-T grad phi_j), j >= 1 (grad
// phi_0 = 0), into the pair accumulators; Fb, Gb = the x and y fluxes of ub.
template <int P>
__device__ __forceinline__ void volume_df(const DfBlock<P>& B, const double (&Fb)[4], const double (&Gb)[4],
                                          const double* __restrict__ ji, DfAcc<P>& acc) {
  using D = TriDim<P>;
  constexpr int NP = D::NP;
  const TriDfTab<P>& T = tri_dftab<P>();
  const double2 j0 = __ldg(reinterpret_cast<const double2*>(ji));
  const double2 j1 = __ldg(reinterpret_cast<const double2*>(ji) + 1);
  DGC_UNROLL_Q
  for (int q = 0; q < D::NQV; ++q) {
    double U[4];
#pragma unroll
    for (int k = 0; k < 2; ++k) {
      float2 dh = make_float2(0.0f, 0.0f), dl = dh;
#pragma unroll
      for (int j = 1; j < NP; ++j) df_fma2(dh, dl, T.phiV[q][j], B.ch[k][j - 1], B.cl[k][j - 1]);
      U[2 * k] = B.ub[2 * k] + df_join(DF{dh.x, dl.x});
      U[2 * k + 1] = B.ub[2 * k + 1] + df_join(DF{dh.y, dl.y});
    }
    double F[4], G[4];
    euler_xy(U, F, G);
#pragma unroll
    for (int k = 0; k < 2; ++k) {
      const double dF0 = F[2 * k] - Fb[2 * k], dG0 = G[2 * k] - Gb[2 * k];
      const double dF1 = F[2 * k + 1] - Fb[2 * k + 1], dG1 = G[2 * k + 1] - Gb[2 * k + 1];
      float2 frh, frl, fsh, fsl;
      df_split2(j0.x * dF0 + j0.y * dG0, j0.x * dF1 + j0.y * dG1, frh, frl);
      df_split2(j1.x * dF0 + j1.y * dG0, j1.x * dF1 + j1.y * dG1, fsh, fsl);
#pragma unroll
      for (int j = 1; j < NP; ++j) {
        df_fma2(acc.h[k][j], acc.l[k][j], T.vr[q][j], frh, frl);
        df_fma2(acc.h[k][j], acc.l[k][j], T.vs[q][j], fsh, fsl);
      }
    }
  }
}

// The volume integral of an FP64 block, added into acc (the unfused kernel).
template <int P>
__device__ __forceinline__ void volume_acc64(const double (&c)[TriDim<P>::NV], const double* __restrict__ ji,
                                             double (&acc)[TriDim<P>::NV]) {
  constexpr int NP = TriDim<P>::NP;
  if constexpr (!df_lanes<P>()) {  // Eq. 2 as written, FP64 throughout
    using D = TriDim<P>;
    const TriTab<double, P>& K = tri_tab<double, P>();
    const double2 j0 = __ldg(reinterpret_cast<const double2*>(ji));
    const double2 j1 = __ldg(reinterpret_cast<const double2*>(ji) + 1);
    DGC_UNROLL_Q
    for (int q = 0; q < D::NQV; ++q) {
      double U[4];
#pragma unroll
      for (int m = 0; m < 4; ++m) {
        double s = 0.0;
#pragma unroll
        for (int j = 0; j < NP; ++j) s += K.phiV[q][j] * c[m * NP + j];
        U[m] = s;
      }
      double F[4], G[4];
      euler_xy(U, F, G);
#pragma unroll
      for (int m = 0; m < 4; ++m) {
        const double fr = j0.x * F[m] + j0.y * G[m];
        const double fs = j1.x * F[m] + j1.y * G[m];
#pragma unroll
        for (int j = 0; j < NP; ++j) acc[m * NP + j] += K.vr[q][j] * fr + K.vs[q][j] * fs;
      }
    }
    return;
  }
  DfBlock<P> B;
  B.init(c);
  double Fb[4], Gb[4];
  euler_xy(B.ub, Fb, Gb);
  DfAcc<P> a;
  a.zero();
  volume_df<P>(B, Fb, Gb, ji, a);
#pragma unroll
  for (int m = 0; m < 4; ++m)
#pragma unroll
    for (int j = 1; j < NP; ++j) acc[m * NP + j] += a.get(m, j);
}

// FP32 volume integral in perturbation form: sum_q w_q dF(U_q).(J^-T grad phi_j),
// the constant F(ub) left out (it cancels against the faces); grad phi_0 = 0.
// With DGC_FFMA2 the evaluation and the projection run on two variables at a
// time through the packed FP32 FMA (__ffma2_rn): the same roundings per value.
#ifndef DGC_FFMA2
#define DGC_FFMA2 1
#endif
// LAM: also max_q (|u| + c) of the state at the volume points (the CFL estimate
// of lambda_max_rec, from the same sums), into *lam.  S lanes share an element
// (S = 2: two lanes per edge side): lane sub takes the points sub, sub + S, ...
template <int P, bool LAM = false, int S = 1>
__device__ __forceinline__ void volume_acc32(const PertBlock<P>& B, const PertRef<2>& R,
                                             const double* __restrict__ ji, float (&acc)[TriDim<P>::NV],
                                             float* lam = nullptr, int sub = 0) {
  using D = TriDim<P>;
  constexpr int NP = D::NP;
  const TriTab<float, P>& K = tri_tab<float, P>();
  const double2 j0 = __ldg(reinterpret_cast<const double2*>(ji));
  const double2 j1 = __ldg(reinterpret_cast<const double2*>(ji) + 1);
  const float nr[2] = {d2f(j0.x), d2f(j0.y)}, ns[2] = {d2f(j1.x), d2f(j1.y)};
  const float thr = R.u[1] * nr[0] + R.u[2] * nr[1], ths = R.u[1] * ns[0] + R.u[2] * ns[1];
#if DGC_FFMA2
  // variables in pairs (0, 1), (2, 3): one packed FMA per mode and pair
  const TriPairTab<P>& K2 = tri_ptab<P>();
  float2 c01[NP - 1], c23[NP - 1], a01[NP - 1], a23[NP - 1];
#pragma unroll
  for (int j = 1; j < NP; ++j) {
    c01[j - 1] = make_float2(B.cd[0][j - 1], B.cd[1][j - 1]);
    c23[j - 1] = make_float2(B.cd[2][j - 1], B.cd[3][j - 1]);
    a01[j - 1] = make_float2(acc[j], acc[NP + j]);
    a23[j - 1] = make_float2(acc[2 * NP + j], acc[3 * NP + j]);
  }
  DGC_UNROLL_Q
  for (int q = S == 1 ? 0 : sub; q < D::NQV; q += S) {
    float2 d01 = make_float2(B.lo[0], B.lo[1]), d23 = make_float2(B.lo[2], B.lo[3]);
#pragma unroll
    for (int j = 1; j < NP; ++j) {
      d01 = __ffma2_rn(K2.phiV[q][j], c01[j - 1], d01);
      d23 = __ffma2_rn(K2.phiV[q][j], c23[j - 1], d23);
    }
    const float d[4] = {d01.x, d01.y, d23.x, d23.y};
    if constexpr (LAM) {
      const float U0 = R.u[0] + d[0], U1 = R.u[1] + d[1], U2 = R.u[2] + d[2], U3 = R.u[3] + d[3];
      const float ir = rcp_fast(U0), u = U1 * ir, w = U2 * ir;
      const float q2 = u * u + w * w;
      const float pr = 0.4f * (U3 - 0.5f * U0 * q2);
      *lam = fmaxf(*lam, sqrt_fast(q2) + sqrt_fast(1.4f * pr * ir));
    }
    PertState<2> PS;
    PS.init(R, d);
    float Fr[4], Fs[4];
    pert_flux<2>(R, PS, d, nr, thr, Fr);
    pert_flux<2>(R, PS, d, ns, ths, Fs);
    const float2 r01 = make_float2(Fr[0], Fr[1]), r23 = make_float2(Fr[2], Fr[3]);
    const float2 s01 = make_float2(Fs[0], Fs[1]), s23 = make_float2(Fs[2], Fs[3]);
#pragma unroll
    for (int j = 1; j < NP; ++j) {
      a01[j - 1] = __ffma2_rn(K2.vs[q][j], s01, __ffma2_rn(K2.vr[q][j], r01, a01[j - 1]));
      a23[j - 1] = __ffma2_rn(K2.vs[q][j], s23, __ffma2_rn(K2.vr[q][j], r23, a23[j - 1]));
    }
  }
#pragma unroll
  for (int j = 1; j < NP; ++j) {
    acc[j] = a01[j - 1].x;
    acc[NP + j] = a01[j - 1].y;
    acc[2 * NP + j] = a23[j - 1].x;
    acc[3 * NP + j] = a23[j - 1].y;
  }
#else
  DGC_UNROLL_Q
  for (int q = S == 1 ? 0 : sub; q < D::NQV; q += S) {
    float d[4];
#pragma unroll
    for (int m = 0; m < 4; ++m) {
      float s = B.lo[m];
#pragma unroll
      for (int j = 1; j < NP; ++j) s += K.phiV[q][j] * B.cd[m][j - 1];
      d[m] = s;
    }
    PertState<2> PS;
    PS.init(R, d);
    float Fr[4], Fs[4];
    pert_flux<2>(R, PS, d, nr, thr, Fr);
    pert_flux<2>(R, PS, d, ns, ths, Fs);
#pragma unroll
    for (int m = 0; m < 4; ++m)
#pragma unroll
      for (int j = 1; j < NP; ++j) acc[m * NP + j] += K.vr[q][j] * Fr[m] + K.vs[q][j] * Fs[m];
  }
#endif
}

// An element's right-hand side from a [M][NP] register block: mode-major when
// FP32, [M][NP] when FP64.
template <int P, typename RT, typename AT>
__device__ __forceinline__ void store_rhs(RT* dst, const AT (&acc)[TriDim<P>::NV]) {
  constexpr int NP = TriDim<P>::NP, NV = TriDim<P>::NV;
  RT out[NV];
#pragma unroll
  for (int m = 0; m < 4; ++m)
#pragma unroll
    for (int j = 0; j < NP; ++j) out[sizeof(RT) == 4 ? 4 * j + m : m * NP + j] = (RT)acc[m * NP + j];
  store_block(dst, out);
}

// ---------------------------------------------------------------------------
// Volume kernel (unfused path): one thread per element, rhs = volume integral.
// ---------------------------------------------------------------------------
template <int P, typename CT, typename ST, typename RT>
__device__ __forceinline__ void vol_elem(const ST* __restrict__ c, int sstride, const double* __restrict__ jinv,
                                         RT* __restrict__ rhs, int64_t e) {
  using D = TriDim<P>;
  RT out[D::NV];
  if constexpr (sizeof(CT) == 8) {
    double v[D::NV], acc[D::NV];
    load_block(c + e * D::NV, v);
#pragma unroll
    for (int i = 0; i < D::NV; ++i) acc[i] = 0.0;
    volume_acc64<P>(v, jinv + 4 * e, acc);
#pragma unroll
    for (int i = 0; i < D::NV; ++i) out[i] = (RT)acc[i];
  } else {
    const int64_t stride = sizeof(ST) == 8 ? D::NV : sstride;
    PertBlock<P> B;
    load_pert<P>(c + e * stride, B);
    PertRef<2> R;
    R.init(B.hi);
    float acc[D::NV];
#pragma unroll
    for (int i = 0; i < D::NV; ++i) acc[i] = 0.0f;
    volume_acc32<P>(B, R, jinv + 4 * e, acc);
    store_rhs<P>(rhs + e * D::NV, acc);
    return;
  }
  store_block(rhs + e * D::NV, out);
}

template <int P, typename CT, typename ST, typename RT>
__global__ void __launch_bounds__(128) k_vol_tri(const ST* __restrict__ c, int sstride, const double* __restrict__ jinv,
                                                 RT* __restrict__ rhs, int64_t e0, int64_t ne) {
  const int64_t e = e0 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= ne) return;
  vol_elem<P, CT, ST, RT>(c, sstride, jinv, rhs, e);
}

// ---------------------------------------------------------------------------
// Surface kernel for one color (or all edges for the comparators).
// ---------------------------------------------------------------------------
struct SurfParams {
  int64_t begin, end;
  const int4* __restrict__ topo;
  const double2* __restrict__ fgeo;
  const double* __restrict__ jinv;
  const void* state;
  void* rhs;
  void* buf;
  StageArgs sa;
  int ntab;     // edge tables to stage (3, or 9 on meshes with hanging edges)
  int sstride;  // floats per element of an FP32 state (record or Kahan state)
  int persistent = 0;  // grid-stride over the color with at most one wave of blocks
  // first color of stage 0 of the mixed step (tri_first_est): the record of u0
  // it writes, the elements' FP32 CFL estimates, their minimum, the inradii
  float* rec_first = nullptr;
  float* est = nullptr;
  unsigned* estmin = nullptr;
  const double* inr = nullptr;
  // boundary conditions (FP64 lanes; null: every boundary transmissive): the
  // mesh's boundary block (kBc*), per boundary face its first vertex and edge
  // vector, and the time t0 + tfrac * dt (dt on the device, or none) the
  // boundary states are taken at
  const double* bc = nullptr;
  const BndGeo* bgeo = nullptr;
  const double* t0 = nullptr;
  const double* dtp = nullptr;
  double tfrac = 0.0;
};

// The state outside a boundary face at its edge point q, taken by the second
// lane of the face's pair in place of its own trace (dgc_set_boundary; tp.w =
// kind | state << 4 | boundary face << 8): a slip wall reverses the normal
// momentum, a state face takes its prescribed state, a shock face the state
// behind the moving shock where x < a + b y + c t, else the state ahead;
// transmissive faces keep U (U+ = U-).
__device__ __forceinline__ void bc_outside(const SurfParams& A, int w, double tq, double nx, double ny, double* U) {
  const int kind = w & 15;
  if (kind == DGC_BC_WALL) {
    const double mn = U[1] * nx + U[2] * ny;
    U[1] -= 2.0 * mn * nx;
    U[2] -= 2.0 * mn * ny;
  } else if (kind == DGC_BC_STATE || kind == DGC_BC_SHOCK) {
    int s = (w >> 4) & 15;
    if (kind == DGC_BC_SHOCK) {
      const BndGeo g = A.bgeo[w >> 8];
      const double x = g.x0 + tq * g.dx, y = g.y0 + tq * g.dy;
      const double t = *A.t0 + (A.dtp ? A.tfrac * *A.dtp : 0.0);
      const double* sh = A.bc + kBcShock;
      s = x < sh[0] + sh[1] * y + sh[2] * t ? (int)sh[3] : (int)sh[4];
    }
    const double* S = A.bc + kBcStates + 4 * s;
#pragma unroll
    for (int m = 0; m < 4; ++m) U[m] = S[m];
  }
}

// The same for the FP32 lanes, on the edge coefficients ak of the trace's
// deviation t(xi) = sum_k L_k(xi) ak[k] (L_0 = 1) from the element's reference
// ub, before the point loop: the outside state relative to the same reference
// is affine in t for a wall (the momentum of ub + t reflected) and constant for
// a prescribed state (S - ub), so both map the coefficients.  A shock face's
// state is piecewise constant along the edge and replaces the trace whole: the
// function returns true, and the coefficient registers, no longer needed, carry
// the line f(tq) = al + be tq (negative where the point lies behind the shock)
// as the bits of two doubles in ak[0] (no register held across the point loop
// for it); bc_shock32 then sets each point's deviation.
template <int K1>
__device__ __forceinline__ bool bc_modal32(const SurfParams& A, int w, float nx, float ny, const float* ub,
                                           float (&ak)[K1][4]) {
  const int kind = w & 15;
  if (kind == DGC_BC_WALL) {
#pragma unroll
    for (int kk = 0; kk < K1; ++kk) {
      const float mn = kk == 0 ? (ub[1] + ak[0][1]) * nx + (ub[2] + ak[0][2]) * ny : ak[kk][1] * nx + ak[kk][2] * ny;
      ak[kk][1] -= 2.0f * mn * nx;
      ak[kk][2] -= 2.0f * mn * ny;
    }
  } else if (kind == DGC_BC_STATE) {
    const double* S = A.bc + kBcStates + 4 * ((w >> 4) & 15);
#pragma unroll
    for (int m = 0; m < 4; ++m) {
      ak[0][m] = d2f(S[m] - (double)ub[m]);
#pragma unroll
      for (int kk = 1; kk < K1; ++kk) ak[kk][m] = 0.0f;
    }
  } else if (kind == DGC_BC_SHOCK) {
    const BndGeo g = A.bgeo[w >> 8];
    const double t = *A.t0 + (A.dtp ? A.tfrac * *A.dtp : 0.0);
    const double* sh = A.bc + kBcShock;
    const double al = g.x0 - sh[0] - sh[1] * g.y0 - sh[2] * t, be = g.dx - sh[1] * g.dy;
    ak[0][0] = __int_as_float(__double2hiint(al)), ak[0][1] = __int_as_float(__double2loint(al));
    ak[0][2] = __int_as_float(__double2hiint(be)), ak[0][3] = __int_as_float(__double2loint(be));
    return true;
  }
  return false;
}

// a shock face's deviation at the edge point tq: the state behind the shock
// where al + be tq < 0, else the state ahead, minus the reference (a0: the
// line's bits, as bc_modal32 left them)
__device__ __forceinline__ void bc_shock32(const SurfParams& A, const float (&a0)[4], double tq, const float* ub,
                                           float* t) {
  const double al = __hiloint2double(__float_as_int(a0[0]), __float_as_int(a0[1]));
  const double be = __hiloint2double(__float_as_int(a0[2]), __float_as_int(a0[3]));
  const double* sh = A.bc + kBcShock;
  const double* S = A.bc + kBcStates + 4 * (int)(fma(be, tq, al) < 0.0 ? sh[3] : sh[4]);
#pragma unroll
  for (int m = 0; m < 4; ++m) t[m] = d2f(S[m] - (double)ub[m]);
}

// the contribution of one lane's element is in acc; write it as the mode asks
template <int P, typename RT, int MODE, typename AT>
__device__ __forceinline__ void surf_write(const SurfParams& A, int64_t elem, int64_t k, int side,
                                           const AT (&acc)[TriDim<P>::NV]) {
  using D = TriDim<P>;
  constexpr int NV = D::NV;
  if constexpr (MODE == SURF_RMW) {
    RT* r = static_cast<RT*>(A.rhs) + elem * NV;
    RT old[NV];
    load_plain(r, old);
#pragma unroll
    for (int i = 0; i < NV; ++i) old[i] += (RT)acc[i];
    store_block(r, old);
  } else if constexpr (MODE == SURF_FIRST) {
    RT out[NV];
#pragma unroll
    for (int i = 0; i < NV; ++i) out[i] = (RT)acc[i];
    store_block(static_cast<RT*>(A.rhs) + elem * NV, out);
  } else if constexpr (MODE == SURF_ATOMIC) {
    RT* r = static_cast<RT*>(A.rhs) + elem * NV;
#pragma unroll
    for (int i = 0; i < NV; ++i) atomicAdd(r + i, (RT)acc[i]);
  } else if constexpr (MODE == SURF_BUFFER) {
    RT out[NV];
#pragma unroll
    for (int i = 0; i < NV; ++i) out[i] = (RT)acc[i];
    store_block(static_cast<RT*>(A.buf) + (2 * k + side) * NV, out);
  }
}

// Last color, FP64 form: L = partial rhs + this color, uout = a0 u0 + b0 us +
// (b0 dt) L (1 FMA per value in the first stage, 1 MUL + 2 FMA in the
// others).  us is the state block the fluxes used (in registers).  In chunks
// of CH value pairs, every chunk's loads before its stores (uout may alias us
// and u0, so the compiler keeps later loads behind earlier stores).
template <int P>
__device__ __forceinline__ void fp64_last(const SurfParams& A, int64_t elem, const double (&acc)[TriDim<P>::NV],
                                          const double (&us)[TriDim<P>::NV]) {
  constexpr int NV = TriDim<P>::NV, H = NV / 2, CH = 5;
  const double2* part = reinterpret_cast<const double2*>(static_cast<const double*>(A.rhs) + elem * NV);
  const double2* u02 = reinterpret_cast<const double2*>(A.sa.u0 + elem * NV);
  double2* out2 = reinterpret_cast<double2*>(A.sa.uout + elem * NV);
  const double dt = *A.sa.dt, a0 = A.sa.a0, b0 = A.sa.b0, bdt = b0 * dt;
#pragma unroll
  for (int c0 = 0; c0 < H; c0 += CH) {
    double2 pr[CH], u[CH];
#pragma unroll
    for (int i = 0; i < CH; ++i)
      if (c0 + i < H) {
        pr[i] = part[c0 + i];
        if (a0 != 0.0) u[i] = u02[c0 + i];
      }
#pragma unroll
    for (int i = 0; i < CH; ++i)
      if (c0 + i < H) {
        const int v = 2 * (c0 + i);
        const double L0 = pr[i].x + acc[v], L1 = pr[i].y + acc[v + 1];
        double w0, w1;
        if (a0 == 0.0) {
          w0 = fma(bdt, L0, b0 == 1.0 ? us[v] : b0 * us[v]);
          w1 = fma(bdt, L1, b0 == 1.0 ? us[v + 1] : b0 * us[v + 1]);
        } else {
          w0 = fma(bdt, L0, fma(a0, u[i].x, b0 * us[v]));
          w1 = fma(bdt, L1, fma(a0, u[i].y, b0 * us[v + 1]));
        }
        out2[c0 + i] = make_double2(w0, w1);
      }
  }
}

// the first ntab edge tables of order P into shared memory (the block's
// threads cooperate): 3 on conforming meshes, 9 with hanging edges
template <int P, typename CT>
__device__ __forceinline__ void stage_edge_tables(CT* sphi, CT* sw, int ntab = 3) {
  using D = TriDim<P>;
  const TriTab<CT, P>& K = tri_tab<CT, P>();
  if constexpr (sizeof(CT) == 8 && df_lanes<P>()) {
    // the FP64 lanes read the edge tables as FP32 pairs (hi, hi, lo, lo): 16 bytes
    // per entry, so their buffers hold two doubles per entry (kFp64TabWords)
    const float2* src = &tri_dftab<P>().phiE[0][0][0];
    float4* dst = reinterpret_cast<float4*>(sphi);
    for (int i = threadIdx.x; i < ntab * D::NQE * D::NP; i += blockDim.x) {
      const float2 v = src[i];
      dst[i] = make_float4(v.x, v.x, v.y, v.y);
    }
  } else {
    const CT* src = &K.phiE[0][0][0];
    for (int i = threadIdx.x; i < ntab * D::NQE * D::NP; i += blockDim.x) sphi[i] = src[i];
  }
  if (threadIdx.x < D::NQE) sw[threadIdx.x] = K.wE[threadIdx.x];
}

// ---------------------------------------------------------------------------
// FP32 surface integral of one lane (perturbation form, euler_pert.cuh).
//
// On an edge, phi_j is a polynomial of degree <= P in the edge parameter xi,
// so phi_j(x(xi)) = sum_k T_jk L_k(xi) exactly (Legendre polynomials L_k,
// k <= P; T_jk by Gauss quadrature, a table per local edge, half edge and
// direction).  The lane then works with P+1 edge coefficients instead of the
// NP modes at the 2P+1 points:
//  1. a_k = lo dk0 + sum_{j>=1} T_jk c_j (one mode of the record at a time),
//     and the trace deviations t_q = u(x_q) - ub = sum_k L_k(xi_q) a_k;
//  2. at each point the lane's own flux difference dF = (F(u) - F(ub)).n and
//     wave speed, exchanged with the partner lane, which evaluated its side
//     relative to its own reference ub'; the local Lax-Friedrichs flux minus
//     F(ub).n is then
//        G = (dF + dF' + (F(ub') - F(ub)).n) / 2 - lam (u_R - u_L) / 2,
//     with the bracket evaluated once per edge in perturbation form (deviation
//     ub' - ub), so every term stays proportional to a deviation;
//  3. b_k = sum_q w_q G_q L_k(xi_q), and sum_q w_q G_q phi_j(x_q) =
//     sum_k T_jk b_k for one mode j at a time (four values), handed to the
//     epilogue of the mode as soon as it is complete.
// The point loops use L_k(xi_q), the same for every lane (constant memory);
// the per-lane tables T are read from shared memory, one float4 per mode.
// ---------------------------------------------------------------------------

// Edge tables of the FP32 kernels.  Tk[d][le][j][k]: T_jk of table le (3 local
// edges, then the 6 half edges of a hanging edge's coarse side) with the points
// in the left element's order (d = 0) or reversed, as the right element meets
// them (d = 1; T_jk (-1)^k); k padded to 4.  Lq[q][k] = L_k(xi_q).
template <int P>
struct TriEdgeK {
  float Tk[2][9][TriDim<P>::NP][4];
  float Lq[TriDim<P>::NQE][4];
};
__constant__ TriEdgeK<1> cTriK1;
__constant__ TriEdgeK<2> cTriK2;
__constant__ TriEdgeK<3> cTriK3;
template <int P>
__device__ __forceinline__ const TriEdgeK<P>& tri_ek();
template <> __device__ __forceinline__ const TriEdgeK<1>& tri_ek<1>() { return cTriK1; }
template <> __device__ __forceinline__ const TriEdgeK<2>& tri_ek<2>() { return cTriK2; }
template <> __device__ __forceinline__ const TriEdgeK<3>& tri_ek<3>() { return cTriK3; }

// T by Gauss-Legendre quadrature on the table's own point values (exact: the
// integrand phi_j L_k has degree <= 2P, the rule 2P+1 points).
template <int P>
static void fill_edge_k(TriEdgeK<P>& E, const RefTables& R) {
  using D = TriDim<P>;
  constexpr int NQ = D::NQE, NP = D::NP;
  double x[NQ], w[NQ], L[NQ][4];
  gauss_jacobi(NQ, 0.0, x, w);
  for (int q = 0; q < NQ; ++q) {
    L[q][0] = 1.0;
    L[q][1] = x[q];
    for (int k = 2; k < 4; ++k) L[q][k] = ((2 * k - 1) * x[q] * L[q][k - 1] - (k - 1) * L[q][k - 2]) / k;
    for (int k = 0; k < 4; ++k) E.Lq[q][k] = k <= P ? (float)L[q][k] : 0.0f;
  }
  for (int d = 0; d < 2; ++d)
    for (int le = 0; le < 9; ++le)
      for (int j = 0; j < NP; ++j)
        for (int k = 0; k < 4; ++k) {
          double s = 0.0;
          if (k <= P)
            for (int q = 0; q < NQ; ++q) {
              const int qq = d ? NQ - 1 - q : q;
              const double v = le < 3 ? R.phiF[((size_t)le * NQ + qq) * NP + j]
                                      : R.phiH[((size_t)(le - 3) * NQ + qq) * NP + j];
              s += w[q] * v * L[q][k];
            }
          E.Tk[d][le][j][k] = (float)(0.5 * (2 * k + 1) * s);
        }
}

template <int P>
static void upload_ek(const RefTables& R, const void* sym) {
  static TriEdgeK<P> h;
  fill_edge_k(h, R);
  cudaMemcpyToSymbol(sym, &h, sizeof h);
}

// Shared-memory copy of Tk for the tables a mesh uses: block (d, le) of NP
// float4 rows, the block stride an odd number of float4 so that lanes reading
// different blocks fall into different banks.
template <int P>
struct ETab32 {
  static constexpr int NQ = TriDim<P>::NQE, NP = TriDim<P>::NP;
  static constexpr int BLK = 4 * (NP | 1);
  static constexpr int SIZE = 2 * 9 * BLK;
};

template <int P>
__device__ __forceinline__ void stage_etab32(float* s, int ntab) {
  using T = ETab32<P>;
  const TriEdgeK<P>& E = tri_ek<P>();
  for (int i = threadIdx.x; i < 2 * ntab * T::BLK; i += blockDim.x) {
    const int b = i / T::BLK, r = i - b * T::BLK;
    const int d = b / ntab, le = b - d * ntab;
    s[i] = r < 4 * T::NP ? E.Tk[d][le][r / 4][r % 4] : 0.0f;
  }
}

// Shared-memory float4 accesses kept where they are written (the compiler
// would otherwise hoist the table reads of all modes and hold them in
// registers).
__device__ __forceinline__ void sts4(float* p, float4 v) {
  const unsigned a = (unsigned)__cvta_generic_to_shared(p);
  asm volatile("st.shared.v4.f32 [%0], {%1, %2, %3, %4};" ::"r"(a), "f"(v.x), "f"(v.y), "f"(v.z), "f"(v.w) : "memory");
}
__device__ __forceinline__ float4 lds4(const float4* p) {
  float4 v;
  const unsigned a = (unsigned)__cvta_generic_to_shared(p);
  asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];" : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w) : "r"(a));
  return v;
}

// floats per lane of a shared-memory record slot: the record, as an odd number
// of float4 so that the slots of eight consecutive lanes fall into distinct banks
template <int P>
__host__ __device__ constexpr int rec_slot() {
  return 4 * ((TriDim<P>::NF / 4) | 1);
}

__device__ __forceinline__ float4 f4_add(float4 a, const float (&b)[4]) {
  return make_float4(a.x + b[0], a.y + b[1], a.z + b[2], a.w + b[3]);
}
__device__ __forceinline__ float4 f4_mul_f2(float4 a, F2 c) {
  return make_float4(mul_f2(a.x, c), mul_f2(a.y, c), mul_f2(a.z, c), mul_f2(a.w, c));
}

// sum_k T_jk b_k for the four variables (row = T_j., P+1 coefficients)
template <int P>
__device__ __forceinline__ void mode_sum(const float4 row, const float (&b)[P + 1][4], float (&a)[4]) {
  const float t[4] = {row.x, row.y, row.z, row.w};
#pragma unroll
  for (int m = 0; m < 4; ++m) {
    float s = t[0] * b[0][m];
#pragma unroll
    for (int k = 1; k <= P; ++k) s = fmaf(t[k], b[k][m], s);
    a[m] = s;
  }
}

// Modes per batch of the last-color epilogue, per stage (stage 2 of the mixed
// form needs an even batch: it pairs modes into double2)
#ifndef DGC_JB0
#define DGC_JB0 6
#endif
#ifndef DGC_JB1
#define DGC_JB1 4
#endif
#ifndef DGC_JB2
#define DGC_JB2 4
#endif

// Loop 3 with the last-color epilogue in increment form (incr_form.cuh) for
// STG = the stage (0, 1, 2), or 3 for stage 2 of the Kahan form: L_j = partial
// rhs + this color, then the stage of the increment and of the record (stages
// 0, 1), the FP64 state of the mixed form, in place, u = u0 + (2/3) delta
// (STG 2), or the Kahan pair state (STG 3).  The modes go in batches of JB
// whose loads are all issued before the batch's stores, so that a batch costs
// one memory round trip.  The buffers are distinct arrays.  The lane takes the
// jcnt modes from jbase (all of them with one lane per side; with two lanes per
// side each takes its share, split at an even mode when stage 2 pairs modes).
template <int P, int STG>
__device__ __forceinline__ void last_modes(const float4* tb, const float (&b)[P + 1][4], const float4* rs,
                                           const float4* __restrict__ part, float4* __restrict__ dp,
                                           const float4* __restrict__ r0, float4* __restrict__ ro,
                                           float4* __restrict__ ks, double* __restrict__ u, double dt,
                                           double phi0, int jbase = 0, int jcnt = TriDim<P>::NP) {
  static_assert(STG >= 0 && STG <= 3, "stage");
  constexpr int NP = TriDim<P>::NP, NF4 = NP + 1;
  // modes per batch: stage 2 of an FP64 state pairs modes (j, j+1) into double2
  constexpr int JB = STG == 0 ? DGC_JB0 : STG == 1 ? DGC_JB1 : DGC_JB2;
  constexpr bool PAIRS = NP % 2 == 0, kahan = STG == 3;
  static_assert(STG != 2 || !PAIRS || JB % 2 == 0, "stage 2 pairs modes: even batches");
  const F2 dtp = split_f2(dt);
  float dk[PAIRS ? 1 : NP][4];  // stage 2, FP64 state, odd NP: every mode's increment (jbase = 0)
#pragma unroll
  for (int i0 = 0; i0 < NP; i0 += JB) {
    if (i0 >= jcnt) break;
    float4 pa[JB], da[JB], ha[JB], la[JB];
    double2 ua[(JB + 1) / 2][4];  // stage 2, FP64 state: modes (j + 2h, j + 2h + 1) of variable m
#pragma unroll
    for (int i = 0; i < JB; ++i) {
      const int ii = i0 + i, j = jbase + ii;
      if (ii >= jcnt) continue;
      pa[i] = part[j];
      if (STG >= 1) da[i] = dp[j];
      if (STG == 0 && rs) {
        ha[i] = lds4(rs + (j == 0 ? 0 : j + 1));
        if (j == 0) la[i] = lds4(rs + 1);
      } else if (STG <= 1) {
        ha[i] = r0[j == 0 ? 0 : j + 1];
        if (j == 0) la[i] = r0[1];
      } else if (kahan) {
        ha[i] = ks[j == 0 ? 0 : j + 1];
        la[i] = ks[j == 0 ? 1 : NF4 + j - 1];
      }
    }
    if constexpr (STG == 2 && PAIRS) {
      const double2* a2 = reinterpret_cast<const double2*>(u);
#pragma unroll
      for (int h = 0; h < JB / 2; ++h)
        if (i0 + 2 * h < jcnt)
#pragma unroll
          for (int m = 0; m < 4; ++m) ua[h][m] = a2[(m * NP + jbase + i0 + 2 * h) / 2];
    }
    float dfirst[4];  // stage 2, FP64 state: the first mode of the current pair
#pragma unroll
    for (int i = 0; i < JB; ++i) {
      const int ii = i0 + i, j = jbase + ii;
      if (ii >= jcnt) continue;
      float a[4];
      mode_sum<P>(lds4(tb + j), b, a);
      const float4 dL = f4_mul_f2(f4_add(pa[i], a), dtp);
      if constexpr (STG < 2) {
        float4 d = dL;
        if (STG == 1)
          d = make_float4(0.25f * (da[i].x + dL.x), 0.25f * (da[i].y + dL.y), 0.25f * (da[i].z + dL.z),
                          0.25f * (da[i].w + dL.w));
        dp[j] = d;
        if (j == 0) {
          float4 h = ha[i], l = la[i];
          const F2 p0 = split_f2(phi0);
          pair_add_scaled(h.x, l.x, d.x, p0);
          pair_add_scaled(h.y, l.y, d.y, p0);
          pair_add_scaled(h.z, l.z, d.z, p0);
          pair_add_scaled(h.w, l.w, d.w, p0);
          ro[0] = h;
          ro[1] = l;
        } else {
          ro[j + 1] = make_float4(ha[i].x + d.x, ha[i].y + d.y, ha[i].z + d.z, ha[i].w + d.w);
        }
      } else {
        // stage 2: delta_2 + dt L; b_2 = 2/3 is applied by the state update
        const float d[4] = {da[i].x + dL.x, da[i].y + dL.y, da[i].z + dL.z, da[i].w + dL.w};
        if constexpr (kahan) {
          float4 h = ha[i], l = la[i];
          const F2 c = split_f2(j == 0 ? 2.0 / 3.0 * phi0 : 2.0 / 3.0);
          kahan_add(h.x, l.x, mul_f2(d[0], c));
          kahan_add(h.y, l.y, mul_f2(d[1], c));
          kahan_add(h.z, l.z, mul_f2(d[2], c));
          kahan_add(h.w, l.w, mul_f2(d[3], c));
          ks[j == 0 ? 0 : j + 1] = h;
          ks[j == 0 ? 1 : NF4 + j - 1] = l;
        } else if constexpr (PAIRS) {
          // u = u0 + (2/3) f64(delta): modes (j-1, j) of each variable as one double2
          if (i % 2 == 0) {
#pragma unroll
            for (int m = 0; m < 4; ++m) dfirst[m] = d[m];
          } else {
            double2* o2 = reinterpret_cast<double2*>(u);
#pragma unroll
            for (int m = 0; m < 4; ++m)
              o2[(m * NP + j - 1) / 2] = make_double2(fma(2.0 / 3.0, f2d(dfirst[m]), ua[i / 2][m].x),
                                                      fma(2.0 / 3.0, f2d(d[m]), ua[i / 2][m].y));
          }
        } else {
#pragma unroll
          for (int m = 0; m < 4; ++m) dk[ii][m] = d[m];
        }
      }
    }
  }
  if constexpr (STG == 2 && !PAIRS) {
    // odd NP (p = 1, 12 values): u = u0 + (2/3) f64(delta) over the [M][NP]
    // FP64 block, all loads before the stores; only a lane that holds every
    // mode (jbase = 0, jcnt = NP) writes it
    if (jcnt == NP) {
      constexpr int H = 2 * NP;
      double2* u2 = reinterpret_cast<double2*>(u);
      double2 a[H];
#pragma unroll
      for (int i = 0; i < H; ++i) a[i] = u2[i];
#pragma unroll
      for (int i = 0; i < H; ++i) {
        const int v = 2 * i, m0 = v / NP, j0 = v % NP, m1 = (v + 1) / NP, j1 = (v + 1) % NP;
        u2[i] = make_double2(fma(2.0 / 3.0, f2d(dk[j0][m0]), a[i].x), fma(2.0 / 3.0, f2d(dk[j1][m1]), a[i].y));
      }
    }
  }
}

// Two lanes per edge side (S = 2): the modes each takes in the epilogues.  The
// first lane takes modes [0, split), the second [split, NP); split is even when
// NP is (the FP64 state update of stage 2 pairs modes into double2).
template <int P>
__host__ __device__ constexpr int mode_split() {
  constexpr int NP = TriDim<P>::NP;
  return NP % 2 == 0 ? 2 * ((NP + 2) / 4) : (NP + 1) / 2;
}

// MODE == SURF_FIRST with STG == 0 (FP64 state, FP32 rhs): the first color of
// stage 0 of the mixed step, which also writes its element's record of u0 and
// FP32 CFL estimate (both as pass 1 of the CFL reduction would) into A.rec_first
// and A.est, and returns the estimate in *best (FLT_MAX for lanes that write
// nothing).
// S lanes per edge side (threads per edge 2 S).  S = 2: the two lanes of a
// side (sub = 0, 1; lanes 2 apart, the sides' lanes adjacent) both load the
// element's record and form its edge coefficients; lane sub takes the edge
// points sub, sub + 2, ... and the volume points likewise, their sums are
// combined across the two lanes, and each lane writes its share of the modes
// (mode_split).  FP32 right-hand sides of the colored modes only.
template <int P, typename ST, typename RT, int MODE, int STG = -1, int S = 1, bool BC = false>
__device__ __forceinline__ void surf_fp32(const SurfParams& A, int64_t k, int4 tp, bool valid, int side,
                                          const float* se, float* rslot = nullptr, float* best = nullptr,
                                          int sub = 0) {
  using D = TriDim<P>;
  using T = ETab32<P>;
  constexpr int NP = D::NP, NQ = D::NQE, NV = D::NV, K1 = P + 1;
  // the FP32 path writes FP32 right-hand sides only in the colored modes
  static_assert(sizeof(RT) == 8 || MODE == SURF_FIRST || MODE == SURF_RMW || MODE == SURF_LAST, "FP32 rhs modes");
  static_assert(S == 1 || (S == 2 && sizeof(RT) == 4), "two lanes per side: the FP32 right-hand sides of a step");
  // the modes this lane writes, [jlo, jlo + jn)
  constexpr int JS = S == 1 ? NP : mode_split<P>();
  const int jlo = sub ? JS : 0, jn = sub ? NP - JS : JS;
  const bool bnd = tp.y < 0;  // boundary: both lanes read the left element (U+ = U-)
  const bool right = side && !bnd;
  const int64_t elem = right ? tp.y : tp.x;
  const int le = right ? ((tp.z >> 4) & 15) : (tp.z & 15);
  const bool writer = valid && !(side && bnd);
  const double2 g0 = A.fgeo[2 * k], g1 = A.fgeo[2 * k + 1];
  const float4* tb = reinterpret_cast<const float4*>(se + ((right ? A.ntab : 0) + le) * T::BLK);
  const TriTab<float, P>& K = tri_tab<float, P>();
  const TriEdgeK<P>& EK = tri_ek<P>();

  // The first color reads the record its predecessor (the previous stage's last
  // color) wrote and overwrites the rhs that predecessor read: it waits at once.
  // The other colors read records written two launches back or earlier; they
  // wait only before their epilogue, which reads the predecessor's rhs.
  if constexpr (MODE == SURF_FIRST) {
    pdl_wait();
    pdl_trigger();
  }

  // The element's state.  The first color (volume integral) and FP64 states
  // take it as a [M][NP] block; the other colors load the FP32 record as it is
  // stored (mode-major), all of it in flight at once (the last color's stage 0
  // also parks it in the lane's shared-memory slot for its epilogue).
  constexpr bool BLOCK = MODE == SURF_FIRST || sizeof(ST) == 8;
  PertBlock<P> B;
  float4 rv[BLOCK ? 1 : D::NF / 4];
  float hi[4], lo[4];
  if constexpr (BLOCK) {
    const int64_t stride = sizeof(ST) == 8 ? NV : A.sstride;
    load_pert<P>(static_cast<const ST*>(A.state) + elem * stride, B);
#pragma unroll
    for (int m = 0; m < 4; ++m) {
      hi[m] = B.hi[m];
      lo[m] = B.lo[m];
    }
  } else {
    const float4* src = reinterpret_cast<const float4*>(static_cast<const float*>(A.state) + elem * A.sstride);
#pragma unroll
    for (int i = 0; i < D::NF / 4; ++i) rv[i] = __ldg(src + i);
    if constexpr (MODE == SURF_LAST && STG == 0) {
      // stage 0's epilogue needs this record again (it is the record of u0):
      // it waits in the lane's shared-memory slot instead of being re-read
      if (rslot)
#pragma unroll
        for (int i = 0; i < D::NF / 4; ++i) sts4(rslot + 4 * i, rv[i]);
    }
    hi[0] = rv[0].x, hi[1] = rv[0].y, hi[2] = rv[0].z, hi[3] = rv[0].w;
    lo[0] = rv[1].x, lo[1] = rv[1].y, lo[2] = rv[1].z, lo[3] = rv[1].w;
  }
  PertRef<2> R;
  R.init(hi);

  // 1. edge coefficients a_k of the trace deviation
  float ak[K1][4];
#pragma unroll
  for (int m = 0; m < 4; ++m) {
    ak[0][m] = lo[m];
#pragma unroll
    for (int kk = 1; kk < K1; ++kk) ak[kk][m] = 0.0f;
  }
#pragma unroll
  for (int j = 1; j < NP; ++j) {
    float c[4];
    if constexpr (BLOCK) {
#pragma unroll
      for (int m = 0; m < 4; ++m) c[m] = B.cd[m][j - 1];
    } else {
      const float4 v = rv[j + 1];
      c[0] = v.x, c[1] = v.y, c[2] = v.z, c[3] = v.w;
    }
    const float4 row = lds4(tb + j);
    const float tr[4] = {row.x, row.y, row.z, row.w};
#pragma unroll
    for (int kk = 0; kk < K1; ++kk)
#pragma unroll
      for (int m = 0; m < 4; ++m) ak[kk][m] = fmaf(tr[kk], c[m], ak[kk][m]);
  }
  // the second lane of a boundary face: the outside state (the face normal is g0)
  bool shk = false;
  if constexpr (BC) shk = bnd && side && bc_modal32<K1>(A, tp.w, d2f(g0.x), d2f(g0.y), R.u, ak);

  if constexpr (MODE == SURF_FIRST) {
    // First color: the volume integral, then the edge's points one at a time
    // (the record stays in registers for the volume integral anyway).
    float acc[NV];
#pragma unroll
    for (int i = 0; i < NV; ++i) acc[i] = 0.0f;
    if constexpr (STG == 0 && sizeof(ST) == 8) {
      static_assert(sizeof(RT) == 4, "the stage-0 first color writes the FP32 rhs of the step");
      float lam = 0.0f;
      volume_acc32<P, true, S>(B, R, A.jinv + 4 * elem, acc, &lam, sub);
      if constexpr (S == 2) lam = fmaxf(lam, __shfl_xor_sync(0xffffffffu, lam, 2));
      if (writer) {
        // the record of u0 (mode-major), as the CFL pass 1 writes it (mode j at
        // float4 j + 1, the mean pair at 0 and 1; each lane its share)
        float4* r = reinterpret_cast<float4*>(A.rec_first + elem * D::NF);
        if (jlo == 0) {
          r[0] = make_float4(B.hi[0], B.hi[1], B.hi[2], B.hi[3]);
          r[1] = make_float4(B.lo[0], B.lo[1], B.lo[2], B.lo[3]);
        }
#pragma unroll
        for (int j = 1; j < NP; ++j)
          if (S == 1 || (j >= jlo && j < jlo + jn))
            r[j + 1] = make_float4(B.cd[0][j - 1], B.cd[1][j - 1], B.cd[2][j - 1], B.cd[3][j - 1]);
        if (sub == 0) {
          float dd = d2f(__ldg(A.inr + elem)) / ((2 * P + 1) * lam);
          if (!(dd > 0.0f) || !(dd < FLT_MAX)) dd = 0.0f;  // non-physical: always re-evaluated
          A.est[elem] = dd;
          *best = dd;
        }
      }
    } else {
      volume_acc32<P, false, S>(B, R, A.jinv + 4 * elem, acc, nullptr, sub);
    }
    FaceConst<2> E;
    E.init(R, hi, {d2f(g0.x), d2f(g0.y)}, side);
    const float escale = right ? d2f(g1.y) : -d2f(g1.x);  // the lane's signed edge measure
    float bk[K1][4];
#pragma unroll
    for (int kk = 0; kk < K1; ++kk)
#pragma unroll
      for (int m = 0; m < 4; ++m) bk[kk][m] = 0.0f;
    // (every lane of a pair runs the same number of points: the shuffles of
    // lf_exchange need all 32 lanes; a lane past the last point repeats it
    // with weight 0)
    DGC_UNROLL_Q
    for (int i = 0; i < (NQ + S - 1) / S; ++i) {
      const int q0 = S * i + sub, q = q0 < NQ ? q0 : NQ - 1;
      float L[K1], t[4], G[4];
#pragma unroll
      for (int kk = 0; kk < K1; ++kk) L[kk] = EK.Lq[q][kk];
#pragma unroll
      for (int m = 0; m < 4; ++m) {
        float v = ak[0][m];
#pragma unroll
        for (int kk = 1; kk < K1; ++kk) v = fmaf(L[kk], ak[kk][m], v);
        t[m] = v;
      }
      if (BC && shk) bc_shock32(A, ak[0], tri_tab<double, P>().tE[q], R.u, t);
      lf_exchange<2>(R, E, t, G);
      const float s = q0 < NQ ? escale * K.wE[q] : 0.0f;
#pragma unroll
      for (int m = 0; m < 4; ++m) {
        const float g = s * G[m];
#pragma unroll
        for (int kk = 0; kk < K1; ++kk) bk[kk][m] = fmaf(L[kk], g, bk[kk][m]);
      }
    }
    if constexpr (S == 2) {
      // the two lanes' point sums: edge coefficients and volume integral
#pragma unroll
      for (int kk = 0; kk < K1; ++kk)
#pragma unroll
        for (int m = 0; m < 4; ++m) bk[kk][m] += __shfl_xor_sync(0xffffffffu, bk[kk][m], 2);
#pragma unroll
      for (int m = 0; m < 4; ++m)
#pragma unroll
        for (int j = 1; j < NP; ++j) acc[m * NP + j] += __shfl_xor_sync(0xffffffffu, acc[m * NP + j], 2);
    }
    if (!writer) return;
#pragma unroll
    for (int j = 0; j < NP; ++j) {
      float a[4];
      mode_sum<P>(lds4(tb + j), bk, a);
#pragma unroll
      for (int m = 0; m < 4; ++m) acc[m * NP + j] += a[m];
    }
    if constexpr (S == 2) {
      // this lane's share of the modes of the mode-major FP32 rhs
      float4* r = reinterpret_cast<float4*>(static_cast<float*>(A.rhs) + elem * NV);
#pragma unroll
      for (int j = 0; j < NP; ++j)
        if (j >= jlo && j < jlo + jn) r[j] = make_float4(acc[j], acc[NP + j], acc[2 * NP + j], acc[3 * NP + j]);
    } else if constexpr (sizeof(RT) == 4) {
      store_rhs<P>(static_cast<float*>(A.rhs) + elem * NV, acc);
    } else {
      surf_write<P, RT, MODE>(A, elem, k, side, acc);
    }
  } else {
    // 2. fluxes at every point; then 3. b_k = sum_q w_q G_q L_k(xi_q)
    FaceConst<2> E;
    E.init(R, hi, {d2f(g0.x), d2f(g0.y)}, side);
    const float escale = right ? d2f(g1.y) : -d2f(g1.x);  // the lane's signed edge measure
    float bk[K1][4];
#pragma unroll
    for (int kk = 0; kk < K1; ++kk)
#pragma unroll
      for (int m = 0; m < 4; ++m) bk[kk][m] = 0.0f;
#pragma unroll
    for (int i = 0; i < (NQ + S - 1) / S; ++i) {
      const int q0 = S * i + sub, q = q0 < NQ ? q0 : NQ - 1;  // as in the first color
      float t[4], G[4];
#pragma unroll
      for (int m = 0; m < 4; ++m) {
        float v = ak[0][m];
#pragma unroll
        for (int kk = 1; kk < K1; ++kk) v = fmaf(EK.Lq[q][kk], ak[kk][m], v);
        t[m] = v;
      }
      if (BC && shk) bc_shock32(A, ak[0], tri_tab<double, P>().tE[q], R.u, t);
      lf_exchange<2>(R, E, t, G);
      const float s = q0 < NQ ? escale * K.wE[q] : 0.0f;
#pragma unroll
      for (int m = 0; m < 4; ++m) {
        const float g = s * G[m];
#pragma unroll
        for (int kk = 0; kk < K1; ++kk) bk[kk][m] = fmaf(EK.Lq[q][kk], g, bk[kk][m]);
      }
    }
    if constexpr (S == 2) {
#pragma unroll
      for (int kk = 0; kk < K1; ++kk)
#pragma unroll
        for (int m = 0; m < 4; ++m) bk[kk][m] += __shfl_xor_sync(0xffffffffu, bk[kk][m], 2);
    }

    // modes and epilogue, after the predecessor grid has completed
    pdl_wait();
    pdl_trigger();
    if (!writer) return;
    if constexpr (MODE == SURF_LAST) {
      // (the FP64 state of the mixed form is updated in place: S.u0 == S.uout)
      const StageArgs& SA = A.sa;
      const float4* part = reinterpret_cast<const float4*>(static_cast<const float*>(A.rhs) + elem * NV);
      float4* dp = reinterpret_cast<float4*>(SA.delta + elem * NV);
      const float4* r0 = reinterpret_cast<const float4*>(SA.rec0 + elem * SA.rec0_stride);
      float4* ro = reinterpret_cast<float4*>(SA.rec_out + elem * D::NF);
      float4* ks = SA.kstate ? reinterpret_cast<float4*>(SA.kstate + elem * SA.rec0_stride) : nullptr;
      double* u = SA.uout ? SA.uout + elem * NV : nullptr;
      const double dt = *SA.dt, phi0 = tri_tab<double, P>().phiV[0][0];
      const int stage = STG >= 0 ? STG : (SA.stage == 2 && ks ? 3 : SA.stage);
      const float4* rs = reinterpret_cast<const float4*>(rslot);
      if constexpr (S == 1) {
        if (stage == 0) last_modes<P, 0>(tb, bk, rs, part, dp, r0, ro, ks, u, dt, phi0);
        else if (stage == 1) last_modes<P, 1>(tb, bk, nullptr, part, dp, r0, ro, ks, u, dt, phi0);
        else if (stage == 2) last_modes<P, 2>(tb, bk, nullptr, part, dp, r0, ro, ks, u, dt, phi0);
        else last_modes<P, 3>(tb, bk, nullptr, part, dp, r0, ro, ks, u, dt, phi0);
      } else {
        // stage 2 of the FP64 state with an odd mode count writes the whole
        // [M][NP] block at once: the first lane of the side takes every mode
        const bool whole = stage == 2 && NP % 2 == 1;
        const int b0 = whole ? (sub ? NP : 0) : jlo, n0 = whole ? (sub ? 0 : NP) : jn;
        if (stage == 0) last_modes<P, 0>(tb, bk, rs, part, dp, r0, ro, ks, u, dt, phi0, b0, n0);
        else if (stage == 1) last_modes<P, 1>(tb, bk, nullptr, part, dp, r0, ro, ks, u, dt, phi0, b0, n0);
        else if (stage == 2) last_modes<P, 2>(tb, bk, nullptr, part, dp, r0, ro, ks, u, dt, phi0, b0, n0);
        else last_modes<P, 3>(tb, bk, nullptr, part, dp, r0, ro, ks, u, dt, phi0, b0, n0);
      }
    } else if constexpr (sizeof(RT) == 4) {
      // read-modify-write in batches of JB modes, each batch's loads first
      // (this lane's modes [jlo, jlo + jn))
      constexpr int JB = 5;
      float4* r = reinterpret_cast<float4*>(static_cast<float*>(A.rhs) + elem * NV) + jlo;
#pragma unroll
      for (int j0 = 0; j0 < JS; j0 += JB) {
        if (j0 >= jn) break;
        float4 o[JB];
#pragma unroll
        for (int i = 0; i < JB; ++i)
          if (j0 + i < jn) o[i] = r[j0 + i];
#pragma unroll
        for (int i = 0; i < JB; ++i) {
          if (j0 + i >= jn) continue;
          float a[4];
          mode_sum<P>(lds4(tb + jlo + j0 + i), bk, a);
          r[j0 + i] = f4_add(o[i], a);
        }
      }
    } else {
      float acc[NV];
#pragma unroll
      for (int j = 0; j < NP; ++j) {
        float a[4];
        mode_sum<P>(lds4(tb + j), bk, a);
#pragma unroll
        for (int m = 0; m < 4; ++m) acc[m * NP + j] = a[m];
      }
      surf_write<P, RT, MODE>(A, elem, k, side, acc);
    }
  }
}

void tri_upload_tables(int p, const RefTables& R) {
  if (R.dim != 2 || R.p != p) return;
  if (p == 1) upload_p<1>(R, &cTriD1, &cTriF1);
  if (p == 2) upload_p<2>(R, &cTriD2, &cTriF2);
  if (p == 3) upload_p<3>(R, &cTriD3, &cTriF3);
  if (p == 1) upload_ek<1>(R, &cTriK1);
  if (p == 2) upload_ek<2>(R, &cTriK2);
  if (p == 3) upload_ek<3>(R, &cTriK3);
  if (p == 1) upload_pairs<1>(R, &cTriP1);
  if (p == 2) upload_pairs<2>(R, &cTriP2);
  if (p == 3) upload_pairs<3>(R, &cTriP3);
  if (p == 1) upload_df<1>(R, &cTriDF1);
  if (p == 2) upload_df<2>(R, &cTriDF2);
  if (p == 3) upload_df<3>(R, &cTriDF3);
}

// One lane of the pair that handles edge k (side 0: left element, 1: right).
// Lanes with valid = false shadow a real edge (so both lanes of every pair
// take part in the shuffles) and write nothing.
template <int P, typename CT, typename ST, typename RT, int MODE>
__device__ __forceinline__ void surf_pair(const SurfParams& A, int64_t k, int4 tp, bool valid, int side,
                                          const CT* sphi, const CT* sw);


// Register caps of the FP32 surface kernels, chosen for resident warps
// (blocks of 128 threads: 128 registers give 4 blocks per SM, 96 give 5, 80
// give 6) and measured at p = 3: the middle colors at 80; the last color's
// stage 0 (batches of six modes, two operand arrays) at 104 and its stages 1
// and 2 (batches of four modes, three operand arrays) at 96; the first color
// (volume integral) and the kernels reading an FP64 state (right-hand side
// calls and comparators), which keep the element block in registers, at 128.
// FP64 pair lanes at 168 at p = 2 and uncapped at p = 3 (measured, packed pair
// updates: p = 2 RK step 12.06 ms at 168 against 12.89 at 255; p = 3 21.08 ms
// at 255 against 21.27 at 200 and 21.65 at 168).
#ifndef DGC_REGS_P3_FIRST
#define DGC_REGS_P3_FIRST 128
#endif
#ifndef DGC_REGS_P3
#define DGC_REGS_P3 80
#endif
#ifndef DGC_REGS_P3_LAST
#define DGC_REGS_P3_LAST 104
#endif
#ifndef DGC_REGS_P3_LAST12
#define DGC_REGS_P3_LAST12 96
#endif
#ifndef DGC_REGS_P2_FIRST
#define DGC_REGS_P2_FIRST 96
#endif
#ifndef DGC_REGS_P2
#define DGC_REGS_P2 80
#endif
#ifndef DGC_REGS_FP64
#define DGC_REGS_FP64 168
#endif
#ifndef DGC_REGS_FP64_P3
#define DGC_REGS_FP64_P3 255
#endif
template <int P, typename CT, typename ST, typename RT, int MODE, int STG>
constexpr int surf_regs() {
  return sizeof(CT) == 8                        ? (df_lanes<P>() ? (P == 3 ? DGC_REGS_FP64_P3 : DGC_REGS_FP64) : 255)
         : P == 3 && (sizeof(ST) == 8 || sizeof(RT) == 8 || MODE == SURF_FIRST) ? DGC_REGS_P3_FIRST
         : P == 3 && MODE == SURF_LAST && STG >= 1 ? DGC_REGS_P3_LAST12
         : P == 3 && MODE == SURF_LAST          ? DGC_REGS_P3_LAST
         : P == 3                               ? DGC_REGS_P3
         : P == 2 && (sizeof(ST) == 8 || sizeof(RT) == 8 || MODE == SURF_FIRST) ? DGC_REGS_P2_FIRST
         : P == 2 && MODE == SURF_LAST && STG >= 1 ? DGC_REGS_P2_FIRST
         : P == 2                               ? DGC_REGS_P2
                                                : 128;
}

// BC: the FP32 lanes honour boundary conditions (A.bc set; the FP64 lanes test
// A.bc at run time).  Meshes without take BC = false, whose point loops carry
// no boundary code.
template <int P, typename CT, typename ST, typename RT, int MODE, int STG = -1, int S = 1, bool BC = false>
__global__ void __launch_bounds__(256) __maxnreg__((surf_regs<P, CT, ST, RT, MODE, STG>())) k_surf_tri(const SurfParams A) {
  using D = TriDim<P>;
  // lanes 2S e .. 2S e + 2S - 1 take edge e: side = bit 0, the lane of the side bit 1 (S = 2)
  constexpr int SH = S == 2 ? 2 : 1;
  const int side = threadIdx.x & 1, sub = S == 2 ? (threadIdx.x >> 1) & 1 : 0;
  const int64_t gtid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  // A.persistent: the grid is at most one wave and every warp loops over the
  // color in steps of the whole grid; else one edge per lane group.  The loop
  // test is on the warp's first edge, so a warp runs (and shuffles) together.
  const int64_t step = A.persistent ? ((int64_t)gridDim.x * blockDim.x) >> SH : 0;
  if constexpr (sizeof(CT) == 4) {
    __shared__ __align__(16) float se[ETab32<P>::SIZE];
    extern __shared__ float4 rslots[];  // the last color's stage 0: rec_slot<P>() floats per thread
    stage_etab32<P>(se, A.ntab);
    __syncthreads();
    float* rslot = nullptr;
    if constexpr (MODE == SURF_LAST && STG == 0 && sizeof(ST) == 4)
      rslot = reinterpret_cast<float*>(rslots) + threadIdx.x * rec_slot<P>();
    float best = FLT_MAX;
    for (int64_t k0 = A.begin + (gtid >> SH), kw = A.begin + ((gtid & ~(int64_t)31) >> SH); kw < A.end;
         k0 += step, kw += step) {
      const bool valid = k0 < A.end;
      const int64_t k = valid ? k0 : A.end - 1;  // idle lanes shadow the last edge so both lanes of a pair shuffle
      const int4 tp = A.topo[k];
      if constexpr (MODE == SURF_FIRST && STG == 0) {
        float b = FLT_MAX;
        surf_fp32<P, ST, RT, MODE, STG, S, BC>(A, k, tp, valid, side, se, rslot, &b, sub);
        best = fminf(best, b);
      } else {
        surf_fp32<P, ST, RT, MODE, STG, S, BC>(A, k, tp, valid, side, se, rslot, nullptr, sub);
      }
      if (!step) break;
    }
    if constexpr (MODE == SURF_FIRST && STG == 0) block_min_to(best, A.estmin);
  } else {
    static_assert(S == 1, "FP64 lanes: one per edge side");
    __shared__ __align__(16) double sphi[kFp64TabWords * 9 * D::NQE * D::NP];
    __shared__ double sw[D::NQE];
    stage_edge_tables<P, double>(sphi, sw, A.ntab);
    __syncthreads();
    for (int64_t k0 = A.begin + (gtid >> 1), kw = A.begin + ((gtid & ~(int64_t)31) >> 1); kw < A.end;
         k0 += step, kw += step) {
      const bool valid = k0 < A.end;
      const int64_t k = valid ? k0 : A.end - 1;
      const int4 tp = A.topo[k];
      surf_pair<P, double, ST, RT, MODE>(A, k, tp, valid, side, sphi, sw);
      if (!step) break;
    }
  }
}


template <int P, typename CT, typename ST, typename RT, int MODE>
__device__ __forceinline__ void surf_pair(const SurfParams& A, int64_t k, int4 tp, bool valid, int side,
                                          const CT* sphi, const CT* sw) {
  using D = TriDim<P>;
  constexpr int NP = D::NP, NQ = D::NQE, NV = D::NV;
  const bool bnd = tp.y < 0;  // boundary: both lanes read the left element (U+ = U-)
  const bool right = side && !bnd;
  const int64_t elem = right ? tp.y : tp.x;
  const int le = right ? ((tp.z >> 4) & 15) : (tp.z & 15);
  const bool writer = valid && !(side && bnd);
  const double2 g0 = A.fgeo[2 * k], g1 = A.fgeo[2 * k + 1];
  // (in SURF_LAST the state may alias the stage output, but each element's
  // block is read and written by its own lane only)

  static_assert(sizeof(CT) == 8, "FP64 lanes; the FP32 ones are surf_fp32");
  if constexpr (MODE == SURF_FIRST) {  // programmatic launch: as in surf_fp32
    pdl_wait();
    pdl_trigger();
  }
  if constexpr (!df_lanes<P>()) {
    // ---------------- FP64: Eq. 2 as written ----------------
    double c[NV], acc[NV];
    load_block(static_cast<const double*>(A.state) + elem * NV, c);
#pragma unroll
    for (int i = 0; i < NV; ++i) acc[i] = 0.0;
    if constexpr (MODE == SURF_FIRST) volume_acc64<P>(c, A.jinv + 4 * elem, acc);
    const double nx = g0.x, ny = g0.y, scale = right ? g1.y : -g1.x;
    const CT* ph = sphi + le * NQ * NP;
    DGC_UNROLL_Q
    for (int q = 0; q < NQ; ++q) {
      const int qq = right ? NQ - 1 - q : q;  // the right element runs along the edge backwards
      double phi[NP], U[4], V[4], a[4], b[4], Fs[4];
#pragma unroll
      for (int j = 0; j < NP; ++j) phi[j] = ph[qq * NP + j];
#pragma unroll
      for (int m = 0; m < 4; ++m) {
        double s = 0.0;
#pragma unroll
        for (int j = 0; j < NP; ++j) s += phi[j] * c[m * NP + j];
        U[m] = s;
      }
      // a boundary face's second lane holds the state outside it
      if (bnd && side && A.bc) bc_outside(A, tp.w, tri_tab<double, P>().tE[q], nx, ny, U);
      // own side's normal flux and wave speed, then the partner's
      double Fo[4], Fp[4], wo;
      lf_side(U, nx, ny, Fo, wo);
#pragma unroll
      for (int m = 0; m < 4; ++m) {
        V[m] = __shfl_xor_sync(0xffffffffu, U[m], 1);
        Fp[m] = __shfl_xor_sync(0xffffffffu, Fo[m], 1);
      }
      const double lam = fmax(wo, __shfl_xor_sync(0xffffffffu, wo, 1));
      // F* = (F(a).n + F(b).n)/2 - lam (b - a)/2 with a = left, b = right: the
      // sums are commutative, so both lanes get the same bits (conservation)
#pragma unroll
      for (int m = 0; m < 4; ++m) {
        a[m] = side ? V[m] : U[m];
        b[m] = side ? U[m] : V[m];
        Fs[m] = 0.5 * (Fo[m] + Fp[m]) - (0.5 * lam) * (b[m] - a[m]);
      }
      const double s = scale * sw[q];
#pragma unroll
      for (int m = 0; m < 4; ++m) {
        const double g = s * Fs[m];
#pragma unroll
        for (int j = 0; j < NP; ++j) acc[m * NP + j] += phi[j] * g;
      }
    }
    if constexpr (MODE != SURF_FIRST) {
      pdl_wait();
      pdl_trigger();
    }
    if constexpr (MODE == SURF_LAST) {
      if (writer) fp64_last<P>(A, elem, acc, c);
    } else if (writer) {
      surf_write<P, RT, MODE>(A, elem, k, side, acc);
    }
  } else {
    // ---------------- FP64: Eq. 2, contractions in FP32 pairs ----------------
    DfBlock<P> B;
    {
      double c[NV];
      load_block(static_cast<const double*>(A.state) + elem * NV, c);
      B.init(c);
    }
    double Fb[4], Gb[4];  // the x and y fluxes of the element's mean
    euler_xy(B.ub, Fb, Gb);
    DfAcc<P> acc2;
    acc2.zero();
    if constexpr (MODE == SURF_FIRST) volume_df<P>(B, Fb, Gb, A.jinv + 4 * elem, acc2);
    const double nx = g0.x, ny = g0.y, scale = right ? g1.y : -g1.x;
    double Fbn[4];  // F(ub).n, subtracted from the face flux (the volume integral omits F(ub))
#pragma unroll
    for (int m = 0; m < 4; ++m) Fbn[m] = Fb[m] * nx + Gb[m] * ny;
    const float4* ph = reinterpret_cast<const float4*>(sphi) + le * NQ * NP;
    const DF sdf = df_split(scale);
    DGC_UNROLL_Q
    for (int q = 0; q < NQ; ++q) {
      const int qq = right ? NQ - 1 - q : q;  // the right element runs along the edge backwards
      double U[4], V[4], a[4], b[4], Fs[4];
#pragma unroll
      for (int k = 0; k < 2; ++k) {
        float2 th = make_float2(0.0f, 0.0f), tl = th;
#pragma unroll
        for (int j = 1; j < NP; ++j) df_fma2(th, tl, ph[qq * NP + j], B.ch[k][j - 1], B.cl[k][j - 1]);
        U[2 * k] = B.ub[2 * k] + df_join(DF{th.x, tl.x});
        U[2 * k + 1] = B.ub[2 * k + 1] + df_join(DF{th.y, tl.y});
      }
      // a boundary face's second lane holds the state outside it
      if (bnd && side && A.bc) bc_outside(A, tp.w, tri_tab<double, P>().tE[q], nx, ny, U);
      // own side's normal flux and wave speed, then the partner's
      double Fo[4], Fp[4], wo;
      lf_side(U, nx, ny, Fo, wo);
#pragma unroll
      for (int m = 0; m < 4; ++m) {
        V[m] = __shfl_xor_sync(0xffffffffu, U[m], 1);
        Fp[m] = __shfl_xor_sync(0xffffffffu, Fo[m], 1);
      }
      const double lam = fmax(wo, __shfl_xor_sync(0xffffffffu, wo, 1));
      // F* = (F(a).n + F(b).n)/2 - lam (b - a)/2 with a = left, b = right: the
      // sums are commutative, so both lanes get the same bits (conservation)
#pragma unroll
      for (int m = 0; m < 4; ++m) {
        a[m] = side ? V[m] : U[m];
        b[m] = side ? U[m] : V[m];
        Fs[m] = 0.5 * (Fo[m] + Fp[m]) - (0.5 * lam) * (b[m] - a[m]);
      }
      const DF sq = df_mul(sdf, df_split(sw[q]));
#pragma unroll
      for (int k = 0; k < 2; ++k) {
        const DF g0 = df_mul(sq, df_split(Fs[2 * k] - Fbn[2 * k]));
        const DF g1 = df_mul(sq, df_split(Fs[2 * k + 1] - Fbn[2 * k + 1]));
        const float2 gh = make_float2(g0.h, g1.h), gl = make_float2(g0.l, g1.l);
#pragma unroll
        for (int j = 0; j < NP; ++j) df_fma2(acc2.h[k][j], acc2.l[k][j], ph[qq * NP + j], gh, gl);
      }
    }
    double acc[NV];
#pragma unroll
    for (int m = 0; m < 4; ++m)
#pragma unroll
      for (int j = 0; j < NP; ++j) acc[m * NP + j] = acc2.get(m, j);
    if constexpr (MODE != SURF_FIRST) {
      pdl_wait();
      pdl_trigger();
    }
    if constexpr (MODE == SURF_LAST) {
      double c[NV];  // the stage input block again (cached), for the update
      load_block(static_cast<const double*>(A.state) + elem * NV, c);
      if (writer) fp64_last<P>(A, elem, acc, c);
    } else if (writer) {
      surf_write<P, RT, MODE>(A, elem, k, side, acc);
    }
  }
}

// ---------------------------------------------------------------------------
// CFL reduction: dt = cfl min_e r_e / ((2p+1) max_q (|u| + c)), exact FP64.
// Pass 1 (FP32 arithmetic): every element's estimate, stored, and their
// minimum (one atomicMin per block on the bit pattern); also writes the FP32
// record of the state when asked.  Pass 2 (FP64): only elements whose estimate
// is within kCflMargin of the minimum are evaluated in FP64 and combined with
// one 64-bit atomicMin.  Both minima must hold a large value beforehand.
// ---------------------------------------------------------------------------
template <int P, typename T>
__device__ __forceinline__ T lambda_max(const T (&v)[TriDim<P>::NV]) {
  using D = TriDim<P>;
  constexpr int NP = D::NP;
  const TriTab<T, P>& K = tri_tab<T, P>();
  T lam = T(0);
#pragma unroll
  for (int q = 0; q < D::NQV; ++q) {
    T U[4];
#pragma unroll
    for (int m = 0; m < 4; ++m) {
      T s = T(0);
#pragma unroll
      for (int j = 0; j < NP; ++j) s += K.phiV[q][j] * v[m * NP + j];
      U[m] = s;
    }
    const T ir = T(1) / U[0], u = U[1] * ir, w = U[2] * ir;
    const T q2 = u * u + w * w;
    const T pr = T(0.4) * (U[3] - T(0.5) * U[0] * q2);
    lam = fmax(lam, sqrt(q2) + sqrt(T(1.4) * pr * ir));
  }
  return lam;
}

// The same FP64 maximum evaluated by the whole warp for one element (lane q
// takes the points q, q + 32, ...), valid in every lane.  A GB300 FP64 warp
// instruction occupies the FP64 pipe for ~64 cycles, so one lane alone running
// all points would take tens of microseconds.
template <int P>
__device__ __forceinline__ double lambda_max_warp(const double (&v)[TriDim<P>::NV]) {
  using D = TriDim<P>;
  constexpr int NP = D::NP;
  const TriTab<double, P>& K = tri_tab<double, P>();
  double lam = 0.0;
  for (int q = threadIdx.x & 31; q < D::NQV; q += 32) {
    double U[4];
#pragma unroll
    for (int m = 0; m < 4; ++m) {
      double s = 0.0;
#pragma unroll
      for (int j = 0; j < NP; ++j) s += K.phiV[q][j] * v[m * NP + j];
      U[m] = s;
    }
    const double ir = 1.0 / U[0], u = U[1] * ir, w = U[2] * ir;
    const double q2 = u * u + w * w;
    const double pr = 0.4 * (U[3] - 0.5 * U[0] * q2);
    lam = fmax(lam, sqrt(q2) + sqrt(1.4 * pr * ir));
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) lam = fmax(lam, __shfl_xor_sync(0xffffffffu, lam, o));
  return lam;
}

// FP32 estimate of max_q (|u| + c) from the FP32 record (mean pair + modes)
template <int P>
__device__ __forceinline__ float lambda_max_rec(const float (&r)[TriDim<P>::NF]) {
  using D = TriDim<P>;
  constexpr int NP = D::NP;
  float lam = 0.0f;
#if DGC_FFMA2
  const TriPairTab<P>& K2 = tri_ptab<P>();
#else
  const TriTab<float, P>& K = tri_tab<float, P>();
#endif
  DGC_UNROLL_Q
  for (int q = 0; q < D::NQV; ++q) {
    float U[4];
#if DGC_FFMA2
    // variables in pairs: the record's modes are float4 over the variables
    float2 s01 = make_float2(r[4], r[5]), s23 = make_float2(r[6], r[7]);
#pragma unroll
    for (int j = 1; j < NP; ++j) {
      s01 = __ffma2_rn(K2.phiV[q][j], make_float2(r[4 * (j + 1)], r[4 * (j + 1) + 1]), s01);
      s23 = __ffma2_rn(K2.phiV[q][j], make_float2(r[4 * (j + 1) + 2], r[4 * (j + 1) + 3]), s23);
    }
    U[0] = r[0] + s01.x;
    U[1] = r[1] + s01.y;
    U[2] = r[2] + s23.x;
    U[3] = r[3] + s23.y;
#else
#pragma unroll
    for (int m = 0; m < 4; ++m) {
      float s = r[4 + m];
#pragma unroll
      for (int j = 1; j < NP; ++j) s += K.phiV[q][j] * r[4 * (j + 1) + m];
      U[m] = r[m] + s;
    }
#endif
    const float ir = rcp_fast(U[0]), u = U[1] * ir, w = U[2] * ir;
    const float q2 = u * u + w * w;
    const float pr = 0.4f * (U[3] - 0.5f * U[0] * q2);
    lam = fmaxf(lam, sqrt_fast(q2) + sqrt_fast(1.4f * pr * ir));
  }
  return lam;
}

// pass 1 for element e: its FP32 estimate (stored), and its FP32 record
template <int P>
__device__ __forceinline__ float cfl1_elem(const double* __restrict__ c, const double* __restrict__ inr, int64_t e,
                                           float* __restrict__ est, float* __restrict__ shadow) {
  using D = TriDim<P>;
  double v[D::NV];
  load_block(c + e * D::NV, v);
  float r[D::NF];
  record_of<P>(v, r);
  if (shadow) store_block(shadow + e * D::NF, r);
  float d = d2f(__ldg(inr + e)) / ((2 * P + 1) * lambda_max_rec<P>(r));
  if (!(d > 0.0f) || !(d < FLT_MAX)) d = 0.0f;  // non-physical: always re-evaluated
  est[e] = d;
  return d;
}

// Pass 2 for the warp's elements e (e < 0: none): the FP64 step of each
// candidate (estimate within kCflMargin of the minimum), evaluated one
// candidate at a time by the whole warp; DBL_MAX for the others.  All 32 lanes
// must call it.  KAHAN: the state is the FP32 pair layout (values hi + lo, the
// mean as phi0 c0), else FP64 coefficients.
template <int P, bool KAHAN>
__device__ __forceinline__ double cfl2_warp(const void* __restrict__ state, const double* __restrict__ inr,
                                            int64_t e, double cfl, const float* __restrict__ est, float minest) {
  using D = TriDim<P>;
  constexpr int NP = D::NP;
  const bool cand = e >= 0 && est[e] <= minest * (1.0f + kCflMargin);
  unsigned mask = __ballot_sync(0xffffffffu, cand);
  double best = DBL_MAX;
  while (mask) {
    const int src = __ffs(mask) - 1;
    mask &= mask - 1;
    const long long ec = __shfl_sync(0xffffffffu, (long long)e, src);
    double v[D::NV];
    if constexpr (KAHAN) {
      const float* k = static_cast<const float*>(state) + ec * (8 * NP);
      const double phi0 = tri_tab<double, P>().phiV[0][0];
#pragma unroll
      for (int m = 0; m < 4; ++m) {
        v[m * NP] = (f2d(k[m]) + f2d(k[4 + m])) / phi0;
#pragma unroll
        for (int j = 1; j < NP; ++j) v[m * NP + j] = f2d(k[4 * (j + 1) + m]) + f2d(k[D::NF + 4 * (j - 1) + m]);
      }
    } else {
      load_block(static_cast<const double*>(state) + ec * D::NV, v);
    }
    const double b = cfl * (__ldg(inr + ec) / ((2 * P + 1) * lambda_max_warp<P>(v)));
    if ((threadIdx.x & 31) == src) best = b > 0.0 ? b : DBL_MAX;  // non-physical state: excluded (NaN)
  }
  return best;
}

template <int P>
__global__ void __launch_bounds__(128) k_cfl1_tri(const double* __restrict__ c, const double* __restrict__ inr,
                                                  int64_t ne, float* __restrict__ est, unsigned* minbits,
                                                  float* __restrict__ shadow) {
  pdl_wait();
  pdl_trigger();
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const float best = e < ne ? cfl1_elem<P>(c, inr, e, est, shadow) : FLT_MAX;
  block_min_to(best, minbits);
}

template <int P, bool KAHAN>
__global__ void __launch_bounds__(128) k_cfl2_tri(const void* __restrict__ c, const double* __restrict__ inr,
                                                  int64_t ne, double cfl, const float* __restrict__ est,
                                                  const unsigned* minbits, unsigned long long* dtbits) {
  pdl_wait();
  pdl_trigger();
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const double best = cfl2_warp<P, KAHAN>(c, inr, e < ne ? e : -1, cfl, est, __uint_as_float(*minbits));
  block_min_to(best, dtbits);
}

// Kahan form: pass 1 reads the record part of the FP32 pair state (no record to
// write); pass 2 evaluates candidates in FP64 from hi + lo of every value.
int tri_kahan_floats(int p) { return 8 * ((p + 1) * (p + 2) / 2); }

template <int P>
__global__ void __launch_bounds__(128) k_cfl1_tri_k(const float* __restrict__ ks, const double* __restrict__ inr,
                                                    int64_t ne, float* __restrict__ est, unsigned* minbits) {
  using D = TriDim<P>;
  pdl_wait();
  pdl_trigger();
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  float best = FLT_MAX;
  if (e < ne) {
    float r[D::NF];
    load_block(ks + e * (8 * D::NP), r);
    float d = d2f(__ldg(inr + e)) / ((2 * P + 1) * lambda_max_rec<P>(r));
    if (!(d > 0.0f) || !(d < FLT_MAX)) d = 0.0f;
    est[e] = d;
    best = d;
  }
  block_min_to(best, minbits);
}

int tri_cfl_kahan(const Ctx& x, const float* ks, double cfl, double* dt) {
  const int bs = 128;
  const unsigned grid = (unsigned)((x.ne + bs - 1) / bs);
  auto* bits = reinterpret_cast<unsigned long long*>(dt);
  float* est = x.d->cfl_est;
  unsigned* mn = reinterpret_cast<unsigned*>(x.d->cfl_est + x.ne);
  if (cudaMemsetAsync(mn, 0x7F, sizeof(unsigned), x.st) != cudaSuccess) return -1;
  switch (x.p) {
    case 1:
      launch_k(x, k_cfl1_tri_k<1>, grid, bs, 0, ks, x.d->inr, x.ne, est, mn);
      launch_k(x, k_cfl2_tri<1, true>, grid, bs, 0, ks, x.d->inr, x.ne, cfl, est, mn, bits);
      return 2;
    case 2:
      launch_k(x, k_cfl1_tri_k<2>, grid, bs, 0, ks, x.d->inr, x.ne, est, mn);
      launch_k(x, k_cfl2_tri<2, true>, grid, bs, 0, ks, x.d->inr, x.ne, cfl, est, mn, bits);
      return 2;
    case 3:
      launch_k(x, k_cfl1_tri_k<3>, grid, bs, 0, ks, x.d->inr, x.ne, est, mn);
      launch_k(x, k_cfl2_tri<3, true>, grid, bs, 0, ks, x.d->inr, x.ne, cfl, est, mn, bits);
      return 2;
    default: return -1;
  }
}

// ---------------------------------------------------------------------------
// Batched meshes: one persistent launch per kernel class covering every mesh.
// The host cuts each mesh's color (or element) range into tiles of at most
// one block's worth of work, sorted by order p; each block walks the tiles
// blockIdx.x, blockIdx.x + gridDim.x, ... and re-stages the edge tables of
// shared memory only when p changes (at most a few times per block).
// ---------------------------------------------------------------------------
// The batched FP32 surface kernels take the register caps of the p = 3
// kernels above (the order with the most registers) plus a few for the tile
// loop's state; one kernel per RK stage of the last color (STG), as there.
#ifndef DGC_BATCH_EXTRA_REGS
#define DGC_BATCH_EXTRA_REGS 16
#endif
template <int MODE, bool MIXED, int STG>
constexpr int batch_regs() {
  return !MIXED ? 255 : surf_regs<3, float, float, float, MODE, STG>() + DGC_BATCH_EXTRA_REGS;
}
template <int MODE, bool MIXED, int STG = -1, int S = 1>
__global__ void __launch_bounds__(256) __maxnreg__((batch_regs<MODE, MIXED, STG>()))
    k_batch_surf(const BatchMeshDev* __restrict__ meshes, const BatchTile* __restrict__ tiles, int nt, int stage,
                 double a0, double b0) {
  static_assert(S == 1 || MIXED, "two lanes per edge side: the FP32-mixed form");
  using CT = typename std::conditional<MIXED, float, double>::type;
  using RT = CT;
  using ST = CT;
  // edge tables of the current order: FP32 in the mode-outer layout, FP64 as
  // [table][point][mode]
  constexpr int TAB = MIXED ? 2 * 3 * ETab32<3>::BLK : kFp64TabWords * 3 * TriDim<3>::NQE * TriDim<3>::NP;
  __shared__ __align__(16) CT sphi[TAB];
  __shared__ CT sw[TriDim<3>::NQE];
  int curp = 0;
  for (int ti = blockIdx.x; ti < nt; ti += gridDim.x) {
    const BatchTile T = tiles[ti];
    if (T.p != curp) {  // block-uniform
      __syncthreads();
      if constexpr (MIXED) {
        if (T.p == 1) stage_etab32<1>(sphi, 3);
        else if (T.p == 2) stage_etab32<2>(sphi, 3);
        else stage_etab32<3>(sphi, 3);
      } else {
        if (T.p == 1) stage_edge_tables<1, CT>(sphi, sw);
        else if (T.p == 2) stage_edge_tables<2, CT>(sphi, sw);
        else stage_edge_tables<3, CT>(sphi, sw);
      }
      __syncthreads();
      curp = T.p;
    }
    const BatchMeshDev& B = meshes[T.mesh];
    SurfParams A;
    A.begin = T.begin;
    A.end = T.end;
    A.topo = B.topo;
    A.fgeo = B.fgeo;
    A.jinv = B.jinv;
    if (MIXED) {
      const int nf = 4 * ((T.p + 1) * (T.p + 2) / 2 + 1);
      A.state = stage == 0 ? B.rec0 : B.recs;
      A.sstride = nf;
      A.sa.u0 = B.c;
      A.sa.uout = B.c;
      A.sa.stage = stage;
      A.sa.rec0 = B.rec0;
      A.sa.rec0_stride = nf;
      A.sa.rec_out = B.recs;
      A.sa.delta = B.delta;
      A.sa.kstate = nullptr;
    } else {
      A.state = stage == 0 ? B.c : B.u1;
      A.sa.u0 = B.c;
      A.sa.uout = stage == 2 ? B.c : B.u1;
      A.sa.a0 = a0;
      A.sa.b0 = b0;
    }
    A.rhs = B.rhs;
    A.buf = nullptr;
    A.ntab = 3;
    A.sa.dt = B.dt;
    int64_t k = T.begin + (threadIdx.x >> (S == 2 ? 2 : 1));
    const bool valid = k < T.end;
    if (!valid) k = T.end - 1;
    const int side = threadIdx.x & 1, sub = S == 2 ? (threadIdx.x >> 1) & 1 : 0;
    const int4 tp = A.topo[k];
    if constexpr (MIXED) {
      if (T.p == 1) surf_fp32<1, ST, RT, MODE, STG, S>(A, k, tp, valid, side, sphi, nullptr, nullptr, sub);
      else if (T.p == 2) surf_fp32<2, ST, RT, MODE, STG, S>(A, k, tp, valid, side, sphi, nullptr, nullptr, sub);
      else surf_fp32<3, ST, RT, MODE, STG, S>(A, k, tp, valid, side, sphi, nullptr, nullptr, sub);
    } else {
      if (T.p == 1) surf_pair<1, CT, ST, RT, MODE>(A, k, tp, valid, side, sphi, sw);
      else if (T.p == 2) surf_pair<2, CT, ST, RT, MODE>(A, k, tp, valid, side, sphi, sw);
      else surf_pair<3, CT, ST, RT, MODE>(A, k, tp, valid, side, sphi, sw);
    }
  }
}

// dt and the FP32 minimum of every mesh set to a large value
__global__ void k_batch_init(const BatchMeshDev* __restrict__ meshes, int n) {
  pdl_wait();
  pdl_trigger();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  *reinterpret_cast<unsigned long long*>(meshes[i].dt) = 0x7F7F7F7F7F7F7F7Full;
  *reinterpret_cast<unsigned*>(meshes[i].est + meshes[i].ne) = 0x7F7F7F7Fu;
}

template <bool MIXED>
__global__ void __launch_bounds__(128) k_batch_cfl1(const BatchMeshDev* __restrict__ meshes,
                                                    const BatchTile* __restrict__ tiles, int nt) {
  pdl_wait();
  pdl_trigger();
  for (int ti = blockIdx.x; ti < nt; ti += gridDim.x) {
    const BatchTile T = tiles[ti];
    const BatchMeshDev& B = meshes[T.mesh];
    const int64_t e = T.begin + threadIdx.x;
    float best = FLT_MAX;
    if (e < T.end) {
      float* sh = MIXED ? B.rec0 : nullptr;
      if (T.p == 1) best = cfl1_elem<1>(B.c, B.inr, e, B.est, sh);
      else if (T.p == 2) best = cfl1_elem<2>(B.c, B.inr, e, B.est, sh);
      else best = cfl1_elem<3>(B.c, B.inr, e, B.est, sh);
    }
    block_min_to(best, reinterpret_cast<unsigned*>(B.est + B.ne));
    __syncthreads();  // the block minimum's shared slots are reused by the next tile
  }
}

__global__ void __launch_bounds__(128) k_batch_cfl2(const BatchMeshDev* __restrict__ meshes,
                                                    const BatchTile* __restrict__ tiles, int nt, double cfl) {
  pdl_wait();
  pdl_trigger();
  for (int ti = blockIdx.x; ti < nt; ti += gridDim.x) {
    const BatchTile T = tiles[ti];
    const BatchMeshDev& B = meshes[T.mesh];
    const int64_t e = T.begin + threadIdx.x < T.end ? T.begin + threadIdx.x : -1;
    const float mn = __uint_as_float(*reinterpret_cast<const unsigned*>(B.est + B.ne));
    double best;
    if (T.p == 1) best = cfl2_warp<1, false>(B.c, B.inr, e, cfl, B.est, mn);
    else if (T.p == 2) best = cfl2_warp<2, false>(B.c, B.inr, e, cfl, B.est, mn);
    else best = cfl2_warp<3, false>(B.c, B.inr, e, cfl, B.est, mn);
    block_min_to(best, reinterpret_cast<unsigned long long*>(B.dt));
    __syncthreads();
  }
}

// The batched step's kernels launch with programmatic dependent launch (the
// surface kernels wait before their epilogues, the others at once); captured
// into the step's CUDA graph they become programmatic edges.
static Ctx pdl_ctx(cudaStream_t st) {
  Ctx x;
  x.st = st;
  x.pdl = true;
  return x;
}

static int persistent_grid(const void* kern, int threads, int ntiles) {
  int dev = 0, sms = 0, per = 1;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kern, threads, 0);
  const int g = sms * (per > 0 ? per : 1);
  return ntiles < g ? (ntiles > 0 ? ntiles : 1) : g;
}

int batch_init(cudaStream_t st, const BatchMeshDev* d, int n) {
  launch_k(pdl_ctx(st), k_batch_init, (unsigned)((n + 127) / 128), 128u, 0, d, n);
  return 1;
}

int batch_cfl(cudaStream_t st, const BatchMeshDev* d, const BatchTile* tiles, int nt, double cfl, bool mixed) {
  if (nt <= 0) return 0;
  const void* k1 = mixed ? (const void*)k_batch_cfl1<true> : (const void*)k_batch_cfl1<false>;
  const int g1 = persistent_grid(k1, 128, nt), g2 = persistent_grid((const void*)k_batch_cfl2, 128, nt);
  if (mixed) launch_k(pdl_ctx(st), k_batch_cfl1<true>, (unsigned)g1, 128u, 0, d, tiles, nt);
  else launch_k(pdl_ctx(st), k_batch_cfl1<false>, (unsigned)g1, 128u, 0, d, tiles, nt);
  launch_k(pdl_ctx(st), k_batch_cfl2, (unsigned)g2, 128u, 0, d, tiles, nt, cfl);
  return 2;
}

template <int MODE, bool MIXED, int STG = -1, int S = 1>
static int batch_surf_launch(cudaStream_t st, const BatchMeshDev* d, const BatchTile* tiles, int nt, int stage,
                             double a0, double b0, int threads) {
  if (nt <= 0) return 0;
  if (threads > 256) return -1;
  const int g = persistent_grid((const void*)k_batch_surf<MODE, MIXED, STG, S>, threads, nt);
  launch_k(pdl_ctx(st), k_batch_surf<MODE, MIXED, STG, S>, (unsigned)g, (unsigned)threads, 0, d, tiles, nt, stage,
           a0, b0);
  return 1;
}

template <int MODE, int STG = -1>
static int batch_mixed(cudaStream_t st, const BatchMeshDev* d, const BatchTile* tiles, int nt, int stage, double a0,
                       double b0, int threads, int tpe) {
  if (tpe == 4) return batch_surf_launch<MODE, true, STG, 2>(st, d, tiles, nt, stage, a0, b0, threads);
  return batch_surf_launch<MODE, true, STG, 1>(st, d, tiles, nt, stage, a0, b0, threads);
}

int batch_surf(cudaStream_t st, const BatchMeshDev* d, const BatchTile* tiles, int nt, int stage, double a0,
               double b0, SurfMode mode, bool mixed, int threads, int tpe) {
  if (mixed) {
    if (mode == SURF_FIRST) return batch_mixed<SURF_FIRST>(st, d, tiles, nt, stage, a0, b0, threads, tpe);
    if (mode == SURF_RMW) return batch_mixed<SURF_RMW>(st, d, tiles, nt, stage, a0, b0, threads, tpe);
    if (mode == SURF_LAST) {  // the batch runs the mixed form only: stage 2 updates the FP64 state
      if (stage == 0) return batch_mixed<SURF_LAST, 0>(st, d, tiles, nt, stage, a0, b0, threads, tpe);
      if (stage == 1) return batch_mixed<SURF_LAST, 1>(st, d, tiles, nt, stage, a0, b0, threads, tpe);
      return batch_mixed<SURF_LAST, 2>(st, d, tiles, nt, stage, a0, b0, threads, tpe);
    }
  } else {
    if (tpe != 2) return -1;
    if (mode == SURF_FIRST) return batch_surf_launch<SURF_FIRST, false>(st, d, tiles, nt, stage, a0, b0, threads);
    if (mode == SURF_RMW) return batch_surf_launch<SURF_RMW, false>(st, d, tiles, nt, stage, a0, b0, threads);
    if (mode == SURF_LAST) return batch_surf_launch<SURF_LAST, false>(st, d, tiles, nt, stage, a0, b0, threads);
  }
  return -1;
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
template <int P, typename CT, typename ST, typename RT>
static int vol_p(const Ctx& x, const void* s, int sstride, void* r, int64_t e0) {
  const int bs = 128;
  const int64_t n = x.ne - e0;
  if (n <= 0) return 0;
  k_vol_tri<P, CT, ST, RT><<<(unsigned)((n + bs - 1) / bs), bs, 0, x.st>>>(static_cast<const ST*>(s), sstride,
                                                                          x.d->jinv, static_cast<RT*>(r), e0, x.ne);
  return 1;
}

template <int P>
static int vol_ty(const Ctx& x, TypeCfg ty, const void* s, int ss, void* r, int64_t e0) {
  switch (ty) {
    case TY_D: return vol_p<P, double, double, double>(x, s, ss, r, e0);
    case TY_MD: return vol_p<P, float, double, double>(x, s, ss, r, e0);
    case TY_MF: return vol_p<P, float, float, float>(x, s, ss, r, e0);
    case TY_KD: return vol_p<P, float, float, double>(x, s, ss, r, e0);
    default: return -1;
  }
}

int tri_volume(const Ctx& x, TypeCfg ty, const void* s, int sstride, void* r, int64_t e0) {
  switch (x.p) {
    case 1: return vol_ty<1>(x, ty, s, sstride, r, e0);
    case 2: return vol_ty<2>(x, ty, s, sstride, r, e0);
    case 3: return vol_ty<3>(x, ty, s, sstride, r, e0);
    default: return -1;
  }
}

// the tile class of a surface mode: first, middle, last color (comparators: middle)
constexpr int tile_class(int mode) { return mode == SURF_FIRST ? 0 : mode == SURF_LAST ? 2 : 1; }

template <int P, typename CT, typename ST, typename RT, int MODE, int STG = -1, int S = 1, bool BC = false>
static int surf_launch_s(const Ctx& x, const SurfParams& A) {
  const int64_t n = A.end - A.begin;
  if (n <= 0) return 0;
  const int threads = 2 * S * x.tile_epb[tile_class(MODE)];
  if (threads > 256) return -1;  // the kernels' launch bound
  int64_t grid = (2 * S * n + threads - 1) / threads;
  const size_t smem =
      MODE == SURF_LAST && STG == 0 && sizeof(ST) == 4 ? (size_t)threads * rec_slot<P>() * sizeof(float) : 0;
  SurfParams B = A;
  B.persistent = 0;
  if (x.persistent) {
    // one wave: resident blocks per SM of this instantiation at this block size
    static int per = -1, per_threads = -1;
    if (per_threads != threads) {
      int occ = 0;
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_surf_tri<P, CT, ST, RT, MODE, STG, S, BC>, threads, smem);
      per = occ > 0 ? occ : 1;
      per_threads = threads;
    }
    const int64_t wave = (int64_t)x.sms * per;
    if (grid > wave) {
      grid = wave;
      B.persistent = 1;
    }
  }
  if (smem > 32 * 1024) {  // 256-thread blocks: above the default 48 KB with the static tables
    static bool raised = false;
    if (!raised) {
      cudaFuncSetAttribute(k_surf_tri<P, CT, ST, RT, MODE, STG, S, BC>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           64 * 1024);
      raised = true;
    }
  }
  launch_k(x, k_surf_tri<P, CT, ST, RT, MODE, STG, S, BC>, (unsigned)grid, (unsigned)threads, smem, B);
  return 1;
}

// The FP32 colored kernels of an RK step (FP32 rhs) take their class's threads
// per edge (2 or 4); every other kernel has one lane per edge side.
template <int P, typename CT, typename ST, typename RT, int MODE, int STG = -1>
static int surf_launch(const Ctx& x, const SurfParams& A) {
  // boundary conditions on the FP32 lanes: their instantiation, one lane per side
  if constexpr (sizeof(CT) == 4)
    if (A.bc) return surf_launch_s<P, CT, ST, RT, MODE, STG, 1, true>(x, A);
  if constexpr (sizeof(CT) == 4 && sizeof(RT) == 4) {
    if (x.tile_tpe[tile_class(MODE)] == 4) return surf_launch_s<P, CT, ST, RT, MODE, STG, 2>(x, A);
  }
  return surf_launch_s<P, CT, ST, RT, MODE, STG, 1>(x, A);
}

template <int P, typename CT, typename ST, typename RT>
static int surf_mode(const Ctx& x, SurfMode mode, const SurfParams& A) {
  switch (mode) {
    case SURF_RMW: return surf_launch<P, CT, ST, RT, SURF_RMW>(x, A);
    case SURF_FIRST: return surf_launch<P, CT, ST, RT, SURF_FIRST>(x, A);
    case SURF_ATOMIC: return surf_launch<P, CT, ST, RT, SURF_ATOMIC>(x, A);
    case SURF_BUFFER: return surf_launch<P, CT, ST, RT, SURF_BUFFER>(x, A);
    default: return -1;
  }
}

template <int P>
static int surf_p(const Ctx& x, TypeCfg ty, SurfMode mode, const SurfParams& A) {
  if (mode == SURF_LAST) {
    if (ty == TY_D) return surf_launch<P, double, double, double, SURF_LAST>(x, A);
    if (ty == TY_MF) {  // one kernel per stage of the increment form (3: stage 2 of the Kahan form)
      if (A.sa.stage == 0) return surf_launch<P, float, float, float, SURF_LAST, 0>(x, A);
      if (A.sa.stage == 1) return surf_launch<P, float, float, float, SURF_LAST, 1>(x, A);
      if (A.sa.kstate) return surf_launch<P, float, float, float, SURF_LAST, 3>(x, A);
      return surf_launch<P, float, float, float, SURF_LAST, 2>(x, A);
    }
    return -1;
  }
  switch (ty) {
    case TY_D: return surf_mode<P, double, double, double>(x, mode, A);
    case TY_MD: return surf_mode<P, float, double, double>(x, mode, A);
    case TY_MF:
      if (mode == SURF_RMW) return surf_launch<P, float, float, float, SURF_RMW>(x, A);
      if (mode == SURF_FIRST) return surf_launch<P, float, float, float, SURF_FIRST>(x, A);
      return -1;
    case TY_KD:
      if (mode == SURF_RMW) return surf_launch<P, float, float, double, SURF_RMW>(x, A);
      if (mode == SURF_FIRST) return surf_launch<P, float, float, double, SURF_FIRST>(x, A);
      return -1;
    default: return -1;
  }
}

int tri_surface(const Ctx& x, TypeCfg ty, SurfMode mode, int64_t begin, int64_t end, const void* state,
                int sstride, void* rhs, void* buf, const StageArgs* sa) {
  SurfParams A;
  A.begin = begin;
  A.end = end;
  A.sstride = sstride;
  A.topo = x.d->topo;
  A.fgeo = x.d->fgeo;
  A.jinv = x.d->jinv;
  A.state = state;
  A.rhs = rhs;
  A.buf = buf;
  A.ntab = x.d->edge_tables;
  if (sa) A.sa = *sa;
  A.bc = x.d->bc;
  A.bgeo = x.d->bgeo;
  A.t0 = x.d->time;
  A.dtp = x.dtp;
  A.tfrac = x.tfrac;
  switch (x.p) {
    case 1: return surf_p<1>(x, ty, mode, A);
    case 2: return surf_p<2>(x, ty, mode, A);
    case 3: return surf_p<3>(x, ty, mode, A);
    default: return -1;
  }
}

// ---------------------------------------------------------------------------
// The whole right-hand side in one cooperative launch (dgc_rhs with
// DGC_OPT_COOPERATIVE): the phases of Algorithm 1 -- the first color with the
// volume integral of the elements it reaches and the volume integral of the
// rest (disjoint elements, one phase), then every further color -- separated
// by grid-wide barriers instead of kernel boundaries.  The grid is co-resident
// (cudaLaunchCooperativeKernel refuses one that is not); each warp takes
// chunks of 16 edges (or 32 elements) in a grid-stride loop, so a color with
// fewer edges than the GPU holds threads spreads over every SM.  Per element
// the arithmetic and its order are those of the separate launches.
// ---------------------------------------------------------------------------
struct CoopRhs {
  SurfParams A;
  int off[kMaxColors + 1];  // color offsets of the edges
  int ncolors;
  int fused;      // the first color stores rhs with the volume integral of [0, e_vol0)
  int64_t e_vol0;  // the volume phase covers [e_vol0, ne)
  int64_t ne;
};

template <int P, typename CT, typename ST, typename RT, int MODE>
__device__ __forceinline__ void coop_edges(const SurfParams& A, int64_t begin, int64_t end, const CT* tab,
                                           const CT* sw) {
  const int lane = threadIdx.x & 31;
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  const int64_t wid = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int side = lane & 1;
  for (int64_t ch = wid; begin + 16 * ch < end; ch += warps) {  // warp-uniform trip count
    int64_t k = begin + 16 * ch + (lane >> 1);
    const bool valid = k < end;
    if (!valid) k = end - 1;
    const int4 tp = A.topo[k];
    if constexpr (sizeof(CT) == 4) surf_fp32<P, ST, RT, MODE>(A, k, tp, valid, side, tab);
    else surf_pair<P, CT, ST, RT, MODE>(A, k, tp, valid, side, tab, sw);
  }
}

template <int P, typename CT, typename ST, typename RT>
__global__ void __launch_bounds__(128) __maxnreg__((sizeof(CT) == 8 ? 255 : surf_regs<P, CT, ST, RT, SURF_FIRST, -1>()))
    k_rhs_coop(const CoopRhs C) {
  using D = TriDim<P>;
  namespace cg = cooperative_groups;
  cg::grid_group grid = cg::this_grid();
  constexpr int TAB = sizeof(CT) == 4 ? ETab32<P>::SIZE : kFp64TabWords * 9 * D::NQE * D::NP;
  __shared__ __align__(16) CT tab[TAB];
  __shared__ CT sw[D::NQE];
  if constexpr (sizeof(CT) == 4) stage_etab32<P>(reinterpret_cast<float*>(tab), C.A.ntab);
  else stage_edge_tables<P, double>(reinterpret_cast<double*>(tab), reinterpret_cast<double*>(sw), C.A.ntab);
  __syncthreads();
  const SurfParams& A = C.A;
  // phase 0: the first color (fused) and the volume integral of the others
  if (C.fused) coop_edges<P, CT, ST, RT, SURF_FIRST>(A, C.off[0], C.off[1], tab, sw);
  for (int64_t e = C.e_vol0 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < C.ne;
       e += (int64_t)gridDim.x * blockDim.x)
    vol_elem<P, CT, ST, RT>(static_cast<const ST*>(A.state), A.sstride, A.jinv, static_cast<RT*>(A.rhs), e);
  for (int c = C.fused ? 2 : 1; c <= C.ncolors; ++c) {
    __threadfence();
    grid.sync();
    coop_edges<P, CT, ST, RT, SURF_RMW>(A, C.off[c - 1], C.off[c], tab, sw);
  }
}

template <int P, typename CT, typename ST, typename RT>
static int rhs_coop_launch(const Ctx& x, const CoopRhs& C) {
  static int grid = 0;  // co-resident blocks of this kernel (per instantiation; one device model)
  if (!grid) {
    int dev = 0, sms = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_rhs_coop<P, CT, ST, RT>, 128, 0);
    if (per <= 0) return -1;
    grid = sms * per;
  }
  void* args[] = {const_cast<CoopRhs*>(&C)};
  if (cudaLaunchCooperativeKernel((const void*)k_rhs_coop<P, CT, ST, RT>, dim3(grid), dim3(128), args, 0, x.st) !=
      cudaSuccess)
    return -1;
  return 1;
}

int tri_rhs_coop(const Ctx& x, TypeCfg ty, const int* off, int ncolors, bool fused, int64_t e_vol0,
                 const void* state, void* rhs) {
  if (ncolors > kMaxColors) return -1;
  CoopRhs C;
  C.A.begin = 0;
  C.A.end = 0;
  C.A.sstride = 0;
  C.A.topo = x.d->topo;
  C.A.fgeo = x.d->fgeo;
  C.A.jinv = x.d->jinv;
  C.A.state = state;
  C.A.rhs = rhs;
  C.A.buf = nullptr;
  C.A.ntab = x.d->edge_tables;
  for (int c = 0; c <= ncolors; ++c) C.off[c] = off[c];
  C.ncolors = ncolors;
  C.fused = fused ? 1 : 0;
  C.e_vol0 = fused ? e_vol0 : 0;
  C.ne = x.ne;
  if (ty != TY_D && ty != TY_MD) return -1;
  switch (x.p) {
    case 1: return ty == TY_D ? rhs_coop_launch<1, double, double, double>(x, C)
                              : rhs_coop_launch<1, float, double, double>(x, C);
    case 2: return ty == TY_D ? rhs_coop_launch<2, double, double, double>(x, C)
                              : rhs_coop_launch<2, float, double, double>(x, C);
    case 3: return ty == TY_D ? rhs_coop_launch<3, double, double, double>(x, C)
                              : rhs_coop_launch<3, float, double, double>(x, C);
    default: return -1;
  }
}

// Stage 0 of the mixed step on a mesh where every element has one edge of each
// color: the first color (edges [begin, end)) reads the FP64 state c and, with
// the volume integral and its edge, writes each element's record of u0 (rec0)
// and FP32 CFL estimate, the work of pass 1 of the CFL reduction (the estimate
// comes from the volume integral's own point values).  tri_cfl_pass2 then
// finishes dt before the next color.
int tri_first_est(const Ctx& x, int64_t begin, int64_t end, const double* c, float* rec0, float* rhs) {
  unsigned* mn = reinterpret_cast<unsigned*>(x.d->cfl_est + x.ne);
  if (cudaMemsetAsync(mn, 0x7F, sizeof(unsigned), x.st) != cudaSuccess) return -1;
  SurfParams A;
  A.begin = begin;
  A.end = end;
  A.sstride = 0;
  A.topo = x.d->topo;
  A.fgeo = x.d->fgeo;
  A.jinv = x.d->jinv;
  A.state = c;
  A.rhs = rhs;
  A.buf = nullptr;
  A.ntab = x.d->edge_tables;
  A.rec_first = rec0;
  A.est = x.d->cfl_est;
  A.estmin = mn;
  A.inr = x.d->inr;
  A.bc = x.d->bc;
  A.bgeo = x.d->bgeo;
  A.t0 = x.d->time;
  A.dtp = x.dtp;
  A.tfrac = x.tfrac;
  switch (x.p) {
    case 1: return surf_launch<1, float, double, float, SURF_FIRST, 0>(x, A);
    case 2: return surf_launch<2, float, double, float, SURF_FIRST, 0>(x, A);
    case 3: return surf_launch<3, float, double, float, SURF_FIRST, 0>(x, A);
    default: return -1;
  }
}

int tri_cfl_pass2(const Ctx& x, const double* s, double cfl, double* dt) {
  const int bs = 128;
  const unsigned grid = (unsigned)((x.ne + bs - 1) / bs);
  auto* bits = reinterpret_cast<unsigned long long*>(dt);
  const float* est = x.d->cfl_est;
  const unsigned* mn = reinterpret_cast<const unsigned*>(x.d->cfl_est + x.ne);
  switch (x.p) {
    case 1: launch_k(x, k_cfl2_tri<1, false>, grid, bs, 0, s, x.d->inr, x.ne, cfl, est, mn, bits); return 1;
    case 2: launch_k(x, k_cfl2_tri<2, false>, grid, bs, 0, s, x.d->inr, x.ne, cfl, est, mn, bits); return 1;
    case 3: launch_k(x, k_cfl2_tri<3, false>, grid, bs, 0, s, x.d->inr, x.ne, cfl, est, mn, bits); return 1;
    default: return -1;
  }
}

int tri_cfl(const Ctx& x, const double* s, double cfl, double* dt, float* shadow) {
  const int bs = 128;
  const unsigned grid = (unsigned)((x.ne + bs - 1) / bs);
  auto* bits = reinterpret_cast<unsigned long long*>(dt);
  float* est = x.d->cfl_est;
  unsigned* mn = reinterpret_cast<unsigned*>(x.d->cfl_est + x.ne);
  if (cudaMemsetAsync(mn, 0x7F, sizeof(unsigned), x.st) != cudaSuccess) return -1;
  switch (x.p) {
    case 1:
      launch_k(x, k_cfl1_tri<1>, grid, bs, 0, s, x.d->inr, x.ne, est, mn, shadow);
      launch_k(x, k_cfl2_tri<1, false>, grid, bs, 0, s, x.d->inr, x.ne, cfl, est, mn, bits);
      return 2;
    case 2:
      launch_k(x, k_cfl1_tri<2>, grid, bs, 0, s, x.d->inr, x.ne, est, mn, shadow);
      launch_k(x, k_cfl2_tri<2, false>, grid, bs, 0, s, x.d->inr, x.ne, cfl, est, mn, bits);
      return 2;
    case 3:
      launch_k(x, k_cfl1_tri<3>, grid, bs, 0, s, x.d->inr, x.ne, est, mn, shadow);
      launch_k(x, k_cfl2_tri<3, false>, grid, bs, 0, s, x.d->inr, x.ne, cfl, est, mn, bits);
      return 2;
    default: return -1;
  }
}

// ---------------------------------------------------------------------------
// Limiter (after each RK stage of a limited step, or dgc_limit): the
// Barth-Jespersen limiter on the conserved variables, one thread per element,
// FP64.  Per variable: the element's mean u_e (mode 0 times phi_0) and the
// least and greatest of it and its face neighbours' means bound the deviations
// d_i = sum_{j>=1} c_j phi_j(x_i) at the element's vertices and volume points;
// alpha = min(1, (u_max - u_e) / d_i for d_i > 0, (u_min - u_e) / d_i for
// d_i < 0), and the modes j >= 1 are multiplied by alpha.  A thread writes
// only its element's modes j >= 1 and reads only its neighbours' mode 0, so
// the elements are independent and the state is limited in place.
// ---------------------------------------------------------------------------
template <int P>
__global__ void __launch_bounds__(128) k_limit_tri(double* c, const int4* __restrict__ enb, int64_t ne) {
  using D = TriDim<P>;
  constexpr int NP = D::NP, NV = D::NV;
  const TriTab<double, P>& K = tri_tab<double, P>();
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= ne) return;
  double v[NV];
  load_plain(c + e * NV, v);
  const int4 nb = enb[e];
  const int nbs[3] = {nb.x, nb.y, nb.z};
  const double phi0 = K.phiX[0][0];
#pragma unroll
  for (int m = 0; m < 4; ++m) {
    const double ue = v[m * NP] * phi0;
    double lo = ue, hi = ue;
#pragma unroll
    for (int f = 0; f < 3; ++f)
      if (nbs[f] >= 0) {
        const double u = c[(int64_t)nbs[f] * NV + m * NP] * phi0;
        lo = fmin(lo, u);
        hi = fmax(hi, u);
      }
    // the least ratio over the points is the one at the largest deviation of
    // each sign (a correctly rounded quotient is monotone in its divisor, so
    // this is the same number as the least of the per-point quotients)
    double dmax = 0.0, dmin = 0.0;
    for (int i = 0; i < 3 + D::NQV; ++i) {
      const double* ph = i < 3 ? K.phiX[i] : K.phiV[i - 3];
      double d = 0.0;
#pragma unroll
      for (int j = 1; j < NP; ++j) d += v[m * NP + j] * ph[j];
      dmax = fmax(dmax, d);
      dmin = fmin(dmin, d);
    }
    double alpha = 1.0;
    if (dmax > 0.0) alpha = fmin(alpha, (hi - ue) / dmax);
    if (dmin < 0.0) alpha = fmin(alpha, (lo - ue) / dmin);
#pragma unroll
    for (int j = 1; j < NP; ++j) v[m * NP + j] *= alpha;
  }
  double* dst = c + e * NV;
#pragma unroll
  for (int i = 0; i < NV; ++i)
    if (i % NP) dst[i] = v[i];
}

int tri_limit(const Ctx& x, double* c) {
  if (x.ne <= 0) return 0;
  if (!x.d->enb) return -1;
  const unsigned grid = (unsigned)((x.ne + 127) / 128);
  switch (x.p) {
    case 1: k_limit_tri<1><<<grid, 128, 0, x.st>>>(c, x.d->enb, x.ne); return 1;
    case 2: k_limit_tri<2><<<grid, 128, 0, x.st>>>(c, x.d->enb, x.ne); return 1;
    case 3: k_limit_tri<3><<<grid, 128, 0, x.st>>>(c, x.d->enb, x.ne); return 1;
    default: return -1;
  }
}

// the mesh's time advanced by the step's dt, on the device (one thread)
__global__ void k_time_advance(double* t, const double* dt) { *t += *dt; }

int time_advance(const Ctx& x, const double* dt) {
  if (!x.d->time) return 0;
  k_time_advance<<<1, 1, 0, x.st>>>(x.d->time, dt);
  return 1;
}

}  // namespace dgc
