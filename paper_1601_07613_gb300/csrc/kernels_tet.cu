// Tetrahedral kernels: the 3D form of the colored surface integral (faces
// colored with 4 colors, Sec. 3), the volume integral and the FP64 CFL
// reduction.  Same structure as the triangle kernels: a lane pair per face,
// one lane per neighbouring element, traces exchanged by shuffles, plain
// read-modify-write stores within a color.  The collapsed face rule is not
// symmetric under a permutation of the face's vertices, so the right element
// evaluates its basis through one of six orientation tables (the face's
// vertex permutation is stored per face).  FP64 kernels evaluate Eq. 2 as
// written, FP32 kernels in the perturbation form of euler_pert.cuh.
#include <algorithm>
#include <cfloat>
#include <cmath>

#include "dev_util.cuh"
#include "device.cuh"
#include "euler_pert.cuh"
#include "incr_form.cuh"

namespace dgc {

template <int P>
struct TetDim {
  static constexpr int NP = (P + 1) * (P + 2) * (P + 3) / 6;
  static constexpr int NQV = (P + 2) * (P + 2) * (P + 2);
  static constexpr int NQF = (P + 2) * (P + 2);
  static constexpr int KF = (P + 1) * (P + 2) / 2;  // polynomials of degree P on a face
  static constexpr int M = 5;
  static constexpr int NV = M * NP;
  // FP32 record: hi[M], lo[M], modes j >= 1 as [M][NP-1], padded to 4 floats
  static constexpr int NF = (M * (NP + 1) + 3) / 4 * 4;
};

int tet_record_floats(int p) {
  const int np = (p + 1) * (p + 2) * (p + 3) / 6;
  return (5 * (np + 1) + 3) / 4 * 4;
}

template <typename T, int P>
struct TetTab {
  T phiV[TetDim<P>::NQV][TetDim<P>::NP];
  T vr[TetDim<P>::NQV][TetDim<P>::NP];  // w_q dphi/dr
  T vs[TetDim<P>::NQV][TetDim<P>::NP];
  T vt[TetDim<P>::NQV][TetDim<P>::NP];
  T wF[TetDim<P>::NQF];                 // face weights, sum 1
};

// the FP64 tables the kernels read: the basis at the volume points (the CFL
// pass, phi_0) and the face weights (the FP64 volume integrals take their
// tables as FP32 pairs in shared memory)
template <int P>
struct TetTabD {
  double phiV[TetDim<P>::NQV][TetDim<P>::NP];
  double wF[TetDim<P>::NQF];
};
__constant__ TetTabD<1> cTetD1;
__constant__ TetTabD<2> cTetD2;
__constant__ TetTab<float, 1> cTetF1;
__constant__ TetTab<float, 2> cTetF2;

template <typename T, int P>
__device__ __forceinline__ const TetTab<T, P>& tet_tab();
template <int P>
__device__ __forceinline__ const TetTabD<P>& tet_tabd();
template <> __device__ __forceinline__ const TetTabD<1>& tet_tabd<1>() { return cTetD1; }
template <> __device__ __forceinline__ const TetTabD<2>& tet_tabd<2>() { return cTetD2; }
template <> __device__ __forceinline__ const TetTab<float, 1>& tet_tab<float, 1>() { return cTetF1; }
template <> __device__ __forceinline__ const TetTab<float, 2>& tet_tab<float, 2>() { return cTetF2; }

template <typename T, int P>
static void fill_tet(TetTab<T, P>& K, const RefTables& R) {
  using D = TetDim<P>;
  for (int q = 0; q < D::NQV; ++q)
    for (int j = 0; j < D::NP; ++j) {
      K.phiV[q][j] = (T)R.phiV[q * D::NP + j];
      K.vr[q][j] = (T)(R.vw[q] * R.dphiV[(0 * D::NQV + q) * D::NP + j]);
      K.vs[q][j] = (T)(R.vw[q] * R.dphiV[(1 * D::NQV + q) * D::NP + j]);
      K.vt[q][j] = (T)(R.vw[q] * R.dphiV[(2 * D::NQV + q) * D::NP + j]);
    }
  for (int q = 0; q < D::NQF; ++q) K.wF[q] = (T)R.fw[q];
}

template <int P>
static void upload_tet_p(const RefTables& R, const void* symD, const void* symF) {
  static TetTabD<P> hd;
  static TetTab<float, P> hf;
  for (int q = 0; q < TetDim<P>::NQV; ++q)
    for (int j = 0; j < TetDim<P>::NP; ++j) hd.phiV[q][j] = R.phiV[q * TetDim<P>::NP + j];
  for (int q = 0; q < TetDim<P>::NQF; ++q) hd.wF[q] = R.fw[q];
  fill_tet(hf, R);
  cudaMemcpyToSymbol(symD, &hd, sizeof hd);
  cudaMemcpyToSymbol(symF, &hf, sizeof hf);
}

// The FP32 volume tables with every entry twice, (v, v): the operand of a packed
// two-lane FP32 FMA (__ffma2_rn, one instruction for two variables).
template <int P>
struct TetPairTab {
  float2 phiV[TetDim<P>::NQV][TetDim<P>::NP];
  float2 vr[TetDim<P>::NQV][TetDim<P>::NP];
  float2 vs[TetDim<P>::NQV][TetDim<P>::NP];
  float2 vt[TetDim<P>::NQV][TetDim<P>::NP];
};
__constant__ TetPairTab<1> cTetP1;
__constant__ TetPairTab<2> cTetP2;
template <int P>
__device__ __forceinline__ const TetPairTab<P>& tet_ptab();
template <> __device__ __forceinline__ const TetPairTab<1>& tet_ptab<1>() { return cTetP1; }
template <> __device__ __forceinline__ const TetPairTab<2>& tet_ptab<2>() { return cTetP2; }

// Variable 4 of the volume integral on the packed FMA too: its modes in pairs
// (1, 2), (3, 4), ...; the tables hold (t_j, t_j+1) (0 past the last mode).
template <int P>
struct TetModePairTab {
  static constexpr int NH = TetDim<P>::NP / 2;  // pairs of the modes 1..NP-1
  float2 phiV[TetDim<P>::NQV][NH];
  float2 vr[TetDim<P>::NQV][NH];
  float2 vs[TetDim<P>::NQV][NH];
  float2 vt[TetDim<P>::NQV][NH];
};
__constant__ TetModePairTab<1> cTetQ1;
__constant__ TetModePairTab<2> cTetQ2;
template <int P>
__device__ __forceinline__ const TetModePairTab<P>& tet_qtab();
template <> __device__ __forceinline__ const TetModePairTab<1>& tet_qtab<1>() { return cTetQ1; }
template <> __device__ __forceinline__ const TetModePairTab<2>& tet_qtab<2>() { return cTetQ2; }

template <int P>
static void upload_tet_mode_pairs(const RefTables& R, const void* sym) {
  using D = TetDim<P>;
  static TetTab<float, P> f;
  static TetModePairTab<P> h;
  fill_tet(f, R);
  auto at = [](const float (&t)[D::NQV][D::NP], int q, int j) { return j < D::NP ? t[q][j] : 0.0f; };
  for (int q = 0; q < D::NQV; ++q)
    for (int k = 0; k < TetModePairTab<P>::NH; ++k) {
      const int j = 1 + 2 * k;
      h.phiV[q][k] = make_float2(at(f.phiV, q, j), at(f.phiV, q, j + 1));
      h.vr[q][k] = make_float2(at(f.vr, q, j), at(f.vr, q, j + 1));
      h.vs[q][k] = make_float2(at(f.vs, q, j), at(f.vs, q, j + 1));
      h.vt[q][k] = make_float2(at(f.vt, q, j), at(f.vt, q, j + 1));
    }
  cudaMemcpyToSymbol(sym, &h, sizeof h);
}

template <int P>
static void upload_tet_pairs(const RefTables& R, const void* sym) {
  static TetTab<float, P> f;
  static TetPairTab<P> h;
  fill_tet(f, R);
  for (int q = 0; q < TetDim<P>::NQV; ++q)
    for (int j = 0; j < TetDim<P>::NP; ++j) {
      h.phiV[q][j] = make_float2(f.phiV[q][j], f.phiV[q][j]);
      h.vr[q][j] = make_float2(f.vr[q][j], f.vr[q][j]);
      h.vs[q][j] = make_float2(f.vs[q][j], f.vs[q][j]);
      h.vt[q][j] = make_float2(f.vt[q][j], f.vt[q][j]);
    }
  cudaMemcpyToSymbol(sym, &h, sizeof h);
}

// Face-modal traces of the FP32 lanes.  The traces of the element's basis on a
// face span the polynomials of degree p on that face.  psi_k (k < KF) is a
// basis of that space orthonormal under the face rule (Gram-Schmidt on the
// traces through local face 0 at the face points); the trace of phi_j seen
// through local face f and orientation o is then sum_k T[f][o][k][j] psi_k, with
// T = sum_q w_q psi_k(q) phi_j(q), exactly at the face points (the rule
// integrates degree 2p exactly).  So a lane evaluates its trace from KF face
// coefficients a_k = sum_j T[k][j] c_j, projects its flux onto the psi_k, and
// maps the KF projections back to its modes with T's transpose.
template <int P>
struct TetFaceTab {
  float psi[TetDim<P>::NQF][TetDim<P>::KF];
  float2 psi2[TetDim<P>::NQF][TetDim<P>::KF];  // (psi, psi) for the packed FMA
};
__constant__ TetFaceTab<1> cTetM1;
__constant__ TetFaceTab<2> cTetM2;
template <int P>
__device__ __forceinline__ const TetFaceTab<P>& tet_mtab();
template <> __device__ __forceinline__ const TetFaceTab<1>& tet_mtab<1>() { return cTetM1; }
template <> __device__ __forceinline__ const TetFaceTab<2>& tet_mtab<2>() { return cTetM2; }

// psi [NQF][KF] and T [4][6][KF][NP] from the orientation tables t [4][6][NQF][NP]
static void tet_face_modal(const std::vector<double>& t, const RefTables& R, std::vector<double>& psi,
                           std::vector<double>& T) {
  const int nq = R.nqf, np = R.np, kf = (R.p + 1) * (R.p + 2) / 2;
  auto dot = [&](const double* f, const double* g) {
    double v = 0.0;
    for (int q = 0; q < nq; ++q) v += R.fw[q] * f[q] * g[q];
    return v;
  };
  std::vector<double> basis;  // [k][q]
  std::vector<double> v(nq);
  for (int j = 0; j < np && (int)(basis.size() / nq) < kf; ++j) {
    for (int q = 0; q < nq; ++q) v[q] = t[(size_t)q * np + j];
    const double n0 = std::sqrt(dot(v.data(), v.data()));
    for (int pass = 0; pass < 2; ++pass)
      for (size_t k = 0; k < basis.size() / nq; ++k) {
        const double c = dot(v.data(), basis.data() + k * nq);
        for (int q = 0; q < nq; ++q) v[q] -= c * basis[k * nq + q];
      }
    const double n1 = std::sqrt(dot(v.data(), v.data()));
    if (n1 > 1e-8 * n0)
      for (int q = 0; q < nq; ++q) basis.push_back(v[q] / n1);
  }
  if ((int)(basis.size() / nq) != kf) throw Error{DGC_ERR_UNSUPPORTED, "face-modal basis: wrong rank (internal)"};
  psi.assign((size_t)nq * kf, 0.0);
  for (int q = 0; q < nq; ++q)
    for (int k = 0; k < kf; ++k) psi[(size_t)q * kf + k] = basis[(size_t)k * nq + q];
  T.assign((size_t)24 * kf * np, 0.0);
  for (int fo = 0; fo < 24; ++fo)
    for (int j = 0; j < np; ++j) {
      const double* ph = t.data() + (size_t)fo * nq * np;
      for (int q = 0; q < nq; ++q) v[q] = ph[(size_t)q * np + j];
      double err = 0.0, mx = 0.0;
      for (int k = 0; k < kf; ++k) T[((size_t)fo * kf + k) * np + j] = dot(basis.data() + (size_t)k * nq, v.data());
      for (int q = 0; q < nq; ++q) {
        double r = v[q];
        for (int k = 0; k < kf; ++k) r -= T[((size_t)fo * kf + k) * np + j] * psi[(size_t)q * kf + k];
        err = std::max(err, std::fabs(r));
        mx = std::max(mx, std::fabs(v[q]));
      }
      if (err > 1e-11 * (1.0 + mx)) throw Error{DGC_ERR_UNSUPPORTED, "face-modal traces: not exact at the face points (internal)"};
    }
}

template <int P>
static void upload_tet_modal(const std::vector<double>& psi, const void* sym) {
  static TetFaceTab<P> h;
  for (int q = 0; q < TetDim<P>::NQF; ++q)
    for (int k = 0; k < TetDim<P>::KF; ++k) {
      const float v = (float)psi[(size_t)q * TetDim<P>::KF + k];
      h.psi[q][k] = v;
      h.psi2[q][k] = make_float2(v, v);
    }
  cudaMemcpyToSymbol(sym, &h, sizeof h);
}

void tet_upload_tables(int p, const RefTables& R, DeviceMesh& d) {
  if (R.dim != 3 || R.p != p) return;
  if (p == 1) upload_tet_p<1>(R, &cTetD1, &cTetF1);
  if (p == 2) upload_tet_p<2>(R, &cTetD2, &cTetF2);
  if (p == 1) upload_tet_pairs<1>(R, &cTetP1);
  if (p == 2) upload_tet_pairs<2>(R, &cTetP2);
  if (p == 1) upload_tet_mode_pairs<1>(R, &cTetQ1);
  if (p == 2) upload_tet_mode_pairs<2>(R, &cTetQ2);
  // orientation tables for the faces (FP64) and the FP32 lanes' face-modal
  // tables T [4][6][KF][NP], in global memory
  std::vector<double> t = tet_face_orient_tables(R), psi, T;
  tet_face_modal(t, R, psi, T);
  if (p == 1) upload_tet_modal<1>(psi, &cTetM1);
  if (p == 2) upload_tet_modal<2>(psi, &cTetM2);
  std::vector<float> tf(T.begin(), T.end());
  if (cudaMalloc(&d.ftabd, sizeof(double) * t.size()) != cudaSuccess ||
      cudaMalloc(&d.ftab, sizeof(float) * tf.size()) != cudaSuccess)
    throw Error{DGC_ERR_OOM, "cudaMalloc (face tables)"};
  cudaMemcpy(d.ftabd, t.data(), sizeof(double) * t.size(), cudaMemcpyHostToDevice);
  cudaMemcpy(d.ftab, tf.data(), sizeof(float) * tf.size(), cudaMemcpyHostToDevice);
  // the FP64 kernels' tables as FP32 pairs (hi, lo): the face tables, and the
  // volume tables [4][NQV][NP] (phi_j, w dphi_j/dr, w dphi_j/ds, w dphi_j/dt)
  auto pair = [](double x) {
    const float h = (float)x;
    return make_float2(h, (float)(x - (double)h));
  };
  std::vector<float2> tp(t.size()), vp((size_t)4 * R.nqv * R.np);
  for (size_t i = 0; i < t.size(); ++i) tp[i] = pair(t[i]);
  for (int q = 0; q < R.nqv; ++q)
    for (int j = 0; j < R.np; ++j) {
      vp[(size_t)q * R.np + j] = pair(R.phiV[(size_t)q * R.np + j]);
      for (int a = 0; a < 3; ++a)
        vp[((size_t)(a + 1) * R.nqv + q) * R.np + j] = pair(R.vw[q] * R.dphiV[((size_t)a * R.nqv + q) * R.np + j]);
    }
  if (cudaMalloc(&d.ftabdf, sizeof(float2) * tp.size()) != cudaSuccess ||
      cudaMalloc(&d.vtabdf, sizeof(float2) * vp.size()) != cudaSuccess)
    throw Error{DGC_ERR_OOM, "cudaMalloc (pair tables)"};
  cudaMemcpy(d.ftabdf, tp.data(), sizeof(float2) * tp.size(), cudaMemcpyHostToDevice);
  cudaMemcpy(d.vtabdf, vp.data(), sizeof(float2) * vp.size(), cudaMemcpyHostToDevice);
}

// ---------------------------------------------------------------------------
// loads and stores of element blocks (NV = 5 Np values: 8-byte vectors)
// ---------------------------------------------------------------------------
template <int N>
__device__ __forceinline__ void tload(const double* src, double (&v)[N]) {
  static_assert(N % 2 == 0, "");
  const double2* s = reinterpret_cast<const double2*>(src);
#pragma unroll
  for (int i = 0; i < N / 2; ++i) {
    double2 x = s[i];
    v[2 * i] = x.x;
    v[2 * i + 1] = x.y;
  }
}
template <int N>
__device__ __forceinline__ void tload(const float* src, float (&v)[N]) {
  const float2* s = reinterpret_cast<const float2*>(src);
#pragma unroll
  for (int i = 0; i < N / 2; ++i) {
    float2 x = s[i];
    v[2 * i] = x.x;
    v[2 * i + 1] = x.y;
  }
}
template <int N>
__device__ __forceinline__ void tstore(double* dst, const double (&v)[N]) {
  double2* d = reinterpret_cast<double2*>(dst);
#pragma unroll
  for (int i = 0; i < N / 2; ++i) d[i] = make_double2(v[2 * i], v[2 * i + 1]);
}
template <int N>
__device__ __forceinline__ void tstore(float* dst, const float (&v)[N]) {
  float2* d = reinterpret_cast<float2*>(dst);
#pragma unroll
  for (int i = 0; i < N / 2; ++i) d[i] = make_float2(v[2 * i], v[2 * i + 1]);
}

// ---------------------------------------------------------------------------
// FP32 element state in perturbation form
// ---------------------------------------------------------------------------
template <int P>
struct TetPert {
  using D = TetDim<P>;
  float hi[5], lo[5];
  float cd[5][D::NP - 1];
};

__device__ __forceinline__ void tsplit(double phi0, double c0, float& hi, float& lo) {
  const double u = phi0 * c0;
  hi = d2f(u);
  lo = d2f(u - f2d(hi));
}

template <int P>
__device__ __forceinline__ void tload_pert(const double* src, TetPert<P>& B) {
  using D = TetDim<P>;
  const double phi0 = tet_tabd<P>().phiV[0][0];
  double v[D::NV];
  tload(src, v);
#pragma unroll
  for (int m = 0; m < 5; ++m) {
    tsplit(phi0, v[m * D::NP], B.hi[m], B.lo[m]);
#pragma unroll
    for (int j = 1; j < D::NP; ++j) B.cd[m][j - 1] = d2f(v[m * D::NP + j]);
  }
}

template <int P>
__device__ __forceinline__ void tload_pert(const float* src, TetPert<P>& B) {
  using D = TetDim<P>;
  float v[D::NF];
  tload(src, v);
#pragma unroll
  for (int m = 0; m < 5; ++m) {
    B.hi[m] = v[m];
    B.lo[m] = v[5 + m];
#pragma unroll
    for (int j = 1; j < D::NP; ++j) B.cd[m][j - 1] = v[10 + m * (D::NP - 1) + j - 1];
  }
}

template <int P>
__device__ __forceinline__ void trecord_of(const double (&v)[TetDim<P>::NV], float (&r)[TetDim<P>::NF]) {
  using D = TetDim<P>;
  const double phi0 = tet_tabd<P>().phiV[0][0];
#pragma unroll
  for (int m = 0; m < 5; ++m) {
    tsplit(phi0, v[m * D::NP], r[m], r[5 + m]);
#pragma unroll
    for (int j = 1; j < D::NP; ++j) r[10 + m * (D::NP - 1) + j - 1] = d2f(v[m * D::NP + j]);
  }
#pragma unroll
  for (int i = 5 * (D::NP + 1); i < D::NF; ++i) r[i] = 0.0f;
}

// ---------------------------------------------------------------------------
// FP64 Euler fluxes, Eq. 2 as written
// ---------------------------------------------------------------------------
// Euler flux in direction n (not necessarily unit) and the max wave speed
__device__ __forceinline__ void euler3_n(const double* U, double nx, double ny, double nz, double* F, double& un,
                                         double& c) {
  const double ir = 1.0 / U[0];
  const double u = U[1] * ir, v = U[2] * ir, w = U[3] * ir;
  const double p = 0.4 * (U[4] - 0.5 * (U[1] * u + U[2] * v + U[3] * w));
  un = u * nx + v * ny + w * nz;
  c = sqrt(1.4 * p * ir);
  F[0] = U[0] * un;
  F[1] = U[1] * un + p * nx;
  F[2] = U[2] * un + p * ny;
  F[3] = U[3] * un + p * nz;
  F[4] = (U[4] + p) * un;
}


// The FP64 form with the basis contractions as FP32 pairs (dev_util.cuh), as
// on triangles: the element's mean ub = phi_0 c_0 in FP64, its modes j >= 1 as
// pairs; the volume integral projects F(U) . grad r_k - F(ub) . grad r_k, and
// the faces F* - F(ub).n (the omitted parts cancel exactly for each element),
// so the pairs carry only deviations.  The pair volume tables [4][NQV][NP] sit
// in shared memory (vt).
template <int P>
struct TetDfBlock {
  double ub[5];
  DF cd[5][TetDim<P>::NP - 1];
  __device__ __forceinline__ void init(const double (&c)[TetDim<P>::NV]) {
    constexpr int NP = TetDim<P>::NP;
    const double phi0 = tet_tabd<P>().phiV[0][0];
#pragma unroll
    for (int m = 0; m < 5; ++m) {
      ub[m] = phi0 * c[m * NP];
#pragma unroll
      for (int j = 1; j < NP; ++j) cd[m][j - 1] = df_split(c[m * NP + j]);
    }
  }
};

// the Euler flux of U in direction n (any length), given 1/rho and p
__device__ __forceinline__ void euler3_dir(const double* U, double ir, double p, const double* n, double* F) {
  const double un = (U[1] * n[0] + U[2] * n[1] + U[3] * n[2]) * ir;
  F[0] = U[0] * un;
  F[1] = U[1] * un + p * n[0];
  F[2] = U[2] * un + p * n[1];
  F[3] = U[3] * un + p * n[2];
  F[4] = (U[4] + p) * un;
}

template <int P>
__device__ __forceinline__ void tet_volume_df(const TetDfBlock<P>& B, const double* ji, const float2* vt,
                                              DF (&acc)[5][TetDim<P>::NP]) {
  using D = TetDim<P>;
  constexpr int NP = D::NP, NQV = D::NQV;
  double J[9];
#pragma unroll
  for (int i = 0; i < 9; ++i) J[i] = __ldg(ji + i);
  double Fb[3][5];  // F(ub) . grad r_k
  {
    const double ir = 1.0 / B.ub[0];
    const double p = 0.4 * (B.ub[4] - 0.5 * (B.ub[1] * B.ub[1] + B.ub[2] * B.ub[2] + B.ub[3] * B.ub[3]) * ir);
#pragma unroll
    for (int k = 0; k < 3; ++k) euler3_dir(B.ub, ir, p, J + 3 * k, Fb[k]);
  }
#pragma unroll 1
  for (int q = 0; q < NQV; ++q) {
    double U[5];
#pragma unroll
    for (int m = 0; m < 5; ++m) {
      DF d{0.0f, 0.0f};
#pragma unroll
      for (int j = 1; j < NP; ++j) df_fma(d, vt[q * NP + j], B.cd[m][j - 1]);
      U[m] = B.ub[m] + df_join(d);
    }
    const double ir = 1.0 / U[0];
    const double p = 0.4 * (U[4] - 0.5 * (U[1] * U[1] + U[2] * U[2] + U[3] * U[3]) * ir);
    DF g[3][5];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      double F[5];
      euler3_dir(U, ir, p, J + 3 * k, F);
#pragma unroll
      for (int m = 0; m < 5; ++m) g[k][m] = df_split(F[m] - Fb[k][m]);
    }
#pragma unroll
    for (int m = 0; m < 5; ++m)
#pragma unroll
      for (int j = 1; j < NP; ++j) {
        df_fma(acc[m][j], vt[(NQV + q) * NP + j], g[0][m]);
        df_fma(acc[m][j], vt[(2 * NQV + q) * NP + j], g[1][m]);
        df_fma(acc[m][j], vt[(3 * NQV + q) * NP + j], g[2][m]);
      }
  }
}

// FP32 volume integral in perturbation form (F(ub) left out, grad phi_0 = 0)
template <int P>
__device__ __forceinline__ void tet_volume32(const TetPert<P>& B, const PertRef<3>& R, const double* ji,
                                             float (&acc)[TetDim<P>::NV]) {
  using D = TetDim<P>;
  constexpr int NP = D::NP;
  float J[3][3], th[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
#pragma unroll
    for (int a = 0; a < 3; ++a) J[k][a] = d2f(__ldg(ji + 3 * k + a));
    th[k] = R.u[1] * J[k][0] + R.u[2] * J[k][1] + R.u[3] * J[k][2];
  }
  // variables (0, 1) and (2, 3) in pairs on the packed FP32 FMA (__ffma2_rn),
  // variable 4 with its modes in pairs (1, 2), (3, 4), ...
  const TetPairTab<P>& K2 = tet_ptab<P>();
  const TetModePairTab<P>& K4 = tet_qtab<P>();
  constexpr int NH = TetModePairTab<P>::NH;
  float2 c01[NP - 1], c23[NP - 1], a01[NP - 1], a23[NP - 1], c4[NH], a4[NH];
#pragma unroll
  for (int j = 1; j < NP; ++j) {
    c01[j - 1] = make_float2(B.cd[0][j - 1], B.cd[1][j - 1]);
    c23[j - 1] = make_float2(B.cd[2][j - 1], B.cd[3][j - 1]);
    a01[j - 1] = make_float2(acc[j], acc[NP + j]);
    a23[j - 1] = make_float2(acc[2 * NP + j], acc[3 * NP + j]);
  }
#pragma unroll
  for (int k = 0; k < NH; ++k) {
    const int j = 1 + 2 * k;
    c4[k] = make_float2(B.cd[4][j - 1], j + 1 < NP ? B.cd[4][j] : 0.0f);
    a4[k] = make_float2(acc[4 * NP + j], j + 1 < NP ? acc[4 * NP + j + 1] : 0.0f);
  }
#pragma unroll 2
  for (int q = 0; q < D::NQV; ++q) {
    float2 d01 = make_float2(B.lo[0], B.lo[1]), d23 = make_float2(B.lo[2], B.lo[3]);
    float2 d4p = make_float2(0.0f, 0.0f);
#pragma unroll
    for (int j = 1; j < NP; ++j) {
      d01 = __ffma2_rn(K2.phiV[q][j], c01[j - 1], d01);
      d23 = __ffma2_rn(K2.phiV[q][j], c23[j - 1], d23);
    }
#pragma unroll
    for (int k = 0; k < NH; ++k) d4p = __ffma2_rn(K4.phiV[q][k], c4[k], d4p);
    const float d[5] = {d01.x, d01.y, d23.x, d23.y, B.lo[4] + (d4p.x + d4p.y)};
    PertState<3> S;
    S.init(R, d);
    float Fr[3][5];
#pragma unroll
    for (int k = 0; k < 3; ++k) pert_flux<3>(R, S, d, J[k], th[k], Fr[k]);
    float2 f01[3], f23[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      f01[k] = make_float2(Fr[k][0], Fr[k][1]);
      f23[k] = make_float2(Fr[k][2], Fr[k][3]);
    }
#pragma unroll
    for (int j = 1; j < NP; ++j) {
      a01[j - 1] = __ffma2_rn(K2.vt[q][j], f01[2], __ffma2_rn(K2.vs[q][j], f01[1], __ffma2_rn(K2.vr[q][j], f01[0], a01[j - 1])));
      a23[j - 1] = __ffma2_rn(K2.vt[q][j], f23[2], __ffma2_rn(K2.vs[q][j], f23[1], __ffma2_rn(K2.vr[q][j], f23[0], a23[j - 1])));
    }
    const float2 g0 = make_float2(Fr[0][4], Fr[0][4]), g1 = make_float2(Fr[1][4], Fr[1][4]),
                 g2 = make_float2(Fr[2][4], Fr[2][4]);
#pragma unroll
    for (int k = 0; k < NH; ++k)
      a4[k] = __ffma2_rn(K4.vt[q][k], g2, __ffma2_rn(K4.vs[q][k], g1, __ffma2_rn(K4.vr[q][k], g0, a4[k])));
  }
#pragma unroll
  for (int j = 1; j < NP; ++j) {
    acc[j] = a01[j - 1].x;
    acc[NP + j] = a01[j - 1].y;
    acc[2 * NP + j] = a23[j - 1].x;
    acc[3 * NP + j] = a23[j - 1].y;
  }
#pragma unroll
  for (int k = 0; k < NH; ++k) {
    const int j = 1 + 2 * k;
    acc[4 * NP + j] = a4[k].x;
    if (j + 1 < NP) acc[4 * NP + j + 1] = a4[k].y;
  }
}

template <int P, typename CT, typename ST, typename RT>
__global__ void __launch_bounds__(128) k_vol_tet(const ST* c, int sstride, const double* jinv, RT* rhs, int64_t e0,
                                                 int64_t ne, const float2* vtab) {
  using D = TetDim<P>;
  constexpr int NP = D::NP;
  extern __shared__ float2 vt_s[];  // FP64: the pair volume tables [4][NQV][NP]
  if constexpr (sizeof(CT) == 8) {
    for (int i = threadIdx.x; i < 4 * D::NQV * NP; i += blockDim.x) vt_s[i] = vtab[i];
    __syncthreads();
  }
  const int64_t e = e0 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= ne) return;
  RT out[D::NV];
  if constexpr (sizeof(CT) == 8) {
    TetDfBlock<P> B;
    {
      double v[D::NV];
      tload(c + e * D::NV, v);
      B.init(v);
    }
    DF acc[5][NP];
#pragma unroll
    for (int m = 0; m < 5; ++m)
#pragma unroll
      for (int j = 0; j < NP; ++j) acc[m][j] = DF{0.0f, 0.0f};
    tet_volume_df<P>(B, jinv + 9 * e, vt_s, acc);
#pragma unroll
    for (int m = 0; m < 5; ++m)
#pragma unroll
      for (int j = 0; j < NP; ++j) out[m * NP + j] = j ? (RT)df_join(acc[m][j]) : (RT)0.0;
  } else {
    const int64_t stride = sizeof(ST) == 8 ? D::NV : sstride;
    TetPert<P> B;
    tload_pert<P>(c + e * stride, B);
    PertRef<3> R;
    R.init(B.hi);
    float acc[D::NV];
#pragma unroll
    for (int i = 0; i < D::NV; ++i) acc[i] = 0.0f;
    tet_volume32<P>(B, R, jinv + 9 * e, acc);
#pragma unroll
    for (int i = 0; i < D::NV; ++i) out[i] = (RT)acc[i];
  }
  tstore(rhs + e * D::NV, out);
}

struct TetParams {
  int64_t begin, end;
  const int4* topo;
  const double2* fgeo;
  const double* jinv;
  const void* ftab;  // FP64: [4][6][NQF][NP] as FP32 pairs; FP32: the face-modal T [4][6][KF][NP]
  const float2* vtab = nullptr;  // FP64 first color: the pair volume tables [4][NQV][NP]
  const void* state;
  void* rhs;
  void* buf;
  StageArgs sa;
  int sstride;  // floats per element of an FP32 state (record)
};

template <int P, typename RT, int MODE, typename AT>
__device__ __forceinline__ void tet_write(const TetParams& A, int64_t elem, int64_t k, int side,
                                          const AT (&acc)[TetDim<P>::NV]) {
  using D = TetDim<P>;
  constexpr int NV = D::NV;
  if constexpr (MODE == SURF_RMW) {
    RT* r = static_cast<RT*>(A.rhs) + elem * NV;
    RT old[NV];
    tload(r, old);
#pragma unroll
    for (int i = 0; i < NV; ++i) old[i] += (RT)acc[i];
    tstore(r, old);
  } else if constexpr (MODE == SURF_FIRST) {
    RT out[NV];
#pragma unroll
    for (int i = 0; i < NV; ++i) out[i] = (RT)acc[i];
    tstore(static_cast<RT*>(A.rhs) + elem * NV, out);
  } else if constexpr (MODE == SURF_ATOMIC) {
    RT* r = static_cast<RT*>(A.rhs) + elem * NV;
#pragma unroll
    for (int i = 0; i < NV; ++i) atomicAdd(r + i, (RT)acc[i]);
  } else if constexpr (MODE == SURF_BUFFER) {
    RT out[NV];
#pragma unroll
    for (int i = 0; i < NV; ++i) out[i] = (RT)acc[i];
    tstore(static_cast<RT*>(A.buf) + (2 * k + side) * NV, out);
  }
}

// One variable's NP values of a lane's contribution, written as the mode asks
// (the FP32 lanes but the last color's)
template <int P, typename RT, int MODE>
__device__ __forceinline__ void tet_write_var(const TetParams& A, int64_t elem, int64_t k, int side, int m,
                                              const float (&cm)[TetDim<P>::NP]) {
  constexpr int NP = TetDim<P>::NP, NV = TetDim<P>::NV;
  static_assert(NP % 2 == 0, "one variable's block: 8-byte (float) or 16-byte (double) vectors");
  if constexpr (MODE == SURF_FIRST) {
    RT out[NP];
#pragma unroll
    for (int j = 0; j < NP; ++j) out[j] = (RT)cm[j];
    tstore(static_cast<RT*>(A.rhs) + elem * NV + m * NP, out);
  } else if constexpr (MODE == SURF_RMW) {
    RT* r = static_cast<RT*>(A.rhs) + elem * NV + m * NP;
    RT old[NP];
    tload(r, old);
#pragma unroll
    for (int j = 0; j < NP; ++j) old[j] += (RT)cm[j];
    tstore(r, old);
  } else if constexpr (MODE == SURF_ATOMIC) {
    RT* r = static_cast<RT*>(A.rhs) + elem * NV + m * NP;
#pragma unroll
    for (int j = 0; j < NP; ++j) atomicAdd(r + j, (RT)cm[j]);
  } else if constexpr (MODE == SURF_BUFFER) {
    RT out[NP];
#pragma unroll
    for (int j = 0; j < NP; ++j) out[j] = (RT)cm[j];
    tstore(static_cast<RT*>(A.buf) + (2 * k + side) * NV + m * NP, out);
  }
}

// Last color, FP64 form (as fp64_last for triangles): us = the state block the
// fluxes used (registers); chunks of CH value pairs, loads before stores.
template <int P>
__device__ __forceinline__ void tet_fp64_last(const TetParams& A, int64_t elem, const double (&acc)[TetDim<P>::NV],
                                              const double (&us)[TetDim<P>::NV]) {
  constexpr int NV = TetDim<P>::NV, H = NV / 2, CH = 5;
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

// FP32 surface kernels: a register cap (DGC_TET_REGS) and the minimum resident
// blocks of 256 threads per SM the compiler must allow (DGC_TET_MINB); FP64
// kernels are never capped.  At p = 2 the uncapped kernels take 176-242
// registers (two blocks of 128 threads per SM); 168 keeps them spill-free with
// three (measured: RK step 10.7 -> 9.2 ms on 64^3 x 6 tetrahedra).
#ifndef DGC_TET_REGS
#define DGC_TET_REGS 168
#endif
#ifndef DGC_TET_QUNROLL
#define DGC_TET_QUNROLL 2
#endif
#define DGC_TET_PRAGMA(x) _Pragma(#x)
#define DGC_TET_PRAGMA2(x) DGC_TET_PRAGMA(x)
#define DGC_TET_UNROLL_Q DGC_TET_PRAGMA2(unroll DGC_TET_QUNROLL)
#ifndef DGC_TET_REGS_COLOR
#define DGC_TET_REGS_COLOR 128
#endif
#ifndef DGC_TET_MINB
#define DGC_TET_MINB 1
#endif

template <int P, typename CT, typename ST, typename RT, int MODE>
__global__ void __launch_bounds__(256, (sizeof(CT) == 4 ? DGC_TET_MINB : 1))
    __maxnreg__((sizeof(CT) == 4 ? (MODE == SURF_FIRST || MODE == SURF_LAST ? DGC_TET_REGS : DGC_TET_REGS_COLOR) : 255))
        k_surf_tet(const TetParams A) {
  using D = TetDim<P>;
  constexpr int NP = D::NP, NQ = D::NQF, NV = D::NV;
  extern __shared__ unsigned char smem_raw[];
  // FP64: the orientation tables [4][6][NQ][NP] as FP32 pairs; FP32: the
  // face-modal tables T [4][6][KF][NP]
  constexpr int NTAB = sizeof(CT) == 8 ? 24 * NQ * NP : 24 * D::KF * NP;
  CT* sphi = reinterpret_cast<CT*>(smem_raw);
  {
    const CT* src = static_cast<const CT*>(A.ftab);
    for (int i = threadIdx.x; i < NTAB; i += blockDim.x) sphi[i] = src[i];
  }
  // the FP64 first color: the pair volume tables after the face tables
  float2* vt = reinterpret_cast<float2*>(smem_raw + sizeof(CT) * 24 * NQ * NP);
  if constexpr (sizeof(CT) == 8 && MODE == SURF_FIRST)
    for (int i = threadIdx.x; i < 4 * D::NQV * NP; i += blockDim.x) vt[i] = A.vtab[i];
  __syncthreads();
  // programmatic launch (dev_util.cuh): the first color reads its predecessor's
  // record and overwrites the rhs it read, so it waits at once; the other
  // colors wait before their epilogue, which reads the predecessor's rhs
  if constexpr (MODE == SURF_FIRST) {
    pdl_wait();
    pdl_trigger();
  }

  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  int64_t k = A.begin + (t >> 1);
  const int side = (int)(t & 1);
  const bool valid = k < A.end;
  if (!valid) k = A.end - 1;
  const int4 tp = A.topo[k];
  const bool bnd = tp.y < 0;
  const bool right = side && !bnd;
  const int64_t elem = right ? tp.y : tp.x;
  const int lf = right ? ((tp.z >> 4) & 15) : (tp.z & 15);
  const int orient = right ? ((tp.z >> 8) & 7) : 0;
  const bool writer = valid && !(side && bnd);
  const double2 g0 = A.fgeo[3 * k], g1 = A.fgeo[3 * k + 1], g2 = A.fgeo[3 * k + 2];

  if constexpr (sizeof(CT) == 8) {
    const CT* ph = sphi + (lf * 6 + orient) * NQ * NP;
    // FP64 flux and update, the basis contractions as FP32 pairs on the flux
    // deviations (tet_volume_df)
    const TetTabD<P>& K = tet_tabd<P>();
    const float2* ph2 = reinterpret_cast<const float2*>(ph);
    TetDfBlock<P> B;
    {
      double c[NV];
      tload(static_cast<const double*>(A.state) + elem * NV, c);
      B.init(c);
    }
    DF acc2[5][NP];
#pragma unroll
    for (int m = 0; m < 5; ++m)
#pragma unroll
      for (int j = 0; j < NP; ++j) acc2[m][j] = DF{0.0f, 0.0f};
    if constexpr (MODE == SURF_FIRST) tet_volume_df<P>(B, A.jinv + 9 * elem, vt, acc2);
    const double scale = right ? g2.y : -g2.x;
    const double nn[3] = {g0.x, g0.y, g1.x};
    double Fbn[5];  // F(ub).n, subtracted from the face flux (the volume integral omits F(ub))
    {
      const double ir = 1.0 / B.ub[0];
      const double p = 0.4 * (B.ub[4] - 0.5 * (B.ub[1] * B.ub[1] + B.ub[2] * B.ub[2] + B.ub[3] * B.ub[3]) * ir);
      euler3_dir(B.ub, ir, p, nn, Fbn);
    }
#pragma unroll 2
    for (int q = 0; q < NQ; ++q) {
      double U[5], V[5], a[5], b[5], Fs[5];
#pragma unroll
      for (int m = 0; m < 5; ++m) {
        DF t{0.0f, 0.0f};
#pragma unroll
        for (int j = 1; j < NP; ++j) df_fma(t, ph2[q * NP + j], B.cd[m][j - 1]);
        U[m] = B.ub[m] + df_join(t);
      }
      // each lane evaluates its own side (one division, one square root) and
      // exchanges the normal flux and wave speed with its partner; the sums
      // below are commutative, so both lanes get the same bits
      double Fo[5], Fp[5], uno, co;
      euler3_n(U, g0.x, g0.y, g1.x, Fo, uno, co);
      const double wo = fabs(uno) + co;
#pragma unroll
      for (int m = 0; m < 5; ++m) {
        V[m] = __shfl_xor_sync(0xffffffffu, U[m], 1);
        Fp[m] = __shfl_xor_sync(0xffffffffu, Fo[m], 1);
      }
      const double lam = fmax(wo, __shfl_xor_sync(0xffffffffu, wo, 1));
#pragma unroll
      for (int m = 0; m < 5; ++m) {
        a[m] = side ? V[m] : U[m];
        b[m] = side ? U[m] : V[m];
        Fs[m] = 0.5 * (Fo[m] + Fp[m]) - (0.5 * lam) * (b[m] - a[m]);
      }
      const double sq = scale * K.wF[q];
#pragma unroll
      for (int m = 0; m < 5; ++m) {
        const DF g = df_split(sq * (Fs[m] - Fbn[m]));
#pragma unroll
        for (int j = 0; j < NP; ++j) df_fma(acc2[m][j], ph2[q * NP + j], g);
      }
    }
    double acc[NV];
#pragma unroll
    for (int m = 0; m < 5; ++m)
#pragma unroll
      for (int j = 0; j < NP; ++j) acc[m * NP + j] = df_join(acc2[m][j]);
    if constexpr (MODE != SURF_FIRST) {
      pdl_wait();
      pdl_trigger();
    }
    if constexpr (MODE == SURF_LAST) {
      double c[NV];  // the stage input block again (cached), for the update
      tload(static_cast<const double*>(A.state) + elem * NV, c);
      if (writer) tet_fp64_last<P>(A, elem, acc, c);
    } else if (writer) {
      tet_write<P, RT, MODE>(A, elem, k, side, acc);
    }
  } else {
    // FP32 lanes, face-modal (tet_face_modal): the element block is turned into
    // the volume integral (first color) and the trace's KF face coefficients,
    // and not held through the point loop; variables (0, 1) and (2, 3) in pairs
    // on the packed FP32 FMA, variable 4 alone
    constexpr int KF = D::KF;
    const TetTab<float, P>& K = tet_tab<float, P>();
    const TetFaceTab<P>& FM = tet_mtab<P>();
    const float* Tl = reinterpret_cast<const float*>(sphi) + (lf * 6 + orient) * KF * NP;  // T [KF][NP]
    float* vsm = reinterpret_cast<float*>(sphi) + NTAB;  // first color: [NV][blockDim.x]
    const int64_t stride = sizeof(ST) == 8 ? NV : A.sstride;
    const ST* src = static_cast<const ST*>(A.state) + elem * stride;
    float acc[NV];
#pragma unroll
    for (int i = 0; i < NV; ++i) acc[i] = 0.0f;
    float hi[5], lo[5];
    float2 a01[KF], a23[KF];
    float a4[KF];
    PertRef<3> R;
    {
      TetPert<P> B;
      tload_pert<P>(src, B);
      R.init(B.hi);
#pragma unroll
      for (int m = 0; m < 5; ++m) {
        hi[m] = B.hi[m];
        lo[m] = B.lo[m];
      }
      if constexpr (MODE == SURF_FIRST) {
        // the volume integral waits in shared memory (one value per thread and
        // row: conflict-free) while the point loop runs
        tet_volume32<P>(B, R, A.jinv + 9 * elem, acc);
#pragma unroll
        for (int i = 0; i < NV; ++i) vsm[i * blockDim.x + threadIdx.x] = acc[i];
      }
      // the trace deviation's face coefficients a_k = sum_{j >= 1} T[k][j] c_j
#pragma unroll
      for (int kk = 0; kk < KF; ++kk) {
        a01[kk] = make_float2(0.0f, 0.0f);
        a23[kk] = make_float2(0.0f, 0.0f);
        a4[kk] = 0.0f;
      }
#pragma unroll
      for (int j = 1; j < NP; ++j) {
        const float2 c01 = make_float2(B.cd[0][j - 1], B.cd[1][j - 1]);
        const float2 c23 = make_float2(B.cd[2][j - 1], B.cd[3][j - 1]);
#pragma unroll
        for (int kk = 0; kk < KF; ++kk) {
          const float t = Tl[kk * NP + j];
          const float2 t2 = make_float2(t, t);
          a01[kk] = __ffma2_rn(t2, c01, a01[kk]);
          a23[kk] = __ffma2_rn(t2, c23, a23[kk]);
          a4[kk] = fmaf(t, B.cd[4][j - 1], a4[kk]);
        }
      }
    }
    // each lane evaluates its own side's flux and the pair exchanges one value
    // per variable (euler_pert.cuh, lf_exchange); the lane projects onto psi_k
    FaceConst<3> E;
    E.init(R, hi, {d2f(g0.x), d2f(g0.y), d2f(g1.x)}, side);
    const float scale = right ? d2f(g2.y) : -d2f(g2.x);
    float2 b01[KF], b23[KF];
    float b4[KF];
#pragma unroll
    for (int kk = 0; kk < KF; ++kk) {
      b01[kk] = make_float2(0.0f, 0.0f);
      b23[kk] = make_float2(0.0f, 0.0f);
      b4[kk] = 0.0f;
    }
    DGC_TET_UNROLL_Q
    for (int q = 0; q < NQ; ++q) {
      float2 d01 = make_float2(lo[0], lo[1]), d23 = make_float2(lo[2], lo[3]);
      float d4 = lo[4];
#pragma unroll
      for (int kk = 0; kk < KF; ++kk) {
        d01 = __ffma2_rn(FM.psi2[q][kk], a01[kk], d01);
        d23 = __ffma2_rn(FM.psi2[q][kk], a23[kk], d23);
        d4 = fmaf(FM.psi[q][kk], a4[kk], d4);
      }
      const float ds[5] = {d01.x, d01.y, d23.x, d23.y, d4};  // own trace - ub
      float G[5];
      lf_exchange<3>(R, E, ds, G);
      const float s = scale * K.wF[q];
      const float2 g01 = make_float2(s * G[0], s * G[1]), g23 = make_float2(s * G[2], s * G[3]);
      const float g4 = s * G[4];
#pragma unroll
      for (int kk = 0; kk < KF; ++kk) {
        b01[kk] = __ffma2_rn(FM.psi2[q][kk], g01, b01[kk]);
        b23[kk] = __ffma2_rn(FM.psi2[q][kk], g23, b23[kk]);
        b4[kk] = fmaf(FM.psi[q][kk], g4, b4[kk]);
      }
    }
    // the face's contribution to the lane's modes, sum_k T[k][j] b_k: into acc
    // for the last color; the other modes take it one variable at a time in
    // their write (the whole block is never live beside b)
    auto bvar = [&](int kk, int m) {
      return m == 0 ? b01[kk].x : m == 1 ? b01[kk].y : m == 2 ? b23[kk].x : m == 3 ? b23[kk].y : b4[kk];
    };
    if constexpr (MODE == SURF_LAST) {
#pragma unroll
      for (int m = 0; m < 5; ++m)
#pragma unroll
        for (int j = 0; j < NP; ++j)
#pragma unroll
          for (int kk = 0; kk < KF; ++kk) acc[m * NP + j] = fmaf(Tl[kk * NP + j], bvar(kk, m), acc[m * NP + j]);
    }
    if constexpr (MODE != SURF_FIRST) {
      pdl_wait();
      pdl_trigger();
    }
    if constexpr (MODE == SURF_LAST) {
      // the element's right-hand side is complete: SSP-RK3 stage in increment
      // form (stage 0 writes the record of u0, the block read above: read again)
      if (writer) {
        float L[NV];
        ldv<NV>(static_cast<const float*>(A.rhs) + elem * NV, L);
#pragma unroll
        for (int i = 0; i < NV; ++i) L[i] += acc[i];
        TetPert<P> B;
        if (A.sa.stage == 0) tload_pert<P>(src, B);
        incr_last<5, NP>(A.sa, elem, L, B, tet_tabd<P>().phiV[0][0]);
      }
    } else if (writer) {
      if constexpr (MODE == SURF_RMW && sizeof(RT) == 4) {
        // FP32 rhs: the whole block's loads in flight at once, then each
        // variable's contributions added (the block and b fit beside each other)
        float* r = static_cast<float*>(A.rhs) + elem * NV;
        float old[NV];
        tload(r, old);
#pragma unroll
        for (int m = 0; m < 5; ++m)
#pragma unroll
          for (int j = 0; j < NP; ++j)
#pragma unroll
            for (int kk = 0; kk < KF; ++kk) old[m * NP + j] = fmaf(Tl[kk * NP + j], bvar(kk, m), old[m * NP + j]);
        tstore(r, old);
      } else {
#pragma unroll
        for (int m = 0; m < 5; ++m) {
          float cm[NP];
#pragma unroll
          for (int j = 0; j < NP; ++j) {
            float v = MODE == SURF_FIRST ? vsm[(m * NP + j) * blockDim.x + threadIdx.x] : 0.0f;
#pragma unroll
            for (int kk = 0; kk < KF; ++kk) v = fmaf(Tl[kk * NP + j], bvar(kk, m), v);
            cm[j] = v;
          }
          tet_write_var<P, RT, MODE>(A, elem, k, side, m, cm);
        }
      }
    }
  }
}

// CFL reduction in two passes, as for triangles: FP32 estimates of every
// element, then FP64 only for the elements within kCflMargin of the minimum.
// Pass 1 builds the element's FP32 record one variable at a time and takes the
// estimate from it (mean pair + modes).
template <int P>
__device__ __forceinline__ float tet_lambda_rec(const float (&r)[TetDim<P>::NF]) {
  using D = TetDim<P>;
  constexpr int NP = D::NP;
  const TetTab<float, P>& K = tet_tab<float, P>();
  float lam = 0.0f;
#pragma unroll 2
  for (int q = 0; q < D::NQV; ++q) {
    float U[5];
#pragma unroll
    for (int m = 0; m < 5; ++m) {
      float s = r[5 + m];
#pragma unroll
      for (int j = 1; j < NP; ++j) s += K.phiV[q][j] * r[10 + m * (NP - 1) + j - 1];
      U[m] = r[m] + s;
    }
    const float ir = rcp_fast(U[0]), u = U[1] * ir, w = U[2] * ir, z = U[3] * ir;
    const float q2 = u * u + w * w + z * z;
    const float pr = 0.4f * (U[4] - 0.5f * U[0] * q2);
    lam = fmaxf(lam, sqrt_fast(q2) + sqrt_fast(1.4f * pr * ir));
  }
  return lam;
}

template <int P>
__global__ void __launch_bounds__(128) k_cfl1_tet(const double* c, const double* inr, int64_t ne, float* est,
                                                  unsigned* minbits, float* shadow) {
  using D = TetDim<P>;
  constexpr int NP = D::NP;
  pdl_wait();
  pdl_trigger();
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  float best = FLT_MAX;
  if (e < ne) {
    const double phi0 = tet_tabd<P>().phiV[0][0];
    float r[D::NF];
#pragma unroll
    for (int m = 0; m < 5; ++m) {
      double v[NP];
      tload(c + e * D::NV + m * NP, v);
      tsplit(phi0, v[0], r[m], r[5 + m]);
#pragma unroll
      for (int j = 1; j < NP; ++j) r[10 + m * (NP - 1) + j - 1] = d2f(v[j]);
    }
#pragma unroll
    for (int i = 5 * (NP + 1); i < D::NF; ++i) r[i] = 0.0f;
    if (shadow) tstore(shadow + e * D::NF, r);
    float d = d2f(inr[e]) / ((2 * P + 1) * tet_lambda_rec<P>(r));
    if (!(d > 0.0f) || !(d < FLT_MAX)) d = 0.0f;
    est[e] = d;
    best = d;
  }
  block_min_to(best, minbits);
}

// Pass 2: each candidate is evaluated in FP64 by the whole warp, one volume
// point per lane (a GB300 FP64 warp instruction occupies the FP64 pipe for ~64
// cycles, so one lane running every point would take tens of microseconds).
template <int P>
__global__ void __launch_bounds__(128) k_cfl2_tet(const double* c, const double* inr, int64_t ne, double cfl,
                                                  const float* est, const unsigned* minbits,
                                                  unsigned long long* dtbits) {
  using D = TetDim<P>;
  constexpr int NP = D::NP;
  pdl_wait();
  pdl_trigger();
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const bool cand = e < ne && est[e] <= __uint_as_float(*minbits) * (1.0f + kCflMargin);
  unsigned mask = __ballot_sync(0xffffffffu, cand);
  double best = DBL_MAX;
  const TetTabD<P>& K = tet_tabd<P>();
  while (mask) {
    const int src = __ffs(mask) - 1;
    mask &= mask - 1;
    const long long ec = __shfl_sync(0xffffffffu, (long long)e, src);
    const double* v = c + ec * D::NV;  // the same block for every lane: broadcast loads
    double lam = 0.0;
    for (int q = threadIdx.x & 31; q < D::NQV; q += 32) {
      double U[5];
#pragma unroll
      for (int m = 0; m < 5; ++m) {
        double sum = 0.0;
#pragma unroll
        for (int j = 0; j < NP; ++j) sum += K.phiV[q][j] * v[m * NP + j];
        U[m] = sum;
      }
      const double ir = 1.0 / U[0], u = U[1] * ir, w = U[2] * ir, z = U[3] * ir;
      const double q2 = u * u + w * w + z * z;
      const double pr = 0.4 * (U[4] - 0.5 * U[0] * q2);
      lam = fmax(lam, sqrt(q2) + sqrt(1.4 * pr * ir));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) lam = fmax(lam, __shfl_xor_sync(0xffffffffu, lam, o));
    const double b = cfl * (inr[ec] / ((2 * P + 1) * lam));
    if ((threadIdx.x & 31) == src) best = b > 0.0 ? b : DBL_MAX;
  }
  block_min_to(best, dtbits);
}

// ---------------------------------------------------------------------------
template <int P, typename CT, typename ST, typename RT>
static int tvol_p(const Ctx& x, const void* s, int ss, void* r, int64_t e0) {
  const int bs = 128;
  const int64_t n = x.ne - e0;
  if (n <= 0) return 0;
  using D = TetDim<P>;
  const size_t smem = sizeof(CT) == 8 ? sizeof(float2) * 4 * D::NQV * D::NP : 0;
  if (smem > 48 * 1024) cudaFuncSetAttribute(k_vol_tet<P, CT, ST, RT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
  k_vol_tet<P, CT, ST, RT><<<(unsigned)((n + bs - 1) / bs), bs, smem, x.st>>>(
      static_cast<const ST*>(s), ss, x.d->jinv, static_cast<RT*>(r), e0, x.ne, x.d->vtabdf);
  return 1;
}

int tet_volume(const Ctx& x, TypeCfg ty, const void* s, int ss, void* r, int64_t e0) {
  switch (x.p * 4 + ty) {
    case 4 + TY_D: return tvol_p<1, double, double, double>(x, s, ss, r, e0);
    case 8 + TY_D: return tvol_p<2, double, double, double>(x, s, ss, r, e0);
    case 4 + TY_MD: return tvol_p<1, float, double, double>(x, s, ss, r, e0);
    case 8 + TY_MD: return tvol_p<2, float, double, double>(x, s, ss, r, e0);
    case 4 + TY_MF: return tvol_p<1, float, float, float>(x, s, ss, r, e0);
    case 8 + TY_MF: return tvol_p<2, float, float, float>(x, s, ss, r, e0);
    default: return -1;
  }
}

template <int P, typename CT, typename ST, typename RT, int MODE>
static int tsurf_launch(const Ctx& x, TetParams A) {
  const int64_t n = A.end - A.begin;
  if (n <= 0) return 0;
  using D = TetDim<P>;
  A.ftab = sizeof(CT) == 8 ? (const void*)x.d->ftabdf : (const void*)x.d->ftab;
  A.vtab = x.d->vtabdf;
  const int threads = 2 * x.epb;
  // the face tables; the FP64 first color's pair volume tables, the FP32 first
  // color's volume integrals (NV floats per thread)
  const size_t smem = (sizeof(CT) == 8 ? sizeof(CT) * 24 * D::NQF * D::NP : sizeof(float) * 24 * D::KF * D::NP) +
                      (sizeof(CT) == 8 && MODE == SURF_FIRST ? sizeof(float2) * 4 * D::NQV * D::NP : 0) +
                      (sizeof(CT) == 4 && MODE == SURF_FIRST ? sizeof(float) * D::NV * threads : 0);
  auto kern = k_surf_tet<P, CT, ST, RT, MODE>;
  if (smem > 48 * 1024) cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  launch_k(x, kern, (unsigned)((2 * n + threads - 1) / threads), (unsigned)threads, smem, A);
  return 1;
}

template <int P, typename CT, typename ST, typename RT>
static int tsurf_mode(const Ctx& x, SurfMode mode, const TetParams& A) {
  switch (mode) {
    case SURF_RMW: return tsurf_launch<P, CT, ST, RT, SURF_RMW>(x, A);
    case SURF_FIRST: return tsurf_launch<P, CT, ST, RT, SURF_FIRST>(x, A);
    case SURF_ATOMIC: return tsurf_launch<P, CT, ST, RT, SURF_ATOMIC>(x, A);
    case SURF_BUFFER: return tsurf_launch<P, CT, ST, RT, SURF_BUFFER>(x, A);
    default: return -1;
  }
}

template <int P>
static int tsurf_p(const Ctx& x, TypeCfg ty, SurfMode mode, const TetParams& A) {
  if (mode == SURF_LAST) {
    if (ty == TY_D) return tsurf_launch<P, double, double, double, SURF_LAST>(x, A);
    if (ty == TY_MF) return tsurf_launch<P, float, float, float, SURF_LAST>(x, A);
    return -1;
  }
  switch (ty) {
    case TY_D: return tsurf_mode<P, double, double, double>(x, mode, A);
    case TY_MD: return tsurf_mode<P, float, double, double>(x, mode, A);
    case TY_MF:
      if (mode != SURF_RMW && mode != SURF_FIRST) return -1;
      return tsurf_mode<P, float, float, float>(x, mode, A);
    default: return -1;
  }
}

int tet_surface(const Ctx& x, TypeCfg ty, SurfMode mode, int64_t begin, int64_t end, const void* state,
                int sstride, void* rhs, void* buf, const StageArgs* sa) {
  TetParams A;
  A.begin = begin;
  A.end = end;
  A.sstride = sstride;
  A.topo = x.d->topo;
  A.fgeo = x.d->fgeo;
  A.jinv = x.d->jinv;
  A.ftab = nullptr;
  A.state = state;
  A.rhs = rhs;
  A.buf = buf;
  if (sa) A.sa = *sa;
  switch (x.p) {
    case 1: return tsurf_p<1>(x, ty, mode, A);
    case 2: return tsurf_p<2>(x, ty, mode, A);
    default: return -1;
  }
}

int tet_cfl(const Ctx& x, const double* s, double cfl, double* dt, float* shadow) {
  const int bs = 128;
  const unsigned grid = (unsigned)((x.ne + bs - 1) / bs);
  auto* bits = reinterpret_cast<unsigned long long*>(dt);
  float* est = x.d->cfl_est;
  unsigned* mn = reinterpret_cast<unsigned*>(x.d->cfl_est + x.ne);
  if (cudaMemsetAsync(mn, 0x7F, sizeof(unsigned), x.st) != cudaSuccess) return -1;
  switch (x.p) {
    case 1:
      launch_k(x, k_cfl1_tet<1>, grid, bs, 0, s, x.d->inr, x.ne, est, mn, shadow);
      launch_k(x, k_cfl2_tet<1>, grid, bs, 0, s, x.d->inr, x.ne, cfl, est, mn, bits);
      return 2;
    case 2:
      launch_k(x, k_cfl1_tet<2>, grid, bs, 0, s, x.d->inr, x.ne, est, mn, shadow);
      launch_k(x, k_cfl2_tet<2>, grid, bs, 0, s, x.d->inr, x.ne, cfl, est, mn, bits);
      return 2;
    default: return -1;
  }
}

}  // namespace dgc
