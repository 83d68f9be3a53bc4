// Quadrilateral kernels: Eq. 2 on parallelogram quadrilaterals with the
// tensor-product Legendre space Q_p, phi_{a(p+1)+b}(r, s) = l_a(r) l_b(s) on the
// square [0,1]^2 (l_k(x) = sqrt(2k+1) P_k(2x-1)), edges colored with 4 colors
// (Sec. 3.1, Table 2).  Same structure as the other element types: a lane pair
// per edge, one lane per neighbouring element, the flux exchanged by shuffles,
// plain read-modify-write stores within a color (Algorithm 1).
//
// Edge traces in closed form.  On local edge f the trace of a Q_p function is a
// 1-D series in the edge's free coordinate x (r on edges 0 and 2, s on 1 and 3)
// with the other coordinate fixed at 0 (edges 0, 3) or 1 (edges 1, 2):
//   u|_f(x) = sum_k T_k l_k(x),  T_k = sum_o c_{k,o} l_o(fixed)  (free r)
//                                 T_k = sum_o c_{o,k} l_o(fixed)  (free s)
// A lane forms these p+1 coefficients per variable from its element's block and
// evaluates them at the edge's Gauss points through the uniform 1-D table
// l_k(t_q); the projection onto the element's modes is the transpose, a rank-one
// update c_{a,b} += X_a Y_b per variable.  Edges 2 and 3 run against their free
// coordinate, and the right element runs against its left neighbour; each
// reversal x -> 1 - x multiplies l_k by (-1)^k (the Gauss points and weights are
// symmetric), so a lane carries one parity.  In exact arithmetic this is phi_j at
// the edge points, as Eq. 2 writes it.
//
// FP64 kernels evaluate Eq. 2 as written; FP32 kernels in the perturbation form
// of euler_pert.cuh.  The RK step fuses the volume integral into the first color
// and the stage update into the last (quad_last64 / quad_last32), one variable
// at a time.
#include <cfloat>

#include "dev_util.cuh"
#include "device.cuh"
#include "euler_pert.cuh"
#include "incr_form.cuh"

namespace dgc {

template <int P>
struct QuadDim {
  static constexpr int N1 = P + 1;
  static constexpr int NP = N1 * N1;
  static constexpr int NQV = N1 * N1;
  static constexpr int NQF = 2 * P + 1;
  static constexpr int M = 4;
  static constexpr int NV = M * NP;
  // FP32 record: hi[M], lo[M], modes j >= 1 as [M][NP-1] (a multiple of 4 floats)
  static constexpr int NF = (M * (NP + 1) + 3) / 4 * 4;
};

int quad_record_floats(int p) {
  const int np = (p + 1) * (p + 1);
  return (4 * (np + 1) + 3) / 4 * 4;
}

template <typename T, int P>
struct QuadTab {
  using D = QuadDim<P>;
  T phiV[D::NQV][D::NP];
  T vr[D::NQV][D::NP];  // w_q dphi/dr
  T vs[D::NQV][D::NP];  // w_q dphi/ds
  T Lq[D::NQF][D::N1];  // l_k at the edge points t_q
  T wL[D::NQF][D::N1];  // w_q l_k(t_q), edge weights summing to 1
  T e0[D::N1];          // l_k(0)
  T e1[D::N1];          // l_k(1)
  // the volume rule's 1-D factors: point (i, k) of the square is (x_i, x_k)
  T L1[D::N1][D::N1];   // l_a(x_i)
  T D1[D::N1][D::N1];   // l_a'(x_i)
  T w1[D::N1];          // 1-D weights, summing to 1
};

__constant__ QuadTab<double, 1> cQuadD1;
__constant__ QuadTab<double, 2> cQuadD2;
__constant__ QuadTab<double, 3> cQuadD3;
__constant__ QuadTab<float, 1> cQuadF1;
__constant__ QuadTab<float, 2> cQuadF2;
__constant__ QuadTab<float, 3> cQuadF3;

template <typename T, int P>
__device__ __forceinline__ const QuadTab<T, P>& quad_tab();
template <> __device__ __forceinline__ const QuadTab<double, 1>& quad_tab<double, 1>() { return cQuadD1; }
template <> __device__ __forceinline__ const QuadTab<double, 2>& quad_tab<double, 2>() { return cQuadD2; }
template <> __device__ __forceinline__ const QuadTab<double, 3>& quad_tab<double, 3>() { return cQuadD3; }
template <> __device__ __forceinline__ const QuadTab<float, 1>& quad_tab<float, 1>() { return cQuadF1; }
template <> __device__ __forceinline__ const QuadTab<float, 2>& quad_tab<float, 2>() { return cQuadF2; }
template <> __device__ __forceinline__ const QuadTab<float, 3>& quad_tab<float, 3>() { return cQuadF3; }

template <typename T, int P>
static void fill_quad(QuadTab<T, P>& K, const RefTables& R) {
  using D = QuadDim<P>;
  for (int q = 0; q < D::NQV; ++q)
    for (int j = 0; j < D::NP; ++j) {
      K.phiV[q][j] = (T)R.phiV[q * D::NP + j];
      K.vr[q][j] = (T)(R.vw[q] * R.dphiV[(0 * D::NQV + q) * D::NP + j]);
      K.vs[q][j] = (T)(R.vw[q] * R.dphiV[(1 * D::NQV + q) * D::NP + j]);
    }
  for (int q = 0; q < D::NQF; ++q)
    for (int k = 0; k < D::N1; ++k) {
      K.Lq[q][k] = (T)R.eleg[q * D::N1 + k];
      K.wL[q][k] = (T)(R.fw[q] * R.eleg[q * D::N1 + k]);
    }
  for (int k = 0; k < D::N1; ++k) {
    K.e0[k] = (T)R.lend0[k];
    K.e1[k] = (T)R.lend1[k];
  }
  for (int i = 0; i < D::N1; ++i) {
    K.w1[i] = (T)R.vw1[i];
    for (int a = 0; a < D::N1; ++a) {
      K.L1[i][a] = (T)R.vleg[i * D::N1 + a];
      K.D1[i][a] = (T)R.vdleg[i * D::N1 + a];
    }
  }
}

template <int P>
static void upload_quad_p(const RefTables& R, const void* symD, const void* symF) {
  static QuadTab<double, P> hd;
  static QuadTab<float, P> hf;
  fill_quad(hd, R);
  fill_quad(hf, R);
  if (cudaMemcpyToSymbol(symD, &hd, sizeof hd) != cudaSuccess ||
      cudaMemcpyToSymbol(symF, &hf, sizeof hf) != cudaSuccess)
    throw Error{DGC_ERR_CUDA, "cudaMemcpyToSymbol (quadrilateral tables)"};
}

// The FP32 volume factors with every entry twice, (v, v): operands of the packed
// two-lane FP32 FMA (__ffma2_rn, one instruction for two variables), and the
// projection factors with the point weights folded in.
template <int P>
struct QuadPairTab {
  using D = QuadDim<P>;
  float2 L1[D::N1][D::N1];          // l_a(x_i)
  float2 D1[D::N1][D::N1];          // l_a'(x_i)
  float2 WL[D::N1][D::N1][D::N1];   // w_i w_k l_b(x_k)
  float2 WD[D::N1][D::N1][D::N1];   // w_i w_k l_b'(x_k)
};
__constant__ QuadPairTab<1> cQuadP1;
__constant__ QuadPairTab<2> cQuadP2;
__constant__ QuadPairTab<3> cQuadP3;
template <int P>
__device__ __forceinline__ const QuadPairTab<P>& quad_ptab();
template <> __device__ __forceinline__ const QuadPairTab<1>& quad_ptab<1>() { return cQuadP1; }
template <> __device__ __forceinline__ const QuadPairTab<2>& quad_ptab<2>() { return cQuadP2; }
template <> __device__ __forceinline__ const QuadPairTab<3>& quad_ptab<3>() { return cQuadP3; }

template <int P>
static void upload_quad_pairs(const RefTables& R, const void* sym) {
  using D = QuadDim<P>;
  static QuadTab<float, P> f;
  static QuadPairTab<P> h;
  fill_quad(f, R);
  for (int i = 0; i < D::N1; ++i)
    for (int a = 0; a < D::N1; ++a) {
      h.L1[i][a] = make_float2(f.L1[i][a], f.L1[i][a]);
      h.D1[i][a] = make_float2(f.D1[i][a], f.D1[i][a]);
      for (int b = 0; b < D::N1; ++b) {
        const float wl = f.w1[i] * f.w1[a] * f.L1[a][b], wd = f.w1[i] * f.w1[a] * f.D1[a][b];
        h.WL[i][a][b] = make_float2(wl, wl);
        h.WD[i][a][b] = make_float2(wd, wd);
      }
    }
  if (cudaMemcpyToSymbol(sym, &h, sizeof h) != cudaSuccess)
    throw Error{DGC_ERR_CUDA, "cudaMemcpyToSymbol (quadrilateral pair tables)"};
}

void quad_upload_tables(int p, const RefTables& R) {
  if (!R.quad || R.p != p) return;
  if (p == 1) upload_quad_p<1>(R, &cQuadD1, &cQuadF1);
  if (p == 2) upload_quad_p<2>(R, &cQuadD2, &cQuadF2);
  if (p == 3) upload_quad_p<3>(R, &cQuadD3, &cQuadF3);
  if (p == 1) upload_quad_pairs<1>(R, &cQuadP1);
  if (p == 2) upload_quad_pairs<2>(R, &cQuadP2);
  if (p == 3) upload_quad_pairs<3>(R, &cQuadP3);
}

// ---------------------------------------------------------------------------
// element blocks (16-byte vectors: NV and NF are multiples of 4)
// ---------------------------------------------------------------------------
template <int N>
__device__ __forceinline__ void qload(const double* src, double (&v)[N]) {
  static_assert(N % 2 == 0, "even block");
  const double2* s = reinterpret_cast<const double2*>(src);
#pragma unroll
  for (int i = 0; i < N / 2; ++i) {
    const double2 x = s[i];
    v[2 * i] = x.x;
    v[2 * i + 1] = x.y;
  }
}
template <int N>
__device__ __forceinline__ void qload(const float* src, float (&v)[N]) {
  static_assert(N % 4 == 0, "float4 block");
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
__device__ __forceinline__ void qstore(double* dst, const double (&v)[N]) {
  double2* d = reinterpret_cast<double2*>(dst);
#pragma unroll
  for (int i = 0; i < N / 2; ++i) d[i] = make_double2(v[2 * i], v[2 * i + 1]);
}
template <int N>
__device__ __forceinline__ void qstore(float* dst, const float (&v)[N]) {
  static_assert(N % 4 == 0, "float4 block");
  float4* d = reinterpret_cast<float4*>(dst);
#pragma unroll
  for (int i = 0; i < N / 4; ++i) d[i] = make_float4(v[4 * i], v[4 * i + 1], v[4 * i + 2], v[4 * i + 3]);
}

// ---------------------------------------------------------------------------
// FP32 element state in perturbation form (mean phi_0 c_0 as an FP32 pair)
// ---------------------------------------------------------------------------
template <int P>
struct QuadPert {
  float hi[4], lo[4];
  float cd[4][QuadDim<P>::NP - 1];
};

template <int P>
__device__ __forceinline__ void qload_pert(const double* src, QuadPert<P>& B) {
  using D = QuadDim<P>;
  const double phi0 = quad_tab<double, P>().phiV[0][0];
  double v[D::NV];
  qload(src, v);
#pragma unroll
  for (int m = 0; m < 4; ++m) {
    const double u = phi0 * v[m * D::NP];
    B.hi[m] = d2f(u);
    B.lo[m] = d2f(u - f2d(B.hi[m]));
#pragma unroll
    for (int j = 1; j < D::NP; ++j) B.cd[m][j - 1] = d2f(v[m * D::NP + j]);
  }
}

template <int P>
__device__ __forceinline__ void qload_pert(const float* src, QuadPert<P>& B) {
  using D = QuadDim<P>;
  float v[D::NF];
  qload(src, v);
#pragma unroll
  for (int m = 0; m < 4; ++m) {
    B.hi[m] = v[m];
    B.lo[m] = v[4 + m];
#pragma unroll
    for (int j = 1; j < D::NP; ++j) B.cd[m][j - 1] = v[8 + m * (D::NP - 1) + j - 1];
  }
}

// ---------------------------------------------------------------------------
// FP64 Euler flux, Eq. 2 as written
// ---------------------------------------------------------------------------
// F(U).n for a direction n (any length), the normal velocity u.n and the sound speed
__device__ __forceinline__ void euler2_n(const double* U, double nx, double ny, double* F, double& un, double& c) {
  const double ir = 1.0 / U[0];
  const double u = U[1] * ir, v = U[2] * ir;
  const double p = 0.4 * (U[3] - 0.5 * (U[1] * u + U[2] * v));
  un = u * nx + v * ny;
  c = sqrt(1.4 * p * ir);
  F[0] = U[0] * un;
  F[1] = U[1] * un + p * nx;
  F[2] = U[2] * un + p * ny;
  F[3] = (U[3] + p) * un;
}

// Volume integral sum_q w_q (J^-1 F(U_q)) . grad_ref phi_j, added to acc, by sum
// factorisation over the tensor rule (points (x_i, x_k), weights w_i w_k):
//   U(i, k) = sum_a l_a(x_i) W_{a,k},  W_{a,k} = sum_b c_{a,b} l_b(x_k);
//   acc_{a,b} += sum_i [ l_a'(x_i) A_{i,b} + l_a(x_i) B_{i,b} ],
//   A_{i,b} = sum_k w_i w_k l_b(x_k) F_r(i, k),  B_{i,b} = sum_k w_i w_k l_b'(x_k) F_s(i, k),
// with F_r, F_s the reference-direction fluxes F . grad r, F . grad s.  The same
// sums as point by point over the (p+1)^2 points, in (p+1)^3 FMAs per variable
// and stage instead of (p+1)^4.  c(m, a, b) gives the block.
template <int P, typename F>
__device__ __forceinline__ void quad_volume64(F&& c, const double* ji, double (&acc)[QuadDim<P>::NV]) {
  using D = QuadDim<P>;
  constexpr int NP = D::NP, N1 = D::N1;
  const QuadTab<double, P>& K = quad_tab<double, P>();
  double J[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) J[i] = __ldg(ji + i);
  double W[4][N1][N1];
#pragma unroll
  for (int m = 0; m < 4; ++m)
#pragma unroll
    for (int a = 0; a < N1; ++a)
#pragma unroll
      for (int k = 0; k < N1; ++k) {
        double t = 0.0;
#pragma unroll
        for (int b = 0; b < N1; ++b) t += c(m, a, b) * K.L1[k][b];
        W[m][a][k] = t;
      }
#pragma unroll 1
  for (int i = 0; i < N1; ++i) {
    double A[4][N1], B[4][N1];
#pragma unroll
    for (int m = 0; m < 4; ++m)
#pragma unroll
      for (int b = 0; b < N1; ++b) A[m][b] = B[m][b] = 0.0;
#pragma unroll
    for (int k = 0; k < N1; ++k) {
      double U[4];
#pragma unroll
      for (int m = 0; m < 4; ++m) {
        double t = 0.0;
#pragma unroll
        for (int a = 0; a < N1; ++a) t += K.L1[i][a] * W[m][a][k];
        U[m] = t;
      }
      double Fr[4], Fs[4], un, cs;
      euler2_n(U, J[0], J[1], Fr, un, cs);
      euler2_n(U, J[2], J[3], Fs, un, cs);
      const double w = K.w1[i] * K.w1[k];
#pragma unroll
      for (int m = 0; m < 4; ++m)
#pragma unroll
        for (int b = 0; b < N1; ++b) {
          A[m][b] += (w * K.L1[k][b]) * Fr[m];
          B[m][b] += (w * K.D1[k][b]) * Fs[m];
        }
    }
#pragma unroll
    for (int m = 0; m < 4; ++m)
#pragma unroll
      for (int a = 0; a < N1; ++a)
#pragma unroll
        for (int b = 0; b < N1; ++b) acc[m * NP + a * N1 + b] += K.D1[i][a] * A[m][b] + K.L1[i][a] * B[m][b];
  }
}

// FP32 volume integral in perturbation form, sum-factorised as above: the
// deviation d = u - ub from the modes j >= 1 and lo, F(ub) left out (its
// integral against grad phi_j vanishes), and grad phi_0 = 0.  Variables (0, 1)
// and (2, 3) go in pairs through the packed FP32 FMA (__ffma2_rn).
template <int P>
__device__ __forceinline__ void quad_volume32(const QuadPert<P>& B, const PertRef<2>& R, const double* ji,
                                              float (&acc)[QuadDim<P>::NV]) {
  using D = QuadDim<P>;
  constexpr int NP = D::NP, N1 = D::N1;
  const QuadPairTab<P>& K2 = quad_ptab<P>();
  float J[2][2], th[2];
#pragma unroll
  for (int k = 0; k < 2; ++k) {
    J[k][0] = d2f(__ldg(ji + 2 * k));
    J[k][1] = d2f(__ldg(ji + 2 * k + 1));
    th[k] = R.u[1] * J[k][0] + R.u[2] * J[k][1];
  }
  float2 W[2][N1][N1];  // [pair][a][k]
#pragma unroll
  for (int h = 0; h < 2; ++h)
#pragma unroll
    for (int a = 0; a < N1; ++a)
#pragma unroll
      for (int k = 0; k < N1; ++k) {
        float2 t = make_float2(0.0f, 0.0f);
#pragma unroll
        for (int b = 0; b < N1; ++b)
          if (a + b > 0)
            t = __ffma2_rn(K2.L1[k][b], make_float2(B.cd[2 * h][a * N1 + b - 1], B.cd[2 * h + 1][a * N1 + b - 1]), t);
        W[h][a][k] = t;
      }
  float2 ac[2][NP];
#pragma unroll
  for (int h = 0; h < 2; ++h)
#pragma unroll
    for (int j = 0; j < NP; ++j) ac[h][j] = make_float2(acc[2 * h * NP + j], acc[(2 * h + 1) * NP + j]);
#pragma unroll 1
  for (int i = 0; i < N1; ++i) {
    float2 A[2][N1], Bs[2][N1];
#pragma unroll
    for (int h = 0; h < 2; ++h)
#pragma unroll
      for (int b = 0; b < N1; ++b) A[h][b] = Bs[h][b] = make_float2(0.0f, 0.0f);
#pragma unroll
    for (int k = 0; k < N1; ++k) {
      float2 t01 = make_float2(B.lo[0], B.lo[1]), t23 = make_float2(B.lo[2], B.lo[3]);
#pragma unroll
      for (int a = 0; a < N1; ++a) {
        t01 = __ffma2_rn(K2.L1[i][a], W[0][a][k], t01);
        t23 = __ffma2_rn(K2.L1[i][a], W[1][a][k], t23);
      }
      const float d[4] = {t01.x, t01.y, t23.x, t23.y};
      PertState<2> S;
      S.init(R, d);
      float Fr[4], Fs[4];
      pert_flux<2>(R, S, d, J[0], th[0], Fr);
      pert_flux<2>(R, S, d, J[1], th[1], Fs);
      const float2 r2[2] = {make_float2(Fr[0], Fr[1]), make_float2(Fr[2], Fr[3])};
      const float2 s2[2] = {make_float2(Fs[0], Fs[1]), make_float2(Fs[2], Fs[3])};
#pragma unroll
      for (int h = 0; h < 2; ++h)
#pragma unroll
        for (int b = 0; b < N1; ++b) {
          A[h][b] = __ffma2_rn(K2.WL[i][k][b], r2[h], A[h][b]);
          Bs[h][b] = __ffma2_rn(K2.WD[i][k][b], s2[h], Bs[h][b]);
        }
    }
#pragma unroll
    for (int h = 0; h < 2; ++h)
#pragma unroll
      for (int a = 0; a < N1; ++a)
#pragma unroll
        for (int b = 0; b < N1; ++b)
          if (a + b > 0)
            ac[h][a * N1 + b] = __ffma2_rn(K2.D1[i][a], A[h][b], __ffma2_rn(K2.L1[i][a], Bs[h][b], ac[h][a * N1 + b]));
  }
#pragma unroll
  for (int h = 0; h < 2; ++h)
#pragma unroll
    for (int j = 0; j < NP; ++j) {
      acc[2 * h * NP + j] = ac[h][j].x;
      acc[(2 * h + 1) * NP + j] = ac[h][j].y;
    }
}

template <int P, typename CT, typename ST, typename RT>
__global__ void __launch_bounds__(128) k_vol_quad(const ST* c, int sstride, const double* jinv, RT* rhs, int64_t e0,
                                                  int64_t ne) {
  using D = QuadDim<P>;
  const int64_t e = e0 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= ne) return;
  RT out[D::NV];
  if constexpr (sizeof(CT) == 8) {
    double v[D::NV], acc[D::NV];
    qload(c + e * D::NV, v);
#pragma unroll
    for (int i = 0; i < D::NV; ++i) acc[i] = 0.0;
    quad_volume64<P>([&](int m, int a, int b) { return v[m * D::NP + a * D::N1 + b]; }, jinv + 4 * e, acc);
#pragma unroll
    for (int i = 0; i < D::NV; ++i) out[i] = (RT)acc[i];
  } else {
    const int64_t stride = sizeof(ST) == 8 ? D::NV : sstride;
    QuadPert<P> B;
    qload_pert<P>(c + e * stride, B);
    PertRef<2> R;
    R.init(B.hi);
    float acc[D::NV];
#pragma unroll
    for (int i = 0; i < D::NV; ++i) acc[i] = 0.0f;
    quad_volume32<P>(B, R, jinv + 4 * e, acc);
#pragma unroll
    for (int i = 0; i < D::NV; ++i) out[i] = (RT)acc[i];
  }
  qstore(rhs + e * D::NV, out);
}

// ---------------------------------------------------------------------------
// Surface integral (Algorithm 1): one lane pair per edge
// ---------------------------------------------------------------------------
struct QuadParams {
  int64_t begin, end;
  const int4* topo;
  const double2* fgeo;  // [2k] = unit normal of the left element, [2k+1] = (|f|/detJ_l, |f|/detJ_r)
  const double* jinv;
  const void* state;
  void* rhs;
  void* buf;
  StageArgs sa;
  int sstride;  // floats per element of an FP32 state (record)
};

// One lane's edge: l_o at the fixed coordinate, which coordinate is free
// (s on odd edges) and the parity of the reversals.
template <typename T, int P>
struct QuadEdge {
  T lam[P + 1];
  bool frees, flip;
  __device__ __forceinline__ void init(int f, bool right) {
    const QuadTab<T, P>& K = quad_tab<T, P>();
    const bool fixed0 = f == 0 || f == 3;
#pragma unroll
    for (int k = 0; k <= P; ++k) lam[k] = fixed0 ? K.e0[k] : K.e1[k];
    frees = f & 1;
    flip = (f >= 2) != right;
  }
  // the sign of l_k under the lane's reversals
  __device__ __forceinline__ T sgn(int k) const { return (flip && (k & 1)) ? T(-1) : T(1); }
};

// T[m][k] of a block given as c(m, a, b) (the lane's edge trace coefficients,
// reversal signs included)
template <typename T, int P, typename F>
__device__ __forceinline__ void trace_coeffs(const QuadEdge<T, P>& E, F&& c, T (&Tc)[4][P + 1]) {
#pragma unroll
  for (int m = 0; m < 4; ++m)
#pragma unroll
    for (int k = 0; k <= P; ++k) {
      T te = T(0), to = T(0);
#pragma unroll
      for (int o = 0; o <= P; ++o) {
        te += c(m, k, o) * E.lam[o];
        to += E.lam[o] * c(m, o, k);
      }
      Tc[m][k] = E.sgn(k) * (E.frees ? to : te);
    }
}

// The element's surface contribution c_{a,b} += X_a Y_b from the projected
// flux g[m][k] = sum_q w_q l_k(t_q) G_q and the edge scale, as a functor.
template <typename T, int P>
struct QuadRank1 {
  T X[4][P + 1], Y[4][P + 1];
  __device__ __forceinline__ void init(const QuadEdge<T, P>& E, const T (&g)[4][P + 1], T scale) {
#pragma unroll
    for (int m = 0; m < 4; ++m)
#pragma unroll
      for (int k = 0; k <= P; ++k) {
        const T h = scale * E.sgn(k) * g[m][k];
        X[m][k] = E.frees ? E.lam[k] : h;
        Y[m][k] = E.frees ? h : E.lam[k];
      }
  }
  __device__ __forceinline__ T operator()(int m, int a, int b) const { return X[m][a] * Y[m][b]; }
};

// Loads and stores of one variable's NP values at v (16-byte vectors when the
// row starts on a 16-byte boundary: NP a multiple of 4)
template <int N, typename T>
__device__ __forceinline__ void row_load(const T* v, T (&x)[N]) {
  if constexpr (N % 4 == 0 && sizeof(T) == 4) {
    qload<N>(v, x);
  } else if constexpr (N % 2 == 0 && sizeof(T) == 8) {
    qload<N>(v, x);
  } else {
#pragma unroll
    for (int i = 0; i < N; ++i) x[i] = v[i];
  }
}
template <int N, typename T>
__device__ __forceinline__ void row_store(T* v, const T (&x)[N]) {
  if constexpr (N % 4 == 0 && sizeof(T) == 4) {
    qstore<N>(v, x);
  } else if constexpr (N % 2 == 0 && sizeof(T) == 8) {
    qstore<N>(v, x);
  } else {
#pragma unroll
    for (int i = 0; i < N; ++i) v[i] = x[i];
  }
}

template <int P, typename RT, int MODE, typename AT>
__device__ __forceinline__ void quad_write(const QuadParams& A, int64_t elem, int64_t k, int side,
                                           const QuadRank1<AT, P>& W, const AT* acc) {
  using D = QuadDim<P>;
  constexpr int NV = D::NV, NP = D::NP, N1 = D::N1;
  RT* r = static_cast<RT*>(A.rhs) + elem * NV;
  if constexpr (MODE == SURF_RMW) {
    // one variable at a time: the row's loads, then its stores
#pragma unroll
    for (int m = 0; m < 4; ++m) {
      RT v[NP];
      row_load<NP>(r + m * NP, v);
#pragma unroll
      for (int j = 0; j < NP; ++j) v[j] += (RT)W(m, j / N1, j % N1);
      row_store<NP>(r + m * NP, v);
    }
  } else if constexpr (MODE == SURF_FIRST) {
    RT v[NV];
#pragma unroll
    for (int m = 0; m < 4; ++m)
#pragma unroll
      for (int j = 0; j < NP; ++j) v[m * NP + j] = (RT)(acc[m * NP + j] + W(m, j / N1, j % N1));
    qstore(r, v);
  } else if constexpr (MODE == SURF_ATOMIC) {
#pragma unroll
    for (int m = 0; m < 4; ++m)
#pragma unroll
      for (int j = 0; j < NP; ++j) atomicAdd(r + m * NP + j, (RT)W(m, j / N1, j % N1));
  } else if constexpr (MODE == SURF_BUFFER) {
    RT v[NV];
#pragma unroll
    for (int m = 0; m < 4; ++m)
#pragma unroll
      for (int j = 0; j < NP; ++j) v[m * NP + j] = (RT)W(m, j / N1, j % N1);
    qstore(static_cast<RT*>(A.buf) + (2 * k + side) * NV, v);
  }
}

// Last color, FP64 form: the element's rhs is the stored part plus this edge's
// rank-one term; uout = a0 u0 + b0 (us + dt L), one variable at a time (the
// stage input us is re-read: the lane is the only one touching its element).
template <int P>
__device__ __forceinline__ void quad_last64(const QuadParams& A, int64_t elem, const QuadRank1<double, P>& W) {
  using D = QuadDim<P>;
  constexpr int NP = D::NP, NV = D::NV, N1 = D::N1;
  const double dt = *A.sa.dt, a0 = A.sa.a0, b0 = A.sa.b0, bdt = b0 * dt;
  const double* part = static_cast<const double*>(A.rhs) + elem * NV;
  const double* us = static_cast<const double*>(A.state) + elem * NV;
  const double* u0 = A.sa.u0 + elem * NV;
  double* out = A.sa.uout + elem * NV;
#pragma unroll
  for (int m = 0; m < 4; ++m) {
    double L[NP], u[NP], z[NP];
    row_load<NP>(part + m * NP, L);
    row_load<NP>(us + m * NP, u);
    if (a0 != 0.0) row_load<NP>(u0 + m * NP, z);
#pragma unroll
    for (int j = 0; j < NP; ++j) {
      const double Lj = L[j] + W(m, j / N1, j % N1);
      L[j] = a0 == 0.0 ? fma(bdt, Lj, b0 == 1.0 ? u[j] : b0 * u[j]) : fma(bdt, Lj, fma(a0, z[j], b0 * u[j]));
    }
    row_store<NP>(out + m * NP, L);
  }
}

// Last color, FP32 increment form of the step (incr_form.cuh), one variable at a
// time: stages 0 and 1 write the increment and the record of the next stage's
// state (from the record of u0), stage 2 updates the FP64 state.
template <int P>
__device__ __forceinline__ void quad_last32(const QuadParams& A, int64_t elem, const QuadRank1<float, P>& W) {
  using D = QuadDim<P>;
  constexpr int NP = D::NP, NV = D::NV, N1 = D::N1, NF = D::NF;
  const StageArgs& S = A.sa;
  const F2 dtp = split_f2(*S.dt);
  const float* part = static_cast<const float*>(A.rhs) + elem * NV;
  float* dp = S.delta + elem * NV;
  if (S.stage < 2) {
    const F2 p0 = split_f2(quad_tab<double, P>().phiV[0][0]);
    float r[NF];
    qload<NF>(S.rec0 + elem * S.rec0_stride, r);
#pragma unroll
    for (int m = 0; m < 4; ++m) {
      float d[NP];
      row_load<NP>(part + m * NP, d);
      if (S.stage == 0) {
#pragma unroll
        for (int j = 0; j < NP; ++j) d[j] = mul_f2(d[j] + W(m, j / N1, j % N1), dtp);
      } else {
        float d0[NP];
        row_load<NP>(dp + m * NP, d0);
#pragma unroll
        for (int j = 0; j < NP; ++j) d[j] = 0.25f * (d0[j] + mul_f2(d[j] + W(m, j / N1, j % N1), dtp));
      }
      pair_add_scaled(r[m], r[4 + m], d[0], p0);
#pragma unroll
      for (int j = 1; j < NP; ++j) r[8 + m * (NP - 1) + j - 1] += d[j];
      row_store<NP>(dp + m * NP, d);
    }
    qstore<NF>(S.rec_out + elem * NF, r);
    return;
  }
  // stage 2: delta_2 + dt L; b_2 = 2/3 is applied by the state update
#pragma unroll
  for (int m = 0; m < 4; ++m) {
    float d[NP], d0[NP];
    double z[NP];
    row_load<NP>(part + m * NP, d);
    row_load<NP>(dp + m * NP, d0);
    row_load<NP>(S.u0 + elem * NV + m * NP, z);
#pragma unroll
    for (int j = 0; j < NP; ++j) z[j] = fma(2.0 / 3.0, f2d(d0[j] + mul_f2(d[j] + W(m, j / N1, j % N1), dtp)), z[j]);
    row_store<NP>(S.uout + elem * NV + m * NP, z);
  }
}

// Register cap of the FP32 surface kernels other than the first color: none by
// default.  The middle colors take 121 registers and keep the whole record in
// flight; capped at 96 (five blocks of 128 threads per SM instead of four) they
// measured slower (0.125 -> 0.142 ms at 810 x 810, p = 3).
#ifndef DGC_QUAD_REGS
#define DGC_QUAD_REGS 255
#endif

template <int P, typename CT, typename ST, typename RT, int MODE>
__global__ void __launch_bounds__(256)
    __maxnreg__((sizeof(CT) == 4 && MODE != SURF_FIRST ? DGC_QUAD_REGS : 255)) k_surf_quad(const QuadParams A) {
  using D = QuadDim<P>;
  constexpr int NP = D::NP, NQ = D::NQF, NV = D::NV, N1 = D::N1;
  // programmatic launch (dev_util.cuh): the first color overwrites the rhs its
  // predecessor may still read, so it waits at once; the other colors wait
  // before their epilogue, which reads the predecessor's rhs
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
  const bool writer = valid && !(side && bnd);
  const double2 g0 = A.fgeo[2 * k], g1 = A.fgeo[2 * k + 1];

  if constexpr (sizeof(CT) == 8) {
    const QuadTab<double, P>& K = quad_tab<double, P>();
    QuadEdge<double, P> E;
    E.init(lf, right);
    const double* cs = static_cast<const double*>(A.state) + elem * NV;
    double acc[MODE == SURF_FIRST ? NV : 1];
    double Tc[4][N1];
    if constexpr (MODE == SURF_FIRST) {
      double c[NV];
      qload(cs, c);
#pragma unroll
      for (int i = 0; i < NV; ++i) acc[i] = 0.0;
      trace_coeffs<double, P>(E, [&](int m, int a, int b) { return c[m * NP + a * N1 + b]; }, Tc);
      quad_volume64<P>([&](int m, int a, int b) { return c[m * NP + a * N1 + b]; }, A.jinv + 4 * elem, acc);
    } else {
      double c[NV];
      qload(cs, c);
      trace_coeffs<double, P>(E, [&](int m, int a, int b) { return c[m * NP + a * N1 + b]; }, Tc);
    }
    double g[4][N1];
#pragma unroll
    for (int m = 0; m < 4; ++m)
#pragma unroll
      for (int kk = 0; kk < N1; ++kk) g[m][kk] = 0.0;
#pragma unroll 1
    for (int q = 0; q < NQ; ++q) {
      double U[4], V[4], Fo[4], Fp[4], uno, co;
#pragma unroll
      for (int m = 0; m < 4; ++m) {
        double s = 0.0;
#pragma unroll
        for (int kk = 0; kk < N1; ++kk) s += Tc[m][kk] * K.Lq[q][kk];
        U[m] = s;
      }
      // each lane evaluates its own side and exchanges the normal flux and the
      // wave speed with its partner; the sums below are commutative, so both
      // lanes get the same bits
      euler2_n(U, g0.x, g0.y, Fo, uno, co);
      const double wo = fabs(uno) + co;
#pragma unroll
      for (int m = 0; m < 4; ++m) {
        V[m] = __shfl_xor_sync(0xffffffffu, U[m], 1);
        Fp[m] = __shfl_xor_sync(0xffffffffu, Fo[m], 1);
      }
      const double lam = fmax(wo, __shfl_xor_sync(0xffffffffu, wo, 1));
#pragma unroll
      for (int m = 0; m < 4; ++m) {
        const double a = side ? V[m] : U[m], b = side ? U[m] : V[m];
        const double Fs = 0.5 * (Fo[m] + Fp[m]) - (0.5 * lam) * (b - a);
#pragma unroll
        for (int kk = 0; kk < N1; ++kk) g[m][kk] += K.wL[q][kk] * Fs;
      }
    }
    QuadRank1<double, P> W;
    W.init(E, g, right ? g1.y : -g1.x);
    if constexpr (MODE != SURF_FIRST) {
      pdl_wait();
      pdl_trigger();
    }
    if constexpr (MODE == SURF_LAST) {
      if (writer) quad_last64<P>(A, elem, W);
    } else if (writer) {
      quad_write<P, RT, MODE>(A, elem, k, side, W, acc);
    }
  } else {
    const QuadTab<float, P>& K = quad_tab<float, P>();
    QuadEdge<float, P> E;
    E.init(lf, right);
    const int64_t stride = sizeof(ST) == 8 ? NV : A.sstride;
    QuadPert<P> B;
    qload_pert<P>(static_cast<const ST*>(A.state) + elem * stride, B);
    PertRef<2> R;
    R.init(B.hi);
    // own trace minus ub: the modes j >= 1, and lo on the constant (l_0 = 1)
    float Tc[4][N1];
    trace_coeffs<float, P>(
        E,
        [&](int m, int a, int b) {
          const int j = a * N1 + b;
          return j > 0 ? B.cd[m][j > 0 ? j - 1 : 0] : 0.0f;
        },
        Tc);
#pragma unroll
    for (int m = 0; m < 4; ++m) Tc[m][0] += B.lo[m];
    float acc[MODE == SURF_FIRST ? NV : 1];
    if constexpr (MODE == SURF_FIRST) {
#pragma unroll
      for (int i = 0; i < NV; ++i) acc[i] = 0.0f;
      quad_volume32<P>(B, R, A.jinv + 4 * elem, acc);
    }
    FaceConst<2> F;
    F.init(R, B.hi, {d2f(g0.x), d2f(g0.y)}, side);
    float g[4][N1];
#pragma unroll
    for (int m = 0; m < 4; ++m)
#pragma unroll
      for (int kk = 0; kk < N1; ++kk) g[m][kk] = 0.0f;
#pragma unroll 1
    for (int q = 0; q < NQ; ++q) {
      float ds[4], G[4];
#pragma unroll
      for (int m = 0; m < 4; ++m) {
        float s = 0.0f;
#pragma unroll
        for (int kk = 0; kk < N1; ++kk) s += Tc[m][kk] * K.Lq[q][kk];
        ds[m] = s;
      }
      lf_exchange<2>(R, F, ds, G);
#pragma unroll
      for (int m = 0; m < 4; ++m)
#pragma unroll
        for (int kk = 0; kk < N1; ++kk) g[m][kk] += K.wL[q][kk] * G[m];
    }
    QuadRank1<float, P> W;
    W.init(E, g, right ? d2f(g1.y) : -d2f(g1.x));
    if constexpr (MODE != SURF_FIRST) {
      pdl_wait();
      pdl_trigger();
    }
    if constexpr (MODE == SURF_LAST) {
      if (writer) quad_last32<P>(A, elem, W);
    } else if (writer) {
      quad_write<P, RT, MODE>(A, elem, k, side, W, acc);
    }
  }
}

// ---------------------------------------------------------------------------
// CFL reduction in two passes, as for the other element types: FP32 estimates
// of every element, then FP64 only for the elements within kCflMargin of the
// minimum.
// ---------------------------------------------------------------------------
// FP32 estimate of max_q (|u| + c) from the FP32 record (mean pair + modes)
template <int P>
__device__ __forceinline__ float quad_lambda_rec(const float (&r)[QuadDim<P>::NF]) {
  using D = QuadDim<P>;
  constexpr int NP = D::NP;
  const QuadTab<float, P>& K = quad_tab<float, P>();
  float lam = 0.0f;
#pragma unroll 1
  for (int q = 0; q < D::NQV; ++q) {
    float U[4];
#pragma unroll
    for (int m = 0; m < 4; ++m) {
      float s = r[4 + m];
#pragma unroll
      for (int j = 1; j < NP; ++j) s += K.phiV[q][j] * r[8 + m * (NP - 1) + j - 1];
      U[m] = r[m] + s;
    }
    const float ir = rcp_fast(U[0]), u = U[1] * ir, w = U[2] * ir;
    const float q2 = u * u + w * w;
    const float pr = 0.4f * (U[3] - 0.5f * U[0] * q2);
    lam = fmaxf(lam, sqrt_fast(q2) + sqrt_fast(1.4f * pr * ir));
  }
  return lam;
}

// pass 1: the element's record (written when shadow is set) and its FP32 estimate
template <int P>
__global__ void __launch_bounds__(128) k_cfl1_quad(const double* c, const double* inr, int64_t ne, float* est,
                                                   unsigned* minbits, float* shadow) {
  using D = QuadDim<P>;
  constexpr int NP = D::NP;
  pdl_wait();
  pdl_trigger();
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  float best = FLT_MAX;
  if (e < ne) {
    const double phi0 = quad_tab<double, P>().phiV[0][0];
    float r[D::NF];
#pragma unroll
    for (int m = 0; m < 4; ++m) {
      double v[NP];
      row_load<NP>(c + e * D::NV + m * NP, v);
      const double u = phi0 * v[0];
      r[m] = d2f(u);
      r[4 + m] = d2f(u - f2d(r[m]));
#pragma unroll
      for (int j = 1; j < NP; ++j) r[8 + m * (NP - 1) + j - 1] = d2f(v[j]);
    }
#pragma unroll
    for (int i = 4 * (NP + 1); i < D::NF; ++i) r[i] = 0.0f;
    if (shadow) qstore(shadow + e * D::NF, r);
    float d = d2f(inr[e]) / ((2 * P + 1) * quad_lambda_rec<P>(r));
    if (!(d > 0.0f) || !(d < FLT_MAX)) d = 0.0f;  // non-physical: always re-evaluated
    est[e] = d;
    best = d;
  }
  block_min_to(best, minbits);
}

// Pass 2: each candidate is evaluated in FP64 by the whole warp, one volume
// point per lane.
template <int P>
__global__ void __launch_bounds__(128) k_cfl2_quad(const double* c, const double* inr, int64_t ne, double cfl,
                                                   const float* est, const unsigned* minbits,
                                                   unsigned long long* dtbits) {
  using D = QuadDim<P>;
  constexpr int NP = D::NP;
  pdl_wait();
  pdl_trigger();
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const bool cand = e < ne && est[e] <= __uint_as_float(*minbits) * (1.0f + kCflMargin);
  unsigned mask = __ballot_sync(0xffffffffu, cand);
  double best = DBL_MAX;
  const QuadTab<double, P>& K = quad_tab<double, P>();
  while (mask) {
    const int src = __ffs(mask) - 1;
    mask &= mask - 1;
    const long long ec = __shfl_sync(0xffffffffu, (long long)e, src);
    double lam = 0.0;
    for (int q = threadIdx.x & 31; q < D::NQV; q += 32) {
      double U[4];
#pragma unroll
      for (int m = 0; m < 4; ++m) {
        double sum = 0.0;
#pragma unroll
        for (int j = 0; j < NP; ++j) sum += K.phiV[q][j] * c[ec * D::NV + m * NP + j];
        U[m] = sum;
      }
      const double ir = 1.0 / U[0], u = U[1] * ir, w = U[2] * ir;
      const double q2 = u * u + w * w;
      const double pr = 0.4 * (U[3] - 0.5 * U[0] * q2);
      lam = fmax(lam, sqrt(q2) + sqrt(1.4 * pr * ir));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) lam = fmax(lam, __shfl_xor_sync(0xffffffffu, lam, o));
    const double b = cfl * (inr[ec] / ((2 * P + 1) * lam));
    if ((threadIdx.x & 31) == src) best = b > 0.0 ? b : DBL_MAX;  // non-physical state: excluded (NaN)
  }
  block_min_to(best, dtbits);
}

// ---------------------------------------------------------------------------
template <int P, typename CT, typename ST, typename RT>
static int qvol_p(const Ctx& x, const void* s, int ss, void* r, int64_t e0) {
  const int bs = 128;
  const int64_t n = x.ne - e0;
  if (n <= 0) return 0;
  k_vol_quad<P, CT, ST, RT><<<(unsigned)((n + bs - 1) / bs), bs, 0, x.st>>>(
      static_cast<const ST*>(s), ss, x.d->jinv, static_cast<RT*>(r), e0, x.ne);
  return 1;
}

int quad_volume(const Ctx& x, TypeCfg ty, const void* s, int ss, void* r, int64_t e0) {
  switch (x.p * 4 + ty) {
    case 4 + TY_D: return qvol_p<1, double, double, double>(x, s, ss, r, e0);
    case 8 + TY_D: return qvol_p<2, double, double, double>(x, s, ss, r, e0);
    case 12 + TY_D: return qvol_p<3, double, double, double>(x, s, ss, r, e0);
    case 4 + TY_MD: return qvol_p<1, float, double, double>(x, s, ss, r, e0);
    case 8 + TY_MD: return qvol_p<2, float, double, double>(x, s, ss, r, e0);
    case 12 + TY_MD: return qvol_p<3, float, double, double>(x, s, ss, r, e0);
    case 4 + TY_MF: return qvol_p<1, float, float, float>(x, s, ss, r, e0);
    case 8 + TY_MF: return qvol_p<2, float, float, float>(x, s, ss, r, e0);
    case 12 + TY_MF: return qvol_p<3, float, float, float>(x, s, ss, r, e0);
    default: return -1;
  }
}

template <int P, typename CT, typename ST, typename RT, int MODE>
static int qsurf_launch(const Ctx& x, const QuadParams& A) {
  const int64_t n = A.end - A.begin;
  if (n <= 0) return 0;
  const int threads = 2 * x.epb;
  launch_k(x, k_surf_quad<P, CT, ST, RT, MODE>, (unsigned)((2 * n + threads - 1) / threads), (unsigned)threads, 0,
           A);
  return 1;
}

template <int P, typename CT, typename ST, typename RT>
static int qsurf_mode(const Ctx& x, SurfMode mode, const QuadParams& A) {
  switch (mode) {
    case SURF_RMW: return qsurf_launch<P, CT, ST, RT, SURF_RMW>(x, A);
    case SURF_FIRST: return qsurf_launch<P, CT, ST, RT, SURF_FIRST>(x, A);
    case SURF_ATOMIC: return qsurf_launch<P, CT, ST, RT, SURF_ATOMIC>(x, A);
    case SURF_BUFFER: return qsurf_launch<P, CT, ST, RT, SURF_BUFFER>(x, A);
    default: return -1;
  }
}

template <int P>
static int qsurf_p(const Ctx& x, TypeCfg ty, SurfMode mode, const QuadParams& A) {
  if (mode == SURF_LAST) {
    if (ty == TY_D) return qsurf_launch<P, double, double, double, SURF_LAST>(x, A);
    if (ty == TY_MF && A.sa.kstate == nullptr) return qsurf_launch<P, float, float, float, SURF_LAST>(x, A);
    return -1;
  }
  switch (ty) {
    case TY_D: return qsurf_mode<P, double, double, double>(x, mode, A);
    case TY_MD: return qsurf_mode<P, float, double, double>(x, mode, A);
    case TY_MF:
      if (mode != SURF_RMW && mode != SURF_FIRST) return -1;
      return qsurf_mode<P, float, float, float>(x, mode, A);
    default: return -1;
  }
}

int quad_surface(const Ctx& x, TypeCfg ty, SurfMode mode, int64_t begin, int64_t end, const void* state,
                 int sstride, void* rhs, void* buf, const StageArgs* sa) {
  QuadParams A;
  A.begin = begin;
  A.end = end;
  A.sstride = sstride;
  A.topo = x.d->topo;
  A.fgeo = x.d->fgeo;
  A.jinv = x.d->jinv;
  A.state = state;
  A.rhs = rhs;
  A.buf = buf;
  if (sa) A.sa = *sa;
  switch (x.p) {
    case 1: return qsurf_p<1>(x, ty, mode, A);
    case 2: return qsurf_p<2>(x, ty, mode, A);
    case 3: return qsurf_p<3>(x, ty, mode, A);
    default: return -1;
  }
}

int quad_cfl(const Ctx& x, const double* s, double cfl, double* dt, float* shadow) {
  const int bs = 128;
  const unsigned grid = (unsigned)((x.ne + bs - 1) / bs);
  auto* bits = reinterpret_cast<unsigned long long*>(dt);
  float* est = x.d->cfl_est;
  unsigned* mn = reinterpret_cast<unsigned*>(x.d->cfl_est + x.ne);
  if (cudaMemsetAsync(mn, 0x7F, sizeof(unsigned), x.st) != cudaSuccess) return -1;
  switch (x.p) {
    case 1:
      launch_k(x, k_cfl1_quad<1>, grid, bs, 0, s, x.d->inr, x.ne, est, mn, shadow);
      launch_k(x, k_cfl2_quad<1>, grid, bs, 0, s, x.d->inr, x.ne, cfl, est, mn, bits);
      return 2;
    case 2:
      launch_k(x, k_cfl1_quad<2>, grid, bs, 0, s, x.d->inr, x.ne, est, mn, shadow);
      launch_k(x, k_cfl2_quad<2>, grid, bs, 0, s, x.d->inr, x.ne, cfl, est, mn, bits);
      return 2;
    case 3:
      launch_k(x, k_cfl1_quad<3>, grid, bs, 0, s, x.d->inr, x.ne, est, mn, shadow);
      launch_k(x, k_cfl2_quad<3>, grid, bs, 0, s, x.d->inr, x.ne, cfl, est, mn, bits);
      return 2;
    default: return -1;
  }
}

}  // namespace dgc
