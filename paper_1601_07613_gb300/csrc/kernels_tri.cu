// Triangle kernels: volume integral, colored surface integral (Algorithm 1),
// the atomic / per-edge-buffer comparators and the FP64 CFL reduction.
//
// Eq. 2 with a basis orthonormal on the reference triangle (mass = detJ I):
//   dc_j/dt = sum_q w_q F(U_q).(J^-T grad phi_j)(x_q)
//           - sum_faces |f|/detJ sum_q w_q phi_j(x_q) F*(U-, U+, n).
// Each edge k is handled by a lane pair: the even lane owns the left element,
// the odd lane the right one.  A lane loads its element's modal block with
// 16-byte vector loads, evaluates its trace at the edge points, exchanges it
// with its partner by one shuffle per component, both lanes evaluate the
// Lax-Friedrichs flux, and each projects it onto its own element.  Within one
// color no two edges share an element, so the lanes update rhs with plain
// loads and stores (Sec. 1, Algorithm 1): no atomics, no scratch buffer.
#include <cfloat>

#include "device.cuh"

namespace dgc {

template <int P>
struct TriDim {
  static constexpr int NP = (P + 1) * (P + 2) / 2;
  static constexpr int NQV = (P + 1) * (P + 1);
  static constexpr int NQE = 2 * P + 1;
  static constexpr int M = 4;
  static constexpr int NV = M * NP;
};

template <typename T, int P>
struct TriTab {
  T phiV[TriDim<P>::NQV][TriDim<P>::NP];  // phi_j at volume points
  T vr[TriDim<P>::NQV][TriDim<P>::NP];    // w_q dphi_j/dr
  T vs[TriDim<P>::NQV][TriDim<P>::NP];    // w_q dphi_j/ds
  T phiE[3][TriDim<P>::NQE][TriDim<P>::NP];  // phi_j at the points of local edge 0..2
  T wE[TriDim<P>::NQE];                      // edge weights, sum 1
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
  for (int q = 0; q < D::NQE; ++q) K.wE[q] = (T)R.fw[q];
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

void tri_upload_tables(int p, const RefTables& R) {
  if (R.dim != 2 || R.p != p) return;
  if (p == 1) upload_p<1>(R, &cTriD1, &cTriF1);
  if (p == 2) upload_p<2>(R, &cTriD2, &cTriF2);
  if (p == 3) upload_p<3>(R, &cTriD3, &cTriF3);
}

// ---------------------------------------------------------------------------
// state loads / stores (the element block is M*Np contiguous values)
// ---------------------------------------------------------------------------
template <typename CT, int N>
__device__ __forceinline__ void load_block(const double* __restrict__ src, CT (&v)[N]) {
  static_assert(N % 2 == 0, "even block");
  const double2* s = reinterpret_cast<const double2*>(src);
#pragma unroll
  for (int i = 0; i < N / 2; ++i) {
    double2 x = __ldg(s + i);
    v[2 * i] = (CT)x.x;
    v[2 * i + 1] = (CT)x.y;
  }
}
template <typename CT, int N>
__device__ __forceinline__ void load_block(const float* __restrict__ src, CT (&v)[N]) {
  static_assert(N % 4 == 0, "block of float4");
  const float4* s = reinterpret_cast<const float4*>(src);
#pragma unroll
  for (int i = 0; i < N / 4; ++i) {
    float4 x = __ldg(s + i);
    v[4 * i] = (CT)x.x;
    v[4 * i + 1] = (CT)x.y;
    v[4 * i + 2] = (CT)x.z;
    v[4 * i + 3] = (CT)x.w;
  }
}
// plain (coherent) loads, for blocks another kernel of the same stream wrote
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
// Euler fluxes (gamma = 1.4)
// ---------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ void euler_xy(const T* U, T* F, T* G) {
  const T ir = T(1) / U[0];
  const T u = U[1] * ir, v = U[2] * ir;
  const T p = T(0.4) * (U[3] - T(0.5) * (U[1] * u + U[2] * v));
  F[0] = U[1];
  F[1] = U[1] * u + p;
  F[2] = U[2] * u;
  F[3] = (U[3] + p) * u;
  G[0] = U[2];
  G[1] = U[1] * v;
  G[2] = U[2] * v + p;
  G[3] = (U[3] + p) * v;
}

// local Lax-Friedrichs (Rusanov) flux F*(a, b, n) = (F(a).n + F(b).n)/2 - lam (b - a)/2
template <typename T>
__device__ __forceinline__ void lf_flux(const T* a, const T* b, T nx, T ny, T* Fs) {
  const T ia = T(1) / a[0], ib = T(1) / b[0];
  const T ua = a[1] * ia, va = a[2] * ia, ub = b[1] * ib, vb = b[2] * ib;
  const T pa = T(0.4) * (a[3] - T(0.5) * (a[1] * ua + a[2] * va));
  const T pb = T(0.4) * (b[3] - T(0.5) * (b[1] * ub + b[2] * vb));
  const T una = ua * nx + va * ny, unb = ub * nx + vb * ny;
  const T ca = sqrt(T(1.4) * pa * ia), cb = sqrt(T(1.4) * pb * ib);
  const T lam = fmax(fabs(una) + ca, fabs(unb) + cb);
  const T h = T(0.5), hl = T(0.5) * lam;
  Fs[0] = h * (a[0] * una + b[0] * unb) - hl * (b[0] - a[0]);
  Fs[1] = h * (a[1] * una + pa * nx + b[1] * unb + pb * nx) - hl * (b[1] - a[1]);
  Fs[2] = h * (a[2] * una + pa * ny + b[2] * unb + pb * ny) - hl * (b[2] - a[2]);
  Fs[3] = h * ((a[3] + pa) * una + (b[3] + pb) * unb) - hl * (b[3] - a[3]);
}

// acc += volume integral of element with state c and inverse Jacobian ji
template <int P, typename CT>
__device__ __forceinline__ void volume_acc(const CT (&c)[TriDim<P>::NV], const double* __restrict__ ji,
                                           CT (&acc)[TriDim<P>::NV]) {
  using D = TriDim<P>;
  constexpr int NP = D::NP;
  const TriTab<CT, P>& K = tri_tab<CT, P>();
  const double2 j0 = __ldg(reinterpret_cast<const double2*>(ji));
  const double2 j1 = __ldg(reinterpret_cast<const double2*>(ji) + 1);
  const CT rx = (CT)j0.x, ry = (CT)j0.y, sx = (CT)j1.x, sy = (CT)j1.y;
#pragma unroll
  for (int q = 0; q < D::NQV; ++q) {
    CT U[4];
#pragma unroll
    for (int m = 0; m < 4; ++m) {
      CT s = CT(0);
#pragma unroll
      for (int j = 0; j < NP; ++j) s += K.phiV[q][j] * c[m * NP + j];
      U[m] = s;
    }
    CT F[4], G[4];
    euler_xy(U, F, G);
#pragma unroll
    for (int m = 0; m < 4; ++m) {
      const CT fr = rx * F[m] + ry * G[m];
      const CT fs = sx * F[m] + sy * G[m];
#pragma unroll
      for (int j = 0; j < NP; ++j) acc[m * NP + j] += K.vr[q][j] * fr + K.vs[q][j] * fs;
    }
  }
}

// ---------------------------------------------------------------------------
// Volume kernel: one thread per element, rhs = volume integral (plain store).
// ---------------------------------------------------------------------------
template <int P, typename CT, typename ST, typename RT>
__global__ void __launch_bounds__(128) k_vol_tri(const ST* __restrict__ c, const double* __restrict__ jinv,
                                                 RT* __restrict__ rhs, int64_t ne) {
  using D = TriDim<P>;
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= ne) return;
  CT v[D::NV], acc[D::NV];
  load_block(c + e * D::NV, v);
#pragma unroll
  for (int i = 0; i < D::NV; ++i) acc[i] = CT(0);
  volume_acc<P>(v, jinv + 4 * e, acc);
  RT out[D::NV];
#pragma unroll
  for (int i = 0; i < D::NV; ++i) out[i] = (RT)acc[i];
  store_block(rhs + e * D::NV, out);
}

// ---------------------------------------------------------------------------
// Surface kernel for one color (or all edges for the atomic comparator).
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
};

template <int P, typename CT, typename ST, typename RT, int MODE>
__global__ void __launch_bounds__(256) k_surf_tri(const SurfParams A) {
  using D = TriDim<P>;
  constexpr int NP = D::NP, NQ = D::NQE, NV = D::NV;
  __shared__ CT sphi[3 * NQ * NP];
  __shared__ CT sw[NQ];
  {
    const TriTab<CT, P>& K = tri_tab<CT, P>();
    const CT* src = &K.phiE[0][0][0];
    for (int i = threadIdx.x; i < 3 * NQ * NP; i += blockDim.x) sphi[i] = src[i];
    if (threadIdx.x < NQ) sw[threadIdx.x] = K.wE[threadIdx.x];
  }
  __syncthreads();

  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  int64_t k = A.begin + (t >> 1);
  const int side = (int)(t & 1);
  const bool valid = k < A.end;
  if (!valid) k = A.end - 1;  // idle lanes shadow the last edge so both lanes of a pair shuffle
  const int4 tp = A.topo[k];
  const bool bnd = tp.y < 0;       // boundary: both lanes read the left element (U+ = U-)
  const bool right = side && !bnd;
  const int64_t elem = right ? tp.y : tp.x;
  const int le = right ? ((tp.z >> 4) & 15) : (tp.z & 15);
  const bool writer = valid && !(side && bnd);

  CT c[NV];
  if constexpr (MODE == SURF_LAST) {
    double tmp[NV];
    load_plain(static_cast<const double*>(A.state) + elem * NV, tmp);
#pragma unroll
    for (int i = 0; i < NV; ++i) c[i] = (CT)tmp[i];
  } else {
    load_block(static_cast<const ST*>(A.state) + elem * NV, c);
  }
  CT acc[NV];
#pragma unroll
  for (int i = 0; i < NV; ++i) acc[i] = CT(0);
  if constexpr (MODE == SURF_FIRST) volume_acc<P>(c, A.jinv + 4 * elem, acc);

  const double2 g0 = A.fgeo[2 * k], g1 = A.fgeo[2 * k + 1];
  const CT nx = (CT)g0.x, ny = (CT)g0.y;
  const CT scale = right ? (CT)g1.y : -(CT)g1.x;
  const CT* ph = sphi + le * NQ * NP;

#pragma unroll
  for (int q = 0; q < NQ; ++q) {
    const int qq = right ? NQ - 1 - q : q;  // the right element runs along the edge backwards
    CT phi[NP];
#pragma unroll
    for (int j = 0; j < NP; ++j) phi[j] = ph[qq * NP + j];
    CT U[4], V[4];
#pragma unroll
    for (int m = 0; m < 4; ++m) {
      CT s = CT(0);
#pragma unroll
      for (int j = 0; j < NP; ++j) s += phi[j] * c[m * NP + j];
      U[m] = s;
    }
#pragma unroll
    for (int m = 0; m < 4; ++m) V[m] = __shfl_xor_sync(0xffffffffu, U[m], 1);
    CT a[4], b[4], Fs[4];
#pragma unroll
    for (int m = 0; m < 4; ++m) {
      a[m] = side ? V[m] : U[m];  // left trace
      b[m] = side ? U[m] : V[m];  // right trace
    }
    lf_flux(a, b, nx, ny, Fs);
    const CT s = scale * sw[q];
#pragma unroll
    for (int m = 0; m < 4; ++m) {
      const CT g = s * Fs[m];
#pragma unroll
      for (int j = 0; j < NP; ++j) acc[m * NP + j] += phi[j] * g;
    }
  }
  if (!writer) return;

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
  } else {  // SURF_LAST: rhs = partial + this color; stage update in FP64
    RT part[NV];
    load_plain(static_cast<const RT*>(A.rhs) + elem * NV, part);
    const double dt = *A.sa.dt;
    const double a0 = A.sa.a0, b0 = A.sa.b0;
    double us[NV], u[NV];
    load_plain(static_cast<const double*>(A.state) + elem * NV, us);
    if (a0 != 0.0) load_plain(A.sa.u0 + elem * NV, u);
#pragma unroll
    for (int i = 0; i < NV; ++i) {
      const double L = (double)part[i] + (double)acc[i];
      const double v = b0 * (us[i] + dt * L);
      u[i] = a0 != 0.0 ? a0 * u[i] + v : v;
    }
    store_block(A.sa.uout + elem * NV, u);
    if (A.sa.shadow) {
      float f[NV];
#pragma unroll
      for (int i = 0; i < NV; ++i) f[i] = (float)u[i];
      store_block(A.sa.shadow + elem * NV, f);
    }
  }
}

// ---------------------------------------------------------------------------
// CFL reduction, FP64: dt = cfl min_e r_e / ((2p+1) max_q (|u| + c)).
// Positive doubles order like their bit patterns, so the block minima are
// combined with one 64-bit atomicMin; dt must hold a large value beforehand.
// Optionally writes the FP32 copy of the state (mixed precision).
// ---------------------------------------------------------------------------
template <int P>
__global__ void __launch_bounds__(128) k_cfl_tri(const double* __restrict__ c, const double* __restrict__ inr,
                                                 int64_t ne, double cfl, unsigned long long* dtbits,
                                                 float* __restrict__ shadow) {
  using D = TriDim<P>;
  constexpr int NP = D::NP;
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  double best = DBL_MAX;
  if (e < ne) {
    double v[D::NV];
    load_block(c + e * D::NV, v);
    if (shadow) {
      float f[D::NV];
#pragma unroll
      for (int i = 0; i < D::NV; ++i) f[i] = (float)v[i];
      store_block(shadow + e * D::NV, f);
    }
    const TriTab<double, P>& K = tri_tab<double, P>();
    double lam = 0.0;
#pragma unroll
    for (int q = 0; q < D::NQV; ++q) {
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
    best = cfl * (__ldg(inr + e) / ((2 * P + 1) * lam));
    if (!(best > 0.0)) best = DBL_MAX;  // non-physical state: excluded (NaN)
  }
  // block minimum
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) best = fmin(best, __shfl_xor_sync(0xffffffffu, best, o));
  __shared__ double wmin[32];
  if ((threadIdx.x & 31) == 0) wmin[threadIdx.x >> 5] = best;
  __syncthreads();
  if (threadIdx.x == 0) {
    double b = wmin[0];
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) b = fmin(b, wmin[w]);
    atomicMin(dtbits, (unsigned long long)__double_as_longlong(b));
  }
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
template <int P, typename CT, typename ST, typename RT>
static int vol_p(const Ctx& x, const void* s, void* r) {
  const int bs = 128;
  const int64_t grid = (x.ne + bs - 1) / bs;
  k_vol_tri<P, CT, ST, RT><<<(unsigned)grid, bs, 0, x.st>>>(static_cast<const ST*>(s), x.d->jinv,
                                                             static_cast<RT*>(r), x.ne);
  return 1;
}

int tri_volume(const Ctx& x, TypeCfg ty, const void* s, void* r) {
  switch (x.p * 4 + ty) {
    case 4 + TY_D: return vol_p<1, double, double, double>(x, s, r);
    case 8 + TY_D: return vol_p<2, double, double, double>(x, s, r);
    case 12 + TY_D: return vol_p<3, double, double, double>(x, s, r);
    case 4 + TY_MD: return vol_p<1, float, double, double>(x, s, r);
    case 8 + TY_MD: return vol_p<2, float, double, double>(x, s, r);
    case 12 + TY_MD: return vol_p<3, float, double, double>(x, s, r);
    case 4 + TY_MF: return vol_p<1, float, float, float>(x, s, r);
    case 8 + TY_MF: return vol_p<2, float, float, float>(x, s, r);
    case 12 + TY_MF: return vol_p<3, float, float, float>(x, s, r);
    default: return -1;
  }
}

template <int P, typename CT, typename ST, typename RT, int MODE>
static int surf_launch(const Ctx& x, const SurfParams& A) {
  const int64_t n = A.end - A.begin;
  if (n <= 0) return 0;
  const int threads = 2 * x.epb;
  const int64_t grid = (2 * n + threads - 1) / threads;
  k_surf_tri<P, CT, ST, RT, MODE><<<(unsigned)grid, threads, 0, x.st>>>(A);
  return 1;
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
    if (ty == TY_MLAST) return surf_launch<P, float, double, float, SURF_LAST>(x, A);
    return -1;
  }
  switch (ty) {
    case TY_D: return surf_mode<P, double, double, double>(x, mode, A);
    case TY_MD: return surf_mode<P, float, double, double>(x, mode, A);
    case TY_MF: return surf_mode<P, float, float, float>(x, mode, A);
    default: return -1;
  }
}

int tri_surface(const Ctx& x, TypeCfg ty, SurfMode mode, int64_t begin, int64_t end, const void* state,
                void* rhs, void* buf, const StageArgs* sa) {
  SurfParams A;
  A.begin = begin;
  A.end = end;
  A.topo = x.d->topo;
  A.fgeo = x.d->fgeo;
  A.jinv = x.d->jinv;
  A.state = state;
  A.rhs = rhs;
  A.buf = buf;
  if (sa) A.sa = *sa;
  switch (x.p) {
    case 1: return surf_p<1>(x, ty, mode, A);
    case 2: return surf_p<2>(x, ty, mode, A);
    case 3: return surf_p<3>(x, ty, mode, A);
    default: return -1;
  }
}

int tri_cfl(const Ctx& x, const double* s, double cfl, double* dt, float* shadow) {
  const int bs = 128;
  const unsigned grid = (unsigned)((x.ne + bs - 1) / bs);
  auto* bits = reinterpret_cast<unsigned long long*>(dt);
  switch (x.p) {
    case 1: k_cfl_tri<1><<<grid, bs, 0, x.st>>>(s, x.d->inr, x.ne, cfl, bits, shadow); return 1;
    case 2: k_cfl_tri<2><<<grid, bs, 0, x.st>>>(s, x.d->inr, x.ne, cfl, bits, shadow); return 1;
    case 3: k_cfl_tri<3><<<grid, bs, 0, x.st>>>(s, x.d->inr, x.ne, cfl, bits, shadow); return 1;
    default: return -1;
  }
}

}  // namespace dgc
