// FP64 kernels for hybrid triangle/quadrilateral meshes (Sec. 3.1: Table 2's
// hybrid mesh is colored with C = {1, 2, 3, 4}; Eq. 2 with each element in the
// space of its kind: P_p on a triangle, Q_p on a parallelogram).
//
// The state keeps NPX = (p+1)^2 coefficients per variable for every element; a
// triangle uses the first (p+1)(p+2)/2 and its other entries of the right-hand
// side are written as zero.  The kernels are table driven: per kind, the basis
// and the weighted reference gradients at the (p+1)^2 volume points, and the
// basis at the 2p+1 points of each local edge, zero past the kind's modes, all
// in shared memory.  A color runs as Algorithm 1 states it: one lane per edge
// side, each evaluating its own element's trace and normal flux, the two lanes
// exchanging them with shuffles, each projecting onto its own element's modes
// and adding into its right-hand side (read-modify-write: the coloring makes
// the two elements of an edge the only writers of their blocks in the color).
//
// A general (bilinear) quadrilateral (kind 2) takes the square's tables too; its
// volume integral weights each point's flux by detJ J^-1 at that point, its
// faces' scales are the bare face lengths, and after the last color its
// right-hand side is multiplied by the inverse of its own mass matrix
// M_ij = int phi_i phi_j detJ (k_hyb_mass), where an affine element's mass
// matrix is detJ times the identity and is divided out by the face and volume
// scales instead.
#include "dev_util.cuh"
#include "device.cuh"
#include "euler_pert.cuh"

namespace dgc {

// table layout (doubles): [kind][NQV][NPX] basis, [kind][NQV][NPX] w d/dr,
// [kind][NQV][NPX] w d/ds, [kind][4 faces][NQE][NPX] edge basis, [NQE] weights
template <int P>
struct HybDim {
  static constexpr int NPX = (P + 1) * (P + 1), NPT = (P + 1) * (P + 2) / 2, NQV = (P + 1) * (P + 1),
                       NQE = 2 * P + 1, NV = 4 * NPX;
  static constexpr int VOL = NQV * NPX, EDGE = 4 * NQE * NPX;
  static constexpr int SIZE = 2 * (3 * VOL + EDGE) + NQE;
  __host__ __device__ static constexpr int vol(int kind) { return kind * 3 * VOL; }
  __host__ __device__ static constexpr int edge(int kind) { return 6 * VOL + kind * EDGE; }
  __host__ __device__ static constexpr int wts() { return 6 * VOL + 2 * EDGE; }
};

template <int P>
__device__ __forceinline__ void hyb_stage(double* s, const double* __restrict__ tab) {
  for (int i = threadIdx.x; i < HybDim<P>::SIZE; i += blockDim.x) s[i] = tab[i];
}

// Euler flux components (gamma = 1.4)
__device__ __forceinline__ void hyb_flux(const double* U, double* F, double* G) {
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

// volume integral of element e (kind k): rhs = sum_q w_q F(U_q).(J^-T grad phi_j)
// (kind 2: detJ J^-1 at each point, from bil_G[slot])
template <int P>
__global__ void __launch_bounds__(128) k_hyb_vol(const double* __restrict__ c, const double* __restrict__ jinv,
                                                 const int8_t* __restrict__ kind, const double* __restrict__ tab,
                                                 const int32_t* __restrict__ bil_slot,
                                                 const double* __restrict__ bil_G, double* __restrict__ rhs,
                                                 int64_t ne) {
  using D = HybDim<P>;
  __shared__ double s[D::SIZE];
  hyb_stage<P>(s, tab);
  __syncthreads();
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= ne) return;
  const int k = kind[e];
  const int np = k ? D::NPX : D::NPT;
  const double* phi = s + D::vol(k ? 1 : 0);
  const double* gr = phi + D::VOL;
  const double* gs = gr + D::VOL;
  const double* ce = c + e * D::NV;
  double j00 = jinv[4 * e], j01 = jinv[4 * e + 1], j10 = jinv[4 * e + 2], j11 = jinv[4 * e + 3];
  const double* Gq = k == 2 ? bil_G + (int64_t)bil_slot[e] * (4 * D::NQV) : nullptr;
  double acc[D::NV];
#pragma unroll
  for (int i = 0; i < D::NV; ++i) acc[i] = 0.0;
  for (int q = 0; q < D::NQV; ++q) {
    double U[4] = {0.0, 0.0, 0.0, 0.0};
    for (int j = 0; j < np; ++j) {
      const double b = phi[q * D::NPX + j];
#pragma unroll
      for (int m = 0; m < 4; ++m) U[m] += b * ce[m * D::NPX + j];
    }
    double F[4], G[4];
    hyb_flux(U, F, G);
    if (Gq) j00 = Gq[4 * q], j01 = Gq[4 * q + 1], j10 = Gq[4 * q + 2], j11 = Gq[4 * q + 3];
#pragma unroll
    for (int m = 0; m < 4; ++m) {
      const double fr = j00 * F[m] + j01 * G[m], fs = j10 * F[m] + j11 * G[m];
#pragma unroll
      for (int j = 0; j < D::NPX; ++j) acc[m * D::NPX + j] += gr[q * D::NPX + j] * fr + gs[q * D::NPX + j] * fs;
    }
  }
  double* re = rhs + e * D::NV;
#pragma unroll
  for (int i = 0; i < D::NV; ++i) re[i] = acc[i];  // zero past a triangle's modes (zero tables)
}

// one color's edges [begin, end): two lanes per edge (side 0: left element, 1:
// right); the right element runs along the edge backwards.  ATOMIC: add with
// atomics instead (all edges in one launch; comparator).
template <int P, bool ATOMIC>
__global__ void __launch_bounds__(128) k_hyb_surf(const double* __restrict__ c, const int4* __restrict__ topo,
                                                  const double2* __restrict__ fgeo, const int8_t* __restrict__ kind,
                                                  const double* __restrict__ tab, double* __restrict__ rhs,
                                                  int64_t begin, int64_t end) {
  using D = HybDim<P>;
  constexpr int NQ = D::NQE;
  __shared__ double s[D::SIZE];
  hyb_stage<P>(s, tab);
  __syncthreads();
  const int side = threadIdx.x & 1;
  int64_t k = begin + (((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 1);
  const bool valid = k < end;
  if (!valid) k = end - 1;  // idle lanes shadow the last edge so both lanes of a pair shuffle
  const int4 tp = topo[k];
  const bool bnd = tp.y < 0;  // boundary: both lanes read the left element (U+ = U-)
  const bool right = side && !bnd;
  const int64_t elem = right ? tp.y : tp.x;
  const int le = right ? ((tp.z >> 4) & 15) : (tp.z & 15);
  const bool writer = valid && !(side && bnd);
  const int kd = kind[elem] ? 1 : 0;  // a general quadrilateral takes the square's tables
  const int np = kd ? D::NPX : D::NPT;
  const double2 g0 = fgeo[2 * k], g1 = fgeo[2 * k + 1];
  const double nx = g0.x, ny = g0.y, scale = right ? g1.y : -g1.x;
  const double* ph = s + D::edge(kd) + le * NQ * D::NPX;
  const double* w = s + D::wts();
  const double* ce = c + elem * D::NV;
  double acc[D::NV];
#pragma unroll
  for (int i = 0; i < D::NV; ++i) acc[i] = 0.0;
  for (int q = 0; q < NQ; ++q) {
    const int qq = right ? NQ - 1 - q : q;
    double U[4] = {0.0, 0.0, 0.0, 0.0};
    for (int j = 0; j < np; ++j) {
      const double b = ph[qq * D::NPX + j];
#pragma unroll
      for (int m = 0; m < 4; ++m) U[m] += b * ce[m * D::NPX + j];
    }
    // own normal flux and wave speed, exchanged with the partner lane
    const double ir = 1.0 / U[0];
    const double u = U[1] * ir, v = U[2] * ir;
    const double p = 0.4 * (U[3] - 0.5 * (U[1] * u + U[2] * v));
    const double un = u * nx + v * ny;
    const double Fo[4] = {U[0] * un, U[1] * un + p * nx, U[2] * un + p * ny, (U[3] + p) * un};
    const double wo = fabs(un) + sqrt(1.4 * p * ir);
    double V[4], Fp[4];
#pragma unroll
    for (int m = 0; m < 4; ++m) {
      V[m] = __shfl_xor_sync(0xffffffffu, U[m], 1);
      Fp[m] = __shfl_xor_sync(0xffffffffu, Fo[m], 1);
    }
    const double lam = fmax(wo, __shfl_xor_sync(0xffffffffu, wo, 1));
    const double g = scale * w[q];
#pragma unroll
    for (int m = 0; m < 4; ++m) {
      const double a = side ? V[m] : U[m], b = side ? U[m] : V[m];
      const double Fs = 0.5 * (Fo[m] + Fp[m]) - (0.5 * lam) * (b - a);  // commutative: both lanes' bits agree
      const double gm = g * Fs;
#pragma unroll
      for (int j = 0; j < D::NPX; ++j) acc[m * D::NPX + j] += ph[qq * D::NPX + j] * gm;
    }
  }
  if (!writer) return;
  double* re = rhs + elem * D::NV;
  if constexpr (ATOMIC) {
    for (int i = 0; i < D::NV; ++i)
      if ((i % D::NPX) < np) atomicAdd(re + i, acc[i]);
  } else if (kd) {
#pragma unroll
    for (int i = 0; i < D::NV; ++i) re[i] += acc[i];
  } else {
    // a triangle: its own modes only (the rest stay as the volume kernel wrote them, zero)
#pragma unroll
    for (int m = 0; m < 4; ++m)
#pragma unroll
      for (int j = 0; j < D::NPT; ++j) re[m * D::NPX + j] += acc[m * D::NPX + j];
  }
}

// ---------------------------------------------------------------------------
// FP32-mixed form (flux, quadrature and projection in FP32; FP64 state and
// right-hand side), in the perturbation form the triangle kernels use
// (euler_pert.cuh): each element's reference ub = phi_0 c_0 (FP64, kept as an
// FP32 pair hi + lo), its modes j >= 1 in FP32, and the flux deviations
// F(ub + d) - F(ub) projected in the volume and F* - F(ub).n on the faces.  The
// omitted parts cancel for each element: the volume rule integrates
// grad phi_j against detJ J^-1 exactly (J^-1 constant, or detJ J^-1 linear in
// the reference coordinates on a bilinear element) and the edge rule phi_j on
// each straight edge.  The tables are the FP64 ones, converted while staged.
// ---------------------------------------------------------------------------
template <int P>
__device__ __forceinline__ void hyb_stage32(float* s, const double* __restrict__ tab) {
  for (int i = threadIdx.x; i < HybDim<P>::SIZE; i += blockDim.x) s[i] = d2f(tab[i]);
}

// the element's block in perturbation form: hi + lo = phi_0 c_0, cd = modes j >= 1
template <int P>
struct HybPert {
  float hi[4], lo[4], cd[4][HybDim<P>::NPX - 1];
  __device__ __forceinline__ void load(const double* __restrict__ ce, double phi0, int np) {
#pragma unroll
    for (int m = 0; m < 4; ++m) {
      const double u = phi0 * ce[m * HybDim<P>::NPX];
      hi[m] = d2f(u);
      lo[m] = d2f(u - f2d(hi[m]));
#pragma unroll
      for (int j = 1; j < HybDim<P>::NPX; ++j) cd[m][j - 1] = j < np ? d2f(ce[m * HybDim<P>::NPX + j]) : 0.0f;
    }
  }
  // the deviation of the trace at a point from the reference: lo + sum_j b_j c_j
  __device__ __forceinline__ void dev(const float* b, float (&d)[4]) const {
#pragma unroll
    for (int m = 0; m < 4; ++m) {
      float v = lo[m];
#pragma unroll
      for (int j = 1; j < HybDim<P>::NPX; ++j) v = fmaf(b[j], cd[m][j - 1], v);
      d[m] = v;
    }
  }
};

template <int P>
__global__ void __launch_bounds__(128) k_hyb_vol32(const double* __restrict__ c, const double* __restrict__ jinv,
                                                   const int8_t* __restrict__ kind, const double* __restrict__ tab,
                                                   const int32_t* __restrict__ bil_slot,
                                                   const double* __restrict__ bil_G, double* __restrict__ rhs,
                                                   int64_t ne) {
  using D = HybDim<P>;
  __shared__ float s[D::SIZE];
  hyb_stage32<P>(s, tab);
  __syncthreads();
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= ne) return;
  const int k = kind[e];
  const int np = k ? D::NPX : D::NPT;
  const float* phi = s + D::vol(k ? 1 : 0);
  const float* gr = phi + D::VOL;
  const float* gs = gr + D::VOL;
  HybPert<P> B;
  B.load(c + e * D::NV, tab[D::vol(k ? 1 : 0)], np);  // phi_0 (constant) from the FP64 table
  PertRef<2> R;
  R.init(B.hi);
  float nr[2] = {d2f(jinv[4 * e]), d2f(jinv[4 * e + 1])}, ns[2] = {d2f(jinv[4 * e + 2]), d2f(jinv[4 * e + 3])};
  const double* Gq = k == 2 ? bil_G + (int64_t)bil_slot[e] * (4 * D::NQV) : nullptr;
  float acc[D::NV];
#pragma unroll
  for (int i = 0; i < D::NV; ++i) acc[i] = 0.0f;
  for (int q = 0; q < D::NQV; ++q) {
    float d[4];
    B.dev(phi + q * D::NPX, d);
    if (Gq) nr[0] = d2f(Gq[4 * q]), nr[1] = d2f(Gq[4 * q + 1]), ns[0] = d2f(Gq[4 * q + 2]), ns[1] = d2f(Gq[4 * q + 3]);
    PertState<2> S;
    S.init(R, d);
    float Fr[4], Fs[4];
    pert_flux<2>(R, S, d, nr, R.u[1] * nr[0] + R.u[2] * nr[1], Fr);
    pert_flux<2>(R, S, d, ns, R.u[1] * ns[0] + R.u[2] * ns[1], Fs);
#pragma unroll
    for (int m = 0; m < 4; ++m)
#pragma unroll
      for (int j = 1; j < D::NPX; ++j)
        acc[m * D::NPX + j] = fmaf(gr[q * D::NPX + j], Fr[m], fmaf(gs[q * D::NPX + j], Fs[m], acc[m * D::NPX + j]));
  }
  double* re = rhs + e * D::NV;
#pragma unroll
  for (int i = 0; i < D::NV; ++i) re[i] = (double)acc[i];  // zero past a triangle's modes (zero tables)
}

template <int P, bool ATOMIC>
__global__ void __launch_bounds__(128) k_hyb_surf32(const double* __restrict__ c, const int4* __restrict__ topo,
                                                    const double2* __restrict__ fgeo, const int8_t* __restrict__ kind,
                                                    const double* __restrict__ tab, double* __restrict__ rhs,
                                                    int64_t begin, int64_t end) {
  using D = HybDim<P>;
  constexpr int NQ = D::NQE;
  __shared__ float s[D::SIZE];
  hyb_stage32<P>(s, tab);
  __syncthreads();
  const int side = threadIdx.x & 1;
  int64_t k = begin + (((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 1);
  const bool valid = k < end;
  if (!valid) k = end - 1;  // idle lanes shadow the last edge so both lanes of a pair shuffle
  const int4 tp = topo[k];
  const bool bnd = tp.y < 0;  // boundary: both lanes read the left element (U+ = U-)
  const bool right = side && !bnd;
  const int64_t elem = right ? tp.y : tp.x;
  const int le = right ? ((tp.z >> 4) & 15) : (tp.z & 15);
  const bool writer = valid && !(side && bnd);
  const int kd = kind[elem] ? 1 : 0;  // a general quadrilateral takes the square's tables
  const int np = kd ? D::NPX : D::NPT;
  const double2 g0 = fgeo[2 * k], g1 = fgeo[2 * k + 1];
  const float scale = right ? d2f(g1.y) : -d2f(g1.x);
  const float* ph = s + D::edge(kd) + le * NQ * D::NPX;
  const float* w = s + D::wts();
  HybPert<P> B;
  B.load(c + elem * D::NV, tab[D::vol(kd)], np);
  PertRef<2> R;
  R.init(B.hi);
  // each lane evaluates its own side's flux and the pair exchanges one value per
  // variable (euler_pert.cuh, lf_exchange); all 32 lanes run it
  FaceConst<2> E;
  E.init(R, B.hi, {d2f(g0.x), d2f(g0.y)}, side);
  float acc[D::NV];
#pragma unroll
  for (int i = 0; i < D::NV; ++i) acc[i] = 0.0f;
  for (int q = 0; q < NQ; ++q) {
    const int qq = right ? NQ - 1 - q : q;
    float t[4], G[4];
    B.dev(ph + qq * D::NPX, t);
    lf_exchange<2>(R, E, t, G);
    const float g = scale * w[q];
#pragma unroll
    for (int m = 0; m < 4; ++m) {
      const float gm = g * G[m];
#pragma unroll
      for (int j = 0; j < D::NPX; ++j) acc[m * D::NPX + j] = fmaf(ph[qq * D::NPX + j], gm, acc[m * D::NPX + j]);
    }
  }
  if (!writer) return;
  double* re = rhs + elem * D::NV;
  if constexpr (ATOMIC) {
    for (int i = 0; i < D::NV; ++i)
      if ((i % D::NPX) < np) atomicAdd(re + i, (double)acc[i]);
  } else if (kd) {
#pragma unroll
    for (int i = 0; i < D::NV; ++i) re[i] += (double)acc[i];
  } else {
    // a triangle: its own modes only (the rest stay as the volume kernel wrote them, zero)
#pragma unroll
    for (int m = 0; m < 4; ++m)
#pragma unroll
      for (int j = 0; j < D::NPT; ++j) re[m * D::NPX + j] += (double)acc[m * D::NPX + j];
  }
}

// CFL: dt = cfl min_e r_e / ((2p+1) max_q (|u| + c)), one thread per element,
// FP64, folded into *dt by a 64-bit atomicMin on the bits (positive doubles
// order as their bit patterns); *dt must hold a large value beforehand
template <int P>
__global__ void __launch_bounds__(128) k_hyb_cfl(const double* __restrict__ c, const double* __restrict__ inr,
                                                 const int8_t* __restrict__ kind, const double* __restrict__ tab,
                                                 int64_t ne, double cfl, unsigned long long* dtbits) {
  using D = HybDim<P>;
  __shared__ double s[D::SIZE];
  hyb_stage<P>(s, tab);
  __syncthreads();
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= ne) return;
  const int k = kind[e] ? 1 : 0;
  const int np = k ? D::NPX : D::NPT;
  const double* phi = s + D::vol(k);
  const double* ce = c + e * D::NV;
  double lam = 0.0;
  for (int q = 0; q < D::NQV; ++q) {
    double U[4] = {0.0, 0.0, 0.0, 0.0};
    for (int j = 0; j < np; ++j) {
      const double b = phi[q * D::NPX + j];
#pragma unroll
      for (int m = 0; m < 4; ++m) U[m] += b * ce[m * D::NPX + j];
    }
    const double ir = 1.0 / U[0], u = U[1] * ir, v = U[2] * ir;
    const double q2 = u * u + v * v;
    const double pr = 0.4 * (U[3] - 0.5 * U[0] * q2);
    lam = fmax(lam, sqrt(q2) + sqrt(1.4 * pr * ir));
  }
  const double d = cfl * (inr[e] / ((2 * P + 1) * lam));
  if (d > 0.0) atomicMin(dtbits, (unsigned long long)__double_as_longlong(d));
}

// general quadrilaterals: rhs_e <- M_e^-1 rhs_e per variable, one thread per
// such element (bil_elem: the element of each slot; Minv row-major [NPX][NPX])
template <int P>
__global__ void __launch_bounds__(128) k_hyb_mass(const int32_t* __restrict__ bil_elem,
                                                  const double* __restrict__ Minv, double* __restrict__ rhs,
                                                  int64_t nb) {
  using D = HybDim<P>;
  const int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= nb) return;
  double* re = rhs + (int64_t)bil_elem[b] * D::NV;
  const double* A = Minv + b * (D::NPX * D::NPX);
  double r[D::NV], o[D::NV];
#pragma unroll
  for (int i = 0; i < D::NV; ++i) r[i] = re[i], o[i] = 0.0;
  for (int i = 0; i < D::NPX; ++i)
#pragma unroll
    for (int j = 0; j < D::NPX; ++j) {
      const double a = A[i * D::NPX + j];
#pragma unroll
      for (int m = 0; m < 4; ++m) o[m * D::NPX + i] += a * r[m * D::NPX + j];
    }
#pragma unroll
  for (int i = 0; i < D::NV; ++i) re[i] = o[i];
}

template <int P>
static int hyb_p(const Ctx& x, int what, const double* state, double* rhs, int64_t b, int64_t e, double cfl,
                 double* dt, bool fp32 = false) {
  const int bs = 128;
  const DeviceMesh* d = x.d;
  if (what == 0) {
    if (x.ne <= 0) return 0;
    const unsigned grid = (unsigned)((x.ne + bs - 1) / bs);
    if (fp32)
      k_hyb_vol32<P><<<grid, bs, 0, x.st>>>(state, d->jinv, d->hyb_kind, d->hyb_tab, d->bil_slot, d->bil_G, rhs, x.ne);
    else
      k_hyb_vol<P><<<grid, bs, 0, x.st>>>(state, d->jinv, d->hyb_kind, d->hyb_tab, d->bil_slot, d->bil_G, rhs, x.ne);
    return 1;
  }
  if (what == 4) {
    if (d->nbil <= 0) return 0;
    k_hyb_mass<P><<<(unsigned)((d->nbil + bs - 1) / bs), bs, 0, x.st>>>(d->bil_elem, d->bil_Minv, rhs, d->nbil);
    return 1;
  }
  if (what == 1 || what == 2) {
    const int64_t n = e - b;
    if (n <= 0) return 0;
    const unsigned grid = (unsigned)((2 * n + bs - 1) / bs);
    if (fp32 && what == 1)
      k_hyb_surf32<P, false><<<grid, bs, 0, x.st>>>(state, d->topo, d->fgeo, d->hyb_kind, d->hyb_tab, rhs, b, e);
    else if (fp32)
      k_hyb_surf32<P, true><<<grid, bs, 0, x.st>>>(state, d->topo, d->fgeo, d->hyb_kind, d->hyb_tab, rhs, b, e);
    else if (what == 1)
      k_hyb_surf<P, false><<<grid, bs, 0, x.st>>>(state, d->topo, d->fgeo, d->hyb_kind, d->hyb_tab, rhs, b, e);
    else
      k_hyb_surf<P, true><<<grid, bs, 0, x.st>>>(state, d->topo, d->fgeo, d->hyb_kind, d->hyb_tab, rhs, b, e);
    return 1;
  }
  if (cudaMemsetAsync(dt, 0x7F, sizeof(double), x.st) != cudaSuccess) return -1;
  k_hyb_cfl<P><<<(unsigned)((x.ne + bs - 1) / bs), bs, 0, x.st>>>(state, d->inr, d->hyb_kind, d->hyb_tab, x.ne, cfl,
                                                                  reinterpret_cast<unsigned long long*>(dt));
  return 1;
}

static int hyb(const Ctx& x, int what, const double* state, double* rhs, int64_t b, int64_t e, double cfl,
               double* dt, bool fp32 = false) {
  switch (x.p) {
    case 1: return hyb_p<1>(x, what, state, rhs, b, e, cfl, dt, fp32);
    case 2: return hyb_p<2>(x, what, state, rhs, b, e, cfl, dt, fp32);
    case 3: return hyb_p<3>(x, what, state, rhs, b, e, cfl, dt, fp32);
    default: return -1;
  }
}

int hyb_volume(const Ctx& x, const double* state, double* rhs, bool fp32) {
  return hyb(x, 0, state, rhs, 0, 0, 0.0, nullptr, fp32);
}
int hyb_surface(const Ctx& x, bool atomic, int64_t begin, int64_t end, const double* state, double* rhs, bool fp32) {
  return hyb(x, atomic ? 2 : 1, state, rhs, begin, end, 0.0, nullptr, fp32);
}
int hyb_cfl(const Ctx& x, const double* state, double cfl, double* dt) {
  return hyb(x, 3, state, nullptr, 0, 0, cfl, dt);
}
int hyb_mass(const Ctx& x, double* rhs) { return hyb(x, 4, nullptr, rhs, 0, 0, 0.0, nullptr); }
int hyb_table_doubles(int p) {
  switch (p) {
    case 1: return HybDim<1>::SIZE;
    case 2: return HybDim<2>::SIZE;
    case 3: return HybDim<3>::SIZE;
    default: return -1;
  }
}

}  // namespace dgc
