// Element-wise kernels shared by all element types: the SSP-RK3 stage update
// (used when the update is not fused into the last color) and the gather of
// the per-edge-buffer comparator.
#include "dev_util.cuh"
#include "device.cuh"
#include "incr_form.cuh"

namespace dgc {

// FP64 form: uout = a0 u0 + b0 us + (b0 dt) rhs.  Element-wise, so uout may
// alias us or u0.
__global__ void k_stage(const double* u0, const double* us, const double* rhs, const double* dtp, double a0,
                        double b0, double* uout, int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double bdt = b0 * *dtp;
  uout[i] = a0 != 0.0 ? fma(bdt, rhs[i], fma(a0, u0[i], b0 * us[i])) : fma(bdt, rhs[i], b0 * us[i]);
}

int stage_update(const Ctx& x, bool, const double* us, const void* rhs, const StageArgs& sa) {
  const int64_t n = x.ne * x.M * x.np;
  const int bs = 256;
  const unsigned grid = (unsigned)((n + bs - 1) / bs);
  k_stage<<<grid, bs, 0, x.st>>>(sa.u0, us, static_cast<const double*>(rhs), sa.dt, sa.a0, sa.b0, sa.uout, n);
  return 1;
}

// FP32 forms: one SSP-RK3 stage in increment form (incr_form.cuh), one value
// per thread, for meshes whose last color does not reach every element.
// Thread i is entry i of the FP32 rhs and increment blocks: mode-major ([Np][M],
// triangles) or [M][Np] (tetrahedra), as L.mode_major says; the FP64 state is
// [M][Np].  Record entries: hi[m], lo[m] at m and M + m; mode j >= 1 at
// M (j + 1) + m (mode-major) or 2M + m(np-1) + j-1.  Kahan state: the record,
// then lo of mode j >= 1 at rec + M (j - 1) + m (triangles only).
__global__ void k_incr_stage(const float* __restrict__ rhs, StageArgs S, ShadowLayout L, int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int64_t e = i / L.nv;
  const int l = (int)(i - e * L.nv);
  const int m = L.mode_major ? l % L.M : l / L.np, j = L.mode_major ? l / L.M : l % L.np;
  const F2 dtp = split_f2(*S.dt);
  const float dL = mul_f2(rhs[i], dtp);
  float d = S.stage == 0 ? dL : (S.stage == 1 ? 0.25f * (S.delta[i] + dL) : S.delta[i] + dL);
  const int mode_ix = L.mode_major ? L.M * (j + 1) + m : 2 * L.M + m * (L.np - 1) + j - 1;
  if (S.stage < 2) {
    S.delta[i] = d;
    const float* r0 = S.rec0 + e * S.rec0_stride;
    float* ro = S.rec_out + e * L.rec;
    if (j == 0) {
      float h = r0[m], lo = r0[L.M + m];
      pair_add_scaled(h, lo, d, split_f2(L.phi0));
      ro[m] = h;
      ro[L.M + m] = lo;
    } else {
      ro[mode_ix] = r0[mode_ix] + d;
    }
    if (l == 0)
      for (int k = L.M * (L.np + 1); k < L.rec; ++k) ro[k] = 0.0f;  // padding
  } else if (S.kstate) {
    float* ks = S.kstate + e * S.rec0_stride;
    if (j == 0) kahan_add(ks[m], ks[L.M + m], mul_f2(d, split_f2(2.0 / 3.0 * L.phi0)));
    else kahan_add(ks[mode_ix], ks[L.rec + L.M * (j - 1) + m], mul_f2(d, split_f2(2.0 / 3.0)));
  } else {
    const int64_t u = e * L.nv + m * L.np + j;
    S.uout[u] = fma(2.0 / 3.0, f2d(d), S.u0[u]);
  }
}

int incr_stage_update(const Ctx& x, const float* rhs, const StageArgs& sa) {
  const int64_t n = x.ne * x.M * x.np;
  const int bs = 256;
  const unsigned grid = (unsigned)((n + bs - 1) / bs);
  k_incr_stage<<<grid, bs, 0, x.st>>>(rhs, sa, x.shadow, n);
  return 1;
}

// rhs[e][v] += sum_f buf[slot(e, f)][v]  (second pass of the buffer scheme, Sec. 1)
template <typename RT>
__global__ void k_gather(RT* rhs, const RT* buf, const int32_t* slots, int slot_w, int nv, int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int64_t e = i / nv;
  const int v = (int)(i - e * nv);
  RT s = rhs[i];
  for (int f = 0; f < slot_w; ++f) {
    const int64_t slot = slots[e * slot_w + f];
    if (slot >= 0) s += buf[slot * nv + v];
  }
  rhs[i] = s;
}

int gather_two_pass(const Ctx& x, bool f32, void* rhs, const void* buf) {
  const int nv = x.M * x.np;
  const int64_t n = x.ne * nv;
  const int bs = 256;
  const unsigned grid = (unsigned)((n + bs - 1) / bs);
  if (f32)
    k_gather<float><<<grid, bs, 0, x.st>>>(static_cast<float*>(rhs), static_cast<const float*>(buf),
                                           x.d->slots, x.d->slot_w, nv, n);
  else
    k_gather<double><<<grid, bs, 0, x.st>>>(static_cast<double*>(rhs), static_cast<const double*>(buf),
                                            x.d->slots, x.d->slot_w, nv, n);
  return 1;
}

// Element blocks between original and internal order, two doubles per thread
// (nv is even): one pass over the state in each direction.
__global__ void k_permute(double2* __restrict__ dst, const double2* __restrict__ src, const int32_t* __restrict__ perm,
                          int nv2, int64_t n, bool to_internal) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int64_t e = i / nv2;
  const int v = (int)(i - e * nv2);
  const int64_t pe = perm[e];
  if (to_internal) dst[pe * nv2 + v] = src[i];
  else dst[i] = src[pe * nv2 + v];
}

int permute_blocks(cudaStream_t st, double* dst, const double* src, const int32_t* perm, int nv, int64_t ne,
                   bool to_internal) {
  const int nv2 = nv / 2;
  const int64_t n = ne * nv2;
  const int bs = 256;
  if (n <= 0) return 0;
  k_permute<<<(unsigned)((n + bs - 1) / bs), bs, 0, st>>>(reinterpret_cast<double2*>(dst),
                                                         reinterpret_cast<const double2*>(src), perm, nv2, n,
                                                         to_internal);
  return 1;
}

// ---------------------------------------------------------------------------
// Refinement (Sec. 3.2) on the device: the 6-color map of the refined sides
// from the coarse coloring, and the DG state between the coarse mesh and its
// refinement.
// ---------------------------------------------------------------------------
// One thread per refined side: rule & 15 = 0 keeps base side src's color c,
// 1 and 2 (the half next to the smaller and the larger vertex id) give c and
// c + K (at level 0, K = 3: ((c + 3 m - 4) mod 6) + 1), 3 + k gives the interior
// edge of refined base element src the color of its edge k (the parallel one;
// a split edge's half taken modulo K); K = 3 * 2^(rule >> 4), the palette of the
// base elements' level.
__global__ void k_refine_colors(const int8_t* __restrict__ base_color, const int32_t* __restrict__ base_face_of,
                                const int32_t* __restrict__ src, const int8_t* __restrict__ rule, int64_t ns,
                                int8_t* __restrict__ out) {
  const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= ns) return;
  const int r = rule[s] & 15, K = 3 << (rule[s] >> 4);
  int c;
  if (r == 0) c = base_color[src[s]];
  else if (r <= 2) c = base_color[src[s]] + (r - 1) * K;
  else c = (base_color[base_face_of[(int64_t)src[s] * 3 + (r - 3)]] - 1) % K + 1;
  out[s] = (int8_t)c;
}

int refine_colors(cudaStream_t st, const int8_t* base_color, const int32_t* base_face_of, const int32_t* src,
                  const int8_t* rule, int64_t ns, int8_t* out) {
  if (ns <= 0) return 0;
  const int bs = 256;
  k_refine_colors<<<(unsigned)((ns + bs - 1) / bs), bs, 0, st>>>(base_color, base_face_of, src, rule, ns, out);
  return 1;
}

// Prolongation, one thread per fine element and variable: a child c of coarse
// element src takes out_j = sum_k P_c[j][k] in_k (P_c: the L2 projection of the
// parent's basis onto the child's, [4][NP][NP]); kind 4 copies the element.
__global__ void k_prolong(const double* __restrict__ cc, double* __restrict__ cf, const int32_t* __restrict__ src,
                          const int8_t* __restrict__ kind, const double* __restrict__ P, int64_t nef, int M, int NP) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nef * M) return;
  const int64_t e = i / M;
  const int m = (int)(i - e * M);
  const double* in = cc + ((int64_t)src[e] * M + m) * NP;
  double* out = cf + (e * M + m) * NP;
  const int c = kind[e];
  if (c == 4) {
    for (int j = 0; j < NP; ++j) out[j] = in[j];
    return;
  }
  const double* Pc = P + (int64_t)c * NP * NP;
  double v[16];
  for (int k = 0; k < NP; ++k) v[k] = in[k];
  for (int j = 0; j < NP; ++j) {
    double s = 0.0;
    for (int k = 0; k < NP; ++k) s = fma(Pc[j * NP + k], v[k], s);
    out[j] = s;
  }
}

// Restriction, one thread per coarse element and variable: a refined element
// takes out_k = (1/4) sum_c sum_j P_c[j][k] in^c_j over its children kids[4]
// (each child a quarter of the parent's area); kids[1] < 0 copies kids[0].
__global__ void k_restrict(const double* __restrict__ cf, double* __restrict__ cc, const int32_t* __restrict__ kids,
                           const double* __restrict__ P, int64_t nec, int M, int NP) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nec * M) return;
  const int64_t e = i / M;
  const int m = (int)(i - e * M);
  double* out = cc + (e * M + m) * NP;
  const int32_t* kd = kids + e * 4;
  if (kd[1] < 0) {
    const double* in = cf + ((int64_t)kd[0] * M + m) * NP;
    for (int j = 0; j < NP; ++j) out[j] = in[j];
    return;
  }
  double acc[16];
  for (int k = 0; k < NP; ++k) acc[k] = 0.0;
  for (int c = 0; c < 4; ++c) {
    const double* in = cf + ((int64_t)kd[c] * M + m) * NP;
    const double* Pc = P + (int64_t)c * NP * NP;
    for (int j = 0; j < NP; ++j) {
      const double v = in[j];
      for (int k = 0; k < NP; ++k) acc[k] = fma(Pc[j * NP + k], v, acc[k]);
    }
  }
  for (int k = 0; k < NP; ++k) out[k] = 0.25 * acc[k];
}

int transfer_state(cudaStream_t st, bool prolong, const double* in, double* out, const int32_t* src,
                   const int8_t* kind, const int32_t* kids, const double* P, int64_t n, int M, int NP) {
  if (n <= 0) return 0;
  if (NP > 16) return -1;
  const int bs = 128;
  const unsigned grid = (unsigned)((n * M + bs - 1) / bs);
  if (prolong) k_prolong<<<grid, bs, 0, st>>>(in, out, src, kind, P, n, M, NP);
  else k_restrict<<<grid, bs, 0, st>>>(in, out, kids, P, n, M, NP);
  return 1;
}

}  // namespace dgc
