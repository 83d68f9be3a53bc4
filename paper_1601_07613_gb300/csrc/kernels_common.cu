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

}  // namespace dgc
