// Element-wise kernels shared by all element types: the SSP-RK3 stage update
// (used when the update is not fused into the last color) and the gather of
// the per-edge-buffer comparator.
#include "device.cuh"

namespace dgc {

// uout = a0 u0 + b0 (us + dt rhs), FP64; also the FP32 copy when shadow != null.
// Element-wise, so uout may alias us or u0.
template <typename RT>
__global__ void k_stage(const double* u0, const double* us, const RT* rhs, const double* dtp, double a0,
                        double b0, double* uout, float* shadow, int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double dt = *dtp;
  double v = b0 * (us[i] + dt * (double)rhs[i]);
  if (a0 != 0.0) v += a0 * u0[i];
  uout[i] = v;
  if (shadow) shadow[i] = (float)v;
}

int stage_update(const Ctx& x, bool rhs_f32, const double* us, const void* rhs, const StageArgs& sa) {
  const int64_t n = x.ne * x.M * x.np;
  const int bs = 256;
  const unsigned grid = (unsigned)((n + bs - 1) / bs);
  if (rhs_f32)
    k_stage<float><<<grid, bs, 0, x.st>>>(sa.u0, us, static_cast<const float*>(rhs), sa.dt, sa.a0, sa.b0,
                                          sa.uout, sa.shadow, n);
  else
    k_stage<double><<<grid, bs, 0, x.st>>>(sa.u0, us, static_cast<const double*>(rhs), sa.dt, sa.a0, sa.b0,
                                           sa.uout, sa.shadow, n);
  return 1;
}

// rhs[e][v] += sum_f buf[slot(e, f)][v]  (second pass of the buffer scheme, Sec. 1)
template <typename RT>
__global__ void k_gather(RT* rhs, const RT* buf, const int32_t* slots, int nfpe, int nv, int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int64_t e = i / nv;
  const int v = (int)(i - e * nv);
  RT s = rhs[i];
  for (int f = 0; f < nfpe; ++f) {
    const int64_t slot = slots[e * nfpe + f];
    s += buf[slot * nv + v];
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
                                           x.d->slots, x.nfpe, nv, n);
  else
    k_gather<double><<<grid, bs, 0, x.st>>>(static_cast<double*>(rhs), static_cast<const double*>(buf),
                                            x.d->slots, x.nfpe, nv, n);
  return 1;
}

__global__ void k_shadow(const double* s, float* f, int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) f[i] = (float)s[i];
}

int make_shadow(const Ctx& x, const double* state, float* shadow) {
  const int64_t n = x.ne * x.M * x.np;
  const int bs = 256;
  k_shadow<<<(unsigned)((n + bs - 1) / bs), bs, 0, x.st>>>(state, shadow, n);
  return 1;
}

}  // namespace dgc
