// Element-wise kernels shared by all element types: the SSP-RK3 stage update
// (used when the update is not fused into the last color) and the gather of
// the per-edge-buffer comparator.
#include "dev_util.cuh"
#include "device.cuh"

namespace dgc {

// uout = a0 u0 + b0 us + (b0 dt) rhs in FP64, and the FP32 record of uout when
// shadow != null.  Element-wise, so uout may alias us or u0.
template <typename RT>
__global__ void k_stage(const double* u0, const double* us, const RT* rhs, const double* dtp, double a0,
                        double b0, double* uout, float* shadow, ShadowLayout L, int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double bdt = b0 * *dtp;
  const double R = widen(rhs[i]);
  const double v = a0 != 0.0 ? fma(bdt, R, fma(a0, u0[i], b0 * us[i])) : fma(bdt, R, b0 * us[i]);
  uout[i] = v;
  if (shadow) {
    const int64_t e = i / L.nv;
    const int l = (int)(i - e * L.nv), m = l / L.np, j = l - m * L.np;
    float* rec = shadow + e * L.rec;
    if (!L.split) {
      rec[l] = d2f(v);
    } else if (j == 0) {
      const double u = L.phi0 * v;
      const float hi = d2f(u);
      rec[m] = hi;
      rec[L.M + m] = d2f(u - f2d(hi));
    } else {
      rec[2 * L.M + m * (L.np - 1) + j - 1] = d2f(v);
    }
  }
}

int stage_update(const Ctx& x, bool rhs_f32, const double* us, const void* rhs, const StageArgs& sa) {
  const int64_t n = x.ne * x.M * x.np;
  const int bs = 256;
  const unsigned grid = (unsigned)((n + bs - 1) / bs);
  if (rhs_f32)
    k_stage<float><<<grid, bs, 0, x.st>>>(sa.u0, us, static_cast<const float*>(rhs), sa.dt, sa.a0, sa.b0,
                                          sa.uout, sa.shadow, x.shadow, n);
  else
    k_stage<double><<<grid, bs, 0, x.st>>>(sa.u0, us, static_cast<const double*>(rhs), sa.dt, sa.a0, sa.b0,
                                           sa.uout, sa.shadow, x.shadow, n);
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

}  // namespace dgc
