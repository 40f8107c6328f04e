// Far-field column generation and row accumulation (FP64).
//
// Column side (Sections 4.1, 5.1, 6): the stacked column l of a block holds
//   g_l(n) = exp(i pi V_n^2/(2E)) c_n colpow(n)^u1 omt(n)^(delta-1/2) sum_u2 G_l[u2] beta(n)^u2,
// where the complex G_l merge the Hankel coefficients (-1)^m a_m(mu), the phases
// exp(-i(2mu+1)pi/4) and the rearranged Neumann/Taylor weights of every term whose
// row factor is the same function of k.
// Row side: f_k += Re[ exp(i pi U_k^2/(2E)) sum_l rowpert(k)^u1 rowvar(k)^(delta-1/2) y_l(k) ].
#include <cuda_runtime.h>

#include <algorithm>

#include "kernels.cuh"

namespace hk {

namespace {

__device__ __forceinline__ double ipow(double x, int e) {
  double r = 1.0;
  while (e) {
    if (e & 1) r *= x;
    x *= x;
    e >>= 1;
  }
  return r;
}

__global__ void __launch_bounds__(256) k_gen(GenArgs a) {
  const int cc = blockIdx.y;
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= a.F) return;
  double2* A = a.A + (int64_t)cc * a.F;
  if (t >= a.C) {
    A[t] = make_double2(0.0, 0.0);
    return;
  }
  const int64_t g = a.c0 + cc;
  const int rhs = (int)(g / a.ncols);
  const int l = (int)(g - (int64_t)rhs * a.ncols);
  const DevColSpec& cs = a.cols[l];
  const int64_t i = a.n0 - 1 + t;
  const double bt = a.nodes.betan[i];
  double pr = cs.G[cs.nterm - 1].x, pim = cs.G[cs.nterm - 1].y;
  for (int u = cs.nterm - 2; u >= 0; --u) {
    pr = fma(pr, bt, cs.G[u].x);
    pim = fma(pim, bt, cs.G[u].y);
  }
  const int d = cs.delta;
  double pw = a.nodes.rs_omt[i] * ipow(d >= 0 ? a.nodes.omt[i] : a.nodes.inv_omt[i], d >= 0 ? d : -d);
  if (cs.u1) pw *= ipow(a.nodes.colpow[i], cs.u1);
  const double cv = a.c[(int64_t)rhs * a.ldc + i] * pw;
  const double xr = pr * cv, xi = pim * cv;
  const double2 w = a.wV[t];
  A[t] = make_double2(fma(xr, w.x, -xi * w.y), fma(xr, w.y, xi * w.x));
}

__global__ void __launch_bounds__(256) k_out(OutArgs a) {
  const int64_t kp = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (kp >= a.R) return;
  const int64_t i = a.k0 - 1 + kp;
  const double rv = a.nodes.rowvar[i], irv = a.nodes.inv_rowvar[i], rs = a.nodes.rs_rowvar[i];
  const double rp = a.nodes.rowpert[i];
  const double2 wu = a.wU[kp];
  const double2* Y = a.Y + kp + a.C - 1;
  double ar = 0.0, ai = 0.0;
  int cur = (int)(a.c0 / a.ncols);
  for (int cc = 0; cc < a.nc; ++cc) {
    const int64_t g = a.c0 + cc;
    const int rhs = (int)(g / a.ncols);
    if (rhs != cur) {
      a.f[(int64_t)cur * a.ldf + i] += fma(wu.x, ar, -wu.y * ai);
      ar = ai = 0.0;
      cur = rhs;
    }
    const DevColSpec& cs = a.cols[(int)(g - (int64_t)rhs * a.ncols)];
    const int d = cs.delta;
    double wgt = rs * ipow(d >= 0 ? rv : irv, d >= 0 ? d : -d);
    if (cs.u1) wgt *= ipow(rp, cs.u1);
    const double2 y = Y[(int64_t)cc * a.F];
    ar = fma(wgt, y.x, ar);
    ai = fma(wgt, y.y, ai);
  }
  a.f[(int64_t)cur * a.ldf + i] += fma(wu.x, ar, -wu.y * ai);
}

}  // namespace

void launch_gen(const GenArgs& a, cudaStream_t st) {
  dim3 grid((unsigned)((a.F + 255) / 256), (unsigned)a.nc);
  k_gen<<<grid, 256, 0, st>>>(a);
}

void launch_out(const OutArgs& a, cudaStream_t st) {
  k_out<<<(unsigned)((a.R + 255) / 256), 256, 0, st>>>(a);
}

}  // namespace hk
