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
#include <type_traits>

#include "cplx.cuh"
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

// One CTA row (blockIdx.y) per stacked column at a time, so the column's indices are derived
// once per column; the threads of the row stride over the F points of the column.
template <class C>
__global__ void __launch_bounds__(256) k_gen(GenArgs a) {
  const int64_t ncolumns = (int64_t)a.nc * a.nsegc;
  const int64_t t0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x, dt = (int64_t)gridDim.x * blockDim.x;
  for (int64_t y = blockIdx.y; y < ncolumns; y += gridDim.y) {
    C* A = reinterpret_cast<C*>(a.A) + y * a.F;
    const int64_t cc = y / a.nsegc, sg = y - cc * a.nsegc;
    const int64_t g = a.c0 + cc;
    const int64_t rhs = g / a.ncols;
    const int l = a.lmap[g - rhs * a.ncols];
    const int64_t nlo = sg * a.S;                          // first column offset of this segment
    const int64_t lim = min(a.S, a.C - nlo);               // points t < lim carry data, the rest is padding
    const double* cr = a.c + rhs * a.ldc + (a.n0 - 1 + nlo);
    const double sc = a.scale ? a.scale[l] : 1.0;
    if (a.T) {
      const double2* tr = a.T + (int64_t)l * a.N + (a.n0 - 1 + nlo);
      for (int64_t t = t0; t < a.F; t += dt) {
        double2 v = make_double2(0.0, 0.0);
        if (t < lim) {
          const double cv = cr[t] * sc;
          const double2 x = tr[t];
          v = make_double2(cv * x.x, cv * x.y);
        }
        A[t] = from_d2<C>(v);
      }
      continue;
    }
    const DevColSpec& cs = a.cols[l];
    const int d = cs.delta;
    for (int64_t t = t0; t < a.F; t += dt) {
      if (t >= lim) {
        A[t] = from_d2<C>(make_double2(0.0, 0.0));
        continue;
      }
      const int64_t np = nlo + t;
      const int64_t i = a.n0 - 1 + np;
      const double bt = a.nodes.betan[i];
      double pr = cs.G[cs.nterm - 1].x, pim = cs.G[cs.nterm - 1].y;
      for (int u = cs.nterm - 2; u >= 0; --u) {
        pr = fma(pr, bt, cs.G[u].x);
        pim = fma(pim, bt, cs.G[u].y);
      }
      double pw = a.nodes.rs_omt[i] * ipow(d >= 0 ? a.nodes.omt[i] : a.nodes.inv_omt[i], d >= 0 ? d : -d);
      if (cs.u1) pw *= ipow(a.nodes.colpow[i], cs.u1);
      const double cv = cr[t] * pw * sc;
      const double xr = pr * cv, xi = pim * cv;
      const double2 w = a.wV[np];
      A[t] = from_d2<C>(make_double2(fma(xr, w.x, -xi * w.y), fma(xr, w.y, xi * w.x)));
    }
  }
}

// FP32 plans with per-block tables: every operation of the generation in FP32.
__global__ void __launch_bounds__(256) k_gen_f32(GenArgs a) {
  const int64_t ncolumns = (int64_t)a.nc * a.nsegc;
  const int64_t t0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x, dt = (int64_t)gridDim.x * blockDim.x;
  for (int64_t y = blockIdx.y; y < ncolumns; y += gridDim.y) {
    float2* A = reinterpret_cast<float2*>(a.A) + y * a.F;
    const int64_t cc = y / a.nsegc, sg = y - cc * a.nsegc;
    const int64_t g = a.c0 + cc;
    const int64_t rhs = g / a.ncols, li = g - rhs * a.ncols;  // kept-column position: per-block table row
    const int64_t nlo = sg * a.S;
    const int64_t lim = min(a.S, a.C - nlo);
    const float* cr = a.cf + rhs * a.ldcf + (a.n0 - 1 + nlo);
    const float2* tr = a.Tf + li * a.C + nlo;
    for (int64_t t = t0; t < a.F; t += dt) {
      float2 v = make_float2(0.f, 0.f);
      if (t < lim) {
        const float cv = __ldg(&cr[t]);
        const float2 x = __ldg(&tr[t]);
        v = make_float2(cv * x.x, cv * x.y);
      }
      A[t] = v;
    }
  }
}

// Thread per output row and CTA row (blockIdx.y) per right-hand side of the chunk: the thread
// adds up that right-hand side's stacked columns of the chunk in order l = lo..hi-1, so every
// f entry has one writer per chunk and the sum order is fixed.
template <class C>
__global__ void __launch_bounds__(256) k_out(OutArgs a) {
  const int64_t kp = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (kp >= a.R) return;
  const int64_t i = a.k0 - 1 + kp;
  double rv = 0.0, irv = 0.0, rs = 0.0, rp = 0.0;
  if (!a.W) {
    rv = a.nodes.rowvar[i];
    irv = a.nodes.inv_rowvar[i];
    rs = a.nodes.rs_rowvar[i];
    rp = a.nodes.rowpert[i];
  }
  const double2 wu = a.wU[kp];
  const int64_t sg = kp / a.Sr;
  const C* Y = reinterpret_cast<const C*>(a.Y) + sg * a.F + (kp - sg * a.Sr) + a.off;
  const int64_t r_first = a.c0 / a.ncols, r_last = (a.c0 + a.nc - 1) / a.ncols;
  for (int64_t rhs = r_first + blockIdx.y; rhs <= r_last; rhs += gridDim.y) {
    const int64_t lo = max(a.c0, rhs * a.ncols), hi = min(a.c0 + a.nc, (rhs + 1) * a.ncols);
    double ar = 0.0, ai = 0.0;
    for (int64_t g = lo; g < hi; ++g) {
      const int l = a.lmap[g - rhs * a.ncols];
      double wgt;
      if (a.W) {
        wgt = a.W[(int64_t)l * a.N + i];
      } else {
        const DevColSpec& cs = a.cols[l];
        const int d = cs.delta;
        wgt = rs * ipow(d >= 0 ? rv : irv, d >= 0 ? d : -d);
        if (cs.u1) wgt *= ipow(rp, cs.u1);
      }
      if (a.iscale) wgt *= a.iscale[l];
      const C y = Y[(g - a.c0) * a.nsegr * a.F];
      ar = fma(wgt, (double)y.x, ar);
      ai = fma(wgt, (double)y.y, ai);
    }
    a.f[rhs * a.ldf + i] += fma(wu.x, ar, -wu.y * ai);
  }
}

// FP32 plans with per-block tables: the sum over stacked columns and the row chirp in FP32,
// the addition into f in FP64.
__global__ void __launch_bounds__(256) k_out_f32(OutArgs a) {
  const int64_t kp = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (kp >= a.R) return;
  const int64_t i = a.k0 - 1 + kp;
  const double2 wud = a.wU[kp];
  const float2 wu = make_float2((float)wud.x, (float)wud.y);
  const int64_t sg = kp / a.Sr;
  const float2* Y = reinterpret_cast<const float2*>(a.Y) + sg * a.F + (kp - sg * a.Sr) + a.off;
  const int64_t r_first = a.c0 / a.ncols, r_last = (a.c0 + a.nc - 1) / a.ncols;
  for (int64_t rhs = r_first + blockIdx.y; rhs <= r_last; rhs += gridDim.y) {
    const int64_t lo = max(a.c0, rhs * a.ncols), hi = min(a.c0 + a.nc, (rhs + 1) * a.ncols);
    float ar = 0.f, ai = 0.f;
    for (int64_t g = lo; g < hi; ++g) {
      const int64_t li = g - rhs * a.ncols;  // kept-column position: per-block table row
      const float wgt = __ldg(&a.Wf[li * a.R + kp]);
      const float2 y = Y[(g - a.c0) * a.nsegr * a.F];
      ar = fmaf(wgt, y.x, ar);
      ai = fmaf(wgt, y.y, ai);
    }
    a.f[rhs * a.ldf + i] += (double)fmaf(wu.x, ar, -wu.y * ai);
  }
}

// Overlap-add of column segments: out[cc][t] = sum_s in[cc*nseg + s][t] H[s][t]. A CTA covers
// kMacPts consecutive points of one column; its kMacLanes thread rows split the segments
// (s = lane, lane + kMacLanes, ...) and the partial sums are added in a fixed order.
constexpr int kMacPts = 32, kMacLanes = 8;

template <class C>
__global__ void __launch_bounds__(kMacPts* kMacLanes) k_seg_mac(const C* __restrict__ in, const C* __restrict__ H,
                                                                 C* __restrict__ out, int64_t F, int64_t nseg) {
  typedef typename RealOf<C>::type R;
  __shared__ R sr[kMacLanes][kMacPts], si[kMacLanes][kMacPts];
  const int pt = threadIdx.x % kMacPts, lane = threadIdx.x / kMacPts;
  const int64_t tiles = F / kMacPts;
  const int64_t cc = blockIdx.x / tiles;
  const int64_t t = (blockIdx.x - cc * tiles) * kMacPts + pt;
  const C* x = in + cc * nseg * F + t;
  R ar = 0, ai = 0;
  for (int64_t s = lane; s < nseg; s += kMacLanes) {
    const C v = x[s * F];
    const C h = __ldg(&H[s * F + t]);
    ar = fmar(v.x, h.x, fmar(-v.y, h.y, ar));
    ai = fmar(v.x, h.y, fmar(v.y, h.x, ai));
  }
  sr[lane][pt] = ar;
  si[lane][pt] = ai;
  __syncthreads();
  if (lane == 0) {
    for (int j = 1; j < kMacLanes; ++j) {
      ar += sr[j][pt];
      ai += si[j][pt];
    }
    out[cc * F + t] = mkc(ar, ai);
  }
}

__global__ void __launch_bounds__(256) k_build_tables(TabArgs a) {
  const int64_t total = (int64_t)a.ncols * a.N;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int l = (int)(e / a.N);
    const int64_t i = e - (int64_t)l * a.N;
    const DevColSpec& cs = a.cols[l];
    const int d = cs.delta, ad = d >= 0 ? d : -d;
    const double bt = a.nodes.betan[i];
    double pr = cs.G[cs.nterm - 1].x, pim = cs.G[cs.nterm - 1].y;
    for (int u = cs.nterm - 2; u >= 0; --u) {
      pr = fma(pr, bt, cs.G[u].x);
      pim = fma(pim, bt, cs.G[u].y);
    }
    double pw = a.nodes.rs_omt[i] * ipow(d >= 0 ? a.nodes.omt[i] : a.nodes.inv_omt[i], ad);
    double rw = a.nodes.rs_rowvar[i] * ipow(d >= 0 ? a.nodes.rowvar[i] : a.nodes.inv_rowvar[i], ad);
    if (cs.u1) {
      pw *= ipow(a.nodes.colpow[i], cs.u1);
      rw *= ipow(a.nodes.rowpert[i], cs.u1);
    }
    const double2 w = chirp_phase(a.Va * (i + 1) + a.Vb, a.E, 1.0);
    const double xr = pr * pw, xi = pim * pw;
    a.T[e] = make_double2(fma(xr, w.x, -xi * w.y), fma(xr, w.y, xi * w.x));
    a.W[e] = rw;
  }
}

__global__ void __launch_bounds__(256) k_block_tables_f32(const double2* __restrict__ T, const double* __restrict__ W,
                                                         int64_t N, int nl, const int* __restrict__ lmap, int64_t n0,
                                                         int64_t C, int64_t k0, int64_t R,
                                                         const double* __restrict__ scale,
                                                         const double* __restrict__ iscale, float2* Tf, float* Wf) {
  const int64_t m = C > R ? C : R;
  const int64_t total = (int64_t)nl * m;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t li = e / m, j = e - li * m;
    const int64_t l = lmap[li];
    if (j < C) {
      const double2 x = T[l * N + n0 - 1 + j];
      Tf[li * C + j] = make_float2((float)(x.x * scale[l]), (float)(x.y * scale[l]));
    }
    if (j < R) Wf[li * R + j] = (float)(W[l * N + k0 - 1 + j] * iscale[l]);
  }
}

__global__ void __launch_bounds__(256) k_coeffs_f32(const double* __restrict__ c, int64_t ldc, float* cf, int64_t N,
                                                   int64_t total) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = e / N, i = e - r * N;
    cf[e] = (float)c[r * ldc + i];
  }
}

__global__ void __launch_bounds__(256) k_diag_scale(const double* x, int64_t ldx, const double* __restrict__ v,
                                                    double scale, double* out, int64_t ldo, int64_t N, int64_t total) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = e / N, i = e - r * N;
    out[r * ldo + i] = scale * v[i] * x[r * ldx + i];
  }
}

unsigned grid1d(int64_t n) {
  int64_t g = (n + 255) / 256;
  return (unsigned)std::min<int64_t>(std::max<int64_t>(g, 1), int64_t(152) * 32);
}

}  // namespace

// Each thread writes up to kGenPts points of a column.
constexpr int64_t kGenPts = 4;

template <class C>
void launch_gen(const GenArgs& a, cudaStream_t st) {
  const int64_t ny = std::min<int64_t>((int64_t)a.nc * a.nsegc, 65535);
  dim3 grid((unsigned)((a.F + 256 * kGenPts - 1) / (256 * kGenPts)), (unsigned)ny);
  if (std::is_same<C, float2>::value && a.Tf) k_gen_f32<<<grid, 256, 0, st>>>(a);
  else k_gen<C><<<grid, 256, 0, st>>>(a);
}

template <class C>
void launch_seg_mac(const C* in, const C* H, C* out, int64_t F, int64_t nseg, int nc, cudaStream_t st) {
  // F >= 64 is a multiple of kMacPts
  const int64_t blocks = (F / kMacPts) * nc;
  k_seg_mac<C><<<(unsigned)blocks, kMacPts * kMacLanes, 0, st>>>(in, H, out, F, nseg);
}

void launch_build_tables(const TabArgs& a, cudaStream_t st) {
  k_build_tables<<<grid1d((int64_t)a.ncols * a.N), 256, 0, st>>>(a);
}

template <class C>
void launch_out(const OutArgs& a, cudaStream_t st) {
  const int64_t nr = (a.c0 + a.nc - 1) / a.ncols - a.c0 / a.ncols + 1;  // right-hand sides in the chunk
  dim3 grid((unsigned)((a.R + 255) / 256), (unsigned)std::min<int64_t>(nr, 65535));
  if (std::is_same<C, float2>::value && a.Wf) k_out_f32<<<grid, 256, 0, st>>>(a);
  else k_out<C><<<grid, 256, 0, st>>>(a);
}

void launch_block_tables_f32(const double2* T, const double* W, int64_t N, int nl, const int* lmap, int64_t n0,
                             int64_t C, int64_t k0, int64_t R, const double* scale, const double* iscale, float2* Tf,
                             float* Wf, cudaStream_t st) {
  k_block_tables_f32<<<grid1d((int64_t)nl * std::max(C, R)), 256, 0, st>>>(T, W, N, nl, lmap, n0, C, k0, R, scale,
                                                                            iscale, Tf, Wf);
}

void launch_diag_scale(const double* x, int64_t ldx, const double* v, double scale, double* out, int64_t ldo,
                       int64_t N, int nrhs, cudaStream_t st) {
  const int64_t total = N * nrhs;
  k_diag_scale<<<grid1d(total), 256, 0, st>>>(x, ldx, v, scale, out, ldo, N, total);
}

void launch_coeffs_f32(const double* c, int64_t ldc, float* cf, int64_t N, int nrhs, cudaStream_t st) {
  const int64_t total = N * nrhs;
  k_coeffs_f32<<<grid1d(total), 256, 0, st>>>(c, ldc, cf, N, total);
}

template void launch_gen<double2>(const GenArgs&, cudaStream_t);
template void launch_gen<float2>(const GenArgs&, cudaStream_t);
template void launch_out<double2>(const OutArgs&, cudaStream_t);
template void launch_out<float2>(const OutArgs&, cudaStream_t);
template void launch_seg_mac<double2>(const double2*, const double2*, double2*, int64_t, int64_t, int, cudaStream_t);
template void launch_seg_mac<float2>(const float2*, const float2*, float2*, int64_t, int64_t, int, cudaStream_t);

}  // namespace hk
