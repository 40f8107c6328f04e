// Far-field row accumulation, the overlap-add of column segments, the coefficient conversions
// and the plan-time block tables (column generation runs inside the first forward FFT loads,
// fft.cu).
//
// Column side (Sections 4.1, 5.1, 6): stacked column li of a block holds
//   g_li(n) = c_n V_li(n) exp(i pi V_n^2/(2E)),
// where V_li is either one stacked column of the rearranged expansion -- the complex G merge
// the Hankel coefficients (-1)^m a_m(mu), the phases exp(-i(2mu+1)pi/4) and the Neumann/Taylor
// weights of every term whose row factor is the same function of k -- or a term of the
// block's low-rank form. Row side: f_k += Re[ exp(i pi U_k^2/(2E)) sum_li U_li(k) y_li(k) ].
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

// Thread per output row and CTA row (blockIdx.y) per right-hand side of the chunk: the thread
// adds up that right-hand side's stacked columns of the chunk in order li = lo..hi-1, only the
// real part (the row chirp is folded into the weights Ut), in the plan precision; the addition
// into f is FP64. Every f entry has one writer per chunk and the sum order is fixed.
template <class C>
__global__ void __launch_bounds__(256) k_out(OutArgs a) {
  typedef typename RealOf<C>::type R;
  const int64_t kp = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (kp >= a.R) return;
  const int64_t i = a.k0 - 1 + kp;
  const int64_t sg = kp / a.Sr;
  const C* Y = reinterpret_cast<const C*>(a.Y) + sg * a.F + (kp - sg * a.Sr) + a.off;
  const C* Ut = reinterpret_cast<const C*>(a.Ut) + kp;
  const int64_t r_first = a.c0 / a.ncols, r_last = (a.c0 + a.nc - 1) / a.ncols;
  const int64_t ystride = a.nsegr * a.F;
  for (int64_t rhs = r_first + blockIdx.y; rhs <= r_last; rhs += gridDim.y) {
    const int64_t lo = max(a.c0, rhs * a.ncols), hi = min(a.c0 + a.nc, (rhs + 1) * a.ncols);
    R ar = 0;
    const C* wp = Ut + (lo - rhs * a.ncols) * a.R;
    const C* yp = Y + (lo - a.c0) * ystride;
    // unrolled so that several iterations' loads are in flight; the sum keeps its order
#pragma unroll 4
    for (int g = (int)(hi - lo); g > 0; --g) {
      const C w = ldgc(wp);
      const C y = *yp;
      ar = fmar(w.x, y.x, fmar(-w.y, y.y, ar));
      wp += a.R;
      yp += ystride;
    }
    a.f[rhs * a.ldf + i] += a.cexp ? ldexp((double)ar, a.cexp[rhs]) : (double)ar;
  }
}

// Overlap-add of column segments: out[cc][t] = sum_s in[cc*nseg + s][t] H[s][t]. A CTA of
// kMacThreads threads covers P = kMacThreads / L consecutive points of one column; its L thread
// rows split the segments (s = lane, lane + L, ...) and the L partial sums are added in a fixed
// order. L (1, 2, 4 or 8) depends on the block alone (its segment count and F), so a column's
// result does not depend on how many columns run together.
constexpr int kMacThreads = 256, kMacLogThreads = 8;

template <class C>
__global__ void __launch_bounds__(kMacThreads) k_seg_mac(const C* __restrict__ in, const C* __restrict__ H,
                                                          C* __restrict__ out, int64_t F, int64_t nseg, int logL) {
  typedef typename RealOf<C>::type R;
  __shared__ R sr[kMacThreads], si[kMacThreads];
  const int logP = kMacLogThreads - logL;
  const int pt = threadIdx.x & ((1 << logP) - 1), lane = threadIdx.x >> logP;
  const int64_t tiles = F >> logP;
  const int64_t cc = blockIdx.x / tiles;
  const int64_t t = ((blockIdx.x - cc * tiles) << logP) + pt;
  const C* x = in + cc * nseg * F + lane * F + t;
  const C* hp = H + lane * F + t;
  const int64_t step = F << logL;
  R ar = 0, ai = 0;
  // unrolled so that several iterations' loads are in flight; the sums keep their order
#pragma unroll 4
  for (int s = (int)((nseg - lane + (1 << logL) - 1) >> logL); s > 0; --s) {
    const C v = *x;
    const C h = ldgc(hp);
    ar = fmar(v.x, h.x, fmar(-v.y, h.y, ar));
    ai = fmar(v.x, h.y, fmar(v.y, h.x, ai));
    x += step;
    hp += step;
  }
  if (logL == 0) {  // the same for the whole CTA
    out[cc * F + t] = mkc(ar, ai);
    return;
  }
  sr[threadIdx.x] = ar;
  si[threadIdx.x] = ai;
  __syncthreads();
  if (lane == 0) {
    for (int j = 1; j < (1 << logL); ++j) {
      ar += sr[(j << logP) + pt];
      ai += si[(j << logP) + pt];
    }
    out[cc * F + t] = mkc(ar, ai);
  }
}

// Chebyshev series sum_{j < P} a_j T_j(x) by Clenshaw's recurrence (complex a_j):
// b_j = a_j + 2 x b_{j+1} - b_{j+2}, value a_0 + x b_1 - b_2.
__device__ __forceinline__ double2 cheb_series(const double2* __restrict__ a, int P, double x) {
  const double x2 = 2.0 * x;
  double br = 0.0, bi = 0.0, cr = 0.0, ci = 0.0;  // b_{j+1}, b_{j+2}
  for (int j = P - 1; j >= 1; --j) {
    const double2 aj = __ldg(&a[j]);
    const double tr = fma(x2, br, aj.x - cr), ti = fma(x2, bi, aj.y - ci);
    cr = br;
    ci = bi;
    br = tr;
    bi = ti;
  }
  const double2 a0 = __ldg(&a[0]);
  return make_double2(fma(x, br, a0.x - cr), fma(x, bi, a0.y - ci));
}

// The column table of a block: thread per column n, every li of the block.
template <class C>
__global__ void __launch_bounds__(128) k_block_cols(BlockTabArgs a) {
  C* Vt = reinterpret_cast<C*>(a.Vt);
  for (int64_t np = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; np < a.C; np += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = a.n0 - 1 + np;
    const double2 w = a.wV[np];
    if (a.P > 0) {
      const double x = a.ln1 > a.ln0 ? (2.0 * log((double)(a.n0 + np)) - a.ln0 - a.ln1) / (a.ln1 - a.ln0) : 0.0;
      for (int li = 0; li < a.nl; ++li) {
        const double2 v = cheb_series(a.vcheb + (int64_t)li * a.P, a.P, x);
        const double vr = v.x, vi = v.y;
        const double sc = a.scale ? a.scale[li] : 1.0;
        Vt[(int64_t)li * a.C + np] = from_d2<C>(make_double2(sc * fma(vr, w.x, -vi * w.y), sc * fma(vr, w.y, vi * w.x)));
      }
    } else {
      const double bt = a.nodes.betan[i];
      for (int li = 0; li < a.nl; ++li) {
        const DevColSpec& cs = a.cols[a.lmap[li]];
        double pr = cs.G[cs.nterm - 1].x, pim = cs.G[cs.nterm - 1].y;
        for (int u = cs.nterm - 2; u >= 0; --u) {
          pr = fma(pr, bt, cs.G[u].x);
          pim = fma(pim, bt, cs.G[u].y);
        }
        const int d = cs.delta;
        double pw = a.nodes.rs_omt[i] * ipow(d >= 0 ? a.nodes.omt[i] : a.nodes.inv_omt[i], d >= 0 ? d : -d);
        if (cs.u1) pw *= ipow(a.nodes.colpow[i], cs.u1);
        if (a.scale) pw *= a.scale[li];
        const double xr = pr * pw, xi = pim * pw;
        Vt[(int64_t)li * a.C + np] = from_d2<C>(make_double2(fma(xr, w.x, -xi * w.y), fma(xr, w.y, xi * w.x)));
      }
    }
  }
}

// The row table of a block: thread per row k, every li of the block.
template <class C>
__global__ void __launch_bounds__(128) k_block_rows(BlockTabArgs a) {
  C* Ut = reinterpret_cast<C*>(a.Ut);
  for (int64_t kp = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; kp < a.R; kp += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = a.k0 - 1 + kp;
    const double2 w = a.wU[kp];
    if (a.P > 0) {
      const double x = a.lk1 > a.lk0 ? (2.0 * log((double)(a.k0 + kp)) - a.lk0 - a.lk1) / (a.lk1 - a.lk0) : 0.0;
      for (int li = 0; li < a.nl; ++li) {
        const double2 u = cheb_series(a.ucheb + (int64_t)li * a.P, a.P, x);
        const double isc = a.scale ? 1.0 / a.scale[li] : 1.0;
        Ut[(int64_t)li * a.R + kp] = from_d2<C>(
            make_double2(isc * fma(u.x, w.x, -u.y * w.y), isc * fma(u.x, w.y, u.y * w.x)));
      }
    } else {
      const double rv = a.nodes.rowvar[i], irv = a.nodes.inv_rowvar[i], rs = a.nodes.rs_rowvar[i];
      const double rp = a.nodes.rowpert[i];
      for (int li = 0; li < a.nl; ++li) {
        const DevColSpec& cs = a.cols[a.lmap[li]];
        const int d = cs.delta;
        double wgt = rs * ipow(d >= 0 ? rv : irv, d >= 0 ? d : -d);
        if (cs.u1) wgt *= ipow(rp, cs.u1);
        if (a.scale) wgt /= a.scale[li];
        Ut[(int64_t)li * a.R + kp] = from_d2<C>(make_double2(wgt * w.x, wgt * w.y));
      }
    }
  }
}

__global__ void __launch_bounds__(256) k_coef_exponent(const double* __restrict__ c, int64_t ldc, int64_t N,
                                                       int* cexp) {
  const int64_t r = blockIdx.y;
  int m = 0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x)
    m = max(m, (int)(((unsigned long long)__double_as_longlong(c[r * ldc + i]) >> 52) & 0x7ff));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
  // cexp[r] starts at -1022 (E = 0); the biased exponent E maps to E - 1022
  if ((threadIdx.x & 31) == 0 && m > 0) atomicMax(&cexp[r], m - 1022);
}

__global__ void k_coef_exponent_init(int* cexp, int nrhs) {
  for (int r = threadIdx.x; r < nrhs; r += blockDim.x) cexp[r] = -1022;
}

__global__ void __launch_bounds__(256) k_coeffs_f32(const double* __restrict__ c, int64_t ldc, float* cf, int64_t N,
                                                   int64_t total, const int* __restrict__ cexp) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = e / N, i = e - r * N;
    cf[e] = (float)ldexp(c[r * ldc + i], -cexp[r]);
  }
}

__global__ void __launch_bounds__(256) k_coeffs_df64(const double* __restrict__ c, int64_t ldc, float2* cd,
                                                    int64_t N, int64_t total, const int* __restrict__ cexp) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = e / N, i = e - r * N;
    const double x = ldexp(c[r * ldc + i], -cexp[r]);
    const float h = (float)x;
    cd[e] = make_float2(h, (float)(x - (double)h));
  }
}

__global__ void __launch_bounds__(256) k_add_lanes(double* f, int64_t ldf, const double* __restrict__ a0,
                                                   const double* __restrict__ a1, int64_t N, int64_t total) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = e / N, i = e - r * N;
    double v = f[r * ldf + i] + a0[e];
    if (a1) v += a1[e];
    f[r * ldf + i] = v;
  }
}

__global__ void __launch_bounds__(256) k_diag_scale(const double* x, int64_t ldx, const double* __restrict__ v,
                                                    double scale, double* out, int64_t ldo, int64_t N, int64_t total) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = e / N, i = e - r * N;
    out[r * ldo + i] = scale * v[i] * x[r * ldx + i];
  }
}

// Seeded values in [-1/2, 1/2): doubles (as_float = 0) or floats over n 4-byte words.
__global__ void k_fill_pattern(void* p, int64_t n, int as_float) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x) {
    unsigned long long h = (unsigned long long)t * 0x9E3779B97F4A7C15ULL;
    h ^= h >> 29;
    h *= 0xBF58476D1CE4E5B9ULL;
    h ^= h >> 32;
    const double v = (double)(h >> 11) * 0x1p-53 - 0.5;
    if (as_float) reinterpret_cast<float*>(p)[t] = (float)v;
    else if ((t & 1) == 0 && t + 1 < n) reinterpret_cast<double*>(p)[t >> 1] = v;
  }
}

unsigned grid1d(int64_t n) {
  int64_t g = (n + 255) / 256;
  return (unsigned)std::min<int64_t>(std::max<int64_t>(g, 1), int64_t(152) * 32);
}

}  // namespace


template <class C>
void launch_out(const OutArgs& a, cudaStream_t st) {
  const int64_t nr = (a.c0 + a.nc - 1) / a.ncols - a.c0 / a.ncols + 1;  // right-hand sides in the chunk
  dim3 grid((unsigned)((a.R + 255) / 256), (unsigned)std::min<int64_t>(nr, 65535));
  k_out<C><<<grid, 256, 0, st>>>(a);
}

template <class C>
void launch_block_tables(const BlockTabArgs& a, cudaStream_t st) {
  k_block_cols<C><<<(unsigned)std::min<int64_t>((a.C + 127) / 128, 152 * 16), 128, 0, st>>>(a);
  k_block_rows<C><<<(unsigned)std::min<int64_t>((a.R + 127) / 128, 152 * 16), 128, 0, st>>>(a);
}

void launch_diag_scale(const double* x, int64_t ldx, const double* v, double scale, double* out, int64_t ldo,
                       int64_t N, int nrhs, cudaStream_t st) {
  const int64_t total = N * nrhs;
  k_diag_scale<<<grid1d(total), 256, 0, st>>>(x, ldx, v, scale, out, ldo, N, total);
}

template <class C>
void launch_seg_mac(const C* in, const C* H, C* out, int64_t F, int64_t nseg, int nc, cudaStream_t st) {
  // thread rows per point: one while a thread's segment loop is short, up to eight for long ones;
  // a CTA's points (kMacThreads / L) stay within one column (F >= 64, a power of two)
  int logF = 0;
  while ((int64_t(1) << logF) < F) ++logF;
  int logL = nseg >= 128 ? 3 : nseg >= 64 ? 2 : nseg >= 32 ? 1 : 0;
  logL = std::max(logL, kMacLogThreads - logF);
  const int64_t blocks = (F >> (kMacLogThreads - logL)) * nc;
  k_seg_mac<C><<<(unsigned)blocks, kMacThreads, 0, st>>>(in, H, out, F, nseg, logL);
}

void launch_add_lanes(double* f, int64_t ldf, const double* const* acc, int nacc, int64_t N, int nrhs,
                      cudaStream_t st) {
  const int64_t total = N * (int64_t)nrhs;
  k_add_lanes<<<grid1d(total), 256, 0, st>>>(f, ldf, acc[0], nacc > 1 ? acc[1] : nullptr, N, total);
}

void launch_fill_pattern(void* p, size_t words, int as_float, cudaStream_t st) {
  k_fill_pattern<<<grid1d((int64_t)words), 256, 0, st>>>(p, (int64_t)words, as_float);
}

void launch_coef_exponent(const double* c, int64_t ldc, int64_t N, int nrhs, int* cexp, cudaStream_t st) {
  k_coef_exponent_init<<<1, 256, 0, st>>>(cexp, nrhs);
  const unsigned bx = (unsigned)std::min<int64_t>((N + 255) / 256, std::max<int64_t>(1, 608 / nrhs));
  k_coef_exponent<<<dim3(bx, (unsigned)nrhs), 256, 0, st>>>(c, ldc, N, cexp);
}

void launch_coeffs_f32(const double* c, int64_t ldc, float* cf, int64_t N, int nrhs, const int* cexp,
                       cudaStream_t st) {
  const int64_t total = N * nrhs;
  k_coeffs_f32<<<grid1d(total), 256, 0, st>>>(c, ldc, cf, N, total, cexp);
}

void launch_coeffs_df64(const double* c, int64_t ldc, float2* cd, int64_t N, int nrhs, const int* cexp,
                        cudaStream_t st) {
  const int64_t total = N * (int64_t)nrhs;
  k_coeffs_df64<<<grid1d(total), 256, 0, st>>>(c, ldc, cd, N, total, cexp);
}

template void launch_seg_mac<df64c>(const df64c*, const df64c*, df64c*, int64_t, int64_t, int, cudaStream_t);
template void launch_seg_mac<double2>(const double2*, const double2*, double2*, int64_t, int64_t, int, cudaStream_t);
template void launch_seg_mac<float2>(const float2*, const float2*, float2*, int64_t, int64_t, int, cudaStream_t);
template void launch_block_tables<double2>(const BlockTabArgs&, cudaStream_t);
template void launch_block_tables<float2>(const BlockTabArgs&, cudaStream_t);
template void launch_block_tables<df64c>(const BlockTabArgs&, cudaStream_t);
template void launch_out<df64c>(const OutArgs&, cudaStream_t);
template void launch_out<double2>(const OutArgs&, cudaStream_t);
template void launch_out<float2>(const OutArgs&, cudaStream_t);

}  // namespace hk
