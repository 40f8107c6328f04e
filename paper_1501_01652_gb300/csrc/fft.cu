// Multi-column power-of-two FFT (Stockham autosort, FP64) and the chirp-z
// helpers of the far field.
//
// A pass with current sub-length n and stride s (n*s = F) computes, for
// every pair (p, q) with p < n/R, q < s, the R-point DFT of
// x[q + s(p + j n/R)], j < R, multiplies output r by W_n^{p r}, and stores it
// at y[q + s(R p + r)]; after passes with radices R_1 R_2 ... = F the output
// is in natural order. One CTA handles kTile consecutive pairs (so every
// global load and store touches kTile or more consecutive elements) and does
// the R-point DFT in shared memory with radix-4/radix-2 Stockham steps.
#include <cuda_runtime.h>

#include <algorithm>

#include "kernels.cuh"

namespace hk {

namespace {

constexpr int kTile = 16;
constexpr int kFftThreads = 256;

__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
  return make_double2(fma(a.x, b.x, -a.y * b.y), fma(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ double2 cadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 csub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }

template <bool INV>
__device__ __forceinline__ double2 twiddle(const double2* __restrict__ tw, int64_t idx) {
  double2 t = __ldg(&tw[idx]);
  if (INV) t.y = -t.y;
  return t;
}

// R-point DFTs of kTile sequences held as a[e * kTile + i] (element e, sequence i).
// Returns the buffer (a or b) that holds the result in natural order.
template <int LOGR, bool INV>
__device__ double2* smem_dft(double2* a, double2* b, const double2* __restrict__ tw, int logFmax) {
  constexpr int R = 1 << LOGR;
  int logn = LOGR, logs = 0;
  while (logn >= 2) {
    const int n4 = 1 << (logn - 2);
    const int s = 1 << logs;
    const int tshift = logFmax - logn;
    for (int idx = threadIdx.x; idx < kTile * (R / 4); idx += blockDim.x) {
      const int i = idx & (kTile - 1);
      const int bf = idx / kTile;
      const int pp = bf >> logs, qq = bf & (s - 1);
      const double2 a0 = a[(qq + s * pp) * kTile + i];
      const double2 a1 = a[(qq + s * (pp + n4)) * kTile + i];
      const double2 a2 = a[(qq + s * (pp + 2 * n4)) * kTile + i];
      const double2 a3 = a[(qq + s * (pp + 3 * n4)) * kTile + i];
      const double2 t0 = cadd(a0, a2), t1 = csub(a0, a2), t2 = cadd(a1, a3), t3 = csub(a1, a3);
      // -i t3 (forward) or +i t3 (inverse)
      const double2 jt3 = INV ? make_double2(-t3.y, t3.x) : make_double2(t3.y, -t3.x);
      double2 b0 = cadd(t0, t2), b1 = cadd(t1, jt3), b2 = csub(t0, t2), b3 = csub(t1, jt3);
      if (pp != 0) {
        b1 = cmul(b1, twiddle<INV>(tw, (int64_t)(pp) << tshift));
        b2 = cmul(b2, twiddle<INV>(tw, (int64_t)(2 * pp) << tshift));
        b3 = cmul(b3, twiddle<INV>(tw, (int64_t)(3 * pp) << tshift));
      }
      const int o = qq + s * 4 * pp;
      b[(o)*kTile + i] = b0;
      b[(o + s) * kTile + i] = b1;
      b[(o + 2 * s) * kTile + i] = b2;
      b[(o + 3 * s) * kTile + i] = b3;
    }
    __syncthreads();
    double2* t = a;
    a = b;
    b = t;
    logn -= 2;
    logs += 2;
  }
  if (logn == 1) {
    const int s = 1 << logs;  // = R/2
    for (int idx = threadIdx.x; idx < kTile * (R / 2); idx += blockDim.x) {
      const int i = idx & (kTile - 1);
      const int qq = idx / kTile;
      const double2 a0 = a[qq * kTile + i];
      const double2 a1 = a[(qq + s) * kTile + i];
      b[qq * kTile + i] = cadd(a0, a1);
      b[(qq + s) * kTile + i] = csub(a0, a1);
    }
    __syncthreads();
    double2* t = a;
    a = b;
    b = t;
  }
  return a;
}

template <int LOGR, bool INV>
__global__ void __launch_bounds__(kFftThreads) k_fft_pass(const double2* __restrict__ src, double2* __restrict__ dst,
                                                          int logF, int logS, const double2* __restrict__ tw,
                                                          int logFmax) {
  constexpr int R = 1 << LOGR;
  extern __shared__ double2 sm[];
  double2* v = sm;
  double2* w = sm + R * kTile;
  const int64_t F = int64_t(1) << logF;
  const int64_t FR = F >> LOGR;  // pairs per column, a multiple of kTile
  const int64_t G0 = (int64_t)blockIdx.x * kTile;
  const int64_t col = G0 / FR;
  const int64_t pi0 = G0 - col * FR;
  const double2* x = src + col * F;
  double2* y = dst + col * F;
  for (int idx = threadIdx.x; idx < R * kTile; idx += blockDim.x) {
    const int i = idx & (kTile - 1), j = idx / kTile;
    v[j * kTile + i] = x[pi0 + i + (int64_t)j * FR];
  }
  __syncthreads();
  const double2* res = smem_dft<LOGR, INV>(v, w, tw, logFmax);
  const int64_t s = int64_t(1) << logS;
  const int tshift = logFmax - logF;
  if (s >= kTile) {
    const int64_t p = pi0 >> logS, q0 = pi0 & (s - 1);
    for (int idx = threadIdx.x; idx < R * kTile; idx += blockDim.x) {
      const int i = idx & (kTile - 1), r = idx / kTile;
      double2 val = res[r * kTile + i];
      const int64_t e = ((p * r) << logS) & (F - 1);
      if (e) val = cmul(val, twiddle<INV>(tw, e << tshift));
      y[q0 + i + s * (p * R + r)] = val;
    }
  } else {
    const int64_t p0 = pi0 >> logS;
    const int64_t base = (p0 << logS) << LOGR;  // s R p0
    for (int idx = threadIdx.x; idx < R * kTile; idx += blockDim.x) {
      const int pl = idx >> (logS + LOGR);
      const int rem = idx & ((int)(s << LOGR) - 1);
      const int r = rem >> logS, q = rem & ((int)s - 1);
      double2 val = res[r * kTile + ((pl << logS) + q)];
      const int64_t e = (((p0 + pl) * r) << logS) & (F - 1);
      if (e) val = cmul(val, twiddle<INV>(tw, e << tshift));
      y[base + idx] = val;
    }
  }
}

template <int LOGR, bool INV>
void launch_pass(const double2* src, double2* dst, int logF, int logS, int ncols, const double2* tw, int logFmax,
                 cudaStream_t st) {
  constexpr int R = 1 << LOGR;
  const size_t smem = 2 * (size_t)R * kTile * sizeof(double2);
  static bool configured = false;
  if (!configured) {
    cudaFuncSetAttribute(k_fft_pass<LOGR, INV>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    configured = true;
  }
  const int64_t pairs = ((int64_t)ncols << logF) >> LOGR;
  const int64_t grid = pairs / kTile;
  k_fft_pass<LOGR, INV><<<(unsigned)grid, kFftThreads, smem, st>>>(src, dst, logF, logS, tw, logFmax);
}

template <bool INV>
void launch_pass_r(int logR, const double2* src, double2* dst, int logF, int logS, int ncols, const double2* tw,
                   int logFmax, cudaStream_t st) {
  switch (logR) {
    case 1: launch_pass<1, INV>(src, dst, logF, logS, ncols, tw, logFmax, st); break;
    case 2: launch_pass<2, INV>(src, dst, logF, logS, ncols, tw, logFmax, st); break;
    case 3: launch_pass<3, INV>(src, dst, logF, logS, ncols, tw, logFmax, st); break;
    case 4: launch_pass<4, INV>(src, dst, logF, logS, ncols, tw, logFmax, st); break;
    case 5: launch_pass<5, INV>(src, dst, logF, logS, ncols, tw, logFmax, st); break;
    case 6: launch_pass<6, INV>(src, dst, logF, logS, ncols, tw, logFmax, st); break;
    default: launch_pass<7, INV>(src, dst, logF, logS, ncols, tw, logFmax, st); break;
  }
}

__global__ void k_twiddles(double2* tw, int logF) {
  const int64_t F = int64_t(1) << logF;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < F; t += (int64_t)gridDim.x * blockDim.x) {
    double s, c;
    // exp(-2 pi i t / F): the argument 2t/F is exact in binary
    sincospi(-2.0 * (double)t / (double)F, &s, &c);
    tw[t] = make_double2(c, s);
  }
}

// exp(i pi q / (2E)) for q = v^2 mod 4E (the period of the phase in v^2).
__device__ __forceinline__ double2 chirp_phase(int64_t v, int64_t E, double sign) {
  const int64_t m = 4 * E;
  int64_t a = v % m;
  if (a < 0) a += m;
  // a^2 < 16 E^2 fits in 64 bits for E < 2^30
  const int64_t q = (int64_t)(((unsigned long long)a * (unsigned long long)a) % (unsigned long long)m);
  double s, c;
  sincospi((double)q / (double)(2 * E), &s, &c);
  return make_double2(c, sign * s);
}

__global__ void k_chirps(ChirpGeom g, double2* wU, double2* wV) {
  const int64_t n = g.R > g.C ? g.R : g.C;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x) {
    if (t < g.R) wU[t] = chirp_phase(g.Ua * (g.k0 + t) + g.Ub, g.E, 1.0);
    if (t < g.C) wV[t] = chirp_phase(g.Va * (g.n0 + t) + g.Vb, g.E, 1.0);
  }
}

__global__ void k_seg_hh(SegGeom g, double2* hh) {
  const int64_t total = g.nseg * g.F;
  const int64_t L = g.Rr + g.Cc - 1;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t y = e / g.F, t = e - y * g.F;
    if (t < L) {
      // U_k - V_n with k - n = t - (Cc-1) + (k0 + y dk) - (n0 + y dn)
      const int64_t duv = g.Ua * (t - (g.Cc - 1) + (g.k0 + y * g.dk) - (g.n0 + y * g.dn)) + (g.Ub - g.Vb);
      hh[e] = chirp_phase(duv, g.E, -1.0);
    } else {
      hh[e] = make_double2(0.0, 0.0);
    }
  }
}

__global__ void k_scale_copy(const double2* src, double2* dst, int64_t n, double scale) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x)
    dst[t] = make_double2(src[t].x * scale, src[t].y * scale);
}

__global__ void k_pointwise(double2* y, const double2* __restrict__ H, int64_t F, int64_t total) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x)
    y[t] = cmul(y[t], __ldg(&H[t & (F - 1)]));
}

unsigned grid_for(int64_t n, int threads) {
  int64_t g = (n + threads - 1) / threads;
  return (unsigned)std::min<int64_t>(std::max<int64_t>(g, 1), int64_t(152) * 64);
}

}  // namespace

void launch_twiddles(double2* tw, int logF, cudaStream_t st) {
  k_twiddles<<<grid_for(int64_t(1) << logF, 256), 256, 0, st>>>(tw, logF);
}

void launch_chirps(const ChirpGeom& g, double2* wU, double2* wV, cudaStream_t st) {
  k_chirps<<<grid_for(g.R > g.C ? g.R : g.C, 256), 256, 0, st>>>(g, wU, wV);
}

void launch_seg_hh(const SegGeom& g, double2* hh, cudaStream_t st) {
  k_seg_hh<<<grid_for(g.nseg * g.F, 256), 256, 0, st>>>(g, hh);
}

void launch_scale_copy(const double2* src, double2* dst, int64_t n, double scale, cudaStream_t st) {
  k_scale_copy<<<grid_for(n, 256), 256, 0, st>>>(src, dst, n, scale);
}

void launch_pointwise(double2* y, const double2* H, int64_t F, int ncols, cudaStream_t st) {
  const int64_t total = F * ncols;
  k_pointwise<<<grid_for(total, 256), 256, 0, st>>>(y, H, F, total);
}

int run_fft(double2* a, double2* b, int logF, int ncols, bool inverse, const double2* tw, int logFmax,
            cudaStream_t st, double2** result, int* npasses) {
  if (logF < 6 || logF > logFmax) return HANKEL_EINVAL;
  const int maxlog = std::min(7, logF - 4);  // keeps F/R >= kTile pairs per column
  const int np = (logF + maxlog - 1) / maxlog;
  const int base = logF / np, extra = logF % np;
  double2* src = a;
  double2* dst = b;
  int logS = 0;
  for (int i = 0; i < np; ++i) {
    const int lr = base + (i < extra ? 1 : 0);
    if (inverse) launch_pass_r<true>(lr, src, dst, logF, logS, ncols, tw, logFmax, st);
    else launch_pass_r<false>(lr, src, dst, logF, logS, ncols, tw, logFmax, st);
    logS += lr;
    std::swap(src, dst);
  }
  *result = src;
  if (npasses) *npasses = np;
  return HANKEL_OK;
}

}  // namespace hk
