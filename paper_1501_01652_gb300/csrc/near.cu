// Near field (the direct part J^EVAL of Eqs. 18-19 and the directly summed
// leading rows/columns of Sections 5-6): f_k = sum_{n <= nend(k)} c_n J_nu(r_k omega_n)
// with J evaluated per entry, over tiles of 32 rows x 512 columns of the near set.
//
// J_nu on [0, zmax] comes from a table of Taylor polynomials about the centres of
// intervals of width 1/kJTabSub (built at plan time from the Neumann addition formula,
// Eq. 8, with the degree set by eps), so one evaluation costs a table row load and
// deg FMAs.
#include <cuda_runtime.h>

#include <algorithm>

#include "cplx.cuh"
#include "kernels.cuh"

namespace hk {

namespace {

// Right-hand sides handled per table evaluation: every entry's J is evaluated once per group
// of G vectors (G = 1, 2, 4, 8 or 16, the smallest that covers nrhs, groups of 16 beyond).
constexpr int kMaxRhsGroup = 16;

template <class R>
__device__ __forceinline__ R table_j(const R* __restrict__ jtab, int64_t jt_n, int deg, R z) {
  int64_t i = (int64_t)(z * (R)kJTabSub);
  i = i < 0 ? 0 : (i >= jt_n ? jt_n - 1 : i);
  const R d = z - ((R)i + (R)0.5) * ((R)1 / (R)kJTabSub);
  const R* t = jtab + i * (deg + 1);
  R v = __ldg(&t[deg]);
  for (int j = deg - 1; j >= 0; --j) v = fmar(v, d, __ldg(&t[j]));
  return v;
}

// Warp per tile, lane per row: every lane walks the same columns n (so the loads of omega_n and
// of c_n for each vector are warp-wide broadcasts) and stops at its own prefix end; the sum
// over n is the lane's own, in increasing n, with no cross-lane reduction.
template <class R, int G, class CT>
__global__ void __launch_bounds__(256) k_near(const NearItem* __restrict__ items, int64_t nitems,
                                              const int64_t* __restrict__ nend, int64_t N, R* partial, int nrhs,
                                              const CT* __restrict__ c, int64_t ldc, double* f, int64_t ldf,
                                              const R* __restrict__ r_true, const R* __restrict__ om_true,
                                              const R* __restrict__ jtab, int64_t jt_n, int deg) {
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (warp >= nitems) return;
  const NearItem it = items[warp];
  const int64_t k = it.k0 + lane;
  if (k > N) return;
  const int64_t nhi = min(it.n1, nend[k - 1]);
  const R r = r_true[k - 1];
  for (int r0 = 0; r0 < nrhs; r0 += G) {
    R acc[G];
#pragma unroll
    for (int g = 0; g < G; ++g) acc[g] = 0;
    for (int64_t n = it.n0; n <= nhi; ++n) {
      const R J = table_j(jtab, jt_n, deg, r * __ldg(&om_true[n - 1]));
#pragma unroll
      for (int g = 0; g < G; ++g)
        if (r0 + g < nrhs) acc[g] = fmar((R)__ldg(&c[(int64_t)(r0 + g) * ldc + n - 1]), J, acc[g]);
    }
#pragma unroll
    for (int g = 0; g < G; ++g) {
      if (r0 + g >= nrhs) break;
      if (it.slot < 0) f[(int64_t)(r0 + g) * ldf + k - 1] = acc[g];
      else partial[(it.slot + (int64_t)lane * it.ntile + it.t) * nrhs + r0 + g] = acc[g];
    }
  }
}

template <class R>
__global__ void k_near_combine(const NearRow* __restrict__ rows, int64_t nrows, const R* __restrict__ partial,
                               int nrhs, double* f, int64_t ldf) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nrows * nrhs) return;
  const int64_t i = t / nrhs;
  const int rr = (int)(t - i * nrhs);
  const NearRow row = rows[i];
  R s = 0;
  for (int j = 0; j < row.npieces; ++j) s += partial[(row.slot0 + j) * nrhs + rr];
  f[(int64_t)rr * ldf + row.k - 1] = (double)s;
}

}  // namespace

template <class R, class CT>
void launch_near_t(const NearItem* items, int64_t nitems, const int64_t* nend, int64_t N, R* partial, int nrhs,
                   const CT* c, int64_t ldc, double* f, int64_t ldf, const R* r, const R* om, const R* jtab,
                   int64_t jt_n, int deg, cudaStream_t st) {
  const int64_t threads = nitems * 32;
  const unsigned grid = (unsigned)((threads + 255) / 256);
  if (nrhs <= 1)
    k_near<R, 1><<<grid, 256, 0, st>>>(items, nitems, nend, N, partial, nrhs, c, ldc, f, ldf, r, om, jtab, jt_n, deg);
  else if (nrhs <= 2)
    k_near<R, 2><<<grid, 256, 0, st>>>(items, nitems, nend, N, partial, nrhs, c, ldc, f, ldf, r, om, jtab, jt_n, deg);
  else if (nrhs <= 4)
    k_near<R, 4><<<grid, 256, 0, st>>>(items, nitems, nend, N, partial, nrhs, c, ldc, f, ldf, r, om, jtab, jt_n, deg);
  else if (nrhs <= 8)
    k_near<R, 8><<<grid, 256, 0, st>>>(items, nitems, nend, N, partial, nrhs, c, ldc, f, ldf, r, om, jtab, jt_n, deg);
  else
    k_near<R, kMaxRhsGroup><<<grid, 256, 0, st>>>(items, nitems, nend, N, partial, nrhs, c, ldc, f, ldf, r, om, jtab,
                                                  jt_n, deg);
}

template <class R>
void launch_near(const NearItem* items, int64_t nitems, const NearRow* mrows, int64_t nmrows, const int64_t* nend,
                 int64_t N, R* partial, int nrhs, const double* c, int64_t ldc, const float* cf, double* f,
                 int64_t ldf, const R* r, const R* om, const R* jtab, int64_t jt_n, int deg, cudaStream_t st) {
  if (cf) launch_near_t<R, float>(items, nitems, nend, N, partial, nrhs, cf, N, f, ldf, r, om, jtab, jt_n, deg, st);
  else launch_near_t<R, double>(items, nitems, nend, N, partial, nrhs, c, ldc, f, ldf, r, om, jtab, jt_n, deg, st);
  if (nmrows > 0) {
    const int64_t n = nmrows * nrhs;
    k_near_combine<R><<<(unsigned)((n + 255) / 256), 256, 0, st>>>(mrows, nmrows, partial, nrhs, f, ldf);
  }
}

template void launch_near<double>(const NearItem*, int64_t, const NearRow*, int64_t, const int64_t*, int64_t,
                                  double*, int, const double*, int64_t, const float*, double*, int64_t,
                                  const double*, const double*, const double*, int64_t, int, cudaStream_t);
template void launch_near<float>(const NearItem*, int64_t, const NearRow*, int64_t, const int64_t*, int64_t, float*,
                                 int, const double*, int64_t, const float*, double*, int64_t, const float*,
                                 const float*, const float*, int64_t, int, cudaStream_t);

}  // namespace hk
