// Near field (the direct part J^EVAL of Eqs. 18-19 and the directly summed
// leading rows/columns of Sections 5-6): f_k = sum_{n <= nend(k)} c_n J_nu(r_k omega_n)
// with J evaluated per entry, over tiles of 32 rows x 512 columns of the near set.
//
// J_nu on [0, zmax] comes from a table of Taylor polynomials about the centres of
// intervals of width 1/kJTabSub (built at plan time from the Neumann addition formula,
// Eq. 8, with the degree set by eps), so one evaluation costs a table row load and deg
// Horner steps: FMAs in float for FP32 plans and in double-float for DF64 plans of few
// vectors; 64-bit integer steps on a Q62 copy of the table for FP64 plans and for every
// tensor-core near field (FP64 is the scarce pipe on this part).
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <type_traits>

#include "cplx.cuh"
#include "kernels.cuh"

namespace hk {

namespace {

// Right-hand sides handled per table evaluation: every entry's J is evaluated once per group
// of G vectors (G = 1, 2, 4, 8 or 16, the smallest that covers nrhs, groups of 16 beyond).
constexpr int kMaxRhsGroup = 16;

template <class R>
__device__ __forceinline__ R table_j(const R* __restrict__ jtab, int64_t jt_n, int deg, R z) {
  int i = (int)(z * (R)kJTabSub);
  i = i < 0 ? 0 : (i >= jt_n ? (int)jt_n - 1 : i);
  const R d = z - ((R)i + (R)0.5) * ((R)1 / (R)kJTabSub);
  const R* t = jtab + (int64_t)i * (deg + 1);
  R v = __ldg(&t[deg]);
  for (int j = deg - 1; j >= 0; --j) v = fmar(v, d, __ldg(&t[j]));
  return v;
}

// J_nu(z) from the Q62 table, in two parts. q62_interval finds the interval i = floor(z kJTabSub)
// and U = (z kJTabSub - i - 1/2) 2^64 from the bits of z (z >= 0) by integer operations; the
// caller runs Horner's rule in Q62 with the signed high halves of 64 x 64-bit products (each
// step truncating by less than 2^-62) and rounds (to J 2^53 for the digit split, to double
// otherwise). Every operation but z = r omega is
// on the integer pipe.
__device__ __forceinline__ long long q62_interval(int64_t jt_n, double z, long long& U) {
  const unsigned long long bits = (unsigned long long)__double_as_longlong(z);
  const int E = (int)(bits >> 52) & 0x7ff;
  const unsigned long long M = (bits & 0xfffffffffffffULL) | (E ? (1ULL << 52) : 0ULL);
  const int sh = 52 + 1023 - kJTabLog - E;  // mantissa bits below 1/kJTabSub
  long long i;
  unsigned long long F;  // the fraction z kJTabSub - i, times 2^64
  if (sh <= 0) {
    i = jt_n;
    F = 0;
  } else if (sh <= 52) {
    i = (long long)(M >> sh);
    F = M << (64 - sh);
  } else {
    i = 0;
    F = sh - 53 < 64 ? (M << 11) >> (sh - 53) : 0ULL;
  }
  if (i >= jt_n) {  // beyond the table (the near field stays below zmax < jt_n / kJTabSub)
    i = jt_n - 1;
    F = ~0ULL;
  }
  U = (long long)(F ^ (1ULL << 63));
  return i;
}

// J_nu(z) in FP64 from the Q62 table: Horner's rule on the integer pipe, one rounding to double.
__device__ __forceinline__ double q62_j(const long long* __restrict__ jq, int64_t jt_n, int deg, double z) {
  long long U;
  const long long* t = jq + q62_interval(jt_n, z, U) * (deg + 1);
  long long v = __ldg(&t[deg]);
  for (int j = deg - 1; j >= 0; --j) v = __mul64hi(v, U) + __ldg(&t[j]);
  return __ll2double_rn(v) * 0x1p-62;
}

// Warp per tile, lane per row: every lane walks the same columns n (so the loads of omega_n and
// of c_n for each vector are warp-wide broadcasts) and stops at its own prefix end; the sum
// over n is the lane's own, in increasing n, with no cross-lane reduction.
template <class R, int G, class CT>
__global__ void __launch_bounds__(256) k_near(const NearItem* __restrict__ items, int64_t nitems,
                                              const int64_t* __restrict__ nend, int64_t N, R* partial, int nrhs,
                                              const CT* __restrict__ c, int64_t ldc, double* f, int64_t ldf,
                                              const R* __restrict__ r_true, const R* __restrict__ om_true,
                                              const R* __restrict__ jtab, const long long* __restrict__ jq,
                                              int64_t jt_n, int deg, const int* __restrict__ cexp) {
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
      R J;
      if constexpr (std::is_same<R, double>::value) J = q62_j(jq, jt_n, deg, r * __ldg(&om_true[n - 1]));
      else J = table_j(jtab, jt_n, deg, r * __ldg(&om_true[n - 1]));
#pragma unroll
      for (int g = 0; g < G; ++g)
        if (r0 + g < nrhs) acc[g] = fmar((R)__ldg(&c[(int64_t)(r0 + g) * ldc + n - 1]), J, acc[g]);
    }
#pragma unroll
    for (int g = 0; g < G; ++g) {
      if (r0 + g >= nrhs) break;
      // scaled coefficients (cexp): f gets the sum times 2^e; partial sums stay in the scaled
      // range of R and the combine applies 2^e
      if (it.slot < 0) f[(int64_t)(r0 + g) * ldf + k - 1] = cexp ? ldexp((double)acc[g], cexp[r0 + g]) : (double)acc[g];
      else partial[(it.slot + (int64_t)lane * it.ntile) * nrhs + (int64_t)(r0 + g) * it.ntile + it.t] = acc[g];
    }
  }
}

// Double-float near field (DF64 plans, 1e-11 <= eps < 1e-5). r_k, omega_n, the table and the
// coefficients are (h, l) pairs of floats (about 48 significant bits), and every step runs on
// the FP32 pipe:
//  * z = r_k omega_n as an unnormalised pair (the exact product of the high parts plus the
//    cross terms);
//  * the interval from z.h, and d = z - centre with the rounding of z.h - centre kept (two-sum);
//  * Taylor steps of degree >= 4 in float (their terms are below 16^-4 / 4! of the total, so
//    float rounding there stays under 1e-13), the last four steps in double-float;
//  * per vector, the exact product J.h c.h (FMA) and the cross terms, summed into a float sum
//    whose every rounding error is kept in a second float (two-sum), renormalised every 16
//    columns.
__device__ __forceinline__ df64 table_j_df(const float2* __restrict__ jtab, int64_t jt_n, int deg, float zh,
                                           float zl) {
  int64_t i = (int64_t)(zh * (float)kJTabSub);
  i = i < 0 ? 0 : (i >= jt_n ? jt_n - 1 : i);
  const float ctr = ((float)i + 0.5f) * (1.0f / (float)kJTabSub);
  const float s = zh - ctr;
  const float bb = s - zh;
  const float err = (zh - (s - bb)) + (-ctr - bb);
  const df64 d = fast_two_sum(s, err + zl);
  const float2* t = jtab + i * (deg + 1);
  float v = __ldg(&t[deg]).x;
  int j = deg - 1;
  for (; j >= 4; --j) v = fmaf(v, d.h, __ldg(&t[j]).x);
  df64 w(v, 0.0f);
  if (deg < 4) {
    const float2 a = __ldg(&t[deg]);
    w = df64(a.x, a.y);
    j = deg - 1;
  }
  for (; j >= 0; --j) {
    const float2 a = __ldg(&t[j]);
    w = fmar(w, d, df64(a.x, a.y));
  }
  return w;
}

template <int G>
__global__ void __launch_bounds__(256) k_near_df(const NearItem* __restrict__ items, int64_t nitems,
                                                 const int64_t* __restrict__ nend, int64_t N, double* partial,
                                                 int nrhs, const float2* __restrict__ cd, double* f, int64_t ldf,
                                                 const float2* __restrict__ r_true, const float2* __restrict__ om_true,
                                                 const float2* __restrict__ jtab, int64_t jt_n, int deg,
                                                 const int* __restrict__ cexp) {
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (warp >= nitems) return;
  const NearItem it = items[warp];
  const int64_t k = it.k0 + lane;
  if (k > N) return;
  const int64_t nhi = min(it.n1, nend[k - 1]);
  const float2 r = r_true[k - 1];
  for (int r0 = 0; r0 < nrhs; r0 += G) {
    float hi[G], lo[G];
#pragma unroll
    for (int g = 0; g < G; ++g) hi[g] = lo[g] = 0.0f;
    for (int64_t n = it.n0; n <= nhi; ++n) {
      const float2 om = __ldg(&om_true[n - 1]);
      const float zh = r.x * om.x;
      float zl = fmaf(r.x, om.x, -zh);
      zl = fmaf(r.x, om.y, zl);
      zl = fmaf(r.y, om.x, zl);
      const df64 J = table_j_df(jtab, jt_n, deg, zh, zl);
#pragma unroll
      for (int g = 0; g < G; ++g) {
        if (r0 + g < nrhs) {
          const float2 cv = __ldg(&cd[(int64_t)(r0 + g) * N + n - 1]);
          const float p = J.h * cv.x;
          float e = fmaf(J.h, cv.x, -p);
          e = fmaf(J.h, cv.y, e);
          e = fmaf(J.l, cv.x, e);
          const float s = hi[g] + p;
          const float bb = s - hi[g];
          lo[g] += ((hi[g] - (s - bb)) + (p - bb)) + e;
          hi[g] = s;
        }
      }
      if (((n - it.n0) & 15) == 15) {
#pragma unroll
        for (int g = 0; g < G; ++g) {
          const df64 q = fast_two_sum(hi[g], lo[g]);
          hi[g] = q.h;
          lo[g] = q.l;
        }
      }
    }
#pragma unroll
    for (int g = 0; g < G; ++g) {
      if (r0 + g >= nrhs) break;
      const double v = ldexp((double)hi[g] + (double)lo[g], cexp[r0 + g]);  // back from the scaled coefficients
      if (it.slot < 0) f[(int64_t)(r0 + g) * ldf + k - 1] = v;
      else partial[(it.slot + (int64_t)lane * it.ntile) * nrhs + (int64_t)(r0 + g) * it.ntile + it.t] = v;
    }
  }
}

// Rows whose prefix spans several tiles: the partial sums of row k and vector rr are the
// npieces consecutive values at slot0 nrhs + rr npieces. A warp per row. Rows of up to 32
// pieces take 16 vectors at a time: lane l adds, in order, the pieces l >> 4, (l >> 4) + 2, ...
// of vector l & 15 and one shuffle adds the two halves. Longer rows (the first rows, up to
// N / 512 pieces) take one vector at a time: lane l adds the pieces l, l + 32, ... and the lanes
// combine in a fixed shuffle tree, which keeps the rounding of these long sums at that of
// 64-term sums. Either way the result does not depend on scheduling.
// FP64 near field with the per-vector products on the tensor cores (FP64 plans, 8 to 16 vectors):
// split-digit products (the Ozaki scheme). J (|J| <= 1) and, per 512-column chunk and vector,
// the coefficients scaled by 2^-e (2^e bounds the chunk's largest |c|) are rounded to the
// integers J 2^53 and C 2^54 (below 2^54 in size) and written as 8 balanced base-128 digits in
// [-64, 63], exact in fp16. The digit products of one diagonal D = i + j carry the weight
// 2^(-9 - 7D); fp16 MMAs
// with fp32 accumulation add them up: each product is an integer of at most 2^12 and a
// diagonal of a 512-column tile sums at most 8 x 512 of them, so every partial sum is an
// integer of at most 2^24 and exact (checked on this GPU: the first rounding appears past
// 2^24). Diagonals D <= 8 are kept (the others add at most 2^-57 of the chunk's scale per entry);
// they are combined in FP64 once per tile. The rounding of J and C to the digit grid is 2^-54
// and 2^-55 of their scales: the products are as accurate as FP64 ones, and the sums exact.
constexpr int kTcDig = 8, kTcDiag = 9, kTcChunk = 512;

// The balanced digits of X (|X| <= 2^54) are the base-128 digits of X + kDigOff, less 64
// (kDigOff has every digit 64). Digit i (weight 128^(7 - i)) of two values Yl, Yh = X + kDigOff,
// as an fp16 pair: the bits 0x6400 + e are the fp16 value 1024 + e for 0 <= e < 1024, so one
// packed subtraction of 1088 leaves the digits e - 64, exactly.
constexpr unsigned long long kDigOff = 0x0081020408102040ULL;

template <int I>
__device__ __forceinline__ unsigned digit_pair(unsigned long long Yl, unsigned long long Yh) {
  constexpr int s = 7 * (kTcDig - 1 - I);
  const unsigned el = (unsigned)(Yl >> s) & 127u, eh = (unsigned)(Yh >> s) & 127u;
  const unsigned w = 0x64006400u | el | (eh << 16);
  const __half2 off = __half2(__float2half(1088.0f), __float2half(1088.0f));
  const __half2 v = __hsub2(*reinterpret_cast<const __half2*>(&w), off);
  return *reinterpret_cast<const unsigned*>(&v);
}

__device__ __forceinline__ void mma_f16(float (&d)[4], const unsigned (&a)[4], unsigned b0, unsigned b1) {
  asm(
      "mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// Coefficient digits: one CTA of kTcChunk threads per chunk t; Ce[t * 16 + g] = e and
// Cd[(j * 16 + g) * Npad + n - 1] = digit j of round(c_n^g 2^-e 2^54) (zeros for g >= nrhs and
// n > N), 2^e the smallest power of two above the chunk's largest |c_n^g| (2^-1021 at least).
// Integer operations throughout: the maximum of |c| is the maximum of its bit patterns, e
// comes from the exponent field, and c 2^(54 - e) (below 2^54) from the mantissa shifted right
// with rounding to nearest (ties up).
__global__ void __launch_bounds__(kTcChunk) k_near_cdigits(const double* __restrict__ c, int64_t ldc, int nrhs,
                                                          int64_t N, int64_t Npad, __half* Cd, int* Ce) {
  const int64_t t = blockIdx.x;
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const int64_t n = t * kTcChunk + tid;  // 0-based column
  __shared__ long long wmax[kTcChunk / 32][16];
  __shared__ int sexp[16];
  long long b[16];
#pragma unroll
  for (int g = 0; g < 16; ++g) {
    b[g] = (g < nrhs && n < N) ? __double_as_longlong(c[(int64_t)g * ldc + n]) : 0LL;
    long long m = b[g] & 0x7fffffffffffffffLL;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = max(m, (long long)__shfl_xor_sync(0xffffffffu, m, o));
    if (lane == 0) wmax[w][g] = m;
  }
  __syncthreads();
  if (tid < 16) {
    long long m = 0;
    for (int j = 0; j < kTcChunk / 32; ++j) m = max(m, wmax[j][tid]);
    const int ef = max((int)(m >> 52), 1);      // |c| < 2^(ef - 1022)
    const int e = m > 0 ? ef - 1022 : 0;
    sexp[tid] = e;
    Ce[t * 16 + tid] = e;
  }
  __syncthreads();
#pragma unroll
  for (int g = 0; g < 16; ++g) {
    const int ef = (int)((b[g] >> 52) & 0x7ff);
    const long long M = (b[g] & 0xfffffffffffffLL) | (ef ? (1LL << 52) : 0LL);
    // c = M 2^(max(ef, 1) - 1075), so c 2^(54 - e) = M 2^-s with s = 1021 + e - max(ef, 1) >= -1
    const int sft = 1021 + sexp[g] - max(ef, 1);
    long long X = sft < 0 ? M << 1 : (sft == 0 ? M : (sft < 63 ? (M + (1LL << (sft - 1))) >> sft : 0LL));
    if (b[g] < 0) X = -X;
    const unsigned long long Y = (unsigned long long)X + kDigOff;
#pragma unroll
    for (int j = 0; j < kTcDig; ++j)
      Cd[((int64_t)j * 16 + g) * Npad + n] = __int2half_rn((int)((Y >> (7 * (kTcDig - 1 - j))) & 127u) - 64);
  }
}

// The A fragment of J digit i (register r: entries 2r, 2r + 1) and its products with the
// coefficient digits j < ND with diagonal D = i + j < NG.
template <int I, int ND, int NG>
__device__ __forceinline__ void tc_digit(float (&acc)[NG][2][4], const unsigned long long (&Y)[8],
                                         const unsigned (&b)[ND][2][2]) {
  const unsigned a[4] = {digit_pair<I>(Y[0], Y[1]), digit_pair<I>(Y[2], Y[3]), digit_pair<I>(Y[4], Y[5]),
                         digit_pair<I>(Y[6], Y[7])};
#pragma unroll
  for (int j = 0; j < ND && I + j < NG; ++j)
#pragma unroll
    for (int u = 0; u < 2; ++u) mma_f16(acc[I + j][u], a, b[j][u][0], b[j][u][1]);
}

// A CTA of two warps per near-field tile (NearItem); warp w takes rows k0 + 16w .. k0 + 16w + 15
// and all 16 vector slots, as two m16n8 output tiles. Thread (gq, tq) of a warp evaluates J at
// rows gq, gq + 8 and columns 2tq, 2tq + 1, 2tq + 8, 2tq + 9 of each 16-column step (its A
// fragment) and loads the coefficient digits of columns 2tq, 2tq + 1, 2tq + 8, 2tq + 9 for
// vectors gq and gq + 8 (its B fragments). J comes from the fixed-point table (FP64 and
// double-float plans alike: it is exact to the digit grid either way).
// ND, NG: digits of J and c used (the leading ND of the 8) and diagonals kept. FP64 plans take
// 8 and 9 (86 MMAs per 16-column step, products as accurate as FP64 ones); DF64 plans take 7
// and 7 (56 MMAs): dropping the last digit of each and the diagonals D >= 7 costs at most about
// 2^-46 of the chunk's scale per entry, the accuracy of double-float products.
template <int ND, int NG>
__global__ void __launch_bounds__(64, 7) k_near_tc(const NearItem* __restrict__ items, const int64_t* __restrict__ nend,
                                               int64_t N, double* partial, int nrhs, const __half* __restrict__ Cd,
                                               const int* __restrict__ Ce, int64_t Npad, double* f, int64_t ldf,
                                               const double* __restrict__ r_true, const double* __restrict__ om_true,
                                               const long long* __restrict__ jq, int64_t jt_n, int deg) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, gq = lane >> 2, tq = lane & 3;
  const NearItem it = items[blockIdx.x];
  const int64_t kb = it.k0 + 16 * warp;
  int64_t rend[2];
  double rr[2];
#pragma unroll
  for (int q = 0; q < 2; ++q) {
    const int64_t k = kb + gq + 8 * q;
    rend[q] = k <= N ? min(it.n1, nend[k - 1]) : 0;
    rr[q] = k <= N ? r_true[k - 1] : 0.0;
  }
  int64_t wend = max(rend[0], rend[1]);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) wend = max(wend, (int64_t)__shfl_xor_sync(0xffffffffu, (long long)wend, o));
  float acc[NG][2][4];
#pragma unroll
  for (int D = 0; D < NG; ++D)
#pragma unroll
    for (int u = 0; u < 2; ++u)
#pragma unroll
      for (int q = 0; q < 4; ++q) acc[D][u][q] = 0.0f;
  const unsigned* Cw = reinterpret_cast<const unsigned*>(Cd);  // pairs of digits (columns 2m, 2m+1)
  for (int64_t n0 = it.n0; n0 <= wend; n0 += 16) {
    // A: 8 entries e = 2r + h, register r = (row q = r & 1) x (column block r >> 1), half
    // h = column 2tq + h; their Horner chains advance together (8 independent chains a thread)
    const long long* tp[8];
    long long U[8], v[8];
    bool on[8];
#pragma unroll
    for (int e = 0; e < 8; ++e) {
      const int r = e >> 1, h = e & 1, q = r & 1;
      const int64_t col = n0 + 2 * tq + h + ((r >> 1) ? 8 : 0);
      on[e] = col <= rend[q];
      const double z = on[e] ? rr[q] * __ldg(&om_true[col - 1]) : 0.0;
      tp[e] = jq + q62_interval(jt_n, z, U[e]) * (deg + 1);
      v[e] = __ldg(&tp[e][deg]);
    }
    for (int j = deg - 1; j >= 0; --j)
#pragma unroll
      for (int e = 0; e < 8; ++e) v[e] = __mul64hi(v[e], U[e]) + __ldg(&tp[e][j]);
    unsigned long long Y[8];  // J 2^53 (0 outside the row's prefix) + kDigOff
#pragma unroll
    for (int e = 0; e < 8; ++e) Y[e] = (unsigned long long)(on[e] ? (v[e] + 256) >> 9 : 0LL) + kDigOff;
    // B: digit j, vector tile u: columns (n0 + 2tq, +1) and (n0 + 2tq + 8, +9) of vector 8u + gq
    unsigned b[ND][2][2];
    const int64_t c0 = (n0 - 1 + 2 * tq) >> 1;  // index of the digit pair
#pragma unroll
    for (int j = 0; j < ND; ++j)
#pragma unroll
      for (int u = 0; u < 2; ++u) {
        const int64_t row = ((int64_t)j * 16 + 8 * u + gq) * (Npad >> 1);
        b[j][u][0] = __ldg(&Cw[row + c0]);
        b[j][u][1] = __ldg(&Cw[row + c0 + 4]);
      }
    // digit i of J against digits j <= 8 - i of the coefficients: consecutive products go to
    // different diagonals, so they do not wait on one another
    tc_digit<0, ND, NG>(acc, Y, b);
    tc_digit<1, ND, NG>(acc, Y, b);
    tc_digit<2, ND, NG>(acc, Y, b);
    tc_digit<3, ND, NG>(acc, Y, b);
    tc_digit<4, ND, NG>(acc, Y, b);
    tc_digit<5, ND, NG>(acc, Y, b);
    tc_digit<6, ND, NG>(acc, Y, b);
    if constexpr (ND > 7) tc_digit<7, ND, NG>(acc, Y, b);
  }
  // combine the diagonals in FP64 and write: output (row gq + 8 (q >> 1), vector 8u + 2tq + (q & 1))
  const int64_t t = (it.n0 - 1) / kTcChunk;
#pragma unroll
  for (int u = 0; u < 2; ++u)
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int g = 8 * u + 2 * tq + (q & 1);
      const int rowoff = 16 * warp + gq + 8 * (q >> 1);
      const int64_t k = it.k0 + rowoff;
      double v = 0.0;
#pragma unroll
      for (int D = NG - 1; D >= 0; --D) v = fma(v, 1.0 / 128.0, (double)acc[D][u][q]);
      v = ldexp(v, Ce[t * 16 + g] - 9);
      if (k > N || g >= nrhs) continue;
      if (it.slot < 0) f[(int64_t)g * ldf + k - 1] = v;
      else partial[(it.slot + (int64_t)rowoff * it.ntile) * nrhs + (int64_t)g * it.ntile + it.t] = v;
    }
}

// cexp (FP32 near fields of scaled coefficients): the partial sums of vector rr are in units of
// 2^cexp[rr], applied to the row's total.
template <class R>
__global__ void k_near_combine(const NearRow* __restrict__ rows, int64_t nrows, const R* __restrict__ partial,
                               int nrhs, double* f, int64_t ldf, const int* __restrict__ cexp) {
  const int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31, g = lane & 15, h = lane >> 4;
  if (w >= nrows) return;
  const NearRow row = rows[w];
  if (row.npieces > 32) {
    for (int rr = 0; rr < nrhs; ++rr) {
      const R* p = partial + row.slot0 * nrhs + (int64_t)rr * row.npieces;
      R s = 0;
      for (int j = lane; j < row.npieces; j += 32) s += p[j];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
      if (lane == 0) f[(int64_t)rr * ldf + row.k - 1] = cexp ? ldexp((double)s, cexp[rr]) : (double)s;
    }
    return;
  }
  for (int r0 = 0; r0 < nrhs; r0 += 16) {
    const int rr = r0 + g;
    R s = 0;
    if (rr < nrhs) {
      const R* p = partial + row.slot0 * nrhs + (int64_t)rr * row.npieces;
      for (int j = h; j < row.npieces; j += 2) s += p[j];
    }
    s += __shfl_down_sync(0xffffffffu, s, 16);
    if (h == 0 && rr < nrhs) f[(int64_t)rr * ldf + row.k - 1] = cexp ? ldexp((double)s, cexp[rr]) : (double)s;
  }
}

}  // namespace

template <class R, class CT>
void launch_near_t(const NearItem* items, int64_t nitems, const int64_t* nend, int64_t N, R* partial, int nrhs,
                   const CT* c, int64_t ldc, double* f, int64_t ldf, const R* r, const R* om, const R* jtab,
                   const long long* jq, int64_t jt_n, int deg, const int* cexp, cudaStream_t st) {
  const int64_t threads = nitems * 32;
  const unsigned grid = (unsigned)((threads + 255) / 256);
  if (nrhs <= 1)
    k_near<R, 1><<<grid, 256, 0, st>>>(items, nitems, nend, N, partial, nrhs, c, ldc, f, ldf, r, om, jtab, jq, jt_n,
                                        deg, cexp);
  else if (nrhs <= 2)
    k_near<R, 2><<<grid, 256, 0, st>>>(items, nitems, nend, N, partial, nrhs, c, ldc, f, ldf, r, om, jtab, jq, jt_n,
                                        deg, cexp);
  else if (nrhs <= 4)
    k_near<R, 4><<<grid, 256, 0, st>>>(items, nitems, nend, N, partial, nrhs, c, ldc, f, ldf, r, om, jtab, jq, jt_n,
                                        deg, cexp);
  else if (nrhs <= 8)
    k_near<R, 8><<<grid, 256, 0, st>>>(items, nitems, nend, N, partial, nrhs, c, ldc, f, ldf, r, om, jtab, jq, jt_n,
                                        deg, cexp);
  else
    k_near<R, kMaxRhsGroup><<<grid, 256, 0, st>>>(items, nitems, nend, N, partial, nrhs, c, ldc, f, ldf, r, om, jtab,
                                                  jq, jt_n, deg, cexp);
}

template <class R>
void launch_near(const NearItem* items, int64_t nitems, const NearRow* mrows, int64_t nmrows, const int64_t* nend,
                 int64_t N, R* partial, int nrhs, const double* c, int64_t ldc, const float* cf, double* f,
                 int64_t ldf, const R* r, const R* om, const R* jtab, const long long* jtabq, int64_t jt_n, int deg,
                 const int* cexp, cudaStream_t st) {
  if (cf)
    launch_near_t<R, float>(items, nitems, nend, N, partial, nrhs, cf, N, f, ldf, r, om, jtab, jtabq, jt_n, deg, cexp,
                            st);
  else
    launch_near_t<R, double>(items, nitems, nend, N, partial, nrhs, c, ldc, f, ldf, r, om, jtab, jtabq, jt_n, deg,
                             nullptr, st);
  if (nmrows > 0)
    k_near_combine<R><<<(unsigned)((nmrows * 32 + 255) / 256), 256, 0, st>>>(mrows, nmrows, partial, nrhs, f, ldf,
                                                                           cf ? cexp : nullptr);
}

void launch_near_df(const NearItem* items, int64_t nitems, const NearRow* mrows, int64_t nmrows,
                    const int64_t* nend, int64_t N, double* partial, int nrhs, const float2* cd, double* f,
                    int64_t ldf, const float2* r, const float2* om, const float2* jtab, int64_t jt_n, int deg,
                    const int* cexp, cudaStream_t st) {
  const int64_t threads = nitems * 32;
  const unsigned grid = (unsigned)((threads + 255) / 256);
  if (nrhs <= 1)
    k_near_df<1><<<grid, 256, 0, st>>>(items, nitems, nend, N, partial, nrhs, cd, f, ldf, r, om, jtab, jt_n, deg, cexp);
  else if (nrhs <= 2)
    k_near_df<2><<<grid, 256, 0, st>>>(items, nitems, nend, N, partial, nrhs, cd, f, ldf, r, om, jtab, jt_n, deg, cexp);
  else if (nrhs <= 4)
    k_near_df<4><<<grid, 256, 0, st>>>(items, nitems, nend, N, partial, nrhs, cd, f, ldf, r, om, jtab, jt_n, deg, cexp);
  else if (nrhs <= 8)
    k_near_df<8><<<grid, 256, 0, st>>>(items, nitems, nend, N, partial, nrhs, cd, f, ldf, r, om, jtab, jt_n, deg, cexp);
  else
    k_near_df<kMaxRhsGroup><<<grid, 256, 0, st>>>(items, nitems, nend, N, partial, nrhs, cd, f, ldf, r, om, jtab,
                                                  jt_n, deg, cexp);
  if (nmrows > 0)
    k_near_combine<double><<<(unsigned)((nmrows * 32 + 255) / 256), 256, 0, st>>>(mrows, nmrows, partial, nrhs, f,
                                                                                ldf, nullptr);
}

void launch_near_tc(bool df, const NearItem* items, int64_t nitems, const NearRow* mrows, int64_t nmrows,
                    const int64_t* nend, int64_t N, double* partial, int nrhs, const double* c, int64_t ldc, void* Cdv,
                    int* Ce, int64_t Npad, double* f, int64_t ldf, const double* r, const double* om,
                    const long long* jtabq, int64_t jt_n, int deg, cudaStream_t st) {
  __half* Cd = reinterpret_cast<__half*>(Cdv);
  k_near_cdigits<<<(unsigned)(Npad / kTcChunk), kTcChunk, 0, st>>>(c, ldc, nrhs, N, Npad, Cd, Ce);
  if (df)
    k_near_tc<7, 7><<<(unsigned)nitems, 64, 0, st>>>(items, nend, N, partial, nrhs, Cd, Ce, Npad, f, ldf, r, om, jtabq,
                                                     jt_n, deg);
  else
    k_near_tc<kTcDig, kTcDiag><<<(unsigned)nitems, 64, 0, st>>>(items, nend, N, partial, nrhs, Cd, Ce, Npad, f, ldf,
                                                                r, om, jtabq, jt_n, deg);
  if (nmrows > 0)
    k_near_combine<double><<<(unsigned)((nmrows * 32 + 255) / 256), 256, 0, st>>>(mrows, nmrows, partial, nrhs, f,
                                                                                ldf, nullptr);
}

template void launch_near<double>(const NearItem*, int64_t, const NearRow*, int64_t, const int64_t*, int64_t,
                                  double*, int, const double*, int64_t, const float*, double*, int64_t,
                                  const double*, const double*, const double*, const long long*, int64_t, int,
                                  const int*, cudaStream_t);
template void launch_near<float>(const NearItem*, int64_t, const NearRow*, int64_t, const int64_t*, int64_t, float*,
                                 int, const double*, int64_t, const float*, double*, int64_t, const float*,
                                 const float*, const float*, const long long*, int64_t, int, const int*,
                                 cudaStream_t);

}  // namespace hk
