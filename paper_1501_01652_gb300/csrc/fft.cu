// Multi-column power-of-two FFT (Stockham autosort, decimation in time) in FP64
// (double2) or FP32 (float2), and the chirp-z helpers of the far field.
//
// Transforms of F <= 4096 points run whole in one launch (k_fft_small). Longer ones take
// passes of radix 32..256 (k_fft_pass_reg); after passes with radices R_1 R_2 ... = F the
// output is in natural order. One CTA handles kTile consecutive (p, q) pairs of a pass, so
// every global load and store touches kTile or more consecutive elements, and does the
// R-point DFTs in two register sub-stages with one exchange through shared memory.
#include <cuda_runtime.h>

#include <algorithm>
#include <type_traits>

#include "cplx.cuh"
#include "kernels.cuh"

namespace hk {

namespace {

constexpr int kTile = 16;
constexpr int kRow = kTile + 1;  // padded shared-memory row (elements)
constexpr int kFftThreads = 256;

template <bool INV, class C>
__device__ __forceinline__ C twiddle(const C* __restrict__ tw, uint32_t idx) {
  C t = ldgc(&tw[idx]);
  if (INV) t.y = -t.y;
  return t;
}

// Radix-2 decimation-in-time butterfly on (a0, a1 w): y0 = a0 + w a1, y1 = 2 a0 - y0.
template <class C>
__device__ __forceinline__ void bfly2(C& a0, C& a1, C w) {
  typedef typename RealOf<C>::type R;
  C y0;
  y0.x = fmar(w.x, a1.x, fmar(-w.y, a1.y, a0.x));
  y0.y = fmar(w.x, a1.y, fmar(w.y, a1.x, a0.y));
  a1 = mkc(fmar((R)2, a0.x, -y0.x), fmar((R)2, a0.y, -y0.y));
  a0 = y0;
}

// Fused column generation (FftGen): where column y of the chunk takes its points from.
template <class C>
struct GenCol {
  const C* v;   // the column's table row, from its segment's first point
  int64_t cb;   // index of the segment's first coefficient
  int64_t lim;  // points that carry data
};
template <class C>
__device__ __forceinline__ GenCol<C> gen_col(const FftGen& g, uint64_t y) {
  // chunk columns and stacked-column indices stay below 2^31
  const uint32_t cc = (uint32_t)y / (uint32_t)g.nsegc;
  const int64_t sg = (int64_t)y - (int64_t)cc * g.nsegc;
  const uint32_t gi = (uint32_t)(g.c0 + cc);
  const uint32_t rhs = gi / (uint32_t)g.ncols, li = gi - rhs * (uint32_t)g.ncols;
  const int64_t nlo = sg * g.S;
  GenCol<C> r;
  r.v = reinterpret_cast<const C*>(g.Vt) + (int64_t)li * g.C + nlo;
  r.cb = (int64_t)rhs * g.ldc + g.n0 - 1 + nlo;
  r.lim = min(g.S, g.C - nlo);
  return r;
}
// coefficient i (in the plan's coefficient format) times the table value v
__device__ __forceinline__ double2 coef_times(const void* p, int64_t i, double2 v) {
  const double c = __ldg(reinterpret_cast<const double*>(p) + i);
  return make_double2(c * v.x, c * v.y);
}
__device__ __forceinline__ float2 coef_times(const void* p, int64_t i, float2 v) {
  const float c = __ldg(reinterpret_cast<const float*>(p) + i);
  return make_float2(c * v.x, c * v.y);
}
__device__ __forceinline__ df64c coef_times(const void* p, int64_t i, df64c v) {
  const float2 q = __ldg(reinterpret_cast<const float2*>(p) + i);
  const df64 c(q.x, q.y);
  return mkc(c * v.x, c * v.y);
}

// The double-float butterfly: t = w a1 once, with the exact products of the high parts (FMA),
// their difference by two-sum and the cross terms added into the low part, left unnormalised
// (|low| << |high|); then y0 = a0 + t and y1 = a0 - t, each a two-sum of the high parts with
// the low parts added. About 64 FP32 operations against 90 for the FMA-folded form with
// double-float fmar.
__device__ __forceinline__ df64 df_add_pair(df64 a, float sh, float sl) {
  const float u = a.h + sh;
  const float bb = u - a.h;
  float v = (a.h - (u - bb)) + (sh - bb);
  v += a.l + sl;
  // left unnormalised: |v| stays within a few units in the last place of u, and every later
  // operation takes the high parts through a two-sum or an exact product again
  return df64(u, v);
}
// x0 y0 - x1 y1 (sign = -1) or x0 y0 + x1 y1 (sign = +1) as an unnormalised pair (h, l)
__device__ __forceinline__ void df_dot2(df64 x0, df64 y0, df64 x1, df64 y1, float sign, float& h, float& l) {
  const float p = x0.h * y0.h, q = sign * (x1.h * y1.h);
  const float ep = fmaf(x0.h, y0.h, -p), eq = sign * fmaf(x1.h, y1.h, -sign * q);
  h = p + q;
  const float bb = h - p;
  l = ((p - (h - bb)) + (q - bb)) + (ep + eq);
  l = fmaf(x0.h, y0.l, l);
  l = fmaf(x0.l, y0.h, l);
  l = fmaf(sign * x1.h, y1.l, l);
  l = fmaf(sign * x1.l, y1.h, l);
}
template <>
__device__ __forceinline__ void bfly2<df64c>(df64c& a0, df64c& a1, df64c w) {
  float tx, lx, ty, ly;
  df_dot2(w.x, a1.x, w.y, a1.y, -1.0f, tx, lx);
  df_dot2(w.x, a1.y, w.y, a1.x, 1.0f, ty, ly);
  const df64c y0 = mkc(df_add_pair(a0.x, tx, lx), df_add_pair(a0.y, ty, ly));
  a1 = mkc(df_add_pair(a0.x, -tx, -lx), df_add_pair(a0.y, -ty, -ly));
  a0 = y0;
}

// Twiddle deferral. A pass of radix R multiplies input e of the R-point DFT of sequence
// (p, q) by the pass twiddle W_F^{pt e} (pt = p s). The pass twiddle is never applied on its
// own: in a Stockham sub-stage of stride s_k, the inputs e = qq + s_k (Q pp + j) of a butterfly
// carry W_F^{pt (qq + s_k j)}; the common factor W_F^{pt qq} moves to the butterfly's outputs
// (whose index is qq mod s_k again), and W_F^{pt s_k j} joins the sub-stage's own twiddle
// W_{n_k}^{pp j} in one table lookup. At the last sub-stage s_k = 1, so nothing is left over.
// Every index fits in 32 bits (F <= 2^24).

// Twiddled radix-2^LQ DFT in registers: on return a[r] = sum_j W_Q^{r j} w^j a_j (Q = 2^LQ),
// where w^t is the table entry (t * base) mod Fmax. Iterative radix-2 decimation in time on the
// bit-reversed inputs (a compile-time renaming of registers): the size-m sub-DFTs of stage
// s = log2 m combine as E_k + W_m^k w^{Q/m} O_k, so stage s looks up m/2 twiddles at
// k Fmax/m + base Q/m, and every butterfly is the FMA-folded bfly2.
// bit reversal of j in L <= 4 bits
__host__ __device__ constexpr int bitrev(int j, int L) {
  return (((j & 1) << 3) | ((j & 2) << 1) | ((j & 4) >> 1) | ((j & 8) >> 3)) >> (4 - L);
}

template <int LQ, bool INV, class C>
__device__ __forceinline__ void reg_dft(C (&a)[1 << LQ], uint32_t base, const C* __restrict__ tw, int logFmax,
                                        uint32_t fmask) {
  constexpr int Q = 1 << LQ;
  C b[Q];
#pragma unroll
  for (int j = 0; j < Q; ++j) b[bitrev(j, LQ)] = a[j];
#pragma unroll
  for (int s = 1; s <= LQ; ++s) {
    const int half = 1 << (s - 1);
#pragma unroll
    for (int k = 0; k < half; ++k) {
      const C v = twiddle<INV>(tw, (((uint32_t)k << (logFmax - s)) + (base << (LQ - s))) & fmask);
#pragma unroll
      for (int g = 0; g < Q; g += 2 * half) bfly2(b[g + k], b[g + k + half], v);
    }
  }
#pragma unroll
  for (int j = 0; j < Q; ++j) a[j] = b[j];
}

// reg_dft for base = 0 (the first sub-stage of the first pass of a transform): the twiddles
// are the constants W_{2^s}^k. Those equal to 1 and -i (i for the inverse) become plain
// additions; the others are folded into FMAs as in bfly2.
// cos and sin of 2 pi t / 16, t = 0..7
__host__ __device__ constexpr double cos16(int t) {
  return t == 0 ? 1.0 : t == 1 ? 0.92387953251128675613 : t == 2 ? 0.7071067811865475244
       : t == 3 ? 0.38268343236508977173 : t == 4 ? 0.0 : t == 5 ? -0.38268343236508977173
       : t == 6 ? -0.7071067811865475244 : -0.92387953251128675613;
}
__host__ __device__ constexpr double sin16(int t) { return cos16(t < 4 ? 4 - t : t - 4); }

template <int LQ, bool INV, class C>
__device__ __forceinline__ void reg_dft_unit(C (&a)[1 << LQ]) {
  typedef typename RealOf<C>::type R;
  constexpr int Q = 1 << LQ;
  C b[Q];
#pragma unroll
  for (int j = 0; j < Q; ++j) b[bitrev(j, LQ)] = a[j];
#pragma unroll
  for (int s = 1; s <= LQ; ++s) {
    const int half = 1 << (s - 1);
#pragma unroll
    for (int k = 0; k < half; ++k) {
      const int t16 = k << (4 - s);  // W_{2^s}^k = exp(-2 pi i t16 / 16)
#pragma unroll
      for (int g = 0; g < Q; g += 2 * half) {
        C& x0 = b[g + k];
        C& x1 = b[g + k + half];
        if (t16 == 0) {
          const C y0 = mkc(x0.x + x1.x, x0.y + x1.y);
          x1 = mkc(x0.x - x1.x, x0.y - x1.y);
          x0 = y0;
        } else if (t16 == 4) {
          // w x1 = -i x1 (forward) or i x1 (inverse)
          const C wx = INV ? mkc(-x1.y, x1.x) : mkc(x1.y, -x1.x);
          const C y0 = mkc(x0.x + wx.x, x0.y + wx.y);
          x1 = mkc(x0.x - wx.x, x0.y - wx.y);
          x0 = y0;
        } else {
          const C w = mkc((R)cos16(t16), INV ? (R)sin16(t16) : -(R)sin16(t16));
          bfly2(x0, x1, w);
        }
      }
    }
  }
#pragma unroll
  for (int j = 0; j < Q; ++j) a[j] = b[j];
}

// The same pass as k_fft_pass for 5 <= log2 R <= 8, with the R-point DFTs done as two
// Stockham sub-stages of radix Q1 = 2^L1 and Q2 = 2^L2 (L1 + L2 = log2 R) held in registers.
// Sub-stage 1 (stride R/Q1 = Q2): butterfly qq of sequence i takes elements qq + Q2 j, which for
// pass strides s >= kTile sit kTile-contiguous in global memory and are loaded straight into
// registers (Q1 independent loads per thread); for s < kTile the tile is first transposed
// through shared memory. Its outputs go to shared memory; sub-stage 2 (stride 1) reads
// elements Q2 pp + j there and writes its outputs pp + Q1 r straight to global memory, again
// kTile-contiguous per element. The block has kTile Q2 threads (PassShape). Twiddles are deferred
// as described above; the pass twiddle exponent p s of a thread's sequence is recomputed per
// thread.
// Thread shape of a pass of radix 2^LOGR = Q1 Q2 (L1 = ceil(LOGR / 2)). Sub-stage 1 has kTile Q2
// butterflies of radix Q1, sub-stage 2 kTile Q1 of radix Q2. A thread takes one butterfly of
// sub-stage 1 and B2 = Q1 / Q2 (1 or 2) of sub-stage 2, so no warp waits out a sub-stage (with a
// thread per butterfly of sub-stage 2, half the warps of an odd-LOGR pass idled through sub-stage 1).
template <int LOGR>
struct PassShape {
  static constexpr int L1 = (LOGR + 1) / 2, L2 = LOGR - L1;
  static constexpr int Q1 = 1 << L1, Q2 = 1 << L2;
  static constexpr int NT = kTile * Q2;       // threads = butterflies of sub-stage 1
  static constexpr int B2 = kTile * Q1 / NT;  // butterflies of sub-stage 2 per thread
};

template <int LOGR, bool INV, class C>
__global__ void __launch_bounds__(kFftThreads) k_fft_pass_reg(const C* __restrict__ src, C* __restrict__ dst,
                                                              int logF, int logS, const C* __restrict__ tw,
                                                              int logFmax, const C* __restrict__ hmul,
                                                              int64_t nseg, FftGen gen) {
  typedef PassShape<LOGR> PS;
  constexpr int R = 1 << LOGR;
  constexpr int L1 = PS::L1, L2 = PS::L2, Q1 = PS::Q1, Q2 = PS::Q2;
  constexpr int NT = PS::NT, B2 = PS::B2;
  constexpr int PER = R * kTile / NT;                // points per thread in the transposing fill
  static_assert(NT <= kFftThreads && B2 * NT == kTile * Q1, "thread shape");
  extern __shared__ __align__(16) unsigned char sm_raw[];
  C* v = reinterpret_cast<C*>(sm_raw);
  const int logFR = logF - LOGR;
  const uint64_t G0 = (uint64_t)blockIdx.x * kTile;
  const uint64_t col = G0 >> logFR;
  const uint32_t pi0 = (uint32_t)(G0 & ((1ull << logFR) - 1));
  // with hmul (first pass only, s >= kTile): column col reads source column col / nseg times
  // spectrum col % nseg
  const uint64_t scol = hmul ? col / (uint64_t)nseg : col;
  const C* x = src + (scol << logF);
  const C* hc = hmul ? hmul + ((col - scol * (uint64_t)nseg) << logF) : nullptr;
  C* y = dst + (col << logF);
  const uint32_t s = 1u << logS;
  const int fsh = logFmax - logF;
  const uint32_t fmask = (1u << logFmax) - 1u;
  const uint32_t i = threadIdx.x & (kTile - 1), bf = threadIdx.x / kTile;
  const uint32_t pti = ((pi0 + i) >> logS) << logS;  // p * s of this thread's sequence
  C a[Q1];
  if (s >= kTile) {
    const uint32_t p = pi0 >> logS, q0 = pi0 & (s - 1);
    const uint32_t off = q0 + ((p << LOGR) << logS) + i;
    if (gen.coef) {
      // first pass of a forward transform with generated input (p = 0)
      const GenCol<C> gc = gen_col<C>(gen, col);
#pragma unroll
      for (int j = 0; j < Q1; ++j) {
        const uint32_t t = off + ((bf + Q2 * j) << logS);
        a[j] = (int64_t)t < gc.lim ? coef_times(gen.coef, gc.cb + t, ldgc(gc.v + t))
                                   : mkc((typename RealOf<C>::type)0, (typename RealOf<C>::type)0);
      }
    } else {
      const C* xb = x + off;
#pragma unroll
      for (int j = 0; j < Q1; ++j) a[j] = xb[(bf + Q2 * j) << logS];
    }
    if (hc) {
#pragma unroll
      for (int j = 0; j < Q1; ++j) a[j] = cmul(a[j], ldgc(&hc[off + ((bf + Q2 * j) << logS)]));
    }
  } else {
    const C* xb = x + (pi0 << LOGR);
    const uint32_t srm = (s << LOGR) - 1;
    C t[PER];
#pragma unroll
    for (int u = 0; u < PER; ++u) t[u] = xb[threadIdx.x + u * NT];
#pragma unroll
    for (int u = 0; u < PER; ++u) {
      const uint32_t idx = threadIdx.x + u * NT;
      const uint32_t pl = idx >> (logS + LOGR), rem = idx & srm;
      const uint32_t j = rem >> logS, q = rem & (s - 1);
      v[j * kRow + ((pl << logS) + q)] = t[u];
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < Q1; ++j) a[j] = v[(bf + Q2 * j) * kRow + i];
    __syncthreads();  // sub-stage 1 overwrites the tile in place
  }
  // the first pass (p = 0, pti = 0) has only the constant twiddles of reg_dft_unit here
  if (logS == logF - LOGR) reg_dft_unit<L1, INV>(a);
  else reg_dft<L1, INV>(a, (pti << L2) << fsh, tw, logFmax, fmask);
#pragma unroll
  for (int r = 0; r < Q1; ++r) v[(bf + Q2 * r) * kRow + i] = a[r];
  __syncthreads();
#pragma unroll
  for (int u = 0; u < B2; ++u) {
    const uint32_t b2 = bf + u * (NT / kTile);  // this thread's butterfly of sub-stage 2
    C b[Q2];
#pragma unroll
    for (int j = 0; j < Q2; ++j) b[j] = v[(Q2 * b2 + j) * kRow + i];
    reg_dft<L2, INV>(b, (b2 << (logFmax - LOGR)) + (pti << fsh), tw, logFmax, fmask);
    C* yb = y + pi0 + i;
#pragma unroll
    for (int r = 0; r < Q2; ++r) yb[(b2 + Q1 * r) << logFR] = b[r];
  }
}

// Whole transforms of length F = 2^LOGF <= 4096 in one launch: a CTA holds kSmallPts points
// (kSmallPts / F columns, contiguous in global memory) in shared memory, padded by one element
// per 16 (e -> e + e/16) against bank conflicts of strided butterflies, and runs the Stockham
// decimation-in-time sub-stages of radices 2^L (L <= 4, two sub-stages for LOGF <= 8, three
// above) in registers with reg_dft. Sub-stage k (radix Q, sub-length so far m, stride s = F/(mQ))
// takes butterfly (pp < m, qq < s) from elements qq + s(Q pp + j) and writes qq + s(pp + r m);
// the last one (s = 1) writes straight to global memory. There is no pass twiddle.
constexpr int kSmallPts = 4096;
constexpr int kSmallLog = 12;  // longest transform done by k_fft_small

// Sub-stage radices 2^L(i), i < NS, as equal as possible with the larger first and L <= LQMAX:
// 16 for FP64 and FP32, 8 for double-float (whose 16-point register DFTs need 112 registers a
// thread and leave two CTAs per SM stalled at the barriers). FP64/FP32 CTAs have one thread per
// butterfly of the narrowest sub-stage; double-float CTAs one per butterfly of the widest
// (512 threads), each taking several butterflies of the narrower sub-stages, within 64
// registers so that two CTAs share an SM.
template <int LOGF, class C>
struct SmallSplit {
  static constexpr bool DF = std::is_same<C, df64c>::value;
  static constexpr int LQMAX = DF ? 3 : 4;
  static constexpr int NS = (LOGF + LQMAX - 1) / LQMAX < 2 ? 2 : (LOGF + LQMAX - 1) / LQMAX;
  __host__ __device__ static constexpr int L(int i) { return LOGF / NS + (i < LOGF % NS ? 1 : 0); }
  static constexpr int NT = kSmallPts >> (DF ? L(0) : L(NS - 1));
  static constexpr int MINB = DF ? 2 : 0;  // CTAs per SM the registers must allow (0: no bound)
};

__device__ __forceinline__ uint32_t spad(uint32_t e) { return e + (e >> 4); }

// One in-place sub-stage over the tile (every butterfly of radix 2^LQ; LOGNN = log2 of the
// sub-length after it), NT threads taking butterflies b = thread + u NT. LAST writes to global
// memory instead. The first sub-stage (LOGNN = LQ) has only the constant twiddles of
// reg_dft_unit. tw is the table of this length (2^LOGF).
template <int LOGF, int LQ, int LOGNN, bool LAST, bool INV, int NT, class C>
__device__ __forceinline__ void small_stage(C* v, const C* __restrict__ tw, C* __restrict__ y, int64_t col0,
                                            int64_t ncols) {
  constexpr int F = 1 << LOGF, Q = 1 << LQ;
  constexpr uint32_t Fp = F + F / 16;
  constexpr int NB = kSmallPts / Q;
  constexpr int BPT = (NB + NT - 1) / NT;  // butterflies per thread
  constexpr int logs = LOGF - LOGNN, logm = LOGNN - LQ;
  if constexpr (BPT == 1) {
    const uint32_t b = threadIdx.x;
    const bool act = b < NB;
    C a[Q];
    uint32_t c = 0, pp = 0, qq = 0;
    if (act) {
      c = b >> (LOGF - LQ);
      const uint32_t bb = b & ((F >> LQ) - 1);
      pp = bb >> logs;
      qq = bb & ((1u << logs) - 1);
      const C* vc = v + c * Fp;
#pragma unroll
      for (int j = 0; j < Q; ++j) a[j] = vc[spad(qq + ((pp * Q + j) << logs))];
    }
    if (!LAST) __syncthreads();  // the sub-stage works in place
    if (act) {
      if (LOGNN == LQ) reg_dft_unit<LQ, INV>(a);
      else reg_dft<LQ, INV>(a, pp << (LOGF - LOGNN), tw, LOGF, (uint32_t)F - 1u);
      if (LAST) {
        if (col0 + c < ncols) {
          C* yc = y + (col0 + c) * F;
#pragma unroll
          for (int r = 0; r < Q; ++r) yc[pp + (r << logm)] = a[r];
        }
      } else {
        C* vc = v + c * Fp;
#pragma unroll
        for (int r = 0; r < Q; ++r) vc[spad(qq + ((pp + (r << logm)) << logs))] = a[r];
      }
    }
    if (!LAST) __syncthreads();
  } else {
    C a[BPT][Q];
    uint32_t c[BPT], pp[BPT], qq[BPT];
#pragma unroll
    for (int u = 0; u < BPT; ++u) {
      const uint32_t b = threadIdx.x + u * NT;
      c[u] = pp[u] = qq[u] = 0;
      if (b < NB) {
        c[u] = b >> (LOGF - LQ);
        const uint32_t bb = b & ((F >> LQ) - 1);
        pp[u] = bb >> logs;
        qq[u] = bb & ((1u << logs) - 1);
        const C* vc = v + c[u] * Fp;
#pragma unroll
        for (int j = 0; j < Q; ++j) a[u][j] = vc[spad(qq[u] + ((pp[u] * Q + j) << logs))];
      }
    }
    if (!LAST) __syncthreads();  // the sub-stage works in place
#pragma unroll
    for (int u = 0; u < BPT; ++u) {
      if (threadIdx.x + u * NT >= NB) continue;
      if (LOGNN == LQ) reg_dft_unit<LQ, INV>(a[u]);
      else reg_dft<LQ, INV>(a[u], pp[u] << (LOGF - LOGNN), tw, LOGF, (uint32_t)F - 1u);
      if (LAST) {
        if (col0 + c[u] < ncols) {
          C* yc = y + (col0 + c[u]) * F;
#pragma unroll
          for (int r = 0; r < Q; ++r) yc[pp[u] + (r << logm)] = a[u][r];
        }
      } else {
        C* vc = v + c[u] * Fp;
#pragma unroll
        for (int r = 0; r < Q; ++r) vc[spad(qq[u] + ((pp[u] + (r << logm)) << logs))] = a[u][r];
      }
    }
    if (!LAST) __syncthreads();
  }
}

template <int LOGF, bool INV, class C>
__global__ void __launch_bounds__(SmallSplit<LOGF, C>::NT, SmallSplit<LOGF, C>::MINB)
    k_fft_small(const C* __restrict__ src, C* __restrict__ dst, int64_t ncols, const C* __restrict__ tw, int logFmax,
                const C* __restrict__ hmul, int64_t nseg, FftGen gen) {
  typedef SmallSplit<LOGF, C> S;
  constexpr int F = 1 << LOGF;
  constexpr uint32_t Fp = F + F / 16;
  constexpr int NCOL = kSmallPts / F;
  constexpr int PER = kSmallPts / S::NT;
  extern __shared__ __align__(16) unsigned char sm_raw[];
  C* v = reinterpret_cast<C*>(sm_raw);
  const int64_t col0 = (int64_t)blockIdx.x * NCOL;
  const C* x = src + col0 * F;
  const int64_t avail = (ncols - col0) * F;  // points of this CTA's columns that exist
  C t[PER];
  if (gen.coef) {
    // generated input: per column of the CTA, its table row, first coefficient and length
    __shared__ const C* gv[NCOL];
    __shared__ int64_t gcb[NCOL];
    __shared__ int64_t glim[NCOL];
    if (threadIdx.x < NCOL) {
      const GenCol<C> q = gen_col<C>(gen, (uint64_t)(col0 + threadIdx.x));
      gv[threadIdx.x] = q.v;
      gcb[threadIdx.x] = q.cb;
      glim[threadIdx.x] = q.lim;
    }
    __syncthreads();
#pragma unroll
    for (int u = 0; u < PER; ++u) {
      const uint32_t idx = threadIdx.x + u * S::NT;
      const uint32_t c = idx >> LOGF, e = idx & (F - 1);
      t[u] = ((int64_t)idx < avail && (int64_t)e < glim[c])
                 ? coef_times(gen.coef, gcb[c] + e, ldgc(gv[c] + e))
                 : mkc((typename RealOf<C>::type)0, (typename RealOf<C>::type)0);
    }
  } else if (hmul) {
    // column col0 + c is source column (col0 + c) / nseg times spectrum (col0 + c) % nseg
    __shared__ int64_t scol[NCOL];
    __shared__ int64_t sseg[NCOL];
    if (threadIdx.x < NCOL) {
      const int64_t vc = col0 + threadIdx.x;
      scol[threadIdx.x] = vc / nseg;
      sseg[threadIdx.x] = vc - scol[threadIdx.x] * nseg;
    }
    __syncthreads();
#pragma unroll
    for (int u = 0; u < PER; ++u) {
      const uint32_t idx = threadIdx.x + u * S::NT;
      const uint32_t c = idx >> LOGF, e = idx & (F - 1);
      t[u] = (int64_t)idx < avail ? cmul(src[scol[c] * F + e], ldgc(&hmul[sseg[c] * F + e]))
                                  : mkc((typename RealOf<C>::type)0, (typename RealOf<C>::type)0);
    }
  } else {
#pragma unroll
    for (int u = 0; u < PER; ++u) {
      const uint32_t idx = threadIdx.x + u * S::NT;
      t[u] = (int64_t)idx < avail ? x[idx] : mkc((typename RealOf<C>::type)0, (typename RealOf<C>::type)0);
    }
  }
#pragma unroll
  for (int u = 0; u < PER; ++u) {
    const uint32_t idx = threadIdx.x + u * S::NT;
    v[(idx >> LOGF) * Fp + spad(idx & (F - 1))] = t[u];
  }
  __syncthreads();
  constexpr int L0 = S::L(0), L1 = S::L(1), L2 = S::L(2), L3 = S::L(3), NT = S::NT;
  if constexpr (S::NS == 2) {
    small_stage<LOGF, L0, L0, false, INV, NT>(v, tw, dst, col0, ncols);
    small_stage<LOGF, L1, LOGF, true, INV, NT>(v, tw, dst, col0, ncols);
  } else if constexpr (S::NS == 3) {
    small_stage<LOGF, L0, L0, false, INV, NT>(v, tw, dst, col0, ncols);
    small_stage<LOGF, L1, L0 + L1, false, INV, NT>(v, tw, dst, col0, ncols);
    small_stage<LOGF, L2, LOGF, true, INV, NT>(v, tw, dst, col0, ncols);
  } else {
    static_assert(S::NS == 4, "at most four sub-stages");
    small_stage<LOGF, L0, L0, false, INV, NT>(v, tw, dst, col0, ncols);
    small_stage<LOGF, L1, L0 + L1, false, INV, NT>(v, tw, dst, col0, ncols);
    small_stage<LOGF, L2, L0 + L1 + L2, false, INV, NT>(v, tw, dst, col0, ncols);
    small_stage<LOGF, L3, LOGF, true, INV, NT>(v, tw, dst, col0, ncols);
  }
}

template <int LOGF, bool INV, class C>
void launch_small(const C* src, C* dst, int ncols, const C* tw, int logFmax, const C* hmul, int64_t nseg,
                  const FftGen& gen, cudaStream_t st) {
  constexpr int F = 1 << LOGF;
  constexpr int NCOL = kSmallPts / F;
  const size_t smem = (size_t)NCOL * (F + F / 16) * sizeof(C);
  static bool configured = false;
  if (!configured) {
    cudaFuncSetAttribute(k_fft_small<LOGF, INV, C>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    configured = true;
  }
  const int64_t grid = ((int64_t)ncols + NCOL - 1) / NCOL;
  k_fft_small<LOGF, INV, C><<<(unsigned)grid, SmallSplit<LOGF, C>::NT, smem, st>>>(src, dst, ncols, tw, logFmax,
                                                                                   hmul, nseg, gen);
}

template <bool INV, class C>
void launch_small_f(int logF, const C* src, C* dst, int ncols, const C* tw, int logFmax, const C* hmul, int64_t nseg,
                    const FftGen& gen, cudaStream_t st) {
  switch (logF) {
    case 6: launch_small<6, INV>(src, dst, ncols, tw, logFmax, hmul, nseg, gen, st); break;
    case 7: launch_small<7, INV>(src, dst, ncols, tw, logFmax, hmul, nseg, gen, st); break;
    case 8: launch_small<8, INV>(src, dst, ncols, tw, logFmax, hmul, nseg, gen, st); break;
    case 9: launch_small<9, INV>(src, dst, ncols, tw, logFmax, hmul, nseg, gen, st); break;
    case 10: launch_small<10, INV>(src, dst, ncols, tw, logFmax, hmul, nseg, gen, st); break;
    case 11: launch_small<11, INV>(src, dst, ncols, tw, logFmax, hmul, nseg, gen, st); break;
    default: launch_small<12, INV>(src, dst, ncols, tw, logFmax, hmul, nseg, gen, st); break;
  }
}

template <int LOGR, bool INV, class C>
void launch_pass(const C* src, C* dst, int logF, int logS, int ncols, const C* tw, int logFmax, const C* hmul,
                 int64_t nseg, const FftGen& gen, cudaStream_t st) {
  constexpr int R = 1 << LOGR;
  const int64_t pairs = ((int64_t)ncols << logF) >> LOGR;
  const int64_t grid = pairs / kTile;
  // one buffer (the sub-stages work in place)
  constexpr int threads = PassShape<LOGR>::NT;
  const size_t smem = (size_t)R * kRow * sizeof(C);
  static bool configured = false;
  if (!configured) {
    cudaFuncSetAttribute(k_fft_pass_reg<LOGR, INV, C>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    configured = true;
  }
  k_fft_pass_reg<LOGR, INV, C><<<(unsigned)grid, threads, smem, st>>>(src, dst, logF, logS, tw, logFmax, hmul, nseg,
                                                                      gen);
}

template <bool INV, class C>
void launch_pass_r(int logR, const C* src, C* dst, int logF, int logS, int ncols, const C* tw, int logFmax,
                   const C* hmul, int64_t nseg, const FftGen& gen, cudaStream_t st) {
  // transforms longer than 4096 points split into passes of radix 2^5 .. 2^8
  switch (logR) {
    case 5: launch_pass<5, INV>(src, dst, logF, logS, ncols, tw, logFmax, hmul, nseg, gen, st); break;
    case 6: launch_pass<6, INV>(src, dst, logF, logS, ncols, tw, logFmax, hmul, nseg, gen, st); break;
    case 7: launch_pass<7, INV>(src, dst, logF, logS, ncols, tw, logFmax, hmul, nseg, gen, st); break;
    default: launch_pass<8, INV>(src, dst, logF, logS, ncols, tw, logFmax, hmul, nseg, gen, st); break;
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

template <class C>
__global__ void k_scale_copy(const double2* src, C* dst, int64_t n, double scale) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x)
    dst[t] = from_d2<C>(make_double2(src[t].x * scale, src[t].y * scale));
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

template <class C>
void launch_scale_copy(const double2* src, C* dst, int64_t n, double scale, cudaStream_t st) {
  k_scale_copy<C><<<grid_for(n, 256), 256, 0, st>>>(src, dst, n, scale);
}


FftShape default_fft_shape(int logF, int ncols, int prec) {
  FftShape sh{};
  // few columns of 2^10 .. 2^12 points would give the one-launch kernel only a few CTAs (a CTA
  // holds 4096 points): two passes spread them over 8 to 32 times as many
  const int64_t small_ctas = logF <= kSmallLog ? ((int64_t)ncols + (kSmallPts >> logF) - 1) / (kSmallPts >> logF) : 0;
  const bool few = logF >= 10 && small_ctas < 152;
  if (logF <= kSmallLog && !few) {
    sh.one_launch = 1;
    return sh;
  }
  // passes of radix 2^5 .. 2^8 (logF >= 10), each leaving F/R >= kTile pairs per column. FP64 and
  // FP32 take the fewest passes (radix up to 256); double-float keeps to radix 64 where 2^5 .. 2^6
  // can make up F (its radix-128 pass needs 112 registers a thread and issues on half the cycles
  // of radix 64)
  const int maxlog = prec == kTermDF64 ? 6 : 8;
  int np = (logF + maxlog - 1) / maxlog;
  while (np > 1 && logF / np < 5) --np;
  const int base = logF / np, extra = logF % np;
  sh.npass = np;
  for (int i = 0; i < np && i < 4; ++i) sh.logr[i] = base + (i < extra ? 1 : 0);
  return sh;
}

bool valid_fft_shape(const FftShape& sh, int logF) {
  if (sh.one_launch) return logF >= 6 && logF <= kSmallLog && sh.tc == 0;
  if (sh.npass < 2 || sh.npass > 4) return false;  // a pass leaves F / R >= kTile sequences
  if (sh.tc & ~((1 << sh.npass) - 1)) return false;
  int sum = 0;
  for (int i = 0; i < sh.npass; ++i) {
    if (sh.logr[i] < 5 || sh.logr[i] > 8) return false;
    // a tensor-core pass has radix 32 or 64; below 4096 points only the first pass (no twiddles,
    // its tiles span columns) runs there
    if (((sh.tc >> i) & 1) && ((sh.logr[i] != 5 && sh.logr[i] != 6) || (logF < 12 && i > 0))) return false;
    sum += sh.logr[i];
  }
  return sum == logF;
}

template <class C>
int run_fft(C* a, C* b, int logF, int ncols, bool inverse, const C* tw, int logFmax, cudaStream_t st, C** result,
            int* npasses, const C* hmul, int64_t nseg, const FftGen* gen, const FftShape* shape, const TcTables* tc) {
  if (logF < 6 || logF > logFmax || nseg < 1) return HANKEL_EINVAL;
  if (gen && (inverse || hmul || gen->nsegc < 1 || gen->ncols < 1)) return HANKEL_EINVAL;
  FftGen g0{};
  if (gen) g0 = *gen;
  const FftGen none{};
  // the ladder's table for this length: W_F^t at tw[F + t]
  tw += (size_t)1 << logF;
  logFmax = logF;
  const int prec = std::is_same<C, df64c>::value ? kTermDF64 : std::is_same<C, float2>::value ? kTermFP32 : kTermFP64;
  FftShape sh = (shape && valid_fft_shape(*shape, logF)) ? *shape : default_fft_shape(logF, ncols, prec);
  if (!tc || !std::is_same<C, double2>::value) sh.tc = 0;  // tensor-core passes: FP64 transforms with tables
  if (sh.one_launch) {
    // the whole transform in one launch
    if (inverse) launch_small_f<true, C>(logF, a, b, ncols, tw, logFmax, hmul, nseg, none, st);
    else launch_small_f<false, C>(logF, a, b, ncols, tw, logFmax, hmul, nseg, g0, st);
    *result = b;
    if (npasses) *npasses = 1;
    return HANKEL_OK;
  }
  // the first pass (stride F/R >= kTile) applies the input product or generates the input
  C* src = a;
  C* dst = b;
  int done = 0;  // log2 of the sub-length transformed so far
  for (int i = 0; i < sh.npass; ++i) {
    const int lr = sh.logr[i];
    done += lr;
    const int logS = logF - done;
    const C* h = i == 0 ? hmul : nullptr;
    if ((sh.tc >> i) & 1) {
      if constexpr (std::is_same<C, double2>::value)
        launch_pass_tc(inverse, lr, src, dst, logF, logS, ncols, tc->twq + ((size_t)1 << logF), h, nseg,
                       (!inverse && i == 0) ? g0 : none, inverse ? tc->inv : tc->fwd, tc->err, st);
    } else if (inverse) {
      launch_pass_r<true, C>(lr, src, dst, logF, logS, ncols, tw, logFmax, h, nseg, none, st);
    } else {
      launch_pass_r<false, C>(lr, src, dst, logF, logS, ncols, tw, logFmax, h, nseg, i == 0 ? g0 : none, st);
    }
    std::swap(src, dst);
  }
  *result = src;
  if (npasses) *npasses = sh.npass;
  return HANKEL_OK;
}

template int run_fft<double2>(double2*, double2*, int, int, bool, const double2*, int, cudaStream_t, double2**,
                              int*, const double2*, int64_t, const FftGen*, const FftShape*, const TcTables*);
template int run_fft<float2>(float2*, float2*, int, int, bool, const float2*, int, cudaStream_t, float2**, int*,
                             const float2*, int64_t, const FftGen*, const FftShape*, const TcTables*);
template int run_fft<df64c>(df64c*, df64c*, int, int, bool, const df64c*, int, cudaStream_t, df64c**, int*,
                            const df64c*, int64_t, const FftGen*, const FftShape*, const TcTables*);
template void launch_scale_copy<double2>(const double2*, double2*, int64_t, double, cudaStream_t);
template void launch_scale_copy<float2>(const double2*, float2*, int64_t, double, cudaStream_t);
template void launch_scale_copy<df64c>(const double2*, df64c*, int64_t, double, cudaStream_t);

}  // namespace hk
