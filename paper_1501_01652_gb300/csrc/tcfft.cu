// FP64-accurate radix-32 FFT passes on the tensor cores (tcgen05, TMEM accumulators).
//
// A Stockham pass of radix R = 32 (the mapping of k_fft_pass_reg<5>): for every sequence
// g = p s + q of a column (s the pass stride, p < F/(R s), q < s),
//   y[g + (F/R) r] = sum_{e<R} W_R^{r e} v_e,   v_e = W_F^{p s e} x[q + s (R p + e)],   r < R.
// Written with real and imaginary parts side by side, one pass over 128 sequences is the real
// product Y (128 x 64) = V (128 x 64) B (64 x 64), B the real form of the 32-point DFT matrix:
// a dense contraction, done here on the tensor cores in FP64 accuracy by splitting both
// operands into exact 8-bit digits (the Ozaki scheme):
//  * each sequence's 64 reals are scaled by 2^-E (2^E above the sequence's largest |v|) and
//    rounded to the integers X = v 2^(54-E) (|X| <= 2^54); every entry of B is rounded to
//    W = B 2^54. Both are written as 7 balanced base-256 digits in [-128, 127], exact in fp16;
//  * tcgen05.mma (kind::f16, fp32 accumulation in TMEM) sums the digit products of each
//    diagonal s = a + b (digit a of X, digit b of W) over the 64 reals: a product is at most
//    2^14 in size and a diagonal holds at most 7 x 64 of them, so every partial sum is an
//    integer below 2^23 and exact. Diagonals s <= 7 are kept: the others weigh at most about
//    2^-53 of 2^E per output, the rounding of an FP64 product;
//  * the diagonals are combined in 64-bit integers, Y = sum_s D_s 2^(43 - 8s) = y 2^(55-E)
//    (|y| < 2^(E+6), so |Y| < 2^61), the two smallest diagonals rounded to the nearest unit,
//    and converted to double once (int64 to double, the scale added to the exponent field).
// The pass twiddles W_F^{p s e} multiply the integers X (Q62 twiddles, 64-bit high products,
// rounded back to units of X; a rotation keeps |X| below 2^54.5, inside the digits' range), so the
// FP64 pipe (the scarce one on this part) sees only the two int64-to-double conversions of each
// output and the first pass's column generation or spectrum product (FP64 products on its loads,
// as in the FP64 pass). One CTA per SM (persistent; 168 KB of shared
// memory for the digits, all 512 TMEM columns for the 8 diagonal accumulators): per tile of 128
// sequences it splits the inputs (512 threads: sequence i, quarter qd of its elements), one
// thread issues the 45 MMAs, every thread sends out the loads of the CTA's next tile while
// they run, and after their commit reads back 8 of its sequence's outputs. Waits on mbarriers are bounded: a wait that runs out sets the plan's error word and
// the kernel stops, frees its TMEM and returns.
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <algorithm>
#include <vector>

#include "cplx.cuh"
#include "kernels.cuh"

namespace hk {

namespace {

constexpr int kR = 32;                  // radix
constexpr int kRows = 128;              // sequences per tile (MMA M)
constexpr int kKr = 2 * kR;             // reals per sequence (MMA K = N = 64)
constexpr int kDig = 7;                 // digits per operand
constexpr int kDiag = 8;                // diagonals kept (s = a + b <= 7)
constexpr int kThreads = 512;   // sequence i = thread % 128, quarter thread / 128
constexpr uint32_t kAPlane = kRows * kKr * 2;  // 16 KB per digit plane of the sequences
constexpr uint32_t kBPlane = kKr * kKr * 2;    // 8 KB per digit plane of the DFT matrix
constexpr uint32_t kSmA = 0;
constexpr uint32_t kSmB = kSmA + kDig * kAPlane;           // 112 KB
constexpr uint32_t kSmZero = kSmB + kDig * kBPlane;        // 168 KB: a zero plane of the sequences' layout
constexpr uint32_t kSmBar = kSmZero + kAPlane;             // 184 KB
constexpr uint32_t kSmSlot = kSmBar + 16;
constexpr uint32_t kSmExp = kSmBar + 32;                   // [4][128] exponents
constexpr uint32_t kSmTotal = kSmExp + 4 * kRows * 4;
constexpr uint32_t kTmemCols = 512;                        // kDiag x 64 fp32 columns
// The digits of X are the base-256 digits of X + kOff, less 128 (kOff has every digit 128).
constexpr unsigned long long kOff = 0x0080808080808080ULL;
// Instruction descriptor of tcgen05.mma kind::f16: D in fp32 (bits 4-5 = 1), A and B fp16
// (formats 0), both K-major, N (bits 17-22: N >> 3), M = 128 (bits 24-28: M >> 4).
__host__ __device__ constexpr uint32_t idesc_n(uint32_t n) {
  return (1u << 4) | ((n >> 3) << 17) | ((uint32_t)(kRows >> 4) << 24);
}
constexpr long long kWaitCycles = 2000000000LL;  // about one second at 2 GHz

__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Shared-memory matrix descriptor, K-major without swizzle: core matrices of 8 rows x 16 bytes;
// the next 8 elements along K lie 128 bytes on (leading byte offset), the next 8 rows 1024 bytes
// on (stride byte offset); bits 46-47 hold the descriptor version 1.
__device__ __forceinline__ uint64_t mat_desc(uint32_t addr) {
  return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)(128 >> 4) << 16) | ((uint64_t)(1024 >> 4) << 32) |
         (1ULL << 46);
}

// Byte offset of element (row, k) in a K-major digit plane of 64 K columns.
__host__ __device__ constexpr uint32_t core_off(uint32_t row, uint32_t k) {
  return (row >> 3) * 1024u + (k >> 3) * 128u + (row & 7u) * 16u + (k & 7u) * 2u;
}

__device__ __forceinline__ bool bar_wait(uint32_t bar, uint32_t parity, long long t0) {
  for (;;) {
    uint32_t done = 0;
    asm volatile(
        "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
    if (done) return true;
    if (clock64() - t0 > kWaitCycles) return false;
  }
}

__device__ __forceinline__ void mma_f16(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\ntcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
      "l"(a), "l"(b), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ void tmem_ld8(uint32_t taddr, uint32_t (&r)[8]) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
               : "r"(taddr));
}

// X = round(v 2^(54 - E)) for |v| < 2^E (integer operations on the bits of v, without branches).
__device__ __forceinline__ long long to_fixed(double v, int E) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(v);
  const int ef = (int)((b >> 52) & 0x7ff);
  const unsigned long long M2 = ((b & 0xFFFFFFFFFFFFFULL) | (ef ? (1ULL << 52) : 0ULL)) << 1;
  // v = M2 2^(max(ef, 1) - 1076), so v 2^(54 - E) = M2 2^-t with t = 1022 + E - max(ef, 1) >= 0
  const int t = min(1022 + E - max(ef, 1), 63);
  const long long X = (long long)((M2 + ((1ULL << t) >> 1)) >> t);
  return (long long)b < 0 ? -X : X;
}

// Exponent field of v (0 for zeros and subnormals).
__device__ __forceinline__ int exp_field(double v) {
  return (int)(((unsigned long long)__double_as_longlong(v) >> 52) & 0x7ff);
}

// Fused column generation of a forward transform's first pass (FftGen): column col of the chunk
// takes points t < lim as coef[cb + t] Vt-row[t] and zeros beyond.
struct GenSrc {
  const double* c;
  const double2* v;
  int64_t lim;
};
__device__ __forceinline__ GenSrc gen_source(const FftGen& g, int64_t col) {
  const int64_t cc = col / g.nsegc;
  const int64_t sg = col - cc * g.nsegc;
  const int64_t gi = g.c0 + cc;
  const int64_t rhs = gi / g.ncols, li = gi - rhs * g.ncols;
  const int64_t nlo = sg * g.S;
  GenSrc r;
  r.c = reinterpret_cast<const double*>(g.coef) + rhs * g.ldc + g.n0 - 1 + nlo;
  r.v = reinterpret_cast<const double2*>(g.Vt) + li * g.C + nlo;
  r.lim = min(g.S, g.C - nlo);
  return r;
}

// Loads of one tile's inputs for a thread (its sequence's elements e = e0 + j es, j < 8) into v,
// with the first pass's column generation or spectrum product.
__device__ __forceinline__ void load_inputs(double2 (&v)[8], const double2* __restrict__ src,
                                            const double2* __restrict__ hmul, int64_t nseg, const FftGen& gen,
                                            int logF, int logS, int64_t col, uint32_t ibase, int e0, int es) {
  if (gen.coef) {
    const GenSrc gs = gen_source(gen, col);
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const int64_t t = (int64_t)ibase + ((int64_t)(e0 + j * es) << logS);
      if (t < gs.lim) {
        const double c = __ldg(gs.c + t);
        const double2 w = __ldg(gs.v + t);
        v[j] = make_double2(c * w.x, c * w.y);
      } else {
        v[j] = make_double2(0.0, 0.0);
      }
    }
  } else if (hmul) {
    const int64_t scol = col / nseg, seg = col - scol * nseg;
    const double2* x = src + (scol << logF);
    const double2* hc = hmul + (seg << logF);
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const uint32_t t = ibase + ((uint32_t)(e0 + j * es) << logS);
      v[j] = cmul(x[t], __ldg(&hc[t]));
    }
  } else {
    const double2* x = src + (col << logF);
#pragma unroll
    for (int j = 0; j < 8; ++j) v[j] = x[ibase + ((uint32_t)(e0 + j * es) << logS)];
  }
}

// R64: a radix-64 pass. Each 64-point DFT is two 32-point DFTs, of the even and of the odd
// elements (rows j and 64 + j of the tile, both scaled by the sequence's 2^E), on the tensor cores,
// and one radix-2 step in 64-bit integers: y_r = Z0_r + W_64^r Z1_r, y_{r+32} = Z0_r - W_64^r Z1_r,
// r < 32 (the odd rows' Z1 times the Q62 twiddle, exchanged through shared memory).
template <bool INV, bool R64>
__global__ void __launch_bounds__(kThreads, 1)
    k_fft_pass_tc(const double2* __restrict__ src, double2* __restrict__ dst, int logF, int logS, int64_t ntiles,
                  const longlong2* __restrict__ twq, const double2* __restrict__ hmul, int64_t nseg, FftGen gen,
                  const void* __restrict__ bdig, unsigned* err) {
  extern __shared__ __align__(1024) unsigned char sm[];
  const int tid = threadIdx.x, i = tid & (kRows - 1), qd = tid >> 7, warp = tid >> 5;
  const uint32_t sbase = smem_addr(sm);
  const uint32_t bar_b = sbase + kSmBar, bar_m = sbase + kSmBar + 8;
  uint32_t* slot = reinterpret_cast<uint32_t*>(sm + kSmSlot);
  int* emx = reinterpret_cast<int*>(sm + kSmExp);
  __shared__ int s_fail;
  const long long t0 = clock64();

  for (int z = tid; z < (int)(kAPlane / 16); z += kThreads)
    reinterpret_cast<uint4*>(sm + kSmZero)[z] = make_uint4(0u, 0u, 0u, 0u);
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  if (tid == 0) {
    s_fail = 0;
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar_b), "r"(1));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar_m), "r"(1));
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(sbase + kSmSlot),
                 "r"(kTmemCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tbase = *slot;
  // the DFT matrix digits: one bulk copy into shared memory
  if (tid == 0) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar_b), "r"(kDig * kBPlane)
                 : "memory");
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     sbase + kSmB),
                 "l"(bdig), "r"(kDig * kBPlane), "r"(bar_b)
                 : "memory");
  }

  constexpr int LR = R64 ? 6 : 5;            // log2 of the radix
  constexpr int LT = R64 ? 6 : 7;            // log2 of the sequences per tile
  const int lgs = logF - LR;                 // log2 of the sequences per column
  const int tpc_log = lgs - LT;              // log2 of the tiles per column
  const uint32_t smask = (1u << logS) - 1u;
  const int jrow = R64 ? (i & 63) : i;       // the tile's sequence of this row
  const int par = R64 ? (i >> 6) : 0;        // R64: even (0) or odd (1) elements
  const int e0 = R64 ? 16 * qd + par : 8 * qd, es = R64 ? 2 : 1;  // this thread's elements e0 + j es
  auto seq_of = [&](int64_t tile, int64_t& col, uint32_t& g, uint32_t& p, uint32_t& ibase) {
    col = tile >> tpc_log;
    g = (uint32_t)((tile & ((int64_t(1) << tpc_log) - 1)) << LT) + (uint32_t)jrow;
    p = g >> logS;
    ibase = (g & smask) + ((p << LR) << logS);  // element e at ibase + (e << logS)
  };
  double2 v[8];
  int64_t tile = blockIdx.x;
  if (tile < ntiles) {
    int64_t col;
    uint32_t g, p, ib;
    seq_of(tile, col, g, p, ib);
    load_inputs(v, src, hmul, nseg, gen, logF, logS, col, ib, e0, es);
  }
  // every thread waits; the CTA agrees on the outcome, so all of it leaves the loop together
  if (__syncthreads_or(!bar_wait(bar_b, 0, t0) ? 1 : 0)) s_fail = 1;
  __syncthreads();

  uint32_t phase = 0;
  for (; tile < ntiles && !s_fail; tile += gridDim.x) {
    int64_t col;
    uint32_t g, p, ibase;
    seq_of(tile, col, g, p, ibase);
    // 1. the sequence's scale 2^E (largest exponent over its four quarters, before the twiddles)
    int m = 1;
#pragma unroll
    for (int j = 0; j < 8; ++j) m = max(m, max(exp_field(v[j].x), exp_field(v[j].y)));
    emx[qd * kRows + i] = m;
    __syncthreads();
    int mx = max(max(emx[i], emx[kRows + i]), max(emx[2 * kRows + i], emx[3 * kRows + i]));
    if (R64) {  // both rows of the sequence
      const int o = i ^ 64;
      mx = max(mx, max(max(emx[o], emx[kRows + o]), max(emx[2 * kRows + o], emx[3 * kRows + o])));
    }
    const int E = mx - 1022;
    // 2. X = v 2^(54 - E) in integers, times the pass twiddles W_F^{p s e} (Q62) with the product
    //    rounded back to units of X
    long long xr[8], xi[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      xr[j] = to_fixed(v[j].x, E);
      xi[j] = to_fixed(v[j].y, E);
    }
    if (p != 0) {
      const uint32_t ps = p << logS;
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const longlong2 w = __ldg(&twq[ps * (uint32_t)(e0 + j * es)]);
        const long long wi = INV ? -w.y : w.y;
        // three products (Gauss): re = a c - b d, im = (a + b)(c + d) - a c - b d, with a, b the
        // parts of X shifted left by 7 (at most 2^61 each, their sum at most 2^62) and c, d the
        // twiddle's (|c + d| <= 2^62.5): no product or sum overflows
        const long long ar = xr[j] << 7, ai = xi[j] << 7;
        const long long ac = __mul64hi(ar, w.x), bd = __mul64hi(ai, wi);
        const long long re = (ac - bd) << 1;  // (X w) 2^6, within 4 units
        const long long im = (__mul64hi(ar + ai, w.x + wi) - ac - bd) << 1;
        xr[j] = (re + 32) >> 6;
        xi[j] = (im + 32) >> 6;
      }
    }
    // 3. digits: plane a holds digit a (weight 256^(6 - a)) of every real; this thread writes
    //    K columns 16 qd .. 16 qd + 15 of row i (2 core-matrix rows of 16 bytes per plane). The
    //    digits of X are the bytes of X + kOff less 128: one byte permutation takes byte b of the
    //    real and imaginary parts into the low bytes of the two fp16 halves, whose bits 0x6400 + u
    //    are 1024 + u, and one packed subtraction of 1152 leaves u - 128.
#pragma unroll
    for (int c2 = 0; c2 < 2; ++c2) {
      uint32_t rlo[4], rhi[4], ilo[4], ihi[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const unsigned long long yr = (unsigned long long)xr[4 * c2 + u] + kOff;
        const unsigned long long yi = (unsigned long long)xi[4 * c2 + u] + kOff;
        rlo[u] = (uint32_t)yr;
        rhi[u] = (uint32_t)(yr >> 32);
        ilo[u] = (uint32_t)yi;
        ihi[u] = (uint32_t)(yi >> 32);
      }
      const uint32_t off = core_off((uint32_t)i, (uint32_t)(16 * qd + 8 * c2));
      const __half2 bias = __half2half2(__ushort_as_half(0x6480));
#pragma unroll
      for (int a = 0; a < kDig; ++a) {
        const int b = kDig - 1 - a;      // byte of X + kOff
        const uint32_t sel = (uint32_t)(b & 3) | ((uint32_t)(4 + (b & 3)) << 8);
        uint32_t wd[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const uint32_t pr = b >= 4 ? __byte_perm(rhi[u], ihi[u], sel)
                                     : __byte_perm(rlo[u], ilo[u], sel);
          const uint32_t bits = (pr & 0x00ff00ffu) | 0x64006400u;
          const __half2 d = __hsub2(*reinterpret_cast<const __half2*>(&bits), bias);
          wd[u] = *reinterpret_cast<const uint32_t*>(&d);
        }
        *reinterpret_cast<uint4*>(sm + kSmA + a * kAPlane + off) = make_uint4(wd[0], wd[1], wd[2], wd[3]);
      }
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    // 4. one thread issues the products, K steps of 16 reals (256 bytes). One MMA multiplies digit a
    //    of the sequences by several consecutive digit planes b of the DFT matrix at once (N = 64
    //    per plane, the planes lie one after another): its output for plane b lands 64 b columns
    //    after its start, so starting at diagonal a puts every product on its diagonal a + b.
    //    Planes b <= min(6, 7 - a) are used, as two MMAs (b < 4 and b >= 4); the first K step's
    //    MMAs of digit 0 overwrite diagonals 0-6 and a product with a zero A clears diagonal 7,
    //    so everything after accumulates.
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;");
      const uint64_t zd = mat_desc(sbase + kSmZero);
      mma_f16(tbase + 7 * kKr, zd, mat_desc(sbase + kSmB), idesc_n(kKr), 0u);
#pragma unroll 1
      for (int ks = 0; ks < kKr / 16; ++ks)
#pragma unroll
        for (int a = 0; a < kDig; ++a) {
          const uint64_t ad = mat_desc(sbase + kSmA + a * kAPlane + ks * 256);
          const int nb1 = min(4, kDiag - a), nb2 = max(0, min(kDig - 1, kDiag - 1 - a) - 3);
          const uint32_t acc = (ks > 0 || a > 0) ? 1u : 0u;
          mma_f16(tbase + (uint32_t)(a * kKr), ad, mat_desc(sbase + kSmB + ks * 256), idesc_n(kKr * nb1), acc);
          if (nb2 > 0)
            mma_f16(tbase + (uint32_t)((a + 4) * kKr), ad, mat_desc(sbase + kSmB + 4 * kBPlane + ks * 256),
                    idesc_n(kKr * nb2), acc);
        }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar_m)
                   : "memory");
    }
    // 5. the next tile's loads go out while the products run
    const int64_t next = tile + gridDim.x;
    if (next < ntiles) {
      int64_t ncol;
      uint32_t ng, np, nib;
      seq_of(next, ncol, ng, np, nib);
      load_inputs(v, src, hmul, nseg, gen, logF, logS, ncol, nib, e0, es);
    }
    if (__syncthreads_or(!bar_wait(bar_m, phase, t0) ? 1 : 0)) {
      s_fail = 1;
      break;
    }
    phase ^= 1u;
    asm volatile("tcgen05.fence::after_thread_sync;");
    // 6. read back: lane i (warp quarter warp & 3), columns 16 qd .. 16 qd + 15 of every diagonal;
    //    y = Y 2^(E - 55), applied to the exponent field of the converted Y
    const uint32_t lane_addr = tbase + ((uint32_t)(32 * (warp & 3)) << 16);
    // 2^(E - 55) goes into the exponent field of the converted Y while the result stays a normal
    // number (every realistic input); a warp with a sequence outside that range multiplies instead
    const bool wide_range = __any_sync(0xffffffffu, E - 55 < -900 || E - 55 > 900);
    const double scale2 = wide_range ? ldexp(1.0, E - 55) : 1.0;
    double2* y = dst + (col << logF) + g;
    // R64: the exchange of Z0 and W_64^r Z1 (int64 pairs) at [r][row] of the digit area, which
    // the finished products no longer read
    longlong2* xch = reinterpret_cast<longlong2*>(sm + kSmA);
#pragma unroll 1
    for (int c8 = 0; c8 < 2; ++c8) {
      uint32_t d[kDiag][8];
#pragma unroll
      for (int s = 0; s < kDiag; ++s) tmem_ld8(lane_addr + (uint32_t)(s * kKr + 16 * qd + 8 * c8), d[s]);
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
      long long Ys[8];
#pragma unroll
      for (int n = 0; n < 8; ++n) {
        // diagonals 0-3 hold at most 1, 2, 3, 4 x 2^20 in size: adding 1.5 2^23 puts the integer in
        // the low mantissa bits exactly (|x| <= 2^22); the larger ones convert on the F2I path
        int D[kDiag];
#pragma unroll
        for (int s = 0; s < 4; ++s) D[s] = __float_as_int(__uint_as_float(d[s][n]) + 12582912.0f) - 0x4B400000;
#pragma unroll
        for (int s = 4; s < kDiag; ++s) D[s] = __float2int_rn(__uint_as_float(d[s][n]));
        // D_6 2^-5 + D_7 2^-13, exact as an integer over 2^13 and rounded to the nearest unit; then
        // D_5..D_2 times 2^3, 2^11, 2^19, 2^27 as 32-bit multiply-adds into the 64-bit sum, and
        // D_1 2^35, D_0 2^43 added to its high word: all modulo 2^64, exact since |Y| < 2^61
        long long Y = ((long long)D[6] * 256 + D[7] + 4096) >> 13;
        Y += (long long)D[5] * 8;
        Y += (long long)D[4] * 2048;
        Y += (long long)D[3] * 524288;
        Y += (long long)D[2] * 134217728;
        const unsigned hi = (unsigned)((unsigned long long)Y >> 32) + ((unsigned)D[1] << 3) + ((unsigned)D[0] << 11);
        Ys[n] = (long long)(((unsigned long long)hi << 32) | ((unsigned long long)Y & 0xFFFFFFFFULL));
      }
      if (R64) {
        // |Z| <= 2^60.5 in units of Y (a sum of 32 inputs of modulus at most sqrt(2) 2^E): the odd
        // rows rotate by W_64^r in three products of (Z shifted by 1) with the Q62 twiddle
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int r = 8 * qd + 4 * c8 + u;
          long long zr = Ys[2 * u], zi = Ys[2 * u + 1];
          if (par) {
            const longlong2 w = __ldg(&twq[(uint32_t)r << (logF - 6)]);  // W_64^r = W_F^{r F / 64}
            const long long wi = INV ? -w.y : w.y;
            const long long ar = zr << 1, ai = zi << 1;
            const long long ac = __mul64hi(ar, w.x), bd = __mul64hi(ai, wi);
            const long long im = __mul64hi(ar + ai, w.x + wi) - ac - bd;
            zr = (ac - bd) << 1;
            zi = im << 1;
          }
          xch[r * kRows + i] = make_longlong2(zr, zi);
        }
        continue;
      }
      double o[8];
      if (!wide_range) {
#pragma unroll
        for (int n = 0; n < 8; ++n) {
          const double yd = __ll2double_rn(Ys[n]);  // one rounding; Y = 0 stays 0
          o[n] = Ys[n] ? __longlong_as_double(__double_as_longlong(yd) + ((long long)(E - 55) << 52)) : 0.0;
        }
      } else {
#pragma unroll
        for (int n = 0; n < 8; ++n) o[n] = __ll2double_rn(Ys[n]) * scale2;
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int r = 8 * qd + 4 * c8 + u;  // output r: reals 2r, 2r + 1
        y[(int64_t)r << lgs] = make_double2(o[2 * u], o[2 * u + 1]);
      }
    }
    if (R64) {
      // the radix-2 step: thread (row i, quarter qd) takes outputs r and r + 32 of its sequence for
      // r = 8 qd + 4 (i >> 6) .. + 3
      __syncthreads();
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int r = 8 * qd + 4 * par + u;
        const longlong2 z0 = xch[r * kRows + jrow], z1 = xch[r * kRows + 64 + jrow];
        const long long Ya[4] = {z0.x + z1.x, z0.y + z1.y, z0.x - z1.x, z0.y - z1.y};
        double o[4];
#pragma unroll
        for (int n = 0; n < 4; ++n) {
          const double yd = __ll2double_rn(Ya[n]);
          o[n] = wide_range ? yd * scale2
                            : (Ya[n] ? __longlong_as_double(__double_as_longlong(yd) + ((long long)(E - 55) << 52))
                                     : 0.0);
        }
        y[(int64_t)r << lgs] = make_double2(o[0], o[1]);
        y[(int64_t)(r + 32) << lgs] = make_double2(o[2], o[3]);
      }
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
  }
  // teardown: a failed wait may leave a copy or the products in flight; wait for them (bounded)
  // before the TMEM is freed
  if (s_fail) {
    if (tid == 0) atomicOr(err, 1u);
    const long long t1 = clock64();
    bar_wait(bar_b, 0, t1);
    bar_wait(bar_m, phase, t1);
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tbase), "r"(kTmemCols));
}

__global__ void k_twiddles_q62(const double2* __restrict__ tw, longlong2* twq, int64_t n) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x) {
    const double2 w = tw[t];
    twq[t] = make_longlong2(__double2ll_rn(w.x * 0x1p62), __double2ll_rn(w.y * 0x1p62));
  }
}

// fp16 bits of a small integer d (|d| <= 2048).
uint16_t half_bits(int d) {
  if (d == 0) return 0;
  const uint16_t sign = d < 0 ? 0x8000 : 0;
  int m = d < 0 ? -d : d, e = 0;
  while ((m >> e) >= 2) ++e;
  const uint16_t frac = (uint16_t)(((m << (10 - e)) & 0x3ff));
  return (uint16_t)(sign | ((e + 15) << 10) | frac);
}

}  // namespace

void tc_dft_digits(int inverse, void* out) {
  uint16_t* o = reinterpret_cast<uint16_t*>(out);
  const long double pi = 3.141592653589793238462643383279502884L;
  for (int n = 0; n < kKr; ++n)
    for (int k = 0; k < kKr; ++k) {
      const int r = n >> 1, co = n & 1, e = k >> 1, ci = k & 1;
      const int m = (r * e) % kR;
      const long double c = cosl(2 * pi * m / kR), s = sinl(2 * pi * m / kR);
      const long double wr = c, wi = inverse ? s : -s;  // W_32^{r e} (forward) or its conjugate
      // y_re = sum (wr v_re - wi v_im), y_im = sum (wi v_re + wr v_im)
      const long double bv = co == 0 ? (ci == 0 ? wr : -wi) : (ci == 0 ? wi : wr);
      const long long W = llroundl(ldexpl(bv, 54));
      const unsigned long long Y = (unsigned long long)W + kOff;
      for (int a = 0; a < kDig; ++a) {
        const int dgt = (int)((Y >> (8 * (kDig - 1 - a))) & 0xff) - 128;
        o[(a * kBPlane + core_off((uint32_t)n, (uint32_t)k)) / 2] = half_bits(dgt);
      }
    }
}

size_t tc_dft_digits_bytes() { return (size_t)kDig * kBPlane; }

void launch_twiddles_q62(const double2* tw, longlong2* twq, int64_t n, cudaStream_t st) {
  k_twiddles_q62<<<(unsigned)std::min<int64_t>((n + 255) / 256, 152 * 16), 256, 0, st>>>(tw, twq, n);
}

void launch_pass_tc(bool inverse, int logR, const double2* src, double2* dst, int logF, int logS, int ncols,
                    const longlong2* twq, const double2* hmul, int64_t nseg, const FftGen& gen, const void* bdig,
                    unsigned* err, cudaStream_t st) {
  const int64_t ntiles = ((int64_t)ncols << logF) >> (logR == 6 ? 12 : 12);  // 4096 points per tile
  static bool configured[4] = {false, false, false, false};
  const int k = (inverse ? 1 : 0) + (logR == 6 ? 2 : 0);
  if (!configured[k]) {
    if (k == 0) cudaFuncSetAttribute(k_fft_pass_tc<false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmTotal);
    if (k == 1) cudaFuncSetAttribute(k_fft_pass_tc<true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmTotal);
    if (k == 2) cudaFuncSetAttribute(k_fft_pass_tc<false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmTotal);
    if (k == 3) cudaFuncSetAttribute(k_fft_pass_tc<true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmTotal);
    configured[k] = true;
  }
  int dev = 0, sms = 152;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const unsigned grid = (unsigned)std::min<int64_t>(ntiles, sms);
  switch (k) {
    case 0:
      k_fft_pass_tc<false, false><<<grid, kThreads, kSmTotal, st>>>(src, dst, logF, logS, ntiles, twq, hmul, nseg, gen,
                                                                    bdig, err);
      break;
    case 1:
      k_fft_pass_tc<true, false><<<grid, kThreads, kSmTotal, st>>>(src, dst, logF, logS, ntiles, twq, hmul, nseg, gen,
                                                                   bdig, err);
      break;
    case 2:
      k_fft_pass_tc<false, true><<<grid, kThreads, kSmTotal, st>>>(src, dst, logF, logS, ntiles, twq, hmul, nseg, gen,
                                                                   bdig, err);
      break;
    default:
      k_fft_pass_tc<true, true><<<grid, kThreads, kSmTotal, st>>>(src, dst, logF, logS, ntiles, twq, hmul, nseg, gen,
                                                                  bdig, err);
      break;
  }
}

}  // namespace hk
