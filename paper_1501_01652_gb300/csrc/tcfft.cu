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
// as in the FP64 pass). One CTA per SM (persistent; 168 KB of shared memory for the digits, all
// 512 TMEM columns for the 8 diagonal accumulators): per tile of 128 sequences 512 threads
// (sequence i, quarter qd of its elements) write the digits, one thread issues the 45 MMAs, and
// while they run every thread loads the CTA's next tile and brings it to fixed point; after the
// MMAs' commit the threads write the next tile's digits and read back 8 of their sequence's
// outputs. Waits on mbarriers are bounded: a wait that runs out sets the plan's error word and
// the kernel stops, frees its TMEM and returns.
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <algorithm>
#include <atomic>
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
constexpr int kWorkers = 512;   // sequence i = thread % 128, quarter thread / 128
constexpr int kThreads = kWorkers + 32;  // and one warp that issues the products
constexpr uint32_t kAPlane = kRows * kKr * 2;  // 16 KB per digit plane of the sequences
constexpr uint32_t kBPlane = kKr * kKr * 2;    // 8 KB per digit plane of the DFT matrix
constexpr uint32_t kSmA = 0;
constexpr uint32_t kSmB = kSmA + kDig * kAPlane;           // 112 KB
constexpr uint32_t kSmBar = kSmB + kDig * kBPlane;         // 168 KB
constexpr uint32_t kSmSlot = kSmBar + 16;
constexpr uint32_t kSmExp = kSmBar + 32;                   // [4][128] exponents
constexpr uint32_t kSmW = kSmExp + 4 * kRows * 4;          // R64: [2][32] rotations W_64^r (Q62)
constexpr uint32_t kSmTotal = kSmW + 64 * 16;
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

// Barrier of the 512 worker threads (the issuing warp does not take part).
__device__ __forceinline__ void worker_sync() { asm volatile("bar.sync 1, %0;" ::"n"(kWorkers) : "memory"); }

__device__ __forceinline__ void mma_f16(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\ntcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
      "l"(a), "l"(b), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ void tmem_ld(uint32_t taddr, uint32_t (&r)[2]) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x2.b32 {%0,%1}, [%2];" : "=r"(r[0]), "=r"(r[1]) : "r"(taddr));
}

__device__ __forceinline__ void tmem_ld(uint32_t taddr, uint32_t (&r)[4]) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0,%1,%2,%3}, [%4];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
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

// Y 2^sc as a double (one rounding; Y = 0 stays 0) for a normal result: the FP64 pipe's conversion
// and an add to the exponent field.
__device__ __forceinline__ double ll2double_fp(long long Y, int sc) {
  const double yd = __ll2double_rn(Y);
  return Y ? __longlong_as_double(__double_as_longlong(yd) + ((long long)sc << 52)) : 0.0;
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
  // column and group indices are below 2^31: 32-bit divisions (a 64-bit one is a long sequence)
  const uint32_t cc = (uint32_t)col / (uint32_t)g.nsegc;
  const int64_t sg = col - (int64_t)cc * g.nsegc;
  const uint32_t gi = (uint32_t)g.c0 + cc;
  const uint32_t rhs = gi / (uint32_t)g.ncols, li = gi - rhs * (uint32_t)g.ncols;
  const int64_t nlo = sg * g.S;
  GenSrc r;
  r.c = reinterpret_cast<const double*>(g.coef) + rhs * g.ldc + g.n0 - 1 + nlo;
  r.v = reinterpret_cast<const double2*>(g.Vt) + li * g.C + nlo;
  r.lim = min(g.S, g.C - nlo);
  return r;
}

// The rows of a tile. A pass's sequences are g = p s + q of each column c (stride s = 2^logS,
// p < P = F / (R s), q < s): element e of sequence (c, g) is x[c F + q + s (R p + e)], output r goes
// to y[c F + g + (F / R) r]. A tile holds NS = 4096 / R sequences, in one of two tilings:
//  * by columns (kByColumn): NS consecutive sequences of one column, so p varies along the tile
//    when s < NS, and the pass twiddles W_F^{p s e} multiply the inputs;
//  * by twiddle group: NS sequences with one p, the (c, q) pairs u = c s + q in blocks of NS
//    (from NS / s columns when s < NS), tile t = (u-block) P + p. The pass twiddles then depend on
//    e alone and fold into the tile's DFT matrix; a row past the last column loads zeros and
//    stores nothing. The first pass of a transform (s = F / R, p = 0) has no twiddles.
enum PassMode { kNoTwiddle = 0, kByColumn = 1, kByGroup = 2 };

struct TileRow {
  int64_t c;       // column
  uint32_t g;      // sequence within the column
  uint32_t ibase;  // element e at ibase + (e << logS) of the column
  uint32_t p;      // twiddle group
  bool valid;
};

// A thread's inputs of one tile (its sequence's elements e = e0 + j es, j < 8) in two steps, so that
// the loads can go out a tile ahead: prefetch_inputs sends out the loads that are streamed once
// (the column values, or the coefficients of a generated column) into v, and finish_inputs applies
// the first pass's spectrum product or column generation with the tables these share with other
// columns (mostly in L2).
__device__ __forceinline__ void prefetch_inputs(double2 (&v)[8], const double2* __restrict__ src,
                                                const double2* __restrict__ hmul, int64_t nseg, const FftGen& gen,
                                                int logF, int logS, const TileRow& w, int e0, int es) {
  if (!w.valid) {
#pragma unroll
    for (int j = 0; j < 8; ++j) v[j] = make_double2(0.0, 0.0);
  } else if (gen.coef) {
    const GenSrc gs = gen_source(gen, w.c);
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const int64_t t = (int64_t)w.ibase + ((int64_t)(e0 + j * es) << logS);
      v[j].x = t < gs.lim ? __ldg(gs.c + t) : 0.0;
    }
  } else {
    const double2* x = src + ((hmul ? (int64_t)((uint32_t)w.c / (uint32_t)nseg) : w.c) << logF);
#pragma unroll
    for (int j = 0; j < 8; ++j) v[j] = x[w.ibase + ((uint32_t)(e0 + j * es) << logS)];
  }
}

__device__ __forceinline__ void finish_inputs(double2 (&v)[8], const double2* __restrict__ hmul, int64_t nseg,
                                              const FftGen& gen, int logF, int logS, const TileRow& w, int e0,
                                              int es) {
  if (!w.valid) return;
  if (gen.coef) {
    const GenSrc gs = gen_source(gen, w.c);
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const int64_t t = (int64_t)w.ibase + ((int64_t)(e0 + j * es) << logS);
      const double c = v[j].x;  // 0 beyond the column's points
      const double2 tw = t < gs.lim ? __ldg(gs.v + t) : make_double2(0.0, 0.0);
      v[j] = make_double2(c * tw.x, c * tw.y);
    }
  } else if (hmul) {
    const double2* hc = hmul + ((int64_t)((uint32_t)w.c % (uint32_t)nseg) << logF);
#pragma unroll
    for (int j = 0; j < 8; ++j) v[j] = cmul(v[j], __ldg(&hc[w.ibase + ((uint32_t)(e0 + j * es) << logS)]));
  }
}

// Scale and fixed point of one tile's inputs (steps 1 and 2 of a tile): the sequence's scale
// 2^E (largest exponent over its four quarters, and for R64 over both of its rows, before the
// twiddles), X = v 2^(54 - E) in integers, and, when the twiddles multiply the inputs (TWD), X
// times W_F^{p s e} (Q62) with the product rounded back to units of X. All worker threads call it
// (one worker barrier).
template <bool INV, bool R64, bool TWD>
__device__ __forceinline__ int tile_fixed(const double2 (&v)[8], long long (&xr)[8], long long (&xi)[8],
                                          int* emx, int i, int qd, uint32_t p, int logS,
                                          const longlong2* __restrict__ twq, int e0, int es) {
  int m = 1;
#pragma unroll
  for (int j = 0; j < 8; ++j) m = max(m, max(exp_field(v[j].x), exp_field(v[j].y)));
  emx[qd * kRows + i] = m;
  worker_sync();
  int mx = max(max(emx[i], emx[kRows + i]), max(emx[2 * kRows + i], emx[3 * kRows + i]));
  if (R64) {  // both rows of the sequence
    const int o = i ^ 1;
    mx = max(mx, max(max(emx[o], emx[kRows + o]), max(emx[2 * kRows + o], emx[3 * kRows + o])));
  }
  const int E = mx - 1022;
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    xr[j] = to_fixed(v[j].x, E);
    xi[j] = to_fixed(v[j].y, E);
  }
  if (TWD && p != 0) {
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
  return E;
}

// Digits of four pairs (re[u], im[u]) of 54-bit integers, as 8 consecutive fp16 K elements
// (re, im, re, im, ...) of one core-matrix row in every digit plane (base + a pstride + off). Plane
// a holds digit a (weight 256^(6 - a)). The digits of X are the bytes of X + kOff less 128: one
// byte permutation takes byte b of the two parts into the low bytes of the two fp16 halves, whose
// bits 0x6400 + u are 1024 + u, and one packed subtraction of 1152 leaves u - 128.
__device__ __forceinline__ void put_digits(const long long* re, const long long* im, unsigned char* base,
                                           uint32_t off, uint32_t pstride) {
  uint32_t rlo[4], rhi[4], ilo[4], ihi[4];
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const unsigned long long yr = (unsigned long long)re[u] + kOff;
    const unsigned long long yi = (unsigned long long)im[u] + kOff;
    rlo[u] = (uint32_t)yr;
    rhi[u] = (uint32_t)(yr >> 32);
    ilo[u] = (uint32_t)yi;
    ihi[u] = (uint32_t)(yi >> 32);
  }
  const __half2 bias = __half2half2(__ushort_as_half(0x6480));
#pragma unroll
  for (int a = 0; a < kDig; ++a) {
    const int b = kDig - 1 - a;  // byte of X + kOff
    const uint32_t sel = (uint32_t)(b & 3) | ((uint32_t)(4 + (b & 3)) << 8);
    uint32_t wd[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const uint32_t pr = b >= 4 ? __byte_perm(rhi[u], ihi[u], sel) : __byte_perm(rlo[u], ilo[u], sel);
      const uint32_t bits = (pr & 0x00ff00ffu) | 0x64006400u;
      const __half2 d = __hsub2(*reinterpret_cast<const __half2*>(&bits), bias);
      wd[u] = *reinterpret_cast<const uint32_t*>(&d);
    }
    *reinterpret_cast<uint4*>(base + a * pstride + off) = make_uint4(wd[0], wd[1], wd[2], wd[3]);
  }
}

// Step 3: the sequences' digits; this thread writes K columns 16 qd .. 16 qd + 15 of row i (2
// core-matrix rows of 16 bytes per plane).
__device__ __forceinline__ void store_digits(const long long (&xr)[8], const long long (&xi)[8], unsigned char* sm,
                                             int i, int qd) {
#pragma unroll
  for (int c2 = 0; c2 < 2; ++c2)
    put_digits(xr + 4 * c2, xi + 4 * c2, sm + kSmA, core_off((uint32_t)i, (uint32_t)(16 * qd + 8 * c2)), kAPlane);
}

// By twiddle group: the tile's DFT matrix, the real 64 x 64 form of sum_m W_32^{r m} W_F^{sigma p s m}
// (sigma = 1; for R64 the even elements' 32-point DFT, sigma = 2), from the Q62 table: entry
// (r, m) is W_F^{m (r F / 32 + sigma p s)}. Thread tid takes N row n = tid >> 3 (output r = n >> 1,
// real or imaginary part) and K columns 8 (tid & 7) .. + 7 (inputs m = 4 (tid & 7) .. + 3).
template <bool R64>
__device__ __forceinline__ void load_group_twiddles(longlong2 (&w)[4], const longlong2* __restrict__ twq, int logF,
                                                    int logS, uint32_t p, int tid) {
  const uint32_t r = (uint32_t)(tid >> 4), kg = (uint32_t)(tid & 7);
  const uint32_t mask = (1u << logF) - 1u;
  const uint32_t step = (r << (logF - 5)) + ((p << logS) << (R64 ? 1 : 0));
#pragma unroll
  for (int j = 0; j < 4; ++j) w[j] = __ldg(&twq[((4 * kg + (uint32_t)j) * step) & mask]);
}

// The entries' digits (units 2^-54): real output row (co = 0) takes (wr, -wi) for the (real,
// imaginary) input parts, the imaginary row (wi, wr); the inverse conjugates.
template <bool INV>
__device__ __forceinline__ void store_group_digits(const longlong2 (&w)[4], unsigned char* sm, int tid) {
  const int n = tid >> 3, kg = tid & 7, co = n & 1;
  long long re[4], im[4];
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const long long wr = w[j].x, wi = INV ? -w[j].y : w[j].y;
    re[j] = ((co ? wi : wr) + 128) >> 8;
    im[j] = ((co ? wr : -wi) + 128) >> 8;
  }
  put_digits(re, im, sm + kSmB, core_off((uint32_t)n, (uint32_t)(8 * kg)), kBPlane);
}

// Step 4, issued by one thread: the products, K steps of 16 reals (256 bytes). One MMA multiplies
// digit a of the sequences by several consecutive digit planes b of the DFT matrix at once (N = 64
// per plane, the planes lie one after another): its output for plane b lands 64 b columns after
// its start, so starting at diagonal a puts every product on its diagonal a + b. Planes
// b <= min(6, 7 - a) are used, as two MMAs (b < 4 and b >= 4). In the first K step the MMAs of
// digit 0 overwrite diagonals 0-6 and plane 6 of digit 1 overwrites diagonal 7 (its own MMA), so
// every other product accumulates.
__device__ __forceinline__ void issue_products(uint32_t sbase, uint32_t tbase, uint32_t bar_m) {
  asm volatile("tcgen05.fence::after_thread_sync;");
#pragma unroll 1
  for (int ks = 0; ks < kKr / 16; ++ks)
#pragma unroll
    for (int a = 0; a < kDig; ++a) {
      const uint64_t ad = mat_desc(sbase + kSmA + a * kAPlane + ks * 256);
      const int nb1 = min(4, kDiag - a), nb2 = max(0, min(kDig - 1, kDiag - 1 - a) - 3);
      const uint32_t acc = (ks > 0 || a > 0) ? 1u : 0u;
      mma_f16(tbase + (uint32_t)(a * kKr), ad, mat_desc(sbase + kSmB + ks * 256), idesc_n(kKr * nb1), acc);
      if (ks == 0 && a == 1) {
        mma_f16(tbase + 5u * kKr, ad, mat_desc(sbase + kSmB + 4 * kBPlane), idesc_n(2 * kKr), 1u);
        mma_f16(tbase + 7u * kKr, ad, mat_desc(sbase + kSmB + 6 * kBPlane), idesc_n(kKr), 0u);
      } else if (nb2 > 0) {
        mma_f16(tbase + (uint32_t)((a + 4) * kKr), ad, mat_desc(sbase + kSmB + 4 * kBPlane + ks * 256),
                idesc_n(kKr * nb2), acc);
      }
    }
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar_m)
               : "memory");
}

// R64: a radix-64 pass. Each 64-point DFT is two 32-point DFTs, of the even and of the odd
// elements (rows 2j and 2j + 1 of the tile, both scaled by the sequence's 2^E), on the tensor
// cores, and one radix-2 step in 64-bit integers: y_r = Z0_r + W_64^r Z1_r,
// y_{r+32} = Z0_r - W_64^r Z1_r, r < 32. The two rows of a sequence are neighbouring lanes of one
// warp: of the two outputs r of a quarter of the read-back, the even lane takes the first and the
// odd lane the second, each receiving the other row's Z by one lane exchange. By twiddle group,
// the odd elements' extra factor W_F^{p s} joins the rotation: W_F^{r F / 64 + p s}.
//
// Per CTA the tiles form a pipeline. One warp only issues the products (the issue of 45 MMAs
// holds its thread for about as long as they run). While the products of tile t run, the 512
// worker threads bring tile t + 1 (loaded during tile t - 1) to fixed point; once the products
// are done they write tile t + 1's digits (and, by twiddle group, its DFT matrix) over tile t's
// (which the products no longer read), send out the loads of tile t + 2 and read tile t's sums
// out of TMEM.
template <bool INV, bool R64, int MODE>
__global__ void __launch_bounds__(kThreads, 1)
    k_fft_pass_tc(const double2* __restrict__ src, double2* __restrict__ dst, int logF, int logS, int64_t ncols,
                  int64_t ntiles, const longlong2* __restrict__ twq, const double2* __restrict__ hmul, int64_t nseg,
                  FftGen gen, const void* __restrict__ bdig, unsigned* err) {
  extern __shared__ __align__(1024) unsigned char sm[];
  const int tid = threadIdx.x, i = tid & (kRows - 1), qd = (tid >> 7) & 3, warp = tid >> 5;
  const bool worker = tid < kWorkers, issuer = tid == kWorkers;
  const uint32_t sbase = smem_addr(sm);
  const uint32_t bar_b = sbase + kSmBar, bar_m = sbase + kSmBar + 8;
  uint32_t* slot = reinterpret_cast<uint32_t*>(sm + kSmSlot);
  int* emx = reinterpret_cast<int*>(sm + kSmExp);
  longlong2* tw64 = reinterpret_cast<longlong2*>(sm + kSmW);  // [2][32]: by twiddle group, two p
  const long long t0 = clock64();

  constexpr int LR = R64 ? 6 : 5;            // log2 of the radix
  constexpr int LT = R64 ? 6 : 7;            // log2 of the sequences per tile
  const int lgs = logF - LR;                 // log2 of the sequences per column
  const uint32_t smask = (1u << logS) - 1u;
  const int jrow = R64 ? (i >> 1) : i;       // the tile's sequence of this row
  const int par = R64 ? (i & 1) : 0;         // R64: even (0) or odd (1) elements
  const int e0 = R64 ? 16 * qd + par : 8 * qd, es = R64 ? 2 : 1;  // this thread's elements e0 + j es
  const int tpc_log = lgs - LT;              // by columns: log2 of the tiles per column
  const int64_t nu = ncols << logS;          // by twiddle group: the (c, q) pairs per group
  // CTA b takes tiles b, b + grid, ... (the CTAs stream through neighbouring tiles together), except
  // by twiddle group: there it takes the contiguous range [b ntiles / grid, (b + 1) ntiles / grid)
  // in p-major order, t = p ublocks + ub, so that its tiles mostly share p and its DFT matrix is
  // rebuilt only when p changes; Pos walks it without divisions.
  struct Pos {
    uint32_t t, ub, p;  // tiles number below 2^31 (4096 points of 16 bytes each)
  };
  const uint32_t ublocks = (uint32_t)((nu + (int64_t(1) << LT) - 1) >> LT);
  auto advance = [&](Pos x) {
    if (MODE == kByGroup) {
      ++x.t;
      if (++x.ub == ublocks) {
        x.ub = 0;
        ++x.p;
      }
    } else {
      x.t += gridDim.x;
    }
    return x;
  };
  auto row_of = [&](const Pos& x) {
    TileRow w;
    if (MODE == kByColumn) {
      w.c = (int64_t)(x.t >> tpc_log);
      w.g = ((x.t & ((1u << tpc_log) - 1u)) << LT) + (uint32_t)jrow;
      w.p = w.g >> logS;
      w.ibase = (w.g & smask) + ((w.p << LR) << logS);
      w.valid = true;
    } else {
      w.p = MODE == kByGroup ? x.p : 0u;
      const int64_t u = ((int64_t)(MODE == kByGroup ? x.ub : x.t) << LT) + jrow;
      w.valid = u < nu;
      const uint32_t q = (uint32_t)u & smask;
      w.c = w.valid ? (u >> logS) : 0;
      w.g = (w.p << logS) + q;
      w.ibase = q + (w.p << (logS + LR));
    }
    return w;
  };
  const uint32_t t_end =
      MODE == kByGroup ? (uint32_t)(ntiles * (int64_t)(blockIdx.x + 1) / gridDim.x) : (uint32_t)ntiles;
  Pos cur;
  cur.t = MODE == kByGroup ? (uint32_t)(ntiles * (int64_t)blockIdx.x / gridDim.x) : blockIdx.x;
  cur.p = MODE == kByGroup ? cur.t / ublocks : 0u;
  cur.ub = cur.t - cur.p * ublocks;

  if (R64 && tid < 32) {
    // W_64^r = W_F^{r F / 64}; by twiddle group the first tile's W_F^{r F / 64 + p s}
    tw64[tid] = __ldg(&twq[((uint32_t)tid << (logF - 6)) + (cur.p << logS)]);
  }
  if (tid == 0) {
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
  // the DFT matrix digits (without twiddles): one bulk copy into shared memory
  if (issuer && MODE != kByGroup) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar_b), "r"(kDig * kBPlane)
                 : "memory");
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     sbase + kSmB),
                 "l"(bdig), "r"(kDig * kBPlane), "r"(bar_b)
                 : "memory");
  }

  double2 v[8];
  long long xr[8], xi[8];
  int E = 0;
  if (worker) {  // the grid has at most ntiles CTAs: every CTA has a tile
    const TileRow w0 = row_of(cur);
    prefetch_inputs(v, src, hmul, nseg, gen, logF, logS, w0, e0, es);
    finish_inputs(v, hmul, nseg, gen, logF, logS, w0, e0, es);
    E = tile_fixed<INV, R64, MODE == kByColumn>(v, xr, xi, emx, i, qd, w0.p, logS, twq, e0, es);
    if (MODE == kByGroup) {
      longlong2 gw[4];
      load_group_twiddles<R64>(gw, twq, logF, logS, w0.p, tid);
      store_group_digits<INV>(gw, sm, tid);
    }
    const Pos n1 = advance(cur);
    if (n1.t < t_end) prefetch_inputs(v, src, hmul, nseg, gen, logF, logS, row_of(n1), e0, es);
  }
  const bool b_ok = MODE == kByGroup ? true : bar_wait(bar_b, 0, t0);
  if (worker) store_digits(xr, xi, sm, i, qd);
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  asm volatile("tcgen05.fence::before_thread_sync;");
  // the CTA agrees on every failure, so all of it leaves the loop together
  bool stop = __syncthreads_or(b_ok ? 0 : 1) != 0;

  uint32_t phase = 0;
  int bsel = 0;  // R64 by twiddle group: the rotation table of the current tile's p
  for (; cur.t < t_end && !stop; cur = advance(cur)) {
    const Pos nx = advance(cur);
    const bool has_next = nx.t < t_end;  // the same for the whole CTA
    const bool newp = MODE == kByGroup && has_next && nx.p != cur.p;
    bool fail = false;
    if (issuer) issue_products(sbase, tbase, bar_m);
    if (worker) {
      const int Et = E;
      if (has_next) {
        const TileRow wn = row_of(nx);
        finish_inputs(v, hmul, nseg, gen, logF, logS, wn, e0, es);
        E = tile_fixed<INV, R64, MODE == kByColumn>(v, xr, xi, emx, i, qd, wn.p, logS, twq, e0, es);
        if (R64 && newp && tid < 32)
          tw64[32 * (bsel ^ 1) + tid] = __ldg(&twq[((uint32_t)tid << (logF - 6)) + (nx.p << logS)]);
      }
      fail = !bar_wait(bar_m, phase, t0);
      asm volatile("tcgen05.fence::after_thread_sync;");
      // the products no longer read the digit planes: the next tile's digits (and on a new p its
      // DFT matrix) go in, and the loads of the tile after it go out (they land while this tile is
      // read back)
      if (has_next) {
        store_digits(xr, xi, sm, i, qd);
        if (newp) {
          longlong2 gw[4];
          load_group_twiddles<R64>(gw, twq, logF, logS, nx.p, tid);
          store_group_digits<INV>(gw, sm, tid);
        }
        const Pos n2 = advance(nx);
        if (n2.t < t_end) prefetch_inputs(v, src, hmul, nseg, gen, logF, logS, row_of(n2), e0, es);
      }

      const TileRow wt = row_of(cur);
      // read back: lane i (warp quarter warp & 3), columns 16 qd .. 16 qd + 15 of every diagonal, NR
      // at a time (radix 64: the two outputs of a lane pair); y = Y 2^(Et - 55), applied to the
      // exponent field of the converted Y
      const uint32_t lane_addr = tbase + ((uint32_t)(32 * (warp & 3)) << 16);
      // 2^(Et - 55) goes into the exponent field of the converted Y while the result stays a
      // normal number (every realistic input); a warp with a sequence outside that range multiplies
      const bool wide_range = __any_sync(0xffffffffu, Et - 55 < -900 || Et - 55 > 900);
      const double scale2 = wide_range ? ldexp(1.0, Et - 55) : 1.0;
      double2* y = dst + (wt.c << logF) + wt.g;
      const longlong2* rot = tw64 + 32 * bsel;
      constexpr int NR = R64 ? 4 : 2;
#pragma unroll 1
      for (int c4 = 0; c4 < 16 / NR; ++c4) {
        // diagonals 4-7 first, then 0-3 (radix 64 holds four reals' digits in half the registers)
        long long Ys[NR];
        {
          uint32_t d[4][NR];
#pragma unroll
          for (int s = 0; s < 4; ++s) tmem_ld(lane_addr + (uint32_t)((s + 4) * kKr + 16 * qd + NR * c4), d[s]);
          asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
          for (int n = 0; n < NR; ++n) {
            // diagonals 4-7 convert on the F2I path; D_6 2^-5 + D_7 2^-13 is exact as an integer over
            // 2^13 and rounded to the nearest unit; D_5 and D_4 weigh 2^3 and 2^11
            int D[4];
#pragma unroll
            for (int s = 0; s < 4; ++s) D[s] = __float2int_rn(__uint_as_float(d[s][n]));
            long long Y = ((long long)D[2] * 256 + D[3] + 4096) >> 13;
            Y += (long long)D[1] * 8;
            Y += (long long)D[0] * 2048;
            Ys[n] = Y;
          }
        }
        {
          uint32_t d[4][NR];
#pragma unroll
          for (int s = 0; s < 4; ++s) tmem_ld(lane_addr + (uint32_t)(s * kKr + 16 * qd + NR * c4), d[s]);
          asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
          for (int n = 0; n < NR; ++n) {
            // diagonals 0-3 hold at most 1, 2, 3, 4 x 2^20 in size: adding 1.5 2^23 puts the integer
            // in the low mantissa bits exactly (|x| <= 2^22). D_3 and D_2 weigh 2^19 and 2^27 (32-bit
            // multiply-adds into the 64-bit sum), D_1 2^35 and D_0 2^43 are added to its high word:
            // all modulo 2^64, exact since |Y| < 2^61
            int D[4];
#pragma unroll
            for (int s = 0; s < 4; ++s) D[s] = __float_as_int(__uint_as_float(d[s][n]) + 12582912.0f) - 0x4B400000;
            long long Y = Ys[n];
            Y += (long long)D[3] * 524288;
            Y += (long long)D[2] * 134217728;
            const unsigned hi =
                (unsigned)((unsigned long long)Y >> 32) + ((unsigned)D[1] << 3) + ((unsigned)D[0] << 11);
            Ys[n] = (long long)(((unsigned long long)hi << 32) | ((unsigned long long)Y & 0xFFFFFFFFULL));
          }
        }
        if (R64) {
          // the lane pair's outputs r0 = 8 qd + 2 c4 (even lane) and r0 + 1 (odd lane): each lane sends
          // the other's Z and receives its own sequence's other row
          const long long sr = par ? Ys[0] : Ys[NR - 2], si = par ? Ys[1] : Ys[NR - 1];
          const long long rr = __shfl_xor_sync(0xffffffffu, sr, 1), ri = __shfl_xor_sync(0xffffffffu, si, 1);
          const int r = 8 * qd + 2 * c4 + par;
          const long long z0r = par ? rr : Ys[0], z0i = par ? ri : Ys[1];
          const long long z1r = par ? Ys[NR - 2] : rr, z1i = par ? Ys[NR - 1] : ri;
          // |Z| <= 2^60.5 in units of Y (a sum of 32 inputs of modulus at most sqrt(2) 2^E): Z1 rotates
          // by W_64^r (by twiddle group W_F^{r F / 64 + p s}) in three products of (Z1 shifted by 1)
          // with the Q62 twiddle
          const longlong2 w = rot[r];
          const long long wi = INV ? -w.y : w.y;
          const long long ar = z1r << 1, ai = z1i << 1;
          const long long ac = __mul64hi(ar, w.x), bd = __mul64hi(ai, wi);
          const long long tr = (ac - bd) << 1, ti = (__mul64hi(ar + ai, w.x + wi) - ac - bd) << 1;
          const long long Ya[4] = {z0r + tr, z0i + ti, z0r - tr, z0i - ti};
          double o[4];
#pragma unroll
          for (int n = 0; n < 4; ++n) o[n] = wide_range ? __ll2double_rn(Ya[n]) * scale2 : ll2double_fp(Ya[n], Et - 55);
          if (wt.valid) {
            y[(int64_t)r << lgs] = make_double2(o[0], o[1]);
            y[(int64_t)(r + 32) << lgs] = make_double2(o[2], o[3]);
          }
          continue;
        }
        double o[NR];
        if (!wide_range) {
#pragma unroll
          for (int n = 0; n < NR; ++n) o[n] = ll2double_fp(Ys[n], Et - 55);
        } else {
#pragma unroll
          for (int n = 0; n < NR; ++n) o[n] = __ll2double_rn(Ys[n]) * scale2;
        }
#pragma unroll
        for (int u = 0; u < NR / 2; ++u) {
          const int r = 8 * qd + (NR / 2) * c4 + u;  // output r: reals 2r, 2r + 1
          if (wt.valid) y[(int64_t)r << lgs] = make_double2(o[2 * u], o[2 * u + 1]);
        }
      }
      // the next tile's digits to the tensor cores' view
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    // TMEM free for the next products
    asm volatile("tcgen05.fence::before_thread_sync;");
    stop = __syncthreads_or(fail ? 1 : 0) != 0;
    if (stop) break;
    phase ^= 1u;
    if (newp) bsel ^= 1;
  }
  // teardown: a failed wait may leave a copy or the products in flight; wait for them (bounded)
  // before the TMEM is freed
  if (stop) {
    if (tid == 0) atomicOr(err, 1u);
    const long long t1 = clock64();
    if (MODE != kByGroup) bar_wait(bar_b, 0, t1);
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
  if (ncols <= 0) return;
  using Kern = void (*)(const double2*, double2*, int, int, int64_t, int64_t, const longlong2*, const double2*,
                        int64_t, FftGen, const void*, unsigned*);
  static const Kern kern[12] = {
      k_fft_pass_tc<false, false, kNoTwiddle>, k_fft_pass_tc<true, false, kNoTwiddle>,
      k_fft_pass_tc<false, true, kNoTwiddle>,  k_fft_pass_tc<true, true, kNoTwiddle>,
      k_fft_pass_tc<false, false, kByColumn>,  k_fft_pass_tc<true, false, kByColumn>,
      k_fft_pass_tc<false, true, kByColumn>,   k_fft_pass_tc<true, true, kByColumn>,
      k_fft_pass_tc<false, false, kByGroup>,   k_fft_pass_tc<true, false, kByGroup>,
      k_fft_pass_tc<false, true, kByGroup>,    k_fft_pass_tc<true, true, kByGroup>};
  // the tiling: the first pass of a transform (stride F / R) has no twiddles; the others go by
  // twiddle group when its tiles are at least 7/8 full and a row's outputs come in runs of at
  // least 32 bytes (s >= 2; at s = 1 the rows of a group tile write 16 bytes to each of 64 or 128
  // columns), else by columns
  const int LT = logR == 6 ? 6 : 7;
  const int logP = logF - logR - logS;
  const int64_t nu = (int64_t)ncols << logS, ublocks = (nu + (int64_t(1) << LT) - 1) >> LT;
  int mode = kNoTwiddle;
  if (logP > 0) mode = logS >= 1 && (ublocks << LT) - nu <= (ublocks << LT) / 8 ? kByGroup : kByColumn;
  const int64_t ntiles = mode == kByColumn ? (((int64_t)ncols << logF) >> 12) : (ublocks << logP);  // (below 2^31: a tile is 4096 points of 16 bytes, far more than any device holds)
  const int k = (inverse ? 1 : 0) + (logR == 6 ? 2 : 0) + 4 * mode;
  int dev = 0, sms = 152;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  // the shared-memory opt-in, once per device and kernel
  static std::atomic<unsigned> configured[64];
  const unsigned bit = 1u << k;
  if (dev >= 64 || !(configured[dev].load(std::memory_order_relaxed) & bit)) {
    cudaFuncSetAttribute(kern[k], cudaFuncAttributeMaxDynamicSharedMemorySize, kSmTotal);
    if (dev < 64) configured[dev].fetch_or(bit, std::memory_order_relaxed);
  }
  const unsigned grid = (unsigned)std::min<int64_t>(ntiles, sms);
  kern[k]<<<grid, kThreads, kSmTotal, st>>>(src, dst, logF, logS, ncols, ntiles, twq, hmul, nseg, gen, bdig, err);
}

}  // namespace hk
