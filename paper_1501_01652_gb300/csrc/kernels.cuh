// Kernel-side structures and launch wrappers of the transform.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "plan.h"

namespace hk {

// exp(i pi q / (2E)) for q = v^2 mod 4E (the period of the phase in v^2): the chirp
// factors of the exact phase pi U V / E, reduced in integers before sincospi.
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

// Per-index node tables on the device (0-based index i = k-1 or n-1).
struct NodeTables {
  double* r_true;     // r_k
  double* om_true;    // omega_n
  double* rowvar;     // r_k (Schlomilch, Fourier-Bessel) or r~_k (DHT)
  double* rs_rowvar;  // rowvar^{-1/2}
  double* inv_rowvar; // rowvar^{-1}
  double* rowpert;    // e_k (DHT)
  double* omt;        // omega~_n
  double* rs_omt;     // omega~_n^{-1/2}
  double* inv_omt;    // omega~_n^{-1}
  double* betan;      // b_n / omega~_n
  double* colpow;     // j_{0,n} (DHT)
};

// One stacked column: row factor rowpert^u1 rowvar^(delta-1/2), column factor
// colpow^u1 omt^(delta-1/2) sum_u2 G[u2] betan^u2.
struct DevColSpec {
  int u1, delta, nterm, pad;
  double2 G[kMaxU];
};

// A near-field tile: rows k0..k0+31 (one lane each) over columns n0..n1, each lane stopping at
// its row's prefix end. slot < 0: the tile covers the group's whole prefix and writes f;
// otherwise lane j writes its sum for vector r to partial[(slot + j ntile) nrhs + r ntile + t]
// (the pieces of one row and vector are consecutive).
struct NearItem {
  int64_t k0, n0, n1, slot;
  int32_t ntile, t;
};
// A row whose near prefix is split into npieces tiles with partial slots slot0.. .
struct NearRow {
  int64_t k, slot0;
  int32_t npieces, pad;
};
constexpr int kNearRows = 32;    // rows per tile (one warp)
constexpr int64_t kNearCols = 512;  // columns per tile

struct ChirpGeom {
  int64_t Ua, Ub, Va, Vb, E, k0, n0, R, C, F;
};

// Row accumulation of one chunk: f_k += Re[ sum_li Ut[li][k - k0] y_li(k) ] (the row chirp w_U(k)
// is folded into Ut).
struct OutArgs {
  const void* Y;      // [nc * nsegr][F] inverse-transformed columns (double2 or float2)
  int64_t F, R, k0;
  int64_t off;        // index of output row k0 in a transformed column (convolution offset)
  int64_t Sr;         // rows per row segment (R when the rows are not segmented)
  int64_t nsegr;      // row segments per stacked column
  int nc;
  int64_t c0;
  int ncols;          // stacked columns (transforms) of the block per right-hand side
  double* f;          // f[rhs * ldf + k-1] += ...
  int64_t ldf;
  const void* Ut;     // [ncols][R] block row table times the row chirp (double2, df64c or float2)
  const int* cexp;    // FP32 and double-float groups: the columns were generated from coefficients scaled by
                      // 2^-cexp[rhs], so the row sums are scaled back by 2^cexp[rhs] (nullptr: FP64 groups)
};

// Plan-time block tables (computed in FP64, stored in the plan precision). For a block with a
// low-rank form, column li is V_li (the Chebyshev series vcheb[li] in the variable of log n on
// [log n0, log n1]) and row li is U_li (ucheb[li] in log k); otherwise column li is the stacked
// column lmap[li]:
// colpow^u1 omt^(delta-1/2) poly(beta) and row li its rowpert^u1 rowvar^(delta-1/2).
// Vt[li][np] = V_li(n0+np) wV[np] scale[li], Ut[li][kp] = U_li(k0+kp) wU[kp] / scale[li].
struct BlockTabArgs {
  int nl;
  int64_t k0, R, n0, C;
  const int* lmap;       // direct form: the stacked column of each li
  int P;                 // low-rank form: Chebyshev points (0: direct form)
  const double2* ucheb;  // [nl][P] Chebyshev coefficients of U_li
  const double2* vcheb;  // [nl][P] Chebyshev coefficients of V_li
  double lk0, lk1, ln0, ln1;  // log k0, log k1, log n0, log n1
  NodeTables nodes;
  const DevColSpec* cols;
  const double2* wV;
  const double2* wU;
  const double* scale;   // per li (nullptr: 1)
  void* Vt;
  void* Ut;
};
template <class C>
void launch_block_tables(const BlockTabArgs& a, cudaStream_t st);
// out[r * ldo + i] = scale * v[i] * x[r * ldx + i] for r < nrhs, i < N (out may be x).
void launch_diag_scale(const double* x, int64_t ldx, const double* v, double scale, double* out, int64_t ldo,
                       int64_t N, int nrhs, cudaStream_t st);
// f[r * ldf + i] += acc[0][r * N + i] (+ acc[1][r * N + i]) for r < nrhs, i < N, nacc <= 2.
void launch_add_lanes(double* f, int64_t ldf, const double* const* acc, int nacc, int64_t N, int nrhs,
                      cudaStream_t st);
// Per vector r < nrhs: cexp[r] = E - 1022, E the largest biased FP64 exponent of c[r * ldc + i], i < N
// (E = 0 for a vector of zeros and subnormals), so that |c| 2^-cexp[r] < 1 for every entry. The
// transform is linear, so the FP32 and double-float stages run on the coefficients scaled by that
// power of two (exactly) and scale their sums back: their range then does not depend on the input's.
void launch_coef_exponent(const double* c, int64_t ldc, int64_t N, int nrhs, int* cexp, cudaStream_t st);
// Seeded values in [-1/2, 1/2) over `words` 4-byte words: floats (as_float) or doubles.
void launch_fill_pattern(void* p, size_t words, int as_float, cudaStream_t st);
// cf[r * N + i] = (float) (c[r * ldc + i] 2^-cexp[r]) for r < nrhs, i < N.
void launch_coeffs_f32(const double* c, int64_t ldc, float* cf, int64_t N, int nrhs, const int* cexp,
                       cudaStream_t st);
// cd[r * N + i] = (h, l): x = c[r * ldc + i] 2^-cexp[r], h = (float) x, l = (float)(x - h), for r < nrhs, i < N.
void launch_coeffs_df64(const double* c, int64_t ldc, float2* cd, int64_t N, int nrhs, const int* cexp,
                        cudaStream_t st);

// Convolution kernels of the segments of a block: for y < nseg and t < F,
// hh[y*F + t] = exp(-i pi D^2 / (2E)), D = Ua (t - (Cc-1) + (k0 + y dk) - (n0 + y dn)) + Ub - Vb
// for t < Rr + Cc - 1, and 0 beyond.
struct SegGeom {
  int64_t Ua, Ub, Vb, E, k0, n0, Rr, Cc, dk, dn, nseg, F;
};

void launch_twiddles(double2* tw, int logF, cudaStream_t st);
void launch_chirps(const ChirpGeom& g, double2* wU, double2* wV, cudaStream_t st);
void launch_seg_hh(const SegGeom& g, double2* hh, cudaStream_t st);
// Far-field column generation fused into the first loads of a forward transform: column y of the
// chunk is segment sg = y % nsegc of stacked column g = c0 + y / nsegc (right-hand side
// g / ncols, table row li = g % ncols), and its point t < F is
//   coef[rhs * ldc + n0 - 1 + sg S + t] * Vt[li][sg S + t]   for t < min(S, C - sg S), else 0.
// coef holds double (FP64 plans), float (FP32) or (high, low) float pairs (DF64) coefficients.
struct FftShape {
  int one_launch;  // 1: the whole transform in one launch (2^6 .. 2^12 points)
  int npass;       // otherwise passes of radix 2^logr[i], first to last
  int logr[4];
  int tc;          // bit i: pass i (radix 32 or 64, FP64 transforms of 2^12 or more points) runs on the tensor cores
};

// Tables of the tensor-core passes (tcfft.cu): the digit planes of the 32-point DFT matrix,
// forward and inverse, in their shared-memory layout, and the plan's device error word.
struct TcTables {
  const void* fwd;
  const void* inv;
  unsigned* err;
  const longlong2* twq;  // the twiddle ladder in Q62 integers (W_F^t at twq[F + t])
};
struct FftGen {
  int64_t nsegc, S, C, n0;
  int64_t c0;
  int64_t ncols;
  const void* coef;
  int64_t ldc;
  const void* Vt;
};
// Digit planes of the real 64 x 64 form of the 32-point DFT matrix (inverse: conjugated), written
// into out (tc_dft_digits_bytes() bytes), host side.
void tc_dft_digits(int inverse, void* out);
size_t tc_dft_digits_bytes();
// One Stockham pass of radix 2^logR (5 or 6) of 2^logF-point FP64 transforms (logF >= 12) over ncols
// columns on the tensor cores: the mapping of k_fft_pass_reg<logR>, with hmul or gen on its loads as there
// (first passes only); twq is the Q62 twiddle table of this length (W_F^t at twq[t]).
void launch_pass_tc(bool inverse, int logR, const double2* src, double2* dst, int logF, int logS, int ncols,
                    const longlong2* twq, const double2* hmul, int64_t nseg, const FftGen& gen, const void* bdig,
                    unsigned* err, cudaStream_t st);
// twq[t] = round(tw[t] 2^62) (both parts), t < n.
void launch_twiddles_q62(const double2* tw, longlong2* twq, int64_t n, cudaStream_t st);


// Out-of-place multi-column FFT of length 2^logF over ncols contiguous columns,
// ping-ponging between a (input) and b; *result receives the buffer holding the output.
// C is double2 (FP64) or float2 (FP32); tw is the matching twiddle ladder (W_F^t at tw[F + t]
// for every power of two F = 2^6 .. 2^logFmax).
// With hmul, column j transforms a[j / nseg] times hmul[j % nseg] elementwise (a holds
// ncols / nseg columns; the products of the chirp spectra are folded into the first loads).
// With gen (forward transforms only), the input columns are generated by the first loads as
// FftGen describes and a is used only as workspace.
// shape: how the transform is split into launches (one launch of k_fft_small, or passes of the
// listed radices); nullptr takes default_fft_shape.
template <class C>
int run_fft(C* a, C* b, int logF, int ncols, bool inverse, const C* tw, int logFmax, cudaStream_t st, C** result,
            int* npasses = nullptr, const C* hmul = nullptr, int64_t nseg = 1, const FftGen* gen = nullptr,
            const FftShape* shape = nullptr, const TcTables* tc = nullptr);
// The built-in choice for a transform of 2^logF points over ncols columns in precision prec
// (kTermFP64, kTermDF64, kTermFP32): one launch up to 4096 points unless that gives fewer CTAs
// than SMs; otherwise the fewest passes of radix 2^5 .. 2^8 (2^6 for double-float), as equal
// as possible, the larger first.
FftShape default_fft_shape(int logF, int ncols, int prec);
// Whether shape is a valid split of 2^logF points (passes of radix 2^5 .. 2^8 summing to logF,
// or one launch for logF <= 12; tensor-core passes only of radix 32 with logF >= 12).
bool valid_fft_shape(const FftShape& shape, int logF);
// out[cc][t] = sum_s in[cc*nseg + s][t] * H[s][t]   (overlap-add of column segments)
template <class C>
void launch_seg_mac(const C* in, const C* H, C* out, int64_t F, int64_t nseg, int nc, cudaStream_t st);
template <class C>
void launch_scale_copy(const double2* src, C* dst, int64_t n, double scale, cudaStream_t st);
template <class C>
void launch_out(const OutArgs& a, cudaStream_t st);
// Near field in FP64 (R = double: r, omega, jtab from the FP64 tables) or FP32 (R = float:
// rf, omf, jtabf single-precision copies); sums are accumulated in R, outputs written as double.
template <class R>
// cf: optional coefficients already rounded to FP32 ([nrhs][N]); used instead of c when given.
// jtabq: the J table in Q62 fixed point; FP64 near fields (R = double) evaluate J from it on
// the integer pipe, FP32 ones (R = float, jtabq unused) from jtab.
// cexp: with cf, the exponents of its scaling (launch_coef_exponent), applied to the sums.
void launch_near(const NearItem* items, int64_t nitems, const NearRow* mrows, int64_t nmrows, const int64_t* nend,
                 int64_t N, R* partial, int nrhs, const double* c, int64_t ldc, const float* cf, double* f,
                 int64_t ldf, const R* r, const R* om, const R* jtab, const long long* jtabq, int64_t jt_n, int deg,
                 const int* cexp, cudaStream_t st);

// Near field with the per-vector products as exact split-digit fp16 tensor-core products
// (8 <= nrhs <= 16), FP64 and double-float plans: z = r_n om_n in FP64, J from the Q62
// fixed-point table jtabq on the integer pipe. Cd holds 8 x 16 x Npad fp16 digits and Ce
// (Npad / 512) x 16 exponents, both written here from c (Npad = N rounded up to a multiple of 512).
constexpr int kNearTcMinRhs = 8;
constexpr int kNearTcRhs = 16;  // vectors per tensor-core near-field launch
// df: a DF64 plan (7 digits and 7 diagonals: products to about 2^-46 of the chunk scale).
void launch_near_tc(bool df, const NearItem* items, int64_t nitems, const NearRow* mrows, int64_t nmrows,
                    const int64_t* nend, int64_t N, double* partial, int nrhs, const double* c, int64_t ldc, void* Cd,
                    int* Ce, int64_t Npad, double* f, int64_t ldf, const double* r, const double* om,
                    const long long* jtabq, int64_t jt_n, int deg, cudaStream_t st);
// Near field of DF64 plans in double-float on the FP32 pipe: r, om and jtab hold (high, low)
// float pairs of the FP64 tables, cd the coefficients as pairs ([nrhs][N]) scaled by 2^-cexp[r];
// partial sums and outputs are FP64, scaled back.
void launch_near_df(const NearItem* items, int64_t nitems, const NearRow* mrows, int64_t nmrows,
                    const int64_t* nend, int64_t N, double* partial, int nrhs, const float2* cd, double* f,
                    int64_t ldf, const float2* r, const float2* om, const float2* jtab, int64_t jt_n, int deg,
                    const int* cexp, cudaStream_t st);

}  // namespace hk
