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

// Near-field work item: row k, columns n0..n1 (1-based, inclusive; empty when n0 > n1).
// slot < 0: the item is the whole prefix of its row and writes f directly.
struct NearItem {
  int64_t k, n0, n1, slot;
};
// A row whose near prefix is split into npieces items with partial slots slot0.. .
struct NearRow {
  int64_t k, slot0;
  int32_t npieces, pad;
};

struct ChirpGeom {
  int64_t Ua, Ub, Va, Vb, E, k0, n0, R, C, F;
};

struct GenArgs {
  double2* A;         // [nc * nsegc][F] output columns
  int64_t F, C, n0;   // transform length, block columns, first column (1-based)
  int64_t S;          // columns per segment (C when the columns are not segmented)
  int64_t nsegc;      // column segments per stacked column (1 when not segmented)
  int nc;             // columns in this chunk
  int64_t c0;         // global index of the first column (rhs * ncols + l)
  int ncols;          // stacked columns per right-hand side
  const double* c;    // coefficients, c[rhs * ldc + n-1]
  int64_t ldc;
  NodeTables nodes;
  const DevColSpec* cols;
  const double2* wV;  // column chirp of the block
  const double2* T;   // optional [ncols][N] column factors times the column chirp (nullptr: computed here)
  int64_t N;
};

struct OutArgs {
  const double2* Y;   // [nc * nsegr][F] inverse-transformed columns
  int64_t F, R, k0;
  int64_t off;        // index of output row k0 in a transformed column (convolution offset)
  int64_t Sr;         // rows per row segment (R when the rows are not segmented)
  int64_t nsegr;      // row segments per stacked column
  int nc;
  int64_t c0;
  int ncols;
  double* f;          // f[rhs * ldf + k-1] += ...
  int64_t ldf;
  NodeTables nodes;
  const DevColSpec* cols;
  const double2* wU;  // row chirp of the block
  const double* W;    // optional [ncols][N] row factors (nullptr: computed here)
  int64_t N;
};

// Plan-time tables of the factors that do not depend on c:
// T[l][n-1] = colpow^u1 omt^(delta-1/2) poly_l(beta) exp(i pi V_n^2/(2E)),
// W[l][k-1] = rowpert^u1 rowvar^(delta-1/2).
struct TabArgs {
  double2* T;
  double* W;
  int64_t N;
  int ncols;
  NodeTables nodes;
  const DevColSpec* cols;
  int64_t Va, Vb, E;
};
void launch_build_tables(const TabArgs& a, cudaStream_t st);

// Convolution kernels of the segments of a block: for y < nseg and t < F,
// hh[y*F + t] = exp(-i pi D^2 / (2E)), D = Ua (t - (Cc-1) + (k0 + y dk) - (n0 + y dn)) + Ub - Vb
// for t < Rr + Cc - 1, and 0 beyond.
struct SegGeom {
  int64_t Ua, Ub, Vb, E, k0, n0, Rr, Cc, dk, dn, nseg, F;
};

void launch_twiddles(double2* tw, int logF, cudaStream_t st);
void launch_chirps(const ChirpGeom& g, double2* wU, double2* wV, cudaStream_t st);
void launch_seg_hh(const SegGeom& g, double2* hh, cudaStream_t st);
// out[cc][t] = sum_s in[cc*nseg + s][t] * H[s][t]   (overlap-add of column segments)
void launch_seg_mac(const double2* in, const double2* H, double2* out, int64_t F, int64_t nseg, int nc,
                    cudaStream_t st);
// out[cc*nseg + s][t] = in[cc][t] * H[s][t]         (overlap-save of row segments)
void launch_seg_expand(const double2* in, const double2* H, double2* out, int64_t F, int64_t nseg, int nc,
                       cudaStream_t st);
// Out-of-place multi-column FFT of length 2^logF over ncols contiguous columns,
// ping-ponging between a (input) and b; *result receives the buffer holding the output.
int run_fft(double2* a, double2* b, int logF, int ncols, bool inverse, const double2* tw, int logFmax,
            cudaStream_t st, double2** result, int* npasses = nullptr);
void launch_scale_copy(const double2* src, double2* dst, int64_t n, double scale, cudaStream_t st);
void launch_pointwise(double2* y, const double2* H, int64_t F, int ncols, cudaStream_t st);
void launch_gen(const GenArgs& a, cudaStream_t st);
void launch_out(const OutArgs& a, cudaStream_t st);
void launch_near(const NearItem* items, int64_t nitems, const NearRow* mrows, int64_t nmrows, double* partial,
                 int nrhs, const double* c, int64_t ldc, double* f, int64_t ldf, const NodeTables& nodes,
                 const double* jtab, int64_t jt_n, int deg, cudaStream_t st);

}  // namespace hk
