// Internal plan structures shared by the host planner and the CUDA side.
#pragma once
#include <stdint.h>

#include <complex>
#include <vector>

#include "hankel.h"

namespace hk {

typedef std::complex<double> cplx;

// Largest number of Taylor powers u2 of the column perturbation b_n carried
// by one stacked column (2T+K-2 of Section 5.1 at eps = 1e-16 is 10).
constexpr int kMaxU = 16;
// Near-field Bessel table: 64 Taylor intervals per unit of z, so that degree 6 (eps = 1e-15) or 4
// (1e-8) suffices; 128 would leave the double-float lookup, whose interval offset is formed in
// float, short of its accuracy at z near 100.
constexpr int kJTabLog = 6;                 // near-field J table: 2^kJTabLog Taylor intervals
constexpr int kJTabSub = 1 << kJTabLog;     // per unit of z
constexpr int kJTabDegMax = 10;  // largest Taylor degree of the near-field J table

// How a block's chirp-z convolution is carried out.
enum BlockMode {
  kBlockFull = 0,    // one transform of length F >= R + C - 1
  kBlockRowSeg = 1,  // few rows: columns cut into nseg segments of S, overlap-add, F >= R + S - 1
  kBlockColSeg = 2   // few columns: rows cut into nseg segments of S, overlap-save, F >= S + C - 1
};

// A far-field block: rows k0..k1, columns n0..n1 (1-based, inclusive), and its
// chirp-z convolution in transforms of length F = 2^logF.
struct Block {
  int64_t k0, k1, n0, n1;
  int64_t R, C, F;
  int logF;
  int mode;       // BlockMode
  int64_t S;      // segment length (C for full blocks)
  int64_t nseg;   // number of segments (1 for full blocks)
  std::vector<int> lcols;  // stacked columns this block keeps (indices into HostPlan::cols, ascending)
  double dropped = 0.0;    // bound on |entry change| from the stacked columns it leaves out
  // Low-rank form of the block's kernel K(k, n) = sum_{l in lcols} rowfun_l(k) colfun_l(n):
  // K ~ sum_{a < rank} U_a(k) V_a(n), with U_a and V_a given by their values at P Chebyshev
  // points in log k and log n (rank = 0: the block transforms its kept columns).
  int rank = 0;
  int P = 0;
  std::vector<cplx> ucheb, vcheb;  // [rank][P]
  double lowrank_err = 0.0;        // largest error of the low-rank form on the validation entries
  // Precision of each transform (li < rank, or < lcols.size() for direct blocks): kTermFP64,
  // kTermDF64 or kTermFP32.
  std::vector<int8_t> tprec;
};
enum TermPrecision { kTermFP64 = 0, kTermDF64 = 1, kTermFP32 = 2 };

// One stacked column of a block: the row function rowpert(k)^u1 rowvar(k)^(delta-1/2)
// times the column function colpow(n)^u1 omt(n)^(delta-1/2) sum_u2 G[u2] beta(n)^u2.
struct ColSpec {
  int u1;
  int delta;
  int nterm;            // number of u2 terms (U2)
  cplx G[kMaxU];
};

struct HostPlan {
  hankel_options opt;
  // Table 4 and Eqs. (23)-(24)
  int M = 0, K = 1, T = 1, K2 = 1, T2 = 1, U1 = 1, U2 = 1, P = 0, mu_max = 0;
  double s = 0, alpha = 0, beta = 1;
  int64_t nrd = 0, ncd = 0;  // direct rows / columns
  bool fp32 = false;
  bool df64 = false;  // transforms in double-float
  // exact phase theta~_kn = pi U_k V_n / E with U_k = Ua k + Ub, V_n = Va n + Vb
  int64_t Ua = 1, Ub = 0, Va = 1, Vb = 0, E = 1;
  // partition coordinates X_k = k - x0, Y_n = n + y0, z~ = pi X Y / D
  double x0 = 0, y0 = 0, D = 1;
  // nodes, index i = k-1 or n-1
  std::vector<double> b;        // b_n = j_{0,n} - (n-1/4)pi, n = 1..N+1 (FB, DHT)
  std::vector<double> r_true;   // r_k
  std::vector<double> om_true;  // omega_n
  std::vector<double> rowvar;   // r_k (S, FB) or r~_k (DHT)
  std::vector<double> rowpert;  // e_k (DHT), else 0
  std::vector<double> omt;      // omega~_n = omega_n (S) or (n-1/4)pi
  std::vector<double> betan;    // b_n / omega~_n (FB, DHT), else 0
  std::vector<double> colpow;   // j_{0,n} (DHT), else 1
  // partition
  std::vector<Block> blocks;
  std::vector<int64_t> nend;  // near prefix length per row
  int64_t near_count = 0, far_count = 0;
  double zmax = 0;
  // stacked columns per block
  std::vector<ColSpec> cols;
  // near-field J table: jt_n intervals [i/sub, (i+1)/sub), centre (i + 1/2)/sub, deg+1 Taylor
  // coefficients each
  int jt_deg = kJTabDegMax;
  int jt_sub = kJTabSub;
  int64_t jt_n = 0;
  std::vector<double> jtab;
  // the same polynomials in the variable u = sub (z - z_c) in [-1/2, 1/2), as Q62 fixed-point
  // integers: jtabq[i (deg+1) + d] = round(t_d sub^-d 2^62), rounded from the double-double sums
  std::vector<long long> jtabq;
};

// Builds every host table of a plan. Returns a hankel_status code.
int build_host_plan(const hankel_options& opt, HostPlan& hp);
// Parameter selection only (no nodes or tables). Returns a hankel_status code.
int choose_params(const hankel_options& opt, HostPlan& hp);
// Host value of the plan's representation of entry (k, n), 1-based.
double host_entry(const HostPlan& hp, int64_t k, int64_t n, int* is_far);
// Barycentric interpolation at x in [-1, 1] of values at the P Chebyshev points (first kind)
// cos(pi (i + 1/2) / P).
cplx cheb_interp(const cplx* vals, int P, double x);
// Position of index k of the range [k0, k1] on [-1, 1], linear in log k.
double log_coord(double k, int64_t k0, int64_t k1);
// The far-field expansion of entry (k, n) over the listed stacked columns (all when null),
// wherever (k, n) lies.
double expansion_entry(const HostPlan& hp, int64_t k, int64_t n, const std::vector<int>* lcols);
// Near-field J from the Taylor table (host copy of the device evaluator).
double table_j(const HostPlan& hp, double z);
double table_j_q62(const HostPlan& hp, double z);
// j_{0,n} - (n-1/4)pi for n = 1..count.
void j0_zero_offsets(int64_t count, double* b);
// v_n = 2 / J_1(j_{0,n})^2, n = 1..N, from the offsets b_n (Section 6, the self-inverse relation).
void dht_inverse_weights(int64_t N, const double* b, double* v);

}  // namespace hk
