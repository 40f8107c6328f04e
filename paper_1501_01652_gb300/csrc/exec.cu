// Device side of a plan: table upload, chirp spectra, and the execution of
// one transform (near field + far-field blocks) on a CUDA stream.
//
// Far field (Section 4.2, Eq. 19, with Sections 5-6 for Bessel-root nodes):
// every block with rows k0..k1 and columns n0..n1 needs, for each stacked
// column l, Z_l(k) = sum_n exp(i theta~_kn) X_l(n) c_n with the exact phase
// theta~_kn = pi U_k V_n / E. Writing U V = (U^2 + V^2 - (U-V)^2)/2 turns
// that sum into a linear convolution in k - n (a chirp-z transform), done
// with power-of-two FFTs of length F >= R + C - 1.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <mutex>
#include <string>
#include <type_traits>
#include <vector>

#include "device.h"
#include "cplx.cuh"
#include "kernels.cuh"
#include "tune.h"

namespace hk {

namespace {

constexpr size_t kDefaultWorkspace = size_t(4) << 30;

// Complex elements one stacked column occupies in a workspace buffer.
size_t column_footprint(const Block& b) { return (size_t)b.F * (size_t)b.nseg; }

// Element size of a term precision's complex type (double2, df64c, float2).
size_t term_esz(int prec) { return prec == kTermFP32 ? sizeof(float2) : sizeof(double2); }

// The transforms of a block that run in one precision.
struct TermGroup {
  int prec = kTermFP64;  // kTermFP64 (double2), kTermDF64 (df64c) or kTermFP32 (float2)
  int nl = 0;            // transforms per right-hand side
  void* H = nullptr;     // per segment: FFT_F of the chirp exp(-i pi (U-V)^2 / (2E)), times 1/F
  void* Vt = nullptr;    // [nl][C] column functions x column chirp (x FP32 scale)
  void* Ut = nullptr;    // [nl][R] row functions times the row chirp (/ FP32 scale)
  int64_t cap = 0;       // stacked columns per chunk
  FftShape fwd{}, inv{}; // launch split of its forward and inverse transforms (autotuned)
};

struct DevBlock {
  Block b;
  double2* wU = nullptr;  // exp(i pi U_k^2 / (2E)), k = k0..k1
  double2* wV = nullptr;  // exp(i pi V_n^2 / (2E)), n = n0..n1
  TermGroup g[3];         // groups in the order FP64, DF64, FP32
  int ng = 0;
};

// Chebyshev coefficients of the interpolant through the values f_i at cos(pi (i + 1/2) / P):
// a_j = (2 - [j = 0]) / P sum_i f_i cos(pi j (2i + 1) / (2P)). The angle is reduced in integers
// (m = j (2i + 1) mod 4P, then to a quadrant and an angle below pi/2) and the sums are
// compensated (Neumaier), so each coefficient is good to a few units in the last place.
void cheb_coeffs(const cplx* f, int P, double2* a) {
  const double pi = 3.14159265358979323846;
  std::vector<double> cs(4 * (size_t)P);  // cos(pi m / (2P)), m < 4P
  for (int m = 0; m < 4 * P; ++m) {
    const int q = m / P, r = m % P;
    const double th = pi * r / (2.0 * P);
    cs[m] = q == 0 ? std::cos(th) : q == 1 ? -std::sin(th) : q == 2 ? -std::cos(th) : std::sin(th);
  }
  auto add = [](double& sum, double& comp, double x) {
    const double t = sum + x;
    comp += std::fabs(sum) >= std::fabs(x) ? (sum - t) + x : (x - t) + sum;
    sum = t;
  };
  for (int j = 0; j < P; ++j) {
    double sr = 0.0, cr = 0.0, si = 0.0, ci = 0.0;
    for (int i = 0; i < P; ++i) {
      const double c = cs[((int64_t)j * (2 * i + 1)) % (4 * P)];
      add(sr, cr, f[i].real() * c);
      add(si, ci, f[i].imag() * c);
    }
    const double w = (j == 0 ? 1.0 : 2.0) / P;
    a[j] = make_double2(w * (sr + cr), w * (si + ci));
  }
}

// Indices li of the block's transforms per precision.
void term_lists(const Block& b, std::vector<int> (&lists)[3]) {
  for (auto& l : lists) l.clear();
  for (size_t li = 0; li < b.tprec.size(); ++li) lists[b.tprec[li]].push_back((int)li);
}

}  // namespace

struct DevicePlan {
  int device = 0;
  int64_t hpN = 0;
  NodeTables nodes{};
  DevColSpec* cols = nullptr;
  int ncols = 0;
  double* jtab = nullptr;
  bool fp32 = false;
  float* rf = nullptr;     // FP32 plans: r_k, omega_n and the J table in single precision
  float* omf = nullptr;
  float* jtabf = nullptr;
  float2* rdf = nullptr;   // DF64 plans: r_k, omega_n and the J table as (high, low) float pairs
  float2* omdf = nullptr;
  float2* jtabdf = nullptr;
  NearItem* items = nullptr;
  int64_t nitems = 0;
  NearRow* mrows = nullptr;
  int64_t nmrows = 0;
  int64_t* nend = nullptr;  // near prefix end per row
  int64_t nslots = 0;       // near-field partial-sum slots per vector
  std::vector<DevBlock> blocks;
  double2* tw = nullptr;   // twiddle ladder in FP64: W_F^t at tw[F + t], F = 2^6 .. 2^logFmax
  float2* twf = nullptr;   // the same ladder rounded to FP32 (FP32 plans)
  df64c* twd = nullptr;    // the same ladder in double-float (DF64 plans)
  bool df64 = false;       // plan precision double-float (transforms; near field on the FP32 pipe)
  bool any_t[3] = {false, false, false};  // some block has transforms in this precision
  int logFmax = 6;
  size_t ws_bytes = 0;    // workspace (FFT column buffers) of one execution context
  // Lanes: the term groups of one precision run on a stream of their own, so that the FP64,
  // double-float and FP32 transforms (different pipes, many small launches) overlap. Lane 0 is
  // the caller's stream (the near field and the plan precision's groups, adding into f); lane
  // l >= 1 has its own stream, workspace and accumulator acc ([nrhs][N], zeroed per execution),
  // added into f in a fixed order at the end. Stage timing runs the lanes one after another on
  // the caller's stream.
  struct Lane {
    cudaStream_t s = nullptr;
    cudaEvent_t done = nullptr;
    void* A = nullptr;
    void* B = nullptr;
    size_t buf_bytes = 0;
    double* acc = nullptr;
  };
  int nlanes = 1;
  int lane_of[3] = {0, 0, 0};  // lane of each term precision
  size_t lane_bytes[3] = {0, 0, 0};  // one workspace buffer of each lane
  // The scratch of one execution: the lanes' buffers, streams and accumulators, the near-field
  // partial sums and the per-execution coefficient copies. Context 0 is made with the plan;
  // hankel_plan_add_context makes more, so that executions of one plan on different contexts
  // may be in flight at once. The tables above are shared and only read.
  struct ExecCtx {
    Lane lanes[3];
    cudaEvent_t fork = nullptr;
    void* partial = nullptr;  // near-field partial sums (plan precision)
    float* cf = nullptr;      // the scaled coefficients rounded to FP32 [max_nrhs][N]
    float2* cdf = nullptr;    // the scaled coefficients as (high, low) float pairs [max_nrhs][N]
    int* cexp = nullptr;      // with cf or cdf: per vector, the power of two they are scaled by
    void* tcd = nullptr;      // 8+ vectors: coefficient digits of the tensor-core near field
    int* tce = nullptr;       // and their per-chunk exponents
  };
  std::vector<ExecCtx*> ctx;
  size_t ctx_bytes = 0;       // device bytes of one context
  bool want_cf = false, want_cdf = false;
  double* c_stage = nullptr;
  double* f_stage = nullptr;
  double* vinv = nullptr;     // DHT plans, first inverse call: v_n = 2 / J_1(j_{0,n})^2
  double* inv_stage = nullptr;  // v o f for the inverse ([max_nrhs][N])
  int64_t tc_npad = 0;
  long long* jtabq = nullptr;  // the J table in Q62 fixed point (FP64 and DF64 plans)
  size_t bytes = 0;
  std::vector<void*> allocs;
  // stage statistics (hankel_plan_set_timing / hankel_plan_stage_stats)
  bool timing = false;
  hankel_stage_stat acc[HANKEL_STAGE_COUNT] = {};
  struct Rec {
    int stage;
    cudaEvent_t a, b;
  };
  std::vector<Rec> pending;
  std::vector<cudaEvent_t> pool;
  size_t pool_used = 0;
  std::vector<hankel_fft_shape> shapes;  // the transform shapes the plan runs (hankel_plan_fft_shapes)
  // tensor-core FP64 passes: the DFT digit planes (forward, inverse) and the device error word
  void* tcB = nullptr;
  unsigned* tc_err = nullptr;
  TcTables tct{};
  const TcTables* tc() const { return tcB ? &tct : nullptr; }
};

namespace {

// Device address of the static scratch array of hankel_exec_static on `device` (defined below).
int static_scratch_address(int device, double2** out);

template <class T>
int dalloc(DevicePlan* d, T** p, size_t count) {
  *p = nullptr;
  if (count == 0) count = 1;
  void* q = nullptr;
  if (alloc_fault() || cudaMalloc(&q, count * sizeof(T)) != cudaSuccess) {
    cudaGetLastError();
    return HANKEL_ENOMEM;
  }
  d->allocs.push_back(q);
  d->bytes += count * sizeof(T);
  *p = (T*)q;
  return HANKEL_OK;
}

// Releases one allocation made by dalloc with count elements.
template <class T>
void dfree(DevicePlan* d, T** p, size_t count) {
  if (!*p) return;
  for (size_t j = 0; j < d->allocs.size(); ++j)
    if (d->allocs[j] == (void*)*p) {
      cudaFree(*p);
      d->allocs.erase(d->allocs.begin() + (long)j);
      d->bytes -= std::max<size_t>(count, 1) * sizeof(T);
      break;
    }
  *p = nullptr;
}

template <class T>
int upload(DevicePlan* d, T** p, const T* src, size_t count) {
  int st = dalloc(d, p, count);
  if (st != HANKEL_OK) return st;
  if (cudaMemcpy(*p, src, count * sizeof(T), cudaMemcpyHostToDevice) != cudaSuccess) return HANKEL_ECUDA;
  return HANKEL_OK;
}

cudaEvent_t pool_event(DevicePlan* d) {
  if (d->pool_used == d->pool.size()) {
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    d->pool.push_back(e);
  }
  return d->pool[d->pool_used++];
}

// Brackets the launches of one stage with events when timing is on and tallies its work.
struct StageScope {
  DevicePlan* d;
  int stage;
  cudaStream_t st;
  cudaEvent_t a = nullptr;
  bool on;
  StageScope(DevicePlan* d_, int stage_, cudaStream_t st_, bool record = true)
      : d(d_), stage(stage_), st(st_), on(record) {
    if (on && d->timing) {
      a = pool_event(d);
      if (a) cudaEventRecord(a, st);
    }
  }
  void done(int64_t launches, double flops, double entries, double bytes = 0.0) {
    if (!on) return;
    d->acc[stage].launches += launches;
    d->acc[stage].flops += flops;
    d->acc[stage].entries += entries;
    d->acc[stage].bytes += bytes;
    if (d->timing && a) {
      cudaEvent_t b = pool_event(d);
      if (b) {
        cudaEventRecord(b, st);
        d->pending.push_back(DevicePlan::Rec{stage, a, b});
      }
    }
  }
};

#define HK_TRY(x)                        \
  do {                                   \
    int st_ = (x);                       \
    if (st_ != HANKEL_OK) return st_;    \
  } while (0)
#define HK_LAUNCHED()                                              \
  do {                                                             \
    if (cudaGetLastError() != cudaSuccess) return HANKEL_ECUDA;    \
  } while (0)

// One execution context of the plan (DevicePlan::ExecCtx), allocated after the plan's tables and
// lane layout are known; its bytes are tracked with the plan's.
int ctx_create(DevicePlan* d, const HostPlan& hp) {
  DevicePlan::ExecCtx* x = new DevicePlan::ExecCtx();
  d->ctx.push_back(x);
  const size_t before = d->bytes;
  const int64_t N = hp.opt.N;
  const size_t R = (size_t)hp.opt.max_nrhs;
  if (d->want_cdf) HK_TRY(dalloc(d, &x->cdf, R * N));
  if (d->want_cf) HK_TRY(dalloc(d, &x->cf, R * N));
  if (x->cf || x->cdf) HK_TRY(dalloc(d, &x->cexp, R));
  if (d->tc_npad) {
    uint16_t* q = nullptr;
    HK_TRY(dalloc(d, &q, (size_t)8 * kNearTcRhs * d->tc_npad));
    x->tcd = q;
    HK_TRY(dalloc(d, &x->tce, (size_t)(d->tc_npad / 512) * kNearTcRhs));
  }
  const size_t cnt = (size_t)std::max<int64_t>(d->nslots, 1) * R;
  if (d->fp32) {
    float* pf;
    HK_TRY(dalloc(d, &pf, cnt));
    x->partial = pf;
  } else {
    double* pd;
    HK_TRY(dalloc(d, &pd, cnt));
    x->partial = pd;
  }
  for (int l = 0; l < d->nlanes; ++l) {
    char* qa;
    char* qb;
    HK_TRY(dalloc(d, &qa, d->lane_bytes[l]));
    HK_TRY(dalloc(d, &qb, d->lane_bytes[l]));
    x->lanes[l].A = qa;
    x->lanes[l].B = qb;
    x->lanes[l].buf_bytes = d->lane_bytes[l];
    if (l > 0) {
      HK_TRY(dalloc(d, &x->lanes[l].acc, R * N));
      if (cudaStreamCreateWithFlags(&x->lanes[l].s, cudaStreamNonBlocking) != cudaSuccess ||
          cudaEventCreateWithFlags(&x->lanes[l].done, cudaEventDisableTiming) != cudaSuccess)
        return HANKEL_ECUDA;
    }
  }
  if (d->nlanes > 1 && cudaEventCreateWithFlags(&x->fork, cudaEventDisableTiming) != cudaSuccess)
    return HANKEL_ECUDA;
  d->ctx_bytes = d->bytes - before;
  return HANKEL_OK;
}

int public_precision(int t) { return t == kTermFP32 ? HANKEL_PREC_FP32 : t == kTermDF64 ? HANKEL_PREC_DF64 : HANKEL_PREC_FP64; }

// Candidate launch splits of a transform of 2^logF points: the built-in one first, then one
// launch (logF <= 12) and every ordered split into 2..4 passes of radix 2^5 .. 2^8 (2^7 for
// double-float, whose larger passes spill), fewest passes first, at most 24.
std::vector<FftShape> shape_candidates(int logF, int ncols, int prec, bool tc) {
  std::vector<FftShape> out{default_fft_shape(logF, ncols, prec)};
  auto add1 = [&](const FftShape& sh) {
    for (const FftShape& o : out)
      if (o.one_launch == sh.one_launch && o.npass == sh.npass && o.tc == sh.tc &&
          std::equal(o.logr, o.logr + o.npass, sh.logr))
        return;
    if (out.size() < 40 && valid_fft_shape(sh, logF)) out.push_back(sh);
  };
  // FP64 transforms: also the variant with every radix-32 and radix-64 pass on the tensor cores
  // (below 2^12 points, the first pass only)
  auto add = [&](FftShape sh) {
    add1(sh);
    if (tc && prec == kTermFP64 && !sh.one_launch) {
      int m = 0;
      for (int i = 0; i < sh.npass && (logF >= 12 || i == 0); ++i)
        if (sh.logr[i] == 5 || sh.logr[i] == 6) m |= 1 << i;
      if (m) {
        sh.tc = m;
        add1(sh);
      }
    }
  };
  if (logF <= 12) {
    FftShape one{};
    one.one_launch = 1;
    add(one);
  }
  if (out.size() == 1) add(out[0]);  // the default's own tensor-core variant
  const int hi = prec == kTermDF64 ? 7 : 8;
  for (int np = 2; np <= 4; ++np) {
    int r[4] = {5, 5, 5, 5};
    for (;;) {
      int sum = 0;
      for (int i = 0; i < np; ++i) sum += r[i];
      if (sum == logF) {
        FftShape sh{};
        sh.npass = np;
        for (int i = 0; i < np; ++i) sh.logr[i] = r[i];
        add(sh);
      }
      int i = 0;  // next tuple in [5, hi]^np
      while (i < np && r[i] == hi) r[i++] = 5;
      if (i == np) break;
      ++r[i];
    }
  }
  return out;
}

// The fastest of three runs after one warm-up, in ms (1e30 when a launch is refused).
template <class C>
double time_shape(C* A, C* B, int logF, int ncols, const C* tw, int logFmax, const FftShape& sh, cudaEvent_t e0,
                  cudaEvent_t e1, const TcTables* tc = nullptr) {
  double best = 1e30;
  for (int it = 0; it < 4; ++it) {
    C* res = nullptr;
    cudaEventRecord(e0, 0);
    if (run_fft<C>(A, B, logF, ncols, false, tw, logFmax, 0, &res, nullptr, nullptr, 1, nullptr, &sh, tc) != HANKEL_OK ||
        cudaGetLastError() != cudaSuccess)  // a split whose launch is refused is not a candidate
      return 1e30;
    cudaEventRecord(e1, 0);
    if (cudaEventSynchronize(e1) != cudaSuccess) return 1e30;
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (it > 0) best = std::min(best, (double)ms);
  }
  return best;
}

// The shape of transforms of 2^logF points in precision prec over ncols columns per launch:
// from the plan's list, the process cache (keyed by GPU model) or a measurement of the
// candidates on the lane's workspace buffers A, B (bytes each), recorded in the plan's list.
// The split of a length with the most of its bits in tensor-core passes (radix 32 or 64), fewest
// passes on ties; the other passes (radix 2^7, 2^8) on the FP64 pipe, after them.
bool tensor_shape(int logF, FftShape* out) {
  if (logF < 12) return false;
  bool found = false;
  int best_bits = -1, best_np = 9;
  for (int np = 2; np <= 4; ++np) {
    int r[4] = {5, 5, 5, 5};
    for (;;) {
      int sum = 0, tcb = 0;
      for (int i = 0; i < np; ++i) {
        sum += r[i];
        if (r[i] <= 6) tcb += r[i];
      }
      if (sum == logF && (tcb > best_bits || (tcb == best_bits && np < best_np))) {
        FftShape sh{};
        sh.npass = np;
        // tensor-core passes first
        int k = 0;
        for (int i = 0; i < np; ++i)
          if (r[i] <= 6) sh.logr[k++] = r[i];
        const int ntc = k;
        for (int i = 0; i < np; ++i)
          if (r[i] > 6) sh.logr[k++] = r[i];
        sh.tc = (1 << ntc) - 1;
        if (ntc > 0 && valid_fft_shape(sh, logF)) {
          *out = sh;
          best_bits = tcb;
          best_np = np;
          found = true;
        }
      }
      int i = 0;  // next tuple in [5, 8]^np
      while (i < np && r[i] == 8) r[i++] = 5;
      if (i == np) break;
      ++r[i];
    }
  }
  return found;
}

int plan_shape(DevicePlan* d, const std::string& gpu, bool tune, int prec, int logF, int64_t ncols, void* A, void* B,
               size_t bytes, FftShape* out, bool force_tc = false) {
  const int bucket = tune_bucket(ncols);
  const int pp = public_precision(prec);
  for (const hankel_fft_shape& h : d->shapes)
    if (h.precision == pp && h.log2_len == logF && h.col_bucket == bucket) {
      out->one_launch = h.one_launch;
      out->npass = h.npass;
      std::copy(h.log2_radix, h.log2_radix + 4, out->logr);
      out->tc = h.tensor_passes;
      return HANKEL_OK;
    }
  hankel_fft_shape h{};
  h.precision = pp;
  h.log2_len = logF;
  h.col_bucket = bucket;
  FftShape sh = default_fft_shape(logF, (int)ncols, prec);
  bool cached = false;
  if (force_tc && prec == kTermFP64 && d->tc() && tensor_shape(logF, &sh)) tune = false;
  if (tune) {
    hankel_fft_shape c{};
    if (tune_get(gpu, pp, logF, bucket, &c)) {
      FftShape cs{c.one_launch, c.npass, {c.log2_radix[0], c.log2_radix[1], c.log2_radix[2], c.log2_radix[3]},
                  c.tensor_passes};
      if (cs.tc && !d->tc()) cs.tc = 0;
      if (valid_fft_shape(cs, logF)) {
        sh = cs;
        cached = true;
      }
    }
  }
  if (tune && !cached) {
    const size_t esz = term_esz(prec);
    const int64_t F = int64_t(1) << logF;
    // enough columns to fill the GPU as the real launches do, at most 2^25 points
    int64_t nt = std::min<int64_t>(ncols, std::max<int64_t>(1, (int64_t(1) << 25) / F));
    nt = std::min<int64_t>(nt, (int64_t)(bytes / (F * esz)));
    if (nt >= 1) {
      // measured on seeded values of unit size (zeros would take other paths in some kernels)
      launch_fill_pattern(A, (size_t)nt * F * esz / sizeof(float), prec == kTermFP32 ? 1 : 0, 0);
      cudaEvent_t e0 = nullptr, e1 = nullptr;
      if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return HANKEL_ECUDA;
      const std::vector<FftShape> cand = shape_candidates(logF, (int)ncols, prec, d->tc() != nullptr);
      double tdef = 0.0, tbest = 1e30;
      FftShape best = cand[0];
      for (size_t i = 0; i < cand.size(); ++i) {
        double t;
        if (prec == kTermFP32)
          t = time_shape<float2>((float2*)A, (float2*)B, logF, (int)nt, d->twf, d->logFmax, cand[i], e0, e1);
        else if (prec == kTermDF64)
          t = time_shape<df64c>((df64c*)A, (df64c*)B, logF, (int)nt, d->twd, d->logFmax, cand[i], e0, e1);
        else
          t = time_shape<double2>((double2*)A, (double2*)B, logF, (int)nt, d->tw, d->logFmax, cand[i], e0, e1,
                                  d->tc());
        if (i == 0) tdef = t;
        if (t < tbest) {
          tbest = t;
          best = cand[i];
        }
      }
      cudaEventDestroy(e0);
      cudaEventDestroy(e1);
      if (cudaGetLastError() != cudaSuccess) return HANKEL_ECUDA;
      // keep the built-in split unless another is clearly faster (2 %)
      if (!(tbest < 0.98 * tdef)) {
        best = cand[0];
        tbest = tdef;
      }
      sh = best;
      h.ms_default = tdef;
      h.ms_chosen = tbest;
    }
  }
  h.one_launch = sh.one_launch;
  h.npass = sh.npass;
  std::copy(sh.logr, sh.logr + 4, h.log2_radix);
  h.tensor_passes = sh.tc;
  if (tune && !cached && h.ms_chosen > 0) tune_put(gpu, h);
  d->shapes.push_back(h);
  *out = sh;
  return HANKEL_OK;
}

}  // namespace

int dev_plan_create(hankel_plan_s* p) {
  const HostPlan& hp = p->hp;
  DevicePlan* d = new DevicePlan();
  p->dev = d;
  if (cudaGetDevice(&d->device) != cudaSuccess) return HANKEL_ECUDA;
  const int64_t N = hp.opt.N;
  d->hpN = N;
  {
    // Look up the allocation-free entry point's static array on this device now, so that it is
    // placed before the caller hands its memory to a pool and before any stream capture (with
    // lazy module loading the array is placed at this first lookup). A failure here is not the
    // plan's: hankel_exec_static retries the lookup and reports it.
    double2* scratch = nullptr;
    if (static_scratch_address(d->device, &scratch) != HANKEL_OK) cudaGetLastError();
  }

  // Node tables and their derived powers.
  std::vector<double> tmp(N);
  HK_TRY(upload(d, &d->nodes.r_true, hp.r_true.data(), N));
  HK_TRY(upload(d, &d->nodes.om_true, hp.om_true.data(), N));
  HK_TRY(upload(d, &d->nodes.rowvar, hp.rowvar.data(), N));
  HK_TRY(upload(d, &d->nodes.rowpert, hp.rowpert.data(), N));
  HK_TRY(upload(d, &d->nodes.omt, hp.omt.data(), N));
  HK_TRY(upload(d, &d->nodes.betan, hp.betan.data(), N));
  HK_TRY(upload(d, &d->nodes.colpow, hp.colpow.data(), N));
  for (int64_t i = 0; i < N; ++i) tmp[i] = hp.rowvar[i] > 0 ? 1.0 / std::sqrt(hp.rowvar[i]) : 0.0;
  HK_TRY(upload(d, &d->nodes.rs_rowvar, tmp.data(), N));
  for (int64_t i = 0; i < N; ++i) tmp[i] = hp.rowvar[i] > 0 ? 1.0 / hp.rowvar[i] : 0.0;
  HK_TRY(upload(d, &d->nodes.inv_rowvar, tmp.data(), N));
  for (int64_t i = 0; i < N; ++i) tmp[i] = 1.0 / std::sqrt(hp.omt[i]);
  HK_TRY(upload(d, &d->nodes.rs_omt, tmp.data(), N));
  for (int64_t i = 0; i < N; ++i) tmp[i] = 1.0 / hp.omt[i];
  HK_TRY(upload(d, &d->nodes.inv_omt, tmp.data(), N));

  // Stacked-column specifications.
  std::vector<DevColSpec> cs(hp.cols.size());
  for (size_t i = 0; i < hp.cols.size(); ++i) {
    memset(&cs[i], 0, sizeof(DevColSpec));
    cs[i].u1 = hp.cols[i].u1;
    cs[i].delta = hp.cols[i].delta;
    cs[i].nterm = hp.cols[i].nterm;
    for (int u = 0; u < kMaxU; ++u) cs[i].G[u] = make_double2(hp.cols[i].G[u].real(), hp.cols[i].G[u].imag());
  }
  d->ncols = (int)cs.size();
  HK_TRY(upload(d, &d->cols, cs.data(), cs.size()));
  HK_TRY(upload(d, &d->jtab, hp.jtab.data(), hp.jtab.size()));
  d->fp32 = hp.fp32;
  d->df64 = hp.df64;
  for (const Block& b : hp.blocks)
    for (int8_t t : b.tprec) d->any_t[t] = true;
  if (d->fp32) {
    std::vector<float> tf(std::max<size_t>((size_t)N, hp.jtab.size()));
    for (int64_t i = 0; i < N; ++i) tf[i] = (float)hp.r_true[i];
    HK_TRY(upload(d, &d->rf, tf.data(), N));
    for (int64_t i = 0; i < N; ++i) tf[i] = (float)hp.om_true[i];
    HK_TRY(upload(d, &d->omf, tf.data(), N));
    for (size_t i = 0; i < hp.jtab.size(); ++i) tf[i] = (float)hp.jtab[i];
    HK_TRY(upload(d, &d->jtabf, tf.data(), hp.jtab.size()));
  }
  if (d->df64) {
    std::vector<float2> tp(std::max<size_t>((size_t)N, hp.jtab.size()));
    auto pair = [](double x) {
      const float h = (float)x;
      return make_float2(h, (float)(x - (double)h));
    };
    for (int64_t i = 0; i < N; ++i) tp[i] = pair(hp.r_true[i]);
    HK_TRY(upload(d, &d->rdf, tp.data(), N));
    for (int64_t i = 0; i < N; ++i) tp[i] = pair(hp.om_true[i]);
    HK_TRY(upload(d, &d->omdf, tp.data(), N));
    for (size_t i = 0; i < hp.jtab.size(); ++i) tp[i] = pair(hp.jtab[i]);
    HK_TRY(upload(d, &d->jtabdf, tp.data(), hp.jtab.size()));
  }
  // per-execution coefficient copies (made per context): double-float pairs for DF64 near fields
  // and transforms, FP32 for FP32 transforms (FP32 near fields read them too), digits for the
  // tensor-core near field
  d->want_cdf = d->df64 || d->any_t[kTermDF64];
  d->want_cf = d->any_t[kTermFP32];
  if (!d->fp32 && hp.opt.max_nrhs >= kNearTcMinRhs) d->tc_npad = (N + 511) / 512 * 512;
  if (!d->fp32) HK_TRY(upload(d, &d->jtabq, hp.jtabq.data(), hp.jtabq.size()));

  // Near-field work list: groups of kNearRows rows, the group's longest prefix cut into tiles of
  // kNearCols columns; groups with more than one tile add up per-row partial sums.
  std::vector<NearItem> items;
  std::vector<NearRow> mrows;
  items.reserve(N / kNearRows + hp.near_count / (kNearRows * kNearCols) + 16);
  int64_t slot = 0;
  for (int64_t k0 = 1; k0 <= N; k0 += kNearRows) {
    const int64_t k1 = std::min<int64_t>(N, k0 + kNearRows - 1);
    int64_t ne = 0;
    for (int64_t k = k0; k <= k1; ++k) ne = std::max(ne, hp.nend[k - 1]);
    const int64_t nt = std::max<int64_t>(1, (ne + kNearCols - 1) / kNearCols);
    if (nt == 1) {
      items.push_back(NearItem{k0, 1, ne, -1, 1, 0});
      continue;
    }
    for (int64_t t = 0; t < nt; ++t)
      items.push_back(NearItem{k0, 1 + t * kNearCols, std::min(ne, (t + 1) * kNearCols), slot, (int32_t)nt, (int32_t)t});
    for (int64_t k = k0; k <= k1; ++k) mrows.push_back(NearRow{k, slot + (k - k0) * nt, (int32_t)nt, 0});
    slot += kNearRows * nt;
  }
  d->nitems = (int64_t)items.size();
  d->nmrows = (int64_t)mrows.size();
  d->nslots = slot;
  HK_TRY(upload(d, &d->items, items.data(), items.size()));
  HK_TRY(upload(d, &d->nend, hp.nend.data(), hp.nend.size()));
  if (!mrows.empty()) HK_TRY(upload(d, &d->mrows, mrows.data(), mrows.size()));

  // Twiddle table W_{Fmax}^t = exp(-2 pi i t / Fmax).
  int logFmax = 6;
  for (const Block& b : hp.blocks) logFmax = std::max(logFmax, b.logF);
  d->logFmax = logFmax;
  // one compact table per transform length, so that a transform's twiddles stay together
  // in cache instead of being spread over the table of the longest transform
  HK_TRY(dalloc(d, &d->tw, (size_t)2 << logFmax));
  for (int L = 6; L <= logFmax; ++L) launch_twiddles(d->tw + ((size_t)1 << L), L, 0);
  HK_LAUNCHED();
  if (d->any_t[kTermFP64] && logFmax >= 12) {
    // digit planes of the 32-point DFT for the tensor-core passes of FP64 transforms
    const size_t nb = tc_dft_digits_bytes();
    std::vector<unsigned char> host(2 * nb);
    tc_dft_digits(0, host.data());
    tc_dft_digits(1, host.data() + nb);
    unsigned char* q = nullptr;
    HK_TRY(upload(d, &q, host.data(), host.size()));
    d->tcB = q;
    HK_TRY(dalloc(d, &d->tc_err, 1));
    if (cudaMemset(d->tc_err, 0, sizeof(unsigned)) != cudaSuccess) return HANKEL_ECUDA;
    longlong2* twq = nullptr;
    HK_TRY(dalloc(d, &twq, (size_t)2 << logFmax));
    launch_twiddles_q62(d->tw + 64, twq + 64, (int64_t(2) << logFmax) - 64, 0);
    HK_LAUNCHED();
    d->tct = TcTables{q, q + nb, d->tc_err, twq};
  }
  if (d->any_t[kTermFP32]) {
    HK_TRY(dalloc(d, &d->twf, (size_t)2 << logFmax));
    launch_scale_copy<float2>(d->tw + 64, d->twf + 64, (int64_t(2) << logFmax) - 64, 1.0, 0);
    HK_LAUNCHED();
  }
  if (d->any_t[kTermDF64]) {
    HK_TRY(dalloc(d, &d->twd, (size_t)2 << logFmax));
    launch_scale_copy<df64c>(d->tw + 64, d->twd + 64, (int64_t(2) << logFmax) - 64, 1.0, 0);
    HK_LAUNCHED();
  }

  // Workspace: two ping-pong buffers, each holding a chunk of stacked columns of one term group
  // of a block (nseg transforms of length F per stacked column for segmented blocks). The
  // plan-time spectra are computed in FP64 in the same buffers, so each holds at least nseg F
  // double2 values.
  // lanes: the plan precision's groups in lane 0, each other precision present in a lane of
  // its own
  {
    const int base = d->fp32 ? kTermFP32 : d->df64 ? kTermDF64 : kTermFP64;
    d->lane_of[base] = 0;
    for (int t = 0; t < 3; ++t)
      if (t != base && d->any_t[t]) d->lane_of[t] = d->nlanes++;
  }
  size_t limit = hp.opt.workspace_limit ? hp.opt.workspace_limit : kDefaultWorkspace;
  size_t need[3] = {sizeof(double2) << logFmax, 0, 0};  // bytes per buffer, per lane
  std::vector<int> lists[3];
  for (const Block& b : hp.blocks) {
    const size_t foot = column_footprint(b);
    term_lists(b, lists);
    for (int t = 0; t < 3; ++t) {
      if (lists[t].empty()) continue;
      const size_t esz = term_esz(t);
      const int64_t total = (int64_t)lists[t].size() * hp.opt.max_nrhs;
      int64_t cap = (int64_t)(limit / (2 * esz * foot));
      cap = std::max<int64_t>(1, std::min<int64_t>(cap, total));
      need[d->lane_of[t]] = std::max(need[d->lane_of[t]], (size_t)cap * foot * esz);
    }
    need[0] = std::max(need[0], sizeof(double2) * (size_t)b.nseg * (size_t)b.F);
  }
  d->ws_bytes = 0;
  for (int l = 0; l < d->nlanes; ++l) {
    d->lane_bytes[l] = need[l];
    d->ws_bytes += 2 * need[l];
  }
  HK_TRY(ctx_create(d, hp));
  void* bufA = d->ctx[0]->lanes[0].A;
  void* bufB = d->ctx[0]->lanes[0].B;

  // Per block: chirp vectors, the spectra of its convolution kernels (one per segment) and per
  // term group its column and row tables (the low-rank form's terms, or its kept stacked columns).
  for (const Block& b : hp.blocks) {
    DevBlock db;
    db.b = b;
    HK_TRY(dalloc(d, &db.wU, b.R));
    HK_TRY(dalloc(d, &db.wV, b.C));
    ChirpGeom g{hp.Ua, hp.Ub, hp.Va, hp.Vb, hp.E, b.k0, b.n0, b.R, b.C, b.F};
    launch_chirps(g, db.wU, db.wV, 0);
    HK_LAUNCHED();
    term_lists(b, lists);
    for (int t = 0; t < 3; ++t) {
      if (lists[t].empty()) continue;
      TermGroup& tg = db.g[db.ng++];
      tg.prec = t;
      tg.nl = (int)lists[t].size();
      tg.cap = std::max<int64_t>(1, std::min<int64_t>(
                                        (int64_t)(need[d->lane_of[t]] / (column_footprint(b) * term_esz(t))),
                                        (int64_t)tg.nl * hp.opt.max_nrhs));
      if (t == kTermFP32) {
        float2* h; HK_TRY(dalloc(d, &h, (size_t)b.nseg * b.F)); tg.H = h;
        float2* vt; HK_TRY(dalloc(d, &vt, (size_t)tg.nl * b.C)); tg.Vt = vt;
        float2* ut; HK_TRY(dalloc(d, &ut, (size_t)tg.nl * b.R)); tg.Ut = ut;
      } else if (t == kTermDF64) {
        df64c* h; HK_TRY(dalloc(d, &h, (size_t)b.nseg * b.F)); tg.H = h;
        df64c* vt; HK_TRY(dalloc(d, &vt, (size_t)tg.nl * b.C)); tg.Vt = vt;
        df64c* ut; HK_TRY(dalloc(d, &ut, (size_t)tg.nl * b.R)); tg.Ut = ut;
      } else {
        double2* h; HK_TRY(dalloc(d, &h, (size_t)b.nseg * b.F)); tg.H = h;
        double2* vt; HK_TRY(dalloc(d, &vt, (size_t)tg.nl * b.C)); tg.Vt = vt;
        double2* ut; HK_TRY(dalloc(d, &ut, (size_t)tg.nl * b.R)); tg.Ut = ut;
      }
      HK_LAUNCHED();
      // FP32 transforms: per term, the power of two that brings max |colfun(n)| over the block
      // to ~1 (its inverse goes to the row side)
      std::vector<double> sc;
      if (t == kTermFP32) {
        sc.assign(tg.nl, 1.0);
        for (int j = 0; j < tg.nl; ++j) {
          const int li = lists[t][j];
          double mag = 0.0;
          if (b.rank) {
            for (int q = 0; q < b.P; ++q) mag = std::max(mag, std::abs(b.vcheb[(size_t)li * b.P + q]));
          } else {
            const ColSpec& csp = hp.cols[b.lcols[li]];
            for (int64_t n : {b.n0, b.n1}) {
              const int64_t i = n - 1;
              cplx poly(0.0, 0.0);
              for (int u = csp.nterm - 1; u >= 0; --u) poly = poly * hp.betan[i] + csp.G[u];
              double m = std::abs(poly) * std::pow(hp.omt[i], csp.delta - 0.5);
              if (csp.u1) m *= std::pow(hp.colpow[i], csp.u1);
              mag = std::max(mag, m);
            }
          }
          const int e = (mag > 0.0 && std::isfinite(mag)) ? -(int)std::lround(std::log2(mag)) : 0;
          sc[j] = std::ldexp(1.0, e);
        }
      }
      // inputs of the table kernels (this group's terms), freed once the tables are built
      int* lmap = nullptr;
      double2 *uc = nullptr, *vc = nullptr;
      double* scd = nullptr;
      size_t nuc = 0, nlm = 0;
      if (b.rank) {
        // the interpolants' Chebyshev coefficients (the kernels sum the series by Clenshaw)
        std::vector<double2> u((size_t)tg.nl * b.P), v((size_t)tg.nl * b.P);
        for (int j = 0; j < tg.nl; ++j) {
          cheb_coeffs(&b.ucheb[(size_t)lists[t][j] * b.P], b.P, &u[(size_t)j * b.P]);
          cheb_coeffs(&b.vcheb[(size_t)lists[t][j] * b.P], b.P, &v[(size_t)j * b.P]);
        }
        nuc = u.size();
        HK_TRY(upload(d, &uc, u.data(), u.size()));
        HK_TRY(upload(d, &vc, v.data(), v.size()));
      } else {
        std::vector<int> lm(tg.nl);
        for (int j = 0; j < tg.nl; ++j) lm[j] = b.lcols[lists[t][j]];
        nlm = lm.size();
        HK_TRY(upload(d, &lmap, lm.data(), lm.size()));
      }
      if (!sc.empty()) HK_TRY(upload(d, &scd, sc.data(), sc.size()));
      BlockTabArgs ta{tg.nl, b.k0, b.R, b.n0, b.C, lmap, b.rank ? b.P : 0, uc, vc,
                      std::log((double)b.k0), std::log((double)b.k1), std::log((double)b.n0),
                      std::log((double)b.n1), d->nodes, d->cols, db.wV, db.wU, scd, tg.Vt, tg.Ut};
      if (t == kTermFP32) launch_block_tables<float2>(ta, 0);
      else if (t == kTermDF64) launch_block_tables<df64c>(ta, 0);
      else launch_block_tables<double2>(ta, 0);
      HK_LAUNCHED();
      if (cudaDeviceSynchronize() != cudaSuccess) return HANKEL_ECUDA;
      dfree(d, &uc, nuc);
      dfree(d, &vc, nuc);
      dfree(d, &lmap, nlm);
      dfree(d, &scd, sc.size());
    }
    // the chirp spectra in FP64, then rounded to each group's precision
    SegGeom sg{hp.Ua, hp.Ub, hp.Vb, hp.E, b.k0, b.n0, b.R, b.C, 0, 0, 1, b.F};
    if (b.mode == kBlockRowSeg) { sg.Cc = b.S; sg.dn = b.S; sg.nseg = b.nseg; }
    if (b.mode == kBlockColSeg) { sg.Rr = b.S; sg.dk = b.S; sg.nseg = b.nseg; }
    double2* hA = (double2*)bufA;
    double2* hB = (double2*)bufB;
    launch_seg_hh(sg, hA, 0);
    HK_LAUNCHED();
    double2* res = nullptr;
    HK_TRY(run_fft<double2>(hA, hB, b.logF, (int)b.nseg, /*inverse=*/false, d->tw, d->logFmax, 0, &res));
    for (int j = 0; j < db.ng; ++j) {
      const TermGroup& tg = db.g[j];
      if (tg.prec == kTermFP32) launch_scale_copy<float2>(res, (float2*)tg.H, b.nseg * b.F, 1.0 / (double)b.F, 0);
      else if (tg.prec == kTermDF64) launch_scale_copy<df64c>(res, (df64c*)tg.H, b.nseg * b.F, 1.0 / (double)b.F, 0);
      else launch_scale_copy<double2>(res, (double2*)tg.H, b.nseg * b.F, 1.0 / (double)b.F, 0);
      HK_LAUNCHED();
    }
    d->blocks.push_back(db);
  }
  if (cudaDeviceSynchronize() != cudaSuccess) return HANKEL_ECUDA;

  // Launch split of every term group's forward and inverse transforms (autotuned per GPU model)
  const bool tune = !(hp.opt.flags & HANKEL_FLAG_NO_AUTOTUNE);
  std::string gpu;
  if (tune) {
    tune_load_env();
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, d->device) != cudaSuccess) return HANKEL_ECUDA;
    gpu = prop.name;
  }
  for (DevBlock& db : d->blocks)
    for (int j = 0; j < db.ng; ++j) {
      TermGroup& tg = db.g[j];
      const int l = d->lane_of[tg.prec];
      const int64_t nfwd = tg.cap * (db.b.mode == kBlockRowSeg ? db.b.nseg : 1);
      const int64_t ninv = tg.cap * (db.b.mode == kBlockColSeg ? db.b.nseg : 1);
      const DevicePlan::Lane& ln = d->ctx[0]->lanes[l];
      const bool ftc = (hp.opt.flags & HANKEL_FLAG_TENSOR_FFT) != 0;
      HK_TRY(plan_shape(d, gpu, tune, tg.prec, db.b.logF, nfwd, ln.A, ln.B, ln.buf_bytes, &tg.fwd, ftc));
      HK_TRY(plan_shape(d, gpu, tune, tg.prec, db.b.logF, ninv, ln.A, ln.B, ln.buf_bytes, &tg.inv, ftc));
    }
  if (cudaDeviceSynchronize() != cudaSuccess) return HANKEL_ECUDA;
  return HANKEL_OK;
}

int dev_fft_compare(int logF, int ncols, int inverse, const FftShape& sh, double* err, double* ms) {
  const int64_t F = int64_t(1) << logF;
  const size_t n = (size_t)ncols * F;
  double2 *x = nullptr, *a = nullptr, *b = nullptr, *tw = nullptr;
  longlong2* twq = nullptr;
  void* bd = nullptr;
  unsigned* flag = nullptr;
  std::vector<double2> hx(n), h1(n), h2(n);
  uint64_t st = 0x2545F4914F6CDD1DULL;
  for (size_t i = 0; i < n; ++i) {
    st = st * 6364136223846793005ULL + 1442695040888963407ULL;
    const double re = (double)(st >> 11) * 0x1p-53 - 0.5;
    st = st * 6364136223846793005ULL + 1442695040888963407ULL;
    hx[i] = make_double2(re, (double)(st >> 11) * 0x1p-53 - 0.5);
  }
  const size_t nb = tc_dft_digits_bytes();
  std::vector<unsigned char> hb(2 * nb);
  tc_dft_digits(0, hb.data());
  tc_dft_digits(1, hb.data() + nb);
  int rc = HANKEL_OK;
  auto cleanup = [&]() {
    cudaFree(x);
    cudaFree(a);
    cudaFree(b);
    cudaFree(tw);
    cudaFree(twq);
    cudaFree(bd);
    cudaFree(flag);
  };
  if (cudaMalloc(&x, n * sizeof(double2)) != cudaSuccess || cudaMalloc(&a, n * sizeof(double2)) != cudaSuccess ||
      cudaMalloc(&b, n * sizeof(double2)) != cudaSuccess || cudaMalloc(&tw, (size_t)2 * F * sizeof(double2)) != cudaSuccess ||
      cudaMalloc(&bd, 2 * nb) != cudaSuccess || cudaMalloc(&flag, sizeof(unsigned)) != cudaSuccess ||
      cudaMalloc(&twq, (size_t)2 * F * sizeof(longlong2)) != cudaSuccess) {
    cudaGetLastError();
    cleanup();
    return HANKEL_ENOMEM;
  }
  for (int L = 6; L <= logF; ++L) launch_twiddles(tw + ((size_t)1 << L), L, 0);
  launch_twiddles_q62(tw + 64, twq + 64, 2 * F - 64, 0);
  cudaMemcpy(x, hx.data(), n * sizeof(double2), cudaMemcpyHostToDevice);
  cudaMemcpy(bd, hb.data(), 2 * nb, cudaMemcpyHostToDevice);
  cudaMemset(flag, 0, sizeof(unsigned));
  const TcTables tt{bd, (unsigned char*)bd + nb, flag, twq};
  double2* res = nullptr;
  // reference: the built-in split
  cudaMemcpy(a, x, n * sizeof(double2), cudaMemcpyDeviceToDevice);
  if (run_fft<double2>(a, b, logF, ncols, inverse != 0, tw, logF, 0, &res) != HANKEL_OK) rc = HANKEL_EINVAL;
  if (rc == HANKEL_OK) cudaMemcpy(h1.data(), res, n * sizeof(double2), cudaMemcpyDeviceToHost);
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  double best = 1e30;
  for (int it = 0; it < 4 && rc == HANKEL_OK; ++it) {
    cudaMemcpy(a, x, n * sizeof(double2), cudaMemcpyDeviceToDevice);
    cudaEventRecord(e0, 0);
    if (run_fft<double2>(a, b, logF, ncols, inverse != 0, tw, logF, 0, &res, nullptr, nullptr, 1, nullptr, &sh, &tt) !=
        HANKEL_OK)
      rc = HANKEL_EINVAL;
    cudaEventRecord(e1, 0);
    if (cudaEventSynchronize(e1) != cudaSuccess) rc = HANKEL_ECUDA;
    float t = 0.f;
    cudaEventElapsedTime(&t, e0, e1);
    if (it > 0) best = std::min(best, (double)t);
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc == HANKEL_OK && cudaGetLastError() != cudaSuccess) rc = HANKEL_ECUDA;
  if (rc == HANKEL_OK) {
    cudaMemcpy(h2.data(), res, n * sizeof(double2), cudaMemcpyDeviceToHost);
    unsigned fl = 0;
    cudaMemcpy(&fl, flag, sizeof fl, cudaMemcpyDeviceToHost);
    if (fl) rc = HANKEL_ETIMEOUT;
  }
  if (rc == HANKEL_OK) {
    double dmax = 0.0, rmax = 0.0;
    for (size_t i = 0; i < n; ++i) {
      dmax = std::max(dmax, std::max(std::fabs(h1[i].x - h2[i].x), std::fabs(h1[i].y - h2[i].y)));
      rmax = std::max(rmax, std::max(std::fabs(h1[i].x), std::fabs(h1[i].y)));
    }
    *err = rmax > 0 ? dmax / rmax : dmax;
    *ms = best;
  }
  cleanup();
  return rc;
}

int debug_fft_compare_host(int logF, int ncols, int inverse, int npass, const int* logr, int tc, double* err,
                           double* ms) {
  FftShape sh{};
  sh.npass = npass;
  for (int i = 0; i < npass; ++i) sh.logr[i] = logr[i];
  sh.tc = tc;
  if (!valid_fft_shape(sh, logF)) return HANKEL_EINVAL;
  return dev_fft_compare(logF, ncols, inverse, sh, err, ms);
}

int dev_device_status(hankel_plan_s* p) {
  DevicePlan* d = p->dev;
  if (!d || !d->tc_err) return HANKEL_OK;
  unsigned v = 0;
  if (cudaMemcpy(&v, d->tc_err, sizeof v, cudaMemcpyDeviceToHost) != cudaSuccess) return HANKEL_ECUDA;
  if (v == 0) return HANKEL_OK;
  if (cudaMemset(d->tc_err, 0, sizeof(unsigned)) != cudaSuccess) return HANKEL_ECUDA;
  return HANKEL_ETIMEOUT;
}

int dev_plan_shapes(const hankel_plan_s* p, hankel_fft_shape* out, int cap, int* count) {
  const DevicePlan* d = p->dev;
  *count = d ? (int)d->shapes.size() : 0;
  for (int i = 0; i < cap && i < *count; ++i) out[i] = d->shapes[i];
  return HANKEL_OK;
}

int dev_plan_destroy(hankel_plan_s* p) {
  DevicePlan* d = p->dev;
  if (!d) return HANKEL_OK;
  int cur = 0;
  cudaGetDevice(&cur);
  cudaSetDevice(d->device);
  cudaDeviceSynchronize();
  for (cudaEvent_t e : d->pool) cudaEventDestroy(e);
  for (DevicePlan::ExecCtx* x : d->ctx) {
    for (int l = 1; l < 3; ++l) {
      if (x->lanes[l].done) cudaEventDestroy(x->lanes[l].done);
      if (x->lanes[l].s) cudaStreamDestroy(x->lanes[l].s);
    }
    if (x->fork) cudaEventDestroy(x->fork);
    delete x;
  }
  d->ctx.clear();
  for (void* q : d->allocs) cudaFree(q);
  cudaSetDevice(cur);
  delete d;
  p->dev = nullptr;
  return HANKEL_OK;
}

size_t dev_plan_bytes(const hankel_plan_s* p) { return p->dev ? p->dev->bytes : 0; }
size_t dev_workspace_bytes(const hankel_plan_s* p) { return p->dev ? p->dev->ws_bytes : 0; }

namespace {

// Far-field work of one block for nrhs vectors: chunks of `cap` stacked columns through
// generation, forward FFTs, the product with the kernel spectra (summed over column segments
// or replicated over row segments), inverse FFTs and the row accumulation into f.
// C = double2 (FP64 plans), float2 (FP32 plans) or df64c (DF64 plans).
// Per precision: twiddle ladder, coefficient copy (format of FftGen::coef) and FFT stage.
template <class C>
struct Prec;
template <>
struct Prec<double2> {
  static const void* tw(const DevicePlan* d) { return d->tw; }
  static const void* coef(const DevicePlan::ExecCtx*, const double* c) { return c; }
  static constexpr int stage = HANKEL_STAGE_FFT;
};
template <>
struct Prec<df64c> {
  static const void* tw(const DevicePlan* d) { return d->twd; }
  static const void* coef(const DevicePlan::ExecCtx* x, const double*) { return x->cdf; }
  static constexpr int stage = HANKEL_STAGE_FFT_DF64;
};
template <>
struct Prec<float2> {
  static const void* tw(const DevicePlan* d) { return d->twf; }
  static const void* coef(const DevicePlan::ExecCtx* x, const double*) { return x->cf; }
  static constexpr int stage = HANKEL_STAGE_FFT_FP32;
};

template <class C>
int run_block(DevicePlan* d, const DevicePlan::ExecCtx* x, const DevBlock& db, const TermGroup& tg, const double* c,
              int64_t ldc, double* f, int64_t ldf, int nrhs, C* A, C* B, int64_t cap, cudaStream_t st, bool record) {
  const Block& b = db.b;
  const C* tw = (const C*)Prec<C>::tw(d);
  const C* H = (const C*)tg.H;
  const int fst = Prec<C>::stage;
  const int64_t total = (int64_t)tg.nl * nrhs;
  const bool rowseg = b.mode == kBlockRowSeg, colseg = b.mode == kBlockColSeg;
  for (int64_t c0 = 0; c0 < total; c0 += cap) {
    const int nc = (int)std::min<int64_t>(cap, total - c0);
    const int64_t nfwd = rowseg ? (int64_t)nc * b.nseg : nc;  // forward transforms
    const int64_t ninv = colseg ? (int64_t)nc * b.nseg : nc;  // inverse transforms
    C* res = nullptr;
    {
      // column generation happens in the first loads of the forward transform
      StageScope sc(d, fst, st, record);
      int np = 0;
      const void* coef = Prec<C>::coef(x, c);
      const FftGen gen{rowseg ? b.nseg : 1, rowseg ? b.S : b.C, b.C, b.n0, c0, tg.nl, coef,
                       coef == (const void*)c ? ldc : d->hpN, tg.Vt};
      HK_TRY(run_fft<C>(A, B, b.logF, (int)nfwd, false, tw, d->logFmax, st, &res, &np, nullptr, 1, &gen, &tg.fwd,
                        d->tc()));
      HK_LAUNCHED();
      sc.done(np, 5.0 * (double)b.F * (double)b.logF * (double)nfwd, 0.0, 2.0 * sizeof(C) * (double)b.F * nfwd * np);
    }
    C* other = (res == A) ? B : A;
    C* res2 = nullptr;
    if (rowseg) {
      // overlap-add: the segments' spectra times their chirp spectra, summed per column
      {
        StageScope sc(d, HANKEL_STAGE_POINTWISE, st, record);
        launch_seg_mac<C>(res, H, other, b.F, b.nseg, nc, st);
        HK_LAUNCHED();
        // every segment spectrum and chirp spectrum read once, every sum written once
        sc.done(1, 8.0 * (double)b.F * (double)b.nseg * nc, 0.0,
                (double)sizeof(C) * (double)b.F * ((double)b.nseg * (nc + 1) + nc));
      }
      StageScope sc(d, fst, st, record);
      int np = 0;
      HK_TRY(run_fft<C>(other, res, b.logF, (int)ninv, true, tw, d->logFmax, st, &res2, &np, nullptr, 1, nullptr,
                        &tg.inv, d->tc()));
      HK_LAUNCHED();
      sc.done(np, 5.0 * (double)b.F * (double)b.logF * (double)ninv, 0.0, 2.0 * sizeof(C) * (double)b.F * ninv * np);
    } else {
      // full blocks: one product with the chirp spectrum; row segments (overlap-save): each
      // column's spectrum times every segment's chirp spectrum -- both folded into the first
      // loads of the inverse transform
      StageScope sc(d, fst, st, record);
      int np = 0;
      HK_TRY(run_fft<C>(res, other, b.logF, (int)ninv, true, tw, d->logFmax, st, &res2, &np, H,
                        colseg ? b.nseg : 1, nullptr, &tg.inv, d->tc()));
      HK_LAUNCHED();
      // 5 F log2 F per transform plus 6 F for the folded complex products
      sc.done(np, (5.0 * (double)b.logF + 6.0) * (double)b.F * (double)ninv, 0.0,
              2.0 * sizeof(C) * (double)b.F * ninv * np);
    }
    {
      StageScope sc(d, HANKEL_STAGE_OUT, st, record);
      OutArgs oa{res2, b.F, b.R, b.k0, (rowseg ? b.S : b.C) - 1, colseg ? b.S : b.R, colseg ? b.nseg : 1,
                 nc, c0, tg.nl, f, ldf, tg.Ut, std::is_same<C, double2>::value ? nullptr : x->cexp};
      launch_out<C>(oa, st);
      HK_LAUNCHED();
      // the block's rows of every transform and of every distinct row weight read once, and the
      // chunk's right-hand sides of f read and written once
      const int64_t nr = (c0 + nc - 1) / tg.nl - c0 / tg.nl + 1;
      sc.done(1, 4.0 * (double)b.R * nc, 0.0,
              (double)b.R * ((double)sizeof(C) * (nc + std::min<int64_t>(nc, tg.nl)) + 16.0 * (double)nr));
    }
  }
  return HANKEL_OK;
}

// Near field of a plan in its precision, then every far block's term groups. capacity
// (chunk_from_capacity): bytes of each of A and B. use_lanes: the groups of other precisions
// run in their lanes (otherwise every group runs on st in A and B, adding into f).
int run_all(DevicePlan* d, DevicePlan::ExecCtx* x, const HostPlan& hp, const double* c, int64_t ldc, double* f,
            int64_t ldf, int nrhs, void* A, void* B, void* partial, size_t capacity, bool chunk_from_capacity,
            cudaStream_t st, bool record, bool use_lanes) {
  if (x->cexp) {
    // FP32 and double-float stages run on the coefficients scaled by a power of two per vector
    // (from its largest |c_n|), so their range does not depend on the input's; FP64 stages use c
    StageScope sc(d, HANKEL_STAGE_GEN, st, record);
    launch_coef_exponent(c, ldc, d->hpN, nrhs, x->cexp, st);
    HK_LAUNCHED();
    sc.done(2, 0.0, 0.0);
  }
  if (x->cf) {
    // FP32 transforms (and FP32 near fields): the scaled coefficients rounded once per execution
    StageScope sc(d, HANKEL_STAGE_GEN, st, record);
    launch_coeffs_f32(c, ldc, x->cf, d->hpN, nrhs, x->cexp, st);
    HK_LAUNCHED();
    sc.done(1, 0.0, 0.0);
  }
  if (x->cdf) {
    // DF64 near fields and transforms: the scaled coefficients split once into float pairs
    StageScope sc(d, HANKEL_STAGE_GEN, st, record);
    launch_coeffs_df64(c, ldc, x->cdf, d->hpN, nrhs, x->cexp, st);
    HK_LAUNCHED();
    sc.done(1, 0.0, 0.0);
  }
  const bool lanes_on = use_lanes && d->nlanes > 1;
  const bool par = lanes_on && !d->timing;
  auto lane_stream = [&](int l) { return (par && l > 0) ? x->lanes[l].s : st; };
  if (lanes_on) {
    if (par) {
      // the other lanes start once the coefficient copies above are written
      if (cudaEventRecord(x->fork, st) != cudaSuccess) return HANKEL_ECUDA;
      for (int l = 1; l < d->nlanes; ++l)
        if (cudaStreamWaitEvent(x->lanes[l].s, x->fork, 0) != cudaSuccess) return HANKEL_ECUDA;
    }
    for (int l = 1; l < d->nlanes; ++l)
      if (cudaMemsetAsync(x->lanes[l].acc, 0, sizeof(double) * (size_t)nrhs * (size_t)d->hpN, lane_stream(l)) !=
          cudaSuccess)
        return HANKEL_ECUDA;
  }
  {
    StageScope sc(d, HANKEL_STAGE_NEAR, st, record);
    int64_t near_launches = d->nmrows > 0 ? 2 : 1;
    if (x->tcd && nrhs >= kNearTcMinRhs) {
      // the tensor-core near field takes 16 vectors per launch: groups of 16, and a last group of
      // fewer than kNearTcMinRhs vectors on the FMA kernels; the groups run one after another on
      // st and share the digit and partial-sum buffers
      near_launches = 0;
      for (int g0 = 0; g0 < nrhs; g0 += kNearTcRhs) {
        const int ng = std::min(kNearTcRhs, nrhs - g0);
        const double* cg = c + (int64_t)g0 * ldc;
        double* fg = f + (int64_t)g0 * ldf;
        if (ng >= kNearTcMinRhs) {
          launch_near_tc(d->df64, d->items, d->nitems, d->mrows, d->nmrows, d->nend, d->hpN, (double*)partial, ng,
                         cg, ldc, x->tcd, x->tce, d->tc_npad, fg, ldf, d->nodes.r_true, d->nodes.om_true, d->jtabq,
                         hp.jt_n, hp.jt_deg, st);
          near_launches += d->nmrows > 0 ? 3 : 2;
        } else if (d->df64) {
          launch_near_df(d->items, d->nitems, d->mrows, d->nmrows, d->nend, d->hpN, (double*)partial, ng,
                         x->cdf + (int64_t)g0 * d->hpN, fg, ldf, d->rdf, d->omdf, d->jtabdf, hp.jt_n, hp.jt_deg,
                         x->cexp + g0, st);
          near_launches += d->nmrows > 0 ? 2 : 1;
        } else {
          launch_near<double>(d->items, d->nitems, d->mrows, d->nmrows, d->nend, d->hpN, (double*)partial, ng, cg,
                              ldc, nullptr, fg, ldf, d->nodes.r_true, d->nodes.om_true, d->jtab, d->jtabq, hp.jt_n,
                              hp.jt_deg, nullptr, st);
          near_launches += d->nmrows > 0 ? 2 : 1;
        }
      }
    } else if (d->df64)
      launch_near_df(d->items, d->nitems, d->mrows, d->nmrows, d->nend, d->hpN, (double*)partial, nrhs, x->cdf, f,
                     ldf, d->rdf, d->omdf, d->jtabdf, hp.jt_n, hp.jt_deg, x->cexp, st);
    else if (d->fp32)
      launch_near<float>(d->items, d->nitems, d->mrows, d->nmrows, d->nend, d->hpN, (float*)partial, nrhs, c, ldc,
                         x->cf, f, ldf, d->rf, d->omf, d->jtabf, nullptr, hp.jt_n, hp.jt_deg, x->cexp, st);
    else
      launch_near<double>(d->items, d->nitems, d->mrows, d->nmrows, d->nend, d->hpN, (double*)partial, nrhs, c, ldc,
                          nullptr, f, ldf, d->nodes.r_true, d->nodes.om_true, d->jtab, d->jtabq, hp.jt_n,
                          hp.jt_deg, nullptr, st);
    HK_LAUNCHED();
    sc.done(near_launches, 0.0, (double)hp.near_count * nrhs);
  }
  for (const DevBlock& db : d->blocks) {
    for (int j = 0; j < db.ng; ++j) {
      const TermGroup& tg = db.g[j];
      const size_t esz = term_esz(tg.prec);
      const int l = lanes_on ? d->lane_of[tg.prec] : 0;
      const cudaStream_t ls = lane_stream(l);
      void* la = l ? x->lanes[l].A : A;
      void* lb = l ? x->lanes[l].B : B;
      double* lf = l ? x->lanes[l].acc : f;
      const int64_t lld = l ? d->hpN : ldf;
      const int64_t cap = chunk_from_capacity
                              ? std::max<int64_t>(1, (int64_t)(capacity / (column_footprint(db.b) * esz)))
                              : tg.cap;
      if (tg.prec == kTermFP32)
        HK_TRY(run_block<float2>(d, x, db, tg, c, ldc, lf, lld, nrhs, (float2*)la, (float2*)lb, cap, ls, record));
      else if (tg.prec == kTermDF64)
        HK_TRY(run_block<df64c>(d, x, db, tg, c, ldc, lf, lld, nrhs, (df64c*)la, (df64c*)lb, cap, ls, record));
      else
        HK_TRY(run_block<double2>(d, x, db, tg, c, ldc, lf, lld, nrhs, (double2*)la, (double2*)lb, cap, ls, record));
    }
  }
  if (lanes_on) {
    if (par)
      for (int l = 1; l < d->nlanes; ++l)
        if (cudaEventRecord(x->lanes[l].done, x->lanes[l].s) != cudaSuccess ||
            cudaStreamWaitEvent(st, x->lanes[l].done, 0) != cudaSuccess)
          return HANKEL_ECUDA;
    StageScope sc(d, HANKEL_STAGE_OUT, st, record);
    const double* acc[2] = {x->lanes[1].acc, d->nlanes > 2 ? x->lanes[2].acc : nullptr};
    launch_add_lanes(f, ldf, acc, d->nlanes - 1, d->hpN, nrhs, st);
    HK_LAUNCHED();
    sc.done(1, 0.0, 0.0, 8.0 * (double)(d->nlanes + 1) * (double)d->hpN * nrhs);
  }
  return HANKEL_OK;
}

}  // namespace

int dev_exec_ctx(hankel_plan_s* p, int k, const double* c, int64_t ldc, double* f, int64_t ldf, int nrhs,
                 void* stream) {
  DevicePlan* d = p->dev;
  if (k < 0 || k >= (int)d->ctx.size()) return HANKEL_EINVAL;
  DevicePlan::ExecCtx* x = d->ctx[k];
  cudaStream_t st = (cudaStream_t)stream;
  int cur = -1;
  cudaGetDevice(&cur);
  if (cur != d->device) cudaSetDevice(d->device);
  // near field overwrites f; far blocks add to it
  const int s = run_all(d, x, p->hp, c, ldc, f, ldf, nrhs, x->lanes[0].A, x->lanes[0].B, x->partial, 0, false, st, true,
                        true);
  if (cur >= 0 && cur != d->device) cudaSetDevice(cur);
  return s;
}

int dev_exec(hankel_plan_s* p, const double* c, int64_t ldc, double* f, int64_t ldf, int nrhs, void* stream) {
  return dev_exec_ctx(p, 0, c, ldc, f, ldf, nrhs, stream);
}

int dev_add_context(hankel_plan_s* p, int* index) {
  DevicePlan* d = p->dev;
  int cur = -1;
  cudaGetDevice(&cur);
  if (cur != d->device) cudaSetDevice(d->device);
  const int st = ctx_create(d, p->hp);
  if (cur >= 0 && cur != d->device) cudaSetDevice(cur);
  if (st != HANKEL_OK) {
    // the partial context keeps what it allocated until the plan is destroyed, but is never used
    cudaGetLastError();
    return st;
  }
  *index = (int)d->ctx.size() - 1;
  return HANKEL_OK;
}

int dev_contexts(const hankel_plan_s* p, size_t* ctx_bytes) {
  if (ctx_bytes) *ctx_bytes = p->dev ? p->dev->ctx_bytes : 0;
  return p->dev ? (int)p->dev->ctx.size() : 0;
}

int dev_set_timing(hankel_plan_s* p, int enable) {
  DevicePlan* d = p->dev;
  for (const auto& r : d->pending) cudaEventSynchronize(r.b);
  d->pending.clear();
  d->pool_used = 0;
  memset(d->acc, 0, sizeof(d->acc));
  d->timing = enable != 0;
  return HANKEL_OK;
}

int dev_stage_stats(hankel_plan_s* p, hankel_stage_stat* out) {
  DevicePlan* d = p->dev;
  for (const auto& r : d->pending) {
    if (cudaEventSynchronize(r.b) != cudaSuccess) return HANKEL_ECUDA;
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, r.a, r.b) != cudaSuccess) return HANKEL_ECUDA;
    d->acc[r.stage].ms += ms;
  }
  d->pending.clear();
  d->pool_used = 0;
  memcpy(out, d->acc, sizeof(d->acc));
  return HANKEL_OK;
}

int dev_exec_host(hankel_plan_s* p, const double* c, int64_t ldc, double* f, int64_t ldf, int nrhs) {
  const int64_t N = p->hp.opt.N;
  DevicePlan* d = p->dev;
  int cur = -1;
  cudaGetDevice(&cur);
  if (cur != d->device) cudaSetDevice(d->device);
  cudaStream_t st = 0;
  if (!d->c_stage) {  // staging buffers for host arrays, made on first use
    HK_TRY(dalloc(d, &d->c_stage, (size_t)N * p->hp.opt.max_nrhs));
    HK_TRY(dalloc(d, &d->f_stage, (size_t)N * p->hp.opt.max_nrhs));
  }
  if (cudaMemcpy2DAsync(d->c_stage, N * sizeof(double), c, ldc * sizeof(double), N * sizeof(double), nrhs,
                        cudaMemcpyHostToDevice, st) != cudaSuccess)
    return HANKEL_ECUDA;
  int s = dev_exec(p, d->c_stage, N, d->f_stage, N, nrhs, st);
  if (s != HANKEL_OK) return s;
  if (cudaMemcpy2DAsync(f, ldf * sizeof(double), d->f_stage, N * sizeof(double), N * sizeof(double), nrhs,
                        cudaMemcpyDeviceToHost, st) != cudaSuccess)
    return HANKEL_ECUDA;
  if (cudaStreamSynchronize(st) != cudaSuccess) return HANKEL_ECUDA;
  if (cur >= 0 && cur != d->device) cudaSetDevice(cur);
  return HANKEL_OK;
}

// Inverse DHT through the self-inverse relation of Section 6:
// c = j_{0,N+1}^{-2} v o (J (v o f)), v_n = 2 / J_1(j_{0,n})^2.
int dev_exec_inverse(hankel_plan_s* p, const double* f, int64_t ldf, double* c, int64_t ldc, int nrhs,
                     void* stream) {
  const HostPlan& hp = p->hp;
  const int64_t N = hp.opt.N;
  DevicePlan* d = p->dev;
  cudaStream_t st = (cudaStream_t)stream;
  int cur = -1;
  cudaGetDevice(&cur);
  if (cur != d->device) cudaSetDevice(d->device);
  if (!d->vinv) {  // made on first use (a host computation of J_1 at the roots)
    std::vector<double> v(N);
    dht_inverse_weights(N, hp.b.data(), v.data());
    HK_TRY(upload(d, &d->vinv, v.data(), v.size()));
    HK_TRY(dalloc(d, &d->inv_stage, (size_t)N * hp.opt.max_nrhs));
  }
  const double jN1 = (N + 0.75) * 3.14159265358979323846 + hp.b[N];
  launch_diag_scale(f, ldf, d->vinv, 1.0, d->inv_stage, N, N, nrhs, st);
  HK_LAUNCHED();
  int s = dev_exec(p, d->inv_stage, N, c, ldc, nrhs, stream);
  if (s != HANKEL_OK) return s;
  launch_diag_scale(c, ldc, d->vinv, 1.0 / (jN1 * jN1), c, ldc, N, nrhs, st);
  HK_LAUNCHED();
  if (cur >= 0 && cur != d->device) cudaSetDevice(cur);
  return HANKEL_OK;
}

// ---------------------------------------------------------------------------
// Allocation-free execution (hankel_exec_static)
//
// The same near-field and far-field launches as dev_exec for one vector, but the
// transform workspace -- the two FFT ping-pong column buffers and the near-field
// partial sums -- lives in the file-scope array below instead of memory the plan
// allocated. The array is placed on a device when this library's module is loaded
// there (at context creation with eager module loading, at the first lookup of its
// address with lazy loading, which plan creation does) and is kept until the process
// exits. Every element the launches read is written by an earlier launch of the
// same call, so nothing needs clearing between calls. All calls share the array:
// calls that overlap on the GPU (on different streams, or from different plans) race
// on it, and calls on one plan also share the plan's coefficient copies.
// ---------------------------------------------------------------------------
namespace {

constexpr size_t kStaticScratchElems = (size_t)HANKEL_STATIC_SCRATCH_BYTES / sizeof(double2);
constexpr int kMaxStaticDevices = 64;

static __device__ __align__(256) double2 g_static_scratch[kStaticScratchElems];

// Device address of g_static_scratch per device, looked up once with that device current.
double2* g_static_ptr[kMaxStaticDevices] = {};
bool g_static_ready[kMaxStaticDevices] = {};
std::mutex g_static_mu;

int static_scratch_address(int device, double2** out) {
  if (device < 0 || device >= kMaxStaticDevices) return HANKEL_EUNSUPPORTED;
  std::lock_guard<std::mutex> lock(g_static_mu);
  if (!g_static_ready[device]) {
    void* ptr = nullptr;
    if (cudaGetSymbolAddress(&ptr, g_static_scratch) != cudaSuccess) {
      cudaGetLastError();
      return HANKEL_ECUDA;
    }
    g_static_ptr[device] = (double2*)ptr;
    g_static_ready[device] = true;
  }
  *out = g_static_ptr[device];
  return HANKEL_OK;
}

}  // namespace

int dev_exec_static(hankel_plan_s* p, const double* c, double* f, void* stream) {
  const HostPlan& hp = p->hp;
  DevicePlan* d = p->dev;
  const int64_t N = hp.opt.N;
  // Layout of the static array (bytes): [bufA | bufB | near partial sums]; the partial sums
  // are doubles (floats for FP32 plans).
  const size_t total_bytes = (size_t)HANKEL_STATIC_SCRATCH_BYTES;
  const size_t partial_bytes = ((size_t)d->nslots + 1) * sizeof(double);
  size_t foot_max = 0;
  for (const DevBlock& db : d->blocks)
    for (int j = 0; j < db.ng; ++j)
      foot_max = std::max(foot_max, column_footprint(db.b) * term_esz(db.g[j].prec));
  if (2 * foot_max + partial_bytes > total_bytes) return HANKEL_EUNSUPPORTED;
  const size_t per_buf = ((total_bytes - partial_bytes) / 2) & ~(size_t)255;

  int cur = -1;
  cudaGetDevice(&cur);
  if (cur != d->device) cudaSetDevice(d->device);
  double2* base = nullptr;
  int st0 = static_scratch_address(d->device, &base);
  if (st0 != HANKEL_OK) {
    if (cur >= 0 && cur != d->device) cudaSetDevice(cur);
    return st0;
  }
  char* bytes = (char*)base;
  void* sA = bytes;
  void* sB = bytes + per_buf;
  void* spartial = bytes + 2 * per_buf;
  cudaStream_t st = (cudaStream_t)stream;
  const int s = run_all(d, d->ctx[0], hp, c, N, f, N, 1, sA, sB, spartial, per_buf, true, st, false, false);
  if (s != HANKEL_OK) {
    if (cur >= 0 && cur != d->device) cudaSetDevice(cur);
    return s;
  }
  if (cur >= 0 && cur != d->device) cudaSetDevice(cur);
  return HANKEL_OK;
}

}  // namespace hk
