/*
 * hankel.h -- C ABI of the GB300 (sm_103a) fast Hankel-type transform library.
 *
 * The library evaluates the sums of Townsend, "A fast analysis-based
 * discrete Hankel transform using asymptotic expansions" (arXiv:1501.01652),
 * Eq. (2):
 *
 *     f_k = sum_{n=1}^{N} c_n J_nu(r_k omega_n),   k = 1..N,
 *
 * for the three tasks of Section 1:
 *   HANKEL_SCHLOMILCH      omega_n = (n+gamma) pi (Section 4, Eq. 11; the
 *                          integer shift gamma is Remark 4.1's), any nu >= 0;
 *   HANKEL_FOURIER_BESSEL  omega_n = j_{0,n}, the n-th root of J_0
 *                          (Section 5, Eq. 20), any nu >= 0;
 *   HANKEL_DHT             the discrete Hankel transform of order 0
 *                          (Section 6, Eq. 25): nu = 0, omega_n = j_{0,n},
 *                          r_k = j_{0,k}/j_{0,N+1}.
 * For the first two tasks the sample points are r_k = (k-1)/(N-1)
 * (HANKEL_GRID_UNIT, the default) or the paper's r_k = k/N
 * (HANKEL_GRID_PAPER).
 *
 * Method (Sections 3-6): the N x N matrix J_nu(r omega^T) is split into a
 * near field, summed directly with J evaluated per entry, and the far-field
 * blocks of the recursive partition of Section 4.2 (Eq. 19), where J is
 * replaced by 2M terms of its Hankel expansion (Eq. 4) wrapped, for Bessel-
 * root nodes, in the truncated Neumann-addition/Taylor sums of Sections 5.1
 * and 6 (Eqs. 21, 22, 26). The parameters M, s_{nu,M}(eps), alpha, beta, P,
 * K and T come from the paper's Table 4 and Eqs. (23)-(24). Each far block
 * becomes one multi-column chirp-z transform on the GPU.
 *
 * Conventions shared by every call:
 *  - Index k and n are 1-based in the formulas; arrays are 0-based, so
 *    c[n-1] holds c_n and f[k-1] holds f_k.
 *  - Device pointers are CUDA global-memory pointers of the device the plan
 *    was created on; host pointers are ordinary pageable or pinned memory.
 *  - `stream` is a cudaStream_t passed as void* (NULL = the legacy default
 *    stream). Device-pointer calls are asynchronous and stream-ordered.
 *  - Return values are hankel_status codes; nothing is thrown across the ABI.
 *    On any code other than HANKEL_OK, output buffers hold unspecified data.
 *  - Executions of one plan serialise on its execution contexts: context 0
 *    (made with the plan, used by every call without a context argument)
 *    holds the workspace, so two executions on the same context must not
 *    overlap on the GPU. hankel_plan_add_context makes more contexts for
 *    executions in flight at once (hankel_exec_batched_ctx). Distinct plans
 *    are independent.
 */
#ifndef HANKEL_H
#define HANKEL_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Opaque plan handle. Owned by the caller from hankel_plan*() until hankel_destroy(). */
typedef struct hankel_plan_s* hankel_plan_t;

enum hankel_task {
  HANKEL_SCHLOMILCH = 0,
  HANKEL_FOURIER_BESSEL = 1,
  HANKEL_DHT = 2
};

enum hankel_grid {
  HANKEL_GRID_UNIT = 0,  /* r_k = (k-1)/(N-1) */
  HANKEL_GRID_PAPER = 1  /* r_k = k/N (Sections 4, 5) */
};

enum hankel_precision {
  HANKEL_PREC_AUTO = 0,  /* every stage in FP64 below eps = 1e-5; FP32 transform and near-field stages at
                            eps >= 1e-5 (the accuracy goal then admits FP32 rounding); nodes, phases and
                            plan tables are FP64 in every plan */
  HANKEL_PREC_FP64 = 1,  /* every stage in FP64 */
  HANKEL_PREC_FP32 = 2,  /* FP32 stages; refused (HANKEL_EUNSUPPORTED) when eps < 1e-5 */
  HANKEL_PREC_DF64 = 3,  /* transforms and spectrum products in double-float (pairs of FP32, ~48
                            significant bits), everything else FP64; refused when eps < 1e-11 */
  HANKEL_PREC_MIXED = 4  /* opt-in arithmetic narrower than FP64 below eps = 1e-5: DF64 plans for
                            1e-11 <= eps < 1e-5, FP64 plans below, FP32 stages at eps >= 1e-5; in FP64 and
                            DF64 plans each term of a block's low-rank form runs in the lowest precision
                            whose rounding bound (from the sums of the absolute Chebyshev coefficients of
                            its factors) stays within a quarter of the block's leading term in the plan
                            precision, or within eps / 200 of it (hankel_block.terms_*;
                            HANKEL_FLAG_UNIFORM_TERMS turns this lowering off) */
};

enum hankel_status {
  HANKEL_OK = 0,
  HANKEL_EINVAL = 1,        /* an argument is out of range or inconsistent */
  HANKEL_ENOMEM = 2,        /* a host or device allocation failed */
  HANKEL_ECUDA = 3,         /* a CUDA runtime call or kernel launch failed */
  HANKEL_EUNSUPPORTED = 4,  /* a valid request this build does not serve */
  HANKEL_ETIMEOUT = 5,      /* a bounded device wait expired */
  HANKEL_ECANCELED = 6      /* a queued request was cancelled before it ran (hankel_server_cancel) */
};

/* Plan flags (hankel_options.flags). */
#define HANKEL_FLAG_HOST_ONLY 1u   /* build host tables only; no CUDA call is made */
#define HANKEL_FLAG_NO_SEGMENT 2u  /* one full-length chirp-z transform per block (no segmenting of thin blocks) */
#define HANKEL_FLAG_ALL_COLUMNS 8u /* every block keeps all ncols stacked columns; by default a block leaves
                                      out the columns whose summed bound on its entries stays within
                                      eps per entry, split over the blocks of a row (hankel_block.ncols,
                                      hankel_info.block_cols) */
#define HANKEL_FLAG_NO_LOWRANK 32u /* every block transforms its kept stacked columns; by default a block whose
                                      kernel has a low-rank form exact to eps/2 (Chebyshev interpolation
                                      in log k, log n and cross approximation) transforms its rank instead
                                      (hankel_block.ncols, .kept, .lowrank_err) */
#define HANKEL_FLAG_NO_REFINE 16u  /* keep the blocks of Eq. (19) as they are; by default a block is cut into
                                      smaller ones where that lowers the estimated work (fewer kept columns
                                      away from the near field) */
#define HANKEL_FLAG_UNIFORM_TERMS 64u /* MIXED plans: every far-field term in the plan precision (no per-term
                                         lowering of small low-rank terms) */
#define HANKEL_FLAG_NO_AUTOTUNE 128u /* split every transform into launches by the built-in rule; by default
                                        the plan measures the candidate splits of each transform length it
                                        runs (hankel_fft_shape) once per GPU model and uses the fastest */
#define HANKEL_FLAG_TENSOR_FFT 256u  /* FP64 transforms of 2^12 points or more run as many of their passes as
                                        their length allows as radix-32 passes on the tensor cores (split-digit
                                        products in FP64 accuracy), the rest on the FP64 pipe, without
                                        autotuning; the autotuner otherwise weighs these splits with the others */

/* Options for hankel_plan_ex(). Fill with hankel_options_default() first. */
typedef struct {
  int task;               /* enum hankel_task */
  int nu;                 /* order of J; >= 0; must be 0 for HANKEL_DHT (Section 6 builds the order-0
                             DHT on the nodes j_{0,n}; other orders are refused with EINVAL) */
  int64_t N;              /* number of coefficients and of outputs; 2 <= N <= 2^24 */
  double eps;             /* working accuracy, 1e-16 <= eps < 1 */
  int grid;               /* enum hankel_grid (tasks 0 and 1 only) */
  int64_t gamma;          /* Schlomilch shift: omega_n = (n+gamma) pi; default nu */
  int precision;          /* enum hankel_precision */
  int max_nrhs;           /* largest nrhs a batched call will pass; >= 1 */
  unsigned flags;         /* HANKEL_FLAG_* */
  size_t workspace_limit; /* device bytes the plan may use for FFT columns; 0 = default (4 GiB) */
} hankel_options;

/* Parameters a plan chose (Table 4, Eqs. 23-24) and its sizes. */
typedef struct {
  int task, nu, grid, precision;
  int64_t N, gamma;
  double eps;
  int M;                  /* terms of the Hankel expansion, Eq. (4): 2M terms */
  int mu_max;             /* largest |order| met by the expansion in this task */
  double s;               /* s_{mu_max,M}(eps), Section 3.1 */
  double alpha, beta;     /* partition parameters, Table 4 */
  int P;                  /* number of partition levels, Table 4 */
  int K, T;               /* Neumann / Taylor truncation for the row perturbation (DHT) or column perturbation (FB) */
  int K2, T2;             /* column-perturbation truncation of the DHT (equal to K, T otherwise) */
  int64_t direct_rows;    /* leading rows summed directly (DHT, Section 6) */
  int64_t direct_cols;    /* leading columns summed directly (FB and DHT, Section 5) */
  int nblocks;            /* far-field blocks actually used (1 + 2P at most) */
  int ncols;              /* stacked transform columns per block per right-hand side */
  int npairs;             /* Schlomilch-type evaluations in the paper's count: 1, 2T+K-2 or (2T+K-2)^2 */
  int64_t near_count;     /* matrix entries summed directly */
  int64_t far_count;      /* matrix entries covered by far-field blocks */
  double near_zmax;       /* largest argument r_k omega_n in the near field */
  size_t device_bytes;    /* device memory held by the plan (tables + workspace) */
  size_t workspace_bytes; /* part of device_bytes used as transform workspace */
  int64_t block_cols;     /* transforms per right-hand side summed over blocks (hankel_block.ncols) */
  int fft_shapes;         /* distinct (precision, length, column bucket) transform shapes the plan runs
                             (hankel_plan_fft_shapes) */
  int contexts;           /* execution contexts (1 + those added by hankel_plan_add_context) */
  size_t context_bytes;   /* device bytes of one execution context (workspace, partial sums, coefficient
                             copies), included in device_bytes */
} hankel_info;

/* How one kind of multi-column FFT of the far field is split into kernel launches. Not a step of
 * the paper (whose transforms are DCT/DST library calls); the autotuner of this library measures
 * the candidates on the GPU. */
typedef struct {
  int precision;       /* arithmetic of the transform: HANKEL_PREC_FP64, _DF64 or _FP32 */
  int log2_len;        /* log2 of the transform length F */
  int col_bucket;      /* floor(log2(columns per launch)), clamped to 0..16 (hankel_tune_bucket) */
  int one_launch;      /* 1: the whole transform in one launch (F <= 4096) */
  int npass;           /* otherwise 2..4 passes, */
  int log2_radix[4];   /* of radix 2^log2_radix[i] (5..8 each, summing to log2_len), first to last */
  int tensor_passes;   /* bit i: pass i runs on the tensor cores (radix 32, FP64 transforms of 2^12 points or
                          more; split-digit products in FP64 accuracy), else on the FP64 pipe */
  double ms_default;   /* measured time of the built-in split on the tuning columns (0: not measured) */
  double ms_chosen;    /* measured time of the chosen split */
} hankel_fft_shape;

/* One far-field block of the partition, 1-based inclusive index ranges. */
typedef struct {
  int64_t k0, k1;  /* rows */
  int64_t n0, n1;  /* columns */
  int64_t fft_len; /* length F of its FFTs, a power of two */
  int64_t seg_len; /* segment length S of the long side (= columns for an unsegmented block) */
  int64_t nseg;    /* number of segments (1 = one transform with F >= rows + cols - 1) */
  int mode;        /* 0 unsegmented; 1 columns segmented (overlap-add), F >= rows + S - 1;
                      2 rows segmented (overlap-save), F >= S + cols - 1 */
  int ncols;       /* transforms this block runs per right-hand side: its low-rank form's rank, or its
                      kept stacked columns when it has no low-rank form */
  double dropped;  /* bound on the change of any entry of the block from the columns it leaves out */
  int kept;        /* stacked columns the block keeps (<= hankel_info.ncols) */
  int lowrank;     /* 1 when the block runs its low-rank form */
  double lowrank_err; /* largest error of the low-rank form on its validation entries (<= eps/2) */
  int terms_fp64;  /* of its ncols transforms per right-hand side: those run in FP64, */
  int terms_df64;  /* in double-float */
  int terms_fp32;  /* and in FP32 */
} hankel_block;

/* Fill *o with defaults for (task, nu, N, eps). Host only. Returns HANKEL_OK or HANKEL_EINVAL (o == NULL). */
int hankel_options_default(hankel_options* o, int task, int nu, int64_t N, double eps);

/* Create a plan with default options on the current CUDA device.
 * Computes parameters, nodes (j_{0,n} as (n, b_n)), the partition, weight
 * tables and chirp spectra, and allocates the workspace. Blocking. */
int hankel_plan(hankel_plan_t* out, int task, int nu, int64_t N, double eps);

/* Create a plan from options. With HANKEL_FLAG_HOST_ONLY no CUDA call is made and
 * only hankel_plan_info / hankel_plan_blocks / hankel_plan_entry / hankel_destroy
 * accept the plan. Errors: EINVAL (bad option), EUNSUPPORTED (eps < 1e-16, FP32 asked
 * at eps < 1e-5), ENOMEM, ECUDA. *out is NULL on error. */
int hankel_plan_ex(hankel_plan_t* out, const hankel_options* opts);

/* f = J_nu(r omega^T) c for one vector. c and f are device arrays of N doubles
 * (c read, f overwritten); they may not overlap. Asynchronous on `stream`. */
int hankel_exec(hankel_plan_t p, const double* c, double* f, void* stream);

/* Batched form: for r < nrhs, f[r*ldf + k-1] = sum_n c[r*ldc + n-1] J_nu(r_k omega_n).
 * Device arrays; ldc, ldf >= N; 1 <= nrhs <= max_nrhs of the plan. Asynchronous.
 * FP64 and DF64 plans built with max_nrhs >= 8 sum the near field of calls with nrhs >= 8 as
 * exact split-digit products on the tensor cores (J and each 512-column chunk of c rounded to
 * 2^-53 and 2^-54 of their scales), 16 vectors per launch, a last group of fewer than 8 vectors
 * on the FMA kernels: the results differ from a call with fewer vectors in the last bits, and
 * are at least as close to the exact sums (checked against the oracle). FP32 and double-float
 * stages work on each vector scaled by a power of two from its largest |c_n| and scale their
 * sums back, so their range does not depend on the input's. */
int hankel_exec_batched(hankel_plan_t p, const double* c, int64_t ldc, double* f, int64_t ldf,
                        int nrhs, void* stream);

/* Another execution context for the plan: a second copy of the per-execution scratch (transform
 * workspace, lane streams and accumulators, near-field partial sums, coefficient copies; the
 * plan's tables are shared). Executions on different contexts of one plan may be in flight at
 * the same time, on different streams. *index receives the new context's index (1, 2, ...).
 * Blocking (allocates device memory). Errors: EINVAL (NULL, host-only plan), ENOMEM, ECUDA;
 * after an error the plan and its earlier contexts stay usable. This is a service of the library
 * (a serving layer runs batches of one plan side by side); the paper has no counterpart. */
int hankel_plan_add_context(hankel_plan_t p, int* index);

/* hankel_exec_batched on execution context ctx (0 <= ctx < hankel_info.contexts). */
int hankel_exec_batched_ctx(hankel_plan_t p, int ctx, const double* c, int64_t ldc, double* f, int64_t ldf,
                            int nrhs, void* stream);

/* Size of the library's static device scratch array used by hankel_exec_static (96 MiB). */
#define HANKEL_STATIC_SCRATCH_BYTES (96u << 20)

/* Allocation-free execution. The paper has no counterpart; this is a service of the library.
 * Computes the same f as hankel_exec(p, c, f, stream) for one vector (device arrays of N
 * doubles, asynchronous on `stream`), but the call itself allocates no memory: it calls no
 * cudaMalloc, cudaFree or other allocating routine. The transform workspace (the FFT column
 * buffers and the near-field partial sums) comes from one file-scope device array of
 * HANKEL_STATIC_SCRATCH_BYTES. It is meant for callers that cannot allocate device memory when
 * they run a transform: services whose device memory is all handed to their own pool allocator,
 * and latency-critical loops that must not enter the CUDA allocator. The plan's own tables are
 * still made by hankel_plan*, ahead of time.
 *  - Where the array lives: a device holds it from the moment this library's module is loaded
 *    there until the process exits. With eager module loading that is context creation; with
 *    lazy loading (the CUDA default) it is the first lookup of the array's address, which
 *    hankel_plan* does on the plan's device, with that device current. Create the plan before
 *    handing the device's memory to a pool.
 *  - Should that lookup fail at plan creation (the plan is still made), the first
 *    hankel_exec_static call on the device retries it; that call then does the set-up and must
 *    come before any stream capture begins.
 *  - All calls share the array and its contents persist between calls; every element a call
 *    reads is written earlier in the same call, so no clearing is needed. Calls that overlap
 *    on the GPU (other streams, other plans) race on the array, and any two calls on one plan
 *    (through this or another execution entry point) share the plan's coefficient copies: order
 *    them on one stream.
 *  - Returns HANKEL_EUNSUPPORTED when the plan's largest transform needs more than the array
 *    holds (two columns of F complex values of the plan's precision plus the near-field
 *    partial sums; in practice N up to about 2^20 for an FP64 DHT, twice that for FP32 plans),
 *    HANKEL_EINVAL on NULL arguments or a host-only plan, HANKEL_ECUDA if a launch or the
 *    address lookup fails. */
int hankel_exec_static(hankel_plan_t p, const double* c, double* f, void* stream);

/* End-to-end form with HOST arrays (same layout as hankel_exec_batched): copies c to the
 * device, runs the transform and copies f back. Blocks until f is written. */
int hankel_exec_host(hankel_plan_t p, const double* c, int64_t ldc, double* f, int64_t ldf, int nrhs);

/* Parameters and sizes of a plan. Host only. */
int hankel_plan_info(hankel_plan_t p, hankel_info* out);

/* Copy up to `cap` far-field blocks into out; *count receives the number of blocks. Host only. */
int hankel_plan_blocks(hankel_plan_t p, hankel_block* out, int cap, int* count);

/* Inverse DHT (a second workload of Section 6): c = j_{0,N+1}^{-2} D_v J_0(j_0 j_0^T/j_{0,N+1}) D_v f
 * with v_n = 2/J_1(j_{0,n})^2, the self-inverse relation of the DHT matrix (Section 6, which
 * uses it to test the transform). The relation holds as N -> infinity: for Gaussian f the
 * round trip inverse(forward(c)) - c falls like O(N^-2) for small N and then grows like
 * O(N^{3/2}) from rounding (the paper's Figure on this test). One forward DHT of v o f plus two
 * diagonal scalings on `stream`; device arrays f [nrhs][ldf] (read) and c [nrhs][ldc]
 * (written), which must not overlap. DHT plans only. The first call computes v on the host
 * and allocates N*(1+max_nrhs) doubles on the device; it is blocking. Errors: EINVAL (not a
 * DHT plan, host-only plan, bad sizes), ENOMEM, ECUDA. */
int hankel_exec_inverse(hankel_plan_t p, const double* f, int64_t ldf, double* c, int64_t ldc, int nrhs,
                        void* stream);

/* v_n = 2/J_1(j_{0,n})^2 for n = 1..N (the weights of the inverse DHT), from j_{0,n} carried as
 * (n, b_n): Eq. (4) for nu = 1 with its phase reduced to b_n for large roots, Miller's
 * recurrence in double-double for small ones. Host only. Errors: EINVAL. */
int hankel_dht_inverse_weights(int64_t N, double* v);

/* Host evaluation of the plan's representation of matrix entry (k, n), 1-based:
 * *value receives the number the plan uses for J_nu(r_k omega_n) (the near-field
 * evaluator or the far-field expansion) and *is_far is 1 when (k, n) lies in a
 * far-field block. Slow; for tests. Host only. */
int hankel_plan_entry(hankel_plan_t p, int64_t k, int64_t n, double* value, int* is_far);

/* Host evaluation of the far-field expansion (Eq. 4 with the Neumann/Taylor sums of Eqs. 21-22
 * and 26, every stacked column) at entry (k, n), 1-based, wherever the entry lies: the value
 * the transform would use if the partition of Eq. (19) were dropped and the expansion applied
 * to every entry. Where z = r_k omega_n is below s_{nu,M} it is not eps-accurate (Section 3.1;
 * at r_k = 0 it is not finite). For tests of the partition. Host only. Errors: EINVAL. */
int hankel_plan_expansion_entry(hankel_plan_t p, int64_t k, int64_t n, double* value);

/* The transform shapes a plan runs: up to `cap` entries into out, *count receives the number.
 * Each says how the plan's transforms of one precision, length and column bucket are split into
 * launches, and the times the autotuner measured (zero when the shape came from the built-in rule
 * or from the cache without a measurement in this process). Host only. */
int hankel_plan_fft_shapes(hankel_plan_t p, hankel_fft_shape* out, int cap, int* count);

/* Status of the plan's bounded device waits since the last call: HANKEL_OK, or HANKEL_ETIMEOUT when a
 * tensor-core transform pass gave up waiting for its operand copy or its products (its outputs
 * are then unspecified). Blocking (reads one word from the device); clears the status. */
int hankel_plan_device_status(hankel_plan_t p);

/* The autotuner's shape cache, keyed by (GPU name, precision, log2_len, col_bucket). Plans look a
 * key up before measuring it, and store what they measure. When the environment variable
 * HANKEL_TUNE_CACHE names a file, the first plan of the process loads it and every new entry is
 * appended to it. Host only; no GPU needed. Errors: EINVAL (NULL or empty name, a name with a
 * newline, an unreadable or unwritable path). */
int hankel_tune_cache_put(const char* gpu_name, const hankel_fft_shape* s);
int hankel_tune_cache_get(const char* gpu_name, int precision, int log2_len, int col_bucket, hankel_fft_shape* out,
                          int* found);
int hankel_tune_cache_save(const char* path);
int hankel_tune_cache_load(const char* path);
int hankel_tune_cache_clear(void);
/* The column bucket of a launch of ncols columns: floor(log2(ncols)) clamped to 0..16. */
int hankel_tune_bucket(int64_t ncols);

/* Near-field prefix of row k (1-based): columns 1..*nend are summed directly. Host only. */
int hankel_plan_near_prefix(hankel_plan_t p, int64_t k, int64_t* nend);

/* Execution stages of a plan, for hankel_plan_stage_stats(). */
enum hankel_stage {
  HANKEL_STAGE_NEAR = 0,      /* near-field direct sum (and its partial-sum combine) */
  HANKEL_STAGE_GEN = 1,       /* per-execution coefficient conversion of FP32 and DF64 plans (the
                                 far-field column generation itself runs in the first forward FFT loads) */
  HANKEL_STAGE_FFT = 2,       /* forward and inverse multi-column FFT passes of FP64 transforms, with the
                                 column generation and the single spectrum products folded into their
                                 first loads */
  HANKEL_STAGE_POINTWISE = 3, /* summed products of segment spectra and chirp spectra (column-segmented
                                 blocks) */
  HANKEL_STAGE_OUT = 4,       /* row weights and accumulation into f */
  HANKEL_STAGE_FFT_DF64 = 5,  /* the FFT passes of double-float transforms */
  HANKEL_STAGE_FFT_FP32 = 6,  /* the FFT passes of FP32 transforms */
  HANKEL_STAGE_COUNT = 7
};

/* Accumulated statistics of one stage since timing was (re)enabled. */
typedef struct {
  double ms;         /* summed kernel time from CUDA events on the execution stream (0 when timing is off) */
  double flops;      /* algorithmic floating-point operations (FFT: 5 F log2 F per column transform;
                        segment sums: 8 per point and segment; row sums: 4 per column and row) */
  double entries;    /* near field: matrix entries evaluated (times right-hand sides) */
  double bytes;      /* algorithmic DRAM bytes: FFT, each pass reads and writes every point once (32 B
                        per FP64 point); segment sums and row sums, every operand read once and every
                        result written once (0 for the other stages) */
  int64_t launches;  /* kernel launches */
} hankel_stage_stat;

/* Enable (1) or disable (0) per-stage event timing for later executions of p and reset the
 * accumulated statistics. Launch counts are accumulated in both modes. Host call. */
int hankel_plan_set_timing(hankel_plan_t p, int enable);

/* Copy the accumulated statistics of every stage into out[HANKEL_STAGE_COUNT]. Waits for the
 * recorded events of earlier executions to complete. Host call. */
int hankel_plan_stage_stats(hankel_plan_t p, hankel_stage_stat* out);

/* Release a plan and all memory it holds. NULL is accepted. Synchronises the plan's device work. */
int hankel_destroy(hankel_plan_t p);

/* Static, NUL-terminated description of a status code. Never NULL. */
const char* hankel_status_string(int status);

/* ---- Serving: a request loop over cached plans ----
 *
 * A server owns a dispatcher thread, a set of CUDA streams and a cache of plans keyed by
 * (task, nu, N, eps). Requests carry host arrays of coefficients; the dispatcher admits them
 * by device memory, packs the waiting requests of one plan (up to max_batch vectors) into
 * one batched execution, and runs batches concurrently on its streams: batches of different
 * plans, and up to contexts_per_plan batches of one plan, each on an execution context of its
 * own (so a request for a plan already on the GPU is admitted as a stream and a context free up). Completed results are copied
 * to the request's host output array and the request's latency (submit to completion) is
 * recorded. This layer is a service around the paper's transform, not part of the paper. */
typedef struct hankel_server_s* hankel_server_t;

typedef struct {
  size_t memory_cap;  /* device bytes the server's plans and buffers may hold (0 = 120 GiB) */
  int streams;        /* CUDA streams, i.e. batches in flight at once (default 4, at most 16) */
  int max_batch;      /* most coefficient vectors packed into one execution (default 64) */
  int use_graphs;     /* 1: replay each (plan, batch size, stream, context) launch sequence from a CUDA graph,
                         captured at its second use (its first runs uncaptured) */
  int precision;      /* precision every plan is built with: HANKEL_PREC_AUTO (FP64 below eps = 1e-5, FP32
                         stages at or above), HANKEL_PREC_FP64, or HANKEL_PREC_MIXED (chosen per eps and
                         per term as for a MIXED plan) */
  int pack_requests;  /* 1: pack waiting requests of one plan into one execution; 0: one request each */
  int batch_window_us; /* a plan's batch with fewer than max_batch vectors waits until no request of the
                          plan has arrived for this long (so a burst of submissions stays one batch),
                          or until its oldest request has waited ten times this (default 200; 0: none) */
  int contexts_per_plan; /* batches of one plan in flight at once, each on an execution context of its own
                            (hankel_plan_add_context; made when needed and the memory cap allows; default
                            2, 1..8) */
  int small_batch;       /* 1..max_batch - 1: a batch of at most this many vectors runs on a second plan of
                            its (task, nu, N, eps), built for that many (a plan built for max_batch runs one
                            vector about 15 % slower); 0 (default): one plan per (task, nu, N, eps) */
} hankel_server_options;

/* Statistics since the server was created. */
typedef struct {
  int64_t submitted, completed, failed;  /* requests (failed includes cancelled) */
  int64_t batches;                       /* batched executions launched */
  int64_t vectors;                       /* coefficient vectors transformed */
  double coefficients;                   /* sum over completed requests of N * nrhs */
  int64_t plans_built, plans_evicted;    /* plan cache activity */
  int64_t graphs_captured;               /* CUDA graphs captured */
  size_t device_bytes;                   /* device memory held now */
  int64_t contexts_added;                /* execution contexts added to cached plans (beyond their first) */
  int64_t cancelled;                     /* requests cancelled before they ran */
} hankel_server_stats;

/* Defaults: 120 GiB cap, 4 streams, batches of up to 64 vectors, no graphs, AUTO precision, packing on,
 * a 200 us batch window, 2 contexts per plan. */
int hankel_server_options_default(hankel_server_options* o);

/* Create a server on the current CUDA device and start its dispatcher. */
int hankel_server_create(hankel_server_t* out, const hankel_server_options* o);

/* Queue one request: nrhs vectors of N coefficients in host array c (row r at c + r*N) and the
 * host output array f (same layout). Both must stay valid until the request completes. Page-locked
 * arrays (cudaMallocHost, cudaHostRegister) are copied to and from the device directly; pageable
 * ones through the server's page-locked staging buffers. *ticket receives the request's id.
 * Never blocks on the GPU. Errors: EINVAL (arguments), EUNSUPPORTED (a plan could not be built
 * for these parameters, reported at completion as a failed request). */
int hankel_server_submit(hankel_server_t s, int task, int nu, int64_t N, double eps, const double* c, double* f,
                         int nrhs, int64_t* ticket);

/* Block until request `ticket` completes. *status receives its hankel_status, *latency_ms the
 * time from submission to completion (either pointer may be NULL). */
int hankel_server_wait(hankel_server_t s, int64_t ticket, int* status, double* latency_ms);

/* Cancel a request that is still waiting for dispatch: it completes at once with status
 * HANKEL_ECANCELED and its arrays are not touched again. A request already in a batch on the GPU
 * (or finished) is not affected; *cancelled (may be NULL) tells which happened. Errors: EINVAL. */
int hankel_server_cancel(hankel_server_t s, int64_t ticket, int* cancelled);

/* Block until every submitted request has completed. */
int hankel_server_drain(hankel_server_t s);

int hankel_server_get_stats(hankel_server_t s, hankel_server_stats* out);

/* Stop the dispatcher after draining, and free every plan, stream and buffer. NULL is accepted. */
int hankel_server_destroy(hankel_server_t s);

/* ---- Fault injection for tests (host side; no GPU fault is made) ----
 * After `after` more successful device or page-locked allocations by this library, the next
 * `count` allocations report failure as if the CUDA allocator had refused them (the call returns
 * HANKEL_ENOMEM, or a server request completes with it). count = 0 turns injection off.
 * Process-wide; for tests of the error paths of plan creation and request admission. */
int hankel_debug_fail_allocs(int64_t after, int64_t count);

/* Test access to the multi-column FFT of the far field: ncols columns of 2^log2_len seeded
 * pseudo-random FP64 complex values are transformed (forward, or inverse when inverse != 0) by the
 * built-in FP64 split and by the given one (npass passes of radix 2^log2_radix[i], tensor_passes a
 * bit mask of passes on the tensor cores, as in hankel_fft_shape). *err receives
 * max |difference| / max |built-in result|, *ms the time of the given split (fastest of three
 * runs). Allocates and frees its own device memory; blocking. Errors: EINVAL (a split that is not
 * valid for the length), ENOMEM, ECUDA, ETIMEOUT (a tensor-core pass gave up a wait). */
int hankel_debug_fft_compare(int log2_len, int ncols, int inverse, int npass, const int* log2_radix,
                             int tensor_passes, double* err, double* ms);

/* ---- Host-only parameter formulas (no plan, no GPU) ---- */

/* s_{nu,M}(eps): four fixed-point iterations from s = 1 (Section 3.1, Table 1). */
double hankel_s_nu_M(int nu, int M, double eps);
/* t_{nu,T}(eps) ~ (2^{2T+nu} (T+nu)! T! eps)^{1/(2T+nu)} (Section 3.2, Table 2). */
double hankel_t_nu_T(int nu, int T, double eps);
/* Largest |dz| with 5.2 (e|dz|/2)^K <= eps: (2/e)(eps/5.2)^{1/K} (Eq. 10, Table 3). */
double hankel_neumann_radius(int K, double eps);
/* p_K(eps) of Eq. (23) and q_T(eps) of Eq. (24). */
double hankel_p_K(int K, double eps);
double hankel_q_T(int T, double eps);
/* Parameters a plan with these options would choose, without building it. */
int hankel_params(const hankel_options* opts, hankel_info* out);
/* b[n-1] = j_{0,n} - (n-1/4) pi for n = 1..count (Lemma 3.2), computed to full FP64
 * relative accuracy (host only; b must hold count doubles). Returns HANKEL_EINVAL if
 * count < 1 or b == NULL. */
int hankel_j0_zero_offsets(int64_t count, double* b);

#ifdef __cplusplus
}
#endif
#endif /* HANKEL_H */
