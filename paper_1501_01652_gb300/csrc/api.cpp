// C ABI entry points (include/hankel.h): argument checking, plan lifetime,
// host-only queries. Device work is delegated to the CUDA translation units.
#include <stdlib.h>
#include <string.h>

#include <vector>

#include <atomic>
#include <new>

#include "device.h"
#include "plan.h"

namespace hk {
namespace {
std::atomic<int64_t> g_fault_after{0}, g_fault_count{0};
}
bool alloc_fault() {
  if (g_fault_count.load() <= 0) return false;
  if (g_fault_after.fetch_sub(1) > 0) return false;
  g_fault_after.store(0);
  return g_fault_count.fetch_sub(1) > 0;
}
}  // namespace hk

extern "C" {

int hankel_debug_fail_allocs(int64_t after, int64_t count) {
  if (after < 0 || count < 0) return HANKEL_EINVAL;
  hk::g_fault_count.store(0);
  hk::g_fault_after.store(after);
  hk::g_fault_count.store(count);
  return HANKEL_OK;
}

const char* hankel_status_string(int status) {
  switch (status) {
    case HANKEL_OK: return "success";
    case HANKEL_EINVAL: return "invalid argument";
    case HANKEL_ENOMEM: return "out of memory";
    case HANKEL_ECUDA: return "CUDA error";
    case HANKEL_EUNSUPPORTED: return "unsupported request";
    case HANKEL_ETIMEOUT: return "device wait timed out";
    case HANKEL_ECANCELED: return "request cancelled";
    default: return "unknown status";
  }
}

int hankel_options_default(hankel_options* o, int task, int nu, int64_t N, double eps) {
  if (!o) return HANKEL_EINVAL;
  memset(o, 0, sizeof(*o));
  o->task = task;
  o->nu = nu;
  o->N = N;
  o->eps = eps;
  o->grid = HANKEL_GRID_UNIT;
  o->gamma = (task == HANKEL_SCHLOMILCH) ? nu : 0;
  o->precision = HANKEL_PREC_AUTO;
  o->max_nrhs = 1;
  o->flags = 0;
  o->workspace_limit = 0;
  return HANKEL_OK;
}

static void fill_info(const hankel_plan_s* p, const hk::HostPlan& hp, hankel_info* out) {
  memset(out, 0, sizeof(*out));
  out->task = hp.opt.task;
  out->nu = hp.opt.nu;
  out->grid = hp.opt.grid;
  out->precision = hp.fp32 ? HANKEL_PREC_FP32 : hp.df64 ? HANKEL_PREC_DF64 : HANKEL_PREC_FP64;
  out->N = hp.opt.N;
  out->gamma = hp.opt.gamma;
  out->eps = hp.opt.eps;
  out->M = hp.M;
  out->mu_max = hp.mu_max;
  out->s = hp.s;
  out->alpha = hp.alpha;
  out->beta = hp.beta;
  out->P = hp.P;
  out->K = hp.K;
  out->T = hp.T;
  out->K2 = hp.K2;
  out->T2 = hp.T2;
  out->direct_rows = hp.nrd;
  out->direct_cols = hp.ncd;
  out->nblocks = (int)hp.blocks.size();
  out->ncols = (int)hp.cols.size();
  if (hp.opt.task == HANKEL_SCHLOMILCH) out->npairs = 1;
  else if (hp.opt.task == HANKEL_FOURIER_BESSEL) out->npairs = hp.U2;
  else out->npairs = hp.U1 * hp.U2;
  if (out->ncols == 0) {
    // parameters only: the count the planner would build
    out->ncols = hp.U1 * (2 * hp.M + hp.U2 - 1);
  }
  out->block_cols = 0;
  for (const hk::Block& b : hp.blocks) out->block_cols += b.rank ? b.rank : (int64_t)b.lcols.size();
  out->near_count = hp.near_count;
  out->far_count = hp.far_count;
  out->near_zmax = hp.zmax;
  if (p) {
    out->device_bytes = hk::dev_plan_bytes(p);
    out->workspace_bytes = hk::dev_workspace_bytes(p);
    hk::dev_plan_shapes(p, nullptr, 0, &out->fft_shapes);
    out->contexts = hk::dev_contexts(p, &out->context_bytes);
  }
}

int hankel_j0_zero_offsets(int64_t count, double* b) {
  if (count < 1 || !b) return HANKEL_EINVAL;
  hk::j0_zero_offsets(count, b);
  return HANKEL_OK;
}

int hankel_params(const hankel_options* opts, hankel_info* out) {
  if (!opts || !out) return HANKEL_EINVAL;
  hk::HostPlan hp;
  int st = hk::choose_params(*opts, hp);
  if (st != HANKEL_OK) return st;
  fill_info(nullptr, hp, out);
  return HANKEL_OK;
}

int hankel_plan_ex(hankel_plan_t* out, const hankel_options* opts) {
  if (!out) return HANKEL_EINVAL;
  *out = nullptr;
  if (!opts) return HANKEL_EINVAL;
  hankel_plan_s* p = new (std::nothrow) hankel_plan_s();
  if (!p) return HANKEL_ENOMEM;
  int st;
  try {
    st = hk::build_host_plan(*opts, p->hp);
  } catch (const std::bad_alloc&) {
    st = HANKEL_ENOMEM;
  }
  if (st != HANKEL_OK) {
    delete p;
    return st;
  }
  p->host_only = (opts->flags & HANKEL_FLAG_HOST_ONLY) != 0;
  if (!p->host_only) {
    st = hk::dev_plan_create(p);
    if (st != HANKEL_OK) {
      hk::dev_plan_destroy(p);
      delete p;
      return st;
    }
  }
  *out = p;
  return HANKEL_OK;
}

int hankel_plan(hankel_plan_t* out, int task, int nu, int64_t N, double eps) {
  hankel_options o;
  hankel_options_default(&o, task, nu, N, eps);
  return hankel_plan_ex(out, &o);
}

int hankel_destroy(hankel_plan_t p) {
  if (!p) return HANKEL_OK;
  int st = HANKEL_OK;
  if (!p->host_only) st = hk::dev_plan_destroy(p);
  delete p;
  return st;
}

int hankel_plan_info(hankel_plan_t p, hankel_info* out) {
  if (!p || !out) return HANKEL_EINVAL;
  fill_info(p->host_only ? nullptr : p, p->hp, out);
  return HANKEL_OK;
}

int hankel_plan_blocks(hankel_plan_t p, hankel_block* out, int cap, int* count) {
  if (!p || !count || cap < 0 || (cap > 0 && !out)) return HANKEL_EINVAL;
  const auto& bl = p->hp.blocks;
  *count = (int)bl.size();
  for (int i = 0; i < cap && i < (int)bl.size(); ++i) {
    out[i].k0 = bl[i].k0;
    out[i].k1 = bl[i].k1;
    out[i].n0 = bl[i].n0;
    out[i].n1 = bl[i].n1;
    out[i].fft_len = bl[i].F;
    out[i].seg_len = bl[i].S;
    out[i].nseg = bl[i].nseg;
    out[i].mode = bl[i].mode;
    out[i].ncols = bl[i].rank ? bl[i].rank : (int)bl[i].lcols.size();
    out[i].dropped = bl[i].dropped;
    out[i].kept = (int)bl[i].lcols.size();
    out[i].lowrank = bl[i].rank ? 1 : 0;
    out[i].lowrank_err = bl[i].lowrank_err;
    int cnt[3] = {0, 0, 0};
    for (int8_t t : bl[i].tprec) cnt[t] += 1;
    out[i].terms_fp64 = cnt[hk::kTermFP64];
    out[i].terms_df64 = cnt[hk::kTermDF64];
    out[i].terms_fp32 = cnt[hk::kTermFP32];
  }
  return HANKEL_OK;
}

int hankel_debug_fft_compare(int log2_len, int ncols, int inverse, int npass, const int* log2_radix,
                             int tensor_passes, double* err, double* ms) {
  if (!log2_radix || !err || !ms || npass < 2 || npass > 4 || ncols < 1 || log2_len < 6 || log2_len > 24)
    return HANKEL_EINVAL;
  return hk::debug_fft_compare_host(log2_len, ncols, inverse, npass, log2_radix, tensor_passes, err, ms);
}

int hankel_plan_device_status(hankel_plan_t p) {
  if (!p || p->host_only) return HANKEL_EINVAL;
  return hk::dev_device_status(p);
}

int hankel_plan_fft_shapes(hankel_plan_t p, hankel_fft_shape* out, int cap, int* count) {
  if (!p || !count || cap < 0 || (cap > 0 && !out)) return HANKEL_EINVAL;
  if (p->host_only) {
    *count = 0;
    return HANKEL_OK;
  }
  return hk::dev_plan_shapes(p, out, cap, count);
}

int hankel_plan_entry(hankel_plan_t p, int64_t k, int64_t n, double* value, int* is_far) {
  if (!p || !value || !is_far) return HANKEL_EINVAL;
  if (k < 1 || k > p->hp.opt.N || n < 1 || n > p->hp.opt.N) return HANKEL_EINVAL;
  *value = hk::host_entry(p->hp, k, n, is_far);
  return HANKEL_OK;
}

int hankel_plan_expansion_entry(hankel_plan_t p, int64_t k, int64_t n, double* value) {
  if (!p || !value) return HANKEL_EINVAL;
  if (k < 1 || k > p->hp.opt.N || n < 1 || n > p->hp.opt.N) return HANKEL_EINVAL;
  *value = hk::expansion_entry(p->hp, k, n, nullptr);
  return HANKEL_OK;
}

int hankel_plan_near_prefix(hankel_plan_t p, int64_t k, int64_t* nend) {
  if (!p || !nend || k < 1 || k > p->hp.opt.N) return HANKEL_EINVAL;
  *nend = p->hp.nend[k - 1];
  return HANKEL_OK;
}

int hankel_exec(hankel_plan_t p, const double* c, double* f, void* stream) {
  if (!p) return HANKEL_EINVAL;
  return hankel_exec_batched(p, c, p->hp.opt.N, f, p->hp.opt.N, 1, stream);
}

int hankel_exec_batched(hankel_plan_t p, const double* c, int64_t ldc, double* f, int64_t ldf, int nrhs,
                        void* stream) {
  if (!p || !c || !f || p->host_only) return HANKEL_EINVAL;
  const int64_t N = p->hp.opt.N;
  if (nrhs < 1 || nrhs > p->hp.opt.max_nrhs || ldc < N || ldf < N) return HANKEL_EINVAL;
  return hk::dev_exec(p, c, ldc, f, ldf, nrhs, stream);
}

int hankel_plan_add_context(hankel_plan_t p, int* index) {
  if (!p || !index || p->host_only) return HANKEL_EINVAL;
  return hk::dev_add_context(p, index);
}

int hankel_exec_batched_ctx(hankel_plan_t p, int ctx, const double* c, int64_t ldc, double* f, int64_t ldf,
                            int nrhs, void* stream) {
  if (!p || !c || !f || p->host_only) return HANKEL_EINVAL;
  const int64_t N = p->hp.opt.N;
  if (nrhs < 1 || nrhs > p->hp.opt.max_nrhs || ldc < N || ldf < N) return HANKEL_EINVAL;
  return hk::dev_exec_ctx(p, ctx, c, ldc, f, ldf, nrhs, stream);
}

int hankel_exec_host(hankel_plan_t p, const double* c, int64_t ldc, double* f, int64_t ldf, int nrhs) {
  if (!p || !c || !f || p->host_only) return HANKEL_EINVAL;
  const int64_t N = p->hp.opt.N;
  if (nrhs < 1 || nrhs > p->hp.opt.max_nrhs || ldc < N || ldf < N) return HANKEL_EINVAL;
  return hk::dev_exec_host(p, c, ldc, f, ldf, nrhs);
}

int hankel_exec_inverse(hankel_plan_t p, const double* f, int64_t ldf, double* c, int64_t ldc, int nrhs,
                        void* stream) {
  if (!p || !c || !f || p->host_only || p->hp.opt.task != HANKEL_DHT) return HANKEL_EINVAL;
  const int64_t N = p->hp.opt.N;
  if (nrhs < 1 || nrhs > p->hp.opt.max_nrhs || ldc < N || ldf < N) return HANKEL_EINVAL;
  return hk::dev_exec_inverse(p, f, ldf, c, ldc, nrhs, stream);
}

int hankel_dht_inverse_weights(int64_t N, double* v) {
  if (N < 1 || !v) return HANKEL_EINVAL;
  std::vector<double> b(N);
  hk::j0_zero_offsets(N, b.data());
  hk::dht_inverse_weights(N, b.data(), v);
  return HANKEL_OK;
}

int hankel_exec_static(hankel_plan_t p, const double* c, double* f, void* stream) {
  if (!p || !c || !f || p->host_only) return HANKEL_EINVAL;
  return hk::dev_exec_static(p, c, f, stream);
}

int hankel_plan_set_timing(hankel_plan_t p, int enable) {
  if (!p || p->host_only) return HANKEL_EINVAL;
  return hk::dev_set_timing(p, enable);
}

int hankel_plan_stage_stats(hankel_plan_t p, hankel_stage_stat* out) {
  if (!p || !out || p->host_only) return HANKEL_EINVAL;
  return hk::dev_stage_stats(p, out);
}

}  // extern "C"
