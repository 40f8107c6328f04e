// Interface between the host ABI layer and the CUDA translation units.
#pragma once
#include <stddef.h>

#include "plan.h"

namespace hk {
struct DevicePlan;  // defined in exec.cu
}

struct hankel_plan_s {
  hk::HostPlan hp;
  bool host_only = false;
  hk::DevicePlan* dev = nullptr;
};

namespace hk {
// Fault injection (hankel_debug_fail_allocs): true when this allocation is to be reported failed.
bool alloc_fault();
// Allocate device tables and workspace and build the chirp spectra.
int dev_plan_create(hankel_plan_s* p);
// Free everything dev_plan_create made (also after a partial failure).
int dev_plan_destroy(hankel_plan_s* p);
int dev_exec(hankel_plan_s* p, const double* c, int64_t ldc, double* f, int64_t ldf, int nrhs, void* stream);
int dev_exec_ctx(hankel_plan_s* p, int k, const double* c, int64_t ldc, double* f, int64_t ldf, int nrhs,
                 void* stream);
int dev_add_context(hankel_plan_s* p, int* index);
// Number of execution contexts; *ctx_bytes (optional) receives the device bytes of one.
int dev_contexts(const hankel_plan_s* p, size_t* ctx_bytes);
int dev_exec_host(hankel_plan_s* p, const double* c, int64_t ldc, double* f, int64_t ldf, int nrhs);
int dev_exec_static(hankel_plan_s* p, const double* c, double* f, void* stream);
int dev_exec_inverse(hankel_plan_s* p, const double* f, int64_t ldf, double* c, int64_t ldc, int nrhs, void* stream);
int dev_set_timing(hankel_plan_s* p, int enable);
int dev_stage_stats(hankel_plan_s* p, hankel_stage_stat* out);
size_t dev_plan_bytes(const hankel_plan_s* p);
size_t dev_workspace_bytes(const hankel_plan_s* p);
int dev_plan_shapes(const hankel_plan_s* p, hankel_fft_shape* out, int cap, int* count);
int dev_device_status(hankel_plan_s* p);
// hankel_debug_fft_compare on the current device.
int debug_fft_compare_host(int logF, int ncols, int inverse, int npass, const int* logr, int tc, double* err,
                           double* ms);
}  // namespace hk
