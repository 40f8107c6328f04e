// FFT shape cache of the autotuner (hankel_tune_cache_* in include/hankel.h).
//
// Keys are (GPU name, precision, log2 length, column bucket): a shape measured on one GPU model
// is reused by every later plan on that model in the process, and across processes through a
// text file (HANKEL_TUNE_CACHE, or hankel_tune_cache_save/load). One line per entry:
//   gpu name | precision log2_len col_bucket one_launch npass r0 r1 r2 r3 tensor_passes ms_default ms_chosen
// The name goes first and ends at the last '|', so names with spaces are kept whole.
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <map>
#include <mutex>
#include <string>
#include <tuple>

#include "tune.h"

namespace hk {
namespace {

typedef std::tuple<std::string, int, int, int> Key;

std::mutex g_mu;
std::map<Key, hankel_fft_shape>& table() {
  static std::map<Key, hankel_fft_shape> t;
  return t;
}

bool parse_line(const char* line, std::string* gpu, hankel_fft_shape* s) {
  const char* bar = strrchr(line, '|');
  if (!bar || bar == line) return false;
  gpu->assign(line, (size_t)(bar - line));
  memset(s, 0, sizeof(*s));
  const int n = sscanf(bar + 1, "%d %d %d %d %d %d %d %d %d %d %lf %lf", &s->precision, &s->log2_len, &s->col_bucket,
                       &s->one_launch, &s->npass, &s->log2_radix[0], &s->log2_radix[1], &s->log2_radix[2],
                       &s->log2_radix[3], &s->tensor_passes, &s->ms_default, &s->ms_chosen);
  return n == 12 && !gpu->empty();
}

void format_line(FILE* fh, const std::string& gpu, const hankel_fft_shape& s) {
  fprintf(fh, "%s|%d %d %d %d %d %d %d %d %d %d %.6g %.6g\n", gpu.c_str(), s.precision, s.log2_len, s.col_bucket,
          s.one_launch, s.npass, s.log2_radix[0], s.log2_radix[1], s.log2_radix[2], s.log2_radix[3], s.tensor_passes,
          s.ms_default, s.ms_chosen);
}

int load_file(const char* path) {
  FILE* fh = fopen(path, "r");
  if (!fh) return HANKEL_EINVAL;
  char buf[512];
  while (fgets(buf, sizeof buf, fh)) {
    std::string gpu;
    hankel_fft_shape s;
    if (parse_line(buf, &gpu, &s)) table()[Key(gpu, s.precision, s.log2_len, s.col_bucket)] = s;
  }
  fclose(fh);
  return HANKEL_OK;
}

}  // namespace

int tune_bucket(int64_t ncols) {
  int b = 0;
  while (b < 16 && (int64_t(2) << b) <= ncols) ++b;
  return b;
}

bool tune_get(const std::string& gpu, int precision, int log2_len, int bucket, hankel_fft_shape* out) {
  std::lock_guard<std::mutex> lk(g_mu);
  auto it = table().find(Key(gpu, precision, log2_len, bucket));
  if (it == table().end()) return false;
  *out = it->second;
  return true;
}

void tune_put(const std::string& gpu, const hankel_fft_shape& s) {
  std::lock_guard<std::mutex> lk(g_mu);
  table()[Key(gpu, s.precision, s.log2_len, s.col_bucket)] = s;
  const char* path = getenv("HANKEL_TUNE_CACHE");
  if (path && *path) {
    FILE* fh = fopen(path, "a");
    if (fh) {
      format_line(fh, gpu, s);
      fclose(fh);
    }
  }
}

void tune_load_env() {
  static std::once_flag once;
  std::call_once(once, [] {
    const char* path = getenv("HANKEL_TUNE_CACHE");
    if (path && *path) {
      std::lock_guard<std::mutex> lk(g_mu);
      load_file(path);
    }
  });
}

}  // namespace hk

extern "C" {

int hankel_tune_cache_put(const char* gpu_name, const hankel_fft_shape* s) {
  if (!gpu_name || !*gpu_name || strchr(gpu_name, '\n') || !s) return HANKEL_EINVAL;
  hk::tune_put(gpu_name, *s);
  return HANKEL_OK;
}

int hankel_tune_cache_get(const char* gpu_name, int precision, int log2_len, int col_bucket, hankel_fft_shape* out,
                          int* found) {
  if (!gpu_name || !out || !found) return HANKEL_EINVAL;
  *found = hk::tune_get(gpu_name, precision, log2_len, col_bucket, out) ? 1 : 0;
  return HANKEL_OK;
}

int hankel_tune_cache_save(const char* path) {
  if (!path) return HANKEL_EINVAL;
  FILE* fh = fopen(path, "w");
  if (!fh) return HANKEL_EINVAL;
  {
    std::lock_guard<std::mutex> lk(hk::g_mu);
    for (const auto& kv : hk::table()) hk::format_line(fh, std::get<0>(kv.first), kv.second);
  }
  fclose(fh);
  return HANKEL_OK;
}

int hankel_tune_cache_load(const char* path) {
  if (!path) return HANKEL_EINVAL;
  std::lock_guard<std::mutex> lk(hk::g_mu);
  return hk::load_file(path);
}

int hankel_tune_cache_clear(void) {
  std::lock_guard<std::mutex> lk(hk::g_mu);
  hk::table().clear();
  return HANKEL_OK;
}

int hankel_tune_bucket(int64_t ncols) { return hk::tune_bucket(ncols); }

}  // extern "C"
