// FFT shape cache of the autotuner (host only, no CUDA): the fastest split of a transform into
// launches, measured once per GPU model and kept per (GPU name, precision, log2 length, column
// bucket). The measuring itself runs on the device side of a plan (exec.cu).
#pragma once
#include <string>

#include "hankel.h"

namespace hk {

// Bucket of a launch's column count: floor(log2(ncols)) clamped to [0, 16].
int tune_bucket(int64_t ncols);
// Cached shape for the key, if any.
bool tune_get(const std::string& gpu, int precision, int log2_len, int bucket, hankel_fft_shape* out);
// Store (replace) the shape of its key; appends it to the file named by HANKEL_TUNE_CACHE when set.
void tune_put(const std::string& gpu, const hankel_fft_shape& s);
// Load the file named by HANKEL_TUNE_CACHE into the cache, once per process.
void tune_load_env();

}  // namespace hk
