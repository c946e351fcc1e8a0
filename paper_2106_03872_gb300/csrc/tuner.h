// Launch-shape autotuner of the fused kernels: the first time a decision (a key naming the
// kernel family, the grid and a bucket of the state count) comes up, every candidate runs on the
// live data, timed with CUDA events on the launching stream, and the fastest is kept for the rest
// of the process.  Candidates must be idempotent (they read the same inputs and overwrite the
// same outputs), so timing them changes no result; the first call of each decision waits for its
// timings.  The choices and timings are kept as a log the library reports as JSON.
#pragma once

#include <cuda_runtime.h>

#include <functional>
#include <string>

namespace ks {

// Index of the fastest of ncand candidates for `key`: run(c) launches candidate c on stream s.
// Cached after the first call; thread-safe.
int tune_choice(const std::string& key, int ncand, const std::function<void(int)>& run, cudaStream_t s,
                const char* const* names);

// The log of every decision so far: [{"key": ..., "ms": {name: ms, ...}, "choice": name}, ...].
std::string tune_log_json();

}  // namespace ks
