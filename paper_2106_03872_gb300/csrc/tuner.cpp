// Launch-shape autotuner (tuner.h).
#include "tuner.h"

#include <cstdio>
#include <map>
#include <mutex>
#include <vector>

#include "common.h"

namespace ks {

namespace {

struct Decision {
  int choice = 0;
  std::vector<std::string> names;
  std::vector<float> ms;
};

std::mutex g_mu;
std::map<std::string, Decision>& decisions() {
  static std::map<std::string, Decision> d;
  return d;
}

}  // namespace

int tune_choice(const std::string& key, int ncand, const std::function<void(int)>& run, cudaStream_t s,
                const char* const* names) {
  {
    std::lock_guard<std::mutex> lk(g_mu);
    auto it = decisions().find(key);
    if (it != decisions().end()) return it->second.choice;
  }
  if (ncand <= 1) return 0;
  constexpr int REPS = 3;
  cudaEvent_t a, b;
  KS_CUDA(cudaEventCreate(&a));
  KS_CUDA(cudaEventCreate(&b));
  Decision d;
  for (int c = 0; c < ncand; ++c) {
    run(c);                                                          // warm-up (first-launch costs)
    float best = 1e30f;
    for (int r = 0; r < REPS; ++r) {
      KS_CUDA(cudaEventRecord(a, s));
      run(c);
      KS_CUDA(cudaEventRecord(b, s));
      KS_CUDA(cudaEventSynchronize(b));
      float ms = 0.f;
      KS_CUDA(cudaEventElapsedTime(&ms, a, b));
      best = ms < best ? ms : best;
    }
    d.names.push_back(names[c]);
    d.ms.push_back(best);
    if (best < d.ms[d.choice]) d.choice = c;
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  std::lock_guard<std::mutex> lk(g_mu);
  auto ins = decisions().emplace(key, d);                           // a concurrent tuner may have won
  return ins.first->second.choice;
}

std::string tune_log_json() {
  std::lock_guard<std::mutex> lk(g_mu);
  std::string out = "[";
  bool first = true;
  for (const auto& kv : decisions()) {
    const Decision& d = kv.second;
    out += first ? "" : ", ";
    first = false;
    out += "{\"key\": \"" + kv.first + "\", \"ms\": {";
    for (size_t i = 0; i < d.names.size(); ++i) {
      char buf[64];
      std::snprintf(buf, sizeof(buf), "%.6f", d.ms[i]);
      out += (i ? ", \"" : "\"") + d.names[i] + "\": " + buf;
    }
    out += "}, \"choice\": \"" + d.names[d.choice] + "\"}";
  }
  return out + "]";
}

}  // namespace ks
