// Opt-in per-kernel timing with CUDA events recorded on each kernel's launch
// stream.  Disabled by default; when enabled, every kernel launch of the
// library is bracketed by two events from a fixed pool created at enable
// time (no allocation while timing).  Single-threaded use.  Measurement
// support with no counterpart in the paper.
#include <string.h>

#include <vector>

#include "common.cuh"

namespace gs {

namespace {

constexpr int kPool = 8192;
constexpr int kMaxNames = 64;

struct Rec {
  int name;
  int pair;
};

struct Timing {
  bool on = false;
  std::vector<cudaEvent_t> ev;        // 2 * kPool events
  int next_pair = 0;
  std::vector<Rec> pending;
  const char* names[kMaxNames] = {};
  double ms[kMaxNames] = {};
  int64_t launches[kMaxNames] = {};
  int64_t dropped = 0;
  int open_name = -1;
  int open_pair = -1;
};

Timing& T() {
  static Timing t;
  return t;
}

int name_id(const char* name) {
  Timing& t = T();
  for (int i = 0; i < kMaxNames; ++i) {
    if (t.names[i] == nullptr) {
      t.names[i] = name;
      return i;
    }
    if (strcmp(t.names[i], name) == 0) return i;
  }
  return -1;
}

}  // namespace

void timing_begin(const char* name, cudaStream_t stream) {
  Timing& t = T();
  if (!t.on) return;
  if (t.next_pair >= kPool) {
    ++t.dropped;
    t.open_pair = -1;
    return;
  }
  t.open_name = name_id(name);
  t.open_pair = t.next_pair++;
  cudaEventRecord(t.ev[2 * t.open_pair], stream);
}

void timing_end(cudaStream_t stream) {
  Timing& t = T();
  if (!t.on || t.open_pair < 0) return;
  cudaEventRecord(t.ev[2 * t.open_pair + 1], stream);
  t.pending.push_back({t.open_name, t.open_pair});
  t.open_pair = -1;
}

}  // namespace gs

using namespace gs;

extern "C" {

gs_status gs_timing_enable(int on) {
  Timing& t = T();
  if (on && t.ev.empty()) {
    t.ev.resize(2 * kPool);
    for (auto& e : t.ev)
      if (cudaEventCreate(&e) != cudaSuccess) return GS_ERR_CUDA;
  }
  t.on = on != 0;
  return GS_OK;
}

int gs_timing_collect(gs_kernel_time* out, int max_out) {
  Timing& t = T();
  for (const Rec& r : t.pending) {
    float ms = 0.f;
    if (cudaEventSynchronize(t.ev[2 * r.pair + 1]) == cudaSuccess &&
        cudaEventElapsedTime(&ms, t.ev[2 * r.pair], t.ev[2 * r.pair + 1]) == cudaSuccess && r.name >= 0) {
      t.ms[r.name] += ms;
      t.launches[r.name] += 1;
    }
  }
  t.pending.clear();
  t.next_pair = 0;
  int k = 0;
  for (int i = 0; i < kMaxNames && t.names[i]; ++i) {
    if (t.launches[i] == 0) continue;
    if (out && k < max_out) {
      out[k].name = t.names[i];
      out[k].ms = t.ms[i];
      out[k].launches = t.launches[i];
    }
    ++k;
    t.ms[i] = 0.0;
    t.launches[i] = 0;
  }
  return k;
}

}  // extern "C"
