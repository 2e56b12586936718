// Per-kernel launch counting and optional CUDA-event timing.
//
// Every kernel the library launches goes through Launch{ctx, name, stream}:
// the context counts launches per kernel name always, and, while timing is
// enabled, records a start/stop event pair on the launching stream around
// the launch.  distil_profile_read() synchronises those events and returns
// per-kernel launch counts and summed durations.  Timing stays off during
// CUDA graph capture (the caller enables it only for eager runs).
#pragma once
#include <string>
#include <vector>

#include "common.cuh"

namespace distil {

struct ProfRec {
  int kernel;
  cudaEvent_t a, b;
};

struct Profiler {
  bool timing = false;
  std::vector<std::string> names;
  std::vector<long long> launches;
  std::vector<ProfRec> recs;
  std::vector<cudaEvent_t> pool;
  size_t pool_used = 0;

  int id(const char* name) {
    for (size_t i = 0; i < names.size(); ++i)
      if (names[i] == name) return (int)i;
    names.emplace_back(name);
    launches.push_back(0);
    return (int)names.size() - 1;
  }
  cudaEvent_t ev() {
    if (pool_used == pool.size()) {
      cudaEvent_t e;
      if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
      pool.push_back(e);
    }
    return pool[pool_used++];
  }
  void reset() {
    recs.clear();
    pool_used = 0;
    for (auto& l : launches) l = 0;
  }
  ~Profiler() {
    for (auto e : pool) cudaEventDestroy(e);
  }
};

Profiler& profiler(distil_ctx* ctx);

// Scope around one kernel launch.
struct Launch {
  Profiler* p;
  int k;
  ProfRec rec;
  cudaStream_t s;
  Launch(distil_ctx* ctx, const char* name, cudaStream_t st) : p(ctx ? &profiler(ctx) : nullptr), k(-1), s(st) {
    rec.a = rec.b = nullptr;
    if (!p) return;
    k = p->id(name);
    p->launches[k]++;
    if (p->timing) {
      rec.kernel = k;
      rec.a = p->ev();
      rec.b = p->ev();
      if (rec.a) cudaEventRecord(rec.a, s);
    }
  }
  ~Launch() {
    if (p && p->timing && rec.a && rec.b) {
      cudaEventRecord(rec.b, s);
      p->recs.push_back(rec);
    }
  }
};

}  // namespace distil
