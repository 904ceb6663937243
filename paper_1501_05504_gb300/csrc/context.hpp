// Library context: device, workspace arena, cached device-resident plans.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <memory>
#include <string>
#include <unordered_map>
#include <vector>

#include "plan.hpp"

namespace dmrg3s {

// Device copy of a plan's task tables.
struct DevicePlan {
  Plan host;
  void* mem = nullptr;      // one allocation holding every table
  GemmTile* g1_tiles = nullptr;
  GemmTask* g1_tasks = nullptr;
  GemmSeg* g1_segs = nullptr;
  CombChunk* c2_chunks = nullptr;
  CombTask* c2_tasks = nullptr;
  CombTerm* c2_terms = nullptr;
  GemmTile* g3_tiles = nullptr;
  GemmTask* g3_tasks = nullptr;
  GemmSeg* g3_segs = nullptr;
  ~DevicePlan();
};

struct Context {
  int device = 0;
  char* ws = nullptr;           // workspace arena
  size_t ws_bytes = 0;
  std::unordered_map<uint64_t, std::unique_ptr<DevicePlan>> plans;
  std::string last_error;
};

// FNV-1a fingerprint builder used as the plan-cache key.
struct Hasher {
  uint64_t h = 1469598103934665603ull;
  void bytes(const void* p, size_t n) {
    const unsigned char* c = (const unsigned char*)p;
    for (size_t i = 0; i < n; ++i) {
      h ^= c[i];
      h *= 1099511628211ull;
    }
  }
  template <class T>
  void pod(const T& v) { bytes(&v, sizeof(T)); }
  template <class T>
  void vec(const std::vector<T>& v) {
    pod(v.size());
    if (!v.empty()) bytes(v.data(), v.size() * sizeof(T));
  }
  void bond(const Bond& b);
  void site(const SiteLayout& s);
  void env(const EnvLayout& e);
  void mpo(const MpoLayout& w);
};

// Upload a host plan (allocates the device tables).  Returns CUDA errors.
dmrg3s_status upload_plan(Plan&& host, std::unique_ptr<DevicePlan>* out);

// Enqueue the stages of a plan.  Bases as documented for each plan Kind.
dmrg3s_status run_plan(const DevicePlan& p, const double* g1A, const double* g1B, double* ws1,
                       double* c2out, double c2scale, const double* g3A, const double* g3B,
                       double* g3C, cudaStream_t st);

}  // namespace dmrg3s
