// Internal layout of an H_eff handle, shared by api.cu and the DMRG layer.
#pragma once
#include <vector>

#include "mrd_internal.h"
#include "plan.cuh"

namespace mrd {
struct Lanczos;
void lanczos_free(Lanczos* L);
}  // namespace mrd
struct Tc;
void tc_free(Tc* t);
struct TcPre;
void tc_pre_free(TcPre* t);
struct mrd_heff;
int tc_apply(mrd_heff* h, const double* in, double* out, int32_t prec);
int tc_prepare(mrd_heff* h, int32_t prec);
void tc_prebuild(mrd_heff* h, int32_t prec);
int tc_config(const mrd_heff* h, int32_t* cfg4);
int autotune(mrd_heff* h, int prec);
void tc_env_changed(mrd_heff* h);
int tc_status(mrd_heff* h);
int heff_prefetch_ff(mrd_heff* h);
using mrd::Lanczos;
using mrd::lanczos_free;
using mrd::PlanDims;
using mrd::PlanPtrs;
using namespace mrd;

namespace mrd {

// Device arena: a list of allocations freed together, through the library's memory cache
// (released blocks are reused by later arenas on the same stream).
struct Arena {
  std::vector<void*> ptrs;
  cudaStream_t stream = nullptr;   // stream of the work that uses the arena's memory
  ~Arena() { release(); }
  void release() {
    for (void* p : ptrs) cache_free(p, stream);
    ptrs.clear();
  }
  template <class T>
  cudaError_t alloc(T** out, size_t count) {
    void* p = nullptr;
    cudaError_t e = cache_alloc(&p, count * sizeof(T), stream);
    if (e != cudaSuccess) return e;
    ptrs.push_back(p);
    *out = (T*)p;
    return cudaSuccess;
  }
};

struct Guard {  // switches to a device for the scope
  int prev = -1;
  explicit Guard(int dev) {
    cudaGetDevice(&prev);
    if (prev != dev) cudaSetDevice(dev);
  }
  ~Guard() {
    int cur = -1;
    cudaGetDevice(&cur);
    if (prev >= 0 && cur != prev) cudaSetDevice(prev);
  }
};

inline int kmod(int k, int m) { return ((k % m) + m) % m; }

}  // namespace mrd

using mrd::Arena;
using mrd::Guard;
using mrd::kmod;

struct mrd_heff {
  mrd_ctx* ctx = nullptr;
  PlanDims d{};
  PlanPtrs p{};
  Arena plan_mem;   // tables
  Arena data_mem;   // LW, WR, Z
  int64_t counts[C_NCOUNTS] = {0};
  double* wi_val = nullptr;
  double* wj_val = nullptr;
  double2* lw = nullptr;
  double2* wr = nullptr;
  double2* z = nullptr;
  bool env_loaded = false;
  mutable double def_flops = 0.0;   // definition-order flops, computed on first request
  mutable bool def_flops_done = false;
  int n_sm = 152;
  std::vector<int32_t> left, right, cl, cm, cr, wi_idx, wj_idx;
  std::vector<double> wi_v, wj_v;
  bool timing = false;
  std::vector<cudaEvent_t> ev;   // 3 per recorded apply: before step 1, between, after step 2
  std::vector<cudaEvent_t> ev_pool;
  // the three events of the apply captured in the Lanczos step graph: recorded by the graph at
  // every replay and read back after each one into gms / gcalls
  cudaEvent_t gev[3] = {nullptr, nullptr, nullptr};
  double gms[2] = {0.0, 0.0};
  int32_t gcalls = 0;
  Lanczos* lz = nullptr;
  // host copies of the device-built tables (downloaded once at creation)
  std::vector<int64_t> mid_host, lw_host, wr_host, lmap_host, rmap_host, t1_host, s1_host, t2_host, s2_host, z_host;
  // tensor-core path state (tc_host.cu)
  struct Tc* tc = nullptr;
  struct TcPre* tc_pre = nullptr;   // panel tables being built on a host thread (tc_prebuild)
  // float-float path: LW, WR in float-float layout (prepared after each environment load) and
  // theta staging
  Arena ff_mem;
  float4 *lw_ff = nullptr, *wr_ff = nullptr, *th_ff = nullptr;
  int2 *ff_it1 = nullptr, *ff_it2 = nullptr;   // launch order of the float-float steps (longest K first)
  bool ff_items_built = false;
  bool ff_dirty = true;
  uint64_t gen = 1;          // bumped when apply buffers are reallocated (captured graphs go stale)
  bool use_graph = true;     // capture Lanczos steps as CUDA graphs (MRD_OPT_GRAPH)
  bool per_task = false;     // one GEMM launch per task (MRD_OPT_PER_TASK_LAUNCH)
  bool autotune = true;      // time the tensor-core tile configurations (MRD_OPT_AUTOTUNE)
  uint64_t wait_ns = 1000000000ull;   // limit of each device-side wait (MRD_OPT_WAIT_LIMIT_US)
  bool real = false;         // operands declared real (MRD_OPT_REAL): tensor cores skip imaginary planes
  // per-task launches: [0, tiles of task t] for every task of step 1 and step 2 (device),
  // tiles per task (host), for the FP64 / float-float tiles and for the tensor-core tiles
  Arena pt_mem;
  int64_t* pt_pref1 = nullptr;
  int64_t* pt_pref2 = nullptr;
  std::vector<int64_t> pt_tiles1, pt_tiles2;
  ~mrd_heff() {
    tc_pre_free(tc_pre);   // joins the thread, which reads the host tables
    for (cudaEvent_t e : ev) cudaEventDestroy(e);
    for (cudaEvent_t e : ev_pool) cudaEventDestroy(e);
    for (cudaEvent_t e : gev)
      if (e) cudaEventDestroy(e);
    lanczos_free(lz);
    tc_free(tc);
  }
};

// The H_eff's float-float copies of LW / WR when they are current (prepared by a float-float
// application since the last environment load), else nullptr.
inline const float4* heff_ff_lw(const mrd_heff* h) { return h->lw_ff && !h->ff_dirty ? h->lw_ff : nullptr; }
inline const float4* heff_ff_wr(const mrd_heff* h) { return h->wr_ff && !h->ff_dirty ? h->wr_ff : nullptr; }

inline cudaError_t record_event(cudaEvent_t e, cudaStream_t s, bool captured) {
  if (!e) return cudaSuccess;
  return captured ? cudaEventRecordWithFlags(e, s, cudaEventRecordExternal) : cudaEventRecord(e, s);
}

inline cudaEvent_t take_event(mrd_heff* h) {
  cudaEvent_t e = nullptr;
  if (!h->ev_pool.empty()) {
    e = h->ev_pool.back();
    h->ev_pool.pop_back();
  } else if (cudaEventCreate(&e) != cudaSuccess) {
    return nullptr;
  }
  h->ev.push_back(e);
  return e;
}

// The timing events of one apply on stream s: three pooled events, or, while s is being
// captured into the Lanczos step graph, the graph's own three (external event nodes, so that
// each replay records them). *captured tells which.
inline bool apply_events(mrd_heff* h, cudaStream_t s, cudaEvent_t ev[3], bool* captured) {
  cudaStreamCaptureStatus st = cudaStreamCaptureStatusNone;
  *captured = cudaStreamIsCapturing(s, &st) == cudaSuccess && st == cudaStreamCaptureStatusActive;
  if (!*captured) {
    for (int k = 0; k < 3; ++k)
      if (!(ev[k] = take_event(h))) return false;
    return true;
  }
  for (int k = 0; k < 3; ++k) {
    if (!h->gev[k] && cudaEventCreate(&h->gev[k]) != cudaSuccess) {
      h->gev[k] = nullptr;
      return false;
    }
    ev[k] = h->gev[k];
  }
  return true;
}

