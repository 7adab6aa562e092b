// Internal declarations shared by the translation units of libmrdmrg.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <array>
#include <map>
#include <string>
#include <vector>

#include "../../include/mrdmrg.h"

namespace mrd {

struct HostMPO {
  int n_sites = 0;
  int modulus = 1;
  std::vector<std::vector<int32_t>> bond_charges;  // per bond: 2*dim
  std::vector<std::vector<int32_t>> site_idx;      // per site: 4*nnz
  std::vector<std::vector<double>> site_val;       // per site: 2*nnz
};

int build_mpo_host(const mrd_model& m, HostMPO* out, std::string* err);

// Packed charge key: lexicographic in (N, K).
__host__ __device__ inline int64_t qkey(int32_t n, int32_t k) {
  return ((int64_t)(n + (1 << 29)) << 32) | (int64_t)(uint32_t)k;
}

// Number of kernels this library has launched (all devices, all contexts); a replayed CUDA
// graph counts the kernels it holds.
void count_launch();
void count_launches(int64_t n);
void uncount_launches(int64_t n);
int64_t launch_count_total();

// Device memory cache (pool.cu): cache_alloc hands out a block of at least `bytes`, reusing
// one that was released on the same stream; cache_free returns it; cache_trim frees the
// cached blocks of a device.
cudaError_t cache_alloc(void** out, size_t bytes, cudaStream_t s);
void cache_free(void* p, cudaStream_t s);
void cache_trim(int device);
cudaError_t cache_alloc_host(void** out, size_t bytes);   // pinned host memory, reused by size
void cache_free_host(void* p);

// A device buffer owned by the library.
struct DevBuf {
  void* p = nullptr;
  size_t bytes = 0;
};

}  // namespace mrd

struct mrd_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  std::string err;
  int refs = 0;            // live handles created on this context
  bool destroyed = false;  // mrd_destroy called; deleted when refs drops to 0
  // autotuner decisions: problem class -> tensor-core tile configuration (ntile, stages, order)
  std::map<uint64_t, std::array<int, 3>> tc_tuned;
};

// Reference counting so that handles and contexts may be released in any order.
void mrd_ctx_retain(mrd_ctx* ctx);
void mrd_ctx_release(mrd_ctx* ctx);

struct mrd_mpo {
  mrd_ctx* ctx = nullptr;
  mrd::HostMPO h;
};

// Status helpers: set the context's message and return a code.
int mrd_fail(mrd_ctx* ctx, int code, const std::string& msg);
int mrd_cuda_fail(mrd_ctx* ctx, cudaError_t e, const char* where);

#define MRD_CUDA(ctx, call)                                   \
  do {                                                        \
    cudaError_t e_ = (call);                                  \
    if (e_ != cudaSuccess) return mrd_cuda_fail(ctx, e_, #call); \
  } while (0)
