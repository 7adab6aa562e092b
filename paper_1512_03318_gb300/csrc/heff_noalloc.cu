// H_eff application that allocates nothing (mrd_heff_apply_noalloc).
//
// Some callers cannot call cudaMalloc at the moment they need a matvec: code running under
// an external memory pool that must account for every byte, or a host thread that is not
// allowed to touch the CUDA allocator while other streams are being captured. For them the
// step-1 intermediate Z_{w'} = LW_{w'} theta lives in this file's static device array
// instead of the buffer that mrd_heff_create allocates. Everything else (tables, folded
// environments) was allocated earlier by mrd_heff_create and mrd_heff_set_env.
//
// The array is a host-side symbol in host code; its device address is obtained once per
// device with cudaGetSymbolAddress while that device is current, and passed to the kernels.
// The cached address belongs to the device's primary context: after cudaDeviceReset it is
// stale (as is every handle of this library created before the reset).
#include <mutex>

#include "mrd_internal.h"
#include "plan.cuh"

namespace mrd {
cudaError_t launch_cgemm_fp64(const double2* A, const double2* B, double2* C, const int64_t* tasks,
                              const int64_t* segs, const int64_t* prefix, int64_t n_tasks, int64_t total_tiles,
                              int n_sm, cudaStream_t s);
}  // namespace mrd

namespace {

// MRD_NOALLOC_Z_MAX_ELEMS complex128 elements = 64 MiB, held by every device that loads the
// library until the process exits.
static __device__ __align__(256) double2 g_noalloc_z[MRD_NOALLOC_Z_MAX_ELEMS];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
double2* g_addr[kMaxDevices] = {nullptr};

// Device address of g_noalloc_z on `device` (which must be current); looked up once.
cudaError_t scratch_address(int device, double2** out) {
  std::lock_guard<std::mutex> lock(g_mu);
  if (device < 0 || device >= kMaxDevices) return cudaErrorInvalidDevice;
  if (!g_addr[device]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_z);
    if (e != cudaSuccess) return e;
    g_addr[device] = (double2*)p;
  }
  *out = g_addr[device];
  return cudaSuccess;
}

}  // namespace

namespace mrd {
// Read-only view of a handle, defined in api.cu next to struct mrd_heff.
int mrd_heff_internal_noalloc_view(const mrd_heff* h, PlanPtrs* p, int64_t* counts, const double2** lw,
                                   const double2** wr, int* n_sm, mrd_ctx** ctx, bool* env_loaded);
}  // namespace mrd

extern "C" int mrd_heff_apply_noalloc(mrd_heff* h, const double* theta_in_dev, double* theta_out_dev) try {
  if (!h) return MRD_E_ARG;
  mrd::PlanPtrs p;
  int64_t c[mrd::C_NCOUNTS];
  const double2 *lw = nullptr, *wr = nullptr;
  int n_sm = 0;
  mrd_ctx* ctx = nullptr;
  bool env_loaded = false;
  const int vrc = mrd::mrd_heff_internal_noalloc_view(h, &p, c, &lw, &wr, &n_sm, &ctx, &env_loaded);
  if (vrc != MRD_OK) return vrc;
  if (!env_loaded) return mrd_fail(ctx, MRD_E_STATE, "mrd_heff_apply_noalloc: environments not loaded");
  if (c[mrd::C_ZLEN] > (int64_t)MRD_NOALLOC_Z_MAX_ELEMS)
    return mrd_fail(ctx, MRD_E_ARG,
                    "mrd_heff_apply_noalloc: this problem needs " + std::to_string(c[mrd::C_ZLEN]) +
                        " complex scratch elements, above the static limit of " +
                        std::to_string((long long)MRD_NOALLOC_Z_MAX_ELEMS) + "; use mrd_heff_apply");
  const int64_t n = c[mrd::C_THETA];
  if (n > 0 && (!theta_in_dev || !theta_out_dev))
    return mrd_fail(ctx, MRD_E_ARG, "mrd_heff_apply_noalloc: null theta");
  const char* a = (const char*)theta_in_dev;
  const char* b = (const char*)theta_out_dev;
  if (n > 0 && a < b + n * 16 && b < a + n * 16)
    return mrd_fail(ctx, MRD_E_ARG, "mrd_heff_apply_noalloc: theta_in and theta_out overlap");
  int prev = -1;
  cudaGetDevice(&prev);
  if (prev != ctx->device) cudaSetDevice(ctx->device);
  double2* z = nullptr;
  cudaError_t e = scratch_address(ctx->device, &z);
  cudaStream_t s = ctx->stream;
  // theta_out is cleared first because output blocks without a contributing task are not
  // written. Z needs no clearing: step 2 reads only the rows step 1 wrote in this call.
  if (e == cudaSuccess) e = cudaMemsetAsync(theta_out_dev, 0, (size_t)n * 16, s);
  if (e == cudaSuccess)
    e = mrd::launch_cgemm_fp64(lw, (const double2*)theta_in_dev, z, p.t1, p.seg1, p.tile1, c[mrd::C_NT1],
                               c[mrd::C_TILES1], n_sm, s);
  if (e == cudaSuccess)
    e = mrd::launch_cgemm_fp64(z, wr, (double2*)theta_out_dev, p.t2, p.seg2, p.tile2, c[mrd::C_NT2],
                               c[mrd::C_TILES2], n_sm, s);
  if (prev >= 0 && prev != ctx->device) cudaSetDevice(prev);
  if (e != cudaSuccess) return mrd_cuda_fail(ctx, e, "mrd_heff_apply_noalloc");
  return MRD_OK;
} catch (...) {   // host memory or threads exhausted: no exception crosses the C ABI
  return MRD_E_HOST;
}
