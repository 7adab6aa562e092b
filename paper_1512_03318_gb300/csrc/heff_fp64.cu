// FP64 kernels of the two-site H_eff application.
//
// theta' = H_eff theta is evaluated as
//   step 1   Z_{w'}[(s1',a'), (s2,b)] = sum_{s1,a} LW_{w'}^{(s1',s1)}[a',a] theta[(s1,a),(s2,b)]
//   step 2   theta'[(s1',a'), (s2',b')] = sum_{w',s2,b} Z_{w'}[(s1',a'),(s2,b)] WR_{w'}^{(s2,s2')}[b,b']
// with LW_{w'}^{(s1',s1)} = sum_w W_i[w,w',s1',s1] L_w and
//      WR_{w'}^{(s2,s2')}  = sum_{w''} W_{i+1}[w',w'',s2',s2] R_{w''},
// which is the definition L W_i W_{i+1} R theta with the MPO sums folded into the
// environments once per environment load. Both steps are grouped complex GEMMs over the task
// lists built in plan.cu; every output block is owned by exactly one task, so there are no
// atomics and the result is deterministic.
//
// On GB300 FP64 runs on the CUDA cores at about 1.2 TFLOP/s, far below what shared memory or
// HBM can feed, so a small 32 x 32 complex tile per 256-thread CTA (2 x 2 outputs per
// thread) keeps every DFMA pipe busy while wasting little work on ragged blocks.
#include "mrd_internal.h"
#include "plan.cuh"

namespace mrd {

namespace {

constexpr int kT = 32;   // output tile (complex elements per side)
constexpr int kK = 16;   // K chunk

__device__ __forceinline__ int64_t find_task(const int64_t* prefix, int64_t n, int64_t item) {
  // largest t with prefix[t] <= item (prefix[0] = 0, prefix[n] = total > item)
  int64_t lo = 0, hi = n - 1;
  while (lo < hi) {
    int64_t mid = (lo + hi + 1) >> 1;
    if (prefix[mid] <= item) lo = mid; else hi = mid - 1;
  }
  return lo;
}

__device__ __forceinline__ void cmac(double2& c, const double2 a, const double2 b) {
  c.x = fma(a.x, b.x, c.x);
  c.x = fma(-a.y, b.y, c.x);
  c.y = fma(a.x, b.y, c.y);
  c.y = fma(a.y, b.x, c.y);
}

}  // namespace

__global__ void __launch_bounds__(256) k_cgemm_fp64(const double2* __restrict__ A, const double2* __restrict__ B,
                                                    double2* __restrict__ C, const int64_t* __restrict__ tasks,
                                                    const int64_t* __restrict__ segs,
                                                    const int64_t* __restrict__ prefix, int64_t n_tasks) {
  __shared__ double2 As[kT][kK + 1];
  __shared__ double2 Bs[kK][kT + 1];
  const int tid = threadIdx.x;
  const int ty = tid >> 4, tx = tid & 15;
  const int64_t total = prefix[n_tasks];
  for (int64_t item = blockIdx.x; item < total; item += gridDim.x) {
    const int64_t t = find_task(prefix, n_tasks, item);
    const int64_t* task = tasks + TF * t;
    const int64_t M = task[0], N = task[1], c_off = task[2], ldc = task[3];
    const int64_t seg0 = task[4], nseg = task[5];
    const int64_t tiles_n = (N + kT - 1) / kT;
    const int64_t local = item - prefix[t];
    const int64_t m0 = (local / tiles_n) * kT, n0 = (local % tiles_n) * kT;
    double2 acc[2][2];
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
      for (int j = 0; j < 2; ++j) acc[i][j] = make_double2(0.0, 0.0);
    for (int64_t s = 0; s < nseg; ++s) {
      const int64_t* sg = segs + SF * (seg0 + s);
      const int64_t a_off = sg[0], lda = sg[1], b_off = sg[2], ldb = sg[3], K = sg[4];
      const int64_t flags = sg[5];
      for (int64_t k0 = 0; k0 < K; k0 += kK) {
#pragma unroll
        for (int r = 0; r < 2; ++r) {
          const int e = tid + r * 256;
          if (!(flags & 1)) {                           // A[m, k] at a_off + m * lda + k
            const int ar = e >> 4, ak = e & 15;
            const int64_t gr = m0 + ar, gk = k0 + ak;
            As[ar][ak] = (gr < M && gk < K) ? A[a_off + gr * lda + gk] : make_double2(0.0, 0.0);
          } else {                                      // A[m, k] = conj(A[a_off + k * lda + m])
            const int ar = e & 31, ak = e >> 5;
            const int64_t gr = m0 + ar, gk = k0 + ak;
            double2 v = (gr < M && gk < K) ? A[a_off + gk * lda + gr] : make_double2(0.0, 0.0);
            v.y = -v.y;
            As[ar][ak] = v;
          }
          if (!(flags & 2)) {                           // B[k, n] at b_off + k * ldb + n
            const int bk = e >> 5, bc = e & 31;
            const int64_t gk2 = k0 + bk, gc = n0 + bc;
            Bs[bk][bc] = (gk2 < K && gc < N) ? B[b_off + gk2 * ldb + gc] : make_double2(0.0, 0.0);
          } else {                                      // B[k, n] = conj(B[b_off + n * ldb + k])
            const int bk = e & 15, bc = e >> 4;
            const int64_t gk2 = k0 + bk, gc = n0 + bc;
            double2 v = (gk2 < K && gc < N) ? B[b_off + gc * ldb + gk2] : make_double2(0.0, 0.0);
            v.y = -v.y;
            Bs[bk][bc] = v;
          }
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < kK; ++k) {
          const double2 a0 = As[2 * ty][k], a1 = As[2 * ty + 1][k];
          const double2 b0 = Bs[k][2 * tx], b1 = Bs[k][2 * tx + 1];
          cmac(acc[0][0], a0, b0);
          cmac(acc[0][1], a0, b1);
          cmac(acc[1][0], a1, b0);
          cmac(acc[1][1], a1, b1);
        }
        __syncthreads();
      }
    }
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
      for (int j = 0; j < 2; ++j) {
        const int64_t r = m0 + 2 * ty + i, c = n0 + 2 * tx + j;
        if (r < M && c < N) C[c_off + r * ldc + c] = acc[i][j];
      }
  }
}

// LW / WR fold: out block = sum over its contributing MPO entries of value * env block.
// rows: LW or WR table (10 int64 per row); env_map: [channel][sector] -> env offset;
// perm/idx/val: sorted MPO entries; chan_field: index of the env channel in an entry
// (0 = w for W_i, 1 = w'' for W_{i+1}); sec_field: row field holding the env sector.
__global__ void __launch_bounds__(256) k_fold_env(const double2* __restrict__ env, double2* __restrict__ out,
                                                  const int64_t* __restrict__ rows, int64_t nrows,
                                                  const int64_t* __restrict__ env_map, int n_sec,
                                                  const int32_t* __restrict__ perm, const int32_t* __restrict__ idx,
                                                  const double* __restrict__ val, int chan_field) {
  for (int64_t r = blockIdx.x; r < nrows; r += gridDim.x) {
    const int64_t* row = rows + LWF * r;
    const int64_t sec = row[3], n = row[5] * row[6], off = row[7], cb = row[8], ce = row[9];
    for (int64_t e = threadIdx.x; e < n; e += blockDim.x) {
      double2 acc = make_double2(0.0, 0.0);
      for (int64_t c = cb; c < ce; ++c) {
        const int ent = perm[c];
        const int ch = idx[4 * ent + chan_field];
        const int64_t src = env_map[(int64_t)ch * n_sec + sec];
        const double vr = val[2 * ent], vi = val[2 * ent + 1];
        const double2 x = env[src + e];
        acc.x += vr * x.x - vi * x.y;
        acc.y += vr * x.y + vi * x.x;
      }
      out[off + e] = acc;
    }
  }
}

cudaError_t launch_cgemm_fp64(const double2* A, const double2* B, double2* C, const int64_t* tasks,
                              const int64_t* segs, const int64_t* prefix, int64_t n_tasks, int64_t total_tiles,
                              int n_sm, cudaStream_t s) {
  if (total_tiles <= 0) return cudaSuccess;
  int64_t grid = (int64_t)n_sm * 8;
  if (grid > total_tiles) grid = total_tiles;
  k_cgemm_fp64<<<(unsigned)grid, 256, 0, s>>>(A, B, C, tasks, segs, prefix, n_tasks);
  mrd::count_launch();
  return cudaGetLastError();
}

cudaError_t launch_fold_env(const double2* env, double2* out, const int64_t* rows, int64_t nrows,
                            const int64_t* env_map, int n_sec, const int32_t* perm, const int32_t* idx,
                            const double* val, int chan_field, cudaStream_t s) {
  if (nrows <= 0) return cudaSuccess;
  int64_t grid = nrows < 65535 ? nrows : 65535;
  k_fold_env<<<(unsigned)grid, 256, 0, s>>>(env, out, rows, nrows, env_map, n_sec, perm, idx, val, chan_field);
  mrd::count_launch();
  return cudaGetLastError();
}

}  // namespace mrd
