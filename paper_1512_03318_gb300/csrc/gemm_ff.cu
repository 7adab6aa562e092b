// Grouped complex GEMM in float-float arithmetic (~48-bit products and sums on the FP32 pipes).
//
// Same task and segment tables as the FP64 grouped GEMM (plan.cuh: task = M N c_off ldc
// seg_begin seg_count; segment = a_off lda b_off ldb K flags, flag bit 0: A conjugate-
// transposed, bit 1: B conjugate-transposed), same result layout (FP64 complex). Operands are
// read as FP64 and split into float-float pairs when staged in shared memory; every output
// accumulates its products with exact FMA residuals and TwoSum, renormalised every 16
// terms, so the result carries ~1e-13 relative error (dot products of up to ~10^4 terms)
// against ~1e-16 for FP64, at several times the FP64 rate of GB300. Each output block is
// owned by one task, as in FP64: no atomics, deterministic results.
#include <algorithm>
#include <vector>

#include "ff.cuh"
#include "mrd_internal.h"
#include "plan.cuh"

namespace mrd {

namespace {

constexpr int kT = 32;   // output tile (complex elements per side), 2 x 2 per thread
constexpr int kK = 16;   // K chunk (kT kK a multiple of the 256 threads)
static_assert(kT * kK % 256 == 0, "tile loads: whole rounds of 256 threads");

__device__ __forceinline__ int64_t find_task_ff(const int64_t* prefix, int64_t n, int64_t item) {
  int64_t lo = 0, hi = n - 1;
  while (lo < hi) {
    const int64_t mid = (lo + hi + 1) >> 1;
    if (prefix[mid] <= item) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// complex float-float value (re, im), staged as float4 {re.hi, im.hi, re.lo, im.lo}
__device__ __forceinline__ float4 cff_from(double2 v) {
  const FF r = ff_from(v.x), i = ff_from(v.y);
  return make_float4(r.hi, i.hi, r.lo, i.lo);
}

// Complex products by three real ones (Gauss): rr = sum a_r b_r, ii = sum a_i b_i,
// ss = sum (a_r + a_i)(b_r + b_i); then Re = rr - ii, Im = ss - rr - ii. The operand sums are
// formed once per staged element, so a complex multiply-add costs 3 float-float products (36
// FP32 instructions) instead of 4 (48). Every product still carries ~2^-48 |a||b| absolute
// error, as in the four-product form, so the result's error against the output's scale is
// unchanged in order.
struct CAcc {
  FFAcc rr, ii, ss;
};

// operand element as staged: float-float operands (float4 {re.hi, im.hi, re.lo, im.lo},
// split from FP64 once by k_to_ff) are read as they are
__device__ __forceinline__ float4 ld_op(const float4* p, int64_t i, bool conj) {
  if (i < 0) return make_float4(0.f, 0.f, 0.f, 0.f);
  float4 v = p[i];
  if (conj) { v.y = -v.y; v.w = -v.w; }
  return v;
}
// (Re, Im) of an accumulated product as float-float values
__device__ __forceinline__ void cff_result(const CAcc& a, FF& re, FF& im) {
  const FF rr = ff_norm(a.rr), ii = ff_norm(a.ii), ss = ff_norm(a.ss);
  re = ff_add(rr, ff_neg(ii));
  im = ff_add(ss, ff_neg(ff_add(rr, ii)));
}
__device__ __forceinline__ void st_out(double2* c, int64_t i, const CAcc& a) {
  FF re, im;
  cff_result(a, re, im);
  c[i] = make_double2((double)re.hi + (double)re.lo, (double)im.hi + (double)im.lo);
}
__device__ __forceinline__ void st_out(float4* c, int64_t i, const CAcc& a) {
  FF re, im;
  cff_result(a, re, im);
  c[i] = make_float4(re.hi, im.hi, re.lo, im.lo);
}

// real result (Re = the accumulated real products, Im = 0)
__device__ __forceinline__ void st_out_real(double2* c, int64_t i, const FFAcc& a) {
  const FF re = ff_norm(a);
  c[i] = make_double2((double)re.hi + (double)re.lo, 0.0);
}
__device__ __forceinline__ void st_out_real(float4* c, int64_t i, const FFAcc& a) {
  const FF re = ff_norm(a);
  c[i] = make_float4(re.hi, 0.f, re.lo, 0.f);
}

// a_r + a_i of a staged element (float-float), for the third product
__device__ __forceinline__ float2 cff_sum(float4 a) {
  const FF s = ff_add(FF{a.x, a.z}, FF{a.y, a.w});
  return make_float2(s.hi, s.lo);
}

// c += a * b (complex), sa = a_r + a_i, sb = b_r + b_i
__device__ __forceinline__ void cff_mac(CAcc& c, float4 a, float2 sa, float4 b, float2 sb) {
  ff_mac(c.rr, FF{a.x, a.z}, FF{b.x, b.z});
  ff_mac(c.ii, FF{a.y, a.w}, FF{b.y, b.w});
  ff_mac(c.ss, FF{sa.x, sa.y}, FF{sb.x, sb.y});
}

__device__ __forceinline__ FFAcc ff_renorm(FFAcc a) {
  const FF r = ff_norm(a);
  return {r.hi, r.lo};
}

}  // namespace

// items (optional): (task, tile within task) of every tile in launch order, longest K first
// (ff_item_order), so that no long tile starts at the end of the grid; without it tiles run in
// task order and the task is found by binary search over the tile prefix.
// REAL: the operands are real (their imaginary parts zero, e.g. the sine / cosine machine's
// real arithmetic); only Re = sum a_r b_r is formed, one float-float product per multiply-add
// instead of three, and the result's imaginary parts are written as zero.
template <class TA, class TB, class TC, bool REAL>
__global__ void __launch_bounds__(256, 3) k_cgemm_ff(const TA* __restrict__ A, const TB* __restrict__ B,
                                                  TC* __restrict__ C, const int64_t* __restrict__ tasks,
                                                  const int64_t* __restrict__ segs,
                                                  const int64_t* __restrict__ prefix, int64_t n_tasks,
                                                  const int2* __restrict__ items) {
  __shared__ float4 As[kT][kK + 1];
  __shared__ float4 Bs[kK][kT + 1];
  __shared__ float2 Ass[kT][kK + 1];   // a_r + a_i
  __shared__ float2 Bss[kK][kT + 1];   // b_r + b_i
  const int tid = threadIdx.x;
  const int warp = tid >> 5, lane = tid & 31;
  const int64_t total = prefix[n_tasks];
  for (int64_t item = blockIdx.x; item < total; item += gridDim.x) {
    int64_t t, local;
    if (items) {
      const int2 it = items[item];
      t = it.x;
      local = it.y;
    } else {
      t = find_task_ff(prefix, n_tasks, item);
      local = item - prefix[t];
    }
    const int64_t* task = tasks + TF * t;
    const int64_t M = task[0], N = task[1], c_off = task[2], ldc = task[3];
    const int64_t seg0 = task[4], nseg = task[5];
    const int64_t tiles_n = (N + kT - 1) / kT;
    const int64_t m0 = (local / tiles_n) * kT, n0 = (local % tiles_n) * kT;
    // Each thread owns 2 x 2 outputs, each warp a 4 x 32 strip of the tile. The strips run
    // along the tile's shorter valid side, so that a warp whose strip lies wholly in the
    // padding of a small block (e.g. 4 rows of 32) skips the products and leaves its issue
    // slots to the other CTAs of the SM. Which thread computes an output changes nothing in
    // how it is computed: the results are the same bits either way.
    const int rv = M - m0 < kT ? (int)(M - m0) : kT, cv = N - n0 < kT ? (int)(N - n0) : kT;
    const bool by_col = cv < rv;
    const int ws = 4 * warp, ls = 2 * (lane >> 4), lt = 2 * (lane & 15);
    const int r0 = by_col ? lt : ws + ls, c0 = by_col ? ws + ls : lt;   // first row / column of the thread
    const bool active = (by_col ? cv : rv) > ws;
    CAcc acc[2][2];
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
      for (int j = 0; j < 2; ++j) acc[i][j] = {{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}};
    for (int64_t s = 0; s < nseg; ++s) {
      const int64_t* sg = segs + SF * (seg0 + s);
      const int64_t a_off = sg[0], lda = sg[1], b_off = sg[2], ldb = sg[3], K = sg[4];
      const int64_t flags = sg[5];
      for (int64_t k0 = 0; k0 < K; k0 += kK) {
#pragma unroll
        for (int r = 0; r < kT * kK / 256; ++r) {
          const int e = tid + r * 256;
          if (!(flags & 1)) {                           // A[m, k] at a_off + m * lda + k
            const int ar = e / kK, ak = e % kK;
            const int64_t gr = m0 + ar, gk = k0 + ak;
            const float4 v = ld_op(A, (gr < M && gk < K) ? a_off + gr * lda + gk : -1, false);
            As[ar][ak] = v;
            if (!REAL) Ass[ar][ak] = cff_sum(v);
          } else {                                      // A[m, k] = conj(A[a_off + k * lda + m])
            const int ar = e % kT, ak = e / kT;
            const int64_t gr = m0 + ar, gk = k0 + ak;
            const float4 v = ld_op(A, (gr < M && gk < K) ? a_off + gk * lda + gr : -1, true);
            As[ar][ak] = v;
            if (!REAL) Ass[ar][ak] = cff_sum(v);
          }
          if (!(flags & 2)) {                           // B[k, n] at b_off + k * ldb + n
            const int bk = e / kT, bc = e % kT;
            const int64_t gk2 = k0 + bk, gc = n0 + bc;
            const float4 v = ld_op(B, (gk2 < K && gc < N) ? b_off + gk2 * ldb + gc : -1, false);
            Bs[bk][bc] = v;
            if (!REAL) Bss[bk][bc] = cff_sum(v);
          } else {                                      // B[k, n] = conj(B[b_off + n * ldb + k])
            const int bk = e % kK, bc = e / kK;
            const int64_t gk2 = k0 + bk, gc = n0 + bc;
            const float4 v = ld_op(B, (gk2 < K && gc < N) ? b_off + gc * ldb + gk2 : -1, true);
            Bs[bk][bc] = v;
            if (!REAL) Bss[bk][bc] = cff_sum(v);
          }
        }
        __syncthreads();
        const int kn = !active ? 0 : K - k0 < kK ? (int)(K - k0) : kK;   // zero padding adds nothing: skip it
        for (int k = 0; k < kn; ++k) {
          const float4 a0 = As[r0][k], a1 = As[r0 + 1][k];
          const float4 b0 = Bs[k][c0], b1 = Bs[k][c0 + 1];
          if (REAL) {
            ff_mac(acc[0][0].rr, FF{a0.x, a0.z}, FF{b0.x, b0.z});
            ff_mac(acc[0][1].rr, FF{a0.x, a0.z}, FF{b1.x, b1.z});
            ff_mac(acc[1][0].rr, FF{a1.x, a1.z}, FF{b0.x, b0.z});
            ff_mac(acc[1][1].rr, FF{a1.x, a1.z}, FF{b1.x, b1.z});
          } else {
            const float2 sa0 = Ass[r0][k], sa1 = Ass[r0 + 1][k];
            const float2 sb0 = Bss[k][c0], sb1 = Bss[k][c0 + 1];
            cff_mac(acc[0][0], a0, sa0, b0, sb0);
            cff_mac(acc[0][1], a0, sa0, b1, sb1);
            cff_mac(acc[1][0], a1, sa1, b0, sb0);
            cff_mac(acc[1][1], a1, sa1, b1, sb1);
          }
        }
        // renormalise every accumulator (s, c) <- FastTwoSum(s, c) once per K chunk: the
        // error term c then holds at most 16 products' residuals, and its own FP32 rounding
        // stays ~2^-46 of s instead of growing with K
#pragma unroll
        for (int i = 0; i < 2; ++i)
#pragma unroll
          for (int j = 0; j < 2; ++j) {
            acc[i][j].rr = ff_renorm(acc[i][j].rr);
            if (!REAL) {
              acc[i][j].ii = ff_renorm(acc[i][j].ii);
              acc[i][j].ss = ff_renorm(acc[i][j].ss);
            }
          }
        __syncthreads();
      }
    }
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
      for (int j = 0; j < 2; ++j) {
        const int64_t r = m0 + r0 + i, c = n0 + c0 + j;
        if (r < M && c < N) {
          if (REAL) st_out_real(C, c_off + r * ldc + c, acc[i][j].rr);
          else st_out(C, c_off + r * ldc + c, acc[i][j]);
        }
      }
  }
}

// x (FP64 complex) -> float-float operand layout
__global__ void k_to_ff(const double2* __restrict__ x, float4* __restrict__ y, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    y[i] = cff_from(x[i]);
}

template <class TA, class TB, class TC>
static cudaError_t launch_ff(const TA* A, const TB* B, TC* C, const int64_t* tasks, const int64_t* segs,
                             const int64_t* prefix, int64_t n_tasks, int64_t total_tiles, int n_sm, cudaStream_t s,
                             const int2* items, bool real = false) {
  if (total_tiles <= 0) return cudaSuccess;
  int64_t grid = (int64_t)n_sm * 8;
  if (grid > total_tiles) grid = total_tiles;
  if (real)
    k_cgemm_ff<TA, TB, TC, true><<<(unsigned)grid, 256, 0, s>>>(A, B, C, tasks, segs, prefix, n_tasks, items);
  else
    k_cgemm_ff<TA, TB, TC, false><<<(unsigned)grid, 256, 0, s>>>(A, B, C, tasks, segs, prefix, n_tasks, items);
  mrd::count_launch();
  return cudaGetLastError();
}

// real operands already in float-float layout (imaginary parts zero): Re only, Im written 0
cudaError_t launch_rgemm_ff_packed(const float4* A, const float4* B, float4* c_ff, double2* c64, const int64_t* tasks,
                                   const int64_t* segs, const int64_t* prefix, int64_t n_tasks, int64_t total_tiles,
                                   int n_sm, cudaStream_t s, const int2* items) {
  if (c_ff) return launch_ff(A, B, c_ff, tasks, segs, prefix, n_tasks, total_tiles, n_sm, s, items, true);
  return launch_ff(A, B, c64, tasks, segs, prefix, n_tasks, total_tiles, n_sm, s, items, true);
}

// operands already in float-float layout; result in float-float (c_ff) or FP64 (c64)
cudaError_t launch_cgemm_ff_packed(const float4* A, const float4* B, float4* c_ff, double2* c64, const int64_t* tasks,
                                   const int64_t* segs, const int64_t* prefix, int64_t n_tasks, int64_t total_tiles,
                                   int n_sm, cudaStream_t s, const int2* items) {
  if (c_ff) return launch_ff(A, B, c_ff, tasks, segs, prefix, n_tasks, total_tiles, n_sm, s, items);
  return launch_ff(A, B, c64, tasks, segs, prefix, n_tasks, total_tiles, n_sm, s, items);
}

// Launch order of the tiles of a grouped GEMM (host): (task, tile within task) for every tile
// of 32 x 32 outputs, tasks in decreasing order of their inner dimension (the sum of their
// segments' K, which sets the time of each of their tiles), ties in task order.
std::vector<int2> ff_item_order(const int64_t* tasks, const int64_t* segs, int64_t n_tasks) {
  std::vector<int64_t> cost(n_tasks), idx(n_tasks);
  for (int64_t t = 0; t < n_tasks; ++t) {
    const int64_t* r = tasks + TF * t;
    int64_t k = 0;
    for (int64_t q = 0; q < r[5]; ++q) k += segs[SF * (r[4] + q) + 4];
    cost[t] = k;
    idx[t] = t;
  }
  std::stable_sort(idx.begin(), idx.end(), [&](int64_t a, int64_t b) { return cost[a] > cost[b]; });
  std::vector<int2> items;
  for (int64_t t : idx) {
    const int64_t* r = tasks + TF * t;
    const int64_t n = ((r[0] + kT - 1) / kT) * ((r[1] + kT - 1) / kT);
    for (int64_t l = 0; l < n; ++l) items.push_back(make_int2((int)t, (int)l));
  }
  return items;
}

cudaError_t to_ff(const double2* x, float4* y, int64_t n, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  const int64_t blocks = (n + 255) / 256;
  k_to_ff<<<(unsigned)(blocks < 8192 ? blocks : 8192), 256, 0, s>>>(x, y, n);
  mrd::count_launch();
  return cudaGetLastError();
}

}  // namespace mrd
