// Block SVD of the two-site tensor and truncation to the bond dimension (the Schmidt
// decomposition of Sec. III.C: theta = sum_alpha lambda_alpha |L_alpha>|R_alpha>, with the
// Schmidt states labelled by the charges (N, K) of their block).
//
// theta is block diagonal in the middle charge, so every block M_q (rowdim x coldim) is
// decomposed separately, M_q = U_q S_q V_q^+, by the one-sided Jacobi method (Hestenes):
// the columns of X = M_q (or M_q^+ when it is wide, so that X is tall) are rotated pairwise
// until mutually orthogonal; the column norms are the singular values, the normalised columns
// the left singular vectors of X, the accumulated rotations its right singular vectors. It
// is FP64 throughout and converges to high relative accuracy. All blocks advance together:
// one launch per round of the round-robin pair schedule, one warp per column pair.
//
// Truncation keeps the globally largest chi singular values above cutoff * s_max, ties
// broken by (value desc, block asc, index asc); the kept values are renormalised to
// sum s^2 = 1 and the discarded weight is reported.
#include <cmath>

#include "mrd_internal.h"

namespace mrd {

// Per-block descriptor (int64): m n p r x_off v_off out_u_off out_vh_off s_off wide
enum { SVF = 10 };

namespace {

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// X (p x r, column-major) from the row-major block M (m x n): X = M if m >= n else M^+.
__global__ void k_svd_load(const double2* __restrict__ theta, const int64_t* __restrict__ blk,
                           const int64_t* __restrict__ src_off, int nblk, double2* __restrict__ work) {
  const int b = blockIdx.y;
  if (b >= nblk) return;
  const int64_t* d = blk + SVF * b;
  const int64_t n = d[1], p = d[2], r = d[3], x_off = d[4], v_off = d[5];
  const bool wide = d[9] != 0;
  const double2* M = theta + src_off[b];
  double2* X = work + x_off;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < p * r; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t row = e % p, col = e / p;      // X[row, col]
    double2 v;
    if (!wide) {
      v = M[row * n + col];                       // X = M: X[row, col] = M[row, col]
    } else {
      const double2 t = M[col * n + row];         // X = M^+: X[row, col] = conj(M[col, row])
      v = make_double2(t.x, -t.y);
    }
    X[col * p + row] = v;
  }
  double2* V = work + v_off;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < r * r; e += (int64_t)gridDim.x * blockDim.x)
    V[e] = make_double2((e / r) == (e % r) ? 1.0 : 0.0, 0.0);
}

// One round of the round-robin schedule for every block. Warp w handles pair (w - pair_prefix
// of its block); the block's columns are padded to an even count rr, the dummy column rr-1
// (when r is odd) is skipped.
__global__ void k_svd_round(double2* __restrict__ work, const int64_t* __restrict__ blk,
                            const int64_t* __restrict__ pair_prefix, int nblk, int round, double tol,
                            int* __restrict__ rotated) {
  const int64_t wglob = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (wglob >= pair_prefix[nblk]) return;
  int lo = 0, hi = nblk - 1;   // largest b with pair_prefix[b] <= wglob
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (pair_prefix[mid] <= wglob) lo = mid; else hi = mid - 1;
  }
  const int b = lo;
  const int64_t* d = blk + SVF * b;
  const int64_t p = d[2], r = d[3];
  const int64_t rr = r + (r & 1);
  if (rr < 2 || round >= rr - 1) return;
  const int64_t k = wglob - pair_prefix[b];
  int64_t i, j;
  if (k == 0) {
    i = round;
    j = rr - 1;
  } else {
    i = (round + k) % (rr - 1);
    j = (round - k + (rr - 1)) % (rr - 1);
  }
  if (i >= r || j >= r) return;   // dummy column
  double2* X = work + d[4];
  double2* V = work + d[5];
  double2* xi = X + i * p;
  double2* xj = X + j * p;
  double a = 0.0, bb = 0.0, gr = 0.0, gi = 0.0;
  for (int64_t t = lane; t < p; t += 32) {
    const double2 u = xi[t], v = xj[t];
    a = fma(u.x, u.x, fma(u.y, u.y, a));
    bb = fma(v.x, v.x, fma(v.y, v.y, bb));
    gr = fma(u.x, v.x, fma(u.y, v.y, gr));     // Re(conj(u) v)
    gi = fma(u.x, v.y, fma(-u.y, v.x, gi));    // Im(conj(u) v)
  }
  a = warp_sum(a);
  bb = warp_sum(bb);
  gr = warp_sum(gr);
  gi = warp_sum(gi);
  const double g = sqrt(gr * gr + gi * gi);
  if (!(g > tol * sqrt(a * bb)) || a == 0.0 || bb == 0.0) return;
  // phase-free real rotation on (x_i, e^{-i phi} x_j), phi = arg(gamma)
  const double ph_r = gr / g, ph_i = -gi / g;          // e^{-i phi}
  const double zeta = (bb - a) / (2.0 * g);
  const double t = (zeta >= 0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
  const double c = 1.0 / sqrt(1.0 + t * t), s = c * t;
  for (int64_t q = lane; q < p; q += 32) {
    const double2 u = xi[q], v0 = xj[q];
    const double2 v = make_double2(v0.x * ph_r - v0.y * ph_i, v0.x * ph_i + v0.y * ph_r);
    xi[q] = make_double2(c * u.x - s * v.x, c * u.y - s * v.y);
    xj[q] = make_double2(s * u.x + c * v.x, s * u.y + c * v.y);
  }
  double2* vi = V + i * r;
  double2* vj = V + j * r;
  for (int64_t q = lane; q < r; q += 32) {
    const double2 u = vi[q], v0 = vj[q];
    const double2 v = make_double2(v0.x * ph_r - v0.y * ph_i, v0.x * ph_i + v0.y * ph_r);
    vi[q] = make_double2(c * u.x - s * v.x, c * u.y - s * v.y);
    vj[q] = make_double2(s * u.x + c * v.x, s * u.y + c * v.y);
  }
  if (lane == 0) atomicAdd(rotated, 1);
}

// Per block: singular values (column norms) sorted descending (ties by column index), then
// U (m x r) and Vh (r x n) of M in row-major order, and S.
__global__ void k_svd_finish(const double2* __restrict__ work, const int64_t* __restrict__ blk, int nblk,
                             double2* __restrict__ U, double2* __restrict__ Vh, double* __restrict__ S,
                             int* __restrict__ order_scratch) {
  const int b = blockIdx.x;
  if (b >= nblk) return;
  const int64_t* d = blk + SVF * b;
  const int64_t m = d[0], n = d[1], p = d[2], r = d[3];
  const bool wide = d[9] != 0;
  const double2* X = work + d[4];
  const double2* V = work + d[5];
  double* s = S + d[8];
  int* ord = order_scratch + d[8];
  // norms
  for (int64_t j = threadIdx.x; j < r; j += blockDim.x) {
    double acc = 0.0;
    for (int64_t t = 0; t < p; ++t) {
      const double2 x = X[j * p + t];
      acc = fma(x.x, x.x, fma(x.y, x.y, acc));
    }
    s[j] = sqrt(acc);
  }
  __syncthreads();
  // rank sort (descending value, then ascending index)
  for (int64_t j = threadIdx.x; j < r; j += blockDim.x) {
    const double v = s[j];
    int rank = 0;
    for (int64_t k = 0; k < r; ++k) {
      const double w = s[k];
      rank += (w > v) || (w == v && k < j);
    }
    ord[rank] = (int)j;
  }
  __syncthreads();
  double2* u = U + d[6];
  double2* vh = Vh + d[7];
  // output k-th singular triple from column ord[k]
  for (int64_t e = threadIdx.x; e < m * r; e += blockDim.x) {
    const int64_t row = e / r, kk = e % r;
    const int j = ord[kk];
    const double sig = s[j];
    double2 val;
    if (!wide) {                          // U_M = X / sigma
      const double2 x = X[(int64_t)j * p + row];
      const double inv = sig > 0 ? 1.0 / sig : 0.0;
      val = make_double2(x.x * inv, x.y * inv);
    } else {                              // U_M = V_X
      val = V[(int64_t)j * r + row];
    }
    u[row * r + kk] = val;
  }
  for (int64_t e = threadIdx.x; e < r * n; e += blockDim.x) {
    const int64_t kk = e / n, col = e % n;
    const int j = ord[kk];
    const double sig = s[j];
    double2 val;
    if (!wide) {                          // Vh_M[k, col] = conj(V_X[col, j])
      const double2 v = V[(int64_t)j * r + col];
      val = make_double2(v.x, -v.y);
    } else {                              // Vh_M[k, col] = conj(X[col, j]) / sigma
      const double2 x = X[(int64_t)j * p + col];
      const double inv = sig > 0 ? 1.0 / sig : 0.0;
      val = make_double2(x.x * inv, -x.y * inv);
    }
    vh[kk * n + col] = val;
  }
}

// Values are sorted in place after the vectors were written.
__global__ void k_svd_sort_values(const int64_t* __restrict__ blk, int nblk, double* __restrict__ S,
                                  double* __restrict__ S_sorted) {
  const int b = blockIdx.x;
  if (b >= nblk) return;
  const int64_t* d = blk + SVF * b;
  const int64_t r = d[3];
  const double* s = S + d[8];
  double* o = S_sorted + d[8];
  for (int64_t j = threadIdx.x; j < r; j += blockDim.x) {
    const double v = s[j];
    int rank = 0;
    for (int64_t k = 0; k < r; ++k) {
      const double w = s[k];
      rank += (w > v) || (w == v && k < j);
    }
    o[rank] = v;
  }
}

// Global truncation (one CTA): keep[b] = number of kept values of block b; info[0] = scale
// applied to the kept values (1/sqrt(sum kept s^2)), info[1] = discarded weight
// (sum of discarded s^2 / total), info[2] = s_max.
__global__ void k_truncate(const int64_t* __restrict__ blk, int nblk, const double* __restrict__ S_sorted,
                           int64_t total, int chi, double cutoff, int* __restrict__ keep, double* __restrict__ info,
                           int* __restrict__ flat_block) {
  __shared__ double smax_s;
  const int tid = threadIdx.x;
  // block of every flat index
  for (int b = 0; b < nblk; ++b) {
    const int64_t* d = blk + SVF * b;
    for (int64_t k = tid; k < d[3]; k += blockDim.x) flat_block[d[8] + k] = b;
  }
  if (tid == 0) {
    double mx = 0.0;
    for (int b = 0; b < nblk; ++b) {
      const int64_t* d = blk + SVF * b;
      if (d[3] > 0) mx = fmax(mx, S_sorted[d[8]]);
    }
    smax_s = mx;
  }
  for (int b = tid; b < nblk; b += blockDim.x) keep[b] = 0;
  __syncthreads();
  const double smax = smax_s;
  for (int64_t e = tid; e < total; e += blockDim.x) {
    const double v = S_sorted[e];
    const int be = flat_block[e];
    int64_t rank = 0;
    for (int64_t f = 0; f < total; ++f) {
      const double w = S_sorted[f];
      const int bf = flat_block[f];
      rank += (w > v) || (w == v && (bf < be || (bf == be && f < e)));
    }
    if (rank < chi && v > cutoff * smax) atomicAdd(&keep[be], 1);
  }
  __syncthreads();
  if (tid == 0) {
    double kept = 0.0, all = 0.0;
    for (int b = 0; b < nblk; ++b) {
      const int64_t* d = blk + SVF * b;
      for (int64_t k = 0; k < d[3]; ++k) {
        const double v = S_sorted[d[8] + k];
        all += v * v;
        if (k < keep[b]) kept += v * v;
      }
    }
    info[0] = kept > 0 ? 1.0 / sqrt(kept) : 0.0;
    info[1] = all > 0 ? (all - kept) / all : 0.0;
    info[2] = smax;
  }
}

}  // namespace

cudaError_t svd_load(const double2* theta, const int64_t* blk, const int64_t* src_off, int nblk, double2* work,
                     cudaStream_t s) {
  if (nblk == 0) return cudaSuccess;
  dim3 grid(64, nblk);
  k_svd_load<<<grid, 256, 0, s>>>(theta, blk, src_off, nblk, work);
  mrd::count_launch();
  return cudaGetLastError();
}

cudaError_t svd_round(double2* work, const int64_t* blk, const int64_t* pair_prefix, int nblk, int64_t npairs,
                      int round, double tol, int* rotated, cudaStream_t s) {
  if (npairs == 0) return cudaSuccess;
  const int64_t threads = npairs * 32;
  k_svd_round<<<(unsigned)((threads + 255) / 256), 256, 0, s>>>(work, blk, pair_prefix, nblk, round, tol, rotated);
  mrd::count_launch();
  return cudaGetLastError();
}

cudaError_t svd_finish(const double2* work, const int64_t* blk, int nblk, double2* U, double2* Vh, double* S,
                       double* S_sorted, int* order_scratch, cudaStream_t s) {
  if (nblk == 0) return cudaSuccess;
  k_svd_finish<<<nblk, 256, 0, s>>>(work, blk, nblk, U, Vh, S, order_scratch);
  mrd::count_launch();
  k_svd_sort_values<<<nblk, 256, 0, s>>>(blk, nblk, S, S_sorted);
  mrd::count_launch();
  return cudaGetLastError();
}

cudaError_t svd_truncate(const int64_t* blk, int nblk, const double* S_sorted, int64_t total, int chi, double cutoff,
                         int* keep, double* info, int* flat_block, cudaStream_t s) {
  k_truncate<<<1, 1024, 0, s>>>(blk, nblk, S_sorted, total, chi, cutoff, keep, info, flat_block);
  mrd::count_launch();
  return cudaGetLastError();
}

}  // namespace mrd
