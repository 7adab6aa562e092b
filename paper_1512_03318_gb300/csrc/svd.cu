// Block SVD of the two-site tensor and truncation to the bond dimension (the Schmidt
// decomposition of Sec. III.C: theta = sum_alpha lambda_alpha |L_alpha>|R_alpha>, with the
// Schmidt states labelled by the charges (N, K) of their block).
//
// theta is block diagonal in the middle charge, so every block M_q (rowdim x coldim) is
// decomposed separately, M_q = U_q S_q V_q^+, by the one-sided Jacobi method (Hestenes):
// the columns of X are rotated pairwise until mutually orthogonal; their norms are the
// singular values and the normalised columns an orthonormal set of singular vectors. X = M_q
// gives U_q (the "left" side), X = M_q^+ gives V_q (the "right" side); the caller picks the
// side that must be exactly orthonormal and obtains the other factor by projection
// (U^+ M or M V, an FP64 GEMM). Sweeps run first in FP32 (cheap, columns orthogonal to
// ~1e-6), their accumulated rotation is applied to the FP64 X by one GEMM, and FP64 sweeps
// finish (quadratic convergence, typically 2-3 sweeps). All blocks advance together: one
// launch per round of the round-robin pair schedule, one warp per column pair.
//
// Truncation keeps the globally largest chi singular values above cutoff * s_max, ties
// broken by (value desc, block asc, index asc); the kept values are renormalised to
// sum s^2 = 1 and the discarded weight is reported.
#include <cmath>

#include "mrd_internal.h"

namespace mrd {

// Per-block descriptor (int64): m n p r x_off v_off out_u_off out_vh_off s_off wide
enum { SVF = 12 };   // + field 10: X32 offset, 11: V32 offset (float2 units)

namespace {

// X (p x r, column-major) from the row-major block M (m x n): X = M if m >= n else M^+.
__global__ void k_svd_load(const double2* __restrict__ theta, const int64_t* __restrict__ blk,
                           const int64_t* __restrict__ src_off, int nblk, double2* __restrict__ work,
                           double* __restrict__ fro2) {
  const int b = blockIdx.y;
  if (b >= nblk) return;
  const int64_t* d = blk + SVF * b;
  const int64_t n = d[1], p = d[2], r = d[3], x_off = d[4], v_off = d[5];
  const bool wide = d[9] != 0;
  const double2* M = theta + src_off[b];
  double2* X = work + x_off;
  double part = 0.0;
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
    part = fma(v.x, v.x, fma(v.y, v.y, part));
  }
  for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
  if ((threadIdx.x & 31) == 0 && part != 0.0) atomicAdd(&fro2[b], part);
  double2* V = work + v_off;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < r * r; e += (int64_t)gridDim.x * blockDim.x)
    V[e] = make_double2((e / r) == (e % r) ? 1.0 : 0.0, 0.0);
}

// One round of the round-robin schedule for every block. Warp w handles pair (w - pair_prefix
// of its block); the block's columns are padded to an even count rr, the dummy column rr-1
// (when r is odd) is skipped. T is float (pre-sweeps) or double.
template <class T, class T2>
__global__ void k_svd_round(T2* __restrict__ work, const int64_t* __restrict__ blk, int xf, int vf,
                            const int64_t* __restrict__ pair_prefix, int nblk, int round, T tol,
                            const double* __restrict__ fro2, double zero_rel, int* __restrict__ rotated) {
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
  T2* X = work + d[xf];
  T2* V = vf >= 0 ? work + d[vf] : nullptr;
  T2* xi = X + i * p;
  T2* xj = X + j * p;
  T a = 0, bb = 0, gr = 0, gi = 0;
  for (int64_t t = lane; t < p; t += 32) {
    const T2 u = xi[t], v = xj[t];
    a = fma(u.x, u.x, fma(u.y, u.y, a));
    bb = fma(v.x, v.x, fma(v.y, v.y, bb));
    gr = fma(u.x, v.x, fma(u.y, v.y, gr));     // Re(conj(u) v)
    gi = fma(u.x, v.y, fma(-u.y, v.x, gi));    // Im(conj(u) v)
  }
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_xor_sync(0xffffffffu, a, o);
    bb += __shfl_xor_sync(0xffffffffu, bb, o);
    gr += __shfl_xor_sync(0xffffffffu, gr, o);
    gi += __shfl_xor_sync(0xffffffffu, gi, o);
  }
  const T g = sqrt(gr * gr + gi * gi);
  // a column whose norm is negligible against the block (|x|^2 <= zero_rel |M|_F^2) is a
  // numerical zero (rank deficiency): it is neither rotated nor counted as unconverged
  const double floor2 = zero_rel * fro2[b];
  if ((double)a <= floor2 || (double)bb <= floor2) return;
  if (!(g > tol * sqrt(a * bb))) return;
  // phase-free real rotation on (x_i, e^{-i phi} x_j), phi = arg(gamma)
  const T ph_r = gr / g, ph_i = -gi / g;          // e^{-i phi}
  const T zeta = (bb - a) / (T(2) * g);
  const T t = (zeta >= T(0) ? T(1) : T(-1)) / (fabs(zeta) + sqrt(T(1) + zeta * zeta));
  const T c = T(1) / sqrt(T(1) + t * t), s = c * t;
  for (int64_t q = lane; q < p; q += 32) {
    const T2 u = xi[q], v0 = xj[q];
    T2 v;
    v.x = v0.x * ph_r - v0.y * ph_i;
    v.y = v0.x * ph_i + v0.y * ph_r;
    T2 o1, o2;
    o1.x = c * u.x - s * v.x; o1.y = c * u.y - s * v.y;
    o2.x = s * u.x + c * v.x; o2.y = s * u.y + c * v.y;
    xi[q] = o1;
    xj[q] = o2;
  }
  if (V == nullptr) {
    if (lane == 0) atomicAdd(rotated, 1);
    return;
  }
  T2* vi = V + i * r;
  T2* vj = V + j * r;
  for (int64_t q = lane; q < r; q += 32) {
    const T2 u = vi[q], v0 = vj[q];
    T2 v;
    v.x = v0.x * ph_r - v0.y * ph_i;
    v.y = v0.x * ph_i + v0.y * ph_r;
    T2 o1, o2;
    o1.x = c * u.x - s * v.x; o1.y = c * u.y - s * v.y;
    o2.x = s * u.x + c * v.x; o2.y = s * u.y + c * v.y;
    vi[q] = o1;
    vj[q] = o2;
  }
  if (lane == 0) atomicAdd(rotated, 1);
}

// FP32 working copies: X32 (descriptor field 10) from X, V32 (field 11) = identity.
__global__ void k_svd_to_f32(const double2* __restrict__ work, float2* __restrict__ w32,
                             const int64_t* __restrict__ blk, int nblk) {
  const int b = blockIdx.y;
  if (b >= nblk) return;
  const int64_t* d = blk + SVF * b;
  const int64_t p = d[2], r = d[3];
  const double2* X = work + d[4];
  float2* X32 = w32 + d[10];
  float2* V32 = w32 + d[11];
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < p * r; e += (int64_t)gridDim.x * blockDim.x)
    X32[e] = make_float2((float)X[e].x, (float)X[e].y);
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < r * r; e += (int64_t)gridDim.x * blockDim.x)
    V32[e] = make_float2((e / r) == (e % r) ? 1.f : 0.f, 0.f);
}

// V (FP64, field 5) = V32; the FP64 X is then multiplied by V32 with a grouped GEMM.
__global__ void k_svd_v_from_f32(double2* __restrict__ work, const float2* __restrict__ w32,
                                 const int64_t* __restrict__ blk, int nblk) {
  const int b = blockIdx.y;
  if (b >= nblk) return;
  const int64_t* d = blk + SVF * b;
  const int64_t r = d[3];
  double2* V = work + d[5];
  const float2* V32 = w32 + d[11];
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < r * r; e += (int64_t)gridDim.x * blockDim.x)
    V[e] = make_double2((double)V32[e].x, (double)V32[e].y);
}

// Per block: singular values (column norms of X) sorted descending (ties by column index),
// and the orthonormal factor of the block's side: side 0 (X = M): U (m x r, row-major) with
// column k = X column ord[k] / sigma; side 1 (X = M^+): V^+ (r x n, row-major) with row k =
// conj(X column ord[k]) / sigma. Columns with sigma = 0 are written as zero.
__global__ void k_svd_finish(const double2* __restrict__ work, const int64_t* __restrict__ blk, int nblk,
                             double2* __restrict__ U, double2* __restrict__ Vh, double* __restrict__ S,
                             int* __restrict__ order_scratch, const double* __restrict__ fro2) {
  const int b = blockIdx.x;
  if (b >= nblk) return;
  const int64_t* d = blk + SVF * b;
  const int64_t m = d[0], n = d[1], p = d[2], r = d[3];
  const bool wide = d[9] != 0;
  const double2* X = work + d[4];
  double* s = S + d[8];
  int* ord = order_scratch + d[8];
  for (int64_t j = threadIdx.x; j < r; j += blockDim.x) {
    double acc = 0.0;
    for (int64_t t = 0; t < p; ++t) {
      const double2 x = X[j * p + t];
      acc = fma(x.x, x.x, fma(x.y, x.y, acc));
    }
    s[j] = acc <= 1e-28 * fro2[b] ? 0.0 : sqrt(acc);   // numerical zero (see the rounds)
  }
  __syncthreads();
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
  if (!wide) {
    double2* u = U + d[6];
    for (int64_t e = threadIdx.x; e < m * r; e += blockDim.x) {
      const int64_t row = e / r, kk = e % r;
      const int j = ord[kk];
      const double sig = s[j];
      const double2 x = X[(int64_t)j * p + row];
      const double inv = sig > 0 ? 1.0 / sig : 0.0;
      u[row * r + kk] = make_double2(x.x * inv, x.y * inv);
    }
  } else {
    double2* vh = Vh + d[7];
    for (int64_t e = threadIdx.x; e < r * n; e += blockDim.x) {
      const int64_t kk = e / n, col = e % n;
      const int j = ord[kk];
      const double sig = s[j];
      const double2 x = X[(int64_t)j * p + col];
      const double inv = sig > 0 ? 1.0 / sig : 0.0;
      vh[kk * n + col] = make_double2(x.x * inv, -x.y * inv);
    }
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
                     double* fro2, cudaStream_t s) {
  if (nblk == 0) return cudaSuccess;
  cudaError_t e = cudaMemsetAsync(fro2, 0, (size_t)nblk * 8, s);
  if (e != cudaSuccess) return e;
  dim3 grid(64, nblk);
  k_svd_load<<<grid, 256, 0, s>>>(theta, blk, src_off, nblk, work, fro2);
  mrd::count_launch();
  return cudaGetLastError();
}

cudaError_t svd_round(double2* work, const int64_t* blk, const int64_t* pair_prefix, int nblk, int64_t npairs,
                      int round, double tol, const double* fro2, int* rotated, cudaStream_t s) {
  if (npairs == 0) return cudaSuccess;
  const int64_t threads = npairs * 32;
  k_svd_round<double, double2><<<(unsigned)((threads + 255) / 256), 256, 0, s>>>(work, blk, 4, -1, pair_prefix,
                                                                                nblk, round, tol, fro2, 1e-28,
                                                                                rotated);
  mrd::count_launch();
  return cudaGetLastError();
}

cudaError_t svd_round32(float2* w32, const int64_t* blk, const int64_t* pair_prefix, int nblk, int64_t npairs,
                        int round, float tol, const double* fro2, int* rotated, cudaStream_t s) {
  if (npairs == 0) return cudaSuccess;
  const int64_t threads = npairs * 32;
  k_svd_round<float, float2><<<(unsigned)((threads + 255) / 256), 256, 0, s>>>(w32, blk, 10, 11, pair_prefix, nblk,
                                                                              round, tol, fro2, 1e-12, rotated);
  mrd::count_launch();
  return cudaGetLastError();
}

cudaError_t svd_to_f32(const double2* work, float2* w32, const int64_t* blk, int nblk, cudaStream_t s) {
  if (nblk == 0) return cudaSuccess;
  dim3 grid(64, nblk);
  k_svd_to_f32<<<grid, 256, 0, s>>>(work, w32, blk, nblk);
  mrd::count_launch();
  return cudaGetLastError();
}

cudaError_t svd_v_from_f32(double2* work, const float2* w32, const int64_t* blk, int nblk, cudaStream_t s) {
  if (nblk == 0) return cudaSuccess;
  dim3 grid(16, nblk);
  k_svd_v_from_f32<<<grid, 256, 0, s>>>(work, w32, blk, nblk);
  mrd::count_launch();
  return cudaGetLastError();
}

cudaError_t svd_finish(const double2* work, const int64_t* blk, int nblk, double2* U, double2* Vh, double* S,
                       double* S_sorted, int* order_scratch, const double* fro2, cudaStream_t s) {
  if (nblk == 0) return cudaSuccess;
  k_svd_finish<<<nblk, 256, 0, s>>>(work, blk, nblk, U, Vh, S, order_scratch, fro2);
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
