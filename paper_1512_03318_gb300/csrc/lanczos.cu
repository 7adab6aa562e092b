// Lanczos ground-state solver for the two-site H_eff (standard DMRG eigensolver; the paper
// relies on DMRG as in its refs. W92, S2005, S2011 without restating it).
//
// Krylov recursion with full reorthogonalisation: for j = 0, 1, ...
//   w = H v_j;  a local pass c1 = [v_{j-1} v_j]^+ w, w -= [v_{j-1} v_j] c1 (the three-term
//   recurrence), then one full classical Gram-Schmidt pass c2 = V^+ w, w -= V c2
//   (V = [v_0 .. v_j]); alpha_j = Re of v_j's coefficient summed over both passes;
//   beta_j = |w|;  v_{j+1} = w / beta_j;
//   lowest eigenpair (E_j, y) of the tridiagonal T_j = tridiag(beta, alpha, beta).
// Stops when |E_j - E_{j-1}| < tol |E_j|, when beta_j vanishes (invariant subspace) or at
// max_iter; the ground vector is V y, normalised.
//
// All vector arithmetic runs in FP64 on the device with fixed-shape reductions (partial sums
// per CTA, then one CTA), so results are bit-reproducible run to run. The tridiagonal
// eigenproblem is solved on the device by one warp: Sturm-count multisection for the lowest
// eigenvalue, inverse iteration with a pivoted tridiagonal LU for its vector.
#include <cmath>
#include <vector>

#include "mrd_internal.h"

namespace mrd {

namespace {

constexpr int kRedThreads = 256;
constexpr int kRedBlocks = 304;   // 2 per SM; fixed for reproducible reduction order

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Device state of one Lanczos run. j is the current step: the kernels of a step read it,
// so that one captured CUDA graph of a step serves every step.
struct LzState {
  double alpha[MRD_LANCZOS_MAX_ITER + 1];
  double beta[MRD_LANCZOS_MAX_ITER + 1];
  double y[MRD_LANCZOS_MAX_ITER + 1];
  double ritz[MRD_LANCZOS_MAX_ITER + 1];   // lowest Ritz value after each step of the run
  double energy;
  double beta_last;
  double inv_beta;                         // 1 / beta_j of the current step
  int flags;
  int j;
};

// number of vectors of a reduction: nv >= 0 as given, nv < 0 means v_0 .. v_j of the state
// Vectors of a reduction or combination: nv >= 0: v_0 .. v_{nv-1}; nv = -1: v_0 .. v_j (all);
// nv = -2: v_{j-1}, v_j (the two the three-term recurrence involves; v_0 alone at j = 0).
__device__ __forceinline__ int eff_nv(int nv, const LzState* st) {
  return nv >= 0 ? nv : (nv == -1 ? st->j + 1 : (st->j > 0 ? 2 : 1));
}
__device__ __forceinline__ int first_v(int nv, const LzState* st) { return nv == -2 && st->j > 0 ? st->j - 1 : 0; }

constexpr int kJB = 4;   // vectors per pass of k_multidot (w is read once per pass)

// partial[b * nv + j] = sum over this CTA's share of conj(V_j) . w, j < nv (re, im interleaved)
__global__ void __launch_bounds__(kRedThreads) k_multidot(const double2* __restrict__ V, int64_t ldv, int nv_arg,
                                                          const LzState* __restrict__ st,
                                                          const double2* __restrict__ w, int64_t n,
                                                          double2* __restrict__ partial) {
  __shared__ double sre[kJB][kRedThreads / 32], sim[kJB][kRedThreads / 32];
  const int nv = eff_nv(nv_arg, st);
  V += (int64_t)first_v(nv_arg, st) * ldv;
  const int64_t chunk = (n + gridDim.x - 1) / gridDim.x;
  const int64_t b = blockIdx.x * chunk;
  const int64_t e = b + chunk < n ? b + chunk : n;
  constexpr int kE = 4;   // elements per thread and step: their loads are in flight together
  for (int j0 = 0; j0 < nv; j0 += kJB) {
    double re[kJB], im[kJB];
#pragma unroll
    for (int q = 0; q < kJB; ++q) re[q] = im[q] = 0.0;
    for (int64_t i0 = b + threadIdx.x; i0 < e; i0 += (int64_t)kE * blockDim.x) {
      double2 y[kE];
#pragma unroll
      for (int u = 0; u < kE; ++u) {
        const int64_t i = i0 + (int64_t)u * blockDim.x;
        y[u] = i < e ? w[i] : make_double2(0.0, 0.0);
      }
#pragma unroll
      for (int q = 0; q < kJB; ++q) {
        if (j0 + q < nv) {
          double2 x[kE];
#pragma unroll
          for (int u = 0; u < kE; ++u) {
            const int64_t i = i0 + (int64_t)u * blockDim.x;
            x[u] = i < e ? V[(int64_t)(j0 + q) * ldv + i] : make_double2(0.0, 0.0);
          }
#pragma unroll
          for (int u = 0; u < kE; ++u) {
            re[q] = fma(x[u].x, y[u].x, re[q]);
            re[q] = fma(x[u].y, y[u].y, re[q]);
            im[q] = fma(x[u].x, y[u].y, im[q]);
            im[q] = fma(-x[u].y, y[u].x, im[q]);
          }
        }
      }
    }
#pragma unroll
    for (int q = 0; q < kJB; ++q) {
      re[q] = warp_sum(re[q]);
      im[q] = warp_sum(im[q]);
      if ((threadIdx.x & 31) == 0) {
        sre[q][threadIdx.x >> 5] = re[q];
        sim[q][threadIdx.x >> 5] = im[q];
      }
    }
    __syncthreads();
    if (threadIdx.x < kJB && j0 + (int)threadIdx.x < nv) {
      const int q = threadIdx.x;
      double a = 0.0, c = 0.0;
      for (int k = 0; k < kRedThreads / 32; ++k) {
        a += sre[q][k];
        c += sim[q][k];
      }
      partial[(int64_t)blockIdx.x * nv + j0 + q] = make_double2(a, c);
    }
    __syncthreads();
  }
}

// out[j] = sum_b partial[b * nv + j]; one warp per j, fixed order (lane-strided sums, then
// a shuffle tree).
__global__ void k_finish_dots(const double2* __restrict__ partial, int nblocks, int nv_arg,
                              const LzState* __restrict__ st, double2* __restrict__ out) {
  const int nv = eff_nv(nv_arg, st);
  const int j = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (j >= nv) return;
  double a = 0.0, c = 0.0;
  for (int b = lane; b < nblocks; b += 32) {
    const double2 p = partial[(int64_t)b * nv + j];
    a += p.x;
    c += p.y;
  }
  a = warp_sum(a);
  c = warp_sum(c);
  if (lane == 0) out[j] = make_double2(a, c);
}

// w -= sum_j c[j] V_j
__global__ void k_sub_combination(const double2* __restrict__ V, int64_t ldv, int nv_arg,
                                  const LzState* __restrict__ st, const double2* __restrict__ c,
                                  double2* __restrict__ w, int64_t n) {
  const int nv = eff_nv(nv_arg, st);
  V += (int64_t)first_v(nv_arg, st) * ldv;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    double2 acc = w[i];
    for (int j = 0; j < nv; ++j) {
      const double2 v = V[(int64_t)j * ldv + i], cj = c[j];
      acc.x -= cj.x * v.x - cj.y * v.y;
      acc.y -= cj.x * v.y + cj.y * v.x;
    }
    w[i] = acc;
  }
}

// FP32 form of the full Gram-Schmidt pass, for Lanczos runs whose matvec is itself a
// reduced-precision product (TF32 or split BF16, ~1e-5 .. 1e-3 relative). After the FP64
// local pass the remaining coefficients <v_i, w> are the small residue of rounding; computed
// from FP32 copies of v_i and w their error is ~2^-24 |w| / sqrt(n) (random rounding over n
// terms), which keeps the basis orthogonal to ~1e-10 relative, far inside the sqrt(eps)
// (semi-orthogonality) level that keeps the Ritz values exact to working precision. FP32
// halves the bytes and moves the products off the FP64 pipe (2 operations per clock per SM),
// which bounds the FP64 pass at ~2.5 TB/s.
constexpr int kMD32Chunk = 1024;   // elements of w per CTA of k_multidot32
inline int64_t md32_blocks(int64_t n) { return n > 0 ? (n + kMD32Chunk - 1) / kMD32Chunk : 1; }

__global__ void k_to_f32(const double2* __restrict__ x, float2* __restrict__ y, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double2 v = x[i];
    y[i] = make_float2(__double2float_rn(v.x), __double2float_rn(v.y));
  }
}

// partial[b * nv + j] = conj(V32_j) . w32 over the b-th chunk of kMD32Chunk elements, j <= st->j:
// a skinny GEMV. The CTA stages its chunk of w32 in shared memory; its warps take the basis
// vectors in turn and stream that chunk of each with 8 independent loads per lane. Products
// and sums in FP32 (a warp's sum covers one chunk), stored as FP64 for the cross-chunk sum.
__global__ void __launch_bounds__(256) k_multidot32(const float2* __restrict__ V32, int64_t ldv,
                                                    const LzState* __restrict__ st,
                                                    const float2* __restrict__ w32, int64_t n,
                                                    double2* __restrict__ partial) {
  __shared__ float2 ws[kMD32Chunk];
  const int nv = st->j + 1;
  const int64_t b0 = (int64_t)blockIdx.x * kMD32Chunk;
  const int len = n - b0 < kMD32Chunk ? (int)(n - b0) : kMD32Chunk;
  for (int t = threadIdx.x; t < kMD32Chunk; t += blockDim.x) ws[t] = t < len ? w32[b0 + t] : make_float2(0.f, 0.f);
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarp = blockDim.x >> 5;
  constexpr int kU = 8;
  for (int q = warp; q < nv; q += nwarp) {
    const float2* v = V32 + (int64_t)q * ldv + b0;
    float re = 0.f, im = 0.f;
    for (int t0 = lane; t0 < len; t0 += 32 * kU) {
      float2 x[kU];
#pragma unroll
      for (int u = 0; u < kU; ++u) {
        const int t = t0 + 32 * u;
        x[u] = t < len ? v[t] : make_float2(0.f, 0.f);
      }
#pragma unroll
      for (int u = 0; u < kU; ++u) {
        const float2 y = ws[t0 + 32 * u < kMD32Chunk ? t0 + 32 * u : 0];
        re = __fmaf_rn(x[u].x, y.x, re);
        re = __fmaf_rn(x[u].y, y.y, re);
        im = __fmaf_rn(x[u].x, y.y, im);
        im = __fmaf_rn(-x[u].y, y.x, im);
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      re += __shfl_xor_sync(0xffffffffu, re, o);
      im += __shfl_xor_sync(0xffffffffu, im, o);
    }
    if (lane == 0) partial[(int64_t)blockIdx.x * nv + q] = make_double2((double)re, (double)im);
  }
}

// w -= sum_{j <= st->j} c_j V32_j: the correction is summed in FP32 (coefficients rounded to
// FP32 once per CTA) and subtracted from the FP64 vector
__global__ void k_sub_combination32(const float2* __restrict__ V32, int64_t ldv, const LzState* __restrict__ st,
                                    const double2* __restrict__ c, double2* __restrict__ w, int64_t n) {
  constexpr int kU = 8;   // basis vectors per step of the loop: 8 independent loads in flight
  __shared__ float2 cs[MRD_LANCZOS_MAX_ITER + 1 + kU];
  const int nv = st->j + 1;
  for (int j = threadIdx.x; j < nv + kU; j += blockDim.x)
    cs[j] = j < nv ? make_float2(__double2float_rn(c[j].x), __double2float_rn(c[j].y)) : make_float2(0.f, 0.f);
  __syncthreads();
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    float ax = 0.f, ay = 0.f;
    for (int j0 = 0; j0 < nv; j0 += kU) {
      float2 v[kU];
#pragma unroll
      for (int q = 0; q < kU; ++q) v[q] = j0 + q < nv ? V32[(int64_t)(j0 + q) * ldv + i] : make_float2(0.f, 0.f);
#pragma unroll
      for (int q = 0; q < kU; ++q) {
        const float2 cj = cs[j0 + q];
        ax = __fmaf_rn(cj.x, v[q].x, ax);
        ax = __fmaf_rn(-cj.y, v[q].y, ax);
        ay = __fmaf_rn(cj.x, v[q].y, ay);
        ay = __fmaf_rn(cj.y, v[q].x, ay);
      }
    }
    double2 o = w[i];
    o.x -= (double)ax;
    o.y -= (double)ay;
    w[i] = o;
  }
}

// out = sum_j y[j] V_j with real coefficients y
__global__ void k_combination_real(const double2* __restrict__ V, int64_t ldv, int nv, const double* __restrict__ y,
                                   double2* __restrict__ out, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    double2 acc = make_double2(0.0, 0.0);
    for (int j = 0; j < nv; ++j) {
      const double2 v = V[(int64_t)j * ldv + i];
      acc.x = fma(y[j], v.x, acc.x);
      acc.y = fma(y[j], v.y, acc.y);
    }
    out[i] = acc;
  }
}

// dst = src * (1 / sqrt(norm2)), norm2 read from device memory (real part of *nrm)
// (and its FP32 copy into dst32 when given)
__global__ void k_scale_by_invnorm(const double2* __restrict__ src, double2* __restrict__ dst, int64_t n,
                                   const double2* __restrict__ nrm2, float2* __restrict__ dst32) {
  __shared__ double s_sh;   // one FP64 square root and division per CTA, not per thread
  if (threadIdx.x == 0) s_sh = nrm2->x > 0.0 ? 1.0 / sqrt(nrm2->x) : 0.0;
  __syncthreads();
  const double s = s_sh;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double2 v = src[i];
    const double2 o = make_double2(v.x * s, v.y * s);
    dst[i] = o;
    if (dst32) dst32[i] = make_float2(__double2float_rn(o.x), __double2float_rn(o.y));
  }
}

// Lanczos bookkeeping after the local and the full Gram-Schmidt pass of step j (single thread):
// alpha_j = Re(c1_j) + Re(c2_j).
// c1: coefficients of the local pass (v_{j-1}, v_j), c2: of the full pass (v_0 .. v_j)
__global__ void k_record_alpha(LzState* st, const double2* __restrict__ c1, const double2* __restrict__ c2) {
  const int j = st->j;
  st->alpha[j] = c1[j > 0 ? 1 : 0].x + c2[j].x;
}

__global__ void k_record_beta(LzState* st, const double2* __restrict__ nrm2) {
  const int j = st->j;
  st->beta[j] = sqrt(nrm2->x);
  st->beta_last = st->beta[j];
  st->inv_beta = nrm2->x > 0.0 ? 1.0 / st->beta[j] : 0.0;
}

__global__ void k_set_step(LzState* st, int j) { st->j = j; }
__global__ void k_next_step(LzState* st) { st->j += 1; }

// vin = v_j (j read from the state: one captured iteration serves every j)
__global__ void k_copy_vj(const double2* __restrict__ V, int64_t n, const LzState* __restrict__ st,
                          double2* __restrict__ vin) {
  const double2* v = V + (int64_t)st->j * n;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    vin[i] = v[i];
}

// v_{j+1} = w / |w|
__global__ void k_scale_next(const double2* __restrict__ w, double2* __restrict__ V, int64_t n,
                             const LzState* __restrict__ st, float2* __restrict__ V32) {
  const double sc = st->inv_beta;   // formed once by k_record_beta
  double2* dst = V + (int64_t)(st->j + 1) * n;
  float2* dst32 = V32 ? V32 + (int64_t)(st->j + 1) * n : nullptr;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double2 v = w[i];
    const double2 o = make_double2(v.x * sc, v.y * sc);
    dst[i] = o;
    if (dst32) dst32[i] = make_float2(__double2float_rn(o.x), __double2float_rn(o.y));
  }
}

// Number of eigenvalues of the leading k x k block of tridiag(b, a, b) below x: the sign
// changes of its leading principal minors p_i = det(T_i - x I), from the Sturm recurrence
// p_i = (a_i - x) p_{i-1} - b_{i-1}^2 p_{i-2} (b2 holds the squares). It needs no division:
// three FP64 operations per row, where the pivot-ratio form q_i = p_i / p_{i-1} divides once
// per row, and FP64 division is a long instruction sequence on a part with 2 FP64 operations
// per clock per SM. A zero minor is replaced by 2^-50 times the one before (a tiny positive
// pivot). A row then changes the minors' scale by at most ~2^50 (the guard) and otherwise by
// |a_i - x| + b_{i-1}^2, so every 8 rows both are rescaled by 2^-+500 when p_i has left
// [2^-500, 2^500], and neither leaves the FP64 range in between.
__device__ int sturm_count(const double* a, const double* b2, int k, double x) {
  double pm = 1.0, p = a[0] - x;
  if (p == 0.0) p = 0x1p-50;
  int cnt = p < 0.0;
  for (int i = 1; i < k; ++i) {
    double pn = fma(a[i] - x, p, -b2[i - 1] * pm);
    if (pn == 0.0) pn = p * 0x1p-50;
    cnt += (pn < 0.0) != (p < 0.0);
    pm = p;
    p = pn;
    if ((i & 7) == 0) {
      const double m = fabs(p);
      if (m > 0x1p500) {
        p *= 0x1p-500;
        pm *= 0x1p-500;
      } else if (m < 0x1p-500) {
        p *= 0x1p500;
        pm *= 0x1p500;
      }
    }
  }
  return cnt;
}

// Inverse iteration for the eigenvector of the k x k tridiagonal matrix (diagonal a, off-diagonal
// b) at the eigenvalue lam: (T - lam I) y = y_prev with a pivoted LU of the tridiagonal matrix,
// `passes` times from the uniform vector, normalised; the sign is fixed so that the first
// nonzero component is positive (a deterministic ground vector). One thread; the factors and y
// live in shared memory (not the thread's stack or global memory, whose latency the serial
// recurrences would pay on every access), and the k pivots are inverted once instead of
// dividing in each of the solves. T is double, or float where the Lanczos matvecs carry ~1e-5
// relative error and the vector only needs single precision.
template <class T>
__device__ void tridiag_inverse_iteration(const double* a_s, const double* b_s, int k, double lam, int passes,
                                          double* y_out) {
  __shared__ T d[MRD_LANCZOS_MAX_ITER + 1], du[MRD_LANCZOS_MAX_ITER + 1], du2[MRD_LANCZOS_MAX_ITER + 1];
  __shared__ T dl[MRD_LANCZOS_MAX_ITER + 1], y[MRD_LANCZOS_MAX_ITER + 1];
  __shared__ int piv[MRD_LANCZOS_MAX_ITER + 1];
  const T shift = (T)(lam + 1e-14 * fmax(1.0, fabs(lam)));
  const T y0 = (T)(1.0 / sqrt((double)k));
  for (int i = 0; i < k; ++i) {
    d[i] = (T)a_s[i] - shift;
    du[i] = i + 1 < k ? (T)b_s[i] : T(0);
    dl[i] = du[i];
    du2[i] = T(0);
    y[i] = y0;
  }
  for (int i = 0; i + 1 < k; ++i) {  // LU with partial pivoting (LAPACK gttrf layout)
    if (fabs(d[i]) >= fabs(dl[i])) {
      piv[i] = i;
      const T f = d[i] != T(0) ? dl[i] / d[i] : T(0);
      dl[i] = f;
      d[i + 1] -= f * du[i];
      du2[i] = T(0);
    } else {
      piv[i] = i + 1;
      const T f = d[i] / dl[i];
      d[i] = dl[i];
      dl[i] = f;
      const T t = du[i];
      du[i] = d[i + 1];
      d[i + 1] = t - f * d[i + 1];
      if (i + 2 < k) {
        du2[i] = du[i + 1];
        du[i + 1] = -f * du[i + 1];
      }
    }
  }
  piv[k - 1] = k - 1;
  // floor of a pivot: FP64 keeps the smallest normal scale; FP32 floors it at 2^-24 of the
  // matrix's largest entry (a perturbed pivot, as in LAPACK's inverse iteration), so that one
  // solve grows the vector by 2^24 at most and no square below overflows
  T tiny = (T)1e-300;
  if (sizeof(T) == 4) {
    double mx = 0.0;
    for (int i = 0; i < k; ++i) mx = fmax(mx, fmax(fabs(a_s[i] - lam), i + 1 < k ? fabs(b_s[i]) : 0.0));
    tiny = (T)fmax(mx * 0x1p-24, 1e-30);
  }
  for (int i = 0; i < k; ++i)   // pivots, inverted
    d[i] = T(1) / (fabs(d[i]) > tiny ? d[i] : (sizeof(T) == 4 && d[i] < T(0) ? -tiny : tiny));
  for (int rep = 0; rep < passes; ++rep) {
    for (int i = 0; i + 1 < k; ++i) {  // forward: L
      if (piv[i] == i) {
        y[i + 1] -= dl[i] * y[i];
      } else {
        const T t = y[i];
        y[i] = y[i + 1];
        y[i + 1] = t - dl[i] * y[i + 1];
      }
    }
    for (int i = k - 1; i >= 0; --i) {  // backward: U
      T v = y[i];
      if (i + 1 < k) v -= du[i] * y[i + 1];
      if (i + 2 < k) v -= du2[i] * y[i + 2];
      y[i] = v * d[i];
    }
    T sq = T(0);
    if (sizeof(T) == 4) {   // scale by the largest component first: the squares stay in range
      T mx = T(0);
      for (int i = 0; i < k; ++i) mx = fmax(mx, fabs(y[i]));
      mx = mx > T(0) ? T(1) / mx : T(1);
      for (int i = 0; i < k; ++i) y[i] *= mx;
    }
    for (int i = 0; i < k; ++i) sq += y[i] * y[i];
    sq = T(1) / sqrt(sq);
    for (int i = 0; i < k; ++i) y[i] *= sq;
  }
  double sg = 1.0;
  for (int i = 0; i < k; ++i)
    if (y[i] != T(0)) { sg = y[i] > T(0) ? 1.0 : -1.0; break; }
  if (sizeof(T) == 8) {
    for (int i = 0; i < k; ++i) y_out[i] = (double)y[i] * sg;
  } else {   // renormalise in FP64 so that the vector's norm is exact to FP64
    double sq = 0.0;
    for (int i = 0; i < k; ++i) sq += (double)y[i] * (double)y[i];
    sg /= sqrt(sq);
    for (int i = 0; i < k; ++i) y_out[i] = (double)y[i] * sg;
  }
}

// Lowest eigenpair of the k x k tridiagonal Lanczos matrix, k = j + 1; one warp. The Ritz value
// is FP64 (it decides convergence); the vector comes from FP64 inverse iteration, or FP32
// (vec32) when the Lanczos matvecs are reduced-precision.
__global__ void k_tridiag_lowest(LzState* st, int vec32) {
  const int k = st->j + 1;
  const int lane = threadIdx.x;
  __shared__ double a_s[MRD_LANCZOS_MAX_ITER + 1], b_s[MRD_LANCZOS_MAX_ITER + 1], b2_s[MRD_LANCZOS_MAX_ITER + 1];
  for (int i = lane; i < k; i += 32) {
    a_s[i] = st->alpha[i];
    b_s[i] = st->beta[i];
    b2_s[i] = st->beta[i] * st->beta[i];
  }
  __syncwarp();
  // the lowest eigenvalue lies between the lowest Gershgorin bound and the smallest diagonal
  // element (a Rayleigh quotient of a unit vector); every lane holds the same bracket
  double lo = 1e300, hi = 1e300;
  for (int i = lane; i < k; i += 32) {
    const double r = (i > 0 ? fabs(b_s[i - 1]) : 0.0) + (i + 1 < k ? fabs(b_s[i]) : 0.0);
    lo = fmin(lo, a_s[i] - r);
    hi = fmin(hi, a_s[i]);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    lo = fmin(lo, __shfl_xor_sync(0xffffffffu, lo, o));
    hi = fmin(hi, __shfl_xor_sync(0xffffffffu, hi, o));
  }
  const double pad = 1e-12 * fmax(fabs(lo), fabs(hi)) + 1e-300;
  lo -= pad;
  hi += pad;
  // warm start: by interlacing the lowest eigenvalue of T_k is at most that of T_{k-1}; late
  // in a run it moves little, so try [E_{k-1} - 4|E_{k-1} - E_{k-2}|, E_{k-1}], padded, and
  // keep it where Sturm counts confirm it (no eigenvalue below, at least one below the top),
  // the two counts on lanes 0 and 1; otherwise the Gershgorin bracket
  if (k >= 3) {
    const double e1 = st->ritz[k - 2], e2 = st->ritz[k - 3];
    const double tol = 1e-13 * fmax(fabs(e1), 1.0);
    const double wlo = e1 - 4.0 * fabs(e1 - e2) - tol, whi = e1 + tol;
    if (wlo > lo && whi < hi) {
      const int c = lane < 2 ? sturm_count(a_s, b2_s, k, lane == 0 ? wlo : whi) : 0;
      const int c_lo = __shfl_sync(0xffffffffu, c, 0), c_hi = __shfl_sync(0xffffffffu, c, 1);
      if (c_lo == 0 && c_hi >= 1) {
        lo = wlo;
        hi = whi;
      }
    }
  }
  // multisection to 1e-14 relative width (the Ritz value is compared to 1e-10 and refined
  // afterwards), or until a subdivision no longer shrinks the interval in FP64
  double prev_w = 0.0;
  for (int it = 0; it < 40; ++it) {
    if (!(hi - lo > 1e-14 * fmax(fabs(lo), fabs(hi))) || hi - lo == prev_w) break;
    prev_w = hi - lo;
    const double x = lo + (hi - lo) * (lane + 1) / 33.0;
    const int c = sturm_count(a_s, b2_s, k, x);
    const unsigned m = __ballot_sync(0xffffffffu, c >= 1);
    if (m == 0) {
      lo = lo + (hi - lo) * 32.0 / 33.0;
    } else {
      const int f = __ffs(m) - 1;  // first point with at least one eigenvalue below
      const double nlo = f > 0 ? lo + (hi - lo) * f / 33.0 : lo;
      hi = lo + (hi - lo) * (f + 1) / 33.0;
      lo = nlo;
    }
  }
  if (lane != 0) return;
  const double lam = 0.5 * (lo + hi);
  st->energy = lam;
  st->ritz[k - 1] = lam;
  if (vec32)
    tridiag_inverse_iteration<float>(a_s, b_s, k, lam, 3, st->y);
  else
    tridiag_inverse_iteration<double>(a_s, b_s, k, lam, 3, st->y);
}

}  // namespace

struct Lanczos {
  int64_t n = 0;
  double2* V = nullptr;        // (MRD_LANCZOS_MAX_ITER + 1) vectors of length n
  double2* w = nullptr;
  double2* vin = nullptr;      // v_j staged for the operator (fixed address: graph-capturable)
  double2* partial = nullptr;  // kRedBlocks * (MRD_LANCZOS_MAX_ITER + 1)
  double2* partial32 = nullptr;   // md32_blocks(n) * (MRD_LANCZOS_MAX_ITER + 1), FP32 full pass
  double2* c1 = nullptr;
  double2* c2 = nullptr;
  double2* scal = nullptr;
  float2* V32 = nullptr;       // FP32 copies of the basis and of w for the FP32 full pass
  float2* w32 = nullptr;
  bool fp32_full = false;      // full Gram-Schmidt pass in FP32 (reduced-precision matvecs)
  LzState* st = nullptr;
  LzState* st_host = nullptr;  // pinned
  cudaStream_t stream = nullptr;   // stream of the memory cache the buffers return to
  // captured Lanczos step: valid while the operator's key is unchanged
  cudaStream_t cap_stream = nullptr;
  cudaGraphExec_t step_exec = nullptr;
  uint64_t step_key = 0;
  int step_kernels = 0;
};

void lanczos_free(Lanczos* L) {
  if (!L) return;
  for (void* p : {(void*)L->V, (void*)L->w, (void*)L->vin, (void*)L->partial, (void*)L->c1, (void*)L->c2,
                  (void*)L->scal, (void*)L->st, (void*)L->V32, (void*)L->w32, (void*)L->partial32})
    cache_free(p, L->stream);
  if (L->st_host) cache_free_host(L->st_host);
  if (L->step_exec) cudaGraphExecDestroy(L->step_exec);
  if (L->cap_stream) cudaStreamDestroy(L->cap_stream);
  delete L;
}

cudaError_t lanczos_alloc(Lanczos** out, int64_t n, cudaStream_t stream) {
  Lanczos* L = new Lanczos();
  L->n = n;
  L->stream = stream;
  const int kv = MRD_LANCZOS_MAX_ITER + 1;
  auto dev = [&](auto** p, size_t bytes) { return cache_alloc((void**)p, bytes, stream); };
  cudaError_t e = dev(&L->V, (size_t)kv * (n > 0 ? n : 1) * 16);
  if (e == cudaSuccess) e = dev(&L->w, (size_t)(n > 0 ? n : 1) * 16);
  if (e == cudaSuccess) e = dev(&L->vin, (size_t)(n > 0 ? n : 1) * 16);
  if (e == cudaSuccess) e = dev(&L->partial, (size_t)kRedBlocks * kv * 16);
  if (e == cudaSuccess) e = dev(&L->c1, kv * 16);
  if (e == cudaSuccess) e = dev(&L->c2, kv * 16);
  if (e == cudaSuccess) e = dev(&L->scal, 4 * 16);
  if (e == cudaSuccess) e = dev(&L->st, sizeof(LzState));
  if (e == cudaSuccess) e = cache_alloc_host((void**)&L->st_host, sizeof(LzState));
  if (e != cudaSuccess) {
    lanczos_free(L);
    return e;
  }
  *out = L;
  return cudaSuccess;
}

// Selects the FP32 full Gram-Schmidt pass (for reduced-precision matvecs) or the FP64 one;
// the FP32 copies of the basis are allocated on first use.
cudaError_t lanczos_set_fp32_full(Lanczos* L, bool on) {
  if (on && !L->V32) {
    const size_t n = (size_t)(L->n > 0 ? L->n : 1);
    cudaError_t e = cache_alloc((void**)&L->V32, (size_t)(MRD_LANCZOS_MAX_ITER + 1) * n * 8, L->stream);
    if (e == cudaSuccess) e = cache_alloc((void**)&L->w32, n * 8, L->stream);
    if (e == cudaSuccess)
      e = cache_alloc((void**)&L->partial32, (size_t)md32_blocks(L->n) * (MRD_LANCZOS_MAX_ITER + 1) * 16, L->stream);
    if (e != cudaSuccess) {
      for (void** q : {(void**)&L->V32, (void**)&L->w32, (void**)&L->partial32}) {
        cache_free(*q, L->stream);
        *q = nullptr;
      }
      L->fp32_full = false;
      return e;
    }
  }
  L->fp32_full = on;
  return cudaSuccess;
}

// nv >= 0: dots of v_0 .. v_{nv-1}; nv < 0: of v_0 .. v_j (j from the device state)
static cudaError_t dots(Lanczos* L, const double2* V, int nv, const double2* w, double2* out, cudaStream_t s) {
  k_multidot<<<kRedBlocks, kRedThreads, 0, s>>>(V, L->n, nv, L->st, w, L->n, L->partial);
  mrd::count_launch();
  const int nmax = nv >= 0 ? nv : MRD_LANCZOS_MAX_ITER + 1;
  k_finish_dots<<<(nmax + 3) / 4, 128, 0, s>>>(L->partial, kRedBlocks, nv, L->st, out);
  mrd::count_launch();
  return cudaGetLastError();
}

// Grid of the elementwise kernels (256 threads): one element per thread up to ~1M elements,
// so that every thread's loads are issued at once instead of one grid-stride step at a time.
static unsigned grid_for(int64_t n) {
  int64_t g = (n + 255) / 256;
  return (unsigned)(g < 4096 ? (g > 0 ? g : 1) : 4096);
}

// One Lanczos step j (j in the device state) on the context stream, ending with the copy of
// the state to pinned host memory; no host synchronisation, so it can be captured.
static int lanczos_step(Lanczos* L, mrd_ctx* ctx, int (*apply)(void*, const double2*, double2*), void* op) {
  cudaStream_t s = ctx->stream;
  const int64_t n = L->n;
  k_copy_vj<<<grid_for(n), 256, 0, s>>>(L->V, n, L->st, L->vin);
  mrd::count_launch();
  int rc = apply(op, L->vin, L->w);
  if (rc != MRD_OK) return rc;
  s = ctx->stream;
  // local pass against v_{j-1}, v_j (the three-term recurrence), then one full classical
  // Gram-Schmidt pass against v_0 .. v_j that removes what rounding left
  MRD_CUDA(ctx, dots(L, L->V, -2, L->w, L->c1, s));
  k_sub_combination<<<grid_for(n), 256, 0, s>>>(L->V, n, -2, L->st, L->c1, L->w, n);
  mrd::count_launch();
  if (L->fp32_full) {
    k_to_f32<<<grid_for(n), 256, 0, s>>>(L->w, L->w32, n);
    k_multidot32<<<(unsigned)md32_blocks(n), 256, 0, s>>>(L->V32, n, L->st, L->w32, n, L->partial32);
    k_finish_dots<<<(MRD_LANCZOS_MAX_ITER + 1 + 3) / 4, 128, 0, s>>>(L->partial32, (int)md32_blocks(n), -1, L->st,
                                                                      L->c2);
    k_sub_combination32<<<grid_for(n), 256, 0, s>>>(L->V32, n, L->st, L->c2, L->w, n);
    mrd::count_launches(4);
  } else {
    MRD_CUDA(ctx, dots(L, L->V, -1, L->w, L->c2, s));
    k_sub_combination<<<grid_for(n), 256, 0, s>>>(L->V, n, -1, L->st, L->c2, L->w, n);
    mrd::count_launch();
  }
  k_record_alpha<<<1, 1, 0, s>>>(L->st, L->c1, L->c2);
  mrd::count_launch();
  MRD_CUDA(ctx, dots(L, L->w, 1, L->w, L->scal, s));
  k_record_beta<<<1, 1, 0, s>>>(L->st, L->scal);
  mrd::count_launch();
  k_tridiag_lowest<<<1, 32, 0, s>>>(L->st, L->fp32_full ? 1 : 0);
  mrd::count_launch();
  k_scale_next<<<grid_for(n), 256, 0, s>>>(L->w, L->V, n, L->st, L->fp32_full ? L->V32 : nullptr);
  mrd::count_launch();
  k_next_step<<<1, 1, 0, s>>>(L->st);
  mrd::count_launch();
  MRD_CUDA(ctx, cudaGetLastError());
  MRD_CUDA(ctx, cudaMemcpyAsync(L->st_host, L->st, sizeof(LzState), cudaMemcpyDeviceToHost, s));
  return MRD_OK;
}

// Capture one step as a CUDA graph on a private stream (the context stream may be the legacy
// default stream, which cannot be captured). Returns false (and leaves no graph) if the
// operator could not be captured; the caller then launches the steps directly.
static bool capture_step(Lanczos* L, mrd_ctx* ctx, int (*apply)(void*, const double2*, double2*), void* op,
                         uint64_t key) {
  if (L->step_exec) {
    cudaGraphExecDestroy(L->step_exec);
    L->step_exec = nullptr;
  }
  if (!L->cap_stream && cudaStreamCreateWithFlags(&L->cap_stream, cudaStreamNonBlocking) != cudaSuccess) {
    cudaGetLastError();
    L->cap_stream = nullptr;
    return false;
  }
  cudaStream_t saved = ctx->stream;
  const int64_t c0 = mrd::launch_count_total();
  if (cudaStreamBeginCapture(L->cap_stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  ctx->stream = L->cap_stream;
  const std::string err_saved = ctx->err;
  const int rc = lanczos_step(L, ctx, apply, op);
  ctx->stream = saved;
  cudaGraph_t g = nullptr;
  const cudaError_t e = cudaStreamEndCapture(L->cap_stream, &g);
  const int64_t kernels = mrd::launch_count_total() - c0;
  mrd::uncount_launches(kernels);          // counted again at every replay
  if (rc != MRD_OK || e != cudaSuccess || !g) {
    if (g) cudaGraphDestroy(g);
    cudaGetLastError();
    ctx->err = err_saved;
    return false;
  }
  const cudaError_t ei = cudaGraphInstantiate(&L->step_exec, g, 0);
  cudaGraphDestroy(g);
  if (ei != cudaSuccess) {
    cudaGetLastError();
    L->step_exec = nullptr;
    return false;
  }
  L->step_key = key;
  L->step_kernels = (int)kernels;
  return true;
}

// Runs Lanczos on the operator `apply` (theta_out = H theta_in on stream s). theta: start
// vector in, ground vector out. Host reads one small state record per iteration. With
// graph_key != 0 the step is captured once as a CUDA graph (kept while the key is unchanged)
// and replayed; the operator must then be ready (buffers built, operands packed) and free of
// host synchronisation. `replayed(op)`, if given, runs after every replay of the graph.
int lanczos_run(Lanczos* L, mrd_ctx* ctx, int (*apply)(void*, const double2*, double2*), void* op, double2* theta,
                int max_iter, double tol, double* energy, int* iters, double* beta_last, uint64_t graph_key,
                int (*replayed)(void*)) {
  cudaStream_t s = ctx->stream;
  const int64_t n = L->n;
  if (max_iter < 1 || max_iter > MRD_LANCZOS_MAX_ITER)
    return mrd_fail(ctx, MRD_E_ARG, "mrd_lanczos: max_iter out of range");
  // v_0 = theta / |theta|
  MRD_CUDA(ctx, dots(L, theta, 1, theta, L->scal, s));
  k_scale_by_invnorm<<<grid_for(n), 256, 0, s>>>(theta, L->V, n, L->scal, L->fp32_full ? L->V32 : nullptr);
  mrd::count_launch();
  k_set_step<<<1, 1, 0, s>>>(L->st, 0);
  mrd::count_launch();
  MRD_CUDA(ctx, cudaGetLastError());
  bool graph = graph_key != 0 && (L->step_exec && L->step_key == graph_key);
  if (graph_key != 0 && !graph) graph = capture_step(L, ctx, apply, op, graph_key);
  double e_prev = 0.0;
  int k = 0;
  for (int j = 0; j < max_iter; ++j) {
    if (graph) {
      MRD_CUDA(ctx, cudaGraphLaunch(L->step_exec, s));
      mrd::count_launches(L->step_kernels);
    } else {
      int rc = lanczos_step(L, ctx, apply, op);
      if (rc != MRD_OK) return rc;
    }
    MRD_CUDA(ctx, cudaStreamSynchronize(s));
    if (graph && replayed) {
      const int rc = replayed(op);
      if (rc != MRD_OK) return rc;
    }
    k = j + 1;
    const double e = L->st_host->energy;
    const double b = L->st_host->beta_last;
    if (!std::isfinite(e) || !std::isfinite(b)) return mrd_fail(ctx, MRD_E_NAN, "mrd_lanczos: non-finite value");
    const double scale = std::fabs(L->st_host->alpha[j]) + std::fabs(e) + 1e-300;
    if (j > 0 && std::fabs(e - e_prev) < tol * std::fabs(e)) break;
    if (b < 1e-13 * scale) break;
    e_prev = e;
  }
  // ground vector = V y, normalised
  k_combination_real<<<grid_for(n), 256, 0, s>>>(L->V, n, k, L->st->y, L->w, n);
  mrd::count_launch();
  MRD_CUDA(ctx, dots(L, L->w, 1, L->w, L->scal, s));
  k_scale_by_invnorm<<<grid_for(n), 256, 0, s>>>(L->w, theta, n, L->scal, nullptr);
  mrd::count_launch();
  MRD_CUDA(ctx, cudaGetLastError());
  MRD_CUDA(ctx, cudaStreamSynchronize(s));
  *energy = L->st_host->energy;
  *iters = k;
  if (beta_last) *beta_last = L->st_host->beta_last;
  return MRD_OK;
}

double2* lanczos_work(Lanczos* L) { return L->w; }

// <u, v> on the device into host (re, im); used by refinement and tests.
int vdot(Lanczos* L, mrd_ctx* ctx, const double2* u, const double2* v, double* re, double* im) {
  cudaStream_t s = ctx->stream;
  MRD_CUDA(ctx, dots(L, u, 1, v, L->scal, s));
  double2 h;
  MRD_CUDA(ctx, cudaMemcpyAsync(&h, L->scal, 16, cudaMemcpyDeviceToHost, s));
  MRD_CUDA(ctx, cudaStreamSynchronize(s));
  *re = h.x;
  *im = h.y;
  return MRD_OK;
}

}  // namespace mrd
