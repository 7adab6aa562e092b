// Lanczos ground-state solver for the two-site H_eff (standard DMRG eigensolver; the paper
// relies on DMRG as in its refs. W92, S2005, S2011 without restating it).
//
// Krylov recursion with full reorthogonalisation: for j = 0, 1, ...
//   w = H v_j;  two classical Gram-Schmidt passes c = V^+ w, w -= V c  (V = [v_0 .. v_j]);
//   alpha_j = Re(c_j) summed over both passes;  beta_j = |w|;  v_{j+1} = w / beta_j;
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

// partial[b * nv + j] = sum over this CTA's share of conj(V_j) . w, j < nv (re, im interleaved)
__global__ void __launch_bounds__(kRedThreads) k_multidot(const double2* __restrict__ V, int64_t ldv, int nv,
                                                          const double2* __restrict__ w, int64_t n,
                                                          double2* __restrict__ partial) {
  __shared__ double sre[kRedThreads / 32], sim[kRedThreads / 32];
  const int64_t chunk = (n + gridDim.x - 1) / gridDim.x;
  const int64_t b = blockIdx.x * chunk;
  const int64_t e = b + chunk < n ? b + chunk : n;
  for (int j = 0; j < nv; ++j) {
    const double2* v = V + (int64_t)j * ldv;
    double re = 0.0, im = 0.0;
    for (int64_t i = b + threadIdx.x; i < e; i += blockDim.x) {
      const double2 x = v[i], y = w[i];
      re = fma(x.x, y.x, re);
      re = fma(x.y, y.y, re);
      im = fma(x.x, y.y, im);
      im = fma(-x.y, y.x, im);
    }
    re = warp_sum(re);
    im = warp_sum(im);
    if ((threadIdx.x & 31) == 0) {
      sre[threadIdx.x >> 5] = re;
      sim[threadIdx.x >> 5] = im;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      double a = 0.0, c = 0.0;
      for (int k = 0; k < kRedThreads / 32; ++k) {
        a += sre[k];
        c += sim[k];
      }
      partial[(int64_t)blockIdx.x * nv + j] = make_double2(a, c);
    }
    __syncthreads();
  }
}

// out[j] = sum_b partial[b * nv + j]; one thread per j, fixed order.
__global__ void k_finish_dots(const double2* __restrict__ partial, int nblocks, int nv, double2* __restrict__ out) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= nv) return;
  double a = 0.0, c = 0.0;
  for (int b = 0; b < nblocks; ++b) {
    const double2 p = partial[(int64_t)b * nv + j];
    a += p.x;
    c += p.y;
  }
  out[j] = make_double2(a, c);
}

// w -= sum_j c[j] V_j
__global__ void k_sub_combination(const double2* __restrict__ V, int64_t ldv, int nv, const double2* __restrict__ c,
                                  double2* __restrict__ w, int64_t n) {
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
__global__ void k_scale_by_invnorm(const double2* __restrict__ src, double2* __restrict__ dst, int64_t n,
                                   const double2* __restrict__ nrm2) {
  const double s = nrm2->x > 0.0 ? 1.0 / sqrt(nrm2->x) : 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double2 v = src[i];
    dst[i] = make_double2(v.x * s, v.y * s);
  }
}

// Lanczos bookkeeping after the two Gram-Schmidt passes of step j (single thread):
// alpha_j += Re(c1_j) + Re(c2_j) is accumulated in state.
struct LzState {
  double alpha[MRD_LANCZOS_MAX_ITER + 1];
  double beta[MRD_LANCZOS_MAX_ITER + 1];
  double y[MRD_LANCZOS_MAX_ITER + 1];
  double energy;
  double beta_last;
  int flags;
};

__global__ void k_record_alpha(LzState* st, int j, const double2* __restrict__ c1, const double2* __restrict__ c2) {
  st->alpha[j] = c1[j].x + c2[j].x;
}

__global__ void k_record_beta(LzState* st, int j, const double2* __restrict__ nrm2) {
  st->beta[j] = sqrt(nrm2->x);
  st->beta_last = st->beta[j];
}

__device__ int sturm_count(const double* a, const double* b, int k, double x) {
  // number of eigenvalues of tridiag(b, a, b) smaller than x
  int cnt = 0;
  double q = a[0] - x;
  if (q < 0) ++cnt;
  for (int i = 1; i < k; ++i) {
    double qq = q != 0.0 ? q : 1e-300;
    q = (a[i] - x) - b[i - 1] * b[i - 1] / qq;
    if (q < 0) ++cnt;
  }
  return cnt;
}

// Lowest eigenpair of the k x k tridiagonal Lanczos matrix; one warp.
__global__ void k_tridiag_lowest(LzState* st, int k) {
  const double* a = st->alpha;
  const double* b = st->beta;
  const int lane = threadIdx.x;
  __shared__ double lo_s, hi_s;
  if (lane == 0) {
    double lo = 1e300, hi = -1e300;
    for (int i = 0; i < k; ++i) {
      double r = (i > 0 ? fabs(b[i - 1]) : 0.0) + (i + 1 < k ? fabs(b[i]) : 0.0);
      lo = fmin(lo, a[i] - r);
      hi = fmax(hi, a[i] + r);
    }
    double pad = 1e-12 * fmax(fabs(lo), fabs(hi)) + 1e-300;
    lo_s = lo - pad;
    hi_s = hi + pad;
  }
  __syncwarp();
  for (int it = 0; it < 40; ++it) {
    const double lo = lo_s, hi = hi_s;
    if (!(hi - lo > 4e-16 * fmax(fabs(lo), fabs(hi)))) break;
    const double x = lo + (hi - lo) * (lane + 1) / 33.0;
    const int c = sturm_count(a, b, k, x);
    const unsigned m = __ballot_sync(0xffffffffu, c >= 1);
    __syncwarp();
    if (lane == 0) {
      if (m == 0) {
        lo_s = lo + (hi - lo) * 32.0 / 33.0;
      } else {
        const int f = __ffs(m) - 1;  // first point with at least one eigenvalue below
        hi_s = lo + (hi - lo) * (f + 1) / 33.0;
        lo_s = f > 0 ? lo + (hi - lo) * f / 33.0 : lo;
      }
    }
    __syncwarp();
  }
  if (lane != 0) return;
  const double lam = 0.5 * (lo_s + hi_s);
  st->energy = lam;
  // inverse iteration: (T - lam I) y = y_prev with a pivoted LU of the tridiagonal matrix
  double d[MRD_LANCZOS_MAX_ITER + 1], du[MRD_LANCZOS_MAX_ITER + 1], du2[MRD_LANCZOS_MAX_ITER + 1];
  double dl[MRD_LANCZOS_MAX_ITER + 1];
  int piv[MRD_LANCZOS_MAX_ITER + 1];
  double* y = st->y;
  const double shift = lam + 1e-14 * fmax(1.0, fabs(lam));
  for (int i = 0; i < k; ++i) {
    d[i] = a[i] - shift;
    du[i] = i + 1 < k ? b[i] : 0.0;
    dl[i] = i + 1 < k ? b[i] : 0.0;
    du2[i] = 0.0;
    y[i] = 1.0 / sqrt((double)k);
  }
  for (int i = 0; i + 1 < k; ++i) {  // LU with partial pivoting (LAPACK gttrf layout)
    if (fabs(d[i]) >= fabs(dl[i])) {
      piv[i] = i;
      const double f = d[i] != 0.0 ? dl[i] / d[i] : 0.0;
      dl[i] = f;
      d[i + 1] -= f * du[i];
      du2[i] = 0.0;
    } else {
      piv[i] = i + 1;
      const double f = d[i] / dl[i];
      d[i] = dl[i];
      dl[i] = f;
      const double t = du[i];
      du[i] = d[i + 1];
      d[i + 1] = t - f * d[i + 1];
      if (i + 2 < k) {
        du2[i] = du[i + 1];
        du[i + 1] = -f * du[i + 1];
      }
    }
  }
  piv[k - 1] = k - 1;
  const double tiny = 1e-300;
  for (int rep = 0; rep < 3; ++rep) {
    for (int i = 0; i + 1 < k; ++i) {  // forward: L
      if (piv[i] == i) {
        y[i + 1] -= dl[i] * y[i];
      } else {
        const double t = y[i];
        y[i] = y[i + 1];
        y[i + 1] = t - dl[i] * y[i + 1];
      }
    }
    for (int i = k - 1; i >= 0; --i) {  // backward: U
      double v = y[i];
      if (i + 1 < k) v -= du[i] * y[i + 1];
      if (i + 2 < k) v -= du2[i] * y[i + 2];
      y[i] = v / (fabs(d[i]) > tiny ? d[i] : tiny);
    }
    double s = 0.0;
    for (int i = 0; i < k; ++i) s += y[i] * y[i];
    s = 1.0 / sqrt(s);
    for (int i = 0; i < k; ++i) y[i] *= s;
  }
  // fix the sign: first nonzero component positive (deterministic ground vector)
  double sg = 1.0;
  for (int i = 0; i < k; ++i)
    if (y[i] != 0.0) { sg = y[i] > 0 ? 1.0 : -1.0; break; }
  for (int i = 0; i < k; ++i) y[i] *= sg;
}

}  // namespace

struct Lanczos {
  int64_t n = 0;
  double2* V = nullptr;        // (MRD_LANCZOS_MAX_ITER + 1) vectors of length n
  double2* w = nullptr;
  double2* partial = nullptr;  // kRedBlocks * (MRD_LANCZOS_MAX_ITER + 1)
  double2* c1 = nullptr;
  double2* c2 = nullptr;
  double2* scal = nullptr;
  LzState* st = nullptr;
  LzState* st_host = nullptr;  // pinned
};

void lanczos_free(Lanczos* L) {
  if (!L) return;
  cudaFree(L->V); cudaFree(L->w); cudaFree(L->partial); cudaFree(L->c1); cudaFree(L->c2); cudaFree(L->scal);
  cudaFree(L->st);
  if (L->st_host) cudaFreeHost(L->st_host);
  delete L;
}

cudaError_t lanczos_alloc(Lanczos** out, int64_t n) {
  Lanczos* L = new Lanczos();
  L->n = n;
  const int kv = MRD_LANCZOS_MAX_ITER + 1;
  cudaError_t e = cudaMalloc(&L->V, (size_t)kv * (n > 0 ? n : 1) * 16);
  if (e == cudaSuccess) e = cudaMalloc(&L->w, (size_t)(n > 0 ? n : 1) * 16);
  if (e == cudaSuccess) e = cudaMalloc(&L->partial, (size_t)kRedBlocks * kv * 16);
  if (e == cudaSuccess) e = cudaMalloc(&L->c1, kv * 16);
  if (e == cudaSuccess) e = cudaMalloc(&L->c2, kv * 16);
  if (e == cudaSuccess) e = cudaMalloc(&L->scal, 4 * 16);
  if (e == cudaSuccess) e = cudaMalloc(&L->st, sizeof(LzState));
  if (e == cudaSuccess) e = cudaMallocHost(&L->st_host, sizeof(LzState));
  if (e != cudaSuccess) {
    lanczos_free(L);
    return e;
  }
  *out = L;
  return cudaSuccess;
}

static cudaError_t dots(Lanczos* L, const double2* V, int nv, const double2* w, double2* out, cudaStream_t s) {
  k_multidot<<<kRedBlocks, kRedThreads, 0, s>>>(V, L->n, nv, w, L->n, L->partial);
  mrd::count_launch();
  k_finish_dots<<<(nv + 63) / 64, 64, 0, s>>>(L->partial, kRedBlocks, nv, out);
  mrd::count_launch();
  return cudaGetLastError();
}

static unsigned grid_for(int64_t n) {
  int64_t g = (n + 255) / 256;
  return (unsigned)(g < 1216 ? (g > 0 ? g : 1) : 1216);
}

// Runs Lanczos on the operator `apply` (theta_out = H theta_in on stream s). theta: start
// vector in, ground vector out. Host reads one small state record per iteration.
int lanczos_run(Lanczos* L, mrd_ctx* ctx, int (*apply)(void*, const double2*, double2*), void* op, double2* theta,
                int max_iter, double tol, double* energy, int* iters, double* beta_last) {
  cudaStream_t s = ctx->stream;
  const int64_t n = L->n;
  if (max_iter < 1 || max_iter > MRD_LANCZOS_MAX_ITER)
    return mrd_fail(ctx, MRD_E_ARG, "mrd_lanczos: max_iter out of range");
  // v_0 = theta / |theta|
  MRD_CUDA(ctx, dots(L, theta, 1, theta, L->scal, s));
  k_scale_by_invnorm<<<grid_for(n), 256, 0, s>>>(theta, L->V, n, L->scal);
  mrd::count_launch();
  MRD_CUDA(ctx, cudaGetLastError());
  double e_prev = 0.0;
  int k = 0;
  for (int j = 0; j < max_iter; ++j) {
    double2* vj = L->V + (int64_t)j * n;
    int rc = apply(op, vj, L->w);
    if (rc != MRD_OK) return rc;
    MRD_CUDA(ctx, dots(L, L->V, j + 1, L->w, L->c1, s));
    k_sub_combination<<<grid_for(n), 256, 0, s>>>(L->V, n, j + 1, L->c1, L->w, n);
    mrd::count_launch();
    MRD_CUDA(ctx, dots(L, L->V, j + 1, L->w, L->c2, s));
    k_sub_combination<<<grid_for(n), 256, 0, s>>>(L->V, n, j + 1, L->c2, L->w, n);
    mrd::count_launch();
    k_record_alpha<<<1, 1, 0, s>>>(L->st, j, L->c1, L->c2);
    mrd::count_launch();
    MRD_CUDA(ctx, dots(L, L->w, 1, L->w, L->scal, s));
    k_record_beta<<<1, 1, 0, s>>>(L->st, j, L->scal);
    mrd::count_launch();
    k_tridiag_lowest<<<1, 32, 0, s>>>(L->st, j + 1);
    mrd::count_launch();
    if (j + 1 < max_iter) {
      k_scale_by_invnorm<<<grid_for(n), 256, 0, s>>>(L->w, L->V + (int64_t)(j + 1) * n, n, L->scal);
      mrd::count_launch();
    }
    MRD_CUDA(ctx, cudaGetLastError());
    MRD_CUDA(ctx, cudaMemcpyAsync(L->st_host, L->st, sizeof(LzState), cudaMemcpyDeviceToHost, s));
    MRD_CUDA(ctx, cudaStreamSynchronize(s));
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
  k_scale_by_invnorm<<<grid_for(n), 256, 0, s>>>(L->w, theta, n, L->scal);
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
