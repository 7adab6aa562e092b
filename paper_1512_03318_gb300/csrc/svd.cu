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
// ~1e-5), their accumulated rotation is applied to the FP64 X by one GEMM, and FP64 sweeps
// finish. All blocks advance together in a block-cyclic order: the columns are grouped, one
// launch per round of the round-robin schedule on the groups, one CTA per group pair with its
// columns staged in shared memory, one warp per column pair.
//
// Truncation keeps the globally largest chi singular values above cutoff * s_max, ties
// broken by (value desc, block asc, index asc); the kept values are renormalised to
// sum s^2 = 1 and the discarded weight is reported.
#include <cmath>

#include "ff.cuh"
#include "mrd_internal.h"

namespace mrd {

// Per-block descriptor (int64): m n p r x_off v_off out_u_off out_vh_off s_off wide
// + field 10: X32 offset, 11: V32 offset (float2 units), 12: value slots of the block (r before
// columns were set aside after the FP32 pre-sweeps; the slots past r hold zeros)
enum { SVF = 13 };
constexpr int kSvdMaxSmem = 220 * 1024;

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

// Asynchronous copy global -> shared of one 8- or 16-byte element (the columns of a round are
// staged with these, all in flight at once, then awaited together).
template <class S2>
__device__ __forceinline__ void stage_elem(S2* dst, const S2* src) {
  static_assert(sizeof(S2) == 8 || sizeof(S2) == 16, "8- or 16-byte elements");
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  if constexpr (sizeof(S2) == 16)
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(d), "l"(src) : "memory");
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void stage_wait() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// Rotate the column pair (x_i, x_j) (and the matching columns of V, when given) so that they
// become orthogonal; one warp, columns of length p (V: r). Returns whether it rotated.
// A column whose norm is negligible against the block (|x|^2 <= floor2 = zero_rel |M|_F^2)
// is a numerical zero (rank deficiency): it is neither rotated nor counted as unconverged.
// REAL: the columns are real (imaginary parts zero, the real-arithmetic mode): only the real
// parts enter the dot products and the rotation, whose phase is a sign.
template <class T, class T2, bool REAL>
__device__ __forceinline__ bool jacobi_pair(T2* xi, T2* xj, int p, T2* vi, T2* vj, int r, T tol, double floor2,
                                            int lane) {
  T a = 0, bb = 0, gr = 0, gi = 0;
  for (int t = lane; t < p; t += 32) {
    const T2 u = xi[t], v = xj[t];
    if (REAL) {
      a = fma(u.x, u.x, a);
      bb = fma(v.x, v.x, bb);
      gr = fma(u.x, v.x, gr);
    } else {
      a = fma(u.x, u.x, fma(u.y, u.y, a));
      bb = fma(v.x, v.x, fma(v.y, v.y, bb));
      gr = fma(u.x, v.x, fma(u.y, v.y, gr));     // Re(conj(u) v)
      gi = fma(u.x, v.y, fma(-u.y, v.x, gi));    // Im(conj(u) v)
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_xor_sync(0xffffffffu, a, o);
    bb += __shfl_xor_sync(0xffffffffu, bb, o);
    gr += __shfl_xor_sync(0xffffffffu, gr, o);
    if (!REAL) gi += __shfl_xor_sync(0xffffffffu, gi, o);
  }
  const T g = REAL ? fabs(gr) : sqrt(gr * gr + gi * gi);
  if ((double)a <= floor2 || (double)bb <= floor2) return false;
  if (!(g > tol * sqrt(a * bb))) return false;
  // phase-free real rotation on (x_i, e^{-i phi} x_j), phi = arg(gamma)
  T ph_r, ph_i, c, sn;
  if constexpr (sizeof(T) == 4) {   // FP32 pre-sweeps: fast reciprocal and rsqrt (a few ulp)
    const float ig = 1.f / g;
    ph_r = gr * ig;
    ph_i = -gi * ig;
    const float zeta = 0.5f * (bb - a) * ig, q = 1.f + zeta * zeta;
    // very different norms: t = 1 / (2 zeta), as zeta^2 would overflow
    const float t = fabsf(zeta) > 1e4f ? __fdividef(0.5f, zeta)
                                       : __fdividef(zeta >= 0.f ? 1.f : -1.f, fabsf(zeta) + q * rsqrtf(q));
    c = rsqrtf(1.f + t * t);
    sn = c * t;
  } else {
    ph_r = gr / g;
    ph_i = -gi / g;                               // e^{-i phi}
    const T zeta = (bb - a) / (T(2) * g);
    const T t = (zeta >= T(0) ? T(1) : T(-1)) / (fabs(zeta) + sqrt(T(1) + zeta * zeta));
    c = T(1) / sqrt(T(1) + t * t);
    sn = c * t;
  }
  auto rot = [&](T2* ci, T2* cj, int n) {
    for (int k = lane; k < n; k += 32) {
      const T2 u = ci[k], v0 = cj[k];
      T2 o1, o2;
      if (REAL) {
        const T vx = v0.x * ph_r;
        o1.x = c * u.x - sn * vx; o1.y = T(0);
        o2.x = sn * u.x + c * vx; o2.y = T(0);
      } else {
        T2 v;
        v.x = v0.x * ph_r - v0.y * ph_i;
        v.y = v0.x * ph_i + v0.y * ph_r;
        o1.x = c * u.x - sn * v.x; o1.y = c * u.y - sn * v.y;
        o2.x = sn * u.x + c * v.x; o2.y = sn * u.y + c * v.y;
      }
      ci[k] = o1;
      cj[k] = o2;
    }
  };
  rot(xi, xj, p);
  if (vi != nullptr) rot(vi, vj, r);
  return true;
}

// Float-float version of jacobi_pair: columns of complex float-float values (float4 =
// re.hi, im.hi, re.lo, im.lo) on the FP32 pipes. Dot products are accumulated and reduced
// in float-float (~48 bits, so the orthogonality test resolves 5e-13); the rotation
// coefficients are FP32 numbers derived from them (bb - a formed in float-float), and the
// rotation with these coefficients is applied exactly in float-float. An FP32 coefficient
// makes the rotation unitary only to ~1e-7: the pair is left orthogonal to ~1e-7 of its
// previous overlap (the next sweep removes the rest) and the column norms drift by ~1e-7,
// which the caller absorbs because it takes the singular vectors of one side from the
// orthogonalised columns and the other factor by projection.
template <bool REAL>
__device__ __forceinline__ bool jacobi_pair_ff(float4* xi, float4* xj, int p, float tol, float floor2, FF& na, FF& nb,
                                               int lane) {
  FFAcc GR = {0.f, 0.f}, GI = {0.f, 0.f};
  for (int t = lane; t < p; t += 32) {
    const float4 u4 = xi[t], v4 = xj[t];
    const FF ur = {u4.x, u4.z}, ui = {u4.y, u4.w}, vr = {v4.x, v4.z}, vi = {v4.y, v4.w};
    ff_mac(GR, ur, vr);                        // Re(conj(u) v)
    if (!REAL) {
      ff_mac(GR, ui, vi);
      ff_mac(GI, ur, vi);                      // Im(conj(u) v)
      ff_mac(GI, ff_neg(ui), vr);
    }
  }
  const FF gr2 = ff_warp_sum(ff_norm(GR)), gi2 = REAL ? FF{0.f, 0.f} : ff_warp_sum(ff_norm(GI));
  const float a = na.hi, bb = nb.hi, gr = gr2.hi, gi = gi2.hi;
  const float g = hypotf(gr, gi);               // no intermediate underflow
  if (a <= floor2 || bb <= floor2) return false;
  if (!(g > tol * (sqrtf(a) * sqrtf(bb)))) return false;
  const FF dba = ff_add(nb, ff_neg(na));
  // The coefficients only need to be good FP32 numbers (the rotation is applied exactly with
  // whatever c, s it gets), so they use the fast reciprocal and reciprocal square root: a few
  // ulp, the same order as the FP32 rounding of the exact formulas, on the latency chain of
  // every pair step.
  const float ig = 1.f / g;                      // g > 0 here
  const float ph_r = gr * ig, ph_i = -gi * ig;   // e^{-i phi}
  // columns of very different norms give |zeta| up to ~1e26: take t = 1 / (2 zeta) there
  // (relative error 1 / (4 zeta^2)) instead of squaring zeta
  const float zeta = 0.5f * dba.hi * ig;
  const float q = 1.f + zeta * zeta;
  const float t = fabsf(zeta) > 1e4f ? __fdividef(0.5f, zeta)
                                     : __fdividef(zeta >= 0.f ? 1.f : -1.f, fabsf(zeta) + q * rsqrtf(q));
  if (!(fabsf(t) > 0.f) || !isfinite(t)) return false;   // no representable rotation
  const float c = rsqrtf(1.f + t * t), sn = c * t;
  // x_i' = c u - sigma v, x_j' = s u + kappa v with sigma = s e^{-i phi}, kappa = c e^{-i phi}
  const float sr = sn * ph_r, si = sn * ph_i, kr = c * ph_r, ki = c * ph_i;
  for (int k = lane; k < p; k += 32) {
    const float4 u4 = xi[k], v4 = xj[k];
    const FF ur = {u4.x, u4.z}, ui = {u4.y, u4.w}, vr = {v4.x, v4.z}, vi = {v4.y, v4.w};
    if (REAL) {   // si = ki = 0: x_i' = c u - s_r v, x_j' = s u + k_r v, imaginary parts stay 0
      FFAcc o1r = ff_prod1(ur, c), o2r = ff_prod1(ur, sn);
      ff_mac1(o1r, vr, -sr);
      ff_mac1(o2r, vr, kr);
      const FF a1 = ff_norm(o1r), a3 = ff_norm(o2r);
      xi[k] = make_float4(a1.hi, 0.f, a1.lo, 0.f);
      xj[k] = make_float4(a3.hi, 0.f, a3.lo, 0.f);
      continue;
    }
    FFAcc o1r = ff_prod1(ur, c), o1i = ff_prod1(ui, c), o2r = ff_prod1(ur, sn), o2i = ff_prod1(ui, sn);
    ff_mac1(o1r, vr, -sr); ff_mac1(o1r, vi, si);    // c u_r - (s_r v_r - s_i v_i)
    ff_mac1(o1i, vi, -sr); ff_mac1(o1i, vr, -si);   // c u_i - (s_r v_i + s_i v_r)
    ff_mac1(o2r, vr, kr); ff_mac1(o2r, vi, -ki);    // s u_r + k_r v_r - k_i v_i
    ff_mac1(o2i, vi, kr); ff_mac1(o2i, vr, ki);     // s u_i + k_r v_i + k_i v_r
    const FF a1 = ff_norm(o1r), b1 = ff_norm(o1i), a3 = ff_norm(o2r), b3 = ff_norm(o2i);
    xi[k] = make_float4(a1.hi, b1.hi, a1.lo, b1.lo);
    xj[k] = make_float4(a3.hi, b3.hi, a3.lo, b3.lo);
  }
  // Norms of the rotated columns from the pair's own values, with the coefficients that were
  // applied (exact FP32 numbers, whether or not they form an exactly unitary rotation), g =
  // conj(u) . v:
  //   |c u - sigma v|^2 = c^2 a + |sigma|^2 b - 2 c Re(sigma g),
  //   |s u + kappa v|^2 = s^2 a + |kappa|^2 b + 2 s Re(kappa g).
  // The identities hold for any c, sigma, kappa; in float-float they give the norms to ~1e-14
  // (as summing the rotated elements would), for ~20 operations per pair instead of 4
  // multiply-adds per element and two warp reductions.
  {
    const FF a = na, b = nb;
    FFAcc A = {0.f, 0.f}, B = {0.f, 0.f};
    const FF sig2 = ff_add(ff_two_prod(sr, sr), ff_two_prod(si, si));
    const FF kap2 = ff_add(ff_two_prod(kr, kr), ff_two_prod(ki, ki));
    ff_mac(A, ff_two_prod(c, c), a);
    ff_mac(A, sig2, b);
    ff_mac(A, ff_two_prod(-2.f * c, sr), gr2);         // -2 c (s_r g_r - s_i g_i)
    ff_mac(A, ff_two_prod(2.f * c, si), gi2);
    ff_mac(B, ff_two_prod(sn, sn), a);
    ff_mac(B, kap2, b);
    ff_mac(B, ff_two_prod(2.f * sn, kr), gr2);         // 2 s (k_r g_r - k_i g_i)
    ff_mac(B, ff_two_prod(-2.f * sn, ki), gi2);
    na = ff_norm(A);
    nb = ff_norm(B);
  }
  return true;
}

// Power of two (exact scaling) that brings a block of squared Frobenius norm fro2 to unit
// norm, away from the FP32 underflow range, while its columns are held in float-float.
__device__ __forceinline__ double ff_scale(double fro2) {
  return fro2 > 0.0 ? ldexp(1.0, -ilogb(sqrt(fro2))) : 1.0;
}

// X (FP64, field 4) <-> its float-float copy (float4 {re.hi, im.hi, re.lo, im.lo}, same
// offsets), scaled by ff_scale: to_ff = true converts X -> copy, false copy -> X.
__global__ void k_svd_ff_io(double2* __restrict__ work, float4* __restrict__ xff, const int64_t* __restrict__ blk,
                            int nblk, const double* __restrict__ fro2, bool to_ff) {
  const int b = blockIdx.y;
  if (b >= nblk) return;
  const int64_t* d = blk + SVF * b;
  const int64_t len = d[2] * d[3];
  double2* X = work + d[4];
  float4* F = xff + d[4];
  const double up = ff_scale(fro2[b]), down = 1.0 / up;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < len; e += (int64_t)gridDim.x * blockDim.x) {
    if (to_ff) {
      const FF re = ff_from(X[e].x * up), im = ff_from(X[e].y * up);
      F[e] = make_float4(re.hi, im.hi, re.lo, im.lo);
    } else {
      const float4 v = F[e];
      X[e] = make_double2(((double)v.x + (double)v.z) * down, ((double)v.y + (double)v.w) * down);
    }
  }
}

// pair q of step s of the round-robin schedule on n (even) items
__device__ __forceinline__ void rr_pair(int n, int s, int q, int& i, int& j) {
  if (q == 0) {
    i = s;
    j = n - 1;
  } else {
    i = (s + q) % (n - 1);
    j = (s - q + (n - 1)) % (n - 1);
  }
}

// One round of the block-cyclic schedule for every block. The r columns of a block form
// G = ceil(r / W) groups of W (padded to an even count Gp with an empty group); round
// `round` pairs the groups round-robin and CTA k of the block takes group pair k: it stages
// the (up to) 2W columns of X, and of V when vf >= 0, in shared memory (asynchronous copies,
// all in flight together), rotates every cross pair (one pair per warp, W disjoint pairs per
// step, W steps), in round 0 first every pair inside each of the two groups, and
// writes the columns back. Over Gp - 1 rounds each column pair is rotated once (one sweep).
// T is float (pre-sweeps) or double.
// MODE 0: FP32 columns and V (T2 = float2); 1: FP64 (double2); 2: float-float columns
// (float4, scaled by ff_scale).
template <int MODE, bool REAL, class T, class T2, class S2>
__global__ void __launch_bounds__(512) k_svd_bround(T2* __restrict__ work, const int64_t* __restrict__ blk, int xf,
                                                    int vf, const int64_t* __restrict__ grp_prefix,
                                                    const int64_t* __restrict__ order, int nblk, int round, int W,
                                                    T tol, const double* __restrict__ fro2, double zero_rel,
                                                    int* __restrict__ rotated, int* __restrict__ last_rot, int sweep,
                                                    unsigned long long* __restrict__ wctr,
                                                    const int* __restrict__ prev_rotated) {
  extern __shared__ __align__(16) uint8_t smem_raw[];
  __shared__ int n_rot;
  __shared__ unsigned long long n_tested, n_rotated;   // element-pairs tested / rotated
  __shared__ int s_last[32];   // sweep in which each staged column last rotated
  __shared__ FF s_norm[32];    // float-float column norms (MODE 2)
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarp = blockDim.x >> 5;
  const int64_t cta = blockIdx.x;
  int lo = 0, hi = nblk - 1;   // largest k with grp_prefix[k] <= cta; the CTAs run over the
  while (lo < hi) {            // blocks in the order `order` (longest sweeps first)
    const int mid = (lo + hi + 1) >> 1;
    if (grp_prefix[mid] <= cta) lo = mid; else hi = mid - 1;
  }
  const int b = (int)order[lo];
  const int64_t* d = blk + SVF * b;
  const int p = (int)d[2], r = (int)d[3];
  const int G = (r + W - 1) / W, Gp = G + (G & 1) < 2 ? 2 : G + (G & 1);
  if (r == 0 || round >= Gp - 1) return;
  // Rounds are launched as programmatic dependents of the previous launch: everything above
  // reads only the tables the host wrote before the sweeps; the columns, the last-rotation
  // sweeps and the rotation counts are read after the previous round has completed.
  asm volatile("griddepcontrol.wait;" ::: "memory");
  // the host enqueues each sweep before it has read the previous sweep's rotation count: a
  // sweep that follows one in which nothing rotated (the phase converged) does nothing
  if (prev_rotated != nullptr && *prev_rotated == 0) return;
  const int k = (int)(cta - grp_prefix[lo]);
  int gI, gJ;
  rr_pair(Gp, round, k, gI, gJ);
  const int nI = gI < G ? min(W, r - gI * W) : 0, nJ = gJ < G ? min(W, r - gJ * W) : 0;
  if (nI + nJ < 2) return;
  // From the third sweep on, a pair is tested only if one of its columns rotated in this or
  // the previous sweep (see do_pair); a group pair none of whose columns did has nothing to do.
  if (sweep >= 2) {
    bool live = false;
    if (warp == 0)
      for (int cc = lane; cc < nI + nJ; cc += 32) {
        const int gc = cc < nI ? gI * W + cc : gJ * W + cc - nI;
        live = live || last_rot[d[8] + gc] >= sweep - 1;
      }
    if (__syncthreads_or(live) == 0) return;
  }
  if (threadIdx.x == 0) {
    n_rot = 0;
    n_tested = n_rotated = 0;
  }
  int mine = 0;
  unsigned long long my_tested = 0, my_rotated = 0;   // this warp's element-pairs (counters)
  T2* X = work + d[xf];
  T2* V = vf >= 0 ? work + d[vf] : nullptr;
  S2* sx = (S2*)smem_raw;                      // 2W columns of length p
  S2* sv = sx + (int64_t)2 * W * p;            // 2W columns of length r (V, MODE 0)
  // float-float columns are held scaled by ff_scale(fro2) (svd_ff_io)
  const double up = MODE == 2 ? ff_scale(fro2[b]) : 1.0;
  // stage: local column c < W is column gI*W + c, c >= W is column gJ*W + c - W (one warp
  // per column, lanes along it)
  for (int cc = warp; cc < nI + nJ; cc += nwarp) {
    const int lc = cc < nI ? cc : W + cc - nI;
    const int gc = cc < nI ? gI * W + cc : gJ * W + cc - nI;
    const T2* src = X + (int64_t)gc * p;
    S2* dst = sx + (int64_t)lc * p;
    for (int t = lane; t < p; t += 32) stage_elem<S2>(dst + t, (const S2*)(src + t));
    if constexpr (MODE == 0)
      if (V != nullptr) {
        const T2* vs = V + (int64_t)gc * r;
        S2* vd = sv + (int64_t)lc * r;
        for (int t = lane; t < r; t += 32) stage_elem<S2>(vd + t, (const S2*)(vs + t));
      }
  }
  for (int cc = threadIdx.x; cc < nI + nJ; cc += blockDim.x) {
    const int lc = cc < nI ? cc : W + cc - nI;
    const int gc = cc < nI ? gI * W + cc : gJ * W + cc - nI;
    s_last[lc] = last_rot[d[8] + gc];
  }
  stage_wait();
  __syncthreads();
  if constexpr (MODE == 2) {   // norms of the staged columns, one warp per column
    for (int cc = warp; cc < nI + nJ; cc += nwarp) {
      const int lc = cc < nI ? cc : W + cc - nI;
      const float4* x = sx + (int64_t)lc * p;
      FFAcc A = {0.f, 0.f};
      for (int t = lane; t < p; t += 32) {
        const float4 u = x[t];
        ff_mac(A, FF{u.x, u.z}, FF{u.x, u.z});
        if (!REAL) ff_mac(A, FF{u.y, u.w}, FF{u.y, u.w});
      }
      const FF nrm = ff_warp_sum(ff_norm(A));
      if (lane == 0) s_norm[lc] = nrm;
    }
    __syncthreads();
  }
  const double floor2 = zero_rel * fro2[b];
  // A pair found orthogonal in the previous sweep stays orthogonal while neither column
  // rotates: pairs whose columns last rotated before the previous sweep are skipped (the
  // first two sweeps test every pair, last_rot starting at 0).
  auto do_pair = [&](int i, int j) {
    if (s_last[i] < sweep - 1 && s_last[j] < sweep - 1) return;
    bool rot;
    if constexpr (MODE == 2) {
      FF na = s_norm[i], nb = s_norm[j];
      rot = jacobi_pair_ff<REAL>(sx + (int64_t)i * p, sx + (int64_t)j * p, p, (float)tol, (float)(floor2 * up * up), na,
                           nb, lane);
      if (rot && lane == 0) {
        s_norm[i] = na;
        s_norm[j] = nb;
      }
    } else {
      rot = jacobi_pair<T, T2, REAL>(sx + (int64_t)i * p, sx + (int64_t)j * p, p, V ? sv + (int64_t)i * r : nullptr,
                               V ? sv + (int64_t)j * r : nullptr, r, tol, floor2, lane);
    }
    my_tested += p;
    if (rot) {
      ++mine;
      my_rotated += p;
      if (lane == 0) s_last[i] = s_last[j] = sweep;
    }
    __syncwarp();
  };
  if (round == 0) {
    // pairs inside group I (warps 0 .. W/2-1) and inside group J (warps W/2 .. W-1)
    for (int st = 0; st < W - 1; ++st) {
      const int grp = warp < W / 2 ? 0 : 1;
      int i, j;
      rr_pair(W, st, warp % (W / 2), i, j);
      const int n = grp ? nJ : nI;
      if (i < n && j < n) do_pair(grp * W + i, grp * W + j);
      __syncthreads();
    }
  }
  for (int st = 0; st < W; ++st) {             // cross pairs (I_w, J_{(w + st) mod W})
    const int i = warp, j = (warp + st) % W;
    if (i < nI && j < nJ) do_pair(i, W + j);
    __syncthreads();
  }
  // the next round may be scheduled now; it waits for this one's write-back to complete
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  for (int cc = warp; cc < nI + nJ; cc += nwarp) {
    const int lc = cc < nI ? cc : W + cc - nI;
    const int gc = cc < nI ? gI * W + cc : gJ * W + cc - nI;
    T2* dst = X + (int64_t)gc * p;
    const S2* src = sx + (int64_t)lc * p;
    for (int t = lane; t < p; t += 32) dst[t] = src[t];
    if constexpr (MODE == 0)
      if (V != nullptr) {
        T2* vd = V + (int64_t)gc * r;
        const S2* vs = sv + (int64_t)lc * r;
        for (int t = lane; t < r; t += 32) vd[t] = vs[t];
      }
  }
  for (int cc = threadIdx.x; cc < nI + nJ; cc += blockDim.x) {
    const int lc = cc < nI ? cc : W + cc - nI;
    const int gc = cc < nI ? gI * W + cc : gJ * W + cc - nI;
    last_rot[d[8] + gc] = s_last[lc];
  }
  if (lane == 0 && mine) atomicAdd(&n_rot, mine);
  if (lane == 0 && my_tested) atomicAdd(&n_tested, my_tested);
  if (lane == 0 && my_rotated) atomicAdd(&n_rotated, my_rotated);
  __syncthreads();
  if (threadIdx.x == 0) {
    if (n_rot) atomicAdd(rotated, n_rot);
    atomicAdd(&wctr[0], n_tested);
    atomicAdd(&wctr[1], n_rotated);
  }
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

// Ordering key of a non-negative double: its bit pattern, which orders like the value (the sign
// bit is cleared, so -0 and +0 are equal). Integer compares run on the integer pipe, where FP64
// compares would share the GPU's few FP64 units; keys with ties broken by index also give a
// strict total order, so ranks are a permutation whatever the values.
__device__ __forceinline__ long long order_key(double v) {
  return __double_as_longlong(v) & 0x7fffffffffffffffll;
}

// Per block: singular values (column norms of X) sorted descending (ties by column index),
// and the orthonormal factor of the block's side: side 0 (X = M): U (m x r, row-major) with
// column k = X column ord[k] / sigma; side 1 (X = M^+): V^+ (r x n, row-major) with row k =
// conj(X column ord[k]) / sigma. Columns with sigma = 0 are written as zero. S holds the values
// in column order, S_sorted in decreasing order, zero-padded to the block's slot length; the
// reciprocals 1 / sigma are staged in S_sorted while the vectors are written.
__global__ void k_svd_finish(const double2* __restrict__ work, const int64_t* __restrict__ blk, int nblk,
                             double2* __restrict__ U, double2* __restrict__ Vh, double* __restrict__ S,
                             double* __restrict__ S_sorted, int* __restrict__ order_scratch,
                             const double* __restrict__ fro2) {
  const int b = blockIdx.x;
  if (b >= nblk) return;
  const int64_t* d = blk + SVF * b;
  const int64_t m = d[0], n = d[1], p = d[2], r = d[3];
  const bool wide = d[9] != 0;
  const double2* X = work + d[4];
  double* s = S + d[8];
  double* so = S_sorted + d[8];
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
    const long long v = order_key(s[j]);
    int rank = 0;
    for (int64_t k = 0; k < r; ++k) {
      const long long w = order_key(s[k]);
      rank += (w > v) || (w == v && k < j);
    }
    ord[rank] = (int)j;
  }
  __syncthreads();
  for (int64_t kk = threadIdx.x; kk < r; kk += blockDim.x) {
    const double sig = s[ord[kk]];
    so[kk] = sig > 0 ? 1.0 / sig : 0.0;
  }
  __syncthreads();
  if (!wide) {
    double2* u = U + d[6];
    for (int64_t e = threadIdx.x; e < m * r; e += blockDim.x) {
      const int64_t row = e / r, kk = e % r;
      const double2 x = X[(int64_t)ord[kk] * p + row];
      const double inv = so[kk];
      u[row * r + kk] = make_double2(x.x * inv, x.y * inv);
    }
  } else {
    double2* vh = Vh + d[7];
    for (int64_t e = threadIdx.x; e < r * n; e += blockDim.x) {
      const int64_t kk = e / n, col = e % n;
      const double2 x = X[(int64_t)ord[kk] * p + col];
      const double inv = so[kk];
      vh[kk * n + col] = make_double2(x.x * inv, -x.y * inv);
    }
  }
  __syncthreads();
  for (int64_t kk = threadIdx.x; kk < r; kk += blockDim.x) so[kk] = s[ord[kk]];
  for (int64_t j = r + threadIdx.x; j < d[12]; j += blockDim.x) so[j] = 0.0;
}

// Phase convention of the orthonormal factor (the singular vectors are fixed only up to a phase
// each): every column of U (side 0) or row of V^+ (side 1) is multiplied by the conjugate phase
// of its entry of largest modulus (the first such entry), which makes that entry real and
// positive. One CTA per block, one thread per vector.
__global__ void k_svd_fix_phases(double2* __restrict__ U, double2* __restrict__ Vh, const int64_t* __restrict__ blk,
                                 int nblk, int side) {
  const int b = blockIdx.x;
  if (b >= nblk) return;
  const int64_t* d = blk + SVF * b;
  const int64_t m = d[0], n = d[1], r = d[3];
  for (int64_t k = threadIdx.x; k < r; k += blockDim.x) {
    double2* v = side == 0 ? U + d[6] + k : Vh + d[7] + k * n;   // column k of U or row k of V^+
    const int64_t len = side == 0 ? m : n, stride = side == 0 ? r : 1;
    double best = -1.0;
    double2 at = make_double2(0.0, 0.0);
    for (int64_t i = 0; i < len; ++i) {
      const double2 x = v[i * stride];
      const double a = x.x * x.x + x.y * x.y;
      if (a > best) { best = a; at = x; }
    }
    if (!(best > 0.0)) continue;
    const double inv = 1.0 / sqrt(best);
    const double pr = at.x * inv, pi = -at.y * inv;   // conj(phase)
    for (int64_t i = 0; i < len; ++i) {
      const double2 x = v[i * stride];
      v[i * stride] = make_double2(x.x * pr - x.y * pi, x.x * pi + x.y * pr);
    }
  }
}

// Squared norms of the columns of X (FP64, field 4) of every block, one warp per column:
// out[s_off + j] for j < r.
__global__ void k_svd_colnorm2(const double2* __restrict__ work, const int64_t* __restrict__ blk, int nblk,
                               double* __restrict__ out) {
  const int b = blockIdx.y;
  if (b >= nblk) return;
  const int64_t* d = blk + SVF * b;
  const int64_t p = d[2], r = d[3];
  const int lane = threadIdx.x & 31;
  for (int64_t j = blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5); j < r; j += (int64_t)gridDim.x * (blockDim.x / 32)) {
    const double2* x = work + d[4] + j * p;
    double acc = 0.0;
    for (int64_t t = lane; t < p; t += 32) acc = fma(x[t].x, x[t].x, fma(x[t].y, x[t].y, acc));
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) out[d[8] + j] = acc;
  }
}

// Columns of every block gathered in a new order: X[:, j] = src[:, perm[s_off + j]] for j < r
// (X at field 4 of work, src with the same offsets).
__global__ void k_svd_gather_cols(double2* __restrict__ work, const double2* __restrict__ src,
                                  const int64_t* __restrict__ blk, int nblk, const int* __restrict__ perm) {
  const int b = blockIdx.y;
  if (b >= nblk) return;
  const int64_t* d = blk + SVF * b;
  const int64_t p = d[2], r = d[3];
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < p * r; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t j = e / p, t = e % p;
    work[d[4] + j * p + t] = src[d[4] + (int64_t)perm[d[8] + j] * p + t];
  }
}

// Global truncation, three launches. keep[b] = number of kept values of block b (the chi
// largest over all blocks, ties broken by (block, index), and above cutoff * s_max);
// info[0] = scale applied to the kept values (1/sqrt(sum kept s^2)), info[1] = discarded
// weight (sum of discarded s^2 / total), info[2] = s_max; info[3] holds s_max as bits while
// it is being formed (non-negative doubles order like their bit patterns).
__global__ void k_trunc_prep(const int64_t* __restrict__ blk, int nblk, const double* __restrict__ S_sorted,
                             int* __restrict__ keep, double* __restrict__ info, int* __restrict__ flat_block) {
  const int b = blockIdx.x;
  if (b >= nblk) return;
  const int64_t* d = blk + SVF * b;
  for (int64_t k = threadIdx.x; k < d[12]; k += blockDim.x) flat_block[d[8] + k] = b;
  if (threadIdx.x == 0) {
    keep[b] = 0;
    if (d[3] > 0)
      atomicMax((unsigned long long*)&info[3], (unsigned long long)__double_as_longlong(S_sorted[d[8]]));
  }
}

constexpr int kRankTile = 256;    // threads of a rank CTA, and values staged per tile
constexpr int kRankPerWarp = 4;   // values ranked by each warp
constexpr int kRankPerCta = kRankTile / 32 * kRankPerWarp;

// Rank of every value among all values (ties: lower block, then lower position first); a value
// of rank < chi above the cutoff is kept. Each warp ranks kRankPerWarp values: the CTA stages
// the values' order keys and blocks through shared memory in tiles, each lane compares its
// warp's values with every 32nd staged entry, and the lanes' counts are summed by shuffles, so
// the all-pairs comparison is spread over the whole GPU.
__global__ void __launch_bounds__(kRankTile) k_trunc_rank(const double* __restrict__ S_sorted, int64_t total, int chi,
                                                          double cutoff, int* __restrict__ keep,
                                                          const double* __restrict__ info,
                                                          const int* __restrict__ flat_block) {
  __shared__ long long sv[kRankTile];
  __shared__ int sb[kRankTile];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t e0 = blockIdx.x * (int64_t)kRankPerCta + warp * kRankPerWarp;
  long long v[kRankPerWarp];
  int be[kRankPerWarp], cnt[kRankPerWarp];
#pragma unroll
  for (int u = 0; u < kRankPerWarp; ++u) {
    const bool live = e0 + u < total;
    v[u] = order_key(live ? S_sorted[e0 + u] : 0.0);
    be[u] = live ? flat_block[e0 + u] : 0;
    cnt[u] = 0;
  }
  for (int64_t f0 = 0; f0 < total; f0 += kRankTile) {
    const int64_t f = f0 + threadIdx.x;
    __syncthreads();
    if (f < total) {
      sv[threadIdx.x] = order_key(S_sorted[f]);
      sb[threadIdx.x] = flat_block[f];
    }
    __syncthreads();
    const int n = total - f0 < kRankTile ? (int)(total - f0) : kRankTile;
    for (int q = lane; q < n; q += 32) {
      const long long w = sv[q];
      const int bf = sb[q];
      const int64_t fq = f0 + q;
#pragma unroll
      for (int u = 0; u < kRankPerWarp; ++u)
        cnt[u] += (w > v[u]) || (w == v[u] && (bf < be[u] || (bf == be[u] && fq < e0 + u)));
    }
  }
#pragma unroll
  for (int u = 0; u < kRankPerWarp; ++u)
    for (int o = 16; o > 0; o >>= 1) cnt[u] += __shfl_xor_sync(0xffffffffu, cnt[u], o);
  if (lane < kRankPerWarp) {
    int rank = cnt[0], b = be[0];
    const int64_t e = e0 + lane;
#pragma unroll
    for (int u = 1; u < kRankPerWarp; ++u)
      if (lane == u) { rank = cnt[u]; b = be[u]; }
    if (e < total) {
      const double x = S_sorted[e];
      const double smax = __longlong_as_double((long long)__double_as_longlong(info[3]));
      if (rank < chi && x > cutoff * smax) atomicAdd(&keep[b], 1);
    }
  }
}

// kept and total weight with a fixed reduction order (one CTA of 1024 threads)
__global__ void __launch_bounds__(1024) k_trunc_sums(const int64_t* __restrict__ blk, const double* __restrict__ S_sorted,
                                                     int64_t total, const int* __restrict__ keep,
                                                     double* __restrict__ info, const int* __restrict__ flat_block) {
  __shared__ double s_all[1024], s_kept[1024];
  double all = 0.0, kept = 0.0;
  for (int64_t e = threadIdx.x; e < total; e += 1024) {
    const int b = flat_block[e];
    const double v = S_sorted[e];
    all += v * v;
    if (e - blk[SVF * b + 8] < keep[b]) kept += v * v;
  }
  s_all[threadIdx.x] = all;
  s_kept[threadIdx.x] = kept;
  __syncthreads();
  for (int h = 512; h > 0; h >>= 1) {
    if (threadIdx.x < h) {
      s_all[threadIdx.x] += s_all[threadIdx.x + h];
      s_kept[threadIdx.x] += s_kept[threadIdx.x + h];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const double a = s_all[0], k = s_kept[0];
    info[2] = __longlong_as_double((long long)__double_as_longlong(info[3]));
    info[0] = k > 0 ? 1.0 / sqrt(k) : 0.0;
    info[1] = a > 0 ? (a - k) / a : 0.0;
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

// Shared memory of one CTA of the block rounds for column length p and V length r_v.
int64_t svd_bround_smem(int W, int64_t p, int64_t r_v, bool f32) {
  return (int64_t)2 * W * (p + r_v) * (f32 ? 8 : 16);
}

template <int MODE, bool REAL, class T, class T2>
static cudaError_t launch_bround(T2* work, const int64_t* blk, int xf, int vf, const int64_t* grp_prefix,
                                 const int64_t* order, int nblk, int64_t ncta, int round, int W, int64_t smem, T tol,
                                 const double* fro2, double zero_rel, int* rotated, int* last_rot, int sweep,
                                 unsigned long long* wctr, const int* prev_rotated, cudaStream_t s) {
  if (ncta == 0) return cudaSuccess;
  if (W < 2 || W > 16 || (W & 1)) return cudaErrorInvalidValue;
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(k_svd_bround<MODE, REAL, T, T2, T2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         kSvdMaxSmem);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  // programmatic dependent launch: the round's CTAs are scheduled while the previous round
  // writes back, and wait (griddepcontrol.wait) before reading anything it wrote
  cudaLaunchConfig_t lc = {};
  lc.gridDim = dim3((unsigned)ncta);
  lc.blockDim = dim3((unsigned)(W * 32));
  lc.dynamicSmemBytes = (size_t)smem;
  lc.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  lc.attrs = at;
  lc.numAttrs = 1;
  cudaError_t e = cudaLaunchKernelEx(&lc, k_svd_bround<MODE, REAL, T, T2, T2>, work, blk, xf, vf, grp_prefix, order,
                                     nblk, round, W, tol, fro2, zero_rel, rotated, last_rot, sweep, wctr, prev_rotated);
  mrd::count_launch();
  return e;
}

// FP64 rounds on X (field 4 of work) or, with xff != nullptr, float-float rounds on the
// float-float copy xff (same offsets, see svd_ff_io); real: real columns (float-float only).
cudaError_t svd_bround(double2* work, float4* xff, const int64_t* blk, const int64_t* grp_prefix,
                       const int64_t* order, int nblk, int64_t ncta, int round, int W, int64_t smem, double tol,
                       const double* fro2, int* rotated, int* last_rot, int sweep, unsigned long long* wctr,
                       const int* prev_rotated, bool real, cudaStream_t s) {
  if (xff && real)
    return launch_bround<2, true, double, float4>(xff, blk, 4, -1, grp_prefix, order, nblk, ncta, round, W, smem,
                                                  tol, fro2, 1e-28, rotated, last_rot, sweep, wctr, prev_rotated, s);
  if (xff)
    return launch_bround<2, false, double, float4>(xff, blk, 4, -1, grp_prefix, order, nblk, ncta, round, W, smem,
                                                   tol, fro2, 1e-28, rotated, last_rot, sweep, wctr, prev_rotated, s);
  return launch_bround<1, false, double, double2>(work, blk, 4, -1, grp_prefix, order, nblk, ncta, round, W, smem,
                                                  tol, fro2, 1e-28, rotated, last_rot, sweep, wctr, prev_rotated, s);
}

cudaError_t svd_ff_io(double2* work, float4* xff, const int64_t* blk, int nblk, const double* fro2, bool to_ff,
                      cudaStream_t s) {
  if (nblk == 0) return cudaSuccess;
  dim3 grid(32, nblk);
  k_svd_ff_io<<<grid, 256, 0, s>>>(work, xff, blk, nblk, fro2, to_ff);
  mrd::count_launch();
  return cudaGetLastError();
}

cudaError_t svd_bround32(float2* w32, const int64_t* blk, const int64_t* grp_prefix, const int64_t* order, int nblk,
                         int64_t ncta, int round, int W, int64_t smem, float tol, const double* fro2,
                         int* rotated, int* last_rot, int sweep, unsigned long long* wctr,
                         const int* prev_rotated, bool real, cudaStream_t s) {
  if (real)
    return launch_bround<0, true, float, float2>(w32, blk, 10, 11, grp_prefix, order, nblk, ncta, round, W, smem,
                                                 tol, fro2, 1e-12, rotated, last_rot, sweep, wctr, prev_rotated, s);
  return launch_bround<0, false, float, float2>(w32, blk, 10, 11, grp_prefix, order, nblk, ncta, round, W, smem, tol,
                                                fro2, 1e-12, rotated, last_rot, sweep, wctr, prev_rotated, s);
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
  k_svd_finish<<<nblk, 256, 0, s>>>(work, blk, nblk, U, Vh, S, S_sorted, order_scratch, fro2);
  mrd::count_launch();
  return cudaGetLastError();
}

cudaError_t svd_fix_phases(double2* U, double2* Vh, const int64_t* blk, int nblk, int side, cudaStream_t s) {
  if (nblk == 0) return cudaSuccess;
  k_svd_fix_phases<<<nblk, 128, 0, s>>>(U, Vh, blk, nblk, side);
  mrd::count_launch();
  return cudaGetLastError();
}

cudaError_t svd_colnorm2(const double2* work, const int64_t* blk, int nblk, double* out, cudaStream_t s) {
  if (nblk == 0) return cudaSuccess;
  dim3 grid(16, nblk);
  k_svd_colnorm2<<<grid, 256, 0, s>>>(work, blk, nblk, out);
  mrd::count_launch();
  return cudaGetLastError();
}

cudaError_t svd_gather_cols(double2* work, const double2* src, const int64_t* blk, int nblk, const int* perm,
                            cudaStream_t s) {
  if (nblk == 0) return cudaSuccess;
  dim3 grid(32, nblk);
  k_svd_gather_cols<<<grid, 256, 0, s>>>(work, src, blk, nblk, perm);
  mrd::count_launch();
  return cudaGetLastError();
}

cudaError_t svd_truncate(const int64_t* blk, int nblk, const double* S_sorted, int64_t total, int chi, double cutoff,
                         int* keep, double* info, int* flat_block, cudaStream_t s) {
  if (nblk <= 0) return cudaMemsetAsync(info, 0, 4 * 8, s);
  cudaError_t e = cudaMemsetAsync(info, 0, 4 * 8, s);
  if (e != cudaSuccess) return e;
  k_trunc_prep<<<nblk, 256, 0, s>>>(blk, nblk, S_sorted, keep, info, flat_block);
  mrd::count_launch();
  if (total > 0) {
    k_trunc_rank<<<(unsigned)((total + kRankPerCta - 1) / kRankPerCta), kRankTile, 0, s>>>(S_sorted, total, chi, cutoff,
                                                                                     keep, info, flat_block);
    mrd::count_launch();
  }
  k_trunc_sums<<<1, 1024, 0, s>>>(blk, S_sorted, total, keep, info, flat_block);
  mrd::count_launch();
  return cudaGetLastError();
}

}  // namespace mrd
