// Two-site DMRG on the device: block-sparse MPS, environments, two-site update and sweep.
//
// The paper applies standard finite/infinite DMRG (its refs. W92, S2005, S2011, M08) to the
// mixed-basis MPO; this file is the finite two-site algorithm on an open cylinder:
//   theta = M_i M_{i+1}; ground state of H_eff = L W_i W_{i+1} R by Lanczos; block SVD of
//   theta by middle charge (the Schmidt decomposition, Sec. III.C) truncated to chi;
//   left- or right-canonical factors; environment update L' = A^+ (L W) A or
//   R' = B (W R) B^+; sweep left to right and back.
// Block-sparse MPS tensor M[l, s, r] (r = l + q(s)) is stored either grouped by right sector
// (mode 0: rows (s, l) stacked per r, the layout of U from the SVD) or grouped by left
// sector (mode 1: columns (s, r) side by side per l, the layout of V^+). Both are addressed
// through sub-blocks (l, s) of shape d_l x d_r with a leading dimension.
// All contractions are grouped complex GEMMs (the FP64 kernel of heff_fp64.cu) over task
// lists built here from the sector tables; every output block has one owner task.
#include <algorithm>
#include <array>
#include <chrono>
#include <cmath>
#include <cstring>
#include <map>
#include <string>
#include <vector>

#include "heff_internal.h"

namespace mrd {

cudaError_t launch_cgemm_ff_packed(const float4* A, const float4* B, float4* c_ff, double2* c64, const int64_t* tasks,
                                   const int64_t* segs, const int64_t* prefix, int64_t n_tasks, int64_t total_tiles,
                                   int n_sm, cudaStream_t s, const int2* items = nullptr);
cudaError_t launch_rgemm_ff_packed(const float4* A, const float4* B, float4* c_ff, double2* c64, const int64_t* tasks,
                                   const int64_t* segs, const int64_t* prefix, int64_t n_tasks, int64_t total_tiles,
                                   int n_sm, cudaStream_t s, const int2* items = nullptr);
std::vector<int2> ff_item_order(const int64_t* tasks, const int64_t* segs, int64_t n_tasks);
cudaError_t to_ff(const double2* x, float4* y, int64_t n, cudaStream_t s);
cudaError_t launch_cgemm_fp64(const double2* A, const double2* B, double2* C, const int64_t* tasks,
                              const int64_t* segs, const int64_t* prefix, int64_t n_tasks, int64_t total_tiles,
                              int n_sm, cudaStream_t s);
cudaError_t svd_load(const double2* theta, const int64_t* blk, const int64_t* src_off, int nblk, double2* work,
                     double* fro2, cudaStream_t s);
int64_t svd_bround_smem(int W, int64_t p, int64_t r_v, bool f32);
cudaError_t svd_bround(double2* work, float4* xff, const int64_t* blk, const int64_t* grp_prefix,
                       const int64_t* order, int nblk, int64_t ncta, int round, int W, int64_t smem, double tol,
                       const double* fro2, int* rotated, int* last_rot, int sweep, unsigned long long* wctr,
                       const int* prev_rotated, bool real, cudaStream_t s);
cudaError_t svd_ff_io(double2* work, float4* xff, const int64_t* blk, int nblk, const double* fro2, bool to_ff,
                      cudaStream_t s);
cudaError_t svd_finish(const double2* work, const int64_t* blk, int nblk, double2* U, double2* Vh, double* S,
                       double* S_sorted, int* order_scratch, const double* fro2, cudaStream_t s);
cudaError_t svd_truncate(const int64_t* blk, int nblk, const double* S_sorted, int64_t total, int chi, double cutoff,
                         int* keep, double* info, int* flat_block, cudaStream_t s);
cudaError_t svd_bround32(float2* w32, const int64_t* blk, const int64_t* grp_prefix, const int64_t* order, int nblk,
                         int64_t ncta, int round, int W, int64_t smem, float tol, const double* fro2,
                         int* rotated, int* last_rot, int sweep, unsigned long long* wctr,
                         const int* prev_rotated, bool real, cudaStream_t s);
cudaError_t svd_to_f32(const double2* work, float2* w32, const int64_t* blk, int nblk, cudaStream_t s);
cudaError_t svd_v_from_f32(double2* work, const float2* w32, const int64_t* blk, int nblk, cudaStream_t s);
cudaError_t svd_colnorm2(const double2* work, const int64_t* blk, int nblk, double* out, cudaStream_t s);
cudaError_t svd_fix_phases(double2* U, double2* Vh, const int64_t* blk, int nblk, int side, cudaStream_t s);
cudaError_t svd_gather_cols(double2* work, const double2* src, const int64_t* blk, int nblk, const int* perm,
                            cudaStream_t s);
enum { SVF = 13 };
// After the FP32 pre-sweeps, columns whose norm is below this fraction of the chi-th largest
// column norm over all blocks are set aside: they hold Schmidt weight that the truncation to
// chi discards, so the float-float sweeps run on the other columns only (see block_svd)
constexpr double kSetAsideFrac = 0.5;
constexpr int64_t kSvdMaxSmemHost = 220 * 1024;   // dynamic shared memory of a Jacobi CTA
// orthogonality tolerance |x_i^+ x_j| / (|x_i| |x_j|) of the final sweeps: FP64, and float-float
// (48-bit products: dot products of a few hundred terms carry ~1e-13 relative noise)
constexpr double kTolF64 = 1e-14, kTolFF = 5e-13;
constexpr int kMaxSweeps64 = 60;
// FP32 pre-sweeps stop after this many: they settle the large rotations of the dominant
// columns; graded tails are left to the final sweeps anyway (at chi=3200: 8 FP32 + 18
// float-float sweeps take ~55 ms, against ~62 ms for float-float alone and ~66 ms for FP32 run
// to convergence first)
constexpr int kMaxSweeps32 = 8;

namespace {

constexpr int kTile = 32;

struct Sec {
  int32_t N, K, d;
};
using Secs = std::vector<Sec>;

int find_sec(const Secs& s, int N, int K) {
  const int64_t key = qkey(N, K);
  int lo = 0, hi = (int)s.size() - 1;
  while (lo <= hi) {
    const int m = (lo + hi) >> 1;
    const int64_t k = qkey(s[m].N, s[m].K);
    if (k == key) return m;
    if (k < key) lo = m + 1; else hi = m - 1;
  }
  return -1;
}

// ---------------------------------------------------------------- device buffers

struct Buf {
  void* p = nullptr;
  size_t bytes = 0;
  ~Buf() { if (p) cudaFree(p); }
  cudaError_t need(size_t b) {
    if (b <= bytes && p) return cudaSuccess;
    if (p) cudaFree(p);
    p = nullptr;
    bytes = 0;
    size_t nb = std::max<size_t>(b, 256);
    cudaError_t e = cudaMalloc(&p, nb);
    if (e == cudaSuccess) bytes = nb;
    return e;
  }
  template <class T>
  T* as() const { return (T*)p; }
};

// ---------------------------------------------------------------- kernels

__device__ __forceinline__ uint64_t splitmix64(uint64_t x) {
  // SplitMix64 finaliser (Steele, Lea & Flood 2014) of state x
  x += 0x9E3779B97F4A7C15ull;
  x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
  x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
  return x ^ (x >> 31);
}

// Counter-based uniform [-1, 1) complex entries: element e of stream `seed`.
__global__ void k_fill_random(double2* out, int64_t n, uint64_t seed) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    const uint64_t a = splitmix64(seed + 2 * (uint64_t)e * 0x9E3779B97F4A7C15ull);
    const uint64_t b = splitmix64(seed + (2 * (uint64_t)e + 1) * 0x9E3779B97F4A7C15ull);
    out[e] = make_double2(2.0 * (double)(a >> 11) * 0x1.0p-53 - 1.0, 2.0 * (double)(b >> 11) * 0x1.0p-53 - 1.0);
  }
}

// Strided block copies with optional scaling by singular values:
// task: src_off src_ld dst_off dst_ld rows cols scale_mode(0 none, 1 by column, 2 by row) s_off
enum { CPF = 8 };
__global__ void k_copy_blocks(const double2* __restrict__ src, double2* __restrict__ dst,
                              const int64_t* __restrict__ tasks, int ntasks, const double* __restrict__ S,
                              const double* __restrict__ sscale) {
  const double g = sscale ? *sscale : 1.0;
  for (int t = blockIdx.x; t < ntasks; t += gridDim.x) {
    const int64_t* d = tasks + CPF * t;
    const int64_t rows = d[4], cols = d[5], mode = d[6];
    for (int64_t e = threadIdx.x; e < rows * cols; e += blockDim.x) {
      const int64_t r = e / cols, c = e % cols;
      double2 v = src[d[0] + r * d[1] + c];
      if (mode) {
        const double f = g * S[d[7] + (mode == 1 ? c : r)];
        v.x *= f;
        v.y *= f;
      }
      dst[d[2] + r * d[3] + c] = v;
    }
  }
}

constexpr int kNormParts = 256;

// partial[blockIdx.x] = sum of |x_e|^2 over a fixed strided subset (fixed reduction order)
__global__ void __launch_bounds__(256) k_sumsq_partial(const double2* __restrict__ x, int64_t n,
                                                       double* __restrict__ partial) {
  __shared__ double sm[256];
  double acc = 0.0;
  for (int64_t e = blockIdx.x * 256 + threadIdx.x; e < n; e += (int64_t)kNormParts * 256)
    acc = fma(x[e].x, x[e].x, fma(x[e].y, x[e].y, acc));
  sm[threadIdx.x] = acc;
  __syncthreads();
  for (int h = 128; h > 0; h >>= 1) {
    if (threadIdx.x < h) sm[threadIdx.x] += sm[threadIdx.x + h];
    __syncthreads();
  }
  if (threadIdx.x == 0) partial[blockIdx.x] = sm[0];
}

// Renormalise the centre tensor to unit norm: kept = |x|^2 (the weight captured by the
// orthonormal canonical factor), info[0] = 1/sqrt(kept), info[1] = discarded weight
// 1 - kept / |theta|^2 with |theta|^2 = sum of the blocks' fro2.
// Schmidt values of the bond an update cut (Sec. III.C): per kept bond sector, the norms of the
// centre tensor's rows (moving right: the centre is (a) x (s2, b)) or columns (moving left:
// (s1, a) x (b)). The canonical factor is an isometry, so these are the weights of the
// kept Schmidt states. Table row: offset, values, length of a row/column, leading dimension,
// by_rows, output offset. One CTA per bond sector, fixed summation order.
__global__ void k_schmidt(const double2* __restrict__ c, const int64_t* __restrict__ tab, int nblk,
                          double* __restrict__ out) {
  const int b = blockIdx.x;
  if (b >= nblk) return;
  const int64_t* t = tab + 6 * b;
  const int64_t off = t[0], nv = t[1], len = t[2], ld = t[3], by_rows = t[4], o = t[5];
  for (int64_t v = threadIdx.x; v < nv; v += blockDim.x) {
    double acc = 0.0;
    for (int64_t q = 0; q < len; ++q) {
      const double2 x = by_rows ? c[off + v * ld + q] : c[off + q * ld + v];
      acc = fma(x.x, x.x, fma(x.y, x.y, acc));
    }
    out[o + v] = sqrt(acc);
  }
}

__global__ void __launch_bounds__(256) k_scale_unit(double2* __restrict__ x, int64_t n,
                                                    const double* __restrict__ partial,
                                                    const double* __restrict__ fro2, int nblk,
                                                    double* __restrict__ info) {
  __shared__ double f;
  if (threadIdx.x == 0) {
    double kept = 0.0, all = 0.0;
    for (int q = 0; q < kNormParts; ++q) kept += partial[q];
    for (int b = 0; b < nblk; ++b) all += fro2[b];
    f = kept > 0.0 ? 1.0 / sqrt(kept) : 0.0;
    if (blockIdx.x == 0) {
      info[0] = f;
      info[1] = all > 0.0 ? fmax(0.0, (all - kept) / all) : 0.0;
    }
  }
  __syncthreads();
  const double g = f;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    x[e].x *= g;
    x[e].y *= g;
  }
}

}  // namespace

__global__ void k_zero_imag(double2* __restrict__ x, int64_t n) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
    x[e].y = 0.0;
}

// complex128 <-> complex64 copies of environments stored in single precision (round to
// nearest on the way down, exact on the way up)
__global__ void k_c128_to_c64(const double2* __restrict__ x, float2* __restrict__ y, int64_t n) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
    y[e] = make_float2(__double2float_rn(x[e].x), __double2float_rn(x[e].y));
}

__global__ void k_c64_to_c128(const float2* __restrict__ x, double2* __restrict__ y, int64_t n) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
    y[e] = make_double2((double)x[e].x, (double)x[e].y);
}

// ---------------------------------------------------------------- tensors

struct SiteT {
  Secs left, right;
  int m = 0, mod = 1;
  int mode = 1;
  std::vector<int64_t> goff, gext;
  std::vector<std::array<int64_t, 2>> sub;
  int64_t size = 0;
  Buf data;

  void layout() {
    goff.clear(); gext.clear(); sub.clear(); size = 0;
    if (mode == 0) {
      for (const Sec& r : right) {
        std::array<int64_t, 2> so{-1, -1};
        int64_t rows = 0;
        for (int s = 0; s < 2; ++s) {
          const int li = find_sec(left, r.N - s, kmod(r.K - s * m, mod));
          if (li >= 0) { so[s] = rows; rows += left[li].d; }
        }
        goff.push_back(size); gext.push_back(rows); sub.push_back(so);
        size += rows * r.d;
      }
    } else {
      for (const Sec& l : left) {
        std::array<int64_t, 2> so{-1, -1};
        int64_t cols = 0;
        for (int s = 0; s < 2; ++s) {
          const int ri = find_sec(right, l.N + s, kmod(l.K + s * m, mod));
          if (ri >= 0) { so[s] = cols; cols += right[ri].d; }
        }
        goff.push_back(size); gext.push_back(cols); sub.push_back(so);
        size += (int64_t)l.d * cols;
      }
    }
  }
  // sub-block (li, s): offset and leading dimension; false if absent
  bool subblock(int li, int s, int64_t* off, int64_t* ld, int* ri_out) const {
    const Sec& l = left[li];
    const int ri = find_sec(right, l.N + s, kmod(l.K + s * m, mod));
    if (ri < 0) return false;
    if (ri_out) *ri_out = ri;
    if (mode == 0) {
      if (sub[ri][s] < 0) return false;
      *off = goff[ri] + sub[ri][s] * right[ri].d;
      *ld = right[ri].d;
    } else {
      if (sub[li][s] < 0) return false;
      *off = goff[li] + sub[li][s];
      *ld = gext[li];
    }
    return true;
  }
};

struct EnvT {
  Secs sec;
  std::vector<std::array<int, 2>> ch;
  bool left = true;
  std::vector<int64_t> off;
  int64_t size = 0;
  Buf data;           // complex128, or complex64 when f32
  bool f32 = false;
  void layout(int mod) {
    off.assign(ch.size() * sec.size(), -1);
    size = 0;
    for (size_t w = 0; w < ch.size(); ++w)
      for (size_t x = 0; x < sec.size(); ++x) {
        const int xp = find_sec(sec, sec[x].N + ch[w][0], kmod(sec[x].K + ch[w][1], mod));
        if (xp < 0) continue;
        off[w * sec.size() + x] = size;
        size += (int64_t)sec[x].d * sec[xp].d;
      }
  }
};

struct GemmList {
  std::vector<int64_t> t, s;
  void task(int64_t M, int64_t N, int64_t c_off, int64_t ldc) {
    t.insert(t.end(), {M, N, c_off, ldc, (int64_t)(s.size() / SF), 0});
  }
  void seg(int64_t a_off, int64_t lda, int64_t b_off, int64_t ldb, int64_t K, int64_t flags) {
    s.insert(s.end(), {a_off, lda, b_off, ldb, K, flags});
    t.back() += 1;
  }
  void drop_empty_last() {
    if (!t.empty() && t.back() == 0) t.resize(t.size() - TF);
  }
};

}  // namespace mrd

using namespace mrd;

struct mrd_dmrg {
  mrd_ctx* ctx = nullptr;
  HostMPO mpo;
  int n = 0, ly = 0, mod = 1;
  int n_sm = 152;
  int target_N = 0, target_K = 0;
  std::vector<SiteT> A;
  std::vector<EnvT> L, R;
  Buf gtask, gseg, gpref, gitems, ctask, theta, theta2, svd_blk, svd_src, svd_pref, svd_work, svd_u, svd_vh, svd_s,
      svd_ss, svd_ord, svd_flat, svd_keep, svd_info, svd_w32, svd_x2, svd_fro, svd_last, svd_ctr, tbuf,
      zeros, svd_perm;
  // columns entering the final Jacobi sweeps and columns of all blocks, last block SVD
  double svd_cols[2] = {0, 0};
  // environments stored in complex64 (MRD_DMRG_OPT_ENV_FP32); envx: complex128 working copies
  // of the two environments an H_eff reads and of an update's output
  bool env_fp32 = false;
  Buf envx[3];
  // real arithmetic (MRD_DMRG_OPT_REAL): real MPO and tensors, H_effs declared real
  bool real = false;
  int center0 = 0;      // centre given at creation
  int updates = 0;      // two-site updates run so far
  cudaEvent_t svd_ev[2] = {nullptr, nullptr};
  // last block SVD: [0] ms of the final sweeps, [1] element-pairs tested, [2] rotated, [3] sweeps,
  // [4] ms of the FP32 pre-sweeps, [5] svd_mode
  double svd_stats[6] = {0, 0, 0, 0, 0, 0};
  int svd_sweeps32 = 0, svd_sweeps64 = 0;
  // column pairs rotated in each sweep of the last block SVD: the FP32 pre-sweeps, then the final
  std::vector<int32_t> svd_trace32, svd_trace64;
  std::vector<double> svd_tms32, svd_tms64;   // host ms of each sweep (launches to the count read back)
  int svd_presweeps = kMaxSweeps32;   // MRD_DMRG_OPT_SVD_PRESWEEPS
  Buf svd_rotv;                       // rotation count of each sweep of a phase
  int* svd_hcnt = nullptr;            // pinned host copies of them
  cudaEvent_t svd_sev[2] = {nullptr, nullptr};
  bool gemm_ff = false;   // grouped GEMMs of the update in float-float (refine_prec MRD_PREC_FF)
  double last_energy = 0.0, last_trunc = 0.0;
  // Schmidt values of the bond cut by the last update: bond index, (N, K) and value per state
  int schmidt_bond = -1;
  std::vector<int32_t> schmidt_nk;
  std::vector<double> schmidt_val;
  Buf schmidt_tab, schmidt_out;
  Buf ff_a, ff_b;   // float-float copies of the operands of a grouped GEMM
  int last_iters = 0, last_refine = 0;
  bool timing = false;
  double kms[4] = {0, 0, 0, 0};   // accumulated GEMM ms: tensor-core step 1, step 2, FP64 step 1, step 2
  int64_t kcount[2] = {0, 0};     // applies: tensor core, FP64
  double phase_ms[6] = {0, 0, 0, 0, 0, 0};   // plan, theta, lanczos, svd, tensors, env (last update)
};

namespace {

// Grouped GEMM C += sum over segments A . B on the context stream, FP64 or float-float
// (D->gemm_ff). a_ff / b_ff: the operands already split into float-float (e.g. the H_eff's
// own copies of LW / WR), used instead of converting Aop / Bop again. Asynchronous: the task
// tables are copied from pageable host memory (consumed when the copy call returns) into
// device buffers that later calls reuse in stream order.
int run_gemm(mrd_dmrg* D, GemmList& g, const double2* Aop, int64_t alen, const double2* Bop, int64_t blen, double2* C,
             int64_t clen, const float4* a_ff = nullptr, const float4* b_ff = nullptr, float4* c_ff = nullptr) {
  mrd_ctx* ctx = D->ctx;
  g.drop_empty_last();
  const int64_t nt = (int64_t)g.t.size() / TF;
  if (nt == 0) return MRD_OK;
  std::vector<int64_t> pref(nt + 1, 0);
  auto in = [](int64_t off, int64_t rows, int64_t cols, int64_t ld, int64_t len) {
    if (rows == 0 || cols == 0) return true;
    return off >= 0 && ld >= cols && off + (rows - 1) * ld + cols <= len;
  };
  for (int64_t i = 0; i < nt; ++i) {
    const int64_t* r = &g.t[TF * i];
    if (!in(r[2], r[0], r[1], r[3], clen)) return mrd_fail(ctx, MRD_E_STATE, "internal: GEMM output out of range");
    for (int64_t k = 0; k < r[5]; ++k) {
      const int64_t* q = &g.s[SF * (r[4] + k)];
      const bool ta = q[5] & 1, tb = q[5] & 2;
      bool ok = ta ? in(q[0], q[4], r[0], q[1], alen) : in(q[0], r[0], q[4], q[1], alen);
      ok = ok && (tb ? in(q[2], r[1], q[4], q[3], blen) : in(q[2], q[4], r[1], q[3], blen));
      if (!ok) return mrd_fail(ctx, MRD_E_STATE, "internal: GEMM operand out of range");
    }
    pref[i + 1] = pref[i] + ((r[0] + kTile - 1) / kTile) * ((r[1] + kTile - 1) / kTile);
  }
  cudaStream_t s = ctx->stream;
  MRD_CUDA(ctx, D->gtask.need(g.t.size() * 8));
  MRD_CUDA(ctx, D->gseg.need(std::max<size_t>(g.s.size(), 1) * 8));
  MRD_CUDA(ctx, D->gpref.need(pref.size() * 8));
  MRD_CUDA(ctx, cudaMemcpyAsync(D->gtask.p, g.t.data(), g.t.size() * 8, cudaMemcpyHostToDevice, s));
  if (!g.s.empty()) MRD_CUDA(ctx, cudaMemcpyAsync(D->gseg.p, g.s.data(), g.s.size() * 8, cudaMemcpyHostToDevice, s));
  MRD_CUDA(ctx, cudaMemcpyAsync(D->gpref.p, pref.data(), pref.size() * 8, cudaMemcpyHostToDevice, s));
  if (D->gemm_ff) {
    // float-float: split each operand once (one pass over it) instead of on every tile load,
    // where the FP64 -> float conversions would run on the slow FP64 pipe; same results
    if (!a_ff) {
      MRD_CUDA(ctx, D->ff_a.need((size_t)std::max<int64_t>(alen, 1) * 16));
      MRD_CUDA(ctx, to_ff(Aop, D->ff_a.as<float4>(), alen, s));
      a_ff = D->ff_a.as<float4>();
    }
    if (!b_ff) {
      MRD_CUDA(ctx, D->ff_b.need((size_t)std::max<int64_t>(blen, 1) * 16));
      MRD_CUDA(ctx, to_ff(Bop, D->ff_b.as<float4>(), blen, s));
      b_ff = D->ff_b.as<float4>();
    }
    // tiles in launch order, longest K first (the tile prefix above uses the same 32 x 32 tiles)
    const std::vector<int2> items = ff_item_order(g.t.data(), g.s.data(), nt);
    const int2* it = nullptr;
    if ((int64_t)items.size() == pref[nt] && !items.empty()) {
      MRD_CUDA(ctx, D->gitems.need(items.size() * 8));
      MRD_CUDA(ctx, cudaMemcpyAsync(D->gitems.p, items.data(), items.size() * 8, cudaMemcpyHostToDevice, s));
      it = D->gitems.as<int2>();
    }
    // a real state (MRD_DMRG_OPT_REAL): every operand is real, one float-float product per
    // multiply-add instead of three
    auto gemm = D->real ? launch_rgemm_ff_packed : launch_cgemm_ff_packed;
    MRD_CUDA(ctx, gemm(a_ff, b_ff, c_ff, c_ff ? nullptr : C, D->gtask.as<int64_t>(), D->gseg.as<int64_t>(),
                       D->gpref.as<int64_t>(), nt, pref[nt], D->n_sm, s, it));
  } else {
    MRD_CUDA(ctx, launch_cgemm_fp64(Aop, Bop, C, D->gtask.as<int64_t>(), D->gseg.as<int64_t>(), D->gpref.as<int64_t>(),
                                    nt, pref[nt], D->n_sm, s));
  }
  return MRD_OK;
}

int run_copies(mrd_dmrg* D, const std::vector<int64_t>& t, const double2* src, double2* dst, const double* S,
               const double* sscale) {
  mrd_ctx* ctx = D->ctx;
  const int nt = (int)(t.size() / CPF);
  if (nt == 0) return MRD_OK;
  cudaStream_t s = ctx->stream;
  MRD_CUDA(ctx, D->ctask.need(t.size() * 8));
  MRD_CUDA(ctx, cudaMemcpyAsync(D->ctask.p, t.data(), t.size() * 8, cudaMemcpyHostToDevice, s));
  k_copy_blocks<<<std::min(nt, 4096), 256, 0, s>>>(src, dst, D->ctask.as<int64_t>(), nt, S, sscale);
  mrd::count_launch();
  MRD_CUDA(ctx, cudaGetLastError());
  MRD_CUDA(ctx, cudaStreamSynchronize(s));
  return MRD_OK;
}

std::vector<std::array<int, 2>> mpo_channels(const HostMPO& m, int bond, int mod) {
  std::vector<std::array<int, 2>> c;
  const auto& v = m.bond_charges[bond];
  for (size_t i = 0; i + 1 < v.size(); i += 2) c.push_back({v[i], kmod(v[i + 1], mod)});
  return c;
}

cudaError_t conv_c64(const double2* x, float2* y, int64_t n, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  k_c128_to_c64<<<(unsigned)std::min<int64_t>((n + 255) / 256, 4096), 256, 0, s>>>(x, y, n);
  mrd::count_launch();
  return cudaGetLastError();
}

cudaError_t conv_c128(const float2* x, double2* y, int64_t n, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  k_c64_to_c128<<<(unsigned)std::min<int64_t>((n + 255) / 256, 4096), 256, 0, s>>>(x, y, n);
  mrd::count_launch();
  return cudaGetLastError();
}

// The complex128 data of an environment: its own buffer, or for single-precision storage a
// widened copy in working buffer `slot` (valid until the slot is reused).
int env_fp64(mrd_dmrg* D, EnvT& E, int slot, const double2** out) {
  if (!E.f32) {
    *out = E.data.as<double2>();
    return MRD_OK;
  }
  MRD_CUDA(D->ctx, D->envx[slot].need((size_t)std::max<int64_t>(E.size, 1) * 16));
  MRD_CUDA(D->ctx, conv_c128(E.data.as<float2>(), D->envx[slot].as<double2>(), E.size, D->ctx->stream));
  *out = D->envx[slot].as<double2>();
  return MRD_OK;
}

// Storage of a freshly computed environment: the complex128 result `src` (E.size values)
// becomes E's data, rounded to complex64 when the state stores environments in single precision.
int env_store(mrd_dmrg* D, EnvT& E, const double2* src) {
  mrd_ctx* ctx = D->ctx;
  E.f32 = D->env_fp32;
  if (!E.f32) return MRD_OK;   // computed in place
  MRD_CUDA(ctx, E.data.need((size_t)std::max<int64_t>(E.size, 1) * 8));
  MRD_CUDA(ctx, conv_c64(src, E.data.as<float2>(), E.size, ctx->stream));
  return MRD_OK;
}

// Build the H_eff handle for sites (i, i+1) from the current bonds; env pointers may be the
// zero buffer when a side is only needed for its fold with the MPO.
int make_heff(mrd_dmrg* D, int i, const double2* lenv, const double2* renv, mrd_heff** out) {
  const SiteT& X = D->A[i];
  const SiteT& Y = D->A[i + 1];
  std::vector<int32_t> ls, rs, cl, cm, cr;
  for (const Sec& s : X.left) ls.insert(ls.end(), {s.N, s.K, s.d});
  for (const Sec& s : Y.right) rs.insert(rs.end(), {s.N, s.K, s.d});
  const auto& b0 = D->mpo.bond_charges[i];
  const auto& b1 = D->mpo.bond_charges[i + 1];
  const auto& b2 = D->mpo.bond_charges[i + 2];
  mrd_heff_desc d{};
  d.n_left = (int32_t)X.left.size(); d.left = ls.data();
  d.n_right = (int32_t)Y.right.size(); d.right = rs.data();
  d.m1 = X.m; d.m2 = Y.m;
  d.modulus = D->mod;
  d.d_l = (int32_t)(b0.size() / 2); d.d_m = (int32_t)(b1.size() / 2); d.d_r = (int32_t)(b2.size() / 2);
  d.c_l = b0.data(); d.c_m = b1.data(); d.c_r = b2.data();
  d.nnz_i = (int32_t)(D->mpo.site_idx[i].size() / 4); d.wi_idx = D->mpo.site_idx[i].data(); d.wi_val = D->mpo.site_val[i].data();
  d.nnz_j = (int32_t)(D->mpo.site_idx[i + 1].size() / 4); d.wj_idx = D->mpo.site_idx[i + 1].data();
  d.wj_val = D->mpo.site_val[i + 1].data();
  int rc = mrd_heff_create(D->ctx, &d, out);
  if (rc != MRD_OK) return rc;
  mrd_heff* h = *out;
  // zero stand-ins for absent environments
  const int64_t need = std::max(h->counts[C_LENV], h->counts[C_RENV]);
  if (!lenv || !renv) {
    MRD_CUDA(D->ctx, D->zeros.need((size_t)std::max<int64_t>(need, 1) * 16));
    MRD_CUDA(D->ctx, cudaMemsetAsync(D->zeros.p, 0, (size_t)std::max<int64_t>(need, 1) * 16, D->ctx->stream));
  }
  rc = mrd_heff_set_env(h, (const double*)(lenv ? lenv : D->zeros.as<double2>()),
                        (const double*)(renv ? renv : D->zeros.as<double2>()));
  if (rc != MRD_OK) { mrd_heff_free(h); *out = nullptr; }
  return rc;
}

// theta = X * Y in the middle-sector layout of h (zero where the bond has no sector).
int form_theta(mrd_dmrg* D, mrd_heff* h, const SiteT& X, const SiteT& Y, double2* theta) {
  mrd_ctx* ctx = D->ctx;
  const int64_t n = h->counts[C_THETA];
  MRD_CUDA(ctx, cudaMemsetAsync(theta, 0, (size_t)n * 16, ctx->stream));
  GemmList g;
  const std::vector<int64_t>& mid = h->mid_host;
  for (int64_t q = 0; q < h->counts[C_NMID]; ++q) {
    const int64_t* r = &mid[MIDF * q];
    const int ci = find_sec(X.right, (int)r[0], (int)r[1]);   // bond sector between the sites
    if (ci < 0) continue;
    const int yi = find_sec(Y.left, (int)r[0], (int)r[1]);
    if (yi < 0) continue;
    const int64_t dc = X.right[ci].d;
    for (int s1 = 0; s1 < 2; ++s1) {
      if (r[5 + s1] < 0) continue;
      const int ai = (int)r[5 + s1];
      int64_t xo, xld;
      int rr;
      if (!X.subblock(ai, s1, &xo, &xld, &rr) || rr != ci) continue;
      for (int s2 = 0; s2 < 2; ++s2) {
        if (r[8 + s2] < 0) continue;
        int64_t yo, yld;
        int bi;
        if (!Y.subblock(yi, s2, &yo, &yld, &bi) || bi != (int)r[8 + s2]) continue;
        const int64_t roff = s1 ? r[7] : 0, coff = s2 ? r[10] : 0;
        g.task(X.left[ai].d, Y.right[bi].d, r[4] + roff * r[3] + coff, r[3]);
        g.seg(xo, xld, yo, yld, dc, 0);
      }
    }
  }
  // X and Y live in different buffers: run as two operands
  return run_gemm(D, g, X.data.as<double2>(), X.size, Y.data.as<double2>(), Y.size, theta, n);
}

// Block SVD of the blocks `blk` (SVF rows) of `src`; returns kept counts per block and info.
int block_svd(mrd_dmrg* D, std::vector<int64_t>& blk, const std::vector<int64_t>& src_off, const double2* src,
              int side, int chi, double cutoff, int mode, std::vector<int>& keep, double info[3]) {
  mrd_ctx* ctx = D->ctx;
  cudaStream_t s = ctx->stream;
  const int nb = (int)src_off.size();
  keep.assign(nb, 0);
  if (nb == 0) { info[0] = 1; info[1] = 0; info[2] = 0; return MRD_OK; }
  int64_t work = 0, ulen = 0, vlen = 0, slen = 0;
  for (int b = 0; b < nb; ++b) {
    int64_t* d = &blk[SVF * b];
    const int64_t m = d[0], n = d[1];
    const bool wide = side == 1;   // X = M^+ (orthonormal V) instead of X = M (orthonormal U)
    const int64_t p = wide ? n : m, r = wide ? m : n;
    d[2] = p; d[3] = r; d[9] = wide; d[12] = r;
    d[4] = work; work += p * r;
    d[6] = ulen; ulen += m * r;
    d[7] = vlen; vlen += r * n;
    d[8] = slen; slen += r;
  }
  int64_t xlen = work;
  for (int b = 0; b < nb; ++b) {   // V_X of every block after all X blocks
    blk[SVF * b + 5] = work;
    work += blk[SVF * b + 3] * blk[SVF * b + 3];
  }
  int64_t w32 = 0;                 // FP32 copies: X32 then V32 per block
  for (int b = 0; b < nb; ++b) {
    blk[SVF * b + 10] = w32;
    w32 += blk[SVF * b + 2] * blk[SVF * b + 3];
    blk[SVF * b + 11] = w32;
    w32 += blk[SVF * b + 3] * blk[SVF * b + 3];
  }
  // block-cyclic Jacobi schedules: column groups of W = 8 (256 threads a CTA; measured faster
  // than 16 for the float-float sweeps at chi = 3200, whose largest blocks bound each round),
  // halved while a group pair does not fit in shared memory
  struct Sched {
    int W = 0, rounds = 0;
    int64_t ncta = 0, smem = 0;
  };
  // pp: CTA prefix of the FP32 rounds, of the final rounds (nb + 1 each), then the block order
  // of both: longest sweep first (columns x rows, the per-sweep chain of a block's rounds), so
  // that the CTAs of the largest blocks take the lowest indices and spread over the SMs first
  std::vector<int64_t> pp(3 * nb + 2, 0);
  int64_t* order = pp.data() + 2 * (nb + 1);
  for (int b = 0; b < nb; ++b) order[b] = b;
  // Largest blocks first, then the rest in reverse: once the first CTAs hold one SM each, the
  // CTAs that share an SM with the largest blocks' are the smallest ones (snake order).
  auto order_blocks = [&](int W) {
    std::stable_sort(order, order + nb, [&](int64_t x, int64_t y) {
      return blk[SVF * x + 3] * blk[SVF * x + 2] > blk[SVF * y + 3] * blk[SVF * y + 2];
    });
    int64_t cum = 0;
    int k = 0;
    for (; k < nb && cum < D->n_sm; ++k) {
      const int64_t r = blk[SVF * order[k] + 3], G = (r + W - 1) / W;
      cum += r > 0 ? std::max<int64_t>(2, G + (G & 1)) / 2 : 0;
    }
    std::reverse(order + k, order + nb);
  };
  order_blocks(8);
  auto schedule = [&](int W, bool f32, int64_t* pre) -> Sched {
    Sched sc;
    for (;;) {
      int64_t sm = 0;
      for (int b = 0; b < nb; ++b)
        sm = std::max(sm, svd_bround_smem(W, blk[SVF * b + 2], f32 ? blk[SVF * b + 3] : 0, f32));
      if (sm <= kSvdMaxSmemHost || W == 2) { sc.smem = sm; break; }
      W /= 2;
    }
    sc.W = W;
    pre[0] = 0;
    for (int k = 0; k < nb; ++k) {
      const int64_t r = blk[SVF * order[k] + 3];
      const int64_t G = (r + W - 1) / W, Gp = std::max<int64_t>(2, G + (G & 1));
      pre[k + 1] = pre[k] + (r > 0 ? Gp / 2 : 0);
      if (r > 0) sc.rounds = std::max<int>(sc.rounds, (int)(Gp - 1));
    }
    sc.ncta = pre[nb];
    return sc;
  };
  const Sched s32 = schedule(8, true, pp.data());
  Sched s64 = schedule(8, false, pp.data() + nb + 1);
  if (s32.smem > kSvdMaxSmemHost || s64.smem > kSvdMaxSmemHost)
    return mrd_fail(ctx, MRD_E_OOM, "block SVD: a block is too large for the shared-memory Jacobi rounds");
  MRD_CUDA(ctx, D->svd_blk.need(blk.size() * 8));
  MRD_CUDA(ctx, D->svd_src.need(src_off.size() * 8));
  MRD_CUDA(ctx, D->svd_pref.need(pp.size() * 8));
  MRD_CUDA(ctx, D->svd_work.need((size_t)work * 16));
  MRD_CUDA(ctx, D->svd_w32.need((size_t)std::max<int64_t>(w32, 1) * 8));
  MRD_CUDA(ctx, D->svd_x2.need((size_t)std::max<int64_t>(xlen, 1) * 16));
  MRD_CUDA(ctx, D->svd_u.need((size_t)ulen * 16));
  MRD_CUDA(ctx, D->svd_vh.need((size_t)vlen * 16));
  MRD_CUDA(ctx, D->svd_s.need((size_t)slen * 8));
  MRD_CUDA(ctx, D->svd_ss.need((size_t)slen * 8));
  MRD_CUDA(ctx, D->svd_ord.need((size_t)slen * 4));
  MRD_CUDA(ctx, D->svd_flat.need((size_t)slen * 4));
  MRD_CUDA(ctx, D->svd_last.need((size_t)std::max<int64_t>(slen, 1) * 4));
  MRD_CUDA(ctx, D->svd_keep.need((size_t)nb * 4));
  MRD_CUDA(ctx, D->svd_info.need(4 * 8));
  MRD_CUDA(ctx, D->svd_fro.need((size_t)nb * 8));
  MRD_CUDA(ctx, cudaMemcpyAsync(D->svd_blk.p, blk.data(), blk.size() * 8, cudaMemcpyHostToDevice, s));
  MRD_CUDA(ctx, cudaMemcpyAsync(D->svd_src.p, src_off.data(), src_off.size() * 8, cudaMemcpyHostToDevice, s));
  MRD_CUDA(ctx, cudaMemcpyAsync(D->svd_pref.p, pp.data(), pp.size() * 8, cudaMemcpyHostToDevice, s));
  const int64_t* dblk = D->svd_blk.as<int64_t>();
  const double* fro = D->svd_fro.as<double>();
  MRD_CUDA(ctx, svd_load(src, dblk, D->svd_src.as<int64_t>(), nb, D->svd_work.as<double2>(), D->svd_fro.as<double>(), s));
  const int64_t* pre32 = D->svd_pref.as<int64_t>();
  const int64_t* pre64 = pre32 + nb + 1;
  const int64_t* ord = pre32 + 2 * (nb + 1);
  // per phase: the rounds' time (events around the sweeps) and work (element-pairs tested and
  // rotated, counted by the kernels), reported by mrd_dmrg_svd_stats
  if (!D->svd_ev[0]) {
    MRD_CUDA(ctx, cudaEventCreate(&D->svd_ev[0]));
    MRD_CUDA(ctx, cudaEventCreate(&D->svd_ev[1]));
  }
  MRD_CUDA(ctx, D->svd_ctr.need(2 * 8));
  for (double& v : D->svd_stats) v = 0.0;
  D->svd_stats[5] = mode;
  auto sweep_until_done = [&](bool f32, int max_sweeps, int* used) -> int {
    const Sched& sc = f32 ? s32 : s64;
    const bool ff = mode == MRD_SVD_F32_FF || mode == MRD_SVD_FF;
    int* last = D->svd_last.as<int>();
    unsigned long long* wctr = D->svd_ctr.as<unsigned long long>();
    MRD_CUDA(ctx, cudaMemsetAsync(last, 0, (size_t)slen * 4, s));
    MRD_CUDA(ctx, cudaMemsetAsync(wctr, 0, 2 * 8, s));
    MRD_CUDA(ctx, cudaEventRecord(D->svd_ev[0], s));
    bool done = false;
    std::vector<int32_t>& trace = f32 ? D->svd_trace32 : D->svd_trace64;
    std::vector<double>& tms = f32 ? D->svd_tms32 : D->svd_tms64;
    trace.clear();
    tms.clear();
    // One rotation counter per sweep. Sweep s + 1 is enqueued before the host reads sweep s's
    // count (from pinned memory, after an event), so the device runs on while the host waits;
    // a sweep whose predecessor rotated nothing returns at once (the kernels check).
    MRD_CUDA(ctx, D->svd_rotv.need((size_t)(max_sweeps + 1) * 4));
    int* rotv = D->svd_rotv.as<int>();
    MRD_CUDA(ctx, cudaMemsetAsync(rotv, 0, (size_t)(max_sweeps + 1) * 4, s));
    if (!D->svd_hcnt) MRD_CUDA(ctx, cudaHostAlloc((void**)&D->svd_hcnt, 4 * (kMaxSweeps64 + 65), cudaHostAllocDefault));
    for (cudaEvent_t& ev : D->svd_sev)
      if (!ev) MRD_CUDA(ctx, cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
    auto enqueue_sweep = [&](int sweep) -> int {
      const int* prev = sweep > 0 ? rotv + sweep - 1 : nullptr;
      for (int rd = 0; rd < sc.rounds; ++rd) {
        if (f32)
          MRD_CUDA(ctx, svd_bround32(D->svd_w32.as<float2>(), dblk, pre32, ord, nb, sc.ncta, rd, sc.W, sc.smem, 1e-5f,
                                     fro, rotv + sweep, last, sweep, wctr, prev, D->real, s));
        else
          MRD_CUDA(ctx, svd_bround(D->svd_work.as<double2>(), ff ? D->svd_x2.as<float4>() : nullptr, dblk, pre64, ord, nb,
                                   sc.ncta, rd, sc.W, sc.smem, ff ? kTolFF : kTolF64, fro, rotv + sweep, last, sweep,
                                   wctr, prev, D->real, s));
      }
      MRD_CUDA(ctx, cudaMemcpyAsync(D->svd_hcnt + sweep, rotv + sweep, 4, cudaMemcpyDeviceToHost, s));
      MRD_CUDA(ctx, cudaEventRecord(D->svd_sev[sweep & 1], s));
      return MRD_OK;
    };
    MRD_CUDA(ctx, cudaStreamSynchronize(s));
    auto t_last = std::chrono::steady_clock::now();
    int rc0 = max_sweeps > 0 ? enqueue_sweep(0) : MRD_OK;
    if (rc0 != MRD_OK) return rc0;
    for (int sweep = 0; sweep < max_sweeps && !done; ++sweep) {
      if (sweep + 1 < max_sweeps && (rc0 = enqueue_sweep(sweep + 1)) != MRD_OK) return rc0;
      MRD_CUDA(ctx, cudaEventSynchronize(D->svd_sev[sweep & 1]));
      const int hrot = D->svd_hcnt[sweep];
      *used = sweep + 1;
      trace.push_back(hrot);
      const auto t_now = std::chrono::steady_clock::now();
      tms.push_back(std::chrono::duration<double, std::milli>(t_now - t_last).count());
      t_last = t_now;
      done = hrot == 0;
    }
    MRD_CUDA(ctx, cudaEventRecord(D->svd_ev[1], s));
    unsigned long long cnt[2] = {0, 0};
    MRD_CUDA(ctx, cudaMemcpyAsync(cnt, wctr, 2 * 8, cudaMemcpyDeviceToHost, s));
    MRD_CUDA(ctx, cudaStreamSynchronize(s));
    float ms = 0.f;
    MRD_CUDA(ctx, cudaEventElapsedTime(&ms, D->svd_ev[0], D->svd_ev[1]));
    if (f32) {
      D->svd_stats[4] = ms;
    } else {
      D->svd_stats[0] = ms;
      D->svd_stats[1] = (double)cnt[0];
      D->svd_stats[2] = (double)cnt[1];
      D->svd_stats[3] = *used;
    }
    if (done || f32) return MRD_OK;
    return mrd_fail(ctx, MRD_E_NOCONV, "block SVD: Jacobi sweeps did not converge");
  };
  // FP32 pre-sweeps (MRD_SVD_F32_*) orthogonalise the columns to ~1e-5 (the resolution of FP32
  // dot products of a few hundred terms); their rotations V32 are applied to the FP64 matrix
  // (X <- X V32, one grouped GEMM) and float-float or FP64 sweeps finish the job.
  int rc = MRD_OK;
  D->svd_sweeps32 = 0;
  D->svd_trace32.clear();
  D->svd_tms32.clear();
  D->svd_cols[0] = D->svd_cols[1] = (double)slen;
  if (mode == MRD_SVD_F32_FF || mode == MRD_SVD_F32_F64) {
  MRD_CUDA(ctx, svd_to_f32(D->svd_work.as<double2>(), D->svd_w32.as<float2>(), dblk, nb, s));
  rc = sweep_until_done(true, D->svd_presweeps, &D->svd_sweeps32);
  if (rc != MRD_OK) return rc;
  MRD_CUDA(ctx, svd_v_from_f32(D->svd_work.as<double2>(), D->svd_w32.as<float2>(), dblk, nb, s));
  {
    GemmList g;
    for (int b = 0; b < nb; ++b) {   // X_new^T (r x p) = V^T (r x r) X^T (r x p), all column-major buffers
      const int64_t* d = &blk[SVF * b];
      const int64_t p = d[2], r = d[3];
      if (p == 0 || r == 0) continue;
      g.task(r, p, d[4], p);
      g.seg(d[5], r, d[4], p, r, 0);
    }
    rc = run_gemm(D, g, D->svd_work.as<double2>(), work, D->svd_work.as<double2>(), work, D->svd_x2.as<double2>(),
                  xlen);
    if (rc != MRD_OK) return rc;
  }
  // Columns set aside before the final sweeps. After the pre-sweeps the columns of X = M V32
  // are orthogonal to ~1e-5 and their norms are the singular values to that accuracy. Only the
  // chi largest values over all blocks survive the truncation, so columns of norm below
  // kSetAsideFrac times the chi-th largest norm carry weight that is discarded in any case;
  // they are dropped from X, the final sweeps orthogonalise the remaining columns (the
  // dominant singular subspace, perturbed only through the ~1e-5 overlaps with the dropped
  // columns, a second-order change of the truncated state) and the block keeps r_act values.
  // The canonical factor stays exactly orthonormal; the other factor is the exact projection.
  // The column norms stand for singular values only once the pre-sweeps have run their default
  // budget (or converged): with fewer, no column is set aside.
  bool set_aside = false;
  int64_t cols_all = 0, cols_kept = 0;
  for (int b = 0; b < nb; ++b) cols_all += blk[SVF * b + 3];
  const bool pre_done = D->svd_sweeps32 >= kMaxSweeps32 || (!D->svd_trace32.empty() && D->svd_trace32.back() == 0);
  if (cols_all > chi && chi > 0 && pre_done) {
    MRD_CUDA(ctx, svd_colnorm2(D->svd_x2.as<double2>(), dblk, nb, D->svd_s.as<double>(), s));
    std::vector<double> nrm((size_t)slen, 0.0);
    MRD_CUDA(ctx, cudaMemcpyAsync(nrm.data(), D->svd_s.p, (size_t)slen * 8, cudaMemcpyDeviceToHost, s));
    MRD_CUDA(ctx, cudaStreamSynchronize(s));
    std::vector<double> all;
    all.reserve((size_t)cols_all);
    for (int b = 0; b < nb; ++b)
      for (int64_t j = 0; j < blk[SVF * b + 3]; ++j) all.push_back(nrm[(size_t)(blk[SVF * b + 8] + j)]);
    std::nth_element(all.begin(), all.begin() + (chi - 1), all.end(), std::greater<double>());
    const double tau2 = kSetAsideFrac * kSetAsideFrac * all[(size_t)(chi - 1)];
    std::vector<int32_t> perm((size_t)slen, 0);
    for (int b = 0; b < nb; ++b) {
      int64_t* d = &blk[SVF * b];
      int64_t k = 0;
      for (int pass = 0; pass < 2; ++pass)   // columns that stay first, then those set aside
        for (int64_t j = 0; j < d[3]; ++j)
          if ((nrm[(size_t)(d[8] + j)] >= tau2) == (pass == 0)) perm[(size_t)(d[8] + k++)] = (int32_t)j;
      int64_t act = 0;
      for (int64_t j = 0; j < d[3]; ++j) act += nrm[(size_t)(d[8] + j)] >= tau2;
      // the columns that stay by decreasing norm: groups of similar norms, which the final
      // sweeps orthogonalise in fewer sweeps (de Rijk's ordering, applied once)
      const double* nb0 = &nrm[(size_t)d[8]];
      std::stable_sort(&perm[(size_t)d[8]], &perm[(size_t)d[8]] + act,
                       [&](int32_t x, int32_t y) { return nb0[x] > nb0[y]; });
      d[3] = act;
      cols_kept += act;
    }
    MRD_CUDA(ctx, D->svd_perm.need((size_t)std::max<int64_t>(slen, 1) * 4));
    MRD_CUDA(ctx, cudaMemcpyAsync(D->svd_perm.p, perm.data(), (size_t)slen * 4, cudaMemcpyHostToDevice, s));
    MRD_CUDA(ctx, cudaMemcpyAsync(D->svd_blk.p, blk.data(), blk.size() * 8, cudaMemcpyHostToDevice, s));
    // the final sweeps' schedule on the remaining columns, largest blocks first
    order_blocks(s64.W);
    s64 = schedule(s64.W, false, pp.data() + nb + 1);
    MRD_CUDA(ctx, cudaMemcpyAsync(D->svd_pref.p, pp.data(), pp.size() * 8, cudaMemcpyHostToDevice, s));
    MRD_CUDA(ctx, svd_gather_cols(D->svd_work.as<double2>(), D->svd_x2.as<double2>(), dblk, nb,
                                  D->svd_perm.as<int>(), s));
    MRD_CUDA(ctx, cudaStreamSynchronize(s));   // host tables of the copies above leave scope
    set_aside = true;
  } else {
    cols_kept = cols_all;
    MRD_CUDA(ctx, cudaMemcpyAsync(D->svd_work.p, D->svd_x2.p, (size_t)xlen * 16, cudaMemcpyDeviceToDevice, s));
  }
  D->svd_cols[0] = (double)cols_kept;
  D->svd_cols[1] = (double)cols_all;
  (void)set_aside;
  }
  // float-float sweeps work on a float-float copy of X in svd_x2 (16 bytes per element either way)
  const bool ffm = mode == MRD_SVD_F32_FF || mode == MRD_SVD_FF;
  if (ffm) MRD_CUDA(ctx, svd_ff_io(D->svd_work.as<double2>(), D->svd_x2.as<float4>(), dblk, nb, fro, true, s));
  rc = sweep_until_done(false, kMaxSweeps64, &D->svd_sweeps64);
  if (rc != MRD_OK) return rc;
  if (ffm) MRD_CUDA(ctx, svd_ff_io(D->svd_work.as<double2>(), D->svd_x2.as<float4>(), dblk, nb, fro, false, s));
  MRD_CUDA(ctx, svd_finish(D->svd_work.as<double2>(), dblk, nb, D->svd_u.as<double2>(), D->svd_vh.as<double2>(),
                           D->svd_s.as<double>(), D->svd_ss.as<double>(), D->svd_ord.as<int>(), fro, s));
  MRD_CUDA(ctx, svd_truncate(dblk, nb, D->svd_ss.as<double>(), slen, chi, cutoff, D->svd_keep.as<int>(),
                             D->svd_info.as<double>(), D->svd_flat.as<int>(), s));
  MRD_CUDA(ctx, cudaMemcpyAsync(keep.data(), D->svd_keep.p, nb * 4, cudaMemcpyDeviceToHost, s));
  MRD_CUDA(ctx, cudaMemcpyAsync(info, D->svd_info.p, 3 * 8, cudaMemcpyDeviceToHost, s));
  MRD_CUDA(ctx, cudaStreamSynchronize(s));
  return MRD_OK;
}

// L[i+1] = A^+ (L[i] W_i) A with A = D->A[i] (mode 0) and the LW fold of h (sites i, i+1).
int env_left(mrd_dmrg* D, mrd_heff* h, int i) {
  mrd_ctx* ctx = D->ctx;
  const SiteT& A = D->A[i];
  const Secs& ls = A.left;   // bond i
  const Secs& cs = A.right;  // bond i+1
  auto cm = mpo_channels(D->mpo, i + 1, D->mod);
  const int m1 = A.m, mod = D->mod;
  // LW blocks (w', s', s, a) -> offset, in a flat index over all (w', s', s, a)
  const int64_t nls = (int64_t)ls.size(), ncs = (int64_t)cs.size(), nw = (int64_t)cm.size();
  std::vector<int64_t> lw((size_t)(nw * 4 * nls), -1);
  for (int64_t k = 0; k < h->counts[C_NLW]; ++k) {
    const int64_t* r = &h->lw_host[LWF * k];
    if (r[0] < 0 || r[0] >= nw || r[1] < 0 || r[1] > 1 || r[2] < 0 || r[2] > 1 || r[3] < 0 || r[3] >= nls)
      return mrd_fail(ctx, MRD_E_STATE, "internal: LW block outside the bond's channels or sectors");
    lw[(size_t)(((r[0] * 2 + r[1]) * 2 + r[2]) * nls + r[3])] = r[7];
  }
  // step 1: T(w', c, s') = sum_s LW(w', s', s, a) A(a, s -> c)
  GemmList g1;
  struct TB { int64_t off, rows; };
  std::vector<TB> tblk((size_t)(nw * ncs * 2), TB{-1, 0});   // (w', c, s') -> block of T
  int64_t tlen = 0;
  for (int w = 0; w < (int)cm.size(); ++w)
    for (int c = 0; c < (int)cs.size(); ++c) {
      const int cp = find_sec(cs, cs[c].N + cm[w][0], kmod(cs[c].K + cm[w][1], mod));
      if (cp < 0) continue;
      for (int sp = 0; sp < 2; ++sp) {
        const int ap = find_sec(ls, cs[cp].N - sp, kmod(cs[cp].K - sp * m1, mod));
        if (ap < 0) continue;
        bool started = false;
        for (int s = 0; s < 2; ++s) {
          const int a = find_sec(ls, cs[c].N - s, kmod(cs[c].K - s * m1, mod));
          if (a < 0) continue;
          const int64_t lwo = lw[(size_t)((((int64_t)w * 2 + sp) * 2 + s) * nls + a)];
          if (lwo < 0) continue;
          int64_t ao, ald;
          int rr;
          if (!A.subblock(a, s, &ao, &ald, &rr) || rr != c) continue;
          if (!started) {
            tblk[(size_t)(((int64_t)w * ncs + c) * 2 + sp)] = {tlen, ls[ap].d};
            g1.task(ls[ap].d, cs[c].d, tlen, cs[c].d);
            tlen += (int64_t)ls[ap].d * cs[c].d;
            started = true;
          }
          g1.seg(lwo, ls[a].d, ao, ald, ls[a].d, 0);
        }
      }
    }
  MRD_CUDA(ctx, D->tbuf.need((size_t)std::max<int64_t>(tlen, 1) * 16));
  // with float-float GEMMs T stays in float-float (the same 16 bytes per element) for step 2
  float4* t_ff = D->gemm_ff ? D->tbuf.as<float4>() : nullptr;
  int rc = run_gemm(D, g1, h->lw, h->counts[C_LWLEN], A.data.as<double2>(), A.size, D->tbuf.as<double2>(), tlen,
                    heff_ff_lw(h), nullptr, t_ff);
  if (rc != MRD_OK) return rc;
  // step 2: L'(w', c) = sum_s' A(a', s' -> c')^+ T(w', c, s')
  EnvT& E = D->L[i + 1];
  E.sec = cs;
  E.ch = cm;
  E.left = true;
  E.layout(mod);
  Buf& eout = D->env_fp32 ? D->envx[2] : E.data;   // complex128 result, rounded afterwards in FP32 storage
  MRD_CUDA(ctx, eout.need((size_t)std::max<int64_t>(E.size, 1) * 16));
  MRD_CUDA(ctx, cudaMemsetAsync(eout.p, 0, (size_t)std::max<int64_t>(E.size, 1) * 16, ctx->stream));
  GemmList g2;
  for (int w = 0; w < (int)cm.size(); ++w)
    for (int c = 0; c < (int)cs.size(); ++c) {
      const int64_t off = E.off[(size_t)w * cs.size() + c];
      if (off < 0) continue;
      const int cp = find_sec(cs, cs[c].N + cm[w][0], kmod(cs[c].K + cm[w][1], mod));
      bool started = false;
      for (int sp = 0; sp < 2; ++sp) {
        const TB& tb = tblk[(size_t)(((int64_t)w * ncs + c) * 2 + sp)];
        if (tb.off < 0) continue;
        const int ap = find_sec(ls, cs[cp].N - sp, kmod(cs[cp].K - sp * m1, mod));
        int64_t ao, ald;
        int rr;
        if (!A.subblock(ap, sp, &ao, &ald, &rr) || rr != cp) continue;
        if (!started) { g2.task(cs[cp].d, cs[c].d, off, cs[c].d); started = true; }
        // A-op: conj-transpose of the d_a' x d_c' sub-block
        g2.seg(ao, ald, tb.off, cs[c].d, ls[ap].d, 1);
      }
    }
  rc = run_gemm(D, g2, A.data.as<double2>(), A.size, D->tbuf.as<double2>(), tlen, eout.as<double2>(), E.size, nullptr,
                t_ff);
  if (rc != MRD_OK) return rc;
  return env_store(D, E, eout.as<double2>());
}

// R[i+1] = B (W_{i+1} R[i+2]) B^+ with B = D->A[i+1] (mode 1) and the WR fold of h.
int env_right(mrd_dmrg* D, mrd_heff* h, int i) {
  mrd_ctx* ctx = D->ctx;
  const SiteT& B = D->A[i + 1];
  const Secs& cs = B.left;   // bond i+1
  const Secs& bs = B.right;  // bond i+2
  auto cm = mpo_channels(D->mpo, i + 1, D->mod);
  const int m2 = B.m, mod = D->mod;
  // WR blocks (w', s, s', b) -> offset, in a flat index over all (w', s, s', b)
  const int64_t nbs = (int64_t)bs.size(), ncs = (int64_t)cs.size(), nw = (int64_t)cm.size();
  std::vector<int64_t> wr((size_t)(nw * 4 * nbs), -1);
  for (int64_t k = 0; k < h->counts[C_NWR]; ++k) {
    const int64_t* r = &h->wr_host[WRF * k];
    if (r[0] < 0 || r[0] >= nw || r[1] < 0 || r[1] > 1 || r[2] < 0 || r[2] > 1 || r[3] < 0 || r[3] >= nbs)
      return mrd_fail(ctx, MRD_E_STATE, "internal: WR block outside the bond's channels or sectors");
    wr[(size_t)(((r[0] * 2 + r[1]) * 2 + r[2]) * nbs + r[3])] = r[7];
  }
  // step 1: T(w', c, s') = sum_s B(c, s -> b) WR(w', s, s', b)
  GemmList g1;
  struct TB { int64_t off, cols; };
  std::vector<TB> tblk((size_t)(nw * ncs * 2), TB{-1, 0});   // (w', c, s') -> block of T
  int64_t tlen = 0;
  for (int w = 0; w < (int)cm.size(); ++w)
    for (int c = 0; c < (int)cs.size(); ++c) {
      const int cp = find_sec(cs, cs[c].N + cm[w][0], kmod(cs[c].K + cm[w][1], mod));
      if (cp < 0) continue;
      for (int sp = 0; sp < 2; ++sp) {
        const int bp = find_sec(bs, cs[cp].N + sp, kmod(cs[cp].K + sp * m2, mod));
        if (bp < 0) continue;
        bool started = false;
        for (int s = 0; s < 2; ++s) {
          int64_t bo, bld;
          int b;
          if (!B.subblock(c, s, &bo, &bld, &b)) continue;
          const int64_t wro = wr[(size_t)((((int64_t)w * 2 + s) * 2 + sp) * nbs + b)];
          if (wro < 0) continue;
          if (!started) {
            tblk[(size_t)(((int64_t)w * ncs + c) * 2 + sp)] = {tlen, bs[bp].d};
            g1.task(cs[c].d, bs[bp].d, tlen, bs[bp].d);
            tlen += (int64_t)cs[c].d * bs[bp].d;
            started = true;
          }
          g1.seg(bo, bld, wro, bs[bp].d, bs[b].d, 0);
        }
      }
    }
  MRD_CUDA(ctx, D->tbuf.need((size_t)std::max<int64_t>(tlen, 1) * 16));
  float4* t_ff = D->gemm_ff ? D->tbuf.as<float4>() : nullptr;   // T in float-float for step 2
  int rc = run_gemm(D, g1, B.data.as<double2>(), B.size, h->wr, h->counts[C_WRLEN], D->tbuf.as<double2>(), tlen,
                    nullptr, heff_ff_wr(h), t_ff);
  if (rc != MRD_OK) return rc;
  EnvT& E = D->R[i + 1];
  E.sec = cs;
  E.ch = cm;
  E.left = false;
  E.layout(mod);
  Buf& eout = D->env_fp32 ? D->envx[2] : E.data;   // complex128 result, rounded afterwards in FP32 storage
  MRD_CUDA(ctx, eout.need((size_t)std::max<int64_t>(E.size, 1) * 16));
  MRD_CUDA(ctx, cudaMemsetAsync(eout.p, 0, (size_t)std::max<int64_t>(E.size, 1) * 16, ctx->stream));
  GemmList g2;
  for (int w = 0; w < (int)cm.size(); ++w)
    for (int c = 0; c < (int)cs.size(); ++c) {
      const int64_t off = E.off[(size_t)w * cs.size() + c];
      if (off < 0) continue;
      const int cp = find_sec(cs, cs[c].N + cm[w][0], kmod(cs[c].K + cm[w][1], mod));
      bool started = false;
      for (int sp = 0; sp < 2; ++sp) {
        const TB& tb = tblk[(size_t)(((int64_t)w * ncs + c) * 2 + sp)];
        if (tb.off < 0) continue;
        int64_t bo, bld;
        int bp;
        if (!B.subblock(cp, sp, &bo, &bld, &bp)) continue;
        if (!started) { g2.task(cs[c].d, cs[cp].d, off, cs[cp].d); started = true; }
        // B-op: conj-transpose of the d_c' x d_b' sub-block
        g2.seg(tb.off, tb.cols, bo, bld, bs[bp].d, 2);
      }
    }
  rc = run_gemm(D, g2, D->tbuf.as<double2>(), tlen, B.data.as<double2>(), B.size, eout.as<double2>(), E.size, t_ff);
  if (rc != MRD_OK) return rc;
  return env_store(D, E, eout.as<double2>());
}

int set_trivial_env(mrd_dmrg* D, EnvT& E, const Secs& sec, int bond, bool left) {
  E.sec = sec;
  E.ch = mpo_channels(D->mpo, bond, D->mod);
  E.left = left;
  E.layout(D->mod);
  if (E.size != 1) return mrd_fail(D->ctx, MRD_E_STATE, "boundary environment is not 1 x 1");
  E.f32 = false;
  MRD_CUDA(D->ctx, E.data.need(16));
  const double2 one = make_double2(1.0, 0.0);
  MRD_CUDA(D->ctx, cudaMemcpy(E.data.p, &one, 16, cudaMemcpyHostToDevice));
  return MRD_OK;
}

// Right-orthonormalise the rows of every group of a mode-1 tensor (or the columns of every
// group of a mode-0 tensor) with the block SVD; the data is replaced by V^+ (or U).
int orthonormalise(mrd_dmrg* D, SiteT& T) {
  std::vector<int64_t> blk, src;
  std::vector<int> gi;
  for (size_t g = 0; g < T.goff.size(); ++g) {
    const int64_t rows = T.mode == 1 ? T.left[g].d : T.gext[g];
    const int64_t cols = T.mode == 1 ? T.gext[g] : T.right[g].d;
    if (rows == 0 || cols == 0) continue;
    std::vector<int64_t> d(SVF, 0);
    d[0] = rows; d[1] = cols;
    blk.insert(blk.end(), d.begin(), d.end());
    src.push_back(T.goff[g]);
    gi.push_back((int)g);
  }
  std::vector<int> keep;
  double info[3];
  int rc = block_svd(D, blk, src, T.data.as<double2>(), T.mode == 1 ? 1 : 0, 1 << 30, 0.0, MRD_SVD_FF, keep, info);
  if (rc != MRD_OK) return rc;
  // The factor replaces the tensor without its partner (S V^+ or U S is not carried to the
  // neighbour), so the phase of each singular vector would enter the state: fix it by a
  // convention, which makes the orthonormalised state independent of the Jacobi rotation order.
  MRD_CUDA(D->ctx, svd_fix_phases(D->svd_u.as<double2>(), D->svd_vh.as<double2>(), D->svd_blk.as<int64_t>(),
                                  (int)gi.size(), T.mode == 1 ? 1 : 0, D->ctx->stream));
  std::vector<int64_t> cp;
  for (size_t b = 0; b < gi.size(); ++b) {
    const int64_t* d = &blk[SVF * b];
    const int g = gi[b];
    if (T.mode == 1) {   // rows of Vh: r = min(rows, cols) must equal rows
      if (d[3] != d[0]) return mrd_fail(D->ctx, MRD_E_STATE, "orthonormalise: rank-deficient group");
      cp.insert(cp.end(), {d[7], d[1], T.goff[g], T.gext[g], d[0], d[1], 0, 0});
    } else {
      if (d[3] != d[1]) return mrd_fail(D->ctx, MRD_E_STATE, "orthonormalise: rank-deficient group");
      cp.insert(cp.end(), {d[6], d[3], T.goff[g], T.right[g].d, d[0], d[1], 0, 0});
    }
  }
  return run_copies(D, cp, T.mode == 1 ? D->svd_vh.as<double2>() : D->svd_u.as<double2>(), T.data.as<double2>(),
                    nullptr, nullptr);
}

// Orthonormalise every tensor but the centre's (left of it left-canonical, right of it
// right-canonical) and build the left environments up to the centre and the right ones down to
// centre + 2 (the initial state of mrd_dmrg_create, or its real-valued version).
int canonicalise_and_build_envs(mrd_dmrg* D, int center) {
  const int n = D->n;
  int rcd = MRD_OK;
  for (int j = 0; j < n && rcd == MRD_OK; ++j)
    if (j != center) rcd = orthonormalise(D, D->A[j]);
  if (rcd == MRD_OK) rcd = set_trivial_env(D, D->L[0], D->A[0].left, 0, true);
  if (rcd == MRD_OK) rcd = set_trivial_env(D, D->R[n], D->A[n - 1].right, n, false);
  for (int j = 0; j < center && rcd == MRD_OK; ++j) {
    mrd_heff* h = nullptr;
    const double2* lj = nullptr;
    rcd = env_fp64(D, D->L[j], 0, &lj);
    if (rcd == MRD_OK) rcd = make_heff(D, j, lj, nullptr, &h);
    if (rcd == MRD_OK) rcd = env_left(D, h, j);
    if (h) mrd_heff_free(h);
  }
  for (int j = n - 1; j >= center + 2 && rcd == MRD_OK; --j) {
    mrd_heff* h = nullptr;
    const double2* rj = nullptr;
    rcd = env_fp64(D, D->R[j + 1], 1, &rj);
    if (rcd == MRD_OK) rcd = make_heff(D, j - 1, nullptr, rj, &h);
    if (rcd == MRD_OK) rcd = env_right(D, h, j - 1);
    if (h) mrd_heff_free(h);
  }
  return rcd;
}

}  // namespace

extern "C" {

int mrd_dmrg_create(mrd_ctx* ctx, const mrd_mpo* mpo, int32_t n_part, int32_t k_tot, int32_t chi, uint64_t seed,
                    int32_t center, const int32_t* caps, const int64_t* caps_off, mrd_dmrg** out) try {
  if (!ctx || !mpo || !out || chi < 1) return mrd_fail(ctx, MRD_E_ARG, "mrd_dmrg_create: bad argument");
  *out = nullptr;
  const HostMPO& H = mpo->h;
  const int n = H.n_sites;
  if (n < 2 || center < 0 || center > n - 2) return mrd_fail(ctx, MRD_E_ARG, "mrd_dmrg_create: need n >= 2, 0 <= center <= n-2");
  if (H.bond_charges[0].size() != 2 || H.bond_charges[n].size() != 2)
    return mrd_fail(ctx, MRD_E_ARG, "mrd_dmrg_create: MPO boundary bonds must have dimension 1");
  Guard g(ctx->device);
  mrd_dmrg* D = new mrd_dmrg();
  D->ctx = ctx;
  mrd_ctx_retain(ctx);
  D->mpo = H;
  D->n = n;
  D->mod = H.modulus;
  // ly: the site momentum period (orbital j has momentum j mod ly in the mixed basis)
  D->ly = H.modulus > 1 ? H.modulus : 1;
  D->target_N = n_part;
  D->target_K = kmod(k_tot, D->mod);
  cudaDeviceGetAttribute(&D->n_sm, cudaDevAttrMultiProcessorCount, ctx->device);
  const int mod = D->mod;
  auto site_m = [&](int j) { return mod > 1 ? j % D->ly : 0; };
  // exact state counts left and right of every bond (log scale to avoid overflow)
  std::vector<std::map<int64_t, double>> lc(n + 1), rc(n + 1);
  lc[0][qkey(0, 0)] = 0.0;
  for (int j = 0; j < n; ++j)
    for (auto& kv : lc[j]) {
      const int N = (int)((kv.first >> 32) - (1 << 29)), K = (int)(kv.first & 0xffffffff);
      for (int s = 0; s < 2; ++s) {
        const int64_t k2 = qkey(N + s, kmod(K + s * site_m(j), mod));
        auto it = lc[j + 1].find(k2);
        if (it == lc[j + 1].end()) lc[j + 1][k2] = kv.second;
        else it->second = std::max(it->second, kv.second) + std::log1p(std::exp(-std::fabs(it->second - kv.second)));
      }
    }
  rc[n][qkey(n_part, D->target_K)] = 0.0;
  for (int j = n - 1; j >= 0; --j)
    for (auto& kv : rc[j + 1]) {
      const int N = (int)((kv.first >> 32) - (1 << 29)), K = (int)(kv.first & 0xffffffff);
      for (int s = 0; s < 2; ++s) {
        const int64_t k2 = qkey(N - s, kmod(K - s * site_m(j), mod));
        auto it = rc[j].find(k2);
        if (it == rc[j].end()) rc[j][k2] = kv.second;
        else it->second = std::max(it->second, kv.second) + std::log1p(std::exp(-std::fabs(it->second - kv.second)));
      }
    }
  if (!lc[n].count(qkey(n_part, D->target_K))) {
    mrd_dmrg_free(D);
    return mrd_fail(ctx, MRD_E_CHARGE, "mrd_dmrg_create: target charge unreachable");
  }
  // bond sectors: exact counts, capped by the caller's caps (if given) and by chi
  std::vector<Secs> bond(n + 1);
  for (int j = 0; j <= n; ++j) {
    std::map<int64_t, int> capmap;
    const bool has_cap = caps && caps_off && caps_off[j + 1] > caps_off[j];
    if (has_cap)
      for (int64_t k = caps_off[j]; k < caps_off[j + 1]; ++k)
        capmap[qkey(caps[3 * k], kmod(caps[3 * k + 1], mod))] = caps[3 * k + 2];
    for (auto& kv : lc[j]) {
      auto r = rc[j].find(kv.first);
      if (r == rc[j].end()) continue;
      double lim = std::min(kv.second, r->second);   // log of the exact dimension bound
      int64_t d = lim > 40 ? (int64_t)1 << 40 : (int64_t)std::llround(std::exp(lim));
      d = std::min<int64_t>(d, chi);
      if (has_cap) {
        auto c = capmap.find(kv.first);
        d = c == capmap.end() ? 0 : std::min<int64_t>(d, c->second);
      }
      if (d <= 0) continue;
      const int N = (int)((kv.first >> 32) - (1 << 29)), K = (int)(kv.first & 0xffffffff);
      bond[j].push_back({N, K, (int32_t)d});
    }
    if (!has_cap) {   // keep the total at most chi: scale down proportionally (at least 1 each)
      int64_t tot = 0;
      for (auto& s : bond[j]) tot += s.d;
      if (tot > chi) {
        for (auto& s : bond[j]) s.d = std::max<int32_t>(1, (int32_t)((double)s.d * chi / tot));
      }
    }
  }
  // the dims must be realisable from both sides: shrink until every sector fits its
  // neighbours (d_j(q) <= sum_s d_{j+1}(q + q(s)) and <= sum_s d_{j-1}(q - q(s)))
  for (int pass = 0, changed = 1; changed && pass < 1000; ++pass) {
    changed = 0;
    for (int j = 1; j < n; ++j) {
      for (auto& s : bond[j]) {
        int64_t right = 0, left = 0;
        for (int t = 0; t < 2; ++t) {
          const int r = find_sec(bond[j + 1], s.N + t, kmod(s.K + t * site_m(j), mod));
          if (r >= 0) right += bond[j + 1][r].d;
          const int l = find_sec(bond[j - 1], s.N - t, kmod(s.K - t * site_m(j - 1), mod));
          if (l >= 0) left += bond[j - 1][l].d;
        }
        const int32_t nd = (int32_t)std::min<int64_t>(s.d, std::min(left, right));
        if (nd != s.d) { s.d = nd; changed = 1; }
      }
      bond[j].erase(std::remove_if(bond[j].begin(), bond[j].end(), [](const Sec& s) { return s.d <= 0; }), bond[j].end());
    }
  }
  D->A.resize(n);
  D->L.resize(n + 1);
  D->R.resize(n + 1);
  cudaStream_t s = ctx->stream;
  for (int j = 0; j < n; ++j) {
    SiteT& T = D->A[j];
    T.left = bond[j];
    T.right = bond[j + 1];
    T.m = site_m(j);
    T.mod = mod;
    T.mode = j < center ? 0 : 1;
    T.layout();
    cudaError_t e = T.data.need((size_t)std::max<int64_t>(T.size, 1) * 16);
    if (e != cudaSuccess) { mrd_dmrg_free(D); return mrd_cuda_fail(ctx, e, "mrd_dmrg_create: MPS"); }
    if (T.size > 0) {
      const int64_t grid = std::min<int64_t>((T.size + 255) / 256, 4096);
      k_fill_random<<<(unsigned)grid, 256, 0, s>>>(T.data.as<double2>(), T.size, seed * 0x100000001B3ull + (uint64_t)j * 0x9E3779B97F4A7C15ull);
      mrd::count_launch();
    }
  }
  D->center0 = center;
  int rcd = canonicalise_and_build_envs(D, center);
  if (rcd != MRD_OK) {
    std::string msg = ctx->err;
    mrd_dmrg_free(D);
    return mrd_fail(ctx, rcd, msg);
  }
  *out = D;
  return MRD_OK;
} catch (...) {   // host memory or threads exhausted: no exception crosses the C ABI
  return MRD_E_HOST;
}

int mrd_dmrg_free(mrd_dmrg* D) try {
  if (!D) return MRD_OK;
  mrd_ctx* ctx = D->ctx;
  {
    Guard g(ctx->device);
    cudaStreamSynchronize(ctx->stream);
    for (cudaEvent_t e : D->svd_ev)
      if (e) cudaEventDestroy(e);
    for (cudaEvent_t e : D->svd_sev)
      if (e) cudaEventDestroy(e);
    if (D->svd_hcnt) cudaFreeHost(D->svd_hcnt);
    delete D;
  }
  mrd_ctx_release(ctx);
  return MRD_OK;
} catch (...) {   // host memory or threads exhausted: no exception crosses the C ABI
  return MRD_E_HOST;
}

int mrd_two_site_update(mrd_dmrg* D, int32_t i, int32_t direction, const mrd_dmrg_params* p, double* energy,
                        double* trunc_err) try {
  if (!D || !p) return MRD_E_ARG;
  mrd_ctx* ctx = D->ctx;
  if (i < 0 || i > D->n - 2) return mrd_fail(ctx, MRD_E_ARG, "mrd_two_site_update: site out of range");
  if (p->svd_mode < MRD_SVD_F32_FF || p->svd_mode > MRD_SVD_F64)
    return mrd_fail(ctx, MRD_E_ARG, "mrd_two_site_update: unknown svd_mode");
  if (p->refine_prec != MRD_PREC_FP64 && p->refine_prec != MRD_PREC_FF)
    return mrd_fail(ctx, MRD_E_ARG, "mrd_two_site_update: refine_prec must be MRD_PREC_FP64 or MRD_PREC_FF");
  if (p->prec < MRD_PREC_FP64 || p->prec > MRD_PREC_FF)
    return mrd_fail(ctx, MRD_E_ARG, "mrd_two_site_update: unknown prec");
  D->gemm_ff = p->refine_prec == MRD_PREC_FF;
  if (!D->L[i].data.p || !D->R[i + 2].data.p)
    return mrd_fail(ctx, MRD_E_STATE, "mrd_two_site_update: environments of this bond are not available");
  Guard g(ctx->device);
  using clk = std::chrono::steady_clock;
  auto t0 = clk::now();
  auto lap = [&](int k) {
    cudaStreamSynchronize(ctx->stream);
    auto t1 = clk::now();
    D->phase_ms[k] = std::chrono::duration<double, std::milli>(t1 - t0).count();
    t0 = t1;
  };
  mrd_heff* h = nullptr;
  const double2 *le = nullptr, *re = nullptr;
  int rc = env_fp64(D, D->L[i], 0, &le);
  if (rc == MRD_OK) rc = env_fp64(D, D->R[i + 2], 1, &re);
  if (rc == MRD_OK) rc = make_heff(D, i, le, re, &h);
  if (rc != MRD_OK) return rc;
  struct Free { mrd_heff* h; ~Free() { if (h) mrd_heff_free(h); } } guard{h};
  ++D->updates;
  if (D->real && (rc = mrd_heff_set_option(h, MRD_OPT_REAL, 1)) != MRD_OK) return rc;
  if (D->timing) mrd_heff_timing(h, 1);
  // the tensor-core tables of the Lanczos matvecs are host work: built on a host thread while
  // the device folds the environments, forms theta and converts the refinement's operands
  const bool tc = p->prec == MRD_PREC_TF32 || p->prec == MRD_PREC_BF16X3;
  if (tc) tc_prebuild(h, p->prec);
  auto collect = [&](int which) {
    if (!D->timing) return;
    double a = 0, b = 0;
    int32_t n = 0;
    mrd_heff_timing_collect(h, &a, &b, &n);
    D->kms[2 * which] += a;
    D->kms[2 * which + 1] += b;
    D->kcount[which] += n;
  };
  lap(0);
  const int64_t n = h->counts[C_THETA];
  MRD_CUDA(ctx, D->theta.need((size_t)std::max<int64_t>(n, 1) * 16));
  double2* theta = D->theta.as<double2>();
  if ((rc = form_theta(D, h, D->A[i], D->A[i + 1], theta)) != MRD_OK) return rc;
  lap(1);
  double e = 0.0;
  int32_t it = 0;
  if (tc && p->refine_iter > 0 && p->refine_prec == MRD_PREC_FF && (rc = heff_prefetch_ff(h)) != MRD_OK) return rc;
  if ((rc = mrd_lanczos(h, (double*)theta, p->lanczos_max_iter, p->lanczos_tol, p->prec, &e, &it)) != MRD_OK) return rc;
  D->last_iters = it;
  for (int r = 0; r < p->lanczos_restarts && it == p->lanczos_max_iter; ++r) {
    double e2 = 0.0;
    if ((rc = mrd_lanczos(h, (double*)theta, p->lanczos_max_iter, p->lanczos_tol, p->prec, &e2, &it)) != MRD_OK)
      return rc;
    D->last_iters += it;
    const bool done = std::fabs(e2 - e) < p->lanczos_tol * std::fabs(e2);
    e = e2;
    if (done) break;
  }
  collect(p->prec == MRD_PREC_FP64 || p->prec == MRD_PREC_FF ? 1 : 0);
  D->last_refine = 0;
  if ((p->prec == MRD_PREC_TF32 || p->prec == MRD_PREC_BF16X3) && p->refine_iter > 0) {
    int32_t it2 = 0;
    if ((rc = mrd_lanczos(h, (double*)theta, p->refine_iter, p->refine_tol, p->refine_prec, &e, &it2)) != MRD_OK)
      return rc;
    D->last_refine = it2;
  }
  collect(1);
  lap(2);
  // block SVD of theta by middle charge
  std::vector<int64_t> blk, src;
  std::vector<int> mids;
  for (int64_t q = 0; q < h->counts[C_NMID]; ++q) {
    const int64_t* r = &h->mid_host[MIDF * q];
    std::vector<int64_t> d(SVF, 0);
    d[0] = r[2]; d[1] = r[3];
    blk.insert(blk.end(), d.begin(), d.end());
    src.push_back(r[4]);
    mids.push_back((int)q);
  }
  std::vector<int> keep;
  double info[3];
  const int side = direction > 0 ? 0 : 1;   // the factor that stays in canonical form
  if ((rc = block_svd(D, blk, src, theta, side, p->chi, p->svd_cutoff, p->svd_mode, keep, info)) != MRD_OK) return rc;
  lap(3);
  // new bond i+1
  Secs nb;
  for (size_t b = 0; b < mids.size(); ++b)
    if (keep[b] > 0) {
      const int64_t* r = &h->mid_host[MIDF * mids[b]];
      nb.push_back({(int32_t)r[0], (int32_t)r[1], keep[b]});
    }
  if (nb.empty()) return mrd_fail(ctx, MRD_E_NAN, "mrd_two_site_update: all singular values vanished");
  SiteT& X = D->A[i];
  SiteT& Y = D->A[i + 1];
  X.right = nb; X.mode = 0; X.layout();
  Y.left = nb; Y.mode = 1; Y.layout();
  MRD_CUDA(ctx, X.data.need((size_t)std::max<int64_t>(X.size, 1) * 16));
  MRD_CUDA(ctx, Y.data.need((size_t)std::max<int64_t>(Y.size, 1) * 16));
  // canonical factor: copy of the orthonormal singular vectors; the other factor: exact
  // projection of theta (U^+ theta moving right, theta V moving left), then renormalised
  std::vector<int64_t> cp;
  GemmList proj;
  int nbi = 0;
  for (size_t b = 0; b < mids.size(); ++b) {
    if (keep[b] == 0) continue;
    const int64_t* d = &blk[SVF * b];
    const int64_t m = d[0], ncol = d[1], r = d[3], k = keep[b];
    if (direction > 0) {
      cp.insert(cp.end(), {d[6], r, X.goff[nbi], k, m, k, 0, 0});                 // A_i = U[:, :k]
      proj.task(k, ncol, Y.goff[nbi], Y.gext[nbi]);                                  // M_{i+1} = U_k^+ theta_q
      proj.seg(d[6], r, src[b], ncol, m, 1);
    } else {
      cp.insert(cp.end(), {d[7], ncol, Y.goff[nbi], Y.gext[nbi], k, ncol, 0, 0}); // B_{i+1} = V^+[:k, :]
      proj.task(m, k, X.goff[nbi], k);                                               // M_i = theta_q V_k
      proj.seg(src[b], ncol, d[7], ncol, ncol, 2);
    }
    ++nbi;
  }
  SiteT& canon = direction > 0 ? X : Y;
  SiteT& centre = direction > 0 ? Y : X;
  if ((rc = run_copies(D, cp, direction > 0 ? D->svd_u.as<double2>() : D->svd_vh.as<double2>(),
                       canon.data.as<double2>(), nullptr, nullptr)) != MRD_OK)
    return rc;
  const int64_t svd_ulen = D->svd_u.bytes / 16, svd_vlen = D->svd_vh.bytes / 16;
  if (direction > 0)
    rc = run_gemm(D, proj, D->svd_u.as<double2>(), svd_ulen, theta, n, centre.data.as<double2>(), centre.size);
  else
    rc = run_gemm(D, proj, theta, n, D->svd_vh.as<double2>(), svd_vlen, centre.data.as<double2>(), centre.size);
  if (rc != MRD_OK) return rc;
  if (centre.size > 0) {
    MRD_CUDA(ctx, D->svd_x2.need((size_t)kNormParts * 8));
    k_sumsq_partial<<<kNormParts, 256, 0, ctx->stream>>>(centre.data.as<double2>(), centre.size,
                                                         D->svd_x2.as<double>());
    mrd::count_launch();
    k_scale_unit<<<(unsigned)std::min<int64_t>((centre.size + 255) / 256, 4096), 256, 0, ctx->stream>>>(
        centre.data.as<double2>(), centre.size, D->svd_x2.as<double>(), D->svd_fro.as<double>(), (int)mids.size(),
        D->svd_info.as<double>());
    mrd::count_launch();
    MRD_CUDA(ctx, cudaGetLastError());
    MRD_CUDA(ctx, cudaMemcpyAsync(info, D->svd_info.p, 2 * 8, cudaMemcpyDeviceToHost, ctx->stream));
  }
  {
    // Schmidt values of the new bond i+1
    std::vector<int64_t> tab;
    int64_t nvals = 0;
    int nbi = 0;
    for (size_t b = 0; b < mids.size(); ++b) {
      if (keep[b] == 0) continue;
      const int64_t* d = &blk[SVF * b];
      const int64_t k = keep[b];
      if (direction > 0) tab.insert(tab.end(), {Y.goff[nbi], k, d[1], Y.gext[nbi], 1, nvals});
      else tab.insert(tab.end(), {X.goff[nbi], k, d[0], k, 0, nvals});
      nvals += k;
      ++nbi;
    }
    MRD_CUDA(ctx, D->schmidt_tab.need(std::max<size_t>(tab.size(), 1) * 8));
    MRD_CUDA(ctx, D->schmidt_out.need((size_t)std::max<int64_t>(nvals, 1) * 8));
    D->schmidt_val.assign(nvals, 0.0);
    if (nbi > 0) {
      MRD_CUDA(ctx, cudaMemcpyAsync(D->schmidt_tab.p, tab.data(), tab.size() * 8, cudaMemcpyHostToDevice, ctx->stream));
      k_schmidt<<<nbi, 128, 0, ctx->stream>>>(centre.data.as<double2>(), D->schmidt_tab.as<int64_t>(), nbi,
                                              D->schmidt_out.as<double>());
      mrd::count_launch();
      MRD_CUDA(ctx, cudaGetLastError());
      MRD_CUDA(ctx, cudaMemcpyAsync(D->schmidt_val.data(), D->schmidt_out.p, (size_t)nvals * 8,
                                    cudaMemcpyDeviceToHost, ctx->stream));
      MRD_CUDA(ctx, cudaStreamSynchronize(ctx->stream));   // tab and the host copy
    }
    D->schmidt_nk.clear();
    for (const Sec& q : nb)
      for (int v = 0; v < q.d; ++v) D->schmidt_nk.insert(D->schmidt_nk.end(), {q.N, q.K});
    D->schmidt_bond = i + 1;
  }
  lap(4);
  if (direction > 0) rc = env_left(D, h, i);
  else rc = env_right(D, h, i);
  if (rc != MRD_OK) return rc;
  lap(5);
  D->last_energy = e;
  D->last_trunc = info[1];
  if (energy) *energy = e;
  if (trunc_err) *trunc_err = info[1];
  return MRD_OK;
} catch (...) {   // host memory or threads exhausted: no exception crosses the C ABI
  return MRD_E_HOST;
}

int mrd_sweep(mrd_dmrg* D, const mrd_dmrg_params* p, double* energy) try {
  if (!D || !p) return MRD_E_ARG;
  int rc;
  double e = 0.0;
  for (int i = 0; i <= D->n - 2; ++i)
    if ((rc = mrd_two_site_update(D, i, +1, p, &e, nullptr)) != MRD_OK) return rc;
  for (int i = D->n - 2; i >= 0; --i)
    if ((rc = mrd_two_site_update(D, i, -1, p, &e, nullptr)) != MRD_OK) return rc;
  if (energy) *energy = e;
  return MRD_OK;
} catch (...) {   // host memory or threads exhausted: no exception crosses the C ABI
  return MRD_E_HOST;
}

int mrd_env_update(mrd_dmrg* D, int32_t site, int32_t direction, int32_t prec) try {
  if (!D) return MRD_E_ARG;
  mrd_ctx* ctx = D->ctx;
  if (direction != 1 && direction != -1) return mrd_fail(ctx, MRD_E_ARG, "mrd_env_update: direction must be +1 or -1");
  if (prec != MRD_PREC_FP64 && prec != MRD_PREC_FF)
    return mrd_fail(ctx, MRD_E_ARG, "mrd_env_update: prec must be MRD_PREC_FP64 or MRD_PREC_FF");
  // the fold with the MPO comes from the H_eff of a bond that contains `site`: (site, site+1)
  // for a left environment, (site-1, site) for a right one
  if (direction > 0 && (site < 0 || site > D->n - 2))
    return mrd_fail(ctx, MRD_E_ARG, "mrd_env_update: a left update needs 0 <= site <= n-2");
  if (direction < 0 && (site < 1 || site > D->n - 1))
    return mrd_fail(ctx, MRD_E_ARG, "mrd_env_update: a right update needs 1 <= site <= n-1");
  const EnvT& src = direction > 0 ? D->L[site] : D->R[site + 1];
  if (!src.data.p) return mrd_fail(ctx, MRD_E_STATE, "mrd_env_update: the input environment is not built");
  Guard g(ctx->device);
  D->gemm_ff = prec == MRD_PREC_FF;
  mrd_heff* h = nullptr;
  const int i = direction > 0 ? site : site - 1;
  const double2* ein = nullptr;
  int rc = env_fp64(D, direction > 0 ? D->L[i] : D->R[i + 2], direction > 0 ? 0 : 1, &ein);
  if (rc == MRD_OK)
    rc = direction > 0 ? make_heff(D, i, ein, nullptr, &h) : make_heff(D, i, nullptr, ein, &h);
  if (rc != MRD_OK) return rc;
  rc = direction > 0 ? env_left(D, h, i) : env_right(D, h, i);
  mrd_heff_free(h);
  return rc;
} catch (...) {   // host memory or threads exhausted: no exception crosses the C ABI
  return MRD_E_HOST;
}

int mrd_dmrg_bond(const mrd_dmrg* D, int32_t bond, int32_t* n_sectors, int32_t* sectors) try {
  if (!D || !n_sectors || bond < 0 || bond > D->n) return MRD_E_ARG;
  const Secs& s = bond < D->n ? D->A[bond].left : D->A[D->n - 1].right;
  *n_sectors = (int32_t)s.size();
  if (sectors)
    for (size_t k = 0; k < s.size(); ++k) {
      sectors[3 * k] = s[k].N; sectors[3 * k + 1] = s[k].K; sectors[3 * k + 2] = s[k].d;
    }
  return MRD_OK;
} catch (...) {   // host memory or threads exhausted: no exception crosses the C ABI
  return MRD_E_HOST;
}

int mrd_dmrg_site(mrd_dmrg* D, int32_t site, int32_t* mode, int64_t* len, double* host) try {
  if (!D || !len || site < 0 || site >= D->n) return MRD_E_ARG;
  const SiteT& T = D->A[site];
  if (mode) *mode = T.mode;
  *len = T.size;
  if (host && T.size) {
    Guard g(D->ctx->device);
    MRD_CUDA(D->ctx, cudaStreamSynchronize(D->ctx->stream));
    MRD_CUDA(D->ctx, cudaMemcpy(host, T.data.p, (size_t)T.size * 16, cudaMemcpyDeviceToHost));
  }
  return MRD_OK;
} catch (...) {   // host memory or threads exhausted: no exception crosses the C ABI
  return MRD_E_HOST;
}

int mrd_dmrg_env(mrd_dmrg* D, int32_t bond, int32_t side, int64_t* len, double* host) try {
  if (!D || !len || bond < 0 || bond > D->n) return MRD_E_ARG;
  EnvT& E = side == 0 ? D->L[bond] : D->R[bond];
  *len = E.data.p ? E.size : -1;
  if (host && E.data.p && E.size) {
    Guard g(D->ctx->device);
    MRD_CUDA(D->ctx, cudaStreamSynchronize(D->ctx->stream));
    if (E.f32) {   // complex64 storage, widened on the host
      std::vector<float> t((size_t)E.size * 2);
      MRD_CUDA(D->ctx, cudaMemcpy(t.data(), E.data.p, (size_t)E.size * 8, cudaMemcpyDeviceToHost));
      for (size_t k = 0; k < t.size(); ++k) host[k] = (double)t[k];
    } else {
      MRD_CUDA(D->ctx, cudaMemcpy(host, E.data.p, (size_t)E.size * 16, cudaMemcpyDeviceToHost));
    }
  }
  return MRD_OK;
} catch (...) {   // host memory or threads exhausted: no exception crosses the C ABI
  return MRD_E_HOST;
}

int mrd_dmrg_set_option(mrd_dmrg* D, int32_t option, int64_t value) try {
  if (!D) return MRD_E_ARG;
  mrd_ctx* ctx = D->ctx;
  if (option == MRD_DMRG_OPT_REAL) {
    if (value == 0) { D->real = false; return MRD_OK; }
    if (D->real) return MRD_OK;
    for (const auto& v : D->mpo.site_val)
      for (size_t k = 1; k < v.size(); k += 2)
        if (v[k] != 0.0) return mrd_fail(ctx, MRD_E_ARG, "mrd_dmrg_set_option: MRD_DMRG_OPT_REAL needs a real MPO");
    if (D->updates > 0) return mrd_fail(ctx, MRD_E_STATE, "mrd_dmrg_set_option: MRD_DMRG_OPT_REAL before the first update");
    Guard g(ctx->device);
    for (SiteT& T : D->A)   // the real parts of the seeded random tensors
      if (T.size > 0) {
        k_zero_imag<<<(unsigned)std::min<int64_t>((T.size + 255) / 256, 4096), 256, 0, ctx->stream>>>(
            T.data.as<double2>(), T.size);
        mrd::count_launch();
      }
    MRD_CUDA(ctx, cudaGetLastError());
    D->real = true;
    return canonicalise_and_build_envs(D, D->center0);
  }
  if (option == MRD_DMRG_OPT_SVD_PRESWEEPS) {
    if (value < 0 || value > 64) return mrd_fail(ctx, MRD_E_ARG, "mrd_dmrg_set_option: pre-sweeps outside 0 .. 64");
    D->svd_presweeps = (int)value;
    return MRD_OK;
  }
  if (option != MRD_DMRG_OPT_ENV_FP32) return mrd_fail(ctx, MRD_E_ARG, "mrd_dmrg_set_option: unknown option");
  Guard g(ctx->device);
  D->env_fp32 = value != 0;
  cudaStream_t s = ctx->stream;
  // convert the stored environments (the 1 x 1 boundary ones stay complex128)
  for (std::vector<EnvT>* side : {&D->L, &D->R})
    for (EnvT& E : *side) {
      if (!E.data.p || E.size <= 1 || E.f32 == D->env_fp32) continue;
      Buf nb;
      MRD_CUDA(ctx, nb.need((size_t)E.size * (D->env_fp32 ? 8 : 16)));
      if (D->env_fp32) MRD_CUDA(ctx, conv_c64(E.data.as<double2>(), nb.as<float2>(), E.size, s));
      else MRD_CUDA(ctx, conv_c128(E.data.as<float2>(), nb.as<double2>(), E.size, s));
      MRD_CUDA(ctx, cudaStreamSynchronize(s));
      std::swap(E.data.p, nb.p);
      std::swap(E.data.bytes, nb.bytes);
      E.f32 = D->env_fp32;
    }
  return MRD_OK;
} catch (...) {   // host memory or threads exhausted: no exception crosses the C ABI
  return MRD_E_HOST;
}

int mrd_dmrg_memory(const mrd_dmrg* D, int64_t* out4) try {
  if (!D || !out4) return MRD_E_ARG;
  int64_t env = 0, nenv = 0, mps = 0;
  for (const std::vector<EnvT>* side : {&D->L, &D->R})
    for (const EnvT& E : *side)
      if (E.data.p) {
        env += E.size * (E.f32 ? 8 : 16);
        ++nenv;
      }
  for (const SiteT& T : D->A) mps += T.size * 16;
  out4[0] = env;
  out4[1] = nenv;
  out4[2] = mps;
  out4[3] = D->env_fp32 ? 1 : 0;
  return MRD_OK;
} catch (...) {   // host memory or threads exhausted: no exception crosses the C ABI
  return MRD_E_HOST;
}

int mrd_dmrg_timing(mrd_dmrg* D, int32_t on, double* kernel_ms4, int64_t* applies2) try {
  if (!D) return MRD_E_ARG;
  if (kernel_ms4)
    for (int k = 0; k < 4; ++k) kernel_ms4[k] = D->kms[k];
  if (applies2) { applies2[0] = D->kcount[0]; applies2[1] = D->kcount[1]; }
  for (int k = 0; k < 4; ++k) D->kms[k] = 0;
  D->kcount[0] = D->kcount[1] = 0;
  D->timing = on != 0;
  return MRD_OK;
} catch (...) {   // host memory or threads exhausted: no exception crosses the C ABI
  return MRD_E_HOST;
}

int mrd_dmrg_set_site(mrd_dmrg* D, int32_t site, const double* host) try {
  if (!D || site < 0 || site >= D->n) return MRD_E_ARG;
  SiteT& T = D->A[site];
  if (T.size && !host) return mrd_fail(D->ctx, MRD_E_ARG, "mrd_dmrg_set_site: null data");
  if (T.size) {
    Guard g(D->ctx->device);
    MRD_CUDA(D->ctx, cudaMemcpyAsync(T.data.p, host, (size_t)T.size * 16, cudaMemcpyHostToDevice, D->ctx->stream));
  }
  return MRD_OK;
} catch (...) {   // host memory or threads exhausted: no exception crosses the C ABI
  return MRD_E_HOST;
}

int mrd_dmrg_phase_ms(const mrd_dmrg* D, double* ms8) try {
  if (!D || !ms8) return MRD_E_ARG;
  for (int k = 0; k < 6; ++k) ms8[k] = D->phase_ms[k];
  ms8[6] = D->svd_sweeps32;
  ms8[7] = D->svd_sweeps64;
  return MRD_OK;
} catch (...) {   // host memory or threads exhausted: no exception crosses the C ABI
  return MRD_E_HOST;
}

int mrd_dmrg_schmidt(const mrd_dmrg* D, int32_t* bond, int64_t* n, int32_t* nk, double* values) try {
  if (!D || !n) return MRD_E_ARG;
  if (bond) *bond = D->schmidt_bond;
  *n = (int64_t)D->schmidt_val.size();
  if (nk && !D->schmidt_nk.empty()) std::copy(D->schmidt_nk.begin(), D->schmidt_nk.end(), nk);
  if (values && !D->schmidt_val.empty()) std::copy(D->schmidt_val.begin(), D->schmidt_val.end(), values);
  return MRD_OK;
} catch (...) {   // host memory or threads exhausted: no exception crosses the C ABI
  return MRD_E_HOST;
}

int mrd_dmrg_svd_trace(const mrd_dmrg* D, int32_t cap, int32_t* out, double* ms, int32_t* n2) try {
  if (!D || cap < 0 || (cap > 0 && !out) || !n2) return MRD_E_ARG;
  n2[0] = (int32_t)D->svd_trace32.size();
  n2[1] = (int32_t)D->svd_trace64.size();
  int32_t k = 0;
  for (int ph = 0; ph < 2; ++ph) {
    const std::vector<int32_t>& v = ph ? D->svd_trace64 : D->svd_trace32;
    const std::vector<double>& t = ph ? D->svd_tms64 : D->svd_tms32;
    for (size_t j = 0; j < v.size() && k < cap; ++j, ++k) {
      out[k] = v[j];
      if (ms) ms[k] = j < t.size() ? t[j] : 0.0;
    }
  }
  return MRD_OK;
} catch (...) {   // host memory or threads exhausted: no exception crosses the C ABI
  return MRD_E_HOST;
}

int mrd_dmrg_svd_stats(const mrd_dmrg* D, double* out8) try {
  if (!D || !out8) return MRD_E_ARG;
  for (int k = 0; k < 6; ++k) out8[k] = D->svd_stats[k];
  out8[6] = D->svd_cols[0];
  out8[7] = D->svd_cols[1];
  return MRD_OK;
} catch (...) {   // host memory or threads exhausted: no exception crosses the C ABI
  return MRD_E_HOST;
}

int mrd_dmrg_stats(const mrd_dmrg* D, double* energy, double* trunc_err, int32_t* lanczos_iters) try {
  if (!D) return MRD_E_ARG;
  if (energy) *energy = D->last_energy;
  if (trunc_err) *trunc_err = D->last_trunc;
  if (lanczos_iters) *lanczos_iters = D->last_iters + 1000 * D->last_refine;
  return MRD_OK;
} catch (...) {   // host memory or threads exhausted: no exception crosses the C ABI
  return MRD_E_HOST;
}

}  // extern "C"
