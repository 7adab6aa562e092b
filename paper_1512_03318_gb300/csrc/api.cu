// C ABI entry points (include/mrdmrg.h): argument checks, device memory, launches.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <set>
#include <tuple>
#include <string>
#include <vector>

#include "heff_internal.h"

namespace mrd {
cudaError_t launch_plan(const PlanDims& d, const PlanPtrs& p, cudaStream_t s);
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
cudaError_t launch_fold_env(const double2* env, double2* out, const int64_t* rows, int64_t nrows,
                            const int64_t* env_map, int n_sec, const int32_t* perm, const int32_t* idx,
                            const double* val, int chan_field, cudaStream_t s);
struct Lanczos;
void lanczos_free(Lanczos* L);
cudaError_t lanczos_alloc(Lanczos** out, int64_t n, cudaStream_t stream);
int lanczos_run(Lanczos* L, mrd_ctx* ctx, int (*apply)(void*, const double2*, double2*), void* op, double2* theta,
                int max_iter, double tol, double* energy, int* iters, double* beta_last, uint64_t graph_key,
                int (*replayed)(void*) = nullptr);
int vdot(Lanczos* L, mrd_ctx* ctx, const double2* u, const double2* v, double* re, double* im);
cudaError_t lanczos_set_fp32_full(Lanczos* L, bool on);
double2* lanczos_work(Lanczos* L);
}  // namespace mrd

using namespace mrd;

namespace mrd {
static std::atomic<int64_t> g_launches{0};
void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
void count_launches(int64_t n) { g_launches.fetch_add(n, std::memory_order_relaxed); }
void uncount_launches(int64_t n) { g_launches.fetch_sub(n, std::memory_order_relaxed); }
int64_t launch_count_total() { return g_launches.load(); }
}  // namespace mrd

void mrd_ctx_retain(mrd_ctx* ctx) {
  if (ctx) ++ctx->refs;
}

void mrd_ctx_release(mrd_ctx* ctx) {
  if (!ctx) return;
  if (--ctx->refs == 0 && ctx->destroyed) delete ctx;
}

int mrd_fail(mrd_ctx* ctx, int code, const std::string& msg) {
  if (ctx) ctx->err = msg;
  return code;
}

int mrd_cuda_fail(mrd_ctx* ctx, cudaError_t e, const char* where) {
  std::string m = std::string(where) + ": " + cudaGetErrorString(e);
  return mrd_fail(ctx, e == cudaErrorMemoryAllocation ? MRD_E_OOM : MRD_E_CUDA, m);
}

extern "C" {

int mrd_version(void) { return 100; }

int64_t mrd_launch_count(void) { return mrd::g_launches.load(); }

int mrd_create(mrd_ctx** out, int device, void* stream) try {
  if (!out) return MRD_E_ARG;
  *out = nullptr;
  int n = 0;
  if (cudaGetDeviceCount(&n) != cudaSuccess || device < 0 || device >= n) return MRD_E_ARG;
  mrd_ctx* c = new mrd_ctx();
  c->device = device;
  c->stream = (cudaStream_t)stream;
  *out = c;
  return MRD_OK;
} catch (...) {   // host memory or threads exhausted: no exception crosses the C ABI
  return MRD_E_HOST;
}

int mrd_destroy(mrd_ctx* ctx) try {
  if (!ctx) return MRD_OK;
  ctx->destroyed = true;
  if (ctx->refs == 0) delete ctx;
  return MRD_OK;
} catch (...) {   // host memory or threads exhausted: no exception crosses the C ABI
  return MRD_E_HOST;
}

int mrd_release_cached(mrd_ctx* ctx) try {
  if (!ctx) return MRD_E_ARG;
  Guard g(ctx->device);
  MRD_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  mrd::cache_trim(ctx->device);
  return MRD_OK;
} catch (...) {   // host memory or threads exhausted: no exception crosses the C ABI
  return MRD_E_HOST;
}

int mrd_set_stream(mrd_ctx* ctx, void* stream) try {
  if (!ctx) return MRD_E_ARG;
  ctx->stream = (cudaStream_t)stream;
  return MRD_OK;
} catch (...) {   // host memory or threads exhausted: no exception crosses the C ABI
  return MRD_E_HOST;
}

const char* mrd_last_error(const mrd_ctx* ctx) { return ctx ? ctx->err.c_str() : "null context"; }

// ------------------------------------------------------------------ MPO

int mrd_mpo_build(mrd_ctx* ctx, const mrd_model* model, mrd_mpo** out) try {
  // host-only: ctx may be NULL (then no message is recorded)
  if (!model || !out) return mrd_fail(ctx, MRD_E_ARG, "mrd_mpo_build: null argument");
  *out = nullptr;
  mrd_mpo* m = new mrd_mpo();
  m->ctx = ctx;
  std::string err;
  int rc = build_mpo_host(*model, &m->h, &err);
  if (rc != MRD_OK) {
    delete m;
    return mrd_fail(ctx, rc, err);
  }
  *out = m;
  return MRD_OK;
} catch (...) {   // host memory or threads exhausted: no exception crosses the C ABI
  return MRD_E_HOST;
}

int mrd_mpo_free(mrd_mpo* mpo) try {
  delete mpo;
  return MRD_OK;
} catch (...) {   // host memory or threads exhausted: no exception crosses the C ABI
  return MRD_E_HOST;
}

int mrd_mpo_info(const mrd_mpo* mpo, int32_t* n_sites, int32_t* modulus) try {
  if (!mpo) return MRD_E_ARG;
  if (n_sites) *n_sites = mpo->h.n_sites;
  if (modulus) *modulus = mpo->h.modulus;
  return MRD_OK;
} catch (...) {   // host memory or threads exhausted: no exception crosses the C ABI
  return MRD_E_HOST;
}

int mrd_mpo_bond(const mrd_mpo* mpo, int32_t bond, int32_t* dim, int32_t* charges) try {
  if (!mpo || !dim || bond < 0 || bond > mpo->h.n_sites) return MRD_E_ARG;
  const auto& c = mpo->h.bond_charges[bond];
  *dim = (int32_t)(c.size() / 2);
  if (charges) std::memcpy(charges, c.data(), c.size() * sizeof(int32_t));
  return MRD_OK;
} catch (...) {   // host memory or threads exhausted: no exception crosses the C ABI
  return MRD_E_HOST;
}

int mrd_mpo_site(const mrd_mpo* mpo, int32_t site, int32_t* nnz, int32_t* idx, double* val) try {
  if (!mpo || !nnz || site < 0 || site >= mpo->h.n_sites) return MRD_E_ARG;
  const auto& i = mpo->h.site_idx[site];
  const auto& v = mpo->h.site_val[site];
  *nnz = (int32_t)(i.size() / 4);
  if (idx) std::memcpy(idx, i.data(), i.size() * sizeof(int32_t));
  if (val) std::memcpy(val, v.data(), v.size() * sizeof(double));
  return MRD_OK;
} catch (...) {   // host memory or threads exhausted: no exception crosses the C ABI
  return MRD_E_HOST;
}

int mrd_mpo_stats(const mrd_mpo* mpo, int32_t first, int32_t count, double* out4) try {
  if (!mpo || !out4 || first < 0 || count < 1 || first > mpo->h.n_sites - count) return MRD_E_ARG;
  double dsum = 0.0, fsum = 0.0, nnz = 0.0;
  int64_t dmax = 0;
  for (int32_t j = first; j < first + count; ++j) {
    const int64_t dl = (int64_t)mpo->h.bond_charges[j].size() / 2, dr = (int64_t)mpo->h.bond_charges[j + 1].size() / 2;
    const double n = (double)(mpo->h.site_idx[j].size() / 4);
    dsum += (double)dl;
    dmax = std::max(dmax, dl);
    fsum += dl * dr > 0 ? n / (4.0 * (double)dl * (double)dr) : 0.0;
    nnz += n;
  }
  out4[0] = dsum / count;
  out4[1] = (double)dmax;
  out4[2] = fsum / count;
  out4[3] = nnz;
  return MRD_OK;
} catch (...) {   // host memory or threads exhausted: no exception crosses the C ABI
  return MRD_E_HOST;
}

// ------------------------------------------------------------------ H_eff

static int validate_sectors(mrd_ctx* ctx, const int32_t* s, int n, int mod, const char* what) {
  if (n < 0 || (n > 0 && !s)) return mrd_fail(ctx, MRD_E_ARG, std::string("mrd_heff_create: bad ") + what);
  for (int i = 0; i < n; ++i) {
    if (s[3 * i + 2] <= 0 || s[3 * i + 1] < 0 || s[3 * i + 1] >= mod)
      return mrd_fail(ctx, MRD_E_ARG, std::string("mrd_heff_create: ") + what + " sector with dim <= 0 or K out of range");
    if (i > 0 && qkey(s[3 * i - 3], s[3 * i - 2]) >= qkey(s[3 * i], s[3 * i + 1]))
      return mrd_fail(ctx, MRD_E_ARG, std::string("mrd_heff_create: ") + what + " sectors not strictly increasing in (N, K)");
  }
  return MRD_OK;
}

static int validate_entries(mrd_ctx* ctx, const int32_t* idx, const double* val, int nnz, int d0, int d1,
                            const int32_t* c0, const int32_t* c1, int m, int mod, const char* what) {
  if (nnz < 0 || (nnz > 0 && (!idx || !val))) return mrd_fail(ctx, MRD_E_ARG, std::string("mrd_heff_create: bad ") + what);
  for (int e = 0; e < nnz; ++e) {
    int w = idx[4 * e], wp = idx[4 * e + 1], sp = idx[4 * e + 2], s = idx[4 * e + 3];
    if (w < 0 || w >= d0 || wp < 0 || wp >= d1 || (sp & ~1) || (s & ~1))
      return mrd_fail(ctx, MRD_E_ARG, std::string("mrd_heff_create: ") + what + " entry index out of range");
    if (c1[2 * wp] != c0[2 * w] + sp - s || kmod(c1[2 * wp + 1], mod) != kmod(c0[2 * w + 1] + (sp - s) * m, mod))
      return mrd_fail(ctx, MRD_E_CHARGE, std::string("mrd_heff_create: ") + what + " entry violates charge conservation");
  }
  // duplicates would be summed twice by nobody: reject them
  std::vector<int64_t> keys(nnz);
  for (int e = 0; e < nnz; ++e)
    keys[e] = (((int64_t)idx[4 * e] * d1 + idx[4 * e + 1]) * 2 + idx[4 * e + 2]) * 2 + idx[4 * e + 3];
  std::sort(keys.begin(), keys.end());
  for (int e = 1; e < nnz; ++e)
    if (keys[e] == keys[e - 1]) return mrd_fail(ctx, MRD_E_ARG, std::string("mrd_heff_create: duplicate ") + what + " entry");
  return MRD_OK;
}

int mrd_heff_create(mrd_ctx* ctx, const mrd_heff_desc* desc, mrd_heff** out) try {
  if (!ctx || !desc || !out) return mrd_fail(ctx, MRD_E_ARG, "mrd_heff_create: null argument");
  *out = nullptr;
  const mrd_heff_desc& D = *desc;
  if (D.modulus < 1 || D.d_l < 1 || D.d_m < 1 || D.d_r < 1 || !D.c_l || !D.c_m || !D.c_r || D.m1 < 0 || D.m2 < 0)
    return mrd_fail(ctx, MRD_E_ARG, "mrd_heff_create: bad modulus, MPO dims or channel charges");
  int rc;
  if ((rc = validate_sectors(ctx, D.left, D.n_left, D.modulus, "left")) != MRD_OK) return rc;
  if ((rc = validate_sectors(ctx, D.right, D.n_right, D.modulus, "right")) != MRD_OK) return rc;
  if ((rc = validate_entries(ctx, D.wi_idx, D.wi_val, D.nnz_i, D.d_l, D.d_m, D.c_l, D.c_m, D.m1, D.modulus, "W_i")) != MRD_OK) return rc;
  if ((rc = validate_entries(ctx, D.wj_idx, D.wj_val, D.nnz_j, D.d_m, D.d_r, D.c_m, D.c_r, D.m2, D.modulus, "W_i+1")) != MRD_OK) return rc;
  if (D.n_left == 0 || D.n_right == 0) return mrd_fail(ctx, MRD_E_ARG, "mrd_heff_create: empty bond");

  Guard g(ctx->device);
  mrd_heff* h = new mrd_heff();
  h->ctx = ctx;
  mrd_ctx_retain(ctx);
  cudaDeviceGetAttribute(&h->n_sm, cudaDevAttrMultiProcessorCount, ctx->device);
  h->left.assign(D.left, D.left + 3 * D.n_left);
  h->right.assign(D.right, D.right + 3 * D.n_right);
  h->cl.assign(D.c_l, D.c_l + 2 * D.d_l);
  h->cm.assign(D.c_m, D.c_m + 2 * D.d_m);
  h->cr.assign(D.c_r, D.c_r + 2 * D.d_r);
  for (auto* v : {&h->cl, &h->cm, &h->cr})
    for (size_t i = 1; i < v->size(); i += 2) (*v)[i] = kmod((*v)[i], D.modulus);
  h->wi_idx.assign(D.wi_idx, D.wi_idx + 4 * D.nnz_i);
  h->wj_idx.assign(D.wj_idx, D.wj_idx + 4 * D.nnz_j);
  h->wi_v.assign(D.wi_val, D.wi_val + 2 * D.nnz_i);
  h->wj_v.assign(D.wj_val, D.wj_val + 2 * D.nnz_j);

  PlanDims& d = h->d;
  d.n_l = D.n_left; d.n_r = D.n_right; d.d_l = D.d_l; d.d_m = D.d_m; d.d_r = D.d_r;
  d.nnz_i = D.nnz_i; d.nnz_j = D.nnz_j; d.m1 = D.m1 % D.modulus; d.m2 = D.m2 % D.modulus; d.mod = D.modulus;
  d.mid_cap = 2 * (int64_t)D.n_left;
  d.lw_cap = (int64_t)D.d_m * 4 * D.n_left;
  d.wr_cap = (int64_t)D.d_m * 4 * D.n_right;
  d.z_cap = (int64_t)D.d_m * d.mid_cap;
  d.t1_cap = d.z_cap * 2;
  d.t2_cap = d.mid_cap * 4;
  d.seg2_stride = 2 * (int64_t)D.d_m;
  int64_t sl = d.mid_cap;
  for (int64_t v : {(int64_t)D.d_l * D.n_left, (int64_t)D.d_r * D.n_right, d.lw_cap, d.wr_cap, d.z_cap, d.t1_cap, d.t2_cap})
    sl = v > sl ? v : sl;
  d.scratch_len = sl + 1;

  Arena& A = h->plan_mem;
  A.stream = ctx->stream;
  PlanPtrs& p = h->p;
  int32_t *left = nullptr, *right = nullptr, *cl = nullptr, *cm = nullptr, *cr = nullptr, *wi = nullptr, *wj = nullptr;
  cudaError_t e = cudaSuccess;
#define ALLOC(ptr, n) if (e == cudaSuccess) e = A.alloc(&(ptr), (size_t)(n))
  ALLOC(left, 3 * d.n_l); ALLOC(right, 3 * d.n_r); ALLOC(cl, 2 * d.d_l); ALLOC(cm, 2 * d.d_m); ALLOC(cr, 2 * d.d_r);
  ALLOC(wi, 4 * d.nnz_i); ALLOC(wj, 4 * d.nnz_j); ALLOC(h->wi_val, 2 * d.nnz_i); ALLOC(h->wj_val, 2 * d.nnz_j);
  ALLOC(p.wi_perm, d.nnz_i); ALLOC(p.wj_perm, d.nnz_j); ALLOC(p.trip_i, 8 * d.d_m); ALLOC(p.trip_j, 8 * d.d_m);
  ALLOC(p.mid, MIDF * d.mid_cap); ALLOC(p.counts, C_NCOUNTS);
  ALLOC(p.lmap, (int64_t)d.d_l * d.n_l); ALLOC(p.rmap, (int64_t)d.d_r * d.n_r);
  ALLOC(p.lwmap, d.lw_cap); ALLOC(p.lw, LWF * d.lw_cap); ALLOC(p.wrmap, d.wr_cap); ALLOC(p.wr, WRF * d.wr_cap);
  ALLOC(p.zmap, d.z_cap); ALLOC(p.z, ZF * d.z_cap); ALLOC(p.s1mask, d.z_cap);
  ALLOC(p.t1, TF * d.t1_cap); ALLOC(p.seg1, SF * 2 * d.t1_cap); ALLOC(p.tile1, d.t1_cap + 1);
  ALLOC(p.t2, TF * d.t2_cap); ALLOC(p.seg2, SF * d.t2_cap * d.seg2_stride); ALLOC(p.tile2, d.t2_cap + 1);
  ALLOC(p.scr_a, d.scratch_len); ALLOC(p.scr_b, d.scratch_len);
#undef ALLOC
  if (e != cudaSuccess) {
    delete h;
    mrd_ctx_release(ctx);
    return mrd_cuda_fail(ctx, e, "mrd_heff_create: cudaMalloc");
  }
  p.left = left; p.right = right; p.cl = cl; p.cm = cm; p.cr = cr; p.wi_idx = wi; p.wj_idx = wj;
  cudaStream_t s = ctx->stream;
  auto up = [&](void* dst, const void* src, size_t bytes) {
    if (e == cudaSuccess && bytes) e = cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, s);
  };
  up(left, h->left.data(), h->left.size() * 4); up(right, h->right.data(), h->right.size() * 4);
  up(cl, h->cl.data(), h->cl.size() * 4); up(cm, h->cm.data(), h->cm.size() * 4); up(cr, h->cr.data(), h->cr.size() * 4);
  up(wi, h->wi_idx.data(), h->wi_idx.size() * 4); up(wj, h->wj_idx.data(), h->wj_idx.size() * 4);
  up(h->wi_val, h->wi_v.data(), h->wi_v.size() * 8); up(h->wj_val, h->wj_v.data(), h->wj_v.size() * 8);
  if (e == cudaSuccess) e = launch_plan(d, p, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(h->counts, p.counts, sizeof(h->counts), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    delete h;
    mrd_ctx_release(ctx);
    return mrd_cuda_fail(ctx, e, "mrd_heff_create: plan");
  }
  // Host check of the device-built tables before any kernel reads through them: every
  // GEMM segment and output block, and every fold source, must lie inside its buffer.
  {
    const int64_t* c = h->counts;
    auto dl = [&](std::vector<int64_t>& v, const int64_t* src, size_t n) {
      v.resize(n);
      if (e == cudaSuccess && n) e = cudaMemcpy(v.data(), src, n * 8, cudaMemcpyDeviceToHost);
    };
    std::vector<int64_t>& t1 = h->t1_host;
    std::vector<int64_t>& s1 = h->s1_host;
    std::vector<int64_t>& t2 = h->t2_host;
    std::vector<int64_t>& s2 = h->s2_host;
    std::vector<int64_t>& lw = h->lw_host;
    std::vector<int64_t>& wr = h->wr_host;
    std::vector<int64_t>& lmap = h->lmap_host;
    std::vector<int64_t>& rmap = h->rmap_host;
    std::vector<int32_t> wperm_i(d.nnz_i), wperm_j(d.nnz_j);
    dl(t1, p.t1, (size_t)TF * c[C_NT1]); dl(s1, p.seg1, (size_t)SF * 2 * c[C_NT1]);
    dl(t2, p.t2, (size_t)TF * c[C_NT2]); dl(s2, p.seg2, (size_t)SF * c[C_NT2] * d.seg2_stride);
    dl(lw, p.lw, (size_t)LWF * c[C_NLW]); dl(wr, p.wr, (size_t)WRF * c[C_NWR]);
    dl(lmap, p.lmap, (size_t)d.d_l * d.n_l); dl(rmap, p.rmap, (size_t)d.d_r * d.n_r);
    dl(h->z_host, p.z, (size_t)ZF * std::min(c[C_NZ], d.z_cap));   // Z blocks, for the tensor-core panel tables
    if (e == cudaSuccess && d.nnz_i) e = cudaMemcpy(wperm_i.data(), p.wi_perm, d.nnz_i * 4, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && d.nnz_j) e = cudaMemcpy(wperm_j.data(), p.wj_perm, d.nnz_j * 4, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) { delete h; mrd_ctx_release(ctx); return mrd_cuda_fail(ctx, e, "mrd_heff_create: table download"); }
    bool ok = c[C_NMID] <= d.mid_cap && c[C_NLW] <= d.lw_cap && c[C_NWR] <= d.wr_cap && c[C_NZ] <= d.z_cap;
    auto in = [](int64_t off, int64_t rows, int64_t cols, int64_t ld, int64_t len) {
      if (rows == 0 || cols == 0) return true;
      return off >= 0 && ld >= cols && off + (rows - 1) * ld + cols <= len;
    };
    auto check_tasks = [&](const std::vector<int64_t>& t, const std::vector<int64_t>& sg, int64_t nt, int64_t alen,
                           int64_t blen, int64_t clen) {
      for (int64_t i = 0; i < nt && ok; ++i) {
        const int64_t* r = &t[TF * i];
        if (r[0] == 0 || r[1] == 0) continue;
        ok = ok && in(r[2], r[0], r[1], r[3], clen);
        for (int64_t k = 0; k < r[5] && ok; ++k) {
          const int64_t* q = &sg[SF * (r[4] + k)];
          ok = ok && q[4] > 0 && in(q[0], r[0], q[4], q[1], alen) && in(q[2], q[4], r[1], q[3], blen);
        }
      }
    };
    check_tasks(t1, s1, c[C_NT1], c[C_LWLEN], c[C_THETA], c[C_ZLEN]);
    check_tasks(t2, s2, c[C_NT2], c[C_ZLEN], c[C_WRLEN], c[C_THETA]);
    for (int64_t i = 0; i < c[C_NLW] && ok; ++i) {
      const int64_t* r = &lw[LWF * i];
      ok = ok && r[7] >= 0 && r[7] + r[5] * r[6] <= c[C_LWLEN];
      for (int64_t k = r[8]; k < r[9] && ok; ++k) {
        int w = h->wi_idx[4 * wperm_i[k]];
        int64_t off = lmap[(size_t)w * d.n_l + r[3]];
        ok = ok && off >= 0 && off + r[5] * r[6] <= c[C_LENV];
      }
    }
    for (int64_t i = 0; i < c[C_NWR] && ok; ++i) {
      const int64_t* r = &wr[WRF * i];
      ok = ok && r[7] >= 0 && r[7] + r[5] * r[6] <= c[C_WRLEN];
      for (int64_t k = r[8]; k < r[9] && ok; ++k) {
        int wpp = h->wj_idx[4 * wperm_j[k] + 1];
        int64_t off = rmap[(size_t)wpp * d.n_r + r[3]];
        ok = ok && off >= 0 && off + r[5] * r[6] <= c[C_RENV];
      }
    }
    if (!ok) {
      delete h;
      mrd_ctx_release(ctx);
      return mrd_fail(ctx, MRD_E_STATE, "mrd_heff_create: internal table check failed (out-of-range block)");
    }
  }
  Arena& B = h->data_mem;
  B.stream = ctx->stream;
  if (e == cudaSuccess) e = B.alloc(&h->lw, (size_t)h->counts[C_LWLEN]);
  if (e == cudaSuccess) e = B.alloc(&h->wr, (size_t)h->counts[C_WRLEN]);
  if (e == cudaSuccess) e = B.alloc(&h->z, (size_t)h->counts[C_ZLEN]);
  if (e != cudaSuccess) {
    delete h;
    mrd_ctx_release(ctx);
    return mrd_cuda_fail(ctx, e, "mrd_heff_create: operand buffers");
  }

  // middle-sector table on the host (tensor-core panel tables, flop counts)
  {
    std::vector<int64_t>& mid = h->mid_host;
    mid.resize(MIDF * h->counts[C_NMID]);
    e = cudaMemcpy(mid.data(), p.mid, mid.size() * 8, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) { delete h; mrd_ctx_release(ctx); return mrd_cuda_fail(ctx, e, "mrd_heff_create: table download"); }
  }
  *out = h;
  return MRD_OK;
} catch (...) {   // host memory or threads exhausted: no exception crosses the C ABI
  return MRD_E_HOST;
}

int mrd_heff_free(mrd_heff* h) try {
  if (!h) return MRD_OK;
  mrd_ctx* ctx = h->ctx;
  {
    Guard g(ctx->device);
    cudaStreamSynchronize(ctx->stream);
    delete h;
  }
  mrd_ctx_release(ctx);
  return MRD_OK;
} catch (...) {   // host memory or threads exhausted: no exception crosses the C ABI
  return MRD_E_HOST;
}

int mrd_heff_sizes(const mrd_heff* h, int64_t* theta_len, int64_t* lenv_len, int64_t* renv_len) try {
  if (!h) return MRD_E_ARG;
  if (theta_len) *theta_len = h->counts[C_THETA];
  if (lenv_len) *lenv_len = h->counts[C_LENV];
  if (renv_len) *renv_len = h->counts[C_RENV];
  return MRD_OK;
} catch (...) {   // host memory or threads exhausted: no exception crosses the C ABI
  return MRD_E_HOST;
}

int mrd_heff_set_env(mrd_heff* h, const double* lenv_dev, const double* renv_dev) try {
  if (!h) return MRD_E_ARG;
  mrd_ctx* ctx = h->ctx;
  if ((!lenv_dev && h->counts[C_LENV] > 0) || (!renv_dev && h->counts[C_RENV] > 0))
    return mrd_fail(ctx, MRD_E_ARG, "mrd_heff_set_env: null environment");
  Guard g(ctx->device);
  cudaError_t e = launch_fold_env((const double2*)lenv_dev, h->lw, h->p.lw, h->counts[C_NLW], h->p.lmap, h->d.n_l,
                                  h->p.wi_perm, h->p.wi_idx, h->wi_val, 0, ctx->stream);
  if (e == cudaSuccess)
    e = launch_fold_env((const double2*)renv_dev, h->wr, h->p.wr, h->counts[C_NWR], h->p.rmap, h->d.n_r,
                        h->p.wj_perm, h->p.wj_idx, h->wj_val, 1, ctx->stream);
  if (e != cudaSuccess) return mrd_cuda_fail(ctx, e, "mrd_heff_set_env");
  h->env_loaded = true;
  tc_env_changed(h);
  h->ff_dirty = true;
  return MRD_OK;
} catch (...) {   // host memory or threads exhausted: no exception crosses the C ABI
  return MRD_E_HOST;
}

// Per-task launch tables of the FP64 / float-float GEMM steps (32 x 32 tiles).
static int ensure_per_task(mrd_heff* h) {
  if (h->pt_pref1) return MRD_OK;
  mrd_ctx* ctx = h->ctx;
  const int64_t n1 = h->counts[C_NT1], n2 = h->counts[C_NT2];
  std::vector<int64_t> p1(2 * std::max<int64_t>(n1, 1), 0), p2(2 * std::max<int64_t>(n2, 1), 0);
  h->pt_tiles1.assign(n1, 0);
  h->pt_tiles2.assign(n2, 0);
  for (int64_t t = 0; t < n1; ++t) {
    const int64_t* r = &h->t1_host[TF * t];
    h->pt_tiles1[t] = r[5] > 0 ? ((r[0] + 31) / 32) * ((r[1] + 31) / 32) : 0;
    p1[2 * t + 1] = h->pt_tiles1[t];
  }
  for (int64_t t = 0; t < n2; ++t) {
    const int64_t* r = &h->t2_host[TF * t];
    h->pt_tiles2[t] = r[5] > 0 ? ((r[0] + 31) / 32) * ((r[1] + 31) / 32) : 0;
    p2[2 * t + 1] = h->pt_tiles2[t];
  }
  Arena& A = h->pt_mem;
  A.stream = ctx->stream;
  int64_t *d1 = nullptr, *d2 = nullptr;
  cudaError_t e = A.alloc(&d1, p1.size());
  if (e == cudaSuccess) e = A.alloc(&d2, p2.size());
  if (e == cudaSuccess) e = cudaMemcpyAsync(d1, p1.data(), p1.size() * 8, cudaMemcpyHostToDevice, ctx->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(d2, p2.data(), p2.size() * 8, cudaMemcpyHostToDevice, ctx->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
  if (e != cudaSuccess) return mrd_cuda_fail(ctx, e, "per-task launch tables");
  h->pt_pref1 = d1;
  h->pt_pref2 = d2;
  ++h->gen;
  return MRD_OK;
}

// Everything an application of `prec` needs beyond launching its kernels: tensor-core panel
// tables and packed environments, float-float copies of the folded environments. Allocates
// and may synchronise; a no-op once done (until the environments or the precision change).
// h->gen counts the (re)allocations, which invalidate captured Lanczos steps.
static int heff_prepare(mrd_heff* h, int32_t prec) {
  mrd_ctx* ctx = h->ctx;
  cudaStream_t s = ctx->stream;
  if (prec == MRD_PREC_TF32 || prec == MRD_PREC_BF16X3) return tc_prepare(h, prec);
  if (h->per_task) {
    int rc = ensure_per_task(h);
    if (rc != MRD_OK) return rc;
  }
  if (prec != MRD_PREC_FF) return MRD_OK;
  // float-float operands: LW and WR converted once per environment load, theta per call;
  // Z is written and read in float-float (it reuses the FP64 Z buffer: 16 bytes either way)
  if (!h->lw_ff) {
    Arena& A = h->ff_mem;
    A.stream = s;
    cudaError_t e = A.alloc(&h->lw_ff, (size_t)std::max<int64_t>(h->counts[C_LWLEN], 1));
    if (e == cudaSuccess) e = A.alloc(&h->wr_ff, (size_t)std::max<int64_t>(h->counts[C_WRLEN], 1));
    if (e == cudaSuccess) e = A.alloc(&h->th_ff, (size_t)std::max<int64_t>(h->counts[C_THETA], 1));
    if (e != cudaSuccess) return mrd_cuda_fail(ctx, e, "mrd_heff_apply: float-float buffers");
    h->ff_dirty = true;
    ++h->gen;
  }
  if (h->ff_dirty) {
    MRD_CUDA(ctx, to_ff(h->lw, h->lw_ff, h->counts[C_LWLEN], s));
    MRD_CUDA(ctx, to_ff(h->wr, h->wr_ff, h->counts[C_WRLEN], s));
    h->ff_dirty = false;
  }
  // launch order of the grouped float-float steps (longest K first), once per H_eff; kept
  // only if its tiles add up to the device-built tile prefix
  if (!h->ff_items_built) {
    h->ff_items_built = true;
    const std::vector<int2> i1 = ff_item_order(h->t1_host.data(), h->s1_host.data(), h->counts[C_NT1]);
    const std::vector<int2> i2 = ff_item_order(h->t2_host.data(), h->s2_host.data(), h->counts[C_NT2]);
    if ((int64_t)i1.size() == h->counts[C_TILES1] && (int64_t)i2.size() == h->counts[C_TILES2]) {
      Arena& A = h->ff_mem;
      cudaError_t e = A.alloc(&h->ff_it1, std::max<size_t>(i1.size(), 1));
      if (e == cudaSuccess) e = A.alloc(&h->ff_it2, std::max<size_t>(i2.size(), 1));
      if (e == cudaSuccess && !i1.empty()) e = cudaMemcpyAsync(h->ff_it1, i1.data(), i1.size() * 8, cudaMemcpyHostToDevice, s);
      if (e == cudaSuccess && !i2.empty()) e = cudaMemcpyAsync(h->ff_it2, i2.data(), i2.size() * 8, cudaMemcpyHostToDevice, s);
      if (e != cudaSuccess) return mrd_cuda_fail(ctx, e, "mrd_heff_apply: float-float item tables");
    }
  }
  return MRD_OK;
}

int mrd_heff_apply(mrd_heff* h, const double* theta_in_dev, double* theta_out_dev, int32_t prec) try {
  if (!h) return MRD_E_ARG;
  mrd_ctx* ctx = h->ctx;
  if (!h->env_loaded) return mrd_fail(ctx, MRD_E_STATE, "mrd_heff_apply: environments not loaded");
  if (prec != MRD_PREC_FP64 && prec != MRD_PREC_TF32 && prec != MRD_PREC_BF16X3 && prec != MRD_PREC_FF)
    return mrd_fail(ctx, MRD_E_ARG, "mrd_heff_apply: unsupported precision");
  const int64_t n = h->counts[C_THETA];
  if (n > 0 && (!theta_in_dev || !theta_out_dev)) return mrd_fail(ctx, MRD_E_ARG, "mrd_heff_apply: null theta");
  const char* a = (const char*)theta_in_dev;
  const char* b = (const char*)theta_out_dev;
  if (n > 0 && a < b + n * 16 && b < a + n * 16) return mrd_fail(ctx, MRD_E_ARG, "mrd_heff_apply: theta_in and theta_out overlap");
  Guard g(ctx->device);
  if (prec == MRD_PREC_TF32 || prec == MRD_PREC_BF16X3) return tc_apply(h, theta_in_dev, theta_out_dev, prec);
  int rc = heff_prepare(h, prec);
  if (rc != MRD_OK) return rc;
  cudaStream_t s = ctx->stream;
  cudaEvent_t ev[3] = {nullptr, nullptr, nullptr};
  bool cap = false;
  if (h->timing && !apply_events(h, s, ev, &cap)) return mrd_fail(ctx, MRD_E_CUDA, "mrd_heff_apply: cudaEventCreate");
  const cudaEvent_t e0 = ev[0], e1 = ev[1], e2 = ev[2];
  cudaError_t e = cudaMemsetAsync(theta_out_dev, 0, (size_t)n * 16, s);
  if (prec == MRD_PREC_FF) {
    float4* z_ff = (float4*)h->z;
    // real operands (MRD_OPT_REAL): one float-float product per multiply-add instead of three
    auto gemm = h->real ? launch_rgemm_ff_packed : launch_cgemm_ff_packed;
    if (e == cudaSuccess) e = to_ff((const double2*)theta_in_dev, h->th_ff, n, s);
    if (e == cudaSuccess && e0) e = record_event(e0, s, cap);
    if (!h->per_task) {
      if (e == cudaSuccess)
        e = gemm(h->lw_ff, h->th_ff, z_ff, nullptr, h->p.t1, h->p.seg1, h->p.tile1,
                 h->counts[C_NT1], h->counts[C_TILES1], h->n_sm, s, h->ff_it1);
      if (e == cudaSuccess && e1) e = record_event(e1, s, cap);
      if (e == cudaSuccess)
        e = gemm(z_ff, h->wr_ff, nullptr, (double2*)theta_out_dev, h->p.t2, h->p.seg2, h->p.tile2,
                 h->counts[C_NT2], h->counts[C_TILES2], h->n_sm, s, h->ff_it2);
    } else {
      for (int64_t t = 0; e == cudaSuccess && t < h->counts[C_NT1]; ++t)
        if (h->pt_tiles1[t])
          e = gemm(h->lw_ff, h->th_ff, z_ff, nullptr, h->p.t1 + TF * t, h->p.seg1, h->pt_pref1 + 2 * t, 1,
                   h->pt_tiles1[t], h->n_sm, s, nullptr);
      if (e == cudaSuccess && e1) e = record_event(e1, s, cap);
      for (int64_t t = 0; e == cudaSuccess && t < h->counts[C_NT2]; ++t)
        if (h->pt_tiles2[t])
          e = gemm(z_ff, h->wr_ff, nullptr, (double2*)theta_out_dev, h->p.t2 + TF * t, h->p.seg2,
                   h->pt_pref2 + 2 * t, 1, h->pt_tiles2[t], h->n_sm, s, nullptr);
    }
  } else {
    if (e == cudaSuccess && e0) e = record_event(e0, s, cap);
    if (!h->per_task) {
      if (e == cudaSuccess)
        e = launch_cgemm_fp64(h->lw, (const double2*)theta_in_dev, h->z, h->p.t1, h->p.seg1, h->p.tile1,
                              h->counts[C_NT1], h->counts[C_TILES1], h->n_sm, s);
      if (e == cudaSuccess && e1) e = record_event(e1, s, cap);
      if (e == cudaSuccess)
        e = launch_cgemm_fp64(h->z, h->wr, (double2*)theta_out_dev, h->p.t2, h->p.seg2, h->p.tile2,
                              h->counts[C_NT2], h->counts[C_TILES2], h->n_sm, s);
    } else {
      for (int64_t t = 0; e == cudaSuccess && t < h->counts[C_NT1]; ++t)
        if (h->pt_tiles1[t])
          e = launch_cgemm_fp64(h->lw, (const double2*)theta_in_dev, h->z, h->p.t1 + TF * t, h->p.seg1,
                                h->pt_pref1 + 2 * t, 1, h->pt_tiles1[t], h->n_sm, s);
      if (e == cudaSuccess && e1) e = record_event(e1, s, cap);
      for (int64_t t = 0; e == cudaSuccess && t < h->counts[C_NT2]; ++t)
        if (h->pt_tiles2[t])
          e = launch_cgemm_fp64(h->z, h->wr, (double2*)theta_out_dev, h->p.t2 + TF * t, h->p.seg2,
                                h->pt_pref2 + 2 * t, 1, h->pt_tiles2[t], h->n_sm, s);
    }
  }
  if (e == cudaSuccess && e2) e = record_event(e2, s, cap);
  if (e != cudaSuccess) return mrd_cuda_fail(ctx, e, "mrd_heff_apply");
  return MRD_OK;
} catch (...) {   // host memory or threads exhausted: no exception crosses the C ABI
  return MRD_E_HOST;
}

// Flops of one application in the order of the definition (L, then W_i W_{i+1}, then R, as
// the oracle counts them): host arithmetic on the tables, computed on the first request only.
static double definition_flops(const mrd_heff* h) {
  const std::vector<int64_t>& mid = h->mid_host;
  const PlanDims& d = h->d;
  // theta blocks (a, s1, s2) -> (d_a, d_b, b)
  struct TB { int a, s1, s2, b; int64_t da, db; };
  std::vector<TB> tb;
  for (int64_t m = 0; m < h->counts[C_NMID]; ++m) {
    const int64_t* r = &mid[MIDF * m];
    for (int s1 = 0; s1 < 2; ++s1)
      for (int s2 = 0; s2 < 2; ++s2) {
        if (r[5 + s1] < 0 || r[8 + s2] < 0) continue;
        int a = (int)r[5 + s1], b = (int)r[8 + s2];
        tb.push_back({a, s1, s2, b, h->left[3 * a + 2], h->right[3 * b + 2]});
      }
  }
  auto find = [&](const std::vector<int32_t>& sec, int N, int K) {
    int n = (int)sec.size() / 3;
    for (int i = 0; i < n; ++i) if (sec[3 * i] == N && sec[3 * i + 1] == K) return i;
    return -1;
  };
  double fl = 0.0;
  std::vector<std::vector<std::vector<std::tuple<int, int, int64_t, int64_t>>>> xk(
      d.d_l, std::vector<std::vector<std::tuple<int, int, int64_t, int64_t>>>(4));
  for (const TB& t : tb)
    for (int w = 0; w < d.d_l; ++w) {
      int ap = find(h->left, h->left[3 * t.a] + h->cl[2 * w], kmod(h->left[3 * t.a + 1] + h->cl[2 * w + 1], d.mod));
      if (ap < 0) continue;
      int64_t dp = h->left[3 * ap + 2];
      fl += 8.0 * dp * t.da * t.db;
      xk[w][t.s1 * 2 + t.s2].emplace_back(ap, t.b, dp, t.db);
    }
  std::vector<std::vector<std::tuple<int, int, int, double>>> wj_by(d.d_m);
  for (int e2 = 0; e2 < d.nnz_j; ++e2)
    wj_by[h->wj_idx[4 * e2]].emplace_back(h->wj_idx[4 * e2 + 1], h->wj_idx[4 * e2 + 2], h->wj_idx[4 * e2 + 3], 0.0);
  std::set<std::tuple<int, int, int, int, int>> ykeys;
  std::vector<std::tuple<int, int, int, int, int, int64_t, int64_t>> ylist;
  for (int e1 = 0; e1 < d.nnz_i; ++e1) {
    int w = h->wi_idx[4 * e1], wp = h->wi_idx[4 * e1 + 1], s1p = h->wi_idx[4 * e1 + 2], s1 = h->wi_idx[4 * e1 + 3];
    for (const auto& j : wj_by[wp]) {
      int wpp = std::get<0>(j), s2p = std::get<1>(j), s2 = std::get<2>(j);
      for (const auto& x : xk[w][s1 * 2 + s2]) {
        fl += 8.0 * std::get<2>(x) * std::get<3>(x);
        auto key = std::make_tuple(wpp, std::get<0>(x), s1p, s2p, std::get<1>(x));
        if (ykeys.insert(key).second) ylist.emplace_back(wpp, std::get<0>(x), s1p, s2p, std::get<1>(x), std::get<2>(x), std::get<3>(x));
      }
    }
  }
  for (const auto& y : ylist) {
    int wpp = std::get<0>(y), bi = std::get<4>(y);
    int bp = find(h->right, h->right[3 * bi] + h->cr[2 * wpp], kmod(h->right[3 * bi + 1] + h->cr[2 * wpp + 1], d.mod));
    if (bp >= 0) fl += 8.0 * std::get<5>(y) * std::get<6>(y) * h->right[3 * bp + 2];
  }
  return fl;
}

int mrd_heff_flops(const mrd_heff* h, double* flops4) try {
  if (!h || !flops4) return MRD_E_ARG;
  if (!h->def_flops_done) {
    h->def_flops = definition_flops(h);
    h->def_flops_done = true;
  }
  flops4[0] = h->def_flops;
  flops4[1] = (double)h->counts[C_FLOPS1] + (double)h->counts[C_FLOPS2];
  flops4[2] = (double)h->counts[C_FLOPS1];
  flops4[3] = (double)h->counts[C_FLOPS2];
  return MRD_OK;
} catch (...) {   // host memory or threads exhausted: no exception crosses the C ABI
  return MRD_E_HOST;
}

struct ApplyArg {
  mrd_heff* h;
  int32_t prec;
};

static int apply_cb(void* op, const double2* in, double2* out) {
  ApplyArg* a = (ApplyArg*)op;
  return mrd_heff_apply(a->h, (const double*)in, (double*)out, a->prec);
}

// after each replay of a step graph captured with timing: the GEMM times of its apply
static int replay_timing_cb(void* op) {
  mrd_heff* h = static_cast<ApplyArg*>(op)->h;
  float a = 0.f, b = 0.f;
  MRD_CUDA(h->ctx, cudaEventElapsedTime(&a, h->gev[0], h->gev[1]));
  MRD_CUDA(h->ctx, cudaEventElapsedTime(&b, h->gev[1], h->gev[2]));
  h->gms[0] += a;
  h->gms[1] += b;
  ++h->gcalls;
  return MRD_OK;
}

static int ensure_lanczos(mrd_heff* h) {
  if (h->lz) return MRD_OK;
  cudaError_t e = lanczos_alloc(&h->lz, h->counts[C_THETA], h->ctx->stream);
  if (e != cudaSuccess) return mrd_cuda_fail(h->ctx, e, "Lanczos workspace");
  return MRD_OK;
}

int mrd_lanczos(mrd_heff* h, double* theta_dev, int32_t max_iter, double tol, int32_t prec, double* energy,
                int32_t* iters) try {
  if (!h || !energy || !iters) return MRD_E_ARG;
  mrd_ctx* ctx = h->ctx;
  if (!h->env_loaded) return mrd_fail(ctx, MRD_E_STATE, "mrd_lanczos: environments not loaded");
  if (!theta_dev || h->counts[C_THETA] == 0) return mrd_fail(ctx, MRD_E_ARG, "mrd_lanczos: empty or null theta");
  Guard g(ctx->device);
  int rc = ensure_lanczos(h);
  if (rc != MRD_OK) return rc;
  if (prec != MRD_PREC_FP64 && prec != MRD_PREC_TF32 && prec != MRD_PREC_BF16X3 && prec != MRD_PREC_FF)
    return mrd_fail(ctx, MRD_E_ARG, "mrd_lanczos: unsupported precision");
  if ((rc = heff_prepare(h, prec)) != MRD_OK) return rc;
  ApplyArg arg{h, prec};
  int it = 0;
  // one Lanczos step is captured as a CUDA graph and replayed; the key changes whenever the
  // operator's buffers are reallocated, and a graph captured with GEMM timing records the
  // apply's events at every replay (read back after each one)
  if (h->timing)
    for (cudaEvent_t& ev : h->gev)
      if (!ev) MRD_CUDA(ctx, cudaEventCreate(&ev));
  // with tensor-core matvecs (~1e-5 .. 1e-3 relative) the full reorthogonalisation pass runs
  // in FP32; FP64 and float-float runs keep it in FP64
  MRD_CUDA(ctx, lanczos_set_fp32_full(h->lz, prec == MRD_PREC_TF32 || prec == MRD_PREC_BF16X3));
  const uint64_t key =
      h->use_graph ? ((uint64_t)h->gen << 8 | (h->timing ? 0x80u : 0u) | (uint64_t)(prec + 1)) : 0;
  rc = lanczos_run(h->lz, ctx, apply_cb, &arg, (double2*)theta_dev, max_iter, tol, energy, &it, nullptr, key,
                   h->timing ? replay_timing_cb : nullptr);
  *iters = it;
  if (rc == MRD_OK && (prec == MRD_PREC_TF32 || prec == MRD_PREC_BF16X3)) rc = tc_status(h);
  return rc;
} catch (...) {   // host memory or threads exhausted: no exception crosses the C ABI
  return MRD_E_HOST;
}

int mrd_heff_rayleigh(mrd_heff* h, const double* theta_dev, int32_t prec, double* energy, double* residual) try {
  if (!h || !energy) return MRD_E_ARG;
  mrd_ctx* ctx = h->ctx;
  if (!theta_dev || h->counts[C_THETA] == 0) return mrd_fail(ctx, MRD_E_ARG, "mrd_heff_rayleigh: empty theta");
  Guard g(ctx->device);
  int rc = ensure_lanczos(h);
  if (rc != MRD_OK) return rc;
  double2* hv = lanczos_work(h->lz);   // the workspace's spare vector
  rc = mrd_heff_apply(h, theta_dev, (double*)hv, prec);
  if (rc == MRD_OK && (prec == MRD_PREC_TF32 || prec == MRD_PREC_BF16X3)) rc = tc_status(h);
  if (rc != MRD_OK) return rc;
  double nn, ni, en, ei;
  if ((rc = vdot(h->lz, ctx, (const double2*)theta_dev, (const double2*)theta_dev, &nn, &ni)) != MRD_OK) return rc;
  if ((rc = vdot(h->lz, ctx, (const double2*)theta_dev, hv, &en, &ei)) != MRD_OK) return rc;
  if (!(nn > 0)) return mrd_fail(ctx, MRD_E_ARG, "mrd_heff_rayleigh: zero vector");
  const double e = en / nn;
  *energy = e;
  if (residual) {
    double hh, hi;
    if ((rc = vdot(h->lz, ctx, hv, hv, &hh, &hi)) != MRD_OK) return rc;
    // |Hv - E v|^2 = <Hv,Hv> - 2 E Re<v,Hv> + E^2 <v,v>
    double r2 = hh - 2.0 * e * en + e * e * nn;
    *residual = std::sqrt(r2 > 0 ? r2 : 0.0) / std::sqrt(nn);
  }
  return MRD_OK;
} catch (...) {   // host memory or threads exhausted: no exception crosses the C ABI
  return MRD_E_HOST;
}

int mrd_heff_set_option(mrd_heff* h, int32_t option, int64_t value) try {
  if (!h) return MRD_E_ARG;
  if (option == MRD_OPT_GRAPH) {
    h->use_graph = value != 0;
  } else if (option == MRD_OPT_AUTOTUNE) {
    h->autotune = value != 0;
  } else if (option == MRD_OPT_PER_TASK_LAUNCH) {
    h->per_task = value != 0;
    if (h->tc) tc_env_changed(h);   // tensor-core per-task tables are built with the panels
    ++h->gen;
  } else if (option == MRD_OPT_REAL) {
    const bool on = value != 0;
    if (on)   // the MPO entries must be real (the sine / cosine machine)
      for (const std::vector<double>* v : {&h->wi_v, &h->wj_v})
        for (size_t k = 1; k < v->size(); k += 2)
          if ((*v)[k] != 0.0) return mrd_fail(h->ctx, MRD_E_ARG, "mrd_heff_set_option: MRD_OPT_REAL needs real MPO entries");
    if (on != h->real) {
      h->real = on;
      if (h->tc) { tc_free(h->tc); h->tc = nullptr; }   // panels of the other format
      ++h->gen;
    }
  } else if (option == MRD_OPT_WAIT_LIMIT_US) {
    if (value < 0 || value > 60000000) return mrd_fail(h->ctx, MRD_E_ARG, "mrd_heff_set_option: wait limit outside 0 .. 60 s");
    h->wait_ns = (uint64_t)value * 1000ull;
    ++h->gen;   // captured step graphs hold the old limit in their launch arguments
  } else {
    return mrd_fail(h->ctx, MRD_E_ARG, "mrd_heff_set_option: unknown option");
  }
  return MRD_OK;
} catch (...) {   // host memory or threads exhausted: no exception crosses the C ABI
  return MRD_E_HOST;
}

int mrd_heff_status(mrd_heff* h) try {
  if (!h) return MRD_E_ARG;
  Guard g(h->ctx->device);
  MRD_CUDA(h->ctx, cudaStreamSynchronize(h->ctx->stream));
  return tc_status(h);
} catch (...) {   // host memory or threads exhausted: no exception crosses the C ABI
  return MRD_E_HOST;
}

int mrd_heff_tc_config(const mrd_heff* h, int32_t* cfg4) try {
  if (!h || !cfg4) return MRD_E_ARG;
  return tc_config(h, cfg4);
} catch (...) {   // host memory or threads exhausted: no exception crosses the C ABI
  return MRD_E_HOST;
}

int mrd_heff_timing(mrd_heff* h, int32_t on) try {
  if (!h) return MRD_E_ARG;
  h->timing = on != 0;
  return MRD_OK;
} catch (...) {   // host memory or threads exhausted: no exception crosses the C ABI
  return MRD_E_HOST;
}

int mrd_heff_timing_collect(mrd_heff* h, double* ms_step1, double* ms_step2, int32_t* n_calls) try {
  if (!h) return MRD_E_ARG;
  mrd_ctx* ctx = h->ctx;
  Guard g(ctx->device);
  double a = 0.0, b = 0.0;
  const size_t n = h->ev.size() / 3;
  if (n) MRD_CUDA(ctx, cudaEventSynchronize(h->ev.back()));
  for (size_t i = 0; i < n; ++i) {
    float x = 0.f, y = 0.f;
    MRD_CUDA(ctx, cudaEventElapsedTime(&x, h->ev[3 * i], h->ev[3 * i + 1]));
    MRD_CUDA(ctx, cudaEventElapsedTime(&y, h->ev[3 * i + 1], h->ev[3 * i + 2]));
    a += x;
    b += y;
  }
  for (cudaEvent_t e : h->ev) h->ev_pool.push_back(e);
  h->ev.clear();
  a += h->gms[0];
  b += h->gms[1];
  const int32_t calls = (int32_t)n + h->gcalls;
  h->gms[0] = h->gms[1] = 0.0;
  h->gcalls = 0;
  if (ms_step1) *ms_step1 = a;
  if (ms_step2) *ms_step2 = b;
  if (n_calls) *n_calls = calls;
  return MRD_OK;
} catch (...) {   // host memory or threads exhausted: no exception crosses the C ABI
  return MRD_E_HOST;
}

int mrd_heff_table(const mrd_heff* h, int32_t which, int64_t* rows, int64_t* count) try {
  if (!h || !count) return MRD_E_ARG;
  mrd_ctx* ctx = h->ctx;
  Guard g(ctx->device);
  if (which == 0) {
    const int64_t n = h->counts[C_NMID];
    *count = n;
    if (!rows) return MRD_OK;
    std::vector<int64_t> mid(MIDF * n);
    MRD_CUDA(ctx, cudaMemcpy(mid.data(), h->p.mid, mid.size() * 8, cudaMemcpyDeviceToHost));
    for (int64_t i = 0; i < n; ++i) {
      const int64_t* r = &mid[MIDF * i];
      int64_t* o = rows + 8 * i;
      int64_t flags = (r[5] >= 0 ? 1 : 0) | (r[6] >= 0 ? 2 : 0) | (r[8] >= 0 ? 4 : 0) | (r[9] >= 0 ? 8 : 0);
      o[0] = r[0]; o[1] = r[1]; o[2] = r[2]; o[3] = r[3]; o[4] = r[4];
      o[5] = r[6] >= 0 ? r[7] : -1; o[6] = r[9] >= 0 ? r[10] : -1; o[7] = flags;
    }
    return MRD_OK;
  }
  if (which == 1 || which == 2) {
    const bool lft = which == 1;
    const int nsec = lft ? h->d.n_l : h->d.n_r, nch = lft ? h->d.d_l : h->d.d_r;
    std::vector<int64_t> map((size_t)nsec * nch);
    MRD_CUDA(ctx, cudaMemcpy(map.data(), lft ? h->p.lmap : h->p.rmap, map.size() * 8, cudaMemcpyDeviceToHost));
    const std::vector<int32_t>& sec = lft ? h->left : h->right;
    const std::vector<int32_t>& ch = lft ? h->cl : h->cr;
    int64_t k = 0;
    for (int w = 0; w < nch; ++w)
      for (int x = 0; x < nsec; ++x) {
        int64_t off = map[(size_t)w * nsec + x];
        if (off < 0) continue;
        if (rows) {
          int N = sec[3 * x] + ch[2 * w], K = kmod(sec[3 * x + 1] + ch[2 * w + 1], h->d.mod);
          int xp = -1;
          for (int i = 0; i < nsec; ++i) if (sec[3 * i] == N && sec[3 * i + 1] == K) xp = i;
          int64_t* o = rows + 6 * k;
          o[0] = w; o[1] = x; o[2] = xp; o[3] = off;
          o[4] = lft ? sec[3 * xp + 2] : sec[3 * x + 2];
          o[5] = lft ? sec[3 * x + 2] : sec[3 * xp + 2];
        }
        ++k;
      }
    *count = k;
    return MRD_OK;
  }
  return mrd_fail(ctx, MRD_E_ARG, "mrd_heff_table: unknown table");
} catch (...) {   // host memory or threads exhausted: no exception crosses the C ABI
  return MRD_E_HOST;
}

}  // extern "C"

// Start the float-float conversion of LW / WR (asynchronous device work) ahead of a
// float-float application, e.g. so that it runs while the host builds the tensor-core tables.
int heff_prefetch_ff(mrd_heff* h) {
  Guard g(h->ctx->device);
  return heff_prepare(h, MRD_PREC_FF);
}

namespace mrd {

// Read-only view of a handle for mrd_heff_apply_noalloc (heff_noalloc.cu).
int mrd_heff_internal_noalloc_view(const mrd_heff* h, PlanPtrs* p, int64_t* counts, const double2** lw,
                                   const double2** wr, int* n_sm, mrd_ctx** ctx, bool* env_loaded) {
  *p = h->p;
  for (int i = 0; i < C_NCOUNTS; ++i) counts[i] = h->counts[i];
  *lw = h->lw;
  *wr = h->wr;
  *n_sm = h->n_sm;
  *ctx = h->ctx;
  *env_loaded = h->env_loaded;
  return MRD_OK;
}

}  // namespace mrd
