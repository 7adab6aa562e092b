// Device construction of the charge tables of a two-site problem (one CTA, deterministic).
//
// Charges are (N, K mod M) with the onsite Z_Ly momentum of the mixed basis (Sec. II); a
// site with momentum index m has q(s) = (s, s m mod M). Everything below is integer
// bookkeeping that fixes where each dense charge block lives in memory:
//   * fused middle sectors q_m of theta: rows (s1, a) with q_a + q1(s1) = q_m, columns
//     (s2, b) with q_b - q2(s2) = q_m, sorted by (N, K), with flat offsets;
//   * left / right environment block offsets (order: channel, then sector);
//   * the folded operands LW_{w'}^{(s1',s1)} = sum_w W_i[w,w',s1',s1] L_w and
//     WR_{w'}^{(s2,s2')} = sum_{w''} W_{i+1}[w',w'',s2',s2] R_{w''}, one dense block each;
//   * the intermediate Z_{w'} = LW_{w'} theta, one block per (w', input middle sector);
//   * two grouped-GEMM task lists: step 1 (Z = LW theta) and step 2
//     (theta' = sum_{w'} Z_{w'} WR_{w'}), each task a dense output block accumulated over
//     a list of K segments, plus the exclusive prefix of its 32 x 32 output tiles.
// Task item spaces are dense (tasks with no work have zero tiles), so the order is fixed by
// the charges alone and the tables are bit-exact run to run.
#include "mrd_internal.h"
#include "plan.cuh"

namespace mrd {

namespace {

constexpr int kTile = 32;

__device__ int64_t block_scan(int64_t* v, int64_t n, int64_t* smem) {
  // exclusive prefix sum in place over v[0..n); returns the total. All threads call it; the
  // CTA has a multiple of 32 threads, at most 1024. Each thread sums a contiguous chunk; the
  // chunk sums are scanned by shuffles within each warp and then over the warps' totals.
  const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, wid = tid >> 5, nw = nt >> 5;
  const int64_t chunk = (n + nt - 1) / nt;
  const int64_t b = tid * chunk;
  const int64_t e = b + chunk < n ? b + chunk : n;
  int64_t s = 0;
  for (int64_t i = b; i < e; ++i) s += v[i];
  int64_t x = s;   // inclusive prefix of the chunk sums within the warp
  for (int o = 1; o < 32; o <<= 1) {
    const int64_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) smem[wid] = x;
  __syncthreads();
  if (wid == 0) {   // inclusive prefix of the warps' totals
    int64_t t = lane < nw ? smem[lane] : 0;
    for (int o = 1; o < 32; o <<= 1) {
      const int64_t y = __shfl_up_sync(0xffffffffu, t, o);
      if (lane >= o) t += y;
    }
    smem[32 + lane] = t;
  }
  __syncthreads();
  int64_t acc = (wid > 0 ? smem[32 + wid - 1] : 0) + x - s;
  const int64_t total = smem[32 + nw - 1];
  for (int64_t i = b; i < e; ++i) {
    const int64_t y = v[i];
    v[i] = acc;
    acc += y;
  }
  __syncthreads();
  return total;
}

__device__ __forceinline__ int kmod(int k, int mod) { return ((k % mod) + mod) % mod; }

// Binary search of (N, K) in a sorted (N, K, dim) table; -1 if absent.
__device__ int find_sector(const int32_t* sec, int n, int N, int K) {
  int64_t key = qkey(N, K);
  int lo = 0, hi = n - 1;
  while (lo <= hi) {
    int mid = (lo + hi) >> 1;
    int64_t k = qkey(sec[3 * mid], sec[3 * mid + 1]);
    if (k == key) return mid;
    if (k < key) lo = mid + 1; else hi = mid - 1;
  }
  return -1;
}

__device__ int find_mid(const int64_t* mid, int n, int N, int K) {
  int64_t key = qkey(N, K);
  int lo = 0, hi = n - 1;
  while (lo <= hi) {
    int m = (lo + hi) >> 1;
    int64_t k = qkey((int32_t)mid[MIDF * m], (int32_t)mid[MIDF * m + 1]);
    if (k == key) return m;
    if (k < key) lo = m + 1; else hi = m - 1;
  }
  return -1;
}

// Binary search of a key in a sorted key array; -1 if absent.
__device__ int find_key(const int64_t* keys, int n, int64_t key) {
  int lo = 0, hi = n - 1;
  while (lo <= hi) {
    const int m = (lo + hi) >> 1;
    const int64_t k = keys[m];
    if (k == key) return m;
    if (k < key) lo = m + 1; else hi = m - 1;
  }
  return -1;
}

// middle-sector keys kept in shared memory for the lookups of steps 5 and 7 (global otherwise)
constexpr int kMidKeys = 2048;

__device__ __forceinline__ int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }

}  // namespace

__global__ void __launch_bounds__(1024) k_plan(PlanDims d, PlanPtrs p) {
  __shared__ int64_t smem[1025];
  __shared__ int64_t mkey[kMidKeys];
  const int tid = threadIdx.x, nt = blockDim.x;
  const int M = d.mod;
  const int32_t *L = p.left, *Rs = p.right;

  // ---- P1: sort MPO entries by (w', s1', s1, w) and (w', s2, s2', w''); triple ranges
  for (int i = tid; i < d.nnz_i; i += nt) {
    const int32_t* e = p.wi_idx + 4 * i;
    int64_t ki = (((int64_t)e[1] * 2 + e[2]) * 2 + e[3]) * d.d_l + e[0];
    int r = 0;
    for (int j = 0; j < d.nnz_i; ++j) {
      const int32_t* f = p.wi_idx + 4 * j;
      int64_t kj = (((int64_t)f[1] * 2 + f[2]) * 2 + f[3]) * d.d_l + f[0];
      r += (kj < ki) || (kj == ki && j < i);
    }
    p.wi_perm[r] = i;
  }
  for (int i = tid; i < d.nnz_j; i += nt) {
    const int32_t* e = p.wj_idx + 4 * i;
    // entry (w', w'', s2', s2): key (w', s2, s2', w'')
    int64_t ki = (((int64_t)e[0] * 2 + e[3]) * 2 + e[2]) * d.d_r + e[1];
    int r = 0;
    for (int j = 0; j < d.nnz_j; ++j) {
      const int32_t* f = p.wj_idx + 4 * j;
      int64_t kj = (((int64_t)f[0] * 2 + f[3]) * 2 + f[2]) * d.d_r + f[1];
      r += (kj < ki) || (kj == ki && j < i);
    }
    p.wj_perm[r] = i;
  }
  for (int i = tid; i < d.d_m * 4; i += nt) {
    p.trip_i[2 * i] = p.trip_i[2 * i + 1] = 0;
    p.trip_j[2 * i] = p.trip_j[2 * i + 1] = 0;
  }
  __syncthreads();
  for (int r = tid; r < d.nnz_i; r += nt) {
    const int32_t* e = p.wi_idx + 4 * p.wi_perm[r];
    int trip = (e[1] * 2 + e[2]) * 2 + e[3];
    bool first = r == 0;
    if (!first) { const int32_t* f = p.wi_idx + 4 * p.wi_perm[r - 1]; first = ((f[1] * 2 + f[2]) * 2 + f[3]) != trip; }
    bool last = r == d.nnz_i - 1;
    if (!last) { const int32_t* f = p.wi_idx + 4 * p.wi_perm[r + 1]; last = ((f[1] * 2 + f[2]) * 2 + f[3]) != trip; }
    if (first) p.trip_i[2 * trip] = r;
    if (last) p.trip_i[2 * trip + 1] = r + 1;
  }
  for (int r = tid; r < d.nnz_j; r += nt) {
    const int32_t* e = p.wj_idx + 4 * p.wj_perm[r];
    int trip = (e[0] * 2 + e[3]) * 2 + e[2];
    bool first = r == 0;
    if (!first) { const int32_t* f = p.wj_idx + 4 * p.wj_perm[r - 1]; first = ((f[0] * 2 + f[3]) * 2 + f[2]) != trip; }
    bool last = r == d.nnz_j - 1;
    if (!last) { const int32_t* f = p.wj_idx + 4 * p.wj_perm[r + 1]; last = ((f[0] * 2 + f[3]) * 2 + f[2]) != trip; }
    if (first) p.trip_j[2 * trip] = r;
    if (last) p.trip_j[2 * trip + 1] = r + 1;
  }
  __syncthreads();

  // ---- P2: fused middle sectors
  // candidate i = (a, s1) carries the charge q_a + q1(s1); the distinct charges, in increasing
  // order, are the middle sectors. A candidate that is the first of its charge gets the number
  // of distinct smaller charges as its slot, the others -1. The keys and first-occurrence flags
  // are staged in p.mid, whose rows are written only after this.
  const int ncand = 2 * d.n_l;
  int64_t* ckey = p.mid;
  int64_t* cfirst = p.mid + ncand;
  for (int i = tid; i < ncand; i += nt) {
    const int a = i >> 1, s1 = i & 1;
    ckey[i] = qkey(L[3 * a] + s1, kmod(L[3 * a + 1] + s1 * d.m1, M));
  }
  __syncthreads();
  for (int i = tid; i < ncand; i += nt) {
    const int64_t key = ckey[i];
    int64_t first = 1;
    for (int j = 0; j < i && first; ++j) first = ckey[j] != key;
    cfirst[i] = first;
  }
  __syncthreads();
  for (int i = tid; i < ncand; i += nt) {
    int64_t slot = -1;
    if (cfirst[i]) {
      const int64_t key = ckey[i];
      slot = 0;
      for (int j = 0; j < ncand; ++j) slot += cfirst[j] && ckey[j] < key;
    }
    p.scr_a[i] = slot;
  }
  __syncthreads();
  // candidate slot -> sector data (in scr_b, MIDF per slot; valid flag in scr_a reused)
  for (int i = tid; i < ncand; i += nt) {
    int64_t slot = p.scr_a[i];
    if (slot < 0) continue;
    int a = i >> 1, s1 = i & 1;
    int N = L[3 * a] + s1, K = kmod(L[3 * a + 1] + s1 * d.m1, M);
    int64_t* row = p.mid + MIDF * slot;  // staging, compacted below
    int a0 = find_sector(L, d.n_l, N, K);
    int a1 = find_sector(L, d.n_l, N - 1, kmod(K - d.m1, M));
    int b0 = find_sector(Rs, d.n_r, N, K);
    int b1 = find_sector(Rs, d.n_r, N + 1, kmod(K + d.m2, M));
    int64_t r0 = a0 >= 0 ? L[3 * a0 + 2] : 0, r1 = a1 >= 0 ? L[3 * a1 + 2] : 0;
    int64_t c0 = b0 >= 0 ? Rs[3 * b0 + 2] : 0, c1 = b1 >= 0 ? Rs[3 * b1 + 2] : 0;
    row[0] = N; row[1] = K; row[2] = r0 + r1; row[3] = c0 + c1; row[4] = 0;
    row[5] = a0; row[6] = a1; row[7] = r0; row[8] = b0; row[9] = b1; row[10] = c0; row[11] = 0;
  }
  __syncthreads();
  // number of distinct candidates = number of first occurrences
  for (int i = tid; i < ncand; i += nt) p.scr_b[i] = p.scr_a[i] >= 0 ? 1 : 0;
  __syncthreads();
  const int64_t ndist = block_scan(p.scr_b, ncand, smem);
  for (int i = tid; i < ndist; i += nt) p.scr_b[i] = (p.mid[MIDF * i + 3] > 0) ? 1 : 0;
  __syncthreads();
  const int64_t nmid = block_scan(p.scr_b, ndist, smem);
  // compact in place: slot i moves to scr_b[i] <= i; copy via scr_a staging to avoid overlap
  for (int i = tid; i < ndist; i += nt) {
    bool keep = p.mid[MIDF * i + 3] > 0;
    p.scr_a[i] = keep ? p.scr_b[i] : -1;
  }
  __syncthreads();
  // compaction through a staging copy in p.t1 (12 x its capacity of middle sectors, written
  // only in step 6)
  for (int64_t q = tid; q < ndist * MIDF; q += nt) {
    const int64_t dst = p.scr_a[q / MIDF];
    if (dst >= 0) p.t1[MIDF * dst + q % MIDF] = p.mid[q];
  }
  __syncthreads();
  for (int64_t q = tid; q < nmid * MIDF; q += nt) p.mid[q] = p.t1[q];
  __syncthreads();
  for (int i = tid; i < nmid; i += nt) p.scr_b[i] = p.mid[MIDF * i + 2] * p.mid[MIDF * i + 3];
  __syncthreads();
  const int64_t theta_len = block_scan(p.scr_b, nmid, smem);
  for (int i = tid; i < nmid; i += nt) p.mid[MIDF * i + 4] = p.scr_b[i];
  const bool mkey_ok = nmid <= kMidKeys;
  if (mkey_ok)
    for (int i = tid; i < nmid; i += nt) mkey[i] = qkey((int32_t)p.mid[MIDF * i], (int32_t)p.mid[MIDF * i + 1]);
  __syncthreads();
  auto mid_of = [&](int N, int K) {
    return mkey_ok ? find_key(mkey, (int)nmid, qkey(N, K)) : find_mid(p.mid, (int)nmid, N, K);
  };

  // ---- P3: environment layouts
  for (int64_t i = tid; i < (int64_t)d.d_l * d.n_l; i += nt) {
    int w = (int)(i / d.n_l), a = (int)(i % d.n_l);
    int ap = find_sector(L, d.n_l, L[3 * a] + p.cl[2 * w], kmod(L[3 * a + 1] + p.cl[2 * w + 1], M));
    p.scr_a[i] = ap;
    p.scr_b[i] = ap >= 0 ? (int64_t)L[3 * ap + 2] * L[3 * a + 2] : 0;
  }
  __syncthreads();
  const int64_t lenv_len = block_scan(p.scr_b, (int64_t)d.d_l * d.n_l, smem);
  for (int64_t i = tid; i < (int64_t)d.d_l * d.n_l; i += nt) p.lmap[i] = p.scr_a[i] >= 0 ? p.scr_b[i] : -1;
  __syncthreads();
  for (int64_t i = tid; i < (int64_t)d.d_r * d.n_r; i += nt) {
    int w = (int)(i / d.n_r), b = (int)(i % d.n_r);
    int bp = find_sector(Rs, d.n_r, Rs[3 * b] + p.cr[2 * w], kmod(Rs[3 * b + 1] + p.cr[2 * w + 1], M));
    p.scr_a[i] = bp;
    p.scr_b[i] = bp >= 0 ? (int64_t)Rs[3 * b + 2] * Rs[3 * bp + 2] : 0;
  }
  __syncthreads();
  const int64_t renv_len = block_scan(p.scr_b, (int64_t)d.d_r * d.n_r, smem);
  for (int64_t i = tid; i < (int64_t)d.d_r * d.n_r; i += nt) p.rmap[i] = p.scr_a[i] >= 0 ? p.scr_b[i] : -1;
  __syncthreads();

  // ---- P4: folded operands LW (items (w', s1', s1, a)) and WR (items (w', s2, s2', b))
  const int64_t n_lw_items = (int64_t)d.d_m * 4 * d.n_l;
  for (int64_t i = tid; i < n_lw_items; i += nt) {
    int a = (int)(i % d.n_l);
    int trip = (int)(i / d.n_l);
    int s1 = trip & 1, s1p = (trip >> 1) & 1, wp = trip >> 2;
    int ap = -1;
    if (p.trip_i[2 * trip + 1] > p.trip_i[2 * trip]) {
      int dN = p.cm[2 * wp] - s1p + s1;
      int dK = p.cm[2 * wp + 1] - s1p * d.m1 + s1 * d.m1;
      ap = find_sector(L, d.n_l, L[3 * a] + dN, kmod(L[3 * a + 1] + dK, M));
    }
    p.lwmap[i] = ap;  // staged
    p.scr_a[i] = ap >= 0 ? 1 : 0;
    p.scr_b[i] = ap >= 0 ? (int64_t)L[3 * ap + 2] * L[3 * a + 2] : 0;
  }
  __syncthreads();
  const int64_t n_lw = block_scan(p.scr_a, n_lw_items, smem);
  const int64_t lw_len = block_scan(p.scr_b, n_lw_items, smem);
  for (int64_t i = tid; i < n_lw_items; i += nt) {
    int ap = (int)p.lwmap[i];
    if (ap < 0) continue;
    int a = (int)(i % d.n_l);
    int trip = (int)(i / d.n_l);
    int64_t id = p.scr_a[i];
    int64_t* row = p.lw + LWF * id;
    row[0] = trip >> 2; row[1] = (trip >> 1) & 1; row[2] = trip & 1; row[3] = a; row[4] = ap;
    row[5] = L[3 * ap + 2]; row[6] = L[3 * a + 2]; row[7] = p.scr_b[i];
    row[8] = p.trip_i[2 * trip]; row[9] = p.trip_i[2 * trip + 1];
  }
  __syncthreads();
  for (int64_t i = tid; i < n_lw_items; i += nt) p.lwmap[i] = p.lwmap[i] >= 0 ? p.scr_a[i] : -1;
  __syncthreads();

  const int64_t n_wr_items = (int64_t)d.d_m * 4 * d.n_r;
  for (int64_t i = tid; i < n_wr_items; i += nt) {
    int b = (int)(i % d.n_r);
    int trip = (int)(i / d.n_r);
    int s2p = trip & 1, s2 = (trip >> 1) & 1, wp = trip >> 2;
    int bp = -1;
    if (p.trip_j[2 * trip + 1] > p.trip_j[2 * trip]) {
      // c_{w''} = c_{w'} + q2(s2') - q2(s2); b' = b + c_{w''}
      int dN = p.cm[2 * wp] + s2p - s2;
      int dK = p.cm[2 * wp + 1] + s2p * d.m2 - s2 * d.m2;
      bp = find_sector(Rs, d.n_r, Rs[3 * b] + dN, kmod(Rs[3 * b + 1] + dK, M));
    }
    p.wrmap[i] = bp;
    p.scr_a[i] = bp >= 0 ? 1 : 0;
    p.scr_b[i] = bp >= 0 ? (int64_t)Rs[3 * b + 2] * Rs[3 * bp + 2] : 0;
  }
  __syncthreads();
  const int64_t n_wr = block_scan(p.scr_a, n_wr_items, smem);
  const int64_t wr_len = block_scan(p.scr_b, n_wr_items, smem);
  for (int64_t i = tid; i < n_wr_items; i += nt) {
    int bp = (int)p.wrmap[i];
    if (bp < 0) continue;
    int b = (int)(i % d.n_r);
    int trip = (int)(i / d.n_r);
    int64_t id = p.scr_a[i];
    int64_t* row = p.wr + WRF * id;
    row[0] = trip >> 2; row[1] = (trip >> 1) & 1; row[2] = trip & 1; row[3] = b; row[4] = bp;
    row[5] = Rs[3 * b + 2]; row[6] = Rs[3 * bp + 2]; row[7] = p.scr_b[i];
    row[8] = p.trip_j[2 * trip]; row[9] = p.trip_j[2 * trip + 1];
  }
  __syncthreads();
  for (int64_t i = tid; i < n_wr_items; i += nt) p.wrmap[i] = p.wrmap[i] >= 0 ? p.scr_a[i] : -1;
  __syncthreads();

  // ---- P5: Z blocks, items (w', m_in); rows of s1' written when an LW block feeds them
  const int64_t n_z_items = (int64_t)d.d_m * nmid;
  for (int64_t i = tid; i < n_z_items; i += nt) {
    int wp = (int)(i / nmid), mi = (int)(i % nmid);
    const int64_t* min_ = p.mid + MIDF * mi;
    int mo = mid_of((int)min_[0] + p.cm[2 * wp], kmod((int)min_[1] + p.cm[2 * wp + 1], M));
    int mask = 0;
    if (mo >= 0) {
      const int64_t* mout = p.mid + MIDF * mo;
      for (int s1p = 0; s1p < 2; ++s1p) {
        if (mout[5 + s1p] < 0) continue;
        for (int s1 = 0; s1 < 2; ++s1) {
          int64_t a = min_[5 + s1];
          if (a < 0) continue;
          if (p.lwmap[(((int64_t)wp * 2 + s1p) * 2 + s1) * d.n_l + a] >= 0) mask |= 1 << s1p;
        }
      }
    }
    p.s1mask[i] = mask;
    p.zmap[i] = mask ? mo : -1;  // staged: m_out
    p.scr_a[i] = mask ? 1 : 0;
    p.scr_b[i] = mask ? p.mid[MIDF * mo + 2] * min_[3] : 0;
  }
  __syncthreads();
  const int64_t n_z = block_scan(p.scr_a, n_z_items, smem);
  const int64_t z_len = block_scan(p.scr_b, n_z_items, smem);
  for (int64_t i = tid; i < n_z_items; i += nt) {
    int64_t mo = p.zmap[i];
    if (mo < 0) continue;
    int64_t id = p.scr_a[i];
    int64_t* row = p.z + ZF * id;
    row[0] = i / nmid; row[1] = i % nmid; row[2] = mo; row[3] = p.mid[MIDF * mo + 2];
    row[4] = p.mid[MIDF * (i % nmid) + 3]; row[5] = p.scr_b[i];
    p.zmap[i] = id;
  }
  __syncthreads();

  // ---- P6: step-1 tasks, items (w', m_in, s1'): Z_{w'}[rows s1'] = sum_s1 LW theta[rows s1]
  const int64_t n_t1 = (int64_t)d.d_m * nmid * 2;
  for (int64_t i = tid; i < n_t1; i += nt) {
    int s1p = (int)(i & 1);
    int64_t zi = i >> 1;  // = w' * nmid + m_in
    int wp = (int)(zi / nmid), mi = (int)(zi % nmid);
    int64_t* task = p.t1 + TF * i;
    int64_t zid = p.zmap[zi];
    int cnt = 0;
    int64_t Mrows = 0, Ncols = 0, flops = 0;
    if (zid >= 0 && (p.s1mask[zi] >> s1p & 1)) {
      const int64_t* zrow = p.z + ZF * zid;
      const int64_t* min_ = p.mid + MIDF * mi;
      const int64_t* mout = p.mid + MIDF * zrow[2];
      int64_t ap = mout[5 + s1p];
      Mrows = L[3 * ap + 2];
      Ncols = min_[3];
      int64_t rowoff_out = s1p ? mout[7] : 0;
      task[2] = zrow[5] + rowoff_out * Ncols;
      task[3] = Ncols;
      for (int s1 = 0; s1 < 2; ++s1) {
        int64_t a = min_[5 + s1];
        if (a < 0) continue;
        int64_t lwid = p.lwmap[(((int64_t)wp * 2 + s1p) * 2 + s1) * d.n_l + a];
        if (lwid < 0) continue;
        int64_t* seg = p.seg1 + SF * (2 * i + cnt);
        int64_t K = L[3 * a + 2];
        seg[0] = p.lw[LWF * lwid + 7];
        seg[1] = K;
        seg[2] = min_[4] + (s1 ? min_[7] : 0) * Ncols;
        seg[3] = Ncols;
        seg[4] = K;
        seg[5] = 0;
        flops += 8 * Mrows * Ncols * K;
        ++cnt;
      }
    }
    if (cnt == 0) { Mrows = 0; Ncols = 0; task[2] = 0; task[3] = 0; }
    task[0] = Mrows; task[1] = Ncols; task[4] = 2 * i; task[5] = cnt;
    p.tile1[i] = ceil_div(Mrows, kTile) * ceil_div(Ncols, kTile);
    p.scr_b[i] = flops;
  }
  __syncthreads();
  const int64_t tiles1 = block_scan(p.tile1, n_t1, smem);
  if (tid == 0) p.tile1[n_t1] = tiles1;
  const int64_t flops1 = block_scan(p.scr_b, n_t1, smem);

  // ---- P7: step-2 tasks, items (m_out, s1', s2'): theta'[s1', s2'] = sum_{w', s2} Z WR
  const int64_t n_t2 = nmid * 4;
  for (int64_t i = tid; i < n_t2; i += nt) {
    int mo = (int)(i >> 2), s1p = (int)((i >> 1) & 1), s2p = (int)(i & 1);
    const int64_t* mout = p.mid + MIDF * mo;
    int64_t* task = p.t2 + TF * i;
    int cnt = 0;
    int64_t Mrows = 0, Ncols = 0, flops = 0;
    int64_t ap = mout[5 + s1p], bp = mout[8 + s2p];
    if (ap >= 0 && bp >= 0) {
      Mrows = L[3 * ap + 2];
      Ncols = Rs[3 * bp + 2];
      int64_t rowoff_out = s1p ? mout[7] : 0;
      int64_t coloff_out = s2p ? mout[10] : 0;
      task[2] = mout[4] + rowoff_out * mout[3] + coloff_out;
      task[3] = mout[3];
      for (int wp = 0; wp < d.d_m; ++wp) {
        int mi = mid_of((int)mout[0] - p.cm[2 * wp], kmod((int)mout[1] - p.cm[2 * wp + 1], M));
        if (mi < 0) continue;
        int64_t zi = (int64_t)wp * nmid + mi;
        int64_t zid = p.zmap[zi];
        if (zid < 0 || !(p.s1mask[zi] >> s1p & 1)) continue;
        const int64_t* min_ = p.mid + MIDF * mi;
        for (int s2 = 0; s2 < 2; ++s2) {
          int64_t b = min_[8 + s2];
          if (b < 0) continue;
          int64_t wrid = p.wrmap[(((int64_t)wp * 2 + s2) * 2 + s2p) * d.n_r + b];
          if (wrid < 0) continue;
          int64_t* seg = p.seg2 + SF * (i * d.seg2_stride + cnt);
          int64_t K = Rs[3 * b + 2];
          seg[0] = p.z[ZF * zid + 5] + rowoff_out * min_[3] + (s2 ? min_[10] : 0);
          seg[1] = min_[3];
          seg[2] = p.wr[WRF * wrid + 7];
          seg[3] = Ncols;
          seg[4] = K;
          seg[5] = 0;
          flops += 8 * Mrows * Ncols * K;
          ++cnt;
        }
      }
    }
    if (cnt == 0) { Mrows = 0; Ncols = 0; task[2] = 0; task[3] = 0; }
    task[0] = Mrows; task[1] = Ncols; task[4] = i * d.seg2_stride; task[5] = cnt;
    p.tile2[i] = ceil_div(Mrows, kTile) * ceil_div(Ncols, kTile);
    p.scr_b[i] = flops;
  }
  __syncthreads();
  const int64_t tiles2 = block_scan(p.tile2, n_t2, smem);
  if (tid == 0) p.tile2[n_t2] = tiles2;
  const int64_t flops2 = block_scan(p.scr_b, n_t2, smem);

  if (tid == 0) {
    int64_t* c = p.counts;
    c[C_NMID] = nmid; c[C_THETA] = theta_len; c[C_LENV] = lenv_len; c[C_RENV] = renv_len;
    c[C_NLW] = n_lw; c[C_LWLEN] = lw_len; c[C_NWR] = n_wr; c[C_WRLEN] = wr_len;
    c[C_NZ] = n_z; c[C_ZLEN] = z_len; c[C_NT1] = n_t1; c[C_NT2] = n_t2;
    c[C_TILES1] = tiles1; c[C_TILES2] = tiles2; c[C_FLOPS1] = flops1; c[C_FLOPS2] = flops2;
    c[C_ERR] = 0;
  }
}

cudaError_t launch_plan(const PlanDims& d, const PlanPtrs& p, cudaStream_t s) {
  k_plan<<<1, 1024, 0, s>>>(d, p);
  mrd::count_launch();
  return cudaGetLastError();
}

}  // namespace mrd
