// Host side of the tensor-core H_eff: packed-panel tables (derived on the host from the
// device-built charge tables of plan.cu), packing of the folded environments and of theta,
// and the two grouped-GEMM launches.
#include <algorithm>
#include <map>
#include <new>
#include <queue>
#include <thread>
#include <vector>

#include "heff_internal.h"
#include "tc.cuh"

namespace mrd {
cudaError_t tc_pack(const double2* src, uint8_t* dst, const int64_t* jobs, int njobs, int64_t npieces, int prec,
                    cudaStream_t s);
cudaError_t tc_gemm_init();
cudaError_t tc_gemm(const uint8_t* a_base, const uint8_t* b_base, const int64_t* tasks, const int64_t* segs,
                    const int64_t* prefix, const int2* items, const int32_t* cta_off, const int64_t* rowmap,
                    int64_t n_tasks, int64_t total_tiles, uint8_t* z_out, double2* f_out, int prec, TcCfg cfg,
                    int* err, int n_sm, uint64_t wait_ns, cudaStream_t s);
}  // namespace mrd

struct Tc {
  int prec = 0;
  TcCfg cfg{0, 0, 0};
  int cfg_source = 0;   // 0: default, 1: tuned on this H_eff, 2: tuned earlier on this context
  bool env_dirty = true;
  Arena mem;
  uint8_t *lw = nullptr, *wr = nullptr, *th = nullptr, *z = nullptr;
  int64_t lw_bytes = 0, wr_bytes = 0, th_bytes = 0, z_bytes = 0;
  int64_t *t1 = nullptr, *s1 = nullptr, *p1 = nullptr, *t2 = nullptr, *s2 = nullptr, *p2 = nullptr;
  int64_t n1 = 0, ntiles1 = 0, n2 = 0, ntiles2 = 0;
  int64_t *j_lw = nullptr, *j_wr = nullptr, *j_th = nullptr;
  int n_lw = 0, n_wr = 0, n_th = 0;
  int64_t pc_lw = 0, pc_wr = 0, pc_th = 0;   // pack pieces of each job list
  // per-task launches: [0, tiles of task t] pairs (device) and tiles per task (host)
  int64_t *pt1 = nullptr, *pt2 = nullptr;
  std::vector<int64_t> tiles1, tiles2;
  int2 *it1 = nullptr, *it2 = nullptr;   // item tables of the grouped launches
  int32_t *co1 = nullptr, *co2 = nullptr; // first item of each CTA in them (grid + 1 entries)
  int64_t* rmap1 = nullptr;               // step-1 row map: (Z panel byte offset << 16) | row in panel
  int* err = nullptr;
};

void tc_free(Tc* t) { delete t; }

// Tensor-core precision of an application: complex, or real when the H_eff is declared real
// (MRD_OPT_REAL).
int tc_prec_of(const mrd_heff* h, int32_t prec) {
  if (prec == MRD_PREC_TF32) return h->real ? TC_TF32_REAL : TC_TF32;
  return h->real ? TC_BF16X3_REAL : TC_BF16X3;
}

namespace {

int64_t round_up(int64_t a, int64_t b) { return (a + b - 1) / b * b; }

struct Panel {
  int64_t off, nkt;
};

// Panels keyed by the FP64 element offset of their block: appended in build order, sorted once
// (stably, so that of equal keys, e.g. an empty block and the one after it, the last appended
// wins), then found by binary search. Tens of thousands of lookups per H_eff: a sorted vector
// avoids the per-node allocations and pointer chasing of a tree map.
struct PanelIndex {
  std::vector<std::pair<int64_t, Panel>> v;
  void add(int64_t key, Panel p) { v.push_back({key, p}); }
  void finish() {
    auto lt = [](const std::pair<int64_t, Panel>& a, const std::pair<int64_t, Panel>& b) { return a.first < b.first; };
    if (!std::is_sorted(v.begin(), v.end(), lt)) std::stable_sort(v.begin(), v.end(), lt);
  }
  const Panel* find(int64_t key) const {
    auto it = std::upper_bound(v.begin(), v.end(), key,
                               [](int64_t k, const std::pair<int64_t, Panel>& e) { return k < e.first; });
    if (it == v.begin()) return nullptr;
    --it;
    return it->first == key ? &it->second : nullptr;
  }
};

// bytes of an A panel (128-row tiles) or a B panel (ntile-row tiles, rows padded to 16)
int64_t a_bytes(int64_t rows, int64_t nkt, int planes) { return round_up(rows, 128) * nkt * planes * 128; }
int64_t b_bytes(int64_t rows, int64_t nkt, int planes) { return round_up(rows, 16) * nkt * planes * 128; }

// Host tables of the tensor-core path for one precision and tile configuration: panel
// layouts, pack jobs, tasks, segments, row map and the per-CTA item deal. Built without any
// device call, so that a host thread can build them while the device works (tc_prebuild).
struct TcTables {
  int prec = 0;
  TcCfg cfg{0, 0, 0};
  int n_sm = 0;
  std::vector<int64_t> j_lw, j_wr, j_th, t1, s1, p1, t2, s2, p2, q1, q2, rowmap;
  std::vector<int2> i1, i2;
  std::vector<int32_t> co1, co2;
  int64_t lw_b = 0, wr_b = 0, th_b = 0, z_b = 0, pc_lw = 0, pc_wr = 0, pc_th = 0;
  const char* err = nullptr;   // why the tables could not be built
};

bool tables(const mrd_heff* h, int prec, TcCfg cfg, TcTables& o) {
  auto fail = [&](const char* m) { o.err = m; return false; };
  o.prec = prec;
  o.cfg = cfg;
  o.n_sm = h->n_sm;
  const int aplanes = tc_aplanes(prec), bplanes = tc_bplanes(prec), kpt = tc_kpt(prec), ntile = cfg.ntile;
  const int64_t* c = h->counts;
  PanelIndex wr_map, th_map, z_map;
  wr_map.v.reserve(c[C_NWR]);
  std::vector<int64_t>&j_lw = o.j_lw, &j_wr = o.j_wr, &j_th = o.j_th;
  int64_t &lw_b = o.lw_b, &wr_b = o.wr_b, &th_b = o.th_b, &z_b = o.z_b;
  // (the folded left operand LW is packed below, stacked by input middle sector)
  // folded right operand WR(w', s2, s2', b): B panel of its transpose, rows d_b', K d_b
  for (int64_t k = 0; k < c[C_NWR]; ++k) {
    const int64_t* r = &h->wr_host[WRF * k];
    const int64_t K = r[5], rows = r[6], nkt = (K + kpt - 1) / kpt;
    wr_map.add(r[7], {wr_b, nkt});
    j_wr.insert(j_wr.end(), {r[7], rows, 1, rows, K, wr_b, ntile, nkt, round_up(rows, 16), 0, 1, 0, 0});
    wr_b += b_bytes(rows, nkt, bplanes);
  }
  // theta block (s1, a) x (s2, b) of every middle sector: B panel of its transpose, rows d_b, K d_a
  const std::vector<int64_t>& mid = h->mid_host;
  for (int64_t m = 0; m < c[C_NMID]; ++m) {
    const int64_t* r = &mid[MIDF * m];
    for (int s1 = 0; s1 < 2; ++s1) {
      if (r[5 + s1] < 0) continue;
      const int64_t K = h->left[3 * r[5 + s1] + 2], nkt = (K + kpt - 1) / kpt;
      for (int s2 = 0; s2 < 2; ++s2) {
        if (r[8 + s2] < 0) continue;
        const int64_t rows = h->right[3 * r[8 + s2] + 2];
        const int64_t src = r[4] + (s1 ? r[7] : 0) * r[3] + (s2 ? r[10] : 0);
        th_map.add(src, {th_b, nkt});
        j_th.insert(j_th.end(), {src, r[3], 1, rows, K, th_b, ntile, nkt, round_up(rows, 16), 0, 1, 0, 0});
        th_b += b_bytes(rows, nkt, bplanes);
      }
    }
  }
  // Z(w', m_in) rows (s1') x columns (s2): A panels keyed by their FP64 element offset
  const std::vector<int64_t>& z = h->z_host;   // downloaded with the other tables at creation
  if ((int64_t)z.size() < ZF * c[C_NZ]) return fail("tc: Z table missing");
  const int64_t nmid = c[C_NMID];
  for (int64_t k = 0; k < c[C_NZ]; ++k) {
    const int64_t* zr = &z[ZF * k];
    const int64_t wp = zr[0], mi = zr[1], mo = zr[2];
    const int64_t* rin = &mid[MIDF * mi];
    const int64_t* rout = &mid[MIDF * mo];
    for (int s1p = 0; s1p < 2; ++s1p) {
      const int64_t ti = (wp * nmid + mi) * 2 + s1p;
      if (h->t1_host[TF * ti + 5] == 0) continue;   // no rows of this part written
      const int64_t rows = h->left[3 * rout[5 + s1p] + 2];
      for (int s2 = 0; s2 < 2; ++s2) {
        if (rin[8 + s2] < 0) continue;
        const int64_t K = h->right[3 * rin[8 + s2] + 2], nkt = (K + kpt - 1) / kpt;
        const int64_t key = zr[5] + (s1p ? rout[7] : 0) * rin[3] + (s2 ? rin[10] : 0);
        z_map.add(key, {z_b, nkt});
        z_b += a_bytes(rows, nkt, aplanes);
      }
    }
  }
  wr_map.finish();
  th_map.finish();
  z_map.finish();
  std::vector<int64_t>&t1 = o.t1, &s1 = o.s1, &p1 = o.p1, &t2 = o.t2, &s2 = o.s2, &p2 = o.p2;
  p1.assign(1, 0);
  p2.assign(1, 0);
  // step-2 tasks (theta' = sum Z WR), built on a second host thread while this one builds the
  // step-1 tasks: the two loops share only the finished (read-only) panel indexes
  bool step2_ok = true;
  auto build_step2 = [&] {
    for (int64_t i = 0; i < c[C_NT2]; ++i) {
      const int64_t* t = &h->t2_host[TF * i];
      if (t[5] == 0 || t[0] == 0 || t[1] == 0) continue;
      const int64_t seg0 = (int64_t)s2.size() / TCS;
      for (int64_t k = 0; k < t[5]; ++k) {
        const int64_t* sg = &h->s2_host[SF * (t[4] + k)];
        const Panel* a = z_map.find(sg[0]);
        const Panel* b = wr_map.find(sg[2]);
        if (!a || !b || a->nkt != b->nkt) {
          step2_ok = false;
          return;
        }
        s2.insert(s2.end(), {a->off, b->off, a->nkt, 0});
      }
      t2.insert(t2.end(), {t[0], t[1], t[2], t[3], 0, seg0, t[5], 1, 0, 0});
      p2.push_back(p2.back() + ((t[0] + 127) / 128) * ((t[1] + ntile - 1) / ntile));
    }
  };
  std::thread step2;
  try {
    step2 = std::thread([&] {
      try {
        build_step2();
      } catch (...) {   // out of host memory
        step2_ok = false;
      }
    });
  } catch (...) {   // no thread to be had: build it here, before step 1
    build_step2();
  }
  struct Join {
    std::thread& t;
    ~Join() { if (t.joinable()) t.join(); }
  } join_step2{step2};
  // step-1 tasks (Z = LW theta), stacked: for every input middle sector m_in, the output rows
  // (w', s1', a') of all its Z blocks are stacked along M into one GEMM per column part s2, so
  // that small blocks share 128-row tiles instead of each filling one. Rows are grouped in
  // three classes by the LW blocks that feed them (s1 = 0 only, s1 = 1 only, both), each
  // class a task of its own with the K segments it needs, so no zero block is multiplied.
  // The stacked LW of a class and K segment s1 is one A panel; each output row is scattered to
  // its Z panel through a row map (mode 2).
  std::vector<int64_t>& rowmap = o.rowmap;
  {
    std::vector<int64_t> zrow_of((size_t)c[C_NMID] > 0 ? (size_t)h->d.d_m * nmid : 0, -1);
    for (int64_t k = 0; k < c[C_NZ]; ++k) zrow_of[(size_t)(z[ZF * k] * nmid + z[ZF * k + 1])] = k;
    struct Member { int64_t wp, s1p, rows, row0, lw[2]; };
    for (int64_t mi = 0; mi < nmid; ++mi) {
      const int64_t* rin = &mid[MIDF * mi];
      std::vector<Member> cls[3];
      for (int64_t wp = 0; wp < h->d.d_m; ++wp)
        for (int s1p = 0; s1p < 2; ++s1p) {
          const int64_t ti = (wp * nmid + mi) * 2 + s1p;
          const int64_t* t = &h->t1_host[TF * ti];
          if (t[5] == 0 || t[0] == 0 || t[1] == 0) continue;
          Member mb{wp, s1p, t[0], 0, {-1, -1}};
          for (int64_t k = 0; k < t[5]; ++k) {
            const int64_t* sg = &h->s1_host[SF * (t[4] + k)];
            int q1 = sg[2] == rin[4] + rin[7] * rin[3] ? 1 : 0;   // theta rows of the s1 = 1 part
            if (rin[5] < 0) q1 = 1;
            if (rin[6] < 0) q1 = 0;
            mb.lw[q1] = sg[0];
          }
          const int k = mb.lw[0] >= 0 && mb.lw[1] >= 0 ? 2 : (mb.lw[0] >= 0 ? 0 : 1);
          cls[k].push_back(mb);
        }
      for (int k = 0; k < 3; ++k) {
        if (cls[k].empty()) continue;
        int64_t R = 0;
        for (Member& mb : cls[k]) { mb.row0 = R; R += mb.rows; }
        // the class's stacked A panels, one per K segment s1
        int64_t aoff[2] = {-1, -1}, ank[2] = {0, 0};
        for (int q1 = 0; q1 < 2; ++q1) {
          if (k != 2 && k != q1) continue;
          if (rin[5 + q1] < 0) return fail("tc: LW block without its theta rows");
          const int64_t K = h->left[3 * rin[5 + q1] + 2];
          ank[q1] = (K + kpt - 1) / kpt;
          aoff[q1] = lw_b;
          for (const Member& mb : cls[k])
            j_lw.insert(j_lw.end(), {mb.lw[q1], K, 0, mb.rows, K, lw_b, 128, ank[q1], round_up(R, 128), 0, 0, mb.row0, 0});
          lw_b += a_bytes(R, ank[q1], aplanes);
        }
        for (int s2p = 0; s2p < 2; ++s2p) {
          if (rin[8 + s2p] < 0) continue;
          const int64_t N = h->right[3 * rin[8 + s2p] + 2], coff = s2p ? rin[10] : 0;
          if (N == 0) continue;
          const int64_t seg0 = (int64_t)s1.size() / TCS, map0 = (int64_t)rowmap.size();
          int64_t nseg = 0;
          for (int q1 = 0; q1 < 2; ++q1) {
            if (aoff[q1] < 0) continue;
            const Panel* b = th_map.find(rin[4] + (q1 ? rin[7] : 0) * rin[3] + coff);
            if (!b || b->nkt != ank[q1]) return fail("tc: step-1 operand not packed");
            s1.insert(s1.end(), {aoff[q1], b->off, ank[q1], 0});
            ++nseg;
          }
          const int64_t nkt_z = (N + kpt - 1) / kpt;
          for (const Member& mb : cls[k]) {
            const int64_t zk = zrow_of[(size_t)(mb.wp * nmid + mi)];
            if (zk < 0) return fail("tc: step-1 output block missing");
            const int64_t* zr = &z[ZF * zk];
            const int64_t* rout = &mid[MIDF * zr[2]];
            const Panel* q = z_map.find(zr[5] + (mb.s1p ? rout[7] : 0) * rin[3] + coff);
            if (!q || q->nkt != nkt_z) return fail("tc: step-1 output panel missing");
            for (int64_t r = 0; r < mb.rows; ++r) rowmap.push_back(q->off << 16 | r);
          }
          t1.insert(t1.end(), {R, N, map0, 0, 0, seg0, nseg, 2, nkt_z, 0});
          p1.push_back(p1.back() + ((R + 127) / 128) * ((N + ntile - 1) / ntile));
        }
      }
    }
  }
  if (step2.joinable()) step2.join();
  if (!step2_ok) return fail("tc: step-2 operand not packed");
  // block schedule: tiles are dealt to the persistent CTAs in task order; order 1 puts the
  // tasks with the most work (tiles x K tiles) first so that the long ones start early
  if (cfg.order == 1) {
    auto reorder = [&](std::vector<int64_t>& tk, const std::vector<int64_t>& sg, std::vector<int64_t>& pf) {
      const size_t nt = tk.size() / TCT;
      std::vector<int64_t> work(nt), idx(nt);
      for (size_t i = 0; i < nt; ++i) {
        int64_t kt = 0;
        for (int64_t k = 0; k < tk[TCT * i + 6]; ++k) kt += sg[TCS * (tk[TCT * i + 5] + k) + 2];
        work[i] = (pf[i + 1] - pf[i]) * kt;
        idx[i] = (int64_t)i;
      }
      std::stable_sort(idx.begin(), idx.end(), [&](int64_t a, int64_t b) { return work[a] > work[b]; });
      std::vector<int64_t> t2v(tk.size()), p2v(nt + 1, 0);
      for (size_t i = 0; i < nt; ++i) {
        std::copy(tk.begin() + TCT * idx[i], tk.begin() + TCT * (idx[i] + 1), t2v.begin() + TCT * i);
        p2v[i + 1] = p2v[i] + (pf[idx[i] + 1] - pf[idx[i]]);
      }
      tk.swap(t2v);
      pf.swap(p2v);
    };
    reorder(t1, s1, p1);
    reorder(t2, s2, p2);
  }
  // every tile the kernel reads or writes must lie inside its buffer
  {
    auto chk = [&](const std::vector<int64_t>& tk, const std::vector<int64_t>& sg, int64_t alen, int64_t blen,
                   bool zout) {
      for (size_t i = 0; i < tk.size(); i += TCT) {
        const int64_t M = tk[i], N = tk[i + 1];
        for (int64_t k = 0; k < tk[i + 6]; ++k) {
          const int64_t* q = &sg[TCS * (tk[i + 5] + k)];
          if (q[0] < 0 || q[0] + a_bytes(M, q[2], aplanes) > alen) return false;
          if (q[1] < 0 || q[1] + b_bytes(N, q[2], bplanes) > blen) return false;
        }
        if (zout) {   // every mapped row lies in a Z panel of this task's K-tile count
          if (tk[i + 2] < 0 || tk[i + 2] + M > (int64_t)rowmap.size() || tk[i + 8] * kpt < N) return false;
          for (int64_t r = 0; r < M; ++r) {
            const int64_t off = rowmap[tk[i + 2] + r] >> 16, zr = rowmap[tk[i + 2] + r] & 0xffff;
            if (off < 0 || off + (zr / 128 + 1) * tk[i + 8] * aplanes * 128 * 128 > z_b) return false;
          }
        }
      }
      return true;
    };
    if (!chk(t1, s1, lw_b, th_b, true) || !chk(t2, s2, z_b, wr_b, false))
      return fail("tc: internal panel table check failed");
    if (!tc_cfg_ok(prec, cfg)) return fail("tc: tile configuration does not fit");
  }
  std::vector<int64_t>&q1 = o.q1, &q2 = o.q2;
  q1.assign(2 * std::max<size_t>(p1.size() - 1, 1), 0);
  q2.assign(2 * std::max<size_t>(p2.size() - 1, 1), 0);
  for (size_t t = 0; t + 1 < p1.size(); ++t) q1[2 * t + 1] = p1[t + 1] - p1[t];
  for (size_t t = 0; t + 1 < p2.size(); ++t) q2[2 * t + 1] = p2[t + 1] - p2[t];
  // Item tables: (task, tile within task) of every tile, dealt to the persistent CTAs by
  // longest-processing-time-first: items by decreasing cost (the task's K tiles plus two for the
  // pipeline fill and the epilogue; equal costs in task order), each to the CTA with the least
  // work so far (the lowest-numbered of those). Each CTA's items are stored together,
  // co[c] .. co[c + 1]. A static deal in item order left step 2's SMs between 25% and 91% busy
  // (ncu) because the tiles' K lengths differ by orders of magnitude.
  // Tasks are ordered by a counting sort of their costs, and the least-loaded CTA is found in a
  // bucket queue: bit sets of the CTAs per amount of work, in a ring of cmax + 1 buckets (every
  // CTA's work lies within cmax of the least), so tens of thousands of items cost no sort and
  // no heap operations.
  const int grid_sm = std::max(h->n_sm, 1);
  auto deal = [&](const std::vector<int64_t>& tk, const std::vector<int64_t>& sg, const std::vector<int64_t>& pf,
                  std::vector<int2>& items, std::vector<int32_t>& co) {
    const size_t nt = tk.size() / TCT;
    const int64_t total = pf.back();
    const int G = (int)std::min<int64_t>(total, grid_sm);
    co.assign((size_t)G + 1, 0);
    if (total <= 0) return;
    std::vector<int64_t> cost(nt, 0);
    int64_t cmax = 0;
    for (size_t t = 0; t < nt; ++t) {
      if (pf[t + 1] == pf[t]) continue;   // no tiles
      int64_t kt = 0;
      for (int64_t k = 0; k < tk[TCT * t + 6]; ++k) kt += sg[TCS * (tk[TCT * t + 5] + k) + 2];
      cost[t] = kt + 2;
      cmax = std::max(cmax, cost[t]);
    }
    std::vector<int64_t> first((size_t)cmax + 1, 0);   // first slot of each cost, decreasing costs
    for (size_t t = 0; t < nt; ++t)
      if (pf[t + 1] > pf[t]) ++first[(size_t)cost[t]];
    for (int64_t c = cmax, acc = 0; c >= 0; --c) {
      const int64_t n = first[(size_t)c];
      first[(size_t)c] = acc;
      acc += n;
    }
    size_t n_ord = 0;   // tasks with tiles
    for (size_t t = 0; t < nt; ++t)
      if (pf[t + 1] > pf[t]) ++n_ord;
    std::vector<int32_t> ord(n_ord);
    for (size_t t = 0; t < nt; ++t)
      if (pf[t + 1] > pf[t]) ord[(size_t)first[(size_t)cost[t]]++] = (int32_t)t;
    const int W = (G + 63) / 64;
    const int64_t R = cmax + 1;
    std::vector<uint64_t> bits((size_t)(R * W), 0);   // bucket (work mod R): the CTAs with that work
    for (int c = 0; c < G; ++c) bits[(size_t)(c >> 6)] |= 1ull << (c & 63);
    int64_t lo = 0;   // least work of any CTA
    std::vector<int32_t> owner((size_t)total), count((size_t)G, 0);
    size_t i = 0;
    for (const int32_t t : ord) {
      const int64_t add = cost[(size_t)t];
      for (int64_t l = pf[(size_t)t]; l < pf[(size_t)t + 1]; ++l, ++i) {
        int c = -1;
        for (;; ++lo) {
          const uint64_t* bk = &bits[(size_t)((lo % R) * W)];
          for (int w = 0; w < W && c < 0; ++w)
            if (bk[w]) c = w * 64 + __builtin_ctzll(bk[w]);
          if (c >= 0) break;
        }
        bits[(size_t)((lo % R) * W + (c >> 6))] &= ~(1ull << (c & 63));
        bits[(size_t)(((lo + add) % R) * W + (c >> 6))] |= 1ull << (c & 63);
        owner[i] = c;
        ++count[(size_t)c];
      }
    }
    for (int c = 0; c < G; ++c) co[(size_t)c + 1] = co[(size_t)c] + count[(size_t)c];
    items.assign((size_t)total, make_int2(0, 0));
    std::vector<int32_t> fill(co.begin(), co.end() - 1);
    i = 0;
    for (const int32_t t : ord)
      for (int64_t l = 0; l < pf[(size_t)t + 1] - pf[(size_t)t]; ++l, ++i)
        items[(size_t)fill[(size_t)owner[i]]++] = make_int2(t, (int)l);
  };
  deal(t1, s1, p1, o.i1, o.co1);
  deal(t2, s2, p2, o.i2, o.co2);
  // first piece of every pack job (field 9) and the pieces of each list
  const int kc = tc_is_tf32(prec) ? 4 : 8;
  auto pieces = [&](std::vector<int64_t>& j) {
    int64_t n = 0;
    for (size_t k = 0; k < j.size(); k += TCJ) {
      j[k + 9] = n;
      n += (j[k + 3] * ((j[k + 4] + kc - 1) / kc) + kPackPiece - 1) / kPackPiece;
    }
    return n;
  };
  o.pc_lw = pieces(j_lw);
  o.pc_wr = pieces(j_wr);
  o.pc_th = pieces(j_th);
  return true;
}

// Device buffers of the tables in `o` (which must have been built for this H_eff): allocation,
// upload and zeroed panels; replaces the H_eff's tensor-core state. Synchronises the stream.
int upload(mrd_heff* h, const TcTables& o) {
  mrd_ctx* ctx = h->ctx;
  delete h->tc;
  Tc* T = h->tc = new Tc();
  T->prec = o.prec;
  T->cfg = o.cfg;
  Arena& A = T->mem;
  A.stream = ctx->stream;
  cudaError_t e = cudaSuccess;
#define TALLOC(ptr, n) if (e == cudaSuccess) e = A.alloc(&(ptr), (size_t)std::max<int64_t>((n), 1))
  TALLOC(T->lw, o.lw_b); TALLOC(T->wr, o.wr_b); TALLOC(T->th, o.th_b); TALLOC(T->z, o.z_b);
  TALLOC(T->t1, o.t1.size()); TALLOC(T->s1, o.s1.size()); TALLOC(T->p1, o.p1.size());
  TALLOC(T->t2, o.t2.size()); TALLOC(T->s2, o.s2.size()); TALLOC(T->p2, o.p2.size());
  TALLOC(T->j_lw, o.j_lw.size()); TALLOC(T->j_wr, o.j_wr.size()); TALLOC(T->j_th, o.j_th.size());
  TALLOC(T->err, 1);
  TALLOC(T->pt1, o.q1.size()); TALLOC(T->pt2, o.q2.size());
  TALLOC(T->it1, o.i1.size()); TALLOC(T->it2, o.i2.size());
  TALLOC(T->co1, o.co1.size()); TALLOC(T->co2, o.co2.size());
  TALLOC(T->rmap1, o.rowmap.size());
#undef TALLOC
  if (e != cudaSuccess) return mrd_cuda_fail(ctx, e, "tc: device buffers");
  T->lw_bytes = o.lw_b; T->wr_bytes = o.wr_b; T->th_bytes = o.th_b; T->z_bytes = o.z_b;
  T->n1 = (int64_t)o.t1.size() / TCT; T->ntiles1 = o.p1.back();
  T->n2 = (int64_t)o.t2.size() / TCT; T->ntiles2 = o.p2.back();
  T->n_lw = (int)(o.j_lw.size() / TCJ); T->n_wr = (int)(o.j_wr.size() / TCJ); T->n_th = (int)(o.j_th.size() / TCJ);
  T->pc_lw = o.pc_lw; T->pc_wr = o.pc_wr; T->pc_th = o.pc_th;
  cudaStream_t s = ctx->stream;
  auto up = [&](void* d, const void* v, size_t bytes) {
    if (e == cudaSuccess && bytes) e = cudaMemcpyAsync(d, v, bytes, cudaMemcpyHostToDevice, s);
  };
  for (auto pr : {std::make_pair(T->t1, &o.t1), std::make_pair(T->s1, &o.s1), std::make_pair(T->p1, &o.p1),
                  std::make_pair(T->t2, &o.t2), std::make_pair(T->s2, &o.s2), std::make_pair(T->p2, &o.p2),
                  std::make_pair(T->j_lw, &o.j_lw), std::make_pair(T->j_wr, &o.j_wr), std::make_pair(T->j_th, &o.j_th),
                  std::make_pair(T->pt1, &o.q1), std::make_pair(T->pt2, &o.q2), std::make_pair(T->rmap1, &o.rowmap)})
    up(pr.first, pr.second->data(), pr.second->size() * 8);
  up(T->it1, o.i1.data(), o.i1.size() * 8);
  up(T->it2, o.i2.data(), o.i2.size() * 8);
  up(T->co1, o.co1.data(), o.co1.size() * 4);
  up(T->co2, o.co2.data(), o.co2.size() * 4);
  T->tiles1.resize(o.p1.size() - 1);
  T->tiles2.resize(o.p2.size() - 1);
  for (size_t t = 0; t < T->tiles1.size(); ++t) T->tiles1[t] = o.q1[2 * t + 1];
  for (size_t t = 0; t < T->tiles2.size(); ++t) T->tiles2[t] = o.q2[2 * t + 1];
  // zero padding everywhere (packing and the Z epilogue only write valid elements)
  for (auto pr : {std::make_pair(T->lw, o.lw_b), std::make_pair(T->wr, o.wr_b), std::make_pair(T->th, o.th_b),
                  std::make_pair(T->z, o.z_b)})
    if (e == cudaSuccess && pr.second) e = cudaMemsetAsync(pr.first, 0, (size_t)pr.second, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(T->err, 0, 4, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);   // the host tables may be released after this
  if (e != cudaSuccess) return mrd_cuda_fail(ctx, e, "tc: upload");
  return MRD_OK;
}

int build(mrd_heff* h, int prec, TcCfg cfg) {
  TcTables o;
  if (!tables(h, prec, cfg, o)) return mrd_fail(h->ctx, MRD_E_STATE, o.err);
  return upload(h, o);
}

}  // namespace

namespace {

// Candidate tile configurations per precision (all fit the 227 KB of shared memory).
std::vector<TcCfg> candidates(int prec) {
  if (prec == TC_TF32) return {{128, 2, 0}, {64, 4, 0}, {128, 2, 1}, {64, 4, 1}};
  if (prec == TC_BF16X3) return {{64, 2, 0}, {48, 2, 0}, {64, 2, 1}, {48, 2, 1}};
  return {{128, 3, 0}, {64, 4, 0}, {128, 3, 1}, {64, 4, 1}};   // real operands: 1 or 2 planes
}

// Problem class of an H_eff for the tuning cache: precision, size of theta (powers of two)
// and number of tensor-core step-2 tasks (powers of two).
uint64_t tune_key(const mrd_heff* h, int prec) {
  auto lg = [](int64_t v) { uint64_t b = 0; while (v > 1) { v >>= 1; ++b; } return b; };
  return (uint64_t)prec << 56 | lg(h->counts[C_THETA]) << 40 | lg(h->counts[C_NT2]) << 24 | (uint64_t)h->n_sm;
}

// Kernel time (ms) of steps 1 and 2 with the built configuration, on the packed operands
// (values do not change the time): 1 warm-up, 3 timed applications.
int time_cfg(mrd_heff* h, double* ms) {
  mrd_ctx* ctx = h->ctx;
  Tc* T = h->tc;
  cudaStream_t s = ctx->stream;
  cudaEvent_t a = nullptr, b = nullptr;
  MRD_CUDA(ctx, cudaEventCreate(&a));
  cudaError_t e = cudaEventCreate(&b);
  if (e != cudaSuccess) { cudaEventDestroy(a); return mrd_cuda_fail(ctx, e, "autotune: event"); }
  double2* out = nullptr;   // scratch output of the timing runs
  e = cache_alloc((void**)&out, (size_t)std::max<int64_t>(h->counts[C_THETA], 1) * 16, s);
  for (int r = 0; r < 4 && e == cudaSuccess; ++r) {
    if (r == 1) e = cudaEventRecord(a, s);
    if (e == cudaSuccess)
      e = tc_gemm(T->lw, T->th, T->t1, T->s1, T->p1, T->it1, T->co1, T->rmap1, T->n1, T->ntiles1, T->z, nullptr, T->prec, T->cfg, T->err,
                  h->n_sm, h->wait_ns, s);
    if (e == cudaSuccess)
      e = tc_gemm(T->z, T->wr, T->t2, T->s2, T->p2, T->it2, T->co2, nullptr, T->n2, T->ntiles2, nullptr, out, T->prec, T->cfg, T->err, h->n_sm,
                  h->wait_ns, s);
  }
  float f = 0.f;
  if (e == cudaSuccess) e = cudaEventRecord(b, s);
  if (e == cudaSuccess) e = cudaEventSynchronize(b);
  if (e == cudaSuccess) e = cudaEventElapsedTime(&f, a, b);
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  cache_free(out, s);
  if (e != cudaSuccess) return mrd_cuda_fail(ctx, e, "autotune: timing");
  *ms = f / 3.0;
  return tc_status(h);
}

}  // namespace

// Tables being built on a host thread for a known configuration (tc_prebuild).
struct TcPre {
  std::thread th;
  TcTables tab;
  bool ok = false;
  ~TcPre() {
    if (th.joinable()) th.join();
  }
};

void tc_pre_free(TcPre* t) { delete t; }

namespace {

// The configuration a build of `prec` would use without timing anything: the default when
// tuning is off, the tuned one when this problem class is in the context's cache; false when
// it would have to be tuned.
bool known_cfg(const mrd_heff* h, int prec, TcCfg* cfg) {
  if (!h->autotune) {
    *cfg = tc_default_cfg(prec);
    return true;
  }
  auto it = h->ctx->tc_tuned.find(tune_key(h, prec));
  if (it == h->ctx->tc_tuned.end()) return false;
  *cfg = TcCfg{it->second[0], it->second[1], it->second[2]};
  return true;
}

// Build for (prec, cfg), from the host thread's tables when it built exactly these (its thread
// is joined and its tables released either way).
int build_known(mrd_heff* h, int prec, TcCfg cfg) {
  if (TcPre* pre = h->tc_pre) {
    h->tc_pre = nullptr;
    if (pre->th.joinable()) pre->th.join();
    const TcTables& o = pre->tab;
    const bool same = pre->ok && o.prec == prec && o.n_sm == h->n_sm && o.cfg.ntile == cfg.ntile &&
                      o.cfg.stages == cfg.stages && o.cfg.order == cfg.order;
    int rc = same ? upload(h, o) : MRD_OK;
    delete pre;
    if (same) return rc;
  }
  return build(h, prec, cfg);
}

}  // namespace

// Starts building the tensor-core tables of `prec` on a host thread when their configuration
// is known without timing (tuning off, or this problem class tuned earlier on the context),
// so that the host work (milliseconds at large bond dimension) overlaps device work queued
// meanwhile; the next tc_prepare joins it. Does nothing otherwise, or when the thread cannot be
// started (tc_prepare then builds the tables itself). The host tables of h must not change
// until the thread is joined (tc_prepare, or freeing h).
void tc_prebuild(mrd_heff* h, int32_t prec) {
  const int tp = tc_prec_of(h, prec);
  TcCfg cfg{0, 0, 0};
  if ((h->tc && h->tc->prec == tp) || h->tc_pre || !known_cfg(h, tp, &cfg)) return;
  TcPre* pre = new (std::nothrow) TcPre();
  if (!pre) return;
  try {
    pre->th = std::thread([h, pre, tp, cfg] {
      try {
        pre->ok = tables(h, tp, cfg, pre->tab);
      } catch (...) {   // out of host memory: tc_prepare builds the tables itself
        pre->ok = false;
      }
    });
  } catch (...) {
    delete pre;
    return;
  }
  h->tc_pre = pre;
}

// Pick the tile configuration: from the context's tuning cache for this problem class, else
// by timing every candidate on this H_eff (MRD_OPT_AUTOTUNE, default on), else the default.
int autotune(mrd_heff* h, int prec) {
  mrd_ctx* ctx = h->ctx;
  const uint64_t key = tune_key(h, prec);
  TcCfg known{0, 0, 0};
  if (known_cfg(h, prec, &known)) {
    int rc = build_known(h, prec, known);
    if (rc == MRD_OK) h->tc->cfg_source = h->autotune ? 2 : 0;
    return rc;
  }
  if (h->tc_pre) {   // tables of another precision
    tc_pre_free(h->tc_pre);
    h->tc_pre = nullptr;
  }
  TcCfg best{0, 0, 0};
  double best_ms = 1e300;
  for (const TcCfg& c : candidates(prec)) {
    int rc = build(h, prec, c);
    if (rc != MRD_OK) return rc;
    Tc* T = h->tc;
    MRD_CUDA(ctx, tc_pack(h->lw, T->lw, T->j_lw, T->n_lw, T->pc_lw, prec, ctx->stream));
    MRD_CUDA(ctx, tc_pack(h->wr, T->wr, T->j_wr, T->n_wr, T->pc_wr, prec, ctx->stream));
    double ms = 0.0;
    if ((rc = time_cfg(h, &ms)) != MRD_OK) return rc;
    if (ms < best_ms) { best_ms = ms; best = c; }
  }
  ctx->tc_tuned[key] = {best.ntile, best.stages, best.order};
  const TcCfg last = candidates(prec).back();
  if (best.ntile != last.ntile || best.stages != last.stages || best.order != last.order) {
    int rc = build(h, prec, best);
    if (rc != MRD_OK) return rc;
  }
  h->tc->cfg_source = 1;
  h->tc->env_dirty = true;
  return MRD_OK;
}

void tc_env_changed(mrd_heff* h) {
  if (h->tc) h->tc->env_dirty = true;
}

int tc_status(mrd_heff* h) {
  if (!h->tc) return MRD_OK;
  int herr = 0;
  MRD_CUDA(h->ctx, cudaMemcpyAsync(&herr, h->tc->err, 4, cudaMemcpyDeviceToHost, h->ctx->stream));
  MRD_CUDA(h->ctx, cudaStreamSynchronize(h->ctx->stream));
  if (herr) {   // reported once: the flag is cleared for the next launches
    MRD_CUDA(h->ctx, cudaMemsetAsync(h->tc->err, 0, 4, h->ctx->stream));
    MRD_CUDA(h->ctx, cudaStreamSynchronize(h->ctx->stream));
    return mrd_fail(h->ctx, MRD_E_TIMEOUT, "tensor-core GEMM: a bounded wait gave up (code " + std::to_string(herr) + ")");
  }
  return MRD_OK;
}

// Panel tables and buffers for `prec` (host work, allocation, synchronisation) and the packed
// environments; a no-op when both are current.
int tc_prepare(mrd_heff* h, int32_t prec) {
  mrd_ctx* ctx = h->ctx;
  const int tp = tc_prec_of(h, prec);
  int rc;
  MRD_CUDA(ctx, tc_gemm_init());
  if (!h->tc || h->tc->prec != tp) {
    if (!h->tc) h->tc = new Tc();
    if ((rc = autotune(h, tp)) != MRD_OK) return rc;
    ++h->gen;
  }
  Tc* T = h->tc;
  cudaStream_t s = ctx->stream;
  if (T->env_dirty) {
    MRD_CUDA(ctx, tc_pack(h->lw, T->lw, T->j_lw, T->n_lw, T->pc_lw, tp, s));
    MRD_CUDA(ctx, tc_pack(h->wr, T->wr, T->j_wr, T->n_wr, T->pc_wr, tp, s));
    T->env_dirty = false;
  }
  return MRD_OK;
}

int tc_config(const mrd_heff* h, int32_t* cfg4) {
  if (!h->tc) {
    cfg4[0] = cfg4[1] = cfg4[2] = cfg4[3] = -1;
    return MRD_OK;
  }
  cfg4[0] = h->tc->cfg.ntile;
  cfg4[1] = h->tc->cfg.stages;
  cfg4[2] = h->tc->cfg.order;
  cfg4[3] = h->tc->cfg_source;
  return MRD_OK;
}

int tc_apply(mrd_heff* h, const double* in, double* out, int32_t prec) {
  mrd_ctx* ctx = h->ctx;
  const int tp = tc_prec_of(h, prec);
  int rc = tc_prepare(h, prec);
  if (rc != MRD_OK) return rc;
  Tc* T = h->tc;
  cudaStream_t s = ctx->stream;
  cudaEvent_t ev[3] = {nullptr, nullptr, nullptr};
  bool cap = false;
  if (h->timing && !apply_events(h, s, ev, &cap)) return mrd_fail(ctx, MRD_E_CUDA, "mrd_heff_apply: cudaEventCreate");
  const cudaEvent_t e0 = ev[0], e1 = ev[1], e2 = ev[2];
  MRD_CUDA(ctx, cudaMemsetAsync(out, 0, (size_t)h->counts[C_THETA] * 16, s));
  MRD_CUDA(ctx, tc_pack((const double2*)in, T->th, T->j_th, T->n_th, T->pc_th, tp, s));
  MRD_CUDA(ctx, record_event(e0, s, cap));
  if (!h->per_task) {
    MRD_CUDA(ctx, tc_gemm(T->lw, T->th, T->t1, T->s1, T->p1, T->it1, T->co1, T->rmap1, T->n1, T->ntiles1, T->z, nullptr, tp, T->cfg, T->err,
                          h->n_sm, h->wait_ns, s));
    MRD_CUDA(ctx, record_event(e1, s, cap));
    MRD_CUDA(ctx, tc_gemm(T->z, T->wr, T->t2, T->s2, T->p2, T->it2, T->co2, nullptr, T->n2, T->ntiles2, nullptr, (double2*)out, tp, T->cfg,
                          T->err, h->n_sm, h->wait_ns, s));
  } else {   // one launch per task: the per-block baseline of the grouped persistent launch
    for (int64_t t = 0; t < T->n1; ++t)
      MRD_CUDA(ctx, tc_gemm(T->lw, T->th, T->t1 + TCT * t, T->s1, T->pt1 + 2 * t, nullptr, nullptr, T->rmap1, 1, T->tiles1[t], T->z, nullptr, tp,
                            T->cfg, T->err, h->n_sm, h->wait_ns, s));
    MRD_CUDA(ctx, record_event(e1, s, cap));
    for (int64_t t = 0; t < T->n2; ++t)
      MRD_CUDA(ctx, tc_gemm(T->z, T->wr, T->t2 + TCT * t, T->s2, T->pt2 + 2 * t, nullptr, nullptr, nullptr, 1, T->tiles2[t], nullptr,
                            (double2*)out, tp, T->cfg, T->err, h->n_sm, h->wait_ns, s));
  }
  MRD_CUDA(ctx, record_event(e2, s, cap));
  return MRD_OK;
}
