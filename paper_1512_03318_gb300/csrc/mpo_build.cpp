// Finite-state-machine construction of the cylinder Hamiltonian MPO (Sec. IV).
//
// Every Hamiltonian term family is a product of fermionic "roles" f_1 ... f_n (c+, c or a
// number operator), each tied to a ring relative to the family's base ring, with a
// coefficient that factorises into one phase per role (e^{i p 2 pi m / Ly} for a role placed
// at momentum m). An FSM node is (family, base ring, set of placed roles, cumulative label
// mod Ly); in the mixed basis the label is the momentum placed so far, i.e. the
// momentum-labelled nodes A_mu(k), C_mu(k) of Sec. IV.D (Figs. 9 and 10a), and a path may
// enter the final node F only with total momentum 0. In real space the label is the
// position y and pins the partner site of a hop.
//
// Jordan-Wigner (Sec. IV.C, Eq. JW): the operator a path places on site j is the ordered
// product over roles of I (placed earlier), the role's operator (placed here) or Z (a
// pending fermionic role).
//
// After generation the machine is trimmed (nodes off every R -> F path are removed, Sec. IV.D)
// and nodes with proportional incoming columns (identical pasts) or proportional outgoing
// rows (identical futures) are fused, which is exact. The real-space machine then has
// D = 3 Ly + 2 in the bulk (Sec. IV.C).
#include <algorithm>
#include <cmath>
#include <complex>
#include <map>
#include <set>
#include <string>
#include <tuple>
#include <vector>

#include "mrd_internal.h"

namespace mrd {

using cd = std::complex<double>;

namespace {

enum Op { OP_CD = 0, OP_C = 1, OP_N = 2 };

struct Mat2 {
  cd a[2][2];  // [s'][s]
  Mat2() { a[0][0] = a[0][1] = a[1][0] = a[1][1] = 0.0; }
  bool nonzero(double tol = 0.0) const {
    for (int i = 0; i < 2; ++i)
      for (int j = 0; j < 2; ++j)
        if (std::abs(a[i][j]) > tol) return true;
    return false;
  }
};

Mat2 mat_of(int which) {  // 0 I, 1 Cd, 2 C, 3 N, 4 Z
  Mat2 m;
  switch (which) {
    case 0: m.a[0][0] = 1; m.a[1][1] = 1; break;
    case 1: m.a[1][0] = 1; break;
    case 2: m.a[0][1] = 1; break;
    case 3: m.a[1][1] = 1; break;
    case 4: m.a[0][0] = 1; m.a[1][1] = -1; break;
  }
  return m;
}

Mat2 mul(const Mat2& x, const Mat2& y) {
  Mat2 r;
  for (int i = 0; i < 2; ++i)
    for (int j = 0; j < 2; ++j) r.a[i][j] = x.a[i][0] * y.a[0][j] + x.a[i][1] * y.a[1][j];
  return r;
}

struct Role {
  int op;        // Op
  int ring;      // offset from the base ring; kAnyRing for any
  int phase;     // phase sign
  int label;     // label sign
  int trig = 0;  // 1: factor cos(2 pi m / Ly), 2: sin(2 pi m / Ly) instead of a phase
};

// cos / sin of 2 pi m / ly, exactly zero where the angle is an odd multiple of pi/2 (cos) or a
// multiple of pi (sin): rounded library values there would add spurious transitions
double trig_of(int kind, int m, int ly) {
  const double pi = 3.14159265358979323846;
  if (kind == 2) return (2 * m) % ly == 0 ? 0.0 : std::sin(2.0 * pi * m / ly);
  return (4 * m) % (2 * ly) == ly ? 0.0 : std::cos(2.0 * pi * m / ly);
}
constexpr int kAnyRing = 1 << 20;

struct Family {
  std::string name;
  std::vector<Role> roles;
  int target;
  std::vector<int> bases;
  std::vector<cd> coeff;  // indexed by base ring
};

// Node key; kind 0 = R, 1 = intermediate, 2 = F. Ordered like the tuple
// (kind, family name, base ring, placed bits, label, dN, dK).
struct Key {
  int kind = 0;
  int fam = 0;  // rank of the family name in lexicographic order
  int xb = 0, placed = 0, lab = 0, dn = 0, dk = 0;
  bool operator<(const Key& o) const {
    return std::tie(kind, fam, xb, placed, lab, dn, dk) <
           std::tie(o.kind, o.fam, o.xb, o.placed, o.lab, o.dn, o.dk);
  }
  bool operator==(const Key& o) const {
    return !(*this < o) && !(o < *this);
  }
};

Key key_R() { Key k; k.kind = 0; return k; }
Key key_F() { Key k; k.kind = 2; return k; }

using Trans = std::map<std::pair<Key, Key>, Mat2>;

void add_trans(Trans& t, std::map<Key, int>& out_keys, const Key& src, const Key& dst, const Mat2& m, cd coeff) {
  if (coeff == cd(0.0) || !m.nonzero()) return;
  out_keys.emplace(dst, 0);
  Mat2& acc = t[{src, dst}];
  for (int i = 0; i < 2; ++i)
    for (int j = 0; j < 2; ++j) acc.a[i][j] += coeff * m.a[i][j];
}

Mat2 local_op(const std::vector<Role>& roles, int placed, int here) {
  Mat2 out = mat_of(0);
  for (size_t r = 0; r < roles.size(); ++r) {
    int bit = 1 << r;
    int which;
    if (placed & bit) which = 0;
    else if (here & bit) which = roles[r].op == OP_CD ? 1 : (roles[r].op == OP_C ? 2 : 3);
    else which = (roles[r].op == OP_N) ? 0 : 4;
    out = mul(out, mat_of(which));
  }
  return out;
}

// Sparse vector used by the fusion step: key (other node, s', s) -> value.
using SVec = std::map<std::tuple<Key, int, int>, cd>;

SVec vec_of(const Trans& t, const Key& node, int side) {
  SVec out;
  for (const auto& kv : t) {
    const Key& a = kv.first.first;
    const Key& b = kv.first.second;
    if ((side == 0 ? b : a) == node) {
      const Key& other = side == 0 ? a : b;
      for (int sp = 0; sp < 2; ++sp)
        for (int s = 0; s < 2; ++s)
          if (kv.second.a[sp][s] != cd(0.0)) out[{other, sp, s}] = kv.second.a[sp][s];
    }
  }
  return out;
}

bool proportional(const SVec& u, const SVec& w, cd* f, double tol = 1e-10) {
  if (u.empty() || u.size() != w.size()) return false;
  auto iu = u.begin();
  auto iw = w.begin();
  for (; iu != u.end(); ++iu, ++iw)
    if (!(iu->first == iw->first)) return false;
  cd ratio = u.begin()->second / w.begin()->second;
  for (iu = u.begin(), iw = w.begin(); iu != u.end(); ++iu, ++iw)
    if (std::abs(iu->second - ratio * iw->second) > tol * std::max(1.0, std::abs(iu->second))) return false;
  *f = ratio;
  return true;
}

void fuse(std::vector<std::vector<Key>>& bonds, std::vector<Trans>& trans, int n) {
  bool changed = true;
  while (changed) {
    changed = false;
    for (int j = 1; j < n; ++j) {  // proportional pasts
      std::vector<std::pair<Key, SVec>> reps;
      std::vector<Key> nodes = bonds[j];
      for (const Key& node : nodes) {
        SVec col = vec_of(trans[j - 1], node, 0);
        int hit = -1;
        cd f;
        for (size_t r = 0; r < reps.size(); ++r)
          if (proportional(col, reps[r].second, &f)) { hit = (int)r; break; }
        if (hit < 0) { reps.push_back({node, col}); continue; }
        Key rep = reps[hit].first;
        std::vector<std::pair<Key, Key>> rows;
        for (const auto& kv : trans[j])
          if (kv.first.first == node) rows.push_back(kv.first);
        for (const auto& k : rows) {
          Mat2 m = trans[j][k];
          trans[j].erase(k);
          Mat2& acc = trans[j][{rep, k.second}];
          for (int a = 0; a < 2; ++a)
            for (int b = 0; b < 2; ++b) acc.a[a][b] += f * m.a[a][b];
        }
        std::vector<std::pair<Key, Key>> cols;
        for (const auto& kv : trans[j - 1])
          if (kv.first.second == node) cols.push_back(kv.first);
        for (const auto& k : cols) trans[j - 1].erase(k);
        bonds[j].erase(std::find(bonds[j].begin(), bonds[j].end(), node));
        changed = true;
      }
    }
    for (int j = n - 1; j >= 1; --j) {  // proportional futures
      std::vector<std::pair<Key, SVec>> reps;
      std::vector<Key> nodes = bonds[j];
      for (const Key& node : nodes) {
        SVec row = vec_of(trans[j], node, 1);
        int hit = -1;
        cd f;
        for (size_t r = 0; r < reps.size(); ++r)
          if (proportional(row, reps[r].second, &f)) { hit = (int)r; break; }
        if (hit < 0) { reps.push_back({node, row}); continue; }
        Key rep = reps[hit].first;
        std::vector<std::pair<Key, Key>> cols;
        for (const auto& kv : trans[j - 1])
          if (kv.first.second == node) cols.push_back(kv.first);
        for (const auto& k : cols) {
          Mat2 m = trans[j - 1][k];
          trans[j - 1].erase(k);
          Mat2& acc = trans[j - 1][{k.first, rep}];
          for (int a = 0; a < 2; ++a)
            for (int b = 0; b < 2; ++b) acc.a[a][b] += f * m.a[a][b];
        }
        std::vector<std::pair<Key, Key>> rows;
        for (const auto& kv : trans[j])
          if (kv.first.first == node) rows.push_back(kv.first);
        for (const auto& k : rows) trans[j].erase(k);
        bonds[j].erase(std::find(bonds[j].begin(), bonds[j].end(), node));
        changed = true;
      }
    }
    for (int j = 0; j < n; ++j) {
      std::vector<std::pair<Key, Key>> dead;
      for (const auto& kv : trans[j])
        if (!kv.second.nonzero(1e-14)) dead.push_back(kv.first);
      for (const auto& k : dead) trans[j].erase(k);
    }
  }
}

}  // namespace

int build_mpo_host(const mrd_model& m, HostMPO* out, std::string* err) {
  if (m.ly < 2 || m.lx < 1 || m.flux_q <= 0 ||
      (m.basis != MRD_BASIS_MIXED && m.basis != MRD_BASIS_REAL && m.basis != MRD_BASIS_MIXED_REAL)) {
    *err = "mrd_mpo_build: need ly >= 2, lx >= 1, flux_q > 0 and a known basis";
    return MRD_E_ARG;
  }
  if ((int64_t)m.lx * m.ly > 4096) {
    *err = "mrd_mpo_build: at most 4096 orbitals";
    return MRD_E_ARG;
  }
  const int lx = m.lx, ly = m.ly, n = lx * ly;
  const double pi = 3.14159265358979323846;
  const double phi = 2.0 * pi * (double)m.flux_p / (double)m.flux_q;
  const bool mixed = m.basis == MRD_BASIS_MIXED || m.basis == MRD_BASIS_MIXED_REAL;
  const int modulus = mixed ? ly : 1;
  const double t = m.t, v = m.v;

  std::vector<Family> fams;
  auto bases = [](int lo, int hi) { std::vector<int> b; for (int x = lo; x < hi; ++x) b.push_back(x); return b; };
  auto constant = [&](cd c) { return std::vector<cd>(lx, c); };
  if (mixed) {
    // hops between rings: -t c+_{x,m} c_{x+1,m} and -t c+_{x+1,m} c_{x,m}   (Eq. H_kin)
    fams.push_back({"hopR", {{OP_CD, 0, 0, 1}, {OP_C, 1, 0, -1}}, 0, bases(0, lx - 1), constant(-t)});
    fams.push_back({"hopL", {{OP_CD, 1, 0, 1}, {OP_C, 0, 0, -1}}, 0, bases(0, lx - 1), constant(-t)});
    // intra-ring (V/Ly) sum_q cos q n_q n_{-q} = (V/Ly) sum e^{i(p1-p2)2pi/Ly} c+_p1 c_p2 c+_p3 c_p4
    // (n_q and n_{-q} commute, so cos q may be replaced by e^{iq})           (Eq. H_k_int)
    if (m.basis == MRD_BASIS_MIXED) {
      fams.push_back({"intra", {{OP_CD, 0, 1, 1}, {OP_C, 0, -1, -1}, {OP_CD, 0, 0, 1}, {OP_C, 0, 0, -1}}, 0,
                      bases(0, lx), constant(v / ly)});
    } else {
      // the sine / cosine machine (Sec. IV.D, Eq. rot): the coefficient cos((p1 - p2) alpha) of
      // c+_p1 c_p2 c+_p3 c_p4 is cos(p1 a) cos(p2 a) + sin(p1 a) sin(p2 a), one family per term,
      // every entry real
      fams.push_back({"intrac", {{OP_CD, 0, 0, 1, 1}, {OP_C, 0, 0, -1, 1}, {OP_CD, 0, 0, 1}, {OP_C, 0, 0, -1}}, 0,
                      bases(0, lx), constant(v / ly)});
      fams.push_back({"intras", {{OP_CD, 0, 0, 1, 2}, {OP_C, 0, 0, -1, 2}, {OP_CD, 0, 0, 1}, {OP_C, 0, 0, -1}}, 0,
                      bases(0, lx), constant(v / ly)});
    }
    // inter-ring (V/Ly) sum_q n_{x,-q} n_{x+1,q}                               (Eq. H_k_int)
    fams.push_back({"inter", {{OP_CD, 0, 0, 1}, {OP_C, 0, 0, -1}, {OP_CD, 1, 0, 1}, {OP_C, 1, 0, -1}}, 0,
                    bases(0, lx - 1), constant(v / ly)});
  } else {
    std::vector<cd> e(lx), ec(lx);
    for (int x = 0; x < lx; ++x) {
      e[x] = -t * cd(std::cos(x * phi), std::sin(x * phi));
      ec[x] = std::conj(e[x]);
    }
    fams.push_back({"hopXR", {{OP_CD, 0, 0, 1}, {OP_C, 1, 0, -1}}, 0, bases(0, lx - 1), constant(-t)});
    fams.push_back({"hopXL", {{OP_CD, 1, 0, 1}, {OP_C, 0, 0, -1}}, 0, bases(0, lx - 1), constant(-t)});
    fams.push_back({"hopYF", {{OP_CD, 0, 0, 1}, {OP_C, 0, 0, -1}}, -1, bases(0, lx), e});
    fams.push_back({"hopYB", {{OP_CD, 0, 0, 1}, {OP_C, 0, 0, -1}}, 1, bases(0, lx), ec});
    fams.push_back({"nnX", {{OP_N, 0, 0, 1}, {OP_N, 1, 0, -1}}, 0, bases(0, lx - 1), constant(v)});
    fams.push_back({"nnY", {{OP_N, 0, 0, 1}, {OP_N, 0, 0, -1}}, -1, bases(0, lx), constant(v)});
  }
  // family rank = lexicographic order of names (the node sort order)
  std::vector<std::string> names;
  for (auto& f : fams) names.push_back(f.name);
  std::vector<std::string> sorted_names = names;
  std::sort(sorted_names.begin(), sorted_names.end());
  std::vector<int> rank(fams.size());
  std::vector<int> fam_of_rank(fams.size());
  for (size_t i = 0; i < fams.size(); ++i) {
    rank[i] = (int)(std::find(sorted_names.begin(), sorted_names.end(), names[i]) - sorted_names.begin());
    fam_of_rank[rank[i]] = (int)i;
  }

  auto onsite = [&](int x, int mm) -> double {
    return mixed ? -2.0 * t * std::cos(2.0 * pi * mm / ly + x * phi) : 0.0;
  };

  const Key R = key_R(), F = key_F();
  std::vector<std::vector<Key>> bonds(n + 1);
  std::vector<Trans> trans(n);
  bonds[0].push_back(R);
  for (int j = 0; j < n; ++j) {
    const int x = j / ly, mm = j % ly;
    std::map<Key, int> out_keys;
    Trans& tj = trans[j];
    for (const Key& key : bonds[j]) {
      if (key.kind == 2) { add_trans(tj, out_keys, F, F, mat_of(0), 1.0); continue; }
      struct Start { int f, xb, placed, lab, dn, dk; };
      std::vector<Start> starts;
      if (key.kind == 0) {
        add_trans(tj, out_keys, R, R, mat_of(0), 1.0);
        add_trans(tj, out_keys, R, F, mat_of(3), onsite(x, mm));
        for (int r = 0; r < (int)fams.size(); ++r) {
          int fi = fam_of_rank[r];
          for (int xb : fams[fi].bases) starts.push_back({fi, xb, 0, 0, 0, 0});
        }
      } else {
        starts.push_back({fam_of_rank[key.fam], key.xb, key.placed, key.lab, key.dn, key.dk});
      }
      for (const Start& st : starts) {
        const Family& fam = fams[st.f];
        const int nr = (int)fam.roles.size();
        bool dead = false;
        std::vector<int> allowed;
        for (int r = 0; r < nr; ++r) {
          if (st.placed & (1 << r)) continue;
          const Role& role = fam.roles[r];
          if (role.ring != kAnyRing && st.xb + role.ring < x) dead = true;
          if (role.ring == kAnyRing || st.xb + role.ring == x) allowed.push_back(r);
        }
        if (dead) continue;
        for (int sub = 0; sub < (1 << allowed.size()); ++sub) {
          int here = 0;
          for (size_t i = 0; i < allowed.size(); ++i)
            if (sub >> i & 1) here |= 1 << allowed[i];
          if (st.placed == 0 && here == 0) continue;
          Mat2 mat = local_op(fam.roles, st.placed, here);
          if (!mat.nonzero()) continue;
          cd coeff = st.placed == 0 ? fam.coeff[st.xb] : cd(1.0);
          int lab = st.lab, dn = st.dn, dk = st.dk;
          for (int r = 0; r < nr; ++r) {
            if (!(here >> r & 1)) continue;
            const Role& role = fam.roles[r];
            if (role.trig) {
              coeff *= trig_of(role.trig, mm, ly);
            } else {
              double ang = role.phase * 2.0 * pi * mm / ly;
              coeff *= cd(std::cos(ang), std::sin(ang));
            }
            lab = ((lab + role.label * mm) % ly + ly) % ly;
            if (role.op == OP_CD) { dn += 1; dk += mm; }
            else if (role.op == OP_C) { dn -= 1; dk -= mm; }
          }
          int placed2 = st.placed | here;
          Key src = st.placed == 0 ? R : key;
          if (placed2 == (1 << nr) - 1) {
            if (((lab - fam.target) % ly + ly) % ly == 0) add_trans(tj, out_keys, src, F, mat, coeff);
            continue;
          }
          Key dst;
          dst.kind = 1; dst.fam = rank[st.f]; dst.xb = st.xb; dst.placed = placed2; dst.lab = lab;
          dst.dn = dn; dst.dk = ((dk % ly) + ly) % ly;
          add_trans(tj, out_keys, src, dst, mat, coeff);
        }
      }
    }
    for (auto& kv : out_keys) bonds[j + 1].push_back(kv.first);  // std::map keeps them sorted
  }

  // trimming: keep nodes on some R -> F path
  std::vector<std::set<Key>> alive(n + 1), fwd(n + 1);
  for (const Key& k : bonds[n]) if (k.kind == 2) alive[n].insert(k);
  for (int j = n - 1; j >= 0; --j)
    for (const auto& kv : trans[j])
      if (alive[j + 1].count(kv.first.second)) alive[j].insert(kv.first.first);
  fwd[0].insert(R);
  for (int j = 0; j < n; ++j)
    for (const auto& kv : trans[j])
      if (fwd[j].count(kv.first.first)) fwd[j + 1].insert(kv.first.second);
  for (int j = 0; j <= n; ++j) {
    std::vector<Key> keep;
    for (const Key& k : bonds[j])
      if (alive[j].count(k) && fwd[j].count(k)) keep.push_back(k);
    bonds[j] = keep;
  }
  for (int j = 0; j < n; ++j) {
    std::set<Key> k0(bonds[j].begin(), bonds[j].end()), k1(bonds[j + 1].begin(), bonds[j + 1].end());
    Trans kept;
    for (const auto& kv : trans[j])
      if (k0.count(kv.first.first) && k1.count(kv.first.second)) kept.insert(kv);
    trans[j].swap(kept);
  }

  fuse(bonds, trans, n);

  out->n_sites = n;
  out->modulus = modulus;
  out->bond_charges.assign(n + 1, {});
  out->site_idx.assign(n, {});
  out->site_val.assign(n, {});
  for (int j = 0; j <= n; ++j)
    for (const Key& k : bonds[j]) {
      if (k.kind == 1) {
        out->bond_charges[j].push_back(k.dn);
        out->bond_charges[j].push_back(((k.dk % modulus) + modulus) % modulus);
      } else {
        out->bond_charges[j].push_back(0);
        out->bond_charges[j].push_back(0);
      }
    }
  for (int j = 0; j < n; ++j) {
    std::map<Key, int> i0, i1;
    for (size_t i = 0; i < bonds[j].size(); ++i) i0[bonds[j][i]] = (int)i;
    for (size_t i = 0; i < bonds[j + 1].size(); ++i) i1[bonds[j + 1][i]] = (int)i;
    std::vector<std::tuple<int, int, int, int, cd>> ent;
    for (const auto& kv : trans[j])
      for (int sp = 0; sp < 2; ++sp)
        for (int s = 0; s < 2; ++s)
          if (kv.second.a[sp][s] != cd(0.0))
            ent.emplace_back(i0[kv.first.first], i1[kv.first.second], sp, s, kv.second.a[sp][s]);
    std::sort(ent.begin(), ent.end(), [](const auto& a, const auto& b) {
      return std::make_tuple(std::get<0>(a), std::get<1>(a), std::get<2>(a), std::get<3>(a)) <
             std::make_tuple(std::get<0>(b), std::get<1>(b), std::get<2>(b), std::get<3>(b));
    });
    for (const auto& e : ent) {
      out->site_idx[j].push_back(std::get<0>(e));
      out->site_idx[j].push_back(std::get<1>(e));
      out->site_idx[j].push_back(std::get<2>(e));
      out->site_idx[j].push_back(std::get<3>(e));
      out->site_val[j].push_back(std::get<4>(e).real());
      out->site_val[j].push_back(std::get<4>(e).imag());
    }
  }
  return MRD_OK;
}

}  // namespace mrd
