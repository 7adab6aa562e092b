"""Finite-state-machine construction of the Hofstadter MPO in the real-space and the mixed
real/momentum-space basis (Sec. IV). Test infrastructure only.

The Hamiltonian is a sum of operator strings. An FSM (Sec. IV.A) generates every string as
one path from the ready node R to the final node F; the MPO matrix of site j holds, at
(row, column) = (node before j, node after j), the operator that the transition places on
site j (Sec. IV.B, Eq. M_example).

Nodes used here. Every Hamiltonian term family is a product of fermionic "roles"
f_1 f_2 ... f_n (each c or c+, or a number operator n), each tied to one ring, with a
coefficient that factorises into one phase per role, e^{i p 2 pi m / Ly} for a role placed
at momentum m (p = +1, -1 or 0). An intermediate node is (family, base ring, set of roles
already placed, cumulative label mod Ly). In the mixed basis the label is the cumulative
momentum placed so far, exactly the momentum-labelled nodes A_mu(k), C_mu(k) of Fig. 9 and
Fig. 10(a) (Sec. IV.D); the path closes into F only with total momentum 0 (mod Ly). In real
space the label is the cumulative position y, used to pin the partner site of a hop.

Jordan-Wigner (Sec. IV.C, Eq. JW): c_j = (prod_{i<j} Z_i) C_j with Z = 1 - 2n. For a role
product f_1..f_n the operator on site j is the ordered product over roles r of: identity
if r was placed left of j, its C/Cd/N if placed at j, Z if r is fermionic and still to be
placed right of j (identity for a pending number operator). Several roles may share a site
(e.g. c+_k c_k = n_k); a product that vanishes (Cd Cd) is not a transition.

Trimming (Sec. IV.D): nodes not reachable from R, or from which F cannot be reached, are
deleted. Merging: two nodes at one bond whose incoming columns are proportional (identical
pasts) are fused, summing their outgoing rows with the ratio; likewise for proportional
outgoing rows (identical futures). Both are exact rewrites of the same operator sum. This
is what reduces the real-space machine to D = 3 Ly + 2 (Sec. IV.C); tests pin that value.

Channel charge of a node: the charge (dN, dK) of the operators placed so far, with
c+ at momentum m carrying (+1, +m) and c carrying (-1, -m) (dK taken mod Ly; real space
carries no K). Entry W[w, w', s', s] is nonzero only if c_{w'} = c_w + q(s') - q(s).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

I2 = np.eye(2, dtype=np.complex128)
CD = np.array([[0, 0], [1, 0]], dtype=np.complex128)   # <1|Cd|0> = 1   (creation)
C = np.array([[0, 1], [0, 0]], dtype=np.complex128)    # <0|C|1> = 1    (annihilation)
NUM = np.array([[0, 0], [0, 1]], dtype=np.complex128)
Z = np.array([[1, 0], [0, -1]], dtype=np.complex128)
_OPS = {"cd": CD, "c": C, "n": NUM}
_ODD = {"cd": True, "c": True, "n": False}
_CHARGE_N = {"cd": 1, "c": -1, "n": 0}


def register_op(name: str, matrix, odd: bool = False, dn: int = 0):
    """Add a custom single-site operator (used to restate Eq. M_example with generic A, B)."""
    _OPS[name] = np.asarray(matrix, dtype=np.complex128)
    _ODD[name] = odd
    _CHARGE_N[name] = dn


@dataclass
class Role:
    op: str               # 'cd', 'c' or 'n'
    ring: int | None      # ring offset from the family's base ring (None: any ring)
    phase: int = 0        # placed at momentum m, contributes e^{i phase 2 pi m / Ly}
    label: int = 0        # contributes label * m (mixed) or label * y (real) to the node label
    trig: str = ""        # 'cos' / 'sin': contributes cos / sin(2 pi m / Ly) instead of a phase


@dataclass
class Family:
    name: str
    roles: list
    target: int           # path closes only if the summed label == target (mod Ly)
    coeff: callable       # coefficient as a function of the base ring x
    bases: list           # allowed base rings


@dataclass
class MPO:
    """Site tensors as sparse entry lists plus the node bookkeeping of every bond."""
    n_sites: int
    ly: int
    modulus: int                        # K modulus of the charges: Ly (mixed) or 1 (real)
    site_m: list                        # momentum (or y) label of each site
    bond_charges: list = field(default_factory=list)   # per bond: list of (dN, dK)
    bond_keys: list = field(default_factory=list)      # per bond: node keys (sort order)
    entries: list = field(default_factory=list)        # per site: list of (w, w', s', s, value)

    def dims(self):
        return [len(c) for c in self.bond_charges]

    def dense_site(self, j: int) -> np.ndarray:
        """W_j as an array [w, w', s', s]."""
        d0, d1 = len(self.bond_charges[j]), len(self.bond_charges[j + 1])
        w = np.zeros((d0, d1, 2, 2), dtype=np.complex128)
        for a, b, sp, s, val in self.entries[j]:
            w[a, b, sp, s] += val
        return w


def mixed_families(lx, ly, flux, t, v, penalty=None):
    """Term families of the mixed-basis Hamiltonian (Eqs. H_kin, H_k_int).

    Inter-ring hops  -t c+_{x,m} c_{x+1,m} and -t c+_{x+1,m} c_{x,m}.
    Intra-ring interaction (V/Ly) sum_q cos(q) n_{x,q} n_{x,-q}. Because n_{x,q} and
    n_{x,-q} commute, sum_q cos(q) n_q n_{-q} = sum_q e^{iq} n_q n_{-q}; writing
    e^{iq} = e^{i(k+q)} e^{-ik} attaches one phase to each operator of the first density,
    so the family is (V/Ly) sum e^{i(p1-p2) 2pi/Ly} c+_{p1} c_{p2} c+_{p3} c_{p4} over
    p1 - p2 + p3 - p4 = 0 (mod Ly).
    Inter-ring interaction (V/Ly) sum_q n_{x,-q} n_{x+1,q} (the two densities commute).
    Onsite -2t cos(k + x phi) n_{x,k} is a single-site R->F transition (not a family).
    Optional penalty (mu, N): mu (N_tot - N)^2 = mu N_tot^2 + mu(-2N) N_tot + mu N^2."""
    fams = [
        Family("hopR", [Role("cd", 0, 0, +1), Role("c", 1, 0, -1)], 0, lambda x: -t, list(range(lx - 1))),
        Family("hopL", [Role("cd", 1, 0, +1), Role("c", 0, 0, -1)], 0, lambda x: -t, list(range(lx - 1))),
        Family("intra", [Role("cd", 0, +1, +1), Role("c", 0, -1, -1), Role("cd", 0, 0, +1), Role("c", 0, 0, -1)],
               0, lambda x: v / ly, list(range(lx))),
        Family("inter", [Role("cd", 0, 0, +1), Role("c", 0, 0, -1), Role("cd", 1, 0, +1), Role("c", 1, 0, -1)],
               0, lambda x: v / ly, list(range(lx - 1))),
    ]
    if penalty is not None:
        mu, _ = penalty
        fams.append(Family("pen", [Role("n", None), Role("n", None)], 0, lambda x: mu, [0]))
    phi = 2 * math.pi * flux

    def onsite(x, m):
        return -2 * t * math.cos(2 * math.pi * m / ly + x * phi)
    return fams, onsite


def mixed_real_families(lx, ly, flux, t, v, penalty=None):
    """Term families of the mixed-basis Hamiltonian with real coefficients only (the sine /
    cosine machine of Sec. IV.D, Eq. rot). The phases of the intra-ring interaction come in
    pairs e^{+i alpha}, e^{-i alpha}; rotating each pair into cos alpha, sin alpha makes every
    MPO entry real. Written per term: the literal coefficient of c+_{p1} c_{p2} c+_{p3} c_{p4} in
    (V/Ly) sum_q cos(q) n_q n_{-q} is (V/Ly) cos((p1 - p2) alpha) = (V/Ly) [cos(p1 alpha)
    cos(p2 alpha) + sin(p1 alpha) sin(p2 alpha)], so the family splits into a cosine and a
    sine family whose first two roles each carry one real factor. The hops and the inter-ring
    interaction are real already (the note after Eq. rot)."""
    fams, onsite = mixed_families(lx, ly, flux, t, v, penalty)
    out = []
    for f in fams:
        if f.name != "intra":
            out.append(f)
            continue
        for trig in ("cos", "sin"):
            roles = [Role(r.op, r.ring, 0, r.label, trig if k < 2 else "") for k, r in enumerate(f.roles)]
            out.append(Family("intra" + trig[0], roles, f.target, f.coeff, f.bases))
    return out, onsite


def real_families(lx, ly, flux, t, v, penalty=None):
    """Term families of the real-space Hamiltonian (Eq. H_real); the label is the position
    y, so the hop around the ring c+_{x,y} c_{x,y+1} closes with label sum -1 (mod Ly)."""
    phi = 2 * math.pi * flux
    e = lambda x: complex(math.cos(x * phi), math.sin(x * phi))
    fams = [
        Family("hopXR", [Role("cd", 0, 0, +1), Role("c", 1, 0, -1)], 0, lambda x: -t, list(range(lx - 1))),
        Family("hopXL", [Role("cd", 1, 0, +1), Role("c", 0, 0, -1)], 0, lambda x: -t, list(range(lx - 1))),
        Family("hopYF", [Role("cd", 0, 0, +1), Role("c", 0, 0, -1)], -1, lambda x: -t * e(x), list(range(lx))),
        Family("hopYB", [Role("cd", 0, 0, +1), Role("c", 0, 0, -1)], +1, lambda x: -t * e(x).conjugate(),
               list(range(lx))),
        Family("nnX", [Role("n", 0, 0, +1), Role("n", 1, 0, -1)], 0, lambda x: v, list(range(lx - 1))),
        Family("nnY", [Role("n", 0, 0, +1), Role("n", 0, 0, -1)], -1, lambda x: v, list(range(lx))),
    ]
    if penalty is not None:
        mu, _ = penalty
        fams.append(Family("pen", [Role("n", None), Role("n", None)], 0, lambda x: mu, [0]))
    return fams, (lambda x, m: 0.0)


def _trig(kind: str, m: int, ly: int) -> float:
    """cos or sin of 2 pi m / Ly, exactly zero where the angle is a multiple of pi (sin) or an
    odd multiple of pi / 2 (cos): rounded library values there (~1e-16) would add spurious
    transitions to the machine."""
    if kind == "sin":
        return 0.0 if (2 * m) % ly == 0 else math.sin(2 * math.pi * m / ly)
    return 0.0 if (4 * m) % (2 * ly) == ly else math.cos(2 * math.pi * m / ly)


def _local_op(roles, placed: int, here: int) -> np.ndarray:
    """Ordered product over roles of: I (placed before), the role's operator (placed
    here), Z for a pending fermionic role, I for a pending number operator."""
    out = I2
    for r, role in enumerate(roles):
        bit = 1 << r
        if placed & bit:
            m = I2
        elif here & bit:
            m = _OPS[role.op]
        else:
            m = Z if _ODD[role.op] else I2
        out = out @ m
    return out


def build_mpo(lx: int, ly: int, flux: float, t: float, v: float, basis: str = "mixed",
              penalty=None, merge: bool = True) -> MPO:
    """Build, trim and merge the FSM MPO of the cylinder Hamiltonian.

    basis: 'mixed' (orbitals (x, m), charges (N, K mod Ly)), 'mixed_real' (the same orbitals
    and charges, the sine / cosine machine with real entries) or 'real' (orbitals (x, y), charge
    N only). penalty: optional (mu, N) adding mu (N_tot - N)^2, used only by the symmetry-free
    dense DMRG of this oracle."""
    if ly < 2:
        raise ValueError("Ly >= 2 required")
    make = {"mixed": mixed_families, "mixed_real": mixed_real_families, "real": real_families}[basis]
    fams, onsite = make(lx, ly, flux, t, v, penalty)
    modulus = 1 if basis == "real" else ly
    return build_fsm_mpo(lx, ly, fams, onsite, modulus, penalty=penalty, merge=merge)


def build_fsm_mpo(lx: int, ly: int, fams, onsite, modulus: int, penalty=None, merge: bool = True) -> MPO:
    """FSM -> MPO for arbitrary term families on lx rings of ly orbitals (chain order
    j = x * ly + m). onsite(x, m) is the coefficient of n on orbital (x, m)."""
    n = lx * ly
    site_m = [j % ly for j in range(n)]
    R, F = ("R",), ("F",)
    all_bits = {f.name: (1 << len(f.roles)) - 1 for f in fams}
    fam_by_name = {f.name: f for f in fams}

    def charge_of(key):
        if key in (R, F):
            return (0, 0)
        fname, x, placed, lab, dn, dk = key
        return (dn, dk % modulus)

    # ---- forward generation: bonds[j] = list of node keys, trans[j] = {(a, b): 2x2}
    bonds = [[R]]
    trans = []
    for j in range(n):
        x, m = divmod(j, ly)
        out_keys = {}
        tj = {}

        def add(src, dst, mat, coeff):
            if coeff == 0 or not np.any(mat):
                return
            if dst not in out_keys:
                out_keys[dst] = len(out_keys)
            k = (src, dst)
            tj[k] = tj.get(k, 0) + coeff * mat

        for key in bonds[j]:
            if key == F:
                add(F, F, I2, 1.0)
                continue
            if key == R:
                add(R, R, I2, 1.0)
                # single-site terms: onsite energy and the penalty's linear + constant part
                c1 = onsite(x, m)
                if penalty is not None:
                    mu, nn = penalty
                    c1 += mu * (-2 * nn)
                    add(R, F, I2, mu * nn * nn / n)
                add(R, F, NUM, c1)
                starts = [(f, xb, 0, 0, 0, 0) for f in fams for xb in f.bases]
            else:
                fname, xb, placed, lab, dn, dk = key
                starts = [(fam_by_name[fname], xb, placed, lab, dn, dk)]
            for fam, xb, placed, lab, dn, dk in starts:
                nr = len(fam.roles)
                pending = [r for r in range(nr) if not placed & (1 << r)]
                # pending roles whose ring is already behind this site can never be placed
                if any(fam.roles[r].ring is not None and xb + fam.roles[r].ring < x for r in pending):
                    continue
                allowed = [r for r in pending if fam.roles[r].ring is None or xb + fam.roles[r].ring == x]
                for sub in range(1 << len(allowed)):
                    here = 0
                    for i, r in enumerate(allowed):
                        if sub >> i & 1:
                            here |= 1 << r
                    if placed == 0 and here == 0:
                        continue          # still in R (the R->R identity covers it)
                    mat = _local_op(fam.roles, placed, here)
                    if not np.any(mat):
                        continue
                    coeff = fam.coeff(xb) if placed == 0 else 1.0
                    lab2, dn2, dk2 = lab, dn, dk
                    for r in range(nr):
                        if here >> r & 1:
                            role = fam.roles[r]
                            if role.trig:
                                coeff = coeff * _trig(role.trig, m, ly)
                            else:
                                coeff = coeff * complex(math.cos(role.phase * 2 * math.pi * m / ly),
                                                        math.sin(role.phase * 2 * math.pi * m / ly))
                            lab2 = (lab2 + role.label * m) % ly
                            dn2 += _CHARGE_N[role.op]
                            if role.op == "cd":
                                dk2 += m
                            elif role.op == "c":
                                dk2 -= m
                    placed2 = placed | here
                    src = R if placed == 0 else key
                    if placed2 == all_bits[fam.name]:
                        if lab2 % ly == fam.target % ly:
                            add(src, F, mat, coeff)
                        continue
                    add(src, (fam.name, xb, placed2, lab2, dn2, dk2 % ly), mat, coeff)
        bonds.append(sorted(out_keys, key=_sort_key))
        trans.append(tj)

    # ---- trimming: keep nodes on some R -> F path
    alive = [set() for _ in range(n + 1)]
    alive[n] = {F} & set(bonds[n])
    for j in range(n - 1, -1, -1):
        alive[j] = {a for (a, b) in trans[j] if b in alive[j + 1]}
    fwd = [set() for _ in range(n + 1)]
    fwd[0] = {R}
    for j in range(n):
        fwd[j + 1] = {b for (a, b) in trans[j] if a in fwd[j]}
    for j in range(n + 1):
        bonds[j] = [k for k in bonds[j] if k in alive[j] and k in fwd[j]]
    for j in range(n):
        keep0, keep1 = set(bonds[j]), set(bonds[j + 1])
        trans[j] = {(a, b): mtx for (a, b), mtx in trans[j].items() if a in keep0 and b in keep1}

    if merge:
        _merge(bonds, trans, n)

    mpo = MPO(n_sites=n, ly=ly, modulus=modulus, site_m=site_m)
    for j in range(n + 1):
        mpo.bond_keys.append(list(bonds[j]))
        mpo.bond_charges.append([charge_of(k) for k in bonds[j]])
    for j in range(n):
        i0 = {k: i for i, k in enumerate(bonds[j])}
        i1 = {k: i for i, k in enumerate(bonds[j + 1])}
        ent = []
        for (a, b), mtx in sorted(trans[j].items(), key=lambda kv: (i0[kv[0][0]], i1[kv[0][1]])):
            for sp in (0, 1):
                for s in (0, 1):
                    if mtx[sp, s] != 0:
                        ent.append((i0[a], i1[b], sp, s, complex(mtx[sp, s])))
        mpo.entries.append(ent)
    return mpo


def _sort_key(key):
    if key == ("R",):
        return (0,)
    if key == ("F",):
        return (2,)
    fname, xb, placed, lab, dn, dk = key
    return (1, fname, xb, placed, lab, dn, dk)


def _vec(trans_j, node, side):
    """Incoming column (side=0) or outgoing row (side=1) of a node as {(other, s', s): val}."""
    out = {}
    for (a, b), mtx in trans_j.items():
        if (b if side == 0 else a) != node:
            continue
        other = a if side == 0 else b
        for sp in (0, 1):
            for s in (0, 1):
                if mtx[sp, s] != 0:
                    out[(_sort_key(other), sp, s)] = mtx[sp, s]
    return out


def _proportional(u, w, tol=1e-10):
    """Return f with u = f * w if the two sparse vectors are proportional, else None."""
    if set(u) != set(w) or not u:
        return None
    k0 = min(u)
    f = u[k0] / w[k0]
    for k in u:
        if abs(u[k] - f * w[k]) > tol * max(1.0, abs(u[k])):
            return None
    return f


def _merge(bonds, trans, n):
    """Fuse nodes with proportional pasts (left to right), then with proportional futures
    (right to left), repeating until nothing changes. R and F are never fused away."""
    changed = True
    while changed:
        changed = False
        for j in range(1, n):               # nodes at bond j; pasts from trans[j-1]
            reps = []
            for node in list(bonds[j]):
                col = _vec(trans[j - 1], node, 0)
                hit = None
                for rep, rcol in reps:
                    f = _proportional(col, rcol)
                    if f is not None:
                        hit = (rep, f)
                        break
                if hit is None:
                    reps.append((node, col))
                    continue
                rep, f = hit
                # column(node) = f * column(rep): fold node's outgoing row into rep's
                for (a, b) in [k for k in trans[j] if k[0] == node]:
                    mtx = trans[j].pop((a, b))
                    trans[j][(rep, b)] = trans[j].get((rep, b), 0) + f * mtx
                for k in [k for k in trans[j - 1] if k[1] == node]:
                    trans[j - 1].pop(k)
                bonds[j].remove(node)
                changed = True
        for j in range(n - 1, 0, -1):       # nodes at bond j; futures from trans[j]
            reps = []
            for node in list(bonds[j]):
                row = _vec(trans[j], node, 1)
                hit = None
                for rep, rrow in reps:
                    f = _proportional(row, rrow)
                    if f is not None:
                        hit = (rep, f)
                        break
                if hit is None:
                    reps.append((node, row))
                    continue
                rep, f = hit
                for (a, b) in [k for k in trans[j - 1] if k[1] == node]:
                    mtx = trans[j - 1].pop((a, b))
                    trans[j - 1][(a, rep)] = trans[j - 1].get((a, rep), 0) + f * mtx
                for k in [k for k in trans[j] if k[0] == node]:
                    trans[j].pop(k)
                bonds[j].remove(node)
                changed = True
        for j in range(n):                   # drop transitions that cancelled to zero
            for k in [k for k, mtx in trans[j].items() if not np.any(np.abs(mtx) > 1e-14)]:
                trans[j].pop(k)


def apply_mpo(mpo: MPO, psi: np.ndarray) -> np.ndarray:
    """H|psi> for a dense state psi over all 2^n occupation patterns (bit o of the index is
    the occupation of orbital o), contracting the MPO entries site by site."""
    n = mpo.n_sites
    # axes: axis j of the tensor is orbital n-1-j (C order of the bit index)
    cur = {0: psi.reshape([2] * n)}   # node index at bond 0 -> tensor
    for j in range(n):
        ax = n - 1 - j
        nxt = {}
        for a, b, sp, s, val in mpo.entries[j]:
            if a not in cur:
                continue
            src = np.take(cur[a], s, axis=ax)
            if b not in nxt:
                nxt[b] = np.zeros_like(cur[a])
            idx = [slice(None)] * n
            idx[ax] = sp
            nxt[b][tuple(idx)] += val * src
        cur = nxt
    f_idx = len(mpo.bond_charges[n]) - 1
    return cur.get(f_idx, np.zeros_like(psi.reshape([2] * n))).reshape(-1)
