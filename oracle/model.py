"""Many-body Hamiltonians of the interacting Hofstadter cylinder by direct operator
application on Fock states (exact diagonalisation). Test infrastructure only.

Lattice: rings x = 0..Lx-1 along the cylinder (open ends), positions y = 0..Ly-1 around
it (periodic). Flux phi = 2*pi*p/q per plaquette in Landau gauge A = (0, B x), so hops
around the ring carry e^{i x phi} (Sec. III.A, Eq. H; Sec. IV.C, Eq. H_real).

Chain order (Sec. II): orbital index o = x*Ly + y in real space, o = x*Ly + m in the mixed
basis, where m labels the ring momentum k_m = 2*pi*m/Ly. The Jordan-Wigner sign of c_o on
a Fock state is (-1)^(number of occupied orbitals with index < o) (Sec. IV.C, Eq. JW).

Fourier convention (the paper does not state it): c_{x,y} = Ly^{-1/2} sum_m e^{i k_m y}
c_{x,m}. With it the mixed-basis Hamiltonian written below reproduces the real-space
spectrum; tests/test_oracle_model.py pins this.
"""
from __future__ import annotations

import itertools
import math

import numpy as np

# ---------------------------------------------------------------- Fock-space machinery


def fock_basis(n_orb: int, n_part: int) -> np.ndarray:
    """All n_orb-bit occupation bitmasks with n_part ones, ascending (uint64)."""
    states = [sum(1 << o for o in occ) for occ in itertools.combinations(range(n_orb), n_part)]
    return np.array(sorted(states), dtype=np.uint64)


def _popcount(a: np.ndarray) -> np.ndarray:
    return np.bitwise_count(a).astype(np.int64)


def apply_ops(states: np.ndarray, ops):
    """Apply an operator product to many Fock states at once.

    ops: sequence of (kind, orbital), kind in {'c', 'cd'}, written left to right as in the
    operator product; the rightmost acts first. Returns (new_states, amplitude, alive)."""
    st = states.copy()
    amp = np.ones(len(st), dtype=np.float64)
    alive = np.ones(len(st), dtype=bool)
    for kind, o in reversed(ops):
        bit = np.uint64(1) << np.uint64(o)
        occ = (st & bit) != 0
        below = st & (bit - np.uint64(1))
        sign = 1.0 - 2.0 * (_popcount(below) & 1)
        if kind == "c":
            alive &= occ
            st = st & ~bit
        elif kind == "cd":
            alive &= ~occ
            st = st | bit
        else:
            raise ValueError(kind)
        amp *= sign
    return st, amp, alive


class SectorOperator:
    """Accumulates a many-body operator restricted to a fixed-particle-number basis."""

    def __init__(self, basis: np.ndarray):
        self.basis = basis
        self.dim = len(basis)
        self.rows, self.cols, self.vals = [], [], []

    def add(self, coeff: complex, ops):
        if coeff == 0:
            return
        new, amp, alive = apply_ops(self.basis, ops)
        idx = np.nonzero(alive)[0]
        if len(idx) == 0:
            return
        tgt = np.searchsorted(self.basis, new[idx])
        ok = (tgt < self.dim)
        ok[ok] &= self.basis[tgt[ok]] == new[idx][ok]
        idx, tgt = idx[ok], tgt[ok]
        self.rows.append(tgt)
        self.cols.append(idx)
        self.vals.append(coeff * amp[idx])

    def dense(self) -> np.ndarray:
        h = np.zeros((self.dim, self.dim), dtype=np.complex128)
        for r, c, v in zip(self.rows, self.cols, self.vals):
            np.add.at(h, (r, c), v)
        return h


# ---------------------------------------------------------------- Hamiltonians


def real_space_hamiltonian(lx: int, ly: int, flux: float, t: float, v: float, n_part: int,
                           basis=None) -> np.ndarray:
    """Dense H_real = H_kin + H_int of Sec. IV.C (Eq. H_real) in the N-particle sector.

    H_kin = -t sum_x [ sum_y c+_{x,y} c_{x+1,y} + e^{i x phi} sum_y c+_{x,y} c_{x,y+1} ] + H.c.
    H_int =  V sum_x [ sum_y n_{x,y} n_{x+1,y} + sum_y n_{x,y} n_{x,y+1} ]
    with y+1 taken mod Ly, x+1 terms only for x < Lx-1 (open cylinder), phi = 2 pi flux."""
    n = lx * ly
    basis = fock_basis(n, n_part) if basis is None else basis
    op = SectorOperator(basis)
    phi = 2 * math.pi * flux
    o = lambda x, y: x * ly + (y % ly)
    for x in range(lx):
        for y in range(ly):
            if x + 1 < lx:
                op.add(-t, [("cd", o(x, y)), ("c", o(x + 1, y))])
                op.add(-t, [("cd", o(x + 1, y)), ("c", o(x, y))])
                op.add(v, [("cd", o(x, y)), ("c", o(x, y)), ("cd", o(x + 1, y)), ("c", o(x + 1, y))])
            ph = complex(math.cos(x * phi), math.sin(x * phi))
            op.add(-t * ph, [("cd", o(x, y)), ("c", o(x, y + 1))])
            op.add(-t * ph.conjugate(), [("cd", o(x, y + 1)), ("c", o(x, y))])
            op.add(v, [("cd", o(x, y)), ("c", o(x, y)), ("cd", o(x, y + 1)), ("c", o(x, y + 1))])
    return op.dense()


def mixed_space_hamiltonian(lx: int, ly: int, flux: float, t: float, v: float, n_part: int,
                            basis=None) -> np.ndarray:
    """Dense mixed real/momentum-space H of Sec. IV.D in the N-particle sector.

    H_kin = -t sum_{x,k} [ (c+_{x,k} c_{x+1,k} + H.c.) + 2 cos(k + x phi) n_{x,k} ]  (Eq. H_kin)
    H_int = (V/Ly) sum_{x,q} [ cos(q) n_{x,q} n_{x,-q} + n_{x+1,q} n_{x,-q} ]         (Eq. H_k_int)
    with n_{x,q} = sum_k c+_{x,k+q} c_{x,k} expanded literally (not normal ordered),
    momenta k = 2 pi m / Ly, q = 2 pi m_q / Ly, indices mod Ly."""
    n = lx * ly
    basis = fock_basis(n, n_part) if basis is None else basis
    op = SectorOperator(basis)
    phi = 2 * math.pi * flux
    o = lambda x, m: x * ly + (m % ly)
    for x in range(lx):
        for m in range(ly):
            k = 2 * math.pi * m / ly
            op.add(-2 * t * math.cos(k + x * phi), [("cd", o(x, m)), ("c", o(x, m))])
            if x + 1 < lx:
                op.add(-t, [("cd", o(x, m)), ("c", o(x + 1, m))])
                op.add(-t, [("cd", o(x + 1, m)), ("c", o(x, m))])
        for mq in range(ly):
            cq = math.cos(2 * math.pi * mq / ly)
            for k1 in range(ly):          # n_{x,q} term index k
                for k2 in range(ly):      # n_{x,-q} term index k'
                    # cos q  c+_{x,k+q} c_{x,k} c+_{x,k'-q} c_{x,k'}
                    op.add(v / ly * cq, [("cd", o(x, k1 + mq)), ("c", o(x, k1)),
                                          ("cd", o(x, k2 - mq)), ("c", o(x, k2))])
                    if x + 1 < lx:
                        # n_{x+1,q} n_{x,-q} = c+_{x+1,k+q} c_{x+1,k} c+_{x,k'-q} c_{x,k'}
                        op.add(v / ly, [("cd", o(x + 1, k1 + mq)), ("c", o(x + 1, k1)),
                                        ("cd", o(x, k2 - mq)), ("c", o(x, k2))])
    return op.dense()


# ---------------------------------------------------------------- single-particle problem


def single_particle_levels_momentum(lx: int, ly: int, flux: float, t: float) -> np.ndarray:
    """Closed form at V = 0: for each ring momentum m, the Lx x Lx tridiagonal matrix with
    diagonal -2t cos(k_m + x phi) and off-diagonal -t (Eq. H_kin); union of all spectra,
    sorted ascending."""
    phi = 2 * math.pi * flux
    levels = []
    for m in range(ly):
        k = 2 * math.pi * m / ly
        h = np.diag([-2 * t * math.cos(k + x * phi) for x in range(lx)]).astype(np.float64)
        for x in range(lx - 1):
            h[x, x + 1] = h[x + 1, x] = -t
        levels.extend(np.linalg.eigvalsh(h))
    return np.sort(np.array(levels))


def single_particle_levels_real(lx: int, ly: int, flux: float, t: float) -> np.ndarray:
    """Spectrum of the real-space one-body hopping matrix h (H_kin = sum h_ij c+_i c_j)."""
    phi = 2 * math.pi * flux
    n = lx * ly
    h = np.zeros((n, n), dtype=np.complex128)
    o = lambda x, y: x * ly + (y % ly)
    for x in range(lx):
        for y in range(ly):
            if x + 1 < lx:
                h[o(x, y), o(x + 1, y)] += -t
                h[o(x + 1, y), o(x, y)] += -t
            ph = complex(math.cos(x * phi), math.sin(x * phi))
            h[o(x, y), o(x, y + 1)] += -t * ph
            h[o(x, y + 1), o(x, y)] += -t * ph.conjugate()
    return np.sort(np.linalg.eigvalsh(h))


def free_fermion_ground_energy(lx: int, ly: int, flux: float, t: float, n_part: int) -> float:
    """E_0 at V = 0: the sum of the n_part lowest single-particle levels (Pauli principle)."""
    return float(np.sum(single_particle_levels_momentum(lx, ly, flux, t)[:n_part]))


def ground_energy(h: np.ndarray) -> float:
    return float(np.linalg.eigvalsh(h)[0])


def total_momentum(lx: int, ly: int, state: int) -> int:
    """Ring momentum K = sum of m over occupied mixed-basis orbitals, mod Ly."""
    return sum(o % ly for o in range(lx * ly) if (state >> o) & 1) % ly
