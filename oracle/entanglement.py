"""Momentum-resolved entanglement spectrum (Sec. III.C: the Schmidt decomposition
|psi> = sum_alpha lambda_alpha |L_alpha>|R_alpha>, with Schmidt states labelled by the
particle number N and the ring momentum K of the left part; the entanglement energies are
-2 ln lambda). Test infrastructure only.

Two independent computations:

* `schmidt_spectrum`: from a many-body state (exact diagonalisation), by grouping its Fock
  components by the left orbitals' occupation (orbitals o < cut in chain order) and taking
  the singular values of each (N_left, K_left) block;
* `free_fermion_spectrum`: at V = 0, from the one-body correlation matrix of the left
  orbitals (Peschel, J. Phys. A 36, L205 (2003)): its eigenvalues zeta_k give the many-body
  Schmidt weights as products of zeta_k (mode occupied) and 1 - zeta_k (empty).
"""
from __future__ import annotations

import itertools
import math

import numpy as np


def schmidt_spectrum(psi: np.ndarray, basis: np.ndarray, cut: int, ly: int, tol: float = 1e-12) -> dict:
    """Schmidt values of psi (components over the Fock bitmasks `basis`, mixed basis: orbital
    o = x*Ly + m carries momentum m) across the cut between orbitals < cut and >= cut.
    Returns {(N_left, K_left): values sorted descending, values above tol only}."""
    mask = (1 << cut) - 1
    sectors: dict = {}
    for amp, st in zip(psi, basis):
        st = int(st)
        left, right = st & mask, st >> cut
        n_l = bin(left).count("1")
        k_l = sum(o % ly for o in range(cut) if (left >> o) & 1) % ly
        sectors.setdefault((n_l, k_l), []).append((left, right, amp))
    out = {}
    for key, items in sectors.items():
        rows = {l: i for i, l in enumerate(sorted({l for l, _, _ in items}))}
        cols = {r: i for i, r in enumerate(sorted({r for _, r, _ in items}))}
        m = np.zeros((len(rows), len(cols)), dtype=np.complex128)
        for l, r, a in items:
            m[rows[l], cols[r]] = a
        s = np.linalg.svd(m, compute_uv=False)
        s = s[s > tol]
        if len(s):
            out[key] = np.sort(s)[::-1]
    return out


def free_fermion_spectrum(lx: int, ly: int, flux: float, t: float, n_part: int, cut: int,
                          tol: float = 1e-12) -> dict:
    """Schmidt values of the V = 0 ground state with n_part particles (Slater determinant of
    the n_part lowest levels of Eq. H_kin; the level at the Fermi energy must not be
    degenerate) across the same cut, from the left orbitals' correlation matrix."""
    phi = 2 * math.pi * flux
    modes = []   # (energy, m, vector over x)
    for m in range(ly):
        k = 2 * math.pi * m / ly
        h = np.diag([-2 * t * math.cos(k + x * phi) for x in range(lx)]).astype(np.float64)
        for x in range(lx - 1):
            h[x, x + 1] = h[x + 1, x] = -t
        e, v = np.linalg.eigh(h)
        modes.extend((e[j], m, v[:, j]) for j in range(lx))
    modes.sort(key=lambda z: z[0])
    if n_part < len(modes) and abs(modes[n_part][0] - modes[n_part - 1][0]) < 1e-9:
        raise ValueError("degenerate Fermi level: the free ground state is not unique")
    # correlation matrix <c+_o c_o'> restricted to the left orbitals; block diagonal in m
    n = lx * ly
    corr = np.zeros((n, n), dtype=np.complex128)
    for _, m, v in modes[:n_part]:
        phi_o = np.zeros(n)
        phi_o[[x * ly + m for x in range(lx)]] = v
        corr += np.outer(phi_o.conj(), phi_o)
    ent = []   # (zeta, m) of each entanglement mode
    for m in range(ly):
        idx = [o for o in range(cut) if o % ly == m]
        if not idx:
            continue
        z = np.linalg.eigvalsh(corr[np.ix_(idx, idx)])
        # modes within rounding of 0 or 1 are exactly empty or full (e.g. when the right part
        # cannot hold the particles): snap them so that their products vanish exactly
        z = np.where(z < 1e-13, 0.0, np.where(z > 1.0 - 1e-13, 1.0, z))
        ent.extend((float(zz), m) for zz in z)
    out: dict = {}
    for occ in itertools.product((0, 1), repeat=len(ent)):
        w = 1.0
        for o, (z, _) in zip(occ, ent):
            w *= z if o else 1.0 - z
        if w <= tol * tol:
            continue
        key = (sum(occ), sum(m for o, (_, m) in zip(occ, ent) if o) % ly)
        out.setdefault(key, []).append(math.sqrt(w))
    return {k: np.sort(np.array(v))[::-1] for k, v in out.items()}
