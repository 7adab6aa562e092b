"""Oracle entanglement spectrum (Sec. III.C) against the free-fermion closed form.

At V = 0 the ground state is a Slater determinant, and its Schmidt values across any cut
follow from the eigenvalues of the left orbitals' correlation matrix (Peschel 2003). The
oracle's many-body route (ED ground vector, blocks by the left part's (N, K), SVD) must give
the same spectrum in every sector; the union of the sector spectra must also equal the
singular values of the unblocked coefficient matrix, and the weights must sum to 1."""
import numpy as np
import pytest

from oracle import entanglement as E
from oracle import model


def _ground(lx, ly, fq, v, n):
    basis = model.fock_basis(lx * ly, n)
    h = model.mixed_space_hamiltonian(lx, ly, 1.0 / fq, 1.0, v, n, basis=basis)
    w, vec = np.linalg.eigh(h)
    assert w[1] - w[0] > 1e-8
    return vec[:, 0], basis


@pytest.mark.parametrize("lx,ly,fq,n", [(3, 3, 3, 3), (4, 3, 3, 4), (3, 4, 4, 3), (3, 2, 2, 3)])
def test_schmidt_spectrum_equals_free_fermion_closed_form(lx, ly, fq, n):
    psi, basis = _ground(lx, ly, fq, 0.0, n)
    for cut in range(1, lx * ly):
        got = E.schmidt_spectrum(psi, basis, cut, ly, tol=1e-6)
        ref = E.free_fermion_spectrum(lx, ly, 1.0 / fq, 1.0, n, cut, tol=1e-6)
        assert set(got) == set(ref), (cut, sorted(got), sorted(ref))
        for key in ref:
            assert len(got[key]) == len(ref[key])
            assert np.max(np.abs(got[key] - ref[key])) < 1e-9


def test_schmidt_spectrum_invariants_interacting():
    lx, ly, n = 3, 4, 3
    psi, basis = _ground(lx, ly, 4, 1.0, n)
    for cut in (4, 6, 8):
        sec = E.schmidt_spectrum(psi, basis, cut, ly)
        allv = np.sort(np.concatenate(list(sec.values())))[::-1]
        assert abs(np.sum(allv ** 2) - 1.0) < 1e-12
        mask = (1 << cut) - 1
        lefts = sorted({int(s) & mask for s in basis})
        rights = sorted({int(s) >> cut for s in basis})
        li, ri = {l: i for i, l in enumerate(lefts)}, {r: i for i, r in enumerate(rights)}
        m = np.zeros((len(lefts), len(rights)), dtype=np.complex128)
        for a, s in zip(psi, basis):
            m[li[int(s) & mask], ri[int(s) >> cut]] = a
        full = np.linalg.svd(m, compute_uv=False)
        full = np.sort(full[full > 1e-12])[::-1]
        assert len(full) == len(allv)
        assert np.max(np.abs(full - allv)) < 1e-12
