"""Pins of oracle.dmrg (dense two-site DMRG) against ED, closed forms and invariants."""
import numpy as np
import pytest

import synth
from oracle import dmrg as D
from oracle import model
from oracle import mpo as M


def test_lanczos_matches_dense_eigensolver():
    rng = np.random.default_rng(3)
    a = rng.standard_normal((120, 120)) + 1j * rng.standard_normal((120, 120))
    h = a + a.conj().T
    e, v, it = D.lanczos_ground(lambda x: h @ x, rng.standard_normal(120) + 0j, kmax=120, tol=1e-15)
    w = np.linalg.eigvalsh(h)
    assert abs(e - w[0]) < 1e-10 * abs(w[0])
    assert np.linalg.norm(h @ v - e * v) < 1e-6 * abs(e)


def test_truncate_svd_properties():
    rng = np.random.default_rng(4)
    t = rng.standard_normal((30, 22)) + 1j * rng.standard_normal((30, 22))
    t /= np.linalg.norm(t)
    u, s, vh, disc = D.truncate_svd(t, 100)
    assert np.linalg.norm(u @ np.diag(s) @ vh - t) < 1e-13
    assert np.allclose(u.conj().T @ u, np.eye(len(s)), atol=1e-13)
    assert np.allclose(vh @ vh.conj().T, np.eye(len(s)), atol=1e-13)
    assert abs(np.sum(s ** 2) - 1) < 1e-13 and disc < 1e-25
    u, s, vh, disc = D.truncate_svd(t, 5)
    full = np.linalg.svd(t, compute_uv=False)
    assert len(s) == 5 and abs(disc - np.sum(full[5:] ** 2)) < 1e-13


@pytest.mark.parametrize("basis", ["mixed", "real"])
@pytest.mark.parametrize("lx,ly,n,flux,v", [(2, 4, 2, 0.25, 1.0), (2, 3, 2, 1 / 3, 0.5)])
def test_dmrg_exact_bond_dimension_matches_ed(basis, lx, ly, n, flux, v):
    mpo = M.build_mpo(lx, ly, flux, 1.0, v, basis, penalty=(20.0, n))
    res = D.dmrg(mpo, 64, sweeps=8, seed=11)
    e_ed = model.ground_energy(model.real_space_hamiltonian(lx, ly, flux, 1.0, v, n))
    assert abs(res["energy"] - e_ed) < 1e-10 * abs(e_ed)
    h = M.build_mpo(lx, ly, flux, 1.0, v, basis)
    assert abs(D.mps_expectation_mpo(res["mps"], h).real - e_ed) < 1e-10 * abs(e_ed)
    num = M.build_mpo(lx, ly, 0.0, 0.0, 0.0, basis, penalty=(1.0, 0))   # N_tot^2
    assert abs(D.mps_expectation_mpo(res["mps"], num).real - n * n) < 1e-8


def test_dmrg_free_fermions_closed_form():
    lx, ly, n = 3, 3, 3
    mpo = M.build_mpo(lx, ly, 1 / 3, 1.0, 0.0, "mixed", penalty=(20.0, n))
    res = D.dmrg(mpo, 64, sweeps=8, seed=3)
    e0 = model.free_fermion_ground_energy(lx, ly, 1 / 3, 1.0, n)
    assert abs(res["energy"] - e0) < 1e-10 * abs(e0)


def test_dmrg_truncated_is_variational():
    lx, ly, n = 3, 4, 3
    mpo = M.build_mpo(lx, ly, 0.25, 1.0, 1.0, "mixed", penalty=(20.0, n))
    res = D.dmrg(mpo, 6, sweeps=4, seed=5)
    e_ed = model.ground_energy(model.mixed_space_hamiltonian(lx, ly, 0.25, 1.0, 1.0, n))
    assert res["energy"] > e_ed - 1e-12


def test_heff_hermitian_with_genuine_environments():
    """With environments contracted from an MPS and a Hermitian MPO, H_eff is Hermitian."""
    lx, ly = 2, 4
    mpo = M.build_mpo(lx, ly, 0.25, 1.0, 1.0, "mixed")
    n = lx * ly
    mps = D.random_mps(n, 8, 9)
    ws = [mpo.dense_site(j) for j in range(n)]
    i = 3
    L = np.ones((1, 1, 1), dtype=complex)
    for j in range(i):
        L = D.env_left_update(L, mps[j], ws[j])
    R = np.ones((1, 1, 1), dtype=complex)
    for j in range(n - 1, i + 1, -1):
        R = D.env_right_update(R, mps[j], ws[j])
    shape = (L.shape[1], 2, 2, R.shape[1])
    u = synth.complex_pm1(1, int(np.prod(shape))).reshape(shape)
    v = synth.complex_pm1(2, int(np.prod(shape))).reshape(shape)
    hv = D.heff_apply_dense(L, ws[i], ws[i + 1], R, v)
    hu = D.heff_apply_dense(L, ws[i], ws[i + 1], R, u)
    a, b = np.vdot(u, hv), np.vdot(v, hu)
    assert abs(a - b.conjugate()) < 1e-12 * abs(a)


def test_env_update_matches_dense_expectation():
    """<psi|H|psi> from the left-environment transfer equals the dense-vector value."""
    lx, ly = 2, 3
    mpo = M.build_mpo(lx, ly, 1 / 3, 1.0, 0.8, "mixed")
    mps = D.random_mps(lx * ly, 4, 21)
    psi = mps[0]
    for a in mps[1:]:
        psi = np.tensordot(psi, a, axes=([-1], [0]))
    n = lx * ly
    psi = psi.reshape([2] * n).transpose(list(range(n))[::-1]).reshape(-1)
    dense = np.vdot(psi, M.apply_mpo(mpo, psi)) / np.vdot(psi, psi)
    assert abs(D.mps_expectation_mpo(mps, mpo) - dense) < 1e-12 * abs(dense)
    # right transfer gives the same number
    R = np.ones((1, 1, 1), dtype=complex)
    Nn = np.ones((1, 1), dtype=complex)
    for j in range(n - 1, -1, -1):
        R = D.env_right_update(R, mps[j], mpo.dense_site(j))
        Nn = np.einsum("csb,be,fse->cf", mps[j], Nn, mps[j].conj())
    assert abs(R[0, 0, 0] / Nn[0, 0] - dense) < 1e-12 * abs(dense)


@pytest.mark.slow
def test_dmrg_config1_truncated():
    """4 x 4 cylinder, N = 4, chi = 24 (the centre bond needs 163 for exactness): the
    energy is an upper bound close to ED."""
    mpo = M.build_mpo(4, 4, 0.25, 1.0, 1.0, "mixed", penalty=(20.0, 4))
    res = D.dmrg(mpo, 24, sweeps=2, seed=1234)
    e_ed = model.ground_energy(model.mixed_space_hamiltonian(4, 4, 0.25, 1.0, 1.0, 4))
    assert e_ed - 1e-10 < res["energy"] < e_ed + 2e-2
