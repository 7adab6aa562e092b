"""Pins of oracle.mpo (FSM -> MPO) against exact diagonalisation and the paper's values."""
import numpy as np
import pytest

from oracle import model
from oracle import mpo as M

SMALL = [(2, 4, 0.25, 1.0), (3, 3, 1 / 3, 0.7), (2, 5, 0.2, 1.3), (1, 6, 1 / 6, 1.0)]


def _full_h(basis, lx, ly, flux, v):
    full = np.arange(2 ** (lx * ly), dtype=np.uint64)
    f = model.real_space_hamiltonian if basis == "real" else model.mixed_space_hamiltonian
    return f(lx, ly, flux, 1.0, v, 0, basis=full)


@pytest.mark.parametrize("basis", ["real", "mixed", "mixed_real"])
@pytest.mark.parametrize("lx,ly,flux,v", SMALL)
def test_mpo_equals_ed_operator(basis, lx, ly, flux, v):
    """The MPO applied to random states of the whole Fock space equals the ED operator."""
    h = _full_h(basis, lx, ly, flux, v)
    mpo = M.build_mpo(lx, ly, flux, 1.0, v, basis)
    rng = np.random.default_rng(5)
    for _ in range(2):
        psi = rng.standard_normal(2 ** (lx * ly)) + 1j * rng.standard_normal(2 ** (lx * ly))
        ref = h @ psi
        assert np.max(np.abs(M.apply_mpo(mpo, psi) - ref)) < 1e-13 * np.max(np.abs(ref))


@pytest.mark.parametrize("basis", ["real", "mixed"])
def test_mpo_penalty(basis):
    lx, ly, mu, nn = 2, 4, 3.0, 2
    h = _full_h(basis, lx, ly, 0.25, 1.0)
    ntot = np.bitwise_count(np.arange(2 ** (lx * ly), dtype=np.uint64)).astype(float)
    h = h + np.diag(mu * (ntot - nn) ** 2)
    mpo = M.build_mpo(lx, ly, 0.25, 1.0, 1.0, basis, penalty=(mu, nn))
    psi = np.random.default_rng(1).standard_normal(2 ** (lx * ly)) + 0j
    assert np.max(np.abs(M.apply_mpo(mpo, psi) - h @ psi)) < 1e-12 * np.max(np.abs(h @ psi))


def test_mixed_mpo_config1_sector():
    """4 x 4 cylinder (16 orbitals): MPO and ED agree on random N = 4 states."""
    lx, ly, n = 4, 4, 4
    basis = model.fock_basis(16, n)
    h = model.mixed_space_hamiltonian(lx, ly, 0.25, 1.0, 1.0, n, basis=basis)
    mpo = M.build_mpo(lx, ly, 0.25, 1.0, 1.0, "mixed")
    rng = np.random.default_rng(2)
    c = rng.standard_normal(len(basis)) + 1j * rng.standard_normal(len(basis))
    psi = np.zeros(2 ** 16, dtype=np.complex128)
    psi[basis.astype(np.int64)] = c
    out = M.apply_mpo(mpo, psi)
    assert np.max(np.abs(out[basis.astype(np.int64)] - h @ c)) < 1e-12 * np.max(np.abs(h @ c))
    mask = np.ones(2 ** 16, dtype=bool)
    mask[basis.astype(np.int64)] = False
    assert np.max(np.abs(out[mask])) < 1e-13


@pytest.mark.parametrize("ly", [3, 4, 5, 6, 8])
def test_real_space_bond_dimension(ly):
    """Sec. IV.C: the real-space Hofstadter MPO has D = 3L + 2 in the bulk."""
    mpo = M.build_mpo(3, ly, 1 / ly, 1.0, 1.0, "real")
    d = mpo.dims()
    assert max(d) == 3 * ly + 2
    assert d[ly] == 3 * ly + 2 and d[2 * ly] == 3 * ly + 2


@pytest.mark.parametrize("ly", [3, 4, 6, 8, 10])
def test_mixed_bond_dimension_bound(ly):
    """Sec. IV.D: D <= 26 L + 9 for the momentum-labelled machine."""
    mpo = M.build_mpo(3, ly, 1 / ly, 1.0, 1.0, "mixed")
    assert max(mpo.dims()) <= 26 * ly + 9


@pytest.mark.parametrize("lx,ly", [(2, 4), (1, 6), (2, 6), (3, 8)])
def test_sine_cosine_machine_is_real(lx, ly):
    """Sec. IV.D, Eq. rot: rotating the e^{+i alpha}, e^{-i alpha} pairs into cosines and sines
    leaves every MPO entry real (the hops and the inter-ring terms are real in the mixed
    basis), keeps the charges (N, K) of every channel, and stays within the crude bound
    D <= 26 L + 9; its operator is the mixed Hamiltonian (test above)."""
    mpo = M.build_mpo(lx, ly, 1 / ly, 1.0, 1.0, "mixed_real")
    assert all(e[4].imag == 0.0 for ent in mpo.entries for e in ent)
    assert mpo.modulus == ly
    assert max(mpo.dims()) <= 26 * ly + 9


@pytest.mark.parametrize("basis", ["real", "mixed", "mixed_real"])
def test_channel_charges_conserved(basis):
    """Onsite symmetry (Sec. II): every nonzero W[w, w', s', s] has
    c_{w'} = c_w + q(s') - q(s), q(s) = (s, s m mod M)."""
    lx, ly = 3, 5
    mpo = M.build_mpo(lx, ly, 0.2, 1.0, 1.0, basis)
    mod = mpo.modulus
    for j, ent in enumerate(mpo.entries):
        m = mpo.site_m[j]
        for w, wp, sp, s, val in ent:
            c0, c1 = mpo.bond_charges[j][w], mpo.bond_charges[j + 1][wp]
            assert c1[0] == c0[0] + sp - s
            assert c1[1] % mod == (c0[1] + (sp - s) * m) % mod


def test_eq_m_example():
    """Sec. IV.B, Eq. M_example: the FSM for O = sum_i (A_i B_{i+1} + B_i A_{i+1}) gives, in
    the basis (R, A, B, F), M = [[1, A, B, 0], [0, 0, 0, B], [0, 0, 0, A], [0, 0, 0, 1]]."""
    a = np.array([[0.3, 1.2], [-0.7, 0.1]])
    b = np.array([[1.1, 0.0], [0.4, -2.0]])
    M.register_op("A_ex", a)
    M.register_op("B_ex", b)
    n = 6
    fams = [M.Family("AB", [M.Role("A_ex", 0), M.Role("B_ex", 1)], 0, lambda x: 1.0, list(range(n - 1))),
            M.Family("BA", [M.Role("B_ex", 0), M.Role("A_ex", 1)], 0, lambda x: 1.0, list(range(n - 1)))]
    mpo = M.build_fsm_mpo(n, 1, fams, lambda x, m: 0.0, 1)
    assert mpo.dims() == [1, 3, 4, 4, 4, 3, 1]   # F unreachable after site 0, R dead before site n-1
    w = mpo.dense_site(3)                      # bulk site, [w, w', s', s]
    zero, one = np.zeros((2, 2)), np.eye(2)
    expect = [[one, a, b, zero], [zero, zero, zero, b], [zero, zero, zero, a], [zero, zero, zero, one]]
    for r in range(4):
        for c in range(4):
            assert np.allclose(w[r, c], expect[r][c], atol=1e-15)


def _operator_schmidt_rank(mpo, b):
    """Rank of the Hamiltonian across bond b: the left block's operators per channel (sites
    0..b-1) and the right block's (sites b..n-1), both as vectors of operator entries; the
    rank of left x right^T is that of the product of their QR triangles."""
    L = np.ones((1, 1, 1), dtype=complex)
    for j in range(b):
        W = mpo.dense_site(j)                                   # [w, w', s', s]
        L = np.einsum("abw,wvps->apbsv", L, W).reshape(2 * L.shape[0], 2 * L.shape[1], W.shape[1])
    R = np.ones((1, 1, 1), dtype=complex)
    for j in range(mpo.n_sites - 1, b - 1, -1):
        W = mpo.dense_site(j)
        R = np.einsum("wvps,abv->pasbw", W, R).reshape(2 * R.shape[0], 2 * R.shape[1], W.shape[0])
    d = L.shape[2]
    rl = np.linalg.qr(L.reshape(-1, d))[1]
    rr = np.linalg.qr(R.reshape(-1, d))[1]
    sv = np.linalg.svd(rl @ rr.T, compute_uv=False)
    return d, int(np.sum(sv > 1e-10 * sv[0]))


@pytest.mark.parametrize("ly", [4, 5])
def test_bond_dimension_against_operator_schmidt_rank(ly):
    """The real-space machine is minimal (D = rank = 3L + 2, Sec. IV.C). The mixed machine is
    within one of the Hamiltonian's operator Schmidt rank in the middle of a ring, and that
    rank is above 3L + 2: the trimmed mixed D cannot fall below the real-space one there."""
    b = ly + ly // 2
    d, r = _operator_schmidt_rank(M.build_mpo(3, ly, 1 / ly, 1.0, 1.0, "real"), b)
    assert d == r == 3 * ly + 2
    d, r = _operator_schmidt_rank(M.build_mpo(3, ly, 1 / ly, 1.0, 1.0, "mixed"), b)
    assert r <= d <= r + 1
    assert r > 3 * ly + 2
