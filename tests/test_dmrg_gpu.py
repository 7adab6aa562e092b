"""End-to-end GPU two-site DMRG (C ABI) against exact diagonalisation by the oracle.

The library works in a fixed charge sector (N, K); the oracle diagonalises the mixed-basis
Hamiltonian restricted to the Fock states of that (N, K) (Sec. II: K is conserved), so the
two ground energies must agree to 1e-10 relative at a bond dimension that makes DMRG
exact, and the DMRG energy is an upper bound when the bond dimension truncates."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import model  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    import paper_1512_03318_gb300 as P
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return P.Context(0, torch.cuda.current_stream())


def ed_sector(lx, ly, flux, t, v, n, k=None):
    basis = model.fock_basis(lx * ly, n)
    if k is not None:
        basis = np.array([s for s in basis if model.total_momentum(lx, ly, int(s)) == k], dtype=np.uint64)
    h = model.mixed_space_hamiltonian(lx, ly, flux, t, v, n, basis=basis)
    return float(np.linalg.eigvalsh(h)[0])


def run_dmrg(ctx, lx, ly, fq, t, v, n, k, chi, basis=0, sweeps=8, seed=7):
    import paper_1512_03318_gb300 as P
    mpo = P.MPO(None, lx, ly, 1, fq, t, v, basis)
    d = P.DMRG(ctx, mpo, n, k, chi, seed=seed, center=0)
    p = P.DMRG.params(chi, 1e-14, 40, 1e-14)
    es = []
    for _ in range(sweeps):
        es.append(d.sweep(p))
        if len(es) > 1 and abs(es[-1] - es[-2]) < 1e-12 * abs(es[-1]):
            break
    return es, d


@pytest.mark.parametrize("lx,ly,fq,v,n", [(2, 4, 4, 1.0, 2), (2, 3, 3, 0.5, 2), (3, 4, 4, 1.0, 3)])
def test_dmrg_mixed_matches_ed_every_k(ctx, lx, ly, fq, v, n):
    e_ed = [ed_sector(lx, ly, 1 / fq, 1.0, v, n, k) for k in range(ly)]
    k0 = int(np.argmin(e_ed))
    es, d = run_dmrg(ctx, lx, ly, fq, 1.0, v, n, k0, 128)
    assert abs(es[-1] - e_ed[k0]) < 1e-10 * abs(e_ed[k0])
    # another momentum sector
    k1 = (k0 + 1) % ly
    es1, _ = run_dmrg(ctx, lx, ly, fq, 1.0, v, n, k1, 128)
    assert abs(es1[-1] - e_ed[k1]) < 1e-10 * abs(e_ed[k1])


def test_dmrg_real_basis_matches_ed(ctx):
    import paper_1512_03318_gb300 as P
    lx, ly, n = 2, 4, 3
    e = ed_sector(lx, ly, 0.25, 1.0, 1.0, n)
    es, _ = run_dmrg(ctx, lx, ly, 4, 1.0, 1.0, n, 0, 128, basis=P.MRD_BASIS_REAL)
    assert abs(es[-1] - e) < 1e-10 * abs(e)


def test_dmrg_config1_exact_bond_dimension(ctx):
    """4 x 4 cylinder, flux 1/4, t = V = 1, N = 4: chi = 256 exceeds the largest Schmidt rank
    (163), so DMRG reaches the ED ground energy of the sector."""
    lx, ly, n = 4, 4, 4
    e_ed = [ed_sector(lx, ly, 0.25, 1.0, 1.0, n, k) for k in range(ly)]
    k0 = int(np.argmin(e_ed))
    es, d = run_dmrg(ctx, lx, ly, 4, 1.0, 1.0, n, k0, 256, sweeps=6)
    assert abs(es[-1] - e_ed[k0]) < 1e-10 * abs(e_ed[k0])
    assert min(e_ed) == e_ed[k0]
    # the middle bond is not truncated: its total dimension is the exact Schmidt rank bound
    mid = d.bond(8)
    assert mid[:, 2].sum() <= 163


def test_dmrg_config1_truncated_is_variational(ctx):
    lx, ly, n = 4, 4, 4
    e_ed = [ed_sector(lx, ly, 0.25, 1.0, 1.0, n, k) for k in range(ly)]
    k0 = int(np.argmin(e_ed))
    es, d = run_dmrg(ctx, lx, ly, 4, 1.0, 1.0, n, k0, 24, sweeps=4)
    assert e_ed[k0] - 1e-10 < es[-1] < e_ed[k0] + 5e-2
    assert max(d.bond(b)[:, 2].sum() for b in range(1, 16)) <= 24


def test_dmrg_free_fermions_closed_form(ctx):
    """V = 0: the lowest energy over the K sectors is the sum of the N lowest levels."""
    lx, ly, n = 3, 3, 3
    e0 = model.free_fermion_ground_energy(lx, ly, 1 / 3, 1.0, n)
    best = min(run_dmrg(ctx, lx, ly, 3, 1.0, 0.0, n, k, 64)[0][-1] for k in range(ly))
    assert abs(best - e0) < 1e-10 * abs(e0)
