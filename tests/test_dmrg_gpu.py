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


def run_dmrg(ctx, lx, ly, fq, t, v, n, k, chi, basis=0, sweeps=8, seed=7, svd_mode=None, params=None):
    import paper_1512_03318_gb300 as P
    mpo = P.MPO(None, lx, ly, 1, fq, t, v, basis)
    d = P.DMRG(ctx, mpo, n, k, chi, seed=seed, center=0)
    p = P.DMRG.params(chi, 1e-14, 40, 1e-14, svd_mode=svd_mode) if params is None else params
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


@pytest.mark.parametrize("svd_mode", [3, 1, 0, 2])
def test_dmrg_config1_exact_bond_dimension(ctx, svd_mode):
    """4 x 4 cylinder, flux 1/4, t = V = 1, N = 4: chi = 256 exceeds the largest Schmidt rank
    (163), so DMRG reaches the ED ground energy of the sector, whatever the arithmetic of the
    block SVD sweeps (FP64, float-float, FP32 followed by float-float or FP64)."""
    lx, ly, n = 4, 4, 4
    e_ed = [ed_sector(lx, ly, 0.25, 1.0, 1.0, n, k) for k in range(ly)]
    k0 = int(np.argmin(e_ed))
    es, d = run_dmrg(ctx, lx, ly, 4, 1.0, 1.0, n, k0, 256, sweeps=6, svd_mode=svd_mode)
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


def _isometry_error(site, left, right, m, ly):
    """max |A^+ A - I| over the right-sector blocks of a mode-0 MPS tensor (rows (s, l))."""
    dl = {(int(a), int(b)): int(c) for a, b, c in left}
    off, err = 0, 0.0
    for n_r, k_r, d_r in right:
        rows = sum(dl.get((int(n_r) - s, (int(k_r) - s * m) % ly), 0) for s in (0, 1))
        blk = site[off:off + rows * d_r].reshape(rows, d_r)
        off += rows * d_r
        err = max(err, float(np.abs(blk.conj().T @ blk - np.eye(d_r)).max()))
    assert off == site.size
    return err


@pytest.mark.parametrize("prec,svd_mode", [(0, 3), (2, 1), (2, 0), (2, 2)])
def test_update_canonical_factor_at_production_block_sizes(ctx, prec, svd_mode):
    """One two-site update at the centre of a 10 x 12 cylinder with chi = 1024 (sector blocks
    of a few hundred columns, several column groups of the block-cyclic Jacobi): the
    canonical factor is an isometry to 1e-12, the centre tensor has unit norm and the new bond
    keeps at most chi states."""
    import paper_1512_03318_gb300 as P
    import synth
    lx, ly, chi = 12, 10, 1024
    n_sites = lx * ly
    caps = [[(q[0], q[1], d) for q, d in synth.bond_sectors(chi, ly, round(j / ly), synth.substream(99, 7, j))]
            if 2 <= j <= n_sites - 2 else [] for j in range(n_sites + 1)]
    mpo = P.MPO(None, lx, ly, 1, 10, 1.0, 1.0, P.MRD_BASIS_MIXED)
    i = (lx // 2) * ly + ly // 2 - 1
    d = P.DMRG(ctx, mpo, lx, 0, chi, seed=5, center=i, caps=caps)
    p = P.DMRG.params(chi, 1e-14, 30, 1e-10, prec, 1, 1e-13, restarts=4, svd_mode=svd_mode)
    e, trunc = d.update(i, +1, p)
    assert math.isfinite(e)
    mode, a = d.site(i)
    assert mode == 0
    assert _isometry_error(a, d.bond(i), d.bond(i + 1), i % ly, ly) < 1e-12
    _, c = d.site(i + 1)
    assert abs(np.vdot(c, c).real - 1.0) < 1e-12
    assert d.bond(i + 1)[:, 2].sum() <= chi
    assert 0.0 <= trunc < 1e-2
    d.close()


def _schmidt_after_sweeps(ctx, lx, ly, fq, v, n, k, chi, bond, params=None):
    es, d = run_dmrg(ctx, lx, ly, fq, 1.0, v, n, k, chi, sweeps=8, params=params)
    import paper_1512_03318_gb300 as P
    p = P.DMRG.params(chi, 1e-14, 40, 1e-14) if params is None else params
    for i in range(bond):                   # centre back to the bond, moving right
        d.update(i, +1, p)
    b, spec = d.schmidt()
    d.close()
    assert b == bond
    return es[-1], spec


def _compare_spectra(got, ref, tol):
    keep = lambda sp: {key: val[val > 1e-4] for key, val in sp.items() if np.any(val > 1e-4)}
    got, ref = keep(got), keep(ref)
    assert set(got) == set(ref), (sorted(got), sorted(ref))
    for key in ref:
        assert len(got[key]) == len(ref[key]), key
        assert np.max(np.abs(got[key] - ref[key])) < tol, key


def test_entanglement_spectrum_matches_ed(ctx):
    """Momentum-resolved Schmidt values of the middle bond of the 4 x 4 cylinder (flux 1/4,
    V = 1, N = 4) at exact bond dimension equal those of the ED ground state, sector by
    sector (N, K of the left half)."""
    from oracle import entanglement as E
    lx, ly, n = 4, 4, 4
    e_ed = [ed_sector(lx, ly, 0.25, 1.0, 1.0, n, k) for k in range(ly)]
    k0 = int(np.argmin(e_ed))
    basis = model.fock_basis(lx * ly, n)
    basis = np.array([s for s in basis if model.total_momentum(lx, ly, int(s)) == k0], dtype=np.uint64)
    h = model.mixed_space_hamiltonian(lx, ly, 0.25, 1.0, 1.0, n, basis=basis)
    w, vec = np.linalg.eigh(h)
    ref = E.schmidt_spectrum(vec[:, 0], basis, 8, ly)
    e, got = _schmidt_after_sweeps(ctx, lx, ly, 4, 1.0, n, k0, 256, 8)
    assert abs(e - w[0]) < 1e-10 * abs(w[0])
    assert abs(sum(np.sum(v ** 2) for v in got.values()) - 1.0) < 1e-12
    _compare_spectra(got, ref, 1e-5)


def test_entanglement_spectrum_free_fermions(ctx):
    """V = 0 (3 x 3, flux 1/3, N = 3): the GPU Schmidt values equal the correlation-matrix
    closed form of the Slater determinant."""
    from oracle import entanglement as E
    lx, ly, n = 3, 3, 3
    e0 = model.free_fermion_ground_energy(lx, ly, 1 / 3, 1.0, n)
    ref = E.free_fermion_spectrum(lx, ly, 1 / 3, 1.0, n, 4)
    best = None
    for k in range(ly):
        try:
            e, got = _schmidt_after_sweeps(ctx, lx, ly, 3, 0.0, n, k, 64, 4)
        except Exception:   # sectors without states of this N
            continue
        if best is None or e < best[0]:
            best = (e, got)
    assert abs(best[0] - e0) < 1e-10 * abs(e0)
    _compare_spectra(best[1], ref, 1e-6)


# The reduced-precision forms of the update: Lanczos matvecs on the tensor cores (split BF16 or
# TF32 with FP32 accumulation), the ground vector refined with float-float or FP64 matvecs.
# (prec, refine_iter, refine_prec, svd_mode); the first row is the form the benchmark times
# (60 Lanczos steps per run, up to 8 restarts, one float-float Rayleigh quotient, FP32
# pre-sweeps then float-float Jacobi sweeps, float-float environments).
REDUCED_FORMS = {
    "bf16x3+ff (bench form)": (2, 1, 3, 0),
    "tf32+ff": (1, 20, 3, 0),
    "bf16x3+fp64": (2, 1, 0, 3),
    "tf32+fp64": (1, 20, 0, 2),
}


def reduced_params(P, chi, form):
    prec, refine_iter, refine_prec, svd_mode = REDUCED_FORMS[form]
    return P.DMRG.params(chi, 1e-14, 60, 1e-10, prec, refine_iter, 1e-13, restarts=8, svd_mode=svd_mode,
                         refine_prec=refine_prec)


@pytest.mark.parametrize("form", list(REDUCED_FORMS))
def test_reduced_precision_forms_match_ed(ctx, form):
    """The 1e-9 energy gate of the reduced-precision forms, against exact diagonalisation: on the
    4 x 4 cylinder (flux 1/4, t = V = 1, N = 4) at chi = 256 (no truncation), sweeps of each form
    reach the ED ground energy of the sector within 1e-9 relative."""
    import paper_1512_03318_gb300 as P
    lx, ly, n = 4, 4, 4
    e_ed = [ed_sector(lx, ly, 0.25, 1.0, 1.0, n, k) for k in range(ly)]
    k0 = int(np.argmin(e_ed))
    es, d = run_dmrg(ctx, lx, ly, 4, 1.0, 1.0, n, k0, 256, sweeps=6, params=reduced_params(P, 256, form))
    d.close()
    assert abs(es[-1] - e_ed[k0]) <= 1e-9 * abs(e_ed[k0]), (form, es, e_ed[k0])


def test_bench_form_entanglement_spectrum_matches_ed(ctx):
    """Schmidt values of the middle bond after sweeps of the benchmarked reduced-precision form
    equal those of the ED ground state, sector by sector (4 x 4, V = 1, exact chi)."""
    import paper_1512_03318_gb300 as P
    from oracle import entanglement as E
    lx, ly, n = 4, 4, 4
    e_ed = [ed_sector(lx, ly, 0.25, 1.0, 1.0, n, k) for k in range(ly)]
    k0 = int(np.argmin(e_ed))
    basis = model.fock_basis(lx * ly, n)
    basis = np.array([s for s in basis if model.total_momentum(lx, ly, int(s)) == k0], dtype=np.uint64)
    h = model.mixed_space_hamiltonian(lx, ly, 0.25, 1.0, 1.0, n, basis=basis)
    w, vec = np.linalg.eigh(h)
    ref = E.schmidt_spectrum(vec[:, 0], basis, 8, ly)
    e, got = _schmidt_after_sweeps(ctx, lx, ly, 4, 1.0, n, k0, 256, 8,
                                   params=reduced_params(P, 256, "bf16x3+ff (bench form)"))
    assert abs(e - w[0]) <= 1e-9 * abs(w[0])
    assert abs(sum(np.sum(v ** 2) for v in got.values()) - 1.0) < 1e-12
    _compare_spectra(got, ref, 1e-5)


def test_set_aside_columns_do_not_change_truncated_sweeps(ctx):
    """Truncating sweeps (4 x 4 cylinder, V = 1, chi = 24): the block SVD with FP32 pre-sweeps
    sets aside, before its final sweeps, the columns whose norm is below half the chi-th
    largest (their weight is truncated anyway); the float-float sweeps alone keep every
    column. Both reach the same energy (to 1e-9 relative) and keep at most chi states."""
    import paper_1512_03318_gb300 as P
    lx, ly, n = 4, 4, 4
    e_ed = [ed_sector(lx, ly, 0.25, 1.0, 1.0, n, k) for k in range(ly)]
    k0 = int(np.argmin(e_ed))
    out = {}
    for mode in (P.MRD_SVD_F32_FF, P.MRD_SVD_FF):
        p = P.DMRG.params(24, 1e-14, 40, 1e-14, P.MRD_PREC_FP64, svd_mode=mode, refine_prec=P.MRD_PREC_FF)
        es, d = run_dmrg(ctx, lx, ly, 4, 1.0, 1.0, n, k0, 24, sweeps=6, params=p)
        st = d.svd_stats()
        out[mode] = (es[-1], st[6], st[7])
        assert max(d.bond(b)[:, 2].sum() for b in range(1, 16)) <= 24
        d.close()
    e_a, kept_a, all_a = out[P.MRD_SVD_F32_FF]
    e_b, kept_b, all_b = out[P.MRD_SVD_FF]
    assert kept_b == all_b and kept_a <= all_a
    assert abs(e_a - e_b) <= 1e-9 * abs(e_b)
    assert e_ed[k0] - 1e-10 < e_a


def test_sine_cosine_machine_dmrg_matches_ed(ctx):
    """The real-valued sine / cosine MPO of Sec. IV.D (Eq. rot) drives the same DMRG to the ED
    ground energy of the sector: 4 x 4 cylinder, flux 1/4, V = 1, N = 4, exact chi (plain FP64
    form)."""
    import paper_1512_03318_gb300 as P
    lx, ly, n = 4, 4, 4
    e_ed = [ed_sector(lx, ly, 0.25, 1.0, 1.0, n, k) for k in range(ly)]
    k0 = int(np.argmin(e_ed))
    es, d = run_dmrg(ctx, lx, ly, 4, 1.0, 1.0, n, k0, 256, basis=P.MRD_BASIS_MIXED_REAL, sweeps=6)
    d.close()
    assert abs(es[-1] - e_ed[k0]) < 1e-10 * abs(e_ed[k0])


@pytest.mark.parametrize("form", ["bf16x3+ff (bench form)", "tf32+ff"])
def test_real_arithmetic_dmrg_matches_ed(ctx, form):
    """Real arithmetic end to end (Sec. IV.D, Eq. rot): the sine / cosine MPO, real tensors
    (MRD_DMRG_OPT_REAL) and real tensor-core matvecs; sweeps of the reduced-precision form reach
    the ED energy of the 4 x 4 cylinder (flux 1/4, V = 1, N = 4, chi = 256) within 1e-9, and
    every site tensor stays real."""
    import paper_1512_03318_gb300 as P
    lx, ly, n = 4, 4, 4
    e_ed = [ed_sector(lx, ly, 0.25, 1.0, 1.0, n, k) for k in range(ly)]
    k0 = int(np.argmin(e_ed))
    mpo = P.MPO(None, lx, ly, 1, 4, 1.0, 1.0, P.MRD_BASIS_MIXED_REAL)
    d = P.DMRG(ctx, mpo, n, k0, 256, seed=7, center=0)
    d.set_option(P.MRD_DMRG_OPT_REAL, 1)
    p = reduced_params(P, 256, form)
    es = []
    for _ in range(6):
        es.append(d.sweep(p))
        if len(es) > 1 and abs(es[-1] - es[-2]) < 1e-12 * abs(es[-1]):
            break
    for j in range(lx * ly):
        assert np.all(d.site(j)[1].imag == 0.0)
    d.close()
    dc = P.DMRG(ctx, P.MPO(None, lx, ly, 1, 4, 1.0, 1.0), n, k0, 64, seed=7)   # complex MPO: refused
    with pytest.raises(P.MrdError):
        dc.set_option(P.MRD_DMRG_OPT_REAL, 1)
    dc.close()
    dl = P.DMRG(ctx, mpo, n, k0, 64, seed=7, center=0)                        # after an update: refused
    dl.update(0, +1, p)
    with pytest.raises(P.MrdError):
        dl.set_option(P.MRD_DMRG_OPT_REAL, 1)
    dl.close()
    assert abs(es[-1] - e_ed[k0]) <= 1e-9 * abs(e_ed[k0]), (form, es, e_ed[k0])


@pytest.mark.parametrize("presweeps", [0, 3, 8])
def test_svd_presweeps_and_trace(ctx, presweeps):
    """The FP32 pre-sweep budget (MRD_DMRG_OPT_SVD_PRESWEEPS) changes only how the block SVD
    gets there: sweeps of the 4 x 4 cylinder (flux 1/4, V = 1, N = 4, chi = 256) with the
    benchmarked reduced-precision form reach the ED energy within 1e-9 for every budget. The
    per-sweep trace of the last SVD holds at most `presweeps` pre-sweeps and final sweeps whose
    last one rotated nothing (convergence), with a non-negative time per sweep."""
    import paper_1512_03318_gb300 as P
    lx, ly, n = 4, 4, 4
    e_ed = [ed_sector(lx, ly, 0.25, 1.0, 1.0, n, k) for k in range(ly)]
    k0 = int(np.argmin(e_ed))
    mpo = P.MPO(None, lx, ly, 1, 4, 1.0, 1.0)
    d = P.DMRG(ctx, mpo, n, k0, 256, seed=7, center=0)
    d.set_option(P.MRD_DMRG_OPT_SVD_PRESWEEPS, presweeps)
    p = reduced_params(P, 256, "bf16x3+ff (bench form)")
    es = []
    for _ in range(6):
        es.append(d.sweep(p))
        if len(es) > 1 and abs(es[-1] - es[-2]) < 1e-12 * abs(es[-1]):
            break
    t32, t64, m32, m64 = d.svd_trace(times=True)
    assert len(t32) <= presweeps and len(t64) >= 1 and t64[-1] == 0
    assert all(x >= 0 for x in t32 + t64) and all(x >= 0.0 for x in m32 + m64)
    with pytest.raises(P.MrdError):
        d.set_option(P.MRD_DMRG_OPT_SVD_PRESWEEPS, 65)
    d.close()
    assert abs(es[-1] - e_ed[k0]) <= 1e-9 * abs(e_ed[k0]), (presweeps, es, e_ed[k0])


def _orthonormal_vectors(site, mode, left, right, m, ly):
    """The singular vectors a site tensor holds after orthonormalisation: the columns of every
    right-sector block of a mode-0 tensor (rows (s, l)), the rows of every left-sector block of a
    mode-1 tensor (columns (s, r))."""
    dl = {(int(a), int(b)): int(c) for a, b, c in left}
    dr = {(int(a), int(b)): int(c) for a, b, c in right}
    off, out = 0, []
    if mode == 0:
        for n_r, k_r, d_r in right:
            rows = sum(dl.get((int(n_r) - s, (int(k_r) - s * m) % ly), 0) for s in (0, 1))
            blk = site[off:off + rows * d_r].reshape(rows, d_r)
            off += rows * d_r
            out += [blk[:, c] for c in range(d_r)]
    else:
        for n_l, k_l, d_l in left:
            cols = sum(dr.get((int(n_l) + s, (int(k_l) + s * m) % ly), 0) for s in (0, 1))
            blk = site[off:off + d_l * cols].reshape(d_l, cols)
            off += d_l * cols
            out += [blk[r, :] for r in range(d_l)]
    assert off == site.size
    return out


def test_random_state_phase_convention(ctx):
    """The seeded random MPS is orthonormalised tensor by tensor with the block SVD, whose
    singular vectors are fixed only up to a phase each; the state must not depend on the
    rotation order that picks it. Every singular vector of every tensor but the centre's has its
    entry of largest modulus real and positive (4 x 4 cylinder, chi = 64, centre 7), and the
    tensors are isometries."""
    import paper_1512_03318_gb300 as P
    lx, ly, n, centre = 4, 4, 4, 7
    mpo = P.MPO(None, lx, ly, 1, 4, 1.0, 1.0)
    d = P.DMRG(ctx, mpo, n, 0, 64, seed=7, center=centre)
    checked = 0
    for j in range(lx * ly):
        if j == centre:
            continue
        mode, data = d.site(j)
        for v in _orthonormal_vectors(data, mode, d.bond(j), d.bond(j + 1), j % ly, ly):
            if v.size == 0:
                continue
            x = v[int(np.argmax(v.real ** 2 + v.imag ** 2))]
            assert x.real > 0 and abs(x.imag) <= 1e-13 * abs(x), (j, x)
            assert abs(np.vdot(v, v) - 1.0) < 1e-12
            checked += 1
    d.close()
    assert checked > 100
