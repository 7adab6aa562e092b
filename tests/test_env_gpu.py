"""Environment updates of the library (a8) against the oracle, through the C ABI.

mrd_env_update rebuilds one environment of a DMRG state from its neighbour and the MPS tensor
between them; two-site updates run the same code after the block SVD. The oracle restates the
update block by block (oracle.blocksparse.env_left_update_block / env_right_update_block,
themselves pinned against the dense contraction of oracle.dmrg). Both sides read the same
tensors from the library: the input environment, the MPS tensor and the model MPO.

Cases: FP64 and float-float (MRD_PREC_FF) updates in both directions on the 4 x 4 cylinder;
the float-float environment left by one update of the headline reduced-precision form (split
BF16 Lanczos, float-float refinement, FP32 + float-float SVD) on the same cylinder; and sampled
blocks of that environment at Ly = 10, chi = 1024."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import synth  # noqa: E402
from oracle import blocksparse as B  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    import paper_1512_03318_gb300 as P
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return P.Context(0, torch.cuda.current_stream())


def sectors(d, b):
    return B.BondSectors([((int(n), int(k)), int(dim)) for n, k, dim in d.bond(b)])


def channels(mpo, b):
    return [(int(a), int(c) % mpo.modulus) for a, c in mpo.bond(b)]


def mpo_entries(mpo, j):
    idx, val = mpo.site(j)
    return [(int(w), int(wp), int(sp), int(s), complex(v)) for (w, wp, sp, s), v in zip(idx, val)]


def site_blocks(d, j, mod):
    """{(left index, s): d_l x d_r block} of MPS tensor j in the library's layouts: mode 0 groups
    by right sector (rows (s, l), s = 0 first), mode 1 by left sector (columns (s, r))."""
    mode, data = d.site(j)
    sl, sr = sectors(d, j), sectors(d, j + 1)
    m = j % mod
    out, off = {}, 0
    if mode == 0:
        for ri, qr in enumerate(sr.charges):
            rows = []
            for s in (0, 1):
                ql = B.qsub(qr, B.qsite(s, m, mod), mod)
                if ql in sl.index:
                    rows.append((s, sl.index[ql]))
            nrow = sum(sl.dims[li] for _, li in rows)
            blk = data[off:off + nrow * sr.dims[ri]].reshape(nrow, sr.dims[ri])
            off += nrow * sr.dims[ri]
            r0 = 0
            for s, li in rows:
                out[(li, s)] = blk[r0:r0 + sl.dims[li]]
                r0 += sl.dims[li]
    else:
        for li, ql in enumerate(sl.charges):
            cols = []
            for s in (0, 1):
                qr = B.qadd(ql, B.qsite(s, m, mod), mod)
                if qr in sr.index:
                    cols.append((s, sr.index[qr]))
            ncol = sum(sr.dims[ri] for _, ri in cols)
            blk = data[off:off + sl.dims[li] * ncol].reshape(sl.dims[li], ncol)
            off += sl.dims[li] * ncol
            c0 = 0
            for s, ri in cols:
                out[(li, s)] = blk[:, c0:c0 + sr.dims[ri]]
                c0 += sr.dims[ri]
    assert off == data.size
    return out


def oracle_left(d, mpo, j, lflat, sample=None):
    """Oracle L at bond j+1 from L at bond j (lflat) and MPS tensor j: list of (layout row, block)."""
    mod = mpo.modulus
    sl, sr = sectors(d, j), sectors(d, j + 1)
    cl, cm = channels(mpo, j), channels(mpo, j + 1)
    blocks = site_blocks(d, j, mod)
    W = mpo_entries(mpo, j)
    lay = B.env_left_layout(sr, cm, mod)
    rows = lay if sample is None else [lay[k] for k in sample]
    return [(r, B.env_left_update_block(sl, sr, j % mod, mod, cl, cm, W, lflat, blocks, (r[0], r[1]))) for r in rows]


def oracle_right(d, mpo, j, rflat, sample=None):
    """Oracle R at bond j from R at bond j+1 (rflat) and MPS tensor j."""
    mod = mpo.modulus
    sl, sr = sectors(d, j), sectors(d, j + 1)
    cl, cm = channels(mpo, j), channels(mpo, j + 1)
    blocks = site_blocks(d, j, mod)
    W = mpo_entries(mpo, j)
    lay = B.env_right_layout(sl, cl, mod)
    rows = lay if sample is None else [lay[k] for k in sample]
    return [(r, B.env_right_update_block(sl, sr, j % mod, mod, cl, cm, W, rflat, blocks, (r[0], r[1]))) for r in rows]


def compare(flat, pairs, tol):
    scale = max(np.max(np.abs(blk)) for _, blk in pairs)
    assert scale > 0
    err = 0.0
    for (w, xi, xpi, off, d0, d1), blk in pairs:
        got = flat[off:off + d0 * d1].reshape(d0, d1)
        err = max(err, float(np.max(np.abs(got - blk), initial=0.0)))
    assert err <= tol * scale, (err, scale)
    return err / scale


def cylinder(ctx, chi, center, seed=3):
    import paper_1512_03318_gb300 as P
    lx, ly, n = 4, 4, 4
    mpo = P.MPO(None, lx, ly, 1, 4, 1.0, 1.0, P.MRD_BASIS_MIXED)
    d = P.DMRG(ctx, mpo, n, 1, chi, seed=seed, center=center)
    return mpo, d


@pytest.mark.parametrize("prec,tol", [(0, 1e-12), (3, 1e-11)])
def test_env_update_both_directions(ctx, prec, tol):
    mpo, d = cylinder(ctx, 64, 6)
    # left: L at bond 5 from L at bond 4 and the left-canonical tensor 4
    l4 = d.env(4, 0)
    d.env_update(4, +1, prec)
    compare(d.env(5, 0), oracle_left(d, mpo, 4, l4), tol)
    # right: R at bond 9 from R at bond 10 and the right-canonical tensor 9
    r10 = d.env(10, 1)
    d.env_update(9, -1, prec)
    compare(d.env(9, 1), oracle_right(d, mpo, 9, r10), tol)
    d.close()


def test_env_update_rejects_bad_sites(ctx):
    import paper_1512_03318_gb300 as P
    mpo, d = cylinder(ctx, 32, 3)
    for site, direction in ((15, +1), (0, -1), (-1, +1), (16, -1)):
        with pytest.raises(P.MrdError) as ex:
            d.env_update(site, direction)
        assert ex.value.code == -1
    with pytest.raises(P.MrdError) as ex:     # R at bond 3 needs R at bond 4, which is not built
        d.env_update(3, -1)
    assert ex.value.code == -8
    with pytest.raises(P.MrdError):
        d.env_update(2, +1, 1)                 # TF32 is not an environment precision
    d.close()


def headline_params(P, chi):
    return P.DMRG.params(chi, 1e-14, 60, 1e-10, P.MRD_PREC_BF16X3, 1, 1e-13, restarts=8)


def test_headline_update_leaves_oracle_environment(ctx):
    """One two-site update of the headline form moving right: the float-float environment it
    leaves at bond i+1 equals the oracle's update of L at bond i with the new tensor i."""
    import paper_1512_03318_gb300 as P
    mpo, d = cylinder(ctx, 256, 7)
    l7 = d.env(7, 0)
    d.update(7, +1, headline_params(P, 256))
    compare(d.env(8, 0), oracle_left(d, mpo, 7, l7), 1e-11)
    # and moving left: R at bond 8 from R at bond 9 and the new right-canonical tensor 8
    r9 = d.env(9, 1)
    d.update(7, -1, headline_params(P, 256))
    compare(d.env(8, 1), oracle_right(d, mpo, 8, r9), 1e-11)
    d.close()


def test_headline_environment_at_production_block_sizes(ctx):
    """Ly = 10 cylinder (Lx = 12, flux 1/10, V = 1), chi = 1024 with the synthetic sector caps:
    after one headline update at the centre, sampled blocks of the new left environment (every
    channel of the largest sectors, block sizes of a few hundred) equal the oracle's."""
    import paper_1512_03318_gb300 as P
    lx, ly, chi = 12, 10, 1024
    n_sites = lx * ly
    caps = [[(q[0], q[1], dd) for q, dd in synth.bond_sectors(chi, ly, round(j / ly), synth.substream(99, 7, j))]
            if 2 <= j <= n_sites - 2 else [] for j in range(n_sites + 1)]
    mpo = P.MPO(None, lx, ly, 1, 10, 1.0, 1.0, P.MRD_BASIS_MIXED)
    i = (lx // 2) * ly + ly // 2 - 1
    d = P.DMRG(ctx, mpo, lx, 0, chi, seed=5, center=i, caps=caps)
    li = d.env(i, 0)
    d.update(i, +1, headline_params(P, chi))
    sr = sectors(d, i + 1)
    lay = B.env_left_layout(sr, channels(mpo, i + 1), ly)
    big = set(np.argsort(sr.dims)[-3:].tolist())
    sample = [k for k, r in enumerate(lay) if r[1] in big][:24]
    assert len(sample) >= 8
    compare(d.env(i + 1, 0), oracle_left(d, mpo, i, li, sample), 1e-11)
    d.close()


def test_fp32_environment_storage(ctx):
    """Environments stored in complex64 (MRD_DMRG_OPT_ENV_FP32): the stored values are the
    complex128 ones rounded (2^-24 relative), they take half the bytes, and an environment
    update in that storage equals the oracle's update of the stored input within the FP32
    rounding of its result."""
    import paper_1512_03318_gb300 as P
    mpo, d = cylinder(ctx, 64, 6)
    l4_64 = d.env(4, 0)
    bytes64, n_env, _, f = d.memory()
    assert f == 0
    d.set_option(P.MRD_DMRG_OPT_ENV_FP32, 1)
    bytes32, n_env2, _, f = d.memory()
    assert f == 1 and n_env2 == n_env
    assert bytes32 < 0.52 * bytes64 + 64
    l4 = d.env(4, 0)
    assert np.max(np.abs(l4 - l4_64)) <= 2.0 ** -24 * np.max(np.abs(l4_64))
    d.env_update(4, +1, P.MRD_PREC_FF)
    compare(d.env(5, 0), oracle_left(d, mpo, 4, l4), 3e-7)
    r10 = d.env(10, 1)
    d.env_update(9, -1, P.MRD_PREC_FP64)
    compare(d.env(9, 1), oracle_right(d, mpo, 9, r10), 3e-7)
    d.close()


def test_fp32_environment_sweeps_reach_ed(ctx):
    """Sweeps of the benchmarked reduced-precision form with complex64 environment storage on
    the 4 x 4 cylinder (flux 1/4, V = 1, N = 4, chi = 256): the energy reaches the ED ground
    energy of the sector within 1e-7 relative, the scale of the single-precision rounding of
    the environments that every later H_eff inherits."""
    import paper_1512_03318_gb300 as P
    from oracle import model
    lx, ly, n = 4, 4, 4
    e_ed = []
    for k in range(ly):
        basis = model.fock_basis(lx * ly, n)
        basis = np.array([s for s in basis if model.total_momentum(lx, ly, int(s)) == k], dtype=np.uint64)
        e_ed.append(float(np.linalg.eigvalsh(model.mixed_space_hamiltonian(lx, ly, 0.25, 1.0, 1.0, n, basis=basis))[0]))
    k0 = int(np.argmin(e_ed))
    mpo = P.MPO(None, lx, ly, 1, 4, 1.0, 1.0, P.MRD_BASIS_MIXED)
    d = P.DMRG(ctx, mpo, n, k0, 256, seed=7, center=0)
    d.set_option(P.MRD_DMRG_OPT_ENV_FP32, 1)
    p = headline_params(P, 256)
    es = []
    for _ in range(6):
        es.append(d.sweep(p))
        if len(es) > 1 and abs(es[-1] - es[-2]) < 1e-12 * abs(es[-1]):
            break
    assert d.memory()[3] == 1
    d.close()
    assert abs(es[-1] - e_ed[k0]) <= 1e-7 * abs(e_ed[k0]), (es, e_ed[k0])
