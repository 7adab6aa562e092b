"""Pins of oracle.blocksparse: charge tables by brute-force enumeration, block-sparse
H_eff against the dense contraction."""
import itertools

import numpy as np
import pytest

import synth
from oracle import blocksparse as B
from oracle import dmrg as D


@pytest.mark.parametrize("ly,nsites", [(4, 8), (3, 9), (5, 10), (6, 12)])
def test_fused_sectors_match_enumeration(ly, nsites):
    """Sector dims of a left block = histogram of (N, K) over all 2^n occupations."""
    ms = [j % ly for j in range(nsites)]
    hist = {}
    for bits in itertools.product((0, 1), repeat=nsites):
        q = (sum(bits), sum(b * m for b, m in zip(bits, ms)) % ly)
        hist[q] = hist.get(q, 0) + 1
    assert B.fused_bond_sectors(ms, ly) == sorted(hist.items())


def _random_case(seed, ly, chi_l, chi_r, m1, m2, dl, dm, dr, density=0.7):
    left = B.BondSectors(synth.bond_sectors(chi_l, ly, 10, synth.substream(seed, 1), min_dim=0))
    right = B.BondSectors(synth.bond_sectors(chi_r, ly, 10, synth.substream(seed, 2), min_dim=0))
    cl, cm, cr = synth.random_channel_charges(dl, dm, dr, m1, m2, ly, seed)
    wi = synth.random_mpo_site(cl, cm, ly, m1, synth.substream(seed, 6), density)
    wj = synth.random_mpo_site(cm, cr, ly, m2, synth.substream(seed, 7), density)
    lay = B.theta_layout(left, right, m1, m2, ly)
    ll, rl = B.env_left_layout(left, cl, ly), B.env_right_layout(right, cr, ly)
    lflat = synth.complex_pm1(synth.substream(seed, 8), B.env_size(ll))
    rflat = synth.complex_pm1(synth.substream(seed, 9), B.env_size(rl))
    tflat = synth.complex_pm1(synth.substream(seed, 10), B.theta_size(lay))
    return left, right, cl, cm, cr, wi, wj, lay, ll, rl, lflat, rflat, tflat


def _dense(left, right, m1, m2, mod, cl, cm, cr, wi, wj, lay, ll, rl, lflat, rflat, tflat):
    ol = np.concatenate([[0], np.cumsum(left.dims)]).astype(int)
    orr = np.concatenate([[0], np.cumsum(right.dims)]).astype(int)
    L = np.zeros((len(cl), ol[-1], ol[-1]), complex)
    for w, ai, api, off, dp, da in ll:
        L[w, ol[api]:ol[api] + dp, ol[ai]:ol[ai] + da] = lflat[off:off + dp * da].reshape(dp, da)
    R = np.zeros((len(cr), orr[-1], orr[-1]), complex)
    for w, bi, bpi, off, db, dp in rl:
        R[w, orr[bi]:orr[bi] + db, orr[bpi]:orr[bpi] + dp] = rflat[off:off + db * dp].reshape(db, dp)
    Wi = np.zeros((len(cl), len(cm), 2, 2), complex)
    for a, b, sp, s, v in wi:
        Wi[a, b, sp, s] += v
    Wj = np.zeros((len(cm), len(cr), 2, 2), complex)
    for a, b, sp, s, v in wj:
        Wj[a, b, sp, s] += v

    def to_dense(flat):
        T = np.zeros((ol[-1], 2, 2, orr[-1]), complex)
        for (ai, s1, s2), blk in B.theta_blocks(flat, lay).items():
            qb = B.qadd(B.qadd(left.charges[ai], B.qsite(s1, m1, mod), mod), B.qsite(s2, m2, mod), mod)
            bi = right.index[qb]
            T[ol[ai]:ol[ai] + blk.shape[0], s1, s2, orr[bi]:orr[bi] + blk.shape[1]] = blk
        return T
    return L, Wi, Wj, R, to_dense


@pytest.mark.parametrize("seed,ly,chi_l,chi_r,m1,m2,dl,dm,dr", [
    (1, 4, 40, 44, 1, 2, 5, 6, 7), (3, 5, 60, 50, 4, 0, 6, 5, 8), (5, 3, 36, 30, 2, 1, 9, 7, 4),
    (7, 6, 50, 70, 5, 3, 4, 8, 6)])
def test_blocksparse_heff_equals_dense(seed, ly, chi_l, chi_r, m1, m2, dl, dm, dr):
    case = _random_case(seed, ly, chi_l, chi_r, m1, m2, dl, dm, dr)
    left, right, cl, cm, cr, wi, wj, lay, ll, rl, lflat, rflat, tflat = case
    out = B.heff_apply(left, right, m1, m2, ly, cl, cm, cr, wi, wj, lflat, rflat, tflat)
    L, Wi, Wj, R, to_dense = _dense(left, right, m1, m2, ly, cl, cm, cr, wi, wj, lay, ll, rl, lflat, rflat, tflat)
    ref = D.heff_apply_dense(L, Wi, Wj, R, to_dense(tflat))
    got = to_dense(out)
    assert np.max(np.abs(ref)) > 0
    assert np.max(np.abs(got - ref)) < 1e-13 * np.max(np.abs(ref))
    # the dense result has no weight outside the allowed blocks
    assert abs(np.linalg.norm(ref) - np.linalg.norm(out)) < 1e-12 * np.linalg.norm(ref)


def test_theta_layout_enumerates_allowed_blocks():
    """Every (a, s1, s2, b) with q_a + q1(s1) + q2(s2) = q_b appears exactly once."""
    ly, m1, m2 = 5, 2, 4
    left = B.BondSectors(synth.bond_sectors(50, ly, 6, 11, min_dim=0))
    right = B.BondSectors(synth.bond_sectors(45, ly, 7, 12, min_dim=0))
    lay = B.theta_layout(left, right, m1, m2, ly)
    seen = set()
    for m in lay:
        for s1, ai, da, ro in m["rows"]:
            for s2, bi, db, co in m["cols"]:
                seen.add((ai, s1, s2, bi))
    brute = set()
    for ai, qa in enumerate(left.charges):
        for bi, qb in enumerate(right.charges):
            for s1 in (0, 1):
                for s2 in (0, 1):
                    if (qa[0] + s1 + s2, (qa[1] + s1 * m1 + s2 * m2) % ly) == qb:
                        brute.add((ai, s1, s2, bi))
    assert seen == brute
    assert B.theta_size(lay) == sum(left.dims[a] * right.dims[b] for a, _, _, b in brute)


def test_empty_overlap_gives_empty_theta():
    left = B.BondSectors([((0, 0), 3)])
    right = B.BondSectors([((5, 0), 2)])
    assert B.theta_layout(left, right, 0, 0, 1) == []


_CASES = [(1, 4, 40, 44, 1, 2, 5, 6, 7), (3, 5, 60, 50, 4, 0, 6, 5, 8), (5, 3, 36, 30, 2, 1, 9, 7, 4),
          (7, 6, 50, 70, 5, 3, 4, 8, 6)]


def _offsets(dims):
    return np.concatenate([[0], np.cumsum(dims)]).astype(int)


@pytest.mark.parametrize("seed,ly,chi_l,chi_r,m1,m2,dl,dm,dr", _CASES)
def test_heff_apply_block_equals_dense_block(seed, ly, chi_l, chi_r, m1, m2, dl, dm, dr):
    """heff_apply_block (the sampled reference of the production-size GPU checks) against the
    dense symmetry-free contraction, output block by output block: every allowed block
    (a', s1', s2') of the dense H_eff theta, sliced by the sector offsets, equals the single
    block the function computes."""
    case = _random_case(seed, ly, chi_l, chi_r, m1, m2, dl, dm, dr)
    left, right, cl, cm, cr, wi, wj, lay, ll, rl, lflat, rflat, tflat = case
    L, Wi, Wj, R, to_dense = _dense(left, right, m1, m2, ly, cl, cm, cr, wi, wj, lay, ll, rl, lflat, rflat, tflat)
    ref = D.heff_apply_dense(L, Wi, Wj, R, to_dense(tflat))
    ol, orr = _offsets(left.dims), _offsets(right.dims)
    scale = np.max(np.abs(ref))
    n_checked = 0
    for m in lay:
        for s1p, api, dap, _ in m["rows"]:
            for s2p, bpi, dbp, _ in m["cols"]:
                got = B.heff_apply_block(left, right, m1, m2, ly, cl, cm, cr, wi, wj, lflat, rflat, tflat,
                                         (api, s1p, s2p))
                want = ref[ol[api]:ol[api] + dap, s1p, s2p, orr[bpi]:orr[bpi] + dbp]
                assert got.shape == want.shape
                assert np.max(np.abs(got - want), initial=0.0) < 1e-13 * scale
                n_checked += 1
    assert n_checked >= 20


def _nonzero_blocks(arr, axes_offsets):
    """Index tuples of the sector blocks of a dense array that hold a nonzero entry. axes_offsets:
    per axis, the list of block boundaries (sector offsets, or [0, 1, ..] for plain indices)."""
    import itertools
    out = []
    ranges = [range(len(o) - 1) for o in axes_offsets]
    for idx in itertools.product(*ranges):
        sl = tuple(slice(o[i], o[i + 1]) for o, i in zip(axes_offsets, idx))
        if np.any(arr[sl] != 0):
            out.append(idx)
    return out


@pytest.mark.parametrize("seed,ly,chi_l,chi_r,m1,m2,dl,dm,dr", _CASES[:3])
def test_heff_flops_equals_count_from_dense_blocks(seed, ly, chi_l, chi_r, m1, m2, dl, dm, dr):
    """heff_flops (the flop count behind every H_eff TFLOP/s figure) against a count taken from
    the dense arrays alone: 8 real flops per complex multiply-add of every product of nonzero
    blocks in the definition order L -> W_i W_{i+1} -> R, the nonzero blocks being found in the
    dense L, theta, X = L theta, Y = W W X and R, sliced by the sector offsets (no layout
    function involved)."""
    case = _random_case(seed, ly, chi_l, chi_r, m1, m2, dl, dm, dr)
    left, right, cl, cm, cr, wi, wj, lay, ll, rl, lflat, rflat, tflat = case
    L, Wi, Wj, R, to_dense = _dense(left, right, m1, m2, ly, cl, cm, cr, wi, wj, lay, ll, rl, lflat, rflat, tflat)
    T = to_dense(tflat)
    ol, orr = _offsets(left.dims), _offsets(right.dims)
    dlf, drt = np.diff(ol), np.diff(orr)
    chan_l, chan_r, two = list(range(len(cl) + 1)), list(range(len(cr) + 1)), [0, 1, 2]
    # L step: X_w[a', s1, s2, b] += L_w[a', a] theta[a, s1, s2, b]
    lnz = _nonzero_blocks(L, [chan_l, ol, ol])
    tnz = set(_nonzero_blocks(T, [ol, two, two, orr]))
    fl = 0
    for w, ap, a in lnz:
        for s1 in (0, 1):
            for s2 in (0, 1):
                for b in range(len(right.dims)):
                    if (a, s1, s2, b) in tnz:
                        fl += 8 * dlf[ap] * dlf[a] * drt[b]
    # W step: one scaled block add per pair of MPO entries (W_i[w,w',s1',s1], W_{i+1}[w',w'',s2',s2])
    # and nonzero block X_w[a', s1, s2, b]
    X = np.einsum("wpa,asub->wpsub", L, T)
    xnz = _nonzero_blocks(X, [chan_l, ol, two, two, orr])
    xby = {}
    for w, ap, s1, s2, b in xnz:
        xby.setdefault((w, s1, s2), []).append((ap, b))
    for (w, wp, s1p, s1, _) in wi:
        for (wq, wpp, s2p, s2, _) in wj:
            if wq != wp:
                continue
            for ap, b in xby.get((w, s1, s2), []):
                fl += 8 * dlf[ap] * drt[b]
    # R step: theta'[a', s1', s2', b'] += Y_{w''}[a', s1', s2', b] R_{w''}[b, b']
    Y = np.einsum("zptrb->zptrb", np.einsum("vzru,vptub->zptrb", Wj, np.einsum("wvts,wpsub->vptub", Wi, X)))
    ynz = _nonzero_blocks(Y, [chan_r, ol, two, two, orr])
    rnz = _nonzero_blocks(R, [chan_r, orr, orr])
    rby = {}
    for w, b, bp in rnz:
        rby.setdefault((w, b), []).append(bp)
    for w, ap, s1p, s2p, b in ynz:
        for bp in rby.get((w, b), []):
            fl += 8 * dlf[ap] * drt[b] * drt[bp]
    assert B.heff_flops(left, right, m1, m2, ly, cl, cm, cr, wi, wj) == fl


def _random_site(sec_l, sec_r, m, mod, seed):
    """Dense random MPS tensor A[a, s, c] that is nonzero only on charge-allowed blocks
    q_a + q(s) = q_c (entries complex U[-1, 1))."""
    ol, orr = _offsets(sec_l.dims), _offsets(sec_r.dims)
    A = np.zeros((ol[-1], 2, orr[-1]), complex)
    k = 0
    for ai, qa in enumerate(sec_l.charges):
        for s in (0, 1):
            qc = B.qadd(qa, B.qsite(s, m, mod), mod)
            if qc in sec_r.index:
                ci = sec_r.index[qc]
                blk = synth.complex_pm1(synth.substream(seed, k), sec_l.dims[ai] * sec_r.dims[ci])
                A[ol[ai]:ol[ai + 1], s, orr[ci]:orr[ci + 1]] = blk.reshape(sec_l.dims[ai], sec_r.dims[ci])
                k += 1
    return A


def _env_dense(sec, layout, nchan, flat, left):
    """Dense environment [w, bra, ket] (left) or [w, ket, bra] (right) from a flat one in its layout."""
    o = _offsets(sec.dims)
    env = np.zeros((nchan, o[-1], o[-1]), complex)
    for w, xi, xpi, off, d0, d1 in layout:
        blk = flat[off:off + d0 * d1].reshape(d0, d1)
        if left:
            env[w, o[xpi]:o[xpi] + d0, o[xi]:o[xi] + d1] = blk
        else:
            env[w, o[xi]:o[xi] + d0, o[xpi]:o[xpi] + d1] = blk
    return env


def _layout_mask(sec, layout, nchan, left):
    o = _offsets(sec.dims)
    mask = np.zeros((nchan, o[-1], o[-1]), bool)
    for w, xi, xpi, off, d0, d1 in layout:
        if left:   # L_w block [bra a' = xpi][ket a = xi]
            mask[w, o[xpi]:o[xpi] + d0, o[xi]:o[xi] + d1] = True
        else:      # R_w block [ket b = xi][bra b' = xpi]
            mask[w, o[xi]:o[xi] + d0, o[xpi]:o[xpi] + d1] = True
    return mask


@pytest.mark.parametrize("seed,ly,m,dl,dr", [(2, 4, 1, 5, 7), (4, 5, 3, 6, 4), (6, 3, 2, 8, 5)])
def test_env_contraction_stays_in_layout(seed, ly, m, dl, dr):
    """An environment contracted (dense, oracle.dmrg) from a charge-conserving environment, a
    random charge-allowed MPS tensor and a random charge-conserving MPO site has no weight
    outside the blocks env_left_layout / env_right_layout list for the new bond (a block the
    layouts left out would be dropped by every block-sparse environment, on both sides of a
    comparison that reads them through these layouts)."""
    sec0 = B.BondSectors(synth.bond_sectors(40, ly, 10, synth.substream(seed, 1), min_dim=0))
    # the sectors reachable from sec0 through one orbital of momentum m, random dims
    cand = sorted({B.qadd(q, B.qsite(s, m, ly), ly) for q in sec0.charges for s in (0, 1)})
    u = synth.uniform01(synth.substream(seed, 2), len(cand))
    sec1 = B.BondSectors([(q, 1 + int(5 * x)) for q, x in zip(cand, u)])
    cl, cm, _ = synth.random_channel_charges(dl, dr, 1, m, m, ly, seed)
    W = synth.random_mpo_site(cl, cm, ly, m, synth.substream(seed, 3), 0.8)
    Wd = np.zeros((len(cl), len(cm), 2, 2), complex)
    for a, b, sp, s, v in W:
        Wd[a, b, sp, s] += v
    A = _random_site(sec0, sec1, m, ly, synth.substream(seed, 4))
    # left: L at bond 0 (channels cl) -> L' at bond 1 (channels cm)
    lay0 = B.env_left_layout(sec0, cl, ly)
    L0 = np.zeros((len(cl), A.shape[0], A.shape[0]), complex)
    L0[_layout_mask(sec0, lay0, len(cl), True)] = synth.complex_pm1(synth.substream(seed, 5), B.env_size(lay0))
    L1 = D.env_left_update(L0, A, Wd)
    mask = _layout_mask(sec1, B.env_left_layout(sec1, cm, ly), len(cm), True)
    assert np.max(np.abs(L1)) > 0
    assert np.max(np.abs(L1[~mask]), initial=0.0) == 0.0
    # right: R at bond 1 (channels cm) -> R' at bond 0 (channels cl)
    lay1 = B.env_right_layout(sec1, cm, ly)
    R1 = np.zeros((len(cm), A.shape[2], A.shape[2]), complex)
    R1[_layout_mask(sec1, lay1, len(cm), False)] = synth.complex_pm1(synth.substream(seed, 6), B.env_size(lay1))
    R0 = D.env_right_update(R1, A, Wd)
    mask = _layout_mask(sec0, B.env_right_layout(sec0, cl, ly), len(cl), False)
    assert np.max(np.abs(R0)) > 0
    assert np.max(np.abs(R0[~mask]), initial=0.0) == 0.0


@pytest.mark.parametrize("seed,ly,m,dl,dr", [(2, 4, 1, 5, 7), (4, 5, 3, 6, 4), (6, 3, 2, 8, 5)])
def test_env_update_blocks_equal_dense(seed, ly, m, dl, dr):
    """env_left_update_block / env_right_update_block (the block-by-block environment updates
    that sample the production-size GPU environments) against the dense symmetry-free
    contractions of oracle.dmrg, block by block over the whole layout of the new bond."""
    sec0 = B.BondSectors(synth.bond_sectors(40, ly, 10, synth.substream(seed, 1), min_dim=0))
    cand = sorted({B.qadd(q, B.qsite(s, m, ly), ly) for q in sec0.charges for s in (0, 1)})
    u = synth.uniform01(synth.substream(seed, 2), len(cand))
    sec1 = B.BondSectors([(q, 1 + int(5 * x)) for q, x in zip(cand, u)])
    cl, cm, _ = synth.random_channel_charges(dl, dr, 1, m, m, ly, seed)
    W = synth.random_mpo_site(cl, cm, ly, m, synth.substream(seed, 3), 0.8)
    Wd = np.zeros((len(cl), len(cm), 2, 2), complex)
    for a, b, sp, s, v in W:
        Wd[a, b, sp, s] += v
    A = _random_site(sec0, sec1, m, ly, synth.substream(seed, 4))
    o0, o1 = _offsets(sec0.dims), _offsets(sec1.dims)
    blocks = {}
    for ai, qa in enumerate(sec0.charges):
        for s in (0, 1):
            qc = B.qadd(qa, B.qsite(s, m, ly), ly)
            if qc in sec1.index:
                ci = sec1.index[qc]
                blocks[(ai, s)] = A[o0[ai]:o0[ai + 1], s, o1[ci]:o1[ci + 1]]
    # left
    lay0 = B.env_left_layout(sec0, cl, ly)
    lflat = synth.complex_pm1(synth.substream(seed, 5), B.env_size(lay0))
    L0 = _env_dense(sec0, lay0, len(cl), lflat, True)
    L1 = D.env_left_update(L0, A, Wd)
    scale = np.max(np.abs(L1))
    for w, ci, cpi, off, d0, d1 in B.env_left_layout(sec1, cm, ly):
        got = B.env_left_update_block(sec0, sec1, m, ly, cl, cm, W, lflat, blocks, (w, ci))
        want = L1[w, o1[cpi]:o1[cpi] + d0, o1[ci]:o1[ci] + d1]
        assert np.max(np.abs(got - want), initial=0.0) < 1e-13 * scale
    # right
    lay1 = B.env_right_layout(sec1, cm, ly)
    rflat = synth.complex_pm1(synth.substream(seed, 6), B.env_size(lay1))
    R1 = _env_dense(sec1, lay1, len(cm), rflat, False)
    R0 = D.env_right_update(R1, A, Wd)
    bblocks = {(ai, s): blk for (ai, s), blk in blocks.items()}
    scale = np.max(np.abs(R0))
    for w, ci, cpi, off, d0, d1 in B.env_right_layout(sec0, cl, ly):
        got = B.env_right_update_block(sec0, sec1, m, ly, cl, cm, W, rflat, bblocks, (w, ci))
        want = R0[w, o0[ci]:o0[ci] + d0, o0[cpi]:o0[cpi] + d1]
        assert np.max(np.abs(got - want), initial=0.0) < 1e-13 * scale


def test_two_site_update_matches_dense_restatement():
    """oracle.blocksparse.two_site_update against the dense symmetry-free steps of
    oracle.dmrg on the same operands: the Lanczos energy equals <g|H_eff|g> of the returned
    ground vector in the dense contraction; the kept Schmidt values are the chi largest
    singular values of the dense theta matrix (rows (a, s1), columns (s2, b)) renormalised;
    the projector A A^+ equals that of the dense SVD truncated to chi (phase-free); and the new
    left environment equals the dense env_left_update of the densified A."""
    seed, ly, chi_l, chi_r, m1, m2, dl, dm, dr = 3, 5, 60, 50, 4, 0, 6, 5, 8
    case = _random_case(seed, ly, chi_l, chi_r, m1, m2, dl, dm, dr)
    left, right, cl, cm, cr, wi, wj, lay, ll, rl, lflat, rflat, tflat = case
    L, Wi, Wj, R, to_dense = _dense(left, right, m1, m2, ly, cl, cm, cr, wi, wj, lay, ll, rl, lflat, rflat, tflat)
    # Hermitian operator: H_eff + H_eff^+ as a dense matrix, applied through the block code as
    # (H + H^+) v = H v + (H^+ v); the symmetrisation keeps the Lanczos recurrence meaningful
    n = B.theta_size(lay)
    hmat = np.stack([B.heff_apply(left, right, m1, m2, ly, cl, cm, cr, wi, wj, lflat, rflat, e)
                     for e in np.eye(n, dtype=complex)], axis=1)
    herm = hmat + hmat.conj().T

    def lanczos(mv, v0):
        return D.lanczos_ground(lambda v: herm @ v, v0, kmax=30, tol=1e-13)
    chi = 40
    out = B.two_site_update(left, right, m1, m2, ly, cl, cm, cr, wi, wj, lflat, rflat, tflat, chi, lanczos=lanczos)
    w = np.linalg.eigvalsh(herm)
    e_ref, g, _ = lanczos(None, tflat)
    # the energy is the Ritz value of the returned vector, variational
    assert abs(out["energy"] - np.vdot(g, herm @ g).real) < 1e-10 * abs(w[0])
    assert out["energy"] >= w[0] - 1e-10 * abs(w[0])
    # dense theta matrix of the ground vector: rows (a, s1), columns (s2, b)
    ol, orr = _offsets(left.dims), _offsets(right.dims)
    T = to_dense(g)                                   # [a, s1, s2, b]
    tm = T.reshape(ol[-1] * 2, 2 * orr[-1])
    u, s, vh = np.linalg.svd(tm, full_matrices=False)
    kept = s[:chi] / np.linalg.norm(s[:chi])
    got = np.sort(np.concatenate(list(out["schmidt"].values())))[::-1]
    assert len(got) == chi
    assert np.max(np.abs(got - kept)) < 1e-12
    assert abs(out["discarded"] - (1 - np.sum(s[:chi] ** 2) / np.sum(s ** 2))) < 1e-12
    # densified A[a, s1, c] on the new bond
    bond = out["bond"]
    ob = _offsets(bond.dims)
    A = np.zeros((ol[-1], 2, ob[-1]), complex)
    for (ai, s1), blk in out["a_blocks"].items():
        qc = B.qadd(left.charges[ai], B.qsite(s1, m1, ly), ly)
        ci = bond.index[qc]
        A[ol[ai]:ol[ai + 1], s1, ob[ci]:ob[ci + 1]] = blk
    am = A.reshape(ol[-1] * 2, ob[-1])
    # the truncated projector is as well defined as the gap at the cut allows
    tol_p = 1e-12 + 1e-14 * s[0] / (s[chi - 1] - s[chi])
    assert np.max(np.abs(am @ am.conj().T - u[:, :chi] @ u[:, :chi].conj().T)) < tol_p
    lnew = D.env_left_update(L, A, Wi)
    lay_new = B.env_left_layout(bond, cm, ly)
    want = np.zeros(B.env_size(lay_new), complex)
    for wq, ci, cpi, off, d0, d1 in lay_new:
        want[off:off + d0 * d1] = lnew[wq, ob[cpi]:ob[cpi] + d0, ob[ci]:ob[ci] + d1].reshape(-1)
    assert np.max(np.abs(out["lenv"] - want)) < 1e-12 * np.max(np.abs(want))
