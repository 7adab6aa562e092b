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
