"""Seeded H_eff cases shared by the GPU parity tests and the bench (inputs only)."""
import numpy as np

import synth
from oracle import blocksparse as B


def sectors_array(bs):
    return np.array([[q[0], q[1], d] for q, d in zip(bs.charges, bs.dims)], dtype=np.int32)


def random_case(seed, ly, chi_l, chi_r, m1, m2, dl, dm, dr, density=0.7, n_mean=10):
    left = B.BondSectors(synth.bond_sectors(chi_l, ly, n_mean, synth.substream(seed, 1), min_dim=0))
    right = B.BondSectors(synth.bond_sectors(chi_r, ly, n_mean, synth.substream(seed, 2), min_dim=0))
    cl, cm, cr = synth.random_channel_charges(dl, dm, dr, m1, m2, ly, seed)
    wi = synth.random_mpo_site(cl, cm, ly, m1, synth.substream(seed, 6), density)
    wj = synth.random_mpo_site(cm, cr, ly, m2, synth.substream(seed, 7), density)
    return finish_case(seed, left, right, m1, m2, ly, cl, cm, cr, wi, wj)


def finish_case(seed, left, right, m1, m2, mod, cl, cm, cr, wi, wj):
    lay = B.theta_layout(left, right, m1, m2, mod)
    ll, rl = B.env_left_layout(left, cl, mod), B.env_right_layout(right, cr, mod)
    return dict(left=left, right=right, m1=m1, m2=m2, mod=mod, cl=cl, cm=cm, cr=cr, wi=wi, wj=wj, lay=lay,
                ll=ll, rl=rl,
                lflat=synth.complex_pm1(synth.substream(seed, 8), B.env_size(ll)),
                rflat=synth.complex_pm1(synth.substream(seed, 9), B.env_size(rl)),
                tflat=synth.complex_pm1(synth.substream(seed, 10), B.theta_size(lay)))


def mpo_case(seed, ly, chi, flux_q, site, mpo_sites, mpo_bonds, n_mean):
    """Production-shape case: synthetic bond sectors (sector recipe of synth) around sites
    (site, site+1) of a model MPO given as entry lists / bond charges."""
    left = B.BondSectors(synth.bond_sectors(chi, ly, n_mean, synth.substream(seed, 1)))
    right = B.BondSectors(synth.bond_sectors(chi, ly, n_mean, synth.substream(seed, 2)))
    m1, m2 = site % ly, (site + 1) % ly
    cl = [tuple(c) for c in mpo_bonds[site]]
    cm = [tuple(c) for c in mpo_bonds[site + 1]]
    cr = [tuple(c) for c in mpo_bonds[site + 2]]
    wi, wj = mpo_sites[site], mpo_sites[site + 1]
    return finish_case(seed, left, right, m1, m2, ly, cl, cm, cr, wi, wj)


def heff_args(case):
    wi_idx = np.array([e[:4] for e in case["wi"]], dtype=np.int32).reshape(-1, 4)
    wi_val = np.array([e[4] for e in case["wi"]], dtype=np.complex128)
    wj_idx = np.array([e[:4] for e in case["wj"]], dtype=np.int32).reshape(-1, 4)
    wj_val = np.array([e[4] for e in case["wj"]], dtype=np.complex128)
    return dict(left=sectors_array(case["left"]), right=sectors_array(case["right"]), m1=case["m1"], m2=case["m2"],
                modulus=case["mod"], cl=np.array(case["cl"], dtype=np.int32), cm=np.array(case["cm"], dtype=np.int32),
                cr=np.array(case["cr"], dtype=np.int32), wi_idx=wi_idx, wi_val=wi_val, wj_idx=wj_idx, wj_val=wj_val)


def oracle_mid_table(case):
    rows = []
    for m in case["lay"]:
        flags = 0
        r1 = c1 = -1
        for s1, ai, da, ro in m["rows"]:
            flags |= 1 << s1
            if s1 == 1:
                r1 = ro
        for s2, bi, db, co in m["cols"]:
            flags |= 4 << s2
            if s2 == 1:
                c1 = co
        rows.append([m["q"][0], m["q"][1], m["rowdim"], m["coldim"], m["offset"], r1, c1, flags])
    return np.array(rows, dtype=np.int64).reshape(-1, 8)
