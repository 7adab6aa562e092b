"""Charge bookkeeping and the block-sparse two-site H_eff, restated with plain loops over
charge blocks. Test infrastructure only.

Charges (Sec. II and Sec. III): particle number N (U(1)) and ring momentum K in Z_M, with
M = Ly in the mixed basis (the onsite rotation T_y = prod exp(i k n_{x,k}) makes K an
additive onsite charge) and M = 1 in real space. Local charge of orbital momentum m:
q(s) = (s, s * m mod M) for occupation s.

Tensors are lists of dense blocks, one per allowed charge combination:
  bond sectors      ((N, K), dim), sorted by (N, K)
  theta             fused "middle" blocks: for each middle charge q_m (sorted), rows
                    (s1, a) with q_a + q1(s1) = q_m (s1 = 0 rows first), columns (s2, b) with
                    q_b - q2(s2) = q_m (s2 = 0 first); block row-major; blocks concatenated
  left env  L_w     block (w, a) for every channel w and left sector a whose image
                    q_a + c_w is a left sector; shape d(q_a + c_w) x d(q_a) = [bra][ket];
                    ordered by w, then a; row-major; concatenated
  right env R_w     block (w, b) for every channel w and right sector b with q_b + c_w a
                    right sector; shape d(q_b) x d(q_b + c_w) = [ket][bra]; ordered by w, b
  MPO site          entries (w, w', s', s, value), nonzero only if
                    c_{w'} = c_w + q(s') - q(s)
Complex numbers are stored interleaved (re, im) as complex128.

H_eff (the two-site effective Hamiltonian of DMRG, applied as in the definition):
  X_w[a', s1, s2, b]      = sum_a L_w[a', a] theta[a, s1, s2, b]
  Y_{w''}[a', s1', s2', b] = sum W_i[w, w', s1', s1] W_{i+1}[w', w'', s2', s2] X_w[a', s1, s2, b]
  theta'[a', s1', s2', b'] = sum_{w'', b} Y_{w''}[a', s1', s2', b] R_{w''}[b, b']
"""
from __future__ import annotations

import numpy as np


def qadd(q1, q2, mod):
    return (q1[0] + q2[0], (q1[1] + q2[1]) % mod)


def qsub(q1, q2, mod):
    return (q1[0] - q2[0], (q1[1] - q2[1]) % mod)


def qsite(s, m, mod):
    return (s, (s * m) % mod)


class BondSectors:
    def __init__(self, sectors):
        self.charges = [tuple(q) for q, _ in sectors]
        self.dims = [int(d) for _, d in sectors]
        if self.charges != sorted(self.charges) or len(set(self.charges)) != len(self.charges):
            raise ValueError("bond sectors must be sorted and distinct")
        self.index = {q: i for i, q in enumerate(self.charges)}

    def dim(self, q):
        i = self.index.get(q)
        return 0 if i is None else self.dims[i]


def theta_layout(left, right, m1, m2, mod):
    """Middle sectors of the fused two-site tensor.

    Returns a list of dicts, sorted by middle charge q, each with
    rows: [(s1, a_index, d_a, row_offset)], cols: [(s2, b_index, d_b, col_offset)],
    rowdim, coldim, offset (position of the block in the flat array)."""
    cand = set()
    for q in left.charges:
        for s1 in (0, 1):
            cand.add(qadd(q, qsite(s1, m1, mod), mod))
    out = []
    off = 0
    for q in sorted(cand):
        rows, r = [], 0
        for s1 in (0, 1):
            a = qsub(q, qsite(s1, m1, mod), mod)
            if a in left.index:
                rows.append((s1, left.index[a], left.dim(a), r))
                r += left.dim(a)
        cols, c = [], 0
        for s2 in (0, 1):
            b = qadd(q, qsite(s2, m2, mod), mod)
            if b in right.index:
                cols.append((s2, right.index[b], right.dim(b), c))
                c += right.dim(b)
        if r == 0 or c == 0:
            continue
        out.append({"q": q, "rows": rows, "cols": cols, "rowdim": r, "coldim": c, "offset": off})
        off += r * c
    return out


def theta_size(layout):
    return sum(m["rowdim"] * m["coldim"] for m in layout)


def env_left_layout(left, cw, mod):
    """[(w, a_index, a'_index, offset, d_a', d_a)] for the blocks of L_w."""
    out, off = [], 0
    for w, c in enumerate(cw):
        for ai, qa in enumerate(left.charges):
            qp = qadd(qa, c, mod)
            if qp in left.index:
                dp, da = left.dim(qp), left.dims[ai]
                out.append((w, ai, left.index[qp], off, dp, da))
                off += dp * da
    return out


def env_right_layout(right, cw, mod):
    """[(w, b_index, b'_index, offset, d_b, d_b')] for the blocks of R_w."""
    out, off = [], 0
    for w, c in enumerate(cw):
        for bi, qb in enumerate(right.charges):
            qp = qadd(qb, c, mod)
            if qp in right.index:
                db, dp = right.dims[bi], right.dim(qp)
                out.append((w, bi, right.index[qp], off, db, dp))
                off += db * dp
    return out


def env_size(layout):
    return sum(e[4] * e[5] for e in layout)


def theta_blocks(flat, layout):
    """Flat fused theta -> {(a_index, s1, s2): d_a x d_b array}."""
    out = {}
    for m in layout:
        blk = flat[m["offset"]: m["offset"] + m["rowdim"] * m["coldim"]].reshape(m["rowdim"], m["coldim"])
        for s1, ai, da, ro in m["rows"]:
            for s2, bi, db, co in m["cols"]:
                out[(ai, s1, s2)] = blk[ro:ro + da, co:co + db]
    return out


def theta_flat(blocks, layout):
    flat = np.zeros(theta_size(layout), dtype=np.complex128)
    for m in layout:
        blk = flat[m["offset"]: m["offset"] + m["rowdim"] * m["coldim"]].reshape(m["rowdim"], m["coldim"])
        for s1, ai, da, ro in m["rows"]:
            for s2, bi, db, co in m["cols"]:
                if (ai, s1, s2) in blocks:
                    blk[ro:ro + da, co:co + db] = blocks[(ai, s1, s2)]
    return flat


def heff_apply(left, right, m1, m2, mod, cl, cm, cr, wi, wj, lflat, rflat, tflat, rows=None):
    """theta' = H_eff theta, block by block, in the order of the definition above.

    left/right: BondSectors of the bonds left of site i and right of site i+1; m1, m2:
    momenta of the two sites; cl, cm, cr: channel charges of the MPO bonds left of i,
    between i and i+1, right of i+1; wi, wj: MPO entry lists; lflat, rflat, tflat: flat
    complex128 arrays in the layouts above. rows: optional set of left-sector indices a';
    if given, only output blocks with those a' are computed (others stay zero), which is
    the same arithmetic on a subset (used to bound the CPU timing sample)."""
    lay = theta_layout(left, right, m1, m2, mod)
    theta = theta_blocks(tflat, lay)
    lblk = {(w, ai): lflat[off: off + dp * da].reshape(dp, da)
            for w, ai, api, off, dp, da in env_left_layout(left, cl, mod)}
    rblk = {(w, bi): rflat[off: off + db * dp].reshape(db, dp)
            for w, bi, bpi, off, db, dp in env_right_layout(right, cr, mod)}
    # X_w = L_w theta
    x = {}
    for (ai, s1, s2), blk in theta.items():
        qa = left.charges[ai]
        for w, c in enumerate(cl):
            key = (w, ai)
            if key not in lblk:
                continue
            api = left.index[qadd(qa, c, mod)]
            if rows is not None and api not in rows:
                continue
            x[(w, api, s1, s2, ai)] = lblk[key] @ blk
    # Y_{w''} = sum W_i W_{i+1} X_w
    wj_by_mid = {}
    for (wp, wpp, s2p, s2, val) in wj:
        wj_by_mid.setdefault(wp, []).append((wpp, s2p, s2, val))
    x_by = {}
    for (w, api, s1, s2, ai), xb in x.items():
        x_by.setdefault((w, s1), []).append((api, s2, ai, xb))
    y = {}
    for (w, wp, s1p, s1, vi) in wi:
        for (wpp, s2p, s2, vj) in wj_by_mid.get(wp, []):
            for (api, xs2, ai, xb) in x_by.get((w, s1), []):
                if xs2 != s2:
                    continue
                qb = qadd(qadd(left.charges[ai], qsite(s1, m1, mod), mod), qsite(s2, m2, mod), mod)
                bi = right.index[qb]
                k = (wpp, api, s1p, s2p, bi)
                y[k] = y.get(k, 0) + (vi * vj) * xb
    # theta' = sum Y_{w''} R_{w''}
    out = {}
    for (wpp, api, s1p, s2p, bi), yb in y.items():
        key = (wpp, bi)
        if key not in rblk:
            continue
        qbp = qadd(right.charges[bi], cr[wpp], mod)
        expect = qadd(qadd(left.charges[api], qsite(s1p, m1, mod), mod), qsite(s2p, m2, mod), mod)
        if qbp != expect:
            raise AssertionError("charge conservation violated")
        k = (api, s1p, s2p)
        out[k] = out.get(k, 0) + yb @ rblk[key]
    return theta_flat(out, lay)


def heff_flops(left, right, m1, m2, mod, cl, cm, cr, wi, wj, rows=None):
    """Real flops of heff_apply in the order of the definition: 8 per complex
    multiply-add in the L step, the W step (one scaled block add per matching pair of
    MPO entries) and the R step. This count depends only on the workload (and on the
    optional row subset, as in heff_apply)."""
    lay = theta_layout(left, right, m1, m2, mod)
    blocks = []
    for m in lay:
        for s1, ai, da, ro in m["rows"]:
            for s2, bi, db, co in m["cols"]:
                blocks.append((ai, s1, s2, da, db, bi))
    fl = 0
    xkeys = {}
    for ai, s1, s2, da, db, bi in blocks:
        for w, c in enumerate(cl):
            q = qadd(left.charges[ai], c, mod)
            if q in left.index:
                if rows is not None and left.index[q] not in rows:
                    continue
                dp = left.dim(q)
                fl += 8 * dp * da * db
                xkeys.setdefault((w, s1, s2), []).append((left.index[q], bi, dp, db))
    wj_by_mid = {}
    for (wp, wpp, s2p, s2, val) in wj:
        wj_by_mid.setdefault(wp, []).append((wpp, s2p, s2))
    ykeys = set()
    for (w, wp, s1p, s1, vi) in wi:
        for (wpp, s2p, s2) in wj_by_mid.get(wp, []):
            for api, bi, dp, db in xkeys.get((w, s1, s2), []):
                fl += 8 * dp * db
                ykeys.add((wpp, api, s1p, s2p, bi, dp, db))
    for wpp, api, s1p, s2p, bi, dp, db in ykeys:
        q = qadd(right.charges[bi], cr[wpp], mod)
        if q in right.index:
            fl += 8 * dp * db * right.dim(q)
    return fl


def random_env_from_layout(layout_size, seed):
    import synth
    return synth.complex_pm1(seed, layout_size)


def fused_bond_sectors(site_ms, mod):
    """Exact sectors of the left block spanned by orbitals with momenta site_ms: fusing one
    orbital with local charges q(0) = (0, 0), q(1) = (1, m) at a time (dims add up)."""
    sec = {(0, 0): 1}
    for m in site_ms:
        nxt = {}
        for q, d in sec.items():
            for s in (0, 1):
                q2 = qadd(q, qsite(s, m, mod), mod)
                nxt[q2] = nxt.get(q2, 0) + d
        sec = nxt
    return sorted(sec.items())


def heff_apply_block(left, right, m1, m2, mod, cl, cm, cr, wi, wj, lflat, rflat, tflat, out_key):
    """One output block theta'[(a', s1', s2')] of H_eff theta, by the same definition as
    heff_apply restricted to that block (for sampled checks at sizes where the full
    product is too slow). out_key = (a'_index, s1', s2'); returns a d_a' x d_b' array."""
    api, s1p, s2p = out_key
    lay = theta_layout(left, right, m1, m2, mod)
    theta = theta_blocks(tflat, lay)
    lblk = {(w, ai): (apx, lflat[off: off + dp * da].reshape(dp, da))
            for w, ai, apx, off, dp, da in env_left_layout(left, cl, mod)}
    rblk = {(w, bi): (bpx, rflat[off: off + db * dp].reshape(db, dp))
            for w, bi, bpx, off, db, dp in env_right_layout(right, cr, mod)}
    qbp = qadd(qadd(left.charges[api], qsite(s1p, m1, mod), mod), qsite(s2p, m2, mod), mod)
    bpi = right.index[qbp]
    wi_by_w = {}
    for (w, wp, a1, a2, v) in wi:
        if a1 == s1p:
            wi_by_w.setdefault(wp, []).append((w, a2, v))
    out = np.zeros((left.dims[api], right.dims[bpi]), dtype=np.complex128)
    for (wp, wpp, b1, b2, vj) in wj:
        if b1 != s2p:
            continue
        for (w, s1, vi) in wi_by_w.get(wp, []):
            s2 = b2
            # X_w[a', s1, s2, b] for this a'
            for (ai, t1, t2), blk in theta.items():
                if t1 != s1 or t2 != s2 or (w, ai) not in lblk:
                    continue
                apx, lb = lblk[(w, ai)]
                if apx != api:
                    continue
                qb = qadd(qadd(left.charges[ai], qsite(s1, m1, mod), mod), qsite(s2, m2, mod), mod)
                bi = right.index[qb]
                if (wpp, bi) not in rblk or rblk[(wpp, bi)][0] != bpi:
                    continue
                out += (vi * vj) * ((lb @ blk) @ rblk[(wpp, bi)][1])
    return out


def left_env_blocks(sec_l, cl, mod, lflat):
    """{(w, a_index): (a'_index, d_a' x d_a block)} of a left environment in its layout."""
    return {(w, ai): (api, lflat[off: off + dp * da].reshape(dp, da))
            for w, ai, api, off, dp, da in env_left_layout(sec_l, cl, mod)}


def env_left_update_block(sec_l, sec_r, m, mod, cl, cm, w_entries, lflat, a_blocks, out_key, lblk=None):
    """One block of the left environment update of standard two-site DMRG,
        L'_{w'}[c', c] = sum_{w, a', a, s', s} conj(A[a', s', c']) L_w[a', a] W[w, w', s', s] A[a, s, c],
    restated with loops over charge blocks. sec_l / sec_r: BondSectors of the bonds left and
    right of the site (momentum index m); cl / cm: channel charges of the MPO bonds left and
    right of it; w_entries: the site's (w, w', s', s, value) list; lflat: L in the
    env_left_layout(sec_l, cl) layout; a_blocks: {(a_index, s): d_a x d_c array} of the MPS
    tensor, c the sector q_a + q(s). out_key = (w', c_index); returns the d(c + c_{w'}) x d(c)
    block ([bra][ket]), zero if no term reaches it. lblk: the blocks of lflat from
    left_env_blocks, when the caller evaluates many output blocks of one environment."""
    wp, ci = out_key
    qc = sec_r.charges[ci]
    qcp = qadd(qc, cm[wp], mod)
    out = np.zeros((sec_r.dim(qcp), sec_r.dims[ci]), dtype=np.complex128)
    if qcp not in sec_r.index:
        return out
    if lblk is None:
        lblk = left_env_blocks(sec_l, cl, mod, lflat)
    for (w, wq, sp, s, v) in w_entries:
        if wq != wp:
            continue
        qa = qsub(qc, qsite(s, m, mod), mod)
        qap = qsub(qcp, qsite(sp, m, mod), mod)
        if qa not in sec_l.index or qap not in sec_l.index:
            continue
        ai, api = sec_l.index[qa], sec_l.index[qap]
        if (w, ai) not in lblk or lblk[(w, ai)][0] != api:
            continue
        if (ai, s) not in a_blocks or (api, sp) not in a_blocks:
            continue
        out += v * (a_blocks[(api, sp)].conj().T @ lblk[(w, ai)][1] @ a_blocks[(ai, s)])
    return out


def env_right_update_block(sec_l, sec_r, m, mod, cl, cm, w_entries, rflat, b_blocks, out_key):
    """One block of the right environment update of standard two-site DMRG,
        R'_w[c, c'] = sum_{w', b, b', s', s} B[c, s, b] R_{w'}[b, b'] conj(B[c', s', b']) W[w, w', s', s],
    restated with loops over charge blocks. sec_l / sec_r: BondSectors left and right of the
    site (momentum index m); cl / cm: channel charges of the MPO bonds left and right of it;
    rflat: R in the env_right_layout(sec_r, cm) layout; b_blocks: {(c_index, s): d_c x d_b
    array}, b the sector q_c + q(s). out_key = (w, c_index); returns the d(c) x d(c + c_w)
    block ([ket][bra])."""
    w, ci = out_key
    qc = sec_l.charges[ci]
    qcp = qadd(qc, cl[w], mod)
    out = np.zeros((sec_l.dims[ci], sec_l.dim(qcp)), dtype=np.complex128)
    if qcp not in sec_l.index:
        return out
    cpi = sec_l.index[qcp]
    rblk = {(wq, bi): (bpi, rflat[off: off + db * dp].reshape(db, dp))
            for wq, bi, bpi, off, db, dp in env_right_layout(sec_r, cm, mod)}
    for (wq, wp, sp, s, v) in w_entries:
        if wq != w:
            continue
        qb = qadd(qc, qsite(s, m, mod), mod)
        qbp = qadd(qcp, qsite(sp, m, mod), mod)
        if qb not in sec_r.index or qbp not in sec_r.index:
            continue
        bi, bpi = sec_r.index[qb], sec_r.index[qbp]
        if (wp, bi) not in rblk or rblk[(wp, bi)][0] != bpi:
            continue
        if (ci, s) not in b_blocks or (cpi, sp) not in b_blocks:
            continue
        out += v * (b_blocks[(ci, s)] @ rblk[(wp, bi)][1] @ b_blocks[(cpi, sp)].conj().T)
    return out


def two_site_update(left, right, m1, m2, mod, cl, cm, cr, wi, wj, lflat, rflat, tflat, chi, cutoff=1e-14,
                    kmax=30, tol=1e-13, lanczos=None):
    """One two-site update of standard two-site DMRG (the paper defers the algorithm to its
    refs. W92, S2005, S2011), block by block, moving the centre to the right:
      1. the lowest eigenpair of H_eff (heff_apply) by Lanczos from theta
         (oracle.dmrg.lanczos_ground, or the `lanczos(matvec, v0)` given);
      2. the SVD of every middle-charge block of the ground vector (the Schmidt decomposition
         across the centre bond, Sec. III.C);
      3. the global truncation to at most chi singular values above cutoff * s_max, taken in
         the order (value descending, block ascending, index ascending), renormalised so that
         sum s^2 = 1;
      4. the new left-canonical tensor A = U (rows (s1, a) of each block) and the left
         environment of the new bond, L' = A^+ L W_i A (env_left_update_block).
    Returns a dict: energy, matvecs, discarded weight, the new bond's BondSectors, the
    Schmidt values per new sector, A as {(a_index, s1): block}, and L' in the
    env_left_layout(new bond, cm) layout."""
    from oracle import dmrg as D
    lay = theta_layout(left, right, m1, m2, mod)

    def mv(v):
        return heff_apply(left, right, m1, m2, mod, cl, cm, cr, wi, wj, lflat, rflat, v)
    if lanczos is None:
        e, g, nmv = D.lanczos_ground(mv, tflat, kmax=kmax, tol=tol)
    else:
        e, g, nmv = lanczos(mv, tflat)
    svds = []
    for bi, m in enumerate(lay):
        blk = g[m["offset"]: m["offset"] + m["rowdim"] * m["coldim"]].reshape(m["rowdim"], m["coldim"])
        u, s, vh = np.linalg.svd(blk, full_matrices=False)
        svds.append((u, s, vh))
    allv = [(-s[k], bi, k) for bi, (u, s, vh) in enumerate(svds) for k in range(len(s))]
    allv.sort()
    smax = -allv[0][0]
    kept = [t for t in allv[:chi] if -t[0] > cutoff * smax]
    total = sum(t[0] ** 2 for t in allv)
    keep_w = sum(t[0] ** 2 for t in kept)
    nkeep = {}
    for _, bi, k in kept:
        nkeep[bi] = max(nkeep.get(bi, 0), k + 1)
    new_secs = [(lay[bi]["q"], nkeep[bi]) for bi in sorted(nkeep)]
    bond = BondSectors(new_secs)
    norm = np.sqrt(keep_w)
    schmidt = {lay[bi]["q"]: svds[bi][1][:nkeep[bi]] / norm for bi in sorted(nkeep)}
    a_blocks = {}
    for bi in sorted(nkeep):
        u = svds[bi][0][:, :nkeep[bi]]
        for s1, ai, da, ro in lay[bi]["rows"]:
            a_blocks[(ai, s1)] = u[ro:ro + da]
    lay_new = env_left_layout(bond, cm, mod)
    lnew = np.zeros(env_size(lay_new), dtype=np.complex128)
    lblk = left_env_blocks(left, cl, mod, lflat)
    for w, ci, cpi, off, d0, d1 in lay_new:
        lnew[off:off + d0 * d1] = env_left_update_block(left, bond, m1, mod, cl, cm, wi, lflat, a_blocks,
                                                        (w, ci), lblk=lblk).reshape(-1)
    return {"energy": e, "matvecs": nmv, "discarded": 1.0 - keep_w / total, "bond": bond, "schmidt": schmidt,
            "a_blocks": a_blocks, "lenv": lnew}
