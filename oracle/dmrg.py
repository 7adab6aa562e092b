"""Dense (symmetry-free) two-site DMRG in complex128. Test infrastructure only.

The paper applies standard DMRG (its refs. W92, S2005, S2011) and does not restate it; this
module is the textbook finite-system two-site algorithm written out plainly:

  theta = M_i M_{i+1};  H_eff theta = L W_i W_{i+1} R theta;  Lanczos for the lowest
  eigenpair of H_eff;  SVD theta = U S V^+;  keep the largest chi singular values above
  1e-14 * s_max;  renormalise sum s^2 = 1;  update the environment on the side the centre
  leaves;  sweep left to right and back.

Index conventions (shared with the block-sparse restatement):
  MPS tensor      M[a, s, b]            (left bond, physical, right bond)
  MPO tensor      W[w, w', s', s]       (left channel, right channel, bra, ket)
  left env        L[w, a', a]           (channel, bra, ket);  L at bond 0 = [[[1]]]
  right env       R[w, b, b']           (channel, ket, bra);  R at bond n = [[[1]]]
  H_eff theta[a', s1', s2', b'] = sum L[w,a',a] W_i[w,w',s1',s1] W_{i+1}[w',w'',s2',s2]
                                    R[w'',b,b'] theta[a,s1,s2,b]
"""
from __future__ import annotations

import numpy as np

import synth


def heff_apply_dense(L, Wi, Wj, R, theta):
    """H_eff theta, contracted in the order of its definition: L first, then W_i, W_{i+1},
    then R."""
    x = np.einsum("wpa,asub->wpsub", L, theta)            # X_w[a', s1, s2, b]
    y = np.einsum("wvts,wpsub->vptub", Wi, x)             # Y_{w'}[a', s1', s2, b]
    z = np.einsum("vzru,vptub->zptrb", Wj, y)             # Z_{w''}[a', s1', s2', b]
    return np.einsum("zptrb,zbc->ptrc", z, R)             # theta'[a', s1', s2', b']


def env_left_update(L, A, W):
    """L'[w', c', c] = sum L[w, a', a] conj(A[a', s', c']) W[w, w', s', s] A[a, s, c]."""
    t1 = np.einsum("wpa,asc->wpsc", L, A)
    t2 = np.einsum("wpsc,wvts->vptc", t1, W)
    return np.einsum("vptc,pte->vec", t2, A.conj())


def env_right_update(R, B, W):
    """R'[w, c, c'] = sum B[c, s, b] R[w', b, b'] conj(B[c', s', b']) W[w, w', s', s]."""
    t1 = np.einsum("csb,vbe->vcse", B, R)
    t2 = np.einsum("vcse,wvts->wcte", t1, W)
    return np.einsum("wcte,fte->wcf", t2, B.conj())


def lanczos_ground(matvec, v0, kmax=30, tol=1e-13):
    """Lowest eigenpair of a Hermitian operator by Lanczos with full reorthogonalisation
    (two classical Gram-Schmidt passes), started from v0. Stops when the lowest Ritz value
    changes by less than tol * |E| or the Krylov space is exhausted."""
    nrm = np.linalg.norm(v0)
    vs = [v0 / nrm]
    alphas, betas = [], []
    e_prev = None
    evals = evecs = None
    for j in range(kmax):
        w = matvec(vs[j])
        a = float(np.vdot(vs[j], w).real)
        alphas.append(a)
        for _ in range(2):
            for v in vs:
                w = w - np.vdot(v, w) * v
        b = float(np.linalg.norm(w))
        k = len(alphas)
        t = np.diag(alphas) + np.diag(betas, 1) + np.diag(betas, -1)
        evals, evecs = np.linalg.eigh(t)
        e0 = evals[0]
        if e_prev is not None and abs(e0 - e_prev) < tol * abs(e0):
            break
        if b < 1e-12 * max(1.0, abs(a)):
            break
        e_prev = e0
        if j + 1 < kmax:
            betas.append(b)
            vs.append(w / b)
    y = evecs[:, 0]
    g = sum(y[i] * vs[i] for i in range(len(y)))
    return float(evals[0]), g / np.linalg.norm(g), len(alphas)


def truncate_svd(theta2d, chi, cutoff=1e-14):
    """SVD and truncation: keep at most chi singular values, all above cutoff * s_max;
    renormalise the kept ones to sum s^2 = 1. Returns (U, s, Vh, discarded weight)."""
    u, s, vh = np.linalg.svd(theta2d, full_matrices=False)
    keep = int(min(chi, np.sum(s > cutoff * s[0])))
    disc = float(np.sum(s[keep:] ** 2) / np.sum(s ** 2))
    s_k = s[:keep] / np.linalg.norm(s[:keep])
    return u[:, :keep], s_k, vh[:keep], disc


def random_mps(n, chi, seed):
    """Seeded random MPS (re, im uniform in [-1, 1)), bond j dim min(chi, 2^j, 2^(n-j)),
    right-canonicalised by QR."""
    dims = [min(chi, 2 ** j, 2 ** (n - j)) for j in range(n + 1)]
    mps = []
    for j in range(n):
        vals = synth.complex_pm1(synth.substream(seed, j), dims[j] * 2 * dims[j + 1])
        mps.append(vals.reshape(dims[j], 2, dims[j + 1]))
    for j in range(n - 1, 0, -1):
        dl, _, dr = mps[j].shape
        q, r = np.linalg.qr(mps[j].reshape(dl, 2 * dr).conj().T)
        mps[j] = q.conj().T.reshape(-1, 2, dr)
        mps[j - 1] = np.einsum("asb,bc->asc", mps[j - 1], r.conj().T)
    mps[0] = mps[0] / np.linalg.norm(mps[0])
    return mps


def dmrg(mpo, chi, sweeps=10, seed=1234, tol=1e-12, kmax=30, lanczos_tol=1e-13, mps=None):
    """Finite two-site DMRG. mpo: oracle.mpo.MPO (R at bond 0 and F at bond n are the
    only nodes there). Returns dict with the energy of each sweep and the final MPS."""
    n = mpo.n_sites
    ws = [mpo.dense_site(j) for j in range(n)]
    mps = random_mps(n, chi, seed) if mps is None else [m.copy() for m in mps]
    Ls = [None] * (n + 1)
    Rs = [None] * (n + 1)
    Ls[0] = np.ones((1, 1, 1), dtype=np.complex128)
    Rs[n] = np.ones((1, 1, 1), dtype=np.complex128)
    for j in range(n - 1, 1, -1):
        Rs[j] = env_right_update(Rs[j + 1], mps[j], ws[j])
    energies = []
    e = None
    for sw in range(sweeps):
        order = list(range(n - 1)) + list(range(n - 2, -1, -1))
        for step, i in enumerate(order):
            right = step < n - 1
            theta = np.einsum("asb,buc->asuc", mps[i], mps[i + 1])
            shape = theta.shape
            mv = lambda v: heff_apply_dense(Ls[i], ws[i], ws[i + 1], Rs[i + 2], v.reshape(shape)).reshape(-1)
            e, g, _ = lanczos_ground(mv, theta.reshape(-1), kmax=kmax, tol=lanczos_tol)
            u, s, vh, _ = truncate_svd(g.reshape(shape[0] * 2, 2 * shape[3]), chi)
            if right:
                mps[i] = u.reshape(shape[0], 2, -1)
                mps[i + 1] = (s[:, None] * vh).reshape(-1, 2, shape[3])
                Ls[i + 1] = env_left_update(Ls[i], mps[i], ws[i])
            else:
                mps[i] = (u * s[None, :]).reshape(shape[0], 2, -1)
                mps[i + 1] = vh.reshape(-1, 2, shape[3])
                Rs[i + 1] = env_right_update(Rs[i + 2], mps[i + 1], ws[i + 1])
        energies.append(e)
        if len(energies) > 1 and abs(energies[-1] - energies[-2]) < tol * abs(e):
            break
    return {"energies": energies, "energy": energies[-1], "mps": mps}


def mps_expectation_mpo(mps, mpo):
    """<psi|W|psi> / <psi|psi> by left-to-right transfer."""
    L = np.ones((1, 1, 1), dtype=np.complex128)
    N = np.ones((1, 1), dtype=np.complex128)
    for j, A in enumerate(mps):
        L = env_left_update(L, A, mpo.dense_site(j))
        N = np.einsum("pa,psc,asd->cd", N, A.conj(), A)
    return complex(L[0, 0, 0] / N[0, 0])
