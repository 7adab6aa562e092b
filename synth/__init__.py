"""Seeded synthetic inputs shared by the oracle tests, the GPU parity tests and the bench.

This module holds only random-number generation and input shapes: no Hamiltonian, no
contraction, no charge fusion. Every random number either side consumes is drawn here and
passed in as data.

Generator: SplitMix64 (Steele, Lea & Flood, "Fast splittable pseudorandom number
generators", OOPSLA 2014), used counter-style: the i-th draw of stream `seed` is
mix(seed + (i + 1) * GOLDEN). Doubles are the top 53 bits scaled by 2**-53.

Bond-sector recipe (stand-in for the sector-size histogram of a converged Hofstadter run,
whose figures the paper does not print): sectors (N_rel, K) with N_rel in [-3, 3] around
the mean filling of the bond and K in Z_{L_y}; weight exp(-N_rel^2 / (2 sigma^2)) *
(1 + 0.25 u), u uniform in [-1, 1); every sector first gets the minimum dim 4 and the
remaining chi - 4 * n_sectors is split in proportion to the weights (floor); the largest
sector absorbs the remainder so that the dims sum to chi exactly.
"""
from __future__ import annotations

import numpy as np

GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, n: int, offset: int = 0) -> np.ndarray:
    """Return draws offset..offset+n-1 of the SplitMix64 stream `seed` as uint64."""
    with np.errstate(over="ignore"):
        i = np.arange(offset + 1, offset + n + 1, dtype=np.uint64)
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + i * GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform01(seed: int, n: int, offset: int = 0) -> np.ndarray:
    return (splitmix64(seed, n, offset) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def uniform_pm1(seed: int, n: int, offset: int = 0) -> np.ndarray:
    """Uniform doubles in [-1, 1)."""
    return 2.0 * uniform01(seed, n, offset) - 1.0


def complex_pm1(seed: int, n: int) -> np.ndarray:
    """n complex numbers with re, im uniform in [-1, 1) (re from even draws, im from odd)."""
    u = uniform_pm1(seed, 2 * n)
    return u[0::2] + 1j * u[1::2]


def substream(seed: int, *tags: int) -> int:
    """Derive an independent stream id from a seed and integer tags."""
    s = int(seed) & 0xFFFFFFFFFFFFFFFF
    for t in tags:
        s = int(splitmix64(s ^ (int(t) & 0xFFFFFFFFFFFFFFFF), 1)[0])
    return s


def bond_sectors(chi: int, ly: int, n_mean: int, seed: int, sigma_n: float = 0.6,
                 n_rel_max: int = 3, min_dim: int = 4):
    """Synthetic bond sectors: list of ((N, K), dim) sorted by (N, K), dims summing to chi.

    K ranges over Z_{ly} (ly = 1 gives a single K = 0, the real-space case)."""
    keys = [(n_mean + dn, k) for dn in range(-n_rel_max, n_rel_max + 1) for k in range(ly)]
    u = uniform_pm1(seed, len(keys))
    w = np.array([np.exp(-((n - n_mean) ** 2) / (2 * sigma_n ** 2)) for n, _ in keys]) * (1 + 0.25 * u)
    spare = chi - min_dim * len(keys)
    if spare < 0:
        raise ValueError("chi too small for the sector recipe")
    dims = min_dim + np.floor(spare * w / w.sum()).astype(np.int64)
    big = int(np.argmax(dims))
    dims[big] += chi - int(dims.sum())
    if dims[big] < max(min_dim, 1):
        raise ValueError("chi too small for the sector recipe")
    # min_dim = 0 lets small test cases drop sectors whose share rounds to zero
    return [(k, int(d)) for k, d in zip(keys, dims) if d > 0]


def random_mpo_site(d_left_charges, d_right_charges, modulus: int, m_site: int, seed: int,
                    density: float = 0.5):
    """Random charge-conserving two-level MPO site tensor as a sparse entry list.

    d_left_charges / d_right_charges: lists of channel charges (dN, dK). An entry
    W[w, w', s', s] may be nonzero only when c_{w'} = c_w + q(s') - q(s) with
    q(s) = (s, s * m_site mod modulus). Returns a list of (w, w', s', s, value)."""
    entries = []
    idx = 0
    stream = substream(seed, 17)
    for w, cw in enumerate(d_left_charges):
        for wp, cwp in enumerate(d_right_charges):
            for sp in (0, 1):
                for s in (0, 1):
                    dn = cw[0] + sp - s
                    dk = (cw[1] + (sp - s) * m_site) % modulus
                    if (dn, dk) != (cwp[0], cwp[1] % modulus):
                        continue
                    u = uniform01(stream, 3, offset=3 * idx)
                    idx += 1
                    if u[0] < density:
                        entries.append((w, wp, sp, s, complex(2 * u[1] - 1, 2 * u[2] - 1)))
    return entries


def random_channel_charges(d_left: int, d_mid: int, d_right: int, m1: int, m2: int, modulus: int,
                           seed: int):
    """Channel charges for three consecutive MPO bonds such that every channel of the later
    bonds is reachable: each new channel copies a random earlier channel's charge shifted by
    a random local charge difference q(s') - q(s). Returns (cl, cm, cr) lists of (dN, dK)."""
    st = substream(seed, 23)
    u = uniform01(st, 3 * (d_left + d_mid + d_right))
    k = 0
    cl = []
    for _ in range(d_left):
        cl.append((int(u[k] * 5) - 2, int(u[k + 1] * modulus) % modulus))
        k += 3

    def grow(prev, n, m):
        nonlocal k
        out = []
        for _ in range(n):
            base = prev[int(u[k] * len(prev)) % len(prev)]
            ds = int(u[k + 1] * 3) - 1          # q(s') - q(s) in {-1, 0, +1} occupations
            out.append((base[0] + ds, (base[1] + ds * m) % modulus))
            k += 3
        return out
    cm = grow(cl, d_mid, m1)
    cr = grow(cm, d_right, m2)
    return cl, cm, cr


def hermitian_blocks(dims, seed):
    """Random Hermitian blocks X + X^+ (X entries complex U[-1, 1)), one per dim, flattened
    row-major and concatenated."""
    out = []
    for i, d in enumerate(dims):
        x = complex_pm1(substream(seed, i), d * d).reshape(d, d)
        out.append((x + x.conj().T).reshape(-1))
    return np.concatenate(out) if out else np.zeros(0, dtype=np.complex128)
