"""Host-side checks of the C ABI library (no GPU needed): it loads, exports every symbol
that include/mrdmrg.h declares, and its host MPO builder equals the oracle's MPO."""
import ctypes

import numpy as np
import pytest

import paper_1512_03318_gb300 as P
from paper_1512_03318_gb300 import binding
from oracle import mpo as M


def test_library_exports_declared_symbols():
    lib = P.lib()
    names = binding.declared_symbols()
    assert len(names) >= 15
    for n in names:
        assert hasattr(lib, n), n
    assert lib.mrd_version() >= 100


def test_bindings_cover_header():
    assert set(binding.declared_symbols()) == set(binding._SIGS)


@pytest.mark.parametrize("basis,b", [("mixed", P.MRD_BASIS_MIXED), ("real", P.MRD_BASIS_REAL),
                                     ("mixed_real", P.MRD_BASIS_MIXED_REAL)])
@pytest.mark.parametrize("lx,ly,fp,fq,v", [(3, 4, 1, 4, 1.0), (2, 5, 1, 5, 0.3), (4, 8, 1, 8, 1.0), (3, 10, 1, 10, 1.0),
                                           (2, 6, 1, 3, 7.0)])
def test_product_mpo_equals_oracle_mpo(basis, b, lx, ly, fp, fq, v):
    """The library's MPO builder restates the oracle's machine in C++ (one design written
    twice: a translation check; the oracle's machine is pinned against ED): channel charges
    identical, entries identical in position and equal in value to rounding."""
    m = P.MPO(None, lx, ly, fp, fq, 1.0, v, b)
    o = M.build_mpo(lx, ly, fp / fq, 1.0, v, basis)
    assert m.n_sites == o.n_sites and m.modulus == o.modulus
    for bond in range(m.n_sites + 1):
        assert np.array_equal(m.bond(bond), np.array(o.bond_charges[bond], dtype=np.int32).reshape(-1, 2))
    for j in range(m.n_sites):
        idx, val = m.site(j)
        oi = np.array([e[:4] for e in o.entries[j]], dtype=np.int32)
        ov = np.array([e[4] for e in o.entries[j]])
        assert np.array_equal(idx, oi)
        assert np.max(np.abs(val - ov)) < 1e-13
        if basis == "mixed_real":
            assert np.all(val.imag == 0.0)


def test_mpo_build_rejects_bad_model():
    with pytest.raises(P.MrdError):
        P.MPO(None, 2, 1, 1, 4, 1.0, 1.0, P.MRD_BASIS_MIXED)
    with pytest.raises(P.MrdError):
        P.MPO(None, 2, 4, 1, 0, 1.0, 1.0, P.MRD_BASIS_MIXED)


@pytest.mark.parametrize("basis,b", [("mixed", P.MRD_BASIS_MIXED), ("real", P.MRD_BASIS_REAL)])
@pytest.mark.parametrize("lx,ly", [(3, 4), (3, 6), (3, 8)])
def test_mpo_stats(basis, b, lx, ly):
    """mrd_mpo_stats over the middle ring equals the bookkeeping of the oracle's MPO (bond
    dimensions and nonzero entries counted here); the real-space ring has D = 3L + 2 on every
    bond (Sec. IV.C) and the mixed one stays under the crude bound 26 L + 9 (Sec. IV.D)."""
    m = P.MPO(None, lx, ly, 1, ly, 1.0, 1.0, b)
    o = M.build_mpo(lx, ly, 1 / ly, 1.0, 1.0, basis)
    first, count = ly, ly
    dims = o.dims()
    mean_d, max_d, fill, nnz = m.stats(first, count)
    want_fill = np.mean([len(o.entries[j]) / (4 * dims[j] * dims[j + 1]) for j in range(first, first + count)])
    assert mean_d == pytest.approx(np.mean(dims[first:first + count]), abs=1e-12)
    assert max_d == max(dims[first:first + count])
    assert fill == pytest.approx(want_fill, abs=1e-12)
    assert nnz == sum(len(o.entries[j]) for j in range(first, first + count))
    if basis == "real":
        assert mean_d == 3 * ly + 2 and max_d == 3 * ly + 2
    else:
        assert max_d <= 26 * ly + 9
    with pytest.raises(P.MrdError):
        m.stats(m.n_sites - 1, 2)
