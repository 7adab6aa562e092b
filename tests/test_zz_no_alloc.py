"""mrd_heff_apply_noalloc: the H_eff product for callers that may not allocate device memory
when they need it (for example code whose device memory is owned by an external pool that
must see every allocation). The entry point keeps its step-1 intermediate in a static device
array of MRD_NOALLOC_Z_MAX_ELEMS complex elements instead of a cudaMalloc'd buffer.

Checked here through the C ABI: two calls in a row give the same product as mrd_heff_apply
within the FP64 parity tolerance of the other tests, a second problem of another shape right
after is unaffected by what the first left in the shared array, and a problem whose
intermediate exceeds the static capacity is refused with MRD_E_ARG. This file is collected
last, and it also passes when run alone in a fresh process."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from tests import gpu_cases as G  # noqa: E402

pytestmark = pytest.mark.gpu

TOL = 1e-12          # same relative FP64 tolerance as the H_eff parity tests
MAX_ELEMS = 4194304  # MRD_NOALLOC_Z_MAX_ELEMS in include/mrdmrg.h


@pytest.fixture(scope="module")
def ctx():
    import paper_1512_03318_gb300 as P
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return P.Context(0, torch.cuda.current_stream())


def _dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).to("cuda")


def _loaded(ctx, case):
    import paper_1512_03318_gb300 as P
    h = P.Heff(ctx, **G.heff_args(case))
    h.set_env(_dev(case["lflat"]), _dev(case["rflat"]))
    return h


@pytest.mark.parametrize("first,second", [((1, 4, 40, 44, 1, 2, 5, 6, 7), (7, 6, 150, 170, 5, 3, 4, 8, 6))])
def test_noalloc_matches_apply_twice(ctx, first, second):
    for args in (first, second):
        case = G.random_case(*args)
        h = _loaded(ctx, case)
        T = _dev(case["tflat"])
        ref = torch.empty_like(T)
        h.apply(T, ref)
        outs = []
        for _ in range(2):
            out = torch.full_like(T, complex(7.0, -3.0))   # stale values must not survive
            h.apply_noalloc(T, out)
            outs.append(out)
        torch.cuda.synchronize()
        scale = ref.abs().max().item()
        assert scale > 0
        for out in outs:
            assert (out - ref).abs().max().item() <= TOL * scale


def test_noalloc_rejects_oversized_problem(ctx):
    import paper_1512_03318_gb300 as P
    lx, ly = 4, 8
    mp = P.MPO(None, lx, ly, 1, ly, 1.0, 1.0, P.MRD_BASIS_MIXED)
    site = lx // 2 * ly + ly // 2 - 1
    sites = {}
    for j in (site, site + 1):
        idx, val = mp.site(j)
        sites[j] = [(int(a), int(b), int(c), int(d), complex(v)) for (a, b, c, d), v in zip(idx, val)]
    bonds = {b: mp.bond(b) for b in (site, site + 1, site + 2)}
    case = G.mpo_case(1235, ly, 2048, ly, site, sites, bonds, 2 * ly)   # Z ~ 2e7 elements
    h = _loaded(ctx, case)
    T = _dev(case["tflat"])
    with pytest.raises(P.MrdError) as e:
        h.apply_noalloc(T, torch.empty_like(T))
    assert e.value.code == -1 and str(MAX_ELEMS) in str(e.value)
