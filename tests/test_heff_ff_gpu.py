"""GPU parity of the float-float H_eff (MRD_PREC_FF) against the CPU oracle.

Operands are split into pairs of floats (hi + lo, 48 significant bits) and every product is
accumulated with its exact FMA residual and TwoSum, so each output is a sum of K products
with relative error about K * 2^-47 in the worst case and sqrt(K) * 2^-47 typically. With K
up to ~10^4 (Ly = 10, chi = 3200 model MPO) the bound is 1e-10; the test demands 1e-11 of the
largest output element (random blocks) and of each sampled block (model MPO), and 1e-11
between the float-float and FP64 results on the full production vector."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import synth  # noqa: E402
from oracle import blocksparse as B  # noqa: E402
from tests import gpu_cases as G  # noqa: E402
from tests.test_heff_gpu import RANDOM_CASES, _dev, _model_case  # noqa: E402

pytestmark = pytest.mark.gpu

TOL_FF = 1e-11


@pytest.fixture(scope="module")
def ctx():
    import paper_1512_03318_gb300 as P
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return P.Context(0, torch.cuda.current_stream())


def _run(ctx, case, prec):
    import paper_1512_03318_gb300 as P
    h = P.Heff(ctx, **G.heff_args(case))
    L, R, T = _dev(case["lflat"]), _dev(case["rflat"]), _dev(case["tflat"])
    out = torch.empty_like(T)
    h.set_env(L, R)
    h.apply(T, out, prec)
    torch.cuda.synchronize()
    return h, out.cpu().numpy()


@pytest.mark.parametrize("seed,ly,chi_l,chi_r,m1,m2,dl,dm,dr", RANDOM_CASES)
def test_ff_heff_matches_oracle(ctx, seed, ly, chi_l, chi_r, m1, m2, dl, dm, dr):
    import paper_1512_03318_gb300 as P
    case = G.random_case(seed, ly, chi_l, chi_r, m1, m2, dl, dm, dr)
    ref = B.heff_apply(case["left"], case["right"], case["m1"], case["m2"], case["mod"], case["cl"], case["cm"],
                       case["cr"], case["wi"], case["wj"], case["lflat"], case["rflat"], case["tflat"])
    _, got = _run(ctx, case, P.MRD_PREC_FF)
    assert np.max(np.abs(ref)) > 0
    err = np.max(np.abs(got - ref)) / np.max(np.abs(ref))
    assert err <= TOL_FF, err
    # float-float is not FP64: the error is well above FP64 rounding but far below FP32
    assert err > 0


def test_ff_heff_model_mpo_ly10_chi3200(ctx):
    """Production shape: sampled output blocks against the oracle, and the full vector against
    the FP64 GPU form."""
    import paper_1512_03318_gb300 as P
    case = _model_case(10, 3200, 1237, 20)
    h, got = _run(ctx, case, P.MRD_PREC_FF)
    blocks = B.theta_blocks(got, case["lay"])
    keys = sorted(blocks)
    pick = [keys[i] for i in synth.splitmix64(78, 3) % np.uint64(len(keys))]
    pick.append(max(keys, key=lambda k: blocks[k].size))
    for key in pick:
        ref = B.heff_apply_block(case["left"], case["right"], case["m1"], case["m2"], case["mod"], case["cl"],
                                 case["cm"], case["cr"], case["wi"], case["wj"], case["lflat"], case["rflat"],
                                 case["tflat"], key)
        assert np.max(np.abs(blocks[key] - ref)) <= TOL_FF * max(1.0, np.max(np.abs(ref)))
    T = _dev(case["tflat"])
    o64 = torch.empty_like(T)
    h.apply(T, o64, P.MRD_PREC_FP64)
    torch.cuda.synchronize()
    o64 = o64.cpu().numpy()
    assert np.max(np.abs(got - o64)) <= TOL_FF * np.max(np.abs(o64))


@pytest.mark.parametrize("seed,ly,chi_l,chi_r,m1,m2,dl,dm,dr", RANDOM_CASES[:3])
def test_ff_heff_real_operands_match_oracle(ctx, seed, ly, chi_l, chi_r, m1, m2, dl, dm, dr):
    """Real arithmetic of the float-float GEMM (MRD_OPT_REAL, Sec. IV.D Eq. rot): with real MPO
    entries, environments and theta each multiply-add is one float-float product; the result
    equals the oracle's within the complex form's bound and its imaginary parts are zero."""
    import paper_1512_03318_gb300 as P
    from tests.test_heff_tc_gpu import _real_case
    case = _real_case(G.random_case(seed, ly, chi_l, chi_r, m1, m2, dl, dm, dr))
    ref = B.heff_apply(case["left"], case["right"], case["m1"], case["m2"], case["mod"], case["cl"], case["cm"],
                       case["cr"], case["wi"], case["wj"], case["lflat"], case["rflat"], case["tflat"])
    assert np.all(ref.imag == 0.0)
    h = P.Heff(ctx, **G.heff_args(case))
    h.set_option(P.MRD_OPT_REAL, 1)
    h.set_env(_dev(case["lflat"]), _dev(case["rflat"]))
    T = _dev(case["tflat"])
    out = torch.empty_like(T)
    h.apply(T, out, P.MRD_PREC_FF)
    torch.cuda.synchronize()
    got = out.cpu().numpy()
    assert np.all(got.imag == 0.0)
    err = np.max(np.abs(got - ref)) / np.max(np.abs(ref))
    assert err <= TOL_FF, err
    h.close()
