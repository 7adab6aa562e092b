"""Tensor-core H_eff (tcgen05, TF32 and split BF16) against the FP64 oracle on the same
seeded inputs. Reduced precision has no closed form: the bounds below are those of the
arithmetic (TF32 keeps 11 significant bits, the BF16 pair hi + lo about 16, FP32
accumulation) with margin; the FP64 path of the library is checked to 1e-12 elsewhere."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import blocksparse as B  # noqa: E402
from tests import gpu_cases as G  # noqa: E402

pytestmark = pytest.mark.gpu

# relative to max |theta'|. Each operand of the chain (theta, Z, WR) carries a rounding of
# 2^-11 (TF32) or about 2^-18 (BF16 hi + lo); sums over thousands of terms with partial
# cancellation amplify it relative to the largest output entry.
TOL = {1: 2e-3, 2: 5e-5}           # small random blocks
TOL_MODEL = {1: 1e-2, 2: 2e-4}     # Ly = 10, chi = 3200 model MPO (K up to ~10^4)


@pytest.fixture(scope="module")
def ctx():
    import paper_1512_03318_gb300 as P
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return P.Context(0, torch.cuda.current_stream())


CASES = [
    (1, 4, 40, 44, 1, 2, 5, 6, 7),
    (7, 6, 150, 170, 5, 3, 4, 8, 6),
    (21, 2, 300, 280, 1, 0, 4, 4, 4),
    (35, 1, 600, 500, 0, 0, 4, 4, 4),
]


@pytest.mark.parametrize("prec", [1, 2])
@pytest.mark.parametrize("seed,ly,chi_l,chi_r,m1,m2,dl,dm,dr", CASES)
def test_tc_heff_matches_oracle(ctx, prec, seed, ly, chi_l, chi_r, m1, m2, dl, dm, dr):
    import paper_1512_03318_gb300 as P
    case = G.random_case(seed, ly, chi_l, chi_r, m1, m2, dl, dm, dr)
    ref = B.heff_apply(case["left"], case["right"], case["m1"], case["m2"], case["mod"], case["cl"], case["cm"],
                       case["cr"], case["wi"], case["wj"], case["lflat"], case["rflat"], case["tflat"])
    h = P.Heff(ctx, **G.heff_args(case))
    dev = lambda x: torch.from_numpy(np.ascontiguousarray(x)).cuda()
    h.set_env(dev(case["lflat"]), dev(case["rflat"]))
    T = dev(case["tflat"])
    out = torch.empty_like(T)
    for _ in range(2):                       # second call reuses the packed environments
        h.apply(T, out, prec=prec)
        got = out.cpu().numpy()
        err = np.max(np.abs(got - ref)) / np.max(np.abs(ref))
        assert err < TOL[prec], err
    # packed environments follow a new set_env
    h.set_env(dev(2 * case["lflat"]), dev(case["rflat"]))
    h.apply(T, out, prec=prec)
    err = np.max(np.abs(out.cpu().numpy() - 2 * ref)) / np.max(np.abs(2 * ref))
    assert err < TOL[prec], err


def test_tc_model_mpo_sampled_blocks(ctx):
    """Ly = 10, chi = 3200 model MPO: sampled output blocks, BF16X3 and TF32."""
    import synth
    import paper_1512_03318_gb300 as P
    from tests.test_heff_gpu import _model_case
    case = _model_case(10, 3200, 1237, 20)
    h = P.Heff(ctx, **G.heff_args(case))
    dev = lambda x: torch.from_numpy(np.ascontiguousarray(x)).cuda()
    h.set_env(dev(case["lflat"]), dev(case["rflat"]))
    T = dev(case["tflat"])
    out64, out = torch.empty_like(T), torch.empty_like(T)
    h.apply(T, out64, prec=0)
    for prec in (2, 1):
        h.apply(T, out, prec=prec)
        err = (out - out64).abs().max().item() / out64.abs().max().item()
        assert err < TOL_MODEL[prec], (prec, err)
    lay = case["lay"]
    blocks = B.theta_blocks(out64.cpu().numpy(), lay)
    keys = sorted(blocks)
    key = keys[int(synth.splitmix64(5, 1)[0] % np.uint64(len(keys)))]
    ref = B.heff_apply_block(case["left"], case["right"], case["m1"], case["m2"], case["mod"], case["cl"], case["cm"],
                             case["cr"], case["wi"], case["wj"], case["lflat"], case["rflat"], case["tflat"], key)
    assert np.max(np.abs(blocks[key] - ref)) <= 1e-12 * max(1.0, np.max(np.abs(ref)))


@pytest.mark.parametrize("prec", [1, 2])
def test_autotuned_tile_configuration(ctx, prec):
    """The autotuner times the candidate tile configurations on the first application of a
    problem class, keeps the fastest for the context (a second H_eff of the class reuses it),
    and every configuration computes the same result bit for bit: tiling the output columns
    and reordering the tasks do not change any element's accumulation order."""
    import paper_1512_03318_gb300 as P
    case = G.random_case(21, 2, 300, 280, 1, 0, 4, 4, 4)
    outs, cfgs = [], []
    for tune in (0, 1, 1):
        h = P.Heff(ctx, **G.heff_args(case))
        h.set_option(P.MRD_OPT_AUTOTUNE, tune)
        h.set_env(torch.from_numpy(case["lflat"]).cuda(), torch.from_numpy(case["rflat"]).cuda())
        T = torch.from_numpy(case["tflat"]).cuda()
        out = torch.empty_like(T)
        h.apply(T, out, prec)
        torch.cuda.synchronize()
        outs.append(out.cpu())
        cfgs.append(h.tc_config())
        h.close()
    assert cfgs[0][3] == 0 and cfgs[1][3] in (1, 2) and cfgs[2][3] == 2
    assert cfgs[1][:3] == cfgs[2][:3]
    assert cfgs[1][0] in (32, 48, 64, 128) and cfgs[1][1] in (2, 3, 4) and cfgs[1][2] in (0, 1)
    assert torch.equal(outs[0], outs[1]) and torch.equal(outs[1], outs[2])


@pytest.mark.parametrize("prec", [1, 2])
def test_wait_limit_reports_timeout_and_context_recovers(ctx, prec):
    """Device-side failure detection without a fault: with the wait limit set to zero every
    wait of the tensor-core GEMM gives up before any copy or MMA is issued, the kernel returns
    and the host reads MRD_E_TIMEOUT; with the default limit restored, the next application on
    the same context is correct again."""
    import paper_1512_03318_gb300 as P
    case = G.random_case(7, 6, 150, 170, 5, 3, 4, 8, 6)
    ref = B.heff_apply(case["left"], case["right"], case["m1"], case["m2"], case["mod"], case["cl"], case["cm"],
                       case["cr"], case["wi"], case["wj"], case["lflat"], case["rflat"], case["tflat"])
    h = P.Heff(ctx, **G.heff_args(case))
    dev = lambda x: torch.from_numpy(np.ascontiguousarray(x)).cuda()
    h.set_env(dev(case["lflat"]), dev(case["rflat"]))
    T = dev(case["tflat"])
    out = torch.empty_like(T)
    h.apply(T, out, prec=prec)               # tables and tile configuration with the default limit
    h.status()
    h.set_option(P.MRD_OPT_WAIT_LIMIT_US, 0)
    h.apply(T, out, prec=prec)
    with pytest.raises(P.MrdError) as ex:
        h.status()
    assert ex.value.code == -7
    h.status()                               # reported once, then cleared
    with pytest.raises(P.MrdError):
        h.set_option(P.MRD_OPT_WAIT_LIMIT_US, -1)
    h.set_option(P.MRD_OPT_WAIT_LIMIT_US, 1000000)
    h.apply(T, out, prec=prec)
    h.status()
    err = np.max(np.abs(out.cpu().numpy() - ref)) / np.max(np.abs(ref))
    assert err < TOL[prec], err


def _real_case(case):
    """The same case with every operand real: MPO entries, environments and theta replaced by
    their real parts (the structure of the sine / cosine machine's real arithmetic)."""
    out = dict(case)
    out["wi"] = [(a, b, c, d, complex(v.real, 0.0)) for a, b, c, d, v in case["wi"]]
    out["wj"] = [(a, b, c, d, complex(v.real, 0.0)) for a, b, c, d, v in case["wj"]]
    for k in ("lflat", "rflat", "tflat"):
        out[k] = case[k].real.astype(np.complex128)
    return out


@pytest.mark.parametrize("prec", [1, 2])
@pytest.mark.parametrize("seed,ly,chi_l,chi_r,m1,m2,dl,dm,dr", CASES[:3])
def test_real_operands_match_oracle(ctx, prec, seed, ly, chi_l, chi_r, m1, m2, dl, dm, dr):
    """Real arithmetic (MRD_OPT_REAL, Sec. IV.D Eq. rot): with real MPO entries, environments
    and theta the tensor cores drop the imaginary planes; the product equals the oracle's
    within the same bounds as the complex form and its imaginary parts are exactly zero. An
    H_eff with complex MPO entries refuses the option."""
    import paper_1512_03318_gb300 as P
    case = _real_case(G.random_case(seed, ly, chi_l, chi_r, m1, m2, dl, dm, dr))
    ref = B.heff_apply(case["left"], case["right"], case["m1"], case["m2"], case["mod"], case["cl"], case["cm"],
                       case["cr"], case["wi"], case["wj"], case["lflat"], case["rflat"], case["tflat"])
    h = P.Heff(ctx, **G.heff_args(case))
    h.set_option(P.MRD_OPT_REAL, 1)
    dev = lambda x: torch.from_numpy(np.ascontiguousarray(x)).cuda()
    h.set_env(dev(case["lflat"]), dev(case["rflat"]))
    T = dev(case["tflat"])
    out = torch.empty_like(T)
    for _ in range(2):
        h.apply(T, out, prec=prec)
        got = out.cpu().numpy()
        assert np.all(got.imag == 0.0)
        err = np.max(np.abs(got - ref)) / np.max(np.abs(ref))
        assert err < TOL[prec], err
    h.close()
    hc = P.Heff(ctx, **G.heff_args(G.random_case(seed, ly, chi_l, chi_r, m1, m2, dl, dm, dr)))
    with pytest.raises(P.MrdError):
        hc.set_option(P.MRD_OPT_REAL, 1)
    hc.close()
