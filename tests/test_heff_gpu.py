"""GPU parity of the two-site H_eff (C ABI, FP64) against the CPU oracle.

Charge tables must be bit-exact; theta' = H_eff theta must agree to 1e-12 relative
(FP64 gate). Inputs are seeded synthetic blocks from `synth`."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import synth  # noqa: E402
from oracle import blocksparse as B  # noqa: E402
from oracle import mpo as M  # noqa: E402
from tests import gpu_cases as G  # noqa: E402

pytestmark = pytest.mark.gpu

TOL = 1e-12


@pytest.fixture(scope="module")
def ctx():
    import paper_1512_03318_gb300 as P
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return P.Context(0, torch.cuda.current_stream())


def _dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).to("cuda")


def _run(ctx, case):
    import paper_1512_03318_gb300 as P
    h = P.Heff(ctx, **G.heff_args(case))
    assert h.theta_len == B.theta_size(case["lay"])
    assert h.lenv_len == B.env_size(case["ll"]) and h.renv_len == B.env_size(case["rl"])
    L, R, T = _dev(case["lflat"]), _dev(case["rflat"]), _dev(case["tflat"])
    out = torch.empty_like(T)
    h.set_env(L, R)
    h.apply(T, out)
    torch.cuda.synchronize()
    return h, out.cpu().numpy()


RANDOM_CASES = [
    (1, 4, 40, 44, 1, 2, 5, 6, 7),
    (3, 5, 60, 50, 4, 0, 6, 5, 8),
    (5, 3, 36, 30, 2, 1, 9, 7, 4),
    (7, 6, 150, 170, 5, 3, 4, 8, 6),     # blocks larger than one 32 x 32 tile
    (21, 2, 300, 280, 1, 0, 4, 4, 4),    # few, large blocks (several tiles, ragged edges)
    (35, 1, 600, 500, 0, 0, 4, 4, 4),    # modulus 1 (real-space charges), blocks up to 390
    (11, 8, 64, 64, 7, 7, 12, 16, 10),
]


@pytest.mark.parametrize("seed,ly,chi_l,chi_r,m1,m2,dl,dm,dr", RANDOM_CASES)
def test_tables_bit_exact(ctx, seed, ly, chi_l, chi_r, m1, m2, dl, dm, dr):
    import paper_1512_03318_gb300 as P
    case = G.random_case(seed, ly, chi_l, chi_r, m1, m2, dl, dm, dr)
    h = P.Heff(ctx, **G.heff_args(case))
    assert np.array_equal(h.table(0), G.oracle_mid_table(case))
    assert np.array_equal(h.table(1), np.array(case["ll"], dtype=np.int64).reshape(-1, 6))
    assert np.array_equal(h.table(2), np.array(case["rl"], dtype=np.int64).reshape(-1, 6))


@pytest.mark.parametrize("seed,ly,chi_l,chi_r,m1,m2,dl,dm,dr", RANDOM_CASES)
def test_heff_matches_oracle(ctx, seed, ly, chi_l, chi_r, m1, m2, dl, dm, dr):
    case = G.random_case(seed, ly, chi_l, chi_r, m1, m2, dl, dm, dr)
    ref = B.heff_apply(case["left"], case["right"], case["m1"], case["m2"], case["mod"], case["cl"], case["cm"],
                       case["cr"], case["wi"], case["wj"], case["lflat"], case["rflat"], case["tflat"])
    h, got = _run(ctx, case)
    assert np.max(np.abs(ref)) > 0
    assert np.max(np.abs(got - ref)) <= TOL * np.max(np.abs(ref))
    f_def, f_exec, f1, f2 = h.flops()
    assert f1 + f2 == f_exec
    assert f_def == B.heff_flops(case["left"], case["right"], case["m1"], case["m2"], case["mod"], case["cl"],
                                 case["cm"], case["cr"], case["wi"], case["wj"])
    assert f_exec > 0


def test_heff_no_mpo_entries_gives_zero(ctx):
    case = G.random_case(13, 4, 40, 40, 1, 2, 3, 3, 3, density=0.0)
    h, got = _run(ctx, case)
    assert np.all(got == 0)


def test_heff_rejects_charge_violation(ctx):
    import paper_1512_03318_gb300 as P
    case = G.random_case(1, 4, 40, 44, 1, 2, 5, 6, 7)
    args = G.heff_args(case)
    args["wi_idx"] = args["wi_idx"].copy()
    # flip the ket occupation of one entry: charge no longer conserved
    args["wi_idx"][0, 3] ^= 1
    with pytest.raises(P.MrdError) as e:
        P.Heff(ctx, **args)
    assert e.value.code == -2


def test_heff_apply_before_env_is_an_error(ctx):
    import paper_1512_03318_gb300 as P
    case = G.random_case(1, 4, 40, 44, 1, 2, 5, 6, 7)
    h = P.Heff(ctx, **G.heff_args(case))
    T = _dev(case["tflat"])
    with pytest.raises(P.MrdError) as e:
        h.apply(T, torch.empty_like(T))
    assert e.value.code == -8


def _model_case(ly, chi, seed, n_mean):
    import paper_1512_03318_gb300 as P
    lx = 4
    mp = P.MPO(None, lx, ly, 1, ly, 1.0, 1.0, P.MRD_BASIS_MIXED)
    site = lx // 2 * ly + ly // 2 - 1            # mid-ring pair: the largest MPO bonds
    sites = {}
    for j in (site, site + 1):
        idx, val = mp.site(j)
        sites[j] = [(int(a), int(b), int(c), int(d), complex(v)) for (a, b, c, d), v in zip(idx, val)]
    bonds = {b: mp.bond(b) for b in (site, site + 1, site + 2)}
    return G.mpo_case(seed, ly, chi, ly, site, sites, bonds, n_mean)


def test_heff_model_mpo_ly8_chi256(ctx):
    """Model MPO of the Ly = 8 Hofstadter cylinder at the middle of a ring, chi = 256."""
    case = _model_case(8, 256, 1236, 16)
    ref = B.heff_apply(case["left"], case["right"], case["m1"], case["m2"], case["mod"], case["cl"], case["cm"],
                       case["cr"], case["wi"], case["wj"], case["lflat"], case["rflat"], case["tflat"])
    h, got = _run(ctx, case)
    assert np.max(np.abs(got - ref)) <= TOL * np.max(np.abs(ref))


@pytest.mark.parametrize("ly,chi", [(8, 1024), (10, 3200)])
def test_heff_model_mpo_sampled_blocks(ctx, ly, chi):
    """Production shapes (Ly = 8, chi = 1024 and Ly = 10, chi = 3200): output blocks sampled
    by the oracle one at a time, plus the Hermiticity-free linearity check
    H(a x + y) = a H x + H y on the full vector."""
    import paper_1512_03318_gb300 as P
    case = _model_case(ly, chi, 1235 + (ly == 10) * 2, 2 * ly)
    h, got = _run(ctx, case)
    lay = case["lay"]
    blocks = B.theta_blocks(got, lay)
    keys = sorted(blocks)
    pick = [keys[i] for i in synth.splitmix64(77, 4) % np.uint64(len(keys))]
    pick.append(max(keys, key=lambda k: blocks[k].size))
    for key in pick:
        ref = B.heff_apply_block(case["left"], case["right"], case["m1"], case["m2"], case["mod"], case["cl"],
                                 case["cm"], case["cr"], case["wi"], case["wj"], case["lflat"], case["rflat"],
                                 case["tflat"], key)
        assert np.max(np.abs(blocks[key] - ref)) <= TOL * max(1.0, np.max(np.abs(ref)))
    # linearity on the full vector
    y = synth.complex_pm1(99, h.theta_len)
    T1, T2 = _dev(case["tflat"]), _dev(y)
    o1, o2, o3 = torch.empty_like(T1), torch.empty_like(T1), torch.empty_like(T1)
    a = 0.3 - 0.7j
    h.apply(T1, o1)
    h.apply(T2, o2)
    h.apply(a * T1 + T2, o3)
    lin = (o3 - (a * o1 + o2)).abs().max().item()
    assert lin <= 1e-12 * o3.abs().max().item()
