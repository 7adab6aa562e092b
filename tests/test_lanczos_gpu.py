"""GPU Lanczos (C ABI) against the oracle's Lanczos and a dense eigensolver on a Hermitian
H_eff: one-channel diagonal MPO and Hermitian random environments, so that
H_eff = L_0 (x) diag(h) (x) diag(g) (x) R_0^T."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import synth  # noqa: E402
from oracle import blocksparse as B  # noqa: E402
from oracle import dmrg as D  # noqa: E402
from tests import gpu_cases as G  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    import paper_1512_03318_gb300 as P
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return P.Context(0, torch.cuda.current_stream())


def _hermitian_case(seed, ly, chi_l, chi_r, m1, m2):
    left = B.BondSectors(synth.bond_sectors(chi_l, ly, 10, synth.substream(seed, 1), min_dim=0))
    right = B.BondSectors(synth.bond_sectors(chi_r, ly, 10, synth.substream(seed, 2), min_dim=0))
    u = synth.uniform_pm1(synth.substream(seed, 3), 4)
    cl, cm, cr = [(0, 0)], [(0, 0)], [(0, 0)]
    wi = [(0, 0, 0, 0, complex(1.0 + 0.5 * u[0])), (0, 0, 1, 1, complex(0.7 + 0.5 * u[1]))]
    wj = [(0, 0, 0, 0, complex(1.1 + 0.5 * u[2])), (0, 0, 1, 1, complex(-0.9 + 0.5 * u[3]))]
    case = G.finish_case(seed, left, right, m1, m2, ly, cl, cm, cr, wi, wj)
    case["lflat"] = synth.hermitian_blocks(left.dims, synth.substream(seed, 8))
    case["rflat"] = synth.hermitian_blocks(right.dims, synth.substream(seed, 9))
    return case


def _oracle_op(case):
    def mv(v):
        return B.heff_apply(case["left"], case["right"], case["m1"], case["m2"], case["mod"], case["cl"],
                            case["cm"], case["cr"], case["wi"], case["wj"], case["lflat"], case["rflat"], v)
    return mv


@pytest.mark.parametrize("seed,ly,chi_l,chi_r,m1,m2", [(41, 3, 24, 26, 1, 2), (43, 4, 30, 28, 3, 1)])
def test_lanczos_matches_dense_and_oracle(ctx, seed, ly, chi_l, chi_r, m1, m2):
    import paper_1512_03318_gb300 as P
    case = _hermitian_case(seed, ly, chi_l, chi_r, m1, m2)
    n = B.theta_size(case["lay"])
    mv = _oracle_op(case)
    dense = np.stack([mv(np.eye(n, dtype=np.complex128)[i]) for i in range(n)], axis=1)
    assert np.max(np.abs(dense - dense.conj().T)) < 1e-12 * np.max(np.abs(dense))
    e_exact = np.linalg.eigvalsh(dense)[0]
    h = P.Heff(ctx, **G.heff_args(case))
    h.set_env(torch.from_numpy(case["lflat"]).cuda(), torch.from_numpy(case["rflat"]).cuda())
    th = torch.from_numpy(case["tflat"].copy()).cuda()
    e_gpu, it = h.lanczos(th, max_iter=60, tol=1e-14)
    e_or, v_or, it_or = D.lanczos_ground(mv, case["tflat"].copy(), kmax=60, tol=1e-14)
    assert abs(e_gpu - e_exact) < 1e-9 * abs(e_exact)
    assert abs(e_gpu - e_or) < 1e-9 * abs(e_exact)
    g = th.cpu().numpy()
    assert abs(np.linalg.norm(g) - 1) < 1e-12
    # the returned vector is an eigenvector: residual small, Rayleigh quotient = energy
    r = mv(g) - e_gpu * g
    assert np.linalg.norm(r) < 1e-5 * abs(e_exact)
    e_ray, res = h.rayleigh(th)
    assert abs(e_ray - e_gpu) < 1e-9 * abs(e_exact)
    assert abs(res - np.linalg.norm(r)) < 1e-6 * abs(e_exact)


def test_lanczos_fixed_iterations_match_oracle(ctx):
    """Same start vector, same number of steps: identical Ritz value up to rounding."""
    import paper_1512_03318_gb300 as P
    case = _hermitian_case(47, 5, 60, 64, 2, 4)
    mv = _oracle_op(case)
    h = P.Heff(ctx, **G.heff_args(case))
    h.set_env(torch.from_numpy(case["lflat"]).cuda(), torch.from_numpy(case["rflat"]).cuda())
    for k in (3, 8):
        th = torch.from_numpy(case["tflat"].copy()).cuda()
        e_gpu, it = h.lanczos(th, max_iter=k, tol=0.0)
        e_or, v_or, it_or = D.lanczos_ground(mv, case["tflat"].copy(), kmax=k, tol=0.0)
        assert it == k and it_or == k
        assert abs(e_gpu - e_or) < 1e-11 * abs(e_or)
        assert abs(abs(np.vdot(th.cpu().numpy(), v_or)) - 1) < 1e-9


@pytest.mark.parametrize("prec", [0, 2, 3])
def test_lanczos_graph_replay_is_bitwise_the_direct_launch(ctx, prec):
    """A Lanczos step captured once as a CUDA graph and replayed for every step gives the
    same Ritz values and ground vector, bit for bit, as launching every kernel (all kernels
    are deterministic), and the library's launch counter counts the replayed kernels."""
    import paper_1512_03318_gb300 as P
    case = _hermitian_case(47, 4, 40, 44, 1, 2)
    res = []
    for graph in (1, 0, 1):
        h = P.Heff(ctx, **G.heff_args(case))
        h.set_option(P.MRD_OPT_GRAPH, graph)
        h.set_option(P.MRD_OPT_AUTOTUNE, 0)   # no tuning launches in the counts
        h.set_env(torch.from_numpy(case["lflat"]).cuda(), torch.from_numpy(case["rflat"]).cuda())
        th = torch.from_numpy(case["tflat"].copy()).cuda()
        c0 = P.launch_count()
        e, it = h.lanczos(th, max_iter=25, tol=1e-14, prec=prec)
        res.append((e, it, th.cpu().numpy(), P.launch_count() - c0))
        h.close()
    (e1, it1, v1, n1), (e0, it0, v0, n0), (e2, it2, v2, n2) = res
    assert it1 == it0 == it2 and it1 > 3
    assert e1 == e0 == e2
    assert np.array_equal(v1, v0) and np.array_equal(v1, v2)
    assert n1 == n0 == n2 > 10 * it1


@pytest.mark.parametrize("prec", [0, 2, 3])
def test_gemm_timing_inside_the_step_graph(ctx, prec):
    """With GEMM timing on, the step graph still runs: its apply records its events at every
    replay, so the timed calls equal the Lanczos steps, as with direct launches, and the
    result is the same bits."""
    import paper_1512_03318_gb300 as P
    case = _hermitian_case(53, 4, 40, 44, 1, 2)
    res = []
    for graph in (1, 0):
        h = P.Heff(ctx, **G.heff_args(case))
        h.set_option(P.MRD_OPT_GRAPH, graph)
        h.set_option(P.MRD_OPT_AUTOTUNE, 0)
        h.set_env(torch.from_numpy(case["lflat"]).cuda(), torch.from_numpy(case["rflat"]).cuda())
        h.timing(True)
        th = torch.from_numpy(case["tflat"].copy()).cuda()
        e, it = h.lanczos(th, max_iter=25, tol=1e-14, prec=prec)
        ms1, ms2, n = h.timing_collect()
        res.append((e, it, th.cpu().numpy(), n, ms1, ms2))
        assert h.timing_collect()[2] == 0   # collected once
        h.close()
    (e1, it1, v1, n1, a1, b1), (e0, it0, v0, n0, a0, b0) = res
    assert it1 == it0 > 3
    assert n1 == n0 == it1
    assert e1 == e0 and np.array_equal(v1, v0)
    assert a1 > 0 and b1 > 0 and a0 > 0 and b0 > 0


@pytest.mark.parametrize("prec", [0, 1, 2, 3])
def test_per_task_launch_equals_grouped_launch(ctx, prec):
    """The per-block baseline (one GEMM launch per output task) computes exactly what the
    grouped persistent launch computes."""
    import paper_1512_03318_gb300 as P
    case = G.random_case(7, 6, 150, 170, 5, 3, 4, 8, 6)
    h = P.Heff(ctx, **G.heff_args(case))
    h.set_env(torch.from_numpy(case["lflat"]).cuda(), torch.from_numpy(case["rflat"]).cuda())
    T = torch.from_numpy(case["tflat"]).cuda()
    a, b = torch.empty_like(T), torch.empty_like(T)
    h.apply(T, a, prec)
    h.set_option(P.MRD_OPT_PER_TASK_LAUNCH, 1)
    c0 = P.launch_count()
    h.apply(T, b, prec)
    n_per_task = P.launch_count() - c0
    torch.cuda.synchronize()
    assert torch.equal(a, b)
    assert n_per_task > 10
    h.close()
