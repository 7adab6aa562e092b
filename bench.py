"""Benchmark of the two-site DMRG hot path on GB300 (one JSON line on rank 0).

Step: one two-site update at bond dimension chi = 3200 on the Ly = 10 interacting Hofstadter
cylinder (flux 1/10, t = 1, V = 1, one particle per ring, Lx = 12), mixed real/momentum-space
MPO built by the library: H_eff tables, theta, Lanczos with split-BF16 tensor-core matvecs,
float-float Rayleigh-quotient refinement of the ground vector, block SVD (FP32 pre-sweeps,
float-float Jacobi sweeps) and truncation, float-float environment update. The state is a seeded random MPS, left-canonical
left of the centre and right-canonical right of it, with genuine environments contracted from
the ends; bond sectors follow the synthetic sector recipe of `synth` (70 sectors of dims 4..277
at chi = 3200). Successive steps move the centre one site to the right. `value` is seconds per
update (lower is better).

Also measured in the same run: the plain FP64 form of the update, the energy error of the
mixed form against a converged FP64 reference of the same H_eff, H_eff throughput (TFLOP/s,
definition-order flops) in FP64, float-float, TF32 and split BF16 on the Lx = 20 cylinder's
mid-ring sites with random environments, and the CPU oracle (s/update from a bounded sample).

Launch: python bench.py [--gpus N --steps K --warmup W]; N > 1 under torchrun runs independent
replicas (weak scaling). --impl reference times the CPU oracle in the same unit.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import synth  # noqa: E402

METRIC = "s per two-site update & H_eff TFLOP/s at χ=3200, mixed-prec vs FP64, ΔE≤1e-9"
LY, CHI, FLUX_P, FLUX_Q, T_HOP, V_INT = 10, 3200, 1, 10, 1.0, 1.0
LX_UPDATE = 12            # cylinder of the update steps
LX_MATVEC = 20            # cylinder of the matvec throughput measurement
SEED = 1234 + 3           # workload index 3 (chi = 3200)
FP64_PEAK_TFLOPS = 2 * 2 * 152 * 2.070e9 / 1e12   # 2 DFMA/clk/SM x 2 flop x 152 SMs x 2.07 GHz
FP32_ISSUE_TINSTR = 128 * 152 * 2.070e9 / 1e12     # FP32 instructions per second (lanes x SMs x clock)
FF_INSTR_PER_CMAC = 36   # FP32 instructions of a float-float complex multiply-add (3 products of 12)
PREC = {"fp64": 0, "tf32": 1, "bf16x3": 2, "ff": 3}


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["bf16_tflops"]), float(d.get("bf16_tflops_sustained", d["bf16_tflops"])), "of measured"
    except (OSError, KeyError, ValueError):
        return 1900.0, 1700.0, "of fallback"


def set_chi(chi):
    global CHI
    CHI = chi


def update_centre(lx):
    return (lx // 2) * LY + LY // 2 - 1


def update_caps(lx, chi):
    n = lx * LY
    return [[(q[0], q[1], d) for q, d in synth.bond_sectors(chi, LY, round(j / LY), synth.substream(SEED, 7, j))]
            if 2 <= j <= n - 2 else [] for j in range(n + 1)]


def workload_name(chi):
    return (f"two-site update, mixed-space Hofstadter cylinder Ly={LY} Lx={LX_UPDATE} flux={FLUX_P}/{FLUX_Q} "
            f"t={T_HOP} V={V_INT} N={LX_UPDATE}, chi={chi}, random canonical MPS with synthetic sectors")


class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, device):
        self.device, self.proc, self.path = device, None, None

    def __enter__(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.device), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
            time.sleep(0.3)
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            time.sleep(0.2)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if self.proc is None or not self.path:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["clock sampling unavailable"]}
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) == 7:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        num = lambda x: x.replace(".", "").isdigit()
        sm = [float(r[0]) for r in rows if num(r[0])]
        mx = [float(r[1]) for r in rows if num(r[1])]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[3 + k].lower() == "active"})
        pw = [float(r[2]) for r in rows if num(r[2])]
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows), "power_w_max": max(pw) if pw else None}


# ---------------------------------------------------------------- CPU oracle (baseline / reference arm)

def oracle_workload():
    """The first H_eff of the timed updates for the CPU oracle: the oracle's own MPO of the
    10 x 12 cylinder at the centre sites, the seeded bond sectors that cap the centre bonds of
    the GPU state, random environments and theta of those shapes."""
    from oracle import blocksparse as B
    from oracle import mpo as M
    site = update_centre(LX_UPDATE)
    caps = update_caps(LX_UPDATE, CHI)
    mp = M.build_mpo(LX_UPDATE, LY, FLUX_P / FLUX_Q, T_HOP, V_INT, "mixed")
    left = B.BondSectors([((n, k), d) for n, k, d in caps[site]])
    right = B.BondSectors([((n, k), d) for n, k, d in caps[site + 2]])
    m1, m2, mod = site % LY, (site + 1) % LY, LY
    cl, cm, cr = mp.bond_charges[site], mp.bond_charges[site + 1], mp.bond_charges[site + 2]
    wi, wj = mp.entries[site], mp.entries[site + 1]
    lay = B.theta_layout(left, right, m1, m2, mod)
    s = synth.substream(SEED, 200)
    lflat = synth.complex_pm1(synth.substream(s, 8), B.env_size(B.env_left_layout(left, cl, mod)))
    rflat = synth.complex_pm1(synth.substream(s, 9), B.env_size(B.env_right_layout(right, cr, mod)))
    tflat = synth.complex_pm1(synth.substream(s, 10), B.theta_size(lay))
    return B, (left, right, m1, m2, mod, cl, cm, cr, wi, wj), (lflat, rflat, tflat)


ORACLE_MATVECS = 30   # matvecs of one oracle update: its Lanczos step cap


def oracle_step_factory():
    """One CPU step: the oracle's H_eff restricted to the output blocks of every fourth left
    sector (a fixed quarter of the output, a second or so of work). Returns the step, its flops
    and the flops of the full H_eff."""
    B, args, flats = oracle_workload()
    rows = set(range(0, len(args[0].dims), 4))
    flops = B.heff_flops(*args, rows=rows)
    full = B.heff_flops(*args)

    def step():
        t0 = time.perf_counter()
        B.heff_apply(*args, *flats, rows=rows)
        return time.perf_counter() - t0
    return step, flops, full


def oracle_s_per_update(t_sample, flops, full):
    """Seconds per two-site update of the oracle, from one sample step: the full matvec time
    (sample time x full / sample flops) times ORACLE_MATVECS. The oracle's SVD and environment
    update are left out, so this is a lower bound."""
    return t_sample * full / flops * ORACLE_MATVECS


def oracle_sample_text(flops, full, t):
    return (f"oracle block-sparse H_eff (numpy complex128, loops over charge blocks) of the first update's H_eff "
            f"(Ly={LY}, Lx={LX_UPDATE}, chi={CHI}) on the output blocks of every 4th left sector "
            f"({flops / 1e9:.1f} of {full / 1e9:.1f} GFLOP, {t:.2f} s), scaled to the full matvec and to "
            f"{ORACLE_MATVECS} matvecs per update (the oracle Lanczos cap); SVD and environment update not "
            f"included: a lower bound")


def cpu_baseline(n_steps=3):
    step, flops, full = oracle_step_factory()
    step()
    times = [step() for _ in range(n_steps)]
    t = statistics.median(times)
    return {"value": oracle_s_per_update(t, flops, full), "unit": "s/update", "cores": len(os.sched_getaffinity(0)),
            "kind": "oracle", "sample": oracle_sample_text(flops, full, t) + f"; median of {n_steps} after 1 warm-up"}


def run_reference(args):
    """The reference arm: the CPU oracle, timed on the host cores on bounded samples of the
    update workload, in the bench's own metric (s/update, lower is better)."""
    if rank_env()[0] != 0:   # under torchrun rank 0 alone runs the reference arm
        return 0
    step, flops, full = oracle_step_factory()
    for _ in range(args.warmup):
        step()
    t0 = time.perf_counter()
    times = [step() for _ in range(args.steps)]
    total = time.perf_counter() - t0
    value = oracle_s_per_update(total / args.steps, flops, full)
    cores = len(os.sched_getaffinity(0))
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "s/update", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
            "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "c128", "data": "synthetic",
            "config": {"workload": workload_name(CHI), "chi": CHI, "ly": LY, "lx": LX_UPDATE,
                       "sample": "each step: the oracle H_eff on every 4th left sector's output blocks"},
            "cpu_baseline": {"value": value, "unit": "s/update", "cores": cores, "kind": "oracle",
                             "sample": oracle_sample_text(flops, full, statistics.median(times)) +
                                       f"; {args.steps} steps after {args.warmup} warm-up"},
            "e2e": {"value": value, "unit": "s/update", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


# ---------------------------------------------------------------- GPU measurements

def matvec_throughput(P, ctx, torch, dev, stream, reps=10, precs=None):
    """H_eff TFLOP/s per precision on the Lx = 20 mid-ring sites, random environments."""
    site = update_centre(LX_MATVEC)
    mpo = P.MPO(None, LX_MATVEC, LY, FLUX_P, FLUX_Q, T_HOP, V_INT, P.MRD_BASIS_MIXED)
    sec = lambda tag: np.array([[q[0], q[1], d] for q, d in synth.bond_sectors(CHI, LY, LX_MATVEC // 2,
                                                                              synth.substream(SEED, tag))],
                               dtype=np.int32)
    i_idx, i_val = mpo.site(site)
    j_idx, j_val = mpo.site(site + 1)
    h = P.Heff(ctx, sec(1), sec(2), site % LY, (site + 1) % LY, mpo.modulus, mpo.bond(site), mpo.bond(site + 1),
               mpo.bond(site + 2), i_idx, i_val, j_idx, j_val)
    s = synth.substream(SEED, 100)
    L = torch.from_numpy(synth.complex_pm1(synth.substream(s, 8), h.lenv_len)).to(dev)
    R = torch.from_numpy(synth.complex_pm1(synth.substream(s, 9), h.renv_len)).to(dev)
    T = torch.from_numpy(synth.complex_pm1(synth.substream(s, 10), h.theta_len)).to(dev)
    out = torch.empty_like(T)
    h.set_env(L, R)
    f_def, f_exec, f1, f2 = h.flops()
    res = {}
    for name, prec in PREC.items():
        if precs and name not in precs:
            continue
        n = reps if prec in (1, 2) else 3
        for _ in range(2):
            h.apply(T, out, prec=prec)
        torch.cuda.synchronize(dev)
        h.timing(True)
        h.timing_collect()
        h.timing(True)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(n):
            h.apply(T, out, prec=prec)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        ms1, ms2, calls = h.timing_collect()
        h.timing(False)
        ms = e0.elapsed_time(e1) / n
        res[name] = {"tflops": f_def / (ms / 1e3) / 1e12, "ms": ms, "ms_step1": ms1 / max(calls, 1),
                     "ms_step2": ms2 / max(calls, 1)}
        if prec in (1, 2):
            res[name]["tile_config"] = dict(zip(["cols_per_tile", "stages", "task_order", "source"], h.tc_config()))
    # the per-block baseline: one GEMM launch per output task instead of the grouped launch
    h.set_option(P.MRD_OPT_PER_TASK_LAUNCH, 1)
    for name in ("bf16x3",) if "bf16x3" in res else ():
        h.apply(T, out, prec=PREC[name])
        torch.cuda.synchronize(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(2):
            h.apply(T, out, prec=PREC[name])
        e1.record(stream)
        torch.cuda.synchronize(dev)
        res[name]["ms_per_task_launches"] = e0.elapsed_time(e1) / 2
    h.set_option(P.MRD_OPT_PER_TASK_LAUNCH, 0)
    res["flops_definition"] = f_def
    res["flops_executed"] = f_exec
    res["flops_step1"], res["flops_step2"] = f1, f2
    res["theta_len"] = h.theta_len
    h.close()
    return res


def real_vs_mixed(P, ctx, torch, dev, stream):
    """The paper's comparison of the two bases (Sec. III.B, Fig. 3) on this build's own code:
    the same Hofstadter cylinder (Lx = 20, mid-ring sites) at the same chi, with the mixed
    basis (charges N and K mod Ly, the library's mixed-space MPO) and with the real-space basis
    (charge N only, the real-space MPO, D = 3 Ly + 2). Reports the H_eff time per application
    (BF16X3 and FP64), the definition-order flops and the sizes of theta and of the two
    environments. Operand values are seeded random numbers (timing does not depend on them)."""
    site = update_centre(LX_MATVEC)
    gen = torch.Generator(device=dev)
    gen.manual_seed(SEED)
    out = {}
    for name, basis, ly_q in (("mixed", P.MRD_BASIS_MIXED, LY), ("real", P.MRD_BASIS_REAL, 1)):
        mpo = P.MPO(None, LX_MATVEC, LY, FLUX_P, FLUX_Q, T_HOP, V_INT, basis)
        sec = lambda tag: np.array([[q[0], q[1], d] for q, d in synth.bond_sectors(CHI, ly_q, LX_MATVEC // 2,
                                                                                  synth.substream(SEED, tag))],
                                   dtype=np.int32)
        i_idx, i_val = mpo.site(site)
        j_idx, j_val = mpo.site(site + 1)
        m1, m2 = (site % LY, (site + 1) % LY) if basis == P.MRD_BASIS_MIXED else (0, 0)
        h = P.Heff(ctx, sec(1), sec(2), m1, m2, mpo.modulus, mpo.bond(site), mpo.bond(site + 1), mpo.bond(site + 2),
                   i_idx, i_val, j_idx, j_val)
        rnd = lambda n: torch.randn(n, dtype=torch.complex128, device=dev, generator=gen)
        L, R, T = rnd(h.lenv_len), rnd(h.renv_len), rnd(h.theta_len)
        o = torch.empty_like(T)
        h.set_env(L, R)
        f_def = h.flops()[0]
        res = {"theta_elems": h.theta_len, "env_bytes": 16 * (h.lenv_len + h.renv_len), "flops_definition": f_def,
               "mpo_bond_dim": int(len(mpo.bond(site + 1)))}
        for pname, n in (("bf16x3", 5), ("fp64", 1)):
            prec = PREC[pname]
            h.apply(T, o, prec)
            torch.cuda.synchronize(dev)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(n):
                h.apply(T, o, prec)
            e1.record(stream)
            torch.cuda.synchronize(dev)
            res[f"ms_{pname}"] = e0.elapsed_time(e1) / n
        h.close()
        del L, R, T, o
        out[name] = res
    out["ratio_real_over_mixed"] = {k: out["real"][k] / out["mixed"][k]
                                    for k in ("ms_bf16x3", "ms_fp64", "flops_definition", "env_bytes", "theta_elems")}
    return out


def real_vs_mixed_or_note(P, ctx, torch, dev, stream):
    try:
        return real_vs_mixed(P, ctx, torch, dev, stream)
    except (P.MrdError, torch.cuda.OutOfMemoryError) as e:   # the real-space problem is ~20x larger
        torch.cuda.empty_cache()
        return {"skipped": f"{type(e).__name__}: {e}"}


def mpo_diagnostics(P):
    """Mean and largest MPO bond dimension and mean fill over a bulk ring (the second of three),
    real-space and mixed machines, against the real-space 3L + 2 (Sec. IV.C-D). Host only."""
    out = {}
    for ly in (4, 6, 8, 10, 12):
        row = {"3L+2": 3 * ly + 2}
        for name, basis in (("real", P.MRD_BASIS_REAL), ("mixed", P.MRD_BASIS_MIXED)):
            m = P.MPO(None, 3, ly, 1, ly, T_HOP, V_INT, basis)
            mean_d, max_d, fill, _ = m.stats(ly, ly)
            row[name] = {"mean_D": round(mean_d, 3), "max_D": max_d, "fill": round(fill, 4)}
            m.close()
        out[str(ly)] = row
    return out


# ---------------------------------------------------------------- replicas (N > 1)

def rank_env(env=None):
    """(rank, world size, local rank) of this process, from the torchrun environment."""
    env = os.environ if env is None else env
    return int(env.get("RANK", "0")), int(env.get("WORLD_SIZE", "1")), int(env.get("LOCAL_RANK", "0"))


def replica_seed(rank):
    """Each replica runs its own seeded problem (no data-path collective)."""
    return 11 + rank


def ranks_barrier(dist):
    if dist is not None:
        dist.barrier()


def ranks_max(x, dist, device):
    """The largest of the ranks' values of x (every rank gets it); x itself on one rank."""
    if dist is None:
        return x
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def per_update_value(seconds, steps, world):
    """Whole-job seconds per update: the slowest rank's time over all ranks' updates."""
    return seconds / steps / world


def make_state(P, ctx, mpo, chi, caps, seed):
    return P.DMRG(ctx, mpo, LX_UPDATE, 0, chi, seed=seed, center=update_centre(LX_UPDATE), caps=caps)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=6)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--chi", type=int, default=CHI)
    ap.add_argument("--refine", type=int, default=1, help="FP64 refinement matvecs of the mixed form")
    ap.add_argument("--fp64-steps", type=int, default=1)
    ap.add_argument("--fast-restarts", type=int, default=8, help="restarts of the reduced-precision Lanczos")
    ap.add_argument("--only-matvec", action="store_true", help="H_eff throughput only (profiling runs)")
    ap.add_argument("--precs", default="", help="with --only-matvec: comma-separated precisions (default all)")
    ap.add_argument("--profile-update", action="store_true",
                    help="warm-up updates, then one update inside a CUDA profiler range (ncu --profile-from-start off)")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    if args.impl == "reference":
        return run_reference(args)

    import torch
    import paper_1512_03318_gb300 as P

    rank, world, local = rank_env()
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)
    ctx = P.Context(local, stream)
    chi = args.chi
    n_sites = LX_UPDATE * LY
    centre = update_centre(LX_UPDATE)
    if centre + args.warmup + args.steps + 1 > n_sites - 2:
        raise SystemExit("too many steps for the cylinder length")
    mpo = P.MPO(None, LX_UPDATE, LY, FLUX_P, FLUX_Q, T_HOP, V_INT, P.MRD_BASIS_MIXED)
    caps = update_caps(LX_UPDATE, chi)
    seed = replica_seed(rank)
    # reduced-precision Lanczos restarted until its Ritz value settles, then FP64 refinement
    mixed = P.DMRG.params(chi, 1e-14, 60, 1e-10, PREC["bf16x3"], args.refine, 1e-13, restarts=args.fast_restarts)
    if args.only_matvec:
        set_chi(chi)
        precs = [p for p in args.precs.split(",") if p]
        mv = matvec_throughput(P, ctx, torch, dev, stream, precs=precs)
        done = [k for k in PREC if k in mv]
        print(json.dumps({"only_matvec": True, "chi": chi, "heff_tflops": {k: mv[k]["tflops"] for k in done},
                          "heff_ms_steps": {k: [mv[k]["ms_step1"], mv[k]["ms_step2"]] for k in done}}))
        return 0

    if args.profile_update:
        st = make_state(P, ctx, mpo, chi, caps, seed)   # tuning pass, as before the timed updates
        for k in range(args.warmup + 1):
            st.update(centre + k, +1, mixed)
        st.close()
        st = make_state(P, ctx, mpo, chi, caps, seed)
        for k in range(args.warmup):
            st.update(centre + k, +1, mixed)
        torch.cuda.synchronize(dev)
        torch.cuda.cudart().cudaProfilerStart()
        e, trunc = st.update(centre + args.warmup, +1, mixed)
        torch.cuda.synchronize(dev)
        torch.cuda.cudart().cudaProfilerStop()
        print(json.dumps({"profile_update": True, "chi": chi, "energy": e, "discarded_weight": trunc,
                          "phase_ms": st.phase_ms(), "svd_stats": st.svd_stats(), "lanczos_stats": st.stats()}))
        st.close()
        return 0

    def barrier():
        ranks_barrier(dist)

    def max_over_ranks(x):
        return ranks_max(x, dist, dev)

    # ---- accuracy: mixed form vs converged FP64 reference of the same first H_eff
    ref_state = make_state(P, ctx, mpo, chi, caps, seed)
    e_ref, _ = ref_state.update(centre, +1, P.DMRG.params(chi, 1e-14, 30, 1e-13, PREC["bf16x3"], 60, 1e-15,
                                                          refine_prec=PREC["fp64"]))
    ref_state.close()

    # ---- warm-up pass over every site of the timed updates on a throwaway state: the tile
    # autotuner times its candidates once per problem class (precision, log2 |theta|, log2
    # tasks) and keeps only the chosen configuration, so the timed updates hold no tuning
    # launches but still do all their work
    st = make_state(P, ctx, mpo, chi, caps, seed)
    for k in range(args.warmup + args.steps):
        st.update(centre + k, +1, mixed)
    st.close()

    # ---- timed mixed-precision updates (device resident)
    st = make_state(P, ctx, mpo, chi, caps, seed)
    energies = []
    for k in range(args.warmup):
        e, _ = st.update(centre + k, +1, mixed)
        energies.append(e)
    e_mixed_first = energies[0]
    torch.cuda.synchronize(dev)
    st.timing(True)
    barrier()
    phases = np.zeros(6)
    sweeps = np.zeros(2)
    svd_work = np.zeros(6)   # summed mrd_dmrg_svd_stats of the timed updates
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    launches0 = P.launch_count()
    t_wall = time.perf_counter()
    with ClockSampler(local) as clk:
        e0.record(stream)
        for k in range(args.steps):
            st.update(centre + args.warmup + k, +1, mixed)
            phases += np.array(st.phase_ms())
            sweeps += np.array(st.svd_sweeps())
            svd_work += np.array(st.svd_stats())
        e1.record(stream)
        torch.cuda.synchronize(dev)
    t_wall = time.perf_counter() - t_wall
    launches = P.launch_count() - launches0
    barrier()
    kms, kn = st.timing(False)
    ms_total = max_over_ranks(e0.elapsed_time(e1))
    trunc = st.stats()[1]
    st.close()
    s_per_update = per_update_value(ms_total / 1e3, args.steps, world)

    # ---- e2e: the two site tensors of every step come from pinned host memory and the updated
    # tensors go back to the host, through the public API
    st = make_state(P, ctx, mpo, chi, caps, seed)
    for k in range(args.warmup):
        st.update(centre + k, +1, mixed)
    # one pinned host buffer per site of the timed steps, holding that site's current tensor
    i0 = centre + args.warmup
    nmax = max(st.site_len(j) for j in range(n_sites))
    hsite = {j: torch.empty(2 * nmax, dtype=torch.complex128).pin_memory() for j in range(i0, i0 + args.steps + 1)}
    for j in hsite:
        st.site_into(j, hsite[j])
    torch.cuda.synchronize(dev)
    barrier()
    h2d = d2h = 0
    t_e2e = time.perf_counter()
    for k in range(args.steps):
        i = i0 + k
        h2d += 16 * (st.site_len(i) + st.site_len(i + 1))
        st.set_site(i, hsite[i].data_ptr())
        st.set_site(i + 1, hsite[i + 1].data_ptr())
        st.update(i, +1, mixed)
        d2h += 16 * st.site_into(i, hsite[i])
        d2h += 16 * st.site_into(i + 1, hsite[i + 1])
    torch.cuda.synchronize(dev)
    t_e2e = max_over_ranks(time.perf_counter() - t_e2e)
    st.close()
    e2e_value = per_update_value(t_e2e, args.steps, world)

    # ---- FP64 form at the same accuracy (restarted Lanczos until the Ritz value settles)
    st = make_state(P, ctx, mpo, chi, caps, seed)
    fp64 = P.DMRG.params(chi, 1e-14, 30, 1e-12, PREC["fp64"], 0, 1e-14, restarts=6)
    st.timing(True)
    t64 = time.perf_counter()
    e_fp64 = None
    for k in range(args.fp64_steps):
        e, _ = st.update(centre + k, +1, fp64)
        if k == 0:
            e_fp64 = e
    torch.cuda.synchronize(dev)
    t64 = (time.perf_counter() - t64) / args.fp64_steps
    st.timing(False)
    fp64_matvecs = st.stats()[2]
    st.close()

    # ---- H_eff throughput per precision (Lx = 20 mid-ring sites, random environments)
    mv = matvec_throughput(P, ctx, torch, dev, stream)
    rvm = real_vs_mixed_or_note(P, ctx, torch, dev, stream)

    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return 0

    bf16_peak, bf16_sust, peak_src = measured_peaks()
    tc_ms, hp_ms = kms[0] + kms[1], kms[2] + kms[3]   # tensor-core and float-float H_eff GEMMs
    svd_ms = svd_work[0] + svd_work[4]                 # Jacobi rounds
    f_exec = mv["flops_executed"]
    # the dominant kernel of the timed updates by GPU time
    shares = {"k_svd_bround (Jacobi rounds)": svd_ms, "k_tc_gemm (Lanczos matvecs)": tc_ms,
              "k_cgemm_ff (refinement matvecs)": hp_ms}
    dominant = max(shares, key=shares.get)
    if dominant.startswith("k_svd_bround"):
        # float-float Jacobi: FP32 instructions of the work done (per element of a tested pair:
        # 4 float-float multiply-adds of 12 instructions; per element of a rotated pair: 4
        # exact products of 3, 8 multiply-adds of 11 and 4 FastTwoSums of 3; the rotated
        # norms are per pair, not per element), against the FP32 issue rate
        instr = svd_work[1] * 48 + svd_work[2] * 112
        ach = instr / (svd_work[0] / 1e3) / 1e12
        roof = {"kernel": "k_svd_bround<float-float> (block-cyclic Jacobi rounds)", "bound": "alu", "achieved": ach,
                "peak": FP32_ISSUE_TINSTR, "unit": "T FP32-instr/s", "frac": ach / FP32_ISSUE_TINSTR,
                "traffic": None, "peak_source": "128 FP32 lanes/SM x 152 SMs x 2.07 GHz (derived from unit counts and the maximum SM clock)",
                "ms_per_step": svd_work[0] / args.steps, "share_of_measured_kernels": svd_ms / sum(shares.values())}
    elif dominant.startswith("k_tc_gemm"):
        per = tc_ms / max(kn[0], 1) / 1e3
        hw = 3 * f_exec / per / 1e12
        roof = {"kernel": "k_tc_gemm BF16X3 (steps 1+2)", "bound": "tensor", "achieved": hw, "peak": bf16_sust,
                "unit": "TFLOP/s", "frac": hw / bf16_sust, "traffic": None, "peak_source": f"bf16 sustained {peak_src}",
                "ms_per_step": tc_ms / args.steps, "share_of_measured_kernels": tc_ms / sum(shares.values())}
    else:
        per = hp_ms / max(kn[1], 1) / 1e3
        ach = f_exec / 8 * FF_INSTR_PER_CMAC / per / 1e12
        roof = {"kernel": "k_cgemm_ff (float-float refinement matvec, steps 1+2)", "bound": "alu", "achieved": ach,
                "peak": FP32_ISSUE_TINSTR, "unit": "T FP32-instr/s", "frac": ach / FP32_ISSUE_TINSTR,
                "traffic": None, "peak_source": "128 FP32 lanes/SM x 152 SMs x 2.07 GHz (derived from unit counts and the maximum SM clock)",
                "ms_per_step": hp_ms / args.steps, "share_of_measured_kernels": hp_ms / sum(shares.values())}
    tc = mv["bf16x3"]
    tc_hw = 3 * f_exec / (tc["ms"] / 1e3) / 1e12
    tf = mv["tf32"]
    tf_hw = f_exec / (tf["ms"] / 1e3) / 1e12
    line = {
        "metric": METRIC, "value": s_per_update, "unit": "s/update", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_total / args.steps, "higher_is_better": False, "scaling": "weak",
        "vs_baseline": None, "dtype": "bf16x3+f32x2", "data": "synthetic",
        "config": {"workload": workload_name(chi), "chi": chi, "ly": LY, "lx": LX_UPDATE,
                   "form": f"split-BF16 tensor-core Lanczos (60 per run, up to {args.fast_restarts} restarts) + "
                           f"float-float Rayleigh-quotient refinement ({args.refine} matvec), block SVD by "
                           f"FP32 pre-sweeps + float-float Jacobi sweeps, float-float environment update",
                   "l2": "working set > L2 (folded environments, Z intermediate and Lanczos basis, >1 GB)",
                   "parallelism": f"replicas x{world}"},
        "s_per_update_fp64": t64,
        "fp64_form_matvecs": fp64_matvecs,
        "speedup_vs_fp64": t64 / (ms_total / 1e3 / args.steps),
        "dE_rel_mixed_vs_converged_fp64": abs(e_mixed_first - e_ref) / abs(e_ref),
        "dE_rel_fp64_form_vs_converged_fp64": abs(e_fp64 - e_ref) / abs(e_ref),
        "energy_first_update": {"mixed": e_mixed_first, "fp64_form": e_fp64, "converged_fp64": e_ref},
        "discarded_weight_last": trunc,
        "phase_ms_mean": dict(zip(["tables", "theta", "lanczos+refine", "svd", "tensors", "env"],
                                  (phases / args.steps).round(2).tolist())),
        "svd_jacobi_rounds_mean": dict(zip(["fp32", "fp64"], (sweeps / args.steps).round(1).tolist())),
        "kernel_ms_per_step": {k: round(v / args.steps, 3) for k, v in shares.items()},
        "svd_elem_pairs_per_step": {"tested": svd_work[1] / args.steps, "rotated": svd_work[2] / args.steps},
        "heff_tflops": {k: round(mv[k]["tflops"], 3) for k in PREC},
        "heff_ms": {k: round(mv[k]["ms"], 4) for k in PREC},
        "heff_ms_steps": {k: [round(mv[k]["ms_step1"], 4), round(mv[k]["ms_step2"], 4)] for k in PREC},
        "heff_tile_config": {k: mv[k].get("tile_config") for k in ("tf32", "bf16x3")},
        "heff_bf16x3_ms_grouped_vs_per_task": [round(mv["bf16x3"]["ms"], 4),
                                               round(mv["bf16x3"]["ms_per_task_launches"], 3)],
        "heff_flops": {"definition": mv["flops_definition"], "executed": mv["flops_executed"]},
        "real_vs_mixed_heff": rvm,
        "mpo_diagnostics": mpo_diagnostics(P),
        "roofline": roof,
        "roofline_tc_bf16x3": {"kernel": "k_tc_gemm BF16X3 (steps 1+2), Lx=20 matvec", "bound": "tensor",
                               "achieved": tc_hw, "peak": bf16_peak, "unit": "TFLOP/s", "frac": tc_hw / bf16_peak,
                               "traffic": None, "note": "hardware bf16 flops = 3 x executed complex-product flops "
                                                        f"(split), peak = bf16 burst {peak_src}"},
        "roofline_ff_gemm": {"kernel": "k_cgemm_ff (steps 1+2), Lx=20 matvec", "bound": "alu",
                             "achieved": f_exec / 8 * FF_INSTR_PER_CMAC / (mv["ff"]["ms"] / 1e3) / 1e12, "peak": FP32_ISSUE_TINSTR,
                             "unit": "T FP32-instr/s",
                             "frac": f_exec / 8 * FF_INSTR_PER_CMAC / (mv["ff"]["ms"] / 1e3) / 1e12 / FP32_ISSUE_TINSTR,
                             "traffic": None, "note": "36 FP32 instructions per complex multiply-add (3 float-float products of 12)"},
        "roofline_tc_tf32": {"kernel": "k_tc_gemm TF32 (steps 1+2), Lx=20 matvec", "bound": "tensor",
                             "achieved": tf_hw, "peak": bf16_peak / 2, "unit": "TFLOP/s",
                             "frac": tf_hw / (bf16_peak / 2), "traffic": None,
                             "note": f"TF32 peak = bf16 burst {peak_src} x 1/2 (nominal ratio)"},
        "e2e": {"value": e2e_value, "unit": "s/update", "h2d_bytes_per_step": h2d // args.steps,
                "d2h_bytes_per_step": d2h // args.steps},
        "gpu_launches": launches,
        "clocks": clk.summary(),
        "wall_s_timed": t_wall,
    }
    if world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline()
    print(json.dumps(line))
    if dist is not None:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
