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


def small_profile_caps(lx, chi):
    """Bond caps of the small-footprint profiling state: the synthetic sectors at chi on the
    bonds from 4 left to 12 right of the centre (the profiled updates' bonds, with room for the
    ranks the right end allows), halved per further bond (floor 512), so that the state and its
    environments hold a few GB instead of tens."""
    n, i = lx * LY, update_centre(lx)
    def cap(j):
        dist = 0 if i - 4 <= j <= i + 12 else (i - 4 - j if j < i else j - (i + 12))
        c = chi if dist == 0 else max(512, chi >> dist)
        return [(q[0], q[1], d) for q, d in synth.bond_sectors(c, LY, round(j / LY), synth.substream(SEED, 7, j),
                                                               min_dim=4 if c == chi else 1)]
    return [cap(j) if 2 <= j <= n - 2 else [] for j in range(n + 1)]


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


def oracle_full_update_ly8(chi=1024, matvecs=ORACLE_MATVECS):
    """Seconds of one complete oracle two-site update (oracle.blocksparse.two_site_update:
    Lanczos with `matvecs` block-sparse H_eff applications, block SVD, truncation, new left
    environment) on the Ly = 8 cylinder at chi = 1024 (flux 1/8, t = V = 1, Lx = 16, the centre
    sites), with the oracle's MPO and seeded random environments and theta of those shapes."""
    from oracle import blocksparse as B
    from oracle import dmrg as D
    from oracle import mpo as M
    ly, lx, seed = 8, 16, 1234 + 1
    n = lx * ly
    site = (lx // 2) * ly + ly // 2 - 1
    caps = {j: synth.bond_sectors(chi, ly, round(j / ly), synth.substream(seed, 7, j)) for j in (site, site + 2)}
    mp = M.build_mpo(lx, ly, 1 / 8, T_HOP, V_INT, "mixed")
    left, right = B.BondSectors(caps[site]), B.BondSectors(caps[site + 2])
    m1, m2 = site % ly, (site + 1) % ly
    cl, cm, cr = mp.bond_charges[site], mp.bond_charges[site + 1], mp.bond_charges[site + 2]
    lay = B.theta_layout(left, right, m1, m2, ly)
    s = synth.substream(seed, 200)
    lflat = synth.complex_pm1(synth.substream(s, 8), B.env_size(B.env_left_layout(left, cl, ly)))
    rflat = synth.complex_pm1(synth.substream(s, 9), B.env_size(B.env_right_layout(right, cr, ly)))
    tflat = synth.complex_pm1(synth.substream(s, 10), B.theta_size(lay))
    # a fixed number of Lanczos steps (random environments: the stopping rule plays no part)
    lz = lambda mv, v0: D.lanczos_ground(mv, v0, kmax=matvecs, tol=0.0)
    t0 = time.perf_counter()
    out = B.two_site_update(left, right, m1, m2, ly, cl, cm, cr, mp.entries[site], mp.entries[site + 1], lflat, rflat,
                            tflat, chi, lanczos=lz)
    return time.perf_counter() - t0, out["matvecs"], n


def cpu_baseline(n_steps=3):
    step, flops, full = oracle_step_factory()
    step()
    times = [step() for _ in range(n_steps)]
    t = statistics.median(times)
    t8, mv8, _ = oracle_full_update_ly8()
    return {"value": oracle_s_per_update(t, flops, full), "unit": "s/update", "cores": len(os.sched_getaffinity(0)),
            "kind": "oracle", "sample": oracle_sample_text(flops, full, t) + f"; median of {n_steps} after 1 warm-up",
            "full_update_ly8_chi1024_s": t8, "full_update_ly8_matvecs": mv8,
            "full_update_note": "one complete oracle update (Lanczos, block SVD, truncation, environment) at Ly=8 "
                                "chi=1024, timed as it is"}


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
    free, total = torch.cuda.mem_get_info(dev)   # device memory in use with the H_eff built
    res["device_used_gb"] = (total - free) / 1e9
    h.close()
    return res


def real_vs_mixed(P, ctx, torch, dev, stream):
    """The paper's comparison of the two bases (Sec. III.B, Fig. 3) on the library's own code:
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


def real_arithmetic_update(P, ctx, torch, dev, stream, chi, steps, warmup, refine=1, restarts=8):
    """The timed update in real arithmetic (Sec. IV.D, Eq. rot): the sine / cosine MPO of the same
    cylinder, real site tensors and environments (MRD_DMRG_OPT_REAL), real tensor-core and
    float-float GEMMs. Timed like the complex form (a tuning pass over the same sites on a
    throwaway state, then device-resident updates between CUDA events), gated against the FP64
    form converged on the same real state. Flops: a real multiply-add is 2 definition flops (8 for
    a complex one) and 4 BF16 products on the tensor cores."""
    mpo = P.MPO(None, LX_UPDATE, LY, FLUX_P, FLUX_Q, T_HOP, V_INT, P.MRD_BASIS_MIXED_REAL)
    caps = update_caps(LX_UPDATE, chi)
    centre = update_centre(LX_UPDATE)
    form = mixed_params(P, chi, refine, restarts)

    def state():
        st = make_state(P, ctx, mpo, chi, caps, replica_seed(0))
        st.set_option(P.MRD_DMRG_OPT_REAL, 1)
        return st

    st = state()
    e_ref, _ = st.update(centre, +1, fp64_params(P, chi, tol=1e-14, restarts=8))
    st.close()
    st = state()
    for k in range(warmup + steps):
        st.update(centre + k, +1, form)
    st.close()
    st = state()
    e_first = None
    for k in range(warmup):
        e, _ = st.update(centre + k, +1, form)
        e_first = e if e_first is None else e_first
    torch.cuda.synchronize(dev)
    st.timing(True)
    bonds, counts = [], []
    phases = np.zeros(6)
    svd_ms = 0.0
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for k in range(steps):
        i = centre + warmup + k
        bonds.append((i, st.bond(i), st.bond(i + 2)))
        st.update(i, +1, form)
        counts.append(st.stats()[2])
        phases += np.array(st.phase_ms())
        ss = st.svd_stats()
        svd_ms += ss[0] + ss[4]
    e1.record(stream)
    torch.cuda.synchronize(dev)
    ms = e0.elapsed_time(e1)
    kms, _ = st.timing(False)
    real_tensors = all(np.all(st.site(j)[1].imag == 0.0) for j in range(centre, centre + warmup + steps + 1))
    st.close()
    f_def = f_exec = 0.0
    n_tc = 0
    for (i, lb, rb), cnt in zip(bonds, counts):
        h = heff_of_bonds(P, ctx, mpo, i, lb, rb)
        fd, fe, _, _ = h.flops()
        h.close()
        f_def += fd / 4 * (cnt % 1000)
        f_exec += fe / 4 * (cnt % 1000)
        n_tc += cnt % 1000
    mpo.close()
    tc_ms, ff_ms = kms[0] + kms[1], kms[2] + kms[3]
    dE = abs(e_first - e_ref) / abs(e_ref)
    return {"s_per_update": ms / 1e3 / steps, "steps": steps,
            "basis": "mixed sine/cosine (Eq. rot), real tensors", "dE_rel_vs_fp64_converged": dE,
            "gate_passed": dE <= 1e-9, "site_tensors_real": bool(real_tensors),
            "heff_tflops_bf16x3_real": f_def / (tc_ms / 1e3) / 1e12 if tc_ms > 0 else None,
            "heff_hw_tflops": 4 * f_exec / (tc_ms / 1e3) / 1e12 if tc_ms > 0 else None,
            "kernel_ms_per_update": {"k_tc_gemm": tc_ms / steps, "k_cgemm_ff": ff_ms / steps,
                                     "k_svd_bround": svd_ms / steps},
            "phase_ms_mean": dict(zip(["tables", "theta", "lanczos+refine", "svd", "tensors", "env"],
                                      (phases / steps).round(2).tolist())),
            "heff_applications": n_tc, "e_fp64_converged": e_ref, "e_first": e_first}


def mpo_diagnostics(P):
    """Mean and largest MPO bond dimension and mean fill over a bulk ring (the second of three),
    real-space, mixed (exponential) and mixed sine / cosine machines, against the real-space
    3L + 2 (Sec. IV.C-D, Eq. rot). Host only."""
    out = {}
    for ly in (4, 6, 8, 10, 12):
        row = {"3L+2": 3 * ly + 2}
        for name, basis in (("real", P.MRD_BASIS_REAL), ("mixed", P.MRD_BASIS_MIXED),
                            ("mixed_sin_cos", P.MRD_BASIS_MIXED_REAL)):
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


def make_state(P, ctx, mpo, chi, caps, seed, lx=None, center=None):
    lx = LX_UPDATE if lx is None else lx
    return P.DMRG(ctx, mpo, lx, 0, chi, seed=seed, center=update_centre(lx) if center is None else center, caps=caps)


def mixed_params(P, chi, refine=1, restarts=8, refine_prec=None, svd_mode=None, prec=None):
    """The benchmarked reduced-precision form: split-BF16 tensor-core Lanczos (60 steps per run,
    restarted while the Ritz value moves by more than 1e-10), the ground vector refined with
    float-float matvecs, FP32 + float-float Jacobi SVD, float-float environments."""
    return P.DMRG.params(chi, 1e-14, 60, 1e-10, PREC["bf16x3"] if prec is None else prec, refine, 1e-13,
                         restarts=restarts, svd_mode=svd_mode, refine_prec=refine_prec)


def fp64_params(P, chi, tol=1e-12, restarts=6):
    """The plain FP64 form: FP64 Lanczos restarted until the Ritz value settles to tol, FP64
    Jacobi SVD, FP64 environments."""
    return P.DMRG.params(chi, 1e-14, 30, tol, PREC["fp64"], 0, 1e-14, restarts=restarts)


def heff_of_bonds(P, ctx, mpo, i, left, right):
    """The H_eff handle of an update of sites (i, i+1) whose outer bonds have these sectors
    (no environments: used for its tables and flop counts)."""
    ly = mpo.modulus if mpo.modulus > 1 else 1
    i_idx, i_val = mpo.site(i)
    j_idx, j_val = mpo.site(i + 1)
    return P.Heff(ctx, left, right, i % ly if ly > 1 else 0, (i + 1) % ly if ly > 1 else 0, mpo.modulus,
                  mpo.bond(i), mpo.bond(i + 1), mpo.bond(i + 2), i_idx, i_val, j_idx, j_val)


def traffic_from_profile(kernel_sources):
    """DRAM bytes per H_eff application of the tensor-core GEMM from the committed ncu summary,
    if that summary was taken from the current sources (hash of the kernel files), else None."""
    import hashlib
    import re
    path = os.path.join(ROOT, "profiles", "k_tc_gemm_bf16x3_ly10_chi3200_dram.md")
    try:
        text = open(path).read()
    except OSError:
        return None, "no ncu summary"
    h = hashlib.sha256()
    for f in kernel_sources:
        h.update(open(os.path.join(ROOT, f), "rb").read())
    m_sha = re.search(r"sources sha256: ([0-9a-f]{16})", text)
    m_b = re.search(r"DRAM bytes per H_eff application: ([0-9.e+]+)", text)
    if not m_sha or not m_b:
        return None, "summary without figures"
    if m_sha.group(1) != h.hexdigest()[:16]:
        return None, "kernel changed since the ncu capture"
    return float(m_b.group(1)), path


def ly8_forms(P, ctx, torch, dev, details):
    """Workloads on the Ly = 8 cylinder (flux 1/8, t = V = 1, one particle per ring, Lx = 16,
    the centre bond): at chi = 1024 the plain FP64 form (s per update) and the FP64 H_eff
    against the oracle on sampled output blocks; at chi = 2048 the raw matvec error of TF32 and
    split BF16 against the FP64 H_eff on the same operands, and the first update's energy of
    each reduced-precision form (refined) against the converged plain FP64 form."""
    from oracle import blocksparse as B
    ly, lx = 8, 16
    mpo = P.MPO(None, lx, ly, 1, 8, T_HOP, V_INT, P.MRD_BASIS_MIXED)
    c = (lx // 2) * ly + ly // 2 - 1
    n = lx * ly
    out = {}
    for chi, seed in ((1024, 1234 + 1), (2048, 1234 + 2)):
        caps = [[(q[0], q[1], d) for q, d in synth.bond_sectors(chi, ly, round(j / ly), synth.substream(seed, 7, j))]
                if 2 <= j <= n - 2 else [] for j in range(n + 1)]
        res = {}
        # matvec on seeded random operands of the update's shapes
        left = np.array(caps[c], dtype=np.int32)
        right = np.array(caps[c + 2], dtype=np.int32)
        h = heff_of_bonds(P, ctx, mpo, c, left, right)
        s = synth.substream(seed, 100)
        L = torch.from_numpy(synth.complex_pm1(synth.substream(s, 8), h.lenv_len)).to(dev)
        R = torch.from_numpy(synth.complex_pm1(synth.substream(s, 9), h.renv_len)).to(dev)
        T = torch.from_numpy(synth.complex_pm1(synth.substream(s, 10), h.theta_len)).to(dev)
        h.set_env(L, R)
        o64 = torch.empty_like(T)
        h.apply(T, o64, PREC["fp64"])
        ref = o64.cpu().numpy()
        scale = float(np.max(np.abs(ref)))
        res["heff_flops_definition"] = h.flops()[0]
        if chi == 1024:
            # sampled output blocks against the oracle (the blocks of the two largest left sectors)
            lb = B.BondSectors([((int(a), int(b)), int(d)) for a, b, d in left])
            rb = B.BondSectors([((int(a), int(b)), int(d)) for a, b, d in right])
            i_idx, i_val = mpo.site(c)
            j_idx, j_val = mpo.site(c + 1)
            wi = [(int(a), int(b), int(x), int(y), complex(v)) for (a, b, x, y), v in zip(i_idx, i_val)]
            wj = [(int(a), int(b), int(x), int(y), complex(v)) for (a, b, x, y), v in zip(j_idx, j_val)]
            ch = lambda b: [(int(x), int(y) % ly) for x, y in mpo.bond(b)]
            args = (lb, rb, c % ly, (c + 1) % ly, ly, ch(c), ch(c + 1), ch(c + 2), wi, wj)
            flats = (synth.complex_pm1(synth.substream(s, 8), h.lenv_len),
                     synth.complex_pm1(synth.substream(s, 9), h.renv_len), T.cpu().numpy())
            lay = B.theta_layout(lb, rb, c % ly, (c + 1) % ly, ly)
            big = set(np.argsort(lb.dims)[-2:].tolist())
            err = 0.0
            for m in lay:
                blk = ref[m["offset"]: m["offset"] + m["rowdim"] * m["coldim"]].reshape(m["rowdim"], m["coldim"])
                for s1p, api, dap, ro in m["rows"]:
                    if api not in big:
                        continue
                    for s2p, bpi, dbp, co in m["cols"]:
                        want = B.heff_apply_block(*args, *flats, (api, s1p, s2p))
                        err = max(err, float(np.max(np.abs(blk[ro:ro + dap, co:co + dbp] - want))))
            res["heff_fp64_rel_err_vs_oracle_sampled"] = err / scale
        else:
            for name in ("tf32", "bf16x3"):
                o = torch.empty_like(T)
                h.apply(T, o, PREC[name])
                res[f"heff_{name}_rel_err_vs_fp64"] = float(np.max(np.abs(o.cpu().numpy() - ref))) / scale
        h.close()
        del L, R, T, o64
        # plain FP64 form, converged reference and timed form
        st = make_state(P, ctx, mpo, chi, caps, 11, lx=lx, center=c)
        e_ref, _ = st.update(c, +1, fp64_params(P, chi, tol=1e-14, restarts=8))
        st.close()
        st = make_state(P, ctx, mpo, chi, caps, 11, lx=lx, center=c)
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        e64, _ = st.update(c, +1, fp64_params(P, chi))
        torch.cuda.synchronize(dev)
        res["s_per_update_fp64"] = time.perf_counter() - t0
        res["dE_rel_fp64_form"] = abs(e64 - e_ref) / abs(e_ref)
        st.close()
        if chi == 2048:
            # TF32: the float-float polish runs up to 40 matvecs (it stops once the Ritz value
            # settles); 20 left 2.6e-9 on this H_eff, 40 reach 2e-12
            forms = {"bf16x3+ff": mixed_params(P, chi), "tf32+ff": mixed_params(P, chi, refine=40, prec=PREC["tf32"]),
                     "bf16x3+fp64": mixed_params(P, chi, refine_prec=PREC["fp64"], svd_mode=P.MRD_SVD_F32_F64)}
            for name, prm in forms.items():
                st = make_state(P, ctx, mpo, chi, caps, 11, lx=lx, center=c)
                st.update(c, +1, prm)            # tuning pass for this problem class
                st.close()
                st = make_state(P, ctx, mpo, chi, caps, 11, lx=lx, center=c)
                torch.cuda.synchronize(dev)
                t0 = time.perf_counter()
                e, _ = st.update(c, +1, prm)
                torch.cuda.synchronize(dev)
                res[f"form_{name}"] = {"s_per_update": time.perf_counter() - t0, "dE_rel_vs_fp64": abs(e - e_ref) / abs(e_ref)}
                st.close()
        res["energy_fp64_converged"] = e_ref
        out[f"chi{chi}"] = res
    details["ly8"] = out
    return out


def free_fermion_k(lx, ly, flux, n, t=T_HOP):
    """Momentum sector (sum of the occupied m mod Ly) of the free-fermion ground state of the
    cylinder (Eq. H_kin: per momentum k_m the Lx x Lx tridiagonal with diagonal
    -2t cos(k_m + x phi) and off-diagonal -t); the interacting ground state is taken in it."""
    lev = []
    for m in range(ly):
        k = 2 * np.pi * m / ly
        h = np.diag([-2 * t * np.cos(k + x * 2 * np.pi * flux) for x in range(lx)])
        h += np.diag([-t] * (lx - 1), 1) + np.diag([-t] * (lx - 1), -1)
        lev += [(e, m) for e in np.linalg.eigvalsh(h)]
    lev.sort()
    return sum(m for _, m in lev[:n]) % ly


def sweeps_mixed_vs_real(P, ctx, torch, dev, chi=1024, lx=16, ly=8, max_sweeps=14, tol=1e-8, chi0=128):
    """The paper's basis comparison (Sec. III.B, Fig. 3(c, d)) on the library's own code: finite
    two-site DMRG sweeps from a seeded random MPS to convergence on the Ly = 8 interacting
    Hofstadter cylinder (flux 1/8, t = V = 1, one particle per ring), in the mixed basis
    (charges N, K; K of the free-fermion ground state) and in real space (charge N only), both
    in the benchmarked reduced-precision form. The kept bond dimension doubles every sweep from
    chi0 up to chi, then sweeps repeat until the sweep energy changes by less than tol
    (relative), at most max_sweeps. Reports the time per sweep, the energies and the
    device-memory high-water mark: total minus the least free memory seen after any sweep,
    the library's cache released before each basis (the cache keeps what a run allocated, so
    this includes its transient buffers)."""
    out = {}
    kk = free_fermion_k(lx, ly, 1 / 8, lx)
    for name, basis in (("mixed", P.MRD_BASIS_MIXED), ("real", P.MRD_BASIS_REAL)):
        ctx.release_cached()
        torch.cuda.synchronize(dev)
        free0, total = torch.cuda.mem_get_info(dev)
        mpo = P.MPO(None, lx, ly, 1, 8, T_HOP, V_INT, basis)
        st = P.DMRG(ctx, mpo, lx, kk if basis == P.MRD_BASIS_MIXED else 0, chi, seed=21, center=0)
        free_min = torch.cuda.mem_get_info(dev)[0]
        es, times, chis = [], [], []
        c = chi0
        for _ in range(max_sweeps):
            torch.cuda.synchronize(dev)
            t0 = time.perf_counter()
            es.append(st.sweep(mixed_params(P, c)))
            torch.cuda.synchronize(dev)
            times.append(time.perf_counter() - t0)
            chis.append(c)
            free_min = min(free_min, torch.cuda.mem_get_info(dev)[0])
            if c == chi and len(es) > 1 and chis[-2] == chi and abs(es[-1] - es[-2]) < tol * abs(es[-1]):
                break
            c = min(chi, 2 * c)
        full = [t for t, x in zip(times, chis) if x == chi]
        out[name] = {"energies": es, "chi_per_sweep": chis, "s_per_sweep": times, "sweeps": len(es),
                     "converged": len(full) > 1 and abs(es[-1] - es[-2]) < tol * abs(es[-1]),
                     "s_per_sweep_at_chi": sum(full) / max(len(full), 1), "s_total": sum(times),
                     "mem_high_water_gb": (free0 - free_min) / 1e9,
                     "max_bond": int(max(st.bond(b)[:, 2].sum() for b in range(1, lx * ly)))}
        st.close()
        mpo.close()
    m, r = out["mixed"], out["real"]
    out["ratio_real_over_mixed"] = {"s_per_sweep_at_chi": r["s_per_sweep_at_chi"] / m["s_per_sweep_at_chi"],
                                    "s_total": r["s_total"] / m["s_total"],
                                    "mem_high_water": r["mem_high_water_gb"] / max(m["mem_high_water_gb"], 1e-9)}
    out["dE_rel_real_vs_mixed"] = abs(r["energies"][-1] - m["energies"][-1]) / abs(m["energies"][-1])
    out["workload"] = (f"Ly={ly} Lx={lx} flux=1/8 t=1 V=1 N={lx} K={kk}, chi {chi0}->{chi}, split-BF16 Lanczos + "
                       f"float-float refinement, FP32 + float-float SVD, float-float environments")
    return out


def config5(P, ctx, torch, dev, chi=8000, ly=12, lx=24, fp64_matvecs=53):
    """The memory-bound scale: the Ly = 12 cylinder (flux 1/6, t = V = 1, the lowest band
    filled: 2 particles per ring), chi = 8000 at the centre bonds, environments stored in
    complex64 (MRD_DMRG_OPT_ENV_FP32). A 24-ring cylinder whose bonds carry the synthetic
    sectors at chi within 6 bonds of the centre and half as many per further bond (floor 512, so
    that the state and its environments can be built in seconds) holds one
    two-site update with chi = 8000 on both outer bonds of its H_eff. Reported: seconds of that
    update in the benchmarked reduced-precision form, the split-BF16 H_eff TFLOP/s inside it,
    the HBM GB/s of one environment update (complex64 in and out), the device memory of the
    state, the byte estimate of all environments of a 24-ring cylinder at this bond dimension
    in complex64 and complex128 against the device, and the plain FP64 H_eff matvec time
    (times the FP64 form's matvec count at chi = 3200: an estimate of its update time)."""
    seed5 = 1234 + 4
    n = lx * ly
    i = (lx // 2) * ly + ly // 2 - 1
    def cap(j):   # the synthetic sectors at chi within 6 bonds of the update, halving beyond (floor 512)
        dist = 0 if i <= j <= i + 2 else (i - j if j < i else j - (i + 2))
        c = chi if dist <= 6 else max(512, chi >> (dist - 6))
        return [(q[0], q[1], d) for q, d in synth.bond_sectors(c, ly, round(2 * j / ly), synth.substream(seed5, 7, j),
                                                               min_dim=4 if c == chi else 1)]
    caps = [cap(j) if 2 <= j <= n - 2 else [] for j in range(n + 1)]
    mpo = P.MPO(None, lx, ly, 1, 6, T_HOP, V_INT, P.MRD_BASIS_MIXED)
    out = {"workload": f"Ly={ly} Lx={lx} flux=1/6 t=1 V=1 N={2 * lx}, chi={chi} at the centre bonds, env complex64"}
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    st = P.DMRG(ctx, mpo, 2 * lx, 0, chi, seed=seed5, center=i, caps=caps)
    st.set_option(P.MRD_DMRG_OPT_ENV_FP32, 1)
    torch.cuda.synchronize(dev)
    out["state_build_s"] = time.perf_counter() - t0
    prm = mixed_params(P, chi)
    st.update(i, +1, prm)                       # tile tuning for this problem class
    lb, rb = st.bond(i + 1), st.bond(i + 3)
    out["bond_dims"] = [int(lb[:, 2].sum()), int(rb[:, 2].sum())]
    st.timing(True)
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    e, trunc = st.update(i + 1, +1, prm)
    torch.cuda.synchronize(dev)
    out["s_per_update"] = time.perf_counter() - t0
    kms, kn = st.timing(False)
    out["phase_ms"] = dict(zip(["tables", "theta", "lanczos+refine", "svd", "tensors", "env"],
                               np.round(st.phase_ms(), 1).tolist()))
    cnt = st.stats()[2]
    h = heff_of_bonds(P, ctx, mpo, i + 1, lb, rb)
    fd, fe, _, _ = h.flops()
    theta_len, lenv_len, renv_len = h.theta_len, h.lenv_len, h.renv_len
    h.close()
    ntc = cnt % 1000
    out["heff_flops_definition"] = fd
    out["heff_tflops_bf16x3"] = fd * ntc / (kms[0] + kms[1]) / 1e9 if kms[0] + kms[1] > 0 else None
    out["heff_bf16x3_ms"] = (kms[0] + kms[1]) / max(ntc, 1)
    out["theta_elems"] = theta_len
    # one environment update in complex64 storage: read L (8 B), the site tensor (16 B), write L'
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    st.env_update(i + 1, +1, PREC["ff"])
    torch.cuda.synchronize(dev)
    t_env = time.perf_counter() - t0
    l_in, l_out, a_len = lenv_len, st.env_len(i + 2, 0), st.site_len(i + 1)
    env_bytes = 8 * (l_in + l_out) + 16 * a_len
    out["env_update_ms"] = 1e3 * t_env
    out["env_update_gbs"] = env_bytes / t_env / 1e9
    mem = st.memory()
    out["state_memory_gb"] = {"environments": mem[0] / 1e9, "environments_built": mem[1], "mps": mem[2] / 1e9}
    # byte estimate of the environments a finite sweep holds on the 24-ring cylinder at this
    # bond dimension: one per bond (left ones left of the centre, right ones right of it), each
    # of the centre environment's size per MPO channel times its bond's MPO dimension
    d_c = len(mpo.bond(i + 1))
    per_channel = 8.0 * l_out / d_c
    env_all = sum(len(mpo.bond(j)) for j in range(1, n)) * per_channel
    free, total = torch.cuda.mem_get_info(dev)
    out["env_estimate_gb"] = {"complex64": env_all / 1e9, "complex128": 2 * env_all / 1e9,
                              "device_total": total / 1e9, "budget": 180.0,
                              "note": "one environment per bond of the 24-ring cylinder, sized by the centre "
                                      "environment per MPO channel times the bond's MPO dimension"}
    out["energy"], out["discarded_weight"] = e, trunc
    st.close()
    # plain FP64 H_eff on the same shapes (seeded random environments)
    h = heff_of_bonds(P, ctx, mpo, i + 1, lb, rb)
    s = synth.substream(seed5, 100)
    L = torch.from_numpy(synth.complex_pm1(synth.substream(s, 8), h.lenv_len)).to(dev)
    R = torch.from_numpy(synth.complex_pm1(synth.substream(s, 9), h.renv_len)).to(dev)
    T = torch.from_numpy(synth.complex_pm1(synth.substream(s, 10), h.theta_len)).to(dev)
    o = torch.empty_like(T)
    h.set_env(L, R)
    h.apply(T, o, PREC["fp64"])
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    h.apply(T, o, PREC["fp64"])
    torch.cuda.synchronize(dev)
    t64 = time.perf_counter() - t0
    h.close()
    del L, R, T, o
    out["fp64_matvec_s"] = t64
    out["fp64_form_s_per_update_estimate"] = t64 * fp64_matvecs
    out["speedup_vs_fp64_estimate"] = t64 * fp64_matvecs / out["s_per_update"]
    mpo.close()
    ctx.release_cached()
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=6)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--chi", type=int, default=CHI)
    ap.add_argument("--refine", type=int, default=1, help="float-float refinement matvecs of the mixed form")
    ap.add_argument("--fp64-steps", type=int, default=1)
    ap.add_argument("--fast-restarts", type=int, default=8, help="restarts of the reduced-precision Lanczos")
    ap.add_argument("--only-matvec", action="store_true", help="H_eff throughput only (profiling runs)")
    ap.add_argument("--precs", default="", help="with --only-matvec: comma-separated precisions (default all)")
    ap.add_argument("--profile-update", action="store_true",
                    help="warm-up updates, then one update inside a CUDA profiler range (ncu --profile-from-start off)")
    ap.add_argument("--small", action="store_true",
                    help="with --profile-update: the small-footprint state (full chi only near the centre)")
    ap.add_argument("--details", default="bench_details.json", help="file for the per-workload details")
    ap.add_argument("--quick", action="store_true", help="skip the side measurements (Ly = 8 forms, real vs mixed)")
    ap.add_argument("--sweeps", action="store_true",
                    help="only: converged sweeps in the mixed and the real-space basis (Ly = 8), one JSON line")
    ap.add_argument("--config5", action="store_true",
                    help="only: the Ly = 12, chi = 8000 update with complex64 environments, one JSON line")
    ap.add_argument("--sweeps-chi", type=int, default=1024)
    ap.add_argument("--sweeps-lx", type=int, default=16)
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
    mixed = mixed_params(P, chi, args.refine, args.fast_restarts)
    if args.only_matvec:
        set_chi(chi)
        precs = [p for p in args.precs.split(",") if p]
        mv = matvec_throughput(P, ctx, torch, dev, stream, precs=precs)
        done = [k for k in PREC if k in mv]
        print(json.dumps({"only_matvec": True, "chi": chi, "heff_tflops": {k: mv[k]["tflops"] for k in done},
                          "heff_ms_steps": {k: [mv[k]["ms_step1"], mv[k]["ms_step2"]] for k in done},
                          "device_used_gb": mv["device_used_gb"]}))
        return 0

    if args.config5:
        print(json.dumps({"config5": config5(P, ctx, torch, dev)}, default=float))
        return 0

    if args.sweeps:
        res = sweeps_mixed_vs_real(P, ctx, torch, dev, chi=args.sweeps_chi, lx=args.sweeps_lx)
        print(json.dumps({"sweeps_mixed_vs_real": res}))
        return 0

    if args.profile_update:
        if args.small:
            caps = small_profile_caps(LX_UPDATE, chi)
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
        t32, t64 = st.svd_trace()
        free, total = torch.cuda.mem_get_info(dev)   # the device memory in use (state, caches, context)
        print(json.dumps({"profile_update": True, "chi": chi, "small": args.small, "energy": e,
                          "device_used_gb": (total - free) / 1e9,
                          "discarded_weight": trunc, "bonds": [int(st.bond(centre + args.warmup)[:, 2].sum()),
                                                               int(st.bond(centre + args.warmup + 2)[:, 2].sum())],
                          "phase_ms": st.phase_ms(), "svd_stats": st.svd_stats(), "svd_sweeps": [len(t32), len(t64)],
                          "lanczos_stats": st.stats()}))
        st.close()
        return 0

    def barrier():
        ranks_barrier(dist)

    def max_over_ranks(x):
        return ranks_max(x, dist, dev)

    details = {}
    peaks = ctx.measure_peaks()   # FP32 / FP64 FMA instructions per second, SMs, clock
    fp32_peak = peaks[0] / 1e12

    # ---- accuracy reference: the plain FP64 form converged (FP64 Lanczos restarted to 1e-14,
    # FP64 Jacobi SVD) on the first timed H_eff (same state, same environments)
    ref_state = make_state(P, ctx, mpo, chi, caps, seed)
    e_ref, _ = ref_state.update(centre, +1, fp64_params(P, chi, tol=1e-14, restarts=8))
    ref_matvecs = ref_state.stats()[2]
    ref_state.close()

    # ---- warm-up pass over every site of the timed updates on a throwaway state: the tile
    # autotuner times its candidates once per problem class and keeps only the chosen
    # configuration, so the timed updates hold no tuning launches but still do all their work
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
    svd_work = np.zeros(8)   # summed mrd_dmrg_svd_stats of the timed updates
    bonds, counts = [], []   # outer bonds and matvec counts of each timed update's H_eff
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    launches0 = P.launch_count()
    t_wall = time.perf_counter()
    with ClockSampler(local) as clk:
        e0.record(stream)
        for k in range(args.steps):
            i = centre + args.warmup + k
            bonds.append((i, st.bond(i), st.bond(i + 2)))
            st.update(i, +1, mixed)
            counts.append(st.stats()[2])
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

    # ---- the plain FP64 form at the gate's accuracy (FP64 Lanczos restarted until the Ritz
    # value settles to 1e-12)
    st = make_state(P, ctx, mpo, chi, caps, seed)
    torch.cuda.synchronize(dev)
    t64 = time.perf_counter()
    e_fp64 = None
    for k in range(args.fp64_steps):
        e, _ = st.update(centre + k, +1, fp64_params(P, chi))
        if k == 0:
            e_fp64 = e
    torch.cuda.synchronize(dev)
    t64 = (time.perf_counter() - t64) / args.fp64_steps
    fp64_matvecs = st.stats()[2]
    st.close()

    # ---- the reduced-precision form with FP64 refinement, FP64 Jacobi sweeps after the FP32
    # pre-sweeps and FP64 environments (the FP64-polished variant), two updates
    f64r = mixed_params(P, chi, args.refine, args.fast_restarts, refine_prec=PREC["fp64"],
                        svd_mode=P.MRD_SVD_F32_F64)
    st = make_state(P, ctx, mpo, chi, caps, seed)
    torch.cuda.synchronize(dev)
    t_f64r = time.perf_counter()
    e_f64r = None
    for k in range(2):
        e, _ = st.update(centre + k, +1, f64r)
        if k == 0:
            e_f64r = e
    torch.cuda.synchronize(dev)
    t_f64r = (time.perf_counter() - t_f64r) / 2
    st.close()

    # ---- flops of the timed updates' own H_effs (tables rebuilt from the recorded bonds)
    f_def = f_exec = f_exec_ff = 0.0
    n_tc = n_ff = 0
    for (i, lb, rb), cnt in zip(bonds, counts):
        h = heff_of_bonds(P, ctx, mpo, i, lb, rb)
        fd, fe, _, _ = h.flops()
        h.close()
        ntc, nff = cnt % 1000, cnt // 1000
        f_def += fd * ntc
        f_exec += fe * ntc
        f_exec_ff += fe * nff
        n_tc += ntc
        n_ff += nff

    # ---- side measurements
    set_chi(chi)
    mv = matvec_throughput(P, ctx, torch, dev, stream)
    details["heff_lx20_mid_ring"] = mv
    if not args.quick:
        details["real_vs_mixed_heff"] = real_vs_mixed_or_note(P, ctx, torch, dev, stream)
        try:
            ly8_forms(P, ctx, torch, dev, details)
        except (P.MrdError, torch.cuda.OutOfMemoryError) as e:
            details["ly8"] = {"skipped": f"{type(e).__name__}: {e}"}
        try:
            details["real_arithmetic"] = real_arithmetic_update(P, ctx, torch, dev, stream, chi, args.steps,
                                                                args.warmup, args.refine, args.fast_restarts)
        except (P.MrdError, torch.cuda.OutOfMemoryError) as e:
            details["real_arithmetic"] = {"skipped": f"{type(e).__name__}: {e}"}
        try:
            details["config5"] = config5(P, ctx, torch, dev, fp64_matvecs=max(fp64_matvecs % 1000, 1))
        except (P.MrdError, torch.cuda.OutOfMemoryError) as e:
            details["config5"] = {"skipped": f"{type(e).__name__}: {e}"}
    details["mpo_diagnostics"] = mpo_diagnostics(P)

    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return 0

    bf16_peak, bf16_sust, peak_src = measured_peaks()
    tc_ms, ff_ms = kms[0] + kms[1], kms[2] + kms[3]
    svd_ms = svd_work[0] + svd_work[4]
    # the headline kernel: the split-BF16 H_eff of the timed updates (both grouped launches of
    # every application). Algorithmic flops: the definition order L -> W -> R of the H_eff,
    # 8 per complex multiply-add (definition-order work). Hardware flops: what the tensor cores
    # execute, 4 BF16 products (hi and lo of each operand) per real product of the folded
    # contraction. The kernel runs inside a long step: sustained BF16 peak.
    t_tc = tc_ms / 1e3
    ach = f_def / t_tc / 1e12
    hw = 4 * f_exec / t_tc / 1e12
    traffic, traffic_src = traffic_from_profile(["paper_1512_03318_gb300/csrc/heff_tc.cu",
                                                 "paper_1512_03318_gb300/csrc/tc_host.cu"])
    roof = {"kernel": "k_tc_gemm BF16X3 (H_eff steps 1+2, the timed updates' own H_effs)", "bound": "tensor",
            "achieved": ach, "peak": bf16_sust, "unit": "TFLOP/s", "frac": ach / bf16_sust,
            "traffic": traffic, "traffic_unit": "bytes per H_eff application (2 launches)",
            "hw_achieved": hw, "hw_frac": hw / bf16_sust,
            "peak_source": f"bf16 sustained {peak_src}", "applications": n_tc,
            "ms_per_application": tc_ms / max(n_tc, 1), "ms_per_update": tc_ms / args.steps,
            "note": "achieved: definition-order flops (8 per complex multiply-add); hw: 4 BF16 products "
                    "per real product of the folded contraction"}
    # the Jacobi rounds of the block SVD: FP32 instructions of the float-float work done (per
    # element of a tested pair 48, per element of a rotated pair 112) against the measured FP32
    # fused multiply-add issue rate of this device
    svd_instr = svd_work[1] * 48 + svd_work[2] * 112
    svd_ach = svd_instr / (svd_work[0] / 1e3) / 1e12 if svd_work[0] > 0 else 0.0
    roof_svd = {"kernel": "k_svd_bround<float-float> (block-cyclic Jacobi rounds)", "bound": "alu",
                "achieved": svd_ach, "peak": fp32_peak, "unit": "T FP32-instr/s", "frac": svd_ach / fp32_peak,
                "peak_source": "FP32 FMA issue rate measured in this run (mrd_measure_peaks)",
                "ms_per_update": svd_ms / args.steps}
    # float-float refinement matvecs: 36 FP32 instructions per complex multiply-add executed
    ff_ach = f_exec_ff / 8 * FF_INSTR_PER_CMAC / (ff_ms / 1e3) / 1e12 if ff_ms > 0 else 0.0
    dE = abs(e_mixed_first - e_ref) / abs(e_ref)
    line = {
        "metric": METRIC, "value": s_per_update, "unit": "s/update", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_total / args.steps, "higher_is_better": False, "scaling": "weak",
        "vs_baseline": None, "dtype": "bf16x3+f32x2", "data": "synthetic",
        "dE_rel_mixed_vs_converged_fp64": dE,
        "s_per_update_fp64": t64,
        "speedup_vs_fp64": t64 / (ms_total / 1e3 / args.steps),
        "heff_tflops_bf16x3_timed": ach,
        "config": {"workload": f"two-site update Ly={LY} Lx={LX_UPDATE} flux=1/10 V=1 N={LX_UPDATE} chi={chi}, centre",
                   "chi": chi, "ly": LY, "lx": LX_UPDATE,
                   "form": "BF16X3 Lanczos + float-float refinement, FP32+float-float Jacobi SVD, float-float env",
                   "gate": {"dE_rel_vs_fp64_converged": dE, "limit": 1e-9, "passed": dE <= 1e-9},
                   "fp64_form": {"s_per_update": t64, "dE_rel": abs(e_fp64 - e_ref) / abs(e_ref),
                                 "matvecs": fp64_matvecs},
                   "fp64_refined_form": {"s_per_update": t_f64r, "dE_rel": abs(e_f64r - e_ref) / abs(e_ref)},
                   "l2": "working set > L2 (environments, Z, Lanczos basis > 1 GB)",
                   "parallelism": f"replicas x{world}"},
        "roofline": roof,
        "roofline_svd": roof_svd,
        "roofline_ff_gemm": {"kernel": "k_cgemm_ff (float-float refinement and environment GEMMs)", "bound": "alu",
                             "achieved": ff_ach, "peak": fp32_peak, "unit": "T FP32-instr/s",
                             "frac": ff_ach / fp32_peak, "ms_per_update": ff_ms / args.steps,
                             "applications": n_ff},
        "kernel_ms_per_update": {"k_tc_gemm": round(tc_ms / args.steps, 3), "k_cgemm_ff": round(ff_ms / args.steps, 3),
                                 "k_svd_bround": round(svd_ms / args.steps, 3)},
        "phase_ms_mean": dict(zip(["tables", "theta", "lanczos+refine", "svd", "tensors", "env"],
                                  (phases / args.steps).round(2).tolist())),
        "e2e": {"value": e2e_value, "unit": "s/update", "h2d_bytes_per_step": h2d // args.steps,
                "d2h_bytes_per_step": d2h // args.steps},
        "gpu_launches": launches,
        "clocks": clk.summary(),
        "wall_s_timed": t_wall,
    }
    details["accuracy"] = {"e_ref_fp64_converged": e_ref, "ref_matvecs": ref_matvecs, "e_mixed_first": e_mixed_first,
                           "e_fp64_form": e_fp64, "e_fp64_refined_form": e_f64r}
    details["svd"] = {"jacobi_sweeps_mean": dict(zip(["fp32", "final"], (sweeps / args.steps).round(1).tolist())),
                      "elem_pairs_per_update": {"tested": svd_work[1] / args.steps, "rotated": svd_work[2] / args.steps},
                      "columns_final_sweeps_per_update": svd_work[6] / args.steps,
                      "columns_all_per_update": svd_work[7] / args.steps}
    details["measured_issue_rates"] = {"fp32_fma_per_s": peaks[0], "fp64_fma_per_s": peaks[1], "sms": peaks[2],
                                       "max_sm_clock_hz": peaks[3]}
    details["roofline_traffic_source"] = traffic_src
    if "ly8" in details and "chi2048" in details.get("ly8", {}):
        l8 = details["ly8"]
        line["ly8"] = {"chi1024_fp64_s_per_update": l8["chi1024"]["s_per_update_fp64"],
                       "chi1024_fp64_heff_err_vs_oracle": l8["chi1024"].get("heff_fp64_rel_err_vs_oracle_sampled"),
                       "chi2048_heff_err": {k: l8["chi2048"][f"heff_{k}_rel_err_vs_fp64"] for k in ("tf32", "bf16x3")},
                       "chi2048_forms": {k[5:]: v for k, v in l8["chi2048"].items() if k.startswith("form_")},
                       "chi2048_fp64_s_per_update": l8["chi2048"]["s_per_update_fp64"]}
    ra = details.get("real_arithmetic", {})
    if "s_per_update" in ra:
        line["real_arithmetic"] = {k: ra[k] for k in ("s_per_update", "dE_rel_vs_fp64_converged", "gate_passed",
                                                       "heff_tflops_bf16x3_real", "kernel_ms_per_update")}
        line["real_arithmetic"]["speedup_vs_complex"] = s_per_update / ra["s_per_update"]
    c5 = details.get("config5", {})
    if "s_per_update" in c5:
        line["ly12_chi8000"] = {"s_per_update": c5["s_per_update"], "heff_tflops_bf16x3": c5["heff_tflops_bf16x3"],
                                "bond_dims": c5["bond_dims"], "env_update_gbs": c5["env_update_gbs"],
                                "env_storage": "complex64",
                                "env_estimate_gb": {k: c5["env_estimate_gb"][k] for k in ("complex64", "complex128")},
                                "fp64_form_s_per_update_estimate": c5["fp64_form_s_per_update_estimate"]}
    if world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline()
    line["details"] = args.details
    try:
        with open(args.details, "w") as f:
            json.dump(details, f, indent=1, default=float)
    except OSError as e:
        line["details"] = f"not written: {e}"
    print(json.dumps(line))
    if dist is not None:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
