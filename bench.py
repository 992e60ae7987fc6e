#!/usr/bin/env python
"""Throughput of one randomised primal-dual (PD-R) iteration on GB300.

Workload (default "c5"): 2048x2048 image, 4096x4096 complex64 grid,
M = 16,777,216 visibilities with radially decaying density (inner 8x denser),
256 uneven blocks (32 annuli x 8 sectors), 8x8 Kaiser-Bessel kernel evaluated
on the fly, Dirac + db1..db8 at 4 levels, every block and basis drawn with
p = 0.5, 30 dB noise. One step = one full iteration of Algorithm 1 (draws,
F Z x~, degridding + l2-ball duals, gridding, wavelet duals, F^H + primal).

Prints one JSON line. Multi-GPU runs (torchrun) solve one independent problem
per rank (weak scaling, no collective on the data path).
"""
import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOADS = {
    "c5": dict(n=2048, m=16_777_216, nannuli=32, nsectors=8, J=8, bases=list(range(9)), levels=4, p=0.5,
               snr=30.0),
    # c5 shrunk 4x (profiling captures: inputs still larger than L2, ~0.3 GB on the device)
    "c5_div4": dict(n=1024, m=4_194_304, nannuli=32, nsectors=8, J=8, bases=list(range(9)), levels=4, p=0.5,
                    snr=30.0),
    # the reference arm and the CPU baseline run the oracle on this 16x smaller version of c5
    "c5_div16": dict(n=512, m=1_048_576, nannuli=32, nsectors=8, J=8, bases=list(range(9)), levels=4, p=0.5,
                     snr=30.0),
    "small": dict(n=256, m=65_536, nannuli=4, nsectors=4, J=8, bases=list(range(9)), levels=4, p=0.5, snr=30.0),
}
METRIC = "PD iters/s @2048^2 img, 16.8M vis (FP32 batched graph)"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="c5", choices=sorted(WORKLOADS))
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--fp64-steps", type=int, default=10)
    ap.add_argument("--no-operators", action="store_true")
    ap.add_argument("--no-csr", action="store_true")
    ap.add_argument("--no-sara", action="store_true")
    ap.add_argument("--no-dde", action="store_true")
    ap.add_argument("--no-synthesis", action="store_true")
    ap.add_argument("--csr-steps", type=int, default=20)
    ap.add_argument("--g-mode", default="on_the_fly", choices=["on_the_fly", "csr"],
                    help="form of G for --profile-run")
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--tile", type=int, default=0, help="gridding tile edge (0: the plan's default)")
    ap.add_argument("--profile-run", type=int, default=0,
                    help="profiling target: plan the workload, set data and start values, run this many eager "
                         "iterations with fixed step sizes (no power method, no timing) and exit")
    ap.add_argument("--no-autotune", action="store_true",
                    help="skip pd_plan_autotune (16, 32, 64) and plan with --tile (0: the plan's default)")
    ap.add_argument("--cpu-full", type=int, default=0,
                    help="time this many oracle iterations on the full c5 workload (CPU only) and exit")
    return ap.parse_args()


def make_inputs(cfg, seed):
    from paper_1610_08895_gb300 import synth
    uv = synth.uv_radial(cfg["m"], seed=seed + 1)
    blk = synth.blocks_annuli(uv, cfg["nannuli"], cfg["nsectors"])
    x_true = synth.test_image(cfg["n"], seed=seed + 2)
    noise = synth.complex_noise(cfg["m"], seed=seed + 3)
    return uv, blk, x_true, noise


def epsilon(sigma_n, sizes):
    from scipy.stats import chi2
    m = np.maximum(np.asarray(sizes, dtype=np.float64), 1.0)
    return sigma_n / np.sqrt(2.0) * np.sqrt(chi2.ppf(0.99, 2.0 * m))


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        d = json.load(open(path))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


class Clocks:
    """nvidia-smi sampler (its own child process, 50 ms period) of SM clocks and throttle
    reasons during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.samples = []
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "50"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            time.sleep(0.3)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is None:
            return
        time.sleep(0.1)
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=10)
        except Exception:
            self.proc.kill()
            out, _ = self.proc.communicate()
        for line in out.splitlines():
            cols = [c.strip() for c in line.split(",")]
            if len(cols) >= 8:
                self.samples.append(cols)

    def summary(self):
        if not self.samples:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}

        def num(v):
            try:
                return float(v)
            except ValueError:
                return None
        sm = [num(s[1]) for s in self.samples if num(s[1]) is not None]
        mx = [num(s[2]) for s in self.samples if num(s[2]) is not None]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for s in self.samples for k in range(4) if s[4 + k].lower() == "active"})
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.samples)}


# committed ncu summaries with the measured DRAM traffic of a kernel, per bench phase
PROFILE_OF_PHASE = {"grid_dual": "k_grid8w_gridding_c5.md", "degrid_dual": "k_degrid_degridding_c5.md"}


def kernel_source_hash(path, name):
    """sha256 of a kernel's definition text in a .cu file (from `__global__` to the
    closing brace of its body), or None if the kernel is not found."""
    import hashlib
    import re
    text = open(path).read()
    start = None
    for m in re.finditer(r"\b" + re.escape(name) + r"\(", text):
        # the declaration this name opens: text since the previous statement or block end
        lo = max(text.rfind(";", 0, m.start()), text.rfind("}", 0, m.start())) + 1
        g = text.find("__global__", lo, m.start())
        if g >= 0:
            start = g
            break
    if start is None:
        return None
    depth = 0
    for j in range(text.index("{", m.end()), len(text)):
        if text[j] == "{":
            depth += 1
        elif text[j] == "}":
            depth -= 1
            if depth == 0:
                return hashlib.sha256(text[start:j + 1].encode()).hexdigest()
    return None


def measured_traffic(phase, workload):
    """DRAM read + write bytes per launch of a phase's kernel from its committed ncu
    summary, or None when there is none or the kernel's definition no longer has the
    hash recorded at capture time (the counters then describe another kernel)."""
    import re
    name = PROFILE_OF_PHASE.get(phase)
    if name is None or workload != "c5":
        return None
    path = os.path.join(ROOT, "profiles", name)
    if not os.path.exists(path):
        return None
    text = open(path).read()
    m_src = re.search(r"`([^`]+\.cu)` kernel `(\w+)` sha256 ([0-9a-f]{64})", text)
    m_tr = re.search(r"traffic per launch \(DRAM read \+ write\) \| (\d+) B", text)
    if not m_src or not m_tr:
        return None
    src = os.path.join(ROOT, m_src.group(1))
    if not os.path.exists(src) or kernel_source_hash(src, m_src.group(2)) != m_src.group(3):
        return None
    return int(m_tr.group(1))


def job_throughput(ms_local, steps, device="cuda"):
    """Max over ranks of the timed region (ms) and the whole-job throughput. Every rank
    solves its own problem (weak scaling), so value = world * steps / max time."""
    import torch
    import torch.distributed as dist
    world = dist.get_world_size() if dist.is_available() and dist.is_initialized() else 1
    ms = float(ms_local)
    if world > 1:
        t = torch.tensor([ms], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    return ms, world * steps / (ms / 1e3)


def rank_seed(seed, rank):
    """Data seed of a rank's independent problem."""
    return seed + 100 * rank


def algorithmic_bytes(cfg, plan_info, m_active, tiles_active_frac, bases_active, dirac_active):
    """Bytes each phase must move per launch (FP32): the reads and writes its result needs."""
    n = cfg["n"]
    N = n * n
    K = 4 * N
    L = cfg["levels"]
    ll = sum(8.0 * N / 4 ** l for l in range(1, L))          # one write + one read of the approximations
    wav = bases_active - dirac_active
    # the forward passes keep the half spectrum (columns 0 .. n of the 2n-wide grid: F Z x is
    # Hermitian for a real image); the inverse passes read the full gridded U once
    return {
        "fwd_rows": 4 * N + 8 * N,
        "fwd_cols": 8 * N + 16 * N,
        "degrid_dual": 36 * m_active + 8 * K * tiles_active_frac,
        "grid_dual": 36 * m_active + 16 * K * tiles_active_frac,
        "wavelet_analysis": 4 * N + wav * (12 * N + ll) + dirac_active * 12 * N,
        "wavelet_synthesis": wav * (4 * N + ll) + dirac_active * 4 * N + 8 * N,
        "inv_cols": 32 * N + 8 * N,
        "inv_rows_primal": 8 * N + 16 * N,
    }


def _time_ms(fn, reps, stream):
    import torch
    fn()
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for _ in range(reps):
        fn()
    b.record(stream)
    torch.cuda.synchronize()
    return a.elapsed_time(b) / reps


def run_operators(peak, stream, reps=20):
    """Phi and Phi^H alone on a batch of 8 images: 1024^2 image, 2048^2 grid,
    M = 4,194,304 Gaussian uv points, J = 8, FP32. Algorithmic bytes per image are the
    sums of the per-pass figures: 100 N + 24 M for either operator (N pixels, M points)."""
    import torch
    from paper_1610_08895_gb300 import synth
    from paper_1610_08895_gb300.api import Plan
    n, m, batch = 1024, 4_194_304, 8
    plan = Plan(n, n, synth.uv_gaussian(m, seed=31), np.zeros(m, np.int32), 1, kernel_width=8, precision="f32")
    x = torch.tensor(synth.random_images(batch, n, n, seed=4), dtype=torch.float32, device="cuda")
    y = torch.empty((batch, m), dtype=torch.complex64, device="cuda")
    xa = torch.empty_like(x)
    ms_phi = _time_ms(lambda: plan.pd_apply_phi(x, y), reps, stream)
    ms_adj = _time_ms(lambda: plan.pd_apply_phi_adj(y, xa), reps, stream)
    alg = (100.0 * n * n + 24.0 * m) * batch
    plan.close()
    out = {"workload": f"{n}x{n} image, {2 * n}x{2 * n} grid, M={m} Gaussian uv, J=8, batch {batch}, f32"}
    for name, ms in (("phi", ms_phi), ("phi_adj", ms_adj)):
        gbs = alg / (ms / 1e3) / 1e9
        out[name] = {"ms_per_batch": round(ms, 4), "GBps": round(gbs, 1), "frac": round(gbs / peak, 4)}
    return out


def run_cufft(n, stream, reps=20):
    """cuFFT (torch.fft) 2-D transforms of one full (2n)^2 complex64 grid: the library
    counterpart of the FFT passes (which skip the zero rows of Z and the cropped rows)."""
    import torch
    g = torch.randn((2 * n, 2 * n), dtype=torch.complex64, device="cuda")
    return {"grid": f"{2 * n}x{2 * n} c64", "fft2_ms": round(_time_ms(lambda: torch.fft.fft2(g), reps, stream), 4),
            "ifft2_ms": round(_time_ms(lambda: torch.fft.ifft2(g), reps, stream), 4)}


# our kernels per iteration: draws; 2 forward passes; degridding + block norms; 4 gridding
# colour launches; L analysis levels + the Dirac basis; L synthesis levels + the ordered
# sum; 2 inverse passes; the primal norm sums
KERNELS_PER_ITER = lambda L: 1 + 2 + 2 + 4 + (L + 1) + (L + 1) + 2 + 1   # noqa: E731


# ---------------------------------------------------------------------------------------------
def run_ours(args):
    import torch
    import torch.distributed as dist

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl", init_method="env://")
    torch.cuda.set_device(local)
    import __graft_entry__ as ge
    ge.build()
    from paper_1610_08895_gb300.api import Plan, State

    cfg = WORKLOADS[args.workload]
    n, m = cfg["n"], cfg["m"]
    t0 = time.time()
    uv, blk, x_true, noise = make_inputs(cfg, rank_seed(args.seed, rank))
    d = int(blk.max()) + 1
    b = len(cfg["bases"])
    tile, tune = args.tile, None
    if not args.no_autotune and not args.tile:
        from paper_1610_08895_gb300.api import autotune_tile
        tile, tune = autotune_tile(n, n, uv, blk, d, kernel_width=cfg["J"], basis_ids=cfg["bases"],
                                   levels=cfg["levels"], candidates=(16, 32, 64), iters=5)
    plan = Plan(n, n, uv, blk, d, kernel_width=cfg["J"], basis_ids=cfg["bases"], levels=cfg["levels"],
                precision="f32", tile=tile)
    info = plan.info()
    if tune is not None:
        info["autotune_ms_per_iteration"] = {str(k): round(v, 4) for k, v in tune.items()}
    sizes = np.bincount(blk, minlength=d)
    # measurements y = Phi x + n (Phi on the GPU), bounds from the chi-square quantile
    xt = torch.tensor(x_true, dtype=torch.float32, device="cuda")
    phix = plan.pd_apply_phi(xt)
    sig = float(torch.linalg.vector_norm(phix.to(torch.complex128)).item()) / np.sqrt(m) * 10 ** (-cfg["snr"] / 20)
    y_host = (phix.cpu().numpy().astype(np.complex128) + sig * noise).astype(np.complex64)
    y = torch.tensor(y_host, device="cuda")
    eps = epsilon(sig, sizes)
    x0 = torch.tensor(np.random.default_rng(9).normal(size=(n, n)), dtype=torch.float32, device="cuda")
    phi2, psi2, _ = plan.pd_operator_norms(x0, max_iter=20, tol=1e-3)
    kw = dict(tau=0.49, sigma=1.0 / psi2, varsigma=1.0 / phi2, kappa=1e-3, psi_norm=float(np.sqrt(psi2)),
              seed=args.seed, p_block=[cfg["p"]] * d, p_basis=[cfg["p"]] * b)
    st = State(plan)
    st.pd_state_set_data(y, eps)
    setup_s = time.time() - t0

    # ---- warm-up, then the timed region: K graph replays of one iteration
    st.pd_iterate(args.warmup, use_graph=True, **kw)
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    with Clocks(local) as clk:
        e0.record(stream)
        st.pd_iterate(args.steps, use_graph=True, **kw)
        e1.record(stream)
        torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    ms, value = job_throughput(e0.elapsed_time(e1), args.steps)

    # ---- per-kernel times (CUDA events on the launching stream) over K instrumented iterations
    st.profile(reset=True)
    m_act, t_act, nb_act, dirac_act = 0.0, 0.0, 0.0, 0.0
    dirac_slots = [k for k, bid in enumerate(cfg["bases"]) if bid == 0]
    for _ in range(args.steps):
        st.pd_iterate(1, profile=True, **kw)
        rep = st.report()
        m_act += float(sizes[rep["block_active"]].sum())
        t_act += rep["active_tiles"] / info["kx"] / info["ky"] * info["tile"] ** 2
        nb_act += float(rep["basis_active"].sum())
        dirac_act += float(sum(rep["basis_active"][k] for k in dirac_slots))
    prof = st.profile()
    k_steps = float(args.steps)
    alg = algorithmic_bytes(cfg, info, m_act / k_steps, t_act / k_steps, nb_act / k_steps, dirac_act / k_steps)
    kernels = {}
    for name, (tot_ms, cnt) in prof.items():
        if cnt == 0 or tot_ms == 0.0:
            continue
        avg = tot_ms / cnt
        entry = {"ms": round(avg, 4)}
        if name in alg:
            entry["GBps"] = round(alg[name] / (avg / 1e3) / 1e9, 1)
        kernels[name] = entry
    dom = max((k for k in kernels if k in alg), key=lambda k: kernels[k]["ms"])
    peak, peak_kind = peaks()
    achieved = kernels[dom]["GBps"]
    roofline = {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": round(achieved / peak, 4), "peak_source": peak_kind,
                "traffic": measured_traffic(dom, args.workload), "algorithmic_bytes_per_launch": int(alg[dom])}

    # ---- Phi / Phi^H alone, and cuFFT as a timed comparison of the FFT passes
    operators = None
    if not args.no_operators:
        operators = run_operators(peak, stream)
        cf = run_cufft(n, stream)
        cf["ours_forward_ms"] = round(kernels["fwd_rows"]["ms"] + kernels["fwd_cols"]["ms"], 4)
        cf["ours_inverse_ms"] = round(kernels["inv_cols"]["ms"] + kernels["inv_rows_primal"]["ms"], 4)
        operators["cufft_vs_fft_passes"] = cf

    # ---- end to end through the public API with host buffers
    e2e = None
    if not args.no_e2e:
        y_pin = torch.from_numpy(y_host).pin_memory()
        x_pin = torch.empty((n, n), dtype=torch.float32).pin_memory()
        y_dev = torch.empty(m, dtype=torch.complex64, device="cuda")
        st2 = State(plan)
        torch.cuda.synchronize()
        t_a = time.perf_counter()
        y_dev.copy_(y_pin, non_blocking=True)
        st2.pd_state_set_data(y_dev, eps)
        d2h = 0
        for _ in range(args.steps):
            st2.pd_iterate(1, **kw)
            st2.report()                      # per-step result to host: t, ||dx||^2, ||x||^2 (+ block data)
            d2h += 8 + 16 + d * (8 + 8 + 4) + b * 4
        x_pin.copy_(st2.x(), non_blocking=True)
        torch.cuda.synchronize()
        t_b = time.perf_counter()
        d2h += n * n * 4
        h2d = m * 8 + args.steps * (d + b) * 8
        e2e = {"value": round(args.steps / (t_b - t_a), 3), "unit": "PD iters/s",
               "h2d_bytes_per_step": int(h2d / args.steps), "d2h_bytes_per_step": int(d2h / args.steps)}
        st2.close()

    # ---- FP64 forms of the same workload: the plain per-block form (the host draws the active
    # sets and launches each data-fidelity operator once per active block, each sparsity operator
    # once per active basis) and the batched graph form with FP64 bulk data
    fp64 = None
    if not args.no_fp64:
        plan64 = Plan(n, n, uv, blk, d, kernel_width=cfg["J"], basis_ids=cfg["bases"], levels=cfg["levels"],
                      precision="f64", tile=tile)
        fp64 = {}
        for form, extra in (("per_block", dict(per_block=True)), ("batched_graph", dict(use_graph=True))):
            st64 = State(plan64)
            st64.pd_state_set_data(torch.tensor(y_host.astype(np.complex128), device="cuda"), eps)
            st64.pd_iterate(2, **extra, **kw)
            torch.cuda.synchronize()
            f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            f0.record(stream)
            st64.pd_iterate(args.fp64_steps, **extra, **kw)
            f1.record(stream)
            torch.cuda.synchronize()
            ms64 = f0.elapsed_time(f1)
            fp64[form] = {"value": round(args.fp64_steps / (ms64 / 1e3), 3), "unit": "PD iters/s",
                          "ms_per_step": round(ms64 / args.fp64_steps, 3), "steps": args.fp64_steps}
            st64.close()
        fp64["per_block"]["form"] = ("FP64 throughout; host-drawn active sets; one degridding, ball update, "
                                     "gridding (per tile colour) launch per active block and one analysis / "
                                     "synthesis launch set per active basis; eager")
        fp64["batched_graph"]["form"] = "FP64 bulk data in the batched kernels, one CUDA graph per iteration"
        plan64.close()

    # ---- the same workload with G held as a sparse matrix (CSR, built on the device at plan time)
    csr = None
    if not args.no_csr:
        csr = run_csr(args, cfg, uv, blk, d, tile, y, eps, kw, sizes, stream)

    # ---- the reweighted prior (SARA): the same iterations with per-coefficient weights
    sara = None
    if not args.no_sara:
        sara = run_sara(args, plan, st, kw, stream)

    # ---- DDE-aware G: 6x6 Kaiser-Bessel kernels convolved with 3x3 Fourier-domain DDE kernels
    dde = None
    if not args.no_dde:
        dde = run_dde(args, cfg, uv, blk, d, tile, y, eps, kw, stream)

    # ---- the synthesis formulation on the same data (eager iterations)
    synthesis = None
    if not args.no_synthesis:
        synthesis = run_synthesis(plan, y, eps, kw, stream)

    # ---- errors of this run's results against the FP64 oracle on sampled outputs
    errors = None
    if rank == 0 and not args.no_cpu_baseline:
        errors = sampled_errors(cfg, uv, x_true, phix)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(args.seed, steps=2, warmup=1)

    if rank == 0:
        line = {
            "metric": METRIC, "value": round(value, 3), "unit": "PD iters/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms / args.steps, 4),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic", "gpu_launches": KERNELS_PER_ITER(cfg["levels"]) * args.steps,
            "config": {"workload": f"{args.workload}: {n}x{n} image, {2 * n}x{2 * n} grid, M={m}, "
                                   f"{d} uneven blocks (annuli x sectors), J={cfg['J']} KB on the fly, "
                                   f"{b} bases x {cfg['levels']} levels, p_block=p_basis={cfg['p']}",
                       "global_batch": world, "parallelism": f"replicas x{world} (independent problems)",
                       "l2": "working set > L2 (grid 134 MB + visibilities 600 MB per iteration)",
                       "graph": "one CUDA graph per iteration, replayed", "setup_s": round(setup_s, 1),
                       "plan": info},
            "roofline": roofline, "kernels": kernels, "clocks": clk.summary(), "e2e": e2e,
            "fp64": fp64, "csr": csr, "sara": sara, "dde": dde, "synthesis": synthesis, "operators": operators, "cpu_baseline": cpu, "errors": errors,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def run_csr(args, cfg, uv, blk, d, tile, y, eps, kw, sizes, stream):
    """FP32 batched graph iterations with G stored as a sparse matrix (J^2 column/weight
    pairs per visibility) instead of evaluated in the kernels, and the degridding and
    gridding kernel times with their algorithmic bytes (the stored entries dominate)."""
    import torch
    from paper_1610_08895_gb300.api import Plan, State
    n, J = cfg["n"], cfg["J"]
    plan = Plan(n, n, uv, blk, d, kernel_width=J, basis_ids=cfg["bases"], levels=cfg["levels"],
                precision="f32", tile=tile, g_mode="csr")
    info = plan.info()
    st = State(plan)
    st.pd_state_set_data(y, eps)
    st.pd_iterate(3, use_graph=True, **kw)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    st.pd_iterate(args.csr_steps, use_graph=True, **kw)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    st.profile(reset=True)
    m_act, t_act, reps = 0.0, 0.0, 5
    for _ in range(reps):
        st.pd_iterate(1, profile=True, **kw)
        rep = st.report()
        m_act += float(sizes[rep["block_active"]].sum())
        t_act += rep["active_tiles"] / info["kx"] / info["ky"] * info["tile"] ** 2
    prof = st.profile()
    K = 4 * n * n
    per_vis = 24 + 8 * J * J             # y, v in, r out (or r, v in, v out) + the stored row of G
    alg = {"degrid_dual": per_vis * m_act / reps + 8 * K * t_act / reps,
           "grid_dual": per_vis * m_act / reps + 16 * K * t_act / reps}
    kernels = {}
    for name in ("degrid_dual", "grid_dual"):
        tot, cnt = prof.get(name, (0.0, 0))
        if cnt:
            avg = tot / cnt
            kernels[name] = {"ms": round(avg, 4), "GBps": round(alg[name] / (avg / 1e3) / 1e9, 1),
                             "algorithmic_bytes_per_launch": int(alg[name])}
    st.close()
    out = {"value": round(args.csr_steps / (ms / 1e3), 3), "unit": "PD iters/s",
           "ms_per_step": round(ms / args.csr_steps, 4), "steps": args.csr_steps,
           "g_bytes": int(J * J * 8 * cfg["m"]), "device_bytes": info.get("device_bytes"),
           "kernels": kernels,
           "form": "FP32 batched graph; G as CSR with J^2 (int32 cell, fp32 weight) entries per visibility"}
    plan.close()
    return out


def run_sara(args, plan, st, kw, stream, steps=20):
    """Batched graph iterations with the reweighted prior: weights from the current
    iterate (pd_sara_weights), then timed iterations that read them in step 13."""
    import torch
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    w = plan.pd_sara_weights(st.x(), 1e-3)
    t0.record(stream)
    plan.pd_sara_weights(st.x(), 1e-3, weights=w)
    t1.record(stream)
    st.pd_iterate(3, use_graph=True, weights=w, **kw)
    torch.cuda.synchronize()
    rule_ms = t0.elapsed_time(t1)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    st.pd_iterate(steps, use_graph=True, weights=w, **kw)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    return {"value": round(steps / (ms / 1e3), 3), "unit": "PD iters/s", "ms_per_step": round(ms / steps, 4),
            "steps": steps, "reweight_ms": round(rule_ms, 4),
            "form": "FP32 batched graph, step 13 with per-coefficient weights W = delta/(delta + |Psi^H x|)"}


def run_dde(args, cfg, uv, blk, d, tile, y, eps, kw, stream, steps=10):
    """Batched graph iterations with the DDE-aware G stored as complex CSR rows: 6 x 6
    interpolation kernels convolved with per-visibility 3 x 3 Fourier-domain DDE kernels
    (seeded near-identity complex values), a footprint of 8 x 8 like the headline's J = 8."""
    import torch
    from paper_1610_08895_gb300.api import Plan, State
    n, m = cfg["n"], cfg["m"]
    rng = np.random.default_rng(args.seed + 7)
    dk = (0.2 * (rng.standard_normal((m, 3, 3), dtype=np.float32)
                 + 1j * rng.standard_normal((m, 3, 3), dtype=np.float32))).astype(np.complex128)
    dk[:, 1, 1] += 1.0
    t0 = time.time()
    plan = Plan(n, n, uv, blk, d, kernel_width=6, basis_ids=cfg["bases"], levels=cfg["levels"], precision="f32",
                tile=tile, g_mode="csr", dde_kernels=dk)
    setup = time.time() - t0
    del dk
    info = plan.info()
    st = State(plan)
    st.pd_state_set_data(y, eps)
    st.pd_iterate(3, use_graph=True, **kw)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    st.pd_iterate(steps, use_graph=True, **kw)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    st.profile(reset=True)
    st.pd_iterate(3, profile=True, **kw)
    prof = st.profile()
    kern = {k: round(prof[k][0] / prof[k][1], 4) for k in ("degrid_dual", "grid_dual") if prof.get(k, (0, 0))[1]}
    st.close()
    plan.close()
    return {"value": round(steps / (ms / 1e3), 3), "unit": "PD iters/s", "ms_per_step": round(ms / steps, 4),
            "steps": steps, "kernels_ms": kern, "plan_s": round(setup, 1), "device_bytes": info.get("device_bytes"),
            "form": "FP32 batched graph; G = 6x6 Kaiser-Bessel kernel convolved with a 3x3 complex DDE kernel per "
                    "visibility, complex CSR rows of 64 entries"}


def run_synthesis(plan, y, eps, kw, stream, steps=10):
    """Eager iterations of the synthesis formulation (pd_synthesis_iterate): x = Psi alpha,
    l1 on the coefficients, positivity as a dual; same data, blocks and draws."""
    import torch
    from paper_1610_08895_gb300.api import State
    st = State(plan)
    st.pd_state_set_data(y, eps)
    args = dict(tau=kw["tau"], sigma=1.0, varsigma=kw["varsigma"], kappa=kw["kappa"], seed=kw["seed"],
                p_block=kw["p_block"])
    st.pd_synthesis_iterate(2, **args)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    st.pd_synthesis_iterate(steps, **args)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    st.close()
    return {"value": round(steps / (ms / 1e3), 3), "unit": "PD iters/s", "ms_per_step": round(ms / steps, 4),
            "steps": steps, "form": "FP32, eager (one call of `steps` iterations, the image Psi alpha formed "
                                    "once at the end); every coefficient updated every iteration"}


# ---------------------------------------------------------------------------------------------
def run_profile_target(args):
    """A short, deterministic launch sequence for ncu: plan, y from synthetic noise, start
    values x^(0) = x~^(0) = the test image, then args.profile_run eager iterations (per
    iteration: draws, 4 analysis + 4 synthesis levels and the sum, 2 forward passes,
    degridding, block norms, 4 gridding colour launches, 2 inverse passes, primal sums)."""
    import torch
    import __graft_entry__ as ge
    ge.build()
    from paper_1610_08895_gb300.api import Plan, State
    cfg = WORKLOADS[args.workload]
    n, m = cfg["n"], cfg["m"]
    uv, blk, x_true, noise = make_inputs(cfg, args.seed)
    d = int(blk.max()) + 1
    b = len(cfg["bases"])
    plan = Plan(n, n, uv, blk, d, kernel_width=cfg["J"], basis_ids=cfg["bases"], levels=cfg["levels"],
                precision="f32", tile=args.tile, g_mode=args.g_mode)
    st = State(plan)
    st.pd_state_set_data(torch.tensor(10.0 * noise, dtype=torch.complex64, device="cuda"), np.full(d, 30.0))
    x0 = torch.tensor(x_true, dtype=torch.float32, device="cuda")
    st.pd_state_set_start(x0, x0)
    st.pd_iterate(args.profile_run, tau=0.49, sigma=1.0, varsigma=1e-7, kappa=1e-3, psi_norm=1.0, seed=args.seed,
                  p_block=[cfg["p"]] * d, p_basis=[cfg["p"]] * b)
    torch.cuda.synchronize()
    print(json.dumps({"profile_run": args.profile_run, "workload": args.workload, "plan": plan.info()}))


def oracle_problem(cfg, seed):
    """The oracle's problem on a workload (used only by the CPU legs)."""
    from oracle import experiment as EX
    from oracle import measurement as meas
    from oracle import pd as PD
    uv, blk, x_true, noise = make_inputs(cfg, seed)
    d = int(blk.max()) + 1
    prob = PD.Problem(meas.Geometry(cfg["n"], cfg["n"], cfg["J"]), uv, blk, d, cfg["bases"], cfg["levels"])
    phix = prob.phi(x_true)
    sn = EX.noise_sigma(phix, cfg["snr"])
    prob.y = phix + sn * noise
    prob.eps = EX.epsilon_bounds(sn, [max(len(ix), 1) for ix in prob.block_index])
    return prob


def sampled_errors(cfg, uv, x_true, phix_gpu, nsample=20000, seed=7):
    """Relative error of this run's FP32 Phi x_true against the FP64 oracle at nsample
    visibilities (the oracle's F Z x in full, its G at the samples only)."""
    from oracle import measurement as meas
    geo = meas.Geometry(cfg["n"], cfg["n"], cfg["J"])
    idx = np.random.default_rng(seed).choice(len(uv), size=nsample, replace=False)
    ref = geo.degrid(geo.fft(geo.zpad(x_true)), uv[idx])
    got = phix_gpu.cpu().numpy()[idx].astype(np.complex128)
    return {"phi_sampled_rel_l2": float(np.linalg.norm(got - ref) / np.linalg.norm(ref)),
            "sample": f"Phi x_true at {nsample} of {len(uv)} visibilities",
            "parity_tests": "the iterate and operator errors of the -m gpu parity tests are tabulated with "
                            "the design notes (C1 200 it., C2 500 it., C3, C5 Phi^H full image, C5 iteration)"}


def host_cpu():
    """CPU model and thread count of this host (lscpu, else /proc/cpuinfo)."""
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.startswith("Model name:"):
                model = line.split(":", 1)[1].strip()
                break
    except Exception:
        pass
    if model is None:
        try:
            for line in open("/proc/cpuinfo"):
                if line.lower().startswith(("model name", "cpu part")):
                    model = line.split(":", 1)[1].strip()
                    break
        except OSError:
            pass
    return {"model": model or "unknown", "nproc": os.cpu_count()}


def oracle_iterations(cfg, seed, steps, warmup):
    """Seconds per oracle iteration (Algorithm 1 in FP64 numpy, as it stands) on a workload,
    after `warmup` untimed iterations. The oracle's numpy steps (FFT, bincount, elementwise)
    run on one thread."""
    from oracle import pd as PD
    prob = oracle_problem(cfg, seed)
    d, b = prob.nblocks, len(prob.basis_ids)
    kw = dict(tau=0.49, sigma=1.0, varsigma=1e-6, kappa=1e-3, psi_norm=1.0, seed=seed,
              p_block=[cfg["p"]] * d, p_basis=[cfg["p"]] * b)
    st = PD.PDState(prob)
    for _ in range(warmup):
        PD.pd_iteration(prob, st, **kw)
    t = time.perf_counter()
    for _ in range(steps):
        PD.pd_iteration(prob, st, **kw)
    return (time.perf_counter() - t) / steps


def _oracle_replica(seed):
    """Seconds of one scaled-sample oracle iteration in a worker process."""
    return oracle_iterations(WORKLOADS["c5_div16"], seed, 1, 0)


def _noop(_):
    return 0


def oracle_all_cores(n):
    """The oracle as it stands on every host core at once: n independent replicas of the
    scaled sample (one per core, spawned processes, one numpy thread each), each timing
    one iteration while the others run. Returns (aggregate c5 iterations/s, seconds per
    iteration of each replica)."""
    import multiprocessing as mp
    with mp.get_context("spawn").Pool(n) as pool:
        pool.map(_noop, range(n))                       # start the workers and import first
        dts = pool.map(_oracle_replica, [100 + k for k in range(n)])
    return sum(1.0 / dt for dt in dts) / 16.0, dts


def cpu_baseline(seed, steps, warmup, full=False):
    """Oracle iterations/s on this host's cores. Default: a bounded sample -- the c5 workload
    shrunk 16x in pixels and visibilities (512^2 image, 1,048,576 visibilities, same blocks,
    bases and levels), its measured time per iteration multiplied by 16 to express one c5
    iteration (the cost is linear in both up to the FFT's log factor, so this overstates the
    oracle's full-size speed slightly). full=True times the c5 workload itself (minutes per
    iteration)."""
    cfg = WORKLOADS["c5" if full else "c5_div16"]
    dt = oracle_iterations(cfg, seed, steps, warmup)
    scale = 1.0 if full else 16.0
    cpu = host_cpu()
    what = ("the c5 workload itself (2048^2 image, 16,777,216 visibilities, 256 blocks, 9 bases, 4 levels)"
            if full else "a scaled sample: the c5 workload shrunk 16x (512^2 image, 1,048,576 visibilities, "
                         "256 blocks, 9 bases, 4 levels), time x 16 for one c5 iteration")
    allc = None
    if not full and (cpu["nproc"] or 1) > 1:
        n = min(int(cpu["nproc"]), 16)
        rate, dts = oracle_all_cores(n)
        allc = {"value": round(rate, 6), "unit": "PD iters/s", "cores": n,
                "s_per_iteration_per_replica": round(float(np.median(dts)), 3),
                "sample": f"{n} independent replicas of the scaled sample, one per core, one iteration each, "
                          "aggregate throughput x 1/16 for c5 iterations"}
    return {"value": round(1.0 / (dt * scale), 6), "unit": "PD iters/s", "cores": 1, "kind": "oracle",
            "scaled": not full, "s_per_iteration_measured": round(dt, 3), "all_cores": allc,
            "s_per_c5_iteration": round(dt * scale, 2), "host": cpu,
            "sample": f"{steps} oracle iterations (after {warmup} warm-up) of {what}; numpy, one thread "
                      f"(the oracle's FFT, bincount and elementwise steps are single-threaded; "
                      f"{cpu['nproc']} threads on the host)"}


def run_reference(args):
    """The oracle as the reference arm, on the c5 workload's metric. Each step is a bounded
    sample: one oracle iteration of c5 shrunk 16x, timed and multiplied by 16 (a scaled
    sample, stated in the line's config), so that K steps fit in a few minutes; a full c5
    oracle iteration takes minutes (bench.py --cpu-full measures it)."""
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from oracle import pd as PD
    cfg = WORKLOADS["c5_div16"]
    prob = oracle_problem(cfg, args.seed)
    d, b = prob.nblocks, len(prob.basis_ids)
    kw = dict(tau=0.49, sigma=1.0, varsigma=1e-6, kappa=1e-3, psi_norm=1.0, seed=args.seed,
              p_block=[cfg["p"]] * d, p_basis=[cfg["p"]] * b)
    st = PD.PDState(prob)
    for _ in range(args.warmup):
        PD.pd_iteration(prob, st, **kw)
    t = time.perf_counter()
    for _ in range(args.steps):
        PD.pd_iteration(prob, st, **kw)
    dt = time.perf_counter() - t
    value = args.steps / dt / 16.0
    cpu = host_cpu()
    sample = (f"each step: one oracle iteration of the c5 workload shrunk 16x (512^2 image, "
              f"1,048,576 visibilities, 256 blocks, 9 bases, 4 levels), {dt / args.steps:.2f} s measured, "
              f"x 16 for one c5 iteration; numpy, one thread of {cpu['nproc']} ({cpu['model']})")
    line = {"impl": "reference", "metric": METRIC, "value": round(value, 6), "unit": "PD iters/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(dt / args.steps * 1e3, 1), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "c5 (2048^2 image, 16,777,216 visibilities, 256 blocks, 9 bases x 4 levels, "
                                   "p = 0.5)", "sample": "scaled: each step times c5 shrunk 16x; value = "
                                                         "steps / time / 16", "host": cpu},
            "cpu_baseline": {"value": round(value, 6), "unit": "PD iters/s", "cores": 1, "kind": "oracle",
                             "scaled": True, "sample": sample},
            "e2e": {"value": round(value, 6), "unit": "PD iters/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_cpu_full(args):
    """Oracle iterations/s on the c5 workload itself (no scaling), on this host."""
    res = cpu_baseline(args.seed, steps=args.cpu_full, warmup=0, full=True)
    print(json.dumps({"cpu_full": res}), flush=True)


if __name__ == "__main__":
    a = parse()
    if a.profile_run:
        run_profile_target(a)
    elif a.cpu_full:
        run_cpu_full(a)
    elif a.impl == "reference":
        run_reference(a)
    else:
        run_ours(a)
