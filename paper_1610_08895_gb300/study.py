"""Synthetic convergence studies of Algorithm 1 on the GPU path (the analogues of the
paper's Sec. 5 experiments, on synthetic data: the M31 image is not used).

Reconstruction SNR = 20 log10(||x_true|| / ||x_true - x^(t)||) against iteration t:

* ``uniform``: 256^2 image, 65,536 Gaussian uv points in 16 equal blocks, every
  block drawn with the same probability p in {1, 0.75, 0.5, 0.25} (Sec. 5, Fig. 2).
* ``adaptive``: 512^2 image, 1,048,576 radially decaying uv points in 64 equal-width
  annuli (uneven blocks); uniform p = n/d against the adaptive probabilities of
  Sec. 4 with the same budget n = d/4 (p_min = 0.05, p_max = 0.5), with c_i taken
  from the last pass of each block (lagged) or from Phi_i x^(t) (exact), and a
  baseline that only ever updates the 16 innermost (low-frequency) annuli (Fig. 3).

Every run uses 9 bases (Dirac, db1-db8) x 4 levels, J = 8, 30 dB noise, tau = 0.49,
sigma = 1/||Psi||^2, varsigma = 1/||Phi||^2, kappa = 1e-3.

    python -m paper_1610_08895_gb300.study [--iters 2000] [--every 100] [--which uniform,adaptive]

prints one markdown table per study (SNR in dB at each reported iteration, and the
mean number of active blocks per iteration). The CUDA library must be built first
(``python -c "import __graft_entry__ as g; g.build()"``).
"""
import argparse
import json

import numpy as np


def _problem(n, m, uv_kind, nannuli, nblocks_equal, seed=0, snr=30.0):
    import torch
    from scipy.stats import chi2

    from . import synth
    from .api import Plan, State
    uv = synth.uv_gaussian(m, seed=seed + 1) if uv_kind == "gaussian" else synth.uv_radial(m, seed=seed + 1)
    blk = synth.blocks_equal(uv, nblocks_equal) if nannuli is None else synth.blocks_annuli(uv, nannuli, 1)
    d = int(blk.max()) + 1
    x_true = synth.test_image(n, seed=seed + 2)
    plan = Plan(n, n, uv, blk, d, kernel_width=8, basis_ids=list(range(9)), levels=4, precision="f32")
    xt = torch.tensor(x_true, dtype=torch.float32, device="cuda")
    phix = plan.pd_apply_phi(xt).to(torch.complex128)
    sig = float(torch.linalg.vector_norm(phix)) / np.sqrt(m) * 10 ** (-snr / 20)
    y = (phix.cpu().numpy() + sig * synth.complex_noise(m, seed=seed + 3)).astype(np.complex64)
    sizes = np.maximum(np.bincount(blk, minlength=d), 1).astype(np.float64)
    eps = sig / np.sqrt(2.0) * np.sqrt(chi2.ppf(0.99, 2.0 * sizes))
    x0 = torch.tensor(synth.start_vector(n, n, seed=9), dtype=torch.float32, device="cuda")
    phi2, psi2, _ = plan.pd_operator_norms(x0, max_iter=200, tol=1e-6)
    steps = dict(tau=0.49, sigma=1.0 / psi2, varsigma=1.0 / phi2, kappa=1e-3, psi_norm=float(np.sqrt(psi2)))
    return plan, State, torch.tensor(y, device="cuda"), eps, x_true, d, steps


def _run(plan, State, y, eps, x_true, steps, iters, every, **iterate_kw):
    import torch
    st = State(plan)
    st.pd_state_set_data(y, eps)
    xt = torch.tensor(x_true, dtype=torch.float64, device="cuda")
    nrm = float(torch.linalg.vector_norm(xt))
    snr, active = [], 0.0
    done = 0
    while done < iters:
        k = min(every, iters - done)
        for _ in range(k):
            st.pd_iterate(1, **steps, **iterate_kw)
            active += float(st.report()["block_active"].sum())
        done += k
        err = float(torch.linalg.vector_norm(st.x().to(torch.float64) - xt))
        snr.append((done, 20.0 * np.log10(nrm / max(err, 1e-300))))
    st.close()
    return snr, active / iters


def _table(title, runs):
    its = [t for t, _ in next(iter(runs.values()))[0]]
    head = "| run | mean active blocks | " + " | ".join(f"t={t}" for t in its) + " |"
    sep = "|---|---|" + "---|" * len(its)
    rows = [f"| {name} | {act:.2f} | " + " | ".join(f"{v:.2f}" for _, v in snr) + " |"
            for name, (snr, act) in runs.items()]
    return "\n".join([f"### {title}", "", head, sep] + rows)


def uniform_study(iters, every):
    plan, State, y, eps, x_true, d, steps = _problem(256, 65536, "gaussian", None, 16)
    runs = {}
    for p in (1.0, 0.75, 0.5, 0.25):
        runs[f"p = {p}"] = _run(plan, State, y, eps, x_true, steps, iters, every, seed=0,
                                p_block=[p] * d, p_basis=[1.0] * 9, use_graph=False)
    plan.close()
    return _table("SNR (dB) against iteration, uniform block probabilities (256², 16 equal blocks)", runs)


def adaptive_study(iters, every):
    plan, State, y, eps, x_true, d, steps = _problem(512, 1_048_576, "radial", 64, None)
    n = d / 4.0
    ad = {"n": n, "p_min": 0.05, "p_max": 0.5}
    inner = [1.0 if i < 16 else 1e-12 for i in range(d)]
    runs = {
        f"uniform p = {n / d:g}": _run(plan, State, y, eps, x_true, steps, iters, every, seed=0,
                                       p_block=[n / d] * d, p_basis=[1.0] * 9),
        "adaptive, lagged c_i": _run(plan, State, y, eps, x_true, steps, iters, every, seed=0,
                                     p_basis=[1.0] * 9, adaptive=ad),
        "adaptive, exact c_i": _run(plan, State, y, eps, x_true, steps, iters, every, seed=0,
                                    p_basis=[1.0] * 9, adaptive=dict(ad, exact=True)),
        "16 innermost annuli only": _run(plan, State, y, eps, x_true, steps, iters, every, seed=0,
                                         p_block=inner, p_basis=[1.0] * 9),
        "p = 1 (all blocks)": _run(plan, State, y, eps, x_true, steps, iters, every, seed=0,
                                   p_block=[1.0] * d, p_basis=[1.0] * 9),
    }
    plan.close()
    return _table("SNR (dB) against iteration, adaptive vs uniform (512², 64 annuli, budget n = 16)", runs)


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--iters", type=int, default=2000)
    ap.add_argument("--every", type=int, default=250)
    ap.add_argument("--which", default="uniform,adaptive")
    a = ap.parse_args(argv)
    out = []
    if "uniform" in a.which:
        out.append(uniform_study(a.iters, a.every))
    if "adaptive" in a.which:
        out.append(adaptive_study(a.iters, a.every))
    print("\n\n".join(out))
    return out


if __name__ == "__main__":
    main()
