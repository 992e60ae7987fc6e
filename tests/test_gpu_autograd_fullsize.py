"""Phi as a torch.autograd.Function (backward = the CUDA gridding adjoint), and sampled
parity at the full bench workload (2048^2 image, 16.8M visibilities) in the launch
configuration bench.py times."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from gpu_util import TOL_OP32, rel  # noqa: E402
from oracle import experiment as EX  # noqa: E402
from oracle import measurement as meas  # noqa: E402
from oracle import philox as PH  # noqa: E402
from paper_1610_08895_gb300 import synth  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import __graft_entry__ as ge
    ge.build()
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"


def _plan(n, uv, blk, d, J, precision, bases=(0,), levels=1):
    from paper_1610_08895_gb300.api import Plan
    return Plan(n, n, uv, blk, d, kernel_width=J, basis_ids=list(bases), levels=levels, precision=precision)


@pytest.mark.parametrize("precision", ["f64", "f32"])
def test_phi_autograd_gradient_oracle_and_finite_differences(precision):
    from paper_1610_08895_gb300.autograd import phi
    n, m = 32, 3000
    uv = synth.uv_gaussian(m, seed=21)
    blk = np.zeros(m, np.int32)
    plan = _plan(n, uv, blk, 1, 8, precision)
    geo = meas.Geometry(n, n, 8)
    rng = np.random.default_rng(3)
    x0 = rng.uniform(0, 1, size=(n, n))
    yv = rng.normal(size=m) + 1j * rng.normal(size=m)
    rdt = plan.real_dtype
    x = torch.tensor(x0, dtype=rdt, device="cuda", requires_grad=True)
    y = torch.tensor(yv, dtype=plan.cplx_dtype, device="cuda")
    loss = 0.5 * (phi(x, plan) - y).abs().pow(2).sum()
    loss.backward()
    g = x.grad.detach().cpu().numpy()
    g_ref = geo.phi_adj(geo.phi(x0, uv) - yv, uv)          # oracle gradient of 1/2 ||Phi x - y||^2
    assert rel(g, g_ref) < (TOL_OP32 if precision == "f32" else 1e-11)
    # central differences, h = 1e-3, on 64 random pixels; the loss is summed in FP64
    h = 1e-3
    pix = rng.choice(n * n, size=64, replace=False)

    def L(xx):
        with torch.no_grad():
            r = plan.pd_apply_phi(xx).to(torch.complex128) - torch.tensor(yv, device="cuda")
            return 0.5 * float((r.abs() ** 2).sum())
    fd = []
    for p in pix:
        xp = x.detach().clone()
        xm = x.detach().clone()
        xp.view(-1)[p] += h
        xm.view(-1)[p] -= h
        fd.append((L(xp) - L(xm)) / (2 * h))
    fd = np.array(fd)
    # FP64: differences agree to rounding. FP32: the loss of an FP32 Phi carries rounding
    # noise of order 2^-24 sum_m |r_m| |(Phi x)_m|, amplified by 1/h in the difference
    # (measured 0.7% of the largest gradient entry here); the FP32 gradient itself was
    # checked against the FP64 oracle gradient above at 1e-5.
    tol = 1e-6 if precision == "f64" else 2e-2
    assert np.max(np.abs(fd - g.ravel()[pix])) <= tol * np.max(np.abs(g))


def test_phi_autograd_batch_of_eight_at_1024():
    """Config: 1024^2 image, 2048^2 grid, M = 4,194,304, J = 8, batch of 8 random images in [0, 1)."""
    from paper_1610_08895_gb300.autograd import phi
    n, m = 1024, 4_194_304
    uv = synth.uv_gaussian(m, seed=31)
    blk = np.zeros(m, np.int32)
    plan = _plan(n, uv, blk, 1, 8, "f32")
    xs = synth.random_images(8, n, n, seed=4)
    x = torch.tensor(xs, dtype=torch.float32, device="cuda", requires_grad=True)
    yv = phi(x, plan)
    cot = torch.tensor(synth.uniform_vis(m, seed=6, batch=8), dtype=torch.complex64, device="cuda")
    (yv.real * cot.real + yv.imag * cot.imag).sum().backward()     # d/dx Re<Phi x, c> = Re Phi^H c
    g = x.grad.detach()
    # adjoint identity over the batch, accumulated in FP64
    lhs = float((yv.detach().to(torch.complex128).conj() * cot.to(torch.complex128)).real.sum())
    rhs = float((x.detach().double() * g.double()).sum())
    assert abs(lhs - rhs) <= 1e-5 * abs(lhs)
    # the backward equals the adjoint entry point image by image
    g2 = plan.pd_apply_phi_adj(cot)
    assert torch.equal(g2, g)
    # FP64 oracle gradient of image 0 at 32 pixels, and of Phi at 2000 visibilities
    geo = meas.Geometry(n, n, 8)
    rng = np.random.default_rng(8)
    pix = [(int(a), int(b)) for a, b in rng.integers(0, n, size=(32, 2))]
    ref = geo.phi_adj_at(cot[0].cpu().numpy().astype(np.complex128), uv, pix)
    got = g[0].cpu().numpy()[tuple(np.array(pix).T)]
    assert np.max(np.abs(got - ref)) <= 1e-5 * np.sqrt(np.mean(g[0].double().cpu().numpy() ** 2))
    sel = rng.choice(m, size=2000, replace=False)
    y_ref = geo.degrid(geo.fft(geo.zpad(xs[0])), uv[sel])
    assert rel(yv[0].detach().cpu().numpy()[sel], y_ref) < TOL_OP32


def test_full_bench_workload_sampled_parity():
    """C5 in the bench configuration: 2048^2, 4096^2 grid, 16.8M radial visibilities in 256
    annulus x sector blocks, J = 8, 9 bases x 4 levels, p = 0.5 for blocks and bases."""
    from paper_1610_08895_gb300.api import State
    n, m = 2048, 16_777_216
    uv = synth.uv_radial(m, seed=1)
    blk = synth.blocks_annuli(uv, 32, 8)
    x_true = synth.test_image(n, seed=2)
    d = int(blk.max()) + 1
    plan = _plan(n, uv, blk, d, 8, "f32", bases=range(9), levels=4)
    geo = meas.Geometry(n, n, 8)
    # Phi on sampled visibilities
    y = plan.pd_apply_phi(torch.tensor(x_true, dtype=torch.float32, device="cuda"))
    rng = np.random.default_rng(1)
    sel = rng.choice(m, size=4000, replace=False)
    bt = geo.fft(geo.zpad(x_true))
    y_ref = geo.degrid(bt, uv[sel])
    assert rel(y.cpu().numpy()[sel], y_ref) < TOL_OP32
    del bt
    # measurements, bounds and one PD iteration from zero (graph mode, as in the bench)
    phix = y.cpu().numpy().astype(np.complex128)
    sn = EX.noise_sigma(phix, 30.0)
    yv = phix + sn * synth.complex_noise(m, seed=3)
    sizes = np.bincount(blk, minlength=d)
    eps = EX.epsilon_bounds(sn, np.maximum(sizes, 1))
    st = State(plan)
    st.pd_state_set_data(torch.tensor(yv, dtype=torch.complex64, device="cuda"), eps)
    tau, sigma, varsigma = 0.49, 1.0, 2.5e-8
    st.pd_iterate(1, tau=tau, sigma=sigma, varsigma=varsigma, kappa=1e-3, psi_norm=1.0, seed=0,
                  p_block=[0.5] * d, p_basis=[0.5] * 9, use_graph=True)
    x1 = st.x().cpu().numpy()
    rep = st.report()
    act = PH.active_set(0, 1, 0, [0.5] * d)
    assert list(rep["block_active"]) == act
    # x^(1) = max(0, tau varsigma Re Phi^H (sum over active blocks of c_i y_i)), c_i = max(0, 1 - eps_i/||y_i||)
    nrm = np.sqrt(np.bincount(blk, weights=np.abs(yv) ** 2, minlength=d))
    c = np.where(np.array(act) & (nrm > eps), 1.0 - eps / np.maximum(nrm, 1e-300), 0.0)
    w = c[blk] * yv
    pix = [(1024, 1024), (1000, 1100), (700, 1500), (1300, 900), (512, 512), (1600, 400)]
    ref = np.maximum(0.0, tau * varsigma * geo.phi_adj_at(w, uv, pix))
    got = x1[tuple(np.array(pix).T)]
    scale = np.sqrt(np.mean(x1.astype(np.float64) ** 2))
    assert scale > 0
    assert np.max(np.abs(got - ref)) <= 1e-4 * max(scale, np.max(np.abs(ref)))
