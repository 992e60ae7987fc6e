"""Python face of the PD-R CUDA library: Plan and State over torch CUDA tensors.

Marshalling only: shapes and dtypes are checked, pointers and the current
stream are handed to the C ABI (include/pd.h), and every computation runs in
the library's kernels. Method names follow the C entry points.
"""
import ctypes

import numpy as np
import torch

from . import _binding as B

_REAL = {B.PD_F32: torch.float32, B.PD_F64: torch.float64}
_CPLX = {B.PD_F32: torch.complex64, B.PD_F64: torch.complex128}


def _stream():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr())


def _need(t, dtype, shape, name):
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must have dtype {dtype}, got {t.dtype}")
    if tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} must have shape {tuple(shape)}, got {tuple(t.shape)}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")


# kernel phases timed by pd_iterate(profile=True) (pd_phase_name 0 .. N_PHASES - 1)
N_PHASES = 11

_G_MODE = {"on_the_fly": B.PD_G_ON_THE_FLY, "csr": B.PD_G_CSR}


class Plan:
    """pd_plan_create: image size, oversampling 2, uv points, blocks, kernel width, bases.

    g_mode "on_the_fly" evaluates the Kaiser-Bessel weights of G in the kernels; "csr"
    builds G once as a sparse matrix on the device (J^2 column/weight pairs per
    visibility, J <= 8) and reads it in every application. dde_kernels (with "csr"):
    complex [nvis, d, d] Fourier-domain DDE kernels, d odd, user order; G's row m is
    then the interpolation kernel convolved with kernel m (J + d - 1 <= 8)."""

    def __init__(self, nx, ny, uv, block_of_vis, nblocks, kernel_width=8, basis_ids=(0,), levels=1,
                 precision="f32", tile=0, kb_beta=0.0, g_mode="on_the_fly", dde_kernels=None):
        B.load()
        self.nx, self.ny = int(nx), int(ny)
        self.uv = np.ascontiguousarray(uv, dtype=np.float64)
        self.block_of_vis = np.ascontiguousarray(block_of_vis, dtype=np.int32)
        self.nvis = len(self.uv)
        self.nblocks = int(nblocks)
        self.basis_ids = np.ascontiguousarray(basis_ids, dtype=np.int32)
        self.nbases = len(self.basis_ids)
        self.levels = int(levels)
        self.prec = {"f32": B.PD_F32, "f64": B.PD_F64}[precision] if isinstance(precision, str) else int(precision)
        self.real_dtype = _REAL[self.prec]
        self.cplx_dtype = _CPLX[self.prec]
        if g_mode not in _G_MODE:
            raise ValueError(f"g_mode must be one of {sorted(_G_MODE)}, got {g_mode!r}")
        self.g_mode = g_mode
        dde_w, dde_ptr = 0, None
        if dde_kernels is not None:
            self.dde = np.ascontiguousarray(dde_kernels, dtype=np.complex128)
            if self.dde.ndim != 3 or self.dde.shape[0] != self.nvis or self.dde.shape[1] != self.dde.shape[2]:
                raise ValueError(f"dde_kernels must have shape (nvis, d, d), got {self.dde.shape}")
            dde_w, dde_ptr = self.dde.shape[1], self.dde.ctypes.data
        d = B.PdPlanDesc(nx=self.nx, ny=self.ny, osf=2, nvis=self.nvis, uv=self.uv.ctypes.data,
                         nblocks=self.nblocks, block_of_vis=self.block_of_vis.ctypes.data,
                         kernel_width=int(kernel_width), kb_beta=float(kb_beta), nbases=self.nbases,
                         basis_ids=self.basis_ids.ctypes.data, levels=self.levels, precision=self.prec,
                         tile=int(tile), g_mode=_G_MODE[g_mode], dde_width=dde_w, dde_kernels=dde_ptr)
        h = ctypes.c_void_p()
        B.call("pd_plan_create", ctypes.byref(d), ctypes.byref(h))
        self._h = h

    @property
    def handle(self):
        return self._h

    def info(self):
        ky, kx, tile = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
        beta = ctypes.c_double()
        ns, nc, nb = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
        B.call("pd_plan_info", self._h, ctypes.byref(ky), ctypes.byref(kx), ctypes.byref(beta),
               ctypes.byref(tile), ctypes.byref(ns), ctypes.byref(nc), ctypes.byref(nb))
        return {"ky": ky.value, "kx": kx.value, "beta": beta.value, "tile": tile.value,
                "nsegments": ns.value, "ntiles_nonempty": nc.value, "device_bytes": nb.value}

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            B.load().pd_plan_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ---- operators
    def pd_apply_phi(self, x, y=None):
        """y = Phi x for x of shape [ny, nx] or [batch, ny, nx]."""
        batch = x.shape[0] if x.dim() == 3 else 1
        _need(x, self.real_dtype, (batch, self.ny, self.nx) if x.dim() == 3 else (self.ny, self.nx), "x")
        shape = (batch, self.nvis) if x.dim() == 3 else (self.nvis,)
        if y is None:
            y = torch.empty(shape, dtype=self.cplx_dtype, device=x.device)
        _need(y, self.cplx_dtype, shape, "y")
        B.call("pd_apply_phi", self._h, _ptr(x), _ptr(y), batch, _stream())
        return y

    def pd_apply_phi_adj(self, y, x=None):
        """x = Re(Phi^H y) for y of shape [nvis] or [batch, nvis]."""
        batch = y.shape[0] if y.dim() == 2 else 1
        _need(y, self.cplx_dtype, (batch, self.nvis) if y.dim() == 2 else (self.nvis,), "y")
        shape = (batch, self.ny, self.nx) if y.dim() == 2 else (self.ny, self.nx)
        if x is None:
            x = torch.empty(shape, dtype=self.real_dtype, device=y.device)
        _need(x, self.real_dtype, shape, "x")
        B.call("pd_apply_phi_adj", self._h, _ptr(y), _ptr(x), batch, _stream())
        return x

    def pd_apply_psi_adj(self, x, coeffs=None):
        _need(x, self.real_dtype, (self.ny, self.nx), "x")
        if coeffs is None:
            coeffs = torch.empty((self.nbases, self.ny, self.nx), dtype=self.real_dtype, device=x.device)
        _need(coeffs, self.real_dtype, (self.nbases, self.ny, self.nx), "coeffs")
        B.call("pd_apply_psi_adj", self._h, _ptr(x), _ptr(coeffs), _stream())
        return coeffs

    def pd_sara_weights(self, x, delta, weights=None):
        """pd_sara_weights: delta / (delta + |Psi^H x|) per coefficient, [nbases, ny, nx]."""
        _need(x, self.real_dtype, (self.ny, self.nx), "x")
        if weights is None:
            weights = torch.empty((self.nbases, self.ny, self.nx), dtype=self.real_dtype, device=x.device)
        _need(weights, self.real_dtype, (self.nbases, self.ny, self.nx), "weights")
        B.call("pd_sara_weights", self._h, _ptr(x), ctypes.c_double(float(delta)), _ptr(weights), _stream())
        return weights

    def pd_apply_psi(self, coeffs, x=None):
        _need(coeffs, self.real_dtype, (self.nbases, self.ny, self.nx), "coeffs")
        if x is None:
            x = torch.empty((self.ny, self.nx), dtype=self.real_dtype, device=coeffs.device)
        _need(x, self.real_dtype, (self.ny, self.nx), "x")
        B.call("pd_apply_psi", self._h, _ptr(coeffs), _ptr(x), _stream())
        return x

    def pd_operator_norms(self, x0, max_iter=1000, tol=1e-8):
        """(||Phi||_S^2, ||Psi||_S^2, iterations) by the power method from x0."""
        _need(x0, self.real_dtype, (self.ny, self.nx), "x0")
        a, b, it = ctypes.c_double(), ctypes.c_double(), ctypes.c_int32()
        st = B.load().pd_operator_norms(self._h, _ptr(x0), int(max_iter), float(tol), ctypes.byref(a),
                                        ctypes.byref(b), ctypes.byref(it), _stream())
        if st not in (B.PD_OK, B.PD_ENOTCONV):
            B.check(st, "pd_operator_norms")
        return a.value, b.value, it.value


class State:
    """Algorithm 1 state (pd_state_create / pd_state_set_data / pd_iterate)."""

    def __init__(self, plan):
        self.plan = plan
        h = ctypes.c_void_p()
        B.call("pd_state_create", plan.handle, ctypes.byref(h))
        self._h = h

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            B.load().pd_state_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def pd_state_set_data(self, y, eps):
        p = self.plan
        _need(y, p.cplx_dtype, (p.nvis,), "y")
        eps = np.ascontiguousarray(eps, dtype=np.float64)
        if eps.shape != (p.nblocks,):
            raise ValueError("eps must have one entry per block")
        B.call("pd_state_set_data", p.handle, self._h, _ptr(y), eps.ctypes.data, _stream())

    def pd_state_set_start(self, x0=None, x_tilde0=None, s0=None, v0=None):
        """Start values x^(0), x~^(0), s^(0), v^(0) (None = zero); call after pd_state_set_data."""
        p = self.plan
        args = []
        for t, dt, shape, name in ((x0, p.real_dtype, (p.ny, p.nx), "x0"),
                                   (x_tilde0, p.real_dtype, (p.ny, p.nx), "x_tilde0"),
                                   (s0, p.real_dtype, (p.nbases, p.ny, p.nx), "s0"),
                                   (v0, p.cplx_dtype, (p.nvis,), "v0")):
            if t is None:
                args.append(ctypes.c_void_p())
            else:
                _need(t, dt, shape, name)
                args.append(_ptr(t))
        B.call("pd_state_set_start", p.handle, self._h, *args, _stream())

    def pd_iterate(self, niter, tau, sigma, varsigma, kappa, psi_norm=1.0, seed=0, p_block=None, p_basis=None,
                   adaptive=None, use_graph=False, profile=False, per_block=False, weights=None):
        """pd_iterate. weights: None (l1 prior) or a device tensor [nbases, ny, nx] of the
        reweighted prior's per-coefficient weights (kept referenced by the state, since a
        captured graph reads it on every replay)."""
        p = self.plan
        if weights is not None:
            _need(weights, p.real_dtype, (p.nbases, p.ny, p.nx), "weights")
        self._weights = weights
        pb = np.ascontiguousarray(np.ones(p.nblocks) if p_block is None else p_block, dtype=np.float64)
        ps = np.ascontiguousarray(np.ones(p.nbases) if p_basis is None else p_basis, dtype=np.float64)
        prm = B.PdParams(tau=tau, sigma=sigma, varsigma=varsigma, kappa=kappa, psi_norm=psi_norm, seed=int(seed),
                         p_block=pb.ctypes.data, p_basis=ps.ctypes.data, adaptive=0, adapt_n=0.0,
                         adapt_p_min=0.0, adapt_p_max=0.0, use_graph=int(bool(use_graph)),
                         profile=int(bool(profile)), per_block=int(bool(per_block)),
                         sparsity_weights=None if weights is None else weights.data_ptr())
        if adaptive is not None:
            prm.adaptive = 1
            prm.adapt_n = float(adaptive["n"])
            prm.adapt_p_min = float(adaptive["p_min"])
            prm.adapt_p_max = float(adaptive["p_max"])
            prm.adapt_exact = int(bool(adaptive.get("exact", False)))
        B.call("pd_iterate", p.handle, self._h, ctypes.byref(prm), int(niter), _stream())

    def pd_synthesis_iterate(self, niter, tau, sigma, varsigma, kappa, seed=0, p_block=None):
        """pd_synthesis_iterate: the synthesis formulation (x = Psi alpha, l1 on alpha,
        positivity as a dual); alpha is read with s(), the image with x()."""
        p = self.plan
        pb = np.ascontiguousarray(np.ones(p.nblocks) if p_block is None else p_block, dtype=np.float64)
        prm = B.PdParams(tau=tau, sigma=sigma, varsigma=varsigma, kappa=kappa, psi_norm=1.0, seed=int(seed),
                         p_block=pb.ctypes.data, p_basis=None)
        B.call("pd_synthesis_iterate", p.handle, self._h, ctypes.byref(prm), int(niter), _stream())

    def x(self):
        p = self.plan
        out = torch.empty((p.ny, p.nx), dtype=p.real_dtype, device="cuda")
        B.call("pd_state_get_x", self._h, _ptr(out), _stream())
        return out

    def x_tilde(self):
        p = self.plan
        out = torch.empty((p.ny, p.nx), dtype=p.real_dtype, device="cuda")
        B.call("pd_state_get_x_tilde", self._h, _ptr(out), _stream())
        return out

    def s(self):
        p = self.plan
        out = torch.empty((p.nbases, p.ny, p.nx), dtype=p.real_dtype, device="cuda")
        B.call("pd_state_get_s", self._h, _ptr(out), _stream())
        return out

    def v(self):
        p = self.plan
        out = torch.empty((p.nvis,), dtype=p.cplx_dtype, device="cuda")
        B.call("pd_state_get_v", p.handle, self._h, _ptr(out), _stream())
        return out

    def report(self):
        p = self.plan
        t, dx2, x2 = ctypes.c_int64(), ctypes.c_double(), ctypes.c_double()
        res = np.zeros(p.nblocks)
        pb = np.zeros(p.nblocks)
        ba = np.zeros(p.nblocks, dtype=np.int32)
        sa = np.zeros(p.nbases, dtype=np.int32)
        work = np.zeros(2, dtype=np.int32)
        B.call("pd_state_report", p.handle, self._h, ctypes.byref(t), ctypes.byref(dx2), ctypes.byref(x2),
               res.ctypes.data, pb.ctypes.data, ba.ctypes.data, sa.ctypes.data, work.ctypes.data, _stream())
        return {"t": t.value, "dx2": dx2.value, "x2": x2.value, "res_norm": res, "p_block": pb,
                "block_active": ba.astype(bool), "basis_active": sa.astype(bool),
                "active_segments": int(work[0]), "active_tiles": int(work[1])}

    def profile(self, reset=False):
        """{phase name: (total ms, iterations)} from iterations run with profile=True."""
        ms = np.zeros(N_PHASES)
        n = np.zeros(N_PHASES, dtype=np.int64)
        B.call("pd_state_profile", self._h, ms.ctypes.data, n.ctypes.data, N_PHASES, int(bool(reset)))
        lib = B.load()
        return {lib.pd_phase_name(k).decode(): (float(ms[k]), int(n[k])) for k in range(N_PHASES)}

    def save(self):
        p = self.plan
        n = B.load().pd_state_bytes(p.handle)
        buf = np.zeros(n, dtype=np.uint8)
        B.call("pd_state_save", p.handle, self._h, buf.ctypes.data, _stream())
        return buf

    def load(self, buf):
        buf = np.ascontiguousarray(buf, dtype=np.uint8)
        B.call("pd_state_load", self.plan.handle, self._h, buf.ctypes.data, _stream())


def autotune_tile(nx, ny, uv, block_of_vis, nblocks, kernel_width=8, basis_ids=(0,), levels=1, precision="f32",
                  candidates=(16, 32, 64), iters=5):
    """pd_plan_autotune: time Algorithm 1 iterations with each candidate gridding tile
    and return (best tile, {tile: ms per iteration})."""
    B.load()
    uv = np.ascontiguousarray(uv, dtype=np.float64)
    blk = np.ascontiguousarray(block_of_vis, dtype=np.int32)
    ids = np.ascontiguousarray(basis_ids, dtype=np.int32)
    prec = {"f32": B.PD_F32, "f64": B.PD_F64}[precision] if isinstance(precision, str) else int(precision)
    d = B.PdPlanDesc(nx=int(nx), ny=int(ny), osf=2, nvis=len(uv), uv=uv.ctypes.data, nblocks=int(nblocks),
                     block_of_vis=blk.ctypes.data, kernel_width=int(kernel_width), kb_beta=0.0, nbases=len(ids),
                     basis_ids=ids.ctypes.data, levels=int(levels), precision=prec, tile=0)
    cand = np.ascontiguousarray(candidates, dtype=np.int32)
    ms = np.zeros(len(cand))
    best = ctypes.c_int32()
    B.call("pd_plan_autotune", ctypes.byref(d), cand.ctypes.data, len(cand), int(iters), ctypes.byref(best),
           ms.ctypes.data, _stream())
    return best.value, {int(c): float(t) for c, t in zip(cand, ms)}


def psi_adj_noalloc(x, basis_ids, levels, coeffs=None):
    """Psi^H x through pd_apply_psi_adj_noalloc: no plan, no device allocation by the
    library (coeffs must be passed in by callers that cannot allocate)."""
    if not isinstance(x, torch.Tensor) or not x.is_cuda or x.dim() != 2 or not x.is_contiguous():
        raise TypeError("x must be a contiguous 2-D CUDA tensor")
    prec = {torch.float32: B.PD_F32, torch.float64: B.PD_F64}[x.dtype]
    ids = np.ascontiguousarray(basis_ids, dtype=np.int32)
    ny, nx = x.shape
    if coeffs is None:
        coeffs = torch.empty((len(ids), ny, nx), dtype=x.dtype, device=x.device)
    _need(coeffs, x.dtype, (len(ids), ny, nx), "coeffs")
    B.call("pd_apply_psi_adj_noalloc", _ptr(x), _ptr(coeffs), nx, ny, int(levels), ids.ctypes.data, len(ids), prec,
           _stream())
    return coeffs


def daubechies_filter(k):
    """Low-pass filter of db_k as derived by the library (host)."""
    h = np.zeros(2 * k)
    B.call("pd_daubechies_filter", int(k), h.ctypes.data)
    return h
