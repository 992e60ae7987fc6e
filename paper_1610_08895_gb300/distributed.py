"""Data blocks spread over several GPUs (Sec. 3, "Implementation details": the data
blocks are processed in parallel and only their gridded dual contributions travel back
to the primal update).

Layout: the blocks are split over the ranks by uv region (contiguous ranges of blocks
ordered by the mean radius, then the mean angle, of their points, with near-equal
visibility counts), so each rank's gridded contribution covers a compact part of the
grid. Every rank plans only its own visibilities but with the global block count, so
the counter-based draws of Algorithm 1 step 3 are the same everywhere; the primal
variables x, x~ and the sparsity duals s are replicated (every rank runs the same
primal and sparsity updates on the same data). Per iteration the one exchange is a sum
over ranks of U_r = G_r^T v_r (the rank's gridded dual sum), a full complex grid of
Kx Ky elements: one all-reduce.

`run(engine, niter, all_reduce)` drives any rank-local engine (dual_step, u_sum_buffer,
primal_step); `GpuShard` is the engine on this library's C ABI.
"""
import ctypes

import numpy as np
import torch

from . import _binding as B
from .api import Plan, State, _need, _ptr, _stream


def shard_blocks(uv, block_of_vis, nblocks, world):
    """Global block ids of each rank: blocks ordered by (mean radius, mean angle) of their
    points and cut into `world` contiguous groups of near-equal visibility counts."""
    uv = np.asarray(uv, dtype=np.float64)
    blk = np.asarray(block_of_vis, dtype=np.int64)
    counts = np.bincount(blk, minlength=nblocks).astype(np.float64)
    r = np.bincount(blk, weights=np.hypot(uv[:, 0], uv[:, 1]), minlength=nblocks) / np.maximum(counts, 1)
    th = np.bincount(blk, weights=np.mod(np.arctan2(uv[:, 1], uv[:, 0]), 2 * np.pi), minlength=nblocks)
    th = th / np.maximum(counts, 1)
    order = np.lexsort((th, r))
    cum = np.cumsum(counts[order])
    total = cum[-1] if len(cum) else 0.0
    cut = [int(np.searchsorted(cum, total * (k + 1) / world, side="left")) + 1 for k in range(world - 1)]
    groups = np.split(order, cut)
    return [np.sort(g).astype(np.int64) for g in groups]


def local_visibilities(block_of_vis, blocks):
    """Indices (in the caller's order) of the visibilities of the given blocks."""
    return np.nonzero(np.isin(np.asarray(block_of_vis), blocks))[0]


def run(engine, niter, all_reduce):
    """niter iterations of Algorithm 1 across the ranks: each rank's dual steps, the sum
    of the gridded dual contributions over the ranks, then the replicated primal step."""
    for _ in range(niter):
        engine.dual_step()
        u = engine.u_sum_buffer()
        all_reduce(u)
        engine.primal_step(u)


class _DevArray:
    """__cuda_array_interface__ view of a device pointer (no copy, no ownership)."""

    def __init__(self, ptr, n, typestr):
        self.__cuda_array_interface__ = {"shape": (n,), "typestr": typestr, "data": (ptr, False), "version": 3}


class GpuShard:
    """Rank-local engine on the C ABI: the plan and state of this rank's visibilities."""

    def __init__(self, nx, ny, uv, block_of_vis, nblocks, blocks, iterate_kw, **plan_kw):
        self.vis = local_visibilities(block_of_vis, blocks)
        self.plan = Plan(nx, ny, np.asarray(uv)[self.vis], np.asarray(block_of_vis)[self.vis], nblocks, **plan_kw)
        self.state = State(self.plan)
        self.kw = dict(iterate_kw)
        p = self.plan
        pb = np.ascontiguousarray(self.kw.pop("p_block"), dtype=np.float64)
        ps = np.ascontiguousarray(self.kw.pop("p_basis"), dtype=np.float64)
        self._keep = (pb, ps)
        self.params = B.PdParams(p_block=pb.ctypes.data, p_basis=ps.ctypes.data, seed=int(self.kw.pop("seed", 0)),
                                 **{k: float(v) for k, v in self.kw.items()})
        ptr, n = ctypes.c_void_p(), ctypes.c_int64()
        B.call("pd_state_u", self.state._h, ctypes.byref(ptr), ctypes.byref(n))
        typestr = "<c8" if p.cplx_dtype == torch.complex64 else "<c16"
        self.u_local = torch.as_tensor(_DevArray(ptr.value, n.value, typestr), device="cuda")
        self.u_sum = torch.empty_like(self.u_local)

    def set_data(self, y, eps):
        """y: this rank's visibilities (device, in the order of self.vis); eps: every block's bound."""
        self.state.pd_state_set_data(y, eps)

    def dual_step(self):
        B.call("pd_iterate_dual", self.plan.handle, self.state._h, ctypes.byref(self.params), _stream())

    def u_sum_buffer(self):
        self.u_sum.copy_(self.u_local)
        return self.u_sum

    def primal_step(self, u):
        _need(u, self.u_local.dtype, tuple(self.u_local.shape), "u")
        B.call("pd_iterate_primal", self.plan.handle, self.state._h, ctypes.byref(self.params), _ptr(u), _stream())

    def x(self):
        return self.state.x()
