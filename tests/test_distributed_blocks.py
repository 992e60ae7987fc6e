"""Data blocks over two ranks (gloo, world size 2, CPU): the blocks are split by uv region
with paper_1610_08895_gb300.distributed.shard_blocks, each rank runs the dual steps of
its own blocks, the gridded dual contributions U_r = G_r^T v_r are summed by one
all-reduce, and every rank runs the same primal step (Sec. 3, "Implementation details").
The rank-local steps here are the oracle's operators; the iterate after the run must
equal the single-process oracle run of Algorithm 1."""
import os
import socket
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HERE = os.path.dirname(os.path.abspath(__file__))
NITER = 12


def _problem():
    from gpu_util import make_problem
    from oracle import pd as PD
    from paper_1610_08895_gb300 import synth
    prob, _ = make_problem(32, 3000, 8, 4, (0, 1, 2), 2, uv_kind="radial", blocks="annuli", nannuli=8)
    x0 = synth.start_vector(32, 32, seed=9)
    phi2, psi2 = PD.operator_norms(prob, x0, max_iter=300, tol=1e-10)
    kw = dict(tau=0.49, sigma=1.0 / psi2, varsigma=1.0 / phi2, kappa=1e-3, psi_norm=float(np.sqrt(psi2)), seed=3,
              p_block=[0.5] * 8, p_basis=[0.6] * 3)
    return prob, kw


class OracleShard:
    """Rank-local steps of Algorithm 1 with the oracle's operators: the dual updates of
    this rank's blocks (steps 5-9), the replicated sparsity update (steps 13-14), this
    rank's G_r^T v_r, and the replicated primal update (steps 17-18) from the summed U."""

    def __init__(self, prob, blocks, kw):
        from paper_1610_08895_gb300.distributed import local_visibilities
        g = prob.geom
        self.prob, self.kw = prob, kw
        self.blocks = [int(b) for b in blocks]
        self.vis = local_visibilities(prob.block_of_vis, blocks)
        self.pos = {int(m): k for k, m in enumerate(self.vis)}
        self.x = np.zeros((g.ny, g.nx))
        self.xt = np.zeros((g.ny, g.nx))
        self.s = np.zeros((len(prob.basis_ids), g.ny, g.nx))
        self.v = np.zeros(len(self.vis), dtype=np.complex128)
        self.t = 0

    def dual_step(self):
        from oracle import philox as PH
        from oracle import prox as PX
        from oracle import wavelets as W
        prob, kw, geo = self.prob, self.kw, self.prob.geom
        self.t += 1
        act = PH.active_set(kw["seed"], self.t, PH.STREAM_BLOCKS, kw["p_block"])
        actb = PH.active_set(kw["seed"], self.t, PH.STREAM_BASES, kw["p_basis"])
        b_tilde = geo.fft(geo.zpad(self.xt))
        for i in self.blocks:
            if act[i]:
                ix = prob.block_index[i]
                loc = np.array([self.pos[int(m)] for m in ix], dtype=np.int64)
                gb = geo.degrid(b_tilde, prob.uv[ix])
                self.v[loc] = PX.dual_data_update(self.v[loc], gb, prob.y[ix], prob.eps[i])
        b = len(prob.basis_ids)
        for k, j in enumerate(prob.basis_ids):
            if actb[k]:
                w = W.psi_j_adj(self.xt, j, prob.levels) / np.sqrt(b)
                self.s[k] = PX.dual_sparsity_update(self.s[k], w, kw["kappa"] * kw["psi_norm"])
        self.u_local = geo.grid(self.v, prob.uv[self.vis])

    def u_sum_buffer(self):
        return torch.view_as_real(torch.from_numpy(self.u_local.copy())).contiguous()

    def primal_step(self, u):
        from oracle import prox as PX
        geo, kw = self.prob.geom, self.kw
        U = torch.view_as_complex(u).numpy()
        back = np.real(geo.zpad_adj(geo.fft_adj(U)))
        x_new = PX.proj_positive(self.x - kw["tau"] * (kw["sigma"] * self.prob.psi(self.s) + kw["varsigma"] * back))
        self.xt = 2.0 * x_new - self.x
        self.x = x_new


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    for p in (ROOT, HERE):
        sys.path.insert(0, p)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import torch.distributed as dist
    from paper_1610_08895_gb300 import distributed as D
    dist.init_process_group("gloo", init_method="env://", rank=rank, world_size=world)
    prob, kw = _problem()
    shards = D.shard_blocks(prob.uv, prob.block_of_vis, prob.nblocks, world)
    eng = OracleShard(prob, shards[rank], kw)
    D.run(eng, NITER, lambda u: dist.all_reduce(u, op=dist.ReduceOp.SUM))
    out.put((rank, [int(b) for b in shards[rank]], eng.x))
    dist.barrier()
    dist.destroy_process_group()


def test_shards_are_contiguous_uv_regions_with_balanced_counts():
    from paper_1610_08895_gb300 import distributed as D
    from paper_1610_08895_gb300 import synth
    uv = synth.uv_radial(20000, seed=4)
    blk = synth.blocks_annuli(uv, 8, 4)
    groups = D.shard_blocks(uv, blk, 32, 2)
    assert sorted(np.concatenate(groups).tolist()) == list(range(32))
    counts = [np.isin(blk, g).sum() for g in groups]
    assert abs(counts[0] - counts[1]) < 0.2 * len(blk)
    ring = lambda g: set(int(b) // 4 for b in g)           # noqa: E731  (annulus of each block)
    assert max(ring(groups[0])) <= min(ring(groups[1]))     # inner annuli on one rank, outer on the other


def test_two_ranks_sum_the_gridded_duals_and_match_the_single_process_run():
    from oracle import pd as PD
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=300) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    res.sort()
    assert sorted(res[0][1] + res[1][1]) == list(range(8))     # every block on exactly one rank
    assert res[0][1] and res[1][1]
    sys.path.insert(0, HERE)
    prob, kw = _problem()
    st, _ = PD.pd_run(prob, NITER, **kw)
    for _, _, x in res:
        assert np.linalg.norm(x - st.x) / np.linalg.norm(st.x) < 1e-12
