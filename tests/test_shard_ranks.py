"""The row-sharded step on CPU ranks (gloo, world sizes 2, 3 and 4).

Each rank owns a slab of whole z planes of the grid (the split op_step_sharded uses:
sizes differ by at most one plane, the first slabs take the extra planes) plus one halo
plane per neighbour.  The ranks run the exchange schedule of a row-sharded step with the
oracle's FP64 arithmetic on their own rows:
  - Step 1 (§4.1, p independent source problems): CG, preconditioned with diag(H + sigma)
    or not, warm-started from W; one halo exchange of W at the start and of the
    direction block per iteration; all-reduces of (r.z, r.r, u.u) at the start and of
    p.q and (r.z, r.r) per iteration;
  - Steps 2-3: all-reduce of the slab partials of <W,U> and <W,W>; the core computed on
    every rank from the sums (oracle.core_from_inner);
  - Step 4 on the own rows; one halo exchange of U+ and an all-reduce of the energy.
The result must equal the unsplit oracle step (block CG to the same tolerance) up to the
order of the sums, and the exchange counts must follow the schedule that the library's
op_shard_stats reports (halo rounds per step: CG iterations + 2; sums: 2 x iterations + 3).
"""
import os
import socket
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _split(nslow, ws, rank):
    own = [nslow // ws + (q < nslow % ws) for q in range(ws)]
    return sum(own[:rank]), own[rank]


class _Comm:
    """Halo exchanges and all-reduces of one rank, counted."""

    def __init__(self, rank, ws, plane, lo, own):
        self.rank, self.ws, self.plane, self.lo, self.own = rank, ws, plane, lo, own
        self.halo_copies = 0
        self.reductions = 0

    def exchange(self, X):
        pl, lo, own = self.plane, self.lo, self.own
        reqs, recv = [], {}
        if self.rank > 0:
            recv["lo"] = torch.empty((pl, X.shape[1]), dtype=torch.float64)
            reqs.append(dist.isend(torch.from_numpy(X[lo * pl:(lo + 1) * pl].copy()),
                                   self.rank - 1))
            reqs.append(dist.irecv(recv["lo"], self.rank - 1))
        if self.rank + 1 < self.ws:
            recv["hi"] = torch.empty((pl, X.shape[1]), dtype=torch.float64)
            reqs.append(dist.isend(torch.from_numpy(X[(lo + own - 1) * pl:(lo + own) * pl].copy()),
                                   self.rank + 1))
            reqs.append(dist.irecv(recv["hi"], self.rank + 1))
        for r in reqs:
            r.wait()
        if "lo" in recv:
            X[:pl] = recv["lo"].numpy()
        if "hi" in recv:
            X[(lo + own) * pl:(lo + own + 1) * pl] = recv["hi"].numpy()
        # count the copies of the whole job once (rank 0 counts every face)
        self.halo_copies += 2 * (self.ws - 1)

    def allreduce(self, a):
        t = torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64))
        dist.all_reduce(t)
        self.reductions += 1
        return t.numpy()


def _sharded_cg(A_loc, d_own, U_own, W_loc, own, comm, rtol, jacobi, max_iter=5000):
    """Block CG (block_cg / block_pcg_jacobi's iteration) on the rank's own rows."""
    comm.exchange(W_loc)
    R = U_own - (A_loc @ W_loc)[own]
    Z = R / d_own[:, None] if jacobi else R
    P_loc = np.zeros_like(W_loc)
    P_loc[own] = Z
    rho, rr, bb = comm.allreduce(np.stack([(R * Z).sum(0), (R * R).sum(0),
                                           (U_own * U_own).sum(0)]))
    target = rtol * rtol * bb
    W_own = W_loc[own]
    it = 0
    while it < max_iter:
        active = rr > target
        if not np.any(active):
            break
        comm.exchange(P_loc)
        Q = (A_loc @ P_loc)[own]
        pq = comm.allreduce((P_loc[own] * Q).sum(0))
        alpha = np.where(active & (pq > 0), rho / np.where(pq > 0, pq, 1.0), 0.0)
        W_own += P_loc[own] * alpha
        R -= Q * alpha
        Z = R / d_own[:, None] if jacobi else R
        rho_new, rr = comm.allreduce(np.stack([(R * Z).sum(0), (R * R).sum(0)]))
        beta = np.where(active & (rho > 0), rho_new / np.where(rho > 0, rho, 1.0), 0.0)
        P_loc[own] = Z + P_loc[own] * beta
        rho = rho_new
        it += 1
    return it


def _setup(shape, p, seed):
    import oracle as o
    import synthetic as syn
    lo, hi = (-6.0,) * 3, (6.0,) * 3
    V = syn.potential(shape, lo, hi, 0.5, syn.draw_wells(seed, 3, lo, hi))
    H = o.hamiltonian(shape, lo, hi, V)
    sigma = o.default_sigma(shape, lo, hi, V)
    tau = o.default_tau(shape, lo, hi, V, sigma)
    U = o.householder_orthonormalize(syn.gaussian_block(seed, H.shape[0], p))
    return H, sigma, tau, U


def _worker(rank, ws, port, out, shape, p, nsteps, jacobi):
    import scipy.sparse as sp

    import oracle as o
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(ws), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", init_method="env://", rank=rank, world_size=ws)
    try:
        rtol = 1e-13
        H, sigma, tau, U = _setup(shape, p, seed=7)
        n = H.shape[0]
        A = (H + sigma * sp.identity(n, format="csr")).tocsr()
        plane = shape[0] * shape[1]
        z0, own_planes = _split(shape[2], ws, rank)
        lo = 1 if rank > 0 else 0
        hi = 1 if rank + 1 < ws else 0
        rows = np.arange((z0 - lo) * plane, (z0 + own_planes + hi) * plane)
        own = slice(lo * plane, (lo + own_planes) * plane)
        A_loc = A[rows][:, rows]          # the stencil restricted to own + halo planes
        H_loc = H[rows][:, rows]
        d_own = A.diagonal()[rows][own]
        comm = _Comm(rank, ws, plane, lo, own_planes)
        U_loc = U[rows].copy()
        W_loc = np.zeros_like(U_loc)
        energies, iters = [], []
        for _ in range(nsteps):
            k = _sharded_cg(A_loc, d_own, U_loc[own], W_loc, own, comm, rtol, jacobi)
            iters.append(k)
            U_own, W_own = U_loc[own], W_loc[own]
            CS = comm.allreduce(np.stack([W_own.T @ U_own, W_own.T @ W_own]))
            Am, Bm, _ = o.core_from_inner(CS[0], CS[1], tau)
            U_loc[own] = o.update(U_own, W_own, Am, Bm, tau)
            comm.exchange(U_loc)
            e = comm.allreduce(np.array([(U_loc[own] * (H_loc @ U_loc)[own]).sum()]))
            energies.append(0.5 * float(e[0]))
        # the unsplit oracle steps from the same U, with the same CG and tolerance
        cg = o.block_pcg_jacobi if jacobi else o.block_cg
        Uf, Wf = U.copy(), np.zeros_like(U)
        ref_e, ref_it = [], []
        for _ in range(nsteps):
            Wf, k = cg(A, Uf, Wf, rtol)
            ref_it.append(k)
            Uf = o.scheme_step(Uf, Wf, tau)
            ref_e.append(o.energy(H, Uf))
        rows_own = rows[own]
        out.put((rank, float(np.abs(U_loc[own] - Uf[rows_own]).max()),
                 float(np.abs(W_loc[own] - Wf[rows_own]).max()), energies, ref_e, iters, ref_it,
                 comm.halo_copies, comm.reductions))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("ws,jacobi", [(2, True), (3, False), (4, True)],
                         ids=["ws2_jacobi", "ws3_cg", "ws4_jacobi"])
def test_row_sharded_step_on_gloo_ranks_matches_the_unsplit_step(ws, jacobi):
    shape, p, nsteps = (9, 8, 11), 5, 3
    port = free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, ws, port, q, shape, p, nsteps, jacobi))
             for r in range(ws)]
    for pr in procs:
        pr.start()
    res = sorted(q.get(timeout=180) for _ in range(ws))
    for pr in procs:
        pr.join(timeout=60)
        assert pr.exitcode == 0
    for rank, du, dw, e, e_ref, it, it_ref, halo, red in res:
        assert du <= 1e-12, (rank, du)
        assert dw <= 1e-11, (rank, dw)
        assert np.allclose(e, e_ref, rtol=1e-13, atol=0)
        assert all(abs(a - b) <= 1 for a, b in zip(it, it_ref))
        # the schedule op_step_sharded reports: per step, iterations + 2 halo rounds of
        # 2 (ws - 1) plane copies, and 2 iterations + 3 sums
        assert halo == sum(2 * (ws - 1) * (k + 2) for k in it)
        assert red == sum(2 * k + 3 for k in it)
    # every rank took the same iterations (the sums are global)
    assert len({tuple(r[5]) for r in res}) == 1
