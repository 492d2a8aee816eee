"""One stream's replicas sharded over two ranks, on CPU (gloo, world size 2),
with the FP64 oracle's steps.  The replicas are compressed and decomposed
independently (Sec. "Parallel Compression and Decomposition"), so each rank
keeps only the summaries Y_p of its own replicas, compresses every batch into
them, runs their CP-ALS and anchor match (Sec. "Factor match for
identifiability"), and the aligned Q x R blocks are all-gathered; every rank
then lifts A and B (Eq. 7), solves the new rows of C and updates G_p
redundantly.  The update equals the single-process oracle's bit for bit: the
per-replica steps are the same calls on the same inputs, and the exchange
moves fp64 arrays unchanged."""
import os
import socket

import numpy as np
import pytest

import oracle
from tests._cases import Case

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

CASE = Case(48, 40, 3, 4, 10, 3, 6, (5, 4, 6), 8, seed=77)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _sharded_run(rank, world):
    c = CASE
    d = c.make()
    P, Q, S = c.P, c.Q, c.S
    split = lambda M: [oracle.replica_block(np.asarray(M, np.float64), p, Q, S) for p in range(P)]
    mine = [p for p in range(P) if p % world == rank]
    U, V = split(d["U"]), split(d["V"])          # projections: known to every rank
    W0 = split(d["W"][0])
    Y = {p: oracle.compress(d["X"][:c.t_old], U[p], V[p], W0[p]) for p in mine}
    A = np.asarray(d["A0"], np.float64).copy()
    B = np.asarray(d["B0"], np.float64).copy()
    C = np.asarray(d["C0"], np.float64).copy()
    G = [W0[p].T @ C for p in range(P)]           # G_p of every replica, updated on every rank
    k = c.t_old
    out = []
    for b, t in enumerate(c.batches):
        Xb = d["X"][k:k + t]
        k += t
        Wb = split(d["W"][b + 1])
        for p in mine:
            Y[p] = Y[p] + oracle.compress(Xb, U[p], V[p], Wb[p])
        ref_a = (U[0].T @ A)[:S]                  # the anchor rows, as every replica sees them
        ref_b = (V[0].T @ B)[:S]
        hat_mine = {}
        for p in mine:
            At, Bt, Ct = oracle.cp_als(Y[p], U[p].T @ A, V[p].T @ B, c.iters)
            hat_mine[p] = oracle.align(At, Bt, Ct, ref_a, ref_b, S)
        gathered = [None] * world
        dist.all_gather_object(gathered, hat_mine)
        hat = {}
        for g in gathered:
            hat.update(g)
        assert sorted(hat) == list(range(P))
        hats = [hat[p] for p in range(P)]
        A_new = oracle.lift_factor(A, U, [h[0] for h in hats])
        B_new = oracle.lift_factor(B, V, [h[1] for h in hats])
        C_new = oracle.lift_C(Wb, [h[2] for h in hats], G)
        G = [G[p] + Wb[p].T @ C_new for p in range(P)]
        A, B, C = A_new, B_new, np.vstack([C, C_new])
        out.append((A, B, C))
    return out, {p: Y[p] for p in mine}


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        q.put((rank, *_sharded_run(rank, world)))
    finally:
        dist.destroy_process_group()


def test_replica_sharded_update_equals_single_process():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = [q.get(timeout=300) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    d = CASE.make()
    _, ref = CASE.oracle_run(d)
    for rank, states, Y in got:
        assert sorted(Y) == [p for p in range(CASE.P) if p % 2 == rank]
        for p, y in Y.items():
            assert np.array_equal(y, ref[-1]["Y"][p])
        for (A, B, C), r in zip(states, ref):
            assert np.array_equal(A, r["A"]) and np.array_equal(B, r["B"])
            assert np.array_equal(C, r["C"])
