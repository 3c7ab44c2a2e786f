"""The multi-rank partition of the hot path (paper_2212_05159_gb300.shard) on CPU with two
gloo ranks: row blocks of a power-law matrix balanced by entries, X all-gathered before
Y = A X, gA from the gathered X, and gX = A^T G reduce-scattered from every rank's partial.
The local products are the FP64 oracle's (the same orchestration drives the CUDA kernels
over NCCL); the reassembled Y, gA and gX must equal the unsharded oracle's.  Also the
data-parallel gradient all-reduce and the partition of independent systems.  Not run on
GPUs here: one GPU per run."""
import os
import socket
import sys

import numpy as np
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _matrix():
    import synth
    A = synth.powerlaw_csr(3000, seed=21, max_len=400)
    X = synth.normal((A.n, 6), seed=22).astype(np.float64)
    G = synth.normal((A.m, 6), seed=23).astype(np.float64)
    return A, X, G


def _rank_main(rank, ws, port, out):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    import oracle
    import synth
    from paper_2212_05159_gb300 import shard
    A, X, G = _matrix()
    sh = shard.RowSharded(A.indptr, A.m, A.n)
    e0, e1 = int(A.indptr[sh.r0]), int(A.indptr[sh.r1])
    Ar = synth.CSR(sh.r1 - sh.r0, A.n, A.indptr[sh.r0:sh.r1 + 1] - e0, A.indices[e0:e1], A.values[e0:e1])
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a))  # noqa: E731
    Y, Xfull = sh.forward(lambda Xf: t(oracle.spmm(Ar, Xf.numpy())), t(X[sh.c0:sh.c1]))
    gA, gX = sh.backward(lambda Gr, Xf: t(oracle.sddmm(Ar, Gr.numpy(), Xf.numpy())),
                         lambda Gr: t(oracle.spmm_t(Ar, Gr.numpy())), t(G[sh.r0:sh.r1]), Xfull)
    grad = torch.full((5,), float(rank + 1), dtype=torch.float64)
    shard.allreduce_gradients(grad)
    out.put((rank, sh.r0, sh.r1, sh.c0, sh.c1, Y.numpy(), gA.numpy(), gX.numpy(), grad.numpy(),
             bool(np.array_equal(Xfull.numpy(), X))))
    dist.destroy_process_group()


def test_two_ranks_reassemble_the_oracle_products():
    sys.path.insert(0, ROOT)
    import oracle
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted((q.get(timeout=180) for _ in procs), key=lambda x: x[0])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    A, X, G = _matrix()
    Y = np.concatenate([r[5] for r in res])
    gA = np.concatenate([r[6] for r in res])
    gX = np.concatenate([r[7] for r in res])
    assert res[0][1] == 0 and res[0][2] == res[1][1] and res[1][2] == A.m     # the row blocks tile A
    assert res[0][3] == 0 and res[0][4] == res[1][3] and res[1][4] == A.n     # the X slices tile X
    assert all(r[9] for r in res)                                             # X gathered exactly
    np.testing.assert_array_equal(Y, oracle.spmm(A, X))                       # rows whole on one rank
    np.testing.assert_array_equal(gA, oracle.sddmm(A, G, X))
    ref = oracle.spmm_t(A, G)
    np.testing.assert_allclose(gX, ref, rtol=0, atol=1e-12 * np.abs(ref).max())   # two partials summed
    for r in res:
        np.testing.assert_array_equal(r[8], np.full(5, 3.0))                  # 1 + 2


def test_row_blocks_balance_entries_and_systems_balance_cost():
    sys.path.insert(0, ROOT)
    import synth
    from paper_2212_05159_gb300 import shard
    A = synth.powerlaw_csr(20000, seed=3)
    lens = np.diff(A.indptr)
    for parts in (2, 3, 8):
        b = shard.row_blocks_by_nnz(A.indptr, parts)
        assert b[0] == 0 and b[-1] == A.m and np.all(np.diff(b) >= 0)
        counts = [int(A.indptr[b[p + 1]] - A.indptr[b[p]]) for p in range(parts)]
        assert max(counts) <= A.nnz / parts + lens.max()
    # a hub row holding most entries: blocks stay contiguous, some may be empty
    ip = np.array([0, 1, 1001, 1002, 1003])
    b = shard.row_blocks_by_nnz(ip, 4)
    assert b[0] == 0 and b[-1] == 4 and np.all(np.diff(b) >= 0)
    costs = [256 * 256 * 1000, 32 * 32 * 300, 128 * 128 * 700, 256 * 256 * 900, 64 * 64 * 500]
    parts = shard.partition_systems(costs, 2)
    assert sorted(sum(parts, [])) == list(range(5))
    loads = [sum(costs[i] for i in p) for p in parts]
    assert max(loads) - min(loads) <= max(costs)                              # largest-first greedy bound
    np.testing.assert_array_equal(shard.even_slices(10, 3), [0, 3, 6, 10])
