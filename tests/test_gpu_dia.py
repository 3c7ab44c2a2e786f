"""PCG with M = L L^T (Section 4.3), L in diagonal form (spx_dia_analyse, spx_dia_fill), M's
lower diagonals formed from it (spx_dia_square) and kept in shared memory by the PCG
(spx_cg_batched_dia), against the FP64 oracle's PCG with the same BF16-rounded factor:
systems large enough that a cluster has several blocks (rows of q and of M read from the
neighbouring blocks), and the unsupported cases reported per system."""
import numpy as np
import pytest
import torch

import oracle
import synth

pytestmark = pytest.mark.gpu
spx = pytest.importorskip("paper_2212_05159_gb300")
from paper_2212_05159_gb300 import abi, solve  # noqa: E402


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def host(t):
    return t.detach().cpu().numpy()


def _bf16(a):
    return torch.from_numpy(np.asarray(a, np.float32)).to(torch.bfloat16).to(torch.float32).numpy()


def _factor(A, seed, spread=0.2):
    """A random lower-triangular factor on tril(A): diagonal ~ a_ii^-1/2, the rest small."""
    l_ip, l_ix, _ = oracle.tril_pattern(A)
    rows = np.repeat(np.arange(A.m), np.diff(l_ip))
    d = oracle.diagonal(A)
    rng = np.random.default_rng(seed)
    v = rng.uniform(-spread, spread, l_ix.size) / np.sqrt(d[rows])
    on = rows == l_ix
    v[on] = (1.0 + rng.uniform(-0.1, 0.1, int(on.sum()))) / np.sqrt(d[rows[on]])
    return synth.CSR(A.m, A.m, l_ip, l_ix, v.astype(np.float32))


def _block(M, ptr, s):
    a, c = int(ptr[s]), int(ptr[s + 1])
    e0, e1 = int(M.indptr[a]), int(M.indptr[c])
    return synth.CSR(c - a, c - a, M.indptr[a:c + 1] - e0, M.indices[e0:e1] - a, M.values[e0:e1]), a, c


def _batch(sides, seed):
    mats = [synth.diffusion2d(s, 1.0, seed + i) for i, s in enumerate(sides)]
    return synth.block_diag(mats)


def test_analyse_and_fill_are_exact():
    sides = [1, 2, 7, 33]
    A, ptr = _batch(sides, 4)
    L = _factor(A, seed=5)
    batch = solve.SystemBatch(spx.CSR.from_host(A), ptr)
    dL = spx.CSR.from_host(L)
    F = solve.DiagonalFactor(batch, dL)
    assert F.supported
    offs, nd = host(F.offsets).reshape(-1, 3), host(F.nd)
    for s, side in enumerate(sides):
        want = [0, -1, -side] if side > 1 else [0]
        assert nd[s] == len(want) and list(offs[s, :nd[s]]) == want, (s, offs[s], nd[s])
    F.fill(dL.values)
    got = host(F.values.view(torch.int16)).reshape(3, -1)
    ref = np.zeros((3, A.m), np.float32)
    rows = np.repeat(np.arange(A.m), np.diff(L.indptr))
    sys_of = np.searchsorted(ptr, rows, side="right") - 1
    for e in range(L.nnz):
        d = list(offs[sys_of[e], :nd[sys_of[e]]]).index(int(L.indices[e]) - int(rows[e]))
        ref[d, rows[e]] = L.values[e]
    ref16 = torch.from_numpy(ref).to(torch.bfloat16).view(torch.int16).numpy()
    np.testing.assert_array_equal(got, ref16)


def test_square_forms_the_lower_diagonals_of_L_LT_exactly():
    """M = L L^T from L's BF16 diagonals: the distances 0, 1, N - 1, N of a 5-point grid of side
    N (fewer for tiny systems), and every value the FP32 sum, in (d, e) order, of the exact
    products of L's BF16 values, rounded to BF16 -- bit for bit."""
    sides = [1, 2, 7, 33]
    A, ptr = _batch(sides, 4)
    L = _factor(A, seed=6)
    batch = solve.SystemBatch(spx.CSR.from_host(A), ptr)
    dL = spx.CSR.from_host(L)
    F = solve.DiagonalFactor(batch, dL).fill(dL.values)
    loffs, lnd = host(F.offsets).reshape(-1, 3), host(F.nd)
    moffs, mnd = host(F.m_offsets).reshape(-1, 4), host(F.m_nd)
    Ld = host(F.values.float()).reshape(3, -1).astype(np.float32)
    got = host(F.m_values.view(torch.int16)).reshape(4, -1)
    ref = np.zeros((4, A.m), np.float32)
    for s, side in enumerate(sides):
        sd = [-int(o) for o in loffs[s, :lnd[s]]]
        want = sorted({0} | {a - b for a in sd for b in sd if a > b})
        assert mnd[s] == len(want) and list(moffs[s, :mnd[s]]) == want, (s, moffs[s], mnd[s])
        for i in range(int(ptr[s]), int(ptr[s + 1])):
            for q, o in enumerate(want):
                t = np.float32(0.0)
                if i - o >= ptr[s]:
                    for d in range(lnd[s]):
                        for e in range(lnd[s]):
                            if sd[d] - sd[e] == o:
                                t = np.float32(t + np.float32(Ld[d, i] * Ld[e, i - o]))
                ref[q, i] = t
    ref16 = torch.from_numpy(ref).to(torch.bfloat16).view(torch.int16).numpy()
    np.testing.assert_array_equal(got, ref16)


@pytest.mark.parametrize("sides", [[40, 100, 130, 64, 7], [256, 256]])
def test_dia_pcg_matches_oracle(sides):
    """Every system to a true residual of 1e-8 in about as many iterations as the FP64
    oracle's PCG with the BF16-rounded factor; the 130^2 system spans 4 blocks, 256^2 8."""
    A, ptr = _batch(sides, 11)
    L = _factor(A, seed=12)
    batch = solve.SystemBatch(spx.CSR.from_host(A), ptr)
    dL = spx.CSR.from_host(L)
    F = solve.DiagonalFactor(batch, dL).fill(dL.values)
    assert batch.launch_for(5)[1] >= 4
    b = synth.normal(A.m, seed=13)
    x, iters, status, relres = solve.cg(batch, dev(b), pc="dia", dia=F, tol=1e-8)
    x, iters, status, relres = host(x), host(iters), host(status), host(relres)
    assert np.all(status == 0), status
    Lr = synth.CSR(L.m, L.n, L.indptr, L.indices, _bf16(L.values))
    for s in range(len(sides)):
        As, a, c = _block(A, ptr, s)
        r = b[a:c].astype(np.float64) - oracle.spmm(As, x[a:c])
        assert np.linalg.norm(r) / np.linalg.norm(b[a:c]) <= 1e-8
        assert relres[s] <= 1e-8
        Ls, _, _ = _block(Lr, ptr, s)
        xo, st, it8 = oracle.pcg(As, b[a:c], tol=1e-8, pc="llt", L=(Ls.indptr, Ls.indices, Ls.values))
        assert st == 0
        assert iters[s] <= 1.3 * it8 + 5, (s, int(iters[s]), it8)
        assert np.linalg.norm(x[a:c] - xo) <= 1e-5 * np.linalg.norm(xo)


def test_dia_pcg_reports_unsupported_systems():
    # a factor with more than three diagonals (tril of A + A^2: seven offsets)
    A, ptr = _batch([9, 12], 3)
    batch = solve.SystemBatch(spx.CSR.from_host(A), ptr)
    from oracle import mpnn
    rows = mpnn.square_pattern(A)
    ip = np.concatenate([[0], np.cumsum([sum(1 for j in r if j <= i) for i, r in enumerate(rows)])])
    ix = np.array([j for i, r in enumerate(rows) for j in r if j <= i], np.int32)
    wide = synth.CSR(A.m, A.m, ip, ix, np.full(ix.size, 0.1, np.float32))
    dW = spx.CSR.from_host(wide)
    F = solve.DiagonalFactor(batch, dW).fill(dW.values)
    assert not F.supported and np.all(host(F.nd) == -1)
    b = dev(synth.normal(A.m, seed=1))
    _, _, status, relres = solve.cg(batch, b, pc="dia", dia=F, tol=1e-8)
    assert np.all(host(status) == 10) and np.all(host(relres) == -1.0)     # SPX_NOT_SUPPORTED
    # a halo deeper than a block's rows: side 12 over 16 blocks (9 rows each)
    L = _factor(A, seed=2)
    dL = spx.CSR.from_host(L)
    F = solve.DiagonalFactor(batch, dL).fill(dL.values)
    batch.launch = (1024, 16, 0)
    _, _, status, _ = solve.cg(batch, b, pc="dia", dia=F, tol=1e-8)
    assert host(status).tolist() == [10, 10]
    batch.launch = None
    _, _, status, _ = solve.cg(batch, b, pc="dia", dia=F, tol=1e-8)
    assert np.all(host(status) == 0)
    abi.spx_check_device()
