"""GPU parity of the batched PCG solve and its adjoint against the FP64 oracle
(Section 4.3 PCG, Table 1 SpSolve VJPs), through the C ABI."""
import numpy as np
import pytest
import torch

import oracle
import synth
from helpers import assert_close_normalised

pytestmark = pytest.mark.gpu
spx = pytest.importorskip("paper_2212_05159_gb300")
from paper_2212_05159_gb300 import solve  # noqa: E402


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def host(t):
    return t.detach().cpu().numpy()


def _block(A, ptr, s):
    a, c = int(ptr[s]), int(ptr[s + 1])
    e0, e1 = int(A.indptr[a]), int(A.indptr[c])
    return synth.CSR(c - a, c - a, A.indptr[a:c + 1] - e0, A.indices[e0:e1] - a, A.values[e0:e1]), a, c


def _true_relres(A, x, b):
    r = np.asarray(b, np.float64) - oracle.spmm(A, x)
    return np.linalg.norm(r) / np.linalg.norm(b)


@pytest.fixture(scope="module")
def small_batch():
    A, ptr, sides, _ = synth.diffusion_batch(12, seed=3, side_lo=4, side_hi=40, sigma=1.0)
    return A, ptr, solve.SystemBatch(spx.CSR.from_host(A), ptr)


@pytest.mark.parametrize("pc", ["none", "jacobi"])
def test_cg_matches_oracle(small_batch, pc):
    A, ptr, batch = small_batch
    b = synth.normal(A.m, seed=7)
    x, iters, status, relres = solve.cg(batch, dev(b), pc=pc, tol=1e-8)
    x = host(x)
    assert np.all(host(status) == 0)
    for s in range(batch.nsys):
        As, a, c = _block(A, ptr, s)
        rr = _true_relres(As, x[a:c], b[a:c])
        assert rr <= 1e-8, (s, rr)
        assert abs(rr - host(relres)[s]) <= 1e-9 + 1e-3 * rr
        xo, st, it = oracle.pcg(As, b[a:c], tol=1e-12, pc=pc)
        # x agrees with the FP64 solution to the conditioning of the system
        assert np.linalg.norm(x[a:c] - xo) <= 1e-5 * np.linalg.norm(xo)
        # the FP32 iteration with reliable updates needs about as many steps as FP64 PCG
        _, _, it8 = oracle.pcg(As, b[a:c], tol=1e-8, pc=pc)
        assert host(iters)[s] <= 1.5 * it8 + 5


def test_llt_factor_matches_oracle(small_batch):
    A, ptr, batch = small_batch
    l_ip, l_ix, _ = oracle.tril_pattern(A)
    d = oracle.diagonal(A)
    rows = np.repeat(np.arange(A.m), np.diff(l_ip))
    rng = np.random.default_rng(1)
    lv = rng.uniform(-0.1, 0.1, l_ix.size) / np.sqrt(d[rows])
    on = rows == l_ix
    lv[on] = 1.0 / np.sqrt(d[rows[on]])
    Lh = synth.CSR(A.m, A.m, l_ip, l_ix, lv.astype(np.float32))
    fac = solve.Factor(spx.CSR.from_host(Lh))
    b = synth.normal(A.m, seed=5)
    x, iters, status, relres = solve.cg(batch, dev(b), pc="llt", factor=fac, tol=1e-8)
    x = host(x)
    assert np.all(host(status) == 0)
    for s in range(batch.nsys):
        As, a, c = _block(A, ptr, s)
        assert _true_relres(As, x[a:c], b[a:c]) <= 1e-8
        Ls, _, _ = _block(Lh, ptr, s)
        _, _, it8 = oracle.pcg(As, b[a:c], tol=1e-8, pc="llt", L=(Ls.indptr, Ls.indices, Ls.values))
        assert host(iters)[s] <= 1.5 * it8 + 5


def test_status_codes():
    A = synth.poisson2d(12)
    ptr = np.array([0, A.m], np.int32)
    batch = solve.SystemBatch(spx.CSR.from_host(A), ptr)
    b = synth.normal(A.m, seed=1)
    _, it, st, _ = solve.cg(batch, dev(b), pc="jacobi", tol=1e-12, maxit=3)
    assert host(st)[0] == 5 and host(it)[0] == 3                       # SPX_MAXITER
    bad = b.copy()
    bad[3] = np.nan
    _, _, st, _ = solve.cg(batch, dev(bad), pc="jacobi")
    assert host(st)[0] == 7                                           # SPX_NONFINITE
    n = A.m
    Lz = synth.CSR(n, n, np.arange(n + 1), np.arange(n), np.where(np.arange(n) % 2 == 0, 0.0, 1.0))
    fac = solve.Factor(spx.CSR.from_host(Lz))
    e = np.zeros(n, np.float32)
    e[0] = 1.0
    _, _, st, _ = solve.cg(batch, dev(e), pc="llt", factor=fac)
    assert host(st)[0] == 6                                           # SPX_BREAKDOWN
    x, it, st, rr = solve.cg(batch, dev(np.zeros(n, np.float32)), pc="jacobi")
    assert host(st)[0] == 0 and host(it)[0] == 0 and np.all(host(x) == 0)


def test_eigenvector_one_iteration():
    N = 15
    A = synth.poisson2d(N)
    ix, iy = np.meshgrid(np.arange(1, N + 1), np.arange(1, N + 1), indexing="ij")
    v = (np.sin(ix * 2 * np.pi / (N + 1)) * np.sin(iy * 3 * np.pi / (N + 1))).ravel().astype(np.float32)
    batch = solve.SystemBatch(spx.CSR.from_host(A), np.array([0, A.m], np.int32))
    x, it, st, rr = solve.cg(batch, dev(v), pc="none", tol=1e-6)
    assert host(st)[0] == 0 and host(it)[0] <= 2


def test_adjoint_matches_oracle(small_batch):
    A, ptr, batch = small_batch
    b = synth.normal(A.m, seed=2)
    g = synth.normal(A.m, seed=3)
    vals = dev(A.values).requires_grad_(True)
    bt = dev(b).requires_grad_(True)
    x = solve.Solve.apply(vals, bt, batch, "jacobi", 1e-10)
    x.backward(dev(g.astype(np.float64)))
    gA = host(vals.grad)
    gb = host(bt.grad)
    xh = host(x)
    for s in range(batch.nsys):
        As, a, c = _block(A, ptr, s)
        e0, e1 = int(A.indptr[a]), int(A.indptr[c])
        lam, ga = oracle.solve_adjoint(As, xh[a:c], g[a:c])
        np.testing.assert_allclose(gb[a:c], lam, rtol=0, atol=1e-6 * np.abs(lam).max())
        norm = oracle.sddmm(As, np.abs(lam).reshape(-1, 1), np.abs(xh[a:c]).reshape(-1, 1))
        # lam carries the solve's own error (tol 1e-10 times the conditioning)
        assert_close_normalised(gA[e0:e1], ga, norm, rel=1e-5, what=f"grad A system {s}")


def test_full_size_batch_256():
    """The 256-system workload (sides 32..256) with Jacobi, checked on sampled systems."""
    A, ptr, sides, _ = synth.diffusion_batch(256, seed=0, side_lo=32, side_hi=256, sigma=1.0)
    batch = solve.SystemBatch(spx.CSR.from_host(A), ptr)
    b = synth.normal(A.m, seed=1)
    x, iters, status, relres = solve.cg(batch, dev(b), pc="jacobi", tol=1e-8)
    torch.cuda.synchronize()
    assert np.all(host(status) == 0)
    assert np.all(host(relres) <= 1e-8)
    xh = host(x)
    order = np.argsort(np.diff(ptr))
    for s in list(order[:2]) + list(order[-2:]):
        As, a, c = _block(A, ptr, s)
        assert _true_relres(As, xh[a:c], b[a:c]) <= 1e-8


def test_ic0_factor_and_pcg_match_oracle(small_batch):
    A, ptr, batch = small_batch
    ic = solve.IC0(batch)
    assert np.all(host(ic.status) == 0)
    lv = host(ic.values)
    l_ip = host(ic.Lpat.indptr)
    b = synth.normal(A.m, seed=9)
    x, iters, status, relres = solve.cg(batch, dev(b), pc="ic0", ic0=ic, tol=1e-8)
    x = host(x)
    assert np.all(host(status) == 0)
    for s in range(batch.nsys):
        As, a, c = _block(A, ptr, s)
        o_ip, o_ix, o_v = oracle.ic0(As)
        e0, e1 = int(l_ip[a]), int(l_ip[c])
        np.testing.assert_array_equal(host(ic.Lpat.indices)[e0:e1] - a, o_ix)
        np.testing.assert_allclose(lv[e0:e1], o_v, rtol=2e-5, atol=1e-6 * np.abs(o_v).max())
        assert _true_relres(As, x[a:c], b[a:c]) <= 1e-8
        _, _, it8 = oracle.pcg(As, b[a:c], tol=1e-8, pc="ic0", L=(o_ip, o_ix, o_v))
        assert host(iters)[s] <= 1.5 * it8 + 5


def test_ic0_tridiagonal_one_iteration():
    """IC(0) of A_N is its exact Cholesky factor: PCG converges in one iteration."""
    A = synth.poisson1d(300)
    batch = solve.SystemBatch(spx.CSR.from_host(A), np.array([0, A.m], np.int32))
    ic = solve.IC0(batch)
    b = synth.normal(A.m, seed=2)
    _, it, st, rr = solve.cg(batch, dev(b), pc="ic0", ic0=ic, tol=1e-6)
    assert host(st)[0] == 0 and host(it)[0] <= 2


def test_cg_adjoint_entry_point_matches_autograd_and_oracle(small_batch):
    """spx_cg_adjoint (one C call) gives the autograd Solve's gradients bit for bit, and the
    oracle's within tolerance."""
    from paper_2212_05159_gb300 import abi
    A, ptr, batch = small_batch
    b = synth.normal(A.m, seed=12)
    g = synth.normal(A.m, seed=13)
    x, _, st, _ = solve.cg(batch, dev(b), pc="jacobi", tol=1e-10)
    x = x.clone()
    lam = torch.empty(A.m, dtype=torch.float64, device="cuda")
    gA = torch.empty(A.nnz, dtype=torch.float32, device="cuda")
    iters = torch.empty(batch.nsys, dtype=torch.int32, device="cuda")
    status = torch.empty_like(iters)
    relres = torch.empty(batch.nsys, dtype=torch.float64, device="cuda")
    abi.spx_cg_set_launch(*batch.launch_for(1))
    abi.spx_cg_adjoint(batch.A.struct(), batch.sys_ptr, batch.nsys, batch.order, x, dev(g), lam, gA, 1,
                       batch.dinv(), None, None, 1e-10, 20 * A.m, 0.1, iters, status, relres, batch.ws)
    assert abi.spx_sync_status(status) == [0] * batch.nsys
    vals = batch.A.values.clone().requires_grad_(True)
    bt = dev(b).requires_grad_(True)
    xx = solve.Solve.apply(vals, bt, batch, "jacobi", 1e-10)
    xx.backward(dev(g.astype(np.float64)))
    np.testing.assert_array_equal(host(gA), host(vals.grad))
    np.testing.assert_array_equal(host(lam).astype(np.float32), host(bt.grad))
    xh = host(x)
    for s in range(batch.nsys):
        As, a, c = _block(A, ptr, s)
        lam_o, _ = oracle.solve_adjoint(As, xh[a:c], g[a:c])
        np.testing.assert_allclose(host(lam)[a:c], lam_o, rtol=0, atol=1e-6 * np.abs(lam_o).max())


def test_sync_status_reports_the_first_failure():
    from paper_2212_05159_gb300.abi import SpxError, spx_sync_status
    A, ptr = synth.block_diag([synth.poisson2d(8), synth.poisson2d(12)])
    batch = solve.SystemBatch(spx.CSR.from_host(A), ptr)
    b = synth.normal(A.m, seed=1)
    _, _, st, _ = solve.cg(batch, dev(b), pc="jacobi", tol=1e-12, maxit=3)
    with pytest.raises(SpxError, match="MAXITER"):
        spx_sync_status(st)
    _, _, st, _ = solve.cg(batch, dev(b), pc="jacobi")
    assert spx_sync_status(st) == [0, 0]


@pytest.mark.parametrize("kind", [0, 1, 2, 3, 4])
def test_precond_apply_matches_oracle(small_batch, kind):
    """z = M r outside the solver for every preconditioner kind of the PCG."""
    from paper_2212_05159_gb300 import abi
    from paper_2212_05159_gb300.csr import CSR
    A, ptr, batch = small_batch
    r = synth.normal(A.m, seed=21)
    z = torch.empty(A.m, device="cuda")
    tmp = torch.empty(A.m, device="cuda")
    diag = oracle.diagonal(A)
    l_ip, l_ix, l_v = oracle.ic0(A)                       # a lower factor with the IC(0) pattern
    Lh = synth.CSR(A.m, A.m, l_ip, l_ix, l_v.astype(np.float32))
    dL = CSR.from_host(Lh)
    t_ip, t_ix, perm = dL.transpose_pattern()
    lt = dL.values[perm.long()].contiguous()
    sL = dL.struct()
    sLT = abi.csr_struct(A.m, A.m, t_ip, t_ix, lt)
    if kind == 0:
        abi.spx_precond_apply(0, dev(r), z)
        ref = r.astype(np.float64)
    elif kind == 1:
        abi.spx_precond_apply(1, dev(r), z, dinv=dev((1.0 / diag).astype(np.float32)))
        ref = r / diag.astype(np.float32).astype(np.float64)
    elif kind == 2:
        abi.spx_precond_apply(2, dev(r), z, L=sL, LT=sLT, tmp=tmp)
        ref = oracle.spmm(Lh, oracle.spmm_t(Lh, r))
    elif kind == 3:
        abi.spx_precond_apply(3, dev(r), z, L=batch.A.struct())
        ref = oracle.spmm(A, r)
    else:
        levels = abi.spx_ic0_analyse(sL, batch.sys_ptr, batch.nsys, "cuda")
        abi.spx_precond_apply(4, dev(r), z, L=sL, LT=sLT, nsys=batch.nsys, levels=levels, tmp=tmp)
        ref = oracle.trsv_lower_t(l_ip, l_ix, Lh.values, oracle.trsv_lower(l_ip, l_ix, Lh.values, r))
    np.testing.assert_allclose(host(z), ref, rtol=2e-5, atol=2e-5 * np.abs(ref).max())


def _spd_band(A, ptr):
    """A symmetric, strictly diagonally dominant M on each system's rows: 2 on the diagonal,
    -0.5 between rows i and i + 1 of the same system (a sparse product that gathers r)."""
    rows, cols, vals = [], [], []
    for s in range(len(ptr) - 1):
        a, c = int(ptr[s]), int(ptr[s + 1])
        for i in range(a, c):
            for j, v in ((i - 1, -0.5), (i, 2.0), (i + 1, -0.5)):
                if a <= j < c:
                    rows.append(i)
                    cols.append(j)
                    vals.append(v)
    ip = np.zeros(A.m + 1, np.int64)
    np.add.at(ip, np.asarray(rows) + 1, 1)
    return spx.CSR.from_host(synth.CSR(A.m, A.m, np.cumsum(ip), np.asarray(cols), np.asarray(vals, np.float32)))


@pytest.mark.parametrize("pc", ["none", "jacobi", "M"])
@pytest.mark.parametrize("launch", [(256, 1, 0), (1024, 2, 0)])
def test_vector_residency_is_bitwise_neutral(pc, launch):
    """Private PCG vectors in shared memory or in the workspace: the same arithmetic in the
    same order, so x, iterations, status and residuals agree bit for bit.  With 256-thread
    blocks of one (shared memory for 2048 rows per block) the batch mixes systems that fit
    (sides 8..45) with systems that do not (sides 46..70) in one launch."""
    A, ptr, _, _ = synth.diffusion_batch(10, seed=11, side_lo=8, side_hi=70, sigma=1.0)
    batch = solve.SystemBatch(spx.CSR.from_host(A), ptr)
    batch.launch = launch
    M = _spd_band(A, ptr) if pc == "M" else None
    b = dev(synth.normal(A.m, seed=12))
    out = []
    try:
        for res in (1, 0):
            spx.abi.spx_cg_set_vector_residency(res)
            x, it, st, rr = solve.cg(batch, b, pc=pc, M=M, tol=1e-8)
            out.append((host(x).copy(), host(it).copy(), host(st).copy(), host(rr).copy()))
    finally:
        spx.abi.spx_cg_set_vector_residency(1)
    assert np.all(out[0][2] == 0)
    for u, w in zip(out[0], out[1]):
        np.testing.assert_array_equal(u, w)
    sides = np.sqrt(np.diff(ptr)).astype(int)
    if launch[0] == 256:
        assert (sides * sides <= 2048).any() and (sides * sides > 2048).any()


@pytest.mark.parametrize("pc", ["none", "jacobi", "M"])
@pytest.mark.parametrize("residency", [1, 0])
def test_empty_and_one_row_systems(pc, residency):
    """A batch holding an empty system (repeated offset) and a 1 x 1 system between two
    grids: the empty one reports OK after 0 iterations with residual 0, the 1 x 1 one
    x = b / a in one iteration, the grids converge as usual."""
    one = synth.CSR(1, 1, np.array([0, 1]), np.array([0]), np.array([2.0], np.float32))
    A, ptr = synth.block_diag([synth.diffusion2d(5, 1.0, 1), one, synth.diffusion2d(4, 1.0, 2)])
    ptr = np.array([0, 25, 25, 26, 42], np.int32)
    batch = solve.SystemBatch(spx.CSR.from_host(A), ptr)
    M = _spd_band(A, ptr) if pc == "M" else None
    b = synth.normal(A.m, seed=3)
    try:
        spx.abi.spx_cg_set_vector_residency(residency)
        x, it, st, rr = solve.cg(batch, dev(b), pc=pc, M=M, tol=1e-8)
    finally:
        spx.abi.spx_cg_set_vector_residency(1)
    x, it, st, rr = host(x), host(it), host(st), host(rr)
    assert list(st) == [0, 0, 0, 0]
    assert it[1] == 0 and rr[1] == 0.0
    assert it[2] == 1 and abs(x[25] - b[25] / 2.0) <= 1e-7 * abs(b[25] / 2.0)
    for s in (0, 3):
        As, a, c = _block(A, ptr, s)
        assert _true_relres(As, x[a:c], b[a:c]) <= 1e-8


def test_explicit_m_matches_oracle(small_batch):
    """PCG with an explicit M = L L^T (formed on the host in FP64, stored FP32): every system
    to the true residual 1e-8 in about as many iterations as the FP64 oracle's PCG with the
    same L applied as L (L^T r)."""
    A, ptr, batch = small_batch
    l_ip, l_ix, _ = oracle.tril_pattern(A)
    d = oracle.diagonal(A)
    rows = np.repeat(np.arange(A.m), np.diff(l_ip))
    rng = np.random.default_rng(2)
    lv = rng.uniform(-0.15, 0.15, l_ix.size) / np.sqrt(d[rows])
    on = rows == l_ix
    lv[on] = 1.0 / np.sqrt(d[rows[on]])
    Ld = np.zeros((A.m, A.m))
    Ld[rows, l_ix] = lv
    Md = Ld @ Ld.T
    mr, mc = np.nonzero(Md)
    mip = np.concatenate([[0], np.cumsum(np.bincount(mr, minlength=A.m))])
    M = spx.CSR.from_host(synth.CSR(A.m, A.m, mip, mc, Md[mr, mc].astype(np.float32)))
    b = synth.normal(A.m, seed=6)
    x, iters, status, relres = solve.cg(batch, dev(b), pc="M", M=M, tol=1e-8)
    x = host(x)
    assert np.all(host(status) == 0)
    for s in range(batch.nsys):
        As, a, c = _block(A, ptr, s)
        assert _true_relres(As, x[a:c], b[a:c]) <= 1e-8
        Ls = synth.CSR(c - a, c - a, l_ip[a:c + 1] - l_ip[a], l_ix[l_ip[a]:l_ip[c]] - a, lv[l_ip[a]:l_ip[c]])
        _, _, it8 = oracle.pcg(As, b[a:c], tol=1e-8, pc="llt", L=(Ls.indptr, Ls.indices, Ls.values))
        assert host(iters)[s] <= 1.5 * it8 + 5, (s, int(host(iters)[s]), it8)
