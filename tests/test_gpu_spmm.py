"""GPU parity of SpMM / SpMV, SDDMM, the CSR transpose and transpose-SpMM against the
FP64 oracle, through the C ABI (Section 3.1.1, 3.1.3 and Table 1)."""
import numpy as np
import pytest
import torch

import oracle
import synth
from helpers import abs_csr, assert_close_normalised, sub_rows

pytestmark = pytest.mark.gpu

spx = pytest.importorskip("paper_2212_05159_gb300")


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def host(t):
    return t.detach().cpu().numpy()


MATS = {
    "poisson2d_64": lambda: synth.poisson2d(64),
    "ragged": lambda: synth.empty_rows_csr(3001, 2500, seed=4, max_len=70),
    "powerlaw_20k": lambda: synth.powerlaw_csr(20000, seed=1, max_len=2000),
    "poisson3d_16": lambda: synth.poisson3d(16),
    "rect_wide": lambda: synth.random_k_per_row(777, 5, seed=3, ncols=4099),
}


@pytest.fixture(scope="module", params=list(MATS))
def mat(request):
    A = MATS[request.param]()
    return request.param, A, spx.CSR.from_host(A)


@pytest.mark.parametrize("k", [1, 3, 8, 32, 36, 128])
def test_spmm_matches_oracle(mat, k):
    name, A, dA = mat
    X = synth.normal((A.n, k), seed=k)
    Y = host(spx.spmm(dA, dev(X)))
    ref = oracle.spmm(A, X)
    norm = oracle.spmm(abs_csr(A), np.abs(X))
    assert_close_normalised(Y, ref, norm, what=f"spmm {name} k={k}")


def test_spmv_1d_and_alpha_beta(mat):
    name, A, dA = mat
    x = synth.normal(A.n, seed=3)
    y0 = synth.normal(A.m, seed=4)
    out = dev(y0.copy())
    y = host(spx.spmm(dA, dev(x), out=out, alpha=0.5, beta=-2.0))
    ref = 0.5 * oracle.spmm(A, x) - 2.0 * y0.astype(np.float64)
    norm = 0.5 * oracle.spmm(abs_csr(A), np.abs(x)) + 2.0 * np.abs(y0)
    assert_close_normalised(y, ref, norm, what=f"spmv {name}")


@pytest.mark.parametrize("k", [1, 8, 12, 32, 33, 128])
def test_sddmm_matches_oracle(mat, k):
    name, A, dA = mat
    G = synth.normal((A.m, k), seed=10 + k)
    X = synth.normal((A.n, k), seed=20 + k)
    out = host(spx.sddmm(dA, dev(G), dev(X)))
    ref = oracle.sddmm(A, G, X)
    norm = oracle.sddmm(A, np.abs(G), np.abs(X))
    assert_close_normalised(out, ref, norm, what=f"sddmm {name} k={k}")


def test_transpose_bit_exact(mat):
    name, A, dA = mat
    t_ip, t_ix, perm = dA.transpose_pattern()
    r_ip, r_ix, r_perm = oracle.transpose(A)
    np.testing.assert_array_equal(host(t_ip), r_ip)
    np.testing.assert_array_equal(host(t_ix), r_ix)
    np.testing.assert_array_equal(host(perm), r_perm)


@pytest.mark.parametrize("k", [1, 8, 32, 128])
def test_spmm_t_matches_oracle(mat, k):
    name, A, dA = mat
    G = synth.normal((A.m, k), seed=30 + k)
    gX = host(spx.spmm_t(dA, dev(G)))
    ref = oracle.spmm_t(A, G)
    norm = oracle.spmm_t(abs_csr(A), np.abs(G))
    assert_close_normalised(gX, ref, norm, what=f"spmm_t {name} k={k}")


def test_masked_outer_scale(mat):
    name, A, dA = mat
    u = synth.normal(A.m, seed=1)
    v = synth.normal(A.n, seed=2)
    out = host(spx.masked_outer(dA, dev(u), dev(v), scale=-1.0))
    ref = -oracle.sddmm(A, u.reshape(-1, 1), v.reshape(-1, 1))
    norm = np.abs(ref)
    assert_close_normalised(out, ref, norm, what=f"masked_outer {name}")


def test_deterministic_repeats(mat):
    name, A, dA = mat
    X = dev(synth.normal((A.n, 32), seed=5))
    G = dev(synth.normal((A.m, 32), seed=6))
    a1, a2 = host(spx.spmm(dA, X)), host(spx.spmm(dA, X))
    b1, b2 = host(spx.sddmm(dA, G, X)), host(spx.sddmm(dA, G, X))
    c1, c2 = host(spx.spmm_t(dA, G)), host(spx.spmm_t(dA, G))
    assert np.array_equal(a1, a2) and np.array_equal(b1, b2) and np.array_equal(c1, c2)


def test_autograd_spmm(mat):
    name, A, dA = mat
    from paper_2212_05159_gb300 import autograd
    k = 8
    X = synth.normal((A.n, k), seed=11)
    V = synth.normal((A.m, k), seed=12)
    vals = dev(A.values).requires_grad_(True)
    Xt = dev(X).requires_grad_(True)
    Y = autograd.spmm(dA, Xt, values=vals)
    Y.backward(dev(V))
    assert_close_normalised(host(vals.grad), oracle.sddmm(A, V, X),
                            oracle.sddmm(A, np.abs(V), np.abs(X)), what="autograd dA")
    assert_close_normalised(host(Xt.grad), oracle.spmm_t(A, V),
                            oracle.spmm_t(abs_csr(A), np.abs(V)), what="autograd dX")


def test_empty_and_degenerate():
    # no stored entries at all
    A = synth.CSR(5, 7, np.zeros(6, np.int32), np.zeros(0, np.int32), np.zeros(0, np.float32))
    dA = spx.CSR.from_host(A)
    Y = host(spx.spmm(dA, dev(np.ones((7, 4), np.float32))))
    assert Y.shape == (5, 4) and np.all(Y == 0)
    assert spx.sddmm(dA, dev(np.ones((5, 4), np.float32)), dev(np.ones((7, 4), np.float32))).numel() == 0
    gX = host(spx.spmm_t(dA, dev(np.ones((5, 4), np.float32))))
    assert np.all(gX == 0)
    # 1 x 1
    B = synth.CSR(1, 1, np.array([0, 1]), np.array([0]), np.array([3.0], np.float32))
    dB = spx.CSR.from_host(B)
    assert host(spx.spmm(dB, dev(np.array([[2.0]], np.float32))))[0, 0] == 6.0


def test_validate_rejects_bad_patterns():
    from paper_2212_05159_gb300.abi import SpxError
    good = synth.poisson2d(5)
    spx.CSR.from_host(good).validate()
    bad = synth.CSR(good.m, good.n, good.indptr, good.indices.copy(), good.values)
    bad.indices[1], bad.indices[2] = bad.indices[2], bad.indices[1]
    with pytest.raises(SpxError, match="UNSORTED"):
        spx.CSR.from_host(bad).validate()
    oob = synth.CSR(good.m, good.n, good.indptr, good.indices.copy(), good.values)
    oob.indices[-1] = good.n + 3
    with pytest.raises(SpxError, match="BAD_PATTERN"):
        spx.CSR.from_host(oob).validate()


@pytest.mark.parametrize("kind,k,backward", [("powerlaw", 32, "tuned"), ("powerlaw", 128, "tuned"),
                                             ("poisson3d", 32, "tuned"), ("powerlaw", 32, "fused"),
                                             ("powerlaw", 32, "separate")])
def test_full_size_bench_configuration_sampled(kind, k, backward):
    """The benchmark's own workloads (power-law n = 2^20 at k = 32 and 128, 3D Poisson 128^3 at
    k = 32), built and autotuned exactly as bench.py does and run through its launch calls
    (the backward as tuned, or forced to the fused pass or to the three separate launches);
    sampled rows of Y, gA and gX against the oracle computed on those rows alone."""
    import bench
    W = bench.Workload(kind, k=k)
    if backward == "fused":
        W.backward, W.KERNELS = ("fused", 0, W.t_plan, "tuned"), ("spmm", "backward")
    elif backward == "separate":
        W.backward, W.KERNELS = None, ("spmm", "sddmm", "gather", "spmm_t")
    for kname in W.KERNELS:
        W.run_kernel(kname)
    torch.cuda.synchronize()
    A = W.host
    X, G = host(W.X).astype(np.float64), host(W.G).astype(np.float64)
    Y, gA, gX = host(W.Y), host(W.gA), host(W.gX)
    rng = np.random.default_rng(1)
    lens = A.row_lengths()
    rows = np.concatenate([rng.choice(A.m, 300, replace=False), np.argsort(lens)[-10:]])
    S, take = sub_rows(A, rows)
    assert_close_normalised(Y[rows], oracle.spmm(S, X), oracle.spmm(abs_csr(S), np.abs(X)), what=f"Y {kind}")
    Gs = G[rows]
    assert_close_normalised(gA[take], oracle.sddmm(S, Gs, X), oracle.sddmm(S, np.abs(Gs), np.abs(X)),
                            what=f"gA {kind}")
    t_ip, t_ix, perm = oracle.transpose(A)
    AT = synth.CSR(A.n, A.m, t_ip, t_ix, A.values[perm])
    cols = rng.choice(A.n, 300, replace=False)
    ST, _ = sub_rows(AT, cols)
    assert_close_normalised(gX[cols], oracle.spmm(ST, G), oracle.spmm(abs_csr(ST), np.abs(G)), what=f"gX {kind}")


@pytest.mark.parametrize("k", [32])
def test_full_size_powerlaw_sampled(k):
    """The n = 2^20 power-law workload in the benchmark's launch configuration, checked
    on sampled rows / columns that the oracle computes one by one."""
    A = synth.powerlaw_csr(1 << 20, seed=0)
    dA = spx.CSR.from_host(A)
    rng = np.random.default_rng(0)
    X = synth.normal((A.n, k), seed=1)
    G = synth.normal((A.m, k), seed=2)
    Y = host(spx.spmm(dA, dev(X)))
    gA = host(spx.sddmm(dA, dev(G), dev(X)))
    gX = host(spx.spmm_t(dA, dev(G)))
    lens = A.row_lengths()
    rows = np.concatenate([rng.choice(A.m, 400, replace=False), np.argsort(lens)[-20:]])
    S, take = sub_rows(A, rows)
    assert_close_normalised(Y[rows], oracle.spmm(S, X), oracle.spmm(abs_csr(S), np.abs(X)), what="Y")
    Gs = G[rows]
    assert_close_normalised(gA[take], oracle.sddmm(S, Gs, X), oracle.sddmm(S, np.abs(Gs), np.abs(X)),
                            what="gA")
    t_ip, t_ix, perm = oracle.transpose(A)
    AT = synth.CSR(A.n, A.m, t_ip, t_ix, A.values[perm])
    cols = rng.choice(A.n, 400, replace=False)
    ST, _ = sub_rows(AT, cols)
    assert_close_normalised(gX[cols], oracle.spmm(ST, G), oracle.spmm(abs_csr(ST), np.abs(G)), what="gX")
    # the transpose itself, bit-exact on the sampled rows of A^T
    d_ip, d_ix, d_perm = [host(t) for t in dA.transpose_pattern()]
    np.testing.assert_array_equal(d_ip, t_ip)
    np.testing.assert_array_equal(d_ix, t_ix)
    np.testing.assert_array_equal(d_perm, perm)


@pytest.mark.parametrize("cb,rpg,engine", [(4, 1, 0), (8, 3, 0), (16, 2, 0), (32, 4, 0),
                                           (8, 1, 1), (16, 3, 1), (32, 2, 1), (32, 1, 2), (32, 3, 2)])
def test_tuning_variants_match_oracle(mat, cb, rpg, engine):
    """Every column-block / rows-per-group / gather-engine setting the autotuner may pick is
    correct (engine 1: TMA-engine bulk copies)."""
    from paper_2212_05159_gb300 import abi
    name, A, dA = mat
    k = 32
    X = synth.normal((A.n, k), seed=40)
    G = synth.normal((A.m, k), seed=41)
    base = dA.plan()
    plan = base.with_params(cb, rpg, engine)
    Y = torch.empty(A.m, k, device="cuda")
    ws = abi.workspace(abi.spx_spmm_workspace_size(dA.struct(), k, plan), "cuda")
    abi.spx_spmm(dA.struct(), dev(X), Y, 1.0, 0.0, plan, ws)
    abi.spx_check_device()
    assert_close_normalised(host(Y), oracle.spmm(A, X), oracle.spmm(abs_csr(A), np.abs(X)),
                            what=f"spmm {name} cb={cb} rpg={rpg} engine={engine}")
    tb = dA.t_plan()
    tplan = tb.with_params(cb, rpg, engine)
    gX = torch.empty(A.n, k, device="cuda")
    _, _, perm = dA.transpose_pattern()
    abi.spx_spmm_t(dA.t_struct(), perm, dev(G), gX, 1.0, 0.0, tplan, None)   # gather through perm
    assert_close_normalised(host(gX), oracle.spmm_t(A, G), oracle.spmm_t(abs_csr(A), np.abs(G)),
                            what=f"spmm_t {name} cb={cb} no workspace")
    abi.spx_spmm_t(dA.t_struct(), perm, dev(G), gX, 1.0, 0.0, tplan,
                   abi.workspace(abi.spx_spmm_t_workspace_size(dA.t_struct(), k, tplan), "cuda"))
    abi.spx_check_device()
    assert_close_normalised(host(gX), oracle.spmm_t(A, G), oracle.spmm_t(abs_csr(A), np.abs(G)),
                            what=f"spmm_t {name} cb={cb}")
    out = torch.empty(A.nnz, device="cuda")
    for p in (None, plan):
        abi.spx_sddmm(dA.struct(), dev(G), dev(X), out, 1.0, cb,
                      abi.workspace(abi.spx_sddmm_workspace_size(dA.struct(), k, cb), "cuda"), plan=p)
        assert_close_normalised(host(out), oracle.sddmm(A, G, X), oracle.sddmm(A, np.abs(G), np.abs(X)),
                                what=f"sddmm {name} cb={cb} plan={p is not None}")


@pytest.mark.parametrize("k", [8, 32, 128])
def test_bulk_engine_k_widths_and_alpha_beta(mat, k):
    """TMA-engine gathers at each lane-group width, with alpha / beta and empty rows."""
    from paper_2212_05159_gb300 import abi
    name, A, dA = mat
    X = synth.normal((A.n, k), seed=50 + k)
    y0 = synth.normal((A.m, k), seed=60 + k)
    base = dA.plan()
    plan = base.with_params(k, 2, 1)
    Y = dev(y0.copy())
    abi.spx_spmm(dA.struct(), dev(X), Y, 0.5, -1.5, plan, None)
    abi.spx_check_device()
    ref = 0.5 * oracle.spmm(A, X) - 1.5 * y0.astype(np.float64)
    norm = 0.5 * oracle.spmm(abs_csr(A), np.abs(X)) + 1.5 * np.abs(y0)
    assert_close_normalised(host(Y), ref, norm, what=f"bulk spmm {name} k={k}")


@pytest.mark.parametrize("n_parts", [2, 3, 5])
def test_column_parts_split_offsets(mat, n_parts):
    """spx_rowplan_build_parts: the offset of the first entry of each row at or past each
    column boundary, bit-exact against a per-row binary search on the host."""
    name, A, dA = mat
    if n_parts > A.n:
        pytest.skip("more parts than columns")
    pp, _ = dA.parts(n_parts)
    got = host(pp)[: (n_parts - 1) * A.m].reshape(n_parts - 1, A.m)
    w = -(-A.n // n_parts)
    for p in range(1, n_parts):
        want = np.array([A.indptr[i] + np.searchsorted(A.indices[A.indptr[i]:A.indptr[i + 1]], p * w)
                         for i in range(A.m)], dtype=np.int64)
        np.testing.assert_array_equal(got[p - 1], want, err_msg=f"{name} part {p}")


@pytest.mark.parametrize("n_parts,cb,rpg", [(2, 32, 4), (3, 16, 2), (4, 8, 1), (2, 4, 3)])
def test_column_parts_products_match_oracle(mat, n_parts, cb, rpg):
    """SpMM, A^T G and SDDMM with the rows split into column parts (one pass per part,
    later passes adding into the output), with alpha / beta on the forward product."""
    from paper_2212_05159_gb300 import abi
    name, A, dA = mat
    if n_parts > min(A.n, A.m):
        pytest.skip("more parts than columns")
    k = 32
    X = synth.normal((A.n, k), seed=70)
    G = synth.normal((A.m, k), seed=71)
    y0 = synth.normal((A.m, k), seed=72)
    plan = dA.plan().with_params(cb, rpg, 0, dA.parts(n_parts))
    Y = dev(y0.copy())
    ws = abi.workspace(abi.spx_spmm_workspace_size(dA.struct(), k, plan), "cuda")
    abi.spx_spmm(dA.struct(), dev(X), Y, 0.5, -1.5, plan, ws)
    ref = 0.5 * oracle.spmm(A, X) - 1.5 * y0.astype(np.float64)
    norm = 0.5 * oracle.spmm(abs_csr(A), np.abs(X)) + 1.5 * np.abs(y0)
    assert_close_normalised(host(Y), ref, norm, what=f"spmm parts={n_parts} {name} cb={cb}")
    tplan = dA.t_plan().with_params(cb, rpg, 0, dA.t_parts(n_parts))
    gX = torch.empty(A.n, k, device="cuda")
    _, _, perm = dA.transpose_pattern()
    abi.spx_spmm_t(dA.t_struct(), perm, dev(G), gX, 1.0, 0.0, tplan,
                   abi.workspace(abi.spx_spmm_t_workspace_size(dA.t_struct(), k, tplan), "cuda"))
    assert_close_normalised(host(gX), oracle.spmm_t(A, G), oracle.spmm_t(abs_csr(A), np.abs(G)),
                            what=f"spmm_t parts={n_parts} {name} cb={cb}")
    out = torch.full((A.nnz,), float("nan"), device="cuda")          # every entry must be written
    splan = dA.plan().with_params(cb, 2, 0, dA.parts(n_parts))
    abi.spx_sddmm(dA.struct(), dev(G), dev(X), out, 1.0, cb,
                  abi.workspace(abi.spx_sddmm_workspace_size(dA.struct(), k, cb), "cuda"), plan=splan)
    abi.spx_check_device()
    assert_close_normalised(host(out), oracle.sddmm(A, G, X), oracle.sddmm(A, np.abs(G), np.abs(X)),
                            what=f"sddmm parts={n_parts} {name} cb={cb}")


def test_spmm_autotune_entry_point(mat):
    """spx_spmm_autotune picks launch parameters by timing; the chosen plan computes A X."""
    from paper_2212_05159_gb300 import abi
    name, A, dA = mat
    k = 32
    X = synth.normal((A.n, k), seed=80)
    Y = torch.empty(A.m, k, device="cuda")
    plan, ms = abi.spx_spmm_autotune(dA.struct(), dev(X), Y, dA.plan())
    assert ms > 0 and plan.rows_per_group in (1, 2, 4, 8) and plan.engine in (0, 1)
    Y.zero_()
    abi.spx_spmm(dA.struct(), dev(X), Y, 1.0, 0.0, plan, None)
    abi.spx_check_device()
    assert_close_normalised(host(Y), oracle.spmm(A, X), oracle.spmm(abs_csr(A), np.abs(X)),
                            what=f"spmm {name} autotuned rpg={plan.rows_per_group} engine={plan.engine}")


@pytest.mark.parametrize("k", [8, 32, 128])
def test_short_row_order_is_bitwise_neutral(mat, k):
    """The plan's length-grouped short-row order only reschedules rows: SpMM, A^T G and
    SDDMM give bit-identical results with and without it; the order is a permutation of
    the short rows grouped by 8-entry batch count, longest group first."""
    from paper_2212_05159_gb300 import abi
    name, A, dA = mat
    X, G = dev(synth.normal((A.n, k), seed=50)), dev(synth.normal((A.m, k), seed=51))
    base, tb = dA.plan(), dA.t_plan()
    _, _, perm = dA.transpose_pattern()
    outs = []
    for so in (True, False):
        plan, tplan = base.with_params(k, 4, 0, short_order=so), tb.with_params(k, 4, 0, short_order=so)
        Y = torch.empty(A.m, k, device="cuda")
        abi.spx_spmm(dA.struct(), X, Y, 1.0, 0.0, plan)
        gX = torch.empty(A.n, k, device="cuda")
        abi.spx_spmm_t(dA.t_struct(), perm, G, gX, 1.0, 0.0, tplan,
                       abi.workspace(abi.spx_spmm_t_workspace_size(dA.t_struct(), k, tplan), "cuda"))
        gA = torch.empty(A.nnz, device="cuda")
        abi.spx_sddmm(dA.struct(), G, X, gA, 1.0, k, abi.workspace(abi.spx_sddmm_workspace_size(dA.struct(), k, k),
                                                                  "cuda"), plan=plan)
        outs.append((host(Y), host(gX), host(gA)))
    for u, w in zip(*outs):
        np.testing.assert_array_equal(u, w)
    if base.short_rows:
        rows_t = dA._plan[0][2]
        order = host(rows_t)[: base.n_short]
        lens = np.diff(np.asarray(A.indptr, np.int64))
        thr = base.medium_threshold if base.n_medium > 0 else base.threshold
        short = np.nonzero(lens <= thr)[0]
        assert sorted(order.tolist()) == short.tolist()
        key = np.minimum((lens[order] + 7) // 8, 8)
        assert np.all(np.diff(key) <= 0)
        for kk in np.unique(key):
            ids = order[key == kk]
            assert np.all(np.diff(ids) > 0)


@pytest.mark.parametrize("k", [4, 32, 128])
@pytest.mark.parametrize("unroll,bps", [(1, 8), (2, 5), (4, 4)])
def test_gather_probe_reads_every_row_once(k, unroll, bps):
    """The gather-bound probe reads row indices[e] of X for every entry (and nothing else):
    the sum of its per-thread sums is the sum of those rows, in float64 within float32
    accumulation error; indices outside [0, n) are skipped."""
    A = synth.powerlaw_csr(20000, seed=3, max_len=500)
    idx = A.indices.astype(np.int32).copy()
    idx[::97] = -5                                  # out of range: skipped
    idx[1::89] = A.n + 3
    X = synth.normal((A.n, k), seed=4)
    out = spx.abi.spx_gather_probe(torch.from_numpy(idx).cuda(), A.n, torch.from_numpy(X).cuda(), unroll, bps)
    got = float(out.double().sum())
    ok = (idx >= 0) & (idx < A.n)
    rows = X.astype(np.float64)[idx[ok]]
    want = float(rows.sum())
    assert abs(got - want) <= 1e-5 * float(np.abs(rows).sum())


def test_lean_engine_equals_the_register_path_bitwise(mat):
    """Plan engine 2 (short rows without a batch held ahead) does the same sums in the same
    order as engine 0: the same bits, forward and transposed."""
    from paper_2212_05159_gb300 import abi
    name, A, dA = mat
    for k in (8, 32, 128):
        X = dev(synth.normal((A.n, k), seed=50 + k))
        outs = []
        for engine in (0, 2):
            plan = dA.plan().with_params(k, 2, engine)
            Y = torch.empty(A.m, k, device="cuda")
            abi.spx_spmm(dA.struct(), X, Y, 1.0, 0.0, plan, None)
            outs.append(host(Y))
        np.testing.assert_array_equal(outs[0].view(np.int32), outs[1].view(np.int32))
    abi.spx_check_device()
