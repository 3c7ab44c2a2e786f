"""Host logic of the batched PCG launch shape (no GPU): the cluster chosen per
preconditioner kind from the batch's system sizes."""
import types

import pytest

solve = pytest.importorskip("paper_2212_05159_gb300.solve")


def _shape(kind, max_rows, mean_rows=None, launch=None):
    stub = types.SimpleNamespace(launch=launch, max_rows=float(max_rows),
                                 mean_rows=float(mean_rows if mean_rows is not None else max_rows))
    return solve.SystemBatch.launch_for(stub, kind)


@pytest.mark.parametrize("kind", [0, 1, 3])
@pytest.mark.parametrize("max_rows,cluster", [(1, 1), (1024, 1), (8192, 1), (8193, 2), (32768, 4),
                                              (65536, 8), (65537, 16), (131072, 16), (10 ** 6, 16)])
def test_vector_kinds_take_the_smallest_cluster_holding_the_largest_system(kind, max_rows, cluster):
    # shared memory holds 8 rows per thread of a 1024-thread block
    assert _shape(kind, max_rows, mean_rows=max_rows / 3) == (1024, cluster, 0)


def test_ic0_runs_one_block_per_system():
    assert _shape(4, 65536) == (1024, 1, 0)
    assert _shape(4, 10 ** 6) == (1024, 1, 0)


@pytest.mark.parametrize("mean_rows,cluster", [(1024, 1), (8192, 2), (65536, 16), (10 ** 6, 16)])
def test_llt_keeps_about_four_rows_per_thread(mean_rows, cluster):
    assert _shape(2, 10 ** 6, mean_rows=mean_rows) == (1024, cluster, 0)


def test_an_explicit_launch_wins():
    assert _shape(1, 65536, launch=(512, 2, 7)) == (512, 2, 7)
