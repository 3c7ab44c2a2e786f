"""Host logic of the unrolled-PCG training (Section 4.3), no GPU: the workspace the reverse
pass needs with every iterate stored or recomputed from checkpoints (the documented count of
float vectors), and the trainer's choice of checkpoint interval under a memory budget."""
import types

import pytest

from paper_2212_05159_gb300 import abi, learned


def _size(n, n_it, s):
    return abi._size("spx_pcg_train_workspace_size", n, n_it, s)


def _documented(n, n_it, s):
    """5 (s + 1) + 6 + 2 ceil(n_it / s) float vectors for 1 <= s < n_it, else 5 (n_it + 1) + 6;
    plus the 256 bytes of alignment slack."""
    if 1 <= s < n_it:
        vectors = 5 * (s + 1) + 6 + 2 * (-(-n_it // s))
    else:
        vectors = 5 * (n_it + 1) + 6
    return vectors * n * 4 + 256


@pytest.mark.parametrize("n", [1, 1000, 65536, 3_000_000])
@pytest.mark.parametrize("n_it", [1, 2, 4, 10, 64])
def test_workspace_matches_the_documented_count(n, n_it):
    for s in range(0, n_it + 2):
        assert _size(n, n_it, s) == _documented(n, n_it, s), (n, n_it, s)


def test_checkpoints_shrink_the_workspace():
    n, n_it = 100_000, 64
    full = _size(n, n_it, 0)
    best = min(range(1, n_it), key=lambda s: _size(n, n_it, s))
    assert best == 5                                  # 5 s + 2 ceil(n_it / s): smallest near sqrt(2 n_it / 5) = 5.06
    assert _size(n, n_it, best) < full / 4
    assert _size(n, n_it, n_it) == full and _size(n, n_it, n_it + 5) == full


def test_workspace_rejects_bad_arguments():
    for n, n_it in [(-1, 4), (10, 0), (10, 65)]:
        with pytest.raises(abi.SpxError):
            _size(n, n_it, 0)


def _trainer(budget, n_it=64):
    net = types.SimpleNamespace(device="cpu")         # interval() touches only the sizes
    return learned.Trainer(net, n_it=n_it, gamma=0.9, checkpoint="auto", max_workspace_bytes=budget)


def test_auto_interval_keeps_everything_when_it_fits():
    n = 50_000
    assert _trainer(_size(n, 64, 0)).interval(n) == 0


def test_auto_interval_takes_the_largest_interval_that_fits():
    n = 50_000
    for s in (40, 17, 8):
        budget = _size(n, 64, s)
        got = _trainer(budget).interval(n)
        assert _size(n, 64, got) <= budget
        assert all(_size(n, 64, t) > budget for t in range(got + 1, 64))   # least recomputation


def test_auto_interval_falls_back_to_the_smallest_workspace():
    n = 50_000
    got = _trainer(1024).interval(n)
    assert _size(n, 64, got) == min(_size(n, 64, s) for s in range(1, 64))


def test_fixed_interval_is_taken_as_given():
    net = types.SimpleNamespace(device="cpu")
    assert learned.Trainer(net, n_it=10, checkpoint=3).interval(123) == 3
    assert learned.Trainer(net, n_it=10, checkpoint=0).interval(123) == 0


def test_loss_weights_are_normalised_geometric():
    """Section 4.3's weighted residual loss: weight gamma^(N_it - i) on iteration i, normalised."""
    w = learned.loss_weights(4, 0.6)
    assert abs(float(w.sum()) - 1.0) < 1e-6
    assert w[-1] == max(w)
    for i in range(3):
        assert abs(w[i] / w[i + 1] - 0.6) < 1e-6
