"""The seeded synthetic inputs (no GPU): each configuration has the shapes, block layout,
value distributions and noise level of its stated recipe, and is reproducible from its seeds."""
import numpy as np
import pytest

from paper_2112_03985_gb300 import workloads as W


def _noise_level(w):
    clean = W._cp_tensor(w.truth)
    return np.linalg.norm((w.T - clean).ravel()) / np.linalg.norm(clean.ravel())


@pytest.mark.parametrize("c", [1, 2, 5])
def test_configurations_are_reproducible(c):
    a, b = W.make_config(c), W.make_config(c)
    np.testing.assert_array_equal(a.T, b.T)
    for ga, gb in zip(a.init, b.init):
        for ua, ub in zip(ga, gb):
            np.testing.assert_array_equal(ua, ub)
    assert [list(D) for D in a.left_out] == [list(D) for D in b.left_out]


def test_configuration_1_recipe():
    w = W.make_config(1)
    assert w.dims == (20, 30, 40) and w.n_hat == 0 and w.sweeps == 50 and w.dtype == "f64"
    assert w.K == 21 and w.ranks == [3] * 21 and w.C == 63
    assert [list(D) for D in w.left_out[:20]] == [[p] for p in range(20)] and len(w.left_out[20]) == 0
    assert all(0.0 <= u.min() and u.max() <= 1.0 for u in w.truth)
    assert abs(_noise_level(w) - 0.01) < 1e-12


def test_configuration_2_recipe():
    w = W.make_config(2)
    assert w.dims == (300, 100, 50) and w.K == 300 and w.C == 1500 and w.sweeps == 100
    assert [list(D) for D in w.left_out] == [[p] for p in range(300)]
    # FP32 tensor: every value exactly representable
    np.testing.assert_array_equal(w.T.astype(np.float32).astype(np.float64), w.T)
    U1, U2, U3 = w.truth
    assert U1.min() > 0.0                                     # lognormal sample scores
    for U in (U2, U3):                                        # Gaussian bumps: peak 1 inside the mode
        assert U.min() >= 0.0 and U.max() <= 1.0
    assert abs(_noise_level(w) - 0.02) < 1e-6          # FP32 rounding of T on top of 2%


def test_configuration_5_recipe():
    w = W.make_config(5)
    assert w.dims == (100, 60, 60, 40) and w.K == 100 and w.ranks == [8] * 100 and w.n_hat == 0
    np.testing.assert_array_equal(w.T.astype(np.float32).astype(np.float64), w.T)
    assert abs(_noise_level(w) - 0.01) < 1e-6


def test_configuration_4_batch_recipe():
    ws = W.make_config4_batch(8)
    assert len(ws) == 8
    for w in ws:
        I1, I2, I3 = w.dims
        assert 20 <= I1 <= 400 and 30 <= I2 <= 150 and 30 <= I3 <= 150
        R = w.ranks[0]
        assert 2 <= R <= 8 and w.ranks == [R] * I1 and w.K == I1
        np.testing.assert_array_equal(w.T.astype(np.float32).astype(np.float64), w.T)
    assert len({w.dims for w in ws}) == len(ws)              # uneven sizes


def test_group_blocks_are_contiguous_and_cover_the_mode():
    b = W.group_blocks(400, 10)
    assert len(b) == 40
    assert np.array_equal(np.concatenate(b), np.arange(400))
    assert all(np.array_equal(D, np.arange(10 * g, 10 * g + 10)) for g, D in enumerate(b))


def test_all_ranks_layout_repeats_each_sample_per_rank():
    """Sec. 5.1 "All": every left-out sample once per rank, ranks cycling within a sample."""
    blocks, ranks = W.all_ranks_blocks(3, (3, 5))
    assert [list(b) for b in blocks] == [[0], [0], [1], [1], [2], [2]]
    assert ranks == [3, 5, 3, 5, 3, 5]
