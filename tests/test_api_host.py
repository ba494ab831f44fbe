"""Host-side helpers of the Python binding (no GPU): block layout and initial multi-matrices."""
import numpy as np

from paper_2112_03985_gb300 import api


def test_left_out_csr_layout():
    ptr, idx = api.left_out_csr([[3], [], [0, 2]])
    assert list(ptr) == [0, 1, 1, 3] and list(idx) == [3, 0, 2]
    ptr, idx = api.left_out_csr([[], []])      # only full models: a one-element index array
    assert list(ptr) == [0, 0, 0] and idx.size == 1


def test_multi_init_places_blocks_side_by_side():
    rng = np.random.default_rng(2)
    blocks = [[rng.random((I, r)) for I in (4, 5)] for r in (2, 3, 1)]
    M = api.multi_init(blocks)
    assert [m.shape for m in M] == [(4, 6), (5, 6)]
    np.testing.assert_array_equal(M[1][:, 2:5], blocks[1][1])
    assert all(m.flags["C_CONTIGUOUS"] and m.dtype == np.float64 for m in M)


def test_init_from_model_repeats_the_model_per_submodel():
    """Alg. 2 / Alg. 3 initialisation: every submodel starts from the fitted model."""
    rng = np.random.default_rng(3)
    U = [rng.random((I, 4)) for I in (6, 5, 7)]
    M = api.init_from_model(U, 3)
    assert [m.shape for m in M] == [(6, 12), (5, 12), (7, 12)]
    for n in range(3):
        for g in range(3):
            np.testing.assert_array_equal(M[n][:, 4 * g:4 * g + 4], U[n])
