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


def _noalloc_args(dims=(4, 5, 6), C=3, mode=1):
    import torch
    U = [torch.zeros((I, C), dtype=torch.float64) for I in dims]
    J = int(np.prod([d for k, d in enumerate(dims) if k != mode]))
    Tn = torch.zeros((dims[mode], J), dtype=torch.float64)
    out = torch.zeros((dims[mode], C), dtype=torch.float64)
    return Tn, U, out


def test_noalloc_binding_accepts_consistent_shapes_and_a_missing_U_mode():
    Tn, U, out = _noalloc_args()
    assert api._check_noalloc_args(Tn, U, 1, out) == ([4, 5, 6], 3)
    U[1] = None                                # not read by the kernel
    assert api._check_noalloc_args(Tn, U, 1, out) == ([4, 5, 6], 3)


def test_noalloc_binding_rejects_what_the_c_abi_cannot_see():
    """The C ABI sees only pointers, so sizes and dtypes are checked in the binding:
    each mistake below would make the kernels read or write past a buffer's end."""
    import pytest
    import torch
    cases = []
    Tn, U, out = _noalloc_args()
    cases.append(("float64", (Tn.float(), U, out)))                          # wrong dtype
    Tn, U, out = _noalloc_args()
    cases.append(("unfolding", (Tn[:, :-1].contiguous(), U, out)))          # J too small
    Tn, U, out = _noalloc_args()
    cases.append(("out must be", (Tn, U, torch.zeros((5, 4), dtype=torch.float64))))
    Tn, U, out = _noalloc_args()
    U[2] = torch.zeros((6, 4), dtype=torch.float64)                         # C mismatch
    cases.append(("columns", (Tn, U, out)))
    Tn, U, out = _noalloc_args()
    cases.append(("contiguous", (Tn, [U[0], U[1], U[2].t().contiguous().t()], out)))
    Tn, U, out = _noalloc_args()
    U[0] = None                                                             # a factor that is read
    cases.append(("missing", (Tn, U, out)))
    Tn, U, out = _noalloc_args()
    cases.append(("matrix", (Tn.reshape(-1), U, out)))
    for what, (t, u, o) in cases:
        with pytest.raises(ValueError, match=what):
            api._check_noalloc_args(t, u, 1, o)
    Tn, U, out = _noalloc_args()
    with pytest.raises(ValueError, match="mode"):
        api._check_noalloc_args(Tn, U, 3, out)
