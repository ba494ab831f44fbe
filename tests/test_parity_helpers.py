"""The comparison helpers of the GPU parity tests, checked on the CPU with the
oracle on both sides and mistakes planted on one side: element-wise parity
catches an error that a relative Frobenius norm would hide; the derived loss
bound holds for a legitimately perturbed model and rejects a planted loss error;
the standard-error bound holds for any pair of estimate sets."""
import numpy as np
import pytest

import oracle as O

from _helpers import assert_elementwise, loss_bound, reconstruct, se_perturbation_bound


def test_reconstruct_equals_the_oracle_reconstruction():
    rng = np.random.default_rng(0)
    for dims in [(4, 5, 6), (3, 4, 2, 5)]:
        U = [rng.standard_normal((I, 3)) for I in dims]
        np.testing.assert_allclose(reconstruct(U), O.cp_reconstruct(U), rtol=0, atol=1e-13)


def test_elementwise_parity_catches_one_wrong_small_entry():
    rng = np.random.default_rng(1)
    ref = rng.uniform(0.5, 1.0, size=(200, 50))
    ref[17, 3] = 1e-3                       # a small entry, e.g. a ragged tail element
    got = ref.copy()
    got[17, 3] *= 1.0 + 5e-4                # wrong in its fourth digit
    frob = np.linalg.norm(got - ref) / np.linalg.norm(ref)
    assert frob < 1e-8                      # a 1e-8 Frobenius bar would pass it
    with pytest.raises(AssertionError):
        assert_elementwise(got, ref, 1e-8)
    assert assert_elementwise(ref, ref, 1e-12) == 0.0


def _als_pair(seed, delta):
    """A 1%-noise rank-2 problem fitted 3 sweeps by the oracle, and the same fit
    from an initial point moved by `delta` (a legitimately different model)."""
    rng = np.random.default_rng(seed)
    dims = (8, 7, 6)
    A = [rng.uniform(0, 1, size=(I, 2)) for I in dims]
    T = O.cp_reconstruct(A)
    E = rng.standard_normal(dims)
    T = T + 0.01 * np.linalg.norm(T) / np.linalg.norm(E) * E
    U0 = [rng.uniform(0, 1, size=(I, 2)) for I in dims]
    a = O.cp_als(T, U0, 3)
    b = O.cp_als(T, [u + delta * rng.standard_normal(u.shape) for u in U0], 3)
    return T, a, b


def test_loss_bound_holds_for_a_perturbed_model_and_rejects_a_planted_error():
    T, a, b = _als_pair(2, 1e-7)
    eps_m = 1e-8
    # "GPU" side: model b, its loss through the efficient formula with the last
    # mode's MTTKRP perturbed by a relative eps_m (worst-case direction: along U_N)
    N = T.ndim
    M = O.mttkrp(T, b.factors, N - 1)
    dM = eps_m * np.linalg.norm(M) * b.factors[N - 1] / np.linalg.norm(b.factors[N - 1])
    H = O.hadamard_of_grams(b.factors, N - 1)
    e_gpu = O.cp_loss_efficient(float(np.sum(T * T)), H, b.factors[N - 1], M + dM)
    e_ora = a.losses[-1]
    bound = loss_bound(T, b.factors, a.factors, eps_m)
    assert abs(e_gpu - e_ora) <= bound
    # the bound is not vacuous: a loss off by 10x the bound is rejected
    assert abs((e_ora + 10 * bound) - e_ora) > bound
    # and the distance term grows with the model difference
    _, a2, b2 = _als_pair(2, 1e-4)
    assert loss_bound(T, b2.factors, a2.factors, eps_m) > 10 * bound


def test_se_perturbation_bound_is_the_reverse_triangle_inequality():
    rng = np.random.default_rng(3)
    a = rng.standard_normal((30, 40))
    for scale in (1e-9, 1e-3, 1.0):
        b = a + scale * rng.standard_normal(a.shape)
        d = np.abs(O.jackknife_se(a) - O.jackknife_se(b))
        assert np.all(d <= se_perturbation_bound(a, b) * (1 + 1e-12) + 1e-15)
    # a shift shared by every submodel moves no standard error and no bound
    np.testing.assert_allclose(se_perturbation_bound(a, a + 0.5), 0.0, atol=1e-14)
