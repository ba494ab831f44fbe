"""GPU parity of the Alg. 2 post-processing on the device (jkcals_jackknife_se): every
submodel adjusted to a reference model (signs, then the best column permutation), and the
jackknife standard errors, against the oracle's align_to_reference and jackknife_se on the
same factors.  Permutations are index results and must agree exactly; the adjusted factors
are the handle's own entries permuted and negated, so they must agree exactly too; the
standard errors are sums in submodel order on both sides (1e-13 relative)."""
import numpy as np
import pytest

import oracle as O
from paper_2112_03985_gb300 import api, workloads as W

from _helpers import offsets

pytestmark = pytest.mark.gpu


def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _check(w_ranks, n_hat, left_out, U, ref, S, perm, aligned):
    offs = offsets(w_ranks)
    sub = [g for g in range(len(w_ranks)) if len(left_out[g]) > 0]
    est = []
    for i, g in enumerate(sub):
        Ug = [u[:, offs[g]:offs[g + 1]] for u in U]
        A, p = O.align_to_reference(Ug, ref, n_hat, return_perm=True)
        np.testing.assert_array_equal(perm[i], np.asarray(p, dtype=np.int32))
        for n in range(len(U)):
            np.testing.assert_array_equal(aligned[n][i], A[n])
        est.append(np.concatenate([A[n].ravel() for n in range(len(U)) if n != n_hat]))
    se = O.jackknife_se(np.asarray(est))
    got = np.concatenate([S[n].ravel() for n in range(len(U)) if n != n_hat])
    assert S[n_hat] is None
    np.testing.assert_allclose(got, se, rtol=1e-13, atol=1e-15 * np.abs(se).max())


def test_se_cfg1_against_the_full_model_block():
    """Configuration 1 (20 leave-one-out submodels and the full model, R = 3), 50 sweeps;
    the reference is the full-model block fitted in the same handle."""
    _cuda()
    w = W.make_config(1)
    full = [g for g in range(w.K) if len(w.left_out[g]) == 0]
    assert full
    with api.from_workload(w) as h:
        h.als_sweep(w.sweeps)
        U = h.get_factors()
        S, perm, aligned = h.jackknife_se(ref_block=full[0])
    offs = offsets(w.ranks)
    ref = [u[:, offs[full[0]]:offs[full[0] + 1]] for u in U]
    _check(w.ranks, w.n_hat, w.left_out, U, ref, S, perm, aligned)


def test_se_four_way_delete_groups_sampled_mode_two():
    """Four-way tensor, sampled mode 2, delete-2 groups (the grouped jackknife), 20 sweeps;
    the reference is the first submodel itself (its own permutation is the identity)."""
    _cuda()
    w = W.make_workload("t", (6, 5, 8, 7), 3, n_hat=2, blocks=W.group_blocks(8, 2), noise=0.01, seed=12)
    with api.from_workload(w) as h:
        h.als_sweep(20)
        U = h.get_factors()
        S, perm, aligned = h.jackknife_se(ref_block=0)
    ref = [u[:, 0:3] for u in U]
    np.testing.assert_array_equal(perm[0], np.arange(3, dtype=np.int32))
    _check(w.ranks, w.n_hat, w.left_out, U, ref, S, perm, aligned)


@pytest.mark.parametrize("R", [5, 8, 10, 20])
def test_se_planted_permutations_external_reference(R):
    """Submodels planted as the reference with permuted, sign-flipped columns plus noise:
    brute force (R <= 8) and the assignment solver (R > 8) both recover the planted
    permutation, and agree with the oracle exactly."""
    _cuda()
    dims = (10, 30, 25)
    rng = np.random.default_rng(70 + R)
    K = dims[0]
    blocks = W.loo_blocks(K)
    ref = [rng.standard_normal((I, R)) for I in dims]
    U = [np.zeros((I, R * K)) for I in dims]
    planted = []
    for g in range(K):
        q = rng.permutation(R)
        flip = rng.integers(0, 2, size=R) * 2 - 1
        for n in range(3):
            col = ref[n][:, q] + 1e-3 * rng.standard_normal((dims[n], R))
            if n in (1, 2):
                col = col * flip[None, :]
            U[n][:, g * R:(g + 1) * R] = col
        U[0][g, g * R:(g + 1) * R] = 0.0   # the left-out row
        planted.append(q)
    T = rng.standard_normal(dims)
    with api.JKCALS(T, 0, [R] * K, blocks, [u.copy() for u in U]) as h:
        h.set_factors(U)
        Uh = h.get_factors()
        S, perm, aligned = h.jackknife_se(ref=ref)
    for g in range(K):
        assert [int(planted[g][p]) for p in perm[g]] == list(range(R))
    _check([R] * K, 0, blocks, Uh, ref, S, perm, aligned)


def test_se_argument_errors():
    _cuda()
    w = W.make_workload("t", (6, 5, 4), 2, blocks=[np.array([0]), np.zeros(0, dtype=np.int64)], seed=3)
    with api.from_workload(w) as h:
        with pytest.raises(api.JKError):        # one submodel only
            h.jackknife_se(ref_block=1)
    w = W.make_workload("t", (6, 5, 4), 2, blocks=W.loo_blocks(6), seed=3, ranks=[2, 2, 3, 2, 2, 2])
    with api.from_workload(w) as h:
        with pytest.raises(api.JKError):        # submodels of different ranks
            h.jackknife_se(ref_block=0)
