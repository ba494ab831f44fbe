"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test pins a part of ``oracle/`` to something other than the oracle itself:
a hand-derived worked example, brute force, a closed form, an identity stated
by the paper (Sec. 4.1 Case I/II, Sec. 4.2 operation counts), an invariant of
ALS, or finite differences.
"""
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle as O
from paper_2112_03985_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _rng(s=0):
    return np.random.default_rng(s)


def _load_golden():
    unf, mtt = {}, {}
    with open(os.path.join(GOLDEN, "mttkrp_2x2x2.txt")) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            head, vals = line.split(":")
            kind, n, _, row = head.split()
            v = [float(x) for x in vals.split()]
            (unf if kind == "unfold" else mtt).setdefault(int(n), {})[int(row)] = v
    return unf, mtt


def _golden_problem():
    T = np.zeros((2, 2, 2))
    for i in range(2):
        for j in range(2):
            for k in range(2):
                T[i, j, k] = 1 + i + 2 * j + 4 * k
    U = [np.array([[1.0, 1], [2, -1]]), np.array([[1.0, 2], [3, 1]]), np.array([[2.0, 1], [1, -1]])]
    return T, U


# --------------------------------------------------------------------------- MTTKRP

def test_golden_unfold_and_mttkrp():
    """Hand-derived 2x2x2 example (tests/golden/mttkrp_2x2x2.txt)."""
    unf, mtt = _load_golden()
    T, U = _golden_problem()
    for n in range(3):
        Tn = O.unfold(T, n)
        M = O.mttkrp(T, U, n)
        Mb = O.mttkrp_bruteforce(T, U, n)
        for row in range(2):
            np.testing.assert_array_equal(Tn[row], unf[n][row])
            np.testing.assert_array_equal(M[row], mtt[n][row])
            np.testing.assert_array_equal(Mb[row], mtt[n][row])


@pytest.mark.parametrize("dims", [(3, 4, 5), (2, 3, 4, 5)])
def test_kolda_mapping(dims):
    """unfold() places T(i_1..i_N) at column j of Eq. kolda_mapping."""
    T = _rng(1).standard_normal(dims)
    for n in range(len(dims)):
        Tn = O.unfold(T, n)
        assert Tn.shape == (dims[n], int(np.prod(dims)) // dims[n])
        for idx in np.ndindex(*dims):
            assert Tn[idx[n], O.kolda_column(idx, dims, n)] == T[idx]


def test_khatri_rao_is_columnwise_kronecker():
    A, B = _rng(2).standard_normal((3, 4)), _rng(3).standard_normal((5, 4))
    K = O.khatri_rao(A, B)
    for r in range(4):
        np.testing.assert_array_equal(K[:, r], np.kron(A[:, r], B[:, r]))


@pytest.mark.parametrize("dims", [(3, 4, 5), (2, 3, 4, 5), (4, 1, 3)])
def test_mttkrp_vs_bruteforce(dims):
    rng = _rng(4)
    T = rng.standard_normal(dims)
    U = [rng.standard_normal((I, 3)) for I in dims]
    for n in range(len(dims)):
        np.testing.assert_allclose(O.mttkrp(T, U, n), O.mttkrp_bruteforce(T, U, n), rtol=1e-13, atol=1e-13)


def test_mttkrp_order2_is_gemm():
    """N = 2: M_1 = T U_2 and M_2 = T^T U_1."""
    rng = _rng(5)
    T = rng.standard_normal((7, 9))
    U = [rng.standard_normal((7, 4)), rng.standard_normal((9, 4))]
    np.testing.assert_allclose(O.mttkrp(T, U, 0), T @ U[1], rtol=1e-14)
    np.testing.assert_allclose(O.mttkrp(T, U, 1), T.T @ U[0], rtol=1e-14)


def test_mttkrp_rank1_closed_form():
    """T = a o b o c and rank-1 factors u_k: M_1 = a (b.u_2)(c.u_3), etc."""
    rng = _rng(6)
    a, b, c = rng.standard_normal(6), rng.standard_normal(7), rng.standard_normal(8)
    T = np.multiply.outer(np.multiply.outer(a, b), c)
    u = [rng.standard_normal((6, 1)), rng.standard_normal((7, 1)), rng.standard_normal((8, 1))]
    np.testing.assert_allclose(O.mttkrp(T, u, 0)[:, 0], a * (b @ u[1][:, 0]) * (c @ u[2][:, 0]), rtol=1e-13)
    np.testing.assert_allclose(O.mttkrp(T, u, 1)[:, 0], b * (a @ u[0][:, 0]) * (c @ u[2][:, 0]), rtol=1e-13)
    np.testing.assert_allclose(O.mttkrp(T, u, 2)[:, 0], c * (a @ u[0][:, 0]) * (b @ u[1][:, 0]), rtol=1e-13)


@pytest.mark.parametrize("dims,n_hat,d", [((6, 4, 5), 0, 1), ((6, 4, 5), 1, 2), ((4, 3, 5, 2), 2, 1)])
def test_case_I_and_II_identity(dims, n_hat, d):
    """Sec. 4.1: the zero-padded concurrent MTTKRP on the full tensor equals every
    submodel's own MTTKRP on its sliced tensor; Case I rows D_g are discarded."""
    rng = _rng(7)
    T = rng.standard_normal(dims)
    I = dims[n_hat]
    blocks = W.group_blocks(I, d) if d > 1 else W.loo_blocks(I, include_full=True)
    ranks = [2 + (g % 3) for g in range(len(blocks))]
    offs = np.concatenate([[0], np.cumsum(ranks)])
    sub = [[rng.standard_normal((dims[k] - (len(D) if k == n_hat else 0), R)) for k in range(len(dims))]
           for D, R in zip(blocks, ranks)]
    Ubar = [np.concatenate([O.insert_zero_rows(s[k], dims[k], D) if k == n_hat else s[k]
                            for s, D in zip(sub, blocks)], axis=1) for k in range(len(dims))]
    for n in range(len(dims)):
        Mbar = O.concurrent_mttkrp_padded(T, Ubar, n)
        for g, D in enumerate(blocks):
            Tg = O.slice_tensor(T, n_hat, D)
            Mg = O.mttkrp(Tg, sub[g], n)
            Mpad = Mbar[:, offs[g]:offs[g + 1]]
            if n == n_hat:
                Mpad = O.remove_rows(Mpad, D)        # Case I: E_p discards rows
            err = np.linalg.norm(Mpad - Mg) / max(np.linalg.norm(Mg), 1e-300)
            assert err <= 1e-14, (n, g, err)


# --------------------------------------------------------------------------- solve / loss

def test_solve_residual_and_not_spd():
    rng = _rng(8)
    A = rng.standard_normal((30, 6))
    H = A.T @ A
    M = rng.standard_normal((11, 6))
    U = O.solve_normal_equations(M, H)
    assert np.linalg.norm(U @ H - M) / np.linalg.norm(M) <= 1e-13
    A[:, 3] = A[:, 2]                                  # duplicate column: singular H
    with pytest.raises(O.NotSPD):
        O.solve_normal_equations(M, A.T @ A - 1e-9 * np.eye(6))


def test_loss_formula_sign_against_explicit():
    """Alg. 1 error line, sign read as '+': equals ||T - [[U]]||^2 for any factors."""
    rng = _rng(9)
    T = rng.standard_normal((5, 6, 7))
    U = [rng.standard_normal((I, 3)) for I in T.shape]
    M = O.mttkrp(T, U, 2)
    H = O.hadamard_of_grams(U, 2)
    e = O.cp_loss_efficient(float(np.sum(T * T)), H, U[2], M)
    assert abs(e - O.cp_loss_explicit(T, U)) <= 1e-12 * np.sum(T * T)
    e_minus = float(np.sum(T * T) - np.sum(H * O.gram(U[2])) - 2 * np.sum(U[2] * M))
    assert abs(e_minus - O.cp_loss_explicit(T, U)) > 1e-3   # the printed sign does not hold


def test_als_loss_monotone_and_efficient_equals_explicit():
    """ALS solves each mode's least-squares problem exactly (Sec. 3.2), so the loss
    never increases after a mode update; the efficient error equals the explicit one."""
    w = W.make_workload("t", (8, 9, 10), 3, noise=0.05, seed=11)
    r = O.cp_als(w.T, w.init[0], 15, normalise=False, record_explicit=True, record_modes=True)
    ml = np.array(r.mode_losses)
    assert np.all(ml[1:] <= ml[:-1] * (1 + 1e-12))
    np.testing.assert_allclose(r.losses, r.explicit_losses, rtol=1e-10)


def test_normalisation_does_not_change_loss_path():
    w = W.make_workload("t", (8, 9, 10), 3, noise=0.05, seed=12)
    a = O.cp_als(w.T, w.init[0], 12, normalise=True)
    b = O.cp_als(w.T, w.init[0], 12, normalise=False)
    np.testing.assert_allclose(a.losses, b.losses, rtol=1e-9)
    np.testing.assert_allclose(O.cp_reconstruct(a.factors), O.cp_reconstruct(b.factors), rtol=1e-8, atol=1e-10)
    for u in a.factors[:-1]:
        np.testing.assert_allclose(np.linalg.norm(u, axis=0), 1.0, rtol=1e-13)


def test_planted_recovery_noise_free():
    """Exact recovery of a planted noise-free rank-3 tensor (well conditioned, near init)."""
    rng = _rng(13)
    truth = [rng.standard_normal((I, 3)) for I in (8, 9, 10)]
    T = O.cp_reconstruct(truth)
    init = [u + 1e-2 * rng.standard_normal(u.shape) for u in truth]
    r = O.cp_als(T, init, 200)
    nT2 = np.sum(T * T)
    # the efficient error formula cancels down to about eps * ||T||^2; the
    # explicit residual shows the exact fit
    assert r.losses[-1] <= 1e-13 * nT2
    assert O.cp_loss_explicit(T, r.factors) <= 1e-20 * nT2
    for k in range(3):
        a = r.factors[k] / np.linalg.norm(r.factors[k], axis=0)
        b = truth[k] / np.linalg.norm(truth[k], axis=0)
        cong = np.abs(np.diag(a.T @ b))
        assert np.all(cong > 1 - 1e-10)


def test_not_spd_block_is_flagged():
    w = W.make_workload("t", (6, 7, 8), 3, noise=0.01, seed=14)
    init = [u.copy() for u in w.init[0]]
    for u in init:
        u[:, 1] = u[:, 0]          # identical columns in every mode -> singular H
    r = O.cp_als(w.T, init, 3)
    assert r.not_spd


def test_tolerance_stop():
    w = W.make_workload("t", (8, 9, 10), 2, noise=0.0, seed=15)
    r = O.cp_als(w.T, w.init[0], 500, tol=1e-3)
    assert r.converged and r.sweeps_done < 500


# --------------------------------------------------------------------------- jackknife

def test_jk_als_blocks_match_separate_cp_als():
    w = W.make_workload("t", (6, 5, 4), 2, noise=0.01, seed=16, sweeps=5)
    r = O.jk_als(w.T, 0, w.left_out, w.init, 5)
    for g in (0, 3):
        D = w.left_out[g]
        Tg = O.slice_tensor(w.T, 0, D)
        assert Tg.shape == (5, 5, 4)
        s = O.cp_als(Tg, [O.remove_rows(w.init[g][0], D), w.init[g][1], w.init[g][2]], 5)
        np.testing.assert_array_equal(O.remove_rows(r.factors[g][0], D), s.factors[0])
        assert np.all(r.factors[g][0][D] == 0)
        np.testing.assert_allclose(r.normT2[g], np.sum(Tg * Tg))


def test_noise_free_jackknife_submodels_agree_after_adjustment():
    """An exact low-rank tensor stays exact when a slice is removed, so every leave-one-out
    submodel recovers the planted model.  Started from column orders permuted per submodel,
    the adjustment must undo each permutation; the jackknife SE then vanishes for the middle mode
    and for the column directions of the last mode (its column scales and signs differ by
    design: they carry the norms and sign flips of the sampled mode's columns, which lose a
    different row per submodel)."""
    rng = _rng(22)
    dims, R = (9, 8, 7), 3
    truth = [rng.standard_normal((I, R)) for I in dims]
    T = O.cp_reconstruct(truth)
    blocks = W.loo_blocks(dims[0])
    perms, init = [], []
    for _ in blocks:
        q = rng.permutation(R)
        perms.append(q)
        init.append([u[:, q] + 1e-3 * rng.standard_normal(u.shape) for u in truth])
    r = O.jk_als(T, 0, blocks, init, 300)
    est = []
    for g, D in enumerate(blocks):
        Tg = O.slice_tensor(T, 0, D)
        Ug = [O.remove_rows(r.factors[g][0], D), r.factors[g][1], r.factors[g][2]]
        assert O.cp_loss_explicit(Tg, Ug) <= 1e-20 * np.sum(Tg * Tg)
        A, p = O.align_to_reference(r.factors[g], truth, 0, return_perm=True)
        assert [int(perms[g][j]) for j in p] == list(range(R))
        last = A[2] / np.linalg.norm(A[2], axis=0)
        last = last * np.sign(last[np.abs(last).argmax(axis=0), np.arange(R)])
        est.append(np.concatenate([A[1].ravel(), last.ravel()]))
    est = np.asarray(est)
    assert O.jackknife_se(est).max() <= 1e-9 * np.abs(est).max()


def test_jackknife_se_of_mean_is_s_over_sqrt_n():
    """Textbook identity: the jackknife SE of the sample mean equals s / sqrt(n)."""
    x = _rng(17).standard_normal(23)
    loo = np.array([np.delete(x, i).mean() for i in range(x.size)])
    assert abs(O.jackknife_se(loo) - x.std(ddof=1) / np.sqrt(x.size)) <= 1e-14


def test_grouped_jackknife_se_of_mean_is_se_of_group_means():
    """Delete-d with G equal groups: leaving out group g moves the mean by -(ybar_g - xbar)/(G-1),
    so the grouped jackknife SE of the mean equals std(group means, ddof=1) / sqrt(G)."""
    G, d = 9, 4
    x = _rng(21).standard_normal(G * d)
    groups = x.reshape(G, d)
    est = np.array([np.delete(x, np.arange(g * d, (g + 1) * d)).mean() for g in range(G)])
    want = groups.mean(axis=1).std(ddof=1) / np.sqrt(G)
    assert abs(O.jackknife_se(est) - want) <= 1e-14


def test_alignment_recovers_permutation_and_signs():
    rng = _rng(18)
    ref = [rng.standard_normal((I, 4)) for I in (5, 6, 7)]
    for k in range(2):
        ref[k] /= np.linalg.norm(ref[k], axis=0)
    perm = [2, 0, 3, 1]
    sub = [u[:, perm].copy() for u in ref]
    sub[0][:, 1] *= -1
    sub[2][:, 1] *= -1          # sign flip compensated in the last mode
    al = O.align_to_reference(sub, ref, n_hat=0)
    ref_fixed = O.sign_fix(ref, 2)
    for k in range(3):
        np.testing.assert_allclose(al[k], ref_fixed[k], rtol=1e-14, atol=1e-15)


@pytest.mark.parametrize("R", [8, 10, 20])
def test_alignment_recovers_a_planted_permutation(R):
    """Brute force (R = 8, 40320 permutations) and the assignment solver (R > 8) both
    undo a planted column permutation with sign flips under small noise."""
    rng = _rng(19 + R)
    dims = (9, 30, 25)
    ref = [rng.standard_normal((I, R)) for I in dims]
    q = rng.permutation(R)
    sub = [u[:, q] + 1e-3 * rng.standard_normal((u.shape[0], R)) for u in ref]
    flip = rng.integers(0, 2, size=R) * 2 - 1
    sub[1] = sub[1] * flip[None, :]
    sub[2] = sub[2] * flip[None, :]
    al, perm = O.align_to_reference(sub, ref, n_hat=0, return_perm=True)
    assert [int(q[p]) for p in perm] == list(range(R))   # sub column perm[s] is ref column s
    ref_fixed = O.sign_fix(ref, 2)
    for k in (1, 2):
        assert np.abs(al[k] - ref_fixed[k]).max() <= 1e-2


def test_flop_counts_sec_4_2():
    """Sec. 4.2: JK-CALS / JK-ALS MTTKRP flops = I/(I-d) <= 2; the JK-ALS count
    equals 2R times the element count of the sliced tensors actually fitted."""
    for dims, d in [((20, 30, 40), 1), ((400, 40, 50), 10), ((8, 3, 3), 4)]:
        R = 5
        a, c = O.flops_jk_als(dims, 0, d, R), O.flops_jk_cals(dims, 0, d, R)
        assert Fraction(c, a) == Fraction(dims[0], dims[0] - d) <= 2
        T = np.zeros(dims)
        blocks = W.group_blocks(dims[0], d) if d > 1 else W.loo_blocks(dims[0])
        assert a == sum(2 * R * O.slice_tensor(T, 0, D).size for D in blocks)


# --------------------------------------------------------------------------- gradient

def test_gradient_central_differences():
    """d/dU sum_g ||T_{-g} - [[U^(g)]]||^2 against FP64 central differences (10x8x8x6, R=2)."""
    rng = _rng(19)
    dims = (10, 8, 8, 6)
    T = rng.standard_normal(dims)
    blocks = W.loo_blocks(10)[:3]
    ranks = [2] * 3
    Ubar = [rng.standard_normal((I, 6)) for I in dims]
    for g, D in enumerate(blocks):
        Ubar[0][D, 2 * g:2 * g + 2] = 0.0
    f0, G = O.jk_loss_grad(T, 0, blocks, ranks, Ubar)
    checked = 0
    for k in range(4):
        for (i, c) in [(1, 0), (3, 5), (dims[k] - 1, 3)]:
            if k == 0 and any(i in D and 2 * g <= c < 2 * g + 2 for g, D in enumerate(blocks)):
                continue
            h = 1e-6 * max(1.0, abs(Ubar[k][i, c]))
            Up = [u.copy() for u in Ubar]
            Um = [u.copy() for u in Ubar]
            Up[k][i, c] += h
            Um[k][i, c] -= h
            fd = (O.jk_loss_grad(T, 0, blocks, ranks, Up)[0] - O.jk_loss_grad(T, 0, blocks, ranks, Um)[0]) / (2 * h)
            assert abs(fd - G[k][i, c]) <= 1e-7 * max(1.0, abs(fd)), (k, i, c, fd, G[k][i, c])
            checked += 1
    assert checked >= 10
