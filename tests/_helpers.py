"""Shared test helpers: oracle-side references and comparisons (no library code).

Parity is asserted element by element: every entry of a GPU result must satisfy
|got - ref| <= bar * (|ref| + max|ref|) against the oracle's value, with bar the
tolerance of the form (numpy's assert_allclose with rtol = bar and atol =
bar * max|ref| over the compared block).  The relative Frobenius error is
returned as well, as a report.
"""
import numpy as np

import oracle as O


def offsets(ranks):
    return np.concatenate([[0], np.cumsum(ranks)]).astype(int)


def assert_elementwise(got, ref, bar, what=""):
    """Element-wise parity at the bar; returns the relative Frobenius error."""
    got = np.asarray(got)
    ref = np.asarray(ref)
    assert got.shape == ref.shape, (what, got.shape, ref.shape)
    scale = float(np.abs(ref).max()) if ref.size else 0.0
    np.testing.assert_allclose(got, ref, rtol=bar, atol=bar * scale, err_msg=what)
    return float(np.linalg.norm(got - ref) / max(np.linalg.norm(ref), 1e-300))


def oracle_block_mttkrp(w, U_multi, n, g):
    """Submodel g's own MTTKRP on its sliced tensor (Alg. 2 fitting step), from the
    block's columns of the multi-matrices, rows D_g removed in the sampled mode."""
    offs = offsets(w.ranks)
    cols = slice(offs[g], offs[g + 1])
    D = np.asarray(w.left_out[g], dtype=np.int64)
    Tg = O.slice_tensor(w.T, w.n_hat, D)
    Ug = [O.remove_rows(U_multi[k][:, cols], D) if k == w.n_hat else U_multi[k][:, cols]
          for k in range(w.T.ndim)]
    return O.mttkrp(Tg, Ug, n)


def compare_mttkrp(w, M_gpu, U_multi, n, rtol, blocks=None):
    """Element-wise parity of the concurrent MTTKRP against each submodel's own
    MTTKRP (Case I rows D_g dropped), block by block.  Returns the largest
    relative Frobenius error over the blocks (a report)."""
    offs = offsets(w.ranks)
    worst = 0.0
    for g in (range(w.K) if blocks is None else blocks):
        ref = oracle_block_mttkrp(w, U_multi, n, g)
        got = M_gpu[:, offs[g]:offs[g + 1]]
        if n == w.n_hat:
            got = O.remove_rows(got, w.left_out[g])
        worst = max(worst, assert_elementwise(got, ref, rtol, f"mode {n} block {g}"))
    return worst


def factor_errors(w, U_gpu, ref_factors, blocks):
    """Relative Frobenius error per (block, mode) of the GPU factors against the
    oracle's re-expanded per-submodel factors ref_factors[col][n] (a report)."""
    offs = offsets(w.ranks)
    errs = np.zeros((len(blocks), w.T.ndim))
    for col, g in enumerate(blocks):
        for n in range(w.T.ndim):
            ref = ref_factors[col][n]
            got = U_gpu[n][:, offs[g]:offs[g + 1]]
            errs[col, n] = np.linalg.norm(got - ref) / max(np.linalg.norm(ref), 1e-300)
    return errs


def assert_factors(w, U_gpu, ref_factors, blocks, bar):
    """Element-wise parity of the GPU factors with the oracle's re-expanded
    per-submodel factors ref_factors[col][n], per (block, mode); returns the
    relative Frobenius errors (blocks x modes) as a report."""
    offs = offsets(w.ranks)
    for col, g in enumerate(blocks):
        for n in range(w.T.ndim):
            assert_elementwise(U_gpu[n][:, offs[g]:offs[g + 1]], ref_factors[col][n], bar,
                               f"factors: block {g} mode {n}")
    return factor_errors(w, U_gpu, ref_factors, blocks)


def block_factors(w, U_multi, g):
    """Submodel g's factors from the multi-matrices, rows D_g removed in the sampled mode."""
    offs = offsets(w.ranks)
    D = np.asarray(w.left_out[g], dtype=np.int64)
    return [O.remove_rows(u[:, offs[g]:offs[g + 1]], D) if k == w.n_hat else u[:, offs[g]:offs[g + 1]]
            for k, u in enumerate(U_multi)]


def reconstruct(U):
    """[[U]] through the mode-0 unfolding X_(0) = U_0 KRP_0^T (oracle primitives)."""
    dims = [u.shape[0] for u in U]
    X0 = U[0] @ O.krp_except(U, 0).T
    return np.reshape(X0, dims, order="F")


def loss_bound(Tg, U_gpu_g, U_ora_g, eps_m):
    """Bound on |e_gpu - e_ora| for one submodel after a sweep (Alg. 3 error line),
    from what each side computes:

    * the oracle's e is ||T_g - X||^2 with X = [[U_ora]] (FP64, pinned against the
      explicit reconstruction);
    * the GPU's e is the same formula on its own factors U' with the last mode's
      MTTKRP M'_N carrying a relative error of at most eps_m (the form's MTTKRP
      bar), so e_gpu = ||T_g - X'||^2 - 2 <U'_N, dM'_N> and the second term is at
      most 2 eps_m ||U'_N|| ||M'_N||;
    * ||T - X'||^2 - ||T - X||^2 = -2 <T - X, X' - X> + ||X' - X||^2 exactly, so
      by Cauchy-Schwarz it is at most 2 ||T - X|| ||X' - X|| + ||X' - X||^2.

    A slack of 1e-12 ||T_g||^2 covers FP64 rounding of the two evaluations."""
    X = reconstruct(U_ora_g)
    Xp = reconstruct(U_gpu_g)
    r = float(np.linalg.norm(Tg - X))
    dx = float(np.linalg.norm(Xp - X))
    N = Tg.ndim
    Mp = O.mttkrp(Tg, U_gpu_g, N - 1)
    return (2.0 * eps_m * float(np.linalg.norm(U_gpu_g[N - 1])) * float(np.linalg.norm(Mp))
            + 2.0 * r * dx + dx * dx + 1e-12 * float(np.sum(Tg * Tg)))


def stepwise_loss_check(w, h, blocks, sweeps, eps_m, check_at=None, inits=None):
    """Runs `sweeps` sweeps on the handle one at a time and the oracle's Alg. 1 on
    each sampled submodel's sliced tensor alongside (from w.init[g], or inits[g]),
    and asserts after each sweep in `check_at` (default: all) that the GPU loss is
    within loss_bound of the oracle's.  Returns (GPU losses sweeps x K, oracle
    losses sweeps x len(blocks), the largest |diff| / bound, final oracle factors
    re-expanded)."""
    check_at = set(range(1, sweeps + 1)) if check_at is None else set(check_at)
    state = []
    for g in blocks:
        D = np.asarray(w.left_out[g], dtype=np.int64)
        Tg = O.slice_tensor(w.T, w.n_hat, D)
        init = w.init[g] if inits is None else inits[g]
        U0 = [O.remove_rows(u, D) if k == w.n_hat else np.array(u) for k, u in enumerate(init)]
        state.append([Tg, [O.unfold(Tg, n) for n in range(Tg.ndim)], U0])
    L = np.zeros((sweeps, w.K))
    Lo = np.zeros((sweeps, len(blocks)))
    worst = 0.0
    for k in range(1, sweeps + 1):
        L[k - 1] = h.als_sweep(1)[0]
        Ug = h.get_factors() if k in check_at else None
        for col, (g, st) in enumerate(zip(blocks, state)):
            r = O.cp_als(st[0], st[2], 1, unfoldings=st[1])
            st[2] = r.factors
            Lo[k - 1, col] = r.losses[0]
            if Ug is not None:
                b = loss_bound(st[0], block_factors(w, Ug, g), st[2], eps_m)
                d = abs(L[k - 1, g] - Lo[k - 1, col])
                worst = max(worst, d / b)
                assert d <= b, f"sweep {k} block {g}: |e_gpu - e_ora| = {d:.3e} > bound {b:.3e}"
    facs = []
    for g, st in zip(blocks, state):
        D = np.asarray(w.left_out[g], dtype=np.int64)
        facs.append([O.insert_zero_rows(u, w.T.shape[k], D) if k == w.n_hat else u for k, u in enumerate(st[2])])
    return L, Lo, worst, facs


def se_perturbation_bound(est_a, est_b):
    """Per-entry bound on |SE(a) - SE(b)| for two sets of jackknife estimates
    (G x p): SE(x) = sqrt((G-1)/G) ||x - mean(x)|| over the G submodels, so the
    reverse triangle inequality gives |SE(a) - SE(b)| <= SE(a - b) exactly."""
    return O.jackknife_se(np.asarray(est_a) - np.asarray(est_b))
