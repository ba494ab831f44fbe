"""FP64 CPU oracle for jackknife CP-ALS -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this module.  The library (``paper_2112_03985_gb300``)
never calls it, and it shares no code with the CUDA path.

It computes the *straightforward* workflow of the paper: every jackknife
submodel is fitted on its own, explicitly sliced tensor (JK-ALS, Alg. 2), with
plain CP-ALS (Alg. 1) inside.  Everything is float64 NumPy; the only library
primitives used as steps are matrix products, ``numpy.linalg.cholesky`` and
triangular solves.

Readings of points where the paper is silent or garbled (applied identically
by the CUDA path):

* Error formula (Alg. 1 error line, Alg. 3 error line): the printed formula
  subtracts the model-norm term.  Since ||T - M||^2 = ||T||^2 + ||M||^2 -
  2<T, M>, with ||M||^2 = sum(H_N * U_N^T U_N) and <T, M> = sum(U_N * M_N),
  the sign is read as "+".  ``test_oracle_pins`` pins it against the explicit
  reconstruction.
* Pseudoinverse (Alg. 1 update line): H_n is symmetric positive definite when
  the factors have full column rank, so U_n = M_n H_n^{-1} is taken by a
  Cholesky solve.  A non-positive pivot marks the submodel NOT_SPD and freezes
  it (its factors stay as they were before the failing update).
* Column normalisation (not in the paper): after updating mode n < N-1
  (0-based), every column of U_n is scaled to unit 2-norm and the norm is
  dropped; a zero column is left untouched.  Each ALS update is invariant to
  column scaling of the other factors, so the loss after the last mode equals
  that of unnormalised ALS.
* Order inside one mode update (Alg. 3): solve, zero the left-out rows (only
  for the sampled mode), normalise, then refresh the Gram.
* Convergence (Alg. 1, Sec. 3.2 stopping rule): a submodel stops when
  |e_prev - e| / ||T_g||^2 < tol; tol = 0 means a fixed sweep count.

Parity status: every function here is pinned by ``tests/test_oracle_pins.py``
(brute force, closed forms, invariants, finite differences); the factor values
of the full configurations have no printed worked example in the paper and
are pinned only through those properties.
"""
from __future__ import annotations

import itertools
from dataclasses import dataclass, field
from typing import List, Optional, Sequence

import numpy as np
from scipy.linalg import solve_triangular

__all__ = [
    "unfold", "kolda_column", "khatri_rao", "krp_except", "mttkrp", "mttkrp_bruteforce",
    "gram", "hadamard_of_grams", "solve_normal_equations", "cp_reconstruct",
    "cp_loss_explicit", "cp_loss_efficient", "cp_als", "CPALSResult",
    "slice_tensor", "remove_rows", "insert_zero_rows", "jk_als", "JKResult",
    "concurrent_mttkrp_padded", "cp_loss_grad", "jk_loss_grad",
    "jackknife_se", "align_to_reference", "sign_fix", "flops_jk_als", "flops_jk_cals",
    "NotSPD",
]


class NotSPD(Exception):
    """Cholesky of the Hadamard-of-Grams matrix met a non-positive pivot."""


# ----------------------------------------------------------------------------
# Sec. 3.1 notation: unfolding, Khatri-Rao product, the "sum of all entries"
# ----------------------------------------------------------------------------

def kolda_column(idx: Sequence[int], dims: Sequence[int], n: int) -> int:
    """Column j (0-based) of T_(n) holding T(i_1..i_N), Eq. kolda_mapping (Sec. 4.1).

    j = sum_{k != n} i_k * prod_{m < k, m != n} I_m   (0-based form of the equation)
    """
    j, stride = 0, 1
    for k in range(len(dims)):
        if k == n:
            continue
        j += idx[k] * stride
        stride *= dims[k]
    return j


def unfold(T: np.ndarray, n: int) -> np.ndarray:
    """Mode-n unfolding T_(n) (Sec. 3.1): columns are the mode-n fibres, ordered
    by Eq. kolda_mapping (lowest remaining mode index varies fastest)."""
    I_n = T.shape[n]
    return np.reshape(np.moveaxis(T, n, 0), (I_n, -1), order="F")


def khatri_rao(A: np.ndarray, B: np.ndarray) -> np.ndarray:
    """A (.) B: column-wise Kronecker product (Sec. 3.1); row (a*I_B + b) = A[a] * B[b]."""
    assert A.shape[1] == B.shape[1]
    IA, IB = A.shape[0], B.shape[0]
    out = np.empty((IA * IB, A.shape[1]))
    for a in range(IA):
        out[a * IB:(a + 1) * IB, :] = A[a][None, :] * B
    return out


def krp_except(U: Sequence[np.ndarray], n: int) -> np.ndarray:
    """U_N (.) ... (.) U_{n+1} (.) U_{n-1} (.) ... (.) U_1, the order of Eq. MTTKRP
    (Sec. 4.1), so that U_1's row index varies fastest, matching kolda_mapping."""
    order = [k for k in reversed(range(len(U))) if k != n]
    out = U[order[0]]
    for k in order[1:]:
        out = khatri_rao(out, U[k])
    return out


def mttkrp(T: np.ndarray, U: Sequence[np.ndarray], n: int) -> np.ndarray:
    """M_n = T_(n) (U_N (.) ... (.) U_1 without U_n): Alg. 1 MTTKRP line, Eq. MTTKRP."""
    return unfold(T, n) @ krp_except(U, n)


def mttkrp_bruteforce(T: np.ndarray, U: Sequence[np.ndarray], n: int) -> np.ndarray:
    """Layout-free element loop: M(i_n, r) = sum_{all i} T(i) prod_{k != n} U_k(i_k, r).

    Pure Python; tiny tensors only."""
    R = U[0].shape[1]
    M = np.zeros((T.shape[n], R))
    for idx in itertools.product(*[range(I) for I in T.shape]):
        t = T[idx]
        for r in range(R):
            p = t
            for k in range(T.ndim):
                if k != n:
                    p *= U[k][idx[k], r]
            M[idx[n], r] += p
    return M


def gram(U: np.ndarray) -> np.ndarray:
    return U.T @ U


def hadamard_of_grams(U: Sequence[np.ndarray], n: int) -> np.ndarray:
    """H_n = *_{i != n} U_i^T U_i (Alg. 1 Hadamard line)."""
    R = U[0].shape[1]
    H = np.ones((R, R))
    for k, Uk in enumerate(U):
        if k != n:
            H = H * gram(Uk)
    return H


def solve_normal_equations(M: np.ndarray, H: np.ndarray) -> np.ndarray:
    """U = M H^{-1} via Cholesky H = L L^T (Alg. 1 update line, read as a solve).

    Raises NotSPD when a pivot is not positive."""
    try:
        L = np.linalg.cholesky(H)
    except np.linalg.LinAlgError as e:  # pragma: no cover - exercised via tests
        raise NotSPD(str(e))
    if not np.all(np.isfinite(L)) or np.any(np.diag(L) <= 0):
        raise NotSPD("non-positive pivot")
    # U H = M  <=>  H U^T = M^T  <=>  L (L^T U^T) = M^T
    Y = solve_triangular(L, M.T, lower=True)
    X = solve_triangular(L.T, Y, lower=False)
    return X.T


def cp_reconstruct(U: Sequence[np.ndarray]) -> np.ndarray:
    """[[U_1, ..., U_N]] = sum_r u_1r o ... o u_Nr, built column by column."""
    dims = [u.shape[0] for u in U]
    R = U[0].shape[1]
    out = np.zeros(dims)
    for r in range(R):
        t = U[0][:, r]
        for k in range(1, len(U)):
            t = np.multiply.outer(t, U[k][:, r])
        out += t
    return out


def cp_loss_explicit(T: np.ndarray, U: Sequence[np.ndarray]) -> float:
    d = T - cp_reconstruct(U)
    return float(np.sum(d * d))


def cp_loss_efficient(normT2: float, H_N: np.ndarray, U_N: np.ndarray, M_N: np.ndarray) -> float:
    """e = ||T||^2 + sum(H_N * U_N^T U_N) - 2 sum(U_N * M_N) (Alg. 1 error line,
    Phan et al.; sign of the middle term read as '+', see module docstring)."""
    return float(normT2 + np.sum(H_N * gram(U_N)) - 2.0 * np.sum(U_N * M_N))


# ----------------------------------------------------------------------------
# Alg. 1: CP-ALS
# ----------------------------------------------------------------------------

@dataclass
class CPALSResult:
    factors: List[np.ndarray]
    losses: List[float]                      # efficient formula after each sweep
    explicit_losses: List[float] = field(default_factory=list)
    mode_losses: List[float] = field(default_factory=list)  # explicit, after every mode update
    sweeps_done: int = 0
    not_spd: bool = False
    converged: bool = False


def cp_als(T: np.ndarray, U0: Sequence[np.ndarray], sweeps: int, *, normalise: bool = True,
           tol: float = 0.0, record_explicit: bool = False, record_modes: bool = False,
           unfoldings: Optional[List[np.ndarray]] = None) -> CPALSResult:
    """Alg. 1 (CP-ALS) for a fixed number of sweeps (or until the tolerance test).

    One sweep = for n = 1..N: MTTKRP, Hadamard of Grams, solve; then the error.
    """
    N = T.ndim
    U = [np.array(u, dtype=np.float64, copy=True) for u in U0]
    Tn = unfoldings if unfoldings is not None else [unfold(T, n) for n in range(N)]
    normT2 = float(np.sum(T * T))
    res = CPALSResult(factors=U, losses=[])
    e_prev = None
    for s in range(sweeps):
        M = None
        H = None
        for n in range(N):
            M = Tn[n] @ krp_except(U, n)
            H = hadamard_of_grams(U, n)
            try:
                Un = solve_normal_equations(M, H)
            except NotSPD:
                res.not_spd = True
                res.sweeps_done = s
                return res
            if normalise and n < N - 1:
                nrm = np.sqrt(np.sum(Un * Un, axis=0))
                nrm[nrm == 0] = 1.0
                Un = Un / nrm[None, :]
            U[n] = Un
            if record_modes:
                res.mode_losses.append(cp_loss_explicit(T, U))
        e = cp_loss_efficient(normT2, H, U[N - 1], M)
        res.losses.append(e)
        if record_explicit:
            res.explicit_losses.append(cp_loss_explicit(T, U))
        res.sweeps_done = s + 1
        if tol > 0 and e_prev is not None and abs(e_prev - e) / normT2 < tol:
            res.converged = True
            break
        e_prev = e
    return res


# ----------------------------------------------------------------------------
# Alg. 2: JK-ALS (straightforward jackknife), the reference workflow
# ----------------------------------------------------------------------------

def slice_tensor(T: np.ndarray, n_hat: int, D: Sequence[int]) -> np.ndarray:
    """T_{-p}: remove the slices with indices D from mode n_hat (Alg. 2 line 1 of the loop)."""
    keep = np.setdiff1d(np.arange(T.shape[n_hat]), np.asarray(D, dtype=np.int64))
    return np.take(T, keep, axis=n_hat)


def remove_rows(U: np.ndarray, D: Sequence[int]) -> np.ndarray:
    """P_{-p}: remove rows D from a factor matrix (Alg. 2, second loop line)."""
    keep = np.setdiff1d(np.arange(U.shape[0]), np.asarray(D, dtype=np.int64))
    return U[keep]


def insert_zero_rows(U_red: np.ndarray, I: int, D: Sequence[int]) -> np.ndarray:
    """Inverse of remove_rows with zeros at D (Alg. 3 initialisation, red branch)."""
    keep = np.setdiff1d(np.arange(I), np.asarray(D, dtype=np.int64))
    out = np.zeros((I, U_red.shape[1]))
    out[keep] = U_red
    return out


@dataclass
class JKResult:
    """Per-submodel results, factors re-expanded to full rows (zeros at D_g in mode n_hat)."""
    factors: List[List[np.ndarray]]
    losses: np.ndarray            # sweeps x K (efficient formula), NaN after a stop
    sweeps_done: List[int]
    not_spd: List[bool]
    normT2: np.ndarray            # ||T_{-g}||^2 per block
    explicit_losses: Optional[np.ndarray] = None


def jk_als(T: np.ndarray, n_hat: int, left_out: Sequence[Sequence[int]],
           init: Sequence[Sequence[np.ndarray]], sweeps: int, *, normalise: bool = True,
           tol: float = 0.0, blocks: Optional[Sequence[int]] = None,
           record_explicit: bool = False) -> JKResult:
    """Alg. 2 without the alignment/std lines: every block fitted on its own sliced tensor.

    init[g][n] is I_n x R_g with all rows; rows D_g of mode n_hat are removed
    before fitting (Alg. 2, model sub-sampling line).  ``blocks`` restricts the
    fit to a subset of block indices (each block is independent)."""
    K = len(left_out)
    sel = list(range(K)) if blocks is None else list(blocks)
    facs, sd, nspd, norms = [], [], [], []
    losses = np.full((sweeps, len(sel)), np.nan)
    expl = np.full((sweeps, len(sel)), np.nan) if record_explicit else None
    for col, g in enumerate(sel):
        D = np.asarray(left_out[g], dtype=np.int64)
        Tg = slice_tensor(T, n_hat, D)
        U0 = [remove_rows(u, D) if k == n_hat else u for k, u in enumerate(init[g])]
        r = cp_als(Tg, U0, sweeps, normalise=normalise, tol=tol, record_explicit=record_explicit)
        full = [insert_zero_rows(u, T.shape[k], D) if k == n_hat else u
                for k, u in enumerate(r.factors)]
        facs.append(full)
        losses[:len(r.losses), col] = r.losses
        if record_explicit:
            expl[:len(r.explicit_losses), col] = r.explicit_losses
        sd.append(r.sweeps_done)
        nspd.append(r.not_spd)
        norms.append(float(np.sum(Tg * Tg)))
    return JKResult(factors=facs, losses=losses, sweeps_done=sd, not_spd=nspd,
                    normT2=np.array(norms), explicit_losses=expl)


def concurrent_mttkrp_padded(T: np.ndarray, Ubar: Sequence[np.ndarray], n: int) -> np.ndarray:
    """Alg. 3 MTTKRP line on the *full* tensor with multi-matrices whose blocks
    carry zero rows at D_g in the sampled mode (Sec. 4.1, Case II).  Used only to
    pin the paper's Case I/II identities inside the oracle."""
    return mttkrp(T, Ubar, n)


# ----------------------------------------------------------------------------
# Loss and gradient of the summed reconstruction error (gradient-based CP)
# ----------------------------------------------------------------------------

def cp_loss_grad(T: np.ndarray, U: Sequence[np.ndarray]):
    """f = ||T - [[U]]||^2 and df/dU_n = 2 (U_n H_n - M_n)."""
    N = T.ndim
    f = cp_loss_explicit(T, U)
    grads = [2.0 * (U[n] @ hadamard_of_grams(U, n) - mttkrp(T, U, n)) for n in range(N)]
    return f, grads


def jk_loss_grad(T: np.ndarray, n_hat: int, left_out, ranks, Ubar: Sequence[np.ndarray]):
    """Sum over blocks g of ||T_{-g} - [[U^(g)]]||^2 and its gradient w.r.t. the
    multi-matrices Ubar (I_n x sum R_g).  Block g uses columns [off_g, off_g+R_g)
    and, in mode n_hat, only the rows outside D_g; the gradient at rows D_g of
    mode n_hat is zero (those entries do not enter block g's model)."""
    N = T.ndim
    offs = np.concatenate([[0], np.cumsum(ranks)])
    total = 0.0
    G = [np.zeros_like(u) for u in Ubar]
    for g, D in enumerate(left_out):
        D = np.asarray(D, dtype=np.int64)
        cols = slice(offs[g], offs[g + 1])
        Tg = slice_tensor(T, n_hat, D)
        Ug = [remove_rows(Ubar[k][:, cols], D) if k == n_hat else Ubar[k][:, cols] for k in range(N)]
        f, grads = cp_loss_grad(Tg, Ug)
        total += f
        for k in range(N):
            gk = insert_zero_rows(grads[k], T.shape[k], D) if k == n_hat else grads[k]
            G[k][:, cols] += gk
    return total, G


# ----------------------------------------------------------------------------
# Alg. 2 post-processing: permutation/scale adjustment and the jackknife std
# ----------------------------------------------------------------------------

def sign_fix(U: Sequence[np.ndarray], last: int) -> List[np.ndarray]:
    """Make the largest-|.| entry of every column positive in all modes but
    ``last``; the flips are compensated in mode ``last`` so the model is unchanged."""
    U = [u.copy() for u in U]
    for k in range(len(U)):
        if k == last:
            continue
        for r in range(U[k].shape[1]):
            col = U[k][:, r]
            if col.size == 0:
                continue
            i = int(np.argmax(np.abs(col)))
            if col[i] < 0:
                U[k][:, r] = -col
                U[last][:, r] = -U[last][:, r]
    return U


def align_to_reference(U_sub: Sequence[np.ndarray], U_ref: Sequence[np.ndarray], n_hat: int,
                       return_perm: bool = False):
    """Permutation and scale adjustment of a submodel against the overall model
    (Alg. 2 adjustment line, method of Riu & Bro).  Reading: columns of modes
    other than the last are unit-norm (normalisation above) with the sign rule
    of ``sign_fix``; the permutation maximises sum_r prod_{n != n_hat}
    |cos(U_n^sub(:, r), U_n^ref(:, pi r))|, brute force for R <= 8, ties to the
    lexicographically smallest permutation.  Returns the permuted factors (and,
    with ``return_perm``, perm: reference column s <- submodel column perm[s])."""
    N = len(U_sub)
    R = U_sub[0].shape[1]
    A = sign_fix(U_sub, N - 1)
    B = sign_fix(U_ref, N - 1)
    score = np.ones((R, R))
    for k in range(N):
        if k == n_hat:
            continue
        a = A[k] / np.maximum(np.linalg.norm(A[k], axis=0), 1e-300)[None, :]
        b = B[k] / np.maximum(np.linalg.norm(B[k], axis=0), 1e-300)[None, :]
        score = score * np.abs(a.T @ b)   # score[r, s] = |cos(sub r, ref s)|
    if R <= 8:
        best, best_p = -1.0, None
        for p in itertools.permutations(range(R)):
            s = sum(score[p[s_], s_] for s_ in range(R))
            if s > best + 1e-15:
                best, best_p = s, p
        perm = best_p    # ref column s_ <- sub column perm[s_]
    else:
        from scipy.optimize import linear_sum_assignment
        rows, cols = linear_sum_assignment(-score)
        perm = [0] * R
        for r_, s_ in zip(rows, cols):
            perm[s_] = r_
    out = [a[:, list(perm)] for a in A]
    return (out, list(perm)) if return_perm else out


def jackknife_se(estimates: np.ndarray) -> np.ndarray:
    """Jackknife standard error over the leading axis (G submodels or groups):
    S = sqrt((G-1)/G * sum_g (theta_g - mean)^2)  (Alg. 2 std line, read as the
    delete-one / delete-a-group jackknife SE)."""
    G = estimates.shape[0]
    mean = estimates.mean(axis=0)
    return np.sqrt((G - 1.0) / G * np.sum((estimates - mean) ** 2, axis=0))


# ----------------------------------------------------------------------------
# Sec. 4.2 operation counts
# ----------------------------------------------------------------------------

def flops_jk_als(dims: Sequence[int], n_hat: int, d: int, R: int) -> int:
    """MTTKRP flops of JK-ALS for one mode, all I/d submodels: (I/d) 2R (I-d) prod_{i!=n_hat} I_i."""
    I = dims[n_hat]
    other = int(np.prod([x for k, x in enumerate(dims) if k != n_hat]))
    return (I // d) * 2 * R * (I - d) * other


def flops_jk_cals(dims: Sequence[int], n_hat: int, d: int, R: int) -> int:
    """Fused MTTKRP flops of JK-CALS for one mode: 2 (I/d) R prod_i I_i."""
    I = dims[n_hat]
    return 2 * (I // d) * R * int(np.prod(dims))
