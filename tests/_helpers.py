"""Shared test helpers: oracle-side references and comparisons (no library code)."""
import numpy as np

import oracle as O


def offsets(ranks):
    return np.concatenate([[0], np.cumsum(ranks)]).astype(int)


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
    """Per-block relative Frobenius error of the concurrent MTTKRP against each
    submodel's own MTTKRP (Case I rows D_g dropped).  Returns the max error."""
    offs = offsets(w.ranks)
    worst = 0.0
    for g in (range(w.K) if blocks is None else blocks):
        ref = oracle_block_mttkrp(w, U_multi, n, g)
        got = M_gpu[:, offs[g]:offs[g + 1]]
        if n == w.n_hat:
            got = O.remove_rows(got, w.left_out[g])
        err = np.linalg.norm(got - ref) / max(np.linalg.norm(ref), 1e-300)
        worst = max(worst, err)
        assert err <= rtol, f"mode {n} block {g}: rel err {err:.3e} > {rtol:.1e}"
    return worst


def factor_errors(w, U_gpu, ora, blocks):
    """Relative Frobenius error per (block, mode) of the GPU factors against the
    oracle's re-expanded per-submodel factors."""
    offs = offsets(w.ranks)
    errs = np.zeros((len(blocks), w.T.ndim))
    for col, g in enumerate(blocks):
        for n in range(w.T.ndim):
            ref = ora.factors[col][n]
            got = U_gpu[n][:, offs[g]:offs[g + 1]]
            errs[col, n] = np.linalg.norm(got - ref) / max(np.linalg.norm(ref), 1e-300)
    return errs
