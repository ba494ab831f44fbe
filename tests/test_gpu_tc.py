"""GPU parity of the tensor-core (tcgen05) forms of the concurrent MTTKRP.

The reduced-precision forms accumulate in FP32 in TMEM; their error against the
FP64 oracle grows with the length of the accumulation chain (each split-K
chain of ~J/S terms), so the bounds below are per shape class.  bench.py
reports them; none of these forms is "at parity".
"""
import numpy as np
import pytest

import oracle as O
from paper_2112_03985_gb300 import api, workloads as W

from _helpers import (assert_elementwise, assert_factors, compare_mttkrp, offsets, se_perturbation_bound,
                      stepwise_loss_check)

pytestmark = pytest.mark.gpu

# relative Frobenius error per block per mode, small shapes (chains of <= ~1200 terms)
SMALL_RTOL = {"3xtf32": 1e-5, "split_bf16": 1e-5, "tf32": 2e-3, "bf16": 1e-2}
# configuration 2 (chains of ~2500 terms)
CFG2_RTOL = {"3xtf32": 1e-4, "split_bf16": 1e-4, "tf32": 1e-3, "bf16": 1e-3}


def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _w(dims, R, n_hat=0, seed=0, ranks=None, d=1):
    I = dims[n_hat]
    blocks = W.group_blocks(I, d) if d > 1 else W.loo_blocks(I, include_full=True)
    return W.make_workload("t", dims, R, n_hat=n_hat, blocks=blocks, noise=0.01, seed=seed, ranks=ranks)


SHAPES = [
    ("cfg1 20x30x40 R3", lambda: W.make_config(1)),
    ("ragged 129x17x33 R4 (C=520)", lambda: _w((129, 17, 33), 4, seed=1)),
    ("1-row mode 5x1x7", lambda: _w((5, 1, 7), 2, seed=2)),
    ("4-way n_hat=2", lambda: _w((6, 5, 4, 3), 3, n_hat=2, seed=3)),
    ("two N tiles 300x9x7 R2", lambda: _w((300, 9, 7), 2, seed=4)),
    ("delete-3 mixed ranks 12x21x10", lambda: _w((12, 21, 10), 2, d=3, seed=5, ranks=[1, 5, 2, 7])),
]


@pytest.mark.parametrize("prec", ["3xtf32", "split_bf16", "tf32", "bf16"])
@pytest.mark.parametrize("name,make", SHAPES, ids=[s[0] for s in SHAPES])
def test_tc_mttkrp_matches_each_submodel(prec, name, make):
    _cuda()
    w = make()
    with api.from_workload(w, precision=prec) as h:
        U = h.get_factors()
        for n in range(w.T.ndim):
            compare_mttkrp(w, h.mttkrp(n), U, n, SMALL_RTOL[prec])


@pytest.mark.parametrize("prec", ["3xtf32", "split_bf16", "tf32", "bf16"])
def test_tc_mttkrp_cfg2_full_size_sampled_blocks(prec):
    _cuda()
    w = W.make_config(2)
    with api.from_workload(w, precision=prec) as h:
        U = h.get_factors()
        for n in range(3):
            compare_mttkrp(w, h.mttkrp(n), U, n, CFG2_RTOL[prec], blocks=[0, 77, 299])


def test_tc_is_deterministic_and_zero_rows_stay_zero():
    _cuda()
    w = _w((40, 33, 65), 3, seed=6)
    res = []
    for _ in range(2):
        with api.from_workload(w, precision="3xtf32") as h:
            l = h.als_sweep(5)
            res.append((l, h.get_factors()))
    np.testing.assert_array_equal(res[0][0], res[1][0])
    offs = offsets(w.ranks)
    for a, b in zip(res[0][1], res[1][1]):
        np.testing.assert_array_equal(a, b)
    for g, D in enumerate(w.left_out):
        assert np.all(res[0][1][0][D, offs[g]:offs[g + 1]] == 0)


def test_tc_als_tracks_oracle_on_cfg1():
    """3xTF32 ALS against the FP64 oracle (configuration 1, 50 sweeps): factors
    within 1e-4 element by element, and the loss after every sweep within the
    bound derived from the form's MTTKRP bar (1e-5) and the distance between the
    two models; a reported bound, not a parity claim."""
    _cuda()
    w = W.make_config(1)
    sel = [0, 7, 20]
    with api.from_workload(w, precision="3xtf32") as h:
        _, _, ratio, facs = stepwise_loss_check(w, h, sel, w.sweeps, SMALL_RTOL["3xtf32"])
        U = h.get_factors()
    errs = assert_factors(w, U, facs, sel, 1e-4)
    print(f"\ncfg1 3xtf32: factor rel err {errs.max():.2e}; loss error at most {ratio:.2f} of its bound")


def test_tc_gradient_matches_oracle():
    _cuda()
    rng = np.random.default_rng(16)
    w = _w((10, 8, 8, 6), 2, seed=16)
    U = [rng.standard_normal((I, w.C)) for I in w.T.shape]
    with api.from_workload(w, precision="3xtf32") as h:
        f, G = h.grad(U)
    offs = offsets(w.ranks)
    for g, D in enumerate(w.left_out):
        U[0][D, offs[g]:offs[g + 1]] = 0.0
    f_ref, G_ref = O.jk_loss_grad(w.T, 0, w.left_out, w.ranks, U)
    assert abs(f - f_ref) <= 1e-5 * abs(f_ref)
    for n in range(4):
        err = np.linalg.norm(G[n] - G_ref[n]) / np.linalg.norm(G_ref[n])
        assert err <= 1e-4, (n, err)


def test_jackknife_se_error_per_form_cfg2():
    """Configuration 2, 100 sweeps: factor and jackknife standard-error (Alg. 2
    std line, modes != n_hat) errors of every precision form against the FP64
    path (itself matched to the oracle on sampled blocks).  Each submodel is
    aligned (Alg. 2 adjustment line) to submodel 0 of the FP64 run.

    Bars: the exact-chain form's factors within 1e-6 of FP64, element by element.
    The standard errors are held, entry by entry, to the bound that the factor
    differences themselves imply: SE(x) = sqrt((G-1)/G) ||x - mean(x)|| is a norm
    over the G submodels, so |SE(a) - SE(b)| <= SE(a - b) (reverse triangle
    inequality); an SE therefore moves by up to the jackknife SE of the aligned
    factor differences, i.e. by about sqrt(G) times the per-submodel factor error
    when those errors do not share a sign, which is why the relative SE error of a
    form exceeds its relative factor error.  The per-form figures are printed."""
    _cuda()
    w = W.make_config(2)
    offs = offsets(w.ranks)

    def fit(prec):
        with api.from_workload(w, precision=prec, device="cuda") as h:
            h.als_sweep(w.sweeps)
            return h.get_factors()

    def estimates(U, ref):
        est = []
        for g in range(w.K):
            Ug = [u[:, offs[g]:offs[g + 1]] for u in U]
            A = O.align_to_reference(Ug, ref, w.n_hat)
            est.append(np.concatenate([A[k].ravel() for k in range(3) if k != w.n_hat]))
        return np.asarray(est)

    U64 = fit("fp64")
    ref = [u[:, offs[0]:offs[1]] for u in U64]
    est64 = estimates(U64, ref)
    se64 = O.jackknife_se(est64)
    report = {}
    for prec in ("exact_bf16", "3xtf32", "split_bf16", "tf32", "bf16"):
        U = fit(prec)
        ferr = max(float(np.abs(a - b).max() / np.abs(b).max()) for a, b in zip(U, U64))
        est = estimates(U, ref)
        se = O.jackknife_se(est)
        bound = se_perturbation_bound(est, est64)
        serr = float(np.abs(se - se64).max() / np.abs(se64).max())
        report[prec] = (ferr, serr, float(bound.max() / np.abs(se64).max()))
        # reverse triangle inequality (up to rounding of the two SE evaluations)
        assert np.all(np.abs(se - se64) <= bound + 1e-13 * np.abs(se64).max()), prec
        if prec == "exact_bf16":
            for a, b in zip(U, U64):
                assert_elementwise(a, b, 1e-6, "exact form factors vs FP64")
            # with the same alignment per submodel, every aligned difference is at
            # most 2e-6 max|U_n| by the factor bar, so SE(diff) <= sqrt(G - 1) 2e-6 max|U_n|
            G = w.K
            col = 0
            for k in range(3):
                if k == w.n_hat:
                    continue
                m = w.dims[k] * w.ranks[0]
                lim = np.sqrt(G - 1.0) * 2e-6 * np.abs(est64[:, col:col + m]).max()
                assert np.all(np.abs(se - se64)[col:col + m] <= lim), (k, np.abs(se - se64)[col:col + m].max(), lim)
                col += m
    print("\ncfg2 100 sweeps, vs FP64 (max relative): " + ", ".join(
        f"{p}: factors {f:.1e} SE {s:.1e} (bound {b:.1e})" for p, (f, s, b) in report.items()))
    for p, (f, s, b) in report.items():
        assert np.isfinite(f) and np.isfinite(s)
