"""GPU parity of plain concurrent ALS (Sec. 3.3, CALS): K models of one tensor, each with its
own initial factors and rank, no left-out rows, advanced together through one MTTKRP per mode.
Each model must follow its own CP-ALS run (Alg. 1) in the oracle.  Also the MTTKRP of the
50x200x200 rank-sweep tensor (Sec. 3.2 figure) at the smallest column counts, every form.
"""
import numpy as np
import pytest

import oracle as O
from paper_2112_03985_gb300 import api, workloads as W

from _helpers import offsets

pytestmark = pytest.mark.gpu

# MTTKRP relative error, factor relative error, loss error relative to ||T||^2
FORMS = {"fp64": (1e-12, 1e-10, 1e-12), "exact_bf16": (1e-8, 1e-6, 1e-7)}
REDUCED = {"3xtf32": 1e-5, "split_bf16": 1e-5, "tf32": 2e-3, "bf16": 1e-2}


def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _cals(dims, ranks, seed):
    """Planted rank-3 tensor; models of the given ranks, each with its own U[0,1] init."""
    K = len(ranks)
    w = W.make_workload("cals", dims, 3, blocks=[np.zeros(0, dtype=np.int64)] * K, noise=0.01, seed=seed,
                        ranks=ranks)
    rng = np.random.default_rng(seed + 10)
    inits = [[rng.uniform(0.0, 1.0, size=(I, r)) for I in dims] for r in ranks]
    return w, inits


@pytest.mark.parametrize("prec", list(FORMS))
@pytest.mark.parametrize("dims", [(20, 30, 40), (9, 150, 30)], ids=["20x30x40", "9x150x30"])
def test_cals_models_follow_their_own_cp_als(prec, dims):
    """On 9x150x30 the exact form runs modes 0 and 2 on the two-step kernel."""
    _cuda()
    ranks = [2, 3, 5, 1, 4, 3]
    sweeps = 10
    w, inits = _cals(dims, ranks, seed=40)
    _, ftol, ltol = FORMS[prec]
    normT2 = float(np.sum(w.T * w.T))
    offs = offsets(ranks)
    with api.JKCALS(w.T, 0, ranks, w.left_out, api.multi_init(inits), precision=prec) as h:
        losses = h.als_sweep(sweeps)
        U = h.get_factors()
    for k, r in enumerate(ranks):
        ref = O.cp_als(w.T, inits[k], sweeps)
        for n in range(3):
            got = U[n][:, offs[k]:offs[k + 1]]
            err = np.linalg.norm(got - ref.factors[n]) / np.linalg.norm(ref.factors[n])
            assert err <= ftol, (prec, k, n, err)
        assert np.all(np.abs(losses[:, k] - np.asarray(ref.losses)) <= ltol * normT2), (prec, k)


@pytest.mark.parametrize("prec", list(FORMS) + list(REDUCED))
@pytest.mark.parametrize("C", [1, 2, 5])
def test_rank_sweep_tensor_mttkrp_few_columns(prec, C):
    """One model of C components on the 50x200x200 tensor: the narrowest tile shapes."""
    _cuda()
    w, inits = _cals((50, 200, 200), [C], seed=41)
    rtol = FORMS[prec][0] if prec in FORMS else REDUCED[prec]
    with api.JKCALS(w.T, 0, [C], w.left_out, api.multi_init(inits), precision=prec) as h:
        U = h.get_factors()
        for n in range(3):
            ref = O.mttkrp(w.T, U, n)
            got = h.mttkrp(n)
            err = np.linalg.norm(got - ref) / np.linalg.norm(ref)
            assert err <= rtol, (prec, C, n, err)
