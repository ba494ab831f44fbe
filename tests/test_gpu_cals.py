"""GPU parity of plain concurrent ALS (Sec. 3.3, CALS): K models of one tensor, each with its
own initial factors and rank, no left-out rows, advanced together through one MTTKRP per mode.
Each model must follow its own CP-ALS run (Alg. 1) in the oracle.  Also the MTTKRP of the
50x200x200 rank-sweep tensor (Sec. 3.2 figure) at the smallest column counts, every form.
"""
import numpy as np
import pytest

import oracle as O
from paper_2112_03985_gb300 import api, workloads as W

from _helpers import assert_elementwise, assert_factors, offsets, stepwise_loss_check

pytestmark = pytest.mark.gpu

# element-wise bars: MTTKRP, factors; FP64 losses within 1e-12 ||T||^2, the exact
# form's within the bound derived from its MTTKRP bar (tests/_helpers.loss_bound)
FORMS = {"fp64": (1e-12, 1e-10), "exact_bf16": (1e-8, 1e-6)}
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
    mtol, ftol = FORMS[prec]
    normT2 = float(np.sum(w.T * w.T))
    with api.JKCALS(w.T, 0, ranks, w.left_out, api.multi_init(inits), precision=prec) as h:
        if prec == "fp64":
            losses = h.als_sweep(sweeps)
            refs = [O.cp_als(w.T, inits[k], sweeps) for k in range(len(ranks))]
            facs = [r.factors for r in refs]
            for k, r in enumerate(refs):
                assert np.all(np.abs(losses[:, k] - np.asarray(r.losses)) <= 1e-12 * normT2), (prec, k)
        else:
            _, _, ratio, facs = stepwise_loss_check(w, h, list(range(len(ranks))), sweeps, mtol, inits=inits)
            print(f"\nCALS {dims} {prec}: loss error at most {ratio:.2f} of its bound")
        U = h.get_factors()
    assert_factors(w, U, facs, list(range(len(ranks))), ftol)


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
            assert_elementwise(h.mttkrp(n), O.mttkrp(w.T, U, n), rtol, f"{prec} C={C} mode {n}")
