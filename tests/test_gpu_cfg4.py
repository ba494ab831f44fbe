"""Configuration 4: a batch of independent LOO jackknife problems of uneven
sizes and ranks (I1 in [20, 400], I2, I3 in [30, 150], R in [2, 8], FP32),
advanced together by one CUDA graph per sweep (jkcals_batch_*): grouped
launches over all problems when they share a one-step tensor-core form, else
(or with opt.batch_branches) one graph branch per problem; the split factors
picked by the autotuner (opt.autotune)."""
import numpy as np
import pytest

import oracle as O
from paper_2112_03985_gb300 import api, workloads as W

from _helpers import assert_factors

pytestmark = pytest.mark.gpu


def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


@pytest.fixture(scope="module")
def problems():
    return W.make_config4_batch(64)


def _handles(ws, **kw):
    return [api.from_workload(w, device="cuda", **kw) for w in ws]


@pytest.mark.parametrize("precision,branches", [("3xtf32", False), ("3xtf32", True), ("exact_bf16", False)])
def test_batched_sweeps_equal_individual_sweeps(problems, precision, branches):
    """Both batch forms (grouped launches; per-problem branches, which the
    exact-chain form's two-step modes also take) compute each problem's sweep
    bit for bit as its own handle does."""
    _cuda()
    ws = problems[:8]
    hs_a = _handles(ws, precision=precision)
    hs_b = _handles(ws, precision=precision, batch_branches=branches)
    try:
        ref = [(h.als_sweep(5), h.get_factors()) for h in hs_a]
        with api.Batch(hs_b, max_sweeps=5) as b:
            b.sweep(5)
            b.sync()
            got = [(h.loss_history(5), h.get_factors()) for h in hs_b]
        for (la, Ua), (lb, Ub) in zip(ref, got):
            np.testing.assert_array_equal(la, lb)
            for x, y in zip(Ua, Ub):
                np.testing.assert_array_equal(x, y)
    finally:
        for h in hs_a + hs_b:
            h.close()


def test_batched_fp64_matches_oracle_on_sampled_problems(problems):
    _cuda()
    picks = [3, 41]
    ws = [problems[i] for i in picks]
    sweeps = 5
    hs = _handles(problems[:48:6] + ws, precision="fp64")   # the sampled problems among others
    try:
        with api.Batch(hs, max_sweeps=sweeps) as b:
            b.sweep(sweeps)
            b.sync()
        for w, h in zip(ws, hs[-2:]):
            losses = h.loss_history(sweeps)
            U = h.get_factors()
            blocks = [0, w.K - 1]
            ora = O.jk_als(w.T, w.n_hat, w.left_out, w.init, sweeps, blocks=blocks)
            errs = assert_factors(w, U, ora.factors, blocks, 1e-10)
            lrel = np.abs(losses[:, blocks] - ora.losses) / np.abs(ora.losses)
            assert errs.max() <= 1e-10, errs.max()
            assert lrel.max() <= 1e-10, lrel.max()
    finally:
        for h in hs:
            h.close()


def test_all_64_problems_3xtf32_autotuned(problems):
    """The full batch, 3xTF32 MTTKRP with autotuned split factors, 50 sweeps;
    factor errors against the FP64 path of the same problems are reported and
    bounded by the form's accuracy."""
    _cuda()
    sweeps = 50
    hs = _handles(problems, precision="3xtf32", autotune=True)
    try:
        with api.Batch(hs, max_sweeps=sweeps) as b:
            b.sweep(sweeps)
            b.sync()
        worst = 0.0
        for i in (0, 17, 63):
            w = problems[i]
            with api.from_workload(w, device="cuda", precision="fp64") as hf:
                hf.als_sweep(sweeps)
                Uf = hf.get_factors()
            U = hs[i].get_factors()
            assert np.all(hs[i].block_status() == 0)
            for a, c in zip(U, Uf):
                worst = max(worst, float(np.abs(a - c).max() / np.abs(c).max()))
            _, splits = hs[i].sweep_info()
            assert all(s >= 1 for s in splits)
        print(f"\ncfg4 3xTF32 batched vs FP64 after {sweeps} sweeps: factor rel err {worst:.2e}")
        assert worst < 1e-2
    finally:
        for h in hs:
            h.close()
