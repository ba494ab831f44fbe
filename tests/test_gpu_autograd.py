"""Configuration 5: the differentiable summed jackknife loss (torch.autograd.Function
with the hand-written concurrent-MTTKRP backward).

* FD instance 10x8x8x6, R = 2, all 10 LOO submodels, FP64 path: the autograd
  gradient against FP64 central differences of the same loss (directional
  derivatives), and against the oracle's analytic gradient.
* Full size 100x60x60x40, rank 8, 100 LOO submodels: the autograd gradient of
  sampled submodels against the oracle's analytic gradient of those submodels
  alone (block g's gradient depends on block g's columns only), FP64 and the
  exact-chain form.
* A gradient-based fit (L-BFGS on the autograd loss) beside ALS from the same
  initial factors and for the same wall time: both lower the loss.
"""
import time

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
    return torch


def _fd_instance():
    return W.make_workload("fd 10x8x8x6 R2", (10, 8, 8, 6), 2, n_hat=0, blocks=W.loo_blocks(10),
                           noise=0.01, seed=5100, sweeps=1, factor_kind="normal", init_kind="normal")


def test_autograd_matches_central_differences_and_oracle():
    torch = _cuda()
    w = _fd_instance()
    rng = np.random.default_rng(5101)
    U0 = [rng.standard_normal((I, w.C)) for I in w.T.shape]
    with api.from_workload(w, device="cuda") as h:
        U = [torch.tensor(u, device="cuda", requires_grad=True) for u in U0]
        f = h.loss(U)
        f.backward()
        G = [u.grad.cpu().numpy() for u in U]
        # central differences of the same loss along random directions
        for k in range(4):
            V = [rng.standard_normal(u.shape) for u in U0]
            eps = 1e-5
            with torch.no_grad():
                up = h.loss([torch.tensor(u + eps * v, device="cuda") for u, v in zip(U0, V)]).item()
                dn = h.loss([torch.tensor(u - eps * v, device="cuda") for u, v in zip(U0, V)]).item()
            fd = (up - dn) / (2 * eps)
            an = sum(float(np.sum(g * v)) for g, v in zip(G, V))
            assert abs(fd - an) <= 1e-6 * max(abs(an), 1.0), (k, fd, an)
    # the oracle sees the sampled mode with rows D_g zeroed per block
    Uz = [u.copy() for u in U0]
    offs = offsets(w.ranks)
    for g, D in enumerate(w.left_out):
        Uz[0][D, offs[g]:offs[g + 1]] = 0.0
    f_ref, G_ref = O.jk_loss_grad(w.T, 0, w.left_out, w.ranks, Uz)
    assert abs(f.item() - f_ref) <= 1e-10 * abs(f_ref)
    for n in range(4):
        np.testing.assert_allclose(G[n], G_ref[n], rtol=1e-9, atol=1e-10 * np.abs(G_ref[n]).max())


@pytest.mark.parametrize("precision,rtol", [("fp64", 1e-9), ("exact_bf16", 1e-6)])
def test_autograd_cfg5_sampled_blocks_full_size(precision, rtol):
    torch = _cuda()
    w = W.make_config(5)
    rng = np.random.default_rng(5102)
    U0 = [rng.standard_normal((I, w.C)) for I in w.T.shape]
    with api.from_workload(w, precision=precision, device="cuda") as h:
        U = [torch.tensor(u, device="cuda", requires_grad=True) for u in U0]
        f = h.loss(U)
        f.backward()
        G = [u.grad.cpu().numpy() for u in U]
    offs = offsets(w.ranks)
    for g in (0, 57, 99):
        cols = slice(offs[g], offs[g + 1])
        Ug = [u[:, cols].copy() for u in U0]
        Ug[0][w.left_out[g], :] = 0.0
        _, Gg = O.jk_loss_grad(w.T, 0, [w.left_out[g]], [w.ranks[g]], Ug)
        for n in range(4):
            ref = Gg[n]
            err = np.abs(G[n][:, cols] - ref).max() / np.abs(ref).max()
            assert err <= rtol, (precision, g, n, err)
    assert np.isfinite(f.item()) and f.item() > 0


def test_gradient_fit_beside_als_equal_wall_time():
    """L-BFGS on the autograd loss and ALS sweeps, same initial factors and wall
    time (exact-chain form): both lower the summed loss."""
    torch = _cuda()
    w = W.make_config(5)
    with api.from_workload(w, precision="exact_bf16", device="cuda") as h:
        U = [u.clone().requires_grad_(True) for u in h.get_factors(device="cuda")]
        with torch.no_grad():
            f0 = h.loss(U).item()
        t0 = time.perf_counter()
        losses = h.als_sweep(10)
        t_als = time.perf_counter() - t0
        f_als = float(np.nansum(losses[-1]))
        opt = torch.optim.LBFGS(U, lr=1.0, max_iter=5, history_size=10, line_search_fn="strong_wolfe")

        def closure():
            opt.zero_grad()
            f = h.loss(U)
            f.backward()
            return f

        t0 = time.perf_counter()
        while time.perf_counter() - t0 < t_als:
            opt.step(closure)
        with torch.no_grad():
            f_grad = h.loss(U).item()
    print(f"\ncfg5 equal wall time {t_als * 1e3:.1f} ms: start {f0:.6e}, ALS {f_als:.6e}, L-BFGS {f_grad:.6e}")
    assert f_als < f0 and f_grad < f0
