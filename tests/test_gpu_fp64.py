"""GPU parity of the FP64 path against the FP64 oracle (through the C ABI).

Tolerances, element by element (|got - ref| <= bar (|ref| + max|ref|) per block
and mode): concurrent MTTKRP 1e-12; factors 1e-10 after the fixed sweep count;
losses 1e-10 relative, entry by entry.
"""
import numpy as np
import pytest

import oracle as O
from paper_2112_03985_gb300 import api, workloads as W

from _helpers import assert_factors, compare_mttkrp, offsets

pytestmark = pytest.mark.gpu

MTTKRP_RTOL = 1e-12
FACTOR_RTOL = 1e-10


def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def _ragged(dims, R, n_hat=0, d=1, full=True, ranks=None, seed=0, sweeps=5, noise=0.01):
    I = dims[n_hat]
    blocks = W.group_blocks(I, d) if d > 1 else W.loo_blocks(I, include_full=full)
    return W.make_workload("t", dims, R, n_hat=n_hat, blocks=blocks, noise=noise, seed=seed,
                           sweeps=sweeps, ranks=ranks)


MTTKRP_CASES = [
    ("cfg1", None),
    ("ragged 129x17x33 R4", _ragged((129, 17, 33), 4, seed=1)),
    ("tiny 1-row mode 5x1x7 R2", _ragged((5, 1, 7), 2, seed=2)),
    ("4-way 6x5x4x3 R3 n_hat=2", _ragged((6, 5, 4, 3), 3, n_hat=2, seed=3)),
    ("delete-3 12x9x8 R1", _ragged((12, 9, 8), 1, d=3, seed=4)),
    ("mixed ranks 9x20x11", _ragged((9, 20, 11), 3, ranks=[1, 2, 3, 4, 5, 6, 7, 8, 9, 32], seed=5)),
]


@pytest.mark.parametrize("name,w", MTTKRP_CASES, ids=[c[0] for c in MTTKRP_CASES])
def test_concurrent_mttkrp_matches_each_submodel(name, w):
    _cuda()
    if w is None:
        w = W.make_config(1)
    with api.from_workload(w) as h:
        U = h.get_factors()
        # rows D_g of the sampled mode are zero after create (Alg. 3 initialisation)
        offs = offsets(w.ranks)
        for g, D in enumerate(w.left_out):
            assert np.all(U[w.n_hat][D, offs[g]:offs[g + 1]] == 0)
        for n in range(w.T.ndim):
            M = h.mttkrp(n)
            compare_mttkrp(w, M, U, n, MTTKRP_RTOL)
            # Case I rows D_g hold the full-tensor values (computed, then discarded)
            if n == w.n_hat:
                Mfull = O.mttkrp(w.T, U, n)
                np.testing.assert_allclose(M, Mfull, rtol=1e-11, atol=1e-11 * np.abs(Mfull).max())


def test_mttkrp_split_k_is_deterministic_and_split_independent():
    torch = _cuda()
    w = _ragged((40, 33, 65), 3, seed=6)
    outs = []
    for splits in (1, 3, 0):
        with api.from_workload(w, splits=splits) as h:
            a = h.mttkrp(1)
            b = h.mttkrp(1)
            np.testing.assert_array_equal(a, b)       # bit-reproducible
            outs.append(a)
    np.testing.assert_allclose(outs[0], outs[1], rtol=1e-13, atol=1e-13 * np.abs(outs[0]).max())
    np.testing.assert_allclose(outs[0], outs[2], rtol=1e-13, atol=1e-13 * np.abs(outs[0]).max())
    del torch


def _als_parity(w, sweeps, blocks=None, device=None, **kw):
    with api.from_workload(w, device=device, **kw) as h:
        losses = h.als_sweep(sweeps)
        U = h.get_factors()
        st = h.block_status()
    sel = list(range(w.K)) if blocks is None else list(blocks)
    ora = O.jk_als(w.T, w.n_hat, w.left_out, w.init, sweeps, blocks=sel)
    errs = assert_factors(w, U, ora.factors, sel, FACTOR_RTOL)
    lrel = np.abs(losses[:, sel] - ora.losses) / np.abs(ora.losses)
    return errs, lrel, st, losses, ora


@pytest.mark.parametrize("update_mode", [1, 2], ids=["fused", "two_phase"])
def test_cfg1_fp64_als_parity_50_sweeps(update_mode):
    """Configuration 1: 20x30x40, R=3, 20 LOO + full model, 50 sweeps, FP64."""
    _cuda()
    w = W.make_config(1)
    errs, lrel, st, losses, ora = _als_parity(w, w.sweeps, update_mode=update_mode)
    assert np.all(st == 0)
    assert errs.max() <= FACTOR_RTOL, errs.max()
    assert lrel.max() <= FACTOR_RTOL, lrel.max()


@pytest.mark.parametrize("update_mode", [1, 2], ids=["fused", "two_phase"])
@pytest.mark.parametrize("case", ["4way_nhat2", "delete3", "mixed_ranks", "nhat_last", "rank20"])
def test_als_parity_variants(case, update_mode):
    _cuda()
    if case == "4way_nhat2":
        w = _ragged((6, 5, 7, 4), 2, n_hat=2, seed=7)
    elif case == "delete3":
        w = _ragged((12, 9, 8), 2, d=3, seed=8)
    elif case == "mixed_ranks":
        w = _ragged((9, 20, 11), 2, ranks=[1, 2, 3, 2, 1, 3, 2, 1, 2, 3], seed=9)
    elif case == "rank20":
        w = _ragged((30, 24, 22), 20, seed=18, d=10)
    else:
        w = _ragged((7, 6, 9), 2, n_hat=2, seed=10)
    errs, lrel, st, _, _ = _als_parity(w, 20, update_mode=update_mode)
    assert np.all(st == 0)
    assert errs.max() <= FACTOR_RTOL, errs.max()
    assert lrel.max() <= FACTOR_RTOL, lrel.max()


def test_graph_and_eager_paths_agree_bitwise():
    _cuda()
    w = _ragged((10, 12, 14), 3, seed=11)
    res = []
    for g in (True, False):
        with api.from_workload(w, use_graph=g) as h:
            l = h.als_sweep(7)
            res.append((l, h.get_factors()))
    np.testing.assert_array_equal(res[0][0], res[1][0])
    for a, b in zip(res[0][1], res[1][1]):
        np.testing.assert_array_equal(a, b)


def test_host_and_device_buffers_agree():
    torch = _cuda()
    w = _ragged((10, 12, 14), 3, seed=12)
    with api.from_workload(w) as h:
        la = h.als_sweep(4)
        Ua = h.get_factors()
    with api.from_workload(w, device="cuda") as h:
        lb = h.als_sweep(4, device="cuda").cpu().numpy()
        Ub = [u.cpu().numpy() for u in h.get_factors(device="cuda")]
    np.testing.assert_array_equal(la, lb)
    for a, b in zip(Ua, Ub):
        np.testing.assert_array_equal(a, b)
    del torch


def test_not_spd_block_is_frozen_and_reported():
    _cuda()
    w = _ragged((8, 7, 9), 3, seed=13)
    bad = 2
    init = [u.copy() for u in w.init[bad]]
    init[1][:, 1] = 0.0          # zero column -> H(1,1) = 0 exactly -> zero pivot
    w.init = list(w.init)
    w.init[bad] = init
    with api.from_workload(w) as h:
        U0 = h.get_factors()
        l = h.als_sweep(3)
        st = h.block_status()
        U1 = h.get_factors()
        with pytest.raises(api.JKError) as ei:
            h.als_sweep(1, raise_not_spd=True)
        assert ei.value.status == 4
    assert st[bad] & 1
    assert np.all(st[np.arange(w.K) != bad] == 0)
    assert np.all(np.isnan(l[:, bad]))
    offs = offsets(w.ranks)
    for n in range(3):
        np.testing.assert_array_equal(U1[n][:, offs[bad]:offs[bad + 1]], U0[n][:, offs[bad]:offs[bad + 1]])
    ora = O.jk_als(w.T, w.n_hat, w.left_out, w.init, 3, blocks=[bad])
    assert ora.not_spd[0]


def test_run_with_tolerance_freezes_converged_blocks():
    _cuda()
    w = _ragged((9, 8, 10), 2, seed=14, noise=0.0)
    with api.from_workload(w) as h:
        done, final = h.run(400, tol=1e-9)
        st = h.block_status()
    assert np.all(st & 2)
    assert done < 400
    ora = O.jk_als(w.T, w.n_hat, w.left_out, w.init, 400, tol=1e-9, blocks=[0, 3])
    assert np.isfinite(final).all()
    for col, g in enumerate([0, 3]):
        last = ora.losses[:, col][np.isfinite(ora.losses[:, col])][-1]
        assert abs(final[g] - last) <= 1e-8 * ora.normT2[col]


def test_set_get_factors_roundtrip_and_resume():
    """Checkpoint/resume: 3 sweeps, save, 2 more == 5 sweeps straight."""
    _cuda()
    w = _ragged((10, 9, 8), 2, seed=15)
    with api.from_workload(w) as h:
        h.als_sweep(3)
        ck = h.get_factors()
        l_a = h.als_sweep(2)
        Ua = h.get_factors()
    with api.from_workload(w) as h:
        h.set_factors(ck)
        l_b = h.als_sweep(2)
        Ub = h.get_factors()
    # set_factors recomputes the Grams in another summation order than the
    # sweep's fused Gram refresh, so agreement is to rounding, not bitwise
    np.testing.assert_allclose(l_a, l_b, rtol=1e-12)
    for a, b in zip(Ua, Ub):
        np.testing.assert_allclose(a, b, rtol=1e-11, atol=1e-13)


def test_gradient_matches_oracle():
    _cuda()
    rng = np.random.default_rng(16)
    w = _ragged((10, 8, 8, 6), 2, seed=16)
    U = [rng.standard_normal((I, w.C)) for I in w.T.shape]
    with api.from_workload(w) as h:
        f, G = h.grad(U)
    for g, D in enumerate(w.left_out):
        U[0][D, 2 * g:2 * g + 2] = 0.0
    f_ref, G_ref = O.jk_loss_grad(w.T, 0, w.left_out, w.ranks, U)
    assert abs(f - f_ref) <= 1e-10 * abs(f_ref)
    for n in range(4):
        np.testing.assert_allclose(G[n], G_ref[n], rtol=1e-9, atol=1e-10 * np.abs(G_ref[n]).max())


def test_invalid_arguments_and_memory_cap():
    _cuda()
    w = _ragged((6, 5, 4), 2, seed=17)
    with pytest.raises(api.JKError) as ei:
        api.JKCALS(w.T, 5, w.ranks, w.left_out, api.multi_init(w.init))
    assert ei.value.status == 1
    with pytest.raises(api.JKError) as ei:
        api.JKCALS(w.T, 0, w.ranks, [[0, 0]] + list(w.left_out[1:]), api.multi_init(w.init))
    assert ei.value.status == 1
    with pytest.raises(api.JKError) as ei:
        api.JKCALS(w.T, 0, [33] * w.K, w.left_out, [np.zeros((I, 33 * w.K)) for I in w.T.shape])
    assert ei.value.status == 7
    with pytest.raises(api.JKError) as ei:
        api.from_workload(w, max_device_bytes=4096)
    assert ei.value.status == 3
    with api.from_workload(w) as h:       # a failed create leaves the device usable
        assert h.als_sweep(1).shape == (1, w.K)


def test_cfg2_fp64_sampled_blocks_full_size():
    """Configuration 2 at full size (300x100x50, 300 LOO, 100 sweeps), oracle on sampled blocks."""
    _cuda()
    w = W.make_config(2)
    blocks = [0, 151, 299]
    errs, lrel, st, _, _ = _als_parity(w, w.sweeps, blocks=blocks)
    assert np.all(st == 0)
    assert errs.max() <= FACTOR_RTOL, errs.max()
    assert lrel.max() <= FACTOR_RTOL, lrel.max()
