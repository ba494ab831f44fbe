"""Seeded synthetic workloads shaped like the paper's experiments.

This module only *draws inputs*: planted CP factors, the noisy target tensor
built from them, the shared initial factor set and the jackknife block layout
(which samples each submodel leaves out).  It holds none of the fitting
method's arithmetic (no MTTKRP, no Gram, no solve, no loss), so both the FP64
oracle and the CUDA library can consume its output without sharing code.

Shapes follow Sec. 5 of the paper (few samples in mode 1, many variables in the
other modes; Sec. 5.1 synthetic 50 x m x m tensors and the chemometrics
shapes of Sec. 5.2), made concrete by five configurations:

    1  20x30x40, planted rank 3, U ~ U[0,1], 1% noise, FP64, 20 LOO + full
    2  300x100x50 fluorescence-like, rank 5, lognormal sample scores and
       Gaussian-bump spectra, 2% noise, FP32 tensor, 300 LOO submodels
    3  400x400x400 FP32, rank R in {5,10,20}, column congruence 0.5,
       1% noise, delete-d with 40 contiguous groups of 10 samples
    4  64 independent LOO problems of uneven size and rank, FP32
    5  100x60x60x40 4-way, rank 8, 1% noise, 100 LOO submodels

Seeds: factors = 1000c+0, noise = 1000c+1, init = 1000c+2, sizes = 1000c+3.
Noise E ~ N(0,1) is scaled so that ||E||_F = level * ||T_clean||_F.  An FP32
configuration rounds T once to FP32; every consumer then sees exactly those
values (upcast to FP64 where it computes in FP64).
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import List, Optional, Sequence

import numpy as np

__all__ = [
    "Workload",
    "planted_tensor",
    "loo_blocks",
    "group_blocks",
    "make_workload",
    "make_config",
    "make_config4_batch",
]


@dataclass
class Workload:
    """One jackknife problem.

    T           target tensor (np.float64 array; for ``dtype == 'f32'`` every
                value is exactly representable in FP32)
    n_hat       sampled mode, 0-based (the paper's \\hat{n} minus one)
    ranks       R_g for every block (submodel) g
    left_out    D_g for every block: sorted int64 indices of the samples of
                mode n_hat that block g leaves out (empty = the full model)
    init        init[g][n]: initial factor of mode n for block g, I_n x R_g,
                with all I_n rows (the solver pads/zeroes rows itself)
    sweeps      number of ALS sweeps the configuration runs
    truth       planted factors (for recovery checks), or None
    """

    name: str
    T: np.ndarray
    n_hat: int
    ranks: List[int]
    left_out: List[np.ndarray]
    init: List[List[np.ndarray]]
    sweeps: int
    dtype: str = "f64"
    truth: Optional[List[np.ndarray]] = None
    meta: dict = field(default_factory=dict)

    @property
    def dims(self):
        return tuple(int(d) for d in self.T.shape)

    @property
    def K(self) -> int:
        return len(self.ranks)

    @property
    def C(self) -> int:
        return int(sum(self.ranks))


def _cp_tensor(factors: Sequence[np.ndarray]) -> np.ndarray:
    """Dense tensor sum_r u_1r o u_2r o ... o u_Nr (data synthesis only)."""
    N = len(factors)
    letters = "abcdefghijklmnopq"[:N]
    spec = ",".join(f"{l}z" for l in letters) + "->" + letters
    return np.einsum(spec, *factors, optimize=True)


def planted_tensor(factors, noise_level, noise_seed, dtype="f64"):
    """Planted CP tensor plus Gaussian noise scaled to ``noise_level`` of its norm."""
    T = _cp_tensor(factors)
    if noise_level > 0:
        rng = np.random.default_rng(noise_seed)
        E = rng.standard_normal(T.shape)
        E *= noise_level * np.linalg.norm(T.ravel()) / np.linalg.norm(E.ravel())
        T = T + E
    if dtype == "f32":
        T = T.astype(np.float32).astype(np.float64)
    return np.ascontiguousarray(T)


def loo_blocks(I_hat: int, include_full: bool = False) -> List[np.ndarray]:
    """Leave-one-out: block p leaves out sample p (Alg. 2); optional full model last."""
    blocks = [np.array([p], dtype=np.int64) for p in range(I_hat)]
    if include_full:
        blocks.append(np.zeros(0, dtype=np.int64))
    return blocks


def group_blocks(I_hat: int, d: int) -> List[np.ndarray]:
    """Delete-d with contiguous groups {d*g, ..., d*g+d-1} (Sec. 4.1, last remark)."""
    if d < 1 or I_hat % d != 0:
        raise ValueError(f"group size {d} must divide the {I_hat} samples")
    return [np.arange(g * d, (g + 1) * d, dtype=np.int64) for g in range(I_hat // d)]


def all_ranks_blocks(I_hat: int, ranks=(3, 5, 7, 9)):
    """The "All" layout of Sec. 5.1: every left-out sample jackknifed with one model
    per rank in ``ranks``, side by side in one concurrent fit.  Returns (blocks, ranks)
    with block k leaving out sample k // len(ranks) at rank ranks[k % len(ranks)]."""
    blocks = [np.array([p], dtype=np.int64) for p in range(I_hat) for _ in ranks]
    return blocks, [int(r) for _ in range(I_hat) for r in ranks]


def make_workload(name, dims, R, *, n_hat=0, blocks=None, noise=0.01, seed=0,
                  sweeps=10, dtype="f64", factor_kind="uniform", init_kind="uniform",
                  ranks=None):
    """Generic planted-CP jackknife problem with one shared initial factor set.

    ``ranks`` (optional) gives a rank per block (heterogeneous models fitted
    together, the "All" experiment of Sec. 5.1); the planted rank is ``R``.
    """
    rng_f = np.random.default_rng(seed + 0)
    N = len(dims)
    if factor_kind == "uniform":
        truth = [rng_f.uniform(0.0, 1.0, size=(I, R)) for I in dims]
    elif factor_kind == "normal":
        truth = [rng_f.standard_normal((I, R)) for I in dims]
    else:
        raise ValueError(factor_kind)
    T = planted_tensor(truth, noise, seed + 1, dtype)
    if blocks is None:
        blocks = loo_blocks(dims[n_hat])
    if ranks is None:
        ranks = [R] * len(blocks)
    rng_i = np.random.default_rng(seed + 2)
    shared = {}
    init = []
    for r in ranks:
        if r not in shared:
            if init_kind == "uniform":
                shared[r] = [rng_i.uniform(0.0, 1.0, size=(I, r)) for I in dims]
            else:
                shared[r] = [rng_i.standard_normal((I, r)) for I in dims]
        init.append(shared[r])
    return Workload(name=name, T=T, n_hat=n_hat, ranks=list(ranks), left_out=list(blocks),
                    init=init, sweeps=sweeps, dtype=dtype, truth=truth)


def _bumps(I, R, rng):
    """Nonnegative Gaussian bumps exp(-(x-mu)^2/(2 sigma^2)), mu ~ U[0,I), sigma ~ U[.05,.15]*I."""
    mu = rng.uniform(0.0, I, size=R)
    sigma = rng.uniform(0.05, 0.15, size=R) * I
    x = np.arange(I, dtype=np.float64)[:, None]
    return np.exp(-((x - mu[None, :]) ** 2) / (2.0 * sigma[None, :] ** 2))


def make_config(c: int, R: Optional[int] = None, include_full: Optional[bool] = None) -> Workload:
    """Configurations 1, 2, 3 and 5 (configuration 4 is ``make_config4_batch``)."""
    base = 1000 * c
    if c == 1:
        dims, R0 = (20, 30, 40), 3
        w = make_workload("cfg1 20x30x40 R3 LOO+full FP64", dims, R0, n_hat=0,
                          blocks=loo_blocks(20, include_full=True if include_full is None else include_full),
                          noise=0.01, seed=base, sweeps=50, dtype="f64")
        return w
    if c == 2:
        dims, R0 = (300, 100, 50), 5 if R is None else R
        rng_f = np.random.default_rng(base + 0)
        U1 = rng_f.lognormal(0.0, 0.5, size=(dims[0], R0))
        U2 = _bumps(dims[1], R0, rng_f)
        U3 = _bumps(dims[2], R0, rng_f)
        truth = [U1, U2, U3]
        T = planted_tensor(truth, 0.02, base + 1, "f32")
        blocks = loo_blocks(dims[0], include_full=bool(include_full))
        rng_i = np.random.default_rng(base + 2)
        init1 = [rng_i.uniform(0.0, 1.0, size=(I, R0)) for I in dims]
        return Workload(name="cfg2 300x100x50 R5 LOO fluorescence-like", T=T, n_hat=0,
                        ranks=[R0] * len(blocks), left_out=blocks, init=[init1] * len(blocks),
                        sweeps=100, dtype="f32", truth=truth)
    if c == 3:
        R0 = 10 if R is None else R
        dims = (400, 400, 400)
        rng_f = np.random.default_rng(base + 0)
        S = 0.5 * np.ones((R0, R0)) + 0.5 * np.eye(R0)
        L = np.linalg.cholesky(S)
        truth = [rng_f.standard_normal((I, R0)) @ L.T for I in dims]
        T = planted_tensor(truth, 0.01, base + 1, "f32")
        blocks = group_blocks(400, 10)
        rng_i = np.random.default_rng(base + 2)
        init1 = [rng_i.uniform(0.0, 1.0, size=(I, R0)) for I in dims]
        return Workload(name=f"cfg3 400^3 R{R0} delete-10 x40 FP32", T=T, n_hat=0,
                        ranks=[R0] * len(blocks), left_out=blocks, init=[init1] * len(blocks),
                        sweeps=20, dtype="f32", truth=truth)
    if c == 5:
        dims, R0 = (100, 60, 60, 40), 8
        return make_workload("cfg5 100x60x60x40 R8 LOO", dims, R0, n_hat=0,
                             blocks=loo_blocks(100), noise=0.01, seed=base, sweeps=10,
                             dtype="f32", factor_kind="normal", init_kind="normal")
    raise ValueError(f"unknown configuration {c}")


def make_config4_batch(n_problems: int = 64, seed_offset: int = 0) -> List[Workload]:
    """Configuration 4: independent LOO problems of uneven sizes and ranks."""
    base = 4000 + seed_offset
    rng_s = np.random.default_rng(base + 3)
    out = []
    for b in range(n_problems):
        I1 = int(rng_s.integers(20, 401))
        I2 = int(rng_s.integers(30, 151))
        I3 = int(rng_s.integers(30, 151))
        R = int(rng_s.integers(2, 9))
        w = make_workload(f"cfg4[{b}] {I1}x{I2}x{I3} R{R}", (I1, I2, I3), R, n_hat=0,
                          blocks=loo_blocks(I1), noise=0.01, seed=base + 10 * b,
                          sweeps=50, dtype="f32")
        out.append(w)
    return out
