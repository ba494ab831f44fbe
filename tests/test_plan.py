"""Host-side planning (no GPU): jkcals_plan_query runs the planner jkcals_create uses and
reports, per mode, the MTTKRP kernel, rows per CTA, pipeline stages and split-K factor."""
import itertools

import pytest

from paper_2112_03985_gb300 import api

FORMS = ("fp64", "tf32", "3xtf32", "bf16", "split_bf16", "exact_bf16")
EXACT_BK = 32            # BF16 elements per 64-byte operand row of the exact form
EXACT_CHAIN_MAX = 1024   # columns of one exact chain


def test_fluorescence_workload_plan_is_the_profiled_launch():
    """300x100x50, 300 rank-5 submodels, exact-chain form on 152 SMs: the grids of the ncu
    capture (12 x 2 x 6, 12 x 2 x 6 and 12 x 1 x 12 CTAs)."""
    p = api.plan_query((300, 100, 50), [5] * 300, "exact_bf16", num_sms=152)
    assert [m["kernel"] for m in p] == ["tensor-core", "two-step", "two-step"]
    assert [m["tile_rows"] for m in p] == [160, 64, 64]
    assert [m["splits"] for m in p] == [6, 6, 12]


SHAPES = [(300, 100, 50), (20, 30, 40), (9, 150, 30), (129, 17, 33), (5, 1, 7), (6, 5, 4, 3), (140, 20, 12, 9),
          (400, 400, 400), (50, 200, 200), (100, 60, 60, 40), (8, 70, 60), (1000, 1100, 3)]


@pytest.mark.parametrize("prec", FORMS)
@pytest.mark.parametrize("dims", SHAPES, ids=["x".join(map(str, s)) for s in SHAPES])
def test_plan_invariants(prec, dims):
    K, R = 12, 4
    p = api.plan_query(dims, [R] * K, prec)
    assert len(p) == len(dims)
    for n, m in enumerate(p):
        assert m["splits"] >= 1
        if prec == "fp64":
            assert m == {"kernel": "fp64", "tile_rows": 64, "stages": 0, "splits": m["splits"]}
            continue
        assert m["tile_rows"] % 16 == 0 and 16 <= m["tile_rows"] <= 256
        assert 2 <= m["stages"] <= 4
        tiles_n = -(-dims[n] // m["tile_rows"])
        assert tiles_n * m["tile_rows"] - dims[n] < m["tile_rows"]   # no empty N tile
        big = max(d for k, d in enumerate(dims) if k != n)
        two_step = (prec == "exact_bf16" and dims[n] <= 128 and big >= 128
                    and -(-big // EXACT_BK) * EXACT_BK <= EXACT_CHAIN_MAX)
        assert (m["kernel"] == "two-step") == two_step, (n, m)
        if two_step:
            assert m["tile_rows"] <= 64
            others = 1
            for k, d in enumerate(dims):
                if k != n:
                    others *= d
            assert m["splits"] <= others // big        # whole index values o per split


def test_fp64_small_modes_spread_over_the_sms():
    """20x30x40, 21 rank-3 blocks: each mode's output is 64 x 64 at most, so the FP64
    MTTKRP splits down to one k-step of 16 columns of J per CTA rather than four,
    filling about half of 148 SMs instead of a tenth; larger outputs keep four."""
    p = api.plan_query((20, 30, 40), [3] * 21, "fp64", num_sms=148)
    J = [30 * 40, 20 * 40, 20 * 30]
    assert [m["splits"] for m in p] == [-(-j // 16) for j in J]
    big = api.plan_query((300, 100, 50), [5] * 300, "fp64", num_sms=148)
    ksteps = [-(-j // 16) for j in (5000, 15000, 30000)]
    assert all(m["splits"] <= k // 4 for m, k in zip(big, ksteps))


def test_user_split_factor_is_kept():
    p = api.plan_query((20, 30, 40), [3] * 21, "fp64", splits=3)
    assert [m["splits"] for m in p] == [3, 3, 3]


def test_plan_scales_splits_with_the_sm_count():
    few = api.plan_query((300, 100, 50), [5] * 300, "tf32", num_sms=38)
    many = api.plan_query((300, 100, 50), [5] * 300, "tf32", num_sms=152)
    assert all(a["splits"] <= b["splits"] for a, b in zip(few, many))
    assert any(a["splits"] < b["splits"] for a, b in zip(few, many))


@pytest.mark.parametrize("dims,ranks,prec", [
    ((5,), [2], "fp64"),                       # one mode
    ((5, 4, 3), [], "fp64"),                   # no blocks
    ((5, 0, 3), [2], "fp64"),                  # empty mode
    ((5, 4, 3), [0], "fp64"),                  # rank 0
])
def test_plan_argument_errors(dims, ranks, prec):
    with pytest.raises(api.JKError) as ei:
        api.plan_query(dims, ranks, prec)
    assert ei.value.status == 1   # JKCALS_ERR_ARG


@pytest.mark.parametrize("dims,ranks,prec", [
    ((5, 4, 3), [33], "fp64"),                          # rank above 32
    ((2, 50000, 50000), [2], "tf32"),                   # 2.5e9 columns: 32-bit column index
])
def test_plan_unsupported_shapes(dims, ranks, prec):
    with pytest.raises(api.JKError) as ei:
        api.plan_query(dims, ranks, prec)
    assert ei.value.status == 7   # JKCALS_ERR_UNSUPPORTED


def test_every_form_plans_every_small_shape():
    for prec, dims in itertools.product(FORMS, [(3, 3, 3), (1, 7, 2), (2, 2, 2, 2, 2)]):
        assert len(api.plan_query(dims, [1, 2], prec)) == len(dims)

