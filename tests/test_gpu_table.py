"""GPU tests of tor_all_patterns: the Torontonian of every click pattern of a
state from one walk and a Moebius transform, against per-pattern evaluation
(the batch path and the oracle) and against the sum-to-one of Eq. 1."""
import math
from fractions import Fraction

import numpy as np
import pytest
import torch

import oracle
from paper_2009_01177_gb300 import gbs_inputs as gi

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx(cuda_lib):
    c = cuda_lib.Context(0)
    yield c
    c.close()


def all_masks(M):
    return ((np.arange(1 << M)[:, None] >> np.arange(M)[None, :]) & 1).astype(np.uint8)


@pytest.mark.parametrize("M,prec", [(5, "fp64"), (10, "fp64"), (10, "dd"), (11, "fx128")])
def test_table_matches_per_pattern_batches(ctx, M, prec):
    # M = 5 takes the per-bit transform, M >= 10 the tiled one (M = 11: a one-bit last pass)
    st = gi.lossy_gbs_state(M, 0.5, 1.0, 0.5, 40 + M)
    Od = torch.from_numpy(st.O).cuda()
    tab = ctx.all_patterns(Od, prec=prec)
    ref = ctx.batch_patterns(Od, all_masks(M), prec="dd" if prec == "fp64" else prec)
    assert np.all(tab["status"] == 0)
    for S in range(1 << M):
        r = ref[S]
        assert r.status == 0
        diff = abs((Fraction(tab["hi"][S]) + Fraction(tab["lo"][S])) - (Fraction(r.hi) + Fraction(r.lo)))
        assert float(diff) <= tab["err_est"][S] + r.err_est + 1e-300, S
        assert abs(tab["sum_abs"][S] - r.sum_abs) <= 1e-12 * r.sum_abs, S


def test_table_probabilities_sum_to_one(ctx):
    M = 12
    st = gi.lossy_gbs_state(M, 0.6, 1.2, 0.4, 52)
    tab = ctx.all_patterns(torch.from_numpy(st.O).cuda(), prec="fx128")
    scale = math.exp(-0.5 * np.linalg.slogdet(st.Sigma)[1])
    total = float(np.sum(tab["hi"]) + np.sum(tab["lo"])) * scale
    assert abs(total - 1.0) <= 1e-12 + float(np.sum(tab["err_est"])) * scale
    assert (tab["hi"] + tab["lo"]).min() > -np.max(tab["err_est"])     # probabilities are non-negative


@pytest.mark.parametrize("prec", ["fp64", "dd", "fx128"])
def test_table_against_oracle(ctx, prec):
    M = 14
    st = gi.lossy_gbs_state(M, 0.5, 1.0, 0.5, 53)
    tab = ctx.all_patterns(torch.from_numpy(st.O).cuda(), prec=prec)
    rng = np.random.default_rng(53)
    masks = [0, 1, (1 << M) - 1] + [int(x) for x in rng.integers(0, 1 << M, 12)]
    for S in masks:
        modes = [j for j in range(M) if S >> j & 1]
        ref = oracle.tor(gi.select(st.O, modes)) if modes else None
        got = Fraction(tab["hi"][S]) + Fraction(tab["lo"][S])
        want = (Fraction(ref.hi) + Fraction(ref.lo)) if ref else Fraction(1)
        assert float(abs(got - want)) <= tab["err_est"][S] + float(abs(want)) * 2.0 ** -100, (S, prec)


def test_large_table_sampled_entries(ctx, cuda_lib):
    # 2^24 patterns; sampled entries against single Torontonians of their submatrices
    M = 24
    st = gi.lossy_gbs_state(M, 0.5, 1.0, 0.5, 54)
    Od = torch.from_numpy(st.O).cuda()
    out = torch.zeros((1 << M) * cuda_lib.RESULT_BYTES, dtype=torch.uint8, device="cuda")
    ctx.all_patterns_async(Od, out, prec="fx128")
    rng = np.random.default_rng(54)
    masks = [(1 << M) - 1, (1 << 23) | 5] + [int(x) for x in rng.integers(0, 1 << M, 10)]
    rows = out.view(1 << M, cuda_lib.RESULT_BYTES)[torch.tensor(masks, device="cuda")]
    got = cuda_lib.results_from_tensor(rows.reshape(-1), len(masks))
    for S, r in zip(masks, got):
        modes = [j for j in range(M) if S >> j & 1]
        s1 = ctx.single(torch.from_numpy(gi.select(st.O, modes)).cuda(), prec="fx128")
        assert r.status == 0
        diff = abs((Fraction(r.hi) + Fraction(r.lo)) - (Fraction(s1.hi) + Fraction(s1.lo)))
        assert float(diff) <= r.err_est + s1.err_est, S
        assert abs(r.sum_abs - s1.sum_abs) <= 1e-12 * s1.sum_abs, S


def test_table_argument_checks(ctx, cuda_lib):
    st = gi.lossy_gbs_state(6, 0.5, 1.0, 0.5, 55)
    with pytest.raises(cuda_lib.TorError):
        ctx.all_patterns(torch.from_numpy(st.O).cuda(), prec="fx256")
    big = torch.zeros((62, 62), dtype=torch.float64, device="cuda")    # M = 31 > TOR_TABLE_MAX_M
    out = torch.zeros(64, dtype=torch.uint8, device="cuda")
    assert ctx.lib.tor_all_patterns(ctx.h, big.data_ptr(), 31, 62, 1, None, out.data_ptr()) == cuda_lib.TOR_EINVAL


@pytest.mark.parametrize("M", [1, 9])
def test_smallest_tables(ctx, M):
    # M = 1 (two patterns) and M = 9 (the per-bit transform's largest size)
    st = gi.lossy_gbs_state(M, 0.5, 1.0, 0.5, 56 + M)
    Od = torch.from_numpy(st.O).cuda()
    tab = ctx.all_patterns(Od, prec="dd")
    assert (tab["hi"][0], tab["lo"][0]) == (1.0, 0.0)           # Tor of no clicks is 1
    for S in range(1, 1 << M):
        modes = [j for j in range(M) if S >> j & 1]
        r = ctx.single(torch.from_numpy(gi.select(st.O, modes)).cuda(), prec="dd")
        diff = abs((Fraction(tab["hi"][S]) + Fraction(tab["lo"][S])) - (Fraction(r.hi) + Fraction(r.lo)))
        assert float(diff) <= tab["err_est"][S] + r.err_est, S


def test_largest_table(ctx, cuda_lib):
    # M = 30 (TOR_TABLE_MAX_M): 2^30 patterns, 43 GB of results; sampled entries and the total
    M = 30
    st = gi.lossy_gbs_state(M, 0.5, 1.0, 0.5, 60)
    Od = torch.from_numpy(st.O).cuda()
    n = 1 << M
    out = torch.zeros(n * cuda_lib.RESULT_BYTES, dtype=torch.uint8, device="cuda")
    ctx.all_patterns_async(Od, out, prec="fp64")
    rec = out.view(n, cuda_lib.RESULT_BYTES)
    hi = rec[:, 0:8].contiguous().view(torch.float64).view(-1)
    lo = rec[:, 8:16].contiguous().view(torch.float64).view(-1)
    status = rec[:, 36:40].contiguous().view(torch.int32).view(-1)
    assert int((status != 0).sum()) == 0
    total = float((hi.sum() + lo.sum()).item()) * math.exp(-0.5 * np.linalg.slogdet(st.Sigma)[1])
    assert abs(total - 1.0) < 1e-9
    rng = np.random.default_rng(60)
    masks = [(1 << 29) | 3] + [int(x) & int(rng.integers(0, n)) for x in rng.integers(0, n, 6)]
    got = cuda_lib.results_from_tensor(rec[torch.tensor(masks, device="cuda")].reshape(-1), len(masks))
    for S, r in zip(masks, got):
        modes = [j for j in range(M) if S >> j & 1]
        s1 = ctx.single(torch.from_numpy(gi.select(st.O, modes)).cuda(), prec="fp64")
        diff = abs((Fraction(r.hi) + Fraction(r.lo)) - (Fraction(s1.hi) + Fraction(s1.lo)))
        assert float(diff) <= r.err_est + s1.err_est, S
    del out, rec, hi, lo, status
    torch.cuda.empty_cache()
