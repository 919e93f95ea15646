"""GPU tests of tor_levels: the paper's level-by-level schedule with a fresh elimination per
subset, against the oracle and against the prefix-tree walk."""
from fractions import Fraction

import numpy as np
import pytest
import torch

import oracle
from paper_2009_01177_gb300 import gbs_inputs as gi

pytestmark = pytest.mark.gpu


def dev(O):
    return torch.from_numpy(np.ascontiguousarray(O)).cuda()


def val(r):
    return Fraction(r.hi) + Fraction(r.lo)


@pytest.mark.parametrize("prec", ["fp64", "dd", "fx128"])
@pytest.mark.parametrize("k", [1, 6, 12])
def test_levels_against_oracle(cuda_lib, prec, k):
    st, pat, O32 = gi.workload_m100(32)
    O = gi.select(st.O, pat[:k])
    ref = oracle.tor(O)
    r = cuda_lib.levels(dev(O), prec=prec)
    assert r.status == 0
    assert float(abs(val(r) - (Fraction(ref.hi) + Fraction(ref.lo)))) <= r.err_est + abs(ref.value) * 2.0 ** -104
    assert abs(r.sum_abs - ref.sum_abs) <= 1e-12 * ref.sum_abs


@pytest.mark.parametrize("k", [20, 22])
def test_levels_against_the_walk(cuda_lib, k):
    # two GPU evaluations with nothing in common but the input: every level in
    # double-double here, the walk in double-double and fixed point
    st, pat, O32 = gi.workload_m100(32)
    Od = dev(gi.select(st.O, pat[:k]))
    ctx = cuda_lib.Context(0)
    try:
        walk = [ctx.single(Od, prec=p) for p in ("dd", "fx128")]
    finally:
        ctx.close()
    r = cuda_lib.levels(Od, prec="dd")
    for w in walk:
        assert float(abs(val(r) - val(w))) <= r.err_est + w.err_est
        assert abs(r.sum_abs - w.sum_abs) <= 1e-12 * w.sum_abs


def test_per_level_precision(cuda_lib):
    # the paper's per-|Z| choice: FP64 for small subsets, double-double for large
    st, pat, O32 = gi.workload_m100(32)
    k = 14
    O = gi.select(st.O, pat[:k])
    ref = oracle.tor(O)
    lp = ["fp64"] * 7 + ["dd"] * (k + 1 - 7)
    r = cuda_lib.levels(dev(O), level_prec=lp)
    r64 = cuda_lib.levels(dev(O), prec="fp64")
    assert r.tier == 1                                    # the least precise tier used
    e = float(abs(val(r) - (Fraction(ref.hi) + Fraction(ref.lo))))
    assert e <= r.err_est < r64.err_est                    # mixing tightens the bound


def test_levels_edge_cases(cuda_lib):
    r = cuda_lib.levels(torch.zeros((0, 0), dtype=torch.float64, device="cuda"))
    assert (r.hi, r.lo, r.status) == (1.0, 0.0, 0)
    r = cuda_lib.levels(dev(gi.thermal_O(5, 0.25)))
    assert abs(r.value - (1 / 3) ** 5) <= r.err_est
    with pytest.raises(cuda_lib.TorError):
        cuda_lib.levels(dev(gi.thermal_O(3, 0.25)), prec="fx256")
    with pytest.raises(ValueError):
        cuda_lib.levels(dev(gi.thermal_O(3, 0.25)), level_prec=["fp64"] * 3)
