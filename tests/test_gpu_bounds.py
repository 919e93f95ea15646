"""GPU tests of the FP32 bound pass (tor_bounds) and the AUTO precision router."""
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


def reference_bound(O, tol):
    """The bound pass's formulas in numpy FP64 (the kernel computes them in FP32)."""
    k = O.shape[0] // 2
    B = np.eye(2 * k) - O
    tau = np.array([1 / math.sqrt(np.linalg.det(B[np.ix_([j, k + j], [j, k + j])])) for j in range(k)])
    lm = float(np.sum(np.log(np.maximum(tau - 1, 1e-30))))
    lp = float(np.sum(np.log(tau + 1)))
    sign, ld = np.linalg.slogdet(B)
    bits = (lp - lm) / math.log(2) + math.log2(4 * max(k, 1)) + math.log2(1 / tol)
    return {"log_tmax": -0.5 * ld, "log_tor_est": lm, "log_kappa_est": lp - lm, "bits_needed": bits}


def test_bounds_match_reference_formulas(ctx):
    st, pat, O32 = gi.workload_m100(32)
    mats = [gi.select(st.O, pat[:k]) for k in (1, 4, 9, 16, 25, 32)]
    mats.append(gi.workload_m16_k10()[2])
    got = ctx.bounds([torch.from_numpy(O).cuda() for O in mats], tol=1e-10)
    for O, g in zip(mats, got):
        ref = reference_bound(O, 1e-10)
        for key in ("log_tmax", "log_tor_est", "log_kappa_est", "bits_needed"):
            assert abs(g[key] - ref[key]) <= 1e-3 * max(1.0, abs(ref[key])), (key, g[key], ref[key])
        bits, lt = ref["bits_needed"], ref["log_tmax"] / math.log(2)
        want = (1 if bits <= 72 else 3 if (lt <= 11 and bits <= 120) else 2 if bits <= 124
                else 4 if lt <= 30 else 2)
        assert g["tier"] == want, (bits, lt, g["tier"])


def test_bounds_thermal_are_exact_estimates(ctx):
    # O = a I: Tor_est is exact, (a/(1-a))^k, and t_max = (1-a)^-k
    a, k = 0.25, 6
    g = ctx.bounds([torch.from_numpy(gi.thermal_O(k, a)).cuda()], tol=1e-3)[0]
    assert abs(g["log_tor_est"] - k * math.log(1 / 3)) < 1e-4
    assert abs(g["log_tmax"] - k * math.log(4 / 3)) < 1e-4


def test_kappa_estimate_is_conservative_on_gbs_states(ctx):
    st, pat, O32 = gi.workload_m100(32)
    mats = [gi.select(st.O, pat[:k]) for k in (6, 8, 10, 12)] + [gi.workload_m16_k10()[2]]
    got = ctx.bounds([torch.from_numpy(O).cuda() for O in mats], tol=1e-10)
    for O, g in zip(mats, got):
        kappa = oracle.tor(O).kappa
        assert g["log_kappa_est"] >= math.log(kappa) - 0.1


def test_bounds_flag_not_positive_definite_and_invalid(ctx):
    g = ctx.bounds([torch.from_numpy(2.0 * np.eye(6)).cuda()], tol=1e-10)[0]
    assert math.isinf(g["bits_needed"]) and g["tier"] == 2


@pytest.mark.parametrize("tol", [1e-4, 1e-8, 1e-12, 1e-18])
def test_auto_meets_tolerance_or_reports(ctx, cuda_lib, tol):
    st, pat, O32 = gi.workload_m100(32)
    for k in (6, 10, 14):
        O = gi.select(st.O, pat[:k])
        ref = oracle.tor(O)
        try:
            r = ctx.single(torch.from_numpy(O).cuda(), prec="auto", tol=tol)
        except cuda_lib.TorError as e:
            assert e.code == cuda_lib.TOR_EPREC
            continue
        assert abs((r.hi - ref.hi) + (r.lo - ref.lo)) <= max(r.err_est, 0) <= tol * abs(ref.value) * (1 + 1e-6)


def test_auto_uses_fixed_point_between_fp64_and_double_double(ctx):
    # kappa = 4e15: FP64's bound (64 u kappa = 30) misses 1e-12, fixed point's (2e-13) meets it
    st, pat, O32 = gi.workload_m100(32)
    O = gi.select(st.O, pat[:16])
    ref = oracle.tor(O)
    r = ctx.single(torch.from_numpy(O).cuda(), prec="auto", tol=1e-12)
    assert r.tier == 3
    err = abs(float(Fraction(r.hi) + Fraction(r.lo) - Fraction(ref.hi) - Fraction(ref.lo)))
    assert err <= r.err_est <= 1e-12 * abs(ref.value)


def test_auto_picks_fp64_when_well_conditioned(ctx):
    st = gi.lossy_gbs_state(24, 1.6, 2.0, 0.9, 77)
    O = gi.select(st.O, gi.random_pattern(24, 8, 77))
    r = ctx.single(torch.from_numpy(O).cuda(), prec="auto", tol=1e-6)
    assert r.tier == 1
    ref = oracle.tor(O)
    assert abs(r.value - ref.value) <= 1e-6 * abs(ref.value)
