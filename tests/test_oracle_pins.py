"""Pins for the CPU oracle (-m "not gpu").

Each test ties the oracle to something other than itself: exact rational
arithmetic, closed forms from the physics, structural identities of Eq. 2,
normalisation of Eq. 1, and an independent vacuum-probability formulation.
The last test plants known mistakes in the oracle and checks that the pins
catch every one of them.
"""
from decimal import Decimal
from fractions import Fraction
import itertools
import math

import numpy as np
import pytest

import oracle
from paper_2009_01177_gb300 import gbs_inputs as gi
from tests import exact_small as ex


def dd_frac(hi, lo):
    return Fraction(hi) + Fraction(lo)


def rel(a, b):
    a, b = Fraction(a), Fraction(b)
    return abs(a - b) / abs(b) if b != 0 else abs(a - b)


# --------------------------------------------------------- fixed-point type
def test_fixed_point_ops_exact():
    rng = np.random.default_rng(7)
    for _ in range(200):
        a = float(rng.uniform(1e-3, 4.0)) * (1 if rng.random() < 0.8 else -1)
        b = float(rng.uniform(-4.0, 4.0))
        r = oracle.fx_ops(a, b)
        fa, fb = Fraction(a), Fraction(b)
        assert rel(dd_frac(*r[0]), fa * fb) < 2.0 ** -100
        assert dd_frac(*r[1]) == fa + fb            # exact
        assert dd_frac(*r[2]) == fa - fb            # exact
        if a > 0:
            assert rel(dd_frac(*r[3]), 1 / fa) < 2.0 ** -100
            exact = Decimal(1) / ex.frac_to_dec(fa).sqrt()
            got = ex.frac_to_dec(dd_frac(*r[4]))
            assert abs(got - exact) / exact < Decimal(2) ** -100


# ------------------------------------------------- determinants, brute force
@pytest.mark.parametrize("seed", [3, 4, 5])
def test_det_matches_exact_rational(seed):
    st = gi.lossy_gbs_state(6, 0.4, 1.1, 0.6, seed)
    O = gi.select(st.O, [0, 2, 3, 5])
    for mask in range(1, 16):
        hi, lo = oracle.det(O, mask)
        exact = ex.det_exact(ex.I_minus_OZ(O, mask))
        assert rel(dd_frac(hi, lo), exact) < 1e-30


@pytest.mark.parametrize("k,seed", [(1, 11), (2, 12), (3, 13), (4, 14), (5, 15)])
def test_tor_matches_exact_brute_force(k, seed):
    st = gi.lossy_gbs_state(8, 0.5, 1.0, 0.5, seed)
    O = gi.select(st.O, gi.random_pattern(8, k, seed))
    r = oracle.tor(O)
    exact = ex.tor_exact(O)
    got = ex.frac_to_dec(dd_frac(r.hi, r.lo))
    assert abs(got - exact) / abs(exact) < Decimal("1e-28")


# ------------------------------------------------------------ closed forms
@pytest.mark.parametrize("a", [0.1, 0.16, 0.25, 0.4])
@pytest.mark.parametrize("k", [1, 2, 3, 6, 10])
def test_thermal_closed_form(a, k):
    # O = a I: every t_Z = (1-a)^-|Z|, so Tor = (1/(1-a) - 1)^k (lower bound of Sec. 5.1 at k_corr = 0)
    r = oracle.tor(gi.thermal_O(k, a))
    fa = Fraction(a)
    exact = (1 / (1 - fa) - 1) ** k
    assert rel(dd_frac(r.hi, r.lo), exact) < 1e-28


@pytest.mark.parametrize("r,eta", [(0.3, 1.0), (0.8, 1.0), (1.2, 0.5), (0.9, 0.3)])
def test_single_mode_closed_form(r, eta):
    st = gi.lossy_gbs_state(1, r, r, eta, 0, U=np.eye(1), r=np.array([r]))
    sxx = eta * math.exp(-2 * r) / 2 + 1 - eta / 2
    spp = eta * math.exp(2 * r) / 2 + 1 - eta / 2
    tor_cf = math.sqrt(sxx * spp) - 1.0          # Tor = 1/sqrt(det Sigma^-1) - 1
    res = oracle.tor(st.O)
    assert abs(res.value - tor_cf) / tor_cf < 1e-13
    p1, p1lo, _ = oracle.prob(st.O, [1])
    p_click = 1.0 - 1.0 / math.sqrt(sxx * spp)
    assert abs(p1 + p1lo - p_click) / p_click < 1e-13
    if eta == 1.0:
        assert abs(p1 - (1 - 1 / math.cosh(r))) < 1e-14


def test_lossless_two_mode_squeezed_vacuum():
    r = 0.7
    bs = np.array([[1, 1], [1, -1]]) / math.sqrt(2)
    st = gi.lossy_gbs_state(2, r, r, 1.0, 0, U=bs.astype(complex), r=np.array([r, -r]))
    p10 = sum(oracle.prob(st.O, [1, 0])[:2])
    p01 = sum(oracle.prob(st.O, [0, 1])[:2])
    p11 = sum(oracle.prob(st.O, [1, 1])[:2])
    p00 = sum(oracle.prob(st.O, [0, 0])[:2])
    assert abs(p10) < 1e-14 and abs(p01) < 1e-14          # photon numbers perfectly correlated
    assert abs(p11 - (1 - 1 / math.cosh(r) ** 2)) < 1e-14
    assert abs(p00 - 1 / math.cosh(r) ** 2) < 1e-14


# ------------------------------------------------------ structural identities
@pytest.mark.parametrize("k1,k2,seed", [(2, 3, 21), (4, 4, 22), (5, 6, 23)])
def test_block_factorisation(k1, k2, seed):
    st1 = gi.lossy_gbs_state(10, 0.5, 1.0, 0.5, seed)
    st2 = gi.lossy_gbs_state(10, 0.6, 1.2, 0.3, seed + 100)
    O1 = gi.select(st1.O, gi.random_pattern(10, k1, seed))
    O2 = gi.select(st2.O, gi.random_pattern(10, k2, seed + 1))
    r1, r2 = oracle.tor(O1), oracle.tor(O2)
    r12 = oracle.tor(gi.block_diag_modes(O1, O2))
    assert rel(dd_frac(r12.hi, r12.lo), dd_frac(r1.hi, r1.lo) * dd_frac(r2.hi, r2.lo)) < 1e-28


@pytest.mark.parametrize("M,seed", [(4, 31), (5, 32), (7, 33)])
def test_click_probabilities_sum_to_one(M, seed):
    st = gi.lossy_gbs_state(M, 0.4, 1.0, 0.6, seed)
    total = Fraction(0)
    for pat in itertools.product([0, 1], repeat=M):
        hi, lo, _ = oracle.prob(st.O, pat, threads=1)
        assert hi >= -1e-15
        total += dd_frac(hi, lo)
    # floor: the float64 rounding of Sigma^-1 when O was built
    assert abs(float(total) - 1.0) < 1e-13


@pytest.mark.parametrize("M,seed", [(3, 41), (4, 42)])
def test_vacuum_probability_formulation(M, seed):
    # second formulation on different matrices: dets of Sigma's submatrices
    st = gi.lossy_gbs_state(M, 0.5, 1.0, 0.5, seed)
    for pat in itertools.product([0, 1], repeat=M):
        hi, lo, _ = oracle.prob(st.O, pat, threads=1)
        ref = ex.vacuum_prob_formula(st.Sigma, pat)
        assert abs(Decimal(hi) + Decimal(lo) - ref) < Decimal("1e-14")


def test_invariants():
    st = gi.lossy_gbs_state(12, 0.5, 1.2, 0.4, 51)
    O = gi.select(st.O, gi.random_pattern(12, 6, 51))
    k = 6
    dets = {mask: sum(oracle.det(O, mask)) if mask else 1.0 for mask in range(1 << k)}
    for mask, d in dets.items():
        assert 0 < d <= 1.0 + 1e-15                            # t_Z >= 1 (Sec. 5.1)
        for j in range(k):
            if not mask >> j & 1:
                assert dets[mask | 1 << j] <= d * (1 + 1e-14)  # det below its principal minors
    r = oracle.tor(O)
    assert 0 < r.value
    assert r.sum_abs >= abs(r.value)
    # Tor(O_S) <= sqrt(det Sigma_S): p(S) <= 1 for the marginal state of the clicked modes
    assert r.value * math.sqrt(dets[(1 << k) - 1]) <= 1.0


# ----------------------------------------------------------- self-consistency
def test_precision_and_thread_invariance():
    st, pat, O = gi.workload_m16_k10()
    a = oracle.tor(O, frac_bits=200, threads=1)
    b = oracle.tor(O, frac_bits=200, threads=4)
    c = oracle.tor(O, frac_bits=150, threads=4)
    assert (a.hi, a.lo, a.sum_abs) == (b.hi, b.lo, b.sum_abs)    # exact fixed-point sums
    assert rel(dd_frac(c.hi, c.lo), dd_frac(a.hi, a.lo)) < 1e-30


def test_range_split_adds_up():
    st, pat, O = gi.workload_m16_k10()
    whole = oracle.tor(O)
    parts = [oracle.tor_range(O, lo, lo + 256) for lo in range(0, 1024, 256)]
    s = sum(dd_frac(p.hi, p.lo) for p in parts)
    assert rel(s, dd_frac(whole.hi, whole.lo)) < 1e-30


# -------------------------------------------- planted mistakes must be caught
def _quick_pins(mutation):
    """Return the list of pins that FAIL for the oracle with `mutation` planted."""
    failed = []
    r = oracle.tor(gi.thermal_O(3, 0.25), mutation=mutation)
    if rel(dd_frac(r.hi, r.lo), Fraction(1, 27)) > 1e-28:
        failed.append("thermal")
    st = gi.lossy_gbs_state(8, 0.5, 1.0, 0.5, 13)
    O = gi.select(st.O, gi.random_pattern(8, 3, 13))
    r = oracle.tor(O, mutation=mutation)
    exact = ex.tor_exact(O)
    if abs(ex.frac_to_dec(dd_frac(r.hi, r.lo)) - exact) / abs(exact) > Decimal("1e-28"):
        failed.append("brute_force")
    return failed


def test_pins_catch_planted_mistakes():
    assert _quick_pins(0) == []
    # 1 drops Z = {}, 2 uses (-1)^|Z|, 3 picks the x row for p, 4 forms I + O,
    # 5 drops the first elimination update, 6 sums sqrt(det) instead of 1/sqrt(det)
    for mutation in range(1, 7):
        assert _quick_pins(mutation), f"mutation {mutation} not caught"


# ---- the exact (raw fixed-point) output, used to check the 256-bit GPU tier
@pytest.mark.parametrize("k", [1, 5, 9, 12])
def test_exact_output_thermal_closed_form(k):
    # O = I/4: Tor = (1/3)^k and sum t = (7/3)^k; the fixed-point evaluation must
    # land within a few 2^-200 units per term, far below the double-double output
    tor_x, sabs_x = oracle.tor_exact(gi.thermal_O(k, 0.25))
    sabs = Fraction(7, 3) ** k
    assert abs(tor_x - Fraction(1, 3) ** k) <= Fraction(1, 2 ** 195) * sabs
    assert abs(sabs_x - sabs) <= Fraction(1, 2 ** 195) * sabs


@pytest.mark.parametrize("k1,k2,seed", [(3, 4, 21), (4, 5, 22)])
def test_exact_output_block_factorisation(k1, k2, seed):
    # Tor(O1 (+) O2) = Tor(O1) Tor(O2) to the full fixed-point precision
    st = gi.lossy_gbs_state(k1 + k2, 0.6, 1.2, 0.5, seed)
    pat = np.arange(k1 + k2)
    O1, O2 = gi.select(st.O, pat[:k1]), gi.select(st.O, pat[k1:])
    t1, s1 = oracle.tor_exact(O1)
    t2, s2 = oracle.tor_exact(O2)
    t12, s12 = oracle.tor_exact(gi.block_diag_modes(O1, O2))
    assert abs(t12 - t1 * t2) <= Fraction(1, 2 ** 190) * s12
    assert abs(s12 - s1 * s2) <= Fraction(1, 2 ** 190) * s12


def test_exact_output_agrees_with_the_double_double_output():
    st, pat, O = gi.workload_m16_k10()
    ref = oracle.tor(O)
    tor_x, sabs_x = oracle.tor_exact(O)
    assert abs(Fraction(ref.hi) + Fraction(ref.lo) - tor_x) <= Fraction(1, 2 ** 104) * abs(tor_x)
    assert abs(Fraction(ref.sum_abs) + Fraction(ref.sum_abs_lo) - sabs_x) <= Fraction(1, 2 ** 104) * sabs_x
    # and a mask range is the sum of its halves, exactly
    a = oracle.tor_exact(O, 0, 300)
    b = oracle.tor_exact(O, 300, 1 << 10)
    assert (a[0] + b[0], a[1] + b[1]) == (tor_x, sabs_x)


def test_exact_output_mask_range_at_k64():
    # the largest k, masks above 2^63: O = I/4 gives t_Z = (4/3)^|Z| with sign (-1)^(64-|Z|)
    k = 64
    lo = (1 << 63) | (0x5A << 40)
    hi = lo + 4096
    tor_x, sabs_x = oracle.tor_exact(gi.thermal_O(k, 0.25), lo, hi)
    exact_t = sum((-1) ** (k - bin(m).count("1")) * Fraction(4, 3) ** bin(m).count("1") for m in range(lo, hi))
    exact_s = sum(Fraction(4, 3) ** bin(m).count("1") for m in range(lo, hi))
    assert abs(sabs_x - exact_s) <= Fraction(1, 2 ** 190) * exact_s
    assert abs(tor_x - exact_t) <= Fraction(1, 2 ** 190) * exact_s
