"""CPU tests of the chain-rule sampler's host logic, both forms, with the oracle's
Torontonians in place of the batched GPU ones (M = 6: every pattern's exact
probability is known)."""
import numpy as np
import pytest

import oracle
from paper_2009_01177_gb300 import chainrule
from paper_2009_01177_gb300 import gbs_inputs as gi


def oracle_evaluator():
    cache = {}

    def evaluate(j, Oj, cand):
        val = np.empty(cand.shape[0])
        for r, row in enumerate(cand):
            key = (j, row.tobytes())
            if key not in cache:
                modes = np.nonzero(row)[0]
                cache[key] = oracle.tor(gi.select(Oj, modes)).value if modes.size else 1.0
            val[r] = cache[key]
        return val, val > 0
    return evaluate


def exact_table(st):
    p = np.empty(1 << st.M)
    for code in range(1 << st.M):
        pat = ((code >> np.arange(st.M)) & 1).astype(np.uint8)
        hi, lo, _ = oracle.prob(st.O, pat)
        p[code] = hi + lo
    return p


def chi2_pvalue(p, pats):
    from scipy.stats import chi2
    codes = (pats.astype(np.int64) << np.arange(pats.shape[1])[None, :]).sum(1)
    obs = np.bincount(codes, minlength=p.size).astype(float)
    exp = p * len(pats)
    keep = exp >= 5
    o = np.append(obs[keep], obs[~keep].sum())
    e = np.append(exp[keep], exp[~keep].sum())
    o, e = o[e > 0], e[e > 0]
    return float(chi2.sf(np.sum((o - e) ** 2 / e), len(o) - 1))


@pytest.fixture(scope="module")
def state():
    st = gi.lossy_gbs_state(6, 0.5, 1.0, 0.5, 81)
    return st, exact_table(st)


def test_exact_table_sums_to_one(state):
    _, p = state
    assert abs(p.sum() - 1.0) < 1e-12


@pytest.mark.parametrize("form", ["noclick", "click"])
def test_samples_follow_the_exact_distribution(state, form):
    st, p = state
    stats = {}
    pats = chainrule.sample(None, st.Sigma, 20000, seed=5, form=form, stats=stats,
                            evaluate=oracle_evaluator())
    assert pats.shape == (20000, 6)
    assert chi2_pvalue(p, pats) > 1e-4
    assert chainrule.tv_against_table(p, pats) < 0.03
    assert stats["torontonians"] >= 20000 * 6


def test_noclick_form_evaluates_half_the_subsets(state):
    st, _ = state
    s0, s1 = {}, {}
    chainrule.sample(None, st.Sigma, 4000, seed=6, form="noclick", stats=s0, evaluate=oracle_evaluator())
    chainrule.sample(None, st.Sigma, 4000, seed=6, form="click", stats=s1, evaluate=oracle_evaluator())
    assert s0["torontonians"] == s1["torontonians"]      # one per live sample and mode
    assert s0["subsets"] < 0.6 * s1["subsets"]           # 2^k against 2^(k+1)


def test_click_window_is_the_conditional_distribution(state):
    st, p = state
    k = np.array([bin(c).count("1") for c in range(p.size)])
    pc = np.where((k >= 2) & (k <= 3), p, 0.0)
    pc /= pc.sum()
    pats = chainrule.sample(None, st.Sigma, 15000, seed=7, k_min=2, k_max=3, evaluate=oracle_evaluator())
    ks = pats.sum(1)
    assert ks.min() >= 2 and ks.max() <= 3
    assert chi2_pvalue(pc, pats) > 1e-4


def test_a_failed_evaluation_is_an_error(state):
    st, _ = state
    inner = oracle_evaluator()

    def failing(j, Oj, cand):
        val, ok = inner(j, Oj, cand)
        if j == 4:
            ok = ok.copy()
            ok[0] = False
        return val, ok
    with pytest.raises(RuntimeError, match="mode 4"):
        chainrule.sample(None, st.Sigma, 100, seed=2, evaluate=failing)


def test_unknown_form_is_rejected(state):
    st, _ = state
    with pytest.raises(ValueError):
        chainrule.sample(None, st.Sigma, 10, seed=1, form="both", evaluate=oracle_evaluator())
