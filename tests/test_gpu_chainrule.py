"""GPU tests of the chain-rule sampler against the exact all-pattern table."""
import math

import numpy as np
import pytest
import torch

from paper_2009_01177_gb300 import chainrule
from paper_2009_01177_gb300 import gbs_inputs as gi

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx(cuda_lib):
    c = cuda_lib.Context(0)
    yield c
    c.close()


def table_p(ctx, st):
    tab = ctx.all_patterns(torch.from_numpy(st.O).cuda(), prec="fx128")
    return (tab["hi"] + tab["lo"]) * math.exp(-0.5 * np.linalg.slogdet(st.Sigma)[1])


def g_test_pvalue(p, pats):
    """G-test of the samples' counts against p (bins with expected count < 5 merged)."""
    from scipy.stats import chi2
    n = len(pats)
    codes = (pats.astype(np.int64) << np.arange(pats.shape[1])[None, :]).sum(1)
    obs = np.bincount(codes, minlength=p.size).astype(float)
    exp = p * n
    big = exp >= 5
    o = np.append(obs[big], obs[~big].sum())
    e = np.append(exp[big], exp[~big].sum())
    keep = e > 0
    o, e = o[keep], e[keep]
    with np.errstate(divide="ignore", invalid="ignore"):
        g = 2.0 * np.sum(np.where(o > 0, o * np.log(o / e), 0.0))
    return float(chi2.sf(g, len(o) - 1))


def test_reduced_state_prefix_probabilities_are_marginals(ctx):
    st = gi.lossy_gbs_state(7, 0.5, 1.1, 0.6, 71)
    p = table_p(ctx, st)
    M = st.M
    for j in (1, 3, 5):
        Oj, logdet = chainrule.reduced_O(st.Sigma, j)
        tab = ctx.all_patterns(torch.from_numpy(Oj).cuda(), prec="fx128")
        pj = (tab["hi"] + tab["lo"]) * math.exp(-0.5 * logdet)
        marg = np.zeros(1 << j)
        np.add.at(marg, np.arange(1 << M) & ((1 << j) - 1), p)
        assert np.max(np.abs(pj - marg)) < 1e-12, j


@pytest.mark.parametrize("form", ["noclick", "click"])
def test_chain_rule_samples_follow_the_exact_distribution(ctx, form):
    st = gi.lossy_gbs_state(10, 0.5, 1.0, 0.5, 72)
    p = table_p(ctx, st)
    pats = chainrule.sample(ctx, st.Sigma, 60000, seed=72, prec="auto", tol=1e-9, form=form)
    assert pats.shape == (60000, 10)
    assert g_test_pvalue(p, pats) > 1e-4
    assert chainrule.tv_against_table(p, pats) < 0.1


def test_chain_rule_click_window(ctx):
    st = gi.lossy_gbs_state(10, 0.6, 1.2, 0.5, 73)
    p = table_p(ctx, st)
    k = np.array([bin(c).count("1") for c in range(p.size)])
    pc = np.where((k >= 2) & (k <= 4), p, 0.0)
    pc /= pc.sum()
    pats = chainrule.sample(ctx, st.Sigma, 30000, seed=73, k_min=2, k_max=4, prec="auto", tol=1e-9)
    ks = pats.sum(1)
    assert ks.min() >= 2 and ks.max() <= 4
    assert g_test_pvalue(pc, pats) > 1e-4
