"""GPU tests of the Metropolis-Hastings step (gbs_sample_step).

The step is replayed on the CPU: proposals from the Python Philox4x32-10 and
the same marginals, exact probabilities from the oracle (Eq. 1), the same
acceptance rule; the chain's stationary distribution is checked against the
oracle's exact probabilities, and the learned proposal against the plain one.
"""
import itertools
import math

import numpy as np
import pytest
import torch

import oracle
from paper_2009_01177_gb300 import gbs_inputs as gi
from paper_2009_01177_gb300.tor import pack_patterns
from tests import philox_ref

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx(cuda_lib):
    c = cuda_lib.Context(0)
    yield c
    c.close()


def marginals(st):
    M = st.M
    out = []
    for j in range(M):
        S = st.Sigma[np.ix_([j, M + j], [j, M + j])]
        out.append(1.0 - 1.0 / math.sqrt(np.linalg.det(S)))
    return np.array(out)


def exact_probs(st):
    M = st.M
    pats = list(itertools.product([0, 1], repeat=M))
    p = np.array([sum(oracle.prob(st.O, pat, threads=1)[:2]) for pat in pats])
    codes = np.array([sum(b << j for j, b in enumerate(pat)) for pat in pats])
    out = np.zeros(1 << M)
    out[codes] = p
    return out


class Chains:
    def __init__(self, st, C):
        self.st, self.C = st, C
        self.M = st.M
        self.O = torch.from_numpy(st.O).cuda()
        self.logdet = float(np.linalg.slogdet(st.Sigma)[1])
        self.pat = torch.zeros((C, 1), dtype=torch.int64, device="cuda")
        self.logp = torch.full((C,), -math.inf, dtype=torch.float64, device="cuda")
        self.logq = torch.zeros(C, dtype=torch.float64, device="cuda")
        self.acc = torch.zeros(C, dtype=torch.int32, device="cuda")
        self.marg = torch.tensor(marginals(st), dtype=torch.float64, device="cuda")

    def step(self, ctx, seed, step, proposal=None):
        ctx.sample_step(self.O, self.logdet, self.pat, self.logp, self.logq, self.acc, seed, step,
                        marg_p=self.marg, proposal=proposal, prec="auto", tol=1e-9)
        return self.acc.cpu().numpy()


def test_plain_step_replays_on_cpu(ctx):
    st = gi.lossy_gbs_state(6, 0.4, 1.0, 0.6, 61)
    C, seed = 256, 1234
    ch = Chains(st, C)
    ch.step(ctx, seed, 0)                     # initialise: every chain accepts its first proposal
    assert np.all(ch.acc.cpu().numpy() == 1)
    before = ch.pat[:, 0].cpu().numpy().copy()
    lp_before = ch.logp.cpu().numpy().copy()
    lq_before = ch.logq.cpu().numpy().copy()
    acc = ch.step(ctx, seed, 1)
    after = ch.pat[:, 0].cpu().numpy()
    marg = marginals(st)
    checked = 0
    for c in range(C):
        us = [philox_ref.uniform(seed, 1, c, j) for j in range(st.M)]
        prop = [1 if us[j] < marg[j] else 0 for j in range(st.M)]
        code = sum(b << j for j, b in enumerate(prop))
        lq_new = sum(math.log(marg[j]) if prop[j] else math.log1p(-marg[j]) for j in range(st.M))
        p_new = sum(oracle.prob(st.O, prop, threads=1)[:2])
        la = (math.log(p_new) - lp_before[c]) + (lq_before[c] - lq_new)
        lu = math.log(philox_ref.uniform(seed, 1, c, st.M))
        if abs(lu - la) < 1e-6:
            continue                          # a near-tie: either decision is right
        expect = lu < la
        assert (acc[c] == 1) == expect and acc[c] in (0, 1), c
        assert after[c] == (code if expect else before[c])
        checked += 1
    assert checked > 0.95 * C


def test_chain_converges_to_exact_distribution(ctx):
    st = gi.lossy_gbs_state(5, 0.5, 1.1, 0.7, 62)
    p = exact_probs(st)
    assert abs(p.sum() - 1) < 1e-12
    ch = Chains(st, 8192)
    for step in range(40):
        ch.step(ctx, 77, step)
    freq = np.bincount(ch.pat[:, 0].cpu().numpy(), minlength=1 << st.M) / ch.C
    assert 0.5 * np.abs(freq - p).sum() < 0.05


def test_learned_proposal_beats_plain(ctx, cuda_lib):
    st = gi.lossy_gbs_state(8, 0.5, 1.0, 0.5, 63)
    M = st.M
    p = exact_probs(st)
    allx = ((np.arange(1 << M)[:, None] >> np.arange(M)[None, :]) & 1).astype(np.float64)
    net = cuda_lib.MLP(ctx, M, 128, seed=11)
    P = pack_patterns(allx, M).cuda()
    w = torch.tensor(p, dtype=torch.float32, device="cuda")
    for _ in range(400):                      # forward KL on exact probabilities
        net.train_step(P, w, lr=3e-3)
    results = {}
    for name, prop in (("plain", None), ("learned", net)):
        ch = Chains(st, 16384)
        accs, tvs = [], []
        for step in range(8):
            a = ch.step(ctx, 5, step, proposal=prop)
            if step:
                accs.append((a == 1).mean())
            freq = np.bincount(ch.pat[:, 0].cpu().numpy(), minlength=1 << M) / ch.C
            tvs.append(0.5 * float(np.abs(freq - p).sum()))
        results[name] = (float(np.mean(accs)), tvs)
    (a_plain, tv_plain), (a_learn, tv_learn) = results["plain"], results["learned"]
    # more proposals accepted, so fewer exact Torontonians per independent sample
    assert a_learn > a_plain + 0.1, results
    # and the chains start (and stay) closer to p while the plain chains are still burning in
    assert tv_learn[0] < tv_plain[0] and tv_learn[1] < tv_plain[1], results
    net.close()


def test_click_cap_targets_the_conditional_distribution(ctx):
    st = gi.lossy_gbs_state(6, 0.5, 1.1, 0.7, 64)
    M, k_cap = st.M, 2
    p = exact_probs(st)
    clicks = np.array([bin(c).count("1") for c in range(1 << M)])
    p_cond = np.where(clicks <= k_cap, p, 0.0)
    p_cond /= p_cond.sum()
    ch = Chains(st, 8192)
    capped = 0
    for step in range(40):
        ctx.sample_step(ch.O, ch.logdet, ch.pat, ch.logp, ch.logq, ch.acc, 91, step,
                        marg_p=ch.marg, prec="auto", tol=1e-9, k_cap=k_cap)
        codes = ch.pat[:, 0].cpu().numpy()
        # a chain holds its initial empty pattern until a proposal within the cap is accepted
        assert clicks[codes].max() <= k_cap
        # every rejection says why: the Metropolis test (0) or the cap (-1); nothing failed
        acc = ch.acc.cpu().numpy()
        assert set(np.unique(acc)) <= {-1, 0, 1}
        capped += int((acc == -1).sum())
    assert capped > 0
    freq = np.bincount(codes, minlength=1 << M) / ch.C
    assert 0.5 * np.abs(freq - p_cond).sum() < 0.05


# ------------------------------------------------------- delayed acceptance
class DAChains(Chains):
    def __init__(self, st, C, net):
        super().__init__(st, C)
        self.net = net
        self.logs = torch.zeros(C, dtype=torch.float64, device="cuda")

    def step_da(self, ctx, seed, step, k_cap=0):
        ctx.sample_step_da(self.O, self.logdet, self.pat, self.logp, self.logq, self.logs, self.acc, seed, step,
                           marg_p=self.marg, surrogate=self.net, prec="auto", tol=1e-9, k_cap=k_cap)
        return self.acc.cpu().numpy()


def _surrogate(cuda_lib, ctx, st, seed, scale):
    """A MADE network started at the plain proposal and then perturbed: a surrogate of p that
    is deliberately imperfect (the second test has to correct it)."""
    from oracle import made
    M = st.M
    net = cuda_lib.MLP(ctx, M, 32, seed=seed)
    net.set_marginals(marginals(st))
    th = net.get_params(0).astype(np.float64)
    th += scale * made.random_theta(M, 32, seed, scale=1.0) * (net.get_params(2) > 0)
    net.set_params(th)
    return net


def test_delayed_acceptance_step_replays_on_cpu(ctx, cuda_lib):
    st = gi.lossy_gbs_state(6, 0.4, 1.0, 0.6, 65)
    C, seed, M = 256, 4321, 6
    net = _surrogate(cuda_lib, ctx, st, 3, 0.5)
    ch = DAChains(st, C, net)
    acc0 = ch.step_da(ctx, seed, 0)           # initialise: uninitialised chains skip the first test
    assert np.all(acc0 == 1)
    allx = ((np.arange(1 << M)[:, None] >> np.arange(M)[None, :]) & 1).astype(np.float64)
    logs_all = net.logq(pack_patterns(allx, M).cuda()).cpu().numpy()   # the surrogate, every pattern
    before = ch.pat[:, 0].cpu().numpy().copy()
    assert np.allclose(ch.logs.cpu().numpy(), logs_all[before])
    lp_before, lq_before = ch.logp.cpu().numpy().copy(), ch.logq.cpu().numpy().copy()
    acc = ch.step_da(ctx, seed, 1)
    after = ch.pat[:, 0].cpu().numpy()
    marg = marginals(st)
    checked = screened = 0
    for c in range(C):
        us = [philox_ref.uniform(seed, 1, c, j) for j in range(M)]
        prop = [1 if us[j] < marg[j] else 0 for j in range(M)]
        code = sum(b << j for j, b in enumerate(prop))
        lq_new = sum(math.log(marg[j]) if prop[j] else math.log1p(-marg[j]) for j in range(M))
        la1 = (logs_all[code] - logs_all[before[c]]) + (lq_before[c] - lq_new)
        lu1 = math.log(philox_ref.uniform(seed, 1, c, M))
        if abs(lu1 - la1) < 1e-6:
            continue
        if not lu1 < la1:                     # screened out: no Torontonian, the chain stays
            assert acc[c] == -4 and after[c] == before[c], c
            screened += 1
            continue
        p_new = sum(oracle.prob(st.O, prop, threads=1)[:2])
        la2 = (math.log(p_new) - lp_before[c]) + (logs_all[before[c]] - logs_all[code])
        lu2 = math.log(philox_ref.uniform(seed, 1, c, M + 1))
        if abs(lu2 - la2) < 1e-6:
            continue
        expect = lu2 < la2
        assert acc[c] == (1 if expect else 0), c
        assert after[c] == (code if expect else before[c])
        checked += 1
    assert checked + screened > 0.95 * C and screened > 0 and checked > 0
    net.close()


def test_delayed_acceptance_targets_p_whatever_the_surrogate(ctx, cuda_lib):
    # a poor surrogate costs acceptance, never correctness: the exact second test makes the
    # chain reversible for p (Christen and Fox 2005)
    st = gi.lossy_gbs_state(5, 0.5, 1.1, 0.7, 62)
    p = exact_probs(st)
    net = _surrogate(cuda_lib, ctx, st, 4, 2.0)
    ch = DAChains(st, 8192, net)
    codes_seen = set()
    for step in range(60):
        codes_seen |= set(np.unique(ch.step_da(ctx, 78, step)).tolist())
    freq = np.bincount(ch.pat[:, 0].cpu().numpy(), minlength=1 << st.M) / ch.C
    assert 0.5 * np.abs(freq - p).sum() < 0.05
    assert codes_seen <= {-4, 0, 1} and -4 in codes_seen
    net.close()
