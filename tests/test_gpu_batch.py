"""GPU tests of tor_batch: many Torontonians of uneven k in one scheduled launch."""
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


def mats_uneven(seed=4, n=40, k_lo=0, k_hi=16):
    st = gi.lossy_gbs_state(100, 0.6, 1.2, 0.3, seed)
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(n):
        k = int(rng.integers(k_lo, k_hi + 1))
        out.append(gi.select(st.O, np.sort(rng.choice(100, size=k, replace=False))))
    return out


def err(r, ref):
    return abs(float(Fraction(r.hi) + Fraction(r.lo) - Fraction(ref.hi) - Fraction(ref.lo)))


@pytest.mark.parametrize("prec", ["fp64", "dd"])
def test_batch_matches_single_and_oracle(ctx, prec):
    mats = mats_uneven()
    dmats = [torch.from_numpy(O).cuda() for O in mats]
    res = ctx.batch(dmats, prec=prec)
    for i, (O, Od, r) in enumerate(zip(mats, dmats, res)):
        assert r.status == 0, (i, r)
        s = ctx.single(Od, prec=prec) if O.shape[0] else None
        if s is not None:
            assert abs((r.hi - s.hi) + (r.lo - s.lo)) <= r.err_est + s.err_est
            assert abs(r.sum_abs - s.sum_abs) <= 1e-12 * s.sum_abs
        if O.shape[0] <= 24:
            ref = oracle.tor(O)
            assert err(r, ref) <= r.err_est, (i, O.shape[0] // 2)


def test_batch_is_deterministic(ctx):
    dmats = [torch.from_numpy(O).cuda() for O in mats_uneven(seed=9, n=64, k_hi=20)]
    a = ctx.batch(dmats, prec="fp64")
    b = ctx.batch(dmats, prec="fp64")
    assert [(x.hi, x.lo, x.sum_abs) for x in a] == [(x.hi, x.lo, x.sum_abs) for x in b]


def test_batch_statuses(ctx, cuda_lib):
    good = gi.workload_m16_k10()[2]
    bad = 2.0 * np.eye(8)
    dm = [torch.from_numpy(O).cuda() for O in (good, bad, np.zeros((0, 0)), good)]
    res = ctx.batch(dm, prec="fp64")
    assert res[0].status == 0 and res[3].status == 0
    assert (res[0].hi, res[0].lo) == (res[3].hi, res[3].lo)
    assert res[1].status == cuda_lib.TOR_ENOTPD
    assert (res[2].hi, res[2].lo, res[2].status) == (1.0, 0.0, 0)


def test_batch_rejects_k_beyond_reservation(ctx, cuda_lib):
    ctx.batch_reserve(8, 6)
    mats = [gi.thermal_O(4, 0.2), gi.thermal_O(9, 0.2)]
    dm = [torch.from_numpy(O).cuda() for O in mats]
    ptrs = torch.tensor([O.data_ptr() for O in dm], dtype=torch.int64, device="cuda")
    ks = torch.tensor([4, 9], dtype=torch.int32, device="cuda")
    lds = torch.tensor([8, 18], dtype=torch.int32, device="cuda")
    out = torch.zeros(2 * cuda_lib.RESULT_BYTES, dtype=torch.uint8, device="cuda")
    ctx.batch_async(ptrs, ks, lds, out, prec="fp64")
    r = cuda_lib.results_from_tensor(out, 2)
    assert r[0].status == 0 and abs(r[0].value - (0.25) ** 4) < 1e-14
    assert r[1].status == cuda_lib.TOR_EINVAL


def test_batch_auto_mixes_tiers(ctx, cuda_lib):
    bright = gi.lossy_gbs_state(24, 1.6, 2.0, 0.9, 77)
    mats = [gi.select(bright.O, gi.random_pattern(24, 8, s)) for s in range(4)] + mats_uneven(n=8, k_lo=6, k_hi=12)
    dm = [torch.from_numpy(O).cuda() for O in mats]
    tol = 1e-8
    res = ctx.batch(dm, prec="auto", tol=tol)
    tiers = {r.tier for r in res}
    assert 1 in tiers and len(tiers) >= 2 and tiers <= {1, 2, 3, 4}
    for O, r in zip(mats, res):
        ref = oracle.tor(O)
        if r.status == cuda_lib.TOR_EPREC:
            continue
        assert r.status == 0
        assert err(r, ref) <= r.err_est <= tol * abs(ref.value) * (1 + 1e-9)


def test_batch_fixed_point_tier(ctx, cuda_lib):
    mats = mats_uneven(n=12, k_lo=1, k_hi=14) + [0.99 * np.eye(40)]   # the last: t_max = 10^40
    dm = [torch.from_numpy(O).cuda() for O in mats]
    res = ctx.batch(dm, prec="fx128")
    for O, r in zip(mats[:-1], res[:-1]):
        ref = oracle.tor(O)
        assert r.status == 0 and r.tier == 3
        assert err(r, ref) <= r.err_est
    assert res[-1].status == cuda_lib.TOR_EINVAL      # outside the fixed-point range: refused


def test_batch_fx256_tier_against_the_exact_oracle(ctx, cuda_lib):
    # explicit 256-bit batches, per-instance matrices and click patterns of one state; the
    # last instance (t_max = 10^40 > 2^26) lies outside the range and is refused
    st, pat, O32 = gi.workload_m100(32)
    ks = (0, 1, 3, 7, 11, 14)
    mats = [gi.select(st.O, pat[:k]) for k in ks] + [0.99 * np.eye(40)]
    res = ctx.batch([torch.from_numpy(O).cuda() for O in mats], prec="fx256")
    P = np.zeros((len(ks), 100), dtype=np.uint8)
    for row, k in enumerate(ks):
        P[row, pat[:k]] = 1
    res_p = ctx.batch_patterns(torch.from_numpy(st.O).cuda(), P, prec="fx256")
    for k, O, r, rp in zip(ks, mats, res, res_p):
        ref_t, ref_s = oracle.tor_exact(O)
        for x in (r, rp):
            assert x.status == 0 and x.tier == 4, (k, x)
            assert abs(Fraction(x.hi) + Fraction(x.lo) - ref_t) <= Fraction(x.err_est) + abs(ref_t) * Fraction(1, 2 ** 104)
            assert abs(x.sum_abs - float(ref_s)) <= 1e-15 * float(ref_s)
        assert (r.hi, r.lo) == (rp.hi, rp.lo)          # the same chunks, the same exact sums
    assert res[-1].status == cuda_lib.TOR_EINVAL


def test_batch_auto_reaches_256_bits(ctx, cuda_lib):
    # kappa grows with k: at tol = 1e-25 the FP64 and 128-bit tiers fall short and the
    # escalation has to end in the 256-bit tier; every result meets tol against the exact sum
    st, pat, O32 = gi.workload_m100(32)
    ks = (4, 10, 16, 20)
    mats = [gi.select(st.O, pat[:k]) for k in ks]
    tol = 1e-25
    res = ctx.batch([torch.from_numpy(O).cuda() for O in mats], prec="auto", tol=tol)
    assert 4 in {r.tier for r in res}
    for k, O, r in zip(ks, mats, res):
        ref_t, ref_s = oracle.tor_exact(O)
        assert r.status == 0, (k, r)
        e = abs(Fraction(r.hi) + Fraction(r.lo) - ref_t)
        assert e <= Fraction(r.err_est) + abs(ref_t) * Fraction(1, 2 ** 104)
        assert r.err_est <= tol * abs(float(ref_t))


def test_batch_auto_escalates_through_fixed_point(ctx, cuda_lib):
    st, pat, O32 = gi.workload_m100(32)
    mats = [gi.select(st.O, pat[:k]) for k in (6, 10, 14, 16)]
    dm = [torch.from_numpy(O).cuda() for O in mats]
    tol = 1e-12                                   # k = 16: kappa = 4e15, beyond FP64, within fixed point
    res = ctx.batch(dm, prec="auto", tol=tol)
    singles = [ctx.single(O, prec="auto", tol=tol) for O in dm]
    for O, r, s1 in zip(mats, res, singles):
        ref = oracle.tor(O)
        assert r.status == 0 and r.tier == s1.tier
        assert err(r, ref) <= r.err_est <= tol * abs(ref.value) * (1 + 1e-9)
    assert 3 in {r.tier for r in res}


def test_batch_in_cuda_graph_replays_with_new_inputs(ctx, cuda_lib):
    n, kmax = 24, 14
    ctx.batch_reserve(n, kmax)
    A = mats_uneven(seed=21, n=n, k_lo=2, k_hi=kmax)
    Bm = mats_uneven(seed=22, n=n, k_lo=2, k_hi=kmax)
    # fixed device buffers: each slot holds a 2 kmax x 2 kmax matrix; ld = 2 kmax
    slots = torch.zeros((n, 2 * kmax, 2 * kmax), dtype=torch.float64, device="cuda")
    ptrs = torch.tensor([slots[i].data_ptr() for i in range(n)], dtype=torch.int64, device="cuda")
    ks = torch.zeros(n, dtype=torch.int32, device="cuda")
    lds = torch.full((n,), 2 * kmax, dtype=torch.int32, device="cuda")
    out = torch.zeros(n * cuda_lib.RESULT_BYTES, dtype=torch.uint8, device="cuda")

    def load(mats):
        slots.zero_()
        for i, O in enumerate(mats):
            m = O.shape[0]
            slots[i, :m, :m] = torch.from_numpy(O)
        ks.copy_(torch.tensor([O.shape[0] // 2 for O in mats], dtype=torch.int32))

    load(A)
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        ctx.batch_async(ptrs, ks, lds, out, prec="fp64", stream=s)      # warm-up outside capture
    torch.cuda.current_stream().wait_stream(s)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        ctx.batch_async(ptrs, ks, lds, out, prec="fp64", stream=s)
    for mats in (A, Bm):
        load(mats)
        g.replay()
        torch.cuda.synchronize()
        res = cuda_lib.results_from_tensor(out, n)
        direct = ctx.batch([torch.from_numpy(O).cuda() for O in mats], prec="fp64")
        assert [(r.hi, r.lo) for r in res] == [(r.hi, r.lo) for r in direct]


def test_batches_accept_larger_k_after_small(cuda_lib):
    # without an explicit reservation a later, larger-k batch grows the workspace
    c = cuda_lib.Context(0)
    try:
        st, pat, O32 = gi.workload_m100(32)
        small = [torch.from_numpy(gi.select(st.O, pat[:6])).cuda() for _ in range(3)]
        big = [torch.from_numpy(gi.select(st.O, pat[:k])).cuda() for k in (14, 17, 9)]
        assert all(r.status == 0 for r in c.batch(small, prec="fp64"))
        res = c.batch(big, prec="fp64")
        for Od, r in zip(big, res):
            ref = c.single(Od, prec="fp64")
            assert r.status == 0
            assert abs(r.value - ref.value) <= r.err_est + ref.err_est
    finally:
        c.close()


def test_pattern_batches_accept_larger_k_after_small(ctx):
    # a first batch of few clicks must not limit a later batch of the same state
    st = gi.lossy_gbs_state(30, 0.6, 1.2, 0.3, 31)
    Od = torch.from_numpy(st.O).cuda()
    small = np.zeros((8, 30), dtype=np.uint8)
    small[:, :3] = 1
    big = np.zeros((4, 30), dtype=np.uint8)
    big[:, :18] = 1
    ctx.batch_patterns(Od, small, prec="fp64")
    res = ctx.batch_patterns(Od, big, prec="fp64")
    assert all(r.status == 0 for r in res)
    ref = ctx.single(torch.from_numpy(gi.select(st.O, np.arange(18))).cuda(), prec="fp64")
    assert abs(res[0].value - ref.value) <= res[0].err_est + ref.err_est


def test_plain_proposal_is_the_initial_network(ctx, cuda_lib):
    from paper_2009_01177_gb300.tor import pack_patterns
    M = 12
    marg = np.linspace(0.1, 0.6, M)
    net = cuda_lib.MLP(ctx, M, 64, seed=2)
    net.set_marginals(marg)
    X = (np.random.default_rng(1).random((64, M)) < 0.4).astype(np.float64)
    lq = net.logq(pack_patterns(X, M).cuda()).cpu().numpy()
    ref = (X * np.log(marg) + (1 - X) * np.log1p(-marg)).sum(1)
    assert np.allclose(lq, ref, atol=1e-5)
    net.close()
