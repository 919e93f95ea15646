"""GPU parity tests: the CUDA path (through the C ABI) against the CPU oracle.

Tolerances.  Each term t_Z is computed in the tier's arithmetic and summed
exactly, so the error of a result is bounded by gamma * u * sum_Z t_Z with
gamma = 4k, u = 2^-53 (FP64) or 2^-104 (double-double): every test asserts
|GPU - oracle| <= err_est.  Where the instance's condition number allows it,
tests also assert the relative targets 1e-10 (FP64) and 1e-20 (dd).
"""
from fractions import Fraction

import numpy as np
import pytest
import torch

import oracle
from paper_2009_01177_gb300 import gbs_inputs as gi

pytestmark = pytest.mark.gpu


def dev(O):
    return torch.from_numpy(np.ascontiguousarray(O)).to("cuda:0")


@pytest.fixture(scope="module")
def ctx(cuda_lib):
    c = cuda_lib.Context(0)
    yield c
    c.close()


def err_vs(r, ref):
    return abs(float(Fraction(r.hi) + Fraction(r.lo) - Fraction(ref.hi) - Fraction(ref.lo)))


TARGET = {"fp64": 1e-10, "dd": 1e-20}


def check(r, ref, prec):
    """|err| within the a-posteriori bound always; the relative target where kappa allows it."""
    e = err_vs(r, ref)
    assert r.status == 0
    assert e <= r.err_est, (e, r.err_est)
    if r.err_est <= TARGET[prec] * abs(ref.value):
        assert e <= TARGET[prec] * abs(ref.value), (e / abs(ref.value), ref.kappa)
    return e


def test_empty_pattern(ctx):
    r = ctx.single(torch.zeros((0, 0), dtype=torch.float64, device="cuda:0"), prec="fp64")
    assert (r.hi, r.lo, r.status) == (1.0, 0.0, 0)


@pytest.mark.parametrize("prec", ["fp64", "dd"])
@pytest.mark.parametrize("k", [1, 2, 3, 5, 8, 11, 13])
def test_thermal_closed_form(ctx, prec, k):
    # O = a I: Tor = (a/(1-a))^k exactly; kappa = ((2-a)/a)^k = 7^k at a = 1/4
    a = 0.25
    r = ctx.single(dev(gi.thermal_O(k, a)), prec=prec)
    exact = Fraction(1, 3) ** k
    got = Fraction(r.hi) + Fraction(r.lo)
    assert abs(float(got - exact)) <= r.err_est
    target = 1e-10 if prec == "fp64" else 1e-20
    if r.err_est <= target * float(exact):          # the conditioning allows the relative target
        assert abs(float((got - exact) / exact)) <= target


@pytest.mark.parametrize("prec", ["fp64", "dd"])
def test_m16_k10_against_oracle(ctx, prec):
    st, pat, O = gi.workload_m16_k10()
    ref = oracle.tor(O)
    r = ctx.single(dev(O), prec=prec)
    check(r, ref, prec)
    assert abs(r.sum_abs - ref.sum_abs) <= 1e-12 * ref.sum_abs
    if prec == "dd":                       # kappa = 1.7e8 leaves dd well inside 1e-20
        assert err_vs(r, ref) <= 1e-20 * abs(ref.value)


@pytest.mark.parametrize("prec", ["fp64", "dd"])
@pytest.mark.parametrize("k", [12, 14, 16])
def test_m100_nested_patterns_against_oracle(ctx, prec, k):
    st, pat, O32 = gi.workload_m100(32)
    O = gi.select(st.O, pat[:k])
    ref = oracle.tor(O)
    r = ctx.single(dev(O), prec=prec)
    check(r, ref, prec)


@pytest.mark.parametrize("prec", ["fp64", "dd"])
def test_well_conditioned_meets_relative_targets(ctx, prec):
    # bright modes: click probabilities near 1 make the sum well conditioned
    st = gi.lossy_gbs_state(24, 1.6, 2.0, 0.9, 77)
    O = gi.select(st.O, gi.random_pattern(24, 14, 77))
    ref = oracle.tor(O)
    r = ctx.single(dev(O), prec=prec)
    rel = err_vs(r, ref) / abs(ref.value)
    assert rel <= (1e-10 if prec == "fp64" else 1e-20), (rel, ref.kappa)


def test_chunk_partials_match_oracle_ranges(ctx):
    st, pat, O32 = gi.workload_m100(32)
    O = gi.select(st.O, pat[:14])
    k, d = 14, 5
    part = ctx.chunks(dev(O), d, 0, 1 << d, prec="fp64").cpu().numpy()
    from paper_2009_01177_gb300.tor import limbs_to_int
    for c in [0, 1, 7, 19, 31]:
        ref = oracle.tor_range(O, c << (k - d), (c + 1) << (k - d))
        got = Fraction(limbs_to_int(part[c, :4]), 1 << 128)
        sabs = Fraction(limbs_to_int(part[c, 4:]), 1 << 128)
        assert abs(float(sabs) - ref.sum_abs) <= 1e-13 * ref.sum_abs
        assert abs(float(got - Fraction(ref.hi) - Fraction(ref.lo))) <= 4 * k * 2.0 ** -53 * ref.sum_abs


def test_sharded_chunks_add_up_exactly(ctx):
    st, pat, O32 = gi.workload_m100(32)
    O = gi.select(st.O, pat[:18])
    Od = dev(O)
    d = 8
    whole = ctx.chunks(Od, d, 0, 1 << d, prec="fp64").cpu().numpy()
    a = ctx.chunks(Od, d, 0, 100, prec="fp64").cpu().numpy()
    b = ctx.chunks(Od, d, 100, 1 << d, prec="fp64").cpu().numpy()
    assert np.array_equal(np.concatenate([a, b]), whole)        # chunks are independent
    from paper_2009_01177_gb300.tor import limbs_to_int, fixed_to_result
    tot = [sum(limbs_to_int(whole[c, 4 * h:4 * h + 4]) for c in range(1 << d)) for h in (0, 1)]
    limbs = []
    for v in tot:
        v &= (1 << 256) - 1
        limbs += [(v >> (64 * i)) & 0xFFFFFFFFFFFFFFFF for i in range(4)]
    r_sh = fixed_to_result(limbs, 18)
    ctx.set_chunk_bits(d)
    r = ctx.single(Od, prec="fp64")
    ctx.set_chunk_bits(-1)
    assert (r_sh.hi, r_sh.lo) == (r.hi, r.lo)


_K32_CHUNK_REF = {}


@pytest.mark.parametrize("prec", ["fp64", "dd", "fx128", "fx256"])
def test_k32_sampled_chunks_at_bench_depth(ctx, prec):
    # the benchmark's instance at its autotuned chunk depth (d = 16: 2^16 chunks of 2^16
    # subsets): one chunk with none of the 16 fixed modes in Z and one with all of them
    # (64 x 64 determinants), each against the oracle's own mask range
    from paper_2009_01177_gb300.tor import limbs_to_int
    st, pat, O = gi.workload_m100(32)
    Od = dev(O)
    k, d = 32, 16
    u = {"fp64": 2.0 ** -53, "dd": 2.0 ** -104, "fx128": 2.0 ** -100, "fx256": 2.0 ** -196}[prec]
    for c in (0x0000, 0xFFFF):
        if c not in _K32_CHUNK_REF:
            _K32_CHUNK_REF[c] = oracle.tor_exact(O, c << (k - d), (c + 1) << (k - d))
        ref_t, ref_s = _K32_CHUNK_REF[c]
        part = ctx.chunks(Od, d, c, c + 1, prec=prec).cpu().numpy()[0]
        L = part.size // 2
        got = Fraction(limbs_to_int(part[:L]), 1 << (32 * L))
        sabs = Fraction(limbs_to_int(part[L:]), 1 << (32 * L))
        assert abs(sabs - ref_s) <= Fraction(1e-12) * ref_s, c
        assert abs(got - ref_t) <= 4 * k * Fraction(u) * ref_s + ref_s * Fraction(1, 2 ** 190), c


def test_launch_shape_does_not_change_bits(ctx):
    st, pat, O = gi.workload_m16_k10()
    O = gi.select(st.O, gi.random_pattern(16, 15, 3))
    Od = dev(O)
    base = ctx.single(Od, prec="fp64")
    for tpb, bps in [(32, 1), (64, 3), (128, 1)]:
        ctx.set_launch(tpb, bps)
        r = ctx.single(Od, prec="fp64")
        assert (r.hi, r.lo, r.sum_abs) == (base.hi, base.lo, base.sum_abs)
    ctx.set_launch(0, 0)


def test_chunk_depth_changes_only_rounding(ctx):
    st, pat, O32 = gi.workload_m100(32)
    O = gi.select(st.O, pat[:16])
    ref = oracle.tor(O)
    Od = dev(O)
    for d in [0, 3, 8, 16]:
        ctx.set_chunk_bits(d)
        r = ctx.single(Od, prec="fp64")
        assert err_vs(r, ref) <= r.err_est, d
    ctx.set_chunk_bits(-1)


def test_layouts_agree(ctx):
    st, pat, O = gi.workload_m16_k10()
    k = O.shape[0] // 2
    perm = np.empty(2 * k, dtype=int)
    perm[0::2] = np.arange(k)
    perm[1::2] = k + np.arange(k)
    Oi = O[np.ix_(perm, perm)]
    a = ctx.single(dev(O), layout="xxpp", prec="fp64")
    b = ctx.single(dev(Oi), layout="xpxp", prec="fp64")
    assert (a.hi, a.lo) == (b.hi, b.lo)


def test_leading_dimension(ctx):
    st, pat, O = gi.workload_m16_k10()
    big = np.zeros((O.shape[0], O.shape[1] + 7))
    big[:, :O.shape[1]] = O
    a = ctx.single(dev(O), prec="fp64")
    b = ctx.single(dev(big)[:, :O.shape[1]], prec="fp64")
    assert (a.hi, a.lo) == (b.hi, b.lo)


def test_not_positive_definite_is_reported(ctx, cuda_lib):
    O = 2.0 * np.eye(8)   # B = I - O = -I
    with pytest.raises(cuda_lib.TorError) as ei:
        ctx.single(dev(O), prec="fp64")
    assert ei.value.code == cuda_lib.TOR_ENOTPD


def test_invalid_arguments(ctx, cuda_lib):
    with pytest.raises(cuda_lib.TorError):
        ctx.set_launch(48, 1)
    with pytest.raises(cuda_lib.TorError):
        ctx.chunks(dev(np.zeros((8, 8))), 5, 0, 1, prec="fp64")   # chunk_bits > k


@pytest.mark.slow
def test_k32_block_factorisation(ctx):
    # full-size check at the resolving tier: Tor(O1 (+) O2) = Tor(O1) Tor(O2) with 16 + 16 modes
    # of the M = 100 state (the 2^32 subsets factorise over the two blocks), against the
    # product of the oracle's exact k = 16 sums.  kappa of the product is about 1e31, so the
    # 256-bit tier's bound has to resolve it to 1e-20 relative for the check to mean anything.
    st, pat, O32 = gi.workload_m100(32)
    O1 = gi.select(st.O, pat[:16])
    O2 = gi.select(st.O, pat[16:])
    (t1, s1), (t2, s2) = oracle.tor_exact(O1), oracle.tor_exact(O2)
    prod, sprod = t1 * t2, s1 * s2
    r = ctx.single(dev(gi.block_diag_modes(O1, O2)), prec="fx256")
    assert r.status == 0 and r.tier == 4
    got = Fraction(r.hi) + Fraction(r.lo)
    # both halves' exact sums carry the oracle's own rounding, far below 2^-188 of their sums of terms
    assert abs(got - prod) <= Fraction(r.err_est) + sprod * Fraction(1, 2 ** 188) + abs(prod) * Fraction(1, 2 ** 104)
    assert r.err_est <= 1e-20 * abs(float(prod))
    assert abs(got - prod) <= Fraction(1, 10 ** 20) * abs(prod)
    assert abs(r.sum_abs - float(sprod)) <= 1e-12 * float(sprod)


def test_autotune_picks_and_caches(ctx, tmp_path):
    cache = str(tmp_path / "tune.jsonl")
    st, pat, O32 = gi.workload_m100(32)
    O = gi.select(st.O, pat[:20])
    before = ctx.single(dev(O), prec="fp64")
    d, bps = ctx.autotune(20, "fp64", cache)
    assert 0 <= d <= 20 and 1 <= bps <= 4
    lines = open(cache).read().strip().splitlines()
    assert len(lines) == 1 and '"k": 20' in lines[0]
    assert ctx.autotune(20, "fp64", cache) == (d, bps)           # served from the cache
    assert len(open(cache).read().strip().splitlines()) == 1
    after = ctx.single(dev(O), prec="fp64")
    assert abs(after.value - before.value) <= after.err_est + before.err_est
    assert after.sum_abs == pytest.approx(before.sum_abs, rel=1e-12)


def test_shard_ranges_gather_to_the_single_result(ctx):
    from paper_2009_01177_gb300 import shard
    from paper_2009_01177_gb300.tor import fixed_to_result
    st, pat, O32 = gi.workload_m100(32)
    O = gi.select(st.O, pat[:18])
    Od = dev(O)
    d, world = 8, 3
    parts = []
    for r in range(world):
        lo, hi = shard.chunk_range(r, world, 1 << d)
        parts.append(shard.sum_partials(ctx.chunks(Od, d, lo, hi, prec="fp64").cpu().numpy().view(np.uint64)))
    total = shard.sum_partials(np.stack(parts))
    r_sh = fixed_to_result([int(x) for x in total], 18)
    ctx.set_chunk_bits(d)
    r = ctx.single(Od, prec="fp64")
    ctx.set_chunk_bits(-1)
    assert (r_sh.hi, r_sh.lo, r_sh.sum_abs) == (r.hi, r.lo, r.sum_abs)


@pytest.mark.parametrize("prec", ["fp64", "dd"])
def test_tail_split_matches_the_unsplit_chunk_sum(ctx, prec):
    # 2^18 chunks on the default grid leave a partial last round, which
    # tor_single cuts into finer sub-chunks: the same subsets, other rounding
    from paper_2009_01177_gb300 import shard
    from paper_2009_01177_gb300.tor import fixed_to_result
    st, pat, O32 = gi.workload_m100(32)
    k, d = 22, 18
    Od = dev(gi.select(st.O, pat[:k]))
    tot = shard.sum_partials(ctx.chunks(Od, d, 0, 1 << d, prec=prec).cpu().numpy().view(np.uint64))
    r_chunks = fixed_to_result([int(x) for x in tot], k, prec)
    ctx.set_chunk_bits(d)
    r = ctx.single(Od, prec=prec)
    ctx.set_chunk_bits(-1)
    assert r.status == 0
    # a missing or doubled sub-chunk would move sum_abs by about 2^-18 of itself
    assert abs(r.sum_abs - r_chunks.sum_abs) <= 1e-12 * r.sum_abs
    diff = abs((Fraction(r.hi) + Fraction(r.lo)) - (Fraction(r_chunks.hi) + Fraction(r_chunks.lo)))
    assert float(diff) <= r.err_est + r_chunks.err_est


# ------------------------------------------------------- 128-bit fixed point
@pytest.mark.parametrize("k", [1, 4, 9, 13])
def test_fx128_thermal_closed_form(ctx, k):
    r = ctx.single(dev(gi.thermal_O(k, 0.25)), prec="fx128")
    exact = Fraction(1, 3) ** k
    got = Fraction(r.hi) + Fraction(r.lo)
    assert r.tier == 3
    assert abs(float(got - exact)) <= r.err_est
    assert r.err_est <= 1e-16 * float(exact)     # kappa = (7/3)^k / (1/3)^k = 7^k at most 1e11 here


@pytest.mark.parametrize("k", [10, 14, 16, 20])
def test_fx128_against_oracle(ctx, k):
    st, pat, O32 = gi.workload_m100(32)
    O = gi.select(st.O, pat[:k])
    ref = oracle.tor(O)
    r = ctx.single(dev(O), prec="fx128")
    e = err_vs(r, ref)
    assert r.status == 0 and e <= r.err_est
    # absolute truncation 2^-104 per product: measured errors sit near 2^-110 sum_Z t_Z
    assert e <= 2.0 ** -100 * r.sum_abs
    check(r, ref, "dd")                           # the 1e-20 target wherever the bound allows it


def test_fx128_agrees_with_double_double_at_k32(ctx):
    st, pat, O = gi.workload_m100(32)         # t_max = 2^8.3: 1/det2 up to 2^16.6, inside the range
    Od = dev(O)
    fx = ctx.single(Od, prec="fx128")
    dd = ctx.single(Od, prec="dd")
    assert fx.status == 0 and fx.tier == 3
    diff = abs((Fraction(fx.hi) + Fraction(fx.lo)) - (Fraction(dd.hi) + Fraction(dd.lo)))
    assert float(diff) <= fx.err_est + dd.err_est
    assert float(diff) <= 2.0 ** -100 * fx.sum_abs  # two independent ~104-bit evaluations agree


def test_fx128_chunks_add_to_single(ctx):
    st, pat, O32 = gi.workload_m100(32)
    O = gi.select(st.O, pat[:16])
    Od = dev(O)
    from paper_2009_01177_gb300 import shard
    from paper_2009_01177_gb300.tor import fixed_to_result
    tot = shard.sum_partials(ctx.chunks(Od, 6, 0, 64, prec="fx128").cpu().numpy().view(np.uint64))
    r_sh = fixed_to_result([int(x) for x in tot], 16, "fx128")
    ctx.set_chunk_bits(6)
    r = ctx.single(Od, prec="fx128")
    ctx.set_chunk_bits(-1)
    assert (r_sh.hi, r_sh.lo) == (r.hi, r.lo)


def test_fx128_rejects_out_of_range(ctx, cuda_lib):
    O = 0.99 * np.eye(40)      # t_max = 0.01^-20: beyond the fixed-point range
    with pytest.raises(cuda_lib.TorError) as ei:
        ctx.single(dev(O), prec="fx128")
    assert ei.value.code == cuda_lib.TOR_EINVAL


# ------------------------------------------------------- 256-bit fixed point
def _fx9_value(limbs):
    return sum(int(x) << (29 * i) for i, x in enumerate(limbs))


def _fx9_balanced(R: int):
    """R (units of 2^-203) as nine balanced 29-bit limbs, and whether it does not fit."""
    out = []
    for _ in range(9):
        m = ((R + (1 << 28)) % (1 << 29)) - (1 << 28)
        out.append(m)
        R = (R - m) >> 29
    return out, R != 0


def _fx9_fma2_reference(s, a1, b1, a2, b2):
    """The 256-bit-class tier's fused s + a1 b1 + a2 b2 restated on Python integers: the limb
    products a_i b_j with i + j >= 6 (units of 2^-406) and s, rounded to nearest at 2^-203 with
    ties up, then split into balanced limbs (overflow when nine do not hold it)."""
    X = _fx9_value(s) << 203
    for a, b in ((a1, b1), (a2, b2)):
        for i in range(9):
            for j in range(9):
                if i + j >= 6:
                    X += int(a[i]) * int(b[j]) << (29 * (i + j))
    return _fx9_balanced((X + (1 << 202)) >> 203)


def test_fx256_fma2_matches_big_integer_definition(cuda_lib):
    rng = np.random.default_rng(5)
    n = 3000
    ops = []
    for _ in range(5):
        arr = np.zeros((n, 9), dtype=np.int64)
        for r in range(n):
            top = int(rng.integers(0, 10))           # limbs from `top` up are zero
            lim = (1 << 28) if rng.random() < 0.8 else (1 << 29) - 1   # balanced, or any below 2^29
            arr[r, :top] = rng.integers(-lim, lim, size=top)
        ops.append(arr)
    ops[0][:8] = 0
    ops[1][:8] = [[0] * 8 + [(1 << 28) - 1]] * 8      # largest products: overflow expected
    out, ovf = cuda_lib.fx256_fma2(*[torch.from_numpy(a.astype(np.int32)).cuda() for a in ops])
    out, ovf = out.cpu().numpy(), ovf.cpu().numpy()
    checked = 0
    for r in range(n):
        s, a1, b1, a2, b2 = (a[r] for a in ops)
        ref, ref_ovf = _fx9_fma2_reference(s, a1, b1, a2, b2)
        assert bool(ovf[r]) == ref_ovf, r
        if ref_ovf:
            continue
        # the value exactly (its limbs may split it differently), limbs within the stated range
        assert _fx9_value(out[r]) == _fx9_value(ref), r
        assert np.all(np.abs(out[r]) <= (1 << 28)), r
        # against the exact value: off by the rounding (half a unit of 2^-203) and the unformed
        # columns i + j < 6 at most; with balanced limbs that is 1.5 units per product
        exact = Fraction(_fx9_value(s)) + Fraction(_fx9_value(a1) * _fx9_value(b1) + _fx9_value(a2) * _fx9_value(b2),
                                                   1 << 203)
        dropped = sum(abs(int(a[i]) * int(b[j])) << (29 * (i + j))
                      for a, b in ((a1, b1), (a2, b2)) for i in range(9) for j in range(9) if i + j < 6)
        assert abs(_fx9_value(ref) - exact) <= Fraction(1, 2) + Fraction(dropped, 1 << 203)
        if max(abs(int(x)) for x in np.concatenate([a1, b1, a2, b2])) <= (1 << 28):
            assert abs(_fx9_value(ref) - exact) <= Fraction(7, 2)
        checked += 1
    assert checked > 2500


def _fx256_chunk_total(ctx, Od, k, d):
    from paper_2009_01177_gb300 import shard
    part = ctx.chunks(Od, d, 0, 1 << d, prec="fx256").cpu().numpy().view(np.uint64)
    lo, hi = shard.limbs_to_ints(shard.sum_partials(part))
    sgn = lambda v: v - (1 << 512) if v >> 511 else v
    return Fraction(sgn(lo), 1 << 256), Fraction(hi, 1 << 256)


@pytest.mark.parametrize("k", [1, 4, 9, 13])
def test_fx256_thermal_closed_form(ctx, k):
    Od = dev(gi.thermal_O(k, 0.25))
    tor_x, sabs_x = _fx256_chunk_total(ctx, Od, k, min(k, 3))
    bound = 4 * k * Fraction(1, 2 ** 196) * sabs_x
    assert abs(tor_x - Fraction(1, 3) ** k) <= bound
    r = ctx.single(Od, prec="fx256")
    assert r.tier == 4 and r.status == 0
    assert abs(Fraction(r.hi) + Fraction(r.lo) - Fraction(1, 3) ** k) <= Fraction(r.err_est) + Fraction(1, 3) ** k * Fraction(1, 2 ** 104)


@pytest.mark.parametrize("k", [8, 12, 15])
def test_fx256_against_the_exact_oracle(ctx, k):
    st, pat, O32 = gi.workload_m100(32)
    O = gi.select(st.O, pat[:k])
    ref_t, ref_s = oracle.tor_exact(O)
    got_t, got_s = _fx256_chunk_total(ctx, dev(O), k, 4)
    # both sides: a few units of 2^-203 / 2^-200 per term; the GPU bound 4k 2^-196 sum t covers both
    assert abs(got_t - ref_t) <= 4 * k * Fraction(1, 2 ** 196) * ref_s
    # the sum of terms keeps the terms' bits from 2^-58 up only
    assert abs(got_s - ref_s) <= Fraction(1, 2 ** 52) * ref_s
    # kappa up to 1e16 here: the relative error stays near 2^-196 kappa, far below 1e-20
    assert abs((got_t - ref_t) / ref_t) < 1e-20


def test_auto_routes_beyond_double_double_to_256_bits(ctx):
    # k = 20 of the M = 100 state: kappa = 1.2e19, so tol = 1e-25 needs about 150 bits
    st, pat, O32 = gi.workload_m100(32)
    O = gi.select(st.O, pat[:20])
    ref_t, ref_s = oracle.tor_exact(O)
    r = ctx.single(dev(O), prec="auto", tol=1e-25)
    assert r.tier == 4 and r.status == 0
    err = abs(Fraction(r.hi) + Fraction(r.lo) - ref_t)
    assert err <= Fraction(r.err_est) + abs(ref_t) * Fraction(1, 2 ** 104)
    assert r.err_est <= 1e-25 * abs(float(ref_t))


def test_fx256_rejects_out_of_range(ctx, cuda_lib):
    O = 0.99 * np.eye(40)      # t_max = 10^40 > 2^26
    with pytest.raises(cuda_lib.TorError) as ei:
        ctx.single(dev(O), prec="fx256")
    assert ei.value.code == cuda_lib.TOR_EINVAL


@pytest.mark.parametrize("prec", ["fp64", "fx256"])
def test_long_run_cancel_and_resume(ctx, prec, tmp_path):
    # windows of tor_chunks with a checkpoint: stopped after three windows, resumed, and
    # bit-identical to the partials summed in one go
    from paper_2009_01177_gb300 import longrun, shard
    from paper_2009_01177_gb300.tor import fixed_to_result
    st_, pat, O32 = gi.workload_m100(32)
    k, d, window = 20, 12, 512
    Od = dev(gi.select(st_.O, pat[:k]))
    ck = str(tmp_path / "long.npz")
    stops = iter([False, False, False, True])
    r0, s0 = longrun.tor_long(ctx, Od, prec, d, window, ck, should_stop=lambda: next(stops, True))
    assert r0 is None and s0.done.sum() == 3
    r1, s1 = longrun.tor_long(ctx, Od, prec, d, window, ck)
    assert s1.complete
    whole = shard.sum_partials(ctx.chunks(Od, d, 0, 1 << d, prec=prec).cpu().numpy().view(np.uint64))
    assert np.array_equal(s1.total, whole)
    ref = fixed_to_result([int(x) for x in whole], k, prec)
    assert (r1.hi, r1.lo, r1.sum_abs) == (ref.hi, ref.lo, ref.sum_abs)


@pytest.mark.parametrize("prec", ["fp64", "fx256"])
def test_maximum_k_sampled_chunk(ctx, prec):
    # k = 64 (TOR_MAX_K, a 128 x 128 matrix): one chunk of 4096 subsets at d = 52 whose six
    # fixed modes in Z include the highest one (masks above 2^63), against the oracle's exact range
    from paper_2009_01177_gb300.tor import limbs_to_int
    st, pat, O = gi.workload_m100(64)
    k, d = 64, 52
    c = (1 << 51) | (1 << 30) | 0xF
    ref_t, ref_s = oracle.tor_exact(O, c << (k - d), (c + 1) << (k - d))
    part = ctx.chunks(dev(O), d, c, c + 1, prec=prec).cpu().numpy()[0]
    L = part.size // 2
    got = Fraction(limbs_to_int(part[:L]), 1 << (32 * L))
    sabs = Fraction(limbs_to_int(part[L:]), 1 << (32 * L))
    u = {"fp64": 2.0 ** -53, "fx256": 2.0 ** -196}[prec]
    assert abs(sabs - ref_s) <= Fraction(1e-12) * ref_s
    assert abs(got - ref_t) <= 4 * k * Fraction(u) * ref_s + ref_s * Fraction(1, 2 ** 190)


@pytest.mark.parametrize("k", [40, 50])
def test_adaptive_instances_sampled_chunks_at_bench_depth(ctx, k):
    # the adaptive-precision workload (M = 100, r ~ U[0.8, 1.4], eta = 0.3, seed 3; nested
    # patterns of k = 40 and 50 clicks, pattern seed 1003) at the depth the bench's 256-bit
    # windows walk (17 walked modes per chunk): the chunk whose only fixed mode in Z is the
    # highest, and one with every other fixed mode in Z, against the oracle's mask ranges
    from paper_2009_01177_gb300.tor import limbs_to_int
    st = gi.lossy_gbs_state(100, 0.8, 1.4, 0.3, 3)
    pat = gi.random_pattern(100, 50, 1003)
    O = gi.select(st.O, pat[:k])
    r1 = 17
    d = k - r1
    for c in (1 << (d - 1), 0x5555555555555555 & ((1 << d) - 1)):
        ref_t, ref_s = oracle.tor_exact(O, c << r1, (c + 1) << r1)
        part = ctx.chunks(dev(O), d, c, c + 1, prec="fx256").cpu().numpy()[0]
        L = part.size // 2
        got = Fraction(limbs_to_int(part[:L]), 1 << (32 * L))
        sabs = Fraction(limbs_to_int(part[L:]), 1 << (32 * L))
        assert abs(sabs - ref_s) <= Fraction(1e-12) * ref_s, c
        assert abs(got - ref_t) <= 4 * k * Fraction(2.0 ** -196) * ref_s + ref_s * Fraction(1, 2 ** 190), c


def test_chunk_depth_above_the_old_limit_and_k_limits(ctx, cuda_lib):
    st, pat, O = gi.workload_m100(64)
    Od = dev(O)
    ctx.chunks(Od, 63, 5, 6, prec="fp64")                         # d = 63: a chunk of two subsets
    with pytest.raises(cuda_lib.TorError):
        ctx.chunks(Od, 64, 0, 1, prec="fp64")                     # d = k = 64 is beyond 63
    with pytest.raises(cuda_lib.TorError):
        ctx.single(dev(np.zeros((130, 130))), prec="fp64")        # k = 65 > TOR_MAX_K
