"""CPU-only checks of the C ABI: the library builds, loads, and exports every
entry point include/torontonian.h declares; the binding declares the same set.
No compute call is made (there is no GPU here)."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "torontonian.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b((?:tor|gbs)_[a-z0-9_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    from paper_2009_01177_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("tor_single", "tor_batch", "tor_bounds", "gbs_sample_step", "tor_create",
                     "tor_destroy", "tor_last_error", "tor_chunks"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_declares_exactly_the_header(lib):
    from paper_2009_01177_gb300 import tor
    assert sorted(tor.SIGNATURES) == declared_functions()


def test_create_without_gpu_fails_cleanly(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_2009_01177_gb300 import tor
    tor.load_library()
    h = ctypes.c_void_p()
    rc = tor._lib.tor_create(ctypes.byref(h), 0)
    assert rc != tor.TOR_OK
    assert tor._lib.tor_last_error().decode()


def test_fixed_point_conversion_on_host(lib):
    # tor_fixed_to_result is pure host code: 3 * 2^128 -> 3.0; -0.5 -> (-0.5)
    from paper_2009_01177_gb300 import tor
    tor.load_library()
    three = [0, 0, 3, 0, 0, 0, 3, 0]
    r = tor.fixed_to_result(three, 5)
    assert (r.hi, r.lo, r.sum_abs) == (3.0, 0.0, 3.0)
    neg_half = (-(1 << 127)) & ((1 << 256) - 1)
    limbs = [(neg_half >> (64 * i)) & 0xFFFFFFFFFFFFFFFF for i in range(4)] + [0, 0, 1, 0]
    r = tor.fixed_to_result(limbs, 5)
    assert (r.hi, r.lo, r.sum_abs) == (-0.5, 0.0, 1.0)
    # hi + lo split of 1 + 2^-100
    v = (1 << 128) + (1 << 28)
    limbs = [(v >> (64 * i)) & 0xFFFFFFFFFFFFFFFF for i in range(4)] + [0, 0, 1, 0]
    r = tor.fixed_to_result(limbs, 5)
    assert (r.hi, r.lo) == (1.0, 2.0 ** -100)


def test_fixed_point_conversion_of_512_bit_partials(lib):
    # the 256-bit-class tier's partials: two 8-limb values with 256 fraction bits
    from paper_2009_01177_gb300 import tor
    tor.load_library()

    def limbs8(v):
        v &= (1 << 512) - 1
        return [(v >> (64 * i)) & 0xFFFFFFFFFFFFFFFF for i in range(8)]

    r = tor.fixed_to_result(limbs8(3 << 256) + limbs8(5 << 256), 7, "fx256")
    assert (r.hi, r.lo, r.sum_abs, r.tier) == (3.0, 0.0, 5.0, 4)
    # -(2^-100 + 2^-200): its low part lies far below the 128-bit tiers' resolution
    v = -((1 << 156) + (1 << 56))
    r = tor.fixed_to_result(limbs8(v) + limbs8(1 << 256), 7, "fx256")
    assert (r.hi, r.lo) == (-(2.0 ** -100), -(2.0 ** -200))
    # error model: 4k u sum_abs with u = 2^-196
    assert r.err_est == 4 * 7 * 2.0 ** -196 * 1.0
    with pytest.raises(ValueError):
        tor.fixed_to_result(limbs8(1) + limbs8(1), 7, "fp64")   # 16 limbs given, 8 expected


def test_shard_sums_of_512_bit_partials():
    from paper_2009_01177_gb300 import shard
    a = shard.ints_to_limbs(-(1 << 400), 1 << 400, limbs=16)
    b = shard.ints_to_limbs(3, 7, limbs=16)
    tot = shard.sum_partials(np.stack([a, b]))
    assert tot.shape == (16,)
    lo, hi = shard.limbs_to_ints(tot)
    assert lo == (3 - (1 << 400)) % (1 << 512) and hi == (1 << 400) + 7


@pytest.mark.parametrize("tier", ["fp64", "fx256"])
def test_library_sum_of_partials_is_the_big_integer_sum(lib, tier):
    # tor_sum_partials (host code) against Python integers: signed sums that wrap and carry
    # across every limb, both widths, n = 0 and n = 1
    import random
    from paper_2009_01177_gb300 import shard, tor
    tor.load_library()
    n_limbs = tor.partial_limbs(tier)
    L = n_limbs // 2
    rng = random.Random(11)
    rows, lo, hi = [], 0, 0
    for i in range(64):
        a = rng.getrandbits(64 * L) - (1 << (64 * L - 1)) if i % 3 else (1 << (64 * L)) - 1
        b = rng.getrandbits(64 * L - 8)
        rows.append(shard.ints_to_limbs(a, b, limbs=n_limbs))
        lo, hi = lo + a, hi + b
    got = tor.sum_partials(np.stack(rows), tier)
    assert np.array_equal(got, shard.ints_to_limbs(lo, hi, limbs=n_limbs))
    assert np.array_equal(tor.sum_partials(np.zeros((0, n_limbs), dtype=np.uint64), tier),
                          np.zeros(n_limbs, dtype=np.uint64))
    assert np.array_equal(tor.sum_partials(rows[5], tier), rows[5])


def test_library_sum_of_partials_refuses_bad_arguments(lib):
    from paper_2009_01177_gb300 import tor
    tor.load_library()
    L = tor._lib
    buf = (ctypes.c_uint64 * 16)()
    EINVAL = tor.TOR_EINVAL
    assert L.tor_sum_partials(None, 1, tor.PREC_FP64, buf) == EINVAL
    assert L.tor_sum_partials(buf, 1, tor.PREC_FP64, None) == EINVAL
    assert L.tor_sum_partials(buf, -1, tor.PREC_FP64, buf) == EINVAL
    assert L.tor_sum_partials(buf, 1, tor.PREC_FX256 + 1, buf) == EINVAL
    assert L.tor_sum_partials(buf, 1, tor.PREC_AUTO, buf) == EINVAL
    assert "tier" in tor._lib.tor_last_error().decode()


def test_bad_arguments_are_refused_before_any_device_call(lib):
    # every check below returns before the library touches CUDA, so it runs without a GPU
    from paper_2009_01177_gb300 import tor
    tor.load_library()
    L = tor._lib
    EINVAL = tor.TOR_EINVAL
    O = np.eye(6)                                    # host memory: never dereferenced here
    Op = O.ctypes.data_as(ctypes.c_void_p)
    res = tor.TorResultC()
    dummy = ctypes.c_void_p(O.ctypes.data)           # a non-null pointer for the output slots
    XXPP, XPXP = 0, 1
    hdr = open(HEADER).read()
    MAX_K = int(re.search(r"#define TOR_MAX_K (\d+)", hdr).group(1))
    LEVELS_MAX_K = int(re.search(r"#define TOR_LEVELS_MAX_K (\d+)", hdr).group(1))

    # context calls with a null context
    assert L.tor_single(None, Op, 3, 6, XXPP, tor.PREC_FP64, 0.0, None, ctypes.byref(res)) == EINVAL
    assert "null context" in L.tor_last_error().decode()
    assert L.tor_single_async(None, Op, 3, 6, XXPP, tor.PREC_FP64, None, dummy) == EINVAL
    assert L.tor_chunks(None, Op, 3, 6, XXPP, tor.PREC_FP64, 1, 0, 2, None, dummy) == EINVAL
    assert L.tor_all_patterns(None, Op, 3, 6, tor.PREC_FP64, None, dummy) == EINVAL
    assert L.tor_batch_reserve(None, 16, 8) == EINVAL

    # host-side conversion: null pointers and a tier that is not an explicit one
    limbs = (ctypes.c_uint64 * 12)()
    assert L.tor_fixed_to_result(None, 3, tor.PREC_FP64, ctypes.byref(res)) == EINVAL
    assert L.tor_fixed_to_result(limbs, 3, tor.PREC_FP64, None) == EINVAL
    assert L.tor_fixed_to_result(limbs, 3, tor.PREC_AUTO, ctypes.byref(res)) == EINVAL
    assert L.tor_fixed_to_result(limbs, 3, tor.PREC_FX256 + 1, ctypes.byref(res)) == EINVAL

    # the context-free single call
    fp64 = tor.PREC_FP64
    assert L.tor_single_noalloc(Op, MAX_K + 1, 2 * MAX_K + 2, XXPP, fp64, None, dummy) == EINVAL
    assert L.tor_single_noalloc(None, 3, 6, XXPP, fp64, None, dummy) == EINVAL
    assert L.tor_single_noalloc(Op, 3, 5, XXPP, fp64, None, dummy) == EINVAL
    assert "ld = 5 < 2k = 6" in L.tor_last_error().decode()
    assert L.tor_single_noalloc(Op, 3, 6, 7, fp64, None, dummy) == EINVAL
    assert L.tor_single_noalloc(Op, 3, 6, XPXP, tor.PREC_FX128, None, dummy) == EINVAL
    assert L.tor_single_noalloc(Op, 3, 6, XPXP, fp64, None, None) == EINVAL

    # the level scheduler: sizes, pointers, layout and per-level tiers
    ws = ctypes.c_void_p(O.ctypes.data)
    nbytes = ctypes.c_size_t()
    assert L.tor_levels_workspace(3, 0, None) == EINVAL
    assert L.tor_levels_workspace(LEVELS_MAX_K + 1, 0, ctypes.byref(nbytes)) == EINVAL
    assert L.tor_levels(Op, -1, 6, XXPP, fp64, None, ws, 1 << 20, None, dummy) == EINVAL
    assert L.tor_levels(Op, LEVELS_MAX_K + 1, 200, XXPP, fp64, None, ws, 1 << 20, None, dummy) == EINVAL
    assert L.tor_levels(None, 3, 6, XXPP, fp64, None, ws, 1 << 20, None, dummy) == EINVAL
    assert L.tor_levels(Op, 3, 6, XXPP, fp64, None, None, 1 << 20, None, dummy) == EINVAL
    assert L.tor_levels(Op, 3, 6, XXPP, fp64, None, ws, 1 << 20, None, None) == EINVAL
    assert L.tor_levels(Op, 3, 5, XXPP, fp64, None, ws, 1 << 20, None, dummy) == EINVAL
    assert L.tor_levels(Op, 3, 6, 2, fp64, None, ws, 1 << 20, None, dummy) == EINVAL
    for bad in (tor.PREC_AUTO, tor.PREC_FX256):
        tiers = (ctypes.c_int * 4)(fp64, fp64, bad, fp64)
        assert L.tor_levels(Op, 3, 6, XXPP, fp64, tiers, ws, 1 << 20, None, dummy) == EINVAL
        assert "level tiers" in L.tor_levels_last_error().decode()
    mask = ctypes.c_uint64()
    assert L.tor_level_kth_mask(3, 4, 0, ctypes.byref(mask)) == EINVAL
    assert L.tor_level_kth_mask(3, 1, 0, None) == EINVAL
    assert L.tor_level_kth_mask(3, 1, 3, ctypes.byref(mask)) == EINVAL   # C(3, 1) = 3 ranks

    # the 256-bit product helper
    assert L.tor_fx256_fma2(None, None, None, None, None, -1, None, None, None) == EINVAL
    assert L.tor_fx256_fma2(None, dummy, dummy, dummy, dummy, 1, dummy, dummy, None) == EINVAL
