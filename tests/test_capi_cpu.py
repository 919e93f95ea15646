"""CPU-only checks of the C ABI: the library builds, loads, and exports every
entry point include/torontonian.h declares; the binding declares the same set.
No compute call is made (there is no GPU here)."""
import ctypes
import os
import re

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
