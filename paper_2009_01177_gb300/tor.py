"""Python binding of the C ABI in include/torontonian.h (argument marshalling only).

Every step of the Torontonian runs in the CUDA library libtorontonian.so; this
module converts torch tensors to device pointers and streams, and results to
Python objects.  There is no CPU fallback: if the library is missing or no
GPU is present, the calls raise.
"""
from __future__ import annotations

import ctypes
import dataclasses
import os
import threading

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libtorontonian.so")

TOR_OK, TOR_EINVAL, TOR_ENOTPD, TOR_ECUDA, TOR_ETIMEOUT, TOR_EPREC, TOR_ENOMEM = range(7)
PREC_AUTO, PREC_FP64, PREC_DD, PREC_FX128, PREC_FX256 = 0, 1, 2, 3, 4
LAYOUT_XXPP, LAYOUT_XPXP = 0, 1
_PREC = {"auto": PREC_AUTO, "fp64": PREC_FP64, "dd": PREC_DD, "fx128": PREC_FX128, "fx256": PREC_FX256}


def partial_limbs(prec: str) -> int:
    """64-bit limbs of one chunk partial: two 256-bit sums (128 fraction bits), or two 512-bit
    sums (256 fraction bits) for fx256."""
    return 16 if prec == "fx256" else 8
_LAYOUT = {"xxpp": LAYOUT_XXPP, "xpxp": LAYOUT_XPXP}


class TorResultC(ctypes.Structure):
    _fields_ = [("hi", ctypes.c_double), ("lo", ctypes.c_double), ("sum_abs", ctypes.c_double),
                ("err_est", ctypes.c_double), ("tier", ctypes.c_int), ("status", ctypes.c_int)]


class TorBoundC(ctypes.Structure):
    _fields_ = [("log_tmax", ctypes.c_float), ("log_tor_est", ctypes.c_float),
                ("log_kappa_est", ctypes.c_float), ("bits_needed", ctypes.c_float),
                ("tier", ctypes.c_int)]


RESULT_BYTES = ctypes.sizeof(TorResultC)
BOUND_BYTES = ctypes.sizeof(TorBoundC)


class TorError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"[{code}] {msg}")
        self.code = code


@dataclasses.dataclass
class TorResult:
    hi: float
    lo: float
    sum_abs: float
    err_est: float
    tier: int
    status: int

    @property
    def value(self) -> float:
        return self.hi + self.lo

    @property
    def kappa(self) -> float:
        return self.sum_abs / abs(self.hi) if self.hi else float("inf")

    @classmethod
    def from_c(cls, r: TorResultC) -> "TorResult":
        return cls(r.hi, r.lo, r.sum_abs, r.err_est, r.tier, r.status)

    @classmethod
    def from_bytes(cls, b: bytes) -> "TorResult":
        return cls.from_c(TorResultC.from_buffer_copy(b))


_lib = None
_lock = threading.Lock()

# name -> (restype, argtypes); the same names as include/torontonian.h
_VP, _I, _D, _U64 = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_uint64
SIGNATURES = {
    "tor_create": (_I, [ctypes.POINTER(_VP), _I]),
    "tor_destroy": (None, [_VP]),
    "tor_last_error": (ctypes.c_char_p, []),
    "tor_set_launch": (_I, [_VP, _I, _I]),
    "tor_set_chunk_bits": (_I, [_VP, _I]),
    "tor_single": (_I, [_VP, _VP, _I, _I, _I, _I, _D, _VP, ctypes.POINTER(TorResultC)]),
    "tor_single_async": (_I, [_VP, _VP, _I, _I, _I, _I, _VP, _VP]),
    "tor_chunks": (_I, [_VP, _VP, _I, _I, _I, _I, _I, _U64, _U64, _VP, _VP]),
    "tor_fixed_to_result": (_I, [ctypes.POINTER(_U64), _I, _I, ctypes.POINTER(TorResultC)]),
    "tor_sum_partials": (_I, [ctypes.POINTER(_U64), _I, _I, ctypes.POINTER(_U64)]),
    "tor_fx256_fma2": (_I, [_VP, _VP, _VP, _VP, _VP, _I, _VP, _VP, _VP]),
    "tor_levels_workspace": (_I, [_I, _I, ctypes.POINTER(ctypes.c_size_t)]),
    "tor_levels": (_I, [_VP, _I, _I, _I, _I, ctypes.POINTER(_I), _VP, ctypes.c_size_t, _VP, _VP]),
    "tor_levels_last_error": (ctypes.c_char_p, []),
    "tor_level_next_mask": (_U64, [_U64]),
    "tor_level_kth_mask": (_I, [_I, _I, _U64, ctypes.POINTER(_U64)]),
    "tor_all_patterns": (_I, [_VP, _VP, _I, _I, _I, _VP, _VP]),
    "tor_batch": (_I, [_VP, _VP, _VP, _VP, _I, _I, _I, _D, _VP, _VP]),
    "tor_bounds": (_I, [_VP, _VP, _VP, _VP, _I, _I, _D, _VP, _VP]),
    "tor_batch_reserve": (_I, [_VP, _I, _I]),
    "tor_batch_patterns": (_I, [_VP, _VP, _I, _I, _VP, _I, _I, _D, _VP, _VP]),
    "tor_fp64_peak": (_I, [_VP, ctypes.POINTER(_D), ctypes.POINTER(_D)]),
    "tor_int_peak": (_I, [_VP, ctypes.POINTER(_D)]),
    "tor_single_noalloc": (_I, [_VP, _I, _I, _I, _I, _VP, _VP]),
    "tor_mlp_create": (_I, [_VP, _I, _I, _U64, ctypes.POINTER(_VP)]),
    "tor_mlp_destroy": (None, [_VP]),
    "tor_mlp_num_params": (_I, [_VP]),
    "tor_mlp_get_params": (_I, [_VP, ctypes.POINTER(ctypes.c_float), _I]),
    "tor_mlp_set_params": (_I, [_VP, ctypes.POINTER(ctypes.c_float)]),
    "tor_mlp_set_marginals": (_I, [_VP, ctypes.POINTER(_D)]),
    "tor_mlp_logq": (_I, [_VP, _VP, _I, _VP, _VP]),
    "tor_mlp_logits": (_I, [_VP, _VP, _I, ctypes.POINTER(ctypes.c_float)]),
    "tor_mlp_grad": (_I, [_VP, _VP, _VP, _I, ctypes.POINTER(ctypes.c_float), _VP]),
    "tor_mlp_train_step": (_I, [_VP, _VP, _VP, _I, ctypes.c_float, ctypes.POINTER(ctypes.c_float), _VP]),
    "tor_mlp_sample": (_I, [_VP, _I, _U64, _U64, _VP, _VP, _VP]),
    "gbs_sample_step": (_I, [_VP, _VP, _I, _I, _D, _VP, _VP, _I, _VP, _VP, _VP, _VP, _U64, _U64, _I, _D, _I,
                             _VP]),
    "gbs_sample_step_da": (_I, [_VP, _VP, _I, _I, _D, _VP, _VP, _I, _VP, _VP, _VP, _VP, _VP, _U64, _U64, _I,
                                _D, _I, _VP]),
    "tor_autotune": (_I, [_VP, _I, _I, ctypes.c_char_p, ctypes.POINTER(_I), ctypes.POINTER(_I)]),
    "tor_set_timing": (_I, [_VP, _I]),
    "tor_walk_time": (_I, [_VP, ctypes.POINTER(ctypes.c_float)]),
    "tor_transform_time": (_I, [_VP, ctypes.POINTER(ctypes.c_float)]),
}


def load_library(path: str = LIB_PATH):
    """Load libtorontonian.so and declare every exported entry point."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(path):
                raise RuntimeError(f"{path} is missing: build it first "
                                   "(python -c 'import __graft_entry__ as g; g.build()')")
            lib = ctypes.CDLL(path)
            for name, (res, args) in SIGNATURES.items():
                f = getattr(lib, name)
                f.restype = res
                f.argtypes = args
            _lib = lib
    return _lib


def _check(rc: int):
    if rc != TOR_OK:
        raise TorError(rc, load_library().tor_last_error().decode())


def _stream(stream) -> int:
    if stream is None:
        return torch.cuda.current_stream().cuda_stream
    return getattr(stream, "cuda_stream", stream)


def _mat(O: torch.Tensor):
    if not (isinstance(O, torch.Tensor) and O.is_cuda and O.dtype == torch.float64 and O.dim() == 2):
        raise ValueError("O must be a 2-D float64 CUDA tensor")
    if O.shape[0] != O.shape[1] or O.shape[0] % 2:
        raise ValueError("O must be 2k x 2k")
    if O.shape[0] == 0:
        return 0, 1
    if O.stride(1) != 1:
        raise ValueError("O must be row-major (unit column stride)")
    return O.shape[0] // 2, O.stride(0)


def pack_patterns(patterns, M: int) -> torch.Tensor:
    """(n, M) 0/1 array-like -> int64 tensor (n, ceil(M/64)) of bitsets (bit j = mode j)."""
    import numpy as np
    a = np.asarray(patterns, dtype=np.uint8).reshape(-1, M)
    words = (M + 63) // 64
    out = np.zeros((a.shape[0], words), dtype=np.uint64)
    for j in range(M):
        out[:, j // 64] |= a[:, j].astype(np.uint64) << np.uint64(j % 64)
    return torch.from_numpy(out.view(np.int64))


RESULT_DTYPE = [("hi", "<f8"), ("lo", "<f8"), ("sum_abs", "<f8"), ("err_est", "<f8"), ("tier", "<i4"),
                ("status", "<i4")]


def results_array(out: torch.Tensor, n: int):
    """The n tor_result records of a uint8 CUDA tensor as a numpy structured array."""
    import numpy as np
    return np.frombuffer(out[:n * RESULT_BYTES].cpu().numpy().tobytes(), dtype=np.dtype(RESULT_DTYPE))


def results_from_tensor(out: torch.Tensor, n: int):
    raw = out.cpu().numpy().tobytes()
    return [TorResult.from_bytes(raw[i * RESULT_BYTES:(i + 1) * RESULT_BYTES]) for i in range(n)]


class Context:
    """A library context on one CUDA device (workspace, launch settings)."""

    def __init__(self, device: int = 0):
        self.lib = load_library()
        self.device = device
        h = ctypes.c_void_p()
        _check(self.lib.tor_create(ctypes.byref(h), device))
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            self.lib.tor_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_launch(self, threads_per_block: int = 0, blocks_per_sm: int = 0):
        _check(self.lib.tor_set_launch(self.h, threads_per_block, blocks_per_sm))

    def set_chunk_bits(self, d: int):
        _check(self.lib.tor_set_chunk_bits(self.h, d))

    def single(self, O: torch.Tensor, prec: str = "auto", layout: str = "xxpp", tol: float = 1e-10,
               stream=None) -> TorResult:
        """Tor(O) of one 2k x 2k matrix (blocking)."""
        k, ld = _mat(O)
        out = TorResultC()
        _check(self.lib.tor_single(self.h, O.data_ptr(), k, ld, _LAYOUT[layout], _PREC[prec], tol,
                                   _stream(stream), ctypes.byref(out)))
        return TorResult.from_c(out)

    def single_async(self, O: torch.Tensor, out: torch.Tensor, prec: str,
                     layout: str = "xxpp", stream=None):
        """Enqueue Tor(O); the raw tor_result lands in the uint8 CUDA tensor `out`."""
        k, ld = _mat(O)
        if out.dtype != torch.uint8 or out.numel() < RESULT_BYTES or not out.is_cuda:
            raise ValueError(f"out must be a uint8 CUDA tensor of >= {RESULT_BYTES} bytes")
        _check(self.lib.tor_single_async(self.h, O.data_ptr(), k, ld, _LAYOUT[layout], _PREC[prec],
                                         _stream(stream), out.data_ptr()))

    def chunks(self, O: torch.Tensor, chunk_bits: int, c_begin: int, c_end: int, prec: str,
               layout: str = "xxpp", stream=None) -> torch.Tensor:
        """Exact per-chunk partials, an int64 CUDA tensor (c_end - c_begin, 8) of raw limbs
        ((c_end - c_begin, 16) for fx256)."""
        k, ld = _mat(O)
        part = torch.zeros((max(c_end - c_begin, 0), partial_limbs(prec)), dtype=torch.int64, device=O.device)
        _check(self.lib.tor_chunks(self.h, O.data_ptr(), k, ld, _LAYOUT[layout], _PREC[prec],
                                   chunk_bits, c_begin, c_end, _stream(stream), part.data_ptr()))
        return part

    def all_patterns_async(self, Ofull: torch.Tensor, out: torch.Tensor, prec: str = "fp64", stream=None):
        """tor_all_patterns: out is a uint8 CUDA tensor of 2^M * RESULT_BYTES."""
        M, ld = _mat(Ofull)
        if out.numel() < (1 << M) * RESULT_BYTES:
            raise ValueError("out too small")
        _check(self.lib.tor_all_patterns(self.h, Ofull.data_ptr(), M, ld, _PREC[prec], _stream(stream),
                                         out.data_ptr()))

    def all_patterns(self, Ofull: torch.Tensor, prec: str = "fp64"):
        """Tor(O_S) of every pattern S of the M-mode state (index = mask); a numpy structured array."""
        M = Ofull.shape[0] // 2
        out = torch.zeros((1 << M) * RESULT_BYTES, dtype=torch.uint8, device=Ofull.device)
        self.all_patterns_async(Ofull, out, prec=prec)
        return results_array(out, 1 << M)

    def bounds(self, Os, tol: float = 1e-10, layout: str = "xxpp", stream=None):
        """FP32 bound pass for a list of 2k x 2k float64 CUDA tensors; returns a list of dicts."""
        n = len(Os)
        if n == 0:
            return []
        dev = Os[0].device
        ptrs = torch.tensor([O.data_ptr() for O in Os], dtype=torch.int64, device=dev)
        ks = torch.tensor([_mat(O)[0] for O in Os], dtype=torch.int32, device=dev)
        lds = torch.tensor([_mat(O)[1] for O in Os], dtype=torch.int32, device=dev)
        out = torch.zeros(n * BOUND_BYTES, dtype=torch.uint8, device=dev)
        _check(self.lib.tor_bounds(self.h, ptrs.data_ptr(), ks.data_ptr(), lds.data_ptr(), n,
                                   _LAYOUT[layout], tol, _stream(stream), out.data_ptr()))
        raw = out.cpu().numpy().tobytes()
        res = []
        for i in range(n):
            b = TorBoundC.from_buffer_copy(raw[i * BOUND_BYTES:(i + 1) * BOUND_BYTES])
            res.append({f: getattr(b, f) for f, _ in TorBoundC._fields_})
        return res

    def batch_reserve(self, n_max: int, k_max: int):
        """Size the batch workspace once (then tor_batch allocates nothing and is capturable)."""
        _check(self.lib.tor_batch_reserve(self.h, n_max, k_max))

    def batch_async(self, ptrs: torch.Tensor, ks: torch.Tensor, lds: torch.Tensor, out: torch.Tensor,
                    prec: str = "auto", tol: float = 1e-10, layout: str = "xxpp", stream=None):
        """tor_batch on device arrays: ptrs int64, ks/lds int32, out uint8 (n * RESULT_BYTES)."""
        n = ptrs.numel()
        if out.numel() < n * RESULT_BYTES:
            raise ValueError("out too small")
        _check(self.lib.tor_batch(self.h, ptrs.data_ptr(), ks.data_ptr(), lds.data_ptr(), n, _LAYOUT[layout],
                                  _PREC[prec], tol, _stream(stream), out.data_ptr()))

    def batch(self, Os, prec: str = "auto", tol: float = 1e-10, layout: str = "xxpp", stream=None):
        """Tor of a list of 2k x 2k float64 CUDA tensors (blocking); returns a list of TorResult."""
        n = len(Os)
        if n == 0:
            return []
        dev = Os[0].device
        ptrs = torch.tensor([O.data_ptr() for O in Os], dtype=torch.int64, device=dev)
        ks = torch.tensor([_mat(O)[0] for O in Os], dtype=torch.int32, device=dev)
        lds = torch.tensor([_mat(O)[1] for O in Os], dtype=torch.int32, device=dev)
        out = torch.zeros(n * RESULT_BYTES, dtype=torch.uint8, device=dev)
        self.batch_async(ptrs, ks, lds, out, prec=prec, tol=tol, layout=layout, stream=stream)
        raw = out.cpu().numpy().tobytes()
        return [TorResult.from_bytes(raw[i * RESULT_BYTES:(i + 1) * RESULT_BYTES]) for i in range(n)]

    def batch_patterns_async(self, Ofull: torch.Tensor, patterns: torch.Tensor, out: torch.Tensor,
                             prec: str = "auto", tol: float = 1e-10, stream=None):
        """tor_batch_patterns: patterns is an int64 CUDA tensor (n, ceil(M/64)) of bitsets."""
        k2, ld = _mat(Ofull)
        n = patterns.shape[0]
        if out.numel() < n * RESULT_BYTES:
            raise ValueError("out too small")
        _check(self.lib.tor_batch_patterns(self.h, Ofull.data_ptr(), k2, ld, patterns.data_ptr(), n,
                                           _PREC[prec], tol, _stream(stream), out.data_ptr()))

    def batch_patterns(self, Ofull: torch.Tensor, patterns, prec: str = "auto", tol: float = 1e-10):
        """Tor(O_S) for each 0/1 pattern (rows of a (n, M) array-like); blocking."""
        M = Ofull.shape[0] // 2
        bits = pack_patterns(patterns, M).to(Ofull.device)
        n = bits.shape[0]
        out = torch.zeros(n * RESULT_BYTES, dtype=torch.uint8, device=Ofull.device)
        self.batch_patterns_async(Ofull, bits, out, prec=prec, tol=tol)
        return results_from_tensor(out, n)

    def sample_step(self, Ofull: torch.Tensor, logdet_sigma: float, patterns: torch.Tensor, logp: torch.Tensor,
                    logq: torch.Tensor, accepted: torch.Tensor, seed: int, step: int, marg_p=None,
                    proposal=None, prec: str = "auto", tol: float = 1e-10, k_cap: int = 0, stream=None):
        """gbs_sample_step on device state tensors (patterns int64 (C, W), logp/logq float64, accepted int32)."""
        k2, ld = _mat(Ofull)
        C = patterns.shape[0]
        _check(self.lib.gbs_sample_step(self.h, Ofull.data_ptr(), k2, ld, float(logdet_sigma),
                                        marg_p.data_ptr() if marg_p is not None else None,
                                        proposal.h if proposal is not None else None, C, patterns.data_ptr(),
                                        logp.data_ptr(), logq.data_ptr(), accepted.data_ptr(),
                                        seed & 0xFFFFFFFFFFFFFFFF, step & 0xFFFFFFFFFFFFFFFF, _PREC[prec], tol,
                                        int(k_cap), _stream(stream)))

    def sample_step_da(self, Ofull: torch.Tensor, logdet_sigma: float, patterns: torch.Tensor, logp: torch.Tensor,
                       logq: torch.Tensor, logs: torch.Tensor, accepted: torch.Tensor, seed: int, step: int,
                       marg_p, surrogate, prec: str = "auto", tol: float = 1e-10, k_cap: int = 0, stream=None):
        """gbs_sample_step_da: plain proposals screened by the surrogate network (logs: its log density
        of the current states, float64 (C,), in/out), the exact Torontonian only for the survivors."""
        k2, ld = _mat(Ofull)
        C = patterns.shape[0]
        _check(self.lib.gbs_sample_step_da(self.h, Ofull.data_ptr(), k2, ld, float(logdet_sigma), marg_p.data_ptr(),
                                           surrogate.h, C, patterns.data_ptr(), logp.data_ptr(), logq.data_ptr(),
                                           logs.data_ptr(), accepted.data_ptr(), seed & 0xFFFFFFFFFFFFFFFF,
                                           step & 0xFFFFFFFFFFFFFFFF, _PREC[prec], tol, int(k_cap), _stream(stream)))

    def autotune(self, k: int, prec: str, cache_path: str | None = None):
        """Time chunk depths and launch shapes for k clicks; returns (chunk_bits, blocks_per_sm)."""
        d, b = ctypes.c_int(), ctypes.c_int()
        _check(self.lib.tor_autotune(self.h, k, _PREC[prec], cache_path.encode() if cache_path else None,
                                     ctypes.byref(d), ctypes.byref(b)))
        return d.value, b.value

    def set_timing(self, on: bool):
        _check(self.lib.tor_set_timing(self.h, int(bool(on))))

    def transform_time_ms(self) -> float:
        ms = ctypes.c_float()
        _check(self.lib.tor_transform_time(self.h, ctypes.byref(ms)))
        return ms.value

    def walk_time_ms(self) -> float:
        ms = ctypes.c_float()
        _check(self.lib.tor_walk_time(self.h, ctypes.byref(ms)))
        return ms.value

    def fp64_peak(self):
        """(measured DFMA per second, nominal SM clock in Hz)."""
        r, c = ctypes.c_double(), ctypes.c_double()
        _check(self.lib.tor_fp64_peak(self.h, ctypes.byref(r), ctypes.byref(c)))
        return r.value, c.value

    def int_peak(self) -> float:
        """Measured signed 32 x 32 -> 64-bit integer multiply-adds per second."""
        r = ctypes.c_double()
        _check(self.lib.tor_int_peak(self.h, ctypes.byref(r)))
        return r.value


def single_noalloc(O: torch.Tensor, out: torch.Tensor, prec: str, layout: str = "xxpp",
                   stream=None):
    """tor_single_noalloc: enqueue Tor(O) with no device allocation; result bytes into `out`.

    For callers that cannot allocate device memory: all scratch comes from a
    fixed array inside the library.  Calls on one device must not overlap.
    """
    k, ld = _mat(O)
    if out.dtype != torch.uint8 or out.numel() < RESULT_BYTES or not out.is_cuda:
        raise ValueError(f"out must be a uint8 CUDA tensor of >= {RESULT_BYTES} bytes")
    _check(load_library().tor_single_noalloc(O.data_ptr(), k, ld, _LAYOUT[layout], _PREC[prec],
                                             _stream(stream), out.data_ptr()))


def fixed_to_result(limbs, k: int, tier: str = "fp64") -> TorResult:
    """Convert raw limbs (signed sum, sum_abs): 8 limbs of 256-bit fixed point with 128 fraction
    bits, or 16 limbs of 512-bit fixed point with 256 fraction bits for fx256."""
    n = partial_limbs(tier)
    limbs = list(limbs)
    if len(limbs) != n:
        raise ValueError(f"{tier} partials have {n} limbs, got {len(limbs)}")
    arr = (ctypes.c_uint64 * n)(*[int(x) & 0xFFFFFFFFFFFFFFFF for x in limbs])
    out = TorResultC()
    _check(load_library().tor_fixed_to_result(arr, k, _PREC[tier], ctypes.byref(out)))
    return TorResult.from_c(out)


def sum_partials(rows, tier: str) -> "np.ndarray":
    """tor_sum_partials: the exact sum of partial-sum pairs (rows of 2 L uint64 limbs, L = 8 for
    fx256, else 4) as one pair of 2 L limbs."""
    import numpy as np
    n_limbs = partial_limbs(tier)
    rows = np.ascontiguousarray(np.asarray(rows).astype(np.uint64, copy=False).reshape(-1, n_limbs))
    out = np.zeros(n_limbs, dtype=np.uint64)
    _check(load_library().tor_sum_partials(rows.ctypes.data_as(ctypes.POINTER(_U64)), rows.shape[0],
                                           _PREC[tier], out.ctypes.data_as(ctypes.POINTER(_U64))))
    return out


def levels(O: torch.Tensor, prec: str = "fp64", level_prec=None, layout: str = "xxpp", stream=None) -> TorResult:
    """tor_levels: Tor(O) by the paper's level-by-level schedule with a fresh elimination per
    subset; level_prec: optional list of k + 1 tier names for the levels |Z| = 0..k."""
    lib = load_library()
    k, ld = _mat(O)
    nbytes = ctypes.c_size_t()
    rc = lib.tor_levels_workspace(k, O.device.index or 0, ctypes.byref(nbytes))
    if rc:
        raise TorError(rc, "tor_levels_workspace failed")
    ws = torch.empty(max(nbytes.value, 1), dtype=torch.uint8, device=O.device)
    out = torch.zeros(RESULT_BYTES, dtype=torch.uint8, device=O.device)
    lp = None
    if level_prec is not None:
        if len(level_prec) != k + 1:
            raise ValueError("level_prec needs k + 1 entries")
        lp = (ctypes.c_int * (k + 1))(*[_PREC[p] for p in level_prec])
    rc = lib.tor_levels(O.data_ptr(), k, ld, _LAYOUT[layout], _PREC[prec], lp, ws.data_ptr(), nbytes.value,
                        _stream(stream), out.data_ptr())
    if rc:
        raise TorError(rc, lib.tor_levels_last_error().decode())
    return TorResult.from_bytes(out.cpu().numpy().tobytes())


def level_next_mask(mask: int) -> int:
    """The next smaller mask with the same popcount (Algorithm 2); 0 when none is left."""
    return int(load_library().tor_level_next_mask(mask & 0xFFFFFFFFFFFFFFFF))


def level_kth_mask(k: int, m: int, r: int) -> int:
    """The r-th mask of popcount m over k bits, in decreasing order (Algorithm 2)."""
    out = ctypes.c_uint64()
    _check(load_library().tor_level_kth_mask(k, m, r, ctypes.byref(out)))
    return out.value


def fx256_fma2(s: torch.Tensor, a1: torch.Tensor, b1: torch.Tensor, a2: torch.Tensor, b2: torch.Tensor):
    """Elementwise s + a1 b1 + a2 b2 as the fx256 tier's Schur updates form it: int32 CUDA tensors
    (n, 9) of limbs (value = sum_i l_i 2^(29 i - 203)); returns (result (n, 9), overflow (n,))."""
    n = s.shape[0]
    for x in (s, a1, b1, a2, b2):
        if x.dtype != torch.int32 or tuple(x.shape) != (n, 9) or not x.is_cuda or not x.is_contiguous():
            raise ValueError("operands must be contiguous int32 CUDA tensors of shape (n, 9)")
    out = torch.zeros_like(s)
    ovf = torch.zeros(n, dtype=torch.int32, device=s.device)
    _check(load_library().tor_fx256_fma2(s.data_ptr(), a1.data_ptr(), b1.data_ptr(), a2.data_ptr(),
                                         b2.data_ptr(), n, out.data_ptr(), ovf.data_ptr(), None))
    torch.cuda.synchronize(s.device)
    return out, ovf


def limbs_to_int(limbs) -> int:
    """Signed Python integer of L little-endian 64-bit limbs (value = int / 2^(32 L): 4 limbs
    with 128 fraction bits, or 8 limbs with 256 for fx256)."""
    limbs = list(limbs)
    v = 0
    for i, x in enumerate(limbs):
        v |= (int(x) & 0xFFFFFFFFFFFFFFFF) << (64 * i)
    nb = 64 * len(limbs)
    if v >> (nb - 1):
        v -= 1 << nb
    return v


class MLP:
    """The MADE proposal network (tor_mlp_*): BF16 tensor-core forward/backward, FP32 Adam."""

    def __init__(self, ctx: Context, M: int, hidden: int = 256, seed: int = 0):
        self.lib = load_library()
        self.M, self.H = M, hidden
        self.words = (M + 63) // 64
        h = ctypes.c_void_p()
        _check(self.lib.tor_mlp_create(ctx.h, M, hidden, seed, ctypes.byref(h)))
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            self.lib.tor_mlp_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def num_params(self) -> int:
        return self.lib.tor_mlp_num_params(self.h)

    def get_params(self, which: int = 0):
        import numpy as np
        out = np.zeros(self.num_params, dtype=np.float32)
        _check(self.lib.tor_mlp_get_params(self.h, out.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), which))
        return out

    def set_params(self, theta):
        import numpy as np
        a = np.ascontiguousarray(theta, dtype=np.float32)
        if a.size != self.num_params:
            raise ValueError("wrong parameter count")
        _check(self.lib.tor_mlp_set_params(self.h, a.ctypes.data_as(ctypes.POINTER(ctypes.c_float))))

    def set_marginals(self, marg):
        """Start at the plain proposal (independent clicks with probabilities marg)."""
        import numpy as np
        a = np.ascontiguousarray(marg, dtype=np.float64)
        _check(self.lib.tor_mlp_set_marginals(self.h, a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))))

    def logq(self, patterns: torch.Tensor, stream=None) -> torch.Tensor:
        B = patterns.shape[0]
        out = torch.empty(B, dtype=torch.float64, device=patterns.device)
        _check(self.lib.tor_mlp_logq(self.h, patterns.data_ptr(), B, out.data_ptr(), _stream(stream)))
        return out

    def logits(self, patterns: torch.Tensor):
        import numpy as np
        B = patterns.shape[0]
        out = np.zeros((B, self.M), dtype=np.float32)
        _check(self.lib.tor_mlp_logits(self.h, patterns.data_ptr(), B,
                                       out.ctypes.data_as(ctypes.POINTER(ctypes.c_float))))
        return out

    def grad(self, patterns: torch.Tensor, w: torch.Tensor, stream=None) -> float:
        loss = ctypes.c_float()
        _check(self.lib.tor_mlp_grad(self.h, patterns.data_ptr(), w.data_ptr(), patterns.shape[0],
                                     ctypes.byref(loss), _stream(stream)))
        return loss.value

    def train_step(self, patterns: torch.Tensor, w: torch.Tensor, lr: float = 1e-3, stream=None) -> float:
        loss = ctypes.c_float()
        _check(self.lib.tor_mlp_train_step(self.h, patterns.data_ptr(), w.data_ptr(), patterns.shape[0],
                                           ctypes.c_float(lr), ctypes.byref(loss), _stream(stream)))
        return loss.value

    def sample(self, B: int, seed: int, step: int, device="cuda", stream=None):
        pats = torch.zeros((B, self.words), dtype=torch.int64, device=device)
        lq = torch.zeros(B, dtype=torch.float64, device=device)
        _check(self.lib.tor_mlp_sample(self.h, B, seed & 0xFFFFFFFFFFFFFFFF, step & 0xFFFFFFFFFFFFFFFF,
                                       pats.data_ptr(), lq.data_ptr(), _stream(stream)))
        return pats, lq


_default = None


def default_context(device: int = 0) -> Context:
    global _default
    if _default is None:
        _default = Context(device)
    return _default


def tor_single(O: torch.Tensor, prec: str = "auto", layout: str = "xxpp", tol: float = 1e-10,
               stream=None) -> TorResult:
    return default_context(O.device.index or 0).single(O, prec=prec, layout=layout, tol=tol, stream=stream)
