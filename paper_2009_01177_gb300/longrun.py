"""Long Torontonian runs (k >= 40): chunk-window progress, checkpoint and resume.

A k = 40 Torontonian in the 256-bit tier takes about two hours on one GB300
and k = 50 far longer, so the chunk space [0, 2^d) is walked in windows of
consecutive chunks (tor_chunks), and after every window the exact partial
sum (integer limbs) and a done bitmap over the windows go to a checkpoint
file keyed by a hash of the instance.  Partials add exactly, so a run that
was cancelled and resumed, or whose windows ran in any order or on several
processes, gives the same total bit for bit as one uninterrupted run.

Each window's launch is watched from the host: the stream is polled until it
finishes or a deadline passes (TimeoutError; the kernel itself has no wait
that could hang).  Cancellation is cooperative, between windows.
"""
from __future__ import annotations

import hashlib
import os
import time
from dataclasses import dataclass, field

import numpy as np

from . import shard


def instance_key(O: np.ndarray, prec: str, chunk_bits: int) -> str:
    """Hash of the matrix bytes, tier and chunk depth: a checkpoint only resumes the same run."""
    h = hashlib.sha256()
    h.update(np.ascontiguousarray(O, dtype=np.float64).tobytes())
    h.update(f"{O.shape}|{prec}|{chunk_bits}".encode())
    return h.hexdigest()


@dataclass
class RunState:
    key: str
    chunk_bits: int
    window: int
    limbs: int                       # 8, or 16 for the 256-bit tier
    done: np.ndarray                 # bool per window
    total: np.ndarray                # exact partial sum of the finished windows (uint64 limbs)
    seconds: float = 0.0             # wall time spent in finished windows
    extra: dict = field(default_factory=dict)

    @property
    def nwindows(self) -> int:
        return self.done.size

    @property
    def complete(self) -> bool:
        return bool(self.done.all())


def save_checkpoint(path: str, st: RunState):
    """Atomically replace the checkpoint (write a temporary file, then rename)."""
    tmp = path + ".tmp.npz"
    np.savez(tmp, key=np.array(st.key), chunk_bits=st.chunk_bits, window=st.window, limbs=st.limbs,
             done=st.done, total=st.total, seconds=st.seconds)
    os.replace(tmp, path)


def load_checkpoint(path: str, key: str, chunk_bits: int, window: int, limbs: int) -> RunState | None:
    """The saved state if it belongs to this run (same instance hash, depth, window, width)."""
    if not os.path.exists(path):
        return None
    with np.load(path) as z:
        if (str(z["key"]) != key or int(z["chunk_bits"]) != chunk_bits or int(z["window"]) != window
                or int(z["limbs"]) != limbs):
            return None
        return RunState(key, chunk_bits, window, limbs, z["done"].astype(bool).copy(),
                        z["total"].astype(np.uint64).copy(), float(z["seconds"]))


def run_chunks(chunk_fn, nchunks: int, window: int, limbs: int, key: str, chunk_bits: int,
               checkpoint: str | None = None, should_stop=None, on_window=None) -> RunState:
    """Walk windows [w W, (w+1) W) of the chunk space with chunk_fn(c0, c1) -> (c1 - c0, limbs)
    partials, skipping windows a matching checkpoint marks done.  should_stop() is asked
    between windows; on_window(state, w) after each.  Returns the (possibly partial) state."""
    nwin = (nchunks + window - 1) // window
    st = load_checkpoint(checkpoint, key, chunk_bits, window, limbs) if checkpoint else None
    if st is None:
        st = RunState(key, chunk_bits, window, limbs, np.zeros(nwin, dtype=bool),
                      np.zeros(limbs, dtype=np.uint64))
    for w in range(nwin):
        if st.done[w]:
            continue
        if should_stop is not None and should_stop():
            break
        c0, c1 = w * window, min(nchunks, (w + 1) * window)
        t0 = time.perf_counter()
        part = np.asarray(chunk_fn(c0, c1), dtype=np.uint64).reshape(-1, limbs)
        st.total = shard.sum_partials(np.vstack([st.total[None, :], part]))
        st.seconds += time.perf_counter() - t0
        st.done[w] = True
        if checkpoint:
            save_checkpoint(checkpoint, st)
        if on_window is not None:
            on_window(st, w)
    return st


def watched(stream_query, deadline_s: float, poll_s: float = 0.01):
    """Poll stream_query() until it returns True; TimeoutError once deadline_s has passed."""
    t_end = time.monotonic() + deadline_s
    while not stream_query():
        if time.monotonic() > t_end:
            raise TimeoutError(f"launch still running after {deadline_s:.1f} s")
        time.sleep(poll_s)


def tor_long(ctx, O_dev, prec: str, chunk_bits: int, window: int, checkpoint: str | None = None,
             deadline_s: float = 3600.0, should_stop=None, on_window=None):
    """Tor(O) in windows of `window` chunks of depth chunk_bits with checkpoints; returns
    (TorResult or None if stopped early, RunState)."""
    import torch
    from . import tor
    k = O_dev.shape[0] // 2
    key = instance_key(O_dev.cpu().numpy(), prec, chunk_bits)
    limbs = tor.partial_limbs(prec)
    stream = torch.cuda.Stream(O_dev.device)

    def chunk_fn(c0, c1):
        with torch.cuda.stream(stream):
            part = ctx.chunks(O_dev, chunk_bits, c0, c1, prec=prec, stream=stream)
        watched(stream.query, deadline_s)
        return part.cpu().numpy().view(np.uint64)

    st = run_chunks(chunk_fn, 1 << chunk_bits, window, limbs, key, chunk_bits, checkpoint,
                    should_stop, on_window)
    if not st.complete:
        return None, st
    return tor.fixed_to_result([int(x) for x in st.total], k, prec), st
