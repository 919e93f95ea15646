"""Host logic of long runs: windows, checkpoint, resume, watchdog (no GPU: a fake chunk
function stands in for tor_chunks)."""
import numpy as np
import pytest

from paper_2009_01177_gb300 import longrun, shard


def fake_partials(limbs):
    """Deterministic exact partials per chunk: a signed sum and a positive sum_abs."""
    def value(c):
        rng = np.random.default_rng(c)
        v = int(rng.integers(-2 ** 62, 2 ** 62)) << int(rng.integers(0, 120))
        return v, abs(v) + 1

    calls = []

    def chunk_fn(c0, c1):
        calls.append((c0, c1))
        return np.stack([shard.ints_to_limbs(*value(c), limbs=limbs) for c in range(c0, c1)])

    def exact(n):
        lo = sum(value(c)[0] for c in range(n))
        hi = sum(value(c)[1] for c in range(n))
        return lo % (1 << (32 * limbs)), hi
    return chunk_fn, exact, calls


@pytest.mark.parametrize("limbs", [8, 16])   # the widths the tiers write
def test_uninterrupted_run_is_the_exact_sum(limbs):
    fn, exact, calls = fake_partials(limbs)
    st = longrun.run_chunks(fn, 100, 16, limbs, "k", 7)
    assert st.complete and st.nwindows == 7
    assert shard.limbs_to_ints(st.total) == exact(100)
    assert calls[-1] == (96, 100)                      # a ragged last window


def test_cancel_and_resume_gives_the_same_bits(tmp_path):
    ck = str(tmp_path / "run.npz")
    fn, exact, calls = fake_partials(8)
    stops = iter([False, False, False, True])
    st = longrun.run_chunks(fn, 64, 8, 8, "inst", 6, ck, should_stop=lambda: next(stops, True))
    assert not st.complete and st.done.sum() == 3
    first = list(calls)
    st2 = longrun.run_chunks(fn, 64, 8, 8, "inst", 6, ck)
    assert st2.complete
    assert shard.limbs_to_ints(st2.total) == exact(64)
    # every window computed exactly once across the two runs
    assert sorted(calls) == sorted(set(calls)) and len(calls) == 8
    assert set(first) == {(0, 8), (8, 16), (16, 24)}


def test_checkpoint_of_another_instance_is_ignored(tmp_path):
    ck = str(tmp_path / "run.npz")
    fn, exact, calls = fake_partials(8)
    longrun.run_chunks(fn, 32, 8, 8, "one", 5, ck)
    calls.clear()
    st = longrun.run_chunks(fn, 32, 8, 8, "another", 5, ck)
    assert len(calls) == 4 and st.complete              # started over
    assert longrun.load_checkpoint(ck, "another", 5, 8, 8) is not None
    assert longrun.load_checkpoint(ck, "another", 5, 16, 8) is None    # another window size


def test_instance_key_depends_on_matrix_tier_and_depth():
    O = np.eye(4) * 0.25
    k1 = longrun.instance_key(O, "fx256", 10)
    assert k1 == longrun.instance_key(O.copy(), "fx256", 10)
    assert k1 != longrun.instance_key(O * 1.0000001, "fx256", 10)
    assert k1 != longrun.instance_key(O, "dd", 10)
    assert k1 != longrun.instance_key(O, "fx256", 11)


def test_watchdog_deadline():
    longrun.watched(lambda: True, 0.01)
    with pytest.raises(TimeoutError):
        longrun.watched(lambda: False, 0.05, poll_s=0.01)
