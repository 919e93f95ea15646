"""The Python Philox4x32-10 against the published known-answer vectors (CPU)."""
from tests.philox_ref import philox4x32_10, uniform


def test_known_answer_vectors():
    assert philox4x32_10((0, 0, 0, 0), (0, 0)) == (0x6627e8d5, 0xe169c58d, 0xbc57ac4c, 0x9b00dbd8)
    f = 0xFFFFFFFF
    assert philox4x32_10((f, f, f, f), (f, f)) == (0x408f276d, 0x41c83b0e, 0xa20bc7c6, 0x6d5451fd)
    assert philox4x32_10((0x243f6a88, 0x85a308d3, 0x13198a2e, 0x03707344), (0xa4093822, 0x299f31d0)) == \
        (0xd16cfe09, 0x94fdcceb, 0x5001e420, 0x24126ea1)


def test_uniforms_in_open_interval_and_distinct():
    us = [uniform(7, 3, c, j) for c in range(4) for j in range(8)]
    assert all(0.0 < u < 1.0 for u in us)
    assert len(set(us)) == len(us)
