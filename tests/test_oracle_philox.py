"""Pins for the oracle's Philox4x32-10 generator (Salmon et al., SC'11).

The known-answer vectors are the published ones for Philox4x32 with ten
rounds; a mistake anywhere in the round function, the multipliers, the Weyl
key schedule or the word order changes every output word.
"""
import numpy as np

from oracle.oracle import philox4x32_10


def test_kat_zero():
    assert philox4x32_10((0, 0, 0, 0), (0, 0)) == (0x6627E8D5, 0xE169C58D, 0xBC57AC4C, 0x9B00DBD8)


def test_kat_all_ones():
    assert philox4x32_10((0xFFFFFFFF,) * 4, (0xFFFFFFFF,) * 2) == (
        0x408F276D, 0x41C83B0E, 0xA20BC7C6, 0x6D5451FD)


def test_kat_pi_digits():
    ctr = (0x243F6A88, 0x85A308D3, 0x13198A2E, 0x03707344)
    key = (0xA4093822, 0x299F31D0)
    assert philox4x32_10(ctr, key) == (0xD16CFE09, 0x94FDCCEB, 0x5001E420, 0x24126EA1)


def test_counter_stream_is_uniform():
    # 4096 consecutive counters: every output bit is set about half the time
    words = np.array([philox4x32_10((k, 7, 1, 0), (1, 0)) for k in range(4096)], dtype=np.uint64)
    bits = ((words[:, :, None] >> np.arange(32, dtype=np.uint64)) & 1).mean(axis=0)
    assert np.all(np.abs(bits - 0.5) < 0.05)
