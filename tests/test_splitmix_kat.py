"""Known-answer pin of the SplitMix64 generator shared, by definition only,
by the input generator (synth.splitmix64_stream) and the oracle's
counter-based noise of the variational start (oracle.init_noise).

Both are checked against the published first outputs of the reference
generator for seed 1234567 (tests/golden/splitmix64_seed1234567.txt), so a
wrong constant or shift in either would be caught even if both sides made it.
"""
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
GOLD = 0x9E3779B97F4A7C15
MASK = (1 << 64) - 1


def _published():
    with open(os.path.join(HERE, "golden", "splitmix64_seed1234567.txt")) as f:
        return [int(l) for l in f if l.strip() and not l.startswith("#")]


def test_stream_reproduces_the_published_outputs():
    from paper_1311_6696_gb300 import synth
    got = [int(v) for v in synth.splitmix64_stream(1234567, 5)]
    assert got == _published()


def test_stream_offset_continues_the_sequence():
    from paper_1311_6696_gb300 import synth
    assert [int(v) for v in synth.splitmix64_stream(1234567, 3, start=2)] == _published()[2:5]


def test_uniform01_takes_the_top_53_bits():
    from paper_1311_6696_gb300 import synth
    u = synth.uniform01(1234567, 5)
    want = np.array([(z >> 11) * 2.0 ** -53 for z in _published()])
    assert np.array_equal(u, want)


def test_oracle_noise_is_the_same_mix():
    """init_noise(seed, tag, y, x, n)[i] is the first SplitMix64 output for the
    state key + i with key = seed*golden + (tag<<56 | y<<44 | x<<32).  With
    tag = y = x = 0 and seed = (1234567 + j*golden) * golden^-1 (mod 2^64) the
    key is the state of the published sequence before its output j+1."""
    from oracle import peps_oracle as O
    inv = pow(GOLD, -1, 1 << 64)
    for j, z in enumerate(_published()):
        seed = ((1234567 + j * GOLD) * inv) & MASK
        got = O.init_noise(seed, 0, 0, 0, 1)[0]
        assert got == (z >> 11) * 2.0 ** -52 - 1.0
    # consecutive entries step the state by one, not by golden: entry i of key k
    # is entry 0 of key k + i
    seed = (1234567 * inv) & MASK
    row = O.init_noise(seed, 0, 0, 0, 4)
    for i in range(4):
        s_i = ((1234567 + i) * inv) & MASK
        assert row[i] == O.init_noise(s_i, 0, 0, 0, 1)[0]
