"""The seeded input generator (the one module the oracle side and the CUDA
side share; it draws bits and holds none of the method's arithmetic), pinned
to the published SplitMix64 and to its own stated rules."""
import numpy as np
import pytest

from paper_2302_10083_gb300 import synth

MASK64 = (1 << 64) - 1


def splitmix64_next(state):
    """SplitMix64 as published (Steele, Lea and Flood, OOPSLA 2014; Vigna's
    splitmix64.c), on Python integers: returns (new state, output)."""
    state = (state + 0x9E3779B97F4A7C15) & MASK64
    z = state
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
    return state, z ^ (z >> 31)


def test_splitmix64_published_sequence():
    """Seeded with 0, SplitMix64's first outputs are the widely printed
    e220a8397b1dcdaf, 6e789e6aa1b965f4, 06c45d188009454f; the generator's mix
    of state z is the output that follows state z."""
    want = [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]
    s = 0
    for k, w in enumerate(want):
        z = s
        s, out = splitmix64_next(s)
        assert out == w
        assert int(synth._mix(np.uint64(z))) == w, k


@pytest.mark.parametrize("seed,stream", [(1, 0), (2, 1), (0xFFFFFFFF, 2), (12345678901234, 3)])
def test_draws_match_scalar_definition(seed, stream):
    """u(seed, stream, x) = mix(key + x), key = mix(seed xor stream * golden),
    on Python integers against the vectorised uint64 form."""
    _, key = splitmix64_next((seed ^ (stream * 0x9E3779B97F4A7C15)) & MASK64)
    xs = np.array([0, 1, 2, 1000, (1 << 40) + 7, MASK64], dtype=np.uint64)
    got = synth.draws(seed, stream, xs)
    for x, g in zip(xs.tolist(), got.tolist()):
        assert splitmix64_next((key + x) & MASK64)[1] == g


def test_bernoulli_rule_and_frequency():
    assert synth.bernoulli(1, 0, 100, 1.0).all()
    assert not synth.bernoulli(1, 0, 100, 0.0).any()
    u = synth.draws(3, 0, np.arange(1 << 16, dtype=np.uint64))
    b = synth.bernoulli(3, 0, 1 << 16, 0.3)
    assert np.array_equal(b, u < np.uint64(int(0.3 * 2.0 ** 64)))
    for p in (0.05, 0.5, 0.85):
        m = 1 << 18
        f = synth.bernoulli(7, 0, m, p).mean()
        assert abs(f - p) < 5 * (p * (1 - p) / m) ** 0.5, (p, f)


@pytest.mark.parametrize("n", [0, 1, 2, 3, 9])
def test_random_function_layout(n):
    """ceil(2^n/8) LSB-first bytes, zero tail bits, DC drawn on stream 1 and
    kept only where ON is 0."""
    on, dc = synth.random_function(n, 5, 0.6, 0.5)
    assert on.size == dc.size == synth.tt_bytes(n)
    m = 1 << n
    on_b = synth.unpack(on, n)
    dc_b = synth.unpack(dc, n)
    assert np.array_equal(on_b, synth.bernoulli(5, synth.STREAM_ON, m, 0.6))
    assert np.array_equal(dc_b, synth.bernoulli(5, synth.STREAM_DC, m, 0.5) & ~on_b)
    for t in range(m):
        assert bool((on[t >> 3] >> (t & 7)) & 1) == on_b[t]
    if m < 8:
        assert (on[0] >> m) == 0 and (dc[0] >> m) == 0
    assert synth.random_function(n, 5, 0.6)[1] is None
