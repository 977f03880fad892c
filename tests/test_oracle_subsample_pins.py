"""Pins of the oracle's stochastic viewgraph sub-sampling (Appendix A.3, Algorithm 3: a fresh
uniform random subset of min(|E|, M) pairs every step).  The random keys come from SplitMix64
(Steele, Lea and Flood, OOPSLA 2014), whose reference sequence from seed 0 is published; the
subset must have the stated size, and over many steps every pair, and every couple of pairs,
must be drawn with the frequencies of a uniform subset."""
from pathlib import Path

import numpy as np

import oracle

# SplitMix64's first outputs from seed 0 (the generator's published reference sequence)
_GOLDEN = (Path(__file__).parent / "golden" / "splitmix64_seed0.txt").read_text().splitlines()
SPLITMIX64_SEED0 = [int(ln.split()[0], 16) for ln in _GOLDEN if ln.strip() and not ln.startswith("#")]


def test_splitmix64_reference_sequence():
    gamma = 0x9E3779B97F4A7C15
    got = [oracle.splitmix64((k * gamma) % 2**64) for k in range(4)]
    assert got == SPLITMIX64_SEED0


def test_subset_size_and_determinism():
    for P, M in ((100, 10), (7, 10), (10, 10), (1, 1), (513, 512)):
        for step in (0, 1, 99):
            m = oracle.subsample(12345, step, P, M)
            assert m.sum() == min(P, M)
            assert np.array_equal(m, oracle.subsample(12345, step, P, M))
    a, b = oracle.subsample(1, 0, 100, 10), oracle.subsample(1, 1, 100, 10)
    assert not np.array_equal(a, b)  # a fresh draw each step
    assert not np.array_equal(oracle.subsample(1, 0, 100, 10), oracle.subsample(2, 0, 100, 10))


def test_subsets_are_uniform():
    P, M, S = 50, 10, 3000
    masks = np.array([oracle.subsample(2026, s, P, M) for s in range(S)])
    freq = masks.mean(axis=0)
    p1 = M / P
    assert np.all(np.abs(freq - p1) <= 4.5 * np.sqrt(p1 * (1 - p1) / S))
    # a uniform subset includes a given couple of pairs with probability M(M-1) / (P(P-1))
    p2 = M * (M - 1) / (P * (P - 1))
    for i, j in ((0, 1), (3, 41), (48, 49)):
        f2 = np.mean(masks[:, i] & masks[:, j])
        assert abs(f2 - p2) <= 4.5 * np.sqrt(p2 * (1 - p2) / S)
