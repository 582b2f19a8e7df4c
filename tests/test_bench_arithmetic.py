"""The roofline arithmetic bench.py reports, checked on CPU against counts
done here independently: element-Givens of a rotation by enumerating the
strings a Givens rotation touches, and the bytes and flops per launch."""

import itertools
import math
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def touched_fraction(N, n, p):
    """Fraction of the strings of n electrons in N orbitals that an
    adjacent Givens rotation on (p, p+1) moves (exactly one of the two
    orbitals occupied), by enumeration."""
    tot = hit = 0
    for occ in itertools.combinations(range(N), n):
        s = set(occ)
        tot += 1
        hit += (p in s) != (p + 1 in s)
    return hit / tot


def test_element_givens_per_amplitude():
    # N(N-1)/2 rotations, each touching the same fraction of strings
    N, n = 8, 4
    eg = N * (N - 1) / 2 * touched_fraction(N, n, 3)
    flops = bench.algorithmic_flops("sweep_beta_f32", N, (n, n), 1)
    assert math.isclose(flops, 10 * eg, rel_tol=1e-12)
    # the N=16 (8,8) figure quoted in the design notes: 64 per amplitude,
    # 10 real flops each (2 for c x, 6 for the complex product s y, 2 for the sum)
    assert math.isclose(bench.algorithmic_flops("sweep_beta_f32", 16, (8, 8), 1), 10 * 64,
                        rel_tol=1e-12)


def test_reverse_sweep_flops_add_the_transition_reduction():
    # two states rotated, plus n(N-n) + n complex multiply-adds per amplitude
    N, n = 16, 8
    fwd = bench.algorithmic_flops("sweep_beta_f32", N, (n, n), 1)
    rev = bench.algorithmic_flops("sweep_vjp_beta_f32", N, (n, n), 1)
    assert math.isclose(rev, 2 * fwd + 8 * (n * (N - n) + n), rel_tol=1e-12)
    # per launch at full size (the benchmark's algorithmic flops)
    amps = math.comb(16, 8) ** 2
    assert math.isclose(bench.algorithmic_flops("sweep_vjp_beta_f32", N, (n, n), amps),
                        3.074e11, rel_tol=1e-3)


def test_bytes_per_launch():
    S = 8 * math.comb(16, 8) ** 2  # one complex64 state
    assert bench.algorithmic_bytes("sweep_beta_f32", S, 10) == 2 * S
    assert bench.algorithmic_bytes("sweep_vjp_beta_f32", S, 10) == 4 * S
    assert bench.algorithmic_bytes("phase_tc_f32", S, 10) == 2 * S
    assert bench.algorithmic_bytes("transpose", S, 10) is None
