"""The host-built tables behind the sweeps, checked on the CPU.

The window sweeps and the transition reduction run from tables built on the
host (`window_tables_host`, `tpass_tables_host` in fs_host.cpp): per window
position the orbits (strings sharing their occupation outside the window)
with the address of every member, and per four-orbital pass the records of
the transition reduction with their sign bits.  The GPU parity tests use
them only through the kernels' results; here a small C++ driver prints them
and every address is checked against the oracle's string enumeration (the
combinatorial-number-system order of the paper's addressing, §3.1):

- each orbit lists the strings O u S for the C(W, m) subsets S of the window
  in ascending-mask order, and the orbits of a position cover every string
  with 1..W-1 electrons in the window exactly once;
- each class (value of m) starts on a multiple of 32 items;
- every unordered orbital pair and every diagonal is owned by exactly one
  pass, and a pass's records cover every string with 1..4 electrons in the
  pass's orbitals exactly once, with the gap parities and sign bits the
  reduction folds into the amplitudes;
- the bank-aware order keeps the modelled shared-memory wavefronts of the
  16-byte gathers (eight lanes per wavefront, cell index mod 8 per bank
  group) near the ideal at N = 16, and spaces too large for one CTA keep the
  combinatorial order.
"""

import os
import shutil
import subprocess

import numpy as np
import pytest

import oracle

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def driver(tmp_path_factory):
    gxx = shutil.which("g++")
    cuda_inc = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "include")
    if gxx is None or not os.path.exists(os.path.join(cuda_inc, "cuda_runtime.h")):
        pytest.skip("needs g++ and the CUDA headers")
    exe = str(tmp_path_factory.mktemp("host_tables") / "host_tables_driver")
    csrc = os.path.join(ROOT, "paper_2605_03123_gb300", "csrc")
    cmd = [gxx, "-O2", "-std=c++17", "-I", cuda_inc, "-I", os.path.join(ROOT, "include"),
           "-I", csrc, os.path.join(ROOT, "tests", "host_tables_driver.cpp"),
           os.path.join(csrc, "fs_host.cpp"), "-o", exe]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr[-2000:]
    return exe


def _tables(exe, N, n, W):
    out = subprocess.run([exe, str(N), str(n), str(W)], capture_output=True, text=True,
                         check=True).stdout.split("\n")
    win, passes = [], []
    for line in out:
        t = line.split()
        if not t:
            continue
        if t[0] == "orbit":
            a, m, clo, ro = map(int, t[1:5])
            win.append((a, m, clo, ro, [int(x) for x in t[5:]]))
        elif t[0] == "pad":
            win.append((int(t[1]), 0, 0, 0, []))
        elif t[0] == "pass":
            passes.append(([int(x) for x in t[1:5]], int(t[5]), []))
        elif t[0] == "rec":
            passes[-1][2].append((int(t[1]), int(t[2]), int(t[3]), [int(x) for x in t[4:]]))
        elif t[0] == "rpad":
            passes[-1][2].append(None)
    return win, passes


def _masks(W, m):
    return [s for s in range(1 << W) if bin(s).count("1") == m]


def _rank_of(strings):
    return {int(s): i for i, s in enumerate(strings)}


@pytest.mark.parametrize("N,n", [(8, 4), (10, 3), (12, 6), (9, 5)])
def test_window_orbits_cover_each_string_once(driver, N, n):
    W = 6
    win, _ = _tables(driver, N, n, W)
    strings = oracle.strings(N, n)
    rank = _rank_of(strings)
    by_pos = {}
    for item in win:
        by_pos.setdefault(item[0], []).append(item)
    for a in range(N - W + 1):
        items = by_pos.get(a, [])
        wmask = ((1 << W) - 1) << a
        seen = set()
        prev_m = None
        for pos, (_, m, clo, ro, addrs) in enumerate(items):
            if m == 0:
                continue
            if m != prev_m:  # a new class starts on a warp boundary
                assert pos % 32 == 0, (a, m, pos)
                prev_m = m
            subs = _masks(W, m)
            assert len(addrs) == len(subs)
            outside = int(strings[addrs[0]]) & ~wmask
            assert bin(outside & ((1 << a) - 1)).count("1") == clo
            for S, e in zip(subs, addrs):
                s = outside | (S << a)
                assert rank[s] == e, (a, m, S)
                assert e not in seen
                seen.add(e)
        want = {i for i, s in enumerate(strings) if 1 <= bin(int(s) & wmask).count("1") <= W - 1}
        assert seen == want, a
        assert len(items) % 32 == 0


@pytest.mark.parametrize("N,n", [(8, 4), (10, 3), (12, 6), (13, 6), (16, 8)])
def test_transition_passes_own_every_pair_once(driver, N, n):
    _, passes = _tables(driver, N, n, 6)
    owned = np.zeros((N, N), int)
    for q, keep, _ in passes:
        for i in range(4):
            for j in range(4):
                if (keep >> (4 * i + j)) & 1:
                    owned[q[i], q[j]] += 1
    assert np.all(owned == 1), owned
    if N == 16:  # the affine plane AG(2,4): 20 passes, every pair in exactly one
        assert len(passes) == 20


@pytest.mark.parametrize("N,n", [(8, 4), (10, 3), (12, 6)])
def test_transition_records_addresses_and_signs(driver, N, n):
    _, passes = _tables(driver, N, n, 6)
    strings = oracle.strings(N, n)
    rank = _rank_of(strings)
    for q, _, recs in passes:
        qmask = sum(1 << x for x in q)
        seen = set()
        prev_m = None
        for pos, rc in enumerate(recs):
            if rc is None:
                continue
            m, gbits, flips, addrs = rc
            if m != prev_m:
                assert pos % 32 == 0
                prev_m = m
            subs = _masks(4, m)
            assert len(addrs) == len(subs)
            outside = int(strings[addrs[0]]) & ~qmask
            # gbits bit j: parity of the outside orbitals between q_0 and q_j
            for j in range(1, 4):
                between = bin(outside & ((1 << q[j]) - 1) & ~((2 << q[0]) - 1)).count("1")
                assert ((gbits >> j) & 1) == between % 2
            for k, (S, e) in enumerate(zip(subs, addrs)):
                s = outside
                for i in range(4):
                    if (S >> i) & 1:
                        s |= 1 << q[i]
                assert rank[s] == e
                omega = 0
                for j in range(1, 4):
                    if (S >> j) & 1:
                        omega ^= (gbits >> j) & 1
                assert ((flips >> k) & 1) == omega
                assert e not in seen
                seen.add(e)
        want = {i for i, s in enumerate(strings) if 1 <= bin(int(s) & qmask).count("1") <= 4}
        assert seen == want


def _wavefronts(groups):
    """Modelled 16-byte shared-memory wavefronts: per aligned group of eight
    lanes and per member k, the largest number of distinct cells that fall
    on one bank group (cell index mod 8)."""
    tot = ideal = 0
    for g in groups:
        ns = max(len(x) for x in g)
        for k in range(ns):
            cells = {}
            for x in g:
                if k < len(x):
                    cells.setdefault(x[k] % 8, set()).add(x[k])
            tot += max(len(v) for v in cells.values())
            ideal += 1
    return tot / ideal


def test_bank_aware_order_at_n16(driver):
    win, passes = _tables(driver, 16, 8, 6)
    groups = []
    items = [w[4] for w in win]
    for i in range(0, len(items), 8):
        g = [x for x in items[i:i + 8] if x]
        if g:
            groups.append(g)
    assert _wavefronts(groups) < 1.45  # combinatorial order: 1.72
    groups = []
    for _, _, recs in passes:
        r = [x[3] if x else [] for x in recs]
        for i in range(0, len(r), 8):
            g = [x for x in r[i:i + 8] if x]
            if g:
                groups.append(g)
    assert _wavefronts(groups) < 1.7  # combinatorial order: 3.15


def test_cluster_sized_spaces_keep_the_combinatorial_order(driver):
    """N=17 (8): a complex64 vector of psi and g (24310 strings x 16 bytes)
    exceeds one CTA, so the sweeps run on clusters and the lists stay in the
    combinatorial order: within each class the outside configurations
    ascend."""
    N, n, W = 17, 8, 6
    win, passes = _tables(driver, N, n, W)
    strings = oracle.strings(N, n)
    last = {}
    for a, m, _, _, addrs in win:
        if m == 0:
            continue
        wmask = ((1 << W) - 1) << a
        outside = int(strings[addrs[0]]) & ~wmask
        key = (a, m)
        assert last.get(key, -1) < outside
        last[key] = outside
    for q, _, recs in passes[:3]:
        qmask = sum(1 << x for x in q)
        prev = {}
        for rc in recs:
            if rc is None:
                continue
            outside = int(strings[rc[3][0]]) & ~qmask
            assert prev.get(rc[0], -1) < outside
            prev[rc[0]] = outside
