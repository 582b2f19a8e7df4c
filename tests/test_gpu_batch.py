"""Batched LUCJ forward + VJP over uneven circuits in one CUDA graph: every
circuit against the oracle and against the single-circuit path."""

import os

import numpy as np
import pytest

import oracle
from paper_2605_03123_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def lib():
    assert torch.cuda.is_available(), "the GPU tests need a CUDA device"
    from paper_2605_03123_gb300 import build, fsgpu
    if not os.path.exists(build.lib_path()):
        build.build()
    fsgpu.load_library()
    return fsgpu


def dev(v, dt):
    return torch.from_numpy(np.ascontiguousarray(v)).to(
        "cuda", torch.complex128 if dt == "c128" else torch.complex64)


def host(t):
    return t.cpu().numpy().astype(np.complex128)


def _rel(a, b):
    return float(np.linalg.norm(np.ravel(a - b)) / max(np.linalg.norm(np.ravel(b)), 1e-300))


def _circuits(seed, n_reps=2):
    g = inputs.rng(seed)
    specs = [(8, (4, 4), True), (6, (3, 2), False), (10, (5, 5), True), (7, (2, 4), False),
             (8, (4, 4), False), (9, (4, 4), True), (6, (3, 3), True), (11, (5, 4), False)]
    out = []
    for norb, nelec, hf in specs:
        K = np.array([inputs.random_antihermitian(norb, 0.4, g) for _ in range(n_reps)])
        Ja = np.array([inputs.random_symmetric(norb, 0.5, g) for _ in range(n_reps)])
        Jb = np.array([g.normal(0, 0.5, (norb, norb)) for _ in range(n_reps)])
        v = None if hf else inputs.random_state(norb, nelec, g)
        c = inputs.random_state(norb, nelec, g)
        out.append(dict(norb=norb, nelec=nelec, from_hf=hf, K=K, J_aa=Ja, J_ab=Jb, v=v, c=c))
    return out


def _start(c):
    if c["from_hf"]:
        return np.zeros_like(oracle.hartree_fock(c["norb"], c["nelec"]))
    return c["v"]


@pytest.mark.parametrize("dt", ["c128", "c64"])
def test_batch_matches_oracle_and_single_path(lib, dt):
    cir = _circuits(16000)
    # a from_hf circuit overwrites its state buffer: start those from zeros
    vecs = [dev(_start(c), dt) for c in cir]
    cots = [dev(c["c"], dt) for c in cir]
    grads = lib.lucj_batch_(vecs, cots, cir, do_vjp=True)
    tol_g = 1e-11 if dt == "c128" else 2e-4
    tol_v = 1e-12 if dt == "c128" else 2e-5
    for c, (dK, dJa, dJb), x, y in zip(cir, grads, vecs, cots):
        rK, rJa, rJb, rv = oracle.lucj_vjp(c["K"], c["J_aa"], c["J_ab"], c["c"], c["norb"],
                                           c["nelec"], vec=c["v"])
        assert _rel(dK, rK) < tol_g and _rel(dJa, rJa) < tol_g and _rel(dJb, rJb) < tol_g
        v_in = oracle.hartree_fock(c["norb"], c["nelec"]) if c["from_hf"] else c["v"]
        assert np.max(np.abs(host(x) - v_in)) < tol_v
        if not c["from_hf"]:
            assert np.max(np.abs(host(y) - rv)) < tol_v
        # the single-circuit path on the same inputs
        xs = dev(_start(c), dt)
        lib.lucj_forward_(xs, c["K"], c["J_aa"], c["J_ab"], c["norb"], c["nelec"],
                          from_hf=c["from_hf"])
        ys = dev(c["c"], dt)
        sK, sJa, sJb = lib.lucj_vjp_(xs, ys, c["K"], c["J_aa"], c["J_ab"], c["norb"], c["nelec"],
                                     from_hf=c["from_hf"])
        assert _rel(dK, sK) < tol_g and _rel(dJb, sJb) < tol_g


@pytest.mark.parametrize("dt", ["c128", "c64"])
def test_batch_forward_only(lib, dt):
    cir = _circuits(16500, n_reps=1)
    vecs = [dev(_start(c), dt) for c in cir]
    lib.lucj_batch_(vecs, None, cir, do_vjp=False)
    for c, x in zip(cir, vecs):
        ref = oracle.lucj_forward(c["K"], c["J_aa"], c["J_ab"], c["norb"], c["nelec"], vec=c["v"])
        assert np.max(np.abs(host(x) - ref)) < (1e-12 if dt == "c128" else 2e-5)


def test_batch_rejects_mixed_reps(lib):
    cir = _circuits(16900, n_reps=1)[:2]
    cir[1]["K"] = np.concatenate([cir[1]["K"]] * 2)
    cir[1]["J_aa"] = np.concatenate([cir[1]["J_aa"]] * 2)
    cir[1]["J_ab"] = np.concatenate([cir[1]["J_ab"]] * 2)
    vecs = [dev(_start(c), "c64") for c in cir]
    with pytest.raises(lib.FsError):
        lib.lucj_batch_(vecs, None, cir, do_vjp=False)


def test_batch_autotuner_choices_and_results(lib):
    """The slab-width autotuner picks, per sector and sweep kind, one of the
    timed widths (the fastest), and a tuned batch gives the same states and
    gradients as an untuned one."""
    ctx = lib.context(0)
    cir = _circuits(17000)
    res = {}
    for on in (0, 1):
        ctx.set_batch_tuning(on)
        vecs = [dev(_start(c), "c64") for c in cir]
        cots = [dev(c["c"], "c64") for c in cir]
        grads = lib.lucj_batch_(vecs, cots, cir, do_vjp=True, ctx=ctx)
        res[on] = ([host(x) for x in vecs], [host(y) for y in cots], grads)
        if on:
            rep = ctx.tuning_report()
            assert rep, "the autotuner recorded no choice"
            for r in rep:
                ms, widths = r["ms"], r["widths"]
                assert len(ms) == len(widths) >= 2 and all(t > 0 for t in ms)
                assert r["vectors_per_cta"] == widths[int(np.argmin(ms))]
                if r["dtype"] == 0 and r["states"] == 1:
                    # complex64 forward sweeps run on packed vector pairs
                    assert min(widths) >= 2
    ctx.set_batch_tuning(1)
    for a, b in zip(res[0][0], res[1][0]):
        assert np.max(np.abs(a - b)) < 2e-5
    for a, b in zip(res[0][1], res[1][1]):
        assert np.max(np.abs(a - b)) < 2e-5
    for ga, gb in zip(res[0][2], res[1][2]):
        for a, b in zip(ga, gb):
            assert _rel(a, b) < 1e-4
