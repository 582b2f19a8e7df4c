"""Oracle runs for the GPU parity tests that are slow enough to spread over
the host cores (imported by worker processes started with `spawn`; test
infrastructure only, never by the product path)."""

import numpy as np

import oracle
from paper_2605_03123_gb300 import inputs


def host_cotangent(circuit):
    """The cotangent of one batch circuit, drawn on the host from its own seed."""
    return inputs.random_state(circuit["norb"], circuit["nelec"],
                               inputs.rng(circuit["cot_seed"]))


def lucj_forward_and_vjp(circuit):
    """Forward state and (dK, dJ_aa, dJ_ab, dL/dpsi_in) of one circuit from
    Hartree-Fock, by the oracle's literal composition and stored-state
    reverse mode."""
    c = circuit
    fwd = oracle.lucj_forward(c["K"], c["J_aa"], c["J_ab"], c["norb"], c["nelec"])
    vjp = oracle.lucj_vjp(c["K"], c["J_aa"], c["J_ab"], host_cotangent(c), c["norb"],
                          c["nelec"])
    return fwd, vjp


def lucj_forward_only(circuit):
    c = circuit
    return oracle.lucj_forward(c["K"], c["J_aa"], c["J_ab"], c["norb"], c["nelec"])
