"""CPU checks of the GPU-vs-oracle comparison helpers (tests/parity.py).

forced_replay is exercised with a stand-in for the CUDA path built from the
oracle itself (CPU tensors, the oracle's own selections and stage
combination): the replay must then reproduce the oracle's free SSP-RK3 run
bit for bit, and a stand-in with a wrong stage coefficient (a plausible
slip in a stage epilogue) must be caught by the 1e-10 gate.
"""
import numpy as np
import pytest
import torch

import oracle
from parity import assert_values, forced_replay
from paper_2311_15504_gb300 import workloads as wl

RK = {1: (0.0, 1.0), 2: (0.75, 0.25), 3: (1.0 / 3.0, 2.0 / 3.0)}


def _fake_path(R, h, c1_stage2=0.25):
    def sel(U):
        return oracle.rhs_advection(U.numpy(), h, R, want_sel=True)["sel"].reshape(-1)

    def stage(s, Un, Us, out, dt):
        L = oracle.rhs_advection(Us.numpy(), h, R)["rhs"]
        c0, c1 = RK[s]
        if s == 2:
            c1 = c1_stage2
        if s == 1:
            out.copy_(torch.from_numpy(Us.numpy() + dt * L))
        else:
            out.copy_(torch.from_numpy(c0 * Un.numpy() + c1 * (Us.numpy() + dt * L)))
    return stage, sel


@pytest.mark.parametrize("R", [5, 9])
def test_forced_replay_of_the_oracle_is_its_free_run(R):
    u, h = wl.advection_step(64)
    dt = 0.5 * h
    steps = [dt] * 20
    stage, sel = _fake_path(R, h)
    fin, V, flips, nst = forced_replay(
        stage, sel, lambda U: U.numpy().copy(),
        lambda V, s: oracle.rhs_advection(V, h, R, forced=s)["rhs"],
        torch.from_numpy(u.copy()), u, steps,
        lambda U, s: int((oracle.rhs_advection(U, h, R, want_sel=True)["sel"].reshape(-1)
                          != s).sum()))
    P = oracle.Problem(oracle.EQ_ADVECTION, R, 64, dx=h, bc=oracle.BC_PERIODIC)
    free = u.copy()
    for d in steps:
        free = P.step_ssprk3(free, d)
    assert flips == 0 and nst == 60
    assert np.array_equal(V, free)
    assert np.array_equal(fin, free)


def test_forced_replay_catches_a_wrong_stage_coefficient():
    R = 5
    u, h = wl.advection_step(64)
    dt = 0.5 * h
    stage, sel = _fake_path(R, h, c1_stage2=0.25 * (1 + 1e-9))
    fin, V, _, _ = forced_replay(
        stage, sel, lambda U: U.numpy().copy(),
        lambda V, s: oracle.rhs_advection(V, h, R, forced=s)["rhs"],
        torch.from_numpy(u.copy()), u, [dt] * 20)
    assert np.abs(fin - V).mean() > 1e-10


def test_assert_values_strict_bound():
    ref = np.array([1.0, -2.0, 0.5])
    # within 1e-12 ||L||: passes both bounds
    assert_values(ref + 1e-13, ref, 10.0)
    # a flux term far above ||L|| relaxes the bound to 1e-12 ||F||/h ...
    assert_values(ref + 1e-11, ref, 1e3)
    # ... but not where ||F||/h is within the strict ratio of ||L||
    with pytest.raises(AssertionError):
        assert_values(ref + 1e-11, ref, 10.0)
