"""The algorithmic work model behind the bench's roofline fraction
(`bench.sweep_work`, `bench.flat_interfaces`), checked on CPU against hand
counts for fields whose interface classes are known: a uniform field (every
interface flat on one state, one distinct cell per line) and a field with one
jump per line (one flat interface between two states per line)."""
import os
import sys

import numpy as np
import pytest

import oracle
from paper_2311_15504_gb300 import workloads as wl

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

C = 4
CELL, FLUX_DIFF, STAGE = 15, 2 * C, 4 * C        # ops, per the model's table
EIGEN, ROE_AVG, PROJ, SPLIT = 16 + 19, 11, 20, 3


def _counts_and_work(U, R, axis, stage):
    import torch
    import bench
    ny, nx = U.shape[1:]
    n_lines, n = (ny, nx) if axis == 0 else (nx, ny)  # x sweep: the lines are rows
    n_int = n_lines * (n + 1)
    c = bench.flat_interfaces(torch.from_numpy(U), axis)
    T = oracle.num_tested(R)
    sel = np.zeros(T + 3)
    sel[T + 2] = 2 * C * c[0]  # every window of a flat interface takes S(0,0)
    return c, bench.sweep_work(R, C, sel, n_int, c, stage_epilogue=stage), n_lines, n_int


@pytest.mark.parametrize("stage", [False, True])
def test_uniform_field(stage):
    n = 16
    U = wl.conserved_2d(np.full((n, n), 1.0), 0.1, 0.2, 1.0)
    c, (flops, ops), n_lines, n_int = _counts_and_work(U, 9, 0, stage)
    assert c == (n_int, n_int, n_int, n_lines)
    assert ops == n_lines * CELL + n_int * (FLUX_DIFF + (STAGE if stage else 0))
    assert flops == n_lines * 18 + n_int * (2 * C + (6 * C if stage else 0))


@pytest.mark.parametrize("axis", [0, 1])
def test_one_jump_per_line(axis):
    n, k = 20, 9
    rho = np.full((n, n), 1.0)
    if axis == 0:
        rho[:, k:] = 0.5
    else:
        rho[k:, :] = 0.5
    U = wl.conserved_2d(rho, 0.1, 0.2, 1.0)
    c, (flops, ops), n_lines, n_int = _counts_and_work(U, 9, axis, False)
    # per line: the jump interface is flat (three equal cells on each side)
    # but not on one state; every other interface is flat on one state
    assert c == (n_int, n_int - n_lines, n_int - n_lines, 2 * n_lines)
    expect = (2 * n_lines * CELL + n_int * FLUX_DIFF
              + n_lines * (EIGEN + ROE_AVG + 2 * PROJ + C * SPLIT))
    assert ops == expect
