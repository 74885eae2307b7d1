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
CELL, FLUX_DIFF, ADD, STAGE = 15, 2 * C, C, 7 * C / 3   # ops, per the model's table
EIGEN, ROE_AVG, PROJ, SPLIT = 16 + 19, 11, 20, 3


def _counts_and_work(U, R, axis, stage):
    import torch
    import bench
    ny, nx = U.shape[1:]
    n_lines, n = (ny, nx) if axis == 0 else (nx, ny)  # x sweep: the lines are rows
    n_int = n_lines * (n + 1)
    c = bench.sweep_counts(torch.from_numpy(U), axis, R)
    T = oracle.num_tested(R)
    sel = np.zeros(T + 3)
    sel[T + 2] = 2 * C * c[0]  # every window of a flat interface takes S(0,0)
    return c, bench.sweep_work(R, C, sel, n_int, c, stage_epilogue=stage), n_lines, n_int


@pytest.mark.parametrize("stage", [False, True])
def test_uniform_field(stage):
    n = 16
    U = wl.conserved_2d(np.full((n, n), 1.0), 0.1, 0.2, 1.0)
    c, (flops, ops), n_lines, n_int = _counts_and_work(U, 9, 0, stage)
    # every tile on one state: no flux difference anywhere
    assert c == (n_int, n_int, n_int, n_lines, 0)
    assert ops == pytest.approx(n_lines * CELL + n_int * (STAGE if stage else 0))
    assert flops == pytest.approx(n_lines * 18 + n_int * (4 * C if stage else 0))


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
    # but not on one state; every other interface is flat on one state; the
    # one tile along each line (n < 127) is not on one state
    assert c == (n_int, n_int - n_lines, n_int - n_lines, 2 * n_lines, n * n)
    expect = (2 * n_lines * CELL + n * n * FLUX_DIFF
              + n_lines * (EIGEN + ROE_AVG + 2 * PROJ + C * SPLIT))
    assert ops == expect
    # carrying the stage: the other sweep's part is added in the tiles not on
    # one state, and every cell takes the stage combination
    _, (_, ops_s), _, _ = _counts_and_work(U, 9, axis, True)
    assert ops_s == pytest.approx(expect + n * n * ADD + n_int * STAGE)


def _busy_brute(U, axis, R):
    """Cells in tiles not on one state per line, tile by tile and line by
    line (the sweep's geometry: TP - 1 cells written per tile, g staged
    beyond them on either side, ghost cells repeating the edge cell, the
    last line group padded with copies of the last line)."""
    import bench
    TP, NL = bench.SWEEP_TILES[axis]
    g = (R + 1) // 2
    X = U if axis == 0 else U.transpose(0, 2, 1)
    nl, n = X.shape[1], X.shape[2]
    total = 0
    for l0 in range(0, nl, NL):
        for x0 in range(0, n, TP - 1):
            varies = False
            for line in range(l0, l0 + NL):
                L = min(line, nl - 1)
                cells = [X[:, L, min(max(c, 0), n - 1)] for c in range(x0 - g, x0 + TP + g - 1)]
                varies = varies or any(not np.array_equal(a, b) for a, b in zip(cells, cells[1:]))
            if varies:
                total += (min(l0 + NL, nl) - l0) * (min(x0 + TP - 1, n) - x0)
    return total


@pytest.mark.parametrize("axis", [0, 1])
@pytest.mark.parametrize("R", [5, 17])
def test_busy_cells_brute_force(axis, R):
    import torch
    import bench
    rng = np.random.Generator(np.random.PCG64(R + axis))
    ny, nx = 37, 300
    rho = np.ones((ny, nx))
    for _ in range(4):  # a few jumps along random lines, at random places
        if axis == 0:
            rho[rng.integers(ny), rng.integers(nx):] = rng.uniform(0.5, 2.0)
        else:
            rho[rng.integers(ny):, rng.integers(nx)] = rng.uniform(0.5, 2.0)
    rho[:, 140:143] = 0.7 if axis == 0 else rho[:, 140:143]
    U = wl.conserved_2d(rho, 0.1, 0.2, 1.0)
    got = bench.busy_cells(torch.from_numpy(U), axis, R)
    assert got == _busy_brute(U, axis, R)
    assert 0 < got < nx * ny
