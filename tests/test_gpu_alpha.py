"""The per-line split speeds alpha_k and the CFL maximum on the GPU.

The reduction evaluates only representative cells (a cell bitwise equal to
its left neighbour, or to the one above, repeats that cell's speeds), so
these tests pin it to the plain maxima over all cells:
- invariance: a line's maxima do not depend on the order of its cells, so
  permuting the columns of a piecewise-constant field (which breaks its
  runs of equal cells into short ones) leaves every row's alpha bitwise
  unchanged and permutes the columns' alpha; likewise for rows;
- the values against the maxima of the per-cell speeds computed on the
  host (relative 1e-14: the GPU takes 1/rho and the square root its own
  way);
- the CFL step against the oracle's.
"""
import numpy as np
import pytest

import oracle
from paper_2311_15504_gb300 import workloads as wl

pytestmark = pytest.mark.gpu
GAMMA = 1.4


@pytest.fixture(scope="module")
def E():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as ge
    ge.build_cuda()
    from paper_2311_15504_gb300 import enomr
    return enomr


def dev(x):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def _field(nx, ny, seed):
    """Four quadrant states, a stripe of a fifth state, and a smooth patch
    in which every cell differs from its neighbours."""
    U, dx, dy = wl.riemann2d(nx, ny, seed=seed, xc=0.55, yc=0.4)
    rng = np.random.Generator(np.random.PCG64(seed))
    stripe = wl.conserved_2d(np.array([0.7]), 0.3, -0.2, 1.1)[:, 0]
    U[:, :, nx // 3:nx // 3 + 5] = stripe[:, None, None]
    U[:, ny // 5:ny // 5 + 2, :] = stripe[:, None, None]
    a, b = ny // 2, nx // 2
    h, w = min(40, ny - a), min(37, nx - b)
    patch = wl.conserved_2d(1.0 + 0.3 * rng.random((h, w)), rng.uniform(-1, 1, (h, w)),
                            rng.uniform(-1, 1, (h, w)), 1.0 + 0.5 * rng.random((h, w)))
    U[:, a:a + h, b:b + w] = patch
    return U, dx, dy


def _speeds(U):
    rho, u, v = U[0], U[1] / U[0], U[2] / U[0]
    p = (GAMMA - 1) * (U[3] - 0.5 * rho * (u * u + v * v))
    c = np.sqrt(GAMMA * p / rho)
    return u, v, c


def _alpha(E, U, dx, dy):
    ny, nx = U.shape[1:]
    s = E.Solver(E.EULER, (ny, nx), order=9, dx=dx, dy=dy, bc=E.TRANSMISSIVE)
    s.rhs(dev(U))
    ax, ay = s.debug_alpha()[:2]
    s.check_status()
    return ax.cpu().numpy(), ay.cpu().numpy()


@pytest.mark.parametrize("nx,ny", [(300, 200), (64, 96), (33, 31)])
def test_alpha_permutation_invariant_and_exact(E, nx, ny):
    U, dx, dy = _field(nx, ny, seed=nx)
    ax, ay = _alpha(E, U, dx, dy)
    rng = np.random.Generator(np.random.PCG64(ny))
    pc, pr = rng.permutation(nx), rng.permutation(ny)
    ax_c, ay_c = _alpha(E, U[:, :, pc], dx, dy)
    assert np.array_equal(ax_c, ax) and np.array_equal(ay_c, ay[pc])
    ax_r, ay_r = _alpha(E, U[:, pr, :], dx, dy)
    assert np.array_equal(ay_r, ay) and np.array_equal(ax_r, ax[pr])
    u, v, c = _speeds(U)
    ref_x = np.stack([np.abs(u - c).max(1), np.abs(u).max(1), np.abs(u + c).max(1)], 1)
    ref_y = np.stack([np.abs(v - c).max(0), np.abs(v).max(0), np.abs(v + c).max(0)], 1)
    assert np.allclose(ax, ref_x, rtol=1e-14, atol=0) and np.allclose(ay, ref_y, rtol=1e-14, atol=0)


def test_alpha_1d_permutation_invariant(E):
    rng = np.random.Generator(np.random.PCG64(3))
    N = 517
    rho = np.repeat(rng.uniform(0.5, 2.0, 11), 47)[:N]
    U = wl.conserved_1d(rho, np.repeat(rng.uniform(-1, 1, 11), 47)[:N], 1.0 + 0.0 * rho)
    U[:, 200:230] = wl.conserved_1d(1.0 + rng.random(30), rng.uniform(-1, 1, 30),
                                    1.0 + rng.random(30))
    out = []
    for V in (U, U[:, rng.permutation(N)]):
        s = E.Solver(E.EULER, N, order=7, dx=0.01, bc=E.TRANSMISSIVE)
        s.rhs(dev(V))
        out.append(s.debug_alpha()[0].cpu().numpy())
        s.check_status()
    assert np.array_equal(out[0], out[1])


def test_cfl_dt_of_piecewise_constant_field(E):
    U, dx, dy = _field(300, 200, seed=9)
    s = E.Solver(E.EULER, (200, 300), order=9, dx=dx, dy=dy, bc=E.TRANSMISSIVE)
    P = oracle.Problem(oracle.EQ_EULER2D, 9, 300, 200, dx=dx, dy=dy, bc=oracle.BC_TRANSMISSIVE)
    assert s.cfl_dt(dev(U), 0.5) == pytest.approx(P.cfl_dt(U, 0.5), rel=1e-14)
    s.check_status()


def test_nonphysical_cell_inside_a_constant_run_is_flagged(E):
    U, dx, dy = _field(128, 64, seed=4)
    U[3, 10, 60:80] = -1.0  # a run of equal cells with negative energy
    s = E.Solver(E.EULER, (64, 128), order=5, dx=dx, dy=dy, bc=E.TRANSMISSIVE)
    with pytest.raises(E.EnomrError):
        s.cfl_dt(dev(U), 0.5)
        s.check_status()
