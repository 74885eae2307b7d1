"""The TMA-staged 2D sweeps against the sweeps that stage with plain loads.

Both stagings run the same arithmetic on the same staged values, so their
right-hand sides, selections and steps must agree bit for bit.  The shapes
cover tiles at both ends of the lines (ghosts filled after the copy),
ragged last tiles, line counts that are not a multiple of the tile's lines
(rows or columns past the grid), lines shorter than one tile, both boundary
types and every order; the CUDA path's agreement with the oracle is checked
by the parity tests, which take the TMA path wherever nx is even.
"""
import numpy as np
import pytest

from paper_2311_15504_gb300 import workloads as wl

pytestmark = pytest.mark.gpu
ORDERS = [5, 7, 9, 11, 13, 15, 17]


@pytest.fixture(scope="module")
def E():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as ge
    ge.build_cuda()
    from paper_2311_15504_gb300 import enomr
    return enomr


def _pair(E, shape, R, dx, dy, bc):
    ny, nx = shape
    a = E.Solver(E.EULER, shape, order=R, dx=dx, dy=dy, bc=bc)
    b = E.Solver(E.EULER, shape, order=R, dx=dx, dy=dy, bc=bc)
    a.set_staging(E.STAGING_LOADS)
    b.set_staging(E.STAGING_TMA)
    return a, b


def _state(kind, ny, nx, seed):
    if kind == "riemann":
        U, dx, dy = wl.riemann2d(nx, ny, seed=seed)
        return U, dx, dy
    U = wl.smooth_random_euler2d(nx, ny, seed=seed)
    return U, 1.0 / nx, 1.0 / ny


SHAPES = [(70, 130), (9, 254), (33, 260), (1, 300), (131, 2), (40, 18), (257, 384)]


@pytest.mark.parametrize("R", ORDERS)
@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("kind,bc", [("riemann", 1), ("smooth", 0)])
def test_tma_rhs_and_selection_bitwise(E, R, shape, kind, bc):
    import torch
    ny, nx = shape
    g = (R + 1) // 2
    if bc == 0 and (nx < 2 * g or ny < 2 * g):
        pytest.skip("periodic lines need at least 2g cells")
    U, dx, dy = _state(kind, ny, nx, seed=R + nx)
    a, b = _pair(E, shape, R, dx, dy, bc)
    Ud = torch.from_numpy(U).cuda()
    ra, rb = a.rhs(Ud), b.rhs(Ud)
    assert torch.equal(ra, rb), float((ra - rb).abs().max())
    assert torch.equal(a.selection(Ud), b.selection(Ud))
    Ua, Ub = Ud.clone(), Ud.clone()
    for _ in range(2):
        a.step(Ua, 0.0, 0.4)
        b.step(Ub, 0.0, 0.4)
    assert torch.equal(Ua, Ub)
    a.check_status()
    b.check_status()


def test_tma_requires_even_rows_and_aligned_state(E):
    import torch
    U, dx, dy = wl.riemann2d(133, 40, seed=1)
    s = E.Solver(E.EULER, (40, 133), order=9, dx=dx, dy=dy, bc=E.TRANSMISSIVE)
    Ud = torch.from_numpy(U).cuda()
    ref = s.rhs(Ud)  # automatic staging: plain loads for odd nx
    s.set_staging(E.STAGING_TMA)
    with pytest.raises(E.EnomrError):
        s.rhs(Ud)
    # an 8-byte offset state (not 16-byte aligned): automatic staging falls
    # back to plain loads, the TMA-only setting refuses it
    U2, dx, dy = wl.riemann2d(130, 40, seed=2)
    s2 = E.Solver(E.EULER, (40, 130), order=9, dx=dx, dy=dy, bc=E.TRANSMISSIVE)
    buf = torch.empty(U2.size + 1, dtype=torch.float64, device="cuda")
    Uo = buf[1:].view(4, 40, 130)
    Uo.copy_(torch.from_numpy(U2))
    Ua = torch.from_numpy(U2).cuda()
    r_auto = s2.rhs(Uo)
    s2.set_staging(E.STAGING_TMA)
    assert torch.equal(s2.rhs(Ua), r_auto)
    with pytest.raises(E.EnomrError):
        s2.rhs(Uo)
    s.check_status()
    s2.check_status()
    assert ref.shape == Ud.shape


def test_tma_full_size_steps_bitwise(E):
    """The benchmark workload (4096^2, order 9): two CFL steps with each
    staging, bitwise equal."""
    import torch
    n = 4096
    U, dx, dy = wl.riemann2d(n, n, seed=0)
    a, b = _pair(E, (n, n), 9, dx, dy, E.TRANSMISSIVE)
    Ua = torch.from_numpy(U).cuda()
    Ub = Ua.clone()
    for _ in range(2):
        a.step(Ua, 0.0, 0.5)
        b.step(Ub, 0.0, 0.5)
    assert torch.equal(Ua, Ub)
    a.check_status()
    b.check_status()


@pytest.mark.parametrize("R", [5, 9, 17])
@pytest.mark.parametrize("kind,bc,shape", [("riemann", 1, (70, 300)), ("smooth", 0, (64, 96)),
                                          ("riemann", 1, (33, 131))])
def test_occupancy_and_staging_instances_bitwise(E, R, kind, bc, shape):
    """Every sweep instance -- plain loads or TMA, high or low occupancy --
    gives the same right-hand side, selections and steps bit for bit (odd
    nx: the TMA setting is refused and the loading instances run)."""
    import torch
    ny, nx = shape
    U, dx, dy = _state(kind, ny, nx, seed=R + 7 * nx)
    s = E.Solver(E.EULER, shape, order=R, dx=dx, dy=dy, bc=bc)
    Ud = torch.from_numpy(U).cuda()
    ref = None
    for stg in (E.STAGING_LOADS, E.STAGING_TMA, E.STAGING_AUTO):
        for occ in (E.OCCUPANCY_HIGH, E.OCCUPANCY_LOW, E.OCCUPANCY_AUTO):
            s.set_staging(stg)
            s.set_occupancy(occ)
            if stg == E.STAGING_TMA and nx % 2:
                with pytest.raises(E.EnomrError):
                    s.rhs(Ud)
                continue
            r = s.rhs(Ud)
            sel = s.selection(Ud)
            Us = Ud.clone()
            s.step(Us, 0.0, 0.4)
            s.step(Us, 0.0, 0.4)
            if ref is None:
                ref = (r, sel, Us)
            else:
                assert torch.equal(r, ref[0]), (stg, occ)
                assert torch.equal(sel, ref[1]), (stg, occ)
                assert torch.equal(Us, ref[2]), (stg, occ)
    s.check_status()
