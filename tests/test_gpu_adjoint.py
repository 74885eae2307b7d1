"""Adjoint: transpose-Jacobian products of the RHS and of an SSP-RK3 step,
with the forward pass's discrete choices frozen.

Checks: dot-product identity <v, J d> = <J^T v, d> with J d from central
differences of the GPU RHS and from central differences of the oracle with
the GPU's selection forced (an oracle-side reference); the same for one
SSP-RK3 step; and the gradient of a loss after several steps through the
autograd wrapper against central differences.

Finite differences are only meaningful where no discrete choice changes
between U - eps d and U + eps d.  Directions are therefore smooth (a few low
Fourier modes times the state): a random per-cell perturbation would swamp
the top candidates' indicators of smooth data (which scale like h^(R-1)) and
flip selections everywhere.  Where an interface still flips, the cotangent
is masked on its two cells.  Data with exactly constant regions is avoided
in the FD checks because equal cells tie in the per-line alpha maxima.
"""
import numpy as np
import pytest

import oracle
from paper_2311_15504_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def E():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as ge
    ge.build_cuda()
    from paper_2311_15504_gb300 import enomr
    return enomr


def smooth_dir(U, seed):
    """State-shaped smooth direction: U times a sum of low Fourier modes."""
    rng = np.random.Generator(np.random.PCG64(seed))
    shape = U.shape[1:] if U.ndim > 1 else U.shape
    grids = np.meshgrid(*[np.arange(n) / n for n in shape], indexing="ij")
    comps = U.shape[0] if U.ndim > 1 else 1
    out = np.zeros((comps,) + shape)
    for c in range(comps):
        f = np.zeros(shape)
        for _ in range(3):
            k = rng.integers(1, 3, size=len(shape))
            f += rng.uniform(0.3, 1.0) * np.sin(2 * np.pi * sum(
                kk * gg for kk, gg in zip(k, grids)) + rng.uniform(0, 2 * np.pi))
        out[c] = f
    return (out.reshape(U.shape) * (np.abs(U) + 0.1))


def smooth_euler1d(n):
    """Periodic smooth 1D state with varying density, velocity and pressure
    (so that each per-line alpha maximum is attained at one cell)."""
    x = np.arange(n) / n
    rho = 1.0 + 0.2 * np.sin(2 * np.pi * x)
    u = 0.4 + 0.3 * np.sin(4 * np.pi * x + 1.0)
    p = 1.0 + 0.2 * np.cos(2 * np.pi * x + 0.3)
    return wl.conserved_1d(rho, u, p), 1.0 / n


def _cases(E):
    U2 = wl.smooth_random_euler2d(133, 70, seed=4)
    U1, h1 = smooth_euler1d(150)
    ua, ha = wl.advection_sine(300, power=2)
    ua = ua + 0.3 * np.cos(np.pi * np.linspace(-1, 1, 300, endpoint=False))
    return {
        "euler2d": (E.EULER, (70, 133), U2, dict(dx=1.0 / 133, dy=1.0 / 70, bc=E.PERIODIC)),
        "euler1d": (E.EULER, 150, U1, dict(dx=h1, bc=E.PERIODIC)),
        "advection": (E.ADVECTION, 300, ua, dict(dx=ha, bc=E.PERIODIC, adv_speed=-0.7)),
    }


def _flip_mask(s, sel0, sels, U):
    """1 on cells not adjacent to an interface whose selection flipped."""
    mask = np.ones(U.shape[1:] if U.ndim > 1 else U.shape)
    flips = np.zeros(sel0.shape, dtype=bool)
    for sl in sels:
        flips |= (sl != sel0)
    if not flips.any():
        return mask, 0
    if s.eq == 0:
        f = flips.reshape(2, s.nx + 1).any(axis=0)
        for k in np.nonzero(f)[0]:
            for c in (k - 1, k):
                mask[c % s.nx] = 0
    elif s.ndim == 1:
        f = flips.reshape(2, 3, s.nx + 1).any(axis=(0, 1))
        for k in np.nonzero(f)[0]:
            for c in (k - 1, k):
                mask[c % s.nx] = 0
    else:
        ny, nx = s.ny, s.nx
        nsx = 8 * ny * (nx + 1)
        fx = flips[:nsx].reshape(2, 4, ny, nx + 1).any(axis=(0, 1))
        fy = flips[nsx:].reshape(2, 4, nx, ny + 1).any(axis=(0, 1))
        for y, k in zip(*np.nonzero(fx)):
            mask[y, (k - 1) % nx] = mask[y, k % nx] = 0
        for x, k in zip(*np.nonzero(fy)):
            mask[(k - 1) % ny, x] = mask[k % ny, x] = 0
    return mask, int(flips.sum())


@pytest.mark.parametrize("case", ["euler2d", "euler1d", "advection"])
@pytest.mark.parametrize("R", [5, 9, 17])
def test_rhs_vjp_dot_product_fd(E, case, R):
    import torch
    eq, shape, U, kw = _cases(E)[case]
    s = E.Solver(eq, shape, order=R, **kw)
    Ud = torch.from_numpy(U).cuda()
    d = smooth_dir(U, R)
    v = np.random.Generator(np.random.PCG64(R + 1)).standard_normal(U.shape)
    dd = torch.from_numpy(d).cuda()
    eps = 1e-8
    Up, Um = Ud + eps * dd, Ud - eps * dd
    sel0 = s.selection(Ud).cpu().numpy()
    mask, nflip = _flip_mask(s, sel0, [s.selection(Up).cpu().numpy(),
                                       s.selection(Um).cpu().numpy()], U)
    assert nflip <= 0.02 * sel0.size
    v = v * (mask[None] if U.ndim > 1 else mask)
    vd = torch.from_numpy(v).cuda()
    jd = (s.rhs(Up) - s.rhs(Um)) / (2 * eps)
    lhs = float((vd * jd).sum())
    rhs = float((s.rhs_vjp(Ud, vd) * dd).sum())
    scale = float((vd.abs() * jd.abs()).sum())
    assert abs(lhs - rhs) <= 1e-6 * scale, (lhs, rhs, scale, nflip)
    # accumulate flag and scale
    out = torch.ones_like(Ud)
    s.rhs_vjp(Ud, vd, out=out, scale=2.0, accumulate=True)
    assert abs(float(((out - 1.0) * dd).sum()) - 2.0 * rhs) <= 1e-9 * abs(rhs) + 1e-12 * scale
    s.check_status()


@pytest.mark.parametrize("R", [5, 9, 17])
def test_rhs_vjp_against_oracle_frozen_fd(E, R):
    """Oracle-side reference: J d by central differences of the oracle with
    every discrete choice frozen -- the GPU's stencil choices forced and each
    per-line alpha taken at the oracle's maximising cell of U -- which makes
    it a smooth function of U.  Any direction works, including per-cell
    random ones."""
    import torch
    cases = _cases(E)
    for name in ("euler2d", "euler1d"):
        eq, shape, U, kw = cases[name]
        s = E.Solver(eq, shape, order=R, **kw)
        Ud = torch.from_numpy(U).cuda()
        sel = s.selection(Ud).cpu().numpy()
        rng = np.random.Generator(np.random.PCG64(7 + R))
        d = rng.standard_normal(U.shape) * (np.abs(U) + 0.1)
        v = rng.standard_normal(U.shape)
        eps = 1e-6
        if name == "euler2d":
            _, am = oracle.rhs_euler2d_frozen(U, kw["dx"], kw["dy"], R, sel, bc=0)
            f = lambda X: oracle.rhs_euler2d_frozen(X, kw["dx"], kw["dy"], R, sel, amax=am, bc=0)  # noqa: E731
        else:
            _, am = oracle.rhs_euler1d_frozen(U, kw["dx"], R, sel, bc=0)
            f = lambda X: oracle.rhs_euler1d_frozen(X, kw["dx"], R, sel, amax=am, bc=0)  # noqa: E731
        jd = (f(U + eps * d) - f(U - eps * d)) / (2 * eps)
        lhs = float((v * jd).sum())
        rhs = float((s.rhs_vjp(Ud, torch.from_numpy(v).cuda()).cpu().numpy() * d).sum())
        assert abs(lhs - rhs) <= 1e-7 * float(np.abs(v * jd).sum()), (name, lhs, rhs)


@pytest.mark.parametrize("case", ["euler2d", "euler1d", "advection"])
def test_step_vjp_dot_product_fd(E, case):
    import torch
    eq, shape, U, kw = _cases(E)[case]
    R = 9
    s = E.Solver(eq, shape, order=R, **kw)
    Ud = torch.from_numpy(U).cuda()
    dt = 0.5 * s.cfl_dt(Ud, 0.5)
    d = smooth_dir(U, 11)
    v = np.random.Generator(np.random.PCG64(12)).standard_normal(U.shape)
    dd, vd = torch.from_numpy(d).cuda(), torch.from_numpy(v).cuda()
    eps = 1e-9
    Up, Um = Ud + eps * dd, Ud - eps * dd
    s.step(Up, dt=dt)
    s.step(Um, dt=dt)
    jd = (Up - Um) / (2 * eps)
    lhs = float((vd * jd).sum())
    rhs = float((s.step_vjp(Ud, dt, vd) * dd).sum())
    assert abs(lhs - rhs) <= 1e-6 * float((vd.abs() * jd.abs()).sum()), (lhs, rhs)


def _loss_grad_check(E, s, U0, target, steps, d_list, comp=0):
    import torch
    tgt = torch.from_numpy(target).cuda()
    x = torch.from_numpy(U0).cuda().requires_grad_(True)
    out = E.rollout(x, s, steps, cfl=0.5)
    loss = 0.5 * ((out[comp] - tgt) ** 2).sum()
    loss.backward()
    grad = x.grad.detach()
    dts = []
    Ut = torch.from_numpy(U0).cuda()
    for _ in range(steps):
        dts.append(s.step(Ut, 0.0, 0.5, return_dt=True))

    def loss_at(U):
        Uc = U.clone()
        for dt in dts:
            s.step(Uc, dt=dt)
        return 0.5 * float(((Uc[comp] - tgt) ** 2).sum())

    base = torch.from_numpy(U0).cuda()
    for k, d in enumerate(d_list):
        dd = torch.from_numpy(d).cuda()
        eps = 1e-8
        fd = (loss_at(base + eps * dd) - loss_at(base - eps * dd)) / (2 * eps)
        ad = float((grad * dd).sum())
        assert abs(fd - ad) <= 1e-6 * abs(fd) + 1e-12, (k, fd, ad)


def test_rollout_gradient_smooth_field(E):
    """1/2 ||rho(t_n) - rho_target||^2 after 8 CFL steps of a smooth periodic
    2D field (64^2, order 9), along 3 smooth directions."""
    n, R = 64, 9
    U0 = wl.smooth_random_euler2d(n, n, seed=9)
    target = U0[0] * (1 + 0.01 * np.sin(2 * np.pi * np.arange(n) / n))[None, :]
    s = E.Solver(E.EULER, (n, n), order=R, dx=1.0 / n, dy=1.0 / n, bc=E.PERIODIC)
    _loss_grad_check(E, s, U0, target, 8, [smooth_dir(U0, 20 + k) for k in range(3)])


def test_rollout_gradient_vortex(E):
    """The isentropic vortex (128^2 on [0,10]^2, order 9, 8 steps) with a
    target density perturbed by 1e-3 noise.  Directions are localised to the
    vortex core: in the far field the state is flat to ~1e-11, so any
    perturbation there would change selections.  The centre is moved off the
    grid's symmetry axes: a centred vortex has mirror-equal cells that tie
    in the per-line alpha maxima, where max() has no derivative."""
    n, R = 128, 9  # ~20 cells across the core: resolved for the 9-point stencils
    U0, h, _ = wl.isentropic_vortex(n, centre=(5.0 + 0.37 * 10 / n, 5.0 - 0.21 * 10 / n))
    rng = np.random.Generator(np.random.PCG64(5))
    target = U0[0] + 1e-3 * rng.standard_normal((n, n))
    x = (np.arange(n) + 0.5) * h
    X, Y = np.meshgrid(x, x)
    bump = np.exp(-((X - 5.06) ** 2 + (Y - 4.97) ** 2) / 2.0)
    s = E.Solver(E.EULER, (n, n), order=R, dx=h, dy=h, bc=E.PERIODIC)
    _loss_grad_check(E, s, U0, target, 8,
                     [smooth_dir(U0, 30 + k) * bump[None] for k in range(3)])


def test_rollout_gradient_vortex_512_200_steps(E):
    """The adjoint workload at its stated size: isentropic vortex 512^2 on
    [0,10]^2 (periodic, order 9), 200 CFL steps with per-step checkpoints,
    loss 1/2 ||rho(t) - rho_target||^2 with the target's initial density
    perturbed by 1e-3 N(0,1).  Central differences along 8 seeded directions
    localised to the vortex core, 1e-6 relative.  Over 600 stage
    evaluations a perturbation of 1e-8 crosses near-ties of the selection
    somewhere (every direction did, changing the plain loss's derivative by
    0.5-20 %), so the differences are taken of the map the adjoint
    transposes: the +-eps runs are advanced stage by stage beside the
    reference trajectory with its discrete choices (enomr_stage_frozen with
    Uref = the reference stage state)."""
    import torch
    n, R, steps = 512, 9, 200
    h = 10.0 / n
    centre = (5.0 + 0.37 * h, 5.0 - 0.21 * h)
    U0, h, _ = wl.isentropic_vortex(n, centre=centre)
    rng = np.random.Generator(np.random.PCG64(2024))
    Ut0, _, _ = wl.isentropic_vortex(n, centre=centre)
    Ut0[0] = Ut0[0] + 1e-3 * rng.standard_normal((n, n))
    s = E.Solver(E.EULER, (n, n), order=R, dx=h, dy=h, bc=E.PERIODIC)
    # target run from the perturbed initial density, same step count
    Ut = torch.from_numpy(Ut0).cuda()
    for _ in range(steps):
        s.step(Ut, 0.0, 0.5)
    tgt = Ut[0].clone()
    torch.cuda.synchronize()
    torch.cuda.reset_peak_memory_stats()
    x = torch.from_numpy(U0).cuda().requires_grad_(True)
    out = E.rollout(x, s, steps, cfl=0.5)
    loss = 0.5 * ((out[0] - tgt) ** 2).sum()
    loss.backward()
    grad = x.grad.detach()
    peak = torch.cuda.max_memory_allocated()
    dts = []
    Uc = torch.from_numpy(U0).cuda()
    for _ in range(steps):
        dts.append(s.step(Uc, 0.0, 0.5, return_dt=True))
    assert abs(float(loss) - 0.5 * float(((Uc[0] - tgt) ** 2).sum())) <= 1e-12 * float(loss)

    xs = (np.arange(n) + 0.5) * h
    X, Y = np.meshgrid(xs, xs)
    bump = np.exp(-((X - centre[0]) ** 2 + (Y - centre[1]) ** 2) / 2.0)
    eps = 1e-8
    bufs = [torch.empty_like(Uc) for _ in range(9)]

    def frozen_fd(dd):
        """Central difference of the loss along dd of the frozen-choice map
        of the reference trajectory (the one the rollout took)."""
        b, p, m = x.detach().clone(), x.detach() + eps * dd, x.detach() - eps * dd
        B1, B2, B3, P1, P2, P3, M1, M2, M3 = bufs
        for dt in dts:
            for st, (bs, bo, ps, po, ms, mo) in enumerate(
                    ((b, B1, p, P1, m, M1), (B1, B2, P1, P2, M1, M2),
                     (B2, B3, P2, P3, M2, M3)), start=1):
                s.stage_frozen(st, p, ps, po, dt, bs)
                s.stage_frozen(st, m, ms, mo, dt, bs)
                s.stage(st, b, bs, bo, dt)
            b, B3 = B3, b
            p, P3 = P3, p
            m, M3 = M3, m
            bufs[2], bufs[5], bufs[8] = B3, P3, M3
        assert torch.equal(b, Uc)  # the reference trajectory is the rollout's
        lp = 0.5 * float(((p[0] - tgt) ** 2).sum())
        lm = 0.5 * float(((m[0] - tgt) ** 2).sum())
        return (lp - lm) / (2 * eps)

    for k in range(8):
        d = torch.from_numpy(smooth_dir(U0, 40 + k) * bump[None]).cuda()
        fd = frozen_fd(d)
        ad = float((grad * d).sum())
        rel = abs(fd - ad) / abs(fd)
        print(f"vortex 512^2, 200 steps, direction {k}: frozen-choice fd {fd:.12e} "
              f"adjoint {ad:.12e} rel {rel:.2e}")
        assert rel <= 1e-6, (k, fd, ad)
    print(f"vortex 512^2 x 200 steps: peak torch memory {peak / 2**30:.2f} GiB "
          f"(checkpoints {steps} x {U0.nbytes / 2**20:.0f} MiB)")
    s.check_status()


def test_stage_frozen_is_the_plain_stage_at_its_reference(E):
    """enomr_stage_frozen with Uref = Us: the plain stage up to the rounding
    of the one-state flat interfaces (which the frozen form evaluates in
    full); on a state without flat windows, bit for bit."""
    import torch
    n = 96
    U = wl.smooth_random_euler2d(n, n, seed=3)
    s = E.Solver(E.EULER, (n, n), order=9, dx=1.0 / n, dy=1.0 / n, bc=E.PERIODIC)
    Ud = torch.from_numpy(U).cuda()
    dt = 0.5 * s.cfl_dt(Ud, 0.5)
    a, b = torch.empty_like(Ud), torch.empty_like(Ud)
    s.stage(1, Ud, Ud, a, dt)
    s.stage_frozen(1, Ud, Ud, b, dt, Ud)
    assert torch.equal(a, b)
    Ur, dx, dy = wl.riemann2d(130, 70, seed=4)
    r = E.Solver(E.EULER, (70, 130), order=9, dx=dx, dy=dy, bc=E.TRANSMISSIVE)
    Urd = torch.from_numpy(Ur).cuda()
    for _ in range(3):
        r.step(Urd, 0.0, 0.5)
    dt = r.cfl_dt(Urd, 0.5)
    a, b = torch.empty_like(Urd), torch.empty_like(Urd)
    r.stage(1, Urd, Urd, a, dt)
    r.stage_frozen(1, Urd, Urd, b, dt, Urd)
    assert float((a - b).abs().max()) <= 1e-13 * float(a.abs().max())
    s.check_status()
    r.check_status()
