"""Pins of the FP64 CPU oracle against what the mathematics fixes.

Each test checks the oracle against a closed form, an invariant or an
independent re-derivation, chosen so that a dropped term, a wrong sign, a
wrong stagger offset or a transposed operand fails at least one of them.
No GPU is needed.
"""
import itertools
import math

import numpy as np
import pytest

from oracle import oracle as O

RNG = np.random.Generator(np.random.Philox(777))


# ----------------------------------------------------------------- shapes
@pytest.mark.parametrize("order", [1, 2])
def test_shape_moments(order):
    """Partition of unity, exact first moment, and the second moment of the
    linear (f(1-f)) and quadratic (1/4) B-spline shapes."""
    for xi in RNG.uniform(-3.0, 3.0, 300):
        nodes = np.arange(math.floor(xi) - 3, math.floor(xi) + 4)
        S = np.array([O.shape(order, n - xi) for n in nodes])
        assert abs(S.sum() - 1.0) < 1e-14
        assert abs((nodes * S).sum() - xi) < 1e-13
        f = xi - math.floor(xi)
        m2 = ((nodes - xi) ** 2 * S).sum()
        assert abs(m2 - (f * (1.0 - f) if order == 1 else 0.25)) < 1e-13
    assert O.shape(2, 0.0) == 0.75 and O.shape(2, 1.0) == 0.125 and O.shape(2, 1.5) == 0.0
    assert O.shape(1, 0.0) == 1.0 and O.shape(1, 1.0) == 0.0


# ----------------------------------------------------------------- gather
STAG_E = [(0.5, 0, 0), (0, 0.5, 0), (0, 0, 0.5)]
STAG_B = [(0, 0.5, 0.5), (0.5, 0, 0.5), (0.5, 0.5, 0)]


def _fill_linear(grid, coef):
    """Every component F_c = a + b X + c Y + d Z + e X Y at its own staggered
    node positions (X, Y, Z)."""
    nz, ny, fx = grid.E[0].shape
    k, j, i = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(fx), indexing="ij")
    for arrs, stag, cset in ((grid.E, STAG_E, coef[:3]), (grid.B, STAG_B, coef[3:])):
        for c in range(3):
            X = (i + stag[c][0]) * grid.dx
            Y = (j + stag[c][1]) * grid.dy
            Z = (k + stag[c][2]) * grid.dz if grid.dim == 3 else 0.0
            a, b, cc, d, e = cset[c]
            arrs[c][...] = a + b * X + cc * Y + (d * Z if grid.dim == 3 else 0.0) + e * X * Y


@pytest.mark.parametrize("dim,order", [(2, 1), (2, 2), (3, 1), (3, 2)])
def test_gather_reproduces_bilinear_fields(dim, order):
    n = (14, 12, 11)[:dim]
    h = (0.3, 0.2, 0.25)[:dim]
    g = O.Grid(dim, n, h, 0.05, order)
    coef = RNG.uniform(-1, 1, (6, 5))
    _fill_linear(g, coef)
    for _ in range(50):
        pos = np.array([RNG.uniform(4.0, n[d] - 4.0) * h[d] for d in range(dim)])
        E, B = O.gather(g, pos)
        x, y = pos[0], pos[1]
        z = pos[2] if dim == 3 else 0.0
        for c in range(3):
            for val, cs in ((E[c], coef[c]), (B[c], coef[3 + c])):
                a, b, cc, d, e = cs
                expect = a + b * x + cc * y + (d * z if dim == 3 else 0.0) + e * x * y
                assert abs(val - expect) < 1e-12 * (1 + abs(expect))


# ------------------------------------------------------------------ Boris
def test_boris_rotation_angle_sign_and_norm():
    """E = 0: |u| is conserved and u_perp turns by -sign(q) 2 atan(|q| B dt / (2 m gamma))."""
    for _ in range(200):
        q = RNG.choice([-1.0, 1.0]) * RNG.uniform(0.5, 2.0)
        m = RNG.uniform(0.5, 3.0)
        dt = RNG.uniform(0.01, 0.5)
        u = RNG.normal(0, 1.0, 3)
        B = RNG.normal(0, 2.0, 3)
        u1 = O.boris(q, m, dt, u, [0, 0, 0], B)
        assert abs(np.linalg.norm(u1) - np.linalg.norm(u)) < 1e-13 * np.linalg.norm(u)
        bh = B / np.linalg.norm(B)
        assert abs(u1 @ bh - u @ bh) < 1e-13 * np.linalg.norm(u)
        p0, p1 = u - (u @ bh) * bh, u1 - (u1 @ bh) * bh
        ang = math.atan2(np.cross(p0, p1) @ bh, p0 @ p1)
        gam = math.sqrt(1 + u @ u)
        expect = -math.copysign(1.0, q) * 2 * math.atan(abs(q) * np.linalg.norm(B) * dt / (2 * m * gam))
        assert abs(ang - expect) < 1e-12


def test_boris_pure_electric_kick():
    """B = 0: u advances by q E dt / m exactly."""
    u = np.array([0.1, -0.2, 0.3])
    E = np.array([0.5, 0.25, -1.0])
    u1 = O.boris(-1.0, 2.0, 0.1, u, E, [0, 0, 0])
    assert np.allclose(u1, u + (-1.0 / 2.0) * 0.1 * E, rtol=0, atol=1e-15)


def _uniform_field_grid(Ez=(0, 0, 0), Bz=(0, 0, 0), n=64, h=0.1, order=1):
    g = O.Grid(2, (n, n), (h, h), 0.95 * h / math.sqrt(2), order)
    for c in range(3):
        g.E[c][...] = Ez[c]
        g.B[c][...] = Bz[c]
    return g


def test_larmor_circle_exact():
    """Uniform B: the integer-time positions x^n lie exactly on the Larmor
    circle r_L = m |u_perp| / (|q| B) (the x^{n+1/2} form a regular polygon
    whose side midpoints are the x^n)."""
    B0 = 2.0
    g = _uniform_field_grid(Bz=(0, 0, B0))
    u0 = np.array([0.3, 0.1, 0.2])
    sp = O.Species(-1.0, 1.0, np.array([[3.2], [3.2]]), u0.reshape(3, 1), [1e-3])
    pts = []
    for _ in range(80):
        O.push_species(g, sp)
        pts.append(sp.x[:2, 0].copy())
    P = np.array(pts)
    # algebraic circle fit
    A = np.c_[2 * P, np.ones(len(P))]
    sol, *_ = np.linalg.lstsq(A, (P ** 2).sum(1), rcond=None)
    c = sol[:2]
    r = np.linalg.norm(P - c, axis=1)
    rL = 1.0 * math.hypot(u0[0], u0[1]) / (1.0 * B0)
    assert np.max(np.abs(r - rL)) < 1e-10
    assert abs(sp.u[2, 0] - u0[2]) < 1e-15


def test_exb_drift():
    """Crossed uniform E_y and B_z: a particle launched at the drift velocity
    E x B / B^2 keeps it (gyration-free), and one launched at rest drifts at
    that velocity on average."""
    E0, B0 = 0.01, 1.0
    g = _uniform_field_grid(Ez=(0, E0, 0), Bz=(0, 0, B0), n=128)
    vd = E0 / B0
    ud = vd / math.sqrt(1 - vd * vd)
    sp = O.Species(1.0, 1.0, np.array([[1.0], [6.4]]), np.array([[ud], [0.0], [0.0]]), [1e-3])
    x0 = sp.x[0, 0]
    nsteps = 200
    for _ in range(nsteps):
        O.push_species(g, sp)
    vx = (sp.x[0, 0] - x0) / (nsteps * g.dt)
    assert abs(vx - vd) < 1e-6 * vd
    assert abs(sp.u[1, 0]) < 1e-6 * vd
    # from rest: average over whole discrete gyro-periods
    sp2 = O.Species(-1.0, 1.0, np.array([[1.0], [6.4]]), np.zeros((3, 1)), [1e-3])
    th = 2 * math.atan(B0 * g.dt / 2)
    per = 2 * math.pi / th
    nper = 12
    nst = int(round(nper * per))
    xs = [sp2.x[0, 0]]
    for _ in range(nst):
        O.push_species(g, sp2)
        xs.append(sp2.x[0, 0])
    vbar = (xs[-1] - xs[0]) / (nst * g.dt)
    assert abs(vbar - vd) < 0.02 * vd


# -------------------------------------------------------------- Esirkepov
def _single(grid, q, w, pos):
    return O.Species(q, 1.0, np.asarray(pos, float).reshape(-1, 1), np.zeros((3, 1)), [w])


def _divJ(grid):
    J = grid.J
    d = (J[0] - np.roll(J[0], 1, axis=2)) / grid.dx + (J[1] - np.roll(J[1], 1, axis=1)) / grid.dy
    if grid.dim == 3:
        d = d + (J[2] - np.roll(J[2], 1, axis=0)) / grid.dz
    return d


def _random_move(dim, n, h, frac=0.9):
    x0 = np.array([RNG.uniform(0, n[d]) * h[d] for d in range(dim)])
    # put some particles right at the periodic seam
    if RNG.random() < 0.3:
        x0[0] = RNG.choice([0.02, n[0] - 0.02]) * h[0]
    dx = np.array([RNG.uniform(-frac, frac) * h[d] for d in range(dim)])
    return x0, x0 + dx


@pytest.mark.parametrize("dim,order", [(2, 1), (2, 2), (3, 1), (3, 2)])
def test_esirkepov_continuity_and_total_current(dim, order):
    n = (8, 8, 8)[:dim]
    h = (0.3, 0.2, 0.25)[:dim]
    dt = 0.07
    for _ in range(60):
        g = O.Grid(dim, n, h, dt, order)
        q, w, vz = -1.0, RNG.uniform(0.5, 2.0), RNG.uniform(-0.5, 0.5)
        x0, x1 = _random_move(dim, n, h)
        O.deposit(g, q * w, x0, x1, vz)
        r0 = O.rho(g, _single(g, q, w, x0))
        r1 = O.rho(g, _single(g, q, w, x1))
        res = (r1 - r0) + dt * _divJ(g)
        assert np.max(np.abs(res)) < 1e-13 * np.max(np.abs(r0))
        dV = g.dV
        for d in range(dim):
            assert abs(g.J[d].sum() * dV - q * w * (x1[d] - x0[d]) / dt) < 1e-13 * abs(q * w)
        if dim == 2:
            assert abs(g.J[2].sum() * dV - q * w * vz) < 1e-13 * abs(q * w)


@pytest.mark.parametrize("dim,order", [(2, 1), (2, 2), (3, 1), (3, 2)])
def test_esirkepov_at_rest_deposits_nothing(dim, order):
    n = (8, 8, 8)[:dim]
    h = (0.3, 0.2, 0.25)[:dim]
    g = O.Grid(dim, n, h, 0.07, order)
    x0 = np.array([RNG.uniform(0, n[d]) * h[d] for d in range(dim)])
    O.deposit(g, 1.7, x0, x0, 0.0)
    for c in range(3):
        assert np.all(g.J[c] == 0.0)


def _periodic_shape(order, xi, n):
    s = np.zeros(n)
    for i in range(math.floor(xi) - 3, math.floor(xi) + 4):
        s[i % n] += O.shape(order, i - xi)
    return s


def _prefix_from(D, start):
    """Running sum of D along axis 0 starting (with zero) at index ``start``."""
    n = D.shape[0]
    out = np.zeros_like(D)
    run = np.zeros(D.shape[1:])
    for t in range(n):
        i = (start + t) % n
        run = run + D[i]
        out[i] = run
    return out


def _sequential_moves_J(dim, order, n, h, dt, qw, x0, x1, vz):
    """Independent construction: the current of a straight move is the average,
    over every order of the axes, of moving one axis at a time while the other
    shapes stay where they are; each one-axis move is fixed by 1D continuity.
    2D J_z is the path integral of the product of linearly interpolated shapes
    (Simpson's rule, exact for the quadratic integrand)."""
    S0 = [_periodic_shape(order, x0[d] / h[d], n[d]) for d in range(dim)]
    S1 = [_periodic_shape(order, x1[d] / h[d], n[d]) for d in range(dim)]
    start = [(math.floor(min(x0[d], x1[d]) / h[d]) - 3) % n[d] for d in range(dim)]
    J = [np.zeros(tuple(n[::-1]) if dim == 3 else (n[1], n[0])) for _ in range(3)]
    perms = list(itertools.permutations(range(dim)))
    for perm in perms:
        cur = list(S0)
        for d in perm:
            D = S1[d] - cur[d]
            others = [e for e in range(dim) if e != d]
            area = np.prod([h[e] for e in others]) if dim == 3 else h[others[0]]
            # tensor with axis order (d, others...) then moved to array layout
            if dim == 3:
                T = np.einsum("a,b,c->abc", D, cur[others[0]], cur[others[1]])
                flux = -qw / (dt * area) * _prefix_from(T, start[d])
                # axes are (d, o0, o1) in x/y/z numbering; array layout is (z, y, x)
                order_xyz = [d] + others
                flux = np.transpose(flux, np.argsort(order_xyz))      # -> (x, y, z)
                J[d] += np.transpose(flux, (2, 1, 0)) / len(perms)
            else:
                T = np.einsum("a,b->ab", D, cur[others[0]])
                flux = -qw / (dt * area) * _prefix_from(T, start[d])
                fl = flux if d == 0 else flux.T                         # -> (x, y)
                J[d] += fl.T / len(perms)
            cur[d] = S1[d]
    if dim == 2:
        f = lambda s: np.outer(S0[1] + s * (S1[1] - S0[1]), S0[0] + s * (S1[0] - S0[0]))
        Wz = (f(0.0) + 4 * f(0.5) + f(1.0)) / 6.0
        J[2] = qw * vz * Wz / (h[0] * h[1])
    return J


@pytest.mark.parametrize("dim,order", [(2, 1), (2, 2), (3, 1), (3, 2)])
def test_esirkepov_equals_sequential_move_average(dim, order):
    n = (9, 8, 7)[:dim]
    h = (0.3, 0.2, 0.25)[:dim]
    dt = 0.07
    for _ in range(25):
        g = O.Grid(dim, n, h, dt, order)
        qw, vz = RNG.uniform(-2, 2), RNG.uniform(-0.5, 0.5)
        x0, x1 = _random_move(dim, n, h)
        O.deposit(g, qw, x0, x1, vz)
        ref = _sequential_moves_J(dim, order, n, h, dt, qw, x0, x1, vz)
        scale = abs(qw) / (dt * min(h) ** 2)
        for c in range(3 if dim == 3 else 3):
            got = g.J[c] if dim == 3 else g.J[c][0]
            assert np.max(np.abs(got - ref[c])) < 1e-12 * scale, c


def test_villasenor_buneman_limit():
    """2D CIC, a move inside one cell: J_x(i+1/2, j) = qw dX (1 - ybar) / (dt dx dy),
    J_x(i+1/2, j+1) = qw dX ybar / (dt dx dy) with ybar the mean in-cell y."""
    n, h, dt = (8, 8), (0.3, 0.2), 0.07
    for _ in range(40):
        i, j = RNG.integers(1, 6, 2)
        f0, f1 = RNG.uniform(0.05, 0.95, 2), RNG.uniform(0.05, 0.95, 2)
        x0 = np.array([(i + f0[0]) * h[0], (j + f0[1]) * h[1]])
        x1 = np.array([(i + f1[0]) * h[0], (j + f1[1]) * h[1]])
        qw = RNG.uniform(-2, 2)
        g = O.Grid(2, n, h, dt, 1)
        O.deposit(g, qw, x0, x1, 0.0)
        dX, dY = x1 - x0
        yb, xb = 0.5 * (f0[1] + f1[1]), 0.5 * (f0[0] + f1[0])
        c = qw / (dt * h[0] * h[1])
        Jx, Jy = g.J[0][0], g.J[1][0]
        assert abs(Jx[j, i] - c * dX * (1 - yb)) < 1e-13 * abs(c)
        assert abs(Jx[j + 1, i] - c * dX * yb) < 1e-13 * abs(c)
        assert abs(Jy[j, i] - c * dY * (1 - xb)) < 1e-13 * abs(c)
        assert abs(Jy[j, i + 1] - c * dY * xb) < 1e-13 * abs(c)
        mask = np.ones_like(Jx, bool)
        mask[j, i] = mask[j + 1, i] = False
        assert np.max(np.abs(Jx[mask])) < 1e-13 * abs(c)


# ------------------------------------------------------------------- Yee
def _mode_run(grid, field, sample, nsteps):
    vals = []
    for _ in range(nsteps):
        O.maxwell_half(grid, 0)
        O.maxwell_half(grid, 1)
        vals.append(field()[sample])
    return np.array(vals)


def _check_recurrence(vals, cos_expect):
    big = np.abs(vals[1:-1]) > 0.3 * np.max(np.abs(vals))
    c = (vals[2:] + vals[:-2])[big] / (2 * vals[1:-1][big])
    assert big.sum() > 5
    assert np.max(np.abs(c - cos_expect)) < 1e-12


def _cos_w_dt(k, h, dt):
    s2 = dt * dt * sum((math.sin(kd * hd / 2) / hd) ** 2 for kd, hd in zip(k, h))
    return 1.0 - 2.0 * s2


@pytest.mark.parametrize("pol", ["Ez", "Bz"])
def test_yee_dispersion_2d(pol):
    """A discrete plane-wave eigenmode advances by exactly omega dt per step,
    sin^2(omega dt/2)/dt^2 = sum_d sin^2(k_d h_d/2)/h_d^2 (c = 1)."""
    n, h = (16, 12), (0.3, 0.2)
    dt = 0.9 / math.sqrt(sum(1 / x ** 2 for x in h))
    g = O.Grid(2, n, h, dt, 1)
    k = (2 * math.pi * 2 / (n[0] * h[0]), 2 * math.pi * 1 / (n[1] * h[1]))
    j, i = np.meshgrid(np.arange(n[1]), np.arange(n[0]), indexing="ij")
    if pol == "Ez":
        g.E[2][0] = np.cos(k[0] * i * h[0] + k[1] * j * h[1])
        field = lambda: g.E[2][0]
    else:
        g.B[2][0] = np.cos(k[0] * (i + 0.5) * h[0] + k[1] * (j + 0.5) * h[1])
        field = lambda: g.B[2][0]
    vals = _mode_run(g, field, (3, 5), 60)
    _check_recurrence(vals, _cos_w_dt(k, h, dt))


def test_yee_dispersion_3d():
    n, h = (6, 8, 10), (0.3, 0.2, 0.25)
    dt = 0.9 / math.sqrt(sum(1 / x ** 2 for x in h))
    g = O.Grid(3, n, h, dt, 1)
    k = (0.0, 2 * math.pi / (n[1] * h[1]), 2 * math.pi * 2 / (n[2] * h[2]))
    kk, jj, ii = np.meshgrid(np.arange(n[2]), np.arange(n[1]), np.arange(n[0]), indexing="ij")
    # E_x independent of x is divergence-free
    g.E[0][...] = np.cos(k[1] * jj * h[1] + k[2] * kk * h[2])
    vals = _mode_run(g, lambda: g.E[0], (3, 2, 1), 60)
    _check_recurrence(vals, _cos_w_dt(k, h, dt))


# ------------------------------------------------------- full-loop physics
def _thermal_state(dim, n, h, order, ppc, vth, seed):
    from paper_2607_13507_b300 import workloads as W
    wl = W.Workload("t", dim, n, h, W.cfl_dt(h), order, False,
                    [W.SpeciesSpec(q=-1.0, m=1.0, ppc=ppc, vth=vth)], 1, seed=seed)
    p = W.load_species(wl, 0)
    g = O.Grid(dim, n, h, wl.dt, order)
    x = (p.cell + p.off) * np.array(h)[:, None]
    return g, O.Species(p.q, p.m, x, p.u, p.w)


def _rho_at(g, sp, shift):
    x = sp.x.copy()
    gam = np.sqrt(1 + (sp.u ** 2).sum(0))
    x[: g.dim] += shift * g.dt * sp.u[: g.dim] / gam
    return O.rho(g, O.Species(sp.q, sp.m, x[: g.dim], sp.u, sp.w))


@pytest.mark.parametrize("dim,order", [(2, 1), (2, 2), (3, 2)])
def test_gauss_law_constancy(dim, order):
    """div E - (rho(x - dt v/2) + rho(x + dt v/2)) / 2 is the same after every
    step: E changes only through the deposited current, which conserves the
    charge of the half-step positions exactly."""
    n = (12, 10, 8)[:dim]
    h = (0.1,) * dim
    g, sp = _thermal_state(dim, n, h, order, 4, 0.2, 99)
    G = []
    for s in range(6):
        O.step(g, [sp], s * g.dt)
        G.append(O.div_e(g) - 0.5 * (_rho_at(g, sp, -0.5) + _rho_at(g, sp, 0.5)))
    scale = np.max(np.abs(_rho_at(g, sp, 0.0)))
    for Gs in G[1:]:
        assert np.max(np.abs(Gs - G[0])) < 1e-12 * scale


def test_cold_langmuir_frequency_and_stability():
    """Cold plasma with a small sinusoidal velocity: E_x oscillates at omega
    with sin(omega dt/2) = omega_p dt/2 (to the 1% finite-grid level) and its
    amplitude neither grows nor decays by more than 1% over three periods."""
    nx, ny, h = 64, 4, 0.1
    dt = 0.95 * h / math.sqrt(2)
    g = O.Grid(2, (nx, ny), (h, h), dt, 1)
    ppx = 2
    xs = (np.arange(nx * ppx) + 0.5) * h / ppx
    ys = (np.arange(ny * ppx) + 0.5) * h / ppx
    X, Y = np.meshgrid(xs, ys, indexing="ij")
    X, Y = X.ravel(), Y.ravel()
    npart = X.size
    w = 1.0 * h * h / (ppx * ppx)
    L = nx * h
    k = 2 * math.pi / L
    V = 1e-3
    u = np.zeros((3, npart))
    u[0] = V * np.sin(k * X)
    sp = O.Species(-1.0, 1.0, np.stack([X, Y]), u, np.full(npart, w))
    xe = (np.arange(nx) + 0.5) * h
    amp = []
    for s in range(300):
        O.step(g, [sp], s * dt)
        amp.append(np.mean(g.E[0][0], axis=0) @ np.sin(k * xe) * 2 / nx)
    a = np.array(amp)
    c = np.sum((a[2:] + a[:-2]) * a[1:-1]) / np.sum(2 * a[1:-1] ** 2)
    w_meas = math.acos(c) / dt
    w_theory = 2 * math.asin(dt / 2) / dt
    assert abs(w_meas / w_theory - 1) < 0.01
    per = int(round(2 * math.pi / w_meas / dt))
    first = np.max(np.abs(a[:per]))
    last = np.max(np.abs(a[-per:]))
    assert abs(last / first - 1) < 0.01


def test_translation_by_whole_cells_commutes_with_a_step():
    dim, n, h, order = 2, (10, 12), (0.1, 0.1), 2
    g, sp = _thermal_state(dim, n, h, order, 3, 0.1, 5)
    for c in range(3):
        g.E[c][...] = RNG.normal(0, 0.01, g.E[c].shape)
        g.B[c][...] = RNG.normal(0, 0.01, g.B[c].shape)
    g2 = O.Grid(dim, n, h, g.dt, order)
    sh = (3, 2)   # cells in x, y
    for c in range(3):
        g2.E[c][...] = np.roll(g.E[c], sh, axis=(2, 1))
        g2.B[c][...] = np.roll(g.B[c], sh, axis=(2, 1))
    x2 = sp.x.copy()
    for d in range(dim):
        x2[d] = np.mod(x2[d] + sh[d] * h[d], n[d] * h[d])
    sp2 = O.Species(sp.q, sp.m, x2[:dim], sp.u.copy(), sp.w.copy())
    O.step(g, [sp], 0.0)
    O.step(g2, [sp2], 0.0)
    for c in range(3):
        assert np.max(np.abs(np.roll(g.E[c], sh, axis=(2, 1)) - g2.E[c])) < 1e-12
        assert np.max(np.abs(np.roll(g.J[c], sh, axis=(2, 1)) - g2.J[c])) < 1e-10
    assert np.max(np.abs(sp.u - sp2.u)) < 1e-12


# --------------------------------------------------- absorbing edge + laser
def test_mur_edge_injects_and_absorbs_plane_wave():
    """Plane-wave laser through the x-min edge: the field 20 cells in follows
    the incident waveform, and once the pulse has left through x-max almost
    no energy stays in the box (first-order Mur, normal incidence)."""
    lam = 2 * math.pi
    dx = lam / 32
    nx, ny = 256, 4
    dt = 0.95 * dx / math.sqrt(2)
    laser = O.Laser(a0=1.0, w0=1e9, tau=2 * lam, omega=1.0, yc=0.0)
    g = O.Grid(2, (nx, ny), (dx, dx), dt, 1, absorb_x=True, laser=laser)
    probe = 20
    err, peak_e = 0.0, 0.0
    T = laser.tau + nx * dx + 8.0
    nst = int(T / dt)
    for s in range(nst):
        t = s * dt
        O.step(g, [], t)
        ey = g.E[1][0, 1, probe]
        inc = O.laser_ey(g, probe * dx, 1.5 * dx, 0.0, t + dt)
        err = max(err, abs(ey - inc))
        ek, ef, _ = O.energy(g, [])
        peak_e = max(peak_e, ef)
    assert err < 0.02 * laser.a0
    assert ef < 1e-4 * peak_e


@pytest.mark.parametrize("dim,order", [(2, 1), (2, 2), (3, 1), (3, 2)])
def test_free_streaming_relativistic_step(dim, order):
    """No fields: u is unchanged, x advances by dt u / gamma, and the step's
    current carries q w v (v = u / gamma, all three components) and sits on
    the path from x + dt v / 2 to x + 3 dt v / 2."""
    n = (10, 9, 8)[:dim]
    h = (0.3, 0.2, 0.25)[:dim]
    dt = 0.9 / math.sqrt(sum(1 / x ** 2 for x in h))
    for _ in range(10):
        g = O.Grid(dim, n, h, dt, order)
        u = RNG.normal(0, 2.0, 3)
        gam = math.sqrt(1 + u @ u)
        v = u / gam
        x0 = np.array([RNG.uniform(0, n[d]) * h[d] for d in range(dim)])
        q, w = -1.0, 0.37
        sp = O.Species(q, 1.0, x0.reshape(-1, 1), u.reshape(3, 1), [w])
        O.push_species(g, sp)
        L = np.array(n) * np.array(h)
        xe = np.mod(x0 + dt * v[:dim], L)
        assert np.max(np.abs(sp.x[:dim, 0] - xe)) < 1e-12
        assert np.max(np.abs(sp.u[:, 0] - u)) == 0.0
        for c in range(3):
            assert abs(g.J[c].sum() * g.dV - q * w * v[c]) < 1e-12 * w
        ref = O.Grid(dim, n, h, dt, order)
        O.deposit(ref, q * w, x0 + 0.5 * dt * v[:dim], x0 + 1.5 * dt * v[:dim], v[2])
        for c in range(3):
            assert np.max(np.abs(ref.J[c] - g.J[c])) < 1e-12 * w / min(h) ** 2
