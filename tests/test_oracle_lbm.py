"""Pins of the CPU FP64 oracle's time step against mathematics the paper fixes:
the textbook moment basis, exact invariants, the BGK + Guo special case, the planar
mechanical-stability coexistence, the Laplace law, and exactness of the FD stencils
(no GPU)."""
import math

import numpy as np
import pytest

import workloads as W
from oracle import oracle, thermo

CX = np.array([0, 1, 0, -1, 0, 1, -1, -1, 1])
CY = np.array([0, 0, 1, 0, -1, 1, 1, -1, -1])
WEQ = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)
EPS = np.finfo(np.float64).eps


@pytest.fixture(scope="module")
def pr08():
    e = thermo.PR()
    T = 0.8 * e.Tc
    rv, rl, _ = thermo.maxwell(e, T)
    return e, T, rv, rl


def test_moment_matrix_is_lallemand_luo_basis():
    # rows of M are the textbook polynomials of the lattice velocities (Lallemand & Luo 2000)
    M, Minv = oracle.matrices()
    c2 = CX ** 2 + CY ** 2
    rows = [np.ones(9), -4 + 3 * c2, 4 - 21 / 2 * c2 + 9 / 2 * c2 ** 2, CX, (-5 + 3 * c2) * CX, CY,
            (-5 + 3 * c2) * CY, CX ** 2 - CY ** 2, CX * CY]
    np.testing.assert_array_equal(M, np.array(rows))
    np.testing.assert_allclose(Minv @ M, np.eye(9), atol=1e-15)
    G = M @ M.T
    np.testing.assert_array_equal(G, np.diag(np.diag(G)))


def test_uniform_state_is_a_fixed_point(pr08):
    e, T, rv, rl = pr08
    cfg = W.base_config(9, 5, sigma=0.1, kappa=0.3, gy=-1e-4, s=[1.0, 0.8, 0.8, 1.0, 1.1, 1.0, 1.1, 1.3, 1.3])
    rho = np.full((5, 9), 2.5)
    z = np.zeros((5, 9))
    o = oracle.Oracle(cfg, rho, z, z, np.full((5, 9), T))
    f0 = o.f.copy()
    o.step(10)
    np.testing.assert_allclose(o.f, f0, rtol=0, atol=20 * EPS)


def test_mass_and_momentum_exact_in_periodic_box(pr08):
    # S_0 = C_0 = 0 and streaming permutes populations: sum rho is invariant; the
    # Shan-Chen force and g (rho - rho_bar) sum to zero over a periodic box, and
    # m*_3 = j + F for any rate s_j, so sum_i f_i c_i is invariant as well.
    e, T, rv, rl = pr08
    cfg, ic = W.static_droplet(e.Tc, rv, rl, nx=40, ny=33, R0=9.0, kappa=0.2)
    cfg.update(gx=2e-5, gy=-3e-5, s=[1.0, 0.8, 0.8, 0.7, 1.1, 0.7, 1.1, 1.2, 1.2])
    o = oracle.Oracle(cfg, *ic)
    m0 = o.f.sum()
    jx0 = np.tensordot(CX, o.f, axes=(0, 0)).sum()
    jy0 = np.tensordot(CY, o.f, axes=(0, 0)).sum()
    n = 150
    o.step(n)
    assert abs(o.f.sum() - m0) / m0 < n * 4 * EPS
    scale = o.f.sum() * 0.1
    assert abs(np.tensordot(CX, o.f, axes=(0, 0)).sum() - jx0) < n * 16 * EPS * scale
    assert abs(np.tensordot(CY, o.f, axes=(0, 0)).sum() - jy0) < n * 16 * EPS * scale
    fl = o.fields()
    assert abs(np.abs(fl["ux"]).max()) < 0.05


def _bgk_guo_step(f, tau, e, T, G, gx, gy):
    """Textbook BGK with Guo forcing and the Shan-Chen force (Guo 2002), periodic."""
    rho = f.sum(axis=0)
    psi = e.psi(rho, T)
    wf = np.array([0, 1 / 3, 1 / 3, 1 / 3, 1 / 3, 1 / 12, 1 / 12, 1 / 12, 1 / 12])
    sx = np.zeros_like(rho)
    sy = np.zeros_like(rho)
    for i in range(1, 9):
        nb = np.roll(np.roll(psi, -CX[i], axis=1), -CY[i], axis=0)
        sx += wf[i] * nb * CX[i]
        sy += wf[i] * nb * CY[i]
    rbar = rho.mean()
    Fx = -G * psi * sx + gx * (rho - rbar)
    Fy = -G * psi * sy + gy * (rho - rbar)
    ux = (np.tensordot(CX, f, axes=(0, 0)) + Fx / 2) / rho
    uy = (np.tensordot(CY, f, axes=(0, 0)) + Fy / 2) / rho
    out = np.empty_like(f)
    for i in range(9):
        cu = CX[i] * ux + CY[i] * uy
        feq = WEQ[i] * rho * (1 + 3 * cu + 4.5 * cu * cu - 1.5 * (ux * ux + uy * uy))
        src = WEQ[i] * ((3 * (CX[i] - ux) + 9 * cu * CX[i]) * Fx + (3 * (CY[i] - uy) + 9 * cu * CY[i]) * Fy)
        post = f[i] - (f[i] - feq) / tau + (1 - 1 / (2 * tau)) * src
        out[i] = np.roll(np.roll(post, CX[i], axis=1), CY[i], axis=0)
    return out


def test_single_rate_mrt_reduces_to_bgk_guo(pr08):
    # Sec. 2: with sigma = 0 the Li source is Guo forcing; with kappa = 0 and every
    # rate equal to 1/tau the MRT operator is BGK.
    e, T, rv, rl = pr08
    tau = 0.8
    nx, ny = 23, 17
    cfg = W.base_config(nx, ny, s=[1 / tau] * 9, gx=1e-4, gy=-2e-4)
    rho = W.random_smooth_density(nx, ny, 1.0, 5.5, seed=3)
    ux = 0.01 * np.sin(2 * np.pi * np.arange(nx) / nx)[None, :] * np.ones((ny, 1))
    uy = np.zeros((ny, nx))
    o = oracle.Oracle(cfg, rho, ux, uy, np.full((ny, nx), T))
    f = o.f.copy()
    for _ in range(4):
        f = _bgk_guo_step(f, tau, e, T, -1.0, 1e-4, -2e-4)
    o.step(4)
    np.testing.assert_allclose(o.f, f, rtol=1e-11, atol=1e-13)


def test_planar_coexistence_matches_mechanical_stability(pr08):
    # Sec. 3.2 Eq. (integral_coexistence_curve): a planar interface settles on the
    # densities of the mechanical-stability integral at the given sigma. The lattice
    # interface is ~4 nodes wide at a = 3/49, so the vapour density carries an O(dx^2)
    # discretisation error of a few 0.1% (halving dx cuts it ~3x: slow test below).
    e, T, rv, rl = pr08
    mv, ml, _ = thermo.mechanical_coexistence(e, T, 0.1)
    nx = 128
    cfg = W.base_config(nx, 4, sigma=0.1)
    o = oracle.Oracle(cfg, *W.slab_fields(nx, 4, nx / 4, 3 * nx / 4, 3.0, rl, rv, T))
    o.step(20000)
    r = o.fields()["rho"][0]
    assert r.min() == pytest.approx(mv, rel=5e-3)
    assert r.max() == pytest.approx(ml, rel=1e-3)
    # the vapour branch is very sensitive to the sigma term: 20% less sigma moves it by ~27%
    mv8, _, _ = thermo.mechanical_coexistence(e, T, 0.08)
    assert abs(mv8 / mv - 1) > 0.2


@pytest.mark.slow
def test_planar_coexistence_error_shrinks_with_refinement():
    # Eq. (a-deltax): a -> a/4 is one halving of dx; the interface doubles in width.
    errs = []
    for afac, nx, steps in ((1.0, 128, 20000), (0.25, 256, 40000)):
        e = thermo.PR(a=3 / 49 * afac)
        T = 0.8 * e.Tc
        rv, rl, _ = thermo.maxwell(e, T)
        mv, ml, _ = thermo.mechanical_coexistence(e, T, 0.1)
        cfg = W.base_config(nx, 4, a=e.a, sigma=0.1)
        o = oracle.Oracle(cfg, *W.slab_fields(nx, 4, nx / 4, 3 * nx / 4, 3.0 / math.sqrt(afac), rl, rv, T))
        o.step(steps)
        r = o.fields()["rho"][0]
        errs.append(abs(r.min() / mv - 1))
    assert errs[1] < errs[0] / 2.5


@pytest.mark.slow
def test_laplace_law_and_kappa_scaling(pr08):
    # Eq. (laplace-equation): dP = gamma / R, with gamma the planar tension of
    # Eq. (surface_tension), which is linear in (1 - kappa) (the kappa terms cancel in
    # the normal stress, so the profile does not change). Finite-width interfaces
    # (w/R ~ 0.2-0.3) allow a few % curvature corrections.
    e, T, rv, rl = pr08
    g0 = thermo.planar_gamma(e, T, 0.1, 0.0)

    def run(R0, kappa):
        cfg, ic = W.static_droplet(e.Tc, rv, rl, nx=64, ny=64, R0=R0, kappa=kappa)
        o = oracle.Oracle(cfg, *ic)
        o.step(3000)
        r = o.fields()["rho"]
        rin, rout = r[31:33, 31:33].mean(), r[0:2, 0:2].mean()
        dP = float(e.p(rin, T) - e.p(rout, T))
        R = math.sqrt(((r - rout) / (rin - rout)).sum() / math.pi)
        return dP, R

    dP9, R9 = run(9.0, 0.0)
    dP15, R15 = run(15.0, 0.0)
    dPk, Rk = run(15.0, 0.5)
    assert dP9 / dP15 == pytest.approx(R15 / R9, rel=5e-2)
    assert dP15 * R15 == pytest.approx(g0, rel=6e-2)
    assert (dPk * Rk) / (dP15 * R15) == pytest.approx(0.5, rel=3e-2)


def test_fd_operator_exact_on_polynomials(pr08):
    # The lattice-weight stencils are exact for quadratic T and linear rho, u, so the
    # discrete operator equals Eq. (energy-equation) evaluated analytically.
    e, T0, rv, rl = pr08
    nx, ny = 12, 11
    cfg = W.base_config(nx, ny, cv=4.0, lambda_l=3.0, lambda_v=0.5, rho_l=rl, rho_v=rv)
    y, x = np.mgrid[0:ny, 0:nx].astype(np.float64)
    T = T0 * (1 + 0.01 * x - 0.02 * y + 3e-4 * x * x + 2e-4 * x * y - 1e-4 * y * y)
    rho = 3.0 + 0.05 * x + 0.07 * y
    ux = 1e-3 + 2e-4 * x - 1e-4 * y
    uy = -2e-3 + 3e-4 * x + 1e-4 * y
    L = oracle.energy_rhs(cfg, rho, ux, uy, T)
    Tx = T0 * (0.01 + 6e-4 * x + 2e-4 * y)
    Ty = T0 * (-0.02 + 2e-4 * x - 2e-4 * y)
    lapT = T0 * (6e-4 - 2e-4)
    lam = (3.0 * (rho - rv) + 0.5 * (rl - rho)) / (rl - rv)
    dlam = (3.0 - 0.5) / (rl - rv)
    div = 2e-4 + 1e-4
    want = (-(ux * Tx + uy * Ty) + (lam * lapT + dlam * (0.05 * Tx + 0.07 * Ty)) / (rho * 4.0)
            - T * e.dp_dT(rho, T) * div / (rho * 4.0))
    inner = (slice(1, ny - 1), slice(1, nx - 1))
    np.testing.assert_allclose(L[inner], want[inner], rtol=1e-11, atol=1e-16)


def test_fd_operator_wall_mirror_exact(pr08):
    # Adiabatic walls at y = 0 and y = ny-1 mirror rho, T and u_x and flip u_y: fields
    # even about y = 0 (u_y odd) keep the stencils exact on the wall row.
    e, T0, rv, rl = pr08
    nx, ny = 10, 9
    cfg = W.base_config(nx, ny, cv=5.0, lambda_l=2.0, lambda_v=0.4, rho_l=rl, rho_v=rv,
                        hydro_bc=[W.PERIODIC, W.PERIODIC, W.WALL, W.WALL],
                        thermal_bc=[W.T_PERIODIC, W.T_PERIODIC, W.T_ADIABATIC, W.T_ADIABATIC])
    y, x = np.mgrid[0:ny, 0:nx].astype(np.float64)
    T = T0 * (1 + 2e-3 * y * y)
    rho = 3.0 + 0.01 * y * y
    ux = 1e-3 * np.ones_like(x)
    uy = 2e-4 * y
    L = oracle.energy_rhs(cfg, rho, ux, uy, T)
    Ty = T0 * 4e-3 * y
    lam = (2.0 * (rho - rv) + 0.4 * (rl - rho)) / (rl - rv)
    dlam_y = (2.0 - 0.4) / (rl - rv) * 0.02 * y
    want = (-(uy * Ty) + (lam * T0 * 4e-3 + dlam_y * Ty) / (rho * 5.0)
            - T * e.dp_dT(rho, T) * 2e-4 / (rho * 5.0))
    np.testing.assert_allclose(L[0], want[0], rtol=1e-11, atol=1e-16)
    np.testing.assert_allclose(L[1:4], want[1:4], rtol=1e-11, atol=1e-16)


@pytest.mark.parametrize("u0", [(0.0, 0.0), (0.03, -0.02)])
def test_heun_amplification_of_a_fourier_mode(pr08, u0):
    # Uniform rho and u, and a small Fourier mode of T. To first order in its
    # amplitude eps the mode is an eigenvector of the semi-discrete operator with
    # eigenvalue z = -i u.g(k) + alpha Lap(k); psi(rho, T) also feels the mode, so
    # the Shan-Chen force drives div u = (G psi psi_T / (2 rho)) (g_W . g) eps, and
    # the compression term adds a stage-independent source c. One Heun step maps the
    # amplitude d to d (1 + z + z^2/2) + c (1 + z/2) (RK2 with frozen coefficients).
    e, T0, rv, rl = pr08
    nx, ny = 16, 12
    rho0, cv, lam, G = 2.0, 5.0, 0.6, -1.0
    cfg = W.base_config(nx, ny, cv=cv, lambda_l=lam, lambda_v=lam, rho_l=rl, rho_v=rv, energy_on=1)
    kx, ky = 2 * np.pi * 2 / nx, 2 * np.pi * 1 / ny
    y, x = np.mgrid[0:ny, 0:nx].astype(np.float64)
    eps = 1e-7 * T0
    T = T0 + eps * np.cos(kx * x + ky * y)
    o = oracle.Oracle(cfg, np.full((ny, nx), rho0), np.full((ny, nx), u0[0]), np.full((ny, nx), u0[1]), T)
    o.step(1)
    kc = kx * CX + ky * CY
    wf = np.array([0, 1 / 3, 1 / 3, 1 / 3, 1 / 3, 1 / 12, 1 / 12, 1 / 12, 1 / 12])
    lap = 6 * np.sum(WEQ * (np.cos(kc) - 1))
    g = np.array([3 * np.sum(WEQ * CX * np.sin(kc)), 3 * np.sum(WEQ * CY * np.sin(kc))])
    gw = np.array([np.sum(wf * CX * np.sin(kc)), np.sum(wf * CY * np.sin(kc))])
    z = -1j * (u0[0] * g[0] + u0[1] * g[1]) + lam / (rho0 * cv) * lap
    psi0 = float(e.psi(rho0, T0))
    pT = float(e.dp_dT(rho0, T0))
    psiT = pT / (G * psi0)
    div_amp = G * psi0 * psiT / (2 * rho0) * (gw @ g)
    c = -T0 * pT * div_amp / (rho0 * cv)
    amp = (1 + z + z * z / 2) + c * (1 + z / 2)
    want = eps * np.real(amp * np.exp(1j * (kx * x + ky * y)))
    got = o.T - T0
    assert abs(c) > 1e-3 * abs(z)  # the coupling is really exercised
    np.testing.assert_allclose(got, want, rtol=0, atol=1e-6 * eps)


def test_boundary_invariants_after_a_step(pr08):
    # Dirichlet nodes hold their value; the outflow column is a copy of the first
    # interior column.
    e = pr08[0]
    rv, rl, _ = thermo.maxwell(e, 0.86 * e.Tc)
    cfg, ic = W.stefan_strip(e.Tc, rv, rl, 0.1032, nx=40, ny=3, n_vapour=8)
    o = oracle.Oracle(cfg, *ic)
    o.step(30)
    f = o.f
    np.testing.assert_array_equal(o.T[:, 0], cfg["T_side"][0])
    np.testing.assert_array_equal(f[:, :, -1], f[:, :, -2])
    np.testing.assert_array_equal(o.T[:, -1], o.T[:, -2])


def test_psi_argument_error_is_reported():
    # A supercritical-pressure state with p > rho/3 has no real psi (Eq. psi, G = -1).
    e = thermo.PR()
    cfg = W.base_config(6, 5)
    rho = np.full((5, 6), 9.0)  # close to 1/b: p blows up
    z = np.zeros((5, 6))
    o = oracle.Oracle(cfg, rho, z, z, np.full((5, 6), 2.0 * e.Tc))
    with pytest.raises(FloatingPointError):
        o.step(1)


def test_wall_film_reaches_no_slip_rest(pr08):
    # A liquid film on a psi-based wall (Zou-He wet nodes at y = 0 and y = ny-1) settles
    # to rest: with the half-force velocity the no-slip wall node carries the momentum
    # -F/2, so u -> 0 there as the force field becomes steady (an unforced closure would
    # leave u = F/(2 rho) at the wall, O(1e-1) here).
    e, T, rv, rl = pr08
    nx, ny = 6, 40
    cfg = W.base_config(nx, ny, sigma=0.1, hydro_bc=[W.PERIODIC, W.PERIODIC, W.WALL, W.WALL],
                        rho_w_side=[0.0, 0.0, rl, rv])
    rho = 0.5 * (rl + rv) + 0.5 * (rl - rv) * np.tanh(2.0 * (15.0 - np.arange(ny)) / 3.0)
    rho = np.repeat(rho[:, None], nx, axis=1)
    z = np.zeros((ny, nx))
    o = oracle.Oracle(cfg, rho, z, z, np.full((ny, nx), T))
    o.step(4000)
    fl = o.fields()
    assert np.abs(fl["uy"][[0, -1]]).max() < 1e-6   # the relaxation decays ~e-fold per 200 steps
    assert np.abs(fl["uy"]).max() < 1e-5
    assert np.abs(fl["ux"]).max() < 1e-12
    assert fl["rho"][:, 0].max() == pytest.approx(rl, rel=0.05)


@pytest.mark.parametrize("steps,g", [(1, 3e-5), (2, 0.0)])
def test_window_step_reproduces_the_full_domain(steps, g):
    # A window padded by 3 nodes per step on its open sides depends on nothing outside the
    # padding, so its nodes equal those of the whole-domain step (rho_bar given).
    e = thermo.PR()
    rv, rl, _ = thermo.maxwell(e, 0.86 * e.Tc)
    cfg, ic = W.pool_boiling(e.Tc, rv, rl, 0.1032, nx=40, ny=36, g=g, g_ref_height=36)
    full = oracle.Oracle(cfg, *ic)
    full.step(steps)
    rbar = float(np.mean(ic[0]))
    for (x0, x1, y0, y1) in [(0, 12, 0, 9), (30, 40, 5, 20), (14, 26, 28, 36), (35, 45, 10, 14)]:
        f, T = oracle.window_step(cfg, ic, x0, x1, y0, y1, rbar, steps=steps)
        xs = np.arange(x0, x1) % 40
        np.testing.assert_allclose(f, full.f[:, y0:y1][:, :, xs], rtol=1e-12, atol=1e-14)
        np.testing.assert_allclose(T, full.T[y0:y1][:, xs], rtol=1e-12, atol=0)


def _smooth_wall_state(nx, ny, rv, rl, T0, seed):
    rng = np.random.default_rng(seed)
    y, x = np.mgrid[0:ny, 0:nx].astype(float)
    rho = 0.5 * (rl + rv) + 0.45 * (rl - rv) * np.sin(2 * np.pi * x / nx + rng.random()) * np.cos(np.pi * y / ny)
    T = T0 * (1.0 + 0.02 * np.cos(2 * np.pi * y / ny + rng.random()))
    ux = 0.01 * np.sin(2 * np.pi * y / ny)
    uy = 0.01 * np.cos(2 * np.pi * x / nx)
    return rho, ux, uy, T


@pytest.mark.parametrize("axis", ["y", "x"])
def test_modified_psi_model_reduces_to_psi_based(pr08, axis):
    # Eq. (mod-psi-based-formula) with G_w = G gives the force of Eq. (psi-based-formula)
    # when psi_w = psi(x), i.e. rho_w(x) equal to the wall node's own density (same T), and
    # Eq. (Q-mod-psi-based) equals Eq. (Q-psi-based) then (psi_w - psi = 0 on solid links).
    # With G_w = 0 and kappa = 0 it equals the psi-based model with rho_w = 0 (psi_w = 0).
    e, T, rv, rl = pr08
    nx, ny = (10, 14) if axis == "y" else (14, 10)
    rho, ux, uy, T0 = _smooth_wall_state(nx, ny, rv, rl, T, 4)
    if axis == "x":
        rho, ux, uy, T0 = rho.T.copy(), uy.T.copy(), ux.T.copy(), T0.T.copy()
        nx, ny = ny, nx
    hb = [W.PERIODIC, W.PERIODIC, W.WALL, W.WALL] if axis == "y" else [W.WALL, W.WALL, W.PERIODIC, W.PERIODIC]
    base = W.base_config(nx, ny, sigma=0.1, kappa=0.4, hydro_bc=hb, s=W.RATES_STEFAN_POOL)
    lines = ([rho[0, :], rho[-1, :]] if axis == "y" else [rho[:, 0], rho[:, -1]])
    rho_w = [None] * 4
    lo, hi = (2, 3) if axis == "y" else (0, 1)
    rho_w[lo], rho_w[hi] = lines[0].copy(), lines[1].copy()
    ic = (rho, ux, uy, T0)

    a = oracle.Oracle(dict(base, rho_w=rho_w), *ic)
    b = oracle.Oracle(dict(base, contact_model=W.CONTACT_MOD_PSI, G_w=base["G"]), *ic)
    a.step(1)
    b.step(1)
    np.testing.assert_allclose(b.f, a.f, rtol=1e-13, atol=1e-15)

    k0 = dict(base, kappa=0.0)
    c = oracle.Oracle(dict(k0, rho_w_side=[0.0] * 4), *ic)
    d = oracle.Oracle(dict(k0, contact_model=W.CONTACT_MOD_PSI, G_w=0.0), *ic)
    c.step(1)
    d.step(1)
    np.testing.assert_allclose(d.f, c.f, rtol=1e-13, atol=1e-15)
    # and the adhesion is not a no-op: another G_w changes the wall rows only at first
    g = oracle.Oracle(dict(base, contact_model=W.CONTACT_MOD_PSI, G_w=-0.8), *ic)
    g.step(1)
    assert np.abs(g.f - b.f).max() > 1e-4


def _wall_momentum(f, row):
    """Population momentum sum_i f_i c_i on one row of wall nodes."""
    return (np.tensordot(CX, f[:, row, :], axes=1), np.tensordot(CY, f[:, row, :], axes=1))


def test_body_force_poiseuille_between_zou_he_walls(pr08):
    # Uniform fluid between two wet-node walls (y = 0 and y = H = ny-1), psi-based walls
    # whose density equals the bulk density (so F^m and F^ads vanish), driven along x by the
    # body force g (rho - rho_bar) of Eq. (gravitational_force) with rho_bar held below rho:
    # a uniform force F. The steady half-force velocity (Eq. DensityAndVelocityRelationToF)
    # is the plane Poiseuille parabola u(y) = F y (H - y) / (2 rho nu), nu = c_s^2 (tau - 1/2),
    # zero on the wall nodes. A closure that left the wall momentum at 0 (unforced) or got the
    # tangential term's factor wrong leaves the wall node at u = O(F / rho) instead.
    e, T, rv, rl = pr08
    rho0 = rl
    nx, ny = 4, 21
    H = ny - 1
    g, drho = 2e-6, 1.0
    cfg = W.base_config(nx, ny, hydro_bc=[W.PERIODIC, W.PERIODIC, W.WALL, W.WALL],
                        rho_w_side=[0.0, 0.0, rho0, rho0], gx=g, rho_l=rl, rho_v=rv)
    cfg["rho_bar_fixed"] = rho0 - drho
    F = g * drho
    nu = (1.0 / 3.0) * (1.0 / cfg["s"][7] - 0.5)
    z = np.zeros((ny, nx))
    o = oracle.Oracle(cfg, np.full((ny, nx), rho0), z, z, np.full((ny, nx), T))
    o.step(20000)  # ~ 8 viscous times H^2 / nu
    fl = o.fields()
    y = np.arange(ny, dtype=np.float64)
    u_exact = F * y * (H - y) / (2.0 * rho0 * nu)
    umax = u_exact.max()
    assert np.abs(fl["ux"][[0, -1]]).max() < 1e-9 * umax  # no slip on the wall nodes
    np.testing.assert_allclose(fl["ux"], np.repeat(u_exact[:, None], nx, axis=1), rtol=0, atol=1e-8 * umax)
    assert np.abs(fl["uy"]).max() < 1e-9 * umax
    np.testing.assert_allclose(fl["rho"], rho0, rtol=1e-9)


def test_zou_he_wall_momentum_is_minus_half_the_force_of_the_streaming_step(pr08):
    # Reading of the forced Zou-He closure: after step n the wall node's population momentum
    # J^{n+1} = sum f^{n+1} c equals -F^n / 2, F^n being the force of step n at that node. The
    # half-force velocity of state n (Eq. DensityAndVelocityRelationToF) gives that force
    # from the oracle's own outputs, F^n = 2 (rho^n u^n - J^n), so the check needs no second
    # implementation of the force. A transient (a perturbed liquid film relaxing, gravity on)
    # makes F change every step, so a closure that used the new step's force, or any other
    # factor, fails.
    e, T, rv, rl = pr08
    nx, ny = 8, 24
    cfg = W.base_config(nx, ny, sigma=0.1, kappa=0.2, gx=1e-4, gy=-2e-4,
                        hydro_bc=[W.PERIODIC, W.PERIODIC, W.WALL, W.WALL],
                        rho_w_side=[0.0, 0.0, 0.8 * rl, 1.3 * rv], rho_l=rl, rho_v=rv)
    yy, xx = np.mgrid[0:ny, 0:nx].astype(np.float64)
    rho = 0.5 * (rl + rv) + 0.5 * (rl - rv) * np.tanh(2.0 * (10.0 + 1.5 * np.sin(2 * np.pi * xx / nx) - yy) / 3.0)
    ux = 1e-3 * np.sin(2 * np.pi * yy / ny)
    o = oracle.Oracle(cfg, rho, ux, np.zeros((ny, nx)), np.full((ny, nx), T))
    checked = 0
    for _ in range(40):
        fl = o.fields()
        f0 = o.f.copy()
        o.step(1)
        for row in (0, ny - 1):
            jx0, jy0 = _wall_momentum(f0, row)
            Fx = 2.0 * (fl["rho"][row] * fl["ux"][row] - jx0)
            Fy = 2.0 * (fl["rho"][row] * fl["uy"][row] - jy0)
            jx1, jy1 = _wall_momentum(o.f, row)
            np.testing.assert_allclose(jx1, -0.5 * Fx, rtol=0, atol=1e-14)
            np.testing.assert_allclose(jy1, -0.5 * Fy, rtol=0, atol=1e-14)
            assert np.abs(Fy).max() > 1e-4  # a real force at the wall, varying in time
            checked += 1
    assert checked == 80


def test_psi_based_adhesion_single_wall_node_by_hand(pr08):
    # Eq. (psi-based-formula) with Eq. (shanchen-walls), one wall node of a uniform fluid at
    # rest: the fluid links of a bottom wall node (c = +x, -x, +y, +x+y, -x+y) carry
    # psi_0 each and the solid links (-y, +x-y, -x-y) carry psi_w = psi(rho_w, T), so with
    # G = -1 the total force is F = (0, psi_0 (psi_0 - psi_w) / 2) (the y components of the
    # weights of either set sum to 1/2; x cancels), and minus that on a top wall. Interior
    # nodes feel nothing. The half-force velocity of the initial state (J = 0) is F / (2 rho).
    e, T, rv, rl = pr08
    rho0 = 1.7
    nx, ny = 5, 9
    rw_bot, rw_top = 4.2, 0.9
    cfg = W.base_config(nx, ny, hydro_bc=[W.PERIODIC, W.PERIODIC, W.WALL, W.WALL],
                        rho_w_side=[0.0, 0.0, rw_bot, rw_top], rho_l=rl, rho_v=rv)
    z = np.zeros((ny, nx))
    o = oracle.Oracle(cfg, np.full((ny, nx), rho0), z, z, np.full((ny, nx), T))
    fl = o.fields()
    psi = lambda r: math.sqrt(2.0 * (float(e.p(r, T)) - r / 3.0) / cfg["G"])
    p0 = psi(rho0)
    Fb = 0.5 * p0 * (p0 - psi(rw_bot))
    Ft = -0.5 * p0 * (p0 - psi(rw_top))
    np.testing.assert_allclose(fl["uy"][0], Fb / (2.0 * rho0), rtol=1e-13)
    np.testing.assert_allclose(fl["uy"][-1], Ft / (2.0 * rho0), rtol=1e-13)
    assert np.abs(fl["ux"]).max() < 1e-17
    assert np.abs(fl["uy"][1:-1]).max() < 1e-17
