"""Pins of the oracle's cross-mesh differences (Sec. 4.3, Eqs. rel-diff-timestep and
global-rel-diff) against hand-computed cases, exactness of linear interpolation, and the
second-order error of bilinear interpolation of a smooth field."""
import numpy as np
import pytest

from oracle import norms


def test_periodic_hand_case():
    # coarse nodes at x = 1/4, 3/4 with values 0, 4 (periodic); fine nodes at 1/8 .. 7/8:
    # 1/8 lies between 3/4 - 1 (value 4) and 1/4 (value 0), a quarter from the first
    coarse = np.array([[0.0, 4.0]] * 2)
    got = norms.interpolate(coarse, (4, 4), True, True)
    np.testing.assert_allclose(got, np.array([[1.0, 1.0, 3.0, 3.0]] * 4), atol=1e-15)


def test_bounded_hand_case():
    # 2x2 coarse on the corners of the square, 3x3 fine: mid-edges and centre are averages
    coarse = np.array([[0.0, 1.0], [2.0, 3.0]])
    want = np.array([[0.0, 0.5, 1.0], [1.0, 1.5, 2.0], [2.0, 2.5, 3.0]])
    np.testing.assert_allclose(norms.interpolate(coarse, (3, 3), False, False), want, atol=1e-15)


def test_mixed_axes_hand_case():
    # x periodic (2 -> 4 nodes), y bounded (2 -> 3 nodes): the y midpoint averages the rows
    coarse = np.array([[0.0, 4.0], [8.0, 12.0]])
    got = norms.interpolate(coarse, (3, 4), True, False)
    row0 = np.array([1.0, 1.0, 3.0, 3.0])
    np.testing.assert_allclose(got, np.stack([row0, row0 + 4.0, row0 + 8.0]), atol=1e-14)


def test_linear_field_is_reproduced_on_bounded_axes():
    nxc, nyc, nxf, nyf = 7, 5, 19, 13
    f = lambda X, Y: 1.5 + 2.0 * X - 3.0 * Y + 0.25 * X * Y  # bilinear: exact under I
    Xc, Yc = np.meshgrid(norms.positions(nxc, False), norms.positions(nyc, False))
    Xf, Yf = np.meshgrid(norms.positions(nxf, False), norms.positions(nyf, False))
    num, den = norms.rel_diff_terms(f(Xc, Yc), f(Xf, Yf), False, False)
    assert num < 1e-12 * den


@pytest.mark.parametrize("px,py", [(True, True), (False, False), (True, False)])
def test_same_mesh_is_identity(px, py):
    a = np.random.default_rng(3).random((9, 11)) + 1.0
    num, den = norms.rel_diff_terms(a, a, px, py)
    assert num < 1e-13 * den
    assert den == pytest.approx(np.abs(a).sum(), rel=1e-15)


def test_constant_fields_and_denominator():
    num, den = norms.rel_diff_terms(np.full((4, 6), 2.0), np.full((9, 13), 3.0), True, False)
    assert num == pytest.approx(9 * 13 * 1.0, rel=1e-14)
    assert den == pytest.approx(9 * 13 * 3.0, rel=1e-14)


def test_brute_force_nodes():
    # a few fine nodes evaluated by the textbook bilinear formula written out here
    rng = np.random.default_rng(11)
    nxc, nyc, nxf, nyf = 6, 5, 15, 11
    c = rng.random((nyc, nxc))
    got = norms.interpolate(c, (nyf, nxf), True, False)
    for (j, i) in [(0, 0), (4, 7), (10, 14), (7, 2)]:
        X = (i + 0.5) * nxc / nxf - 0.5  # periodic x, in coarse index units
        Y = j * (nyc - 1) / (nyf - 1)  # bounded y
        i0, j0 = int(np.floor(X)), min(int(np.floor(Y)), nyc - 2)
        wx, wy = X - i0, Y - j0
        v = lambda jj, ii: c[jj, ii % nxc]
        want = ((1 - wy) * ((1 - wx) * v(j0, i0) + wx * v(j0, i0 + 1))
                + wy * ((1 - wx) * v(j0 + 1, i0) + wx * v(j0 + 1, i0 + 1)))
        assert got[j, i] == pytest.approx(want, rel=1e-14, abs=1e-15)


def test_second_order_convergence_of_a_smooth_field():
    field = lambda n: (lambda X, Y: 2.0 + np.sin(2 * np.pi * X) * np.cos(2 * np.pi * Y))(
        *np.meshgrid(norms.positions(n, True), norms.positions(n, True)))
    d1 = norms.rel_diff(field(16), field(32), True, True)
    d2 = norms.rel_diff(field(32), field(64), True, True)
    assert norms.convergence_order(d1, d2, 1 / 16, 1 / 32) == pytest.approx(2.0, abs=0.05)


def test_global_difference_sums_over_times():
    rng = np.random.default_rng(5)
    pairs = [(rng.random((4, 5)) + 1, rng.random((8, 10)) + 1) for _ in range(3)]
    terms = [norms.rel_diff_terms(c, f, True, True) for c, f in pairs]
    D = norms.global_rel_diff(pairs, True, True)
    assert D == pytest.approx(sum(t[0] for t in terms) / sum(t[1] for t in terms), rel=1e-15)
    # one time: D = d; the same time twice: D = d
    d = norms.rel_diff(*pairs[0], True, True)
    assert norms.global_rel_diff(pairs[:1], True, True) == pytest.approx(d, rel=1e-15)
    assert norms.global_rel_diff([pairs[0]] * 2, True, True) == pytest.approx(d, rel=1e-15)


def test_convergence_order_of_a_power_law():
    assert norms.convergence_order(3.0 * 0.1 ** 1.7, 3.0 * 0.05 ** 1.7, 0.1, 0.05) == pytest.approx(1.7)


def test_phase_area_limits_and_disc():
    assert norms.phase_area(np.full((5, 7), 0.3), 0.3, 6.0) == 0.0
    assert norms.phase_area(np.full((5, 7), 6.0), 0.3, 6.0) == 35.0
    assert norms.phase_area(np.array([[0.0, 3.15, 9.0]]), 0.3, 6.0) == pytest.approx(0.5 + 1.0)
    # a tanh disc of radius R0 and width W: the continuum integral of the fraction
    # 1/2 (1 + tanh(2 (R0 - d) / W)) over the plane is pi R0^2 + pi^3 W^2 / 48
    # (the odd part cancels; the even part is (W/2)^2 * 2 * int u / (e^{2u} + 1) du)
    n, R0, W = 96, 20.0, 3.0
    y, x = np.mgrid[0:n, 0:n]
    d = np.hypot(x - (n - 1) / 2, y - (n - 1) / 2)
    rho = 0.3 + 0.5 * (6.0 - 0.3) * (1 + np.tanh(2 * (R0 - d) / W))
    assert norms.phase_area(rho, 0.3, 6.0) == pytest.approx(np.pi * R0 ** 2 + np.pi ** 3 * W ** 2 / 48, rel=1e-4)


def test_relative_change_hand_case():
    assert norms.relative_change_R([1.0, 2.0, 3.0], [1.0, 2.5, 2.0]) == pytest.approx(1.5 / 5.5)
    assert norms.relative_change_R([4.0, 4.0], [4.0, 4.0]) == 0.0


@pytest.mark.parametrize("side", [0, 1, 2, 3])
def test_wall_heat_flux_exact_on_quadratic_profiles(side):
    # the one-sided difference is exact for quadratics; constant lambda at rho = rho_v
    ny, nx = 9, 12
    y, x = np.mgrid[0:ny, 0:nx].astype(float)
    n = {0: x, 1: nx - 1 - x, 2: y, 3: ny - 1 - y}[side]  # inward distance from the side
    T = 1.0 + 0.3 * n - 0.02 * n ** 2
    rho = np.full((ny, nx), 0.4)
    q = norms.wall_heat_flux(rho, T, side, 0.4, 6.0, 0.7, 3.0)
    assert q == pytest.approx(-0.7 * 0.3, rel=1e-13)  # dT/dn = 0.3 at the line


def test_wall_heat_flux_lambda_law_and_mean():
    # lambda(rho) linear: at rho_l it is lambda_l; the mean runs over the line
    ny, nx = 5, 4
    T = np.tile(np.array([2.0, 1.0, 0.0, -1.0, -2.0])[:, None], (1, nx))  # dT/dy = -1
    rho = np.full((ny, nx), 6.0)
    rho[0, :2] = 0.4  # half the line at rho_v
    q = norms.wall_heat_flux(rho, T, 2, 0.4, 6.0, 0.7, 3.0)
    assert q == pytest.approx(0.5 * (0.7 + 3.0), rel=1e-14)


@pytest.mark.parametrize("yc", [-15.0, 0.0, 12.0])
def test_contact_angle_of_a_circular_cap(yc):
    # a tanh-smoothed circle of radius 30 cut by the wall line y = 0 at height yc of its
    # centre: theta = 90 deg + asin(yc / R) through the liquid
    nx, ny, R, W = 160, 90, 30.0, 3.0
    y, x = np.mgrid[0:ny, 0:nx].astype(float)
    d = np.hypot(x - 80.3, y - yc)
    rho = 0.38 + 0.5 * (6.5 - 0.38) * (1 + np.tanh(2 * (R - d) / W))
    want = 90.0 + np.degrees(np.arcsin(yc / R))
    assert norms.contact_angle(rho, 0.5 * (6.5 + 0.38)) == pytest.approx(want, abs=1.0)


def test_contact_angle_with_a_depleted_wall_layer():
    # a density layer on the wall line hides the foot there: the base is read on the first
    # line above it and the cap is still the circle of the droplet
    nx, ny, R, W, yc = 160, 90, 30.0, 3.0, -8.0  # theta = 74.5 deg
    y, x = np.mgrid[0:ny, 0:nx].astype(float)
    rho = 0.38 + 0.5 * (6.5 - 0.38) * (1 + np.tanh(2 * (R - np.hypot(x - 80.3, y - yc)) / W))
    rho[0, :] = np.minimum(rho[0, :], 2.0)
    want = 90.0 + np.degrees(np.arcsin(yc / R))
    assert norms.contact_angle(rho, 0.5 * (6.5 + 0.38)) == pytest.approx(want, abs=1.0)
    # a droplet that left the wall reads as 180 deg (its circle no longer reaches the wall);
    # a liquid film over the whole wall has no base
    d = np.hypot(x - 80.3, y - 40.0)
    assert norms.contact_angle(0.38 + 3.06 * (1 + np.tanh(2 * (20 - d) / W)), 3.44) == 180.0
    film = np.where(y < 10, 6.5, 0.38)
    assert np.isnan(norms.contact_angle(film, 3.44))


@pytest.mark.slow
def test_workload_wall_density_gives_a_60_degree_angle():
    # the pool workload's wall density (written by oracle.contact_calibration) reproduces
    # its angle in the oracle, and the angle falls as rho_w rises
    import workloads as W
    from oracle import contact_calibration as C
    assert C.static_angle(W.RHO_W_60DEG) == pytest.approx(60.0, abs=1.0)
    assert C.static_angle(2.3) > 80.0
