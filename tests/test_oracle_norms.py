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
