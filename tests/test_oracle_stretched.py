"""Pins for the stretched-grid oracle (Eq 4.18 and the non-uniform operators of
Eqs 3.20-3.24): closed forms of the map, exactness classes of the operators,
the midpoint rule's exact error on quadratics, the discrete divergence theorem,
second-order convergence of the Neumann solve and of the quadrature, and the
projection's exact discrete continuity."""

import numpy as np
import pytest

from oracle import stretched as G
from conftest import golden


def _axis(n, alpha):
    return G.Axis(G.tanh_faces(n, alpha))


# ---------------------------------------------------------------- Eq 4.18 map

@pytest.mark.parametrize("n,alpha", [(16, 0.5), (64, 3.0), (216, 6.0)])
def test_map_fixes_the_ends_and_clusters_at_both_walls(n, alpha):
    xf = G.tanh_faces(n, alpha)
    assert xf[0] == pytest.approx(0.0, abs=1e-15) and xf[-1] == pytest.approx(1.0, abs=1e-15)
    dx = np.diff(xf)
    assert np.all(dx > 0)
    np.testing.assert_allclose(xf[::-1], 1.0 - xf, atol=1e-15)       # mirror symmetry about 1/2
    assert dx.argmin() in (0, n - 1) and abs(dx.argmax() - (n - 1) / 2) <= 0.5
    assert np.all(np.diff(dx[: n // 2]) > 0)                          # growing towards the centre


def test_map_tends_to_the_identity():
    s = np.arange(33) / 32
    assert np.max(np.abs(G.tanh_faces(32, 1e-4) - s)) < 1e-8
    assert np.array_equal(G.tanh_faces(32, 0.0), s)


def test_printed_form_differs_by_a_constant():
    """The extracted form of Eq 4.18 and the map used have the same spacings."""
    for alpha in (0.7, 2.0, 5.0):
        s = np.arange(41) / 40
        printed = (1.0 + np.tanh(alpha * (s - 0.5))) / (2.0 * np.tanh(alpha / 2.0))
        diff = printed - G.tanh_faces(40, alpha)
        np.testing.assert_allclose(diff, 0.5 / np.tanh(alpha / 2.0) - 0.5, rtol=0, atol=1e-14)


@pytest.mark.parametrize("alpha", [1.0, 3.0, 6.0])
def test_spacing_ratio_tends_to_cosh_squared(alpha):
    """The map's slope is alpha sech^2(alpha (s - 1/2)) / (2 tanh(alpha/2)), so
    the centre-to-wall slope ratio is cosh^2(alpha/2); the discrete ratio (of
    mean slopes over the end and centre cells) approaches it at first order."""
    want = np.cosh(alpha / 2.0) ** 2
    errs = [abs(G.spacing_ratio(n, alpha) / want - 1.0) for n in (256, 512, 1024)]
    assert errs[-1] < 1e-2
    ratios = np.array(errs[:-1]) / np.array(errs[1:])
    assert np.all(np.abs(ratios - 2.0) < 0.05), ratios


@pytest.mark.parametrize("n,ratio", [(64, 2.0), (96, 2.0), (216, 2.0), (64, 21.0), (216, 21.0)])
def test_alpha_hits_the_requested_spacing_ratio(n, ratio):
    """The grids of the cavity study: max spacing 2 and 21 times the minimum."""
    a = G.alpha_for_ratio(n, ratio)
    assert G.spacing_ratio(n, a) == pytest.approx(ratio, rel=1e-10)
    assert a == pytest.approx(2.0 * np.arccosh(np.sqrt(ratio)), rel=0.05)
    assert G.alpha_for_ratio(n, 1.0) == 0.0


def test_stretched_grids_have_the_printed_largest_spacing():
    """Tables 3 and 4 print max(dx_i) of every stretched grid of the cavity's
    grid studies.  Eq 4.18 on the faces i/n, with alpha solved for
    max(dx) = m min(dx), gives all eight within one unit of the last printed
    digit (the table truncates some and rounds others).  A uniform grid misses
    them by far more, and a one-sided tanh clustering with the same ratio
    misses the first (0.019533 on 64 cells)."""
    rows = golden("cavity_grid_spacing_tables3_4.txt")
    assert len(rows) == 8
    for m, n, want in rows:
        m, n, want = float(m), int(n), float(want)
        dx = np.diff(G.tanh_faces(n, G.alpha_for_ratio(n, m)))
        assert abs(dx.max() - want) < 1e-5, (m, n, dx.max(), want)
        assert dx.max() / dx.min() == pytest.approx(m, rel=1e-10)
        assert abs(1.0 / n - want) > 0.15 * want                # far from the uniform width


def test_alpha_grows_with_the_ratio():
    a = [G.alpha_for_ratio(96, r) for r in (1.5, 2.0, 5.0, 10.0, 21.0)]
    assert np.all(np.diff(a) > 0)


# ------------------------------------------------- Eqs 3.20 and 3.21 operators

def test_operators_are_exact_on_linear_fields():
    ax = _axis(17, 3.0)
    a, b = 0.3, -1.7
    phi = a + b * ax.xc
    np.testing.assert_allclose(G.interp_to_faces(phi, ax), a + b * ax.xf[1:-1], atol=1e-14)
    np.testing.assert_allclose(G.diff_to_faces(phi, ax), b, atol=1e-12)
    np.testing.assert_allclose(G.diff2(phi, ax), b, atol=1e-12)
    np.testing.assert_allclose(G.faces_diff_to_cells(a + b * ax.xf, ax), b, atol=1e-12)


def test_operators_on_quadratics_have_their_closed_forms():
    """phi = x^2: the linear interpolant overshoots by (x_f - x_l)(x_r - x_f);
    a difference quotient of x^2 over [x_l, x_r] is x_l + x_r."""
    ax = _axis(23, 4.0)
    phi = ax.xc ** 2
    xl, xr, xf = ax.xc[:-1], ax.xc[1:], ax.xf[1:-1]
    np.testing.assert_allclose(G.interp_to_faces(phi, ax) - xf ** 2, (xf - xl) * (xr - xf),
                               rtol=1e-12, atol=1e-16)
    np.testing.assert_allclose(G.diff_to_faces(phi, ax), xl + xr, rtol=1e-12)
    np.testing.assert_allclose(G.diff2(phi, ax), ax.xc[:-2] + ax.xc[2:], rtol=1e-12)
    np.testing.assert_allclose(G.faces_diff_to_cells(ax.xf ** 2, ax), 2.0 * ax.xc, rtol=1e-12)


def test_uniform_grid_reduces_to_the_textbook_stencils():
    n = 12
    ax = _axis(n, 0.0)
    phi = np.random.default_rng(1).standard_normal(n)
    np.testing.assert_allclose(G.interp_to_faces(phi, ax), 0.5 * (phi[1:] + phi[:-1]), atol=1e-15)
    np.testing.assert_allclose(G.diff_to_faces(phi, ax), n * np.diff(phi), rtol=1e-13)
    np.testing.assert_allclose(G.diff2(phi, ax), 0.5 * n * (phi[2:] - phi[:-2]), rtol=1e-13)


def test_operators_act_along_the_requested_axis():
    ax_x, ax_y = _axis(7, 2.0), _axis(5, 1.0)
    Y, X = np.meshgrid(ax_y.xc, ax_x.xc, indexing="ij")
    phi = 2.0 * X - 3.0 * Y
    np.testing.assert_allclose(G.diff_to_faces(phi, ax_x, axis=1), 2.0, atol=1e-12)
    np.testing.assert_allclose(G.diff_to_faces(phi, ax_y, axis=0), -3.0, atol=1e-12)
    assert G.interp_to_faces(phi, ax_y, axis=0).shape == (4, 7)


def test_local_truncation_order_of_the_face_derivative():
    """Eq 3.21 with n = 1 at a face of a smoothly stretched grid: the error
    against the exact derivative at the face falls at second order."""
    errs = []
    for n in (32, 64, 128):
        ax = _axis(n, 3.0)
        d = G.diff_to_faces(np.sin(2.0 * ax.xc), ax)
        errs.append(np.max(np.abs(d - 2.0 * np.cos(2.0 * ax.xf[1:-1]))))
    orders = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(orders > 1.9), orders


# ----------------------------------------------------------- Eq 3.22 quadrature

def test_midpoint_rule_closed_forms():
    ax_x, ax_y, ax_z = _axis(13, 3.0), _axis(9, 1.5), _axis(5, 0.0)
    assert G.integrate(np.ones(13), [ax_x]) == pytest.approx(1.0, abs=1e-15)
    assert G.integrate(ax_x.xc, [ax_x]) == pytest.approx(0.5, abs=1e-15)
    # each cell of width h misses h^3 / 12 of the integral of x^2
    assert G.integrate(ax_x.xc ** 2, [ax_x]) == pytest.approx(1 / 3 - np.sum(ax_x.dx ** 3) / 12,
                                                               abs=1e-15)
    Y, X = np.meshgrid(ax_y.xc, ax_x.xc, indexing="ij")
    assert G.integrate(X ** 2 + Y, [ax_x, ax_y]) == pytest.approx(
        1 / 3 - np.sum(ax_x.dx ** 3) / 12 + 0.5, abs=1e-15)
    Zc, Yc, Xc = np.meshgrid(ax_z.xc, ax_y.xc, ax_x.xc, indexing="ij")
    assert G.integrate(Xc * Yc * Zc, [ax_x, ax_y, ax_z]) == pytest.approx(0.125, abs=1e-15)
    assert np.sum(G.volumes([ax_x, ax_y, ax_z])) == pytest.approx(1.0, abs=1e-14)


def test_midpoint_rule_is_second_order_on_stretched_grids():
    exact = 2.0 / np.pi
    errs = [abs(G.integrate(np.sin(np.pi * _axis(n, 4.0).xc), [_axis(n, 4.0)]) - exact)
            for n in (16, 32, 64)]
    orders = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(np.abs(orders - 2.0) < 0.1), orders


# ------------------------------------------------------- Eqs 3.23-3.24 pressure

def _dense(axes, shape):
    N = int(np.prod(shape))
    A = np.zeros((N, N))
    for k in range(N):
        e = np.zeros(N)
        e[k] = 1.0
        A[:, k] = G.laplacian_neumann(e.reshape(shape), axes).ravel()
    return A


def test_pressure_operator_structure():
    """Zero-flux boundary: constants in the kernel, the volume-weighted sum of
    any image is zero (discrete divergence theorem), and W A is symmetric and
    negative semi-definite with a one-dimensional kernel."""
    axes = [_axis(6, 2.5), _axis(5, 1.0)]
    shape = (5, 6)
    P = np.random.default_rng(2).standard_normal(shape)
    assert np.max(np.abs(G.laplacian_neumann(np.full(shape, 3.0), axes))) < 1e-12
    assert abs(G.integrate(G.laplacian_neumann(P, axes), axes)) < 1e-12
    A = _dense(axes, shape)
    WA = G.volumes(axes).ravel()[:, None] * A
    np.testing.assert_allclose(WA, WA.T, atol=1e-12)
    ev = np.linalg.eigvalsh(0.5 * (WA + WA.T))
    assert ev[-1] < 1e-10 and ev[-2] < -1e-3


def test_pressure_operator_on_a_uniform_grid_is_the_five_point_stencil():
    n = 6
    axes = [_axis(n, 0.0), _axis(n, 0.0)]
    P = np.random.default_rng(3).standard_normal((n, n))
    Q = np.pad(P, 1, mode="edge")                    # mirrored ghosts: zero boundary flux
    five = n * n * (Q[1:-1, 2:] + Q[1:-1, :-2] + Q[2:, 1:-1] + Q[:-2, 1:-1] - 4.0 * P)
    np.testing.assert_allclose(G.laplacian_neumann(P, axes), five, rtol=1e-12, atol=1e-10)


def test_neumann_solve_converges_at_second_order():
    """P = cos(pi x) cos(pi y) has zero normal derivative on the unit square
    and Laplacian -2 pi^2 P; the discrete solution's error falls at second
    order on a fixed stretching."""
    errs = []
    for n in (12, 24, 48):
        axes = [_axis(n, 2.0), _axis(n, 2.0)]
        Y, X = np.meshgrid(axes[1].xc, axes[0].xc, indexing="ij")
        Pe = np.cos(np.pi * X) * np.cos(np.pi * Y)
        Pe = Pe - G.integrate(Pe, axes)
        P = G.solve_neumann(-2.0 * np.pi ** 2 * Pe, axes)
        errs.append(np.max(np.abs(P - Pe)))
    orders = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert errs[-1] < 1e-3 and orders[0] > 1.6 and orders[1] > 1.85, (errs, orders)


@pytest.mark.parametrize("dim", [2, 3])
def test_projection_gives_exact_discrete_continuity(dim):
    """Eq 3.24 after Eq 3.23: the projected face fluxes satisfy
    d_t rho + delta_1 F_j / delta_1 x_j = 0 to round-off, boundary faces keep
    their (zero) values and P has zero volume-weighted mean."""
    rng = np.random.default_rng(4 + dim)
    ns = [6, 5, 4][:dim]
    axes = [_axis(n, a) for n, a in zip(ns, [3.0, 1.0, 2.0])]
    shape = tuple(reversed(ns))
    Fs = []
    for d in range(dim):
        fs = list(shape)
        fs[dim - 1 - d] += 1
        f = rng.standard_normal(fs)
        idx = [slice(None)] * dim
        idx[dim - 1 - d] = 0
        f[tuple(idx)] = 0.0
        idx[dim - 1 - d] = -1
        f[tuple(idx)] = 0.0
        Fs.append(f)
    drho = rng.standard_normal(shape)
    drho -= G.integrate(drho, axes) / np.sum(G.volumes(axes))
    F, P = G.project(Fs, axes, drho)
    assert np.max(np.abs(G.cell_divergence(F, axes) + drho)) < 1e-10
    assert abs(G.integrate(P, axes)) < 1e-12
    for d in range(dim):
        idx = [slice(None)] * dim
        idx[dim - 1 - d] = 0
        assert np.all(F[d][tuple(idx)] == 0.0)
