"""Pins for the oracle's finite-element operators (Sec. 2.2), all on CPU."""
import numpy as np
import pytest
import scipy.sparse as sp

from oracle import fem, inexact
from oracle_golden import element_matrices

@pytest.mark.parametrize("h", [1.0, 0.25, 1.0 / 64])
def test_1d_element_matrices_closed_forms(h):
    g = element_matrices()
    scale = {"h/30": h / 30, "1/(3h)": 1 / (3 * h), "h/6": h / 6, "1/h": 1 / h}
    m2, k2 = fem.element_matrices_1d(2, h)
    m1, k1 = fem.element_matrices_1d(1, h)
    for name, mat in [("q2_mass", m2), ("q2_stiff", k2), ("q1_mass", m1), ("q1_stiff", k1)]:
        sc, ref = g[name]
        np.testing.assert_allclose(mat, scale[sc] * ref, rtol=1e-13, atol=1e-13 * abs(scale[sc]))


def test_jacobi_mass_bounds():
    g = element_matrices()
    np.testing.assert_allclose(inexact.element_jacobi_bounds(2), g["q2_jacobi_bounds"], rtol=1e-12)
    np.testing.assert_allclose(inexact.element_jacobi_bounds(1), g["q1_jacobi_bounds"], rtol=1e-12)


@pytest.mark.parametrize("N,x0,x1", [(2, 0.0, 1.0), (4, -1.0, 1.0), (8, 0.0, 1.0)])
def test_mass_integrates_area_and_stiffness_kills_affine(N, x0, x1):
    ops = fem.assemble(N, x0, x1)
    area = (x1 - x0) ** 2
    assert abs(ops.M.sum() - area) < 1e-12
    assert abs(ops.Mp.sum() - area) < 1e-12
    g = ops.grid
    X, Y = g.q2_coords()
    aff = 0.3 + 1.7 * X - 2.2 * Y
    ii = g.velocity_interior()
    assert np.abs((ops.K @ aff)[ii]).max() < 1e-11
    Xp, Yp = g.q1_coords()
    affp = 0.3 + 1.7 * Xp - 2.2 * Yp
    # interior Q1 rows only (boundary rows carry the normal-derivative term)
    n1 = g.n1
    ix, iy = np.arange(g.nq) % n1, np.arange(g.nq) // n1
    inner = (ix > 0) & (ix < n1 - 1) & (iy > 0) & (iy < n1 - 1)
    assert np.abs((ops.Kp @ affp)[inner]).max() < 1e-11
    # constants are in the kernel of K and K_p
    assert np.abs(ops.K @ np.ones(g.ns)).max() < 1e-11
    assert np.abs(ops.Kp @ np.ones(g.nq)).max() < 1e-11


@pytest.mark.parametrize("N", [2, 4, 8])
def test_divergence_of_divergence_free_quadratic_is_zero(N):
    ops = fem.assemble(N, -1.0, 1.0)
    X, Y = ops.grid.q2_coords()
    # stream function x^2 y + 0.5 x y^2 - 0.3 y^3 -> v = (psi_y, -psi_x), quadratic
    vx = X ** 2 + X * Y - 0.9 * Y ** 2
    vy = -(2 * X * Y + 0.5 * Y ** 2)
    assert np.abs(ops.Bx @ vx + ops.By @ vy).max() < 1e-12
    # not divergence free -> nonzero (the test can fail)
    assert np.abs(ops.Bx @ (X ** 2)).max() > 1e-3
    # B^T 1 = 0 on interior velocity rows (constants lie in ker B^T)
    ii = ops.grid.velocity_interior()
    one = np.ones(ops.grid.nq)
    assert np.abs((ops.Bx.T @ one)[ii]).max() < 1e-12
    assert np.abs((ops.By.T @ one)[ii]).max() < 1e-12


@pytest.mark.parametrize("N", [2, 4, 8])
def test_convection_skew_and_constants(N):
    ops = fem.assemble(N, -1.0, 1.0, fem.recirculating_wind)
    g = ops.grid
    ii = g.velocity_interior()
    Nr = ops.N[ii][:, ii]
    assert abs(Nr + Nr.T).max() < 1e-13
    assert abs(ops.Np + ops.Np.T).max() < 1e-13
    assert np.abs(ops.N @ np.ones(g.ns)).max() < 1e-13
    assert abs(Nr).max() > 1e-3
    # exactness: N applied to a linear field x gives the mass matrix times w_x
    X, Y = g.q2_coords()
    wx, wy = fem.recirculating_wind(X, Y)
    # int phi_i w . grad(x) = int phi_i w_x ; w_x quadratic -> exactly M wx
    np.testing.assert_allclose(ops.N @ X, ops.M @ wx, atol=1e-13)
    np.testing.assert_allclose(ops.N @ Y, ops.M @ wy, atol=1e-13)


def test_wind_divergence_free_and_tangential():
    rng = np.random.default_rng(0)
    x, y = rng.uniform(-1, 1, 50), rng.uniform(-1, 1, 50)
    e = 1e-6
    div = (fem.recirculating_wind(x + e, y)[0] - fem.recirculating_wind(x - e, y)[0]) / (2 * e) + \
          (fem.recirculating_wind(x, y + e)[1] - fem.recirculating_wind(x, y - e)[1]) / (2 * e)
    assert np.abs(div).max() < 1e-8
    assert np.abs(fem.recirculating_wind(np.ones(5), y[:5])[0]).max() == 0.0
    assert np.abs(fem.recirculating_wind(x[:5], -np.ones(5))[1]).max() == 0.0


@pytest.mark.parametrize("Nc", [1, 2, 4])
def test_prolongation_reproduces_polynomials(Nc):
    # Q2: quadratic interpolated on the coarse grid is reproduced on the fine grid
    P2 = fem.prolongation_2d(Nc, 2)
    gc, gf = fem.Grid(Nc, 0.0, 1.0), fem.Grid(2 * Nc, 0.0, 1.0)
    f = lambda x, y: 1 + 2 * x - y + 3 * x * x - x * y + 0.5 * y * y + x * x * y * y
    np.testing.assert_allclose(P2 @ f(*gc.q2_coords()), f(*gf.q2_coords()), atol=1e-13)
    P1 = fem.prolongation_2d(Nc, 1)
    g = lambda x, y: 1 + 2 * x - y + 0.7 * x * y
    np.testing.assert_allclose(P1 @ g(*gc.q1_coords()), g(*gf.q1_coords()), atol=1e-13)
    assert np.allclose(np.asarray(P2.sum(axis=1)).ravel(), 1.0)
    assert set(np.round(fem.prolongation_1d(Nc, 2).data, 12)) <= {1.0, 0.375, 0.75, -0.125}


@pytest.mark.parametrize("Nc", [1, 2, 4])
def test_galerkin_equals_rediscretisation(Nc):
    fine = fem.assemble(2 * Nc, -1.0, 1.0, fem.recirculating_wind)
    coarse = fem.assemble(Nc, -1.0, 1.0, fem.recirculating_wind)
    P2 = fem.prolongation_2d(Nc, 2)
    P1 = fem.prolongation_2d(Nc, 1)
    for Af, Ac, P in [(fine.M, coarse.M, P2), (fine.K, coarse.K, P2), (fine.N, coarse.N, P2),
                      (fine.Mp, coarse.Mp, P1), (fine.Kp, coarse.Kp, P1), (fine.Np, coarse.Np, P1)]:
        G = (P.T @ Af @ P).toarray()
        np.testing.assert_allclose(G, Ac.toarray(), atol=1e-12 * max(1.0, abs(Ac).max()))


@pytest.mark.parametrize("N", [4, 8])
def test_assembled_jacobi_mass_spectrum_within_element_bounds(N):
    ops = fem.assemble(N, 0.0, 1.0)
    g = ops.grid
    ii, pf = g.velocity_interior(), g.pressure_free()
    for A, (lo, hi) in [(ops.M[ii][:, ii], inexact.element_jacobi_bounds(2)),
                        (ops.Mp[pf][:, pf], inexact.element_jacobi_bounds(1))]:
        A = A.toarray()
        ev = np.linalg.eigvals(np.diag(1 / np.diag(A)) @ A).real
        assert ev.min() >= lo - 1e-12 and ev.max() <= hi + 1e-12


def test_two_vortex_wind_properties():
    """Sec. 5.2 wind: divergence free, zero on and near the boundary (outside
    both ellipses), tangent to the ellipses c = const, one vortex turning each
    way about (+-1/2, 0)."""
    rng = np.random.default_rng(1)
    x, y = rng.uniform(-1, 1, 400), rng.uniform(-1, 1, 400)
    A, B = fem.TWO_VORTEX_A, fem.TWO_VORTEX_B
    c1 = 1 - np.sqrt((B * (x - 0.5)) ** 2 + (A * y) ** 2)
    c2 = 1 - np.sqrt((B * (x + 0.5)) ** 2 + (A * y) ** 2)
    ok = (np.minimum(np.abs(c1), np.abs(c2)) > 1e-3) & (np.minimum(np.abs(c1 - 1), np.abs(c2 - 1)) > 1e-3)
    x, y, c1, c2 = x[ok], y[ok], c1[ok], c2[ok]
    w = fem.two_vortex_wind
    e = 1e-6
    div = (w(x + e, y)[0] - w(x - e, y)[0]) / (2 * e) + (w(x, y + e)[1] - w(x, y - e)[1]) / (2 * e)
    assert np.abs(div).max() < 1e-7
    wx, wy = w(x, y)
    for c, s in ((c1, 0.5), (c2, -0.5)):
        inside = c > 0
        gx, gy = B * B * (x - s), A * A * y          # grad of the ellipse's level function (up to a factor)
        assert np.abs((wx * gx + wy * gy)[inside]).max() < 1e-12
    assert np.all(wx[(c1 < 0) & (c2 < 0)] == 0) and np.all(wy[(c1 < 0) & (c2 < 0)] == 0)
    t = np.linspace(-1, 1, 41)
    for bx, by in ((t, -np.ones_like(t)), (t, np.ones_like(t)), (-np.ones_like(t), t), (np.ones_like(t), t)):
        assert np.abs(np.concatenate(w(bx, by))).max() == 0.0
    # above each centre the flow goes +x (right vortex, clockwise) and -x (left vortex)
    assert w(np.array([0.5]), np.array([0.3]))[0][0] > 0 > w(np.array([-0.5]), np.array([0.3]))[0][0]


def test_two_vortex_convection():
    """The Gauss-point convection matrix of the two-vortex wind applied to
    the linear field x approaches M w_x as h shrinks (int phi_i w . grad x =
    int phi_i w_x); the skew-symmetric form used for this wind is exactly
    skew and differs from the same form at 16 x 16 Gauss points by a
    quadrature error that shrinks with h."""
    errs, qerrs = [], []
    for N in (8, 16, 32):
        raw = fem.assemble(N, -1.0, 1.0, fem.two_vortex_wind)
        sk = fem.assemble(N, -1.0, 1.0, fem.two_vortex_wind, skew=True)
        sk16 = fem.assemble(N, -1.0, 1.0, fem.two_vortex_wind, npts=16, skew=True)
        g = raw.grid
        ii = g.velocity_interior()
        X, Y = g.q2_coords()
        wx, wy = fem.two_vortex_wind(X, Y)
        errs.append(max(np.abs((raw.N @ X - raw.M @ wx)[ii]).max() / np.abs(raw.M @ wx).max(),
                        np.abs((raw.N @ Y - raw.M @ wy)[ii]).max() / np.abs(raw.M @ wy).max()))
        assert abs(sk.N + sk.N.T).max() == 0.0 and abs(sk.Np + sk.Np.T).max() == 0.0
        qerrs.append(abs(sk.N - sk16.N).max() / abs(sk16.N).max())
    assert errs[0] > errs[1] > errs[2] and errs[2] < 3e-2, errs          # measured 7.8e-2, 3.3e-2, 2.0e-2 (the kink limits the rate)
    assert qerrs[0] > qerrs[2] and qerrs[2] < 1e-2, qerrs


def test_nodal_wind_reproduces_the_polynomial_wind():
    """A caller-given nodal wind is used through its Q2 interpolant, injected
    to coarser grids.  The recirculating wind is a quadratic, so its nodal
    values reproduce it exactly on every level: the convection matrices equal
    the analytic ones (the skew-symmetric form changes nothing for an exactly
    skew N), on the fine grid and on every multigrid level."""
    from oracle import inexact, kkt
    N = 8
    g = fem.Grid(N, -1.0, 1.0)
    X, Y = g.q2_coords()
    W = np.stack(fem.recirculating_wind(X, Y))
    Pn = kkt.Problem("oseen", 3, 4, 0.2, 1e-3, 1e-2, -1.0, 1.0, ("nodal", W))
    Pr = kkt.Problem("oseen", 3, 4, 0.2, 1e-3, 1e-2, -1.0, 1.0, "recirc")
    scale = abs(Pr.ops.N).max()
    assert abs(Pn.ops.N - Pr.ops.N).max() <= 1e-14 * scale
    assert abs(Pn.ops.Np - Pr.ops.Np).max() <= 1e-14 * abs(Pr.ops.Np).max()
    mn = inexact.Multigrid("q2", 3, -1.0, 1.0, ("nodal", W), 1.0 + 0.5j, 0.01, 0.2)
    mr = inexact.Multigrid("q2", 3, -1.0, 1.0, "recirc", 1.0 + 0.5j, 0.01, 0.2)
    assert len(mn.levels) == 3
    for a, b in zip(mn.levels, mr.levels):
        assert abs(a.A - b.A).max() <= 1e-14 * abs(b.A).max()
    # a nodal field that is not a quadratic gives an exactly skew N and
    # differs from the analytic wind's operator by the interpolation error
    W2 = np.stack(fem.two_vortex_wind(X, Y))
    P2 = kkt.Problem("oseen", 3, 4, 0.2, 1e-3, 1e-2, -1.0, 1.0, ("nodal", W2))
    assert abs(P2.ops.N + P2.ops.N.T).max() == 0.0
    Pa = kkt.Problem("oseen", 3, 4, 0.2, 1e-3, 1e-2, -1.0, 1.0, "two_vortex")
    assert 0 < abs(P2.ops.N - Pa.ops.N).max() < 0.2 * abs(Pa.ops.N).max()
