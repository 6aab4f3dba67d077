"""Pins of the oracle's second transport integrator (Remark 3): Crank-Nicolson
for Eq. distansport in which the implicit half keeps its first-order upwind
part implicit and takes the limited slope from the old state, solved by one
upwind sweep over the plane.

Checked against things other than the oracle's own sweep: a dense linear
solve of the same system; the first-order upwind operator's exactness on
linear data and its upwind (triangular, M-matrix) structure; conservation;
the identity for a zero angle; convergence to the exactly shifted Gaussian;
boundedness at Courant numbers where the explicit trapezoid blows up; and the
O(h^2) one-step distance to the explicit trapezoid."""
import numpy as np
import pytest


def _grid(ny, nz, n_ang, d, umax=0.3):
    return dict(ny=ny, nz=nz, nu=n_ang, nv=n_ang, dy=d, dz=d, u_max=umax, v_max=umax, e_faces=np.array([0.0, 1.0]))


def _gauss(ny, nz, d, y0, z0, s):
    y = (np.arange(ny) - ny / 2 + 0.5) * d
    z = (np.arange(nz) - nz / 2 + 0.5) * d
    return np.exp(-0.5 * ((y[:, None] - y0) ** 2 + (z[None, :] - z0) ** 2) / s ** 2)


def _dense(o, uu, vv, first_order):
    n = o.ny * o.nz
    return np.array([o.transport_apply(uu, vv, e.reshape(o.ny, o.nz), first_order).ravel()
                     for e in np.eye(n)]).T  # columns: the operator on unit vectors (linear operators only)


def test_sweep_equals_dense_solve(oracle_mod):
    """(I - h/2 L1) x = psi + h/2 L(psi) + h/2 (L(psi) - L1 psi) by numpy
    (L1, the first-order upwind part, is linear and assembled column by
    column) for all four sign combinations of (u, v), on a non-square plane."""
    ny, nz, h = 5, 7, 0.07
    o = oracle_mod.Oracle(_grid(ny, nz, 2, 0.1))
    o.set_transport_cn(True)
    u = o.tables()["u"]
    psi = np.random.default_rng(3).uniform(0.0, 1.0, size=(1, 2, 2, 2, ny, nz))
    got = o.transport_substep(h, psi)
    for j in range(2):
        for i in range(2):
            L1 = _dense(o, u[i], u[j], True)  # linear (the limited L is not)
            for c in range(2):
                x0 = psi[0, c, j, i].ravel()
                lx = o.transport_apply(u[i], u[j], psi[0, c, j, i], False).ravel()
                rhs = x0 + 0.5 * h * lx + 0.5 * h * (lx - L1 @ x0)
                ref = np.linalg.solve(np.eye(ny * nz) - 0.5 * h * L1, rhs)
                assert np.abs(got[0, c, j, i].ravel() - ref).max() < 1e-14 * np.abs(ref).max()


@pytest.mark.parametrize("sy,sz", [(1, 1), (-1, 1), (1, -1), (-1, -1)])
def test_first_order_part_is_upwind_and_exact_on_linear_data(oracle_mod, sy, sz):
    ny, nz, d = 9, 8, 0.1
    o = oracle_mod.Oracle(_grid(ny, nz, 2, d))
    u = o.tables()["u"]
    uu, vv = sy * abs(u[0]), sz * abs(u[0])
    L1 = _dense(o, uu, vv, True)
    x = np.random.default_rng(1).uniform(size=(ny, nz))
    assert np.abs(L1 @ x.ravel() - o.transport_apply(uu, vv, x, True).ravel()).max() < 1e-13  # linear
    # couplings only to the cell itself and its upstream neighbours, with
    # non-negative weights (an M-matrix after sign): I - h/2 L1 is triangular
    # in the upwind order
    for p in range(ny):
        for q in range(nz):
            row = L1[p * nz + q].reshape(ny, nz)
            nz_idx = {(a, b) for a, b in zip(*np.nonzero(row))}
            allowed = {(p, q), (p - sy, q), (p, q - sz)}
            assert nz_idx <= allowed
            assert row[p, q] < 0 or (p, q) not in nz_idx
            for a, b in nz_idx - {(p, q)}:
                assert row[a, b] > 0
    # linear data: L1 and L give -(u dpsi/dy + v dpsi/dz) away from the edges
    yy, zz = np.meshgrid(np.arange(ny) * d, np.arange(nz) * d, indexing="ij")
    lin = 2.0 + 0.7 * yy - 1.3 * zz
    exact = -(uu * 0.7 + vv * -1.3)
    for fo in (True, False):
        out = o.transport_apply(uu, vv, lin, fo)
        assert np.abs(out[2:-2, 2:-2] - exact).max() < 1e-12


def test_conservation_and_zero_angle_identity(oracle_mod):
    """Away from the edges the plane sum is unchanged; the (0, 0) angle of an
    odd grid is left bit for bit."""
    ny, nz = 44, 40  # the Gaussians sit >= 9 widths inside the plane
    o = oracle_mod.Oracle(_grid(ny, nz, 3, 0.1))
    o.set_transport_cn(True)
    psi = np.zeros((1, 2, 3, 3, ny, nz))
    for j in range(3):
        for i in range(3):
            psi[0, 0, j, i] = _gauss(ny, nz, 0.1, 0.05 * i, -0.05 * j, 0.2)
            psi[0, 1, j, i] = 0.3 * _gauss(ny, nz, 0.1, -0.1, 0.1, 0.25)
    out = o.transport_substep(0.05, psi)
    assert np.abs(out.sum(axis=(-1, -2)) - psi.sum(axis=(-1, -2))).max() < 1e-12
    assert np.array_equal(out[0, :, 1, 1], psi[0, :, 1, 1])


def test_converges_to_the_shifted_gaussian(oracle_mod):
    """One angle, depth 1 at Courant number 0.5: the L1 error against the
    exactly shifted Gaussian falls at order > 1.5 under refinement."""
    errs = []
    for ny in (32, 64, 128):
        d = 4.0 / ny
        o = oracle_mod.Oracle(_grid(ny, ny, 2, d))
        o.set_transport_cn(True)
        uu = o.tables()["u"][1]
        n = int(round(1.0 / (0.5 * d / uu)))
        h = 1.0 / n
        psi = np.zeros((1, 2, 2, 2, ny, ny))
        psi[0, 0, 1, 1] = _gauss(ny, ny, d, -0.3, -0.3, 0.4)
        for _ in range(n):
            psi = o.transport_substep(h, psi)
        errs.append(np.abs(psi[0, 0, 1, 1] - _gauss(ny, ny, d, -0.3 + uu, -0.3 + uu, 0.4)).sum() * d * d)
    orders = [np.log2(errs[k] / errs[k + 1]) for k in range(2)]
    assert min(orders) > 1.5, (errs, orders)


def test_bounded_beyond_the_explicit_courant_limit(oracle_mod):
    """At Courant number 3 per direction ten CN steps stay bounded (max |psi|
    <= 1.1 for a unit Gaussian) while the explicit trapezoid explodes."""
    ny, d = 40, 0.1
    res = {}
    for cn in (False, True):
        o = oracle_mod.Oracle(_grid(ny, ny, 2, d))
        o.set_transport_cn(cn)
        uu = o.tables()["u"][1]
        psi = np.zeros((1, 2, 2, 2, ny, ny))
        psi[0, 0, 1, 1] = _gauss(ny, ny, d, -1.0, -1.0, 0.3)
        for _ in range(10):
            psi = o.transport_substep(3.0 * d / uu, psi)
        res[cn] = np.abs(psi).max()
    assert res[True] < 1.1 and res[False] > 100.0


def test_one_step_distance_to_the_explicit_trapezoid_is_second_order(oracle_mod):
    ny, d = 24, 0.1
    diffs = []
    for h in (0.02, 0.01, 0.005):
        a = oracle_mod.Oracle(_grid(ny, ny, 2, d))
        b = oracle_mod.Oracle(_grid(ny, ny, 2, d))
        b.set_transport_cn(True)
        psi = np.zeros((1, 2, 2, 2, ny, ny))
        psi[0, 0, 1, 0] = _gauss(ny, ny, d, 0.2, -0.1, 0.3)
        psi[0, 1, 0, 1] = _gauss(ny, ny, d, -0.2, 0.1, 0.25)
        diffs.append(np.abs(a.transport_substep(h, psi) - b.transport_substep(h, psi)).max())
    assert 3.5 < diffs[0] / diffs[1] < 4.5 and 3.5 < diffs[1] / diffs[2] < 4.5
