"""Pins of the oracle's lateral transport (Section 3.4, Eq. distansport,
Remark 3) and angular diffusion (Section 3.4, Eqs. sd and fly)."""
import numpy as np
import pytest


def _grid(ny, nz, nu, nv, ng=1, dy=0.1, dz=0.1, u_max=0.15, v_max=0.15):
    return dict(ny=ny, nz=nz, nu=nu, nv=nv, dy=dy, dz=dz, u_max=u_max, v_max=v_max,
                e_faces=np.linspace(50.0, 60.0, ng + 1))


# ---------------------------------------------------------------- transport

def test_transport_conserves_and_centre_angle_is_identity(oracle_mod):
    """Flux form: sum_{y,z} psi is conserved while the border cells are empty;
    the plane with u = v = 0 (odd angle counts) does not move at all."""
    o = oracle_mod.Oracle(_grid(20, 18, 3, 5, ng=2))
    rng = np.random.default_rng(1)
    psi = np.zeros(o.comp_shape)
    psi[..., 5:15, 5:13] = rng.random(psi[..., 5:15, 5:13].shape)
    out = o.transport_substep(0.05, psi)
    assert np.allclose(out.sum(axis=(-1, -2)), psi.sum(axis=(-1, -2)), rtol=1e-13)
    centre = out[:, :, 2, 1]
    assert np.array_equal(centre, psi[:, :, 2, 1])


def _superbee_slope(a, b):
    """Textbook division-free superbee slope: zero at extrema, otherwise
    sign(b) max(min(2|a|, |b|), min(|a|, 2|b|))."""
    if a * b <= 0.0:
        return 0.0
    return np.sign(b) * max(min(2 * abs(a), abs(b)), min(abs(a), 2 * abs(b)))


def _brute_1d(f, s, dy, h):
    """Heun step of the 1-D flux-limited upwind scheme with zero ghosts,
    written from the division-free slope above."""
    n = len(f)

    def rhs(w):
        g = np.concatenate([[0.0, 0.0], w, [0.0, 0.0]])
        flux = np.zeros(n + 1)  # faces -1/2 .. n-1/2
        for m in range(-1, n):
            k = m + 2
            if s > 0:
                flux[m + 1] = s * (g[k] + 0.5 * _superbee_slope(g[k] - g[k - 1], g[k + 1] - g[k]))
            else:
                flux[m + 1] = s * (g[k + 1] - 0.5 * _superbee_slope(g[k + 2] - g[k + 1], g[k + 1] - g[k]))
        return -(flux[1:] - flux[:-1]) / dy

    l0 = rhs(f)
    st = f + h * l0
    return f + 0.5 * h * (l0 + rhs(st))


def test_transport_matches_brute_force_1d(oracle_mod):
    """With nz = 1 the z flux vanishes, so each (u) plane is the 1-D scheme."""
    o = oracle_mod.Oracle(_grid(8, 1, 4, 1))
    rng = np.random.default_rng(7)
    psi = rng.random(o.comp_shape)
    psi[0, 0, 0, 1, 3] = psi[0, 0, 0, 1, 2]  # a flat pair exercises the zero denominator
    h = 0.3
    out = o.transport_substep(h, psi)
    u = o.tables()["u"]
    for i in range(4):
        for c in range(2):
            ref = _brute_1d(psi[0, c, 0, i, :, 0], u[i], 0.1, h)
            assert np.allclose(out[0, c, 0, i, :, 0], ref, rtol=1e-13, atol=1e-15)


def test_transport_linear_data_moves_exactly(oracle_mod):
    """Away from the edges and from extrema the limiter returns theta = 1 on
    linear data, the scheme is the central flux, and Heun shifts a linear
    profile exactly: psi_new = psi - h u slope."""
    o = oracle_mod.Oracle(_grid(24, 1, 2, 1))
    y = np.arange(24) * 0.1
    psi = np.zeros(o.comp_shape)
    psi[0, :, 0, :, :, 0] = 1.0 + 0.5 * y
    h = 0.2
    out = o.transport_substep(h, psi)
    u = o.tables()["u"]
    for i in range(2):
        interior = slice(6, 18)
        assert np.allclose(out[0, 0, 0, i, interior, 0], psi[0, 0, 0, i, interior, 0] - h * u[i] * 0.5,
                           rtol=1e-13)


def test_transport_is_tvd_and_positive(oracle_mod):
    o = oracle_mod.Oracle(_grid(16, 16, 4, 4))
    rng = np.random.default_rng(11)
    psi = rng.random(o.comp_shape) ** 3
    out = o.transport_substep(0.05, psi)
    assert out.min() >= -1e-15
    assert out.max() <= psi.max() * (1 + 1e-14)
    # total variation does not grow in 1-D (nz = 1: no z flux)
    o1 = oracle_mod.Oracle(_grid(40, 1, 4, 1))
    p1 = rng.random(o1.comp_shape) ** 3
    q1 = o1.transport_substep(0.3, p1)
    tv = lambda w: np.abs(np.diff(np.concatenate([np.zeros(w.shape[:-2] + (1, 1)), w,
                                                  np.zeros(w.shape[:-2] + (1, 1))], axis=-2), axis=-2)).sum(axis=-2)
    assert np.all(tv(q1) <= tv(p1) * (1 + 1e-12))


def _shift_error(oracle_mod, n, steps_per_unit):
    """L1 error of a Gaussian advected with speed u in y against the exact
    shifted cell averages: (whole line, away from the extremum)."""
    from scipy.special import erf
    L = 4.0
    dy = L / n
    o = oracle_mod.Oracle(dict(ny=n, nz=1, nu=2, nv=1, dy=dy, dz=1.0, u_max=0.75, v_max=0.1,
                               e_faces=np.array([1.0, 2.0])))
    u = o.tables()["u"][1]  # +0.25
    sig = 0.35
    edges = (np.arange(n + 1) - n / 2) * dy
    centres = 0.5 * (edges[1:] + edges[:-1])

    def cell_avg(shift):
        c = (erf((edges[1:] - shift) / (np.sqrt(2) * sig)) - erf((edges[:-1] - shift) / (np.sqrt(2) * sig))) / 2
        return c / dy

    psi = np.zeros(o.comp_shape)
    psi[0, 0, 0, 1, :, 0] = cell_avg(-0.5)
    x_end = 4.0
    n_steps = int(steps_per_unit * x_end)
    h = x_end / n_steps
    for _ in range(n_steps):
        psi = o.transport_substep(h, psi)
    exact = cell_avg(-0.5 + u * x_end)
    err = np.abs(psi[0, 0, 0, 1, :, 0] - exact)
    far = np.abs(centres - (-0.5 + u * x_end)) > 0.5
    return err.sum() * dy, err[far].sum() * dy


def test_transport_pure_shift_converges(oracle_mod):
    """Pure-shift solution psi0(y - u x): the L1 error falls with refinement,
    at second order in the smooth part (the limiter clips the extremum, which
    costs order there, as for any TVD scheme)."""
    (a1, f1), (a2, f2), (a3, f3) = (_shift_error(oracle_mod, n, n // 4) for n in (80, 160, 320))
    assert a2 < a1 and a3 < a2
    assert np.log2(a2 / a3) > 1.6, (a1, a2, a3)
    assert np.log2(f2 / f3) > 1.9, (f1, f2, f3)


# ---------------------------------------------------------------- angular

def _dense_laplacian(n, d):
    return (np.diag(-2 * np.ones(n)) + np.diag(np.ones(n - 1), 1) + np.diag(np.ones(n - 1), -1)) / d ** 2


@pytest.mark.parametrize("nu,nv", [(4, 4), (6, 3), (8, 8)])
def test_angular_dst_equals_dense_cn_solve(oracle_mod, nu, nv):
    """The sine-transform Crank-Nicolson step equals the dense Kronecker
    five-point-Laplacian CN solve done with numpy's LU."""
    o = oracle_mod.Oracle(_grid(3, 2, nu, nv, ng=2))
    ts = o.tables()["ts"]
    rng = np.random.default_rng(2)
    psi = rng.random(o.comp_shape)
    rho = np.array([[1.0, 1.85], [0.26, 1.0], [0.7, 1.3]])
    h = 2.5  # a long step so that the diffusion is visible
    out = o.angular_substep(h, rho, psi)
    lap = np.kron(np.eye(nv), _dense_laplacian(nu, o.du)) + np.kron(_dense_laplacian(nv, o.dv), np.eye(nu))
    I = np.eye(nu * nv)
    for g in range(2):
        for c in range(2):
            for p in range(3):
                for q in range(2):
                    k = rho[p, q] * ts[g]
                    x0 = psi[g, c, :, :, p, q].reshape(-1)
                    ref = np.linalg.solve(I - 0.5 * h * 0.5 * k * lap, (I + 0.5 * h * 0.5 * k * lap) @ x0)
                    assert np.allclose(out[g, c, :, :, p, q].reshape(-1), ref, rtol=1e-11, atol=1e-13)


@pytest.mark.parametrize("nu,nv", [(4, 4), (6, 3), (8, 8)])
def test_angular_exact_integrator_equals_matrix_exponential(oracle_mod, nu, nv):
    """The exact-exponential angular integrator (the paper's "ODE solver"
    reading) equals the exact solution of the semi-discrete system,
    expm(h kappa/2 L) psi with L the dense Kronecker five-point Laplacian
    (scipy's expm), and it is a semigroup: two steps h/2 = one step h."""
    from scipy.linalg import expm
    o = oracle_mod.Oracle(_grid(3, 2, nu, nv, ng=2))
    o.set_angular_exact(True)
    ts = o.tables()["ts"]
    rng = np.random.default_rng(3)
    psi = rng.random(o.comp_shape)
    rho = np.array([[1.0, 1.85], [0.26, 1.0], [0.7, 1.3]])
    h = 2.5
    out = o.angular_substep(h, rho, psi)
    lap = np.kron(np.eye(nv), _dense_laplacian(nu, o.du)) + np.kron(_dense_laplacian(nv, o.dv), np.eye(nu))
    for g in range(2):
        for c in range(2):
            for p in range(3):
                for q in range(2):
                    k = rho[p, q] * ts[g]
                    ref = expm(0.5 * h * k * lap) @ psi[g, c, :, :, p, q].reshape(-1)
                    assert np.allclose(out[g, c, :, :, p, q].reshape(-1), ref, rtol=1e-10, atol=1e-13)
    half = o.angular_substep(0.5 * h, rho, o.angular_substep(0.5 * h, rho, psi))
    assert np.allclose(half, out, rtol=1e-12, atol=1e-14)
    # Crank-Nicolson is not a semigroup: the two integrators differ at this step
    o.set_angular_exact(False)
    cn = o.angular_substep(h, rho, psi)
    assert np.abs(cn - out).max() > 1e-6 * np.abs(out).max()


def test_angular_mass_change_is_wall_flux(oracle_mod):
    """d/dx sum psi = (kappa/2) [sum of -(psi_1 + psi_N)/du^2 over rows and
    columns]; CN makes the change the trapezoid of that wall term."""
    nu = nv = 6
    o = oracle_mod.Oracle(_grid(1, 1, nu, nv, ng=1))
    ts = o.tables()["ts"][0]
    rng = np.random.default_rng(4)
    psi = rng.random(o.comp_shape)
    h = 7.0
    out = o.angular_substep(h, np.ones((1, 1)), psi)

    def wall(x):
        x = x.reshape(nv, nu)
        return -(x[:, 0].sum() + x[:, -1].sum()) / o.du ** 2 - (x[0, :].sum() + x[-1, :].sum()) / o.dv ** 2

    for c in range(2):
        a = psi[0, c, :, :, 0, 0]
        b = out[0, c, :, :, 0, 0]
        assert b.sum() - a.sum() == pytest.approx(0.5 * h * 0.5 * ts * (wall(a) + wall(b)), rel=1e-11)


def test_angular_second_moment_grows_linearly(oracle_mod):
    """Away from the walls d<u^2>/dx = kappa exactly for the five-point
    Laplacian, and CN integrates it exactly: <u^2> = <u^2>_0 + kappa h."""
    n = 31
    o = oracle_mod.Oracle(dict(ny=1, nz=1, nu=n, nv=n, dy=0.1, dz=0.1, u_max=0.3, v_max=0.3,
                               e_faces=np.array([50.0, 51.0])))
    t = o.tables()
    ts, u = t["ts"][0], t["u"]
    psi = np.zeros(o.comp_shape)
    psi[0, 0, n // 2, n // 2] = 1.0
    h = 1.0
    out = psi
    for _ in range(3):
        out = o.angular_substep(h, np.ones((1, 1)), out)
    x = out[0, 0, :, :, 0, 0]
    m0 = x.sum()
    m2u = (x * u[None, :] ** 2).sum() / m0
    assert m2u == pytest.approx(ts * 3 * h, rel=1e-5)  # the residue is wall leakage of the ringing CN modes
    assert m0 == pytest.approx(1.0, rel=1e-6)
