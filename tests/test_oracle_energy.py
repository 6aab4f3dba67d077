"""Pins of the oracle's energy operator and energy Crank-Nicolson step
(Section 3.2, Eq. 0041-d; Section 3.3) against closed forms, a dense library
solve and conservation identities."""
import os

import numpy as np
import pytest
from scipy import integrate

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _lane_grid(ng, e_min, e_max):
    return dict(ny=1, nz=1, nu=1, nv=1, dy=0.1, dz=0.1, u_max=0.1, v_max=0.1,
                e_faces=np.linspace(e_min, e_max, ng + 1))


def test_constant_state_constant_s_is_steady(oracle_mod):
    """With S constant (p = 1 makes S = 1/alpha) and no removal, a state that
    is constant in E has d/dE(S psi) = 0: every group below the top one must
    have a zero right-hand side.  The printed minus sign in the phi^2-tested
    lower-face flux would give -6 S c / dE in the psi^2 row instead."""
    o = oracle_mod.Oracle(_lane_grid(12, 10.0, 70.0), dict(bk_p=1.0, sigma_ct=0.0))
    x = np.zeros((12, 2))
    x[:, 0] = 3.7
    out = o.energy_apply(1.0, x).reshape(12, 2)
    assert np.max(np.abs(out[:-1])) < 1e-12 * (3.7 / 0.0022)
    assert abs(out[-1, 0]) > 1.0  # the top group drains (nothing enters above it)


def _linear_in_group_s(o, g):
    t = o.tables()
    sp, sm = t["s_face"][g + 1], t["s_face"][g]
    ec, de = t["e_c"][g], t["de"][g]
    return lambda e: 0.5 * (sp + sm) + (sp - sm) / de * (e - ec)


@pytest.mark.parametrize("p", [1.0, 1.77])
def test_linear_state_exact_moments(oracle_mod, p):
    """For psi(E) = a0 + b0 E (continuous) the upwind interface values are exact,
    so both rows must equal the exact moments of d/dE(S psi) with the
    linear-in-group S of Eq. appSE:  (1/dE) int d/dE(S psi) and
    (3/dE) int d/dE(S psi) phi^2, evaluated by quadrature."""
    G = 10
    o = oracle_mod.Oracle(_lane_grid(G, 20.0, 120.0), dict(bk_p=p, sigma_ct=0.0))
    t = o.tables()
    a0, b0 = 0.7, 0.013
    x = np.zeros((G, 2))
    x[:, 0] = a0 + b0 * t["e_c"]
    x[:, 1] = b0 * t["de"] / 2.0
    out = o.energy_apply(1.0, x).reshape(G, 2)
    for g in range(G - 1):
        lo, hi = o.e_faces[g], o.e_faces[g + 1]
        de, ec = hi - lo, 0.5 * (lo + hi)
        s = _linear_in_group_s(o, g)
        psi = lambda e: a0 + b0 * e
        phi2 = lambda e: 2.0 * (e - ec) / de
        # d/dE (S psi) with S linear in the group and psi linear
        ds = (t["s_face"][g + 1] - t["s_face"][g]) / de
        dsp = lambda e: ds * psi(e) + s(e) * b0
        m1 = integrate.quad(dsp, lo, hi, epsrel=1e-13)[0] / de
        # first row uses the exact face values S_{g+1/2} psi(E+) - S_{g-1/2} psi(E-)
        m1_faces = (t["s_face"][g + 1] * psi(hi) - t["s_face"][g] * psi(lo)) / de
        assert out[g, 0] == pytest.approx(m1_faces, rel=1e-12)
        assert m1 == pytest.approx(m1_faces, rel=1e-10)
        m2 = 3.0 / de * integrate.quad(lambda e: dsp(e) * phi2(e), lo, hi, epsrel=1e-13)[0]
        assert out[g, 1] == pytest.approx(m2, rel=1e-10, abs=1e-10)


def _dense_operator(o, rho):
    n = 2 * o.ng
    A = np.zeros((n, n))
    for k in range(n):
        e = np.zeros(n)
        e[k] = 1.0
        A[:, k] = o.energy_apply(rho, e)
    return A


def test_cn_scan_matches_dense_solve(oracle_mod):
    """The descending block substitution solves (I - h/2 A) x = (I + h/2 A) x0
    + h/2 src exactly as numpy's dense LU does."""
    G = 9
    o = oracle_mod.Oracle(_lane_grid(G, 0.0, 60.0))
    rng = np.random.default_rng(3)
    x0 = rng.random(2 * G)
    src = rng.random(G)
    for rho, h in ((1.0, 0.05), (1.85, 0.3), (0.26, 0.01)):
        A = _dense_operator(o, rho)
        I = np.eye(2 * G)
        rhs = (I + 0.5 * h * A) @ x0
        rhs[0::2] += 0.5 * h * src
        x_ref = np.linalg.solve(I - 0.5 * h * A, rhs)
        x, dep, dep_w = o.energy_cn_lane(rho, h, x0, src)
        assert np.allclose(x, x_ref, rtol=1e-12, atol=1e-14 * np.abs(x_ref).max())
        assert dep == pytest.approx(dep_w, rel=1e-11)


def test_particle_count_balance(oracle_mod):
    """sum_g dE psi^1 changes only by outflow through the lowest face and by
    catastrophic removal: N1 - N0 = -h/2 [rho S_1/2 ((psi1-psi2)_0 old + new)
    + rho sigma sum dE (psi^1 old + new)] - exact up to rounding."""
    G = 16
    o = oracle_mod.Oracle(_lane_grid(G, 0.0, 40.0))
    t = o.tables()
    rng = np.random.default_rng(5)
    x0 = rng.random((G, 2))
    rho, h = 1.3, 0.07
    x1, _, _ = o.energy_cn_lane(rho, h, x0)
    x1 = x1.reshape(G, 2)
    n0 = np.sum(t["de"] * x0[:, 0])
    n1 = np.sum(t["de"] * x1[:, 0])
    out = rho * t["s_face"][0] * ((x0[0, 0] - x0[0, 1]) + (x1[0, 0] - x1[0, 1]))
    rem = rho * 0.012 * np.sum(t["de"] * (x0[:, 0] + x1[:, 0]))
    assert n1 - n0 == pytest.approx(-0.5 * h * (out + rem), rel=1e-12)


def _count_curve(o, e0, dx, n_steps):
    beam = dict(e0=e0, sigma_e=1.0, sigma_y=1.0, sigma_z=1.0)
    rho = np.ones((n_steps, 1, 1))
    r = o.march(rho, n_steps, dx, beam=beam, do_transport=False, do_angular=False)
    return r


def test_csda_range_of_the_march(oracle_mod):
    """With scattering, transport and removal off, the depth at which the
    particle count of a lane falls to 50 % is the CSDA range R(E0) = alpha E0^p
    (golden values), and the deposited energy adds up to the beam energy."""
    rows = {}
    with open(os.path.join(GOLDEN, "csda_range.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                e, r = line.split()
                rows[float(e)] = float(r)
    e0 = 100.0
    o = oracle_mod.Oracle(_lane_grid(220, 0.0, 110.0), dict(sigma_ct=0.0))
    dx = 0.02
    n = int(8.0 / dx)
    r = _count_curve(o, e0, dx, n)
    flu = r["fluence"][:, 0, 0] * 0.01  # protons (lane area 0.1 x 0.1 cm)
    depth = np.arange(n + 1) * dx
    k = np.nonzero(flu < 0.5)[0][0]
    x50 = depth[k - 1] + (0.5 - flu[k - 1]) / (flu[k] - flu[k - 1]) * dx
    assert x50 == pytest.approx(rows[e0], rel=3e-3)
    # all the energy is deposited (E_dep = dose * rho * volume)
    edep = r["dose"][:, 0, 0].sum() * dx * 0.01
    t = o.tables()
    psi0 = o.init_beam(dict(e0=e0, sigma_e=1.0, sigma_y=1.0, sigma_z=1.0))
    e_in = np.sum(t["de"] * (t["e_c"] * psi0[:, 0, 0, 0, 0, 0] + t["de"] * psi0[:, 1, 0, 0, 0, 0] / 6.0)) \
        * o.du * o.dv * 0.01
    psi1 = r["psi"][0, :, :, 0, 0, 0, 0]
    e_left = np.sum(t["de"] * (t["e_c"] * psi1[:, 0] + t["de"] * psi1[:, 1] / 6.0)) * o.du * o.dv * 0.01
    assert edep + e_left == pytest.approx(e_in, rel=1e-12)
    # Crank-Nicolson is not L-stable: the stiff lowest groups ring with
    # alternating sign and leave a small (here negative) residue after the range
    assert abs(e_left) < 1e-3 * e_in
    assert e_in == pytest.approx(e0, rel=1e-3)


def test_mean_energy_follows_range_law(oracle_mod):
    """Mean energy of the lane at depth x follows E(x) = ((R0 - x)/alpha)^(1/p)."""
    o = oracle_mod.Oracle(_lane_grid(440, 0.0, 110.0), dict(sigma_ct=0.0))
    dx, n = 0.02, 200
    beam = dict(e0=100.0, sigma_e=1.0, sigma_y=1.0, sigma_z=1.0)
    r = o.march(np.ones((n, 1, 1)), n, dx, beam=beam, do_transport=False, do_angular=False)
    t = o.tables()
    psi = r["psi"][0, :, :, 0, 0, 0, 0]
    e_mean = np.sum(t["de"] * (t["e_c"] * psi[:, 0] + t["de"] * psi[:, 1] / 6.0)) / np.sum(t["de"] * psi[:, 0])
    R0 = 0.0022 * 100.0 ** 1.77
    e_exp = ((R0 - n * dx) / 0.0022) ** (1 / 1.77)
    assert e_mean == pytest.approx(e_exp, rel=2e-3)


def _error1(o, dx, n_steps, e0=50.0):
    """error_1 of Eq. (error): sum_g sum_s |psi^1_{dx} - psi^1_{dx/2}| dx dE_g on
    the (y,z,u,v)-integrated state (one lane in water)."""
    beam = dict(e0=e0, sigma_e=1.0, sigma_y=1.0, sigma_z=1.0)
    t = o.tables()

    def run(h, n):
        out = []
        psi = o.init_beam(beam)[None]
        for s in range(n):
            psi = o.march(np.ones((1, 1, 1)), 1, h, psi=psi, do_transport=False, do_angular=False)["psi"]
            out.append(psi[0, :, 0, 0, 0, 0, 0].copy())
        return np.array(out)

    a = run(dx, n_steps)
    b = run(dx / 2, 2 * n_steps)[1::2]
    return np.sum(np.abs(a - b) * t["de"][None, :]) * dx


def test_second_order_in_depth(oracle_mod):
    """Strang + CN converges at second order in dx (Section 4.1): error_1
    falls by about 4 when dx halves."""
    o = oracle_mod.Oracle(_lane_grid(60, 0.0, 60.0))
    e1 = _error1(o, 0.04, 25)
    e2 = _error1(o, 0.02, 50)
    ratio = e1 / e2
    assert 3.3 < ratio < 4.8, ratio
