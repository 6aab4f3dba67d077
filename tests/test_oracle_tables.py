"""Pins of the oracle's physics tables against closed forms, quadrature and
geometry that do not reuse the oracle's own formulas."""
import math
import os

import numpy as np
import pytest
from scipy import integrate, special

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _grid(ng=64, e_max=110.0, e_min=0.0, n=8, u_max=0.1, ny=4):
    return dict(ny=ny, nz=ny, nu=n, nv=n, dy=0.1, dz=0.1, u_max=u_max, v_max=u_max,
                e_faces=np.linspace(e_min, e_max, ng + 1))


def _golden_rows(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append(line.split())
    return rows


def test_csda_range_from_stopping_power(oracle_mod):
    """R(E0) = int dE / S(E) must give the tabulated Bragg-Kleeman ranges:
    integrate 1/S from the oracle's face values on a fine grid."""
    o = oracle_mod.Oracle(_grid(ng=4000, e_min=1.0, e_max=231.0))
    t = o.tables()
    e = o.e_faces
    inv_s = 1.0 / t["s_face"]
    cum = np.concatenate([[0.0], np.cumsum(0.5 * (inv_s[1:] + inv_s[:-1]) * np.diff(e))])
    alpha, p = 0.0022, 1.77
    for e0, r in _golden_rows("csda_range.txt"):
        e0, r = float(e0), float(r)
        r_num = np.interp(e0, e, cum) + alpha * 1.0 ** p  # add the range below 1 MeV
        assert abs(r_num - r) < 2e-3 * r, (e0, r_num, r)


def test_energy_floor_face(oracle_mod):
    """A face at E = 0 takes S at half the lowest group width."""
    o = oracle_mod.Oracle(_grid(ng=10, e_max=10.0))
    s = o.tables()["s_face"]
    s_half = 0.5 ** (1 - 1.77) / (0.0022 * 1.77)
    assert s[0] == pytest.approx(s_half, rel=1e-14)
    assert np.all(np.diff(s) < 0)  # stopping power falls with energy


def test_highland_kinematics(oracle_mod):
    """p*v from relativistic kinematics (gamma, beta) equals the oracle's
    E(E+2M)/(E+M) inside the Highland scattering power."""
    M = 938.272
    for e in (1.0, 10.0, 100.0, 230.0):
        gam = 1.0 + e / M
        beta = math.sqrt(1.0 - 1.0 / gam ** 2)
        pv = gam * beta ** 2 * M  # p c * beta
        expect = (13.6 / pv) ** 2 / 36.08
        assert oracle_mod.highland(e) == pytest.approx(expect, rel=1e-12)


def test_scattering_power_group_average(oracle_mod):
    """sigma_tr,g is the group average (after Eq. 0041-d): compare the oracle's
    closed-form primitive with adaptive quadrature of the pointwise value."""
    o = oracle_mod.Oracle(_grid(ng=16, e_min=0.0, e_max=160.0))
    ts = o.tables()["ts"]
    floor = 0.5 * 10.0
    for g in range(16):
        lo = max(o.e_faces[g], floor)
        hi = o.e_faces[g + 1]
        val, _ = integrate.quad(lambda e: oracle_mod.highland(e), lo, hi, epsabs=0, epsrel=1e-13)
        assert ts[g] == pytest.approx(val / (hi - lo), rel=1e-10)


def test_p1_exponential_and_normalised(oracle_mod):
    o = oracle_mod.Oracle(_grid(ng=32))
    t = o.tables()
    p1, de = t["p1"], t["de"]
    lam = 0.05
    assert np.allclose(p1.sum(axis=1), 1.0, atol=1e-14)
    assert np.all(np.triu(p1, 1) == 0.0)  # protons only lose energy
    for gp in (5, 20, 31):
        ratio = p1[gp, 1:gp + 1] / p1[gp, 0:gp]
        assert np.allclose(ratio, math.exp(lam * de[0]), rtol=1e-12)  # closer to g' is likelier


def _direction(u, v):
    w = np.array([1.0, u, v])
    return w / np.linalg.norm(w)


def test_p2_geometry_and_normalisation(oracle_mod):
    """P^2 depends on the 3-D angle between the directions (1,u,v) and
    (1,u',v') through a Gamma density, and integrates to one over (u,v)."""
    n = 6
    o = oracle_mod.Oracle(_grid(ng=2, n=n, u_max=0.15))
    t = o.tables()
    p2, u, v = t["p2"], t["u"], t["v"]
    na = n * n
    assert np.allclose(p2.sum(axis=1) * o.du * o.dv, 1.0, atol=1e-13)
    al, be = 2.0, 40.0
    for ap in (0, 7, 20, 35):
        dp = _direction(u[ap % n], v[ap // n])
        th = []
        for a in range(na):
            d = _direction(u[a % n], v[a // n])
            th.append(math.atan2(np.linalg.norm(np.cross(d, dp)), float(np.dot(d, dp))))
        th = np.array(th)
        dens = be ** al / special.gamma(al) * th ** (al - 1) * np.exp(-be * th)
        k = dens.sum() * o.du * o.dv
        assert np.allclose(p2[0, :, ap], dens / k, rtol=1e-10, atol=1e-12)
    # mirror symmetry u -> -u maps column ap to its mirror
    grid = p2[0].reshape(n, n, n, n)  # [j][i][j'][i']
    assert np.allclose(grid, grid[:, ::-1, :, ::-1], rtol=1e-12, atol=1e-14)
    assert np.allclose(grid, grid.transpose(1, 0, 3, 2), rtol=1e-12, atol=1e-14)


def test_angle_nodes(oracle_mod):
    for n in (7, 8, 16):
        o = oracle_mod.Oracle(_grid(ng=2, n=n, u_max=0.15))
        u = o.tables()["u"]
        du = 0.3 / (n + 1)
        assert np.allclose(np.diff(u), du, rtol=1e-13)
        assert np.allclose(u, -u[::-1], atol=1e-16)
        assert u[0] == pytest.approx(-0.15 + du, rel=1e-13)
