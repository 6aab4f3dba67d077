"""Pins of the oracle's energy straggling (Section 3.2, Eq. 0041-d with the
terms Q_1, Q_2; Appendix A.2): the interior-penalty (SIPG) form of
(rho/2) d/dE(T dpsi/dE), the drift (rho/2) d/dE(T' psi) folded into the
stopping power, the two time integrators (straggling explicit inside CN, or
inside CN), and the Williams straggling coefficient of water.

Properties checked (each fails for a plausible slip: a dropped symmetric
term, a wrong jump sign or index, a missing 1/2, a penalty without T):
  * the mass-weighted SIPG matrix is symmetric and negative semi-definite
    with the paper's penalty alpha = (p + 1)^2 / 2 = 2;
  * it conserves the particle count, and with constant T it keeps the mean
    energy and grows <E^2> by exactly rho T per unit depth (the continuous
    operator's moments);
  * with T linear in E the SIPG part plus the T'/2 drift keep the mean energy;
  * the CN solves equal dense linear solves of the same systems;
  * the explicit form converges to the CN form at first order in h;
  * with the Appendix-A physics the integrated depth dose reproduces the
    landmarks and the distal width the paper prints.
"""
import os

import numpy as np
import pytest


def _oracle(orc, G=24, nonuniform=False, t_face=None, seed=0, **phys):
    rng = np.random.default_rng(seed)
    if nonuniform:
        faces = np.concatenate([[0.0], np.cumsum(rng.uniform(0.6, 1.4, G))])
    else:
        faces = np.linspace(0.0, float(G), G + 1)
    o = orc.Oracle(dict(ny=1, nz=1, nu=1, nv=1, dy=1.0, dz=1.0, u_max=0.1, v_max=0.1, e_faces=faces), phys)
    if t_face is not None:
        o.set_straggling_table(t_face(faces) if callable(t_face) else t_face)
    return o, faces


def _dense(apply, G, rho):
    cols = [apply(rho, e) for e in np.eye(2 * G)]
    return np.array(cols).T


def _mass(faces):
    de = np.diff(faces)
    return np.ravel(np.column_stack([de, de / 3.0]))  # int phi^l phi^l = dE / (2l - 1)


def _gauss_state(faces, mu, sd):
    """P1 L2 projection of a Gaussian in E onto the groups (Gauss-Legendre)."""
    x, w = np.polynomial.legendre.leggauss(8)
    out = np.zeros(2 * (len(faces) - 1))
    for g in range(len(faces) - 1):
        lo, hi = faces[g], faces[g + 1]
        e = 0.5 * (lo + hi) + 0.5 * (hi - lo) * x
        f = np.exp(-0.5 * ((e - mu) / sd) ** 2)
        out[2 * g] = 0.5 * np.sum(w * f)
        out[2 * g + 1] = 1.5 * np.sum(w * f * x)
    return out


def _moments(faces, x):
    de, ec = np.diff(faces), 0.5 * (faces[1:] + faces[:-1])
    p1, p2 = x[0::2], x[1::2]
    n = np.sum(de * p1)
    m1 = np.sum(de * (ec * p1 + de * p2 / 6.0))
    m2 = np.sum(de * (ec ** 2 + de ** 2 / 12.0) * p1 + de ** 2 * ec * p2 / 3.0)
    return n, m1, m2


@pytest.mark.parametrize("nonuniform", [False, True])
@pytest.mark.parametrize("tkind", ["const", "random"])
def test_sipg_symmetric_negative_semidefinite_conservative(oracle_mod, nonuniform, tkind):
    G = 20
    rng = np.random.default_rng(5)
    tf = np.ones(G + 1) if tkind == "const" else rng.uniform(0.3, 2.0, G + 1)
    o, faces = _oracle(oracle_mod, G, nonuniform, tf)
    A = _dense(o.straggle_apply, G, 1.3)
    B = _mass(faces)[:, None] * A
    scale = np.abs(B).max()
    assert np.abs(B - B.T).max() < 1e-13 * scale
    assert np.linalg.eigvalsh(0.5 * (B + B.T)).max() < 1e-12 * scale
    # particle count: sum dE (A x)^1 = 0 for every x
    assert np.abs(np.diff(faces) @ A[0::2]).max() < 1e-13 * scale
    # the blocks are the dense matrix's 2x2 pieces
    for g in (0, 7, G - 1):
        alo, agg, aup = o.straggle_blocks(g, 1.3)
        assert np.allclose(agg, A[2 * g:2 * g + 2, 2 * g:2 * g + 2], rtol=0, atol=1e-14 * scale)
        if g > 0:
            assert np.allclose(alo, A[2 * g:2 * g + 2, 2 * g - 2:2 * g], rtol=0, atol=1e-14 * scale)
        if g + 1 < G:
            assert np.allclose(aup, A[2 * g:2 * g + 2, 2 * g + 2:2 * g + 4], rtol=0, atol=1e-14 * scale)


def test_penalty_is_coercive(oracle_mod):
    """With alpha = 2 the mass-weighted SIPG matrix has a one-dimensional
    null space (the constants) and its other eigenvalues are bounded away
    from zero: the penalty is coercive, not marginal (with alpha = 1 or a
    penalty without T the largest eigenvalue turns positive)."""
    G = 16
    o, faces = _oracle(oracle_mod, G, False, np.ones(G + 1))
    B = _mass(faces)[:, None] * _dense(o.straggle_apply, G, 1.0)
    ev = np.sort(np.linalg.eigvalsh(0.5 * (B + B.T)))
    assert abs(ev[-1]) < 1e-12 and ev[-2] < -1e-3


@pytest.mark.parametrize("nonuniform,tol2", [(False, 1e-10), (True, 1e-3)])
def test_constant_T_moments(oracle_mod, nonuniform, tol2):
    """Constant T, a state that vanishes at both ends: d N / dx = 0 and
    d<E>/dx = 0 exactly, and d<E^2>/dx = rho T N as for the continuous
    operator (rho/2) T d^2/dE^2 -- exactly on uniform groups, to the
    discretisation error on uneven ones."""
    G, rho, T = 60, 1.7, 0.8
    o, faces = _oracle(oracle_mod, G, nonuniform, np.full(G + 1, T), seed=3)
    x = _gauss_state(faces, 0.5 * faces[-1], 0.05 * faces[-1])
    n, _, _ = _moments(faces, x)
    dn, dm1, dm2 = _moments(faces, o.straggle_apply(rho, x))
    assert abs(dn) < 1e-12 * n and abs(dm1) < 1e-12 * n * faces[-1]
    assert abs(dm2 - rho * T * n) < tol2 * rho * T * n


def test_linear_T_drift_keeps_the_mean_energy(oracle_mod):
    """T = a + b E: (rho/2) d^2(T psi)/dE^2 keeps N and <E> and grows <E^2>
    by rho int T psi.  The SIPG part alone changes <E> by rho b N / 2; the
    T'/2 drift folded into the stopping power (with S and removal off) must
    cancel it."""
    G, rho = 50, 1.2
    lin = lambda f: 0.3 + 0.02 * f  # noqa: E731
    o, faces = _oracle(oracle_mod, G, False, lin, s_scale=0.0, sigma_ct=0.0)
    tb = o.straggling()
    assert np.allclose(tb["t_face"], lin(faces)) and not tb["s_base"].any()
    assert np.allclose(o.tables()["s_face"], 0.5 * 0.02)  # T'/2 at every face
    x = _gauss_state(faces, 25.0, 4.0)
    n, _, _ = _moments(faces, x)
    ax = o.straggle_apply(rho, x) + o.energy_apply(rho, x)
    dn, dm1, dm2 = _moments(faces, ax)
    assert abs(dn) < 1e-8 * n and abs(dm1) < 1e-8 * n * 25.0
    de, ec = np.diff(faces), 0.5 * (faces[1:] + faces[:-1])
    int_t_psi = np.sum(de * ((0.3 + 0.02 * ec) * x[0::2] + 0.02 * de / 6.0 * x[1::2]))
    assert abs(dm2 - rho * int_t_psi) < 1e-6 * rho * int_t_psi
    # the SIPG part alone does move the mean
    assert abs(_moments(faces, o.straggle_apply(rho, x))[1] - 0.5 * rho * 0.02 * n) < 1e-8 * n


@pytest.mark.parametrize("full", [False, True])
def test_cn_solves_equal_dense_solves(oracle_mod, full):
    G, rho, h = 18, 1.4, 0.3
    rng = np.random.default_rng(9)
    o, faces = _oracle(oracle_mod, G, True, rng.uniform(0.5, 3.0, G + 1), seed=4)
    o.set_straggling_cn(full)
    AS = _dense(o.energy_apply, G, rho)
    AT = _dense(o.straggle_apply, G, rho)
    x0 = rng.uniform(0.0, 1.0, 2 * G)
    src = rng.uniform(0.0, 0.5, G)
    s2 = np.zeros(2 * G)
    s2[0::2] = src
    I = np.eye(2 * G)
    if full:
        ref = np.linalg.solve(I - 0.5 * h * (AS + AT), (I + 0.5 * h * (AS + AT)) @ x0 + 0.5 * h * s2)
    else:
        ref = np.linalg.solve(I - 0.5 * h * AS, (I + 0.5 * h * AS) @ x0 + h * AT @ x0 + 0.5 * h * s2)
    got, dep, dep_w = o.energy_cn_lane(rho, h, x0, src)
    assert np.abs(got - ref).max() < 1e-12 * np.abs(ref).max()
    assert abs(dep - dep_w) < 1e-11 * max(abs(dep), 1e-30)


def test_explicit_straggling_converges_to_cn_at_first_order(oracle_mod):
    """Straggling alone (S and removal off, constant T): march the same depth
    with h and h/2.  The explicit form's distance to the CN form halves."""
    G, rho, depth = 60, 1.0, 2.0
    T = 0.5  # h rho T / dE^2 <= 0.125: inside the explicit form's stability range
    o, faces = _oracle(oracle_mod, G, False, np.full(G + 1, T), s_scale=0.0, sigma_ct=0.0)
    x0 = _gauss_state(faces, 30.0, 3.0)

    def run(full, n):
        o.set_straggling_cn(full)
        x = x0.copy()
        for _ in range(n):
            x = o.energy_cn_lane(rho, depth / n, x)[0]
        return x

    d = [np.abs(run(False, n) - run(True, n)).max() for n in (16, 32, 64)]
    assert 1.8 < d[0] / d[1] < 2.2 and 1.8 < d[1] / d[2] < 2.2
    # and the CN result has the exact variance growth rho T depth
    n0, m10, m20 = _moments(faces, x0)
    n1, m11, m21 = _moments(faces, run(True, 32))
    var0, var1 = m20 / n0 - (m10 / n0) ** 2, m21 / n1 - (m11 / n1) ** 2
    assert abs((var1 - var0) - rho * T * depth) < 1e-9


def test_williams_coefficient_bohr_limit(oracle_mod):
    """At high energy the binding correction shrinks to a few 1e-3 (it keeps
    4 I / (3 m_e c^2) ln(2 m_e c^2 / I) as v -> c in this non-relativistic
    form) and T approaches Bohr's 4 pi r_e^2 (m_e c^2)^2 N_A <Z/A> (about
    0.0871 MeV^2 cm^2/g for water), written here with the classical electron
    radius instead of e^2; toward low energy the correction grows."""
    r_e, mec2, n_a = 2.8179403262e-13, 0.51099895, 6.02214076e23
    za = 0.111894 * 1.0 / 1.00794 + 0.888106 * 8.0 / 15.9994
    bohr = 4.0 * np.pi * r_e ** 2 * mec2 ** 2 * n_a * za
    assert 0.0869 < bohr < 0.0873
    t = [oracle_mod.williams_water(e) for e in (1e5, 1000.0, 200.0, 50.0, 10.0, 2.0)]
    assert 0.0 < t[0] / bohr - 1.0 < 3e-3
    assert all(a < b for a, b in zip(t, t[1:]))


def _landmarks(orc, e0, t_scale, dx=0.02, de=0.5):
    emax = e0 + 10.0
    faces = np.linspace(0.0, emax, int(round(emax / de)) + 1)
    o = orc.Oracle(dict(ny=1, nz=1, nu=1, nv=1, dy=1.0, dz=1.0, u_max=0.1, v_max=0.1, e_faces=faces),
                   dict(model=1, t_scale=t_scale))
    n = int((0.0022 * e0 ** 1.77 * 1.08 + 0.5) / dx)
    r = o.march(np.ones((n, 1, 1)), n, dx, beam=dict(e0=e0, sigma_e=1.0, sigma_y=1.0, sigma_z=1.0), n_scatter=1,
                do_transport=False, do_angular=False)
    idd = r["dose"][:, 0, 0]
    assert np.abs(r["dose"] - r["dose_w"]).max() < 1e-11 * idd.max()
    x = (np.arange(n) + 0.5) * dx
    i = int(np.argmax(idd))
    top = idd[i]

    def crossing(level, side):
        j = i
        if side < 0:
            while j > 0 and idd[j] > level:
                j -= 1
            return x[j] + (level - idd[j]) / (idd[j + 1] - idd[j]) * dx
        while j < n - 1 and idd[j] > level:
            j += 1
        return x[j - 1] + (idd[j - 1] - level) / (idd[j - 1] - idd[j]) * dx

    return np.array([x[i], crossing(0.9 * top, -1), crossing(0.9 * top, 1), crossing(0.2 * top, 1)])


@pytest.mark.parametrize("e0", [50, 100, 230])
def test_straggling_reproduces_the_paper_distal_falloff(oracle_mod, e0):
    """With Appendix A (Bethe-Bloch stopping, Williams straggling) the depth
    dose puts BP, P90, D90 and D20 within 0.5 % of the deterministic column
    of the paper's water table (tests/golden/paper_idd_landmarks.txt), and the
    distal width D20 - D90 within 6 % of the printed one; without straggling
    the width is 3-33 % short."""
    ref = None
    with open(os.path.join(os.path.dirname(__file__), "golden", "paper_idd_landmarks.txt")) as f:
        for line in f:
            s = line.split()
            if s and s[0] == "water" and int(s[1]) == e0:
                ref = np.array([float(v) for v in s[2:6]])
    got = _landmarks(oracle_mod, float(e0), 1.0)
    assert np.all(np.abs(got / ref - 1.0) < 0.005), (got, ref)
    w, w_ref = got[3] - got[2], ref[3] - ref[2]
    assert abs(w / w_ref - 1.0) < 0.06, (w, w_ref)
    none = _landmarks(oracle_mod, float(e0), 0.0)
    assert abs((none[3] - none[2]) / w_ref - 1.0) > abs(w / w_ref - 1.0)


@pytest.mark.parametrize("full", [False, True])
def test_march_energy_balance_with_straggling(oracle_mod, full):
    """A K = 1 march with straggling (Appendix-A physics), transport on and
    angular diffusion off so that nothing leaves through the walls: the
    energy content lost by the state equals the tallied deposit (difference
    form) and the operator-form tally, for both straggling integrators."""
    G, n, dx = 60, 20, 0.05
    grid = dict(ny=16, nz=16, nu=4, nv=4, dy=0.1, dz=0.1, u_max=0.1, v_max=0.1,
                e_faces=np.linspace(0.0, 60.0, G + 1))
    o = oracle_mod.Oracle(grid, dict(model=1, t_scale=5.0))
    o.set_straggling_cn(full)
    t = o.tables()
    beam = dict(e0=45.0, sigma_e=1.5, sigma_y=0.15, sigma_z=0.15)
    r = o.march(np.ones((n, 16, 16)), n, dx, beam=beam, n_scatter=1, do_angular=False)
    psi0 = o.init_beam(beam)

    def content(p):  # p: [..., g, c, j, i, y, z]
        e = (t["de"] * t["e_c"])[:, None, None, None, None] * p[..., :, 0, :, :, :, :] + \
            (t["de"] ** 2 / 6)[:, None, None, None, None] * p[..., :, 1, :, :, :, :]
        return e.sum() * o.du * o.dv * o.dy * o.dz

    dep = r["dose"].sum() * dx * o.dy * o.dz  # rho = 1
    assert content(psi0) - content(r["psi"]) == pytest.approx(dep, rel=1e-10)
    assert r["dose"] == pytest.approx(r["dose_w"], rel=1e-9, abs=1e-12 * np.abs(r["dose"]).max())
