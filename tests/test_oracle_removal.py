"""Pins of the group-dependent catastrophic removal sigma_c,t,g (Section 4:
the removal term of Eq. 0041-do and sigma_c,s = sigma_c,t P^1 P^2; Remark 1).

The reading frozen in the oracle and the library: group g loses protons at
its own rate rho sigma_g, and the source a group receives from g' >= g
carries sigma_g' of the emitting group.  With a constant sigma every reading
coincides, so each pin below uses a table that varies by two orders of
magnitude across the groups."""
import numpy as np
import pytest


def _grid(ny, nz, nu, ng, e_min, e_max):
    return dict(ny=ny, nz=nz, nu=nu, nv=nu, dy=0.1, dz=0.1, u_max=0.15, v_max=0.15,
                e_faces=np.linspace(e_min, e_max, ng + 1))


def _sigma_table(ng, seed=4):
    """Strongly group-dependent removal: log-uniform in [1e-3, 1e-1] cm^2/g."""
    return 10.0 ** np.random.default_rng(seed).uniform(-3.0, -1.0, size=ng)


def test_removal_alone_decays_each_group_at_its_own_rate(oracle_mod):
    """With the stopping power off (S = 0) the energy operator is diagonal,
    d psi_g / dx = -rho sigma_g psi_g for both DG coefficients, and its
    Crank-Nicolson step over h is the closed form
    psi_new = (1 - h rho sigma_g / 2) / (1 + h rho sigma_g / 2) psi_old.
    A removal term that took a neighbouring group's sigma, dropped rho or
    mixed the coefficients fails this."""
    ng = 9
    o = oracle_mod.Oracle(_grid(3, 2, 2, ng, 0.0, 90.0), dict(s_scale=0.0))
    sig = _sigma_table(ng)
    o.set_sigma(sig)
    assert np.array_equal(o.tables()["sig"], sig)
    rng = np.random.default_rng(1)
    psi = rng.random(o.comp_shape)
    rho = rng.uniform(0.2, 1.9, size=(3, 2))
    h = 3.0
    out, edep, edep_w = o.energy_substep(h, rho, psi)
    q = h * rho[None, :, :] * sig[:, None, None] / 2.0          # [g][p][q]
    fac = (1.0 - q) / (1.0 + q)
    ref = psi * fac[:, None, None, None, :, :]
    assert np.allclose(out, ref, rtol=1e-13, atol=0.0)
    # the removed protons take their energy content with them: the tally of
    # the substep equals the loss of du dv dy dz sum_g dE (E_g psi^1 + dE psi^2 / 6)
    t = o.tables()
    w1 = (t["de"] * t["e_c"])[:, None, None, None, None]
    w2 = (t["de"] ** 2 / 6.0)[:, None, None, None, None]
    content = lambda x: ((w1 * x[:, 0] + w2 * x[:, 1]).sum(axis=(0, 1, 2))) * o.du * o.dv * 0.1 * 0.1
    assert np.allclose(edep, content(psi) - content(out), rtol=1e-12)
    assert np.allclose(edep_w, edep, rtol=1e-11)


def _destination_sigma_source(o, rho, prev, sig):
    """The other reading of Section 4 (sigma of the receiving group), written
    out only to show that the pin below tells the two apart."""
    t = o.tables()
    G, na = o.ng, o.nu * o.nv
    p1, p2, de = t["p1"], t["p2"], t["de"]
    ps1 = prev[:, 0].reshape(G, na, o.ny, o.nz)
    out = np.zeros((G, na, o.ny, o.nz))
    for g in range(G):
        r = np.zeros((na, o.ny, o.nz))
        for gp in range(g, G):
            r += rho * sig[g] * p1[gp, g] * ps1[gp] * de[gp] / de[g]
        out[g] = o.du * o.dv * np.einsum("ab,byz->ayz", p2[g], r)
    return out.reshape(o.src_shape)


def test_source_injects_what_group_dependent_removal_takes(oracle_mod):
    """Particle bookkeeping with a strongly varying sigma_g: with P^1 summing
    to one over the receiving groups and P^2 normalised over the outgoing
    angles, the source of component k+1 puts back, per (y, z), exactly what
    removal takes from component k:
        du dv sum_{g,a} src dE_g = du dv sum_{g',a'} rho sigma_g' psi^1_g' dE_g'.
    The destination-group reading breaks this identity by tens of percent."""
    ng = 14
    o = oracle_mod.Oracle(_grid(3, 4, 4, ng, 0.0, 70.0))
    sig = _sigma_table(ng, seed=7)
    o.set_sigma(sig)
    t = o.tables()
    rng = np.random.default_rng(11)
    prev = rng.random(o.comp_shape)
    rho = rng.uniform(0.3, 1.9, size=(3, 4))
    de5 = t["de"][:, None, None, None, None]
    src = o.source(rho, prev)
    injected = (src * de5).sum(axis=(0, 1, 2)) * o.du * o.dv
    removed = rho * (sig[:, None, None, None, None] * prev[:, 0] * de5).sum(axis=(0, 1, 2)) * o.du * o.dv
    assert np.allclose(injected, removed, rtol=1e-12)
    wrong = (_destination_sigma_source(o, rho, prev, sig) * de5).sum(axis=(0, 1, 2)) * o.du * o.dv
    assert np.min(np.abs(wrong / removed - 1.0)) > 0.05


@pytest.mark.parametrize("seed", [2, 3])
def test_particle_count_balance_with_group_dependent_removal(oracle_mod, seed):
    """One CN energy step of one lane with stopping power and a varying
    sigma_g: the particle count sum_g dE psi^1 changes only by the outflow
    through the lowest face and by removal at each group's own rate,
    N1 - N0 = -h/2 [rho S_1/2 ((psi^1 - psi^2)_0 old + new)
                    + rho sum_g sigma_g dE_g (psi^1_g old + new)],
    exact up to rounding."""
    G = 16
    o = oracle_mod.Oracle(dict(ny=1, nz=1, nu=1, nv=1, dy=0.1, dz=0.1, u_max=0.1, v_max=0.1,
                               e_faces=np.linspace(0.0, 40.0, G + 1)))
    sig = _sigma_table(G, seed=seed)
    o.set_sigma(sig)
    t = o.tables()
    rng = np.random.default_rng(seed)
    x0 = rng.random((G, 2))
    rho, h = 1.3, 0.4
    x1, _, _ = o.energy_cn_lane(rho, h, x0)
    x1 = x1.reshape(G, 2)
    n0 = np.sum(t["de"] * x0[:, 0])
    n1 = np.sum(t["de"] * x1[:, 0])
    out = rho * t["s_face"][0] * ((x0[0, 0] - x0[0, 1]) + (x1[0, 0] - x1[0, 1]))
    rem = rho * np.sum(sig * t["de"] * (x0[:, 0] + x1[:, 0]))
    assert n1 - n0 == pytest.approx(-0.5 * h * (out + rem), rel=1e-12)


def test_march_conserves_protons_across_components(oracle_mod):
    """A K = 1 march with transport and scattering off, a varying sigma_g and
    a catastrophic scatter that keeps energy and direction (P^1, P^2 ->
    delta): what psi_p loses by removal psi_s1 gains, so the count of
    psi_p + psi_s1 equals the count of the march without removal up to the
    protons psi_s1 itself loses again, a second-order remainder bounded by
    3 (sigma_max x)^2."""
    ng = 20
    g = dict(ny=1, nz=1, nu=2, nv=2, dy=0.1, dz=0.1, u_max=0.1, v_max=0.1,
             e_faces=np.linspace(0.0, 60.0, ng + 1))
    sig = _sigma_table(ng, seed=5) * 0.3
    phys = dict(lambda_p1=1e4, g_alpha=1.0, g_beta=1e5)
    o = oracle_mod.Oracle(g, phys)
    o.set_sigma(sig)
    o0 = oracle_mod.Oracle(g, dict(phys, sigma_ct=0.0))
    n, dx = 10, 0.05
    beam = dict(e0=45.0, sigma_y=0.2, sigma_z=0.2)
    rho = np.ones((n, 1, 1))
    r1 = o.march(rho, n, dx, beam=beam, n_scatter=1, do_transport=False, do_angular=False)
    r0 = o0.march(rho, n, dx, beam=beam, do_transport=False, do_angular=False)
    de = np.diff(o.e_faces)[:, None, None, None, None]
    count = lambda p: float((p[:, 0] * de).sum())
    tot = count(r1["psi"][0]) + count(r1["psi"][1])
    ref = count(r0["psi"][0])
    sx = sig.max() * n * dx
    assert abs(tot - ref) / ref < 3.0 * sx ** 2
    # and the primary alone lost about sigma x of its protons (the energy-
    # weighted sigma of the groups the beam crossed)
    assert count(r1["psi"][0]) < ref
