"""Pins of the oracle's beam projection (Section 4, Eq. bdy; DG projection of
Section 3.2) against moments of the Gaussian."""
import numpy as np
import pytest


def test_beam_projection_moments(oracle_mod):
    grid = dict(ny=80, nz=80, nu=4, nv=4, dy=0.05, dz=0.05, u_max=0.1, v_max=0.1,
                e_faces=np.linspace(80.0, 120.0, 21))
    o = oracle_mod.Oracle(grid)
    t = o.tables()
    beam = dict(e0=101.3, sigma_e=2.0, y0=0.1, z0=-0.05, sigma_y=0.3, sigma_z=0.25)
    psi = o.init_beam(beam)
    de, ec = t["de"], t["e_c"]
    w = o.du * o.dv * o.dy * o.dz
    n = (psi[:, 0].sum(axis=(1, 2, 3, 4)) * de).sum() * w
    assert n == pytest.approx(1.0, rel=1e-13)
    # DG content int E psi dE is the Gaussian's mean energy (the tails beyond
    # the grid are below 1e-20 here)
    e_content = ((ec * de * psi[:, 0].sum(axis=(1, 2, 3, 4))) + de ** 2 / 6 * psi[:, 1].sum(axis=(1, 2, 3, 4))).sum() * w
    assert e_content == pytest.approx(101.3, rel=1e-12)
    # lateral cell averages: mean y0 and variance sigma^2 + dy^2/12 (Sheppard)
    f = psi[0, 0].sum(axis=(0, 1))
    y = (np.arange(80) + 0.5 - 40) * 0.05
    wy = f.sum(axis=1)
    my = (wy * y).sum() / wy.sum()
    assert my == pytest.approx(0.1, abs=1e-9)
    vy = (wy * (y - my) ** 2).sum() / wy.sum()
    assert vy == pytest.approx(0.09 + 0.05 ** 2 / 12, rel=1e-6)
    # sub-grid angular width: the even grid has no node at 0, the beam is
    # split evenly over the four central nodes
    a = psi[10, 0, :, :, 40, 40]
    assert np.count_nonzero(a > 1e-300) == 4
    assert a[1, 1] == a[2, 2] == a[1, 2] == a[2, 1]
