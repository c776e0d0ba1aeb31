"""The angular-distribution diagnostic of the oracle (Fig. 4: emitted energy
by direction around the laser axis) against what geometry fixes: a direction
built at known (theta, phi) lands in its bin, energy along the axis sits in
the first polar bin, an isotropic set fills the bins in proportion to their
solid angle, and nothing beyond theta_max is counted."""
import math

import numpy as np
import pytest

import oracle as O


def _dirs(theta, phi, axis, ref):
    a = np.asarray(axis, float) / np.linalg.norm(axis)
    r = np.asarray(ref, float)
    e1 = r - (r @ a) * a
    e1 /= np.linalg.norm(e1)
    e2 = np.cross(a, e1)
    st = np.sin(theta)[:, None]
    return (st * np.cos(phi)[:, None] * e1 + st * np.sin(phi)[:, None] * e2
            + np.cos(theta)[:, None] * a)


@pytest.mark.parametrize("axis,ref", [((1, 0, 0), (0, 1, 0)), ((0.3, -1, 2), (1, 1, 0))])
def test_known_direction_lands_in_its_bin(axis, ref):
    rng = np.random.default_rng(1)
    nt, nph, tmax = 18, 24, math.pi / 2
    it = rng.integers(0, nt, 200)
    ip = rng.integers(0, nph, 200)
    th = (it + rng.uniform(0.05, 0.95, 200)) * tmax / nt
    ph = (ip + rng.uniform(0.05, 0.95, 200)) * 2 * math.pi / nph
    n = _dirs(th, ph, axis, ref)
    e = rng.uniform(0.5, 2.0, 200)
    h = O.angular_histogram(n[:, 0], n[:, 1], n[:, 2], e, np.ones(200), axis, ref, nt, nph,
                            tmax)
    ref_h = np.zeros((nt, nph))
    np.add.at(ref_h, (it, ip), e)
    np.testing.assert_allclose(h, ref_h, rtol=1e-12, atol=1e-12)


def test_axis_direction_and_hemisphere_cut():
    n = np.array([[1.0, 0, 0], [-1.0, 0, 0], [0, 0.6, -0.8]])
    h = O.angular_histogram(n[:, 0], n[:, 1], n[:, 2], np.array([2.0, 5.0, 7.0]),
                            np.array([1.5, 1.0, 1.0]), (1, 0, 0), (0, 1, 0), 10, 8,
                            math.pi / 2)
    assert h[0].sum() == pytest.approx(3.0)        # along the axis: first polar bin
    assert h.sum() == pytest.approx(3.0 + 7.0)     # the backward record is cut
    assert h[9].sum() == pytest.approx(7.0)        # theta = pi/2: last bin


def test_isotropic_directions_fill_solid_angle():
    rng = np.random.default_rng(2)
    m = 400_000
    v = rng.normal(size=(m, 3))
    v /= np.linalg.norm(v, axis=1)[:, None]
    nt, nph = 12, 16
    h = O.angular_histogram(v[:, 0], v[:, 1], v[:, 2], np.ones(m), np.ones(m), (0, 0, 1),
                            (1, 0, 0), nt, nph, math.pi)
    edges = np.linspace(0, math.pi, nt + 1)
    expect = m * (np.cos(edges[:-1]) - np.cos(edges[1:]))[:, None] / 2 / nph * np.ones(nph)
    z = (h - expect) / np.sqrt(expect)
    assert np.abs(z).max() < 5 and abs(h.sum() - m) < 1e-6
