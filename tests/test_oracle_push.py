"""Pins of the oracle's particle push, field models and effective field.

Closed forms: the Boris rotation in a pure B field (|u| conserved, angle
2 atan(|B| dt / 2 gamma) per step), the exact linear growth in a pure E field,
H_eff of a particle in a pure B field and in a counter-propagating circularly
polarised wave, the chord identity of Eq. (9) on a Boris step, the plane
wave's Poynting direction, and the quadratic-spline gather reproducing
constant and linear fields exactly on every staggered component.
"""
import math

import numpy as np
import pytest

import oracle as O
from paper_1409_5574_gb300 import workloads as W


def _rot(v, axis, ang):
    axis = axis / np.linalg.norm(axis)
    c, s = math.cos(ang), math.sin(ang)
    return v * c + np.cross(axis, v) * s + axis * np.dot(axis, v) * (1 - c)


def test_boris_pure_B_closed_form_rotation():
    B = np.array([0.3, -0.2, 1.7])
    u0 = np.array([120.0, -35.0, 80.0])
    q, dtn = -1.0, 0.37
    g = math.sqrt(1 + u0 @ u0)
    theta = 2 * math.atan(q * np.linalg.norm(B) * dtn / (2 * g))
    u = u0.copy()
    for n in range(1, 1001):
        u = O.boris(u, np.zeros(3), B, q, dtn)
        if n in (1, 10, 1000):
            # du/dt = q u x B / gamma rotates u about B by -q|B|t/gamma
            ref = _rot(u0, B, -theta * n)
            assert np.allclose(u, ref, rtol=0, atol=1e-10 * np.linalg.norm(u0) * n)
    assert abs(np.linalg.norm(u) / np.linalg.norm(u0) - 1) < 1e-13


def test_boris_pure_E_linear():
    E = np.array([0.5, -1.5, 2.0])
    u = np.array([3.0, 4.0, -1.0])
    q, dtn = -1.0, 0.05
    u0 = u.copy()
    for _ in range(400):
        u = O.boris(u, E, np.zeros(3), q, dtn)
    assert np.allclose(u, u0 + q * E * dtn * 400, rtol=1e-13, atol=1e-12)


def test_heff_field_form_pure_B_and_E():
    B = np.array([0.0, 0.0, 2.5])
    for pitch in (0.1, 0.7, math.pi / 2):
        beta = 0.999 * np.array([math.sin(pitch), 0.0, math.cos(pitch)])
        assert O.heff_field(np.zeros(3), B, beta) == pytest.approx(
            2.5 * 0.999 * math.sin(pitch), rel=1e-14)
    # pure E: H^2 = E^2 - (E.beta)^2 = E_perp^2 + E_par^2 / gamma^2
    E = np.array([1.0, 2.0, 0.0])
    beta = np.array([0.6, 0.0, 0.0])
    g2 = 1 / (1 - 0.36)
    assert O.heff_field(E, np.zeros(3), beta) == pytest.approx(
        math.sqrt(4.0 + 1.0 / g2), rel=1e-14)


def test_heff_counter_propagating_cp_wave():
    """A particle moving along -x against the +x CP wave sees H = (1+beta)E0."""
    wl = W.plane_wave(a0=300.0, n=4)
    p = O.Problem(**wl.problem_kwargs())
    gamma = 1000.0
    beta = -math.sqrt(1 - 1 / gamma ** 2)
    for x in (0.0, 1.3, 4.0):
        for step in (0, 17):
            E, B = O.fields(p, x, 0.0, 0.0, step)
            h = O.heff_field(E, B, np.array([beta, 0.0, 0.0]))
            assert h == pytest.approx((1 - beta) * 300.0, rel=1e-12)


def test_plane_wave_is_a_cp_vacuum_wave():
    wl = W.plane_wave(a0=50.0, n=4)
    for d in (1, -1):
        p = O.Problem(**{**wl.problem_kwargs(), "direction": d})
        E, B = O.fields(p, 0.7, 0.0, 0.0, 3)
        assert np.linalg.norm(E) == pytest.approx(50.0, rel=1e-13)
        assert np.linalg.norm(B) == pytest.approx(50.0, rel=1e-13)
        assert abs(E @ B) < 1e-10
        S = np.cross(E, B)
        assert S[0] * d > 0 and abs(S[1]) < 1e-9 and abs(S[2]) < 1e-9
        # phase: moving along +dir x at c with t keeps the field fixed
        dtn = wl.dt * wl.omega_ref
        E2, _ = O.fields(p, 0.7 + d * 5 * dtn, 0.0, 0.0, 8)
        assert np.allclose(E, E2, atol=1e-9)


def test_heff_momentum_form_chord_identity():
    """Eq. (9) on a Boris step in a pure perpendicular B returns |B| exactly
    (|dp| / |p_avg| = 2 tan(theta/2) = |B| dt / gamma)."""
    B = np.array([0.0, 0.0, 3.2])
    for umag, dtn in ((5.0, 0.2), (800.0, 0.05), (3000.0, 1.3)):
        u0 = np.array([umag * 0.6, umag * 0.8, 0.0])
        u1 = O.boris(u0, np.zeros(3), B, -1.0, dtn)
        assert O.heff_momentum(u0, u1, dtn) == pytest.approx(3.2, rel=1e-12)


def test_heff_forms_agree_in_a_wave():
    """Field form and Eq. (9) differ by O(1/gamma^2, dt^2) only."""
    wl = W.plane_wave(a0=100.0, n=4, steps_per_period=2000)
    p = O.Problem(**wl.problem_kwargs())
    dtn = wl.dt * wl.omega_ref
    u0 = np.array([-999.0, 10.0, -3.0])
    E, B = O.fields(p, 0.4, 0.0, 0.0, 5)
    u1 = O.boris(u0, E, B, -1.0, dtn)
    ua = 0.5 * (u0 + u1)
    beta = ua / math.sqrt(1 + ua @ ua)
    hf = O.heff_field(E, B, beta)
    hm = O.heff_momentum(u0, u1, dtn)
    assert hm == pytest.approx(hf, rel=1e-4)


def _yee_problem(planes, dxn=0.3, dyn=0.45, x0=-1.0, y0=2.0):
    return O.Problem(omega_ref=1.0, dt=0.1, field_kind=O.FIELD_YEE2D, dims=2,
                     yee=planes, dx=dxn, dy=dyn, x0=x0, y0=y0)


def test_yee_gather_constant_and_linear_fields_exact():
    """Quadratic-spline gather reproduces linear fields on every staggered
    component (this pins the stagger offsets and the weights)."""
    nx, ny, dxn, dyn, x0, y0 = 40, 36, 0.3, 0.45, -1.0, 2.0
    sx = [0.5, 0.0, 0.0, 0.0, 0.5, 0.5]
    sy = [0.0, 0.5, 0.0, 0.5, 0.0, 0.5]
    coef = [(1.0, 0.5, -0.25), (2.0, -1.0, 0.3), (-3.0, 0.2, 0.1),
            (0.5, 0.0, 1.0), (1.5, 1.0, 0.0), (0.0, -0.7, -0.6)]
    planes = []
    for c in range(6):
        xs = x0 + (np.arange(nx) + sx[c]) * dxn
        ys = y0 + (np.arange(ny) + sy[c]) * dyn
        a, bx, by = coef[c]
        planes.append((a + bx * xs[None, :] + by * ys[:, None]).astype(np.float64))
    p = _yee_problem([pl.astype(np.float32) for pl in planes], dxn, dyn, x0, y0)
    rng = np.random.default_rng(5)
    for _ in range(50):
        px = x0 + rng.uniform(3, nx - 3) * dxn
        py = y0 + rng.uniform(3, ny - 3) * dyn
        E, B = O.fields(p, px, py, 0.0, 0)
        got = np.concatenate([E, B])
        for c in range(6):
            a, bx, by = coef[c]
            # float32 storage of the planes bounds the agreement
            assert got[c] == pytest.approx(a + bx * px + by * py, abs=2e-5)
    # constant fields, including across the periodic edge
    const = [np.full((ny, nx), v, dtype=np.float32) for v in (1, 2, 3, 4, 5, 6)]
    p = _yee_problem(const, dxn, dyn, x0, y0)
    for px, py in ((x0, y0), (x0 + nx * dxn - 1e-9, y0 + 0.1), (x0 + 5.0, y0 + 7.3)):
        E, B = O.fields(p, px, py, 0.0, 0)
        assert np.allclose(np.concatenate([E, B]), [1, 2, 3, 4, 5, 6], rtol=1e-12)


def test_yee_gather_single_node_weights():
    """A unit value on one Ez node is seen with the quadratic-spline weights
    1/2 (1/2 -+ d)^2 and 3/4 - d^2 in each direction."""
    nx = ny = 16
    planes = [np.zeros((ny, nx), dtype=np.float32) for _ in range(6)]
    planes[2][7, 5] = 1.0          # Ez node (i=5, j=7), unstaggered
    p = _yee_problem(planes, 1.0, 1.0, 0.0, 0.0)
    for px, py in ((5.2, 7.0), (4.7, 6.6), (5.5 - 1e-9, 7.4)):
        E, _ = O.fields(p, px, py, 0.0, 0)
        def w1(d):
            return 0.75 - d * d if abs(d) <= 0.5 else 0.5 * (1.5 - abs(d)) ** 2
        assert E[2] == pytest.approx(w1(px - 5) * w1(py - 7), rel=1e-12)
