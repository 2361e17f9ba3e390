"""Pins of the FP64 oracle to things other than itself: closed forms, hand-reduced special cases
of the paper's equations, invariants, brute force and finite differences.

Each pin is chosen so that a plausible mistake in the oracle (a dropped term, a wrong sign, a
transposed operand, a wrong index) changes the checked value.
"""
import json
import os

import numpy as np
import pytest

import worlds as Wd
from paper_2603_12185_gb300 import scenes as S

G = 9.81
DT = 0.002
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ------------------------------------------------------------------------------------------
# Eq. r_scaling: the MuJoCo solimp gap scaling
# ------------------------------------------------------------------------------------------
def test_solimp_r_table(oracle):
    """Values worked by hand from Eq. r_scaling with (0.9, 0.95, 0.001, 0.5, 2) -- see
    tests/golden/solimp_r.json for the arithmetic."""
    g = json.load(open(os.path.join(GOLDEN, "solimp_r.json")))
    for aphi, r in zip(g["abs_phi"], g["r"]):
        assert oracle.solimp_r(aphi, g["solimp"]) == pytest.approx(r, abs=1e-15)


# ------------------------------------------------------------------------------------------
# closed forms without contact
# ------------------------------------------------------------------------------------------
def test_free_flight_projectile(oracle):
    """Semi-implicit Euler under gravity: v_n = v0 + n g dt, x_n = x0 + n dt v0 + g dt^2 n(n+1)/2."""
    d = Wd.sphere_on_plane()
    p = Wd.params()
    x0, v0, w = np.array([0.1, -0.2, 50.0]), np.array([1.0, 2.0, 3.0]), np.array([0.3, -0.2, 0.5])
    q, v = Wd.free_state(x0, lin=v0, ang=w)
    n = 200
    q, v, nc = oracle.step(d, p, DT, n, q, v)
    g = np.array([0, 0, -G])
    assert nc == 0
    np.testing.assert_allclose(v[:3], v0 + n * g * DT, rtol=0, atol=1e-12)
    np.testing.assert_allclose(q[:3], x0 + n * DT * v0 + g * DT * DT * n * (n + 1) / 2, rtol=0, atol=1e-11)
    np.testing.assert_allclose(v[3:], w, atol=1e-14)  # isotropic body: no gyroscopic torque


def test_isotropic_spin_is_exact(oracle):
    """Torque-free isotropic body: body-frame omega is constant and the exponential-map update
    composes to q_n = q0 (x) (cos(n|w|dt/2), sin(n|w|dt/2) w/|w|)."""
    d = Wd.sphere_on_plane()
    p = Wd.params(gravity=(0.0, 0.0, 0.0))
    q0 = S.quat_about((1, 2, 3), 0.7)
    w = np.array([2.0, -1.0, 0.5])
    q, v = Wd.free_state((0, 0, 10.0), quat=q0, ang=w)
    n = 500
    q, v, _ = oracle.step(d, p, DT, n, q, v)
    ang = np.linalg.norm(w) * n * DT
    dq = np.concatenate([[np.cos(ang / 2)], np.sin(ang / 2) * w / np.linalg.norm(w)])
    a, b = q0, dq
    expect = np.array([a[0] * b[0] - a[1] * b[1] - a[2] * b[2] - a[3] * b[3],
                       a[0] * b[1] + a[1] * b[0] + a[2] * b[3] - a[3] * b[2],
                       a[0] * b[2] - a[1] * b[3] + a[2] * b[0] + a[3] * b[1],
                       a[0] * b[3] + a[1] * b[2] - a[2] * b[1] + a[3] * b[0]])
    np.testing.assert_allclose(q[3:], expect, atol=1e-12)


def test_torque_free_asymmetric_body_conserves_world_angular_momentum(oracle):
    """The gyroscopic bias w x I w (sign and frame) keeps the world-frame angular momentum
    R I w fixed up to the O(dt) error of explicit integration; a flipped sign or a world-frame
    inertia drifts it at O(1)."""
    inertia = np.array([1e-3, 2e-3, 3.5e-3])
    d = Wd.world([dict(mass=1.0, inertia=inertia)], [dict(type=S.SPHERE, body=0, size=(0.05, 0, 0))])
    p = Wd.params(gravity=(0.0, 0.0, 0.0))
    q, v = Wd.free_state((0, 0, 0), quat=S.quat_about((0.3, 1, 0.2), 0.4), ang=(0.4, 3.0, 0.2))

    def Lworld(q, v):
        _, _, poses = oracle.dynamics(d, (0, 0, 0), q, v)
        R = poses[0, 3:12].reshape(3, 3)
        return R @ (inertia * v[3:])

    L0 = Lworld(q, v)
    q1, v1, _ = oracle.step(d, p, 1e-4, 5000, q, v)
    assert np.linalg.norm(Lworld(q1, v1) - L0) < 2e-3 * np.linalg.norm(L0)


# ------------------------------------------------------------------------------------------
# the worked single-contact step: the general dense-Jacobian path must reduce to scalar
# arithmetic of Eqs. smooth_vel, tilde_defs, cf_wrench, k_d_setting, r_scaling, vel_correction
# ------------------------------------------------------------------------------------------
def _sphere_plane_by_hand(v0x):
    """Sphere r=0.05, m=1, I=1e-3 on the plane z=0 (t1=x, t2=y), centre height 0.048 (phi=-2 mm),
    linear velocity (v0x, 0, 0), 4 facets {+t1,+t2,-t1,-t2}, mu=0.5, k=0.1, d=0.001, dt=2 ms."""
    r, m, I, mu, k, dd, phi = 0.05, 1.0, 1e-3, 0.5, 0.1, 0.001, -0.002
    vz = -G * DT                             # Eq. smooth_vel: contact-free velocity
    lever = np.array([0.0, 0.0, -(r + phi / 2)])  # midpoint of surface points minus the centre
    rr = 0.95                                # |phi|/w = 2 -> clamped to 1 -> r_max
    trace = 3 / m + (lever @ lever) * 3 / I - (lever @ lever) / I   # 3/m + |l|^2 tr(I^-1) - l^T I^-1 l
    Mphi = rr / (1 - rr) / trace
    d_dirs = [(1, 0), (0, 1), (-1, 0), (0, -1)]
    lam = []
    for dx, dy in d_dirs:
        s = vz - mu * (dx * v0x + dy * 0.0)  # J~ v_s = J_n v - mu d^T J_t v
        lam.append(max(0.0, -k * Mphi * (s * DT + phi) - dd * Mphi * s))
    f = np.array([-mu * sum(l * dx for l, (dx, dy) in zip(lam, d_dirs)),
                  -mu * sum(l * dy for l, (dx, dy) in zip(lam, d_dirs)), sum(lam)])
    torque = np.cross(lever, f)
    v = np.array([v0x, 0, vz]) + f / m
    w = torque / I
    return Mphi, lam, v, w


@pytest.mark.parametrize("v0x", [0.0, 0.1])
def test_worked_single_contact_step(oracle, v0x):
    d = Wd.sphere_on_plane()
    p = Wd.params(n_t=4)
    q, v = Wd.free_state((0, 0, 0.048), lin=(v0x, 0, 0))
    rec = oracle.step_record(d, p, DT, q, v)
    Mphi, lam, v_exp, w_exp = _sphere_plane_by_hand(v0x)
    assert len(rec["contacts"]) == 1
    c = rec["contacts"][0]
    assert c["phi"] == pytest.approx(-0.002, abs=1e-15)
    np.testing.assert_allclose(c["pos"], [0, 0, -0.001], atol=1e-15)
    assert c["mphi"] == pytest.approx(Mphi, rel=1e-12)
    assert c["lam_sum"] == pytest.approx(sum(lam), rel=1e-12)
    np.testing.assert_allclose(rec["v"][:3], v_exp, rtol=1e-12, atol=1e-15)
    np.testing.assert_allclose(rec["v"][3:], w_exp, rtol=1e-12, atol=1e-15)
    np.testing.assert_allclose(rec["q"][:3], np.array([0, 0, 0.048]) + DT * v_exp, rtol=1e-12, atol=1e-15)
    # the wrench record: normal impulse and the friction along t1 = x, t2 = y
    dirs = [(1, 0), (0, 1), (-1, 0), (0, -1)]
    f_t = [-0.5 * sum(l * dx for l, (dx, dy) in zip(lam, dirs)), -0.5 * sum(l * dy for l, (dx, dy) in zip(lam, dirs))]
    np.testing.assert_allclose(c["wrench"][:3], [sum(lam)] + f_t, rtol=1e-12, atol=1e-18)
    assert (c["wrench"][1] < 0.0) == (v0x > 0.0)          # friction opposes the slide
    if v0x == 0.0:
        assert sum(lam) == pytest.approx(4 * Mphi * 0.000223544, rel=1e-9)  # printed digits of the hand sum


@pytest.mark.parametrize("mu_sphere,mu_plane", [(0.2, 0.5), (0.5, 0.2)])
def test_pair_friction_is_the_larger_coefficient(oracle, mu_sphere, mu_plane):
    """A contact takes the larger of its two geoms' friction coefficients, whichever geom holds
    it: the sliding worked step with mu 0.5 on one geom and 0.2 on the other matches the by-hand
    step at mu = 0.5 (at 0.2 every facet impulse and the friction change)."""
    d = Wd.world([dict(mass=1.0, inertia=(1e-3,) * 3)],
                 [dict(type=S.PLANE, body=-1, mu=(mu_plane, 0, 0)),
                  dict(type=S.SPHERE, body=0, size=(0.05, 0, 0), mu=(mu_sphere, 0, 0))])
    q, v = Wd.free_state((0, 0, 0.048), lin=(0.1, 0, 0))
    rec = oracle.step_record(d, Wd.params(n_t=4), DT, q, v)
    Mphi, lam, v_exp, w_exp = _sphere_plane_by_hand(0.1)
    assert rec["contacts"][0]["lam_sum"] == pytest.approx(sum(lam), rel=1e-12)
    np.testing.assert_allclose(rec["v"], np.concatenate([v_exp, w_exp]), rtol=1e-12, atol=1e-15)


def test_hinge_link_contact_by_hand(oracle):
    """A hinged link pressed into the floor, by hand.  The hinge sits at a = (0, 0, 0.1); its body
    frame is the world frame turned 90 degrees about z, and its axis is body x, so the world axis
    is e_y.  A capsule (r = 1 cm) runs 10 cm from the hinge along body -y: at angle q the link
    points along (cos q, 0, -sin q) (a turn by q about +y), and at sin q = 0.92 its tip sphere
    is 2 mm into the floor.  The centre of mass is on the axis, so gravity exerts no torque and
    M = I_x.  The contact row of the hinge rate is e_y x l with l the lever from the hinge to the
    contact midpoint; its trace is |e_y x l|^2 / M.  Four facets {+-x, +-y} with mu = 0.5 take
    the impulse law of Eq. cf_wrench, and v+ = v + sum_j J~_j lambda_j / M."""
    I = (2e-4, 3e-4, 4e-4)
    rz = (np.cos(np.pi / 4), 0.0, 0.0, np.sin(np.pi / 4))      # body frame: 90 degrees about z
    rx = (np.cos(np.pi / 4), np.sin(np.pi / 4), 0.0, 0.0)      # capsule axis z -> body -y
    d = Wd.world([dict(parent=-1, jnt=S.HINGE, pos=(0, 0, 0.1), quat=rz, axis=(1, 0, 0), mass=0.5, inertia=I)],
                 [dict(type=S.PLANE, body=-1),
                  dict(type=S.CAPSULE, body=0, pos=(0, -0.05, 0), quat=rx, size=(0.01, 0.05, 0))])
    q0, v0 = np.arcsin(0.92), 1.5
    rec = oracle.step_record(d, Wd.params(n_t=4), DT, [q0], [v0])
    assert len(rec["contacts"]) == 1
    c = rec["contacts"][0]
    tip = np.array([0.1 * np.cos(q0), 0.0, 0.1 - 0.1 * np.sin(q0)])
    assert c["phi"] == pytest.approx(tip[2] - 0.01, abs=1e-15)
    p = np.array([tip[0], 0.0, (tip[2] - 0.01) / 2])          # midpoint of the two surface points
    np.testing.assert_allclose(c["pos"], p, atol=1e-15)
    lever = p - np.array([0, 0, 0.1])
    Jl = np.cross([0.0, 1.0, 0.0], lever)                      # point velocity per unit hinge rate
    M = I[0]
    trace = Jl @ Jl / M
    assert c["trace_a"] == pytest.approx(trace, rel=1e-12) and c["trace_b"] == 0.0
    Mphi = 0.95 / 0.05 / trace
    assert c["mphi"] == pytest.approx(Mphi, rel=1e-12)
    pgen, lam_sum = 0.0, 0.0
    for dx, dy in [(1, 0), (0, 1), (-1, 0), (0, -1)]:
        row = Jl[2] - 0.5 * (dx * Jl[0] + dy * Jl[1])          # J~ = J_n - mu d^T J_t
        s_j = row * v0
        lam = max(0.0, -0.1 * Mphi * (s_j * DT + c["phi"]) - 0.001 * Mphi * s_j)
        pgen += row * lam
        lam_sum += lam
    assert c["lam_sum"] == pytest.approx(lam_sum, rel=1e-12)
    assert rec["v"][0] == pytest.approx(v0 + pgen / M, rel=1e-12)
    assert rec["q"][0] == pytest.approx(q0 + DT * rec["v"][0], rel=1e-14)
    assert rec["v"][0] < v0                                    # the floor slows the link


# ------------------------------------------------------------------------------------------
# the 6D cone's torsional and rolling rows (Sec. III-A, Eqs. primal_cone, dual_cone,
# dual_polyhedral, tilde_defs), by hand on a sphere 2 mm into the plane z = 0 with the C2
# cone (8 tangential, 2 torsional, 8 rolling facets; mu = 0.8, 0.005, 0.005)
# ------------------------------------------------------------------------------------------
MU6 = (0.8, 0.005, 0.005)
LEVER = 0.049                            # centre to the contact midpoint (r + phi/2)


def _lam_6d(s):
    """Facet impulse of Eq. cf_wrench at the worked contact: lambda dt = (-k M (s dt + phi) - d M s)+
    with M(phi) = r_max/(1 - r_max) / trace, trace = 3/m + 2 l^2 / I (unit mass, I = 1e-3)."""
    trace = 3.0 + 2.0 * LEVER ** 2 / 1e-3
    M = 19.0 / trace
    return max(0.0, -0.1 * M * (s * DT - 0.002) - 0.001 * M * s)


@pytest.mark.parametrize("omega", [20.0, 60.0])
def test_torsional_facets_by_hand(oracle, omega):
    """A sphere spinning at omega about the normal: J_tor v = n . omega = omega while the contact
    point does not slide (omega is parallel to the lever) and no rolling row sees the spin.  The
    two torsional facets J~ = J_n -+ mu_tor J_tor have s = v_n -+ mu_tor omega; the other 16
    facets have s = v_n.  The wrench's torsion -mu_tor (lambda_+ - lambda_-) is the only angular
    impulse, so omega+ = omega + torsion / I.  At 60 rad/s the retarding facet is inactive.
    A linear row in place of J_tor (s = v_n (1 -+ mu_tor)), a dropped mu_tor or a flipped sign
    each change v+ or omega+ far beyond the tolerance."""
    d = Wd.sphere_on_plane(mu=MU6)
    q, v = Wd.free_state((0, 0, 0.048), ang=(0, 0, omega))
    rec = oracle.step_record(d, Wd.params(n_t=8, n_tor=2, n_rol=8), DT, q, v)
    vz = -G * DT
    lp, lm = _lam_6d(vz - MU6[1] * omega), _lam_6d(vz + MU6[1] * omega)
    N = 16 * _lam_6d(vz) + lp + lm
    torsion = -MU6[1] * (lp - lm)
    c = rec["contacts"][0]
    assert len(rec["contacts"]) == 1 and c["nfacet"] == 18
    assert c["nactive"] == (18 if lm > 0 else 17)
    assert (lm > 0) == (omega == 20.0)
    assert c["wrench"][0] == pytest.approx(N, rel=1e-12)
    assert c["wrench"][3] == pytest.approx(torsion, rel=1e-12)
    np.testing.assert_allclose(c["wrench"][[1, 2, 4, 5]], 0.0, atol=1e-18)
    np.testing.assert_allclose(rec["v"][:3], [0.0, 0.0, vz + N], rtol=1e-12, atol=1e-15)
    np.testing.assert_allclose(rec["v"][3:], [0.0, 0.0, omega + torsion / 1e-3], rtol=1e-12, atol=1e-15)


@pytest.mark.parametrize("omega_y", [10.0, 40.0])
def test_rolling_facets_by_hand(oracle, omega_y):
    """A sphere rolling without slip along +x: omega = (0, w, 0) and v_x = l w, so the contact
    point is at rest (every tangential facet has s = v_n) and J_tor v = 0, while the rolling rows
    see (t1 . omega, t2 . omega) = (0, w).  Rolling facet j (direction (cos, sin)(2 pi j / 8))
    has s_j = v_n - mu_rol sin_j w.  The rolling moment (R1, R2) = -mu_rol sum_j (cos_j, sin_j)
    lambda_j is the only angular impulse (the normal force passes through the centre), so
    omega+ = (R1, w + R2, 0) / I.  Rows built from the linear point velocity (zero here) would
    leave omega unchanged; a dropped mu_rol or sign flips R2."""
    d = Wd.sphere_on_plane(mu=MU6)
    q, v = Wd.free_state((0, 0, 0.048), lin=(LEVER * omega_y, 0, 0), ang=(0, omega_y, 0))
    rec = oracle.step_record(d, Wd.params(n_t=8, n_tor=2, n_rol=8), DT, q, v)
    vz = -G * DT
    th = 2 * np.pi * np.arange(8) / 8
    lam_r = np.array([_lam_6d(vz - MU6[2] * np.sin(t) * omega_y) for t in th])
    N = 10 * _lam_6d(vz) + lam_r.sum()
    R1 = -MU6[2] * np.sum(np.cos(th) * lam_r)
    R2 = -MU6[2] * np.sum(np.sin(th) * lam_r)
    assert R2 < 0.0                       # resists the rolling
    assert (lam_r.min() > 0) == (omega_y == 10.0)
    c = rec["contacts"][0]
    assert c["wrench"][0] == pytest.approx(N, rel=1e-12)
    assert c["wrench"][5] == pytest.approx(R2, rel=1e-12)
    assert abs(c["wrench"][4] - R1) < 1e-15 * N
    np.testing.assert_allclose(rec["v"][:3], [LEVER * omega_y, 0.0, vz + N], rtol=1e-12, atol=1e-15)
    np.testing.assert_allclose(rec["v"][3:], [R1 / 1e-3, omega_y + R2 / 1e-3, 0.0], rtol=1e-12, atol=1e-12)


# ------------------------------------------------------------------------------------------
# the tangent frame of non-plane contacts (the paper fixes none): t1 = normalize(e_z x n) when
# |n_z| < 0.5, else normalize(e_x x n); t2 = n x t1
# ------------------------------------------------------------------------------------------
def _two_spheres(n, u=(0.0, 0.0, 0.0), overlap=0.002):
    """Sphere A (geom 0, 1 kg, I 1e-3) touching sphere B (geom 1, 2 kg, I 3e-3) along unit n
    from B to A, both r = 0.05, A moving at u; no gravity."""
    n = np.asarray(n, float)
    d = Wd.world([dict(mass=1.0, inertia=(1e-3,) * 3), dict(mass=2.0, inertia=(3e-3,) * 3)],
                 [dict(type=S.SPHERE, body=0, size=(0.05, 0, 0), mu=(0.5, 0, 0)),
                  dict(type=S.SPHERE, body=1, size=(0.05, 0, 0), mu=(0.5, 0, 0))])
    qa, va = Wd.free_state(tuple((0.1 - overlap) * n + np.array([0, 0, 1.0])), lin=tuple(u))
    qb, vb = Wd.free_state((0, 0, 1.0))
    return d, np.concatenate([qa, qb]), np.concatenate([va, vb])


# (n, expected t1): the four cases worked by hand from the rule
FRAMES = [
    ((1.0, 0.0, 0.0), (0.0, 1.0, 0.0)),                                   # e_z x e_x = e_y
    ((0.0, 0.0, 1.0), (0.0, -1.0, 0.0)),                                  # e_x x e_z = -e_y
    ((0.8, 0.36, 0.48), (-0.36 / np.hypot(0.36, 0.8), 0.8 / np.hypot(0.36, 0.8), 0.0)),   # |n_z| < 0.5
    ((0.48, 0.36, 0.8), (0.0, -0.8 / np.hypot(0.8, 0.36), 0.36 / np.hypot(0.8, 0.36))),   # |n_z| >= 0.5
]


@pytest.mark.parametrize("n,t1", FRAMES)
def test_tangent_frame_rule(oracle, n, t1):
    d, q, v = _two_spheres(n)
    rec = oracle.step_record(d, Wd.params(n_t=4, gravity=(0.0, 0.0, 0.0)), DT, q, v)
    c = rec["contacts"][0]
    np.testing.assert_allclose(c["normal"], n, atol=1e-12)
    np.testing.assert_allclose(c["t1"], t1, atol=1e-12)
    np.testing.assert_allclose(c["t2"], np.cross(n, t1), atol=1e-12)


def test_tangent_frame_decides_the_pyramid_friction(oracle):
    """A sliding sphere-sphere contact through the anisotropic 4-facet pyramid, by hand in the
    frame the rule gives for n = (0.48, 0.36, 0.8).  The other branch's frame is turned by 137
    degrees about n (not a symmetry of the pyramid), so taking it changes the friction impulse
    and both bodies' velocities.  At 1 m/s the facet leaning along the slide is inactive
    (with all four active the soft law gives friction exactly against the slide, in any frame),
    so the friction is not anti-parallel to the slide."""
    n, t1 = np.array(FRAMES[3][0]), np.array(FRAMES[3][1])
    t2 = np.cross(n, t1)
    slide = 1.0 * (np.cos(0.4) * t1 + np.sin(0.4) * t2)     # tangential, 0.4 rad from t1
    d, q, v = _two_spheres(n, u=slide)
    rec = oracle.step_record(d, Wd.params(n_t=4, gravity=(0.0, 0.0, 0.0)), DT, q, v)
    la, lb = -0.049 * n, 0.049 * n                           # levers to the contact midpoint
    trace = (3.0 + 2 * 0.049 ** 2 / 1e-3) + (1.5 + 2 * 0.049 ** 2 / 3e-3)
    M = 19.0 / trace
    dirs = [(1, 0), (0, 1), (-1, 0), (0, -1)]
    vt = (slide @ t1, slide @ t2)
    lam = [max(0.0, -0.1 * M * (s * DT - 0.002) - 0.001 * M * s)
           for s in (-0.5 * (dc * vt[0] + ds * vt[1]) for dc, ds in dirs)]
    f = sum(lam) * n - 0.5 * sum(l * dc for l, (dc, ds) in zip(lam, dirs)) * t1 \
        - 0.5 * sum(l * ds for l, (dc, ds) in zip(lam, dirs)) * t2
    np.testing.assert_allclose(rec["v"][:3], slide + f, rtol=1e-12, atol=1e-15)
    np.testing.assert_allclose(rec["v"][3:6], np.cross(la, f) / 1e-3, rtol=1e-12, atol=1e-13)
    np.testing.assert_allclose(rec["v"][6:9], -f / 2.0, rtol=1e-12, atol=1e-15)
    np.testing.assert_allclose(rec["v"][9:], -np.cross(lb, f) / 3e-3, rtol=1e-12, atol=1e-13)
    assert min(lam) == 0.0 and max(lam) > 0.0
    assert abs(np.cross(f - (f @ n) * n, slide) @ n) > 1e-2 * np.linalg.norm(f)  # friction not along -slide


# ------------------------------------------------------------------------------------------
# the MPC costs (Sec. V, Eq. mpc) on a hand-built state
# ------------------------------------------------------------------------------------------
class _W:
    w_quat, w_pos, w_contact, w_joint, w_fallen, fall_radius, term_pos, term_quat = 2.0, 3.0, 10.0, 0.05, 5.0, 0.08, 50.0, 20.0


def _cost_world():
    """A free cube (body 0); a one-link finger hinged at (0.1, 0, 0) about y (body 1, capsule
    half length 0.02 at (0, 0, 0.02): a fingertip); a two-link finger hinged at (-0.1, 0, 0)
    about x (body 2 with a capsule: not a tip; its child body 3 at (0, 0, 0.04), capsule half
    length 0.015 at (0, 0, 0.015): a tip)."""
    cap = lambda b, h: dict(type=S.CAPSULE, body=b, pos=(0, 0, h), size=(0.01, h, 0))
    return Wd.world([dict(mass=0.1, inertia=(6e-5,) * 3),
                     dict(parent=-1, jnt=S.HINGE, pos=(0.1, 0, 0), axis=(0, 1, 0)),
                     dict(parent=-1, jnt=S.HINGE, pos=(-0.1, 0, 0), axis=(1, 0, 0)),
                     dict(parent=2, jnt=S.HINGE, pos=(0, 0, 0.04), axis=(1, 0, 0))],
                    [dict(type=S.PLANE, body=-1), dict(type=S.BOX, body=0, size=(0.03,) * 3),
                     cap(1, 0.02), cap(2, 0.02), cap(3, 0.015)])


@pytest.mark.parametrize("fall_radius", [0.08, 0.02])
def test_mpc_cost_by_hand(oracle, fall_radius):
    """Cube at p = (0.01, 0.02, 0.03) turned 0.5 rad about z, target (0, 0, 0.05) turned 1 rad:
    q*^T q = cos 0.25.  Hinges (pi/2, 0, pi/2), home pose 0.1 each.  Tips: finger 1 turned by
    pi/2 about y points along +x, tip (0.14, 0, 0); finger 2's second link turned by pi/2 about
    x points along -y, tip (-0.1, -0.03, 0.04).  The cube is 0.0224 m from the target
    horizontally: fallen only for the 0.02 m radius."""
    d = _cost_world()
    p = np.array([0.01, 0.02, 0.03])
    q = np.concatenate([p, [np.cos(0.25), 0, 0, np.sin(0.25)], [np.pi / 2, 0.0, np.pi / 2]])
    goal = np.array([0.0, 0.0, 0.05, np.cos(0.5), 0, 0, np.sin(0.5)])
    qref = np.concatenate([np.zeros(7), [0.1, 0.1, 0.1]])
    w = _W()
    w.fall_radius = fall_radius
    run, term = oracle.mpc_cost(d, q, goal, qref, w)
    cq = np.sin(0.25) ** 2
    tips = np.sum((p - [0.14, 0, 0]) ** 2) + np.sum((p - [-0.1, -0.03, 0.04]) ** 2)
    joint = 2 * (np.pi / 2 - 0.1) ** 2 + 0.1 ** 2
    exp = 2.0 * cq + 3.0 * (0.01 + 0.02 + 0.02) + 10.0 * tips + 0.05 * joint + (5.0 if fall_radius == 0.02 else 0.0)
    assert run == pytest.approx(exp, rel=1e-13)
    assert term == pytest.approx(50.0 * (0.01 ** 2 + 0.02 ** 2 + 0.02 ** 2) + 20.0 * cq, rel=1e-13)


def test_exact_impedance_worked_step(oracle):
    """The exact diagonal impedance of Sec. III-B (trace_mode 2), by hand: a 1 kg sphere
    (r = 0.05, I = 1e-3) at rest 2 mm into the plane, 4 facets, mu = 0.5.  Facet j's row is
    (u_j, l x u_j) with u_j = n - mu d_j and lever l = (0, 0, -(r - 0.001)); its diagonal
    w_j = |u_j|^2 / m + |l x u_j|^2 / I = 1.25 + (0.5 * 0.049)^2 / 1e-3 = 1.85025, and
    M_j = 1 / ((k dt + d) w_j) takes the place of M(phi)."""
    k, dd, mu, phi = 0.1, 0.001, 0.5, -0.002
    w = 1.25 + (0.5 * 0.049) ** 2 / 1e-3
    Mj = 1.0 / ((k * DT + dd) * w)
    s = -G * DT
    lam = -k * Mj * (s * DT + phi) - dd * Mj * s
    assert lam == pytest.approx(450.389 * 0.000223544, rel=1e-5)   # printed digits of the hand values
    d = Wd.sphere_on_plane()
    q, v = Wd.free_state((0, 0, 0.048))
    rec = oracle.step_record(d, Wd.params(n_t=4, trace_mode=2), DT, q, v)
    c = rec["contacts"][0]
    assert c["lam_sum"] == pytest.approx(4 * lam, rel=1e-12)
    np.testing.assert_allclose(rec["v"][:3], [0, 0, s + 4 * lam], rtol=1e-12, atol=1e-15)
    np.testing.assert_allclose(rec["v"][3:], 0.0, atol=1e-15)


def test_exact_impedance_cancels_each_facet_velocity(oracle):
    """With k = 0 the diagonal form gives every active facet the impulse -s_j / w_j that alone
    brings its own velocity to zero.  Frictionless 4-facet contact of a sphere falling at 1 m/s:
    four equal facets J_n with w = 1/m, so v+_n = s - 4 s = -3 s, s = v_n - g dt."""
    d = Wd.sphere_on_plane(mu=(0.0, 0.0, 0.0))
    q, v = Wd.free_state((0, 0, 0.05 - 1e-6), lin=(0, 0, -1.0))
    p = Wd.params(n_t=4, trace_mode=2, k_user=0.0, d_user=0.001)
    rec = oracle.step_record(d, p, DT, q, v)
    s = -1.0 - G * DT
    np.testing.assert_allclose(rec["v"][:3], [0, 0, -3 * s], rtol=1e-12, atol=1e-14)
    np.testing.assert_allclose(rec["v"][3:], 0.0, atol=1e-14)


def _hinge(axis, ipos, rng=(0.0, 0.0), fl=0.0, inertia=(1e-3, 1e-3, 2e-3)):
    return Wd.world([dict(parent=-1, jnt=S.HINGE, pos=(0, 0, 1.0), axis=axis, ipos=ipos, mass=1.0, inertia=inertia,
                          range=rng, frictionloss=fl)],
                    [dict(type=S.PLANE, body=-1)])


@pytest.mark.parametrize("q0,v_exp", [(-0.51, 0.019), (0.51, -0.019), (0.2, 0.0)])
def test_joint_limit_closed_form(oracle, q0, v_exp):
    """A limit is a one-row constraint with the contact impulse law (the paper names joint limits
    in its system model without a formula; this is the reading taken).  A vertical
    hinge (no gravity torque) at rest, 1 cm past its limit [-0.5, 0.5]: r(|gap|) = r_max = 0.95,
    M = r/(1-r) / (M~^-1)_kk, lambda dt = k M |gap|, so v+ = (M~^-1)_kk lambda dt =
    k r/(1-r) |gap| = 0.1 * 19 * 0.01 = 0.019 rad/s whatever the inertia; inside the range
    nothing happens."""
    d = _hinge((0, 0, 1), (0, 0, 0), rng=(-0.5, 0.5))
    q, v, _ = oracle.step(d, Wd.params(), DT, 1, [q0], [0.0])
    assert v[0] == pytest.approx(v_exp, rel=1e-12, abs=1e-15)
    assert q[0] == pytest.approx(q0 + DT * v_exp, rel=1e-12)


@pytest.mark.parametrize("fl", [2.0, 0.5])
def test_dry_joint_friction_closed_form(oracle, fl):
    """Dry joint friction (the stopping impulse -v_s / (M~^-1)_kk clamped to +-f dt): a horizontal hinge (axis y) with its 1 kg centre of mass
    10 cm out along x carries the gravity torque 0.981 N m about M = 1e-3 + 1 * 0.1^2 = 0.011.
    The stopping impulse -v_s M = -0.981 dt fits inside +-fl dt for fl = 2 (the joint holds:
    v+ = 0); for fl = 0.5 it saturates: v+ = (0.981 - 0.5) dt / 0.011."""
    d = _hinge((0, 1, 0), (0.1, 0, 0), fl=fl)
    q, v, _ = oracle.step(d, Wd.params(), DT, 1, [0.0], [0.0])
    exp = 0.0 if fl == 2.0 else (0.981 - 0.5) * DT / 0.011
    assert v[0] == pytest.approx(exp, rel=1e-9, abs=1e-15)


def test_rest_penetration_fixed_point(oracle):
    """A sphere at rest settles where the F facet impulses carry its weight:
    F M(phi) (k (g dt^2 + |phi|) + d g dt) = m g dt (all facets see s = -g dt), with M(phi) at
    r_max and the lever arm r - |phi|/2 of the midpoint contact."""
    r, m, I, k, dd = 0.05, 1.0, 1e-3, 0.1, 0.001
    for nt, ntor, nrol in [(4, 0, 0), (8, 2, 8)]:
        F = nt + ntor + nrol
        lo, hi = 1e-3, 0.04
        for _ in range(200):  # bisection on the balance residual
            a = 0.5 * (lo + hi)
            lev = r - a / 2
            Mp = 19.0 / (3 / m + 2 * lev * lev / I)
            res = F * Mp * (k * (G * DT * DT + a) + dd * G * DT) - m * G * DT
            lo, hi = (a, hi) if res < 0 else (lo, a)
        d = Wd.sphere_on_plane(mu=(0.5, 0.005, 0.005))
        q, v = Wd.free_state((0, 0, 0.05))
        q, v, _ = oracle.step(d, Wd.params(n_t=nt, n_tor=ntor, n_rol=nrol), DT, 6000, q, v)
        assert r - q[2] == pytest.approx(0.5 * (lo + hi), rel=1e-6)
        assert np.abs(v).max() < 1e-9


# Table tbl:depths (Sec. IV-A): mean penetration depth (mm) of the method in a dense drop of
# ~5 cm primitives at dt = 2 ms, for each (k_user, d_user)
DEPTH_TABLE = [((0.1, 0.001), 3.9), ((0.1, 0.005), 3.8), ((0.3, 0.001), 1.6), ((0.3, 0.005), 1.4),
               ((0.5, 0.001), 1.0), ((0.5, 0.005), 0.9)]


def _resting_depth(oracle, body, k, d, trace_mode=0):
    """Depth (m) of a 5 cm body settled on the plane z = 0 with the 6D cone, 3000 steps of 2 ms."""
    mu = (0.5, 0.005, 0.005)
    if body == "sphere":
        w = Wd.sphere_on_plane(mu=mu)
        q, v = Wd.free_state((0, 0, 0.05))
    else:
        h = 0.025
        m, inert = S.box_mass_inertia((h, h, h), 1000 * (2 * h) ** 3)
        w = Wd.world([dict(mass=m, inertia=inert)], [dict(type=S.PLANE, body=-1, mu=mu),
                                                    dict(type=S.BOX, body=0, size=(h, h, h), mu=mu)])
        q, v = Wd.free_state((0, 0, h))
    p = Wd.params(n_t=8, n_tor=2, n_rol=8, k_user=k, d_user=d, trace_mode=trace_mode)
    q, v, _ = oracle.step(w, p, DT, 3000, q, v)
    assert np.abs(v).max() < 1e-9
    return -min(c["phi"] for c in oracle.step_record(w, p, DT, q, v)["contacts"])


def test_resting_depths_follow_the_papers_depth_table(oracle):
    """Table tbl:depths orders the six impedance settings by depth: a larger k_user and a larger
    d_user both penetrate less.  (The sentence beside the table states the opposite for k_user;
    the table agrees with Eq. cf_wrench, where k_user scales the stiffness of the gap term, and is
    the reading taken.)  A 5 cm, 1 kg sphere and a 5 cm cube settled on a plane reproduce that
    strict order.  The sphere's depths also land within a third of the table's means, although
    the scenes differ (one resting body against a dense drop of mixed primitives).  The other
    reading of the trace in M(phi), 1/m per body (trace_mode 1), puts them out of that band and
    out of order: the printed values pin the translational point-Jacobian trace."""
    for body in ("sphere", "cube"):
        depths = [_resting_depth(oracle, body, k, d) for (k, d), _ in DEPTH_TABLE]
        assert all(a > b for a, b in zip(depths, depths[1:])), (body, depths)
    sphere = np.array([_resting_depth(oracle, "sphere", k, d) for (k, d), _ in DEPTH_TABLE])
    table = np.array([mm for _, mm in DEPTH_TABLE]) * 1e-3
    assert np.all((sphere / table > 0.75) & (sphere / table < 4 / 3)), sphere / table
    alt = np.array([_resting_depth(oracle, "sphere", k, d, trace_mode=1) for (k, d), _ in DEPTH_TABLE])
    assert not np.all((alt / table > 0.75) & (alt / table < 4 / 3))
    assert not all(a > b for a, b in zip(alt, alt[1:]))


# ------------------------------------------------------------------------------------------
# the paper's qualitative behaviours (Sec. IV-B, IV-C) on the oracle
# ------------------------------------------------------------------------------------------
def _trajectory(oracle, d, p, q, v, dt, steps, every):
    out = []
    for _ in range(steps // every):
        q, v, _ = oracle.step(d, p, dt, every, q, v)
        out.append((q.copy(), v.copy()))
    return out


def test_torsional_friction_decays_a_spin_faster_for_a_larger_coefficient(oracle):
    """Sec. IV-B: a sphere held to spin about the normal (a vertical hinge through its centre,
    2 mm into the floor) loses its spin monotonically, faster for the larger mu_tor.  The contact
    point lies on the hinge axis, so the translational trace is zero; the per-body 1/m
    impedance (trace_mode 1) is used."""
    finals = {}
    for mu_tor in (0.002, 0.01):
        d = Wd.world([dict(parent=-1, jnt=S.HINGE, pos=(0, 0, 0.048), axis=(0, 0, 1), mass=1.0,
                           inertia=(1e-3, 1e-3, 1e-3))],
                     [dict(type=S.PLANE, body=-1, mu=(0.5, mu_tor, 0.0)),
                      dict(type=S.SPHERE, body=0, size=(0.05, 0, 0), mu=(0.5, mu_tor, 0.0))])
        p = Wd.params(n_t=4, n_tor=2, n_rol=0, trace_mode=1)
        w = np.array([v[0] for _, v in _trajectory(oracle, d, p, [0.0], [10.0], DT, 500, 25)])
        assert np.all(np.diff(w) < 0.0) and w[-1] > 0.0
        finals[mu_tor] = w[-1]
    assert finals[0.01] < finals[0.002]


def test_rolling_friction_decays_a_roll_faster_for_a_larger_coefficient(oracle):
    """Sec. IV-B: a capsule rolling without slip along +x slows monotonically, faster for the
    larger mu_rol."""
    finals = {}
    for mu_rol in (0.002, 0.01):
        d = Wd.world([dict(mass=1.0, inertia=(2e-3, 2e-3, 5e-4))],
                     [dict(type=S.PLANE, body=-1, mu=(0.8, 0.0, mu_rol)),
                      dict(type=S.CAPSULE, body=0, size=(0.03, 0.05, 0), mu=(0.8, 0.0, mu_rol))])
        p = Wd.params(n_t=8, n_tor=2, n_rol=8)
        R = np.array([[1, 0, 0], [0, 0, -1], [0, 1, 0]], float)      # capsule axis along y
        q0 = np.array([0, 0, 0.028, *S.quat_about((1, 0, 0), np.pi / 2)])
        v0 = np.array([0.5, 0, 0, *(R.T @ np.array([0, 0.5 / 0.03, 0]))])
        vx = np.array([v[0] for _, v in _trajectory(oracle, d, p, q0, v0, DT, 1000, 50)])
        assert np.all(np.diff(vx[2:]) < 0.0) and vx[-1] > 0.0
        finals[mu_rol] = vx[-1]
    assert finals[0.01] < finals[0.002]


@pytest.mark.parametrize("dt", [0.002, 0.02])
def test_thrown_cube_slides_to_rest_without_drift(oracle, dt):
    """Sec. IV-C: a cube thrown onto a plane with v = (2, 0, 0) and omega = (0.1, 0.1, 0.1) slides
    to rest; its horizontal speed never grows once it slides, and it settles without drift, also
    at dt = 0.02 s (where it rests deeper: about 17 mm against 2.2 mm at dt = 2 ms)."""
    d = Wd.world([dict(mass=1.0, inertia=S.box_mass_inertia([0.05] * 3, 1.0)[1])],
                 [dict(type=S.PLANE, body=-1, mu=(0.5, 0, 0)),
                  dict(type=S.BOX, body=0, size=(0.05, 0.05, 0.05), mu=(0.5, 0, 0))])
    p = Wd.params(n_t=4, k_user=0.3, d_user=0.005)
    steps = int(round(3.0 / dt))
    tr = _trajectory(oracle, d, p, np.array([0, 0, 0.2, 1, 0, 0, 0.0]), np.array([2.0, 0, 0, 0.1, 0.1, 0.1]), dt,
                     steps, max(1, steps // 60))
    speed = np.array([np.hypot(v[0], v[1]) for _, v in tr])
    z = np.array([q[2] for q, _ in tr])
    assert speed[-1] < 0.05 * 2.0
    land = int(np.argmax(z < 0.06))
    assert np.all(np.diff(speed[land + 1:]) <= 1e-9)
    # at rest without drift, penetrating (the gap term's g dt^2 deepens the rest at dt = 0.02 s)
    assert abs(z[-1] - z[-5]) < 1e-4 and (0.045 if dt == 0.002 else 0.03) < z[-1] < 0.05


# ------------------------------------------------------------------------------------------
# invariants
# ------------------------------------------------------------------------------------------
def test_sphere_sphere_conserves_momentum(oracle):
    """Equal and opposite J^T lambda: linear and angular momentum (about the origin) of two
    colliding spheres are conserved without gravity, including an oblique, spinning impact
    through the 6D cone."""
    d = Wd.world([dict(mass=1.0, inertia=(1e-3,) * 3), dict(mass=2.0, inertia=(3e-3,) * 3)],
                 [dict(type=S.SPHERE, body=0, size=(0.05, 0, 0), mu=(0.8, 0.005, 0.005)),
                  dict(type=S.SPHERE, body=1, size=(0.06, 0, 0), mu=(0.8, 0.005, 0.005))])
    p = Wd.params(gravity=(0.0, 0.0, 0.0), n_t=8, n_tor=2, n_rol=8)
    qa, va = Wd.free_state((-0.2, 0.01, 0.02), quat=S.quat_about((1, 0, 0), 0.3), lin=(1.0, 0, 0), ang=(0, 5, 1))
    qb, vb = Wd.free_state((0.2, -0.01, 0.0), lin=(-0.5, 0.1, 0), ang=(3, 0, -2))
    q, v = np.concatenate([qa, qb]), np.concatenate([va, vb])
    m = np.array([1.0, 2.0])
    inert = [np.full(3, 1e-3), np.full(3, 3e-3)]

    def momenta(q, v):
        _, _, poses = oracle.dynamics(d, (0, 0, 0), q, v)
        P = sum(m[i] * v[6 * i:6 * i + 3] for i in range(2))
        L = sum(np.cross(q[7 * i:7 * i + 3], m[i] * v[6 * i:6 * i + 3])
                + poses[i, 3:12].reshape(3, 3) @ (inert[i] * v[6 * i + 3:6 * i + 6]) for i in range(2))
        return P, L

    P0, L0 = momenta(q, v)
    total = 0
    for _ in range(60):
        q, v, nc = oracle.step(d, p, DT, 10, q, v)
        total += nc
    P1, L1 = momenta(q, v)
    assert total > 0
    np.testing.assert_allclose(P1, P0, atol=1e-13)
    np.testing.assert_allclose(L1, L0, atol=1e-12)


def _pile_record(oracle, nbody=16, seed=3, settle=150):
    b = S.make_pile(1, nbody, seed=seed)
    d = b.world(0)
    q, v, _ = oracle.step(d, b.params, b.dt, settle, b.q0[0], b.v0[0])
    return b, d, q, v, oracle.step_record(d, b.params, b.dt, q, v)


def test_facet_impulses_stay_in_the_primal_cone(oracle):
    """lambda_j >= 0 for every facet, so the resultant satisfies Eq. primal_cone: the tangential
    part lies in mu N_t conv{d_j} (within mu N_t), torsion within mu_tor N_tor, rolling within
    mu_rol N_rol, with N_s the normal impulse of subspace s (all <= the total N)."""
    b, d, q, v, rec = _pile_record(oracle)
    assert len(rec["contacts"]) > 5
    mu = S.PILE_MU
    for c in rec["contacts"]:
        w = c["wrench"]
        assert w[0] >= 0.0
        assert np.hypot(w[1], w[2]) <= mu[0] * w[0] * (1 + 1e-12) + 1e-18
        assert abs(w[3]) <= mu[1] * w[0] * (1 + 1e-12) + 1e-18
        assert np.hypot(w[4], w[5]) <= mu[2] * w[0] * (1 + 1e-12) + 1e-18
        assert c["nfacet"] == 18 and 0 <= c["nactive"] <= 18
        # the frame is orthonormal and right handed
        fr = np.stack([c["normal"], c["t1"], c["t2"]])
        np.testing.assert_allclose(fr @ fr.T, np.eye(3), atol=1e-12)
        assert np.linalg.det(np.stack([c["t1"], c["t2"], c["normal"]])) == pytest.approx(1.0, abs=1e-12)


def test_four_facet_friction_polytope(oracle):
    """With facets {+-t1, +-t2}: |F_t1| + |F_t2| <= mu N (the 1-norm ball of the pyramid)."""
    d = Wd.sphere_on_plane()
    q, v = Wd.free_state((0, 0, 0.047), lin=(0.3, -0.7, 0.1), ang=(2, 1, 0))
    rec = oracle.step_record(d, Wd.params(n_t=4), DT, q, v)
    w = rec["contacts"][0]["wrench"]
    assert abs(w[1]) + abs(w[2]) <= 0.5 * w[0] * (1 + 1e-12)
    assert abs(w[1]) + abs(w[2]) > 0.1 * w[0]


def test_permutation_invariance(oracle):
    """Decoupling across contacts: relabelling the bodies (and with them every contact) changes
    the next state only at rounding level."""
    b, d, q, v, _ = _pile_record(oracle, settle=120)
    n = len(d["body_parent"])
    perm = np.random.default_rng(0).permutation(n)
    d2 = {k: np.array(x) for k, x in d.items()}
    for k in ("body_mass", "body_inertia"):
        d2[k] = d[k][perm]
    for k in ("geom_type", "geom_size", "geom_pos", "geom_quat", "geom_mu"):
        d2[k][:n] = d[k][:n][perm]
    q2 = q.reshape(n, 7)[perm].reshape(-1)
    v2 = v.reshape(n, 6)[perm].reshape(-1)
    qa, va, _ = oracle.step(d, b.params, b.dt, 1, q, v)
    qb, vb, _ = oracle.step(d2, b.params, b.dt, 1, q2, v2)
    np.testing.assert_allclose(vb.reshape(n, 6), va.reshape(n, 6)[perm], rtol=1e-9, atol=1e-13)
    np.testing.assert_allclose(qb.reshape(n, 7), qa.reshape(n, 7)[perm], rtol=1e-12, atol=1e-14)


def test_stick_slip_switches_at_tan_theta_equal_mu(oracle):
    """A non-rotating block on an incline with the 4-facet cone aligned with the slope: below
    tan(theta) = mu the slide settles to a bounded (viscous) terminal speed; above it, only the
    downhill facet stays active and the acceleration approaches Coulomb's g(sin - mu cos)."""
    mu = 0.5
    res = {}
    for ratio in (0.8, 1.2):
        th = np.arctan(ratio * mu)
        pq = S.quat_about((0, 1, 0), th)
        d = Wd.world([dict(mass=1.0, inertia=(1e9,) * 3)],
                     [dict(type=S.PLANE, body=-1, quat=pq, mu=(mu, 0, 0)),
                      dict(type=S.SPHERE, body=0, size=(0.05, 0, 0), mu=(mu, 0, 0))])
        slope = np.array([np.cos(th), 0, -np.sin(th)])
        q, v = Wd.free_state(0.05 * np.array([np.sin(th), 0, np.cos(th)]))
        speeds = []
        for _ in range(10):
            q, v, _ = oracle.step(d, Wd.params(n_t=4), DT, 1000, q, v)
            speeds.append(v[:3] @ slope)
        res[ratio] = (np.array(speeds), G * (np.sin(th) - mu * np.cos(th)))
    sp, _ = res[0.8]
    assert abs(sp[-1] - sp[-2]) < 0.02 * abs(sp[-1])          # terminal speed reached
    sp, coulomb = res[1.2]
    acc = (sp[-1] - sp[-5]) / 8.0
    assert acc == pytest.approx(coulomb, rel=0.08)


# ------------------------------------------------------------------------------------------
# rigid-body dynamics: kinematics, inertia, bias, factorisation
# ------------------------------------------------------------------------------------------
def _planar_arm(l1=0.3, l2=0.2):
    """Two hinges about the world y axis; link 1 from the origin along +x, link 2 along +x."""
    bodies = [dict(parent=-1, jnt=S.HINGE, axis=(0, 1, 0), ipos=(l1 / 2, 0, 0), mass=1.3, inertia=(1e-3, 8e-3, 9e-3),
                   damping=0.1),
              dict(parent=0, jnt=S.HINGE, pos=(l1, 0, 0), axis=(0, 1, 0), ipos=(l2 / 2, 0, 0), mass=0.7,
                   inertia=(5e-4, 3e-3, 3.2e-3), damping=0.1)]
    return Wd.world(bodies, [dict(type=S.CAPSULE, body=0, pos=(l1 / 2, 0, 0), size=(0.02, 0.1, 0))])


def _spatial_arm():
    """Three hinges with non-parallel axes: about z at the origin; about y at (0.25, 0, 0) in a
    child frame turned 0.3 rad about x; about x at (0, 0.1, 0.15) in a grandchild frame turned
    0.5 rad about z.  Off-axis centres of mass, anisotropic inertias, joint damping."""
    bodies = [dict(parent=-1, jnt=S.HINGE, axis=(0, 0, 1), ipos=(0.1, 0.02, 0), mass=1.1,
                   inertia=(1e-3, 6e-3, 7e-3), damping=0.2),
              dict(parent=0, jnt=S.HINGE, pos=(0.25, 0, 0), quat=S.quat_about((1, 0, 0), 0.3), axis=(0, 1, 0),
                   ipos=(0.03, 0.05, 0.06), mass=0.6, inertia=(2e-3, 1e-3, 2.5e-3), damping=0.1),
              dict(parent=1, jnt=S.HINGE, pos=(0, 0.1, 0.15), quat=S.quat_about((0, 0, 1), 0.5), axis=(1, 0, 0),
                   ipos=(0.02, -0.01, 0.04), mass=0.3, inertia=(4e-4, 5e-4, 2e-4), damping=0.05)]
    return Wd.world(bodies, [dict(type=S.CAPSULE, body=2, pos=(0, 0, 0.04), size=(0.01, 0.03, 0))])


def test_forward_kinematics_planar_arm(oracle):
    """Closed form of a planar two-link arm: a rotation by +a about +y takes x to (cos a, 0, -sin a)."""
    l1, l2 = 0.3, 0.2
    d = _planar_arm(l1, l2)
    a1, a2 = 0.4, -1.1
    _, _, poses = oracle.dynamics(d, (0, 0, -G), np.array([a1, a2]), np.zeros(2))
    e = lambda a: np.array([np.cos(a), 0, -np.sin(a)])
    np.testing.assert_allclose(poses[1, :3], l1 * e(a1), atol=1e-14)
    np.testing.assert_allclose(poses[1, 12:15], l1 * e(a1) + l2 / 2 * e(a1 + a2), atol=1e-14)


def _kinetic_fd(oracle, d, q, h=1e-6):
    """M by polarisation of the kinetic energy, with body velocities from central differences of
    the forward kinematics (hinge worlds: q + h v is a valid perturbation)."""
    nv = len(q)
    mass, inert = d["body_mass"], d["body_inertia"]

    def T(vel):
        _, _, pp = oracle.dynamics(d, (0, 0, 0), q + h * vel, np.zeros(nv))
        _, _, pm = oracle.dynamics(d, (0, 0, 0), q - h * vel, np.zeros(nv))
        e = 0.0
        for b in range(len(mass)):
            vc = (pp[b, 12:15] - pm[b, 12:15]) / (2 * h)
            Rp, Rm = pp[b, 3:12].reshape(3, 3), pm[b, 3:12].reshape(3, 3)
            W = (Rp - Rm) / (2 * h) @ ((Rp + Rm) / 2).T      # skew(omega_world)
            w = np.array([W[2, 1], W[0, 2], W[1, 0]])
            R = (Rp + Rm) / 2
            e += 0.5 * mass[b] * vc @ vc + 0.5 * w @ (R @ np.diag(inert[b]) @ R.T) @ w
        return e

    M = np.zeros((nv, nv))
    I = np.eye(nv)
    for i in range(nv):
        for j in range(nv):
            M[i, j] = T(I[i] + I[j]) - T(I[i]) - T(I[j])
    return M


def test_mass_matrix_matches_kinetic_energy(oracle):
    for d, q in [(_planar_arm(), np.array([0.4, -1.1])), (_spatial_arm(), np.array([0.7, -0.4, 1.2])),
                 (S.hand_template(seed=2).__dict__, None)]:
        if q is None:
            t = S.hand_template(seed=2)
            d = {k: getattr(t, k) for k in t.__dataclass_fields__ if k not in ("name", "pile")}
            # fingers only: drop the free cube (its quasi-velocity is not a q-derivative)
            keep = np.arange(1, t.nbody)
            d = {k: (v[keep] if k.startswith("body_") and v is not None else v) for k, v in d.items()}
            d["body_parent"] = np.where(d["body_parent"] > 0, d["body_parent"] - 1, -1).astype(np.int32)
            d["geom_body"] = np.where(d["geom_body"] > 0, d["geom_body"] - 1, -1).astype(np.int32)
            d["geom_type"] = np.where(d["geom_body"] >= 0, d["geom_type"], S.PLANE).astype(np.int32)
            q = np.random.default_rng(1).uniform(-0.5, 0.5, 16)
        M, _, _ = oracle.dynamics(d, (0, 0, -G), q, np.zeros(len(q)))
        Mfd = _kinetic_fd(oracle, d, q)
        np.testing.assert_allclose(M, Mfd, rtol=1e-6, atol=1e-9 * np.abs(M).max())
        np.testing.assert_allclose(M, M.T, atol=1e-16)


@pytest.mark.parametrize("arm", ["planar", "spatial"])
def test_bias_forces_match_euler_lagrange(oracle, arm):
    """c(q, v) = Mdot v - dT/dq + dV/dq (Euler-Lagrange with zero joint acceleration), each term
    by central differences of the (separately pinned) inertia and of the potential sum m g z.
    The spatial arm's non-parallel axes make the velocity-product terms that a planar chain
    cancels (a child axis turning with its parent) count."""
    if arm == "planar":
        d, q, v = _planar_arm(), np.array([0.4, -1.1]), np.array([1.7, -2.3])
    else:
        d, q, v = _spatial_arm(), np.array([0.7, -0.4, 1.2]), np.array([1.3, -2.1, 2.6])
    n = len(q)
    h = 1e-6
    M = lambda qq: oracle.dynamics(d, (0, 0, -G), qq, v)[0]
    Mdot = (M(q + h * v) - M(q - h * v)) / (2 * h)
    dT = np.array([(0.5 * v @ M(q + h * e) @ v - 0.5 * v @ M(q - h * e) @ v) / (2 * h) for e in np.eye(n)])

    def V(qq):
        _, _, p = oracle.dynamics(d, (0, 0, -G), qq, v)
        return sum(d["body_mass"][b] * G * p[b, 14] for b in range(n))

    dV = np.array([(V(q + h * e) - V(q - h * e)) / (2 * h) for e in np.eye(n)])
    _, c, _ = oracle.dynamics(d, (0, 0, -G), q, v)
    np.testing.assert_allclose(c, Mdot @ v - dT + dV, rtol=1e-7, atol=1e-9)


def test_cholesky_matches_numpy(oracle):
    rng = np.random.default_rng(0)
    A = rng.standard_normal((7, 7))
    A = A @ A.T + 0.1 * np.eye(7)
    np.testing.assert_allclose(oracle.cholesky(A), np.linalg.cholesky(A), rtol=1e-12, atol=1e-14)


def test_implicit_damping_smooth_velocity(oracle):
    """Eq. smooth_vel with implicit damping on a single hinge without gravity: the rate decays
    as v1 = v0 (I - 0) / (I + dt b) ... i.e. (M + dt b) v1 = M v0 for M = const."""
    d = Wd.world([dict(parent=-1, jnt=S.HINGE, axis=(0, 0, 1), mass=1.0, inertia=(1e-2, 1e-2, 2e-2), damping=0.3)],
                 [dict(type=S.SPHERE, body=0, size=(0.01, 0, 0))])
    q, v, _ = oracle.step(d, Wd.params(gravity=(0.0, 0.0, 0.0)), DT, 1, np.zeros(1), np.array([2.0]))
    assert v[0] == pytest.approx(2.0 * 2e-2 / (2e-2 + DT * 0.3), rel=1e-14)
    assert q[0] == pytest.approx(DT * v[0], rel=1e-14)


def test_smooth_prediction_on_a_coupled_chain(oracle):
    """Eq. smooth_vel on the spatial arm (no contacts): v+ = v + dt (M + dt B)^-1 (tau - c - B v),
    with M and c from the separately pinned inertia and bias and the solve done by numpy; the
    chain's M is dense, so each factor and substitution step of the oracle's solve counts."""
    d = _spatial_arm()
    q, v, tau = np.array([0.7, -0.4, 1.2]), np.array([1.3, -2.1, 2.6]), np.array([0.4, -0.3, 0.05])
    M, c, _ = oracle.dynamics(d, (0, 0, -G), q, v)
    assert np.abs(M[0, 1]) > 1e-3 and np.abs(M[1, 2]) > 1e-4 and np.abs(M[0, 2]) > 1e-4
    B = np.diag(d["body_damping"])
    v_exp = v + DT * np.linalg.solve(M + DT * B, tau - c - B @ v)
    q1, v1, nc = oracle.step(d, Wd.params(), DT, 1, q, v, tau=tau[None])
    assert nc == 0
    np.testing.assert_allclose(v1, v_exp, rtol=1e-13, atol=1e-14)
    np.testing.assert_allclose(q1, q + DT * v_exp, rtol=1e-13, atol=1e-15)


# ------------------------------------------------------------------------------------------
# narrowphase against brute force
# ------------------------------------------------------------------------------------------
def _box_sdf(x, half):
    qd = np.abs(x) - half
    return np.linalg.norm(np.maximum(qd, 0), axis=-1) + np.minimum(qd.max(axis=-1), 0)


def test_capsule_box_minimiser_brute_force(oracle):
    """The exact piecewise minimiser of the box SDF along the segment agrees with a dense grid."""
    rng = np.random.default_rng(5)
    half = np.array([0.03, 0.04, 0.05])
    for _ in range(300):
        w = rng.standard_normal(3)
        w /= np.linalg.norm(w)
        x0 = rng.uniform(-0.12, 0.12, 3)
        h = rng.uniform(0.01, 0.06)
        t = oracle.capsule_box_param(x0, w, h, half)
        grid = np.linspace(-h, h, 200001)
        f = _box_sdf(x0[None] + grid[:, None] * w[None], half)
        ft = _box_sdf((x0 + t * w)[None], half)[0]
        assert -h - 1e-15 <= t <= h + 1e-15
        assert ft <= f.min() + 1e-9


def _two_body_contact(oracle, ga, gb, qa, qb):
    d = Wd.world([dict(mass=1.0), dict(mass=1.0)], [dict(ga, body=0), dict(gb, body=1)])
    rec = oracle.step_record(d, Wd.params(gravity=(0.0, 0.0, 0.0), margin=1.0), DT, np.concatenate([qa, qb]),
                             np.zeros(12))
    return rec["contacts"]


def _surface_points(g, q, n=60000, rng=None):
    """Dense samples of a geom's surface in world coordinates."""
    rng = rng or np.random.default_rng(0)
    u = rng.standard_normal((n, 3))
    u /= np.linalg.norm(u, axis=1, keepdims=True)
    r = g["size"][0]
    if g["type"] == S.SPHERE:
        pts = r * u
    elif g["type"] == S.CAPSULE:
        t = rng.uniform(-1, 1, n)
        core = np.zeros((n, 3))
        core[:, 2] = t * g["size"][1]
        pts = core + r * u
        keep = np.abs(pts[:, 2]) >= 0  # core + sphere shell: the outer envelope is the capsule surface
        pts = pts[keep]
    else:
        half = np.array(g["size"])
        face = rng.integers(0, 3, n)
        pts = rng.uniform(-1, 1, (n, 3)) * half
        sgn = np.where(rng.random(n) < 0.5, -1, 1)
        pts[np.arange(n), face] = sgn * half[face]
    w, x, y, z = q[3:]
    R = np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
                  [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
                  [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)]])
    return q[:3] + pts @ R.T


def _inside(g, q, pts):
    w, x, y, z = q[3:]
    R = np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
                  [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
                  [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)]])
    l = (pts - q[:3]) @ R
    if g["type"] == S.SPHERE:
        return np.linalg.norm(l, axis=1) < g["size"][0]
    if g["type"] == S.CAPSULE:
        t = np.clip(l[:, 2], -g["size"][1], g["size"][1])
        return np.hypot(np.hypot(l[:, 0], l[:, 1]), l[:, 2] - t) < g["size"][0]
    return np.all(np.abs(l) < np.array(g["size"]), axis=1)


@pytest.mark.parametrize("ta,tb", [(S.SPHERE, S.SPHERE), (S.SPHERE, S.CAPSULE), (S.CAPSULE, S.SPHERE),
                                   (S.CAPSULE, S.CAPSULE), (S.SPHERE, S.BOX), (S.CAPSULE, S.BOX), (S.BOX, S.CAPSULE)])
def test_narrowphase_distance_brute_force(oracle, ta, tb):
    """Separated pairs: phi equals the minimum distance between dense surface samples; the
    normal is the unit vector between the surface points and points from B to A."""
    rng = np.random.default_rng(ta * 10 + tb)
    size = {S.SPHERE: (0.04, 0, 0), S.CAPSULE: (0.03, 0.05, 0), S.BOX: (0.03, 0.04, 0.05)}
    done = 0
    for trial in range(40):
        qa = np.concatenate([rng.uniform(-0.02, 0.02, 3), S.random_quats(rng, 1)[0]])
        qb = np.concatenate([rng.uniform(-0.02, 0.02, 3) + rng.standard_normal(3) / 6, S.random_quats(rng, 1)[0]])
        ga, gb = dict(type=ta, size=size[ta]), dict(type=tb, size=size[tb])
        cs = _two_body_contact(oracle, ga, gb, qa, qb)
        assert len(cs) == 1
        c = cs[0]
        if c["phi"] < 0.005:
            continue
        pa, pb = _surface_points(ga, qa, rng=rng), _surface_points(gb, qb, rng=rng)
        from scipy.spatial import cKDTree
        dist, _ = cKDTree(pb).query(pa)
        assert c["phi"] <= dist.min() + 1e-9           # no pair of surface points is closer
        assert c["phi"] >= dist.min() - 3e-3           # ... up to the sampling resolution
        sa = c["pos"] + c["phi"] / 2 * c["normal"]     # surface point of A (n points from B to A)
        sb = c["pos"] - c["phi"] / 2 * c["normal"]     # surface point of B
        assert np.linalg.norm(sa - sb) == pytest.approx(c["phi"], rel=1e-12)
        assert _inside(ga, qa, (sa + 1e-4 * c["normal"])[None])[0]
        assert not _inside(ga, qa, (sa - 1e-4 * c["normal"])[None])[0]
        assert _inside(gb, qb, (sb - 1e-4 * c["normal"])[None])[0]
        assert not _inside(gb, qb, (sb + 1e-4 * c["normal"])[None])[0]
        done += 1
        if done >= 6:
            break
    assert done >= 3


@pytest.mark.parametrize("sphere_first", [True, False])
def test_sphere_centre_inside_a_box_leaves_through_the_nearest_face(oracle, sphere_first):
    """A sphere (r = 2 cm) whose centre lies inside a turned box at local (0.04, 0.01, -0.005),
    half extents (0.05, 0.04, 0.03): the face depths are 0.01, 0.03, 0.025, so the +x face is
    nearest.  The gap is -(0.01 + r), the normal is the box's +x axis from the box to the sphere
    (negated when the box is A), and the point is the midpoint of the sphere's deepest point and
    the centre's projection onto that face."""
    half = np.array([0.05, 0.04, 0.03])
    qbox = np.concatenate([[0.1, -0.2, 0.3], S.quat_about((1, 2, -1), 0.8)])
    R = _quat_mat(qbox[3:])
    local = np.array([0.04, 0.01, -0.005])
    centre = qbox[:3] + R @ local
    qs = np.concatenate([centre, [1.0, 0, 0, 0]])
    gs, gbx = dict(type=S.SPHERE, size=(0.02, 0, 0)), dict(type=S.BOX, size=tuple(half))
    cs = (_two_body_contact(oracle, gs, gbx, qs, qbox) if sphere_first
          else _two_body_contact(oracle, gbx, gs, qbox, qs))
    assert len(cs) == 1
    c = cs[0]
    nb = R[:, 0]                                       # out of the +x face
    assert c["phi"] == pytest.approx(-(0.01 + 0.02), abs=1e-15)
    np.testing.assert_allclose(c["normal"], nb if sphere_first else -nb, atol=1e-15)
    face = qbox[:3] + R @ np.array([0.05, 0.01, -0.005])
    np.testing.assert_allclose(c["pos"], 0.5 * ((centre - 0.02 * nb) + face), atol=1e-15)


@pytest.mark.parametrize("offset_x", [0.02, 0.08])
def test_crossed_capsules_closed_form(oracle, offset_x):
    """Capsule A along x (r = 1 cm, half length 5 cm) at the origin; capsule B along y
    (r = 1.5 cm, half length 5 cm) centred at (offset_x, 0.03, 0.05).  At offset 0.02 the
    closest axis points are (0.02, 0, 0) and (0.02, 0, 0.05), both inside their segments: gap
    0.05 - 0.025, normal -z.  At 0.08 A's closest point clamps to its end (0.05, 0, 0), and B's
    closest point to that is (0.08, 0, 0.05): gap |(-0.03, 0, -0.05)| - 0.025 along that
    direction.  The contact point is the midpoint of the two surface points."""
    qa = np.concatenate([[0.0, 0.0, 0.0], S.quat_about((0, 1, 0), np.pi / 2)])    # z -> x
    qb = np.concatenate([[offset_x, 0.03, 0.05], S.quat_about((1, 0, 0), -np.pi / 2)])   # z -> y
    cs = _two_body_contact(oracle, dict(type=S.CAPSULE, size=(0.01, 0.05, 0)),
                           dict(type=S.CAPSULE, size=(0.015, 0.05, 0)), qa, qb)
    assert len(cs) == 1
    c = cs[0]
    pa = np.array([min(offset_x, 0.05), 0.0, 0.0])
    pb = np.array([offset_x, 0.0, 0.05])
    dist = np.linalg.norm(pa - pb)
    n = (pa - pb) / dist
    assert c["phi"] == pytest.approx(dist - 0.025, abs=1e-15)
    np.testing.assert_allclose(c["normal"], n, atol=1e-15)
    np.testing.assert_allclose(c["pos"], 0.5 * ((pa - 0.01 * n) + (pb + 0.015 * n)), atol=1e-15)


def _quat_mat(q):
    w, x, y, z = q / np.linalg.norm(q)
    return np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
                     [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
                     [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)]])


def _box_sdf_point(p, c, R, hs):
    """Signed distance of point p to a box (textbook: outside part plus inside part)."""
    l = R.T @ (p - c)
    d = np.abs(l) - hs
    return np.linalg.norm(np.maximum(d, 0.0)) + min(max(d[0], d[1], d[2]), 0.0)


def _box_pair_contacts(oracle, ha, hb, qa, qb, margin=0.0):
    d = Wd.world([dict(mass=1.0), dict(mass=1.0)],
                 [dict(type=S.BOX, body=0, size=tuple(ha)), dict(type=S.BOX, body=1, size=tuple(hb))])
    rec = oracle.step_record(d, Wd.params(gravity=(0.0, 0.0, 0.0), margin=margin), DT, np.concatenate([qa, qb]),
                             np.zeros(12))
    return {c["sub"]: c for c in rec["contacts"]}


def test_box_box_is_symmetric_under_swapping_the_boxes(oracle):
    """The box-box contacts (the face of least penetration is the reference face, the other box's
    incident face is clipped against it, and each clipped vertex below the margin is a contact)
    do not depend on which box is A (random overlapping pairs, no ties): the same reference face
    and clipped polygon, so the same subs, gaps and points, normals negated."""
    rng = np.random.default_rng(21)
    ha, hb = np.array([0.03, 0.04, 0.05]), np.array([0.045, 0.025, 0.035])
    seen = 0
    for trial in range(40):
        qa = np.concatenate([rng.uniform(-0.01, 0.01, 3), S.random_quats(rng, 1)[0]])
        qb = np.concatenate([rng.uniform(-0.01, 0.01, 3) + rng.standard_normal(3) * 0.04, S.random_quats(rng, 1)[0]])
        ab = _box_pair_contacts(oracle, ha, hb, qa, qb, margin=0.005)
        ba = _box_pair_contacts(oracle, hb, ha, qb, qa, margin=0.005)
        assert set(ab) == set(ba)
        for k, c in ab.items():
            o = ba[k]
            assert o["phi"] == pytest.approx(c["phi"], abs=1e-12)
            np.testing.assert_allclose(o["normal"], -np.asarray(c["normal"]), atol=1e-12)
            np.testing.assert_allclose(o["pos"], c["pos"], atol=1e-12)
            assert abs(np.linalg.norm(c["normal"]) - 1.0) < 1e-12
        seen += len(ab)
    assert seen > 30


def test_box_box_rotated_cube_on_a_slab(oracle):
    """A 10 cm cube turned 45 degrees about z rests 1 mm into a 40 x 40 x 10 cm slab: the slab's
    top face is the reference, the cube's bottom face lies inside it unclipped, so its four
    corners are the contacts: gap -1 mm, normal from the cube (B) down to the slab (A), points
    halfway between the corners and the slab's top."""
    c45 = np.cos(np.pi / 8)
    qa = np.array([0, 0, 0.05, 1, 0, 0, 0], float)
    qb = np.array([0.01, 0.02, 0.149, c45, 0, 0, np.sin(np.pi / 8)], float)
    cs = _box_pair_contacts(oracle, (0.2, 0.2, 0.05), (0.05, 0.05, 0.05), qa, qb)
    assert sorted(cs) == [0, 1, 2, 3]
    r = 0.05 * np.sqrt(2)
    got = sorted((round(c["pos"][0], 9), round(c["pos"][1], 9)) for c in cs.values())
    want = sorted((round(0.01 + r * np.cos(a), 9), round(0.02 + r * np.sin(a), 9))
                  for a in np.pi / 4 + np.pi / 4 + np.arange(4) * np.pi / 2)
    np.testing.assert_allclose(got, want, atol=1e-9)
    for c in cs.values():
        assert c["phi"] == pytest.approx(-0.001, abs=1e-12)
        np.testing.assert_allclose(c["normal"], [0, 0, -1], atol=1e-12)
        assert c["pos"][2] == pytest.approx(0.0995, abs=1e-12)


def test_box_box_offset_faces_clip_to_the_overlap_rectangle(oracle):
    """Equal 10 cm cubes face to face, the upper offset (1, 0.5) cm and 2 mm deep: the clipped
    polygon is the overlap rectangle x in [-0.04, 0.05], y in [-0.045, 0.05]."""
    q = np.array([0, 0, 0.05, 1, 0, 0, 0, 0.01, 0.005, 0.148, 1, 0, 0, 0], float)
    cs = _box_pair_contacts(oracle, (0.05,) * 3, (0.05,) * 3, q[:7], q[7:])
    assert len(cs) == 4
    got = sorted((round(c["pos"][0], 12), round(c["pos"][1], 12)) for c in cs.values())
    np.testing.assert_allclose(got, sorted([(-0.04, -0.045), (-0.04, 0.05), (0.05, -0.045), (0.05, 0.05)]), atol=1e-12)
    for c in cs.values():
        assert c["phi"] == pytest.approx(-0.002, abs=1e-12)
        np.testing.assert_allclose(c["normal"], [0, 0, -1], atol=1e-12)


def test_box_box_stack_settles_in_place(oracle):
    """Three aligned 10 cm cubes stacked on the floor hold for 0.4 s: each rests within 1.2 cm
    of its stacking height (the contacts are soft and sink under the load above) and has moved
    less than 5 mm sideways.  k = 1, d = 0.01, 4 facets.  (Over longer horizons this stack
    creeps sideways slowly, and the softer k = 0.3 rocks it over: a property of the impedance
    reading, recorded in the design notes.)"""
    h = (0.05, 0.05, 0.05)
    d = Wd.world([dict(mass=1.0, inertia=S.box_mass_inertia(h, 1.0)[1]) for _ in range(3)],
                 [dict(type=S.PLANE, body=-1)] + [dict(type=S.BOX, body=i, size=h) for i in range(3)])
    q = np.array([0, 0, 0.05, 1, 0, 0, 0, 0.005, 0, 0.151, 1, 0, 0, 0, -0.004, 0.003, 0.252, 1, 0, 0, 0], float)
    q1, v1, _ = oracle.step(d, Wd.params(n_t=4, k_user=1.0, d_user=0.01), DT, 200, q, np.zeros(18))
    q1 = q1.reshape(3, 7)
    assert np.abs(v1).max() < 0.1
    for i in range(3):
        assert abs(q1[i, 2] - (0.05 + 0.1 * i)) < 0.012
        assert np.hypot(*(q1[i, :2] - q.reshape(3, 7)[i, :2])) < 0.005


def _plane_contacts(oracle, geom, q):
    d = Wd.world([dict(mass=1.0)], [dict(type=S.PLANE, body=-1), dict(geom, body=0)])
    rec = oracle.step_record(d, Wd.params(gravity=(0.0, 0.0, 0.0), margin=1.0), DT, q, np.zeros(6))
    return {c["sub"]: c for c in rec["contacts"]}


def test_ellipsoid_plane_is_the_lowest_surface_point(oracle):
    """Ellipsoid on a plane, one contact at the surface point furthest along -n: the gap of an
    ellipsoid over the floor is its lowest surface point's height
    (dense surface samples), at any orientation; unrotated it is z - c."""
    rng = np.random.default_rng(31)
    e = np.array([0.05, 0.03, 0.02])
    cs = _plane_contacts(oracle, dict(type=S.ELLIPSOID, size=tuple(e)), np.array([0, 0, 0.1, 1, 0, 0, 0.0]))
    assert cs[0]["phi"] == pytest.approx(0.08, abs=1e-12)
    u = rng.standard_normal((200000, 3))
    u /= np.linalg.norm(u, axis=1, keepdims=True)
    for trial in range(5):
        qu = S.random_quats(rng, 1)[0]
        cs = _plane_contacts(oracle, dict(type=S.ELLIPSOID, size=tuple(e)), np.concatenate([[0.01, 0.02, 0.1], qu]))
        pts = (u * e) @ _quat_mat(qu).T + np.array([0.01, 0.02, 0.1])
        assert cs[0]["phi"] == pytest.approx(pts[:, 2].min(), abs=2e-6)
        assert cs[0]["phi"] <= pts[:, 2].min() + 1e-12


def test_cylinder_plane_rim_points(oracle):
    """Cylinder on a plane, six candidate points (three rim points 120 degrees apart on each
    cap, starting from the cap's lowest rim point): standing, the bottom rim's three points carry the cylinder (gap z - h); lying,
    each cap's lowest rim point (gap z - r); tilted, the lowest of the six is the lowest point of
    the solid (dense rim samples)."""
    r, h = 0.03, 0.05
    g = dict(type=S.CYLINDER, size=(r, h, 0))
    cs = _plane_contacts(oracle, g, np.array([0, 0, 0.2, 1, 0, 0, 0.0]))
    for k in (0, 1, 2):
        assert cs[k]["phi"] == pytest.approx(0.2 - h, abs=1e-12)
    qy = S.quat_about((1, 0, 0), np.pi / 2)
    cs = _plane_contacts(oracle, g, np.concatenate([[0, 0, 0.2], qy]))
    assert cs[0]["phi"] == pytest.approx(0.2 - r, abs=1e-12) and cs[3]["phi"] == pytest.approx(0.2 - r, abs=1e-12)
    rng = np.random.default_rng(32)
    th = np.linspace(0, 2 * np.pi, 100001)
    for trial in range(5):
        qu = S.random_quats(rng, 1)[0]
        cs = _plane_contacts(oracle, g, np.concatenate([[0, 0, 0.2], qu]))
        R = _quat_mat(qu)
        rim = np.concatenate([np.stack([r * np.cos(th), r * np.sin(th), np.full_like(th, z)], 1) for z in (-h, h)])
        low = (rim @ R.T)[:, 2].min() + 0.2
        assert min(c["phi"] for c in cs.values()) == pytest.approx(low, abs=1e-8)


@pytest.mark.parametrize("sphere_first", [True, False])
def test_sphere_centre_inside_a_cylinder_leaves_through_the_nearer_surface(oracle, sphere_first):
    """A sphere (r = 1 cm) whose centre lies inside a turned solid cylinder (r = 3 cm, half
    length 5 cm).  At local (0.025, 0, 0.01) the side is 0.005 deep and the cap 0.04: it leaves
    through the side, normal along the radial direction, contact point on the mantle.  At local
    (0.01, 0, 0.045) the cap (0.005) is nearer than the side (0.02): normal along the axis, point
    on the cap.  The normal points from the cylinder to the sphere (negated when the cylinder is A)
    and the contact point is the midpoint of the sphere's deepest point and the exit point."""
    qc = np.concatenate([[0.1, 0.05, -0.2], S.quat_about((2, -1, 1), 1.1)])
    R = _quat_mat(qc[3:])
    gc, gs = dict(type=S.CYLINDER, size=(0.03, 0.05, 0)), dict(type=S.SPHERE, size=(0.01, 0, 0))
    for local, n_local, depth, exit_local in [((0.025, 0, 0.01), (1, 0, 0), 0.005, (0.03, 0, 0.01)),
                                               ((0.01, 0, 0.045), (0, 0, 1), 0.005, (0.01, 0, 0.05))]:
        centre = qc[:3] + R @ np.array(local)
        qs = np.concatenate([centre, [1.0, 0, 0, 0]])
        cs = (_two_body_contact(oracle, gs, gc, qs, qc) if sphere_first
              else _two_body_contact(oracle, gc, gs, qc, qs))
        assert len(cs) == 1
        c = cs[0]
        nb = R @ np.array(n_local, float)
        assert c["phi"] == pytest.approx(-(depth + 0.01), abs=1e-15)
        np.testing.assert_allclose(c["normal"], nb if sphere_first else -nb, atol=1e-15)
        exit_point = qc[:3] + R @ np.array(exit_local)
        np.testing.assert_allclose(c["pos"], 0.5 * ((centre - 0.01 * nb) + exit_point), atol=1e-15)


def test_sphere_cylinder_distance_brute_force(oracle):
    """Sphere against a solid cylinder: for separated pairs the gap is the distance from the sphere centre
    to the solid cylinder (dense surface samples) minus the radius; for centres inside, the
    smaller of the side and cap depths."""
    rng = np.random.default_rng(33)
    r, h, rs = 0.03, 0.05, 0.02
    th = rng.uniform(0, 2 * np.pi, 300000)
    zz = rng.uniform(-h, h, 300000)
    side = np.stack([r * np.cos(th), r * np.sin(th), zz], 1)
    rr = r * np.sqrt(rng.uniform(0, 1, 200000))
    t2 = rng.uniform(0, 2 * np.pi, 200000)
    caps = np.concatenate([np.stack([rr * np.cos(t2), rr * np.sin(t2), np.full_like(rr, z)], 1) for z in (-h, h)])
    surf = np.concatenate([side, caps])
    from scipy.spatial import cKDTree
    done = 0
    for trial in range(30):
        qc = np.concatenate([[0, 0, 0], S.random_quats(rng, 1)[0]])
        ps = rng.uniform(-0.09, 0.09, 3)
        d = Wd.world([dict(mass=1.0), dict(mass=1.0)], [dict(type=S.SPHERE, body=0, size=(rs, 0, 0)),
                                                         dict(type=S.CYLINDER, body=1, size=(r, h, 0))])
        rec = oracle.step_record(d, Wd.params(gravity=(0.0, 0.0, 0.0), margin=1.0), DT,
                                 np.concatenate([ps, [1, 0, 0, 0], qc]), np.zeros(12))
        c = rec["contacts"][0]
        R = _quat_mat(qc[3:])
        loc = R.T @ ps
        inside = abs(loc[2]) <= h and np.hypot(loc[0], loc[1]) <= r
        if inside:
            want = -min(r - np.hypot(loc[0], loc[1]), h - abs(loc[2])) - rs
        else:
            want = cKDTree(surf @ R.T).query(ps)[0] - rs
        assert c["phi"] == pytest.approx(want, abs=2e-4 if not inside else 1e-12)
        done += 1
    assert done == 30


def test_box_plane_corners_and_capsule_plane_endpoints(oracle):
    """Box-plane emits every corner below the margin; capsule-plane both end spheres."""
    d = Wd.world([dict(mass=1.0), dict(mass=1.0)],
                 [dict(type=S.PLANE, body=-1), dict(type=S.BOX, body=0, size=(0.03, 0.04, 0.05)),
                  dict(type=S.CAPSULE, body=1, size=(0.02, 0.06, 0))])
    tilt = S.quat_about((1, 0, 0), 0.3)
    qa, _ = Wd.free_state((0, 0, 0.01), quat=tilt)
    qb, _ = Wd.free_state((1.0, 0, 0.015), quat=S.quat_about((0, 1, 0), np.pi / 2 - 0.05))
    rec = oracle.step_record(d, Wd.params(gravity=(0.0, 0.0, 0.0)), DT, np.concatenate([qa, qb]), np.zeros(12))
    box = [c for c in rec["contacts"] if c["body_a"] == 0]
    caps = [c for c in rec["contacts"] if c["body_a"] == 1]
    R = np.array(oracle.dynamics(d, (0, 0, 0), np.concatenate([qa, qb]), np.zeros(12))[2][0, 3:12]).reshape(3, 3)
    corners = [np.array([0, 0, 0.01]) + R @ (np.array([sx, sy, sz]) * [0.03, 0.04, 0.05])
               for sx in (-1, 1) for sy in (-1, 1) for sz in (-1, 1)]
    below = sorted(c[2] for c in corners if c[2] < 0)
    assert sorted(c["phi"] for c in box) == pytest.approx(below, abs=1e-15)
    assert len(caps) == 2
    ends_z = sorted(0.015 + s * 0.06 * np.sin(0.05) for s in (-1, 1))
    assert sorted(c["phi"] for c in caps) == pytest.approx([z - 0.02 for z in ends_z], abs=1e-14)


# ------------------------------------------------------------------------------------------
# reference gradient: forward-mode duals against central differences
# ------------------------------------------------------------------------------------------
def test_dual_gradient_matches_finite_differences(oracle):
    b = S.make_hand(2, seed=4)
    d = b.world(0)
    nv = len(b.v0[0])
    T = 20
    rng = np.random.default_rng(0)
    tau = np.zeros((T, nv))
    tau[:, 6:] = rng.normal(0, 0.05, (T, 16))
    dv0 = np.zeros(nv)
    dv0[6:] = rng.standard_normal(16)
    dtau = np.zeros((T, nv))
    dtau[:, 6:] = rng.standard_normal((T, 16))
    tp, tq = np.array([0.0, 0.0, 0.05]), S.quat_about((0, 0, 1), 0.5)
    args = lambda eps: (d, b.params, b.dt, b.q0[0], b.v0[0] + eps * dv0, tau + eps * dtau, np.zeros(len(b.q0[0])),
                        dv0, dtau, 0, tp, tq)
    L, dL = oracle.rollout_loss_dir(*args(0.0))
    h = 1e-6
    Lp, _ = oracle.rollout_loss_dir(*args(h))
    Lm, _ = oracle.rollout_loss_dir(*args(-h))
    assert dL == pytest.approx((Lp - Lm) / (2 * h), rel=1e-5, abs=1e-9)


def test_batch_runner_equals_single_world_steps(oracle):
    """The OpenMP batch entry point (the timed CPU baseline and the parity runs) steps every world
    exactly as the single-world step does: same bits, any thread count."""
    sb = S.make_mixed(4, seed=4)                     # a 16-, 64- and 256-body pile and a hand
    q = np.concatenate([np.asarray(x, np.float64) for x in sb.q0])
    v = np.concatenate([np.asarray(x, np.float64) for x in sb.v0])
    outs = []
    for threads in (1, 3):
        runner = oracle.BatchRunner([sb.world(w) for w in range(sb.nworld)], sb.params)
        qb, vb = q.copy(), v.copy()
        counts = runner.run(qb, vb, sb.dt, 10, nthreads=threads)
        outs.append((qb, vb, counts))
    assert np.array_equal(outs[0][0], outs[1][0]) and np.array_equal(outs[0][1], outs[1][1])
    qo = vo = 0
    for w in range(sb.nworld):
        nq, nv = len(sb.q0[w]), len(sb.v0[w])
        qs, vs, nc = oracle.step(sb.world(w), sb.params, sb.dt, 10, sb.q0[w], sb.v0[w])
        assert np.array_equal(outs[0][0][qo:qo + nq], qs) and np.array_equal(outs[0][1][vo:vo + nv], vs)
        assert outs[0][2][w] == nc
        qo += nq
        vo += nv
