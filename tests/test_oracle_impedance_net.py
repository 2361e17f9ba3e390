"""Pins of the oracle's learned impedance (Sec. III-B: K(q), D(q) learned instead of set by the
heuristic; the model, its inputs and its target are readings) to things other than itself:
the heuristic it must reduce to, a constant scaling that must equal scaling (k, d), the
features and the exact facet impedance worked by hand from the paper's definitions, the
network's layout against a hand-written evaluation, its gradient against central differences
and the first Adam step against the optimiser's definition."""
import numpy as np
import pytest

import worlds as Wd
from paper_2603_12185_gb300 import scenes as S

DT = 0.002
G = 9.81
H, F = 8, 4                      # hidden units, inputs
NP = H * F + 2 * H + 1


def theta_parts(th):
    th = np.asarray(th, float)
    return th[:H * F].reshape(H, F), th[H * F:H * F + H], th[H * F + H:H * F + 2 * H], th[-1]


def make_theta(W1=None, b1=None, w2=None, b2=0.0):
    th = np.zeros(NP)
    if W1 is not None:
        th[:H * F] = np.asarray(W1, float).reshape(-1)
    if b1 is not None:
        th[H * F:H * F + H] = b1
    if w2 is not None:
        th[H * F + H:H * F + 2 * H] = w2
    th[-1] = b2
    return th


def g_by_hand(th, x):
    W1, b1, w2, b2 = theta_parts(th)
    return b2 + np.tanh(np.asarray(x, float) @ W1.T + b1) @ w2


def small_pile():
    b = S.make_pile(nworld=2, nbody=16, seed=3, jammed=True)
    return [(b.world(w), b.q0[w], b.v0[w], b.params) for w in range(2)]


def hand():
    b = S.make_hand(nworld=2, seed=4)
    return [(b.world(w), b.q0[w], b.v0[w], b.params) for w in range(2)]


def with_mode(p, mode, **kw):
    q = S.Params(**{k: getattr(p, k) for k in p.__dataclass_fields__})
    q.trace_mode = mode
    for k, v in kw.items():
        setattr(q, k, v)
    return q


def test_parameter_count(oracle):
    assert oracle.impnet_params() == NP == 49


@pytest.mark.parametrize("scene", ["pile", "hand"])
def test_zero_output_layer_is_the_heuristic(oracle, scene):
    """g = 0 (any first layer, w2 = 0, b2 = 0) multiplies M(phi) by exp(0) = 1: the learned
    mode equals the mode-0 heuristic bit for bit, over several steps."""
    rng = np.random.default_rng(0)
    th = make_theta(W1=rng.normal(size=(H, F)), b1=rng.normal(size=H))
    for d, q0, v0, p in (small_pile() if scene == "pile" else hand()):
        qa, va, na = oracle.step(d, with_mode(p, 0), DT, 5, q0, v0)
        qb, vb, nb = oracle.step(d, with_mode(p, 3), DT, 5, q0, v0, impnet=th)
        assert na == nb and na > 0
        np.testing.assert_array_equal(qa, qb)
        np.testing.assert_array_equal(va, vb)


@pytest.mark.parametrize("scene", ["pile", "hand"])
def test_constant_network_is_scaled_k_and_d(oracle, scene):
    """g = ln 2 everywhere doubles M(phi) in K = k M/dt and D = d M/dt of Eq. k_d_setting,
    which is the heuristic with k_user and d_user doubled (no joint limits in these worlds)."""
    th = make_theta(b2=np.log(2.0))
    for d, q0, v0, p in (small_pile() if scene == "pile" else hand()):
        qa, va, _ = oracle.step(d, with_mode(p, 0, k_user=2 * p.k_user, d_user=2 * p.d_user), DT, 1, q0, v0)
        qb, vb, _ = oracle.step(d, with_mode(p, 3), DT, 1, q0, v0, impnet=th)
        np.testing.assert_allclose(vb, va, rtol=1e-11, atol=1e-12)
        np.testing.assert_allclose(qb, qa, rtol=1e-12, atol=1e-13)


def test_features_of_a_uniform_sphere_on_a_plane(oracle):
    """A uniform sphere (I = 0.4 m r^2) touching a plane: its lever is parallel to the normal,
    tr(J M^-1 J^T) = 3/m + 2 r_c^2 / I with r_c the lever length, so the rotational share is
    x1 = 1 - (3/m) / tr, and the normal row n^T J M^-1 J^T n = 1/m (no rotation) gives
    x2 = (1/m) / tr.  x0 = phi / width, x3 = 1 (a static plane)."""
    m, r = 2.0, 0.05
    I = 0.4 * m * r * r
    d = Wd.sphere_on_plane(r=r, m=m, inertia=I)
    phi = -0.0004
    q, v = Wd.free_state((0, 0, r + phi))
    rec = oracle.step_record(d, Wd.params(n_t=4), DT, q, v)
    c, = rec["contacts"]
    lever = r + phi / 2                     # the contact point sits mid-way through the overlap
    tr = 3 / m + 2 * lever ** 2 / I
    np.testing.assert_allclose(c["feat"], [phi / 0.001, 1 - 3 / m / tr, 1 / m / tr, 1.0], rtol=1e-12, atol=1e-15)
    assert c["trace_a"] + c["trace_b"] == pytest.approx(tr, rel=1e-12)


def test_features_of_a_capsule_end_on_a_capsule(oracle):
    """Two free bodies, no static side (x3 = 0), a slanted normal and levers that are not
    parallel to the normal: the trace (x1) and the normal row (x2) are worked from the
    definition J M^-1 J^T = I/m + [l]x I^-1 [l]x^T of a free body's translational point
    Jacobian, summed over the two bodies."""
    r, h = 0.02, 0.05
    ma, mb = 0.3, 0.7
    Ia, Ib = np.array([2e-4, 3e-4, 1e-4]), np.array([5e-4, 4e-4, 6e-4])
    qa = S.quat_about((0, 1, 0), 0.4)
    d = Wd.world([dict(mass=ma, inertia=tuple(Ia)), dict(mass=mb, inertia=tuple(Ib))],
                 [dict(type=S.CAPSULE, body=0, size=(r, h, 0)), dict(type=S.SPHERE, body=1, size=(r, 0, 0))])
    # the sphere sits just past the capsule's upper end, off its axis
    Ra = np.array([[np.cos(0.4), 0, np.sin(0.4)], [0, 1, 0], [-np.sin(0.4), 0, np.cos(0.4)]])
    end = Ra @ np.array([0, 0, h])
    off = np.array([0.6, 0.3, 0.75])
    off /= np.linalg.norm(off)
    xb = end + (2 * r - 0.003) * off
    q = np.concatenate([[0, 0, 1.0], qa, xb + [0, 0, 1.0], [1, 0, 0, 0]])
    v = np.zeros(12)
    rec = oracle.step_record(d, Wd.params(n_t=4, gravity=(0, 0, 0)), DT, q, v)
    c, = rec["contacts"]
    p = np.array(c["pos"])
    n = np.array(c["normal"])

    def delassus(m, I, R, x):
        lx = p - x
        K = np.array([[0, -lx[2], lx[1]], [lx[2], 0, -lx[0]], [-lx[1], lx[0], 0]])
        Iinv = R @ np.diag(1 / I) @ R.T
        return np.eye(3) / m + K @ Iinv @ K.T

    W = delassus(ma, Ia, Ra, np.array([0, 0, 1.0])) + delassus(mb, Ib, np.eye(3), xb + [0, 0, 1.0])
    tr = np.trace(W)
    phi = c["phi"]
    assert phi == pytest.approx(-0.003, abs=1e-12)
    x_exp = [max(-1.0, phi / 0.001), 1 - 3 * (1 / ma + 1 / mb) / tr, n @ W @ n / tr, 0.0]
    np.testing.assert_allclose(c["feat"], x_exp, rtol=1e-12, atol=1e-14)
    assert 0.0 < x_exp[1] < 1.0 and n @ W @ n > 1 / ma + 1 / mb


def test_features_of_a_hinged_link(oracle):
    """A link on a vertical hinge (anchor 0.3 m up, 1 kg, centre of mass 0.1 m out, I_zz =
    2e-3) carrying a sphere that touches the floor below its centre of mass.  Its point
    Jacobian is a x (p - anchor) = (0, 0.1, 0), so tr = 0.1^2 / (2e-3 + 1 * 0.1^2) = 5/6 and the
    rotational share 1 - 3 (1/m) / tr = -2.6 clamps to -1.  Taken as a free body the link's lever
    from its centre of mass is parallel to the normal: w_n = 1/m = 1, x2 = 1 / (5/6) = 1.2."""
    r = 0.02
    d = Wd.world([dict(parent=-1, jnt=S.HINGE, pos=(0, 0, 0.3), axis=(0, 0, 1), ipos=(0.1, 0, 0), mass=1.0,
                       inertia=(1e-3, 1e-3, 2e-3))],
                 [dict(type=S.PLANE, body=-1), dict(type=S.SPHERE, body=0, pos=(0.1, 0, -0.3 + r - 0.0002),
                                                    size=(r, 0, 0))])
    rec = oracle.step_record(d, Wd.params(n_t=4), DT, [0.0], [0.0])
    c, = rec["contacts"]
    tr = 0.01 / 0.012
    assert c["trace_a"] + c["trace_b"] == pytest.approx(tr, rel=1e-12)
    np.testing.assert_allclose(c["feat"], [-0.2, -1.0, 1.0 / tr, 1.0], rtol=1e-10, atol=1e-12)


def test_network_layout_against_a_hand_evaluation(oracle):
    """theta = [W1 (8 x 4, row-major), b1, w2, b2]: evaluation against numpy, and a sparse
    network worked by hand, g = 0.1 + 0.7 tanh(x0) - 0.4 tanh(0.3 + 2 x3)."""
    rng = np.random.default_rng(1)
    th = rng.normal(size=NP)
    x = rng.normal(size=(50, F))
    np.testing.assert_allclose(oracle.impnet_eval(th, x), g_by_hand(th, x), rtol=1e-13, atol=1e-13)
    W1 = np.zeros((H, F)); W1[0, 0] = 1.0; W1[1, 3] = 2.0
    b1 = np.zeros(H); b1[1] = 0.3
    w2 = np.zeros(H); w2[0] = 0.7; w2[1] = -0.4
    th = make_theta(W1, b1, w2, 0.1)
    for xi in x[:5]:
        exp = 0.1 + 0.7 * np.tanh(xi[0]) - 0.4 * np.tanh(0.3 + 2 * xi[3])
        assert oracle.impnet_eval(th, xi[None])[0] == pytest.approx(exp, rel=1e-14, abs=1e-15)


def test_learned_impedance_of_one_contact(oracle):
    """The learned mode scales M(phi) by exp(g(x)) at the contact's own features: with the
    sparse network above on the sphere of the feature pin, the recorded impedance is the
    heuristic M(phi) = r/(1-r)/tr times exp(0.1 + 0.7 tanh(x0) - 0.4 tanh(0.3 + 2)), and the
    resting sphere's normal impulse over its four active facets grows by the same factor."""
    m, r = 2.0, 0.05
    I = 0.4 * m * r * r
    d = Wd.sphere_on_plane(r=r, m=m, inertia=I)
    phi = -0.0004
    q, v = Wd.free_state((0, 0, r + phi))
    W1 = np.zeros((H, F)); W1[0, 0] = 1.0; W1[1, 3] = 2.0
    b1 = np.zeros(H); b1[1] = 0.3
    w2 = np.zeros(H); w2[0] = 0.7; w2[1] = -0.4
    th = make_theta(W1, b1, w2, 0.1)
    base = oracle.step_record(d, Wd.params(n_t=4), DT, q, v)["contacts"][0]
    lrn = oracle.step_record(d, Wd.params(n_t=4, trace_mode=3), DT, q, v, impnet=th)["contacts"][0]
    fac = np.exp(0.1 + 0.7 * np.tanh(-0.4) - 0.4 * np.tanh(2.3))
    assert base["mphi"] == pytest.approx(base["r"] / (1 - base["r"]) / (base["trace_a"] + base["trace_b"]), rel=1e-14)
    assert lrn["mphi"] == pytest.approx(fac * base["mphi"], rel=1e-13)
    assert base["nactive"] == lrn["nactive"] == 4
    assert lrn["lam_sum"] == pytest.approx(fac * base["lam_sum"], rel=1e-12)


def test_output_clamp(oracle):
    """|g| is clamped to 8 before the exponential (a bound on how far the learned impedance
    may move from the heuristic)."""
    d = Wd.sphere_on_plane()
    q, v = Wd.free_state((0, 0, 0.0496))
    base = oracle.step_record(d, Wd.params(n_t=4), DT, q, v)["contacts"][0]
    for b2, g in ((20.0, 8.0), (-30.0, -8.0)):
        lrn = oracle.step_record(d, Wd.params(n_t=4, trace_mode=3), DT, q, v, impnet=make_theta(b2=b2))["contacts"][0]
        assert lrn["mphi"] == pytest.approx(np.exp(g) * base["mphi"], rel=1e-13)


def test_mean_exact_impedance_of_a_sphere_by_hand(oracle):
    """The learning target's ingredient, the exact diagonal impedance of Sec. III-B averaged over
    the facets, for a sphere (m = 1, I = 1e-3, r = 0.05) 2 mm into a plane with the 6D cone
    (4 tangential, 2 torsional, 4 rolling facets).  The lever l (length 0.049) is parallel to n,
    so J_n = (n, 0) and the facet diagonals are: tangential 1/m + mu_t^2 (1/m + |l|^2 / I),
    torsional 1/m + mu_tor^2 / I, rolling 1/m + mu_rol^2 / I."""
    mu = (0.5, 0.01, 0.02)
    d = Wd.sphere_on_plane(mu=mu)
    q, v = Wd.free_state((0, 0, 0.048))
    p = Wd.params(n_t=4, n_tor=2, n_rol=4)
    c, = oracle.step_record(d, p, DT, q, v)["contacts"]
    kd = p.k_user * DT + p.d_user
    w = [1 + mu[0] ** 2 * (1 + 0.049 ** 2 / 1e-3)] * 4 + [1 + mu[1] ** 2 / 1e-3] * 2 + [1 + mu[2] ** 2 / 1e-3] * 4
    assert c["nfacet"] == 10
    assert c["m_exact"] == pytest.approx(np.mean([1 / (kd * wj) for wj in w]), rel=1e-12)
    # the same mean from the exact mode's own facet impulses: with k = 0 and a 1 m/s approach
    # every facet is active with lambda_j = -s_j / w_j, s_j = v_n
    q2, v2 = Wd.free_state((0, 0, 0.0499), lin=(0, 0, -1.0))
    p0 = Wd.params(n_t=4, n_tor=2, n_rol=4, k_user=0.0, trace_mode=2)
    c2, = oracle.step_record(d, p0, DT, q2, v2)["contacts"]
    s = -1.0 - G * DT
    w2 = [1 + mu[0] ** 2 * (1 + 0.04995 ** 2 / 1e-3)] * 4 + w[4:]
    assert c2["lam_sum"] == pytest.approx(sum(-s / wj for wj in w2), rel=1e-12)


def test_gradient_matches_central_differences(oracle):
    rng = np.random.default_rng(2)
    th = rng.normal(scale=0.7, size=NP)
    x = rng.uniform(-1, 1, size=(40, F))
    y = rng.normal(size=40)
    L, g = oracle.impnet_loss_grad(th, x, y)
    assert L == pytest.approx(np.mean((g_by_hand(th, x) - y) ** 2), rel=1e-13)
    h = 1e-6
    fd = np.array([(oracle.impnet_loss_grad(th + h * e, x, y)[0] - oracle.impnet_loss_grad(th - h * e, x, y)[0]) / (2 * h)
                   for e in np.eye(NP)])
    np.testing.assert_allclose(g, fd, rtol=1e-6, atol=1e-9)


def test_adam_first_step_and_descent(oracle):
    """Adam's first bias-corrected step is lr * g / (|g| + eps) per parameter (m^ = g, v^ = g^2);
    and full-batch Adam drives the loss of a target the network can represent far down."""
    rng = np.random.default_rng(3)
    th0 = rng.normal(scale=0.5, size=NP)
    x = rng.uniform(-1, 1, size=(200, F))
    y = g_by_hand(rng.normal(scale=0.8, size=NP), x)
    _, g = oracle.impnet_loss_grad(th0, x, y)
    th1, _ = oracle.impnet_adam(th0, x, y, 1, 0.01)
    np.testing.assert_allclose(th1, th0 - 0.01 * g / (np.abs(g) + 1e-8), rtol=1e-12, atol=1e-15)
    _, losses = oracle.impnet_adam(th0, x, y, 1500, 0.02)
    assert losses[-1] < 0.02 * losses[0]


def test_features_explain_the_exact_impedance_of_pile_contacts(oracle):
    """The learning problem itself, in FP64: targets ln(M_exact / M(phi)) and features of the
    contacts of jammed 64-body piles (spheres and capsules against each other and the bin),
    a fit by full-batch Adam on 12 worlds, and held-out worlds whose target spread the network
    explains almost entirely (the best constant explains none of it)."""
    def data(seed, n):
        sb = S.make_pile(n, 64, seed=seed, jammed=True)
        p = with_mode(sb.params, 2)
        X, y = [], []
        for w in range(n):
            for c in oracle.step_record(sb.world(w), p, sb.dt, sb.q0[w], sb.v0[w])["contacts"]:
                mh = c["r"] / (1 - c["r"]) / (c["trace_a"] + c["trace_b"])
                X.append(c["feat"])
                y.append(np.log(c["m_exact"] / mh))
        return np.array(X), np.array(y)

    X, y = data(41, 12)
    Xt, yt = data(42, 4)
    assert len(y) > 300 and len(yt) > 100 and y.std() > 0.1
    th0 = make_theta(W1=np.random.default_rng(0).normal(scale=0.5, size=(H, F)))
    th, losses = oracle.impnet_adam(th0, X, y, 2000, 0.02)
    r2 = 1 - np.mean((oracle.impnet_eval(th, Xt) - yt) ** 2) / np.mean((yt - y.mean()) ** 2)
    assert losses[-1] < 1e-3 * losses[0] and r2 > 0.9
