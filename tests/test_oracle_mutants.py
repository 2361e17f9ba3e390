"""Mutation check of the oracle's pins.

Each entry of MUTANTS plants one plausible mistake in a copy of oracle/oracle.cpp: a dropped
term, a wrong sign, a transposed operand or index, a quantity taken in the wrong frame.  The
copy is built into a temporary library, and the pins of test_oracle_pins.py and
test_oracle_impedance_net.py run against it.  For every mutant at least one pin must fail: a
mutant that passes them all marks a part of the oracle that nothing outside it fixes.  The
oracle's own source and library are not touched.

The table lists (what the mistake is, the exact text it replaces, the text put in its place);
the text must occur exactly once in oracle.cpp, so that an edit of the oracle cannot silently
turn a mutant into a copy of the original.
"""
import concurrent.futures as cf
import importlib.util
import inspect
import os
import re

import numpy as np
import pytest

from oracle import oracle as O

HERE = os.path.dirname(os.path.abspath(__file__))
SOURCE = os.path.join(os.path.dirname(HERE), "oracle", "oracle.cpp")
PIN_MODULES = ("test_oracle_pins", "test_oracle_impedance_net")
SLOW = ("brute_force",)  # dense sampling: tried only when every other pin passes
SELF = ("batch_runner_equals",)  # compare the oracle with itself: no mutant can fail them

MUTANTS = [
    # the smooth prediction, Eq. smooth_vel, and the velocity correction, Eq. vel_correction
    ("smooth prediction drops the bias forces c",
     "vs[i] = (tau ? tau[i] : S(0.0)) - c[i] - damp[i] * v[i];",
     "vs[i] = (tau ? tau[i] : S(0.0)) - damp[i] * v[i];"),
    ("joint damping with the wrong sign",
     "vs[i] = (tau ? tau[i] : S(0.0)) - c[i] - damp[i] * v[i];",
     "vs[i] = (tau ? tau[i] : S(0.0)) - c[i] + damp[i] * v[i];"),
    ("implicit damping added to M without dt",
     "L[t][(size_t)i * n + i] += DT * damp[st.tree_dofs[t][i]];",
     "L[t][(size_t)i * n + i] += damp[st.tree_dofs[t][i]];"),
    ("smooth prediction without dt",
     "vs[i] = v[i] + vs[i] * DT;",
     "vs[i] = v[i] + vs[i];"),
    ("velocity correction added to v instead of v_s",
     "v[i] = vs[i] + dv[i];",
     "v[i] = v[i] + dv[i];"),
    # the impulse law, Eq. cf_wrench, and the facet rows, Eqs. dual_polyhedral and tilde_defs
    ("impulse law: damping term with the wrong sign",
     "lam = -kM * (sv * DT + k.phi) - dM * sv;",
     "lam = -kM * (sv * DT + k.phi) + dM * sv;"),
    ("impulse law: gap term without dt",
     "lam = -kM * (sv * DT + k.phi) - dM * sv;",
     "lam = -kM * (sv + k.phi) - dM * sv;"),
    ("facet row: friction part with the wrong sign",
     "Jf[i] = Jn[i] - mu[sub] * dj;",
     "Jf[i] = Jn[i] + mu[sub] * dj;"),
    ("facet row: friction coefficient dropped",
     "Jf[i] = Jn[i] - mu[sub] * dj;",
     "Jf[i] = Jn[i] - dj;"),
    ("torsional row from the linear point Jacobian",
     "row(Ja, k.n, Jtor);",
     "row(Jl, k.n, Jtor);"),
    ("rolling rows with t1 and t2 swapped",
     "row(Ja, t1, Jr1); row(Ja, t2, Jr2);",
     "row(Ja, t2, Jr1); row(Ja, t1, Jr2);"),
    ("tangential wrench record with the wrong sign",
     "if (sub == 0) { wrench[1] -= mu[0] * ca * lam; wrench[2] -= mu[0] * sa_ * lam; }",
     "if (sub == 0) { wrench[1] += mu[0] * ca * lam; wrench[2] += mu[0] * sa_ * lam; }"),
    ("torsional facets both along +n",
     "facet(1, S(j % 2 == 0 ? 1.0 : -1.0), S(0.0));",
     "facet(1, S(1.0), S(0.0));"),
    ("tangential facet directions over half the circle",
     "double th = 2.0 * M_PI * j / prm->n_t;",
     "double th = M_PI * j / prm->n_t;"),
    ("pair friction: the smaller coefficient",
     "mu[i] = S(std::max(w->geom_mu[3 * ga + i], w->geom_mu[3 * gb + i]));",
     "mu[i] = S(std::min(w->geom_mu[3 * ga + i], w->geom_mu[3 * gb + i]));"),
    # the impedance: Eqs. k_d_setting and r_scaling, the exact form of Sec. III-B, joint limits
    ("trace without M~^-1",
     "for (int i = 0; i < st.nv; ++i) trace[side] += jl[r][i] * tmp[i];",
     "for (int i = 0; i < st.nv; ++i) trace[side] += jl[r][i] * jl[r][i];"),
    ("M(phi) with body A's trace only",
     "S mphi = r / (S(1.0) - r) / (trace[0] + trace[1]);",
     "S mphi = r / (S(1.0) - r) / trace[0];"),
    ("M(phi) with r/(1-r) inverted",
     "S mphi = r / (S(1.0) - r) / (trace[0] + trace[1]);",
     "S mphi = (S(1.0) - r) / r / (trace[0] + trace[1]);"),
    ("r(|phi|): first branch without its factor m",
     "S g = x < m ? m * pow(x / m, si[4])",
     "S g = x < m ? pow(x / m, si[4])"),
    ("r(|phi|): second branch without its factor (1 - m)",
     ": S(1.0) - (S(1.0) - m) * pow((S(1.0) - x) / (S(1.0) - m), si[4]);",
     ": S(1.0) - pow((S(1.0) - x) / (S(1.0) - m), si[4]);"),
    ("exact impedance without dt",
     "Mj = S(1.0) / ((S(prm->k_user) * DT + S(prm->d_user)) * wj);",
     "Mj = S(1.0) / ((S(prm->k_user) + S(prm->d_user)) * wj);"),
    ("exact impedance: facet diagonal without M~^-1",
     "for (int i = 0; i < st.nv; ++i) wj += Jf[i] * tmp[i];",
     "for (int i = 0; i < st.nv; ++i) wj += Jf[i] * Jf[i];"),
    ("joint limit impulse with the lower limit's sign at both ends",
     "if (lam > S(0.0)) pgen[kd] += sgn * lam;",
     "if (lam > S(0.0)) pgen[kd] += lam;"),
    ("joint limit: impedance over M~ instead of M~^-1",
     "Mk = r / (S(1.0) - r) / wkk;",
     "Mk = r / (S(1.0) - r) * wkk;"),
    ("dry joint friction capped at f instead of f dt",
     "const S cap = S(fl) * DT;",
     "const S cap = S(fl);"),
    ("learned impedance: rotational-share feature without its factor 3",
     "x[1] = clampv(S(1.0) - S(3.0 * im_sum) / trace_sum, S(-1.0), S(1.0));",
     "x[1] = clampv(S(1.0) - S(im_sum) / trace_sum, S(-1.0), S(1.0));"),
    ("learned impedance: hidden units without their bias",
     "S a(b1[h]);",
     "S a(0.0);"),
    ("learned impedance: gap feature not scaled by the solimp width",
     "x[0] = clampv(phi / S(width), S(-1.0), S(1.0));",
     "x[0] = clampv(phi, S(-1.0), S(1.0));"),
    ("learned impedance: normal-row feature clamped at 1 instead of 4",
     "x[2] = clampv(w_n / trace_sum, S(0.0), S(4.0));",
     "x[2] = clampv(w_n / trace_sum, S(0.0), S(1.0));"),
    ("learned impedance: static-side flag inverted",
     "x[3] = S(b_static ? 1.0 : 0.0);",
     "x[3] = S(b_static ? 0.0 : 1.0);"),
    ("learned impedance: free-body lever from the body origin instead of the centre of mass",
     "V3<S> u = mulT(P[b].R, cross(p - P[b].com, n));",
     "V3<S> u = mulT(P[b].R, cross(p - P[b].x, n));"),
    ("learned impedance: network output not clamped",
     "if (prm->trace_mode == 3) mphi *= exp(clampv(impnet_g(prm->impnet, feat), S(-IMP_CLAMP), S(IMP_CLAMP)));",
     "if (prm->trace_mode == 3) mphi *= exp(impnet_g(prm->impnet, feat));"),
    ("learned impedance: hidden units linear instead of tanh",
     "g += S(w2[h]) * tanh(a);",
     "g += S(w2[h]) * a;"),
    # the contact frame
    ("left-handed contact frame",
     "t2 = cross(n, t1);",
     "t2 = cross(t1, n);"),
    ("tangent rule: helper axes swapped at |n_z| = 0.5",
     "V3<S> a = fabs(n.z) < S(0.5) ? V3<S>(S(0.0), S(0.0), S(1.0)) : V3<S>(S(1.0), S(0.0), S(0.0));",
     "V3<S> a = fabs(n.z) < S(0.5) ? V3<S>(S(1.0), S(0.0), S(0.0)) : V3<S>(S(0.0), S(0.0), S(1.0));"),
    ("tangent rule without normalisation",
     "t1 = (S(1.0) / norm(c)) * c;",
     "t1 = c;"),
    # integration (semi-implicit Euler, exponential map of the body-frame angular velocity)
    ("orientation update composed in the world frame",
     "quat_mul(qb + 3, dq, nq);",
     "quat_mul(dq, qb + 3, nq);"),
    ("orientation update by the full angle",
     "S half = S(0.5) * wn * DT;",
     "S half = wn * DT;"),
    ("position integrated with the smooth velocity",
     "for (int i = 0; i < 3; ++i) qb[i] += vb[i] * DT;",
     "for (int i = 0; i < 3; ++i) qb[i] += vs[st.vadr[b] + i] * DT;"),
    # rigid-body dynamics: kinematics, Jacobians, inertia, bias forces, factorisation
    ("gyroscopic term with the wrong sign",
     "V3<S> gyro = cross(wb, Iw);",
     "V3<S> gyro = cross(Iw, wb);"),
    ("free-body gravity with the wrong sign",
     "for (int i = 0; i < 3; ++i) c[d + i] = -m * comp(g, i);",
     "for (int i = 0; i < 3; ++i) c[d + i] = m * comp(g, i);"),
    ("hinge rotation applied before the fixed frame",
     "o.R = mul(Rfix, axis_angle(ax, q[st.qadr[b]]));",
     "o.R = mul(axis_angle(ax, q[st.qadr[b]]), Rfix);"),
    ("hinge anchor offset not rotated by the parent",
     "o.x = xp + mul(Rp, vload<S>(w->body_pos + 3 * b));",
     "o.x = xp + vload<S>(w->body_pos + 3 * b);"),
    ("hinge axis taken in the parent frame",
     "o.axis = mul(Rfix, ax);",
     "o.axis = mul(Rp, ax);"),
    ("hinge Jacobian column with the wrong sign",
     "V3<S> lin = cross(P[a].axis, p - P[a].x);",
     "V3<S> lin = cross(p - P[a].x, P[a].axis);"),
    ("free-body Jacobian lever with the wrong sign",
     "V3<S> lin = cross(c, rp);",
     "V3<S> lin = cross(rp, c);"),
    ("free-body angular Jacobian with R^T in place of R",
     "Ja[r][d + 3 + i] = comp(c, r);",
     "Ja[r][d + 3 + i] = comp(P[a].R.col(r), i);"),
    ("world inertia R^T I R instead of R I R^T",
     "s += P[b].R.m[3 * i + k] * S(w->body_inertia[3 * b + k]) * P[b].R.m[3 * j + k];",
     "s += P[b].R.m[3 * k + i] * S(w->body_inertia[3 * b + k]) * P[b].R.m[3 * k + j];"),
    ("Newton-Euler: joint-rate coupling in the angular acceleration dropped",
     "omd[b] = omdp + cross(omp, qd * P[b].axis);",
     "omd[b] = omdp;"),
    ("Newton-Euler: centripetal term of the anchor dropped",
     "V3<S> aanchor = p >= 0 ? ap + cross(omdp, ro) + cross(omp, cross(omp, ro)) : ap;",
     "V3<S> aanchor = p >= 0 ? ap + cross(omdp, ro) : ap;"),
    ("Cholesky diagonal from the unfactored upper triangle",
     "for (int k = 0; k < j; ++k) s -= A[(size_t)j * n + k] * A[(size_t)j * n + k];",
     "for (int k = 0; k < j; ++k) s -= A[(size_t)k * n + j] * A[(size_t)k * n + j];"),
    ("back substitution with L in place of L^T",
     "for (int k = i + 1; k < n; ++k) s -= L[(size_t)k * n + i] * x[k];",
     "for (int k = i + 1; k < n; ++k) s -= L[(size_t)i * n + k] * x[k];"),
    # narrowphase
    ("sphere-sphere normal from A to B",
     "V3<S> d = ca - cb;\n  S dist = norm(d);",
     "V3<S> d = cb - ca;\n  S dist = norm(d);"),
    ("sphere-plane point on the sphere's surface instead of the midpoint",
     "V3<S> sa = c - r * nz, sb = c - dist * nz;",
     "V3<S> sa = c - r * nz, sb = c - r * nz;"),
    ("sphere-box: centre inside takes the far face",
     "S sg = lc[k] >= S(0.0) ? S(1.0) : S(-1.0);",
     "S sg = lc[k] >= S(0.0) ? S(-1.0) : S(1.0);"),
    ("segment-segment: second parameter with the wrong sign of f",
     "t = (b * s + f) / e;\n  if (t < zero)",
     "t = (b * s - f) / e;\n  if (t < zero)"),
    ("capsule-plane: both end spheres at the same end",
     "sphere_plane(G[ga].c + S(sa[1]) * axa, S(sa[0]), o, nz, raw);",
     "sphere_plane(G[ga].c - S(sa[1]) * axa, S(sa[0]), o, nz, raw);"),
    ("box-plane corners: one half extent used twice",
     "V3<S> corner = G[ga].c + mul(G[ga].R, V3<S>(S(cx * sa[0]), S(cy * sa[1]), S(cz * sa[2])));",
     "V3<S> corner = G[ga].c + mul(G[ga].R, V3<S>(S(cx * sa[0]), S(cy * sa[1]), S(cz * sa[1])));"),
    ("box-box: reference axis of greatest overlap",
     "if (k == 0 || sep > best_sep) { best_sep = sep; best = k; }",
     "if (k == 0 || sep < best_sep) { best_sep = sep; best = k; }"),
    ("box-box: incident face on the far side of the incident box",
     "const S si = dot(RI.col(ji), nR) > S(0.0) ? S(-1.0) : S(1.0);",
     "const S si = dot(RI.col(ji), nR) > S(0.0) ? S(1.0) : S(-1.0);"),
    ("box-box: contact point at the clipped vertex instead of the midpoint",
     "k.p = poly[v] - (S(0.5) * dist) * nR;",
     "k.p = poly[v];"),
    ("ellipsoid support point with D instead of D^2",
     "const V3<S> pl(e.x * dn.x / len, e.y * dn.y / len, e.z * dn.z / len);",
     "const V3<S> pl(dn.x / len, dn.y / len, dn.z / len);"),
    ("cylinder rim points from the highest direction",
     "V3<S> w = -(n - dot(n, u) * u);",
     "V3<S> w = (n - dot(n, u) * u);"),
    ("sphere-cylinder: centre inside leaves through the deeper surface",
     "if (side <= cap) {",
     "if (side >= cap) {"),
    # the MPC cost of Sec. V and the dual numbers of the reference gradient
    ("MPC cost: fingertip at the capsule centre",
     "const V3<double> tip = centre + w->geom_size[3 * g + 1] * Rg.col(2);",
     "const V3<double> tip = centre;"),
    ("MPC cost: orientation term 1 - q*.q without the square",
     "const double c_quat = 1.0 - align * align;",
     "const double c_quat = 1.0 - align;"),
    ("dual numbers: product rule drops a term",
     "return Dual(a.v * b.v, a.d * b.v + a.v * b.d);",
     "return Dual(a.v * b.v, a.d * b.v);"),
    ("dual numbers: square-root derivative without the 1/2",
     "return Dual(s, s > 0 ? a.d / (2 * s) : 0.0);",
     "return Dual(s, s > 0 ? a.d / s : 0.0);"),
]

IDS = ["-".join(re.findall(r"[a-z0-9]+", name.lower())[:9]) for name, _, _ in MUTANTS]

# what a failing pin raises: a failed check, or the oracle refusing the step it was given
FAILURES = (AssertionError, RuntimeError, ArithmeticError, np.linalg.LinAlgError)


def _cases(mod):
    """(name, function, keyword arguments) for every test of a pin module, its parametrize
    marks expanded; every pin takes the `oracle` fixture and its parameters only."""
    out = []
    for name, fn in inspect.getmembers(mod, inspect.isfunction):
        if not name.startswith("test_") or fn.__module__ != mod.__name__:
            continue
        combos = [{}]
        for mark in [m for m in getattr(fn, "pytestmark", []) if m.name == "parametrize"]:
            names = mark.args[0]
            names = [n.strip() for n in names.split(",")] if isinstance(names, str) else list(names)
            grown = []
            for c in combos:
                for val in mark.args[1]:
                    val = tuple(val.values) if hasattr(val, "values") else ((val,) if len(names) == 1 else tuple(val))
                    grown.append({**c, **dict(zip(names, val))})
            combos = grown
        for c in combos:
            assert set(inspect.signature(fn).parameters) == {"oracle"} | set(c), f"{name} needs another fixture"
            out.append((name, fn, c))
    return out


def _first_failure(cases):
    for name, fn, kw in cases:
        try:
            fn(oracle=O, **kw)
        except FAILURES as e:
            return f"{name}{kw or ''}: {type(e).__name__}"
    return None


@pytest.fixture(scope="module")
def pins():
    cases = []
    for mod_name in PIN_MODULES:
        spec = importlib.util.spec_from_file_location("mutation_" + mod_name, os.path.join(HERE, mod_name + ".py"))
        mod = importlib.util.module_from_spec(spec)
        spec.loader.exec_module(mod)
        cases += [c for c in _cases(mod) if not any(k in c[0] for k in SELF)]
    slow = [c for c in cases if any(k in c[0] for k in SLOW)]
    return [c for c in cases if c not in slow], slow


@pytest.fixture(scope="module")
def libraries(tmp_path_factory):
    """The unmutated copy (key -1) and every mutant, built in parallel with the same flags."""
    src = open(SOURCE).read()
    out_dir = tmp_path_factory.mktemp("oracle_mutants")

    def build(i):
        text = src if i < 0 else src.replace(MUTANTS[i][1], MUTANTS[i][2])
        path = os.path.join(out_dir, f"mutant{i + 1}.cpp")
        with open(path, "w") as f:
            f.write(text)
        return i, O.compile_source(path, os.path.join(out_dir, f"libmutant{i + 1}.so"), opt="-O1")

    with cf.ThreadPoolExecutor(max(2, os.cpu_count() or 2)) as ex:
        return dict(ex.map(build, range(-1, len(MUTANTS))))


def test_every_mutant_changes_exactly_one_place():
    src = open(SOURCE).read()
    for name, old, new in MUTANTS:
        assert old != new, name
        assert src.count(old) == 1, f"{name}: the replaced text occurs {src.count(old)} times"
    assert len(set(IDS)) == len(IDS)


def test_the_pins_pass_on_an_unmutated_copy(libraries, pins, monkeypatch):
    """The harness itself: built the same way but unchanged, the copy passes every fast pin, so a
    failure below comes from the planted mistake."""
    monkeypatch.setattr(O, "_lib", O.load(libraries[-1]))
    assert _first_failure(pins[0]) is None


@pytest.mark.parametrize("i", range(len(MUTANTS)), ids=IDS)
def test_a_pin_catches_the_mutant(i, libraries, pins, monkeypatch):
    monkeypatch.setattr(O, "_lib", O.load(libraries[i]))
    fast, slow = pins
    caught = _first_failure(fast) or _first_failure(slow)
    assert caught, f"no pin fails with the oracle mutated: {MUTANTS[i][0]}"


# ------------------------------------------------------------------------------------------
# the MLP oracle (oracle/mlp.py) against the pins of test_mlp_oracle.py.  Its BF16 rounding
# points mirror what the tensor-core kernels store and have no CPU pin: only the GPU
# comparison fixes them, so no mutant moves one.
# ------------------------------------------------------------------------------------------
MLP_SOURCE = os.path.join(os.path.dirname(HERE), "oracle", "mlp.py")

MLP_MUTANTS = [
    ("BF16 rounding ties away from zero",
     "u = (u + 0x7FFF + lsb) & 0xFFFF0000",
     "u = (u + 0x8000) & 0xFFFF0000"),
    ("BF16 rounding by truncation",
     "u = (u + 0x7FFF + lsb) & 0xFFFF0000",
     "u = u & 0xFFFF0000"),
    ("GELU with erf(z / 2)",
     "return 0.5 * z * (1.0 + _erf(z / math.sqrt(2.0)))",
     "return 0.5 * z * (1.0 + _erf(z / 2.0))"),
    ("GELU derivative without the density term",
     "return 0.5 * (1.0 + _erf(z / math.sqrt(2.0))) + z * np.exp(-0.5 * z * z) / math.sqrt(2.0 * math.pi)",
     "return 0.5 * (1.0 + _erf(z / math.sqrt(2.0)))"),
    ("first layer without its bias",
     'Z1 = X0 @ W1.T + P["b1"]',
     "Z1 = X0 @ W1.T"),
    ("second layer without its bias",
     'Z2 = H1 @ W2.T + P["b2"]',
     "Z2 = H1 @ W2.T"),
    ("second layer fed the first layer's pre-activation",
     'Z2 = H1 @ W2.T + P["b2"]',
     'Z2 = Z1 @ W2.T + P["b2"]'),
    ("a GELU on the output layer",
     'Y = H2 @ W3.T + P["b3"]',
     'Y = gelu(H2 @ W3.T + P["b3"])'),
    ("log-std not clamped",
     "s = np.clip(sr, lo, hi)",
     "s = sr"),
    ("NLL with exp(-s) for the inverse variance",
     "iv = np.exp(-2.0 * s)",
     "iv = np.exp(-s)"),
    ("NLL averaged over samples only",
     "n = a.shape[0] * D",
     "n = a.shape[0]"),
    ("NLL mean gradient with the wrong sign",
     "dY[:, :D] = -e * iv / n",
     "dY[:, :D] = e * iv / n"),
    ("gradient flows through the clamped log-std",
     "dY[:, D:] = np.where((sr > lo) & (sr < hi), (1.0 - e * e * iv) / n, 0.0)",
     "dY[:, D:] = (1.0 - e * e * iv) / n"),
    ("output weights' gradient from the first hidden layer",
     'g = {"W3": dY.T @ c["H2"], "b3": dY.sum(0)}',
     'g = {"W3": dY.T @ c["H1"], "b3": dY.sum(0)}'),
    ("second layer's GELU derivative at the first layer's pre-activation",
     'dA2 = r((dY @ c["W3"]) * gelu_grad(c["Z2"]))',
     'dA2 = r((dY @ c["W3"]) * gelu_grad(c["Z1"]))'),
    ("back-propagation through W2 transposed",
     'dA1 = r((dA2 @ c["W2"]) * gelu_grad(c["Z1"]))',
     'dA1 = r((dA2 @ c["W2"].T) * gelu_grad(c["Z1"]))'),
    ("first bias gradient averaged instead of summed",
     'g["W1"], g["b1"] = dA1.T @ c["X0"], dA1.sum(0)',
     'g["W1"], g["b1"] = dA1.T @ c["X0"], dA1.mean(0)'),
]

MLP_IDS = ["-".join(re.findall(r"[a-z0-9]+", name.lower())[:9]) for name, _, _ in MLP_MUTANTS]


def _mlp_module(text, name):
    spec = importlib.util.spec_from_loader(name, loader=None)
    mod = importlib.util.module_from_spec(spec)
    exec(compile(text, MLP_SOURCE, "exec"), mod.__dict__)
    return mod


@pytest.fixture(scope="module")
def mlp_pins():
    spec = importlib.util.spec_from_file_location("mutation_test_mlp_oracle", os.path.join(HERE, "test_mlp_oracle.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    cases = []
    for name, fn in inspect.getmembers(mod, inspect.isfunction):
        if not name.startswith("test_") or fn.__module__ != mod.__name__:
            continue
        marks = [m for m in getattr(fn, "pytestmark", []) if m.name == "parametrize"]
        assert len(marks) <= 1 and (not marks or isinstance(marks[0].args[0], str) and "," not in marks[0].args[0])
        for val in (marks[0].args[1] if marks else [None]):
            cases.append((name, fn, {} if val is None else {marks[0].args[0]: val}))
    return mod, cases


def _mlp_first_failure(mod, cases, mlp, monkeypatch):
    monkeypatch.setattr(mod, "M", mlp)
    for name, fn, kw in cases:
        try:
            fn(**kw)
        except FAILURES as e:
            return f"{name}{kw or ''}: {type(e).__name__}"
    return None


def test_every_mlp_mutant_changes_exactly_one_place():
    src = open(MLP_SOURCE).read()
    for name, old, new in MLP_MUTANTS:
        assert old != new, name
        assert src.count(old) == 1, f"{name}: the replaced text occurs {src.count(old)} times"
    assert len(set(MLP_IDS)) == len(MLP_IDS)


def test_the_mlp_pins_pass_on_an_unmutated_copy(mlp_pins, monkeypatch):
    mod, cases = mlp_pins
    assert _mlp_first_failure(mod, cases, _mlp_module(open(MLP_SOURCE).read(), "mlp_copy"), monkeypatch) is None


@pytest.mark.parametrize("i", range(len(MLP_MUTANTS)), ids=MLP_IDS)
def test_a_pin_catches_the_mlp_mutant(i, mlp_pins, monkeypatch):
    name, old, new = MLP_MUTANTS[i]
    mod, cases = mlp_pins
    mutant = _mlp_module(open(MLP_SOURCE).read().replace(old, new), f"mlp_mutant{i}")
    caught = _mlp_first_failure(mod, cases, mutant, monkeypatch)
    assert caught, f"no pin fails with the MLP oracle mutated: {name}"
