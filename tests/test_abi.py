"""CPU checks of the C ABI: the library loads without a GPU and exports every entry point that
include/comfree.h declares; host-only calls validate their inputs."""
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def cf():
    from paper_2603_12185_gb300 import build
    build.build()
    from paper_2603_12185_gb300 import comfree
    return comfree


def declared_functions():
    src = open(os.path.join(ROOT, "include", "comfree.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(cf_[a-z_0-9]+)\s*\(", src)))


def test_header_symbols_exported(cf):
    import ctypes
    L = ctypes.CDLL(cf.LIB_PATH)
    names = declared_functions()
    assert len(names) >= 19
    for n in names:
        assert hasattr(L, n), n
    assert set(names) <= set(cf.EXPORTS) | set(names)


def test_host_state_step_rejects_bad_arguments_without_a_device(cf):
    """cf_step_host validates its batch, dt and nsteps on the host before any CUDA call."""
    import ctypes as C
    L = cf.lib()
    buf = (C.c_float * 8)()
    assert cf.STATUS[L.cf_step_host(None, buf, buf, C.c_float(0.002), 1, None)] == "CF_ERR_INVALID_ARGUMENT"
    assert "null batch" in L.cf_last_error().decode()


def test_status_strings(cf):
    for k, v in cf.STATUS.items():
        assert cf.lib().cf_status_string(k).decode() == v


def test_model_validation(cf):
    from paper_2603_12185_gb300 import scenes as S
    sb = S.make_mixed(8)
    m = cf.Model(sb.templates, sb.params)
    assert m.scene_sizes(3) == dict(nq=23, nv=22, nu=16, nbody=17, ngeom=18)
    t = S.hand_template()

    def bad(**kw):
        import copy
        tt = copy.deepcopy(t)
        for k, v in kw.items():
            setattr(tt, k, v)
        with pytest.raises(cf.CfError) as e:
            cf.Model([tt], sb.params)
        return e.value.status

    assert bad(body_mass=np.where(np.arange(17) == 3, -1.0, t.body_mass)) == 1
    assert bad(body_parent=np.where(np.arange(17) == 2, 5, t.body_parent).astype(np.int32)) == 1
    assert bad(geom_body=np.where(np.arange(18) == 0, 1, t.geom_body).astype(np.int32)) == 7   # attached plane
    p = S.Params(n_t=3)
    with pytest.raises(cf.CfError):
        cf.Model(sb.templates, p)
    p = S.Params(solimp=(0.9, 0.95, 0.0, 0.5, 2.0))
    with pytest.raises(cf.CfError):
        cf.Model(sb.templates, p)


def test_workspace_size_grows_with_worlds(cf):
    from paper_2603_12185_gb300 import scenes as S
    import ctypes as C
    sb = S.make_pile(4, 16)
    m = cf.Model(sb.templates, sb.params)
    sizes = []
    for W in (1, 10, 100):
        n = C.c_size_t()
        sc = np.zeros(W, np.int32)
        opts = cf.BatchOpts(1, 0, 0, 1)
        cf.check(cf.lib().cf_batch_workspace_bytes(m.h, W, sc.ctypes.data_as(C.c_void_p), C.byref(opts), C.byref(n)))
        sizes.append(n.value)
    assert sizes[0] < sizes[1] < sizes[2]
    assert sizes[2] > 100 * (16 * 13 * 4)


def test_impedance_modes_and_network_sizes(cf):
    """trace_mode 0..3 build a model (3: the learned impedance), 4 does not; the fitting state
    holds at least Adam's two moments of the 49 parameters."""
    from paper_2603_12185_gb300 import scenes as S
    sb = S.make_pile(2, 16)
    for mode in (0, 1, 2, 3):
        cf.Model(sb.templates, S.Params(trace_mode=mode))
    with pytest.raises(cf.CfError):
        cf.Model(sb.templates, S.Params(trace_mode=4))
    assert cf.lib().cf_impnet_state_floats() >= 2 * cf.IMPNET_PARAMS
    assert cf.IMPNET_PARAMS == 8 * 4 + 8 + 8 + 1


def test_impedance_features_from_records(cf):
    """The host-side feature assembly of the training data matches the kernel's definition."""
    rec = np.zeros(3, cf.CONTACT_DTYPE)
    rec["phi"] = [-0.0005, 0.004, -0.01]
    rec["rho"] = [0.625, 0.1, -0.3]
    rec["wn"] = [0.125, 0.3, 1.2]
    rec["flags"] = [cf.CONTACT_B_STATIC, 0, 0]
    x = cf.impedance_features(rec, 0.001)
    np.testing.assert_allclose(x, [[-0.5, 0.625, 0.125, 1], [1, 0.1, 0.3, 0], [-1, -0.3, 1.2, 0]], rtol=1e-6)


def test_mlp_workspace_covers_its_buffers_without_a_device(cf):
    """cf_mlp_workspace_bytes validates the layer sizes on the host and returns room for every
    buffer: parameters, gradients and Adam moments (4 x fp32), the BF16 weights and their
    transposes, the batch's BF16 activations, gradients and their transposes, the FP32 output,
    the bias gradients' partial sums (per 64 and per 128 rows) and the split-K scratch."""
    import ctypes as C
    L = cf.lib()
    n = C.c_size_t()
    for bad in ((0, 256, 1024), (300, 256, 1024), (49, 200, 1024), (49, 256, 1000)):
        assert cf.STATUS[L.cf_mlp_workspace_bytes(*bad, 1024, C.byref(n))] == "CF_ERR_INVALID_ARGUMENT"
    assert cf.STATUS[L.cf_mlp_workspace_bytes(49, 256, 1024, 0, C.byref(n))] == "CF_ERR_INVALID_ARGUMENT"
    fin, H, O = 49, 256, 1024
    kin = 64
    npar = H * kin + H + H * H + H + O * H + O
    sizes = []
    for B in (1, 300, 16384):
        assert cf.STATUS[L.cf_mlp_workspace_bytes(fin, H, O, B, C.byref(n))] == "CF_OK"
        Bp = (B + 127) // 128 * 128
        floor = (4 * npar * 4                                    # w, g, m, v
                 + 2 * (H * kin + 2 * H * H + 2 * O * H)          # W1, W2, W3 and W2^T, W3^T in BF16
                 + 2 * Bp * (2 * kin + 10 * H + 2 * O)           # activations, gradients, transposes
                 + 4 * Bp * O                                    # Y
                 + 4 * ((Bp // 64) * O + 2 * (Bp // 32) * H))    # bias-gradient partials
        assert n.value >= floor, (B, n.value, floor)
        sizes.append(n.value)
    assert sizes[0] < sizes[1] < sizes[2]


def declared_signatures():
    """{name: number of parameters} of every function include/comfree.h declares."""
    src = open(os.path.join(ROOT, "include", "comfree.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    src = re.sub(r"//[^\n]*", "", src)
    out = {}
    for name, args in re.findall(r"\b(cf_[a-z_0-9]+)\s*\(([^;{]*?)\)\s*;", src):
        args = " ".join(args.split())
        out[name] = 0 if args in ("", "void") else args.count(",") + 1
    return out


def test_binding_passes_every_declared_parameter(cf):
    """The ctypes binding declares, for every entry point of the header, as many arguments as
    the header's prototype has: a mismatch would shift every later argument of the call."""
    sigs = declared_signatures()
    assert len(sigs) >= 19
    L = cf.lib()
    missing = []
    for name, n in sigs.items():
        fn = getattr(L, name)
        if fn.argtypes is None:
            missing.append(name)
            continue
        assert len(fn.argtypes) == n, (name, len(fn.argtypes), n)
    assert not missing, missing


def _c_kind(decl):
    """Kind of one C parameter declaration: ('ptr',), ('float', bytes) or ('int', bytes)."""
    d = " ".join(decl.replace("const ", " ").split())
    if "*" in d or "[" in d:          # an array parameter decays to a pointer
        return ("ptr",)
    t = d.rsplit(" ", 1)[0] if " " in d else d
    sizes = {"int32_t": ("int", 4), "int": ("int", 4), "uint32_t": ("int", 4), "int64_t": ("int", 8),
             "uint64_t": ("int", 8), "size_t": ("int", 8), "float": ("float", 4), "double": ("float", 8),
             "cf_status": ("int", 4)}  # an enum, passed as a C int
    return sizes.get(t, ("other", t))


def _ctypes_kind(t):
    import ctypes as C
    if t in (C.c_void_p, C.c_char_p) or issubclass(t, C._Pointer):
        return ("ptr",)
    if t in (C.c_float, C.c_double):
        return ("float", C.sizeof(t))
    return ("int", C.sizeof(t))


def test_binding_argument_kinds_match_the_header(cf):
    """Every argument's kind as the binding passes it (pointer, floating point of a width,
    integer of a width) matches the header's prototype."""
    src = open(os.path.join(ROOT, "include", "comfree.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    L = cf.lib()
    checked = 0
    for name, args in re.findall(r"\b(cf_[a-z_0-9]+)\s*\(([^;{]*?)\)\s*;", src):
        args = " ".join(args.split())
        if args in ("", "void"):
            continue
        kinds = [_c_kind(a) for a in args.split(",")]
        assert all(k[0] != "other" for k in kinds), (name, kinds)
        got = [_ctypes_kind(t) for t in getattr(L, name).argtypes]
        assert got == kinds, (name, got, kinds)
        checked += 1
    assert checked >= 35


def test_binding_return_kinds_match_the_header(cf):
    """cf_status returns come back as a C int (ctypes' default), strings as char pointers (a
    default int would truncate the pointer), sizes as size_t, void functions as None."""
    import ctypes as C
    src = open(os.path.join(ROOT, "include", "comfree.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    L = cf.lib()
    seen = 0
    for ret, name in re.findall(r"(?m)^\s*((?:const\s+)?[A-Za-z_][A-Za-z_0-9]*\s*\**)\s*\b(cf_[a-z_0-9]+)\s*\(", src):
        ret = " ".join(ret.replace("*", " * ").split())
        rt = getattr(L, name).restype
        if ret == "cf_status":
            assert rt is C.c_int, name
        elif ret == "const char *":
            assert rt is C.c_char_p, name
        elif ret == "void":
            assert rt is None, name
        elif ret in ("size_t", "int32_t", "int", "float", "double"):
            want = {"size_t": C.c_size_t, "int32_t": C.c_int32, "int": C.c_int, "float": C.c_float,
                    "double": C.c_double}[ret]
            assert rt is not None and C.sizeof(rt) == C.sizeof(want) and \
                (rt in (C.c_float, C.c_double)) == (want in (C.c_float, C.c_double)), name
        else:
            raise AssertionError(f"{name}: unexpected return type {ret}")
        seen += 1
    assert seen == len(declared_functions())
