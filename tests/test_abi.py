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
