"""The C-ABI library builds, loads and exports every symbol include/shacsim.h
declares (no GPU needed: no compute call is made)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def header_functions():
    src = open(os.path.join(ROOT, "include", "shacsim.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(shac_[a-z_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_2204_07137_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = header_functions()
    for n in ("shac_model_create", "shac_batch_create", "shac_step", "shac_step_adjoint", "shac_window_forward",
              "shac_window_adjoint", "shac_get_status"):
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in header_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_lists_every_declared_symbol():
    from paper_2204_07137_gb300 import _lib
    assert sorted(_lib.EXPORTED) == header_functions()


def test_model_validation_on_host(lib):
    """shac_model_create validates on the host (no device work)."""
    import numpy as np
    from paper_2204_07137_gb300 import _lib, inputs as I
    _lib.load()
    h = _lib.ModelHandle(I.ant())
    assert (h.nq, h.nv, h.na) == (15, 14, 8)
    bad = I.cartpole().replace(parent=np.array([-1, 1], np.int32))      # parent after child
    with pytest.raises(_lib.ShacError) as e:
        _lib.ModelHandle(bad)
    assert e.value.status == 2
    free_not_root = I.ant().replace(joint_type=np.array([1] + [0] + [1] * 7, np.int32))
    with pytest.raises(_lib.ShacError):
        _lib.ModelHandle(free_not_root)
    dup = I.ant().replace(act_dof=np.array([6, 6, 7, 8, 9, 10, 11, 12], np.int32))
    with pytest.raises(_lib.ShacError):
        _lib.ModelHandle(dup)
    hp = _lib.ModelHandle(I.hopper())
    assert (hp.nq, hp.nv, hp.na) == (6, 6, 3)
    for kw in ({"height_q": 6}, {"vx_dof": 6}, {"height_q": -2}):   # reward coordinates out of range
        with pytest.raises(_lib.ShacError) as e:
            _lib.ModelHandle(I.hopper().replace(**kw))
        assert e.value.status == 2
    assert _lib.status_string(5) == "capacity exceeded"
    from helpers import long_chain
    assert _lib.ModelHandle(long_chain(26)).nv == 32        # the compiled maximum
    with pytest.raises(_lib.ShacError) as e:
        _lib.ModelHandle(long_chain(27))                     # 33 DOF
    assert e.value.status == 5


def test_product_path_does_not_use_the_oracle():
    """No package module imports, loads or runs anything under oracle/."""
    pkg = os.path.join(ROOT, "paper_2204_07137_gb300")
    pat = re.compile(r"(^|\n)\s*(from|import)\s+oracle|liboracle|shac_oracle")
    for fn in os.listdir(pkg):
        if fn.endswith(".py"):
            assert not pat.search(open(os.path.join(pkg, fn)).read()), fn


def header_arities():
    """Parameter count of every declaration in include/shacsim.h."""
    src = open(os.path.join(ROOT, "include", "shacsim.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    out = {}
    for name, params in re.findall(r"\b(shac_[a-z_]+)\s*\(([^;{()]*)\)\s*;", src):
        ps = [p for p in params.split(",") if p.strip()]
        out[name] = 0 if len(ps) == 1 and ps[0].strip() == "void" else len(ps)
    return out


def test_binding_argument_lists_match_the_header(lib):
    """Every declared call has its ctypes argument list, as long as the C
    declaration's (a changed signature fails here instead of passing
    mis-marshalled arguments)."""
    from paper_2204_07137_gb300 import _lib
    from paper_2204_07137_gb300 import build
    L = _lib.load(build.LIB)
    arity = header_arities()
    assert sorted(arity) == header_functions()
    for name, n in arity.items():
        argtypes = getattr(L, name).argtypes
        assert argtypes is not None, f"{name}: no argtypes in the binding"
        assert len(argtypes) == n, f"{name}: binding passes {len(argtypes)} arguments, the header declares {n}"
