"""The C ABI library loads without a GPU and exports every entry point the header declares."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    with open(os.path.join(ROOT, "include", "pfsm.h")) as f:
        src = f.read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    for m in re.finditer(r"^\s*(?:const\s+)?\w[\w\s\*]*?\b(pfsm_\w+)\s*\(", src, flags=re.M):
        names.add(m.group(1))
    return names


@pytest.fixture(scope="module")
def lib():
    from paper_1502_07806_b300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = _declared()
    for n in ("pfsm_init", "pfsm_solve", "pfsm_backward", "pfsm_get_status", "pfsm_last_error",
              "pfsm_destroy", "pfsm_default_params", "pfsm_get_diagnostic"):
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in sorted(_declared()) if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_lists_the_same_names():
    import paper_1502_07806_b300 as pf
    assert set(pf.EXPORTED) == _declared()


def test_default_params_and_last_error_without_gpu(lib):
    import paper_1502_07806_b300 as pf
    p = pf.default_params()
    assert p.halo == -1 and p.fs_iters == 3 and p.alpha_theta == 1.0
    assert p.cluster_tol == 1e-5 and p.degen_tol == 1e-8 and p.precision == pf.FP64
    pf.load_library().pfsm_last_error.restype = ctypes.c_char_p
    assert isinstance(pf.load_library().pfsm_last_error(), bytes)


def test_init_rejects_bad_arguments_before_touching_the_gpu(lib):
    import paper_1502_07806_b300 as pf
    for n, nb in ((0, 1), (10, 0), (10, 11), (70000, 4)):
        with pytest.raises(pf.PFSMError) as e:
            pf.Handle(n, nb)
        assert e.value.code == pf.INVALID_ARG
    with pytest.raises(pf.PFSMError) as e:
        pf.Handle(10, 2, slice_sizes=[3, 4])
    assert e.value.code == pf.INVALID_ARG
    with pytest.raises(pf.PFSMError) as e:
        pf.Handle(10, 2, fs_iters=-1)
    assert e.value.code == pf.INVALID_ARG
