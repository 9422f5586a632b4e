"""The C-ABI library builds for sm_103a, loads without a GPU, and exports every entry point that
include/hyperim.h declares; the Python binding wraps exactly those names and refuses to compute
without a CUDA device (there is no CPU fallback)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared():
    src = open(os.path.join(ROOT, "include", "hyperim.h")).read()
    return sorted(set(re.findall(r"^(?:hyperim_status|void|uint64_t|const char\*)\s+(hyperim_\w+)\(", src, re.M)))


@pytest.fixture(scope="module")
def libpath():
    from paper_2406_01911_gb300 import build
    return build.build()


def test_header_declares_the_boundary():
    names = declared()
    for n in ("hyperim_load", "hyperim_plan_theta", "hyperim_sample_rr", "hyperim_select_seeds",
              "hyperim_spread"):
        assert n in names


def test_library_exports_every_declared_symbol(libpath):
    lib = ctypes.CDLL(libpath)
    for name in declared():
        assert hasattr(lib, name), name


def test_binding_names_match_header(libpath):
    import paper_2406_01911_gb300 as H
    assert H.exported_symbols() == declared()
    H.lib()


def test_no_cpu_fallback(libpath):
    import torch
    import paper_2406_01911_gb300 as H
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(RuntimeError):
        H.Graph(3, [0, 2], [0, 1])


def test_load_rejects_bad_arguments_before_touching_the_device(libpath):
    import paper_2406_01911_gb300 as H
    import numpy as np
    off = np.array([0, 2], np.int32)
    mem = np.array([0, 1], np.int32)
    for kw in ({"model": "uniform_pair", "uniform_threshold": (1 << 32) + 1},):
        with pytest.raises(H.HyperIMError) as e:
            H.hyperim_load(3, off, mem, stream=0, **kw)
        assert e.value.status == -1
    with pytest.raises(H.HyperIMError):
        H.hyperim_load(0, off, mem, stream=0)


def test_batch_and_tuning_reject_bad_arguments_before_touching_the_device(libpath):
    # argument checks of the batched seed selection and the tuning calls run on the host alone
    import ctypes as C
    import paper_2406_01911_gb300 as H
    lib = H.lib()
    assert lib.hyperim_select_seeds_batch(None, 0) == -1  # no queries
    q = (H.BatchQuery * 1)()
    q[0] = H.BatchQuery(None, None, None, 5, 0.1, 1.0, None, None)
    assert lib.hyperim_select_seeds_batch(q, 1) == -1  # null graph and pools
    assert lib.hyperim_graph_set_tuning(None, C.byref(H.Tuning(0, 4, 0))) == -1
    assert lib.hyperim_graph_set_wait_limit(None, 1) == -1
    assert "null" in lib.hyperim_last_error().decode()
