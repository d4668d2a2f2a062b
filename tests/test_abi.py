"""The C-ABI library loads without a GPU and exports every entry point that
include/crbm.h declares (no compute calls here)."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            with open(os.path.join(ROOT, "include", f)) as fh:
                txt = fh.read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names |= set(re.findall(r"\b(crbm_[a-z0-9_]+)\s*\(", txt))
    return names


def test_header_declares_expected_entry_points():
    names = declared_functions()
    for n in ("crbm_create", "crbm_sweep", "crbm_observables", "crbm_destroy"):
        assert n in names


def test_library_exports_every_declared_symbol():
    import ctypes
    import paper_2511_20911_gb300 as crbm
    path = crbm.build()
    lib = ctypes.CDLL(path)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing
    assert set(crbm.ABI_FUNCTIONS) >= declared_functions()


def test_no_cpu_fallback_without_gpu():
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("GPU present")
    import paper_2511_20911_gb300 as crbm
    with pytest.raises(crbm.CrbmError):
        crbm.Sampler(6, dict(J=[1.0], Jp=[1.0], h=[0.5], beta=[2.0]), 32)


def test_workloads_shapes():
    from paper_2511_20911_gb300 import workloads
    w = workloads.grid_workload()
    assert w["n_chains"] == 3 * 16 * 16 * 16 and len(w["params"]["J"]) == 768
    assert all(abs(x * 16 - round(x * 16)) < 1e-12 for x in w["params"]["h"])
