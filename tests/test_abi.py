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


def test_binding_struct_layout_matches_the_header(tmp_path):
    """The ctypes mirror of crbm_params and crbm_bond has the C layout
    (size and every field offset, as gcc lays out include/crbm.h)."""
    import ctypes
    import subprocess
    import paper_2511_20911_gb300 as crbm
    structs = {"crbm_params": crbm.crbm_params, "crbm_bond": crbm.crbm_bond}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "crbm.h"', "int main(void) {"]
    for name, cls in structs.items():
        lines.append(f'printf("{name} sizeof %zu\\n", sizeof({name}));')
        for field, _ in cls._fields_:
            lines.append(f'printf("{name} {field} %zu\\n", offsetof({name}, {field}));')
    lines.append("return 0; }")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.check_call(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)])
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split("\n")
    got = {tuple(l.split()[:2]): int(l.split()[2]) for l in out if l.strip()}
    for name, cls in structs.items():
        assert got[(name, "sizeof")] == ctypes.sizeof(cls), name
        for field, _ in cls._fields_:
            assert got[(name, field)] == getattr(cls, field).offset, (name, field)


def test_pass_record_layout_matches_the_header(tmp_path):
    """The numpy record of crbm_proposal_inspect has the C layout of
    crbm_pass_record (size and every field offset)."""
    import subprocess
    import paper_2511_20911_gb300 as crbm
    dt = crbm.PASS_RECORD
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "crbm.h"', "int main(void) {",
             'printf("sizeof %zu\\n", sizeof(crbm_pass_record));']
    for field in dt.names:
        lines.append(f'printf("{field} %zu\\n", offsetof(crbm_pass_record, {field}));')
    lines.append("return 0; }")
    src = tmp_path / "rec.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "rec"
    subprocess.check_call(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)])
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split("\n")
    got = {l.split()[0]: int(l.split()[1]) for l in out if l.strip()}
    assert got["sizeof"] == dt.itemsize
    for field in dt.names:
        assert got[field] == dt.fields[field][1], field
