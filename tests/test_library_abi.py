"""CPU checks of the C-ABI library: it builds for sm_103a, loads, and exports
every entry point include/pbs.h declares (no compute call without a GPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    with open(os.path.join(ROOT, "include", "pbs.h")) as f:
        text = f.read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(pbs_[a-z_0-9]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    from paper_2504_00340_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert len(names) >= 20
    for n in names:
        assert hasattr(lib, n), n


def test_binding_covers_the_header():
    from paper_2504_00340_gb300 import binding
    bound = {n for n, _, _ in binding.SIGNATURES}
    assert bound == set(_declared())


def test_status_strings(lib):
    lib.pbs_status_string.restype = ctypes.c_char_p
    assert lib.pbs_status_string(0) == b"ok"
    assert lib.pbs_status_string(-4) == b"call out of order"


def test_null_arguments_are_rejected_without_a_device(lib):
    # argument checks run before any CUDA call
    assert lib.pbs_create(None, None, 0, None) == -1
    assert lib.pbs_workspace_size(None, None) == -1
    assert lib.pbs_step(None, 1) == -1


def test_product_package_does_not_import_the_oracle():
    pkg = os.path.join(ROOT, "paper_2504_00340_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                with open(os.path.join(dirpath, f)) as fh:
                    src = fh.read()
                assert "import oracle" not in src and "pbs_oracle" not in src, f


def test_binding_structs_match_the_header(tmp_path):
    """Size and field offsets of every struct the binding marshals equal the
    C compiler's for include/pbs.h (a field added on one side only would
    shift everything after it)."""
    import subprocess

    from paper_2504_00340_gb300 import binding as B
    structs = {"pbs_grid": B.PbsGrid, "pbs_physics": B.PbsPhysics, "pbs_beam": B.PbsBeam,
               "pbs_options": B.PbsOptions, "pbs_tuning": B.PbsTuning, "pbs_batch_options": B.PbsBatchOptions}
    lines = ["#include <stddef.h>", "#include <stdio.h>", '#include "pbs.h"', "int main(void) {"]
    for name, cls in structs.items():
        lines.append(f'  printf("{name} size %zu\\n", sizeof({name}));')
        for field, _ in cls._fields_:
            lines.append(f'  printf("{name} {field} %zu\\n", offsetof({name}, {field}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c99", "-I", os.path.join(ROOT, "include"), "-o", str(exe), str(src)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    got = {tuple(l.split()[:2]): int(l.split()[2]) for l in out if l.strip()}
    for name, cls in structs.items():
        assert got[(name, "size")] == ctypes.sizeof(cls), name
        for field, _ in cls._fields_:
            assert got[(name, field)] == getattr(cls, field).offset, (name, field)
