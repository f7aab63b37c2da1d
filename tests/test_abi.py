"""The C-ABI library loads and exports every symbol include/*.h declares,
and the binding's structs match the header's layout.  No GPU is needed: no
test here launches a kernel."""
import ctypes as C
import os
import re
import subprocess

import pytest

from conftest import ROOT

HEADER = os.path.join(ROOT, "include", "rdsel.h")


@pytest.fixture(scope="module")
def rdsel():
    from paper_1806_08901_gb300 import _build, rdsel as R

    _build.build()
    R.lib()
    return R


def _declared_functions():
    inc = os.path.join(ROOT, "include")
    text = "".join(open(os.path.join(inc, h)).read() for h in sorted(os.listdir(inc)) if h.endswith(".h"))
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(rd_[a-z0-9_]+)\s*\(", text)))


def test_every_declared_symbol_is_exported(rdsel):
    names = _declared_functions()
    assert len(names) >= 14
    L = C.CDLL(rdsel.LIB_PATH)
    for n in names:
        assert hasattr(L, n), n
    out = subprocess.run(["nm", "-D", "--defined-only", rdsel.LIB_PATH], capture_output=True,
                         text=True, check=True).stdout
    exported = set(re.findall(r"\bT (rd_[a-z0-9_]+)", out))
    assert set(names) <= exported
    # the binding wraps exactly the declared entry points
    assert sorted(rdsel.exported_symbols()) == names


def test_struct_layout_matches_header(rdsel, tmp_path):
    """Compile a probe against include/rdsel.h with the host compiler and
    compare sizeof / offsetof with the ctypes mirrors."""
    structs = {"rd_field": rdsel.rd_field, "rd_params": rdsel.rd_params,
               "rd_result": rdsel.rd_result, "rd_truth": rdsel.rd_truth,
               "rd_batch_config": rdsel.rd_batch_config,
               "rd_rd_point": rdsel.rd_rd_point,
               "rd_log_result": rdsel.rd_log_result,
               "rd_server_config": rdsel.rd_server_config,
               "rd_server_completion": rdsel.rd_server_completion,
               "rd_server_stats": rdsel.rd_server_stats}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "rdsel.h"', "int main(void){"]
    for sname, cls in structs.items():
        lines.append(f'printf("{sname} sizeof %zu\\n", sizeof({sname}));')
        for fname, _ in cls._fields_:
            lines.append(f'printf("{sname} {fname} %zu\\n", offsetof({sname}, {fname}));')
    lines.append("return 0;}")
    src = tmp_path / "probe.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "probe"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split("\n")
    for line in filter(None, out):
        sname, fname, val = line.split()
        cls = structs[sname]
        if fname == "sizeof":
            assert C.sizeof(cls) == int(val), sname
        else:
            assert getattr(cls, fname).offset == int(val), (sname, fname)


def test_status_strings(rdsel):
    for code in (0, -1, -2, -3, -4, -5, -6, -7):
        assert rdsel.status_string(code) != "unknown status"
    assert rdsel.status_string(-99) == "unknown status"


def test_context_without_gpu_fails_cleanly(rdsel):
    import torch

    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(rdsel.RdselError) as e:
        rdsel.rd_context_create(0)
    assert e.value.code in (rdsel.RD_ERR_CUDA, rdsel.RD_ERR_INVALID_ARG)


def test_product_package_does_not_import_oracle():
    """The CUDA package and the oracle share no code and neither imports the
    other."""
    pkg = os.path.join(ROOT, "paper_1806_08901_gb300")
    for dirpath, _, files in os.walk(pkg):
        for fn in files:
            if fn.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                text = open(os.path.join(dirpath, fn)).read()
                assert "oracle" not in re.sub(r"#.*|//.*", "", text).replace("oracles", ""), fn
                assert "rdo_" not in text, fn
    for fn in os.listdir(os.path.join(ROOT, "oracle")):
        if fn.endswith((".py", ".c", ".h")):
            text = open(os.path.join(ROOT, "oracle", fn)).read()
            assert "paper_1806_08901_gb300" not in text and "rdsel" not in text, fn
