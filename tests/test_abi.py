"""The C-ABI library loads and exports every entry point include/pdlp.h declares
(no GPU needed: nothing here launches a kernel)."""
import os
import re
import subprocess
import ctypes as C

import pytest

import __graft_entry__ as G

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADERS = [os.path.join(ROOT, "include", h) for h in os.listdir(os.path.join(ROOT, "include"))
           if h.endswith(".h")]


def declared_functions():
    names = set()
    for h in HEADERS:
        src = re.sub(r"/\*.*?\*/", "", open(h).read(), flags=re.S)
        for m in re.finditer(r"^\s*[A-Za-z_][\w\s\*]*?\b([a-z_][a-z0-9_]*)\s*\(", src, flags=re.M):
            if not m.group(0).lstrip().startswith(("typedef", "#", "return")):
                names.add(m.group(1))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    G.build()
    import paper_2503_10344_gb300 as P
    return P.lib()


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert "pdlp_solve" in names and "pdlp_solve_device" in names
    assert "gnn_train" in names and "pdlp_solve_warm" in names
    for n in names:
        assert hasattr(lib, n), n


def test_struct_layouts_match_the_header(tmp_path):
    """Compile a C program against the header and compare sizeof/offsetof with ctypes."""
    import paper_2503_10344_gb300.binding as B
    import paper_2503_10344_gb300.gnn as N
    prog = tmp_path / "sz.c"
    fields = {"pdlp_params": B.PdlpParams, "pdlp_result": B.PdlpResult, "pdlp_csr": B.PdlpCsr,
              "pdlp_diagnostics": B.PdlpDiagnostics, "fp_params": B.FpParams,
              "fp_result": B.FpResult, "gnn_adam": N.GnnAdam, "gnn_train_params": N.GnnTrainParams,
              "gnn_warm_info": N.GnnWarmInfo}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "pdlp.h"', '#include "gnn.h"',
             "int main(void){"]
    for s, cls in fields.items():
        lines.append(f'printf("{s} %zu\\n", sizeof({s}));')
        for f, _ in cls._fields_:
            lines.append(f'printf("{s}.{f} %zu\\n", offsetof({s}, {f}));')
    lines.append("return 0;}")
    prog.write_text("\n".join(lines))
    exe = tmp_path / "sz"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(prog), "-o", str(exe)], check=True)
    out = dict(l.rsplit(" ", 1) for l in subprocess.run([str(exe)], capture_output=True, text=True,
                                                         check=True).stdout.split("\n") if l)
    for s, cls in fields.items():
        assert int(out[s]) == C.sizeof(cls), s
        for f, _ in cls._fields_:
            assert int(out[f"{s}.{f}"]) == getattr(cls, f).offset, (s, f)


def test_default_params(lib):
    import paper_2503_10344_gb300 as P
    p = P.default_params()
    assert p.struct_size == C.sizeof(type(p))
    assert p.tol == 1e-4 and p.check_period == 64 and p.ruiz_iters == 10 and p.pc_alpha == 1.0
    assert p.adaptive_step == 1 and p.restarts == 1 and p.terminate == 1
    assert p.precision == P.PDLP_FP64
    assert p.detect_infeasibility == 1 and p.persistent == 0 and p.autotune == 0


def test_workspace_size_rejects_bad_sizes(lib):
    import paper_2503_10344_gb300 as P
    assert P.workspace_size(10, 20, 30) > 0
    assert P.workspace_size(-1, 20, 30) == 0
    assert P.workspace_size(10, 0, 30) == 0


def test_error_strings(lib):
    for code, name in [(0, b"PDLP_OK"), (-1, b"PDLP_ERR_INVALID_INPUT"), (-2, b"PDLP_ERR_CUDA"),
                       (-3, b"PDLP_ERR_OOM"), (-4, b"PDLP_ERR_TIMEOUT")]:
        assert lib.pdlp_error_string(code) == name
