"""The C-ABI library builds, loads, and exports every symbol include/dwf.h declares
(no compute calls: these run without a GPU)."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    text = open(os.path.join(ROOT, "include", "dwf.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b((?:dwf|mspcg)_[a-z0-9_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def libpath():
    from paper_1811_08488_gb300 import build
    return build.build()


def test_header_declares_the_boundary():
    names = declared_functions()
    for n in ["dwf_create", "dwf_gauge_load", "dwf_dslash_eo", "dwf_m5inv", "mspcg_solve",
              "dwf_last_error", "dwf_destroy"]:
        assert n in names


def test_library_exports_every_declared_symbol(libpath):
    lib = ctypes.CDLL(libpath)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True, text=True)
    exported = set(l.split()[-1] for l in out.stdout.splitlines() if l.strip())
    assert set(declared_functions()) <= exported


def test_binding_covers_the_header(libpath):
    from paper_1811_08488_gb300 import dwf
    assert sorted(dwf.EXPORTS) == declared_functions()


def test_binding_struct_layouts_match_header(libpath):
    """The ctypes structs follow the C structs (checked through the library's
    own default-filling function, which runs on the host)."""
    from paper_1811_08488_gb300 import dwf
    p = dwf.default_params()
    assert p.tol == 1e-10 and p.maxiter == 100000 and p.inner_iters == 6
    assert p.outer == dwf.DWF_FP32 and p.inner == dwf.DWF_FP16
    assert p.delta == 0.001 and p.snake == 1 and p.use_graph == 1 and p.check_every == 10
    assert p.flexible == 0
    e = dwf.default_eig_params()
    assert e.n_ev == 16 and e.degree == 20 and e.max_passes == 30 and e.tol == 1e-6
    assert e.lambda_max == 0.0 and e.power_steps == 30 and e.schur == 0


def c_layout(struct, fields, tmp_path):
    """sizeof(struct) and offsetof(struct, f) for each field, as a C compiler
    lays them out from include/dwf.h."""
    src = tmp_path / "layout.c"
    body = "".join(f'  printf("%zu\\n", offsetof({struct}, {f}));\n' for f in fields)
    src.write_text("#include <stddef.h>\n#include <stdio.h>\n#include \"dwf.h\"\n"
                   f"int main(void) {{\n  printf(\"%zu\\n\", sizeof({struct}));\n{body}"
                   "  return 0;\n}\n")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c99", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                   check=True)
    vals = [int(v) for v in subprocess.run([str(exe)], capture_output=True, text=True,
                                           check=True).stdout.split()]
    return vals[0], vals[1:]


@pytest.mark.parametrize("cname,pyname", [("dwf_action", "Action"),
                                          ("dwf_solver_params", "SolverParams"),
                                          ("dwf_solve_info", "SolveInfo"),
                                          ("dwf_kernel_time", "KernelTime"),
                                          ("dwf_eig_params", "EigParams"),
                                          ("dwf_eig_info", "EigInfo")])
def test_binding_structs_match_the_c_layout(cname, pyname, tmp_path):
    """Every ctypes struct of the binding has the size and field offsets that a
    C compiler gives the header's struct (dwf_solve_info includes dslash_gbs)."""
    from paper_1811_08488_gb300 import dwf
    cls = getattr(dwf, pyname)
    fields = [f for f, _ in cls._fields_]
    size, offs = c_layout(cname, fields, tmp_path)
    assert ctypes.sizeof(cls) == size
    assert [getattr(cls, f).offset for f in fields] == offs
    if cname == "dwf_solve_info":
        assert "dslash_gbs" in fields


def test_no_cpu_fallback_without_device(libpath):
    """Without a usable GPU the context cannot be created: the library fails
    loudly instead of computing on the CPU."""
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_1811_08488_gb300 import dwf
    with pytest.raises(dwf.DwfError):
        dwf.Context((4, 4, 4, 4), 4)
