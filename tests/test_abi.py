"""The C-ABI library builds for sm_103a, loads, and exports every entry point that
include/gdm.h declares (no GPU needed: no compute call is made here)."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def header_functions():
    src = open(os.path.join(ROOT, "include", "gdm.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(gdm_[a-z_0-9]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_2505_09545_gb300 import binding
    return binding.lib()


def test_header_declares_the_hot_path():
    fns = header_functions()
    for name in ("gdm_assemble", "gdm_solve", "gdm_nearfield", "gdm_cross_sections", "gdm_backward"):
        assert name in fns


def test_library_exports_every_declared_symbol(lib):
    missing = [f for f in header_functions() if not hasattr(lib, f)]
    assert not missing, missing


def test_status_strings(lib):
    for code, name in [(0, "GDM_OK"), (4, "GDM_ERR_SINGULAR"), (8, "GDM_ERR_TIMEOUT"), (9, "GDM_ERR_UNSUPPORTED")]:
        assert lib.gdm_status_string(code).decode() == name


def test_null_context_is_rejected_without_touching_the_gpu(lib):
    from paper_2505_09545_gb300 import binding
    p = binding.Problem(10, 3, 0, 0, 0, 0, 10.0, 1.0, 500.0)
    assert lib.gdm_assemble(None, C.byref(p), 1, None, 32) == 1
    assert lib.gdm_solve(None, C.byref(p), 1, None, 32, None, None, None, 1, None, None) == 1
    assert lib.gdm_cross_sections(None, C.byref(p), None, None, 1, None, None, None, None) == 1


def test_workspace_size_is_host_only(lib):
    from paper_2505_09545_gb300 import binding
    p = binding.Problem(12000, 3, 0, 0, 0, 0, 10.0, 1.0, 500.0)
    b = C.c_size_t(0)
    assert lib.gdm_workspace_size(C.byref(p), 2, 1, C.byref(b)) == 0
    assert b.value > 36000 * 2 * 16
    # TF32 at 3N = 36,000: the recursive factorisation's L embedding (2 x 36,000 x 2 x 512 FP32), the
    # tensor-core operand buffers of the same size plus a U12 copy, and the U12 block operator's row block
    b32 = C.c_size_t(0)
    assert lib.gdm_workspace_size(C.byref(p), 2, binding.PRECISION["tf32"], C.byref(b32)) == 0
    emb = 2 * 36000 * 2 * 512 * 4
    assert b32.value >= 2 * emb + 36000 * 2 * 512 * 4 + 512 * 36000 * 8


def test_built_for_sm103a():
    from paper_2505_09545_gb300 import _build
    assert "arch=compute_103a,code=sm_103a" in " ".join(_build.ARCH)
    assert os.path.exists(_build.LIB)


@pytest.mark.parametrize("cname,pyname", [("gdm_batch_item", "BatchItem"), ("gdm_backward_item", "BackwardItem"),
                                          ("gdm_gmres_opts", "GmresOpts"), ("gdm_solve_info", "SolveInfo"),
                                          ("gdm_problem", "Problem")])
def test_batch_item_layout_matches_the_header(tmp_path, cname, pyname):
    """The ctypes mirrors of the batch structs have the C compiler's size and field offsets."""
    import shutil
    import subprocess
    from paper_2505_09545_gb300 import binding
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    cls = getattr(binding, pyname)
    fields = [f for f, _ in cls._fields_]
    src = tmp_path / "layout.c"
    body = "".join(f'printf("%zu\\n", offsetof({cname}, {f}));' for f in fields)
    src.write_text('#include <stdio.h>\n#include <stddef.h>\n#include "gdm.h"\n'
                   f'int main(void) {{ printf("%zu\\n", sizeof({cname})); {body} return 0; }}\n')
    exe = tmp_path / "layout"
    subprocess.run([cc, "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = [int(v) for v in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()]
    assert out[0] == C.sizeof(cls)
    assert out[1:] == [getattr(cls, f).offset for f in fields]


def test_batched_and_autotune_reject_a_null_context(lib):
    assert lib.gdm_solve_batched(None, 2, None, 0, None, 0, None) == 1
    assert lib.gdm_autotune(None, 2, None, 0, None) == 1
    assert lib.gdm_backward_batched(None, 2, None, 0, 0, None, None, None) == 1
    assert lib.gdm_solve_gmres(None, 2, None, None, None, 1, None, None) == 1


def test_refine_stop_measure_is_host_only(lib):
    """The refinements' stopping measure: with GDM_SOLVE_ERR_ESTIMATE and corrections contracting by
    rho = c / c_prev <= 1/4, the tail rho c / (1 - rho) of the corrections still to come; else (no flag, no
    step before, or rho above 1/4) the last correction itself. On an exactly geometric sequence of
    corrections the measure equals the sum of all later corrections."""
    from paper_2505_09545_gb300 import binding
    f = lib.gdm_refine_stop_measure
    E = binding.SOLVE_ERR_ESTIMATE
    # corrections measured on the 40 x 30 x 10 cuboid after steps 2 and 3
    c, p = 5.981e-10, 1.441e-6
    rho = c / p
    assert f(c, p, E) == pytest.approx(rho * c / (1 - rho), rel=1e-15)
    assert f(c, p, E) < 1e-10 < c
    assert f(c, p, 0) == c
    assert f(c, -1.0, E) == c
    assert f(0.3, 1.0, E) == 0.3
    assert f(0.25, 1.0, E) == pytest.approx(0.25 * 0.25 / 0.75, rel=1e-15)
    assert f(0.0, 1e-9, E) == 0.0
    c0, q = 1e-3, 1e-2
    for k in range(1, 5):
        tail = sum(c0 * q ** j for j in range(k + 1, 60))
        assert f(c0 * q ** k, c0 * q ** (k - 1), E) == pytest.approx(tail, rel=1e-12)
