"""Host-only checks of the C ABI: the shared library builds and loads, it
exports every function include/cvxb300.h declares, the ctypes layouts match
the C struct layouts, defaults are as documented, and calls fail cleanly (no
crash) where no GPU is present."""
import ctypes as C
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "cvxb300.h")


def _declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\**\s+\**([A-Za-z_][A-Za-z0-9_]*)\s*\(",
                       src, flags=re.M)
    return sorted(set(names) - {"if", "while"})


def test_library_exports_every_declared_symbol():
    from paper_1609_03488_b300 import binding
    declared = _declared_functions()
    assert len(declared) >= 20
    missing = [n for n in declared if not hasattr(binding.lib, n)]
    assert not missing, missing
    assert sorted(binding.EXPORTED) == declared


def test_struct_layouts_match_c(tmp_path):
    from paper_1609_03488_b300 import binding
    prog = tmp_path / "sz.c"
    prog.write_text('#include "cvxb300.h"\n#include <stdio.h>\n#include <stddef.h>\n'
                    'int main(void){printf("%zu %zu %zu %zu %zu\\n", sizeof(cf_settings), sizeof(cf_info),'
                    ' sizeof(cf_cone), offsetof(cf_info, kernel_launches), offsetof(cf_settings, setup_cg_tol));'
                    'return 0;}\n')
    exe = tmp_path / "sz"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(prog), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split()
    got = [C.sizeof(binding.cf_settings), C.sizeof(binding.cf_info), C.sizeof(binding.cf_cone),
           binding.cf_info.kernel_launches.offset, binding.cf_settings.setup_cg_tol.offset]
    assert [int(v) for v in out] == got


def test_team_struct_layouts_match_c(tmp_path):
    from paper_1609_03488_b300 import binding as b
    prog = tmp_path / "sz2.c"
    prog.write_text('#include "cvxb300.h"\n#include <stdio.h>\n#include <stddef.h>\n'
                    'int main(void){printf("%zu %zu %zu %zu %zu %d %d %d\\n", sizeof(cf_schedule),'
                    ' sizeof(cf_tune_info), offsetof(cf_tune_info, best), offsetof(cf_settings, engine),'
                    ' offsetof(cf_schedule, team_bytes), CF_ENGINE_AUTO, CF_ENGINE_GRAPH, CF_ENGINE_TEAM);'
                    'return 0;}\n')
    exe = tmp_path / "sz2"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(prog), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split()
    got = [C.sizeof(b.cf_schedule), C.sizeof(b.cf_tune_info), b.cf_tune_info.best.offset,
           b.cf_settings.engine.offset, b.cf_schedule.team_bytes.offset,
           b.CF_ENGINE_AUTO, b.CF_ENGINE_GRAPH, b.CF_ENGINE_TEAM]
    assert [int(v) for v in out] == got


def test_team_entry_points_reject_bad_arguments_without_a_device():
    from paper_1609_03488_b300 import binding as b
    s = b.cf_schedule()
    assert b.lib.cf_ctx_get_schedule(None, C.byref(s)) == b.CF_E_INVALID
    assert b.lib.cf_ctx_set_schedule(None, C.byref(s)) == b.CF_E_INVALID
    assert b.lib.solve_batch_tune(None, -1, 10, None) == b.CF_E_INVALID
    assert b.lib.solve_batch_tune(None, 0, 0, None) == b.CF_E_INVALID
    assert b.lib.solve_batch_tune(None, 0, 10, None) == b.CF_OK    # empty batch: nothing to time


def test_settings_defaults():
    from paper_1609_03488_b300 import binding
    s = binding.cf_settings_default()
    assert (s.eps, s.eps_infeas, s.alpha, s.max_iters, s.check_interval) == (1e-4, 1e-4, 1.5, 100000, 10)
    assert (s.cg_max_iters, s.cg_fixed_iters, s.cg_tol_rel, s.cg_tol_exp) == (50, 0, 1.0, 1.5)
    assert s.engine == binding.CF_ENGINE_AUTO and s.host_loop == 0


def test_null_arguments_are_rejected_without_a_device():
    from paper_1609_03488_b300 import binding as b
    h = C.c_void_p()
    assert b.lib.cf_op_dense(None, 2, 2, None, 0, C.byref(h)) == b.CF_E_INVALID
    assert "bad arguments" in b.cf_last_error()
    assert b.lib.solve(None, None, None, None, None, None, None, None) == b.CF_E_INVALID
    assert b.lib.cone_problem_create(None, None, None, 0, None, 0, None, C.byref(h)) == b.CF_E_INVALID
    assert b.lib.serve_wait(None, 1, 0, None, None, None, None) == b.CF_E_INVALID
    assert b.lib.cone_problem_set_inner(None, None) == b.CF_E_INVALID
    assert "NULL problem" in b.cf_last_error()
    b.lib.cf_op_destroy(None)
    b.lib.cf_problem_destroy(None)
    b.lib.serve_destroy(None)


def test_context_without_gpu_fails_cleanly():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_1609_03488_b300 import binding as b
    with pytest.raises(b.CfError) as e:
        b.Context(0)
    assert e.value.code == b.CF_E_CUDA
