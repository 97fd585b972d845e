"""CPU checks of the boundary: the library builds for sm_103a, loads, and exports every entry point
declared in include/kiops.h (no compute calls without a GPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def header_functions():
    src = open(os.path.join(ROOT, "include", "kiops.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(kiops_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def libpath():
    from paper_1804_05126_gb300 import build
    return build.build()


def test_header_declares_the_boundary():
    names = header_functions()
    for must in ("kiops_create", "kiops_destroy", "kiops_solve", "kiops_op_csr", "kiops_op_stencil2d",
                 "kiops_op_stencil3d", "kiops_solve_batch", "kiops_solve_host", "kiops_expm"):
        assert must in names


def test_library_exports_every_declared_symbol(libpath):
    lib = ctypes.CDLL(libpath)
    missing = [n for n in header_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_every_declared_symbol(libpath):
    from paper_1804_05126_gb300 import kiops
    assert set(header_functions()) <= set(kiops.exported_symbols())
    kiops.lib()


def test_defaults_match_the_paper(libpath):
    from paper_1804_05126_gb300 import kiops
    from tests.golden_util import paper_constants
    pc = paper_constants()
    cfg = kiops.kiops_config_default()
    assert cfg.m_min == pc["m_min_default"] and cfg.m_max == pc["m_max_default"]
    delta, gamma, gamma_max, kappa, clip, m_o = kiops.kiops_constants()
    assert (delta, gamma, gamma_max, kappa, clip, m_o) == (pc["delta"], pc["gamma"], pc["gamma_max"],
                                                           pc["kappa_default"], pc["tau_clip_high"], pc["m_o_default"])


def test_engineering_defaults(libpath):
    from paper_1804_05126_gb300 import kiops
    cfg = kiops.kiops_config_default()
    assert cfg.fuse_stencil == 1 and cfg.fused_smem == -1 and cfg.batch_team_blocks == 0
    assert cfg.grid_blocks == 0 and cfg.profile == 0 and cfg.normalize_B == 1


def test_status_strings_and_null_handling(libpath):
    from paper_1804_05126_gb300 import kiops
    L = kiops.lib()
    assert L.kiops_status_string(0) == b"ok"
    assert L.kiops_destroy(None) == 1          # EINVAL, no crash
    assert L.kiops_last_error(None) == b"NULL context"
    assert L.kiops_config_default(None) == 1


MIRRORED = ["kiops_config", "kiops_stats", "kiops_trace_rec", "kiops_stencil2d_desc", "kiops_stencil3d_desc",
            "kiops_server_config", "kiops_request", "kiops_pde", "kiops_integrate_stats"]


def test_binding_structs_match_the_header_layout(tmp_path):
    """Every struct the Python binding mirrors has the header's size and member offsets (a C program built
    with the host compiler prints them)."""
    import shutil
    import subprocess

    from paper_1804_05126_gb300 import kiops
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no host C compiler")
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "kiops.h"', "int main(void) {"]
    for name in MIRRORED:
        cls = getattr(kiops, name)
        lines.append(f'  printf("{name} size %zu\\n", sizeof({name}));')
        for fname, _ in cls._fields_:
            lines.append(f'  printf("{name} {fname} %zu\\n", offsetof({name}, {fname}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.check_call([cc, "-std=c99", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)])
    got = {}
    for ln in subprocess.check_output([str(exe)], text=True).splitlines():
        name, member, value = ln.split()
        got[(name, member)] = int(value)
    for name in MIRRORED:
        cls = getattr(kiops, name)
        assert got[(name, "size")] == ctypes.sizeof(cls), name
        for fname, _ in cls._fields_:
            assert got[(name, fname)] == getattr(cls, fname).offset, (name, fname)


def test_gray_scott_shared_fields_describe_the_same_block():
    """The Gray-Scott workload's coupling block in its two forms: const + weight * field (weights +-1) gives
    every entry of "diag" exactly."""
    import numpy as np

    from paper_1804_05126_gb300 import workloads as W
    op = W.problem_gray_scott(n=48, seed=3).op
    sh = op["shared_fields"]
    assert len(sh["fields"]) == 2 and set(sh["entries"]) == set(op["diag"])
    for rc, (f, const, weight) in sh["entries"].items():
        assert np.array_equal(const + weight * sh["fields"][f], op["diag"][rc]), rc
