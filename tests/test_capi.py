"""The C ABI library loads and exports every symbol include/cdv.h declares (no GPU calls)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "cdv.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(cdv_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_1711_11224_gb300 import build
    build.build()
    from paper_1711_11224_gb300 import _binding
    return _binding.load()


def test_exports_every_declared_symbol(lib):
    from paper_1711_11224_gb300 import _binding
    names = _declared()
    assert len(names) >= 16
    for n in names:
        assert hasattr(lib, n), n
    assert set(names) == set(_binding.EXPORTS)


def test_status_strings_and_argument_errors(lib):
    assert lib.cdv_status_string(0) == b"CDV_OK"
    assert lib.cdv_status_string(9) == b"CDV_ERR_NO_PSF"
    h = ctypes.c_void_p()
    m = (ctypes.c_int64 * 3)(4, 5, 6)
    p = (ctypes.c_int32 * 3)(1, 1, 1)
    assert lib.cdv_plan_create(ctypes.byref(h), 4, m, p, 0, None) == 2          # SHAPE: n = 4
    assert lib.cdv_plan_create(None, 3, m, p, 0, None) == 1                     # INVALID_ARG
    bad = (ctypes.c_int32 * 3)(1, -1, 1)
    assert lib.cdv_plan_create(ctypes.byref(h), 3, m, bad, 0, None) == 2        # p < 0
    assert lib.cdv_plan_create(ctypes.byref(h), 3, m, p, 7, None) == 1          # unknown mode
    assert lib.cdv_plan_destroy(None) == 0


def test_no_cpu_fallback_without_device(lib):
    """Without a CUDA device every computing call reports CDV_ERR_CUDA; nothing computes on the host."""
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    h = ctypes.c_void_p()
    m = (ctypes.c_int64 * 2)(8, 8)
    p = (ctypes.c_int32 * 2)(1, 1)
    assert lib.cdv_plan_create(ctypes.byref(h), 2, m, p, 0, None) == 5
    assert not h.value


def test_iter_opts_defaults(lib):
    from paper_1711_11224_gb300 import _binding as B
    o = B.IterOpts()
    lib.cdv_iter_opts_default(ctypes.byref(o))
    assert (o.x0_policy, o.delta0, o.beta, o.max_halvings, o.max_rejects, o.use_graph) == (0, 0.0, 0.5, 20, 16, 1)


def test_struct_layouts_match_the_header(tmp_path):
    """Every field offset and size of the ctypes structures equals the C compiler's for include/cdv.h."""
    import shutil
    import subprocess
    from paper_1711_11224_gb300 import _binding as B
    cc = shutil.which("gcc") or shutil.which("cc")
    if not cc:
        pytest.skip("no C compiler")
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    structs = {"cdv_iter_opts": B.IterOpts, "cdv_iter_report": B.IterReport, "cdv_plan_info": B.PlanInfo}
    lines = ["#include <stddef.h>", "#include <stdio.h>", '#include "cdv.h"', "int main(void) {"]
    for cname, cls in structs.items():
        lines.append('printf("%s sizeof %%zu\\n", sizeof(%s));' % (cname, cname))
        for f in cls._fields_:
            lines.append('printf("%s %s %%zu\\n", offsetof(%s, %s));' % (cname, f[0], cname, f[0]))
    lines += ["return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-std=c11", "-I", os.path.join(root, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    got = {tuple(l.split()[:2]): int(l.split()[2]) for l in out if l.strip()}
    for cname, cls in structs.items():
        assert got[(cname, "sizeof")] == ctypes.sizeof(cls), cname
        for f in cls._fields_:
            assert got[(cname, f[0])] == getattr(cls, f[0]).offset, (cname, f[0])
