"""The C-ABI library builds, loads without a GPU and exports every entry point that
include/prdpt.h declares (no compute calls here), and the Python binding mirrors
the header's names and struct layouts."""
import ctypes
import os
import re

import pytest

from paper_2211_17263_gb300 import capi

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "prdpt.h")


def _declared():
    text = open(HEADER).read()
    return sorted(set(re.findall(r"\b(prdpt_[a-z_0-9]+)\s*\(", text)))


def test_header_declarations_are_exported():
    lib = capi.load()
    names = _declared()
    assert len(names) >= 20
    for n in names:
        assert hasattr(lib, n), n
    assert sorted(capi.EXPORTS) == names


def test_struct_layouts_match_header():
    # sizes the C compiler gives the header's structs (natural alignment, LP64)
    assert ctypes.sizeof(capi.prdpt_param_binding) == 12
    assert ctypes.sizeof(capi.prdpt_scene_desc) == 8 + 7 * 8
    assert ctypes.sizeof(capi.prdpt_render_opts) == 5 * 4 + 4 + 8 + 4 * 4 + 8
    assert ctypes.sizeof(capi.prdpt_grad_opts) == 9 * 4 + 4 + 8 + 7 * 4 + 4  # trailing pad to 8-byte alignment
    assert ctypes.sizeof(capi.prdpt_job_desc) == ctypes.sizeof(capi.prdpt_grad_opts) + 3 * 8 + 7 * 4 + 4


def test_struct_layouts_match_c_compiler(tmp_path):
    """Compile a tiny C program against the header and compare sizeof/offsetof."""
    src = tmp_path / "layout.c"
    src.write_text('#include <stdio.h>\n#include <stddef.h>\n#include "prdpt.h"\n'
                   'int main(void){printf("%zu %zu %zu %zu %zu %zu %zu\\n", sizeof(prdpt_scene_desc),'
                   ' sizeof(prdpt_param_binding), sizeof(prdpt_render_opts), sizeof(prdpt_grad_opts),'
                   ' sizeof(prdpt_job_desc), offsetof(prdpt_grad_opts, seed), offsetof(prdpt_job_desc, lr));'
                   'return 0;}\n')
    exe = tmp_path / "layout"
    rc = os.system(f"gcc -I{os.path.join(ROOT, 'include')} {src} -o {exe}")
    if rc != 0:
        pytest.skip("no C compiler")
    out = os.popen(str(exe)).read().split()
    got = [int(x) for x in out]
    exp = [ctypes.sizeof(capi.prdpt_scene_desc), ctypes.sizeof(capi.prdpt_param_binding),
           ctypes.sizeof(capi.prdpt_render_opts), ctypes.sizeof(capi.prdpt_grad_opts),
           ctypes.sizeof(capi.prdpt_job_desc), capi.prdpt_grad_opts.seed.offset, capi.prdpt_job_desc.lr.offset]
    assert got == exp


def test_create_without_gpu_fails_cleanly():
    try:
        import torch
        if torch.cuda.is_available():
            pytest.skip("a GPU is present")
    except Exception:
        pass
    lib = capi.load()
    h = ctypes.c_void_p()
    rc = lib.prdpt_create(ctypes.byref(h), 0, 0)
    assert rc in (capi.PRDPT_E_CUDA, capi.PRDPT_E_INVALID_ARG)
    assert not h.value
    assert len(lib.prdpt_last_error(None)) > 0
