"""The ctypes structures of the Python binding have the sizes and field
offsets the C header gives its structures (compiled with the host C
compiler; no GPU, no library needed)."""
import ctypes
import json
import os
import shutil
import subprocess

import pytest

from paper_2605_04509_gb300 import lfd

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

# (C type, ctypes class, C field names in the ctypes field order)
LAYOUTS = [
    ("lfd_panel", lfd.CPanel, ["width", "height", "num_views", "tan_slant", "pitch", "k_offset"]),
    ("lfd_opts", lfd.COpts, ["tile_w", "tile_h", "views_per_cluster", "remap", "sort_mode", "bg",
                             "subpixels_per_thread"]),
    ("lfd_gaussians", lfd.CGaussians, ["means", "scales", "quats", "opacities", "sh", "count",
                                       "sh_degree", "attr_dtype"]),
    ("lfd_camera", lfd.CCamera, ["R"]),
    ("lfd_plan_info", lfd.CPlanInfo, ["num_clusters", "tiles_x", "tiles_y", "tile_capacity", "bit_k",
                                      "bit_t", "max_segment"]),
    ("lfd_stats", lfd.CStats, ["num_pairs", "num_visits", "num_evals", "ms_project", "ms_keygen",
                               "ms_sort", "ms_blend"]),
    ("lfd_stage_times", lfd.CStageTotals, ["frames", "ms_project", "ms_keygen", "ms_sort",
                                           "ms_blend"]),
]


@pytest.fixture(scope="module")
def c_layouts(tmp_path_factory):
    cc = shutil.which("gcc") or shutil.which("cc")
    if not cc:
        pytest.skip("no host C compiler")
    d = tmp_path_factory.mktemp("layout")
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "lfd.h"', "int main(void) {",
             '  printf("{");']
    first = True
    for ctype, _cls, fields in LAYOUTS:
        sep = "" if first else ","
        first = False
        offs = ", ".join(f'\\"{f}\\": %zu' for f in fields)
        args = ", ".join(f"offsetof({ctype}, {f})" for f in fields)
        lines.append(f'  printf("{sep}\\"{ctype}\\": {{\\"size\\": %zu, {offs}}}", sizeof({ctype}), {args});')
    lines += ['  printf("}\\n");', "  return 0;", "}"]
    src = d / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = d / "layout"
    subprocess.run([cc, "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                   check=True)
    return json.loads(subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout)


@pytest.mark.parametrize("ctype,cls,fields", LAYOUTS, ids=[l[0] for l in LAYOUTS])
def test_binding_matches_header(c_layouts, ctype, cls, fields):
    want = c_layouts[ctype]
    assert ctypes.sizeof(cls) == want["size"], ctype
    names = [f for f, _ in cls._fields_]
    for cname, pyname in zip(fields, names):
        assert getattr(cls, pyname).offset == want[cname], (ctype, cname)
