"""The ctypes structures of the binding have the layout of the C structures in
include/alb.h: gcc compiles a small program against the header that prints
the size of each structure and the offset of each field, and the test
compares them with ctypes' own sizes and offsets (no GPU, no library load)."""
import ctypes
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

STRUCTS = ("alb_config", "alb_stats", "alb_batch_tuning", "alb_server_config", "alb_request",
           "alb_result", "alb_server_stats")


def binding_structs():
    from paper_2009_13426_gb300 import alb
    return {name: getattr(alb, name) for name in STRUCTS}


def c_layout(tmp_path, structs):
    gcc = shutil.which("gcc") or shutil.which("cc")
    if gcc is None:
        pytest.skip("no C compiler")
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "alb.h"', "int main(void) {"]
    for name, cls in structs.items():
        lines.append('  printf("%s %%zu\\n", sizeof(%s));' % (name, name))
        for field in cls._fields_:
            f = field[0]
            lines.append('  printf("%s.%s %%zu\\n", offsetof(%s, %s));' % (name, f, name, f))
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    exe = tmp_path / "layout"
    src.write_text("\n".join(lines) + "\n")
    subprocess.run([gcc, "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                   check=True, capture_output=True, text=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout
    return dict((k, int(v)) for k, v in (line.split() for line in out.splitlines()))


def test_binding_structures_match_the_header(tmp_path):
    structs = binding_structs()
    c = c_layout(tmp_path, structs)
    for name, cls in structs.items():
        assert ctypes.sizeof(cls) == c[name], name
        for field in cls._fields_:
            f = field[0]
            assert getattr(cls, f).offset == c["%s.%s" % (name, f)], (name, f)


def test_stats_fields_follow_the_header_order():
    """alb_stats is a run of uint64 counters: the binding names them in the
    header's order, including the FP32 form's multiplicative-update count."""
    import re
    src = open(os.path.join(ROOT, "include", "alb.h")).read()
    body = re.search(r"typedef struct \{(.*?)\} alb_stats;", src, flags=re.S).group(1)
    body = re.sub(r"/\*.*?\*/", "", body, flags=re.S)
    names = re.findall(r"uint64_t\s+(\w+)\s*;", body)
    from paper_2009_13426_gb300 import alb
    assert [f[0] for f in alb.alb_stats._fields_] == names
    assert "fp64_updates" in names
