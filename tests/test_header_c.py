"""include/vegas.h as a C compiler sees it (host only, no GPU).

A C99 program compiled with every warning as an error includes the header, prints the
offset and size of every field of the four option/sample/statistics structs (the field
names coming from the Python binding, so a name missing from the header fails to compile),
takes the address of every declared function (so a missing export fails to link), and calls
the entry points that need no device. The test compares the compiler's layout with the
binding's ctypes layout field by field, and the field lists with the header's own.
"""

import ctypes as C
import os
import re
import shutil
import subprocess

import pytest

from conftest import ROOT

import paper_1803_07030_gb300 as vg
from paper_1803_07030_gb300 import vegas as vb

STRUCTS = [("vegas_sample", vb.vegas_sample), ("vegas_options", vb.vegas_options),
           ("vegas_stats_t", vb.vegas_stats_t), ("vegas_ising_options", vb.vegas_ising_options)]
HEADER = os.path.join(ROOT, "include", "vegas.h")


def header_fields(name):
    """Field names of a struct in the header, in order (comments stripped)."""
    text = re.sub(r"/\*.*?\*/", "", open(HEADER).read(), flags=re.S)
    m = re.search(r"typedef struct \{([^{}]*)\}\s*" + name + r";", text)
    assert m, name
    names = []
    for decl in m.group(1).split(";"):
        parts = decl.strip().split(",")
        if parts[0]:
            names += [re.findall(r"\w+", p)[-1] for p in parts]
    return names


def declared_functions():
    text = re.sub(r"/\*.*?\*/", "", open(HEADER).read(), flags=re.S)
    return sorted(set(re.findall(r"\b(vegas_[a-z_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def c_program(tmp_path_factory):
    if shutil.which("gcc") is None:
        pytest.skip("no C compiler")
    lib = vg.build()
    d = tmp_path_factory.mktemp("hdr")
    lines = ["#include <stddef.h>", "#include <stdio.h>", "#include <string.h>", '#include "vegas.h"', "",
             "typedef void (*fn_t)(void);", "int main(void) {"]
    for cname, _ in STRUCTS:
        lines.append(f'    printf("size {cname} %zu\\n", sizeof({cname}));')
    for cname, cls in STRUCTS:
        for f, _ in cls._fields_:
            lines.append(f'    printf("field {cname}.{f} %zu %zu\\n", offsetof({cname}, {f}), '
                         f'sizeof((({cname} *)0)->{f}));')
    funcs = declared_functions()
    lines.append("    fn_t fns[] = {" + ", ".join(f"(fn_t)(size_t){f}" for f in funcs) + "};")
    lines.append('    for (size_t i = 0; i < sizeof fns / sizeof fns[0]; ++i) if (!fns[i]) return 2;')
    lines += [
        "    vegas_options o; memset(&o, 0xff, sizeof o); vegas_default_options(&o);",
        '    printf("defaults %d %d %llu %d %d %d\\n", o.precision, o.replicas, (unsigned long long)o.seed, '
        'o.device, o.variant, o.graphs);',
        "    const int64_t rp[5] = {0, 2, 4, 6, 8}; const int32_t col[8] = {1, 3, 0, 2, 1, 3, 0, 2};",
        "    int32_t colour[4] = {-1, -1, -1, -1};",
        "    const int32_t nc = vegas_greedy_colour(4, rp, col, colour);",
        '    printf("ring %d %d %d %d %d\\n", nc, colour[0], colour[1], colour[2], colour[3]);',
        "    vegas_ctx *ctx = (vegas_ctx *)1;",
        "    const int st = (int)vegas_create(NULL, 0, NULL, &ctx);",
        '    printf("create %d %d\\n", st, ctx == NULL);',
        '    printf("message %d\\n", vegas_last_error(NULL) != NULL && vegas_last_error(NULL)[0] != 0);',
        "    vegas_destroy(NULL);",
        "    return 0;", "}"]
    src = d / "hdr.c"
    src.write_text("\n".join(lines) + "\n")
    exe = d / "hdr"
    cmd = ["gcc", "-std=c99", "-Wall", "-Wextra", "-pedantic", "-Werror", "-Wno-pedantic-ms-format",
           "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe), "-L", os.path.dirname(lib), "-lvegas",
           "-Wl,-rpath," + os.path.dirname(lib)]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0 and "pedantic-ms-format" in r.stderr:
        cmd.remove("-Wno-pedantic-ms-format")
        r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    run = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)
    assert run.returncode == 0, run.stdout + run.stderr
    return run.stdout.splitlines()


def test_struct_layouts_match_the_binding(c_program):
    sizes = {l.split()[1]: int(l.split()[2]) for l in c_program if l.startswith("size ")}
    fields = {l.split()[1]: (int(l.split()[2]), int(l.split()[3])) for l in c_program if l.startswith("field ")}
    for cname, cls in STRUCTS:
        assert sizes[cname] == C.sizeof(cls), cname
        assert [f for f, _ in cls._fields_] == header_fields(cname), cname
        for f, _ in cls._fields_:
            desc = getattr(cls, f)
            assert fields[f"{cname}.{f}"] == (desc.offset, desc.size), (cname, f)


def test_every_declared_function_links_and_host_calls_work(c_program):
    out = {l.split()[0]: l.split()[1:] for l in c_program if not l.startswith(("size ", "field "))}
    assert out["defaults"] == ["32", "1", "1", "-1", "-1", "1"]
    assert out["ring"] == ["2", "0", "1", "0", "1"]          # a 4-ring is 2-coloured
    assert out["create"] == [str(vb.EINVAL), "1"]            # no samples: EINVAL and *out = NULL
    assert out["message"] == ["1"]
    assert set(declared_functions()) == set(vb.SIGNATURES)
