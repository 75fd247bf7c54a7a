"""The C-ABI library loads and exports every symbol include/eic.h declares (no GPU)."""
import ctypes
import os
import re
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2506_19349_gb300 import build

    build.build()
    from paper_2506_19349_gb300 import binding

    return binding.load_library()


def _declared():
    text = open(os.path.join(ROOT, "include", "eic.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(eic_[a-z_0-9]+)\s*\(", text)))


def test_header_declares_expected_entry_points():
    from paper_2506_19349_gb300 import binding

    assert set(_declared()) == set(binding.EXPORTS)


def test_library_exports_every_declared_symbol(lib):
    for name in _declared():
        assert hasattr(lib, name), name


def test_host_only_calls(lib):
    from paper_2506_19349_gb300 import binding

    p = binding.default_params()
    assert (p.alpha, p.beta, p.st_num, p.gap_shift, p.flags) == (3, 0.9, 1024, 0, 0)
    assert lib.eic_params_default(None) == binding.EINVAL
    for code in range(9):
        assert lib.eic_strerror(code) and lib.eic_strerror(code) != b"unknown status"
    assert lib.eic_strerror(99) == b"unknown status"
    assert lib.eic_version() >= 100
    out = ctypes.c_void_p()
    # argument checks happen before any device call
    assert lib.eic_graph_create(None, None, None, 0, 10, 0, None, None) == binding.EINVAL
    assert lib.eic_graph_create(None, None, None, 0, 0, 0, None, ctypes.byref(out)) == binding.EINVAL
    assert lib.eic_graph_create(None, None, None, 5, 10, 0, None, ctypes.byref(out)) == binding.EINVAL
    assert lib.eic_graph_info(None, None, None, None, None, None, None) == binding.EINVAL
    assert lib.eic_graph_destroy(None) == binding.OK
    assert lib.eic_sssp(None, 0, None, None, None, None, None) == binding.EINVAL
    assert lib.eic_sssp_batch(None, None, 0, None, None, None, None) == binding.OK
    assert lib.eic_sssp_batch(None, None, 3, None, None, None, None) == binding.EINVAL
    assert lib.eic_batch_create(None, None, 1, None, None, None) == binding.EINVAL
    assert lib.eic_batch_create(None, None, 1, None, None, ctypes.byref(out)) == binding.EINVAL
    assert lib.eic_batch_run(None, None) == binding.EINVAL
    assert lib.eic_batch_wait(None, None, None) == binding.EINVAL
    assert lib.eic_batch_tune(None, None, None) == binding.EINVAL
    assert lib.eic_batch_info(None, None) == binding.EINVAL
    assert lib.eic_batch_destroy(None) == binding.OK
    t = ctypes.c_uint64()
    assert lib.eic_server_create(None, 0, None, None, ctypes.byref(out)) == binding.EINVAL
    assert lib.eic_server_create(None, 1, None, None, None) == binding.EINVAL
    assert lib.eic_server_submit(None, 0, 0, ctypes.byref(t)) == binding.EINVAL
    assert lib.eic_server_poll(None, 0, None) == binding.EINVAL
    assert lib.eic_server_wait(None, 0, 1, None) == binding.EINVAL
    assert lib.eic_server_result(None, 0, None, None, None) == binding.EINVAL
    assert lib.eic_server_release(None, 0) == binding.EINVAL
    assert lib.eic_server_stats(None, None) == binding.EINVAL
    assert lib.eic_server_reset_stats(None) == binding.EINVAL
    assert lib.eic_server_tune(None, None, None) == binding.EINVAL
    assert lib.eic_server_destroy(None) == binding.OK


def test_struct_layouts_match_the_header():
    from paper_2506_19349_gb300 import binding

    # eic_params: u32, (pad), f64, 6 x u32, batch_groups, reserved[7]
    assert ctypes.sizeof(binding.Params) == 4 + 4 + 8 + 6 * 4 + 4 + 7 * 4
    assert binding.Params.batch_groups.offset == 40
    # eic_batch_config: 8 x u32, u64, f64
    assert ctypes.sizeof(binding.BatchConfig) == 8 * 4 + 8 + 8


def test_ctypes_mirrors_match_the_c_layout(tmp_path):
    """sizeof/offsetof of the header's structs, compiled by the C compiler,
    equal the binding's ctypes mirrors."""
    import shutil
    import subprocess

    from paper_2506_19349_gb300 import binding

    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    checks = {"eic_params": (binding.Params, ["beta", "st_num", "flags", "batch_groups", "reserved"]),
              "eic_step": (binding.Step, ["lb", "ub", "st", "gap_lb", "sumd_lb", "highd_lb", "rounds", "settled",
                                          "flags", "reserved"]),
              "eic_stats": (binding.Stats, ["steps", "pull_items", "trace", "trace_cap", "trace_len", "timeline",
                                            "timeline_cap", "timeline_len", "kernel_ms"]),
              "eic_batch_config": (binding.BatchConfig, ["groups", "queries", "scratch_bytes", "tuned_ms"]),
              "eic_server_config": (binding.ServerConfig, ["groups", "ring_entries", "output_bytes", "idle_us",
                                                            "reserved"]),
              "eic_server_report": (binding.ServerReport, ["submitted", "kernel_launches", "scratch_bytes", "groups",
                                                            "blocks_per_group", "latency_p50_ms", "latency_count"])}
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "eic.h"', "int main(void) {"]
    for st, (_, fields) in checks.items():
        lines.append(f'  printf("{st} %zu\\n", sizeof({st}));')
        for f in fields:
            lines.append(f'  printf("{st}.{f} %zu\\n", offsetof({st}, {f}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = dict(line.split() for line in subprocess.run([str(exe)], check=True, capture_output=True,
                                                        text=True).stdout.splitlines())
    for st, (cls, fields) in checks.items():
        assert int(got[st]) == ctypes.sizeof(cls), st
        for f in fields:
            assert int(got[f"{st}.{f}"]) == getattr(cls, f).offset, f"{st}.{f}"


def test_traffic_key_ignores_comments_only():
    """The bench's measured-traffic key hashes kernel code without comments:
    comment and blank-line edits keep it, code edits change it, and comment
    markers inside string literals are code."""
    sys.path.insert(0, ROOT)
    import bench

    strip = bench.strip_c_comments
    base = 'int f(int x) {\n  return x + 1;  // add one\n}\n'
    assert strip(base) == strip('/* header */\nint f(int x) {\n\n  return x + 1;\n}  // end\n')
    assert strip(base) != strip(base.replace("x + 1", "x + 2"))
    code = 'asm("ld.global // not a comment /* nor this */ %0;" : "=r"(v));'
    assert strip(code) == code
    assert strip("char c = '/'; // tail") == "char c = '/';"
    assert strip('s = "a\\"//b"; // c') == 's = "a\\"//b";'


def test_product_path_never_imports_the_oracle():
    """Importing the package, its binding, its generators and build step (in a
    fresh interpreter) loads nothing from oracle/; and no product source
    imports it or loads its library."""
    import subprocess

    code = ("import sys; sys.path.insert(0, %r)\n"
            "import paper_2506_19349_gb300, paper_2506_19349_gb300.binding, paper_2506_19349_gb300.build\n"
            "import paper_2506_19349_gb300.graphgen\n"
            "print(any(m == 'oracle' or m.startswith('oracle.') for m in sys.modules))\n") % ROOT
    out = subprocess.run([sys.executable, "-c", code], check=True, capture_output=True, text=True).stdout.strip()
    assert out == "False"
    pkg = os.path.join(ROOT, "paper_2506_19349_gb300")
    for base, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".c")):
                with open(os.path.join(base, f), encoding="utf-8") as fh:
                    assert not re.search(r"^\s*(import|from)\s+oracle\b|liboracle|oracle/", fh.read(), re.M), \
                        os.path.join(base, f)


def test_binding_noalloc_limits_equal_the_header():
    from paper_2506_19349_gb300 import binding

    text = open(os.path.join(ROOT, "include", "eic.h")).read()
    for name in ("VERTICES", "ENTRIES", "WEIGHT", "DEGREES", "STEPS"):
        m = re.search(rf"#define EIC_NOALLOC_MAX_{name} \(?(1u << (\d+)|(\d+)u)\)?", text)
        assert m, name
        val = 1 << int(m.group(2)) if m.group(2) else int(m.group(3))
        assert getattr(binding, f"NOALLOC_MAX_{name}") == val, name
