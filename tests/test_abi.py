"""The C ABI library builds for sm_103a, loads, and exports every function
that include/wedge.h declares; the benchmark's probe library does the same
for include/wedge_probe.h (no device calls: runs without a GPU)."""
import os
import re
import subprocess

import pytest

import paper_1903_07754_gb300 as pkg
from paper_1903_07754_gb300 import build as wbuild
from paper_1903_07754_gb300 import wedge

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "wedge.h")
PROBE_HEADER = os.path.join(ROOT, "include", "wedge_probe.h")


def _declared(headers=(HEADER,)):
    names = set()
    for h in headers:
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^\s*[A-Za-z_][\w\s\*]*?\b(wedge_\w+)\s*\(", text, flags=re.M):
            names.add(m.group(1))
    return names


@pytest.fixture(scope="module")
def lib():
    wbuild.build()
    return wedge.load()


def _exported(path):
    out = subprocess.run(["nm", "-D", "--defined-only", path], capture_output=True, text=True, check=True).stdout
    return {line.split()[-1] for line in out.splitlines() if " T " in line}


def test_headers_are_the_engine_and_the_probe():
    assert sorted(f for f in os.listdir(os.path.join(ROOT, "include")) if f.endswith(".h")) == \
        ["wedge.h", "wedge_probe.h"]


def test_probe_library_is_separate(lib):
    from paper_1903_07754_gb300 import probe
    declared = _declared((PROBE_HEADER,))
    assert declared == set(probe.EXPORTS) == {"wedge_probe_gather"}
    assert declared <= _exported(wbuild.PROBE_LIB_PATH)
    assert not (declared & _exported(wbuild.LIB_PATH)), "the engine library must not carry the probe"
    assert hasattr(probe.load(), "wedge_probe_gather")


def test_every_declared_symbol_is_exported(lib):
    declared = _declared()
    assert {"wedge_graph_create", "wedge_frontier_transform", "wedge_pull_iterate", "wedge_run_bfs",
            "wedge_run_cc", "wedge_run_sssp", "wedge_run_pr"} <= declared
    exported = _exported(wbuild.LIB_PATH)
    missing = declared - exported
    assert not missing, f"declared but not exported: {sorted(missing)}"
    for name in declared:
        assert hasattr(lib, name)
    assert set(wedge.EXPORTS) == declared


def test_build_targets_sm_103a_only():
    assert wbuild.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]


def test_host_only_entry_points(lib):
    assert wedge.wedge_version().startswith("wedge-gb300")
    o = wedge.wedge_default_opts("bfs")
    assert (o.tau_bp, o.log2_coarsen, o.switch_mode) == (100, 0, wedge.SWITCH_THRESHOLD)
    o = wedge.wedge_default_opts("sssp")
    assert (o.tau_bp, o.log2_coarsen) == (2000, 0xFFFFFFFF)  # 16-edge entries
    assert isinstance(wedge.wedge_kernel_launches(), int)


def test_package_exports_c_names():
    for name in ("wedge_graph_create", "wedge_frontier_transform", "wedge_pull_iterate", "wedge_run_bfs",
                 "wedge_run_cc", "wedge_run_sssp", "wedge_run_pr"):
        assert callable(getattr(pkg, name))


_C_TYPES = {"uint32_t": ("u", 4), "uint64_t": ("u", 8), "int": ("i", 4), "double": ("f", 8), "float": ("f", 4)}


def _header_structs():
    """{name: [(field, kind, size, count)]} for every `typedef struct {...} name;`."""
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    out = {}
    for m in re.finditer(r"typedef\s+struct\s*\{(.*?)\}\s*(\w+)\s*;", text, flags=re.S):
        fields = []
        for decl in m.group(1).split(";"):
            decl = decl.strip()
            if not decl:
                continue
            fm = re.fullmatch(r"(\w+)\s+(\w+)(?:\[(\d+)\])?", decl)
            assert fm, decl
            kind, size = _C_TYPES[fm.group(1)]
            fields.append((fm.group(2), kind, size, int(fm.group(3) or 1)))
        out[m.group(2)] = fields
    return out


def _ctypes_fields(cls):
    import ctypes
    res = []
    for name, t in cls._fields_:
        count = 1
        if issubclass(t, ctypes.Array):
            count, t = t._length_, t._type_
        kind = "f" if t in (ctypes.c_double, ctypes.c_float) else ("i" if t in (ctypes.c_int, ctypes.c_int32) else "u")
        res.append((name, kind, ctypes.sizeof(t), count))
    return res


def test_binding_structs_match_the_header():
    """The ctypes mirrors have the header's fields, in order, with the same
    widths (a drifted struct would shift every later option)."""
    structs = _header_structs()
    assert {"wedge_opts", "wedge_stats", "wedge_iter_record", "wedge_tuning", "wedge_graph_info"} <= set(structs)
    for name, fields in structs.items():
        cls = getattr(wedge, name)
        assert _ctypes_fields(cls) == fields, name


def test_default_opts_leave_the_extensions_off(lib):
    for app in ("bfs", "cc", "sssp", "pr"):
        o = wedge.wedge_default_opts(app)
        assert (o.synchronous, o.sparse_push, o.trace, o.max_iters) == (0, 0, 0, 0)
        assert list(o.reserved) == [0]


def test_argument_checks_before_any_device_work(lib):
    """Malformed calls are rejected on the host with INVALID_ARG and a
    message, before any CUDA call (so these run without a GPU)."""
    L = lib
    cases = [
        (lambda: L.wedge_csc_relabel_by_degree(0, 0, None, None, None, None, None, None, None, None, None), "V must be"),
        (lambda: L.wedge_csc_relabel_by_degree(4, 1 << 40, None, None, None, None, None, None, None, None, None),
         "E must be"),
        (lambda: L.wedge_permute_rows(0, 1, None, None, None, None), "V and width"),
        (lambda: L.wedge_permute_rows(4, 0, None, None, None, None), "V and width"),
        (lambda: L.wedge_cc_labels_to_original(0, None, None, None, None, None), "V must be"),
        (lambda: L.wedge_pr_order(None, None, None), "NULL"),
        (lambda: L.wedge_pr_pull_ordered(None, None, None, None), "NULL"),
        (lambda: L.wedge_run_bfs_batch_u8(None, None, None, 1, 1, None, None, None, None), "NULL"),
        (lambda: L.wedge_graph_create(0, 0, None, None, None, None, None, 32, None, None), "out is NULL"),
    ]
    for call, text in cases:
        st = call()
        assert st == 1, (text, st)  # WEDGE_ERR_INVALID_ARG
        assert text in wedge.wedge_last_error(), (text, wedge.wedge_last_error())
