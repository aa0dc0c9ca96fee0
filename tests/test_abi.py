"""The C ABI library builds for sm_103a, loads, and exports every function
that include/wedge.h declares (no device calls: runs without a GPU)."""
import os
import re
import subprocess

import pytest

import paper_1903_07754_gb300 as pkg
from paper_1903_07754_gb300 import build as wbuild
from paper_1903_07754_gb300 import wedge

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADERS = [os.path.join(ROOT, "include", f) for f in os.listdir(os.path.join(ROOT, "include")) if f.endswith(".h")]


def _declared():
    names = set()
    for h in HEADERS:
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^\s*[A-Za-z_][\w\s\*]*?\b(wedge_\w+)\s*\(", text, flags=re.M):
            names.add(m.group(1))
    return names


@pytest.fixture(scope="module")
def lib():
    wbuild.build()
    return wedge.load()


def test_every_declared_symbol_is_exported(lib):
    declared = _declared()
    assert {"wedge_graph_create", "wedge_frontier_transform", "wedge_pull_iterate", "wedge_run_bfs",
            "wedge_run_cc", "wedge_run_sssp", "wedge_run_pr"} <= declared
    out = subprocess.run(["nm", "-D", "--defined-only", wbuild.LIB_PATH], capture_output=True, text=True,
                         check=True).stdout
    exported = {line.split()[-1] for line in out.splitlines() if " T " in line}
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
    assert (o.tau_bp, o.log2_coarsen, o.switch_mode) == (100, 3, wedge.SWITCH_THRESHOLD)
    o = wedge.wedge_default_opts("sssp")
    assert (o.tau_bp, o.log2_coarsen) == (2000, 2)
    assert isinstance(wedge.wedge_kernel_launches(), int)


def test_package_exports_c_names():
    for name in ("wedge_graph_create", "wedge_frontier_transform", "wedge_pull_iterate", "wedge_run_bfs",
                 "wedge_run_cc", "wedge_run_sssp", "wedge_run_pr"):
        assert callable(getattr(pkg, name))
