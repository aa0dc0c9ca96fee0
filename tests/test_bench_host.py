"""Host-side arithmetic of bench.py (no GPU): credited edges, the
gather-rate bound, the measured-peak file, and the digest that ties the
committed ncu counters to the device code they were taken on."""
import os
import shutil
import types

import numpy as np

import bench
import graphgen as gg
import oracle


def test_credited_edges_is_the_out_degree_sum_of_reached_vertices():
    g = gg.rmat(10, 8)
    lvl = oracle.bfs_push(g, 0)
    reached = lvl != oracle.INF
    od = oracle.outdeg(g)
    # Graph500 style: every edge leaving a reached vertex, counted once
    want = int(g.src.size) - int(od[~reached].sum())
    assert bench.credited_edges(od, reached) == want
    assert bench.credited_edges(od, np.zeros(g.V, dtype=bool)) == 0


def test_gather_bound_arithmetic(monkeypatch):
    props = types.SimpleNamespace(multi_processor_count=152)
    import torch
    monkeypatch.setattr(torch.cuda, "get_device_properties", lambda dev: props)
    edges, t, probe_t = 65_000_000, 0.25e-3, 0.2e-3
    b = bench._gather_bound(torch, 0, edges, t, {"sm_mhz": 2000.0}, probe_t)
    assert abs(b["peak"] - 152 * 2.0) < 1e-9
    assert abs(b["achieved"] - edges / t / 1e9) < 1e-9
    assert abs(b["frac"] - b["achieved"] / b["peak"]) < 1e-12
    assert abs(b["measured_peak"] - edges / probe_t / 1e9) < 1e-9
    assert abs(b["frac_of_measured"] - probe_t / t) < 1e-12
    assert "measured_peak" not in bench._gather_bound(torch, 0, edges, t, None)
    lib_t = 0.3e-3
    b = bench._gather_bound(torch, 0, edges, t, None, probe_t, lib_t)
    assert abs(b["library_gather"] - edges / lib_t / 1e9) < 1e-9
    assert abs(b["frac_of_library_gather"] - lib_t / t) < 1e-12


def test_measured_peaks_are_used_when_present():
    peak, kind = bench.peaks()
    if os.path.exists(os.path.join(bench.ROOT, "MEASURED_PEAKS.json")):
        assert kind == "measured" and peak > 1000
    else:
        assert (peak, kind) == (6800.0, "fallback")


def _digest_of(tmp_path, monkeypatch, edit=None):
    csrc = tmp_path / "paper_1903_07754_gb300" / "csrc"
    if not csrc.exists():
        shutil.copytree(os.path.join(bench.ROOT, "paper_1903_07754_gb300", "csrc"), csrc)
    if edit:
        name, old, new = edit
        p = csrc / name
        text = p.read_text()
        assert old in text
        p.write_text(text.replace(old, new, 1))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    return bench._kernel_digest()


def test_digest_follows_device_code_only(tmp_path, monkeypatch):
    base = _digest_of(tmp_path, monkeypatch)
    # comments and the host part of common.cuh do not count
    assert _digest_of(tmp_path, monkeypatch, ("pull.cuh", "namespace wedge {", "namespace wedge {\n// a note")) == base
    assert _digest_of(tmp_path, monkeypatch, ("common.cuh", "struct wedge_graph {",
                                              "struct wedge_graph {\n    int unused_host_field = 0;")) == base
    # nor does code of other kernels or of the host side
    assert _digest_of(tmp_path, monkeypatch, ("xform.cuh", "constexpr unsigned kAppendStage = 256;",
                                              "constexpr unsigned kAppendStage = 128;")) == base
    assert _digest_of(tmp_path, monkeypatch, ("engine.cu", "static PullParams pull_params(",
                                              "static PullParams  pull_params(")) == base
    assert _digest_of(tmp_path, monkeypatch, ("pull.cuh", "constexpr unsigned long long kSkipVisitedMinChunks",
                                              "constexpr unsigned long long  kSkipVisitedMinChunks")) == base
    # the pull's device code does (edits accumulate on the copy: this one last)
    assert _digest_of(tmp_path, monkeypatch, ("common.cuh", "constexpr unsigned kFull = 0xFFFFFFFFu;",
                                              "constexpr unsigned kFull = 0xFFFFFFFFu + 0u;")) != base


def test_committed_ncu_counters_belong_to_the_current_device_code():
    """Every committed capture's digest is the current one (a change of a
    kernel's device code must come with a new capture, or its counters go
    back to pending), so bench.py never reports stale counters."""
    for key, (val, us, digest) in bench.TRAFFIC.items():
        if val is None:
            assert us is None and digest is None, key
        else:
            assert digest == bench._kernel_digest(key), key
            assert bench._traffic(key) == val


def test_balance_summary_arithmetic():
    # three warps over a 100 ns span: busy 100, 50 and 10 ns -> idle 1 - 160/300
    rec = np.zeros((3, 2, 4), dtype=np.uint64)
    rec[:, 0, 0] = [1000, 1000, 1050]
    rec[:, 0, 1] = [1100, 1050, 1060]
    rec[:, 0, 2] = [200, 100, 20]
    b = bench.balance_summary(rec, 0)
    assert abs(b["span_us"] - 0.1) < 1e-12
    assert abs(b["idle_frac"] - (1 - 160 / 300)) < 1e-12
    assert abs(b["busy_max_over_mean"] - 100 / (160 / 3)) < 1e-12
    assert abs(b["cycles_max_over_mean"] - 200 / (320 / 3)) < 1e-12
