"""Host-side helpers of bench.py (CPU): the traffic records read from the
profile summaries.

A record names the kernel, the problem's edge count, optionally the stored
message size, its unit of work (a candidate-iteration, a launch or a shot)
and the hash of the kernel sources it was captured with; a record whose
sources have changed since, or that belongs to another problem, is not
used, so the benchmark line reports null traffic instead of a stale figure.
"""
import os

import numpy as np

import pytest

import bench


def _tree(tmp_path, src_text):
    csrc = tmp_path / "paper_2512_07057_gb300" / "csrc"
    csrc.mkdir(parents=True)
    (csrc / "bsd_internal.cuh").write_text("// header\n")
    (csrc / "bsd_kernels.cu").write_text(src_text)
    (tmp_path / "profiles").mkdir()
    return tmp_path


def _record(root, name, kernel, unit, value, edges, msg_bytes=None):
    h = bench._source_hash(["bsd_internal.cuh", "bsd_kernels.cu"])
    lines = [f"# {kernel} traffic", "", "sources: bsd_internal.cuh bsd_kernels.cu", f"source_hash: {h}",
             f"kernel: {kernel}", f"edges: {edges}"]
    if msg_bytes is not None:
        lines.append(f"msg_bytes: {msg_bytes}")
    lines.append(f"bytes_per_{unit}: {value}")
    (root / "profiles" / name).write_text("\n".join(lines) + "\n")


@pytest.fixture
def tree(tmp_path, monkeypatch):
    root = _tree(tmp_path, "// kernels v1\n")
    monkeypatch.setattr(bench, "ROOT", str(root))
    return root


def test_record_units_and_filters(tree):
    _record(tree, "k_round_traffic_a.md", "k_round", "candidate_iteration", 44.13, 432)
    _record(tree, "k_seed_traffic_a4.md", "k_seed", "shot", 180.8, 6912, msg_bytes=4)
    _record(tree, "k_seed_traffic_a2.md", "k_seed", "shot", 179.9, 6912, msg_bytes=2)
    _record(tree, "k_u_var_traffic_a.md", "k_u_var", "launch", 197014355, 6912)
    assert bench._traffic_record("k_round", 432) == (44.13, "candidate_iteration")
    assert bench._traffic_record("k_round", 6912) is None                 # another problem
    assert bench._traffic_record("k_seed", 6912, 4) == (180.8, "shot")
    assert bench._traffic_record("k_seed", 6912, 2) == (179.9, "shot")
    assert bench._traffic_record("k_u_var", 6912) == (197014355.0, "launch")
    assert bench._traffic_record("k_select", 432) is None                 # no record


def test_record_goes_stale_when_the_sources_change(tree):
    _record(tree, "k_round_traffic_a.md", "k_round", "candidate_iteration", 44.13, 432)
    assert bench._traffic_record("k_round", 432) is not None
    (tree / "paper_2512_07057_gb300" / "csrc" / "bsd_kernels.cu").write_text("// kernels v2\n")
    assert bench._traffic_record("k_round", 432) is None


def test_committed_records_parse():
    """Every traffic record under profiles/ names its kernel, sources, hash,
    edges and exactly one unit of work."""
    import re
    prof = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "profiles")
    names = [n for n in os.listdir(prof) if "_traffic_" in n]
    assert names
    for n in names:
        txt = open(os.path.join(prof, n)).read()
        for key in ("kernel", "sources", "source_hash", "edges"):
            assert re.search(rf"^{key}: \S+", txt, re.M), (n, key)
        assert len(re.findall(r"^bytes_per_(candidate_iteration|launch|shot): [0-9.]+$", txt, re.M)) == 1, n


def _memory(root, name, kernel, edges, dram_bytes, duration_us, l2_hit_pct):
    h = bench._source_hash(["bsd_internal.cuh", "bsd_kernels.cu"])
    lines = [f"# {kernel} memory", "", "sources: bsd_internal.cuh bsd_kernels.cu", f"source_hash: {h}",
             f"kernel: {kernel}", f"edges: {edges}", "case: 200000 shots, p = 0.05",
             f"dram_bytes: {dram_bytes}", f"duration_us: {duration_us}", f"l2_hit_pct: {l2_hit_pct}"]
    (root / "profiles" / name).write_text("\n".join(lines) + "\n")


def test_memory_record_gives_dram_throughput_and_l2_hit(tree):
    """The measured DRAM throughput of one launch is its DRAM bytes over its
    duration; the L2 hit rate is passed through as a fraction; the record
    goes stale with the sources and is not used for another problem."""
    _memory(tree, "k_round_memory_a.md", "k_round", 432, 2.0e8, 500.0, 61.5)
    r = bench._memory_record("k_round", 432)
    assert abs(r["dram_gbs"] - 400.0) < 1e-9 and abs(r["l2_hit"] - 0.615) < 1e-12
    assert r["record"] == os.path.join("profiles", "k_round_memory_a.md")
    assert bench._memory_record("k_round", 6912) is None
    assert bench._memory_record("k_seed", 432) is None
    (tree / "paper_2512_07057_gb300" / "csrc" / "bsd_kernels.cu").write_text("// kernels v2\n")
    assert bench._memory_record("k_round", 432) is None


def test_ops_per_update_is_the_algorithmic_count():
    """Six ALU operations per message update: two for the compare-exchange
    into the row's two smallest magnitudes, one sign XOR, one signed select
    of the outgoing magnitude, one add into the posterior, one extrinsic
    subtraction."""
    assert bench.OPS_PER_UPDATE == 2 + 1 + 1 + 1 + 1


def _prof(kind_ms, kind_ln, exec_iters, screen=0):
    ms = np.zeros(12)
    ln = np.zeros(12, np.int64)
    for k, v in kind_ms.items():
        ms[k] = v
    for k, v in kind_ln.items():
        ln[k] = v
    return {"kinds": {"ms": ms, "launches": ln}, "exec_iters": np.array(exec_iters, np.uint64),
            "screen_updates": screen}


def test_roofline_picks_the_dominant_kernel_and_its_bound(monkeypatch):
    """The per-candidate round kernel is measured against the lane-operation
    peak (6 operations per message update), the batched error-node pass
    against HBM with its algorithmic bytes per slot iteration."""
    import types
    fake_torch = types.SimpleNamespace(cuda=types.SimpleNamespace(
        get_device_properties=lambda dev: types.SimpleNamespace(multi_processor_count=152)))
    monkeypatch.setitem(__import__("sys").modules, "torch", fake_torch)
    monkeypatch.setattr(bench, "peaks", lambda: ({"hbm_gbs": 6000.0, "sm_max_mhz": 2000.0}, "measured"))
    monkeypatch.setattr(bench, "_traffic_record", lambda *a, **k: None)
    monkeypatch.setattr(bench, "_memory_record", lambda *a, **k: None)
    E, M = 432, 72
    # k_round: 10 launches, 2 ms in all, 1e6 candidate-iterations
    r, _ = bench.alu_roofline([_prof({0: 0.5, 1: 2.0, 2: 0.1}, {0: 1, 1: 10, 2: 10}, [1000, 10**6, 0])], E, 0, "case",
                              M=M)
    peak = 152 * 128 * 2000e6 / 1e12
    assert r["kernel"] == "k_round" and r["bound"] == "alu" and abs(r["peak"] - peak) < 1e-9
    assert abs(r["achieved"] - 6 * (1e6 * E / 10) / (0.2e-3) / 1e12) < 1e-9
    assert abs(r["frac"] - r["achieved"] / peak) < 1e-12
    # k_bs_var dominant: 4 launches of 8 ms in all, 2048 slot iterations, 2-byte messages
    E2, M2 = 35110, 936
    r, _ = bench.alu_roofline([_prof({0: 1.0, 1: 0.2, 8: 3.0, 9: 8.0, 10: 1.0}, {0: 1, 1: 2, 8: 4, 9: 4, 10: 4},
                                     [3000, 50, 2048])], E2, 0, "case", msg_bytes=2, M=M2)
    assert r["kernel"] == "k_bs_var" and r["bound"] == "hbm" and r["unit"] == "GB/s"
    per_slot = 2 * 2 * E2 + 8 * M2
    assert abs(r["achieved"] - per_slot * (2048 / 4) / 2e-3 / 1e9) < 1e-6
    assert abs(r["frac"] - r["achieved"] / 6000.0) < 1e-12 and np.isfinite(r["alu_view"]["frac"])
