"""Host-side logic of the benchmark and the autotuner (no GPU): the
algorithmic byte counts behind the roofline, the guard that keeps a DRAM
traffic figure only while the kernel source it was captured on is unchanged,
and the autotuner's result cache."""
import hashlib
import json
import os
import sys
import types

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402
import meshgen  # noqa: E402
import oracle  # noqa: E402


def _counts(n):
    """Closed-form sizes of the n^3 x 6 Kuhn grid: nodes, edges (axis, face
    diagonal and body diagonal edges), boundary triangles, boundary nodes."""
    nv = (n + 1) ** 3
    ne = 3 * n * (n + 1) ** 2 + 3 * n * n * (n + 1) + n ** 3
    return nv, ne, 12 * n * n, (n + 1) ** 3 - (n - 1) ** 3


def test_closed_form_counts_match_a_built_grid():
    m = meshgen.generate.kuhn_cube(3, 0.2, permute=True, morton=True)
    t = oracle.topology(3, m.elems, m.x)
    nv, ne, nb, nbn = _counts(3)
    assert (m.n_nodes, t.n_edges, len(t.bface), len(t.bnode)) == (nv, ne, nb, nbn)


def test_algorithmic_bytes_of_the_benchmark_grid():
    """The per-step byte counts quoted for the 160^3 grid: 74 B/tet forward
    (1.82 GB) and 108 B/tet fused (2.65 GB); the fused step reads the mesh
    once, so fused = forward + adjoint - mesh inputs."""
    n = 160
    nv, ne, nb, nbn = _counts(n)
    m = types.SimpleNamespace(n_elems=6 * n ** 3, n_nodes=nv, dim=3)
    topo = types.SimpleNamespace(n_edges=ne, n_bfaces=nb, n_bnodes=nbn)
    fwd = bench.algorithmic_bytes(m, topo, "fwd", "tiled")
    adj = bench.algorithmic_bytes(m, topo, "adj", "tiled")
    fused = bench.algorithmic_bytes(m, topo, "fused", "tiled")
    mesh_in = 16 * m.n_elems + 24 * m.n_elems + 24 * nv + 16 * nb + 4 * nbn
    assert fused == fwd + adj - mesh_in
    assert round(fwd / m.n_elems) == 74 and abs(fwd / 1e9 - 1.82) < 0.005
    assert round(fused / m.n_elems) == 108 and abs(fused / 1e9 - 2.65) < 0.005
    assert fused == 2646684280            # the figure in the benchmark line's roofline


def test_kernel_traffic_requires_the_captured_source(tmp_path, monkeypatch):
    src = tmp_path / "k.cu"
    src.write_text("// kernel source\n")
    (tmp_path / "profiles").mkdir()
    entry = {"source": "k.cu", "source_sha1": hashlib.sha1(src.read_bytes()).hexdigest(),
             "dram_bytes_per_launch": 1000, "tile_nodes": 256, "scale_to_full": 2.5}
    (tmp_path / "profiles" / "traffic.json").write_text(json.dumps({"kern|tile256": entry}))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.kernel_traffic("kern", 256) == pytest.approx(2500.0)
    assert bench.kernel_traffic("kern", 96) is None          # captured at another tile size
    assert bench.kernel_traffic("other", 256) is None
    src.write_text("// kernel source, changed\n")
    assert bench.kernel_traffic("kern", 256) is None         # source changed since the capture
    # several sources: a change in a header with device code drops the figure too
    hdr = tmp_path / "k.cuh"
    hdr.write_text("// device helpers\n")
    entry = {"sources": ["k.cu", "k.cuh"], "dram_bytes_per_launch": 1000, "tile_nodes": 256, "scale_to_full": 1.0}
    entry["source_sha1"] = hashlib.sha1(src.read_bytes() + hdr.read_bytes()).hexdigest()
    (tmp_path / "profiles" / "traffic.json").write_text(json.dumps({"kern|tile256": entry}))
    assert bench.kernel_traffic("kern", 256) == pytest.approx(1000.0)
    hdr.write_text("// device helpers, changed\n")
    assert bench.kernel_traffic("kern", 256) is None


def _device_sources(cu):
    """The .cu file and every csrc header it includes, directly or through
    other csrc headers (the public header holds no device code)."""
    import re
    d = os.path.dirname(cu)
    seen, todo = [], [cu]
    while todo:
        f = todo.pop(0)
        if f in seen:
            continue
        seen.append(f)
        for inc in re.findall(r'#include "([^"/]+)"', open(os.path.join(ROOT, f)).read()):
            todo.append(os.path.join(d, inc))
    return sorted(seen)


def test_committed_figures_cover_the_kernels_includes():
    for name in ("traffic.json", "fp64_ops.json"):
        j = json.load(open(os.path.join(ROOT, "profiles", name)))
        for key, ent in j.items():
            if key.startswith("_"):
                continue
            assert sorted(ent["sources"]) == _device_sources(ent["sources"][0]), (name, key)


def test_committed_traffic_matches_its_source():
    """Every committed traffic figure names source files that exist and
    carries their current checksum (otherwise the benchmark drops it)."""
    j = json.load(open(os.path.join(ROOT, "profiles", "traffic.json")))
    for key, ent in j.items():
        if key.startswith("_"):      # notes
            continue
        for rel in ent["sources"]:
            assert os.path.exists(os.path.join(ROOT, rel)), (key, rel)
        assert bench.sources_sha1(ent) == ent["source_sha1"], key
        assert ent["dram_bytes_per_launch"] > 0 and ent["scale_to_full"] > 0


def test_committed_fp64_counts_match_their_source():
    """The FP64 instruction counts behind the ALU ceiling of the native-FP64
    forms: every entry names its kernel's source at the captured checksum, and
    the benchmark reads them back."""
    j = json.load(open(os.path.join(ROOT, "profiles", "fp64_ops.json")))
    kernels = [k for k in j if not k.startswith("_")]
    assert "k_fwd_atomic3<fp64>" in kernels
    for key in kernels:
        ent = j[key]
        assert bench.sources_sha1(ent) == ent["source_sha1"], key
        per = ent["fp64_pipe_thread_inst"] / ent["elements"]
        assert abs(per - ent["fp64_ops_per_element"]) < 0.01
        assert bench.fp64_ops(key) == pytest.approx(ent["fp64_ops_per_element"])
    assert bench.fp64_peak_ops() == pytest.approx(2 * 152 * 2.07e9)


def test_autotune_cache_roundtrip(tmp_path, monkeypatch):
    pytest.importorskip("torch")
    from paper_2502_00778_gb300 import autotune
    monkeypatch.setenv("EM_AUTOTUNE_CACHE", str(tmp_path / "sub" / "cache.json"))
    assert autotune._load() == {}
    d = {"k": {"path": "tiled", "tile_nodes": 256, "ms": 4.6, "sweep": {"tiled/256": 4.6}}}
    autotune._store(d)
    assert autotune._load() == d
    (tmp_path / "sub" / "cache.json").write_text("{not json")
    assert autotune._load() == {}                            # a damaged cache is ignored
    assert 256 in autotune.CANDIDATES and all(t % 32 == 0 for t in autotune.CANDIDATES)


def test_oracle_sample_is_self_contained():
    """The oracle sample timed for the CPU baseline: the first elements of
    the grid renumbered onto exactly the nodes they use."""
    m = meshgen.generate.kuhn_cube(4, 0.2, permute=True, morton=True)
    el, x, topo, w, c = bench.oracle_sample(m, 100)
    assert el.shape[0] == 100
    used = np.unique(el[:, :4])
    assert np.array_equal(used, np.arange(x.shape[0]))      # every sampled node used, ids dense
    assert np.array_equal(np.sort(m.x[np.unique(m.elems[:100, :4])], axis=0), np.sort(x, axis=0))
    assert w.shape == (topo.n_edges, 3) and c.shape == (x.shape[0],)


@pytest.mark.parametrize("dim", [2, 3])
def test_multicore_baseline_computes_the_oracle_result(dim):
    """The benchmark's all-cores CPU baseline (the oracle's element arithmetic
    with its loops split over threads, atomic accumulation) gives the serial
    oracle's forward and gradient up to summation order."""
    try:
        oracle.lib_omp()
    except Exception as ex:  # gcc without OpenMP: the benchmark reports it unavailable
        pytest.skip(f"oracle_omp not built: {ex}")
    if dim == 3:
        m = meshgen.kuhn_cube(9, jitter=0.25, seed=611, offset=1000.0)
    else:
        m = meshgen.tri_square(17, jitter=0.3, seed=612)
    t = oracle.topology(dim, m.elems, m.x)
    w, c = meshgen.generate.loss_weights(t.n_edges, m.n_nodes, dim)
    rn, rv, rb = oracle.direct(dim, m.x, m.elems, t)
    rg = oracle.adjoint(dim, m.x, m.elems, t, w, c)
    for threads in (1, 4):
        n, v, b, g = oracle.fused_omp(dim, m.x, m.elems, t, w, c, threads=threads)
        assert np.abs(n - rn).max() <= 1e-12 * m.h ** (dim - 1)
        assert np.abs(v - rv).max() <= 1e-12 * m.h ** dim
        assert np.abs(b - rb).max() <= 1e-12 * m.h ** (dim - 1)
        assert np.abs(g - rg).max() <= 1e-12 * np.abs(rg).max()
