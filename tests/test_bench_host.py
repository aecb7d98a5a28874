"""Host logic of bench.py on CPU: the units of a step, the oracle's throughput on the step's unit
mix, the autotuner's source, and the reference arm's line (same config as the GPU arm)."""
import json
import os
import subprocess
import sys

import numpy as np

import bench
import oracle
from paper_1911_09135_gb300 import graphgen as gg

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_unit_counts_follow_their_definitions():
    # 0-1-2 path plus an isolated vertex 3 and a separate edge 4-5 (symmetric)
    g = gg.from_edges(6, [(0, 1), (1, 2), (4, 5)], [1, 1, 1], symmetrize=True, name="t")
    deg = g.degrees()
    inf = bench.INF
    lv = np.array([0, 1, 2, inf, inf, inf], dtype=np.uint32)
    core = np.array([1, 1, 0, 0, 1, 1], dtype=np.uint32)   # peeled: 2 and 3
    u = bench.unit_counts(g, {"bfs": lv, "sssp": lv, "cc": None, "kcore": core, "pr": None}, 7)
    assert u["bfs"] == u["sssp"] == int(deg[:3].sum()) == 4
    assert u["cc"] == g.m == 6
    assert u["kcore"] == int(deg[2] + deg[3]) == 1
    assert u["pr"] == 7 * g.m


def test_mix_rate_weights_each_app_by_its_units():
    # app a: 10 units in 1 s (10/s); app b: 30 units in 1 s over two samples (15/s)
    samples = {"a": [(10, 1.0)], "b": [(10, 1.0), (20, 1.0)]}
    step = {"a": 20, "b": 30}          # 2 s + 2 s for 50 units
    assert abs(bench.mix_rate(step, samples) - 12.5) < 1e-12


def test_tune_source_is_a_non_isolated_vertex_other_than_the_source():
    g = gg.rmat(10, 16 << 10, 3, symmetrize=True)
    src = g.max_degree_vertex()
    t = bench.tune_source(g, src)
    assert t != src and g.degrees()[t] > 0 and t == bench.tune_source(g, src)


def test_reference_arm_line_has_the_gpu_arms_config():
    out = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--workload", "rmat16",
                          "--steps", "2", "--warmup", "1"], cwd=ROOT, capture_output=True, text=True,
                         timeout=600, env=dict(os.environ, CUDA_VISIBLE_DEVICES=""))
    assert out.returncode == 0, out.stderr[-3000:]
    d = json.loads([ln for ln in out.stdout.splitlines() if ln.startswith("{")][-1])
    g, desc, apps = bench.workload("rmat16")
    assert d["config"] == json.loads(json.dumps(bench.step_config(g, desc, apps, g.max_degree_vertex(), 1)))
    lv = oracle.bfs(g.n, g.offsets, g.indices, g.max_degree_vertex())
    assert d["per_app"]["bfs"]["units"] == bench.unit_counts(g, {"bfs": lv}, 0)["bfs"]
    assert d["impl"] == "reference" and d["steps"] == 2 and d["value"] > 0
