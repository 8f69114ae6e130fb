"""CPU checks of bench.py's contract: the reference arm (the oracle on the
host) prints one JSON line with the fields the driver reads, the other ranks
of a multi-rank launch exit without work, and the served trace is seeded."""
import json
import os
import subprocess
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(args, env_extra=None, timeout=300):
    env = dict(os.environ)
    env.update(env_extra or {})
    p = subprocess.run([sys.executable, "bench.py"] + args, cwd=ROOT, env=env, capture_output=True, text=True,
                       timeout=timeout)
    return p


def test_reference_arm_prints_one_contract_line():
    p = _run(["--impl", "reference", "--steps", "1", "--warmup", "0"])
    assert p.returncode == 0, p.stderr[-2000:]
    lines = [l for l in p.stdout.splitlines() if l.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["metric"] == "PNE terms contracted/sec" and d["unit"] == "terms/s"
    assert d["value"] > 0 and d["higher_is_better"] is True and d["steps"] == 1
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": "terms/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    assert d["config"]["workload"].startswith("2D random-tensor network 16x16")


def test_reference_arm_other_ranks_exit_without_work():
    p = _run(["--impl", "reference", "--steps", "1", "--warmup", "0"], {"RANK": "1", "WORLD_SIZE": "2"},
             timeout=120)
    assert p.returncode == 0, p.stderr[-2000:]
    assert p.stdout.strip() == ""


def test_served_trace_is_seeded_and_poisson_like():
    sys.path.insert(0, ROOT)
    import bench
    t1, r1 = bench.serve_trace(400, 2000.0, 7)
    t2, r2 = bench.serve_trace(400, 2000.0, 7)
    assert np.array_equal(t1, t2) and r1 == r2
    gaps = np.diff(np.concatenate([[0.0], t1]))
    assert np.all(gaps >= 0)
    assert 0.5 / 2000.0 < gaps.mean() < 2.0 / 2000.0          # mean inter-arrival near 1 / rate
    kinds = {r[0] for r in r1}
    assert kinds == {"aklt", "rand3d"}
    assert all(4 <= r[3] <= 8 for r in r1)                    # orders K in 4..8


def test_every_registered_workload_is_defined():
    # the extras table names functions resolved only when the default run
    # reaches it on a GPU; check here that each one exists
    import ast
    src = open(os.path.join(ROOT, "bench.py")).read()
    tree = ast.parse(src)
    defined = {n.name for n in tree.body if isinstance(n, ast.FunctionDef)}
    called = set()
    for node in ast.walk(tree):
        if isinstance(node, ast.Tuple) and len(node.elts) == 2 and isinstance(node.elts[0], ast.Constant) \
                and isinstance(node.elts[0].value, str) and isinstance(node.elts[1], ast.Name):
            called.add(node.elts[1].id)
    assert {"run_cfg3", "run_strip_extra", "run_dense_extra", "run_rank_r_extra"} <= called
    assert called <= defined, called - defined
