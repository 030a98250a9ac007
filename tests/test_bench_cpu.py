"""Host-side helpers of bench.py: recall, tie-tolerant recall, the host exact
k-NN and the threaded oracle runner (no GPU)."""
import os
import sys

import numpy as np

from paper_1603_09320_gb300 import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def set_recall(ids, gt):
    return sum(len(set(ids[i].tolist()) & set(gt[i].tolist())) for i in range(len(gt))) / gt.size


def test_recall_matches_the_set_definition():
    rng = np.random.default_rng(3)
    gt = np.array([rng.choice(1000, 10, replace=False) for _ in range(200)])
    ids = np.array([rng.choice(1000, 10, replace=False) for _ in range(200)])
    ids[:50] = gt[:50][:, ::-1]  # some exact rows, in another order
    assert bench.recall_at(ids, gt) == set_recall(ids, gt)
    assert bench.recall_at(gt, gt) == 1.0


def test_tie_tolerant_recall_counts_ties_at_the_kth_distance():
    rng = np.random.default_rng(0)
    X = rng.integers(0, 4, (500, 4)).astype(np.float32)  # many equal distances
    Q = rng.integers(0, 4, (50, 4)).astype(np.float32)
    gt = bench.exact_knn_numpy(X, Q, 5)
    alt = np.array([np.lexsort((-np.arange(500), ((X - Q[i]) ** 2).sum(1)))[:5] for i in range(50)])
    assert bench.recall_at(alt, gt) < 1.0  # ties broken the other way
    assert bench.recall_tie_tolerant(X, Q, alt, gt) == 1.0
    far = np.tile(np.argsort(-((X - Q[0]) ** 2).sum(1))[:5], (50, 1))
    assert bench.recall_tie_tolerant(X, Q, far, gt) <= bench.recall_at(far, gt) + 0.2


def test_host_exact_knn_equals_the_oracle_brute_force():
    from oracle import oracle as O
    X = synth.base("tiny", 3000)
    Q = synth.queries("tiny", 40)
    ids, _ = O.brute_force(X, Q, 10)
    np.testing.assert_array_equal(bench.exact_knn_numpy(X, Q, 10), ids.astype(np.int64))


def test_threaded_oracle_runner_matches_one_thread():
    from oracle import oracle as O
    p = synth.params("tiny")
    X = synth.base("tiny", 2000)
    g = O.Graph.build(X, synth.level_uniforms("tiny", 2000), **p)
    Q = synth.queries("tiny", 64)
    one, _, _ = bench.oracle_run(g, Q, 10, 32, 1, 1e9)
    many, bounds, _ = bench.oracle_run(g, Q, 10, 32, 4, 1e9)
    a = np.array([i for part in one for i in part[0]])
    b = np.array([i for part in many for i in part[0]])
    np.testing.assert_array_equal(a, b)
    assert list(bounds) == [0, 16, 32, 48, 64]
    assert isinstance(bench.cpu_model(), str) and bench.cpu_model()


def test_fp64_exact_knn_equals_the_oracle_on_tight_clusters():
    # the low-d ground truth (fp64 expansion + fp64 rescoring), run with torch on the CPU
    from oracle import oracle as O
    X = synth.base("lowd", 5000)
    Q = synth.queries("lowd", 64)
    ids, _ = O.brute_force(X, Q, 10)
    np.testing.assert_array_equal(bench.exact_knn_fp64(X, Q, 10, "cpu"), ids.astype(np.int64))


def test_algorithmic_bytes_by_hand():
    class Info:
        row_bytes, storage, Mmax0, Mmax = 256, 1, 32, 16  # bf16 rows of 128 coordinates
    stats = np.array([[1000, 60, 20], [500, 30, 10]], dtype=np.uint32)
    # per query: rows + layer-0 lists (32 ids) + upper lists (16 ids + offset) + query + results
    q0 = 1000 * 256 + 60 * 128 + 20 * 68 + 128 * 4 + 10 * 8
    q1 = 500 * 256 + 30 * 128 + 10 * 68 + 128 * 4 + 10 * 8
    total, m = bench.algorithmic_bytes(Info, stats, 10, 50, False, 128)
    assert total == q0 + q1 and m["bytes_per_query"] == (q0 + q1) / 2
    total, _ = bench.algorithmic_bytes(Info, stats, 10, 50, True, 128)  # + 50 fp32 rerank rows
    assert total == q0 + q1 + 2 * 50 * 512

    class Fp8:
        row_bytes, storage, Mmax0, Mmax = 128, 2, 32, 16  # + the 4-byte row scale
    total, _ = bench.algorithmic_bytes(Fp8, stats[:1], 10, 5, True, 128)  # ef' = max(ef, k) = 10
    assert total == 1000 * 132 + 60 * 128 + 20 * 68 + 512 + 80 + 10 * 512


def test_clock_samples_are_summarised(tmp_path):
    c = bench.Clocks(0, enabled=False)
    assert c.stop() is None

    class Done:
        def terminate(self):
            pass

        def wait(self):
            pass
    c.p, c.path = Done(), str(tmp_path / "clocks.csv")
    rows = ["0, 1965, 2070, 900.1, 0x0, Not Active, Not Active, Not Active, Not Active",
            "0, 1980, 2070, 1100.0, 0x4, Not Active, Not Active, Not Active, Active",
            "0, 2010, 2070, 1180.5, 0x4, Not Active, Not Active, Not Active, Active",
            "0, [N/A], 2070, 0, 0x0, Not Active, Not Active, Not Active, Not Active",
            "garbage"]
    open(c.path, "w").write("\n".join(rows) + "\n")
    s = c.stop()
    assert s == {"sm_mhz": 1980.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"], "samples": 3}


def test_traffic_counters_only_for_the_same_kernel_source():
    traffic, sha = bench.load_traffic("no-such-kernel", 50)
    assert traffic is None and len(sha) == 16
    # the committed counters belong to this kernel's code, at the bench's ef
    traffic, sha = bench.load_traffic("hnsw_search_kernel:bf16r", 50)
    assert traffic is not None and traffic > 1e9
    assert bench.load_traffic("hnsw_search_kernel:bf16r", 64)[0] is None


def test_kernel_hash_ignores_comments(tmp_path, monkeypatch):
    # a comment edit keeps the hash; a code edit changes it
    src = open(os.path.join(ROOT, "paper_1603_09320_gb300", "csrc", "search.cu")).read()
    d = tmp_path / "paper_1603_09320_gb300" / "csrc"
    d.mkdir(parents=True)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    (d / "search.cu").write_text(src)
    h0 = bench.kernel_source_sha()
    (d / "search.cu").write_text(src.replace("// search.cu --", "// search.cu (edited comment) --", 1) + "\n// x\n")
    assert bench.kernel_source_sha() == h0
    (d / "search.cu").write_text(src.replace("constexpr int kMaxDeg = 64;", "constexpr int kMaxDeg = 32;", 1))
    assert bench.kernel_source_sha() != h0


def test_reference_arm_prints_the_contract_line():
    # the reference arm runs the oracle on the host cores only: run it end to
    # end on a small base and check its JSON line
    import json
    import subprocess
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--n-base", "5000",
                        "--n-queries", "1000", "--batches", "5", "--steps", "2", "--warmup", "1"],
                       capture_output=True, text=True, timeout=900, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-3000:]
    line = json.loads(r.stdout.strip().splitlines()[-1])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in line, key
    assert line["impl"] == "reference" and line["value"] > 0 and line["unit"] == "queries/s"
    assert (line["n_gpus"], line["steps"], line["warmup"], line["higher_is_better"]) == (1, 2, 1, True)
    assert line["vs_baseline"] is None and "workload" in line["config"]
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == line["value"] and cb["cores"] >= 1 and cb["sample"]
    assert line["e2e"] == {"value": line["value"], "unit": "queries/s", "h2d_bytes_per_step": 0,
                           "d2h_bytes_per_step": 0}


def test_reference_arm_other_ranks_exit_without_work():
    import subprocess
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--n-base", "5000",
                        "--steps", "2", "--warmup", "1"], capture_output=True, text=True, timeout=300, cwd=ROOT,
                       env=env)
    assert r.returncode == 0 and r.stdout.strip() == "", r.stderr[-2000:]
