"""Host logic of bench.py (no GPU): the algorithmic byte count behind the
roofline (postings scored under the anytime break), the oracle's
reconstruction of the streamed collection, the comment-insensitive source
hash that ties a profile to the kernel it measured, the figures and traffic
scaling read from that profile, and the clock sampler's parsing."""
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import bench  # noqa: E402
from paper_2301_10622_gb300 import synth  # noqa: E402


def _csr(rows):
    ip = np.concatenate([[0], np.cumsum([len(r) for r in rows])]).astype(np.uint64)
    idx = np.array([c for r in rows for c, _ in r], np.uint32)
    val = np.array([v for r in rows for _, v in r], np.float32)
    return synth.CSR(ip, idx, val)


def test_algorithmic_bytes_by_hand():
    w = synth.scaled(synth.WORKLOADS["tiny"], 3, n=5, m=4, h=2)
    # |I[0]| = 2, |I[1]| = 1 (an explicit zero is not a posting), |I[3]| = 3
    docs = _csr([[(0, 1.0), (3, 2.0)], [(0, -1.0), (1, 0.0), (3, 1.0)], [(1, 5.0), (3, 4.0)]])
    qs = _csr([[(0, 1.0), (3, -2.0)], [(1, 0.0), (2, 1.0)], []])
    lens = bench.list_lengths(w, docs)
    assert list(lens) == [2, 1, 0, 3, 0]
    P = bench.scored_postings(qs, lens)
    assert list(P) == [5, 0, 0]  # the zero-valued query term reads no list
    # 4-byte id + h = 2 four-byte bins per posting
    assert list(bench.algorithmic_bytes(w, P)) == [5 * 12, 0, 0]


def test_scored_postings_follow_the_anytime_break():
    """Terms in Alg. 6 order (|q_j| descending, ties j ascending); scoring
    stops after the first term at which the postings reach the budget."""
    lens = np.array([10, 20, 30, 40, 50], np.int64)
    # |q|: coord 4 (3.0) > coord 1 (2.0) = coord 3 (-2.0) > coord 0 (0.5)
    qs = _csr([[(0, 0.5), (1, 2.0), (3, -2.0), (4, 3.0)]] * 5)
    got = bench.scored_postings(qs, lens, np.array([0, 1, 50, 51, 10 ** 6]))
    # order 4 (50), 1 (20), 3 (40), 0 (10): running 50, 70, 110, 120
    assert list(got) == [120, 50, 50, 70, 120]


def test_reconstruct_matches_the_id_reuse_rule():
    """Each step deletes ids and re-inserts as many vectors, which take the
    freed ids in ascending order; the reconstruction equals doing that by
    hand."""
    w = synth.scaled(synth.WORKLOADS["tiny"], 40, n=50)
    docs = synth.make_docs(w)
    rng = np.random.default_rng(0)
    dels, parts, rows = [], [], [list(zip(*docs.row(i))) for i in range(docs.rows)]
    for s in range(3):
        d = rng.choice(40, size=7, replace=False)
        ins = synth.make_docs(w, n_docs=7, seed=100 + s)
        dels.append(torch.from_numpy(d.astype(np.int32)))
        parts.append((None, None, None, ins))
        for slot, i in enumerate(np.sort(d)):
            rows[i] = list(zip(*ins.row(slot)))
    got = bench.reconstruct(docs, parts, dels, [0, 1, 2])
    want = _csr(rows)
    assert np.array_equal(got.indptr.astype(np.int64), want.indptr.astype(np.int64))
    assert np.array_equal(got.indices, want.indices)
    assert np.array_equal(got.values, want.values)
    # only the executed steps count
    first = bench.reconstruct(docs, parts, dels, [0])
    assert not np.array_equal(first.indptr.astype(np.int64), got.indptr.astype(np.int64)) or \
        not np.array_equal(first.values, got.values)


def test_source_hash_ignores_comments_only(tmp_path):
    a = tmp_path / "a.cu"
    a.write_text("int f(int x) {\n  return x + 1;  // one more\n}\n/* block\n comment */\n")
    h = bench.source_code_hash(str(a))
    a.write_text("// header\nint f(int x) {\n\n  return x + 1;   \n}\n")
    assert bench.source_code_hash(str(a)) == h
    a.write_text("int f(int x) {\n  return x + 2;\n}\n")
    assert bench.source_code_hash(str(a)) != h


def test_profile_figures_scale_and_check_their_source(tmp_path, monkeypatch):
    src = tmp_path / "paper_2301_10622_gb300" / "csrc"
    src.mkdir(parents=True)
    (src / "search.cu").write_text("__global__ void k() {}\n")
    (tmp_path / "profiles").mkdir()
    h = bench.source_code_hash(str(src / "search.cu"))
    prof = tmp_path / "profiles" / "k_score_emit_text.md"
    prof.write_text(f"# title: words\nsource_code_sha256_16: {h}\n"
                    "traffic_bytes_per_launch: 1000000\nqueries_per_launch: 100\n"
                    "docs_in_index: 5000\nl2_throughput_frac: 0.5\n"
                    "sectors_per_request: 8.5\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    fig = bench.profile_figures("k_score_emit_text")
    assert fig["traffic_bytes_per_launch"] == 1e6 and fig["docs_in_index"] == 5000
    # 95 queries per launch: 0.95 of the bytes; 1 ms per launch at 1000 GB/s peak
    d = bench.dram_figures(fig, 1.0, 1000.0, 95, 5000)
    assert d["traffic"] == pytest.approx(950000.0)
    assert d["dram_frac"] == pytest.approx(950000.0 / 1e-3 / 1e9 / 1000.0)
    assert d["l2_frac"] == 0.5 and d["l1_frac"] is None and d["sectors_per_request"] == 8.5
    # launches half the profiled size: no scaled traffic, the fractions stay
    d = bench.dram_figures(fig, 1.0, 1000.0, 50, 5000)
    assert d["traffic"] is None and d["dram_frac"] is None and d["l2_frac"] == 0.5
    assert bench.dram_figures(fig, 1.0, 1000.0, 50, 6000)["traffic"] is None  # another size
    (src / "search.cu").write_text("__global__ void k() { int x; }\n")
    assert bench.profile_figures("k_score_emit_text") is None                  # kernel changed
    os.remove(prof)
    assert bench.profile_figures("k_score_emit_text") is None


def test_clock_summary_reads_throttle_reasons():
    c = bench.ClockSampler(0)
    c.lines = ["0, 2070, 2070, 900.1, 0x0, Not Active, Not Active, Not Active, Not Active",
               "0, 1980, 2070, 1399.0, 0x4, Not Active, Not Active, Not Active, Active",
               "0, 2070, 2070, 950.0, 0x0, Not Active, Not Active, Not Active, Not Active",
               "garbage line"]
    s = c.summary()
    assert s["sm_mhz"] == 2070.0 and s["sm_max_mhz"] == 2070.0 and s["samples"] == 3
    assert s["reasons"] == ["sw_power_cap"]
    c.lines = ["0, 1400, 2070, 500, 0x0, Active, Not Active, Active, Not Active"]
    assert c.summary()["reasons"] == ["hw_slowdown", "sw_thermal_slowdown"]
    c.lines = []
    assert c.summary()["reasons"] == ["unsampled"]


def test_recall_counts_ties_from_the_exact_list():
    """recall@10: an id of the exact top 10 is a hit; a missed id is a hit
    exactly when its exact score ties the 10th (taken from the exact list,
    or from the dense exact scores when the whole list ties the 10th)."""
    class FakeOracle:
        def __init__(self, ids, scores, dense):
            self.ids, self.scores, self.dense, self.dense_calls = ids, scores, dense, 0

        def linscan_topk(self, ip, ix, v, k, threads):
            return {"ids": self.ids[:, :k], "scores": self.scores[:, :k]}

        def exact_scores(self, qi, qv):
            self.dense_calls += 1
            return self.dense

    D = bench.TRUTH_DEPTH
    ids = np.arange(D, dtype=np.int64)[None, :]
    sc = np.linspace(10.0, 1.0, D)[None, :]
    sc[0, 10] = sc[0, 9]                    # id 10 ties the 10th
    qs = _csr([[(0, 1.0)]])
    ora = FakeOracle(ids, sc, None)
    got = np.array([[0, 1, 2, 3, 4, 5, 6, 7, 10, 11]])   # 8 of the top 10, the tie, a miss
    assert bench.recall_at_10(ora, qs, got, 1) == 0.9
    assert bench.recall_at_10(ora, qs, np.array([[0, 1, 2, 3, 4, 5, 6, 7, 8, 500]]), 1) == 0.9
    assert ora.dense_calls == 0             # the list ends below the tie: 500 is a miss
    flat = np.full((1, D), 3.0)
    dense = np.zeros(1000)
    dense[500] = 3.0
    ora2 = FakeOracle(ids, flat, dense)     # every listed score ties the 10th
    assert bench.recall_at_10(ora2, qs, np.array([[0, 1, 2, 3, 4, 5, 6, 7, 8, 500]]), 1) == 1.0
    assert ora2.dense_calls == 1


def _profile_commands():
    """Shell commands of the committed ncu summaries, continuation lines
    joined: (file, command) pairs."""
    import glob
    out = []
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    for path in sorted(glob.glob(os.path.join(root, "profiles", "*.md"))):
        text = open(path).read().replace("\\\n", " ")
        for ln in text.splitlines():
            if ln.startswith("    "):                      # indented code lines
                out.append((os.path.basename(path), ln.strip()))
    return out


def test_profile_commands_parse_with_the_bench_flags():
    """Every bench.py command a profile gives is one bench.py accepts."""
    import re
    import shlex
    seen = 0
    for name, cmd in _profile_commands():
        m = re.search(r'bench\.py([^"#>]*)', cmd)
        if not m:
            continue
        seen += 1
        try:
            bench.arg_parser().parse_args(shlex.split(m.group(1)))
        except SystemExit:
            pytest.fail(f"{name}: bench.py rejects {m.group(1).strip()!r}")
    assert seen >= 6


def test_profile_ncu_commands_leave_the_clocks_alone():
    """Every ncu command in the summaries passes --clock-control none."""
    cmds = [(n, c) for n, c in _profile_commands() if c.startswith("ncu ")]
    assert len(cmds) >= 6
    for name, cmd in cmds:
        assert "--clock-control none" in cmd, (name, cmd)
