"""The library built with every index check compiled in (-DSINN_BOUNDS_CHECK,
the stand-in for a memory checker: an out-of-range index sets a device error
and is not accessed) runs streaming inserts and deletes with searches on the
batched and the dense paths, a learned-k' search and a recorded search, all
checked against the oracle, with no index out of range."""
import os
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SCRIPT = r"""
import sys
import numpy as np
import torch
from paper_2301_10622_gb300 import sinnamon, synth
sinnamon._build.LIB = sys.argv[1]
sinnamon.load()
from tests.test_gpu_parity import _check_search, _ip, _ix, _pair

# streaming: inserts that grow the capacity and the store, deletes, reuse
w = synth.scaled(synth.WORKLOADS["mixed"], 0, n=2000)
pool = synth.make_docs(w, n_docs=6000, seed=5)
qs = synth.make_queries(w, n_q=40, seed=6)
gpu, ora = _pair(w, None, tile_docs=1024)
rng = np.random.default_rng(0)
pos = 0
for step in range(5):
    part = pool.slice(pos, min(pos + int(rng.integers(300, 1500)), pool.rows))
    pos += part.rows
    gpu.insert(_ip(part), _ix(part), part.values)
    ora.insert(part.indptr, part.indices, part.values)
    live = ora.live_ids()
    dele = rng.choice(live, size=min(live.size, int(rng.integers(50, 400))), replace=False)
    gpu.delete(dele.astype(np.int32))
    ora.delete(dele.astype(np.uint32))
    _check_search(gpu, ora, qs, 10, 200)          # 40 queries: batched scorer
    _check_search(gpu, ora, qs.slice(0, 5), 10, 200)  # 5 queries: dense scorer
# text-like lists (bitmap containers), learned k' and a recorded search
w = synth.scaled(synth.WORKLOADS["text"], 9000, n=5000)
docs, qs = synth.make_docs(w), synth.make_queries(w, n_q=48)
gpu, ora = _pair(w, docs, tile_docs=2048)
_check_search(gpu, ora, qs, 10, 300)
mlp = sinnamon.MLP(sinnamon.KP_FEATURES, 64, seed=3)
ids, _, kp = gpu.search_learned(mlp, _ip(qs), _ix(qs), qs.values, 10, 10, 500)
gpu.sync()
mlp.sync()
q = tuple(torch.as_tensor(x).cuda() for x in (_ip(qs), _ix(qs), qs.values))
plan = sinnamon.Plan(gpu, *q, k=10, k_prime_max=300, scratch_bytes=64 << 20)
plan.run()
gpu.sync()
plan.close()
print("bounds ok")
"""


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def test_bounds_checked_build_finds_no_index_out_of_range():
    from paper_2301_10622_gb300 import build
    lib = build.build(bounds_check=True)
    r = subprocess.run([sys.executable, "-c", SCRIPT, lib], cwd=ROOT, capture_output=True,
                       text=True, timeout=900)
    assert r.returncode == 0 and "bounds ok" in r.stdout, r.stdout[-3000:] + r.stderr[-3000:]
