"""The learned per-query k': CUDA network forward/gradient against the FP64
reference, features against their definition, labels against the oracle,
and what the trained network gains over a fixed k'."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle  # noqa: E402
from oracle import mlp as omlp  # noqa: E402
from paper_2301_10622_gb300 import kprime, sinnamon, synth  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()


# bf16 keeps 8 significant bits: each operand the GEMMs read (inputs, weights,
# hidden activations, back-propagated terms) carries a relative rounding
# error of at most 2^-8; accumulation is fp32
U_BF16 = 2.0 ** -8


def _separated_biases(p, X, mean, std, n_in, hid, rng):
    """Biases that keep every pre-activation of the batch clearly away from
    zero: each unit is on for every row or off for every row, by a margin
    wider than the bf16 error bound of its inputs' terms, so no ReLU can
    flip between the GPU's evaluation and the FP64 one and the element-wise
    bound needs no flip allowance.  Weights stay as initialised."""
    W1, b1, W2, b2, w3, b3 = omlp.unpack(p, n_in, hid)
    Xn = (X.astype(np.float64) - mean) / std
    A = Xn @ W1.T
    S1 = np.abs(Xn) @ np.abs(W1).T
    b1 = np.where(rng.random(hid) < 0.5, -1.0, 1.0) * (
        1.25 * (np.abs(A).max(0) + 2 * U_BF16 * S1.max(0)) + 0.25)
    on1 = (A + b1) > 0
    A2 = np.maximum(A + b1, 0) @ W2.T
    S2 = ((S1 + np.abs(b1)) * on1) @ np.abs(W2).T
    b2 = np.where(rng.random(hid) < 0.5, -1.0, 1.0) * (
        1.25 * (np.abs(A2).max(0) + 5 * U_BF16 * S2.max(0)) + 0.25)
    q = np.array(p, np.float64)
    o = hid * n_in
    q[o:o + hid] = b1
    o2 = o + hid + hid * hid
    q[o2:o2 + hid] = b2
    return q.astype(np.float32)


@pytest.mark.parametrize("B,n_in", [(300, sinnamon.KP_FEATURES), (64, sinnamon.KP_FEATURES),
                                    (1, sinnamon.KP_FEATURES), (200, sinnamon.KP_FEATURES + 1)])
def test_network_forward_and_gradient_match_fp64(B, n_in):
    """Element by element: each output and each parameter's gradient is
    within 6 * 2^-8 of the magnitude of its terms (the sum of their absolute
    values, from the FP64 reference over |W|, |X|, |dy|: oracle.mlp
    .error_bounds) of the FP64 value.  Biases keep every pre-activation away
    from zero, so no ReLU flips and the bound needs no flip allowance."""
    hid = 256
    net = sinnamon.MLP(n_in, hid, seed=3)
    rng = np.random.default_rng(B)
    X = rng.normal(2.0, 3.0, (B, n_in)).astype(np.float32)
    mean, std = X.mean(0), X.std(0) + 1e-3
    if B == 1:
        mean, std = np.zeros(n_in, np.float32), np.ones(n_in, np.float32)
    net.set_normalizer(mean, std)
    m64, s64 = mean.astype(np.float64), std.astype(np.float64)
    net.set_params(_separated_biases(net.params(), X, m64, s64, n_in, hid, rng))
    p = net.params()
    y = net.forward(X).cpu().numpy().astype(np.float64)
    y_ref, _ = omlp.forward(p, X, m64, s64, n_in, hid)
    # targets away from the outputs: no pinball residual can change sign
    ya, _, _ = omlp.error_bounds(p, X, y_ref, 0.9, m64, s64, n_in, hid, U_BF16)
    t = (y_ref + np.where(rng.random(B) < 0.5, -1.0, 1.0) *
         (12 * U_BF16 * ya + 0.5 + rng.random(B))).astype(np.float32)
    ya, gm, gf = omlp.error_bounds(p, X, t, 0.9, m64, s64, n_in, hid, U_BF16)
    assert gf.max() == 0.0        # no ReLU or residual near its sign change
    bad = np.abs(y - y_ref) > 6 * U_BF16 * ya
    assert not bad.any(), (np.nonzero(bad)[0][:5], y[bad][:5], y_ref[bad][:5])
    g, loss = net.grad(X, t, 0.9)
    g = g.cpu().numpy().astype(np.float64)
    g_ref, l_ref = omlp.grad(p, X, t, 0.9, m64, s64, n_in, hid)
    assert abs(float(loss.item()) - l_ref) <= 6 * U_BF16 * np.mean(ya) + 1e-6
    err = np.abs(g - g_ref)
    lim = 6 * U_BF16 * gm + gf + 1e-12
    bad = err > lim
    assert not bad.any(), (np.nonzero(bad)[0][:5], err[bad][:5], lim[bad][:5])
    # not vacuous: a sign error would exceed the limit on most elements
    nz = gm > 0
    assert np.mean(2 * np.abs(g_ref[nz]) > lim[nz]) > (0.3 if B == 1 else 0.8)


def test_training_reduces_the_loss():
    net = sinnamon.MLP(sinnamon.KP_FEATURES, 64, seed=1)
    rng = np.random.default_rng(0)
    X = torch.from_numpy(rng.normal(0, 1, (2048, sinnamon.KP_FEATURES)).astype(np.float32)).cuda()
    w = rng.normal(0, 1, sinnamon.KP_FEATURES).astype(np.float32)
    t = (X.cpu().numpy() @ w).astype(np.float32)
    t = torch.from_numpy(t).cuda()
    first = float(net.train_step(X, t, 0.5, 1e-2).item())
    for _ in range(200):
        last = float(net.train_step(X, t, 0.5, 1e-2).item())
    assert last < 0.2 * first


def test_features_match_their_definition():
    w = synth.scaled(synth.WORKLOADS["text"], 5000, n=3000)
    docs, qs = synth.make_docs(w), synth.make_queries(w, n_q=40)
    ix = sinnamon.Index(w.n, w.m, w.h, tile_docs=1024)
    ix.insert(docs.indptr.astype(np.int64), docs.indices.astype(np.int32), docs.values)
    ix.delete(np.arange(0, 5000, 7, dtype=np.int32))  # tombstones still count
    F = ix.kp_features(qs.indptr.astype(np.int64), qs.indices.astype(np.int32),
                       qs.values).cpu().numpy()
    lens = np.bincount(docs.indices[docs.values != 0], minlength=w.n)
    for r in range(qs.rows):
        i, v = qs.row(r)
        keep = v != 0
        i, v = i[keep], v[keep].astype(np.float64)
        assert abs(F[r, 0] - np.log2(1 + i.size)) < 1e-5
        assert abs(F[r, 1] - np.abs(v).sum()) < 1e-4 * (1 + np.abs(v).sum())
        assert abs(F[r, 2] - np.sqrt((v * v).sum())) < 1e-4 * (1 + np.sqrt((v * v).sum()))
        order = np.lexsort((i, -np.abs(v)))[:16]
        want = np.zeros(16)
        want[:order.size] = np.log2(1 + lens[i[order]])
        np.testing.assert_allclose(F[r, 3:], want, rtol=1e-5, atol=1e-5)


def test_labels_match_the_oracle():
    """The 9th smallest approximate rank of the exact top 10, from the GPU's
    own scores, equals the same quantity from the FP64 oracle (up to fp32
    near-ties in the approximate order)."""
    w = synth.scaled(synth.WORKLOADS["text"], 20000, n=5000)
    docs, qs = synth.make_docs(w), synth.make_queries(w, n_q=60)
    ix = sinnamon.Index(w.n, w.m, w.h, tile_docs=2048)
    ix.insert(docs.indptr.astype(np.int64), docs.indices.astype(np.int32), docs.values)
    kp, cert, ex_ids = kprime.labels(ix, qs, cap=20000)
    assert cert.all()  # every live id is a candidate here
    ora = oracle.OracleIndex(w.n, w.m, w.h)
    ora.insert(docs.indptr, docs.indices, docs.values)
    ex = ora.exact_topk(qs.indptr, qs.indices, qs.values, k=10)
    agree = 0
    for r in range(qs.rows):
        qi, qv = qs.row(r)
        approx = ora.scores(qi, qv)
        order = np.lexsort((np.arange(approx.size), -approx))
        rank = np.empty(approx.size, np.int64)
        rank[order] = np.arange(1, approx.size + 1)
        want = np.sort(rank[ex["ids"][r].astype(np.int64)])[8]
        agree += int(kp[r] == want)
        assert abs(kp[r] - want) <= max(3, 0.02 * want), (r, kp[r], want)
        assert len(set(ex_ids[r]) & set(ex["ids"][r].astype(np.int64))) >= 9
    assert agree >= 0.9 * qs.rows


def test_learned_kprime_beats_fixed_kprime():
    """Trained on the method's own labels, the network keeps recall@10 >= 0.9
    with a much smaller mean k' than the fixed fallback of 1000."""
    w = synth.scaled(synth.WORKLOADS["text"], 100_000)
    docs = synth.make_docs(w)
    train_q = synth.make_queries(w, n_q=4000, seed=3000)
    test_q = synth.make_queries(w, n_q=400, seed=3001)
    ix = sinnamon.Index(w.n, w.m, w.h, tile_docs=4096)
    ix.insert(docs.indptr.astype(np.int64), docs.indices.astype(np.int32), docs.values)
    kp_train, cert, _ = kprime.labels(ix, train_q, cap=20000)
    assert cert.mean() > 0.95
    net = kprime.train(ix, train_q, kp_train, epochs=40, batch=1024)
    _, _, ex_test = kprime.labels(ix, test_q, cap=20000)
    res = kprime.evaluate(ix, net, test_q, ex_test, fixed=1000)
    assert res["recall_learned"] >= 0.9, res
    assert res["mean_kprime_learned"] < 0.5 * res["fixed_kprime"], res
    # the learned search equals sinn_search_kp at the k' it chose
    ip, ii = test_q.indptr.astype(np.int64), test_q.indices.astype(np.int32)
    ids_l, sc_l, kps = ix.search_learned(net, ip, ii, test_q.values, 10, 10, 20000)
    ids_k, sc_k = ix.search(ip, ii, test_q.values, k=10, k_prime=kps.cpu().numpy(),
                            k_prime_max=20000)
    assert np.array_equal(ids_l.cpu().numpy(), ids_k.cpu().numpy())
