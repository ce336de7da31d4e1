"""The serving loop (katz_server_*): update batches for several graphs,
submitted in arrival order and run concurrently, give each request the same
answer as applying that graph's batches one by one alone, and the last state
of every graph matches the oracle session fed the same batches."""
from __future__ import annotations

import numpy as np
import pytest

import graphgen as gg
import oracle
from tests.parity import assert_same_ranking

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
K = pytest.importorskip("paper_1807_03847_gb300")

EPS = 1e-9


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _handle(g, k, D):
    h = K.Katz(_dev(g.rowptr), _dev(g.col), K.katz_default_opts(keep_history=1, deg_bound=D, r_max=128))
    h.rank(0.0, k, EPS)
    return h


def _workloads():
    out = []
    for i, (scale, k, max_size) in enumerate([(12, 50, 400), (13, 32, 2000), (11, 100, 60)]):
        g = gg.rmat(scale, 16, seed=300 + i)
        D = g.deg_max() + 64
        st = gg.stream(g, 12, seed=500 + i, max_size=max_size, rate=2000.0, deg_bound=D)
        out.append((g, k, D, st))
    return out


def _alone(g, k, D, st):
    """Each batch applied in order with katz_apply_update_batch, no server."""
    h = _handle(g, k, D)
    res = []
    for j in range(len(st)):
        info = h.update(*st.batch(j))
        res.append((info.r, h.ranking(k).copy()))
    h.close()
    return res


def test_same_result_alone_and_in_the_mix():
    wl = _workloads()
    alone = [_alone(*w) for w in wl]
    handles = [_handle(g, k, D) for g, k, D, _ in wl]
    srv = K.Server(workers=3, slots=4, slot_updates=2000)
    for h, (g, k, D, st) in zip(handles, wl):
        srv.attach(h, k)
    # all requests in one arrival order (merged Poisson streams), submitted at once
    order = sorted(((st.arrival[j], w, j) for w, (_, _, _, st) in enumerate(wl) for j in range(len(st))))
    tickets = {}
    for _, w, j in order:
        tickets[(w, j)] = srv.submit(handles[w], *wl[w][3].batch(j))
    for (w, j), t in tickets.items():
        status, ids, res = srv.wait(t)
        assert status == 0, (w, j, status)
        r_alone, ids_alone = alone[w][j]
        assert res.info.r == r_alone, (w, j)
        np.testing.assert_array_equal(ids, ids_alone, err_msg=f"graph {w} batch {j}")
    srv.close()
    # the final state of each graph against the oracle fed the same batches
    for h, (g, k, D, st) in zip(handles, wl):
        s = oracle.Session(g.rowptr, g.col, True, D)
        assert s.rank_static(0.0, k, EPS, 128) == oracle.OK
        for j in range(len(st)):
            assert s.apply_update(*st.batch(j)) == oracle.OK
        c, l, u = s.bounds()
        assert_same_ranking(h.ranking(k), s.ranking(), l)
        h.close()


def test_rejected_batch_leaves_the_graph_and_later_requests_intact():
    g = gg.rmat(11, 16, seed=31)
    D, k = g.deg_max() + 64, 20
    st = gg.stream(g, 4, seed=32, max_size=50, deg_bound=D)
    h = _handle(g, k, D)
    ref = _alone(g, k, D, st)
    srv = K.Server(workers=2, slots=2, slot_updates=100)
    srv.attach(h, k)
    # a delete of a pair that is not an edge (0 has no self-loop) is invalid
    t0 = srv.submit(h, *st.batch(0))
    bad = srv.submit(h, np.array([0], np.int32), np.array([0], np.int32), np.array([0], np.uint8))
    rest = [srv.submit(h, *st.batch(j)) for j in range(1, len(st))]
    s0, ids0, _ = srv.wait(t0)
    sb, idsb, _ = srv.wait(bad)
    assert s0 == 0 and sb == 1  # KATZ_EINVAL
    np.testing.assert_array_equal(idsb, ids0)  # unchanged ranking
    for j, t in enumerate(rest, start=1):
        status, ids, _ = srv.wait(t)
        assert status == 0
        np.testing.assert_array_equal(ids, ref[j][1])
    with pytest.raises(K.KatzError):  # larger than a slot
        srv.submit(h, np.zeros(101, np.int32), np.ones(101, np.int32), np.ones(101, np.uint8))
    srv.close()
    h.close()


def test_wait_times_out_and_one_slot_serialises_admission():
    g = gg.rmat(12, 16, seed=41)
    D, k = g.deg_max() + 64, 10
    st = gg.stream(g, 6, seed=42, max_size=500, deg_bound=D)
    ref = _alone(g, k, D, st)
    h = _handle(g, k, D)
    srv = K.Server(workers=4, slots=1, slot_updates=500)
    srv.attach(h, k)
    ts = [srv.submit(h, *st.batch(j)) for j in range(len(st))]
    with pytest.raises(K.KatzError) as e:
        srv.wait(ts[-1], timeout_ms=0)
    assert e.value.name == "KATZ_ETIMEOUT"
    for j, t in enumerate(ts):
        status, ids, res = srv.wait(t)
        assert status == 0
        np.testing.assert_array_equal(ids, ref[j][1])
        assert res.latency_ms >= res.service_ms
    srv.close()
    h.close()


def test_a_byte_budget_admits_one_batch_at_a_time():
    """admit_bytes below the staging memory of two batches: each request is
    admitted only after the one before it has finished, and the answers are
    those of applying the batches one by one."""
    g = gg.rmat(12, 16, seed=43)
    D, k = g.deg_max() + 64, 10
    st = gg.stream(g, 5, seed=44, min_size=300, max_size=300, deg_bound=D)
    ref = _alone(g, k, D, st)
    h = _handle(g, k, D)
    srv = K.Server(workers=4, slots=8, slot_updates=300, admit_bytes=18 * 400)
    srv.attach(h, k)
    ts = [srv.submit(h, *st.batch(j)) for j in range(len(st))]
    res = [srv.wait(t) for t in ts]
    for j, (status, ids, r) in enumerate(res):
        assert status == 0
        np.testing.assert_array_equal(ids, ref[j][1])
        if j > 0:  # admitted (queue_ms after submit) no earlier than the previous request finished
            assert r.queue_ms >= res[j - 1][2].latency_ms - 1.0
    srv.close()
    h.close()


@pytest.mark.parametrize("directed,fp32", [(False, False), (True, False), (False, True), (True, True)])
def test_pipelined_batches_on_one_handle_match_sequential(directed, fp32):
    # two workers on one handle: the prepare of each batch (validation and
    # the rebuilt graph, on the handle's second stream) overlaps the repair
    # of the batch before it; every answer must equal the batch-by-batch one
    g = gg.rmat(13, 16, seed=61)
    if directed:
        g = gg.orient(g, seed=62)
    D, k = g.deg_max() + 64, 40
    batches, cur = [], g
    for j in range(20):
        m = [3, 800, 40, 2000, 1][j % 5]
        if directed:
            b = gg.directed_update_batch(cur, m, seed=700 + j, deg_bound=D)
            cur = gg.apply_directed_batch(cur, *b)
        else:
            b = gg.update_batch(cur, m, seed=700 + j)
            cur = gg.apply_batch(cur, *b)
        batches.append(b)
    opts = dict(keep_history=1, deg_bound=D, r_max=128, undirected=0 if directed else 1)
    eps = EPS
    if fp32:  # FP32-certified levels from level 3 on
        opts.update(precision=K.KATZ_FP32_CERT, fp32_from=3)
        eps = 1e-4
    seq = K.Katz(_dev(g.rowptr), _dev(g.col), K.katz_default_opts(**opts))
    seq.rank(0.0, k, eps)
    ref = []
    for b in batches:
        info = seq.update(*b)
        ref.append((info.r, seq.ranking(k).copy(), seq.bounds()[0].copy()))
    h = K.Katz(_dev(g.rowptr), _dev(g.col), K.katz_default_opts(**opts))
    h.rank(0.0, k, eps)
    srv = K.Server(workers=2, slots=4, slot_updates=2000)
    srv.attach(h, k)
    tickets = [srv.submit(h, *b) for b in batches]
    for j, t in enumerate(tickets):
        status, ids, res = srv.wait(t, timeout_ms=120000)
        assert status == 0, (j, status)
        assert res.info.r == ref[j][0], j
        np.testing.assert_array_equal(ids, ref[j][1], err_msg=f"batch {j}")
    srv.close()
    np.testing.assert_array_equal(h.bounds()[0], ref[-1][2])
    s = oracle.Session(g.rowptr, g.col, not directed, D)
    assert s.rank_static(0.0, k, eps, 128) == oracle.OK
    for b in batches:
        assert s.apply_update(*b) == oracle.OK
    c, l, u = s.bounds()
    assert_same_ranking(h.ranking(k), s.ranking(), l, atol=eps if fp32 else 0.0)
    seq.close()
    h.close()


@pytest.mark.parametrize("fp32", [False, True])
@pytest.mark.parametrize("graph", ["rmat", "hubs"])
def test_two_state_pass_gives_the_bits_of_batch_by_batch_repairs(fp32, graph):
    """pair_batches = 2: queued batches of one graph go through the two-state
    pass (both graph states' levels in one pass, the rows the second batch
    changed recomputed from the first state's graph).  Each answer equals the
    batch-by-batch one, and the final walk levels and bounds are the same
    bits.  The 'hubs' graph has rows of several 2048-arc chunks whose chunk
    count the batches change."""
    if graph == "rmat":
        g = gg.rmat(13, 16, seed=81)
    else:  # stars of 3000 to 7000 leaves joined by a sparse random graph
        rng = np.random.default_rng(82)
        n = 40000
        u, v = [], []
        for c, leaves in enumerate((7000, 5000, 4100, 3000)):
            ls = rng.choice(np.arange(10, n), leaves, replace=False)
            u.append(np.full(leaves, c))
            v.append(ls)
        u.append(rng.integers(0, n, 60000))
        v.append(rng.integers(0, n, 60000))
        g = gg.from_edges(n, np.concatenate(u), np.concatenate(v))
    D, k = g.deg_max() + 2500, 40
    batches, cur = [], g
    for j in range(12):
        m = [3, 800, 40, 2000][j % 4]
        if graph == "hubs" and j % 3 == 0:  # grow and shrink the hubs across chunk boundaries
            hub = j % 4
            nb = set(cur.col[cur.rowptr[hub]:cur.rowptr[hub + 1]].tolist())
            cand = [x for x in range(10, g.n) if x not in nb and x != hub][: m]
            b = (np.full(len(cand), hub, np.int32), np.array(cand, np.int32), np.ones(len(cand), np.uint8))
        else:
            b = gg.update_batch(cur, m, seed=900 + j)
        cur = gg.apply_batch(cur, *b)
        batches.append(b)
    opts = dict(keep_history=1, deg_bound=D, r_max=128)
    eps = EPS
    if fp32:
        opts.update(precision=K.KATZ_FP32_CERT, fp32_from=3)
        eps = 1e-4
    seq = K.Katz(_dev(g.rowptr), _dev(g.col), K.katz_default_opts(**opts))
    seq.rank(0.0, k, eps)
    ref = []
    for b in batches:
        info = seq.update(*b)
        ref.append((info.r, seq.ranking(k).copy()))
    h = K.Katz(_dev(g.rowptr), _dev(g.col), K.katz_default_opts(**opts))
    h.rank(0.0, k, eps)
    srv = K.Server(workers=2, slots=8, slot_updates=4000, pair_batches=2)
    srv.attach(h, k)
    tickets = [srv.submit(h, *b) for b in batches]
    paired = 0
    for j, t in enumerate(tickets):
        status, ids, res = srv.wait(t, timeout_ms=120000)
        assert status == 0, (j, status)
        assert res.info.r == ref[j][0], j
        np.testing.assert_array_equal(ids, ref[j][1], err_msg=f"batch {j}")
        paired += res.paired
    srv.close()
    assert paired >= 4  # the pass really ran
    for a, b in zip(h.bounds(), seq.bounds()):
        np.testing.assert_array_equal(a, b)
    for i in range(1, ref[-1][0] + 1):
        np.testing.assert_array_equal(h.walk(i), seq.walk(i), err_msg=f"s_{i}")
    seq.close()
    h.close()


@pytest.mark.parametrize("fp32", [False, True])
def test_submit_and_poll_match_applying_the_batches_in_order(fp32):
    # katz_submit_update_batch / katz_poll: the asynchronous form of
    # katz_apply_update_batch on one handle (its private serving queue)
    import time

    g = gg.rmat(13, 16, seed=63)
    D, k = g.deg_max() + 64, 40
    opts = dict(keep_history=1, deg_bound=D, r_max=128)
    eps = EPS
    if fp32:
        opts.update(precision=K.KATZ_FP32_CERT, fp32_from=3)
        eps = 1e-4
    batches, cur = [], g
    for j in range(8):
        b = gg.update_batch(cur, [5, 900, 30, 3000][j % 4], seed=800 + j)
        cur = gg.apply_batch(cur, *b)
        batches.append(b)
    seq = K.Katz(_dev(g.rowptr), _dev(g.col), K.katz_default_opts(**opts))
    seq.rank(0.0, k, eps)
    ref = [seq.update(*b) for b in batches]
    h = K.Katz(_dev(g.rowptr), _dev(g.col), K.katz_default_opts(**opts))
    h.rank(0.0, k, eps)
    tickets = [h.submit(*b) for b in batches]

    def result(t):
        deadline = time.time() + 120
        while True:
            info = h.poll(t)
            if info is not None:
                return info
            assert time.time() < deadline, "batch did not finish"
            time.sleep(0.001)

    infos = [result(t) for t in tickets]
    for j, (a, b) in enumerate(zip(infos, ref)):
        assert a.status == 0 and a.r == b.r and a.nnz == b.nnz and a.converged == 1, j
    np.testing.assert_array_equal(h.ranking(k), seq.ranking(k))
    for x, y in zip(h.bounds(), seq.bounds()):
        np.testing.assert_array_equal(x, y)
    with pytest.raises(K.KatzError) as e:  # each ticket is reported once
        h.poll(tickets[0])
    assert e.value.name == "KATZ_ESTATE"
    # a rejected batch (an edge that is already there) changes nothing
    u = 0 if cur.rowptr[1] > cur.rowptr[0] else int(np.argmax(np.diff(cur.rowptr) > 0))
    v = int(cur.col[cur.rowptr[u]])
    before = h.ranking(k).copy()
    t = h.submit(np.array([u], np.int32), np.array([v], np.int32), np.array([1], np.uint8))
    info = result(t)
    assert info.status == 1  # KATZ_EINVAL
    np.testing.assert_array_equal(h.ranking(k), before)
    # batches still queued when the handle is destroyed are dropped
    for j in range(3):
        h.submit(*gg.update_batch(cur, 50, seed=900 + j))
    h.close()
    seq.close()


def test_submit_needs_a_ranked_handle_with_history():
    g = gg.rmat(10, 8, seed=64)
    h = K.Katz(_dev(g.rowptr), _dev(g.col), K.katz_default_opts(keep_history=1))
    src, dst, ins = gg.update_batch(g, 10, seed=1)
    with pytest.raises(K.KatzError) as e:
        h.submit(src, dst, ins)
    assert e.value.name == "KATZ_ESTATE"
    with pytest.raises(K.KatzError) as e:  # nothing submitted yet
        h.poll(1)
    assert e.value.name == "KATZ_ESTATE"
    h.close()
