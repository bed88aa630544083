"""Serving: the transaction pool, bulk generator and continuous batching.

The server assigns every submitted transaction the next id (its timestamp),
closes bulks under a deadline, keeps several bulks on the device at once and
applies them in id order, so the whole served stream must equal serial
execution in id order, bit for bit (integer columns, tolerance 0).
"""
import time

import numpy as np
import pytest

import oracle
import paper_1103_3105_gb300 as G
import workloads as W
from tests._helpers import check_indexes, gpu_logical_state, oracle_logical_state, state_diff, states_equal

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()


def dc_db(B=10, T=100, A=10_000, cap=1 << 20, max_bulk=1 << 14):
    g = G.Database(dc=(B, T, A), history_capacity=cap, max_bulk=max_bulk)
    g.register(G.DC_TYPES)
    return g


def trickle(srv, bulk, rng, max_chunk=3000, pause_s=0.0002):
    """Submit a bulk's transactions in random-size chunks, as clients would."""
    n = len(bulk["ts"])
    i, first = 0, None
    while i < n:
        k = int(rng.integers(1, max_chunk + 1))
        f = srv.submit(bulk["type"][i:i + k], bulk["params"][i:i + k])
        first = f if first is None else first
        i += k
        if pause_s:
            time.sleep(pause_s)
    return first


@pytest.mark.parametrize("strategy,mode,inflight", [("kset", 0, 3), ("kset", 1, 1), ("tpl", 1, 2),
                                                    ("part", 0, 2), ("auto", 0, 3), ("scan", 0, 3)])
def test_served_stream_equals_serial_execution(strategy, mode, inflight):
    A = 10_000
    g = dc_db(A=A)
    o = oracle.OracleDB(dc=W.dc_tables(10, 100, A), hist_cap=1 << 20)
    srv = G.Server(g, deadline_us=300, max_bulk=4096, max_inflight=inflight, strategy=strategy,
                   conflict_mode=mode)
    bulk = W.dc_bulk(60_000, A, 0.8, seed=31)
    first = trickle(srv, bulk, np.random.default_rng(1))
    srv.drain()
    assert first == 0
    st, vals, done_ns, nd = srv.results(0, 60_000)
    stats = srv.stats()
    srv.close()
    assert nd == 60_000 and stats["completed"] == 60_000
    assert stats["bulks"] > 1 and 0 < stats["p50_us"] <= stats["p99_us"]
    ost, oout = o.execute(bulk, R=1)
    assert np.array_equal(st, ost) and np.array_equal(vals, oout)
    gs, os_ = gpu_logical_state(g, dc=True), oracle_logical_state(o)
    assert states_equal(gs, os_), state_diff(gs, os_)
    g.close()


@pytest.mark.parametrize("theta,mode", [(0.0, 0), (0.99, 0), (0.99, 1)])
def test_zero_set_serving_equals_serial_execution(theta, mode):
    """Incremental 0-set serving (Section 5.3): arrivals join the device pool
    and each step runs its 0-set; results complete out of id order, yet the
    stream equals serial execution in id order."""
    A = 10_000
    g = dc_db(A=A)
    o = oracle.OracleDB(dc=W.dc_tables(10, 100, A), hist_cap=1 << 20)
    srv = G.Server(g, deadline_us=300, max_bulk=4096, zero_set=True, conflict_mode=mode)
    bulk = W.dc_bulk(30_000, A, theta, seed=33 + mode)
    trickle(srv, bulk, np.random.default_rng(2))
    srv.drain()
    st, vals, done_ns, nd = srv.results(0, 30_000)
    stats = srv.stats()
    srv.close()
    assert nd == 30_000 and stats["completed"] == 30_000 and stats["bulks"] > 1
    ost, oout = o.execute(bulk, R=1)
    assert np.array_equal(st, ost) and np.array_equal(vals, oout)
    gs, os_ = gpu_logical_state(g, dc=True), oracle_logical_state(o)
    assert states_equal(gs, os_), state_diff(gs, os_)
    g.close()


def test_each_result_is_the_same_alone_and_in_the_mix():
    """Client A's transactions touch branches 0-4, client B's branches 5-9.
    A's results are identical whether A runs alone or interleaved with B on
    the device (their bulks mixed and overlapping)."""
    A = 10_000
    rng = np.random.default_rng(5)
    a = W.dc_bulk(20_000, A // 2, 0.9, seed=41)            # accounts [0, 5000): branches 0-4
    b = W.dc_bulk(20_000, A // 2, 0.9, seed=42)
    b["params"][:, 0] += A // 2                            # accounts [5000, 10000): branches 5-9
    # alone
    g1 = dc_db(A=A)
    s1 = G.Server(g1, deadline_us=200, max_bulk=2048, max_inflight=3)
    f1 = trickle(s1, a, rng)
    s1.drain()
    ra = s1.results(f1, 20_000)
    s1.close()
    # in the mix: interleave chunks of A and B
    g2 = dc_db(A=A)
    s2 = G.Server(g2, deadline_us=200, max_bulk=2048, max_inflight=3)
    ids_a = []
    ia = ib = 0
    while ia < 20_000 or ib < 20_000:
        if ia < 20_000:
            k = int(rng.integers(1, 900))
            f = s2.submit(a["type"][ia:ia + k], a["params"][ia:ia + k])
            ids_a.extend(range(f, f + min(k, 20_000 - ia)))
            ia += k
        if ib < 20_000:
            k = int(rng.integers(1, 900))
            s2.submit(b["type"][ib:ib + k], b["params"][ib:ib + k])
            ib += k
    s2.drain()
    ids_a = np.asarray(ids_a)
    st2, v2, _, nd = s2.results(0, 40_000)
    s2.close()
    assert nd == 40_000
    assert np.array_equal(st2[ids_a], ra[0]) and np.array_equal(v2[ids_a], ra[1])
    # A's accounts end the same in both databases
    acc1 = g1.read(G.TBL_DC_ACCOUNT)[:, 0]
    acc2 = g2.read(G.TBL_DC_ACCOUNT)[:, 0]
    assert np.array_equal(acc1[: A // 2], acc2[: A // 2])
    g1.close()
    g2.close()


def test_mixed_schemas_served():
    """Subscriber inserts/deletes and order-entry transactions through the
    server (insert slots and hash indexes across consecutive bulks)."""
    n_sub, n_wh, n_items = 400, 2, 300
    sub = W.sub_tables(n_sub, seed=3)
    oe = W.oe_tables(n_wh, n_items=n_items, seed=4)
    cap = 1 << 17
    g = G.Database(sub=n_sub, oe=(n_wh, n_items), order_capacity=cap, orderline_capacity=cap * 15,
                   sub_child_capacity=1 << 15, max_bulk=1 << 13)
    g.register(G.SUB_TYPES + G.OE_TYPES)
    for rows in (W.sub_rows(sub), W.oe_rows(oe)):
        for t, r in rows.items():
            g.load(t, r)
    o = oracle.OracleDB(sub=sub, oe=oe, ord_cap=cap, ol_cap=cap * 15, oid_cap=cap)
    n = 30_000
    rng = np.random.default_rng(9)
    parts = [W.sub_bulk(n, n_sub, 0.6, seed=7), W.oe_bulk(n, n_wh, n_items=n_items, remote_frac=0.1, seed=8)]
    bulk = W.concat_bulks(parts, rng.integers(0, 2, size=n))
    srv = G.Server(g, deadline_us=300, max_bulk=4096, max_inflight=3, params_per_txn=bulk["P"],
                   conflict_mode=G.CONFLICT_ADD)
    trickle(srv, bulk, rng, max_chunk=2000)
    srv.drain()
    st, vals, _, nd = srv.results(0, n)
    srv.close()
    assert nd == n
    ost, oout = o.execute(bulk, R=g.width)
    assert np.array_equal(st, ost) and np.array_equal(vals, oout)
    gs = gpu_logical_state(g, sub=True, oe=True, n_sub=n_sub)
    os_ = oracle_logical_state(o)
    assert states_equal(gs, os_), state_diff(gs, os_)
    g.close()


def test_admission_refuses_what_does_not_fit():
    g = dc_db(cap=5000)
    srv = G.Server(g, deadline_us=100, max_bulk=1024, queue_capacity=3000)
    bulk = W.dc_bulk(4000, 10_000, 0.0, seed=1)
    with pytest.raises(G.GputxError) as e:
        srv.submit(bulk["type"], bulk["params"])           # above the queue capacity
    assert e.value.status == G.ENOMEM
    srv.submit(bulk["type"][:2500], bulk["params"][:2500])
    srv.drain()
    srv.submit(bulk["type"][2500:4000], bulk["params"][2500:4000])
    srv.drain()
    with pytest.raises(G.GputxError) as e:                 # history holds 5000 rows
        srv.submit(bulk["type"][:1500], bulk["params"][:1500])
    assert e.value.status == G.ENOMEM
    stats = srv.stats()
    assert stats["completed"] == 4000 and stats["refused"] == 4000 + 1500
    srv.close()
    g.close()


def test_admission_by_free_device_memory():
    """With min_free_bytes set, a submission is refused (ENOMEM, counted)
    while free device memory is below the limit, and the same submission is
    admitted once memory is freed."""
    import torch
    torch.cuda.init()
    g = dc_db()
    bulk = W.dc_bulk(2000, 10_000, 0.0, seed=2)
    probe = G.Server(g, deadline_us=100, max_bulk=1024)   # the server's own allocations
    probe.submit(bulk["type"][:10], bulk["params"][:10])
    probe.drain()
    probe.close()
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    limit = free0 - (2 << 30)
    srv = G.Server(g, deadline_us=100, max_bulk=1024, min_free_bytes=limit)
    srv.submit(bulk["type"][:500], bulk["params"][:500])  # 2 GiB above the limit: admitted
    srv.drain()
    hog = torch.empty(6 << 30, dtype=torch.uint8, device="cuda")
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] < limit
    with pytest.raises(G.GputxError) as e:
        srv.submit(bulk["type"][500:2000], bulk["params"][500:2000])
    assert e.value.status == G.ENOMEM
    assert srv.stats()["refused"] == 1500
    del hog
    torch.cuda.empty_cache()
    torch.cuda.synchronize()
    srv.submit(bulk["type"][500:2000], bulk["params"][500:2000])
    srv.drain()
    st, vals, _, nd = srv.results(0, 2000)
    stats = srv.stats()
    srv.close()
    assert nd == 2000 and stats["completed"] == 2000 and stats["refused"] == 1500
    o = oracle.OracleDB(dc=W.dc_tables(10, 100, 10_000), hist_cap=1 << 20)
    o.execute({"ts": bulk["ts"][:10], "type": bulk["type"][:10], "params": bulk["params"][:10], "P": 2}, R=1)
    ost, oout = o.execute(bulk, R=1)
    assert np.array_equal(st, ost) and np.array_equal(vals, oout)
    g.close()


def test_served_mix_config5_against_the_oracle():
    """The served mix: debit-credit (10M accounts) and subscriber (2M
    subscribers with their child tables) in one device-resident database,
    a 50/50 mix submitted open-loop at Poisson arrival times (5M txn/s,
    1 ms deadline, three bulks in flight).  The whole served stream equals
    serial execution in id order: every result, every table, every index."""
    A, n_sub, n = 10_000_000, 2_000_000, 1_000_000
    sub = W.sub_tables(n_sub, seed=W.seed_for(5, 1))
    dc = W.dc_tables(1000, 10_000, A)
    g = G.Database(dc=(1000, 10_000, A), sub=n_sub, history_capacity=n, sub_child_capacity=6 * n_sub,
                   max_bulk=1 << 20)
    g.register(G.DC_TYPES + G.SUB_TYPES)
    for rows in (W.dc_rows(dc), W.sub_rows(sub)):
        for t, r in rows.items():
            g.load(t, r)
    bulk = W.served_mix(n, A, n_sub, 0.0, 5e6)
    srv = G.Server(g, deadline_us=1000, max_bulk=1 << 20, max_inflight=3, params_per_txn=bulk["P"])
    t0 = G.gputx_clock_ns() + 2_000_000
    arrivals = t0 + bulk["arrival_offset_ns"]
    i = 0
    while i < n:
        j = int(np.searchsorted(arrivals, G.gputx_clock_ns(), side="right"))
        if j > i:
            srv.submit(bulk["type"][i:j], bulk["params"][i:j], arrivals[i:j])
            i = j
        else:
            time.sleep(20e-6)
    srv.drain()
    st, vals, _, nd = srv.results(0, n)
    stats = srv.stats()
    srv.close()
    assert nd == n and stats["completed"] == n and stats["bulks"] > 1
    o = oracle.OracleDB(dc=dc, sub=sub, hist_cap=n)
    ost, oout = o.execute(bulk, R=g.width)
    bad = np.flatnonzero((st != ost) | (vals != oout).any(axis=1))
    assert len(bad) == 0, (len(bad), bad[:5])
    gs = gpu_logical_state(g, dc=True, sub=True, n_sub=n_sub)
    os_ = oracle_logical_state(o)
    assert states_equal(gs, os_), state_diff(gs, os_)
    assert not check_indexes(g, o, sub=True)
    g.close()
