"""Batched execution through captured CUDA graphs, and the online autotuner.

A stream of uneven, mixed-type transactions runs as consecutive fixed-capacity
bulks replayed from CUDA graphs (padding the last bulk); the autotuner tries
configurations on the stream's own first bulks.  Every transaction runs
exactly once in timestamp order, so results and state must equal serial
execution bit for bit (tolerance 0).
"""
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


@pytest.mark.parametrize("strategy,mode,size", [("kset", 0, 4096), ("kset", 1, 1 << 14), ("tpl", 0, 4096),
                                                ("tpl", 1, 1 << 14)])
def test_graph_bulks_equal_serial_execution(strategy, mode, size):
    A = 20_000
    g = G.Database(dc=(20, 200, A), history_capacity=1 << 20, max_bulk=1 << 16)
    g.register(G.DC_TYPES)
    o = oracle.OracleDB(dc=W.dc_tables(20, 200, A), hist_cap=1 << 20)
    bt = G.Batcher(g, tune=False, strategy=strategy, conflict_mode=mode, bulk_size=size)
    ts0 = 0
    for k, n in enumerate([10_001, 3, 25_000]):     # not multiples of the bulk size
        bulk = W.dc_bulk(n, A, 0.8, seed=70 + k, ts0=ts0)
        ts0 += n
        st, out = bt.run(bulk["ts"], bulk["type"], bulk["params"])
        ost, oout = o.execute(bulk, R=1)
        assert np.array_equal(st, ost) and np.array_equal(out, oout), (k, n)
    bt.close()
    gs, os_ = gpu_logical_state(g, dc=True), oracle_logical_state(o)
    assert states_equal(gs, os_), state_diff(gs, os_)
    g.close()


@pytest.mark.parametrize("mode", [G.CONFLICT_PAPER, G.CONFLICT_ADD])
def test_autotuned_order_entry_stream(mode):
    """Order-entry (multi-item transactions: the exact-depth pass runs on the
    device inside the graph) with the autotuner choosing strategy, bulk size
    and block shape on the stream's first bulks."""
    n_wh, n_items = 8, 20_000
    init = W.oe_tables(n_wh, n_items=n_items, seed=W.seed_for(4, 50))
    cap = 1 << 22
    g = G.Database(oe=(n_wh, n_items), order_capacity=cap, orderline_capacity=cap * 15, max_bulk=1 << 18)
    g.register(G.OE_TYPES)
    for t, rows in W.oe_rows(init).items():
        g.load(t, rows)
    o = oracle.OracleDB(oe=init, ord_cap=cap, ol_cap=cap * 15, oid_cap=1 << 16)
    bt = G.Batcher(g, tune=True, conflict_mode=mode, bulk_size_max=1 << 18, params_per_txn=W.OE_PARAMS)
    rng = np.random.default_rng(W.seed_for(4, 51))
    ts0 = 0
    for k in range(4):
        n = int(2 ** rng.uniform(10, 19))
        bulk = W.oe_bulk(n, n_wh, n_items=n_items, seed=W.seed_for(4, 60 + k), ts0=ts0)
        ts0 += n
        st, out = bt.run(bulk["ts"], bulk["type"], bulk["params"])
        ost, oout = o.execute(bulk, R=g.width)
        assert np.array_equal(st, ost) and np.array_equal(out, oout), (k, n)
    big = W.oe_bulk(1_500_000, n_wh, n_items=n_items, seed=W.seed_for(4, 70), ts0=ts0)
    st, out = bt.run(big["ts"], big["type"], big["params"])
    ost, oout = o.execute(big, R=g.width)
    assert np.array_equal(st, ost) and np.array_equal(out, oout)
    ch = bt.choice()
    bt.close()
    assert ch["tuned"] and len(ch["measured"]) >= 3
    assert ch["strategy"] in (G.KSET, G.TPL, G.PART) and ch["bulk_size"] <= 1 << 18
    gs, os_ = gpu_logical_state(g, oe=True), oracle_logical_state(o)
    assert states_equal(gs, os_), state_diff(gs, os_)
    g.close()


def test_mixed_schema_stream_through_graphs():
    B, T, A, n_sub = 8, 32, 3200, 300
    sub = W.sub_tables(n_sub, seed=13)
    dc = W.dc_tables(B, T, A)
    g = G.Database(dc=(B, T, A), sub=n_sub, history_capacity=1 << 18, sub_child_capacity=1 << 15,
                   max_bulk=1 << 14)
    g.register(G.DC_TYPES + G.SUB_TYPES)
    for rows in (W.dc_rows(dc), W.sub_rows(sub)):
        for t, r in rows.items():
            g.load(t, r)
    o = oracle.OracleDB(dc=dc, sub=sub, hist_cap=1 << 18)
    n = 40_000
    rng = np.random.default_rng(14)
    bulk = W.concat_bulks([W.dc_bulk(n, A, 0.5, seed=15), W.sub_bulk(n, n_sub, 0.5, seed=16)],
                          rng.integers(0, 2, size=n))
    bt = G.Batcher(g, tune=True, params_per_txn=bulk["P"], bulk_size_max=1 << 14)
    st, out = bt.run(bulk["ts"], bulk["type"], bulk["params"])
    bt.close()
    ost, oout = o.execute(bulk, R=g.width)
    assert np.array_equal(st, ost) and np.array_equal(out, oout)
    gs = gpu_logical_state(g, dc=True, sub=True, n_sub=n_sub)
    os_ = oracle_logical_state(o)
    assert states_equal(gs, os_), state_diff(gs, os_)
    g.close()


def test_config4_stream_at_full_size():
    """The benchmark's batched order-entry run: 64 warehouses x 10 districts
    x 3,000 customers, 100,000 items, 18 uneven bulks of 2^10..2^21 (4.28M
    transactions) through the tuned graph batcher, bulk boundaries kept.  Every output, every
    table and the order index equal serial execution of the whole stream."""
    n_wh, n_items = 64, 100_000
    init = W.oe_tables(n_wh, n_items=n_items, seed=W.seed_for(4))
    sizes, bulk = W.oe_stream(3_000_000, n_wh, n_items)
    total = sum(sizes)
    cap = 2 * total + (1 << 22)
    g = G.Database(oe=(n_wh, n_items), order_capacity=cap, orderline_capacity=cap * 15, max_bulk=1 << 21)
    g.register(G.OE_TYPES)
    for t, rows in W.oe_rows(init).items():
        g.load(t, rows)
    bt = G.Batcher(g, tune=True, params_per_txn=W.OE_PARAMS, bulk_size_max=1 << 21)
    st, out = bt.run_bulks(bulk["ts"], bulk["type"], bulk["params"], sizes)
    ch = bt.choice()
    bt.close()
    assert len(ch["measured"]) >= 3 and 0 < ch["p50_us"] <= ch["p99_us"]
    o = oracle.OracleDB(oe=init, ord_cap=total, ol_cap=total * 15, oid_cap=1 << 16)
    ost, oout = o.execute(bulk, R=g.width)
    bad = np.flatnonzero((st != ost) | (out != oout).any(axis=1))
    assert len(bad) == 0, (len(bad), bad[:5])
    gs, os_ = gpu_logical_state(g, oe=True), oracle_logical_state(o)
    assert states_equal(gs, os_), state_diff(gs, os_)
    assert not check_indexes(g, o, oe=True)
    g.close()


@pytest.mark.parametrize("strategy,mode", [("kset", 0), ("kset", 1), ("tpl", 0), ("part", 0)])
@pytest.mark.parametrize("schema", ["dc", "oe"])
def test_uneven_bulks_in_segments(strategy, mode, schema):
    """Bulks of uneven sizes (empty and one-transaction bulks among them, and
    bulks larger than the segment capacity) through segmented graph replays:
    several bulks share one persistent launch, each with its own k-sets under
    K-SET.  A PART segment holding a cross-partition order-entry transaction
    runs nothing and is re-run with TPL.  Results equal serial execution."""
    rng = np.random.default_rng(81)
    sizes = [0, 1, 3000, 17, 9000, 1, 40000, 0, 2500, 777, 65536, 12]
    total = sum(sizes)
    if schema == "dc":
        A = 20_000
        g = G.Database(dc=(20, 200, A), history_capacity=1 << 20, max_bulk=1 << 15)
        g.register(G.DC_TYPES)
        o = oracle.OracleDB(dc=W.dc_tables(20, 200, A), hist_cap=1 << 20)
        bulk = W.dc_bulk(total, A, 0.8, seed=82)
        kw = {}
    else:
        n_wh, n_items = 4, 2000
        init = W.oe_tables(n_wh, n_items=n_items, seed=83)
        cap = 1 << 18
        g = G.Database(oe=(n_wh, n_items), order_capacity=cap, orderline_capacity=cap * 15, max_bulk=1 << 15)
        g.register(G.OE_TYPES)
        for t, rows in W.oe_rows(init).items():
            g.load(t, rows)
        o = oracle.OracleDB(oe=init, ord_cap=cap, ol_cap=cap * 15, oid_cap=1 << 16)
        bulk = W.oe_bulk(total, n_wh, n_items=n_items, remote_frac=0.002, seed=84)
        kw = {"params_per_txn": W.OE_PARAMS}
    bt = G.Batcher(g, tune=False, strategy=strategy, conflict_mode=mode, bulk_size=1 << 15, **kw)
    st, out = bt.run_bulks(bulk["ts"], bulk["type"], bulk["params"], sizes)
    ch = bt.choice()
    bt.close()
    assert ch["bulks_run"] < len([x for x in sizes if x])    # bulks share segments
    ost, oout = o.execute(bulk, R=g.width)
    bad = np.flatnonzero((st != ost) | (out != oout).any(axis=1))
    assert len(bad) == 0, (len(bad), bad[:5])
    kw2 = {"dc": True} if schema == "dc" else {"oe": True}
    gs, os_ = gpu_logical_state(g, **kw2), oracle_logical_state(o)
    assert states_equal(gs, os_), state_diff(gs, os_)
    g.close()
