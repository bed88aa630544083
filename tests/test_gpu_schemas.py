"""Subscriber-location, order-entry and mixed-schema parity against the oracle.

Bit-exact (integer columns, tolerance 0): per-transaction status and outputs,
and the logical database state (keyed tables compared row by row, child and
order tables compared as sets keyed by their primary keys, history by ts).
"""
import numpy as np
import pytest

import oracle
import paper_1103_3105_gb300 as G
import workloads as W
from tests._helpers import check_indexes, gpu_logical_state, oracle_logical_state, state_diff, states_equal

pytestmark = pytest.mark.gpu

STRATS = ["kset", "part", "tpl", "auto"]


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()


# ---------------------------------------------------------------------------
# builders
# ---------------------------------------------------------------------------
def sub_pair(n_sub, seed=1, max_bulk=1 << 16, **kw):
    init = W.sub_tables(n_sub, seed=seed)
    g = G.Database(sub=n_sub, max_bulk=max_bulk, **kw)
    g.register(G.SUB_TYPES)
    for t, rows in W.sub_rows(init).items():
        g.load(t, rows)
    return g, oracle.OracleDB(sub=init)


def oe_pair(n_wh, n_items, seed=2, max_bulk=1 << 16, ord_cap=1 << 18, **kw):
    init = W.oe_tables(n_wh, n_items=n_items, seed=seed)
    g = G.Database(oe=(n_wh, n_items), order_capacity=ord_cap, orderline_capacity=ord_cap * 15,
                   max_bulk=max_bulk, **kw)
    g.register(G.OE_TYPES)
    for t, rows in W.oe_rows(init).items():
        g.load(t, rows)
    # o_ids per district stay far below the total order count
    oid_cap = max(1000, 3 * ord_cap // (n_wh * 10))
    o = oracle.OracleDB(oe=init, ord_cap=ord_cap, ol_cap=ord_cap * 15, oid_cap=oid_cap)
    return g, o


def run_both(g, o, bulk, strategy, mode=0, R=None):
    b = g.submit_dict(bulk).execute(strategy, conflict_mode=mode)
    stats = b.sync()
    st, out = b.results()
    b.free()
    ost, oout = o.execute(bulk, R=g.width)
    return stats, st, out, ost, oout


def check(g, o, st, out, ost, oout, **kw):
    bad = np.flatnonzero((st != ost) | (out != oout).any(axis=1))
    assert len(bad) == 0, (len(bad), bad[:5], st[bad[:5]], ost[bad[:5]], out[bad[:3]], oout[bad[:3]])
    gs, os_ = gpu_logical_state(g, **kw), oracle_logical_state(o)
    assert states_equal(gs, os_), state_diff(gs, os_)
    # the primary indexes themselves: every live row found by its key, every
    # entry pointing at a live row with that key
    bad = check_indexes(g, o, sub=kw.get("sub", False), oe=kw.get("oe", False))
    assert not bad, bad


# ---------------------------------------------------------------------------
# subscriber-location
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("strategy", STRATS)
@pytest.mark.parametrize("theta", [0.0, 0.8])
def test_subscriber_mix(strategy, theta):
    n_sub = 3000
    g, o = sub_pair(n_sub)
    ts0 = 0
    for k, n in enumerate([1, 700, 9000, 20000]):
        bulk = W.sub_bulk(n, n_sub, theta, seed=10 * k + int(theta * 10), ts0=ts0)
        ts0 += n
        _, st, out, ost, oout = run_both(g, o, bulk, strategy, k % 2)
        check(g, o, st, out, ost, oout, sub=True, n_sub=n_sub)
    g.close()


def test_subscriber_insert_delete_churn():
    """Insert/delete-heavy bulks on few subscribers: hash tombstones are
    reused, deleted keys come back, and later levels see earlier inserts."""
    n_sub = 50
    g, o = sub_pair(n_sub, seed=5, sub_child_capacity=1 << 15)
    mix = (0.1, 0.05, 0.15, 0.05, 0.05, 0.35, 0.25)
    ts0 = 0
    for k in range(6):
        bulk = W.sub_bulk(3000, n_sub, 0.5, seed=100 + k, ts0=ts0, mix=mix)
        ts0 += 3000
        _, st, out, ost, oout = run_both(g, o, bulk, STRATS[k % 3])
        check(g, o, st, out, ost, oout, sub=True, n_sub=n_sub)
    g.close()


def test_subscriber_full_size():
    """10,000,000 subscribers, a bulk of 2^20 mixed transactions, Zipf 0.8."""
    n_sub = 10_000_000
    g, o = sub_pair(n_sub, seed=W.seed_for(3), max_bulk=1 << 20)
    bulk = W.sub_bulk(1 << 20, n_sub, 0.8, seed=W.seed_for(3, 1))
    _, st, out, ost, oout = run_both(g, o, bulk, "kset")
    assert np.array_equal(st, ost) and np.array_equal(out, oout)
    # every table, child-row fields included, and the three indexes
    check(g, o, st, out, ost, oout, sub=True, n_sub=n_sub)
    g.close()


# ---------------------------------------------------------------------------
# order-entry
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("strategy", STRATS)
@pytest.mark.parametrize("mode", [G.CONFLICT_PAPER, G.CONFLICT_ADD])
def test_order_entry_mix(strategy, mode):
    n_wh, n_items = 2, 500
    g, o = oe_pair(n_wh, n_items)
    ts0 = 0
    for k, n in enumerate([1, 300, 5000, 12000]):
        bulk = W.oe_bulk(n, n_wh, n_items=n_items, remote_frac=0.05, invalid_frac=0.02, seed=k, ts0=ts0)
        ts0 += n
        stats, st, out, ost, oout = run_both(g, o, bulk, strategy, mode)
        check(g, o, st, out, ost, oout, oe=True)
    g.close()


@pytest.mark.parametrize("mode", [G.CONFLICT_PAPER, G.CONFLICT_ADD])
def test_order_entry_levels_exact(mode):
    """Multi-item transactions need the exact-depth pass: the engine's depth
    and 0-set size must equal the longest-path depths of the oracle."""
    n_wh, n_items = 3, 200
    g, o = oe_pair(n_wh, n_items)
    bulk = W.oe_bulk(6000, n_wh, n_items=n_items, remote_frac=0.2, invalid_frac=0.02, seed=77)
    obj, cls, root = o.extract(bulk, mode, oracle.MAX_OPS)
    lv = oracle.levels(obj, cls, o.num_objects())
    d, w0, c = oracle.graph_stats(lv, root)
    stats, st, out, ost, oout = run_both(g, o, bulk, "kset", mode)
    check(g, o, st, out, ost, oout, oe=True)
    assert (stats["depth"], stats["w0"], stats["cross"]) == (d, w0, c)
    g.close()


def test_order_entry_part_falls_back_on_cross_partition():
    g, o = oe_pair(4, 300)
    bulk = W.oe_bulk(4000, 4, n_items=300, remote_frac=0.3, seed=8)
    stats, st, out, ost, oout = run_both(g, o, bulk, "part")
    assert stats["fallback"] == 1 and stats["strategy"] == G.TPL
    check(g, o, st, out, ost, oout, oe=True)
    local = W.oe_bulk(4000, 4, n_items=300, remote_frac=0.0, seed=9, ts0=4000)
    stats, st, out, ost, oout = run_both(g, o, local, "part")
    assert stats["fallback"] == 0 and stats["strategy"] == G.PART
    check(g, o, st, out, ost, oout, oe=True)
    g.close()


@pytest.mark.parametrize("mode", [G.CONFLICT_PAPER, G.CONFLICT_ADD])
def test_auto_refines_only_for_kset(mode):
    """AUTO decides on the one-pass ranks: a TPL or PART pick runs no
    exact-depth pass; a K-SET pick (forced by a zero 0-set threshold) runs
    it and reaches the exact longest-path depths."""
    n_wh, n_items = 3, 200
    bulk = W.oe_bulk(6000, n_wh, n_items=n_items, remote_frac=0.2, invalid_frac=0.02, seed=78)
    ob = oracle.OracleDB(oe=W.oe_tables(n_wh, n_items=n_items, seed=2), ord_cap=1, ol_cap=1, oid_cap=1)
    obj, cls, root = ob.extract(bulk, mode, oracle.MAX_OPS)
    lv = oracle.levels(obj, cls, ob.num_objects())
    d, w0, c = oracle.graph_stats(lv, root)
    # Algorithm 1's K-SET threshold above any 0-set: TPL (c > 0), no rounds
    g, o = oe_pair(n_wh, n_items, kset_w0_min=1 << 30)
    stats, st, out, ost, oout = run_both(g, o, bulk, "auto", mode)
    assert stats["strategy"] == G.TPL and stats["fixpoint_rounds"] == 0
    assert stats["w0"] == w0 and stats["cross"] == c and stats["depth"] <= d
    check(g, o, st, out, ost, oout, oe=True)
    g.close()
    # threshold 1: K-SET, refined to the exact depths
    g, o = oe_pair(n_wh, n_items, kset_w0_min=1)
    stats, st, out, ost, oout = run_both(g, o, bulk, "auto", mode)
    assert stats["strategy"] == G.KSET and stats["fixpoint_rounds"] > 0
    assert (stats["depth"], stats["w0"], stats["cross"]) == (d, w0, c)
    check(g, o, st, out, ost, oout, oe=True)
    g.close()


def test_order_entry_config4_uneven_bulks():
    """64 warehouses x 10 districts x 3,000 customers, 100,000 items; bulks
    of uneven size between 2^10 and 2^21."""
    n_wh, n_items = 64, 100_000
    g, o = oe_pair(n_wh, n_items, seed=W.seed_for(4), max_bulk=1 << 21, ord_cap=1 << 22)
    rng = np.random.default_rng(W.seed_for(4, 1))
    ts0 = 0
    for k in range(4):
        n = int(2 ** rng.uniform(10, 21))
        bulk = W.oe_bulk(n, n_wh, n_items=n_items, seed=W.seed_for(4, 10 + k), ts0=ts0)
        ts0 += n
        stats, st, out, ost, oout = run_both(g, o, bulk, ["kset", "tpl", "auto", "kset"][k], k % 2)
        assert np.array_equal(st, ost) and np.array_equal(out, oout), (k, n)
    check(g, o, st, out, ost, oout, oe=True)
    g.close()


# ---------------------------------------------------------------------------
# all three schemas in one database and one bulk
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("strategy", STRATS)
def test_mixed_schemas(strategy):
    B, T, A, n_sub, n_wh, n_items = 8, 32, 3200, 500, 2, 300
    sub = W.sub_tables(n_sub, seed=3)
    oe = W.oe_tables(n_wh, n_items=n_items, seed=4)
    dc = W.dc_tables(B, T, A)
    cap = 1 << 16
    g = G.Database(dc=(B, T, A), sub=n_sub, oe=(n_wh, n_items), history_capacity=cap,
                   order_capacity=cap, orderline_capacity=cap * 15, max_bulk=1 << 15)
    g.register(G.DC_TYPES + G.SUB_TYPES + G.OE_TYPES)
    for rows in (W.dc_rows(dc), W.sub_rows(sub), W.oe_rows(oe)):
        for t, r in rows.items():
            g.load(t, r)
    o = oracle.OracleDB(dc=dc, sub=sub, oe=oe, hist_cap=cap, ord_cap=cap, ol_cap=cap * 15, oid_cap=cap)
    ts0 = 0
    for k, n in enumerate([5000, 12000]):
        rng = np.random.default_rng(k)
        parts = [W.dc_bulk(n, A, 0.5, seed=k), W.sub_bulk(n, n_sub, 0.5, seed=k + 1),
                 W.oe_bulk(n, n_wh, n_items=n_items, remote_frac=0.1, seed=k + 2)]
        bulk = W.concat_bulks(parts, rng.integers(0, 3, size=n))
        bulk["ts"] += ts0
        ts0 += n
        stats, st, out, ost, oout = run_both(g, o, bulk, strategy, k % 2)
        check(g, o, st, out, ost, oout, dc=True, sub=True, oe=True, n_sub=n_sub)
    g.close()
