"""Relaxed timestamp constraint (Appendix G): serializability.

PART_RELAXED groups by partition with counters (no sort) and TPL_RELAXED uses
plain spin locks, so a bulk's results equal serial execution in SOME order.
The engine reports that order (gputx_bulk_order); the oracle executes the bulk
serially in exactly that order, and every status, output and the final
database must match bit for bit (tolerance 0).
"""
import numpy as np
import pytest

import oracle
import paper_1103_3105_gb300 as G
import workloads as W
from tests._helpers import gpu_logical_state, oracle_logical_state, state_diff, states_equal

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()


def run_relaxed(g, o, bulk, strategy, mode=G.CONFLICT_PAPER, R=1):
    b = g.submit_dict(bulk).execute(strategy, conflict_mode=mode)
    stats = b.sync()
    st, out = b.results()
    order = b.order()
    b.free()
    n = len(bulk["ts"])
    assert np.array_equal(np.sort(order), np.arange(n, dtype=np.uint32))   # a permutation
    ost, oout = o.execute(bulk, R=R, order=order.astype(np.int64))
    assert np.array_equal(st, ost)
    assert np.array_equal(out, oout)
    return stats, order


@pytest.mark.parametrize("strategy", ["part_relaxed", "tpl_relaxed"])
@pytest.mark.parametrize("theta", [0.0, 0.99])
def test_debit_credit(strategy, theta):
    B, T, A = 20, 200, 20_000
    g = G.Database(dc=(B, T, A), history_capacity=1 << 18, max_bulk=1 << 16)
    g.register(G.DC_TYPES)
    o = oracle.OracleDB(dc=W.dc_tables(B, T, A), hist_cap=1 << 18)
    for k, mode in enumerate([G.CONFLICT_PAPER, G.CONFLICT_ADD]):
        bulk = W.dc_bulk(30_000 + k, A, theta, seed=W.seed_for(6, int(theta * 100) + k), ts0=k * 40_000)
        stats, order = run_relaxed(g, o, bulk, strategy, mode)
        if strategy == "part_relaxed":
            # one partition per branch: the order keeps each branch's
            # transactions together
            br = bulk["params"][order, 0] // (A // B)
            assert len(np.unique(br)) == len(np.flatnonzero(np.diff(br) != 0)) + 1
    gs, os_ = gpu_logical_state(g, dc=True), oracle_logical_state(o)
    assert states_equal(gs, os_), state_diff(gs, os_)
    g.close()


@pytest.mark.parametrize("strategy", ["part_relaxed", "tpl_relaxed"])
def test_mixed_schemas(strategy):
    """Subscriber and order-entry transactions (inserts, deletes, hash
    indexes, multi-item access sets).  Remote order lines make transactions
    cross partitions: PART_RELAXED falls back to TPL_RELAXED."""
    n_sub, n_wh, n_items = 300, 3, 200
    sub = W.sub_tables(n_sub, seed=41)
    oe = W.oe_tables(n_wh, n_items=n_items, seed=42)
    cap = 1 << 16
    g = G.Database(sub=n_sub, oe=(n_wh, n_items), order_capacity=cap, orderline_capacity=cap * 15,
                   sub_child_capacity=1 << 15, max_bulk=1 << 15)
    g.register(G.SUB_TYPES + G.OE_TYPES)
    for rows in (W.sub_rows(sub), W.oe_rows(oe)):
        for t, r in rows.items():
            g.load(t, r)
    o = oracle.OracleDB(sub=sub, oe=oe, ord_cap=cap, ol_cap=cap * 15, oid_cap=cap)
    rng = np.random.default_rng(43)
    n = 12_000
    for k, remote in enumerate([0.0, 0.1]):
        parts = [W.sub_bulk(n, n_sub, 0.6, seed=44 + k, ts0=k * n),
                 W.oe_bulk(n, n_wh, n_items=n_items, remote_frac=remote, seed=46 + k, ts0=k * n)]
        bulk = W.concat_bulks(parts, rng.integers(0, 2, size=n))
        stats, _ = run_relaxed(g, o, bulk, strategy, R=g.width)
        if strategy == "part_relaxed":
            assert stats["fallback"] == (1 if remote > 0 else 0)
    gs = gpu_logical_state(g, sub=True, oe=True, n_sub=n_sub)
    os_ = oracle_logical_state(o)
    assert states_equal(gs, os_), state_diff(gs, os_)
    g.close()


@pytest.mark.parametrize("strategy", ["part_relaxed", "tpl_relaxed"])
def test_invalid_bulk_changes_nothing(strategy):
    g = G.Database(dc=(4, 40, 4000), history_capacity=1 << 14, max_bulk=1 << 12)
    g.register(G.DC_TYPES)
    before = gpu_logical_state(g, dc=True)
    bulk = W.dc_bulk(500, 4000, 0.0, seed=51)
    bulk["params"][123, 0] = -1
    b = g.submit_dict(bulk).execute(strategy)
    with pytest.raises(G.GputxError) as e:
        b.sync()
    assert e.value.status == G.EINVAL
    b.free()
    assert states_equal(before, gpu_logical_state(g, dc=True))
    g.close()


def test_spin_locks_time_out_instead_of_hanging():
    """A 1 ns wait limit on contended spin locks: ETIMEOUT, and the database
    stays usable (every lock released)."""
    g = G.Database(dc=(4, 40, 4000), history_capacity=1 << 16, max_bulk=1 << 14, spin_limit_ns=1)
    g.register(G.DC_TYPES)
    b = g.submit_dict(W.dc_bulk(4096, 4000, 0.0, seed=52)).execute("tpl_relaxed")
    with pytest.raises(G.GputxError) as e:
        b.sync()
    assert e.value.status == G.ETIMEOUT
    b.free()
    # one transaction per branch: nothing contends, so with the same 1 ns
    # limit any lock left held would time out again
    one = {"ts": np.arange(4, dtype=np.int64), "type": np.zeros(4, np.int32),
           "params": np.array([[0, 5], [1000, 6], [2000, 7], [3000, 8]], dtype=np.int64), "P": 2}
    b = g.submit_dict(one).execute("tpl_relaxed")
    st, _ = b.results()
    assert np.array_equal(st, np.zeros(4, np.int32))
    b.free()
    g.close()


def test_spin_locks_time_out_on_other_schemas():
    """The same 1 ns limit in the general relaxed kernel (subscriber
    transactions on 8 subscribers, so nearly every lock is contended):
    ETIMEOUT, and a following bulk on distinct subscribers runs clean."""
    n_sub = 64
    sub = W.sub_tables(n_sub, seed=61)
    g = G.Database(sub=n_sub, sub_child_capacity=1 << 12, max_bulk=1 << 12, spin_limit_ns=1)
    g.register(G.SUB_TYPES)
    for t, r in W.sub_rows(sub).items():
        g.load(t, r)
    bulk = W.sub_bulk(4096, 8, 0.0, seed=62)
    b = g.submit_dict(bulk).execute("tpl_relaxed")
    with pytest.raises(G.GputxError) as e:
        b.sync()
    assert e.value.status == G.ETIMEOUT
    b.free()
    one = W.sub_bulk(n_sub, n_sub, 0.0, seed=63, ts0=10_000)
    one["params"][:, 0] = np.arange(n_sub)          # one transaction per subscriber
    one["type"][:] = G.T_SUB_GET_SUBSCRIBER         # reads only: nothing to insert
    one["params"][:, 1:] = 0
    b = g.submit_dict(one).execute("tpl_relaxed")
    st, _ = b.results()
    assert np.array_equal(st, np.zeros(n_sub, np.int32))
    b.free()
    g.close()


@pytest.mark.parametrize("theta", [0.0, 0.99])
@pytest.mark.parametrize("strategy,mode", [("tpl_relaxed", G.CONFLICT_PAPER), ("tpl_relaxed", G.CONFLICT_ADD),
                                           ("part_relaxed", G.CONFLICT_PAPER)])
def test_debit_credit_at_the_benchmark_size(theta, strategy, mode):
    """The relaxed strategies on the benchmark's tables (1,000 branches, 10,000
    tellers, 10,000,000 accounts) at 2^22 transactions (TPL_RELAXED: the
    CTA-combining kernel).  The oracle replays the reported order over the
    whole bulk; every output and every table must match."""
    A = 10_000_000
    tabs = W.dc_tables(1000, 10000, A)
    g = G.Database(dc=(1000, 10000, A), history_capacity=1 << 22, max_bulk=1 << 22)
    g.register(G.DC_TYPES)
    for t, r in W.dc_rows(tabs).items():
        g.load(t, r)
    o = oracle.OracleDB(dc=tabs, hist_cap=1 << 22)
    bulk = W.dc_bulk(1 << 22, A, theta, seed=W.seed_for(2, 700 + int(theta * 100)))
    run_relaxed(g, o, bulk, strategy, mode)
    assert np.array_equal(g.read(G.TBL_DC_ACCOUNT)[:, 0], o["acc_bal"])
    assert np.array_equal(g.read(G.TBL_DC_BRANCH)[:, 0], o["br_bal"])
    assert np.array_equal(g.read(G.TBL_DC_TELLER)[:, 0], o["tel_bal"])
    # the history rows are the same set; the oracle appended them in the
    # replayed order, so both sides are compared by timestamp
    h, oh = g.read(G.TBL_DC_HISTORY), o.history()
    assert np.array_equal(h[np.argsort(h[:, 0])], oh[np.argsort(oh[:, 0])])
    g.close()


@pytest.mark.parametrize("strategy", ["tpl_relaxed", "part_relaxed"])
def test_subscribers_at_the_benchmark_size(strategy):
    """The relaxed strategies (TPL_RELAXED with shared readers) on 10,000,000
    subscribers with their child tables, a bulk of 2^20 mixed transactions,
    Zipf 0.8: the oracle replays the reported order; outputs and the logical
    state must match."""
    n_sub = 10_000_000
    sub = W.sub_tables(n_sub, seed=W.seed_for(3))
    g = G.Database(sub=n_sub, sub_child_capacity=6 * n_sub, max_bulk=1 << 20)
    g.register(G.SUB_TYPES)
    for t, r in W.sub_rows(sub).items():
        g.load(t, r)
    o = oracle.OracleDB(sub=sub)
    bulk = W.sub_bulk(1 << 20, n_sub, 0.8, seed=W.seed_for(3, 1))
    run_relaxed(g, o, bulk, strategy, R=g.width)
    gs = gpu_logical_state(g, sub=True, n_sub=n_sub)
    os_ = oracle_logical_state(o)
    assert states_equal(gs, os_), state_diff(gs, os_)
    g.close()


def test_timestamp_strategies_report_timestamp_order():
    g = G.Database(dc=(4, 40, 4000), history_capacity=1 << 14, max_bulk=1 << 12)
    g.register(G.DC_TYPES)
    for s in ("kset", "part", "tpl", "scan"):
        b = g.submit_dict(W.dc_bulk(300, 4000, 0.0, seed=54)).execute(s)
        assert np.array_equal(b.order(), np.arange(300, dtype=np.uint32))
        b.free()
    g.close()
