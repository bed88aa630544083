"""Incremental 0-set execution (Section 5.3) against the oracle.

Transactions join a device-resident pool in chunks; every step executes the
pool's current 0-set.  Whatever the interleaving of adds and steps, the
outputs of all steps and the final database must equal serial execution of
the whole stream in timestamp order, bit for bit (tolerance 0).
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


def slice_bulk(bulk, a, b):
    return {"ts": bulk["ts"][a:b], "type": bulk["type"][a:b], "params": bulk["params"][a:b], "P": bulk["P"]}


def run_stream(g, pool, bulk, rng, max_chunk, steps_per_add=1):
    """Adds the bulk in random chunks with steps in between, then drains;
    returns {ts: (status, values)} and the number of steps."""
    got = {}
    n = len(bulk["ts"])
    i = steps = 0

    def step():
        nonlocal steps
        k = pool.step()
        if k:
            steps += 1
            ts, st, vals = pool.results()
            assert len(ts) == k and np.all(np.diff(ts) > 0)
            for t, s, v in zip(ts.tolist(), st.tolist(), vals):
                assert t not in got
                got[t] = (s, v.copy())
        return k

    while i < n:
        c = int(rng.integers(1, max_chunk + 1))
        part = slice_bulk(bulk, i, min(n, i + c))
        pool.add(part["ts"], part["type"], part["params"])
        i += len(part["ts"])
        for _ in range(steps_per_add):
            step()
    while pool.pending:
        assert step() > 0   # the oldest pending transaction is always in the 0-set
    return got, steps


def assert_matches(got, bulk, ost, oout):
    ts = bulk["ts"].tolist()
    assert sorted(got) == ts
    st = np.array([got[t][0] for t in ts], dtype=np.int32)
    out = np.stack([got[t][1] for t in ts])
    assert np.array_equal(st, ost)
    assert np.array_equal(out, oout)


@pytest.mark.parametrize("theta,mode", [(0.0, G.CONFLICT_PAPER), (0.99, G.CONFLICT_PAPER),
                                        (0.99, G.CONFLICT_ADD)])
def test_debit_credit_stream(theta, mode):
    B, T, A = 20, 200, 20_000
    tabs = W.dc_tables(B, T, A)
    g = G.Database(dc=(B, T, A), history_capacity=1 << 18, max_bulk=1 << 16)
    g.register(G.DC_TYPES)
    o = oracle.OracleDB(dc=tabs, hist_cap=1 << 18)
    pool = G.Pool(g, capacity=1 << 16, conflict_mode=mode)
    bulk = W.dc_bulk(60_000, A, theta, seed=W.seed_for(5, int(theta * 100) + mode))
    got, steps = run_stream(g, pool, bulk, np.random.default_rng(3), 4000)
    pool.close()
    ost, oout = o.execute(bulk, R=1)
    assert_matches(got, bulk, ost, oout)
    assert steps > 1
    gs, os_ = gpu_logical_state(g, dc=True), oracle_logical_state(o)
    assert states_equal(gs, os_), state_diff(gs, os_)
    g.close()


@pytest.mark.parametrize("mode", [G.CONFLICT_PAPER, G.CONFLICT_ADD])
def test_first_steps_are_the_zero_and_one_sets(mode):
    """One add, then steps: the first executes exactly the 0-set (level 0 of
    the oracle's exact levels), the second the former 1-set."""
    B, T, A = 4, 40, 4000
    g = G.Database(dc=(B, T, A), history_capacity=1 << 16, max_bulk=1 << 14)
    g.register(G.DC_TYPES)
    ob = oracle.OracleDB(dc=W.dc_tables(B, T, A), hist_cap=1 << 16)
    bulk = W.dc_bulk(3000, A, 0.8, seed=11 + mode)
    obj, cls, _ = ob.extract(bulk, mode, 3)
    lv = oracle.levels(obj, cls, ob.num_objects())
    pool = G.Pool(g, capacity=4096, conflict_mode=mode)
    pool.add(bulk["ts"], bulk["type"], bulk["params"])
    for level in (0, 1):
        k = pool.step()
        ts, _, _ = pool.results()
        assert k == int((lv == level).sum())
        assert np.array_equal(ts, bulk["ts"][lv == level])
    while pool.pending:
        pool.step()
    pool.close()
    g.close()


@pytest.mark.parametrize("mode", [G.CONFLICT_PAPER, G.CONFLICT_ADD])
def test_mixed_schema_stream(mode):
    """Subscriber inserts/deletes (hash indexes, insert areas) and order-entry
    transactions (multi-item access sets, inserts) through the pool."""
    n_sub, n_wh, n_items = 300, 2, 200
    sub = W.sub_tables(n_sub, seed=21)
    oe = W.oe_tables(n_wh, n_items=n_items, seed=22)
    cap = 1 << 16
    g = G.Database(sub=n_sub, oe=(n_wh, n_items), order_capacity=cap, orderline_capacity=cap * 15,
                   sub_child_capacity=1 << 15, max_bulk=1 << 14)
    g.register(G.SUB_TYPES + G.OE_TYPES)
    for rows in (W.sub_rows(sub), W.oe_rows(oe)):
        for t, r in rows.items():
            g.load(t, r)
    o = oracle.OracleDB(sub=sub, oe=oe, ord_cap=cap, ol_cap=cap * 15, oid_cap=cap)
    n = 20_000
    rng = np.random.default_rng(23 + mode)
    parts = [W.sub_bulk(n, n_sub, 0.6, seed=24), W.oe_bulk(n, n_wh, n_items=n_items, remote_frac=0.1, seed=25)]
    bulk = W.concat_bulks(parts, rng.integers(0, 2, size=n))
    pool = G.Pool(g, capacity=1 << 15, params_per_txn=bulk["P"], conflict_mode=mode)
    got, steps = run_stream(g, pool, bulk, rng, 1500, steps_per_add=2)
    pool.close()
    ost, oout = o.execute(bulk, R=g.width)
    assert_matches(got, bulk, ost, oout)
    gs = gpu_logical_state(g, sub=True, oe=True, n_sub=n_sub)
    os_ = oracle_logical_state(o)
    assert states_equal(gs, os_), state_diff(gs, os_)
    g.close()


def test_capacity_and_invalid_adds_change_nothing():
    g = G.Database(dc=(4, 40, 4000), history_capacity=1 << 16, max_bulk=1 << 14)
    g.register(G.DC_TYPES)
    o = oracle.OracleDB(dc=W.dc_tables(4, 40, 4000), hist_cap=1 << 16)
    pool = G.Pool(g, capacity=1000)
    bulk = W.dc_bulk(1500, 4000, 0.0, seed=31)
    pool.add(bulk["ts"][:900], bulk["type"][:900], bulk["params"][:900])
    with pytest.raises(G.GputxError) as e:            # 900 + 200 pending > 1000
        pool.add(bulk["ts"][900:1100], bulk["type"][900:1100], bulk["params"][900:1100])
    assert e.value.status == G.ECAPACITY and pool.pending == 900
    bad = {k: bulk[k][900:1000].copy() for k in ("ts", "type", "params")}
    bad["params"][50, 0] = 4000                       # account out of range
    with pytest.raises(G.GputxError) as e:
        pool.add(bad["ts"], bad["type"], bad["params"])
    assert e.value.status == G.EINVAL and pool.pending == 900
    with pytest.raises(G.GputxError) as e:            # timestamps must keep increasing
        pool.add(bulk["ts"][:10], bulk["type"][:10], bulk["params"][:10])
    assert e.value.status == G.EINVAL
    got = {}
    while pool.pending:
        pool.step()
        ts, st, vals = pool.results()
        got.update({t: (s, v.copy()) for t, s, v in zip(ts.tolist(), st.tolist(), vals)})
    pool.add(bulk["ts"][900:], bulk["type"][900:], bulk["params"][900:])
    while pool.pending:
        pool.step()
        ts, st, vals = pool.results()
        got.update({t: (s, v.copy()) for t, s, v in zip(ts.tolist(), st.tolist(), vals)})
    assert pool.step() == 0
    pool.close()
    ost, oout = o.execute(bulk, R=1)
    assert_matches(got, bulk, ost, oout)
    g.close()
