"""Debit-credit parity: the CUDA engine against the CPU oracle, bit for bit.

All columns are int64, so the tolerance is zero: database state, per
transaction status and output, and the structural statistics d and w0 must be
identical to serial execution in timestamp order (Definition 1).
"""
import numpy as np
import pytest

import oracle
import paper_1103_3105_gb300 as G
import workloads as W
from tests._helpers import gpu_logical_state, oracle_logical_state, state_diff, states_equal

pytestmark = pytest.mark.gpu

STRATS = ["kset", "part", "tpl", "scan"]
MODES = [G.CONFLICT_PAPER, G.CONFLICT_ADD]


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()


def make_pair(B, T, A, cap, max_bulk=1 << 16, **kw):
    tabs = W.dc_tables(B, T, A)
    g = G.Database(dc=(B, T, A), history_capacity=cap, max_bulk=max_bulk, **kw)
    g.register(G.DC_TYPES)
    for t, rows in W.dc_rows(tabs).items():
        g.load(t, rows)
    o = oracle.OracleDB(dc=tabs, hist_cap=cap)
    return g, o


def run_both(g, o, bulk, strategy, mode, **kw):
    b = g.submit_dict(bulk).execute(strategy, conflict_mode=mode, **kw)
    stats = b.sync()
    st, out = b.results()
    b.free()
    ost, oout = o.execute(bulk, R=1)
    return stats, st, out, ost, oout


def assert_same(g, o, st, out, ost, oout):
    assert np.array_equal(st, ost)
    assert np.array_equal(out, oout)
    gs = gpu_logical_state(g, dc=True)
    os_ = oracle_logical_state(o)
    assert states_equal(gs, os_), state_diff(gs, os_)


@pytest.mark.parametrize("strategy", STRATS)
@pytest.mark.parametrize("mode", MODES)
def test_config1_tiny_bank(strategy, mode):
    """4 branches, 40 tellers, 4,000 accounts, 4,096 transactions."""
    g, o = make_pair(4, 40, 4000, 8192)
    bulk = W.dc_bulk(4096, 4000, 0.0, seed=W.seed_for(1))
    stats, st, out, ost, oout = run_both(g, o, bulk, strategy, mode)
    assert_same(g, o, st, out, ost, oout)
    if strategy == "kset":
        ob = oracle.OracleDB(dc=W.dc_tables(4, 40, 4000), hist_cap=8192)
        obj, cls, root = ob.extract(bulk, mode, 3)
        lv = oracle.levels(obj, cls, ob.num_objects())
        d, w0, c = oracle.graph_stats(lv, root)
        assert (stats["depth"], stats["w0"], stats["cross"]) == (d, w0, c)
    g.close()


@pytest.mark.parametrize("n", [1, 2, 31, 257, 8191, 8193, 20000])
@pytest.mark.parametrize("strategy", STRATS)
def test_ragged_sizes(n, strategy):
    """Sizes around warp, CTA, scan-tile (2,048) and sort-tile (8,192) edges."""
    g, o = make_pair(10, 100, 10000, 1 << 16)
    bulk = W.dc_bulk(n, 10000, 0.5, seed=n)
    for mode in MODES:
        stats, st, out, ost, oout = run_both(g, o, bulk, strategy, mode)
        assert_same(g, o, st, out, ost, oout)
        bulk = W.dc_bulk(n, 10000, 0.5, seed=n + 1, ts0=int(bulk["ts"][-1]) + 1)
    g.close()


@pytest.mark.parametrize("theta", [0.0, 0.5, 0.99])
@pytest.mark.parametrize("strategy", STRATS)
def test_skew(theta, strategy):
    """Zipf-skewed accounts (hot rows give deep graphs and long partitions)."""
    g, o = make_pair(100, 1000, 100000, 1 << 18)
    for k in range(2):
        bulk = W.dc_bulk(30000, 100000, theta, seed=int(theta * 100) + k, ts0=k * 30000)
        stats, st, out, ost, oout = run_both(g, o, bulk, strategy, MODES[k])
        assert_same(g, o, st, out, ost, oout)
    g.close()


@pytest.mark.parametrize("B,T,A", [(4, 40, 160), (8, 8, 64), (3, 96, 960), (2, 66, 660)])
def test_part_dense_repeats(B, T, A):
    """PART with few accounts per branch: an account recurs within a few
    transactions of its partition (the early account loads must see the
    writes in between), and many accounts share a slot of the recent-write
    table.  Covers 1, 10 and 32 tellers per branch (shared-memory tellers)
    and 33 (the general partition runner)."""
    g, o = make_pair(B, T, A, 1 << 17)
    ts0 = 0
    for k, theta in enumerate([0.0, 0.9]):
        bulk = W.dc_bulk(20_000 + 13 * k, A, theta, seed=300 + k, ts0=ts0)
        ts0 += len(bulk["ts"])
        stats, st, out, ost, oout = run_both(g, o, bulk, "part", 0)
        assert stats["strategy"] == G.PART
        assert_same(g, o, st, out, ost, oout)
    g.close()


def test_strategies_agree_across_a_sequence():
    """Bulks run back to back with different strategies equal one serial run."""
    g, o = make_pair(20, 200, 20000, 1 << 17)
    ts0 = 0
    for k, (s, m) in enumerate([("kset", 0), ("tpl", 1), ("part", 0), ("kset", 1), ("tpl", 0),
                                ("auto", 0), ("scan", 0), ("auto", 1), ("scan", 1)]):
        bulk = W.dc_bulk(5000 + 37 * k, 20000, 0.7, seed=50 + k, ts0=ts0)
        ts0 += len(bulk["ts"])
        stats, st, out, ost, oout = run_both(g, o, bulk, s, m)
        assert np.array_equal(st, ost) and np.array_equal(out, oout), (s, m)
    gs, os_ = gpu_logical_state(g, dc=True), oracle_logical_state(o)
    assert states_equal(gs, os_), state_diff(gs, os_)
    g.close()


def test_empty_bulk():
    g, o = make_pair(4, 40, 4000, 1024)
    for s in STRATS + ["auto", "part_relaxed", "tpl_relaxed"]:
        b = g.submit(np.zeros(0, np.int64), np.zeros(0, np.int32), np.zeros((0, 2), np.int64))
        b.execute(s)
        st, out = b.results()
        assert st.shape == (0,) and out.shape == (0, 1)
        b.free()
    assert len(g.read(G.TBL_DC_HISTORY)) == 0
    g.close()


@pytest.mark.parametrize("flaw", ["type", "account", "ts"])
def test_invalid_bulk_is_rejected_and_leaves_state(flaw):
    g, o = make_pair(4, 40, 4000, 8192)
    good = W.dc_bulk(100, 4000, 0.0, seed=3)
    run_both(g, o, good, "kset", 0)
    bad = W.dc_bulk(100, 4000, 0.0, seed=4, ts0=100)
    if flaw == "type":
        bad["type"][50] = G.T_SUB_GET_SUBSCRIBER   # not registered
    elif flaw == "account":
        bad["params"][70, 0] = 4000
    else:
        bad["ts"][10] = bad["ts"][9]
    before = gpu_logical_state(g, dc=True)
    for s in STRATS:
        b = g.submit_dict(bad).execute(s)
        with pytest.raises(G.GputxError) as e:
            b.sync()
        assert e.value.status == G.EINVAL
        b.free()
    after = gpu_logical_state(g, dc=True)
    assert states_equal(before, after), state_diff(before, after)
    g.close()


def test_device_resident_inputs():
    torch = pytest.importorskip("torch")
    g, o = make_pair(10, 100, 10000, 1 << 16)
    bulk = W.dc_bulk(10000, 10000, 0.3, seed=9)
    dev = {k: torch.from_numpy(bulk[k]).cuda() for k in ("ts", "type", "params")}
    b = g.submit(dev["ts"], dev["type"], dev["params"]).execute("kset")
    st, out = b.results()
    b.free()
    ost, oout = o.execute(bulk, 1)
    assert np.array_equal(st, ost) and np.array_equal(out, oout)
    g.close()


def test_execute_twice_is_refused():
    g, o = make_pair(4, 40, 4000, 8192)
    b = g.submit_dict(W.dc_bulk(10, 4000, 0.0, seed=1)).execute("kset")
    with pytest.raises(G.GputxError) as e:
        b.execute("kset")
    assert e.value.status == G.ESTATE
    b.sync()
    b.free()
    g.close()


@pytest.mark.parametrize("strategy,launch,mode", [("kset", 1, 0), ("tpl", 0, 0), ("tpl", 0, 1)])
def test_bounded_wait_reports_timeout(strategy, launch, mode):
    """A 1 ns wait limit makes the per-level waits of a 1,000-deep persistent
    K-SET launch (or TPL's lock waits) run out: the engine must report
    ETIMEOUT instead of hanging, and stay usable.  TPL under R/W locks the 4
    branches (chains of about 1,000: the CTA-group kernel); under ADD it
    locks the 4,000 accounts (chains of a few: the warp-group kernel)."""
    g = G.Database(dc=(4, 40, 4000), history_capacity=1 << 16, max_bulk=1 << 14, spin_limit_ns=1)
    g.register(G.DC_TYPES)
    bulk = W.dc_bulk(4096, 4000, 0.0, seed=2)
    if mode:
        # every account twice in a row, 2,048 apart: each second visit waits
        acct = np.arange(2048, dtype=np.int64)
        bulk["params"][:, 0] = np.concatenate([acct, acct])
    b = g.submit_dict(bulk).execute(strategy, conflict_mode=mode, kset_launch=launch)
    with pytest.raises(G.GputxError) as e:
        b.sync()
    assert e.value.status == G.ETIMEOUT
    b.free()
    g.close()
    # the context still works
    g2, o = make_pair(4, 40, 4000, 8192)
    stats, st, out, ost, oout = run_both(g2, o, W.dc_bulk(500, 4000, 0.0, seed=3), "kset", 0)
    assert np.array_equal(out, oout)
    g2.close()


@pytest.mark.parametrize("strategy,mode", [("kset", 0), ("kset", 1), ("tpl", 0), ("tpl", 1), ("part", 0),
                                           ("scan", 0), ("auto", 0)])
def test_full_size_config2(strategy, mode):
    """The benchmark's workload: 1,000 branches, 10,000 tellers, 10,000,000
    accounts, a bulk of 2^22 transactions, in the benchmark's launch shape.
    The oracle runs the whole bulk serially, so every output is compared."""
    A = 10_000_000
    g, o = make_pair(1000, 10000, A, 1 << 22, max_bulk=1 << 22)
    bulk = W.dc_bulk(1 << 22, A, 0.0, seed=W.seed_for(2, 22))
    stats, st, out, ost, oout = run_both(g, o, bulk, strategy, mode)
    if strategy == "auto":
        assert stats["strategy"] == G.SCAN   # a debit-credit-only database
    assert np.array_equal(st, ost)
    assert np.array_equal(out, oout)
    assert np.array_equal(g.read(G.TBL_DC_ACCOUNT)[:, 0], o["acc_bal"])
    assert np.array_equal(g.read(G.TBL_DC_BRANCH)[:, 0], o["br_bal"])
    assert np.array_equal(g.read(G.TBL_DC_TELLER)[:, 0], o["tel_bal"])
    h = g.read(G.TBL_DC_HISTORY)
    assert np.array_equal(h[np.argsort(h[:, 0])], o.history())
    g.close()


@pytest.mark.parametrize("lg", [20, 22])
@pytest.mark.parametrize("strategy,mode", [("kset", 0), ("kset", 1), ("part", 0), ("tpl", 0), ("tpl", 1)])
def test_hot_accounts_at_sweep_sizes(lg, strategy, mode):
    """Zipf 0.99 accounts at the sweep's 2^20 and 2^22 transactions over the
    benchmark's tables: hot accounts make graphs thousands of levels deep,
    a hot branch partition and long lock chains.  Every output and the
    whole state are compared."""
    A = 10_000_000
    g, o = make_pair(1000, 10000, A, 1 << lg, max_bulk=1 << lg)
    bulk = W.dc_bulk(1 << lg, A, 0.99, seed=W.seed_for(2, 199 + lg))
    stats, st, out, ost, oout = run_both(g, o, bulk, strategy, mode)
    assert np.array_equal(st, ost)
    assert np.array_equal(out, oout)
    if strategy == "kset":
        ob = oracle.OracleDB(dc=W.dc_tables(1000, 10000, A), hist_cap=1)
        obj, cls, root = ob.extract(bulk, mode, 3)
        lv = oracle.levels(obj, cls, ob.num_objects())
        assert (stats["depth"], stats["w0"]) == (int(lv.max()), int((lv == 0).sum()))
    assert np.array_equal(g.read(G.TBL_DC_ACCOUNT)[:, 0], o["acc_bal"])
    assert np.array_equal(g.read(G.TBL_DC_BRANCH)[:, 0], o["br_bal"])
    assert np.array_equal(g.read(G.TBL_DC_TELLER)[:, 0], o["tel_bal"])
    h = g.read(G.TBL_DC_HISTORY)
    assert np.array_equal(h[np.argsort(h[:, 0])], o.history())
    g.close()


@pytest.mark.parametrize("hot_ops", [128, 129])
@pytest.mark.parametrize("mode", MODES)
def test_tpl_executor_pick_at_the_hot_chain(hot_ops, mode):
    """Debit-credit TPL runs one of two executors: lock groups over a warp, or
    over the whole CTA once some lock's chain reaches n/512 operations (128 of
    2^16).  The lock is the branch under R/W and the account under ADD.  Here
    2,048 branches of 20 accounts keep every other chain short (about 32
    operations per branch), and one account -- alone in its branch -- takes
    128 operations (warp groups) or 129 (CTA groups), spread over the bulk
    with a run of 20 consecutive ones in one chunk.  Both executors must give
    the serial result."""
    n = 1 << 16
    B, T, A = 2048, 8192, 40960
    g, o = make_pair(B, T, A, n, max_bulk=n)
    bulk = W.dc_bulk(n, A, 0.0, seed=W.seed_for(1, hot_ops))
    rng = np.random.default_rng(hot_ops)
    hot = 777 * 20 + 3                       # an account of branch 777
    acct = bulk["params"][:, 0]
    acct[acct // 20 == 777] += 20            # the rest of branch 777 moves to branch 778
    idx = np.concatenate([np.arange(1000, 1020), rng.choice(np.arange(2000, n), hot_ops - 20, replace=False)])
    acct[idx] = hot
    assert int((acct // 20 == 777).sum()) == hot_ops and int((acct == hot).sum()) == hot_ops
    assert np.bincount(acct // 20).max() == hot_ops   # no other branch as long
    stats, st, out, ost, oout = run_both(g, o, bulk, "tpl", mode)
    assert_same(g, o, st, out, ost, oout)
    g.close()


@pytest.mark.parametrize("strategy,mode", [("kset", 0), ("kset", 1), ("tpl", 0), ("part", 0), ("scan", 0)])
def test_back_to_back_bulks_without_sync(strategy, mode):
    """Bulks executed one after another without waiting: each bulk's analysis
    overlaps the previous bulk's execution on the device, yet they apply in
    call order."""
    g, o = make_pair(20, 200, 20000, 1 << 18)
    bulks, handles, ts0 = [], [], 0
    for k in range(6):
        bulk = W.dc_bulk(7000 + 911 * k, 20000, 0.8, seed=300 + k, ts0=ts0)
        ts0 += len(bulk["ts"])
        bulks.append(bulk)
        handles.append(g.submit_dict(bulk).execute(strategy, conflict_mode=mode))
    for bulk, h in zip(bulks, handles):
        st, out = h.results()
        h.free()
        ost, oout = o.execute(bulk, R=1)
        assert np.array_equal(st, ost) and np.array_equal(out, oout)
    gs, os_ = gpu_logical_state(g, dc=True), oracle_logical_state(o)
    assert states_equal(gs, os_), state_diff(gs, os_)
    g.close()


def test_scan_full_size_hot_accounts():
    """SCAN at the benchmark's size with Zipf 0.99 accounts: a dependency
    graph over 200,000 levels deep, executed as prefix sums."""
    A = 10_000_000
    g, o = make_pair(1000, 10000, A, 1 << 22, max_bulk=1 << 22)
    bulk = W.dc_bulk(1 << 22, A, 0.99, seed=W.seed_for(2, 99))
    stats, st, out, ost, oout = run_both(g, o, bulk, "scan", 0)
    assert np.array_equal(st, ost) and np.array_equal(out, oout)
    assert np.array_equal(g.read(G.TBL_DC_ACCOUNT)[:, 0], o["acc_bal"])
    assert np.array_equal(g.read(G.TBL_DC_BRANCH)[:, 0], o["br_bal"])
    assert np.array_equal(g.read(G.TBL_DC_TELLER)[:, 0], o["tel_bal"])
    h = g.read(G.TBL_DC_HISTORY)
    assert np.array_equal(h[np.argsort(h[:, 0])], o.history())
    g.close()


def test_scan_history_full_writes_nothing():
    """SCAN runs a bulk whole or not at all: history rows that do not fit
    fail the bulk with ECAPACITY and leave the database as it was."""
    g, o = make_pair(4, 40, 4000, 150)
    run_both(g, o, W.dc_bulk(100, 4000, 0.0, seed=5), "scan", 0)
    before = gpu_logical_state(g, dc=True)
    b = g.submit_dict(W.dc_bulk(100, 4000, 0.0, seed=6, ts0=100)).execute("scan")
    with pytest.raises(G.GputxError) as e:
        b.sync()
    assert e.value.status == G.ECAPACITY
    b.free()
    assert states_equal(before, gpu_logical_state(g, dc=True))
    g.close()


@pytest.mark.parametrize("strategy", ["kset", "part", "tpl", "part_relaxed", "tpl_relaxed"])
@pytest.mark.parametrize("mode", [G.CONFLICT_PAPER, G.CONFLICT_ADD])
def test_history_full_is_an_error(strategy, mode):
    """A bulk whose history rows overflow the table fails with ECAPACITY on
    every executor (the debit-credit level runners, the TPL kernel for
    debit-credit bulks, PART); no wait hangs on a transaction that was not
    executed."""
    g = G.Database(dc=(4, 40, 4000), history_capacity=150, max_bulk=1 << 10)
    g.register(G.DC_TYPES)
    b = g.submit_dict(W.dc_bulk(400, 4000, 0.5, seed=8)).execute(strategy, conflict_mode=mode)
    with pytest.raises(G.GputxError) as e:
        b.sync()
    assert e.value.status == G.ECAPACITY
    b.free()
    g.close()


def test_scan_needs_debit_credit_only():
    g = G.Database(dc=(4, 40, 4000), sub=100, history_capacity=1024, sub_child_capacity=1024, max_bulk=1024)
    g.register(G.DC_TYPES + G.SUB_TYPES)
    b = g.submit_dict(W.dc_bulk(10, 4000, 0.0, seed=1))
    with pytest.raises(G.GputxError) as e:
        b.execute("scan")
    assert e.value.status == G.EINVAL
    b.free()
    g.close()


def test_timing_stats_for_every_strategy():
    """Phase timing on every strategy, bulk after bulk: phases a strategy does
    not have report 0 and leave no error behind for the next bulk."""
    g, o = make_pair(10, 100, 10000, 1 << 16)
    ts0 = 0
    for s in ("kset", "part", "tpl", "auto", "scan", "part_relaxed", "tpl_relaxed") * 2:
        bulk = W.dc_bulk(2000, 10000, 0.5, seed=ts0 + 7, ts0=ts0)
        ts0 += 2000
        b = g.submit_dict(bulk).execute(s, timing=True)
        stats = b.sync()
        b.free()
        assert stats["ms_total"] > 0 and stats["ms_execute"] >= 0 and stats["ms_sort"] >= 0, s
    g.close()


def test_level_chain_probe():
    """The bare level-chain skeleton: positive, more traffic per level never
    faster than less, and below the full runner's time per level."""
    floor_min = G.gputx_probe_level_chain(2000, 16, 64, 1, 1)
    floor_dc = G.gputx_probe_level_chain(2000, 16, 64, 3, 10)
    floor_split = G.gputx_probe_level_chain(2000, 16, 64, 3, 3, 7)
    floor_rmw = G.gputx_probe_level_chain(2000, 16, 64, 0, 3, 7, rmw=1)
    floor_rand = G.gputx_probe_level_chain(2000, 16, 64, 0, 1, 9, rmw=2)
    for f in (floor_min, floor_dc, floor_split, floor_rmw, floor_rand):
        assert 0 < f < 50_000
    assert floor_dc > 0.8 * floor_min


def test_atomics_probe():
    """L2 atomic throughput: positive and finite for a hot table (1,000 cells)
    and a large one, reductions and fetch-and-adds; spreading the additions
    over many cells is never slower than piling them on one."""
    rates = {}
    for cells in (1, 1000, 10_000_000):
        for fetch in (0, 1):
            rates[(cells, fetch)] = G.gputx_probe_atomics(cells, fetch)
            assert 0 < rates[(cells, fetch)] < 1e4, (cells, fetch)
    assert rates[(1000, 0)] > rates[(1, 0)]


@pytest.mark.parametrize("strategy", STRATS + ["auto", "part_relaxed", "tpl_relaxed"])
def test_bulk_of_exactly_max_bulk(strategy):
    """A bulk filling max_bulk exactly (every per-bulk scratch array at its
    capacity), twice in a row on one database."""
    g, o = make_pair(10, 100, 10000, 1 << 17, max_bulk=1 << 15)
    for k in range(2):
        bulk = W.dc_bulk(1 << 15, 10000, 0.3, seed=400 + k, ts0=k << 15)
        b = g.submit_dict(bulk).execute(strategy)
        st, out = b.results()
        order = b.order().astype(np.int64)
        b.free()
        ost, oout = o.execute(bulk, R=1, order=order)
        assert np.array_equal(st, ost) and np.array_equal(out, oout)
    gs, os_ = gpu_logical_state(g, dc=True), oracle_logical_state(o)
    assert states_equal(gs, os_), state_diff(gs, os_)
    with pytest.raises(G.GputxError) as e:   # one more than max_bulk
        g.submit_dict(W.dc_bulk((1 << 15) + 1, 10000, 0.0, seed=9))
    assert e.value.status == G.EINVAL
    g.close()


@pytest.mark.parametrize("mode", MODES)
def test_narrow_run_cut_into_segments(mode):
    """A run of narrow levels whose width falls from a cluster's class to one
    CTA's for hundreds of levels (127 branches with 100 transactions each,
    one branch with 400): the run executes as two launches of different
    shapes, and every result still matches serial execution."""
    B, A = 128, 128 * 100
    g, o = make_pair(B, B * 10, A, 1 << 16)
    rng = np.random.default_rng(W.seed_for(2, 7))
    per = A // B
    branch = np.concatenate([np.repeat(np.arange(B - 1), 100), np.full(400, B - 1)])
    rng.shuffle(branch)
    n = len(branch)
    acct = branch * per + rng.integers(0, per, size=n)
    bulk = {"ts": np.arange(n, dtype=np.int64), "type": np.zeros(n, np.int32),
            "params": np.stack([acct, rng.integers(-99999, 100000, size=n)], axis=1).astype(np.int64), "P": 2}
    stats, st, out, ost, oout = run_both(g, o, bulk, "kset", mode)
    if mode == G.CONFLICT_PAPER:
        assert stats["depth"] == 399
    assert_same(g, o, st, out, ost, oout)
    g.close()
