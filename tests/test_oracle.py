"""Pins for the CPU oracle against what the paper and mathematics fix.

Each test names the passage it pins.  None of them re-derives the oracle's
formula: they use closed forms, the paper's Figure 1 example, Properties 1-2,
an independent algorithm (Appendix B graph + topological sort) or brute force
over serial orders.
"""
import os

import numpy as np
import pytest

import oracle
import workloads as W
from tests._helpers import (check_properties, conflict_pairs, linear_extensions,
                            oracle_logical_state, state_diff, states_equal)

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _cls_code(c):
    return {"R": oracle.CLS_R, "W": oracle.CLS_W, "A": oracle.CLS_A}[c]


# ---------------------------------------------------------------------------
# Figure 1 (Sections 4.1-4.2)
# ---------------------------------------------------------------------------
def _fig1():
    rows, edges = [], []
    for line in open(os.path.join(GOLDEN, "fig1_group_a.txt")):
        line = line.split("#")[0].split()
        if not line:
            continue
        if line[0] == "E":
            edges.append((int(line[1]), int(line[2])))
        else:
            rows.append((int(line[0]), _cls_code(line[1]), int(line[2]), int(line[3])))
    return rows, edges


def test_fig1_ranks_levels_edges():
    rows, edges = _fig1()
    n = len(rows)
    obj = np.zeros((n, 1), dtype=np.int64)
    cls = np.array([[r[1]] for r in rows], dtype=np.int32)
    want_rank = [r[2] for r in rows]
    want_level = [r[3] for r in rows]
    lv1, rk = oracle.onepass_levels(obj, cls)
    assert rk[:, 0].tolist() == want_rank
    assert lv1.tolist() == want_level
    assert oracle.levels(obj, cls, 1).tolist() == want_level
    e = oracle.appb_edges(obj, cls, 1)
    assert sorted(map(tuple, e.tolist())) == sorted(edges)
    assert oracle.topo_levels(n, e).tolist() == want_level
    # T1 and T4 conflict but share no edge (condition (c))
    assert (0, 3) not in set(map(tuple, e.tolist()))


def test_onepass_is_not_exact_for_multi_item_transactions():
    """T1 W{a}, T2 W{a,b}, T3 W{b}: the per-group ranks give T3 rank 1 on b,
    yet T3 conflicts with T2 (depth 1), so its depth is 2 (Section 4.1's
    longest path; Property 1 would fail with depth 1)."""
    obj = np.array([[0, -1], [0, 1], [1, -1]], dtype=np.int64)
    cls = np.full((3, 2), oracle.CLS_W, dtype=np.int32)
    one, _ = oracle.onepass_levels(obj, cls)
    assert one.tolist() == [0, 1, 1]
    assert check_properties(one, obj, cls)           # one-pass violates P1
    exact = oracle.levels(obj, cls, 2)
    assert exact.tolist() == [0, 1, 2]
    assert check_properties(exact, obj, cls) == []
    assert oracle.topo_levels(3, oracle.appb_edges(obj, cls, 2)).tolist() == [0, 1, 2]


# ---------------------------------------------------------------------------
# debit-credit closed forms (Definition 1)
# ---------------------------------------------------------------------------
def _dc_db(b=4, t=40, a=4000, cap=1 << 16):
    return oracle.OracleDB(dc=W.dc_tables(b, t, a), hist_cap=cap)


@pytest.mark.parametrize("theta", [0.0, 0.9])
def test_dc_closed_forms(theta):
    A, T, B, n = 4000, 40, 4, 4096
    db = _dc_db(B, T, A)
    bulk = W.dc_bulk(n, A, theta, seed=W.seed_for(1, 1))
    st, out = db.execute(bulk, R=1)
    acct, delta = bulk["params"][:, 0], bulk["params"][:, 1]
    teller, branch = acct // (A // T), acct // (A // B)
    assert (st == 0).all()
    # final balance of every row = sum of the deltas applied to it
    assert np.array_equal(db["acc_bal"], np.bincount(acct, weights=None, minlength=A) * 0
                          + np.array([delta[acct == i].sum() for i in range(A)]))
    assert np.array_equal(db["tel_bal"], np.array([delta[teller == i].sum() for i in range(T)]))
    assert np.array_equal(db["br_bal"], np.array([delta[branch == i].sum() for i in range(B)]))
    # output of txn t = inclusive prefix sum of its account's deltas up to t
    order = np.lexsort((np.arange(n), acct))
    cs = np.zeros(n, dtype=np.int64)
    run = {}
    for i in order:
        run[acct[i]] = run.get(acct[i], 0) + delta[i]
        cs[i] = run[acct[i]]
    assert np.array_equal(out[:, 0], cs)
    # conservation across the four tables
    s = delta.sum()
    assert db["acc_bal"].sum() == s == db["tel_bal"].sum() == db["br_bal"].sum()
    h = db.history()
    assert len(h) == n and h[:, 4].sum() == s
    assert np.array_equal(h[:, 0], bulk["ts"])
    assert np.array_equal(h[:, 1], acct) and np.array_equal(h[:, 2], teller)
    assert np.array_equal(h[:, 3], branch) and np.array_equal(h[:, 4], delta)


def test_dc_two_bulks_accumulate():
    A = 4000
    db = _dc_db()
    b1 = W.dc_bulk(1000, A, 0.0, seed=1)
    b2 = W.dc_bulk(1000, A, 0.0, seed=2, ts0=1000)
    db.execute(b1, 1)
    db.execute(b2, 1)
    want = np.zeros(A, dtype=np.int64)
    np.add.at(want, b1["params"][:, 0], b1["params"][:, 1])
    np.add.at(want, b2["params"][:, 0], b2["params"][:, 1])
    assert np.array_equal(db["acc_bal"], want)
    assert db.hist_n == 2000


# ---------------------------------------------------------------------------
# depth (Sections 4.1, 4.2, 5.1, Appendix B)
# ---------------------------------------------------------------------------
def _cumcount(keys):
    """0-based count of earlier equal keys, per position."""
    out = np.zeros(len(keys), dtype=np.int64)
    seen = {}
    for i, k in enumerate(keys.tolist()):
        out[i] = seen.get(k, 0)
        seen[k] = out[i] + 1
    return out


@pytest.mark.parametrize("theta", [0.0, 0.99])
def test_dc_depth_is_branch_position(theta):
    """Section 5.1: with every transaction writing its branch balance, the
    T-dependency graph is one path per branch, so a transaction's depth is
    the number of earlier transactions on its branch."""
    A, n = 4000, 4096
    db = _dc_db()
    bulk = W.dc_bulk(n, A, theta, seed=7)
    obj, cls, root = db.extract(bulk, oracle.MODE_PAPER, 3)
    lv = oracle.levels(obj, cls, db.num_objects())
    assert np.array_equal(lv, _cumcount(bulk["params"][:, 0] // 1000))
    one, _ = oracle.onepass_levels(obj, cls)
    assert np.array_equal(one, lv)
    d, w0, c = oracle.graph_stats(lv, root)
    assert w0 == len(np.unique(bulk["params"][:, 0] // 1000)) and c == 0


def test_dc_add_mode_depth_is_account_position():
    """With teller and branch increments as blind commutative additions, only
    the account item orders transactions: depth = earlier txns on the same
    account."""
    A, n = 4000, 4096
    db = _dc_db()
    bulk = W.dc_bulk(n, A, 0.5, seed=8)
    obj, cls, _ = db.extract(bulk, oracle.MODE_ADD, 3)
    lv = oracle.levels(obj, cls, db.num_objects())
    assert np.array_equal(lv, _cumcount(bulk["params"][:, 0]))


def _mixed_small_db():
    sub = W.sub_tables(6, seed=3)
    oe = W.oe_tables(2, n_items=40, seed=4)
    return dict(dc=W.dc_tables(2, 4, 8), sub=sub, oe=oe, hist_cap=4096, ord_cap=4096,
                ol_cap=65536, oid_cap=4096)


def _mixed_bulk(n, seed, db_kwargs):
    """Interleave small debit-credit, subscriber and order-entry bulks."""
    rng = np.random.default_rng(seed)
    parts = [W.dc_bulk(n, 8, 0.0, seed=seed),
             W.sub_bulk(n, 6, 0.0, seed=seed + 1),
             W.oe_bulk(n, 2, n_items=40, item_theta=0.5, remote_frac=0.3,
                       invalid_frac=0.1, seed=seed + 2)]
    P = max(p["P"] for p in parts)
    pick = rng.integers(0, 3, size=n)
    params = np.zeros((n, P), dtype=np.int64)
    types = np.zeros(n, dtype=np.int32)
    for k, p in enumerate(parts):
        m = pick == k
        params[m, : p["P"]] = p["params"][m]
        types[m] = p["type"][m]
    return {"ts": np.arange(n, dtype=np.int64), "type": types, "params": params, "P": P}


@pytest.mark.parametrize("mode", [oracle.MODE_PAPER, oracle.MODE_ADD])
@pytest.mark.parametrize("seed", [1, 2, 3])
def test_levels_match_appendix_b_and_properties(mode, seed):
    """Exact depth equals the topological-sort depth of the Appendix B graph
    (an independent construction), level 0 is exactly the graph's sources,
    and Properties 1-2 hold."""
    kw = _mixed_small_db()
    db = oracle.OracleDB(**kw)
    bulk = _mixed_bulk(300, seed, kw)
    obj, cls, _ = db.extract(bulk, mode, oracle.MAX_OPS)
    lv = oracle.levels(obj, cls, db.num_objects())
    e = oracle.appb_edges(obj, cls, db.num_objects())
    assert np.array_equal(oracle.topo_levels(len(lv), e), lv)
    has_pred = np.zeros(len(lv), dtype=bool)
    has_pred[e[:, 1]] = True
    assert np.array_equal(lv == 0, ~has_pred)
    assert check_properties(lv, obj, cls) == []
    # every App B edge joins conflicting, timestamp-ordered transactions
    pairs = conflict_pairs(obj, cls)
    assert all((int(a), int(b)) in pairs and a < b for a, b in e)


def test_property_checker_catches_planted_mistake():
    """A level array with one transaction moved into its predecessor's level
    must fail Property 1 (guards the checker used above)."""
    A, n = 4000, 512
    db = _dc_db()
    bulk = W.dc_bulk(n, A, 0.0, seed=5)
    obj, cls, _ = db.extract(bulk, oracle.MODE_PAPER, 3)
    lv = oracle.levels(obj, cls, db.num_objects())
    t = int(np.flatnonzero(lv == 1)[0])
    bad = lv.copy()
    bad[t] = 0
    assert check_properties(bad, obj, cls) != []


# ---------------------------------------------------------------------------
# brute force: every serial order consistent with the graph gives one state
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("mode", [oracle.MODE_PAPER, oracle.MODE_ADD])
@pytest.mark.parametrize("seed", range(6))
def test_brute_force_linear_extensions(mode, seed):
    """Definition 1 fixes one result; any order that keeps every conflicting
    pair in timestamp order must reach it.  This validates the declared
    access sets of all eleven procedures on tiny hot bulks."""
    kw = _mixed_small_db()
    bulk = _mixed_bulk(8, 100 + seed, kw)
    ref_db = oracle.OracleDB(**kw)
    obj, cls, _ = ref_db.extract(bulk, mode, oracle.MAX_OPS)
    st0, out0 = ref_db.execute(bulk, R=8)
    s0 = oracle_logical_state(ref_db)
    pairs = conflict_pairs(obj, cls)
    orders = linear_extensions(len(bulk["ts"]), pairs, limit=300, seed=seed)
    assert len(orders) >= 1
    for order in orders:
        db = oracle.OracleDB(**kw)
        st, out = db.execute(bulk, R=8, order=order)
        s = oracle_logical_state(db)
        assert states_equal(s0, s), (order, state_diff(s0, s))
        assert np.array_equal(st, st0) and np.array_equal(out, out0), order


def test_brute_force_detects_a_missing_conflict():
    """Guard for the brute-force test: dropping the account operation from
    debit-credit's access set (in ADD mode only the account orders
    transactions) lets reorderings change the outputs."""
    kw = _mixed_small_db()
    db0 = oracle.OracleDB(**kw)
    bulk = W.dc_bulk(6, 8, 0.0, seed=11)
    bulk["params"][:, 0] = [1, 1, 2, 1, 2, 1]
    obj, cls, _ = db0.extract(bulk, oracle.MODE_ADD, 3)
    obj[:, 0] = -1                                   # planted mistake
    st0, out0 = db0.execute(bulk, R=1)
    diff = False
    for order in linear_extensions(6, conflict_pairs(obj, cls), limit=50):
        db = oracle.OracleDB(**kw)
        _, out = db.execute(bulk, R=1, order=order)
        diff |= not np.array_equal(out, out0)
    assert diff


# ---------------------------------------------------------------------------
# subscriber and order-entry invariants
# ---------------------------------------------------------------------------
def test_subscriber_invariants():
    n_sub, n = 64, 4000
    init = W.sub_tables(n_sub, seed=9)
    db = oracle.OracleDB(sub=init)
    bulk = W.sub_bulk(n, n_sub, 0.0, seed=10)
    st, out = db.execute(bulk, R=8)
    ty, p = bulk["type"], bulk["params"]
    ins_ok = ((ty == W.SUB_INSERT_CF) & (st == 0)).sum()
    del_ok = ((ty == W.SUB_DELETE_CF) & (st == 0)).sum()
    # row counts = initial + committed inserts - committed deletes
    assert db["cf_present"].sum() == init["cf_present"].sum() + ins_ok - del_ok
    # only inserts/deletes change presence; child rows need their facility
    assert not (db["cf_present"].astype(bool) & ~db["sf_present"].astype(bool)[:, :, None]).any()
    # aborted writers leave no trace: statuses are 0/1/2 only where allowed
    assert set(np.unique(st[ty == W.SUB_GET_SUBSCRIBER])) <= {0}
    assert set(np.unique(st[ty == W.SUB_UPDATE_LOCATION])) <= {0}
    assert set(np.unique(st[ty == W.SUB_INSERT_CF])) <= {0, 1, 2}
    # read outputs equal direct lookups for subscribers no earlier writer touched
    writer = np.isin(ty, [W.SUB_UPDATE_LOCATION, W.SUB_UPDATE_FACILITY,
                          W.SUB_INSERT_CF, W.SUB_DELETE_CF])
    first_write = {}
    for i in np.flatnonzero(writer):
        first_write.setdefault(int(p[i, 0]), int(i))
    for i in np.flatnonzero(ty == W.SUB_GET_SUBSCRIBER)[:200]:
        s = int(p[i, 0])
        if first_write.get(s, n) < i:
            continue
        row = init["sub"][s].astype(np.int64) & 0xFFFFFFFF
        want = row[0::2] | (row[1::2] << 32)
        assert np.array_equal(out[i].view(np.uint64), want.astype(np.uint64))
    for i in np.flatnonzero(ty == W.SUB_GET_ACCESS)[:200]:
        s, a = int(p[i, 0]), int(p[i, 1]) - 1
        if first_write.get(s, n) < i:
            continue
        assert st[i] == (0 if init["ai_present"][s, a] else 1)
    # update-location returns the previous location: chain per subscriber
    last = init["sub"][:, 15].astype(np.int64).copy()
    for i in np.flatnonzero(ty == W.SUB_UPDATE_LOCATION):
        s = int(p[i, 0])
        assert out[i, 0] == last[s]
        last[s] = p[i, 1]
    assert np.array_equal(db["sub"][:, 15].astype(np.int64), last)


def test_order_entry_invariants():
    n_wh, n_items, n = 2, 200, 3000
    init = W.oe_tables(n_wh, n_items=n_items, seed=12)
    db = oracle.OracleDB(oe=init, ord_cap=n, ol_cap=n * 15, oid_cap=n + 2)
    bulk = W.oe_bulk(n, n_wh, n_items=n_items, remote_frac=0.1, invalid_frac=0.05, seed=13)
    st, out = db.execute(bulk, R=4)
    ty, p = bulk["type"], bulk["params"]
    pay = ty == W.OE_PAYMENT
    amt = p[pay, 3].sum()
    # payment conservation
    assert db["w_ytd"].sum() == amt == db["d_ytd"].sum() == db["c_ytd"].sum()
    assert db["c_balance"].sum() == -amt
    assert db["c_payment_cnt"].sum() == pay.sum()
    # a new-order aborts exactly when one of its items is not in the catalogue
    no = np.flatnonzero(ty == W.OE_NEW_ORDER)
    bad = np.array([((p[i, 4:4 + p[i, 3]] & 0xFFFFFF) >= n_items).any() for i in no])
    assert np.array_equal(st[no] != 0, bad)
    ok = no[~bad]
    # order and order-line rows = committed new-orders and their lines
    assert len(db.orders()) == len(ok)
    assert len(db.order_lines()) == p[ok, 3].sum()
    # o_ids are dense per district, starting at 1
    assert (db["d_next_o_id"] - 1).sum() == len(ok)
    dist = p[ok, 0] * 10 + p[ok, 1]
    assert np.array_equal(np.bincount(dist, minlength=n_wh * 10), db["d_next_o_id"] - 1)
    # stock ytd grows by the committed quantities
    qty = sum(int(((p[i, 4:4 + p[i, 3]] >> 40) & 0xFF).sum()) for i in ok)
    assert db["s_ytd"].sum() == qty
    # order-status sees the customer's latest committed order
    last = {}
    for i in range(n):
        key = (int(p[i, 0]), int(p[i, 1]), int(p[i, 2]))
        if ty[i] == W.OE_NEW_ORDER and st[i] == 0:
            last[key] = (int(out[i, 0]), int(p[i, 3]))
        if ty[i] == W.OE_ORDER_STATUS:
            if key in last:
                assert st[i] == 0 and out[i, 1] == last[key][0] and out[i, 2] == last[key][1]
            else:
                assert st[i] == 1 and out[i, 1] == 0


def test_extract_rejects_unknown_type():
    db = _dc_db()
    bulk = W.dc_bulk(4, 4000, 0.0, seed=1)
    bulk["type"][2] = 99
    with pytest.raises(ValueError):
        db.extract(bulk, oracle.MODE_PAPER, 3)
    with pytest.raises(ValueError):
        db.execute(bulk, 1)


# ---------------------------------------------------------------------------
# Replay in a given serial order (Appendix G: serializability)
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("seed", [3, 4])
def test_dc_replay_in_a_given_order(seed):
    """Executed in a permutation of the bulk, a debit-credit transaction's
    output is its account's deltas summed over the transactions at or before
    it in that order, and every final balance is the order-free sum."""
    A, T, B, n = 400, 40, 4, 2000
    db = _dc_db(B, T, A)
    bulk = W.dc_bulk(n, A, 0.9, seed=W.seed_for(1, seed))
    order = np.random.default_rng(seed).permutation(n)
    st, out = db.execute(bulk, R=1, order=order)
    acct, delta = bulk["params"][:, 0], bulk["params"][:, 1]
    assert (st == 0).all()
    run, want = {}, np.zeros(n, dtype=np.int64)
    for t in order:
        run[acct[t]] = run.get(acct[t], 0) + delta[t]
        want[t] = run[acct[t]]
    assert np.array_equal(out[:, 0], want)
    assert np.array_equal(db["acc_bal"], np.array([delta[acct == i].sum() for i in range(A)]))
    assert np.array_equal(db["br_bal"], np.array([delta[acct // (A // B) == i].sum() for i in range(B)]))


# ---------------------------------------------------------------------------
# Algorithm 1's structural parameters (Appendix D)
# ---------------------------------------------------------------------------
def test_graph_stats_by_hand():
    """d, w0 and c of a hand-built example: c counts a transaction whose root
    keys fall in two partitions of part_size consecutive keys, and nothing
    else (one partition, one key, no operation)."""
    level = np.array([0, 1, 0, 2, 1])
    root = np.array([[0, 1], [1, 2], [5, -1], [-1, -1], [6, 7]])
    assert oracle.graph_stats(level, root, part_size=2) == (2, 2, 1)
    # partitions of one key: every two-key transaction is cross-partition
    assert oracle.graph_stats(level, root, part_size=1) == (2, 2, 3)
    # one partition holds keys 0..7: nothing crosses
    assert oracle.graph_stats(level, root, part_size=8) == (2, 2, 0)


@pytest.mark.parametrize("mode", [oracle.MODE_PAPER, oracle.MODE_ADD])
@pytest.mark.parametrize("seed", [5, 6])
def test_removing_the_0set_makes_the_1set_the_new_0set(mode, seed):
    """Section 5.3 / Figure 2(d): once the 0-set leaves the pool, the depths
    of the remaining transactions, recomputed on what remains, are their old
    depths minus one -- so the former 1-set is the new 0-set.  Repeating the
    step drains the bulk in exactly depth + 1 steps."""
    kw = _mixed_small_db()
    db = oracle.OracleDB(**kw)
    bulk = _mixed_bulk(300, seed, kw)
    obj, cls, _ = db.extract(bulk, mode, oracle.MAX_OPS)
    lv = oracle.levels(obj, cls, db.num_objects())
    keep = np.arange(len(lv))
    steps = 0
    while len(keep):
        sub = oracle.levels(obj[keep], cls[keep], db.num_objects())
        assert np.array_equal(sub, lv[keep] - steps)
        keep = keep[sub > 0]
        steps += 1
    assert steps == lv.max() + 1


# ---------------------------------------------------------------------------
# Subscriber procedures on a hand-built database (Appendix E stand-ins)
# ---------------------------------------------------------------------------
def _pack2(lo, hi):
    return (int(lo) & 0xFFFFFFFF) | ((int(hi) & 0xFFFFFFFF) << 32)


def test_subscriber_procedures_by_hand():
    """Each subscriber type on a two-subscriber database whose every row is
    written out here, with the expected status and outputs worked by hand
    from the procedures' definitions: lookups by key, the call-forwarding
    range test (start_time <= the given start, end_time > the given end),
    duplicate and missing keys, and the two-phase aborts."""
    t = {
        "sub": np.stack([np.arange(16) + 100, np.arange(16) + 200]).astype(np.int32),
        "ai_present": np.array([[1, 0, 0, 0], [0, 1, 0, 0]], dtype=np.int32),
        "ai_data": np.arange(2 * 4 * 4, dtype=np.int32).reshape(2, 4, 4) + 1000,
        "sf_present": np.array([[1, 1, 0, 0], [0, 0, 1, 0]], dtype=np.int32),
        "sf_active": np.array([[1, 0, 0, 0], [0, 0, 1, 0]], dtype=np.int32),
        "sf_err": np.zeros((2, 4), dtype=np.int32),
        "sf_data_a": np.zeros((2, 4), dtype=np.int32),
        "sf_data_b": np.zeros((2, 4), dtype=np.int32),
        "cf_present": np.zeros((2, 4, 3), dtype=np.int32),
        "cf_end": np.zeros((2, 4, 3), dtype=np.int32),
        "cf_numberx": np.zeros((2, 4, 3), dtype=np.int32),
    }
    # subscriber 0, facility 1: start 0 until 5 -> 111, start 8 until 12 -> 222
    t["cf_present"][0, 0, :2] = 1
    t["cf_end"][0, 0, :2] = (5, 12)
    t["cf_numberx"][0, 0, :2] = (111, 222)
    S = W
    txns = [  # (type, params, status, outputs)
        (S.SUB_GET_SUBSCRIBER, [0], 0, [_pack2(100 + 2 * j, 101 + 2 * j) for j in range(8)]),
        (S.SUB_GET_ACCESS, [0, 1], 0, [_pack2(1000, 1001), _pack2(1002, 1003)]),
        (S.SUB_GET_ACCESS, [0, 2], 1, []),
        (S.SUB_GET_NEW_DEST, [0, 1, 8, 10], 0, [1, 222]),
        (S.SUB_GET_NEW_DEST, [0, 2, 8, 10], 1, []),            # facility 2 inactive
        (S.SUB_INSERT_CF, [0, 1, 16, 20, 333], 0, []),
        (S.SUB_INSERT_CF, [0, 1, 16, 21, 444], 2, []),          # duplicate key
        (S.SUB_INSERT_CF, [0, 3, 0, 5, 555], 1, []),            # no facility 3
        (S.SUB_GET_NEW_DEST, [0, 1, 16, 17], 0, [1, 333]),
        (S.SUB_DELETE_CF, [0, 1, 8], 0, []),
        (S.SUB_DELETE_CF, [0, 1, 8], 1, []),                    # already gone
        (S.SUB_GET_NEW_DEST, [0, 1, 16, 4], 0, [2, 111, 333]),
        (S.SUB_UPDATE_LOCATION, [1, 77], 0, [215]),
        (S.SUB_UPDATE_LOCATION, [1, 88], 0, [77]),
        (S.SUB_UPDATE_FACILITY, [0, 1, 1, 9], 0, []),
        (S.SUB_UPDATE_FACILITY, [1, 1, 1, 9], 1, []),           # subscriber 1 has no facility 1
        (S.SUB_GET_SUBSCRIBER, [0], 0, [_pack2(1, 101)] + [_pack2(102 + 2 * j, 103 + 2 * j) for j in range(7)]),
    ]
    n = len(txns)
    params = np.zeros((n, W.SUB_PARAMS), dtype=np.int64)
    for i, (_, p, _, _) in enumerate(txns):
        params[i, :len(p)] = p
    bulk = {"ts": np.arange(n, dtype=np.int64), "type": np.array([x[0] for x in txns], dtype=np.int32),
            "params": params, "P": W.SUB_PARAMS}
    db = oracle.OracleDB(sub=t)
    st, out = db.execute(bulk, R=8)
    for i, (_, _, want_st, want_out) in enumerate(txns):
        assert st[i] == want_st, i
        got = [int(v) & 0xFFFFFFFFFFFFFFFF for v in out[i]]
        want = [v & 0xFFFFFFFFFFFFFFFF for v in want_out] + [0] * (8 - len(want_out))
        assert got == want, i
    assert db["cf_present"][0, 0].tolist() == [1, 0, 1]
    assert db["cf_end"][0, 0, 2] == 20 and db["cf_numberx"][0, 0, 2] == 333
    assert db["sub"][1, 15] == 88 and db["sub"][0, 0] == 1 and db["sf_data_a"][0, 0] == 9
    assert db["sf_data_a"][1, 0] == 0


# ---------------------------------------------------------------------------
# Order-entry procedures on a hand-built database (Appendix E stand-ins)
# ---------------------------------------------------------------------------
def test_order_entry_procedures_by_hand():
    """New-order, payment and order-status on one warehouse and four items,
    every expected value worked by hand: the stock rule (take the quantity,
    or take it and add 91 when fewer than quantity + 10 remain), the total
    with discount and taxes in basis points, order ids from the district's
    counter, a read-phase abort on an unknown item, and order-status reading
    back the customer's last order and its lines."""
    n_d, n_c, n_items = W.OE_DISTRICTS, W.OE_DISTRICTS * W.OE_CUSTOMERS, 4
    t = {
        "w_tax": np.array([1000], dtype=np.int64), "w_ytd": np.zeros(1, dtype=np.int64),
        "d_tax": np.zeros(n_d, dtype=np.int64), "d_ytd": np.zeros(n_d, dtype=np.int64),
        "d_next_o_id": np.ones(n_d, dtype=np.int64),
        "c_discount": np.zeros(n_c, dtype=np.int64), "c_balance": np.zeros(n_c, dtype=np.int64),
        "c_ytd": np.zeros(n_c, dtype=np.int64), "c_payment_cnt": np.zeros(n_c, dtype=np.int64),
        "c_last_o_id": np.zeros(n_c, dtype=np.int64),
        "i_price": np.array([100, 250, 1000, 40], dtype=np.int64),
        "s_quantity": np.array([50, 12, 9, 100], dtype=np.int32),
        "s_ytd": np.zeros(n_items, dtype=np.int64), "s_order_cnt": np.zeros(n_items, dtype=np.int32),
    }
    t["d_tax"][0] = 500
    t["c_discount"][0] = 2000

    def line(item, qty, sw=0):
        return item | (sw << 24) | (qty << 40)

    NO, PAY, OS = W.OE_NEW_ORDER, W.OE_PAYMENT, W.OE_ORDER_STATUS
    txns = [  # (type, [w, d, c, x, lines...], status, outputs)
        (NO, [0, 0, 0, 3, line(0, 5), line(1, 3), line(2, 2)], 0, [1, 2990, 3]),
        (OS, [0, 0, 0], 0, [0, 1, 3, 3250]),
        (PAY, [0, 0, 0, 700], 0, [-700]),
        (OS, [0, 0, 1], 1, [0, 0]),                              # customer 1: no order yet
        (NO, [0, 0, 1, 2, line(3, 10), line(7, 1)], 1, []),       # item 7 does not exist
        (NO, [0, 0, 1, 1, line(0, 40)], 0, [2, 4600, 1]),
        (OS, [0, 0, 1], 0, [0, 2, 1, 4000]),
    ]
    n = len(txns)
    params = np.zeros((n, W.OE_PARAMS), dtype=np.int64)
    for i, (_, p, _, _) in enumerate(txns):
        params[i, :len(p)] = p
    bulk = {"ts": np.arange(n, dtype=np.int64), "type": np.array([x[0] for x in txns], dtype=np.int32),
            "params": params, "P": W.OE_PARAMS}
    db = oracle.OracleDB(oe=t, ord_cap=16, ol_cap=64, oid_cap=16)
    st, out = db.execute(bulk, R=4)
    for i, (_, _, want_st, want_out) in enumerate(txns):
        assert st[i] == want_st, i
        assert out[i].tolist() == want_out + [0] * (4 - len(want_out)), i
    # 3,250 x (1 - 20 %) x (1 + 10 % + 5 %) = 2,990 (first order)
    assert db["s_quantity"].tolist() == [96, 100, 98, 100]
    assert db["s_ytd"].tolist() == [45, 3, 2, 0] and db["s_order_cnt"].tolist() == [2, 1, 1, 0]
    assert db["d_next_o_id"][0] == 3 and db["w_ytd"][0] == 700 and db["d_ytd"][0] == 700
    assert db["c_balance"][0] == -700 and db["c_payment_cnt"][0] == 1 and db["c_last_o_id"][1] == 2
    assert len(db.orders()) == 2 and len(db.order_lines()) == 4


@pytest.mark.parametrize("mode", [oracle.MODE_PAPER, oracle.MODE_ADD])
def test_random_linear_extensions_of_a_larger_bulk(mode):
    """The brute-force check at a size where the orders cannot be listed:
    random orders that keep every conflicting pair in timestamp order, over
    a hot mixed bulk of 160 transactions, all reach Definition 1's result."""
    kw = _mixed_small_db()
    bulk = _mixed_bulk(160, 777, kw)
    ref_db = oracle.OracleDB(**kw)
    obj, cls, _ = ref_db.extract(bulk, mode, oracle.MAX_OPS)
    st0, out0 = ref_db.execute(bulk, R=8)
    s0 = oracle_logical_state(ref_db)
    orders = linear_extensions(len(bulk["ts"]), conflict_pairs(obj, cls), limit=40, seed=5)
    assert len(orders) == 40
    assert sum(not np.array_equal(o, np.arange(len(o))) for o in orders) >= 30
    for order in orders:
        db = oracle.OracleDB(**kw)
        st, out = db.execute(bulk, R=8, order=order)
        assert states_equal(s0, oracle_logical_state(db))
        assert np.array_equal(st, st0) and np.array_equal(out, out0)
