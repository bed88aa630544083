"""Test-side helpers: logical database state, property checks, linear
extensions.  Pure numpy/python; shared by oracle and GPU parity tests."""
from __future__ import annotations

import itertools
import random

import numpy as np

CLS_R, CLS_W, CLS_A = 0, 1, 2


def conflicts(c1: int, c2: int) -> bool:
    """Two basic operations on one item conflict unless both read or both are
    blind additions (Section 4.1, plus the ADD refinement)."""
    if c1 == CLS_R and c2 == CLS_R:
        return False
    if c1 == CLS_A and c2 == CLS_A:
        return False
    return True


def conflict_pairs(obj, cls):
    """All (i, j) with i < j whose transactions conflict, as a set."""
    n, K = obj.shape
    by_obj: dict = {}
    for i in range(n):
        for j in range(K):
            if obj[i, j] >= 0:
                by_obj.setdefault(int(obj[i, j]), []).append((i, int(cls[i, j])))
    pairs = set()
    for accs in by_obj.values():
        for (a, ca), (b, cb) in itertools.combinations(accs, 2):
            if a != b and conflicts(ca, cb):
                pairs.add((min(a, b), max(a, b)))
    return pairs


def check_properties(level, obj, cls):
    """Property 1 (a k-set is conflict-free) and Property 2 (every member of
    a k-set, k >= 1, conflicts with an earlier member of the (k-1)-set).
    Returns a list of violations (empty when both hold)."""
    bad = []
    pairs = conflict_pairs(obj, cls)
    preds: dict = {}
    for a, b in pairs:
        if level[a] == level[b]:
            bad.append(("P1", a, b))
        preds.setdefault(b, []).append(a)
    for t in range(len(level)):
        if level[t] >= 1:
            if not any(level[p] == level[t] - 1 for p in preds.get(t, [])):
                bad.append(("P2", t))
        elif t in preds and level[t] == 0:
            bad.append(("source-with-pred", t))
    return bad


def linear_extensions(n, pairs, limit=400, seed=0):
    """Up to ``limit`` orders of 0..n-1 that respect every (a, b) in pairs
    (a before b).  Exhaustive when there are at most ``limit``; otherwise a
    random sample (including the identity)."""
    succ = {i: set() for i in range(n)}
    indeg = [0] * n
    for a, b in pairs:
        if b not in succ[a]:
            succ[a].add(b)
            indeg[b] += 1
    out = []

    def rec(prefix, indeg, avail):
        if len(out) > limit:
            return
        if len(prefix) == n:
            out.append(list(prefix))
            return
        for v in sorted(avail):
            nd = indeg[:]
            na = set(avail)
            na.discard(v)
            for s in succ[v]:
                nd[s] -= 1
                if nd[s] == 0:
                    na.add(s)
            prefix.append(v)
            rec(prefix, nd, na)
            prefix.pop()

    rec([], indeg, {i for i in range(n) if indeg[i] == 0})
    if len(out) <= limit:
        return out
    rng = random.Random(seed)
    sample = [list(range(n))]
    while len(sample) < limit:
        nd = indeg[:]
        avail = [i for i in range(n) if nd[i] == 0]
        order = []
        while avail:
            v = avail.pop(rng.randrange(len(avail)))
            order.append(v)
            for s in succ[v]:
                nd[s] -= 1
                if nd[s] == 0:
                    avail.append(s)
        sample.append(order)
    return sample


def oracle_logical_state(db):
    """The oracle database as comparable arrays; append-only tables are
    compared as multisets keyed by their primary keys (physical row order is
    not part of the state)."""
    st = {}
    for k in ("acc_bal", "tel_bal", "br_bal", "sub", "ai_present",
              "sf_present", "w_ytd", "d_ytd", "d_next_o_id", "c_balance", "c_ytd",
              "c_payment_cnt", "c_last_o_id", "s_quantity", "s_ytd", "s_order_cnt"):
        if k in db.a:
            st[k] = db.a[k].copy()
    # child-row fields exist only where the row does
    if "ai_data" in db.a:
        st["ai_data"] = np.where(db.a["ai_present"].astype(bool)[:, :, None], db.a["ai_data"], 0)
    for k in ("sf_active", "sf_err", "sf_data_a", "sf_data_b"):
        if k in db.a:
            st[k] = np.where(db.a["sf_present"].astype(bool), db.a[k], 0)
    if "cf_present" in db.a:
        p = db.a["cf_present"].astype(bool)
        st["cf_present"] = p.copy()
        st["cf_end"] = np.where(p, db.a["cf_end"], 0)
        st["cf_numberx"] = np.where(p, db.a["cf_numberx"], 0)
    if "hist" in db.a:
        h = db.history()
        st["history"] = h[np.argsort(h[:, 0], kind="stable")].copy()
    if "ord" in db.a:
        orders = db.orders()
        ol = db.order_lines()
        st["orders"] = _sorted_rows(orders[:, :5])
        keys = orders[ol[:, 0].astype(np.int64), :3] if len(ol) else np.zeros((0, 3), np.int64)
        st["order_lines"] = _sorted_rows(np.column_stack([keys, ol[:, 1:5]]).reshape(-1, 7))
    return st


def _sorted_rows(a):
    """Rows of a 2-D int array in lexicographic order (a canonical multiset)."""
    a = np.asarray(a, dtype=np.int64)
    if len(a) == 0:
        return a.reshape(0, a.shape[1] if a.ndim == 2 else 0)
    return a[np.lexsort(a.T[::-1])]


def states_equal(a, b):
    if a.keys() != b.keys():
        return False
    for k in a:
        x, y = a[k], b[k]
        if isinstance(x, np.ndarray):
            if x.shape != y.shape or not np.array_equal(x, y):
                return False
        elif x != y:
            return False
    return True


def state_diff(a, b):
    out = []
    for k in sorted(set(a) | set(b)):
        if k not in a or k not in b:
            out.append(k)
            continue
        x, y = a[k], b[k]
        if isinstance(x, np.ndarray):
            if x.shape != y.shape or not np.array_equal(x, y):
                out.append(k)
        elif x != y:
            out.append(k)
    return out


def gpu_logical_state(db, dc=False, sub=False, oe=False, n_sub=0, n_wh=0, n_items=0):
    """The engine's database read back through gputx_read_table, in the same
    logical form as ``oracle_logical_state``."""
    import paper_1103_3105_gb300 as G
    st = {}
    if dc:
        st["acc_bal"] = db.read(G.TBL_DC_ACCOUNT)[:, 0]
        st["tel_bal"] = db.read(G.TBL_DC_TELLER)[:, 0]
        st["br_bal"] = db.read(G.TBL_DC_BRANCH)[:, 0]
        h = db.read(G.TBL_DC_HISTORY)
        st["history"] = h[np.argsort(h[:, 0], kind="stable")]
    if sub:
        st["sub"] = db.read(G.TBL_SUB_SUBSCRIBER).astype(np.int32)
        ai = db.read(G.TBL_SUB_ACCESS_INFO)
        p = np.zeros((n_sub, 4), dtype=np.uint8)
        d = np.zeros((n_sub, 4, 4), dtype=np.int32)
        p[ai[:, 0], ai[:, 1] - 1] = 1
        d[ai[:, 0], ai[:, 1] - 1] = ai[:, 2:6]
        st["ai_present"], st["ai_data"] = p, d
        sf = db.read(G.TBL_SUB_SPECIAL_FACILITY)
        sp = np.zeros((n_sub, 4), dtype=np.uint8)
        sp[sf[:, 0], sf[:, 1] - 1] = 1
        st["sf_present"] = sp
        for j, k in enumerate(("sf_active", "sf_err", "sf_data_a", "sf_data_b")):
            a = np.zeros((n_sub, 4), dtype=np.int32)
            a[sf[:, 0], sf[:, 1] - 1] = sf[:, 2 + j]
            st[k] = a
        cf = db.read(G.TBL_SUB_CALL_FORWARDING)
        cp = np.zeros((n_sub, 4, 3), dtype=bool)
        ce = np.zeros((n_sub, 4, 3), dtype=np.int32)
        cn = np.zeros((n_sub, 4, 3), dtype=np.int32)
        idx = (cf[:, 0], cf[:, 1] - 1, cf[:, 2] // 8)
        flat = (cf[:, 0] * 4 + (cf[:, 1] - 1)) * 3 + cf[:, 2] // 8
        assert len(np.unique(flat)) == len(cf), "duplicate live call_forwarding key"
        cp[idx] = True
        ce[idx] = cf[:, 3]
        cn[idx] = cf[:, 4]
        st["cf_present"], st["cf_end"], st["cf_numberx"] = cp, ce, cn
    if oe:
        w = db.read(G.TBL_OE_WAREHOUSE)
        d = db.read(G.TBL_OE_DISTRICT)
        c = db.read(G.TBL_OE_CUSTOMER)
        s = db.read(G.TBL_OE_STOCK)
        st["w_ytd"] = w[:, 1]
        st["d_ytd"], st["d_next_o_id"] = d[:, 1], d[:, 2]
        st["c_balance"], st["c_ytd"], st["c_payment_cnt"], st["c_last_o_id"] = c[:, 1], c[:, 2], c[:, 3], c[:, 4]
        st["s_quantity"], st["s_ytd"], st["s_order_cnt"] = (s[:, 0].astype(np.int32), s[:, 1],
                                                            s[:, 2].astype(np.int32))
        st["orders"] = _sorted_rows(db.read(G.TBL_OE_ORDER))
        st["order_lines"] = _sorted_rows(db.read(G.TBL_OE_ORDER_LINE))
    return st


# ---------------------------------------------------------------------------
# primary-index consistency: every live row is found by its key, and every
# index entry points to a live row with that key
# ---------------------------------------------------------------------------
HKEY_EMPTY = np.uint64((1 << 64) - 1)
HKEY_TOMB = np.uint64((1 << 64) - 2)


def murmur_fmix64(k):
    """The 64-bit finaliser of MurmurHash3 (Appleby), the index's hash."""
    k = np.asarray(k, dtype=np.uint64).copy()
    with np.errstate(over="ignore"):
        k ^= k >> np.uint64(33)
        k *= np.uint64(0xFF51AFD7ED558CCD)
        k ^= k >> np.uint64(33)
        k *= np.uint64(0xC4CEB9FE1A85EC53)
        k ^= k >> np.uint64(33)
    return k


def slot_keys(table, slots):
    """Index key of every storage slot (rows of gputx_read_slots)."""
    import paper_1103_3105_gb300 as G
    s = slots.astype(np.int64)
    if table in (G.TBL_SUB_ACCESS_INFO, G.TBL_SUB_SPECIAL_FACILITY):
        return (s[:, 0] * 4 + (s[:, 1] - 1)).astype(np.uint64)
    if table == G.TBL_SUB_CALL_FORWARDING:
        return ((s[:, 0] * 4 + (s[:, 1] - 1)) * 3 + s[:, 2] // 8).astype(np.uint64)
    if table == G.TBL_OE_ORDER:
        return ((((s[:, 0] * 10 + s[:, 1]) << 32) | (s[:, 2] & 0xFFFFFFFF))).astype(np.uint64)
    raise ValueError(table)


def index_violations(keys, rows, slots, table, expected_keys):
    """Checks one open-addressing index against its table's slots.

    keys/rows: the raw index arrays; slots: the table's storage with a live
    flag in the last column; expected_keys: the live keys of the oracle's
    table.  Returns a list of violations (empty when the index is exact)."""
    bad = []
    size = len(keys)
    if size == 0 or size & (size - 1):
        return [f"index size {size} is not a power of two"]
    mask = np.uint64(size - 1)
    occ = (keys != HKEY_EMPTY) & (keys != HKEY_TOMB)
    pos = np.flatnonzero(occ)
    k = keys[pos]
    r = rows[pos].astype(np.int64)
    if len(r) and r.max() >= len(slots):
        return [f"entry points past the table ({r.max()} >= {len(slots)})"]
    if not (slots[r, -1] == 1).all():
        bad.append(f"{int((slots[r, -1] != 1).sum())} entries point at dead rows")
    sk = slot_keys(table, slots[r])
    if not np.array_equal(sk, k):
        bad.append(f"{int((sk != k).sum())} entries point at a row with another key")
    if len(np.unique(k)) != len(k):
        bad.append("a key is indexed twice")
    if len(np.unique(r)) != len(r):
        bad.append("a row is indexed twice")
    n_live = int(slots[:, -1].sum())
    if n_live != len(k):
        bad.append(f"{n_live} live rows but {len(k)} index entries")
    # a lookup probes linearly from the key's home slot and stops at the
    # first empty slot: no empty slot may lie between home and the key
    home = (murmur_fmix64(k) & mask).astype(np.int64)
    dist = (pos - home) & (size - 1)
    empty = (keys == HKEY_EMPTY).astype(np.int64)
    cs = np.concatenate([[0], np.cumsum(np.concatenate([empty, empty]))])
    gaps = cs[home + dist] - cs[home]
    if (gaps > 0).any():
        bad.append(f"{int((gaps > 0).sum())} keys sit behind an empty slot (not found by a lookup)")
    exp = np.sort(np.asarray(expected_keys, dtype=np.uint64))
    if not np.array_equal(np.sort(k), exp):
        bad.append(f"key set differs from the oracle's ({len(k)} vs {len(exp)} keys)")
    return bad


def oracle_index_keys(o, table):
    """Live keys of the oracle's child or order table."""
    import paper_1103_3105_gb300 as G
    if table == G.TBL_SUB_ACCESS_INFO:
        return np.flatnonzero(o["ai_present"].reshape(-1)).astype(np.uint64)
    if table == G.TBL_SUB_SPECIAL_FACILITY:
        return np.flatnonzero(o["sf_present"].reshape(-1)).astype(np.uint64)
    if table == G.TBL_SUB_CALL_FORWARDING:
        return np.flatnonzero(o["cf_present"].reshape(-1)).astype(np.uint64)
    if table == G.TBL_OE_ORDER:
        od = o.orders()
        return (((od[:, 0] * 10 + od[:, 1]) << 32) | od[:, 2]).astype(np.uint64)
    raise ValueError(table)


def check_indexes(g, o, sub=False, oe=False):
    """Every primary index of the engine's database against its table and
    the oracle's live keys; returns {index name: violations}."""
    import paper_1103_3105_gb300 as G
    pairs = []
    if sub:
        pairs += [(G.INDEX_ACCESS_INFO, G.TBL_SUB_ACCESS_INFO), (G.INDEX_SPECIAL_FACILITY, G.TBL_SUB_SPECIAL_FACILITY),
                  (G.INDEX_CALL_FORWARDING, G.TBL_SUB_CALL_FORWARDING)]
    if oe:
        pairs += [(G.INDEX_ORDER, G.TBL_OE_ORDER)]
    out = {}
    for idx, table in pairs:
        keys, rows = g.read_index(idx)
        slots = g.read_slots(table)
        v = index_violations(keys, rows, slots, table, oracle_index_keys(o, table))
        if v:
            out[table] = v
    return out
