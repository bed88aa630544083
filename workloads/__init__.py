"""Seeded synthetic inputs for the bulk transaction engine and its oracle.

This module only draws random inputs: transaction signatures ``<ts, type,
params>`` (paper Section 3.2) and the initial contents of the tables.  It holds
none of the method's arithmetic (no procedure, no conflict analysis), so both
the CUDA path and the CPU oracle may consume what it produces.

Stand-in workloads (the benchmark kits are not available):
  * debit-credit (TPC-B-shaped, paper Section 5.1 / Fig. 2): branches, tellers,
    accounts with int64 balances and an append-only history table;
  * subscriber-location (TM-1-shaped, paper Appendix E): subscriber rows of 16
    int32 fields with access_info / special_facility / call_forwarding
    children, seven transaction types;
  * order-entry (TPC-C-shaped, paper Appendix E): warehouses, districts,
    customers, items, stock, new-order / payment / order-status.

Skewed keys use the Zipf generator of Gray et al. (SIGMOD 1994, "Quickly
generating billion-record synthetic databases") followed by a fixed Feistel
permutation so hot keys do not cluster in one branch or partition.
"""
from __future__ import annotations

import numpy as np

# ---------------------------------------------------------------------------
# transaction type identifiers (shared vocabulary of the C-ABI)
# ---------------------------------------------------------------------------
DC_DEBIT_CREDIT = 0
SUB_GET_SUBSCRIBER = 1
SUB_GET_ACCESS = 2
SUB_GET_NEW_DEST = 3
SUB_UPDATE_LOCATION = 4
SUB_UPDATE_FACILITY = 5
SUB_INSERT_CF = 6
SUB_DELETE_CF = 7
OE_NEW_ORDER = 8
OE_PAYMENT = 9
OE_ORDER_STATUS = 10

SUB_TYPES = (SUB_GET_SUBSCRIBER, SUB_GET_ACCESS, SUB_GET_NEW_DEST,
             SUB_UPDATE_LOCATION, SUB_UPDATE_FACILITY, SUB_INSERT_CF,
             SUB_DELETE_CF)
# read-only lookups 30/25/25 %, updates and inserts/deletes 8/8/2/2 %
SUB_MIX = (0.30, 0.25, 0.25, 0.08, 0.08, 0.02, 0.02)
OE_TYPES = (OE_NEW_ORDER, OE_PAYMENT, OE_ORDER_STATUS)
OE_MIX = (0.45, 0.43, 0.12)

DC_PARAMS = 2           # account, delta
SUB_PARAMS = 5          # s_id, a, b, c, d
OE_MAX_LINES = 15
OE_PARAMS = 4 + OE_MAX_LINES  # w, d, c, ol_cnt, packed lines

DELTA_MAX = 99999
SUB_START_TIMES = (0, 8, 16)


def seed_for(config: int, variant: int = 0) -> int:
    """Seed convention: 1103_0000 + config*100 + variant."""
    return 1103_0000 + config * 100 + variant


# ---------------------------------------------------------------------------
# key distributions
# ---------------------------------------------------------------------------
_ZETA_CACHE: dict = {}


def _zeta(n: int, theta: float) -> float:
    key = (n, theta)
    if key not in _ZETA_CACHE:
        i = np.arange(1, n + 1, dtype=np.float64)
        _ZETA_CACHE[key] = float(np.sum(i ** (-theta)))
    return _ZETA_CACHE[key]


def zipf_ranks(rng: np.random.Generator, n: int, theta: float, size: int) -> np.ndarray:
    """Zipf(theta) ranks in [0, n) by Gray et al.'s closed-form inversion.

    theta == 0 degenerates to the uniform distribution.
    """
    if theta == 0.0:
        return rng.integers(0, n, size=size, dtype=np.int64)
    if not (0.0 < theta < 1.0):
        raise ValueError("theta must be in [0, 1)")
    zetan = _zeta(n, theta)
    zeta2 = 1.0 + 0.5 ** theta
    alpha = 1.0 / (1.0 - theta)
    eta = (1.0 - (2.0 / n) ** (1.0 - theta)) / (1.0 - zeta2 / zetan)
    u = rng.random(size)
    uz = u * zetan
    r = (n * np.power(eta * u - eta + 1.0, alpha)).astype(np.int64)
    r = np.where(uz < 1.0 + 0.5 ** theta, 1, r)
    r = np.where(uz < 1.0, 0, r)
    return np.clip(r, 0, n - 1)


def _feistel_round(x: np.ndarray, k: int, half: int, mask: int) -> np.ndarray:
    lo = x & mask
    hi = x >> half
    f = ((lo * 0x9E3779B1 + k) ^ (lo >> 3)) & mask
    return (lo << half) | (hi ^ f)


def scramble(keys: np.ndarray, n: int, seed: int = 0x5EED) -> np.ndarray:
    """Fixed bijection of [0, n): 4-round Feistel on an even bit width with
    cycle walking, so Zipf-hot ranks land on unrelated keys."""
    keys = np.asarray(keys, dtype=np.int64)
    if n <= 2:
        return keys.copy()
    bits = max(2, int(np.ceil(np.log2(n))))
    bits += bits & 1
    half = bits // 2
    mask = (1 << half) - 1
    rk = [(seed * (i + 7) * 0x2545F491) & mask for i in range(4)]
    out = keys.copy()
    todo = np.ones(out.shape, dtype=bool)
    cur = out.copy()
    while todo.any():
        x = cur[todo]
        for k in rk:
            x = _feistel_round(x, k, half, mask)
        cur[todo] = x
        done_now = x < n
        idx = np.flatnonzero(todo)
        out[idx[done_now]] = x[done_now]
        todo[idx[done_now]] = False
    return out


def _packed_lines(items, supply_w, qty):
    """One int64 per order line: item (bits 0..23), supply warehouse (24..39),
    quantity (40..47)."""
    return (items.astype(np.int64)
            | (supply_w.astype(np.int64) << 24)
            | (qty.astype(np.int64) << 40))


# ---------------------------------------------------------------------------
# debit-credit
# ---------------------------------------------------------------------------
def dc_bulk(n: int, n_accounts: int, theta: float = 0.0, seed: int = 0,
            ts0: int = 0) -> dict:
    """A bulk of ``n`` debit-credit transactions.

    account: uniform (theta = 0) or Zipf(theta) then scrambled;
    delta: uniform int64 in [-99999, 99999]; ts: ts0 .. ts0+n-1.
    """
    rng = np.random.default_rng(seed)
    ranks = zipf_ranks(rng, n_accounts, theta, n)
    acct = ranks if theta == 0.0 else scramble(ranks, n_accounts)
    delta = rng.integers(-DELTA_MAX, DELTA_MAX + 1, size=n, dtype=np.int64)
    params = np.empty((n, DC_PARAMS), dtype=np.int64)
    params[:, 0] = acct
    params[:, 1] = delta
    return {
        "ts": np.arange(ts0, ts0 + n, dtype=np.int64),
        "type": np.full(n, DC_DEBIT_CREDIT, dtype=np.int32),
        "params": params,
        "P": DC_PARAMS,
    }


def dc_tables(n_branches: int, n_tellers: int, n_accounts: int) -> dict:
    """Initial debit-credit tables: every balance starts at zero."""
    return {
        "branch_balance": np.zeros(n_branches, dtype=np.int64),
        "teller_balance": np.zeros(n_tellers, dtype=np.int64),
        "account_balance": np.zeros(n_accounts, dtype=np.int64),
    }


# ---------------------------------------------------------------------------
# subscriber-location
# ---------------------------------------------------------------------------
def _random_subsets(rng, rows: int, universe: int, kmin: int, kmax: int):
    """Boolean [rows, universe] masks, each row a uniform random subset whose
    size is uniform in [kmin, kmax]."""
    k = rng.integers(kmin, kmax + 1, size=rows)
    order = np.argsort(rng.random((rows, universe)), axis=1)
    rank = np.empty_like(order)
    np.put_along_axis(rank, order, np.arange(universe)[None, :].repeat(rows, 0), axis=1)
    return rank < k[:, None]


def sub_tables(n_sub: int, seed: int = 0) -> dict:
    """Logical initial state of the subscriber schema (dense form).

    subscriber: n_sub x 16 int32 fields.
    access_info: 1-4 of ai_type 1..4 per subscriber, fields data1..data4.
    special_facility: 1-4 of sf_type 1..4 per subscriber, fields is_active
      (85 % active), error_cntrl, data_a, data_b.
    call_forwarding: 0-3 of start_time {0, 8, 16} per facility, fields
      end_time (start_time + 1..8) and numberx.
    """
    rng = np.random.default_rng(seed)
    sub = rng.integers(0, 1 << 30, size=(n_sub, 16), dtype=np.int64).astype(np.int32)
    ai_present = _random_subsets(rng, n_sub, 4, 1, 4)
    ai_data = rng.integers(0, 1 << 30, size=(n_sub, 4, 4), dtype=np.int64).astype(np.int32)
    sf_present = _random_subsets(rng, n_sub, 4, 1, 4)
    sf_active = (rng.random((n_sub, 4)) < 0.85).astype(np.int32)
    sf_err = rng.integers(0, 256, size=(n_sub, 4), dtype=np.int64).astype(np.int32)
    sf_data_a = rng.integers(0, 256, size=(n_sub, 4), dtype=np.int64).astype(np.int32)
    sf_data_b = rng.integers(0, 1 << 30, size=(n_sub, 4), dtype=np.int64).astype(np.int32)
    cf_present = _random_subsets(rng, n_sub * 4, 3, 0, 3).reshape(n_sub, 4, 3)
    cf_present &= sf_present[:, :, None]
    st = np.array(SUB_START_TIMES, dtype=np.int32)[None, None, :]
    cf_end = (st + rng.integers(1, 9, size=(n_sub, 4, 3))).astype(np.int32)
    cf_numberx = rng.integers(0, 1 << 30, size=(n_sub, 4, 3), dtype=np.int64).astype(np.int32)
    return {
        "sub": sub,
        "ai_present": ai_present, "ai_data": ai_data,
        "sf_present": sf_present, "sf_active": sf_active, "sf_err": sf_err,
        "sf_data_a": sf_data_a, "sf_data_b": sf_data_b,
        "cf_present": cf_present, "cf_end": cf_end, "cf_numberx": cf_numberx,
    }


def sub_bulk(n: int, n_sub: int, theta: float = 0.0, seed: int = 0,
             ts0: int = 0, mix=SUB_MIX) -> dict:
    """A bulk of ``n`` mixed subscriber transactions.

    s_id uniform or Zipf(theta) then scrambled.  Parameters per type
    (columns a, b, c, d after s_id):
      GET_SUBSCRIBER    -
      GET_ACCESS        ai_type 1..4
      GET_NEW_DEST      sf_type 1..4, start_time {0,8,16}, end_time 1..24
      UPDATE_LOCATION   location
      UPDATE_FACILITY   sf_type 1..4, bit 0/1, data_a 0..255
      INSERT_CF         sf_type 1..4, start_time {0,8,16}, end_time, numberx
      DELETE_CF         sf_type 1..4, start_time {0,8,16}
    """
    rng = np.random.default_rng(seed)
    ranks = zipf_ranks(rng, n_sub, theta, n)
    sid = ranks if theta == 0.0 else scramble(ranks, n_sub)
    cum = np.cumsum(np.asarray(mix, dtype=np.float64))
    cum /= cum[-1]
    t_idx = np.searchsorted(cum, rng.random(n), side="right")
    t_idx = np.minimum(t_idx, len(SUB_TYPES) - 1)
    types = np.asarray(SUB_TYPES, dtype=np.int32)[t_idx]
    params = np.zeros((n, SUB_PARAMS), dtype=np.int64)
    params[:, 0] = sid
    ai = rng.integers(1, 5, size=n)
    sf = rng.integers(1, 5, size=n)
    st = np.asarray(SUB_START_TIMES, dtype=np.int64)[rng.integers(0, 3, size=n)]
    et = rng.integers(1, 25, size=n)
    loc = rng.integers(0, 1 << 30, size=n)
    bit = rng.integers(0, 2, size=n)
    da = rng.integers(0, 256, size=n)
    numx = rng.integers(0, 1 << 30, size=n)
    m = types == SUB_GET_ACCESS
    params[m, 1] = ai[m]
    m = types == SUB_GET_NEW_DEST
    params[m, 1], params[m, 2], params[m, 3] = sf[m], st[m], et[m]
    m = types == SUB_UPDATE_LOCATION
    params[m, 1] = loc[m]
    m = types == SUB_UPDATE_FACILITY
    params[m, 1], params[m, 2], params[m, 3] = sf[m], bit[m], da[m]
    m = types == SUB_INSERT_CF
    params[m, 1], params[m, 2] = sf[m], st[m]
    params[m, 3], params[m, 4] = st[m] + rng.integers(1, 9, size=int(m.sum())), numx[m]
    m = types == SUB_DELETE_CF
    params[m, 1], params[m, 2] = sf[m], st[m]
    return {
        "ts": np.arange(ts0, ts0 + n, dtype=np.int64),
        "type": types,
        "params": params,
        "P": SUB_PARAMS,
    }


# ---------------------------------------------------------------------------
# order-entry
# ---------------------------------------------------------------------------
OE_DISTRICTS = 10
OE_CUSTOMERS = 3000


def oe_tables(n_wh: int, n_items: int = 100_000, seed: int = 0) -> dict:
    """Initial order-entry tables.

    warehouse: tax (0..2000 basis points), ytd;
    district (10 per warehouse): tax, ytd, next_o_id (starts at 1);
    customer (3,000 per district): discount (0..5000 bp), balance, ytd_payment,
      payment_cnt, last_o_id (0 = none);
    item: price (100..10000); stock (n_wh x n_items): quantity (10..100),
      ytd, order_cnt.
    """
    rng = np.random.default_rng(seed)
    n_d = n_wh * OE_DISTRICTS
    n_c = n_d * OE_CUSTOMERS
    return {
        "w_tax": rng.integers(0, 2001, size=n_wh, dtype=np.int64),
        "w_ytd": np.zeros(n_wh, dtype=np.int64),
        "d_tax": rng.integers(0, 2001, size=n_d, dtype=np.int64),
        "d_ytd": np.zeros(n_d, dtype=np.int64),
        "d_next_o_id": np.ones(n_d, dtype=np.int64),
        "c_discount": rng.integers(0, 5001, size=n_c, dtype=np.int64),
        "c_balance": np.zeros(n_c, dtype=np.int64),
        "c_ytd": np.zeros(n_c, dtype=np.int64),
        "c_payment_cnt": np.zeros(n_c, dtype=np.int64),
        "c_last_o_id": np.zeros(n_c, dtype=np.int64),
        "i_price": rng.integers(100, 10001, size=n_items, dtype=np.int64),
        "s_quantity": rng.integers(10, 101, size=n_wh * n_items, dtype=np.int64).astype(np.int32),
        "s_ytd": np.zeros(n_wh * n_items, dtype=np.int64),
        "s_order_cnt": np.zeros(n_wh * n_items, dtype=np.int32),
    }


def oe_bulk(n: int, n_wh: int, n_items: int = 100_000, item_theta: float = 0.8,
            remote_frac: float = 0.01, invalid_frac: float = 0.01, seed: int = 0,
            ts0: int = 0, mix=OE_MIX) -> dict:
    """A bulk of ``n`` order-entry transactions.

    params: w, d, c, ol_cnt, then ol_cnt packed lines (item, supply_w, qty).
    new-order: 5..15 distinct items, Zipf(item_theta) then scrambled, qty
      1..10, supply warehouse remote with probability remote_frac, and with
      probability invalid_frac the last item id is n_items (not a valid item:
      the order aborts in its read phase).
    payment: params[3] = amount 1..5000.
    order-status: no extra parameters.
    """
    rng = np.random.default_rng(seed)
    cum = np.cumsum(np.asarray(mix, dtype=np.float64))
    cum /= cum[-1]
    t_idx = np.minimum(np.searchsorted(cum, rng.random(n), side="right"), 2)
    types = np.asarray(OE_TYPES, dtype=np.int32)[t_idx]
    params = np.zeros((n, OE_PARAMS), dtype=np.int64)
    w = rng.integers(0, n_wh, size=n)
    d = rng.integers(0, OE_DISTRICTS, size=n)
    c = rng.integers(0, OE_CUSTOMERS, size=n)
    params[:, 0], params[:, 1], params[:, 2] = w, d, c
    pay = types == OE_PAYMENT
    params[pay, 3] = rng.integers(1, 5001, size=int(pay.sum()))
    no = np.flatnonzero(types == OE_NEW_ORDER)
    m = len(no)
    if m:
        cnt = rng.integers(5, OE_MAX_LINES + 1, size=m)
        # distinct items per order: draw 2x candidates, keep first distinct
        cand = scramble(zipf_ranks(rng, n_items, item_theta, m * 32), n_items).reshape(m, 32)
        cand.sort(axis=1)
        uniq = np.ones_like(cand, dtype=bool)
        uniq[:, 1:] = cand[:, 1:] != cand[:, :-1]
        # stable: distinct values first (ascending), duplicates after
        pick = np.argsort(~uniq, axis=1, kind="stable")[:, :OE_MAX_LINES]
        items = np.take_along_axis(cand, pick, axis=1)
        short = np.flatnonzero(uniq.sum(axis=1) < OE_MAX_LINES)
        for r in short:  # rare: fewer than 15 distinct draws in 32
            u = np.unique(cand[r])
            extra = np.setdiff1d(np.arange(n_items), u)[: OE_MAX_LINES - len(u)]
            items[r] = np.concatenate([u, extra])[:OE_MAX_LINES]
        bad = rng.random(m) < invalid_frac
        items[np.arange(m), cnt - 1] = np.where(bad, n_items, items[np.arange(m), cnt - 1])
        remote = rng.random((m, OE_MAX_LINES)) < remote_frac
        other = (w[no][:, None] + rng.integers(1, max(2, n_wh), size=(m, OE_MAX_LINES))) % n_wh
        sw = np.where(remote & (n_wh > 1), other, w[no][:, None])
        qty = rng.integers(1, 11, size=(m, OE_MAX_LINES))
        lines = _packed_lines(items, sw, qty)
        valid = np.arange(OE_MAX_LINES)[None, :] < cnt[:, None]
        lines = np.where(valid, lines, 0)
        params[no, 3] = cnt
        params[no, 4:] = lines
    return {
        "ts": np.arange(ts0, ts0 + n, dtype=np.int64),
        "type": types,
        "params": params,
        "P": OE_PARAMS,
    }


# ---------------------------------------------------------------------------
# row formats of the engine's table loader (int64 fields per row)
# ---------------------------------------------------------------------------
def dc_rows(t: dict) -> dict:
    """{table id: rows} for gputx_load_table (branch, teller, account)."""
    return {0: t["branch_balance"].reshape(-1, 1), 1: t["teller_balance"].reshape(-1, 1),
            2: t["account_balance"].reshape(-1, 1)}


def sub_rows(t: dict) -> dict:
    """{table id: rows}: subscriber (16 fields), access_info (s_id, ai_type,
    data1..4), special_facility (s_id, sf_type, is_active, error_cntrl,
    data_a, data_b), call_forwarding (s_id, sf_type, start_time, end_time,
    numberx) -- child rows only where present."""
    n = t["sub"].shape[0]
    s_ai, a_ai = np.nonzero(t["ai_present"])
    ai = np.column_stack([s_ai, a_ai + 1, t["ai_data"][s_ai, a_ai]]).astype(np.int64)
    s_sf, a_sf = np.nonzero(t["sf_present"])
    sf = np.column_stack([s_sf, a_sf + 1, t["sf_active"][s_sf, a_sf], t["sf_err"][s_sf, a_sf],
                          t["sf_data_a"][s_sf, a_sf], t["sf_data_b"][s_sf, a_sf]]).astype(np.int64)
    s_cf, a_cf, k_cf = np.nonzero(t["cf_present"])
    cf = np.column_stack([s_cf, a_cf + 1, 8 * k_cf, t["cf_end"][s_cf, a_cf, k_cf],
                          t["cf_numberx"][s_cf, a_cf, k_cf]]).astype(np.int64)
    return {4: t["sub"].astype(np.int64).reshape(n, 16), 5: ai.reshape(-1, 6),
            6: sf.reshape(-1, 6), 7: cf.reshape(-1, 5)}


def oe_rows(t: dict) -> dict:
    """{table id: rows}: warehouse (tax, ytd), district (tax, ytd,
    next_o_id), customer (discount, balance, ytd_payment, payment_cnt,
    last_o_id), item (price), stock (quantity, ytd, order_cnt)."""
    return {
        8: np.column_stack([t["w_tax"], t["w_ytd"]]),
        9: np.column_stack([t["d_tax"], t["d_ytd"], t["d_next_o_id"]]),
        10: np.column_stack([t["c_discount"], t["c_balance"], t["c_ytd"], t["c_payment_cnt"],
                             t["c_last_o_id"]]),
        11: t["i_price"].reshape(-1, 1),
        12: np.column_stack([t["s_quantity"].astype(np.int64), t["s_ytd"],
                             t["s_order_cnt"].astype(np.int64)]),
    }


def concat_bulks(parts, pick) -> dict:
    """Interleave bulks of different schemas: transaction i comes from
    parts[pick[i]] (its i-th transaction); parameters are zero-padded to the
    widest schema."""
    n = len(pick)
    P = max(p["P"] for p in parts)
    params = np.zeros((n, P), dtype=np.int64)
    types = np.zeros(n, dtype=np.int32)
    for k, p in enumerate(parts):
        m = pick == k
        params[m, : p["P"]] = p["params"][m]
        types[m] = p["type"][m]
    return {"ts": np.arange(n, dtype=np.int64), "type": types, "params": params, "P": P}


def uneven_sizes(total: int, lo_log2: float = 10, hi_log2: float = 21, seed: int = 0) -> list:
    """Bulk sizes 2^U(lo_log2, hi_log2) (log-uniform, seeded), drawn until
    they add up to at least ``total``."""
    rng = np.random.default_rng(seed)
    sizes, acc = [], 0
    while acc < total:
        k = int(2 ** rng.uniform(lo_log2, hi_log2))
        sizes.append(k)
        acc += k
    return sizes


def oe_stream(total: int, n_wh: int = 64, n_items: int = 100_000, variant: int = 0, ts0: int = 0) -> tuple:
    """The batched order-entry stream: uneven bulk sizes 2^10..2^21 adding
    up to at least ``total`` transactions, and one order-entry bulk holding
    all of them in timestamp order (from ts0).  Returns (sizes, bulk)."""
    sizes = uneven_sizes(total, 10, 21, seed=seed_for(4, 1 + 10 * variant))
    bulk = oe_bulk(sum(sizes), n_wh, n_items=n_items, seed=seed_for(4, 2 + 10 * variant), ts0=ts0)
    return sizes, bulk


def served_mix(n: int, n_accounts: int, n_sub: int, theta: float, rate: float, seed_variant: int = 0) -> dict:
    """The served mix: n transactions, half debit-credit (accounts
    uniform/Zipf theta over n_accounts) and half subscriber (the 30/25/25/
    8/8/2/2 mix over n_sub subscribers), interleaved at random, with
    open-loop Poisson arrival offsets (ns) at ``rate`` transactions/s."""
    rng = np.random.default_rng(seed_for(5, seed_variant))
    tag = int(rate // 1e6)
    parts = [dc_bulk(n, n_accounts, theta, seed=seed_for(5, tag)),
             sub_bulk(n, n_sub, theta, seed=seed_for(5, 50 + tag))]
    bulk = concat_bulks(parts, rng.integers(0, 2, size=n))
    gaps = rng.exponential(1e9 / rate, size=n)
    bulk["arrival_offset_ns"] = np.cumsum(gaps).astype(np.int64)
    return bulk
