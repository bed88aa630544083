"""The index checker used by the parity tests, checked on hand-built indexes
(no GPU): an exact index passes, and each planted fault is reported."""
import numpy as np

import paper_1103_3105_gb300 as G
from tests._helpers import HKEY_EMPTY, HKEY_TOMB, index_violations, murmur_fmix64


def _build(keys_in, size):
    """Linear-probing insert of keys_in (row i holds key i) into `size` slots."""
    keys = np.full(size, HKEY_EMPTY, dtype=np.uint64)
    rows = np.zeros(size, dtype=np.uint32)
    for r, k in enumerate(keys_in):
        i = int(murmur_fmix64(np.uint64(k))) & (size - 1)
        while keys[i] != HKEY_EMPTY:
            i = (i + 1) & (size - 1)
        keys[i] = k
        rows[i] = r
    return keys, rows


def _cf_slots(keys_in):
    """call_forwarding slots whose key is keys_in[i] (s, type, start, ..., live)."""
    k = np.asarray(keys_in, dtype=np.int64)
    start = 8 * (k % 3)
    st = k // 3
    return np.column_stack([st // 4, st % 4 + 1, start, np.zeros_like(k), np.zeros_like(k), np.ones_like(k)])


def test_exact_index_passes_and_planted_faults_are_reported():
    rng = np.random.default_rng(3)
    keys_in = np.unique(rng.integers(0, 3000, size=200))
    keys, rows = _build(keys_in, 512)
    slots = _cf_slots(keys_in)
    T = G.TBL_SUB_CALL_FORWARDING
    assert index_violations(keys, rows, slots, T, keys_in) == []
    # a dead row still indexed
    s2 = slots.copy()
    s2[5, -1] = 0
    assert any("dead" in v for v in index_violations(keys, rows, s2, T, keys_in))
    # an entry pointing at the wrong row
    r2 = rows.copy()
    occ = np.flatnonzero(keys != HKEY_EMPTY)
    r2[occ[0]], r2[occ[1]] = r2[occ[1]], r2[occ[0]]
    assert any("another key" in v for v in index_violations(keys, r2, slots, T, keys_in))
    # a key moved to the next empty slot: its old slot, now empty, lies
    # between its home and it, so a lookup would stop before reaching it
    k3, r3 = keys.copy(), rows.copy()
    p = occ[0]
    q = np.flatnonzero(k3 == HKEY_EMPTY)
    q = q[q > p][0]
    k3[q], r3[q] = k3[p], r3[p]
    k3[p] = HKEY_EMPTY
    assert any("behind an empty" in v for v in index_violations(k3, r3, slots, T, keys_in))
    # a live row missing from the index
    k4 = keys.copy()
    k4[occ[2]] = HKEY_TOMB
    v = index_violations(k4, rows, slots, T, keys_in)
    assert any("live rows" in x for x in v) and any("key set" in x for x in v)
    # a key indexed twice
    k5, r5 = keys.copy(), rows.copy()
    emp = np.flatnonzero(k5 == HKEY_EMPTY)[0]
    k5[emp], r5[emp] = k5[occ[3]], r5[occ[3]]
    assert any("twice" in x for x in index_violations(k5, r5, slots, T, keys_in))
