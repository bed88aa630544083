// procs.cuh -- the registered stored procedures and their access sets.
//
// Section 3.2: every transaction type is a device function and one kernel
// dispatches on the type with a switch.  Each procedure is written two-phase
// (Appendix D): a read phase that may abort (status != 0, no writes) and a
// write phase that never aborts, so no undo log is needed.
//
// access_set() declares the basic operations (Section 4.1) of a transaction
// from its parameters alone, at field granularity (Section 3.2): a read or a
// write on an item identified by a dense object id.  Items that are never
// written (item prices, warehouse and district tax, customer discount) carry
// no operation.  In GPUTX_CONFLICT_ADD mode, increments whose old value is
// never read are class ADD.
#pragma once
#include "common.cuh"
#include "dc.cuh"

namespace gtx {

// ---------------------------------------------------------------------------
// validation of one signature (bulk contents are checked on the device)
// ---------------------------------------------------------------------------
__device__ __forceinline__ bool valid_txn(const DevDB &db, int32_t type, const int64_t *p, int P)
{
    if (type < 0 || type >= GPUTX_NUM_TYPES || !((db.registered >> type) & 1u)) return false;
    switch (type) {
    case GPUTX_T_DC_DEBIT_CREDIT:
        return P >= 2 && p[0] >= 0 && p[0] < db.n_acc;
    case GPUTX_T_SUB_GET_SUBSCRIBER:
        return P >= 1 && p[0] >= 0 && p[0] < db.n_sub;
    case GPUTX_T_SUB_GET_ACCESS:
        return P >= 2 && p[0] >= 0 && p[0] < db.n_sub && p[1] >= 1 && p[1] <= 4;
    case GPUTX_T_SUB_GET_NEW_DEST:
        return P >= 4 && p[0] >= 0 && p[0] < db.n_sub && p[1] >= 1 && p[1] <= 4;
    case GPUTX_T_SUB_UPDATE_LOCATION:
        return P >= 2 && p[0] >= 0 && p[0] < db.n_sub;
    case GPUTX_T_SUB_UPDATE_FACILITY:
        return P >= 4 && p[0] >= 0 && p[0] < db.n_sub && p[1] >= 1 && p[1] <= 4;
    case GPUTX_T_SUB_INSERT_CF:
        return P >= 5 && p[0] >= 0 && p[0] < db.n_sub && p[1] >= 1 && p[1] <= 4 &&
               (p[2] == 0 || p[2] == 8 || p[2] == 16);
    case GPUTX_T_SUB_DELETE_CF:
        return P >= 3 && p[0] >= 0 && p[0] < db.n_sub && p[1] >= 1 && p[1] <= 4 &&
               (p[2] == 0 || p[2] == 8 || p[2] == 16);
    case GPUTX_T_OE_NEW_ORDER: {
        if (P < 4 || p[0] < 0 || p[0] >= db.n_wh || p[1] < 0 || p[1] >= OE_DIST || p[2] < 0 ||
            p[2] >= OE_CUST || p[3] < 1 || p[3] > OE_MAX_LINES || P < 4 + p[3])
            return false;
        // items must be distinct; an item id of n_items or more is allowed
        // (the order aborts in its read phase), a bad warehouse is not
        for (int j = 0; j < (int)p[3]; j++) {
            int64_t line = p[4 + j];
            int64_t item = line & 0xFFFFFF, sw = (line >> 24) & 0xFFFF, qty = (line >> 40) & 0xFF;
            if (line < 0 || sw >= db.n_wh || qty < 1) return false;
            for (int k = 0; k < j; k++)
                if ((p[4 + k] & 0xFFFFFF) == item) return false;
        }
        return true;
    }
    case GPUTX_T_OE_PAYMENT:
        return P >= 4 && p[0] >= 0 && p[0] < db.n_wh && p[1] >= 0 && p[1] < OE_DIST &&
               p[2] >= 0 && p[2] < OE_CUST;
    case GPUTX_T_OE_ORDER_STATUS:
        return P >= 3 && p[0] >= 0 && p[0] < db.n_wh && p[1] >= 0 && p[1] < OE_DIST &&
               p[2] >= 0 && p[2] < OE_CUST;
    }
    return false;
}

// ---------------------------------------------------------------------------
// basic operations (Section 4.1): obj, class and root key of each
// ---------------------------------------------------------------------------
// Returns the number of operations written (<= MAX_OPS).  The root key is the
// primary key of the schema's root relation (Section 5.1): the branch, the
// subscriber, the warehouse.
__device__ __forceinline__ int access_set(const DevDB &db, int32_t type, const int64_t *p, int mode,
                                          uint32_t *obj, uint8_t *cls, uint32_t *root)
{
    const uint8_t blind = (mode == GPUTX_CONFLICT_ADD) ? CLS_A : CLS_W;
    int k = 0;
    switch (type) {
    case GPUTX_T_DC_DEBIT_CREDIT: {
        // The transaction writes its account, teller and branch balances.
        // With reads and writes only, every pair of debit-credit transactions
        // that conflicts on an account or a teller also conflicts on the
        // branch above it (both write it), so the branch -- the root key of
        // Section 5.1 -- stands for all three: same conflict relation, same
        // depths, one operation.  With ADD, teller and branch increments
        // commute with each other and no procedure reads them, so only the
        // account orders transactions.
        const int64_t a = p[0];
        const uint32_t b = db.div_br.div((uint32_t)a);
        if (mode == GPUTX_CONFLICT_ADD) {
            obj[0] = db.o_acc + (uint32_t)a; cls[0] = CLS_W; root[0] = b;
        } else {
            obj[0] = db.o_br + b; cls[0] = CLS_W; root[0] = b;
        }
        (void)blind;
        return 1;
    }
    case GPUTX_T_SUB_GET_SUBSCRIBER:
    case GPUTX_T_SUB_GET_ACCESS:
    case GPUTX_T_SUB_GET_NEW_DEST:
        obj[0] = db.o_sub + (uint32_t)p[0]; cls[0] = CLS_R; root[0] = (uint32_t)p[0];
        return 1;
    case GPUTX_T_SUB_UPDATE_LOCATION:
    case GPUTX_T_SUB_UPDATE_FACILITY:
    case GPUTX_T_SUB_INSERT_CF:
    case GPUTX_T_SUB_DELETE_CF:
        obj[0] = db.o_sub + (uint32_t)p[0]; cls[0] = CLS_W; root[0] = (uint32_t)p[0];
        return 1;
    case GPUTX_T_OE_NEW_ORDER: {
        uint32_t w = (uint32_t)p[0], d = w * OE_DIST + (uint32_t)p[1];
        uint32_t c = d * OE_CUST + (uint32_t)p[2];
        obj[k] = db.o_dnext + d; cls[k] = CLS_W; root[k] = w; k++;
        obj[k] = db.o_clast + c; cls[k] = CLS_W; root[k] = w; k++;
        int cnt = (int)p[3];
        for (int j = 0; j < cnt; j++) {
            int64_t line = p[4 + j];
            int64_t item = line & 0xFFFFFF, sw = (line >> 24) & 0xFFFF;
            if (item >= db.n_items) continue;
            obj[k] = db.o_stock + (uint32_t)(sw * db.n_items + item); cls[k] = CLS_W;
            root[k] = (uint32_t)sw; k++;
        }
        return k;
    }
    case GPUTX_T_OE_PAYMENT: {
        uint32_t w = (uint32_t)p[0], d = w * OE_DIST + (uint32_t)p[1];
        uint32_t c = d * OE_CUST + (uint32_t)p[2];
        obj[0] = db.o_wytd + w;  cls[0] = blind; root[0] = w;
        obj[1] = db.o_dytd + d;  cls[1] = blind; root[1] = w;
        obj[2] = db.o_cpay + c;  cls[2] = CLS_W; root[2] = w;
        return 3;
    }
    case GPUTX_T_OE_ORDER_STATUS: {
        uint32_t w = (uint32_t)p[0], d = w * OE_DIST + (uint32_t)p[1];
        uint32_t c = d * OE_CUST + (uint32_t)p[2];
        obj[0] = db.o_cpay + c;  cls[0] = CLS_R; root[0] = w;
        obj[1] = db.o_clast + c; cls[1] = CLS_R; root[1] = w;
        return 2;
    }
    }
    return 0;
}

// number of operations without materialising them
__device__ __forceinline__ int op_count(const DevDB &db, int32_t type, const int64_t *p)
{
    switch (type) {
    case GPUTX_T_DC_DEBIT_CREDIT: return 1;
    case GPUTX_T_OE_NEW_ORDER: {
        int k = 2, cnt = (int)p[3];
        for (int j = 0; j < cnt; j++) k += ((p[4 + j] & 0xFFFFFF) < db.n_items);
        return k;
    }
    case GPUTX_T_OE_PAYMENT: return 3;
    case GPUTX_T_OE_ORDER_STATUS: return 2;
    default: return 1;
    }
}

// ---------------------------------------------------------------------------
// hash index probes (linear probing on a multiplicative hash)
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint64_t hmix(unsigned long long k)
{
    k ^= k >> 33;
    k *= 0xff51afd7ed558ccdull;
    k ^= k >> 33;
    k *= 0xc4ceb9fe1a85ec53ull;
    k ^= k >> 33;
    return k;
}

// returns the row slot or -1
__device__ __forceinline__ int64_t hash_find(const HashIndex &h, unsigned long long key)
{
    uint64_t i = hmix(key) & h.mask;
    for (uint64_t probe = 0; probe <= h.mask; probe++, i = (i + 1) & h.mask) {
        unsigned long long k = __ldcg(&h.keys[i]);
        if (k == key) return (int64_t)__ldcg(&h.rows[i]);
        if (k == HKEY_EMPTY) return -1;
    }
    return -1;
}

// Inserts key -> row.  The caller guarantees no concurrent operation on the
// same key (its transactions conflict on the root item, so they never run at
// the same time); other keys may be inserted concurrently, hence the CAS.
// Reuses the first tombstone on the probe path.  Returns false when full.
__device__ __forceinline__ bool hash_insert(const HashIndex &h, unsigned long long key, uint32_t row)
{
    // an empty home slot is the one the probe below would pick: one round trip
    const uint64_t home = hmix(key) & h.mask;
    if (atomicCAS(&h.keys[home], HKEY_EMPTY, key) == HKEY_EMPTY) {
        __stcg(&h.rows[home], row);
        return true;
    }
    for (int attempt = 0; attempt < 64; attempt++) {
        uint64_t i = hmix(key) & h.mask;
        int64_t tomb = -1;
        uint64_t slot = ~0ull;
        for (uint64_t probe = 0; probe <= h.mask; probe++, i = (i + 1) & h.mask) {
            unsigned long long k = __ldcg(&h.keys[i]);
            if (k == HKEY_TOMB) { if (tomb < 0) tomb = (int64_t)i; continue; }
            if (k == HKEY_EMPTY) { slot = tomb >= 0 ? (uint64_t)tomb : i; break; }
        }
        if (slot == ~0ull) {
            if (tomb < 0) return false;
            slot = (uint64_t)tomb;
        }
        unsigned long long expect = __ldcg(&h.keys[slot]);
        if (expect != HKEY_EMPTY && expect != HKEY_TOMB) continue;   // raced
        if (atomicCAS(&h.keys[slot], expect, key) == expect) {
            // readers of this key run in a later level / after this
            // transaction's release, so the row may follow the key
            __stcg(&h.rows[slot], row);
            return true;
        }
    }
    return false;
}

__device__ __forceinline__ bool hash_erase(const HashIndex &h, unsigned long long key)
{
    uint64_t i = hmix(key) & h.mask;
    for (uint64_t probe = 0; probe <= h.mask; probe++, i = (i + 1) & h.mask) {
        unsigned long long k = __ldcg(&h.keys[i]);
        if (k == key) { atomicExch(&h.keys[i], HKEY_TOMB); return true; }
        if (k == HKEY_EMPTY) return false;
    }
    return false;
}

__device__ __forceinline__ unsigned long long ai_key(int64_t s, int64_t t) { return (unsigned long long)(s * 4 + (t - 1)); }
__device__ __forceinline__ unsigned long long sf_key(int64_t s, int64_t t) { return (unsigned long long)(s * 4 + (t - 1)); }
__device__ __forceinline__ unsigned long long cf_key(int64_t s, int64_t t, int64_t st)
{
    return (unsigned long long)((s * 4 + (t - 1)) * 3 + st / 8);
}
__device__ __forceinline__ unsigned long long ord_key(int64_t dist, int64_t o_id)
{
    return ((unsigned long long)dist << 32) | (unsigned long long)(uint32_t)o_id;
}

__device__ __forceinline__ int64_t pack2(int32_t lo, int32_t hi)
{
    return (int64_t)((unsigned long long)(uint32_t)lo | ((unsigned long long)(uint32_t)hi << 32));
}

// A transaction as the executors see it: its signature (from the bulk, or
// from the records gathered into execution order) and where its results go.
struct TxnView {
    const int64_t *p;     // parameter list
    int64_t p0, p1;       // its first two entries, loaded with the view
    int64_t ts;
    int64_t hist_slot;    // history row of a debit-credit transaction
    uint32_t t;           // index in the bulk: outputs, status, insert slots
    int32_t type;
};

// signature at position pos of the gathered execution-order records; the
// loads are issued here, so building a view early hides their latency
// (a debug build turns a position or index outside the bulk into a view of
// type -1, which no procedure executes)
__device__ __forceinline__ TxnView view_at(const DevBulk &b, uint32_t pos, int64_t hist_base)
{
    TxnView v;
    bool bad = !dbg_in(pos, b.n, b.err);
    if (kDebug && bad) pos = 0;
    v.p = b.rec_params + (int64_t)pos * b.P;
    v.p0 = __ldg(&v.p[0]);
    v.p1 = b.P > 1 ? __ldg(&v.p[1]) : 0;
    v.ts = __ldg(&b.rec_ts[pos]);
    v.type = __ldg(&b.rec_type[pos]);
    v.t = __ldg(&b.rec_t[pos]);
    if (kDebug && !dbg_in(v.t, b.n, b.err)) {
        bad = true;
        v.t = 0;
    }
    if (kDebug && bad) v.type = -1;
    v.hist_slot = hist_base + (b.slot_hist ? (int64_t)__ldg(&b.slot_hist[v.t]) : (int64_t)pos);
    return v;
}

// signature of transaction t straight from the bulk (timestamp order)
__device__ __forceinline__ TxnView view_of(const DevBulk &b, uint32_t t, int64_t hist_base)
{
    TxnView v;
    const bool bad = !dbg_in(t, b.n, b.err);
    if (kDebug && bad) t = 0;
    v.p = b.params + (int64_t)t * b.P;
    v.p0 = __ldg(&v.p[0]);
    v.p1 = b.P > 1 ? __ldg(&v.p[1]) : 0;
    v.ts = __ldg(&b.ts[t]);
    v.type = (kDebug && bad) ? -1 : __ldg(&b.type[t]);
    v.t = t;
    v.hist_slot = hist_base + (b.slot_hist ? (int64_t)__ldg(&b.slot_hist[t]) : (int64_t)t);
    return v;
}

// L1 prefetch of the record lines at position pos (no data dependency)
__device__ __forceinline__ void prefetch_record_l1(const DevBulk &b, uint32_t pos)
{
    asm volatile("prefetch.global.L1 [%0];" ::"l"(b.rec_params + (int64_t)pos * b.P));
    asm volatile("prefetch.global.L1 [%0];" ::"l"(b.rec_ts + pos));
    asm volatile("prefetch.global.L1 [%0];" ::"l"(b.rec_type + pos));
    asm volatile("prefetch.global.L1 [%0];" ::"l"(b.rec_t + pos));
}

__device__ __forceinline__ void prefetch_txn(const DevDB &db, const TxnView &v)
{
    const int64_t *p = v.p;
    switch (v.type) {
    case GPUTX_T_DC_DEBIT_CREDIT: {
        const uint32_t a = (uint32_t)v.p0;
        prefetch_l2(&db.acc_bal[a]);
        prefetch_l2(&db.tel_bal[db.div_tel.div(a)]);
        prefetch_l2(&db.br_bal[db.div_br.div(a)]);
        break;
    }
    case GPUTX_T_SUB_GET_SUBSCRIBER:
    case GPUTX_T_SUB_UPDATE_LOCATION:
    case GPUTX_T_SUB_UPDATE_FACILITY:
        prefetch_l2(db.sub_rows + v.p0 * SUB_FIELDS);
        break;
    case GPUTX_T_OE_PAYMENT: {
        const int64_t w = __ldg(&p[0]), d = w * OE_DIST + __ldg(&p[1]), c = d * OE_CUST + __ldg(&p[2]);
        prefetch_l2(&db.c_balance[c]);
        prefetch_l2(&db.c_ytd[c]);
        prefetch_l2(&db.c_payment_cnt[c]);
        break;
    }
    case GPUTX_T_OE_NEW_ORDER: {
        const int64_t w = __ldg(&p[0]), d = w * OE_DIST + __ldg(&p[1]);
        prefetch_l2(&db.d_next_o_id[d]);
        const int cnt = (int)__ldg(&p[3]);
        for (int j = 0; j < cnt && j < OE_MAX_LINES; j++) {
            const int64_t line = __ldg(&p[4 + j]);
            const int64_t item = line & 0xFFFFFF, sw = (line >> 24) & 0xFFFF;
            if (item < db.n_items) prefetch_l2(&db.s_quantity[sw * db.n_items + item]);
        }
        break;
    }
    default:
        break;
    }
}

// ---------------------------------------------------------------------------
// the combined procedure kernel body (Section 3.2's switch)
// ---------------------------------------------------------------------------
// How procedures read and write mutable int64 cells.
//   GlobalCells  L2 is the coherence point (ld.cg / st.cg); any strategy.
//   CachedCells  write-through cache of recently touched cells in this
//                thread's shared memory.  Only for a thread that owns its
//                cells for the whole launch -- PART, whose partition is
//                touched by no other thread -- where a cell written by one
//                transaction and read by the next stays on chip instead of
//                making an L2 round trip.
struct GlobalCells {
    __device__ __forceinline__ int64_t ld(const int64_t *p) const { return __ldcg(p); }
    __device__ __forceinline__ void st(int64_t *p, int64_t v) const { __stcg(p, v); }
};

struct CachedCells {
    static constexpr int kSlots = 16;
    unsigned long long *tag;   // kSlots entries of this thread (shared memory)
    int64_t *val;
    __device__ __forceinline__ int slot(const int64_t *p) const
    {
        return (int)((((unsigned long long)p >> 3) * 0x9E3779B97F4A7C15ull) >> 60);
    }
    __device__ __forceinline__ int64_t ld(const int64_t *p)
    {
        const int i = slot(p);
        if (tag[i] == (unsigned long long)p) return val[i];
        const int64_t x = __ldcg(p);
        tag[i] = (unsigned long long)p;
        val[i] = x;
        return x;
    }
    __device__ __forceinline__ void st(int64_t *p, int64_t x)
    {
        __stcg(p, x);
        const int i = slot(p);
        tag[i] = (unsigned long long)p;
        val[i] = x;
    }
};

// atomic_add: execute ADD-class increments with atomics (several
// transactions of one level may add to one item).  False when the history
// is full (the transaction is not executed; status 3).
template <class Cells>
__device__ __forceinline__ bool dc_state_core(const DevDB &db, const DevBulk &b, int64_t a, int64_t tl, int64_t br,
                                              int64_t delta, int64_t ts, uint32_t t, int64_t slot, bool atomic_add,
                                              Cells &cells, DcOut &o)
{
    if (!dbg_dc_rows(db, b, a, tl, br, t)) return false;
    // every load before any store: the three rows are distinct cells but the
    // compiler cannot prove it, so interleaving would serialise three L2
    // round trips
    const int64_t old_a = cells.ld(&db.acc_bal[a]);
    int64_t old_t = 0, old_b = 0;
    if (!atomic_add) {
        old_t = cells.ld(&db.tel_bal[tl]);
        old_b = cells.ld(&db.br_bal[br]);
    }
    if (slot >= db.hist_cap) {              // history full: not executed
        set_err(b.err, ERR_CAPACITY);
        b.status[t] = 3;
        return false;
    }
    // account: read-modify-write, its new value is the output
    const int64_t na = wrap_add(old_a, delta);
    cells.st(&db.acc_bal[a], na);
    if (atomic_add) {
        atomicAdd((unsigned long long *)&db.tel_bal[tl], (unsigned long long)delta);
        atomicAdd((unsigned long long *)&db.br_bal[br], (unsigned long long)delta);
    } else {
        cells.st(&db.tel_bal[tl], wrap_add(old_t, delta));
        cells.st(&db.br_bal[br], wrap_add(old_b, delta));
    }
    o.slot = slot;
    o.ts = ts;
    o.delta = delta;
    o.na = na;
    o.a = a;
    o.tl = tl;
    o.br = br;
    o.t = t;
    return true;
}

template <class Cells>
__device__ __forceinline__ bool dc_state(const DevDB &db, const DevBulk &b, const TxnView &v, bool atomic_add,
                                         Cells &cells, DcOut &o)
{
    const int64_t a = v.p0;
    return dc_state_core(db, b, a, db.div_tel.div((uint32_t)a), db.div_br.div((uint32_t)a), v.p1, v.ts, v.t,
                         v.hist_slot, atomic_add, cells, o);
}

template <class Cells>
__device__ __forceinline__ void exec_dc(const DevDB &db, const DevBulk &b, const TxnView &v, bool atomic_add,
                                        Cells &cells)
{
    DcOut o;
    if (dc_state(db, b, v, atomic_add, cells, o)) dc_finish(db, b, o);
}

// one whole transaction of a wide k-set from its packed record, reading its
// balances then writing them (atomic_add: teller and branch by atomics)
__device__ __forceinline__ void exec_dc_record(const DevDB &db, const DevBulk &b, const DcRecord &r, int64_t slot,
                                               bool atomic_add)
{
    GlobalCells g;
    DcOut o;
    if (dc_state_core(db, b, r.a, r.tl, r.br, r.delta, r.ts, r.t, slot, atomic_add, g, o)) dc_finish(db, b, o);
}

// subscriber-location procedures (stand-ins shaped like TM-1, Appendix E)
__device__ __forceinline__ void exec_sub(const DevDB &db, const DevBulk &b, const TxnView &v)
{
    const int64_t *p = v.p;
    const uint32_t t = v.t;
    const int32_t type = v.type;
    int64_t *out = b.out + (int64_t)t * b.R;
    const int64_t s = p[0];
    int32_t *row = db.sub_rows + s * SUB_FIELDS;
    int32_t st = 0;
    switch (type) {
    case GPUTX_T_SUB_GET_SUBSCRIBER: {
        const int4 *r4 = reinterpret_cast<const int4 *>(row);
#pragma unroll
        for (int q = 0; q < 4; q++) {
            int4 v = __ldcg(r4 + q);
            out[2 * q] = pack2(v.x, v.y);
            out[2 * q + 1] = pack2(v.z, v.w);
        }
        break;
    }
    case GPUTX_T_SUB_GET_ACCESS: {
        int64_t r = hash_find(db.ai_idx, ai_key(s, p[1]));
        if (r < 0) { st = 1; break; }
        if (!dbg_in(r, db.child_cap, b.err)) { st = 3; break; }
        const int4 v = __ldcg(reinterpret_cast<const int4 *>(db.ai_data + r * 4));
        out[0] = pack2(v.x, v.y);
        out[1] = pack2(v.z, v.w);
        break;
    }
    case GPUTX_T_SUB_GET_NEW_DEST: {
        int64_t r = hash_find(db.sf_idx, sf_key(s, p[1]));
        if (r >= 0 && !dbg_in(r, db.child_cap, b.err)) { st = 3; break; }
        if (r < 0 || __ldcg(&db.sf_active[r]) != 1) { st = 1; break; }
        int cnt = 0;
        for (int k = 0; k < 3; k++) {
            const int64_t stt = 8 * k;
            if (stt > p[2]) continue;
            int64_t c = hash_find(db.cf_idx, cf_key(s, p[1], stt));
            if (c >= 0 && !dbg_in(c, db.child_cap, b.err)) c = -1;
            if (c >= 0 && __ldcg(&db.cf_end[c]) > p[3]) out[1 + cnt++] = __ldcg(&db.cf_numberx[c]);
        }
        out[0] = cnt;
        st = cnt ? 0 : 1;
        break;
    }
    case GPUTX_T_SUB_UPDATE_LOCATION:
        out[0] = ldg_cg(&row[15]);
        stg_cg(&row[15], (int32_t)p[1]);
        break;
    case GPUTX_T_SUB_UPDATE_FACILITY: {
        int64_t r = hash_find(db.sf_idx, sf_key(s, p[1]));
        if (r < 0) { st = 1; break; }                  // read phase: abort
        if (!dbg_in(r, db.child_cap, b.err)) { st = 3; break; }
        stg_cg(&row[0], (int32_t)p[2]);
        stg_cg(&db.sf_data_a[r], (int32_t)p[3]);
        break;
    }
    case GPUTX_T_SUB_INSERT_CF: {
        if (hash_find(db.sf_idx, sf_key(s, p[1])) < 0) { st = 1; break; }
        const unsigned long long key = cf_key(s, p[1], p[2]);
        if (hash_find(db.cf_idx, key) >= 0) { st = 2; break; }
        const int64_t slot = b.base->cf + b.slot_cf[t];
        if (slot >= db.child_cap) { set_err(b.err, ERR_CAPACITY); st = 3; break; }
        db.cf_sid[slot] = (int32_t)s;
        db.cf_type[slot] = (int32_t)p[1];
        db.cf_start[slot] = (int32_t)p[2];
        stg_cg(&db.cf_end[slot], (int32_t)p[3]);
        stg_cg(&db.cf_numberx[slot], (int32_t)p[4]);
        stg_cg(&db.cf_live[slot], (uint8_t)1);
        if (!hash_insert(db.cf_idx, key, (uint32_t)slot)) { set_err(b.err, ERR_CAPACITY); st = 3; }
        break;
    }
    case GPUTX_T_SUB_DELETE_CF: {
        const unsigned long long key = cf_key(s, p[1], p[2]);
        int64_t r = hash_find(db.cf_idx, key);
        if (r < 0) { st = 1; break; }
        if (!dbg_in(r, db.child_cap, b.err)) { st = 3; break; }
        hash_erase(db.cf_idx, key);
        stg_cg(&db.cf_live[r], (uint8_t)0);
        break;
    }
    }
    b.status[t] = st;
}

// order-entry procedures (stand-ins shaped like TPC-C, Appendix E)
template <class Cells>
__device__ __forceinline__ void exec_oe(const DevDB &db, const DevBulk &b, const TxnView &v, bool atomic_add,
                                        Cells &cells)
{
    const int64_t *p = v.p;
    const uint32_t t = v.t;
    const int32_t type = v.type;
    int64_t *out = b.out + (int64_t)t * b.R;
    const int64_t w = p[0], d = w * OE_DIST + p[1], c = d * OE_CUST + p[2];
    int32_t st = 0;
    switch (type) {
    case GPUTX_T_OE_NEW_ORDER: {
        const int cnt = (int)p[3];
        for (int j = 0; j < cnt; j++)                                  // read phase
            if ((p[4 + j] & 0xFFFFFF) >= db.n_items) { st = 1; break; }
        if (st) break;
        const int64_t oslot = b.base->ord + b.slot_ord[t];
        const int64_t lslot = b.base->ol + b.slot_ol[t];
        if (oslot >= db.ord_cap || lslot + cnt > db.ol_cap) {
            set_err(b.err, ERR_CAPACITY); st = 3; break;
        }
        // the lines in chunks of kLineChunk: each chunk's loads first, then its
        // stores.  The items are distinct (the signature was validated), so no
        // store changes a row a later load reads, and a chunk's loads overlap
        // in one round trip instead of one per line (chunks bound the
        // registers the other executors of the same kernel pay for)
        constexpr int kLineChunk = 5;
        // the district's next order id and the read-only rates with the first
        // chunk's loads, in one round trip: the district's counter is stored
        // only after them
        const int64_t o_id = cells.ld(&db.d_next_o_id[d]);
        const int64_t disc = __ldg(&db.c_discount[c]), w_tax = __ldg(&db.w_tax[w]), d_tax = __ldg(&db.d_tax[d]);
        int64_t total = 0;
        for (int j0 = 0; j0 < cnt; j0 += kLineChunk) {
            int64_t price[kLineChunk], sy[kLineChunk];
            int32_t q[kLineChunk], so[kLineChunk];
#pragma unroll
            for (int u = 0; u < kLineChunk; u++) {
                if (j0 + u < cnt) {
                    const int64_t line = p[4 + j0 + u];
                    const int64_t item = line & 0xFFFFFF, sw = (line >> 24) & 0xFFFF;
                    const int64_t s = sw * db.n_items + item;
                    price[u] = __ldg(&db.i_price[item]);
                    q[u] = ldg_cg(&db.s_quantity[s]);
                    sy[u] = cells.ld(&db.s_ytd[s]);
                    so[u] = ldg_cg(&db.s_order_cnt[s]);
                }
            }
            if (j0 == 0) cells.st(&db.d_next_o_id[d], o_id + 1);
#pragma unroll
            for (int u = 0; u < kLineChunk; u++) {
                if (j0 + u < cnt) {
                    const int j = j0 + u;
                    const int64_t line = p[4 + j];
                    const int64_t item = line & 0xFFFFFF, sw = (line >> 24) & 0xFFFF;
                    const int64_t qty = (line >> 40) & 0xFF;
                    const int64_t amount = qty * price[u];
                    total += amount;
                    const int64_t s = sw * db.n_items + item;
                    const int32_t nq = (q[u] >= qty + 10) ? (int32_t)(q[u] - qty) : (int32_t)(q[u] - qty + 91);
                    stg_cg(&db.s_quantity[s], nq);
                    cells.st(&db.s_ytd[s], sy[u] + qty);
                    stg_cg(&db.s_order_cnt[s], so[u] + 1);
                    db.ol_item[lslot + j] = (int32_t)item;
                    db.ol_sw[lslot + j] = (int32_t)sw;
                    db.ol_qty[lslot + j] = (int32_t)qty;
                    stg_cg(&db.ol_amount[lslot + j], amount);
                }
            }
        }
        db.o_w[oslot] = (int32_t)w;
        db.o_d[oslot] = (int32_t)p[1];
        db.o_c[oslot] = (int32_t)p[2];
        stg_cg(&db.o_cnt[oslot], (int32_t)cnt);
        stg_cg(&db.o_id[oslot], o_id);
        stg_cg(&db.o_first[oslot], lslot);
        stg_cg(&db.o_live[oslot], (uint8_t)1);
        if (!hash_insert(db.ord_idx, ord_key(d, o_id), (uint32_t)oslot)) {
            set_err(b.err, ERR_CAPACITY); st = 3; break;
        }
        cells.st(&db.c_last_o_id[c], o_id);
        out[0] = o_id;
        out[1] = total * (10000 - disc) * (10000 + w_tax + d_tax) / 100000000;
        out[2] = cnt;
        break;
    }
    case GPUTX_T_OE_PAYMENT: {
        const int64_t amount = p[3];
        // loads first (see exec_dc), then the stores
        int64_t wy = 0, dy = 0;
        if (!atomic_add) {
            wy = cells.ld(&db.w_ytd[w]);
            dy = cells.ld(&db.d_ytd[d]);
        }
        const int64_t cb = cells.ld(&db.c_balance[c]), cy = cells.ld(&db.c_ytd[c]);
        const int64_t cn = cells.ld(&db.c_payment_cnt[c]);
        if (atomic_add) {
            atomicAdd((unsigned long long *)&db.w_ytd[w], (unsigned long long)amount);
            atomicAdd((unsigned long long *)&db.d_ytd[d], (unsigned long long)amount);
        } else {
            cells.st(&db.w_ytd[w], wrap_add(wy, amount));
            cells.st(&db.d_ytd[d], wrap_add(dy, amount));
        }
        const int64_t bal = wrap_add(cb, -amount);
        cells.st(&db.c_balance[c], bal);
        cells.st(&db.c_ytd[c], wrap_add(cy, amount));
        cells.st(&db.c_payment_cnt[c], cn + 1);
        out[0] = bal;
        break;
    }
    case GPUTX_T_OE_ORDER_STATUS: {
        const int64_t o = cells.ld(&db.c_last_o_id[c]);
        out[0] = cells.ld(&db.c_balance[c]);
        out[1] = o;
        if (o == 0) { st = 1; break; }
        const int64_t r = hash_find(db.ord_idx, ord_key(d, o));
        if (r < 0) { set_err(b.err, ERR_BOUNDS); st = 1; break; }
        if (!dbg_in(r, db.ord_cap, b.err)) { st = 1; break; }
        const int cnt = ldg_cg(&db.o_cnt[r]);
        const int64_t first = ldg_cg(&db.o_first[r]);
        if (kDebug && (cnt < 0 || !dbg_in(first, db.ol_cap - cnt + 1, b.err))) { st = 1; break; }
        int64_t sum = 0;
        for (int j = 0; j < cnt; j++) sum += ldg_cg(&db.ol_amount[first + j]);
        out[2] = cnt;
        out[3] = sum;
        break;
    }
    }
    b.status[t] = st;
}

// ---------------------------------------------------------------------------
// order-entry's line-parallel procedures: one transaction on a group of 16
// lanes (a half warp).  A new-order's lines touch distinct stock rows (its
// items are distinct), so they need no order among themselves: lane l runs
// line l, and the reads of all lines go out in one round trip instead of one
// per chunk of lines.  Lane 0 also runs the transaction's own part (district
// counter, order row, index, customer, outputs).  The results equal
// exec_oe's bit for bit.  Every lane of the group calls these together;
// `gl` is the lane's index in its group.
// ---------------------------------------------------------------------------
constexpr int kGroup = 16;

// lanes a level [lo, hi) takes: one per transaction, 16 per new-order and
// order-status, each run of groups starting on a half warp.  cut = where the
// level's types >= new-order, payment, order-status start (null: no groups)
__host__ __device__ inline uint32_t level_lane_count(uint32_t lo, uint32_t hi, const uint32_t *cut)
{
    if (!cut) return hi - lo;
    const uint32_t c8 = cut[0], c9 = cut[1], c10 = cut[2];
    const uint32_t a1 = (c8 - lo + kGroup - 1) & ~(uint32_t)(kGroup - 1);
    const uint32_t b1 = a1 + kGroup * (c9 - c8);
    const uint32_t a2 = (b1 + (c10 - c9) + kGroup - 1) & ~(uint32_t)(kGroup - 1);
    return a2 + kGroup * (hi - c10);
}

__device__ __forceinline__ uint32_t group_mask() { return 0xFFFFu << ((threadIdx.x & 31) & 16); }

__device__ __forceinline__ int64_t group_sum16(uint32_t gm, int64_t x)
{
#pragma unroll
    for (int o = 8; o > 0; o >>= 1) x += __shfl_xor_sync(gm, x, o, kGroup);
    return x;
}

// the first slot at or after `home` (in probe order) whose key satisfies
// `want` (1: equals key or empty -- a lookup; 2: empty or deleted -- an
// insert), probing 16 slots per round trip; -1 if none
__device__ __forceinline__ int64_t group_probe(uint32_t gm, uint32_t gl, const HashIndex &h, unsigned long long key,
                                               int want, unsigned long long *found)
{
    const uint64_t home = hmix(key) & h.mask;
    for (uint64_t base = 0; base <= h.mask; base += kGroup) {
        const uint64_t i = (home + base + gl) & h.mask;
        const unsigned long long k = (base + gl <= h.mask) ? __ldcg(&h.keys[i]) : key + 1;
        const bool hit = (want == 1) ? (k == key || k == HKEY_EMPTY) : (k == HKEY_EMPTY || k == HKEY_TOMB);
        const uint32_t m = __ballot_sync(gm, hit) & gm;
        if (m) {
            const int src = __ffs(m) - 1;
            *found = __shfl_sync(gm, k, src & 15, kGroup);
            return (int64_t)((home + base + (uint64_t)((src & 15))) & h.mask);
        }
    }
    return -1;
}

template <class Cells>
__device__ __forceinline__ void exec_new_order_group(const DevDB &db, const DevBulk &b, const TxnView &v, uint32_t gl,
                                                     Cells &cells)
{
    if (kDebug && (v.type != GPUTX_T_OE_NEW_ORDER || !valid_txn(db, v.type, v.p, b.P))) {
        if (gl == 0) set_err(b.err, ERR_BOUNDS);   // the group's lanes all leave here
        return;
    }
    const uint32_t gm = group_mask();
    const int64_t *p = v.p;
    const uint32_t t = v.t;
    const int64_t w = v.p0, d = w * OE_DIST + v.p1;
    const int64_t cw = __ldg(&p[2]);
    const int64_t c = d * OE_CUST + cw;
    const int cnt = (int)__ldg(&p[3]);
    const bool mine = (int)gl < cnt;
    int64_t line = 0, item = 0, sw = 0, qty = 0, s = 0;
    if (mine) {
        line = __ldg(&p[4 + gl]);
        item = line & 0xFFFFFF;
        sw = (line >> 24) & 0xFFFF;
        qty = (line >> 40) & 0xFF;
    }
    // every read in one round trip, issued before the checks below so that
    // the insert slots' loads overlap them: the district's counter and the
    // rates on lane 0, each line's item and stock row on its lane (a line
    // with an unknown item reads nothing)
    const int64_t ob = b.base->ord, lb = b.base->ol;
    const int64_t os = b.slot_ord[t], ls = b.slot_ol[t];
    int64_t o_id = 0, disc = 0, w_tax = 0, d_tax = 0, price = 0, sy = 0;
    int32_t q = 0, so = 0;
    if (gl == 0) {
        o_id = cells.ld(&db.d_next_o_id[d]);
        disc = __ldg(&db.c_discount[c]);
        w_tax = __ldg(&db.w_tax[w]);
        d_tax = __ldg(&db.d_tax[d]);
    }
    if (mine && item < db.n_items) {
        s = sw * db.n_items + item;
        price = __ldg(&db.i_price[item]);
        q = ldg_cg(&db.s_quantity[s]);
        sy = cells.ld(&db.s_ytd[s]);
        so = ldg_cg(&db.s_order_cnt[s]);
    }
    // read phase: an unknown item aborts the order (status 1, no writes)
    if (__any_sync(gm, mine && item >= db.n_items)) {
        if (gl == 0) b.status[t] = 1;
        return;
    }
    const int64_t oslot = ob + os;
    const int64_t lslot = lb + ls;
    if (oslot >= db.ord_cap || lslot + cnt > db.ol_cap) {
        if (gl == 0) {
            set_err(b.err, ERR_CAPACITY);
            b.status[t] = 3;
        }
        return;
    }
    int64_t amount = 0;
    if (mine) {
        amount = qty * price;
        const int32_t nq = (q >= qty + 10) ? (int32_t)(q - qty) : (int32_t)(q - qty + 91);
        stg_cg(&db.s_quantity[s], nq);
        cells.st(&db.s_ytd[s], sy + qty);
        stg_cg(&db.s_order_cnt[s], so + 1);
        db.ol_item[lslot + gl] = (int32_t)item;
        db.ol_sw[lslot + gl] = (int32_t)sw;
        db.ol_qty[lslot + gl] = (int32_t)qty;
        stg_cg(&db.ol_amount[lslot + gl], amount);
    }
    const int64_t total = group_sum16(gm, amount);
    o_id = __shfl_sync(gm, o_id, 0, kGroup);
    // the order index: the first free slot on the key's probe path, claimed
    // by compare-and-swap (other orders' inserts may race for it)
    const unsigned long long key = ord_key(d, o_id);
    bool inserted = false;
    {
        // an empty home slot is the slot the probe would find first: taken
        // at once, one round trip instead of two (the common case at a load
        // factor of at most one half)
        const uint64_t home = hmix(key) & db.ord_idx.mask;
        unsigned long long prev = 0;
        if (gl == 0) prev = atomicCAS(&db.ord_idx.keys[home], HKEY_EMPTY, key);
        prev = __shfl_sync(gm, prev, 0, kGroup);
        if (prev == HKEY_EMPTY) {
            if (gl == 0) __stcg(&db.ord_idx.rows[home], (uint32_t)oslot);
            inserted = true;
        }
    }
    for (int attempt = 0; attempt < 64 && !inserted; attempt++) {
        unsigned long long cur = 0;
        const int64_t slot = group_probe(gm, gl, db.ord_idx, key, 2, &cur);
        if (slot < 0) break;
        unsigned long long prev = 0;
        if (gl == 0) prev = atomicCAS(&db.ord_idx.keys[slot], cur, key);
        prev = __shfl_sync(gm, prev, 0, kGroup);
        if (prev == cur) {
            if (gl == 0) __stcg(&db.ord_idx.rows[slot], (uint32_t)oslot);
            inserted = true;
        }
    }
    if (gl == 0) {
        cells.st(&db.d_next_o_id[d], o_id + 1);
        db.o_w[oslot] = (int32_t)w;
        db.o_d[oslot] = (int32_t)v.p1;
        db.o_c[oslot] = (int32_t)cw;
        stg_cg(&db.o_cnt[oslot], (int32_t)cnt);
        stg_cg(&db.o_id[oslot], o_id);
        stg_cg(&db.o_first[oslot], lslot);
        stg_cg(&db.o_live[oslot], (uint8_t)1);
        int64_t *out = b.out + (int64_t)t * b.R;
        if (!inserted) {
            set_err(b.err, ERR_CAPACITY);
            b.status[t] = 3;
            return;
        }
        cells.st(&db.c_last_o_id[c], o_id);
        out[0] = o_id;
        out[1] = total * (10000 - disc) * (10000 + w_tax + d_tax) / 100000000;
        out[2] = cnt;
        b.status[t] = 0;
    }
}

template <class Cells>
__device__ __forceinline__ void exec_order_status_group(const DevDB &db, const DevBulk &b, const TxnView &v,
                                                        uint32_t gl, Cells &cells)
{
    if (kDebug && (v.type != GPUTX_T_OE_ORDER_STATUS || !valid_txn(db, v.type, v.p, b.P))) {
        if (gl == 0) set_err(b.err, ERR_BOUNDS);   // the group's lanes all leave here
        return;
    }
    const uint32_t gm = group_mask();
    const int64_t *p = v.p;
    const uint32_t t = v.t;
    const int64_t w = v.p0, d = w * OE_DIST + v.p1, c = d * OE_CUST + __ldg(&p[2]);
    int64_t *out = b.out + (int64_t)t * b.R;
    int64_t o = 0;
    if (gl == 0) {
        o = cells.ld(&db.c_last_o_id[c]);
        const int64_t bal = cells.ld(&db.c_balance[c]);
        out[0] = bal;
        out[1] = o;
    }
    o = __shfl_sync(gm, o, 0, kGroup);
    if (o == 0) {
        if (gl == 0) b.status[t] = 1;
        return;
    }
    unsigned long long k = 0;
    const int64_t slot = group_probe(gm, gl, db.ord_idx, ord_key(d, o), 1, &k);
    if (slot < 0 || k != ord_key(d, o)) {
        if (gl == 0) {
            set_err(b.err, ERR_BOUNDS);
            b.status[t] = 1;
        }
        return;
    }
    int64_t r = (int64_t)__ldcg(&db.ord_idx.rows[slot]);
    if (kDebug && !dbg_in(r, db.ord_cap, b.err)) r = 0;
    int cnt = ldg_cg(&db.o_cnt[r]);
    const int64_t first = ldg_cg(&db.o_first[r]);
    if (kDebug && (cnt < 0 || cnt > kGroup || !dbg_in(first, db.ol_cap - cnt + 1, b.err))) cnt = 0;
    const int64_t amt = (int)gl < cnt ? ldg_cg(&db.ol_amount[first + gl]) : 0;
    const int64_t sum = group_sum16(gm, amt);
    if (gl == 0) {
        out[2] = cnt;
        out[3] = sum;
        b.status[t] = 0;
    }
}

// L2 prefetch of the rows lane gl of a group will touch
__device__ __forceinline__ void prefetch_group(const DevDB &db, const TxnView &v, uint32_t gl)
{
    if (kDebug && v.type < 0) return;
    const int64_t *p = v.p;
    if (v.type == GPUTX_T_OE_NEW_ORDER) {
        if (gl == 0) prefetch_l2(&db.d_next_o_id[v.p0 * OE_DIST + v.p1]);
        const int cnt = (int)__ldg(&p[3]);
        if ((int)gl < cnt) {
            const int64_t line = __ldg(&p[4 + gl]);
            const int64_t item = line & 0xFFFFFF, sw = (line >> 24) & 0xFFFF;
            if (item < db.n_items) {
                prefetch_l2(&db.s_quantity[sw * db.n_items + item]);
                prefetch_l2(&db.s_ytd[sw * db.n_items + item]);
            }
        }
    } else if (gl == 0) {
        const int64_t c = (v.p0 * OE_DIST + v.p1) * OE_CUST + __ldg(&p[2]);
        prefetch_l2(&db.c_last_o_id[c]);
        prefetch_l2(&db.c_balance[c]);
    }
}

template <class Cells>
__device__ __forceinline__ void exec_txn(const DevDB &db, const DevBulk &b, const TxnView &v, bool atomic_add,
                                         Cells &cells)
{
    // a debug build re-validates the signature it was handed (the rows its
    // parameters name) before any access
    if (kDebug && v.type >= 0 && !valid_txn(db, v.type, v.p, b.P)) {
        set_err(b.err, ERR_BOUNDS);
        return;
    }
    switch (v.type) {
    case GPUTX_T_DC_DEBIT_CREDIT: exec_dc(db, b, v, atomic_add, cells); break;
    case GPUTX_T_SUB_GET_SUBSCRIBER:
    case GPUTX_T_SUB_GET_ACCESS:
    case GPUTX_T_SUB_GET_NEW_DEST:
    case GPUTX_T_SUB_UPDATE_LOCATION:
    case GPUTX_T_SUB_UPDATE_FACILITY:
    case GPUTX_T_SUB_INSERT_CF:
    case GPUTX_T_SUB_DELETE_CF: exec_sub(db, b, v); break;
    case GPUTX_T_OE_NEW_ORDER:
    case GPUTX_T_OE_PAYMENT:
    case GPUTX_T_OE_ORDER_STATUS: exec_oe(db, b, v, atomic_add, cells); break;
    }
}

__device__ __forceinline__ void exec_txn(const DevDB &db, const DevBulk &b, const TxnView &v, bool atomic_add)
{
    GlobalCells g;
    exec_txn(db, b, v, atomic_add, g);
}

}  // namespace gtx
