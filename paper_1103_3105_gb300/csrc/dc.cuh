// dc.cuh -- the debit-credit procedure's parts shared by every executor
// that runs it from packed records (Section 5.1's debit-credit workload):
// what a transaction writes once its balances are updated, and the balance
// updates of a level's transaction as atomics performed at L2.
#pragma once
#include "common.cuh"

namespace gtx {

// A debit-credit transaction in two parts.  dc_state updates the three
// balances -- the only cells later transactions of the bulk read -- and
// returns what dc_finish writes: the history row and the outputs, which no
// transaction of the bulk reads.  An executor may therefore publish the
// state part (a barrier's release) before writing the rest.
struct DcOut {
    int64_t slot, ts, delta, na, a, tl, br;
    uint32_t t;
};

// a debug build's check of the rows a debit-credit transaction touches and of
// its index in the bulk (always true in a release build)
__device__ __forceinline__ bool dbg_dc_rows(const DevDB &db, const DevBulk &b, int64_t a, int64_t tl, int64_t br,
                                            int64_t t)
{
    if (!kDebug) return true;
    return dbg_in(a, db.n_acc, b.err) && dbg_in(tl, db.n_tel, b.err) && dbg_in(br, db.n_br, b.err) &&
           dbg_in(t, b.n, b.err);
}

__device__ __forceinline__ void dc_finish(const DevDB &db, const DevBulk &b, const DcOut &o)
{
    db.h_ts[o.slot] = o.ts;
    db.h_acc[o.slot] = o.a;
    db.h_tel[o.slot] = o.tl;
    db.h_br[o.slot] = o.br;
    db.h_delta[o.slot] = o.delta;
    b.out[(int64_t)o.t * b.R] = o.na;
    b.status[o.t] = 0;
}

// A transaction of one k-set from a packed record (teller and branch
// precomputed), with its balance updates as atomics performed at L2 and split
// by what a later level of the bulk depends on.
//
// dc_account_rmw: the fetch-and-add on the account, whose returned old value
// gives the output.  Within a level no other transaction touches the account
// (Property 1 under either conflict model: the account is a written object in
// both), so this equals the read-add-write bit for bit; a later level's
// transaction on the same account must see it, so it precedes the level
// barrier's release.  No load precedes it: a level's critical path loses the
// round trip of reading the balance.
//
// dc_finish_rmw: the additions to teller and branch, the history row and the
// outputs.  No transaction of the bulk reads teller or branch balances or the
// history, and integer additions commute, so these may complete in any order
// before the launch ends: they follow the release, off the level's critical
// path.  False from dc_account_rmw when the history is full (status 3, the
// transaction is not executed).
__device__ __forceinline__ bool dc_account_rmw(const DevDB &db, const DevBulk &b, const DcRecord &r, int64_t slot,
                                               DcOut &o)
{
    if (!dbg_dc_rows(db, b, r.a, r.tl, r.br, r.t)) return false;
    if (slot >= db.hist_cap) {              // history full: not executed
        set_err(b.err, ERR_CAPACITY);
        b.status[r.t] = 3;
        return false;
    }
    const int64_t old_a = (int64_t)atomicAdd((unsigned long long *)&db.acc_bal[r.a], (unsigned long long)r.delta);
    o.slot = slot;
    o.ts = r.ts;
    o.delta = r.delta;
    o.na = wrap_add(old_a, r.delta);
    o.a = r.a;
    o.tl = r.tl;
    o.br = r.br;
    o.t = r.t;
    return true;
}

__device__ __forceinline__ void dc_finish_rmw(const DevDB &db, const DevBulk &b, const DcOut &o)
{
    atomicAdd((unsigned long long *)&db.tel_bal[o.tl], (unsigned long long)o.delta);
    atomicAdd((unsigned long long *)&db.br_bal[o.br], (unsigned long long)o.delta);
    dc_finish(db, b, o);
}

// one whole transaction of a k-set from its packed record, by atomics
__device__ __forceinline__ void exec_dc_record_rmw(const DevDB &db, const DevBulk &b, const DcRecord &r, int64_t slot)
{
    DcOut o;
    if (dc_account_rmw(db, b, r, slot, o)) dc_finish_rmw(db, b, o);
}

}  // namespace gtx
