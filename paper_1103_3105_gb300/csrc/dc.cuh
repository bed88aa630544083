// dc.cuh -- the debit-credit procedure's parts shared by every executor
// that runs it from packed records (Section 5.1's debit-credit workload):
// what a transaction writes once its balances are updated, and the balance
// update of a level's transaction as atomics performed at L2.
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

// The state part of a transaction of one k-set, from a packed record (teller
// and branch precomputed), as three read-modify-writes performed at L2: a
// fetch-and-add on the account, whose returned old value gives the output,
// and additions on teller and branch whose results nothing reads.  Within a
// level no other transaction touches the account (Property 1 under either
// conflict model: the account is a written object in both), and integer
// additions to teller and branch commute, so this equals the read-add-write
// of dc_state_core bit for bit.  No load precedes the updates: a level's
// critical path loses the round trip of reading the balances.
__device__ __forceinline__ bool dc_state_rmw(const DevDB &db, const DevBulk &b, const DcRecord &r, int64_t slot,
                                             DcOut &o)
{
    if (slot >= db.hist_cap) {              // history full: not executed
        set_err(b.err, ERR_CAPACITY);
        b.status[r.t] = 3;
        return false;
    }
    const unsigned long long d = (unsigned long long)r.delta;
    const int64_t old_a = (int64_t)atomicAdd((unsigned long long *)&db.acc_bal[r.a], d);
    atomicAdd((unsigned long long *)&db.tel_bal[r.tl], d);
    atomicAdd((unsigned long long *)&db.br_bal[r.br], d);
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

// one whole transaction of a k-set from its packed record, by atomics
__device__ __forceinline__ void exec_dc_record_rmw(const DevDB &db, const DevBulk &b, const DcRecord &r, int64_t slot)
{
    DcOut o;
    if (dc_state_rmw(db, b, r, slot, o)) dc_finish(db, b, o);
}

}  // namespace gtx
