// exec.cu -- the three bulk execution strategies (Section 5).
//
//   K-SET (Section 5.3)  the k-sets run in order with no conflict control
//       inside a level (Property 1).  Three launch shapes:
//         wide level     one full-grid launch per level (kernel boundary =
//                        the level barrier);
//         narrow levels  one thread-block cluster (or one CTA) walks a run of
//                        consecutive narrow levels, separated by cluster (or
//                        CTA) barriers, loading the next level's signatures
//                        and prefetching its rows into L2 before each barrier
//                        (debit-credit-only bulks: exec_dc.cu);
//         persistent     a grid claims level-ordered chunks of one CTA; a
//                        chunk of level k starts once every transaction of
//                        level k-1 has finished (per-level counters).  Chunks
//                        are claimed in increasing order, so every chunk a
//                        waiting CTA depends on is held by a running CTA.
//   PART (Section 5.2)   one thread per non-empty partition runs its
//       transactions serially in timestamp order.
//   TPL (Section 5.1)    ordered counter locks: an operation whose group has
//       `ticket` earlier operations before its run waits until that many have
//       released the item's counter, then the transaction runs and every
//       operation releases (+1).  Transactions are handed out in timestamp
//       order, so the earliest unfinished one never waits: no deadlock.
// Every wait is bounded by the configured limit; on expiry the kernel sets
// ERR_TIMEOUT in the bulk's error word and returns.
#include <algorithm>
#include <vector>
#include <cooperative_groups.h>

#include "engine.h"
#include "levels.cuh"
#include "procs.cuh"
#include "cta_groups.cuh"

namespace cg = cooperative_groups;

namespace gtx {

namespace {

struct KsetArgs {
    DevDB db;
    DevBulk b;
    BulkCtl *ctl;
    const uint32_t *order, *level_off, *chunk_off, *chunk_level;
    const uint32_t *type_cut;   // per level, where new-order, payment, order-status start (or null)
    uint32_t *done;
    int64_t levels;
    uint64_t spin_limit_ns;
    bool atomic_add;
};

// waits until *p >= need; false on timeout.  The sleep between polls grows
// with the number of releases still missing (each costs at least one
// hand-off), so a waiter far back in a long chain polls rarely instead of
// flooding L2 with acquire loads.
// per_gap_ns = 0 keeps a short fixed poll (level counters, whose missing
// releases arrive together).
__device__ __forceinline__ bool wait_at_least(const uint32_t *p, uint32_t need, uint64_t limit_ns,
                                              uint32_t per_gap_ns = 0)
{
    uint32_t v = ld_acquire(p);
    if (v >= need) return true;
    const uint64_t t0 = globaltimer();
    uint32_t spins = 0;
    while (v < need) {
        const uint32_t gap = need - v;
        if (per_gap_ns && gap > 1) __nanosleep(gap > 64 ? 64 * per_gap_ns : per_gap_ns * gap);
        else if (++spins > 64) __nanosleep(32);
        if (globaltimer() - t0 > limit_ns) return false;
        v = ld_acquire(p);
    }
    return true;
}

// a bulk known to hold no two conflicting transactions (a 0-set): every
// transaction at once, straight from the bulk's signatures (timestamp order)
__global__ void __launch_bounds__(256) independent_kernel(DevDB db, DevBulk b, const BulkCtl *ctl, bool atomic_add)
{
    if (ctl->err) return;
    const int64_t hb = ctl->base.hist;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < b.n; t += (int64_t)gridDim.x * blockDim.x)
        exec_txn(db, b, view_of(b, (uint32_t)t, hb), atomic_add);
}

// The lanes of one level.  Records are sorted by (level, type) (Appendix
// D's grouping by type), so a level is a run of each type in turn.  With
// type cuts, order-entry's new-orders and order-statuses take 16 lanes each
// (their line-parallel procedures), every group starting on a half warp;
// every other transaction takes one lane.  Lane x maps to the record at
// `pos`; gl = its index in a group, or -1 for a one-lane transaction.
struct LevelLanes {
    uint32_t lo, c8, c9, c10, a1, b1, a2, v;
    __device__ __forceinline__ void make(uint32_t lo_, uint32_t hi, const uint32_t *cut)
    {
        lo = lo_;
        if (!cut) {
            c8 = c9 = c10 = hi;
            a1 = b1 = a2 = v = hi - lo;
            return;
        }
        c8 = __ldg(&cut[0]);
        c9 = __ldg(&cut[1]);
        c10 = __ldg(&cut[2]);
        a1 = (c8 - lo + kGroup - 1) & ~(uint32_t)(kGroup - 1);      // new-order groups start here
        b1 = a1 + kGroup * (c9 - c8);                               // payments
        a2 = (b1 + (c10 - c9) + kGroup - 1) & ~(uint32_t)(kGroup - 1);   // order-status groups
        v = a2 + kGroup * (hi - c10);
    }
    // false for an idle lane (alignment padding before a group run)
    __device__ __forceinline__ bool at(uint32_t x, uint32_t &pos, int &gl) const
    {
        gl = -1;
        if (x < c8 - lo) { pos = lo + x; return true; }
        if (x < a1) return false;
        if (x < b1) { pos = c8 + (x - a1) / kGroup; gl = (int)((x - a1) % kGroup); return true; }
        if (x < b1 + (c10 - c9)) { pos = c9 + (x - b1); return true; }
        if (x < a2) return false;
        pos = c10 + (x - a2) / kGroup;
        gl = (int)((x - a2) % kGroup);
        return true;
    }
};

__device__ __forceinline__ void exec_lane(const DevDB &db, const DevBulk &b, const TxnView &v, int gl,
                                          bool atomic_add)
{
    GlobalCells g;
    if (gl < 0) exec_txn(db, b, v, atomic_add, g);
    else if (v.type == GPUTX_T_OE_NEW_ORDER) exec_new_order_group(db, b, v, (uint32_t)gl, g);
    else exec_order_status_group(db, b, v, (uint32_t)gl, g);
}

// one wide level [level_off[k0], level_off[k0+1]) over the whole grid
__global__ void __launch_bounds__(256) kset_level_kernel(LevelArgs a)
{
    if (a.ctl->err) return;
    const int64_t hb = a.ctl->base.hist;
    const uint32_t lo = __ldg(&a.level_off[a.k0]), hi = __ldg(&a.level_off[a.k0 + 1]);
    if (a.rec_dc) {
        for (uint32_t pos = lo + blockIdx.x * blockDim.x + threadIdx.x; pos < hi; pos += gridDim.x * blockDim.x)
            exec_dc_record(a.db, a.b, a.rec_dc[pos], hb + pos, a.atomic_add);
        return;
    }
    LevelLanes L;
    L.make(lo, hi, a.type_cut ? a.type_cut + 3 * (int64_t)a.k0 : nullptr);
    for (uint32_t x = blockIdx.x * blockDim.x + threadIdx.x; x < L.v; x += gridDim.x * blockDim.x) {
        uint32_t pos;
        int gl;
        if (L.at(x, pos, gl)) exec_lane(a.db, a.b, view_at(a.b, pos, hb), gl, a.atomic_add);
    }
}

// a run of narrow levels [k0, k1) on one thread-block cluster (CLUSTER) or
// one CTA.  While level k executes, level k+1's records come into L1; after
// it, level k+1's rows are prefetched into L2; then the barrier.
template <bool CLUSTER, int MAXT>
__global__ void __launch_bounds__(MAXT, 1) kset_narrow_kernel(LevelArgs a)
{
    if (a.ctl->err) return;   // set by an earlier launch only: uniform here
    const int64_t hb = a.ctl->base.hist;
    uint32_t nthreads = blockDim.x, rank = threadIdx.x;
    if (CLUSTER) {
        cg::cluster_group cl = cg::this_cluster();
        nthreads = cl.num_threads();
        rank = cl.thread_rank();
    }
    const uint32_t *cut = a.type_cut;
    LevelLanes L;
    L.make(__ldg(&a.level_off[a.k0]), __ldg(&a.level_off[a.k0 + 1]), cut ? cut + 3 * (int64_t)a.k0 : nullptr);
    // this thread's first lane of the current level, loaded ahead
    TxnView v{};
    uint32_t pos;
    int gl = -1;
    bool has = rank < L.v && L.at(rank, pos, gl);
    if (has) {
        v = view_at(a.b, pos, hb);
        if (gl < 0) prefetch_txn(a.db, v);
        else prefetch_group(a.db, v, (uint32_t)gl);
    }
    for (uint32_t k = a.k0; k < a.k1; k++) {
        LevelLanes N;
        if (k + 1 < a.k1)
            N.make(__ldg(&a.level_off[k + 1]), __ldg(&a.level_off[k + 2]), cut ? cut + 3 * (int64_t)(k + 1) : nullptr);
        else N.make(0, 0, nullptr);
        // the next level's first record for this thread: loads in flight
        // while this level executes
        TxnView nv{};
        uint32_t npos;
        int ngl = -1;
        const bool has_next = rank < N.v && N.at(rank, npos, ngl);
        if (has_next) {
            nv = view_at(a.b, npos, hb);
            // the parameters this lane reads beyond the first two (a group
            // lane's order line) into L1 while this level runs
            if (a.b.P > 2) {
                asm volatile("prefetch.global.L1 [%0];" ::"l"(nv.p + 2));
                if (ngl >= 0 && 4 + ngl < a.b.P) asm volatile("prefetch.global.L1 [%0];" ::"l"(nv.p + 4 + ngl));
            }
        }
        if (has) exec_lane(a.db, a.b, v, gl, a.atomic_add);
        for (uint32_t x = rank + nthreads; x < L.v; x += nthreads) {
            uint32_t p2;
            int g2;
            if (L.at(x, p2, g2)) exec_lane(a.db, a.b, view_at(a.b, p2, hb), g2, a.atomic_add);
        }
        if (has_next) {                             // rows into L2 before the barrier
            if (ngl < 0) prefetch_txn(a.db, nv);
            else prefetch_group(a.db, nv, (uint32_t)ngl);
        }
        if (CLUSTER) cg::this_cluster().sync();   // release/acquire at cluster scope
        else __syncthreads();
        L = N;
        v = nv;
        has = has_next;
        gl = ngl;
    }
}

__global__ void kset_kernel(KsetArgs a)
{
    __shared__ uint32_t s_k, s_start, s_cnt, s_stop;
    const int64_t levels = (int64_t)a.ctl->depth + 1;   // from the analysis, on the device
    const uint32_t nchunks = a.chunk_off[levels];
    const int64_t hb = a.ctl->base.hist;
    const uint32_t *cut = a.type_cut;
    while (true) {
        if (threadIdx.x == 0) {
            uint32_t stop = *(volatile uint32_t *)&a.ctl->err ? 1u : 0u;
            const uint32_t c = stop ? nchunks : atomicAdd(&a.ctl->claim, 1u);
            if (c < nchunks) {
                // a chunk is a run of blockDim lanes of one level
                const uint32_t k = a.chunk_level[c];
                const uint32_t w = level_lane_count(a.level_off[k], a.level_off[k + 1], cut ? cut + 3 * k : nullptr);
                const uint32_t start = (c - a.chunk_off[k]) * blockDim.x;
                const uint32_t cnt = (w - start) < blockDim.x ? (w - start) : blockDim.x;
                s_k = k;
                s_start = start;
                s_cnt = cnt;
            } else {
                stop = 1;
            }
            s_stop = stop;
        }
        __syncthreads();
        if (s_stop) break;
        LevelLanes L;
        L.make(a.level_off[s_k], a.level_off[s_k + 1], cut ? cut + 3 * (int64_t)s_k : nullptr);
        // signatures are immutable: load them and prefetch the rows while the
        // previous level may still be running
        TxnView v{};
        uint32_t pos;
        int gl = -1;
        const bool mine = threadIdx.x < s_cnt && L.at(s_start + threadIdx.x, pos, gl);
        if (mine) {
            v = view_at(a.b, pos, hb);
            if (gl < 0) prefetch_txn(a.db, v);
            else prefetch_group(a.db, v, (uint32_t)gl);
        }
        if (threadIdx.x == 0 && s_k > 0) {
            const uint32_t k = s_k;
            const uint32_t prev = level_lane_count(a.level_off[k - 1], a.level_off[k], cut ? cut + 3 * (k - 1) : nullptr);
            if (!wait_at_least(&a.done[k - 1], prev, a.spin_limit_ns)) {
                set_err(&a.ctl->err, ERR_TIMEOUT);
                s_stop = 1;
            }
        }
        __syncthreads();
        if (s_stop) break;
        if (mine) {
            exec_lane(a.db, a.b, v, gl, a.atomic_add);
            __threadfence();
        }
        __syncthreads();
        if (threadIdx.x == 0) red_release_add(&a.done[s_k], s_cnt);
    }
}

__global__ void part_kernel(DevDB db, DevBulk b, const BulkCtl *ctl, const uint32_t *pkeys,
                            const uint32_t *part_start)
{
    extern __shared__ unsigned long long part_smem[];
    const uint32_t p = blockIdx.x * blockDim.x + threadIdx.x;
    // the partition's cells stay with this thread for the whole launch: a
    // write-through cache in shared memory serves its repeated reads
    CachedCells cells;
    cells.tag = part_smem + threadIdx.x * CachedCells::kSlots;
    cells.val = (int64_t *)(part_smem + (blockDim.x + threadIdx.x) * CachedCells::kSlots);
    for (int i = 0; i < CachedCells::kSlots; i++) cells.tag[i] = 0;
    if (p >= ctl->npart || ctl->err) return;
    const int64_t hb = ctl->base.hist;
    const uint32_t n = (uint32_t)b.n;
    uint32_t i = part_start[p];
    if (!dbg_in(i, n, b.err)) return;
    const uint32_t key = __ldg(&pkeys[i]);
    // a two-deep pipeline along the partition's timestamp order: while
    // transaction i executes, i+1's rows are already in L2 and i+2's record
    // is loading; the partition's own order is the only dependency
    TxnView v = view_at(b, i, hb);
    prefetch_txn(db, v);
    bool has1 = i + 1 < n && __ldg(&pkeys[i + 1]) == key;
    TxnView v1{};
    if (has1) {
        v1 = view_at(b, i + 1, hb);
        prefetch_txn(db, v1);
    }
    while (true) {
        const bool has2 = has1 && i + 2 < n && __ldg(&pkeys[i + 2]) == key;
        TxnView v2{};
        if (has2) v2 = view_at(b, i + 2, hb);
        exec_txn(db, b, v, false, cells);
        if (!has1) break;
        if (has2) prefetch_txn(db, v2);
        v = v1;
        v1 = v2;
        has1 = has2;
        i++;
    }
}

constexpr int kPartDcTellers = 32;   // tellers per branch the PART runner keeps on chip


constexpr uint32_t kFull = 0xffffffffu;

// sum of `x` over the lanes of `m` (this lane's group) and its inclusive
// prefix up to this lane, in lane order; every lane of the warp calls it
__device__ __forceinline__ void group_sum(uint32_t m, int64_t x, int64_t &pre, int64_t &tot)
{
    const uint32_t lane = threadIdx.x & 31;
    pre = 0;
    tot = 0;
#pragma unroll 4
    for (int L = 0; L < 32; L++) {
        const int64_t d = __shfl_sync(kFull, x, L);
        if ((m >> L) & 1u) {
            tot += d;
            if ((uint32_t)L <= lane) pre += d;
        }
    }
}

// one addition per distinct cell among the lanes with `on`, by the lowest
// lane of each: `key` selects the cell; every lane of the warp calls it
__device__ __forceinline__ void warp_add(bool on, uint32_t key, unsigned long long *cell, int64_t x)
{
    const uint32_t lane = threadIdx.x & 31;
    const uint32_t m = __match_any_sync(kFull, on ? key : (0xFFFFFFE0u | lane));
    if (__any_sync(kFull, on && __popc(m) > 1)) {
        int64_t pre, tot;
        group_sum(m, x, pre, tot);
        x = tot;
    }
    if (on && lane == (uint32_t)(__ffs(m) - 1)) atomicAdd(cell, (unsigned long long)x);
}

// PART for debit-credit bulks with one warp per partition (branch).  The
// warp runs its partition's transactions in timestamp order, 32 at a time:
// each step loads 32 records and their accounts at once, and lanes that
// share an account within the step are grouped by __match_any_sync -- each
// lane's new balance is the balance loaded for the step plus the inclusive
// prefix of the group's deltas in lane (timestamp) order, and the group's
// last lane writes the account back.  That is the result of running the
// step's transactions one by one, so the partition still executes serially
// in the sense of Section 5.2 (no other partition touches its rows, no
// locks); the step only spreads the order-independent work (records,
// history rows, outputs, teller and branch sums) over the lanes.  The
// branch balance and its tellers stay on chip for the whole partition.
// __syncwarp between steps orders one step's account stores before the
// next step's loads.
__global__ void __launch_bounds__(256) part_dc_warp_kernel(DevDB db, DevBulk b, const BulkCtl *ctl,
                                                           const DcRecord *rec, const uint32_t *pkeys,
                                                           const uint32_t *part_start)
{
    __shared__ int64_t s_tel[8][32];   // this warp's tellers (at most 32 per branch)
    const uint32_t lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const uint32_t p = blockIdx.x * (blockDim.x >> 5) + wib;
    if (p >= ctl->npart || ctl->err) return;   // whole warps; no block barrier below
    const int64_t hb = ctl->base.hist;
    const uint32_t lo = part_start[p], hi = part_start[p + 1];
    if (kDebug && (lo >= hi || !dbg_in(hi, b.n + 1, b.err))) {   // warp-uniform
        set_err(b.err, ERR_BOUNDS);
        return;
    }
    const uint32_t br = __ldg(&pkeys[lo]);     // partition key = branch
    const uint32_t tpb = (uint32_t)(db.acc_per_br / db.acc_per_tel);
    const uint32_t tel0 = br * tpb;
    if (kDebug && (tpb > 32 || !dbg_in((int64_t)tel0 + tpb, db.n_tel + 1, b.err))) {
        set_err(b.err, ERR_BOUNDS);
        return;
    }
    int64_t *tel = s_tel[wib];
    tel[lane] = lane < tpb ? __ldcg(&db.tel_bal[tel0 + lane]) : 0;
    int64_t bsum = 0;
    __syncwarp();
    // the first step's records and accounts on their way
    DcRecord r{};
    if (lo + lane < hi) r = rec[lo + lane];
    for (uint32_t base = lo; base < hi; base += 32) {
        const uint32_t i = base + lane;
        bool act = i < hi;
        if (kDebug && act && !(dbg_dc_rows(db, b, r.a, r.tl, r.br, r.t) && r.br == br && r.tl >= tel0 &&
                               r.tl < tel0 + tpb)) {
            set_err(b.err, ERR_BOUNDS);       // a record outside this partition's rows
            act = false;
        }
        const int64_t slot = hb + i;
        const bool run = act && slot < db.hist_cap;
        if (act && !run) {                     // history full: not executed
            set_err(b.err, ERR_CAPACITY);
            b.status[r.t] = 3;
        }
        const int64_t old = run ? __ldcg(&db.acc_bal[r.a]) : 0;
        // the next step's records, and its accounts into L2
        DcRecord nr{};
        if (base + 32 + lane < hi) {
            nr = rec[base + 32 + lane];
            if (!kDebug || nr.a < db.n_acc) prefetch_l2(&db.acc_bal[nr.a]);
        }
        const uint32_t am = __match_any_sync(kFull, run ? r.a : (0xFFFFFFE0u | lane));
        int64_t pre = r.delta, tot = r.delta;
        if (__any_sync(kFull, run && __popc(am) > 1)) group_sum(am, r.delta, pre, tot);
        if (run) {
            const int64_t na = wrap_add(old, pre);
            if (lane == 31u - (uint32_t)__clz(am)) __stcg(&db.acc_bal[r.a], wrap_add(old, tot));
            db.h_ts[slot] = r.ts;
            db.h_acc[slot] = r.a;
            db.h_tel[slot] = r.tl;
            db.h_br[slot] = br;
            db.h_delta[slot] = r.delta;
            b.out[(int64_t)r.t * b.R] = na;
            b.status[r.t] = 0;
        }
        // teller sums: one addition per teller by its group's first lane
        const uint32_t tm = __match_any_sync(kFull, run ? r.tl : (0xFFFFFFE0u | lane));
        int64_t tpre, ttot = r.delta;
        if (__any_sync(kFull, run && __popc(tm) > 1)) group_sum(tm, r.delta, tpre, ttot);
        if (run && lane == (uint32_t)(__ffs(tm) - 1)) tel[r.tl - tel0] = wrap_add(tel[r.tl - tel0], ttot);
        bsum = wrap_add(bsum, run ? r.delta : 0);
        __syncwarp();   // this step's account stores before the next step's loads
        r = nr;
    }
    // the branch: the sum of every lane's deltas
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) bsum = wrap_add(bsum, __shfl_xor_sync(kFull, bsum, o));
    if (lane == 0) __stcg(&db.br_bal[br], wrap_add(__ldcg(&db.br_bal[br]), bsum));
    if (lane < tpb) __stcg(&db.tel_bal[tel0 + lane], tel[lane]);
}

struct TplArgs {
    DevDB db;
    DevBulk b;
    BulkCtl *ctl;
    const uint32_t *lock_key, *lock_ticket, *op_off;
    uint32_t *done;
    int uniform_k;
    uint64_t spin_limit_ns;
    bool atomic_add;
    bool graph;          // fixed-capacity bulk: K slots per transaction, only the
                         // first op_count are real; padding transactions skipped
    LockSlots slot;      // item -> its counter in `done`
    int when_hot;        // debit-credit executors: -1 run, 1 run only if ctl->hot, 0 only if not
};

// whether a debit-credit TPL executor sits this bulk out (the other one runs)
__device__ __forceinline__ bool tpl_skip(const TplArgs &a)
{
    if (a.when_hot < 0) return false;
    const bool hot = *(volatile const uint32_t *)&a.ctl->hot != 0u;
    return hot != (a.when_hot == 1);
}


// releases of the lanes with `rel` (every lane of the warp calls it): lanes
// releasing the same counter are grouped by __match_any_sync and their
// lowest lane adds the group's size (warp-aggregated atomics)
__device__ __forceinline__ void warp_release(const TplArgs &a, bool rel, int64_t off, int cnt)
{
    const uint32_t lane = threadIdx.x & 31;
    const int jmax = __reduce_max_sync(kFull, rel ? (uint32_t)cnt : 0u);
    for (int j = 0; j < jmax; j++) {
        const bool r = rel && j < cnt;
        const uint32_t key = r ? a.slot(__ldg(&a.lock_key[off + j])) : (0xFFFFFFE0u | lane);
        const uint32_t m = __match_any_sync(kFull, key);
        if (r && lane == (uint32_t)(__ffs(m) - 1)) red_release_add(&a.done[key], (uint32_t)__popc(m));
    }
}

// TPL for any registered types.  Each transaction holds one ordered counter
// lock per basic operation (Section 5.1, Appendix C's counter lock with
// ticket semantics): an operation whose group has `ticket` operations before
// its run may proceed once that many have released the item's counter.
// Tickets follow the timestamp order of the group, so the earliest unfinished
// transaction never waits and no deadlock can form.
//
// A warp runs its 32 transactions in lockstep rounds.  A waiting lane polls
// all its locks not yet granted at once (relaxed loads in flight together:
// one round trip, not one per lock; a granted lock stays granted, since no
// later operation releases before this one), then only the lock furthest
// behind, again after about 500 ns per release that lock still misses.
// Every lane whose locks are all granted takes one acquire fence and runs
// its procedure: first the short ones, then the new-orders (up to four of
// them on a half warp each, one lane per order line), each phase followed by
// its releases.  Releases are warp-aggregated: lanes releasing the same
// counter in a phase are grouped by __match_any_sync and their lowest lane
// adds the group's size.  A round in which nothing is granted sleeps until
// the first lane is due to poll, so a lane about to be granted never sleeps
// behind one far back in its chain.
__global__ void __launch_bounds__(512) tpl_kernel(TplArgs a)
{
    __shared__ uint32_t s_c, s_stop;
    const int64_t n = a.b.n;
    const int64_t hb = a.ctl->base.hist;
    const uint32_t lane = threadIdx.x & 31;
    while (true) {
        if (threadIdx.x == 0) {
            s_stop = *(volatile uint32_t *)&a.ctl->err ? 1u : 0u;
            s_c = atomicAdd(&a.ctl->claim, 1u);
        }
        __syncthreads();
        const int64_t start = (int64_t)s_c * blockDim.x;
        if (s_stop || start >= n) break;
        const int64_t t = start + threadIdx.x;
        const bool live = t < n && !(a.b.n_live && t >= (int64_t)*a.b.n_live);
        int64_t off = 0;
        int cnt = 0;
        TxnView v{};
        if (live) {
            off = a.op_off ? (int64_t)a.op_off[t] : t * a.uniform_k;
            cnt = a.op_off ? (int)(a.op_off[t + 1] - a.op_off[t])
                           : (a.graph ? op_count(a.db, a.b.type[t], a.b.params + t * a.b.P) : a.uniform_k);
            v = view_of(a.b, (uint32_t)t, hb);
            prefetch_txn(a.db, v);
        }
        uint32_t granted = 0;                                  // bit j: lock j granted
        const uint32_t all = cnt >= 32 ? kFull : ((1u << cnt) - 1u);
        int blk = -1;              // the lock holding this lane back (-1: poll every lock)
        uint64_t t_next = 0;       // when this lane polls next
        bool pending = live;
        uint64_t t_prog = globaltimer();
        uint32_t idle = 0;
        while (__any_sync(kFull, pending)) {
            const uint64_t now = globaltimer();
            if (pending && granted != all && now >= t_next) {
                uint32_t gap = 0;
                if (blk >= 0) {        // only the lock that held it back last time
                    const uint32_t tk = __ldg(&a.lock_ticket[off + blk]);
                    const uint32_t c = ld_relaxed_gpu(&a.done[a.slot(__ldg(&a.lock_key[off + blk]))]);
                    if (c >= tk) {
                        granted |= 1u << blk;
                        blk = -1;
                    } else {
                        gap = tk - c;
                    }
                }
                if (blk < 0 && granted != all) {
                    uint32_t c[MAX_OPS], tk[MAX_OPS];
#pragma unroll
                    for (int j = 0; j < MAX_OPS; j++) {         // the polls, all in flight
                        tk[j] = 0;
                        c[j] = 0;
                        if (j < cnt && !((granted >> j) & 1u)) {
                            tk[j] = __ldg(&a.lock_ticket[off + j]);
                            if (tk[j]) c[j] = ld_relaxed_gpu(&a.done[a.slot(__ldg(&a.lock_key[off + j]))]);
                        }
                    }
#pragma unroll
                    for (int j = 0; j < MAX_OPS; j++) {
                        if (j < cnt && !((granted >> j) & 1u)) {
                            if (c[j] >= tk[j]) {
                                granted |= 1u << j;
                            } else if (tk[j] - c[j] > gap) {   // the furthest behind
                                gap = tk[j] - c[j];
                                blk = j;
                            }
                        }
                    }
                }
                // a lock missing `gap` releases needs at least that many
                // hand-offs: poll again after about that long
                if (granted != all) t_next = now + (gap > 1 ? (uint64_t)(gap > 64 ? 64 : gap) * 500 : 0);
            }
            bool ready = pending && granted == all;
            bool failed = false;
            if (!__any_sync(kFull, ready)) {
                if (now - t_prog > a.spin_limit_ns) {
                    // nothing granted within the limit: give up, but release,
                    // so no later waiter hangs on these counters
                    failed = ready = pending;
                    if (failed) set_err(&a.ctl->err, ERR_TIMEOUT);
                } else {
                    // sleep until the first lane is due to poll
                    const uint32_t due = (pending && t_next > now) ? (uint32_t)min(t_next - now, (uint64_t)32000)
                                                                    : (pending ? 0u : kFull);
                    const uint32_t d = __reduce_min_sync(kFull, due);
                    if (d > 0 && d != kFull) __nanosleep(d);
                    else if (++idle > 64) __nanosleep(32);
                    continue;
                }
            }
            if (ready && !failed) fence_acquire_gpu();   // with the polls: acquire of every granted lock
            // The round runs in two phases, each ending with its releases, so
            // a short transaction's hand-off never waits for a new-order of
            // the same warp.  Phase 1: every other granted transaction, one
            // lane each (and the releases of timed-out ones).
            const bool no = ready && !failed && v.type == GPUTX_T_OE_NEW_ORDER;
            const bool r1 = ready && !no;
            if (r1 && !failed) exec_txn(a.db, a.b, v, a.atomic_add);
            __syncwarp();   // every lane's writes precede the releases of its phase
            warp_release(a, r1, off, cnt);
            // Phase 2: the granted new-orders.  Up to four run on a half warp
            // each, two at a time (the line-parallel procedure: one lane per
            // order line, as in the K-SET runners); more run one lane each.
            uint32_t m2 = __ballot_sync(kFull, no);
            if (m2 && __popc(m2) <= 4) {
                while (m2) {
                    const int l0 = __ffs(m2) - 1;
                    m2 &= m2 - 1;
                    const int l1 = m2 ? __ffs(m2) - 1 : -1;
                    if (l1 >= 0) m2 &= m2 - 1;
                    const int src = (lane < 16 || l1 < 0) ? l0 : l1;
                    TxnView g;
                    g.p = (const int64_t *)__shfl_sync(kFull, (unsigned long long)v.p, src);
                    g.p0 = __shfl_sync(kFull, v.p0, src);
                    g.p1 = __shfl_sync(kFull, v.p1, src);
                    g.ts = __shfl_sync(kFull, v.ts, src);
                    g.hist_slot = __shfl_sync(kFull, v.hist_slot, src);
                    g.t = __shfl_sync(kFull, v.t, src);
                    g.type = __shfl_sync(kFull, v.type, src);
                    if (lane < 16 || l1 >= 0) {
                        GlobalCells gc;
                        exec_new_order_group(a.db, a.b, g, lane & 15u, gc);
                    }
                }
            } else if (no) {
                exec_txn(a.db, a.b, v, a.atomic_add);
            }
            __syncwarp();
            warp_release(a, no, off, cnt);
            pending = pending && !ready;
            t_prog = globaltimer();
            idle = 0;
        }
        __syncthreads();
    }
}

// TPL for debit-credit-only bulks.  A transaction's one lock is its root
// key's counter (the branch under R/W, the account under ADD).  Once it is
// granted, the account takes a fetch-and-add at L2 (its old value gives the
// output) and the lock is released; the teller and branch additions, the
// history row and the outputs follow the release.  No transaction of the
// bulk reads a teller or branch balance or the history, and integer
// additions commute, so the next holder may run before those land: the
// hand-off waits for one atomic round trip instead of a load, the stores and
// their acknowledgement.
//
// A warp works on 32 consecutive transactions and resolves the conflicts
// among them itself.  __match_any_sync groups the lanes that need the same
// counter.  Every operation here is a write and the warp holds consecutive
// timestamps, so no other transaction's operation on that item lies between
// two lanes of a group: their tickets are consecutive, and the whole group
// runs, in lane (timestamp) order, as soon as its first lane's ticket is
// granted.  Only that lane polls the counter, and one addition of the group's
// size releases it.  Within a group, lanes on the same account combine their
// deltas (warp-aggregated atomics): one fetch-and-add of the sum, each lane's
// new balance = the old value plus the inclusive prefix of the deltas in lane
// order -- the serial result bit for bit.  Teller and branch additions are
// aggregated the same way.  The warp polls in lockstep rounds: each group
// polls again after about 500 ns per release it still misses, and the warp
// sleeps until the first group is due, so a group whose counter is about to
// be released never sleeps behind one far back in its chain.  A warp in
// which no two lanes share a counter needs none of this: there each lane
// waits on its own counter and runs as soon as it is granted.
__global__ void tpl_dc_kernel(TplArgs a)
{
    __shared__ uint32_t s_c, s_stop;
    if (tpl_skip(a)) return;
    const int64_t n = a.b.n;
    const int64_t hb = a.ctl->base.hist;
    const uint32_t lane = threadIdx.x & 31;
    while (true) {
        if (threadIdx.x == 0) {
            s_stop = *(volatile uint32_t *)&a.ctl->err ? 1u : 0u;
            s_c = atomicAdd(&a.ctl->claim, 1u);
        }
        __syncthreads();
        const int64_t start = (int64_t)s_c * blockDim.x;
        if (s_stop || start >= n) break;
        const int64_t t = start + threadIdx.x;
        const bool live = t < n;
        DcRecord r{};
        uint32_t key = 0xFFFFFFE0u | lane, tk = 0;   // a key of its own for an idle lane
        bool rows_ok = true;   // a debug build's check of the record's rows
        if (live) {
            r.a = (uint32_t)__ldg(&a.b.params[t * a.b.P]);
            r.delta = __ldg(&a.b.params[t * a.b.P + 1]);
            r.ts = __ldg(&a.b.ts[t]);
            r.t = (uint32_t)t;
            r.tl = a.db.div_tel.div(r.a);
            r.br = a.db.div_br.div(r.a);
            rows_ok = dbg_dc_rows(a.db, a.b, r.a, r.tl, r.br, r.t);
            if (rows_ok) prefetch_l2(&a.db.acc_bal[r.a]);
            key = a.slot(a.lock_key[t]);
            tk = a.lock_ticket[t];
        }
        const uint32_t grp = __match_any_sync(kFull, key);
        if (!__any_sync(kFull, live && __popc(grp) > 1)) {
            // no two lanes of the warp share a counter: each waits on its own,
            // without the warp's lockstep rounds
            if (live) {
                const bool ok = !tk || wait_at_least(&a.done[key], tk, a.spin_limit_ns, 500);
                if (!ok) set_err(&a.ctl->err, ERR_TIMEOUT);
                DcOut o;
                const bool pend = ok && dc_account_rmw(a.db, a.b, r, hb + t, o);
                red_release_add(&a.done[key], 1u);
                if (pend) dc_finish_rmw(a.db, a.b, o);
            }
        } else {
            const uint32_t leader = __ffs(grp) - 1;
            const uint32_t need = __shfl_sync(kFull, tk, leader);   // the group's first ticket
            bool pending = live;
            uint64_t t_prog = globaltimer(), t_next = 0;   // t_next: when the group polls next
            uint32_t idle = 0, seen = 0;
            while (__any_sync(kFull, pending)) {
                const uint64_t now = globaltimer();
                uint32_t v = need ? seen : need;
                if (pending && lane == leader && need && now >= t_next) {
                    v = seen = ld_acquire(&a.done[key]);
                    // missing `gap` releases take at least that many hand-offs
                    const uint32_t gap = v < need ? need - v : 0;
                    t_next = now + (gap > 1 ? (uint64_t)(gap > 64 ? 64 : gap) * 500 : 0);
                }
                v = __shfl_sync(kFull, v, leader);
                bool ready = pending && v >= need;
                bool failed = false;
                if (!__any_sync(kFull, ready)) {
                    if (now - t_prog > a.spin_limit_ns) {
                        // no group made progress within the limit: give up, but
                        // release, so no later waiter hangs on these counters
                        failed = ready = pending;
                        if (failed && lane == leader) set_err(&a.ctl->err, ERR_TIMEOUT);
                    } else {
                        // sleep until the first group is due to poll
                        const uint32_t due = (pending && lane == leader)
                                                 ? (t_next > now ? (uint32_t)min(t_next - now, (uint64_t)32000) : 0u)
                                                 : kFull;
                        const uint32_t d = __reduce_min_sync(kFull, due);
                        if (d > 0 && d != kFull) __nanosleep(d);
                        else if (++idle > 64) __nanosleep(32);
                        continue;
                    }
                }
                // the lanes of `ready` groups run now; the leader's acquire
                // orders the members' accesses after the previous holder's
                __syncwarp();
                const int64_t slot = hb + t;
                const bool run = ready && !failed && rows_ok && slot < a.db.hist_cap;
                if (ready && !failed && rows_ok && !run) {      // history full: not executed
                    set_err(a.b.err, ERR_CAPACITY);
                    a.b.status[r.t] = 3;
                }
                // the account: one fetch-and-add per distinct account
                const uint32_t am = __match_any_sync(kFull, run ? r.a : (0xFFFFFFE0u | lane));
                int64_t pre = r.delta, tot = r.delta;
                if (__any_sync(kFull, run && __popc(am) > 1)) group_sum(am, r.delta, pre, tot);
                const uint32_t al = __ffs(am) - 1;
                int64_t old = 0;
                if (run && lane == al)
                    old = (int64_t)atomicAdd((unsigned long long *)&a.db.acc_bal[r.a], (unsigned long long)tot);
                old = __shfl_sync(kFull, old, al);
                __syncwarp();
                // one release per group: every member's update precedes it
                if (ready && lane == leader) red_release_add(&a.done[key], (uint32_t)__popc(grp));
                warp_add(run, r.tl, (unsigned long long *)&a.db.tel_bal[r.tl], r.delta);
                warp_add(run, r.br, (unsigned long long *)&a.db.br_bal[r.br], r.delta);
                if (run) {
                    DcOut o;
                    o.slot = slot;
                    o.ts = r.ts;
                    o.delta = r.delta;
                    o.na = wrap_add(old, pre);
                    o.a = r.a;
                    o.tl = r.tl;
                    o.br = r.br;
                    o.t = r.t;
                    dc_finish(a.db, a.b, o);
                }
                pending = pending && !ready;
                t_prog = globaltimer();
                idle = 0;
            }
        }
        __syncthreads();
    }
}

// TPL for debit-credit-only bulks with the lock groups formed over the whole
// CTA (up to 256 consecutive transactions) instead of one warp
// (cta_groups.cuh).  The chunk holds consecutive timestamps, so a group's
// tickets are consecutive and the group runs as soon as its first member's
// ticket is granted: that member waits on the counter and publishes the grant
// in shared memory; once every member has its account balance it releases
// the counter by the group's size.  On a hot item a whole chunk's operations
// cost one hand-off through L2.
__global__ void __launch_bounds__(kCtaMax) tpl_dc_block_kernel(TplArgs a)
{
    __shared__ uint32_t s_c, s_stop;
    __shared__ CtaGroupTables g;
    if (tpl_skip(a)) return;
    const int64_t n = a.b.n;
    const int64_t hb = a.ctl->base.hist;
    const uint32_t tid = threadIdx.x;
    while (true) {
        if (tid == 0) {
            s_stop = *(volatile uint32_t *)&a.ctl->err ? 1u : 0u;
            s_c = atomicAdd(&a.ctl->claim, 1u);
        }
        cta_groups_reset(g, tid, blockDim.x);
        __syncthreads();
        const int64_t start = (int64_t)s_c * blockDim.x;
        if (s_stop || start >= n) break;
        const int64_t t = start + tid;
        const bool live = t < n;
        DcRecord r{};
        bool rows_ok = true;   // a debug build's check of the record's rows
        uint32_t key = 0, tk = 0, e = 0;
        if (live) {
            r.a = (uint32_t)__ldg(&a.b.params[t * a.b.P]);
            r.delta = __ldg(&a.b.params[t * a.b.P + 1]);
            r.ts = __ldg(&a.b.ts[t]);
            r.t = (uint32_t)t;
            r.tl = a.db.div_tel.div(r.a);
            r.br = a.db.div_br.div(r.a);
            rows_ok = dbg_dc_rows(a.db, a.b, r.a, r.tl, r.br, r.t);
            if (rows_ok) prefetch_l2(&a.db.acc_bal[r.a]);
            key = a.slot(a.lock_key[t]);
            tk = a.lock_ticket[t];
            e = cta_group_join(g, key, tid);
        }
        const int64_t slot = hb + t;
        const bool run = live && rows_ok && slot < a.db.hist_cap;
        g.delta[tid] = run ? r.delta : 0;
        g.acct[tid] = r.a;
        g.aflag[tid] = 0;
        __syncthreads();
        if (live) {
            CtaMember c;
            cta_member(g, e, tid, r.a, c);
            if (c.size == 1) {
                // the only transaction of the chunk on its counter: it waits
                // on its own and runs as soon as it is granted
                const bool ok1 = !tk || wait_at_least(&a.done[key], tk, a.spin_limit_ns, 500);
                if (!ok1) set_err(&a.ctl->err, ERR_TIMEOUT);
                DcOut o;
                const bool pend = ok1 && dc_account_rmw(a.db, a.b, r, slot, o);
                red_release_add(&a.done[key], 1u);
                if (pend) dc_finish_rmw(a.db, a.b, o);
                goto next_chunk;
            }
            volatile uint32_t *state = &g.state[e];
            bool ok = true;
            if (tid == c.leader) {
                ok = !tk || wait_at_least(&a.done[key], tk, a.spin_limit_ns, 500);
                if (!ok) set_err(&a.ctl->err, ERR_TIMEOUT);
                __threadfence_block();
                *state = ok ? 1u : 2u;
            } else if (!wait_smem(state, a.spin_limit_ns) || *state != 1u) {
                ok = false;
                if (*state == 0u) set_err(&a.ctl->err, ERR_TIMEOUT);
            }
            __threadfence_block();   // the leader's acquire before this member's accesses
            if (ok && !run && rows_ok) {           // history full: not executed
                set_err(a.b.err, ERR_CAPACITY);
                a.b.status[r.t] = 3;
            }
            int64_t old = 0;
            const bool have = ok && run &&
                              cta_account_update(g, c, tid, &a.db.acc_bal[r.a], a.spin_limit_ns, &a.ctl->err, old);
            // every member counted once its account update is done (or it gave up)
            __threadfence_block();
            atomicAdd(&g.fin[e], 1u);
            if (tid == c.leader) {
                // the group's updates precede its one release
                if (!cta_wait_members(g, e, c.size, a.spin_limit_ns)) set_err(&a.ctl->err, ERR_TIMEOUT);
                red_release_add(&a.done[key], c.size);
            }
            if (have) {
                atomicAdd((unsigned long long *)&a.db.tel_bal[r.tl], (unsigned long long)r.delta);
                atomicAdd((unsigned long long *)&a.db.br_bal[r.br], (unsigned long long)r.delta);
                DcOut o;
                o.slot = slot;
                o.ts = r.ts;
                o.delta = r.delta;
                o.na = wrap_add(old, c.pre);
                o.a = r.a;
                o.tl = r.tl;
                o.br = r.br;
                o.t = r.t;
                dc_finish(a.db, a.b, o);
            }
        }
    next_chunk:
        __syncthreads();
    }
}

}  // namespace

// size class of the launch shape a level of width w needs.  Class 0: one
// CTA of up to 64 threads (a CTA barrier).  Class 1: a cluster of up to
// 16 x 64 threads, whose level costs about what one CTA's does.  Classes 2,
// 3, 4: 16 CTAs of 128, 256, 512 threads, each class markedly dearer per
// level than the one below.
static int width_class(uint32_t w)
{
    if (w <= 64) return 0;
    int c = 1;
    while (c < 16 && (1024u << (c - 1)) < w) c++;
    return c;
}

// The end of the segment of narrow levels that starts at k within the run
// [k, run_end).  One launch executes a segment in the shape its widest level
// needs, so a long tail of narrow levels (a skewed bulk's hot chain) must not
// share a launch with a few wide ones: the segment is cut where the width
// class rises, or where a stretch of at least kMinSegment levels of a smaller
// class begins.  Shorter stretches stay in the segment, so every launch but a
// run's last covers at least kMinSegment levels and the launch overhead stays
// small against the levels' own latency.
static int64_t narrow_segment_end(const uint32_t *width, int64_t k, int64_t run_end)
{
    constexpr int64_t kMinSegment = 64;
    auto cls = [&](int64_t j) { return width_class(width[j]); };
    int cmax = cls(k);
    int64_t j = k + 1;
    while (j < run_end) {
        const int c = cls(j);
        if (c > cmax) {
            if (j - k >= kMinSegment) break;
            cmax = c;
            j++;
        } else if (c < cmax) {
            int64_t r = j;
            while (r < run_end && r - j < kMinSegment && cls(r) < cmax) r++;
            if (r - j >= kMinSegment) break;
            j = r;
        } else {
            j++;
        }
    }
    return j;
}

// clusters of this size that fit the device at once (0 = none)
int max_cluster_ok(int csize)
{
    static int cache[17] = {0};
    static bool done[17] = {false};
    if (csize < 1 || csize > 16) return 0;
    if (done[csize]) return cache[csize];
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(csize, 1, 1);
    cfg.blockDim = dim3(1024, 1, 1);
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = csize;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int n = 0;
    if (cudaOccupancyMaxActiveClusters(&n, kset_narrow_kernel<true, 1024>, &cfg) != cudaSuccess) {
        cudaGetLastError();
        n = 0;
    }
    cache[csize] = n;
    done[csize] = true;
    return n;
}

int exec_blocks_per_sm(int kind, int block)
{
    int nb = 1;
    if (kind == 0) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kset_kernel, block, 0);
    else if (kind == 2) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, tpl_dc_kernel, block, 0);
    else if (kind == 3) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, tpl_dc_block_kernel, block, 0);
    else cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, tpl_kernel, block, 0);
    return nb < 1 ? 1 : nb;
}

cudaError_t launch_kset(gputx_bulk *b, const uint32_t *order, int64_t nchunks, int block, bool atomic_add)
{
    gputx_db *db = b->db;
    if (b->n == 0 || nchunks == 0) return cudaSuccess;
    KsetArgs a{};
    a.db = db->dev;
    a.b = make_dev_bulk(b, atomic_add ? GPUTX_CONFLICT_ADD : GPUTX_CONFLICT_PAPER);
    a.ctl = b->ctl;
    a.order = order;
    a.level_off = b->sc.level_off;
    a.chunk_off = b->sc.chunk_off;
    a.chunk_level = b->sc.chunk_level;
    a.type_cut = b->sc.type_cut;
    a.done = b->sc.done;
    a.levels = 0;
    a.spin_limit_ns = (uint64_t)db->cfg.spin_limit_ns;
    a.atomic_add = atomic_add;
    cudaError_t e = cudaMemsetAsync(b->sc.done, 0, (size_t)(b->n + 1) * sizeof(uint32_t), b->stream);
    if (e) return e;
    e = cudaMemsetAsync(&b->ctl->claim, 0, sizeof(uint32_t), b->stream);
    if (e) return e;
    int64_t grid = (int64_t)db->num_sms * exec_blocks_per_sm(0, block);
    if (grid > nchunks) grid = nchunks;
    kset_kernel<<<(unsigned)grid, block, 0, b->stream>>>(a);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_kset_levels(gputx_bulk *b, const uint32_t *level_off_host, int64_t depth, int narrow_max,
                               bool atomic_add, const DcRecord *dc_records, const uint32_t *type_cut_host)
{
    gputx_db *db = b->db;
    if (b->n == 0) return cudaSuccess;
    LevelArgs a{};
    a.db = db->dev;
    a.b = make_dev_bulk(b, atomic_add ? GPUTX_CONFLICT_ADD : GPUTX_CONFLICT_PAPER);
    a.ctl = b->ctl;
    a.level_off = b->sc.level_off;
    a.rec_dc = dc_records;
    a.type_cut = (type_cut_host && !dc_records) ? b->sc.type_cut : nullptr;
    a.atomic_add = atomic_add;
    const int64_t levels = depth + 1;
    // lanes per level: the launch shapes follow them
    std::vector<uint32_t> width((size_t)levels);
    for (int64_t j = 0; j < levels; j++)
        width[j] = level_lane_count(level_off_host[j], level_off_host[j + 1], a.type_cut ? type_cut_host + 3 * j : nullptr);
    static bool attr_set = false;
    if (!attr_set) {
        cudaFuncSetAttribute(kset_narrow_kernel<true, 256>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
        cudaFuncSetAttribute(kset_narrow_kernel<true, 512>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
        cudaFuncSetAttribute(kset_narrow_kernel<true, 1024>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
        attr_set = true;
    }
    int64_t k = 0, run_end = 0;
    while (k < levels) {
        const uint32_t w = width[k];
        if ((int64_t)w > narrow_max) {
            a.k0 = (uint32_t)k;
            a.k1 = (uint32_t)k + 1;
            int64_t grid = ((int64_t)w + 255) / 256;
            const int64_t cap = (int64_t)db->num_sms * 8;
            if (grid > cap) grid = cap;
            kset_level_kernel<<<(unsigned)grid, 256, 0, b->stream>>>(a);
            count_launches(1);
            k++;
            continue;
        }
        // a run of narrow levels (found once), cut where a long stretch of
        // levels needs a launch shape of another size class (see
        // narrow_segment_end)
        if (run_end <= k) {
            run_end = k;
            while (run_end < levels && (int64_t)width[run_end] <= narrow_max) run_end++;
        }
        const int64_t e = narrow_segment_end(width.data(), k, run_end);
        uint32_t wmax = 0;
        for (int64_t j = k; j < e; j++) wmax = width[j] > wmax ? width[j] : wmax;
        a.k0 = (uint32_t)k;
        a.k1 = (uint32_t)e;
        // spread a level over up to 16 SMs, about 64 transactions each, so
        // no single SM's load/store pipeline carries a whole level
        int csize = (int)((wmax + 63) / 64);
        csize = csize < 1 ? 1 : (csize > 16 ? 16 : csize);
        while (csize > 1 && max_cluster_ok(csize) == 0) csize >>= 1;
        int threads = (int)((wmax + csize - 1) / csize);
        threads = ((threads + 31) / 32) * 32;
        threads = threads < 32 ? 32 : (threads > 1024 ? 1024 : threads);
        if (a.rec_dc) {
            // the records this bulk was gathered into decide the runner
            cudaError_t e2 = launch_narrow_dc(a, csize, threads, b->stream);
            if (e2) return e2;
        } else if (csize <= 1) {
            if (threads <= 256) kset_narrow_kernel<false, 256><<<1, threads, 0, b->stream>>>(a);
            else kset_narrow_kernel<false, 1024><<<1, threads, 0, b->stream>>>(a);
        } else {
            cudaLaunchConfig_t cfg = {};
            cfg.gridDim = dim3(csize, 1, 1);
            cfg.blockDim = dim3(threads, 1, 1);
            cfg.stream = b->stream;
            cudaLaunchAttribute attr[1];
            attr[0].id = cudaLaunchAttributeClusterDimension;
            attr[0].val.clusterDim.x = csize;
            attr[0].val.clusterDim.y = 1;
            attr[0].val.clusterDim.z = 1;
            cfg.attrs = attr;
            cfg.numAttrs = 1;
            // up to 256 threads a CTA: more registers per thread for the
            // loads in flight
            cudaError_t e2 = threads <= 256   ? cudaLaunchKernelEx(&cfg, kset_narrow_kernel<true, 256>, a)
                             : threads <= 512 ? cudaLaunchKernelEx(&cfg, kset_narrow_kernel<true, 512>, a)
                                              : cudaLaunchKernelEx(&cfg, kset_narrow_kernel<true, 1024>, a);
            if (e2) return e2;
        }
        count_launches(1);
        cudaError_t e3 = cudaGetLastError();
        if (e3) return e3;
        k = e;
    }
    return cudaGetLastError();
}

bool part_dc_applies(const gputx_db *db, int part_size)
{
    const DevDB &d = db->dev;
    return d.registered == (1u << GPUTX_T_DC_DEBIT_CREDIT) && part_size == 1 && d.n_br > 0 &&
           d.acc_per_br / d.acc_per_tel <= kPartDcTellers;
}

cudaError_t launch_part(gputx_bulk *b, const uint32_t *pkeys, int block, int64_t max_parts, int part_size)
{
    gputx_db *db = b->db;
    if (b->n == 0) return cudaSuccess;
    const DevBulk d = make_dev_bulk(b, GPUTX_CONFLICT_PAPER);
    // few partitions per SM: their scattered stores share one load/store
    // pipeline, so spread the possible partitions over every SM
    const int64_t parts = std::max<int64_t>(1, std::min<int64_t>(b->n, max_parts));
    int threads = (int)((parts + db->num_sms - 1) / db->num_sms);
    threads = ((threads + 7) / 8) * 8;
    threads = threads < 8 ? 8 : (threads > block ? block : threads);
    const int64_t grid = (parts + threads - 1) / threads;   // npart <= parts, read on the device
    if (part_dc_applies(db, part_size)) {
        // one warp per partition, 8 warps a CTA
        const int64_t wgrid = (parts + 7) / 8;
        part_dc_warp_kernel<<<(unsigned)wgrid, 256, 0, b->stream>>>(db->dev, d, b->ctl, b->sc.rec_dc, pkeys,
                                                                    b->sc.part_start);
    } else {
        const size_t smem = (size_t)threads * 2 * CachedCells::kSlots * sizeof(unsigned long long);
        part_kernel<<<(unsigned)grid, threads, smem, b->stream>>>(db->dev, d, b->ctl, pkeys, b->sc.part_start);
    }
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_independent(gputx_bulk *b, bool atomic_add)
{
    gputx_db *db = b->db;
    if (b->n == 0) return cudaSuccess;
    int64_t grid = (b->n + 255) / 256;
    if (grid > (int64_t)db->num_sms * 8) grid = (int64_t)db->num_sms * 8;
    independent_kernel<<<(unsigned)grid, 256, 0, b->stream>>>(
        db->dev, make_dev_bulk(b, atomic_add ? GPUTX_CONFLICT_ADD : GPUTX_CONFLICT_PAPER), b->ctl, atomic_add);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_tpl(gputx_bulk *b, int block, bool atomic_add)
{
    gputx_db *db = b->db;
    if (b->n == 0) return cudaSuccess;
    TplArgs a{};
    a.db = db->dev;
    a.b = make_dev_bulk(b, atomic_add ? GPUTX_CONFLICT_ADD : GPUTX_CONFLICT_PAPER);
    a.ctl = b->ctl;
    a.lock_key = b->sc.lock_key;
    a.lock_ticket = b->sc.lock_ticket;
    a.op_off = (db->uniform_k || b->graph) ? nullptr : b->sc.op_off;
    a.done = db->d_done;
    a.uniform_k = b->graph ? db->kmax : db->uniform_k;
    a.graph = b->graph;
    a.spin_limit_ns = (uint64_t)db->cfg.spin_limit_ns;
    a.atomic_add = atomic_add;
    cudaError_t e = cudaMemsetAsync(&b->ctl->claim, 0, sizeof(uint32_t), b->stream);
    if (e) return e;
    a.slot = db->lock_slots;
    // debit-credit-only bulks of single-lock transactions
    const bool dc = db->dev.registered == (1u << GPUTX_T_DC_DEBIT_CREDIT) && !b->graph && db->uniform_k == 1;
    // the general kernel's registers allow CTAs of up to 512 threads; the
    // CTA size changes only how many transactions a CTA claims at once
    if (!dc && block > 512) block = 512;
    int64_t grid = (int64_t)db->num_sms * exec_blocks_per_sm(dc ? 2 : 1, block);
    const int64_t chunks = (b->n + block - 1) / block;
    if (grid > chunks) grid = chunks;
    a.when_hot = -1;
    if (dc && block <= kCtaMax) {
        // CTAs of up to 256 threads can group over the whole CTA: the ticket
        // scan's flag picks that executor when a counter's chain is long
        // enough to put several of its operations in one chunk, else the
        // warp groups (both are launched; the one not picked returns at once)
        a.when_hot = 1;
        int64_t grid_b = (int64_t)db->num_sms * exec_blocks_per_sm(3, block);
        if (grid_b > chunks) grid_b = chunks;
        tpl_dc_block_kernel<<<(unsigned)grid_b, block, 0, b->stream>>>(a);
        a.when_hot = 0;
        tpl_dc_kernel<<<(unsigned)grid, block, 0, b->stream>>>(a);
        count_launches(2);
    } else {
        if (dc)
            tpl_dc_kernel<<<(unsigned)grid, block, 0, b->stream>>>(a);
        else
            tpl_kernel<<<(unsigned)grid, block, 0, b->stream>>>(a);
        count_launches(1);
    }
    return cudaGetLastError();
}

}  // namespace gtx
