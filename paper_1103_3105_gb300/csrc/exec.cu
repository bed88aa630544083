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
#include <cooperative_groups.h>

#include "engine.h"
#include "levels.cuh"
#include "procs.cuh"

namespace cg = cooperative_groups;

namespace gtx {

namespace {

struct KsetArgs {
    DevDB db;
    DevBulk b;
    BulkCtl *ctl;
    const uint32_t *order, *level_off, *chunk_off, *chunk_level;
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

// one wide level [level_off[k0], level_off[k0+1]) over the whole grid
__global__ void __launch_bounds__(256) kset_level_kernel(LevelArgs a)
{
    if (a.ctl->err) return;
    const int64_t hb = a.ctl->base.hist;
    const uint32_t lo = __ldg(&a.level_off[a.k0]), hi = __ldg(&a.level_off[a.k0 + 1]);
    for (uint32_t pos = lo + blockIdx.x * blockDim.x + threadIdx.x; pos < hi; pos += gridDim.x * blockDim.x) {
        if (a.rec_dc) exec_dc_record(a.db, a.b, a.rec_dc[pos], hb + pos, a.atomic_add);
        else exec_txn(a.db, a.b, view_at(a.b, pos, hb), a.atomic_add);
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
    uint32_t lo = __ldg(&a.level_off[a.k0]);
    uint32_t hi = __ldg(&a.level_off[a.k0 + 1]);
    // this thread's first transaction of the current level, loaded ahead
    TxnView v{};
    if (lo + rank < hi) {
        v = view_at(a.b, lo + rank, hb);
        prefetch_txn(a.db, v);
    }
    for (uint32_t k = a.k0; k < a.k1; k++) {
        const uint32_t nlo = hi;
        const uint32_t nhi = (k + 1 < a.k1) ? __ldg(&a.level_off[k + 2]) : nlo;
        // the next level's first signature for this thread: loads in flight
        // while this level executes
        TxnView nv{};
        const bool has_next = nlo + rank < nhi;
        if (has_next) nv = view_at(a.b, nlo + rank, hb);
        if (lo + rank < hi) exec_txn(a.db, a.b, v, a.atomic_add);
        for (uint32_t pos = lo + rank + nthreads; pos < hi; pos += nthreads)
            exec_txn(a.db, a.b, view_at(a.b, pos, hb), a.atomic_add);
        if (has_next) prefetch_txn(a.db, nv);     // rows into L2 before the barrier
        if (CLUSTER) cg::this_cluster().sync();   // release/acquire at cluster scope
        else __syncthreads();
        lo = nlo;
        hi = nhi;
        v = nv;
    }
}

__global__ void kset_kernel(KsetArgs a)
{
    __shared__ uint32_t s_k, s_start, s_cnt, s_stop;
    const int64_t levels = (int64_t)a.ctl->depth + 1;   // from the analysis, on the device
    const uint32_t nchunks = a.chunk_off[levels];
    const int64_t hb = a.ctl->base.hist;
    while (true) {
        if (threadIdx.x == 0) {
            uint32_t stop = *(volatile uint32_t *)&a.ctl->err ? 1u : 0u;
            const uint32_t c = stop ? nchunks : atomicAdd(&a.ctl->claim, 1u);
            if (c < nchunks) {
                const uint32_t k = a.chunk_level[c];
                const uint32_t lo = a.level_off[k], hi = a.level_off[k + 1];
                const uint32_t start = lo + (c - a.chunk_off[k]) * blockDim.x;
                const uint32_t cnt = (hi - start) < blockDim.x ? (hi - start) : blockDim.x;
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
        // signatures are immutable: load them and prefetch the rows while the
        // previous level may still be running
        TxnView v{};
        if (threadIdx.x < s_cnt) {
            v = view_at(a.b, s_start + threadIdx.x, hb);
            prefetch_txn(a.db, v);
        }
        if (threadIdx.x == 0 && s_k > 0) {
            const uint32_t k = s_k, lo = a.level_off[k];
            if (!wait_at_least(&a.done[k - 1], lo - a.level_off[k - 1], a.spin_limit_ns)) {
                set_err(&a.ctl->err, ERR_TIMEOUT);
                s_stop = 1;
            }
        }
        __syncthreads();
        if (s_stop) break;
        if (threadIdx.x < s_cnt) {
            exec_txn(a.db, a.b, v, a.atomic_add);
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

// PART for bulks of debit-credit transactions only, one partition per
// branch (Section 5.2 with the branch as partition key).  No transaction of
// another partition touches this branch, its tellers or its accounts, so:
//   - the branch balance lives in a register and the branch's tellers in
//     shared memory for the whole partition, and are written back once;
//   - the partition runs in batches of G transactions.  A batch issues all
//     its record and account loads at once (one memory round trip, the
//     accounts already prefetched into L2 by the batch before), then executes
//     its transactions one by one in timestamp order.  An account loaded for
//     the batch may have been written by an earlier transaction of the same
//     batch: that transaction's new balance is forwarded instead (compared in
//     registers); writes of earlier batches precede the loads in program
//     order, so the loaded values include them.
// The result equals running the partition's transactions one by one.
constexpr int kPartDcTellers = 32;   // tellers per branch held in shared memory

template <int G>
__global__ void __launch_bounds__(128) part_dc_kernel(DevDB db, DevBulk b, const BulkCtl *ctl,
                                                      const DcRecord *rec, const uint32_t *pkeys,
                                                      const uint32_t *part_start)
{
    extern __shared__ unsigned long long part_smem[];
    const uint32_t nt = blockDim.x, x = threadIdx.x;
    int64_t *tel = (int64_t *)part_smem;   // teller k of thread x at [k * nt + x]
    const uint32_t p = blockIdx.x * nt + x;
    if (p >= ctl->npart || ctl->err) return;   // no block barrier below
    const int64_t hb = ctl->base.hist;
    const uint32_t lo = part_start[p], hi = part_start[p + 1];
    const uint32_t br = __ldg(&pkeys[lo]);     // partition key = branch
    const uint32_t tpb = (uint32_t)(db.acc_per_br / db.acc_per_tel);
    const uint32_t tel0 = br * tpb;
    int64_t bbal = __ldcg(&db.br_bal[br]);
    for (uint32_t k = 0; k < tpb; k++) tel[k * nt + x] = __ldcg(&db.tel_bal[tel0 + k]);
    // the first batch's accounts into L2
    for (uint32_t k = 0; k < G && lo + k < hi; k++) prefetch_l2(&db.acc_bal[__ldg(&rec[lo + k].a)]);
    for (uint32_t base = lo; base < hi; base += G) {
        const uint32_t cnt = min((uint32_t)G, hi - base);
        DcRecord r[G];
        uint32_t an[G];
        int64_t v[G];
#pragma unroll
        for (int k = 0; k < G; k++) {
            if (k < (int)cnt) r[k] = rec[base + k];
            else r[k] = DcRecord{0, 0, 0, 0, 0, 0};
        }
#pragma unroll
        for (int k = 0; k < G; k++) an[k] = (base + G + k < hi) ? __ldg(&rec[base + G + k].a) : 0xffffffffu;
#pragma unroll
        for (int k = 0; k < G; k++) v[k] = (k < (int)cnt) ? __ldcg(&db.acc_bal[r[k].a]) : 0;
        // the next batch's accounts into L2, the records after it into L1
#pragma unroll
        for (int k = 0; k < G; k++)
            if (an[k] != 0xffffffffu) prefetch_l2(&db.acc_bal[an[k]]);
#pragma unroll
        for (int k = 0; k < G; k += 4)
            if (base + 2 * G + k < hi) asm volatile("prefetch.global.L1 [%0];" ::"l"(rec + base + 2 * G + k));
#pragma unroll
        for (int k = 0; k < G; k++) {
            if (k >= (int)cnt) break;
            // the newest balance: forwarded from an earlier transaction of
            // this batch on the same account, else the loaded value
            int64_t old = v[k];
#pragma unroll
            for (int j = 0; j < k; j++)
                if (r[j].a == r[k].a) old = v[j];
            const int64_t slot = hb + base + k;
            if (slot >= db.hist_cap) {          // history full: not executed
                set_err(b.err, ERR_CAPACITY);
                b.status[r[k].t] = 3;
                v[k] = old;                     // later forwards see the unchanged balance
                continue;
            }
            const int64_t na = wrap_add(old, r[k].delta);
            v[k] = na;                          // from here on: this transaction's new balance
            __stcg(&db.acc_bal[r[k].a], na);
            int64_t *tc = &tel[(r[k].tl - tel0) * nt + x];
            *tc = wrap_add(*tc, r[k].delta);
            bbal = wrap_add(bbal, r[k].delta);
            db.h_ts[slot] = r[k].ts;
            db.h_acc[slot] = r[k].a;
            db.h_tel[slot] = r[k].tl;
            db.h_br[slot] = br;
            db.h_delta[slot] = r[k].delta;
            b.out[(int64_t)r[k].t * b.R] = na;
            b.status[r[k].t] = 0;
        }
    }
    __stcg(&db.br_bal[br], bbal);
    for (uint32_t k = 0; k < tpb; k++) __stcg(&db.tel_bal[tel0 + k], tel[k * nt + x]);
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
};

__global__ void tpl_kernel(TplArgs a)
{
    __shared__ uint32_t s_c, s_stop;
    const int64_t n = a.b.n;
    const int64_t hb = a.ctl->base.hist;
    while (true) {
        if (threadIdx.x == 0) {
            s_stop = *(volatile uint32_t *)&a.ctl->err ? 1u : 0u;
            s_c = atomicAdd(&a.ctl->claim, 1u);
        }
        __syncthreads();
        const int64_t start = (int64_t)s_c * blockDim.x;
        if (s_stop || start >= n) break;
        const int64_t t = start + threadIdx.x;
        if (t < n && !(a.b.n_live && t >= (int64_t)*a.b.n_live)) {
            const int64_t off = a.op_off ? (int64_t)a.op_off[t] : t * a.uniform_k;
            const int cnt = a.op_off ? (int)(a.op_off[t + 1] - a.op_off[t])
                                     : (a.graph ? op_count(a.db, a.b.type[t], a.b.params + t * a.b.P)
                                                : a.uniform_k);
            const TxnView v = view_of(a.b, (uint32_t)t, hb);
            prefetch_txn(a.db, v);
            bool ok = true;
            for (int j = 0; j < cnt && ok; j++) {
                const uint32_t tk = a.lock_ticket[off + j];
                if (tk && !wait_at_least(&a.done[a.slot(a.lock_key[off + j])], tk, a.spin_limit_ns, 500)) {
                    set_err(&a.ctl->err, ERR_TIMEOUT);
                    ok = false;
                }
            }
            if (ok) exec_txn(a.db, a.b, v, a.atomic_add);
            // each release is a release: this transaction's writes before it
            for (int j = 0; j < cnt; j++) red_release_add(&a.done[a.slot(a.lock_key[off + j])], 1u);
        }
        __syncthreads();
    }
}

// TPL for debit-credit-only bulks.  A transaction's one lock is its root
// key's counter (the branch under R/W, the account under ADD).  Once it is
// granted, the account takes a fetch-and-add at L2 (dc_account_rmw: its old
// value gives the output) and the lock is released; the teller and branch
// additions, the history row and the outputs follow the release.  No
// transaction of the bulk reads a teller or branch balance or the history,
// and integer additions commute, so the next holder may run before those
// land: the hand-off waits for one atomic round trip instead of a load, the
// stores and their acknowledgement.
__global__ void tpl_dc_kernel(TplArgs a)
{
    __shared__ uint32_t s_c, s_stop;
    const int64_t n = a.b.n;
    const int64_t hb = a.ctl->base.hist;
    while (true) {
        if (threadIdx.x == 0) {
            s_stop = *(volatile uint32_t *)&a.ctl->err ? 1u : 0u;
            s_c = atomicAdd(&a.ctl->claim, 1u);
        }
        __syncthreads();
        const int64_t start = (int64_t)s_c * blockDim.x;
        if (s_stop || start >= n) break;
        const int64_t t = start + threadIdx.x;
        if (t < n) {
            DcRecord r;
            r.a = (uint32_t)__ldg(&a.b.params[t * a.b.P]);
            r.delta = __ldg(&a.b.params[t * a.b.P + 1]);
            r.ts = __ldg(&a.b.ts[t]);
            r.t = (uint32_t)t;
            r.tl = a.db.div_tel.div(r.a);
            r.br = a.db.div_br.div(r.a);
            prefetch_l2(&a.db.acc_bal[r.a]);
            const uint32_t key = a.slot(a.lock_key[t]);
            const uint32_t tk = a.lock_ticket[t];
            const bool ok = !tk || wait_at_least(&a.done[key], tk, a.spin_limit_ns, 500);
            if (!ok) set_err(&a.ctl->err, ERR_TIMEOUT);
            DcOut o;
            const bool pending = ok && dc_account_rmw(a.db, a.b, r, hb + t, o);
            red_release_add(&a.done[key], 1u);
            if (pending) dc_finish_rmw(a.db, a.b, o);
        }
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
static int64_t narrow_segment_end(const uint32_t *level_off_host, int64_t k, int64_t run_end)
{
    constexpr int64_t kMinSegment = 64;
    auto cls = [&](int64_t j) { return width_class(level_off_host[j + 1] - level_off_host[j]); };
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
                               bool atomic_add, const DcRecord *dc_records)
{
    gputx_db *db = b->db;
    if (b->n == 0) return cudaSuccess;
    LevelArgs a{};
    a.db = db->dev;
    a.b = make_dev_bulk(b, atomic_add ? GPUTX_CONFLICT_ADD : GPUTX_CONFLICT_PAPER);
    a.ctl = b->ctl;
    a.level_off = b->sc.level_off;
    a.rec_dc = dc_records;
    a.atomic_add = atomic_add;
    const int64_t levels = depth + 1;
    static bool attr_set = false;
    if (!attr_set) {
        cudaFuncSetAttribute(kset_narrow_kernel<true, 256>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
        cudaFuncSetAttribute(kset_narrow_kernel<true, 512>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
        cudaFuncSetAttribute(kset_narrow_kernel<true, 1024>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
        attr_set = true;
    }
    int64_t k = 0, run_end = 0;
    while (k < levels) {
        const uint32_t w = level_off_host[k + 1] - level_off_host[k];
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
            while (run_end < levels &&
                   (int64_t)(level_off_host[run_end + 1] - level_off_host[run_end]) <= narrow_max)
                run_end++;
        }
        const int64_t e = narrow_segment_end(level_off_host, k, run_end);
        uint32_t wmax = 0;
        for (int64_t j = k; j < e; j++) {
            const uint32_t wj = level_off_host[j + 1] - level_off_host[j];
            wmax = wj > wmax ? wj : wmax;
        }
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
        const size_t smem = (size_t)threads * kPartDcTellers * 8;
        if (smem > (48u << 10)) {
            const cudaError_t e = cudaFuncSetAttribute(part_dc_kernel<16>,
                                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e) return e;
        }
        part_dc_kernel<16><<<(unsigned)grid, threads, smem, b->stream>>>(db->dev, d, b->ctl, b->sc.rec_dc, pkeys,
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
    int64_t grid = (int64_t)db->num_sms * exec_blocks_per_sm(1, block);
    const int64_t chunks = (b->n + block - 1) / block;
    if (grid > chunks) grid = chunks;
    // debit-credit-only bulks of single-lock transactions
    if (db->dev.registered == (1u << GPUTX_T_DC_DEBIT_CREDIT) && !b->graph && db->uniform_k == 1)
        tpl_dc_kernel<<<(unsigned)grid, block, 0, b->stream>>>(a);
    else
        tpl_kernel<<<(unsigned)grid, block, 0, b->stream>>>(a);
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace gtx
