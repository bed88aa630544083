// relaxed.cu -- TPL with the timestamp constraint relaxed (Appendix G).
//
// Without the timestamp constraint a bulk only has to be serializable: its
// results must equal serial execution in some order.  TPL then uses plain
// spin locks (the lock of Figure 10) instead of ordered counter locks.  The
// counter-based PART of the same appendix is in analysis.cu (grouping) and
// reuses the PART executors.
#include "engine.h"
#include "procs.cuh"
#include "cta_groups.cuh"

namespace gtx {

namespace {

// Strict two-phase locking with every transaction taking its locks in
// increasing item order (no cycle of waits).  The commit ticket is taken while
// all locks are held, so two conflicting transactions' tickets follow the
// order in which they held their common item: executing the bulk serially in
// ticket order gives the same results.
struct TplRelaxedArgs {
    DevDB db;
    DevBulk b;
    BulkCtl *ctl;
    uint32_t *lock;      // one word per item (zero between bulks)
    LockSlots slot;      // item -> its word of `lock`
    uint32_t *order;     // order[ticket] = transaction
    int mode;
    uint64_t spin_limit_ns;
    bool atomic_add;
};

constexpr uint32_t kFull = 0xffffffffu;

// The lock of Figure 10, extended to shared readers, with a version in the
// word: bits 0..19 count the readers holding it, bit 20 is set while a writer
// holds it, bits 21..31 count the writers' hand-offs.  A writer swaps a word
// with neither readers nor a writer for the same word with bit 20 set; a
// reader swaps a word without a writer for the word plus one.  A writer
// releases by storing the word with bit 20 cleared and the hand-off count
// raised, a reader by subtracting one.  The word changes at every hand-off,
// so a waiter tells a lock passed along a long queue (progress: keep
// waiting) from one whose holder never lets go: the wait limit runs from the
// last change it saw.  Transactions that only read an item share its lock.
// Holding every lock while the commit ticket is taken (strict two-phase
// locking), a writer's ticket follows the tickets of the readers before it
// and precedes those of the readers after it.
constexpr uint32_t kLockWriter = 1u << 20;
constexpr uint32_t kLockReaders = kLockWriter - 1u;
constexpr uint32_t kLockHandoff = 1u << 21;

// compare-and-swap with acquire semantics: a holder sees every write its
// predecessors made before their release
__device__ __forceinline__ bool lock_swap(uint32_t *l, uint32_t v, uint32_t nv)
{
    uint32_t old;
    asm volatile("atom.acquire.gpu.global.cas.b32 %0, [%1], %2, %3;" : "=r"(old) : "l"(l), "r"(v), "r"(nv) : "memory");
    return old == v;
}

__device__ __forceinline__ uint32_t peek(const uint32_t *l)
{
    uint32_t v;
    asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(l) : "memory");
    return v;
}

__device__ __forceinline__ bool lock_open(uint32_t w, bool write)
{
    return write ? !(w & (kLockWriter | kLockReaders)) : !(w & kLockWriter);
}

__device__ __forceinline__ uint32_t lock_taken(uint32_t w, bool write)
{
    return write ? (w | kLockWriter) : w + 1u;
}

// test-and-test-and-set with exponential back-off: waiters read the word
// and try the swap only when it reads open, so a hot lock's line is not
// flooded with atomics.  Returns the word as taken (never 0), or 0 when the
// word did not change for limit_ns.
__device__ __forceinline__ uint32_t rw_lock(uint32_t *l, bool write, uint64_t limit_ns)
{
    uint32_t v = peek(l);
    if (lock_open(v, write) && lock_swap(l, v, lock_taken(v, write))) return lock_taken(v, write);
    uint64_t t0 = globaltimer();
    uint32_t ns = 32;
    while (true) {
        __nanosleep(ns);
        if (ns < 128) ns <<= 1;
        const uint32_t w = peek(l);
        if (w != v) {            // handed on since the last look: progress
            v = w;
            t0 = globaltimer();
        }
        if (lock_open(w, write)) {
            if (lock_swap(l, w, lock_taken(w, write))) return lock_taken(w, write);
        } else if (globaltimer() - t0 > limit_ns) {
            return 0;
        }
    }
}

// the release: this transaction's writes before the lock opens
__device__ __forceinline__ void rw_unlock(uint32_t *l, bool write, uint32_t held)
{
    if (write)
        asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(l), "r"((held & ~kLockWriter) + kLockHandoff)
                     : "memory");
    else
        asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(l), "r"(0xffffffffu) : "memory");
}

__global__ void tpl_relaxed_kernel(TplRelaxedArgs a)
{
    if (*(volatile uint32_t *)&a.ctl->err) return;   // validation failed: uniform, set before this launch
    const int64_t hb = a.ctl->base.hist;
    const uint32_t lane = threadIdx.x & 31;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t base0 = blockIdx.x * (int64_t)blockDim.x + (threadIdx.x & ~31u);
    // whole warps step through the bulk together (the warp combining below
    // needs every lane at the same step)
    for (int64_t t0 = base0; t0 < a.b.n; t0 += stride) {
        const int64_t t = t0 + lane;
        const bool live = t < a.b.n;
        TxnView v{};
        uint32_t items[MAX_OPS];
        uint32_t wmask = 0;   // bit j: lock j is taken to write (else shared, to read)
        int m = 0;
        if (live) {
            v = view_of(a.b, (uint32_t)t, hb);
            uint32_t obj[MAX_OPS], root[MAX_OPS];
            uint8_t cls[MAX_OPS];
            const int k = access_set(a.db, v.type, v.p, a.mode, obj, cls, root);
            for (int j = 0; j < k; j++) {
                if (cls[j] == CLS_A) continue;   // an atomic increment needs no lock
                // insertion into the sorted lock list (its modes alongside)
                int q = m++;
                while (q > 0 && items[q - 1] > obj[j]) {
                    items[q] = items[q - 1];
                    q--;
                }
                items[q] = obj[j];
                const uint32_t below = wmask & ((1u << q) - 1u);
                wmask = below | ((wmask & ~((1u << q) - 1u)) << 1) | ((cls[j] == CLS_R ? 0u : 1u) << q);
            }
            if (kDebug)
                for (int j = 0; j < m; j++)
                    if (!dbg_in(items[j], a.db.n_objects, a.b.err)) {
                        m = 0;          // no lock taken and nothing executed
                        v.type = -1;
                        break;
                    }
        }
        // Warp combining: lanes whose only lock is the same item, taken in
        // the same mode, form a group (__match_any_sync).  Its lowest lane
        // takes the lock once and draws the group's consecutive commit
        // tickets.  Writers run in lane order inside the one critical
        // section, so the ticket order is the order they ran in; readers
        // change nothing another reader sees, so they run at once.
        const bool single = live && m == 1;
        const bool write1 = single && (wmask & 1u);
        const uint32_t grp = __match_any_sync(kFull, single ? (items[0] | (write1 ? 0x80000000u : 0u))
                                                            : (0xFFFFFFE0u | lane));
        const uint32_t leader = __ffs(grp) - 1;
        if (single) {
            uint32_t held = 0;
            if (lane == leader) held = rw_lock(&a.lock[a.slot(items[0])], write1, a.spin_limit_ns);
            held = __shfl_sync(grp, held, leader);
            if (!held) {
                if (lane == leader) set_err(&a.ctl->err, ERR_TIMEOUT);
            } else {
                uint32_t tk = 0;
                if (lane == leader) tk = atomicAdd(&a.ctl->claim, (uint32_t)__popc(grp));
                tk = __shfl_sync(grp, tk, leader);
                __syncwarp(grp);   // the leader's acquire before every member's accesses
                // writers one lane at a time in lane order, readers all in one
                // pass (one call site of the procedures keeps the register count)
                for (uint32_t rest = grp; rest; rest = write1 ? (rest & (rest - 1)) : 0u) {
                    if (!write1 || lane == (uint32_t)(__ffs(rest) - 1)) {
                        exec_txn(a.db, a.b, v, a.atomic_add);
                        a.order[tk + __popc(grp & lanemask_lt())] = (uint32_t)t;
                    }
                    __syncwarp(grp);   // each writer's writes before the next one's reads
                }
                if (lane == leader) rw_unlock(&a.lock[a.slot(items[0])], write1, held);
            }
        } else if (live) {
            uint32_t held_v[MAX_OPS];
            int held = 0;
            bool ok = true;
            for (; held < m; held++) {
                held_v[held] = rw_lock(&a.lock[a.slot(items[held])], (wmask >> held) & 1u, a.spin_limit_ns);
                if (!held_v[held]) {
                    set_err(&a.ctl->err, ERR_TIMEOUT);
                    ok = false;
                    break;
                }
            }
            if (ok) {
                exec_txn(a.db, a.b, v, a.atomic_add);
                a.order[atomicAdd(&a.ctl->claim, 1u)] = (uint32_t)t;
            }
            for (int j = 0; j < held; j++) rw_unlock(&a.lock[a.slot(items[j])], (wmask >> j) & 1u, held_v[j]);
        }
    }
}

// Relaxed TPL for debit-credit-only bulks, with the lock taken once per
// CTA-wide group (cta_groups.cuh).  A CTA claims 256 consecutive
// transactions; those that need the same lock (the branch under R/W, the
// account under ADD) form a group.  Its first member takes the spin lock and
// draws the group's commit tickets in one addition; the members get them in
// thread order and run in that order inside the one critical section (the
// account updates combined, one fetch-and-add per distinct account); the
// first member unlocks once every member has its balance.  Serial execution
// in ticket order gives these results.  Teller and branch additions, history
// rows and outputs follow the unlock: no transaction of the bulk reads them
// and integer additions commute.  A hot lock is then taken once per chunk
// instead of once per warp, and far fewer threads spin on it.
__global__ void __launch_bounds__(kCtaMax) tpl_relaxed_dc_block_kernel(TplRelaxedArgs a)
{
    __shared__ uint32_t s_c, s_stop;
    __shared__ CtaGroupTables g;
    if (*(volatile uint32_t *)&a.ctl->err) return;   // validation failed: uniform, set before this launch
    const int64_t n = a.b.n;
    const int64_t hb = a.ctl->base.hist;
    const uint32_t tid = threadIdx.x;
    const bool by_account = a.mode == GPUTX_CONFLICT_ADD;
    while (true) {
        if (tid == 0) {
            s_stop = *(volatile uint32_t *)&a.ctl->err ? 1u : 0u;
            s_c = atomicAdd(&a.ctl->chunk, 1u);
        }
        cta_groups_reset(g, tid, blockDim.x);
        __syncthreads();
        const int64_t start = (int64_t)s_c * blockDim.x;
        if (s_stop || start >= n) break;
        const int64_t t = start + tid;
        const bool live = t < n;
        DcRecord r{};
        bool rows_ok = true;   // a debug build's check of the record's rows
        uint32_t item = 0, e = 0;
        if (live) {
            r.a = (uint32_t)__ldg(&a.b.params[t * a.b.P]);
            r.delta = __ldg(&a.b.params[t * a.b.P + 1]);
            r.ts = __ldg(&a.b.ts[t]);
            r.t = (uint32_t)t;
            r.tl = a.db.div_tel.div(r.a);
            r.br = a.db.div_br.div(r.a);
            rows_ok = dbg_dc_rows(a.db, a.b, r.a, r.tl, r.br, r.t);
            if (rows_ok) prefetch_l2(&a.db.acc_bal[r.a]);
            // the transaction's one lock, as its access set names it
            item = by_account ? a.db.o_acc + r.a : a.db.o_br + r.br;
            e = cta_group_join(g, item, tid);
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
            uint32_t *lock = &a.lock[a.slot(item)];
            volatile uint32_t *state = &g.state[e];
            bool ok = true;
            uint32_t held = 0;
            if (tid == c.leader) {
                held = rw_lock(lock, true, a.spin_limit_ns);
                ok = held != 0;
                if (ok) g.base[e] = atomicAdd(&a.ctl->claim, c.size);
                else set_err(&a.ctl->err, ERR_TIMEOUT);
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
            if (ok) a.order[g.base[e] + c.rank] = r.t;
            __threadfence_block();
            atomicAdd(&g.fin[e], 1u);
            if (tid == c.leader && held) {
                // every member's account update precedes the unlock
                if (!cta_wait_members(g, e, c.size, a.spin_limit_ns)) set_err(&a.ctl->err, ERR_TIMEOUT);
                rw_unlock(lock, true, held);
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
        __syncthreads();
    }
}

}  // namespace

cudaError_t launch_tpl_relaxed(gputx_bulk *b, uint32_t *order, bool atomic_add)
{
    gputx_db *db = b->db;
    if (b->n == 0) return cudaSuccess;
    TplRelaxedArgs a{};
    a.db = db->dev;
    a.b = make_dev_bulk(b, atomic_add ? GPUTX_CONFLICT_ADD : GPUTX_CONFLICT_PAPER);
    a.ctl = b->ctl;
    a.lock = db->d_done;
    a.slot = db->lock_slots;
    a.order = order;
    a.mode = atomic_add ? GPUTX_CONFLICT_ADD : GPUTX_CONFLICT_PAPER;
    a.spin_limit_ns = (uint64_t)db->cfg.spin_limit_ns;
    a.atomic_add = atomic_add;
    cudaError_t e = cudaMemsetAsync(&b->ctl->claim, 0, sizeof(uint32_t), b->stream);
    if (e) return e;
    // debit-credit-only bulks of single-lock transactions: CTA-wide lock groups
    const bool dc = db->dev.registered == (1u << GPUTX_T_DC_DEBIT_CREDIT) && !b->graph && db->uniform_k == 1;
    if (dc) {
        if ((e = cudaMemsetAsync(&b->ctl->chunk, 0, sizeof(uint32_t), b->stream))) return e;
        static int per_sm = 0;
        if (!per_sm) {
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, tpl_relaxed_dc_block_kernel, kCtaMax, 0);
            if (per_sm < 1) per_sm = 1;
        }
        int64_t grid = (int64_t)db->num_sms * per_sm;
        const int64_t chunks = (b->n + kCtaMax - 1) / kCtaMax;
        if (grid > chunks) grid = chunks;
        tpl_relaxed_dc_block_kernel<<<(unsigned)grid, kCtaMax, 0, b->stream>>>(a);
    } else {
        int64_t grid = (b->n + 255) / 256;
        if (grid > (int64_t)db->num_sms * 8) grid = (int64_t)db->num_sms * 8;
        tpl_relaxed_kernel<<<(unsigned)grid, 256, 0, b->stream>>>(a);
    }
    count_launches(1);
    e = cudaGetLastError();
    if (e) return e;
    // the versioned words return to zero: TPL's ordered counters share them
    return cudaMemsetAsync(db->d_done, 0, (size_t)db->lock_slots.lines.d * 32 * sizeof(uint32_t), b->stream);
}

}  // namespace gtx
