// relaxed.cu -- TPL with the timestamp constraint relaxed (Appendix G).
//
// Without the timestamp constraint a bulk only has to be serializable: its
// results must equal serial execution in some order.  TPL then uses plain
// spin locks (the lock of Figure 10) instead of ordered counter locks.  The
// counter-based PART of the same appendix is in analysis.cu (grouping) and
// reuses the PART executors.
#include "engine.h"
#include "procs.cuh"

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
    uint32_t *lock;      // one word per item, 0 = free (zero between bulks)
    LockSlots slot;      // item -> its word of `lock`
    uint32_t *order;     // order[ticket] = transaction
    int mode;
    uint64_t spin_limit_ns;
    bool atomic_add;
};

// compare-and-swap 0 -> 1 with acquire semantics: a holder sees every write
// its predecessors made before their release
__device__ __forceinline__ bool try_lock(uint32_t *l)
{
    uint32_t old;
    asm volatile("atom.acquire.gpu.global.cas.b32 %0, [%1], 0, 1;" : "=r"(old) : "l"(l) : "memory");
    return old == 0u;
}

// the release: this transaction's writes before the lock reads free
__device__ __forceinline__ void unlock(uint32_t *l)
{
    asm volatile("st.release.gpu.global.u32 [%0], 0;" ::"l"(l) : "memory");
}

__device__ __forceinline__ bool spin_lock(uint32_t *l, uint64_t limit_ns)
{
    if (try_lock(l)) return true;
    const uint64_t t0 = globaltimer();
    uint32_t ns = 32;
    while (true) {
        __nanosleep(ns);
        if (ns < 1024) ns <<= 1;
        if (try_lock(l)) return true;
        if (globaltimer() - t0 > limit_ns) return false;
    }
}

__global__ void tpl_relaxed_kernel(TplRelaxedArgs a)
{
    if (*(volatile uint32_t *)&a.ctl->err) return;   // validation failed: uniform, set before this launch
    const int64_t hb = a.ctl->base.hist;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < a.b.n;
         t += (int64_t)gridDim.x * blockDim.x) {
        const TxnView v = view_of(a.b, (uint32_t)t, hb);
        uint32_t obj[MAX_OPS], root[MAX_OPS], items[MAX_OPS];
        uint8_t cls[MAX_OPS];
        const int k = access_set(a.db, v.type, v.p, a.mode, obj, cls, root);
        int m = 0;
        for (int j = 0; j < k; j++) {
            if (cls[j] == CLS_A) continue;   // an atomic increment needs no lock
            // insertion into the sorted lock list
            int q = m++;
            while (q > 0 && items[q - 1] > obj[j]) {
                items[q] = items[q - 1];
                q--;
            }
            items[q] = obj[j];
        }
        int held = 0;
        bool ok = true;
        for (; held < m; held++)
            if (!spin_lock(&a.lock[a.slot(items[held])], a.spin_limit_ns)) {
                set_err(&a.ctl->err, ERR_TIMEOUT);
                ok = false;
                break;
            }
        if (ok) {
            exec_txn(a.db, a.b, v, a.atomic_add);
            a.order[atomicAdd(&a.ctl->claim, 1u)] = (uint32_t)t;
        }
        for (int j = 0; j < held; j++) unlock(&a.lock[a.slot(items[j])]);
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
    int64_t grid = (b->n + 255) / 256;
    if (grid > (int64_t)db->num_sms * 8) grid = (int64_t)db->num_sms * 8;
    tpl_relaxed_kernel<<<(unsigned)grid, 256, 0, b->stream>>>(a);
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace gtx
