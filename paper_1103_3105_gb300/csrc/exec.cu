// exec.cu -- the three bulk execution strategies (Section 5).
//
//   K-SET (Section 5.3)  a persistent grid walks the level-ordered bulk in
//       chunks of one CTA; a chunk of level k starts once every transaction
//       of level k-1 has finished (per-level completion counters), so the
//       k-sets run in order with no conflict control inside a level
//       (Property 1).  Chunks are claimed in increasing order, so every chunk
//       a waiting CTA depends on is held by a running CTA: the waits end.
//   PART (Section 5.2)   one thread per non-empty partition runs its
//       transactions serially in timestamp order.
//   TPL (Section 5.1)    ordered counter locks: an operation whose group has
//       `ticket` earlier operations before its run waits until that many have
//       released the item's counter, then the transaction runs and every
//       operation releases (+1).  Transactions are handed out in timestamp
//       order, so the earliest unfinished one never waits: no deadlock.
// Every wait is bounded by the configured limit; on expiry the kernel sets
// ERR_TIMEOUT in the bulk's error word and returns.
#include "engine.h"
#include "procs.cuh"

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

// waits until *p >= need; false on timeout
__device__ __forceinline__ bool wait_at_least(const uint32_t *p, uint32_t need, uint64_t limit_ns)
{
    if (ld_acquire(p) >= need) return true;
    const uint64_t t0 = globaltimer();
    uint32_t spins = 0;
    while (ld_acquire(p) < need) {
        if (++spins > 32) __nanosleep(spins < 1024 ? 32 : 256);
        if ((spins & 63) == 0 && globaltimer() - t0 > limit_ns) return false;
    }
    return true;
}

__global__ void kset_kernel(KsetArgs a)
{
    __shared__ uint32_t s_k, s_start, s_cnt, s_stop;
    const uint32_t nchunks = a.chunk_off[a.levels];
    while (true) {
        if (threadIdx.x == 0) {
            uint32_t stop = *(volatile uint32_t *)&a.ctl->err ? 1u : 0u;
            const uint32_t c = stop ? nchunks : atomicAdd(&a.ctl->claim, 1u);
            if (c < nchunks) {
                const uint32_t k = a.chunk_level[c];
                const uint32_t lo = a.level_off[k], hi = a.level_off[k + 1];
                const uint32_t start = lo + (c - a.chunk_off[k]) * blockDim.x;
                const uint32_t cnt = (hi - start) < blockDim.x ? (hi - start) : blockDim.x;
                if (k > 0 && !wait_at_least(&a.done[k - 1], lo - a.level_off[k - 1], a.spin_limit_ns)) {
                    set_err(&a.ctl->err, ERR_TIMEOUT);
                    stop = 1;
                }
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
        if (threadIdx.x < s_cnt) {
            const uint32_t pos = s_start + threadIdx.x;
            exec_txn(a.db, a.b, a.order[pos], pos, a.atomic_add);
            __threadfence();
        }
        __syncthreads();
        if (threadIdx.x == 0) red_release_add(&a.done[s_k], s_cnt);
    }
}

__global__ void part_kernel(DevDB db, DevBulk b, const BulkCtl *ctl, const uint32_t *pkeys, const uint32_t *pvals,
                            const uint32_t *part_start)
{
    const uint32_t p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= ctl->npart || ctl->err) return;
    uint32_t i = part_start[p];
    const uint32_t key = pkeys[i];
    const uint32_t n = (uint32_t)b.n;
    for (; i < n && pkeys[i] == key; i++) exec_txn(db, b, pvals[i], i, false);
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
};

__global__ void tpl_kernel(TplArgs a)
{
    __shared__ uint32_t s_c, s_stop;
    const int64_t n = a.b.n;
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
            const int64_t off = a.op_off ? (int64_t)a.op_off[t] : t * a.uniform_k;
            const int cnt = a.op_off ? (int)(a.op_off[t + 1] - a.op_off[t]) : a.uniform_k;
            bool ok = true;
            for (int j = 0; j < cnt && ok; j++) {
                const uint32_t tk = a.lock_ticket[off + j];
                if (tk && !wait_at_least(&a.done[a.lock_key[off + j]], tk, a.spin_limit_ns)) {
                    set_err(&a.ctl->err, ERR_TIMEOUT);
                    ok = false;
                }
            }
            if (ok) exec_txn(a.db, a.b, (uint32_t)t, (uint32_t)t, a.atomic_add);
            __threadfence();
            for (int j = 0; j < cnt; j++) red_release_add(&a.done[a.lock_key[off + j]], 1u);
        }
        __syncthreads();
    }
}

}  // namespace

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
    a.levels = (int64_t)b->host_ctl.depth + 1;
    a.spin_limit_ns = (uint64_t)db->cfg.spin_limit_ns;
    a.atomic_add = atomic_add;
    cudaError_t e = cudaMemsetAsync(b->sc.done, 0, (size_t)a.levels * sizeof(uint32_t), db->stream);
    if (e) return e;
    e = cudaMemsetAsync(&b->ctl->claim, 0, sizeof(uint32_t), db->stream);
    if (e) return e;
    int64_t grid = (int64_t)db->num_sms * exec_blocks_per_sm(0, block);
    if (grid > nchunks) grid = nchunks;
    kset_kernel<<<(unsigned)grid, block, 0, db->stream>>>(a);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_part(gputx_bulk *b, const uint32_t *pkeys, const uint32_t *pvals, int block)
{
    gputx_db *db = b->db;
    if (b->n == 0) return cudaSuccess;
    const DevBulk d = make_dev_bulk(b, GPUTX_CONFLICT_PAPER);
    const int64_t grid = (b->n + block - 1) / block;   // npart <= n, read on the device
    part_kernel<<<(unsigned)grid, block, 0, db->stream>>>(db->dev, d, b->ctl, pkeys, pvals, b->sc.part_start);
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
    a.op_off = db->uniform_k ? nullptr : b->sc.op_off;
    a.done = db->d_done;
    a.uniform_k = db->uniform_k;
    a.spin_limit_ns = (uint64_t)db->cfg.spin_limit_ns;
    a.atomic_add = atomic_add;
    cudaError_t e = cudaMemsetAsync(&b->ctl->claim, 0, sizeof(uint32_t), db->stream);
    if (e) return e;
    int64_t grid = (int64_t)db->num_sms * exec_blocks_per_sm(1, block);
    const int64_t chunks = (b->n + block - 1) / block;
    if (grid > chunks) grid = chunks;
    tpl_kernel<<<(unsigned)grid, block, 0, db->stream>>>(a);
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace gtx
