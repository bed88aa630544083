// exec_dc.cu -- the K-SET narrow-level runner for debit-credit-only bulks
// (Section 5.3's k-sets over Section 5.1's debit-credit workload).
//
// A run of narrow levels executes on one thread-block cluster: a level's
// transactions spread over the cluster's threads, and a cluster barrier
// separates consecutive levels (Property 1 makes a level's transactions
// independent; the barrier orders the levels).  Each transaction comes from
// a packed 32-byte record gathered in execution order, with teller and
// branch precomputed.
#include <cooperative_groups.h>

#include "dc.cuh"
#include "levels.cuh"

namespace cg = cooperative_groups;

namespace gtx {

namespace {

// the narrow-level runner for debit-credit-only bulks: one packed record per
// transaction (no type dispatch, no divisions), its balances updated by
// atomics at L2, so nothing is loaded between the barrier's acquire and the
// updates.  Only the account's fetch-and-add precedes the barrier's release
// (dc_account_rmw); teller and branch additions, history row and outputs
// follow it (dc_finish_rmw).  The inputs of later levels run ahead in a
// pipeline, each stage a whole level before its use: while level k executes,
// level k+1's and k+2's records are in registers, level k+3's record is
// loading and level k+4's end offset too; after the arrival, level k+2's
// account rows are prefetched into L2, so an account row coming from HBM has
// a whole level to arrive before it is updated.
template <bool CLUSTER, int MAXT>
__global__ void __launch_bounds__(MAXT, 1) kset_narrow_dc_kernel(LevelArgs a)
{
    if (a.ctl->err) return;   // set by an earlier launch only: uniform here
    const int64_t hb = a.ctl->base.hist;
    uint32_t nthreads = blockDim.x, rank = threadIdx.x;
    if (CLUSTER) {
        cg::cluster_group cl = cg::this_cluster();
        nthreads = cl.num_threads();
        rank = cl.thread_rank();
    }
    // the end of level j (the start of level j+1); levels from k1 on are empty
    auto end_of = [&](uint32_t j, uint32_t prev) { return j < a.k1 ? __ldg(&a.level_off[j + 1]) : prev; };
    // level k is [lo, e0); levels k+1, k+2, k+3 end at e1, e2, e3
    uint32_t lo = __ldg(&a.level_off[a.k0]);
    uint32_t e0 = end_of(a.k0, lo);
    uint32_t e1 = end_of(a.k0 + 1, e0);
    uint32_t e2 = end_of(a.k0 + 2, e1);
    uint32_t e3 = end_of(a.k0 + 3, e2);
    DcRecord v{}, r1{}, r2{};
    if (lo + rank < e0) {
        v = a.rec_dc[lo + rank];
        prefetch_l2(&a.db.acc_bal[v.a]);
    }
    if (e0 + rank < e1) {
        r1 = a.rec_dc[e0 + rank];
        prefetch_l2(&a.db.acc_bal[r1.a]);
    }
    if (e1 + rank < e2) r2 = a.rec_dc[e1 + rank];
    for (uint32_t k = a.k0; k < a.k1; k++) {
        const uint32_t e4 = end_of(k + 4, e3);
        DcRecord r3{};
        if (e2 + rank < e3) r3 = a.rec_dc[e2 + rank];
        const bool has2 = e1 + rank < e2;
        // the account update (the only cell a later level reads) before the
        // barrier's release; the rest after this thread has arrived,
        // overlapping the other threads' arrival
        DcOut o;
        bool pending = false;
        if (lo + rank < e0) pending = dc_account_rmw(a.db, a.b, v, hb + lo + rank, o);
        for (uint32_t pos = lo + rank + nthreads; pos < e0; pos += nthreads)
            exec_dc_record_rmw(a.db, a.b, a.rec_dc[pos], hb + pos);
        if (CLUSTER) {
            // split cluster barrier: arrive with release semantics, do the
            // work no other thread waits for, then wait with acquire
            asm volatile("barrier.cluster.arrive.release.aligned;" ::: "memory");
        }
        if (pending) dc_finish_rmw(a.db, a.b, o);
        // teller and branch rows need none: some level updates them nearly
        // every level, so they stay in L2
        if (has2) prefetch_l2(&a.db.acc_bal[r2.a]);
        if (CLUSTER) asm volatile("barrier.cluster.wait.acquire.aligned;" ::: "memory");
        else __syncthreads();
        lo = e0;
        e0 = e1;
        e1 = e2;
        e2 = e3;
        e3 = e4;
        v = r1;
        r1 = r2;
        r2 = r3;
    }
}

}  // namespace

cudaError_t launch_narrow_dc(const LevelArgs &a, int csize, int threads, cudaStream_t s)
{
    static bool attr_set = false;
    if (!attr_set) {
        cudaFuncSetAttribute(kset_narrow_dc_kernel<true, 256>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
        cudaFuncSetAttribute(kset_narrow_dc_kernel<true, 512>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
        cudaFuncSetAttribute(kset_narrow_dc_kernel<true, 1024>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
        attr_set = true;
    }
    if (csize <= 1) {
        if (threads <= 256) kset_narrow_dc_kernel<false, 256><<<1, threads, 0, s>>>(a);
        else if (threads <= 512) kset_narrow_dc_kernel<false, 512><<<1, threads, 0, s>>>(a);
        else kset_narrow_dc_kernel<false, 1024><<<1, threads, 0, s>>>(a);
        return cudaGetLastError();
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(csize, 1, 1);
    cfg.blockDim = dim3(threads, 1, 1);
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = csize;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    // the register budget follows the CTA size: the records in flight need
    // more than the 64 a thread of a 1024-thread CTA may hold
    return threads <= 256   ? cudaLaunchKernelEx(&cfg, kset_narrow_dc_kernel<true, 256>, a)
           : threads <= 512 ? cudaLaunchKernelEx(&cfg, kset_narrow_dc_kernel<true, 512>, a)
                            : cudaLaunchKernelEx(&cfg, kset_narrow_dc_kernel<true, 1024>, a);
}

}  // namespace gtx
