// probe.cu -- the latency floor of a chain of levels on one thread-block
// cluster, measured on the device the engine runs on.
//
// A level of the K-SET narrow-level runner is: updates of rows the previous
// level updated (possibly on another SM of the cluster), as loads then stores
// or as atomics performed at L2, and a cluster barrier with release/acquire
// semantics, split so that stores no later level reads follow the arrival.
// This probe runs exactly that skeleton with no transaction logic: at level k
// every thread loads `loads` values written at level k-1 by threads of the
// next CTA, updates `stores` values (plain stores, or with `rmw` atomic
// additions to cells that threads of the next CTA updated at level k-1: one
// fetch-and-add whose old value is used after the arrival and reductions for
// the rest), arrives at the cluster barrier (release), stores `stores_after`
// more values and waits (acquire).  Its time per level is the floor any
// level-by-level executor with that launch shape and that memory traffic per
// level can reach.
#include <cooperative_groups.h>

#include "engine.h"

namespace cg = cooperative_groups;

namespace gtx {
namespace {

constexpr int kProbeMaxLoads = 8, kProbeMaxStores = 16, kProbeLine = 16;

// buf: (levels + 1) x n x kProbeMaxStores words of stored values, then
// n x kProbeMaxStores cells for the fetch-and-adds, one per 128-byte line
// (kProbeLine words): like a runner's balance rows, every update of a warp
// goes to its own line
__global__ void __launch_bounds__(1024, 1) probe_chain_kernel(int64_t *buf, int64_t *sink, int levels, int loads,
                                                            int stores, int stores_after, int rmw)
{
    cg::cluster_group cl = cg::this_cluster();
    const uint32_t n = cl.num_threads(), r = cl.thread_rank();
    // the rows this thread reads come from the next CTA's threads
    const uint32_t src = (r + blockDim.x) % n;
    unsigned long long *cells =
        reinterpret_cast<unsigned long long *>(buf + (int64_t)(levels + 1) * n * kProbeMaxStores);
    int64_t acc = r;
    for (int k = 1; k <= levels; k++) {
        const int64_t *prev = buf + (int64_t)(k - 1) * n * kProbeMaxStores;
        int64_t *cur = buf + (int64_t)k * n * kProbeMaxStores;
        int64_t v = 0;
        for (int j = 0; j < loads; j++) v += __ldcg(&prev[(int64_t)j * n + src]);
        acc += v;
        int64_t ret = 0;
        if (rmw) {
            // the column the next CTA's thread updated at level k-1
            const uint32_t c = (uint32_t)((r + (uint64_t)k * blockDim.x) % n);
            // one fetch-and-add whose old value is used after the arrival,
            // the rest reductions whose results nothing reads
            ret = (int64_t)atomicAdd(&cells[(int64_t)c * kProbeLine], (unsigned long long)acc);
            for (int j = 1; j < stores; j++)
                atomicAdd(&cells[((int64_t)j * n + c) * kProbeLine], (unsigned long long)(acc + j));
        } else {
            for (int j = 0; j < stores; j++) __stcg(&cur[(int64_t)j * n + r], acc + j);
        }
        asm volatile("barrier.cluster.arrive.release.aligned;" ::: "memory");
        for (int j = 0; j < stores_after; j++) __stcg(&cur[(int64_t)(stores + j) * n + r], acc - j + ret);
        asm volatile("barrier.cluster.wait.acquire.aligned;" ::: "memory");
    }
    sink[r] = acc;   // keeps the chain live
}

}  // namespace
}  // namespace gtx

using namespace gtx;

extern "C" gputx_status gputx_probe_level_chain(int levels, int cluster_size, int threads, int loads, int stores,
                                                int stores_after, int rmw, double *ns_per_level)
{
    if (!ns_per_level || levels < 1 || levels > (1 << 20) || cluster_size < 1 || cluster_size > 16 ||
        threads < 32 || threads > 1024 || threads % 32 || loads < 0 || loads > kProbeMaxLoads || stores < 1 ||
        stores_after < 0 || stores + stores_after > kProbeMaxStores || (rmw != 0 && rmw != 1))
        return GPUTX_EINVAL;
    const int64_t n = (int64_t)cluster_size * threads;
    const int64_t words = ((int64_t)(levels + 1) + kProbeLine) * n * kProbeMaxStores;
    int64_t *buf = nullptr, *sink = nullptr;
    cudaStream_t s = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    gputx_status st = GPUTX_OK;
    cudaError_t e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
    if (!e) e = cudaMalloc(&buf, words * sizeof(int64_t));
    if (!e) e = cudaMalloc(&sink, n * sizeof(int64_t));
    if (!e) e = cudaMemsetAsync(buf, 0, words * sizeof(int64_t), s);
    if (!e) e = cudaEventCreate(&e0);
    if (!e) e = cudaEventCreate(&e1);
    if (!e) e = cudaFuncSetAttribute(probe_chain_kernel, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (!e) {
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(cluster_size, 1, 1);
        cfg.blockDim = dim3(threads, 1, 1);
        cfg.stream = s;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = cluster_size;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        // one warm-up launch, then the timed one
        e = cudaLaunchKernelEx(&cfg, probe_chain_kernel, buf, sink, levels, loads, stores, stores_after, rmw);
        if (!e) e = cudaEventRecord(e0, s);
        if (!e) e = cudaLaunchKernelEx(&cfg, probe_chain_kernel, buf, sink, levels, loads, stores, stores_after, rmw);
        if (!e) e = cudaEventRecord(e1, s);
        if (!e) e = cudaEventSynchronize(e1);
        float ms = 0;
        if (!e) e = cudaEventElapsedTime(&ms, e0, e1);
        if (!e) *ns_per_level = (double)ms * 1e6 / levels;
        count_launches(2);
    }
    if (e) st = e == cudaErrorMemoryAllocation ? GPUTX_ENOMEM : GPUTX_ECUDA;
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (buf) cudaFree(buf);
    if (sink) cudaFree(sink);
    if (s) cudaStreamDestroy(s);
    return st;
}
