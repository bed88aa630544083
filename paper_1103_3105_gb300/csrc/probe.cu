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
constexpr int64_t kProbeTable = 10000000;   // rmw = 2: cells of a table the size of 10M accounts

// rmw = 2: the cell a thread's fetch-and-add takes at level k, uniform over
// the table (SplitMix64 of the thread and the level)
__device__ __forceinline__ uint64_t probe_cell(uint32_t r, int k)
{
    uint64_t z = ((uint64_t)r << 32 | (uint32_t)k) + 0x9e3779b97f4a7c15ull;
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
    return (z ^ (z >> 31)) % (uint64_t)kProbeTable;
}

__global__ void __launch_bounds__(1024, 1) probe_chain_kernel(int64_t *buf, int64_t *sink, int levels, int loads,
                                                            int stores, int stores_after, int rmw,
                                                            unsigned long long *table)
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
            // one fetch-and-add whose old value is used after the arrival
            // (rmw = 2: a random cell of the table, prefetched into L2 two
            // levels ahead as the runner prefetches its accounts), the rest
            // reductions whose results nothing reads
            unsigned long long *cell = &cells[(int64_t)c * kProbeLine];
            if (rmw == 2) {
                cell = &table[probe_cell(r, k)];
                asm volatile("prefetch.global.L2 [%0];" ::"l"(&table[probe_cell(r, k + 2)]));
            }
            ret = (int64_t)atomicAdd(cell, (unsigned long long)acc);
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

// the throughput of 64-bit atomic additions performed at L2: every thread
// adds 1 to `ops` cells drawn uniformly from [0, n_cells) (SplitMix64 on a
// per-thread counter), as reductions (fetch = 0) or as fetch-and-adds whose
// results are summed (fetch = 1)
__global__ void __launch_bounds__(256) probe_atomics_kernel(unsigned long long *cells, uint64_t n_cells, int ops,
                                                            int fetch, uint64_t seed, unsigned long long *sink)
{
    const uint64_t tid = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
    unsigned long long acc = 0;
    for (int i = 0; i < ops; i++) {
        uint64_t z = seed + (tid * (uint64_t)ops + (uint64_t)i + 1) * 0x9E3779B97F4A7C15ull;
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        z ^= z >> 31;
        const uint64_t idx = __umul64hi(z, n_cells);
        if (fetch) acc += atomicAdd(&cells[idx], 1ull);
        else atomicAdd(&cells[idx], 1ull);
    }
    if (fetch && acc == 0x5a5a5a5a5a5a5a5aull) sink[0] = acc;   // keeps the results live
}

}  // namespace
}  // namespace gtx

using namespace gtx;

extern "C" gputx_status gputx_probe_atomics(int64_t n_cells, int fetch, double *gops)
{
    if (!gops || n_cells < 1 || n_cells > (int64_t)1 << 32 || (fetch != 0 && fetch != 1)) return GPUTX_EINVAL;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) return GPUTX_ECUDA;
    const int threads = 256, ops = 64;
    const int64_t grid = (int64_t)sms * 8;
    const double total = (double)grid * threads * ops;
    unsigned long long *cells = nullptr, *sink = nullptr;
    cudaStream_t s = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    gputx_status st = GPUTX_OK;
    cudaError_t e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
    if (!e) e = cudaMalloc(&cells, n_cells * sizeof(unsigned long long));
    if (!e) e = cudaMalloc(&sink, sizeof(unsigned long long));
    if (!e) e = cudaMemsetAsync(cells, 0, n_cells * sizeof(unsigned long long), s);
    if (!e) e = cudaEventCreate(&e0);
    if (!e) e = cudaEventCreate(&e1);
    if (!e) {
        // one warm-up launch (brings a table that fits into L2), then the timed one
        probe_atomics_kernel<<<(unsigned)grid, threads, 0, s>>>(cells, (uint64_t)n_cells, ops, fetch, 1, sink);
        e = cudaGetLastError();
        if (!e) e = cudaEventRecord(e0, s);
        if (!e) probe_atomics_kernel<<<(unsigned)grid, threads, 0, s>>>(cells, (uint64_t)n_cells, ops, fetch, 2, sink);
        if (!e) e = cudaGetLastError();
        if (!e) e = cudaEventRecord(e1, s);
        if (!e) e = cudaEventSynchronize(e1);
        float ms = 0;
        if (!e) e = cudaEventElapsedTime(&ms, e0, e1);
        if (!e) *gops = total / ((double)ms * 1e6);
        count_launches(2);
    }
    if (e) st = e == cudaErrorMemoryAllocation ? GPUTX_ENOMEM : GPUTX_ECUDA;
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (cells) cudaFree(cells);
    if (sink) cudaFree(sink);
    if (s) cudaStreamDestroy(s);
    return st;
}

extern "C" gputx_status gputx_probe_level_chain(int levels, int cluster_size, int threads, int loads, int stores,
                                                int stores_after, int rmw, double *ns_per_level)
{
    if (!ns_per_level || levels < 1 || levels > (1 << 20) || cluster_size < 1 || cluster_size > 16 ||
        threads < 32 || threads > 1024 || threads % 32 || loads < 0 || loads > kProbeMaxLoads || stores < 1 ||
        stores_after < 0 || stores + stores_after > kProbeMaxStores || rmw < 0 || rmw > 2)
        return GPUTX_EINVAL;
    const int64_t n = (int64_t)cluster_size * threads;
    const int64_t words = ((int64_t)(levels + 1) + kProbeLine) * n * kProbeMaxStores;
    int64_t *buf = nullptr, *sink = nullptr;
    unsigned long long *table = nullptr;
    cudaStream_t s = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    gputx_status st = GPUTX_OK;
    cudaError_t e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
    if (!e) e = cudaMalloc(&buf, words * sizeof(int64_t));
    if (!e) e = cudaMalloc(&sink, n * sizeof(int64_t));
    if (!e) e = cudaMemsetAsync(buf, 0, words * sizeof(int64_t), s);
    if (!e && rmw == 2) e = cudaMalloc(&table, kProbeTable * sizeof(unsigned long long));
    if (!e && rmw == 2) e = cudaMemsetAsync(table, 0, kProbeTable * sizeof(unsigned long long), s);
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
        e = cudaLaunchKernelEx(&cfg, probe_chain_kernel, buf, sink, levels, loads, stores, stores_after, rmw, table);
        if (!e) e = cudaEventRecord(e0, s);
        if (!e) e = cudaLaunchKernelEx(&cfg, probe_chain_kernel, buf, sink, levels, loads, stores, stores_after, rmw,
                                       table);
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
    if (table) cudaFree(table);
    if (s) cudaStreamDestroy(s);
    return st;
}
