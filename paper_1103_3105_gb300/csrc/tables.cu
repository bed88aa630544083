// tables.cu -- small fill kernels used when a database is created.
#include <atomic>

#include "engine.h"

namespace gtx {

static std::atomic<unsigned long long> g_launches{0};
void count_launches(int k) { g_launches.fetch_add((unsigned long long)k, std::memory_order_relaxed); }

namespace {
__global__ void fill_i64_kernel(int64_t *p, int64_t n, int64_t v)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        p[i] = v;
}
__global__ void fill_u64_kernel(unsigned long long *p, int64_t n, unsigned long long v)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        p[i] = v;
}
inline unsigned blocks_for(int64_t n)
{
    int64_t b = (n + 255) / 256;
    if (b > 4096) b = 4096;
    return (unsigned)(b < 1 ? 1 : b);
}
}  // namespace

cudaError_t launch_fill_i64(int64_t *p, int64_t n, int64_t v, cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    fill_i64_kernel<<<blocks_for(n), 256, 0, s>>>(p, n, v);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_fill_u64(unsigned long long *p, int64_t n, unsigned long long v, cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    fill_u64_kernel<<<blocks_for(n), 256, 0, s>>>(p, n, v);
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace gtx

extern "C" unsigned long long gputx_launch_count(void) { return gtx::g_launches.load(); }
