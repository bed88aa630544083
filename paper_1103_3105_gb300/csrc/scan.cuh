// scan.cuh -- single-pass tile scans with decoupled look-back, and the
// onesweep LSD radix sort used by the dependency analysis (Section 4.2 steps
// 1 and 4: "a sort operation to perform grouping").
//
// Both follow published designs: decoupled look-back (Merrill & Garland,
// "Single-pass Parallel Prefix Scan with Decoupled Look-back", 2016) and the
// onesweep radix sort built on it (Adinets & Merrill, "Onesweep: A Faster
// Least Significant Digit Radix Sort for GPUs", 2022).  Tiles take their ids
// from an atomic counter, so every tile a look-back waits on has already
// started and publishes its aggregate before it waits on anyone: the waits
// always end.  They are bounded anyway (ERR_TIMEOUT) so that a fault never
// turns into a hang.
#pragma once
#include "common.cuh"

namespace gtx {

// ---------------------------------------------------------------------------
// relaxed gpu-scope accesses for look-back status words
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t ld_relaxed_u32(const uint32_t *p)
{
    uint32_t v;
    asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_relaxed_u32(uint32_t *p, uint32_t v)
{
    asm volatile("st.relaxed.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ uint64_t ld_relaxed_u64(const uint64_t *p)
{
    uint64_t v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_relaxed_u64(uint64_t *p, uint64_t v)
{
    asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

// ===========================================================================
// dual segmented sum: the scan state used by every analysis scan
// ===========================================================================
// 62-bit payload: [61] f1 [60:31] v1 (30 bits) [30] f2 [29:0] v2 (30 bits).
// Each (f, v) field is a segmented sum: a set flag starts a new segment.
// A field whose flag is never set is a plain prefix sum.
struct DualSeg {
    static constexpr uint64_t M30 = (1ull << 30) - 1;
    __device__ __forceinline__ static uint64_t make(uint32_t f1, uint32_t v1, uint32_t f2, uint32_t v2)
    {
        return ((uint64_t)f1 << 61) | ((uint64_t)(v1 & M30) << 31) | ((uint64_t)f2 << 30) | (uint64_t)(v2 & M30);
    }
    __device__ __forceinline__ static uint32_t f1(uint64_t s) { return (uint32_t)(s >> 61) & 1u; }
    __device__ __forceinline__ static uint32_t v1(uint64_t s) { return (uint32_t)((s >> 31) & M30); }
    __device__ __forceinline__ static uint32_t f2(uint64_t s) { return (uint32_t)(s >> 30) & 1u; }
    __device__ __forceinline__ static uint32_t v2(uint64_t s) { return (uint32_t)(s & M30); }
    // a precedes b
    __device__ __forceinline__ static uint64_t combine(uint64_t a, uint64_t b)
    {
        const uint32_t fb1 = f1(b), fb2 = f2(b);
        return make(f1(a) | fb1, fb1 ? v1(b) : v1(a) + v1(b), f2(a) | fb2, fb2 ? v2(b) : v2(a) + v2(b));
    }
};

constexpr uint64_t LB_INVALID = 0, LB_AGG = 1, LB_INC = 2;
constexpr int SCAN_THREADS = 256;
constexpr int SCAN_ITEMS = 8;
constexpr int SCAN_TILE = SCAN_THREADS * SCAN_ITEMS;

// Look-back by warp 0 of a tile: returns the exclusive prefix of `tile`.
// status[t] = flag << 62 | payload.  Called by all 32 lanes of warp 0.
__device__ __forceinline__ uint64_t lookback_prefix(uint64_t *status, uint32_t tile, uint64_t tile_agg,
                                                    uint32_t *err, uint64_t spin_limit_ns)
{
    const int lane = threadIdx.x & 31;
    if (tile == 0) {
        if (lane == 0) st_relaxed_u64(&status[0], (LB_INC << 62) | tile_agg);
        return 0;
    }
    if (lane == 0) st_relaxed_u64(&status[tile], (LB_AGG << 62) | tile_agg);
    uint64_t running = 0;  // identity
    int64_t window_end = (int64_t)tile - 1;  // closest predecessor not yet folded
    const uint64_t t0 = globaltimer();
    while (true) {
        const int64_t t = window_end - lane;
        uint64_t s = 0;
        uint32_t flag;
        if (t >= 0) {
            while (true) {
                s = ld_relaxed_u64(&status[t]);
                flag = (uint32_t)(s >> 62);
                if (flag != LB_INVALID) break;
                if (globaltimer() - t0 > spin_limit_ns) { set_err(err, ERR_TIMEOUT); break; }
            }
        } else {
            flag = (uint32_t)LB_INC;  // before tile 0: behaves like an inclusive identity
            s = (LB_INC << 62);
        }
        const uint32_t inc_mask = __ballot_sync(0xffffffffu, flag == LB_INC);
        // lanes beyond the closest inclusive one contribute nothing
        const int stop = inc_mask ? __ffs(inc_mask) - 1 : 31;
        uint64_t v = (lane <= stop) ? (s & ((1ull << 62) - 1)) : 0;
        // fold farther (higher lane) before nearer (lower lane)
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            uint64_t other = __shfl_down_sync(0xffffffffu, v, off);
            if (lane + off < 32) v = DualSeg::combine(other, v);
        }
        v = __shfl_sync(0xffffffffu, v, 0);
        running = DualSeg::combine(v, running);
        if (inc_mask) break;
        window_end -= 32;
    }
    if (lane == 0) st_relaxed_u64(&status[tile], (LB_INC << 62) | DualSeg::combine(running, tile_agg));
    return running;
}

// Generic single-pass scan of a DualSeg state over [0, count).  Mode
// provides `uint64_t element(int64_t i)` and `void output(int64_t i,
// uint64_t inclusive)`; elements are produced and consumed in blocked order
// (thread t owns SCAN_ITEMS consecutive elements).
template <class Mode>
__global__ void __launch_bounds__(SCAN_THREADS)
dualseg_scan_kernel(Mode mode, int64_t count, uint64_t *status, uint32_t *tile_ctr, uint32_t *err,
                    uint64_t spin_limit_ns)
{
    __shared__ uint32_t s_tile;
    __shared__ uint64_t s_warp[SCAN_THREADS / 32];
    __shared__ uint64_t s_prefix;
    __shared__ uint32_t s_abort;
    // an earlier step failed: consume nothing (a block that returns here has
    // not taken a tile id, so no look-back waits on it); decided once per block
    if (threadIdx.x == 0) {
        s_abort = *(volatile uint32_t *)err;
        if (!s_abort) s_tile = atomicAdd(tile_ctr, 1u);
    }
    __syncthreads();
    if (s_abort) return;
    const uint32_t tile = s_tile;
    const int64_t base = (int64_t)tile * SCAN_TILE + (int64_t)threadIdx.x * SCAN_ITEMS;
    uint64_t incl[SCAN_ITEMS];
    uint64_t acc = 0;
#pragma unroll
    for (int j = 0; j < SCAN_ITEMS; j++) {
        const int64_t i = base + j;
        const uint64_t e = (i < count) ? mode.element(i) : 0;
        acc = j ? DualSeg::combine(acc, e) : e;
        incl[j] = acc;
    }
    // block scan of thread aggregates
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint64_t x = acc;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        uint64_t o = __shfl_up_sync(0xffffffffu, x, off);
        if (lane >= off) x = DualSeg::combine(o, x);
    }
    if (lane == 31) s_warp[warp] = x;
    uint64_t thread_excl = __shfl_up_sync(0xffffffffu, x, 1);
    if (lane == 0) thread_excl = 0;
    __syncthreads();
    if (warp == 0) {
        uint64_t w = (lane < SCAN_THREADS / 32) ? s_warp[lane] : 0;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            uint64_t o = __shfl_up_sync(0xffffffffu, w, off);
            if (lane >= off) w = DualSeg::combine(o, w);
        }
        const uint64_t tile_agg = __shfl_sync(0xffffffffu, w, SCAN_THREADS / 32 - 1);
        uint64_t wexcl = __shfl_up_sync(0xffffffffu, w, 1);
        if (lane == 0) wexcl = 0;
        if (lane < SCAN_THREADS / 32) s_warp[lane] = wexcl;
        const uint64_t pre = lookback_prefix(status, tile, tile_agg, err, spin_limit_ns);
        if (lane == 0) s_prefix = pre;
    }
    __syncthreads();
    const uint64_t prefix = DualSeg::combine(DualSeg::combine(s_prefix, s_warp[warp]), thread_excl);
#pragma unroll
    for (int j = 0; j < SCAN_ITEMS; j++) {
        const int64_t i = base + j;
        if (i < count) mode.output(i, DualSeg::combine(prefix, incl[j]));
    }
}

// ===========================================================================
// segmented 64-bit sums (wrapping): the scan state of the SCAN executor
// ===========================================================================
// (f, v): f set = a segment starts in this span, v = sum since the last
// start (or since the beginning).  A 64-bit sum and its flag do not fit one
// status word, so a tile publishes its value first and then, with release
// semantics, a 32-bit status word; readers acquire the status word before
// reading the value.  Aggregate and inclusive values have separate slots, so
// a value a reader may still fetch is never overwritten.
struct Seg64 {
    uint32_t f;
    uint64_t v;
    __device__ __forceinline__ static Seg64 make(uint32_t f, uint64_t v) { return Seg64{f, v}; }
    __device__ __forceinline__ static Seg64 identity() { return Seg64{0u, 0ull}; }
    // a precedes b
    __device__ __forceinline__ static Seg64 combine(const Seg64 &a, const Seg64 &b)
    {
        return Seg64{a.f | b.f, b.f ? b.v : a.v + b.v};
    }
};

__device__ __forceinline__ uint32_t ld_acquire_gpu_u32(const uint32_t *p)
{
    uint32_t v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release_gpu_u32(uint32_t *p, uint32_t v)
{
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ Seg64 shfl_down_seg(const Seg64 &x, int off)
{
    return Seg64{__shfl_down_sync(0xffffffffu, x.f, off), __shfl_down_sync(0xffffffffu, x.v, off)};
}
__device__ __forceinline__ Seg64 shfl_up_seg(const Seg64 &x, int off)
{
    return Seg64{__shfl_up_sync(0xffffffffu, x.f, off), __shfl_up_sync(0xffffffffu, x.v, off)};
}
__device__ __forceinline__ Seg64 shfl_seg(const Seg64 &x, int lane)
{
    return Seg64{__shfl_sync(0xffffffffu, x.f, lane), __shfl_sync(0xffffffffu, x.v, lane)};
}

struct Seg64Status {
    uint32_t *word;      // per tile: state (LB_*) | f << 2
    uint64_t *agg, *inc; // per tile values
};

// Look-back by warp 0 of a tile; returns the exclusive prefix of `tile`.
__device__ __forceinline__ Seg64 lookback_seg64(const Seg64Status &st, uint32_t tile, const Seg64 &tile_agg,
                                                uint32_t *err, uint64_t spin_limit_ns)
{
    const int lane = threadIdx.x & 31;
    if (tile == 0) {
        if (lane == 0) {
            st.inc[0] = tile_agg.v;
            st_release_gpu_u32(&st.word[0], (uint32_t)LB_INC | (tile_agg.f << 2));
        }
        return Seg64::identity();
    }
    if (lane == 0) {
        st.agg[tile] = tile_agg.v;
        st_release_gpu_u32(&st.word[tile], (uint32_t)LB_AGG | (tile_agg.f << 2));
    }
    Seg64 running = Seg64::identity();
    int64_t window_end = (int64_t)tile - 1;
    const uint64_t t0 = globaltimer();
    while (true) {
        const int64_t t = window_end - lane;
        uint32_t w = (uint32_t)LB_INC;
        Seg64 x = Seg64::identity();
        if (t >= 0) {
            while (true) {
                w = ld_acquire_gpu_u32(&st.word[t]);
                if ((w & 3u) != (uint32_t)LB_INVALID) break;
                if (globaltimer() - t0 > spin_limit_ns) {
                    set_err(err, ERR_TIMEOUT);
                    w = (uint32_t)LB_INC;   // give up: fold nothing more
                    break;
                }
            }
            if ((w & 3u) == (uint32_t)LB_INC) x = Seg64{(w >> 2) & 1u, ld_volatile_u64(&st.inc[t])};
            else if ((w & 3u) == (uint32_t)LB_AGG) x = Seg64{(w >> 2) & 1u, ld_volatile_u64(&st.agg[t])};
        }
        const uint32_t inc_mask = __ballot_sync(0xffffffffu, (w & 3u) == (uint32_t)LB_INC);
        const int stop = inc_mask ? __ffs(inc_mask) - 1 : 31;
        Seg64 v = (lane <= stop) ? x : Seg64::identity();
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const Seg64 other = shfl_down_seg(v, off);
            if (lane + off < 32) v = Seg64::combine(other, v);
        }
        v = shfl_seg(v, 0);
        running = Seg64::combine(v, running);
        if (inc_mask) break;
        window_end -= 32;
    }
    if (lane == 0) {
        const Seg64 incl = Seg64::combine(running, tile_agg);
        st.inc[tile] = incl.v;
        st_release_gpu_u32(&st.word[tile], (uint32_t)LB_INC | (incl.f << 2));
    }
    return running;
}

// Single-pass scan of a Seg64 state over [0, count).  Mode provides
// `Seg64 element(int64_t i)` and `void output(int64_t i, const Seg64 &incl)`;
// thread t owns SCAN_ITEMS consecutive elements.
template <class Mode>
__global__ void __launch_bounds__(SCAN_THREADS)
seg64_scan_kernel(Mode mode, int64_t count, Seg64Status st, uint32_t *tile_ctr, uint32_t *err,
                  uint64_t spin_limit_ns)
{
    __shared__ uint32_t s_tile, s_abort;
    __shared__ Seg64 s_warp[SCAN_THREADS / 32];
    __shared__ Seg64 s_prefix;
    if (threadIdx.x == 0) {
        s_abort = *(volatile uint32_t *)err;
        if (!s_abort) s_tile = atomicAdd(tile_ctr, 1u);
    }
    __syncthreads();
    if (s_abort) return;
    const uint32_t tile = s_tile;
    const int64_t base = (int64_t)tile * SCAN_TILE + (int64_t)threadIdx.x * SCAN_ITEMS;
    Seg64 incl[SCAN_ITEMS];
    // every element's loads first (independent), then the combine chain
#pragma unroll
    for (int j = 0; j < SCAN_ITEMS; j++) {
        const int64_t i = base + j;
        incl[j] = (i < count) ? mode.element(i) : Seg64::identity();
    }
    Seg64 acc = incl[0];
#pragma unroll
    for (int j = 1; j < SCAN_ITEMS; j++) {
        acc = Seg64::combine(acc, incl[j]);
        incl[j] = acc;
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    Seg64 x = acc;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const Seg64 o = shfl_up_seg(x, off);
        if (lane >= off) x = Seg64::combine(o, x);
    }
    if (lane == 31) s_warp[warp] = x;
    Seg64 thread_excl = shfl_up_seg(x, 1);
    if (lane == 0) thread_excl = Seg64::identity();
    __syncthreads();
    if (warp == 0) {
        Seg64 w = (lane < SCAN_THREADS / 32) ? s_warp[lane] : Seg64::identity();
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const Seg64 o = shfl_up_seg(w, off);
            if (lane >= off) w = Seg64::combine(o, w);
        }
        const Seg64 tile_agg = shfl_seg(w, SCAN_THREADS / 32 - 1);
        Seg64 wexcl = shfl_up_seg(w, 1);
        if (lane == 0) wexcl = Seg64::identity();
        if (lane < SCAN_THREADS / 32) s_warp[lane] = wexcl;
        const Seg64 pre = lookback_seg64(st, tile, tile_agg, err, spin_limit_ns);
        if (lane == 0) s_prefix = pre;
    }
    __syncthreads();
    const Seg64 prefix = Seg64::combine(Seg64::combine(s_prefix, s_warp[warp]), thread_excl);
#pragma unroll
    for (int j = 0; j < SCAN_ITEMS; j++) {
        const int64_t i = base + j;
        if (i < count) mode.output(i, Seg64::combine(prefix, incl[j]));
    }
}

// ===========================================================================
// onesweep LSD radix sort of (u32 key, u32 value) pairs, 8-bit digits
// ===========================================================================
// (internal linkage: each translation unit that includes this header gets
// its own copy of these kernels)
namespace {
constexpr int SORT_THREADS = 512;
constexpr int SORT_ITEMS = 16;
constexpr int SORT_TILE = SORT_THREADS * SORT_ITEMS;
constexpr int SORT_WARPS = SORT_THREADS / 32;
constexpr int RADIX = 256;
constexpr uint32_t ST_AGG = 1u << 30, ST_INC = 2u << 30, ST_VAL = (1u << 30) - 1;
constexpr size_t SORT_SMEM = (size_t)SORT_TILE * 8 + (size_t)SORT_WARPS * RADIX * 4;

// Histograms of every digit position in one pass over the keys.
__global__ void __launch_bounds__(256) radix_hist_kernel(const uint32_t *__restrict__ keys, int64_t n,
                                                         int passes, uint32_t *hist, const uint32_t *err)
{
    __shared__ uint32_t sh[4][RADIX];
    __shared__ uint32_t s_abort;
    if (threadIdx.x == 0) s_abort = *(volatile const uint32_t *)err;
    __syncthreads();
    if (s_abort) return;
    for (int i = threadIdx.x; i < 4 * RADIX; i += blockDim.x) (&sh[0][0])[i] = 0;
    __syncthreads();
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t k = keys[i];
        for (int p = 0; p < passes; p++) atomicAdd(&sh[p][(k >> (8 * p)) & 255u], 1u);
    }
    __syncthreads();
    for (int p = 0; p < passes; p++)
        for (int d = threadIdx.x; d < RADIX; d += blockDim.x)
            if (sh[p][d]) atomicAdd(&hist[p * RADIX + d], sh[p][d]);
}

// Exclusive scan of each pass's 256 counts (one block per pass).
__global__ void __launch_bounds__(RADIX) radix_offsets_kernel(const uint32_t *hist, uint32_t *offs)
{
    __shared__ uint32_t s[RADIX];
    const uint32_t *h = hist + blockIdx.x * RADIX;
    uint32_t v = h[threadIdx.x];
    s[threadIdx.x] = v;
    __syncthreads();
    for (int off = 1; off < RADIX; off <<= 1) {
        uint32_t o = threadIdx.x >= off ? s[threadIdx.x - off] : 0;
        __syncthreads();
        s[threadIdx.x] += o;
        __syncthreads();
    }
    offs[blockIdx.x * RADIX + threadIdx.x] = s[threadIdx.x] - v;
}

// One stable counting pass on digit (key >> shift) & 255.
__global__ void __launch_bounds__(SORT_THREADS, 2)
radix_pass_kernel(const uint32_t *__restrict__ kin, const uint32_t *__restrict__ vin, uint32_t *__restrict__ kout,
                  uint32_t *__restrict__ vout, int64_t n, int shift, const uint32_t *__restrict__ digit_off,
                  uint32_t *status, uint32_t *tile_ctr, uint32_t *err, uint64_t spin_limit_ns)
{
    extern __shared__ uint32_t smem[];
    uint32_t *s_keys = smem;
    uint32_t *s_vals = smem + SORT_TILE;
    uint32_t *s_whist = s_vals + SORT_TILE;  // [SORT_WARPS][RADIX]
    __shared__ uint32_t s_tile;
    __shared__ uint32_t s_start[RADIX];      // tile-local start of each digit
    __shared__ int64_t s_gbase[RADIX];       // global position of the digit's first tile element
    __shared__ uint32_t s_scan[RADIX / 32];

    __shared__ uint32_t s_abort;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid == 0) {   // block-uniform abort decision, see dualseg_scan_kernel
        s_abort = *(volatile uint32_t *)err;
        if (!s_abort) s_tile = atomicAdd(tile_ctr, 1u);
    }
    for (int i = tid; i < SORT_WARPS * RADIX; i += SORT_THREADS) s_whist[i] = 0;
    __syncthreads();
    if (s_abort) return;
    const uint32_t tile = s_tile;
    const int64_t base = (int64_t)tile * SORT_TILE;
    const int64_t wbase = base + (int64_t)warp * 32 * SORT_ITEMS;

    uint32_t key[SORT_ITEMS], val[SORT_ITEMS], rank[SORT_ITEMS];
#pragma unroll
    for (int j = 0; j < SORT_ITEMS; j++) {
        const int64_t i = wbase + j * 32 + lane;
        const bool ok = i < n;
        key[j] = ok ? kin[i] : 0xffffffffu;
        val[j] = ok ? vin[i] : 0u;
    }
    uint32_t *wh = s_whist + warp * RADIX;
    const uint32_t lt = lanemask_lt();
#pragma unroll
    for (int j = 0; j < SORT_ITEMS; j++) {
        const int64_t i = wbase + j * 32 + lane;
        const bool ok = i < n;
        const uint32_t d = (key[j] >> shift) & 255u;
        uint32_t peers = __ballot_sync(0xffffffffu, ok);
#pragma unroll
        for (int b = 0; b < 8; b++) {
            const uint32_t m = __ballot_sync(0xffffffffu, (d >> b) & 1u);
            peers &= ((d >> b) & 1u) ? m : ~m;
        }
        uint32_t prior = 0;
        if (ok) prior = wh[d];
        __syncwarp();
        if (ok) {
            rank[j] = prior + __popc(peers & lt);
            if ((peers & lt) == 0) wh[d] = prior + __popc(peers);
        }
        __syncwarp();
    }
    __syncthreads();

    // per digit: exclusive prefix over warps, tile count, look-back
    uint32_t cnt = 0;
    if (tid < RADIX) {
        for (int w = 0; w < SORT_WARPS; w++) {
            const uint32_t c = s_whist[w * RADIX + tid];
            s_whist[w * RADIX + tid] = cnt;
            cnt += c;
        }
        uint32_t *st = status + (int64_t)tile * RADIX + tid;
        uint32_t excl = 0;
        if (tile == 0) {
            st_relaxed_u32(st, ST_INC | cnt);
        } else {
            st_relaxed_u32(st, ST_AGG | cnt);
            int64_t t = (int64_t)tile - 1;
            const uint64_t t0 = globaltimer();
            while (t >= 0) {
                const uint32_t s = ld_relaxed_u32(status + t * RADIX + tid);
                if (s & ST_INC) { excl += s & ST_VAL; break; }
                if (s & ST_AGG) { excl += s & ST_VAL; t--; continue; }
                if (globaltimer() - t0 > spin_limit_ns) { set_err(err, ERR_TIMEOUT); break; }
            }
            st_relaxed_u32(st, ST_INC | (excl + cnt));
        }
        // exclusive scan of the tile counts over digits (8 warps of 32)
        uint32_t x = cnt;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            uint32_t o = __shfl_up_sync(0xffffffffu, x, off);
            if (lane >= off) x += o;
        }
        if (lane == 31) s_scan[warp] = x;
        s_start[tid] = x - cnt;  // within-warp exclusive for now
        s_gbase[tid] = (int64_t)digit_off[tid] + excl;
    }
    __syncthreads();
    if (tid < RADIX) {
        uint32_t add = 0;
        for (int w = 0; w < warp; w++) add += s_scan[w];
        s_start[tid] += add;
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < SORT_ITEMS; j++) {
        const int64_t i = wbase + j * 32 + lane;
        if (i < n) {
            const uint32_t d = (key[j] >> shift) & 255u;
            const uint32_t pos = s_start[d] + s_whist[warp * RADIX + d] + rank[j];
            s_keys[pos] = key[j];
            s_vals[pos] = val[j];
        }
    }
    __syncthreads();
    const int64_t tile_n = (n - base) < SORT_TILE ? (n - base) : SORT_TILE;
    for (int i = tid; i < tile_n; i += SORT_THREADS) {
        const uint32_t k = s_keys[i];
        const uint32_t d = (k >> shift) & 255u;
        const int64_t g = s_gbase[d] + (i - (int64_t)s_start[d]);
        if (g < 0 || g >= n) { set_err(err, ERR_BOUNDS); continue; }  // only after a timeout
        kout[g] = k;
        vout[g] = s_vals[i];
    }
}

}  // namespace

}  // namespace gtx
