// Stable LSD radix sort of (uint64 key, uint32 value) pairs.  Used to sort
// entry segments by t_start for the temporal-bin index (Sec. 4) and query
// segments by their clipped start (Sec. 4: the query set is sorted by
// t_start before its bins are looked up).
//
// Each 8-bit digit pass runs per-tile digit histograms and a stable scatter
// that ranks equal digits in input order inside each tile with warp match
// masks.  The scatter offsets of a (digit, tile) are the keys of smaller
// digits plus the keys of the same digit in earlier tiles: for large inputs
// one exclusive scan over the counts in digit-major order computes them
// between the two kernels; for up to kFusedTiles tiles each scatter block
// derives its own from the tile-major counts (no scan kernel).
#include "scan.cuh"
#include "tdq_internal.cuh"

namespace tdq {
namespace {

constexpr int kThreads = 256;
constexpr int kRadix = 256;
constexpr int kWarps = kThreads / 32;
// Keys per thread of a tile: 16 for large inputs (4096-key tiles); 4 for
// inputs up to 2^20 keys, so that small sorts still spread over the SMs.
constexpr uint64_t kSmallSort = 1u << 20;
inline int items_for(uint64_t n) { return n <= kSmallSort ? 4 : 16; }
constexpr uint32_t kFusedTiles = kSortFusedTiles;
static_assert(kThreads * 4 == kSortTileKeys, "small-path tiles hold kSortTileKeys keys");

// kTileMajor: counts stored as hist[tile][digit], else hist[digit][tile].
// Keys to sort: n, or the device count n_dev when given (never above n).
__device__ __forceinline__ uint64_t sort_count(uint64_t n, const unsigned long long *n_dev)
{
    return n_dev && *n_dev < n ? *n_dev : n;
}

template <int kItems, bool kTileMajor>
__global__ void __launch_bounds__(kThreads) radix_hist(const uint64_t *__restrict__ keys, uint64_t n_launch,
                                                       const unsigned long long *n_dev, int shift,
                                                       uint32_t *__restrict__ hist, uint32_t ntiles)
{
    constexpr int kTile = kThreads * kItems;
    const uint64_t n = sort_count(n_launch, n_dev);
    __shared__ uint32_t h[kRadix];
    h[threadIdx.x] = 0;
    __syncthreads();
    uint64_t base = (uint64_t)blockIdx.x * kTile;
#pragma unroll 4
    for (int i = 0; i < kItems; i++) {
        uint64_t idx = base + (uint64_t)i * kThreads + threadIdx.x;
        if (idx < n) atomicAdd(&h[(keys[idx] >> shift) & 0xff], 1u);
    }
    __syncthreads();
    if (kTileMajor)
        hist[(uint64_t)blockIdx.x * kRadix + threadIdx.x] = h[threadIdx.x];
    else
        hist[(uint64_t)threadIdx.x * ntiles + blockIdx.x] = h[threadIdx.x];
}

// Scatter offset of digit `tid` for this block from the tile-major counts
// of all tiles: keys of smaller digits (block scan of the digit totals) plus
// keys of the same digit in earlier tiles.
__device__ __forceinline__ uint32_t fused_offset(const uint32_t *__restrict__ hist, uint32_t ntiles, int tid)
{
    __shared__ uint32_t wsum[kWarps];
    uint32_t before = 0, total = 0;
#pragma unroll 8
    for (uint32_t t = 0; t < ntiles; t++) {
        const uint32_t c = hist[(uint64_t)t * kRadix + tid];
        total += c;
        before += t < blockIdx.x ? c : 0u;
    }
    const int lane = tid & 31, warp = tid >> 5;
    uint32_t x = total;  // inclusive scan over the digits
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) wsum[warp] = x;
    __syncthreads();
    uint32_t wbase = 0;
    for (int w = 0; w < warp; w++) wbase += wsum[w];
    return wbase + x - total + before;
}

// Tiles past the keys to sort only write zero counts (radix_hist) or do
// nothing (radix_scatter).  next_hist (may be null, zeroed beforehand): the
// scatter adds the digit counts of the pass at next_shift per destination
// tile, tile-major (the next pass then needs no histogram kernel).
template <int kItems, bool kFused>
__global__ void __launch_bounds__(kThreads) radix_scatter(const uint64_t *__restrict__ keys,
                                                          const uint32_t *__restrict__ vals, uint64_t n_launch,
                                                          const unsigned long long *n_dev, int shift,
                                                          const uint32_t *__restrict__ offsets, uint32_t ntiles,
                                                          uint64_t *__restrict__ keys_out,
                                                          uint32_t *__restrict__ vals_out, uint32_t *next_hist,
                                                          int next_shift)
{
    constexpr int kTile = kThreads * kItems;
    __shared__ uint32_t off[kRadix];
    __shared__ uint32_t run[kRadix];
    __shared__ uint32_t wcnt[kWarps][kRadix];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint64_t n = sort_count(n_launch, n_dev);
    if ((uint64_t)blockIdx.x * kTile >= n) return;  // the whole block: no key of this tile is sorted
    off[tid] = kFused ? fused_offset(offsets, (uint32_t)((n + kTile - 1) / kTile), tid)
                      : offsets[(uint64_t)tid * ntiles + blockIdx.x];
    run[tid] = 0;
    const uint64_t base = (uint64_t)blockIdx.x * kTile;
    const unsigned lt_mask = (1u << lane) - 1u;
    for (int i = 0; i < kItems; i++) {
        for (int w = 0; w < kWarps; w++) wcnt[w][tid] = 0;
        __syncthreads();
        uint64_t idx = base + (uint64_t)i * kThreads + tid;
        bool valid = idx < n;
        uint64_t k = valid ? keys[idx] : 0;
        uint32_t v = valid ? vals[idx] : 0;
        uint32_t digit = valid ? (uint32_t)((k >> shift) & 0xff) : (uint32_t)kRadix;
        unsigned peers = __match_any_sync(0xffffffffu, digit);
        uint32_t lrank = __popc(peers & lt_mask);
        if (valid && lrank == 0) wcnt[warp][digit] = __popc(peers);
        __syncthreads();
        {
            // exclusive prefix over warps for digit `tid`, continuing the run
            uint32_t acc = run[tid];
            for (int w = 0; w < kWarps; w++) {
                uint32_t c = wcnt[w][tid];
                wcnt[w][tid] = acc;
                acc += c;
            }
            run[tid] = acc;
        }
        __syncthreads();
        if (valid) {
            uint32_t dst = off[digit] + wcnt[warp][digit] + lrank;
            keys_out[dst] = k;
            vals_out[dst] = v;
            if (next_hist) atomicAdd(&next_hist[(dst / kTile) * kRadix + ((k >> next_shift) & 0xff)], 1u);
        }
        __syncthreads();
    }
}

// Exclusive scan of n counters in one block of 1024 threads.
template <typename T, int kPer>
__global__ void __launch_bounds__(1024) scan_exclusive_block(T *data, uint64_t n, T *total)
{
    block_exclusive_scan<T, 1024, kPer>(data, n, total);
}

}  // namespace

// Histogram words for sorting any count up to n (small counts use smaller
// tiles, hence more of them).
uint64_t sort_hist_words(uint64_t n)
{
    const uint64_t small = n < kSmallSort ? n : kSmallSort;
    const uint64_t t4 = (small + kThreads * 4 - 1) / (kThreads * 4);
    const uint64_t t16 = (n + kThreads * 16 - 1) / (kThreads * 16);
    return (t4 > t16 ? t4 : t16) * kRadix + 1;
}

cudaError_t radix_sort_pairs(uint64_t *keys, uint32_t *vals, uint64_t *keys_alt, uint32_t *vals_alt, uint64_t n,
                             uint32_t *hist, cudaStream_t stream, int key_bits, const unsigned long long *n_dev,
                             uint32_t *prep_hist)
{
    if (n <= 1) return cudaSuccess;
    if (n > 0xffffffffULL) return cudaErrorInvalidValue;  // 32-bit offsets
    const int items = items_for(n);
    const uint64_t tile = (uint64_t)kThreads * items;
    uint32_t ntiles = (uint32_t)((n + tile - 1) / tile);
    uint64_t *src_k = keys, *dst_k = keys_alt;
    uint32_t *src_v = vals, *dst_v = vals_alt;
    const int passes = sort_passes(key_bits < 64 ? key_bits : 64);
    const bool fused = items == 4 && ntiles <= kFusedTiles;
    if (prep_hist && !fused) return cudaErrorInvalidValue;
    for (int shift = 0; shift < 8 * passes; shift += 8) {
        if (fused) {
            // passes 0 and 1 with prep_hist: counts from the key producer and
            // from the first scatter
            const bool given = prep_hist && shift < 16;
            uint32_t *h = given ? prep_hist + (shift ? (uint64_t)ntiles * kRadix : 0) : hist;
            uint32_t *next = prep_hist && shift == 0 ? prep_hist + (uint64_t)ntiles * kRadix : nullptr;
            if (!given) radix_hist<4, true><<<ntiles, kThreads, 0, stream>>>(src_k, n, n_dev, shift, h, ntiles);
            radix_scatter<4, true><<<ntiles, kThreads, 0, stream>>>(src_k, src_v, n, n_dev, shift, h, ntiles,
                                                                     dst_k, dst_v, next, shift + 8);
        } else {
            if (items == 4)
                radix_hist<4, false><<<ntiles, kThreads, 0, stream>>>(src_k, n, n_dev, shift, hist, ntiles);
            else
                radix_hist<16, false><<<ntiles, kThreads, 0, stream>>>(src_k, n, n_dev, shift, hist, ntiles);
            scan_exclusive_block<uint32_t, 8><<<1, 1024, 0, stream>>>(hist, (uint64_t)ntiles * kRadix, nullptr);
            if (items == 4)
                radix_scatter<4, false><<<ntiles, kThreads, 0, stream>>>(src_k, src_v, n, n_dev, shift, hist,
                                                                          ntiles, dst_k, dst_v, nullptr, 0);
            else
                radix_scatter<16, false><<<ntiles, kThreads, 0, stream>>>(src_k, src_v, n, n_dev, shift, hist,
                                                                           ntiles, dst_k, dst_v, nullptr, 0);
        }
        uint64_t *tk = src_k; src_k = dst_k; dst_k = tk;
        uint32_t *tv = src_v; src_v = dst_v; dst_v = tv;
    }
    // an even number of passes: the data is back in keys/vals
    return cudaGetLastError();
}

int sort_kernel_launches(uint64_t n, int key_bits, bool prep_hist)
{
    if (n <= 1) return 0;
    const int passes = sort_passes(key_bits < 64 ? key_bits : 64);
    const uint64_t tile = (uint64_t)kThreads * items_for(n);
    const bool fused = items_for(n) == 4 && (n + tile - 1) / tile <= kFusedTiles;
    if (!fused) return passes * 3;
    return passes * 2 - (prep_hist ? (passes < 2 ? passes : 2) : 0);
}

cudaError_t load_sort_module()
{
    cudaFuncAttributes fa;
    return cudaFuncGetAttributes(&fa, radix_hist<4, true>);
}

}  // namespace tdq
