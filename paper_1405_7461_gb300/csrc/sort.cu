// Stable LSD radix sort of (uint64 key, uint32 value) pairs and a
// single-block exclusive scan.  Used to sort entry segments by t_start for the
// temporal-bin index (Sec. 4) and query segments by their clipped start
// (Sec. 4: the query set is sorted by t_start before its bins are looked up).
//
// Each 8-bit digit pass runs three kernels: per-tile digit histograms, one
// exclusive scan over (digit, tile) counts in digit-major order, and a stable
// scatter that ranks equal digits in input order inside each tile with
// warp match masks.
#include "tdq_internal.cuh"

namespace tdq {
namespace {

constexpr int kThreads = 256;
constexpr int kItems = 16;
constexpr int kTile = kThreads * kItems;  // 4096 keys per tile
constexpr int kRadix = 256;
constexpr int kWarps = kThreads / 32;

__global__ void __launch_bounds__(kThreads) radix_hist(const uint64_t *__restrict__ keys, uint64_t n, int shift,
                                                       uint32_t *__restrict__ hist, uint32_t ntiles)
{
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
    hist[(uint64_t)threadIdx.x * ntiles + blockIdx.x] = h[threadIdx.x];
}

__global__ void __launch_bounds__(kThreads) radix_scatter(const uint64_t *__restrict__ keys,
                                                          const uint32_t *__restrict__ vals, uint64_t n, int shift,
                                                          const uint32_t *__restrict__ offsets, uint32_t ntiles,
                                                          uint64_t *__restrict__ keys_out,
                                                          uint32_t *__restrict__ vals_out)
{
    __shared__ uint32_t off[kRadix];
    __shared__ uint32_t run[kRadix];
    __shared__ uint32_t wcnt[kWarps][kRadix];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    off[tid] = offsets[(uint64_t)tid * ntiles + blockIdx.x];
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
        }
        __syncthreads();
    }
}

// Exclusive scan of 32-bit counts (digit-major histogram) in one block.
template <typename T>
__global__ void __launch_bounds__(1024) scan_exclusive_block(T *data, uint64_t n, T *total)
{
    __shared__ T warp_sums[32];
    __shared__ T carry;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid == 0) carry = 0;
    __syncthreads();
    constexpr int kPer = 4;
    for (uint64_t start = 0; start < n; start += 1024 * kPer) {
        T v[kPer];
        T s = 0;
#pragma unroll
        for (int j = 0; j < kPer; j++) {
            uint64_t idx = start + (uint64_t)tid * kPer + j;
            v[j] = idx < n ? data[idx] : 0;
            s += v[j];
        }
        // inclusive warp scan of per-thread sums
        T x = s;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            T y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) warp_sums[warp] = x;
        __syncthreads();
        if (warp == 0) {
            T w = warp_sums[lane];
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                T y = __shfl_up_sync(0xffffffffu, w, o);
                if (lane >= o) w += y;
            }
            warp_sums[lane] = w;  // inclusive over warps
        }
        __syncthreads();
        T before = carry + (warp > 0 ? warp_sums[warp - 1] : 0) + (x - s);
#pragma unroll
        for (int j = 0; j < kPer; j++) {
            uint64_t idx = start + (uint64_t)tid * kPer + j;
            if (idx < n) data[idx] = before;
            before += v[j];
        }
        __syncthreads();
        if (tid == 0) carry += warp_sums[31];
        __syncthreads();
    }
    if (tid == 0 && total) *total = carry;
}

}  // namespace

uint64_t sort_hist_words(uint64_t n)
{
    uint64_t ntiles = (n + kTile - 1) / kTile;
    return ntiles * kRadix + 1;
}

cudaError_t radix_sort_pairs(uint64_t *keys, uint32_t *vals, uint64_t *keys_alt, uint32_t *vals_alt, uint64_t n,
                             uint32_t *hist, cudaStream_t stream, int key_bits)
{
    if (n <= 1) return cudaSuccess;
    if (n > 0xffffffffULL) return cudaErrorInvalidValue;  // 32-bit offsets
    uint32_t ntiles = (uint32_t)((n + kTile - 1) / kTile);
    uint64_t *src_k = keys, *dst_k = keys_alt;
    uint32_t *src_v = vals, *dst_v = vals_alt;
    const int passes = sort_passes(key_bits < 64 ? key_bits : 64);
    for (int shift = 0; shift < 8 * passes; shift += 8) {
        radix_hist<<<ntiles, kThreads, 0, stream>>>(src_k, n, shift, hist, ntiles);
        scan_exclusive_block<uint32_t><<<1, 1024, 0, stream>>>(hist, (uint64_t)ntiles * kRadix, nullptr);
        radix_scatter<<<ntiles, kThreads, 0, stream>>>(src_k, src_v, n, shift, hist, ntiles, dst_k, dst_v);
        uint64_t *tk = src_k; src_k = dst_k; dst_k = tk;
        uint32_t *tv = src_v; src_v = dst_v; dst_v = tv;
    }
    // an even number of passes: the data is back in keys/vals
    return cudaGetLastError();
}

cudaError_t exclusive_scan_u64(unsigned long long *data, uint64_t n, unsigned long long *total,
                               cudaStream_t stream)
{
    scan_exclusive_block<unsigned long long><<<1, 1024, 0, stream>>>(data, n, total);
    return cudaGetLastError();
}

}  // namespace tdq
