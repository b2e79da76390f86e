// Exclusive prefix sum of n counters in place by one thread block, for the
// sort's digit offsets (sort.cu) and the work-item offsets of the query tiles
// (query_gather's last block, search.cu).
#pragma once

#include <stdint.h>

namespace tdq {

// Every thread of the block calls it.  Each iteration stages kThreads * kPer
// counters in shared memory (one padding word per 32 against bank
// conflicts), scans kPer consecutive counters per thread, scans the thread
// sums across the block, writes the prefixes back and stores them
// coalesced; a carry links the iterations.  The counters of the next
// iteration are loaded (coalesced) while the current ones are scanned, so
// that a load's latency is paid once rather than once per iteration.  The
// data is read through L2 (other blocks may have written it).  total (may be
// null) receives the sum.
template <typename T, int kThreads, int kPer>
__device__ __forceinline__ void block_exclusive_scan(T *data, uint64_t n, T *total)
{
    static_assert(kThreads % 32 == 0 && kThreads <= 1024, "whole warps");
    constexpr int kWarps = kThreads / 32;
    constexpr int kChunk = kThreads * kPer;
    __shared__ T buf[kChunk + kChunk / 32];
    __shared__ T warp_sums[kWarps];
    __shared__ T carry;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    auto pad = [](int i) { return i + (i >> 5); };
    if (tid == 0) carry = 0;
    T nxt[kPer];
#pragma unroll
    for (int j = 0; j < kPer; j++) {
        const int i = j * kThreads + tid;
        nxt[j] = (uint64_t)i < n ? __ldcg(data + i) : (T)0;
    }
    for (uint64_t start = 0; start < n; start += kChunk) {
#pragma unroll
        for (int j = 0; j < kPer; j++) {
            const int i = j * kThreads + tid;
            buf[pad(i)] = nxt[j];
            nxt[j] = start + kChunk + i < n ? __ldcg(data + start + kChunk + i) : (T)0;
        }
        __syncthreads();
        T v[kPer];
        T s = 0;
#pragma unroll
        for (int j = 0; j < kPer; j++) {
            v[j] = buf[pad(tid * kPer + j)];
            s += v[j];
        }
        T x = s;  // inclusive scan of the thread sums within the warp
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const T y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) warp_sums[warp] = x;
        __syncthreads();
        if (warp == 0) {
            T w = lane < kWarps ? warp_sums[lane] : (T)0;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const T y = __shfl_up_sync(0xffffffffu, w, o);
                if (lane >= o) w += y;
            }
            if (lane < kWarps) warp_sums[lane] = w;  // inclusive over warps
        }
        __syncthreads();
        T before = carry + (warp > 0 ? warp_sums[warp - 1] : (T)0) + (x - s);
#pragma unroll
        for (int j = 0; j < kPer; j++) {
            buf[pad(tid * kPer + j)] = before;
            before += v[j];
        }
        __syncthreads();
#pragma unroll
        for (int j = 0; j < kPer; j++) {
            const int i = j * kThreads + tid;
            if (start + i < n) data[start + i] = buf[pad(i)];
        }
        if (tid == 0) carry += warp_sums[kWarps - 1];
        __syncthreads();
    }
    if (tid == 0 && total) *total = carry;
}

}  // namespace tdq
