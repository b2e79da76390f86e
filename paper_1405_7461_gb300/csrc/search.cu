// Distance threshold search on the device: candidate lookup in the
// temporal-bin index (Sec. 4) and the pair kernel (Sec. 5, Algorithm 1).
//
// Pipeline of one search on the caller's stream:
//   query_prep    validate, clip each query segment to the window, velocity,
//                 start position at the clipped start, sort key, candidate
//                 range [lo, hi) of sorted entry positions from the bin
//                 table; filter mode: the exact number of temporal-overlap
//                 pairs of each query segment
//   radix sort    query segments by clipped start (Sec. 4 sorts Q by t_start)
//   query_gather  sorted query SoA; one warp per tile of 32 consecutive
//                 sorted query segments plans the tile: its range is the
//                 union of its members' ranges, cut into chunks of
//                 `entry_chunk` entries, one work item per (tile, chunk); the
//                 last block to finish scans the work-item offsets per tile
//   traj_dist_search_kernel
//                 persistent CTAs take work items from an atomic counter,
//                 stage the tile's queries and the chunk's entries in shared
//                 memory, enumerate the pairs whose spans overlap with
//                 integer time keys, compact them so that all 32 lanes of a
//                 warp evaluate a real pair, and append every pair within d
//                 with one atomic per warp; its last block to finish copies
//                 the search's counters to the caller-visible host mirror.
//
// (The filter mode's pair kernels live in filter.cu, the allocation-free
// entry point in noalloc.cu.)
//
// Design notes for GB300: the FP64 pipe issues ~2 DFMA per clock per SM, so
// FP64 lane-slots are the scarce resource.  Temporal tests and every
// comparison run on the integer pipe; a lane never issues FP64 work for a
// pair whose spans do not overlap; the interval roots (sqrt, two divisions)
// run only for pairs that are within d.
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include "pipeline.cuh"
#include "scan.cuh"

namespace tdq {
namespace {

__device__ __forceinline__ bool is_nan_bits(double x)
{
    int64_t b = __double_as_longlong(x) & 0x7fffffffffffffffLL;
    return b > 0x7ff0000000000000LL;
}

}  // namespace

// Candidate range [lo, hi) of sorted entry positions of one valid query
// segment with clipped span keys [cs, ce): from the first bin whose entries
// can end after cs up to the last entry that starts before ce; with
// count_overlaps also its exact number of temporal-overlap pairs: #{t_start <
// q.t_end} - #{t_end <= q.t_start} (the second set lies inside the first
// because t_end > t_start).
__device__ __forceinline__ void candidate_range(const BinView &bins, int64_t cs, int64_t ce, bool count_overlaps,
                                                int64_t &rlo, int64_t &rhi, unsigned long long &n_overlap,
                                                int64_t &bin_start)
{
    // Three binary searches, advanced together so that their loads overlap
    // (each thread's searches are a chain of dependent loads):
    //  A  the first bin whose extent reaches past the query start -- the
    //     prefix maximum of bin ends is non-decreasing (Sec. 4 uses an index
    //     tree over the bin extents for the same lookup); an entry that ends
    //     after cs starts after cs - max_dur, so the answer is searched
    //     between the bins of cs - max_dur and cs, both ends of that bracket
    //     verified (else the rest of the table);
    //  B  #{t_start < ce}, the end of the range: the bin function is
    //     monotone in time, so the count lies inside the bin of ce in the
    //     sorted t_start keys (bin table bin_begin) -- entries of that bin
    //     that start at or after ce (on a time grid: the whole next step)
    //     are left out;
    //  C  (count_overlaps) #{t_end <= cs}, likewise inside the bin of cs in
    //     the sorted t_end keys (bin table te_bin_begin).
    const double te = key_double(ce), ts = key_double(cs);
    // Last bin that can hold an entry starting before the query end (none
    // when the query ends at or before the first entry start).
    const int64_t jhi = ce <= bins.tmin_key ? -1 : bin_of_key(bins, ce, te);
    const int64_t m = bins.m;
    const int64_t bts = bin_of_key(bins, cs, ts);  // exact: C relies on it
    bin_start = bts;
    int64_t a_lo, a_hi;
    {
        // the lower end only needs to be about right: it is verified
        const int64_t hb = bts + 1 < m ? bts + 1 : m - 1;
        int64_t b0 = bts - bins.dur_bins - 1;
        if (b0 < 0) b0 = 0;
        if (b0 > hb) b0 = hb;
        const bool below = b0 > 0 && bins.bin_pmax_key[b0 - 1] > cs;  // the answer lies before b0
        const bool above = !below && bins.bin_pmax_key[hb] <= cs;     // the answer lies after hb
        a_lo = below ? 0 : (above ? hb + 1 : b0);
        a_hi = below ? b0 : (above ? m : hb + 1);
    }
    int64_t b_lo = 0, b_hi = 0, c_lo = 0, c_hi = 0;
    if (jhi >= 0) {
        b_lo = bins.bin_begin[jhi];
        b_hi = bins.bin_begin[jhi + 1];
        if (count_overlaps && cs > bins.tmin_key) {
            c_lo = bins.te_bin_begin[bts];
            c_hi = bins.te_bin_begin[bts + 1];
        }
    }
    while (a_lo < a_hi || b_lo < b_hi || c_lo < c_hi) {
        if (a_lo < a_hi) {  // first bin with prefix-max end > cs
            const int64_t mid = (a_lo + a_hi) >> 1;
            if (bins.bin_pmax_key[mid] > cs) a_hi = mid; else a_lo = mid + 1;
        }
        if (b_lo < b_hi) {  // first sorted t_start >= ce
            const int64_t mid = (b_lo + b_hi) >> 1;
            if (bins.ts_key[mid] < ce) b_lo = mid + 1; else b_hi = mid;
        }
        if (c_lo < c_hi) {  // first sorted t_end > cs
            const int64_t mid = (c_lo + c_hi) >> 1;
            if (bins.te_sorted[mid] <= cs) c_lo = mid + 1; else c_hi = mid;
        }
    }
    const int64_t jlo = a_lo;
    if (jlo < m && jlo <= jhi) {
        rlo = bins.bin_begin[jlo];
        rhi = b_lo;  // first sorted t_start >= ce
        if (rlo >= rhi) { rlo = INT64_MAX; rhi = INT64_MIN; }
    }
    if (count_overlaps && jhi >= 0) n_overlap = (unsigned long long)(b_lo - c_lo);
}

// One real query slot's input, validated and clipped to its window
// (Sec. 4): the eight columns, d, the start key and the clipped span keys
// [cs, ce).  ok: every value finite, t_end > t_start, d >= 0, the window
// ordered and free of NaN; valid: ok with a non-empty clipped span.
struct SlotIn {
    double c[8];
    double d;
    int64_t ks, cs, ce;
    bool ok, valid;
};

__device__ __forceinline__ SlotIn slot_input(const QueryInput &in, uint64_t i)
{
    SlotIn s;
    bool ok = true;
#pragma unroll
    for (int k = 0; k < 8; k++) {
        s.c[k] = in.c[k][i];
        ok &= finite_bits(s.c[k]);
    }
    s.d = in.d_arr ? in.d_arr[i] : in.d;
    const double t0 = in.t0_arr ? in.t0_arr[i] : in.t0;
    const double t1 = in.t1_arr ? in.t1_arr[i] : in.t1;
    ok &= finite_bits(s.d) && ge0(s.d);
    ok &= !is_nan_bits(t0) && !is_nan_bits(t1);
    s.ks = okey(s.c[3]);
    const int64_t ke = okey(s.c[7]);
    ok &= ke > s.ks;
    const int64_t k0 = ok ? okey(t0) : 0, k1 = ok ? okey(t1) : 0;
    ok &= k0 <= k1;
    s.cs = max(s.ks, k0);
    s.ce = min(ke, k1);
    s.ok = ok;
    s.valid = ok && s.cs < s.ce;
    return s;
}

// A padding slot (at or beyond the real count): an empty span, no sphere,
// an empty range.
__device__ __forceinline__ void slot_padding(const PrepArgs &a, uint64_t i)
{
    a.pre[7][i] = __longlong_as_double(INT64_MAX);
    a.pre[8][i] = __longlong_as_double(INT64_MIN);
    a.pre_sph[i] = make_float4(0.f, 0.f, 0.f, 0.f);
}

// The arithmetic of one real slot: the pre columns (see kPreCols; keys
// stored bitwise in the double arrays), the FP32 bounding sphere (and with
// a.pre_tc the tensor-core record) and the ids.
__device__ __forceinline__ void slot_arith(const PrepArgs &a, uint64_t i, const SlotIn &s)
{
    double *const *pre = a.pre;
    const double *c = s.c;
    const bool valid = s.valid;
    const int64_t cs = s.cs, ce = s.ce;
    // one FP64 division per segment (the FP64 pipe is narrow)
    const double inv = 1.0 / (c[7] - c[3]);
    double vx = (c[4] - c[0]) * inv, vy = (c[5] - c[1]) * inv, vz = (c[6] - c[2]) * inv;
    double px = c[0], py = c[1], pz = c[2];
    if (valid && cs != s.ks) {  // the window cuts the start: position at the clipped start
        double shift = key_double(cs) - c[3];
        px = fma(vx, shift, px);
        py = fma(vy, shift, py);
        pz = fma(vz, shift, pz);
    }
    pre[0][i] = px; pre[1][i] = py; pre[2][i] = pz;
    pre[3][i] = vx; pre[4][i] = vy; pre[5][i] = vz;
    pre[6][i] = s.d * s.d;
    // invalid segments get the empty span (ts' >= te'), like padding
    pre[7][i] = __longlong_as_double(valid ? cs : INT64_MAX);
    pre[8][i] = __longlong_as_double(valid ? ce : INT64_MIN);
    // FP32 bounding sphere of the clipped segment, its radius widened by
    // d (and a relative 2^-30 of d): the pre-test of the filter mode
    float4 sp = make_float4(0.f, 0.f, 0.f, __int_as_float(0x7f800000));
    if (valid) {
        const double h = 0.5 * (key_double(ce) - key_double(cs));
        const float dw = __double2float_ru(s.d);
        sp = sphere32(fma(vx, h, px), fma(vy, h, py), fma(vz, h, pz), __fmul_ru(norm_ru(vx, vy, vz),
                      __double2float_ru(h)), __fmaf_ru(dw, 0x1p-30f, dw));
    }
    a.pre_sph[i] = sp;
    // tensor-core pre-test record of the clipped segment's sphere: center
    // and radius in FP64, snapped to the index's grid
    if (a.pre_tc && valid) {
        const double h = 0.5 * (key_double(ce) - key_double(cs));
        const double r = sqrt(fma(vz, vz, fma(vy, vy, vx * vx))) * h;
        uint4 lo, hi;
        tc_query_record(fma(vx, h, px), fma(vy, h, py), fma(vz, h, pz), r, s.d, a.grid, lo, hi);
        a.pre_tc[2 * i] = lo;
        a.pre_tc[2 * i + 1] = hi;
    }
    pre[kPreSeg][i] = __longlong_as_double(a.in.seg_id[i]);
    pre[kPreTraj][i] = __longlong_as_double(a.in.traj_id ? a.in.traj_id[i] : 0);
}

// The candidate range of one slot into the pre columns (kPreLo, kPreHi;
// empty for an invalid slot) and, with a.count_overlaps, its exact number
// of temporal-overlap pairs (returned); its sort key into `key`: the
// temporal bin of the clipped start (exact, found by the lookup), bins.m
// for an invalid segment (sorted last).
__device__ __forceinline__ unsigned long long slot_range(const PrepArgs &a, uint64_t i, bool valid, int64_t cs,
                                                         int64_t ce, uint64_t &key)
{
    int64_t rlo = INT64_MAX, rhi = INT64_MIN;
    unsigned long long n_overlap = 0;
    key = a.bins.m;
    if (valid) {
        int64_t bin = 0;
        candidate_range(a.bins, cs, ce, a.count_overlaps, rlo, rhi, n_overlap, bin);
        key = (uint64_t)bin;
        if (!TDQ_DBG(a.ctr, kDbgRange, rhi <= rlo || (rlo >= 0 && rhi <= (int64_t)a.n_entries))) {
            rlo = INT64_MAX;
            rhi = INT64_MIN;
        }
    }
    a.pre[kPreLo][i] = __longlong_as_double(rlo);
    a.pre[kPreHi][i] = __longlong_as_double(rhi);
    return n_overlap;
}

// Validate and clip every query segment into the pre columns, with its
// sort key and place: the counting sort's rank inside its bin, or the radix
// sort's first digit counts.  A block takes kPrepSlots slots in two roles:
// its first kPrepSlots threads do the arithmetic of a slot each
// (slot_arith: a chain of FP64 operations on the narrow FP64 pipe), the
// other kPrepSlots threads the candidate ranges of the same slots
// (slot_range: chains of dependent loads from the bin table) and, from the
// bin of the clipped start the lookup finds, the sort keys and places, so
// that the two chains run side by side rather than one after the other.
__global__ void __launch_bounds__(kBlock, 4) query_prep(PrepArgs a)
{
    static_assert(2 * kPrepSlots == kBlock, "two roles of kPrepSlots threads");
    const uint64_t nq = a.nq;
    DevCounters *ctr = a.ctr;
    const bool arith = threadIdx.x < kPrepSlots;
    const uint64_t i = (uint64_t)blockIdx.x * kPrepSlots + (threadIdx.x % kPrepSlots);
    bool valid = false;
    unsigned long long n_overlap = 0;
    uint32_t digit = 256;  // low byte of the sort key (256: not sorted)
    // slots at or beyond the device-side count are padding: empty, not errors
    const uint64_t nreal = a.in.n_real ? a.in.n_real : nq;
    if (i == 0 && arith) ctr->sort_n = nreal < nq ? nreal : nq;
    if (i < nq && arith) {
        if (i >= nreal) {
            slot_padding(a, i);
        } else {
            const SlotIn s = slot_input(a.in, i);
            if (!s.ok) atomicOr(&ctr->error, 1u);
            slot_arith(a, i, s);
            valid = s.valid;
        }
        if (!a.ranges) {  // an index without entries: nothing is sorted
            a.keys[i] = a.bins.m;
            a.vals[i] = (uint32_t)i;
        }
    } else if (i < nq && a.ranges) {
        bool v = false;
        int64_t cs = 0, ce = 0;
        if (i < nreal) {
            const SlotIn s = slot_input(a.in, i);
            v = s.valid;
            cs = s.cs;
            ce = s.ce;
        }
        uint64_t key;
        n_overlap = slot_range(a, i, v, cs, ce, key);
        a.keys[i] = key;
        if (i >= nreal) {
            a.vals[i] = (uint32_t)i;
        } else if (a.bin_cnt) {
            if (v) a.vals[i] = atomicAdd(&a.bin_cnt[key], 1u);
        } else {
            a.vals[i] = (uint32_t)i;
            digit = (uint32_t)(key & 0xff);
        }
    }
    // (the arithmetic threads count the valid segments, the range threads
    // the overlap pairs and the radix sort's digits)
    const unsigned vm = __ballot_sync(kFull, valid);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) n_overlap += __shfl_xor_sync(kFull, n_overlap, o);
    if ((threadIdx.x & 31) == 0) {
        if (vm) atomicAdd(&ctr->valid_queries, (unsigned long long)__popc(vm));
        if (n_overlap) atomicAdd(&ctr->overlap_pairs, n_overlap);
    }
    if (a.bin_cnt) {
        // the block that finishes last turns the bin counts into offsets
        __shared__ bool last;
        __threadfence();
        __syncthreads();
        if (threadIdx.x == 0) last = atomicAdd(&ctr->prep_done, 1ULL) == (unsigned long long)gridDim.x - 1;
        __syncthreads();
        if (last) {
            __threadfence();
            block_exclusive_scan<uint32_t, kBlock, 16>(a.bin_cnt, a.bins.m, nullptr);
        }
    } else if (a.sort_hist) {  // this block's keys lie in one sort tile (kPrepSlots divides kSortTileKeys)
        static_assert(kSortTileKeys % kPrepSlots == 0, "a block's slots lie in one sort tile");
        __shared__ uint32_t h[256];
        for (int d = threadIdx.x; d < 256; d += blockDim.x) h[d] = 0;
        __syncthreads();
        if (digit < 256) atomicAdd(&h[digit], 1u);
        __syncthreads();
        uint32_t *th = a.sort_hist + (uint64_t)blockIdx.x * kPrepSlots / kSortTileKeys * 256;
        for (int d = threadIdx.x; d < 256; d += blockDim.x)
            if (h[d]) atomicAdd(&th[d], h[d]);
    }
}

// A search of at most kSmallPrep query slots is prepared in one launch: each
// block prepares kSmallPrepWarps x 32 slots -- the first kSmallPrepWarps
// warps their arithmetic (slot_arith, one warp per scheduler of an SM, as
// the per-slot FP64 arithmetic is a long dependent chain on a narrow FP64
// pipe), the next kSmallPrepWarps warps their candidate ranges (slot_range)
// at the same time -- and the block that finishes last sorts the valid segments by (bin, slot) in shared
// memory, writes the sorted columns and plans the tiles.  This replaces the
// bin counters' clear and the three kernels of the multi-block preparation,
// whose fixed costs dominate small searches (a serving request).  The sort
// is a bitonic network over the 64-bit words (bin << 32 | slot), invalid
// slots all ones, on the next power of two above the slots: exchanges
// between lanes by shuffles, between warps through shared memory.
__global__ void __launch_bounds__(kSmallPrep) query_prep_small(SmallPrepArgs s)
{
    const PrepArgs &a = s.p;
    DevCounters *ctr = a.ctr;
    __shared__ unsigned long long sk[kSmallPrep];
    __shared__ unsigned long long tw[kSmallPrep / kQT];
    __shared__ int wv[kSmallPrep / 32];
    __shared__ bool last;
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const uint64_t nq = a.nq;  // at most kSmallPrep (host-checked)
    // slots at or beyond the device-side count are padding: not prepared, not sorted
    const uint64_t nreal = a.in.n_real && a.in.n_real < nq ? a.in.n_real : nq;
    if (warp < 2 * kSmallPrepWarps) {
        // warps 0 .. kSmallPrepWarps-1: the arithmetic of the block's slots;
        // the next kSmallPrepWarps warps: their candidate ranges (the two
        // chains side by side, as in query_prep)
        const bool arith = warp < kSmallPrepWarps;
        const uint64_t i = (uint64_t)blockIdx.x * (kSmallPrepWarps * 32) + (t % (kSmallPrepWarps * 32));
        bool valid = false;
        unsigned long long n_overlap = 0;
        if (i < nreal) {
            const SlotIn in = slot_input(a.in, i);
            if (arith) {
                if (!in.ok) atomicOr(&ctr->error, 1u);
                slot_arith(a, i, in);
                valid = in.valid;
            } else if (a.ranges) {
                uint64_t key;
                n_overlap = slot_range(a, i, in.valid, in.cs, in.ce, key);
                a.keys[i] = in.valid ? (key << 32) | i : ~0ull;  // sort word (bins.m < 2^32)
            }
        }
        const unsigned vm = __ballot_sync(kFull, valid);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) n_overlap += __shfl_xor_sync(kFull, n_overlap, o);
        if (lane == 0) {
            if (vm) atomicAdd(&ctr->valid_queries, (unsigned long long)__popc(vm));
            if (n_overlap) atomicAdd(&ctr->overlap_pairs, n_overlap);
        }
    }
    if (gridDim.x > 1) __threadfence();
    __syncthreads();
    // one block: it is the last; more: the one that finishes last goes on
    if (t == 0) last = gridDim.x == 1 || atomicAdd(&ctr->prep_done, 1ULL) == (unsigned long long)gridDim.x - 1;
    __syncthreads();
    if (!last) return;
    if (gridDim.x > 1) __threadfence();
    // the last block: every slot's pre columns and sort word are in place
    const int nvalid = (int)*(volatile unsigned long long *)&ctr->valid_queries;
    unsigned long long v = (uint64_t)t < nreal ? *(volatile unsigned long long *)&a.keys[t] : ~0ull;
    // The slots of a request come in time order, so that their bins are
    // mostly in order already: the valid words are compacted in slot order
    // (a block scan of the valid flags) and, if their bins never decrease,
    // that is the sorted order; else the network sorts them.
    const bool vt = v != ~0ull;
    const unsigned vb = __ballot_sync(kFull, vt);
    if (lane == 0) wv[warp] = __popc(vb);
    __syncthreads();
    int pos = __popc(vb & ((1u << lane) - 1u));
    for (int w = 0; w < warp; w++) pos += wv[w];
    if (vt) sk[pos] = v;
    __syncthreads();
    const bool in_order = __syncthreads_and(t + 1 >= nvalid || (sk[t] >> 32) <= (sk[t + 1] >> 32));
    int n2 = in_order ? 0 : 2;
    while (n2 && (uint64_t)n2 < nreal) n2 <<= 1;  // block-uniform
    if (in_order) v = t < nvalid ? sk[t] : ~0ull;
    for (int k = 2; k <= n2; k <<= 1) {
        for (int j = k >> 1; j > 0; j >>= 1) {
            unsigned long long o;
            if (j >= 32) {
                __syncthreads();  // the previous exchange's reads are done
                sk[t] = v;
                __syncthreads();
                o = sk[t ^ j];
            } else if ((warp << 5) < n2) {  // whole warps (lanes at or above n2 hold all ones)
                o = __shfl_xor_sync(kFull, v, j);
            } else {
                o = v;
            }
            // the lower slot of a pair keeps the minimum in an ascending run
            // (threads at or above n2 hold all ones among themselves)
            v = (((t & j) == 0) == ((t & k) == 0)) ? min(v, o) : max(v, o);
        }
    }
    // sorted position t: the slot of the t-th valid segment (in bin order)
    int64_t rlo = INT64_MAX, rhi = INT64_MIN;
    if (t < nvalid) {
        const uint32_t sl = (uint32_t)v;
        if (TDQ_DBG(ctr, kDbgSmallSlot, (uint64_t)sl < nreal)) {
            double *const *pre = s.cols;
            QuerySoA &q = s.q;
            q.px[t] = pre[0][sl]; q.py[t] = pre[1][sl]; q.pz[t] = pre[2][sl];
            q.vx[t] = pre[3][sl]; q.vy[t] = pre[4][sl]; q.vz[t] = pre[5][sl];
            q.d2[t] = pre[6][sl];
            q.ts_key[t] = __double_as_longlong(pre[7][sl]);
            q.te_key[t] = __double_as_longlong(pre[8][sl]);
            q.qid[t] = __double_as_longlong(pre[kPreSeg][sl]);
            if (q.qtraj) q.qtraj[t] = __double_as_longlong(pre[kPreTraj][sl]);
            q.sph[t] = a.pre_sph[sl];
            rlo = __double_as_longlong(pre[kPreLo][sl]);
            rhi = __double_as_longlong(pre[kPreHi][sl]);
            s.srt_lo[t] = rlo;
            s.srt_hi[t] = rhi;
        }
    }
    // tile plan: warp w plans tile w (the union of its members' ranges, cut
    // into chunks), then warp 0 turns the chunk counts into offsets
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        rlo = min(rlo, (int64_t)__shfl_xor_sync(kFull, (long long)rlo, o));
        rhi = max(rhi, (int64_t)__shfl_xor_sync(kFull, (long long)rhi, o));
    }
    const int ntiles = (int)((nq + kQT - 1) / kQT);
    if (lane == 0) {
        unsigned long long w = 0;
        if (warp < ntiles) {
            if (rhi > rlo) {
                w = (unsigned long long)((rhi - rlo + s.chunk - 1) / s.chunk);
            } else {
                rlo = 0;
                rhi = 0;
            }
            s.tile_lo[warp] = rlo;
            s.tile_hi[warp] = rhi;
        }
        tw[warp] = w;
    }
    __syncthreads();
    if (warp == 0) {
        const unsigned long long x = tw[lane];
        unsigned long long incl = x;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned long long y = __shfl_up_sync(kFull, incl, o);
            if (lane >= o) incl += y;
        }
        if (lane < ntiles) s.tile_work[lane] = incl - x;
        if (lane == 31) {
            s.tile_work[ntiles] = incl;
            ctr->work_items = incl;
            ctr->sort_n = nreal < nq ? nreal : nq;
        }
    }
}

// Copy of the search's counters into the caller-visible pinned host mirror
// (one warp; the counters are a few words).  A kernel, not a copy node: in a
// replayed graph the copy engine's round trip costs more than this launch.
static_assert(sizeof(DevCounters) % 8 == 0, "counters are copied as 64-bit words");
__global__ void publish_counters(const DevCounters *src, DevCounters *dst)
{
    const unsigned long long *s = reinterpret_cast<const unsigned long long *>(src);
    unsigned long long *d = reinterpret_cast<unsigned long long *>(dst);
    for (int i = threadIdx.x; i < (int)(sizeof(DevCounters) / 8); i += 32) d[i] = s[i];
}

// Counting sort, second half: every valid query segment's columns go to
// its sorted position (its bin's offset plus its place in the bin), with its
// candidate range for the tile plan.  Segments of one bin keep no
// particular order (a tile groups segments of nearby bins whatever their
// order; results come in no particular order anyway).
__global__ void query_scatter(ScatterArgs a)
{
    const uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= a.nq) return;
    const int64_t ts = __double_as_longlong(a.pre[7][i]), te = __double_as_longlong(a.pre[8][i]);
    if (!(ts < te)) return;  // invalid or padding: not sorted
    const uint64_t k = (uint64_t)a.bin_off[a.keys[i]] + a.ranks[i];
    if (!TDQ_DBG(a.ctr, kDbgScatterPos, k < a.ctr->valid_queries)) return;
    QuerySoA &q = a.q;
    q.px[k] = a.pre[0][i]; q.py[k] = a.pre[1][i]; q.pz[k] = a.pre[2][i];
    q.vx[k] = a.pre[3][i]; q.vy[k] = a.pre[4][i]; q.vz[k] = a.pre[5][i];
    q.d2[k] = a.pre[6][i];
    q.ts_key[k] = ts;
    q.te_key[k] = te;
    q.qid[k] = __double_as_longlong(a.pre[kPreSeg][i]);
    if (q.qtraj) q.qtraj[k] = __double_as_longlong(a.pre[kPreTraj][i]);
    q.sph[k] = a.pre_sph[i];
    a.srt_lo[k] = __double_as_longlong(a.pre[kPreLo][i]);
    a.srt_hi[k] = __double_as_longlong(a.pre[kPreHi][i]);
    if (a.q_rec) tc_store(a.q_rec, k, a.pre_tc[2 * i], a.pre_tc[2 * i + 1]);
}

// Sorted query SoA; then, one warp per tile of kQT consecutive sorted query
// segments, the tile plan: the tile's entry range is the union of its
// members' candidate ranges, cut into chunks of `chunk` entries, one work item
// per (tile, chunk).  The block that finishes last turns the per-tile chunk
// counts into exclusive offsets (the total into the counters).
__global__ void query_gather(GatherArgs a)
{
    const uint64_t k = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    QuerySoA &q = a.q;
    int64_t rlo = INT64_MAX, rhi = INT64_MIN;
    if (a.srt_lo) {
        // the sorted columns are in place (query_scatter): the ranges only
        if (k < a.nq && k < a.ctr->valid_queries) {
            rlo = a.srt_lo[k];
            rhi = a.srt_hi[k];
        }
    } else if (k < a.nq && k < a.ctr->valid_queries && TDQ_DBG(a.ctr, kDbgGatherOrder, a.order[k] < a.nq)) {
        const uint32_t i = a.order[k];
        q.px[k] = a.pre[0][i]; q.py[k] = a.pre[1][i]; q.pz[k] = a.pre[2][i];
        q.vx[k] = a.pre[3][i]; q.vy[k] = a.pre[4][i]; q.vz[k] = a.pre[5][i];
        q.d2[k] = a.pre[6][i];
        q.ts_key[k] = __double_as_longlong(a.pre[7][i]);
        q.te_key[k] = __double_as_longlong(a.pre[8][i]);
        q.qid[k] = __double_as_longlong(a.pre[kPreSeg][i]);
        if (q.qtraj) q.qtraj[k] = __double_as_longlong(a.pre[kPreTraj][i]);
        q.sph[k] = a.pre_sph[i];
        rlo = __double_as_longlong(a.pre[kPreLo][i]);
        rhi = __double_as_longlong(a.pre[kPreHi][i]);
    }
    // tensor-core records in sorted order (written by query_scatter when
    // srt_lo is given); zero records fill the last supertile
    if (a.q_rec && k < a.nsuper * 128) {
        const bool real = k < a.nq && k < a.ctr->valid_queries;
        if (!real) {
            tc_store(a.q_rec, k, make_uint4(0u, 0u, 0u, 0u), make_uint4(0u, 0u, 0u, 0u));
        } else if (!a.srt_lo) {
            const uint32_t i = a.order[k];
            tc_store(a.q_rec, k, a.pre_tc[2 * i], a.pre_tc[2 * i + 1]);
        }
    }
    // the tile plan: this warp's 32 sorted query segments are tile k / kQT
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        rlo = min(rlo, (int64_t)__shfl_xor_sync(kFull, (long long)rlo, o));
        rhi = max(rhi, (int64_t)__shfl_xor_sync(kFull, (long long)rhi, o));
    }
    // supertiles (tensor-core pre-test): the union of 4 consecutive tiles'
    // ranges, from the block's 8 warps (two supertiles per block)
    static_assert(kBlock == 8 * 32, "two supertiles of 4 warps per block");
    __shared__ int64_t w_lo[8], w_hi[8];
    if (a.q_rec && lane == 0) {
        w_lo[threadIdx.x >> 5] = rlo;
        w_hi[threadIdx.x >> 5] = rhi;
    }
    const uint64_t t = k / kQT;
    if (lane == 0 && t < a.ntiles) {
        unsigned long long w = 0;
        if (rhi > rlo) {
            w = (unsigned long long)((rhi - rlo + a.chunk - 1) / a.chunk);
        } else {
            rlo = 0;
            rhi = 0;
        }
        a.tile_lo[t] = rlo;
        a.tile_hi[t] = rhi;
        a.tile_work[t] = w;
        if (t == 0) a.tile_work[a.ntiles] = 0;  // the scan turns this slot into the total
    }
    if (a.q_rec) {
        __syncthreads();
        const uint64_t st = k / 128;
        if ((threadIdx.x & 127) == 0 && st < a.nsuper) {
            int64_t lo = INT64_MAX, hi = INT64_MIN;
            const int w0 = threadIdx.x >> 5;
            for (int w = w0; w < w0 + 4; w++) {
                if (w_hi[w] > w_lo[w]) {
                    lo = min(lo, w_lo[w]);
                    hi = max(hi, w_hi[w]);
                }
            }
            unsigned long long wk = 0;
            if (hi > lo) {
                wk = (unsigned long long)((hi - lo + a.chunk - 1) / a.chunk);
            } else {
                lo = 0;
                hi = 0;
            }
            a.st_lo[st] = lo;
            a.st_hi[st] = hi;
            a.st_work[st] = wk;
            if (st == 0) a.st_work[a.nsuper] = 0;  // the scan turns this slot into the total
        }
    }
    __shared__ bool last;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) last = atomicAdd(&a.ctr->gather_done, 1ULL) == (unsigned long long)gridDim.x - 1;
    __syncthreads();
    if (last) {
        __threadfence();
        if (a.q_rec)
            block_exclusive_scan<unsigned long long, kBlock, 8>(a.st_work, a.nsuper + 1, &a.ctr->work_items);
        else
            block_exclusive_scan<unsigned long long, kBlock, 8>(a.tile_work, a.ntiles + 1, &a.ctr->work_items);
    }
}

namespace {

// n-th (0-based) set bit of m; m must have more than r bits set.
__device__ __forceinline__ int nth_set_bit(unsigned m, int r)
{
    int p = 0;
#pragma unroll
    for (int s = 16; s >= 1; s >>= 1) {
        int c = __popc(m & ((1u << s) - 1u));
        if (r >= c) {
            r -= c;
            m >>= s;
            p += s;
        }
    }
    return p;
}

// Shared-memory staging of one work item.
struct PairSmem {
    double qp[3][kQT], qv[3][kQT], qd2[kQT];
    int64_t qts[kQT], qte[kQT], qid[kQT], qtraj[kQT];
    long long item;
    long long tile;
    // followed by the entry chunk: 6 double columns + 2 key columns of
    // `chunk` items (the plain FP64 kernel)
};

// GPUTrajDistSearch (Sec. 5, Algorithm 1), tiled: one work item is a tile of
// 32 sorted query segments against a chunk of the tile's candidate entries.
// Every temporal-overlap pair is evaluated in FP64 (the plain method).
__global__ void __launch_bounds__(kPairThreads) traj_dist_search_kernel(PairArgs args)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    PairSmem &S = *reinterpret_cast<PairSmem *>(smem_raw);
    const uint32_t EC = args.chunk;
    unsigned char *ebase = smem_raw + ((sizeof(PairSmem) + 15) & ~(size_t)15);
    // entry chunk columns
    int64_t *ets = reinterpret_cast<int64_t *>(ebase);
    int64_t *ete = ets + EC;
    double *ecol = reinterpret_cast<double *>(ete + EC);
    double *epx = ecol, *epy = ecol + EC, *epz = ecol + 2 * EC;
    double *evx = ecol + 3 * EC, *evy = ecol + 4 * EC, *evz = ecol + 5 * EC;

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const unsigned lt_mask = (1u << lane) - 1u;
    DevCounters *ctr = args.ctr;
    const unsigned long long total = args.tile_work[args.ntiles];
    const uint64_t nvalid = ctr->valid_queries;
    const uint64_t cap = args.out.capacity;

    unsigned long long n_inter = 0, n_overlap = 0;

    for (;;) {
        if (tid == 0) {
            long long item = (long long)atomicAdd(&ctr->work_next, 1ULL);
            long long t = -1;
            if ((unsigned long long)item < total) {
                // last tile whose first work item is <= item
                uint64_t lo = 0, hi = args.ntiles;
                while (hi - lo > 1) {
                    uint64_t mid = (lo + hi) >> 1;
                    if (args.tile_work[mid] <= (unsigned long long)item) lo = mid; else hi = mid;
                }
                t = (long long)lo;
            }
            S.item = item;
            S.tile = t;
        }
        __syncthreads();
        const long long item = S.item;
        if ((unsigned long long)item >= total) break;
        const uint64_t t = (uint64_t)S.tile;
        if (!TDQ_DBG(ctr, kDbgPlainTile, t < args.ntiles)) break;  // (S.tile: the block agrees)
        const int64_t e0 = args.tile_lo[t] + (int64_t)(item - (long long)args.tile_work[t]) * EC;
        const int64_t e1 = min(e0 + (int64_t)EC, args.tile_hi[t]);
        const int ne = (int)(e1 - e0);
        const uint64_t q0 = t * kQT;
        const int nqt = (int)min((uint64_t)kQT, nvalid - q0);
        if (!TDQ_DBG(ctr, kDbgPlainChunk, e0 >= 0 && e0 < e1 && e1 <= (int64_t)args.n_entries)) break;
        if (!TDQ_DBG(ctr, kDbgPlainQueries, nqt > 0 && q0 + nqt <= args.nq_slots)) break;

        // stage the tile's query segments
        if (tid < kQT) {
            if (tid < nqt) {
                uint64_t k = q0 + tid;
                S.qp[0][tid] = args.q.px[k]; S.qp[1][tid] = args.q.py[k]; S.qp[2][tid] = args.q.pz[k];
                S.qv[0][tid] = args.q.vx[k]; S.qv[1][tid] = args.q.vy[k]; S.qv[2][tid] = args.q.vz[k];
                S.qd2[tid] = args.q.d2[k];
                S.qts[tid] = args.q.ts_key[k];
                S.qte[tid] = args.q.te_key[k];
                S.qid[tid] = args.q.qid[k];
                S.qtraj[tid] = args.flags ? args.q.qtraj[k] : 0;
            } else {  // padding: a span that overlaps nothing
                S.qts[tid] = INT64_MAX;
                S.qte[tid] = INT64_MIN;
            }
        }
        // stage the chunk's entry segments (coalesced column loads)
        for (int i = tid; i < (int)EC; i += kPairThreads) {
            if (i < ne) {
                int64_t k = e0 + i;
                ets[i] = args.e.ts_key[k];
                ete[i] = args.e.te_key[k];
                epx[i] = args.e.px[k]; epy[i] = args.e.py[k]; epz[i] = args.e.pz[k];
                evx[i] = args.e.vx[k]; evy[i] = args.e.vy[k]; evz[i] = args.e.vz[k];
            } else {
                ets[i] = INT64_MAX;
                ete[i] = INT64_MIN;
            }
        }
        if (tid == 0) n_inter += (unsigned long long)ne * (unsigned long long)nqt;
        __syncthreads();

        for (int g = 0; g < (int)EC; g += kPairThreads) {
            const int el = g + warp * 32 + lane;
            // temporal intersection of this lane's entry with every query of
            // the tile, as a 32-bit mask (integer keys: strict overlap a < b)
            const int64_t my_ts = ets[el], my_te = ete[el];
            unsigned mask = 0;
#pragma unroll
            for (int j = 0; j < kQT; j++) {
                bool ov = (my_ts < S.qte[j]) & (my_te > S.qts[j]);
                mask |= (unsigned)ov << j;
            }
            const int cnt = __popc(mask);
            int incl = cnt;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                int y = __shfl_up_sync(kFull, incl, o);
                if (lane >= o) incl += y;
            }
            const int excl = incl - cnt;
            const int npairs = __shfl_sync(kFull, incl, 31);
            if (lane == 0) n_overlap += (unsigned long long)npairs;

            // evaluate the selected pairs 32 at a time, one per lane
            for (int base = 0; base < npairs; base += 32) {
                const int kk = base + lane;
                const bool active = kk < npairs;
                int owner = 0;
#pragma unroll
                for (int s = 16; s >= 1; s >>= 1) {
                    int v = __shfl_sync(kFull, incl, owner + s - 1);
                    if (v <= kk) owner += s;
                }
                const unsigned mo = __shfl_sync(kFull, mask, owner);
                const int eo = __shfl_sync(kFull, excl, owner);
                const int j = active ? nth_set_bit(mo, kk - eo) : 0;
                const int ei = active ? (g + warp * 32 + owner) : el;

                PairEval r = eval_pair_fp64(active, ets[ei], ete[ei], S.qts[j], S.qte[j], epx[ei], epy[ei],
                                            epz[ei], evx[ei], evy[ei], evz[ei], S.qp[0][j], S.qp[1][j],
                                            S.qp[2][j], S.qv[0][j], S.qv[1][j], S.qv[2][j], S.qd2[j]);
                const int64_t eseg = active ? args.e.seg_id[e0 + ei] : 0;
                if (args.flags && r.hit)
                    r.hit = pair_allowed(args.flags, S.qtraj[j], S.qid[j], args.e.traj_id[e0 + ei], eseg);
                append_hits(r, ctr, args.out, cap, S.qid[j], eseg, lane, lt_mask);
            }
        }
        __syncthreads();  // the chunk is about to be restaged
    }
    // counters: one atomic per warp
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        n_inter += __shfl_xor_sync(kFull, n_inter, o);
        n_overlap += __shfl_xor_sync(kFull, n_overlap, o);
    }
    if (lane == 0) {
        if (n_inter) atomicAdd(&ctr->interactions, n_inter);
        if (n_overlap) {
            atomicAdd(&ctr->overlap_pairs, n_overlap);
            atomicAdd(&ctr->fp64_pairs, n_overlap);
        }
    }
    publish_when_last(ctr, args.publish);
}

size_t pair_smem_bytes(uint32_t chunk)
{
    return ((sizeof(PairSmem) + 15) & ~(size_t)15) + (size_t)chunk * 64;
}

}  // namespace

// Launch the pair kernel of the requested mode as a persistent grid (as many
// CTAs as fit on every SM at once).  Filter mode: the FP32 pre-test kernel,
// then the FP64 refine kernel over its survivors.  Neither counts the
// overlapping pairs: query_prep does.
// mid (filter mode, may be null): event recorded between the filter and the
// refine kernel with the flags evflags.
cudaError_t launch_pair_kernel(const PairArgs &pa, bool filter, int sm_count, uint2 *surv, uint64_t surv_cap,
                               cudaStream_t stream, cudaEvent_t mid, unsigned evflags, bool inline_refine,
                               const int64_t *q_lo, const int64_t *q_hi)
{
    if (filter)
        return launch_filter_kernels(FilterArgs{pa, surv, surv_cap, q_lo, q_hi}, sm_count, stream, mid, evflags,
                                     inline_refine);
    const size_t smem = pair_smem_bytes(pa.chunk);
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(traj_dist_search_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
        if (e != cudaSuccess) return e;
    }
    int per_sm = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, traj_dist_search_kernel, kPairThreads, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) per_sm = 1;
    traj_dist_search_kernel<<<sm_count * per_sm, kPairThreads, smem, stream>>>(pa);
    return cudaGetLastError();
}



tdq_status ensure_queries(Workspace &w, uint64_t nq, uint32_t m)
{
    if (m <= kCountSortMaxBins && m > w.bin_cap) {
        cudaFree(w.bin_cnt);
        w.bin_cnt = nullptr;
        w.bin_cap = 0;
        if (dev_alloc(&w.bin_cnt, (uint64_t)m * sizeof(uint32_t)) != cudaSuccess) {
            cudaGetLastError();
            return set_error(TDQ_ERR_NOMEM, "search workspace: device allocation of %u bin counters failed", m);
        }
        w.bin_cap = m;
    }
    if (nq <= w.q_cap && w.q_block) return TDQ_OK;
    uint64_t cap = nq > 2 * w.q_cap ? nq : 2 * w.q_cap;
    if (cap < 1024) cap = 1024;
    uint64_t bytes = 10 * carve_bytes(cap, 8)                   // staged host input
                     + kPreCols * carve_bytes(cap, 8)           // pre
                     + 2 * carve_bytes(cap, 8) + 2 * carve_bytes(cap, 4) // sort
                     + 11 * carve_bytes(cap, 8)                 // sorted query SoA
                     + 2 * carve_bytes(cap, 16)                 // query spheres (before / after sorting)
                     + 2 * carve_bytes(cap, 8)                  // candidate ranges in sorted order
                     + carve_bytes(2 * cap, 16)                 // tensor-core records before sorting
                     + carve_bytes(2 * ((cap + 127) / 128 * 128), 16)  // ... sorted, whole supertiles
                     + carve_bytes(kPreCols, sizeof(double *)); // pre pointer table
    uint64_t ntiles = (cap + kQT - 1) / kQT;
    uint64_t nsuper = (cap + 127) / 128;
    uint64_t tbytes = 2 * carve_bytes(ntiles, 8) + carve_bytes(ntiles + 1, 8) + 2 * carve_bytes(nsuper, 8) +
                      carve_bytes(nsuper + 1, 8);
    uint64_t hwords = sort_hist_words(cap);
    cudaFree(w.q_block);
    cudaFree(w.t_block);
    cudaFree(w.sort_hist);
    w.q_block = w.t_block = nullptr;
    w.sort_hist = nullptr;
    w.q_cap = 0;
    if (dev_alloc(&w.q_block, bytes) != cudaSuccess || dev_alloc(&w.t_block, tbytes) != cudaSuccess ||
        dev_alloc(&w.sort_hist, hwords * 4) != cudaSuccess) {
        cudaGetLastError();
        cudaFree(w.q_block);
        cudaFree(w.t_block);
        cudaFree(w.sort_hist);
        w.q_block = w.t_block = nullptr;
        w.sort_hist = nullptr;
        return set_error(TDQ_ERR_NOMEM, "search workspace: device allocation of %llu bytes failed",
                         (unsigned long long)(bytes + tbytes + hwords * 4));
    }
    char *p = (char *)w.q_block;
    for (int c = 0; c < 8; c++) w.in_cols[c] = carve<double>(p, cap);
    w.in_seg = carve<int64_t>(p, cap);
    w.in_traj = carve<int64_t>(p, cap);
    for (int c = 0; c < kPreCols; c++) w.pre[c] = carve<double>(p, cap);
    w.keys = carve<uint64_t>(p, cap);
    w.keys_alt = carve<uint64_t>(p, cap);
    w.vals = carve<uint32_t>(p, cap);
    w.vals_alt = carve<uint32_t>(p, cap);
    QuerySoA &q = w.q;
    q.px = carve<double>(p, cap); q.py = carve<double>(p, cap); q.pz = carve<double>(p, cap);
    q.vx = carve<double>(p, cap); q.vy = carve<double>(p, cap); q.vz = carve<double>(p, cap);
    q.d2 = carve<double>(p, cap);
    q.ts_key = carve<int64_t>(p, cap); q.te_key = carve<int64_t>(p, cap);
    q.qid = carve<int64_t>(p, cap);
    q.qtraj = carve<int64_t>(p, cap);
    w.pre_sph = carve<float4>(p, cap);
    q.sph = carve<float4>(p, cap);
    w.srt_lo = carve<int64_t>(p, cap);
    w.srt_hi = carve<int64_t>(p, cap);
    w.pre_tc = carve<uint4>(p, 2 * cap);
    q.tc_rec = carve<uint4>(p, 2 * ((cap + 127) / 128 * 128));
    w.pre_dev = carve<double *>(p, kPreCols);
    if (cudaMemcpy(w.pre_dev, w.pre, kPreCols * sizeof(double *), cudaMemcpyHostToDevice) != cudaSuccess)
        return cuda_error(cudaGetLastError(), "search workspace: pointer table");
    char *tp = (char *)w.t_block;
    w.tile_lo = carve<int64_t>(tp, ntiles);
    w.tile_hi = carve<int64_t>(tp, ntiles);
    w.tile_work = carve<unsigned long long>(tp, ntiles + 1);
    w.st_lo = carve<int64_t>(tp, nsuper);
    w.st_hi = carve<int64_t>(tp, nsuper);
    w.st_work = carve<unsigned long long>(tp, nsuper + 1);
    w.q_cap = cap;
    w.t_cap = ntiles;
    w.s_cap = hwords;
    return TDQ_OK;
}

tdq_status ensure_survivors(Workspace &w, uint64_t cap)
{
    if (cap <= w.s_cap_pairs && w.s_block) return TDQ_OK;
    cudaFree(w.s_block);
    w.s_block = nullptr;
    w.surv = nullptr;
    w.s_cap_pairs = 0;
    if (dev_alloc(&w.s_block, cap * sizeof(uint2)) != cudaSuccess) {
        cudaGetLastError();
        return set_error(TDQ_ERR_NOMEM, "tdq_search: survivor list of %llu pairs", (unsigned long long)cap);
    }
    w.surv = (uint2 *)w.s_block;
    w.s_cap_pairs = cap;
    return TDQ_OK;
}

tdq_status parse_params(const tdq_search_params *params, LaunchCfg *cfg)
{
    if (params && params->mode != TDQ_MODE_FP64 && params->mode != TDQ_MODE_FP32_FILTER &&
        params->mode != TDQ_MODE_TC_FILTER)
        return set_error(TDQ_ERR_INVALID, "tdq_search: unknown mode %d", params->mode);
    cfg->filter = params && (params->mode == TDQ_MODE_FP32_FILTER || params->mode == TDQ_MODE_TC_FILTER);
    cfg->tc = params && params->mode == TDQ_MODE_TC_FILTER;
    cfg->flags = params ? params->flags : 0u;
    if (cfg->flags & ~(TDQ_FLAG_OTHER_TRAJECTORIES | TDQ_FLAG_UNORDERED_ONCE))
        return set_error(TDQ_ERR_INVALID, "tdq_search: unknown flags 0x%x", cfg->flags);
    cfg->chunk = (params && params->entry_chunk) ? params->entry_chunk : 512u;
    if (cfg->chunk % kPairThreads != 0 || cfg->chunk > 2048)
        return set_error(TDQ_ERR_INVALID, "tdq_search: entry_chunk must be a multiple of 256, at most 2048");
    if (params && params->query_tile && params->query_tile != (uint32_t)kQT)
        return set_error(TDQ_ERR_INVALID, "tdq_search: query_tile must be 32");
    return TDQ_OK;
}

namespace {

// Whether a search of nq query slots is prepared by query_prep_small (not
// for the tensor-core pre-test, whose supertile records and plan come from
// the multi-block preparation).
bool small_prep(const tdq_index *idx, const LaunchCfg &cfg, uint64_t nq)
{
    return idx->n > 0 && !cfg.tc && nq >= 1 && nq <= (uint64_t)kSmallPrep;
}

// The preparation kernel's arguments (a launch and the re-binding of a
// captured one build them here alike).
PrepArgs prep_args(const tdq_index *idx, Workspace &w, const QueryInput &in, uint64_t nq, const LaunchCfg &cfg)
{
    const bool csort = idx->n > 0 && idx->m <= kCountSortMaxBins;
    const bool fuse = !csort && idx->n > 0 && sort_fusable(nq);
    const bool tc = cfg.tc && idx->n > 0;
    return PrepArgs{in, nq, bin_view(idx), w.pre_dev, w.pre_sph, w.keys, w.vals, w.ctr,
                    fuse ? w.sort_fused_hist : nullptr, idx->n > 0, cfg.filter, tc ? w.pre_tc : nullptr, idx->grid,
                    csort ? w.bin_cnt : nullptr, idx->n};
}

unsigned small_prep_blocks(uint64_t nq)
{
    const uint64_t per = (uint64_t)kSmallPrepWarps * 32;
    return (unsigned)((nq + per - 1) / per);
}

SmallPrepArgs small_prep_args(const tdq_index *idx, Workspace &w, const QueryInput &in, uint64_t nq,
                              const LaunchCfg &cfg)
{
    PrepArgs p{in, nq, bin_view(idx), w.pre_dev, w.pre_sph, w.keys, nullptr, w.ctr, nullptr, true, cfg.filter,
               nullptr, idx->grid, nullptr, idx->n};
    SmallPrepArgs sa{p, {}, w.q, w.tile_lo, w.tile_hi, w.tile_work, w.srt_lo, w.srt_hi, cfg.chunk};
    for (int c = 0; c < kPreCols; c++) sa.cols[c] = w.pre[c];
    return sa;
}

}  // namespace

int search_kernel_launches(const tdq_index *idx, const LaunchCfg &cfg, uint64_t nq)
{
    if (small_prep(idx, cfg, nq)) return 2;  // query_prep_small, the pair kernel (refining its own survivors)
    // without entries: query_prep and publish_counters; with entries:
    // query_prep, the sort of the query keys (counting sort: query_scatter;
    // else the radix sort's kernels), query_gather and the pair kernel
    // (filter modes: the pre-test and the refine kernel), whose last block
    // publishes the counters; a small search: query_prep_small and the pair
    // kernel
    const int sort = idx->m <= kCountSortMaxBins ? 1 : sort_kernel_launches(nq, bin_key_bits(idx->m), true);
    return idx->n > 0 ? 2 + sort + (cfg.filter ? 2 : 1) : 2;
}

// Events are recorded as external event-record nodes when the stream is being
// captured, so the timings stay valid inside a replayed CUDA graph.
cudaError_t enqueue_search(const tdq_index *idx, Workspace &w, const QueryInput &in, uint64_t nq, const LaunchCfg &cfg,
                           const tdq_result_buffer &out, cudaStream_t stream, bool events)
{
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    cudaError_t e = cudaStreamIsCapturing(stream, &cs);
    if (e != cudaSuccess) return e;
    const unsigned evflags = cs == cudaStreamCaptureStatusActive ? cudaEventRecordExternal : cudaEventRecordDefault;
    // the counters, and with the radix sort's small path its two fused
    // histograms (counting sort: the bin counts)
    const bool small = small_prep(idx, cfg, nq);
    const bool csort = !small && idx->n > 0 && idx->m <= kCountSortMaxBins;
    if (csort && (!w.bin_cnt || w.bin_cap < idx->m)) return cudaErrorInvalidValue;  // workspace not sized
    const bool fuse = !small && !csort && idx->n > 0 && sort_fusable(nq);
    const uint64_t sort_tiles = (nq + kSortTileKeys - 1) / kSortTileKeys;
    e = cudaMemsetAsync(w.ctr, 0, fuse ? kCtrBytes + 2 * sort_tiles * 256 * sizeof(uint32_t) : sizeof(DevCounters),
                        stream);
    if (e != cudaSuccess) return e;
    if (csort && (e = cudaMemsetAsync(w.bin_cnt, 0, (size_t)idx->m * sizeof(uint32_t), stream)) != cudaSuccess)
        return e;
    if (events && (e = cudaEventRecordWithFlags(w.ev[0], stream, evflags)) != cudaSuccess) return e;
    double *const *pre = w.pre_dev;
    const bool tc = cfg.tc && idx->n > 0;
    if (small)
        query_prep_small<<<small_prep_blocks(nq), kSmallPrep, 0, stream>>>(small_prep_args(idx, w, in, nq, cfg));
    else
        query_prep<<<prep_grid(nq), kBlock, 0, stream>>>(prep_args(idx, w, in, nq, cfg));
    const uint64_t ntiles = (nq + kQT - 1) / kQT;
    const uint64_t nsuper = (nq + 127) / 128;
    if (idx->n > 0) {
        if (small) {
            // sorted and planned already
        } else if (csort) {
            query_scatter<<<grid_for(nq), kBlock, 0, stream>>>(ScatterArgs{
                pre, w.pre_sph, w.pre_tc, w.keys, w.vals, w.bin_cnt, nq, w.q, tc ? w.q.tc_rec : nullptr, w.srt_lo,
                w.srt_hi, w.ctr});
        } else if ((e = radix_sort_pairs(w.keys, w.vals, w.keys_alt, w.vals_alt, nq, w.sort_hist, stream,
                                         bin_key_bits(idx->m), &w.ctr->sort_n,
                                         fuse ? w.sort_fused_hist : nullptr)) != cudaSuccess) {
            return e;
        }
        if (!small) {
            const GatherArgs ga{pre, w.pre_sph, w.vals, nq, w.ctr, w.q, ntiles, cfg.chunk, w.tile_lo, w.tile_hi,
                                w.tile_work, w.pre_tc, tc ? w.q.tc_rec : nullptr, w.st_lo, w.st_hi, w.st_work, nsuper,
                                csort ? w.srt_lo : nullptr, csort ? w.srt_hi : nullptr};
            query_gather<<<grid_for(tc ? nsuper * 128 : nq), kBlock, 0, stream>>>(ga);
        }
        PairArgs pa{idx->e, w.q, w.tile_lo, w.tile_hi, w.tile_work, ntiles, w.ctr, out, cfg.chunk, cfg.flags,
                    w.ctr_host_dev, idx->n, nq};
        if (events && (e = cudaEventRecordWithFlags(w.ev[1], stream, evflags)) != cudaSuccess) return e;
        if (tc)
            e = launch_tc_filter_kernels(TcArgs{pa, idx->e.tc_rec, w.q.tc_rec, w.st_lo, w.st_hi, w.st_work, nsuper,
                                                w.surv, w.s_cap_pairs, idx->n_rec},
                                         idx->sm_count, stream, events ? w.ev[2] : nullptr, evflags);
        else
            e = launch_pair_kernel(pa, cfg.filter, idx->sm_count, w.surv, w.s_cap_pairs, stream,
                                   events ? w.ev[2] : nullptr, evflags, small, small ? w.srt_lo : nullptr,
                                   small ? w.srt_hi : nullptr);
        if (e != cudaSuccess) return e;
        if (events && (e = cudaEventRecordWithFlags(cfg.filter ? w.ev[4] : w.ev[2], stream, evflags)) != cudaSuccess)
            return e;
    } else {
        if (events)
            for (int k : {1, 2, 4})
                if ((e = cudaEventRecordWithFlags(w.ev[k], stream, evflags)) != cudaSuccess) return e;
        publish_counters<<<1, 32, 0, stream>>>(w.ctr, w.ctr_host_dev);
    }
    if (events && (e = cudaEventRecordWithFlags(w.ev[3], stream, evflags)) != cudaSuccess) return e;
    return cudaGetLastError();
}

tdq_status finish_search(const tdq_index *idx, const Workspace &w, const LaunchCfg &cfg, uint64_t nq,
                         uint64_t capacity, bool events, tdq_stats *s, uint64_t *count, bool *surv_overflow)
{
    const DevCounters &h = *w.ctr_host;
    *surv_overflow = false;
    if (h.error & 1u)
        return set_error(TDQ_ERR_INVALID,
                         "tdq_search: invalid query segment (non-finite value, t_end <= t_start, d < 0 or NaN, "
                         "NaN window or t0 > t1)");
    if (h.error & 4u)
        return set_error(TDQ_ERR_CUDA, "tdq_search: debug build: index bounds check at site %u failed", h.debug_site);
    if (h.error & 2u)
        return set_error(TDQ_ERR_TIMEOUT,
                         "tdq_search: a wait of the tensor-core pre-test pipeline ran out of time (the search "
                         "was abandoned; its results are incomplete)");
    // (a small search's FP32 pre-test refines its survivors in place; else they are listed)
    if (cfg.filter && !small_prep(idx, cfg, nq) && h.survivors > w.s_cap_pairs) {
        *surv_overflow = true;
        return TDQ_OK;
    }
    *s = tdq_stats{};
    s->query_segments = h.valid_queries;
    s->interactions = h.interactions;
    s->overlap_pairs = h.overlap_pairs;
    s->fp64_pairs = h.fp64_pairs;
    s->results = h.results;
    s->work_items = h.work_items;
    s->filter_survivors = cfg.filter ? h.survivors : 0;
    s->mma_issued = h.mma_issued;
    s->kernel_launches = (uint64_t)search_kernel_launches(idx, cfg, nq);
    if (events) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, w.ev[1], w.ev[2]) == cudaSuccess) s->pair_kernel_ms = ms;
        if (cfg.filter && cudaEventElapsedTime(&ms, w.ev[2], w.ev[4]) == cudaSuccess) s->refine_ms = ms;
        if (cudaEventElapsedTime(&ms, w.ev[0], w.ev[3]) == cudaSuccess) s->total_ms = ms;
    }
    *count = h.results;
    return h.results > capacity ? TDQ_ERR_OVERFLOW : TDQ_OK;
}

cudaError_t find_input_nodes(cudaGraph_t g, GraphInputNodes *out)
{
    size_t n = 0;
    cudaError_t e = cudaGraphGetNodes(g, nullptr, &n);
    if (e != cudaSuccess) return e;
    cudaGraphNode_t *nodes = (cudaGraphNode_t *)malloc((n ? n : 1) * sizeof(cudaGraphNode_t));
    if (!nodes) return cudaErrorMemoryAllocation;
    e = cudaGraphGetNodes(g, nodes, &n);
    *out = GraphInputNodes{};
    for (size_t k = 0; k < n && e == cudaSuccess; k++) {
        cudaGraphNodeType t;
        if ((e = cudaGraphNodeGetType(nodes[k], &t)) != cudaSuccess || t != cudaGraphNodeTypeKernel) continue;
        cudaKernelNodeParams kp;
        if ((e = cudaGraphKernelNodeGetParams(nodes[k], &kp)) != cudaSuccess) break;
        if (kp.func == (void *)query_prep || kp.func == (void *)query_prep_small) out->prep = nodes[k];
    }
    free(nodes);
    if (e == cudaSuccess && !out->prep) e = cudaErrorInvalidValue;
    return e;
}

cudaError_t bind_inputs(cudaGraphExec_t exec, const GraphInputNodes &nodes, const tdq_index *idx, Workspace &w,
                        const QueryInput &in, uint64_t nq, const LaunchCfg &cfg)
{
    cudaKernelNodeParams kp{};
    kp.sharedMemBytes = 0;
    if (small_prep(idx, cfg, nq)) {  // the node captured for this size is query_prep_small
        SmallPrepArgs a0 = small_prep_args(idx, w, in, nq, cfg);
        void *args[] = {&a0};
        kp.func = (void *)query_prep_small;
        kp.gridDim = dim3(small_prep_blocks(nq));
        kp.blockDim = dim3(kSmallPrep);
        kp.kernelParams = args;
        return cudaGraphExecKernelNodeSetParams(exec, nodes.prep, &kp);
    }
    PrepArgs a0 = prep_args(idx, w, in, nq, cfg);
    void *args[] = {&a0};
    kp.func = (void *)query_prep;
    kp.gridDim = dim3(prep_grid(nq));
    kp.blockDim = dim3(kBlock);
    kp.kernelParams = args;
    return cudaGraphExecKernelNodeSetParams(exec, nodes.prep, &kp);
}

namespace {

struct SearchSpec {
    double d, t0, t1;
    const double *d_arr, *t0_arr, *t1_arr;
};

tdq_status run_search(tdq_index *idx, const tdq_segments *queries, const SearchSpec &spec,
                      const tdq_search_params *params, cudaStream_t stream, const tdq_result_buffer &out,
                      uint64_t *count)
{
    const uint64_t nq = queries->n;
    Workspace &w = idx->ws;
    idx->last = tdq_stats{};
    *count = 0;
    if (nq == 0) return TDQ_OK;
    if (nq > 0xffffffffULL) return set_error(TDQ_ERR_INVALID, "tdq_search: more than 2^32-1 query segments");
    const double *cols[8] = {queries->xs, queries->ys, queries->zs, queries->ts,
                             queries->xe, queries->ye, queries->ze, queries->te};
    for (int c = 0; c < 8; c++)
        if (!cols[c]) return set_error(TDQ_ERR_INVALID, "tdq_search: query column %d is NULL", c);
    if (!queries->seg_id) return set_error(TDQ_ERR_INVALID, "tdq_search: query seg_id is NULL");
    LaunchCfg cfg;
    tdq_status st = parse_params(params, &cfg);
    if (st != TDQ_OK) return st;
    if ((cfg.flags & TDQ_FLAG_OTHER_TRAJECTORIES) && !queries->traj_id)
        return set_error(TDQ_ERR_INVALID, "tdq_search: TDQ_FLAG_OTHER_TRAJECTORIES needs the queries' traj_id");
    st = ensure_queries(w, nq, idx->m);
    if (st != TDQ_OK) return st;

    QueryInput in{};
    // host arrays in page-locked, mapped memory are read in place (as device
    // arrays are); any other host input is staged into the workspace
    bool mapped = !queries->on_device;
    const void *view[10] = {nullptr};
    for (int c = 0; c < 8 && mapped; c++) mapped = (view[c] = mapped_view(cols[c], nq * 8)) != nullptr;
    if (mapped) mapped = (view[8] = mapped_view(queries->seg_id, nq * 8)) != nullptr;
    if (mapped && queries->traj_id) mapped = (view[9] = mapped_view(queries->traj_id, nq * 8)) != nullptr;
    if (mapped) {
        for (int c = 0; c < 8; c++) in.c[c] = (const double *)view[c];
        in.seg_id = (const int64_t *)view[8];
        in.traj_id = (const int64_t *)view[9];
    } else if (!queries->on_device) {
        for (int c = 0; c < 8; c++) {
            TDQ_CUDA(cudaMemcpyAsync(w.in_cols[c], cols[c], nq * 8, cudaMemcpyHostToDevice, stream));
            in.c[c] = w.in_cols[c];
        }
        TDQ_CUDA(cudaMemcpyAsync(w.in_seg, queries->seg_id, nq * 8, cudaMemcpyHostToDevice, stream));
        in.seg_id = w.in_seg;
        if (cfg.flags && queries->traj_id) {
            TDQ_CUDA(cudaMemcpyAsync(w.in_traj, queries->traj_id, nq * 8, cudaMemcpyHostToDevice, stream));
            in.traj_id = w.in_traj;
        }
    } else {
        for (int c = 0; c < 8; c++) in.c[c] = cols[c];
        in.seg_id = queries->seg_id;
        in.traj_id = queries->traj_id;
    }
    in.d = spec.d;
    in.t0 = spec.t0;
    in.t1 = spec.t1;
    in.d_arr = spec.d_arr;
    in.t0_arr = spec.t0_arr;
    in.t1_arr = spec.t1_arr;
    in.n_real = 0;

    if (cfg.filter && idx->n > 0) {
        st = ensure_survivors(w, w.s_cap_pairs ? w.s_cap_pairs : (nq * 64 > (1u << 20) ? nq * 64 : (1u << 20)));
        if (st != TDQ_OK) return st;
    }
    // The survivor list of the filter mode is sized from the last search; if
    // it overflows, it is grown and the search re-run (like the results).
    for (int attempt = 0;; attempt++) {
        TDQ_CUDA(enqueue_search(idx, w, in, nq, cfg, out, stream, true));
        TDQ_CUDA(cudaStreamSynchronize(stream));
        bool grow = false;
        st = finish_search(idx, w, cfg, nq, out.capacity, true, &idx->last, count, &grow);
        if (!grow) return st;
        if (attempt >= 2) return set_error(TDQ_ERR_NOMEM, "tdq_search: survivor list kept overflowing");
        const uint64_t need = w.ctr_host->survivors;
        st = ensure_survivors(w, need + need / 4 + 1024);
        if (st != TDQ_OK) return st;
    }
}


tdq_status ensure_results(tdq_index *idx, uint64_t cap)
{
    Workspace &w = idx->ws;
    if (cap <= w.r_cap && w.r_block) return TDQ_OK;
    cudaFree(w.r_block);
    w.r_block = nullptr;
    w.r_cap = 0;
    if (dev_alloc(&w.r_block, 4 * carve_bytes(cap, 8)) != cudaSuccess) {
        cudaGetLastError();
        return set_error(TDQ_ERR_NOMEM, "tdq_search: result buffer of %llu items", (unsigned long long)cap);
    }
    char *p = (char *)w.r_block;
    w.r.query_seg_id = carve<int64_t>(p, cap);
    w.r.entry_seg_id = carve<int64_t>(p, cap);
    w.r.t_enter = carve<double>(p, cap);
    w.r.t_exit = carve<double>(p, cap);
    w.r.capacity = cap;
    w.r_cap = cap;
    return TDQ_OK;
}

}  // namespace

tdq_status check_scalars(double d, double t0, double t1)
{
    if (!(d >= 0.0) || isinf(d)) return set_error(TDQ_ERR_INVALID, "tdq_search: d must be finite and >= 0");
    if (isnan(t0) || isnan(t1) || t0 > t1) return set_error(TDQ_ERR_INVALID, "tdq_search: invalid window");
    return TDQ_OK;
}

cudaError_t load_search_module()
{
    cudaFuncAttributes fa;
    return cudaFuncGetAttributes(&fa, query_prep);
}

}  // namespace tdq

using namespace tdq;

extern "C" tdq_status tdq_search_device(tdq_index *idx, const tdq_segments *queries, double d, double t0, double t1,
                                        const tdq_search_params *params, void *stream, const tdq_result_buffer *out,
                                        uint64_t *count)
{
    if (!idx || !queries || !out || !count) return set_error(TDQ_ERR_INVALID, "tdq_search_device: NULL argument");
    if (!queries->on_device)
        return set_error(TDQ_ERR_INVALID, "tdq_search_device: queries must be in device memory");
    if (out->capacity && (!out->query_seg_id || !out->entry_seg_id || !out->t_enter || !out->t_exit))
        return set_error(TDQ_ERR_INVALID, "tdq_search_device: NULL result array");
    tdq_status st = check_scalars(d, t0, t1);
    if (st != TDQ_OK) return st;
    SearchSpec spec{d, t0, t1, nullptr, nullptr, nullptr};
    return run_search(idx, queries, spec, params, (cudaStream_t)stream, *out, count);
}

extern "C" tdq_status tdq_search_device_batched(tdq_index *idx, const tdq_segments *queries,
                                                const double *d_per_query, const double *t0_per_query,
                                                const double *t1_per_query, const tdq_search_params *params,
                                                void *stream, const tdq_result_buffer *out, uint64_t *count)
{
    if (!idx || !queries || !out || !count || !d_per_query || !t0_per_query || !t1_per_query)
        return set_error(TDQ_ERR_INVALID, "tdq_search_device_batched: NULL argument");
    if (!queries->on_device)
        return set_error(TDQ_ERR_INVALID, "tdq_search_device_batched: queries must be in device memory");
    if (out->capacity && (!out->query_seg_id || !out->entry_seg_id || !out->t_enter || !out->t_exit))
        return set_error(TDQ_ERR_INVALID, "tdq_search_device_batched: NULL result array");
    SearchSpec spec{0.0, 0.0, 0.0, d_per_query, t0_per_query, t1_per_query};
    return run_search(idx, queries, spec, params, (cudaStream_t)stream, *out, count);
}

extern "C" tdq_status tdq_search(tdq_index *idx, const tdq_segments *queries, double d, double t0, double t1,
                                 const tdq_search_params *params, void *stream_, tdq_results **out)
{
    if (!out) return set_error(TDQ_ERR_INVALID, "tdq_search: out is NULL");
    *out = nullptr;
    if (!idx || !queries) return set_error(TDQ_ERR_INVALID, "tdq_search: NULL argument");
    tdq_status st = check_scalars(d, t0, t1);
    if (st != TDQ_OK) return st;
    cudaStream_t stream = (cudaStream_t)stream_;
    // Statically sized result buffer, |D| items by default (Sec. 5), grown and
    // the search re-run when the results do not fit.
    uint64_t want = idx->ws.r_cap ? idx->ws.r_cap : (idx->n > 65536 ? idx->n : 65536);
    SearchSpec spec{d, t0, t1, nullptr, nullptr, nullptr};
    uint64_t count = 0;
    for (int attempt = 0; attempt < 3; attempt++) {
        st = ensure_results(idx, want);
        if (st != TDQ_OK) return st;
        st = run_search(idx, queries, spec, params, stream, idx->ws.r, &count);
        if (st != TDQ_ERR_OVERFLOW) break;
        want = count + count / 8 + 1024;
    }
    if (st != TDQ_OK) return st;
    tdq_results *r = (tdq_results *)calloc(1, sizeof(tdq_results));
    if (!r) return set_error(TDQ_ERR_NOMEM, "tdq_search: host allocation failed");
    r->count = count;
    if (count) {
        // one recycled page-locked block for the four arrays (fast copies,
        // no page population); else plain allocations
        char *blk = (char *)host_block_get(4 * count * 8);
        if (blk) {
            r->query_seg_id = (int64_t *)blk;
            r->entry_seg_id = (int64_t *)(blk + count * 8);
            r->t_enter = (double *)(blk + 2 * count * 8);
            r->t_exit = (double *)(blk + 3 * count * 8);
        } else {
            r->query_seg_id = (int64_t *)malloc(count * 8);
            r->entry_seg_id = (int64_t *)malloc(count * 8);
            r->t_enter = (double *)malloc(count * 8);
            r->t_exit = (double *)malloc(count * 8);
        }
        if (!r->query_seg_id || !r->entry_seg_id || !r->t_enter || !r->t_exit) {
            tdq_results_free(r);
            return set_error(TDQ_ERR_NOMEM, "tdq_search: host allocation failed");
        }
        const Workspace &w = idx->ws;
        cudaError_t e = cudaMemcpyAsync(r->query_seg_id, w.r.query_seg_id, count * 8, cudaMemcpyDeviceToHost, stream);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(r->entry_seg_id, w.r.entry_seg_id, count * 8, cudaMemcpyDeviceToHost, stream);
        if (e == cudaSuccess) e = cudaMemcpyAsync(r->t_enter, w.r.t_enter, count * 8, cudaMemcpyDeviceToHost, stream);
        if (e == cudaSuccess) e = cudaMemcpyAsync(r->t_exit, w.r.t_exit, count * 8, cudaMemcpyDeviceToHost, stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
        if (e != cudaSuccess) {
            tdq_results_free(r);
            return cuda_error(e, "tdq_search: D2H result copy");
        }
    }
    *out = r;
    return TDQ_OK;
}

extern "C" tdq_status tdq_self_join(tdq_index *idx, const tdq_segments *entries, double d, double t0, double t1,
                                    const tdq_search_params *params, void *stream, tdq_results **out)
{
    if (!out) return set_error(TDQ_ERR_INVALID, "tdq_self_join: out is NULL");
    *out = nullptr;
    if (!idx || !entries) return set_error(TDQ_ERR_INVALID, "tdq_self_join: NULL argument");
    if (entries->n != idx->n)
        return set_error(TDQ_ERR_INVALID, "tdq_self_join: %llu segments given, the index holds %llu",
                         (unsigned long long)entries->n, (unsigned long long)idx->n);
    if (!entries->traj_id) return set_error(TDQ_ERR_INVALID, "tdq_self_join: traj_id is NULL");
    tdq_search_params p{};
    if (params) p = *params;
    p.flags |= TDQ_FLAG_OTHER_TRAJECTORIES | TDQ_FLAG_UNORDERED_ONCE;
    return tdq_search(idx, entries, d, t0, t1, &p, stream, out);
}

extern "C" void tdq_results_free(tdq_results *res)
{
    if (!res) return;
    if (!host_block_put(res->query_seg_id)) {  // not a recycled block: four allocations
        free(res->query_seg_id);
        free(res->entry_seg_id);
        free(res->t_enter);
        free(res->t_exit);
    }
    free(res);
}

extern "C" tdq_status tdq_get_stats(const tdq_index *idx, tdq_stats *out)
{
    if (!idx || !out) return set_error(TDQ_ERR_INVALID, "tdq_get_stats: NULL argument");
    *out = idx->last;
    return TDQ_OK;
}

