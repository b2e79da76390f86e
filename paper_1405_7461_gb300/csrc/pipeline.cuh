// Definitions shared by the search pipeline's translation units -- search.cu
// (query preparation, the plain FP64 pair kernel, the host side), filter.cu
// (the FP32 pre-test and the FP64 refinement of its survivors) and
// noalloc.cu (the allocation-free entry point): tile sizes, argument
// structs, the kernels and launchers used by more than one file, and the
// per-pair FP64 code (Sec. 5, Algorithm 1) that both pair paths run.
#pragma once

#include <math.h>

#include "tdq_internal.cuh"

namespace tdq {

constexpr int kQT = 32;             // query segments per tile (one bit each in a lane mask)
constexpr int kPairThreads = 256;   // threads of the pair kernels

struct BinView {
    const int64_t *bin_begin, *bin_pmax_key;
    const int64_t *ts_key, *te_sorted, *te_bin_begin;  // sorted t_start / t_end keys and the t_end bin table
    const int64_t *bin_lo_key;  // m + 1: each bin's smallest time key under bin_of
    double t_min, width;
    double inv_width;   // 1 / width (for estimates that are verified afterwards)
    double max_dur;     // longest entry duration
    uint32_t m;
    int64_t tmin_key;   // time key of t_min
    int64_t dur_bins;   // bins a longest entry can span, rounded up (for estimates that are verified afterwards)
};

inline BinView bin_view(const tdq_index *idx)
{
    const double inv = idx->width > 0.0 ? 1.0 / idx->width : 0.0;
    const double db = ceil(idx->max_dur * inv) + 1.0;
    return BinView{idx->bin_begin, idx->bin_pmax_key, idx->e.ts_key, idx->e.te_sorted, idx->te_bin_begin,
                   idx->bin_lo_key, idx->t_min, idx->width, inv, idx->max_dur, idx->m, idx->tmin_key,
                   db < (double)idx->m ? (int64_t)db : (int64_t)idx->m};
}

// The bin of the time t (key k) under bin_of -- floor((t - t_min) / width),
// clamped to [0, m) -- without its FP64 division: an estimate by one
// multiplication and one rounding conversion (downward, saturating; the
// clamp in integers), checked against the table of each bin's smallest key
// (the bin is the last b with bin_lo_key[b] <= k), and if it is off (a
// degenerate width, extreme magnitudes) a bisection of that table.
__device__ __forceinline__ int64_t bin_of_key(const BinView &bins, int64_t k, double t)
{
    const int64_t m = bins.m;
    const long long f = __double2ll_rd((t - bins.t_min) * bins.inv_width);
    const int64_t b = f > 0 ? (f < m - 1 ? (int64_t)f : m - 1) : 0;
    const int64_t lo = bins.bin_lo_key[b], hi = bins.bin_lo_key[b + 1];
    if (k >= lo && k < hi) return b;
    int64_t a = k < lo ? 0 : b + 1, z = k < lo ? b : m;  // bin_lo_key[a] <= k < bin_lo_key[z]
    while (z - a > 1) {
        const int64_t mid = (a + z) >> 1;
        if (bins.bin_lo_key[mid] <= k) a = mid; else z = mid;
    }
    return a;
}

// Arguments of query_prep (one struct, so that a captured launch can be
// re-bound to new inputs in one step).  ranges (the index has entries): also
// the candidate range of every query segment into the pre columns kPreLo /
// kPreHi; count_overlaps: also the exact number of temporal-overlap pairs;
// sort_hist (may be null; zeroed beforehand): also the first sort pass's
// digit counts per tile of kSortTileKeys keys (radix_sort_pairs' prep_hist).
struct PrepArgs {
    QueryInput in;
    uint64_t nq;
    BinView bins;
    double *const *pre;
    float4 *pre_sph;
    uint64_t *keys;
    uint32_t *vals;
    DevCounters *ctr;
    uint32_t *sort_hist;
    bool ranges;
    bool count_overlaps;
    uint4 *pre_tc;  // may be null: also the tensor-core pre-test record of every valid query segment
    TcGrid grid;    // the index's grid (with pre_tc)
    // may be null: the counting sort instead of the radix sort's digit
    // counts -- each valid segment takes its place in its bin (vals) with
    // an atomic on bin_cnt (zeroed beforehand, bins.m words), and the last
    // block turns the counts into offsets
    uint32_t *bin_cnt;
    uint64_t n_entries;  // entries of the index (bound of the debug build's range check)
};

// Query slots up to which a search is prepared in one launch
// (query_prep_small): blocks of kSmallPrep threads whose first
// kSmallPrepWarps warps prepare a slot each, the last block sorting and
// planning all of them.
constexpr int kSmallPrep = 1024;
constexpr int kSmallPrepWarps = 4;

// Arguments of query_prep_small: those of query_prep (keys: the slots' sort
// words; vals, sort_hist and bin_cnt unused), the sorted query columns and
// the tile plan.
struct SmallPrepArgs {
    PrepArgs p;
    double *cols[kPreCols];  // the pre columns (p.pre's table, by value)
    QuerySoA q;
    int64_t *tile_lo, *tile_hi;
    unsigned long long *tile_work;  // exclusive offsets of the tiles' chunks, the total last; ntiles + 1
    int64_t *srt_lo, *srt_hi;       // every sorted segment's candidate range (for the pre-test)
    uint32_t chunk;
};

// Arguments of query_scatter (counting sort): every valid query segment's
// columns to its sorted position bin offset + rank.
struct ScatterArgs {
    const double *const *pre;
    const float4 *pre_sph;
    const uint4 *pre_tc;       // may be null
    const uint64_t *keys;      // bin of each segment
    const uint32_t *ranks;     // place inside its bin
    const uint32_t *bin_off;   // offsets of the bins
    uint64_t nq;
    QuerySoA q;
    uint4 *q_rec;              // may be null (tensor-core records)
    int64_t *srt_lo, *srt_hi;  // candidate ranges in sorted order
    DevCounters *ctr;
};

// Arguments of query_gather (it reads workspace arrays only).
struct GatherArgs {
    const double *const *pre;
    const float4 *pre_sph;
    const uint32_t *order;
    uint64_t nq;
    DevCounters *ctr;
    QuerySoA q;
    uint64_t ntiles;
    uint32_t chunk;
    int64_t *tile_lo, *tile_hi;
    unsigned long long *tile_work;  // chunks per tile, then (last block) their exclusive offsets; ntiles + 1
    // tensor-core pre-test (q_rec may be null): records in sorted order, and
    // the supertile plan (4 tiles of 32) instead of the tile plan's offsets
    const uint4 *pre_tc;
    uint4 *q_rec;
    int64_t *st_lo, *st_hi;
    unsigned long long *st_work;    // chunks per supertile, then their exclusive offsets; nsuper + 1
    uint64_t nsuper;
    // may be null: the sorted columns are in place already (query_scatter);
    // only the tile plan is made, from these candidate ranges in sorted order
    const int64_t *srt_lo, *srt_hi;
};

struct PairArgs {
    EntrySoA e;
    QuerySoA q;
    const int64_t *tile_lo, *tile_hi;
    const unsigned long long *tile_work;
    uint64_t ntiles;
    DevCounters *ctr;
    tdq_result_buffer out;
    uint32_t chunk;
    uint32_t flags;  // TDQ_FLAG_* pair filters (0: every pair)
    DevCounters *publish;  // may be null: host mirror the last pair kernel copies the counters to
    uint64_t n_entries;    // entries of the index, and query slots of the search (bounds of the debug
    uint64_t nq_slots;     // build's checks)
};

// The pair filters of TDQ_FLAG_OTHER_TRAJECTORIES / TDQ_FLAG_UNORDERED_ONCE
// (query (ii) of Sec. 2.1: every trajectory against all other trajectories,
// each unordered pair once when the database is the query set).
__device__ __forceinline__ bool pair_allowed(uint32_t flags, int64_t qtraj, int64_t qseg, int64_t etraj, int64_t eseg)
{
    if ((flags & TDQ_FLAG_OTHER_TRAJECTORIES) && etraj == qtraj) return false;
    if ((flags & TDQ_FLAG_UNORDERED_ONCE) && !(eseg > qseg)) return false;
    return true;
}

struct FilterArgs {
    PairArgs p;
    uint2 *surv;            // survivor list: (sorted entry position, sorted query position)
    uint64_t surv_cap;
    // may be null: every sorted query segment's own candidate range (a small
    // search), by which the pre-test skips the segments whose range misses a
    // pass of entries
    const int64_t *q_lo, *q_hi;
};

// The tensor-core pre-test's arguments (tcfilter.cu): the pair arguments
// (tile ranges, counters, chunk), the entry and query records, the
// supertile plan and the survivor list.
struct TcArgs {
    PairArgs p;
    const uint4 *e_rec, *q_rec;
    const int64_t *st_lo, *st_hi;
    const unsigned long long *st_work;
    uint64_t nsuper;
    uint2 *surv;
    uint64_t surv_cap;
    uint64_t n_rec;  // entry records held (bound of the debug build's checks)
};

// Kernels launched from more than one file (defined in search.cu).
// query_prep: blocks of kBlock threads, each block kPrepSlots query slots
// (prep_grid blocks for nq slots).
constexpr int kPrepSlots = kBlock / 2;
inline unsigned prep_grid(uint64_t nq) { return grid_for(nq, kPrepSlots); }
__global__ void query_prep(PrepArgs a);
__global__ void query_gather(GatherArgs a);
__global__ void query_scatter(ScatterArgs a);
__global__ void publish_counters(const DevCounters *src, DevCounters *dst);

// Pair kernel of the requested mode as a persistent grid (search.cu); the
// filter mode's pair (filter.cu), with inline_refine the pre-test kernel
// refining its own survivors (a small search).
cudaError_t launch_pair_kernel(const PairArgs &pa, bool filter, int sm_count, uint2 *surv, uint64_t surv_cap,
                               cudaStream_t stream, cudaEvent_t mid, unsigned evflags, bool inline_refine = false,
                               const int64_t *q_lo = nullptr, const int64_t *q_hi = nullptr);
cudaError_t launch_filter_kernels(const FilterArgs &fa, int sm_count, cudaStream_t stream, cudaEvent_t mid,
                                  unsigned evflags, bool inline_refine);
// The FP64 refine kernel of the filter modes alone (filter.cu).
cudaError_t launch_refine_kernel(const FilterArgs &fa, int sm_count, cudaStream_t stream);
// The tensor-core pre-test, then the refine kernel (tcfilter.cu).
cudaError_t launch_tc_filter_kernels(const TcArgs &ta, int sm_count, cudaStream_t stream, cudaEvent_t mid,
                                     unsigned evflags);

// TDQ_ERR_INVALID unless d is finite and >= 0 and [t0, t1] is a window (search.cu).
tdq_status check_scalars(double d, double t0, double t1);

namespace {

// Called by every thread of every block of the search's last kernel at its
// end: the block that finishes last copies the counters to dst (when given).
// Each thread fences its own counter updates before the block takes its
// ticket, so the last block reads every block's final values (through L2).
__device__ __forceinline__ void publish_when_last(DevCounters *ctr, DevCounters *dst)
{
    static_assert(sizeof(DevCounters) % 8 == 0 && sizeof(DevCounters) / 8 <= 32, "one warp copies the counters");
    if (!dst) return;
    __shared__ bool last;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) last = atomicAdd(&ctr->pair_done, 1ULL) == (unsigned long long)gridDim.x - 1;
    __syncthreads();
    if (last && threadIdx.x < sizeof(DevCounters) / 8) {
        __threadfence();
        const unsigned long long *s = reinterpret_cast<const unsigned long long *>(ctr);
        reinterpret_cast<unsigned long long *>(dst)[threadIdx.x] = __ldcg(s + threadIdx.x);
    }
}

// calcTimeInterval for a pair that is within d: the roots of
// A tau^2 + 2 Bh tau + C over tau in [0, L] (tau = time since a), by the
// cancellation-free quadratic formula; a tangent contact that rounding pushes
// out of the root bracket collapses to the closest point.
__device__ __noinline__ void pair_interval(double A, double Bh, double C, double disc, double a, double b,
                                           double *tin, double *tout)
{
    double L = b - a;
    double tlo, thi;
    if (le0(A)) {  // no relative motion: the whole span
        tlo = 0.0;
        thi = L;
    } else {
        double sq = sqrt(lt0(disc) ? 0.0 : disc);
        double qq = -(Bh + copysign(sq, Bh));
        double r1, r2;
        if (qq == 0.0) {
            r1 = 0.0;
            r2 = 0.0;
        } else {
            r1 = qq / A;
            r2 = C / qq;
        }
        double lo = fmin(r1, r2), hi = fmax(r1, r2);
        tlo = fmax(lo, 0.0);
        thi = fmin(hi, L);
        if (tlo > thi) {
            double ts = fmin(fmax(-Bh / A, 0.0), L);
            tlo = ts;
            thi = ts;
        }
    }
    *tin = le0(tlo) ? a : (tlo >= L ? b : a + tlo);
    *tout = thi >= L ? b : (le0(thi) ? a : a + thi);
}

// ---------------------------------------------------------------------------
// FP64 evaluation of one pair, shared by both pair kernels so that a pair
// gets bitwise the same decision and interval in either mode.
//
// temporalIntersection: common span [a, b] from the integer time keys; S is
// the segment that starts at a, O the other one.  calcTimeInterval: with
// tau = t - a, |dp + dv tau|^2 - d^2 = A tau^2 + 2 Bh tau + C, dp = O - S at
// a, dv = v_O - v_S.  The minimum over [0, L] is <= 0 without dividing:
// C <= 0 (in range at a), or approaching (Bh < 0) with a real root pair
// (disc >= 0) whose closest point lies inside the span or whose value at L
// is <= 0.  All lanes of the warp must call it (warp vote inside).
// ---------------------------------------------------------------------------
struct PairEval {
    double A, Bh, C, disc, a, b;
    bool hit;
};

__device__ __forceinline__ PairEval eval_pair_fp64(bool active, int64_t ets_k, int64_t ete_k, int64_t qts_k,
                                                   int64_t qte_k, double epx_, double epy_, double epz_,
                                                   double evx_, double evy_, double evz_, double qpx_, double qpy_,
                                                   double qpz_, double qvx_, double qvy_, double qvz_, double d2)
{
    PairEval r;
    const bool e_later = ets_k >= qts_k;
    const int64_t a_k = e_later ? ets_k : qts_k;
    const int64_t b_k = min(ete_k, qte_k);
    const int64_t o_k = e_later ? qts_k : ets_k;
    r.a = key_double(a_k);
    r.b = key_double(b_k);
    const double o_ts = key_double(o_k);
    const double opx = e_later ? qpx_ : epx_, opy = e_later ? qpy_ : epy_, opz = e_later ? qpz_ : epz_;
    const double ovx = e_later ? qvx_ : evx_, ovy = e_later ? qvy_ : evy_, ovz = e_later ? qvz_ : evz_;
    const double spx = e_later ? epx_ : qpx_, spy = e_later ? epy_ : qpy_, spz = e_later ? epz_ : qpz_;
    const double svx = e_later ? evx_ : qvx_, svy = e_later ? evy_ : qvy_, svz = e_later ? evz_ : qvz_;
    const double dt = r.a - o_ts;
    const double dpx = fma(ovx, dt, opx) - spx;
    const double dpy = fma(ovy, dt, opy) - spy;
    const double dpz = fma(ovz, dt, opz) - spz;
    const double dvx = ovx - svx, dvy = ovy - svy, dvz = ovz - svz;
    r.A = fma(dvz, dvz, fma(dvy, dvy, dvx * dvx));
    r.Bh = fma(dpz, dvz, fma(dpy, dvy, dpx * dvx));
    r.C = fma(dpz, dpz, fma(dpy, dpy, fma(dpx, dpx, -d2)));
    r.disc = fma(r.Bh, r.Bh, -(r.A * r.C));
    bool hit = le0(r.C);
    const bool need_L = !hit && lt0(r.Bh) && ge0(r.disc);
    if (__any_sync(kFull, active && need_L)) {
        const double L = r.b - r.a;
        const double gL = fma(r.A, L, r.Bh);
        const double fL = fma(gL + r.Bh, L, r.C);
        hit = hit || (need_L && (gt0(gL) || le0(fL)));
    }
    r.hit = hit && active;
    return r;
}

// Append the hits of a warp: one atomic per warp, writes past the capacity
// skipped while the count keeps counting.
__device__ __forceinline__ void append_hits(const PairEval &r, DevCounters *ctr, const tdq_result_buffer &out,
                                            uint64_t cap, int64_t qid, int64_t eid, int lane, unsigned lt_mask)
{
    const unsigned hm = __ballot_sync(kFull, r.hit);
    if (!hm) return;
    unsigned long long rbase = 0;
    const int leader = __ffs(hm) - 1;
    if (lane == leader) rbase = atomicAdd(&ctr->results, (unsigned long long)__popc(hm));
    rbase = __shfl_sync(kFull, rbase, leader);
    if (r.hit) {
        double tin, tout;
        pair_interval(r.A, r.Bh, r.C, r.disc, r.a, r.b, &tin, &tout);
        const unsigned long long pos = rbase + __popc(hm & lt_mask);
        if (pos < cap) {
            out.query_seg_id[pos] = qid;
            out.entry_seg_id[pos] = eid;
            out.t_enter[pos] = tin;
            out.t_exit[pos] = tout;
        }
    }
}

}  // namespace
}  // namespace tdq
