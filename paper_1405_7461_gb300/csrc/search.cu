// Distance threshold search on the device: candidate lookup in the
// temporal-bin index (Sec. 4) and the pair kernel (Sec. 5, Algorithm 1).
//
// Pipeline of one search, all on the caller's stream:
//   query_prep    validate, clip each query segment to the window, velocity,
//                 start position at the clipped start, sort key
//   radix sort    query segments by clipped start (Sec. 4 sorts Q by t_start)
//   query_gather  sorted query SoA + candidate range [lo, hi) of sorted entry
//                 positions per query segment, from the bin table; one warp
//                 per tile of 32 consecutive sorted query segments also
//                 plans the tile: its range is the union of its members'
//                 ranges, cut into chunks of `entry_chunk` entries, one work
//                 item per (tile, chunk); filter mode: the exact number of
//                 temporal-overlap pairs of each query segment
//   scan          work-item offsets per tile
//   traj_dist_search_kernel
//                 persistent CTAs take work items from an atomic counter,
//                 stage the tile's queries and the chunk's entries in shared
//                 memory, enumerate the pairs whose spans overlap with
//                 integer time keys, compact them so that all 32 lanes of a
//                 warp evaluate a real pair, and append every pair within d
//                 with one atomic per warp.
//
// Design notes for GB300: the FP64 pipe issues ~2 DFMA per clock per SM, so
// FP64 lane-slots are the scarce resource.  Temporal tests and every
// comparison run on the integer pipe; a lane never issues FP64 work for a
// pair whose spans do not overlap; the interval roots (sqrt, two divisions)
// run only for pairs that are within d.
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include "tdq_internal.cuh"

namespace tdq {
namespace {

constexpr int kQT = 32;             // query segments per tile (one bit each in a lane mask)
constexpr int kPairThreads = 256;   // threads of the pair kernel
constexpr int kBlock = 256;
constexpr unsigned kFull = 0xffffffffu;

inline unsigned grid_for(uint64_t n, int block = kBlock)
{
    uint64_t g = (n + block - 1) / block;
    return (unsigned)(g > 0 ? g : 1);
}

__device__ __forceinline__ bool is_nan_bits(double x)
{
    int64_t b = __double_as_longlong(x) & 0x7fffffffffffffffLL;
    return b > 0x7ff0000000000000LL;
}

__device__ __forceinline__ int64_t bin_of(double t, double t_min, double width, uint32_t m)
{
    double f = floor((t - t_min) / width);
    if (!(f < (double)(m - 1))) return (int64_t)m - 1;
    if (f < 0.0) return 0;
    return (int64_t)f;
}

struct BinView {
    const int64_t *bin_begin, *bin_pmax_key;
    const int64_t *ts_key, *te_sorted, *te_bin_begin;  // sorted t_start / t_end keys and the t_end bin table
    double t_min, width;
    uint32_t m;
    float inv_width_f;  // 1 / width in FP32 (for sort keys only)
};

inline BinView bin_view(const tdq_index *idx)
{
    return BinView{idx->bin_begin, idx->bin_pmax_key, idx->e.ts_key, idx->e.te_sorted, idx->te_bin_begin,
                   idx->t_min, idx->width, idx->m, idx->width > 0.0 ? (float)(1.0 / idx->width) : 0.f};
}

// Validate and clip every query segment.  pre[] columns: px py pz vx vy vz d2
// ts_key te_key (keys stored bitwise in the double arrays).
__global__ void query_prep(QueryInput in, uint64_t nq, BinView bins, double *const *pre, float4 *pre_sph,
                           uint64_t *keys, uint32_t *vals, DevCounters *ctr)
{
    uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    bool valid = false;
    // slots at or beyond the device-side count are padding: empty, not errors
    const uint64_t nreal = in.n_real ? in.n_real : nq;
    if (i == 0) ctr->sort_n = nreal < nq ? nreal : nq;
    if (i < nq && i >= nreal) {
        pre[7][i] = __longlong_as_double(INT64_MAX);
        pre[8][i] = __longlong_as_double(INT64_MIN);
        pre_sph[i] = make_float4(0.f, 0.f, 0.f, 0.f);
        keys[i] = (uint64_t)bins.m;
        vals[i] = (uint32_t)i;
    } else if (i < nq) {
        bool ok = true;
        double c[8];
#pragma unroll
        for (int k = 0; k < 8; k++) {
            c[k] = in.c[k][i];
            ok &= finite_bits(c[k]);
        }
        double d = in.d_arr ? in.d_arr[i] : in.d;
        double t0 = in.t0_arr ? in.t0_arr[i] : in.t0;
        double t1 = in.t1_arr ? in.t1_arr[i] : in.t1;
        ok &= finite_bits(d) && ge0(d);
        ok &= !is_nan_bits(t0) && !is_nan_bits(t1);
        int64_t ks = okey(c[3]), ke = okey(c[7]);
        ok &= ke > ks;
        int64_t k0 = ok ? okey(t0) : 0, k1 = ok ? okey(t1) : 0;
        ok &= k0 <= k1;
        if (!ok) atomicOr(&ctr->error, 1u);
        int64_t cs = max(ks, k0), ce = min(ke, k1);
        valid = ok && cs < ce;
        // one FP64 division per segment (the FP64 pipe is narrow)
        const double inv = 1.0 / (c[7] - c[3]);
        double vx = (c[4] - c[0]) * inv, vy = (c[5] - c[1]) * inv, vz = (c[6] - c[2]) * inv;
        double px = c[0], py = c[1], pz = c[2];
        if (valid && cs != ks) {  // the window cuts the start: position at the clipped start
            double shift = key_double(cs) - c[3];
            px = fma(vx, shift, px);
            py = fma(vy, shift, py);
            pz = fma(vz, shift, pz);
        }
        pre[0][i] = px; pre[1][i] = py; pre[2][i] = pz;
        pre[3][i] = vx; pre[4][i] = vy; pre[5][i] = vz;
        pre[6][i] = d * d;
        pre[7][i] = __longlong_as_double(cs);
        pre[8][i] = __longlong_as_double(ce);
        // FP32 bounding sphere of the clipped segment, its radius widened by
        // d (and a relative 2^-30 of d): the pre-test of the filter mode
        float4 sp = make_float4(0.f, 0.f, 0.f, __int_as_float(0x7f800000));
        if (valid) {
            const double h = 0.5 * (key_double(ce) - key_double(cs));
            const float dw = __double2float_ru(d);
            sp = sphere32(fma(vx, h, px), fma(vy, h, py), fma(vz, h, pz), __fmul_ru(norm_ru(vx, vy, vz),
                          __double2float_ru(h)), __fmaf_ru(dw, 0x1p-30f, dw));
        }
        pre_sph[i] = sp;
        // sort key: the temporal bin of the clipped start, in FP32 (it only
        // groups the segments into tiles of 32 that span few bins); invalid
        // segments sort last
        uint64_t key = bins.m;
        if (valid) {
            const float f = floorf(__double2float_rn(key_double(cs) - bins.t_min) * bins.inv_width_f);
            key = f < 0.f ? 0 : (f < (float)(bins.m - 1) ? (uint64_t)f : (uint64_t)(bins.m - 1));
        }
        keys[i] = key;
        vals[i] = (uint32_t)i;
    }
    unsigned vm = __ballot_sync(kFull, valid);
    if ((threadIdx.x & 31) == 0 && vm) atomicAdd(&ctr->valid_queries, (unsigned long long)__popc(vm));
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

// Arguments of query_gather (one struct, so that a captured launch can be
// re-bound to new inputs in one step).
struct GatherArgs {
    const double *const *pre;
    const float4 *pre_sph;
    const int64_t *seg_id;
    const int64_t *traj_id;  // may be null (then 0)
    const uint32_t *order;
    uint64_t nq;
    DevCounters *ctr;
    BinView bins;
    QuerySoA q;
    uint64_t ntiles;
    uint32_t chunk;
    int64_t *tile_lo, *tile_hi;
    unsigned long long *tile_work;  // chunks per tile (the scan turns it into offsets); ntiles + 1
    bool count_overlaps;
};

// First position in keys[lo, hi) whose key is >= x (strict: > x).
__device__ __forceinline__ int64_t lower_bound_key(const int64_t *keys, int64_t lo, int64_t hi, int64_t x, bool strict)
{
    while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        const int64_t v = keys[mid];
        if (v < x || (strict && v == x)) lo = mid + 1; else hi = mid;
    }
    return lo;
}

// Sorted query SoA and the candidate range of each query segment; then, one
// warp per tile of kQT sorted query segments, the tile plan; in filter mode
// also the exact number of temporal-overlap pairs of each query segment:
// #{t_start < q.t_end} - #{t_end <= q.t_start} (the second set lies inside
// the first because t_end > t_start).  The bin function is monotone in time,
// so each count lies inside the bin of its bound: a short binary search in
// the sorted t_start keys (bin table bin_begin) and in the sorted t_end keys
// (bin table te_bin_begin).
__global__ void query_gather(GatherArgs a)
{
    const uint64_t k = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const BinView &bins = a.bins;
    QuerySoA &q = a.q;
    int64_t rlo = INT64_MAX, rhi = INT64_MIN;
    unsigned long long n_overlap = 0;
    if (k < a.nq && k < a.ctr->valid_queries) {
        const uint32_t i = a.order[k];
        q.px[k] = a.pre[0][i]; q.py[k] = a.pre[1][i]; q.pz[k] = a.pre[2][i];
        q.vx[k] = a.pre[3][i]; q.vy[k] = a.pre[4][i]; q.vz[k] = a.pre[5][i];
        q.d2[k] = a.pre[6][i];
        const int64_t cs = __double_as_longlong(a.pre[7][i]);
        const int64_t ce = __double_as_longlong(a.pre[8][i]);
        q.ts_key[k] = cs;
        q.te_key[k] = ce;
        q.qid[k] = a.seg_id[i];
        if (q.qtraj) q.qtraj[k] = a.traj_id ? a.traj_id[i] : 0;
        q.sph[k] = a.pre_sph[i];
        // First bin whose extent reaches past the query start: the prefix
        // maximum of bin ends is non-decreasing, so this is a binary search
        // (Sec. 4 uses an index tree over the bin extents for the same lookup).
        uint32_t lo = 0, hi = bins.m;
        while (lo < hi) {
            uint32_t mid = (lo + hi) >> 1;
            if (bins.bin_pmax_key[mid] > cs) hi = mid; else lo = mid + 1;
        }
        const int64_t jlo = lo;
        // Last bin that can hold an entry starting before the query end.
        const double te = key_double(ce);
        const int64_t jhi = le0(te - bins.t_min) ? -1 : bin_of(te, bins.t_min, bins.width, bins.m);
        if (jlo < (int64_t)bins.m && jlo <= jhi) {
            rlo = bins.bin_begin[jlo];
            rhi = bins.bin_begin[jhi + 1];
            if (rlo >= rhi) { rlo = INT64_MAX; rhi = INT64_MIN; }
        }
        q.lo[k] = rlo;
        q.hi[k] = rhi;
        if (a.count_overlaps && jhi >= 0) {
            const int64_t n_start = lower_bound_key(bins.ts_key, bins.bin_begin[jhi], bins.bin_begin[jhi + 1], ce,
                                                    false);
            const double ts = key_double(cs);
            int64_t n_end = 0;
            if (!le0(ts - bins.t_min)) {
                const int64_t b = bin_of(ts, bins.t_min, bins.width, bins.m);
                n_end = lower_bound_key(bins.te_sorted, bins.te_bin_begin[b], bins.te_bin_begin[b + 1], cs, true);
            }
            n_overlap = (unsigned long long)(n_start - n_end);
        }
    }
    // the tile plan: this warp's 32 sorted query segments are tile k / kQT
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        rlo = min(rlo, (int64_t)__shfl_xor_sync(kFull, (long long)rlo, o));
        rhi = max(rhi, (int64_t)__shfl_xor_sync(kFull, (long long)rhi, o));
        n_overlap += __shfl_xor_sync(kFull, n_overlap, o);
    }
    const uint64_t t = k / kQT;
    if (lane == 0) {
        if (n_overlap) atomicAdd(&a.ctr->overlap_pairs, n_overlap);
        if (t < a.ntiles) {
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
    }
}

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

// ---------------------------------------------------------------------------
// Filter mode: conservative FP32 pre-test, FP64 for the survivors.
// ---------------------------------------------------------------------------

// Work items of the filter kernel are (tile, chunk) pairs as for the plain
// kernel, but each is processed by one warp: the warps of the grid split the
// items into contiguous ranges, and a warp treats its items of one tile as
// one run of consecutive sorted entries.  It walks those runs tile by tile,
// keeps the tile's 32 query segments in its own slice of shared memory, and
// streams the entries through registers, four per lane per pass over the
// queries (128 per pass); the next pass's records -- in the same run or at
// the start of the next one -- are loaded while the current pass is tested.
// No CTA-wide barrier is involved.
//
// For a pass, lane j forms the bound R_j = w_max + w_j (rounded up), w_max
// the largest entry radius of the pass (one warp max-reduction over the
// records already in registers), and
//   K_j = |c_j|^2 (1 - g) - R_j^2   (rounded down, g = 2^-20);
// each entry carries E_e = |c_e|^2 (1 - g) rounded down.  Per candidate pair
// the test is one add and three FMAs -- issued as paired FP32 instructions
// that evaluate two queries at once -- and one funnel shift that moves the
// sign of
//   v = E_e + K_j - 2 c_j . c_e  =  |c_e - c_j|^2 - R_j^2 - g (|c_e|^2 + |c_j|^2)
// into the lane's 32-bit mask.  v is negative whenever the exact spheres
// meet: with u = 2^-24 the four roundings of v add at most
// u (8 (|c_e|^2 + |c_j|^2) + 4 R^2), less than the g (|c_e|^2 + |c_j|^2) = 16u (...)
// subtracted and the 32u R^2 by which R_j^2 exceeds the exact bound (the
// radii carry a factor 1 + 2^-20); R >= 2^-60 keeps every quantity normal.
// Segments beyond 2^60 in magnitude carry a zero sphere and E = -inf, or an
// infinite radius and K = -inf, and are never rejected.  The survivors
// (entry, query) are appended to a list through a per-warp shared-memory
// buffer (one atomic per 256 survivors: dense workloads pass many pairs to
// the refinement, and per-lane atomics on one counter would serialise);
// traj_dist_refine_kernel then evaluates them in FP64.
// Warps per block of the filter kernel.  It has no block-wide step, but the
// warps of a block take adjacent item ranges, whose entry records largely
// coincide, so that they share the SM's L1 cache.
constexpr int kFilterWarps = 8;
constexpr int kFilterThreads = 32 * kFilterWarps;
constexpr int kPer = 4;            // entries per lane per pass
constexpr int kSurvBuf = 256;      // survivors a warp buffers before one atomic on the list
constexpr int kPass = 32 * kPer;   // entries per pass

// One entry's pre-test terms, each duplicated into both halves of a paired
// FP32 operand.
struct EntryDup {
    float2 x, y, z, e;
};

__device__ __forceinline__ EntryDup dup(float4 s, float e)
{
    return EntryDup{make_float2(s.x, s.x), make_float2(s.y, s.y), make_float2(s.z, s.z), make_float2(e, e)};
}

// v for the two queries j, j+1 of a pair at once; qa = (-2x_j, -2x_j+1,
// -2y_j, -2y_j+1), qb = (-2z_j, -2z_j+1, K_j, K_j+1).
__device__ __forceinline__ float2 sphere_gap_pair(const EntryDup &e, float4 qa, float4 qb)
{
    float2 v = __fadd2_rn(e.e, make_float2(qb.z, qb.w));
    v = __ffma2_rn(make_float2(qa.x, qa.y), e.x, v);
    v = __ffma2_rn(make_float2(qa.z, qa.w), e.y, v);
    return __ffma2_rn(make_float2(qb.x, qb.y), e.z, v);
}

// The warp's run of entries in tile t: its items there are
// [max(ibeg, tile_work[t]), min(iend, tile_work[t+1])), chunk_len entries each.
__device__ __forceinline__ void filter_run(const PairArgs &args, uint64_t t, unsigned long long ibeg,
                                           unsigned long long iend, int64_t &eb, int64_t &ee)
{
    const unsigned long long wb = args.tile_work[t], wn = args.tile_work[t + 1];
    const int64_t lo = args.tile_lo[t], hi = args.tile_hi[t];
    eb = lo + (int64_t)(max(ibeg, wb) - wb) * args.chunk;
    ee = min(lo + (int64_t)(min(iend, wn) - wb) * args.chunk, hi);
}

// Query terms of lane j for its tile: -2 c_j into the warp's table (pairs of
// queries interleaved: qr[2i] = (-2x, -2y of queries 2i, 2i+1), qr[2i+1].xy =
// -2z of both; qr[2i+1].zw receives K of both every pass), and |c_j|^2 (1 - g)
// and w_j kept in registers.  Lanes past the tile's last query hold zeros.
__device__ __forceinline__ void stage_queries(float4 s, bool real, int lane, float4 *qr, float &c2g, float &w)
{
    if (!real) s = make_float4(0.f, 0.f, 0.f, 0.f);
    float X = -2.0f * s.x, Y = -2.0f * s.y, Z = -2.0f * s.z;
    w = s.w;
    if (isinf(s.w)) {  // huge magnitudes: K = -inf, never rejected
        X = Y = Z = 0.f;
        c2g = 0.f;
    } else {
        c2g = __fmul_rd(__fmaf_rd(s.z, s.z, __fmaf_rd(s.y, s.y, __fmul_rd(s.x, s.x))), 1.0f - 0x1p-20f);
    }
    const bool odd = lane & 1;
    const float r1 = __shfl_xor_sync(kFull, odd ? X : Z, 1);
    const float r2 = __shfl_xor_sync(kFull, Y, 1);
    __syncwarp();  // the previous tile's table is no longer read
    if (odd)
        *reinterpret_cast<float2 *>(&qr[lane]) = make_float2(r1, Z);
    else
        qr[lane] = make_float4(X, r1, Y, r2);
}

struct FilterArgs {
    PairArgs p;
    uint2 *surv;            // survivor list: (sorted entry position, sorted query position)
    uint64_t surv_cap;
};

__global__ void __launch_bounds__(kFilterThreads, 2) traj_dist_filter_kernel(FilterArgs fa)
{
    const PairArgs &args = fa.p;
    __shared__ float4 qr_all[kFilterWarps][kQT];
    __shared__ uint2 sbuf_all[kFilterWarps][kSurvBuf];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    float4 *qr = qr_all[warp];
    uint2 *sbuf = sbuf_all[warp];  // this warp's survivors not yet in the list
    int nbuf = 0;                   // (warp-uniform)
    float *qrf = reinterpret_cast<float *>(qr);
    const int k_slot = (lane >> 1) * 8 + 6 + (lane & 1);  // this lane's K in qr[2i+1].zw
    DevCounters *ctr = args.ctr;
    const unsigned long long total = args.tile_work[args.ntiles];
    const uint64_t nvalid = ctr->valid_queries;
    const unsigned long long nwarps = (unsigned long long)gridDim.x * kFilterWarps;
    const unsigned long long gw = (unsigned long long)blockIdx.x * kFilterWarps + warp;
    const unsigned long long per = (total + nwarps - 1) / nwarps;
    const unsigned long long ibeg = min(gw * per, total);
    const unsigned long long iend = min(ibeg + per, total);
    const float4 *esph = args.e.sph;
    const float *esphe = args.e.sph_e;
    unsigned long long n_inter = 0;
    // moves the buffered survivors to the list (called by the whole warp)
    auto flush_survivors = [&]() {
        if (nbuf == 0) return;
        unsigned long long base = 0;
        if (lane == 0) base = atomicAdd(&ctr->survivors, (unsigned long long)nbuf);
        base = __shfl_sync(kFull, base, 0);
        __syncwarp();
        for (int i = lane; i < nbuf; i += 32)
            if (base + i < fa.surv_cap) fa.surv[base + i] = sbuf[i];
        __syncwarp();
        nbuf = 0;
    };

    if (ibeg < iend) {
        uint64_t t = 0;
        {
            uint64_t lo = 0, hi = args.ntiles;  // last tile whose first item is <= ibeg
            while (hi - lo > 1) {
                uint64_t mid = (lo + hi) >> 1;
                if (args.tile_work[mid] <= ibeg) lo = mid; else hi = mid;
            }
            t = lo;
        }
        int64_t eb, ee;
        filter_run(args, t, ibeg, iend, eb, ee);
        int nqt = (int)min((uint64_t)kQT, nvalid - (uint64_t)t * kQT);
        float my_c2g, my_w;
        stage_queries(args.q.sph[(int64_t)t * kQT + min(lane, nqt - 1)], lane < nqt, lane, qr, my_c2g, my_w);
        float4 ns[kPer];
        float nse[kPer];
#pragma unroll
        for (int k = 0; k < kPer; k++) {
            const int64_t e = eb + lane + 32 * k;
            ns[k] = e < ee ? esph[e] : make_float4(0.f, 0.f, 0.f, 0.f);
            nse[k] = e < ee ? esphe[e] : 0.f;
        }
        for (;;) {
            // the next run of this warp (a later tile with items in range),
            // located and its queries fetched while this run is tested
            uint64_t tn = t + 1;
            const bool has_next = args.tile_work[tn] < iend;
            int64_t ebn = 0, een = 0;
            int nqn = 0;
            float4 qn = make_float4(0.f, 0.f, 0.f, 0.f);
            if (has_next) {
                while (args.tile_work[tn + 1] == args.tile_work[tn]) tn++;
                filter_run(args, tn, ibeg, iend, ebn, een);
                nqn = (int)min((uint64_t)kQT, nvalid - tn * kQT);
                qn = args.q.sph[(int64_t)tn * kQT + min(lane, nqn - 1)];
            }
            const int64_t q0 = (int64_t)t * kQT;
            const unsigned qvalid = 0xffffffffu << (kQT - nqt);  // bit 31-j <-> query j
            if (lane == 0) n_inter += (unsigned long long)(ee - eb) * (unsigned long long)nqt;
            for (int64_t pe = eb; pe < ee; pe += kPass) {
                EntryDup ed[kPer];
                float wl = 0.f;
#pragma unroll
                for (int k = 0; k < kPer; k++) {
                    ed[k] = dup(ns[k], nse[k]);
                    wl = fmaxf(wl, ns[k].w);
                }
                // the next pass's records: this run, else the next run's first pass
                {
                    const bool same = pe + kPass < ee;
                    const int64_t nb = same ? pe + kPass : ebn;
                    const int left = (int)min(same ? ee - nb : een - nb, (int64_t)kPass);
                    const float4 *ps = esph + nb + lane;
                    const float *pse = esphe + nb + lane;
#pragma unroll
                    for (int k = 0; k < kPer; k++) {
                        const bool in = lane + 32 * k < left;
                        ns[k] = in ? ps[32 * k] : make_float4(0.f, 0.f, 0.f, 0.f);
                        nse[k] = in ? pse[32 * k] : 0.f;
                    }
                }
                // radii are non-negative: their bit patterns order like the values
                const float wmax = __uint_as_float(__reduce_max_sync(kFull, __float_as_uint(wl)));
                const float Rj = __fadd_ru(wmax, my_w);
                const float Kj = __fsub_rd(my_c2g, __fmul_ru(Rj, Rj));
                __syncwarp();  // the previous pass's K are no longer read
                qrf[k_slot] = Kj;
                __syncwarp();
                // two independent mask chains per entry (queries 0-15 and
                // 16-31), joined afterwards: the funnel shifts of one chain
                // depend on each other
                unsigned m[kPer], mh[kPer];
#pragma unroll
                for (int k = 0; k < kPer; k++) m[k] = mh[k] = 0u;
#pragma unroll
                for (int j = 0; j < kQT; j += 2) {
                    const float4 qa = qr[j], qb = qr[j + 1];
#pragma unroll
                    for (int k = 0; k < kPer; k++) {
                        const float2 v = sphere_gap_pair(ed[k], qa, qb);
                        unsigned &mm = j < kQT / 2 ? mh[k] : m[k];
                        mm = __funnelshift_l(__float_as_uint(v.x), mm, 1);
                        mm = __funnelshift_l(__float_as_uint(v.y), mm, 1);
                    }
                }
#pragma unroll
                for (int k = 0; k < kPer; k++) m[k] = __byte_perm(m[k], mh[k], 0x5410);
                unsigned any = 0u;
                const int here = (int)min(ee - pe, (int64_t)kPass);
#pragma unroll
                for (int k = 0; k < kPer; k++) {
                    m[k] = lane + 32 * k < here ? (m[k] & qvalid) : 0u;
                    any |= m[k];
                }
                if (!__any_sync(kFull, any != 0u)) continue;
                // append the warp's survivors: ranks by a warp scan, then into
                // the warp's buffer (flushed to the list with one atomic per
                // kSurvBuf survivors), or, for a pass with more survivors than
                // the buffer holds, straight to the list
                int cnt = 0;
#pragma unroll
                for (int k = 0; k < kPer; k++) cnt += __popc(m[k]);
                int incl = cnt;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const int y = __shfl_up_sync(kFull, incl, o);
                    if (lane >= o) incl += y;
                }
                const int total = __shfl_sync(kFull, incl, 31);
                if (nbuf + total > kSurvBuf) flush_survivors();
                const bool direct = total > kSurvBuf;
                unsigned long long pos = nbuf + (incl - cnt);
                if (direct) {
                    unsigned long long base = 0;
                    if (lane == 0) base = atomicAdd(&ctr->survivors, (unsigned long long)total);
                    pos = __shfl_sync(kFull, base, 0) + (incl - cnt);
                }
#pragma unroll
                for (int k = 0; k < kPer; k++) {
                    unsigned mk = m[k];
                    const uint32_t ek = (uint32_t)(pe + lane + 32 * k);
                    while (mk) {
                        const int bit = 31 - __clz(mk);
                        mk &= ~(1u << bit);
                        const uint2 sv = make_uint2(ek, (uint32_t)(q0 + 31 - bit));
                        if (!direct)
                            sbuf[pos] = sv;
                        else if (pos < fa.surv_cap)
                            fa.surv[pos] = sv;
                        pos++;
                    }
                }
                if (!direct) nbuf += total;
            }
            if (!has_next) break;
            t = tn;
            eb = ebn;
            ee = een;
            nqt = nqn;
            stage_queries(qn, lane < nqt, lane, qr, my_c2g, my_w);
        }
        flush_survivors();
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) n_inter += __shfl_xor_sync(kFull, n_inter, o);
    if (lane == 0 && n_inter) atomicAdd(&ctr->interactions, n_inter);
}

// FP64 evaluation of the filter's survivors.  The pre-test ignores time, so
// most survivors do not overlap in time; a warp checks the exact span keys
// of 32 survivors at a time, queues the overlapping ones in its slice of
// shared memory, and runs the FP64 code of the plain kernel (then the
// warp-aggregated append) on full batches of 32 queued pairs: the FP64 pipe
// is busy for a warp instruction whatever the number of active lanes.
constexpr int kRefineWarps = kPairThreads / 32;

__device__ __forceinline__ void refine_batch(const PairArgs &args, uint2 sv, bool active, uint64_t cap, int lane,
                                             unsigned lt_mask)
{
    const int64_t ek = sv.x, qk = sv.y;
    const PairEval r = eval_pair_fp64(active, args.e.ts_key[ek], args.e.te_key[ek], args.q.ts_key[qk],
                                      args.q.te_key[qk], args.e.px[ek], args.e.py[ek], args.e.pz[ek], args.e.vx[ek],
                                      args.e.vy[ek], args.e.vz[ek], args.q.px[qk], args.q.py[qk], args.q.pz[qk],
                                      args.q.vx[qk], args.q.vy[qk], args.q.vz[qk], args.q.d2[qk]);
    append_hits(r, args.ctr, args.out, cap, args.q.qid[qk], args.e.seg_id[ek], lane, lt_mask);
}

__global__ void __launch_bounds__(kPairThreads) traj_dist_refine_kernel(FilterArgs fa)
{
    const PairArgs &args = fa.p;
    __shared__ uint2 queue_all[kRefineWarps][64];
    DevCounters *ctr = args.ctr;
    const int lane = threadIdx.x & 31;
    uint2 *queue = queue_all[threadIdx.x >> 5];
    const unsigned lt_mask = (1u << lane) - 1u;
    const uint64_t cap = args.out.capacity;
    const unsigned long long ns = min(ctr->survivors, (unsigned long long)fa.surv_cap);
    const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
    unsigned long long n_fp64 = 0;
    int queued = 0;  // warp-uniform, < 32 between chunks
    // warp-uniform trip count (the ballots, eval_pair_fp64 and append_hits vote over the warp)
    const unsigned long long first = (unsigned long long)blockIdx.x * blockDim.x + (threadIdx.x & ~31u);
    for (unsigned long long wb = first; wb < ns; wb += stride) {
        const unsigned long long k = wb + lane;
        const bool valid = k < ns;
        const uint2 sv = valid ? fa.surv[k] : make_uint2(0u, 0u);
        bool active = valid && args.e.ts_key[sv.x] < args.q.te_key[sv.y] &&
                      args.e.te_key[sv.x] > args.q.ts_key[sv.y];
        if (args.flags && active)
            active = pair_allowed(args.flags, args.q.qtraj[sv.y], args.q.qid[sv.y], args.e.traj_id[sv.x],
                                  args.e.seg_id[sv.x]);
        const unsigned am = __ballot_sync(kFull, active);
        if (active) queue[queued + __popc(am & lt_mask)] = sv;
        queued += __popc(am);
        n_fp64 += __popc(am);
        __syncwarp();
        if (queued >= 32) {
            const uint2 qv = queue[lane];
            const uint2 rest = lane + 32 < queued ? queue[lane + 32] : make_uint2(0u, 0u);
            __syncwarp();
            if (lane + 32 < queued) queue[lane] = rest;
            queued -= 32;
            __syncwarp();
            refine_batch(args, qv, true, cap, lane, lt_mask);
        }
    }
    if (queued > 0) {  // the last, partial batch
        const bool active = lane < queued;
        refine_batch(args, active ? queue[lane] : make_uint2(0u, 0u), active, cap, lane, lt_mask);
    }
    if (lane == 0 && n_fp64) atomicAdd(&ctr->fp64_pairs, n_fp64);
}

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
        const int64_t e0 = args.tile_lo[t] + (int64_t)(item - (long long)args.tile_work[t]) * EC;
        const int64_t e1 = min(e0 + (int64_t)EC, args.tile_hi[t]);
        const int ne = (int)(e1 - e0);
        const uint64_t q0 = t * kQT;
        const int nqt = (int)min((uint64_t)kQT, nvalid - q0);

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
}

size_t pair_smem_bytes(uint32_t chunk)
{
    return ((sizeof(PairSmem) + 15) & ~(size_t)15) + (size_t)chunk * 64;
}

// Launch the pair kernel of the requested mode as a persistent grid (as many
// CTAs as fit on every SM at once).  Filter mode: the FP32 pre-test kernel,
// then the FP64 refine kernel over its survivors.  Neither counts the
// overlapping pairs: query_gather does.
// mid (filter mode, may be null): event recorded between the filter and the
// refine kernel with the flags evflags.
cudaError_t launch_pair_kernel(const PairArgs &pa, bool filter, int sm_count, uint2 *surv, uint64_t surv_cap,
                               cudaStream_t stream, cudaEvent_t mid, unsigned evflags)
{
    if (filter) {
        FilterArgs fa{pa, surv, surv_cap};
        int per_sm = 0;
        cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, traj_dist_filter_kernel, kFilterThreads,
                                                                      0);
        if (e != cudaSuccess) return e;
        if (per_sm < 1) per_sm = 1;
        traj_dist_filter_kernel<<<sm_count * per_sm, kFilterThreads, 0, stream>>>(fa);
        if (mid && (e = cudaEventRecordWithFlags(mid, stream, evflags)) != cudaSuccess) return e;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, traj_dist_refine_kernel, kPairThreads, 0);
        if (e != cudaSuccess) return e;
        if (per_sm < 1) per_sm = 1;
        traj_dist_refine_kernel<<<sm_count * per_sm, kPairThreads, 0, stream>>>(fa);
        return cudaGetLastError();
    }
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


template <typename T>
T *carve(char *&p, uint64_t count)
{
    T *r = (T *)p;
    p += (count * sizeof(T) + 255) & ~(uint64_t)255;
    return r;
}
inline uint64_t cb(uint64_t count, uint64_t size) { return (count * size + 255) & ~(uint64_t)255; }

}  // namespace

tdq_status ensure_queries(Workspace &w, uint64_t nq)
{
    if (nq <= w.q_cap && w.q_block) return TDQ_OK;
    uint64_t cap = nq > 2 * w.q_cap ? nq : 2 * w.q_cap;
    if (cap < 1024) cap = 1024;
    uint64_t bytes = 10 * cb(cap, 8)                   // staged host input
                     + 9 * cb(cap, 8)                  // pre
                     + 2 * cb(cap, 8) + 2 * cb(cap, 4) // sort
                     + 13 * cb(cap, 8)                 // sorted query SoA
                     + 2 * cb(cap, 16)                 // query spheres (before / after sorting)
                     + cb(9, sizeof(double *));        // pre pointer table
    uint64_t ntiles = (cap + kQT - 1) / kQT;
    uint64_t tbytes = 2 * cb(ntiles, 8) + cb(ntiles + 1, 8);
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
    for (int c = 0; c < 9; c++) w.pre[c] = carve<double>(p, cap);
    w.keys = carve<uint64_t>(p, cap);
    w.keys_alt = carve<uint64_t>(p, cap);
    w.vals = carve<uint32_t>(p, cap);
    w.vals_alt = carve<uint32_t>(p, cap);
    QuerySoA &q = w.q;
    q.px = carve<double>(p, cap); q.py = carve<double>(p, cap); q.pz = carve<double>(p, cap);
    q.vx = carve<double>(p, cap); q.vy = carve<double>(p, cap); q.vz = carve<double>(p, cap);
    q.d2 = carve<double>(p, cap);
    q.ts_key = carve<int64_t>(p, cap); q.te_key = carve<int64_t>(p, cap);
    q.qid = carve<int64_t>(p, cap); q.lo = carve<int64_t>(p, cap); q.hi = carve<int64_t>(p, cap);
    q.qtraj = carve<int64_t>(p, cap);
    w.pre_sph = carve<float4>(p, cap);
    q.sph = carve<float4>(p, cap);
    w.pre_dev = carve<double *>(p, 9);
    if (cudaMemcpy(w.pre_dev, w.pre, 9 * sizeof(double *), cudaMemcpyHostToDevice) != cudaSuccess)
        return cuda_error(cudaGetLastError(), "search workspace: pointer table");
    char *tp = (char *)w.t_block;
    w.tile_lo = carve<int64_t>(tp, ntiles);
    w.tile_hi = carve<int64_t>(tp, ntiles);
    w.tile_work = carve<unsigned long long>(tp, ntiles + 1);
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
    if (params && params->mode != TDQ_MODE_FP64 && params->mode != TDQ_MODE_FP32_FILTER)
        return set_error(TDQ_ERR_INVALID, "tdq_search: unknown mode %d", params->mode);
    cfg->filter = params && params->mode == TDQ_MODE_FP32_FILTER;
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

int search_kernel_launches(const tdq_index *idx, const LaunchCfg &cfg, uint64_t nq)
{
    // query_prep and publish_counters; with entries: the sort of the query
    // keys, query_gather, scan, pair kernel (filter mode: filter and refine)
    return idx->n > 0 ? 2 + sort_kernel_launches(nq, bin_key_bits(idx->m)) + 2 + (cfg.filter ? 2 : 1) : 2;
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
    e = cudaMemsetAsync(w.ctr, 0, sizeof(DevCounters), stream);
    if (e != cudaSuccess) return e;
    if (events && (e = cudaEventRecordWithFlags(w.ev[0], stream, evflags)) != cudaSuccess) return e;
    double *const *pre = w.pre_dev;
    const BinView bins = bin_view(idx);
    query_prep<<<grid_for(nq), kBlock, 0, stream>>>(in, nq, bins, pre, w.pre_sph, w.keys, w.vals, w.ctr);
    const uint64_t ntiles = (nq + kQT - 1) / kQT;
    if (idx->n > 0) {
        if ((e = radix_sort_pairs(w.keys, w.vals, w.keys_alt, w.vals_alt, nq, w.sort_hist, stream,
                                  bin_key_bits(idx->m), &w.ctr->sort_n)) != cudaSuccess)
            return e;
        const GatherArgs ga{pre, w.pre_sph, in.seg_id, in.traj_id, w.vals, nq, w.ctr, bins, w.q, ntiles, cfg.chunk,
                            w.tile_lo, w.tile_hi, w.tile_work, cfg.filter};
        query_gather<<<grid_for(nq), kBlock, 0, stream>>>(ga);
        if ((e = exclusive_scan_u64(w.tile_work, ntiles + 1, &w.ctr->work_items, stream)) != cudaSuccess) return e;
        PairArgs pa{idx->e, w.q, w.tile_lo, w.tile_hi, w.tile_work, ntiles, w.ctr, out, cfg.chunk, cfg.flags};
        if (events && (e = cudaEventRecordWithFlags(w.ev[1], stream, evflags)) != cudaSuccess) return e;
        if ((e = launch_pair_kernel(pa, cfg.filter, idx->sm_count, w.surv, w.s_cap_pairs, stream,
                                    events ? w.ev[2] : nullptr, evflags)) != cudaSuccess)
            return e;
        if (events && (e = cudaEventRecordWithFlags(cfg.filter ? w.ev[4] : w.ev[2], stream, evflags)) != cudaSuccess)
            return e;
    } else if (events) {
        for (int k : {1, 2, 4})
            if ((e = cudaEventRecordWithFlags(w.ev[k], stream, evflags)) != cudaSuccess) return e;
    }
    publish_counters<<<1, 32, 0, stream>>>(w.ctr, w.ctr_host_dev);
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
    if (cfg.filter && idx->n > 0 && h.survivors > w.s_cap_pairs) {
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
        if (kp.func == (void *)query_prep) out->prep = nodes[k];
        if (kp.func == (void *)query_gather) out->gather = nodes[k];
    }
    free(nodes);
    if (e == cudaSuccess && (!out->prep || !out->gather)) e = cudaErrorInvalidValue;
    return e;
}

cudaError_t bind_inputs(cudaGraphExec_t exec, const GraphInputNodes &nodes, const tdq_index *idx, Workspace &w,
                        const QueryInput &in, uint64_t nq, const LaunchCfg &cfg)
{
    const BinView bins = bin_view(idx);
    double *const *pre = w.pre_dev;
    {
        QueryInput a0 = in;
        uint64_t a1 = nq;
        BinView a2 = bins;
        double *const *a3 = pre;
        float4 *a4 = w.pre_sph;
        uint64_t *a5 = w.keys;
        uint32_t *a6 = w.vals;
        DevCounters *a7 = w.ctr;
        void *args[] = {&a0, &a1, &a2, &a3, &a4, &a5, &a6, &a7};
        cudaKernelNodeParams kp{};
        kp.func = (void *)query_prep;
        kp.gridDim = dim3(grid_for(nq));
        kp.blockDim = dim3(kBlock);
        kp.sharedMemBytes = 0;
        kp.kernelParams = args;
        cudaError_t e = cudaGraphExecKernelNodeSetParams(exec, nodes.prep, &kp);
        if (e != cudaSuccess) return e;
    }
    {
        GatherArgs a0{pre, w.pre_sph, in.seg_id, in.traj_id, w.vals, nq, w.ctr, bins, w.q, (nq + kQT - 1) / kQT,
                      cfg.chunk, w.tile_lo, w.tile_hi, w.tile_work, cfg.filter};
        void *args[] = {&a0};
        cudaKernelNodeParams kp{};
        kp.func = (void *)query_gather;
        kp.gridDim = dim3(grid_for(nq));
        kp.blockDim = dim3(kBlock);
        kp.sharedMemBytes = 0;
        kp.kernelParams = args;
        return cudaGraphExecKernelNodeSetParams(exec, nodes.gather, &kp);
    }
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
    st = ensure_queries(w, nq);
    if (st != TDQ_OK) return st;

    QueryInput in{};
    if (!queries->on_device) {
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

tdq_status check_scalars(double d, double t0, double t1)
{
    if (!(d >= 0.0) || isinf(d)) return set_error(TDQ_ERR_INVALID, "tdq_search: d must be finite and >= 0");
    if (isnan(t0) || isnan(t1) || t0 > t1) return set_error(TDQ_ERR_INVALID, "tdq_search: invalid window");
    return TDQ_OK;
}

tdq_status ensure_results(tdq_index *idx, uint64_t cap)
{
    Workspace &w = idx->ws;
    if (cap <= w.r_cap && w.r_block) return TDQ_OK;
    cudaFree(w.r_block);
    w.r_block = nullptr;
    w.r_cap = 0;
    if (dev_alloc(&w.r_block, 4 * cb(cap, 8)) != cudaSuccess) {
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
        r->query_seg_id = (int64_t *)malloc(count * 8);
        r->entry_seg_id = (int64_t *)malloc(count * 8);
        r->t_enter = (double *)malloc(count * 8);
        r->t_exit = (double *)malloc(count * 8);
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
    free(res->query_seg_id);
    free(res->entry_seg_id);
    free(res->t_enter);
    free(res->t_exit);
    free(res);
}

extern "C" tdq_status tdq_get_stats(const tdq_index *idx, tdq_stats *out)
{
    if (!idx || !out) return set_error(TDQ_ERR_INVALID, "tdq_get_stats: NULL argument");
    *out = idx->last;
    return TDQ_OK;
}

// ---------------------------------------------------------------------------
// Allocation-free search (tdq_search_device_noalloc).
//
// For callers that must not allocate device memory: a process whose device
// memory is already owned by another allocator (a framework's caching pool),
// or a latency-critical loop that cannot afford cudaMalloc/cudaFree, which
// may synchronize the whole device.  The index is built beforehand; this
// entry point then runs the same kernels as tdq_search_device, with all of
// their per-search scratch (clipped query SoA, sort buffers, tile table,
// counters) carved from one fixed file-scope device array instead of the
// index's workspace.  The array is sized for kNoAllocMaxQueries query
// segments and stays resident on every device that loads the library.
// ---------------------------------------------------------------------------
#include <mutex>

namespace tdq {
namespace {

constexpr uint64_t kNoAllocMaxQueries = 8192;
constexpr uint64_t kNoAllocTiles = kNoAllocMaxQueries / kQT;
constexpr uint64_t kNoAllocHistWords = (kNoAllocMaxQueries + 1023) / 1024 * 256 + 1;  // 1024-key sort tiles
constexpr uint64_t na_bytes(uint64_t count, uint64_t size) { return (count * size + 255) & ~(uint64_t)255; }
constexpr uint64_t kNoAllocScratchBytes =
    9 * na_bytes(kNoAllocMaxQueries, 8)                                      // pre columns
    + 2 * na_bytes(kNoAllocMaxQueries, 8) + 2 * na_bytes(kNoAllocMaxQueries, 4)  // sort keys / values
    + 12 * na_bytes(kNoAllocMaxQueries, 8)                                   // sorted query SoA
    + 2 * na_bytes(kNoAllocMaxQueries, 16)                                   // query spheres
    + 2 * na_bytes(kNoAllocTiles, 8) + na_bytes(kNoAllocTiles + 1, 8)        // tile table
    + na_bytes(kNoAllocHistWords, 4)                                         // sort histogram
    + na_bytes(1, sizeof(DevCounters))                                       // counters
    + na_bytes(9, sizeof(double *));                                         // pre pointer table

// The scratch.  In host code this name is only a host-side stand-in for the
// symbol; its device address comes from cudaGetSymbolAddress below.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

struct NoAllocScratch {
    double *pre[9];
    double **pre_dev;
    float4 *pre_sph;
    uint64_t *keys, *keys_alt;
    uint32_t *vals, *vals_alt;
    QuerySoA q;
    int64_t *tile_lo, *tile_hi;
    unsigned long long *tile_work;
    uint32_t *hist;
    DevCounters *ctr;
};

constexpr int kNoAllocMaxDevices = 64;
std::mutex g_noalloc_mu;
bool g_noalloc_ready[kNoAllocMaxDevices];
NoAllocScratch g_noalloc[kNoAllocMaxDevices];

// Once per device, with that device current: resolve the array's device
// address, carve it, and store the device copy of the column-pointer table.
tdq_status noalloc_setup(int dev, NoAllocScratch **out)
{
    if (dev < 0 || dev >= kNoAllocMaxDevices)
        return set_error(TDQ_ERR_INVALID, "tdq_search_device_noalloc: device %d out of range", dev);
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_ready[dev]) {
        unsigned char *base = nullptr;
        cudaError_t e = cudaGetSymbolAddress((void **)&base, g_noalloc_scratch);
        if (e != cudaSuccess) return cuda_error(e, "tdq_search_device_noalloc: cudaGetSymbolAddress");
        NoAllocScratch s{};
        char *p = (char *)base;
        for (int c = 0; c < 9; c++) s.pre[c] = carve<double>(p, kNoAllocMaxQueries);
        s.keys = carve<uint64_t>(p, kNoAllocMaxQueries);
        s.keys_alt = carve<uint64_t>(p, kNoAllocMaxQueries);
        s.vals = carve<uint32_t>(p, kNoAllocMaxQueries);
        s.vals_alt = carve<uint32_t>(p, kNoAllocMaxQueries);
        QuerySoA &q = s.q;
        q.px = carve<double>(p, kNoAllocMaxQueries); q.py = carve<double>(p, kNoAllocMaxQueries);
        q.pz = carve<double>(p, kNoAllocMaxQueries); q.vx = carve<double>(p, kNoAllocMaxQueries);
        q.vy = carve<double>(p, kNoAllocMaxQueries); q.vz = carve<double>(p, kNoAllocMaxQueries);
        q.d2 = carve<double>(p, kNoAllocMaxQueries);
        q.ts_key = carve<int64_t>(p, kNoAllocMaxQueries); q.te_key = carve<int64_t>(p, kNoAllocMaxQueries);
        q.qid = carve<int64_t>(p, kNoAllocMaxQueries); q.lo = carve<int64_t>(p, kNoAllocMaxQueries);
        q.hi = carve<int64_t>(p, kNoAllocMaxQueries);
        q.qtraj = nullptr;  // no pair filters here
        s.pre_sph = carve<float4>(p, kNoAllocMaxQueries);
        q.sph = carve<float4>(p, kNoAllocMaxQueries);
        s.tile_lo = carve<int64_t>(p, kNoAllocTiles);
        s.tile_hi = carve<int64_t>(p, kNoAllocTiles);
        s.tile_work = carve<unsigned long long>(p, kNoAllocTiles + 1);
        s.hist = carve<uint32_t>(p, kNoAllocHistWords);
        s.ctr = carve<DevCounters>(p, 1);
        s.pre_dev = carve<double *>(p, 9);
        if ((uint64_t)(p - (char *)base) > kNoAllocScratchBytes || sort_hist_words(kNoAllocMaxQueries) > kNoAllocHistWords)
            return set_error(TDQ_ERR_CUDA, "tdq_search_device_noalloc: scratch layout exceeds the array");
        e = cudaMemcpy(s.pre_dev, s.pre, 9 * sizeof(double *), cudaMemcpyHostToDevice);
        if (e != cudaSuccess) return cuda_error(e, "tdq_search_device_noalloc: pointer table");
        g_noalloc[dev] = s;
        g_noalloc_ready[dev] = true;
    }
    *out = &g_noalloc[dev];
    return TDQ_OK;
}

}  // namespace
}  // namespace tdq

extern "C" tdq_status tdq_search_device_noalloc(tdq_index *idx, const tdq_segments *queries, double d, double t0,
                                                double t1, const tdq_search_params *params, void *stream_,
                                                const tdq_result_buffer *out, uint64_t *count)
{
    if (!idx || !queries || !out || !count)
        return set_error(TDQ_ERR_INVALID, "tdq_search_device_noalloc: NULL argument");
    *count = 0;
    if (!queries->on_device)
        return set_error(TDQ_ERR_INVALID, "tdq_search_device_noalloc: queries must be in device memory");
    if (out->capacity && (!out->query_seg_id || !out->entry_seg_id || !out->t_enter || !out->t_exit))
        return set_error(TDQ_ERR_INVALID, "tdq_search_device_noalloc: NULL result array");
    tdq_status st = check_scalars(d, t0, t1);
    if (st != TDQ_OK) return st;
    const uint64_t nq = queries->n;
    if (nq > kNoAllocMaxQueries)
        return set_error(TDQ_ERR_INVALID,
                         "tdq_search_device_noalloc: %llu query segments exceed the fixed maximum of %llu",
                         (unsigned long long)nq, (unsigned long long)kNoAllocMaxQueries);
    if (params && params->flags)
        return set_error(TDQ_ERR_INVALID, "tdq_search_device_noalloc: pair filters (flags) are not supported");
    if (params && params->mode == TDQ_MODE_FP32_FILTER)
        return set_error(TDQ_ERR_INVALID,
                         "tdq_search_device_noalloc: the filter mode needs a survivor list; use TDQ_MODE_FP64");
    uint32_t chunk = (params && params->entry_chunk) ? params->entry_chunk : 512u;
    if (chunk % kPairThreads != 0 || chunk > 2048)
        return set_error(TDQ_ERR_INVALID, "tdq_search_device_noalloc: entry_chunk must be a multiple of 256, <= 2048");
    if (params && params->query_tile && params->query_tile != (uint32_t)kQT)
        return set_error(TDQ_ERR_INVALID, "tdq_search_device_noalloc: query_tile must be 32");
    int dev = 0;
    TDQ_CUDA(cudaGetDevice(&dev));
    if (dev != idx->device)
        return set_error(TDQ_ERR_INVALID, "tdq_search_device_noalloc: index lives on device %d, current is %d",
                         idx->device, dev);
    NoAllocScratch *s = nullptr;
    st = noalloc_setup(dev, &s);
    if (st != TDQ_OK) return st;
    if (nq == 0) return TDQ_OK;
    const double *cols[8] = {queries->xs, queries->ys, queries->zs, queries->ts,
                             queries->xe, queries->ye, queries->ze, queries->te};
    for (int c = 0; c < 8; c++)
        if (!cols[c]) return set_error(TDQ_ERR_INVALID, "tdq_search_device_noalloc: query column %d is NULL", c);
    if (!queries->seg_id) return set_error(TDQ_ERR_INVALID, "tdq_search_device_noalloc: query seg_id is NULL");

    cudaStream_t stream = (cudaStream_t)stream_;
    QueryInput in{};
    for (int c = 0; c < 8; c++) in.c[c] = cols[c];
    in.seg_id = queries->seg_id;
    in.d = d;
    in.t0 = t0;
    in.t1 = t1;
    // the array keeps the previous call's contents: clear the counters
    TDQ_CUDA(cudaMemsetAsync(s->ctr, 0, sizeof(DevCounters), stream));
    const BinView bins = bin_view(idx);
    query_prep<<<grid_for(nq), kBlock, 0, stream>>>(in, nq, bins, s->pre_dev, s->pre_sph, s->keys, s->vals, s->ctr);
    const uint64_t ntiles = (nq + kQT - 1) / kQT;
    if (idx->n > 0) {
        TDQ_CUDA(radix_sort_pairs(s->keys, s->vals, s->keys_alt, s->vals_alt, nq, s->hist, stream,
                                  bin_key_bits(idx->m)));
        const GatherArgs ga{s->pre_dev, s->pre_sph, in.seg_id, nullptr, s->vals, nq, s->ctr, bins, s->q, ntiles,
                            chunk, s->tile_lo, s->tile_hi, s->tile_work, false};
        query_gather<<<grid_for(nq), kBlock, 0, stream>>>(ga);
        TDQ_CUDA(exclusive_scan_u64(s->tile_work, ntiles + 1, &s->ctr->work_items, stream));
        PairArgs pa{idx->e, s->q, s->tile_lo, s->tile_hi, s->tile_work, ntiles, s->ctr, *out, chunk, 0u};
        TDQ_CUDA(launch_pair_kernel(pa, false, idx->sm_count, nullptr, 0, stream, nullptr, 0));
    }
    TDQ_CUDA(cudaGetLastError());
    DevCounters h{};
    TDQ_CUDA(cudaMemcpyAsync(&h, s->ctr, sizeof(DevCounters), cudaMemcpyDeviceToHost, stream));
    TDQ_CUDA(cudaStreamSynchronize(stream));
    if (h.error & 1u)
        return set_error(TDQ_ERR_INVALID,
                         "tdq_search_device_noalloc: invalid query segment (non-finite value, t_end <= t_start, "
                         "d < 0 or NaN, NaN window or t0 > t1)");
    *count = h.results;
    return h.results > out->capacity ? TDQ_ERR_OVERFLOW : TDQ_OK;
}
