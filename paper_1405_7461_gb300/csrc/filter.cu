// Filter mode (TDQ_MODE_FP32_FILTER): a conservative FP32 bounding-sphere
// pre-test of every candidate pair, then the FP64 evaluation of the
// survivors with the plain path's per-pair code (Sec. 5, Algorithm 1), so
// that the result set equals the plain FP64 search's.
#include "pipeline.cuh"

namespace tdq {
namespace {

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
// infinite radius and K = -inf, and are never rejected.
//
// The survivors (entry, query) collect in a per-warp shared-memory buffer,
// and then (kInline false) go to a list with one atomic per 256 of them
// (dense workloads pass many pairs to the refinement, and per-lane atomics
// on one counter would serialise), which traj_dist_refine_kernel evaluates
// in FP64 over the whole grid.  A small search (kInline true: at most
// kSmallPrep query slots, few survivors) saves that launch: once a warp's
// buffer holds kRefineAt survivors (a dense pass fills it in rounds), the
// warp refines them itself, as the refine kernel does (refine_due,
// refine_batch), and the block that finishes last copies the counters to
// the host mirror.  (On a large batch the in-kernel refinement was measured
// slower than the separate kernel: the FP64 batches stall the warps' FP32
// work and leave more partial batches.)
//
// A small search is typically one trajectory's segments in time order, so
// that a tile's 32 segments span 32 time steps and its union range is many
// times each segment's own candidate range (Sec. 4's wasteful
// interactions).  The small-search kernel therefore also holds every lane's
// query segment's own range and, per pass, skips the segments whose range
// misses the pass's entries: a pass that none meets is skipped, and with at
// most kSparseAt segments left only their pairs are evaluated.  (Measured on
// the large batch, whose tiles hold segments of nearly the same time, the
// per-pass test cost more than it saved.)

// Warps per block of the filter kernel.  It has no block-wide step, but the
// warps of a block take adjacent item ranges, whose entry records largely
// coincide, so that they share the SM's L1 cache.
constexpr int kFilterWarps = 8;
constexpr int kFilterThreads = 32 * kFilterWarps;
constexpr int kPer = 4;            // entries per lane per pass
constexpr int kSurvBuf = 256;      // survivors a warp buffers
constexpr int kRefineAt = 64;      // kInline: buffered survivors at which the warp refines them
constexpr int kSparseAt = 16;      // kInline: active query segments of a pass up to which only their pairs run
constexpr int kPass = 32 * kPer;   // entries per pass

// FP64 evaluation (Sec. 5, Algorithm 1) of one batch of queued survivors,
// one per lane, and the append of the hits (the whole warp); the FP64 pipe
// is busy for a warp instruction whatever the number of active lanes, so
// that survivors are evaluated in full batches of 32 wherever possible.
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

// The exact span-key check (and the pair filters) of one survivor: whether
// its FP64 evaluation is due.
__device__ __forceinline__ bool refine_due(const PairArgs &args, uint2 sv)
{
    if (!TDQ_DBG(args.ctr, kDbgRefine, sv.x < args.n_entries && sv.y < args.nq_slots)) return false;
    bool due = args.e.ts_key[sv.x] < args.q.te_key[sv.y] && args.e.te_key[sv.x] > args.q.ts_key[sv.y];
    if (args.flags && due)
        due = pair_allowed(args.flags, args.q.qtraj[sv.y], args.q.qid[sv.y], args.e.traj_id[sv.x],
                           args.e.seg_id[sv.x]);
    return due;
}

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

template <bool kInline>
__global__ void __launch_bounds__(kFilterThreads, 2) traj_dist_filter_kernel(FilterArgs fa)
{
    const PairArgs &args = fa.p;
    __shared__ float4 qr_all[kFilterWarps][kQT];
    __shared__ uint2 sbuf_all[kFilterWarps][kSurvBuf];
    __shared__ uint2 queue_all[kInline ? kFilterWarps : 1][64];
    __shared__ uint2 pool[kInline ? kFilterWarps * 32 : 1];
    __shared__ int pooled;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    float4 *qr = qr_all[warp];
    uint2 *sbuf = sbuf_all[warp];   // this warp's survivors not yet listed (refined)
    uint2 *queue = queue_all[kInline ? warp : 0];  // kInline: survivors due for the FP64 code, < 32 between batches
    int nbuf = 0;                   // (warp-uniform)
    int queued = 0;                 // (warp-uniform)
    const unsigned lt_mask = (1u << lane) - 1u;
    const uint64_t cap = args.out.capacity;
    if (threadIdx.x == 0) pooled = 0;
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
    unsigned long long n_inter = 0, n_surv = 0, n_fp64 = 0;
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
    // kInline: refines the buffered survivors (called by the whole warp)
    auto refine_buffered = [&]() {
        for (int b = 0; b < nbuf; b += 32) {
            const bool valid = b + lane < nbuf;
            const uint2 sv = valid ? sbuf[b + lane] : make_uint2(0u, 0u);
            const bool due = valid && refine_due(args, sv);
            const unsigned am = __ballot_sync(kFull, due);
            if (due) queue[queued + __popc(am & lt_mask)] = sv;
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
        if (!TDQ_DBG(ctr, kDbgFilterRun, eb >= 0 && eb < ee && ee <= (int64_t)args.n_entries)) ee = eb;
        int nqt = (int)min((uint64_t)kQT, nvalid - (uint64_t)t * kQT);
        float my_c2g, my_w;
        stage_queries(args.q.sph[(int64_t)t * kQT + min(lane, nqt - 1)], lane < nqt, lane, qr, my_c2g, my_w);
        // kInline with q_lo: this lane's query segment's own candidate range
        // (an empty one past the tile's last segment)
        int64_t my_lo = INT64_MAX, my_hi = INT64_MIN;
        if (kInline && fa.q_lo && lane < nqt) {
            my_lo = fa.q_lo[(int64_t)t * kQT + lane];
            my_hi = fa.q_hi[(int64_t)t * kQT + lane];
        }
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
            int64_t lon = INT64_MAX, hin = INT64_MIN;
            if (has_next) {
                while (args.tile_work[tn + 1] == args.tile_work[tn]) tn++;
                filter_run(args, tn, ibeg, iend, ebn, een);
                if (!TDQ_DBG(ctr, kDbgFilterRun, ebn >= 0 && ebn < een && een <= (int64_t)args.n_entries)) een = ebn;
                nqn = (int)min((uint64_t)kQT, nvalid - tn * kQT);
                qn = args.q.sph[(int64_t)tn * kQT + min(lane, nqn - 1)];
                if (kInline && fa.q_lo && lane < nqn) {
                    lon = fa.q_lo[(int64_t)tn * kQT + lane];
                    hin = fa.q_hi[(int64_t)tn * kQT + lane];
                }
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
                    int left = (int)min(same ? ee - nb : een - nb, (int64_t)kPass);
                    if (!TDQ_DBG(ctr, kDbgFilterNext, left <= 0 || (nb >= 0 && nb + left <= (int64_t)args.n_entries)))
                        left = 0;
                    const float4 *ps = esph + nb + lane;
                    const float *pse = esphe + nb + lane;
#pragma unroll
                    for (int k = 0; k < kPer; k++) {
                        const bool in = lane + 32 * k < left;
                        ns[k] = in ? ps[32 * k] : make_float4(0.f, 0.f, 0.f, 0.f);
                        nse[k] = in ? pse[32 * k] : 0.f;
                    }
                }
                // kInline with q_lo: the tile's query segments whose own
                // candidate range meets this pass (bit 31-j <-> query j);
                // none: the pass is skipped
                unsigned act = qvalid;
                if (kInline && fa.q_lo) {
                    const int64_t pend = min(pe + kPass, ee);
                    act = __brev(__ballot_sync(kFull, my_lo < pend && my_hi > pe));
                    if (act == 0u) continue;
                }
                // radii are non-negative: their bit patterns order like the values
                const float wmax = __uint_as_float(__reduce_max_sync(kFull, __float_as_uint(wl)));
                const float Rj = __fadd_ru(wmax, my_w);
                const float Kj = __fsub_rd(my_c2g, __fmul_ru(Rj, Rj));
                __syncwarp();  // the previous pass's K are no longer read
                qrf[k_slot] = Kj;
                __syncwarp();
                unsigned m[kPer];
                // every query pair: two independent mask chains per entry
                // (queries 0-15 and 16-31), joined afterwards -- the funnel
                // shifts of one chain depend on each other
                auto dense_masks = [&]() {
                    unsigned mh[kPer];
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
                };
                if constexpr (!kInline) {
                    dense_masks();
                } else if (__popc(act) > kSparseAt) {
                    dense_masks();
                } else {
                    // the active query pairs only, each sign bit put in place
#pragma unroll
                    for (int k = 0; k < kPer; k++) m[k] = 0u;
                    for (unsigned rem = act; rem;) {
                        const int j = __clz(rem) & ~1;  // the pair's first query
                        rem &= ~(0xc0000000u >> j);
                        const float4 qa = qr[j], qb = qr[j + 1];
#pragma unroll
                        for (int k = 0; k < kPer; k++) {
                            const float2 v = sphere_gap_pair(ed[k], qa, qb);
                            m[k] |= ((__float_as_uint(v.x) >> 31) << (31 - j)) |
                                    ((__float_as_uint(v.y) >> 31) << (30 - j));
                        }
                    }
                }
                unsigned any = 0u;
                const int here = (int)min(ee - pe, (int64_t)kPass);
#pragma unroll
                for (int k = 0; k < kPer; k++) {
                    m[k] = lane + 32 * k < here ? (m[k] & qvalid & act) : 0u;
                    any |= m[k];
                }
                if (!__any_sync(kFull, any != 0u)) continue;
                // the warp's survivors: ranks by a warp scan, then into the
                // warp's buffer
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
                if constexpr (!kInline) {
                    // (flushed to the list with one atomic per kSurvBuf
                    // survivors), or, for a pass with more survivors than the
                    // buffer holds, straight to the list
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
                            if (!TDQ_DBG(ctr, kDbgFilterQuery, (uint64_t)(q0 + 31 - bit) < nvalid)) {
                            } else if (!direct) {
                                if (TDQ_DBG(ctr, kDbgFilterBuf, pos < (unsigned long long)kSurvBuf)) sbuf[pos] = sv;
                            } else if (pos < fa.surv_cap) {
                                fa.surv[pos] = sv;
                            }
                            pos++;
                        }
                    }
                    if (!direct) nbuf += total;
                    continue;
                }
                // kInline: a pass with more survivors than the buffer has room
                // for fills it in rounds, each full buffer refined before the
                // next round
                n_surv += (unsigned long long)total;
                for (int done = 0; done < total;) {
                    if (nbuf == kSurvBuf) refine_buffered();
                    const int take = min(total - done, kSurvBuf - nbuf);
                    int r = incl - cnt;  // this lane's first rank in the pass
#pragma unroll
                    for (int k = 0; k < kPer; k++) {
                        unsigned mk = m[k];
                        const uint32_t ek = (uint32_t)(pe + lane + 32 * k);
                        while (mk) {
                            const int bit = 31 - __clz(mk);
                            mk &= ~(1u << bit);
                            if (r >= done && r < done + take) {
                                const int pos = nbuf + (r - done);
                                // (debug build: a failed check leaves a survivor
                                // that the refinement's own check drops)
                                if (TDQ_DBG(ctr, kDbgFilterBuf, pos < kSurvBuf))
                                    sbuf[pos] = TDQ_DBG(ctr, kDbgFilterQuery, (uint64_t)(q0 + 31 - bit) < nvalid)
                                                    ? make_uint2(ek, (uint32_t)(q0 + 31 - bit))
                                                    : make_uint2(0xffffffffu, 0xffffffffu);
                            }
                            r++;
                        }
                    }
                    __syncwarp();
                    nbuf += take;
                    done += take;
                }
                if (nbuf >= kRefineAt) refine_buffered();
            }
            if (!has_next) break;
            t = tn;
            eb = ebn;
            ee = een;
            nqt = nqn;
            my_lo = lon;
            my_hi = hin;
            stage_queries(qn, lane < nqt, lane, qr, my_c2g, my_w);
        }
        if constexpr (kInline)
            refine_buffered();
        else
            flush_survivors();
    }
    if constexpr (!kInline) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) n_inter += __shfl_xor_sync(kFull, n_inter, o);
        if (lane == 0 && n_inter) atomicAdd(&ctr->interactions, n_inter);
        return;
    }
    // kInline: pool the warps' remainders and run them as full batches (the
    // last one partial)
    __syncthreads();
    if (queued > 0) {
        int base = 0;
        if (lane == 0) base = atomicAdd(&pooled, queued);
        base = __shfl_sync(kFull, base, 0);
        if (lane < queued) pool[base + lane] = queue[lane];
    }
    __syncthreads();
    const int np = pooled;
    for (int bt = warp; bt * 32 < np; bt += kFilterWarps) {
        const bool active = bt * 32 + lane < np;
        refine_batch(args, active ? pool[bt * 32 + lane] : make_uint2(0u, 0u), active, cap, lane, lt_mask);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) n_inter += __shfl_xor_sync(kFull, n_inter, o);
    if (lane == 0) {
        if (n_inter) atomicAdd(&ctr->interactions, n_inter);
        if (n_surv) atomicAdd(&ctr->survivors, n_surv);
        if (n_fp64) atomicAdd(&ctr->fp64_pairs, n_fp64);
    }
    publish_when_last(ctr, args.publish);
}

// FP64 evaluation of the filter's survivors.  The pre-test ignores time, so
// most survivors do not overlap in time; a warp checks the exact span keys
// of 32 survivors at a time (and the pair filters), queues the overlapping
// ones in its slice of shared memory, and runs the FP64 code of the plain
// kernel (then the warp-aggregated append) on full batches of 32 queued
// pairs: the FP64 pipe is busy for a warp instruction whatever the number of
// active lanes.  The warps of a block pool what is left in their queues at
// the end (fewer than 32 pairs each), so that a block runs at most one
// partial batch.  The block that finishes last copies the counters to the
// host mirror.
constexpr int kRefineWarps = kPairThreads / 32;

__global__ void __launch_bounds__(kPairThreads) traj_dist_refine_kernel(FilterArgs fa)
{
    const PairArgs &args = fa.p;
    __shared__ uint2 queue_all[kRefineWarps][64];
    __shared__ uint2 pool[kRefineWarps * 32];
    __shared__ int pooled;
    DevCounters *ctr = args.ctr;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint2 *queue = queue_all[warp];
    const unsigned lt_mask = (1u << lane) - 1u;
    const uint64_t cap = args.out.capacity;
    const unsigned long long ns = min(ctr->survivors, (unsigned long long)fa.surv_cap);
    const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
    unsigned long long n_fp64 = 0;
    int queued = 0;  // warp-uniform, < 32 between chunks
    if (threadIdx.x == 0) pooled = 0;
    // warp-uniform trip count (the ballots, eval_pair_fp64 and append_hits vote over the warp)
    const unsigned long long first = (unsigned long long)blockIdx.x * blockDim.x + (threadIdx.x & ~31u);
    for (unsigned long long wb = first; wb < ns; wb += stride) {
        const unsigned long long k = wb + lane;
        const bool valid = k < ns;
        const uint2 sv = valid ? fa.surv[k] : make_uint2(0u, 0u);
        const bool active = valid && refine_due(args, sv);
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
    // pool the warps' remainders and run them as full batches (the last one partial)
    __syncthreads();
    if (queued > 0) {
        int base = 0;
        if (lane == 0) base = atomicAdd(&pooled, queued);
        base = __shfl_sync(kFull, base, 0);
        if (lane < queued) pool[base + lane] = queue[lane];
    }
    __syncthreads();
    const int np = pooled;
    for (int bt = warp; bt * 32 < np; bt += kRefineWarps) {
        const bool active = bt * 32 + lane < np;
        refine_batch(args, active ? pool[bt * 32 + lane] : make_uint2(0u, 0u), active, cap, lane, lt_mask);
    }
    if (lane == 0 && n_fp64) atomicAdd(&ctr->fp64_pairs, n_fp64);
    publish_when_last(ctr, args.publish);
}

}  // namespace

// The filter mode's kernels as persistent grids (as many CTAs as fit on
// every SM at once): the FP32 pre-test, then the FP64 refinement of its
// survivors -- in the pre-test kernel itself for a small search (inline) --
// with mid (may be null) recorded between them with the flags evflags.
cudaError_t launch_filter_kernels(const FilterArgs &fa, int sm_count, cudaStream_t stream, cudaEvent_t mid,
                                  unsigned evflags, bool inline_refine)
{
    int per_sm = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
        &per_sm, inline_refine ? traj_dist_filter_kernel<true> : traj_dist_filter_kernel<false>, kFilterThreads, 0);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) per_sm = 1;
    if (inline_refine)
        traj_dist_filter_kernel<true><<<sm_count * per_sm, kFilterThreads, 0, stream>>>(fa);
    else
        traj_dist_filter_kernel<false><<<sm_count * per_sm, kFilterThreads, 0, stream>>>(fa);
    if (mid && (e = cudaEventRecordWithFlags(mid, stream, evflags)) != cudaSuccess) return e;
    return inline_refine ? cudaGetLastError() : launch_refine_kernel(fa, sm_count, stream);
}

cudaError_t launch_refine_kernel(const FilterArgs &fa, int sm_count, cudaStream_t stream)
{
    int per_sm = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, traj_dist_refine_kernel, kPairThreads, 0);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) per_sm = 1;
    traj_dist_refine_kernel<<<sm_count * per_sm, kPairThreads, 0, stream>>>(fa);
    return cudaGetLastError();
}

cudaError_t load_filter_module()
{
    cudaFuncAttributes fa;
    cudaError_t e = cudaFuncGetAttributes(&fa, traj_dist_filter_kernel<false>);
    return e != cudaSuccess ? e : cudaFuncGetAttributes(&fa, traj_dist_filter_kernel<true>);
}

}  // namespace tdq
