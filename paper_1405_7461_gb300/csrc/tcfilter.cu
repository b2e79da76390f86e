// Tensor-core pre-test (TDQ_MODE_TC_FILTER): the sphere test of every
// candidate pair as an exact integer GEMM on the 5th-generation tensor cores
// (records and bound: tcgrid.cuh), then the FP64 refine kernel of the filter
// mode over the survivors (Sec. 5, Algorithm 1), so that the result set
// equals the plain FP64 search's.
//
// Work: query segments are sorted and cut into tiles of 32 (one bit each in a
// survivor mask); four consecutive tiles form a supertile of 128 query
// segments whose entry range is the union of its tiles' candidate ranges.
// Work items are (supertile, chunk of entries); the CTAs of a persistent grid
// take contiguous item ranges, i.e. runs of consecutive sorted entries of one
// supertile each.  A run is cut into passes of 128 entries (starting on a
// multiple of 8, the records' group size): per pass one
//     tcgen05.mma.cta_group::1.kind::f16  M = 128 entries, N = 128 queries, K = 16
// from shared memory into a 128 x 128 FP32 accumulator in tensor memory.
//
// Roles in a CTA of 10 warps (two CTAs per SM):
//   warp 8, one thread: the loader -- bulk copies (cp.async.bulk, the TMA
//     engine) of each pass's 4 KB of entry records into an 8-stage ring and
//     of each run's 4 KB of query records into one of two buffers;
//   warp 9, one thread: the MMA issuer -- the MMA of each pass into one of
//     two accumulator stages (256 TMEM columns), its completion signalled
//     through the stage's mbarrier by tcgen05.commit;
//   warps 0-7: the epilogue, two groups of four -- group w / 4 takes the
//     passes of its accumulator stage (every other pass), so that two passes
//     are looked at at once; warp w reads accumulator lanes 32 (w % 4) .. + 31
//     (one entry each) and the 32 columns of each of the four tiles whose own
//     range meets the pass, two tiles at a time with tcgen05.ld (one wait per
//     pair), ORs each tile's 32 values and, only where a sign bit is set
//     (v < 0: the spheres can meet), builds the entry's 32-bit survivor mask,
//     hands the stage back once all four tiles are read, and then appends the
//     survivors (entry, query) through a per-warp shared-memory buffer at
//     ranks taken by a warp scan.
// Tiles whose own range misses a pass are skipped.  Every wait is bounded;
// a wait that runs out sets error bit 2 (reported as TDQ_ERR_TIMEOUT) and the
// CTA winds down, waiting for its own copies and MMAs in flight before it
// frees its tensor memory.
#include "pipeline.cuh"
#include "tcgrid.cuh"

namespace tdq {
namespace {

constexpr int kTcEpiWarps = 8;             // two warpgroups: lanes by warp % 4, tiles 2 (warp / 4) and + 1
constexpr int kTcThreads = 32 * (kTcEpiWarps + 2);  // + the loader warp and the MMA warp
constexpr int kTcM = 128;                   // entries per pass (MMA M)
constexpr int kTcN = 128;                   // query slots per supertile (MMA N)
constexpr int kTcTiles = kTcN / kQT;        // tiles of 32 per supertile
constexpr int kTcAStages = 8;               // ring of entry-record stages
constexpr int kTcAcc = 2;                   // accumulator stages (256 TMEM columns; two CTAs fill an SM)
constexpr int kTcGroupWarps = kTcEpiWarps / kTcAcc;  // epilogue warps per accumulator stage (one per lane quarter)
constexpr uint32_t kTcPassBytes = kTcM * 32;
constexpr uint32_t kTcBBytes = kTcN * 32;
constexpr uint32_t kTcCols = kTcAcc * kTcN;  // tensor-memory columns per CTA
constexpr int kTcSurvBuf = 256;
constexpr long long kTcWaitCycles = 1LL << 31;  // ~1 s at the GB300's clocks
// instruction descriptor of kind::f16: FP32 accumulator (bits 4-5 = 1),
// FP16 A and B (bits 7-12 = 0), both K-major (bits 15-16 = 0), N >> 3 at
// bit 17, M >> 4 at bit 24
constexpr uint32_t kTcIdesc = (1u << 4) | ((uint32_t)(kTcN >> 3) << 17) | ((uint32_t)(kTcM >> 4) << 24);
// dynamic shared memory requested per CTA: more than the kernel uses, so
// that at most two CTAs share an SM (their 2 x 256 TMEM columns fill it, so
// no allocation ever waits)
constexpr size_t kTcSmemRequest = 100 * 1024;

struct TcSmem {
    uint4 a[kTcAStages][kTcPassBytes / 16];
    uint4 b[2][kTcBBytes / 16];
    uint2 surv[kTcEpiWarps][kTcSurvBuf];
    int4 tiles[kTcEpiWarps][kTcTiles];  // each epilogue warp's copy of the run's tiles: (segments, lo, hi) rel. to p0
    unsigned long long a_full[kTcAStages], mma_done[kTcAStages];
    unsigned long long acc_empty[kTcAcc];
    unsigned long long b_full[2], b_free[2], drain;
    uint32_t tmem_base;
    int abort;
};
static_assert(sizeof(TcSmem) + 1024 <= kTcSmemRequest, "shared memory layout fits the request");

__device__ __forceinline__ uint32_t smem_addr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void bar_init(unsigned long long *b, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(b)), "r"(count) : "memory");
}
__device__ __forceinline__ void bar_arrive(unsigned long long *b)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(b)) : "memory");
}
__device__ __forceinline__ void bar_expect(unsigned long long *b, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(b)), "r"(bytes) : "memory");
}
// Non-blocking test of the completion of the phase of parity `parity`.
// (try_wait was measured to suspend the waiting thread for 1000-2000 cycles
// past the phase's completion, which at one MMA per pass dominated the
// pipeline; every wait here is a spin on test_wait instead.)
__device__ __forceinline__ bool bar_test(unsigned long long *b, uint32_t parity)
{
    uint32_t ok;
    asm volatile("{ .reg .pred p; mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2; selp.u32 %0, 1, 0, p; }"
                 : "=r"(ok)
                 : "r"(smem_addr(b)), "r"(parity)
                 : "memory");
    return ok;
}
// Wait for the completion of the phase of parity `parity`; false when it did
// not come within kTcWaitCycles or the CTA is winding down.
__device__ __noinline__ bool bar_wait_slow(unsigned long long *b, uint32_t parity, volatile int *abort)
{
    const long long t0 = clock64();
    for (;;) {
        if (bar_test(b, parity)) return true;
        if (*abort || clock64() - t0 > kTcWaitCycles) return false;
    }
}
__device__ __forceinline__ bool bar_wait(unsigned long long *b, uint32_t parity, volatile int *abort)
{
    return bar_test(b, parity) || bar_wait_slow(b, parity, abort);
}

__device__ __forceinline__ void bulk_load(void *dst, const void *src, uint32_t bytes, unsigned long long *b)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_addr(dst)),
                 "l"(src), "r"(bytes), "r"(smem_addr(b))
                 : "memory");
}

// Shared-memory matrix descriptor: no swizzle, K-major, core matrices 128 B
// apart along K (leading byte offset) and 256 B apart along M/N (stride byte
// offset), descriptor version 1 at bit 46.
__device__ __forceinline__ uint64_t smem_desc(const void *p)
{
    return (uint64_t)((smem_addr(p) >> 4) & 0x3FFF) | ((uint64_t)(128 >> 4) << 16) | ((uint64_t)(256 >> 4) << 32) |
           ((uint64_t)1 << 46);
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tc_mma(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc)
{
    asm volatile(
        "{ .reg .pred p; setp.ne.b32 p, %4, 0;\n"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p; }" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(kTcIdesc), "r"(0)
        : "memory");
}
__device__ __forceinline__ void tc_commit(unsigned long long *b)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_addr(b))
                 : "memory");
}

__device__ __forceinline__ void tc_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// 32 consecutive accumulator columns of this warp's 32 lanes into v[0..31]
// (tc_wait_ld waits for them).
__device__ __forceinline__ void tc_load32_nowait(uint32_t taddr, uint32_t *v)
{
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
                 "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
                 : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
                   "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]),
                   "=r"(v[15]), "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]),
                   "=r"(v[22]), "=r"(v[23]), "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]),
                   "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
                 : "r"(taddr)
                 : "memory");
}

// Sign bits of 32 words as a mask (bit j = sign of v[j]): four independent
// chains of funnel shifts, joined.
__device__ __forceinline__ uint32_t signs32(const uint32_t *v)
{
    uint32_t m[4] = {0u, 0u, 0u, 0u};
#pragma unroll
    for (int j = 7; j >= 0; j--) {
#pragma unroll
        for (int c = 0; c < 4; c++) m[c] = __funnelshift_l(v[8 * c + j], m[c], 1);
    }
    return m[0] | (m[1] << 8) | (m[2] << 16) | (m[3] << 24);
}

// Bitwise OR of 32 words as a tree of three-input ORs (depth 4, not a chain
// of 16 dependent operations).
__device__ __forceinline__ uint32_t or32(const uint32_t *v)
{
    uint32_t a[11];
#pragma unroll
    for (int k = 0; k < 10; k++) a[k] = v[3 * k] | v[3 * k + 1] | v[3 * k + 2];
    a[10] = v[30] | v[31];
    const uint32_t b0 = a[0] | a[1] | a[2], b1 = a[3] | a[4] | a[5], b2 = a[6] | a[7] | a[8], b3 = a[9] | a[10];
    return (b0 | b1 | b2) | b3;
}

// A run: the CTA's items in supertile s, as sorted entry positions [eb, ee);
// its passes start at p0 (eb rounded down to a multiple of 8).
struct TcRun {
    uint64_t s;
    int64_t eb, ee, p0;
    uint32_t np;
};

__device__ __forceinline__ void tc_run_bounds(const TcArgs &a, uint64_t s, unsigned long long ibeg,
                                              unsigned long long iend, TcRun &r)
{
    const unsigned long long wb = a.st_work[s], wn = a.st_work[s + 1];
    const int64_t lo = a.st_lo[s], hi = a.st_hi[s];
    r.s = s;
    r.eb = lo + (int64_t)(max(ibeg, wb) - wb) * a.p.chunk;
    r.ee = min(lo + (int64_t)(min(iend, wn) - wb) * a.p.chunk, hi);
    r.p0 = r.eb & ~(int64_t)7;
    r.np = (uint32_t)((r.ee - r.p0 + kTcM - 1) / kTcM);
}

// The run holding item ibeg (the last supertile whose first item is <= ibeg).
__device__ __forceinline__ bool tc_first_run(const TcArgs &a, unsigned long long ibeg, unsigned long long iend,
                                             TcRun &r)
{
    if (ibeg >= iend) return false;
    uint64_t lo = 0, hi = a.nsuper;
    while (hi - lo > 1) {
        const uint64_t mid = (lo + hi) >> 1;
        if (a.st_work[mid] <= ibeg) lo = mid; else hi = mid;
    }
    tc_run_bounds(a, lo, ibeg, iend, r);
    return true;
}

__device__ __forceinline__ bool tc_next_run(const TcArgs &a, unsigned long long ibeg, unsigned long long iend,
                                            TcRun &r)
{
    uint64_t s = r.s + 1;
    while (s < a.nsuper && a.st_work[s + 1] == a.st_work[s]) s++;
    if (s >= a.nsuper || a.st_work[s] >= iend) return false;
    tc_run_bounds(a, s, ibeg, iend, r);
    return true;
}

// The loader: bulk copies of the entry records of every pass into the ring
// of kTcAStages stages (a stage is reused once the MMA that read it is done)
// and of each run's query records into one of two buffers (reused once the
// run before the previous one has finished its MMAs).  Returns false if a
// wait ran out; n_loaded / b_loaded: copies issued.
__device__ bool tc_load_all(const TcArgs &a, TcSmem &sm, unsigned long long ibeg, unsigned long long iend,
                            uint64_t &n_loaded, uint32_t &b_loaded)
{
    volatile int *abort = &sm.abort;
    TcRun r;
    bool h = tc_first_run(a, ibeg, iend, r);
    uint32_t p = 0, rix = 0;
    uint64_t g = 0;
    bool ok = true;
    b_loaded = 0;
    while (h) {
        if (!TDQ_DBG(a.p.ctr, kDbgTcRecords, r.p0 >= 0 && (uint64_t)(r.p0 + (int64_t)kTcM * (p + 1)) <= a.n_rec) ||
            !TDQ_DBG(a.p.ctr, kDbgTcSuper, r.s < a.nsuper)) {
            ok = false;
            break;
        }
        if (p == 0) {
            const uint32_t bb = rix & 1;
            if (rix >= 2 && !(ok = bar_wait(&sm.b_free[bb], ((rix - 2) >> 1) & 1, abort))) break;
            bar_expect(&sm.b_full[bb], kTcBBytes);
            bulk_load(sm.b[bb], a.q_rec + r.s * (kTcBBytes / 16), kTcBBytes, &sm.b_full[bb]);
            b_loaded = rix + 1;
        }
        const uint32_t s = (uint32_t)(g % kTcAStages);
        if (g >= kTcAStages && !(ok = bar_wait(&sm.mma_done[s], (uint32_t)((g / kTcAStages - 1) & 1), abort))) break;
        bar_expect(&sm.a_full[s], kTcPassBytes);
        bulk_load(sm.a[s], a.e_rec + (uint64_t)(r.p0 + (int64_t)kTcM * p) * 2, kTcPassBytes, &sm.a_full[s]);
        g++;
        if (++p == r.np) {
            p = 0;
            rix++;
            h = tc_next_run(a, ibeg, iend, r);
        }
    }
    n_loaded = g;
    return ok;
}

// The MMA issuer: per pass, once its entry records (and, first in a run, the
// run's query records) have landed and the epilogue has handed back the
// accumulator stage, one MMA and one commit to the pass's stage barrier
// (which the epilogue waits on and which frees the stage for the loader);
// after a run's last MMA a commit frees its query buffer.
__device__ bool tc_mma_all(const TcArgs &a, TcSmem &sm, uint32_t tmem, unsigned long long ibeg,
                           unsigned long long iend, uint64_t &n_mma)
{
    volatile int *abort = &sm.abort;
    TcRun r;
    bool h = tc_first_run(a, ibeg, iend, r);
    uint32_t p = 0, rix = 0;
    uint64_t g = 0;
    bool ok = true;
    while (h) {
        const uint32_t bb = rix & 1;
        if (p == 0 && !(ok = bar_wait(&sm.b_full[bb], (rix >> 1) & 1, abort))) break;
        const uint32_t s = (uint32_t)(g % kTcAStages), acc = (uint32_t)(g % kTcAcc);
        if (!(ok = bar_wait(&sm.a_full[s], (uint32_t)((g / kTcAStages) & 1), abort))) break;
        if (g >= kTcAcc && !(ok = bar_wait(&sm.acc_empty[acc], (uint32_t)((g / kTcAcc - 1) & 1), abort))) break;
        tc_fence_after();
        tc_mma(tmem + acc * kTcN, smem_desc(sm.a[s]), smem_desc(sm.b[bb]));
        tc_commit(&sm.mma_done[s]);
        g++;
        if (++p == r.np) {
            tc_commit(&sm.b_free[bb]);
            p = 0;
            rix++;
            h = tc_next_run(a, ibeg, iend, r);
        }
    }
    n_mma = g;
    return ok;
}

}  // namespace

__global__ void __launch_bounds__(kTcThreads, 2) traj_dist_tc_filter_kernel(TcArgs a)
{
    extern __shared__ __align__(1024) unsigned char tc_smem_raw[];
    TcSmem &sm = *reinterpret_cast<TcSmem *>(
        (unsigned char *)(((uintptr_t)tc_smem_raw + 1023) & ~(uintptr_t)1023));
    const PairArgs &args = a.p;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    DevCounters *ctr = args.ctr;
    const unsigned long long total = a.st_work[a.nsuper];
    const unsigned long long per = (total + gridDim.x - 1) / gridDim.x;
    const unsigned long long ibeg = min((unsigned long long)blockIdx.x * per, total);
    const unsigned long long iend = min(ibeg + per, total);

    if (threadIdx.x == 0) {
        for (int i = 0; i < kTcAStages; i++) {
            bar_init(&sm.a_full[i], 1);
            bar_init(&sm.mma_done[i], 1);
        }
        for (int i = 0; i < kTcAcc; i++) bar_init(&sm.acc_empty[i], kTcGroupWarps);
        for (int i = 0; i < 2; i++) {
            bar_init(&sm.b_full[i], 1);
            bar_init(&sm.b_free[i], 1);
        }
        bar_init(&sm.drain, 1);
        sm.abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(&sm.tmem_base)),
                     "r"(kTcCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = sm.tmem_base;
    volatile int *abort = &sm.abort;

    if (warp == kTcEpiWarps) {
        if (lane == 0) {
            uint64_t n_loaded = 0;
            uint32_t b_loaded = 0;
            if (!tc_load_all(a, sm, ibeg, iend, n_loaded, b_loaded)) {
                atomicOr(&ctr->error, 2u);
                *abort = 1;
            }
            // wind down: every copy issued has landed before the CTA's
            // shared memory goes away (copies the MMA issuer consumed have
            // landed already; the waits then return at once)
            int quiet = 0;
            for (uint64_t g = n_loaded > kTcAStages ? n_loaded - kTcAStages : 0; g < n_loaded; g++)
                bar_wait(&sm.a_full[g % kTcAStages], (uint32_t)((g / kTcAStages) & 1), &quiet);
            for (uint32_t j = b_loaded > 2 ? b_loaded - 2 : 0; j < b_loaded; j++)
                bar_wait(&sm.b_full[j & 1], (j >> 1) & 1, &quiet);
        }
    } else if (warp == kTcEpiWarps + 1) {
        if (lane == 0) {
            uint64_t n_mma = 0;
            if (!tc_mma_all(a, sm, tmem, ibeg, iend, n_mma)) {
                atomicOr(&ctr->error, 2u);
                *abort = 1;
            }
            if (n_mma) atomicAdd(&ctr->mma_issued, (unsigned long long)n_mma);
            // wind down: every MMA issued has finished before the tensor
            // memory is freed
            tc_commit(&sm.drain);
            int quiet = 0;
            bar_wait(&sm.drain, 0, &quiet);
        }
    } else {
        // epilogue warp: accumulator lanes 32 quarter .. 32 quarter + 31 (one
        // entry each), all four tiles, of the passes of its group (the passes
        // g with g % kTcAcc == group, i.e. its accumulator stage): the two
        // groups work on two passes at once
        const int quarter = warp & 3, group = warp / kTcGroupWarps;
        uint2 *sbuf = sm.surv[warp];
        int nbuf = 0;  // (warp-uniform)
        unsigned long long n_inter = 0;
        const uint64_t nvalid = ctr->valid_queries;
        // moves the buffered survivors to the list (called by the whole warp)
        auto flush = [&]() {
            if (nbuf == 0) return;
            unsigned long long base = 0;
            if (lane == 0) base = atomicAdd(&ctr->survivors, (unsigned long long)nbuf);
            base = __shfl_sync(kFull, base, 0);
            __syncwarp();
            for (int i = lane; i < nbuf; i += 32)
                if (base + i < a.surv_cap) a.surv[base + i] = sbuf[i];
            __syncwarp();
            nbuf = 0;
        };
        TcRun r;
        bool h = tc_first_run(a, ibeg, iend, r);
        uint32_t p = 0;
        uint64_t gm = 0;
        // the run's four tiles (lane k computes tile k): query segments, and
        // the part of the tile's own range inside the run, relative to p0
        int4 *tiles = sm.tiles[warp];
        auto run_tiles = [&]() {
            __syncwarp();  // the previous run's tiles are no longer read
            if (lane < kTcTiles) {
                const uint64_t t = r.s * kTcTiles + lane;
                const int64_t left = (int64_t)nvalid - (int64_t)t * kQT;
                int n = t < args.ntiles ? (int)max((int64_t)0, min(left, (int64_t)kQT)) : 0;
                const int64_t lo = n ? max(args.tile_lo[t], r.eb) : 0, hi = n ? min(args.tile_hi[t], r.ee) : 0;
                if (hi <= lo) n = 0;
                tiles[lane] = make_int4(n, (int32_t)(lo - r.p0), (int32_t)(hi - r.p0), 0);
                // candidates: the tile's range inside this run, times its query segments
                if (quarter == 0 && group == 0 && n) n_inter += (unsigned long long)(hi - lo) * (unsigned long long)n;
            }
            __syncwarp();
        };
        // one tile's survivor mask of this lane's entry el (relative to p0):
        // bit j set where the value of query slot j is negative (v < 0: the
        // spheres can meet); the OR of the 32 values decides whether the
        // mask needs building at all
        auto mask_of = [&](int k, const uint32_t *v, bool act, int32_t el) -> uint32_t {
            if (!act) return 0u;
            const int4 ti = tiles[k];
            const bool hit = el >= ti.y && el < ti.z && (or32(v) >> 31);
            if (!__any_sync(kFull, hit)) return 0u;
            uint32_t m = 0u;
            if (hit) {
                m = signs32(v);
                if (ti.x < 32) m &= (1u << ti.x) - 1u;
            }
            return m;
        };
        // the survivors (entry, query) of one tile's masks into the warp's
        // buffer at ranks taken by a warp scan, the buffer flushed to the list
        // when full; a tile with more survivors than the buffer holds goes
        // straight to the list
        auto append = [&](int k, uint32_t m, int32_t el) {
            if (!__any_sync(kFull, m != 0u)) return;
            const uint32_t e = (uint32_t)(r.p0 + el);
            const uint32_t q0 = (uint32_t)((r.s * kTcTiles + k) * kQT);
            // (the highest set bit of m is the last query slot used)
            if (m && !TDQ_DBG(ctr, kDbgTcSurvivor, e < args.n_entries && q0 + 32 - __clz(m) <= nvalid)) m = 0u;
            const int cnt = __popc(m);
            int incl = cnt;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(kFull, incl, o);
                if (lane >= o) incl += y;
            }
            const int total = __shfl_sync(kFull, incl, 31);
            if (total == 0) return;
            if (nbuf + total > kTcSurvBuf) flush();
            const bool direct = total > kTcSurvBuf;
            unsigned long long pos = nbuf + (incl - cnt);
            if (direct) {
                unsigned long long base = 0;
                if (lane == 0) base = atomicAdd(&ctr->survivors, (unsigned long long)total);
                pos = __shfl_sync(kFull, base, 0) + (incl - cnt);
            }
            while (m) {
                const int bit = __ffs(m) - 1;
                m &= m - 1;
                const uint2 sv = make_uint2(e, q0 + bit);
                if (!direct) {
                    if (TDQ_DBG(ctr, kDbgTcSurvivor, pos < (unsigned long long)kTcSurvBuf)) sbuf[pos] = sv;
                } else if (pos < a.surv_cap) {
                    a.surv[pos] = sv;
                }
                pos++;
            }
            __syncwarp();
            if (!direct) nbuf += total;
        };
        if (h) run_tiles();
        while (h) {
            if ((int)(gm % kTcAcc) == group) {
                const uint32_t acc = (uint32_t)group;
                // the pass's MMA is done: one lane waits, the warp follows its
                // verdict (the tensor-memory loads below need all 32 lanes)
                int got = 0;
                if (lane == 0)
                    got = bar_wait(&sm.mma_done[gm % kTcAStages], (uint32_t)((gm / kTcAStages) & 1), abort);
                got = __shfl_sync(kFull, got, 0);
                if (!got) {
                    if (lane == 0) {
                        atomicOr(&ctr->error, 2u);
                        *abort = 1;
                    }
                    break;
                }
                // the pass's entries relative to p0; which tiles' own ranges
                // meet them (warp-uniform)
                const int32_t pr = (int32_t)(kTcM * p);
                unsigned act = 0u;  // bit k: tile k's own range meets the pass
#pragma unroll
                for (int k = 0; k < kTcTiles; k++) {
                    const int4 ti = tiles[k];
                    act |= (ti.x > 0 && ti.y < pr + kTcM && ti.z > pr) ? 1u << k : 0u;
                }
                const int32_t el = pr + 32 * quarter + lane;  // this lane's entry, relative to p0
                const uint32_t tcol = tmem + ((uint32_t)(32 * quarter) << 16) + acc * kTcN;
                uint32_t v0[kQT], v1[kQT];
                tc_fence_after();
                // tiles 0 and 1 (one wait for both loads), looked at while
                // the accumulator is still held
                if (act & 1u) tc_load32_nowait(tcol, v0);
                if (act & 2u) tc_load32_nowait(tcol + kQT, v1);
                if (act & 3u) tc_wait_ld();
                const uint32_t m0 = mask_of(0, v0, act & 1u, el), m1 = mask_of(1, v1, act & 2u, el);
                // tiles 2 and 3, then the stage goes back to the MMA issuer;
                // the survivors are appended after that
                if (act & 4u) tc_load32_nowait(tcol + 2 * kQT, v0);
                if (act & 8u) tc_load32_nowait(tcol + 3 * kQT, v1);
                if (act & 12u) tc_wait_ld();
                const uint32_t m2 = mask_of(2, v0, act & 4u, el), m3 = mask_of(3, v1, act & 8u, el);
                tc_fence_before();
                __syncwarp();
                if (lane == 0) bar_arrive(&sm.acc_empty[acc]);
                append(0, m0, el);
                append(1, m1, el);
                append(2, m2, el);
                append(3, m3, el);
            }
            gm++;
            if (++p == r.np) {
                p = 0;
                h = tc_next_run(a, ibeg, iend, r);
                if (h) run_tiles();
            }
        }
        flush();
        if (n_inter) atomicAdd(&ctr->interactions, n_inter);
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTcCols) : "memory");
}

// The tensor-core pre-test as a persistent grid of two CTAs per SM, then the
// filter mode's FP64 refine kernel over its survivors; mid (may be null) is
// recorded between them with the flags evflags.
cudaError_t launch_tc_filter_kernels(const TcArgs &ta, int sm_count, cudaStream_t stream, cudaEvent_t mid,
                                     unsigned evflags)
{
    static_assert(kTcSmemRequest <= 227 * 1024, "shared memory request");
    cudaError_t e = cudaFuncSetAttribute(traj_dist_tc_filter_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)kTcSmemRequest);
    if (e != cudaSuccess) return e;
    traj_dist_tc_filter_kernel<<<sm_count * 2, kTcThreads, kTcSmemRequest, stream>>>(ta);
    if (mid && (e = cudaEventRecordWithFlags(mid, stream, evflags)) != cudaSuccess) return e;
    return launch_refine_kernel(FilterArgs{ta.p, ta.surv, ta.surv_cap, nullptr, nullptr}, sm_count, stream);
}

cudaError_t load_tc_module()
{
    cudaFuncAttributes fa;
    return cudaFuncGetAttributes(&fa, traj_dist_tc_filter_kernel);
}

}  // namespace tdq
