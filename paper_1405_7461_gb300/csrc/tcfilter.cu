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
// Roles in a CTA of 5 warps (two CTAs per SM):
//   warp 4, one thread: the producer -- bulk copies (cp.async.bulk, the TMA
//     engine) of each pass's 4 KB of entry records into an 8-stage ring, of
//     each run's 4 KB of query records into one of two buffers, and the MMA
//     of each pass into one of two accumulator stages (256 TMEM columns),
//     each completion signalled through an mbarrier by tcgen05.commit;
//   warps 0-3: the epilogue -- warp w reads accumulator lanes 32w..32w+31
//     (one entry each) with tcgen05.ld, 32 columns (one tile) at a time, ORs
//     the 32 values' bits and, only where a sign bit is set (v < 0: the
//     spheres can meet), builds the entry's 32-bit survivor mask, then
//     appends the survivors (entry, query) through a per-warp buffer.
// Tiles whose own range misses a pass are skipped.  Every wait is bounded;
// a wait that runs out sets error bit 2 (reported as TDQ_ERR_TIMEOUT) and the
// CTA winds down, waiting for its own copies and MMAs in flight before it
// frees its tensor memory.
#include "pipeline.cuh"
#include "tcgrid.cuh"

namespace tdq {
namespace {

constexpr int kTcEpiWarps = 4;
constexpr int kTcThreads = 32 * (kTcEpiWarps + 1);
constexpr int kTcM = 128;                   // entries per pass (MMA M)
constexpr int kTcN = 128;                   // query slots per supertile (MMA N)
constexpr int kTcTiles = kTcN / kQT;        // tiles of 32 per supertile
constexpr int kTcAStages = 8;               // ring of entry-record stages
constexpr int kTcAcc = 2;                   // accumulator stages
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
    unsigned long long a_full[kTcAStages], a_empty[kTcAStages];
    unsigned long long acc_full[kTcAcc], acc_empty[kTcAcc];
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
// Wait for the completion of the phase of parity `parity`; false when it did
// not come within kTcWaitCycles or the CTA is winding down.
__device__ __noinline__ bool bar_wait(unsigned long long *b, uint32_t parity, volatile int *abort)
{
    const long long t0 = clock64();
    for (;;) {
        uint32_t ok;
        asm volatile(
            "{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2; selp.u32 %0, 1, 0, p; }"
            : "=r"(ok)
            : "r"(smem_addr(b)), "r"(parity)
            : "memory");
        if (ok) return true;
        if (*abort || clock64() - t0 > kTcWaitCycles) return false;
    }
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

// 32 consecutive accumulator columns of this warp's 32 lanes (one value per
// column into v[0..31]) and the wait for them.
__device__ __forceinline__ void tc_load32(uint32_t taddr, uint32_t (&v)[32])
{
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
          "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]),
          "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]),
          "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
        : "r"(taddr)
        : "memory");
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
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

// The producer: bulk copies and MMAs, in pass order, loads running up to
// kTcAStages passes ahead.  Returns false if a wait ran out.
__device__ bool tc_produce(const TcArgs &a, TcSmem &sm, uint32_t tmem, unsigned long long ibeg,
                           unsigned long long iend, uint64_t &n_loaded, uint64_t &n_mma, uint32_t &b_loaded,
                           uint32_t &b_used)
{
    volatile int *abort = &sm.abort;
    TcRun rl, rm;
    bool hl = tc_first_run(a, ibeg, iend, rl);
    bool hm = hl;
    rm = rl;
    uint32_t pl = 0, pm = 0;  // pass within the load / MMA cursor's run
    uint64_t gl = 0, gm = 0;  // passes loaded / multiplied
    uint32_t rix = 0;         // index of the MMA cursor's run (B buffer rix & 1)
    b_loaded = b_used = 0;    // runs whose query records were fetched / waited for
    if (hm) {
        bar_expect(&sm.b_full[0], kTcBBytes);
        bulk_load(sm.b[0], a.q_rec + rm.s * (kTcBBytes / 16), kTcBBytes, &sm.b_full[0]);
        b_loaded = 1;
    }
    bool ok = true;
    while (hm && ok) {
        while (hl && gl < gm + kTcAStages) {
            const uint32_t s = (uint32_t)(gl % kTcAStages);
            if (gl >= kTcAStages && !(ok = bar_wait(&sm.a_empty[s], (uint32_t)((gl / kTcAStages - 1) & 1), abort)))
                break;
            bar_expect(&sm.a_full[s], kTcPassBytes);
            bulk_load(sm.a[s], a.e_rec + (uint64_t)(rl.p0 + (int64_t)kTcM * pl) * 2, kTcPassBytes, &sm.a_full[s]);
            gl++;
            if (++pl == rl.np) {
                pl = 0;
                hl = tc_next_run(a, ibeg, iend, rl);
            }
        }
        if (!ok) break;
        const uint32_t bsel = rix & 1;
        if (pm == 0) {
            if (!(ok = bar_wait(&sm.b_full[bsel], (rix >> 1) & 1, abort))) break;
            b_used = rix + 1;
        }
        const uint32_t s = (uint32_t)(gm % kTcAStages), acc = (uint32_t)(gm % kTcAcc);
        if (!(ok = bar_wait(&sm.a_full[s], (uint32_t)((gm / kTcAStages) & 1), abort))) break;
        if (gm >= kTcAcc && !(ok = bar_wait(&sm.acc_empty[acc], (uint32_t)((gm / kTcAcc - 1) & 1), abort))) break;
        tc_fence_after();
        tc_mma(tmem + acc * kTcN, smem_desc(sm.a[s]), smem_desc(sm.b[bsel]));
        tc_commit(&sm.acc_full[acc]);
        tc_commit(&sm.a_empty[s]);
        gm++;
        const bool last_of_run = pm + 1 == rm.np;
        if (last_of_run) tc_commit(&sm.b_free[bsel]);
        if (pm == 0) {
            // fetch the next run's query records into the other buffer once
            // the run before this one no longer reads it
            TcRun nx = rm;
            if (tc_next_run(a, ibeg, iend, nx)) {
                const uint32_t nb = bsel ^ 1;
                if (rix >= 1 && !(ok = bar_wait(&sm.b_free[nb], ((rix - 1) >> 1) & 1, abort))) break;
                bar_expect(&sm.b_full[nb], kTcBBytes);
                bulk_load(sm.b[nb], a.q_rec + nx.s * (kTcBBytes / 16), kTcBBytes, &sm.b_full[nb]);
                b_loaded = rix + 2;
            }
        }
        if (last_of_run) {
            pm = 0;
            rix++;
            hm = tc_next_run(a, ibeg, iend, rm);
        } else {
            pm++;
        }
    }
    n_loaded = gl;
    n_mma = gm;
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
            bar_init(&sm.a_empty[i], 1);
        }
        for (int i = 0; i < kTcAcc; i++) {
            bar_init(&sm.acc_full[i], 1);
            bar_init(&sm.acc_empty[i], kTcEpiWarps);
        }
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
            uint64_t n_loaded = 0, n_mma = 0;
            uint32_t b_loaded = 0, b_used = 0;
            const bool ok = tc_produce(a, sm, tmem, ibeg, iend, n_loaded, n_mma, b_loaded, b_used);
            if (!ok) {
                atomicOr(&ctr->error, 2u);
                *abort = 1;
            }
            // wind down: every MMA issued has finished (before the tensor
            // memory is freed) and every copy issued has landed (before the
            // CTA's shared memory goes away)
            tc_commit(&sm.drain);
            int quiet = 0;
            bar_wait(&sm.drain, 0, &quiet);
            for (uint64_t g = n_mma; g < n_loaded; g++)
                bar_wait(&sm.a_full[g % kTcAStages], (uint32_t)((g / kTcAStages) & 1), &quiet);
            for (uint32_t j = b_used; j < b_loaded; j++) bar_wait(&sm.b_full[j & 1], (j >> 1) & 1, &quiet);
        }
    } else {
        // epilogue warp: accumulator lanes 32*warp .. 32*warp + 31
        uint2 *sbuf = sm.surv[warp];
        int nbuf = 0;
        unsigned long long n_inter = 0;
        const uint64_t nvalid = ctr->valid_queries;
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
        int64_t tlo[kTcTiles], thi[kTcTiles];
        int tnq[kTcTiles];
        auto run_tiles = [&]() {
#pragma unroll
            for (int g = 0; g < kTcTiles; g++) {
                const uint64_t t = r.s * kTcTiles + g;
                const int64_t left = (int64_t)nvalid - (int64_t)t * kQT;
                tnq[g] = t < args.ntiles ? (int)max((int64_t)0, min(left, (int64_t)kQT)) : 0;
                tlo[g] = tnq[g] ? args.tile_lo[t] : 0;
                thi[g] = tnq[g] ? args.tile_hi[t] : 0;
                // candidates: the tile's range inside this run, times its query segments
                if (warp == 0 && lane == 0 && tnq[g]) {
                    const int64_t c0 = max(tlo[g], r.eb), c1 = min(thi[g], r.ee);
                    if (c1 > c0) n_inter += (unsigned long long)(c1 - c0) * (unsigned long long)tnq[g];
                }
            }
        };
        if (h) run_tiles();
        while (h) {
            const uint32_t acc = (uint32_t)(gm % kTcAcc);
            // one lane waits, the warp follows its verdict (the tensor-memory
            // loads below need all 32 lanes)
            int got = 0;
            if (lane == 0) got = bar_wait(&sm.acc_full[acc], (uint32_t)((gm / kTcAcc) & 1), abort);
            got = __shfl_sync(kFull, got, 0);
            if (!got) {
                if (lane == 0) {
                    atomicOr(&ctr->error, 2u);
                    *abort = 1;
                }
                break;
            }
            tc_fence_after();
            const int64_t pb = r.p0 + (int64_t)kTcM * p;
            const int64_t lo_run = max(pb, r.eb), hi_run = min(pb + kTcM, r.ee);
            const int64_t e = pb + 32 * warp + lane;
            const bool e_in = e >= lo_run && e < hi_run;
#pragma unroll
            for (int g = 0; g < kTcTiles; g++) {
                if (tnq[g] == 0 || tlo[g] >= hi_run || thi[g] <= lo_run) continue;  // warp-uniform
                uint32_t v[32];
                tc_load32(tmem + ((uint32_t)(32 * warp) << 16) + acc * kTcN + g * kQT, v);
                uint32_t any = 0;
#pragma unroll
                for (int j = 0; j < 32; j += 2) any |= v[j] | v[j + 1];
                const bool hit = (any >> 31) && e_in && e >= tlo[g] && e < thi[g];
                if (!__any_sync(kFull, hit)) continue;
                uint32_t m = 0;
                if (hit) {
#pragma unroll
                    for (int j = 0; j < 32; j++) m |= (v[j] >> 31) << j;
                    if (tnq[g] < 32) m &= (1u << tnq[g]) - 1u;
                }
                const int cnt = __popc(m);
                int incl = cnt;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const int y = __shfl_up_sync(kFull, incl, o);
                    if (lane >= o) incl += y;
                }
                const int tot = __shfl_sync(kFull, incl, 31);
                if (tot == 0) continue;
                if (nbuf + tot > kTcSurvBuf) flush();
                const bool direct = tot > kTcSurvBuf;
                unsigned long long pos = nbuf + (incl - cnt);
                if (direct) {
                    unsigned long long base = 0;
                    if (lane == 0) base = atomicAdd(&ctr->survivors, (unsigned long long)tot);
                    pos = __shfl_sync(kFull, base, 0) + (incl - cnt);
                }
                const uint32_t q0 = (uint32_t)((r.s * kTcTiles + g) * kQT);
                while (m) {
                    const int bit = __ffs(m) - 1;
                    m &= m - 1;
                    const uint2 sv = make_uint2((uint32_t)e, q0 + bit);
                    if (!direct)
                        sbuf[pos] = sv;
                    else if (pos < a.surv_cap)
                        a.surv[pos] = sv;
                    pos++;
                }
                __syncwarp();
                if (!direct) nbuf += tot;
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) bar_arrive(&sm.acc_empty[acc]);
            gm++;
            if (++p == r.np) {
                p = 0;
                h = tc_next_run(a, ibeg, iend, r);
                if (h) run_tiles();
            }
        }
        flush();
        if (warp == 0 && lane == 0 && n_inter) atomicAdd(&ctr->interactions, n_inter);
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
    return launch_refine_kernel(FilterArgs{ta.p, ta.surv, ta.surv_cap}, sm_count, stream);
}

cudaError_t load_tc_module()
{
    cudaFuncAttributes fa;
    return cudaFuncGetAttributes(&fa, traj_dist_tc_filter_kernel);
}

}  // namespace tdq
