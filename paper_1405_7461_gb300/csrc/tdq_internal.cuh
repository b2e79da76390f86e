// Internal declarations of libtdq (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "tcgrid.cuh"
#include "tdq.h"

namespace tdq {

// ---------------------------------------------------------------------------
// Time keys.  On GB300 the FP64 pipe issues about two DFMA per clock per SM,
// sixty times fewer than the integer and FP32 pipes, so every comparison of
// times (overlap tests, max/min of span ends) is done on 64-bit integer keys
// whose signed order equals the order of the (finite, non-NaN) doubles.
// The map is an involution, so the double is recovered exactly.
// ---------------------------------------------------------------------------
__host__ __device__ __forceinline__ int64_t key_from_bits(int64_t b)
{
    return b ^ ((b >> 63) & 0x7fffffffffffffffLL);
}

__device__ __forceinline__ int64_t okey(double x)
{
    int64_t b = __double_as_longlong(x);
    if (b == (int64_t)0x8000000000000000ULL) b = 0;  // -0.0 sorts with +0.0
    return key_from_bits(b);
}

__device__ __forceinline__ double key_double(int64_t k)
{
    return __longlong_as_double(key_from_bits(k));
}

// Unsigned radix key with the same order as okey.
__device__ __forceinline__ uint64_t ukey(double x)
{
    return (uint64_t)okey(x) ^ 0x8000000000000000ULL;
}

__device__ __forceinline__ bool finite_bits(double x)
{
    return (__double_as_longlong(x) & 0x7ff0000000000000LL) != 0x7ff0000000000000LL;
}

// Sign tests on the bit pattern (integer pipe).  NaN never reaches them.
__device__ __forceinline__ bool le0(double x)  // x <= 0
{
    return __double_as_longlong(x) <= 0 || __double_as_longlong(x) == (int64_t)0x8000000000000000ULL;
}
__device__ __forceinline__ bool gt0(double x) { return !le0(x); }  // x > 0
__device__ __forceinline__ bool lt0(double x)  // x < 0
{
    int64_t b = __double_as_longlong(x);
    return b < 0 && b != (int64_t)0x8000000000000000ULL;
}
__device__ __forceinline__ bool ge0(double x) { return !lt0(x); }  // x >= 0

// ---------------------------------------------------------------------------
// Launch and allocation helpers shared by the translation units.
constexpr int kBlock = 256;              // threads of the simple one-item-per-thread kernels
constexpr unsigned kFull = 0xffffffffu;  // full warp mask

inline unsigned grid_for(uint64_t n, int block = kBlock)
{
    uint64_t g = (n + block - 1) / block;
    return (unsigned)(g > 0 ? g : 1);
}

// Device view of a host array of `bytes` bytes when all of it lies in
// page-locked memory mapped into the device's address space (cudaHostAlloc,
// cudaHostRegister, pinned tensors); null otherwise.  On a Grace-Blackwell
// node the kernels then read such input in place over the coherent CPU-GPU
// link, so a search needs no staging copies for it.
inline const void *mapped_view(const void *host_ptr, uint64_t bytes)
{
    if (!host_ptr || bytes == 0) return nullptr;
    cudaPointerAttributes a, b;
    if (cudaPointerGetAttributes(&a, host_ptr) != cudaSuccess ||
        cudaPointerGetAttributes(&b, (const char *)host_ptr + bytes - 1) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    if (a.type != cudaMemoryTypeHost || b.type != cudaMemoryTypeHost || !a.devicePointer || !b.devicePointer)
        return nullptr;
    if ((const char *)b.devicePointer - (const char *)a.devicePointer != (ptrdiff_t)(bytes - 1)) return nullptr;
    return a.devicePointer;
}

// Sub-allocation of one device block: 256-byte aligned slices.
template <typename T>
T *carve(char *&p, uint64_t count)
{
    T *r = (T *)p;
    p += (count * sizeof(T) + 255) & ~(uint64_t)255;
    return r;
}
inline uint64_t carve_bytes(uint64_t count, uint64_t size) { return (count * size + 255) & ~(uint64_t)255; }

// Temporal bin of time t (Sec. 4): min(m - 1, floor((t - t_min) / width)),
// 0 below t_min.  Monotone non-decreasing in t: the index build, the
// candidate lookup and the overlap counts rely on one and the same function.
__device__ __forceinline__ int64_t bin_of(double t, double t_min, double width, uint32_t m)
{
    double f = floor((t - t_min) / width);
    if (!(f < (double)(m - 1))) return (int64_t)m - 1;
    if (f < 0.0) return 0;
    return (int64_t)f;
}

// FP32 upper bound of sqrt(a^2 + b^2 + c^2) (every rounding upward).
__device__ __forceinline__ float norm_ru(double a, double b, double c)
{
    const float x = __double2float_ru(fabs(a)), y = __double2float_ru(fabs(b)), z = __double2float_ru(fabs(c));
    return __fsqrt_ru(__fmaf_ru(z, z, __fmaf_ru(y, y, __fmul_ru(x, x))));
}

// Conservative FP32 bounding sphere of a segment piece whose FP64 center is
// (cx,cy,cz) and whose radius is at most r (r and extra are FP32 upper
// bounds), for the filter mode's pre-test.  The center is rounded to
// nearest.  The radius w is widened by 2^-22 * max|c| (more than the
// sqrt(3) * 2^-24 * max|c| the center's rounding can move it, and more than
// any FP64 rounding of the positions the FP64 path evaluates; max|c| is
// bounded through the rounded center, |c| <= |c~| (1 + 2^-23)), by r * 2^-40,
// by `extra` (the threshold d, for a query) and by 2^-60 (so that w > 0 and
// w^2 stays a normal number), then scaled by (1 + 2^-20); every rounding of
// w is upward.  Magnitudes beyond 2^60 get an infinite radius, which never
// rejects.
__device__ __forceinline__ float4 sphere32(double cx, double cy, double cz, float r, float extra)
{
    const float x = __double2float_rn(cx), y = __double2float_rn(cy), z = __double2float_rn(cz);
    const float m = __fmul_ru(fmaxf(fabsf(x), fmaxf(fabsf(y), fabsf(z))), 1.0f + 0x1p-23f);
    float fr = __int_as_float(0x7f800000);
    if (m < 0x1p60f && r < 0x1p60f && extra < 0x1p60f) {
        const float w = __fadd_ru(__fadd_ru(__fmaf_ru(r, 0x1p-40f, r), __fmaf_ru(m, 0x1p-22f, extra)), 0x1p-60f);
        fr = __fmaf_ru(w, 0x1p-20f, w);
    }
    return make_float4(x, y, z, fr);
}

// Device-side counters of one search, cleared by one memset per search.
// ---------------------------------------------------------------------------
struct DevCounters {
    unsigned long long results;        // appended result items (may exceed capacity)
    unsigned long long work_next;      // dynamic work-item dispenser of the pair kernel
    unsigned long long interactions;
    unsigned long long overlap_pairs;
    unsigned long long fp64_pairs;
    unsigned long long valid_queries;  // query segments with a non-empty clipped span
    unsigned long long work_items;
    unsigned long long survivors;      // filter mode: pairs that passed the FP32 pre-test
    unsigned long long sort_n;         // query slots the sort covers (the real ones; padding follows them)
    unsigned long long gather_done;    // blocks of query_gather that have finished (the last one scans)
    unsigned long long pair_done;      // blocks of the last pair kernel that have finished (the last one
                                       // copies the counters to the host mirror)
    unsigned long long mma_issued;     // tensor-core pre-test: MMAs issued
    unsigned long long prep_done;      // blocks of query_prep that have finished (the last one scans the
                                       // bin counts of the counting sort)
    unsigned int error;                // bit 0: invalid query input; bit 1: a pipeline wait ran out;
                                       // bit 2 (debug build): an index bounds check failed
    unsigned int debug_site;           // debug build: the first failed check's site (TdqDebugSite)
};

// Bounds checks of the debug build (compiled with -DTDQ_DEBUG; the GPU
// counterpart of a memory checker, which this library's tests cannot use).
// TDQ_DBG(ctr, site, cond) is the constant true in normal builds; in the
// debug build it evaluates cond and, when it fails, sets error bit 2 and
// records the first failing site, so that the guarded access is skipped and
// the host reports TDQ_ERR_CUDA naming the site -- never a trap.
enum TdqDebugSite : unsigned {
    kDbgPlainTile = 1,      // plain kernel: tile index < tiles
    kDbgPlainChunk = 2,     // plain kernel: entry chunk inside the entries
    kDbgPlainQueries = 3,   // plain kernel: the tile's query slots inside the sorted queries
    kDbgFilterRun = 4,      // FP32 pre-test: a run's entries inside the entries
    kDbgFilterNext = 5,     // FP32 pre-test: the prefetched pass inside the entries
    kDbgFilterQuery = 6,    // FP32 pre-test: a survivor's query inside the valid queries
    kDbgFilterBuf = 7,      // FP32 pre-test: survivor buffer slot
    kDbgRefine = 8,         // refine: a survivor's entry and query positions
    kDbgGatherOrder = 9,    // query_gather: sorted order inside the query slots
    kDbgScatterPos = 10,    // query_scatter: sorted position inside the valid queries
    kDbgRange = 11,         // query_prep: candidate range inside the entries
    kDbgTcRecords = 12,     // tensor-core pre-test: a pass's entry records inside the records
    kDbgTcSuper = 13,       // tensor-core pre-test: supertile index
    kDbgTcSurvivor = 14,    // tensor-core pre-test: a survivor's entry and query positions
    kDbgSmallSlot = 15,     // query_prep_small: sorted slot inside the query slots
};
#ifdef TDQ_DEBUG
__device__ __forceinline__ bool dbg_check(DevCounters *c, unsigned site, bool ok)
{
    if (!ok) {
        atomicOr(&c->error, 4u);
        atomicCAS(&c->debug_site, 0u, site);
    }
    return ok;
}
#define TDQ_DBG(ctr, site, cond) (::tdq::dbg_check((ctr), (site), (cond)))
#else
#define TDQ_DBG(ctr, site, cond) (true)
#endif

// Sorted entry segments in device memory (structure of arrays).
struct EntrySoA {
    double *px, *py, *pz;  // position at t_start
    double *vx, *vy, *vz;  // velocity (end - start) / (t_end - t_start)
    int64_t *ts_key, *te_key;
    int64_t *seg_id, *traj_id, *orig;
    float4 *sph;           // FP32 bounding sphere: center (rounded to nearest) and radius w (rounded up);
                           // (0, 0, 0, 0) for huge magnitudes
    float *sph_e;          // E = |center|^2 (1 - 2^-20), rounded down; -inf for huge magnitudes (the
                           // pair is then never rejected)
    int64_t *te_sorted;    // t_end keys in ascending order (for exact overlap counts)
    uint4 *tc_rec;         // tensor-core pre-test records (tcgrid.cuh), groups of 8, padded with zero
                           // records to n_rec
};

// Sorted, clipped query segments in device memory.
struct QuerySoA {
    double *px, *py, *pz;  // position at the clipped start
    double *vx, *vy, *vz;
    double *d2;            // squared threshold
    int64_t *ts_key, *te_key;  // clipped span [max(ts,t0), min(te,t1)]
    int64_t *qid;          // caller's segment id
    int64_t *qtraj;        // caller's trajectory id (0 when not given)
    float4 *sph;           // FP32 bounding sphere of the clipped segment; w = radius + d, rounded up
    uint4 *tc_rec;         // tensor-core pre-test records in sorted order, groups of 8, zero records up
                           // to a whole supertile of 128
};

constexpr int kSearchEvents = 5;

// The counter block of a workspace: the counters, then two histograms of
// the query sort's small path (kSortFusedTiles tiles of 256 digit counts
// each), so that one memset clears them all.
constexpr uint64_t kCtrBytes = 256;
constexpr uint32_t kSortFusedTiles = 256;  // tiles of kSortTileKeys keys
constexpr uint32_t kSortTileKeys = 1024;
constexpr uint64_t kCtrBlockBytes = kCtrBytes + 2ull * kSortFusedTiles * 256 * sizeof(uint32_t);
static_assert(sizeof(DevCounters) <= kCtrBytes, "counters fit their slot");

// Per-query columns before sorting, in input order (64-bit words): px py pz
// vx vy vz d2 at the clipped start, the clipped span keys ts' te', the
// candidate range [lo, hi) of sorted entry positions, and the caller's
// segment and trajectory ids (integers stored bitwise).  The ids are copied
// here with coalesced loads, so that the gather into sorted order never reads
// the caller's arrays at random (they may be host memory read in place).
constexpr int kPreCols = 13;
constexpr int kPreLo = 9, kPreHi = 10, kPreSeg = 11, kPreTraj = 12;

struct Workspace {
    uint64_t q_cap = 0;    // queries the buffers below hold
    void *q_block = nullptr;
    // host-query staging (8 columns + seg id)
    double *in_cols[8] = {nullptr};
    int64_t *in_seg = nullptr;
    int64_t *in_traj = nullptr;
    // per-query arrays before sorting
    double *pre[kPreCols] = {nullptr};  // see kPreCols
    double **pre_dev = nullptr;         // device copy of pre[]
    float4 *pre_sph = nullptr;   // per-query sphere before sorting
    uint4 *pre_tc = nullptr;     // per-query tensor-core record before sorting (2 x uint4 each)
    uint64_t *keys = nullptr, *keys_alt = nullptr;
    uint32_t *vals = nullptr, *vals_alt = nullptr;
    // counting sort of the query segments by temporal bin: per-bin counts
    // (then offsets) and the candidate ranges in sorted order
    uint32_t *bin_cnt = nullptr;
    uint32_t bin_cap = 0;
    int64_t *srt_lo = nullptr, *srt_hi = nullptr;
    QuerySoA q{};
    // tiles
    uint64_t t_cap = 0;
    void *t_block = nullptr;
    int64_t *tile_lo = nullptr, *tile_hi = nullptr;
    unsigned long long *tile_work = nullptr;  // chunks per tile, then exclusive offsets (t_cap+1)
    // supertiles of 4 tiles (tensor-core pre-test): union range, chunks then
    // exclusive offsets (ceil(t_cap / 4) + 1)
    int64_t *st_lo = nullptr, *st_hi = nullptr;
    unsigned long long *st_work = nullptr;
    // sort scratch
    uint64_t s_cap = 0;
    uint32_t *sort_hist = nullptr;
    // counters (kCtrBytes, then the query sort's two fused histograms:
    // kCtrBlockBytes in all, cleared together at the start of a search) + host
    // mirror
    DevCounters *ctr = nullptr;
    uint32_t *sort_fused_hist = nullptr;  // inside the counter block
    DevCounters *ctr_host = nullptr;      // pinned, mapped into the device address space
    DevCounters *ctr_host_dev = nullptr;  // device view of ctr_host (the last pair kernel writes it)
    // results owned by tdq_search (device)
    uint64_t r_cap = 0;
    void *r_block = nullptr;
    tdq_result_buffer r{};
    // filter mode: survivors of the FP32 pre-test (entry, query) positions
    uint64_t s_cap_pairs = 0;
    void *s_block = nullptr;
    uint2 *surv = nullptr;
    // search start, pair kernel start, pair kernel end (filter mode: filter
    // kernel end), search end, refine kernel end
    cudaEvent_t ev[kSearchEvents] = {nullptr, nullptr, nullptr, nullptr, nullptr};
};

}  // namespace tdq

struct tdq_index {
    int device = 0;
    int sm_count = 0;
    uint64_t n = 0;
    uint32_t m = 0;
    double t_min = 0.0, t_max = 0.0, width = 0.0;
    double max_dur = 0.0;  // longest entry duration (t_end - t_start)
    void *e_block = nullptr;
    tdq::EntrySoA e{};
    void *b_block = nullptr;
    int64_t *bin_begin = nullptr;   // m + 1 sorted positions
    int64_t *bin_end_key = nullptr; // m, largest t_end key (INT64_MIN when empty)
    int64_t *bin_pmax_key = nullptr;// m, prefix max of bin_end_key
    int64_t *bin_lo_key = nullptr;  // m + 1: the smallest time key of each bin under bin_of (INT64_MIN, ..., INT64_MAX)
    int64_t tmin_key = 0;           // time key of t_min
    int64_t *te_bin_begin = nullptr;// m + 1: first position in e.te_sorted whose t_end lies in bin >= b
    tdq::TcGrid grid{};             // integer grid of the tensor-core pre-test (over the entries' centers)
    uint64_t n_rec = 0;             // tensor-core records held (n rounded up to 8, plus one pass of 128)
    tdq::Workspace ws;
    tdq_stats last{};
};

namespace tdq {

// Query input of one search: device columns and either one threshold and
// window or one per query segment.  n_real: number of real query segments
// when the launch covers more slots (captured searches have fixed launch
// shapes); slots at or beyond it are empty padding.  0: all slots are real.
struct QueryInput {
    const double *c[8];  // xs ys zs ts xe ye ze te
    const int64_t *seg_id;
    const int64_t *traj_id;  // may be null
    double d, t0, t1;
    const double *d_arr, *t0_arr, *t1_arr;
    uint64_t n_real;
};

struct LaunchCfg {
    uint32_t chunk;
    bool filter;     // a pre-test, then the FP64 refine of its survivors
    uint32_t flags;  // TDQ_FLAG_*
    bool tc;         // the pre-test runs on the tensor cores (TDQ_MODE_TC_FILTER)
};

// search.cu: workspace sizing, parameters, and one search split into a part
// that only enqueues device work (capturable in a CUDA graph) and a part that
// reads the counters once the stream has reached the end of it.
// Search workspace for nq query segments against an index of m bins.
tdq_status ensure_queries(Workspace &w, uint64_t nq, uint32_t m);
// Bins up to which query segments are ordered by a counting sort (per-bin
// counts, one scan) rather than the radix sort.
constexpr uint32_t kCountSortMaxBins = 1u << 17;
tdq_status ensure_survivors(Workspace &w, uint64_t cap);
tdq_status parse_params(const tdq_search_params *params, LaunchCfg *cfg);
int search_kernel_launches(const tdq_index *idx, const LaunchCfg &cfg, uint64_t nq);
cudaError_t enqueue_search(const tdq_index *idx, Workspace &w, const QueryInput &in, uint64_t nq, const LaunchCfg &cfg,
                           const tdq_result_buffer &out, cudaStream_t stream, bool events);
tdq_status finish_search(const tdq_index *idx, const Workspace &w, const LaunchCfg &cfg, uint64_t nq,
                         uint64_t capacity, bool events, tdq_stats *s, uint64_t *count, bool *surv_overflow);
// The kernel of a captured search that reads the caller's input (query
// preparation); re-pointed per batch without re-capturing.
struct GraphInputNodes {
    cudaGraphNode_t prep = nullptr;
};
cudaError_t find_input_nodes(cudaGraph_t g, GraphInputNodes *out);
cudaError_t bind_inputs(cudaGraphExec_t exec, const GraphInputNodes &nodes, const tdq_index *idx, Workspace &w,
                        const QueryInput &in, uint64_t nq, const LaunchCfg &cfg);

// Loading of the library's device code.  CUDA loads a translation unit's
// module (its kernels and file-scope device arrays) lazily, on first use,
// and a module load allocates device memory; tdq_build_index loads them all
// (load_device_code), so that no later search call does -- in particular
// not the allocation-free one.  One loader per translation unit with
// device code.
cudaError_t load_search_module();   // search.cu
cudaError_t load_filter_module();   // filter.cu
cudaError_t load_noalloc_module();  // noalloc.cu
cudaError_t load_sort_module();     // sort.cu
cudaError_t load_tc_module();       // tcfilter.cu
inline cudaError_t load_device_code()
{
    cudaError_t e;
    if ((e = load_search_module()) != cudaSuccess) return e;
    if ((e = load_filter_module()) != cudaSuccess) return e;
    if ((e = load_tc_module()) != cudaSuccess) return e;
    if ((e = load_sort_module()) != cudaSuccess) return e;
    return load_noalloc_module();
}

// Allocation gate (api.cu).  Every device and pinned-host allocation of the
// library goes through dev_alloc / host_alloc; tdq_debug_fail_allocations
// makes a chosen one fail, to test the error paths without touching a GPU.
cudaError_t alloc_gate();
template <typename T>
inline cudaError_t dev_alloc(T **p, size_t bytes)
{
    cudaError_t e = alloc_gate();
    if (e != cudaSuccess) {
        *p = nullptr;
        return e;
    }
    return cudaMalloc((void **)p, bytes);
}
template <typename T>
inline cudaError_t host_alloc(T **p, size_t bytes)
{
    cudaError_t e = alloc_gate();
    if (e != cudaSuccess) {
        *p = nullptr;
        return e;
    }
    return cudaMallocHost((void **)p, bytes);
}
// Pinned host memory that kernels write directly; *dev receives its device view.
template <typename T>
inline cudaError_t host_alloc_mapped(T **p, T **dev, size_t bytes)
{
    cudaError_t e = alloc_gate();
    if (e != cudaSuccess) {
        *p = *dev = nullptr;
        return e;
    }
    if ((e = cudaHostAlloc((void **)p, bytes, cudaHostAllocMapped)) != cudaSuccess) {
        *p = *dev = nullptr;
        return e;
    }
    return cudaHostGetDevicePointer((void **)dev, (void *)*p, 0);
}

// Page-locked host blocks for the result arrays handed to callers, recycled
// by size class (host_pool.cu): host_block_get returns a block of at least
// `bytes` bytes (null when page-locked memory cannot be had);
// host_block_put takes a block back (false: p is not one of its blocks).
void *host_block_get(uint64_t bytes);
bool host_block_put(void *p);

// Error reporting (api.cu).
tdq_status set_error(tdq_status st, const char *fmt, ...);
tdq_status cuda_error(cudaError_t e, const char *what);
#define TDQ_CUDA(call)                                          \
    do {                                                        \
        cudaError_t _e = (call);                                \
        if (_e != cudaSuccess) return ::tdq::cuda_error(_e, #call); \
    } while (0)

// Radix sort (sort.cu): stable ascending sort of (keys, vals) of length n.
// keys_alt/vals_alt are scratch of the same size; hist holds
// sort_hist_words(n) words.  The sorted data ends in keys/vals.
// Only the low key_bits bits are sorted on (an even number of 8-bit passes).
uint64_t sort_hist_words(uint64_t n);
// n_dev (may be null): device count of the leading keys to sort (at most n);
// the launch shapes follow n, the work the count.
// prep_hist (may be null; only with sort_fusable(n)): the producer of the
// keys has stored the first pass's digit counts per tile of kSortTileKeys
// keys (tile-major, prep_hist[tile * 256 + digit]) and zeroed the next
// ceil(n / kSortTileKeys) * 256 words, into which the first scatter then adds
// the second pass's counts: the sort runs no histogram kernel for its first
// two passes.
cudaError_t radix_sort_pairs(uint64_t *keys, uint32_t *vals, uint64_t *keys_alt, uint32_t *vals_alt, uint64_t n,
                             uint32_t *hist, cudaStream_t stream, int key_bits = 64,
                             const unsigned long long *n_dev = nullptr, uint32_t *prep_hist = nullptr);
inline int sort_passes(int key_bits) { return 2 * ((key_bits + 15) / 16); }
// The small path of the sort (tiles of kSortTileKeys keys, at most
// kSortFusedTiles of them), which can take prep_hist.
inline bool sort_fusable(uint64_t n)
{
    return n > 1 && (n + kSortTileKeys - 1) / kSortTileKeys <= kSortFusedTiles;
}
// Kernels radix_sort_pairs launches for n keys (with prep_hist: fused).
int sort_kernel_launches(uint64_t n, int key_bits, bool fused);
// Bits of a query sort key: bin indices 0..m-1 and m for invalid segments.
inline int bin_key_bits(uint32_t m)
{
    int b = 1;
    while (b < 32 && ((uint64_t)1 << b) <= (uint64_t)m) b++;
    return b;
}

}  // namespace tdq
