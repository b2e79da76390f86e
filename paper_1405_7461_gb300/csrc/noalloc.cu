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

#include "pipeline.cuh"

namespace tdq {
namespace {

constexpr uint64_t kNoAllocMaxQueries = 8192;
constexpr uint64_t kNoAllocTiles = kNoAllocMaxQueries / kQT;
constexpr uint64_t kNoAllocHistWords = (kNoAllocMaxQueries + 1023) / 1024 * 256 + 1;  // 1024-key sort tiles
constexpr uint64_t na_bytes(uint64_t count, uint64_t size) { return (count * size + 255) & ~(uint64_t)255; }
constexpr uint64_t kNoAllocScratchBytes =
    kPreCols * na_bytes(kNoAllocMaxQueries, 8)                               // pre columns
    + 2 * na_bytes(kNoAllocMaxQueries, 8) + 2 * na_bytes(kNoAllocMaxQueries, 4)  // sort keys / values
    + 10 * na_bytes(kNoAllocMaxQueries, 8)                                   // sorted query SoA
    + 2 * na_bytes(kNoAllocMaxQueries, 16)                                   // query spheres
    + 2 * na_bytes(kNoAllocTiles, 8) + na_bytes(kNoAllocTiles + 1, 8)        // tile table
    + na_bytes(kNoAllocHistWords, 4)                                         // sort histogram
    + na_bytes(1, sizeof(DevCounters))                                       // counters
    + na_bytes(kPreCols, sizeof(double *));                                  // pre pointer table

// The scratch.  In host code this name is only a host-side stand-in for the
// symbol; its device address comes from cudaGetSymbolAddress below.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

struct NoAllocScratch {
    double *pre[kPreCols];
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
        for (int c = 0; c < kPreCols; c++) s.pre[c] = carve<double>(p, kNoAllocMaxQueries);
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
        q.qid = carve<int64_t>(p, kNoAllocMaxQueries);
        q.qtraj = nullptr;  // no pair filters here
        s.pre_sph = carve<float4>(p, kNoAllocMaxQueries);
        q.sph = carve<float4>(p, kNoAllocMaxQueries);
        s.tile_lo = carve<int64_t>(p, kNoAllocTiles);
        s.tile_hi = carve<int64_t>(p, kNoAllocTiles);
        s.tile_work = carve<unsigned long long>(p, kNoAllocTiles + 1);
        s.hist = carve<uint32_t>(p, kNoAllocHistWords);
        s.ctr = carve<DevCounters>(p, 1);
        s.pre_dev = carve<double *>(p, kPreCols);
        if ((uint64_t)(p - (char *)base) > kNoAllocScratchBytes || sort_hist_words(kNoAllocMaxQueries) > kNoAllocHistWords)
            return set_error(TDQ_ERR_CUDA, "tdq_search_device_noalloc: scratch layout exceeds the array");
        e = cudaMemcpy(s.pre_dev, s.pre, kPreCols * sizeof(double *), cudaMemcpyHostToDevice);
        if (e != cudaSuccess) return cuda_error(e, "tdq_search_device_noalloc: pointer table");
        g_noalloc[dev] = s;
        g_noalloc_ready[dev] = true;
    }
    *out = &g_noalloc[dev];
    return TDQ_OK;
}

}  // namespace

cudaError_t load_noalloc_module()
{
    void *p = nullptr;
    return cudaGetSymbolAddress(&p, g_noalloc_scratch);
}

}  // namespace tdq

using namespace tdq;

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
    if (params && params->mode != TDQ_MODE_FP64)
        return set_error(TDQ_ERR_INVALID,
                         "tdq_search_device_noalloc: the filter modes need a survivor list; use TDQ_MODE_FP64");
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
    query_prep<<<prep_grid(nq), kBlock, 0, stream>>>(
        PrepArgs{in, nq, bins, s->pre_dev, s->pre_sph, s->keys, s->vals, s->ctr, nullptr, idx->n > 0, false, nullptr,
                 TcGrid{}, nullptr, idx->n});
    const uint64_t ntiles = (nq + kQT - 1) / kQT;
    if (idx->n > 0) {
        TDQ_CUDA(radix_sort_pairs(s->keys, s->vals, s->keys_alt, s->vals_alt, nq, s->hist, stream,
                                  bin_key_bits(idx->m)));
        const GatherArgs ga{s->pre_dev, s->pre_sph, s->vals, nq, s->ctr, s->q, ntiles, chunk, s->tile_lo,
                            s->tile_hi, s->tile_work};
        query_gather<<<grid_for(nq), kBlock, 0, stream>>>(ga);
        PairArgs pa{idx->e, s->q, s->tile_lo, s->tile_hi, s->tile_work, ntiles, s->ctr, *out, chunk, 0u, nullptr,
                    idx->n, nq};
        TDQ_CUDA(launch_pair_kernel(pa, false, idx->sm_count, nullptr, 0, stream, nullptr, 0));
    }
    TDQ_CUDA(cudaGetLastError());
    DevCounters h{};
    TDQ_CUDA(cudaMemcpyAsync(&h, s->ctr, sizeof(DevCounters), cudaMemcpyDeviceToHost, stream));
    TDQ_CUDA(cudaStreamSynchronize(stream));
    if (h.error & 4u)
        return set_error(TDQ_ERR_CUDA, "tdq_search_device_noalloc: debug build: index bounds check at site %u failed",
                         h.debug_site);
    if (h.error & 1u)
        return set_error(TDQ_ERR_INVALID,
                         "tdq_search_device_noalloc: invalid query segment (non-finite value, t_end <= t_start, "
                         "d < 0 or NaN, NaN window or t0 > t1)");
    *count = h.results;
    return h.results > out->capacity ? TDQ_ERR_OVERFLOW : TDQ_OK;
}
