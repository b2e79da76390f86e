// Batched searches under a CUDA graph, and the autotuner.
//
// A plan owns a search workspace, staging buffers for one batch of query
// segments (each with its own threshold and window), and a result buffer.
// tdq_plan_search stages the batch, then replays the whole search -- counter
// reset, query preparation and sort, candidate ranges, tiles, pair kernels,
// overlap count, counter read-back -- as one CUDA graph launch.  Graphs are
// captured once per size class of the batch -- powers of two up to the
// plan's largest batch, and that size itself (the slots past the batch's real
// size are empty padding) -- so batches of uneven size reuse a few graphs and
// full batches run no padding.  Per batch, the kernel that reads the input (query
// preparation) is re-pointed at it (device and page-locked host inputs in
// place, other host inputs through staging buffers) and told the batch's real
// size, without re-capturing.  The paper processes a query
// in batches of s query segments, one kernel invocation and host round trip
// per batch (Sec. 6.1); here a batch is one graph launch and the batch size
// is chosen by measurement (tdq_autotune).
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <new>

#include "tdq_internal.cuh"

namespace {

constexpr int kMaxGraphs = 24;
constexpr uint64_t kMinClass = 1024;

uint64_t size_class(uint64_t n)
{
    uint64_t c = kMinClass;
    while (c < n) c <<= 1;
    return c;
}

}  // namespace

struct tdq_plan {
    tdq_index *idx = nullptr;
    uint64_t max_q = 0;      // largest batch
    uint64_t cap_q = 0;      // size class of the largest batch (buffer capacity)
    tdq::LaunchCfg cfg{};
    bool use_graph = true;
    tdq::Workspace ws;
    void *stage_block = nullptr;
    double *d_arr = nullptr, *t0_arr = nullptr, *t1_arr = nullptr;
    void *r_block = nullptr;     // device result buffer, or page-locked host memory (host_results)
    bool host_results = false;
    tdq_result_buffer res{};       // the kernels' view (device pointers)
    tdq_result_buffer res_host{};  // host pointers of the same arrays (host_results)
    cudaStream_t cap_stream = nullptr;
    struct Graph {
        uint64_t cls;
        cudaGraph_t graph;
        cudaGraphExec_t exec;
        tdq::GraphInputNodes nodes;
        tdq::QueryInput bound;  // inputs the exec's nodes hold (valid when has_bound)
        bool has_bound;
    } graphs[kMaxGraphs];
    int ngraphs = 0;
    uint64_t last_count = 0;
    tdq_stats last{};
};

namespace {

using namespace tdq;

void drop_graphs(tdq_plan *p)
{
    for (int k = 0; k < p->ngraphs; k++) {
        cudaGraphExecDestroy(p->graphs[k].exec);
        cudaGraphDestroy(p->graphs[k].graph);
    }
    p->ngraphs = 0;
}

// The four result arrays of capacity cap in one block, each b bytes.
tdq_result_buffer result_columns(char *c, uint64_t b, uint64_t cap)
{
    tdq_result_buffer r{};
    r.query_seg_id = (int64_t *)c;
    r.entry_seg_id = (int64_t *)(c + b);
    r.t_enter = (double *)(c + 2 * b);
    r.t_exit = (double *)(c + 3 * b);
    r.capacity = cap;
    return r;
}

void free_results(tdq_plan *p)
{
    if (p->r_block) {
        if (p->host_results)
            cudaFreeHost(p->r_block);
        else
            cudaFree(p->r_block);
    }
    p->r_block = nullptr;
    p->res = tdq_result_buffer{};
    p->res_host = tdq_result_buffer{};
}

tdq_status plan_results(tdq_plan *p, uint64_t cap)
{
    if (cap <= p->res.capacity && p->r_block) return TDQ_OK;
    drop_graphs(p);  // captured graphs hold the old pointers
    free_results(p);
    const uint64_t b = (cap * 8 + 255) & ~(uint64_t)255;
    char *dev = nullptr;
    if (p->host_results) {
        void *d = nullptr;
        if (cudaHostAlloc(&p->r_block, 4 * b, cudaHostAllocMapped) != cudaSuccess ||
            cudaHostGetDevicePointer(&d, p->r_block, 0) != cudaSuccess) {
            cudaGetLastError();
            free_results(p);
            return set_error(TDQ_ERR_NOMEM, "tdq_plan: host result buffer of %llu items", (unsigned long long)cap);
        }
        p->res_host = result_columns((char *)p->r_block, b, cap);
        dev = (char *)d;
    } else {
        if (dev_alloc(&p->r_block, 4 * b) != cudaSuccess) {
            cudaGetLastError();
            return set_error(TDQ_ERR_NOMEM, "tdq_plan: result buffer of %llu items", (unsigned long long)cap);
        }
        dev = (char *)p->r_block;
    }
    p->res = result_columns(dev, b, cap);
    return TDQ_OK;
}

tdq_status plan_survivors(tdq_plan *p, uint64_t cap)
{
    if (cap <= p->ws.s_cap_pairs && p->ws.s_block) return TDQ_OK;
    drop_graphs(p);
    return ensure_survivors(p->ws, cap);
}

tdq_plan::Graph *find_graph(tdq_plan *p, uint64_t cls)
{
    for (int k = 0; k < p->ngraphs; k++)
        if (p->graphs[k].cls == cls) return &p->graphs[k];
    return nullptr;
}

QueryInput staged_input(const tdq_plan *p)
{
    QueryInput in{};
    for (int c = 0; c < 8; c++) in.c[c] = p->ws.in_cols[c];
    in.seg_id = p->ws.in_seg;
    in.d_arr = p->d_arr;
    in.t0_arr = p->t0_arr;
    in.t1_arr = p->t1_arr;
    return in;
}

tdq_status capture(tdq_plan *p, uint64_t cls, tdq_plan::Graph **out)
{
    if (p->ngraphs == kMaxGraphs) drop_graphs(p);
    const QueryInput in = staged_input(p);
    TDQ_CUDA(cudaStreamBeginCapture(p->cap_stream, cudaStreamCaptureModeThreadLocal));
    // the events become event-record nodes: the pair kernels stay timed
    cudaError_t e = enqueue_search(p->idx, p->ws, in, cls, p->cfg, p->res, p->cap_stream, true);
    cudaGraph_t g = nullptr;
    cudaError_t e2 = cudaStreamEndCapture(p->cap_stream, &g);
    if (e != cudaSuccess || e2 != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return cuda_error(e != cudaSuccess ? e : e2, "tdq_plan: graph capture");
    }
    tdq_plan::Graph G{cls, g, nullptr, GraphInputNodes{}};
    e = find_input_nodes(g, &G.nodes);
    if (e == cudaSuccess) e = cudaGraphInstantiate(&G.exec, g, 0);
    if (e != cudaSuccess) {
        cudaGraphDestroy(g);
        return cuda_error(e, "tdq_plan: graph instantiation");
    }
    p->graphs[p->ngraphs] = G;
    *out = &p->graphs[p->ngraphs];
    p->ngraphs++;
    return TDQ_OK;
}

void plan_release(tdq_plan *p)
{
    drop_graphs(p);
    Workspace &w = p->ws;
    cudaFree(w.q_block);
    cudaFree(w.t_block);
    cudaFree(w.sort_hist);
    cudaFree(w.s_block);
    cudaFree(w.bin_cnt);
    cudaFree(w.ctr);
    if (w.ctr_host) cudaFreeHost(w.ctr_host);
    for (int k = 0; k < kSearchEvents; k++)
        if (w.ev[k]) cudaEventDestroy(w.ev[k]);
    cudaFree(p->stage_block);
    free_results(p);
    if (p->cap_stream) cudaStreamDestroy(p->cap_stream);
}

}  // namespace

extern "C" tdq_status tdq_plan_create(tdq_index *idx, const tdq_plan_params *params, tdq_plan **out)
{
    if (!out) return set_error(TDQ_ERR_INVALID, "tdq_plan_create: out is NULL");
    *out = nullptr;
    if (!idx || !params) return set_error(TDQ_ERR_INVALID, "tdq_plan_create: NULL argument");
    if (params->max_query_segments == 0 || params->max_query_segments > 0x7fffffffULL)
        return set_error(TDQ_ERR_INVALID, "tdq_plan_create: max_query_segments must be in [1, 2^31)");
    tdq_search_params sp{};
    sp.entry_chunk = params->entry_chunk;
    sp.mode = params->mode;
    LaunchCfg cfg;
    tdq_status st = parse_params(&sp, &cfg);
    if (st != TDQ_OK) return st;
    tdq_plan *p = new (std::nothrow) tdq_plan();
    if (!p) return set_error(TDQ_ERR_NOMEM, "tdq_plan_create: host allocation failed");
    p->idx = idx;
    p->max_q = params->max_query_segments;
    p->cap_q = size_class(p->max_q);
    p->cfg = cfg;
    p->use_graph = !params->no_graph;
    p->host_results = params->host_results != 0;
    do {
        Workspace &w = p->ws;
        bool ok = dev_alloc(&w.ctr, kCtrBlockBytes) == cudaSuccess &&
                  host_alloc_mapped(&w.ctr_host, &w.ctr_host_dev, sizeof(DevCounters)) == cudaSuccess &&
                  dev_alloc(&p->stage_block, 3 * p->cap_q * 8) == cudaSuccess;
        if (!ok) {
            cudaGetLastError();
            st = set_error(TDQ_ERR_NOMEM, "tdq_plan_create: allocation failed");
            break;
        }
        w.sort_fused_hist = (uint32_t *)((char *)w.ctr + kCtrBytes);
        for (int k = 0; k < kSearchEvents && st == TDQ_OK; k++)
            if (cudaEventCreate(&w.ev[k]) != cudaSuccess) st = set_error(TDQ_ERR_CUDA, "tdq_plan_create: events");
        if (st != TDQ_OK) break;
        if (cudaStreamCreateWithFlags(&p->cap_stream, cudaStreamNonBlocking) != cudaSuccess) {
            st = set_error(TDQ_ERR_CUDA, "tdq_plan_create: stream");
            break;
        }
        p->d_arr = (double *)p->stage_block;
        p->t0_arr = p->d_arr + p->cap_q;
        p->t1_arr = p->t0_arr + p->cap_q;
        st = ensure_queries(w, p->cap_q, p->idx->m);
        if (st != TDQ_OK) break;
        const uint64_t rc = params->result_capacity ? params->result_capacity : (idx->n > 65536 ? idx->n : 65536);
        st = plan_results(p, rc);
        if (st != TDQ_OK) break;
        if (cfg.filter && idx->n > 0) {
            st = plan_survivors(p, p->cap_q * 64 > (1u << 20) ? p->cap_q * 64 : (1u << 20));
            if (st != TDQ_OK) break;
        }
    } while (0);
    if (st != TDQ_OK) {
        plan_release(p);
        delete p;
        return st;
    }
    *out = p;
    return TDQ_OK;
}

extern "C" void tdq_plan_free(tdq_plan *p)
{
    if (!p) return;
    plan_release(p);
    delete p;
}

extern "C" tdq_status tdq_plan_search(tdq_plan *p, const tdq_segments *queries, const double *d_per_query,
                                      const double *t0_per_query, const double *t1_per_query, void *stream_,
                                      uint64_t *count)
{
    if (!p || !queries || !count || !d_per_query || !t0_per_query || !t1_per_query)
        return set_error(TDQ_ERR_INVALID, "tdq_plan_search: NULL argument");
    *count = 0;
    p->last = tdq_stats{};
    p->last_count = 0;
    const uint64_t nq = queries->n;
    if (nq > p->max_q)
        return set_error(TDQ_ERR_INVALID, "tdq_plan_search: %llu query segments exceed the plan's %llu",
                         (unsigned long long)nq, (unsigned long long)p->max_q);
    if (nq == 0) return TDQ_OK;
    const double *cols[8] = {queries->xs, queries->ys, queries->zs, queries->ts,
                             queries->xe, queries->ye, queries->ze, queries->te};
    for (int c = 0; c < 8; c++)
        if (!cols[c]) return set_error(TDQ_ERR_INVALID, "tdq_plan_search: query column %d is NULL", c);
    if (!queries->seg_id) return set_error(TDQ_ERR_INVALID, "tdq_plan_search: query seg_id is NULL");
    cudaStream_t stream = (cudaStream_t)stream_;
    Workspace &w = p->ws;
    // the batch's input: the caller's device arrays in place, or host arrays
    // staged into the plan's buffers
    QueryInput in{};
    if (queries->on_device) {
        for (int c = 0; c < 8; c++) in.c[c] = cols[c];
        in.seg_id = queries->seg_id;
        in.d_arr = d_per_query;
        in.t0_arr = t0_per_query;
        in.t1_arr = t1_per_query;
    } else {
        // page-locked, mapped host arrays are read in place; anything else
        // is staged into the plan's buffers
        const void *host[12] = {cols[0], cols[1], cols[2], cols[3], cols[4], cols[5], cols[6], cols[7],
                                queries->seg_id, d_per_query, t0_per_query, t1_per_query};
        const void *view[12];
        bool mapped = true;
        for (int k = 0; k < 12 && mapped; k++) mapped = (view[k] = mapped_view(host[k], nq * 8)) != nullptr;
        if (mapped) {
            for (int c = 0; c < 8; c++) in.c[c] = (const double *)view[c];
            in.seg_id = (const int64_t *)view[8];
            in.d_arr = (const double *)view[9];
            in.t0_arr = (const double *)view[10];
            in.t1_arr = (const double *)view[11];
        } else {
            for (int c = 0; c < 8; c++)
                TDQ_CUDA(cudaMemcpyAsync(w.in_cols[c], cols[c], nq * 8, cudaMemcpyHostToDevice, stream));
            TDQ_CUDA(cudaMemcpyAsync(w.in_seg, queries->seg_id, nq * 8, cudaMemcpyHostToDevice, stream));
            TDQ_CUDA(cudaMemcpyAsync(p->d_arr, d_per_query, nq * 8, cudaMemcpyHostToDevice, stream));
            TDQ_CUDA(cudaMemcpyAsync(p->t0_arr, t0_per_query, nq * 8, cudaMemcpyHostToDevice, stream));
            TDQ_CUDA(cudaMemcpyAsync(p->t1_arr, t1_per_query, nq * 8, cudaMemcpyHostToDevice, stream));
            in = staged_input(p);
        }
    }
    // the batch's size class: a power of two (from kMinClass) up to the plan's
    // largest batch, which is a class of its own (a plan sized for exactly
    // its batches runs no padding slots)
    const uint64_t cls = size_class(nq) < p->max_q ? size_class(nq) : p->max_q;
    in.n_real = nq;
    for (int attempt = 0;; attempt++) {
        if (p->use_graph) {
            tdq_plan::Graph *G = find_graph(p, cls);
            if (!G) {
                tdq_status st = capture(p, cls, &G);
                if (st != TDQ_OK) return st;
            }
            // re-bind only when the inputs differ from the ones the graph holds
            static_assert(sizeof(QueryInput) % 8 == 0, "QueryInput compared bytewise");
            if (!G->has_bound || memcmp(&G->bound, &in, sizeof in) != 0) {
                TDQ_CUDA(bind_inputs(G->exec, G->nodes, p->idx, w, in, cls, p->cfg));
                G->bound = in;
                G->has_bound = true;
            }
            TDQ_CUDA(cudaGraphLaunch(G->exec, stream));
        } else {
            QueryInput direct = in;
            direct.n_real = 0;
            TDQ_CUDA(enqueue_search(p->idx, w, direct, nq, p->cfg, p->res, stream, true));
        }
        TDQ_CUDA(cudaStreamSynchronize(stream));
        bool grow_surv = false;
        uint64_t cnt = 0;
        tdq_status st = finish_search(p->idx, w, p->cfg, p->use_graph ? cls : nq, p->res.capacity, true, &p->last, &cnt,
                                      &grow_surv);
        cudaGetLastError();
        if (st == TDQ_OK && !grow_surv) {
            *count = cnt;
            p->last_count = cnt;
            return TDQ_OK;
        }
        if (attempt >= 3) return st != TDQ_OK ? st : set_error(TDQ_ERR_NOMEM, "tdq_plan_search: kept overflowing");
        if (grow_surv) {
            const uint64_t need = w.ctr_host->survivors;
            st = plan_survivors(p, need + need / 4 + 1024);
        } else if (st == TDQ_ERR_OVERFLOW) {  // the statically sized result buffer was too small (Sec. 5)
            st = plan_results(p, cnt + cnt / 8 + 1024);
        }
        if (st != TDQ_OK) return st;
    }
}

extern "C" tdq_status tdq_plan_results(const tdq_plan *p, tdq_result_buffer *view, uint64_t *count)
{
    if (!p || !view || !count) return set_error(TDQ_ERR_INVALID, "tdq_plan_results: NULL argument");
    *view = p->host_results ? p->res_host : p->res;
    *count = p->last_count;
    return TDQ_OK;
}

namespace {

// The four result columns into caller arrays the device can write (device
// memory, or page-locked host memory over the coherent CPU-GPU link): one
// launch instead of four copies.
__global__ void copy_result_columns(tdq_result_buffer src, uint64_t n, int64_t *qid, int64_t *eid, double *tin,
                                    double *tout)
{
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        qid[i] = src.query_seg_id[i];
        eid[i] = src.entry_seg_id[i];
        tin[i] = src.t_enter[i];
        tout[i] = src.t_exit[i];
    }
}

}  // namespace

extern "C" tdq_status tdq_plan_copy_results(const tdq_plan *p, int64_t *query_seg_id, int64_t *entry_seg_id,
                                            double *t_enter, double *t_exit, uint64_t n, int to_device,
                                            void *stream_)
{
    if (!p) return set_error(TDQ_ERR_INVALID, "tdq_plan_copy_results: NULL plan");
    if (n > p->last_count || n > p->res.capacity)
        return set_error(TDQ_ERR_INVALID, "tdq_plan_copy_results: %llu items requested, %llu available",
                         (unsigned long long)n, (unsigned long long)p->last_count);
    if (n == 0) return TDQ_OK;
    if (!query_seg_id || !entry_seg_id || !t_enter || !t_exit)
        return set_error(TDQ_ERR_INVALID, "tdq_plan_copy_results: NULL array");
    cudaStream_t stream = (cudaStream_t)stream_;
    if (!to_device) {
        void *v[4] = {(void *)mapped_view(query_seg_id, n * 8), (void *)mapped_view(entry_seg_id, n * 8),
                      (void *)mapped_view(t_enter, n * 8), (void *)mapped_view(t_exit, n * 8)};
        if (v[0] && v[1] && v[2] && v[3]) {  // all page-locked and mapped: written by one kernel
            const uint64_t blocks = (n + kBlock - 1) / kBlock, most = 4ull * (uint64_t)p->idx->sm_count;
            copy_result_columns<<<(unsigned)(blocks < most ? blocks : most), kBlock, 0, stream>>>(
                p->res, n, (int64_t *)v[0], (int64_t *)v[1], (double *)v[2], (double *)v[3]);
            TDQ_CUDA(cudaGetLastError());
            TDQ_CUDA(cudaStreamSynchronize(stream));
            return TDQ_OK;
        }
    }
    // (the plan's buffer may be page-locked host memory: the runtime tells the
    // directions apart by address)
    const cudaMemcpyKind kind = cudaMemcpyDefault;
    TDQ_CUDA(cudaMemcpyAsync(query_seg_id, p->res.query_seg_id, n * 8, kind, stream));
    TDQ_CUDA(cudaMemcpyAsync(entry_seg_id, p->res.entry_seg_id, n * 8, kind, stream));
    TDQ_CUDA(cudaMemcpyAsync(t_enter, p->res.t_enter, n * 8, kind, stream));
    TDQ_CUDA(cudaMemcpyAsync(t_exit, p->res.t_exit, n * 8, kind, stream));
    TDQ_CUDA(cudaStreamSynchronize(stream));
    return TDQ_OK;
}

extern "C" tdq_status tdq_plan_get_stats(const tdq_plan *p, tdq_stats *out)
{
    if (!p || !out) return set_error(TDQ_ERR_INVALID, "tdq_plan_get_stats: NULL argument");
    *out = p->last;
    return TDQ_OK;
}

// ---------------------------------------------------------------------------
// Autotuner
// ---------------------------------------------------------------------------

namespace {

struct DeviceSample {
    tdq_segments q{};
    const double *d = nullptr, *t0 = nullptr, *t1 = nullptr;
    void *block = nullptr;
};

// The sample in device memory (copied if it is on the host), so that the
// timings see device-resident inputs.
tdq_status device_sample(const tdq_segments *q, const double *d, const double *t0, const double *t1,
                         DeviceSample *s)
{
    s->q = *q;
    s->d = d;
    s->t0 = t0;
    s->t1 = t1;
    if (q->on_device) return TDQ_OK;
    const uint64_t n = q->n;
    if (dev_alloc(&s->block, n * 8 * 12) != cudaSuccess) {
        cudaGetLastError();
        return set_error(TDQ_ERR_NOMEM, "tdq_autotune: sample staging");
    }
    double *b = (double *)s->block;
    const double *src[8] = {q->xs, q->ys, q->zs, q->ts, q->xe, q->ye, q->ze, q->te};
    double *dst[8];
    for (int c = 0; c < 8; c++) {
        dst[c] = b + c * n;
        TDQ_CUDA(cudaMemcpy(dst[c], src[c], n * 8, cudaMemcpyHostToDevice));
    }
    int64_t *sid = (int64_t *)(b + 8 * n);
    TDQ_CUDA(cudaMemcpy(sid, q->seg_id, n * 8, cudaMemcpyHostToDevice));
    double *dd = b + 9 * n, *tt0 = b + 10 * n, *tt1 = b + 11 * n;
    TDQ_CUDA(cudaMemcpy(dd, d, n * 8, cudaMemcpyHostToDevice));
    TDQ_CUDA(cudaMemcpy(tt0, t0, n * 8, cudaMemcpyHostToDevice));
    TDQ_CUDA(cudaMemcpy(tt1, t1, n * 8, cudaMemcpyHostToDevice));
    s->q.xs = dst[0]; s->q.ys = dst[1]; s->q.zs = dst[2]; s->q.ts = dst[3];
    s->q.xe = dst[4]; s->q.ye = dst[5]; s->q.ze = dst[6]; s->q.te = dst[7];
    s->q.seg_id = sid;
    s->q.traj_id = nullptr;
    s->q.on_device = 1;
    s->d = dd;
    s->t0 = tt0;
    s->t1 = tt1;
    return TDQ_OK;
}

tdq_segments slice(const tdq_segments &q, uint64_t off, uint64_t n)
{
    tdq_segments s = q;
    s.xs += off; s.ys += off; s.zs += off; s.ts += off;
    s.xe += off; s.ye += off; s.ze += off; s.te += off;
    s.seg_id += off;
    if (s.traj_id) s.traj_id += off;
    s.n = n;
    return s;
}

// Time (ms) of searching the whole sample in batches of `batch` query
// segments with a plan: median over `reps` after one warm-up pass.
tdq_status time_batches(tdq_index *idx, const DeviceSample &s, uint64_t batch, uint32_t chunk, int mode, int reps,
                        cudaStream_t stream, double *ms_out, uint64_t *results_out)
{
    tdq_plan_params pp{};
    pp.max_query_segments = batch;
    pp.entry_chunk = chunk;
    pp.mode = mode;
    tdq_plan *p = nullptr;
    tdq_status st = tdq_plan_create(idx, &pp, &p);
    if (st != TDQ_OK) return st;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    double times[16];
    if (reps > 16) reps = 16;
    uint64_t results = 0;
    for (int r = -1; r < reps && st == TDQ_OK; r++) {
        cudaEventRecord(e0, stream);
        uint64_t tot = 0;
        for (uint64_t off = 0; off < s.q.n && st == TDQ_OK; off += batch) {
            const uint64_t n = s.q.n - off < batch ? s.q.n - off : batch;
            tdq_segments q = slice(s.q, off, n);
            uint64_t cnt = 0;
            st = tdq_plan_search(p, &q, s.d + off, s.t0 + off, s.t1 + off, stream, &cnt);
            tot += cnt;
        }
        cudaEventRecord(e1, stream);
        cudaEventSynchronize(e1);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (r >= 0) times[r] = ms;
        results = tot;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    tdq_plan_free(p);
    if (st != TDQ_OK) return st;
    // median
    for (int i = 1; i < reps; i++)
        for (int j = i; j > 0 && times[j] < times[j - 1]; j--) {
            double t = times[j];
            times[j] = times[j - 1];
            times[j - 1] = t;
        }
    *ms_out = times[reps / 2];
    *results_out = results;
    return TDQ_OK;
}

}  // namespace

extern "C" tdq_status tdq_autotune(const tdq_segments *entries, const tdq_segments *sample, const double *d,
                                   const double *t0, const double *t1, const tdq_autotune_params *ap, void *stream_,
                                   tdq_tuning *out)
{
    if (!entries || !sample || !d || !t0 || !t1 || !out)
        return set_error(TDQ_ERR_INVALID, "tdq_autotune: NULL argument");
    if (sample->n == 0) return set_error(TDQ_ERR_INVALID, "tdq_autotune: empty sample");
    cudaStream_t stream = (cudaStream_t)stream_;
    static const uint32_t kBins[] = {1000, 10000, 100000};
    static const uint32_t kChunks[] = {256, 512, 1024};
    const int mode = ap ? ap->mode : TDQ_MODE_FP64;
    const uint32_t *bins = (ap && ap->bin_counts) ? ap->bin_counts : kBins;
    const int nb = (ap && ap->bin_counts) ? ap->n_bin_counts : 3;
    const uint32_t *chunks = (ap && ap->entry_chunks) ? ap->entry_chunks : kChunks;
    const int nc = (ap && ap->entry_chunks) ? ap->n_entry_chunks : 3;
    const int reps = (ap && ap->repeats > 0) ? ap->repeats : 3;
    const double tol = (ap && ap->batch_tolerance > 0) ? ap->batch_tolerance : 0.05;
    if (nb <= 0 || nc <= 0) return set_error(TDQ_ERR_INVALID, "tdq_autotune: empty candidate list");

    DeviceSample s;
    tdq_status st = device_sample(sample, d, t0, t1, &s);
    if (st != TDQ_OK) return st;
    const uint64_t n = s.q.n;
    double best_ms = INFINITY;
    uint32_t best_bins = bins[0], best_chunk = chunks[0];
    uint64_t results = 0;
    // 1. bin count x entry chunk, one batch holding the whole sample
    for (int i = 0; i < nb && st == TDQ_OK; i++) {
        tdq_index_params ip{bins[i]};
        tdq_index *idx = nullptr;
        st = tdq_build_index(entries, &ip, stream, &idx);
        for (int j = 0; j < nc && st == TDQ_OK; j++) {
            double ms = 0;
            uint64_t r = 0;
            st = time_batches(idx, s, n, chunks[j], mode, reps, stream, &ms, &r);
            if (st == TDQ_OK && ms < best_ms) {
                best_ms = ms;
                best_bins = bins[i];
                best_chunk = chunks[j];
                results = r;
            }
        }
        tdq_index_free(idx);
    }
    // 2. batch size: the smallest whose throughput is within tol of the best
    uint64_t best_batch = n;
    double batch_ms = best_ms;
    if (st == TDQ_OK) {
        static const uint64_t kBatches[] = {1024, 4096, 16384, 65536, 262144};
        const uint64_t *bs = (ap && ap->batch_sizes) ? ap->batch_sizes : kBatches;
        const int nbs = (ap && ap->batch_sizes) ? ap->n_batch_sizes : 5;
        tdq_index_params ip{best_bins};
        tdq_index *idx = nullptr;
        st = tdq_build_index(entries, &ip, stream, &idx);
        double tms[32];
        uint64_t cand[32];
        int nt = 0;
        for (int k = 0; k < nbs && k < 31 && st == TDQ_OK; k++) {
            if (bs[k] == 0 || bs[k] >= n) continue;
            double ms = 0;
            uint64_t r = 0;
            st = time_batches(idx, s, bs[k], best_chunk, mode, reps, stream, &ms, &r);
            cand[nt] = bs[k];
            tms[nt++] = ms;
        }
        cand[nt] = n;
        tms[nt++] = best_ms;
        double fastest = INFINITY;
        for (int k = 0; k < nt; k++) fastest = fmin(fastest, tms[k]);
        for (int k = 0; k < nt; k++)
            if (tms[k] <= fastest * (1.0 + tol) && cand[k] <= best_batch) {
                best_batch = cand[k];
                batch_ms = tms[k];
            }
        tdq_index_free(idx);
    }
    cudaFree(s.block);
    if (st != TDQ_OK) return st;
    out->bin_count = best_bins;
    out->entry_chunk = best_chunk;
    out->batch_query_segments = best_batch;
    out->results_per_query_segment = (double)results / (double)n;
    const double est = ceil(out->results_per_query_segment * (double)best_batch);
    out->result_capacity = (uint64_t)(2.0 * est) + 1024;
    out->ms_per_query_segment = batch_ms / (double)n;
    return TDQ_OK;
}
