// Serving loop: continuous batching of distance threshold queries over a
// resident database.
//
// The paper frames the search as online: one database in GPU memory, many
// queries, response time as the objective, and query batches because result
// memory must be reserved up front (Sec. 3).  The server keeps the index
// resident and runs `lanes` worker threads, each with its own CUDA stream and
// batched plan (tdq_plan: one CUDA graph launch per batch).  Requests wait in
// one FIFO queue; a free lane admits requests from its head while
//   - the batch stays within max_batch_query_segments, and
//   - the estimated result-buffer bytes of all admitted, unfinished requests
//     stay within memory_cap_bytes (a lane always admits at least one request
//     when nothing else is in flight, so a large request cannot starve),
// packs them into one batch -- each query segment keeps its request's d and
// window -- and searches it.  While one lane's batch is on the GPU, requests
// that arrive meanwhile are admitted by the other lanes, so batches overlap
// on the device.  Results are split back per request by the position of each
// query segment in the batch.
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <mutex>
#include <new>
#include <thread>
#include <unordered_map>
#include <vector>

#include "tdq_internal.cuh"

namespace {

using Clock = std::chrono::steady_clock;

double ms_between(Clock::time_point a, Clock::time_point b)
{
    return std::chrono::duration<double, std::milli>(b - a).count();
}

struct Request {
    uint64_t ticket = 0;
    uint64_t n = 0;
    std::vector<double> cols[8];
    std::vector<int64_t> seg_id;
    double d = 0, t0 = 0, t1 = 0;
    double est_bytes = 0;
    int state = 0;  // 0 queued, 1 running, 2 done
    tdq_status status = TDQ_OK;
    uint64_t batch = 0, batch_segments = 0;
    Clock::time_point t_submit, t_start, t_done;
    std::vector<int64_t> r_q, r_e;
    std::vector<double> r_tin, r_tout;
};

struct Lane {
    tdq_plan *plan = nullptr;
    cudaStream_t stream = nullptr;
    uint64_t cap = 0;
    double *h_cols[8] = {nullptr};
    int64_t *h_seg = nullptr;
    double *h_d = nullptr, *h_t0 = nullptr, *h_t1 = nullptr;
    std::thread th;
};

bool valid_request(const tdq_segments *q, double d, double t0, double t1)
{
    if (!(d >= 0.0) || isinf(d) || isnan(t0) || isnan(t1) || t0 > t1) return false;
    const double *cols[8] = {q->xs, q->ys, q->zs, q->ts, q->xe, q->ye, q->ze, q->te};
    for (uint64_t i = 0; i < q->n; i++) {
        for (int c = 0; c < 8; c++)
            if (!isfinite(cols[c][i])) return false;
        if (!(q->te[i] > q->ts[i])) return false;
    }
    return true;
}

}  // namespace

struct tdq_server {
    tdq_index *idx = nullptr;
    tdq_server_params prm{};
    double rate = 0.0;  // estimated results per query segment
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<Request *> queue;
    std::unordered_map<uint64_t, Request *> reqs;
    uint64_t next_ticket = 1;
    uint64_t next_batch = 1;
    double bytes_in_flight = 0;
    int running_batches = 0;
    bool stopping = false;
    tdq_status fatal = TDQ_OK;
    std::vector<Lane> lanes;
    tdq_server_stats st{};
};

namespace {

using namespace tdq;

double estimate_bytes(const tdq_server *s, uint64_t n)
{
    // result items (32 B each) at the estimated rate, plus the per-segment
    // workspace of a batch (query columns, sort, tiles, survivors)
    return (double)n * (s->rate * 32.0 * 2.0 + 1024.0) + 4096.0;
}

tdq_status lane_alloc(Lane &L, uint64_t cap)
{
    L.cap = cap;
    for (int c = 0; c < 8; c++)
        if (host_alloc(&L.h_cols[c], cap * 8) != cudaSuccess) return set_error(TDQ_ERR_NOMEM, "server: staging");
    if (host_alloc(&L.h_seg, cap * 8) != cudaSuccess || host_alloc(&L.h_d, cap * 8) != cudaSuccess ||
        host_alloc(&L.h_t0, cap * 8) != cudaSuccess || host_alloc(&L.h_t1, cap * 8) != cudaSuccess)
        return set_error(TDQ_ERR_NOMEM, "server: staging");
    return TDQ_OK;
}

void lane_free(Lane &L)
{
    if (L.plan) tdq_plan_free(L.plan);
    if (L.stream) cudaStreamDestroy(L.stream);
    for (int c = 0; c < 8; c++) cudaFreeHost(L.h_cols[c]);
    cudaFreeHost(L.h_seg);
    cudaFreeHost(L.h_d);
    cudaFreeHost(L.h_t0);
    cudaFreeHost(L.h_t1);
}

// Search one packed batch on a lane and split its results per request.
tdq_status run_batch(tdq_server *s, Lane &L, std::vector<Request *> &batch, uint64_t nseg)
{
    std::vector<uint64_t> offs(batch.size() + 1, 0);
    for (size_t k = 0; k < batch.size(); k++) {
        Request *r = batch[k];
        const uint64_t o = offs[k];
        for (int c = 0; c < 8; c++) memcpy(L.h_cols[c] + o, r->cols[c].data(), r->n * 8);
        for (uint64_t i = 0; i < r->n; i++) {
            L.h_seg[o + i] = (int64_t)(o + i);  // position in the batch: maps results back
            L.h_d[o + i] = r->d;
            L.h_t0[o + i] = r->t0;
            L.h_t1[o + i] = r->t1;
        }
        offs[k + 1] = o + r->n;
    }
    tdq_segments q{};
    q.xs = L.h_cols[0]; q.ys = L.h_cols[1]; q.zs = L.h_cols[2]; q.ts = L.h_cols[3];
    q.xe = L.h_cols[4]; q.ye = L.h_cols[5]; q.ze = L.h_cols[6]; q.te = L.h_cols[7];
    q.seg_id = L.h_seg;
    q.n = nseg;
    q.on_device = 0;
    uint64_t cnt = 0;
    tdq_status st = tdq_plan_search(L.plan, &q, L.h_d, L.h_t0, L.h_t1, L.stream, &cnt);
    if (st != TDQ_OK) return st;
    // the lane's plan keeps its results in page-locked host memory: read in place
    tdq_result_buffer res{};
    st = tdq_plan_results(L.plan, &res, &cnt);
    if (st != TDQ_OK) return st;
    for (Request *r : batch) {
        r->r_q.clear();
        r->r_e.clear();
        r->r_tin.clear();
        r->r_tout.clear();
    }
    for (uint64_t i = 0; i < cnt; i++) {
        const uint64_t pos = (uint64_t)res.query_seg_id[i];
        const size_t k = (size_t)(std::upper_bound(offs.begin(), offs.end(), pos) - offs.begin()) - 1;
        Request *r = batch[k];
        r->r_q.push_back(r->seg_id[pos - offs[k]]);
        r->r_e.push_back(res.entry_seg_id[i]);
        r->r_tin.push_back(res.t_enter[i]);
        r->r_tout.push_back(res.t_exit[i]);
    }
    return TDQ_OK;
}

void lane_main(tdq_server *s, int li)
{
    Lane &L = s->lanes[li];
    cudaSetDevice(s->idx->device);
    std::unique_lock<std::mutex> lk(s->mu);
    for (;;) {
        s->cv_work.wait(lk, [&] {
            if (s->stopping && s->queue.empty()) return true;
            if (s->queue.empty()) return false;
            Request *f = s->queue.front();
            return s->bytes_in_flight == 0 || s->bytes_in_flight + f->est_bytes <= (double)s->prm.memory_cap_bytes;
        });
        if (s->queue.empty()) break;  // stopping
        std::vector<Request *> batch;
        uint64_t nseg = 0;
        const uint64_t bid = s->next_batch++;
        while (!s->queue.empty()) {
            Request *f = s->queue.front();
            if (nseg + f->n > L.cap) break;
            const bool fits = s->bytes_in_flight + f->est_bytes <= (double)s->prm.memory_cap_bytes;
            if (!fits && !(batch.empty() && s->bytes_in_flight == 0)) break;
            s->queue.pop_front();
            s->bytes_in_flight += f->est_bytes;
            f->state = 1;
            f->batch = bid;
            f->t_start = Clock::now();
            batch.push_back(f);
            nseg += f->n;
        }
        s->running_batches++;
        if ((uint64_t)s->running_batches > s->st.max_concurrent_batches)
            s->st.max_concurrent_batches = (uint64_t)s->running_batches;
        if (s->bytes_in_flight > s->st.peak_bytes_in_flight) s->st.peak_bytes_in_flight = s->bytes_in_flight;
        lk.unlock();
        s->cv_work.notify_all();  // other lanes may admit the rest
        const tdq_status st = run_batch(s, L, batch, nseg);
        lk.lock();
        s->running_batches--;
        const Clock::time_point now = Clock::now();
        for (Request *r : batch) {
            r->status = st;
            r->state = 2;
            r->batch_segments = nseg;
            r->t_done = now;
            s->bytes_in_flight -= r->est_bytes;
        }
        if (s->bytes_in_flight < 0.5) s->bytes_in_flight = 0;
        s->st.batches++;
        s->st.requests_completed += batch.size();
        s->st.query_segments += nseg;
        if (st != TDQ_OK) s->st.failed_batches++;
        s->cv_done.notify_all();
        s->cv_work.notify_all();
    }
}

}  // namespace

extern "C" tdq_status tdq_server_create(tdq_index *idx, const tdq_server_params *params, tdq_server **out)
{
    if (!out) return set_error(TDQ_ERR_INVALID, "tdq_server_create: out is NULL");
    *out = nullptr;
    if (!idx || !params) return set_error(TDQ_ERR_INVALID, "tdq_server_create: NULL argument");
    tdq_server *s = new (std::nothrow) tdq_server();
    if (!s) return set_error(TDQ_ERR_NOMEM, "tdq_server_create: host allocation failed");
    s->idx = idx;
    s->prm = *params;
    if (!s->prm.max_batch_query_segments) s->prm.max_batch_query_segments = 65536;
    if (!s->prm.memory_cap_bytes) s->prm.memory_cap_bytes = 16ULL << 30;
    if (s->prm.lanes <= 0) s->prm.lanes = 2;
    if (s->prm.lanes > 16) s->prm.lanes = 16;
    s->rate = s->prm.results_per_query_segment > 0 ? s->prm.results_per_query_segment : 4.0;
    s->lanes.resize(s->prm.lanes);
    tdq_status st = TDQ_OK;
    for (int k = 0; k < s->prm.lanes && st == TDQ_OK; k++) {
        Lane &L = s->lanes[k];
        if (cudaStreamCreateWithFlags(&L.stream, cudaStreamNonBlocking) != cudaSuccess) {
            st = set_error(TDQ_ERR_CUDA, "tdq_server_create: stream");
            break;
        }
        tdq_plan_params pp{};
        pp.max_query_segments = s->prm.max_batch_query_segments;
        pp.mode = s->prm.mode;
        pp.entry_chunk = s->prm.entry_chunk;
        pp.result_capacity = (uint64_t)(s->rate * 2.0 * (double)pp.max_query_segments) + 65536;
        pp.host_results = 1;
        st = tdq_plan_create(idx, &pp, &L.plan);
        if (st == TDQ_OK) st = lane_alloc(L, s->prm.max_batch_query_segments);
    }
    if (st != TDQ_OK) {
        for (Lane &L : s->lanes) lane_free(L);
        delete s;
        return st;
    }
    for (int k = 0; k < s->prm.lanes; k++) s->lanes[k].th = std::thread(lane_main, s, k);
    *out = s;
    return TDQ_OK;
}

extern "C" tdq_status tdq_server_submit(tdq_server *s, const tdq_segments *queries, double d, double t0, double t1,
                                        uint64_t *ticket)
{
    if (!s || !queries || !ticket) return set_error(TDQ_ERR_INVALID, "tdq_server_submit: NULL argument");
    *ticket = 0;
    if (queries->on_device) return set_error(TDQ_ERR_INVALID, "tdq_server_submit: queries must be in host memory");
    if (queries->n == 0 || queries->n > s->prm.max_batch_query_segments)
        return set_error(TDQ_ERR_INVALID, "tdq_server_submit: a request needs 1..%llu query segments",
                         (unsigned long long)s->prm.max_batch_query_segments);
    const double *cols[8] = {queries->xs, queries->ys, queries->zs, queries->ts,
                             queries->xe, queries->ye, queries->ze, queries->te};
    for (int c = 0; c < 8; c++)
        if (!cols[c]) return set_error(TDQ_ERR_INVALID, "tdq_server_submit: query column %d is NULL", c);
    if (!queries->seg_id) return set_error(TDQ_ERR_INVALID, "tdq_server_submit: seg_id is NULL");
    if (!valid_request(queries, d, t0, t1))
        return set_error(TDQ_ERR_INVALID, "tdq_server_submit: invalid query segment, threshold or window");
    Request *r = new (std::nothrow) Request();
    if (!r) return set_error(TDQ_ERR_NOMEM, "tdq_server_submit: host allocation failed");
    r->n = queries->n;
    for (int c = 0; c < 8; c++) r->cols[c].assign(cols[c], cols[c] + r->n);
    r->seg_id.assign(queries->seg_id, queries->seg_id + r->n);
    r->d = d;
    r->t0 = t0;
    r->t1 = t1;
    r->t_submit = Clock::now();
    {
        std::lock_guard<std::mutex> lk(s->mu);
        if (s->stopping) {
            delete r;
            return set_error(TDQ_ERR_INVALID, "tdq_server_submit: server is stopping");
        }
        r->est_bytes = estimate_bytes(s, r->n);
        r->ticket = s->next_ticket++;
        s->reqs[r->ticket] = r;
        s->queue.push_back(r);
        s->st.requests_submitted++;
    }
    s->cv_work.notify_one();
    *ticket = r->ticket;
    return TDQ_OK;
}

extern "C" tdq_status tdq_server_submit_many(tdq_server *s, const tdq_segments *queries, const uint64_t *offsets,
                                             uint64_t count, const double *d, const double *t0, const double *t1,
                                             uint64_t *tickets)
{
    if (!s || !queries || !offsets || !d || !t0 || !t1 || !tickets)
        return set_error(TDQ_ERR_INVALID, "tdq_server_submit_many: NULL argument");
    if (queries->on_device)
        return set_error(TDQ_ERR_INVALID, "tdq_server_submit_many: queries must be in host memory");
    if (count == 0) return TDQ_OK;
    const double *cols[8] = {queries->xs, queries->ys, queries->zs, queries->ts,
                             queries->xe, queries->ye, queries->ze, queries->te};
    for (int c = 0; c < 8; c++)
        if (!cols[c]) return set_error(TDQ_ERR_INVALID, "tdq_server_submit_many: query column %d is NULL", c);
    if (!queries->seg_id) return set_error(TDQ_ERR_INVALID, "tdq_server_submit_many: seg_id is NULL");
    if (offsets[0] != 0 || offsets[count] != queries->n)
        return set_error(TDQ_ERR_INVALID, "tdq_server_submit_many: offsets must run from 0 to queries->n");
    // validate every request first: all or nothing is queued
    for (uint64_t k = 0; k < count; k++) {
        const uint64_t a = offsets[k], b = offsets[k + 1];
        if (b < a || b - a == 0 || b - a > s->prm.max_batch_query_segments)
            return set_error(TDQ_ERR_INVALID, "tdq_server_submit_many: request %llu needs 1..%llu query segments",
                             (unsigned long long)k, (unsigned long long)s->prm.max_batch_query_segments);
        tdq_segments sub = *queries;
        sub.xs = cols[0] + a; sub.ys = cols[1] + a; sub.zs = cols[2] + a; sub.ts = cols[3] + a;
        sub.xe = cols[4] + a; sub.ye = cols[5] + a; sub.ze = cols[6] + a; sub.te = cols[7] + a;
        sub.seg_id = queries->seg_id + a;
        sub.n = b - a;
        if (!valid_request(&sub, d[k], t0[k], t1[k]))
            return set_error(TDQ_ERR_INVALID,
                             "tdq_server_submit_many: request %llu: invalid query segment, threshold or window",
                             (unsigned long long)k);
    }
    std::vector<Request *> made;
    made.reserve(count);
    for (uint64_t k = 0; k < count; k++) {
        Request *r = new (std::nothrow) Request();
        if (!r) {
            for (Request *x : made) delete x;
            return set_error(TDQ_ERR_NOMEM, "tdq_server_submit_many: host allocation failed");
        }
        const uint64_t a = offsets[k];
        r->n = offsets[k + 1] - a;
        for (int c = 0; c < 8; c++) r->cols[c].assign(cols[c] + a, cols[c] + a + r->n);
        r->seg_id.assign(queries->seg_id + a, queries->seg_id + a + r->n);
        r->d = d[k];
        r->t0 = t0[k];
        r->t1 = t1[k];
        made.push_back(r);
    }
    {
        std::lock_guard<std::mutex> lk(s->mu);
        if (s->stopping) {
            for (Request *x : made) delete x;
            return set_error(TDQ_ERR_INVALID, "tdq_server_submit_many: server is stopping");
        }
        const Clock::time_point now = Clock::now();
        for (uint64_t k = 0; k < count; k++) {
            Request *r = made[k];
            r->t_submit = now;
            r->est_bytes = estimate_bytes(s, r->n);
            r->ticket = s->next_ticket++;
            s->reqs[r->ticket] = r;
            s->queue.push_back(r);
            tickets[k] = r->ticket;
        }
        s->st.requests_submitted += count;
    }
    s->cv_work.notify_all();
    return TDQ_OK;
}

extern "C" tdq_status tdq_server_drain(tdq_server *s, int64_t timeout_ms)
{
    if (!s) return set_error(TDQ_ERR_INVALID, "tdq_server_drain: NULL argument");
    std::unique_lock<std::mutex> lk(s->mu);
    auto idle = [&] { return s->queue.empty() && s->running_batches == 0; };
    if (timeout_ms < 0) {
        s->cv_done.wait(lk, idle);
    } else if (!s->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), idle)) {
        return set_error(TDQ_ERR_TIMEOUT, "tdq_server_drain: requests still queued or running after %lld ms",
                         (long long)timeout_ms);
    }
    return TDQ_OK;
}

extern "C" tdq_status tdq_server_wait(tdq_server *s, uint64_t ticket, int64_t timeout_ms, tdq_results **out,
                                      tdq_request_info *info)
{
    if (!s || !out) return set_error(TDQ_ERR_INVALID, "tdq_server_wait: NULL argument");
    *out = nullptr;
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end()) return set_error(TDQ_ERR_INVALID, "tdq_server_wait: unknown ticket %llu",
                                              (unsigned long long)ticket);
    Request *r = it->second;
    auto done = [&] { return r->state == 2; };
    if (timeout_ms < 0) {
        s->cv_done.wait(lk, done);
    } else if (!s->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), done)) {
        return set_error(TDQ_ERR_TIMEOUT, "tdq_server_wait: ticket %llu not done after %lld ms",
                         (unsigned long long)ticket, (long long)timeout_ms);
    }
    s->reqs.erase(it);
    lk.unlock();
    if (info) {
        info->queue_ms = ms_between(r->t_submit, r->t_start);
        info->run_ms = ms_between(r->t_start, r->t_done);
        info->latency_ms = ms_between(r->t_submit, r->t_done);
        info->batch = r->batch;
        info->batch_query_segments = r->batch_segments;
    }
    tdq_status st = r->status;
    if (st != TDQ_OK) {
        delete r;
        return set_error(st, "tdq_server_wait: the request's batch failed");
    }
    tdq_results *res = (tdq_results *)calloc(1, sizeof(tdq_results));
    const uint64_t n = r->r_q.size();
    if (res && n) {
        res->query_seg_id = (int64_t *)malloc(n * 8);
        res->entry_seg_id = (int64_t *)malloc(n * 8);
        res->t_enter = (double *)malloc(n * 8);
        res->t_exit = (double *)malloc(n * 8);
    }
    if (!res || (n && (!res->query_seg_id || !res->entry_seg_id || !res->t_enter || !res->t_exit))) {
        tdq_results_free(res);
        delete r;
        return set_error(TDQ_ERR_NOMEM, "tdq_server_wait: host allocation failed");
    }
    res->count = n;
    if (n) {
        memcpy(res->query_seg_id, r->r_q.data(), n * 8);
        memcpy(res->entry_seg_id, r->r_e.data(), n * 8);
        memcpy(res->t_enter, r->r_tin.data(), n * 8);
        memcpy(res->t_exit, r->r_tout.data(), n * 8);
    }
    delete r;
    *out = res;
    return TDQ_OK;
}

extern "C" tdq_status tdq_server_get_stats(tdq_server *s, tdq_server_stats *out)
{
    if (!s || !out) return set_error(TDQ_ERR_INVALID, "tdq_server_get_stats: NULL argument");
    std::lock_guard<std::mutex> lk(s->mu);
    *out = s->st;
    out->queued = s->queue.size();
    return TDQ_OK;
}

extern "C" void tdq_server_free(tdq_server *s)
{
    if (!s) return;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stopping = true;
    }
    s->cv_work.notify_all();
    for (Lane &L : s->lanes)
        if (L.th.joinable()) L.th.join();
    for (Lane &L : s->lanes) lane_free(L);
    for (auto &kv : s->reqs) delete kv.second;
    delete s;
}
