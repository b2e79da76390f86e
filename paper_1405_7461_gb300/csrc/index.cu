// Temporal-bin index (Sec. 4, Fig. 1), built on the device.
//
//   1. validate each entry segment and compute its velocity;
//   2. stable sort by t_start (radix sort of order-preserving integer keys);
//   3. gather the sorted structure-of-arrays copy that stays resident in HBM
//      for every later search (Sec. 3: D is stored once and for all);
//   4. bins of fixed width b = (t_max - t_min)/m: an entry goes to bin
//      min(m-1, floor((t_start - t_min)/b)); per bin the first sorted position
//      (bins are contiguous runs of the sorted order) and the largest t_end;
//      then the prefix maximum of the bin ends, which turns "first bin whose
//      extent can reach time t" into a binary search.
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <new>

#include "tdq_internal.cuh"

namespace tdq {
namespace {

struct EntryInput {
    const double *c[8];  // xs ys zs ts xe ye ze te
    const int64_t *seg_id, *traj_id;
};

// Validate, and emit the sort key and time range of every entry.  The time
// range is reduced per warp before one atomic per warp.
__global__ void entry_prep(EntryInput in, uint64_t n, uint64_t *keys, uint32_t *vals, unsigned int *err,
                           unsigned long long *tmin_key, unsigned long long *tmax_key, unsigned long long *max_dur,
                           unsigned long long *cbox)
{
    uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    unsigned long long kmin = ~0ULL, kmax = 0ULL, dmax = 0ULL;
    // bounding box of the segments' midpoints (the tensor-core pre-test's
    // grid), as order-preserving unsigned keys: cbox = min x, y, z, max x, y, z
    unsigned long long cmin[3] = {~0ULL, ~0ULL, ~0ULL}, cmax[3] = {0ULL, 0ULL, 0ULL};
    if (i < n) {
        bool ok = true;
#pragma unroll
        for (int c = 0; c < 8; c++) ok &= finite_bits(in.c[c][i]);
        int64_t ks = okey(in.c[3][i]);
        int64_t ke = okey(in.c[7][i]);
        ok &= ke > ks;
        if (!ok) atomicOr(err, 1u);
        keys[i] = (uint64_t)ks ^ 0x8000000000000000ULL;
        vals[i] = (uint32_t)i;
        // time extent as unsigned keys (same order as the doubles)
        kmin = (uint64_t)ks ^ 0x8000000000000000ULL;
        kmax = (uint64_t)ke ^ 0x8000000000000000ULL;
        // longest duration: positive doubles order like their bit patterns
        if (ok) dmax = (unsigned long long)__double_as_longlong(in.c[7][i] - in.c[3][i]);
        if (ok) {
#pragma unroll
            for (int a = 0; a < 3; a++) {
                const unsigned long long kc = ukey(0.5 * in.c[a][i] + 0.5 * in.c[4 + a][i]);
                cmin[a] = kc;
                cmax[a] = kc;
            }
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        kmin = min(kmin, __shfl_xor_sync(0xffffffffu, kmin, o));
        kmax = max(kmax, __shfl_xor_sync(0xffffffffu, kmax, o));
        dmax = max(dmax, __shfl_xor_sync(0xffffffffu, dmax, o));
#pragma unroll
        for (int a = 0; a < 3; a++) {
            cmin[a] = min(cmin[a], __shfl_xor_sync(0xffffffffu, cmin[a], o));
            cmax[a] = max(cmax[a], __shfl_xor_sync(0xffffffffu, cmax[a], o));
        }
    }
    if ((threadIdx.x & 31) == 0) {
        if (kmin != ~0ULL) atomicMin(tmin_key, kmin);
        if (kmax != 0ULL) atomicMax(tmax_key, kmax);
        if (dmax != 0ULL) atomicMax(max_dur, dmax);
#pragma unroll
        for (int a = 0; a < 3; a++) {
            if (cmin[a] != ~0ULL) atomicMin(&cbox[a], cmin[a]);
            if (cmax[a] != 0ULL) atomicMax(&cbox[3 + a], cmax[a]);
        }
    }
}

__global__ void entry_gather(EntryInput in, uint64_t n, const uint32_t *order, EntrySoA e, TcGrid grid)
{
    uint64_t k = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    uint32_t i = order[k];
    double ts = in.c[3][i], te = in.c[7][i];
    double dt = te - ts;
    double xs = in.c[0][i], ys = in.c[1][i], zs = in.c[2][i];
    e.px[k] = xs;
    e.py[k] = ys;
    e.pz[k] = zs;
    e.vx[k] = (in.c[4][i] - xs) / dt;
    e.vy[k] = (in.c[5][i] - ys) / dt;
    e.vz[k] = (in.c[6][i] - zs) / dt;
    e.ts_key[k] = okey(ts);
    e.te_key[k] = okey(te);
    e.seg_id[k] = in.seg_id[i];
    e.traj_id[k] = in.traj_id ? in.traj_id[i] : 0;
    e.orig[k] = (int64_t)i;
    // FP32 bounding sphere: midpoint and half length of the segment, and the
    // pre-test's per-entry term E = |c|^2 (1 - 2^-20), rounded down (the
    // squares of floats are exact in FP64).
    double hx = 0.5 * (in.c[4][i] - xs), hy = 0.5 * (in.c[5][i] - ys), hz = 0.5 * (in.c[6][i] - zs);
    const float4 sp = sphere32(xs + hx, ys + hy, zs + hz, norm_ru(hx, hy, hz), 0.f);
    if (isinf(sp.w)) {
        e.sph[k] = make_float4(0.f, 0.f, 0.f, 0.f);
        e.sph_e[k] = __int_as_float(0xff800000);  // -inf: never rejected
    } else {
        const double c2 = __fma_rd(sp.z, sp.z, __fma_rd(sp.y, sp.y, __dmul_rd(sp.x, sp.x)));
        e.sph[k] = sp;
        e.sph_e[k] = __double2float_rd(__dmul_rd(c2, 1.0 - 0x1p-20));
    }
    // the tensor-core pre-test's record: the same sphere in FP64 on the grid
    uint4 lo, hi;
    tc_entry_record(xs + hx, ys + hy, zs + hz, sqrt(fma(hz, hz, fma(hy, hy, hx * hx))), grid, lo, hi);
    tc_store(e.tc_rec, k, lo, hi);
}

// Unsigned radix keys of the sorted entries' t_end (values unused).
__global__ void te_keys(const int64_t *te_key, uint64_t n, uint64_t *keys, uint32_t *vals)
{
    uint64_t k = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    keys[k] = (uint64_t)te_key[k] ^ 0x8000000000000000ULL;
    vals[k] = 0;
}

__global__ void te_store(const uint64_t *keys, uint64_t n, int64_t *te_sorted)
{
    uint64_t k = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    te_sorted[k] = (int64_t)(keys[k] ^ 0x8000000000000000ULL);
}

__global__ void bin_init(int64_t *bin_end_key, uint32_t m)
{
    uint64_t j = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j < m) bin_end_key[j] = INT64_MIN;
}

// bin_begin[j] = first sorted position whose bin is >= j (bin_begin[m] = n).
__global__ void bin_assign(const int64_t *ts_key, const int64_t *te_key, uint64_t n, double t_min, double width,
                           uint32_t m, int64_t *bin_begin, int64_t *bin_end_key)
{
    uint64_t k = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    int64_t bk = bin_of(key_double(ts_key[k]), t_min, width, m);
    int64_t bprev = (k == 0) ? -1 : bin_of(key_double(ts_key[k - 1]), t_min, width, m);
    for (int64_t j = bprev + 1; j <= bk; j++) bin_begin[j] = (int64_t)k;
    if (k == n - 1)
        for (int64_t j = bk + 1; j <= (int64_t)m; j++) bin_begin[j] = (int64_t)n;
    atomicMax((long long *)&bin_end_key[bk], (long long)te_key[k]);
}

// Bin table over the sorted t_end keys: te_bin_begin[b] = first position
// whose t_end lies in a bin >= b (same bins and bin function as the t_start
// table, so that a count of t_end <= t narrows to the bin of t).
__global__ void te_bin_assign(const int64_t *te_sorted, uint64_t n, double t_min, double width, uint32_t m,
                              int64_t *te_bin_begin)
{
    uint64_t k = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    int64_t bk = bin_of(key_double(te_sorted[k]), t_min, width, m);
    int64_t bprev = (k == 0) ? -1 : bin_of(key_double(te_sorted[k - 1]), t_min, width, m);
    for (int64_t j = bprev + 1; j <= bk; j++) te_bin_begin[j] = (int64_t)k;
    if (k == n - 1)
        for (int64_t j = bk + 1; j <= (int64_t)m; j++) te_bin_begin[j] = (int64_t)n;
}

// Each bin's smallest time key under bin_of: bin_lo_key[b] = the smallest key
// k of a non-NaN time whose bin is >= b (b = 1 .. m-1; bin_of is monotone in
// time), by bisection over the keys of -inf .. +inf; bin_lo_key[0] =
// INT64_MIN, bin_lo_key[m] = INT64_MAX.  The bin of a time with key k is
// then the last b with bin_lo_key[b] <= k, exactly bin_of's.
__global__ void bin_bounds(double t_min, double width, uint32_t m, int64_t *bin_lo_key)
{
    const uint64_t b = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (b > m) return;
    if (b == 0 || b == m) {
        bin_lo_key[b] = b == 0 ? INT64_MIN : INT64_MAX;
        return;
    }
    int64_t lo = okey(__longlong_as_double((long long)0xfff0000000000000ULL));  // -inf
    int64_t hi = okey(__longlong_as_double((long long)0x7ff0000000000000ULL));  // +inf: bin m - 1 >= b
    while (lo < hi) {
        const int64_t mid = lo + (int64_t)(((uint64_t)hi - (uint64_t)lo) >> 1);
        if (bin_of(key_double(mid), t_min, width, m) >= (int64_t)b) hi = mid; else lo = mid + 1;
    }
    bin_lo_key[b] = lo;
}

// Prefix maximum of the bin ends (one block).
__global__ void __launch_bounds__(1024) bin_prefix_max(const int64_t *bin_end_key, uint32_t m, int64_t *pmax)
{
    __shared__ int64_t warp_max[32];
    __shared__ int64_t carry;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid == 0) carry = INT64_MIN;
    __syncthreads();
    for (uint64_t start = 0; start < m; start += 1024) {
        uint64_t j = start + tid;
        int64_t x = j < m ? bin_end_key[j] : INT64_MIN;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int64_t y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x = max(x, y);
        }
        if (lane == 31) warp_max[warp] = x;
        __syncthreads();
        if (warp == 0) {
            int64_t w = warp_max[lane];
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                int64_t y = __shfl_up_sync(0xffffffffu, w, o);
                if (lane >= o) w = max(w, y);
            }
            warp_max[lane] = w;
        }
        __syncthreads();
        int64_t v = max(carry, x);
        if (warp > 0) v = max(v, warp_max[warp - 1]);
        if (j < m) pmax[j] = v;
        __syncthreads();
        if (tid == 0) carry = max(carry, warp_max[31]);
        __syncthreads();
    }
}

__global__ void bin_export(const int64_t *bin_begin, const int64_t *bin_end_key, const int64_t *ts_key, uint32_t m,
                           double *start, double *end, int64_t *first, int64_t *last)
{
    uint64_t j = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= m) return;
    int64_t b = bin_begin[j], e = bin_begin[j + 1];
    if (e > b) {
        start[j] = key_double(ts_key[b]);
        end[j] = key_double(bin_end_key[j]);
        first[j] = b;
        last[j] = e - 1;
    } else {
        start[j] = __longlong_as_double(0x7ff8000000000000LL);
        end[j] = start[j];
        first[j] = -1;
        last[j] = -1;
    }
}

}  // namespace
}  // namespace tdq

using namespace tdq;

extern "C" tdq_status tdq_build_index(const tdq_segments *entries, const tdq_index_params *params, void *stream_,
                                      tdq_index **out)
{
    if (!out) return set_error(TDQ_ERR_INVALID, "tdq_build_index: out is NULL");
    *out = nullptr;
    if (!entries) return set_error(TDQ_ERR_INVALID, "tdq_build_index: entries is NULL");
    const uint64_t n = entries->n;
    if (n > 0) {
        const double *cols[8] = {entries->xs, entries->ys, entries->zs, entries->ts,
                                 entries->xe, entries->ye, entries->ze, entries->te};
        for (int c = 0; c < 8; c++)
            if (!cols[c]) return set_error(TDQ_ERR_INVALID, "tdq_build_index: column %d is NULL", c);
        if (!entries->seg_id) return set_error(TDQ_ERR_INVALID, "tdq_build_index: seg_id is NULL");
        if (n > 0xffffffffULL) return set_error(TDQ_ERR_INVALID, "tdq_build_index: more than 2^32-1 segments");
    }
    uint32_t m = (params && params->bin_count) ? params->bin_count : 10000u;
    cudaStream_t stream = (cudaStream_t)stream_;

    tdq_index *idx = new (std::nothrow) tdq_index();
    if (!idx) return set_error(TDQ_ERR_NOMEM, "tdq_build_index: host allocation failed");
    cudaGetDevice(&idx->device);
    cudaDeviceGetAttribute(&idx->sm_count, cudaDevAttrMultiProcessorCount, idx->device);
    if (load_device_code() != cudaSuccess) {
        delete idx;
        return cuda_error(cudaGetLastError(), "tdq_build_index: loading the device code");
    }
    idx->n = n;
    idx->m = m;
    for (int k = 0; k < kSearchEvents; k++) {
        if (cudaEventCreate(&idx->ws.ev[k]) != cudaSuccess) {
            tdq_index_free(idx);
            return set_error(TDQ_ERR_CUDA, "tdq_build_index: cudaEventCreate failed");
        }
    }
    if (dev_alloc(&idx->ws.ctr, kCtrBlockBytes) != cudaSuccess ||
        host_alloc_mapped(&idx->ws.ctr_host, &idx->ws.ctr_host_dev, sizeof(DevCounters)) != cudaSuccess) {
        tdq_index_free(idx);
        return set_error(TDQ_ERR_NOMEM, "tdq_build_index: counter allocation failed");
    }
    idx->ws.sort_fused_hist = (uint32_t *)((char *)idx->ws.ctr + kCtrBytes);
    if (n == 0) {
        *out = idx;
        return TDQ_OK;
    }

    // Resident sorted copy + bin table.
    idx->n_rec = (n + 7) / 8 * 8 + 128;  // whole groups of 8, and room for a pass of 128 from any group
    uint64_t ebytes = 12 * carve_bytes(n, 8) + carve_bytes(n, 4) + carve_bytes(n, 16) +
                      carve_bytes(2 * idx->n_rec, 16);
    uint64_t bbytes = 3 * carve_bytes(m + 1, 8) + 2 * carve_bytes(m, 8);
    if (dev_alloc(&idx->e_block, ebytes) != cudaSuccess || dev_alloc(&idx->b_block, bbytes) != cudaSuccess) {
        cudaGetLastError();
        tdq_index_free(idx);
        return set_error(TDQ_ERR_NOMEM, "tdq_build_index: device allocation of %llu bytes failed",
                         (unsigned long long)(ebytes + bbytes));
    }
    {
        char *p = (char *)idx->e_block;
        EntrySoA &e = idx->e;
        e.px = carve<double>(p, n); e.py = carve<double>(p, n); e.pz = carve<double>(p, n);
        e.vx = carve<double>(p, n); e.vy = carve<double>(p, n); e.vz = carve<double>(p, n);
        e.ts_key = carve<int64_t>(p, n); e.te_key = carve<int64_t>(p, n);
        e.seg_id = carve<int64_t>(p, n); e.traj_id = carve<int64_t>(p, n); e.orig = carve<int64_t>(p, n);
        e.te_sorted = carve<int64_t>(p, n);
        e.sph_e = carve<float>(p, n);
        e.sph = carve<float4>(p, n);
        e.tc_rec = carve<uint4>(p, 2 * idx->n_rec);
        char *q = (char *)idx->b_block;
        idx->bin_begin = carve<int64_t>(q, m + 1);
        idx->bin_end_key = carve<int64_t>(q, m);
        idx->bin_pmax_key = carve<int64_t>(q, m);
        idx->te_bin_begin = carve<int64_t>(q, m + 1);
        idx->bin_lo_key = carve<int64_t>(q, m + 1);
    }

    // Temporary build memory: staged input (host case), sort buffers, scratch.
    const bool host_in = !entries->on_device;
    uint64_t tbytes = (host_in ? 10 * carve_bytes(n, 8) : 0) + 2 * carve_bytes(n, 8) + 2 * carve_bytes(n, 4) +
                      carve_bytes(sort_hist_words(n), 4) + carve_bytes(4, 8);
    void *tmp = nullptr;
    if (dev_alloc(&tmp, tbytes) != cudaSuccess) {
        cudaGetLastError();
        tdq_index_free(idx);
        return set_error(TDQ_ERR_NOMEM, "tdq_build_index: device allocation of %llu bytes failed",
                         (unsigned long long)tbytes);
    }
    tdq_status st = TDQ_OK;
    do {
        char *p = (char *)tmp;
        EntryInput in{};
        const double *cols[8] = {entries->xs, entries->ys, entries->zs, entries->ts,
                                 entries->xe, entries->ye, entries->ze, entries->te};
        if (host_in) {
            for (int c = 0; c < 8; c++) {
                double *dcol = carve<double>(p, n);
                if (cudaMemcpyAsync(dcol, cols[c], n * 8, cudaMemcpyHostToDevice, stream) != cudaSuccess) {
                    st = cuda_error(cudaGetLastError(), "tdq_build_index: H2D copy");
                    break;
                }
                in.c[c] = dcol;
            }
            if (st != TDQ_OK) break;
            int64_t *sid = carve<int64_t>(p, n);
            int64_t *tid = carve<int64_t>(p, n);
            if (cudaMemcpyAsync(sid, entries->seg_id, n * 8, cudaMemcpyHostToDevice, stream) != cudaSuccess) {
                st = cuda_error(cudaGetLastError(), "tdq_build_index: H2D copy");
                break;
            }
            in.seg_id = sid;
            in.traj_id = nullptr;
            if (entries->traj_id) {
                if (cudaMemcpyAsync(tid, entries->traj_id, n * 8, cudaMemcpyHostToDevice, stream) != cudaSuccess) {
                    st = cuda_error(cudaGetLastError(), "tdq_build_index: H2D copy");
                    break;
                }
                in.traj_id = tid;
            }
        } else {
            for (int c = 0; c < 8; c++) in.c[c] = cols[c];
            in.seg_id = entries->seg_id;
            in.traj_id = entries->traj_id;
        }
        uint64_t *keys = carve<uint64_t>(p, n);
        uint64_t *keys_alt = carve<uint64_t>(p, n);
        uint32_t *vals = carve<uint32_t>(p, n);
        uint32_t *vals_alt = carve<uint32_t>(p, n);
        uint32_t *hist = carve<uint32_t>(p, sort_hist_words(n));
        // err, tmin, tmax, longest duration, midpoint box (min x y z, max x y z)
        unsigned long long *small = carve<unsigned long long>(p, 10);

        unsigned long long init[10] = {0ULL, ~0ULL, 0ULL, 0ULL, ~0ULL, ~0ULL, ~0ULL, 0ULL, 0ULL, 0ULL};
        static_assert(sizeof init <= sizeof(DevCounters), "the host mirror stages the reduction words");
        DevCounters *hc = idx->ws.ctr_host;
        memcpy(hc, init, sizeof init);
        if (cudaMemcpyAsync(small, hc, sizeof init, cudaMemcpyHostToDevice, stream) != cudaSuccess) {
            st = cuda_error(cudaGetLastError(), "tdq_build_index: init copy");
            break;
        }
        entry_prep<<<grid_for(n), kBlock, 0, stream>>>(in, n, keys, vals, (unsigned int *)&small[0], &small[1],
                                                        &small[2], &small[3], &small[4]);
        if (cudaMemcpyAsync(hc, small, sizeof init, cudaMemcpyDeviceToHost, stream) != cudaSuccess ||
            cudaStreamSynchronize(stream) != cudaSuccess) {
            st = cuda_error(cudaGetLastError(), "tdq_build_index: entry validation");
            break;
        }
        unsigned long long back[10];
        memcpy(back, hc, sizeof back);
        if (back[0] & 1ULL) {
            st = set_error(TDQ_ERR_INVALID,
                           "tdq_build_index: invalid entry segment (non-finite value or t_end <= t_start)");
            break;
        }
        // recover t_min / t_max from their keys
        {
            int64_t kmin = (int64_t)(back[1] ^ 0x8000000000000000ULL);
            int64_t kmax = (int64_t)(back[2] ^ 0x8000000000000000ULL);
            int64_t bmin = key_from_bits(kmin), bmax = key_from_bits(kmax);
            memcpy(&idx->t_min, &bmin, 8);
            memcpy(&idx->t_max, &bmax, 8);
            idx->tmin_key = kmin;
            idx->width = (idx->t_max - idx->t_min) / (double)m;
            memcpy(&idx->max_dur, &back[3], 8);
            double box[6];
            for (int a = 0; a < 6; a++) {
                const int64_t b = key_from_bits((int64_t)(back[4 + a] ^ 0x8000000000000000ULL));
                memcpy(&box[a], &b, 8);
            }
            idx->grid = tc_grid_from_box(box[0], box[3], box[1], box[4], box[2], box[5]);
        }
        if (radix_sort_pairs(keys, vals, keys_alt, vals_alt, n, hist, stream) != cudaSuccess) {
            st = cuda_error(cudaGetLastError(), "tdq_build_index: sort");
            break;
        }
        if (cudaMemsetAsync(idx->e.tc_rec + 2 * (n / 8 * 8), 0, 32 * (idx->n_rec - n / 8 * 8), stream) !=
            cudaSuccess) {
            st = cuda_error(cudaGetLastError(), "tdq_build_index: record padding");
            break;
        }
        entry_gather<<<grid_for(n), kBlock, 0, stream>>>(in, n, vals, idx->e, idx->grid);
        bin_init<<<grid_for(m), kBlock, 0, stream>>>(idx->bin_end_key, m);
        bin_assign<<<grid_for(n), kBlock, 0, stream>>>(idx->e.ts_key, idx->e.te_key, n, idx->t_min, idx->width, m,
                                                       idx->bin_begin, idx->bin_end_key);
        bin_prefix_max<<<1, 1024, 0, stream>>>(idx->bin_end_key, m, idx->bin_pmax_key);
        bin_bounds<<<grid_for((uint64_t)m + 1), kBlock, 0, stream>>>(idx->t_min, idx->width, m, idx->bin_lo_key);
        // t_end keys in ascending order: #overlaps(q) = #{ts < q.te} - #{te <= q.ts}
        te_keys<<<grid_for(n), kBlock, 0, stream>>>(idx->e.te_key, n, keys, vals);
        if (radix_sort_pairs(keys, vals, keys_alt, vals_alt, n, hist, stream) != cudaSuccess) {
            st = cuda_error(cudaGetLastError(), "tdq_build_index: t_end sort");
            break;
        }
        te_store<<<grid_for(n), kBlock, 0, stream>>>(keys, n, idx->e.te_sorted);
        te_bin_assign<<<grid_for(n), kBlock, 0, stream>>>(idx->e.te_sorted, n, idx->t_min, idx->width, m,
                                                          idx->te_bin_begin);
        if (cudaStreamSynchronize(stream) != cudaSuccess || cudaGetLastError() != cudaSuccess) {
            st = cuda_error(cudaGetLastError(), "tdq_build_index: index kernels");
            break;
        }
    } while (0);
    cudaFree(tmp);
    if (st != TDQ_OK) {
        tdq_index_free(idx);
        return st;
    }
    *out = idx;
    return TDQ_OK;
}

extern "C" uint64_t tdq_index_size(const tdq_index *idx) { return idx ? idx->n : 0; }

extern "C" tdq_status tdq_index_bins(const tdq_index *idx, uint32_t *m, double *width, double *t_min,
                                     double *bin_start, double *bin_end, int64_t *bin_first, int64_t *bin_last,
                                     int64_t *sorted_index)
{
    if (!idx || !m) return set_error(TDQ_ERR_INVALID, "tdq_index_bins: NULL argument");
    *m = idx->m;
    if (width) *width = idx->width;
    if (t_min) *t_min = idx->t_min;
    if (sorted_index && idx->n) TDQ_CUDA(cudaMemcpy(sorted_index, idx->e.orig, idx->n * 8, cudaMemcpyDeviceToHost));
    if (!bin_start && !bin_end && !bin_first && !bin_last) return TDQ_OK;
    if (!bin_start || !bin_end || !bin_first || !bin_last)
        return set_error(TDQ_ERR_INVALID, "tdq_index_bins: pass all four bin arrays or none");
    const uint32_t mm = idx->m;
    if (idx->n == 0) {
        for (uint32_t j = 0; j < mm; j++) {
            bin_start[j] = bin_end[j] = NAN;
            bin_first[j] = bin_last[j] = -1;
        }
        return TDQ_OK;
    }
    void *tmp = nullptr;
    if (dev_alloc(&tmp, (uint64_t)mm * 32) != cudaSuccess) {
        cudaGetLastError();
        return set_error(TDQ_ERR_NOMEM, "tdq_index_bins: device allocation failed");
    }
    double *s = (double *)tmp;
    double *e = s + mm;
    int64_t *f = (int64_t *)(e + mm);
    int64_t *l = f + mm;
    bin_export<<<grid_for(mm), kBlock>>>(idx->bin_begin, idx->bin_end_key, idx->e.ts_key, mm, s, e, f, l);
    cudaError_t err = cudaMemcpy(bin_start, s, mm * 8, cudaMemcpyDeviceToHost);
    if (err == cudaSuccess) err = cudaMemcpy(bin_end, e, mm * 8, cudaMemcpyDeviceToHost);
    if (err == cudaSuccess) err = cudaMemcpy(bin_first, f, mm * 8, cudaMemcpyDeviceToHost);
    if (err == cudaSuccess) err = cudaMemcpy(bin_last, l, mm * 8, cudaMemcpyDeviceToHost);
    cudaFree(tmp);
    if (err != cudaSuccess) return cuda_error(err, "tdq_index_bins: copy");
    return TDQ_OK;
}

extern "C" void tdq_index_free(tdq_index *idx)
{
    if (!idx) return;
    Workspace &w = idx->ws;
    cudaFree(w.q_block);
    cudaFree(w.t_block);
    cudaFree(w.sort_hist);
    cudaFree(w.r_block);
    cudaFree(w.s_block);
    cudaFree(w.bin_cnt);
    cudaFree(w.ctr);
    if (w.ctr_host) cudaFreeHost(w.ctr_host);
    for (int k = 0; k < kSearchEvents; k++)
        if (w.ev[k]) cudaEventDestroy(w.ev[k]);
    cudaFree(idx->e_block);
    cudaFree(idx->b_block);
    delete idx;
}
