// fem_session.cu -- exact counts kept over a stream that grows by appends.
//
// "Future Work" asks for counting over events that keep arriving.  The
// count stays exact here: the greedy of Algorithm 1 walks the end events in
// time order and needs, per end event j, only its latest start L(j) (every
// occurrence ending at j starts no earlier than t_j - sum(hi)) and the end
// it kept last.  So a session keeps, per episode, the count and the time of
// the last kept end, plus the tail of the stream that a new end can still
// reach back to: the events at or after t_last - max sum(hi).  An append
// counts, by node-by-node local tracking (fem_plt.cu), the tail followed by
// the new events, takes only the ends among the new events, and starts
// the greedy from the stored last end.  Ends inside the tail cannot be kept
// again: their latest start is at most the stored last end (each was either
// kept, moving the last end to its own time, or refused for that reason).
#include <algorithm>
#include <mutex>
#include <vector>

#include "fem_internal.cuh"

struct fem_session {
    fem_ctx *ctx = nullptr;
    uint32_t n_types = 0;
    int64_t n_cand = 0, n_nodes = 0;
    int64_t *d_offs = nullptr;
    uint16_t *d_types = nullptr;
    int32_t *d_lo = nullptr, *d_hi = nullptr;
    uint32_t *d_counts = nullptr;
    int32_t *d_prev = nullptr;       // time of the last kept end per episode (INT32_MIN: none)
    int64_t span_max = 0;            // largest sum(hi) over the episodes
    uint16_t *d_tail_type = nullptr; // retained tail
    int32_t *d_tail_time = nullptr;
    int64_t n_tail = 0, tail_cap = 0;
    std::vector<int64_t> tail_cnt;   // tail events per type
    int64_t seen = 0;                // events appended so far
};

namespace fem {
namespace {

// First index with time >= cut (one thread).
__global__ void k_lower_bound(const int32_t *__restrict__ tm, int64_t n, int64_t cut, int64_t *out) {
    int64_t lo = 0, hi = n;
    while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if ((int64_t)tm[mid] < cut) lo = mid + 1; else hi = mid;
    }
    *out = lo;
}

__global__ void k_type_hist(const uint16_t *__restrict__ ty, int64_t n, unsigned long long *__restrict__ h) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        atomicAdd(&h[ty[i]], 1ull);
}

void session_free_buffers(fem_session *s) {
    fem_ctx *ctx = s->ctx;
    const int64_t ne = std::max<int64_t>(s->n_nodes - s->n_cand, 1);
    dev_free(ctx, s->d_offs, 8 * (s->n_cand + 1));
    dev_free(ctx, s->d_types, 2 * std::max<int64_t>(s->n_nodes, 1));
    dev_free(ctx, s->d_lo, 4 * ne);
    dev_free(ctx, s->d_hi, 4 * ne);
    dev_free(ctx, s->d_counts, 4 * std::max<int64_t>(s->n_cand, 1));
    dev_free(ctx, s->d_prev, 4 * std::max<int64_t>(s->n_cand, 1));
    if (s->tail_cap) {
        dev_free(ctx, s->d_tail_type, 2 * s->tail_cap);
        dev_free(ctx, s->d_tail_time, 4 * s->tail_cap);
    }
}

}  // namespace
}  // namespace fem

using namespace fem;

extern "C" int fem_session_create(fem_ctx *ctx, const fem_cands *c, uint32_t n_types, fem_session **out) {
    if (!ctx || !c || !out || c->n_cand < 0 || c->n_cand > INT32_MAX / 2 || n_types < 1 || n_types > 8192)
        return FEM_ERR_INVAL;
    const int64_t n = c->n_cand;
    if (n > 0 && (!c->offs || !c->types || !c->lo || !c->hi)) return FEM_ERR_INVAL;
    std::lock_guard<std::mutex> g(ctx->mu);
    cudaSetDevice(ctx->device);
    *out = nullptr;
    // candidates to the host for the checks and the span
    std::vector<int64_t> offs(n + 1, 0);
    if (n > 0 && c->ptr_is_device) {
        FEM_CUDA_TRY(cudaMemcpyAsync(offs.data(), c->offs, 8 * (n + 1), cudaMemcpyDeviceToHost, ctx->stream));
        FEM_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
    } else if (n > 0) {
        std::copy(c->offs, c->offs + n + 1, offs.begin());
    }
    if (offs[0] != 0) return FEM_ERR_INVAL;
    for (int64_t i = 0; i < n; ++i)
        if (offs[i + 1] <= offs[i] || offs[i + 1] - offs[i] > FEM_MAX_NODES) return FEM_ERR_INVAL;
    const int64_t n_nodes = offs[n], n_edges = n_nodes - n;
    std::vector<uint16_t> ty(std::max<int64_t>(n_nodes, 1));
    std::vector<int32_t> lo(std::max<int64_t>(n_edges, 1)), hi(std::max<int64_t>(n_edges, 1));
    if (c->ptr_is_device) {
        if (n_nodes > 0) FEM_CUDA_TRY(cudaMemcpyAsync(ty.data(), c->types, 2 * n_nodes, cudaMemcpyDeviceToHost, ctx->stream));
        if (n_edges > 0) {
            FEM_CUDA_TRY(cudaMemcpyAsync(lo.data(), c->lo, 4 * n_edges, cudaMemcpyDeviceToHost, ctx->stream));
            FEM_CUDA_TRY(cudaMemcpyAsync(hi.data(), c->hi, 4 * n_edges, cudaMemcpyDeviceToHost, ctx->stream));
        }
        FEM_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
    } else {
        std::copy(c->types, c->types + n_nodes, ty.begin());
        std::copy(c->lo, c->lo + n_edges, lo.begin());
        std::copy(c->hi, c->hi + n_edges, hi.begin());
    }
    int64_t span_max = 0;
    for (int64_t i = 0; i < n; ++i) {
        int64_t span = 0;
        for (int64_t k = offs[i]; k < offs[i + 1]; ++k)
            if (ty[k] >= n_types) return FEM_ERR_INVAL;
        for (int64_t e = offs[i] - i; e < offs[i + 1] - i - 1; ++e) {
            if (lo[e] < 0 || lo[e] >= hi[e]) return FEM_ERR_INVAL;
            span += hi[e];
        }
        span_max = std::max(span_max, span);
    }
    fem_session *s = new (std::nothrow) fem_session();
    if (!s) return FEM_ERR_NOMEM;
    s->ctx = ctx;
    s->n_types = n_types;
    s->n_cand = n;
    s->n_nodes = n_nodes;
    s->span_max = span_max;
    s->tail_cnt.assign(n_types, 0);
    const int64_t ne = std::max<int64_t>(n_edges, 1), nc = std::max<int64_t>(n, 1);
    void *p[6] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
    const size_t sz[6] = {size_t(8 * (n + 1)), size_t(2 * std::max<int64_t>(n_nodes, 1)), size_t(4 * ne),
                          size_t(4 * ne), size_t(4 * nc), size_t(4 * nc)};
    int st = FEM_OK;
    for (int i = 0; i < 6 && st == FEM_OK; ++i) st = dev_alloc(ctx, &p[i], sz[i]);
    if (st != FEM_OK) {
        for (int i = 0; i < 6; ++i)
            if (p[i]) dev_free(ctx, p[i], sz[i]);
        delete s;
        return st;
    }
    s->d_offs = static_cast<int64_t *>(p[0]);
    s->d_types = static_cast<uint16_t *>(p[1]);
    s->d_lo = static_cast<int32_t *>(p[2]);
    s->d_hi = static_cast<int32_t *>(p[3]);
    s->d_counts = static_cast<uint32_t *>(p[4]);
    s->d_prev = static_cast<int32_t *>(p[5]);
    std::vector<int32_t> prev(nc, INT32_MIN);
    st = copy_in(ctx, s->d_offs, offs.data(), 8 * (n + 1), 0);
    if (st == FEM_OK && n_nodes > 0) st = copy_in(ctx, s->d_types, ty.data(), 2 * n_nodes, 0);
    if (st == FEM_OK && n_edges > 0) st = copy_in(ctx, s->d_lo, lo.data(), 4 * n_edges, 0);
    if (st == FEM_OK && n_edges > 0) st = copy_in(ctx, s->d_hi, hi.data(), 4 * n_edges, 0);
    if (st == FEM_OK) st = copy_in(ctx, s->d_prev, prev.data(), 4 * nc, 0);
    if (st == FEM_OK && cudaMemsetAsync(s->d_counts, 0, 4 * nc, ctx->stream) != cudaSuccess) st = FEM_ERR_CUDA;
    if (st == FEM_OK && cudaStreamSynchronize(ctx->stream) != cudaSuccess) st = FEM_ERR_CUDA;
    if (st != FEM_OK) {
        session_free_buffers(s);
        delete s;
        return st;
    }
    *out = s;
    return FEM_OK;
}

extern "C" int fem_session_append(fem_session *s, const uint16_t *types, const int32_t *times, int64_t n,
                                  int ptr_is_device) {
    if (!s || n < 0 || (n > 0 && (!types || !times))) return FEM_ERR_INVAL;
    if (n == 0) return FEM_OK;
    fem_ctx *ctx = s->ctx;
    std::lock_guard<std::mutex> g(ctx->mu);
    if (s->n_tail + n > INT32_MAX / 2) return FEM_ERR_INVAL;
    cudaSetDevice(ctx->device);
    const double t0 = now_s();
    cudaStream_t st = ctx->stream;
    const int64_t m = s->n_tail + n;
    // tail followed by the new events, validated as one recording (order and
    // repeated (type, time) pairs across the join included)
    fem_stream *fs = nullptr;
    {
        TmpDev tmp(ctx);
        uint16_t *bt;
        int32_t *bm;
        FEM_TRY(tmp.get(&bt, m));
        FEM_TRY(tmp.get(&bm, m));
        if (s->n_tail > 0) {
            FEM_CUDA_TRY(cudaMemcpyAsync(bt, s->d_tail_type, 2 * s->n_tail, cudaMemcpyDeviceToDevice, st));
            FEM_CUDA_TRY(cudaMemcpyAsync(bm, s->d_tail_time, 4 * s->n_tail, cudaMemcpyDeviceToDevice, st));
        }
        FEM_TRY(copy_in(ctx, bt + s->n_tail, types, 2 * n, ptr_is_device));
        FEM_TRY(copy_in(ctx, bm + s->n_tail, times, 4 * n, ptr_is_device));
        FEM_TRY(load_stream_unlocked(ctx, bt, bm, m, s->n_types, 1, &fs));
    }
    fem_stats stats{};
    float ms = 0.f;
    int rc = FEM_OK;
    if (s->n_cand > 0) {
        std::vector<int32_t> work(s->n_cand);
        for (int64_t i = 0; i < s->n_cand; ++i) work[i] = (int32_t)i;
        PltSession ps{&s->tail_cnt, s->d_prev};
        std::vector<fem_stream *> recs{fs};
        rc = count_plt(ctx, recs, s->d_offs, s->d_types, s->d_lo, s->d_hi, nullptr, work, false, s->d_counts, &stats,
                       &ms, 0, &ps);
    }
    // the new tail: events at or after t_last - max sum(hi)
    int64_t cut_idx = 0;
    std::vector<unsigned long long> h(s->n_types, 0);
    if (rc == FEM_OK) {
        TmpDev tmp(ctx);
        int64_t *d_idx;
        unsigned long long *d_h;
        rc = tmp.get(&d_idx, 1);
        if (rc == FEM_OK) rc = tmp.get(&d_h, s->n_types);
        if (rc == FEM_OK) {
            k_lower_bound<<<1, 1, 0, st>>>(fs->d_time, m, (int64_t)fs->t_last - s->span_max, d_idx);
            if (cudaMemcpyAsync(&cut_idx, d_idx, 8, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
                cudaStreamSynchronize(st) != cudaSuccess)
                rc = FEM_ERR_CUDA;
        }
        const int64_t nt = m - cut_idx;
        if (rc == FEM_OK && nt > s->tail_cap) {
            const int64_t cap = std::max<int64_t>(nt, 2 * s->tail_cap);
            void *p1 = nullptr, *p2 = nullptr;
            rc = dev_alloc(ctx, &p1, 2 * cap);
            if (rc == FEM_OK) {
                rc = dev_alloc(ctx, &p2, 4 * cap);
                if (rc != FEM_OK) dev_free(ctx, p1, 2 * cap);
            }
            if (rc == FEM_OK) {
                cudaStreamSynchronize(st);
                if (s->tail_cap) {
                    dev_free(ctx, s->d_tail_type, 2 * s->tail_cap);
                    dev_free(ctx, s->d_tail_time, 4 * s->tail_cap);
                }
                s->d_tail_type = static_cast<uint16_t *>(p1);
                s->d_tail_time = static_cast<int32_t *>(p2);
                s->tail_cap = cap;
            }
        }
        if (rc == FEM_OK) {
            cudaMemsetAsync(d_h, 0, 8 * s->n_types, st);
            cudaMemcpyAsync(s->d_tail_type, fs->d_type + cut_idx, 2 * nt, cudaMemcpyDeviceToDevice, st);
            cudaMemcpyAsync(s->d_tail_time, fs->d_time + cut_idx, 4 * nt, cudaMemcpyDeviceToDevice, st);
            if (nt > 0) {
                const unsigned gsz = (unsigned)std::max<int64_t>(1, std::min<int64_t>((nt + 255) / 256, 4 * ctx->n_sm));
                k_type_hist<<<gsz, 256, 0, st>>>(s->d_tail_type, nt, d_h);
            }
            if (cudaGetLastError() != cudaSuccess ||
                cudaMemcpyAsync(h.data(), d_h, 8 * s->n_types, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
                cudaStreamSynchronize(st) != cudaSuccess)
                rc = FEM_ERR_CUDA;
            else
                s->n_tail = nt;
        }
    }
    stream_free_unlocked(fs);
    // A failure after counting leaves the session unusable for exact counts:
    // the caller gets the error and should recreate it.
    if (rc != FEM_OK) return rc;
    for (uint32_t a = 0; a < s->n_types; ++a) s->tail_cnt[a] = (int64_t)h[a];
    s->seen += n;
    stats.kernel_launches += 2;
    stats.count_kernel_ms = ms;
    stats.total_ms = (now_s() - t0) * 1e3;
    ctx->last = stats;
    return FEM_OK;
}

extern "C" int fem_session_counts(fem_session *s, uint32_t *counts, int out_is_device) {
    if (!s || (s->n_cand > 0 && !counts)) return FEM_ERR_INVAL;
    if (s->n_cand == 0) return FEM_OK;
    fem_ctx *ctx = s->ctx;
    std::lock_guard<std::mutex> g(ctx->mu);
    cudaSetDevice(ctx->device);
    FEM_TRY(copy_out(ctx, counts, s->d_counts, 4 * s->n_cand, out_is_device));
    FEM_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
    return FEM_OK;
}

extern "C" int fem_session_info(const fem_session *s, int64_t *events_seen, int64_t *tail_events) {
    if (!s) return FEM_ERR_INVAL;
    if (events_seen) *events_seen = s->seen;
    if (tail_events) *tail_events = s->n_tail;
    return FEM_OK;
}

extern "C" void fem_session_destroy(fem_session *s) {
    if (!s) return;
    fem_ctx *ctx = s->ctx;
    {
        std::lock_guard<std::mutex> g(ctx->mu);
        cudaSetDevice(ctx->device);
        cudaStreamSynchronize(ctx->stream);
        session_free_buffers(s);
    }
    delete s;
}
