// fem_core.cu -- context, device memory, stream store (load, validation,
// level-1 counts) and the window-density tables that size the per-node rings.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <fstream>
#include <sstream>

#include "fem_internal.cuh"

namespace fem {

double now_s() {
    using namespace std::chrono;
    return duration<double>(steady_clock::now().time_since_epoch()).count();
}

static int ilog2_ceil(int64_t v) {
    int k = 0;
    while (((int64_t)1 << k) < v && k < 62) ++k;
    return k;
}

std::string tune_key(int nclass, int rclass, int64_t n_slots, int64_t n_events, int n_recs) {
    char buf[96];
    std::snprintf(buf, sizeof buf, "n%d.r%d.c%d.e%d.m%d", nclass, rclass, ilog2_ceil(n_slots),
                  ilog2_ceil(n_events), n_recs > 1 ? 2 : 1);
    return buf;
}

bool tune_lookup(fem_ctx *ctx, const std::string &key, TuneVal *out) {
    auto it = ctx->tune.find(key);
    if (it == ctx->tune.end()) return false;
    *out = it->second;
    return true;
}

static void tune_save(fem_ctx *ctx) {
    if (ctx->tune_path.empty()) return;
    const std::string tmp = ctx->tune_path + ".tmp";
    {
        std::ofstream f(tmp);
        if (!f) return;
        f << "{\n";
        size_t i = 0;
        for (auto &kv : ctx->tune) {
            f << "  \"" << kv.first << "\": [" << kv.second.K << ", " << kv.second.T << ", " << kv.second.seg_mult
              << ", " << kv.second.kernel << "]" << (++i < ctx->tune.size() ? "," : "") << "\n";
        }
        f << "}\n";
    }
    std::rename(tmp.c_str(), ctx->tune_path.c_str());
}

void tune_store(fem_ctx *ctx, const std::string &key, const TuneVal &v) {
    ctx->tune[key] = v;
    tune_save(ctx);
}

// Parses {"key": [K, T, m], ...}; returns false on malformed text.
static bool tune_parse(const std::string &text, std::map<std::string, TuneVal> *out) {
    size_t i = text.find('{');
    if (i == std::string::npos) return false;
    for (;;) {
        const size_t q0 = text.find('"', i);
        if (q0 == std::string::npos) break;
        const size_t q1 = text.find('"', q0 + 1);
        const size_t b0 = text.find('[', q1);
        const size_t b1 = text.find(']', b0);
        if (q1 == std::string::npos || b0 == std::string::npos || b1 == std::string::npos) return false;
        TuneVal v{};
        v.kernel = 1;
        const int got = std::sscanf(text.substr(b0 + 1, b1 - b0 - 1).c_str(), "%d , %d , %lf , %d", &v.K, &v.T,
                                    &v.seg_mult, &v.kernel);
        if (got < 3 || v.kernel < 1 || v.kernel > 3) return false;
        if (v.K < 32 || v.K > kMaxWarps * 32 || v.K % 32 || v.T < 256 || v.T > kMaxTile || v.T % 256 ||
            !(v.seg_mult > 0.0 && v.seg_mult < 64.0))
            return false;
        (*out)[text.substr(q0 + 1, q1 - q0 - 1)] = v;
        i = b1 + 1;
    }
    return true;
}

// Device allocations go through a per-context cache of freed blocks: a
// request takes the smallest cached block of at least its size (and at most
// 1.25x + 64 KB of it), else cudaMalloc; a free parks the block in the cache
// while the cache stays below a quarter of the budget (at most 8 GB).  A
// failed cudaMalloc releases the cache and retries once.  `used` counts the
// blocks in use against the context's budget.
static size_t pool_limit(const fem_ctx *ctx) { return std::min<size_t>(ctx->budget / 4, (size_t)8 << 30); }

void pool_release(fem_ctx *ctx) {
    std::lock_guard<std::mutex> g(ctx->pool_mu);
    for (auto &kv : ctx->cached) cudaFree(kv.second);
    ctx->cached.clear();
    ctx->cached_bytes = 0;
}

int dev_alloc(fem_ctx *ctx, void **p, size_t bytes) {
    *p = nullptr;
    if (bytes == 0) bytes = 16;
    bytes = (bytes + 255) & ~size_t(255);
    if (ctx->used.load() + bytes > ctx->budget) return FEM_ERR_NOMEM;
    {
        std::lock_guard<std::mutex> g(ctx->pool_mu);
        auto it = ctx->cached.lower_bound(bytes);
        if (it != ctx->cached.end() && it->first <= bytes + bytes / 4 + (64 << 10)) {
            *p = it->second;
            const size_t sz = it->first;
            ctx->cached_bytes -= sz;
            ctx->cached.erase(it);
            ctx->live[*p] = sz;
            ctx->used += sz;
            return FEM_OK;
        }
    }
    cudaError_t e = cudaMalloc(p, bytes);
    if (e == cudaErrorMemoryAllocation) {
        cudaGetLastError();
        pool_release(ctx);
        e = cudaMalloc(p, bytes);
    }
    if (e != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        return e == cudaErrorMemoryAllocation ? FEM_ERR_NOMEM : FEM_ERR_CUDA;
    }
    std::lock_guard<std::mutex> g(ctx->pool_mu);
    ctx->live[*p] = bytes;
    ctx->used += bytes;
    return FEM_OK;
}

void dev_free(fem_ctx *ctx, void *p, size_t bytes) {
    if (!p) return;
    std::lock_guard<std::mutex> g(ctx->pool_mu);
    auto it = ctx->live.find(p);
    size_t sz = (bytes == 0 ? 16 : (bytes + 255) & ~size_t(255));
    if (it != ctx->live.end()) {
        sz = it->second;
        ctx->live.erase(it);
    }
    ctx->used -= sz;
    if (ctx->cached_bytes + sz <= pool_limit(ctx)) {
        ctx->cached.emplace(sz, p);
        ctx->cached_bytes += sz;
    } else {
        cudaFree(p);
    }
}

int scratch(fem_ctx *ctx, int slot, size_t bytes, void **p) {
    DevBuf &b = ctx->scratch[slot];
    if (b.cap >= bytes && b.p) {
        *p = b.p;
        return FEM_OK;
    }
    size_t want = std::max(bytes, b.cap + b.cap / 2);
    want = std::max<size_t>(want, 4096);
    if (b.p) {
        cudaStreamSynchronize(ctx->stream);
        dev_free(ctx, b.p, b.cap);
        b.p = nullptr;
        b.cap = 0;
    }
    int st = dev_alloc(ctx, &b.p, want);
    if (st != FEM_OK && want > bytes) st = dev_alloc(ctx, &b.p, bytes), want = bytes;
    if (st != FEM_OK) return st;
    b.cap = want;
    *p = b.p;
    return FEM_OK;
}

int sync_status(fem_ctx *ctx) {
    FEM_CUDA_TRY(cudaMemcpyAsync(ctx->h_status, ctx->d_status, sizeof(int), cudaMemcpyDeviceToHost,
                                 ctx->stream));
    FEM_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
    int s = *ctx->h_status;
    if (s) {
        FEM_CUDA_TRY(cudaMemsetAsync(ctx->d_status, 0, sizeof(int), ctx->stream));
        if (s & kStatusTimeout) return FEM_ERR_TIMEOUT;
        if (s & kStatusInval) return FEM_ERR_INVAL;
    }
    return FEM_OK;
}

int copy_in(fem_ctx *ctx, void *dst_dev, const void *src, size_t bytes, int src_is_device) {
    if (bytes == 0) return FEM_OK;
    FEM_CUDA_TRY(cudaMemcpyAsync(dst_dev, src, bytes,
                                 src_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                                 ctx->stream));
    return FEM_OK;
}

int copy_out(fem_ctx *ctx, void *dst, const void *src_dev, size_t bytes, int dst_is_device) {
    if (bytes == 0) return FEM_OK;
    FEM_CUDA_TRY(cudaMemcpyAsync(dst, src_dev, bytes,
                                 dst_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                                 ctx->stream));
    return FEM_OK;
}

// ---------------------------------------------------------------------------
// Stream validation (Definition 1 plus the library's input rules): type in
// range, time >= 0, times non-decreasing, no repeated (type, time).  A
// repeated pair must sit inside one run of equal times, so each event looks
// back only while the time is unchanged.
__global__ void k_validate(const uint16_t *__restrict__ ty, const int32_t *__restrict__ tm, int64_t n,
                           uint32_t n_types, int *err) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    int e = 0;
    for (; i < n; i += stride) {
        const uint16_t a = ty[i];
        const int32_t t = tm[i];
        if (a >= n_types) e |= 1;
        if (t < 0 || t == INT32_MAX) e |= 2;
        if (i > 0) {
            const int32_t tp = tm[i - 1];
            if (tp > t) e |= 4;
            for (int64_t j = i - 1; j >= 0 && tm[j] == t; --j)
                if (ty[j] == a) {
                    e |= 8;
                    break;
                }
        }
    }
    if (e) atomicOr(err, e);
}

// Level 1 (a 1-node episode's count is its frequency): per-type histogram,
// privatised in shared memory when the alphabet fits.  It runs before the
// host has read the validation result, so out-of-range types are skipped.
__global__ void k_histogram(const uint16_t *__restrict__ ty, int64_t n, uint32_t n_types,
                            uint32_t *__restrict__ freq) {
    extern __shared__ uint32_t h[];
    const bool priv = n_types <= 12288;
    if (priv)
        for (uint32_t a = threadIdx.x; a < n_types; a += blockDim.x) h[a] = 0;
    __syncthreads();
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const uint16_t a = ty[i];
        if (a >= n_types) continue;
        if (priv)
            atomicAdd(&h[a], 1u);
        else
            atomicAdd(&freq[a], 1u);
    }
    __syncthreads();
    if (priv)
        for (uint32_t a = threadIdx.x; a < n_types; a += blockDim.x)
            if (h[a]) atomicAdd(&freq[a], h[a]);
}

__global__ void k_fill_pad(uint16_t *ty, int32_t *tm, int64_t from, int64_t to) {
    for (int64_t i = from + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < to;
         i += (int64_t)gridDim.x * blockDim.x) {
        ty[i] = 0xFFFF;
        tm[i] = INT32_MAX;
    }
}

// Window density: dens[a] = largest number of type-a events inside any closed
// window [t - lo, t].  With at most dens[E_k] entries of node k still inside
// their lower bound, a ring of dens + 1 entries always holds the newest entry
// that is past its lower bound (the only one a query needs).  Each event scans
// back while the window lasts; after `cap` steps the type is marked unknown
// (the caller then falls back to the type's frequency, also an upper bound).
__global__ void k_density(const uint16_t *__restrict__ ty, const int32_t *__restrict__ tm, int64_t n,
                          int32_t lo, int cap, uint32_t *__restrict__ dens) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const uint16_t a = ty[i];
        const int64_t lim = (int64_t)tm[i] - lo;
        uint32_t c = 1;
        int steps = 0;
        int64_t j = i - 1;
        for (; j >= 0 && tm[j] >= lim && steps < cap; --j, ++steps)
            if (ty[j] == a) ++c;
        if (j >= 0 && tm[j] >= lim) c = kDensUnknown;
        atomicMax(&dens[a], c);
    }
}

__global__ void k_density_resolve(uint32_t *dens, const uint32_t *freq, uint32_t n_types) {
    for (uint32_t a = blockIdx.x * blockDim.x + threadIdx.x; a < n_types; a += gridDim.x * blockDim.x)
        if (dens[a] == kDensUnknown) dens[a] = freq[a];
}

// Window densities for up to kDensLo lower bounds at once, from the per-type
// lists: event i of type a sees the type-a events in [t_i - lo, t_i] by
// scanning back over a's list only; dens[j][a] = the largest such number
// (kDensUnknown after `cap` steps).  Each thread walks a run of kDensRun
// consecutive list positions (mostly one type) and writes its running
// maxima only when the type changes, so a type's counter sees few atomics.
constexpr int kDensLo = 8;
constexpr int kDensRun = 16;

__global__ void k_density_lists(const int64_t *__restrict__ toff, const int32_t *__restrict__ ttime,
                                uint32_t n_types, int64_t n, const int32_t *__restrict__ los, int n_lo, int cap,
                                uint32_t *const *dens) {
    int32_t lo_v[kDensLo];
#pragma unroll
    for (int k = 0; k < kDensLo; ++k) lo_v[k] = k < n_lo ? los[k] : 0;
    int32_t lo_max = 0;
#pragma unroll
    for (int k = 0; k < kDensLo; ++k) lo_max = max(lo_max, lo_v[k]);
    const int64_t runs = (n + kDensRun - 1) / kDensRun;
    for (int64_t run = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; run < runs;
         run += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i0 = run * kDensRun, i1 = min(n, i0 + kDensRun);
        int lo = 0, hi = (int)n_types;  // type of position i0: toff[a] <= i0 < toff[a + 1]
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (toff[mid] <= i0) lo = mid; else hi = mid;
        }
        int a = lo;
        int64_t b0 = toff[a], b1 = toff[a + 1];
        uint32_t best[kDensLo];
#pragma unroll
        for (int k = 0; k < kDensLo; ++k) best[k] = 0;
        for (int64_t i = i0; i < i1; ++i) {
            while (i >= b1) {  // next type: write this one's maxima
#pragma unroll
                for (int k = 0; k < kDensLo; ++k)
                    if (k < n_lo && best[k]) atomicMax(&dens[k][a], best[k]), best[k] = 0;
                ++a;
                b0 = b1;
                b1 = toff[a + 1];
            }
            const int64_t t = ttime[i];
            uint32_t c[kDensLo];
#pragma unroll
            for (int k = 0; k < kDensLo; ++k) c[k] = 1;
            int64_t j = i - 1;
            int steps = 0;
            for (; j >= b0 && (int64_t)ttime[j] >= t - lo_max && steps < cap; --j, ++steps) {
#pragma unroll
                for (int k = 0; k < kDensLo; ++k)
                    if ((int64_t)ttime[j] >= t - lo_v[k]) c[k] += 1;
            }
            const bool more = j >= b0;
#pragma unroll
            for (int k = 0; k < kDensLo; ++k) {
                const bool unknown = more && (int64_t)ttime[j] >= t - lo_v[k];
                best[k] = max(best[k], unknown ? kDensUnknown : c[k]);
            }
        }
#pragma unroll
        for (int k = 0; k < kDensLo; ++k)
            if (k < n_lo && best[k]) atomicMax(&dens[k][a], best[k]);
    }
}

int stream_densities(fem_ctx *ctx, fem_stream *s, const std::vector<int32_t> &los) {
    std::vector<int32_t> miss;
    for (int32_t l : los)
        if (!s->dens.count(l) && std::find(miss.begin(), miss.end(), l) == miss.end()) miss.push_back(l);
    if (miss.empty() || s->n == 0) return FEM_OK;
    if (stream_bytype(ctx, s) != FEM_OK) return FEM_OK;  // stream_density computes them one by one
    for (size_t g0 = 0; g0 < miss.size(); g0 += kDensLo) {
        const int m = (int)std::min<size_t>(kDensLo, miss.size() - g0);
        std::vector<uint32_t *> outs(m, nullptr);
        for (int k = 0; k < m; ++k) {
            void *p = nullptr;
            const int st = dev_alloc(ctx, &p, sizeof(uint32_t) * s->n_types);
            if (st != FEM_OK) {
                for (int q = 0; q < k; ++q) dev_free(ctx, outs[q], sizeof(uint32_t) * s->n_types);
                return st;
            }
            outs[k] = static_cast<uint32_t *>(p);
            FEM_CUDA_TRY(cudaMemsetAsync(p, 0, sizeof(uint32_t) * s->n_types, ctx->stream));
        }
        struct {
            int32_t lo[kDensLo];
            uint32_t *d[kDensLo];
        } hb{};
        for (int k = 0; k < m; ++k) {
            hb.lo[k] = miss[g0 + k];
            hb.d[k] = outs[k];
        }
        void *pb = nullptr;
        FEM_TRY(scratch(ctx, kSlotDensArgs, sizeof(hb), &pb));
        FEM_CUDA_TRY(cudaMemcpyAsync(pb, &hb, sizeof(hb), cudaMemcpyHostToDevice, ctx->stream));
        const auto *db = static_cast<const char *>(pb);
        const int64_t runs = (s->n + kDensRun - 1) / kDensRun;
        k_density_lists<<<(unsigned)std::max<int64_t>(1, std::min<int64_t>((runs + 255) / 256, 8 * ctx->n_sm)), 256,
                          0, ctx->stream>>>(s->d_toff, s->d_ttime, s->n_types, s->n,
                                            reinterpret_cast<const int32_t *>(db),
                                            m, 4096, reinterpret_cast<uint32_t *const *>(db + sizeof(hb.lo)));
        for (int k = 0; k < m; ++k)
            k_density_resolve<<<(s->n_types + 255) / 256, 256, 0, ctx->stream>>>(outs[k], s->d_freq, s->n_types);
        FEM_CUDA_TRY(cudaGetLastError());
        // the argument block is reused by the next group: wait for this one
        if (g0 + kDensLo < miss.size()) FEM_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
        for (int k = 0; k < m; ++k) {
            s->dens[miss[g0 + k]] = outs[k];
            s->bytes += sizeof(uint32_t) * s->n_types;
        }
    }
    return FEM_OK;
}

int stream_density(fem_ctx *ctx, fem_stream *s, int32_t lo, uint32_t **d_dens) {
    auto it = s->dens.find(lo);
    if (it != s->dens.end()) {
        *d_dens = it->second;
        return FEM_OK;
    }
    void *p = nullptr;
    FEM_TRY(dev_alloc(ctx, &p, sizeof(uint32_t) * s->n_types));
    uint32_t *d = static_cast<uint32_t *>(p);
    FEM_CUDA_TRY(cudaMemsetAsync(d, 0, sizeof(uint32_t) * s->n_types, ctx->stream));
    if (s->n > 0) {
        if (lo == 0) {
            // distinct (type, time): a window of length 0 holds one event of a type
            k_density<<<std::max<int64_t>(1, std::min<int64_t>((s->n + 255) / 256, 4096)), 256, 0,
                        ctx->stream>>>(s->d_type, s->d_time, s->n, 0, 1 << 20, d);
        } else {
            k_density<<<std::max<int64_t>(1, std::min<int64_t>((s->n + 255) / 256, 65536)), 256, 0,
                        ctx->stream>>>(s->d_type, s->d_time, s->n, lo, 4096, d);
        }
        k_density_resolve<<<(s->n_types + 255) / 256, 256, 0, ctx->stream>>>(d, s->d_freq, s->n_types);
        FEM_CUDA_TRY(cudaGetLastError());
    }
    s->dens[lo] = d;
    s->bytes += sizeof(uint32_t) * s->n_types;
    *d_dens = d;
    return FEM_OK;
}

}  // namespace fem

using namespace fem;

// ---------------------------------------------------------------------------
// C ABI: context.
extern "C" int fem_ctx_create(int device, size_t hbm_budget_bytes, void *cuda_stream, fem_ctx **out) {
    if (!out) return FEM_ERR_INVAL;
    *out = nullptr;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess) {
        cudaGetLastError();
        return FEM_ERR_CUDA;
    }
    if (device < 0 || device >= ndev) return FEM_ERR_INVAL;
    FEM_CUDA_TRY(cudaSetDevice(device));
    fem_ctx *ctx = new (std::nothrow) fem_ctx();
    if (!ctx) return FEM_ERR_NOMEM;
    ctx->device = device;
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, device) != cudaSuccess) {
        delete ctx;
        return FEM_ERR_CUDA;
    }
    ctx->n_sm = prop.multiProcessorCount;
    ctx->smem_optin = (int)prop.sharedMemPerBlockOptin;
    size_t fr = 0, tot = 0;
    cudaMemGetInfo(&fr, &tot);
    ctx->budget = hbm_budget_bytes ? hbm_budget_bytes : (size_t)(0.9 * (double)fr);
    if (cuda_stream) {
        ctx->stream = static_cast<cudaStream_t>(cuda_stream);
    } else {
        if (cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking) != cudaSuccess) {
            delete ctx;
            return FEM_ERR_CUDA;
        }
        ctx->own_stream = true;
    }
    void *p = nullptr;
    int st = dev_alloc(ctx, &p, sizeof(int) * 4);
    if (st != FEM_OK) {
        if (ctx->own_stream) cudaStreamDestroy(ctx->stream);
        delete ctx;
        return st;
    }
    ctx->d_status = static_cast<int *>(p);
    cudaMemsetAsync(ctx->d_status, 0, sizeof(int) * 4, ctx->stream);
    if (cudaMallocHost(&ctx->h_status, sizeof(int) * 4) != cudaSuccess) {
        dev_free(ctx, ctx->d_status, sizeof(int) * 4);
        if (ctx->own_stream) cudaStreamDestroy(ctx->stream);
        delete ctx;
        return FEM_ERR_CUDA;
    }
    cudaEventCreate(&ctx->ev0);
    cudaEventCreate(&ctx->ev1);
    cudaStreamSynchronize(ctx->stream);
    *out = ctx;
    return FEM_OK;
}

extern "C" void fem_ctx_destroy(fem_ctx *ctx) {
    if (!ctx) return;
    cudaSetDevice(ctx->device);
    cudaStreamSynchronize(ctx->stream);
    graph_cache_clear(ctx);
    if (ctx->pinned) cudaFreeHost(ctx->pinned);
    ctx->pinned = nullptr;
    for (auto &kv : ctx->scratch) dev_free(ctx, kv.second.p, kv.second.cap);
    ctx->scratch.clear();
    dev_free(ctx, ctx->d_status, sizeof(int) * 4);
    pool_release(ctx);
    for (auto &kv : ctx->live) cudaFree(kv.first);
    ctx->live.clear();
    if (ctx->h_status) cudaFreeHost(ctx->h_status);
    if (ctx->ev0) cudaEventDestroy(ctx->ev0);
    if (ctx->ev1) cudaEventDestroy(ctx->ev1);
    if (ctx->own_stream) cudaStreamDestroy(ctx->stream);
    delete ctx;
}

extern "C" int fem_ctx_set_tuning(fem_ctx *ctx, const fem_tuning *t) {
    if (!ctx) return FEM_ERR_INVAL;
    std::lock_guard<std::mutex> g(ctx->mu);
    if (!t) {
        ctx->tuning = fem_tuning{};
        return FEM_OK;
    }
    if (t->lanes_per_cta < 0 || (t->lanes_per_cta % 32) != 0 || t->lanes_per_cta > kMaxWarps * 32)
        return FEM_ERR_INVAL;
    if (t->segments < 0 || t->tile_events < 0 || (t->tile_events % 256) != 0 ||
        t->tile_events > kMaxTile || t->kernel < 0 || t->kernel > 7 || t->wait_polls < 0 ||
        t->track_last < 0 || t->track_last > 2 || t->prepass < -1 || t->prepass > 2)
        return FEM_ERR_INVAL;
    ctx->tuning = *t;
    return FEM_OK;
}

extern "C" int fem_ctx_set_autotune_cache(fem_ctx *ctx, const char *path) {
    if (!ctx) return FEM_ERR_INVAL;
    std::lock_guard<std::mutex> g(ctx->mu);
    if (!path) {
        ctx->tune_path.clear();
        return FEM_OK;
    }
    std::ifstream f(path);
    if (f) {
        std::stringstream ss;
        ss << f.rdbuf();
        std::map<std::string, TuneVal> m;
        if (!tune_parse(ss.str(), &m)) return FEM_ERR_INVAL;
        for (auto &kv : m) ctx->tune[kv.first] = kv.second;
    }
    ctx->tune_path = path;
    tune_save(ctx);
    return FEM_OK;
}

extern "C" int fem_ctx_last_stats(const fem_ctx *ctx, fem_stats *out) {
    if (!ctx || !out) return FEM_ERR_INVAL;
    *out = ctx->last;
    return FEM_OK;
}

extern "C" int fem_ctx_memory(const fem_ctx *ctx, size_t *used, size_t *budget) {
    if (!ctx) return FEM_ERR_INVAL;
    if (used) *used = ctx->used.load();
    if (budget) *budget = ctx->budget;
    return FEM_OK;
}

// ---------------------------------------------------------------------------
// C ABI: streams.
int fem::load_stream_unlocked(fem_ctx *ctx, const uint16_t *types, const int32_t *times, int64_t n,
                              uint32_t n_types, int ptr_is_device, fem_stream **out) {
    if (!ctx || !out || n < 0 || n_types < 1 || n_types > 65536) return FEM_ERR_INVAL;
    if (n > 0 && (!types || !times)) return FEM_ERR_INVAL;
    if (n > (int64_t)INT32_MAX * 4) return FEM_ERR_INVAL;
    *out = nullptr;
    cudaSetDevice(ctx->device);
    fem_stream *s = new (std::nothrow) fem_stream();
    if (!s) return FEM_ERR_NOMEM;
    s->ctx = ctx;
    s->n = n;
    s->n_types = n_types;
    const int64_t cap = n + kPadEvents;
    void *p1 = nullptr, *p2 = nullptr, *p3 = nullptr;
    int st = dev_alloc(ctx, &p1, sizeof(uint16_t) * cap);
    if (st == FEM_OK) st = dev_alloc(ctx, &p2, sizeof(int32_t) * cap);
    if (st == FEM_OK) st = dev_alloc(ctx, &p3, sizeof(uint32_t) * n_types);
    auto fail = [&](int code) {
        cudaStreamSynchronize(ctx->stream);
        dev_free(ctx, p1, sizeof(uint16_t) * cap);
        dev_free(ctx, p2, sizeof(int32_t) * cap);
        dev_free(ctx, p3, sizeof(uint32_t) * n_types);
        delete s;
        return code;
    };
    if (st != FEM_OK) return fail(st);
    s->d_type = static_cast<uint16_t *>(p1);
    s->d_time = static_cast<int32_t *>(p2);
    s->d_freq = static_cast<uint32_t *>(p3);
    s->bytes = (sizeof(uint16_t) + sizeof(int32_t)) * cap + sizeof(uint32_t) * n_types;
    if (copy_in(ctx, s->d_type, types, sizeof(uint16_t) * n, ptr_is_device) != FEM_OK ||
        copy_in(ctx, s->d_time, times, sizeof(int32_t) * n, ptr_is_device) != FEM_OK)
        return fail(FEM_ERR_CUDA);
    k_fill_pad<<<64, 256, 0, ctx->stream>>>(s->d_type, s->d_time, n, cap);
    cudaMemsetAsync(s->d_freq, 0, sizeof(uint32_t) * n_types, ctx->stream);
    cudaMemsetAsync(ctx->d_status + 1, 0, sizeof(int), ctx->stream);
    if (n > 0) {
        const int blocks = (int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, ctx->n_sm * 8));
        k_validate<<<blocks, 256, 0, ctx->stream>>>(s->d_type, s->d_time, n, n_types, ctx->d_status + 1);
        const size_t hs = n_types <= 12288 ? n_types * sizeof(uint32_t) : 0;
        k_histogram<<<blocks, 256, hs, ctx->stream>>>(s->d_type, n, n_types, s->d_freq);
    }
    if (cudaGetLastError() != cudaSuccess) return fail(FEM_ERR_CUDA);
    if (cudaMemcpyAsync(ctx->h_status + 1, ctx->d_status + 1, sizeof(int), cudaMemcpyDeviceToHost,
                        ctx->stream) != cudaSuccess ||
        cudaStreamSynchronize(ctx->stream) != cudaSuccess)
        return fail(FEM_ERR_CUDA);
    const int e = ctx->h_status[1];
    if (n > 0 && e == 0) {
        int32_t tt[2] = {0, 0};
        if (cudaMemcpy(&tt[0], s->d_time, 4, cudaMemcpyDeviceToHost) != cudaSuccess ||
            cudaMemcpy(&tt[1], s->d_time + n - 1, 4, cudaMemcpyDeviceToHost) != cudaSuccess)
            return fail(FEM_ERR_CUDA);
        s->t_first = tt[0];
        s->t_last = tt[1];
    }
    if (e & 1) return fail(FEM_ERR_INVAL);
    if (e & 2) return fail(FEM_ERR_RANGE);
    if (e & 4) return fail(FEM_ERR_UNSORTED);
    if (e & 8) return fail(FEM_ERR_DUP);
    *out = s;
    return FEM_OK;
}

extern "C" int fem_load_stream(fem_ctx *ctx, const uint16_t *types, const int32_t *times, int64_t n,
                               uint32_t n_types, int ptr_is_device, fem_stream **out) {
    if (!ctx) return FEM_ERR_INVAL;
    std::lock_guard<std::mutex> g(ctx->mu);
    return load_stream_unlocked(ctx, types, times, n, n_types, ptr_is_device, out);
}

extern "C" void fem_stream_free(fem_stream *s) {
    if (!s) return;
    std::lock_guard<std::mutex> g(s->ctx->mu);
    stream_free_unlocked(s);
}

void fem::stream_free_unlocked(fem_stream *s) {
    if (!s) return;
    fem_ctx *ctx = s->ctx;
    cudaSetDevice(ctx->device);
    graph_cache_forget(ctx, s);
    cudaStreamSynchronize(ctx->stream);
    const int64_t cap = s->n + kPadEvents;
    dev_free(ctx, s->d_type, sizeof(uint16_t) * cap);
    dev_free(ctx, s->d_time, sizeof(int32_t) * cap);
    dev_free(ctx, s->d_freq, sizeof(uint32_t) * s->n_types);
    for (auto &kv : s->dens) dev_free(ctx, kv.second, sizeof(uint32_t) * s->n_types);
    for (auto &kv : s->segs) dev_free(ctx, kv.second, sizeof(int64_t) * (kv.first + 1));
    coarse_free(ctx, s);
    if (s->d_toff) dev_free(ctx, s->d_toff, sizeof(int64_t) * (s->n_types + 1));
    if (s->d_ttime) dev_free(ctx, s->d_ttime, sizeof(int32_t) * std::max<int64_t>(s->n, 1));
    if (s->d_tidx) dev_free(ctx, s->d_tidx, sizeof(int32_t) * (size_t)s->n_types * (size_t)(s->tcells + 1));
    delete s;
}

extern "C" int fem_stream_info(const fem_stream *s, int64_t *n, uint32_t *n_types) {
    if (!s) return FEM_ERR_INVAL;
    if (n) *n = s->n;
    if (n_types) *n_types = s->n_types;
    return FEM_OK;
}

extern "C" int fem_stream_freq(fem_ctx *ctx, const fem_stream *s, uint32_t *freq, int out_is_device) {
    if (!ctx || !s || !freq || s->ctx != ctx) return FEM_ERR_INVAL;
    std::lock_guard<std::mutex> g(ctx->mu);
    cudaSetDevice(ctx->device);
    FEM_TRY(copy_out(ctx, freq, s->d_freq, sizeof(uint32_t) * s->n_types, out_is_device));
    FEM_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
    return FEM_OK;
}

extern "C" const char *fem_strerror(int status) {
    switch (status) {
        case FEM_OK: return "ok";
        case FEM_ERR_INVAL: return "invalid argument";
        case FEM_ERR_UNSORTED: return "stream times are not non-decreasing";
        case FEM_ERR_DUP: return "stream repeats a (type, time) event";
        case FEM_ERR_RANGE: return "time out of range (negative or INT32_MAX)";
        case FEM_ERR_NOMEM: return "device memory budget exceeded";
        case FEM_ERR_TIMEOUT: return "device-side wait timed out";
        case FEM_ERR_CUDA: return "CUDA runtime error";
        case FEM_ERR_BUSY: return "busy (queue full or job not finished)";
        case FEM_ERR_NOTFOUND: return "unknown job id";
        default: return "unknown status";
    }
}

extern "C" const char *fem_version(void) { return "fem 0.1.0 sm_103a"; }
