// fem_bound.cu -- coarse-tick upper bound on the count (a cheaper pre-pass).
//
// Pruning ("Temporal Data Mining") drops a candidate whose count cannot pass
// the threshold without counting it exactly.  This bound cuts time into
// ticks of w units, tick(t) = floor(t / w), and keeps per event type a bitmask
// of the ticks holding one of its events.  An edge (lo, hi] joins ticks whose
// difference lies in [dlo, dhi] = [floor((lo + 1) / w), floor((hi + w - 1) / w)];
// with M_1 = the ticks of E_1 and M_{k+1} = the ticks of E_{k+1} reachable
// from M_k, the bound is the number of E_N events in ticks of M_N.  Every
// event that ends an occurrence is among them and non-overlapped occurrences
// end at distinct events, so the bound is never below the count.
//
// With dhi <= 31 (w >= hi / 31) a word of M_{k+1} needs only the same and the
// previous word of M_k: a warp walks the stream 32 words (1024 ticks) at a
// time with one shuffle per node, and since an error in the carried word
// moves forward one word per node, a slice of the stream can start anywhere
// after one chunk of warm-up.  Work per episode is (nodes x words), not
// (nodes x events), and the bitmask rows are shared by all episodes in L2.
#include <algorithm>
#include <mutex>
#include <vector>

#include "fem_internal.cuh"

namespace fem {
namespace {

constexpr unsigned kFull = 0xFFFFFFFFu;
constexpr size_t kCoarseBudget = size_t(256) << 20;  // tables per stream and tick width

__global__ void k_coarse_bits(const uint16_t *__restrict__ ty, const int32_t *__restrict__ tm, int64_t n, int32_t w,
                              int64_t tau0, int64_t W, uint32_t *__restrict__ bits) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t u = (int64_t)tm[i] / w - tau0;
        atomicOr(&bits[(int64_t)ty[i] * W + (u >> 5)], 1u << (u & 31));
    }
}

// cum[a][i] = first position in type a's list with word >= i (rows of W + 1).
__global__ void k_coarse_cum(const int64_t *__restrict__ toff, const int32_t *__restrict__ ttime, int n_types,
                             int64_t n, int32_t w, int64_t tau0, int64_t W, uint32_t *__restrict__ cum) {
    for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < n; g += (int64_t)gridDim.x * blockDim.x) {
        int lo = 0, hi = n_types;  // largest a with toff[a] <= g: the type holding g
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (toff[mid] <= g) lo = mid; else hi = mid;
        }
        const int64_t j = g - toff[lo], f = toff[lo + 1] - toff[lo];
        const int64_t iw = ((int64_t)ttime[g] / w - tau0) >> 5;
        const int64_t ip = j > 0 ? (((int64_t)ttime[g - 1] / w - tau0) >> 5) : -1;
        uint32_t *row = cum + (int64_t)lo * (W + 1);
        for (int64_t i = ip + 1; i <= iw; ++i) row[i] = (uint32_t)j;
        if (j == f - 1)
            for (int64_t i = iw + 1; i <= W; ++i) row[i] = (uint32_t)f;
    }
}

struct CoarseArgs {
    const int64_t *offs;
    const uint16_t *types;
    const int32_t *lo, *hi;
    int64_t n_cand;
    int32_t w;
    const uint32_t *bits, *cum;
    int64_t W, tau0, n_chunks;
    const int64_t *toff;
    const int32_t *ttime;
    int n_slices, slice_chunks;
    uint32_t *ub;
};

// One warp walks chunks [c0, c1) of the stream for one episode (types[N],
// lo / hi[N - 1]) and returns this lane's share of the bound; the chunk
// before c0 (if any) only warms up the carried words.
template <int NMAX>
__device__ __forceinline__ uint32_t coarse_walk(const uint16_t *__restrict__ types, const int32_t *__restrict__ lo,
                                                const int32_t *__restrict__ hi, int N,
                                                const uint32_t *__restrict__ bits, const uint32_t *__restrict__ cum,
                                                const int64_t *__restrict__ toff, const int32_t *__restrict__ ttime,
                                                int64_t W, int64_t tau0, int32_t w, int64_t c0, int64_t c1, int lane) {
    int E[NMAX], dlo[NMAX], lr[NMAX];
    uint32_t carry[NMAX];
#pragma unroll
    for (int k = 0; k < NMAX; ++k) {
        E[k] = k < N ? (int)types[k] : 0;
        dlo[k] = 0;
        lr[k] = 1;
        if (k < N - 1) {
            const int32_t l = lo[k], h = hi[k];
            dlo[k] = (l + 1) / w;
            lr[k] = (int)(((int64_t)h + w - 1) / w) - dlo[k] + 1;
        }
        carry[k] = 0;
    }
    const int last = types[N - 1];  // (not E[N - 1]: a dynamic index would put E in local memory)
    const uint32_t *bl = bits + (int64_t)last * W;
    const uint32_t *cl = cum + (int64_t)last * (W + 1);
    const int32_t *tl = ttime + toff[last];
    uint32_t acc = 0;
    for (int64_t ch = c0 > 0 ? c0 - 1 : 0; ch < c1; ++ch) {
        const int64_t i = ch * 32 + lane;
        uint32_t m = bits[(int64_t)E[0] * W + i];
#pragma unroll
        for (int k = 0; k < NMAX - 1; ++k) {
            if (k < N - 1) {
                uint32_t prev = __shfl_up_sync(kFull, m, 1);
                if (lane == 0) prev = carry[k];
                const uint32_t nc = __shfl_sync(kFull, m, 31);
                const bool any = __any_sync(kFull, m != 0u) || carry[k] != 0u;  // warp-uniform
                carry[k] = nc;
                if (any) {
                    const uint64_t V = ((uint64_t)m << 32) | prev;
                    uint64_t Z = V;  // Z = OR of V << e for e < s, s the largest power of 2 <= lr
                    int s = 1;
#pragma unroll
                    for (int q = 0; q < 5; ++q)
                        if (2 * s <= lr[k]) {
                            Z |= Z << s;
                            s <<= 1;
                        }
                    const uint64_t Y = Z | (Z << (lr[k] - s));
                    const uint32_t D = (uint32_t)((Y << dlo[k]) >> 32);
                    m = D ? (bits[(int64_t)E[k + 1] * W + i] & D) : 0u;
                } else {
                    m = 0u;
                }
            }
        }
        if (ch >= c0 && __any_sync(kFull, m != 0u)) {
            if (m) {
                const uint32_t q0 = cl[i], q1 = cl[i + 1];
                if (q1 - q0 == (uint32_t)__popc(bl[i])) {
                    acc += (uint32_t)__popc(m);  // one event per set tick
                } else {
                    for (uint32_t q = q0; q < q1; ++q) {
                        const int64_t u = (int64_t)tl[q] / w - tau0;
                        acc += (m >> (u & 31)) & 1u;
                    }
                }
            }
        }
    }
    return acc;
}

__device__ __forceinline__ uint32_t warp_sum(uint32_t v) {
#pragma unroll
    for (int q = 16; q > 0; q >>= 1) v += __shfl_down_sync(kFull, v, q);
    return v;
}

// One warp per (episode, slice of the stream).
template <int NMAX>
__global__ void __launch_bounds__(256, NMAX <= 4 ? 4 : (NMAX <= 8 ? 2 : 1)) k_coarse_ub(CoarseArgs a) {
    const int lane = threadIdx.x & 31;
    const int64_t wid = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    if (wid >= a.n_cand * a.n_slices) return;  // whole warps
    const int64_t c = wid / a.n_slices;
    const int sl = (int)(wid % a.n_slices);
    const int64_t o = a.offs[c];
    const int N = (int)(a.offs[c + 1] - o);
    const int64_t eo = o - c;
    if (N == 1) {
        if (sl == 0 && lane == 0) {
            const int e = a.types[o];
            a.ub[c] = (uint32_t)(a.toff[e + 1] - a.toff[e]);
        }
        return;
    }
    const int64_t c0 = (int64_t)sl * a.slice_chunks;
    const int64_t c1 = min(c0 + (int64_t)a.slice_chunks, a.n_chunks);
    const uint32_t acc = warp_sum(coarse_walk<NMAX>(a.types + o, a.lo + eo, a.hi + eo, N, a.bits, a.cum, a.toff,
                                                    a.ttime, a.W, a.tau0, a.w, c0, c1, lane));
    if (lane == 0 && acc) atomicAdd(&a.ub[c], acc);
}

// Inside the captured mining graph: level-N candidates in fixed stride
// (ct[c * N + k], cl / ch[c * (N - 1) + k]) of several recordings, their
// live count in *d_n; each recording's stream cut into n_slices slices.
// Below min_cands candidates the level is not bounded.
template <int NMAX>
__global__ void __launch_bounds__(256, NMAX <= 4 ? 3 : (NMAX <= 8 ? 2 : 1))
    k_coarse_graph(const uint16_t *__restrict__ ct, const int32_t *__restrict__ cl, const int32_t *__restrict__ ch,
                   const uint32_t *__restrict__ crec, const int32_t *__restrict__ d_n, int64_t cap, int N,
                   const CoarseDesc *__restrict__ desc, int n_slices, int64_t min_cands, uint32_t *__restrict__ ub) {
    const int lane = threadIdx.x & 31;
    const int64_t n = min((int64_t)*d_n, cap);
    if (n < min_cands) return;
    const int64_t items = n * n_slices;
    for (int64_t wid = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; wid < items;
         wid += ((int64_t)gridDim.x * blockDim.x) >> 5) {
        const int64_t c = wid / n_slices;
        const int sl = (int)(wid % n_slices);
        const CoarseDesc d = desc[crec[c]];
        const int64_t c0 = (int64_t)sl * d.slice_chunks;
        const int64_t c1 = min(c0 + (int64_t)d.slice_chunks, d.n_chunks);
        if (c0 >= c1) continue;  // warp-uniform
        const uint32_t acc =
            warp_sum(coarse_walk<NMAX>(ct + c * N, cl + c * (N - 1), ch + c * (N - 1), N, d.bits, d.cum, d.toff,
                                       d.ttime, d.W, d.tau0, d.w, c0, c1, lane));
        if (lane == 0 && acc) atomicAdd(&ub[c], acc);
    }
}

// skip[c] = 1 when candidate c's bound cannot pass its recording's threshold.
__global__ void k_coarse_skip(const uint32_t *__restrict__ ub, const uint32_t *__restrict__ crec,
                              const uint32_t *__restrict__ thr, const int32_t *__restrict__ d_n, int64_t cap,
                              int64_t min_cands, uint8_t *__restrict__ skip) {
    const int64_t n = min((int64_t)*d_n, cap);
    const bool on = n >= min_cands;
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < n; c += (int64_t)gridDim.x * blockDim.x)
        skip[c] = on && ub[c] <= thr[crec[c]] ? 1 : 0;
}

int64_t coarse_words(const fem_stream *s, int32_t w) {
    const int64_t ticks = (int64_t)s->t_last / w - (int64_t)s->t_first / w + 1;
    const int64_t words = (ticks + 31) / 32;
    return (words + 31) / 32 * 32;
}

int stream_coarse(fem_ctx *ctx, fem_stream *s, int32_t w, const fem_coarse_tab **out) {
    auto it = s->coarse.find(w);
    if (it != s->coarse.end()) {
        *out = &it->second;
        return FEM_OK;
    }
    FEM_TRY(stream_bytype(ctx, s));
    fem_coarse_tab t;
    t.W = coarse_words(s, w);
    t.tau0 = (int64_t)s->t_first / w;
    const size_t b1 = sizeof(uint32_t) * (size_t)s->n_types * t.W;
    const size_t b2 = sizeof(uint32_t) * (size_t)s->n_types * (t.W + 1);
    void *p1 = nullptr, *p2 = nullptr;
    FEM_TRY(dev_alloc(ctx, &p1, b1));
    if (dev_alloc(ctx, &p2, b2) != FEM_OK) {
        dev_free(ctx, p1, b1);
        return FEM_ERR_NOMEM;
    }
    t.bits = static_cast<uint32_t *>(p1);
    t.cum = static_cast<uint32_t *>(p2);
    t.bytes = b1 + b2;
    cudaStream_t st = ctx->stream;
    cudaMemsetAsync(t.bits, 0, b1, st);
    cudaMemsetAsync(t.cum, 0, b2, st);
    if (s->n > 0) {
        const unsigned g = (unsigned)std::max<int64_t>(1, std::min<int64_t>((s->n + 255) / 256, 8 * ctx->n_sm));
        k_coarse_bits<<<g, 256, 0, st>>>(s->d_type, s->d_time, s->n, w, t.tau0, t.W, t.bits);
        k_coarse_cum<<<g, 256, 0, st>>>(s->d_toff, s->d_ttime, (int)s->n_types, s->n, w, t.tau0, t.W, t.cum);
    }
    if (cudaGetLastError() != cudaSuccess) {
        cudaStreamSynchronize(st);
        dev_free(ctx, p1, b1);
        dev_free(ctx, p2, b2);
        return FEM_ERR_CUDA;
    }
    s->bytes += t.bytes;
    s->coarse[w] = t;
    *out = &s->coarse[w];
    return FEM_OK;
}

}  // namespace

int32_t coarse_tick(const fem_stream *s, int64_t hi_max, size_t budget) {
    int64_t w = std::max<int64_t>(1, (hi_max + 30) / 31);
    if (budget == 0) budget = kCoarseBudget;
    while (w < (int64_t(1) << 30) &&
           (size_t)s->n_types * (2 * (size_t)coarse_words(s, (int32_t)w) + 1) * sizeof(uint32_t) > budget)
        w *= 2;
    return (int32_t)w;
}

void coarse_free(fem_ctx *ctx, fem_stream *s) {
    for (auto &kv : s->coarse) {
        const fem_coarse_tab &t = kv.second;
        dev_free(ctx, t.bits, sizeof(uint32_t) * (size_t)s->n_types * t.W);
        dev_free(ctx, t.cum, sizeof(uint32_t) * (size_t)s->n_types * (t.W + 1));
    }
    s->coarse.clear();
}

int coarse_bound_dev(fem_ctx *ctx, fem_stream *s, int64_t n_cand, const int64_t *d_offs, const uint16_t *d_types,
                     const int32_t *d_lo, const int32_t *d_hi, int max_nodes, int32_t w, uint32_t *d_ub,
                     int64_t *launches) {
    if (n_cand <= 0) return FEM_OK;
    if (w < 1 || max_nodes < 1 || max_nodes > FEM_MAX_NODES) return FEM_ERR_INVAL;
    const fem_coarse_tab *t = nullptr;
    FEM_TRY(stream_coarse(ctx, s, w, &t));
    cudaStream_t st = ctx->stream;
    FEM_CUDA_TRY(cudaMemsetAsync(d_ub, 0, sizeof(uint32_t) * n_cand, st));
    CoarseArgs a{};
    a.offs = d_offs;
    a.types = d_types;
    a.lo = d_lo;
    a.hi = d_hi;
    a.n_cand = n_cand;
    a.w = w;
    a.bits = t->bits;
    a.cum = t->cum;
    a.W = t->W;
    a.tau0 = t->tau0;
    a.n_chunks = t->W / 32;
    a.toff = s->d_toff;
    a.ttime = s->d_ttime;
    a.ub = d_ub;
    // enough warps to fill the GPU: slices of the stream when episodes are few
    const int64_t target = (int64_t)64 * ctx->n_sm;
    int64_t ns = std::min<int64_t>(a.n_chunks, std::max<int64_t>(1, (target + n_cand - 1) / n_cand));
    ns = std::min<int64_t>(ns, std::max<int64_t>(1, ((int64_t)1 << 26) / n_cand));
    a.slice_chunks = (int)((a.n_chunks + ns - 1) / ns);
    a.n_slices = (int)((a.n_chunks + a.slice_chunks - 1) / a.slice_chunks);
    const int64_t warps = n_cand * a.n_slices;
    const unsigned blocks = (unsigned)((warps + 7) / 8);
    if (max_nodes <= 4)
        k_coarse_ub<4><<<blocks, 256, 0, st>>>(a);
    else if (max_nodes <= 8)
        k_coarse_ub<8><<<blocks, 256, 0, st>>>(a);
    else
        k_coarse_ub<16><<<blocks, 256, 0, st>>>(a);
    FEM_CUDA_TRY(cudaGetLastError());
    if (launches) *launches += 1;
    return FEM_OK;
}

int coarse_desc(fem_ctx *ctx, fem_stream *s, int32_t w, int n_slices, CoarseDesc *out) {
    const fem_coarse_tab *t = nullptr;
    FEM_TRY(stream_coarse(ctx, s, w, &t));
    CoarseDesc d{};
    d.bits = t->bits;
    d.cum = t->cum;
    d.toff = s->d_toff;
    d.ttime = s->d_ttime;
    d.W = t->W;
    d.tau0 = t->tau0;
    d.n_chunks = t->W / 32;
    d.w = w;
    d.slice_chunks = (int32_t)((d.n_chunks + n_slices - 1) / n_slices);
    *out = d;
    return FEM_OK;
}

int coarse_graph_level(cudaStream_t st, int n_sm, int N, const uint16_t *ct, const int32_t *cl, const int32_t *ch,
                       const uint32_t *crec, const int32_t *d_n, int64_t cap, const CoarseDesc *d_desc, int n_slices,
                       const uint32_t *thr, int64_t min_cands, uint32_t *ub, uint8_t *skip) {
    if (N < 2 || N > FEM_MAX_NODES || cap <= 0) return FEM_ERR_INVAL;
    FEM_CUDA_TRY(cudaMemsetAsync(ub, 0, sizeof(uint32_t) * cap, st));
    const unsigned blocks = (unsigned)std::max<int64_t>(1, std::min<int64_t>((cap * n_slices + 7) / 8, 16 * n_sm));
    if (N <= 4)
        k_coarse_graph<4><<<blocks, 256, 0, st>>>(ct, cl, ch, crec, d_n, cap, N, d_desc, n_slices, min_cands, ub);
    else if (N <= 8)
        k_coarse_graph<8><<<blocks, 256, 0, st>>>(ct, cl, ch, crec, d_n, cap, N, d_desc, n_slices, min_cands, ub);
    else
        k_coarse_graph<16><<<blocks, 256, 0, st>>>(ct, cl, ch, crec, d_n, cap, N, d_desc, n_slices, min_cands, ub);
    const unsigned sb = (unsigned)std::max<int64_t>(1, std::min<int64_t>((cap + 255) / 256, 8 * n_sm));
    k_coarse_skip<<<sb, 256, 0, st>>>(ub, crec, thr, d_n, cap, min_cands, skip);
    FEM_CUDA_TRY(cudaGetLastError());
    return FEM_OK;
}

}  // namespace fem

using namespace fem;

extern "C" int fem_upper_bound_coarse(fem_ctx *ctx, const fem_stream *s, const fem_cands *c, int32_t tick,
                                      uint32_t *ub, int out_is_device, int32_t *tick_used) {
    if (!ctx || !s || !c || s->ctx != ctx || c->n_cand < 0 || c->n_cand > INT32_MAX / 2 || tick < 0)
        return FEM_ERR_INVAL;
    const int64_t n = c->n_cand;
    if (n > 0 && (!ub || !c->offs || !c->types || !c->lo || !c->hi)) return FEM_ERR_INVAL;
    if (s->n_types > 8192 || s->n > INT32_MAX / 2) return FEM_ERR_INVAL;
    std::lock_guard<std::mutex> g(ctx->mu);
    cudaSetDevice(ctx->device);
    const double t0 = now_s();
    cudaStream_t st = ctx->stream;
    // candidates to the host for the checks
    std::vector<int64_t> offs(n + 1, 0);
    if (n > 0 && c->ptr_is_device) {
        FEM_CUDA_TRY(cudaMemcpyAsync(offs.data(), c->offs, 8 * (n + 1), cudaMemcpyDeviceToHost, st));
        FEM_CUDA_TRY(cudaStreamSynchronize(st));
    } else if (n > 0) {
        std::copy(c->offs, c->offs + n + 1, offs.begin());
    }
    if (offs[0] != 0) return FEM_ERR_INVAL;
    int max_nodes = 1;
    for (int64_t i = 0; i < n; ++i) {
        const int64_t N = offs[i + 1] - offs[i];
        if (N < 1 || N > FEM_MAX_NODES) return FEM_ERR_INVAL;
        max_nodes = std::max<int>(max_nodes, (int)N);
    }
    const int64_t n_nodes = offs[n], n_edges = n_nodes - n;
    std::vector<uint16_t> ty(std::max<int64_t>(n_nodes, 1));
    std::vector<int32_t> lo(std::max<int64_t>(n_edges, 1)), hi(std::max<int64_t>(n_edges, 1));
    if (c->ptr_is_device) {
        if (n_nodes > 0) FEM_CUDA_TRY(cudaMemcpyAsync(ty.data(), c->types, 2 * n_nodes, cudaMemcpyDeviceToHost, st));
        if (n_edges > 0) {
            FEM_CUDA_TRY(cudaMemcpyAsync(lo.data(), c->lo, 4 * n_edges, cudaMemcpyDeviceToHost, st));
            FEM_CUDA_TRY(cudaMemcpyAsync(hi.data(), c->hi, 4 * n_edges, cudaMemcpyDeviceToHost, st));
        }
        FEM_CUDA_TRY(cudaStreamSynchronize(st));
    } else {
        std::copy(c->types, c->types + n_nodes, ty.begin());
        std::copy(c->lo, c->lo + n_edges, lo.begin());
        std::copy(c->hi, c->hi + n_edges, hi.begin());
    }
    int64_t hi_max = 1;
    for (int64_t k = 0; k < n_nodes; ++k)
        if (ty[k] >= s->n_types) return FEM_ERR_INVAL;
    for (int64_t e = 0; e < n_edges; ++e) {
        if (lo[e] < 0 || lo[e] >= hi[e]) return FEM_ERR_INVAL;
        hi_max = std::max<int64_t>(hi_max, hi[e]);
    }
    fem_stream *sm = const_cast<fem_stream *>(s);
    const int32_t w = tick > 0 ? tick : coarse_tick(sm, hi_max, 0);
    if (hi_max > 31 * (int64_t)w) return FEM_ERR_INVAL;
    if (tick_used) *tick_used = w;
    if (n == 0) return FEM_OK;
    TmpDev tmp(ctx);
    const int64_t *d_offs = c->offs;
    const uint16_t *d_types = c->types;
    const int32_t *d_lo = c->lo, *d_hi = c->hi;
    if (!c->ptr_is_device) {
        int64_t *p0;
        uint16_t *p1;
        int32_t *p2, *p3;
        FEM_TRY(tmp.get(&p0, n + 1));
        FEM_TRY(tmp.get(&p1, std::max<int64_t>(n_nodes, 1)));
        FEM_TRY(tmp.get(&p2, std::max<int64_t>(n_edges, 1)));
        FEM_TRY(tmp.get(&p3, std::max<int64_t>(n_edges, 1)));
        FEM_TRY(copy_in(ctx, p0, offs.data(), 8 * (n + 1), 0));
        FEM_TRY(copy_in(ctx, p1, ty.data(), 2 * n_nodes, 0));
        if (n_edges > 0) {
            FEM_TRY(copy_in(ctx, p2, lo.data(), 4 * n_edges, 0));
            FEM_TRY(copy_in(ctx, p3, hi.data(), 4 * n_edges, 0));
        }
        d_offs = p0;
        d_types = p1;
        d_lo = p2;
        d_hi = p3;
    }
    uint32_t *d_ub;
    FEM_TRY(tmp.get(&d_ub, n));
    fem_stats stats{};
    cudaEventRecord(ctx->ev0, st);
    FEM_TRY(coarse_bound_dev(ctx, sm, n, d_offs, d_types, d_lo, d_hi, max_nodes, w, d_ub, &stats.kernel_launches));
    cudaEventRecord(ctx->ev1, st);
    FEM_TRY(copy_out(ctx, ub, d_ub, 4 * n, out_is_device));
    FEM_CUDA_TRY(cudaStreamSynchronize(st));
    float ms = 0.f;
    cudaEventElapsedTime(&ms, ctx->ev0, ctx->ev1);
    stats.count_kernel_ms = ms;
    stats.candidates_counted = n;
    stats.total_ms = (now_s() - t0) * 1e3;
    ctx->last = stats;
    return FEM_OK;
}
