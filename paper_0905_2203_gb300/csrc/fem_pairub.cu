// fem_pairub.cu -- the level-2 upper-bound pre-pass, organised by end type.
//
// For an ordered pair of distinct types (a, b) and a bin (lo, hi], the bound
// is the number of b-events that have an a-event at a distance d with
// lo < d <= hi before them.  Every occurrence of the 2-node episode
// a -(lo,hi]-> b ends at such a b-event and non-overlapped occurrences end
// at distinct events, so the bound is never below the count (the
// anti-monotonicity of section "Temporal Data Mining": a candidate whose
// bound does not exceed the threshold cannot be frequent).
//
// One warp takes a run of up to kPairChunk events of ONE end type b (from
// the per-type lists, with each entry's stream position).  Every lane walks
// back over the stream from its own b-event to hi_max before it and marks,
// in its own bitset, each (a, bin) met; the first mark of a pair adds one to
// the warp's shared-memory histogram of (a, bin) for this b.  At the end of
// the run the warp adds its histogram to the bound table with one global
// atomic per non-zero (a, bin).  Global atomics thus scale with
// (runs x pairs), not with (events x window).
#include <algorithm>

#include "fem_internal.cuh"

namespace fem {

namespace {

constexpr int kPairChunkMax = 1024;  // end events per warp item (at most)
constexpr int kPairWarps = 8;

struct PairRec {
    const uint16_t *type;
    const int32_t *time;
    const int64_t *toff;
    const int32_t *ttime;
    const int32_t *tpos;
    int64_t ub_off;
    uint32_t nt;
    int32_t nchunk;  // runs per type: ceil(longest list / chunk)
};

__global__ void __launch_bounds__(kPairWarps * 32) k_pair_ub_t(const PairRec *__restrict__ recs, int n_recs,
                                                               const int64_t *__restrict__ ipre, int nb,
                                                               const int32_t *__restrict__ blo,
                                                               const int32_t *__restrict__ bhi, int32_t hi_max,
                                                               const uint8_t *__restrict__ lut_g, int lut_words,
                                                               int hist_words, int bit_words, int chunk,
                                                               uint32_t *ub) {
    extern __shared__ uint32_t sm[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    for (int i = threadIdx.x; i < lut_words; i += blockDim.x) sm[i] = reinterpret_cast<const uint32_t *>(lut_g)[i];
    __syncthreads();
    const uint8_t *lut = lut_words ? reinterpret_cast<const uint8_t *>(sm) : nullptr;
    uint32_t *hist = sm + lut_words + warp * (hist_words + 32 * bit_words);
    uint32_t *bits = hist + hist_words + lane;  // word w of this lane at bits[32 * w]
    const int64_t n_items = ipre[n_recs];
    for (int64_t it = (int64_t)blockIdx.x * nw + warp; it < n_items; it += (int64_t)gridDim.x * nw) {
        int lo_r = 0, hi_r = n_recs;  // last recording whose runs start at or before it
        while (hi_r - lo_r > 1) {
            const int mid = (lo_r + hi_r) >> 1;
            if (ipre[mid] <= it) lo_r = mid; else hi_r = mid;
        }
        const PairRec &R = recs[lo_r];
        const int64_t local = it - ipre[lo_r];
        const uint32_t b = (uint32_t)(local / R.nchunk);
        const int64_t j0 = R.toff[b] + (local % R.nchunk) * chunk;
        const int64_t j1 = min(R.toff[b + 1], j0 + chunk);
        if (j0 >= j1) continue;  // warp-uniform
        const int hw = (int)R.nt * nb;
        const int bw = (hw + 31) >> 5;
        for (int w = lane; w < hw; w += 32) hist[w] = 0;
        __syncwarp();
        for (int64_t base = j0; base < j1; base += 32) {
            const int64_t j = base + lane;
            if (j < j1) {
                const int32_t t = R.ttime[j];
                const int64_t P = R.tpos[j];
                for (int w = 0; w < bw; ++w) bits[32 * w] = 0;
                const int32_t lim = t - hi_max;  // t >= 0, hi_max > 0: no overflow
                for (int64_t i = P - 1; i >= 0; --i) {
                    const int32_t ti = R.time[i];
                    if (ti < lim) break;
                    const int32_t d = t - ti;
                    if (d <= 0) continue;  // same time: never inside a bin (lo >= 0)
                    const uint32_t a = R.type[i];
                    if (a == b) continue;
                    uint32_t mask = 0;
                    if (lut) {
                        mask = lut[d];
                    } else {
                        for (int k = 0; k < nb; ++k)
                            if (blo[k] < d && d <= bhi[k]) mask |= 1u << k;
                    }
                    while (mask) {
                        const int k = __ffs(mask) - 1;
                        mask &= mask - 1;
                        const uint32_t bit = a * (uint32_t)nb + (uint32_t)k;
                        const uint32_t m = 1u << (bit & 31);
                        uint32_t &wd = bits[32 * (bit >> 5)];
                        if (!(wd & m)) {
                            wd |= m;
                            atomicAdd(&hist[bit], 1u);
                        }
                    }
                }
            }
        }
        __syncwarp();
        for (int w = lane; w < hw; w += 32) {
            const uint32_t v = hist[w];
            if (v) {
                const uint32_t a = (uint32_t)w / (uint32_t)nb, k = (uint32_t)w % (uint32_t)nb;
                atomicAdd(&ub[R.ub_off + ((int64_t)a * R.nt + b) * nb + k], v);
            }
        }
        __syncwarp();
    }
}

}  // namespace

size_t pair_ub_table_words(const std::vector<fem_stream *> &recs, int nb, std::vector<int64_t> *ub_off) {
    ub_off->assign(recs.size() + 1, 0);
    for (size_t r = 0; r < recs.size(); ++r)
        (*ub_off)[r + 1] = (*ub_off)[r] + (int64_t)recs[r]->n_types * recs[r]->n_types * nb;
    return (size_t)ub_off->back();
}

int pair_ub_setup(fem_ctx *ctx, const std::vector<fem_stream *> &recs, const std::vector<int64_t> &ub_off,
                  const std::vector<int32_t> &blo, const std::vector<int32_t> &bhi, PairUbPlan *plan) {
    const int n_recs = (int)recs.size();
    const int nb = (int)blo.size();
    int32_t hi_max = 0;
    for (auto h : bhi) hi_max = std::max(hi_max, h);
    std::vector<PairRec> pr(n_recs);
    std::vector<int64_t> ipre(n_recs + 1, 0);
    uint32_t nt_max = 1;
    int64_t n_all = 0;
    for (auto *s : recs) {
        nt_max = std::max(nt_max, s->n_types);
        n_all += s->n;
    }
    // By end type pays where the alphabet is large (one global atomic per
    // event and pair is what the stream-order kernels spend); small
    // alphabets keep the stream-order kernels, which give each event its own
    // thread.
    if ((size_t)nt_max * nb < kPairByTypeMinPairs) return FEM_ERR_INVAL;
    // runs of up to 1024 end events, shorter while the launch would hold
    // fewer than about eight runs per resident warp
    int chunk = kPairChunkMax;
    while (chunk > 64 && n_all / chunk < (int64_t)8 * ctx->n_sm * 32) chunk >>= 1;
    for (int r = 0; r < n_recs; ++r) {
        fem_stream *s = recs[r];
        FEM_TRY(stream_bytype(ctx, s));
        const int32_t nchunk = (int32_t)std::max<int64_t>(1, (s->max_list + chunk - 1) / chunk);
        pr[r] = PairRec{s->d_type, s->d_time, s->d_toff, s->d_ttime, s->d_tpos, ub_off[r], s->n_types, nchunk};
        ipre[r + 1] = ipre[r] + (s->n > 0 ? (int64_t)s->n_types * nchunk : 0);
    }
    // bins of each distance 1..hi_max as a byte mask (when it fits)
    std::vector<uint8_t> lut;
    if (hi_max < kPairLutMax) {
        lut.assign(((size_t)hi_max + 4) / 4 * 4, 0);
        for (int32_t d = 1; d <= hi_max; ++d)
            for (int k = 0; k < nb; ++k)
                if (blo[k] < d && d <= bhi[k]) lut[d] |= (uint8_t)(1u << k);
    }
    PairUbPlan &p = *plan;
    p.n_recs = n_recs;
    p.nb = nb;
    p.hi_max = hi_max;
    p.chunk = chunk;
    p.lut_words = (int)(lut.size() / 4);
    p.hist_words = (int)(nt_max * (uint32_t)nb);
    p.bit_words = (p.hist_words + 31) / 32;
    p.smem = (size_t)p.lut_words * 4 + (size_t)kPairWarps * (p.hist_words + 32 * p.bit_words) * 4;
    p.blocks = (int)std::max<int64_t>(1, std::min<int64_t>((ipre[n_recs] + kPairWarps - 1) / kPairWarps,
                                                           (int64_t)ctx->n_sm * 8));
    if (p.smem > (size_t)ctx->smem_optin - 1024) return FEM_ERR_INVAL;
    const size_t bytes = sizeof(PairRec) * n_recs + 8 * (n_recs + 1) + 8 * (nb + 1) * 2 + lut.size() + 64;
    void *q = nullptr;
    FEM_TRY(dev_alloc(ctx, &q, bytes));
    p.buf = q;
    p.buf_bytes = bytes;
    char *c = static_cast<char *>(q);
    p.d_recs = c;
    c += sizeof(PairRec) * n_recs;
    p.d_ipre = reinterpret_cast<int64_t *>(c);
    c += 8 * (n_recs + 1);
    p.d_blo = reinterpret_cast<int32_t *>(c);
    p.d_bhi = p.d_blo + nb;
    c += 8 * (nb + 1) * 2;
    p.d_lut = lut.empty() ? nullptr : reinterpret_cast<uint8_t *>(c);
    cudaStream_t st = ctx->stream;
    FEM_CUDA_TRY(cudaMemcpyAsync(p.d_recs, pr.data(), sizeof(PairRec) * n_recs, cudaMemcpyHostToDevice, st));
    FEM_CUDA_TRY(cudaMemcpyAsync(p.d_ipre, ipre.data(), 8 * (n_recs + 1), cudaMemcpyHostToDevice, st));
    FEM_CUDA_TRY(cudaMemcpyAsync(p.d_blo, blo.data(), 4 * nb, cudaMemcpyHostToDevice, st));
    FEM_CUDA_TRY(cudaMemcpyAsync(p.d_bhi, bhi.data(), 4 * nb, cudaMemcpyHostToDevice, st));
    if (!lut.empty()) FEM_CUDA_TRY(cudaMemcpyAsync(p.d_lut, lut.data(), lut.size(), cudaMemcpyHostToDevice, st));
    if (p.smem > (size_t)ctx->smem_optin - 1024) return FEM_ERR_INVAL;  // the caller uses the stream-order kernel
    if (p.smem > 48 * 1024 &&
        cudaFuncSetAttribute((const void *)k_pair_ub_t, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)p.smem) !=
            cudaSuccess) {
        cudaGetLastError();
        return FEM_ERR_INVAL;
    }
    return FEM_OK;
}

void pair_ub_release(fem_ctx *ctx, PairUbPlan *plan) {
    if (plan->buf) dev_free(ctx, plan->buf, plan->buf_bytes);
    plan->buf = nullptr;
}

int pair_ub_launch(cudaStream_t st, const PairUbPlan &p, uint32_t *ub) {
    k_pair_ub_t<<<(unsigned)p.blocks, kPairWarps * 32, p.smem, st>>>(
        static_cast<const PairRec *>(p.d_recs), p.n_recs, p.d_ipre, p.nb, p.d_blo, p.d_bhi, p.hi_max, p.d_lut,
        p.lut_words, p.hist_words, p.bit_words, p.chunk, ub);
    FEM_CUDA_TRY(cudaGetLastError());
    return FEM_OK;
}

}  // namespace fem
