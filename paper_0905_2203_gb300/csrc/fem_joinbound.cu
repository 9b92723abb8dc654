// fem_joinbound.cu -- an upper bound on the count of every 3-node candidate
// from its two frequent 2-node sub-episodes, taken before the exact count.
//
// A level-3 candidate A -(b1]-> B -(b2]-> C is the join of the frequent
// 2-node episodes alpha = A -(b1]-> B and beta = B -(b2]-> C.  Every
// occurrence of the candidate passes through one B event that has an A event
// inside b1 before it (the B event is a valid end of alpha) and a C event
// inside b2 after it (a valid start of beta), and non-overlapped occurrences
// pass through distinct B events.  So
//     count <= UB = #{ B events that are both },
// the same anti-monotonicity argument ("Temporal Data Mining") as the
// level-2 pair bound.  Every frequent 2-node episode X -(b]-> Y of a
// recording gets two bitsets, one bit per event of a type's list: V over
// Y's list (valid ends) and S over X's list (valid starts), each word one
// ballot of a warp over 32 consecutive events, found with the stream's
// per-type time index.  A candidate's UB is then the popcount of
// V(alpha) AND S(beta), both over B's list: about n_B / 32 word operations,
// where its exact count looks at every entry of alpha.  Candidates whose UB
// is at or below the recording's threshold are skipped by the exact count
// (their count is reported as 0 and they cannot be frequent).
//
// Bitsets are laid out per recording: recording r's frequent 2-node
// episodes f (in their order) take stride[r] words each (the longest list of
// the recording / 32), from base[r]; the pass is skipped (nothing pruned)
// when the total passes the buffers' capacity.
#include "fem_internal.cuh"

namespace fem {

namespace {

constexpr unsigned kFull = 0xFFFFFFFFu;

__device__ __forceinline__ int bin_of(const JoinBoundArgs &a, int32_t lo, int32_t hi) {
    int k = 0;
    while (k < a.nb && !(a.blo[k] == lo && a.bhi[k] == hi)) ++k;
    return k;
}

// First position of the list tl[0, len) (type row `row` of the time index)
// with a time at or after q.
__device__ __forceinline__ int first_at_or_after(const RecInfo &ri, const int32_t *__restrict__ tl, int len,
                                                 const int32_t *__restrict__ row, uint32_t q) {
    const uint32_t tb = (uint32_t)ri.tbase;
    uint32_t c = q > tb ? (q - tb) >> ri.tshift : 0u;
    if (c > (uint32_t)ri.tcells) c = (uint32_t)ri.tcells;
    int pos = row[c];
    while (pos < len && (uint32_t)tl[pos] < q) ++pos;
    return pos;
}

// The (X, Y, bin) -> frequent 2-node episode table (entries set to -1
// before): the episode's index in the frequent set.
__global__ void k_jb_index(JoinBoundArgs a) {
    const int64_t F = *a.f2n;
    for (int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; f < F; f += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t r = a.f2rec[f];
        const int k = bin_of(a, a.f2lo[f], a.f2hi[f]);
        if (k >= a.nb) continue;
        const uint32_t X = a.f2types[2 * f], Y = a.f2types[2 * f + 1];
        a.tab[a.tab_off[r] + ((int64_t)X * a.nt[r] + Y) * a.nb + k] = (int32_t)f;
    }
}

// One thread: the first word of every recording's bitsets and the total.
__global__ void k_jb_base(JoinBoundArgs a) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    int64_t acc = 0;
    for (int r = 0; r < a.n_recs; ++r) {
        a.base[r] = acc;
        acc += (a.f2foff[r + 1] - a.f2foff[r]) * (int64_t)a.stride[r];
    }
    a.base[a.n_recs] = acc;
}

// The V and S bitsets of every frequent 2-node episode, one warp per
// (episode, chunk of 1024 list events): 32 words, one ballot per 32 events.
__global__ void k_jb_bits(JoinBoundArgs a) {
    if (a.base[a.n_recs] > a.cap_words) return;
    const int lane = threadIdx.x & 31;
    const int64_t items = (int64_t)*a.f2n * a.nch;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t it = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; it < items; it += nw) {
        const int64_t f = it / a.nch;
        const int ch = (int)(it % a.nch);
        const uint32_t r = a.f2rec[f];
        const RecInfo &ri = a.ri[r];
        const uint32_t X = a.f2types[2 * f], Y = a.f2types[2 * f + 1];
        const int64_t xb = ri.toff[X], yb = ri.toff[Y];
        const int lenX = (int)(ri.toff[X + 1] - xb), lenY = (int)(ri.toff[Y + 1] - yb);
        const int b0 = ch * 1024;
        if (b0 >= lenX && b0 >= lenY) continue;
        const int32_t lo = a.f2lo[f], hi = a.f2hi[f];
        const int32_t *tlX = ri.ttime + xb;
        const int32_t *tlY = ri.ttime + yb;
        const int32_t *rowX = ri.tidx + (int64_t)X * (ri.tcells + 1);
        const int32_t *rowY = ri.tidx + (int64_t)Y * (ri.tcells + 1);
        const int64_t wb = a.base[r] + (f - a.f2foff[r]) * (int64_t)a.stride[r];
        // V: a Y event at t is a valid end when the newest X event before
        // t - lo exists and is not before t - hi
        for (int b = b0; b < lenY && b < b0 + 1024; b += 32) {
            bool v = false;
            if (b + lane < lenY) {
                const int32_t t = tlY[b + lane];
                const int64_t d = (int64_t)t - lo;
                if (d > 0) {
                    const int pos = first_at_or_after(ri, tlX, lenX, rowX, (uint32_t)d);
                    v = pos > 0 && (int64_t)tlX[pos - 1] >= (int64_t)t - hi;
                }
            }
            const unsigned w = __ballot_sync(kFull, v);
            if (lane == 0) a.vbits[wb + (b >> 5)] = w;
        }
        // S: an X event at t is a valid start when the first Y event after
        // t + lo is not after t + hi
        for (int b = b0; b < lenX && b < b0 + 1024; b += 32) {
            bool s = false;
            if (b + lane < lenX) {
                const uint32_t t = (uint32_t)tlX[b + lane];
                const int pos = first_at_or_after(ri, tlY, lenY, rowY, t + (uint32_t)lo + 1u);
                s = pos < lenY && (uint32_t)tlY[pos] <= t + (uint32_t)hi;
            }
            const unsigned w = __ballot_sync(kFull, s);
            if (lane == 0) a.sbits[wb + (b >> 5)] = w;
        }
    }
}

// One warp per level-3 candidate: UB, and the skip flag when UB is at or
// below the threshold (or-ed into the flags another bound set, if any);
// skipped candidates are counted per recording.
__global__ void k_jb_bound(JoinBoundArgs a) {
    const int lane = threadIdx.x & 31;
    const int64_t C = *a.cn;
    const bool usable = a.base[a.n_recs] <= a.cap_words;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t c = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; c < C; c += nw) {
        const uint32_t r = a.crec[c];
        bool sk = false;
        if (usable) {
            const uint32_t A = a.ct[3 * c], B = a.ct[3 * c + 1], Cc = a.ct[3 * c + 2];
            const int k1 = bin_of(a, a.cl[2 * c], a.ch[2 * c]), k2 = bin_of(a, a.cl[2 * c + 1], a.ch[2 * c + 1]);
            const int64_t to = a.tab_off[r];
            const int64_t nt = a.nt[r];
            const int32_t f1 = k1 < a.nb ? a.tab[to + ((int64_t)A * nt + B) * a.nb + k1] : -1;
            const int32_t f2 = k2 < a.nb ? a.tab[to + ((int64_t)B * nt + Cc) * a.nb + k2] : -1;
            if (f1 >= 0 && f2 >= 0) {
                const RecInfo &ri = a.ri[r];
                const int lenB = (int)(ri.toff[B + 1] - ri.toff[B]);
                const int64_t st = a.stride[r];
                const uint32_t *v = a.vbits + a.base[r] + (f1 - a.f2foff[r]) * st;
                const uint32_t *s = a.sbits + a.base[r] + (f2 - a.f2foff[r]) * st;
                uint32_t acc = 0;
                for (int w = lane; w < (lenB + 31) >> 5; w += 32) acc += __popc(v[w] & s[w]);
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(kFull, acc, o);
                sk = acc <= a.thr[r];
            }
        }
        if (lane == 0) {
            const bool fin = sk || (a.or_skip && a.skip[c]);
            a.skip[c] = fin ? 1 : 0;
            if (fin) atomicAdd(a.skipc + r, 1ull);
        }
    }
}

}  // namespace

int join_bound_level3(cudaStream_t st, int n_sm, const JoinBoundArgs &a) {
    const unsigned g = (unsigned)std::max(1, 8 * n_sm);
    if (cudaMemsetAsync(a.tab, 0xFF, sizeof(int32_t) * (size_t)std::max<int64_t>(a.tab_n, 1), st) != cudaSuccess ||
        cudaMemsetAsync(a.skipc, 0, sizeof(unsigned long long) * (size_t)std::max(a.n_recs, 1), st) != cudaSuccess)
        return FEM_ERR_CUDA;
    k_jb_index<<<g, 256, 0, st>>>(a);
    k_jb_base<<<1, 32, 0, st>>>(a);
    k_jb_bits<<<g, 256, 0, st>>>(a);
    k_jb_bound<<<g, 256, 0, st>>>(a);
    FEM_CUDA_TRY(cudaGetLastError());
    return FEM_OK;
}

}  // namespace fem
