// fem_noalloc.cu -- episode counting that allocates no memory at all.
//
// Some callers cannot allocate device memory at the moment they need a
// count: code running inside a custom allocator or memory-pool callback,
// processes whose device memory is fully reserved by another framework, or
// real-time loops where a cudaMalloc (which may synchronise the device) is
// forbidden.  fem_count_episodes_noalloc serves them: it works only on the
// caller's device buffers plus one fixed scratch array that this file
// declares at file scope.  That array exists on every GPU that loads the
// library, for as long as the library stays loaded.
//
// The kernel is a variant of the library's one-thread-per-episode counter
// (serial state machine, lists kept as rings of recent timestamps), with the
// rings placed in the static array instead of context-owned scratch.
#include <mutex>

#include "fem_internal.cuh"

namespace {

constexpr int kNoallocMaxDevices = 64;
// Scratch size: 16 MiB per device (4 Mi int32 words).  Word 0..7 form a small
// header (status, largest episode size); ring storage starts at word 8.
constexpr size_t kNoallocWords = 4u * 1024u * 1024u;
constexpr int kNoallocHeader = 8;
constexpr int kNoallocMaxRing = 32;

static __device__ __align__(256) int32_t g_noalloc_scratch[kNoallocWords];

int32_t *g_scratch_addr[kNoallocMaxDevices];
std::mutex g_setup_mu;

// Resolves the device address of the scratch array for the current device
// (once per device).  The array's host-side name is only a stand-in: device
// code must be given the address cudaGetSymbolAddress returns.
int noalloc_setup(int dev, int32_t **out) {
    std::lock_guard<std::mutex> g(g_setup_mu);
    if (!g_scratch_addr[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
            cudaGetLastError();
            return FEM_ERR_CUDA;
        }
        g_scratch_addr[dev] = static_cast<int32_t *>(p);
    }
    *out = g_scratch_addr[dev];
    return FEM_OK;
}

// Header: [0] error bits (1 invalid candidate or offs[0] != 0, 2 ring
// capacity exceeded),
// [1] largest episode size.
__global__ void k_noalloc_check(const int64_t *__restrict__ offs, const uint16_t *__restrict__ ctypes,
                                const int32_t *__restrict__ clo, const int32_t *__restrict__ chi, int64_t n_cand,
                                int32_t *hdr) {
    const int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    // The CSR must start at 0: the kernels index types and bounds from
    // offs[c], so a slice of a larger candidate set would read past them.
    if (c == 0 && offs[0] != 0) atomicOr(&hdr[0], 1);
    if (c >= n_cand) return;
    const int64_t o = offs[c];
    const int64_t N = offs[c + 1] - o;
    bool bad = (N < 1 || N > FEM_MAX_NODES);
    if (!bad) {
        const int64_t eo = o - c;
        for (int k = 0; k < N - 1; ++k)
            if (clo[eo + k] < 0 || clo[eo + k] >= chi[eo + k]) bad = true;
        atomicMax(&hdr[1], (int32_t)N);
    }
    (void)ctypes;
    if (bad) atomicOr(&hdr[0], 1);
}

// One thread per episode: the serial state machine of section "Episode
// Counting Algorithm" (reset after each completed occurrence, next occurrence
// must start after the previous one ends), each node's list kept as a ring of
// the R newest timestamps.  A push that would drop an entry still needed by a
// later query sets error bit 2 instead of silently losing it.
__global__ void k_count_noalloc(const uint16_t *__restrict__ ev_type, const int32_t *__restrict__ ev_time,
                                int64_t n, const int64_t *__restrict__ offs, const uint16_t *__restrict__ ctypes,
                                const int32_t *__restrict__ clo, const int32_t *__restrict__ chi, int64_t n_cand,
                                int R, int32_t *__restrict__ scratch, uint32_t *__restrict__ counts) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n_cand) return;
    int32_t *hdr = scratch;
    int32_t *rings = scratch + kNoallocHeader;
    const int64_t o = offs[i];
    const int N = (int)(offs[i + 1] - o);
    const int64_t eo = o - i;
    uint16_t E[FEM_MAX_NODES];
    int32_t lo[FEM_MAX_NODES], hi[FEM_MAX_NODES];
    int head[FEM_MAX_NODES];
    for (int k = 0; k < N; ++k) {
        E[k] = ctypes[o + k];
        head[k] = 0;
        if (k < N - 1) {
            lo[k] = clo[eo + k];
            hi[k] = chi[eo + k];
        }
    }
    const int64_t stride = n_cand;  // ring (k, r) of episode i at ((k*R + r) * n_cand + i)
    for (int k = 0; k < N - 1; ++k)
        for (int r = 0; r < R; ++r) rings[((int64_t)k * R + r) * stride + i] = INT32_MIN;
    int64_t prev_end = INT64_MIN;
    uint32_t count = 0;
    int ovf = 0;
    for (int64_t j = 0; j < n; ++j) {
        const uint16_t ty = ev_type[j];
        const int32_t t = ev_time[j];
        for (int k = N - 1; k >= 0; --k) {
            if (E[k] != ty) continue;
            bool ok;
            if (k == 0) {
                ok = (int64_t)t > prev_end;
            } else {
                ok = false;
                int idx = head[k - 1];
                for (int q = 0; q < R; ++q) {
                    idx = (idx == 0) ? R - 1 : idx - 1;
                    const int32_t tp = rings[((int64_t)(k - 1) * R + idx) * stride + i];
                    if (tp < t - lo[k - 1]) {
                        ok = tp >= t - hi[k - 1];
                        break;
                    }
                }
            }
            if (!ok) continue;
            if (k == N - 1) {
                count++;
                prev_end = t;
                for (int q = 0; q < N - 1; ++q) {
                    head[q] = 0;
                    for (int r = 0; r < R; ++r) rings[((int64_t)q * R + r) * stride + i] = INT32_MIN;
                }
                break;
            }
            const int h = head[k];
            const int h2 = (h + 1 == R) ? 0 : h + 1;
            int32_t *slotp = &rings[((int64_t)k * R + h) * stride + i];
            const int32_t old = *slotp;
            const int32_t old2 = rings[((int64_t)k * R + h2) * stride + i];
            if (old != INT32_MIN && old >= t - hi[k] && old2 >= t - lo[k]) ovf = 1;
            *slotp = t;
            head[k] = h2;
        }
    }
    counts[i] = count;
    if (ovf) atomicOr(&hdr[0], 2);
}

}  // namespace

extern "C" int fem_count_episodes_noalloc(const uint16_t *types, const int32_t *times, int64_t n,
                                          const int64_t *offs, const uint16_t *ep_types, const int32_t *lo,
                                          const int32_t *hi, int64_t n_cand, uint32_t *counts, void *cuda_stream) {
    if (n < 0 || n_cand < 0) return FEM_ERR_INVAL;
    if (n_cand == 0) return FEM_OK;
    if (!offs || !ep_types || !lo || !hi || !counts || (n > 0 && (!types || !times))) return FEM_ERR_INVAL;
    // At least two ring entries per edge: checked against the largest
    // episode below; every episode has at least one edge or none.
    if ((size_t)n_cand * 2 > kNoallocWords - kNoallocHeader) return FEM_ERR_NOMEM;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kNoallocMaxDevices) return FEM_ERR_CUDA;
    int32_t *scratch = nullptr;
    const int st_setup = noalloc_setup(dev, &scratch);
    if (st_setup != FEM_OK) return st_setup;
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    // The header must start at zero on every call (calls share the array).
    if (cudaMemsetAsync(scratch, 0, kNoallocHeader * sizeof(int32_t), st) != cudaSuccess) return FEM_ERR_CUDA;
    const unsigned blocks = (unsigned)((n_cand + 127) / 128);
    k_noalloc_check<<<blocks, 128, 0, st>>>(offs, ep_types, lo, hi, n_cand, scratch);
    int32_t hdr[2] = {0, 0};
    if (cudaGetLastError() != cudaSuccess ||
        cudaMemcpyAsync(hdr, scratch, sizeof(hdr), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return FEM_ERR_CUDA;
    if (hdr[0] & 1) return FEM_ERR_INVAL;
    const int edges = hdr[1] > 1 ? hdr[1] - 1 : 1;
    const size_t avail = kNoallocWords - kNoallocHeader;
    const int64_t R = (int64_t)std::min<size_t>(kNoallocMaxRing, avail / ((size_t)n_cand * edges));
    if (R < 2) return FEM_ERR_NOMEM;
    k_count_noalloc<<<blocks, 128, 0, st>>>(types, times, n, offs, ep_types, lo, hi, n_cand, (int)R, scratch,
                                            counts);
    if (cudaGetLastError() != cudaSuccess ||
        cudaMemcpyAsync(hdr, scratch, sizeof(int32_t), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return FEM_ERR_CUDA;
    if (hdr[0] & 2) return FEM_ERR_NOMEM;  // the stream's bursts need longer rings than fit
    return FEM_OK;
}
