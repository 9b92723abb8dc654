// fem_serve.cu -- serving loop for level-wise mining jobs with continuous
// batching.
//
// One worker thread owns a context.  Each tick it
//   1. admits waiting jobs, in arrival order, while a slot is free and the
//      job's estimated device memory fits next to what the context already
//      holds (the stream is uploaded once and stays resident);
//   2. counts the current candidates of every admitted job -- each job at
//      its own level -- in one batched counting call;
//   3. advances every job by one level (threshold, next candidates); jobs
//      that finish hand their result to the waiter and release their memory,
//      which lets waiting jobs in on the next tick.
// Jobs arriving while others are on the GPU therefore join the running batch
// as soon as a slot and memory are free.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <vector>

#include "fem_internal.cuh"

namespace {

struct Job {
    uint64_t id = 0;
    std::vector<uint16_t> types;
    std::vector<int32_t> times;
    uint32_t n_types = 0;
    std::vector<int32_t> blo, bhi;
    uint32_t thr = 0;
    int max_size = 0;
    size_t mem_est = 0;
    fem_stream *s = nullptr;
    fem::MineGroup *g = nullptr;
    fem_result *res = nullptr;
    fem_job_info info{};
    int status = FEM_OK;
    bool done = false;
    int requeues = 0;
};

}  // namespace

struct fem_server {
    fem_ctx *ctx = nullptr;
    int max_jobs = 1;
    std::thread worker;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<Job *> pending;
    std::vector<Job *> active;
    std::map<uint64_t, Job *> jobs;
    uint64_t next_id = 1;
    bool stop = false;
};

namespace {

// Device memory a job is expected to hold: its stream (6 B per event plus
// padding), level-2 candidate arrays and the pair-bound table (both at most
// quadratic in the alphabet), and a fixed allowance for the rest.
size_t estimate_job_bytes(int64_t n, uint32_t n_types, int nb) {
    // stream (6 B/event) + per-type lists (4 B/event kept, 8 B/event while built)
    const size_t stream = (size_t)(n + fem::kPadEvents) * 18;
    const size_t pairs = (size_t)n_types * n_types * (size_t)std::max(nb, 1);
    return stream + pairs * 48 + (size_t)16 * 1024 * 1024;
}

void finish_job(fem_server *srv, Job *j, int status) {
    if (j->g) {
        if (j->res) fem::result_set_stats(j->res, fem::mg_stats(j->g));
        fem::mg_destroy(j->g);
        j->g = nullptr;
    }
    if (j->s) {
        fem::stream_free_unlocked(j->s);
        j->s = nullptr;
    }
    if (status != FEM_OK && j->res) {
        fem_result_free(j->res);
        j->res = nullptr;
    }
    j->info.finish_s = fem::now_s();
    std::lock_guard<std::mutex> g(srv->mu);
    j->status = status;
    j->done = true;
    j->types.clear();
    j->types.shrink_to_fit();
    j->times.clear();
    j->times.shrink_to_fit();
    srv->cv_done.notify_all();
}

// Releases a job's device state and puts it back at the head of the queue:
// it ran out of device memory next to other resident jobs and will be
// retried once memory has been freed.
void requeue_job(fem_server *srv, Job *j) {
    if (j->g) {
        fem::mg_destroy(j->g);
        j->g = nullptr;
    }
    if (j->s) {
        fem::stream_free_unlocked(j->s);
        j->s = nullptr;
    }
    if (j->res) {
        fem_result_free(j->res);
        j->res = nullptr;
    }
    j->status = FEM_OK;
    j->requeues++;
    std::lock_guard<std::mutex> g(srv->mu);
    srv->pending.push_front(j);
}

// Uploads and starts one job (level 1, level-2 candidates).
int start_job(fem_server *srv, Job *j) {
    fem_ctx *ctx = srv->ctx;
    const int64_t n = (int64_t)j->times.size();
    FEM_TRY(fem::load_stream_unlocked(ctx, j->types.data(), j->times.data(), n, j->n_types, 0, &j->s));
    j->res = fem::result_new(1, j->max_size);
    if (!j->res) return FEM_ERR_NOMEM;
    j->g = fem::mg_create(ctx, j->s, j->blo, j->bhi, j->thr, j->max_size, j->res);
    if (!j->g) return FEM_ERR_NOMEM;
    return fem::mg_begin(j->g);
}

void worker_loop(fem_server *srv) {
    fem_ctx *ctx = srv->ctx;
    cudaSetDevice(ctx->device);
    for (;;) {
        std::vector<Job *> admit;
        {
            std::unique_lock<std::mutex> lk(srv->mu);
            srv->cv_work.wait(lk, [&] { return srv->stop || !srv->pending.empty() || !srv->active.empty(); });
            if (srv->stop) break;
            size_t planned = 0;
            while (!srv->pending.empty() && (int)(srv->active.size() + admit.size()) < srv->max_jobs) {
                Job *j = srv->pending.front();
                const bool empty = srv->active.empty() && admit.empty();
                // a job that ran out of memory next to others re-enters only
                // when at most one other job is resident
                if (j->requeues > 0 && srv->active.size() + admit.size() > 1) break;
                if (!empty && ctx->used.load() + planned + j->mem_est > ctx->budget) break;
                srv->pending.pop_front();
                planned += j->mem_est;
                admit.push_back(j);
            }
        }
        {
            std::lock_guard<std::mutex> cg(ctx->mu);
            for (Job *j : admit) {
                j->info.admit_s = fem::now_s();
                const int st = start_job(srv, j);
                if (st == FEM_ERR_NOMEM && !srv->active.empty()) {
                    requeue_job(srv, j);
                } else if (st != FEM_OK) {
                    finish_job(srv, j, st);
                } else if (fem::mg_done(j->g)) {
                    finish_job(srv, j, FEM_OK);
                } else {
                    srv->active.push_back(j);
                }
            }
            if (srv->active.empty()) continue;
            std::vector<fem::MineGroup *> gs;
            for (Job *j : srv->active) gs.push_back(j->g);
            int st = fem::mg_count_batch(ctx, gs);
            if (st == FEM_ERR_NOMEM && gs.size() > 1) {
                // the batch does not fit next to the resident jobs: count the
                // jobs one at a time (each job then fails or succeeds alone)
                st = FEM_OK;
                for (auto *g1 : gs) {
                    const int s1 = fem::mg_count_batch(ctx, {g1});
                    if (s1 != FEM_OK) {
                        for (Job *j : srv->active)
                            if (j->g == g1) j->status = s1;
                    }
                }
            }
            std::vector<Job *> still;
            for (Job *j : srv->active) {
                int sj = st != FEM_OK ? st : j->status;
                if (sj == FEM_OK) sj = fem::mg_advance(j->g);
                if (sj == FEM_ERR_NOMEM && srv->active.size() > 1 && j->requeues < 64) {
                    requeue_job(srv, j);
                } else if (sj != FEM_OK) {
                    finish_job(srv, j, sj);
                } else if (fem::mg_done(j->g)) {
                    const fem_stats &S = fem::mg_stats(j->g);
                    j->info.levels = S.levels;
                    j->info.candidates_counted = S.candidates_counted;
                    j->info.episode_events = S.episode_events;
                    finish_job(srv, j, FEM_OK);
                } else {
                    still.push_back(j);
                }
            }
            srv->active.swap(still);
        }
    }
    // stop: cancel what is still resident
    std::lock_guard<std::mutex> cg(ctx->mu);
    for (Job *j : srv->active) finish_job(srv, j, FEM_ERR_BUSY);
    srv->active.clear();
}

}  // namespace

extern "C" int fem_server_create(int device, size_t hbm_budget_bytes, int max_jobs, fem_server **out) {
    if (!out || max_jobs < 1) return FEM_ERR_INVAL;
    *out = nullptr;
    if (hbm_budget_bytes == 0) {
        if (cudaSetDevice(device) != cudaSuccess) return FEM_ERR_INVAL;
        size_t fr = 0, tot = 0;
        cudaMemGetInfo(&fr, &tot);
        hbm_budget_bytes = (size_t)(0.8 * (double)fr);
    }
    fem_server *srv = new (std::nothrow) fem_server();
    if (!srv) return FEM_ERR_NOMEM;
    const int st = fem_ctx_create(device, hbm_budget_bytes, nullptr, &srv->ctx);
    if (st != FEM_OK) {
        delete srv;
        return st;
    }
    srv->max_jobs = max_jobs;
    try {
        srv->worker = std::thread(worker_loop, srv);
    } catch (...) {
        fem_ctx_destroy(srv->ctx);
        delete srv;
        return FEM_ERR_NOMEM;
    }
    *out = srv;
    return FEM_OK;
}

extern "C" int fem_server_submit(fem_server *srv, const uint16_t *types, const int32_t *times, int64_t n,
                                 uint32_t n_types, const int32_t *bin_lo, const int32_t *bin_hi, int n_bins,
                                 uint32_t threshold, int max_size, uint64_t *job_id) {
    if (!srv || !job_id || n < 0 || (n > 0 && (!types || !times)) || n_types < 1 || n_types > 65536 ||
        max_size < 1 || max_size > FEM_MAX_NODES || n_bins < 0 || (n_bins > 0 && (!bin_lo || !bin_hi)) ||
        (max_size > 1 && n_bins < 1))
        return FEM_ERR_INVAL;
    Job *j = new (std::nothrow) Job();
    if (!j) return FEM_ERR_NOMEM;
    std::vector<std::pair<int32_t, int32_t>> bins;
    for (int b = 0; b < n_bins; ++b) {
        if (bin_lo[b] < 0 || bin_lo[b] >= bin_hi[b]) {
            delete j;
            return FEM_ERR_INVAL;
        }
        bins.push_back({bin_lo[b], bin_hi[b]});
    }
    std::sort(bins.begin(), bins.end());
    bins.erase(std::unique(bins.begin(), bins.end()), bins.end());
    for (auto &b : bins) {
        j->blo.push_back(b.first);
        j->bhi.push_back(b.second);
    }
    try {
        j->types.assign(types, types + n);
        j->times.assign(times, times + n);
    } catch (...) {
        delete j;
        return FEM_ERR_NOMEM;
    }
    j->n_types = n_types;
    j->thr = threshold;
    j->max_size = max_size;
    j->mem_est = estimate_job_bytes(n, n_types, (int)bins.size());
    if (j->mem_est > srv->ctx->budget) {
        delete j;
        return FEM_ERR_NOMEM;
    }
    j->info.n_events = n;
    {
        std::lock_guard<std::mutex> g(srv->mu);
        j->id = srv->next_id++;
        j->info.submit_s = fem::now_s();
        srv->jobs[j->id] = j;
        srv->pending.push_back(j);
    }
    srv->cv_work.notify_one();
    *job_id = j->id;
    return FEM_OK;
}

extern "C" int fem_server_wait(fem_server *srv, uint64_t job_id, int timeout_ms, fem_result **out,
                               fem_job_info *info) {
    if (!srv || !out) return FEM_ERR_INVAL;
    *out = nullptr;
    std::unique_lock<std::mutex> lk(srv->mu);
    auto it = srv->jobs.find(job_id);
    if (it == srv->jobs.end()) return FEM_ERR_NOTFOUND;
    Job *j = it->second;
    auto ready = [&] { return j->done; };
    if (timeout_ms < 0)
        srv->cv_done.wait(lk, ready);
    else if (!srv->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), ready))
        return FEM_ERR_BUSY;
    srv->jobs.erase(it);
    lk.unlock();
    const int st = j->status;
    if (info) *info = j->info;
    *out = j->res;
    delete j;
    return st;
}

extern "C" void fem_server_destroy(fem_server *srv) {
    if (!srv) return;
    {
        std::lock_guard<std::mutex> g(srv->mu);
        srv->stop = true;
    }
    srv->cv_work.notify_all();
    if (srv->worker.joinable()) srv->worker.join();
    for (auto &kv : srv->jobs) {
        Job *j = kv.second;
        if (j->res) fem_result_free(j->res);
        delete j;
    }
    srv->jobs.clear();
    fem_ctx_destroy(srv->ctx);
    delete srv;
}
