// Serving loop: counting requests for graphs of different sizes, admitted by
// device memory, several in flight on separate streams, small requests
// grouped into one batched launch.
//
// Threads: one dispatcher and `slots` workers.  The dispatcher scans the
// queue in arrival order and admits every request whose memory estimate fits
// the remaining budget (so small requests are not stuck behind a large one
// that waits for memory); a small admitted request takes further small ones
// that fit along (up to batch_max) and they run as one tg_batch launch.  Each
// worker owns a CUDA stream; the work of different slots overlaps on the GPU.
// Waits are condition-variable waits with a deadline (TG_ETIMEDOUT).
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <new>
#include <set>
#include <thread>
#include <vector>

#include "tg_internal.cuh"

namespace {

using Clock = std::chrono::steady_clock;

struct Request {
    uint64_t ticket = 0;
    int64_t n = 0, m = 0;
    int32_t L = 1, k = 4;
    std::vector<int32_t> src, dst;
    std::vector<uint8_t> type;
    int64_t est = 0;
    Clock::time_point submitted;
};

struct Result {
    int status = TG_OK;
    int cuda_error = 0;  // cudaError_t behind a TG_ECUDA
    std::vector<uint64_t> counts;
    double latency_ms = 0.0;
};

int64_t estimate_bytes(int64_t n, int64_t m, int32_t L) {
    const int64_t L2 = (int64_t)L * L;
    return 96 * m + 64 * n + 8 * n * L2 + 4 * m * L + ((int64_t)1 << 20);
}

}  // namespace

struct tg_server {
    tg_serve_cfg cfg{};
    std::mutex mu;
    std::condition_variable cv_queue;  // dispatcher: new request or freed budget
    std::condition_variable cv_done;   // waiters
    std::condition_variable cv_work;   // workers: new job
    std::deque<std::unique_ptr<Request>> queue;
    std::deque<std::vector<std::unique_ptr<Request>>> jobs;
    std::map<uint64_t, Result> results;
    std::set<uint64_t> pending;  // submitted and not yet returned by tg_serve_wait
    uint64_t next_ticket = 1;
    int64_t bytes_in_flight = 0;
    int jobs_running = 0;
    bool stop = false;
    std::thread dispatcher;
    std::vector<std::thread> workers;
    // statistics
    std::vector<double> latencies;
    uint64_t completed = 0, failed = 0, batched_launches = 0, grouped_requests = 0;
    int64_t peak_bytes = 0;
    int peak_jobs = 0;
    bool have_first = false;
    Clock::time_point first_submit, last_done;
};

namespace {

void run_job(tg_server *sv, std::vector<std::unique_ptr<Request>> &job, cudaStream_t s) {
    std::vector<Result> res(job.size());
    std::vector<tg_graph *> gs(job.size(), nullptr);
    for (size_t q = 0; q < job.size(); ++q) {
        Request &r = *job[q];
        res[q].status = tg_build_csr(r.n, r.m, r.src.data(), r.dst.data(), r.type.data(), r.L, 0, s,
                                     &gs[q]);
        if (res[q].status == TG_ECUDA) res[q].cuda_error = tg_last_cuda_error();
    }
    if (job.size() == 1) {
        Request &r = *job[0];
        if (res[0].status == TG_OK) {
            res[0].counts.assign((size_t)tg_global_len(r.L, r.k), 0);
            res[0].status = tg_count_global(gs[0], r.k, res[0].counts.data(), s);
            if (res[0].status == TG_ECUDA) res[0].cuda_error = tg_last_cuda_error();
        }
    } else {
        // one batched launch for the grouped requests that built
        std::vector<tg_graph *> ok;
        std::vector<size_t> idx;
        std::vector<int64_t> off;
        int64_t total = 0;
        for (size_t q = 0; q < job.size(); ++q)
            if (res[q].status == TG_OK) {
                ok.push_back(gs[q]);
                idx.push_back(q);
                off.push_back(total);
                total += tg_global_len(job[q]->L, job[q]->k);
            }
        int st = TG_OK;
        uint64_t *d = nullptr;
        if (!ok.empty()) {
            d = (uint64_t *)tg_dalloc((size_t)total * 8, s);
            if (!d) st = TG_ENOMEM;
            std::vector<uint64_t *> outs;
            for (size_t q = 0; q < ok.size() && st == TG_OK; ++q) outs.push_back(d + off[q]);
            // requests of one group share k (the dispatcher groups by k)
            // small requests: the single persistent launch (no union build, no
            // per-launch autotuning on the serving path)
            tg_tune fixed{};
            fixed.kernel = TG_KERNEL_WARP_SEARCH;
            fixed.cta_threads = 256;
            if (st == TG_OK)
                st = tg_count_batch((int32_t)ok.size(), ok.data(), job[idx[0]]->k, TG_BATCH_GLOBAL,
                                    outs.data(), &fixed, s);
            int cerr = st == TG_ECUDA ? tg_last_cuda_error() : 0;
            std::vector<uint64_t> host((size_t)total);
            if (st == TG_OK) {
                cudaError_t e = cudaMemcpyAsync(host.data(), d, (size_t)total * 8,
                                                cudaMemcpyDeviceToHost, s);
                if (e == cudaSuccess) e = cudaStreamSynchronize(s);
                if (e != cudaSuccess) {
                    st = TG_ECUDA;
                    cerr = (int)e;
                }
            }
            for (size_t q = 0; q < ok.size(); ++q) {
                Result &rr = res[idx[q]];
                rr.status = st;
                rr.cuda_error = cerr;
                if (st == TG_OK) {
                    const int64_t len = tg_global_len(job[idx[q]]->L, job[idx[q]]->k);
                    rr.counts.assign(host.begin() + off[q], host.begin() + off[q] + len);
                }
            }
            if (d) tg_dfree(d, (size_t)total * 8, s);
            (void)cudaStreamSynchronize(s);
        }
    }
    for (tg_graph *g : gs)
        if (g) tg_free_graph_on(g, s);  // used on this stream only
    (void)cudaStreamSynchronize(s);
    const auto now = Clock::now();
    std::lock_guard<std::mutex> lk(sv->mu);
    for (size_t q = 0; q < job.size(); ++q) {
        Request &r = *job[q];
        res[q].latency_ms =
            std::chrono::duration<double, std::milli>(now - r.submitted).count();
        if (res[q].status == TG_OK) {
            ++sv->completed;
            sv->latencies.push_back(res[q].latency_ms);
        } else {
            ++sv->failed;
        }
        sv->bytes_in_flight -= r.est;
        sv->results[r.ticket] = std::move(res[q]);
    }
    if (job.size() > 1) {
        ++sv->batched_launches;
        sv->grouped_requests += job.size();
    }
    --sv->jobs_running;
    sv->last_done = now;
    sv->cv_done.notify_all();
    sv->cv_queue.notify_all();
}

void worker_main(tg_server *sv) {
    (void)cudaSetDevice(sv->cfg.device);
    cudaStream_t s = nullptr;
    (void)cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
    for (;;) {
        std::vector<std::unique_ptr<Request>> job;
        {
            std::unique_lock<std::mutex> lk(sv->mu);
            sv->cv_work.wait(lk, [&] { return sv->stop || !sv->jobs.empty(); });
            if (sv->jobs.empty()) break;  // stop requested and nothing left
            job = std::move(sv->jobs.front());
            sv->jobs.pop_front();
        }
        run_job(sv, job, s);
    }
    (void)cudaStreamDestroy(s);
}

void dispatcher_main(tg_server *sv) {
    (void)cudaSetDevice(sv->cfg.device);
    std::unique_lock<std::mutex> lk(sv->mu);
    for (;;) {
        sv->cv_queue.wait(lk, [&] {
            return sv->stop || (!sv->queue.empty() && sv->jobs_running < sv->cfg.slots);
        });
        if (sv->stop && sv->queue.empty()) break;
        if (sv->stop) {
            // refuse what is still queued
            for (auto &r : sv->queue) {
                Result rr;
                rr.status = TG_EBUSY;
                sv->results[r->ticket] = std::move(rr);
                ++sv->failed;
            }
            sv->queue.clear();
            sv->cv_done.notify_all();
            break;
        }
        bool admitted = false;
        for (auto it = sv->queue.begin(); it != sv->queue.end() && sv->jobs_running < sv->cfg.slots;) {
            Request &r = **it;
            if (sv->bytes_in_flight + r.est > sv->cfg.mem_budget_bytes) {
                ++it;
                continue;
            }
            std::vector<std::unique_ptr<Request>> job;
            sv->bytes_in_flight += r.est;
            const bool small = r.m <= sv->cfg.batch_edges;
            const int32_t k = r.k;
            job.push_back(std::move(*it));
            it = sv->queue.erase(it);
            if (small) {
                for (auto jt = it; jt != sv->queue.end() && (int)job.size() < sv->cfg.batch_max;) {
                    Request &x = **jt;
                    if (x.m <= sv->cfg.batch_edges && x.k == k &&
                        sv->bytes_in_flight + x.est <= sv->cfg.mem_budget_bytes) {
                        sv->bytes_in_flight += x.est;
                        job.push_back(std::move(*jt));
                        jt = sv->queue.erase(jt);
                    } else {
                        ++jt;
                    }
                }
                it = sv->queue.begin();
            }
            sv->jobs.push_back(std::move(job));
            ++sv->jobs_running;
            sv->peak_jobs = std::max(sv->peak_jobs, sv->jobs_running);
            sv->peak_bytes = std::max(sv->peak_bytes, sv->bytes_in_flight);
            admitted = true;
            sv->cv_work.notify_one();
        }
        if (!admitted) {
            // nothing fits now: wait for a job to finish (bounded, re-checked)
            sv->cv_queue.wait_for(lk, std::chrono::milliseconds(50));
        }
    }
}

}  // namespace

extern "C" tg_server *tg_serve_create(const tg_serve_cfg *cfg) {
    tg_server *sv = new (std::nothrow) tg_server();
    if (!sv) return nullptr;
    tg_serve_cfg c{};
    c.slots = 4;
    c.mem_budget_bytes = (int64_t)8 << 30;
    c.queue_cap = 4096;
    c.device = 0;
    c.batch_max = 32;
    c.batch_edges = 20000;
    if (cfg) {
        if (cfg->slots > 0) c.slots = cfg->slots;
        if (cfg->mem_budget_bytes > 0) c.mem_budget_bytes = cfg->mem_budget_bytes;
        if (cfg->queue_cap > 0) c.queue_cap = cfg->queue_cap;
        c.device = cfg->device;
        if (cfg->batch_max > 0) c.batch_max = cfg->batch_max;
        if (cfg->batch_edges >= 0) c.batch_edges = cfg->batch_edges;
    }
    sv->cfg = c;
    try {
        sv->dispatcher = std::thread(dispatcher_main, sv);
        for (int w = 0; w < c.slots; ++w) sv->workers.emplace_back(worker_main, sv);
    } catch (...) {
        {
            std::lock_guard<std::mutex> lk(sv->mu);
            sv->stop = true;
        }
        sv->cv_queue.notify_all();
        sv->cv_work.notify_all();
        if (sv->dispatcher.joinable()) sv->dispatcher.join();
        for (auto &t : sv->workers)
            if (t.joinable()) t.join();
        delete sv;
        return nullptr;
    }
    return sv;
}

extern "C" int tg_serve_submit(tg_server *sv, const tg_request *req, uint64_t *ticket) {
    if (!sv || !req || !ticket) return TG_EINVAL;
    if (req->n < 1 || req->n > TG_MAX_NODES || req->m < 0 || req->L < 1 || req->L > TG_MAX_TYPES ||
        (req->k != 3 && req->k != 4) || (req->m > 0 && (!req->src || !req->dst)) || !req->type)
        return TG_EINVAL;
    for (int64_t v = 0; v < req->n; ++v)
        if (req->type[v] >= req->L) return TG_EINVAL;
    for (int64_t e = 0; e < req->m; ++e)
        if (req->src[e] < 0 || req->src[e] >= req->n || req->dst[e] < 0 || req->dst[e] >= req->n)
            return TG_EINVAL;
    const int64_t est = estimate_bytes(req->n, req->m, req->L);
    if (est > sv->cfg.mem_budget_bytes) return TG_ENOMEM_ADMIT;
    auto r = std::unique_ptr<Request>(new (std::nothrow) Request());
    if (!r) return TG_ENOMEM;
    r->n = req->n;
    r->m = req->m;
    r->L = req->L;
    r->k = req->k;
    r->est = est;
    try {
        r->src.assign(req->src, req->src + req->m);
        r->dst.assign(req->dst, req->dst + req->m);
        r->type.assign(req->type, req->type + req->n);
    } catch (...) {
        return TG_ENOMEM;
    }
    std::lock_guard<std::mutex> lk(sv->mu);
    if (sv->stop) return TG_EINVAL;
    if ((int)sv->queue.size() >= sv->cfg.queue_cap) return TG_EBUSY;
    r->ticket = sv->next_ticket++;
    r->submitted = Clock::now();
    if (!sv->have_first) {
        sv->have_first = true;
        sv->first_submit = r->submitted;
    }
    *ticket = r->ticket;
    sv->pending.insert(r->ticket);
    sv->queue.push_back(std::move(r));
    sv->cv_queue.notify_all();
    return TG_OK;
}

extern "C" int tg_serve_wait(tg_server *sv, uint64_t ticket, int32_t timeout_ms, uint64_t *out,
                             int64_t out_len, tg_result *info) {
    if (!sv) return TG_EINVAL;
    std::unique_lock<std::mutex> lk(sv->mu);
    if (sv->pending.find(ticket) == sv->pending.end()) return TG_ENOTFOUND;
    const auto deadline = Clock::now() + std::chrono::milliseconds(timeout_ms < 0 ? 0 : timeout_ms);
    while (sv->results.find(ticket) == sv->results.end()) {
        if (sv->cv_done.wait_until(lk, deadline) == std::cv_status::timeout &&
            sv->results.find(ticket) == sv->results.end())
            return TG_ETIMEDOUT;
    }
    auto it = sv->results.find(ticket);
    Result &r = it->second;
    if (info) {
        info->status = r.status;
        info->cuda_error = r.cuda_error;
        info->len = (int64_t)r.counts.size();
        info->latency_ms = r.latency_ms;
    }
    const int st = r.status;
    if (st == TG_OK) {
        if (!out || out_len < (int64_t)r.counts.size()) return TG_EINVAL;  // result kept
        std::copy(r.counts.begin(), r.counts.end(), out);
    }
    sv->results.erase(it);
    sv->pending.erase(ticket);
    return st;
}

extern "C" int tg_serve_stats(tg_server *sv, tg_serve_stats_t *st) {
    if (!sv || !st) return TG_EINVAL;
    std::lock_guard<std::mutex> lk(sv->mu);
    std::vector<double> l = sv->latencies;
    std::sort(l.begin(), l.end());
    auto pct = [&](double q) -> double {
        if (l.empty()) return 0.0;
        size_t i = (size_t)(q * (double)(l.size() - 1) + 0.5);
        return l[std::min(i, l.size() - 1)];
    };
    st->completed = sv->completed;
    st->failed = sv->failed;
    st->queued = sv->queue.size();
    st->p50_ms = pct(0.50);
    st->p99_ms = pct(0.99);
    st->max_ms = l.empty() ? 0.0 : l.back();
    double span = 0.0;
    if (sv->have_first && sv->completed)
        span = std::chrono::duration<double>(sv->last_done - sv->first_submit).count();
    st->graphs_per_s = span > 0 ? (double)sv->completed / span : 0.0;
    st->peak_in_flight = sv->peak_jobs;
    st->peak_bytes = sv->peak_bytes;
    st->batched_launches = sv->batched_launches;
    st->grouped_requests = sv->grouped_requests;
    return TG_OK;
}

extern "C" void tg_serve_destroy(tg_server *sv) {
    if (!sv) return;
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        sv->stop = true;
    }
    sv->cv_queue.notify_all();
    if (sv->dispatcher.joinable()) sv->dispatcher.join();
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        sv->cv_work.notify_all();
    }
    for (auto &t : sv->workers)
        if (t.joinable()) t.join();
    delete sv;
}
