// The serving loop: a native request scheduler over the library's own
// entry points.  Clients submit factor+solve / solve / invert requests of
// uneven order from any thread; one scheduler thread admits them onto the
// GPU as soon as a stream slot and arena memory are free, so work that
// arrives while other requests run overlaps with it on the device
// (continuous batching):
//   * small factor+solve requests (n <= small_n, nrhs <= 32) are gathered
//     into one launch of the batched kernel whenever a batch stream is idle:
//     everything that arrived meanwhile goes into the next batch.  A
//     mixed-mode request of order <= small_n is served in FP64 like the
//     others: the FP64 result meets the mixed mode's accuracy, and at these
//     orders FP64 is at least as fast;
//   * every other request runs on its own stream: FP64 PFTRF + PFTRS
//     (Sections 3-4), the mixed-precision solve, or PFTRI on a copy of a
//     resident factor.
// All device memory comes from one arena allocated at creation; RFP arrays
// stay resident under the caller's key (least recently used evicted first,
// never while in use), i.e. the cache is admitted by RFP bytes n(n+1)/2 * 8.
// Completion times are taken by host callbacks enqueued behind each
// request's result copies; CUDA events around each request's (or batch's)
// GPU work give its device-clock start and end.
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <memory>
#include <mutex>
#include <thread>
#include <unordered_set>
#include <vector>

#include "../../include/rfp.h"
#include "serve_pool.h"

namespace {

using rfp::serve::Arena;
using rfp::serve::CacheEntry;
using rfp::serve::FactorCache;
using rfp::serve::Held;

constexpr int kMaxStreams = 64;
constexpr int kBatchStreams = 2;
constexpr int kSlots = 1 << 15;   // pinned result slots (in-flight jobs)
constexpr int kBatchRhs = 32;     // right-hand sides a batched request may have
// Precision of the mixed-mode solves: the split-BF16 factor, as fast as the
// split-TF32 one at kappa <= 1e4 and faster at 1e6 (fewer refinement steps).
constexpr int kServeMixedPrec = RFP_PREC_BF16X6;

struct ResultSlot {               // pinned host memory, written by D2H copies
    int32_t info;
    int32_t pad;
    rfp_mixed_status_t st;
};

struct Job {
    rfp_serve_request_t req;
    double t_submit = 0, t_start = 0, t_done = 0;
    int64_t arf_off = -1;         // the RFP array (cache entry or temporary)
    bool arf_cached = false;      // arf_off belongs to the cache entry req.key
    bool hit = false, batched = false;
    int64_t b_off = -1, x_off = -1, work_off = -1, tmp_off = -1, stat_off = -1;
    int slot = -1;                // ResultSlot index
    int stream = -1;              // stream slot (-1: batched)
    int32_t status = 0;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;   // around its GPU work (stream jobs)
    double gpu_start_ms = 0, gpu_end_ms = 0;
};

struct Batch {
    std::vector<Job *> jobs;
    int64_t plan_off = -1, info_off = -1;
    int stream = -1;
    double t_done = 0;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;   // around the batch's GPU work
};

double now_s(std::chrono::steady_clock::time_point t0)
{
    return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
}

size_t rfp_bytes(int64_t n) { return (size_t)(n * (n + 1) / 2) * sizeof(double); }

class Server {
public:
    explicit Server(const rfp_serve_config_t &cfg) : cfg_(cfg), arena_(cfg.arena_bytes), cache_(arena_)
    {
        t0_ = std::chrono::steady_clock::now();
    }

    int init()
    {
        if (cudaGetDevice(&dev_) != cudaSuccess) return RFP_ERR_CUDA;
        if (cudaMalloc(&base_, arena_.capacity()) != cudaSuccess) return RFP_ERR_CUDA;
        if (cudaMallocHost(&slots_, sizeof(ResultSlot) * kSlots) != cudaSuccess) return RFP_ERR_CUDA;
        for (int i = kSlots - 1; i >= 0; --i) free_slots_.push_back(i);
        const int ns = cfg_.streams + kBatchStreams;
        streams_.resize(ns);
        for (int i = 0; i < ns; ++i)
            if (cudaStreamCreateWithFlags(&streams_[i], cudaStreamNonBlocking) != cudaSuccess)
                return RFP_ERR_CUDA;
        for (int i = 0; i < cfg_.streams; ++i) free_streams_.push_back(i);
        // reference point of the device-clock stamps
        if (cudaEventCreate(&ref_) != cudaSuccess || cudaEventRecord(ref_, streams_[0]) != cudaSuccess ||
            cudaEventSynchronize(ref_) != cudaSuccess)
            return RFP_ERR_CUDA;
        for (int i = 0; i < kBatchStreams; ++i) free_batch_streams_.push_back(cfg_.streams + i);
        worker_ = std::thread([this] { run(); });
        return RFP_OK;
    }

    ~Server()
    {
        {
            std::lock_guard<std::mutex> lk(mu_);
            stop_ = true;
        }
        cv_.notify_all();
        if (worker_.joinable()) worker_.join();
        for (auto s : streams_) if (s) cudaStreamDestroy(s);
        for (auto ev : free_events_) cudaEventDestroy(ev);
        if (ref_) cudaEventDestroy(ref_);
        if (slots_) cudaFreeHost(slots_);
        if (base_) cudaFree(base_);
    }

    int submit(const rfp_serve_request_t &r)
    {
        auto j = std::make_unique<Job>();
        j->req = r;
        j->t_submit = now_s(t0_);
        {
            std::lock_guard<std::mutex> lk(mu_);
            if (stop_) return -1;
            incoming_.push_back(std::move(j));
            ++submitted_;
        }
        cv_.notify_all();
        return RFP_OK;
    }

    int poll(rfp_serve_completion_t *out, int max, double timeout_s)
    {
        std::unique_lock<std::mutex> lk(cmu_);
        if (completions_.empty() && timeout_s > 0)
            ccv_.wait_for(lk, std::chrono::duration<double>(timeout_s),
                          [&] { return !completions_.empty(); });
        int k = 0;
        while (k < max && !completions_.empty()) {
            out[k++] = completions_.front();
            completions_.pop_front();
        }
        return k;
    }

    void stats(rfp_serve_stats_t *s)
    {
        std::lock_guard<std::mutex> lk(smu_);
        *s = stats_;
        std::lock_guard<std::mutex> lk2(mu_);
        s->submitted = submitted_;
    }

private:
    // ---- callbacks (CUDA host-function thread: no CUDA calls here) ----
    struct Done {
        Server *srv;
        Job *job;
        Batch *batch;
    };
    static void CUDART_CB on_done(void *p)
    {
        Done *d = static_cast<Done *>(p);
        const double t = now_s(d->srv->t0_);
        {
            // Notify while holding the lock: once it is released the scheduler
            // may retire this last job and the server may be destroyed, so the
            // callback must not touch the server after unlocking.
            std::lock_guard<std::mutex> lk(d->srv->mu_);
            if (d->job) {
                d->job->t_done = t;
                d->srv->done_jobs_.push_back(d->job);
            } else {
                d->batch->t_done = t;
                d->srv->done_batches_.push_back(d->batch);
            }
            d->srv->cv_.notify_all();
        }
        delete d;
    }

    double *dptr(int64_t off) { return reinterpret_cast<double *>(static_cast<char *>(base_) + off); }

    void complete(Job *j)
    {
        rfp_serve_completion_t c{};
        c.id = j->req.id;
        c.status = j->status;
        c.cache_hit = j->hit ? 1 : 0;
        c.batched = j->batched ? 1 : 0;
        c.t_submit = j->t_submit;
        c.t_start = j->t_start;
        c.t_done = j->t_done;
        c.gpu_start_ms = j->gpu_start_ms;
        c.gpu_end_ms = j->gpu_end_ms;
        if (j->slot >= 0 && !fp64_path(j->req) && j->req.op != RFP_SERVE_OP_INVERT) {
            c.iterations = slots_[j->slot].st.iterations;
            c.backward_error = slots_[j->slot].st.backward_error;
        }
        {   // counted before it becomes visible to poll()
            std::lock_guard<std::mutex> lk(smu_);
            ++stats_.completed;
            if (j->hit) ++stats_.cache_hits;
        }
        {
            std::lock_guard<std::mutex> lk(cmu_);
            completions_.push_back(c);
        }
        ccv_.notify_all();
    }

    void fail(Job *j, int32_t status)
    {
        j->status = status;
        j->t_start = j->t_done = now_s(t0_);
        complete(j);
    }

    // Release a finished job's buffers; keep its RFP array resident when it
    // holds a valid result under the job's key.
    void retire(Job *j)
    {
        int32_t status = 0;
        if (j->slot >= 0) {
            const ResultSlot &s = slots_[j->slot];
            if (!fp64_path(j->req) && j->req.op != RFP_SERVE_OP_INVERT) {
                if (s.st.info) status = s.st.info;
                else if (s.st.tc_error) status = RFP_SERVE_ECUDA;
                else if (!s.st.converged) status = RFP_SERVE_ENOCONV;
            } else {
                status = s.info;
            }
        }
        if (j->status == 0) j->status = status;
        for (int64_t *off : {&j->b_off, &j->x_off, &j->work_off, &j->tmp_off, &j->stat_off})
            if (*off >= 0) {
                arena_.release(*off);
                *off = -1;
            }
        if (j->arf_cached) {
            CacheEntry *e = cache_.find(j->req.key);
            if (e) {
                --e->pins;
                // a failed factorization leaves no valid factor behind
                if (j->status > 0 && e->held == Held::Factor64 && !j->hit) cache_.erase(j->req.key);
            }
        } else if (j->arf_off >= 0) {
            arena_.release(j->arf_off);
        }
        j->arf_off = -1;
        if (j->slot >= 0) free_slots_.push_back(j->slot);
        if (j->stream >= 0) free_streams_.push_back(j->stream);
        if (j->ev0 && j->ev1) {   // its GPU work is complete (the callback came after ev1)
            j->gpu_start_ms = event_ms(j->ev0);
            j->gpu_end_ms = event_ms(j->ev1);
        }
        put_event(j->ev0);
        put_event(j->ev1);
        j->ev0 = j->ev1 = nullptr;
        complete(j);
        jobs_.erase(j);
    }

    // FP64 requests, and mixed-mode requests of order <= small_n, run the
    // FP64 path (their array is held as an FP64 factor).
    bool fp64_path(const rfp_serve_request_t &r) const
    {
        return r.mode == RFP_SERVE_MODE_FP64 || (cfg_.small_n > 0 && r.n <= cfg_.small_n);
    }

    bool is_small(const Job *j) const
    {
        const auto &r = j->req;
        return r.op == RFP_SERVE_OP_FACTOR_SOLVE && fp64_path(r) && r.n <= cfg_.small_n &&
               r.nrhs <= kBatchRhs;
    }

    // Event pool for the device-clock stamps.
    cudaEvent_t get_event()
    {
        if (!free_events_.empty()) {
            cudaEvent_t e = free_events_.back();
            free_events_.pop_back();
            return e;
        }
        cudaEvent_t e = nullptr;
        return cudaEventCreate(&e) == cudaSuccess ? e : nullptr;
    }
    void put_event(cudaEvent_t e)
    {
        if (e) free_events_.push_back(e);
    }
    double event_ms(cudaEvent_t e)
    {
        float ms = 0.f;
        return cudaEventElapsedTime(&ms, ref_, e) == cudaSuccess ? (double)ms : 0.0;
    }

    int64_t alloc(size_t bytes) { return cache_.alloc_evicting(bytes); }

    // The job's RFP array: the resident entry (hit), a new cache entry, or a
    // temporary.  Returns false if the arena cannot hold it now.
    bool place_arf(Job *j, Held want)
    {
        const auto &r = j->req;
        if (r.key >= 0) {
            CacheEntry *e = cache_.find(r.key);
            if (e && e->held == want && e->n == r.n && e->transr == r.transr && e->uplo == r.uplo) {
                ++e->pins;
                j->arf_off = e->offset;
                j->arf_cached = true;
                j->hit = true;
                return true;
            }
            if (e && e->pins == 0) cache_.erase(r.key);   // stale entry under this key: replace
        }
        const int64_t off = alloc(rfp_bytes(r.n));
        if (off < 0) return false;
        j->arf_off = off;
        if (r.key >= 0 && !cache_.find(r.key)) {
            CacheEntry e{r.key, off, rfp_bytes(r.n), r.n, r.transr, r.uplo, want, 1};
            cache_.insert(e);
            j->arf_cached = true;
        }
        return true;
    }

    // Undo a partial reservation (the job stays pending).
    void unreserve(Job *j)
    {
        for (int64_t *off : {&j->b_off, &j->x_off, &j->work_off, &j->tmp_off, &j->stat_off})
            if (*off >= 0) {
                arena_.release(*off);
                *off = -1;
            }
        if (j->arf_cached) {
            CacheEntry *e = cache_.find(j->req.key);
            if (e) {
                --e->pins;
                if (!j->hit) cache_.erase(j->req.key);
            }
        } else if (j->arf_off >= 0) {
            arena_.release(j->arf_off);
        }
        j->arf_off = -1;
        j->arf_cached = j->hit = false;
    }

    // Bytes a job needs beyond its RFP array (for the too-large check).
    size_t extra_bytes(const Job *j) const
    {
        const auto &r = j->req;
        const size_t bx = (size_t)r.n * (size_t)r.nrhs * sizeof(double);
        if (r.op == RFP_SERVE_OP_INVERT) return rfp_bytes(r.n) + 256;
        if (!fp64_path(r))
            return 2 * bx + rfp_dpfsv_mixed_workspace(r.n, r.nrhs, kServeMixedPrec) + 3 * 256;
        return bx + 256;
    }

    // Reserve everything a stream job needs; false = not now (retry later).
    bool reserve_stream_job(Job *j)
    {
        const auto &r = j->req;
        const size_t bx = (size_t)r.n * (size_t)r.nrhs * sizeof(double);
        const bool mixed = !fp64_path(r);
        if (r.op == RFP_SERVE_OP_FACTOR_SOLVE) {
            if (!place_arf(j, mixed ? Held::Matrix64 : Held::Factor64)) return false;
        } else {   // SOLVE / INVERT need a resident array under the key
            CacheEntry *e = r.key >= 0 ? cache_.find(r.key) : nullptr;
            const Held want = mixed ? Held::Matrix64 : Held::Factor64;
            if (!e || e->n != r.n || e->transr != r.transr || e->uplo != r.uplo ||
                (r.op == RFP_SERVE_OP_SOLVE && e->held != want))
                return fail(j, RFP_SERVE_ENOKEY), true;
            ++e->pins;
            j->arf_off = e->offset;
            j->arf_cached = j->hit = true;
        }
        bool ok = true;
        if (r.op == RFP_SERVE_OP_INVERT) {
            ok = (j->tmp_off = alloc(rfp_bytes(r.n))) >= 0 && (j->stat_off = alloc(256)) >= 0;
        } else {
            ok = (j->b_off = alloc(bx)) >= 0 && (j->stat_off = alloc(256)) >= 0;
            if (ok && mixed) {
                const size_t wb = rfp_dpfsv_mixed_workspace(r.n, r.nrhs, kServeMixedPrec);
                ok = (j->x_off = alloc(bx)) >= 0 && (j->work_off = alloc(wb)) >= 0;
            }
        }
        if (!ok) unreserve(j);
        return ok;
    }

    // Enqueue a reserved stream job.
    void start_stream_job(Job *j)
    {
        const auto &r = j->req;
        cudaStream_t st = streams_[j->stream];
        const size_t bx = (size_t)r.n * (size_t)r.nrhs * sizeof(double);
        const bool mixed = !fp64_path(r);
        ResultSlot *hs = &slots_[j->slot];
        int32_t *d_info = reinterpret_cast<int32_t *>(dptr(j->stat_off));
        int rc = 0;
        cudaError_t e = cudaSuccess;
        j->t_start = now_s(t0_);
        j->ev0 = get_event();
        j->ev1 = get_event();
        if (j->ev0) cudaEventRecord(j->ev0, st);
        if (r.op == RFP_SERVE_OP_INVERT) {
            e = cudaMemcpyAsync(dptr(j->tmp_off), dptr(j->arf_off), rfp_bytes(r.n), cudaMemcpyDeviceToDevice, st);
            CacheEntry *ce = cache_.find(r.key);
            if (!e && ce && ce->held == Held::Matrix64) rc = rfp_dpftrf(r.transr, r.uplo, r.n, dptr(j->tmp_off), d_info, st);
            if (!e && !rc) rc = rfp_dpftri(r.transr, r.uplo, r.n, dptr(j->tmp_off), d_info, st);
            if (!e && !rc) e = cudaMemcpyAsync(r.X, dptr(j->tmp_off), rfp_bytes(r.n), cudaMemcpyDeviceToHost, st);
            if (!e && !rc) e = cudaMemcpyAsync(&hs->info, d_info, sizeof(int32_t), cudaMemcpyDeviceToHost, st);
        } else {
            if (!j->hit) e = cudaMemcpyAsync(dptr(j->arf_off), r.arf, rfp_bytes(r.n), cudaMemcpyHostToDevice, st);
            if (!e) e = cudaMemcpyAsync(dptr(j->b_off), r.B, bx, cudaMemcpyHostToDevice, st);
            if (!e && !mixed) {
                if (!j->hit) rc = rfp_dpftrf(r.transr, r.uplo, r.n, dptr(j->arf_off), d_info, st);
                else e = cudaMemsetAsync(d_info, 0, sizeof(int32_t), st);
                if (!e && !rc) rc = rfp_dpftrs(r.transr, r.uplo, r.n, r.nrhs, dptr(j->arf_off), dptr(j->b_off), r.n, st);
                if (!e && !rc) e = cudaMemcpyAsync(r.X, dptr(j->b_off), bx, cudaMemcpyDeviceToHost, st);
                if (!e && !rc) e = cudaMemcpyAsync(&hs->info, d_info, sizeof(int32_t), cudaMemcpyDeviceToHost, st);
            } else if (!e) {
                auto *d_st = reinterpret_cast<rfp_mixed_status_t *>(d_info);
                const size_t wb = rfp_dpfsv_mixed_workspace(r.n, r.nrhs, kServeMixedPrec);
                rc = rfp_dpfsv_mixed(r.transr, r.uplo, r.n, r.nrhs, dptr(j->arf_off), dptr(j->b_off), r.n,
                                     dptr(j->x_off), r.n, kServeMixedPrec, cfg_.max_iter, cfg_.tol,
                                     dptr(j->work_off), wb, d_st, st);
                if (!rc) e = cudaMemcpyAsync(r.X, dptr(j->x_off), bx, cudaMemcpyDeviceToHost, st);
                if (!e && !rc) e = cudaMemcpyAsync(&hs->st, d_st, sizeof(rfp_mixed_status_t), cudaMemcpyDeviceToHost, st);
            }
        }
        if (e != cudaSuccess || rc != 0) j->status = RFP_SERVE_ECUDA;
        if (j->ev1) cudaEventRecord(j->ev1, st);
        // the completion callback runs after everything enqueued above
        e = cudaLaunchHostFunc(st, on_done, new Done{this, j, nullptr});
        if (e != cudaSuccess) {   // no callback will come: finish now (after the stream drains)
            cudaStreamSynchronize(st);
            j->status = RFP_SERVE_ECUDA;
            j->t_done = now_s(t0_);
            retire(j);
        }
    }

    bool resident_factor(const Job *j)
    {
        const auto &r = j->req;
        CacheEntry *e = r.key >= 0 ? cache_.find(r.key) : nullptr;
        return e && e->held == Held::Factor64 && e->n == r.n && e->transr == r.transr &&
               e->uplo == r.uplo;
    }

    // Reserve a small job's arrays for the forming batch (its factor is not resident).
    bool reserve_small(Job *j)
    {
        const size_t bx = (size_t)j->req.n * (size_t)j->req.nrhs * sizeof(double);
        if (!place_arf(j, Held::Factor64)) return false;
        if ((j->b_off = alloc(bx)) < 0) {
            unreserve(j);
            return false;
        }
        return true;
    }

    void launch_batch()
    {
        auto b = std::make_unique<Batch>();
        b->jobs.swap(forming_);
        const int64_t count = (int64_t)b->jobs.size();
        b->stream = free_batch_streams_.back();
        cudaStream_t st = streams_[b->stream];
        const size_t plan_bytes = rfp_batch_plan_bytes(count);
        b->plan_off = alloc(plan_bytes);
        b->info_off = b->plan_off >= 0 ? alloc((size_t)count * sizeof(int32_t)) : -1;
        if (b->plan_off < 0 || b->info_off < 0) {   // give the jobs back to the queue
            if (b->plan_off >= 0) arena_.release(b->plan_off);
            for (auto it = b->jobs.rbegin(); it != b->jobs.rend(); ++it) {   // keep their order
                Job *j = *it;
                unreserve(j);
                free_slots_.push_back(j->slot);
                j->slot = -1;
                pending_.push_front(j);
            }
            return;
        }
        free_batch_streams_.pop_back();
        std::vector<rfp_batch_entry_t> ent((size_t)count);
        for (int64_t k = 0; k < count; ++k) {
            const auto &r = b->jobs[k]->req;
            rfp_batch_entry_t &e = ent[(size_t)k];
            std::memset(&e, 0, sizeof e);
            e.n = r.n;
            e.arf = b->jobs[k]->arf_off / (int64_t)sizeof(double);
            e.b = b->jobs[k]->b_off / (int64_t)sizeof(double);
            e.nrhs = r.nrhs;
            e.ldb = (int32_t)(r.n > 1 ? r.n : 1);
            e.transr = r.transr;
            e.uplo = r.uplo;
            const int t = (r.transr == 'T' || r.transr == 't') ? 1 : 0;
            int bucket = (int)((r.n + 63) / 64) - 1;
            bucket = bucket < 0 ? 0 : (bucket > 7 ? 7 : bucket);
            e.nb = cfg_.batch_nb[t][bucket] ? cfg_.batch_nb[t][bucket] : 16;
        }
        const int64_t len = (int64_t)(arena_.capacity() / sizeof(double));
        int64_t bad = -1;
        const double t = now_s(t0_);
        int rc = rfp_batch_plan(count, ent.data(), len, len, dptr(b->plan_off), plan_bytes, &bad, st);
        b->ev0 = get_event();
        b->ev1 = get_event();
        if (b->ev0) cudaEventRecord(b->ev0, st);
        cudaError_t e = cudaSuccess;
        for (int64_t k = 0; k < count && !rc && !e; ++k) {
            Job *j = b->jobs[k];
            j->t_start = t;
            j->batched = true;
            e = cudaMemcpyAsync(dptr(j->arf_off), j->req.arf, rfp_bytes(j->req.n), cudaMemcpyHostToDevice, st);
            if (!e) e = cudaMemcpyAsync(dptr(j->b_off), j->req.B,
                                        (size_t)j->req.n * j->req.nrhs * sizeof(double), cudaMemcpyHostToDevice, st);
        }
        int32_t *d_info = reinterpret_cast<int32_t *>(dptr(b->info_off));
        if (!rc && !e) rc = rfp_dpfsv_batched(count, dptr(b->plan_off), reinterpret_cast<double *>(base_),
                                              reinterpret_cast<double *>(base_), d_info, st);
        for (int64_t k = 0; k < count && !rc && !e; ++k) {
            Job *j = b->jobs[k];
            e = cudaMemcpyAsync(j->req.X, dptr(j->b_off), (size_t)j->req.n * j->req.nrhs * sizeof(double),
                                cudaMemcpyDeviceToHost, st);
            if (!e) e = cudaMemcpyAsync(&slots_[j->slot].info, d_info + k, sizeof(int32_t), cudaMemcpyDeviceToHost, st);
        }
        if (rc || e)
            for (Job *j : b->jobs) j->status = RFP_SERVE_ECUDA;
        if (b->ev1) cudaEventRecord(b->ev1, st);
        {
            std::lock_guard<std::mutex> lk(smu_);
            ++stats_.batches;
            stats_.batched_requests += count;
        }
        Batch *raw = b.release();
        batches_.insert(raw);
        if (cudaLaunchHostFunc(st, on_done, new Done{this, nullptr, raw}) != cudaSuccess) {
            cudaStreamSynchronize(st);
            raw->t_done = now_s(t0_);
            for (Job *j : raw->jobs) j->status = RFP_SERVE_ECUDA;
            retire_batch(raw);
        }
    }

    void retire_batch(Batch *b)
    {
        const double g0 = (b->ev0 && b->ev1) ? event_ms(b->ev0) : 0.0;
        const double g1 = (b->ev0 && b->ev1) ? event_ms(b->ev1) : 0.0;
        put_event(b->ev0);
        put_event(b->ev1);
        for (Job *j : b->jobs) {
            j->gpu_start_ms = g0;
            j->gpu_end_ms = g1;
            j->t_done = b->t_done;
            retire(j);
        }
        arena_.release(b->plan_off);
        arena_.release(b->info_off);
        free_batch_streams_.push_back(b->stream);
        batches_.erase(b);
        delete b;
    }

    // Start whatever fits, oldest first.  Large jobs keep FIFO order among
    // themselves (once one does not fit, no later large job starts in this
    // pass); small jobs may pass them, since a batch never waits for memory
    // a large job holds.
    void admit()
    {
        bool large_blocked = false;
        for (auto it = pending_.begin(); it != pending_.end();) {
            Job *j = *it;
            if (free_slots_.empty()) break;
            const size_t need = rfp_bytes(j->req.n) + extra_bytes(j);
            if (need > arena_.capacity()) {
                it = pending_.erase(it);
                fail(j, RFP_SERVE_ETOOLARGE);
                jobs_.erase(j);
                continue;
            }
            if (cfg_.small_n > 0 && is_small(j) && !resident_factor(j)) {
                if ((int)forming_.size() < cfg_.batch_max && reserve_small(j)) {
                    j->slot = take_slot();
                    forming_.push_back(j);
                    it = pending_.erase(it);
                    continue;
                }
                ++it;
                continue;
            }
            // (a small request whose factor is resident runs as a stream solve)
            if (large_blocked || free_streams_.empty()) { ++it; continue; }
            const int32_t before = j->status;
            if (!reserve_stream_job(j)) {
                large_blocked = true;
                ++it;
                continue;
            }
            it = pending_.erase(it);
            if (j->status != before) {   // completed with an error during reservation
                jobs_.erase(j);
                continue;
            }
            j->slot = take_slot();
            j->stream = free_streams_.back();
            free_streams_.pop_back();
            start_stream_job(j);
        }
        if (!forming_.empty() && !free_batch_streams_.empty()) launch_batch();
    }

    int take_slot()
    {
        const int s = free_slots_.back();
        free_slots_.pop_back();
        return s;
    }

    void run()
    {
        cudaSetDevice(dev_);
        std::unique_lock<std::mutex> lk(mu_);
        for (;;) {
            cv_.wait_for(lk, std::chrono::microseconds(200), [&] {
                return stop_ || !incoming_.empty() || !done_jobs_.empty() || !done_batches_.empty();
            });
            std::deque<std::unique_ptr<Job>> incoming;
            incoming.swap(incoming_);
            std::vector<Job *> dj;
            dj.swap(done_jobs_);
            std::vector<Batch *> db;
            db.swap(done_batches_);
            const bool stopping = stop_;
            lk.unlock();
            for (auto &j : incoming) {
                Job *raw = j.release();
                jobs_.insert(raw);
                pending_.push_back(raw);
            }
            for (Job *j : dj) retire(j);
            for (Batch *b : db) retire_batch(b);
            admit();
            {
                std::lock_guard<std::mutex> slk(smu_);
                stats_.cache_entries = (int64_t)cache_.entries();
                stats_.cache_bytes = cache_.bytes();
                stats_.arena_in_use = arena_.in_use();
                stats_.arena_capacity = arena_.capacity();
                stats_.evictions = cache_.evictions();
            }
            lk.lock();
            if (stopping && incoming_.empty() && pending_.empty() && jobs_.empty() && batches_.empty()) break;
        }
        lk.unlock();
        for (auto *j : jobs_) delete j;
    }

    // jobs_ owns every live Job (deleted when retired)
    struct JobSet {
        std::unordered_set<Job *> v;
        void insert(Job *j) { v.insert(j); }
        void erase(Job *j)
        {
            if (v.erase(j)) delete j;
        }
        bool empty() const { return v.empty(); }
        std::unordered_set<Job *>::iterator begin() { return v.begin(); }
        std::unordered_set<Job *>::iterator end() { return v.end(); }
    };
    struct BatchSet {
        std::unordered_set<Batch *> v;
        void insert(Batch *b) { v.insert(b); }
        void erase(Batch *b) { v.erase(b); }
        bool empty() const { return v.empty(); }
    };

    rfp_serve_config_t cfg_;
    Arena arena_;
    FactorCache cache_;
    std::chrono::steady_clock::time_point t0_;
    int dev_ = 0;
    void *base_ = nullptr;
    ResultSlot *slots_ = nullptr;
    std::vector<cudaStream_t> streams_;
    cudaEvent_t ref_ = nullptr;                // device-clock origin of the stamps
    std::vector<cudaEvent_t> free_events_;     // scheduler thread only
    std::vector<int> free_streams_, free_batch_streams_, free_slots_;
    std::thread worker_;

    std::mutex mu_;                                  // incoming_, done_*, stop_, submitted_
    std::condition_variable cv_;
    bool stop_ = false;
    int64_t submitted_ = 0;
    std::deque<std::unique_ptr<Job>> incoming_;
    std::vector<Job *> done_jobs_;
    std::vector<Batch *> done_batches_;

    // scheduler thread only
    std::deque<Job *> pending_;
    std::vector<Job *> forming_;
    JobSet jobs_;
    BatchSet batches_;

    std::mutex cmu_;                                 // completions
    std::condition_variable ccv_;
    std::deque<rfp_serve_completion_t> completions_;

    std::mutex smu_;
    rfp_serve_stats_t stats_{};
};

}  // namespace

extern "C" {

int rfp_serve_create(const rfp_serve_config_t *cfg, void **server)
{
    if (!cfg) return -1;
    if (!server) return -2;
    *server = nullptr;
    if (cfg->arena_bytes < (size_t(1) << 20) || cfg->streams < 1 || cfg->streams > kMaxStreams ||
        cfg->batch_max < 1 || cfg->batch_max > 4096 || cfg->small_n < 0 || cfg->small_n > 512 ||
        cfg->max_iter < 0 || !(cfg->tol > 0))
        return -1;
    for (int t = 0; t < 2; ++t)
        for (int b = 0; b < 8; ++b) {
            const int nb = cfg->batch_nb[t][b];
            if (nb != 0 && nb != 16 && nb != 24 && nb != 32) return -1;
        }
    auto *s = new Server(*cfg);
    const int rc = s->init();
    if (rc != RFP_OK) {
        delete s;
        return rc;
    }
    *server = s;
    return RFP_OK;
}

int rfp_serve_submit(void *server, const rfp_serve_request_t *r)
{
    if (!server) return -1;
    if (!r) return -2;
    const bool tr = r->transr == 'N' || r->transr == 'n' || r->transr == 'T' || r->transr == 't';
    const bool up = r->uplo == 'L' || r->uplo == 'l' || r->uplo == 'U' || r->uplo == 'u';
    const bool op = r->op == RFP_SERVE_OP_FACTOR_SOLVE || r->op == RFP_SERVE_OP_SOLVE ||
                    r->op == RFP_SERVE_OP_INVERT;
    const bool md = r->mode == RFP_SERVE_MODE_FP64 || r->mode == RFP_SERVE_MODE_MIXED;
    const bool needs_b = r->op != RFP_SERVE_OP_INVERT;
    if (!tr || !up || !op || !md || r->n < 1 || r->n > (int64_t(1) << 20) ||
        (needs_b && (r->nrhs < 1 || !r->B)) || (r->op == RFP_SERVE_OP_FACTOR_SOLVE && !r->arf) ||
        !r->X || (r->op != RFP_SERVE_OP_FACTOR_SOLVE && r->key < 0))
        return -2;
    return static_cast<Server *>(server)->submit(*r);
}

int rfp_serve_poll(void *server, rfp_serve_completion_t *out, int max, double timeout_s)
{
    if (!server) return -1;
    if (!out || max < 1) return -2;
    return static_cast<Server *>(server)->poll(out, max, timeout_s);
}

int rfp_serve_stats(void *server, rfp_serve_stats_t *st)
{
    if (!server) return -1;
    if (!st) return -2;
    static_cast<Server *>(server)->stats(st);
    return RFP_OK;
}

int rfp_serve_destroy(void *server)
{
    if (!server) return -1;
    delete static_cast<Server *>(server);
    return RFP_OK;
}

}  // extern "C"
