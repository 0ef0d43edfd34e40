// serve.cu -- batched decisions and the continuous-batching request server.
//
// Both run on a Scheduler: every admitted decision is a Job with its own
// device workspace; each scheduler step advances every active job by one
// layer of eq. (gen-polynomial:3) in one shared layer launch (jobs may sit on
// different graphs, have different k and be at different layers), starts the
// coefficients of jobs that begin a lane batch, and reads out jobs that
// finished one.  Jobs are admitted while the device memory they will hold
// fits the budget, and leave as soon as they finish, so new work joins the
// next launch without waiting for a whole batch to drain.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <vector>

#include "gf64.cuh"
#include "internal.h"

namespace tmo {
namespace {

using Clock = std::chrono::steady_clock;

// Upper bound on the arcs a query keeps: arcs whose two endpoint colours are
// in the multiset (before masks and the time window).
u64 kept_arc_bound(const Graph &g, const QuerySpec &q)
{
    if (g.pair_hist.empty()) return g.m;
    std::vector<u32> cs(q.multiset.begin(), q.multiset.end());
    std::sort(cs.begin(), cs.end());
    cs.erase(std::unique(cs.begin(), cs.end()), cs.end());
    u64 s = 0;
    for (u32 a : cs)
        for (u32 b : cs) s += g.pair_hist[(size_t)a * g.num_colors + b];
    return s;
}

// Device bytes a job on (g, q) can hold: prep arrays, coefficients,
// double-buffered checkpoints (at most one per kept arc), partial sums.
size_t job_estimate(const Graph &g, const QuerySpec &q)
{
    const u64 mf = kept_arc_bound(g, q), n = g.n, m = g.m;
    u64 L = 4;
    while (L < 128 && L < q.p_end - q.p_begin) L <<= 1;
    return (size_t)(n * 13 + (m + 1) * 4 + mf * 32 + n * L * 8 + 2 * mf * L * 8 + ((mf + 127) / 128) * L * 8 +
                    (u64)q.k * L * 8 + 4096 + (m / 4096 + 1) * 4);
}

// Estimated layer work of a request in arc-lane steps (kept arcs x layers x
// points), doubled for an extraction (its shrinking levels add up to about
// one more decision).
double request_work(const Graph &g, const QuerySpec &q, bool extract)
{
    const double w = (double)kept_arc_bound(g, q) * (q.k - 1) * (double)(q.p_end - q.p_begin);
    return extract ? 2 * w : w;
}

// Requests above this much work (about 25 ms of layer time on GB300) are
// "large": they run one at a time in arrival order, while smaller requests
// run beside them and may overtake them.
const double LARGE_WORK = 4e9;

enum JobState { J_BEGIN = 0, J_LAYER = 1, J_READOUT = 2 };

// Device memory shared by the schedulers of one server (or held by one
// batch): a job is admitted while the bytes it may hold fit the budget, or
// when nothing is admitted at all, so that a job larger than the budget's
// free part still runs alone.
struct Budget {
    explicit Budget(size_t b) : budget(b) {}
    bool try_take(size_t bytes)
    {
        std::lock_guard<std::mutex> lock(mu);
        if (in_use != 0 && in_use + bytes > budget) return false;
        in_use += bytes;
        return true;
    }
    void give(size_t bytes)
    {
        std::lock_guard<std::mutex> lock(mu);
        in_use -= bytes;
    }
    const size_t budget;
    std::mutex mu;
    size_t in_use = 0;
};

struct SJob {
    Job job;
    Workspace ws;
    size_t reserved = 0;
    int state = J_BEGIN;
    u64 owner = 0;
    ~SJob() { ws.release(); }
};

class Scheduler {
public:
    // st: the stream of the shared layer launches; prep_st: the stream of
    // job preparation (filter, checkpoints, masks), so that jobs admitted
    // while layers run are prepared beside them (the same stream when equal);
    // budget: the device memory the admitted jobs draw on
    Scheduler(cudaStream_t st, Budget *budget, cudaStream_t prep_st = nullptr)
        : st_(st), prep_st_(prep_st ? prep_st : st), budget_(budget)
    {
    }
    ~Scheduler()
    {
        for (auto &d : dev_params_) d.release();
        status_dev_.release();
        if (host_params_) cudaFreeHost(host_params_);
        if (status_host_) cudaFreeHost(status_host_);
        for (auto &b : pinned_) cudaFreeHost(b.first);
        prof.destroy();
    }

    // Pinned host blocks move from finished jobs to the next ones instead of
    // being freed: cudaFreeHost waits for the whole device, which would hold
    // one server lane up behind the other lane's work.
    void lend_pinned(SJob &sj)
    {
        if (sj.ws.host_pinned) return;
        if (!pinned_.empty()) {
            sj.ws.host_pinned = pinned_.back().first;
            sj.ws.host_pinned_bytes = pinned_.back().second;
            pinned_.pop_back();
        } else if (cudaMallocHost(&sj.ws.host_pinned, kPinnedBlock) == cudaSuccess) {
            sj.ws.host_pinned_bytes = kPinnedBlock;
        } else {
            sj.ws.host_pinned = nullptr;  // the job's own readout path allocates (or reports OOM)
            cudaGetLastError();
        }
    }
    void recycle(SJob &sj)
    {
        if (!sj.ws.host_pinned) return;
        pinned_.push_back({sj.ws.host_pinned, sj.ws.host_pinned_bytes});
        sj.ws.host_pinned = nullptr;
        sj.ws.host_pinned_bytes = 0;
    }

    Status init()
    {
        TM_CUDA(cudaMallocHost(&host_params_, kSlotBytes * kMaxLayersPerSync));
        TM_CUDA(cudaMallocHost(&status_host_, 64));
        for (auto &d : dev_params_) d.stream = st_;
        status_dev_.stream = st_;
        TM_TRY(status_dev_.reserve(64));
        return Status();
    }

    // room for one more job: the job tables of one layer launch stay inside
    // a slot (memory is taken from the budget by the caller)
    bool room() const { return active_.size() + staged_.size() < kMaxActive; }
    bool idle() const { return active_.empty() && staged_.empty(); }

    // Admit a job whose query/graph/mask are set and whose `reserved` bytes
    // the caller took from the budget; runs its prep on the prep stream
    // (which the prep synchronises).  On return the job is staged to join
    // the active jobs at the end of the current step (or at once when no
    // step is running), or finished (nothing kept) and appended to done.
    Status admit(std::unique_ptr<SJob> sj, size_t reserved, std::vector<std::unique_ptr<SJob>> *done)
    {
        sj->reserved = reserved;
        lend_pinned(*sj);
        sj->ws.set_stream(prep_st_);
        sj->job.ws = &sj->ws;
        sj->job.st = prep_st_;
        sj->job.prof = &prof;
        Status s = job_prep(sj->job);
        sj->ws.set_stream(st_);
        sj->job.st = st_;
        if (!s.ok()) {
            budget_->give(reserved);
            return s;
        }
        sj->state = J_BEGIN;
        if (sj->job.done) {
            budget_->give(sj->reserved);
            done->push_back(std::move(sj));
        } else if (in_step_) {
            staged_.push_back(std::move(sj));
        } else {
            active_.push_back(std::move(sj));
        }
        return Status();
    }

    // Upload a probe mask into a job's workspace before admission.
    Status set_mask(SJob &sj, const std::vector<uint8_t> &alive)
    {
        sj.ws.set_stream(prep_st_);
        TM_TRY(sj.ws.alive.reserve(std::max<size_t>(alive.size(), 1)));
        TM_CUDA(cudaMemcpyAsync(sj.ws.alive.p, alive.data(), alive.size(), cudaMemcpyHostToDevice, prep_st_));
        sj.job.d_alive = sj.ws.alive.as<uint8_t>();
        return Status();
    }

    // Advance every active job layer by layer (coefficients for jobs starting
    // a lane batch, one shared layer launch per lane-width class per layer)
    // until some job finishes its lane batch; then read out, sync once, and
    // retire finished jobs.  At most kMaxLayersPerSync layers are enqueued
    // before the host looks again (to admit new work).  `overlap` (may be
    // empty) runs after the launches are enqueued and before the sync: jobs
    // it admits are prepared while the layers run and join after the step.
    template <class F>
    Status step(std::vector<std::unique_ptr<SJob>> *done, F &&overlap)
    {
        for (auto &sj : staged_) active_.push_back(std::move(sj));
        staged_.clear();
        if (active_.empty()) return Status();
        if (whole_jobs_ && active_.size() == 1) return step_whole(done, overlap);
        for (int rounds = 0; rounds < kMaxLayersPerSync; rounds++) {
            std::vector<Job *> layer;
            for (auto &sj : active_) {
                if (sj->state == J_BEGIN) {
                    TM_TRY(job_batch_begin(sj->job));
                    sj->state = J_LAYER;
                }
                layer.push_back(&sj->job);
            }
            TM_TRY(launch_layers(st_, layer, dev_params_[rounds], (char *)host_params_ + rounds * kSlotBytes,
                                 kSlotBytes, &prof));
            bool readout = false;
            for (auto &sj : active_) {
                sj->job.ell++;
                if (sj->job.ell > sj->job.q.k) {
                    TM_TRY(job_readout_enqueue(sj->job));
                    sj->state = J_READOUT;
                    readout = true;
                }
            }
            if (readout) break;
        }
        in_step_ = true;
        Status os = overlap();
        in_step_ = false;
        TM_TRY(status_take_enqueue(st_, status_dev_.as<u32>(), status_host_));
        TM_CUDA(cudaStreamSynchronize(st_));
        TM_TRY(os);
        TM_TRY(status_result(*status_host_));
        TM_TRY(prof.collect());
        steps++;
        std::vector<std::unique_ptr<SJob>> keep;
        for (auto &sj : active_) {
            if (sj->state == J_READOUT) {
                job_readout_finish(sj->job);
                sj->state = J_BEGIN;
                if (sj->job.done) {
                    budget_->give(sj->reserved);
                    done->push_back(std::move(sj));
                    continue;
                }
            }
            keep.push_back(std::move(sj));
        }
        active_.swap(keep);
        for (auto &sj : staged_) active_.push_back(std::move(sj));
        staged_.clear();
        return Status();
    }
    Status step(std::vector<std::unique_ptr<SJob>> *done)
    {
        return step(done, [] { return Status(); });
    }

    // Whole jobs: a job alone in the scheduler runs in one step as a plain
    // decision does -- every lane batch enqueued back to back (the autotuner
    // on its first layer 3 where the graph has no shape yet), one sync.
    void set_whole_jobs(bool on) { whole_jobs_ = on; }

    Profiler prof;
    u64 steps = 0;

private:
    template <class F>
    Status step_whole(std::vector<std::unique_ptr<SJob>> *done, F &&overlap)
    {
        SJob &sj = *active_[0];
        TM_TRY(job_enqueue_all(sj.job, true));
        in_step_ = true;
        Status os = overlap();
        in_step_ = false;
        TM_CUDA(cudaStreamSynchronize(st_));
        TM_TRY(os);
        TM_TRY(prof.collect());
        TM_TRY(job_finish_all(sj.job));
        steps++;
        budget_->give(sj.reserved);
        done->push_back(std::move(active_[0]));
        active_.clear();
        for (auto &x : staged_) active_.push_back(std::move(x));
        staged_.clear();
        return Status();
    }

    static_assert(4096 * (sizeof(LayerParams) + 8) + 6 * (256 + 16) < (1 << 20), "job tables exceed a slot");
    // one job-table slot (host pinned + device) per layer round between syncs
    static const int kMaxLayersPerSync = 8;
    static const size_t kSlotBytes = 1 << 20;
    static const size_t kMaxActive = 4096;  // x (LayerParams + prefix) < kSlotBytes
    cudaStream_t st_, prep_st_;
    Budget *budget_;
    bool in_step_ = false;
    bool whole_jobs_ = false;
    std::vector<std::unique_ptr<SJob>> active_, staged_;
    DevBuf dev_params_[kMaxLayersPerSync];
    void *host_params_ = nullptr;
    DevBuf status_dev_;           // the device status word taken after each step ...
    u32 *status_host_ = nullptr;  // ... and its pinned host copy
    static const size_t kPinnedBlock = 64 * 1024;
    std::vector<std::pair<void *, size_t>> pinned_;  // pinned blocks of finished jobs
};

size_t default_budget()
{
    size_t free_b = 0, total_b = 0;
    if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) return (size_t)8 << 30;
    return (size_t)(free_b * 0.8);
}

}  // namespace
}  // namespace tmo

using namespace tmo;

// ---------------------------------------------------------------------------
// Batched decisions
// ---------------------------------------------------------------------------
extern "C" int tmotif_decide_batch(const tmotif_graph_t *graphs, const tmotif_query *queries, uint32_t count,
                                   tmotif_decision *out)
{
    if (count == 0) return TMOTIF_OK;
    if (!graphs || !queries || !out) return fail(TMOTIF_ERR_INVALID, "null argument").code;
    try {
        std::vector<QuerySpec> specs(count);
        for (uint32_t i = 0; i < count; i++) {
            if (!graphs[i]) return fail(TMOTIF_ERR_INVALID, "null graph in batch").code;
            Status s = parse_query(*graphs[i], &queries[i], &specs[i]);
            if (!s.ok()) return s.code;
            if (specs[i].flags & TMOTIF_PREPROCESS_STATIC)
                return fail(TMOTIF_ERR_UNSUPPORTED, "batched decisions take no static preprocessing").code;
            if (graphs[i]->stream != graphs[0]->stream)
                return fail(TMOTIF_ERR_INVALID, "graphs of one batch must share a stream").code;
        }
        cudaStream_t st = graphs[0]->stream;
        bool packable = count > 1;
        for (uint32_t i = 0; i < count && packable; i++) packable = pack_eligible(specs[i]);
        if (packable) {
            // many graphs, one pass: the packed form (pack.cu)
            cudaEvent_t e0, e1;
            cudaEventCreate(&e0);
            cudaEventCreate(&e1);
            cudaEventRecord(e0, st);
            std::vector<std::vector<u64>> vals;
            std::vector<Graph *> gp(graphs, graphs + count);
            u64 launches = 0;
            Status ps = pack_decide(gp.data(), specs.data(), count, st, &vals, &launches);
            cudaEventRecord(e1, st);
            cudaEventSynchronize(e1);
            float ms = 0;
            cudaEventElapsedTime(&ms, e0, e1);
            cudaEventDestroy(e0);
            cudaEventDestroy(e1);
            if (!ps.ok()) return ps.code;
            for (uint32_t i = 0; i < count; i++) {
                u64 sum = 0;
                for (u64 v : vals[i]) sum ^= v;
                out[i].found = sum != 0;
                out[i].sieve_sum = sum;
                out[i].ms = ms;
                if (out[i].per_point) std::memcpy(out[i].per_point, vals[i].data(), vals[i].size() * sizeof(u64));
            }
            graphs[0]->prof.stats.launches += launches;
            return TMOTIF_OK;
        }
        Budget budget(default_budget());
        Scheduler sched(st, &budget);
        Status s = sched.init();
        if (!s.ok()) return s.code;
        cudaEvent_t e0, e1;
        cudaEventCreate(&e0);
        cudaEventCreate(&e1);
        cudaEventRecord(e0, st);
        std::vector<std::unique_ptr<SJob>> done;
        auto finish = [&](std::unique_ptr<SJob> &sj) {
            const u64 i = sj->owner;
            out[i].found = sj->job.found;
            out[i].sieve_sum = sj->job.sieve_sum;
            if (out[i].per_point && !sj->job.vals.empty())
                std::memcpy(out[i].per_point, sj->job.vals.data(), sj->job.vals.size() * sizeof(u64));
            else if (out[i].per_point)
                std::memset(out[i].per_point, 0, (specs[i].p_end - specs[i].p_begin) * sizeof(u64));
        };
        uint32_t next = 0;
        while (next < count || !sched.idle()) {
            while (next < count) {
                const size_t need = job_estimate(*graphs[next], specs[next]);
                if (!sched.room() || !budget.try_take(need)) break;
                auto sj = std::make_unique<SJob>();
                sj->owner = next;
                sj->job.g = graphs[next];
                sj->job.q = specs[next];
                s = sched.admit(std::move(sj), need, &done);
                if (!s.ok()) return s.code;
                next++;
            }
            s = sched.step(&done);
            if (!s.ok()) return s.code;
            for (auto &sj : done) {
                finish(sj);
                sched.recycle(*sj);
            }
            done.clear();
        }
        cudaEventRecord(e1, st);
        cudaEventSynchronize(e1);
        float ms = 0;
        cudaEventElapsedTime(&ms, e0, e1);
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        for (uint32_t i = 0; i < count; i++) out[i].ms = ms;
        return TMOTIF_OK;
    } catch (const std::bad_alloc &) {
        return fail(TMOTIF_ERR_OOM, "host allocation failed").code;
    }
}


// ---------------------------------------------------------------------------
// Request server
//
// Two lanes, each a worker thread with its own scheduler, streams and
// finishing workspace, drawing on one memory budget:
//   lane 0 takes the small requests and runs them many at a time in shared
//     layer launches, on streams of the device's least priority;
//   lane 1 takes the large requests (over LARGE_WORK arc-lane steps) one at
//     a time, in arrival order, on streams of its greatest priority; each of
//     their jobs runs whole, as a plain decision does (every lane batch
//     enqueued back to back in the tuned launch shape, one sync).
// Small requests thus run beside a large one instead of queueing behind it:
// their kernels take the SMs the large request leaves free (its preparation,
// readout and synchronisation gaps, its launches' tails), while the large
// request's own blocks are scheduled first.  When the large lane waits for
// memory, the small lane admits nothing new until it has been served.
// ---------------------------------------------------------------------------
namespace {

struct Request {
    u64 ticket = 0;
    Graph *g = nullptr;
    QuerySpec q;
    bool is_extract = false;
    bool halving = false;
    bool large = false;
    ExtractState ex;         // halving procedure
    LocalizedExtract lex;    // localisation procedure
    Clock::time_point t_submit;
    bool done = false;
    std::atomic<bool> cancelled{false};  // tmotif_cancel: complete with CANCELLED at the next chance
    int code = TMOTIF_OK;
    std::string err;
    int found = 0;
    u64 sieve_sum = 0;
    double ms = 0;
    std::vector<u64> vals;   // decide requests: repeat-0 per-point sums on [p_begin, p_end)
    std::vector<u32> verts, times;
};

struct Lane {
    tmotif_server *srv = nullptr;
    bool large = false;
    cudaStream_t st = nullptr, prep_st = nullptr;  // layer launches; job preparation
    std::unique_ptr<Scheduler> sched;
    Workspace finish_ws;  // arc gathering for extraction's final DFS
    std::thread worker;
    std::deque<Request *> pending;  // submitted to this lane, not yet taken (server mutex)
    Request *holder = nullptr;      // large lane: the request now running

    enum { NJ_JOB, NJ_NONE, NJ_FAILED };
    void complete(Request *r, Status s);
    int next_job(Request *r, std::unique_ptr<SJob> *out);
    void finish_extract(Request *r);
    void run();
};

}  // namespace

struct tmotif_server {
    int device = 0;
    std::unique_ptr<Budget> budget;
    Lane lanes[2];  // 0: small requests; 1: large requests
    std::mutex mu;
    std::condition_variable cv;       // work submitted
    std::condition_variable done_cv;  // a request finished (tmotif_wait)
    std::map<u64, std::unique_ptr<Request>> reqs;
    std::atomic<bool> stop{false};
    std::atomic<bool> large_waiting{false};  // the large lane waits for memory
    u64 next_ticket = 1;

    void complete(Request *r, Status s)
    {
        std::lock_guard<std::mutex> lock(mu);
        if (!s.ok()) {
            r->code = s.code;
            r->err = tmotif_last_error();
        }
        r->ms = std::chrono::duration<double, std::milli>(Clock::now() - r->t_submit).count();
        r->done = true;
        done_cv.notify_all();
    }
};

namespace {

void Lane::complete(Request *r, Status s)
{
    if (holder == r) holder = nullptr;
    srv->complete(r, s);
}

// Make the next job of a request (its decision, or its next probe):
// NJ_JOB, NJ_NONE when the request needs no more jobs, or NJ_FAILED when it
// failed and was completed with the error (the caller must not touch it).
int Lane::next_job(Request *r, std::unique_ptr<SJob> *out)
{
    auto sj = std::make_unique<SJob>();
    sj->owner = r->ticket;
    sj->job.g = r->g;
    if (!r->is_extract) {
        sj->job.q = r->q;
        *out = std::move(sj);
        return NJ_JOB;
    }
    if (!r->halving) {
        QuerySpec sub;
        u32 rep = 0;
        const std::vector<uint8_t> *mask = nullptr;
        if (!r->lex.next(&sub, &rep, &mask)) return NJ_NONE;
        sj->job.q = sub;
        sj->job.localize = true;
        sj->job.rep_offset = rep;
        if (mask) {
            Status s = sched->set_mask(*sj, *mask);
            if (!s.ok()) {
                complete(r, s);
                return NJ_FAILED;
            }
        }
        *out = std::move(sj);
        return NJ_JOB;
    }
    QuerySpec pq;
    if (!r->ex.next_probe(&pq)) return NJ_NONE;
    sj->job.q = pq;
    if (r->ex.stage == ExtractState::PROBING) {
        Status s = r->ex.maybe_compact(*r->g, finish_ws, prep_st);
        if (s.ok()) s = sched->set_mask(*sj, r->ex.alive);
        if (!s.ok()) {
            complete(r, s);
            return NJ_FAILED;
        }
        sj->job.g = r->ex.current(*r->g);
    }
    *out = std::move(sj);
    return NJ_JOB;
}

void Lane::finish_extract(Request *r)
{
    r->verts.assign(r->q.k, 0);
    r->times.assign(r->q.k, 0);
    if (!r->halving) {
        r->found = r->lex.found ? 1 : 0;
        if (r->lex.found) {
            r->verts = r->lex.verts;
            r->times = r->lex.times;
        }
        complete(r, Status());
        return;
    }
    Status s;
    if (r->ex.stage == ExtractState::SHRUNK)
        s = extract_finish(*r->ex.current(*r->g), finish_ws, prep_st, sched->prof, r->ex, r->verts.data(),
                           r->times.data(), &r->found);
    else
        r->found = 0;
    complete(r, s);
}

void Lane::run()
{
    cudaSetDevice(srv->device);
    std::deque<std::pair<Request *, std::unique_ptr<SJob>>> waiting;  // admission queue (FIFO)
    std::vector<std::unique_ptr<SJob>> done;
    auto take_pending = [&]() {
        std::lock_guard<std::mutex> lock(srv->mu);
        while (!pending.empty()) {
            Request *r = pending.front();
            pending.pop_front();
            waiting.push_back({r, nullptr});
        }
    };
    // admit in arrival order while the memory budget allows; the large lane
    // runs one request at a time
    auto admit_waiting = [&]() {
        take_pending();
        bool blocked = false;  // large lane: the next request does not fit the budget yet
        for (auto it = waiting.begin(); it != waiting.end();) {
            Request *r = it->first;
            std::unique_ptr<SJob> &sj = it->second;
            if (r->cancelled.load()) {  // dropped before (or between) its decisions
                complete(r, fail(TMOTIF_ERR_CANCELLED, "request cancelled"));
                it = waiting.erase(it);
                continue;
            }
            if (large && holder && holder != r) {
                ++it;
                continue;
            }
            if (!large && srv->large_waiting.load()) break;  // leave the memory to the large lane
            if (!sj) {
                const int nj = next_job(r, &sj);
                if (nj != NJ_JOB) {  // nothing left to run, or failed and completed
                    if (nj == NJ_NONE) finish_extract(r);
                    it = waiting.erase(it);
                    continue;
                }
            }
            const size_t need = job_estimate(*sj->job.g, sj->job.q);
            if (!sched->room() || !srv->budget->try_take(need)) {
                blocked = true;
                break;
            }
            if (large) holder = r;
            Status s = sched->admit(std::move(sj), need, &done);
            it = waiting.erase(it);
            if (!s.ok()) complete(r, s);
        }
        // recomputed on every pass, so that a waiting request that is
        // cancelled or fails does not leave the small lane closed
        if (large) srv->large_waiting.store(blocked);
    };
    while (!srv->stop.load()) {
        {
            std::unique_lock<std::mutex> lock(srv->mu);
            if (pending.empty() && waiting.empty() && sched->idle())
                srv->cv.wait_for(lock, std::chrono::milliseconds(2));
        }
        if (sched->idle()) admit_waiting();
        if (!sched->idle()) {
            // jobs admitted while this step's layers run are prepared
            // beside them (prep stream) and join after the step
            Status s = sched->step(&done, [&] {
                admit_waiting();
                return Status();
            });
            if (!s.ok()) {  // fail every request of this lane in flight
                std::lock_guard<std::mutex> lock(srv->mu);
                const std::string msg = tmotif_last_error();
                for (auto &kv : srv->reqs)
                    if (!kv.second->done && kv.second->large == large) {
                        kv.second->code = s.code;
                        kv.second->err = msg;
                        kv.second->done = true;
                    }
                if (large) srv->large_waiting.store(false);
                srv->done_cv.notify_all();
                return;
            }
        } else if (!waiting.empty()) {
            // waiting for memory the other lane holds
            std::this_thread::sleep_for(std::chrono::microseconds(200));
        }
        for (auto &sj : done) {
            Request *r = nullptr;
            {
                std::lock_guard<std::mutex> lock(srv->mu);
                auto it = srv->reqs.find(sj->owner);
                if (it != srv->reqs.end()) r = it->second.get();
            }
            if (!r) continue;
            if (r->cancelled.load()) {  // its current decision finished; no more
                complete(r, fail(TMOTIF_ERR_CANCELLED, "request cancelled"));
                continue;
            }
            if (!r->is_extract) {
                r->found = sj->job.found;
                r->sieve_sum = sj->job.sieve_sum;
                r->vals = std::move(sj->job.vals);
                complete(r, Status());
                continue;
            }
            if (!r->halving) {
                u32 best = NONE, a = 0, b = 0, t = 0;
                Status s = sj->job.done && sj->job.mf == 0 ? Status() : job_first_arc(sj->job, &best, &a, &b, &t);
                if (!s.ok()) {
                    complete(r, s);
                    continue;
                }
                r->lex.result(best, a, b, t);
                if (r->lex.done) {
                    finish_extract(r);
                    continue;
                }
            } else {
                r->ex.result(sj->job.found != 0);
                if (r->ex.stage == ExtractState::NOT_FOUND) {
                    finish_extract(r);
                    continue;
                }
            }
            // next level/probe joins the front of the admission queue (the request keeps its turn)
            std::unique_ptr<SJob> nj;
            const int st = next_job(r, &nj);
            if (st == NJ_JOB) waiting.push_front({r, std::move(nj)});
            else if (st == NJ_NONE) finish_extract(r);
        }
        for (auto &sj : done) sched->recycle(*sj);
        done.clear();
    }
}

}  // namespace

extern "C" int tmotif_server_create(size_t hbm_budget_bytes, tmotif_server_t *out)
{
    if (!out) return fail(TMOTIF_ERR_INVALID, "null output handle").code;
    *out = nullptr;
    try {
        auto s = std::make_unique<tmotif_server>();
        if (cudaGetDevice(&s->device) != cudaSuccess) return fail(TMOTIF_ERR_CUDA, "no CUDA device").code;
        s->budget = std::make_unique<Budget>(hbm_budget_bytes ? hbm_budget_bytes : default_budget());
        int least = 0, greatest = 0;
        cudaError_t e = cudaDeviceGetStreamPriorityRange(&least, &greatest);
        for (int i = 0; i < 2 && e == cudaSuccess; i++) {
            Lane &l = s->lanes[i];
            l.srv = s.get();
            l.large = i == 1;
            const int prio = l.large ? greatest : least;
            e = cudaStreamCreateWithPriority(&l.st, cudaStreamNonBlocking, prio);
            if (e == cudaSuccess) e = cudaStreamCreateWithPriority(&l.prep_st, cudaStreamNonBlocking, prio);
        }
        if (e != cudaSuccess) {
            for (Lane &l : s->lanes)
                for (cudaStream_t st : {l.st, l.prep_st})
                    if (st) cudaStreamDestroy(st);
            return cuda_fail(e, "server streams").code;
        }
        for (Lane &l : s->lanes) {
            l.sched = std::make_unique<Scheduler>(l.st, s->budget.get(), l.prep_st);
            l.sched->set_whole_jobs(l.large);
            Status st = l.sched->init();
            if (!st.ok()) {
                for (Lane &m : s->lanes)
                    for (cudaStream_t x : {m.st, m.prep_st})
                        if (x) cudaStreamDestroy(x);
                return st.code;
            }
            l.finish_ws.set_stream(l.prep_st);
        }
        for (Lane &l : s->lanes) {
            Lane *raw = &l;
            l.worker = std::thread([raw] { raw->run(); });
        }
        *out = s.release();
        return TMOTIF_OK;
    } catch (const std::bad_alloc &) {
        return fail(TMOTIF_ERR_OOM, "host allocation failed").code;
    }
}

extern "C" int tmotif_submit(tmotif_server_t s, tmotif_graph_t g, const tmotif_query *q, int is_extract,
                             uint64_t *ticket)
{
    if (!s || !g || !ticket) return fail(TMOTIF_ERR_INVALID, "null argument").code;
    try {
        auto r = std::make_unique<Request>();
        Status st = parse_query(*g, q, &r->q);
        if (!st.ok()) return st.code;
        if (r->q.flags & TMOTIF_PREPROCESS_STATIC)
            return fail(TMOTIF_ERR_UNSUPPORTED, "the server takes no static preprocessing").code;
        if (is_extract && (r->q.p_begin != 0 || r->q.p_end != (1ull << r->q.k)))
            return fail(TMOTIF_ERR_INVALID, "extraction needs the full point range").code;
        if (job_estimate(*g, r->q) > s->budget->budget)
            return fail(TMOTIF_ERR_BUSY, "request needs more device memory than the server budget").code;
        r->g = g;
        r->is_extract = is_extract != 0;
        r->halving = (r->q.flags & TMOTIF_EXTRACT_HALVING) != 0;
        r->large = request_work(*g, r->q, r->is_extract) > LARGE_WORK;
        if (r->is_extract) {
            Status hc = ensure_host_colors(*g);
            if (!hc.ok()) return hc.code;
        }
        if (r->is_extract && r->halving) r->ex.init(*g, r->q);
        if (r->is_extract && !r->halving) r->lex.init(*g, r->q);
        r->t_submit = Clock::now();
        std::lock_guard<std::mutex> lock(s->mu);
        r->ticket = s->next_ticket++;
        *ticket = r->ticket;
        s->lanes[r->large ? 1 : 0].pending.push_back(r.get());
        s->reqs[r->ticket] = std::move(r);
        s->cv.notify_all();
        return TMOTIF_OK;
    } catch (const std::bad_alloc &) {
        return fail(TMOTIF_ERR_OOM, "host allocation failed").code;
    }
}

// Hand out a finished request's result and forget it (s->mu held).
static int take_result(tmotif_server_t s, std::map<u64, std::unique_ptr<Request>>::iterator it,
                       tmotif_decision *out, uint32_t *verts, uint32_t *times)
{
    Request *r = it->second.get();
    const int code = r->code;
    if (code != TMOTIF_OK) set_error(r->err);
    if (out) {
        out->found = r->found;
        out->sieve_sum = r->sieve_sum;
        out->ms = r->ms;
        if (out->per_point && !r->is_extract && code == TMOTIF_OK) {
            const u64 npts = r->q.p_end - r->q.p_begin;
            if (r->vals.size() == npts) std::memcpy(out->per_point, r->vals.data(), npts * sizeof(u64));
            else std::memset(out->per_point, 0, npts * sizeof(u64));
        }
    }
    if (r->is_extract && r->found) {
        if (verts) std::copy(r->verts.begin(), r->verts.begin() + r->q.k, verts);
        if (times) std::copy(r->times.begin(), r->times.begin() + (r->q.k - 1), times);
    }
    s->reqs.erase(it);
    return code;
}

extern "C" int tmotif_poll(tmotif_server_t s, uint64_t ticket, tmotif_decision *out, uint32_t *verts,
                           uint32_t *times, int *done)
{
    if (!s || !done) return fail(TMOTIF_ERR_INVALID, "null argument").code;
    std::lock_guard<std::mutex> lock(s->mu);
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end()) return fail(TMOTIF_ERR_NOT_FOUND, "unknown ticket").code;
    *done = it->second->done ? 1 : 0;
    if (!*done) return TMOTIF_OK;
    return take_result(s, it, out, verts, times);
}

extern "C" int tmotif_wait(tmotif_server_t s, uint64_t ticket, uint32_t timeout_ms, tmotif_decision *out,
                           uint32_t *verts, uint32_t *times)
{
    if (!s) return fail(TMOTIF_ERR_INVALID, "null argument").code;
    std::unique_lock<std::mutex> lock(s->mu);
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end()) return fail(TMOTIF_ERR_NOT_FOUND, "unknown ticket").code;
    Request *r = it->second.get();
    if (!s->done_cv.wait_for(lock, std::chrono::milliseconds(timeout_ms), [r] { return r->done; }))
        return fail(TMOTIF_ERR_TIMEOUT, "request not finished within the timeout").code;
    return take_result(s, s->reqs.find(ticket), out, verts, times);
}

extern "C" int tmotif_cancel(tmotif_server_t s, uint64_t ticket)
{
    if (!s) return fail(TMOTIF_ERR_INVALID, "null argument").code;
    std::lock_guard<std::mutex> lock(s->mu);
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end()) return fail(TMOTIF_ERR_NOT_FOUND, "unknown ticket").code;
    if (!it->second->done) it->second->cancelled.store(true);
    s->cv.notify_all();
    return TMOTIF_OK;
}

extern "C" void tmotif_server_destroy(tmotif_server_t s)
{
    if (!s) return;
    s->stop.store(true);
    s->cv.notify_all();
    for (Lane &l : s->lanes)
        if (l.worker.joinable()) l.worker.join();
    for (Lane &l : s->lanes) {
        l.sched.reset();
        l.finish_ws.release();
    }
    s->reqs.clear();  // extraction subgraphs free on their lane's prep stream
    for (Lane &l : s->lanes)
        for (cudaStream_t st : {l.st, l.prep_st})
            if (st) {
                cudaStreamSynchronize(st);
                cudaStreamDestroy(st);
            }
    delete s;
}
