// vs_serve.cu -- continuous batching of smoothing jobs on one GPU.
//
// A scheduler thread owns every admitted job.  Jobs wait in arrival order and
// are admitted (first fit in arrival order) while a slot is free and the sum
// of the device footprints of the running jobs stays within the HBM budget.
// Each running job has its own field and stream; its sweeps are enqueued in
// chunks (one replay of a CUDA graph holding `chunk` annealed sweeps and the
// re-unitarisation that follows them), at most two chunks in flight per job.
// Chunk graphs are kept per shape (extents, precision, storage, staple kind,
// chunk length): a finished job returns its instantiated graph to the pool of
// its shape, and the next job of that shape updates it in place with its own
// field pointers and parameters (cudaGraphExecUpdate of a fresh capture, which
// costs less than instantiating the graph anew),
// so the work of all running jobs overlaps on the device and a job that
// arrives while others run is admitted as soon as a slot and memory free up.
// Kernels are deterministic and jobs share no device memory, so a job's
// result does not depend on what else runs.  A job runs on a stream whose
// priority follows its total work (link updates, log scale, smaller work more
// urgent): the device's block scheduler then serves the short jobs' kernels
// first, an approximation of shortest-job-first that keeps short jobs from
// queueing behind long ones.
#include <algorithm>
#include <cmath>
#include <cstring>

#include "vs_api_internal.h"

using namespace vs;

namespace vs {

enum JobState { WAITING, RUNNING, DONE };

// What fixes the node structure of a job's chunk graph.
struct GraphKey {
    int32_t dims[4];
    int32_t precision, storage, rect, chunk, reunit_every, redecide;
    bool operator<(const GraphKey &o) const {
        return std::memcmp(this, &o, sizeof *this) < 0;
    }
};

struct Job {
    int64_t ticket = 0;
    vs_job spec{};
    std::vector<int8_t> labels;
    JobState state = WAITING;
    bool cancel = false;
    uint64_t footprint = 0;
    vs_field *f = nullptr;
    cudaStream_t stream = nullptr;
    int slot = -1;
    int sweeps_enqueued = 0;
    int chunk = 10;
    cudaGraphExec_t graph = nullptr;
    GraphKey key{};
    std::deque<cudaEvent_t> inflight;
    vs_result result{};
};

struct Serve {
    vs_ctx *ctx = nullptr;
    std::mutex mu;
    std::condition_variable cv_done;   // poll waiters
    std::condition_variable cv_work;   // scheduler wake-up
    std::map<int64_t, std::shared_ptr<Job>> jobs;
    std::deque<int64_t> waiting;
    std::vector<int64_t> running;
    std::vector<cudaStream_t> streams;   // [slot][priority level], level 0 most urgent
    int n_levels = 1;
    std::vector<bool> slot_busy;
    std::vector<cudaEvent_t> event_pool;
    std::map<GraphKey, std::vector<cudaGraphExec_t>> graph_pool;   // idle chunk graphs per shape
    int64_t graphs_instantiated = 0, graphs_reused = 0;
    int64_t next_ticket = 1;
    uint64_t bytes_in_use = 0, peak_bytes = 0;
    int64_t n_submitted = 0, n_completed = 0, n_cancelled = 0;
    bool stop = false;
    std::thread thr;

    void loop();
    bool admit_one(std::unique_lock<std::mutex> &lk);
    void step_running(std::unique_lock<std::mutex> &lk, bool &progressed);
    void finish(Job &j, vs_status st);
    cudaEvent_t get_event();
    cudaGraphExec_t take_graph(const GraphKey &k);
};

static double now_ms(vs_ctx *c) { return vs_now_ms(c); }

cudaEvent_t Serve::get_event() {
    if (!event_pool.empty()) {
        cudaEvent_t e = event_pool.back();
        event_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreateWithFlags(&e, cudaEventDisableTiming);
    return e;
}

static uint64_t job_footprint(const vs_job &s) {
    uint64_t b = field_footprint(s.dims, s.precision, s.storage);
    uint64_t V = (uint64_t)s.dims[0] * s.dims[1] * s.dims[2] * s.dims[3];
    if (s.links_out) b += 4 * V * 18 * sizeof(double);   // read-back staging
    else b += 4 * V;                                      // label staging
    return b;
}

// Priority level of a job from its work, 4 V (n_sweeps + n_cool) link
// updates: below 2^24, 2^26, 2^28, and above (0 is the most urgent).
static int work_level(const vs_job &s, int n_levels) {
    const double V = (double)s.dims[0] * s.dims[1] * s.dims[2] * s.dims[3];
    const double w = 4.0 * V * ((double)s.n_sweeps + (double)std::max(s.n_cool, 0));
    const int lev = w < 16777216.0 ? 0 : w < 67108864.0 ? 1 : w < 268435456.0 ? 2 : 3;
    return std::min(lev, n_levels - 1);
}

// Called with the lock held.  Releases it around device work.
bool Serve::admit_one(std::unique_lock<std::mutex> &lk) {
    if ((int)running.size() >= ctx->opt.max_slots) return false;
    const uint64_t budget = ctx->opt.hbm_budget_bytes;
    for (auto it = waiting.begin(); it != waiting.end(); ++it) {
        auto &j = *jobs[*it];
        if (budget && bytes_in_use + j.footprint > budget && !running.empty()) continue;
        if (budget && j.footprint > budget) {
            // can never fit: fail it rather than block the queue
            int64_t t = *it;
            waiting.erase(it);
            j.result.t_admit_ms = now_ms(ctx);
            finish(*jobs[t], fail(VS_ENOMEM, "job footprint %llu exceeds the HBM budget",
                                  (unsigned long long)j.footprint));
            return true;
        }
        int64_t t = *it;
        waiting.erase(it);
        int slot = (int)(std::find(slot_busy.begin(), slot_busy.end(), false) - slot_busy.begin());
        slot_busy[slot] = true;
        auto jp = jobs[t];
        jp->state = RUNNING;
        jp->slot = slot;
        jp->stream = streams[(size_t)slot * n_levels + work_level(jp->spec, n_levels)];
        jp->result.t_admit_ms = now_ms(ctx);
        bytes_in_use += jp->footprint;
        peak_bytes = std::max(peak_bytes, bytes_in_use);
        running.push_back(t);
        lk.unlock();
        vs_status st = vs_field_create(ctx, jp->spec.dims, jp->spec.precision, jp->spec.storage,
                                       (void *)jp->stream, &jp->f);
        if (st == VS_OK) {
            if (!jp->labels.empty()) st = vs_load_field(jp->f, nullptr, jp->labels.data(), VS_HOST);
            else st = vs_load_cooled(jp->f, jp->spec.seed, jp->spec.n_cool);
        }
        if (st == VS_OK && jp->spec.omega >= 0)
            st = vs_centrifuge(jp->f, jp->spec.omega, jp->spec.centrifuge_seed);
        if (st == VS_OK)
            if (init_sweep_counters(jp->f->d_sweep, 1, jp->stream) != cudaSuccess)
                st = fail(VS_EDEVICE, "counter reset failed");
        lk.lock();
        if (st != VS_OK) finish(*jp, st);
        return true;
    }
    return false;
}

void Serve::finish(Job &j, vs_status st) {
    // lock held
    j.result.status = j.cancel ? VS_ECANCELED : st;
    j.result.t_done_ms = now_ms(ctx);
    if (j.state == RUNNING) {
        running.erase(std::remove(running.begin(), running.end(), j.ticket), running.end());
        slot_busy[j.slot] = false;
        bytes_in_use -= j.footprint;
    } else {
        waiting.erase(std::remove(waiting.begin(), waiting.end(), j.ticket), waiting.end());
    }
    if (j.f) {
        vs_field_destroy(j.f);
        j.f = nullptr;
    }
    if (j.graph) {
        // idle now (the job's chunks have completed): the next job of this shape updates it
        graph_pool[j.key].push_back(j.graph);
        j.graph = nullptr;
    }
    for (auto e : j.inflight) event_pool.push_back(e);
    j.inflight.clear();
    j.state = DONE;
    if (j.cancel) ++n_cancelled;
    else ++n_completed;
    cv_done.notify_all();
    cv_work.notify_all();
}

// An idle chunk graph of the job's shape, or nullptr (lock held).
cudaGraphExec_t Serve::take_graph(const GraphKey &k) {
    auto it = graph_pool.find(k);
    if (it == graph_pool.end() || it->second.empty()) return nullptr;
    cudaGraphExec_t g = it->second.back();
    it->second.pop_back();
    return g;
}

// Enqueue the next chunk of a running job (lock released by caller).
static vs_status enqueue_chunk(Serve &sv, std::unique_lock<std::mutex> &lk, Job &j, unsigned long long *ctr) {
    NvtxRange range("vs served chunk");
    vs_field *f = j.f;
    const vs_job &s = j.spec;
    int left = s.n_sweeps - j.sweeps_enqueued;
    int n = std::min(left, j.chunk);
    vs_anneal a;
    memset(&a, 0, sizeof a);
    a.kind = VS_ANNEALED;
    a.reunit_every = s.reunit_every;
    a.fp64_redecide = s.fp64_redecide != 0;
    if (n == j.chunk && (s.reunit_every <= 0 || j.chunk % s.reunit_every == 0)) {
        if (!j.graph) {
            cudaGraph_t g = nullptr;
            f->sweeps_done = 0;      // the captured chunk starts a re-unitarisation period
            if (cudaStreamBeginCapture(f->stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
                return fail(VS_EDEVICE, "stream capture failed");
            vs_status st = smooth_enqueue(f, n, s.rho, s.epsilon, s.u0, &a, s.vortex_preserve, false, ctr);
            cudaError_t e = cudaStreamEndCapture(f->stream, &g);
            if (st != VS_OK) {
                if (g) cudaGraphDestroy(g);
                return st;
            }
            if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture");
            j.key = GraphKey{{s.dims[0], s.dims[1], s.dims[2], s.dims[3]}, s.precision, s.storage,
                             s.epsilon != 1.0, j.chunk, s.reunit_every, s.fp64_redecide != 0};
            lk.lock();
            cudaGraphExec_t pooled = sv.take_graph(j.key);
            lk.unlock();
            bool reused = false;
            if (pooled) {
                // same node structure, this job's pointers and parameters
                cudaGraphExecUpdateResultInfo info;
                if (cudaGraphExecUpdate(pooled, g, &info) == cudaSuccess) {
                    j.graph = pooled;
                    reused = true;
                } else {
                    cudaGetLastError();
                    cudaGraphExecDestroy(pooled);
                }
            }
            if (!reused) e = cudaGraphInstantiate(&j.graph, g, 0);
            cudaGraphDestroy(g);
            if (e != cudaSuccess) return cuda_fail(e, "cudaGraphInstantiate");
            lk.lock();
            ++(reused ? sv.graphs_reused : sv.graphs_instantiated);
            lk.unlock();
        }
        cudaError_t e = cudaGraphLaunch(j.graph, f->stream);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGraphLaunch");
    } else {
        // final partial chunk: graph replays do not advance the host-side sweep
        // count, so set the re-unitarisation phase from the sweeps enqueued
        f->sweeps_done = j.sweeps_enqueued;
        vs_status st = smooth_enqueue(f, n, s.rho, s.epsilon, s.u0, &a, s.vortex_preserve, false, ctr);
        if (st != VS_OK) return st;
    }
    j.sweeps_enqueued += n;
    return VS_OK;
}

void Serve::step_running(std::unique_lock<std::mutex> &lk, bool &progressed) {
    std::vector<int64_t> ids = running;
    for (int64_t t : ids) {
        auto it = jobs.find(t);
        if (it == jobs.end()) continue;
        auto jp = it->second;
        Job &j = *jp;
        if (j.state != RUNNING) continue;
        // retire completed chunks
        while (!j.inflight.empty() && cudaEventQuery(j.inflight.front()) == cudaSuccess) {
            event_pool.push_back(j.inflight.front());
            j.inflight.pop_front();
            progressed = true;
        }
        if (j.cancel) {
            if (j.inflight.empty()) {
                lk.unlock();
                cudaStreamSynchronize(j.stream);
                lk.lock();
                finish(j, VS_OK);
                progressed = true;
            }
            continue;
        }
        if (j.sweeps_enqueued < j.spec.n_sweeps) {
            if (j.inflight.size() < 2) {
                cudaEvent_t ev = get_event();
                lk.unlock();
                vs_status st = enqueue_chunk(*this, lk, j, j.f->d_sweep);
                if (st == VS_OK && cudaEventRecord(ev, j.stream) != cudaSuccess)
                    st = fail(VS_EDEVICE, "event record failed");
                lk.lock();
                if (st != VS_OK) {
                    event_pool.push_back(ev);
                    finish(j, st);
                } else {
                    j.inflight.push_back(ev);
                }
                progressed = true;
            }
            continue;
        }
        if (!j.inflight.empty()) continue;
        // all sweeps done: observables and read-back
        lk.unlock();
        vs_status st = VS_OK;
        unsigned long long cnt[2] = {0, 0};
        if (cudaMemcpyAsync(cnt, j.f->d_sweep, sizeof cnt, cudaMemcpyDeviceToHost, j.stream) != cudaSuccess ||
            cudaStreamSynchronize(j.stream) != cudaSuccess)
            st = fail(VS_EDEVICE, "job counters read failed");
        double S = 0;
        vs_vortex_report rep{};
        if (st == VS_OK) st = vs_action(j.f, &S);
        if (st == VS_OK) st = vs_vortex_check(j.f, &rep);
        if (st == VS_OK && j.spec.links_out) st = vs_read_field(j.f, j.spec.links_out, VS_HOST);
        lk.lock();
        j.result.action = S;
        j.result.n_reject = (int64_t)cnt[0];
        j.result.n_label_diff = rep.n_label_diff;
        finish(j, st);
        progressed = true;
    }
}

void Serve::loop() {
    cudaSetDevice(ctx->opt.device);
    std::unique_lock<std::mutex> lk(mu);
    while (!stop) {
        bool progressed = false;
        while (!stop && admit_one(lk)) progressed = true;
        step_running(lk, progressed);
        if (stop) break;
        if (running.empty() && waiting.empty()) {
            cv_work.wait(lk);
        } else if (!progressed) {
            cv_work.wait_for(lk, std::chrono::microseconds(50));
        }
    }
}

static Serve *serve_of(vs_ctx *c) {
    std::lock_guard<std::mutex> g(c->serve_init_mu);
    if (!c->serve) {
        auto s = std::make_unique<Serve>();
        s->ctx = c;
        cudaSetDevice(c->opt.device);
        int least = 0, greatest = 0;   // numerically: greatest <= least
        if (cudaDeviceGetStreamPriorityRange(&least, &greatest) != cudaSuccess) least = greatest = 0;
        s->n_levels = std::max(1, std::min(4, least - greatest + 1));
        for (int k = 0; k < c->opt.max_slots; ++k) {
            for (int l = 0; l < s->n_levels; ++l) {
                cudaStream_t st = nullptr;
                if (cudaStreamCreateWithPriority(&st, cudaStreamNonBlocking, greatest + l) != cudaSuccess)
                    return nullptr;
                s->streams.push_back(st);
            }
            s->slot_busy.push_back(false);
        }
        Serve *raw = s.release();
        raw->thr = std::thread([raw] { raw->loop(); });
        c->serve = raw;
    }
    return c->serve;
}

void serve_shutdown(vs_ctx *c) {
    if (!c->serve) return;
    Serve *s = c->serve;
    {
        std::lock_guard<std::mutex> g(s->mu);
        s->stop = true;
        for (auto &kv : s->jobs) kv.second->cancel = true;
    }
    s->cv_work.notify_all();
    if (s->thr.joinable()) s->thr.join();
    cudaSetDevice(c->opt.device);
    for (auto &kv : s->jobs) {
        Job &j = *kv.second;
        if (j.stream) cudaStreamSynchronize(j.stream);
        if (j.f) vs_field_destroy(j.f);
        if (j.graph) cudaGraphExecDestroy(j.graph);
        for (auto e : j.inflight) cudaEventDestroy(e);
    }
    for (auto e : s->event_pool) cudaEventDestroy(e);
    for (auto &kv : s->graph_pool)
        for (auto g : kv.second) cudaGraphExecDestroy(g);
    for (auto st : s->streams) cudaStreamDestroy(st);
    delete s;
    c->serve = nullptr;
}

}  // namespace vs

extern "C" vs_status vs_submit(vs_ctx *c, const vs_job *job, int64_t *ticket) {
    if (!c || !job || !ticket) return fail(VS_EINVAL, "vs_submit: NULL argument");
    int32_t d[4] = {job->dims[0], job->dims[1], job->dims[2], job->dims[3]};
    if (!valid_dims(d))
        return fail(VS_EINVAL, "vs_submit: extents must be positive multiples of 4 with at most 2^30 layout positions");
    if (job->precision != VS_FP32 && job->precision != VS_FP64) return fail(VS_EINVAL, "vs_submit: bad precision");
    if (job->storage != VS_LINK18 && job->storage != VS_LINK12) return fail(VS_EINVAL, "vs_submit: bad storage");
    if (job->precision == VS_FP64 && job->storage == VS_LINK12) return fail(VS_EUNSUPPORTED, "vs_submit: FP64 12-real");
    if (job->n_sweeps < 0 || job->n_cool < 0 || job->reunit_every < 0) return fail(VS_EINVAL, "vs_submit: negative count");
    if (!(job->omega < 0.25) || !std::isfinite(job->rho) || !std::isfinite(job->epsilon) || !(job->u0 > 0))
        return fail(VS_EINVAL, "vs_submit: bad omega / rho / epsilon / u0");
    Serve *s = serve_of(c);
    if (!s) return fail(VS_EDEVICE, "vs_submit: could not start the scheduler");
    auto j = std::make_shared<Job>();
    j->spec = *job;
    if (job->labels) {
        size_t n = 4 * (size_t)d[0] * d[1] * d[2] * d[3];
        j->labels.assign(job->labels, job->labels + n);
        for (int8_t v : j->labels)
            if (v < -1 || v > 1) return fail(VS_EINVAL, "vs_submit: label outside {-1,0,1}");
        j->spec.labels = nullptr;
    }
    if (j->spec.reunit_every > 0) j->chunk = j->spec.reunit_every;
    j->footprint = job_footprint(j->spec);
    std::lock_guard<std::mutex> g(s->mu);
    if ((int)s->waiting.size() >= c->opt.max_queue) return fail(VS_EBUSY, "vs_submit: queue full");
    j->ticket = s->next_ticket++;
    j->result.t_submit_ms = vs_now_ms(c);
    s->jobs[j->ticket] = j;
    s->waiting.push_back(j->ticket);
    ++s->n_submitted;
    *ticket = j->ticket;
    s->cv_work.notify_all();
    return VS_OK;
}

extern "C" vs_status vs_poll(vs_ctx *c, int64_t ticket, int32_t timeout_ms, vs_result *out) {
    if (!c || !out) return fail(VS_EINVAL, "vs_poll: NULL argument");
    if (!c->serve) return fail(VS_ENOTFOUND, "vs_poll: unknown ticket %lld", (long long)ticket);
    Serve *s = c->serve;
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->jobs.find(ticket);
    if (it == s->jobs.end()) return fail(VS_ENOTFOUND, "vs_poll: unknown ticket %lld", (long long)ticket);
    auto jp = it->second;
    auto done = [&] { return jp->state == DONE; };
    if (!done()) {
        if (timeout_ms == 0) return VS_EAGAIN;
        if (timeout_ms < 0) s->cv_done.wait(lk, done);
        else if (!s->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), done))
            return fail(VS_ETIMEDOUT, "vs_poll: ticket %lld not done after %d ms", (long long)ticket, timeout_ms);
    }
    *out = jp->result;
    s->jobs.erase(ticket);
    return VS_OK;
}

extern "C" vs_status vs_cancel(vs_ctx *c, int64_t ticket) {
    if (!c || !c->serve) return fail(VS_ENOTFOUND, "vs_cancel: unknown ticket");
    Serve *s = c->serve;
    std::lock_guard<std::mutex> g(s->mu);
    auto it = s->jobs.find(ticket);
    if (it == s->jobs.end() || it->second->state == DONE)
        return fail(VS_ENOTFOUND, "vs_cancel: unknown or finished ticket %lld", (long long)ticket);
    Job &j = *it->second;
    j.cancel = true;
    if (j.state == WAITING) s->finish(j, VS_OK);
    s->cv_work.notify_all();
    return VS_OK;
}

extern "C" vs_status vs_serve_stats_get(vs_ctx *c, vs_serve_stats *out) {
    if (!c || !out) return fail(VS_EINVAL, "vs_serve_stats_get: NULL argument");
    memset(out, 0, sizeof *out);
    if (!c->serve) return VS_OK;
    Serve *s = c->serve;
    std::lock_guard<std::mutex> g(s->mu);
    out->submitted = s->n_submitted;
    out->completed = s->n_completed;
    out->cancelled = s->n_cancelled;
    out->running = (int64_t)s->running.size();
    out->waiting = (int64_t)s->waiting.size();
    out->bytes_in_use = s->bytes_in_use;
    out->peak_bytes_in_use = s->peak_bytes;
    out->graphs_instantiated = s->graphs_instantiated;
    out->graphs_reused = s->graphs_reused;
    return VS_OK;
}
