// rms_serve.cu -- continuous-batching serving loop for simulation requests.
//
// Requests (a sequence -- hence a resident substrate -- plus walkers, seed
// and precision) arrive at any time.  A scheduler thread admits them while
// the device-memory budget and the request slots allow, and then, tick by
// tick, advances EVERY active request by up to `steps_per_tick` steps with
// one batched launch per (precision, shape-count bucket): each block of the
// launch carries a block of walkers of one request (walk_batched_kernel), so
// requests of different substrates, sizes and sequences share the GPU in the
// same kernels.  The tick (task-table upload + the batched launches) is
// captured into a CUDA graph and replayed; when the next tick has the same
// shape the executable graph is updated in place instead of re-instantiated.
// A request that has taken all its steps gets its moment sums and read-out
// (the same kernels as rms_run) and leaves; its memory and slot go to the
// next request in the queue.
//
// A request's result does not depend on what it shares the GPU with: its
// walkers keep their blocks and their counter-based random streams, and its
// reductions run over its own blocks in a fixed order.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <vector>

#include "rms_handles.h"
#include "rms_internal.h"

using namespace rms;

namespace {

using Clock = std::chrono::steady_clock;

enum class St { Pending, Active, Finalizing, Done, Failed, Cancelled };

struct Request {
    int64_t ticket = 0;
    rms_sequence *seq = nullptr;
    int64_t W = 0;
    uint64_t seed = 0;
    int32_t precision = RMS_FP64;
    rms_run_handle *run = nullptr;
    int64_t progress = 0;
    size_t bytes = 0;
    int slot = -1;
    int bucket = 1;
    St st = St::Pending;
    bool cancel = false;
    rms_status err = RMS_OK;
    std::string msg;
    Clock::time_point t_submit, t_admit, t_done;
    int64_t ticks = 0;  // ticks the request took part in
    double *h_out = nullptr;  // pinned: S [2*(n_combo+1)], moments [n_rec*22], status word
    size_t h_out_bytes = 0;
    cudaEvent_t done_ev = nullptr;
    std::vector<double> S, moments;
    double alpha_sum = 0;
};

int bucket_of(int n_shapes) { return n_shapes <= 1 ? 1 : n_shapes <= 2 ? 2 : n_shapes <= 4 ? 4 : 8; }
int bucket_index(int b) { return b == 1 ? 0 : b == 2 ? 1 : b == 4 ? 2 : 3; }

}  // namespace

struct rms_server {
    int device = 0;
    rms_server_config cfg{};
    cudaStream_t stream = nullptr;
    std::thread th;
    std::mutex mu;
    std::condition_variable cv, cv_done;
    bool stop = false;
    int64_t next_ticket = 1;
    std::deque<Request *> pending;
    std::vector<Request *> active, finalizing;
    std::map<int64_t, Request *> reqs;
    size_t mem_used = 0;
    std::vector<int> free_slots;
    ReqDesc<float> *d_req32 = nullptr, *h_req32 = nullptr;
    ReqDesc<double> *d_req64 = nullptr, *h_req64 = nullptr;
    BlockTask *h_tasks[2] = {nullptr, nullptr}, *d_tasks[2] = {nullptr, nullptr};
    int64_t task_cap = 0;
    cudaEvent_t buf_ev[2] = {nullptr, nullptr};
    // written by the scheduler thread only; atomic because rms_server_stats
    // reads them from other threads while it runs
    std::atomic<int64_t> tick{0};
    cudaGraphExec_t exec = nullptr;
    std::atomic<int64_t> graph_updates{0}, graph_instantiations{0};
    std::vector<std::pair<double *, size_t>> pinned_pool;
    // block slots of the batched kernel: [precision: 0 FP32, 1 FP64][shape bucket]
    int64_t slots[2][4] = {};
    // statistics
    std::vector<double> lat_ms;
    std::atomic<double> walker_steps{0.0};  // scheduler thread only (see tick)
    std::atomic<int> in_flight{0};          // active + finalizing, published by the scheduler thread
    Clock::time_point t_first, t_last;
    bool have_first = false;
    int64_t completed = 0;
    int peak_active = 0;
};

namespace {

// active + finalizing for rms_server_stats; called by the scheduler thread,
// the only writer of both lists, after it changes either
void publish_in_flight(rms_server *s)
{
    s->in_flight.store((int)(s->active.size() + s->finalizing.size()));
}

double *take_pinned(rms_server *s, size_t bytes)
{
    for (size_t i = 0; i < s->pinned_pool.size(); ++i)
        if (s->pinned_pool[i].second >= bytes) {
            double *p = s->pinned_pool[i].first;
            s->pinned_pool.erase(s->pinned_pool.begin() + i);
            return p;
        }
    double *p = nullptr;
    if (cudaMallocHost((void **)&p, bytes) != cudaSuccess) return nullptr;
    return p;
}

rms_status grow_tasks(rms_server *s, int64_t need)
{
    if (need <= s->task_cap) return RMS_OK;
    RMS_CUDA(cudaStreamSynchronize(s->stream));
    int64_t cap = std::max<int64_t>(need, 2 * s->task_cap);
    for (int j = 0; j < 2; ++j) {
        if (s->h_tasks[j]) cudaFreeHost(s->h_tasks[j]);
        if (s->d_tasks[j]) cudaFree(s->d_tasks[j]);
        RMS_CUDA(cudaMallocHost((void **)&s->h_tasks[j], sizeof(BlockTask) * cap));
        RMS_CUDA(cudaMalloc((void **)&s->d_tasks[j], sizeof(BlockTask) * cap));
    }
    s->task_cap = cap;
    return RMS_OK;
}

// The sequence reference is released under the same lock that makes the
// failure visible: a waiter may delete the request as soon as it sees it.
void fail_request(rms_server *s, Request *q, rms_status err, const char *msg)
{
    std::lock_guard<std::mutex> lk(s->mu);
    q->seq->refs.fetch_sub(1);
    q->st = St::Failed;
    q->err = err;
    q->msg = msg;
    s->cv_done.notify_all();
}

// Admit queued requests while slots and the memory budget allow (at least
// one request is always admitted when nothing else is in flight).
void admit(rms_server *s)
{
    for (;;) {
        Request *q = nullptr;
        size_t need = 0;
        {
            std::lock_guard<std::mutex> lk(s->mu);
            while (!s->pending.empty() && s->pending.front()->cancel) {
                Request *c = s->pending.front();
                s->pending.pop_front();
                c->st = St::Cancelled;
                c->seq->refs.fetch_sub(1);
                s->cv_done.notify_all();
            }
            if (s->pending.empty() || s->free_slots.empty()) return;
            q = s->pending.front();
            need = run_state_bytes(q->seq, q->W, q->precision, 0);
            const bool idle = s->active.empty() && s->finalizing.empty();
            if (!idle && s->mem_used + need > (size_t)s->cfg.memory_budget_bytes) return;
            s->pending.pop_front();
        }
        rms_run_handle *r = new (std::nothrow) rms_run_handle();
        if (!r) {
            fail_request(s, q, RMS_E_OOM, "host allocation");
            continue;
        }
        r->seq = q->seq;
        r->W = q->W;
        r->seed = q->seed;
        r->precision = q->precision;
        r->stream = s->stream;
        rms_status st = run_setup(r, false);
        if (st == RMS_OK) st = run_init(r);
        const int n_combo = q->seq->S * q->seq->n_dirs * q->seq->n_b;
        q->h_out_bytes = sizeof(double) * (2 * (size_t)(n_combo + 1) + (size_t)q->seq->n_rec * kMoments + 1);
        q->h_out = st == RMS_OK ? take_pinned(s, q->h_out_bytes) : nullptr;
        if (st == RMS_OK && !q->h_out) st = RMS_E_OOM;
        if (st == RMS_OK && cudaEventCreateWithFlags(&q->done_ev, cudaEventDisableTiming) != cudaSuccess)
            st = RMS_E_CUDA;
        if (st != RMS_OK) {
            run_free(r, true);
            delete r;
            if (q->h_out) {  // back to the pool: the request never ran
                s->pinned_pool.emplace_back(q->h_out, q->h_out_bytes);
                q->h_out = nullptr;
            }
            fail_request(s, q, st, rms_last_error());
            continue;
        }
        int slot;
        {
            std::lock_guard<std::mutex> lk(s->mu);
            slot = s->free_slots.back();
            s->free_slots.pop_back();
        }
        if (q->precision == RMS_FP32) {
            s->h_req32[slot] = run_desc<float>(r);
            cudaMemcpyAsync(s->d_req32 + slot, s->h_req32 + slot, sizeof(ReqDesc<float>), cudaMemcpyHostToDevice,
                            s->stream);
        } else {
            s->h_req64[slot] = run_desc<double>(r);
            cudaMemcpyAsync(s->d_req64 + slot, s->h_req64 + slot, sizeof(ReqDesc<double>), cudaMemcpyHostToDevice,
                            s->stream);
        }
        q->run = r;
        q->slot = slot;
        q->bytes = need;
        q->bucket = bucket_of(q->seq->S);
        s->mem_used += need;
        s->active.push_back(q);
        publish_in_flight(s);
        std::lock_guard<std::mutex> lk(s->mu);
        q->t_admit = Clock::now();
        q->st = St::Active;
        s->peak_active = std::max<int>(s->peak_active, (int)(s->active.size() + s->finalizing.size()));
    }
}

// One tick: every active request advances by up to steps_per_tick steps.
rms_status tick_once(rms_server *s)
{
    NvtxRange nvtx_range("rms: serving tick");
    const int j = (int)(s->tick.load() & 1);
    RMS_CUDA(cudaEventSynchronize(s->buf_ev[j]));  // the upload from buffer j has run
    // drop cancelled requests from the active set (their memory is released
    // stream-ordered, after every launch that may still use it)
    for (size_t i = 0; i < s->active.size();) {
        Request *q = s->active[i];
        bool c;
        {
            std::lock_guard<std::mutex> lk(s->mu);
            c = q->cancel;
        }
        if (c) {
            run_free(q->run, false);
            delete q->run;
            q->run = nullptr;
            s->mem_used -= q->bytes;
            s->pinned_pool.emplace_back(q->h_out, q->h_out_bytes);
            cudaEventDestroy(q->done_ev);
            std::lock_guard<std::mutex> lk(s->mu);
            s->free_slots.push_back(q->slot);
            q->st = St::Cancelled;
            q->seq->refs.fetch_sub(1);
            s->cv_done.notify_all();
            s->active.erase(s->active.begin() + i);
            publish_in_flight(s);
        } else {
            ++i;
        }
    }
    if (s->active.empty()) return RMS_OK;
    int64_t need = 0;
    for (Request *q : s->active) need += q->run->n_blocks;
    RMS_TRY(grow_tasks(s, need));
    BlockTask *T = s->h_tasks[j];
    int64_t start[8], count[8], off = 0;
    std::vector<std::pair<int64_t, int64_t>> range(s->active.size());
    for (int g = 0; g < 8; ++g) {  // groups: precision x shape bucket
        const int prec = g / 4 == 0 ? RMS_FP32 : RMS_FP64;
        start[g] = off;
        // RMS_SERVE_FILL: the launch of this group lasts `waves` x steps_per_tick
        // block-steps (its blocks over the GPU's block slots); requests whose
        // blocks fit in one wave take that many steps
        int64_t blocks = 0;
        for (Request *q : s->active)
            if (q->precision == prec && bucket_index(q->bucket) == g % 4) blocks += q->run->n_blocks;
        const int64_t slots = s->slots[g / 4][g % 4];
        const int64_t waves = std::min<int64_t>(64, std::max<int64_t>(1, blocks / std::max<int64_t>(slots, 1)));
        // the requests that run the whole launch go first, so that their blocks
        // take slots from the start instead of stretching its end
        for (int pass = 0; pass < 2; ++pass)
            for (size_t i = 0; i < s->active.size(); ++i) {
                Request *q = s->active[i];
                if (q->precision != prec || bucket_index(q->bucket) != g % 4) continue;
                const bool filling = s->cfg.policy == RMS_SERVE_FILL && q->run->n_blocks < slots && waves > 1;
                if (filling != (pass == 0)) continue;
                const int64_t quota = s->cfg.steps_per_tick * (filling ? waves : 1);
                const int64_t k0 = q->progress;
                const int64_t k1 = std::min<int64_t>(q->seq->n_steps, k0 + quota);
                range[i] = {k0, k1};
                ++q->ticks;
                for (int64_t b = 0; b < q->run->n_blocks; ++b) T[off++] = BlockTask{q->slot, 0, b, k0, k1};
            }
        count[g] = off - start[g];
    }
    cudaGraph_t graph = nullptr;
    RMS_CUDA(cudaStreamBeginCapture(s->stream, cudaStreamCaptureModeThreadLocal));
    cudaMemcpyAsync(s->d_tasks[j], T, sizeof(BlockTask) * off, cudaMemcpyHostToDevice, s->stream);
    for (int g = 0; g < 8; ++g) {
        if (!count[g]) continue;
        const int bucket = 1 << (g % 4);
        if (g / 4 == 0)
            launch_walk_batched<float>(bucket, (int32_t)count[g], s->stream, s->d_req32, s->d_tasks[j] + start[g]);
        else
            launch_walk_batched<double>(bucket, (int32_t)count[g], s->stream, s->d_req64, s->d_tasks[j] + start[g]);
    }
    RMS_CUDA(cudaStreamEndCapture(s->stream, &graph));
    if (s->exec) {
        cudaGraphExecUpdateResultInfo info;
        if (cudaGraphExecUpdate(s->exec, graph, &info) == cudaSuccess) {
            ++s->graph_updates;
        } else {
            cudaGetLastError();
            cudaGraphExecDestroy(s->exec);
            s->exec = nullptr;
        }
    }
    if (!s->exec) {
        const cudaError_t e = cudaGraphInstantiate(&s->exec, graph, 0);
        if (e != cudaSuccess) {
            cudaGraphDestroy(graph);
            RMS_CUDA(e);
        }
        ++s->graph_instantiations;
    }
    cudaGraphDestroy(graph);
    RMS_CUDA(cudaGraphLaunch(s->exec, s->stream));
    RMS_CUDA(cudaEventRecord(s->buf_ev[j], s->stream));
    ++s->tick;
    // requests that have taken all their steps: reductions, read-out, copy-back
    for (size_t i = 0; i < s->active.size();) {
        Request *q = s->active[i];
        s->walker_steps.store(s->walker_steps.load() + (double)q->W * (double)(range[i].second - range[i].first));
        q->progress = range[i].second;
        if (q->progress >= q->seq->n_steps) {
            rms_run_handle *r = q->run;
            RMS_TRY(run_finalize(r));
            const size_t nS = 2 * (size_t)(r->n_combo + 1);
            RMS_CUDA(cudaMemcpyAsync(q->h_out, normalised_S(r), sizeof(double) * nS, cudaMemcpyDeviceToHost,
                                     s->stream));
            if (q->seq->n_rec > 0)
                RMS_CUDA(cudaMemcpyAsync(q->h_out + nS, r->d_mom, sizeof(double) * q->seq->n_rec * kMoments,
                                         cudaMemcpyDeviceToHost, s->stream));
            RMS_CUDA(cudaMemcpyAsync(q->h_out + nS + (size_t)q->seq->n_rec * kMoments, r->d_status, sizeof(int32_t),
                                     cudaMemcpyDeviceToHost, s->stream));
            RMS_CUDA(cudaEventRecord(q->done_ev, s->stream));
            {
                std::lock_guard<std::mutex> lk(s->mu);
                q->st = St::Finalizing;
            }
            s->finalizing.push_back(q);
            s->active.erase(s->active.begin() + i);
            publish_in_flight(s);
            range.erase(range.begin() + i);
        } else {
            ++i;
        }
    }
    return RMS_OK;
}

// Requests whose results have reached host memory.
void poll_finalizing(rms_server *s)
{
    for (size_t i = 0; i < s->finalizing.size();) {
        Request *q = s->finalizing[i];
        if (cudaEventQuery(q->done_ev) != cudaSuccess) {
            ++i;
            continue;
        }
        rms_run_handle *r = q->run;
        const size_t nS = 2 * (size_t)(r->n_combo + 1);
        const int n_combo = r->n_combo;
        const size_t nm = (size_t)q->seq->n_rec * kMoments;
        int32_t status = 0;
        std::memcpy(&status, q->h_out + nS + nm, sizeof(int32_t));
        std::vector<double> S(q->h_out, q->h_out + nS), M(q->h_out + nS, q->h_out + nS + nm);
        run_free(r, false);
        delete r;
        q->run = nullptr;
        cudaEventDestroy(q->done_ev);
        s->pinned_pool.emplace_back(q->h_out, q->h_out_bytes);
        q->h_out = nullptr;
        s->mem_used -= q->bytes;
        std::lock_guard<std::mutex> lk(s->mu);
        q->t_done = Clock::now();
        s->t_last = q->t_done;
        q->S.assign(S.begin(), S.begin() + 2 * n_combo);
        q->alpha_sum = S[2 * n_combo];
        q->moments = std::move(M);
        if (status) {
            q->st = St::Failed;
            q->err = RMS_E_DEVICE;
            q->msg = "a kernel reported a broken invariant";
        } else {
            q->st = St::Done;
        }
        s->lat_ms.push_back(std::chrono::duration<double, std::milli>(q->t_done - q->t_submit).count());
        ++s->completed;
        s->free_slots.push_back(q->slot);
        q->seq->refs.fetch_sub(1);
        s->cv_done.notify_all();
        s->finalizing.erase(s->finalizing.begin() + i);
        publish_in_flight(s);
    }
}

void scheduler(rms_server *s)
{
    cudaSetDevice(s->device);
    for (;;) {
        {
            std::unique_lock<std::mutex> lk(s->mu);
            if (s->stop && s->active.empty() && s->finalizing.empty()) {
                for (Request *q : s->pending) {
                    q->st = St::Cancelled;
                    q->seq->refs.fetch_sub(1);
                }
                s->pending.clear();
                s->cv_done.notify_all();
                break;
            }
            if (s->stop)
                for (Request *q : s->pending) q->cancel = true;
        }
        admit(s);
        if (!s->active.empty()) {
            const rms_status st = tick_once(s);
            if (st != RMS_OK) {
                // a CUDA failure: fail everything in flight and stop scheduling
                cudaStreamSynchronize(s->stream);
                std::vector<Request *> all(s->active);
                all.insert(all.end(), s->finalizing.begin(), s->finalizing.end());
                for (Request *q : all) {
                    if (q->run) {
                        run_free(q->run, true);
                        delete q->run;
                        q->run = nullptr;
                    }
                    s->mem_used -= q->bytes;
                    std::lock_guard<std::mutex> lk(s->mu);
                    s->free_slots.push_back(q->slot);
                    q->st = St::Failed;
                    q->err = st;
                    q->msg = "serving tick failed";
                    q->seq->refs.fetch_sub(1);
                }
                s->active.clear();
                s->finalizing.clear();
                publish_in_flight(s);
                s->cv_done.notify_all();
            }
        }
        poll_finalizing(s);
        if (s->active.empty()) {
            std::unique_lock<std::mutex> lk(s->mu);
            const bool waiting_results = !s->finalizing.empty();
            s->cv.wait_for(lk, std::chrono::microseconds(waiting_results ? 50 : 1000),
                           [&] { return s->stop || (!s->pending.empty() && !s->free_slots.empty()); });
        }
    }
}

}  // namespace

extern "C" rms_status rms_server_create(const rms_server_config *cfg, rms_server **out)
{
    if (!out) return fail(RMS_E_INVALID_ARG, "null argument");
    *out = nullptr;
    rms_server_config c = cfg ? *cfg : rms_server_config{};
    if (c.memory_budget_bytes < 0 || c.max_active < 0 || c.max_active > 1024 || c.steps_per_tick < 0 ||
        (c.policy != RMS_SERVE_STEPS && c.policy != RMS_SERVE_FILL))
        return fail(RMS_E_INVALID_ARG, "server config out of range");
    if (c.memory_budget_bytes == 0) c.memory_budget_bytes = 8ll << 30;
    if (c.max_active == 0) c.max_active = 64;
    if (c.steps_per_tick == 0) c.steps_per_tick = 256;
    rms_server *s = new (std::nothrow) rms_server();
    if (!s) return fail(RMS_E_OOM, "host allocation");
    s->cfg = c;
    cudaGetDevice(&s->device);
    int sms = 1;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, s->device);
    for (int b = 0; b < 4; ++b) {
        s->slots[0][b] = (int64_t)sms * batched_blocks_per_sm<float>(1 << b);
        s->slots[1][b] = (int64_t)sms * batched_blocks_per_sm<double>(1 << b);
    }
    auto bail = [&](cudaError_t e) {
        rms_status st = fail(e == cudaErrorMemoryAllocation ? RMS_E_OOM : RMS_E_CUDA, cudaGetErrorString(e));
        if (s->stream) cudaStreamDestroy(s->stream);
        delete s;
        return st;
    };
    cudaError_t e;
    if ((e = cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking)) != cudaSuccess) return bail(e);
    if ((e = cudaMalloc((void **)&s->d_req32, sizeof(ReqDesc<float>) * c.max_active)) != cudaSuccess) return bail(e);
    if ((e = cudaMalloc((void **)&s->d_req64, sizeof(ReqDesc<double>) * c.max_active)) != cudaSuccess) return bail(e);
    if ((e = cudaMallocHost((void **)&s->h_req32, sizeof(ReqDesc<float>) * c.max_active)) != cudaSuccess)
        return bail(e);
    if ((e = cudaMallocHost((void **)&s->h_req64, sizeof(ReqDesc<double>) * c.max_active)) != cudaSuccess)
        return bail(e);
    for (int j = 0; j < 2; ++j)
        if ((e = cudaEventCreateWithFlags(&s->buf_ev[j], cudaEventDisableTiming)) != cudaSuccess) return bail(e);
    for (int i = c.max_active - 1; i >= 0; --i) s->free_slots.push_back(i);
    s->th = std::thread(scheduler, s);
    *out = s;
    return RMS_OK;
}

extern "C" rms_status rms_server_submit(rms_server *s, rms_sequence *seq, int64_t n_walkers, uint64_t seed,
                                        int32_t precision, int64_t *ticket)
{
    if (!s || !seq || !ticket) return fail(RMS_E_INVALID_ARG, "null argument");
    if (n_walkers < 1 || n_walkers > (1ll << 31) - 1) return fail(RMS_E_INVALID_ARG, "n_walkers out of range");
    if (precision != RMS_FP32 && precision != RMS_FP64) return fail(RMS_E_INVALID_ARG, "precision");
    if (seq->d_Tmt) return fail(RMS_E_INVALID_ARG, "served requests have no absorbing membranes (rho); use rms_run");
    Request *q = new (std::nothrow) Request();
    if (!q) return fail(RMS_E_OOM, "host allocation");
    q->seq = seq;
    q->W = n_walkers;
    q->seed = seed;
    q->precision = precision;
    q->t_submit = Clock::now();
    seq->refs.fetch_add(1);
    {
        std::lock_guard<std::mutex> lk(s->mu);
        if (s->stop) {
            seq->refs.fetch_sub(1);
            delete q;
            return fail(RMS_E_INVALID_ARG, "server is shutting down");
        }
        q->ticket = s->next_ticket++;
        if (!s->have_first) {
            s->have_first = true;
            s->t_first = q->t_submit;
        }
        s->reqs[q->ticket] = q;
        s->pending.push_back(q);
    }
    s->cv.notify_all();
    *ticket = q->ticket;
    return RMS_OK;
}

extern "C" rms_status rms_server_poll(rms_server *s, int64_t ticket)
{
    if (!s) return fail(RMS_E_INVALID_ARG, "null server");
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end()) return fail(RMS_E_INVALID_ARG, "unknown ticket");
    const St st = it->second->st;
    return (st == St::Done || st == St::Failed || st == St::Cancelled) ? RMS_OK : RMS_E_NOT_READY;
}

extern "C" rms_status rms_server_wait(rms_server *s, int64_t ticket, int64_t timeout_ms, double *S_re, double *S_im,
                                      double *moments, double *alpha_sum)
{
    if (!s) return fail(RMS_E_INVALID_ARG, "null server");
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end()) return fail(RMS_E_INVALID_ARG, "unknown ticket");
    Request *q = it->second;
    auto done = [&] { return q->st == St::Done || q->st == St::Failed || q->st == St::Cancelled; };
    if (timeout_ms < 0)
        s->cv_done.wait(lk, done);
    else if (!s->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), done))
        return fail(RMS_E_TIMEOUT, "request not finished within the timeout");
    rms_status st = RMS_OK;
    if (q->st == St::Cancelled) {
        st = fail(RMS_E_CANCELLED, "request was cancelled");
    } else if (q->st == St::Failed) {
        st = fail(q->err, q->msg);
    } else {
        const size_t n = q->S.size() / 2;
        for (size_t k = 0; k < n; ++k) {
            if (S_re) S_re[k] = q->S[2 * k];
            if (S_im) S_im[k] = q->S[2 * k + 1];
        }
        if (moments) std::copy(q->moments.begin(), q->moments.end(), moments);
        if (alpha_sum) *alpha_sum = q->alpha_sum;
    }
    s->reqs.erase(it);
    delete q;
    return st;
}

extern "C" rms_status rms_server_request_info(rms_server *s, int64_t ticket, double *out)
{
    if (!s || !out) return fail(RMS_E_INVALID_ARG, "null argument");
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end()) return fail(RMS_E_INVALID_ARG, "unknown ticket");
    const Request *q = it->second;
    if (q->st != St::Done) return q->st == St::Failed || q->st == St::Cancelled
                                      ? fail(RMS_E_INVALID_ARG, "the request did not complete")
                                      : RMS_E_NOT_READY;
    out[0] = std::chrono::duration<double, std::milli>(q->t_admit - q->t_submit).count();
    out[1] = std::chrono::duration<double, std::milli>(q->t_done - q->t_submit).count();
    out[2] = (double)q->W * (double)q->seq->n_steps;
    out[3] = (double)q->ticks;
    return RMS_OK;
}

extern "C" rms_status rms_server_cancel(rms_server *s, int64_t ticket)
{
    if (!s) return fail(RMS_E_INVALID_ARG, "null server");
    {
        std::lock_guard<std::mutex> lk(s->mu);
        auto it = s->reqs.find(ticket);
        if (it == s->reqs.end()) return fail(RMS_E_INVALID_ARG, "unknown ticket");
        it->second->cancel = true;
    }
    s->cv.notify_all();
    return RMS_OK;
}

extern "C" rms_status rms_server_stats(rms_server *s, double *out)
{
    if (!s || !out) return fail(RMS_E_INVALID_ARG, "null argument");
    std::lock_guard<std::mutex> lk(s->mu);
    std::vector<double> l(s->lat_ms);
    std::sort(l.begin(), l.end());
    auto pct = [&](double p) {
        if (l.empty()) return 0.0;
        const double x = p * (l.size() - 1);
        const size_t i = (size_t)x;
        const double f = x - i;
        return i + 1 < l.size() ? l[i] * (1 - f) + l[i + 1] * f : l[i];
    };
    double mean = 0;
    for (double v : l) mean += v;
    mean = l.empty() ? 0.0 : mean / l.size();
    const double span = s->have_first && s->completed
                            ? std::chrono::duration<double>(s->t_last - s->t_first).count()
                            : 0.0;
    out[0] = pct(0.50);
    out[1] = pct(0.99);
    out[2] = mean;
    out[3] = span > 0 ? s->walker_steps.load() / span : 0.0;
    out[4] = (double)s->completed;
    out[5] = (double)s->in_flight.load();
    out[6] = (double)s->pending.size();
    out[7] = (double)s->peak_active;
    out[8] = (double)s->tick.load();
    out[9] = (double)s->graph_updates.load();
    out[10] = (double)s->graph_instantiations.load();
    return RMS_OK;
}

extern "C" rms_status rms_server_destroy(rms_server *s)
{
    if (!s) return RMS_OK;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
        for (auto &kv : s->reqs) kv.second->cancel = true;
    }
    s->cv.notify_all();
    if (s->th.joinable()) s->th.join();
    cudaStreamSynchronize(s->stream);
    for (auto &kv : s->reqs) delete kv.second;
    if (s->exec) cudaGraphExecDestroy(s->exec);
    for (int j = 0; j < 2; ++j) {
        if (s->h_tasks[j]) cudaFreeHost(s->h_tasks[j]);
        if (s->d_tasks[j]) cudaFree(s->d_tasks[j]);
        if (s->buf_ev[j]) cudaEventDestroy(s->buf_ev[j]);
    }
    for (auto &p : s->pinned_pool) cudaFreeHost(p.first);
    cudaFree(s->d_req32);
    cudaFree(s->d_req64);
    cudaFreeHost(s->h_req32);
    cudaFreeHost(s->h_req64);
    cudaStreamDestroy(s->stream);
    delete s;
    return RMS_OK;
}
