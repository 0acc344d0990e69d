// Serving loop: continuous batching of QQMC requests (Q_1..Q_nmax of one dot
// each) over a parameter sweep.
//
// A worker thread owns the device work.  Requests wait in a FIFO queue and are
// admitted while the device-memory budget allows (tables + shift words +
// partial sums of every order of the request).  Each admission round turns
// the newly admitted requests into ONE batched plan (all their orders share a
// persistent kernel launch) on its own stream; rounds overlap on the device:
// a request that arrives while earlier batches run is admitted as soon as
// memory frees up and its kernels start as SMs drain (rounds with less work on
// higher-priority streams, see round_priority).  Completed batches are
// detected with events, their results finalised per request, and their memory
// returned to the budget.
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <chrono>
#include <condition_variable>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "qqmc_internal.h"

using namespace qqmc;
using Clock = std::chrono::steady_clock;

namespace {

enum State { PENDING, ADMITTED, DONE, FAILED, CANCELLED };

struct Req {
    uint64_t handle;
    qqmc_request r;
    Clock::time_point t_submit, t_admit;
    State state = PENDING;
    int status = QQMC_PENDING;
    qqmc_series out{};
    uint64_t bytes = 0;
};

struct Batch {
    uint64_t id = 0;  // admission round
    std::vector<uint64_t> handles;
    std::vector<qqmc_problem *> problems;
    qqmc_plan *plan = nullptr;
    cudaStream_t stream = nullptr;
    cudaEvent_t done = nullptr;
    uint64_t bytes = 0;
};

// Stream priority of an admission round: the less work (Keldysh determinants,
// N K 2^n summed over the round's items), the higher the priority, so that a
// short round's blocks are dispatched as a long round's persistent blocks retire,
// ahead of that round's remaining kernels, instead of queueing behind all of them.
int round_priority(const std::vector<qqmc_request> &rq) {
    int least = 0, greatest = 0;
    if (cudaDeviceGetStreamPriorityRange(&least, &greatest) != cudaSuccess) return 0;
    double work = 1.0;
    for (const auto &r : rq)
        for (int n = 1; n <= r.n_max; ++n) work += (double)r.n_points * r.n_shifts * ldexp(1.0, n);
    double x = (log2(work) - 20.0) / 10.0;  // 2^20 determinants and less: greatest; 2^30 and more: least
    x = x < 0.0 ? 0.0 : (x > 1.0 ? 1.0 : x);
    return greatest + (int)lround(x * (least - greatest));
}

uint64_t request_bytes(const qqmc_request &r) {
    uint64_t b = (uint64_t)(r.params.n_table / 2 + 1) * (32 + 16);
    uint64_t cps = (r.n_points + kChunk - 1) / kChunk;
    for (int n = 1; n <= r.n_max; ++n) b += (uint64_t)r.n_shifts * (cps * 36 + 4 * n + 24) + 256;
    return b;
}

}  // namespace

struct qqmc_server {
    qqmc_server_opts opts{};
    int device = 0;
    std::mutex mu;
    std::condition_variable cv;
    std::deque<uint64_t> queue;
    std::unordered_map<uint64_t, Req> reqs;
    std::vector<Batch> inflight;
    // Finished rounds whose plans and problems wait to be freed: cudaFree waits for the whole
    // device, so it runs only when no round is in flight (or at shutdown).
    std::vector<Batch> retired;
    void free_retired();
    uint64_t next_handle = 1;
    uint64_t next_batch = 1;
    uint64_t bytes_in_use = 0;
    bool stop = false;
    std::thread worker;
    void run();
    void finish_batch(Batch &b);
    void fail_batch(Batch &b, int code);
};

void qqmc_server::fail_batch(Batch &b, int code) {
    for (uint64_t h : b.handles) {
        auto it = reqs.find(h);
        if (it == reqs.end()) continue;
        if (it->second.state == ADMITTED) {
            it->second.state = FAILED;
            it->second.status = code;
            it->second.out.status = code;
        }
    }
}

void qqmc_server::finish_batch(Batch &b) {
    // results of all items (ordered request by request, order 1..n_max)
    size_t n_items = 0;
    std::vector<int> nmax;
    {
        std::lock_guard<std::mutex> lk(mu);
        for (uint64_t h : b.handles) {
            auto it = reqs.find(h);
            int nm = it != reqs.end() ? it->second.r.n_max : 0;
            nmax.push_back(nm);
            n_items += nm;
        }
    }
    std::vector<qqmc_result> res(n_items);
    int rc = qqmc_plan_results(b.plan, res.data(), nullptr);
    uint64_t t0 = 0, t1 = 0;
    if (rc == QQMC_OK || rc == QQMC_E_NONFINITE) qqmc_plan_device_span(b.plan, &t0, &t1);
    Clock::time_point now = Clock::now();
    std::lock_guard<std::mutex> lk(mu);
    size_t off = 0;
    for (size_t q = 0; q < b.handles.size(); ++q) {
        auto it = reqs.find(b.handles[q]);
        if (it == reqs.end()) {
            off += nmax[q];
            continue;
        }
        Req &R = it->second;
        // a non-finite sum fails only the requests whose own items carry it
        bool bad = false;
        if (rc == QQMC_E_NONFINITE)
            for (int n = 1; n <= nmax[q]; ++n) bad = bad || res[off + n - 1].n_nonfinite != 0;
        const int rq = bad ? QQMC_E_NONFINITE : (rc == QQMC_E_NONFINITE ? QQMC_OK : rc);
        if (R.state == ADMITTED) {
            if (rq != QQMC_OK) {
                R.state = FAILED;
                R.status = rq;
                R.out.status = rq;
            } else {
                double U = R.r.U, Un = 1.0, sum = R.out.q[0];
                for (int n = 1; n <= R.r.n_max; ++n) {
                    const qqmc_result &x = res[off + n - 1];
                    R.out.q[n] = x.q_mean;
                    R.out.q_err[n] = x.q_err;
                    R.out.n_in_domain += x.n_in_domain;
                    Un *= U;
                    sum += x.q_mean * Un;
                }
                R.out.series_sum = sum;
                R.out.batch = b.id;
                R.out.device_start_ns = t0;
                R.out.device_end_ns = t1;
                R.out.latency_ms = std::chrono::duration<double, std::milli>(now - R.t_submit).count();
                R.out.status = QQMC_OK;
                R.state = DONE;
                R.status = QQMC_OK;
            }
        }
        off += nmax[q];
    }
    bytes_in_use -= b.bytes;
    cv.notify_all();
}

void qqmc_server::free_retired() {
    for (Batch &b : retired) {
        qqmc_plan_destroy(b.plan);
        for (auto *p : b.problems) qqmc_destroy_problem(p);
    }
    retired.clear();
}

void qqmc_server::run() {
    cudaSetDevice(device);
    std::unique_lock<std::mutex> lk(mu);
    while (true) {
        // 1. completed batches
        for (size_t i = 0; i < inflight.size();) {
            cudaError_t q = cudaEventQuery(inflight[i].done);
            if (q == cudaErrorNotReady) {
                ++i;
                continue;
            }
            Batch b = inflight[i];
            inflight.erase(inflight.begin() + i);
            lk.unlock();
            if (q != cudaSuccess) {
                lk.lock();
                fail_batch(b, cuda_error(q, "batch execution"));
                bytes_in_use -= b.bytes;
                lk.unlock();
            } else {
                finish_batch(b);
            }
            cudaEventDestroy(b.done);
            cudaStreamDestroy(b.stream);
            b.done = nullptr;
            b.stream = nullptr;
            lk.lock();
            retired.push_back(b);
        }
        if (inflight.empty() && !retired.empty()) {
            lk.unlock();
            free_retired();
            lk.lock();
        }
        // 2. timeouts of queued requests
        if (opts.request_timeout_s > 0) {
            Clock::time_point now = Clock::now();
            for (auto it = queue.begin(); it != queue.end();) {
                Req &R = reqs[*it];
                double age = std::chrono::duration<double>(now - R.t_submit).count();
                if (R.state == PENDING && age > opts.request_timeout_s) {
                    R.state = FAILED;
                    R.status = QQMC_E_TIMEOUT;
                    R.out.status = QQMC_E_TIMEOUT;
                    it = queue.erase(it);
                } else {
                    ++it;
                }
            }
        }
        // 3. admission by device memory, FIFO
        std::vector<uint64_t> admit;
        int items = 0;
        while (!queue.empty()) {
            uint64_t h = queue.front();
            Req &R = reqs[h];
            if (R.state != PENDING) {
                queue.pop_front();
                continue;
            }
            if (bytes_in_use + R.bytes > opts.device_memory_limit && !(inflight.empty() && admit.empty())) break;
            if (items + R.r.n_max > opts.max_batch_items && !admit.empty()) break;
            bytes_in_use += R.bytes;
            R.state = ADMITTED;
            R.t_admit = Clock::now();
            R.out.queue_ms = std::chrono::duration<double, std::milli>(R.t_admit - R.t_submit).count();
            items += R.r.n_max;
            admit.push_back(h);
            queue.pop_front();
        }
        if (!admit.empty()) {
            std::vector<qqmc_request> rq;
            for (uint64_t h : admit) rq.push_back(reqs[h].r);
            Batch b;
            b.id = next_batch++;
            b.handles = admit;
            for (uint64_t h : admit) b.bytes += reqs[h].bytes;
            lk.unlock();
            int rc = QQMC_OK;
            std::vector<qqmc_item> its;
            for (size_t q = 0; q < rq.size() && rc == QQMC_OK; ++q) {
                qqmc_problem *pr = nullptr;
                rc = qqmc_create_problem(&rq[q].params, &pr);
                if (rc != QQMC_OK) break;
                b.problems.push_back(pr);
                for (int n = 1; n <= rq[q].n_max; ++n) {
                    qqmc_item it{};
                    it.problem = pr;
                    it.order = n;
                    it.n_shifts = rq[q].n_shifts;
                    it.n_points = rq[q].n_points;
                    its.push_back(it);
                }
            }
            if (rc == QQMC_OK) rc = qqmc_plan_create(its.data(), (int)its.size(), opts.precision, &b.plan);
            if (rc == QQMC_OK && cudaStreamCreateWithPriority(&b.stream, cudaStreamNonBlocking,
                                                              round_priority(rq)) != cudaSuccess)
                rc = set_error(QQMC_E_CUDA, "stream create");
            if (rc == QQMC_OK && cudaEventCreateWithFlags(&b.done, cudaEventDisableTiming) != cudaSuccess)
                rc = set_error(QQMC_E_CUDA, "event create");
            if (rc == QQMC_OK) rc = qqmc_plan_launch(b.plan, b.stream, opts.use_graph);
            if (rc == QQMC_OK && cudaEventRecord(b.done, b.stream) != cudaSuccess)
                rc = set_error(QQMC_E_CUDA, "event record");
            lk.lock();
            for (size_t q = 0; q < admit.size(); ++q) {
                Req &R = reqs[admit[q]];
                // order 0 from the problem's own tables: Q_0 = -2i g^<(0), I_0 = -4 Re gamma g^<_01(0)
                R.out.q[0] = q < b.problems.size()
                                 ? order0_value(*reinterpret_cast<const Problem *>(b.problems[q]))
                                 : 0.0;
                R.out.n_max = rq[q].n_max;
            }
            if (rc != QQMC_OK) {
                fail_batch(b, rc);
                bytes_in_use -= b.bytes;
                lk.unlock();
                qqmc_plan_destroy(b.plan);
                for (auto *p : b.problems) qqmc_destroy_problem(p);
                if (b.done) cudaEventDestroy(b.done);
                if (b.stream) cudaStreamDestroy(b.stream);
                lk.lock();
            } else {
                inflight.push_back(b);
            }
            cv.notify_all();
            continue;
        }
        if (stop && inflight.empty()) {
            lk.unlock();
            free_retired();
            lk.lock();
            break;
        }
        if (inflight.empty())
            cv.wait_for(lk, std::chrono::milliseconds(50));
        else
            cv.wait_for(lk, std::chrono::microseconds(200));
    }
}

extern "C" int qqmc_server_create(const qqmc_server_opts *opts, qqmc_server **out) {
    if (!out) return set_error(QQMC_E_INVAL, "out is NULL");
    *out = nullptr;
    qqmc_server *s = new (std::nothrow) qqmc_server();
    if (!s) return set_error(QQMC_E_NOMEM, "host allocation failed");
    if (opts) s->opts = *opts;
    if (s->opts.device_memory_limit == 0) s->opts.device_memory_limit = 4ull << 30;
    if (s->opts.max_queue <= 0) s->opts.max_queue = 4096;
    if (s->opts.max_batch_items <= 0) s->opts.max_batch_items = 256;
    if (s->opts.precision != QQMC_PREC_FP64 && s->opts.precision != QQMC_PREC_MIXED) {
        delete s;
        return set_error(QQMC_E_INVAL, "precision must be QQMC_PREC_FP64 or QQMC_PREC_MIXED");
    }
    if (cudaGetDevice(&s->device) != cudaSuccess) {
        delete s;
        return set_error(QQMC_E_CUDA, "no CUDA device");
    }
    s->worker = std::thread([s] { s->run(); });
    *out = s;
    return QQMC_OK;
}

extern "C" int qqmc_submit(qqmc_server *s, const qqmc_request *r, uint64_t *handle) {
    if (!s || !r || !handle) return set_error(QQMC_E_INVAL, "NULL argument");
    if (r->n_max < 1 || r->n_max > kMaxOrder) return set_error(QQMC_E_RANGE, "n_max outside 1..QQMC_MAX_ORDER");
    if (r->n_shifts < 2 || r->n_shifts > 1024) return set_error(QQMC_E_INVAL, "n_shifts must be in 2..1024");
    if (r->n_points < 1 || r->n_points > (1ull << QQMC_MAX_POINTS_LOG2))
        return set_error(QQMC_E_INVAL, "n_points must be in 1..2^30");
    std::string why;
    if (!valid_params(&r->params, why)) return set_error(QQMC_E_INVAL, "malformed request parameters: " + why);
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->stop) return set_error(QQMC_E_CANCELLED, "server is shutting down");
    if ((int)s->queue.size() >= s->opts.max_queue) return set_error(QQMC_E_BUSY, "request queue is full");
    Req R;
    R.handle = s->next_handle++;
    R.r = *r;
    R.t_submit = Clock::now();
    R.bytes = request_bytes(*r);
    R.out.n_max = r->n_max;
    R.out.status = QQMC_PENDING;
    s->reqs.emplace(R.handle, R);
    s->queue.push_back(R.handle);
    *handle = R.handle;
    s->cv.notify_all();
    return QQMC_OK;
}

extern "C" int qqmc_poll(qqmc_server *s, uint64_t handle, qqmc_series *out) {
    if (!s || !out) return set_error(QQMC_E_INVAL, "NULL argument");
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->reqs.find(handle);
    if (it == s->reqs.end()) return set_error(QQMC_E_NOTFOUND, "unknown handle");
    Req &R = it->second;
    if (R.state == PENDING || R.state == ADMITTED) return QQMC_PENDING;
    *out = R.out;
    int st = R.status;
    s->reqs.erase(it);
    return st;
}

extern "C" int qqmc_request_state(qqmc_server *s, uint64_t handle) {
    if (!s) return set_error(QQMC_E_INVAL, "NULL server");
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->reqs.find(handle);
    if (it == s->reqs.end()) return set_error(QQMC_E_NOTFOUND, "unknown handle");
    const Req &R = it->second;
    if (R.state == PENDING) return QQMC_PENDING;
    if (R.state == ADMITTED) return QQMC_RUNNING;
    return R.status;
}

extern "C" int qqmc_cancel(qqmc_server *s, uint64_t handle) {
    if (!s) return set_error(QQMC_E_INVAL, "NULL server");
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->reqs.find(handle);
    if (it == s->reqs.end()) return set_error(QQMC_E_NOTFOUND, "unknown handle");
    Req &R = it->second;
    if (R.state == PENDING || R.state == ADMITTED) {
        R.state = CANCELLED;
        R.status = QQMC_E_CANCELLED;
        R.out.status = QQMC_E_CANCELLED;
    }
    return QQMC_OK;
}

extern "C" int qqmc_server_destroy(qqmc_server *s) {
    if (!s) return QQMC_OK;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
        for (uint64_t h : s->queue) {
            Req &R = s->reqs[h];
            if (R.state == PENDING) {
                R.state = CANCELLED;
                R.status = QQMC_E_CANCELLED;
            }
        }
        s->queue.clear();
        s->cv.notify_all();
    }
    if (s->worker.joinable()) s->worker.join();
    delete s;
    return QQMC_OK;
}
