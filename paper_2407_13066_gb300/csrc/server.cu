// Serving loop: several resident operators, Hessian-action requests of
// 1..max_batch vectors, admission under a device-memory budget, and
// continuous batching per operator.  Host code (a scheduler thread); the
// work itself is btt_hessian_batched on one CUDA stream per operator.
//
// Life of a request
//   submit   -> inbox (caller thread), ticket returned at once
//   admit    -> the scheduler takes requests in arrival order; a request
//               whose vectors are in host memory needs device slots for
//               its input and output, carved from a fixed pool; the head of
//               the queue waits until the pool has room (no overtaking), its
//               input is copied on the upload stream as soon as it is
//               admitted
//   batch    -> whenever an operator's stream has finished its previous
//               batch, all its admitted requests (arrival order, whole
//               requests, at most max_batch vectors) form the next batch:
//               one Hessian call over their vectors, in place, through a
//               pointer table -- so requests that arrived while the
//               previous batch ran join the next one, and the operators'
//               batches overlap on the device
//   complete -> results of host requests are copied back on the download
//               stream; the request is done when that copy has finished,
//               its pool slots are freed, waiters are woken
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstdio>
#include <deque>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "../../include/btt.h"
#include "kernels.h"

#define BTT_API extern "C" __attribute__((visibility("default")))

namespace btt {
void set_last_error(const char* msg);
}

namespace {

double now_s()
{
    using namespace std::chrono;
    return duration<double>(steady_clock::now().time_since_epoch()).count();
}

bool is_device_ptr(const void* p)
{
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// First-fit allocator over byte offsets of one device buffer.
class Pool {
public:
    explicit Pool(size_t size) : size_(size) { if (size) free_[0] = size; }
    bool alloc(size_t n, size_t* off)
    {
        n = (n + 255) / 256 * 256;
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second >= n) {
                *off = it->first;
                const size_t rest = it->second - n;
                const size_t at = it->first + n;
                free_.erase(it);
                if (rest) free_[at] = rest;
                in_use_ += n;
                high_ = std::max(high_, in_use_);
                return true;
            }
        }
        return false;
    }
    void release(size_t off, size_t n)
    {
        n = (n + 255) / 256 * 256;
        in_use_ -= n;
        auto it = free_.emplace(off, n).first;
        auto nx = std::next(it);
        if (nx != free_.end() && it->first + it->second == nx->first) {
            it->second += nx->second;
            free_.erase(nx);
        }
        if (it != free_.begin()) {
            auto pv = std::prev(it);
            if (pv->first + pv->second == it->first) {
                pv->second += it->second;
                free_.erase(it);
            }
        }
    }
    size_t size() const { return size_; }
    size_t in_use() const { return in_use_; }
    size_t high() const { return high_; }

private:
    size_t size_, in_use_ = 0, high_ = 0;
    std::map<size_t, size_t> free_;
};

enum ReqState { R_WAITING = 0, R_ADMITTED = 1, R_RUNNING = 2, R_DONE = 3, R_FAILED = 4 };

struct Request {
    long long ticket = 0;
    int op = 0, nvec = 0;
    const float* m = nullptr;
    float* y = nullptr;
    bool m_host = false, y_host = false;
    size_t slot_off = 0, slot_bytes = 0;
    float* din = nullptr;
    float* dout = nullptr;
    cudaEvent_t uploaded = nullptr, done = nullptr;
    int state = R_WAITING;
    btt_status status = BTT_OK;
    double t_submit = 0, t_done = 0;
};

struct OpSlot {
    btt_op* op = nullptr;
    const float* gamma = nullptr;
    int N_t = 0, N_m = 0;
    cudaStream_t stream = nullptr;
    cudaEvent_t batch_done = nullptr;
    bool busy = false;
    std::deque<Request*> ready;
    std::vector<Request*> running;
};

}  // namespace

struct btt_server {
    int device = 0;
    int max_batch = 1;
    std::vector<OpSlot> ops;
    cudaStream_t upload = nullptr, download = nullptr;
    void* pool_base = nullptr;
    Pool pool{0};
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<Request*> inbox, waiting;
    std::map<long long, Request*> reqs;
    std::thread worker;
    bool stop = false;
    int waiters = 0;               // threads inside btt_server_wait
    int fault = 0;                 // injected host-side failure for the next batch / admission
    long long next_ticket = 1;
    // statistics (under mu)
    long long submitted = 0, completed = 0, failed = 0, vectors_done = 0, batches = 0, batch_vectors = 0;
    std::vector<double> lat_ms;
    double t_first = 0, t_last = 0;

    void run();
    void finish(Request* r, btt_status s);
};

void btt_server::finish(Request* r, btt_status s)
{
    // caller holds mu
    if (r->slot_bytes) pool.release(r->slot_off, r->slot_bytes);
    r->slot_bytes = 0;
    if (r->uploaded) cudaEventDestroy(r->uploaded);
    if (r->done) cudaEventDestroy(r->done);
    r->uploaded = r->done = nullptr;
    r->status = s;
    r->state = s == BTT_OK ? R_DONE : R_FAILED;
    r->t_done = now_s();
    if (s == BTT_OK) {
        ++completed;
        vectors_done += r->nvec;
        lat_ms.push_back((r->t_done - r->t_submit) * 1e3);
        t_last = r->t_done;
    } else {
        ++failed;
    }
}

void btt_server::run()
{
    cudaSetDevice(device);
    std::vector<const float*> in_tab;
    std::vector<float*> out_tab;
    for (;;) {
        bool progress = false;
        std::unique_lock<std::mutex> lk(mu);
        if (stop) break;
        while (!inbox.empty()) {
            waiting.push_back(inbox.front());
            inbox.pop_front();
            progress = true;
        }
        // ---- admission, in arrival order, under the pool budget
        while (!waiting.empty()) {
            Request* r = waiting.front();
            const size_t vbytes = (size_t)r->nvec * ops[r->op].N_t * ops[r->op].N_m * sizeof(float);
            const size_t need = (r->m_host ? vbytes : 0) + (r->y_host ? vbytes : 0);
            size_t off = 0;
            if (fault == 2) {
                fault = 0;
                waiting.pop_front();
                finish(r, BTT_ERR_OOM);
                cv_done.notify_all();
                progress = true;
                continue;
            }
            if (need && !pool.alloc(need, &off)) break;   // wait for memory
            waiting.pop_front();
            r->slot_off = off;
            r->slot_bytes = need;
            unsigned char* base = static_cast<unsigned char*>(pool_base) + off;
            r->din = r->m_host ? reinterpret_cast<float*>(base) : const_cast<float*>(r->m);
            r->dout = r->y_host ? reinterpret_cast<float*>(base + (r->m_host ? vbytes : 0)) : r->y;
            cudaError_t e = cudaSuccess;
            if (r->m_host) {
                e = cudaMemcpyAsync(r->din, r->m, vbytes, cudaMemcpyHostToDevice, upload);
                if (e == cudaSuccess) e = cudaEventCreateWithFlags(&r->uploaded, cudaEventDisableTiming);
                if (e == cudaSuccess) e = cudaEventRecord(r->uploaded, upload);
            }
            if (e != cudaSuccess) {
                finish(r, BTT_ERR_CUDA);
                cv_done.notify_all();
            } else {
                r->state = R_ADMITTED;
                ops[r->op].ready.push_back(r);
            }
            progress = true;
        }
        // ---- per operator: retire the finished batch, start the next one
        for (OpSlot& o : ops) {
            if (o.busy && cudaEventQuery(o.batch_done) == cudaSuccess) {
                o.busy = false;
                progress = true;
            }
            if (o.busy || o.ready.empty()) continue;
            std::vector<Request*> batch;
            int nb = 0;
            while (!o.ready.empty() && nb + o.ready.front()->nvec <= max_batch) {
                batch.push_back(o.ready.front());
                nb += o.ready.front()->nvec;
                o.ready.pop_front();
            }
            in_tab.clear();
            out_tab.clear();
            const size_t vstride = (size_t)o.N_t * o.N_m;
            for (Request* r : batch) {
                if (r->uploaded) cudaStreamWaitEvent(o.stream, r->uploaded, 0);
                for (int v = 0; v < r->nvec; ++v) {
                    in_tab.push_back(r->din + v * vstride);
                    out_tab.push_back(r->dout + v * vstride);
                }
                r->state = R_RUNNING;
            }
            btt_status s = BTT_OK;
            if (fault == 1) {
                fault = 0;
                s = BTT_ERR_CUDA;
                btt::set_last_error("injected batch failure");
            } else {
                s = btt_hessian_batched(o.op, in_tab.data(), o.gamma, out_tab.data(), nb, o.stream);
            }
            if (s != BTT_OK) {
                for (Request* r : batch) finish(r, s);
                cv_done.notify_all();
                progress = true;
                continue;
            }
            cudaEventRecord(o.batch_done, o.stream);
            ++batches;
            batch_vectors += nb;
            for (Request* r : batch) {
                cudaEventCreateWithFlags(&r->done, cudaEventDisableTiming);
                if (r->y_host) {
                    cudaStreamWaitEvent(download, o.batch_done, 0);
                    cudaMemcpyAsync(r->y, r->dout, (size_t)r->nvec * vstride * sizeof(float), cudaMemcpyDeviceToHost,
                                    download);
                    cudaEventRecord(r->done, download);
                } else {
                    cudaEventRecord(r->done, o.stream);
                }
                o.running.push_back(r);
            }
            o.busy = true;
            progress = true;
        }
        // ---- completions
        bool woke = false;
        for (OpSlot& o : ops) {
            for (size_t i = 0; i < o.running.size();) {
                Request* r = o.running[i];
                if (cudaEventQuery(r->done) == cudaSuccess) {
                    finish(r, BTT_OK);
                    o.running[i] = o.running.back();
                    o.running.pop_back();
                    woke = true;
                } else {
                    ++i;
                }
            }
        }
        if (woke) {
            cv_done.notify_all();
            progress = true;
        }
        if (!progress) cv_work.wait_for(lk, std::chrono::microseconds(20));
    }
}

BTT_API btt_status btt_server_create(btt_server** out, btt_op* const* ops, const float* const* gamma_inv, int n_ops,
                                     size_t pool_bytes, int max_batch)
{
    btt::set_last_error("");
    if (!out || !ops || n_ops < 1 || max_batch < 1) {
        btt::set_last_error("btt_server_create: bad arguments");
        return BTT_ERR_ARG;
    }
    *out = nullptr;
    btt_server* s = new btt_server;
    cudaGetDevice(&s->device);
    s->max_batch = max_batch;
    cudaError_t e = cudaSuccess;
    for (int i = 0; i < n_ops && e == cudaSuccess; ++i) {
        if (!ops[i]) {
            delete s;
            btt::set_last_error("btt_server_create: null operator");
            return BTT_ERR_ARG;
        }
        OpSlot o;
        o.op = ops[i];
        o.gamma = gamma_inv ? gamma_inv[i] : nullptr;
        btt_operator_shape(ops[i], &o.N_t, nullptr, &o.N_m);
        e = cudaStreamCreateWithFlags(&o.stream, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&o.batch_done, cudaEventDisableTiming);
        s->ops.push_back(o);
    }
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s->upload, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s->download, cudaStreamNonBlocking);
    if (e == cudaSuccess && pool_bytes) e = cudaMalloc(&s->pool_base, pool_bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        char buf[160];
        snprintf(buf, sizeof buf, "btt_server_create: %s", cudaGetErrorString(e));
        btt::set_last_error(buf);
        for (OpSlot& o : s->ops) {
            if (o.stream) cudaStreamDestroy(o.stream);
            if (o.batch_done) cudaEventDestroy(o.batch_done);
        }
        if (s->upload) cudaStreamDestroy(s->upload);
        if (s->download) cudaStreamDestroy(s->download);
        delete s;
        return e == cudaErrorMemoryAllocation ? BTT_ERR_OOM : BTT_ERR_CUDA;
    }
    s->pool = Pool(pool_bytes);
    s->worker = std::thread([s] { s->run(); });
    *out = s;
    return BTT_OK;
}

BTT_API btt_status btt_server_submit(btt_server* s, int op, const float* m, float* y, int nvec, long long* ticket)
{
    btt::set_last_error("");
    if (!s || !m || !y || !ticket || op < 0 || op >= (int)s->ops.size() || nvec < 1) {
        btt::set_last_error("btt_server_submit: bad arguments");
        return BTT_ERR_ARG;
    }
    if (nvec > s->max_batch) {
        btt::set_last_error("btt_server_submit: more vectors than the server's max_batch");
        return BTT_ERR_ARG;
    }
    Request* r = new Request;
    r->op = op;
    r->nvec = nvec;
    r->m = m;
    r->y = y;
    r->m_host = !is_device_ptr(m);
    r->y_host = !is_device_ptr(y);
    const size_t vbytes = (size_t)nvec * s->ops[op].N_t * s->ops[op].N_m * sizeof(float);
    const size_t need = (r->m_host ? vbytes : 0) + (r->y_host ? vbytes : 0);
    if ((need + 255) / 256 * 256 > s->pool.size()) {
        delete r;
        btt::set_last_error("btt_server_submit: request needs more device memory than the whole pool");
        return BTT_ERR_OOM;
    }
    {
        std::lock_guard<std::mutex> lk(s->mu);
        r->ticket = s->next_ticket++;
        r->t_submit = now_s();
        if (s->submitted == 0) s->t_first = r->t_submit;
        ++s->submitted;
        s->reqs[r->ticket] = r;
        s->inbox.push_back(r);
    }
    s->cv_work.notify_one();
    *ticket = r->ticket;
    return BTT_OK;
}

BTT_API btt_status btt_server_poll(btt_server* s, long long ticket, int* state)
{
    if (!s || !state) return BTT_ERR_ARG;
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end()) return BTT_ERR_ARG;
    *state = it->second->state;
    return BTT_OK;
}

BTT_API btt_status btt_server_wait(btt_server* s, long long ticket, double timeout_s)
{
    btt::set_last_error("");
    if (!s) return BTT_ERR_ARG;
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end()) {
        btt::set_last_error("btt_server_wait: unknown ticket");
        return BTT_ERR_ARG;
    }
    Request* r = it->second;
    ++s->waiters;
    const bool ok = s->cv_done.wait_for(lk, std::chrono::duration<double>(timeout_s < 0 ? 1e9 : timeout_s),
                                        [r] { return r->state == R_DONE || r->state == R_FAILED; });
    --s->waiters;
    s->cv_done.notify_all();
    if (!ok) {
        btt::set_last_error("btt_server_wait: timed out");
        return BTT_ERR_TIMEOUT;
    }
    const btt_status st = r->status;
    if (!s->stop) {
        s->reqs.erase(r->ticket);
        delete r;
    }
    if (st != BTT_OK) btt::set_last_error("btt_server_wait: the request failed");
    return st;
}

BTT_API btt_status btt_server_stats(btt_server* s, btt_serving_stats* out, int reset)
{
    if (!s || !out) return BTT_ERR_ARG;
    std::lock_guard<std::mutex> lk(s->mu);
    out->submitted = s->submitted;
    out->completed = s->completed;
    out->failed = s->failed;
    out->vectors_completed = s->vectors_done;
    out->batches = s->batches;
    out->mean_batch_vectors = s->batches ? (double)s->batch_vectors / s->batches : 0.0;
    std::vector<double> l = s->lat_ms;
    std::sort(l.begin(), l.end());
    auto q = [&l](double p) { return l.empty() ? 0.0 : l[std::min(l.size() - 1, (size_t)(p * (l.size() - 1) + 0.5))]; };
    out->latency_p50_ms = q(0.50);
    out->latency_p99_ms = q(0.99);
    double sum = 0;
    for (double v : l) sum += v;
    out->latency_mean_ms = l.empty() ? 0.0 : sum / l.size();
    out->span_s = s->t_last > s->t_first ? s->t_last - s->t_first : 0.0;
    out->pool_bytes = s->pool.size();
    out->pool_in_use = s->pool.in_use();
    out->pool_high_water = s->pool.high();
    long long w = (long long)s->waiting.size() + (long long)s->inbox.size(), a = 0, run = 0;
    for (const OpSlot& o : s->ops) {
        a += (long long)o.ready.size();
        run += (long long)o.running.size();
    }
    out->waiting = w;
    out->admitted = a;
    out->running = run;
    if (reset) {
        s->lat_ms.clear();
        s->submitted = s->completed = s->failed = s->vectors_done = s->batches = s->batch_vectors = 0;
        s->t_first = s->t_last = 0;
    }
    return BTT_OK;
}

BTT_API btt_status btt_server_inject(btt_server* s, int fault)
{
    if (!s || fault < 0 || fault > 2) return BTT_ERR_ARG;
    std::lock_guard<std::mutex> lk(s->mu);
    s->fault = fault;
    return BTT_OK;
}

BTT_API btt_status btt_server_destroy(btt_server* s)
{
    if (!s) return BTT_OK;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
    }
    s->cv_work.notify_all();
    if (s->worker.joinable()) s->worker.join();
    for (OpSlot& o : s->ops) cudaStreamSynchronize(o.stream);
    cudaStreamSynchronize(s->download);
    cudaStreamSynchronize(s->upload);
    {
        // requests not finished are failed; waiters are released before the
        // requests are freed
        std::unique_lock<std::mutex> lk(s->mu);
        for (auto& kv : s->reqs) {
            Request* r = kv.second;
            if (r->state != R_DONE && r->state != R_FAILED) {
                r->status = BTT_ERR_ARG;
                r->state = R_FAILED;
            }
        }
        s->cv_done.notify_all();
        s->cv_done.wait(lk, [s] { return s->waiters == 0; });
        for (auto& kv : s->reqs) {
            Request* r = kv.second;
            if (r->uploaded) cudaEventDestroy(r->uploaded);
            if (r->done) cudaEventDestroy(r->done);
            delete r;
        }
        s->reqs.clear();
    }
    for (OpSlot& o : s->ops) {
        cudaStreamDestroy(o.stream);
        cudaEventDestroy(o.batch_done);
    }
    cudaStreamDestroy(s->upload);
    cudaStreamDestroy(s->download);
    if (s->pool_base) cudaFree(s->pool_base);
    delete s;
    return BTT_OK;
}
