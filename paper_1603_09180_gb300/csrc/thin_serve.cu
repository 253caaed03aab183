// thin_serve.cu -- serving: continuous batching under a device-memory budget.
//
// A server owns eight worker lanes, each a host thread with its own CUDA
// streams.  submit copies the caller's image into a pinned host buffer and
// queues it.  An idle lane admits queued requests in arrival order while the
// slot count and the byte budget allow (at most its share of the slots),
// allocates their device images, copies them in and launches them as one
// batch.  Images that fit a thread-block cluster run on the resident engine,
// which posts a completion record for each image as soon as that image is
// finished; the lane then copies the image back on a second stream and
// retires the request at once, returning its bytes and slot while the rest
// of the batch still runs, so queued requests are admitted by the next idle
// lane as slots and memory free up.  Images too large for a cluster wait in
// a queue of their own; at most two lanes at a time run a batch of them on
// the tiled engine, each on at most a quarter of the SMs, and they retire
// when their batch ends.  So small requests keep flowing on the other SMs
// while large ones run.  (The tiled launch is cooperative: it starts only
// when all its blocks fit at once.  Capped at half of the SMs it waited for
// the long resident jobs to drain, and the small launches queued behind it;
// two quarter-size launches start sooner and keep the same share.)
// Lanes run side by side on the device (the resident engine gives each image
// its own cluster and takes only the SMs it needs).  Each image's result depends
// only on the image and its lambda: it is the same alone and in any mix.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "thin_internal.h"

namespace thin {
namespace {

constexpr int kLanes = 8;          // batches in flight at once
constexpr int kLargeLanes = 2;     // of which batches of large (tiled-engine) requests
constexpr int kMaxBatch = 512;     // requests one lane admits at a time

enum ReqState { kQueued, kRunning, kDone };

struct Req {
    uint64_t ticket;
    int w, h, dtype;
    uint32_t lam;
    size_t row;       // w * element size: the packed host row
    size_t dpitch;    // device pitch (16-byte multiple)
    size_t charge;    // bytes counted against the budget
    void *host;       // pinned: the input, then the result
    size_t host_cap;
    void *dev;
    int state;
    int rc;
    bool large;       // too large for one cluster's shared memory: the tiled engine
    thin_stats st;
};

// Pinned host staging: one arena allocated when the server is created,
// carved first-fit into 256-byte aligned blocks (neighbouring free blocks
// merge again).  submit never calls the CUDA allocator.
class PinnedArena {
public:
    ~PinnedArena()
    {
        if (base_) cudaFreeHost(base_);
    }
    cudaError_t init(size_t bytes)
    {
        bytes_ = (bytes + 255) / 256 * 256;
        const cudaError_t e = cudaHostAlloc(&base_, bytes_, cudaHostAllocPortable);
        if (e != cudaSuccess) {
            base_ = nullptr;
            return e;
        }
        free_[0] = bytes_;
        return cudaSuccess;
    }
    size_t size() const { return bytes_; }
    void *get(size_t n, size_t *cap)
    {
        n = std::max<size_t>(256, (n + 255) / 256 * 256);
        std::lock_guard<std::mutex> g(mu_);
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second < n) continue;
            const size_t off = it->first, len = it->second;
            free_.erase(it);
            if (len > n) free_[off + n] = len - n;
            *cap = n;
            return static_cast<char *>(base_) + off;
        }
        return nullptr;
    }
    void put(void *p, size_t cap)
    {
        if (!p) return;
        std::lock_guard<std::mutex> g(mu_);
        size_t off = static_cast<size_t>(static_cast<char *>(p) - static_cast<char *>(base_)), len = cap;
        auto next = free_.lower_bound(off);
        if (next != free_.end() && next->first == off + len) {  // merge with the block after
            len += next->second;
            next = free_.erase(next);
        }
        if (next != free_.begin()) {  // and with the block before
            auto prev = std::prev(next);
            if (prev->first + prev->second == off) {
                prev->second += len;
                return;
            }
        }
        free_[off] = len;
    }

private:
    void *base_ = nullptr;
    size_t bytes_ = 0;
    std::mutex mu_;
    std::map<size_t, size_t> free_;  // offset -> length
};

}  // namespace
}  // namespace thin

struct thin_server {
    size_t budget = 0;
    int max_slots = 0, queue_cap = 0;
    int device = 0;
    std::mutex mu;
    std::condition_variable cv;
    std::deque<thin::Req *> queue;        // requests that fit a cluster (the resident engine)
    std::deque<thin::Req *> queue_large;  // the rest (the tiled engine)
    int large_running = 0;                // lanes running a batch of large requests (kLargeLanes at most)
    size_t res_smem_limit = 0;            // a resident block's shared memory (one block per SM)
    std::unordered_map<uint64_t, thin::Req *> reqs;
    std::deque<uint64_t> finished;  // tickets in the order they finished, for thin_serve_wait_any
    size_t used = 0;   // bytes charged by admitted requests
    int in_flight = 0;
    bool stop = false;
    uint64_t next_ticket = 1;
    std::vector<std::thread> lanes;
    thin::PinnedArena pool;
};

namespace thin {
namespace {

size_t charge_of(int w, int h, int dtype, size_t *dpitch)
{
    const size_t row = size_t(w) * elem_size(dtype);
    *dpitch = (row + 15) / 16 * 16;
    const size_t img = *dpitch * size_t(h);
    // the image itself, plus the tiled engine's scratch for images too large
    // for one cluster (a second buffer and 4 bytes per 8 x 2 cell), plus job
    // tables
    return img + img + size_t(w) * h / 4 + (64 << 10);
}

// Ends a request: its result is in r->host (or r->rc holds its error);
// returns its bytes and slot and posts it to the completion queue.  A client
// may poll and free the request as soon as this returns: the caller must not
// touch r afterwards.
void retire(thin_server *S, Req *r)
{
    {
        std::lock_guard<std::mutex> g(S->mu);
        r->dev = nullptr;
        r->state = kDone;
        S->used -= r->charge;
        --S->in_flight;
        S->finished.push_back(r->ticket);
        // callers that only poll never drain the list: keep it bounded
        const size_t cap = 4 * size_t(S->max_slots + S->queue_cap);
        while (S->finished.size() > cap) S->finished.pop_front();
    }
    S->cv.notify_all();
}

void lane_main(thin_server *S)
{
    cudaSetDevice(S->device);
    cudaStream_t stream = nullptr, copy = nullptr;
    ResDone *done_host = nullptr, *done_dev = nullptr;
    std::vector<cudaEvent_t> copied(kMaxBatch, nullptr);
    bool ok_lane = cudaStreamCreateWithFlags(&stream, cudaStreamNonBlocking) == cudaSuccess &&
                   cudaStreamCreateWithFlags(&copy, cudaStreamNonBlocking) == cudaSuccess &&
                   cudaHostAlloc(reinterpret_cast<void **>(&done_host), sizeof(ResDone) * kMaxBatch,
                                 cudaHostAllocMapped | cudaHostAllocPortable) == cudaSuccess &&
                   cudaHostGetDevicePointer(reinterpret_cast<void **>(&done_dev), done_host, 0) == cudaSuccess;
    for (auto &e : copied)
        if (ok_lane) ok_lane = cudaEventCreateWithFlags(&e, cudaEventDisableTiming) == cudaSuccess;
    if (!ok_lane) cudaGetLastError();
    cudaStream_t *side = nullptr;
    cudaEvent_t *side_ev = nullptr;
    if (ok_lane && thread_side_streams(&side, &side_ev) != cudaSuccess) {
        cudaGetLastError();
        ok_lane = false;
    }
    // a large batch's tiled launch takes at most a quarter of the SMs (two may run), so that
    // the resident launches of the other lanes keep running beside them
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, S->device);
    const int tiled_cap = std::max(1, sms / (2 * kLargeLanes));
    std::vector<Req *> batch;
    for (;;) {
        batch.clear();
        bool large = false;
        {
            std::unique_lock<std::mutex> g(S->mu);
            // wait for work that fits, or for the stop signal; large requests run one batch at a time
            auto fits = [&](const std::deque<Req *> &q) {
                return !q.empty() && S->used + q.front()->charge <= S->budget;
            };
            S->cv.wait(g, [&] {
                if (S->stop) return true;
                if (S->in_flight >= S->max_slots) return false;
                return fits(S->queue) || (S->large_running < kLargeLanes && fits(S->queue_large));
            });
            if (S->stop) break;
            large = S->large_running < kLargeLanes && fits(S->queue_large);
            if (large) ++S->large_running;
            std::deque<Req *> &q = large ? S->queue_large : S->queue;
            // a lane takes at most its share of the slots, so that under load the other lanes
            // keep admitting while this lane's batch runs
            const int share = std::max(1, std::min(kMaxBatch, S->max_slots / kLanes));
            while (!q.empty() && S->in_flight < S->max_slots && int(batch.size()) < share) {
                Req *r = q.front();
                if (S->used + r->charge > S->budget) break;
                q.pop_front();
                S->used += r->charge;
                ++S->in_flight;
                r->state = kRunning;
                batch.push_back(r);
            }
            if (batch.empty() && large) --S->large_running;
        }
        if (batch.empty()) continue;
        NvtxRange nv("thin_serve batch");
        // device images and input copies
        std::vector<JobSpec> jobs;
        std::vector<Req *> run;
        std::vector<char> in_run(batch.size(), 0);
        for (size_t i = 0; i < batch.size(); ++i) {
            Req *r = batch[i];
            r->rc = THIN_OK;
            r->dev = nullptr;
            cudaError_t e = ok_lane ? cudaMallocAsync(&r->dev, r->dpitch * r->h, stream) : cudaErrorInvalidResourceHandle;
            if (e == cudaSuccess)
                e = cudaMemcpy2DAsync(r->dev, r->dpitch, r->host, r->row, r->row, r->h, cudaMemcpyHostToDevice, stream);
            if (e != cudaSuccess) {
                cudaGetLastError();
                r->rc = cuda_status(e);
                continue;
            }
            JobSpec j{r->dev, r->w, r->h, r->dpitch, r->dtype, r->lam, THIN_ADJ_8_4};
            j.done_slot = int(run.size());
            jobs.push_back(j);
            run.push_back(r);
            in_run[i] = 1;
        }
        const int n = int(run.size());
        // 0: running, 1: result copy in flight, 2: retired
        std::vector<int> phase(n, 0);
        int retired = 0;
        int rc = THIN_OK;
        thin_options o;
        thin_default_options(&o);
        Grouping G;
        Execution X;
        X.done = done_dev;
        X.tiled_max_grid = tiled_cap;
        bool launched = false;
        if (n > 0) {
            for (int k = 0; k < n; ++k) done_host[k].flag = 0u;
            // the lanes share the GPU: no wide launch (it would hold every SM for one image)
            rc = group_jobs(jobs, o, &G, false);
            if (rc == THIN_OK) rc = X.prepare(jobs, G, o, stream, true);
            if (rc == THIN_OK) {
                const cudaError_t e = X.enqueue(stream, side, side_ev);
                if (e != cudaSuccess) rc = cuda_status(e);
                else launched = true;
            }
        }
        // retire each resident image as its completion record appears; the rest when the stream is done
        auto start_copy = [&](int k) {
            Req *r = run[k];
            const cudaError_t e =
                cudaMemcpy2DAsync(r->host, r->row, r->dev, r->dpitch, r->row, r->h, cudaMemcpyDeviceToHost, copy);
            if (e == cudaSuccess) cudaEventRecord(copied[k], copy);
            else if (r->rc == THIN_OK) r->rc = cuda_status(e);
            phase[k] = 1;
        };
        auto finish_copy = [&](int k, bool wait) {
            if (wait) cudaEventSynchronize(copied[k]);
            else if (cudaEventQuery(copied[k]) != cudaSuccess) return false;
            Req *r = run[k];
            cudaFreeAsync(r->dev, copy);
            phase[k] = 2;
            ++retired;
            retire(S, r);
            return true;
        };
        while (launched && retired < n) {
            bool progress = false;
            for (int k = 0; k < n; ++k) {
                if (phase[k] == 0 && __atomic_load_n(&done_host[k].flag, __ATOMIC_ACQUIRE) == 1u) {
                    resident_stats(done_host[k].st, done_host[k].error, o, &run[k]->st);
                    if (run[k]->st.status != THIN_OK) run[k]->rc = run[k]->st.status;
                    start_copy(k);
                    progress = true;
                }
                if (phase[k] == 1) progress |= finish_copy(k, false);
            }
            if (progress) continue;
            if (cudaStreamQuery(stream) != cudaErrorNotReady) break;  // the batch is over (or failed)
            std::this_thread::sleep_for(std::chrono::microseconds(20));
        }
        // what is left: tiled images, and any image the batch ended without posting
        if (n > 0) {
            std::vector<thin_stats> st(n);
            if (launched) {
                const int crc = X.collect(stream, st.data());  // waits for the stream
                if (rc == THIN_OK && crc != THIN_OK && crc != THIN_ERR_NOT_CONVERGED) rc = crc;
            } else if (stream) {
                cudaStreamSynchronize(stream);  // the input copies are done before the copy stream reads back
            }
            for (int k = 0; k < n; ++k) {
                if (phase[k] != 0) continue;
                Req *r = run[k];
                r->st = st[k];
                if (r->st.status != THIN_OK) r->rc = r->st.status;
                else if (rc != THIN_OK) r->rc = rc;
                start_copy(k);
            }
            for (int k = 0; k < n; ++k)
                if (phase[k] == 1) finish_copy(k, true);
        }
        X.release(stream);
        const cudaError_t e = stream ? cudaStreamSynchronize(stream) : cudaSuccess;
        if (e != cudaSuccess) cudaGetLastError();
        for (size_t i = 0; i < batch.size(); ++i) {  // requests whose device image could not be set up
            if (in_run[i]) continue;  // retired above (and perhaps already freed by a poll)
            Req *r = batch[i];
            if (r->dev) cudaFreeAsync(r->dev, stream);
            retire(S, r);
        }
        if (large) {
            {
                std::lock_guard<std::mutex> g(S->mu);
                --S->large_running;
            }
            S->cv.notify_all();
        }
    }
    if (copy) cudaStreamSynchronize(copy);
    for (auto e : copied)
        if (e) cudaEventDestroy(e);
    if (done_host) cudaFreeHost(done_host);
    if (copy) cudaStreamDestroy(copy);
    if (stream) cudaStreamDestroy(stream);
}

}  // namespace
}  // namespace thin

using namespace thin;

extern "C" {

int thin_serve_create(size_t device_budget_bytes, int max_slots, int queue_cap, thin_server **out)
{
    if (!out) return THIN_ERR_ARG;
    *out = nullptr;
    if (device_budget_bytes == 0 || max_slots <= 0 || queue_cap <= 0) return THIN_ERR_ARG;
    thin_server *S = new thin_server;
    S->budget = device_budget_bytes;
    S->max_slots = max_slots;
    S->queue_cap = queue_cap;
    if (cudaGetDevice(&S->device) != cudaSuccess) {
        cudaGetLastError();
        delete S;
        return THIN_ERR_CUDA;
    }
    S->res_smem_limit = resident_smem_limit(1);
    // host staging for waiting and running requests: a quarter of the device
    // budget, between 256 MiB and 4 GiB
    const size_t host = std::min<size_t>(std::max<size_t>(device_budget_bytes / 4, size_t(256) << 20), size_t(4) << 30);
    if (S->pool.init(host) != cudaSuccess) {
        cudaGetLastError();
        delete S;
        return THIN_ERR_OOM;
    }
    for (int k = 0; k < kLanes; ++k) S->lanes.emplace_back(lane_main, S);
    *out = S;
    return THIN_OK;
}

int thin_serve_submit(thin_server *S, const void *host_img, int w, int h, size_t pitch, thin_dtype dt,
                      uint32_t lambda, uint64_t *ticket)
{
    if (!S || !ticket || w < 0 || h < 0 || (dt != THIN_U8 && dt != THIN_U16)) return THIN_ERR_ARG;
    const size_t row = size_t(w) * elem_size(dt);
    if ((w > 0 && h > 0) && (!host_img || pitch < row)) return THIN_ERR_ARG;
    Req *r = new Req;
    std::memset(r, 0, sizeof *r);
    r->w = w;
    r->h = h;
    r->dtype = dt;
    r->lam = lambda;
    r->row = row;
    r->charge = charge_of(w, h, dt, &r->dpitch);
    if (r->charge > S->budget) {
        delete r;
        return THIN_ERR_TOO_LARGE;  // could never be admitted
    }
    {
        std::lock_guard<std::mutex> g(S->mu);
        if (S->stop) {
            delete r;
            return THIN_ERR_ARG;
        }
        if (int(S->queue.size() + S->queue_large.size()) >= S->queue_cap) {
            delete r;
            return THIN_EAGAIN;
        }
    }
    r->large = resident_cluster_size(w, h, dt, S->res_smem_limit, 16, nullptr, nullptr) == 0;
    if (row * h > S->pool.size()) {
        delete r;
        return THIN_ERR_TOO_LARGE;  // could never be staged
    }
    r->host = S->pool.get(std::max<size_t>(row * h, 1), &r->host_cap);
    if (!r->host) {  // staging full: the waiting and running requests hold it all
        delete r;
        return THIN_EAGAIN;
    }
    for (int y = 0; y < h; ++y)
        std::memcpy(static_cast<char *>(r->host) + size_t(y) * row, static_cast<const char *>(host_img) + size_t(y) * pitch,
                    row);
    {
        std::lock_guard<std::mutex> g(S->mu);
        if (int(S->queue.size() + S->queue_large.size()) >= S->queue_cap) {
            S->pool.put(r->host, r->host_cap);
            delete r;
            return THIN_EAGAIN;
        }
        r->ticket = S->next_ticket++;
        *ticket = r->ticket;
        if (w < 3 || h < 3) {  // no interior point: finished as it is
            r->state = kDone;
            r->st.converged = 1;
            r->st.last_change_phase = -1;
            S->finished.push_back(r->ticket);
        } else {
            r->state = kQueued;
            (r->large ? S->queue_large : S->queue).push_back(r);
        }
        S->reqs[r->ticket] = r;
    }
    S->cv.notify_all();
    return THIN_OK;
}

int thin_serve_poll(thin_server *S, uint64_t ticket, void *host_out, size_t out_pitch, int *done, thin_stats *stats)
{
    if (!S || !done) return THIN_ERR_ARG;
    *done = 0;
    Req *r = nullptr;
    {
        std::lock_guard<std::mutex> g(S->mu);
        auto it = S->reqs.find(ticket);
        if (it == S->reqs.end()) return THIN_ERR_ARG;
        if (it->second->state != kDone) return THIN_OK;
        r = it->second;
        if (r->w > 0 && r->h > 0 && (!host_out || out_pitch < r->row)) return THIN_ERR_ARG;
        S->reqs.erase(it);
    }
    for (int y = 0; y < r->h; ++y)
        std::memcpy(static_cast<char *>(host_out) + size_t(y) * out_pitch, static_cast<const char *>(r->host) + size_t(y) * r->row,
                    r->row);
    if (stats) *stats = r->st;
    const int rc = r->rc;
    S->pool.put(r->host, r->host_cap);
    delete r;
    *done = 1;
    return rc;
}

int thin_serve_wait_any(thin_server *S, int timeout_ms, uint64_t *ticket)
{
    if (!S || !ticket) return THIN_ERR_ARG;
    std::unique_lock<std::mutex> g(S->mu);
    const auto until = std::chrono::steady_clock::now() + std::chrono::milliseconds(std::max(0, timeout_ms));
    for (;;) {
        while (!S->finished.empty()) {
            const uint64_t t = S->finished.front();
            S->finished.pop_front();
            if (S->reqs.count(t)) {  // not yet retired by a poll
                *ticket = t;
                return THIN_OK;
            }
        }
        if (S->stop) return THIN_EAGAIN;
        if (S->cv.wait_until(g, until) == std::cv_status::timeout && S->finished.empty()) return THIN_EAGAIN;
    }
}

int thin_serve_destroy(thin_server *S)
{
    if (!S) return THIN_ERR_ARG;
    {
        std::lock_guard<std::mutex> g(S->mu);
        S->stop = true;
    }
    S->cv.notify_all();
    for (auto &t : S->lanes) t.join();  // a lane finishes the batch it admitted before it stops
    for (auto &kv : S->reqs) {
        S->pool.put(kv.second->host, kv.second->host_cap);
        delete kv.second;
    }
    delete S;
    return THIN_OK;
}

}  // extern "C"
