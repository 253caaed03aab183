// thin_serve.cu -- serving: continuous batching under a device-memory budget.
//
// A server owns a few worker lanes, each a host thread with its own CUDA
// stream.  submit copies the caller's image into a pinned host buffer and
// queues it.  An idle lane admits queued requests in arrival order while the
// slot count and the byte budget allow, allocates their device images, copies
// them in, thins them all with one thin_batch call, copies the results back
// and retires them, returning their bytes and slots at once.  Requests that
// arrive while a lane is busy are admitted by the next idle lane, so their
// work runs on the device next to the batches already there (the resident
// engine gives each image its own thread-block cluster and takes only the
// SMs it needs).  Each image's result depends only on the image and its
// lambda: it is the same alone and in any mix.
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

constexpr int kLanes = 4;          // batches in flight at once
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
    std::deque<thin::Req *> queue;
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

void lane_main(thin_server *S)
{
    cudaSetDevice(S->device);
    cudaStream_t stream = nullptr;
    if (cudaStreamCreateWithFlags(&stream, cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        stream = nullptr;
    }
    std::vector<Req *> batch;
    std::vector<thin_stats> st;
    for (;;) {
        batch.clear();
        {
            std::unique_lock<std::mutex> g(S->mu);
            // wait for work that fits, or for the stop signal
            S->cv.wait(g, [&] {
                if (S->stop) return true;
                if (S->queue.empty() || S->in_flight >= S->max_slots) return false;
                return S->used + S->queue.front()->charge <= S->budget;
            });
            if (S->stop) break;
            // a lane takes at most its share of the slots, so that under load the other lanes
            // keep admitting while one lane's batch waits for its slowest image
            const int share = std::max(1, std::min(kMaxBatch, S->max_slots / kLanes));
            while (!S->queue.empty() && S->in_flight < S->max_slots && int(batch.size()) < share) {
                Req *r = S->queue.front();
                if (S->used + r->charge > S->budget) break;
                S->queue.pop_front();
                S->used += r->charge;
                ++S->in_flight;
                r->state = kRunning;
                batch.push_back(r);
            }
        }
        if (batch.empty()) continue;
        NvtxRange nv("thin_serve batch");
        // device slots, input copies, one batch, result copies
        std::vector<JobSpec> jobs;
        std::vector<Req *> ok;
        for (Req *r : batch) {
            r->rc = THIN_OK;
            r->dev = nullptr;
            cudaError_t e = stream ? cudaMallocAsync(&r->dev, r->dpitch * r->h, stream) : cudaErrorInvalidResourceHandle;
            if (e == cudaSuccess)
                e = cudaMemcpy2DAsync(r->dev, r->dpitch, r->host, r->row, r->row, r->h, cudaMemcpyHostToDevice, stream);
            if (e != cudaSuccess) {
                r->rc = cuda_status(e);
                continue;
            }
            jobs.push_back(JobSpec{r->dev, r->w, r->h, r->dpitch, r->dtype, r->lam, THIN_ADJ_8_4});
            ok.push_back(r);
        }
        st.assign(ok.size(), thin_stats{});
        int rc = THIN_OK;
        if (!ok.empty()) {
            // the lanes share the GPU: no wide launch (it would hold every SM for one image)
            thin_options o;
            thin_default_options(&o);
            rc = batch_validated(jobs, o, stream, st.data(), false);
        }
        for (size_t k = 0; k < ok.size(); ++k) {
            Req *r = ok[k];
            r->st = st[k];
            if (r->st.status != THIN_OK) r->rc = r->st.status;
            else if (rc != THIN_OK && rc != THIN_ERR_NOT_CONVERGED) r->rc = rc;
            const cudaError_t e =
                cudaMemcpy2DAsync(r->host, r->row, r->dev, r->dpitch, r->row, r->h, cudaMemcpyDeviceToHost, stream);
            if (e != cudaSuccess && r->rc == THIN_OK) r->rc = cuda_status(e);
        }
        for (Req *r : batch)
            if (r->dev) cudaFreeAsync(r->dev, stream);
        const cudaError_t e = stream ? cudaStreamSynchronize(stream) : cudaSuccess;
        {
            std::lock_guard<std::mutex> g(S->mu);
            for (Req *r : batch) {
                if (e != cudaSuccess && r->rc == THIN_OK) r->rc = cuda_status(e);
                r->dev = nullptr;
                r->state = kDone;
                S->used -= r->charge;
                --S->in_flight;
                S->finished.push_back(r->ticket);
            }
            // callers that only poll never drain the list: keep it bounded
            const size_t cap = 4 * size_t(S->max_slots + S->queue_cap);
            while (S->finished.size() > cap) S->finished.pop_front();
        }
        S->cv.notify_all();
    }
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
        if (int(S->queue.size()) >= S->queue_cap) {
            delete r;
            return THIN_EAGAIN;
        }
    }
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
        if (int(S->queue.size()) >= S->queue_cap) {
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
            S->queue.push_back(r);
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
