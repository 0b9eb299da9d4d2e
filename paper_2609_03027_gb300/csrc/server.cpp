// Streaming server: continuous batching of voltage blocks from several stations
// (each with its own plan) onto one GPU.  The server owns one device pool,
// carved first-fit into per-block ranges, and a set of slots (CUDA streams),
// each with its own call memory (grid / tile scratch, split bookkeeping and a
// bounded-wait flag, sized for the largest plan it has run).  A submitted block
// waits in a queue until a slot is free, pool memory for it is free and no
// earlier block with the same output images is queued or running (blocks that
// accumulate into one set of images run in submission order); then its host
// block is copied into its range and imaged on the slot's stream with the slot's
// call memory.  Blocks therefore overlap on the device, those of one plan
// included.  Images stay on the device in caller-owned accumulators
// (EPIC_ACCUMULATE continues an integration).  The latency of a block is the
// wall time from submission to the completion of its kernels, taken in a
// stream host callback, which also reads the slot's bounded-wait flag (copied
// to pinned host memory behind the block's kernels) into the block's status.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <new>
#include <thread>
#include <vector>

#include "epic_internal.h"

namespace {

using Clock = std::chrono::steady_clock;
constexpr size_t kAlign = 256;

struct Job {
    uint64_t ticket = 0;
    int waiters = 0;                // threads inside epic_server_wait for this ticket
    bool released = false;          // collected by a waiter: no longer in the ticket map
    epic_plan_t plan = nullptr;
    int T = 0;
    float* out = nullptr;
    unsigned flags = 0;
    const uint8_t* host = nullptr;  // caller's block: valid until the ticket completes
    size_t bytes = 0;
    size_t off = 0;                 // range in the device pool
    Clock::time_point submitted;
    int slot = -1;
    double latency_ms = -1.0;
    epic_status status = EPIC_OK;
    bool done = false;
};

struct Callback {
    epic_server_s* srv;
    int slot;
};

}  // namespace

struct epic_server_s {
    int device = 0;
    uint8_t* pool = nullptr;
    size_t pool_bytes = 0;
    std::vector<std::pair<size_t, size_t>> ranges;  // allocated [off, off+len), sorted by off
    std::vector<cudaStream_t> streams;
    std::vector<Job*> slot_job;
    std::vector<Callback> callbacks;
    std::vector<epic::CallScratch> slot_mem;  // call memory of each slot
    int* slot_flag = nullptr;                 // pinned host copies of the slots' bounded-wait flags
    std::mutex mu;
    std::condition_variable cv;       // dispatcher wake-up
    std::condition_variable done_cv;  // ticket waiters
    std::deque<Job*> pending;
    std::map<uint64_t, Job*> jobs;
    std::vector<float*> busy_outs;    // output images of the blocks on the device
    std::vector<double> latencies;
    size_t queue_limit = 0;
    uint64_t next_ticket = 1;
    bool stop = false;
    std::thread worker;
};

namespace {

size_t round_up(size_t v) { return (v + kAlign - 1) / kAlign * kAlign; }

// first-fit range of `len` bytes in the pool (caller holds the lock)
bool pool_alloc(epic_server_s* s, size_t len, size_t* off)
{
    len = round_up(std::max<size_t>(len, 1));
    size_t cur = 0;
    for (size_t i = 0; i <= s->ranges.size(); ++i) {
        const size_t end = i < s->ranges.size() ? s->ranges[i].first : s->pool_bytes;
        if (end >= cur && end - cur >= len) {
            s->ranges.insert(s->ranges.begin() + i, {cur, len});
            *off = cur;
            return true;
        }
        if (i < s->ranges.size()) cur = s->ranges[i].first + s->ranges[i].second;
    }
    return false;
}

void pool_free(epic_server_s* s, size_t off)
{
    for (size_t i = 0; i < s->ranges.size(); ++i)
        if (s->ranges[i].first == off) {
            s->ranges.erase(s->ranges.begin() + i);
            return;
        }
}

bool out_busy(epic_server_s* s, float* out)
{
    return std::find(s->busy_outs.begin(), s->busy_outs.end(), out) != s->busy_outs.end();
}

// Host callback after a block's kernels: bookkeeping only (no CUDA calls allowed here).
void CUDART_CB on_complete(void* arg)
{
    Callback* cb = static_cast<Callback*>(arg);
    epic_server_s* s = cb->srv;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        Job* j = s->slot_job[cb->slot];
        if (j) {
            j->latency_ms = std::chrono::duration<double, std::milli>(Clock::now() - j->submitted).count();
            if (s->slot_flag[cb->slot]) j->status = EPIC_ERR_TIMEOUT;  // a bounded device wait ran out
            j->done = true;
            s->latencies.push_back(j->latency_ms);
            pool_free(s, j->off);
            s->busy_outs.erase(std::find(s->busy_outs.begin(), s->busy_outs.end(), j->out));
            s->slot_job[cb->slot] = nullptr;
        }
    }
    s->cv.notify_all();
    s->done_cv.notify_all();
}

// Pick the first startable job (FIFO per output), reserve its slot, range and output.
Job* select_locked(epic_server_s* s)
{
    std::vector<float*> seen;
    for (auto it = s->pending.begin(); it != s->pending.end(); ++it) {
        Job* j = *it;
        const bool first_of_out = std::find(seen.begin(), seen.end(), j->out) == seen.end();
        seen.push_back(j->out);
        if (!first_of_out || out_busy(s, j->out)) continue;
        int slot = -1;
        for (size_t k = 0; k < s->slot_job.size(); ++k)
            if (!s->slot_job[k]) {
                slot = (int)k;
                break;
            }
        if (slot < 0) return nullptr;
        size_t off = 0;
        if (!pool_alloc(s, j->bytes, &off)) continue;  // memory: try a smaller block of another plan
        j->off = off;
        j->slot = slot;
        s->slot_job[slot] = j;
        s->busy_outs.push_back(j->out);
        s->pending.erase(it);
        return j;
    }
    return nullptr;
}

void worker_loop(epic_server_s* s)
{
    cudaSetDevice(s->device);
    std::unique_lock<std::mutex> lk(s->mu);
    while (!s->stop) {
        Job* j = select_locked(s);
        if (!j) {
            s->cv.wait_for(lk, std::chrono::milliseconds(20));
            continue;
        }
        lk.unlock();
        const int slot = j->slot;
        cudaStream_t st = s->streams[slot];
        uint8_t* dev = s->pool + j->off;
        epic::CallScratch& mem = s->slot_mem[slot];
        // the slot's call memory grows to the plan's needs (the slot's previous block is done)
        epic_status status = epic::call_scratch_fit(j->plan, mem);
        cudaError_t e = cudaSuccess;
        if (status == EPIC_OK) e = cudaMemsetAsync(mem.status, 0, sizeof(int), st);
        if (e == cudaSuccess && j->bytes) e = cudaMemcpyAsync(dev, j->host, j->bytes, cudaMemcpyHostToDevice, st);
        if (e != cudaSuccess) status = EPIC_ERR_CUDA;
        if (status == EPIC_OK) {
            if (j->T > 0) status = epic::image_run_with(j->plan, mem, dev, j->T, st, j->out, j->flags);
            else status = epic_image(j->plan, dev, 0, st, j->out, j->flags);
        }
        if (status == EPIC_OK) {
            e = cudaMemcpyAsync(&s->slot_flag[slot], mem.status, sizeof(int), cudaMemcpyDeviceToHost, st);
            if (e != cudaSuccess) status = EPIC_ERR_CUDA;
        }
        if (status == EPIC_OK) {
            e = cudaLaunchHostFunc(st, on_complete, &s->callbacks[slot]);
            if (e != cudaSuccess) {
                cudaStreamSynchronize(st);
                on_complete(&s->callbacks[slot]);
            }
            lk.lock();
        } else {
            cudaStreamSynchronize(st);  // nothing of this block may still use its range
            lk.lock();
            j->status = status;
            j->done = true;
            j->latency_ms = std::chrono::duration<double, std::milli>(Clock::now() - j->submitted).count();
            pool_free(s, j->off);
            s->busy_outs.erase(std::find(s->busy_outs.begin(), s->busy_outs.end(), j->out));
            s->slot_job[slot] = nullptr;
            s->done_cv.notify_all();
        }
    }
}

}  // namespace

extern "C" {

epic_status epic_server_create(size_t max_device_bytes, int max_slots, epic_server_t* out)
{
    if (!out) return EPIC_ERR_INVALID_ARG;
    *out = nullptr;
    if (max_slots < 1 || max_slots > 64 || max_device_bytes < kAlign) return EPIC_ERR_INVALID_ARG;
    epic_server_s* s = new (std::nothrow) epic_server_s();
    if (!s) return EPIC_ERR_OOM;
    if (cudaGetDevice(&s->device) != cudaSuccess) {
        delete s;
        return EPIC_ERR_CUDA;
    }
    s->pool_bytes = round_up(max_device_bytes);
    if (cudaMalloc(&s->pool, s->pool_bytes) != cudaSuccess) {
        cudaGetLastError();
        delete s;
        return EPIC_ERR_OOM;
    }
    s->streams.assign(max_slots, nullptr);
    s->slot_job.assign(max_slots, nullptr);
    s->callbacks.resize(max_slots);
    s->slot_mem.resize(max_slots);
    if (cudaMallocHost(&s->slot_flag, sizeof(int) * max_slots) != cudaSuccess) {
        cudaGetLastError();
        cudaFree(s->pool);
        delete s;
        return EPIC_ERR_OOM;
    }
    for (int k = 0; k < max_slots; ++k) s->slot_flag[k] = 0;
    for (int k = 0; k < max_slots; ++k) {
        s->callbacks[k] = Callback{s, k};
        if (cudaStreamCreateWithFlags(&s->streams[k], cudaStreamNonBlocking) != cudaSuccess) {
            for (auto st : s->streams)
                if (st) cudaStreamDestroy(st);
            cudaFree(s->pool);
            cudaFreeHost(s->slot_flag);
            delete s;
            return EPIC_ERR_CUDA;
        }
    }
    s->queue_limit = 4 * (size_t)max_slots;
    s->worker = std::thread(worker_loop, s);
    *out = s;
    return EPIC_OK;
}

epic_status epic_server_submit(epic_server_t s, epic_plan_t plan, const uint8_t* volt_host, int T, float* out_dev,
                               unsigned flags, uint64_t* ticket)
{
    if (!s || !plan || !out_dev || !ticket || T < 0 || T > plan->max_time || (T > 0 && !volt_host) ||
        (flags & ~(EPIC_ACCUMULATE | EPIC_TIME_KERNELS)))
        return EPIC_ERR_INVALID_ARG;
    if (plan->sub > 0 && T % plan->sub != 0) return EPIC_ERR_INVALID_ARG;
    cudaPointerAttributes at{};
    if (cudaPointerGetAttributes(&at, out_dev) != cudaSuccess ||
        (at.type != cudaMemoryTypeDevice && at.type != cudaMemoryTypeManaged)) {
        cudaGetLastError();
        return EPIC_ERR_INVALID_ARG;  // the images must be device memory
    }
    const size_t bytes = (size_t)T * plan->C * plan->A * plan->P * (plan->bits / 4);
    if (round_up(bytes) > s->pool_bytes) return EPIC_ERR_OOM;
    Job* j = new (std::nothrow) Job();
    if (!j) return EPIC_ERR_OOM;
    j->plan = plan;
    j->T = T;
    j->out = out_dev;
    j->flags = flags & EPIC_ACCUMULATE;
    j->host = volt_host;
    j->bytes = bytes;
    j->submitted = Clock::now();
    {
        std::lock_guard<std::mutex> lk(s->mu);
        if (s->pending.size() >= s->queue_limit) {  // admission: bounded queue
            delete j;
            return EPIC_ERR_BUSY;
        }
        j->ticket = s->next_ticket++;
        s->jobs[j->ticket] = j;
        s->pending.push_back(j);
        *ticket = j->ticket;
    }
    s->cv.notify_all();
    return EPIC_OK;
}

epic_status epic_server_poll(epic_server_t s, uint64_t ticket, int* done, double* latency_ms)
{
    if (!s || !done) return EPIC_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->jobs.find(ticket);
    if (it == s->jobs.end()) return EPIC_ERR_NOT_FOUND;
    *done = it->second->done ? 1 : 0;
    if (latency_ms) *latency_ms = it->second->latency_ms;
    return it->second->done ? it->second->status : EPIC_OK;
}

epic_status epic_server_wait(epic_server_t s, uint64_t ticket, int timeout_ms, double* latency_ms)
{
    if (!s) return EPIC_ERR_INVALID_ARG;
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->jobs.find(ticket);
    if (it == s->jobs.end()) return EPIC_ERR_NOT_FOUND;
    Job* j = it->second;
    ++j->waiters;  // the job outlives every waiter: the last one out of a released job frees it
    const bool done =
        s->done_cv.wait_for(lk, std::chrono::milliseconds(std::max(0, timeout_ms)), [&] { return j->done; });
    --j->waiters;
    epic_status st = EPIC_ERR_TIMEOUT;
    if (j->released) {
        st = EPIC_ERR_NOT_FOUND;  // another waiter collected the ticket first
    } else if (done) {
        if (latency_ms) *latency_ms = j->latency_ms;
        st = j->status;
        s->jobs.erase(ticket);
        j->released = true;
    }
    if (j->released && j->waiters == 0) delete j;
    return st;
}

epic_status epic_server_stats(epic_server_t s, int* completed, double* p50_ms, double* p99_ms, int* in_flight)
{
    if (!s) return EPIC_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(s->mu);
    if (completed) *completed = (int)s->latencies.size();
    if (in_flight) {
        int n = 0;
        for (auto* j : s->slot_job) n += j ? 1 : 0;
        *in_flight = n;
    }
    auto pct = [&](double q) {
        if (s->latencies.empty()) return -1.0;
        std::vector<double> w = s->latencies;
        const size_t k = std::min(w.size() - 1, (size_t)(q * (double)(w.size() - 1) + 0.5));
        std::nth_element(w.begin(), w.begin() + k, w.end());
        return w[k];
    };
    if (p50_ms) *p50_ms = pct(0.50);
    if (p99_ms) *p99_ms = pct(0.99);
    return EPIC_OK;
}

epic_status epic_server_destroy(epic_server_t s)
{
    if (!s) return EPIC_OK;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
    }
    s->cv.notify_all();
    if (s->worker.joinable()) s->worker.join();
    for (auto st : s->streams) {
        cudaStreamSynchronize(st);
        cudaStreamDestroy(st);
    }
    for (auto& m : s->slot_mem) epic::call_scratch_free(m);
    cudaFreeHost(s->slot_flag);
    cudaFree(s->pool);
    for (auto& kv : s->jobs) delete kv.second;
    delete s;
    return EPIC_OK;
}

}  // extern "C"
