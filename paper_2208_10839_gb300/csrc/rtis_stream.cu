// Streaming service: the paper's sensor-to-processor queue (Sec. 3: measurements
// arrive over the network at a fixed rate and workers turn them into images)
// as a ring of pinned host slots on one GPU.  A producer submits host
// measurements; each slot's input copy and result copy run on the slot's own
// stream, the chain itself on one compute stream (the plan's workspaces are
// shared), so copies of one measurement overlap the processing of others.  A
// consumer waits for a ticket, with a bound, and receives the energyscape in
// host memory.
#include <chrono>
#include <cstring>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "rtis_internal.h"

namespace {
struct Slot {
    int16_t* h_in = nullptr;   // pinned [M][N]
    int16_t* d_in = nullptr;
    float* d_out = nullptr;
    cudaStream_t copy = nullptr;
    cudaEvent_t in_ready = nullptr, computed = nullptr, out_ready = nullptr;
    cudaGraphExec_t chain = nullptr;  // rtis_process(plan, d_in, d_out) on the compute stream
    int64_t ticket = -1;       // the measurement in this slot, -1 when free
};
}  // namespace

struct rtis_stream {
    rtis_plan* plan = nullptr;
    cudaStream_t compute = nullptr;
    std::vector<Slot> slots;
    int64_t next = 0;
    std::mutex mu;
};

namespace {

using rtis::cuda_fail;
using rtis::fail;

void destroy_stream(rtis_stream* s) {
    if (!s) return;
    for (Slot& sl : s->slots) {
        if (sl.h_in) cudaFreeHost(sl.h_in);
        if (sl.d_in) cudaFree(sl.d_in);
        if (sl.d_out) cudaFree(sl.d_out);
        if (sl.copy) cudaStreamDestroy(sl.copy);
        if (sl.in_ready) cudaEventDestroy(sl.in_ready);
        if (sl.computed) cudaEventDestroy(sl.computed);
        if (sl.out_ready) cudaEventDestroy(sl.out_ready);
        if (sl.chain) cudaGraphExecDestroy(sl.chain);
    }
    if (s->compute) cudaStreamDestroy(s->compute);
    delete s;
}

}  // namespace

extern "C" {

rtis_status rtis_stream_create(rtis_stream** out, rtis_plan* plan, int depth) {
    if (rtis::fault_mode() == rtis::kFaultAlloc) return fail(RTIS_ERR_OOM, "rtis_stream_create: injected allocation failure");
    if (!out || !plan) return fail(RTIS_ERR_INVALID_ARG, "rtis_stream_create: NULL argument");
    *out = nullptr;
    if (depth < 1 || depth > 64) return fail(RTIS_ERR_INVALID_ARG, "rtis_stream_create: depth must be in [1, 64]");
    const rtis::Plan& p = plan->p;
    rtis_stream* s = new (std::nothrow) rtis_stream();
    if (!s) return fail(RTIS_ERR_OOM, "rtis_stream_create: host allocation failed");
    s->plan = plan;
    s->slots.resize(depth);
    const size_t in_bytes = static_cast<size_t>(p.M) * p.N * sizeof(int16_t);
    const size_t out_bytes = static_cast<size_t>(p.D) * p.n_out * sizeof(float);
    cudaError_t e = cudaStreamCreateWithFlags(&s->compute, cudaStreamNonBlocking);  // the chain, in order
    for (Slot& sl : s->slots) {
        if (e == cudaSuccess) e = cudaMallocHost(&sl.h_in, in_bytes);
        if (e == cudaSuccess) e = cudaMalloc(&sl.d_in, in_bytes);
        if (e == cudaSuccess) e = cudaMalloc(&sl.d_out, out_bytes);
        if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&sl.copy, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&sl.in_ready, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&sl.computed, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&sl.out_ready, cudaEventDisableTiming);
    }
    if (e != cudaSuccess) {
        destroy_stream(s);
        cudaGetLastError();
        return (e == cudaErrorMemoryAllocation) ? fail(RTIS_ERR_OOM, "rtis_stream_create: allocation failed")
                                                : cuda_fail(e, "rtis_stream_create");
    }
    // the tables are written before the capture, so the graphs hold the chain alone
    if (plan->p.table_dirty) e = rtis::launch_steering_table(plan->p, s->compute);
    for (Slot& sl : s->slots) {
        if (e != cudaSuccess) break;
        e = cudaStreamBeginCapture(s->compute, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) break;
        const rtis_status st = rtis_process(plan, sl.d_in, sl.d_out, s->compute);
        cudaGraph_t g = nullptr;
        e = cudaStreamEndCapture(s->compute, &g);
        if (st != RTIS_OK) {
            if (g) cudaGraphDestroy(g);
            destroy_stream(s);
            return st;
        }
        if (e == cudaSuccess) e = cudaGraphInstantiate(&sl.chain, g, 0);
        if (g) cudaGraphDestroy(g);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->compute);
    if (e != cudaSuccess) {
        destroy_stream(s);
        cudaGetLastError();
        return cuda_fail(e, "rtis_stream_create: graph capture");
    }
    *out = s;
    return RTIS_OK;
}

rtis_status rtis_stream_submit(rtis_stream* s, const int16_t* host_in, float* host_out, int64_t* ticket) {
    if (rtis::fault_mode() == rtis::kFaultLaunch) return fail(RTIS_ERR_CUDA, "rtis_stream_submit: injected launch failure");
    if (!s || !host_in || !host_out || !ticket) return fail(RTIS_ERR_INVALID_ARG, "rtis_stream_submit: NULL argument");
    std::lock_guard<std::mutex> lock(s->mu);
    const rtis::Plan& p = s->plan->p;
    const int depth = static_cast<int>(s->slots.size());
    Slot& sl = s->slots[static_cast<size_t>(s->next % depth)];
    if (sl.ticket >= 0) return fail(RTIS_ERR_BUSY, "rtis_stream_submit: ring full (wait for the oldest ticket first)");
    const size_t in_bytes = static_cast<size_t>(p.M) * p.N * sizeof(int16_t);
    const size_t out_bytes = static_cast<size_t>(p.D) * p.n_out * sizeof(float);
    std::memcpy(sl.h_in, host_in, in_bytes);  // the caller's buffer is free on return
    cudaError_t e = cudaMemcpyAsync(sl.d_in, sl.h_in, in_bytes, cudaMemcpyHostToDevice, sl.copy);
    if (e == cudaSuccess) e = cudaEventRecord(sl.in_ready, sl.copy);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(s->compute, sl.in_ready, 0);
    if (e != cudaSuccess) return cuda_fail(e, "rtis_stream_submit: input copy");
    e = cudaGraphLaunch(sl.chain, s->compute);
    if (e != cudaSuccess) return cuda_fail(e, "rtis_stream_submit: chain");
    e = cudaEventRecord(sl.computed, s->compute);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(sl.copy, sl.computed, 0);
    if (e == cudaSuccess) e = cudaMemcpyAsync(host_out, sl.d_out, out_bytes, cudaMemcpyDeviceToHost, sl.copy);
    if (e == cudaSuccess) e = cudaEventRecord(sl.out_ready, sl.copy);
    if (e != cudaSuccess) return cuda_fail(e, "rtis_stream_submit: result copy");
    sl.ticket = s->next++;
    *ticket = sl.ticket;
    return RTIS_OK;
}

rtis_status rtis_stream_wait(rtis_stream* s, int64_t ticket, int timeout_ms) {
    if (!s) return fail(RTIS_ERR_INVALID_ARG, "rtis_stream_wait: NULL argument");
    cudaEvent_t ev = nullptr;
    {
        std::lock_guard<std::mutex> lock(s->mu);
        const int depth = static_cast<int>(s->slots.size());
        if (ticket < 0 || ticket >= s->next) return fail(RTIS_ERR_INVALID_ARG, "rtis_stream_wait: unknown ticket");
        Slot& sl = s->slots[static_cast<size_t>(ticket % depth)];
        if (sl.ticket != ticket) return fail(RTIS_ERR_INVALID_ARG, "rtis_stream_wait: ticket already collected");
        ev = sl.out_ready;
    }
    // bounded wait: poll the result event, sleeping briefly between polls
    const auto t0 = std::chrono::steady_clock::now();
    for (;;) {
        const cudaError_t q = cudaEventQuery(ev);
        if (q == cudaSuccess) break;
        if (q != cudaErrorNotReady) return cuda_fail(q, "rtis_stream_wait");
        const auto ms = std::chrono::duration_cast<std::chrono::milliseconds>(std::chrono::steady_clock::now() - t0);
        if (ms.count() >= timeout_ms) return fail(RTIS_ERR_TIMEOUT, "rtis_stream_wait: result not ready in time");
        std::this_thread::sleep_for(std::chrono::microseconds(20));
    }
    std::lock_guard<std::mutex> lock(s->mu);
    s->slots[static_cast<size_t>(ticket % static_cast<int64_t>(s->slots.size()))].ticket = -1;
    return RTIS_OK;
}

void rtis_stream_destroy(rtis_stream* s) {
    if (!s) return;
    cudaDeviceSynchronize();
    destroy_stream(s);
}

}  // extern "C"
