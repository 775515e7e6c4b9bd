// Many sensors in one pass: the paper's multi-sensor network (Sec. 3, and
// Sec. 5's several sensors on one GPU) as a batch of plans with uneven
// record lengths, geometries and direction sets.  Every sensor's matched
// filter runs, then ONE persistent launch of the time-domain beamformer walks
// the tiles of all sensors.  The first run of a batch autotunes the
// beamformer's stage layout and persistent grid size by timing the
// candidates; later runs replay the whole batch from a CUDA graph.
#include <algorithm>
#include <cstring>
#include <string>
#include <vector>

#include "rtis_internal.h"

struct rtis_batch {
    std::vector<rtis_plan*> plans;
    rtis::TdMaps maps;
    rtis::TdBatch bt;
    int n_sm = 1;
    int variant = 0, grid = 0;
    bool tuned = false;
    float tuned_ms = 0.f;
    cudaStream_t stream = nullptr;  // graph replay stream
    cudaEvent_t ev_in = nullptr, ev_out = nullptr;
    cudaGraphExec_t exec = nullptr;
    std::vector<const void*> key;  // input/output pointers the graph was captured with
    unsigned* d_status = nullptr;  // shared status word for the batched launch
};

namespace {

using rtis::cuda_fail;
using rtis::fail;

rtis_status validate_io(const rtis_batch* b, const int16_t* const* d_in, float* const* d_out, const char* who) {
    if (!d_in || !d_out) return fail(RTIS_ERR_INVALID_ARG, std::string(who) + ": NULL pointer array");
    for (size_t i = 0; i < b->plans.size(); ++i) {
        if (!d_in[i] || !d_out[i]) return fail(RTIS_ERR_INVALID_ARG, std::string(who) + ": NULL input or output");
        if (reinterpret_cast<uintptr_t>(d_in[i]) % 8 || reinterpret_cast<uintptr_t>(d_out[i]) % 4)
            return fail(RTIS_ERR_INVALID_ARG, std::string(who) + ": misaligned input or output");
    }
    return RTIS_OK;
}

// every sensor's matched filter in two launches (forward FFTs, then phase IFFTs, over
// all sensors' channels at their own sizes), then the one batched beamformer launch
cudaError_t enqueue(rtis_batch* b, const int16_t* const* d_in, float* const* d_out, int variant, int grid,
                    cudaStream_t st) {
    const rtis::Plan* ps[rtis::kMfMaxSensors];
    const int n = static_cast<int>(b->plans.size());
    for (int i = 0; i < n; ++i) {
        ps[i] = &b->plans[i]->p;
        b->bt.s[i].E = d_out[i];
    }
    cudaError_t e = rtis::launch_mf_ragged(ps, n, d_in, st);
    if (e != cudaSuccess) return e;
    return rtis::launch_td_batch(b->maps, b->bt, variant, grid, st);
}

rtis_status refresh_tables(rtis_batch* b, cudaStream_t st) {
    for (rtis_plan* pl : b->plans) {
        if (!pl->p.table_dirty) continue;
        cudaError_t e = rtis::launch_steering_table(pl->p, st);
        if (e != cudaSuccess) return cuda_fail(e, "rtis_batch: steering table launch");
    }
    return RTIS_OK;
}

// times every (stage layout, grid) candidate on the real inputs; keeps the fastest
rtis_status autotune(rtis_batch* b, const int16_t* const* d_in, float* const* d_out, cudaStream_t st) {
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
        return cuda_fail(cudaGetLastError(), "rtis_batch: event create");
    float best = 1e30f;
    // grids: one persistent CTA per SM, or one CTA per tile
    const int grids[2] = {std::min(b->bt.total_tiles, b->n_sm), b->bt.total_tiles};
    bool fast = true;
    for (int i = 0; i < b->bt.n_sensors; ++i) fast = fast && rtis::td_fast_epilogue(b->bt.s[i].R, b->bt.s[i].lpf_len);
    cudaError_t err = cudaSuccess;
    for (int v = 0; v < rtis::kTdVariants && err == cudaSuccess; ++v) {
        if (!rtis::td_variant_fits(b->bt.row_max, fast, v)) continue;
        for (int mi = 0; mi < 2 && err == cudaSuccess; ++mi) {
            const int grid = grids[mi];
            err = enqueue(b, d_in, d_out, v, grid, st);  // warm-up (also sets function attributes)
            if (err != cudaSuccess) break;
            float total = 0.f;
            for (int r = 0; r < 3 && err == cudaSuccess; ++r) {
                cudaEventRecord(e0, st);
                err = rtis::launch_td_batch(b->maps, b->bt, v, grid, st);
                cudaEventRecord(e1, st);
                if (err == cudaSuccess) err = cudaEventSynchronize(e1);
                float ms = 0.f;
                if (err == cudaSuccess) err = cudaEventElapsedTime(&ms, e0, e1);
                total += ms;
            }
            if (err == cudaSuccess && total < best) {
                best = total;
                b->variant = v;
                b->grid = grid;
            }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (err != cudaSuccess) return cuda_fail(err, "rtis_batch: autotune");
    b->tuned = true;
    b->tuned_ms = best / 3.f;
    return RTIS_OK;
}

// per-sensor tensor maps and the tile table of a list of plans
rtis_status build_tables(rtis_plan* const* plans, int n, rtis::TdMaps* maps, rtis::TdBatch* bt) {
    if (!plans || n < 1 || n > rtis::kTdMaxSensors) return fail(RTIS_ERR_INVALID_ARG, "batch: need 1 <= n <= 16 plans");
    std::memset(bt, 0, sizeof(*bt));
    int tiles = 0, row_max = 0, lpf_max = 0;
    bool fast = true;
    for (int i = 0; i < n; ++i) {
        if (!plans[i]) return fail(RTIS_ERR_INVALID_ARG, "batch: NULL plan");
        const rtis::Plan& p = plans[i]->p;
        if (p.a_bf16 != plans[0]->p.a_bf16)
            return fail(RTIS_ERR_INVALID_ARG, "batch: plans must share one storage precision (FP32 or BF16)");
        maps->m[i] = p.a_bf16 ? p.tmap_a16 : p.tmap_a;
        rtis::td_fill_sensor(p, nullptr, tiles, &bt->s[i]);
        tiles += rtis::td_tiles(p);
        row_max = std::max(row_max, p.td_row);
        lpf_max = std::max(lpf_max, p.lpf_len);
        fast = fast && rtis::td_fast_epilogue(p.R, p.lpf_len);
    }
    bt->n_sensors = n;
    bt->bf16 = plans[0]->p.a_bf16 ? 1 : 0;
    bt->stall = 0;  // set per run (fault injection)
    bt->total_tiles = tiles;
    bt->row_max = row_max;
    bt->lpf_max = lpf_max;
    if (!rtis::td_variant_fits(row_max, fast, rtis::kTdVariants - 1))
        return fail(RTIS_ERR_UNSUPPORTED, "batch: staged halo too large");
    return RTIS_OK;
}

void drop_graph(rtis_batch* b) {
    if (b->exec) cudaGraphExecDestroy(b->exec);
    b->exec = nullptr;
    b->key.clear();
}

}  // namespace

extern "C" {

rtis_status rtis_batch_create(rtis_batch** out, rtis_plan* const* plans, int n) {
    if (rtis::fault_mode() == rtis::kFaultAlloc) return rtis::fail(RTIS_ERR_OOM, "rtis_batch_create: injected allocation failure");
    if (!out) return fail(RTIS_ERR_INVALID_ARG, "rtis_batch_create: out is NULL");
    *out = nullptr;
    rtis_batch* b = new (std::nothrow) rtis_batch();
    if (!b) return fail(RTIS_ERR_OOM, "rtis_batch_create: host allocation failed");
    rtis_status s = build_tables(plans, n, &b->maps, &b->bt);
    if (s != RTIS_OK) {
        delete b;
        return s;
    }
    b->plans.assign(plans, plans + n);
    const int tiles = b->bt.total_tiles;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&b->n_sm, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaMalloc(&b->d_status, sizeof(unsigned));
    if (e == cudaSuccess) e = cudaMemset(b->d_status, 0, sizeof(unsigned));
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->ev_in, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->ev_out, cudaEventDisableTiming);
    if (e != cudaSuccess) {
        rtis_batch_destroy(b);
        return cuda_fail(e, "rtis_batch_create");
    }
    b->bt.status = b->d_status;
    b->grid = tiles;
    *out = b;
    return RTIS_OK;
}

void rtis_batch_destroy(rtis_batch* b) {
    if (!b) return;
    if (b->stream) cudaStreamSynchronize(b->stream);
    drop_graph(b);
    if (b->ev_in) cudaEventDestroy(b->ev_in);
    if (b->ev_out) cudaEventDestroy(b->ev_out);
    if (b->stream) cudaStreamDestroy(b->stream);
    if (b->d_status) cudaFree(b->d_status);
    delete b;
}

rtis_status rtis_batch_run(rtis_batch* b, const int16_t* const* d_in, float* const* d_out, void* stream) {
    if (rtis::fault_mode() == rtis::kFaultLaunch) return rtis::fail(RTIS_ERR_CUDA, "rtis_batch_run: injected launch failure");
    if (!b) return fail(RTIS_ERR_INVALID_ARG, "rtis_batch_run: NULL batch");
    rtis_status s = validate_io(b, d_in, d_out, "rtis_batch_run");
    if (s != RTIS_OK) return s;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    s = refresh_tables(b, st);
    if (s != RTIS_OK) return s;
    if (!b->tuned) {
        s = autotune(b, d_in, d_out, st);
        if (s != RTIS_OK) return s;
        drop_graph(b);
    }
    const size_t n = b->plans.size();
    std::vector<const void*> key;
    key.reserve(2 * n);
    for (size_t i = 0; i < n; ++i) {
        key.push_back(d_in[i]);
        key.push_back(d_out[i]);
    }
    cudaError_t e = cudaSuccess;
    if (!b->exec || key != b->key) {
        drop_graph(b);
        cudaGraph_t g = nullptr;
        e = cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeRelaxed);
        if (e == cudaSuccess) {
            cudaError_t le = enqueue(b, d_in, d_out, b->variant, b->grid, b->stream);
            e = cudaStreamEndCapture(b->stream, &g);
            if (le != cudaSuccess) e = le;
        }
        if (e == cudaSuccess) e = cudaGraphInstantiate(&b->exec, g, 0);
        if (g) cudaGraphDestroy(g);
        if (e != cudaSuccess) {
            drop_graph(b);
            return cuda_fail(e, "rtis_batch_run: graph capture");
        }
        b->key = key;
    }
    e = cudaEventRecord(b->ev_in, st);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(b->stream, b->ev_in, 0);
    if (e == cudaSuccess) e = cudaGraphLaunch(b->exec, b->stream);
    if (e == cudaSuccess) e = cudaEventRecord(b->ev_out, b->stream);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(st, b->ev_out, 0);
    return e == cudaSuccess ? RTIS_OK : cuda_fail(e, "rtis_batch_run: graph launch");
}

rtis_status rtis_batch_get_info(const rtis_batch* b, rtis_batch_info* info) {
    if (!b || !info) return fail(RTIS_ERR_INVALID_ARG, "rtis_batch_get_info: NULL argument");
    info->n_sensors = static_cast<int>(b->plans.size());
    info->total_tiles = b->bt.total_tiles;
    info->tuned = b->tuned ? 1 : 0;
    info->variant = b->variant;
    info->grid = b->grid;
    info->tuned_ms = b->tuned_ms;
    return RTIS_OK;
}

rtis_status rtis_batch_sync(rtis_batch* b, unsigned* bits_out) {
    if (!b) return fail(RTIS_ERR_INVALID_ARG, "rtis_batch_sync: NULL batch");
    cudaError_t e = cudaStreamSynchronize(b->stream);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    unsigned bits = 0;
    if (e == cudaSuccess) e = cudaMemcpy(&bits, b->d_status, sizeof(unsigned), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemset(b->d_status, 0, sizeof(unsigned));
    if (e != cudaSuccess) return cuda_fail(e, "rtis_batch_sync");
    if (bits_out) *bits_out = bits;
    if (bits & RTIS_DEV_TIMEOUT) return fail(RTIS_ERR_TIMEOUT, "rtis_batch_sync: a bounded device wait ran out");
    return RTIS_OK;
}

rtis_status rtis_process_batch(rtis_plan* const* plans, int n, const int16_t* const* d_in, float* const* d_out,
                               void* stream) {
    if (rtis::fault_mode() == rtis::kFaultLaunch) return rtis::fail(RTIS_ERR_CUDA, "rtis_process_batch: injected launch failure");
    // allocation-free: a stack-built tile table, plain launches on the caller's stream
    rtis_batch b;
    rtis_status s = build_tables(plans, n, &b.maps, &b.bt);
    if (s != RTIS_OK) return s;
    b.plans.assign(plans, plans + n);
    s = validate_io(&b, d_in, d_out, "rtis_process_batch");
    if (s != RTIS_OK) return s;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    s = refresh_tables(&b, st);
    if (s != RTIS_OK) return s;
    int dev = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&b.n_sm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) b.n_sm = 1;
    b.bt.status = plans[0]->p.d_status;  // device checks report to the first plan's status word
    cudaError_t e = enqueue(&b, d_in, d_out, 0, b.bt.total_tiles, st);
    return e == cudaSuccess ? RTIS_OK : cuda_fail(e, "rtis_process_batch: launch");
}

}  // extern "C"
