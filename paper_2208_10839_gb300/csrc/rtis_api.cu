// Host side of the C ABI declared in include/rtis.h: argument checks, the
// plan (tables and workspaces allocated once, paper Sec. 4.3), and the
// launch sequence of each entry point.  No C++ exception leaves this file.
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include <cudaTypedefs.h>

#include "rtis_internal.h"

// one kernel launch (expression returning cudaError_t) bracketed by the plan's trace events
#define RTIS_TRACED(plan, stream, kind, expr)                                   \
    ([&]() -> cudaError_t {                                                     \
        const int trace_slot_ = rtis::trace_begin((plan), (stream), (kind));    \
        const cudaError_t trace_err_ = (expr);                                  \
        rtis::trace_end((plan), (stream), trace_slot_);                         \
        return trace_err_;                                                      \
    }())

namespace rtis {

namespace {
thread_local std::string g_last_error;

bool all_finite(const float* v, size_t n) {
    for (size_t i = 0; i < n; ++i)
        if (!std::isfinite(v[i])) return false;
    return true;
}

template <typename T>
cudaError_t dev_alloc(T** ptr, size_t count, size_t* total) {
    *total += count * sizeof(T);
    return cudaMalloc(reinterpret_cast<void**>(ptr), std::max<size_t>(count, 1) * sizeof(T));
}

void free_plan_buffers(Plan& p) {
    void* bufs[] = {p.d_mic, p.d_dirs, p.d_gain, p.d_delay, p.d_tw, p.d_C, p.d_h,
                    p.d_shift, p.d_wt, p.d_dphase, p.d_wraw, p.d_wder, p.d_adj, p.d_adj_red, p.d_Z, p.d_a, p.d_A, p.d_a16,
                    p.d_X, p.d_Y, p.d_kbin, p.d_xmax, p.d_Zb, p.d_ab, p.d_fdtc, p.d_status,
                    p.d_bshift, p.d_bwt, p.d_brot, p.d_hb};
    for (void* b : bufs)
        if (b) cudaFree(b);
}

bool aligned(const void* ptr, size_t a) { return (reinterpret_cast<uintptr_t>(ptr) % a) == 0; }

void destroy_trace_events(Plan& p) {
    for (cudaEvent_t& ev : p.trace_ev)
        if (ev) {
            cudaEventDestroy(ev);
            ev = nullptr;
        }
    p.trace_on = false;
    p.trace_live = false;
    p.trace_n = 0;
}
}  // namespace

void trace_call(Plan& p, cudaStream_t st) {
    p.trace_live = false;
    if (!p.trace_on) return;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) return;
    p.trace_n = 0;
    p.trace_live = true;
}

int trace_begin(Plan& p, cudaStream_t st, int kind) {
    if (!p.trace_live || p.trace_n >= RTIS_TRACE_MAX) return -1;
    const int slot = p.trace_n++;
    p.trace_kind[slot] = kind;
    cudaEventRecord(p.trace_ev[2 * slot], st);
    return slot;
}

void trace_end(Plan& p, cudaStream_t st, int slot) {
    if (slot >= 0) cudaEventRecord(p.trace_ev[2 * slot + 1], st);
}

void set_error(const std::string& msg) { g_last_error = msg; }

int fault_mode() {
    const char* f = std::getenv("RTIS_FAULT");
    if (!f || !*f) return kFaultNone;
    if (!std::strcmp(f, "alloc")) return kFaultAlloc;
    if (!std::strcmp(f, "launch")) return kFaultLaunch;
    if (!std::strcmp(f, "stall")) return kFaultStall;
    return kFaultNone;
}

rtis_status fail(rtis_status s, const std::string& msg) {
    set_error(msg);
    return s;
}

rtis_status cuda_fail(cudaError_t e, const char* what) {
    set_error(std::string(what) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")");
    return RTIS_ERR_CUDA;
}

bool encode_tmap(CUtensorMap* map, CUtensorMapDataType dtype, uint32_t rank, const void* base, const uint64_t* dims,
                 const uint64_t* strides, const uint32_t* box, CUtensorMapSwizzle swizzle, std::string* err) {
    static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
    if (encode == nullptr) {
        void* fn = nullptr;
        cudaDriverEntryPointQueryResult q{};
        cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q);
        if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || fn == nullptr) {
            *err = "cuTensorMapEncodeTiled entry point not available";
            return false;
        }
        encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
    }
    cuuint64_t d[5];
    cuuint64_t st[4];
    cuuint32_t bx[5], es[5];
    for (uint32_t i = 0; i < rank; ++i) {
        d[i] = dims[i];
        bx[i] = box[i];
        es[i] = 1;
        if (i + 1 < rank) st[i] = strides[i];
    }
    CUresult r = encode(map, dtype, rank, const_cast<void*>(base), d, st, bx, es, CU_TENSOR_MAP_INTERLEAVE_NONE, swizzle,
                        CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) {
        *err = "cuTensorMapEncodeTiled failed with CUresult " + std::to_string(static_cast<int>(r));
        return false;
    }
    return true;
}

bool encode_tmap_2d_u32(CUtensorMap* map, const void* base, uint64_t cols, uint64_t rows, uint32_t box_cols,
                        uint32_t box_rows, std::string* err) {
    const uint64_t dims[2] = {cols, rows};
    const uint64_t strides[1] = {cols * 4};
    const uint32_t box[2] = {box_cols, box_rows};
    return encode_tmap(map, CU_TENSOR_MAP_DATA_TYPE_UINT32, 2, base, dims, strides, box, CU_TENSOR_MAP_SWIZZLE_NONE,
                       err);
}

bool encode_tmap_2d_u64(CUtensorMap* map, const void* base, uint64_t cols, uint64_t rows, uint32_t box_cols,
                        uint32_t box_rows, std::string* err) {
    const uint64_t dims[2] = {cols, rows};
    const uint64_t strides[1] = {cols * 8};
    const uint32_t box[2] = {box_cols, box_rows};
    return encode_tmap(map, CU_TENSOR_MAP_DATA_TYPE_UINT64, 2, base, dims, strides, box, CU_TENSOR_MAP_SWIZZLE_NONE,
                       err);
}

}  // namespace rtis

using rtis::Plan;
using rtis::fail;
using rtis::cuda_fail;

extern "C" {

void rtis_options_default(rtis_options* opt) {
    if (!opt) return;
    std::memset(opt, 0, sizeof(*opt));
    opt->c = 343.0;
    opt->decim = 10;
    opt->lpf_len = 0;
    opt->lpf_taps = nullptr;
    opt->band_lo_hz = 20e3;
    opt->band_hi_hz = 80e3;
    opt->path = RTIS_PATH_TD;
    opt->precision = RTIS_PREC_FP32;
    opt->max_delay_s = 10e-6;
    opt->position_slack_m = 0.01;
}

const char* rtis_status_string(rtis_status s) {
    switch (s) {
        case RTIS_OK: return "ok";
        case RTIS_ERR_INVALID_ARG: return "invalid argument";
        case RTIS_ERR_CUDA: return "CUDA error";
        case RTIS_ERR_OOM: return "out of device memory";
        case RTIS_ERR_UNSUPPORTED: return "unsupported configuration";
        case RTIS_ERR_TIMEOUT: return "device wait timed out";
        case RTIS_ERR_NONFINITE: return "non-finite input";
        case RTIS_ERR_DEVICE: return "device-side check failed";
        case RTIS_ERR_BUSY: return "no free slot";
    }
    return "unknown status";
}

const char* rtis_last_error(void) { return rtis::g_last_error.c_str(); }

// TMA view of the baseband signal z (in d_a): Nb complex samples per row, rows bb_stride apart
static bool encode_bb_map(Plan& p, std::string* err) {
    const uint64_t dims[2] = {static_cast<uint64_t>(p.Nb), static_cast<uint64_t>(p.M)};
    const uint64_t strides[1] = {static_cast<uint64_t>(p.bb_stride) * 8};
    const uint32_t box[2] = {static_cast<uint32_t>(rtis::kBbBox), 1};
    return rtis::encode_tmap(&p.tmap_zb, CU_TENSOR_MAP_DATA_TYPE_UINT64, 2, p.d_a, dims, strides, box,
                             CU_TENSOR_MAP_SWIZZLE_NONE, err);
}

// TMA views of the per-measurement analytic signals of rtis_process_many
static bool encode_batch_maps(Plan& p, std::string* err) {
    p.tmap_ab.resize(p.max_batch);
    for (int t = 0; t < p.max_batch; ++t)
        if (!rtis::encode_tmap_2d_u64(&p.tmap_ab[t], p.d_ab + static_cast<size_t>(t) * p.M * p.N,
                                      static_cast<uint64_t>(p.N), static_cast<uint64_t>(p.M), rtis::kTdBox, 1, err))
            return false;
    return true;
}

rtis_status rtis_plan_create(rtis_plan** out, const float* mic_xyz, int n_mics, double fs, const float* chirp,
                             int chirp_len, const float* directions, int n_dirs, int n_samples,
                             const rtis_options* opt_in) {
    if (!out) return fail(RTIS_ERR_INVALID_ARG, "rtis_plan_create: out is NULL");
    *out = nullptr;
    if (!mic_xyz || !chirp || !directions)
        return fail(RTIS_ERR_INVALID_ARG, "rtis_plan_create: mic_xyz, chirp and directions must be non-NULL");
    rtis_options opt;
    rtis_options_default(&opt);
    if (opt_in) opt = *opt_in;
    if (n_mics < 1 || n_mics > rtis::kMaxMics)
        return fail(RTIS_ERR_UNSUPPORTED, "rtis_plan_create: n_mics must be in [1, 32]");
    if (n_dirs < 1) return fail(RTIS_ERR_INVALID_ARG, "rtis_plan_create: n_dirs must be >= 1");
    if (chirp_len < 1) return fail(RTIS_ERR_INVALID_ARG, "rtis_plan_create: chirp_len must be >= 1");
    if (n_samples < 64 || n_samples % 4 != 0)
        return fail(RTIS_ERR_INVALID_ARG, "rtis_plan_create: n_samples must be a multiple of 4 and >= 64");
    if (!(fs > 0.0) || !std::isfinite(fs)) return fail(RTIS_ERR_INVALID_ARG, "rtis_plan_create: fs must be > 0");
    if (!(opt.c > 0.0) || !std::isfinite(opt.c)) return fail(RTIS_ERR_INVALID_ARG, "rtis_plan_create: c must be > 0");
    if (opt.decim < 1) return fail(RTIS_ERR_INVALID_ARG, "rtis_plan_create: decim must be >= 1");
    const int lpf_len = opt.lpf_len ? opt.lpf_len : 4 * opt.decim + 1;
    if (lpf_len < 1 || lpf_len % 2 == 0 || lpf_len > rtis::kTdWarpSamples - 1)
        return fail(RTIS_ERR_INVALID_ARG, "rtis_plan_create: lpf_len must be odd and < 992");
    if (opt.lpf_len == 0 && opt.lpf_taps != nullptr)
        return fail(RTIS_ERR_INVALID_ARG, "rtis_plan_create: lpf_taps given without lpf_len");
    if (!(opt.band_lo_hz >= 0.0) || !(opt.band_hi_hz > opt.band_lo_hz))
        return fail(RTIS_ERR_INVALID_ARG, "rtis_plan_create: need 0 <= band_lo_hz < band_hi_hz");
    if (!(opt.max_delay_s >= 0.0) || !(opt.position_slack_m >= 0.0))
        return fail(RTIS_ERR_INVALID_ARG, "rtis_plan_create: max_delay_s and position_slack_m must be >= 0");
    if (opt.path != RTIS_PATH_TD && opt.path != RTIS_PATH_FD && opt.path != RTIS_PATH_BB)
        return fail(RTIS_ERR_INVALID_ARG, "rtis_plan_create: unknown path");
    if (opt.precision != RTIS_PREC_FP32 && opt.precision != RTIS_PREC_BF16)
        return fail(RTIS_ERR_UNSUPPORTED, "rtis_plan_create: precision must be RTIS_PREC_FP32 or RTIS_PREC_BF16");
    if (opt.max_batch < 0 || opt.max_batch > rtis::kFdMaxFrames)
        return fail(RTIS_ERR_INVALID_ARG, "rtis_plan_create: max_batch must be in [0, 64]");
    if (opt.precision == RTIS_PREC_BF16 && opt.path != RTIS_PATH_TD)
        return fail(RTIS_ERR_UNSUPPORTED, "rtis_plan_create: BF16 storage applies to the time-domain path only");
    if (opt.fd_ifft < RTIS_FD_IFFT_AUTO || opt.fd_ifft > RTIS_FD_IFFT_TC)
        return fail(RTIS_ERR_INVALID_ARG, "rtis_plan_create: fd_ifft must be RTIS_FD_IFFT_AUTO, _FFT or _TC");
    if (opt.td_layout < 0 || opt.td_layout > rtis::kTdVariants || opt.bb_layout < 0 ||
        opt.bb_layout > rtis::kBbVariants || opt.grid_mode < 0 || opt.grid_mode > 2)
        return fail(RTIS_ERR_INVALID_ARG, "rtis_plan_create: td_layout, bb_layout or grid_mode out of range");
    if (!rtis::all_finite(mic_xyz, 3 * static_cast<size_t>(n_mics)) ||
        !rtis::all_finite(directions, 3 * static_cast<size_t>(n_dirs)) ||
        !rtis::all_finite(chirp, chirp_len) || (opt.lpf_taps && !rtis::all_finite(opt.lpf_taps, lpf_len)))
        return fail(RTIS_ERR_NONFINITE, "rtis_plan_create: non-finite geometry, chirp or taps");

    int64_t F = 1;
    while (F < static_cast<int64_t>(n_samples) + chirp_len - 1) F *= 2;
    if (F > 65536 || F < 256)
        return fail(RTIS_ERR_UNSUPPORTED, "rtis_plan_create: FFT length must be in [256, 65536] (N + L - 1 too large)");
    const int k_lo = static_cast<int>(std::ceil(opt.band_lo_hz * F / fs));
    const int k_hi = static_cast<int>(std::floor(opt.band_hi_hz * F / fs));
    if (k_hi < k_lo) return fail(RTIS_ERR_INVALID_ARG, "rtis_plan_create: band holds no FFT bin");
    if (k_hi >= F / 4)
        return fail(RTIS_ERR_UNSUPPORTED, "rtis_plan_create: band must lie below fs/4");
    if (n_samples / opt.decim < 1) return fail(RTIS_ERR_INVALID_ARG, "rtis_plan_create: decim larger than N");

    if (rtis::fault_mode() == rtis::kFaultAlloc) return fail(RTIS_ERR_OOM, "rtis_plan_create: injected allocation failure");
    rtis_plan* plan = new (std::nothrow) rtis_plan();
    if (!plan) return fail(RTIS_ERR_OOM, "rtis_plan_create: host allocation failed");
    Plan& p = plan->p;
    p.opt = opt;
    p.M = n_mics;
    p.N = n_samples;
    p.D = n_dirs;
    p.L = chirp_len;
    p.F = static_cast<int>(F);
    p.P = p.F / 4;
    p.logP = 0;
    while ((1 << p.logP) < p.P) ++p.logP;
    p.k_lo = k_lo;
    p.k_hi = k_hi;
    p.Kb = k_hi - k_lo + 1;
    p.R = opt.decim;
    p.lpf_len = lpf_len;
    p.n_out = n_samples / opt.decim;
    p.fs = fs;
    p.c = opt.c;
    p.a_bf16 = (opt.precision == RTIS_PREC_BF16);
    p.max_batch = opt.max_batch;

    // largest |delta| the geometry (plus calibration slack) can produce
    double pmax = 0.0, umax = 0.0;
    for (int m = 0; m < n_mics; ++m) {
        const double x = mic_xyz[3 * m], y = mic_xyz[3 * m + 1], z = mic_xyz[3 * m + 2];
        pmax = std::max(pmax, std::sqrt(x * x + y * y + z * z));
    }
    for (int d = 0; d < n_dirs; ++d) {
        const double x = directions[3 * d], y = directions[3 * d + 1], z = directions[3 * d + 2];
        umax = std::max(umax, std::sqrt(x * x + y * y + z * z));
    }
    const double dmax = fs * ((pmax + opt.position_slack_m) * umax / opt.c + opt.max_delay_s);
    int H = static_cast<int>(std::ceil(dmax)) + 3;
    H = (H + 3) & ~3;
    p.H = H;
    p.Jlim = H - 2;
    // a lane reads pairs from an even index up to lane_base + Jlim + T + 3, and the
    // row starts up to 3 samples before n_start - H (x0 rounded down to 4 for BF16)
    p.td_nbox = (H + p.Jlim + rtis::kTdWarpSamples + 8 + rtis::kTdBox - 1) / rtis::kTdBox;
    p.td_row = p.td_nbox * rtis::kTdBox;
    p.td_bins_per_tile = (rtis::kTdWarpSamples - lpf_len) / p.R + 1;
    if (rtis::td_smem_bytes(p) > 227 * 1024) {
        delete plan;
        return fail(RTIS_ERR_UNSUPPORTED, "rtis_plan_create: steering delays too large for the staged halo");
    }
    if (p.max_batch > 0) {
        // the batched frequency-domain path's inverse transform: the FFT kernel unless the
        // caller asks for the dense DFT stages on the tensor cores (which need F = 32768)
        const bool tc_ok = rtis::fdtc_supported(p);
        if (opt.fd_ifft == RTIS_FD_IFFT_TC && !tc_ok) {
            delete plan;
            return fail(RTIS_ERR_UNSUPPORTED,
                        "rtis_plan_create: the tensor-core IFFT needs F = 32768, at most 4608 in-band bins and at most 127 low-pass taps");
        }
        p.fd_ifft = (opt.fd_ifft == RTIS_FD_IFFT_TC) ? RTIS_FD_IFFT_TC : RTIS_FD_IFFT_FFT;
    }
    if (opt.path == RTIS_PATH_FD && rtis::fdes_smem_bytes(p) > 227 * 1024) {
        delete plan;
        return fail(RTIS_ERR_UNSUPPORTED,
                    "rtis_plan_create: the frequency-domain path needs F <= 65536 and its buffers in shared memory (N <= ~46000 at R = 10)");
    }
    if (opt.path == RTIS_PATH_BB) {
        // coarse grid: every 4th sample; |floor(delta/4)| <= bb_Jlim whenever |floor(delta)| <= Jlim
        p.Nb = n_samples / rtis::kBbQ;
        p.bb_stride = (p.Nb + 1) & ~1;
        p.k_c = (k_lo + k_hi) / 2;
        p.bb_Jlim = (p.Jlim + 3) / rtis::kBbQ + 1;
        p.bb_H = p.bb_Jlim + 2;
        const int half = (lpf_len - 1) / 2;
        p.bb_ntap = (2 * half) / rtis::kBbQ + 1;
        // a lane reads up to H + 1 + 31 T - 1 + Jlim_b + T + 3 elements into the row
        p.bb_nbox = (p.bb_H + p.bb_Jlim + rtis::kBbWarpSamples + 4 + rtis::kBbBox - 1) / rtis::kBbBox;
        p.bb_row = p.bb_nbox * rtis::kBbBox;
        p.bb_bins_per_tile = (rtis::kBbQ * (rtis::kBbWarpSamples - 1 - p.bb_ntap)) / p.R + 1;
        bool fits = p.bb_bins_per_tile >= 1 && rtis::bb_smem_bytes(p) <= 227 * 1024;
        // every output bin's taps lie inside its warp's kBbWarpSamples coarse samples
        for (int i0 = 0; fits && i0 < p.n_out; i0 += p.bb_bins_per_tile) {
            const int jS = -((half - p.R * i0) >> 2);
            for (int i = i0; fits && i < std::min(p.n_out, i0 + p.bb_bins_per_tile); ++i) {
                const int jlo = -((half - p.R * i) >> 2);
                fits = jlo - jS >= 0 && jlo - jS + p.bb_ntap <= rtis::kBbWarpSamples;
            }
        }
        if (!fits) {
            delete plan;
            return fail(RTIS_ERR_UNSUPPORTED, "rtis_plan_create: baseband tiling does not fit (decim or halo too large)");
        }
    }

    // ---- host tables (FP64, rounded to float once) ----
    std::vector<double> cs(F), sn(F);
    for (int64_t j = 0; j < F; ++j) {
        const double ang = 2.0 * M_PI * static_cast<double>(j) / static_cast<double>(F);
        cs[j] = std::cos(ang);
        sn[j] = -std::sin(ang);
    }
    std::vector<float2> tw(F);
    for (int64_t j = 0; j < F; ++j) tw[j] = make_float2(static_cast<float>(cs[j]), static_cast<float>(sn[j]));
    // C[k'] = 2 conj(S[k]) / F, S[k] = sum_l s[l] exp(-2 pi i k l / F)
    std::vector<float2> C(p.Kb);
    for (int kp = 0; kp < p.Kb; ++kp) {
        const int64_t k = k_lo + kp;
        double re = 0.0, im = 0.0;
        for (int l = 0; l < chirp_len; ++l) {
            const int64_t idx = (k * l) & (F - 1);
            re += chirp[l] * cs[idx];
            im += chirp[l] * sn[idx];
        }
        C[kp] = make_float2(static_cast<float>(2.0 * re / F), static_cast<float>(-2.0 * im / F));
    }
    std::vector<float> h(lpf_len);
    if (opt.lpf_taps) {
        for (int j = 0; j < lpf_len; ++j) h[j] = opt.lpf_taps[j];
    } else {
        const int half = (lpf_len - 1) / 2;
        std::vector<double> hd(lpf_len);
        double sum = 0.0;
        for (int j = 0; j < lpf_len; ++j) {
            const double t = j - half;
            const double x = t / p.R;
            const double sinc = (t == 0) ? 1.0 : std::sin(M_PI * x) / (M_PI * x);
            hd[j] = sinc * 0.5 * (1.0 + std::cos(M_PI * t / (half + 1)));
            sum += hd[j];
        }
        for (int j = 0; j < lpf_len; ++j) h[j] = static_cast<float>(hd[j] / sum);
    }
    // baseband low-pass: the taps at the coarse offsets t = t0 + 4l (t0 = -half +
    // ((4 - c) mod 4) for residue c = (R i - half) mod 4), renormalised per residue
    std::vector<float> hb(opt.path == RTIS_PATH_BB ? 4 * p.bb_ntap : 0, 0.0f);
    if (opt.path == RTIS_PATH_BB) {
        const int half = (lpf_len - 1) / 2;
        for (int c = 0; c < 4; ++c) {
            const int t0 = -half + ((4 - c) & 3);
            double sum = 0.0;
            for (int l = 0; t0 + 4 * l <= half; ++l) sum += h[t0 + 4 * l + half];
            if (!(std::fabs(sum) > 0.0)) {
                delete plan;
                return fail(RTIS_ERR_UNSUPPORTED, "rtis_plan_create: a coarse phase of the low-pass taps sums to 0");
            }
            for (int l = 0; t0 + 4 * l <= half; ++l) hb[c * p.bb_ntap + l] = static_cast<float>(h[t0 + 4 * l + half] / sum);
        }
    }
    std::vector<float> ones(n_mics, 1.0f), zeros(n_mics, 0.0f);

    // ---- device buffers, allocated once ----
    size_t total = 0;
    cudaError_t e = cudaSuccess;
#define RTIS_ALLOC(ptr, count)                                   \
    if (e == cudaSuccess) e = rtis::dev_alloc(&(ptr), (count), &total);
    RTIS_ALLOC(p.d_mic, 3 * n_mics)
    RTIS_ALLOC(p.d_dirs, 3 * static_cast<size_t>(n_dirs))
    RTIS_ALLOC(p.d_gain, n_mics)
    RTIS_ALLOC(p.d_delay, n_mics)
    RTIS_ALLOC(p.d_tw, F)
    RTIS_ALLOC(p.d_C, p.Kb)
    RTIS_ALLOC(p.d_h, lpf_len)
    RTIS_ALLOC(p.d_shift, static_cast<size_t>(n_dirs) * n_mics)
    RTIS_ALLOC(p.d_wt, static_cast<size_t>(n_dirs) * n_mics)
    RTIS_ALLOC(p.d_dphase, static_cast<size_t>(n_dirs) * n_mics)
    RTIS_ALLOC(p.d_wraw, static_cast<size_t>(n_dirs) * n_mics)
    RTIS_ALLOC(p.d_wder, static_cast<size_t>(n_dirs) * n_mics)
    // adjoint partials [range tiles][D][M]; also the loss's per-block partials (<= 1024 floats)
    RTIS_ALLOC(p.d_adj, std::max<size_t>(512, static_cast<size_t>((p.n_out + p.td_bins_per_tile - 1) /
                                                                   p.td_bins_per_tile) * n_dirs * n_mics))
    RTIS_ALLOC(p.d_adj_red, static_cast<size_t>(n_mics) * 16 * 5)
    if (p.max_batch > 0) {
        RTIS_ALLOC(p.d_X, static_cast<size_t>(p.Kb) * n_mics * p.max_batch)
        RTIS_ALLOC(p.d_Y, static_cast<size_t>(p.Kb) * n_dirs * p.max_batch)
        RTIS_ALLOC(p.d_kbin, static_cast<size_t>(p.Kb))
        RTIS_ALLOC(p.d_xmax, static_cast<size_t>(n_mics))
        RTIS_ALLOC(p.d_Zb, static_cast<size_t>(p.max_batch) * n_mics * 2 * p.P)
        RTIS_ALLOC(p.d_ab, static_cast<size_t>(p.max_batch) * n_mics * n_samples)
        if (p.fd_ifft == RTIS_FD_IFFT_TC) RTIS_ALLOC(p.d_fdtc, rtis::fdtc_const_bytes())
    }
    if (opt.path == RTIS_PATH_BB) {
        RTIS_ALLOC(p.d_bshift, static_cast<size_t>(n_dirs) * n_mics)
        RTIS_ALLOC(p.d_bwt, static_cast<size_t>(n_dirs) * n_mics)
        RTIS_ALLOC(p.d_brot, static_cast<size_t>(n_dirs) * n_mics)
        RTIS_ALLOC(p.d_hb, hb.size())
    }
    RTIS_ALLOC(p.d_A, static_cast<size_t>(n_mics) * p.Kb)
    RTIS_ALLOC(p.d_Z, static_cast<size_t>(n_mics) * 2 * p.P)
    RTIS_ALLOC(p.d_a, static_cast<size_t>(n_mics) * n_samples)
    if (p.a_bf16) RTIS_ALLOC(p.d_a16, static_cast<size_t>(n_mics) * n_samples)
    RTIS_ALLOC(p.d_status, 1)
#undef RTIS_ALLOC
    p.bytes = total;
    if (e != cudaSuccess) {
        rtis::free_plan_buffers(p);
        delete plan;
        cudaGetLastError();
        return (e == cudaErrorMemoryAllocation) ? fail(RTIS_ERR_OOM, "rtis_plan_create: cudaMalloc failed")
                                                : cuda_fail(e, "rtis_plan_create: cudaMalloc");
    }
#define RTIS_UP(dst, src, bytes) \
    if (e == cudaSuccess) e = cudaMemcpy((dst), (src), (bytes), cudaMemcpyHostToDevice);
    RTIS_UP(p.d_mic, mic_xyz, 3 * n_mics * sizeof(float))
    RTIS_UP(p.d_dirs, directions, 3 * static_cast<size_t>(n_dirs) * sizeof(float))
    RTIS_UP(p.d_gain, ones.data(), n_mics * sizeof(float))
    RTIS_UP(p.d_delay, zeros.data(), n_mics * sizeof(float))
    std::vector<float2> kbin(p.max_batch > 0 ? p.Kb : 0);
    for (int kp = 0; kp < static_cast<int>(kbin.size()); ++kp) kbin[kp] = make_float2(static_cast<float>(k_lo + kp), 0.f);
    if (p.max_batch > 0) RTIS_UP(p.d_kbin, kbin.data(), kbin.size() * sizeof(float2))
    RTIS_UP(p.d_tw, tw.data(), F * sizeof(float2))
    RTIS_UP(p.d_C, C.data(), p.Kb * sizeof(float2))
    RTIS_UP(p.d_h, h.data(), lpf_len * sizeof(float))
    if (!hb.empty()) RTIS_UP(p.d_hb, hb.data(), hb.size() * sizeof(float))
    if (p.d_fdtc) {
        std::vector<unsigned char> img;
        rtis::fdtc_build_constants(p, img);
        RTIS_UP(p.d_fdtc, img.data(), img.size())
    }
#undef RTIS_UP
    if (e == cudaSuccess) e = cudaMemset(p.d_status, 0, sizeof(unsigned));
    if (e == cudaSuccess) e = rtis::launch_steering_table(p, 0);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) {
        rtis::free_plan_buffers(p);
        delete plan;
        return cuda_fail(e, "rtis_plan_create: table upload");
    }
    std::string err;
    if (!rtis::encode_tmap_2d_u64(&p.tmap_a, p.d_a, static_cast<uint64_t>(n_samples), static_cast<uint64_t>(n_mics),
                                  rtis::kTdBox, 1, &err) ||
        (p.a_bf16 && !rtis::encode_tmap_2d_u32(&p.tmap_a16, p.d_a16, static_cast<uint64_t>(n_samples),
                                               static_cast<uint64_t>(n_mics), rtis::kTdBox, 1, &err)) ||
        (opt.path == RTIS_PATH_BB && !encode_bb_map(p, &err)) ||
        !encode_batch_maps(p, &err)) {
        rtis::free_plan_buffers(p);
        delete plan;
        return fail(RTIS_ERR_CUDA, "rtis_plan_create: " + err);
    }
    {
        int dev = 0;
        cudaGetDevice(&dev);
        if (cudaDeviceGetAttribute(&p.n_sm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) p.n_sm = 1;
    }
    unsigned bits = 0;
    cudaMemcpy(&bits, p.d_status, sizeof(unsigned), cudaMemcpyDeviceToHost);
    if (!(bits & RTIS_DEV_DELAY_RANGE)) {
        // autotune the beamformer on the zeroed workspace with a scratch output
        float* scratch = nullptr;
        e = cudaMemset(p.d_a, 0, static_cast<size_t>(n_mics) * n_samples * sizeof(float2));
        if (e == cudaSuccess && p.a_bf16) e = cudaMemset(p.d_a16, 0, static_cast<size_t>(n_mics) * n_samples * 4);
        if (e == cudaSuccess) e = cudaMalloc(&scratch, static_cast<size_t>(n_dirs) * p.n_out * sizeof(float));
        int n_sm = 1, dev = 0;
        cudaGetDevice(&dev);
        if (cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) n_sm = 1;
        if (opt.td_layout > 0) {  // forced: no autotuning
            if (!rtis::td_variant_fits(p.td_row, rtis::td_fast_epilogue(p.R, p.lpf_len), opt.td_layout - 1)) {
                cudaFree(scratch);
                rtis::free_plan_buffers(p);
                delete plan;
                return fail(RTIS_ERR_UNSUPPORTED, "rtis_plan_create: the forced td_layout does not fit shared memory");
            }
            p.td_variant = opt.td_layout - 1;
            p.td_grid = opt.grid_mode == 2 ? std::min(rtis::td_tiles(p), n_sm) : rtis::td_tiles(p);
        } else if (e == cudaSuccess) {
            e = rtis::td_autotune(p, scratch);
        }
        if (opt.path == RTIS_PATH_BB && opt.bb_layout > 0) {
            if (!rtis::bb_variant_fits(p, opt.bb_layout - 1)) {
                cudaFree(scratch);
                rtis::free_plan_buffers(p);
                delete plan;
                return fail(RTIS_ERR_UNSUPPORTED, "rtis_plan_create: the forced bb_layout does not fit shared memory");
            }
            p.bb_variant = opt.bb_layout - 1;
            p.bb_grid = opt.grid_mode == 2 ? std::min(rtis::bb_tiles(p), n_sm) : rtis::bb_tiles(p);
        } else if (e == cudaSuccess && opt.path == RTIS_PATH_BB) {
            e = rtis::bb_autotune(p, scratch);
        }
        if (scratch) cudaFree(scratch);
        if (e == cudaSuccess) e = cudaMemcpy(&bits, p.d_status, sizeof(unsigned), cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) {
            rtis::free_plan_buffers(p);
            delete plan;
            cudaGetLastError();
            return cuda_fail(e, "rtis_plan_create: beamformer autotune");
        }
        if (bits & RTIS_DEV_TIMEOUT) {
            rtis::free_plan_buffers(p);
            delete plan;
            return fail(RTIS_ERR_TIMEOUT, "rtis_plan_create: beamformer autotune timed out");
        }
    }
    if (bits & RTIS_DEV_DELAY_RANGE) {
        rtis::free_plan_buffers(p);
        delete plan;
        return fail(RTIS_ERR_DEVICE, "rtis_plan_create: a steering delay exceeds the staged halo");
    }
    *out = plan;
    return RTIS_OK;
}

void rtis_plan_destroy(rtis_plan* plan) {
    if (!plan) return;
    cudaDeviceSynchronize();
    rtis::destroy_trace_events(plan->p);
    rtis::free_plan_buffers(plan->p);
    delete plan;
}

rtis_status rtis_plan_get_info(const rtis_plan* plan, rtis_plan_info* info) {
    if (!plan || !info) return fail(RTIS_ERR_INVALID_ARG, "rtis_plan_get_info: NULL argument");
    const Plan& p = plan->p;
    info->n_mics = p.M;
    info->n_samples = p.N;
    info->n_dirs = p.D;
    info->chirp_len = p.L;
    info->fft_len = p.F;
    info->k_lo = p.k_lo;
    info->k_hi = p.k_hi;
    info->decim = p.R;
    info->lpf_len = p.lpf_len;
    info->n_out = p.n_out;
    info->halo = p.H;
    info->max_shift = p.Jlim;
    info->workspace_bytes = p.bytes;
    info->td_variant = p.td_variant;
    info->td_grid = p.td_grid;
    info->td_tuned_ms = p.td_tuned_ms;
    info->n_coarse = p.Nb;
    info->k_c = p.k_c;
    info->bb_variant = p.bb_variant;
    info->bb_grid = p.bb_grid;
    info->bb_tuned_ms = p.bb_tuned_ms;
    for (int i = 0; i < 16; ++i) {
        info->td_layout_ms[i] = p.td_variant_ms[i];
        info->bb_layout_ms[i] = p.bb_variant_ms[i];
    }
    info->fd_ifft = p.max_batch > 0 ? p.fd_ifft : 0;
    return RTIS_OK;
}

static rtis_status ensure_table(Plan& p, cudaStream_t st) {
    if (!p.table_dirty) return RTIS_OK;
    cudaError_t e = RTIS_TRACED(p, st, RTIS_KERNEL_STEERING_TABLE, rtis::launch_steering_table(p, st));
    return e == cudaSuccess ? RTIS_OK : cuda_fail(e, "steering table launch");
}

rtis_status rtis_matched_filter(rtis_plan* plan, const int16_t* d_in, float* d_a, float* d_A, void* stream) {
    if (rtis::fault_mode() == rtis::kFaultLaunch) return rtis::fail(RTIS_ERR_CUDA, "rtis_matched_filter: injected launch failure");
    if (!plan || !d_in) return fail(RTIS_ERR_INVALID_ARG, "rtis_matched_filter: NULL plan or input");
    if (!rtis::aligned(d_in, 8)) return fail(RTIS_ERR_INVALID_ARG, "rtis_matched_filter: d_in must be 8-byte aligned");
    if ((d_a && !rtis::aligned(d_a, 8)) || (d_A && !rtis::aligned(d_A, 8)))
        return fail(RTIS_ERR_INVALID_ARG, "rtis_matched_filter: outputs must be 8-byte aligned");
    Plan& p = plan->p;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    rtis::trace_call(p, st);
    cudaError_t e = RTIS_TRACED(p, st, RTIS_KERNEL_MF_FORWARD, rtis::launch_mf_forward(p, d_in, st));
    if (e != cudaSuccess) return cuda_fail(e, "rtis_matched_filter: forward launch");
    e = RTIS_TRACED(p, st, RTIS_KERNEL_MF_INVERSE,
                    rtis::launch_mf_inverse(p, reinterpret_cast<float2*>(d_a), reinterpret_cast<float2*>(d_A), st));
    if (e != cudaSuccess) return cuda_fail(e, "rtis_matched_filter: inverse launch");
    return RTIS_OK;
}

rtis_status rtis_beamform_td(rtis_plan* plan, const float* d_a, float* d_out, void* stream) {
    if (rtis::fault_mode() == rtis::kFaultLaunch) return rtis::fail(RTIS_ERR_CUDA, "rtis_beamform_td: injected launch failure");
    if (!plan || !d_a || !d_out) return fail(RTIS_ERR_INVALID_ARG, "rtis_beamform_td: NULL argument");
    if (!rtis::aligned(d_a, 16)) return fail(RTIS_ERR_INVALID_ARG, "rtis_beamform_td: d_a must be 16-byte aligned");
    if (!rtis::aligned(d_out, 4)) return fail(RTIS_ERR_INVALID_ARG, "rtis_beamform_td: d_out must be 4-byte aligned");
    Plan& p = plan->p;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    CUtensorMap map;
    std::string err;
    if (!rtis::encode_tmap_2d_u64(&map, d_a, p.N, p.M, rtis::kTdBox, 1, &err))
        return fail(RTIS_ERR_CUDA, "rtis_beamform_td: " + err);
    rtis::trace_call(p, st);
    rtis_status s = ensure_table(p, st);
    if (s != RTIS_OK) return s;
    cudaError_t e = RTIS_TRACED(p, st, RTIS_KERNEL_TD_BEAMFORM,
                                rtis::launch_td_beamform(p, map, false, d_out, st));  // the caller's complex-float a
    return e == cudaSuccess ? RTIS_OK : cuda_fail(e, "rtis_beamform_td: launch");
}

rtis_status rtis_baseband_signal(rtis_plan* plan, const int16_t* d_in, float* d_z, void* stream) {
    if (rtis::fault_mode() == rtis::kFaultLaunch) return rtis::fail(RTIS_ERR_CUDA, "rtis_baseband_signal: injected launch failure");
    if (!plan || !d_in || !d_z) return fail(RTIS_ERR_INVALID_ARG, "rtis_baseband_signal: NULL argument");
    if (!rtis::aligned(d_in, 8) || !rtis::aligned(d_z, 8))
        return fail(RTIS_ERR_INVALID_ARG, "rtis_baseband_signal: d_in and d_z must be 8-byte aligned");
    Plan& p = plan->p;
    if (p.opt.path != RTIS_PATH_BB)
        return fail(RTIS_ERR_UNSUPPORTED, "rtis_baseband_signal: the plan was not created for RTIS_PATH_BB");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    rtis::trace_call(p, st);
    cudaError_t e = RTIS_TRACED(p, st, RTIS_KERNEL_MF_FORWARD, rtis::launch_mf_forward(p, d_in, st));
    if (e == cudaSuccess)
        e = RTIS_TRACED(p, st, RTIS_KERNEL_MF_INVERSE,
                        rtis::launch_mf_inverse_bb(p, reinterpret_cast<float2*>(d_z), p.Nb, st));
    return e == cudaSuccess ? RTIS_OK : cuda_fail(e, "rtis_baseband_signal: launch");
}

rtis_status rtis_beamform_bb(rtis_plan* plan, const float* d_z, float* d_out, void* stream) {
    if (rtis::fault_mode() == rtis::kFaultLaunch) return rtis::fail(RTIS_ERR_CUDA, "rtis_beamform_bb: injected launch failure");
    if (!plan || !d_z || !d_out) return fail(RTIS_ERR_INVALID_ARG, "rtis_beamform_bb: NULL argument");
    if (!rtis::aligned(d_z, 16)) return fail(RTIS_ERR_INVALID_ARG, "rtis_beamform_bb: d_z must be 16-byte aligned");
    if (!rtis::aligned(d_out, 4)) return fail(RTIS_ERR_INVALID_ARG, "rtis_beamform_bb: d_out must be 4-byte aligned");
    Plan& p = plan->p;
    if (p.opt.path != RTIS_PATH_BB)
        return fail(RTIS_ERR_UNSUPPORTED, "rtis_beamform_bb: the plan was not created for RTIS_PATH_BB");
    if (p.Nb % 2 != 0)
        return fail(RTIS_ERR_UNSUPPORTED, "rtis_beamform_bb: rows of an odd number of coarse samples (N/4) are not 16-byte strided");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    CUtensorMap map;
    std::string err;
    if (!rtis::encode_tmap_2d_u64(&map, d_z, p.Nb, p.M, rtis::kBbBox, 1, &err))
        return fail(RTIS_ERR_CUDA, "rtis_beamform_bb: " + err);
    rtis::trace_call(p, st);
    rtis_status s = ensure_table(p, st);
    if (s != RTIS_OK) return s;
    cudaError_t e = RTIS_TRACED(p, st, RTIS_KERNEL_BB_BEAMFORM, rtis::launch_bb_beamform(p, map, d_out, st));
    return e == cudaSuccess ? RTIS_OK : cuda_fail(e, "rtis_beamform_bb: launch");
}

rtis_status rtis_process(rtis_plan* plan, const int16_t* d_in, float* d_out, void* stream) {
    if (rtis::fault_mode() == rtis::kFaultLaunch) return rtis::fail(RTIS_ERR_CUDA, "rtis_process: injected launch failure");
    if (!plan || !d_in || !d_out) return fail(RTIS_ERR_INVALID_ARG, "rtis_process: NULL argument");
    if (!rtis::aligned(d_in, 8)) return fail(RTIS_ERR_INVALID_ARG, "rtis_process: d_in must be 8-byte aligned");
    if (!rtis::aligned(d_out, 4)) return fail(RTIS_ERR_INVALID_ARG, "rtis_process: d_out must be 4-byte aligned");
    Plan& p = plan->p;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    rtis::trace_call(p, st);
    rtis_status s = ensure_table(p, st);
    if (s != RTIS_OK) return s;
    using rtis::launch_mf_inverse;
    cudaError_t e = RTIS_TRACED(p, st, RTIS_KERNEL_MF_FORWARD, rtis::launch_mf_forward(p, d_in, st));
    if (p.opt.path == RTIS_PATH_FD) {
        if (e == cudaSuccess) e = RTIS_TRACED(p, st, RTIS_KERNEL_MF_INVERSE, launch_mf_inverse(p, nullptr, p.d_A, st));
        if (e == cudaSuccess)
            e = RTIS_TRACED(p, st, RTIS_KERNEL_FD_ENERGYSCAPE, rtis::launch_fd_energyscape(p, p.d_A, d_out, st));
    } else if (p.opt.path == RTIS_PATH_BB) {
        if (e == cudaSuccess)
            e = RTIS_TRACED(p, st, RTIS_KERNEL_MF_INVERSE, rtis::launch_mf_inverse_bb(p, p.d_a, p.bb_stride, st));
        if (e == cudaSuccess)
            e = RTIS_TRACED(p, st, RTIS_KERNEL_BB_BEAMFORM, rtis::launch_bb_beamform(p, p.tmap_zb, d_out, st));
    } else {
        if (p.a_bf16) {
            if (e == cudaSuccess)
                e = RTIS_TRACED(p, st, RTIS_KERNEL_MF_INVERSE, launch_mf_inverse(p, nullptr, nullptr, st, p.d_a16));
            if (e == cudaSuccess)
                e = RTIS_TRACED(p, st, RTIS_KERNEL_TD_BEAMFORM, rtis::launch_td_beamform(p, p.tmap_a16, true, d_out, st));
        } else {
            if (e == cudaSuccess) e = RTIS_TRACED(p, st, RTIS_KERNEL_MF_INVERSE, launch_mf_inverse(p, p.d_a, nullptr, st));
            if (e == cudaSuccess)
                e = RTIS_TRACED(p, st, RTIS_KERNEL_TD_BEAMFORM, rtis::launch_td_beamform(p, p.tmap_a, false, d_out, st));
        }
    }
    return e == cudaSuccess ? RTIS_OK : cuda_fail(e, "rtis_process: launch");
}

rtis_status rtis_process_many(rtis_plan* plan, const int16_t* d_in, int n, float* d_out_td, float* d_out_fd,
                              void* stream) {
    if (rtis::fault_mode() == rtis::kFaultLaunch) return rtis::fail(RTIS_ERR_CUDA, "rtis_process_many: injected launch failure");
    if (!plan || !d_in || (!d_out_td && !d_out_fd)) return fail(RTIS_ERR_INVALID_ARG, "rtis_process_many: NULL argument");
    if (n < 1) return fail(RTIS_ERR_INVALID_ARG, "rtis_process_many: n must be >= 1");
    if (!rtis::aligned(d_in, 8) || (d_out_td && !rtis::aligned(d_out_td, 4)) || (d_out_fd && !rtis::aligned(d_out_fd, 4)))
        return fail(RTIS_ERR_INVALID_ARG, "rtis_process_many: d_in must be 8-byte and the outputs 4-byte aligned");
    Plan& p = plan->p;
    if (d_out_fd && n > p.max_batch)
        return fail(RTIS_ERR_INVALID_ARG, "rtis_process_many: n exceeds the plan's max_batch (rtis_options)");
    if (d_out_fd && rtis::fdes_smem_bytes(p) > 227 * 1024)
        return fail(RTIS_ERR_UNSUPPORTED, "rtis_process_many: the frequency-domain path needs F <= 65536 and its buffers in shared memory");
    const size_t in_stride = static_cast<size_t>(p.M) * p.N, out_stride = static_cast<size_t>(p.D) * p.n_out;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    rtis::trace_call(p, st);
    rtis_status s = ensure_table(p, st);
    if (s != RTIS_OK) return s;
    cudaError_t e = cudaSuccess;
    if (n <= p.max_batch && !(d_out_td && p.a_bf16)) {
        // all n matched filters in two launches (grid z = measurement): analytic
        // signals into d_ab[t], spectra into frame t of X; then the time-domain
        // beamformer over up to 16 measurements per persistent launch
        rtis::MfBatch mb;
        mb.n = n;
        mb.x_stride = in_stride;
        mb.Z = p.d_Zb;
        mb.z_stride = static_cast<size_t>(p.M) * 2 * p.P;
        mb.a_stride = in_stride;
        mb.A_tstride = 1;
        e = RTIS_TRACED(p, st, RTIS_KERNEL_MF_FORWARD, rtis::launch_mf_forward(p, d_in, st, mb));
        if (e == cudaSuccess)
            e = RTIS_TRACED(p, st, RTIS_KERNEL_MF_INVERSE,
                            rtis::launch_mf_inverse(p, d_out_td ? p.d_ab : nullptr, d_out_fd ? p.d_X : nullptr, st,
                                                    nullptr, n, p.M * n, mb));
        const int per_sensor = rtis::td_tiles(p);
        for (int t0 = 0; d_out_td && t0 < n && e == cudaSuccess; t0 += rtis::kTdMaxSensors) {
            const int cnt = std::min(rtis::kTdMaxSensors, n - t0);
            rtis::TdMaps maps;
            rtis::TdBatch bt;
            std::memset(&bt, 0, sizeof(bt));
            for (int i = 0; i < cnt; ++i) {
                maps.m[i] = p.tmap_ab[t0 + i];
                rtis::td_fill_sensor(p, d_out_td + (t0 + i) * out_stride, i * per_sensor, &bt.s[i]);
            }
            bt.n_sensors = cnt;
            bt.total_tiles = cnt * per_sensor;
            bt.row_max = p.td_row;
            bt.lpf_max = p.lpf_len;
            bt.status = p.d_status;
            bt.stall = (rtis::fault_mode() == rtis::kFaultStall) ? 1 : 0;
            // the plan's tuned grid: one CTA per tile, or its persistent CTA count
            const int grid = (p.td_grid <= 0 || p.td_grid >= per_sensor) ? bt.total_tiles : p.td_grid;
            e = RTIS_TRACED(p, st, RTIS_KERNEL_TD_BEAMFORM, rtis::launch_td_batch(maps, bt, p.td_variant, grid, st));
        }
    }
    // per measurement: matched filter -> analytic signal (time domain) and/or the
    // in-band spectra as frame t of X [Kb][M][n]; the time-domain energyscape
    for (int t = 0; (n > p.max_batch || (d_out_td && p.a_bf16)) && t < n && e == cudaSuccess; ++t) {
        e = RTIS_TRACED(p, st, RTIS_KERNEL_MF_FORWARD, rtis::launch_mf_forward(p, d_in + t * in_stride, st));
        float2* a32 = (d_out_td && !p.a_bf16) ? p.d_a : nullptr;
        uint32_t* a16 = (d_out_td && p.a_bf16) ? p.d_a16 : nullptr;
        float2* Xt = d_out_fd ? p.d_X + t : nullptr;
        if (e == cudaSuccess)
            e = RTIS_TRACED(p, st, RTIS_KERNEL_MF_INVERSE, rtis::launch_mf_inverse(p, a32, Xt, st, a16, n, p.M * n));
        if (e == cudaSuccess && d_out_td)
            e = RTIS_TRACED(p, st, RTIS_KERNEL_TD_BEAMFORM,
                            rtis::launch_td_beamform(p, p.a_bf16 ? p.tmap_a16 : p.tmap_a, p.a_bf16,
                                                     d_out_td + t * out_stride, st));
    }
    if (e == cudaSuccess && d_out_fd) {
        // the steering GEMM: "frequency" k' + k_lo (exact) times "delay" delta/F (the
        // steering table's phase slope), so the phases equal the per-direction path's
        rtis::FdGemmPlan g;
        g.M = p.M;
        g.D = p.D;
        g.K = p.Kb;
        g.T = n;
        g.precision = RTIS_PREC_FP32;
        g.y_dkt = 1;  // per direction, the bins of all measurements together
        int dev = 0;
        cudaGetDevice(&dev);
        if (cudaDeviceGetAttribute(&g.n_sm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) g.n_sm = 1;
        g.d_tau = p.d_dphase;
        g.d_freq = p.d_kbin;
        g.d_gain = p.d_gain;
        g.d_scale = p.d_xmax;
        g.d_status = p.d_status;
        CUtensorMap ymap;
        const CUtensorMap* ym = nullptr;
        if (n % 2 == 0 && n >= 16) {
            std::string err;
            if (!rtis::fd_gemm_encode_ymap(g, p.d_Y, &ymap, &err)) return fail(RTIS_ERR_CUDA, "rtis_process_many: " + err);
            ym = &ymap;
        }
        e = RTIS_TRACED(p, st, RTIS_KERNEL_FD_GEMM, rtis::launch_fd_gemm(g, p.d_X, p.d_Y, ym, st));
        if (e == cudaSuccess && p.d_fdtc)
            e = RTIS_TRACED(p, st, RTIS_KERNEL_FD_ENERGYSCAPE,
                            rtis::launch_fd_energyscape_tc(p, p.d_fdtc, p.d_Y, n, d_out_fd, g.n_sm, st));
        else if (e == cudaSuccess)
            e = RTIS_TRACED(p, st, RTIS_KERNEL_FD_ENERGYSCAPE,
                            rtis::launch_fd_energyscape_from_y(p, p.d_Y, n, d_out_fd, st));
    }
    return e == cudaSuccess ? RTIS_OK : cuda_fail(e, "rtis_process_many: launch");
}

rtis_status rtis_beamform_fd(rtis_plan* plan, const float* d_A, float* d_out, void* stream) {
    if (rtis::fault_mode() == rtis::kFaultLaunch) return rtis::fail(RTIS_ERR_CUDA, "rtis_beamform_fd: injected launch failure");
    if (!plan || !d_A || !d_out) return fail(RTIS_ERR_INVALID_ARG, "rtis_beamform_fd: NULL argument");
    if (!rtis::aligned(d_A, 8) || !rtis::aligned(d_out, 4))
        return fail(RTIS_ERR_INVALID_ARG, "rtis_beamform_fd: d_A must be 8-byte aligned");
    Plan& p = plan->p;
    if (rtis::fdes_smem_bytes(p) > 227 * 1024)
        return fail(RTIS_ERR_UNSUPPORTED, "rtis_beamform_fd: needs F <= 65536 and its buffers in shared memory");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    rtis::trace_call(p, st);
    rtis_status s = ensure_table(p, st);
    if (s != RTIS_OK) return s;
    cudaError_t e = RTIS_TRACED(p, st, RTIS_KERNEL_FD_ENERGYSCAPE,
                                rtis::launch_fd_energyscape(p, reinterpret_cast<const float2*>(d_A), d_out, st));
    return e == cudaSuccess ? RTIS_OK : cuda_fail(e, "rtis_beamform_fd: launch");
}

rtis_status rtis_steering_table(rtis_plan* plan, int32_t* d_shift, float* d_weight, void* stream) {
    if (rtis::fault_mode() == rtis::kFaultLaunch) return rtis::fail(RTIS_ERR_CUDA, "rtis_steering_table: injected launch failure");
    if (!plan || !d_shift || !d_weight) return fail(RTIS_ERR_INVALID_ARG, "rtis_steering_table: NULL argument");
    if (!rtis::aligned(d_weight, 16) || !rtis::aligned(d_shift, 4))
        return fail(RTIS_ERR_INVALID_ARG, "rtis_steering_table: d_weight must be 16-byte aligned");
    Plan& p = plan->p;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    rtis_status s = ensure_table(p, st);
    if (s != RTIS_OK) return s;
    const size_t n = static_cast<size_t>(p.D) * p.M;
    cudaError_t e = cudaMemcpyAsync(d_shift, p.d_shift, n * sizeof(int), cudaMemcpyDeviceToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_weight, p.d_wt, n * sizeof(float4), cudaMemcpyDeviceToDevice, st);
    return e == cudaSuccess ? RTIS_OK : cuda_fail(e, "rtis_steering_table: copy");
}

rtis_status rtis_fd_gemm_create(rtis_fd_gemm** out, const float* mic_xyz, int n_mics, const float* directions,
                                int n_dirs, const double* freqs_hz, int n_bins, int n_frames, double c,
                                const float* gain, const float* delay_s, int precision) {
    if (rtis::fault_mode() == rtis::kFaultAlloc) return rtis::fail(RTIS_ERR_OOM, "rtis_fd_gemm_create: injected allocation failure");
    if (!out) return fail(RTIS_ERR_INVALID_ARG, "rtis_fd_gemm_create: out is NULL");
    *out = nullptr;
    if (!mic_xyz || !directions || !freqs_hz)
        return fail(RTIS_ERR_INVALID_ARG, "rtis_fd_gemm_create: mic_xyz, directions and freqs_hz must be non-NULL");
    if (n_mics < 1 || n_mics > rtis::kMaxMics)
        return fail(RTIS_ERR_UNSUPPORTED, "rtis_fd_gemm_create: n_mics must be in [1, 32]");
    if (n_dirs < 1 || n_bins < 1) return fail(RTIS_ERR_INVALID_ARG, "rtis_fd_gemm_create: n_dirs and n_bins must be >= 1");
    if (n_frames < 1 || n_frames > rtis::kFdMaxFrames)
        return fail(RTIS_ERR_UNSUPPORTED, "rtis_fd_gemm_create: n_frames must be in [1, 64]");
    if (!(c > 0.0) || !std::isfinite(c)) return fail(RTIS_ERR_INVALID_ARG, "rtis_fd_gemm_create: c must be > 0");
    if (precision != RTIS_PREC_FP32 && precision != RTIS_PREC_BF16 && precision != RTIS_PREC_FP16)
        return fail(RTIS_ERR_INVALID_ARG, "rtis_fd_gemm_create: unknown precision");
    if (!rtis::all_finite(mic_xyz, 3 * static_cast<size_t>(n_mics)) ||
        !rtis::all_finite(directions, 3 * static_cast<size_t>(n_dirs)) ||
        (gain && !rtis::all_finite(gain, n_mics)) || (delay_s && !rtis::all_finite(delay_s, n_mics)))
        return fail(RTIS_ERR_NONFINITE, "rtis_fd_gemm_create: non-finite geometry, gain or delay");
    for (int k = 0; k < n_bins; ++k)
        if (!std::isfinite(freqs_hz[k])) return fail(RTIS_ERR_NONFINITE, "rtis_fd_gemm_create: non-finite frequency");

    rtis_fd_gemm* plan = new (std::nothrow) rtis_fd_gemm();
    if (!plan) return fail(RTIS_ERR_OOM, "rtis_fd_gemm_create: host allocation failed");
    rtis::FdGemmPlan& g = plan->g;
    g.M = n_mics;
    g.D = n_dirs;
    g.K = n_bins;
    g.T = n_frames;
    g.precision = precision;
    {
        int dev = 0;
        cudaGetDevice(&dev);
        if (cudaDeviceGetAttribute(&g.n_sm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) g.n_sm = 1;
        cudaGetLastError();
    }
    // tau_dm in FP64, carried to the device as an unevaluated float pair hi + lo
    std::vector<float2> tau(static_cast<size_t>(n_dirs) * n_mics), fr(n_bins);
    for (int d = 0; d < n_dirs; ++d)
        for (int m = 0; m < n_mics; ++m) {
            const double dot = static_cast<double>(mic_xyz[3 * m]) * directions[3 * d] +
                               static_cast<double>(mic_xyz[3 * m + 1]) * directions[3 * d + 1] +
                               static_cast<double>(mic_xyz[3 * m + 2]) * directions[3 * d + 2];
            const double t = (delay_s ? static_cast<double>(delay_s[m]) : 0.0) - dot / c;
            const float hi = static_cast<float>(t);
            tau[static_cast<size_t>(d) * n_mics + m] = make_float2(hi, static_cast<float>(t - hi));
        }
    for (int k = 0; k < n_bins; ++k) {
        const float hi = static_cast<float>(freqs_hz[k]);
        fr[k] = make_float2(hi, static_cast<float>(freqs_hz[k] - hi));
    }
    std::vector<float> gv(n_mics, 1.0f);
    if (gain)
        for (int m = 0; m < n_mics; ++m) gv[m] = gain[m];
    size_t total = 0;
    cudaError_t e = rtis::dev_alloc(&g.d_tau, tau.size(), &total);
    if (e == cudaSuccess) e = rtis::dev_alloc(&g.d_freq, fr.size(), &total);
    if (e == cudaSuccess) e = rtis::dev_alloc(&g.d_gain, gv.size(), &total);
    if (e == cudaSuccess) e = rtis::dev_alloc(&g.d_scale, static_cast<size_t>(n_mics), &total);
    if (e == cudaSuccess) e = rtis::dev_alloc(&g.d_status, 1, &total);
    if (e == cudaSuccess) e = cudaMemcpy(g.d_tau, tau.data(), tau.size() * sizeof(float2), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(g.d_freq, fr.data(), fr.size() * sizeof(float2), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(g.d_gain, gv.data(), gv.size() * sizeof(float), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(g.d_status, 0, sizeof(unsigned));
    if (e != cudaSuccess) {
        rtis_fd_gemm_destroy(plan);
        cudaGetLastError();
        return (e == cudaErrorMemoryAllocation) ? fail(RTIS_ERR_OOM, "rtis_fd_gemm_create: cudaMalloc failed")
                                                : cuda_fail(e, "rtis_fd_gemm_create: upload");
    }
    *out = plan;
    return RTIS_OK;
}

rtis_status rtis_fd_gemm_run(rtis_fd_gemm* plan, const float* d_X, float* d_Y, void* stream) {
    if (rtis::fault_mode() == rtis::kFaultLaunch) return rtis::fail(RTIS_ERR_CUDA, "rtis_fd_gemm_run: injected launch failure");
    if (!plan || !d_X || !d_Y) return fail(RTIS_ERR_INVALID_ARG, "rtis_fd_gemm_run: NULL argument");
    if (!rtis::aligned(d_X, 8) || !rtis::aligned(d_Y, 16))
        return fail(RTIS_ERR_INVALID_ARG, "rtis_fd_gemm_run: d_X must be 8-byte and d_Y 16-byte aligned");
    rtis::FdGemmPlan& g = plan->g;
    CUtensorMap ymap;
    const CUtensorMap* ym = nullptr;
    if (g.T % 2 == 0 && g.T >= 16) {  // rows of 2T floats: 16-byte strides, at least one 128-byte box
        std::string err;
        if (!rtis::fd_gemm_encode_ymap(g, reinterpret_cast<float2*>(d_Y), &ymap, &err))
            return fail(RTIS_ERR_CUDA, "rtis_fd_gemm_run: " + err);
        ym = &ymap;
    }
    cudaError_t e = rtis::launch_fd_gemm(g, reinterpret_cast<const float2*>(d_X), reinterpret_cast<float2*>(d_Y), ym,
                                         static_cast<cudaStream_t>(stream));
    return e == cudaSuccess ? RTIS_OK : cuda_fail(e, "rtis_fd_gemm_run: launch");
}

void rtis_fd_gemm_destroy(rtis_fd_gemm* plan) {
    if (!plan) return;
    cudaDeviceSynchronize();
    rtis::FdGemmPlan& g = plan->g;
    void* bufs[] = {g.d_tau, g.d_freq, g.d_gain, g.d_scale, g.d_status};
    for (void* b : bufs)
        if (b) cudaFree(b);
    delete plan;
}

rtis_status rtis_set_calibration(rtis_plan* plan, const float* d_mic_xyz, const float* d_gain, const float* d_delay_s,
                                 void* stream) {
    if (rtis::fault_mode() == rtis::kFaultLaunch) return rtis::fail(RTIS_ERR_CUDA, "rtis_set_calibration: injected launch failure");
    if (!plan) return fail(RTIS_ERR_INVALID_ARG, "rtis_set_calibration: NULL plan");
    Plan& p = plan->p;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    cudaError_t e = cudaSuccess;
    if (d_mic_xyz) e = cudaMemcpyAsync(p.d_mic, d_mic_xyz, 3 * p.M * sizeof(float), cudaMemcpyDeviceToDevice, st);
    if (e == cudaSuccess && d_gain) e = cudaMemcpyAsync(p.d_gain, d_gain, p.M * sizeof(float), cudaMemcpyDeviceToDevice, st);
    if (e == cudaSuccess && d_delay_s)
        e = cudaMemcpyAsync(p.d_delay, d_delay_s, p.M * sizeof(float), cudaMemcpyDeviceToDevice, st);
    if (e != cudaSuccess) return cuda_fail(e, "rtis_set_calibration: copy");
    p.table_dirty = true;
    rtis::trace_call(p, st);
    return ensure_table(p, st);
}

rtis_status rtis_backward(rtis_plan* plan, const int16_t* d_in, const float* d_grad_out, float* d_grad_xyz,
                          float* d_grad_gain, float* d_grad_delay, void* stream) {
    if (rtis::fault_mode() == rtis::kFaultLaunch) return rtis::fail(RTIS_ERR_CUDA, "rtis_backward: injected launch failure");
    if (!plan || !d_in || !d_grad_out) return fail(RTIS_ERR_INVALID_ARG, "rtis_backward: NULL argument");
    if (!d_grad_xyz && !d_grad_gain && !d_grad_delay)
        return fail(RTIS_ERR_INVALID_ARG, "rtis_backward: no gradient requested");
    if (!rtis::aligned(d_in, 8) || !rtis::aligned(d_grad_out, 4))
        return fail(RTIS_ERR_INVALID_ARG, "rtis_backward: misaligned pointer");
    Plan& p = plan->p;
    // every sample a tile owns must lie inside the window the tile beamforms
    const int half = (p.lpf_len - 1) / 2;
    const int n_tiles = (p.n_out + p.td_bins_per_tile - 1) / p.td_bins_per_tile;
    const int last_start = p.R * (n_tiles - 1) * p.td_bins_per_tile - half;
    if (p.R * p.td_bins_per_tile + half > rtis::kTdWarpSamples || p.N > last_start + rtis::kTdWarpSamples)
        return fail(RTIS_ERR_UNSUPPORTED, "rtis_backward: decimation too coarse for the beamformer tile");
    if (rtis::adj_smem_bytes(p) > 227 * 1024) return fail(RTIS_ERR_UNSUPPORTED, "rtis_backward: halo too large");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    rtis::trace_call(p, st);
    rtis_status s = ensure_table(p, st);
    if (s != RTIS_OK) return s;
    cudaError_t e = RTIS_TRACED(p, st, RTIS_KERNEL_MF_FORWARD, rtis::launch_mf_forward(p, d_in, st));  // recompute the MF
    if (e == cudaSuccess) e = RTIS_TRACED(p, st, RTIS_KERNEL_MF_INVERSE, rtis::launch_mf_inverse(p, p.d_a, nullptr, st));
    if (e == cudaSuccess)
        e = RTIS_TRACED(p, st, RTIS_KERNEL_ADJOINT,
                        rtis::launch_td_adjoint(p, d_grad_out, d_grad_xyz, d_grad_gain, d_grad_delay, st));
    return e == cudaSuccess ? RTIS_OK : cuda_fail(e, "rtis_backward: launch");
}

rtis_status rtis_loss_l2(rtis_plan* plan, const float* d_E, const float* d_E_ref, float* d_grad_out, float* d_loss,
                         void* stream) {
    if (rtis::fault_mode() == rtis::kFaultLaunch) return rtis::fail(RTIS_ERR_CUDA, "rtis_loss_l2: injected launch failure");
    if (!plan || !d_E || !d_E_ref || !d_loss) return fail(RTIS_ERR_INVALID_ARG, "rtis_loss_l2: NULL argument");
    cudaError_t e = rtis::launch_l2_loss(plan->p, d_E, d_E_ref, d_grad_out, d_loss, static_cast<cudaStream_t>(stream));
    return e == cudaSuccess ? RTIS_OK : cuda_fail(e, "rtis_loss_l2: launch");
}

rtis_status rtis_plan_set_tracing(rtis_plan* plan, int enable) {
    if (!plan) return fail(RTIS_ERR_INVALID_ARG, "rtis_plan_set_tracing: NULL plan");
    Plan& p = plan->p;
    if (!enable) {
        cudaDeviceSynchronize();  // no recorded event is still pending when it is destroyed
        rtis::destroy_trace_events(p);
        return RTIS_OK;
    }
    if (p.trace_on) return RTIS_OK;
    for (cudaEvent_t& ev : p.trace_ev) {
        const cudaError_t e = cudaEventCreate(&ev);
        if (e != cudaSuccess) {
            rtis::destroy_trace_events(p);
            return cuda_fail(e, "rtis_plan_set_tracing: cudaEventCreate");
        }
    }
    p.trace_on = true;
    p.trace_n = 0;
    return RTIS_OK;
}

rtis_status rtis_plan_get_trace(rtis_plan* plan, rtis_trace_entry* out, int capacity, int* n_out) {
    if (!plan) return fail(RTIS_ERR_INVALID_ARG, "rtis_plan_get_trace: NULL plan");
    Plan& p = plan->p;
    if (!p.trace_on) return fail(RTIS_ERR_INVALID_ARG, "rtis_plan_get_trace: tracing is off");
    if (capacity > 0 && !out) return fail(RTIS_ERR_INVALID_ARG, "rtis_plan_get_trace: NULL output");
    if (p.trace_n > 0) {
        const cudaError_t e = cudaEventSynchronize(p.trace_ev[2 * p.trace_n - 1]);
        if (e != cudaSuccess) return cuda_fail(e, "rtis_plan_get_trace: cudaEventSynchronize");
    }
    for (int i = 0; i < p.trace_n && i < capacity; ++i) {
        float ms = 0.f;
        const cudaError_t e = cudaEventElapsedTime(&ms, p.trace_ev[2 * i], p.trace_ev[2 * i + 1]);
        if (e != cudaSuccess) return cuda_fail(e, "rtis_plan_get_trace: cudaEventElapsedTime");
        out[i].kernel = p.trace_kind[i];
        out[i].index = i;
        out[i].ms = ms;
    }
    if (n_out) *n_out = p.trace_n;
    return RTIS_OK;
}

rtis_status rtis_plan_sync(rtis_plan* plan, unsigned* bits_out) {
    if (!plan) return fail(RTIS_ERR_INVALID_ARG, "rtis_plan_sync: NULL plan");
    Plan& p = plan->p;
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return cuda_fail(e, "rtis_plan_sync: synchronize");
    unsigned bits = 0;
    e = cudaMemcpy(&bits, p.d_status, sizeof(unsigned), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemset(p.d_status, 0, sizeof(unsigned));
    if (e != cudaSuccess) return cuda_fail(e, "rtis_plan_sync: status word");
    if (bits_out) *bits_out = bits;
    if (bits & RTIS_DEV_TIMEOUT) return fail(RTIS_ERR_TIMEOUT, "rtis_plan_sync: a bounded device wait ran out");
    if (bits & RTIS_DEV_DELAY_RANGE)
        return fail(RTIS_ERR_DEVICE, "rtis_plan_sync: a steering delay exceeded the staged halo");
    if (bits & RTIS_DEV_NONFINITE)
        return fail(RTIS_ERR_NONFINITE, "rtis_plan_sync: an energyscape value was NaN or infinite");
    return RTIS_OK;
}

}  // extern "C"
