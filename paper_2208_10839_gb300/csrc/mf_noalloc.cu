// Matched filter that allocates nothing: the same FFT kernels as
// rtis_matched_filter, with every table and workspace they need placed in
// one statically sized device array instead of a plan's cudaMalloc'd
// buffers.  For callers that are not allowed to allocate device memory.
#include <cmath>
#include <mutex>
#include <string>

#include <cudaTypedefs.h>

#include "rtis_internal.h"

// Scratch shared by every call on a device: twiddles [F], chirp spectrum
// [Kb] and the half-size spectra [M][2][F/4], all complex64.  Every GPU that
// loads the library holds this array until the process exits.
static __device__ __align__(256) unsigned char g_mf_scratch[RTIS_NOALLOC_SCRATCH_BYTES];

namespace rtis {
namespace {

constexpr int kMaxDevices = 64;
std::mutex g_addr_mutex;
void* g_addr[kMaxDevices] = {};
unsigned long long g_ctx[kMaxDevices] = {};

// tw[j] = exp(-2 pi i j / F), from an FP64 sincospi of the exact ratio 2j/F
__global__ void noalloc_twiddles(float2* __restrict__ tw, int F) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= F) return;
    double s, c;
    sincospi(2.0 * static_cast<double>(j) / static_cast<double>(F), &s, &c);
    tw[j] = make_float2(static_cast<float>(c), static_cast<float>(-s));
}

// C[k'] = 2 conj(S[k]) / F with S[k] = sum_l s[l] exp(-2 pi i k l / F), k = k_lo + k':
// one warp per bin, the lanes striding over l, FP64 sums reduced across the warp
constexpr int kChirpWarps = 8;
__global__ void noalloc_chirp_spectrum(const float* __restrict__ chirp, int L, const float2* __restrict__ tw,
                                       int F, int k_lo, int Kb, float2* __restrict__ C) {
    const int kp = blockIdx.x * kChirpWarps + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (kp >= Kb) return;  // warp-uniform
    const unsigned k = static_cast<unsigned>(k_lo + kp);
    const unsigned mask = static_cast<unsigned>(F - 1);
    double re = 0.0, im = 0.0;
    for (int l = lane; l < L; l += 32) {
        const float2 w = tw[(k * static_cast<unsigned>(l)) & mask];
        const double s = chirp[l];
        re += s * w.x;
        im += s * w.y;
    }
    for (int o = 16; o > 0; o >>= 1) {
        re += __shfl_xor_sync(0xffffffffu, re, o);
        im += __shfl_xor_sync(0xffffffffu, im, o);
    }
    if (lane == 0) C[kp] = make_float2(static_cast<float>(2.0 * re / F), static_cast<float>(-2.0 * im / F));
}

// The unique id of the calling thread's current context (0 when there is none yet, or
// when the driver cannot say).  A cudaDeviceReset ends the device's primary context;
// the next one has a new id, and the module holding g_mf_scratch may load elsewhere.
unsigned long long current_context_id() {
    static PFN_cuCtxGetCurrent_v4000 get_current = nullptr;
    static PFN_cuCtxGetId_v12000 get_id = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* fn = nullptr;
        cudaDriverEntryPointQueryResult q{};
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &fn, 4000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_current = reinterpret_cast<PFN_cuCtxGetCurrent_v4000>(fn);
        fn = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &fn, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_id = reinterpret_cast<PFN_cuCtxGetId_v12000>(fn);
    });
    CUcontext ctx = nullptr;
    unsigned long long id = 0;
    if (get_current == nullptr || get_id == nullptr || get_current(&ctx) != CUDA_SUCCESS || ctx == nullptr) return 0;
    if (get_id(ctx, &id) != CUDA_SUCCESS) return 0;
    return id;
}

// The device address of g_mf_scratch on the current device: looked up with
// cudaGetSymbolAddress (that device current; a host-side lookup that allocates nothing)
// once per device and context, then cached.  A call that finds a different context
// than the cached one (the device was reset in between) looks the address up again.
rtis_status scratch_address(void** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "rtis_matched_filter_noalloc: cudaGetDevice");
    if (dev < 0 || dev >= kMaxDevices) return fail(RTIS_ERR_UNSUPPORTED, "rtis_matched_filter_noalloc: device index");
    std::lock_guard<std::mutex> lock(g_addr_mutex);
    const unsigned long long ctx = current_context_id();
    if (g_addr[dev] == nullptr || ctx == 0 || ctx != g_ctx[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_mf_scratch);
        if (e != cudaSuccess || p == nullptr) {
            g_addr[dev] = nullptr;
            return cuda_fail(e, "rtis_matched_filter_noalloc: cudaGetSymbolAddress of the static scratch");
        }
        g_addr[dev] = p;
        g_ctx[dev] = current_context_id();  // the lookup made the primary context current if it was not
    }
    *out = g_addr[dev];
    return RTIS_OK;
}

}  // namespace
}  // namespace rtis

extern "C" rtis_status rtis_matched_filter_noalloc(const int16_t* d_in, int n_mics, int n_samples,
                                                   const float* d_chirp, int chirp_len, double fs,
                                                   double band_lo_hz, double band_hi_hz, float* d_a,
                                                   float* d_A, void* stream) {
    if (rtis::fault_mode() == rtis::kFaultLaunch) return rtis::fail(RTIS_ERR_CUDA, "rtis_matched_filter_noalloc: injected launch failure");
    using namespace rtis;
    if (!d_in || !d_chirp) return fail(RTIS_ERR_INVALID_ARG, "rtis_matched_filter_noalloc: NULL input");
    if (!d_a && !d_A) return fail(RTIS_ERR_INVALID_ARG, "rtis_matched_filter_noalloc: no output requested");
    if (reinterpret_cast<uintptr_t>(d_in) % 8 != 0 || reinterpret_cast<uintptr_t>(d_a) % 8 != 0 ||
        reinterpret_cast<uintptr_t>(d_A) % 8 != 0 || reinterpret_cast<uintptr_t>(d_chirp) % 4 != 0)
        return fail(RTIS_ERR_INVALID_ARG, "rtis_matched_filter_noalloc: misaligned pointer");
    if (n_mics < 1 || chirp_len < 1 || n_samples < 64 || n_samples % 4 != 0)
        return fail(RTIS_ERR_INVALID_ARG,
                    "rtis_matched_filter_noalloc: need n_mics >= 1, chirp_len >= 1, n_samples >= 64 and a multiple of 4");
    if (!(fs > 0.0) || !(band_lo_hz >= 0.0) || !(band_hi_hz > band_lo_hz))
        return fail(RTIS_ERR_INVALID_ARG, "rtis_matched_filter_noalloc: need fs > 0 and 0 <= band_lo < band_hi");
    int64_t F = 1;
    while (F < static_cast<int64_t>(n_samples) + chirp_len - 1) F *= 2;
    if (F < 256 || F > 65536)
        return fail(RTIS_ERR_UNSUPPORTED, "rtis_matched_filter_noalloc: FFT length outside [256, 65536]");
    const int k_lo = static_cast<int>(std::ceil(band_lo_hz * F / fs));
    const int k_hi = static_cast<int>(std::floor(band_hi_hz * F / fs));
    if (k_hi < k_lo) return fail(RTIS_ERR_INVALID_ARG, "rtis_matched_filter_noalloc: band holds no FFT bin");
    if (k_hi >= F / 4) return fail(RTIS_ERR_UNSUPPORTED, "rtis_matched_filter_noalloc: band must lie below fs/4");
    const int Kb = k_hi - k_lo + 1;
    const int P = static_cast<int>(F / 4);
    const size_t tw_bytes = static_cast<size_t>(F) * sizeof(float2);
    const size_t c_bytes = ((static_cast<size_t>(Kb) * sizeof(float2) + 255) / 256) * 256;
    const size_t z_bytes = static_cast<size_t>(n_mics) * 2 * P * sizeof(float2);
    if (tw_bytes + c_bytes + z_bytes > static_cast<size_t>(RTIS_NOALLOC_SCRATCH_BYTES))
        return fail(RTIS_ERR_INVALID_ARG,
                    "rtis_matched_filter_noalloc: needs " + std::to_string(tw_bytes + c_bytes + z_bytes) +
                        " bytes of scratch, more than the static maximum of " +
                        std::to_string(static_cast<long long>(RTIS_NOALLOC_SCRATCH_BYTES)) +
                        " (reduce n_mics or n_samples)");

    void* base = nullptr;
    rtis_status s = scratch_address(&base);
    if (s != RTIS_OK) return s;
    unsigned char* b = static_cast<unsigned char*>(base);

    // a throw-away plan view: sizes plus pointers into the static scratch
    Plan p;
    p.M = n_mics;
    p.N = n_samples;
    p.L = chirp_len;
    p.F = static_cast<int>(F);
    p.P = P;
    p.logP = 0;
    while ((1 << p.logP) < P) ++p.logP;
    p.k_lo = k_lo;
    p.k_hi = k_hi;
    p.Kb = Kb;
    p.fs = fs;
    p.d_tw = reinterpret_cast<float2*>(b);
    p.d_C = reinterpret_cast<float2*>(b + tw_bytes);
    p.d_Z = reinterpret_cast<float2*>(b + tw_bytes + c_bytes);

    cudaStream_t st = static_cast<cudaStream_t>(stream);
    noalloc_twiddles<<<static_cast<int>((F + 255) / 256), 256, 0, st>>>(p.d_tw, p.F);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "rtis_matched_filter_noalloc: twiddle launch");
    noalloc_chirp_spectrum<<<(Kb + kChirpWarps - 1) / kChirpWarps, 32 * kChirpWarps, 0, st>>>(
        d_chirp, chirp_len, p.d_tw, p.F, k_lo, Kb, p.d_C);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "rtis_matched_filter_noalloc: chirp spectrum launch");
    e = launch_mf_forward(p, d_in, st);
    if (e != cudaSuccess) return cuda_fail(e, "rtis_matched_filter_noalloc: forward launch");
    e = launch_mf_inverse(p, reinterpret_cast<float2*>(d_a), reinterpret_cast<float2*>(d_A), st);
    if (e != cudaSuccess) return cuda_fail(e, "rtis_matched_filter_noalloc: inverse launch");
    return RTIS_OK;
}
