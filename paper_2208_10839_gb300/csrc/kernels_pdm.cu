// PDM front end.  The eRTIS microphones record through a 1-bit sigma-delta
// ADC (Sec. 2); the processing unpacks the bits and demodulates them with a
// low-pass filter before the matched filter (Sec. 4.3).  Here:
//
//   b_m[k]  = +1 / -1 for bit m of word k = 1 / 0 (0 outside [0, K))
//   x_m[n]  = sat16( (sum_j g[j] b_m[D n + j - c] + r) >> shift ),  c = (L - 1) / 2,
//             r = 2^(shift-1) for shift > 0 (halves round up), else 0
//
// The taps g are integers, so the sum is exact and the result is the same
// integer on every device.  One CTA takes kPdmOut output samples of every mic:
// the (kPdmOut - 1) D + L words they read carry all 32 mics, so they are
// staged once in shared memory (0 outside the record, with a validity mask).
// Lane = mic: every lane of a warp reads the same word (a shared-memory
// broadcast) and takes its own bit; warp w computes outputs w, w + 8, ... of
// the tile.  The results go through shared memory, so that each int16 row
// segment is written as one contiguous store.
#include <algorithm>
#include <cstring>
#include <vector>

#include "rtis_internal.h"

namespace rtis {
namespace {

constexpr int kPdmOut = 16;      // output samples per CTA (1024 CTAs at 16384 samples)
constexpr int kPdmThreads = 256;

struct PdmArgs {
    const uint32_t* words;
    int16_t* x;
    long long K;                 // words in the record
    int M, N, D, L, c, shift;
    int32_t g[kPdmMaxTaps];
};

__global__ void __launch_bounds__(kPdmThreads) pdm_demod_kernel(const __grid_constant__ PdmArgs A) {
    extern __shared__ uint32_t sw[];  // [span] words, then [span] validity masks
    const int span = (kPdmOut - 1) * A.D + A.L;
    uint32_t* sv = sw + span;
    __shared__ int32_t gs[kPdmMaxTaps];
    __shared__ int16_t xs[32][kPdmOut + 2];  // [mic][output], rows padded
    const int n0 = blockIdx.x * kPdmOut;
    const long long k0 = static_cast<long long>(n0) * A.D - A.c;  // word of tap 0 for output n0
    for (int i = threadIdx.x; i < span; i += kPdmThreads) {
        const long long k = k0 + i;
        const bool ok = k >= 0 && k < A.K;
        sw[i] = ok ? __ldg(A.words + k) : 0u;
        sv[i] = ok ? 0xffffffffu : 0u;
    }
    for (int j = threadIdx.x; j < A.L; j += kPdmThreads) gs[j] = A.g[j];
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int32_t rnd = A.shift > 0 ? (1 << (A.shift - 1)) : 0;
    for (int t = warp; t < kPdmOut; t += kPdmThreads / 32) {
        const uint32_t* w = sw + t * A.D;
        const uint32_t* v = sv + t * A.D;
        int32_t acc = 0;
#pragma unroll 4
        for (int j = 0; j < A.L; ++j) {
            // +1 / -1 from this lane's bit, 0 outside the record (same word for the whole warp)
            const int32_t b = (static_cast<int32_t>((w[j] >> lane) & 1u) * 2 - 1) & static_cast<int32_t>(v[j]);
            acc += gs[j] * b;
        }
        const int32_t y = (acc + rnd) >> A.shift;
        xs[lane][t] = static_cast<int16_t>(max(-32768, min(32767, y)));
    }
    __syncthreads();
    // rows out: warp w writes mics w, w + 8, ...; a lane two consecutive samples
    for (int m = warp; m < A.M; m += kPdmThreads / 32) {
        for (int t = 2 * lane; t < kPdmOut; t += 64) {  // kPdmOut <= 64: one pass
            const int n = n0 + t;
            int16_t* dst = A.x + static_cast<size_t>(m) * A.N + n;
            if (n + 1 < A.N && ((reinterpret_cast<uintptr_t>(dst) & 3) == 0)) {
                *reinterpret_cast<short2*>(dst) = make_short2(xs[m][t], xs[m][t + 1]);
            } else {
                if (n < A.N) dst[0] = xs[m][t];
                if (n + 1 < A.N) dst[1] = xs[m][t + 1];
            }
        }
    }
}

}  // namespace

cudaError_t launch_pdm_demod(const uint32_t* d_words, long long n_words, int n_mics, int n_samples, int decim,
                             const int32_t* taps, int n_taps, int shift, int16_t* d_x, cudaStream_t st) {
    PdmArgs A;
    std::memset(&A, 0, sizeof(A));
    A.words = d_words;
    A.x = d_x;
    A.K = n_words;
    A.M = n_mics;
    A.N = n_samples;
    A.D = decim;
    A.L = n_taps;
    A.c = (n_taps - 1) / 2;
    A.shift = shift;
    std::memcpy(A.g, taps, sizeof(int32_t) * n_taps);
    const size_t smem = static_cast<size_t>(2) * ((kPdmOut - 1) * decim + n_taps) * sizeof(uint32_t);
    cudaError_t e = cudaFuncSetAttribute(pdm_demod_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         static_cast<int>(smem));
    if (e != cudaSuccess) return e;
    const int grid = (n_samples + kPdmOut - 1) / kPdmOut;
    pdm_demod_kernel<<<grid, kPdmThreads, smem, st>>>(A);
    return cudaGetLastError();
}

}  // namespace rtis

extern "C" {

rtis_status rtis_pdm_demodulate(const uint32_t* d_words, long long n_words, int n_mics, int n_samples, int decim,
                                const int32_t* taps, int n_taps, int shift, int16_t* d_x, void* stream) {
    if (rtis::fault_mode() == rtis::kFaultLaunch)
        return rtis::fail(RTIS_ERR_CUDA, "rtis_pdm_demodulate: injected launch failure");
    if (!d_x || (!d_words && n_words > 0)) return rtis::fail(RTIS_ERR_INVALID_ARG, "rtis_pdm_demodulate: NULL argument");
    if (reinterpret_cast<uintptr_t>(d_words) % 4 != 0 || reinterpret_cast<uintptr_t>(d_x) % 2 != 0)
        return rtis::fail(RTIS_ERR_INVALID_ARG, "rtis_pdm_demodulate: d_words must be 4-byte and d_x 2-byte aligned");
    if (n_mics < 1 || n_mics > 32) return rtis::fail(RTIS_ERR_INVALID_ARG, "rtis_pdm_demodulate: n_mics must be in [1, 32]");
    if (n_samples < 1 || n_words < 0) return rtis::fail(RTIS_ERR_INVALID_ARG, "rtis_pdm_demodulate: empty output or negative n_words");
    if (decim < 1 || decim > 64) return rtis::fail(RTIS_ERR_INVALID_ARG, "rtis_pdm_demodulate: decim must be in [1, 64]");
    if (shift < 0 || shift > 30) return rtis::fail(RTIS_ERR_INVALID_ARG, "rtis_pdm_demodulate: shift must be in [0, 30]");
    int32_t g[rtis::kPdmMaxTaps];
    if (taps == nullptr) {  // order-4 CIC kernel: the length-D boxcar convolved with itself 4 times
        n_taps = 4 * (decim - 1) + 1;
        std::vector<long long> h(1, 1);
        for (int r = 0; r < 4; ++r) {
            std::vector<long long> nh(h.size() + decim - 1, 0);
            for (size_t i = 0; i < h.size(); ++i)
                for (int k = 0; k < decim; ++k) nh[i + k] += h[i];
            h.swap(nh);
        }
        for (int j = 0; j < n_taps; ++j) g[j] = static_cast<int32_t>(h[j]);
    } else {
        if (n_taps < 1 || n_taps > rtis::kPdmMaxTaps)
            return rtis::fail(RTIS_ERR_INVALID_ARG, "rtis_pdm_demodulate: n_taps must be in [1, 256]");
        for (int j = 0; j < n_taps; ++j) g[j] = taps[j];
    }
    long long sum_abs = 0;
    for (int j = 0; j < n_taps; ++j) sum_abs += g[j] < 0 ? -static_cast<long long>(g[j]) : g[j];
    if (sum_abs > (1ll << 30))
        return rtis::fail(RTIS_ERR_INVALID_ARG, "rtis_pdm_demodulate: sum |taps| above 2^30 (the int32 sum could overflow)");
    cudaError_t e = rtis::launch_pdm_demod(d_words, n_words, n_mics, n_samples, decim, g, n_taps, shift, d_x,
                                           static_cast<cudaStream_t>(stream));
    return e == cudaSuccess ? RTIS_OK : rtis::cuda_fail(e, "rtis_pdm_demodulate: launch");
}

}  // extern "C"
