// A straightforward GPU form of the time-domain chain, built the way the
// paper's GPU implementation is described (Sec. 4.3: filters as cuFFT
// convolutions, separate kernels for the multiply, the beamforming and the
// envelope, intermediates in device memory).  It exists as a comparison
// point for the fused kernels: same definitions, same plan tables, same
// results to FP32 rounding.
//
//   1. int16 -> float, zero-padded to F, per channel
//   2. cuFFT R2C, F points, batch M
//   3. A[k] = X[k] C[k - k_lo] on the band, 0 elsewhere (C = 2 conj(S)/F)
//   4. cuFFT C2C inverse, F points, batch M: a_m[n], n < N
//   5. one thread per (direction, sample): b = sum_m sum_q W[d][m][q] a_m[n + J + q - 1],
//      |b| written to a [D][N] envelope array
//   6. one thread per (direction, output bin): E = sum_j h[j] |b|[R i + j - half]
#include <cufft.h>

#include <string>

#include "rtis_internal.h"

struct rtis_baseline {
    const rtis_plan* plan = nullptr;
    cufftHandle fwd = 0, inv = 0;
    bool have_fwd = false, have_inv = false;
    float* d_xf = nullptr;        // [M][F] real input
    cufftComplex* d_X = nullptr;  // [M][F/2 + 1]
    cufftComplex* d_S = nullptr;  // [M][F] band spectrum, then a (in place)
    float* d_env = nullptr;       // [D][N]
};

namespace {

using rtis::Plan;
using rtis::cuda_fail;
using rtis::fail;

__global__ void bl_to_float(const int16_t* __restrict__ x, int M, int N, int F, float* __restrict__ xf) {
    const size_t i = static_cast<size_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= static_cast<size_t>(M) * F) return;
    const int m = static_cast<int>(i / F), n = static_cast<int>(i % F);
    xf[i] = n < N ? x[static_cast<size_t>(m) * N + n] * (1.0f / 32768.0f) : 0.f;
}

__global__ void bl_band(const cufftComplex* __restrict__ X, const float2* __restrict__ C, int M, int F, int k_lo,
                        int k_hi, cufftComplex* __restrict__ S) {
    const size_t i = static_cast<size_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= static_cast<size_t>(M) * F) return;
    const int m = static_cast<int>(i / F), k = static_cast<int>(i % F);
    cufftComplex v = make_cuComplex(0.f, 0.f);
    if (k >= k_lo && k <= k_hi) {
        const cufftComplex x = X[static_cast<size_t>(m) * (F / 2 + 1) + k];
        const float2 c = C[k - k_lo];
        v = make_cuComplex(x.x * c.x - x.y * c.y, x.x * c.y + x.y * c.x);
    }
    S[i] = v;
}

__global__ void bl_das(const cufftComplex* __restrict__ a, int F, const int* __restrict__ shift,
                       const float4* __restrict__ wt, int M, int N, float* __restrict__ env) {
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    const int d = blockIdx.y;
    if (n >= N) return;
    float br = 0.f, bi = 0.f;
    for (int m = 0; m < M; ++m) {
        const int J = shift[static_cast<size_t>(d) * M + m];
        const float4 w = wt[static_cast<size_t>(d) * M + m];
        const float ww[4] = {w.x, w.y, w.z, w.w};
        const cufftComplex* am = a + static_cast<size_t>(m) * F;
        for (int q = 0; q < 4; ++q) {
            const int idx = n + J + q - 1;
            if (idx >= 0 && idx < N) {
                br = fmaf(ww[q], am[idx].x, br);
                bi = fmaf(ww[q], am[idx].y, bi);
            }
        }
    }
    env[static_cast<size_t>(d) * N + n] = sqrtf(br * br + bi * bi);
}

__global__ void bl_lpf(const float* __restrict__ env, const float* __restrict__ h, int L, int R, int N, int n_out,
                       float* __restrict__ E) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int d = blockIdx.y;
    if (i >= n_out) return;
    const int half = (L - 1) / 2;
    const float* e = env + static_cast<size_t>(d) * N;
    float s = 0.f;
    for (int j = 0; j < L; ++j) {
        const int n = R * i + j - half;
        if (n >= 0 && n < N) s = fmaf(h[j], e[n], s);
    }
    E[static_cast<size_t>(d) * n_out + i] = s;
}

void destroy(rtis_baseline* b) {
    if (!b) return;
    if (b->have_fwd) cufftDestroy(b->fwd);
    if (b->have_inv) cufftDestroy(b->inv);
    void* bufs[] = {b->d_xf, b->d_X, b->d_S, b->d_env};
    for (void* p : bufs)
        if (p) cudaFree(p);
    delete b;
}

}  // namespace

extern "C" {

rtis_status rtis_baseline_create(rtis_baseline** out, const rtis_plan* plan) {
    if (rtis::fault_mode() == rtis::kFaultAlloc)
        return fail(RTIS_ERR_OOM, "rtis_baseline_create: injected allocation failure");
    if (!out || !plan) return fail(RTIS_ERR_INVALID_ARG, "rtis_baseline_create: NULL argument");
    *out = nullptr;
    const Plan& p = plan->p;
    rtis_baseline* b = new (std::nothrow) rtis_baseline();
    if (!b) return fail(RTIS_ERR_OOM, "rtis_baseline_create: host allocation failed");
    b->plan = plan;
    const size_t MF = static_cast<size_t>(p.M) * p.F;
    cudaError_t e = cudaMalloc(&b->d_xf, MF * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&b->d_X, static_cast<size_t>(p.M) * (p.F / 2 + 1) * sizeof(cufftComplex));
    if (e == cudaSuccess) e = cudaMalloc(&b->d_S, MF * sizeof(cufftComplex));
    if (e == cudaSuccess) e = cudaMalloc(&b->d_env, static_cast<size_t>(p.D) * p.N * sizeof(float));
    if (e != cudaSuccess) {
        destroy(b);
        cudaGetLastError();
        return fail(RTIS_ERR_OOM, "rtis_baseline_create: cudaMalloc failed");
    }
    int n[1] = {p.F};
    if (cufftPlanMany(&b->fwd, 1, n, nullptr, 1, p.F, nullptr, 1, p.F / 2 + 1, CUFFT_R2C, p.M) != CUFFT_SUCCESS) {
        destroy(b);
        return fail(RTIS_ERR_CUDA, "rtis_baseline_create: cufftPlanMany (forward)");
    }
    b->have_fwd = true;
    if (cufftPlanMany(&b->inv, 1, n, nullptr, 1, p.F, nullptr, 1, p.F, CUFFT_C2C, p.M) != CUFFT_SUCCESS) {
        destroy(b);
        return fail(RTIS_ERR_CUDA, "rtis_baseline_create: cufftPlanMany (inverse)");
    }
    b->have_inv = true;
    *out = b;
    return RTIS_OK;
}

rtis_status rtis_baseline_process(rtis_baseline* b, const int16_t* d_in, float* d_out, void* stream) {
    if (rtis::fault_mode() == rtis::kFaultLaunch)
        return fail(RTIS_ERR_CUDA, "rtis_baseline_process: injected launch failure");
    if (!b || !d_in || !d_out) return fail(RTIS_ERR_INVALID_ARG, "rtis_baseline_process: NULL argument");
    const Plan& p = b->plan->p;
    if (p.table_dirty)
        return fail(RTIS_ERR_INVALID_ARG, "rtis_baseline_process: run the plan once first (steering table)");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const size_t MF = static_cast<size_t>(p.M) * p.F;
    const int nt = 256;
    const unsigned g1 = static_cast<unsigned>((MF + nt - 1) / nt);
    bl_to_float<<<g1, nt, 0, st>>>(d_in, p.M, p.N, p.F, b->d_xf);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "rtis_baseline_process: convert");
    if (cufftSetStream(b->fwd, st) != CUFFT_SUCCESS || cufftSetStream(b->inv, st) != CUFFT_SUCCESS ||
        cufftExecR2C(b->fwd, b->d_xf, b->d_X) != CUFFT_SUCCESS)
        return fail(RTIS_ERR_CUDA, "rtis_baseline_process: cuFFT forward");
    bl_band<<<g1, nt, 0, st>>>(b->d_X, p.d_C, p.M, p.F, p.k_lo, p.k_hi, b->d_S);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "rtis_baseline_process: band");
    if (cufftExecC2C(b->inv, b->d_S, b->d_S, CUFFT_INVERSE) != CUFFT_SUCCESS)
        return fail(RTIS_ERR_CUDA, "rtis_baseline_process: cuFFT inverse");
    bl_das<<<dim3((p.N + nt - 1) / nt, p.D), nt, 0, st>>>(b->d_S, p.F, p.d_shift, p.d_wt, p.M, p.N, b->d_env);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "rtis_baseline_process: delay-and-sum");
    bl_lpf<<<dim3((p.n_out + nt - 1) / nt, p.D), nt, 0, st>>>(b->d_env, p.d_h, p.lpf_len, p.R, p.N, p.n_out, d_out);
    e = cudaGetLastError();
    return e == cudaSuccess ? RTIS_OK : cuda_fail(e, "rtis_baseline_process: low-pass");
}

void rtis_baseline_destroy(rtis_baseline* b) {
    if (!b) return;
    cudaDeviceSynchronize();
    destroy(b);
}

}  // extern "C"
