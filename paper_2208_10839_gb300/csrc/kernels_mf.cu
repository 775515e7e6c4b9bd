// Matched filter + analytic signal as FFT convolution (paper Sec. 4.1 and
// Sec. 4.3: the filters run as FFT convolutions, the filter's group delay is
// removed).  Per channel m, with F = nextpow2(N + L - 1) and P = F/4:
//
//   forward  X_m[k] = sum_q w_F^{-kq} X_{m,q}[k],  X_{m,q} = DFT_P(x_m[4p+q])
//            The four real polyphase sequences are packed in pairs as complex
//            inputs z_a = x_0 + i x_1, z_b = x_2 + i x_3 -> two P-point FFTs.
//   spectrum A_m[k] = X_m[k] * C[k],  C[k] = 2 conj(S[k]) / F, k in the band.
//   inverse  The band lies below F/4, so with n = 4p + q:
//            a_m[n] = w_F^{k_lo n} IDFT_P( A_m[k_lo + k'] w_F^{k' q} )[p]
//            -- four P-point inverse FFTs per channel, one per phase q.
//   baseband z_m[j] = a_m[4j] exp(-2 pi i k_c 4j / F)
//            = w_F^{(k_c - k_lo) 4j} IDFT_P( A_m[k_lo + k'] )[j]: phase 0 alone.
//
// Each P-point FFT runs in shared memory as a mixed-radix Stockham
// autosort FFT (radix 16 passes plus one smaller pass), each thread holding
// its butterflies in registers between passes; twiddles come from an F-point
// table computed on the host in FP64.
#include <cuda_bf16.h>

#include <algorithm>
#include <cstring>

#include "fft.cuh"
#include "rtis_internal.h"

namespace rtis {
namespace {

using namespace fft;

constexpr int kMfThreads = 512;

// One polyphase pair of one channel: h = 0 packs x[4p], x[4p+1], h = 1 packs
// x[4p+2], x[4p+3] as a complex sequence; its P-point FFT goes to Z[(2m + h) P ...].
template <int LOGP>
__device__ __forceinline__ void mf_forward_body(float2* sbuf, const int16_t* __restrict__ x, int N,
                                                float2* __restrict__ Z, const float2* __restrict__ tw, int F, int m,
                                                int h) {
    constexpr int P = 1 << LOGP;
    const short4* xr = reinterpret_cast<const short4*>(x + static_cast<size_t>(m) * N);
    const int nq = N >> 2;
    const float sc = 1.0f / 32768.0f;
    for (int p = threadIdx.x; p < P; p += kMfThreads) {
        float2 z = make_float2(0.f, 0.f);
        if (p < nq) {
            const short4 q = __ldg(xr + p);
            z = h ? make_float2(q.z * sc, q.w * sc) : make_float2(q.x * sc, q.y * sc);
        }
        sbuf[spad(p)] = z;
    }
    __syncthreads();
    fft_smem<LOGP, false, kMfThreads>(sbuf, GlobalTwiddles{tw}, F);
    float2* out = Z + (static_cast<size_t>(m) * 2 + h) * P;
    for (int k = threadIdx.x; k < P; k += kMfThreads) out[k] = sbuf[spad(k)];
}

// grid (M, 2, n): channel m, polyphase pair h, measurement blockIdx.z (input and
// spectra advance by their strides)
template <int LOGP>
__global__ void __launch_bounds__(kMfThreads) mf_forward_kernel(const int16_t* __restrict__ x, int N,
                                                                float2* __restrict__ Z,
                                                                const float2* __restrict__ tw, int F,
                                                                size_t x_stride, size_t z_stride) {
    extern __shared__ float2 sbuf[];
    mf_forward_body<LOGP>(sbuf, x + blockIdx.z * x_stride, N, Z + blockIdx.z * z_stride, tw, F,
                          static_cast<int>(blockIdx.x), static_cast<int>(blockIdx.y));
}

// Channel m, output phase q: rebuilds the in-band spectrum A_m[k] from the two
// half-size spectra, optionally stores it (q == 0), then inverse-transforms phase q.
template <int LOGP>
__device__ __forceinline__ void mf_inverse_body(float2* sbuf, const float2* __restrict__ Z,
                                                const float2* __restrict__ C, const float2* __restrict__ tw, int F,
                                                int k_lo, int Kb, int N, float2* __restrict__ a,
                                                float2* __restrict__ A_out, uint32_t* __restrict__ a16, int a_ms,
                                                int a_ks, float2* __restrict__ zb, int Nb, int zb_stride, int k_c,
                                                int m, int q) {
    constexpr int P = 1 << LOGP;
    const float2* Za = Z + static_cast<size_t>(m) * 2 * P;
    const float2* Zb = Za + P;
    for (int kp = threadIdx.x; kp < P; kp += kMfThreads) {
        float2 g = make_float2(0.f, 0.f);
        if (kp < Kb) {
            const int k = k_lo + kp;
            const int km = (P - k) & (P - 1);
            const float2 za = __ldg(Za + k), zam = __ldg(Za + km);
            const float2 zb = __ldg(Zb + k), zbm = __ldg(Zb + km);
            // real-input unpacking: X0 = (za + conj(zam))/2, X1 = (za - conj(zam))/(2i)
            const float2 x0 = make_float2(0.5f * (za.x + zam.x), 0.5f * (za.y - zam.y));
            const float2 x1 = make_float2(0.5f * (za.y + zam.y), -0.5f * (za.x - zam.x));
            const float2 x2 = make_float2(0.5f * (zb.x + zbm.x), 0.5f * (zb.y - zbm.y));
            const float2 x3 = make_float2(0.5f * (zb.y + zbm.y), -0.5f * (zb.x - zbm.x));
            float2 X = x0;
            const float2 t1 = cmul(__ldg(tw + k), x1);
            const float2 t2 = cmul(__ldg(tw + 2 * k), x2);
            const float2 t3 = cmul(__ldg(tw + 3 * k), x3);
            X.x += t1.x + t2.x + t3.x;
            X.y += t1.y + t2.y + t3.y;
            const float2 Av = cmul(X, __ldg(C + kp));
            if (A_out != nullptr && q == 0)
                A_out[static_cast<size_t>(m) * a_ms + static_cast<size_t>(kp) * a_ks] = Av;
            g = (q == 0) ? Av : cmul(Av, conjf2(__ldg(tw + ((kp * q) & (F - 1)))));
        }
        sbuf[spad(kp)] = g;
    }
    if (a == nullptr && a16 == nullptr && zb == nullptr) return;  // spectrum only (uniform across the block)
    __syncthreads();
    fft_smem<LOGP, true, kMfThreads>(sbuf, GlobalTwiddles{tw}, F);
    const unsigned fmask = static_cast<unsigned>(F - 1);
    if (zb) {  // baseband (grid y = 1, q = 0): demodulate by k_c, keep every 4th sample
        const unsigned sh = static_cast<unsigned>(k_lo - k_c);  // (k_lo - k_c) mod 2^32
        for (int p = threadIdx.x; p < Nb; p += kMfThreads) {
            const unsigned idx = (sh * (4u * static_cast<unsigned>(p))) & fmask;
            zb[static_cast<size_t>(m) * zb_stride + p] = cmul(sbuf[spad(p)], conjf2(__ldg(tw + idx)));
        }
        return;
    }
    for (int p = threadIdx.x; p < P; p += kMfThreads) {
        const int n = 4 * p + q;
        if (n < N) {
            const unsigned idx = (static_cast<unsigned>(k_lo) * static_cast<unsigned>(n)) & fmask;
            const float2 v = cmul(sbuf[spad(p)], conjf2(__ldg(tw + idx)));
            if (a) a[static_cast<size_t>(m) * N + n] = v;
            if (a16) {  // round to nearest even; re in the low half, im in the high half
                const __nv_bfloat162 h = __floats2bfloat162_rn(v.x, v.y);
                a16[static_cast<size_t>(m) * N + n] = *reinterpret_cast<const uint32_t*>(&h);
            }
        }
    }
}

// grid (M, nq, n): channel m, output phase q, measurement blockIdx.z
template <int LOGP>
__global__ void __launch_bounds__(kMfThreads) mf_inverse_kernel(const float2* __restrict__ Z,
                                                                const float2* __restrict__ C,
                                                                const float2* __restrict__ tw, int F,
                                                                int k_lo, int Kb, int N,
                                                                float2* __restrict__ a,
                                                                float2* __restrict__ A_out,
                                                                uint32_t* __restrict__ a16, int a_ms, int a_ks,
                                                                size_t z_stride, size_t a_stride, size_t A_tstride,
                                                                float2* __restrict__ zb, int Nb, int zb_stride,
                                                                int k_c) {
    extern __shared__ float2 sbuf[];
    mf_inverse_body<LOGP>(sbuf, Z + blockIdx.z * z_stride, C, tw, F, k_lo, Kb, N, a ? a + blockIdx.z * a_stride : a,
                          A_out ? A_out + blockIdx.z * A_tstride : A_out, a16 ? a16 + blockIdx.z * a_stride : a16,
                          a_ms, a_ks, zb, Nb, zb_stride, k_c, static_cast<int>(blockIdx.x),
                          static_cast<int>(blockIdx.y));
}

// Several sensors with their own record lengths in one launch: block b runs work
// item b of the flat list (sensor s: items item0[s] ..), each with its sensor's FFT
// size.  The bodies are the single-sensor kernels' own, so the results are the same
// bit for bit.  FWD: items (m, h) = (j / 2, j % 2); otherwise (m, q) = (j / 4, j % 4).
template <bool FWD>
__global__ void __launch_bounds__(kMfThreads) mf_ragged_kernel(const __grid_constant__ MfRagged r) {
    extern __shared__ float2 sbuf[];
    const int b = static_cast<int>(blockIdx.x);
    int s = 0;
    while (s + 1 < r.n && b >= r.s[s + 1].item0) ++s;
    const MfRaggedSensor& S = r.s[s];
    const int j = b - S.item0;
    if constexpr (FWD) {
        const int m = j >> 1, h = j & 1;
        switch (S.logP) {
#define RTIS_MF_FWD(L) case L: mf_forward_body<L>(sbuf, S.x, S.N, S.Z, S.tw, S.F, m, h); break;
            RTIS_MF_FWD(6) RTIS_MF_FWD(7) RTIS_MF_FWD(8) RTIS_MF_FWD(9) RTIS_MF_FWD(10) RTIS_MF_FWD(11)
            RTIS_MF_FWD(12) RTIS_MF_FWD(13) RTIS_MF_FWD(14)
#undef RTIS_MF_FWD
            default: break;
        }
    } else {
        const int m = j >> 2, q = j & 3;
        switch (S.logP) {
#define RTIS_MF_INV(L) \
    case L: mf_inverse_body<L>(sbuf, S.Z, S.C, S.tw, S.F, S.k_lo, S.Kb, S.N, S.a, nullptr, S.a16, S.Kb, 1, nullptr, 0, 0, 0, m, q); break;
            RTIS_MF_INV(6) RTIS_MF_INV(7) RTIS_MF_INV(8) RTIS_MF_INV(9) RTIS_MF_INV(10) RTIS_MF_INV(11)
            RTIS_MF_INV(12) RTIS_MF_INV(13) RTIS_MF_INV(14)
#undef RTIS_MF_INV
            default: break;
        }
    }
}

template <int LOGP>
size_t mf_smem() {
    return static_cast<size_t>(spad((1 << LOGP) - 1) + 1) * sizeof(float2);
}

template <int LOGP>
cudaError_t mf_forward_t(const Plan& p, const int16_t* d_in, cudaStream_t st, const MfBatch& mb) {
    const size_t sm = mf_smem<LOGP>();
    cudaError_t e = cudaFuncSetAttribute(mf_forward_kernel<LOGP>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         static_cast<int>(sm));
    if (e != cudaSuccess) return e;
    mf_forward_kernel<LOGP><<<dim3(p.M, 2, mb.n), kMfThreads, sm, st>>>(d_in, p.N, mb.Z ? mb.Z : p.d_Z, p.d_tw,
                                                                         p.F, mb.x_stride, mb.z_stride);
    return cudaGetLastError();
}

template <int LOGP>
cudaError_t mf_inverse_t(const Plan& p, float2* d_a, float2* d_A, uint32_t* d_a16, int a_ms, int a_ks,
                         cudaStream_t st, const MfBatch& mb) {
    const size_t sm = mf_smem<LOGP>();
    cudaError_t e = cudaFuncSetAttribute(mf_inverse_kernel<LOGP>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         static_cast<int>(sm));
    if (e != cudaSuccess) return e;
    const int nq = (d_a || d_a16) ? 4 : 1;
    mf_inverse_kernel<LOGP><<<dim3(p.M, nq, mb.n), kMfThreads, sm, st>>>(
        mb.Z ? mb.Z : p.d_Z, p.d_C, p.d_tw, p.F, p.k_lo, p.Kb, p.N, d_a, d_A, d_a16, a_ms, a_ks, mb.z_stride,
        mb.a_stride, mb.A_tstride, nullptr, 0, 0, 0);
    return cudaGetLastError();
}

template <int LOGP>
cudaError_t mf_inverse_bb_t(const Plan& p, float2* d_z, int stride, cudaStream_t st) {
    const size_t sm = mf_smem<LOGP>();
    cudaError_t e = cudaFuncSetAttribute(mf_inverse_kernel<LOGP>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         static_cast<int>(sm));
    if (e != cudaSuccess) return e;
    mf_inverse_kernel<LOGP><<<dim3(p.M, 1, 1), kMfThreads, sm, st>>>(p.d_Z, p.d_C, p.d_tw, p.F, p.k_lo, p.Kb, p.N,
                                                                      nullptr, nullptr, nullptr, p.Kb, 1, 0, 0, 0,
                                                                      d_z, p.Nb, stride, p.k_c);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_mf_inverse_bb(const Plan& p, float2* d_z, int stride, cudaStream_t st) {
    switch (p.logP) {
        case 6: return mf_inverse_bb_t<6>(p, d_z, stride, st);
        case 7: return mf_inverse_bb_t<7>(p, d_z, stride, st);
        case 8: return mf_inverse_bb_t<8>(p, d_z, stride, st);
        case 9: return mf_inverse_bb_t<9>(p, d_z, stride, st);
        case 10: return mf_inverse_bb_t<10>(p, d_z, stride, st);
        case 11: return mf_inverse_bb_t<11>(p, d_z, stride, st);
        case 12: return mf_inverse_bb_t<12>(p, d_z, stride, st);
        case 13: return mf_inverse_bb_t<13>(p, d_z, stride, st);
        case 14: return mf_inverse_bb_t<14>(p, d_z, stride, st);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_mf_ragged(const Plan* const* plans, int n, const int16_t* const* d_in, cudaStream_t st) {
    if (n < 1 || n > kMfMaxSensors) return cudaErrorInvalidValue;
    MfRagged fw, iv;
    std::memset(&fw, 0, sizeof(fw));
    fw.n = n;
    int items_f = 0, items_i = 0, logp_max = 0;
    for (int i = 0; i < n; ++i) {
        const Plan& p = *plans[i];
        if (p.logP < 6 || p.logP > 14) return cudaErrorInvalidValue;
        MfRaggedSensor& S = fw.s[i];
        S.x = d_in[i];
        S.N = p.N;
        S.Z = p.d_Z;
        S.tw = p.d_tw;
        S.F = p.F;
        S.logP = p.logP;
        S.C = p.d_C;
        S.k_lo = p.k_lo;
        S.Kb = p.Kb;
        S.a = p.a_bf16 ? nullptr : p.d_a;
        S.a16 = p.a_bf16 ? p.d_a16 : nullptr;
        S.item0 = items_f;
        items_f += 2 * p.M;
        logp_max = std::max(logp_max, p.logP);
    }
    iv = fw;
    for (int i = 0; i < n; ++i) {
        iv.s[i].item0 = items_i;
        items_i += 4 * plans[i]->M;
    }
    const size_t sm = static_cast<size_t>(spad((1 << logp_max) - 1) + 1) * sizeof(float2);
    cudaError_t e = cudaFuncSetAttribute(mf_ragged_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         static_cast<int>(sm));
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(mf_ragged_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 static_cast<int>(sm));
    if (e != cudaSuccess) return e;
    mf_ragged_kernel<true><<<items_f, kMfThreads, sm, st>>>(fw);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    mf_ragged_kernel<false><<<items_i, kMfThreads, sm, st>>>(iv);
    return cudaGetLastError();
}

cudaError_t launch_mf_forward(const Plan& p, const int16_t* d_in, cudaStream_t st, const MfBatch& mb) {
    switch (p.logP) {
        case 6: return mf_forward_t<6>(p, d_in, st, mb);
        case 7: return mf_forward_t<7>(p, d_in, st, mb);
        case 8: return mf_forward_t<8>(p, d_in, st, mb);
        case 9: return mf_forward_t<9>(p, d_in, st, mb);
        case 10: return mf_forward_t<10>(p, d_in, st, mb);
        case 11: return mf_forward_t<11>(p, d_in, st, mb);
        case 12: return mf_forward_t<12>(p, d_in, st, mb);
        case 13: return mf_forward_t<13>(p, d_in, st, mb);
        case 14: return mf_forward_t<14>(p, d_in, st, mb);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_mf_inverse(const Plan& p, float2* d_a, float2* d_A, cudaStream_t st, uint32_t* d_a16, int a_ms,
                              int a_ks, const MfBatch& mb) {
    if (a_ms < 0) a_ms = p.Kb;
    switch (p.logP) {
        case 6: return mf_inverse_t<6>(p, d_a, d_A, d_a16, a_ms, a_ks, st, mb);
        case 7: return mf_inverse_t<7>(p, d_a, d_A, d_a16, a_ms, a_ks, st, mb);
        case 8: return mf_inverse_t<8>(p, d_a, d_A, d_a16, a_ms, a_ks, st, mb);
        case 9: return mf_inverse_t<9>(p, d_a, d_A, d_a16, a_ms, a_ks, st, mb);
        case 10: return mf_inverse_t<10>(p, d_a, d_A, d_a16, a_ms, a_ks, st, mb);
        case 11: return mf_inverse_t<11>(p, d_a, d_A, d_a16, a_ms, a_ks, st, mb);
        case 12: return mf_inverse_t<12>(p, d_a, d_A, d_a16, a_ms, a_ks, st, mb);
        case 13: return mf_inverse_t<13>(p, d_a, d_A, d_a16, a_ms, a_ks, st, mb);
        case 14: return mf_inverse_t<14>(p, d_a, d_A, d_a16, a_ms, a_ks, st, mb);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace rtis
