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
//
// Each P-point FFT runs in shared memory as a mixed-radix Stockham
// autosort FFT (radix 16 passes plus one smaller pass), each thread holding
// its butterflies in registers between passes; twiddles come from an F-point
// table computed on the host in FP64.
#include "rtis_internal.h"

namespace rtis {
namespace {

__host__ __device__ __forceinline__ constexpr int spad(int i) { return i + (i >> 4); }  // bank-skew padding

__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ float2 conjf2(float2 a) { return make_float2(a.x, -a.y); }

// cos and sin of 2*pi*e/16 for e = 0..7 (folded to constants once unrolled)
__device__ __forceinline__ float cos16(int e) {
    switch (e) {
        case 0: return 1.0f;
        case 1: return 0.92387953251128674f;
        case 2: return 0.70710678118654752f;
        case 3: return 0.38268343236508977f;
        case 4: return 0.0f;
        case 5: return -0.38268343236508977f;
        case 6: return -0.70710678118654752f;
        default: return -0.92387953251128674f;
    }
}
__device__ __forceinline__ float sin16(int e) {
    switch (e) {
        case 0: return 0.0f;
        case 1: return 0.38268343236508977f;
        case 2: return 0.70710678118654752f;
        case 3: return 0.92387953251128674f;
        case 4: return 1.0f;
        case 5: return 0.92387953251128674f;
        case 6: return 0.70710678118654752f;
        default: return 0.38268343236508977f;
    }
}

// d * exp(-/+ 2 pi i e / 16)  (forward: minus; inverse: plus)
template <bool INV>
__device__ __forceinline__ float2 rot16(float2 d, int e) {
    if (e == 0) return d;
    if (e == 4) return INV ? make_float2(-d.y, d.x) : make_float2(d.y, -d.x);
    const float c = cos16(e);
    const float s = INV ? sin16(e) : -sin16(e);
    return make_float2(d.x * c - d.y * s, d.x * s + d.y * c);
}

template <int R>
__device__ __forceinline__ constexpr int bitrev(int k) {
    int r = 0;
    for (int b = 1; b < R; b <<= 1) {
        r = (r << 1) | (k & 1);
        k >>= 1;
    }
    return r;
}

// In-register radix-R DFT (R = 2, 4, 8, 16): decimation-in-frequency
// butterflies, then a static bit-reversal reorder.
template <int R, bool INV>
__device__ __forceinline__ void dft_reg(float2 (&v)[R]) {
#pragma unroll
    for (int len = R; len >= 2; len >>= 1) {
        const int half = len >> 1;
#pragma unroll
        for (int s = 0; s < R; s += len) {
#pragma unroll
            for (int i = 0; i < half; ++i) {
                const float2 a = v[s + i], b = v[s + i + half];
                v[s + i] = make_float2(a.x + b.x, a.y + b.y);
                v[s + i + half] = rot16<INV>(make_float2(a.x - b.x, a.y - b.y), i * (16 / len));
            }
        }
    }
    float2 t[R];
#pragma unroll
    for (int k = 0; k < R; ++k) t[k] = v[bitrev<R>(k)];
#pragma unroll
    for (int k = 0; k < R; ++k) v[k] = t[k];
}

// One Stockham pass of radix R over P = 2^LOGP points held in shared memory
// (padded layout).  Ns = product of the radices of the earlier passes.
template <int LOGP, int R, bool INV, int NT>
__device__ __forceinline__ void stockham_pass(float2* buf, int Ns, const float2* __restrict__ tw,
                                              int tw_scale) {
    constexpr int P = 1 << LOGP;
    constexpr int NB = P / R;
    constexpr int BPT = (NB + NT - 1) / NT;
    float2 v[BPT][R];
#pragma unroll
    for (int b = 0; b < BPT; ++b) {
        const int j = threadIdx.x + b * NT;
        if (NB % NT == 0 || j < NB) {
#pragma unroll
            for (int r = 0; r < R; ++r) v[b][r] = buf[spad(j + r * NB)];
        }
    }
    __syncthreads();
#pragma unroll
    for (int b = 0; b < BPT; ++b) {
        const int j = threadIdx.x + b * NT;
        if (NB % NT == 0 || j < NB) {
            const int k = j & (Ns - 1);
            if (Ns > 1) {
#pragma unroll
                for (int r = 1; r < R; ++r) {
                    float2 w = __ldg(tw + r * k * tw_scale);
                    if (INV) w.y = -w.y;
                    v[b][r] = cmul(v[b][r], w);
                }
            }
            dft_reg<R, INV>(v[b]);
            const int base = (j - k) * R + k;
#pragma unroll
            for (int r = 0; r < R; ++r) buf[spad(base + r * Ns)] = v[b][r];
        }
    }
    __syncthreads();
}

// Full P-point FFT in shared memory; tw is the F-point table exp(-2 pi i j/F).
template <int LOGP, bool INV, int NT>
__device__ __forceinline__ void fft_smem(float2* buf, const float2* __restrict__ tw, int F) {
    int Ns = 1;
    constexpr int rem = LOGP % 4;
    if constexpr (rem == 1) {
        stockham_pass<LOGP, 2, INV, NT>(buf, Ns, tw, F / (Ns * 2));
        Ns *= 2;
    } else if constexpr (rem == 2) {
        stockham_pass<LOGP, 4, INV, NT>(buf, Ns, tw, F / (Ns * 4));
        Ns *= 4;
    } else if constexpr (rem == 3) {
        stockham_pass<LOGP, 8, INV, NT>(buf, Ns, tw, F / (Ns * 8));
        Ns *= 8;
    }
#pragma unroll 1
    for (int i = 0; i < LOGP / 4; ++i) {
        stockham_pass<LOGP, 16, INV, NT>(buf, Ns, tw, F / (Ns * 16));
        Ns *= 16;
    }
}

constexpr int kMfThreads = 512;

// grid (M, 2): channel m, polyphase pair h (h = 0: x[4p], x[4p+1]; h = 1: x[4p+2], x[4p+3])
template <int LOGP>
__global__ void __launch_bounds__(kMfThreads) mf_forward_kernel(const int16_t* __restrict__ x, int N,
                                                                float2* __restrict__ Z,
                                                                const float2* __restrict__ tw, int F) {
    extern __shared__ float2 sbuf[];
    constexpr int P = 1 << LOGP;
    const int m = blockIdx.x, h = blockIdx.y;
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
    fft_smem<LOGP, false, kMfThreads>(sbuf, tw, F);
    float2* out = Z + (static_cast<size_t>(m) * 2 + h) * P;
    for (int k = threadIdx.x; k < P; k += kMfThreads) out[k] = sbuf[spad(k)];
}

// grid (M, nq): channel m, output phase q.  Rebuilds the in-band spectrum
// A_m[k] from the two half-size spectra, optionally stores it (q == 0), then
// inverse-transforms phase q.
template <int LOGP>
__global__ void __launch_bounds__(kMfThreads) mf_inverse_kernel(const float2* __restrict__ Z,
                                                                const float2* __restrict__ C,
                                                                const float2* __restrict__ tw, int F,
                                                                int k_lo, int Kb, int N,
                                                                float2* __restrict__ a,
                                                                float2* __restrict__ A_out) {
    extern __shared__ float2 sbuf[];
    constexpr int P = 1 << LOGP;
    const int m = blockIdx.x, q = blockIdx.y;
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
            if (A_out != nullptr && q == 0) A_out[static_cast<size_t>(m) * Kb + kp] = Av;
            g = (q == 0) ? Av : cmul(Av, conjf2(__ldg(tw + ((kp * q) & (F - 1)))));
        }
        sbuf[spad(kp)] = g;
    }
    if (a == nullptr) return;  // spectrum only (uniform across the block)
    __syncthreads();
    fft_smem<LOGP, true, kMfThreads>(sbuf, tw, F);
    float2* arow = a + static_cast<size_t>(m) * N;
    const unsigned fmask = static_cast<unsigned>(F - 1);
    for (int p = threadIdx.x; p < P; p += kMfThreads) {
        const int n = 4 * p + q;
        if (n < N) {
            const unsigned idx = (static_cast<unsigned>(k_lo) * static_cast<unsigned>(n)) & fmask;
            arow[n] = cmul(sbuf[spad(p)], conjf2(__ldg(tw + idx)));
        }
    }
}

template <int LOGP>
size_t mf_smem() {
    return static_cast<size_t>(spad((1 << LOGP) - 1) + 1) * sizeof(float2);
}

template <int LOGP>
cudaError_t mf_forward_t(const Plan& p, const int16_t* d_in, cudaStream_t st) {
    const size_t sm = mf_smem<LOGP>();
    cudaError_t e = cudaFuncSetAttribute(mf_forward_kernel<LOGP>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         static_cast<int>(sm));
    if (e != cudaSuccess) return e;
    mf_forward_kernel<LOGP><<<dim3(p.M, 2), kMfThreads, sm, st>>>(d_in, p.N, p.d_Z, p.d_tw, p.F);
    return cudaGetLastError();
}

template <int LOGP>
cudaError_t mf_inverse_t(const Plan& p, float2* d_a, float2* d_A, cudaStream_t st) {
    const size_t sm = mf_smem<LOGP>();
    cudaError_t e = cudaFuncSetAttribute(mf_inverse_kernel<LOGP>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         static_cast<int>(sm));
    if (e != cudaSuccess) return e;
    const int nq = d_a ? 4 : 1;
    mf_inverse_kernel<LOGP><<<dim3(p.M, nq), kMfThreads, sm, st>>>(p.d_Z, p.d_C, p.d_tw, p.F, p.k_lo, p.Kb,
                                                                  p.N, d_a, d_A);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_mf_forward(const Plan& p, const int16_t* d_in, cudaStream_t st) {
    switch (p.logP) {
        case 6: return mf_forward_t<6>(p, d_in, st);
        case 7: return mf_forward_t<7>(p, d_in, st);
        case 8: return mf_forward_t<8>(p, d_in, st);
        case 9: return mf_forward_t<9>(p, d_in, st);
        case 10: return mf_forward_t<10>(p, d_in, st);
        case 11: return mf_forward_t<11>(p, d_in, st);
        case 12: return mf_forward_t<12>(p, d_in, st);
        case 13: return mf_forward_t<13>(p, d_in, st);
        case 14: return mf_forward_t<14>(p, d_in, st);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_mf_inverse(const Plan& p, float2* d_a, float2* d_A, cudaStream_t st) {
    switch (p.logP) {
        case 6: return mf_inverse_t<6>(p, d_a, d_A, st);
        case 7: return mf_inverse_t<7>(p, d_a, d_A, st);
        case 8: return mf_inverse_t<8>(p, d_a, d_A, st);
        case 9: return mf_inverse_t<9>(p, d_a, d_A, st);
        case 10: return mf_inverse_t<10>(p, d_a, d_A, st);
        case 11: return mf_inverse_t<11>(p, d_a, d_A, st);
        case 12: return mf_inverse_t<12>(p, d_a, d_A, st);
        case 13: return mf_inverse_t<13>(p, d_a, d_A, st);
        case 14: return mf_inverse_t<14>(p, d_a, d_A, st);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace rtis
