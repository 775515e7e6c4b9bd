// Shared-memory FFT building blocks (device code) used by the matched filter
// and the frequency-domain beamformer: an in-register radix-2 .. 32 DFT and a
// mixed-radix Stockham autosort FFT over P = 2^LOGP points held in shared
// memory (1-in-16 padded layout), twiddles from an F-point table
// tw[j] = exp(-2 pi i j / F) computed in FP64.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace rtis {
namespace fft {

__host__ __device__ __forceinline__ constexpr int spad(int i) { return i + (i >> 4); }  // bank-skew padding

__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ float2 conjf2(float2 a) { return make_float2(a.x, -a.y); }

// complex a + b and a - b as one packed FP32x2 instruction each (sm_100 and later);
// the same IEEE sums as two scalar adds
__device__ __forceinline__ float2 cadd(float2 a, float2 b) {
    uint64_t r;
    asm("{\n\t.reg .b64 pa, pb;\n\tmov.b64 pa, {%1, %2};\n\tmov.b64 pb, {%3, %4};\n\t"
        "add.rn.f32x2 %0, pa, pb;\n\t}"
        : "=l"(r)
        : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
    float2 o;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(o.x), "=f"(o.y) : "l"(r));
    return o;
}
__device__ __forceinline__ float2 csub(float2 a, float2 b) {
    uint64_t r;
    asm("{\n\t.reg .b64 pa, pb;\n\tmov.b64 pa, {%1, %2};\n\tmov.b64 pb, {%3, %4};\n\t"
        "sub.rn.f32x2 %0, pa, pb;\n\t}"
        : "=l"(r)
        : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
    float2 o;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(o.x), "=f"(o.y) : "l"(r));
    return o;
}

// cos and sin of 2*pi*e/32 for e = 0..15 (folded to constants once unrolled)
__device__ __forceinline__ float cos32(int e) {
    switch (e) {
        case 0: return 1.0f;
        case 1: return 0.98078528040323044913f;
        case 2: return 0.92387953251128674f;
        case 3: return 0.83146961230254523708f;
        case 4: return 0.70710678118654752f;
        case 5: return 0.55557023301960222474f;
        case 6: return 0.38268343236508977f;
        case 7: return 0.19509032201612826785f;
        case 8: return 0.0f;
        case 9: return -0.19509032201612826785f;
        case 10: return -0.38268343236508977f;
        case 11: return -0.55557023301960222474f;
        case 12: return -0.70710678118654752f;
        case 13: return -0.83146961230254523708f;
        case 14: return -0.92387953251128674f;
        default: return -0.98078528040323044913f;
    }
}
__device__ __forceinline__ float sin32(int e) { return e <= 8 ? cos32(8 - e) : cos32(e - 8); }

// d * exp(-/+ 2 pi i e / 32)  (forward: minus; inverse: plus)
template <bool INV>
__device__ __forceinline__ float2 rot32(float2 d, int e) {
    if (e == 0) return d;
    if (e == 8) return INV ? make_float2(-d.y, d.x) : make_float2(d.y, -d.x);
    const float c = cos32(e);
    const float s = INV ? sin32(e) : -sin32(e);
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

// In-register radix-R DFT (R = 1, 2, 4, 8, 16, 32): decimation-in-frequency
// butterflies, then a static bit-reversal reorder.  NZ < R: only the first NZ
// inputs can be nonzero, and the first stage skips the sums with the zeros
// (v[i + R/2] = 0 gives v[i] = a and v[i + R/2] = rot(a); both zero gives zeros).
template <int R, bool INV, int NZ = R, bool LOW = false>
__device__ __forceinline__ void dft_reg(float2 (&v)[R]) {
#pragma unroll
    for (int len = R; len >= 2; len >>= 1) {
        const int half = len >> 1;
#pragma unroll
        for (int s = 0; s < R; s += len) {
#pragma unroll
            for (int i = 0; i < half; ++i) {
                const float2 a = v[s + i], b = v[s + i + half];
                if (len == R && NZ < R && i + half >= NZ) {
                    if (i >= NZ) {
                        v[s + i] = make_float2(0.f, 0.f);
                        v[s + i + half] = make_float2(0.f, 0.f);
                    } else {
                        v[s + i + half] = rot32<INV>(a, i * (32 / len));
                    }
                    continue;
                }
                v[s + i] = cadd(a, b);
                // LOW: only the outputs k < R/2 are wanted; they sit at the even positions
                // before the bit reversal, so the last stage's differences are not formed
                if (!(LOW && len == 2)) v[s + i + half] = rot32<INV>(csub(a, b), i * (32 / len));
            }
        }
    }
    float2 t[R];
#pragma unroll
    for (int k = 0; k < R; ++k) t[k] = v[bitrev<R>(k)];
#pragma unroll
    for (int k = 0; k < R; ++k) v[k] = t[k];
}

// Twiddle sources: tw(j) = exp(-2 pi i j / F), 0 <= j < F.
struct GlobalTwiddles {  // the F-point table in global memory (read through L1)
    const float2* __restrict__ t;
    __device__ __forceinline__ float2 operator()(int j) const { return __ldg(t + j); }
};
struct SplitTwiddles {  // two small shared-memory tables: w^j = hi[j >> 8] * lo[j & 255]
    const float2* hi;
    const float2* lo;
    __device__ __forceinline__ float2 operator()(int j) const { return cmul(hi[j >> 8], lo[j & 255]); }
};

// One Stockham pass of radix R over P = 2^LOGP points held in shared memory
// (padded layout).  Ns = product of the radices of the earlier passes.
template <int LOGP, int R, bool INV, int NT, typename TW>
__device__ __forceinline__ void stockham_pass(float2* buf, int Ns, const TW& tw, int tw_scale) {
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
                // w^r from table values w^(2^i): w^r = w^(r - lowbit) * w^lowbit, at most
                // log2(R) rounded factors deep
                float2 w[R];
#pragma unroll
                for (int r = 1; r < R; r <<= 1) w[r] = tw(r * k * tw_scale);
#pragma unroll
                for (int r = 3; r < R; ++r)
                    if (r & (r - 1)) w[r] = cmul(w[r & (r - 1)], w[r & -r]);
#pragma unroll
                for (int r = 1; r < R; ++r) {
                    float2 wr = w[r];
                    if (INV) wr.y = -wr.y;
                    v[b][r] = cmul(v[b][r], wr);
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

// Full P-point FFT in shared memory; tw(j) = exp(-2 pi i j/F).
template <int LOGP, bool INV, int NT, typename TW>
__device__ __forceinline__ void fft_smem(float2* buf, const TW& tw, int F) {
    int Ns = 1;
    constexpr int rem = LOGP % 4;
    if constexpr (rem == 1) {
        stockham_pass<LOGP, 2, INV, NT, TW>(buf, Ns, tw, F / (Ns * 2));
        Ns *= 2;
    } else if constexpr (rem == 2) {
        stockham_pass<LOGP, 4, INV, NT, TW>(buf, Ns, tw, F / (Ns * 4));
        Ns *= 4;
    } else if constexpr (rem == 3) {
        stockham_pass<LOGP, 8, INV, NT, TW>(buf, Ns, tw, F / (Ns * 8));
        Ns *= 8;
    }
#pragma unroll 1
    for (int i = 0; i < LOGP / 4; ++i) {
        stockham_pass<LOGP, 16, INV, NT, TW>(buf, Ns, tw, F / (Ns * 16));
        Ns *= 16;
    }
}

}  // namespace fft
}  // namespace rtis
