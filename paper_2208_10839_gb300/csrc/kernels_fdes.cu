// Frequency-domain delay-and-sum energyscape (the phase-ramp form of the
// paper's delay-and-sum, Fig. 3 / Sec. 4.1, with the envelope, low-pass and
// subsampling of Sec. 4.3).  One CTA per direction d:
//
//   B_d[k] = sum_m g_m exp(+2 pi i k delta_dm / F) A_m[k],  k = k_lo .. k_hi
//   b_d[n] = IDFT_F(B_d)[n],  n < N     (A carries the 1/F of the transform)
//   E[d][i] = sum_j h[j] |b_d[R i + j - half]|
//
// B_d: thread t owns the bins k' = t + 256 c (coalesced loads of A); per mic
// and chunk of up to 16 bins it anchors the steering phase exactly (compensated FP32
// product k * delta/F, integer cycles removed) and then advances it with one
// complex multiply by exp(2 pi i 256 delta/F) per bin.  b_d: with n = 4p + q
// the band (below F/4) needs four P = F/4 point inverse FFTs of
// B_d[k_lo + k'] w_F^{k' q}; the remaining factor w_F^{k_lo n} has unit
// modulus and drops out of |b_d|.  Each phase IFFT is three Stockham passes
// of radix P/256, 16, 16 (256 threads, one butterfly or two per thread per
// pass; for P = 16384, 512 threads and radix 32, 32, 16): the first pass reads the steered spectrum and applies the phase's
// pre-twiddle in registers (skipping the zero bins above the band), the last
// writes |b| as floats, only for the samples n < N.  After each phase the
// low-pass taps that fall on n = q (mod 4) are added to the outputs each
// thread owns.  The pre-twiddles come from two small shared tables
// (w^j = hi[j >> 8] lo[j & 255]) instead of the F-point table; the radix-16
// passes take w = e^{2 pi i x/P} from two more (32 + 16 entries, read without
// bank conflicts) and its powers by squaring and products.
#include <algorithm>

#include "fft.cuh"
#include "rtis_internal.h"

namespace rtis {
namespace {

using namespace fft;

constexpr int kFdesChunk = 16;  // slots of 256 bins per thread per anchor (tail: 8, 4, 2, 1)
constexpr int kFoldOut = 8;     // register fold: output bins per thread (n_out <= 2048)
constexpr int kFoldTaps = 11;   // register fold: taps per residue class (low-pass length <= 44)

struct FdesArgs {
    const float2* A;      // [M][Kb] in-band matched-filter spectra (already / F)
    const float2* dphase; // [D][M] delta_dm / F in cycles per bin, hi + lo
    const float* gain;    // [M]
    const float2* tw;     // [F]
    const float* h;       // [lpf_len]
    float* E;             // [D][n_out], or [T][D][n_out] from Y
    const float2* Y;      // [D][Kb][T] steered spectra (from-Y variant)
    int T;
    unsigned* status;
    int M, D, N, F, k_lo, Kb, R, lpf_len, n_out;
    int pf_ahead;         // from Y: blocks resident at once (the block pf_ahead later starts next)
};

// fractional part of k * (hi + lo) in cycles, compensated FP32 (k an exact integer)
__device__ __forceinline__ float frac_cycles(float k, float2 ph) {
    const float p = k * ph.x;
    const float e = fmaf(k, ph.x, -p);
    const float r = p - rintf(p);
    return r + fmaf(k, ph.y, e);
}

struct FdesSmem {
    int fbuf, B, twhi, twlo, Eacc, hs, step, gs, ct, bytes;
};

__host__ __device__ constexpr int fpad(int i) { return i + (i >> 5); }  // 1-in-32 bank skew
// entries of the coarse pass-twiddle table: x = 32 h + l covers x < P/16
__host__ __device__ constexpr int fdes_ct_hi(int P) { return P / 512 > 16 ? P / 512 : 16; }
// threads per CTA: 256, and 512 for P = 16384 (the first pass stays radix 32)
__host__ __device__ constexpr int fdes_threads(int logP) { return logP >= 14 ? 512 : 256; }

// nb: entries of the steered-spectrum buffer B (Kb, or the pruned first pass's padded
// NZ x 256 slots, zeros past Kb)
__host__ __device__ inline FdesSmem fdes_layout(int P, int F, int nb, int n_out, int lpf_len, int M) {
    FdesSmem L;
    int o = 0;
    L.fbuf = o;
    o += (fpad(P - 1) + 1) * 8;
    L.B = o;
    o += nb * 8;
    L.twhi = o;
    o += (F / 256) * 8;
    L.twlo = o;
    o += 256 * 8;
    L.step = o;
    o += M * 8;
    L.Eacc = o;
    o += n_out * 4;
    L.hs = o;
    o += lpf_len * 4;
    L.gs = o;
    o += M * 4;
    o = (o + 7) & ~7;
    L.ct = o;  // pass twiddles: 32 x e^{+2 pi i l/P}, then max(16, P/512) x e^{+2 pi i 32 h/P}
    o += (32 + fdes_ct_hi(P)) * 8;
    L.bytes = o;
    return L;
}

// Steered spectrum on NBIN slots of one thread: bins kp0 + NT i, i < NBIN.
// Per mic the phase is anchored exactly at kp0 (compensated FP32, integer
// cycles removed) and advanced by exp(2 pi i NT delta/F) per slot.
template <int NBIN, int NT>
__device__ __forceinline__ void fdes_gemv_chunk(const FdesArgs& a, const float2* __restrict__ dph,
                                                const float* gs, const float2* step, float2* B, int kp0) {
    const int M = a.M, Kb = a.Kb;
    float2 acc[NBIN];
#pragma unroll
    for (int i = 0; i < NBIN; ++i) acc[i] = make_float2(0.f, 0.f);
    const float k0 = static_cast<float>(a.k_lo + kp0);
#pragma unroll 4
    for (int m = 0; m < M; ++m) {
        float s, c;
        __sincosf(6.28318530717958647692f * frac_cycles(k0, __ldg(dph + m)), &s, &c);
        const float g = gs[m];
        float2 w = make_float2(g * c, g * s);
        const float2 st = step[m];
        const float2* Am = a.A + static_cast<size_t>(m) * Kb;
#pragma unroll
        for (int i = 0; i < NBIN; ++i) {
            const int kp = kp0 + i * NT;
            if (kp < Kb) {
                const float2 v = __ldg(Am + kp);
                acc[i].x = fmaf(w.x, v.x, fmaf(-w.y, v.y, acc[i].x));
                acc[i].y = fmaf(w.x, v.y, fmaf(w.y, v.x, acc[i].y));
            }
            if (i + 1 < NBIN) w = cmul(w, st);
        }
    }
#pragma unroll
    for (int i = 0; i < NBIN; ++i) {
        const int kp = kp0 + i * NT;
        if (kp < Kb) B[kp] = acc[i];
    }
}

// One inverse radix-R (16 or 32) Stockham pass over P points (padded layout fpad),
// Ns = product of the earlier radices, NT threads.  The last pass (Ns = P/R) writes
// env[p] = |b(4p + q)| for p < e_end (the samples n < N of this phase) and
// zeros for e_end <= p < p_fill (the low-pass reads past the record's end),
// instead of the complex values.  HALF (last pass, e_end <= P/2): the outputs
// r >= R/2 lie past the record, so they are neither formed nor measured, only
// the zeros below p_fill are written.
template <int LOGP, int R, int NS, bool LAST, int NT, bool HALF = false>
__device__ __forceinline__ void fdes_pass(float2* buf, float* env, const float2* ct, int e_end, int p_fill) {
    constexpr int P = 1 << LOGP;
    constexpr int NB = P / R;
    constexpr int BPT = (NB + NT - 1) / NT;
    static_assert(R == 16 || R == 32, "radix 16 or 32");
    static_assert(!LAST || NS == NB, "the last pass has Ns = P/R");
    static_assert(!HALF || LAST, "output pruning applies to the last pass");
    float2 v[BPT][R];
    // with NB a multiple of 32, fpad(j + r NB) = fpad(j) + r (NB + NB/32) for j < NB
    constexpr int NBP = NB + NB / 32;
#pragma unroll
    for (int b = 0; b < BPT; ++b) {
        const int j = threadIdx.x + b * NT;
        if (NB % NT == 0 || j < NB) {
            if constexpr (NB % 32 == 0) {
                const float2* src = buf + fpad(j);
#pragma unroll
                for (int r = 0; r < R; ++r) v[b][r] = src[r * NBP];
            } else {
#pragma unroll
                for (int r = 0; r < R; ++r) v[b][r] = buf[fpad(j + r * NB)];
            }
        }
    }
    __syncthreads();
    // radix 16: w^r = w^(r - lowbit) w^lowbit from w^1, w^2, w^4, w^8 (a 16-entry table);
    // radix 32: w^r by a running product (two registers instead of 32 entries).
    // When Ns divides the thread count every butterfly of a thread has the same k.
    constexpr bool SHARED_K = (NS <= NT);
    constexpr int RT = R == 16 ? 16 : 2;
    float2 w[RT];
    // w = e^{+2 pi i k/(R Ns)} = e^{+2 pi i x/P} with x = k P/(R Ns) < P/R, from two
    // small tables read without bank conflicts (x = 32 h + l)
    auto twiddles = [&](int k) {
        const int x = k * (P / (R * NS));
        const float2 w1 = cmul(ct[32 + (x >> 5)], ct[x & 31]);
        w[1] = w1;
        if constexpr (R == 16) {
            w[2] = cmul(w1, w1);
            w[4] = cmul(w[2], w[2]);
            w[8] = cmul(w[4], w[4]);
#pragma unroll
            for (int r = 3; r < 16; ++r)
                if (r & (r - 1)) w[r & (RT - 1)] = cmul(w[(r & (r - 1)) & (RT - 1)], w[(r & -r) & (RT - 1)]);
        }
    };
    if (SHARED_K && NS > 1) twiddles(threadIdx.x & (NS - 1));
    // the second butterfly of a thread (k = t + NT) has w_k^r = w_t^r e^{+2 pi i NT r / P}
    // = w_t^r rot32(r) when P = 32 NT: exact rotations instead of a second table walk
    constexpr bool ROT2 = !SHARED_K && BPT == 2 && P == 32 * NT && R == 16;
#pragma unroll
    for (int b = 0; b < BPT; ++b) {
        const int j = threadIdx.x + b * NT;
        if (NB % NT == 0 || j < NB) {
            const int k = j & (NS - 1);
            if (NS > 1) {
                if (!SHARED_K) {
                    if (b == 0 || !ROT2) twiddles(k);
                }
                if constexpr (R == 16) {
#pragma unroll
                    for (int r = 1; r < 16; ++r) {
                        float2 wr = w[r];
                        if constexpr (ROT2) {
                            if (b == 1) wr = rot32<true>(wr, r);
                        }
                        v[b][r] = cmul(v[b][r], wr);
                    }
                } else {
                    float2 wr = w[1];
#pragma unroll
                    for (int r = 1; r < R; ++r) {
                        v[b][r] = cmul(v[b][r], wr);
                        if (r + 1 < R) wr = cmul(wr, w[1]);
                    }
                }
            }
            dft_reg<R, true, R, HALF>(v[b]);
            if constexpr (!LAST) {
                const int base = (j - k) * R + k;
                if constexpr (NS % 32 == 0) {  // fpad(base + r NS) = fpad(base) + r (NS + NS/32)
                    float2* dst = buf + fpad(base);
#pragma unroll
                    for (int r = 0; r < R; ++r) dst[r * (NS + NS / 32)] = v[b][r];
                } else {
#pragma unroll
                    for (int r = 0; r < R; ++r) buf[fpad(base + r * NS)] = v[b][r];
                }
            } else {
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    const int p = k + r * NS;
                    if (HALF && r >= R / 2) {
                        if (p < p_fill) env[p] = 0.f;
                    } else {
                        const float mag = magnitude_from_norm(v[b][r].x * v[b][r].x + v[b][r].y * v[b][r].y);
                        if (p < p_fill) env[p] = p < e_end ? mag : 0.f;
                    }
                }
            }
        }
    }
    __syncthreads();
}

// FROM_Y: the steered spectra come from the batched GEMM (Y[d][k'][t]); CTA b
// handles direction b / T of measurement b % T (neighbouring measurements share
// Y's sectors and run side by side).  Otherwise the CTA steers direction b itself.
// NZ: bins k' = t + NT r can be nonzero only for r < NZ (the band's slots; the rest
// of the first pass's inputs are the zero padding up to P).  FOLD: every output
// bin of a thread (i = t + NT m) has the same residue (R i - half) mod 4, so per
// phase the thread's low-pass taps are one comb j0 + 4 s, held in registers, and
// its outputs accumulate in registers across the four phases.
template <int LOGP, bool FROM_Y, int NZ, bool FOLD, int NT, bool HALF>
__global__ void __launch_bounds__(NT, NT == 256 ? 2 : 1) fd_energyscape_kernel(const FdesArgs a) {
    constexpr int P = 1 << LOGP;
    extern __shared__ __align__(16) unsigned char sm[];
    constexpr bool PADB = NZ < P / NT;  // B holds NZ x NT slots, zeros past Kb
    const int nb = PADB ? NZ * NT : a.Kb;
    const FdesSmem L = fdes_layout(P, a.F, nb, a.n_out, a.lpf_len, a.M);
    float2* fbuf = reinterpret_cast<float2*>(sm + L.fbuf);
    float2* B = reinterpret_cast<float2*>(sm + L.B);
    float2* twhi = reinterpret_cast<float2*>(sm + L.twhi);
    float2* twlo = reinterpret_cast<float2*>(sm + L.twlo);
    float2* step = reinterpret_cast<float2*>(sm + L.step);  // exp(2 pi i NT delta/F)
    float* Eacc = reinterpret_cast<float*>(sm + L.Eacc);
    float* hs = reinterpret_cast<float*>(sm + L.hs);
    float* gs = reinterpret_cast<float*>(sm + L.gs);

    const int d = FROM_Y ? static_cast<int>(blockIdx.x) / a.T : static_cast<int>(blockIdx.x);
    const int t_meas = FROM_Y ? static_cast<int>(blockIdx.x) - d * a.T : 0;
    const int tid = threadIdx.x;
    const int M = a.M, Kb = a.Kb;
    for (int j = tid; j < 256; j += NT) twlo[j] = __ldg(a.tw + j);
    for (int j = tid; j < a.F / 256; j += NT) twhi[j] = __ldg(a.tw + j * 256);
    for (int j = tid; j < a.lpf_len; j += NT) hs[j] = a.h[j];
    float2* ct = reinterpret_cast<float2*>(sm + L.ct);
    if (tid < 32 + fdes_ct_hi(P)) {  // e^{+2 pi i l/P} = conj(tw[4 l]), e^{+2 pi i 32 h/P} = conj(tw[128 h]) (F = 4P)
        const int idx = tid < 32 ? 4 * tid : 128 * (tid - 32);
        ct[tid] = conjf2(__ldg(a.tw + (idx & (a.F - 1))));
    }
    for (int i = tid; i < a.n_out; i += NT) Eacc[i] = 0.f;
    if (tid < M) {
        const float2 ph = __ldg(a.dphase + static_cast<size_t>(d) * M + tid);
        float s, c;
        sincospif(2.0f * frac_cycles(static_cast<float>(NT), ph), &s, &c);
        step[tid] = make_float2(c, s);
        gs[tid] = a.gain[tid];
    }
    __syncthreads();
    const SplitTwiddles tws{twhi, twlo};

    if constexpr (FROM_Y) {
        {  // bring the spectrum of the block that starts about one block lifetime later into L2
           // (one block of each four neighbouring measurements, which share the 32-byte sectors)
            const int nbk = static_cast<int>(blockIdx.x) + a.pf_ahead;
            if (a.pf_ahead > 0 && nbk < static_cast<int>(gridDim.x)) {
                const int d2 = nbk / a.T, t2 = nbk - d2 * a.T;
                if ((t2 & 3) == 0)
                    for (int kp = tid; kp < Kb; kp += NT)
                        asm volatile("prefetch.global.L2 [%0];" ::"l"(a.Y + (static_cast<size_t>(d2) * Kb + kp) * a.T + t2));
            }
        }
        for (int kp = tid; kp < nb; kp += NT)
            B[kp] = kp < Kb ? __ldg(a.Y + (static_cast<size_t>(d) * Kb + kp) * a.T + t_meas) : make_float2(0.f, 0.f);
        __syncthreads();
    } else {
        for (int kp = Kb + tid; kp < nb; kp += NT) B[kp] = make_float2(0.f, 0.f);
        // ---- steered spectrum B_d ------------------------------------------------
        // slots of NT bins: full chunks of kFdesChunk slots, then the tail in chunks
        // of 8, 4, 2, 1 so that no thread advances the recurrence past the band
        const float2* dph = a.dphase + static_cast<size_t>(d) * M;
        const int nslots = (Kb + NT - 1) / NT;
        int c0 = 0;
        for (; c0 + kFdesChunk <= nslots; c0 += kFdesChunk)
            fdes_gemv_chunk<kFdesChunk, NT>(a, dph, gs, step, B, c0 * NT + tid);
        static_assert(kFdesChunk == 16, "the tail below covers remainders up to 15 slots");
        if ((nslots - c0) & 8) {
            fdes_gemv_chunk<8, NT>(a, dph, gs, step, B, c0 * NT + tid);
            c0 += 8;
        }
        if ((nslots - c0) & 4) {
            fdes_gemv_chunk<4, NT>(a, dph, gs, step, B, c0 * NT + tid);
            c0 += 4;
        }
        if ((nslots - c0) & 2) {
            fdes_gemv_chunk<2, NT>(a, dph, gs, step, B, c0 * NT + tid);
            c0 += 2;
        }
        if ((nslots - c0) & 1) fdes_gemv_chunk<1, NT>(a, dph, gs, step, B, c0 * NT + tid);
        __syncthreads();
    }

    // ---- four phase IFFTs, each folded into the low-pass outputs ------------
    constexpr int R0 = P / NT;  // first-pass radix, 1 .. 32
    static_assert(R0 >= 1 && R0 <= 32, "P = 256 .. 8192 (256 threads), 16384 (512 threads)");
    static_assert(NZ >= 1 && NZ <= R0, "nonzero first-pass slots");
    float* env = reinterpret_cast<float*>(fbuf);  // |b(4p + q)|, written by the last pass
    const int half = (a.lpf_len - 1) >> 1;
    // the register fold: outputs i = tid + NT m, m < kFoldOut; taps j0 + 4 s, s < kFoldTaps.
    // The sums over the phases stay in registers (FACC_REGS) or go to the thread's own entries
    // of Eacc: the per-direction kernel, whose steering loop needs the registers, measured
    // faster with Eacc (spills 56 -> 36 B), the from-Y kernel with the registers
    constexpr bool FACC_REGS = FROM_Y;
    float facc[kFoldOut];
#pragma unroll
    for (int m = 0; m < kFoldOut; ++m) facc[m] = 0.f;
    const int res = ((a.R * tid - half) % 4 + 4) & 3;  // (R i - half) mod 4 for all of this thread's i
    for (int q = 0; q < 4; ++q) {
        {  // first pass (radix R0, Ns = 1): bins k' = t + NT r, pre-twiddled by e^{+2 pi i k' q / F}
            // = e^{+2 pi i t q / F} e^{+2 pi i NT q r / F}: a start value and a constant step per phase
            float2 v[R0];
            float2 w = q == 0 ? make_float2(1.f, 0.f) : conjf2(tws(static_cast<int>((static_cast<unsigned>(tid) * q) & (a.F - 1))));
            const float2 wstep = q == 0 ? make_float2(1.f, 0.f) : conjf2(tws(NT * q));
#pragma unroll
            for (int r = 0; r < R0; ++r) {
                float2 g = make_float2(0.f, 0.f);
                if (r < NZ) {
                    const int kp = tid + r * NT;
                    if (PADB || kp < Kb) g = (q == 0) ? B[kp] : cmul(B[kp], w);
                    if (q != 0 && r + 1 < NZ) w = cmul(w, wstep);
                }
                v[r] = g;
            }
            dft_reg<R0, true, NZ>(v);
            // R0 divides 32, so t R0 + r stays in one 32-point block: fpad is linear in r
            float2* dst = fbuf + fpad(tid * R0);
#pragma unroll
            for (int r = 0; r < R0; ++r) dst[r] = v[r];
        }
        __syncthreads();
        const int e_end = (a.N - q + 3) >> 2;  // env entries of this phase with n = 4p + q < N
        // the rest of P: NT = 16 x (NT/16) points per first-pass output column
        fdes_pass<LOGP, NT / 16, R0, false, NT>(fbuf, env, ct, e_end, 0);
        fdes_pass<LOGP, 16, (NT / 16) * R0, true, NT, HALF>(fbuf, env, ct, e_end, e_end + 4 * kFoldTaps + 4);
        if constexpr (FOLD) {
            // taps j = j0 + 4 s read env[(R i - half + j0 - q) / 4 + s]; entries past the record's
            // end were written as zeros, entries before its start are skipped below
            const int j0 = (q - res + 4) & 3;
            float hreg[kFoldTaps];
#pragma unroll
            for (int s4 = 0; s4 < kFoldTaps; ++s4) {
                const int j = j0 + 4 * s4;
                hreg[s4] = j < a.lpf_len ? hs[j] : 0.f;
            }
#pragma unroll
            for (int m = 0; m < kFoldOut; ++m) {
                const int i = tid + m * NT;
                if (i < a.n_out) {
                    const int e0 = (a.R * i - half + j0 - q) >> 2;
                    float acc = 0.f;
                    if (m > 0 || e0 >= 0) {  // i >= NT starts well inside the record
#pragma unroll
                        for (int s4 = 0; s4 < kFoldTaps; ++s4) acc = fmaf(hreg[s4], env[e0 + s4], acc);
                    } else {
#pragma unroll
                        for (int s4 = 0; s4 < kFoldTaps; ++s4)
                            if (e0 + s4 >= 0) acc = fmaf(hreg[s4], env[e0 + s4], acc);
                    }
                    if constexpr (FACC_REGS)
                        facc[m] += acc;
                    else
                        Eacc[i] += acc;
                }
            }
        } else {
            for (int i = tid; i < a.n_out; i += NT) {
                const int n0 = a.R * i - half;          // n = n0 + j
                const int j0 = ((q - n0) % 4 + 4) & 3;  // first tap with n = q (mod 4)
                // taps j = j0 + 4 s read env[e0 + s] (n0 + j0 - q is a multiple of 4); only
                // 0 <= n < N count, i.e. 0 <= e0 + s < e_end
                const int e0 = (n0 + j0 - q) >> 2;
                const int s_lo = max(0, -e0);
                const int s_hi = min((a.lpf_len - j0 + 3) >> 2, e_end - e0);
                float acc = 0.f;
                for (int sk = s_lo; sk < s_hi; ++sk) acc = fmaf(hs[j0 + 4 * sk], env[e0 + sk], acc);
                Eacc[i] += acc;
            }
        }
        __syncthreads();
    }
    float* Erow = a.E + (static_cast<size_t>(t_meas) * a.D + d) * a.n_out;
    if constexpr (FOLD && FACC_REGS) {
#pragma unroll
        for (int m = 0; m < kFoldOut; ++m) {
            const int i = tid + m * NT;
            if (i < a.n_out) {
                if (!isfinite(facc[m])) atomicOr(a.status, RTIS_DEV_NONFINITE);
                Erow[i] = facc[m];
            }
        }
    } else {
        for (int i = tid; i < a.n_out; i += NT) {
            const float e = Eacc[i];
            if (!isfinite(e)) atomicOr(a.status, RTIS_DEV_NONFINITE);
            Erow[i] = e;
        }
    }
}

template <int LOGP, bool FROM_Y, int NZ, bool FOLD, bool HALF = false>
cudaError_t fdes_launch_t(const Plan& p, const float2* d_A, const float2* d_Y, int T, float* d_out, cudaStream_t st) {
    constexpr int NT = fdes_threads(LOGP);
    constexpr int R0 = (1 << LOGP) / NT;
    const int nb = NZ < R0 ? NZ * NT : p.Kb;
    const size_t sm = static_cast<size_t>(fdes_layout(1 << LOGP, p.F, nb, p.n_out, p.lpf_len, p.M).bytes);
    cudaError_t e = cudaFuncSetAttribute(fd_energyscape_kernel<LOGP, FROM_Y, NZ, FOLD, NT, HALF>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(sm));
    if (e != cudaSuccess) return e;
    FdesArgs a;
    a.A = d_A;
    a.dphase = p.d_dphase;
    a.gain = p.d_gain;
    a.tw = p.d_tw;
    a.h = p.d_h;
    a.E = d_out;
    a.Y = d_Y;
    a.T = T;
    a.M = p.M;
    a.D = p.D;
    a.N = p.N;
    a.F = p.F;
    a.k_lo = p.k_lo;
    a.Kb = p.Kb;
    a.R = p.R;
    a.lpf_len = p.lpf_len;
    a.n_out = p.n_out;
    a.status = p.d_status;
    a.pf_ahead = FROM_Y ? std::max(1, p.n_sm) * (NT == 256 ? 2 : 1) : 0;
    fd_energyscape_kernel<LOGP, FROM_Y, NZ, FOLD, NT, HALF><<<p.D * (FROM_Y ? T : 1), NT, sm, st>>>(a);
    return cudaGetLastError();
}

// The common case (the band fills at most R0/2 + 2 of the first pass's NT-bin slots,
// at most 8 NT output bins, a low-pass of at most 44 taps) runs the pruned first pass
// and the register fold, and when N <= F/2 the last pass pruned to its low half;
// anything else the general kernel.
template <int LOGP, bool FROM_Y>
cudaError_t fdes_launch_pick(const Plan& p, const float2* d_A, const float2* d_Y, int T, float* d_out,
                             cudaStream_t st) {
    constexpr int NT = fdes_threads(LOGP);
    constexpr int R0 = (1 << LOGP) / NT;
    constexpr int NZH = R0 / 2 + 2 < R0 ? R0 / 2 + 2 : R0;
    const int nz = (p.Kb + NT - 1) / NT;
    const bool fold = p.n_out <= kFoldOut * NT && (p.lpf_len + 3) / 4 <= kFoldTaps;
    // every sample n < N of a phase has p < P/2: the last pass forms only the low half
    const bool half = ((p.N + 3) >> 2) <= (1 << LOGP) / 2;
    if (nz <= NZH && fold && half) return fdes_launch_t<LOGP, FROM_Y, NZH, true, true>(p, d_A, d_Y, T, d_out, st);
    if (nz <= NZH && fold) return fdes_launch_t<LOGP, FROM_Y, NZH, true>(p, d_A, d_Y, T, d_out, st);
    return fdes_launch_t<LOGP, FROM_Y, R0, false>(p, d_A, d_Y, T, d_out, st);
}

template <bool FROM_Y>
cudaError_t fdes_dispatch(const Plan& p, const float2* d_A, const float2* d_Y, int T, float* d_out, cudaStream_t st) {
    switch (p.logP) {
        case 8: return fdes_launch_pick<8, FROM_Y>(p, d_A, d_Y, T, d_out, st);
        case 9: return fdes_launch_pick<9, FROM_Y>(p, d_A, d_Y, T, d_out, st);
        case 10: return fdes_launch_pick<10, FROM_Y>(p, d_A, d_Y, T, d_out, st);
        case 11: return fdes_launch_pick<11, FROM_Y>(p, d_A, d_Y, T, d_out, st);
        case 12: return fdes_launch_pick<12, FROM_Y>(p, d_A, d_Y, T, d_out, st);
        case 13: return fdes_launch_pick<13, FROM_Y>(p, d_A, d_Y, T, d_out, st);
        case 14: return fdes_launch_pick<14, FROM_Y>(p, d_A, d_Y, T, d_out, st);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace

size_t fdes_smem_bytes(const Plan& p) {
    if (p.logP < 8 || p.logP > 14) return ~static_cast<size_t>(0);
    // the larger of the two kernels' buffers (the padded one holds at most R0/2 + 2 slots)
    const int NT = fdes_threads(p.logP);
    const int R0 = p.P / NT;
    const int nb = std::max(p.Kb, std::min(R0, R0 / 2 + 2) * NT);
    return static_cast<size_t>(fdes_layout(p.P, p.F, nb, p.n_out, p.lpf_len, p.M).bytes);
}

cudaError_t launch_fd_energyscape(const Plan& p, const float2* d_A, float* d_out, cudaStream_t st) {
    return fdes_dispatch<false>(p, d_A, nullptr, 1, d_out, st);
}

cudaError_t launch_fd_energyscape_from_y(const Plan& p, const float2* d_Y, int T, float* d_out, cudaStream_t st) {
    return fdes_dispatch<true>(p, nullptr, d_Y, T, d_out, st);
}

}  // namespace rtis
