// Frequency-domain energyscapes from the batched GEMM's steered spectra, with
// the inverse transform as two dense DFT stages on the tcgen05 tensor cores
// (the phase-ramp form of the paper's delay-and-sum, Fig. 3 / Sec. 4.1, with
// the envelope, low-pass and subsampling of Sec. 4.3).
//
// For one direction d and measurement t the band B[k'] = Y[d][k'][t],
// k' < Kb (bins k_lo + k', already carrying the 1/F of the transform), gives
//
//   b[n] = sum_k' B[k'] exp(+2 pi i k' n / F),   n < N
//
// (the factor exp(2 pi i k_lo n / F) is dropped: it has unit modulus).  With
// F = N1 P2 = 512 x 64, k' = 64 k1 + k2 and n = n1 + 512 n2:
//
//   T1[n1][k2] = sum_k1 w512^(k1 n1) B[64 k1 + k2]        (stage 1, k1 < K1 <= 72)
//   T2[n1][k2] = w_F^(k2 n1) T1[n1][k2]                   (twiddle)
//   b[n1 + 512 n2] = sum_k2 w64^(k2 n2) T2[n1][k2]       (stage 2, n2 < 32: n < F/2)
//
// with w_X = exp(+2 pi i / X).  Both stages are real GEMMs on the complex
// data (each output column pair is (re, im)), in FP32 as three BF16 products
// hi.hi + hi.lo + lo.hi accumulated in FP32 in tensor memory.
//
// CTA shape: one CTA per SM, 384 threads.  The 512 values of n1 form four
// tiles of 128 (the MMA's M); CTA c owns tile c % 4 for every item, so its
// stage-1 matrix (128 n1 x 72 k1, hi and lo, 72 KB) and the stage-2 matrix
// (32 KB) stay in shared memory for the whole launch.  The CTAs of one tile
// walk the items (d, t) in the same order as the other tiles' CTAs, so a
// spectrum read by one tile is still in L2 for the others.
//   warp 0     lane 0 issues the MMAs (stage 1 into D1, stage 2 into D2, both
//              double-buffered in tensor memory) and commits to mbarriers;
//   warps 1-3  build the stage-1 data operand from Y (hi/lo BF16, K-major);
//   warps 4-11 read D1 (lane = n1), apply the twiddle, split it into the
//              stage-2 operand in a ring of four K-step slots, then read D2,
//              form |b| and fold the low-pass over this tile's samples.
// A tile holds the samples n = 512 n2 + 128 tile + r (runs of 128 consecutive
// samples).  An output bin whose taps lie inside one run is stored; a bin
// whose taps straddle two runs (two tiles) gets both partial sums added to
// the zeroed output, and with exactly two addends the result does not depend
// on their order.  Every mbarrier wait is bounded.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include <cuda_bf16.h>

#include "ptx.cuh"
#include "rtis_internal.h"

namespace rtis {
namespace {

constexpr int kTcN1 = 512, kTcP2 = 64, kTcK1 = 72, kTcN2 = 32;
constexpr int kTcTiles = kTcN1 / 128;
constexpr int kTcThreads = 384;
constexpr int kTcEpiWarp0 = 4;              // warps 4..11: epilogue
constexpr int kTcLoadThreads = 96;          // warps 1..3: operand builder
constexpr uint32_t kTcPolls = 1u << 20;
constexpr uint32_t kTcHintNs = 20000;

// shared-memory image (bytes); every operand is K-major without swizzle: core
// matrices of 8 rows x 16 bytes, LBO = 128 between K-neighbours, SBO between
// 8-row groups
constexpr uint32_t kW1Sbo = (2 * kTcK1 / 8) * 128;      // 18 core columns: 2304
constexpr uint32_t kW1Bytes = 128 * 2 * kTcK1 * 2;      // one split: 36864
constexpr uint32_t kW2Sbo = (2 * kTcP2 / 8) * 128;      // 16 core columns: 2048
constexpr uint32_t kW2Bytes = 2 * kTcN2 * 2 * kTcP2 * 2;  // one split: 16384
constexpr uint32_t kA2Sbo = 256;                        // one K-step: 2 core columns
constexpr uint32_t kA2Split = 128 * 16 * 2;             // 4096
constexpr uint32_t kA2Slot = 2 * kA2Split;
constexpr uint32_t kOffW1 = 0;
constexpr uint32_t kOffB1 = kOffW1 + 2 * kW1Bytes;
constexpr uint32_t kOffW2 = kOffB1 + 2 * kW1Bytes;
constexpr uint32_t kOffA2 = kOffW2 + 2 * kW2Bytes;
constexpr uint32_t kOffEnv = kOffA2 + 4 * kA2Slot;
constexpr int kEnvStride = 136;                         // floats per run of 128 samples (bank skew)
constexpr uint32_t kOffH = kOffEnv + kTcN2 * kEnvStride * 4;
constexpr int kTcMaxTaps = 127;
constexpr uint32_t kOffBar = kOffH + 128 * 4;
constexpr uint32_t kTcSmem = kOffBar + 32 * 8 + 16;
static_assert(kTcSmem <= 227 * 1024, "shared-memory image");
constexpr size_t kTcConstBytes = static_cast<size_t>(kTcTiles) * 2 * kW1Bytes + 2 * kW2Bytes;

// tensor-memory columns: D1[b] (128 each), D2[b] (2 N2 = 64 each)
constexpr uint32_t kTmemCols = 512;
constexpr uint32_t kD1Col = 0, kD2Col = 256;

struct FdtcArgs {
    const float2* Y;          // [D][Kb][T]
    const unsigned char* W;   // constants: [tile][W1 hi | lo] then [W2 hi | lo]
    const float* h;           // [lpf_len]
    float* E;                 // [T][D][n_out], zeroed before the launch
    unsigned* status;
    int D, T, Kb, N, R, lpf_len, n_out, n_items, groups;
};

// bf16 pair packing: hi = RN(a), lo = RN(a - hi)
__device__ __forceinline__ uint32_t bf2(float a, float b) {
    __nv_bfloat162 v = __floats2bfloat162_rn(a, b);
    return *reinterpret_cast<uint32_t*>(&v);
}
__device__ __forceinline__ void split8(const float (&v)[8], uint4& hi, uint4& lo) {
    float r[8];
#pragma unroll
    for (int e = 0; e < 8; ++e) r[e] = v[e] - __bfloat162float(__float2bfloat16_rn(v[e]));
    hi = make_uint4(bf2(v[0], v[1]), bf2(v[2], v[3]), bf2(v[4], v[5]), bf2(v[6], v[7]));
    lo = make_uint4(bf2(r[0], r[1]), bf2(r[2], r[3]), bf2(r[4], r[5]), bf2(r[6], r[7]));
}
__device__ __forceinline__ void st16(unsigned char* base, uint32_t off, uint4 v) {
    *static_cast<uint4*>(__builtin_assume_aligned(base + off, 16)) = v;
}
__host__ __device__ constexpr uint32_t w1_off(int r, int kc) {  // row r, core column kc
    return static_cast<uint32_t>((r >> 3) * kW1Sbo + kc * 128 + (r & 7) * 16);
}

struct Bars {
    uint64_t* cst;       // constants landed (tx)
    uint64_t* b1_full;   // stage-1 data operand built (3 loader warps)
    uint64_t* s1_done;   // stage-1 MMAs of an item retired (commit): operand free
    uint64_t* d1_full;   // [2] commit
    uint64_t* d1_empty;  // [2] 8 epilogue warps
    uint64_t* a2_full;   // [4] 4 warps of one half
    uint64_t* a2_empty;  // [4] commit
    uint64_t* d2_full;   // [2] commit
    uint64_t* d2_empty;  // [2] 8 epilogue warps
    uint64_t* env_full;  // 8 epilogue warps
    uint64_t* env_free;  // 8 epilogue warps
    uint64_t* fin;       // final commit
};

__global__ void __launch_bounds__(kTcThreads, 1) fd_energyscape_tc_kernel(const FdtcArgs a) {
    extern __shared__ __align__(128) unsigned char sm[];
    uint64_t* bar = reinterpret_cast<uint64_t*>(sm + kOffBar);
    Bars B;
    B.cst = bar + 0;
    B.b1_full = bar + 1;
    B.s1_done = bar + 2;
    B.d1_full = bar + 3;
    B.d1_empty = bar + 5;
    B.a2_full = bar + 7;
    B.a2_empty = bar + 11;
    B.d2_full = bar + 15;
    B.d2_empty = bar + 17;
    B.env_full = bar + 19;
    B.env_free = bar + 20;
    B.fin = bar + 21;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bar + 32);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
    float* hs = reinterpret_cast<float*>(sm + kOffH);
    float* env = reinterpret_cast<float*>(sm + kOffEnv);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int tile = static_cast<int>(blockIdx.x) % kTcTiles;
    const int group = static_cast<int>(blockIdx.x) / kTcTiles;
    const int n_local = group < a.n_items ? (a.n_items - 1 - group) / a.groups + 1 : 0;

    if (tid == 0) {
        ptx::mbar_init(B.cst, 1);
        ptx::mbar_init(B.b1_full, 3);
        ptx::mbar_init(B.s1_done, 1);
        for (int i = 0; i < 2; ++i) {
            ptx::mbar_init(&B.d1_full[i], 1);
            ptx::mbar_init(&B.d1_empty[i], 8);
            ptx::mbar_init(&B.d2_full[i], 1);
            ptx::mbar_init(&B.d2_empty[i], 8);
        }
        for (int i = 0; i < 4; ++i) {
            ptx::mbar_init(&B.a2_full[i], 4);
            ptx::mbar_init(&B.a2_empty[i], 1);
        }
        ptx::mbar_init(B.env_full, 8);
        ptx::mbar_init(B.env_free, 8);
        ptx::mbar_init(B.fin, 1);
        *abort_flag = 0;
        ptx::fence_mbar_init();
        // this tile's stage-1 matrix and the stage-2 matrix, hi and lo, by bulk copies
        ptx::mbar_arrive_expect_tx(B.cst, 2 * kW1Bytes + 2 * kW2Bytes);
        ptx::bulk_load(sm + kOffW1, a.W + static_cast<size_t>(tile) * 2 * kW1Bytes, 2 * kW1Bytes, B.cst);
        ptx::bulk_load(sm + kOffW2, a.W + static_cast<size_t>(kTcTiles) * 2 * kW1Bytes, 2 * kW2Bytes, B.cst);
    }
    for (int j = tid; j < a.lpf_len; j += kTcThreads) hs[j] = a.h[j];
    if (warp == 0) {
        ptx::tmem_alloc(tmem_slot, kTmemCols);
        ptx::tmem_relinquish();
    }
    ptx::tc_fence_before();
    __syncthreads();
    ptx::tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    // bounded wait; gives up early once another role has given up
    auto wait = [&](uint64_t* b, uint32_t parity, bool hinted) -> bool {
        for (uint32_t i = 0; i < kTcPolls; i += 32) {
            if (*abort_flag) return false;
#pragma unroll 1
            for (int k = 0; k < 32; ++k) {
                const bool ok = hinted ? ptx::mbar_wait_hinted(b, parity, 1, kTcHintNs) : ptx::mbar_try_wait(b, parity);
                if (ok) return true;
            }
        }
        *abort_flag = 1;
        atomicOr(a.status, RTIS_DEV_TIMEOUT);
        return false;
    };

    if (warp == 0) {
        // ---------------- MMA issuer ----------------
        if (lane == 0) {
            constexpr uint32_t IDESC1 = ptx::idesc_f16(1u, 128u, 128u);             // N = 64 k2 x (re, im)
            constexpr uint32_t IDESC2 = ptx::idesc_f16(1u, 128u, 2u * kTcN2);       // N = 32 n2 x (re, im)
            bool ok = wait(B.cst, 0, false);
            for (int i = 0; ok && i < n_local; ++i) {
                const int b = i & 1;
                if (!wait(B.b1_full, static_cast<uint32_t>(i & 1), false)) break;
                if (i >= 2 && !wait(&B.d1_empty[b], static_cast<uint32_t>(((i >> 1) - 1) & 1), false)) break;
                ptx::tc_fence_after();
                const uint32_t d1 = tmem + kD1Col + 128u * b;
#pragma unroll 1
                for (int pass = 0; pass < 3; ++pass) {
                    const unsigned char* Ap = sm + kOffW1 + (pass == 2 ? kW1Bytes : 0u);
                    const unsigned char* Bp = sm + kOffB1 + (pass == 1 ? kW1Bytes : 0u);
#pragma unroll
                    for (int ks = 0; ks < 2 * kTcK1 / 16; ++ks) {
                        const uint64_t ad = ptx::smem_desc_kmajor(Ap + ks * 256, 128, kW1Sbo);
                        const uint64_t bd = ptx::smem_desc_kmajor(Bp + ks * 256, 128, kW1Sbo);
                        ptx::tc_mma_f16(d1, ad, bd, IDESC1, (pass | ks) != 0 ? 1u : 0u);
                    }
                }
                ptx::tc_commit(B.s1_done);
                ptx::tc_commit(&B.d1_full[b]);
                if (i >= 2 && !wait(&B.d2_empty[b], static_cast<uint32_t>(((i >> 1) - 1) & 1), false)) break;
                const uint32_t d2 = tmem + kD2Col + 64u * b;
                bool live = true;
#pragma unroll 1
                for (int s = 0; s < kTcP2 / 8; ++s) {
                    const int u = s & 3, m = 2 * i + (s >> 2);
                    if (!wait(&B.a2_full[u], static_cast<uint32_t>(m & 1), false)) {
                        live = false;
                        break;
                    }
                    ptx::tc_fence_after();
                    const unsigned char* slot = sm + kOffA2 + u * kA2Slot;
#pragma unroll
                    for (int pass = 0; pass < 3; ++pass) {
                        const uint64_t ad = ptx::smem_desc_kmajor(slot + (pass == 2 ? kA2Split : 0u), 128, kA2Sbo);
                        const uint64_t bd =
                            ptx::smem_desc_kmajor(sm + kOffW2 + (pass == 1 ? kW2Bytes : 0u) + s * 256, 128, kW2Sbo);
                        ptx::tc_mma_f16(d2, ad, bd, IDESC2, (s | pass) != 0 ? 1u : 0u);
                    }
                    ptx::tc_commit(&B.a2_empty[u]);
                }
                if (!live) break;
                ptx::tc_commit(&B.d2_full[b]);
            }
            // every MMA issued so far has retired before tensor memory is released
            ptx::tc_commit(B.fin);
            ptx::mbar_wait_bounded(B.fin, 0, kTcPolls);
        }
    } else if (warp < kTcEpiWarp0) {
        // ---------------- stage-1 data operand from Y ----------------
        // unit (k2, g): bins k' = 64 (8 g + e) + k2, e < 8 -> rows 2 k2 = [Re | -Im] and
        // 2 k2 + 1 = [Im | Re] (K = [Re k1 0..71 | Im k1 0..71]), core columns g and g + 9.
        // Each thread owns kUnits units; the next item's spectrum is loaded into registers
        // while this item's stage-1 MMAs still read the operand.
        constexpr int kUnits = kTcP2 * (kTcK1 / 8) / kTcLoadThreads;
        static_assert(kUnits * kTcLoadThreads == kTcP2 * (kTcK1 / 8), "units divide evenly");
        const int lt = tid - 32;
        unsigned char* b1 = sm + kOffB1;
        float2 pre[kUnits][8];
        auto fetch = [&](int i) {
            const int item = group + i * a.groups;
            const int d = item / a.T, t = item - d * a.T;
            const float2* Yd = a.Y + static_cast<size_t>(d) * a.Kb * a.T + t;
#pragma unroll
            for (int w = 0; w < kUnits; ++w) {
                const int u = lt + kTcLoadThreads * w;
                const int k2 = u % kTcP2, g = u / kTcP2;
#pragma unroll
                for (int e = 0; e < 8; ++e) {
                    const int k = kTcP2 * (8 * g + e) + k2;
                    pre[w][e] = k < a.Kb ? __ldg(Yd + static_cast<size_t>(k) * a.T) : make_float2(0.f, 0.f);
                }
            }
        };
        if (n_local > 0) fetch(0);
        for (int i = 0; i < n_local; ++i) {
            if (i >= 1 && !wait(B.s1_done, static_cast<uint32_t>((i - 1) & 1), false)) break;
#pragma unroll
            for (int w = 0; w < kUnits; ++w) {
                const int u = lt + kTcLoadThreads * w;
                const int k2 = u % kTcP2, g = u / kTcP2;
                float re[8], im[8], nim[8];
#pragma unroll
                for (int e = 0; e < 8; ++e) {
                    re[e] = pre[w][e].x;
                    im[e] = pre[w][e].y;
                    nim[e] = -pre[w][e].y;
                }
                uint4 h0, l0;
                split8(re, h0, l0);
                st16(b1, w1_off(2 * k2, g), h0);
                st16(b1 + kW1Bytes, w1_off(2 * k2, g), l0);
                st16(b1, w1_off(2 * k2 + 1, g + kTcK1 / 8), h0);
                st16(b1 + kW1Bytes, w1_off(2 * k2 + 1, g + kTcK1 / 8), l0);
                split8(im, h0, l0);
                st16(b1, w1_off(2 * k2 + 1, g), h0);
                st16(b1 + kW1Bytes, w1_off(2 * k2 + 1, g), l0);
                split8(nim, h0, l0);
                st16(b1, w1_off(2 * k2, g + kTcK1 / 8), h0);
                st16(b1 + kW1Bytes, w1_off(2 * k2, g + kTcK1 / 8), l0);
            }
            ptx::fence_proxy_async();
            __syncwarp();
            if (lane == 0) ptx::mbar_arrive(B.b1_full);
            if (i + 1 < n_local) fetch(i + 1);
        }
    } else {
        // ---------------- epilogue: twiddle + stage-2 operand, |b|, low-pass ----------------
        const int we = warp - kTcEpiWarp0;          // 0..7
        const int q = warp & 3, hf = we >> 2;       // TMEM lane quarter, K-step / column half
        const int r = 32 * q + lane;                // row of the tile = TMEM lane
        const int n1 = 128 * tile + r;
        const uint32_t lane_addr = static_cast<uint32_t>(32 * q) << 16;
        // w_F^(k2 n1) for this thread's K-steps s = hf + 2 si (k2 = 8 s + e), exact anchors
        float2 tw[4][8];
#pragma unroll
        for (int si = 0; si < 4; ++si)
#pragma unroll
            for (int e = 0; e < 8; ++e) {
                const int k2 = 8 * (hf + 2 * si) + e;
                const int mph = (k2 * n1) & (kTcN1 * kTcP2 - 1);
                float sn, cs;
                sincospif(static_cast<float>(mph) * (2.0f / (kTcN1 * kTcP2)), &sn, &cs);
                tw[si][e] = make_float2(cs, sn);
            }
        const int half = (a.lpf_len - 1) >> 1;
        // the fold's fixed bounds: thread et serves run f_run = et / 8 (samples f_start .. f_end)
        // and the output bins f_i0, f_i0 + 8, ... below f_i1 whose taps reach into the run
        const int et = tid - 32 * kTcEpiWarp0;
        const int f_run = et >> 3;
        const int f_start = kTcN1 * f_run + 128 * tile;
        const bool run_live = f_start < a.N;
        const int f_end = min(f_start + 127, a.N - 1);
        int f_i0 = 0, f_i1 = 0;
        if (run_live) {
            const int num = f_start + half - (a.lpf_len - 1);  // first bin: R i - half + lpf_len - 1 >= f_start
            f_i0 = (num > 0 ? (num + a.R - 1) / a.R : 0) + (et & 7);
            f_i1 = min(a.n_out, (f_end + half) / a.R + 1);     // last bin: R i - half <= f_end
        }
        bool live = true;
        for (int i = 0; live && i < n_local; ++i) {
            const int b = i & 1;
            const int item = group + i * a.groups;
            const int d = item / a.T, t = item - d * a.T;
            if (!wait(&B.d1_full[b], static_cast<uint32_t>((i >> 1) & 1), false)) break;
            ptx::tc_fence_after();
#pragma unroll
            for (int si = 0; si < 4; ++si) {
                const int s = hf + 2 * si;
                const int u = s & 3, m = 2 * i + (s >> 2);
                if (m >= 1 && !wait(&B.a2_empty[u], static_cast<uint32_t>((m - 1) & 1), false)) {
                    live = false;
                    break;
                }
                uint32_t v[16];
                ptx::tmem_ld_32x32b_x16(tmem + lane_addr + kD1Col + 128u * b + 16u * s, v);
                ptx::tmem_ld_wait_regs16(v);
                float re[8], im[8];
#pragma unroll
                for (int e = 0; e < 8; ++e) {
                    const float x = __uint_as_float(v[2 * e]), y = __uint_as_float(v[2 * e + 1]);
                    const float2 w = tw[si][e];
                    re[e] = fmaf(x, w.x, -y * w.y);
                    im[e] = fmaf(x, w.y, y * w.x);
                }
                unsigned char* slot = sm + kOffA2 + u * kA2Slot;
                const uint32_t off = static_cast<uint32_t>((r >> 3) * kA2Sbo + (r & 7) * 16);
                uint4 h0, l0;
                split8(re, h0, l0);
                st16(slot, off, h0);
                st16(slot + kA2Split, off, l0);
                split8(im, h0, l0);
                st16(slot, off + 128, h0);
                st16(slot + kA2Split, off + 128, l0);
                ptx::fence_proxy_async();
                __syncwarp();
                if (lane == 0) ptx::mbar_arrive(&B.a2_full[u]);
            }
            if (!live) break;
            ptx::tc_fence_before();
            __syncwarp();
            if (lane == 0) ptx::mbar_arrive(&B.d1_empty[b]);
            // |b| of the samples n = 512 n2 + n1, n2 = 16 hf .. 16 hf + 15
            if (i >= 1 && !wait(B.env_free, static_cast<uint32_t>((i - 1) & 1), false)) break;
            if (!wait(&B.d2_full[b], static_cast<uint32_t>((i >> 1) & 1), false)) break;
            ptx::tc_fence_after();
            {
                uint32_t v[32];
                ptx::tmem_ld_32x32b_x32(tmem + lane_addr + kD2Col + 64u * b + 32u * hf, v);
                ptx::tmem_ld_wait_regs(v);
#pragma unroll
                for (int c = 0; c < 16; ++c) {
                    const float x = __uint_as_float(v[2 * c]), y = __uint_as_float(v[2 * c + 1]);
                    env[(16 * hf + c) * kEnvStride + r] = magnitude_from_norm(fmaf(x, x, y * y));
                }
            }
            ptx::tc_fence_before();
            __syncwarp();
            if (lane == 0) {
                ptx::mbar_arrive(&B.d2_empty[b]);
                ptx::mbar_arrive(B.env_full);
            }
            if (!wait(B.env_full, static_cast<uint32_t>(i & 1), false)) break;
            // low-pass over this tile's runs: run n2 = et / 8 holds n in [n_start, n_end]; its eight
            // threads take the output bins touching it in turn (bounds fixed per thread, see above)
            float* Erow = a.E + (static_cast<size_t>(t) * a.D + d) * a.n_out;
            if (run_live) {
#pragma unroll 1
                for (int ib = f_i0, n0 = a.R * f_i0 - half; ib < f_i1; ib += 8, n0 += 8 * a.R) {
                    const int j_lo = max(0, f_start - n0), j_hi = min(a.lpf_len - 1, f_end - n0);
                    const float* er = env + f_run * kEnvStride + (n0 - f_start);
                    float s0 = 0.f, s1 = 0.f, s2 = 0.f, s3 = 0.f;
                    int j = j_lo;
#pragma unroll 2
                    for (; j + 3 <= j_hi; j += 4) {
                        s0 = fmaf(hs[j], er[j], s0);
                        s1 = fmaf(hs[j + 1], er[j + 1], s1);
                        s2 = fmaf(hs[j + 2], er[j + 2], s2);
                        s3 = fmaf(hs[j + 3], er[j + 3], s3);
                    }
                    for (; j <= j_hi; ++j) s0 = fmaf(hs[j], er[j], s0);
                    const float acc = (s0 + s1) + (s2 + s3);
                    if (!isfinite(acc)) atomicOr(a.status, RTIS_DEV_NONFINITE);
                    const int lo = max(0, n0), hi = min(a.N - 1, n0 + a.lpf_len - 1);
                    if (lo >= f_start && hi <= f_end)
                        Erow[ib] = acc;              // every tap in this run: the only contribution
                    else
                        atomicAdd(Erow + ib, acc);   // one of two partial sums
                }
            }
            __syncwarp();
            if (lane == 0) ptx::mbar_arrive(B.env_free);
        }
    }
    ptx::tc_fence_before();
    __syncthreads();
    ptx::tc_fence_after();
    if (warp == 0) ptx::tmem_dealloc(tmem, kTmemCols);
}

// float -> bf16 bits, round to nearest even (finite inputs)
uint16_t host_bf16(float x) {
    uint32_t u;
    std::memcpy(&u, &x, 4);
    u += 0x7FFFu + ((u >> 16) & 1u);
    return static_cast<uint16_t>(u >> 16);
}
float host_bf16_value(uint16_t b) {
    const uint32_t u = static_cast<uint32_t>(b) << 16;
    float x;
    std::memcpy(&x, &u, 4);
    return x;
}
void put_split(unsigned char* hi, unsigned char* lo, uint32_t off, double v) {
    const float x = static_cast<float>(v);
    const uint16_t h = host_bf16(x);
    const uint16_t l = host_bf16(x - host_bf16_value(h));
    std::memcpy(hi + off, &h, 2);
    std::memcpy(lo + off, &l, 2);
}

}  // namespace

bool fdtc_supported(const Plan& p) {
    return p.F == kTcN1 * kTcP2 && p.Kb <= kTcP2 * kTcK1 && p.N <= kTcN1 * kTcN2 && p.lpf_len <= kTcMaxTaps &&
           p.R >= 1 && p.lpf_len <= 128;
}

size_t fdtc_const_bytes() { return kTcConstBytes; }

// The two DFT matrices in the kernel's shared-memory layout, hi and lo BF16:
// per tile the stage-1 rows n1 = 128 tile + r, K = [Re | Im] w512^(k1 n1) for
// k1 < K1 (zeros above), then the stage-2 rows (2 n2, 2 n2 + 1) = ([Re | -Im],
// [Im | Re]) w64^(k2 n2), K-step s holding k2 = 8 s .. 8 s + 7.
void fdtc_build_constants(const Plan& p, std::vector<unsigned char>& img) {
    img.assign(kTcConstBytes, 0);
    const int K1 = (p.Kb + kTcP2 - 1) / kTcP2;
    const double two_pi = 6.283185307179586476925286766559;
    for (int tl = 0; tl < kTcTiles; ++tl) {
        unsigned char* hi = img.data() + static_cast<size_t>(tl) * 2 * kW1Bytes;
        unsigned char* lo = hi + kW1Bytes;
        for (int r = 0; r < 128; ++r) {
            const int n1 = 128 * tl + r;
            for (int k1 = 0; k1 < K1; ++k1) {
                const double ph = two_pi * static_cast<double>((k1 * n1) % kTcN1) / kTcN1;
                const int kr = k1, ki = kTcK1 + k1;
                put_split(hi, lo, w1_off(r, kr >> 3) + (kr & 7) * 2, std::cos(ph));
                put_split(hi, lo, w1_off(r, ki >> 3) + (ki & 7) * 2, std::sin(ph));
            }
        }
    }
    unsigned char* hi = img.data() + static_cast<size_t>(kTcTiles) * 2 * kW1Bytes;
    unsigned char* lo = hi + kW2Bytes;
    auto off2 = [](int row, int K) {
        return static_cast<uint32_t>((row >> 3) * kW2Sbo + (K >> 3) * 128 + (row & 7) * 16 + (K & 7) * 2);
    };
    for (int n2 = 0; n2 < kTcN2; ++n2)
        for (int k2 = 0; k2 < kTcP2; ++k2) {
            const double ph = two_pi * static_cast<double>((k2 * n2) % kTcP2) / kTcP2;
            const double c = std::cos(ph), s = std::sin(ph);
            const int st = k2 >> 3, e = k2 & 7;
            const int Kre = 16 * st + e, Kim = 16 * st + 8 + e;
            put_split(hi, lo, off2(2 * n2, Kre), c);
            put_split(hi, lo, off2(2 * n2, Kim), -s);
            put_split(hi, lo, off2(2 * n2 + 1, Kre), s);
            put_split(hi, lo, off2(2 * n2 + 1, Kim), c);
        }
}

cudaError_t launch_fd_energyscape_tc(const Plan& p, const unsigned char* d_W, const float2* d_Y, int T, float* d_out,
                                     int n_sm, cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(d_out, 0, static_cast<size_t>(T) * p.D * p.n_out * sizeof(float), st);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(fd_energyscape_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             static_cast<int>(kTcSmem));
    if (e != cudaSuccess) return e;
    FdtcArgs a;
    a.Y = d_Y;
    a.W = d_W;
    a.h = p.d_h;
    a.E = d_out;
    a.status = p.d_status;
    a.D = p.D;
    a.T = T;
    a.Kb = p.Kb;
    a.N = p.N;
    a.R = p.R;
    a.lpf_len = p.lpf_len;
    a.n_out = p.n_out;
    a.n_items = p.D * T;
    a.groups = std::max(1, std::min(n_sm / kTcTiles, a.n_items));
    fd_energyscape_tc_kernel<<<a.groups * kTcTiles, kTcThreads, kTcSmem, st>>>(a);
    return cudaGetLastError();
}

}  // namespace rtis
