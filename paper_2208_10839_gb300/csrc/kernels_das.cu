// Delay-and-sum beamforming in the time domain with the envelope detector,
// low-pass filter and subsampling fused into its epilogue (paper Fig. 3 and
// Sec. 4.1: one beam per direction of interest, whose envelope is the
// reflector distribution over range; Sec. 4.3: subsampling after the
// envelope detector, filter group delay removed).
//
//   b_d[n] = sum_m sum_{q=-1..2} W[d][m][q] a_m[n + J[d][m] + q]
//   E[d][i] = sum_j h[j] |b_d[R i + j - half]|     (|b| = 0 outside [0, N))
//
// W = g_m * Catmull-Rom weights of mu = delta_dm - floor(delta_dm) and
// J = floor(delta_dm) come from a per-(direction, mic) table built in FP64.
//
// Tiling (one CTA = 8 directions x 960 consecutive samples, one warp per
// direction, each lane 30 consecutive samples):
//   * the channel rows a_m[x0 .. x0 + 960 + 2H) of 2 mics at a time are
//     staged into shared memory by TMA (4-deep mbarrier ring; samples outside
//     [0, N) arrive as zeros from the TMA out-of-bounds fill).  A buffer is
//     refilled by the last warp of the CTA to finish with it, so warps never
//     meet at a CTA barrier inside the mic loop;
//   * each lane loads its 34-sample window as 16-byte pairs (lane stride of
//     30 samples keeps quarter-warps conflict-free) and accumulates the four
//     taps with packed (re, im) FP32 FMAs; per-mic steering values are
//     broadcast across the warp by shuffles;
//   * the epilogue writes |b| for the tile to shared memory and each warp
//     filters and subsamples its own direction, storing E coalesced.
// The tile's 960 samples cover bins_per_tile output bins plus the low-pass
// halo, so no beam sample ever goes to global memory.
#include <algorithm>
#include <cstring>

#include "ptx.cuh"
#include "rtis_internal.h"

namespace rtis {
namespace {

constexpr uint32_t kStallPolls = 1u << 12;  // the injected-stall test's short bound
// the time-domain beamformer's ring waits sleep up to kRingHintNs per poll
// instead of spinning (a poll that spins takes issue slots from the warps
// that have data); bounds: kRingPolls x kRingHintNs ~ 1.3 s, and the stall
// test's kStallPolls x kRingHintNs ~ 80 ms
constexpr uint32_t kRingHintNs = 20000;
constexpr uint32_t kRingPolls = 1u << 16;

__global__ void steering_table_kernel(const float* __restrict__ mic, const float* __restrict__ dirs,
                                      const float* __restrict__ gain, const float* __restrict__ delay_s,
                                      int M, int D, double fs, double fs_over_c, int Jlim, double inv_F,
                                      int* __restrict__ shift, float4* __restrict__ wt,
                                      float2* __restrict__ dphase, float4* __restrict__ wraw,
                                      float4* __restrict__ wder, unsigned* __restrict__ status, int k_c, int Jlim_b,
                                      int* __restrict__ bshift, float4* __restrict__ bwt,
                                      float2* __restrict__ brot) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= M * D) return;
    const int d = idx / M;
    const int m = idx - d * M;
    const double dot = static_cast<double>(mic[3 * m]) * dirs[3 * d] +
                       static_cast<double>(mic[3 * m + 1]) * dirs[3 * d + 1] +
                       static_cast<double>(mic[3 * m + 2]) * dirs[3 * d + 2];
    const double delta = fs * static_cast<double>(delay_s[m]) - fs_over_c * dot;
    const double jf = floor(delta);
    const double mu = delta - jf;
    const double mu2 = mu * mu, mu3 = mu2 * mu;
    const double g = 0.5 * static_cast<double>(gain[m]);
    float4 w = make_float4(static_cast<float>(g * (-mu3 + 2.0 * mu2 - mu)),
                           static_cast<float>(g * (3.0 * mu3 - 5.0 * mu2 + 2.0)),
                           static_cast<float>(g * (-3.0 * mu3 + 4.0 * mu2 + mu)),
                           static_cast<float>(g * (mu3 - mu2)));
    // gain-free weights and their slopes d/dmu, for the adjoint
    float4 wr = make_float4(static_cast<float>(0.5 * (-mu3 + 2.0 * mu2 - mu)),
                            static_cast<float>(0.5 * (3.0 * mu3 - 5.0 * mu2 + 2.0)),
                            static_cast<float>(0.5 * (-3.0 * mu3 + 4.0 * mu2 + mu)),
                            static_cast<float>(0.5 * (mu3 - mu2)));
    float4 wd = make_float4(static_cast<float>(0.5 * (-3.0 * mu2 + 4.0 * mu - 1.0)),
                            static_cast<float>(0.5 * (9.0 * mu2 - 10.0 * mu)),
                            static_cast<float>(0.5 * (-9.0 * mu2 + 8.0 * mu + 1.0)),
                            static_cast<float>(0.5 * (3.0 * mu2 - 2.0 * mu)));
    int j = 0;
    if (fabs(jf) <= static_cast<double>(Jlim)) {
        j = static_cast<int>(jf);
    } else {  // outside the staged halo (or not finite): contribute nothing, report
        atomicOr(status, RTIS_DEV_DELAY_RANGE);
        w = make_float4(0.f, 0.f, 0.f, 0.f);
        wr = w;
        wd = w;
    }
    shift[idx] = j;
    wt[idx] = w;
    wraw[idx] = wr;
    wder[idx] = wd;
    // frequency-domain form: delta / F cycles per bin, as an unevaluated pair hi + lo
    const double dp = delta * inv_F;
    const float dp_hi = static_cast<float>(dp);
    dphase[idx] = make_float2(dp_hi, static_cast<float>(dp - dp_hi));
    if (bshift) {
        // baseband form: Catmull-Rom on the coarse grid at delta / 4, and the carrier's
        // phase 2 pi k_c delta / F (cycles reduced to [0, 1) before the sine)
        const double u = 0.25 * delta;
        const double jb = floor(u);
        const double nu = u - jb, nu2 = nu * nu, nu3 = nu2 * nu;
        float4 bw = make_float4(static_cast<float>(0.5 * (-nu3 + 2.0 * nu2 - nu)),
                                static_cast<float>(0.5 * (3.0 * nu3 - 5.0 * nu2 + 2.0)),
                                static_cast<float>(0.5 * (-3.0 * nu3 + 4.0 * nu2 + nu)),
                                static_cast<float>(0.5 * (nu3 - nu2)));
        double cyc = static_cast<double>(k_c) * dp;
        cyc -= floor(cyc);
        double sn, cs;
        sincospi(2.0 * cyc, &sn, &cs);
        const double gm = static_cast<double>(gain[m]);
        float2 r = make_float2(static_cast<float>(gm * cs), static_cast<float>(gm * sn));
        int jbi = 0;
        if (fabs(jb) <= static_cast<double>(Jlim_b)) {
            jbi = static_cast<int>(jb);
        } else {
            atomicOr(status, RTIS_DEV_DELAY_RANGE);
            bw = make_float4(0.f, 0.f, 0.f, 0.f);
            r = make_float2(0.f, 0.f);
        }
        bshift[idx] = jbi;
        bwt[idx] = bw;
        brot[idx] = r;
    }
}

using ptx::fma2;
using ptx::pack2;
using ptx::unpack2;

// One mic's contribution to a lane's T samples.  `p` points at the 16-byte
// aligned pair holding the first tap (or the sample before it when ODD).
template <bool ODD>
__device__ __forceinline__ void td_mic(uint64_t (&acc)[kTdOutPerThread], const ulonglong2* __restrict__ p,
                                       uint64_t w0, uint64_t w1, uint64_t w2, uint64_t w3) {
    constexpr int T = kTdOutPerThread;
    constexpr int NP = (T + 4) / 2;  // pairs covering T + 3 taps from an even start
    uint64_t v[2 * NP];
#pragma unroll
    for (int k = 0; k < NP; ++k) {
        const ulonglong2 q = p[k];
        v[2 * k] = q.x;
        v[2 * k + 1] = q.y;
    }
    // blocks of TB outputs: consecutive FMAs hit different accumulators, and
    // the window is consumed in the order its loads were issued
    constexpr int TB = 6;
    static_assert(T % TB == 0, "T must be a multiple of the FMA block");
#pragma unroll
    for (int tb = 0; tb < T; tb += TB) {
#pragma unroll
        for (int t = tb; t < tb + TB; ++t) fma2(acc[t], w0, v[t + ODD]);
#pragma unroll
        for (int t = tb; t < tb + TB; ++t) fma2(acc[t], w1, v[t + 1 + ODD]);
#pragma unroll
        for (int t = tb; t < tb + TB; ++t) fma2(acc[t], w2, v[t + 2 + ODD]);
#pragma unroll
        for (int t = tb; t < tb + TB; ++t) fma2(acc[t], w3, v[t + 3 + ODD]);
    }
}

// The same with BF16 (re, im) pairs staged, 4 bytes per sample: `p` points at
// the 8-byte aligned pair of samples holding the first tap (or the sample
// before it when ODD); each sample widens to FP32 exactly (BF16 is the top
// half of an FP32) before the packed FMAs.
__device__ __forceinline__ uint64_t widen_bf16x2(uint32_t u) {
    return pack2(__uint_as_float(u << 16), __uint_as_float(u & 0xffff0000u));
}
template <bool ODD>
__device__ __forceinline__ void td_mic_bf16(uint64_t (&acc)[kTdOutPerThread], const uint2* __restrict__ p,
                                            uint64_t w0, uint64_t w1, uint64_t w2, uint64_t w3) {
    constexpr int T = kTdOutPerThread;
    constexpr int NP = (T + 4) / 2;
    uint64_t v[2 * NP];
#pragma unroll
    for (int k = 0; k < NP; ++k) {
        const uint2 q = p[k];
        v[2 * k] = widen_bf16x2(q.x);
        v[2 * k + 1] = widen_bf16x2(q.y);
    }
    constexpr int TB = 6;
#pragma unroll
    for (int tb = 0; tb < T; tb += TB) {
#pragma unroll
        for (int t = tb; t < tb + TB; ++t) fma2(acc[t], w0, v[t + ODD]);
#pragma unroll
        for (int t = tb; t < tb + TB; ++t) fma2(acc[t], w1, v[t + 1 + ODD]);
#pragma unroll
        for (int t = tb; t < tb + TB; ++t) fma2(acc[t], w2, v[t + 2 + ODD]);
#pragma unroll
        for (int t = tb; t < tb + TB; ++t) fma2(acc[t], w3, v[t + 3 + ODD]);
    }
}

// The low-pass and subsampling of one warp's beam, straight from the lanes'
// accumulators, for R = 10 and the 41-tap filter (half = 20): lane l holds the
// tile samples p = 30 l + t (t < 30), and output bin il of the tile sits at
// p = 10 il + 20 with taps h[p - 10 il], p - 10 il in [0, 40].  Each lane forms
// the partial sums P_k = sum_t h[t - 10 k] |b[30 l + t]| of the seven bins
// il = 3 l + k (k = -4 .. 2) its samples touch, and owns bins 3 l, 3 l + 1,
// 3 l + 2: E(3l) = P_0 + P_-3 of lane l+1, E(3l+1) = P_1 + P_-2 of lane l+1,
// E(3l+2) = P_2 + P_-1 of lane l+1 + P_-4 of lane l+2.  No shared memory, no
// barrier.
constexpr int kFastR = 10, kFastTaps = 41;
static_assert(kTdOutPerThread == 3 * kFastR, "the register epilogue assumes 30 samples per lane");
__device__ __forceinline__ void td_epilogue_fast(const uint64_t (&acc)[kTdOutPerThread], int lane, int n_start, int N,
                                                 const float* __restrict__ h, float* __restrict__ Erow, int i0,
                                                 int nb, unsigned* status) {
    constexpr int T = kTdOutPerThread;
    float env[T];
#pragma unroll
    for (int t = 0; t < T; ++t) {
        const int n = n_start + lane * T + t;
        const float2 v = ptx::unpack2(acc[t]);
        env[t] = (n >= 0 && n < N) ? magnitude_from_norm(v.x * v.x + v.y * v.y) : 0.f;
    }
    float hr[kFastTaps];
#pragma unroll
    for (int j = 0; j < kFastTaps; ++j) hr[j] = __ldg(h + j);
    float P[7];  // P[k + 4], k = -4 .. 2
#pragma unroll
    for (int k = -4; k <= 2; ++k) {
        float a = 0.f;
#pragma unroll
        for (int t = 0; t < T; ++t) {
            const int j = t - kFastR * k;
            if (j >= 0 && j < kFastTaps) a = fmaf(hr[j], env[t], a);
        }
        P[k + 4] = a;
    }
    const float n1m3 = __shfl_down_sync(0xffffffffu, P[1], 1);  // P_-3 of lane + 1
    const float n1m2 = __shfl_down_sync(0xffffffffu, P[2], 1);  // P_-2 of lane + 1
    const float n1m1 = __shfl_down_sync(0xffffffffu, P[3], 1);  // P_-1 of lane + 1
    const float n2m4 = __shfl_down_sync(0xffffffffu, P[0], 2);  // P_-4 of lane + 2
    const float e0 = P[4] + n1m3;
    const float e1 = P[5] + n1m2;
    const float e2 = (P[6] + n1m1) + n2m4;
    const int il = 3 * lane;
    if (il < nb) Erow[i0 + il] = e0;
    if (il + 1 < nb) Erow[i0 + il + 1] = e1;
    if (il + 2 < nb) Erow[i0 + il + 2] = e2;
    if ((il < nb && !isfinite(e0)) || (il + 1 < nb && !isfinite(e1)) || (il + 2 < nb && !isfinite(e2)))
        atomicOr(status, RTIS_DEV_NONFINITE);
}

// Any R and filter length: |b| of the warp's tile samples into the warp's own
// row of shared memory, then each lane filters bins lane, lane + 32, lane + 64
// of each group of 96 in one pass over the taps.
__device__ __forceinline__ void td_epilogue_generic(const uint64_t (&acc)[kTdOutPerThread], int lane, int n_start,
                                                    const TdSensor& S, float* __restrict__ env, float* __restrict__ Erow,
                                                    int i0, int nb, unsigned* status) {
    constexpr int T = kTdOutPerThread;
#pragma unroll
    for (int t = 0; t < T; ++t) {
        const int n = n_start + lane * T + t;
        const float2 v = ptx::unpack2(acc[t]);
        env[lane * T + t] = (n >= 0 && n < S.N) ? magnitude_from_norm(v.x * v.x + v.y * v.y) : 0.f;
    }
    __syncwarp();
    for (int base = 0; base < nb; base += 96) {
        const int il0 = base + lane, il1 = il0 + 32, il2 = il0 + 64;
        const float* e0 = env + S.R * min(il0, nb - 1);
        const float* e1 = env + S.R * min(il1, nb - 1);
        const float* e2 = env + S.R * min(il2, nb - 1);
        float a0 = 0.f, a1 = 0.f, a2 = 0.f;
#pragma unroll 4
        for (int j = 0; j < S.lpf_len; ++j) {
            const float h = __ldg(S.h + j);
            a0 = fmaf(h, e0[j], a0);
            a1 = fmaf(h, e1[j], a1);
            a2 = fmaf(h, e2[j], a2);
        }
        if (il0 < nb) Erow[i0 + il0] = a0;
        if (il1 < nb) Erow[i0 + il1] = a1;
        if (il2 < nb) Erow[i0 + il2] = a2;
        if ((il0 < nb && !isfinite(a0)) || (il1 < nb && !isfinite(a1)) || (il2 < nb && !isfinite(a2)))
            atomicOr(status, RTIS_DEV_NONFINITE);
    }
    __syncwarp();  // the row is rewritten by the warp's next tile
}

// Five warpgroups, one CTA per SM: warps 0..15 beamform one direction each,
// warp 16 is the producer and warps 17..19 only hand their registers back.
// At launch every thread holds 96 registers (640 x 96 fit the SM); the
// producer warpgroup then drops to kTdProducerRegs and the consumers rise to
// kTdConsumerRegs, within the block's launch allocation
// (512 x 112 + 128 x 24 <= 640 x 96).
// Persistent over a flat list of tiles that may span several sensors (each
// with its own geometry, record length and direction set).  Tile t of sensor
// s covers 16 directions (direction group t % n_dgroups) x one range tile.
// The producer  The producer walks the CTA's tiles and stages, waits until a
// buffer's previous contents were released by all eight consumers (its
// "empty" mbarrier), then re-arms the buffer's "full" mbarrier and issues the
// TMA boxes (one lane per box).  The ring runs on across tile boundaries, so
// the next tile's first stages land while the consumers are still in this
// tile's epilogue, and nothing waits at a CTA barrier after the start.
// Every wait is bounded: a timeout sets the status word and the CTA's abort
// flag, the producer stops issuing, and the producer lets every copy it
// issued land before it exits.
template <int MS, int NS, bool BF, bool FAST>
__global__ void __launch_bounds__(kTdThreads, 1)
    td_beamform_kernel(const __grid_constant__ TdMaps maps, const __grid_constant__ TdBatch bt) {
    constexpr int NW = kTdWarps;  // consumer warps
    constexpr int T = kTdOutPerThread;
    constexpr int ES = BF ? 4 : 8;  // bytes per staged sample
    extern __shared__ __align__(128) unsigned char smem_raw[];
    unsigned char* stage = smem_raw;
    const size_t ring_bytes = static_cast<size_t>(NS) * MS * bt.row_max * 8;
    uint64_t* full = reinterpret_cast<uint64_t*>(smem_raw + ring_bytes);
    uint64_t* empty = full + NS;
    int* abort_flag = reinterpret_cast<int*>(empty + NS);
    int* issued = abort_flag + 1;  // [NS]: uses of each buffer issued so far (producer only)
    float* env_all = reinterpret_cast<float*>(smem_raw + ring_bytes + kTdBarrierBytes);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int b = 0; b < NS; ++b) {
            ptx::mbar_init(&full[b], 1);
            ptx::mbar_init(&empty[b], NW);
            issued[b] = 0;
        }
        *abort_flag = 0;
        ptx::fence_mbar_init();
        ptx::fence_proxy_async();
    }
    __syncthreads();
    volatile int* vabort = abort_flag;
    const uint32_t polls = bt.stall ? kStallPolls : kRingPolls;

    if (warp >= NW) {
        // ---------------- producer warpgroup: warp NW issues, the other three leave ----------------
        ptx::setmaxnreg_dec<kTdProducerRegs>();
        if (warp != NW) return;
        int g = 0;  // stages issued (or skipped) by this CTA so far
        bool stop = false;
        for (int tile = blockIdx.x; tile < bt.total_tiles && !stop; tile += gridDim.x) {
            int si = 0;
            while (si + 1 < bt.n_sensors && tile >= bt.s[si + 1].tile_base) ++si;
            const TdSensor& S = bt.s[si];
            const CUtensorMap* tmap = &maps.m[si];
            const int local = tile - S.tile_base;
            const int i0 = (local / S.n_dgroups) * S.bins_per_tile;
            const int n_start = S.R * i0 - ((S.lpf_len - 1) >> 1);
            // TMA x coordinate: x0 * ES a multiple of 16 bytes
            const int x0 = BF ? ((n_start - S.H) & ~3) : ((n_start - S.H) & ~1);
            const int nstages = (S.M + MS - 1) / MS;
            const uint32_t stage_bytes = static_cast<uint32_t>(MS * S.nbox * kTdBox * ES);
            if (lane == 0) ptx::prefetch_tmap(tmap);
            for (int st = 0; st < nstages; ++st, ++g) {
                const int b = g % NS;
                const int use = g / NS;
                const bool skip = bt.stall && g == 0;  // injected stall: withhold the CTA's first copy
                int ok = 1;
                if (lane == 0) {
                    if (*vabort) {
                        ok = 0;
                    } else if (use > 0 && !ptx::mbar_wait_hinted(&empty[b], static_cast<uint32_t>((use - 1) & 1), polls,
                                                                 kRingHintNs)) {
                        ok = 0;
                        atomicOr(bt.status, RTIS_DEV_TIMEOUT);
                        *vabort = 1;
                    }
                    if (ok && !skip) {
                        ptx::fence_proxy_async();
                        ptx::mbar_arrive_expect_tx(&full[b], stage_bytes);
                        issued[b] = use + 1;
                    }
                }
                ok = __shfl_sync(0xffffffffu, ok, 0);
                if (!ok) {
                    stop = true;
                    break;
                }
                if (!skip) {
                    for (int j = lane; j < MS * S.nbox; j += 32) {
                        const int mi = j / S.nbox;
                        const int bx = j - mi * S.nbox;
                        unsigned char* dst = stage + (static_cast<size_t>(b * MS + mi) * S.row + bx * kTdBox) * ES;
                        ptx::tma_load_2d(dst, tmap, x0 + bx * kTdBox, st * MS + mi, &full[b]);
                    }
                }
            }
        }
        // every copy this CTA issued lands before the CTA can exit
        if (lane == 0) {
            for (int b = 0; b < NS; ++b)
                if (issued[b] > 0)
                    ptx::mbar_wait_hinted(&full[b], static_cast<uint32_t>((issued[b] - 1) & 1), polls, kRingHintNs);
        }
        return;
    }

    // ---------------- consumers: warp = direction within the tile ----------------
    ptx::setmaxnreg_inc<kTdConsumerRegs>();
    int g = 0;
    for (int tile = blockIdx.x; tile < bt.total_tiles; tile += gridDim.x) {
        int si = 0;
        while (si + 1 < bt.n_sensors && tile >= bt.s[si + 1].tile_base) ++si;
        const TdSensor& S = bt.s[si];
        const int local = tile - S.tile_base;
        const int dg = local % S.n_dgroups;
        const int d = dg * NW + warp;
        const int i0 = (local / S.n_dgroups) * S.bins_per_tile;
        const int n_start = S.R * i0 - ((S.lpf_len - 1) >> 1);
        const int x0 = BF ? ((n_start - S.H) & ~3) : ((n_start - S.H) & ~1);
        const int M = S.M, row = S.row;
        const int nstages = (M + MS - 1) / MS;

        // lane m holds the steering entry of mic m for this warp's direction
        const bool dir_ok = d < S.D;
        int my_shift = 0;
        float4 my_w = make_float4(0.f, 0.f, 0.f, 0.f);
        if (dir_ok && lane < M) {
            my_shift = __ldg(S.shift + static_cast<size_t>(d) * M + lane);
            my_w = __ldg(S.wt + static_cast<size_t>(d) * M + lane);
        }

        uint64_t acc[T];
#pragma unroll
        for (int t = 0; t < T; ++t) acc[t] = 0ull;
        const int lane_base = n_start - x0 + lane * T - 1;  // smem index of a[n_start + lane*T - 1]

        bool failed = false;
        for (int st = 0; st < nstages; ++st, ++g) {
            const int b = g % NS;
            const uint32_t par = static_cast<uint32_t>((g / NS) & 1);
            bool ok = !*vabort && ptx::mbar_wait_hinted(&full[b], par, polls, kRingHintNs);
            if (!__all_sync(0xffffffffu, ok)) {
                failed = true;
                break;
            }
            // every warp runs the mic loop: a direction past the set's end has zero
            // weights and shift, so it reads inside the staged row and sums zeros (a
            // branch around the loop costs the compiler's scheduling of it ~15 %)
            {
#pragma unroll
                for (int mi = 0; mi < MS; ++mi) {
                    const int m = st * MS + mi;
                    if (m >= M) break;
                    const int J = __shfl_sync(0xffffffffu, my_shift, m);
                    const float f0 = __shfl_sync(0xffffffffu, my_w.x, m);
                    const float f1 = __shfl_sync(0xffffffffu, my_w.y, m);
                    const float f2 = __shfl_sync(0xffffffffu, my_w.z, m);
                    const float f3 = __shfl_sync(0xffffffffu, my_w.w, m);
                    const int s0 = lane_base + J;  // parity is warp-uniform (T even)
                    const unsigned char* rowp = stage + (static_cast<size_t>(b * MS + mi) * row + (s0 & ~1)) * ES;
                    if constexpr (BF) {
                        const uint2* p = reinterpret_cast<const uint2*>(rowp);
                        if (s0 & 1)
                            td_mic_bf16<true>(acc, p, pack2(f0, f0), pack2(f1, f1), pack2(f2, f2), pack2(f3, f3));
                        else
                            td_mic_bf16<false>(acc, p, pack2(f0, f0), pack2(f1, f1), pack2(f2, f2), pack2(f3, f3));
                    } else {
                        const ulonglong2* p = reinterpret_cast<const ulonglong2*>(rowp);
                        if (s0 & 1)
                            td_mic<true>(acc, p, pack2(f0, f0), pack2(f1, f1), pack2(f2, f2), pack2(f3, f3));
                        else
                            td_mic<false>(acc, p, pack2(f0, f0), pack2(f1, f1), pack2(f2, f2), pack2(f3, f3));
                    }
                }
            }
            __syncwarp();
            if (lane == 0) ptx::mbar_arrive(&empty[b]);  // the producer may refill buffer b
        }
        if (failed) {
            if (lane == 0) {
                if (!*vabort) atomicOr(bt.status, RTIS_DEV_TIMEOUT);
                *vabort = 1;
            }
            break;
        }
        // every warp runs the epilogue too (branch-free around acc, as for the mic loop);
        // a direction past the set's end stores nothing (nb = 0)
        {
            float* Erow = S.E + static_cast<size_t>(dir_ok ? d : 0) * S.n_out;
            const int nb = dir_ok ? min(S.bins_per_tile, S.n_out - i0) : 0;
            if constexpr (FAST)
                td_epilogue_fast(acc, lane, n_start, S.N, S.h, Erow, i0, nb, bt.status);
            else
                td_epilogue_generic(acc, lane, n_start, S, env_all + warp * kTdWarpSamples, Erow, i0, nb, bt.status);
        }
    }
}

}  // namespace

cudaError_t launch_steering_table(Plan& p, cudaStream_t st) {
    const int total = p.M * p.D;
    const int nt = 256;
    steering_table_kernel<<<(total + nt - 1) / nt, nt, 0, st>>>(p.d_mic, p.d_dirs, p.d_gain, p.d_delay, p.M, p.D,
                                                              p.fs, p.fs / p.c, p.Jlim, 1.0 / p.F, p.d_shift,
                                                              p.d_wt, p.d_dphase, p.d_wraw, p.d_wder, p.d_status,
                                                              p.k_c, p.bb_Jlim, p.d_bshift, p.d_bwt, p.d_brot);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) p.table_dirty = false;
    return e;
}

bool td_fast_epilogue(int R, int lpf_len) { return R == kFastR && lpf_len == kFastTaps; }

namespace {
constexpr int kTdLayouts[kTdVariants][2] = {{2, 8}, {4, 4}, {2, 10}, {4, 5}, {1, 8}};
}  // namespace
int td_variant_ms(int v) { return kTdLayouts[v][0]; }
int td_variant_ns(int v) { return kTdLayouts[v][1]; }

size_t td_smem_bytes(int row_max, bool fast, int variant) {
    // stage ring, then barriers, flags and counters, then (any other low-pass) one
    // envelope row per consumer warp
    return static_cast<size_t>(td_variant_ms(variant)) * td_variant_ns(variant) * row_max * 8 + kTdBarrierBytes +
           (fast ? 0 : static_cast<size_t>(kTdWarps) * kTdWarpSamples * 4);
}
bool td_variant_fits(int row_max, bool fast, int variant) {
    return variant >= 0 && variant < kTdVariants && td_smem_bytes(row_max, fast, variant) <= 227 * 1024;
}
size_t td_smem_bytes(const Plan& p) { return td_smem_bytes(p.td_row, td_fast_epilogue(p.R, p.lpf_len), kTdVariants - 1); }

namespace {
template <int MS, int NS, bool BF, bool FAST>
cudaError_t td_launch_t(const TdMaps& maps, const TdBatch& bt, int grid, size_t smem, cudaStream_t st) {
    static_assert(16 * NS + 4 * (NS + 1) <= kTdBarrierBytes, "barrier area");
    cudaError_t e = cudaFuncSetAttribute(td_beamform_kernel<MS, NS, BF, FAST>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
    if (e != cudaSuccess) return e;
    td_beamform_kernel<MS, NS, BF, FAST><<<grid, kTdThreads, smem, st>>>(maps, bt);
    return cudaGetLastError();
}
template <bool BF, bool FAST>
cudaError_t td_launch_v(const TdMaps& maps, const TdBatch& bt, int variant, int grid, size_t smem, cudaStream_t st) {
    switch (variant) {
        case 0: return td_launch_t<2, 8, BF, FAST>(maps, bt, grid, smem, st);
        case 1: return td_launch_t<4, 4, BF, FAST>(maps, bt, grid, smem, st);
        case 2: return td_launch_t<2, 10, BF, FAST>(maps, bt, grid, smem, st);
        case 3: return td_launch_t<4, 5, BF, FAST>(maps, bt, grid, smem, st);
        case 4: return td_launch_t<1, 8, BF, FAST>(maps, bt, grid, smem, st);
        default: return cudaErrorInvalidValue;
    }
}
}  // namespace

void td_fill_sensor(const Plan& p, float* d_out, int tile_base, TdSensor* s) {
    s->shift = p.d_shift;
    s->wt = p.d_wt;
    s->h = p.d_h;
    s->E = d_out;
    s->M = p.M;
    s->N = p.N;
    s->D = p.D;
    s->R = p.R;
    s->lpf_len = p.lpf_len;
    s->n_out = p.n_out;
    s->H = p.H;
    s->row = p.td_row;
    s->nbox = p.td_nbox;
    s->bins_per_tile = p.td_bins_per_tile;
    s->n_dgroups = (p.D + kTdWarps - 1) / kTdWarps;
    s->tile_base = tile_base;
}

int td_tiles(const Plan& p) {
    return ((p.D + kTdWarps - 1) / kTdWarps) * ((p.n_out + p.td_bins_per_tile - 1) / p.td_bins_per_tile);
}

cudaError_t launch_td_batch(const TdMaps& maps, const TdBatch& bt, int variant, int grid, cudaStream_t st) {
    bool fast = true;
    for (int i = 0; i < bt.n_sensors; ++i) fast = fast && td_fast_epilogue(bt.s[i].R, bt.s[i].lpf_len);
    if (!td_variant_fits(bt.row_max, fast, variant)) return cudaErrorInvalidValue;
    const size_t smem = td_smem_bytes(bt.row_max, fast, variant);
    grid = std::max(1, std::min(grid, bt.total_tiles));
    if (bt.bf16) return fast ? td_launch_v<true, true>(maps, bt, variant, grid, smem, st)
                             : td_launch_v<true, false>(maps, bt, variant, grid, smem, st);
    return fast ? td_launch_v<false, true>(maps, bt, variant, grid, smem, st)
                : td_launch_v<false, false>(maps, bt, variant, grid, smem, st);
}

// Times every stage layout that fits shared memory with one CTA per tile and
// with one persistent CTA per SM on the plan's own workspace (the timing does
// not depend on the data) and keeps the fastest.
cudaError_t td_autotune(Plan& p, float* d_scratch_out) {
    TdMaps maps;
    maps.m[0] = p.a_bf16 ? p.tmap_a16 : p.tmap_a;
    TdBatch bt;
    std::memset(&bt, 0, sizeof(bt));
    bt.bf16 = p.a_bf16 ? 1 : 0;
    td_fill_sensor(p, d_scratch_out, 0, &bt.s[0]);
    bt.n_sensors = 1;
    bt.total_tiles = td_tiles(p);
    bt.row_max = p.td_row;
    bt.lpf_max = p.lpf_len;
    bt.status = p.d_status;
    int n_sm = 1, dev = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) n_sm = 1;
    // [2v]: one CTA per tile; [2v + 1]: one persistent CTA per SM
    const int grids[2] = {bt.total_tiles, std::min(bt.total_tiles, n_sm)};
    const bool fast = td_fast_epilogue(p.R, p.lpf_len);
    cudaEvent_t e0, e1;
    cudaError_t e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    if (e != cudaSuccess) return e;
    float best = 1e30f;
    for (int v = 0; v < kTdVariants && e == cudaSuccess; ++v) {
        if (!td_variant_fits(p.td_row, fast, v)) continue;
        for (int gi = 0; gi < 2 && e == cudaSuccess; ++gi) {
            e = launch_td_batch(maps, bt, v, grids[gi], 0);  // warm-up
            float total = 0.f;
            for (int r = 0; r < 2 && e == cudaSuccess; ++r) {
                cudaEventRecord(e0, 0);
                e = launch_td_batch(maps, bt, v, grids[gi], 0);
                cudaEventRecord(e1, 0);
                if (e == cudaSuccess) e = cudaEventSynchronize(e1);
                float ms = 0.f;
                if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
                total += ms;
            }
            if (e == cudaSuccess) p.td_variant_ms[2 * v + gi] = total / 2.f;
            if (e == cudaSuccess && total < best) {
                best = total;
                p.td_variant = v;
                p.td_grid = grids[gi];
            }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    p.td_tuned_ms = best / 2.f;
    return e;
}

cudaError_t launch_td_beamform(const Plan& p, const CUtensorMap& tmap, bool bf16, float* d_out, cudaStream_t st) {
    TdMaps maps;
    maps.m[0] = tmap;
    TdBatch bt;
    std::memset(&bt, 0, sizeof(bt));
    bt.bf16 = bf16 ? 1 : 0;
    bt.stall = (fault_mode() == kFaultStall) ? 1 : 0;
    td_fill_sensor(p, d_out, 0, &bt.s[0]);
    bt.n_sensors = 1;
    bt.total_tiles = td_tiles(p);
    bt.row_max = p.td_row;
    bt.lpf_max = p.lpf_len;
    bt.status = p.d_status;
    return launch_td_batch(maps, bt, p.td_variant, p.td_grid > 0 ? p.td_grid : bt.total_tiles, st);
}

}  // namespace rtis
