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

constexpr uint32_t kWaitPolls = 1u << 22;   // bounded mbarrier wait (~ seconds)
constexpr uint32_t kStallPolls = 1u << 12;  // the injected-stall test's short bound

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

// Persistent over a flat list of tiles that may span several sensors (each
// with its own geometry, record length and direction set).  Tile t of sensor
// s covers 8 directions (direction group t % n_dgroups) x one range tile.
// Stages are released without CTA barriers: after a warp finishes a stage it
// bumps that buffer's counter, and the last of the CTA's warps to do so
// issues the TMA refill.  Barrier phases run on across tiles.  Waits are
// bounded; a timeout sets the status word, stops the CTA's compute, and the
// CTA drains its copies before exit.
template <int MS, int NS, bool BF>
__global__ void __launch_bounds__(32 * kTdDirsPerCta, 2)
    td_beamform_kernel(const __grid_constant__ TdMaps maps, const __grid_constant__ TdBatch bt) {
    constexpr int NT = 32 * kTdDirsPerCta;
    constexpr int T = kTdOutPerThread;
    constexpr int ES = BF ? 4 : 8;  // bytes per staged sample
    extern __shared__ __align__(128) unsigned char smem_raw[];
    unsigned char* stage = smem_raw;
    uint64_t* bar = reinterpret_cast<uint64_t*>(smem_raw + static_cast<size_t>(NS) * MS * bt.row_max * 8);
    int* done = reinterpret_cast<int*>(bar + NS);
    int* issued = done + NS;
    float* hs = reinterpret_cast<float*>(issued + NS);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int b = 0; b < NS; ++b) {
            ptx::mbar_init(&bar[b], 1);
            done[b] = 0;
            issued[b] = 0;
        }
        ptx::fence_mbar_init();
        ptx::fence_proxy_async();
    }

    int g0 = 0;  // stages consumed by this CTA before the current tile
    bool timed_out = false;
    const uint32_t polls = bt.stall ? kStallPolls : kWaitPolls;
    bool first_tile = true;
    for (int tile = blockIdx.x; tile < bt.total_tiles; tile += gridDim.x) {
        int si = 0;
        while (si + 1 < bt.n_sensors && tile >= bt.s[si + 1].tile_base) ++si;
        const TdSensor& S = bt.s[si];
        const CUtensorMap* tmap = &maps.m[si];
        const int local = tile - S.tile_base;
        const int dg = local % S.n_dgroups;
        const int d = dg * kTdDirsPerCta + warp;
        const int i0 = (local / S.n_dgroups) * S.bins_per_tile;
        const int half = (S.lpf_len - 1) >> 1;
        const int n_start = S.R * i0 - half;
        // TMA x coordinate: x0 * ES a multiple of 16 bytes
        const int x0 = BF ? ((n_start - S.H) & ~3) : ((n_start - S.H) & ~1);
        const int M = S.M, row = S.row;
        const int nstages = (M + MS - 1) / MS;
        const uint32_t stage_bytes = static_cast<uint32_t>(MS * S.nbox * kTdBox * ES);

        auto issue = [&](int st) {
            const int b = (g0 + st) % NS;
            issued[b] += 1;
            ptx::mbar_arrive_expect_tx(&bar[b], stage_bytes);
            for (int mi = 0; mi < MS; ++mi) {
                unsigned char* dst = stage + static_cast<size_t>(b * MS + mi) * row * ES;
                for (int bx = 0; bx < S.nbox; ++bx)
                    ptx::tma_load_2d(dst + static_cast<size_t>(bx) * kTdBox * ES, tmap, x0 + bx * kTdBox,
                                     st * MS + mi, &bar[b]);
            }
        };

        __syncthreads();  // the previous tile's epilogue is done with the stage buffers and taps
        if (threadIdx.x == 0) {
            ptx::prefetch_tmap(tmap);
            for (int st = 0; st < NS && st < nstages; ++st)
                if (!(bt.stall && first_tile && st == 0)) issue(st);  // injected stall: withhold one copy
        }
        first_tile = false;
        for (int j = threadIdx.x; j < S.lpf_len; j += NT) hs[j] = S.h[j];

        // lane m of each warp holds the steering entry of mic m for this warp's direction
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

        for (int st = 0; st < nstages; ++st) {
            const int b = (g0 + st) % NS;
            if (!timed_out) {
                const uint32_t par = static_cast<uint32_t>(((g0 + st) / NS) & 1);
                if (!ptx::mbar_wait_bounded(&bar[b], par, polls)) {
                    timed_out = true;
                    atomicOr(bt.status, RTIS_DEV_TIMEOUT);
                }
            }
            const bool warp_timed_out = __any_sync(0xffffffffu, timed_out);
            if (dir_ok && !warp_timed_out) {
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
            // release buffer b; the CTA's last warp to get here refills it
            __syncwarp();
            if (lane == 0) {
                __threadfence_block();
                const int prev = atomicAdd(&done[b], 1);
                if (prev == kTdDirsPerCta - 1) {
                    done[b] = 0;
                    __threadfence_block();
                    if (st + NS < nstages && !warp_timed_out) {  // no refills once a wait has given up
                        ptx::fence_proxy_async();
                        issue(st + NS);
                    }
                }
            }
        }
        g0 += nstages;

        if (__syncthreads_or(timed_out)) break;  // uniform: leave the tile loop, drain below

        // epilogue: envelope of this warp's beam over the tile, then low-pass + subsample
        float* env = reinterpret_cast<float*>(smem_raw) + warp * kTdWarpSamples;
#pragma unroll
        for (int t = 0; t < T; ++t) {
            const int n = n_start + lane * T + t;
            const float2 v = unpack2(acc[t]);
            env[lane * T + t] = (n >= 0 && n < S.N) ? magnitude_from_norm(v.x * v.x + v.y * v.y) : 0.f;
        }
        __syncwarp();
        if (dir_ok) {
            // each lane takes bins lane, lane + 32, lane + 64 of a group of 96 in one pass over
            // the taps (each tap loaded once for three bins); lanes past the tile's last bin
            // compute that bin again and discard it
            float* Erow = S.E + static_cast<size_t>(d) * S.n_out;
            const int nb = min(S.bins_per_tile, S.n_out - i0);
            for (int base = 0; base < nb; base += 96) {
                const int il0 = base + lane, il1 = il0 + 32, il2 = il0 + 64;
                const float* e0 = env + S.R * min(il0, nb - 1);
                const float* e1 = env + S.R * min(il1, nb - 1);
                const float* e2 = env + S.R * min(il2, nb - 1);
                float a0 = 0.f, a1 = 0.f, a2 = 0.f;
#pragma unroll 4
                for (int j = 0; j < S.lpf_len; ++j) {
                    const float h = hs[j];
                    a0 = fmaf(h, e0[j], a0);
                    a1 = fmaf(h, e1[j], a1);
                    a2 = fmaf(h, e2[j], a2);
                }
                if (il0 < nb) Erow[i0 + il0] = a0;
                if (il1 < nb) Erow[i0 + il1] = a1;
                if (il2 < nb) Erow[i0 + il2] = a2;
                if ((il0 < nb && !isfinite(a0)) || (il1 < nb && !isfinite(a1)) || (il2 < nb && !isfinite(a2)))
                    atomicOr(bt.status, RTIS_DEV_NONFINITE);
            }
        }
    }

    if (__syncthreads_or(timed_out)) {
        // give copies still in flight a bounded chance to land, then leave
        if (threadIdx.x == 0) {
            for (int b = 0; b < NS; ++b)
                if (issued[b] > 0)
                    ptx::mbar_wait_bounded(&bar[b], static_cast<uint32_t>((issued[b] - 1) & 1), polls);
        }
        __syncthreads();
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

size_t td_smem_bytes(int row_max, int lpf_max) {
    // stage ring (the same bytes for every (mics per stage, stages) variant), then
    // barriers and counters for up to 8 stages, then the low-pass taps
    return static_cast<size_t>(kTdStages) * kTdMicsPerStage * row_max * 8 + 8 * (8 + 4 + 4) +
           static_cast<size_t>(lpf_max) * 4;
}
size_t td_smem_bytes(const Plan& p) { return td_smem_bytes(p.td_row, p.lpf_len); }

namespace {
template <int MS, int NS, bool BF>
cudaError_t td_launch_t(const TdMaps& maps, const TdBatch& bt, int grid, size_t smem, cudaStream_t st) {
    static_assert(MS * NS == kTdMicsPerStage * kTdStages, "variants share one shared-memory size");
    cudaError_t e = cudaFuncSetAttribute(td_beamform_kernel<MS, NS, BF>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
    if (e != cudaSuccess) return e;
    td_beamform_kernel<MS, NS, BF><<<grid, 32 * kTdDirsPerCta, smem, st>>>(maps, bt);
    return cudaGetLastError();
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
    s->n_dgroups = (p.D + kTdDirsPerCta - 1) / kTdDirsPerCta;
    s->tile_base = tile_base;
}

int td_tiles(const Plan& p) {
    return ((p.D + kTdDirsPerCta - 1) / kTdDirsPerCta) * ((p.n_out + p.td_bins_per_tile - 1) / p.td_bins_per_tile);
}

cudaError_t launch_td_batch(const TdMaps& maps, const TdBatch& bt, int variant, int grid, cudaStream_t st) {
    const size_t smem = td_smem_bytes(bt.row_max, bt.lpf_max);
    if (bt.bf16) {
        switch (variant) {
            case 0: return td_launch_t<2, 4, true>(maps, bt, grid, smem, st);
            case 1: return td_launch_t<4, 2, true>(maps, bt, grid, smem, st);
            case 2: return td_launch_t<1, 8, true>(maps, bt, grid, smem, st);
            default: return cudaErrorInvalidValue;
        }
    }
    switch (variant) {
        case 0: return td_launch_t<2, 4, false>(maps, bt, grid, smem, st);
        case 1: return td_launch_t<4, 2, false>(maps, bt, grid, smem, st);
        case 2: return td_launch_t<1, 8, false>(maps, bt, grid, smem, st);
        default: return cudaErrorInvalidValue;
    }
}

// Times every stage layout with one CTA per tile and with two persistent CTAs
// per SM on the plan's own workspace (the timing does not depend on the data)
// and keeps the fastest.
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
    const int grids[2] = {bt.total_tiles, std::min(bt.total_tiles, 2 * n_sm)};
    cudaEvent_t e0, e1;
    cudaError_t e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    if (e != cudaSuccess) return e;
    float best = 1e30f;
    for (int v = 0; v < kTdVariants && e == cudaSuccess; ++v) {
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
