// Complex-baseband delay-and-sum -> energyscape.  The paper subsamples the
// recording before its filters (Sec. 4.3); here the subsampling follows the
// matched filter instead, on the analytic signal demodulated to 0 Hz, where
// the 60 kHz band leaves room for a grid 4x coarser than the recording's:
//
//   z_m[j]  = a_m[4j] exp(-2 pi i k_c 4j / F)            (mf_inverse_kernel, phase 0 only)
//   b_d[j]  = sum_m r_dm sum_{q=-1..2} w_q(mu_dm) z_m[j + J_dm + q]
//             J_dm = floor(delta_dm / 4), mu_dm = delta_dm / 4 - J_dm (Catmull-Rom),
//             r_dm = g_m exp(+2 pi i k_c delta_dm / F): the carrier's exact phase
//   E[d][i] = sum_j h_i(4j - R i) |b_d[j]|: the plan's low-pass taps read at
//             the coarse offsets from R i, renormalised to unit DC gain
//
// The layout follows the time-domain beamformer: one persistent CTA per SM of
// 16 direction warps and a producer warpgroup; a CTA tile is 16 directions x
// one range tile of 32 lanes x 14 coarse samples.  Channel rows arrive by TMA
// through a full/empty mbarrier ring of NS stages x MS mics that runs across
// tile boundaries; the envelope, low-pass and subsampling run in the epilogue
// out of a shared-memory row per warp.  Per mic and coarse sample a lane forms
// s = sum_q w_q z (one packed multiply and three packed FMAs on (re, im)) and
// accumulates cr * s and ci * s (two packed FMAs), r = cr + i ci; the beam is
// (acc_c.re - acc_s.im, acc_c.im + acc_s.re).  That is 6 packed FMAs per
// (mic, coarse sample) against 4 per (mic, sample) on the full-rate grid:
// 2.7x fewer.  Every wait is bounded as in the other kernels.
#include <algorithm>
#include <cstring>

#include "ptx.cuh"
#include "rtis_internal.h"

namespace rtis {
namespace {

// coarse low-pass taps per residue class for R = 10 and the 41-tap filter
constexpr int kBbFastTaps = 11;

using ptx::fma2;
using ptx::mul2;
using ptx::pack2;
using ptx::unpack2;

// ring waits sleep up to kBbHintNs per poll; kBbPolls x kBbHintNs ~ 1.3 s bounds a wait
constexpr uint32_t kBbHintNs = 20000;
constexpr uint32_t kBbPolls = 1u << 16;

struct BbArgs {
    const int* shift;    // [D][M]
    const float4* wt;    // [D][M]
    const float2* rot;   // [D][M]
    const float* hb;     // [4][ntap]
    float* E;            // [D][n_out]
    unsigned* status;
    int M, Nb, D, R, half, n_out, bins_per_tile, n_dgroups, total_tiles, H, row, nbox, ntap;
    uint32_t stage_area;  // bytes of the stage ring; barriers, envelope rows and taps follow it
};

// one mic's contribution to a lane's T coarse samples; p points at the 16-byte
// aligned pair holding the first tap (or the sample before it when ODD)
template <bool ODD>
__device__ __forceinline__ void bb_mic(uint64_t (&ac)[kBbOutPerThread], uint64_t (&as)[kBbOutPerThread],
                                       const ulonglong2* __restrict__ p, uint64_t w0, uint64_t w1, uint64_t w2,
                                       uint64_t w3, uint64_t rc, uint64_t rs) {
    constexpr int T = kBbOutPerThread;
    constexpr int NP = (T + 4) / 2;
    uint64_t v[2 * NP];
#pragma unroll
    for (int k = 0; k < NP; ++k) {
        const ulonglong2 q = p[k];
        v[2 * k] = q.x;
        v[2 * k + 1] = q.y;
    }
    // blocks of TB samples, tap by tap: consecutive instructions are independent
    constexpr int TB = 7;
    static_assert(T % TB == 0, "T must be a multiple of the block");
#pragma unroll
    for (int tb = 0; tb < T; tb += TB) {
        uint64_t s[TB];
#pragma unroll
        for (int t = 0; t < TB; ++t) s[t] = mul2(w0, v[tb + t + ODD]);
#pragma unroll
        for (int t = 0; t < TB; ++t) fma2(s[t], w1, v[tb + t + 1 + ODD]);
#pragma unroll
        for (int t = 0; t < TB; ++t) fma2(s[t], w2, v[tb + t + 2 + ODD]);
#pragma unroll
        for (int t = 0; t < TB; ++t) fma2(s[t], w3, v[tb + t + 3 + ODD]);
#pragma unroll
        for (int t = 0; t < TB; ++t) fma2(ac[tb + t], rc, s[t]);
#pragma unroll
        for (int t = 0; t < TB; ++t) fma2(as[tb + t], rs, s[t]);
    }
}

// Five warpgroups, one CTA per SM, as in the time-domain beamformer: warps
// 0..15 beamform one direction each, warp 16 is the producer and warps 17..19
// only hand their registers back (512 x 112 + 128 x 24 <= 640 x 96).
// The producer walks the CTA's tiles and stages, waits until all 16 consumers
// released a buffer's previous contents (its "empty" mbarrier), re-arms its
// "full" mbarrier and issues the TMA boxes, one lane per box.  The ring runs
// across tile boundaries, so the next tile's first rows land while the
// consumers are still in this tile's epilogue.  A timeout sets the status word
// and the CTA's abort flag; the producer then stops issuing and lets every
// copy it issued land before it exits.
template <int MS, int NS>
__global__ void __launch_bounds__(kBbThreads, 1)
    bb_beamform_kernel(const __grid_constant__ CUtensorMap zmap, const __grid_constant__ BbArgs A) {
    constexpr int NW = kBbWarps;
    constexpr int T = kBbOutPerThread;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    unsigned char* stage = smem_raw;
    uint64_t* full = reinterpret_cast<uint64_t*>(smem_raw + A.stage_area);
    uint64_t* empty = full + NS;
    int* abort_flag = reinterpret_cast<int*>(empty + NS);
    int* issued = abort_flag + 1;  // [NS]: uses of each buffer issued so far (producer only)
    float* env_all = reinterpret_cast<float*>(smem_raw + A.stage_area + kTdBarrierBytes);  // [NW][kBbWarpSamples]
    float* hs = env_all + NW * kBbWarpSamples;                                              // [4][ntap]

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
    for (int j = threadIdx.x; j < 4 * A.ntap; j += kBbThreads) hs[j] = A.hb[j];
    __syncthreads();
    volatile int* vabort = abort_flag;

    const int M = A.M, row = A.row;
    const int nstages = (M + MS - 1) / MS;
    // TMA x of a tile's rows: an even element (16 bytes) at or before its first
    // coarse sample jS = ceil((R i0 - half) / 4) minus the halo
    auto tile_x0 = [&](int t) {
        const int i0t = (t / A.n_dgroups) * A.bins_per_tile;
        return (-((A.half - A.R * i0t) >> 2) - A.H) & ~1;
    };

    if (warp >= NW) {
        // ---------------- producer warpgroup: warp NW issues, the other three leave ----------------
        ptx::setmaxnreg_dec<kTdProducerRegs>();
        if (warp != NW) return;
        const uint32_t stage_bytes = static_cast<uint32_t>(MS * A.nbox * kBbBox * 8);
        if (lane == 0) ptx::prefetch_tmap(&zmap);
        int g = 0;  // stages issued by this CTA so far
        bool stop = false;
        for (int tile = blockIdx.x; tile < A.total_tiles && !stop; tile += gridDim.x) {
            const int x0 = tile_x0(tile);
            for (int st = 0; st < nstages; ++st, ++g) {
                const int b = g % NS;
                const int use = g / NS;
                int ok = 1;
                if (lane == 0) {
                    if (*vabort) {
                        ok = 0;
                    } else if (use > 0 && !ptx::mbar_wait_hinted(&empty[b], static_cast<uint32_t>((use - 1) & 1),
                                                                 kBbPolls, kBbHintNs)) {
                        ok = 0;
                        atomicOr(A.status, RTIS_DEV_TIMEOUT);
                        *vabort = 1;
                    }
                    if (ok) {
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
                // rows st * MS + mi >= M lie outside the tensor and arrive as zeros
                for (int k = lane; k < MS * A.nbox; k += 32) {
                    const int mi = k / A.nbox, bx = k - mi * A.nbox;
                    unsigned char* dst =
                        stage + (static_cast<size_t>(b * MS + mi) * row + static_cast<size_t>(bx) * kBbBox) * 8;
                    ptx::tma_load_2d(dst, &zmap, x0 + bx * kBbBox, st * MS + mi, &full[b]);
                }
            }
        }
        // every copy this CTA issued lands before the CTA can exit
        if (lane == 0) {
            for (int b = 0; b < NS; ++b)
                if (issued[b] > 0)
                    ptx::mbar_wait_hinted(&full[b], static_cast<uint32_t>((issued[b] - 1) & 1), kBbPolls, kBbHintNs);
        }
        return;
    }

    // ---------------- consumers: warp = direction within the tile ----------------
    ptx::setmaxnreg_inc<kTdConsumerRegs>();
    float* env = env_all + warp * kBbWarpSamples;
    int g = 0;
    for (int tile = blockIdx.x; tile < A.total_tiles; tile += gridDim.x) {
        const int dg = tile % A.n_dgroups;
        const int d = dg * NW + warp;
        const int i0 = (tile / A.n_dgroups) * A.bins_per_tile;
        const int jS = -((A.half - A.R * i0) >> 2);  // ceil((R i0 - half) / 4): first coarse sample
        const int x0 = tile_x0(tile);

        // lane m holds the steering entry of mic m for this warp's direction; a
        // direction past the set's end keeps zero weights and shift, so it reads
        // inside the staged rows and sums zeros (no branch around the mic loop)
        const bool dir_ok = d < A.D;
        int my_shift = 0;
        float4 my_w = make_float4(0.f, 0.f, 0.f, 0.f);
        float2 my_r = make_float2(0.f, 0.f);
        if (dir_ok && lane < M) {
            const size_t k = static_cast<size_t>(d) * M + lane;
            my_shift = __ldg(A.shift + k);
            my_w = __ldg(A.wt + k);
            my_r = __ldg(A.rot + k);
        }

        uint64_t ac[T], as[T];
#pragma unroll
        for (int t = 0; t < T; ++t) {
            ac[t] = 0ull;
            as[t] = 0ull;
        }
        const int lane_base = jS - x0 + lane * T - 1;  // smem index of z[jS + lane T - 1]

        bool failed = false;
        for (int st = 0; st < nstages; ++st, ++g) {
            const int b = g % NS;
            const uint32_t par = static_cast<uint32_t>((g / NS) & 1);
            const bool ok = !*vabort && ptx::mbar_wait_hinted(&full[b], par, kBbPolls, kBbHintNs);
            if (!__all_sync(0xffffffffu, ok)) {
                failed = true;
                break;
            }
#pragma unroll
            for (int mi = 0; mi < MS; ++mi) {
                const int m = st * MS + mi;
                if (m >= M) break;
                const int J = __shfl_sync(0xffffffffu, my_shift, m);
                const float f0 = __shfl_sync(0xffffffffu, my_w.x, m);
                const float f1 = __shfl_sync(0xffffffffu, my_w.y, m);
                const float f2 = __shfl_sync(0xffffffffu, my_w.z, m);
                const float f3 = __shfl_sync(0xffffffffu, my_w.w, m);
                const float rc = __shfl_sync(0xffffffffu, my_r.x, m);
                const float rs = __shfl_sync(0xffffffffu, my_r.y, m);
                const int s0 = lane_base + J;  // parity is warp-uniform (T even)
                const ulonglong2* p = reinterpret_cast<const ulonglong2*>(
                    stage + (static_cast<size_t>(b * MS + mi) * row + (s0 & ~1)) * 8);
                if (s0 & 1)
                    bb_mic<true>(ac, as, p, pack2(f0, f0), pack2(f1, f1), pack2(f2, f2), pack2(f3, f3), pack2(rc, rc),
                                 pack2(rs, rs));
                else
                    bb_mic<false>(ac, as, p, pack2(f0, f0), pack2(f1, f1), pack2(f2, f2), pack2(f3, f3),
                                  pack2(rc, rc), pack2(rs, rs));
            }
            __syncwarp();
            if (lane == 0) ptx::mbar_arrive(&empty[b]);  // the producer may refill buffer b
        }
        if (failed) {
            if (lane == 0) {
                if (!*vabort) atomicOr(A.status, RTIS_DEV_TIMEOUT);
                *vabort = 1;
            }
            break;
        }

        // epilogue: |b| over the warp's coarse samples into its own row, then the
        // coarse low-pass
#pragma unroll
        for (int t = 0; t < T; ++t) {
            const int j = jS + lane * T + t;
            const float2 c = unpack2(ac[t]), s = unpack2(as[t]);
            const float br = c.x - s.y, bi = c.y + s.x;
            env[lane * T + t] = (j >= 0 && j < A.Nb) ? magnitude_from_norm(br * br + bi * bi) : 0.f;
        }
        __syncwarp();
        if (dir_ok) {
            float* Erow = A.E + static_cast<size_t>(d) * A.n_out;
            for (int il = lane; il < A.bins_per_tile; il += 32) {
                const int i = i0 + il;
                if (i >= A.n_out) break;
                const int num = A.R * i - A.half;
                const int jlo = -((-num) >> 2);  // ceil(num / 4): first coarse tap
                const float* e = env + (jlo - jS);
                const float* hc = hs + (num & 3) * A.ntap;  // taps for this residue of R i - half
                float acc_e = 0.f;
                if (A.ntap == kBbFastTaps) {  // R = 10 with the 41-tap low-pass: unrolled, same order
#pragma unroll
                    for (int l = 0; l < kBbFastTaps; ++l) acc_e = fmaf(hc[l], e[l], acc_e);
                } else {
                    for (int l = 0; l < A.ntap; ++l) acc_e = fmaf(hc[l], e[l], acc_e);
                }
                if (!isfinite(acc_e)) atomicOr(A.status, RTIS_DEV_NONFINITE);
                Erow[i] = acc_e;
            }
        }
        __syncwarp();  // the row is rewritten by the warp's next tile
    }
}

// stage layouts the autotuner picks from: (mics per stage, stages in the ring)
constexpr int kBbVariantMS[kBbVariants] = {2, 4, 4, 2, 4, 8};
constexpr int kBbVariantNS[kBbVariants] = {8, 4, 5, 10, 8, 4};

uint32_t bb_stage_area(const Plan& p, int variant) {
    const size_t ring = static_cast<size_t>(kBbVariantMS[variant]) * kBbVariantNS[variant] * p.bb_row * 8;
    return static_cast<uint32_t>((ring + 127) & ~static_cast<size_t>(127));
}

size_t bb_smem_variant(const Plan& p, int variant) {
    // ring, barriers + abort flag + issue counters, one envelope row per consumer warp, taps
    return bb_stage_area(p, variant) + kTdBarrierBytes + static_cast<size_t>(kBbWarps) * kBbWarpSamples * 4 +
           static_cast<size_t>(4) * p.bb_ntap * 4;
}

template <int MS, int NS>
cudaError_t bb_launch_t(const CUtensorMap& zmap, const BbArgs& A, int grid, size_t smem, cudaStream_t st) {
    static_assert(16 * NS + 4 * (NS + 1) <= kTdBarrierBytes, "barrier area");
    cudaError_t e = cudaFuncSetAttribute(bb_beamform_kernel<MS, NS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         static_cast<int>(smem));
    if (e != cudaSuccess) return e;
    bb_beamform_kernel<MS, NS><<<grid, kBbThreads, smem, st>>>(zmap, A);
    return cudaGetLastError();
}

cudaError_t bb_launch(const Plan& p, const CUtensorMap& zmap, float* d_out, int variant, int grid, cudaStream_t st) {
    BbArgs A;
    std::memset(&A, 0, sizeof(A));
    A.shift = p.d_bshift;
    A.wt = p.d_bwt;
    A.rot = p.d_brot;
    A.hb = p.d_hb;
    A.E = d_out;
    A.status = p.d_status;
    A.M = p.M;
    A.Nb = p.Nb;
    A.D = p.D;
    A.R = p.R;
    A.half = (p.lpf_len - 1) / 2;
    A.n_out = p.n_out;
    A.bins_per_tile = p.bb_bins_per_tile;
    A.n_dgroups = (p.D + kBbWarps - 1) / kBbWarps;
    A.total_tiles = bb_tiles(p);
    A.H = p.bb_H;
    A.row = p.bb_row;
    A.nbox = p.bb_nbox;
    A.ntap = p.bb_ntap;
    A.stage_area = bb_stage_area(p, variant);
    const size_t smem = bb_smem_variant(p, variant);
    switch (variant) {
        case 0: return bb_launch_t<2, 8>(zmap, A, grid, smem, st);
        case 1: return bb_launch_t<4, 4>(zmap, A, grid, smem, st);
        case 2: return bb_launch_t<4, 5>(zmap, A, grid, smem, st);
        case 3: return bb_launch_t<2, 10>(zmap, A, grid, smem, st);
        case 4: return bb_launch_t<4, 8>(zmap, A, grid, smem, st);
        case 5: return bb_launch_t<8, 4>(zmap, A, grid, smem, st);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace

size_t bb_smem_bytes(const Plan& p) { return bb_smem_variant(p, 0); }  // the smallest layout's
bool bb_variant_fits(const Plan& p, int variant) {
    return variant >= 0 && variant < kBbVariants && bb_smem_variant(p, variant) <= 227 * 1024;
}

int bb_tiles(const Plan& p) {
    return ((p.D + kBbWarps - 1) / kBbWarps) * ((p.n_out + p.bb_bins_per_tile - 1) / p.bb_bins_per_tile);
}

// Times every stage layout with one CTA per tile and with one persistent CTA
// per SM on the plan's own (zeroed) workspace and keeps the fastest.
cudaError_t bb_autotune(Plan& p, float* d_scratch_out) {
    int n_sm = 1, dev = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) n_sm = 1;
    const int tiles = bb_tiles(p);
    const int grids[2] = {tiles, std::min(tiles, n_sm)};
    cudaEvent_t e0, e1;
    cudaError_t e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    if (e != cudaSuccess) return e;
    float best = 1e30f;
    for (int v = 0; v < kBbVariants && e == cudaSuccess; ++v) {
        if (!bb_variant_fits(p, v)) continue;
        for (int gi = 0; gi < 2 && e == cudaSuccess; ++gi) {
            e = bb_launch(p, p.tmap_zb, d_scratch_out, v, grids[gi], 0);  // warm-up
            float total = 0.f;
            for (int r = 0; r < 2 && e == cudaSuccess; ++r) {
                cudaEventRecord(e0, 0);
                e = bb_launch(p, p.tmap_zb, d_scratch_out, v, grids[gi], 0);
                cudaEventRecord(e1, 0);
                if (e == cudaSuccess) e = cudaEventSynchronize(e1);
                float ms = 0.f;
                if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
                total += ms;
            }
            if (e == cudaSuccess) p.bb_variant_ms[2 * v + gi] = total / 2.f;
            if (e == cudaSuccess && total < best) {
                best = total;
                p.bb_variant = v;
                p.bb_grid = grids[gi];
            }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    p.bb_tuned_ms = best / 2.f;
    return e;
}

cudaError_t launch_bb_beamform(const Plan& p, const CUtensorMap& zmap, float* d_out, cudaStream_t st) {
    int grid = p.bb_grid;
    if (grid <= 0) {
        int n_sm = 1, dev = 0;
        cudaGetDevice(&dev);
        if (cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) n_sm = 1;
        grid = std::min(bb_tiles(p), n_sm);
    }
    return bb_launch(p, zmap, d_out, p.bb_variant, grid, st);
}

}  // namespace rtis
