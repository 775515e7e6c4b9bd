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
// The layout follows the time-domain beamformer: one CTA is 8 warps = 8
// directions x one range tile of 32 lanes x 14 coarse samples; channel rows
// arrive by TMA through an mbarrier ring of NS stages x MS mics; the envelope,
// low-pass and subsampling run in the epilogue out of shared memory.  Per mic
// and coarse sample a lane forms s = sum_q w_q z (one packed multiply and three
// packed FMAs on (re, im)) and accumulates cr * s and ci * s (two packed FMAs),
// r = cr + i ci; the beam is (acc_c.re - acc_s.im, acc_c.im + acc_s.re).
// That is 6 packed FMAs per (mic, coarse sample) against 4 per (mic, sample) on
// the full-rate grid: 2.7x fewer.  Waits are bounded as in the other kernels.
#include <algorithm>
#include <cstring>

#include "ptx.cuh"
#include "rtis_internal.h"

namespace rtis {
namespace {

using ptx::fma2;
using ptx::mul2;
using ptx::pack2;
using ptx::unpack2;

constexpr uint32_t kBbWaitPolls = 1u << 22;  // bounded mbarrier wait (~ seconds)

struct BbArgs {
    const int* shift;    // [D][M]
    const float4* wt;    // [D][M]
    const float2* rot;   // [D][M]
    const float* hb;     // [4][ntap]
    float* E;            // [D][n_out]
    unsigned* status;
    int M, Nb, D, R, half, n_out, bins_per_tile, n_dgroups, total_tiles, H, row, nbox, ntap;
    uint32_t stage_area;  // bytes of the stage ring; the envelope rows follow it
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

template <int MS, int NS>
__global__ void __launch_bounds__(32 * kTdDirsPerCta, 2)
    bb_beamform_kernel(const __grid_constant__ CUtensorMap zmap, const __grid_constant__ BbArgs A) {
    constexpr int NT = 32 * kTdDirsPerCta;
    constexpr int T = kBbOutPerThread;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    unsigned char* stage = smem_raw;
    float* env_all = reinterpret_cast<float*>(smem_raw + A.stage_area);  // [8][kBbWarpSamples]
    uint64_t* bar = reinterpret_cast<uint64_t*>(env_all + kTdDirsPerCta * kBbWarpSamples);
    int* done = reinterpret_cast<int*>(bar + NS);
    int* issued = done + NS;
    int* next_issued = issued + NS;  // stages of this CTA's next tile already in flight
    float* hs = reinterpret_cast<float*>(next_issued + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int b = 0; b < NS; ++b) {
            ptx::mbar_init(&bar[b], 1);
            done[b] = 0;
            issued[b] = 0;
        }
        *next_issued = 0;
        ptx::fence_mbar_init();
        ptx::fence_proxy_async();
    }
    for (int j = threadIdx.x; j < 4 * A.ntap; j += NT) hs[j] = A.hb[j];

    const int M = A.M, row = A.row;
    const int nstages = (M + MS - 1) / MS;
    const uint32_t stage_bytes = static_cast<uint32_t>(MS * A.nbox * kBbBox * 8);
    // TMA x of a tile's rows: an even element (16 bytes) at or before its first
    // coarse sample jS = ceil((R i0 - half) / 4) minus the halo
    auto tile_x0 = [&](int t) {
        const int i0t = (t / A.n_dgroups) * A.bins_per_tile;
        return (-((A.half - A.R * i0t) >> 2) - A.H) & ~1;
    };
    // stage st of a tile whose rows start at x, into ring slot g (global stage count):
    // a whole warp issues it, lane 0 arming the barrier and every lane one box
    auto issue_warp = [&](int g, int x, int st) {
        const int b = g % NS;
        if (lane == 0) {
            issued[b] += 1;
            ptx::mbar_arrive_expect_tx(&bar[b], stage_bytes);
        }
        __syncwarp();
        for (int k = lane; k < MS * A.nbox; k += 32) {
            const int mi = k / A.nbox, bx = k - mi * A.nbox;
            unsigned char* dst = stage + (static_cast<size_t>(b * MS + mi) * row + static_cast<size_t>(bx) * kBbBox) * 8;
            ptx::tma_load_2d(dst, &zmap, x + bx * kBbBox, st * MS + mi, &bar[b]);
        }
    };
    int g0 = 0;
    bool timed_out = false;
    for (int tile = blockIdx.x; tile < A.total_tiles; tile += gridDim.x) {
        const int dg = tile % A.n_dgroups;
        const int d = dg * kTdDirsPerCta + warp;
        const int i0 = (tile / A.n_dgroups) * A.bins_per_tile;
        const int jS = -((A.half - A.R * i0) >> 2);  // ceil((R i0 - half) / 4): first coarse sample
        const int x0 = tile_x0(tile);
        const int next_tile = tile + gridDim.x;

        __syncthreads();  // the previous tile's refills are all issued
        if (warp == 0) {
            if (lane == 0 && tile == static_cast<int>(blockIdx.x)) ptx::prefetch_tmap(&zmap);
            // the first stages not already prefetched while the previous tile finished
            const int pre = *next_issued;
            for (int st = pre; st < NS && st < nstages; ++st) issue_warp(g0 + st, x0, st);
            __syncwarp();
            if (lane == 0) *next_issued = 0;
        }

        // lane m holds the steering entry of mic m for this warp's direction
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

        for (int st = 0; st < nstages; ++st) {
            const int b = (g0 + st) % NS;
            if (!timed_out) {
                const uint32_t par = static_cast<uint32_t>(((g0 + st) / NS) & 1);
                if (!ptx::mbar_wait_bounded(&bar[b], par, kBbWaitPolls)) {
                    timed_out = true;
                    atomicOr(A.status, RTIS_DEV_TIMEOUT);
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
                    const float rc = __shfl_sync(0xffffffffu, my_r.x, m);
                    const float rs = __shfl_sync(0xffffffffu, my_r.y, m);
                    const int s0 = lane_base + J;  // parity is warp-uniform (T even)
                    const ulonglong2* p = reinterpret_cast<const ulonglong2*>(
                        stage + (static_cast<size_t>(b * MS + mi) * row + (s0 & ~1)) * 8);
                    if (s0 & 1)
                        bb_mic<true>(ac, as, p, pack2(f0, f0), pack2(f1, f1), pack2(f2, f2), pack2(f3, f3),
                                     pack2(rc, rc), pack2(rs, rs));
                    else
                        bb_mic<false>(ac, as, p, pack2(f0, f0), pack2(f1, f1), pack2(f2, f2), pack2(f3, f3),
                                      pack2(rc, rc), pack2(rs, rs));
                }
            }
            // release buffer b; the CTA's last warp to get here refills it with the
            // stage NS later: of this tile, or else of the CTA's next tile
            __syncwarp();
            int last = 0;
            if (lane == 0) {
                __threadfence_block();
                const int prev = atomicAdd(&done[b], 1);
                if (prev == kTdDirsPerCta - 1) {
                    done[b] = 0;
                    __threadfence_block();
                    last = 1;
                }
            }
            last = __shfl_sync(0xffffffffu, last, 0);
            if (last && !warp_timed_out) {  // no refills once a wait has given up
                const int nst = st + NS;
                if (nst < nstages) {
                    ptx::fence_proxy_async();
                    issue_warp(g0 + nst, x0, nst);
                } else if (next_tile < A.total_tiles && nst - nstages < nstages) {
                    ptx::fence_proxy_async();
                    issue_warp(g0 + nst, tile_x0(next_tile), nst - nstages);
                    if (lane == 0) atomicAdd(next_issued, 1);
                }
            }
        }
        g0 += nstages;

        if (__syncthreads_or(timed_out)) break;  // uniform: leave the tile loop, drain below

        // epilogue (its own shared memory: the ring may already hold the next tile's rows):
        // |b| over the warp's coarse samples, then the coarse low-pass
        float* env = env_all + warp * kBbWarpSamples;
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
                for (int l = 0; l < A.ntap; ++l) acc_e = fmaf(hc[l], e[l], acc_e);
                if (!isfinite(acc_e)) atomicOr(A.status, RTIS_DEV_NONFINITE);
                Erow[i] = acc_e;
            }
        }
    }

    if (__syncthreads_or(timed_out)) {
        // give copies still in flight a bounded chance to land, then leave
        if (threadIdx.x == 0) {
            for (int b = 0; b < NS; ++b)
                if (issued[b] > 0)
                    ptx::mbar_wait_bounded(&bar[b], static_cast<uint32_t>((issued[b] - 1) & 1), kBbWaitPolls);
        }
        __syncthreads();
    }
}

// stage layouts the autotuner picks from: (mics per stage, stages in the ring)
constexpr int kBbVariantMS[kBbVariants] = {2, 2, 4, 1, 4, 2};
constexpr int kBbVariantNS[kBbVariants] = {4, 8, 4, 8, 5, 10};

uint32_t bb_stage_area(const Plan& p, int variant) {
    const size_t ring = static_cast<size_t>(kBbVariantMS[variant]) * kBbVariantNS[variant] * p.bb_row * 8;
    return static_cast<uint32_t>((ring + 127) & ~static_cast<size_t>(127));
}

size_t bb_smem_variant(const Plan& p, int variant) {
    // ring, envelope rows, barriers + counters (<= 10 stages), next-tile count, taps
    return bb_stage_area(p, variant) + static_cast<size_t>(kTdDirsPerCta) * kBbWarpSamples * 4 + 10 * (8 + 4 + 4) +
           16 + static_cast<size_t>(4) * p.bb_ntap * 4;
}

template <int MS, int NS>
cudaError_t bb_launch_t(const CUtensorMap& zmap, const BbArgs& A, int grid, size_t smem, cudaStream_t st) {
    cudaError_t e = cudaFuncSetAttribute(bb_beamform_kernel<MS, NS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         static_cast<int>(smem));
    if (e != cudaSuccess) return e;
    bb_beamform_kernel<MS, NS><<<grid, 32 * kTdDirsPerCta, smem, st>>>(zmap, A);
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
    A.n_dgroups = (p.D + kTdDirsPerCta - 1) / kTdDirsPerCta;
    A.total_tiles = bb_tiles(p);
    A.H = p.bb_H;
    A.row = p.bb_row;
    A.nbox = p.bb_nbox;
    A.ntap = p.bb_ntap;
    A.stage_area = bb_stage_area(p, variant);
    const size_t smem = bb_smem_variant(p, variant);
    switch (variant) {
        case 0: return bb_launch_t<2, 4>(zmap, A, grid, smem, st);
        case 1: return bb_launch_t<2, 8>(zmap, A, grid, smem, st);
        case 2: return bb_launch_t<4, 4>(zmap, A, grid, smem, st);
        case 3: return bb_launch_t<1, 8>(zmap, A, grid, smem, st);
        case 4: return bb_launch_t<4, 5>(zmap, A, grid, smem, st);
        case 5: return bb_launch_t<2, 10>(zmap, A, grid, smem, st);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace

size_t bb_smem_bytes(const Plan& p) { return bb_smem_variant(p, 0); }  // the smallest layout's
bool bb_variant_fits(const Plan& p, int variant) {
    return variant >= 0 && variant < kBbVariants && bb_smem_variant(p, variant) <= 227 * 1024;
}

int bb_tiles(const Plan& p) {
    return ((p.D + kTdDirsPerCta - 1) / kTdDirsPerCta) * ((p.n_out + p.bb_bins_per_tile - 1) / p.bb_bins_per_tile);
}

// Times every stage layout with one CTA per tile and with two persistent CTAs
// per SM on the plan's own (zeroed) workspace and keeps the fastest.
cudaError_t bb_autotune(Plan& p, float* d_scratch_out) {
    int n_sm = 1, dev = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) n_sm = 1;
    const int tiles = bb_tiles(p);
    const int grids[2] = {tiles, std::min(tiles, 2 * n_sm)};
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
        grid = std::min(bb_tiles(p), 2 * n_sm);
    }
    return bb_launch(p, zmap, d_out, p.bb_variant, grid, st);
}

}  // namespace rtis
