// Reverse pass of the time-domain energyscape with respect to the array's
// calibration: microphone positions p_m, per-channel gains g_m and delays
// Delta_m (the delay-and-sum of the paper's Fig. 3 / Sec. 4.1 and the
// envelope / low-pass / subsampling of Sec. 4.3, differentiated by hand).
//
// With t = n + delta_dm, I = sum_q w_q(mu) a_m[j+q] and I' = dI/dt, and G the
// cotangent of the energyscape:
//   G_env[n] = sum_i G[i] h[n - R i + half]           (transposed low-pass)
//   G_b[n]   = G_env[n] b[n] / |b[n]|                 (0 where b = 0)
//   dL/d delta_dm = g_m sum_n Re(conj(G_b) I'),   dL/d g_m = sum_{d,n} Re(conj(G_b) I)
//   dL/d Delta_m = fs sum_d dL/d delta_dm,        dL/d p_m = -(fs/c) sum_d dL/d delta_dm u_d
//
// Nothing per direction is stored between passes: each tile (16 directions x
// 960 samples, the forward tiling) recomputes its beams from the staged
// channel rows, turns them into G_b in registers, then streams the rows a
// second time and forms, per mic, the four tap correlations
//   C_q = sum_t Re(conj(G_b[t]) a[t + q])
// from which both sums follow with the value and slope weights (so the
// second pass costs what the first does).  Each tile owns the samples of its
// output bins; per-(tile, direction, mic) partials are reduced in a fixed
// order by a second kernel, so the gradient is deterministic.
#include <algorithm>
#include <cstring>

#include "ptx.cuh"
#include "rtis_internal.h"

namespace rtis {
namespace {

// ring waits sleep up to kAdjHintNs per poll; kAdjPolls x kAdjHintNs ~ 1.3 s bounds a wait
constexpr uint32_t kAdjHintNs = 20000;
constexpr uint32_t kAdjPolls = 1u << 16;
constexpr int kAdjMS = 4, kAdjNS = 4;  // mics per stage, ring depth

struct AdjArgs {
    const int* shift;
    const float4* wraw;
    const float4* wder;
    const float* gain;
    const float* h;
    const float* G;       // [D][n_out] cotangent
    float2* part;         // [range tiles][D][M]: (dL/d delta, dL/d g) partials
    unsigned* status;
    int M, N, D, R, lpf_len, n_out, H, row, nbox, bins_per_tile, seg;
};

using ptx::fma2;
using ptx::pack2;
using ptx::unpack2;

// forward: one mic's contribution to a lane's T samples (as the forward kernel)
template <bool ODD>
__device__ __forceinline__ void adj_fwd_mic(uint64_t (&acc)[kTdOutPerThread], const ulonglong2* __restrict__ p,
                                            uint64_t w0, uint64_t w1, uint64_t w2, uint64_t w3) {
    constexpr int T = kTdOutPerThread;
    constexpr int NP = (T + 4) / 2;
    uint64_t v[2 * NP];
#pragma unroll
    for (int k = 0; k < NP; ++k) {
        const ulonglong2 q = p[k];
        v[2 * k] = q.x;
        v[2 * k + 1] = q.y;
    }
#pragma unroll
    for (int t = 0; t < T; ++t) {
        fma2(acc[t], w0, v[t + ODD]);
        fma2(acc[t], w1, v[t + 1 + ODD]);
        fma2(acc[t], w2, v[t + 2 + ODD]);
        fma2(acc[t], w3, v[t + 3 + ODD]);
    }
}

// reverse: C_q = sum_t Re(conj(G_b[t]) a[t + q]), q = 0..3 (taps j-1 .. j+2).
// (re, im) pairs multiply lane-wise with packed FMAs; the two halves are added
// at the end.  Even and odd t accumulate separately for more independent chains.
template <bool ODD>
__device__ __forceinline__ float4 adj_corr_mic(const uint64_t (&gb)[kTdOutPerThread], const ulonglong2* __restrict__ p) {
    constexpr int T = kTdOutPerThread;
    constexpr int NP = (T + 4) / 2;
    uint64_t v[2 * NP];
#pragma unroll
    for (int k = 0; k < NP; ++k) {
        const ulonglong2 q = p[k];
        v[2 * k] = q.x;
        v[2 * k + 1] = q.y;
    }
    uint64_t c[4][2] = {{0ull, 0ull}, {0ull, 0ull}, {0ull, 0ull}, {0ull, 0ull}};
#pragma unroll
    for (int t = 0; t < T; ++t) {
#pragma unroll
        for (int q = 0; q < 4; ++q) fma2(c[q][t & 1], gb[t], v[t + q + ODD]);
    }
    float r[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const float2 e = unpack2(c[q][0]), o = unpack2(c[q][1]);
        r[q] = (e.x + e.y) + (o.x + o.y);
    }
    return make_float4(r[0], r[1], r[2], r[3]);
}

// Pass-B reduction of one pair of mics (m0, m0 + 1) from the raw tap correlations: the
// eight sums C_q of the two mics are reduce-scattered over the warp (after the xor-16, 8
// and 4 exchanges lane bits (4, 3, 2) select (mic, q); then a plain sum), lane m0 + h
// gathers its mic's four totals and applies its own value and slope weights.
__device__ __forceinline__ void adj_pair_reduce_c(const float4& c0, const float4& c1, int lane, int m0,
                                                  const float4& w, const float4& wd, float& sum_g, float& sum_d) {
    const bool b16 = lane & 16, b8 = lane & 8, b4 = lane & 4;
    float k[4];
    {
        const float4 keep = b16 ? c1 : c0, send = b16 ? c0 : c1;
        k[0] = keep.x + __shfl_xor_sync(0xffffffffu, send.x, 16);
        k[1] = keep.y + __shfl_xor_sync(0xffffffffu, send.y, 16);
        k[2] = keep.z + __shfl_xor_sync(0xffffffffu, send.z, 16);
        k[3] = keep.w + __shfl_xor_sync(0xffffffffu, send.w, 16);
    }
    const float k0 = (b8 ? k[2] : k[0]) + __shfl_xor_sync(0xffffffffu, b8 ? k[0] : k[2], 8);
    const float k1 = (b8 ? k[3] : k[1]) + __shfl_xor_sync(0xffffffffu, b8 ? k[1] : k[3], 8);
    float t = (b4 ? k1 : k0) + __shfl_xor_sync(0xffffffffu, b4 ? k0 : k1, 4);
    t += __shfl_xor_sync(0xffffffffu, t, 2);
    t += __shfl_xor_sync(0xffffffffu, t, 1);
    // lane 16 h + 4 q holds C_q of mic m0 + h
    const int base = (lane == m0 + 1) ? 16 : 0;
    const float C0 = __shfl_sync(0xffffffffu, t, base), C1 = __shfl_sync(0xffffffffu, t, base + 4);
    const float C2 = __shfl_sync(0xffffffffu, t, base + 8), C3 = __shfl_sync(0xffffffffu, t, base + 12);
    if (lane == m0 || lane == m0 + 1) {
        sum_g = fmaf(w.x, C0, fmaf(w.y, C1, fmaf(w.z, C2, w.w * C3)));
        sum_d = fmaf(wd.x, C0, fmaf(wd.y, C1, fmaf(wd.z, C2, wd.w * C3)));
    }
}

// The forward beamformer's shape: one persistent CTA per SM, 16 direction warps and a
// producer warpgroup (warp 16 issues the TMA boxes, warps 17..19 hand their registers
// back through setmaxnreg), full/empty mbarrier ring running across tiles.  A tile is
// 16 directions x one range tile; its stages are the mic groups twice over (pass A
// recomputes the beams, pass B correlates G_b with the same rows).  Every direction
// warp runs every loop (a direction past the set's end has zero weights and cotangent)
// and writes its partials only for a real direction.
// FASTG: R = 10 and the 41-tap low-pass (30 samples per lane = 3 bins), so the transposed
// low-pass of a lane's samples reads 5 cotangent bins per run of 10 samples with taps fixed
// at compile time.
constexpr int kAdjFastR = 10, kAdjFastTaps = 41;
static_assert(kTdOutPerThread == 3 * kAdjFastR, "the fast G_b transform assumes 30 samples per lane");

template <int MS, int NS, bool FASTG>
__global__ void __launch_bounds__(kTdThreads, 1)
    td_adjoint_kernel(const __grid_constant__ CUtensorMap tmap, const AdjArgs args) {
    constexpr int NW = kTdWarps;
    constexpr int T = kTdOutPerThread;
    static_assert(MS % 2 == 0, "pass B reduces the mics of a stage in pairs");
    extern __shared__ __align__(128) unsigned char smem_raw[];
    const int row = args.row;
    float2* stage = reinterpret_cast<float2*>(smem_raw);
    const size_t ring_bytes = static_cast<size_t>(NS) * MS * row * 8;
    uint64_t* full = reinterpret_cast<uint64_t*>(smem_raw + ring_bytes);
    uint64_t* empty = full + NS;
    int* abort_flag = reinterpret_cast<int*>(empty + NS);
    int* issued = abort_flag + 1;  // [NS], producer only
    float* hs = reinterpret_cast<float*>(smem_raw + ring_bytes + kTdBarrierBytes);
    float* gseg = hs + ((args.lpf_len + 3) & ~3);  // [16 warps][seg]

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
    for (int j = threadIdx.x; j < args.lpf_len; j += kTdThreads) hs[j] = args.h[j];
    __syncthreads();
    volatile int* vabort = abort_flag;
    const int half = (args.lpf_len - 1) >> 1;
    const int M = args.M;
    const int ngroups = (M + MS - 1) / MS;
    const int nstages = 2 * ngroups;  // pass A then pass B over the same rows
    const int n_dgroups = (args.D + NW - 1) / NW;
    const int total = n_dgroups * ((args.n_out + args.bins_per_tile - 1) / args.bins_per_tile);

    if (warp >= NW) {
        // ---------------- producer ----------------
        ptx::setmaxnreg_dec<kTdProducerRegs>();
        if (warp != NW) return;
        const uint32_t stage_bytes = static_cast<uint32_t>(MS * args.nbox * kTdBox * 8);
        if (lane == 0) ptx::prefetch_tmap(&tmap);
        int g = 0;
        bool stop = false;
        for (int tile = blockIdx.x; tile < total && !stop; tile += gridDim.x) {
            const int i0 = (tile / n_dgroups) * args.bins_per_tile;
            const int x0 = (args.R * i0 - half - args.H) & ~1;
            for (int st = 0; st < nstages; ++st, ++g) {
                const int b = g % NS;
                const int use = g / NS;
                int ok = 1;
                if (lane == 0) {
                    if (*vabort) {
                        ok = 0;
                    } else if (use > 0 && !ptx::mbar_wait_hinted(&empty[b], static_cast<uint32_t>((use - 1) & 1),
                                                                 kAdjPolls, kAdjHintNs)) {
                        ok = 0;
                        atomicOr(args.status, RTIS_DEV_TIMEOUT);
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
                const int grp = st % ngroups;
                for (int j = lane; j < MS * args.nbox; j += 32) {
                    const int mi = j / args.nbox;
                    const int bx = j - mi * args.nbox;
                    ptx::tma_load_2d(stage + static_cast<size_t>(b * MS + mi) * row + bx * kTdBox, &tmap,
                                     x0 + bx * kTdBox, grp * MS + mi, &full[b]);
                }
            }
        }
        if (lane == 0) {
            for (int b = 0; b < NS; ++b)
                if (issued[b] > 0)
                    ptx::mbar_wait_hinted(&full[b], static_cast<uint32_t>((issued[b] - 1) & 1), kAdjPolls, kAdjHintNs);
        }
        return;
    }

    // ---------------- direction warps ----------------
    ptx::setmaxnreg_inc<kTdConsumerRegs>();
    const int reach = (half + args.R - 1) / args.R + 1;
    float* gs = gseg + warp * args.seg;
    int g = 0;
    for (int tile = blockIdx.x; tile < total; tile += gridDim.x) {
        const int dg = tile % n_dgroups;
        const int nt = tile / n_dgroups;
        const int d = dg * NW + warp;
        const int i0 = nt * args.bins_per_tile;
        const int n_start = args.R * i0 - half;
        const int x0 = (n_start - args.H) & ~1;
        // samples this tile owns: those of its output bins (the last tile: up to N)
        const int own_lo = args.R * i0;
        const bool last_tile = (i0 + args.bins_per_tile >= args.n_out);
        const int own_hi = last_tile ? args.N : args.R * (i0 + args.bins_per_tile);

        const bool dir_ok = d < args.D;
        int my_shift = 0;
        float4 my_w = make_float4(0.f, 0.f, 0.f, 0.f), my_wd = my_w;
        float my_g = 0.f;
        if (dir_ok && lane < M) {
            const size_t e = static_cast<size_t>(d) * M + lane;
            my_shift = __ldg(args.shift + e);
            my_w = __ldg(args.wraw + e);
            my_wd = __ldg(args.wder + e);
            my_g = __ldg(args.gain + lane);
        }
        // cotangent segment of this warp's direction, bins [iseg0, iseg0 + seg)
        const int iseg0 = i0 - reach;
        __syncwarp();  // the previous tile's reads of the segment are done
        for (int k = lane; k < args.seg; k += 32) {
            const int i = iseg0 + k;
            gs[k] = (dir_ok && i >= 0 && i < args.n_out) ? __ldg(args.G + static_cast<size_t>(d) * args.n_out + i)
                                                         : 0.f;
        }

        uint64_t acc[T];
#pragma unroll
        for (int t = 0; t < T; ++t) acc[t] = 0ull;
        const int lane_base = n_start - x0 + lane * T - 1;
        float sum_d = 0.f, sum_g = 0.f;  // lane m keeps mic m's totals
        bool failed = false;

        // pass A: the tile's beams
        for (int st = 0; st < ngroups; ++st, ++g) {
            const int b = g % NS;
            const uint32_t par = static_cast<uint32_t>((g / NS) & 1);
            const bool ok = !*vabort && ptx::mbar_wait_hinted(&full[b], par, kAdjPolls, kAdjHintNs);
            if (!__all_sync(0xffffffffu, ok)) {
                failed = true;
                break;
            }
            // the stage's mics in a rolled loop (as in pass B): each mic's body is already
            // 120 packed FMAs, and unrolled the two passes overflow the instruction cache
#pragma unroll 1
            for (int mi = 0; mi < MS; ++mi) {
                const int m = st * MS + mi;
                if (m >= M) break;
                const int J = __shfl_sync(0xffffffffu, my_shift, m);
                const int s0 = lane_base + J;
                const ulonglong2* p =
                    reinterpret_cast<const ulonglong2*>(stage + static_cast<size_t>(b * MS + mi) * row + (s0 & ~1));
                const float gm = __shfl_sync(0xffffffffu, my_g, m);
                const float f0 = gm * __shfl_sync(0xffffffffu, my_w.x, m);
                const float f1 = gm * __shfl_sync(0xffffffffu, my_w.y, m);
                const float f2 = gm * __shfl_sync(0xffffffffu, my_w.z, m);
                const float f3 = gm * __shfl_sync(0xffffffffu, my_w.w, m);
                if (s0 & 1)
                    adj_fwd_mic<true>(acc, p, pack2(f0, f0), pack2(f1, f1), pack2(f2, f2), pack2(f3, f3));
                else
                    adj_fwd_mic<false>(acc, p, pack2(f0, f0), pack2(f1, f1), pack2(f2, f2), pack2(f3, f3));
            }
            __syncwarp();
            if (lane == 0) ptx::mbar_arrive(&empty[b]);  // the producer may refill buffer b
        }
        if (!failed) {
            // the beams are complete: turn them into G_b = G_env b / |b| on owned samples.
            // G_env[n] sums the bins i in [ceil((n - half)/R), floor((n + half)/R)] (tap
            // j = n - R i + half); both ends advance incrementally with n.
            __syncwarp();
            const int R = args.R;
            const int n_first = n_start + lane * T;
            if constexpr (FASTG) {
                // n = n_first + t = R (i0 + 3 lane) - half + t: in the run r of samples t = 10 r + u,
                // bin i0 + 3 lane + r + e - 4 reaches sample t with tap u + 40 - 10 e (e = 0 only
                // for u = 0), so five bins are live at a time; the bins are summed in increasing
                // order, as the general loop below does
                const float* gl = gs + 3 * lane - 4 + reach;  // lane 0's gl[0] is never used
                float g0 = lane > 0 ? gl[0] : 0.f, g1 = gl[1], g2 = gl[2], g3 = gl[3], g4 = gl[4];
#pragma unroll
                for (int r = 0; r < 3; ++r) {
                    if (r > 0) {
                        g0 = g1;
                        g1 = g2;
                        g2 = g3;
                        g3 = g4;
                        g4 = gl[r + 4];
                    }
#pragma unroll
                    for (int u = 0; u < 10; ++u) {
                        // keep each sample's tap loads next to their use (hoisted, the taps would
                        // crowd out the beams' registers)
                        asm volatile("" ::: "memory");
                        const int t = 10 * r + u;
                        const int n = n_first + t;
                        float ge = 0.f;
                        if (u == 0) ge = fmaf(g0, hs[40], ge);
                        ge = fmaf(g1, hs[u + 30], ge);
                        ge = fmaf(g2, hs[u + 20], ge);
                        ge = fmaf(g3, hs[u + 10], ge);
                        ge = fmaf(g4, hs[u], ge);
                        if (!(n >= own_lo && n < own_hi && n < args.N)) ge = 0.f;
                        const float2 v = unpack2(acc[t]);
                        const float m2 = v.x * v.x + v.y * v.y;
                        const float sc = m2 > 0.f ? ge * rsqrtf(m2) : 0.f;
                        acc[t] = pack2(sc * v.x, sc * v.y);
                    }
                }
            } else {
                const int xo = n_first - half + R * reach * 4;  // > 0
                int i_lo = (xo + R - 1) / R - reach * 4;           // ceil((n - half)/R)
                int r_lo = (i_lo + reach * 4) * R - xo;            // R i_lo - (n - half), in [0, R)
                const int yo = n_first + half + R * reach * 4;
                int i_hi = yo / R - reach * 4;                     // floor((n + half)/R)
                int r_hi = yo - (i_hi + reach * 4) * R;            // (n + half) - R i_hi, in [0, R)
#pragma unroll
                for (int t = 0; t < T; ++t) {
                    const int n = n_first + t;
                    float ge = 0.f;
                    if (n >= own_lo && n < own_hi && n >= 0 && n < args.N) {
                        int j = 2 * half - r_lo;  // tap of bin i_lo
                        for (int i = i_lo; i <= i_hi; ++i, j -= R) ge = fmaf(gs[i - iseg0], hs[j], ge);
                    }
                    const float2 v = unpack2(acc[t]);
                    const float m2 = v.x * v.x + v.y * v.y;
                    const float sc = m2 > 0.f ? ge * rsqrtf(m2) : 0.f;
                    acc[t] = pack2(sc * v.x, sc * v.y);
                    // n -> n + 1
                    if (--r_lo < 0) {
                        r_lo += R;
                        ++i_lo;
                    }
                    if (++r_hi == R) {
                        r_hi = 0;
                        ++i_hi;
                    }
                }
            }
        }
        // pass B: correlate G_b with the same rows, streamed again
        for (int st = 0; st < ngroups && !failed; ++st, ++g) {
            const int b = g % NS;
            const uint32_t par = static_cast<uint32_t>((g / NS) & 1);
            const bool ok = !*vabort && ptx::mbar_wait_hinted(&full[b], par, kAdjPolls, kAdjHintNs);
            if (!__all_sync(0xffffffffu, ok)) {
                failed = true;
                break;
            }
#pragma unroll 1
            for (int pr = 0; pr < MS / 2; ++pr) {
                // both mics' tap correlations, then one joint reduction; each owner lane weights
                // its own mic's totals
                float4 cc[2];
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int mi = 2 * pr + h;
                    cc[h] = make_float4(0.f, 0.f, 0.f, 0.f);
                    const int m = st * MS + mi;
                    if (m < M) {
                        const int J = __shfl_sync(0xffffffffu, my_shift, m);
                        const int s0 = lane_base + J;
                        const ulonglong2* p = reinterpret_cast<const ulonglong2*>(
                            stage + static_cast<size_t>(b * MS + mi) * row + (s0 & ~1));
                        cc[h] = (s0 & 1) ? adj_corr_mic<true>(acc, p) : adj_corr_mic<false>(acc, p);
                    }
                }
                adj_pair_reduce_c(cc[0], cc[1], lane, st * MS + 2 * pr, my_w, my_wd, sum_g, sum_d);
            }
            __syncwarp();
            if (lane == 0) ptx::mbar_arrive(&empty[b]);  // the producer may refill buffer b
        }
        if (failed) {
            if (lane == 0) {
                if (!*vabort) atomicOr(args.status, RTIS_DEV_TIMEOUT);
                *vabort = 1;
            }
            break;
        }
        if (dir_ok && lane < M) args.part[(static_cast<size_t>(nt) * args.D + d) * M + lane] = make_float2(my_g * sum_d, sum_g);
    }
}

// Two-stage fixed-order reduction of the per-(tile, direction, mic) partials.
// Stage 1: CTA (m, blk) sums directions [blk D/NB, (blk + 1) D/NB) over all
// range tiles into five values: sum dL/d delta, sum dL/d g, sum dL/d delta u.
constexpr int kAdjRedBlocks = 16, kAdjRedThreads = 256;

__global__ void __launch_bounds__(kAdjRedThreads) adj_reduce1_kernel(const float2* __restrict__ part,
                                                                     const float* __restrict__ dirs, int M, int D,
                                                                     int n_tiles, float* __restrict__ red5) {
    const int m = blockIdx.x, blk = blockIdx.y;
    const int d_lo = static_cast<int>((static_cast<long long>(blk) * D) / kAdjRedBlocks);
    const int d_hi = static_cast<int>((static_cast<long long>(blk + 1) * D) / kAdjRedBlocks);
    float v[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
    for (int d = d_lo + threadIdx.x; d < d_hi; d += kAdjRedThreads) {
        float pd = 0.f, pg = 0.f;
        for (int t = 0; t < n_tiles; ++t) {
            const float2 x = part[(static_cast<size_t>(t) * D + d) * M + m];
            pd += x.x;
            pg += x.y;
        }
        v[0] += pd;
        v[1] += pg;
        v[2] = fmaf(pd, dirs[3 * d], v[2]);
        v[3] = fmaf(pd, dirs[3 * d + 1], v[3]);
        v[4] = fmaf(pd, dirs[3 * d + 2], v[4]);
    }
    __shared__ float red[5][kAdjRedThreads];
#pragma unroll
    for (int k = 0; k < 5; ++k) red[k][threadIdx.x] = v[k];
    __syncthreads();
    for (int w = kAdjRedThreads / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w)
#pragma unroll
            for (int k = 0; k < 5; ++k) red[k][threadIdx.x] += red[k][threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x < 5) red5[(m * kAdjRedBlocks + blk) * 5 + threadIdx.x] = red[threadIdx.x][0];
}

// Stage 2: one thread per mic sums the blocks in order and applies the chain rule.
__global__ void adj_reduce2_kernel(const float* __restrict__ red5, int M, double fs, double fs_over_c,
                                   float* __restrict__ gxyz, float* __restrict__ ggain, float* __restrict__ gdelay) {
    const int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= M) return;
    double v[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
    for (int blk = 0; blk < kAdjRedBlocks; ++blk)
#pragma unroll
        for (int k = 0; k < 5; ++k) v[k] += red5[(m * kAdjRedBlocks + blk) * 5 + k];
    if (gdelay) gdelay[m] = static_cast<float>(fs * v[0]);
    if (ggain) ggain[m] = static_cast<float>(v[1]);
    if (gxyz) {
        gxyz[3 * m] = static_cast<float>(-fs_over_c * v[2]);
        gxyz[3 * m + 1] = static_cast<float>(-fs_over_c * v[3]);
        gxyz[3 * m + 2] = static_cast<float>(-fs_over_c * v[4]);
    }
}

// L2 calibration loss: per-block partial sums of (E - E_ref)^2 (fixed tree), G = 2 (E - E_ref)
constexpr int kLossThreads = 256, kLossBlocks = 4 * 152;

__global__ void __launch_bounds__(kLossThreads) l2_loss_kernel(const float* __restrict__ E,
                                                               const float* __restrict__ Eref,
                                                               float* __restrict__ G, float* __restrict__ part,
                                                               size_t n) {
    float s = 0.f;
    for (size_t i = static_cast<size_t>(blockIdx.x) * kLossThreads + threadIdx.x; i < n;
         i += static_cast<size_t>(gridDim.x) * kLossThreads) {
        const float r = E[i] - Eref[i];
        if (G) G[i] = 2.f * r;
        s = fmaf(r, r, s);
    }
    __shared__ float red[kLossThreads];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int w = kLossThreads / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = red[0];
}

__global__ void l2_final_kernel(const float* __restrict__ part, int nb, float* __restrict__ loss) {
    __shared__ double red[kLossThreads];
    double s = 0.0;
    for (int i = threadIdx.x; i < nb; i += kLossThreads) s += part[i];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int w = kLossThreads / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) *loss = static_cast<float>(red[0]);
}

int adj_seg(const Plan& p) {
    const int half = (p.lpf_len - 1) / 2;
    const int reach = (half + p.R - 1) / p.R + 1;
    return p.td_bins_per_tile + 3 * reach + 2;
}

}  // namespace

size_t adj_smem_bytes(const Plan& p) {
    return static_cast<size_t>(kAdjNS) * kAdjMS * p.td_row * 8 + kTdBarrierBytes +
           static_cast<size_t>((p.lpf_len + 3) & ~3) * 4 + static_cast<size_t>(kTdWarps) * adj_seg(p) * 4;
}

cudaError_t launch_td_adjoint(const Plan& p, const float* d_grad_out, float* d_gxyz, float* d_ggain, float* d_gdelay,
                              cudaStream_t st) {
    AdjArgs a;
    a.shift = p.d_shift;
    a.wraw = p.d_wraw;
    a.wder = p.d_wder;
    a.gain = p.d_gain;
    a.h = p.d_h;
    a.G = d_grad_out;
    a.part = p.d_adj;
    a.status = p.d_status;
    a.M = p.M;
    a.N = p.N;
    a.D = p.D;
    a.R = p.R;
    a.lpf_len = p.lpf_len;
    a.n_out = p.n_out;
    a.H = p.H;
    a.row = p.td_row;
    a.nbox = p.td_nbox;
    a.bins_per_tile = p.td_bins_per_tile;
    a.seg = adj_seg(p);
    const size_t smem = adj_smem_bytes(p);
    const bool fastg = p.R == kAdjFastR && p.lpf_len == kAdjFastTaps;
    auto kern = fastg ? td_adjoint_kernel<kAdjMS, kAdjNS, true> : td_adjoint_kernel<kAdjMS, kAdjNS, false>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
    if (e != cudaSuccess) return e;
    int n_sm = 1, dev = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) n_sm = 1;
    const int n_tiles = (p.n_out + p.td_bins_per_tile - 1) / p.td_bins_per_tile;
    const int total = ((p.D + kTdWarps - 1) / kTdWarps) * n_tiles;
    kern<<<std::min(total, n_sm), kTdThreads, smem, st>>>(p.tmap_a, a);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    adj_reduce1_kernel<<<dim3(p.M, kAdjRedBlocks), kAdjRedThreads, 0, st>>>(p.d_adj, p.d_dirs, p.M, p.D, n_tiles,
                                                                         p.d_adj_red);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    adj_reduce2_kernel<<<1, kMaxMics, 0, st>>>(p.d_adj_red, p.M, p.fs, p.fs / p.c, d_gxyz, d_ggain, d_gdelay);
    return cudaGetLastError();
}

cudaError_t launch_l2_loss(const Plan& p, const float* d_E, const float* d_Eref, float* d_G, float* d_loss,
                           cudaStream_t st) {
    const size_t n = static_cast<size_t>(p.D) * p.n_out;
    float* part = reinterpret_cast<float*>(p.d_adj);  // the adjoint's partials, free between calls
    const int nb = static_cast<int>(std::min<size_t>(kLossBlocks, (n + kLossThreads - 1) / kLossThreads));
    if (nb == 0) return cudaMemsetAsync(d_loss, 0, sizeof(float), st);
    l2_loss_kernel<<<nb, kLossThreads, 0, st>>>(d_E, d_Eref, d_G, part, n);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    l2_final_kernel<<<1, kLossThreads, 0, st>>>(part, nb, d_loss);
    return cudaGetLastError();
}

}  // namespace rtis
