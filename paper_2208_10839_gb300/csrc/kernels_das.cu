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
// Tiling (one CTA = 8 directions x 992 consecutive samples, one warp per
// direction, each lane 31 consecutive samples):
//   * the channel rows a_m[x0 .. x0 + 992 + 2H) of 4 mics at a time are
//     staged into shared memory by TMA (2-stage mbarrier ring; samples outside
//     [0, N) arrive as zeros from the TMA out-of-bounds fill);
//   * each lane walks its 31 samples with a 4-tap sliding window in
//     registers: one 8-byte shared load and 8 FMAs per sample and mic, the
//     per-mic steering values broadcast across the warp by shuffles;
//   * the epilogue writes |b| for the tile to shared memory and each warp
//     filters and subsamples its own direction, storing E coalesced.
// The tile's 992 samples cover bins_per_tile output bins plus the low-pass
// halo, so no beam sample ever goes to global memory.
#include "ptx.cuh"
#include "rtis_internal.h"

namespace rtis {
namespace {

constexpr uint32_t kWaitPolls = 1u << 22;  // bounded mbarrier wait (~ seconds)

__global__ void steering_table_kernel(const float* __restrict__ mic, const float* __restrict__ dirs,
                                      const float* __restrict__ gain, const float* __restrict__ delay_s,
                                      int M, int D, double fs, double fs_over_c, int Jlim,
                                      int* __restrict__ shift, float4* __restrict__ wt,
                                      unsigned* __restrict__ status) {
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
    int j = 0;
    if (fabs(jf) <= static_cast<double>(Jlim)) {
        j = static_cast<int>(jf);
    } else {  // outside the staged halo (or not finite): contribute nothing, report
        atomicOr(status, RTIS_DEV_DELAY_RANGE);
        w = make_float4(0.f, 0.f, 0.f, 0.f);
    }
    shift[idx] = j;
    wt[idx] = w;
}

struct TdArgs {
    const int* shift;
    const float4* wt;
    const float* h;
    float* E;
    unsigned* status;
    int M, N, D, R, lpf_len, n_out, H, row, nbox, bins_per_tile;
};

__global__ void __launch_bounds__(32 * kTdDirsPerCta, 2)
    td_beamform_kernel(const __grid_constant__ CUtensorMap tmap, const TdArgs args) {
    constexpr int NT = 32 * kTdDirsPerCta;
    constexpr int MS = kTdMicsPerStage;
    constexpr int T = kTdOutPerThread;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    const int row = args.row;
    float2* stage = reinterpret_cast<float2*>(smem_raw);
    uint64_t* bar = reinterpret_cast<uint64_t*>(smem_raw + static_cast<size_t>(kTdStages) * MS * row * 8);
    float* hs = reinterpret_cast<float*>(bar + kTdStages);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int d = blockIdx.x * kTdDirsPerCta + warp;
    const int i0 = blockIdx.y * args.bins_per_tile;
    const int half = (args.lpf_len - 1) >> 1;
    const int n_start = args.R * i0 - half;
    const int x0 = (n_start - args.H) & ~1;  // even: 16-byte aligned TMA x coordinate
    const int M = args.M;
    const int nstages = (M + MS - 1) / MS;
    const uint32_t stage_bytes = static_cast<uint32_t>(MS * args.nbox * kTdBox * 8);

    auto issue = [&](int s) {
        const int b = s % kTdStages;
        ptx::mbar_arrive_expect_tx(&bar[b], stage_bytes);
        for (int mi = 0; mi < MS; ++mi) {
            float2* dst = stage + static_cast<size_t>(b * MS + mi) * row;
            for (int bx = 0; bx < args.nbox; ++bx)
                ptx::tma_load_2d(dst + bx * kTdBox, &tmap, x0 + bx * kTdBox, s * MS + mi, &bar[b]);
        }
    };

    if (threadIdx.x == 0) {
        ptx::prefetch_tmap(&tmap);
        for (int s = 0; s < kTdStages; ++s) ptx::mbar_init(&bar[s], 1);
        ptx::fence_mbar_init();
        ptx::fence_proxy_async();
    }
    for (int j = threadIdx.x; j < args.lpf_len; j += NT) hs[j] = args.h[j];
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int s = 0; s < kTdStages && s < nstages; ++s) issue(s);
    }

    // lane m of each warp holds the steering entry of mic m for this warp's direction
    const bool dir_ok = d < args.D;
    int my_shift = 0;
    float4 my_w = make_float4(0.f, 0.f, 0.f, 0.f);
    if (dir_ok && lane < M) {
        my_shift = __ldg(args.shift + static_cast<size_t>(d) * M + lane);
        my_w = __ldg(args.wt + static_cast<size_t>(d) * M + lane);
    }

    float2 acc[T];
#pragma unroll
    for (int t = 0; t < T; ++t) acc[t] = make_float2(0.f, 0.f);
    const int lane_base = n_start - x0 + lane * T - 1;  // smem index of a[n_start + lane*T - 1]

    int s = 0;
    bool timed_out = false;
    for (; s < nstages; ++s) {
        const int b = s % kTdStages;
        const uint32_t par = static_cast<uint32_t>((s / kTdStages) & 1);
        const bool ok = ptx::mbar_wait_bounded(&bar[b], par, kWaitPolls);
        if (__syncthreads_or(!ok)) {
            timed_out = true;
            break;
        }
        if (dir_ok) {
#pragma unroll 1
            for (int mi = 0; mi < MS; ++mi) {
                const int m = s * MS + mi;
                if (m >= M) break;
                const int J = __shfl_sync(0xffffffffu, my_shift, m);
                const float w0 = __shfl_sync(0xffffffffu, my_w.x, m);
                const float w1 = __shfl_sync(0xffffffffu, my_w.y, m);
                const float w2 = __shfl_sync(0xffffffffu, my_w.z, m);
                const float w3 = __shfl_sync(0xffffffffu, my_w.w, m);
                const float2* rp = stage + static_cast<size_t>(b * MS + mi) * row + lane_base + J;
                float2 v0 = rp[0], v1 = rp[1], v2 = rp[2];
#pragma unroll
                for (int t = 0; t < T; ++t) {
                    const float2 v3 = rp[t + 3];
                    float ax = acc[t].x, ay = acc[t].y;
                    ax = fmaf(w0, v0.x, ax);
                    ay = fmaf(w0, v0.y, ay);
                    ax = fmaf(w1, v1.x, ax);
                    ay = fmaf(w1, v1.y, ay);
                    ax = fmaf(w2, v2.x, ax);
                    ay = fmaf(w2, v2.y, ay);
                    ax = fmaf(w3, v3.x, ax);
                    ay = fmaf(w3, v3.y, ay);
                    acc[t] = make_float2(ax, ay);
                    v0 = v1;
                    v1 = v2;
                    v2 = v3;
                }
            }
        }
        __syncthreads();  // buffer b fully consumed
        if (threadIdx.x == 0 && s + kTdStages < nstages) issue(s + kTdStages);
    }

    if (timed_out) {
        // report, then give copies still in flight a bounded chance to land
        if (threadIdx.x == 0) {
            atomicOr(args.status, RTIS_DEV_TIMEOUT);
            for (int r = s; r < nstages && r < s + kTdStages; ++r)
                ptx::mbar_wait_bounded(&bar[r % kTdStages], static_cast<uint32_t>((r / kTdStages) & 1),
                                       kWaitPolls);
        }
        __syncthreads();
        return;
    }

    // epilogue: envelope of this warp's beam over the tile, then low-pass + subsample
    float* env = reinterpret_cast<float*>(smem_raw) + warp * kTdWarpSamples;
#pragma unroll
    for (int t = 0; t < T; ++t) {
        const int n = n_start + lane * T + t;
        const float e = (n >= 0 && n < args.N) ? sqrtf(acc[t].x * acc[t].x + acc[t].y * acc[t].y) : 0.f;
        env[lane * T + t] = e;
    }
    __syncwarp();
    if (dir_ok) {
        float* Erow = args.E + static_cast<size_t>(d) * args.n_out;
        for (int il = lane; il < args.bins_per_tile; il += 32) {
            const int i = i0 + il;
            if (i >= args.n_out) break;
            const float* e = env + args.R * il;
            float acc_e = 0.f;
            for (int j = 0; j < args.lpf_len; ++j) acc_e = fmaf(hs[j], e[j], acc_e);
            Erow[i] = acc_e;
        }
    }
}

}  // namespace

cudaError_t launch_steering_table(Plan& p, cudaStream_t st) {
    const int total = p.M * p.D;
    const int nt = 256;
    steering_table_kernel<<<(total + nt - 1) / nt, nt, 0, st>>>(p.d_mic, p.d_dirs, p.d_gain, p.d_delay, p.M, p.D,
                                                              p.fs, p.fs / p.c, p.Jlim, p.d_shift, p.d_wt,
                                                              p.d_status);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) p.table_dirty = false;
    return e;
}

size_t td_smem_bytes(const Plan& p) {
    return static_cast<size_t>(kTdStages) * kTdMicsPerStage * p.td_row * 8 + kTdStages * 8 +
           static_cast<size_t>(p.lpf_len) * 4;
}

cudaError_t td_configure(const Plan& p) {
    return cudaFuncSetAttribute(td_beamform_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                static_cast<int>(td_smem_bytes(p)));
}

cudaError_t launch_td_beamform(const Plan& p, const CUtensorMap& tmap, float* d_out, cudaStream_t st) {
    TdArgs a;
    a.shift = p.d_shift;
    a.wt = p.d_wt;
    a.h = p.d_h;
    a.E = d_out;
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
    const dim3 grid((p.D + kTdDirsPerCta - 1) / kTdDirsPerCta,
                    (p.n_out + p.td_bins_per_tile - 1) / p.td_bins_per_tile);
    td_beamform_kernel<<<grid, 32 * kTdDirsPerCta, td_smem_bytes(p), st>>>(tmap, a);
    return cudaGetLastError();
}

}  // namespace rtis
