// Frequency-domain delay-and-sum as a batched complex GEMM on the tcgen05
// tensor cores.  For every frequency bin k:
//
//   Y[k][d][t] = sum_m W[k][d][m] X[k][m][t],   W = g_m exp(+2 pi i f_k tau_dm)
//
// (the phase ramp of a delay tau_dm, i.e. delay-and-sum of the paper's Fig. 3
// and Sec. 4.1 written per frequency).  The complex product runs as one real
// GEMM whose output columns interleave (re, im):
//
//   A[d]       = [ Re W[d][0..31] | Im W[d][0..31] ]            (M = 128 directions, K = 64)
//   B[2t]      = [ Re X[0..31][t] | -Im X[0..31][t] ]           (N = 2 x 64 frames)
//   B[2t + 1]  = [ Im X[0..31][t] |  Re X[0..31][t] ]
//   C[d][2t + c] = A[d] . B[2t + c] = (Re, Im) Y[k][d][t]
//
// so one accumulator row is one output row in its final interleaved layout.
// The steering operand is never read from memory: threads evaluate the phases
// in compensated FP32 (f and tau carried as hi + lo pairs, the product's
// rounding error recovered with an FMA, integer cycles removed exactly) and
// write W straight into shared memory in the canonical K-major layout.  X and
// W are scaled per channel by powers of two (X / s_m, W s_m / S, Y x S) so
// FP16 operands stay in range.  Precision modes: BF16 or FP16 operands, or
// "FP32" as three BF16 products hi.hi + hi.lo + lo.hi accumulated in FP32.
//
// Persistent CTAs: CTA c owns a contiguous run of (direction tile, bin)
// items in tile-major order, so its 128 directions' delays stay in registers
// while it walks consecutive bins.  Per item: X of the next bin arrives by a
// bulk async copy; A and B are built; one thread issues the MMAs; an earlier
// item's accumulator goes TMEM -> registers -> 128B-swizzled shared staging
// -> 3-D TMA tensor stores (which clip ragged tiles and frames).  Separate
// warps build and drain, so the two overlap: 8 and 8 with BF16 or FP16
// operands, 16 and 4 in the FP32 mode, whose build (hi and lo halves of both
// operands) is twice as large.
#include <algorithm>
#include <cstring>
#include <string>

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "ptx.cuh"
#include "rtis_internal.h"

namespace rtis {
namespace {

constexpr int kFdDirTile = 128;  // directions per item (MMA M)
constexpr int kFdFrames = 64;    // frames per item (MMA N = 128)
constexpr int kFdK = 64;         // 2 x 32 mics
constexpr uint32_t kFdLbo = 128, kFdSbo = 1024;
constexpr uint32_t kFdPolls = 1u << 22;

struct FdArgs {
    const float2* X;      // [K][M][T]
    float2* Y;            // [K][D][T] (direct-store path)
    const float2* tau;    // [D][M] seconds, hi/lo
    const float2* freq;   // [K] Hz, hi/lo
    const float* gain;    // [M]
    const float* scale;   // [M] per-channel max |Re X|, |Im X| as float bits (fd_absmax_kernel)
    unsigned* status;
    int K, M, D, T;
    int n_items;          // direction tiles x bins, item = tile * K + k
    int bulk_x;           // X rows of one bin fetched by one bulk copy (M*T*8 % 16 == 0)
    int tma_y;            // Y written by TMA tensor stores (T even)
    int y_dkt;            // Y laid out [D][K][T] instead of [K][D][T]
};

__device__ __forceinline__ uint32_t kmajor_off(int r, int kc) {
    return static_cast<uint32_t>((r >> 3) * kFdSbo + kc * kFdLbo + (r & 7) * 16);
}

template <int PREC>
__device__ __forceinline__ uint32_t pack_hi(float a, float b) {
    if constexpr (PREC == RTIS_PREC_FP16) {
        __half2 h = __floats2half2_rn(a, b);
        return *reinterpret_cast<uint32_t*>(&h);
    } else {
        __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
        return *reinterpret_cast<uint32_t*>(&h);
    }
}
// residual a - bf16(a), rounded to bf16 (second term of the split)
__device__ __forceinline__ uint32_t pack_lo(float a, float b) {
    const float ra = a - __bfloat162float(__float2bfloat16_rn(a));
    const float rb = b - __bfloat162float(__float2bfloat16_rn(b));
    __nv_bfloat162 h = __floats2bfloat162_rn(ra, rb);
    return *reinterpret_cast<uint32_t*>(&h);
}

// 8 values -> one 16-byte core-matrix row chunk (hi, and lo in FP32 mode)
template <int PREC>
__device__ __forceinline__ void store_chunk(unsigned char* hi, unsigned char* lo, uint32_t off, const float (&v)[8]) {
    uint4 h;
    h.x = pack_hi<PREC>(v[0], v[1]);
    h.y = pack_hi<PREC>(v[2], v[3]);
    h.z = pack_hi<PREC>(v[4], v[5]);
    h.w = pack_hi<PREC>(v[6], v[7]);
    *static_cast<uint4*>(__builtin_assume_aligned(hi + off, 16)) = h;
    if constexpr (PREC == RTIS_PREC_FP32) {
        uint4 l;
        l.x = pack_lo(v[0], v[1]);
        l.y = pack_lo(v[2], v[3]);
        l.z = pack_lo(v[4], v[5]);
        l.w = pack_lo(v[6], v[7]);
        *static_cast<uint4*>(__builtin_assume_aligned(lo + off, 16)) = l;
    }
}

// phase of f * tau in cycles, reduced to about [-1/2, 1/2], in compensated
// FP32: p + e is the exact product of the hi parts.
__device__ __forceinline__ float phase_cycles(float2 f, float2 tau) {
    const float p = f.x * tau.x;
    const float e = fmaf(f.x, tau.x, -p);
    const float r = p - rintf(p);  // exact: r and p are within one unit of each other
    return r + (e + fmaf(f.x, tau.y, f.y * tau.x));
}

template <int PREC>
struct FdSmem {
    static constexpr int NPASS = (PREC == RTIS_PREC_FP32) ? 3 : 1;
    static constexpr int NSPLIT = (PREC == RTIS_PREC_FP32) ? 2 : 1;  // hi (+ lo) copies
    static constexpr uint32_t OP_BYTES = 128 * 128;                  // 128 rows x 64 K x 2 B (A and B alike)
    static constexpr uint32_t X_BYTES = 32 * kFdFrames * 8;          // one bin of X, fp32 complex
    static constexpr uint32_t STG_WARP = 32 * 128;                   // per-warp box: 32 rows x 128 B
    static constexpr uint32_t STG_OFF = 0;                           // 1024-byte aligned (128B swizzle)
    static constexpr uint32_t A_OFF = STG_OFF + 16 * STG_WARP;
    static constexpr uint32_t B_OFF = A_OFF + 2 * NSPLIT * OP_BYTES;  // [buf][split]
    static constexpr uint32_t X_OFF = B_OFF + 2 * NSPLIT * OP_BYTES;
    static constexpr uint32_t BAR_OFF = X_OFF + 2 * X_BYTES;
    static constexpr uint32_t BYTES = BAR_OFF + 6 * 8 + 4 + 65 * 4;
    static constexpr uint32_t ALLOC = BYTES + 1024;                  // room to align the base
};

// The warp-specialised form: NB builder warps build item j's operands (X and W into buffer
// j & 1) and thread 0 issues its MMAs once every builder has passed a named barrier; the drain
// warps after them empty the accumulators (TMEM -> registers -> swizzled staging -> TMA store).
// The two groups hand over through mbarriers: mma_bar (MMAs of an item retired: its operand
// buffer is free and its accumulator ready) and tfree (an accumulator drained).  NB = 8 (BF16,
// FP16: 8 drain warps, each builder thread two mic octets of W and both rows of a frame's X
// octet) or 16 (FP32, whose hi/lo build is twice as large: 4 drain warps, each builder thread one
// octet of W and one row of X, as in the all-warps form).
template <int NB>
__host__ __device__ constexpr int fd_ws_threads() { return 32 * (NB + (NB == 8 ? 8 : 4)); }

template <int PREC, int NB>
__global__ void __launch_bounds__(fd_ws_threads<NB>(), 1)
    fd_gemm_kernel_ws(const __grid_constant__ CUtensorMap ymap, const FdArgs args) {
    static_assert(NB == 8 || NB == 16, "8 or 16 builder warps");
    constexpr int NDW = NB == 8 ? 8 : 4;       // drain warps
    constexpr int NOCT = NB == 8 ? 2 : 1;      // W mic octets per builder thread
    constexpr int GPW = 16 / NDW;              // 32-column groups per drain warp
    using L = FdSmem<PREC>;
    constexpr uint32_t NCOL = 2 * kFdFrames;  // accumulator columns per buffer
    constexpr uint32_t IDESC = ptx::idesc_f16(PREC == RTIS_PREC_FP16 ? 0u : 1u, 128u, NCOL);
    extern __shared__ __align__(16) unsigned char sm_raw[];
    unsigned char* sm = sm_raw + ((1024 - (ptx::smem_u32(sm_raw) & 1023)) & 1023);
    uint64_t* mma_bar = reinterpret_cast<uint64_t*>(sm + L::BAR_OFF);  // [2]
    uint64_t* x_bar = mma_bar + 2;                                       // [2]
    uint64_t* tfree = x_bar + 2;                                         // [2] accumulator drained
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(tfree + 2);
    float* s_scale = reinterpret_cast<float*>(tmem_slot + 1);  // [65]: s_m, S, 1/s_m
    auto A_ptr = [&](int buf, int split) { return sm + L::A_OFF + (buf * L::NSPLIT + split) * L::OP_BYTES; };
    auto B_ptr = [&](int buf, int split) { return sm + L::B_OFF + (buf * L::NSPLIT + split) * L::OP_BYTES; };
    auto X_ptr = [&](int buf) { return reinterpret_cast<float2*>(sm + L::X_OFF + buf * L::X_BYTES); };

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int M = args.M, D = args.D, T = args.T, K = args.K;
    const int first = static_cast<int>((static_cast<long long>(blockIdx.x) * args.n_items) / gridDim.x);
    const int last = static_cast<int>((static_cast<long long>(blockIdx.x + 1) * args.n_items) / gridDim.x);
    const int n_local = last - first;
    const uint32_t x_bytes = static_cast<uint32_t>(M * T * 8);

    if (warp == 0) {
        ptx::tmem_alloc(tmem_slot, 2 * NCOL);
        ptx::tmem_relinquish();
    }
    if (tid == 0) {
        for (int i = 0; i < 2; ++i) {
            ptx::mbar_init(&mma_bar[i], 1);
            ptx::mbar_init(&x_bar[i], 1);
            ptx::mbar_init(&tfree[i], NDW);  // the drain warps
        }
        ptx::fence_mbar_init();
        if (args.tma_y) ptx::prefetch_tmap(&ymap);
    }
    if (tid < 32) {
        // s_m = smallest power of two >= max |Re X|, |Im X| of mic m (1 if silent or not finite)
        float s = 1.f;
        if (tid < M) {
            const float amax = __uint_as_float(reinterpret_cast<const unsigned*>(args.scale)[tid]);
            if (amax > 0.f && isfinite(amax)) s = exp2f(ceilf(log2f(amax)));
        }
        float mx = tid < M ? s : 0.f;
        for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        s_scale[tid] = s;
        s_scale[33 + tid] = 1.0f / s;  // exact: s is a power of two
        if (tid == 0) s_scale[32] = mx;
    }
    ptx::tc_fence_before();
    __syncthreads();
    ptx::tc_fence_after();
    const float S = s_scale[32];
    const uint32_t tmem = *tmem_slot;

    auto issue_x = [&](int j) {  // thread 0: bin of local item j -> X buffer j & 1
        if (!args.bulk_x || j >= n_local) return;
        const int k = (first + j) % K;
        ptx::mbar_arrive_expect_tx(&x_bar[j & 1], x_bytes);
        ptx::bulk_load(X_ptr(j & 1), args.X + static_cast<size_t>(k) * M * T, x_bytes, &x_bar[j & 1]);
    };
    if (tid == 0) issue_x(0);

    bool timed_out = false;
    auto wait_bar = [&](uint64_t* bar, uint32_t parity) {
        if (!timed_out && !ptx::mbar_wait_bounded(bar, parity, kFdPolls)) {
            timed_out = true;
            atomicOr(args.status, RTIS_DEV_TIMEOUT);
        }
    };

    if (warp < NB) {
        // ---------------- builders: X and W into the operand buffers, then the MMAs
        const int bt_id = tid;                           // 0 .. 32 NB - 1
        // A role: 128 directions x mic octets {mo0, mo0 + 2} (NB = 8) or {mo0} (NB = 16)
        const int dl = bt_id & 127, mo0 = bt_id >> 7;
        float gsc[NOCT][8];
#pragma unroll
        for (int o = 0; o < NOCT; ++o)
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                const int m = (mo0 + 2 * o) * 8 + i;
                gsc[o][i] = m < M ? __ldg(args.gain + m) * (s_scale[m] / S) : 0.f;
            }
        float2 tv[NOCT][8];
        int tile_loaded = -1;
        // B role: frame bt, mic octet bo; rows 2t ([Re X | -Im X]) and 2t + 1 ([Im X | Re X]),
        // both (NB = 8) or row 2t + bpart (NB = 16)
        const int bt = bt_id & 63, bo = (bt_id >> 6) & 3, bpart = bt_id >> 8;
        float bsc[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const int m = bo * 8 + i;
            bsc[i] = (m < M && bt < T) ? s_scale[33 + m] : 0.f;  // zero also masks padded mics and frames
        }
        int tile = first / K, k = first - tile * K;  // item j = tile * K + k
        float2 f_next = n_local > 0 ? __ldg(args.freq + k) : make_float2(0.f, 0.f);
        for (int j = 0; j < n_local; ++j) {
            const int b = j & 1;
            if (bt_id == 0) issue_x(j + 1);  // its X buffer was last read by item j - 1, before the last barrier
            const float2 f = f_next;
            {
                const int kn = (k + 1 == K) ? 0 : k + 1;
                if (j + 1 < n_local) f_next = __ldg(args.freq + kn);
            }
            if (args.bulk_x) wait_bar(&x_bar[b], static_cast<uint32_t>((j >> 1) & 1));
            // operand buffer b was last read by the MMAs of item j - 2
            if (j >= 2) wait_bar(&mma_bar[b], static_cast<uint32_t>(((j - 2) >> 1) & 1));
            if (!timed_out) {
                float va[8], vb[8], wa[8], wb[8];  // rows 2t: [Re X | -Im X], 2t + 1: [Im X | Re X]
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                    const int m = bo * 8 + i;
                    float2 x = make_float2(0.f, 0.f);
                    if (bsc[i] != 0.f)
                        x = args.bulk_x ? X_ptr(b)[m * T + bt]
                                        : __ldg(args.X + (static_cast<size_t>(k) * M + m) * T + bt);
                    const float xr = x.x * bsc[i], xi = x.y * bsc[i];
                    va[i] = xr;
                    vb[i] = -xi;
                    wa[i] = xi;
                    wb[i] = xr;
                }
                if (NB == 8 || bpart == 0) {
                    store_chunk<PREC>(B_ptr(b, 0), B_ptr(b, L::NSPLIT - 1), kmajor_off(2 * bt, bo), va);
                    store_chunk<PREC>(B_ptr(b, 0), B_ptr(b, L::NSPLIT - 1), kmajor_off(2 * bt, 4 + bo), vb);
                }
                if (NB == 8 || bpart == 1) {
                    store_chunk<PREC>(B_ptr(b, 0), B_ptr(b, L::NSPLIT - 1), kmajor_off(2 * bt + 1, bo), wa);
                    store_chunk<PREC>(B_ptr(b, 0), B_ptr(b, L::NSPLIT - 1), kmajor_off(2 * bt + 1, 4 + bo), wb);
                }
                if (tile != tile_loaded) {
                    const int d = tile * kFdDirTile + dl;
#pragma unroll
                    for (int o = 0; o < NOCT; ++o)
#pragma unroll
                        for (int i = 0; i < 8; ++i) {
                            const int m = (mo0 + 2 * o) * 8 + i;
                            tv[o][i] = (d < D && m < M) ? __ldg(args.tau + static_cast<size_t>(d) * M + m)
                                                        : make_float2(0.f, 0.f);
                        }
                    tile_loaded = tile;
                }
#pragma unroll
                for (int o = 0; o < NOCT; ++o) {
                    float wr[8], wi[8];
#pragma unroll
                    for (int i = 0; i < 8; ++i) {
                        float sn, cs;
                        __sincosf(6.28318530717958647692f * phase_cycles(f, tv[o][i]), &sn, &cs);
                        wr[i] = cs * gsc[o][i];
                        wi[i] = sn * gsc[o][i];
                    }
                    const int mo = mo0 + 2 * o;
                    store_chunk<PREC>(A_ptr(b, 0), A_ptr(b, L::NSPLIT - 1), kmajor_off(dl, mo), wr);
                    store_chunk<PREC>(A_ptr(b, 0), A_ptr(b, L::NSPLIT - 1), kmajor_off(dl, 4 + mo), wi);
                }
            }
            // the operands are visible to the tensor core once every builder has passed here
            ptx::fence_proxy_async();
            asm volatile("bar.sync 1, %0;" ::"n"(32 * NB) : "memory");
            if (bt_id == 0) {
                // accumulator b was last read by the drain of item j - 2
                if (j >= 2) wait_bar(&tfree[b], static_cast<uint32_t>(((j - 2) >> 1) & 1));
                ptx::tc_fence_after();
                if (!timed_out) {
                    const uint32_t d_tmem = tmem + static_cast<uint32_t>(b) * NCOL;
#pragma unroll
                    for (int pass = 0; pass < L::NPASS; ++pass) {
                        const unsigned char* Ap = A_ptr(b, pass == 2 ? 1 : 0);
                        const unsigned char* Bp = B_ptr(b, pass == 1 ? 1 : 0);
#pragma unroll
                        for (int ks = 0; ks < kFdK / 16; ++ks) {
                            const uint64_t ad = ptx::smem_desc_kmajor(Ap + ks * 2 * kFdLbo, kFdLbo, kFdSbo);
                            const uint64_t bd = ptx::smem_desc_kmajor(Bp + ks * 2 * kFdLbo, kFdLbo, kFdSbo);
                            ptx::tc_mma_f16(d_tmem, ad, bd, IDESC, (pass | ks) != 0 ? 1u : 0u);
                        }
                    }
                    ptx::tc_commit(&mma_bar[b]);
                }
            }
            if (++k == K) {
                k = 0;
                ++tile;
            }
        }
    } else {
        // ---------------- drain: accumulator -> registers -> staging -> TMA
        // TMEM lane quarter q; column groups GPW h .. GPW h + GPW - 1 (32 columns = 16 frames each)
        const int dw = warp - NB;
        const int q = dw & 3, h = dw >> 2;
        const int row = 32 * q + lane;
        for (int j = 0; j < n_local; ++j) {
            const int b = j & 1;
            const int item = first + j;
            const int ptile = item / K, pk = item - ptile * K;
            wait_bar(&mma_bar[b], static_cast<uint32_t>((j >> 1) & 1));
            ptx::tc_fence_after();
            if (!__any_sync(0xffffffffu, timed_out)) {
#pragma unroll
                for (int c2 = 0; c2 < GPW; ++c2) {
                    const int cg = GPW * h + c2;
                    unsigned char* stg = sm + L::STG_OFF + (GPW * dw + c2) * L::STG_WARP;
                    uint32_t r[32];
                    ptx::tmem_ld_32x32b_x32(
                        tmem + (static_cast<uint32_t>(32 * q) << 16) + static_cast<uint32_t>(b) * NCOL + 32u * cg, r);
                    ptx::tmem_ld_wait_regs(r);
                    if (args.tma_y) {
                        if (lane == 0) ptx::bulk_wait_read0();  // this warp's earlier boxes have been read
                        __syncwarp();
                        // row `lane`, 16-byte chunk c at (c ^ (lane & 7)): the 128B swizzle
#pragma unroll
                        for (int c = 0; c < 8; ++c) {
                            const float4 v =
                                make_float4(S * __uint_as_float(r[4 * c]), S * __uint_as_float(r[4 * c + 1]),
                                            S * __uint_as_float(r[4 * c + 2]), S * __uint_as_float(r[4 * c + 3]));
                            *static_cast<float4*>(__builtin_assume_aligned(stg + lane * 128 + ((c ^ (lane & 7)) << 4), 16)) = v;
                        }
                        ptx::fence_proxy_async();
                        __syncwarp();
                        if (lane == 0) {
                            if (args.y_dkt)
                                ptx::tma_store_3d(&ymap, stg, 32 * cg, pk, ptile * kFdDirTile + 32 * q);
                            else
                                ptx::tma_store_3d(&ymap, stg, 32 * cg, ptile * kFdDirTile + 32 * q, pk);
                            ptx::bulk_commit();
                        }
                    } else {
                        const int d = ptile * kFdDirTile + row;
                        if (d < D) {
                            float2* dst = args.Y + (args.y_dkt ? (static_cast<size_t>(d) * K + pk)
                                                               : (static_cast<size_t>(pk) * D + d)) * T;
#pragma unroll
                            for (int c = 0; c < 16; ++c) {
                                const int t = 16 * cg + c;
                                if (t < T)
                                    dst[t] = make_float2(S * __uint_as_float(r[2 * c]), S * __uint_as_float(r[2 * c + 1]));
                            }
                        }
                    }
                }
            }
            // accumulator b may be overwritten by item j + 2
            ptx::tc_fence_before();
            __syncwarp();
            if (lane == 0) ptx::mbar_arrive(&tfree[b]);
        }
        if (lane == 0 && args.tma_y) ptx::bulk_wait0();
    }

    // on a timeout: give MMAs and copies in flight a bounded chance to finish before TMEM is released
    if (__syncthreads_or(timed_out)) {
        if (tid == 0) {
            for (int i = 0; i < 2; ++i) {
                ptx::mbar_wait_bounded(&mma_bar[i], 0u, kFdPolls);
                ptx::mbar_wait_bounded(&mma_bar[i], 1u, kFdPolls);
                ptx::mbar_wait_bounded(&x_bar[i], 0u, kFdPolls);
                ptx::mbar_wait_bounded(&x_bar[i], 1u, kFdPolls);
            }
        }
        __syncthreads();
    }
    ptx::tc_fence_after();
    if (warp == 0) ptx::tmem_dealloc(tmem, 2 * NCOL);
}

// Per-mic max of |Re X|, |Im X| over bins and frames, as float bits (the
// values are non-negative, so their bit patterns order like the floats):
// CTAs stride over bins, each thread keeps the maxima of its (mic, frame)
// slots, then shared and global atomicMax.  bits[] starts at zero.
__global__ void __launch_bounds__(256) fd_absmax_kernel(const float2* __restrict__ X, int K, int M, int T,
                                                        unsigned* __restrict__ bits) {
    __shared__ unsigned smax[kMaxMics];
    if (threadIdx.x < kMaxMics) smax[threadIdx.x] = 0u;
    __syncthreads();
    const int MT = M * T;  // <= 32 x 64 = 8 x 256
    float mx[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) mx[j] = 0.f;
    for (int k = blockIdx.x; k < K; k += gridDim.x) {
        const float2* Xk = X + static_cast<size_t>(k) * MT;
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const int i = threadIdx.x + 256 * j;
            if (i < MT) {
                const float2 x = __ldg(Xk + i);
                mx[j] = fmaxf(mx[j], fmaxf(fabsf(x.x), fabsf(x.y)));
            }
        }
    }
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        const int i = threadIdx.x + 256 * j;
        if (i < MT) atomicMax(&smax[i / T], __float_as_uint(mx[j]));
    }
    __syncthreads();
    if (threadIdx.x < M) atomicMax(&bits[threadIdx.x], smax[threadIdx.x]);
}

template <int PREC>
cudaError_t fd_launch_t(const CUtensorMap& ymap, const FdArgs& a, int grid, cudaStream_t st) {
    const size_t sm = FdSmem<PREC>::ALLOC;
    // warp-specialised: 8 builder and 8 drain warps (BF16 / FP16), 16 and 4 (FP32)
    constexpr int NB = (PREC == RTIS_PREC_FP32) ? 16 : 8;
    auto kern = fd_gemm_kernel_ws<PREC, NB>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(sm));
    if (e != cudaSuccess) return e;
    kern<<<grid, fd_ws_threads<NB>(), sm, st>>>(ymap, a);
    return cudaGetLastError();
}

}  // namespace

bool fd_gemm_encode_ymap(const FdGemmPlan& g, float2* d_Y, CUtensorMap* map, std::string* err) {
    if (g.y_dkt) {
        // Y as float32 [D][K][2T]; box = 32 floats (128 B) x 1 bin x 32 directions, 128B swizzle
        uint64_t dims[3] = {static_cast<uint64_t>(2 * g.T), static_cast<uint64_t>(g.K), static_cast<uint64_t>(g.D)};
        uint64_t strides[2] = {static_cast<uint64_t>(g.T) * 8, static_cast<uint64_t>(g.K) * g.T * 8};
        uint32_t box[3] = {32, 1, 32};
        return encode_tmap(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, d_Y, dims, strides, box,
                           CU_TENSOR_MAP_SWIZZLE_128B, err);
    }
    // Y as float32 [K][D][2T]; box = 32 floats (128 B) x 32 directions x 1 bin, 128B swizzle
    uint64_t dims[3] = {static_cast<uint64_t>(2 * g.T), static_cast<uint64_t>(g.D), static_cast<uint64_t>(g.K)};
    uint64_t strides[2] = {static_cast<uint64_t>(g.T) * 8, static_cast<uint64_t>(g.D) * g.T * 8};
    uint32_t box[3] = {32, 32, 1};  // one warp's 32 rows x 128 bytes
    return encode_tmap(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, d_Y, dims, strides, box, CU_TENSOR_MAP_SWIZZLE_128B,
                       err);
}

cudaError_t launch_fd_gemm(const FdGemmPlan& g, const float2* d_X, float2* d_Y, const CUtensorMap* ymap,
                           cudaStream_t st) {
    // per-channel scales come from the max |X| of this call's input
    cudaError_t e = cudaMemsetAsync(g.d_scale, 0, static_cast<size_t>(g.M) * sizeof(float), st);
    if (e != cudaSuccess) return e;
    fd_absmax_kernel<<<std::min(g.K, 4 * std::max(g.n_sm, 1)), 256, 0, st>>>(
        d_X, g.K, g.M, g.T, reinterpret_cast<unsigned*>(g.d_scale));
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    FdArgs a;
    a.X = d_X;
    a.Y = d_Y;
    a.tau = g.d_tau;
    a.freq = g.d_freq;
    a.gain = g.d_gain;
    a.scale = g.d_scale;
    a.status = g.d_status;
    a.K = g.K;
    a.M = g.M;
    a.D = g.D;
    a.T = g.T;
    const int n_tiles = (g.D + kFdDirTile - 1) / kFdDirTile;
    a.n_items = n_tiles * g.K;
    a.bulk_x = ((static_cast<size_t>(g.M) * g.T * 8) % 16 == 0 && reinterpret_cast<uintptr_t>(d_X) % 16 == 0) ? 1 : 0;
    a.tma_y = ymap != nullptr ? 1 : 0;
    a.y_dkt = g.y_dkt;
    CUtensorMap dummy;
    std::memset(&dummy, 0, sizeof(dummy));
    const CUtensorMap& ym = ymap ? *ymap : dummy;
    const int grid = std::min(a.n_items, g.n_sm > 0 ? g.n_sm : 1);
    switch (g.precision) {
        case RTIS_PREC_FP32: return fd_launch_t<RTIS_PREC_FP32>(ym, a, grid, st);
        case RTIS_PREC_BF16: return fd_launch_t<RTIS_PREC_BF16>(ym, a, grid, st);
        case RTIS_PREC_FP16: return fd_launch_t<RTIS_PREC_FP16>(ym, a, grid, st);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace rtis
