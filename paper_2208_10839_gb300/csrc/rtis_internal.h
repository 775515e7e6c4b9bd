// Internal definitions shared by the host API and the kernels of the eRTIS
// energyscape library.  Not part of the public ABI (see include/rtis.h).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/rtis.h"

namespace rtis {

// ----------------------------------------------------------------------------
// time-domain beamformer tiling (kernels_das.cu)
// ----------------------------------------------------------------------------
constexpr int kTdOutPerThread = 30;                   // even: 16-byte pair loads, conflict-free
constexpr int kTdWarpSamples = 32 * kTdOutPerThread;  // samples one warp beamforms
constexpr int kTdWarps = 16;                          // time-domain beamformer: directions (consumer warps) per CTA
constexpr int kTdBox = 256;                           // TMA box width (8-byte elements)
constexpr int kTdBarrierBytes = 256;                  // full/empty mbarriers, abort flag, issue counters
constexpr int kTdThreads = 32 * (kTdWarps + 4);       // consumer warps + a producer warpgroup, one CTA per SM
constexpr int kTdConsumerRegs = 112;                  // after setmaxnreg: 512 x 112 + 128 x 24 <= 640 x 96
constexpr int kTdProducerRegs = 24;
constexpr int kMaxMics = 32;                          // lanes hold per-mic steering

// complex-baseband beamformer (kernels_bb.cu): the same CTA shape on a grid of
// every 4th sample
constexpr int kBbWarps = 16;                          // directions (consumer warps) per CTA
constexpr int kBbThreads = 32 * (kBbWarps + 4);       // + a producer warpgroup; registers as kTd*Regs
constexpr int kBbQ = 4;                               // full-rate samples per coarse sample
constexpr int kBbOutPerThread = 14;                   // coarse samples per lane: T/2 odd, conflict-free 16-byte loads
constexpr int kBbWarpSamples = 32 * kBbOutPerThread;
constexpr int kBbBox = 96;                            // TMA box width (8-byte elements)
constexpr int kBbVariants = 6;  // stage layouts: (2, 8), (4, 4), (4, 5), (2, 10), (4, 8), (8, 4)

// |z| from |z|^2 = x^2 + y^2 as n2 rsqrt(n2) (a few ulp, no slow path); 0 for 0, and a
// NaN stays NaN (n2 * 0) so non-finite inputs still show in the output
__device__ __forceinline__ float magnitude_from_norm(float n2) { return n2 > 0.f ? n2 * rsqrtf(n2) : n2 * 0.f; }

// PDM demodulation (kernels_pdm.cu)
constexpr int kPdmMaxTaps = 256;

// ----------------------------------------------------------------------------
// plan
// ----------------------------------------------------------------------------
struct Plan {
    // sizes
    int M = 0, N = 0, D = 0, L = 0;
    int F = 0, P = 0, logP = 0;       // FFT length and quarter length (P = F/4)
    int k_lo = 0, k_hi = 0, Kb = 0;   // in-band bins
    int R = 0, lpf_len = 0, n_out = 0;
    int H = 0, Jlim = 0;              // TD staging halo and accepted |shift|
    int td_bins_per_tile = 0, td_row = 0, td_nbox = 0;
    int td_variant = 0, td_grid = 0;  // beamformer stage layout and grid, autotuned at creation
    float td_tuned_ms = 0.f;
    float td_variant_ms[2 * 8] = {};  // autotuner: mean ms per (layout, grid choice), 0 if not tried
    double fs = 0, c = 0;
    rtis_options opt{};

    // device tables (owned)
    float* d_mic = nullptr;     // [M][3]
    float* d_dirs = nullptr;    // [D][3]
    float* d_gain = nullptr;    // [M]
    float* d_delay = nullptr;   // [M] seconds
    float2* d_tw = nullptr;     // [F] exp(-2 pi i j / F)
    float2* d_C = nullptr;      // [Kb] 2 conj(S[k]) / F
    float* d_h = nullptr;       // [lpf_len]
    int* d_shift = nullptr;     // [D][M]
    float4* d_wt = nullptr;     // [D][M]
    float2* d_dphase = nullptr; // [D][M] delta / F (hi, lo)
    float4* d_wraw = nullptr;   // [D][M] Catmull-Rom weights without the gain (adjoint)
    float4* d_wder = nullptr;   // [D][M] their slopes d/dmu (adjoint)
    float2* d_adj = nullptr;    // [range tiles][D][M] adjoint partials (d/d delta, d/d gain)
    float* d_adj_red = nullptr; // [M][16][5] first-stage sums of the adjoint reduction
    // device workspaces (owned)
    float2* d_Z = nullptr;      // [M][2][P] half-size spectra
    float2* d_a = nullptr;      // [M][N] analytic matched-filter output
    float2* d_A = nullptr;      // [M][Kb] in-band matched-filter spectra (frequency-domain path)
    uint32_t* d_a16 = nullptr;  // [M][N] a as BF16 (re, im) pairs (time-domain path, BF16 storage)
    // batched frequency-domain path (rtis_process_many): spectra of up to max_batch
    // measurements as GEMM frames, the steered spectra, and the GEMM's bin "frequencies" k
    int max_batch = 0;
    float2* d_X = nullptr;      // [Kb][M][T] in-band spectra, frame t = measurement t
    float2* d_Y = nullptr;      // [D][Kb][T] steered spectra
    float2* d_kbin = nullptr;   // [Kb] (k_lo + k', 0): phase k delta/F uses d_dphase as "tau"
    float* d_xmax = nullptr;    // [M] per-channel max |X| bits for the GEMM scales
    float2* d_Zb = nullptr;     // [max_batch][M][2][P] half spectra, one set per measurement
    float2* d_ab = nullptr;     // [max_batch][M][N] analytic signals, one per measurement
    unsigned char* d_fdtc = nullptr;  // the tensor-core IFFT's two DFT matrices (hi/lo BF16), or null
    int fd_ifft = 0;            // RTIS_FD_IFFT_FFT or RTIS_FD_IFFT_TC (batched frequency-domain path)
    int n_sm = 0;               // multiprocessors of the plan's device
    std::vector<CUtensorMap> tmap_ab;  // TMA views of the d_ab rows (time-domain beamformer)
    unsigned* d_status = nullptr;
    size_t bytes = 0;

    // complex-baseband path (RTIS_PATH_BB): z [M][Nb] lives in d_a
    int Nb = 0, k_c = 0;        // coarse samples N/4; demodulation bin floor((k_lo + k_hi)/2)
    int bb_stride = 0;          // row stride of z in elements (Nb rounded up to even: 16-byte rows)
    int bb_H = 0, bb_Jlim = 0;  // coarse staging halo and accepted |floor(delta/4)|
    int bb_row = 0, bb_nbox = 0, bb_bins_per_tile = 0, bb_ntap = 0;
    int bb_variant = 0, bb_grid = 0;  // baseband stage layout and grid, autotuned at creation
    float bb_tuned_ms = 0.f;
    float bb_variant_ms[2 * 8] = {};
    int* d_bshift = nullptr;    // [D][M] floor(delta / 4)
    float4* d_bwt = nullptr;    // [D][M] Catmull-Rom weights of delta/4 - floor(delta/4)
    float2* d_brot = nullptr;   // [D][M] g_m (cos, sin)(2 pi k_c delta / F)
    float* d_hb = nullptr;      // [4][bb_ntap] coarse low-pass taps by (R i - half) mod 4
    CUtensorMap tmap_zb;        // TMA view of z as [M][Nb] 8-byte elements, rows bb_stride apart

    CUtensorMap tmap_a;         // TMA view of d_a as [M][N] 8-byte elements
    CUtensorMap tmap_a16;       // TMA view of d_a16 as [M][N] 4-byte elements (BF16 plans)
    bool a_bf16 = false;        // rtis_process / batches beamform from the BF16 copy of a
    bool table_dirty = true;

    // kernel tracing (rtis_plan_set_tracing): an event pair around every launch of a
    // traced call, in launch order; the list restarts with each traced call
    bool trace_on = false;
    bool trace_live = false;    // the current call records (tracing on, stream not capturing)
    int trace_n = 0;
    cudaEvent_t trace_ev[2 * RTIS_TRACE_MAX] = {};
    int trace_kind[RTIS_TRACE_MAX] = {};
};

// tracing helpers: trace_call starts a traced call's list; trace_begin/trace_end
// bracket one launch (slot -1: not recorded)
void trace_call(Plan& p, cudaStream_t st);
int trace_begin(Plan& p, cudaStream_t st, int kind);
void trace_end(Plan& p, cudaStream_t st, int slot);

// ----------------------------------------------------------------------------
// frequency-domain beamforming GEMM (kernels_fd.cu)
// ----------------------------------------------------------------------------
constexpr int kFdMaxFrames = 64;
struct FdGemmPlan {
    int M = 0, D = 0, K = 0, T = 0, precision = 0;
    int y_dkt = 0;              // output layout: 0 = [K][D][T] (public ABI), 1 = [D][K][T]
    int n_sm = 0;               // persistent grid size
    float2* d_tau = nullptr;    // [D][M] seconds, (hi, lo)
    float2* d_freq = nullptr;   // [K] Hz, (hi, lo)
    float* d_gain = nullptr;    // [M]
    float* d_scale = nullptr;   // [M] per-channel max |Re X|, |Im X| of the last run (float bits)
    unsigned* d_status = nullptr;
};
// ymap: TMA view of Y (fd_gemm_encode_ymap) or nullptr for plain stores
cudaError_t launch_fd_gemm(const FdGemmPlan& g, const float2* d_X, float2* d_Y, const CUtensorMap* ymap,
                           cudaStream_t st);
bool fd_gemm_encode_ymap(const FdGemmPlan& g, float2* d_Y, CUtensorMap* map, std::string* err);

// ----------------------------------------------------------------------------
// error reporting (thread-local last message)
// ----------------------------------------------------------------------------
void set_error(const std::string& msg);
// host fault injection (RTIS_FAULT): 0 none, 1 alloc, 2 launch, 3 stall
enum { kFaultNone = 0, kFaultAlloc = 1, kFaultLaunch = 2, kFaultStall = 3 };
int fault_mode();
rtis_status fail(rtis_status s, const std::string& msg);
rtis_status cuda_fail(cudaError_t e, const char* what);

// ----------------------------------------------------------------------------
// launchers (return cudaGetLastError() of the launch)
// ----------------------------------------------------------------------------
// several measurements per matched-filter launch (grid z): measurement t reads
// d_in + t x_stride and uses the half spectra Z + t z_stride (Z = nullptr: the
// plan's single buffer), and writes a + t a_stride, A + t A_tstride
struct MfBatch {
    int n = 1;
    size_t x_stride = 0;
    float2* Z = nullptr;
    size_t z_stride = 0, a_stride = 0, A_tstride = 0;
};
cudaError_t launch_mf_forward(const Plan& p, const int16_t* d_in, cudaStream_t st, const MfBatch& mb = MfBatch());
// writes a (complex float) and/or a16 (BF16 pairs) and/or the in-band spectra A,
// A_m[k'] at d_A[m a_ms + k' a_ks] (default a_ms = Kb, a_ks = 1)
cudaError_t launch_mf_inverse(const Plan& p, float2* d_a, float2* d_A, cudaStream_t st, uint32_t* d_a16 = nullptr,
                              int a_ms = -1, int a_ks = 1, const MfBatch& mb = MfBatch());
cudaError_t launch_steering_table(Plan& p, cudaStream_t st);
// the matched filters of several sensors (their own N, F, band) in two launches:
// every sensor's forward FFTs, then every sensor's four phase IFFTs, into each
// plan's own workspaces (a, or a16 for BF16 plans)
constexpr int kMfMaxSensors = 16;
struct MfRaggedSensor {
    const int16_t* x;
    float2* Z;
    const float2* tw;
    const float2* C;
    float2* a;
    uint32_t* a16;
    int N, F, logP, k_lo, Kb, item0;
};
struct MfRagged {
    MfRaggedSensor s[kMfMaxSensors];
    int n;
};
cudaError_t launch_mf_ragged(const Plan* const* plans, int n, const int16_t* const* d_in, cudaStream_t st);
// z_m[j] = a_m[4j] exp(-2 pi i k_c 4j / F), j < Nb, into d_z rows `stride` elements apart
// (phase-0 inverse only; the half spectra come from launch_mf_forward)
cudaError_t launch_mf_inverse_bb(const Plan& p, float2* d_z, int stride, cudaStream_t st);
// zmap: TMA view of z as [M][Nb] 8-byte elements
cudaError_t launch_bb_beamform(const Plan& p, const CUtensorMap& zmap, float* d_out, cudaStream_t st);
// x [n_mics][n_samples] int16 from n_words PDM words (taps: host, n_taps <= kPdmMaxTaps)
cudaError_t launch_pdm_demod(const uint32_t* d_words, long long n_words, int n_mics, int n_samples, int decim,
                             const int32_t* taps, int n_taps, int shift, int16_t* d_x, cudaStream_t st);
size_t bb_smem_bytes(const Plan& p);  // the smallest stage layout's
bool bb_variant_fits(const Plan& p, int variant);
int bb_tiles(const Plan& p);
cudaError_t bb_autotune(Plan& p, float* d_scratch_out);
// bf16: tmap views BF16 pairs (4-byte elements) rather than complex floats
cudaError_t launch_td_beamform(const Plan& p, const CUtensorMap& tmap, bool bf16, float* d_out, cudaStream_t st);
// the smallest layout's shared memory (what a plan needs at least)
size_t td_smem_bytes(const Plan& p);
// fast: every sensor uses R = 10 and the 41-tap low-pass (the register epilogue)
size_t td_smem_bytes(int row_max, bool fast, int variant);
bool td_variant_fits(int row_max, bool fast, int variant);
bool td_fast_epilogue(int R, int lpf_len);
cudaError_t launch_fd_energyscape(const Plan& p, const float2* d_A, float* d_out, cudaStream_t st);
// energyscapes of T measurements from their steered spectra Y [D][Kb][T]; out [T][D][n_out]
cudaError_t launch_fd_energyscape_from_y(const Plan& p, const float2* d_Y, int T, float* d_out, cudaStream_t st);
size_t fdes_smem_bytes(const Plan& p);
// the same from Y with the inverse transform as two dense DFT stages on the tensor
// cores (kernels_fdtc.cu); d_W holds fdtc_build_constants' image, d_out is zeroed first
bool fdtc_supported(const Plan& p);
size_t fdtc_const_bytes();
void fdtc_build_constants(const Plan& p, std::vector<unsigned char>& img);
cudaError_t launch_fd_energyscape_tc(const Plan& p, const unsigned char* d_W, const float2* d_Y, int T, float* d_out,
                                     int n_sm, cudaStream_t st);

// persistent multi-sensor time-domain beamformer
constexpr int kTdMaxSensors = 16;
constexpr int kTdVariants = 5;  // (mics per stage, stages): (2, 8), (4, 4), (2, 10), (4, 5), (1, 8)
int td_variant_ms(int variant);  // mics per stage of a layout
int td_variant_ns(int variant);  // its ring depth
struct TdSensor {
    const int* shift;
    const float4* wt;
    const float* h;
    float* E;
    int M, N, D, R, lpf_len, n_out, H, row, nbox, bins_per_tile;
    int n_dgroups, tile_base;  // tiles: n_dgroups x range tiles, from tile_base on
};
struct TdBatch {
    TdSensor s[kTdMaxSensors];
    int n_sensors, total_tiles, row_max, lpf_max;
    int bf16;  // the staged rows are BF16 (re, im) pairs, 4 bytes per sample
    int stall;  // fault injection: withhold each CTA's first copy and wait for it briefly
    unsigned* status;
};
struct TdMaps {
    CUtensorMap m[kTdMaxSensors];
};
void td_fill_sensor(const Plan& p, float* d_out, int tile_base, TdSensor* s);
int td_tiles(const Plan& p);
cudaError_t td_autotune(Plan& p, float* d_scratch_out);
cudaError_t launch_td_adjoint(const Plan& p, const float* d_grad_out, float* d_gxyz, float* d_ggain, float* d_gdelay,
                              cudaStream_t st);
cudaError_t launch_l2_loss(const Plan& p, const float* d_E, const float* d_Eref, float* d_G, float* d_loss,
                           cudaStream_t st);
size_t adj_smem_bytes(const Plan& p);
cudaError_t launch_td_batch(const TdMaps& maps, const TdBatch& bt, int variant, int grid, cudaStream_t st);

bool encode_tmap_2d_u64(CUtensorMap* map, const void* base, uint64_t cols, uint64_t rows,
                        uint32_t box_cols, uint32_t box_rows, std::string* err);
bool encode_tmap_2d_u32(CUtensorMap* map, const void* base, uint64_t cols, uint64_t rows,
                        uint32_t box_cols, uint32_t box_rows, std::string* err);
// generic tiled tensor map: dims[rank], strides[rank-1] in bytes, box[rank]
bool encode_tmap(CUtensorMap* map, CUtensorMapDataType dtype, uint32_t rank, const void* base, const uint64_t* dims,
                 const uint64_t* strides, const uint32_t* box, CUtensorMapSwizzle swizzle, std::string* err);

}  // namespace rtis

struct rtis_plan {
    rtis::Plan p;
};

struct rtis_fd_gemm {
    rtis::FdGemmPlan g;
};
