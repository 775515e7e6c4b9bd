// Internal definitions shared by the host API and the kernels of the eRTIS
// energyscape library.  Not part of the public ABI (see include/rtis.h).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "../../include/rtis.h"

namespace rtis {

// ----------------------------------------------------------------------------
// time-domain beamformer tiling (kernels_das.cu)
// ----------------------------------------------------------------------------
constexpr int kTdOutPerThread = 30;                   // even: 16-byte pair loads, conflict-free
constexpr int kTdWarpSamples = 32 * kTdOutPerThread;  // samples one warp beamforms
constexpr int kTdDirsPerCta = 8;                      // one warp per direction
constexpr int kTdMicsPerStage = 2;                    // mics per TMA stage
constexpr int kTdStages = 4;                          // smem ring depth
constexpr int kTdBox = 256;                           // TMA box width (8-byte elements)
constexpr int kMaxMics = 32;                          // lanes hold per-mic steering

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
    // device workspaces (owned)
    float2* d_Z = nullptr;      // [M][2][P] half-size spectra
    float2* d_a = nullptr;      // [M][N] analytic matched-filter output
    unsigned* d_status = nullptr;
    size_t bytes = 0;

    CUtensorMap tmap_a;         // TMA view of d_a as [M][N] 8-byte elements
    bool table_dirty = true;
};

// ----------------------------------------------------------------------------
// error reporting (thread-local last message)
// ----------------------------------------------------------------------------
void set_error(const std::string& msg);
rtis_status fail(rtis_status s, const std::string& msg);
rtis_status cuda_fail(cudaError_t e, const char* what);

// ----------------------------------------------------------------------------
// launchers (return cudaGetLastError() of the launch)
// ----------------------------------------------------------------------------
cudaError_t launch_mf_forward(const Plan& p, const int16_t* d_in, cudaStream_t st);
cudaError_t launch_mf_inverse(const Plan& p, float2* d_a, float2* d_A, cudaStream_t st);
cudaError_t launch_steering_table(Plan& p, cudaStream_t st);
cudaError_t launch_td_beamform(const Plan& p, const CUtensorMap& tmap, float* d_out, cudaStream_t st);
size_t td_smem_bytes(const Plan& p);
cudaError_t td_configure(const Plan& p);

bool encode_tmap_2d_u64(CUtensorMap* map, const void* base, uint64_t cols, uint64_t rows,
                        uint32_t box_cols, uint32_t box_rows, std::string* err);

}  // namespace rtis

struct rtis_plan {
    rtis::Plan p;
};
