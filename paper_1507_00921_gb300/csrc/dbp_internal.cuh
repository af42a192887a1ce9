// Internal types shared by the planner and the kernels of libdbp.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "dbp.h"

namespace dbp {

// Three-pass FFT geometry N = N2 * N1 * N0 (passes in that order, strides N0*N1, N0, 1).
// The last pass (radix N0) is contiguous; its output sits at the digit-reversed position
// p = k2 + N0 k1 + N0 N1 k0 of frequency k = k0 + N2 k1 + N2 N1 k2.
template <int N>
struct Geo {
    static constexpr int N0 = (N >= 8192) ? 32 : 16;
    static constexpr int N1 = (N <= 512) ? 8 : 16;
    static constexpr int N2 = N / (N0 * N1);
    static constexpr int T = N / 16;                 // threads per CTA
    static constexpr int S1 = N0 * N1;               // stride of the first pass
    static constexpr int PADN = N + 2 * (N / N0);    // float2 per polarization (+16 B per N0)
    static constexpr int PADP = N + 4 * (N / 16);    // floats of P / theta (+16 B per 16)
    static constexpr int MINB = (512 / T) > 0 ? (512 / T) : 1;
    static constexpr size_t SMEM_SSFM = (size_t)2 * PADN * sizeof(float2);
    static constexpr size_t SMEM_ESSFM = SMEM_SSFM + (size_t)2 * PADP * sizeof(float);
};

inline void host_geo(int n, int &n0, int &n1, int &n2) {
    n0 = (n >= 8192) ? 32 : 16;
    n1 = (n <= 512) ? 8 : 16;
    n2 = n / (n0 * n1);
}

// Number of 8-tap filter blocks used by the kernels for N_c taps.
inline int tap_blocks(int n_taps) { return (n_taps + 7) / 8; }

struct FwdParams {
    const float2 *in;
    float2 *out;
    long long n;            // samples per polarization per waveform
    int n_blocks;           // overlap-save blocks per waveform
    int valid;              // N - O
    int half_overlap;       // O / 2
    int boundary;           // DBP_PERIODIC / DBP_ZERO
    int n_steps;
    int n_tapblk;           // 8-tap filter blocks (ESSFM)
    int taps_stride;        // floats per step in `taps`
    long long h_stride;     // float2 between consecutive steps' H tables (0: shared)
    const float2 *H;        // [steps][N] H_s / N at digit-reversed positions
    const float *taps;      // [steps][taps_stride]: gamma_eff_s * c_{s,i}, zero padded
    const float2 *tw1;      // [N0 N1][N2] W_N^{c k}
    const float2 *tw2;      // [N0][N1] W_{N0 N1}^{n0 k1}
};

struct PlanImpl {
    dbp_link link;
    dbp_signal signal;
    dbp_plan_info info;
    int method;
    int coeffs_per_step;
    int n_tapblk;
    int taps_stride;
    bool h_shared;            // all steps share one H table
    int device;
    // device tables
    float2 *d_H = nullptr;
    float *d_taps = nullptr;
    float2 *d_tw1 = nullptr;
    float2 *d_tw2 = nullptr;
    // host copies
    double *step_dz = nullptr;
    double *step_geff = nullptr;
    // host-staging scratch for dbp_run_host
    void *d_stage_in = nullptr;
    void *d_stage_out = nullptr;
    size_t stage_bytes = 0;
    cudaStream_t aux[2] = {nullptr, nullptr};
    cudaEvent_t ev[3] = {nullptr, nullptr, nullptr};
};

// Kernel launchers (one translation unit per block length).
int launch_fwd_512(const FwdParams &, int n_wave, bool essfm, cudaStream_t);
int launch_fwd_1024(const FwdParams &, int n_wave, bool essfm, cudaStream_t);
int launch_fwd_2048(const FwdParams &, int n_wave, bool essfm, cudaStream_t);
int launch_fwd_4096(const FwdParams &, int n_wave, bool essfm, cudaStream_t);
int launch_fwd_8192(const FwdParams &, int n_wave, bool essfm, cudaStream_t);

}  // namespace dbp

struct dbp_plan {
    dbp::PlanImpl impl;
};
