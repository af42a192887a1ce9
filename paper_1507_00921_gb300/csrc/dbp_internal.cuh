// Internal types shared by the planner and the kernels of libdbp.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "dbp.h"

namespace dbp {

// Three-pass FFT geometry N = N2 * N1 * N0 (passes in that order, strides N0*N1, N0, 1).
// The last pass (radix N0) is contiguous; its output sits at the digit-reversed position
// p = k2 + N0 k1 + N0 N1 k0 of frequency k = k0 + N2 k1 + N2 N1 k2.
// Shared memory (bytes): the block with both polarizations interleaved, one float4
// (x_pol0, x_pol1) per position plus one float4 of padding per N0 positions; the step's
// H table; the split first-pass twiddles W_N^{c k} = A[c mod 16][k] * B[c div 16][k];
// the second-pass twiddles; the current step's filter taps.  The ESSFM intensity P and
// phase theta arrays reuse the
// block buffer while the block is held in registers.
template <int N>
struct Geo {
    static constexpr int N0 = (N >= 8192) ? 32 : 16;
    static constexpr int N1 = (N <= 512) ? 8 : 16;
    static constexpr int N2 = N / (N0 * N1);
    static constexpr int T = N / 16;                 // threads per CTA
    static constexpr int S1 = N0 * N1;               // stride of the first pass
    static constexpr int PADX = N + N / N0;          // float4 slots of the block buffer
    static constexpr int PADP = N + 4 * (N / 16);    // floats of P / theta (+16 B per 16)
    static constexpr int PADH = N + 2 * (N / N0);    // float2 of the H table (+16 B per N0)
    // P with circular copies of HALO samples on each side (forward filter), then theta
    static constexpr int HALO = ((8 * ((DBP_MAX_TAPS + 7) / 8) + 15) / 16) * 16;
    static constexpr int PADPH = (N + 2 * HALO) + 4 * ((N + 2 * HALO) / 16);
    static constexpr int TWA = 16 * N2;
    static constexpr int TWB = (S1 / 16) * N2;
    static constexpr int TW2 = N0 * N1;
    static constexpr size_t OFF_H = (size_t)PADX * 16;
    static constexpr size_t OFF_TWA = OFF_H + (size_t)PADH * 8;
    static constexpr size_t OFF_TWB = OFF_TWA + (size_t)TWA * 8;
    static constexpr size_t OFF_TW2 = OFF_TWB + (size_t)TWB * 8;
    static constexpr size_t OFF_TAPS = OFF_TW2 + (size_t)TW2 * 8;
    static constexpr int TAPS_MAX = 1 + DBP_MAX_TAPS + 15;   // one step's taps, 8-padded
    static constexpr size_t SMEM = OFF_TAPS + (size_t)TAPS_MAX * 4;
    static constexpr int MINB = (512 / T) > 0 ? (512 / T) : 1;
    static_assert(2 * PADP * 4 <= PADX * 16, "P/theta must fit in the block buffer");
    static_assert((PADPH + PADP) * 4 <= PADX * 16 && HALO <= N, "haloed P/theta must fit in the block buffer");
    static_assert(N0 * N1 >= HALO, "the halo copies come from the first and last pass-1 rows");
    static_assert(SMEM <= 227 * 1024, "shared memory budget");
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
    const float2 *twA;      // [N2][16] W_N^{cl k}
    const float2 *twB;      // [N2][N0 N1 / 16] W_{N/16}^{ch k}
    const float2 *tw2;      // [N1][N0] W_{N0 N1}^{n0 k1}
    int prefetch_ahead;     // nonzero: each CTA prefetches into L2 the input window of the block it
                            // runs next, one wave of the persistent grid ahead (0: off)
    int linear_only;        // 1: skip the nonlinear sub-step (FFE)
    int single_pol;         // 1: one-polarization waveforms [n], two blocks per CTA
    int bulk_store;         // 1: outputs staged in shared memory, written by bulk copies
                            //    (out 16-byte aligned and n even; ESSFM kernels)
    int fast_exp;           // 1: hardware exponential (ESSFM plans of at most two steps)
};

// One job of a batched launch: a plan's parameters with its own input/output buffers.
struct BatchJob {
    FwdParams p;
    long long item0;        // first item of this job within its block-length group
    int essfm;
    int pad;
    const int *ready;       // publish flag (non-zero: input is in place)
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
    int prefetch_ahead = 1;   // L2 prefetch of the next block's window (0: off)
    int precision = DBP_FP32;
    int scheme = DBP_SCHEME_FUSED;
    int user_overlap = 0;
    void *d_pp = nullptr;     // per-step scheme: intermediate waveform buffer
    size_t pp_bytes = 0;
    int dft_block = 0;
    float2 *d_Hn = nullptr;   // split precisions: H_s / N in natural frequency order
    float2 *d_Wn = nullptr;   // split precisions: W_N^m
    uint32_t *d_F = nullptr;  // split precisions: DFT-matrix hi/lo tables
    uint4 *d_Fu = nullptr;    // split precisions, N_a = 64: the same in the tcgen05 operand layout
    int *d_err = nullptr;     // split precisions: bounded-wait status of the tensor-core kernel
    int device;
    // device tables
    float2 *d_H = nullptr;
    float *d_taps = nullptr;
    float2 *d_twA = nullptr;
    float2 *d_twB = nullptr;
    float2 *d_tw2 = nullptr;
    // host copies
    double *step_dz = nullptr;
    double *step_geff = nullptr;
    float *coeffs = nullptr;        // [n_steps][n_taps + 1] unscaled c_{s,i}
    // adjoint: device copies of c and gamma_eff, and scratch (allocated on first dbp_grad)
    float *d_craw = nullptr;
    double *d_geff = nullptr;
    void *d_adj = nullptr;
    size_t adj_bytes = 0;
    // host-staging scratch for dbp_run_host
    void *d_stage_in = nullptr;
    void *d_stage_out = nullptr;
    size_t stage_bytes = 0;
    cudaStream_t aux[3] = {nullptr, nullptr, nullptr};
    cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
};

// Planner pieces shared by the entry points (plan.cu).
int describe(const dbp_link *link, const dbp_signal *sig, const dbp_steps *st, dbp_plan_info *info, double *dz,
             double *geff);
bool overlaps(const void *a, const void *b, size_t bytes);
int launch(const PlanImpl &P, const void *in, void *out, int n_wave, cudaStream_t st);
__global__ void build_h_kernel(float2 *H, int N, int n0, int n1, int n2, double beta2, double fs, const double *dz,
                               int n_tables);
__global__ void build_twiddle_kernel(float2 *twA, float2 *twB, float2 *tw2, int N, int n0, int n1, int n2);

struct AdjParams;
struct GemmParams;
int launch_gemm_bf16(const GemmParams &, int N, int NA, int n_wave, bool essfm, cudaStream_t);
int launch_gemm_fp16(const GemmParams &, int N, int NA, int n_wave, bool essfm, cudaStream_t);
int build_f_tables_bf16(uint32_t *F, int NA);
int build_f_tables_fp16(uint32_t *F, int NA);
int launch_gemm_plan(const PlanImpl &P, const void *in, void *out, int n_wave, cudaStream_t st);
bool umma_supported(int N, int NA);
int build_fu_tables(uint4 *Fu, int precision);
int launch_umma(const GemmParams &q, const uint4 *Fu, int *err, int precision, int N, int n_wave, bool essfm,
                cudaStream_t st, bool *used);
int build_gemm_tables(PlanImpl &P);
int launch_adj_512(const AdjParams &, int n_wave, bool essfm, cudaStream_t);
int launch_adj_1024(const AdjParams &, int n_wave, bool essfm, cudaStream_t);
int launch_adj_2048(const AdjParams &, int n_wave, bool essfm, cudaStream_t);
int launch_adj_4096(const AdjParams &, int n_wave, bool essfm, cudaStream_t);
int launch_adj_8192(const AdjParams &, int n_wave, bool essfm, cudaStream_t);
int upload_taps(PlanImpl &P, const float *host_coeffs);
int dev_alloc(void **p, size_t bytes);
int build_h_tables(PlanImpl &P);
void fill_fwd_params(const PlanImpl &P, FwdParams &p);

// Uneven batches: one persistent kernel over work units of every block length (batch_kernel.cu).
struct BatchGroupDev {
    const BatchJob *jobs;   // the group's jobs, item0 ascending
    int n_jobs;
    int N;                  // block length of the group
};
struct BatchUnit {
    long long item0;        // first item (job, waveform, block) of the unit within its group
    int group;
    int count;              // items in the unit: at most batch_unit_blocks(N)
};
int batch_unit_blocks(int N);
int prepare_batch_unified(int *grid);
int launch_batch_unified(const BatchGroupDev *groups, const BatchUnit *units, long long n_units,
                         unsigned long long *counter, int *error, int max_spins, int grid, cudaStream_t st);

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
