// Building blocks of the fused DBP kernels: one CTA holds one overlap-save block of N
// vector samples (both polarizations) and moves it through the steps of Section II.
//
// FFT (operations (i) and (iii) of Section II) in three passes, N = N2 * N1 * N0:
//   pass 1  radix-N2 DFT over the top digit (stride N0 N1), twiddle W_N^{c k0}
//   pass 2  radix-N1 DFT (stride N0), twiddle W_{N0 N1}^{n0 k1}
//   pass 3  radix-N0 DFT (contiguous); the spectrum is then at digit-reversed positions
// The inverse FFT runs the passes backwards with conjugate twiddles.  Pass 3 takes a
// "mid" operation that works on the spectrum in registers between the forward and the
// inverse radix-N0 DFTs (x H_s for the linear sub-step, Eq. 1; x conj(H_s) and the
// step-length gradient for the adjoint).  Between passes the block lives in shared
// memory, both polarizations as one float4 per position; before pass 1 and after pass
// 1' it lives in registers in the pass-1 layout, where thread t owns positions
// (t + T i) + S1 j.
#pragma once
#include "dbp_internal.cuh"
#include "dft_regs.cuh"

namespace dbp {

template <int N0>
__device__ __forceinline__ int xphys(int e) { return e + e / N0; }           // float4 slots
template <int N0>
__device__ __forceinline__ int hphys(int e) { return e + 2 * (e / N0); }     // float2 slots
__device__ __forceinline__ int pphys(int e) { return e + 4 * (e >> 4); }     // float slots

__device__ __forceinline__ void cp_async16(void *smem, const void *gmem) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

// Bulk (TMA-unit) copies: shared -> global stores tracked per issuing thread with bulk
// groups, and L2 prefetches of a contiguous global range.  Addresses 16-byte aligned,
// sizes multiples of 16 bytes.
__device__ __forceinline__ void fence_proxy_async_smem() { asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory"); }
__device__ __forceinline__ void bulk_store(void *gdst, const void *ssrc, unsigned bytes) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(ssrc);
    asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;\n" ::"l"(gdst), "r"(s), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_read_all() { asm volatile("cp.async.bulk.wait_group.read 0;\n" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;\n" ::: "memory"); }
__device__ __forceinline__ void bulk_prefetch_l2(const void *g, unsigned bytes) {
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;\n" ::"l"(g), "r"(bytes) : "memory");
}

// Tensor memory (TMEM) used as per-thread storage: tcgen05.alloc by one warp (the address
// goes to shared memory), 32-bit columns of the thread's lane read and written with the
// 32x32b shapes.  A warp reaches only the 32 lanes of its quarter of the warpgroup
// (lanes 32 (warp % 4) ...); the lane goes in the address's upper 16 bits.
__device__ __forceinline__ void tmem_alloc(uint32_t *smem_dst, uint32_t ncols) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem_dst);
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(s), "r"(ncols) : "memory");
}
__device__ __forceinline__ void tmem_relinquish() {
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void tmem_fence_before_sync() { asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory"); }
__device__ __forceinline__ void tmem_fence_after_sync() { asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory"); }
// r[0..31] -> columns taddr .. taddr + 31 of this thread's lane; returns when written
__device__ __forceinline__ void tmem_st32(uint32_t taddr, const uint32_t (&r)[32]) {
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, "
        "%14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31, %32};\n" ::"r"(taddr),
        "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]), "r"(r[8]), "r"(r[9]),
        "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]), "r"(r[15]), "r"(r[16]), "r"(r[17]), "r"(r[18]),
        "r"(r[19]), "r"(r[20]), "r"(r[21]), "r"(r[22]), "r"(r[23]), "r"(r[24]), "r"(r[25]), "r"(r[26]), "r"(r[27]),
        "r"(r[28]), "r"(r[29]), "r"(r[30]), "r"(r[31])
        : "memory");
    asm volatile("tcgen05.wait::st.sync.aligned;\n" ::: "memory");
}
// columns taddr .. taddr + 7 of this thread's lane -> r[0..7]; the wait takes the
// registers as operands so that no use is scheduled before the data has arrived
__device__ __forceinline__ void tmem_ld8(uint32_t taddr, uint32_t (&r)[8]) {
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];\n"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
                 : "r"(taddr)
                 : "memory");
    asm volatile("tcgen05.wait::ld.sync.aligned;\n"
                 : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]), "+r"(r[7])
                 :
                 : "memory");
}

// exp(+j theta) for the nonlinear rotation.
// Accurate (default): theta = q pi/2 + r with a three-constant Cody-Waite reduction
// (pi/2 = 1.5703125 + 4.837512969970703e-4 + 7.549790126404332e-8; the first two
// constants have 12 significant bits, so q times each is exact for |q| < 2^12, i.e.
// |theta| < 6400 rad), then Taylor polynomials of sin and cos on |r| <= pi/4
// (truncation below 2e-9, under half an FP32 ulp), and the quadrant q mod 4
// selects/negates.  Absolute error about 7e-8.
// FAST: reduction by 2 pi (6.28125 + 1.9353071795864769e-3, the first with 9
// significant bits) to [-pi, pi] and the hardware sine/cosine approximations, absolute
// error below 4e-7 there.  The error adds up over the steps of a plan, so the forward
// kernels take it only for plans of at most two steps (at most 8e-7 of phase, against
// a parity bar of 1e-5 relative).
template <bool FAST = false>
__device__ __forceinline__ float2 expj(float th) {
    if constexpr (FAST) {
        const float k = rintf(th * 0.15915494309189535f);
        float r = fmaf(-k, 6.28125f, th);
        r = fmaf(-k, 1.9353071795864769e-3f, r);
        float s, c;
        __sincosf(r, &s, &c);
        return make_float2(c, s);
    } else {
        const float q = rintf(th * 0.63661977236758134f);
        float r = fmaf(-q, 1.5703125f, th);
        r = fmaf(-q, 4.837512969970703e-4f, r);
        r = fmaf(-q, 7.549790126404332e-8f, r);
        const float r2 = r * r;
        // sin r = r - r^3/3! + r^5/5! - r^7/7! + r^9/9!
        float ps = fmaf(r2, 2.7557319223985893e-6f, -1.9841269841269841e-4f);
        ps = fmaf(r2, ps, 8.3333333333333333e-3f);
        ps = fmaf(r2, ps, -1.6666666666666667e-1f);
        const float sn = fmaf(r * r2, ps, r);
        // cos r = 1 - r^2/2! + r^4/4! - r^6/6! + r^8/8! - r^10/10!
        float pc = fmaf(r2, -2.7557319223985891e-7f, 2.4801587301587302e-5f);
        pc = fmaf(r2, pc, -1.3888888888888889e-3f);
        pc = fmaf(r2, pc, 4.1666666666666667e-2f);
        pc = fmaf(r2, pc, -0.5f);
        const float cs = fmaf(r2, pc, 1.0f);
        const int quad = ((int)q) & 3;
        const float c1 = (quad & 1) ? sn : cs;
        const float s1 = (quad & 1) ? cs : sn;
        return make_float2((quad == 1 || quad == 2) ? -c1 : c1, (quad >= 2) ? -s1 : s1);
    }
}

// TF32 helpers for the tensor-core filter: x = hi + lo with both parts TF32-rounded
// (about 22 significant bits together).
__device__ __forceinline__ uint32_t tf32_rna(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ void split_tf32(float x, uint32_t &hi, uint32_t &lo) {
    hi = tf32_rna(x);
    lo = tf32_rna(x - __uint_as_float(hi));
}
__device__ __forceinline__ void mma_tf32(float (&c)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

__device__ __forceinline__ float joint_intensity(float2 y0, float2 y1) {
    return fmaf(y0.x, y0.x, fmaf(y0.y, y0.y, fmaf(y1.x, y1.x, y1.y * y1.y)));
}

// GRP: the block is handled by a sub-group of N / 16 threads of a larger CTA (several
// blocks side by side, each with its own shared-memory slice), synchronised with the
// named barrier bar_id; otherwise by the whole CTA with __syncthreads.
template <int N>
__device__ __noinline__ void fir16_one_copy(int t, const float *src, float *dst, const float *a, int n_tapblk);

template <int N, bool GRP = false>
struct Blk {
    using G = Geo<N>;
    static constexpr int N0 = G::N0, N1 = G::N1, N2 = G::N2, T = G::T, S1 = G::S1;
    static constexpr int C1 = 16 / N2;    // pass-1 columns per thread (both polarizations)
    static constexpr int C2 = 16 / N1;    // pass-2 columns per thread (both polarizations)
    using Regs = float2[2][C1][N2];

    float4 *xs;
    float2 *sH;
    float2 *sA;
    float2 *sB;
    float2 *s2;
    float *sa;     // current step's taps gamma_eff c_i (shared, broadcast reads)
    int t;
    uint32_t twt = 0;   // TMEM address of this thread's pass-1 twiddles (twiddles_to_tmem)
    int bar_id = 0;     // GRP: named barrier of the sub-group (1 .. 15)

    // barrier over the threads that handle this block
    __device__ __forceinline__ void sync() const {
        if constexpr (GRP)
            asm volatile("bar.sync %0, %1;\n" ::"r"(bar_id), "n"(G::T) : "memory");
        else
            __syncthreads();
    }

    __device__ __forceinline__ Blk(unsigned char *smem, int tid)
        : xs(reinterpret_cast<float4 *>(smem)),
          sH(reinterpret_cast<float2 *>(smem + G::OFF_H)),
          sA(reinterpret_cast<float2 *>(smem + G::OFF_TWA)),
          sB(reinterpret_cast<float2 *>(smem + G::OFF_TWB)),
          s2(reinterpret_cast<float2 *>(smem + G::OFF_TW2)),
          sa(reinterpret_cast<float *>(smem + G::OFF_TAPS)),
          t(tid) {}

    // Stages one step's taps (n floats) in shared memory; visible after the next barrier.
    __device__ __forceinline__ void stage_taps(const float *__restrict__ a, int n) {
        for (int i = t; i < n; i += T) sa[i] = __ldg(a + i);
    }

    // float views of the block buffer for the nonlinear sub-step (valid while the block
    // is in registers): k = 0 joint intensity, 1 phase, 2 (adjoint) phase gradient.
    __device__ __forceinline__ float *farr(int k) const { return reinterpret_cast<float *>(xs) + k * G::PADP; }
    // The forward kernels' layout instead: P at logical positions [-HALO, N + HALO)
    // (pphys(e + HALO)), the positions outside [0, N) holding circular copies, then theta.
    __device__ __forceinline__ float *phalo() const { return reinterpret_cast<float *>(xs); }
    __device__ __forceinline__ float *tharr() const { return reinterpret_cast<float *>(xs) + G::PADPH; }

    __device__ __forceinline__ int pos1(int i, int j) const { return (t + T * i) + S1 * j; }

    // Twiddle tables (k-major: twA [N2][16], twB [N2][N0 N1/16], tw2 [N1][N0]).
    __device__ __forceinline__ void load_tables(const float2 *twA, const float2 *twB, const float2 *tw2) {
        for (int i = t; i < G::TWA; i += T) sA[i] = __ldg(twA + i);
        for (int i = t; i < G::TWB; i += T) sB[i] = __ldg(twB + i);
        for (int i = t; i < G::TW2; i += T) s2[i] = __ldg(tw2 + i);
    }

    // Copies one step's H table (N float2, 16-byte chunks) into padded shared memory.
    // Warp w copies positions [512 w, 512 w + 512): exactly the ones its own threads read
    // in pass 3 (16 positions a thread at N0 = 16; one polarization of 32 at N0 = 32), so
    // a warp's own copies and a __syncwarp make them visible where pass 3 needs them.
    __device__ __forceinline__ void prefetch_h(const float2 *__restrict__ H) {
        static_assert(T % 32 == 0 && N == 512 * (T / 32), "512 positions per warp");
        const int e0 = 512 * (t >> 5) + 2 * (t & 31);
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const int e = e0 + 64 * q;
            cp_async16(sH + hphys<N0>(e), H + e);
        }
        cp_async_commit();
    }

    // Block window [win0, win0 + N) of both polarizations of a waveform (pol-major
    // [2][n] complex64) into the pass-1 layout; periodic or zero outside [0, n).
    // SINGLE: a one-polarization waveform [n], lane l holding the window of the block
    // `shift` samples later, [win0 + l shift, win0 + l shift + N).
    template <bool SINGLE = false>
    __device__ __forceinline__ void load_window(Regs &v, const float2 *__restrict__ in, long long n, long long win0,
                                                int boundary, int shift = 0) const {
        if (win0 >= 0 && win0 + (SINGLE ? shift : 0) + N <= n) {
#pragma unroll
            for (int pol = 0; pol < 2; ++pol) {
                const float2 *base = SINGLE ? in + win0 + (long long)pol * shift : in + pol * n + win0;
#pragma unroll
                for (int i = 0; i < C1; ++i)
#pragma unroll
                    for (int j = 0; j < N2; ++j) v[pol][i][j] = __ldg(base + pos1(i, j));
            }
        } else {
#pragma unroll
            for (int pol = 0; pol < 2; ++pol) {
                const float2 *base = SINGLE ? in : in + pol * n;
                const long long w0 = SINGLE ? win0 + (long long)pol * shift : win0;
#pragma unroll
                for (int i = 0; i < C1; ++i)
#pragma unroll
                    for (int j = 0; j < N2; ++j) {
                        long long idx = w0 + pos1(i, j);
                        float2 val = make_float2(0.f, 0.f);
                        if (boundary == DBP_PERIODIC) {
                            idx %= n;
                            if (idx < 0) idx += n;
                            val = __ldg(base + idx);
                        } else if (idx >= 0 && idx < n) {
                            val = __ldg(base + idx);
                        }
                        v[pol][i][j] = val;
                    }
            }
        }
    }

    // Prefetches a block window's 2 x N complex64 samples into L2, clamped to [0, n); a
    // hint only, for the block that will run on this SM next.  SINGLE: the N + shift
    // samples of a one-polarization block pair.
    // BULK: bulk prefetches of 16 KB pieces, one per thread among the first threads of
    // the CTA, each trimmed inward to 16-byte boundaries; otherwise one 128-byte line per
    // thread and instruction.
    template <bool SINGLE = false, bool BULK = false>
    __device__ __forceinline__ void prefetch_window_l2(const float2 *in, long long n, long long win0,
                                                       int shift = 0) const {
        const long long lo = win0 < 0 ? 0 : win0;
        const long long end = win0 + N + (SINGLE ? shift : 0);
        const long long hi = end > n ? n : end;
        if constexpr (BULK) {
            constexpr int CHUNK = 16384;
            constexpr int CH = (int)(((SINGLE ? 2 : 1) * (long long)N * 8 + CHUNK - 1) / CHUNK);   // pieces per row
            constexpr int NPOL = SINGLE ? 1 : 2;
            if (t >= NPOL * CH) return;
            const int pol = t / CH, c = t - pol * CH;
            const char *row = reinterpret_cast<const char *>(in + pol * n);
            unsigned long long a = reinterpret_cast<unsigned long long>(row + lo * 8) + (unsigned long long)c * CHUNK;
            unsigned long long z = reinterpret_cast<unsigned long long>(row + hi * 8);
            if (a + CHUNK < z) z = a + CHUNK;
            a = (a + 15) & ~15ull;
            z &= ~15ull;
            if (hi > lo && z > a) bulk_prefetch_l2(reinterpret_cast<const void *>(a), (unsigned)(z - a));
        } else {
            if (hi <= lo) return;
            const char *base0 = reinterpret_cast<const char *>(in + lo);
            const long long bytes = (hi - lo) * (long long)sizeof(float2);
            for (long long off = (long long)t * 128; off < bytes; off += (long long)T * 128) {
                asm volatile("prefetch.global.L2 [%0];" ::"l"(base0 + off));
                if (!SINGLE)
                    asm volatile("prefetch.global.L2 [%0];" ::"l"(base0 + off + n * (long long)sizeof(float2)));
            }
        }
    }

    // Inter-pass twiddles of a thread that owns one pass-1 column and one pass-2 column
    // (C1 = C2 = 1, N1 = N2 = 16): pass 1 W_N^{c k} and pass 2 W_{N0 N1}^{n0 k}, k = 1 .. 15,
    // computed once from the tables and kept in 64 TMEM columns of the thread's lane at twt
    // (pass 1 in columns 0-29, pass 2 in 32-61), so that each pass reads them with four
    // tcgen05.ld instead of table reads (and, for pass 1, a complex product) per k.
    static constexpr uint32_t TW_COLS = 64;
    __device__ __forceinline__ void twiddles_to_tmem() {
        static_assert(C1 == 1 && N2 == 16 && C2 == 1 && N1 == 16, "one column of 16 per thread in passes 1 and 2");
        const float2 *ta = sA + (t & 15);
        const float2 *tb = sB + (t >> 4);
        uint32_t r[32];
#pragma unroll
        for (int k = 1; k < 16; ++k) {
            const float2 wk = cmul(ta[16 * k], tb[(S1 / 16) * k]);
            r[2 * k - 2] = __float_as_uint(wk.x);
            r[2 * k - 1] = __float_as_uint(wk.y);
        }
        r[30] = r[31] = 0u;
        tmem_st32(twt, r);
        const float2 *tw = s2 + t % N0;
#pragma unroll
        for (int k = 1; k < 16; ++k) {
            const float2 wk = tw[N0 * k];
            r[2 * k - 2] = __float_as_uint(wk.x);
            r[2 * k - 1] = __float_as_uint(wk.y);
        }
        tmem_st32(twt + 32, r);
    }
    // u_k *= w_k (CONJ: conj(w_k)), k = 1 .. 15, with w from TMEM columns col ...
    template <bool CONJ>
    __device__ __forceinline__ void twiddle_tmem(float2 (&u0)[16], float2 (&u1)[16], uint32_t col = 0) const {
        twiddle_tmem_at<CONJ>(twt, u0, u1, col);
    }
    template <bool CONJ>
    static __device__ __forceinline__ void twiddle_tmem_at(uint32_t twt, float2 (&u0)[16], float2 (&u1)[16],
                                                           uint32_t col) {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            uint32_t r[8];
            tmem_ld8(twt + col + 8 * q, r);
#pragma unroll
            for (int m = 0; m < 4; ++m) {
                const int k = 4 * q + m + 1;
                if (k >= 16) break;
                const float2 wk = make_float2(__uint_as_float(r[2 * m]), __uint_as_float(r[2 * m + 1]));
                u0[k] = CONJ ? cmulc(u0[k], wk) : cmul(u0[k], wk);
                u1[k] = CONJ ? cmulc(u1[k], wk) : cmul(u1[k], wk);
            }
        }
    }

    // pass 1 (forward): DFT over the top digit, twiddle, registers -> shared memory.
    // TM: the twiddles come from TMEM (twiddles_to_tmem).
    template <bool TM = false>
    __device__ __forceinline__ void pass1_fwd(Regs &v) {
#pragma unroll
        for (int i = 0; i < C1; ++i) {
            const int c = t + T * i;
            const float2 *ta = sA + (c & 15);
            const float2 *tb = sB + (c >> 4);
            Dft<N2, false>::run(v[0][i]);
            Dft<N2, false>::run(v[1][i]);
            if constexpr (TM) {
                twiddle_tmem<false>(v[0][i], v[1][i]);
            } else {
#pragma unroll
                for (int k = 1; k < N2; ++k) {
                    const float2 wk = cmul(ta[16 * k], tb[(S1 / 16) * k]);
                    v[0][i][k] = cmul(v[0][i][k], wk);
                    v[1][i][k] = cmul(v[1][i][k], wk);
                }
            }
#pragma unroll
            for (int k = 0; k < N2; ++k)
                xs[xphys<N0>(c + S1 * k)] = make_float4(v[0][i][k].x, v[0][i][k].y, v[1][i][k].x, v[1][i][k].y);
        }
    }

    // pass 2: radix N1, stride N0 (forward: DFT then twiddle; inverse: conj twiddle then IDFT).
    // TM: the twiddles come from TMEM (twiddles_to_tmem).
    template <bool INV, bool TM = false>
    __device__ __forceinline__ void pass2() {
        pass2_at<INV, TM>(t, xs, s2, twt);
    }
    template <bool INV, bool TM>
    static __device__ __forceinline__ void pass2_at(int t, float4 *xs, const float2 *s2, uint32_t twt) {
#pragma unroll
        for (int i = 0; i < C2; ++i) {
            const int c2 = t + T * i;
            const int n0 = c2 % N0, k0 = c2 / N0;
            const int base = n0 + S1 * k0;
            float2 u0[N1], u1[N1];
#pragma unroll
            for (int j = 0; j < N1; ++j) {
                const float4 f = xs[xphys<N0>(base + N0 * j)];
                u0[j] = make_float2(f.x, f.y);
                u1[j] = make_float2(f.z, f.w);
            }
            const float2 *tw = s2 + n0;
            if constexpr (!INV) {
                Dft<N1, false>::run(u0);
                Dft<N1, false>::run(u1);
                if constexpr (TM) {
                    twiddle_tmem_at<false>(twt, u0, u1, 32);
                } else {
#pragma unroll
                    for (int k = 1; k < N1; ++k) {
                        const float2 wk = tw[N0 * k];
                        u0[k] = cmul(u0[k], wk);
                        u1[k] = cmul(u1[k], wk);
                    }
                }
            } else {
                if constexpr (TM) {
                    twiddle_tmem_at<true>(twt, u0, u1, 32);
                } else {
#pragma unroll
                    for (int k = 1; k < N1; ++k) {
                        const float2 wk = tw[N0 * k];
                        u0[k] = cmulc(u0[k], wk);
                        u1[k] = cmulc(u1[k], wk);
                    }
                }
                Dft<N1, true>::run(u0);
                Dft<N1, true>::run(u1);
            }
#pragma unroll
            for (int k = 0; k < N1; ++k)
                xs[xphys<N0>(base + N0 * k)] = make_float4(u0[k].x, u0[k].y, u1[k].x, u1[k].y);
        }
    }

    // pass 3: contiguous radix-N0 DFT, mid operation on the spectrum, inverse DFT.
    // N0 == 16: thread t owns positions 16t..16t+15 of both polarizations and calls
    //           mid(u0, u1, base);  N0 == 32: thread t owns polarization t & 1 of
    //           positions 32(t>>1).. and calls mid.one(u, pol, base).
    template <class Mid>
    __device__ __forceinline__ void pass3(Mid &mid) {
        pass3_at(t, xs, mid);
    }
    template <class Mid>
    static __device__ __forceinline__ void pass3_at(int t, float4 *xs, Mid &mid) {
        if constexpr (N0 == 16) {
            const int base = 16 * t;
            float2 u0[16], u1[16];
#pragma unroll
            for (int j = 0; j < 16; ++j) {
                const float4 f = xs[xphys<16>(base + j)];
                u0[j] = make_float2(f.x, f.y);
                u1[j] = make_float2(f.z, f.w);
            }
            Dft<16, false>::run(u0);
            Dft<16, false>::run(u1);
            mid.two(u0, u1, base);
            Dft<16, true>::run(u0);
            Dft<16, true>::run(u1);
#pragma unroll
            for (int j = 0; j < 16; ++j) xs[xphys<16>(base + j)] = make_float4(u0[j].x, u0[j].y, u1[j].x, u1[j].y);
        } else {
            const int pol = t & 1;
            const int base = N0 * (t >> 1);
            float2 *xh = reinterpret_cast<float2 *>(xs);
            float2 u[N0];
#pragma unroll
            for (int j = 0; j < N0; ++j) u[j] = xh[2 * xphys<N0>(base + j) + pol];
            Dft<N0, false>::run(u);
            mid.one(u, pol, base);
            Dft<N0, true>::run(u);
#pragma unroll
            for (int j = 0; j < N0; ++j) xh[2 * xphys<N0>(base + j) + pol] = u[j];
        }
    }

    // pass 1' (inverse): conjugate twiddle, inverse radix-N2 DFT, shared memory -> registers
    template <bool TM = false>
    __device__ __forceinline__ void pass1_inv(Regs &v) const {
#pragma unroll
        for (int i = 0; i < C1; ++i) {
            const int c = t + T * i;
            const float2 *ta = sA + (c & 15);
            const float2 *tb = sB + (c >> 4);
#pragma unroll
            for (int j = 0; j < N2; ++j) {
                const float4 f = xs[xphys<N0>(c + S1 * j)];
                v[0][i][j] = make_float2(f.x, f.y);
                v[1][i][j] = make_float2(f.z, f.w);
            }
            if constexpr (TM) {
                twiddle_tmem<true>(v[0][i], v[1][i]);
            } else {
#pragma unroll
                for (int k = 1; k < N2; ++k) {
                    const float2 wk = cmul(ta[16 * k], tb[(S1 / 16) * k]);
                    v[0][i][k] = cmulc(v[0][i][k], wk);
                    v[1][i][k] = cmulc(v[1][i][k], wk);
                }
            }
            Dft<N2, true>::run(v[0][i]);
            Dft<N2, true>::run(v[1][i]);
        }
    }

    // Symmetric filter over 16 consecutive positions 16t..16t+15 (circular in the block):
    // out_k = a_0 src_k + sum_{i=1}^{8 n_tapblk} a_i (src_{k-i} + src_{k+i}), read from
    // the float array src and written to dst (both pphys-indexed).  Eq. 3 when src = P.
    __device__ __forceinline__ void fir16(const float *src, float *dst, const float *a, int n_tapblk) const {
        fir16_at(t, src, dst, a, n_tapblk);
    }
    static __device__ __forceinline__ void fir16_at(int t, const float *src, float *dst, const float *a,
                                                    int n_tapblk) {
        const int k0 = 16 * t;
        float th[16];
        {
            const float4 *pc = reinterpret_cast<const float4 *>(src + pphys(k0));
            const float a0 = a[0];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const float4 f = pc[q];
                th[4 * q + 0] = a0 * f.x;
                th[4 * q + 1] = a0 * f.y;
                th[4 * q + 2] = a0 * f.z;
                th[4 * q + 3] = a0 * f.w;
            }
        }
        for (int blk = 0; blk < n_tapblk; ++blk) {
            const int i0 = 8 * blk;
            float lw[24], rw[24];
#pragma unroll
            for (int q = 0; q < 6; ++q) {
                const int el = (k0 - i0 - 8 + 4 * q) & (N - 1);
                const int er = (k0 + i0 + 4 * q) & (N - 1);
                const float4 fl = *reinterpret_cast<const float4 *>(src + pphys(el));
                const float4 fr = *reinterpret_cast<const float4 *>(src + pphys(er));
                lw[4 * q + 0] = fl.x; lw[4 * q + 1] = fl.y; lw[4 * q + 2] = fl.z; lw[4 * q + 3] = fl.w;
                rw[4 * q + 0] = fr.x; rw[4 * q + 1] = fr.y; rw[4 * q + 2] = fr.z; rw[4 * q + 3] = fr.w;
            }
#pragma unroll
            for (int ii = 1; ii <= 8; ++ii) {
                const float ai = a[i0 + ii];
#pragma unroll
                for (int r = 0; r < 16; ++r) th[r] = fmaf(ai, lw[r - ii + 8] + rw[r + ii], th[r]);
            }
        }
        float4 *pt = reinterpret_cast<float4 *>(dst + pphys(k0));
#pragma unroll
        for (int q = 0; q < 4; ++q) pt[q] = make_float4(th[4 * q], th[4 * q + 1], th[4 * q + 2], th[4 * q + 3]);
    }

    // fir16 reading P from the haloed layout (phalo), so that no window index wraps.  With
    // k0 = 16 t and k0 + HALO a multiple of 16, a window starting at logical k0 + 16 a + 8 b
    // (b = 0 or 1) has its six float4 at 20 a + 8 b + {0, 4, 8 + 4 b, 12 + 4 b, 20, 24}
    // floats after the thread's own first position (the layout pads 4 floats per 16).
    __device__ __forceinline__ void fir16h(const float *srch, float *dst, const float *a, int n_tapblk) const {
        const int k0 = 16 * t;
        const float *pc = srch + pphys(k0 + G::HALO);
        float th[16];
        {
            const float a0 = a[0];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const float4 f = reinterpret_cast<const float4 *>(pc)[q];
                th[4 * q + 0] = a0 * f.x;
                th[4 * q + 1] = a0 * f.y;
                th[4 * q + 2] = a0 * f.z;
                th[4 * q + 3] = a0 * f.w;
            }
        }
        for (int blk = 0; blk < n_tapblk; ++blk) {
            // tap block blk: left window from k0 - 8 (blk + 1), right window from k0 + 8 blk
            const int bl = (blk + 1) & 1, br = blk & 1;
            const float *pl = pc + (8 * bl - 20 * ((blk + 2) >> 1));
            const float *pr = pc + (8 * br + 20 * (blk >> 1));
            float lw[24], rw[24];
#pragma unroll
            for (int q = 0; q < 6; ++q) {
                const int ol = q < 2 ? 4 * q : (q < 4 ? 4 * q + 4 * bl : 4 * q + 4);
                const int orr = q < 2 ? 4 * q : (q < 4 ? 4 * q + 4 * br : 4 * q + 4);
                const float4 fl = *reinterpret_cast<const float4 *>(pl + ol);
                const float4 fr = *reinterpret_cast<const float4 *>(pr + orr);
                lw[4 * q + 0] = fl.x; lw[4 * q + 1] = fl.y; lw[4 * q + 2] = fl.z; lw[4 * q + 3] = fl.w;
                rw[4 * q + 0] = fr.x; rw[4 * q + 1] = fr.y; rw[4 * q + 2] = fr.z; rw[4 * q + 3] = fr.w;
            }
            const float *ab = a + 8 * blk;
#pragma unroll
            for (int ii = 1; ii <= 8; ++ii) {
                const float ai = ab[ii];
#pragma unroll
                for (int r = 0; r < 16; ++r) th[r] = fmaf(ai, lw[r - ii + 8] + rw[r + ii], th[r]);
            }
        }
        float4 *pt = reinterpret_cast<float4 *>(dst + pphys(k0));
#pragma unroll
        for (int q = 0; q < 4; ++q) pt[q] = make_float4(th[4 * q], th[4 * q + 1], th[4 * q + 2], th[4 * q + 3]);
    }

    // fir16h with the tap blocks in pairs: the float at logical k0 + x sits x + 4 floor(x / 16)
    // floats after the one at k0, and the windows of tap block 2m + b are those of tap
    // block b moved by 16 m positions (20 m floats), so every offset inside a pair is a
    // constant.  Measured faster than fir16h in the N = 8192 kernels (one CTA per SM) and
    // slower in the shorter blocks' kernels (several CTAs per SM; by 8-10 % at N_c = 16,
    // where the loop body of twice the length runs once per block).
    static __host__ __device__ constexpr int hoff(int x) { return x + 4 * (x >= 0 ? x / 16 : -((15 - x) / 16)); }
    template <int PAR>
    __device__ __forceinline__ void fir16h_block(const float *pl, const float *pr, const float *a, float (&th)[16]) const {
        float lw[24], rw[24];
#pragma unroll
        for (int q = 0; q < 6; ++q) {
            const float4 fl = *reinterpret_cast<const float4 *>(pl + hoff(4 * q - 8 - 8 * PAR));
            const float4 fr = *reinterpret_cast<const float4 *>(pr + hoff(4 * q + 8 * PAR));
            lw[4 * q + 0] = fl.x; lw[4 * q + 1] = fl.y; lw[4 * q + 2] = fl.z; lw[4 * q + 3] = fl.w;
            rw[4 * q + 0] = fr.x; rw[4 * q + 1] = fr.y; rw[4 * q + 2] = fr.z; rw[4 * q + 3] = fr.w;
        }
#pragma unroll
        for (int ii = 1; ii <= 8; ++ii) {
            const float ai = a[ii];
#pragma unroll
            for (int r = 0; r < 16; ++r) th[r] = fmaf(ai, lw[r - ii + 8] + rw[r + ii], th[r]);
        }
    }
    __device__ __forceinline__ void fir16h_pairs(const float *srch, float *dst, const float *a, int n_tapblk) const {
        const int k0 = 16 * t;
        const float *pc = srch + pphys(k0 + G::HALO);
        float th[16];
        {
            const float a0 = a[0];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const float4 f = reinterpret_cast<const float4 *>(pc)[q];
                th[4 * q + 0] = a0 * f.x;
                th[4 * q + 1] = a0 * f.y;
                th[4 * q + 2] = a0 * f.z;
                th[4 * q + 3] = a0 * f.w;
            }
        }
        for (int m = 0; 2 * m < n_tapblk; ++m) {
            fir16h_block<0>(pc - 20 * m, pc + 20 * m, a + 16 * m, th);
            if (2 * m + 1 < n_tapblk) fir16h_block<1>(pc - 20 * m, pc + 20 * m, a + 16 * m + 8, th);
        }
        float4 *pt = reinterpret_cast<float4 *>(dst + pphys(k0));
#pragma unroll
        for (int q = 0; q < 4; ++q) pt[q] = make_float4(th[4 * q], th[4 * q + 1], th[4 * q + 2], th[4 * q + 3]);
    }

    // The same filter on the tensor cores, for all N positions of the block: with
    // NCP = 8 n_tapblk taps a side, output group q (positions 16q..16q+15) is
    //   theta[16q + r] = sum_u W[q][u] B[u][r],  W[q][u] = src[16q - NCP + u] (circular),
    //   B[u][r] = a_|u - NCP - r| inside the band |u - NCP - r| <= NCP, else 0,
    // a (groups x (16 + 2 NCP)) by ((16 + 2 NCP) x 16) matrix product computed with
    // mma.sync m16n8k8 in TF32 with both operands split hi + lo (three products,
    // FP32 accumulation, ~2^-21 relative per term).  Each warp owns two tiles of 16
    // groups; the B fragments are formed from the taps and shared by both tiles.
    // Selected with DBP_FIR_TC; on GB300 the register FMA filter (fir16) measured faster
    // inside the fused kernel (3200 km ESSFM-1, N_c = 32: 49.7 vs 41.6 G samples/s).
    __device__ __forceinline__ void fir_tc(const float *src, float *dst, const float *a, int n_tapblk) const {
        const int lane = t & 31, warp = t >> 5, g = lane >> 2, tq = lane & 3;
        const int ncp = 8 * n_tapblk;
        const int ksteps = 2 + 2 * n_tapblk;            // (16 + 2 NCP) / 8
        float c[2][2][4];
#pragma unroll
        for (int i = 0; i < 2; ++i)
#pragma unroll
            for (int j = 0; j < 2; ++j)
#pragma unroll
                for (int k = 0; k < 4; ++k) c[i][j][k] = 0.f;
        for (int ks = 0; ks < ksteps; ++ks) {
            uint32_t bh[2][2], bl[2][2];
#pragma unroll
            for (int nt = 0; nt < 2; ++nt)
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int d = 8 * ks + tq + 4 * h - ncp - (8 * nt + g);
                    const int ad = d < 0 ? -d : d;
                    const float coef = ad <= ncp ? a[ad] : 0.f;
                    split_tf32(coef, bh[nt][h], bl[nt][h]);
                }
#pragma unroll
            for (int tile = 0; tile < 2; ++tile) {
                const int q0 = (2 * warp + tile) * 16 + g;
                const int e0 = 16 * q0 - ncp + 8 * ks + tq;
                const float w0 = src[pphys(e0 & (N - 1))];
                const float w1 = src[pphys((e0 + 128) & (N - 1))];
                const float w2 = src[pphys((e0 + 4) & (N - 1))];
                const float w3 = src[pphys((e0 + 132) & (N - 1))];
                uint32_t ah[4], al[4];
                split_tf32(w0, ah[0], al[0]);
                split_tf32(w1, ah[1], al[1]);
                split_tf32(w2, ah[2], al[2]);
                split_tf32(w3, ah[3], al[3]);
#pragma unroll
                for (int nt = 0; nt < 2; ++nt) {
                    mma_tf32(c[tile][nt], ah, bh[nt][0], bh[nt][1]);
                    mma_tf32(c[tile][nt], ah, bl[nt][0], bl[nt][1]);
                    mma_tf32(c[tile][nt], al, bh[nt][0], bh[nt][1]);
                }
            }
        }
#pragma unroll
        for (int tile = 0; tile < 2; ++tile)
#pragma unroll
            for (int nt = 0; nt < 2; ++nt) {
                const int q0 = (2 * warp + tile) * 16 + g;
                const int r = 8 * nt + 2 * tq;
                *reinterpret_cast<float2 *>(dst + pphys(16 * q0 + r)) = make_float2(c[tile][nt][0], c[tile][nt][1]);
                *reinterpret_cast<float2 *>(dst + pphys(16 * (q0 + 8) + r)) =
                    make_float2(c[tile][nt][2], c[tile][nt][3]);
            }
    }

    // ESSFM phase theta (Eq. 3) of the block in registers, for the forward kernels: P into
    // the haloed layout (positions within HALO of either end written twice), the filter by
    // fir16h / fir16h_pairs, theta into tharr().  The block buffer must be free (a barrier
    // after the last pass-1' read); returns after a barrier, with theta visible to all
    // threads.  LANE < 0: P is the joint intensity of the two polarizations; LANE = 0 or
    // 1: P = |y|^2 of that lane alone (one-polarization blocks, the scalar form that
    // Eq. 3 extends).
    template <int LANE = -1>
    __device__ __forceinline__ void essfm_theta_fwd(const Regs &v, const float *a, int n_tapblk) {
        float *sP = phalo();
#pragma unroll
        for (int i = 0; i < C1; ++i)
#pragma unroll
            for (int j = 0; j < N2; ++j) {
                float pk;
                if constexpr (LANE < 0) {
                    pk = joint_intensity(v[0][i][j], v[1][i][j]);
                } else {
                    const float2 y = v[LANE][i][j];
                    pk = fmaf(y.x, y.x, y.y * y.y);
                }
                const int e = pos1(i, j);
                sP[pphys(e + G::HALO)] = pk;
                // e = t + T i + S1 j with S1 >= HALO: only j = 0 (and i = 0 when T >= HALO)
                // can fall in the first HALO positions, only the last j (and i) in the last
                if (j == 0 && (T < G::HALO || i == 0) && e < G::HALO) sP[pphys(e + N + G::HALO)] = pk;
                if (j == N2 - 1 && (T < G::HALO || i == C1 - 1) && e >= N - G::HALO)
                    sP[pphys(e - N + G::HALO)] = pk;
            }
        sync();
        if constexpr (N >= 8192)
            fir16h_pairs(sP, tharr(), a, n_tapblk);
        else
            fir16h(sP, tharr(), a, n_tapblk);
        sync();
    }

    // The same with P in farr(0) (no halo, the wrapping fir16) and theta into farr(1): the
    // adjoint's layout, which keeps a third array (the phase gradient) in the block buffer.
    // ONE_COPY: the filter through fir16_one_copy (one non-inlined copy of its code for
    // every call site of a kernel).
    template <int LANE = -1, bool ONE_COPY = false>
    __device__ __forceinline__ void essfm_theta(const Regs &v, const float *a, int n_tapblk) {
        float *sP = farr(0);
#pragma unroll
        for (int i = 0; i < C1; ++i)
#pragma unroll
            for (int j = 0; j < N2; ++j) {
                float pk;
                if constexpr (LANE < 0) {
                    pk = joint_intensity(v[0][i][j], v[1][i][j]);
                } else {
                    const float2 y = v[LANE][i][j];
                    pk = fmaf(y.x, y.x, y.y * y.y);
                }
                sP[pphys(pos1(i, j))] = pk;
            }
        sync();
#ifdef DBP_FIR_TC
        fir_tc(sP, farr(1), a, n_tapblk);
#else
        if constexpr (ONE_COPY)
            fir16_one_copy<N>(t, sP, farr(1), a, n_tapblk);
        else
            fir16(sP, farr(1), a, n_tapblk);
#endif
        sync();
    }
};

// Blk::fir16 as a called function: kernels that filter at several places (the adjoint:
// theta in the forward and reverse sweeps, then dL/dP) keep one copy of its code instead
// of one inlined copy per call site.  Arguments are pointers and integers only.
template <int N>
__device__ __noinline__ void fir16_one_copy(int t, const float *src, float *dst, const float *a, int n_tapblk) {
    Blk<N>::fir16_at(t, src, dst, a, n_tapblk);
}

// Blk::pass2 with the table twiddles as a called function, for the same reason: the
// adjoint runs pass 2 and its inverse in the forward sweep, the recomputed linear
// sub-step and the adjoint linear sub-step.  Shared memory in and out, no register
// arguments beyond pointers.
template <int N, bool INV>
__device__ __noinline__ void pass2_one_copy(int t, float4 *xs, const float2 *s2) {
    Blk<N>::template pass2_at<INV, false>(t, xs, s2, 0u);
}

// Multiplies the spectrum by the step's H table in shared memory (Eq. 1, inverted).
template <int N>
struct MidMulH {
    const float2 *sH;
    __device__ __forceinline__ void two(float2 (&u0)[16], float2 (&u1)[16], int base) {
        const float4 *hrow = reinterpret_cast<const float4 *>(sH + hphys<16>(base));
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const float4 h = hrow[j];
            u0[2 * j] = cmul(u0[2 * j], make_float2(h.x, h.y));
            u1[2 * j] = cmul(u1[2 * j], make_float2(h.x, h.y));
            u0[2 * j + 1] = cmul(u0[2 * j + 1], make_float2(h.z, h.w));
            u1[2 * j + 1] = cmul(u1[2 * j + 1], make_float2(h.z, h.w));
        }
    }
    template <int R>
    __device__ __forceinline__ void one(float2 (&u)[R], int, int base) {
        const float4 *hrow = reinterpret_cast<const float4 *>(sH + hphys<R>(base));
#pragma unroll
        for (int j = 0; j < R / 2; ++j) {
            const float4 h = hrow[j];
            u[2 * j] = cmul(u[2 * j], make_float2(h.x, h.y));
            u[2 * j + 1] = cmul(u[2 * j + 1], make_float2(h.z, h.w));
        }
    }
};

// Opt a kernel into more than 48 KB of dynamic shared memory, once per device.
template <typename K>
inline bool set_smem_once(K kernel, size_t bytes, unsigned long long &done_mask) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return false;
    const unsigned long long bit = 1ull << dev;
    if (done_mask & bit) return true;
    if (cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes) != cudaSuccess)
        return false;
    done_mask |= bit;
    return true;
}

}  // namespace dbp
