// In-register DFTs of length 2..32 for the shared-memory FFT passes.
//
// Convention: forward X_k = sum_n x_n exp(-j 2 pi n k / R); inverse uses +j and is
// unscaled.  Lengths above 4 are split Cooley-Tukey style, R = R1 * R2 with
// n = a + R1 b, k = kb + R2 ka:
//   X[kb + R2 ka] = sum_a W_R1^{a ka} W_R^{a kb} (sum_b x[a + R1 b] W_R2^{b kb}).
// All indices are compile-time, so the reordering costs no instructions.  Internal
// twiddles are compile-time constants; multiples of pi/4 use additions/swaps only.
#pragma once
#include <cuda_runtime.h>

#ifndef DBP_HD
#define DBP_HD __host__ __device__ __forceinline__
#endif

namespace dbp {

DBP_HD float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
DBP_HD float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
DBP_HD float2 cmul(float2 a, float2 b) {
    return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
// a * conj(b)
DBP_HD float2 cmulc(float2 a, float2 b) {
    return make_float2(fmaf(a.x, b.x, a.y * b.y), fmaf(a.y, b.x, -a.x * b.y));
}
// multiply by -j (forward) or +j (inverse)
template <bool INV>
DBP_HD float2 mul_mj(float2 a) {
    return INV ? make_float2(-a.y, a.x) : make_float2(a.y, -a.x);
}

// cos(2 pi m / 32) as a compile-time double (first-octant values written out).
__host__ __device__ constexpr double cos32(int m) {
    m = ((m % 32) + 32) % 32;
    if (m > 16) m = 32 - m;                // cos is even
    const bool neg = m > 8;
    if (neg) m = 16 - m;                   // cos(pi - x) = -cos x
    double c = 0.0;
    switch (m) {
        case 0: c = 1.0; break;
        case 1: c = 0.98078528040323044913; break;   // cos(pi/16)
        case 2: c = 0.92387953251128675613; break;   // cos(pi/8)
        case 3: c = 0.83146961230254523708; break;   // cos(3pi/16)
        case 4: c = 0.70710678118654752440; break;   // cos(pi/4)
        case 5: c = 0.55557023301960222474; break;   // cos(5pi/16)
        case 6: c = 0.38268343236508977173; break;   // cos(3pi/8)
        case 7: c = 0.19509032201612826785; break;   // cos(7pi/16)
        default: c = 0.0; break;
    }
    return neg ? -c : c;
}
__host__ __device__ constexpr double sin32(int m) { return cos32(8 - m); }

// v * W_R^M; forward W = exp(-j 2 pi / R), inverse exp(+j 2 pi / R); R divides 32.
template <int R, int M, bool INV>
DBP_HD float2 twid(float2 v) {
    constexpr int m32 = (((M * (32 / R)) % 32) + 32) % 32;   // angle in units of 2 pi / 32
    constexpr int mm = INV ? (32 - m32) % 32 : m32;           // multiply by exp(-j 2 pi mm / 32)
    constexpr float h = 0.70710678118654752440f;
    if constexpr (mm == 0) {
        return v;
    } else if constexpr (mm == 8) {
        return make_float2(v.y, -v.x);
    } else if constexpr (mm == 16) {
        return make_float2(-v.x, -v.y);
    } else if constexpr (mm == 24) {
        return make_float2(-v.y, v.x);
    } else if constexpr (mm == 4) {
        return make_float2((v.x + v.y) * h, (v.y - v.x) * h);
    } else if constexpr (mm == 12) {
        return make_float2((v.y - v.x) * h, -(v.x + v.y) * h);
    } else if constexpr (mm == 20) {
        return make_float2(-(v.x + v.y) * h, (v.x - v.y) * h);
    } else if constexpr (mm == 28) {
        return make_float2((v.x - v.y) * h, (v.x + v.y) * h);
    } else {
        constexpr float c = (float)cos32(mm);
        constexpr float s = (float)(-sin32(mm));
        return make_float2(fmaf(v.x, c, -v.y * s), fmaf(v.x, s, v.y * c));
    }
}

template <int R, bool INV>
struct Dft;

template <bool INV>
struct Dft<1, INV> {
    DBP_HD static void run(float2 *) {}
};

template <bool INV>
struct Dft<2, INV> {
    DBP_HD static void run(float2 *v) {
        float2 a = v[0], b = v[1];
        v[0] = cadd(a, b);
        v[1] = csub(a, b);
    }
};

template <bool INV>
struct Dft<4, INV> {
    DBP_HD static void run(float2 *v) {
        float2 t0 = cadd(v[0], v[2]), t1 = csub(v[0], v[2]);
        float2 t2 = cadd(v[1], v[3]), t3 = mul_mj<INV>(csub(v[1], v[3]));
        v[0] = cadd(t0, t2);
        v[2] = csub(t0, t2);
        v[1] = cadd(t1, t3);
        v[3] = csub(t1, t3);
    }
};

template <int R, bool INV>
struct Dft {
    static constexpr int R1 = (R >= 16) ? 4 : 2;
    static constexpr int R2 = R / R1;

    template <int I>
    DBP_HD static void apply_tw(float2 (&t)[R1][R2]) {
        if constexpr (I < R1 * R2) {
            constexpr int A = I / R2, KB = I % R2;
            t[A][KB] = twid<R, A * KB, INV>(t[A][KB]);
            apply_tw<I + 1>(t);
        }
    }

    DBP_HD static void run(float2 *v) {
        float2 t[R1][R2];
#pragma unroll
        for (int a = 0; a < R1; ++a) {
#pragma unroll
            for (int b = 0; b < R2; ++b) t[a][b] = v[a + R1 * b];
            Dft<R2, INV>::run(t[a]);
        }
        apply_tw<0>(t);
#pragma unroll
        for (int kb = 0; kb < R2; ++kb) {
            float2 u[R1];
#pragma unroll
            for (int a = 0; a < R1; ++a) u[a] = t[a][kb];
            Dft<R1, INV>::run(u);
#pragma unroll
            for (int ka = 0; ka < R1; ++ka) v[kb + R2 * ka] = u[ka];
        }
    }
};

}  // namespace dbp
