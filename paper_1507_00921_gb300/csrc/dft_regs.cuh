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

// One radix-4 column of a length-R DFT with the twiddles W_R^{a KB} (a = 0..3) folded
// into the butterfly (cosine-factored form): W^m = c_m (1 - j tan) forward (1 + j tan
// inverse), so input a is pre-rotated by (1 -/+ j tan) with two fused multiply-adds and
// its factor c_m rides along into the radix-4 additions, which become fused
// multiply-adds themselves: 22 floating-point operations for the column instead of 28.
// Used when none of the three twiddles is a multiple of -j (every c_m nonzero).
template <int R, int KB>
struct Col4 {
    static constexpr int m1 = KB % R, m2 = (2 * KB) % R, m3 = (3 * KB) % R;
    // cos / tan of 2 pi m / R as compile-time doubles via the 32-point table (R divides 32)
    __host__ __device__ static constexpr double cosm(int m) { return cos32(m * (32 / R)); }
    __host__ __device__ static constexpr double sinm(int m) { return sin32(m * (32 / R)); }
    static constexpr bool ok = KB != 0 && cosm(m1) != 0.0 && cosm(m2) != 0.0 && cosm(m3) != 0.0;
};

template <int R, int KB, bool INV>
DBP_HD void col4_factored(float2 (&u)[4]) {
    using C = Col4<R, KB>;
    constexpr double c1 = C::cosm(C::m1), c2 = C::cosm(C::m2), c3 = C::cosm(C::m3);
    // forward W^m = cos - j sin = c (1 - j t), t = sin / cos; inverse conjugate
    constexpr float t1 = (float)((INV ? -1.0 : 1.0) * C::sinm(C::m1) / c1);
    constexpr float t2 = (float)((INV ? -1.0 : 1.0) * C::sinm(C::m2) / c2);
    constexpr float t3 = (float)((INV ? -1.0 : 1.0) * C::sinm(C::m3) / c3);
    constexpr float f2 = (float)c2, f1 = (float)c1, r31 = (float)(c3 / c1);
    // pre-rotation by (1 - j t): (x + t y, y - t x)
    const float2 p1 = make_float2(fmaf(t1, u[1].y, u[1].x), fmaf(-t1, u[1].x, u[1].y));
    const float2 p2 = make_float2(fmaf(t2, u[2].y, u[2].x), fmaf(-t2, u[2].x, u[2].y));
    const float2 p3 = make_float2(fmaf(t3, u[3].y, u[3].x), fmaf(-t3, u[3].x, u[3].y));
    // radix 4 on (u0, c1 p1, c2 p2, c3 p3)
    const float2 a = make_float2(fmaf(f2, p2.x, u[0].x), fmaf(f2, p2.y, u[0].y));     // u0 + u2
    const float2 b = make_float2(fmaf(-f2, p2.x, u[0].x), fmaf(-f2, p2.y, u[0].y));   // u0 - u2
    const float2 cc = make_float2(fmaf(r31, p3.x, p1.x), fmaf(r31, p3.y, p1.y));      // (u1 + u3) / c1
    const float2 dd = make_float2(fmaf(-r31, p3.x, p1.x), fmaf(-r31, p3.y, p1.y));    // (u1 - u3) / c1
    u[0] = make_float2(fmaf(f1, cc.x, a.x), fmaf(f1, cc.y, a.y));
    u[2] = make_float2(fmaf(-f1, cc.x, a.x), fmaf(-f1, cc.y, a.y));
    // b -/+ j d (forward: b + (-j) d = (b.x + d.y, b.y - d.x)), d = c1 dd
    if constexpr (!INV) {
        u[1] = make_float2(fmaf(f1, dd.y, b.x), fmaf(-f1, dd.x, b.y));
        u[3] = make_float2(fmaf(-f1, dd.y, b.x), fmaf(f1, dd.x, b.y));
    } else {
        u[1] = make_float2(fmaf(-f1, dd.y, b.x), fmaf(f1, dd.x, b.y));
        u[3] = make_float2(fmaf(f1, dd.y, b.x), fmaf(-f1, dd.x, b.y));
    }
}

template <int R, bool INV>
struct Dft {
    static constexpr int R1 = (R >= 16) ? 4 : 2;
    static constexpr int R2 = R / R1;

    // second stage for column KB: factored when possible, else twiddle then radix R1
    template <int KB>
    DBP_HD static void column(float2 (&t)[R1][R2], float2 *v) {
        if constexpr (KB < R2) {
            float2 u[R1];
#pragma unroll
            for (int a = 0; a < R1; ++a) u[a] = t[a][KB];
            if constexpr (R1 == 4 && Col4<R, KB>::ok) {
                col4_factored<R, KB, INV>(u);
            } else {
                twid_col<KB>(u);
                Dft<R1, INV>::run(u);
            }
#pragma unroll
            for (int ka = 0; ka < R1; ++ka) v[KB + R2 * ka] = u[ka];
            column<KB + 1>(t, v);
        }
    }
    template <int KB, int A = 0>
    DBP_HD static void twid_col(float2 (&u)[R1]) {
        if constexpr (A < R1) {
            u[A] = twid<R, A * KB, INV>(u[A]);
            twid_col<KB, A + 1>(u);
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
        column<0>(t, v);
    }
};

}  // namespace dbp
