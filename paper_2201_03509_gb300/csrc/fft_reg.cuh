// Precision-generic complex arithmetic, register DFTs and one Stockham pass
// over a tile of vectors in shared memory.  V is float2 (FP32 path) or
// double2 (FP64 path); every routine is written once for both.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>
#include "internal.cuh"

namespace tg {

template <class V> struct VecT;
template <> struct VecT<float2> {
    typedef float S;
    static __device__ __forceinline__ float2 make(float a, float b) { return make_float2(a, b); }
};
template <> struct VecT<double2> {
    typedef double S;
    static __device__ __forceinline__ double2 make(double a, double b) { return make_double2(a, b); }
};

template <class V> __device__ __forceinline__ V vmake(typename VecT<V>::S a, typename VecT<V>::S b) {
    return VecT<V>::make(a, b);
}
template <class V> __device__ __forceinline__ V vzero() { return VecT<V>::make(0, 0); }
template <class V> __device__ __forceinline__ V vadd(V a, V b) { return vmake<V>(a.x + b.x, a.y + b.y); }
template <class V> __device__ __forceinline__ V vsub(V a, V b) { return vmake<V>(a.x - b.x, a.y - b.y); }
template <class V> __device__ __forceinline__ V vmul(V a, V b) {
    return vmake<V>(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
template <class V> __device__ __forceinline__ V vmulc(V a, V b) {     // a * conj(b)
    return vmake<V>(a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y);
}
template <class V> __device__ __forceinline__ V vconj(V a) { return vmake<V>(a.x, -a.y); }
template <class V> __device__ __forceinline__ V vscale(V a, typename VecT<V>::S s) { return vmake<V>(a.x * s, a.y * s); }
// -i a (forward, e^{-i pi/2}) or +i a (inverse)
template <class V> __device__ __forceinline__ V vmuli(V a, bool inv) {
    return inv ? vmake<V>(-a.y, a.x) : vmake<V>(a.y, -a.x);
}
template <class V> __device__ __forceinline__ V vld(const V *p) { return __ldg(p); }

// ---------------------------------------------------------------------------
// Twiddle constants of the composite register DFTs: cos and sin of 2 pi j/R
// from Taylor series after a quarter-turn reduction (|x| < pi/2, 14 terms:
// below 1e-17), evaluated by the compiler.
// ---------------------------------------------------------------------------
constexpr double kTwoPiR = 6.283185307179586476925286766559;
__host__ __device__ constexpr double rq_sin(double x) {
    double term = x, sum = x;
    for (int i = 1; i < 14; ++i) { term *= -x * x / ((2.0 * i) * (2.0 * i + 1.0)); sum += term; }
    return sum;
}
__host__ __device__ constexpr double rq_cos(double x) {
    double term = 1.0, sum = 1.0;
    for (int i = 1; i < 14; ++i) { term *= -x * x / ((2.0 * i - 1.0) * (2.0 * i)); sum += term; }
    return sum;
}
__host__ __device__ constexpr double turn_cos(int j, int R) {
    const int jj = ((j % R) + R) % R;
    const int q = (4 * jj) / R, rem = 4 * jj - q * R;
    const double x = 0.25 * kTwoPiR * rem / R;
    return q == 0 ? rq_cos(x) : q == 1 ? -rq_sin(x) : q == 2 ? -rq_cos(x) : rq_sin(x);
}
__host__ __device__ constexpr double turn_sin(int j, int R) {
    const int jj = ((j % R) + R) % R;
    const int q = (4 * jj) / R, rem = 4 * jj - q * R;
    const double x = 0.25 * kTwoPiR * rem / R;
    return q == 0 ? rq_sin(x) : q == 1 ? rq_cos(x) : q == 2 ? -rq_sin(x) : -rq_cos(x);
}
// v * W_R^J with W = exp(-+2 pi i/R); exact at the quarter turns
template <int R, int J, bool INV, class V>
__device__ __forceinline__ V rtwiddle(V v) {
    typedef typename VecT<V>::S S;
    constexpr int j = J % R;
    if constexpr (j == 0) return v;
    else if constexpr (2 * j == R) return vmake<V>(-v.x, -v.y);
    else if constexpr (4 * j == R) return vmuli(v, INV);
    else if constexpr (4 * j == 3 * R) return vmuli(v, !INV);
    else {
        constexpr S c = static_cast<S>(turn_cos(j, R));
        constexpr S sn = static_cast<S>(INV ? turn_sin(j, R) : -turn_sin(j, R));
        return vmake<V>(v.x * c - v.y * sn, v.x * sn + v.y * c);
    }
}

// ---------------------------------------------------------------------------
// Register DFTs of radix 2, 3, 4, 5 (textbook butterflies) and composite
// radices by Cooley-Tukey in registers.  Sign -1 forward, +1 inverse; no
// normalisation.
// ---------------------------------------------------------------------------
template <int R, bool INV, class V> struct RDft;

template <bool INV, class V> struct RDft<2, INV, V> {
    static __device__ __forceinline__ void run(V *v) {
        const V a = v[0], b = v[1];
        v[0] = vadd(a, b);
        v[1] = vsub(a, b);
    }
};
template <bool INV, class V> struct RDft<3, INV, V> {
    static __device__ __forceinline__ void run(V *v) {
        typedef typename VecT<V>::S S;
        const S s3 = INV ? static_cast<S>(0.86602540378443864676) : static_cast<S>(-0.86602540378443864676);
        const V a = v[0], t1 = vadd(v[1], v[2]), dd = vsub(v[1], v[2]);
        const V t2 = vmake<V>(a.x - static_cast<S>(0.5) * t1.x, a.y - static_cast<S>(0.5) * t1.y);
        const V t3 = vmake<V>(-s3 * dd.y, s3 * dd.x);
        v[0] = vadd(a, t1);
        v[1] = vadd(t2, t3);
        v[2] = vsub(t2, t3);
    }
};
template <bool INV, class V> struct RDft<4, INV, V> {
    static __device__ __forceinline__ void run(V *v) {
        const V s0 = vadd(v[0], v[2]), d0 = vsub(v[0], v[2]);
        const V s1 = vadd(v[1], v[3]), d1 = vmuli(vsub(v[1], v[3]), INV);
        v[0] = vadd(s0, s1);
        v[2] = vsub(s0, s1);
        v[1] = vadd(d0, d1);
        v[3] = vsub(d0, d1);
    }
};
template <bool INV, class V> struct RDft<5, INV, V> {
    static __device__ __forceinline__ void run(V *v) {
        typedef typename VecT<V>::S S;
        const S c1 = static_cast<S>(0.30901699437494742410), c2 = static_cast<S>(-0.80901699437494742410);
        const S s1 = INV ? static_cast<S>(0.95105651629515357212) : static_cast<S>(-0.95105651629515357212);
        const S s2 = INV ? static_cast<S>(0.58778525229247312917) : static_cast<S>(-0.58778525229247312917);
        const V a = v[0];
        const V be = vadd(v[1], v[4]), bm = vsub(v[1], v[4]);
        const V cd = vadd(v[2], v[3]), cm = vsub(v[2], v[3]);
        const V r1 = vmake<V>(a.x + c1 * be.x + c2 * cd.x, a.y + c1 * be.y + c2 * cd.y);
        const V r2 = vmake<V>(a.x + c2 * be.x + c1 * cd.x, a.y + c2 * be.y + c1 * cd.y);
        const V q1 = vmake<V>(s1 * bm.x + s2 * cm.x, s1 * bm.y + s2 * cm.y);
        const V q2 = vmake<V>(s2 * bm.x - s1 * cm.x, s2 * bm.y - s1 * cm.y);
        const V iq1 = vmake<V>(-q1.y, q1.x), iq2 = vmake<V>(-q2.y, q2.x);
        v[0] = vmake<V>(a.x + be.x + cd.x, a.y + be.y + cd.y);
        v[1] = vadd(r1, iq1);
        v[4] = vsub(r1, iq1);
        v[2] = vadd(r2, iq2);
        v[3] = vsub(r2, iq2);
    }
};

__host__ __device__ constexpr int rdft_first(int R) {
    return (R % 4 == 0) ? 4 : (R % 3 == 0) ? 3 : (R % 5 == 0) ? 5 : 2;
}
// R = A B: X[k1 + A k2] = sum_n2 W_B^{n2 k2} W_R^{n2 k1} sum_n1 x[B n1 + n2] W_A^{n1 k1}
template <int A, int B, bool INV, class V> struct RDftAB {
    template <int N2, int K1>
    static __device__ __forceinline__ void tw(V *u) {
        if constexpr (K1 < A) {
            u[K1] = rtwiddle<A * B, N2 * K1, INV>(u[K1]);
            tw<N2, K1 + 1>(u);
        }
    }
    template <int N2>
    static __device__ __forceinline__ void inner(const V *v, V (&t)[B][A]) {
        if constexpr (N2 < B) {
            V u[A];
#pragma unroll
            for (int n1 = 0; n1 < A; ++n1) u[n1] = v[B * n1 + N2];
            RDft<A, INV, V>::run(u);
            tw<N2, 0>(u);
#pragma unroll
            for (int k1 = 0; k1 < A; ++k1) t[N2][k1] = u[k1];
            inner<N2 + 1>(v, t);
        }
    }
    static __device__ __forceinline__ void run(V *v) {
        V t[B][A];
        inner<0>(v, t);
#pragma unroll
        for (int k1 = 0; k1 < A; ++k1) {
            V w[B];
#pragma unroll
            for (int n2 = 0; n2 < B; ++n2) w[n2] = t[n2][k1];
            RDft<B, INV, V>::run(w);
#pragma unroll
            for (int k2 = 0; k2 < B; ++k2) v[k1 + A * k2] = w[k2];
        }
    }
};
template <int R, bool INV, class V> struct RDft {
    static_assert(R % rdft_first(R) == 0 && R / rdft_first(R) > 1, "composite radix");
    static __device__ __forceinline__ void run(V *v) { RDftAB<rdft_first(R), R / rdft_first(R), INV, V>::run(v); }
};

// ---------------------------------------------------------------------------
// One out-of-place Stockham pass (radix R after Ns points are done) over
// the 2^lgv vectors of length L of a tile in shared memory: element e of
// vector c at c + e 2^lgv (COL: a tile of columns) or c * stride + e (rows).
// Thread t keeps vector t mod 2^lgv (2^lgv divides NT) and takes the
// butterflies j = t >> lgv, j + (NT >> lgv), ..; pass twiddles
// W_L^{r k L/(Ns R)} (k = j mod Ns) from tw (W_L^i, i < L, global).  The
// caller synchronises.  Radices 16, 10, 9, 8, 6, 5, 4, 3, 2.
// ---------------------------------------------------------------------------
template <int R, bool INV, int NT, bool COL, class V>
__device__ __forceinline__ void sp_pass(const V *__restrict__ src, V *__restrict__ dst, int L, const DctStage &st,
                                        int lgv, int stride, const V *__restrict__ tw)
{
    const int LR = L / R;
    const int Ns = st.Ns;
    const int tstep = fdiv(LR, st.fNs);                                             // L / (Ns R)
    const int vec = threadIdx.x & ((1 << lgv) - 1);
    const int es = COL ? (1 << lgv) : 1;
    const int base = COL ? vec : vec * stride;
    const V *s0 = src + base;
    V *d0 = dst + base;
    const int ls = LR * es, ns = Ns * es;
    for (int j = threadIdx.x >> lgv; j < LR; j += NT >> lgv) {
        const V *p = s0 + j * es;
        V v[R];
#pragma unroll
        for (int r = 0; r < R; ++r) v[r] = p[r * ls];
        const int jq = fdiv(j, st.fNs);
        const int k = j - jq * Ns;
        if (Ns > 1) {
            const int ts = k * tstep;
#pragma unroll
            for (int r = 1; r < R; ++r) {
                V t = vld(tw + r * ts);
                if (INV) t.y = -t.y;
                v[r] = vmul(v[r], t);
            }
        }
        RDft<R, INV, V>::run(v);
        V *q = d0 + (jq * Ns * R + k) * es;
#pragma unroll
        for (int r = 0; r < R; ++r) q[r * ns] = v[r];
    }
}

// All passes of a sub-transform, ping-ponging between the two tile buffers
// (a barrier after each); returns the buffer holding the result.
template <bool INV, int NT, bool COL, class V>
__device__ V *sp_transform(V *a, V *b, int L, const DctStage *stages, int nr, int lgv, int stride,
                           const V *__restrict__ tw)
{
    for (int s = 0; s < nr; ++s) {
        const DctStage st = stages[s];
        switch (st.R) {
        case 16: sp_pass<16, INV, NT, COL>(a, b, L, st, lgv, stride, tw); break;
        case 10: sp_pass<10, INV, NT, COL>(a, b, L, st, lgv, stride, tw); break;
        case 9: sp_pass<9, INV, NT, COL>(a, b, L, st, lgv, stride, tw); break;
        case 8: sp_pass<8, INV, NT, COL>(a, b, L, st, lgv, stride, tw); break;
        case 6: sp_pass<6, INV, NT, COL>(a, b, L, st, lgv, stride, tw); break;
        case 5: sp_pass<5, INV, NT, COL>(a, b, L, st, lgv, stride, tw); break;
        case 4: sp_pass<4, INV, NT, COL>(a, b, L, st, lgv, stride, tw); break;
        case 3: sp_pass<3, INV, NT, COL>(a, b, L, st, lgv, stride, tw); break;
        default: sp_pass<2, INV, NT, COL>(a, b, L, st, lgv, stride, tw); break;
        }
        __syncthreads();
        V *t = a; a = b; b = t;
    }
    return a;
}

}  // namespace tg
