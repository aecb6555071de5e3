// A3 batched DCT-II (the mirrored FFT of paper Sect. 4.2), A4 gain draw and
// A5 correlated-noise draw (the gain and n_corr conditionals of Eq.
// `gibbsstart`; Sect. 5 CG gap filling), as persistent thread-block-cluster
// kernels.
//
// One cluster of C CTAs owns one detscan at a time (work list sorted by
// decreasing length; clusters stride through it).  A length-n real DCT-II
// is an m = n/2 complex FFT of the even/odd-packed, reversed-odd sequence
// (Makhoul 1980) followed by a real split.  The FFT is split four-step as
// m = m1 x m2 over the cluster:
//   time layout:  CTA c holds columns j2 in [c*ncolmax, (c+1)*ncolmax) of
//                 z[j1*m2 + j2], stored [j1][local column];
//   freq layout:  CTA c holds the row pairs {p, m1-p}, p in
//                 [c*npmax, (c+1)*npmax), of Z[k1 + m1*k2], stored
//                 [slot][k2] -- a row and its mirror share a CTA, so the real
//                 split that combines Z_k with Z_{m-k} is local.
// Column FFTs (length m1) and row FFTs (length m2) are mixed-radix
// Stockham passes (register DFTs of radix 2 to 16) ping-ponging between two
// shared-memory buffers of ~m/C complex values per CTA; the last column
// pass (forward) or row pass (inverse) writes its outputs, times the
// four-step twiddle, straight into the other CTAs' buffers (DSMEM), which
// is the transpose.  Nothing of a transform touches HBM.
//
// Spectra are kept packed: slot k (1 <= k < m) holds the orthonormal DCT
// coefficients (X_k, X_{n-k}); slot 0 holds (X_0, X_m).
#include <algorithm>
#include <cooperative_groups.h>
#include "common.cuh"
#include "internal.cuh"

namespace cg = cooperative_groups;

namespace tg {

// ---------------------------------------------------------------------------
// small DFTs in registers (sign -1 forward, +1 inverse)
// ---------------------------------------------------------------------------
__device__ __forceinline__ float2 mul_i(float2 a, bool inv) {  // -i*a forward, +i*a inverse
    return inv ? make_float2(-a.y, a.x) : make_float2(a.y, -a.x);
}

template <int R, bool INV> struct Dft;

template <bool INV> struct Dft<2, INV> {
    static __device__ __forceinline__ void run(float2 *v) {
        const float2 a = v[0], b = v[1];
        v[0] = cadd(a, b);
        v[1] = csub(a, b);
    }
};
template <bool INV> struct Dft<4, INV> {
    static __device__ __forceinline__ void run(float2 *v) {
        const float2 s0 = cadd(v[0], v[2]), d0 = csub(v[0], v[2]);
        const float2 s1 = cadd(v[1], v[3]), d1 = mul_i(csub(v[1], v[3]), INV);
        v[0] = cadd(s0, s1);
        v[2] = csub(s0, s1);
        v[1] = cadd(d0, d1);
        v[3] = csub(d0, d1);
    }
};
// 8 = 2 x 4: a_r = v_r + v_{r+4}, b_r = (v_r - v_{r+4}) W8^r; even outputs
// are DFT4(a), odd outputs DFT4(b).
template <bool INV> struct Dft<8, INV> {
    static __device__ __forceinline__ void run(float2 *v) {
        const float c = 0.70710678118654752f;
        float2 a[4], b[4];
#pragma unroll
        for (int r = 0; r < 4; ++r) { a[r] = cadd(v[r], v[r + 4]); b[r] = csub(v[r], v[r + 4]); }
        // W8^1 = (c, -+c), W8^2 = -+i, W8^3 = (-c, -+c)
        b[1] = INV ? make_float2(c * (b[1].x - b[1].y), c * (b[1].x + b[1].y))
                   : make_float2(c * (b[1].x + b[1].y), c * (b[1].y - b[1].x));
        b[2] = mul_i(b[2], INV);
        b[3] = INV ? make_float2(-c * (b[3].x + b[3].y), c * (b[3].x - b[3].y))
                   : make_float2(c * (b[3].y - b[3].x), -c * (b[3].x + b[3].y));
        Dft<4, INV>::run(a);
        Dft<4, INV>::run(b);
#pragma unroll
        for (int u = 0; u < 4; ++u) { v[2 * u] = a[u]; v[2 * u + 1] = b[u]; }
    }
};
template <bool INV> struct Dft<3, INV> {
    static __device__ __forceinline__ void run(float2 *v) {
        const float S3 = INV ? 0.86602540378443865f : -0.86602540378443865f;   // sin(-+2pi/3)
        const float2 a = v[0], t1 = cadd(v[1], v[2]), dd = csub(v[1], v[2]);
        const float2 t2 = make_float2(a.x - 0.5f * t1.x, a.y - 0.5f * t1.y);
        const float2 t3 = make_float2(-S3 * dd.y, S3 * dd.x);                    // i*S3*(b-c)
        v[0] = cadd(a, t1);
        v[1] = cadd(t2, t3);
        v[2] = csub(t2, t3);
    }
};
template <bool INV> struct Dft<5, INV> {
    static __device__ __forceinline__ void run(float2 *v) {
        const float C1 = 0.30901699437494742f, C2 = -0.80901699437494742f;      // cos 2pi/5, cos 4pi/5
        const float S1 = INV ? 0.95105651629515357f : -0.95105651629515357f;    // sin(-+2pi/5)
        const float S2 = INV ? 0.58778525229247313f : -0.58778525229247313f;    // sin(-+4pi/5)
        const float2 a = v[0];
        const float2 be = cadd(v[1], v[4]), bm = csub(v[1], v[4]);
        const float2 cd = cadd(v[2], v[3]), cm = csub(v[2], v[3]);
        const float2 r1 = make_float2(a.x + C1 * be.x + C2 * cd.x, a.y + C1 * be.y + C2 * cd.y);
        const float2 r2 = make_float2(a.x + C2 * be.x + C1 * cd.x, a.y + C2 * be.y + C1 * cd.y);
        const float2 s1 = make_float2(S1 * bm.x + S2 * cm.x, S1 * bm.y + S2 * cm.y);
        const float2 s2 = make_float2(S2 * bm.x - S1 * cm.x, S2 * bm.y - S1 * cm.y);
        const float2 is1 = make_float2(-s1.y, s1.x), is2 = make_float2(-s2.y, s2.x);
        v[0] = make_float2(a.x + be.x + cd.x, a.y + be.y + cd.y);
        v[1] = cadd(r1, is1);
        v[4] = csub(r1, is1);
        v[2] = cadd(r2, is2);
        v[3] = csub(r2, is2);
    }
};

// Composite radix R = A*B (Cooley-Tukey in registers): with n = B n1 + n2
// and k = k1 + A k2,
//   X[k1 + A k2] = sum_n2 W_B^{n2 k2} W_R^{n2 k1} sum_n1 x[B n1 + n2] W_A^{n1 k1}.
// The inner twiddles W_R^{j} are compile-time constants from a Taylor series
// (quarter-turn range reduction, |x| < pi/2, 14 terms: below 1e-17).
constexpr double kTwoPi = 6.283185307179586476925286766559;
__host__ __device__ constexpr double cx_sin_q(double x) {
    double term = x, sum = x;
    for (int i = 1; i < 14; ++i) { term *= -x * x / ((2.0 * i) * (2.0 * i + 1.0)); sum += term; }
    return sum;
}
__host__ __device__ constexpr double cx_cos_q(double x) {
    double term = 1.0, sum = 1.0;
    for (int i = 1; i < 14; ++i) { term *= -x * x / ((2.0 * i - 1.0) * (2.0 * i)); sum += term; }
    return sum;
}
// cos and sin of 2 pi j / R
__host__ __device__ constexpr double cx_cos_turn(int j, int R) {
    const int jj = ((j % R) + R) % R;
    const int q = (4 * jj) / R, rem = 4 * jj - q * R;
    const double x = 0.25 * kTwoPi * rem / R;
    return q == 0 ? cx_cos_q(x) : q == 1 ? -cx_sin_q(x) : q == 2 ? -cx_cos_q(x) : cx_sin_q(x);
}
__host__ __device__ constexpr double cx_sin_turn(int j, int R) {
    const int jj = ((j % R) + R) % R;
    const int q = (4 * jj) / R, rem = 4 * jj - q * R;
    const double x = 0.25 * kTwoPi * rem / R;
    return q == 0 ? cx_sin_q(x) : q == 1 ? cx_cos_q(x) : q == 2 ? -cx_sin_q(x) : -cx_cos_q(x);
}
// v * W_R^{j}, W = exp(-+2 pi i / R); exact for the quarter turns
template <int R, int J, bool INV>
__device__ __forceinline__ float2 twiddle_const(float2 v) {
    constexpr int j = J % R;
    if constexpr (j == 0) return v;
    else if constexpr (2 * j == R) return make_float2(-v.x, -v.y);
    else if constexpr (4 * j == R) return mul_i(v, INV);                 // -i forward
    else if constexpr (4 * j == 3 * R) return mul_i(v, !INV);            // +i forward
    else {
        constexpr float c = static_cast<float>(cx_cos_turn(j, R));
        constexpr float sn = static_cast<float>(INV ? cx_sin_turn(j, R) : -cx_sin_turn(j, R));
        return make_float2(v.x * c - v.y * sn, v.x * sn + v.y * c);
    }
}
__host__ __device__ constexpr int dft_first_factor(int R) {
    return (R % 4 == 0) ? 4 : (R % 3 == 0) ? 3 : (R % 5 == 0) ? 5 : 2;
}
template <int A, int B, bool INV> struct DftAB {
    template <int N2>
    static __device__ __forceinline__ void inner(const float2 *v, float2 (&t)[B][A]) {
        if constexpr (N2 < B) {
            float2 u[A];
#pragma unroll
            for (int n1 = 0; n1 < A; ++n1) u[n1] = v[B * n1 + N2];
            Dft<A, INV>::run(u);
            twid<N2, 0>(u);
#pragma unroll
            for (int k1 = 0; k1 < A; ++k1) t[N2][k1] = u[k1];
            inner<N2 + 1>(v, t);
        }
    }
    template <int N2, int K1>
    static __device__ __forceinline__ void twid(float2 *u) {
        if constexpr (K1 < A) {
            u[K1] = twiddle_const<A * B, N2 * K1, INV>(u[K1]);
            twid<N2, K1 + 1>(u);
        }
    }
    static __device__ __forceinline__ void run(float2 *v) {
        float2 t[B][A];
        inner<0>(v, t);
#pragma unroll
        for (int k1 = 0; k1 < A; ++k1) {
            float2 w[B];
#pragma unroll
            for (int n2 = 0; n2 < B; ++n2) w[n2] = t[n2][k1];
            Dft<B, INV>::run(w);
#pragma unroll
            for (int k2 = 0; k2 < B; ++k2) v[k1 + A * k2] = w[k2];
        }
    }
};
template <int R, bool INV> struct Dft {
    static_assert(R % dft_first_factor(R) == 0 && R / dft_first_factor(R) > 1, "composite radix");
    static __device__ __forceinline__ void run(float2 *v) {
        DftAB<dft_first_factor(R), R / dft_first_factor(R), INV>::run(v);
    }
};

// One butterfly w of a Stockham radix-R pass (Govindaraju et al. 2008
// formulation) over nvec vectors of length L (element stride es, vector
// stride vs): loads its R inputs from src, applies the pass twiddles and
// the register DFT; v gets the outputs, which belong at elements
// jq Ns R + k + r Ns of vector vec.  vfast: consecutive w take consecutive
// vectors (column FFTs) instead of consecutive elements (row FFTs).  Index
// arithmetic uses precomputed multiply-shift divisions.
template <int R, bool INV>
__device__ __forceinline__ void bfly(const float2 *__restrict__ src, int L, const DctStage &st, int nvec,
                                     const FastDiv &fnvec, int es, int vs, bool vfast,
                                     const float2 *__restrict__ tw, int w, float2 (&v)[R], int &vec, int &jq,
                                     int &k)
{
    const int LR = L / R;
    const int Ns = st.Ns;
    const int tstep = L / (Ns * R);
    int j;
    if (vfast) { j = fdiv(w, fnvec); vec = w - j * nvec; }
    else { vec = fdiv(w, st.fLR); j = w - vec * LR; }
    const float2 *p = src + vec * vs + j * es;
#pragma unroll
    for (int r = 0; r < R; ++r) v[r] = p[r * LR * es];
    jq = fdiv(j, st.fNs);
    k = j - jq * Ns;
    if (Ns > 1) {
        if constexpr (R <= 5) {
#pragma unroll
            for (int r = 1; r < R; ++r) {
                float2 t = tw[r * k * tstep];
                if (INV) t.y = -t.y;
                v[r] = cmul(v[r], t);
            }
        } else {
            // W^r for r = 4q + j: W^{4q} from the table, times W^j (j < 4)
            // from W^1 by at most two multiplies
            const int ks = k * tstep;
            float2 w1 = tw[ks];
            if (INV) w1.y = -w1.y;
            const float2 w2 = cmul(w1, w1), w3 = cmul(w2, w1);
#pragma unroll
            for (int q4 = 0; q4 < R; q4 += 4) {
                float2 wq = make_float2(1.f, 0.f);
                if (q4 > 0) { wq = tw[q4 * ks]; if (INV) wq.y = -wq.y; }
#pragma unroll
                for (int jj = 0; jj < 4; ++jj) {
                    const int r = q4 + jj;
                    if (r == 0 || r >= R) continue;
                    const float2 wj = jj == 0 ? make_float2(1.f, 0.f) : jj == 1 ? w1 : jj == 2 ? w2 : w3;
                    const float2 t = q4 == 0 ? wj : (jj == 0 ? wq : cmul(wq, wj));
                    v[r] = cmul(v[r], t);
                }
            }
        }
    }
    Dft<R, INV>::run(v);
}

// One Stockham pass, out of place from src to dst in shared memory; each
// thread loops over whole butterflies; one barrier per pass.
template <int R, bool INV>
__device__ __noinline__ void fft_pass(const float2 *__restrict__ src, float2 *__restrict__ dst, int L,
                                      const DctStage st, int nvec, const FastDiv fnvec, int es, int vs,
                                      bool vfast, const float2 *__restrict__ tw)
{
    const int total = nvec * (L / R);
    const int Ns = st.Ns;
    for (int w = threadIdx.x; w < total; w += DCT_T) {
        float2 v[R];
        int vec, jq, k;
        bfly<R, INV>(src, L, st, nvec, fnvec, es, vs, vfast, tw, w, v, vec, jq, k);
        float2 *q = dst + vec * vs + (jq * Ns * R + k) * es;
#pragma unroll
        for (int r = 0; r < R; ++r) q[r * Ns * es] = v[r];
    }
    __syncthreads();
}

// All passes of one sub-transform, ping-ponging between cur and oth; on
// return cur holds the result.
template <bool INV>
__device__ void fft_seq(float2 *&cur, float2 *&oth, int L, const DctStage *stages, int nr, int nvec,
                        FastDiv fnvec, int es, int vs, bool vfast, const float2 *tw)
{
    for (int s = 0; s < nr; ++s) {
        const DctStage st = stages[s];
        switch (st.R) {
        case 16: fft_pass<16, INV>(cur, oth, L, st, nvec, fnvec, es, vs, vfast, tw); break;
        case 15: fft_pass<15, INV>(cur, oth, L, st, nvec, fnvec, es, vs, vfast, tw); break;
        case 12: fft_pass<12, INV>(cur, oth, L, st, nvec, fnvec, es, vs, vfast, tw); break;
        case 10: fft_pass<10, INV>(cur, oth, L, st, nvec, fnvec, es, vs, vfast, tw); break;
        case 9: fft_pass<9, INV>(cur, oth, L, st, nvec, fnvec, es, vs, vfast, tw); break;
        case 8: fft_pass<8, INV>(cur, oth, L, st, nvec, fnvec, es, vs, vfast, tw); break;
        case 6: fft_pass<6, INV>(cur, oth, L, st, nvec, fnvec, es, vs, vfast, tw); break;
        case 5: fft_pass<5, INV>(cur, oth, L, st, nvec, fnvec, es, vs, vfast, tw); break;
        case 4: fft_pass<4, INV>(cur, oth, L, st, nvec, fnvec, es, vs, vfast, tw); break;
        case 3: fft_pass<3, INV>(cur, oth, L, st, nvec, fnvec, es, vs, vfast, tw); break;
        default: fft_pass<2, INV>(cur, oth, L, st, nvec, fnvec, es, vs, vfast, tw); break;
        }
        float2 *t = cur; cur = oth; oth = t;
    }
}

// ---------------------------------------------------------------------------
// per-detscan transform context (shared memory copy of the plan + this CTA's
// share of it)
// ---------------------------------------------------------------------------
struct Geo {
    int n, m, m1, m2, ncolmax, npmax, P;
    int nr1, nr2;
    int c, C;
    int ncol;    // valid local columns
    int p0, npl; // local row pairs
    FastDiv f_ncolmax, f_m2, f_npmax;
    float sq_fwd, s0_fwd, sq_inv, s0_inv;   // real-split scales
    int m2p;                            // row stride of the frequency layout (odd)
    FastDiv f_2npl;                     // division by the number of local rows
    // twiddles staged in shared memory (see load_plan)
    const float2 *tw1, *tw2;            // W_{m1}^i, W_{m2}^i
    const float2 *sa1, *sb1, *sa5, *sb5;// W_{4n}^{k1}, W_{4n}^{m1 k2}, W_{4n}^{5 k1}, W_{4n}^{5 m1 k2}
    const float2 *t4hi, *t4lo;          // W_m^{64 i}, W_m^i (i < 64)
};
// The shared-memory copy adds the radix stages.  Device code copies the
// Geo part into registers (a local value) before its loops, so stores to
// the transform buffers cannot force the scalars to be reloaded.
struct Ctx : Geo {
    DctStage s1[DCT_MAXR], s2[DCT_MAXR];
};

__device__ __forceinline__ int slot_row(const Geo &X, int slot) {
    const int p = X.p0 + (slot >> 1);
    if (p >= X.P) return -1;
    if ((slot & 1) == 0) return p;
    const int r = X.m1 - p;
    if (p == 0 || r == p) return -1;
    return r;
}

// sample index of position i of the even/odd-reordered sequence v
__device__ __forceinline__ int vpos_t(int i, int n, int m) { return i < m ? 2 * i : 2 * n - 1 - 2 * i; }

// W_m^{r}, 0 <= r < m, from the two-level table (one complex multiply)
__device__ __forceinline__ float2 tw4_lookup(const Geo &X, int r) {
    return cmul(X.t4hi[r >> 6], X.t4lo[r & 63]);
}

// Forward half-split: packed orthonormal coefficients of slot k from Z_k,
// Z_{m-k}: W = e^{-i pi k/2n} A + e^{-i 5 pi k/2n} B, with k = k1 + m1 k2.
__device__ __forceinline__ float2 split_fwd_one(const Geo &X, float2 a, float2 b, int k1, int k2, float sq) {
    const float2 cb = cconj(b);
    const float2 A = cscale(cadd(a, cb), 0.5f);
    const float2 d = csub(a, cb);
    const float2 Bv = make_float2(0.5f * d.y, -0.5f * d.x);                     // -i/2 (a - conj b)
    const float2 e1 = cmul(X.sa1[k1], X.sb1[k2]), e5 = cmul(X.sa5[k1], X.sb5[k2]);
    const float2 W = cadd(cmul(e1, A), cmul(e5, Bv));
    return make_float2(sq * W.x, -sq * W.y);
}
// Inverse of the half-split: Z_k from the packed slots k and m-k.
__device__ __forceinline__ float2 split_inv_one(const Geo &X, float2 yk, float2 yp, int k1, int k2, int q1,
                                                int q2, float sq) {
    // V_k = sqrt(n/2) e^{i pi k/2n} conj(Y_k)   (sq carries sqrt(n/2)/m)
    const float2 ek = cmul(X.sa1[k1], X.sb1[k2]), ep = cmul(X.sa1[q1], X.sb1[q2]);
    const float2 Vk = cscale(cmulc(cconj(yk), ek), sq);
    const float2 Vp = cscale(cmulc(cconj(yp), ep), sq);
    const float2 cVp = cconj(Vp);
    const float2 A = cscale(cadd(Vk, cVp), 0.5f);
    const float2 e4 = cmulc(cmul(X.sa5[k1], X.sb5[k2]), ek);                  // W_{4n}^{4k} = e^{-2 pi i k/n}
    const float2 Bv = cscale(cmulc(csub(Vk, cVp), e4), 0.5f);                  // e^{+2 pi i k/n} (...)
    return make_float2(A.x - Bv.y, A.y + Bv.x);                                 // A + i B
}

// Real split over this CTA's row pairs, in place (forward or inverse).
template <bool INV>
__device__ __noinline__ void split_pass(const Ctx &XS, float2 *__restrict__ U)
{
    const Geo X = XS;       // from shared memory into registers (no by-value copy on the stack)
    const int m2 = X.m2, m2p = X.m2p, m1 = X.m1, p0 = X.p0;
    const float sq = INV ? X.sq_inv : X.sq_fwd;
    const float s0 = INV ? X.s0_inv : X.s0_fwd;
    const int total = X.npl * m2;
    const FastDiv fm2 = X.f_m2;
    for (int e = threadIdx.x; e < total; e += DCT_T) {
        const int pl = fdiv(e, fm2), k2 = e - pl * m2;
        const int p = p0 + pl;
        const int cnt = (p == 0) ? (m2 / 2 + 1) : ((2 * p == m1) ? (m2 + 1) / 2 : m2);
        if (k2 >= cnt) continue;
        // partner m - k: row (m1 - p) mod m1, column m2-1-k2 (p > 0) or (m2-k2) mod m2 (p = 0)
        int ib, q1, q2;
        if (p == 0) { q1 = 0; q2 = (k2 == 0) ? 0 : m2 - k2; ib = 2 * pl * m2p + q2; }
        else { q1 = m1 - p; q2 = m2 - 1 - k2; ib = ((q1 == p) ? 2 * pl : 2 * pl + 1) * m2p + q2; }
        const int ia = 2 * pl * m2p + k2;
        const float2 Za = U[ia], Zb = U[ib];
        if (p == 0 && k2 == 0) {
            if (!INV) {
                const float V0 = Za.x + Za.y, Vm = Za.x - Za.y;
                U[ia] = make_float2(V0 * s0, Vm * s0);
            } else {
                const float V0 = Za.x * s0, Vm = Za.y * s0;
                U[ia] = make_float2(0.5f * (V0 + Vm), 0.5f * (V0 - Vm));
            }
            continue;
        }
        if (!INV) {
            const float2 Ya = split_fwd_one(X, Za, Zb, p, k2, sq);
            if (ib != ia) U[ib] = split_fwd_one(X, Zb, Za, q1, q2, sq);
            U[ia] = Ya;
        } else {
            const float2 Ya = split_inv_one(X, Za, Zb, p, k2, q1, q2, sq);
            if (ib != ia) U[ib] = split_inv_one(X, Zb, Za, q1, q2, p, k2, sq);
            U[ia] = Ya;
        }
    }
    __syncthreads();
}

// Forward split, a per-mode filter and the inverse split in one pass over
// this CTA's row pairs, in place: Z -> Y (packed orthonormal coefficients)
// -> f(e, k, Y) -> Z'.  f gets the element index e and the mode k of Y.x
// (Y.y is mode n - k, or m when k = 0).  Equivalent to split_pass<false>,
// a filter pass and split_pass<true>, with one load and one store.
template <class F>
__device__ __forceinline__ void split_roundtrip(const Geo &XS, float2 *__restrict__ U, F f)
{
    const Geo X = XS;       // registers: the stores to U cannot alias it
    const int m2 = X.m2, m2p = X.m2p, m1 = X.m1, p0 = X.p0;
    const float sqf = X.sq_fwd, s0f = X.s0_fwd, sqi = X.sq_inv, s0i = X.s0_inv;
    const int total = X.npl * m2;
    const FastDiv fm2 = X.f_m2;
    for (int e = threadIdx.x; e < total; e += DCT_T) {
        const int pl = fdiv(e, fm2), k2 = e - pl * m2;
        const int p = p0 + pl;
        const int cnt = (p == 0) ? (m2 / 2 + 1) : ((2 * p == m1) ? (m2 + 1) / 2 : m2);
        if (k2 >= cnt) continue;
        int ib, q1, q2;
        if (p == 0) { q1 = 0; q2 = (k2 == 0) ? 0 : m2 - k2; ib = 2 * pl * m2p + q2; }
        else { q1 = m1 - p; q2 = m2 - 1 - k2; ib = ((q1 == p) ? 2 * pl : 2 * pl + 1) * m2p + q2; }
        const int ia = 2 * pl * m2p + k2;
        const float2 Za = U[ia], Zb = U[ib];
        if (p == 0 && k2 == 0) {
            float2 Y = make_float2((Za.x + Za.y) * s0f, (Za.x - Za.y) * s0f);
            Y = f(ia, 0, Y);
            const float V0 = Y.x * s0i, Vm = Y.y * s0i;
            U[ia] = make_float2(0.5f * (V0 + Vm), 0.5f * (V0 - Vm));
            continue;
        }
        float2 Ya = split_fwd_one(X, Za, Zb, p, k2, sqf);
        Ya = f(ia, p + m1 * k2, Ya);
        if (ib != ia) {
            float2 Yb = split_fwd_one(X, Zb, Za, q1, q2, sqf);
            Yb = f(ib, q1 + m1 * q2, Yb);
            U[ib] = split_inv_one(X, Yb, Ya, q1, q2, p, k2, sqi);
            U[ia] = split_inv_one(X, Ya, Yb, p, k2, q1, q2, sqi);
        } else {
            U[ia] = split_inv_one(X, Ya, Ya, p, k2, q1, q2, sqi);
        }
    }
    __syncthreads();
}

// The inverse split alone, from packed orthonormal coefficients given per
// element: f(e, k) is the coefficient pair of element e (modes k and n - k,
// or 0 and m when k = 0); writes Z into this CTA's row pairs of U, as the
// second half of split_roundtrip does.
template <class F>
__device__ __forceinline__ void split_inverse_from(const Geo &XS, float2 *__restrict__ U, F f)
{
    const Geo X = XS;
    const int m2 = X.m2, m2p = X.m2p, m1 = X.m1, p0 = X.p0;
    const float sqi = X.sq_inv, s0i = X.s0_inv;
    const int total = X.npl * m2;
    const FastDiv fm2 = X.f_m2;
    for (int e = threadIdx.x; e < total; e += DCT_T) {
        const int pl = fdiv(e, fm2), k2 = e - pl * m2;
        const int p = p0 + pl;
        const int cnt = (p == 0) ? (m2 / 2 + 1) : ((2 * p == m1) ? (m2 + 1) / 2 : m2);
        if (k2 >= cnt) continue;
        int ib, q1, q2;
        if (p == 0) { q1 = 0; q2 = (k2 == 0) ? 0 : m2 - k2; ib = 2 * pl * m2p + q2; }
        else { q1 = m1 - p; q2 = m2 - 1 - k2; ib = ((q1 == p) ? 2 * pl : 2 * pl + 1) * m2p + q2; }
        const int ia = 2 * pl * m2p + k2;
        const float2 Ya = f(ia, p + m1 * k2);
        if (p == 0 && k2 == 0) {
            const float V0 = Ya.x * s0i, Vm = Ya.y * s0i;
            U[ia] = make_float2(0.5f * (V0 + Vm), 0.5f * (V0 - Vm));
            continue;
        }
        if (ib != ia) {
            const float2 Yb = f(ib, q1 + m1 * q2);
            U[ib] = split_inv_one(X, Yb, Ya, q1, q2, p, k2, sqi);
            U[ia] = split_inv_one(X, Ya, Yb, p, k2, q1, q2, sqi);
        } else {
            U[ia] = split_inv_one(X, Ya, Ya, p, k2, q1, q2, sqi);
        }
    }
    __syncthreads();
}

// The last Stockham pass of the column FFTs (forward) or of the row FFTs
// (inverse) with the four-step transpose folded in: each output goes,
// times the four-step twiddle W_m^{-+ j2 k1}, straight into the shared
// memory of the CTA that owns it in the other layout, into that CTA's
// buffer dst (the same offset in every CTA).  Forward: vector = local
// column j2, output k1 -> frequency-layout slot of row k1 in the CTA that
// holds the pair {k1, m1-k1}.  Inverse: vector = local row slot (row k1),
// output j2 -> time-layout column j2 of its CTA.  The first butterfly of
// each thread is computed between the two halves of the barrier that
// frees every CTA's dst, hiding its latency; a full cluster barrier at the
// end makes every remote write visible.  Slots and columns that hold no
// data (the odd slot of a single-row pair, the padding columns of the last
// CTA) are not written and are never read.
template <int R, bool INV>
__device__ __noinline__ void fft_push(const Ctx &XS, float2 *__restrict__ src, float2 *dst, int L,
                                      const DctStage st, int nvec, const FastDiv fnvec, int es, int vs,
                                      bool vfast, const float2 *__restrict__ tw, cg::cluster_group &cl)
{
    const Geo X = XS;
    const int total = nvec * (L / R);
    const int Ns = st.Ns;
    const int LR = L / R;
    // The cluster barrier in two halves (every thread of every CTA takes
    // both): arrive once this thread is done with dst and the earlier
    // passes, wait until every thread of the cluster is.  In between, the
    // thread's first butterfly is computed and put back in place (its R
    // inputs are read by no other butterfly): registers live across the
    // wait would go to local memory.
    auto token = cl.barrier_arrive();
    float2 v[R];
    int vec = 0, jq = 0, k = 0;
    if (threadIdx.x < total) {
        bfly<R, INV>(src, L, st, nvec, fnvec, es, vs, vfast, tw, threadIdx.x, v, vec, jq, k);
        float2 *pp = src + vec * vs + k * es;            // the last pass: jq = 0, j = k
#pragma unroll
        for (int r = 0; r < R; ++r) pp[r * LR * es] = v[r];
    }
    cl.barrier_wait(std::move(token));      // every CTA's dst is free
    for (int w = threadIdx.x; w < total; w += DCT_T) {
        if (w != threadIdx.x) {
            bfly<R, INV>(src, L, st, nvec, fnvec, es, vs, vfast, tw, w, v, vec, jq, k);
        } else {
            if (vfast) { k = fdiv(w, fnvec); vec = w - k * nvec; }
            else { vec = fdiv(w, st.fLR); k = w - vec * LR; }
            const float2 *pp = src + vec * vs + k * es;
#pragma unroll
            for (int r = 0; r < R; ++r) v[r] = pp[r * LR * es];
        }
        if (!INV) {
            if (vec >= X.ncol) continue;                     // padding column
            const int j2 = X.c * X.ncolmax + vec;
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const int k1 = k + r * Ns;
                const int p = min(k1, X.m1 - k1);
                const int o = fdiv(p, X.f_npmax);
                const int slot = 2 * (p - o * X.npmax) + (k1 == p ? 0 : 1);
                cl.map_shared_rank(dst, o)[slot * X.m2p + j2] = cmul(v[r], tw4_lookup(X, j2 * k1));
            }
        } else {
            const int k1 = slot_row(X, vec);
            if (k1 < 0) continue;                            // slot without a row
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const int j2 = k + r * Ns;
                const int o = fdiv(j2, X.f_ncolmax);
                cl.map_shared_rank(dst, o)[k1 * X.ncolmax + (j2 - o * X.ncolmax)] =
                    cmulc(v[r], tw4_lookup(X, j2 * k1));
            }
        }
    }
    cl.sync();                // every remote write has landed
}

// The last pass of a sub-transform as fft_push, by radix.
template <bool INV>
__device__ void fft_push_last(const Ctx &XS, float2 *src, float2 *dst, int L, const DctStage &st, int nvec,
                              FastDiv fnvec, int es, int vs, bool vfast, const float2 *tw,
                              cg::cluster_group &cl)
{
    switch (st.R) {
    case 16: fft_push<16, INV>(XS, src, dst, L, st, nvec, fnvec, es, vs, vfast, tw, cl); break;
    case 15: fft_push<15, INV>(XS, src, dst, L, st, nvec, fnvec, es, vs, vfast, tw, cl); break;
    case 12: fft_push<12, INV>(XS, src, dst, L, st, nvec, fnvec, es, vs, vfast, tw, cl); break;
    case 10: fft_push<10, INV>(XS, src, dst, L, st, nvec, fnvec, es, vs, vfast, tw, cl); break;
    case 9: fft_push<9, INV>(XS, src, dst, L, st, nvec, fnvec, es, vs, vfast, tw, cl); break;
    case 8: fft_push<8, INV>(XS, src, dst, L, st, nvec, fnvec, es, vs, vfast, tw, cl); break;
    case 6: fft_push<6, INV>(XS, src, dst, L, st, nvec, fnvec, es, vs, vfast, tw, cl); break;
    case 5: fft_push<5, INV>(XS, src, dst, L, st, nvec, fnvec, es, vs, vfast, tw, cl); break;
    case 4: fft_push<4, INV>(XS, src, dst, L, st, nvec, fnvec, es, vs, vfast, tw, cl); break;
    case 3: fft_push<3, INV>(XS, src, dst, L, st, nvec, fnvec, es, vs, vfast, tw, cl); break;
    default: fft_push<2, INV>(XS, src, dst, L, st, nvec, fnvec, es, vs, vfast, tw, cl); break;
    }
}

// Forward DCT: time layout in cur -> packed spectrum in cur (the two
// buffers may swap roles).
__device__ __noinline__ bool dct_forward(const Ctx &XS, float2 *cur, float2 *oth, const float2 *,
                                         const float2 *, cg::cluster_group &cl)
{
    float2 *const c0 = cur;
    const Geo X = XS;
    const float2 *tw1 = X.tw1, *tw2 = X.tw2;
    fft_seq<false>(cur, oth, X.m1, XS.s1, X.nr1 - 1, X.ncolmax, X.f_ncolmax, X.ncolmax, 1, true, tw1);
    fft_push_last<false>(XS, cur, oth, X.m1, XS.s1[X.nr1 - 1], X.ncolmax, X.f_ncolmax, X.ncolmax, 1, true, tw1, cl);
    { float2 *t = cur; cur = oth; oth = t; }
    fft_seq<false>(cur, oth, X.m2, XS.s2, X.nr2, 2 * X.npl, X.f_2npl, 1, X.m2p, true, tw2);
    split_pass<false>(XS, cur);
    return cur != c0;     // the result is in the caller's other buffer
}
// Inverse (transpose of the orthonormal DCT-II): packed spectrum in cur ->
// time layout in cur, scaled.
__device__ __noinline__ bool dct_inverse(const Ctx &XS, float2 *cur, float2 *oth, const float2 *,
                                         const float2 *, cg::cluster_group &cl)
{
    float2 *const c0 = cur;
    const Geo X = XS;
    const float2 *tw1 = X.tw1, *tw2 = X.tw2;
    split_pass<true>(XS, cur);
    fft_seq<true>(cur, oth, X.m2, XS.s2, X.nr2 - 1, 2 * X.npl, X.f_2npl, 1, X.m2p, true, tw2);
    fft_push_last<true>(XS, cur, oth, X.m2, XS.s2[X.nr2 - 1], 2 * X.npl, X.f_2npl, 1, X.m2p, false, tw2, cl);
    { float2 *t = cur; cur = oth; oth = t; }
    fft_seq<true>(cur, oth, X.m1, XS.s1, X.nr1, X.ncolmax, X.f_ncolmax, X.ncolmax, 1, true, tw1);
    return cur != c0;     // the result is in the caller's other buffer
}

// The two halves of a filter round trip: time layout -> row-FFT output
// (split not applied), and back.
__device__ __noinline__ bool dct_forward_pre(const Ctx &XS, float2 *cur, float2 *oth, cg::cluster_group &cl)
{
    float2 *const c0 = cur;
    const Geo X = XS;
    fft_seq<false>(cur, oth, X.m1, XS.s1, X.nr1 - 1, X.ncolmax, X.f_ncolmax, X.ncolmax, 1, true, X.tw1);
    fft_push_last<false>(XS, cur, oth, X.m1, XS.s1[X.nr1 - 1], X.ncolmax, X.f_ncolmax, X.ncolmax, 1, true, X.tw1,
                         cl);
    { float2 *t = cur; cur = oth; oth = t; }
    fft_seq<false>(cur, oth, X.m2, XS.s2, X.nr2, 2 * X.npl, X.f_2npl, 1, X.m2p, true, X.tw2);
    return cur != c0;     // the result is in the caller's other buffer
}
__device__ __noinline__ bool dct_inverse_post(const Ctx &XS, float2 *cur, float2 *oth, cg::cluster_group &cl)
{
    float2 *const c0 = cur;
    const Geo X = XS;
    fft_seq<true>(cur, oth, X.m2, XS.s2, X.nr2 - 1, 2 * X.npl, X.f_2npl, 1, X.m2p, true, X.tw2);
    fft_push_last<true>(XS, cur, oth, X.m2, XS.s2[X.nr2 - 1], 2 * X.npl, X.f_2npl, 1, X.m2p, false, X.tw2, cl);
    { float2 *t = cur; cur = oth; oth = t; }
    fft_seq<true>(cur, oth, X.m1, XS.s1, X.nr1, X.ncolmax, X.f_ncolmax, X.ncolmax, 1, true, X.tw1);
    return cur != c0;     // the result is in the caller's other buffer
}

// Fill U (time layout) with f(j) = (x_{t(2j)}, x_{t(2j+1)}) for own columns.
template <class F>
__device__ void load_time(const Geo &X, float2 *__restrict__ U, F f)
{
    constexpr int UB = 4;
    const int total = X.m1 * X.ncolmax;
    const FastDiv fnc = X.f_ncolmax;
    for (int e0 = threadIdx.x; e0 < total; e0 += UB * DCT_T) {
        float2 z[UB];
#pragma unroll
        for (int u = 0; u < UB; ++u) {
            const int e = e0 + u * DCT_T;
            z[u] = make_float2(0.f, 0.f);
            if (e < total) {
                const int j1 = fdiv(e, fnc), lc = e - j1 * X.ncolmax;
                if (lc < X.ncol) z[u] = f(j1 * X.m2 + X.c * X.ncolmax + lc);
            }
        }
#pragma unroll
        for (int u = 0; u < UB; ++u) {
            const int e = e0 + u * DCT_T;
            if (e < total) U[e] = z[u];
        }
    }
    __syncthreads();
}

// Cluster-wide sums of two FP32 double-words in a fixed order (identical in
// every CTA): warp trees in double-word FP32, the 16 warp partials and the C
// CTA partials added in FP64 by thread 0 only (FP64 issues at 1/64 of the
// FP32 rate on this part), the result broadcast through shared memory.
__device__ __forceinline__ Acc2 acc_merge2(const Acc2 &a, const Acc2 &b) {
    Acc2 r = a;
    acc_add(r, b.s);
    r.c = __fadd_rn(r.c, b.c);
    return r;
}
// First half: this CTA's partial sums into its slot s_part[parity] (all
// threads take part).  A cluster barrier must follow before the second.
__device__ __forceinline__ void cluster_sum_publish(Acc2 x, Acc2 y, double2 *s_red, double2 *s_part, int parity)
{
#pragma unroll
    for (int o = 16; o; o >>= 1) {
        Acc2 ox, oy;
        ox.s = __shfl_xor_sync(0xffffffffu, x.s, o);
        ox.c = __shfl_xor_sync(0xffffffffu, x.c, o);
        oy.s = __shfl_xor_sync(0xffffffffu, y.s, o);
        oy.c = __shfl_xor_sync(0xffffffffu, y.c, o);
        x = acc_merge2(x, ox);
        y = acc_merge2(y, oy);
    }
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) s_red[warp] = make_double2(acc_value(x), acc_value(y));
    __syncthreads();
    if (threadIdx.x == 0) {
        double2 t = make_double2(0.0, 0.0);
        for (int w = 0; w < DCT_T / 32; ++w) { t.x += s_red[w].x; t.y += s_red[w].y; }
        s_part[parity] = t;
    }
}
// Second half, after the barrier: every CTA's slot added in rank order,
// broadcast to the CTA; flips parity (consecutive sums use alternate slots,
// so a slot is never rewritten while a sibling may still read it).
__device__ __forceinline__ double2 cluster_sum_collect(double2 *s_red, double2 *s_part, int &parity,
                                                       cg::cluster_group &cl)
{
    if (threadIdx.x == 0) {
        double2 tot = make_double2(0.0, 0.0);
        for (int r = 0; r < static_cast<int>(cl.num_blocks()); ++r) {
            const double2 pr = *cl.map_shared_rank(&s_part[parity], r);
            tot.x += pr.x;
            tot.y += pr.y;
        }
        s_red[DCT_T / 32] = tot;
    }
    __syncthreads();
    const double2 tot = s_red[DCT_T / 32];
    parity ^= 1;
    return tot;
}
__device__ __forceinline__ double2 cluster_sum_acc(Acc2 x, Acc2 y, double2 *s_red, double2 *s_part, int &parity,
                                                   cg::cluster_group &cl)
{
    cluster_sum_publish(x, y, s_red, s_part, parity);
    cl.sync();
    return cluster_sum_collect(s_red, s_part, parity, cl);
}

// Per-detscan scalars: FP64 arithmetic (1/64 of the FP32 rate on this
// part) done once by thread 0 and broadcast through shared memory.
struct DetScal { float fscale, alpha, s2, inv_s2, inv_s, g; };
__device__ __forceinline__ DetScal det_scalars(DetScal *sh, const double *psd, int det, int n, double fsamp,
                                               const double *gain, int q)
{
    if (threadIdx.x == 0) {
        const double sig0 = psd[3 * det], fk = psd[3 * det + 1], al = psd[3 * det + 2];
        DetScal v;
        v.fscale = static_cast<float>(fsamp / (2.0 * n * fk));
        v.alpha = static_cast<float>(al);
        v.s2 = static_cast<float>(sig0 * sig0);
        v.inv_s2 = static_cast<float>(1.0 / (sig0 * sig0));
        v.inv_s = static_cast<float>(1.0 / sig0);
        v.g = gain ? static_cast<float>(gain[q]) : 1.0f;
        *sh = v;
    }
    __syncthreads();
    return *sh;
}

__device__ __forceinline__ bool flagged(const uint32_t *flags, int64_t t) {
    return (flags[t >> 5] >> (t & 31)) & 1u;
}

// (f/fknee)^alpha at DCT mode kappa, FP32
__device__ __forceinline__ float fratio_pow(int kappa, float fscale, float alpha) {
    return exp2f(alpha * log2f(static_cast<float>(kappa) * fscale));
}

// shared-memory carve-up common to both kernels: two transform buffers,
// then the twiddle block of the current length, then kernel-specific areas
struct Smem {
    float2 *U0, *U1, *twb;
    const float2 *tw1, *tw2;
    void *tail;
};
__device__ __forceinline__ Smem carve(void *raw, int sz, int twsz)
{
    Smem s;
    float2 *p = static_cast<float2 *>(raw);
    s.U0 = p; p += sz;
    s.U1 = p; p += sz;
    s.twb = p; p += twsz;
    s.tw1 = nullptr;
    s.tw2 = nullptr;
    s.tail = p;
    return s;
}

// Stage plan pi in shared memory: scalars and stage tables into sX, the
// length's twiddle block into sm.twb (all threads copy).  Nothing writes
// either during a detscan, so when the previous detscan of this CTA had the
// same plan (the work list is sorted by length) they are kept.
__device__ __forceinline__ void load_plan(Ctx *sX, const DctPlan *plans, int pi, const float2 *tw, Smem &sm, int c,
                                          int C, int &cur_pi)
{
    __syncthreads();      // previous users of sX and the twiddle block are done
    if (pi == cur_pi) return;
    cur_pi = pi;
    const DctPlan &P = plans[pi];
    const int t = threadIdx.x;
    if (t >= 32 && t < 32 + DCT_MAXR) sX->s1[t - 32] = P.s1[t - 32];
    else if (t >= 64 && t < 64 + DCT_MAXR) sX->s2[t - 64] = P.s2[t - 64];
    else if (t == 0) {
        Ctx &X = *sX;
        X.n = P.n; X.m = P.m; X.m1 = P.m1; X.m2 = P.m2; X.ncolmax = P.ncolmax; X.npmax = P.npmax;
        X.P = P.P; X.nr1 = P.nr1; X.nr2 = P.nr2; X.c = c; X.C = C;
        X.ncol = max(0, min(P.ncolmax, P.m2 - c * P.ncolmax));
        X.p0 = c * P.npmax;
        X.npl = max(0, min(P.npmax, P.P - X.p0));
        X.f_ncolmax = P.f_ncolmax; X.f_m2 = P.f_m2; X.f_npmax = P.f_npmax;
        X.sq_fwd = P.sq_fwd; X.s0_fwd = P.s0_fwd; X.sq_inv = P.sq_inv; X.s0_inv = P.s0_inv;
        X.m2p = P.m2p;
        X.f_2npl = make_fastdiv_dev(static_cast<uint32_t>(max(1, 2 * X.npl)));
        const float2 *b = sm.twb;
        X.tw1 = b; b += P.m1;
        X.tw2 = b; b += P.m2;
        X.sa1 = b; b += P.m1;
        X.sb1 = b; b += P.m2;
        X.sa5 = b; b += P.m1;
        X.sb5 = b; b += P.m2;
        X.t4hi = b; b += P.m / 64 + 1;
        X.t4lo = b;
    }
    const int cnt = 3 * (P.m1 + P.m2) + P.m / 64 + 65;
    const float2 *src = tw + P.twb;
    for (int i = t; i < cnt; i += DCT_T) sm.twb[i] = __ldg(src + i);
    __syncthreads();
    sm.tw1 = sX->tw1;
    sm.tw2 = sX->tw2;
}

// element e of the time layout -> (t0, t1) samples
__device__ __forceinline__ void elem_samples(const Geo &X, int e, int &t0, int &t1, bool &valid)
{
    const int j1 = fdiv(e, X.f_ncolmax), lc = e - j1 * X.ncolmax;
    valid = lc < X.ncol;
    const int j = j1 * X.m2 + X.c * X.ncolmax + lc;
    t0 = vpos_t(2 * j, X.n, X.m);
    t1 = vpos_t(2 * j + 1, X.n, X.m);
}
// sample t -> (owner CTA, element, part)
__device__ __forceinline__ void sample_loc(const Geo &X, int t, int &owner, int &loc)
{
    // position of sample t in the even-then-reversed-odd order: t/2 for even
    // t, n-1-(t-1)/2 = n-1-floor(t/2) for odd t
    const int h = t >> 1;
    const int i = (t & 1) ? (X.n - 1) - h : h;
    const int j = i >> 1;
    const int j1 = fdiv(j, X.f_m2), j2 = j - j1 * X.m2;
    owner = fdiv(j2, X.f_ncolmax);
    const int lc = j2 - owner * X.ncolmax;
    loc = 2 * (j1 * X.ncolmax + lc) + (i & 1);
}


// ---------------------------------------------------------------------------
// A4: gain.  a = sum_{k>=1} shat_k^2 / P_k from the forward transform of
// M s; b = sum_k shat_k dhat_k / P_k = <M s, C^T diag(1/P) C (M d)> in the
// time domain, so two buffers suffice.
// ---------------------------------------------------------------------------
struct GainArgs {
    const float *d, *s;
    const uint32_t *flags;
    const double *psd;
    const int64_t *off;
    const DctPlan *plans;
    const int32_t *q_plan;
    const float2 *tw;
    const int32_t *work;
    int work_begin, work_count;
    int ndet;
    double fsamp;
    tod_rng rng;
    int mode;
    double2 *ab_out;              // (a, b) of each detscan's conditional
    int sz, m1max, m2max, twsz;
};

__global__ void __launch_bounds__(DCT_T, 1) k_gain(GainArgs a)
{
    extern __shared__ __align__(16) float2 smem_raw[];
    __shared__ Ctx sX;
    __shared__ DetScal s_sc;
    __shared__ double2 s_red[DCT_T / 32 + 1];
    __shared__ double2 s_part[2];
    cg::cluster_group cl = cg::this_cluster();
    const int C = static_cast<int>(cl.num_blocks()), c = static_cast<int>(cl.block_rank());
    const int cid = blockIdx.x / C, ncl = gridDim.x / C;
    Smem sm = carve(smem_raw, a.sz, a.twsz);
    int parity = 0;
    int cur_pi = -1;      // plan staged in shared memory
    for (int w = cid; w < a.work_count; w += ncl) {
        const int q = a.work[a.work_begin + w];
        const int det = q % a.ndet;
        const int64_t o = a.off[q];
        load_plan(&sX, a.plans, a.q_plan[q], a.tw, sm, c, C, cur_pi);
        const Ctx &X = sX;     // shared-memory copy (a register copy would live on the stack)
        const int n = X.n, m = X.m;
        const float *sq = a.s + o, *dq = a.d + o;
        const uint32_t *fl = a.flags;
        const DetScal sc = det_scalars(&s_sc, a.psd, det, n, a.fsamp, nullptr, q);
        const float fscale = sc.fscale, alpha = sc.alpha, s2 = sc.s2;
        float2 *cur = sm.U0, *oth = sm.U1;
        // shat = C(M s); a = sum_k shat_k^2 / P_k; then u = C^T(shat / P) and
        // b = sum_t M_t d_t u_t = sum_k shat_k dhat_k / P_k (two transforms)
        load_time(X, cur, [&](int j) {
            const int t0 = vpos_t(2 * j, n, m), t1 = vpos_t(2 * j + 1, n, m);
            const float v0 = __ldg(sq + t0), v1 = __ldg(sq + t1);      // independent of the flags
            return make_float2(flagged(fl, o + t0) ? 0.f : v0, flagged(fl, o + t1) ? 0.f : v1);
        });
        if (dct_forward_pre(sX, cur, oth, cl)) { float2 *t_ = cur; cur = oth; oth = t_; }
        Acc2 sa = {0.f, 0.f}, sb = {0.f, 0.f};
        split_roundtrip(X, cur, [&](int, int k, float2 S) {
            const int ka = k, kb = (k == 0) ? m : n - k;
            const float wa = ka == 0 ? 0.f : 1.0f / (s2 * (1.0f + fratio_pow(ka, fscale, alpha)));
            const float wb = 1.0f / (s2 * (1.0f + fratio_pow(kb, fscale, alpha)));
            const float2 W = make_float2(S.x * wa, S.y * wb);
            acc_add_prod(sa, S.x, W.x);
            acc_add_prod(sa, S.y, W.y);
            return W;
        });
        if (dct_inverse_post(sX, cur, oth, cl)) { float2 *t_ = cur; cur = oth; oth = t_; }
        {
            // four elements per thread with every load in flight, summed in
            // element order (a flagged sample adds an exact zero)
            constexpr int UB = 4;
            const int tot = X.m1 * X.ncolmax;
            for (int e0 = threadIdx.x; e0 < tot; e0 += UB * DCT_T) {
                float2 v[UB], dv[UB];
#pragma unroll
                for (int u = 0; u < UB; ++u) {
                    const int e = e0 + u * DCT_T;
                    v[u] = make_float2(0.f, 0.f);
                    dv[u] = make_float2(0.f, 0.f);
                    if (e < tot) {
                        int t0, t1;
                        bool valid;
                        elem_samples(X, e, t0, t1, valid);
                        if (valid) {
                            v[u] = cur[e];
                            const float d0 = __ldg(dq + t0), d1 = __ldg(dq + t1);
                            dv[u] = make_float2(flagged(fl, o + t0) ? 0.f : d0, flagged(fl, o + t1) ? 0.f : d1);
                        }
                    }
                }
#pragma unroll
                for (int u = 0; u < UB; ++u) {
                    acc_add_prod(sb, dv[u].x, v[u].x);
                    acc_add_prod(sb, dv[u].y, v[u].y);
                }
            }
        }
        const double2 ab = cluster_sum_acc(sa, sb, s_red, s_part,
                                        parity, cl);
        // the FP64 draw (1/64 FP32 rate: long for one thread) runs afterwards
        // in k_gain_draw, off this cluster's critical path
        if (c == 0 && threadIdx.x == 0) a.ab_out[q] = ab;
    }
    cl.sync();     // no CTA leaves while a sibling may still read its cluster-sum slot
}

// The gain draws of the detscans k_gain just summed: g ~ N(b/a, 1/a)
// (mean and rms also written when asked for); a <= 0 (no usable samples)
// gives g = 0 and TOD_ERR_ARG for the detscan.  One thread per detscan.
__global__ void __launch_bounds__(256) k_gain_draw(const double2 *__restrict__ ab, const int32_t *__restrict__ work,
                                                   int work_begin, int work_count, tod_rng rng, int mode,
                                                   double *g_out, double *mu_out, double *sig_out, int32_t *status)
{
    const int w = blockIdx.x * blockDim.x + threadIdx.x;
    if (w >= work_count) return;
    const int q = work[work_begin + w];
    const double A = ab[q].x, B = ab[q].y;
    if (!(A > 0.0)) {
        set_status(status, q, TOD_ERR_ARG);
        g_out[q] = 0.0;
        if (mu_out) mu_out[q] = 0.0;
        if (sig_out) sig_out[q] = 0.0;
        return;
    }
    const double mu = B / A, sg = 1.0 / sqrt(A);
    double z = 0.0;
    if (mode == TOD_MODE_DRAW) {
        const uint64_t it = rng.gibbs_iter_dev ? *rng.gibbs_iter_dev : rng.gibbs_iter;
        const u64x4 wv = philox4x64(0, static_cast<uint64_t>(q), 0, it, rng.seed, rng.band);
        const double u1 = (static_cast<double>(wv.x[0] >> 11) + 0.5) * 1.1102230246251565e-16;
        const double u2 = (static_cast<double>(wv.x[1] >> 11) + 0.5) * 1.1102230246251565e-16;
        z = sqrt(-2.0 * log(u1)) * cospi(2.0 * u2);
    }
    g_out[q] = mu + z * sg;
    if (mu_out) mu_out[q] = mu;
    if (sig_out) sig_out[q] = sg;
}

// ---------------------------------------------------------------------------
// A5: correlated noise.  x0 = B^{-1} b (B = C^T diag(phi + 1/sigma0^2) C)
// is the draw of a gap-free detscan; flagged detscans then solve the Schur
// complement
//   S y = E^T x0,  S = sigma0^2 I - E^T B^{-1} E = E^T C^T diag(gamma) C E
// (E: flagged samples; C^T C = I) by CG and add B^{-1} E y (Woodbury):
// x = A^{-1} b exactly, A = B - E E^T / sigma0^2.
// ---------------------------------------------------------------------------
// Exclusive scan of one int3 per thread over the CTA (warp shuffles, then
// the warp totals); total gets the CTA-wide sum.  s_w holds DCT_T/32 + 1.
__device__ int3 block_exscan3(int3 v, int3 *s_w, int3 &total)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int3 inc = v;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const int x = __shfl_up_sync(0xffffffffu, inc.x, d);
        const int y = __shfl_up_sync(0xffffffffu, inc.y, d);
        const int z = __shfl_up_sync(0xffffffffu, inc.z, d);
        if (lane >= d) { inc.x += x; inc.y += y; inc.z += z; }
    }
    if (lane == 31) s_w[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        constexpr int NW = DCT_T / 32;
        const int3 w = lane < NW ? s_w[lane] : make_int3(0, 0, 0);
        int3 wi = w;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const int x = __shfl_up_sync(0xffffffffu, wi.x, d);
            const int y = __shfl_up_sync(0xffffffffu, wi.y, d);
            const int z = __shfl_up_sync(0xffffffffu, wi.z, d);
            if (lane >= d) { wi.x += x; wi.y += y; wi.z += z; }
        }
        __syncwarp();
        if (lane < NW) s_w[lane] = make_int3(wi.x - w.x, wi.y - w.y, wi.z - w.z);
        if (lane == NW - 1) s_w[NW] = wi;
    }
    __syncthreads();
    const int3 b = s_w[warp];
    total = s_w[DCT_T / 32];
    __syncthreads();       // s_w may be reused after this
    return make_int3(b.x + inc.x - v.x, b.y + inc.y - v.y, b.z + inc.z - v.z);
}

// Own gap blocks of the preconditioner, applied in rounds of at most GB_CAP
// padded elements (see the own-block set-up in k_ncorr).
struct OwnBlocks {
    int len[GAP_CAP], rank[GAP_CAP], off[GAP_CAP], q[GAP_CAP];
    int rnd[GAP_CAP + 1];
    int nrnd;
};

// Thread 0: split the detscan's gaps into blocks of at most lmax samples
// (each with the rank of its first flagged sample); then each block, longest
// first, goes to the CTA with the least work so far (a block's cost grows as
// len^2: triangular Toeplitz products), the lowest rank on ties.  Every CTA
// makes the same assignment, with no exchange.  Fills this CTA's own blocks
// (applied in rounds of at most GB_CAP floats: 8 zeros, the block padded to
// a multiple of 4, 8 zeros); returns the number of blocks (more than
// GAP_CAP: nothing assigned).  Out of line: its registers stay out of the
// kernel's.
__device__ __noinline__ int assign_gap_blocks(OwnBlocks &ob, int &nown, const int *g_beg, const int *g_end, int ngap,
                                              int lmax, int C, int c, int *blen, int *brank, int *bord)
{
    int nb = 0, rank = 0;
    for (int g2 = 0; g2 < ngap; ++g2) {
        for (int b0 = g_beg[g2]; b0 < g_end[g2]; b0 += lmax) {
            const int len = min(lmax, g_end[g2] - b0);
            if (nb < GAP_CAP) { blen[nb] = len; brank[nb] = rank; }
            rank += len;
            ++nb;
        }
    }
    if (nb <= GAP_CAP) {
        for (int i = 0; i < nb; ++i) {            // indices by decreasing length (stable)
            int j = i;
            while (j > 0 && blen[bord[j - 1]] < blen[i]) { bord[j] = bord[j - 1]; --j; }
            bord[j] = i;
        }
        long long load[16];
        for (int r = 0; r < C; ++r) load[r] = 0;
        int rlen = 0, rq = 0;
        for (int i = 0; i < nb; ++i) {
            const int bi = bord[i], len = blen[bi];
            int best = 0;
            for (int r = 1; r < C; ++r)
                if (load[r] < load[best]) best = r;
            load[best] += static_cast<long long>(len) * len;
            if (best != c) continue;
            const int reg = ((len + 3) & ~3) + 16;
            if (nown == 0 || rlen + reg > GB_CAP) { ob.rnd[ob.nrnd++] = nown; rlen = 0; rq = 0; }
            ob.len[nown] = len; ob.rank[nown] = brank[bi]; ob.off[nown] = rlen; ob.q[nown] = rq;
            ++nown;
            rlen += reg;
            rq += (len + 3) >> 2;
        }
    }
    ob.rnd[ob.nrnd] = nown;
    return nb;
}

// CG vector element of global rank k: (CTA k / kper, index k mod kper)
__device__ __forceinline__ float *rank_elem(cg::cluster_group &cl, float *vec, int kper, int k) {
    const int ow = k / kper;
    return cl.map_shared_rank(vec + (k - ow * kper), ow);
}

// Right-hand side of the n_corr system, time-domain part, M (r/s2 + w1/s)
// with r = d - g s, into the time layout of U.  Element j takes normals 2j,
// 2j+1 (pair j mod 4 of Philox block j/4 of stream 1): one thread draws a
// block for four consecutive elements of a row.
__device__ __noinline__ void ncorr_rhs(const Ctx &XS, float2 *__restrict__ U, const float *__restrict__ dq,
                                       const float *__restrict__ sq, const uint32_t *__restrict__ fl, int64_t o,
                                       float g, float inv_s2, float inv_s, bool draw, uint64_t q, uint64_t gi,
                                       uint64_t seed, uint64_t band)
{
    const Geo X = XS;
    const int n = X.n, m = X.m;
    const int ncol = X.ncol, nbr = (ncol + 3) / 4 + 1;     // blocks touching a row
    const int items = X.m1 * nbr;
    for (int w = threadIdx.x; w < items; w += DCT_T) {
        const int j1 = w / nbr, bi = w - j1 * nbr;
        const int js = j1 * X.m2 + X.c * X.ncolmax;          // first element of the row
        const int b = (js >> 2) + bi;
        if (4 * b >= js + ncol) continue;
        u64x4 rw;
        if (draw) rw = philox4x64(static_cast<uint64_t>(b), q, 1, gi, seed, band);
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int j = 4 * b + u;
            if (j < js || j >= js + ncol) continue;
            const int t0 = vpos_t(2 * j, n, m), t1 = vpos_t(2 * j + 1, n, m);
            const float2 w1 = draw ? philox_normal_pair(rw, u) : make_float2(0.f, 0.f);
            const float d0 = __ldg(dq + t0), d1 = __ldg(dq + t1);
            const float s0v = __ldg(sq + t0), s1v = __ldg(sq + t1);
            const float r0 = flagged(fl, o + t0) ? 0.f : fmaf(d0 - g * s0v, inv_s2, w1.x * inv_s);
            const float r1 = flagged(fl, o + t1) ? 0.f : fmaf(d1 - g * s1v, inv_s2, w1.y * inv_s);
            U[j1 * X.ncolmax + (j - js)] = make_float2(r0, r1);
        }
    }
    // padding columns of the last CTA stay zero
    for (int e = threadIdx.x; e < X.m1 * X.ncolmax; e += DCT_T) {
        const int j1 = fdiv(e, X.f_ncolmax);
        if (e - j1 * X.ncolmax >= ncol) U[e] = make_float2(0.f, 0.f);
    }
    __syncthreads();
}

// Per packed slot of this CTA: the filter weights (beta_a, beta_b, gamma_a,
// gamma_b) of its two modes into wt, and the prior term sqrt(phi) w2 into
// nu (zero when not drawing).  Mode k takes normals 2k, 2k+1 (pair k mod 4
// of block k/4 of stream 2); for a fixed k2 the own even slots hold
// k = p0 + pl + m1 k2 and the odd ones k = m1 - p0 - pl + m1 k2 (pl < npl),
// so one thread draws a block for up to four consecutive modes of a parity.
__device__ __noinline__ void ncorr_weights(const Ctx &XS, float2 *__restrict__ nu_out, float4 *__restrict__ wt,
                                           float fscale, float alpha, float s2, float inv_s2, bool draw,
                                           uint64_t q, uint64_t gi, uint64_t seed, uint64_t band)
{
    const Geo X = XS;
    const int n = X.n, m = X.m;
    const int npl = X.npl, m1 = X.m1, m2 = X.m2, p0 = X.p0;
    const int nbk = (npl + 3) / 4 + 1;                  // blocks touching a k range
    const int items = 2 * nbk * m2;
    for (int w = threadIdx.x; w < items; w += DCT_T) {
        const int rest = fdiv(w, X.f_m2), k2 = w - rest * m2;
        const int par = rest / nbk, bi = rest - par * nbk;
        const int kbase = (par == 0 ? p0 : m1 - p0 - (npl - 1)) + m1 * k2;
        const int b = (kbase >> 2) + bi;
        if (npl <= 0 || 4 * b >= kbase + npl) continue;
        u64x4 rw;
        if (draw) rw = philox4x64(static_cast<uint64_t>(b), q, 2, gi, seed, band);
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int k = 4 * b + u;
            if (k < kbase || k >= kbase + npl) continue;
            const int pl = par == 0 ? k - kbase : (npl - 1) - (k - kbase);
            const int p = p0 + pl;
            const int e = (2 * pl + par) * X.m2p + k2;
            if (par == 1 && (p == 0 || m1 - p == p)) {            // slot holds no modes
                wt[e] = make_float4(0.f, 0.f, 0.f, 0.f);
                nu_out[e] = make_float2(0.f, 0.f);
                continue;
            }
            const int ka = k, kb = (k == 0) ? m : n - k;
            const float ra = (ka == 0) ? 0.f : fratio_pow(ka, fscale, -alpha);   // s2 phi
            const float rb = fratio_pow(kb, fscale, -alpha);
            const float ba = s2 / (1.0f + ra), bb = s2 / (1.0f + rb);
            wt[e] = make_float4(ba, bb, ra * ba, rb * bb);
            float2 nu = make_float2(0.f, 0.f);
            if (draw) {
                const float2 w2 = philox_normal_pair(rw, u);
                nu = make_float2(sqrtf(ra * inv_s2) * w2.x, sqrtf(rb * inv_s2) * w2.y);
            }
            nu_out[e] = nu;
        }
    }
    __syncthreads();
}

// element i of this CTA's CG vectors: its sample's value in the transform
// buffer U of CTA (c_loc[i] >> 20), element c_loc[i] & 0xFFFFF (as floats)
__device__ __forceinline__ float *cg_elem(cg::cluster_group &cl, float2 *U, const int *c_loc, int i) {
    const int cli = c_loc[i];
    return cl.map_shared_rank(reinterpret_cast<float *>(U) + (cli & 0xFFFFF), cli >> 20);
}

// z = M^{-1} r with M the block-diagonal Toeplitz preconditioner: each own
// block applies T_L^{-1} = (L(x) L(x)^T - L(w) L(w)^T) / x_0 (Gohberg-
// Semencul; x = T_L^{-1} e_1 from the Durbin tables, w = (0, x_{L-1}, ..,
// x_1)) to its slice of r, gathered from and scattered to the CTAs that
// hold those ranks.  gb points at five GB_CAP float arrays.  The CG sums
// that need z ride on the closing cluster barrier: this CTA publishes
// (rr_part, sum of r z over its own blocks) as its slot of a cluster sum,
// which the caller collects.  With clear non-null, clear[0, nclear) is
// zeroed once the opening barrier has ended every earlier remote read.
__device__ __noinline__ void apply_gap_precond(const OwnBlocks &ob, float *c_r, float *c_z, float *gb,
                                               const float *__restrict__ xt_det, int kper,
                                               cg::cluster_group &cl, Acc2 rr_part, double2 *s_red,
                                               double2 *s_part, int parity, float2 *clear, int nclear)
{
    float *gb_r = gb, *gb_x = gb + GB_CAP, *gb_w = gb + 2 * GB_CAP;
    float *gb_u1 = gb + 3 * GB_CAP, *gb_u2 = gb + 4 * GB_CAP;
    Acc2 rz = {0.f, 0.f};
    cl.sync();     // every CTA's residual is complete before the gathers
    if (clear)
        for (int e = threadIdx.x; e < nclear; e += DCT_T) clear[e] = make_float2(0.f, 0.f);
    for (int rd = 0; rd < ob.nrnd; ++rd) {
        const int b0 = ob.rnd[rd], b1 = ob.rnd[rd + 1];
        const int Ll = ob.len[b1 - 1];
        const int tot = ob.off[b1 - 1] + ((Ll + 3) & ~3) + 16;
        const int totq = ob.q[b1 - 1] + ((Ll + 3) >> 2);
        // gather r and each block's generator x (w_s = x_{L-s}, w_0 = 0)
        // into zero-padded regions; u1, u2 start at zero
        for (int f = threadIdx.x; f < tot; f += DCT_T) {
            int b = b0;
            while (b + 1 < b1 && ob.off[b + 1] <= f) ++b;
            const int L = ob.len[b], li = f - ob.off[b] - 8;
            float rv = 0.f, xv = 0.f, wv = 0.f;
            if (li >= 0 && li < L) {
                const float *xt = xt_det + static_cast<int64_t>(L) * (L - 1) / 2;
                rv = *rank_elem(cl, c_r, kper, ob.rank[b] + li);
                xv = xt[li];
                wv = li == 0 ? 0.f : xt[L - li];
            }
            gb_r[f] = rv; gb_x[f] = xv; gb_w[f] = wv; gb_u1[f] = 0.f; gb_u2[f] = 0.f;
        }
        __syncthreads();
        // u1 = L(x)^T r, u2 = L(w)^T r: four outputs i0..i0+3 per group of
        // QT consecutive threads (QT = 4, 2 or 1 as the round's size allows),
        // float4 loads; the group splits the sum and adds its partials in a
        // fixed order
        const int QT = (totq * 4 <= DCT_T) ? 4 : (totq * 2 <= DCT_T) ? 2 : 1;
        const int qsh = QT == 4 ? 2 : QT == 2 ? 1 : 0;
        const int totw = totq << qsh;
        for (int t0 = 0; t0 < totw; t0 += DCT_T) {
            const int t = t0 + threadIdx.x;
            const bool act = t < totw;
            const int qi = t >> qsh, part = t & (QT - 1);
            float4 a1 = make_float4(0.f, 0.f, 0.f, 0.f), a2 = a1;
            int base = 0, i0 = 0;
            if (act) {
                int b = b0;
                while (b + 1 < b1 && ob.q[b + 1] <= qi) ++b;
                const int L = ob.len[b];
                i0 = 4 * (qi - ob.q[b]);
                base = ob.off[b] + 8;
                const float *xb = gb_x + base, *wb = gb_w + base, *rb = gb_r + base + i0;
                for (int k = 4 * part; k < L - i0; k += 4 * QT) {
                    const float4 xk = *reinterpret_cast<const float4 *>(xb + k);
                    const float4 wk = *reinterpret_cast<const float4 *>(wb + k);
                    const float4 rc = *reinterpret_cast<const float4 *>(rb + k);
                    const float4 rn = *reinterpret_cast<const float4 *>(rb + k + 4);
                    a1.x = fmaf(xk.x, rc.x, fmaf(xk.y, rc.y, fmaf(xk.z, rc.z, fmaf(xk.w, rc.w, a1.x))));
                    a1.y = fmaf(xk.x, rc.y, fmaf(xk.y, rc.z, fmaf(xk.z, rc.w, fmaf(xk.w, rn.x, a1.y))));
                    a1.z = fmaf(xk.x, rc.z, fmaf(xk.y, rc.w, fmaf(xk.z, rn.x, fmaf(xk.w, rn.y, a1.z))));
                    a1.w = fmaf(xk.x, rc.w, fmaf(xk.y, rn.x, fmaf(xk.z, rn.y, fmaf(xk.w, rn.z, a1.w))));
                    a2.x = fmaf(wk.x, rc.x, fmaf(wk.y, rc.y, fmaf(wk.z, rc.z, fmaf(wk.w, rc.w, a2.x))));
                    a2.y = fmaf(wk.x, rc.y, fmaf(wk.y, rc.z, fmaf(wk.z, rc.w, fmaf(wk.w, rn.x, a2.y))));
                    a2.z = fmaf(wk.x, rc.z, fmaf(wk.y, rc.w, fmaf(wk.z, rn.x, fmaf(wk.w, rn.y, a2.z))));
                    a2.w = fmaf(wk.x, rc.w, fmaf(wk.y, rn.x, fmaf(wk.z, rn.y, fmaf(wk.w, rn.z, a2.w))));
                }
            }
            for (int ofs = 1; ofs < QT; ofs <<= 1) {       // every lane of the warp takes part
                a1.x += __shfl_xor_sync(0xffffffffu, a1.x, ofs); a1.y += __shfl_xor_sync(0xffffffffu, a1.y, ofs);
                a1.z += __shfl_xor_sync(0xffffffffu, a1.z, ofs); a1.w += __shfl_xor_sync(0xffffffffu, a1.w, ofs);
                a2.x += __shfl_xor_sync(0xffffffffu, a2.x, ofs); a2.y += __shfl_xor_sync(0xffffffffu, a2.y, ofs);
                a2.z += __shfl_xor_sync(0xffffffffu, a2.z, ofs); a2.w += __shfl_xor_sync(0xffffffffu, a2.w, ofs);
            }
            if (act && part == 0) {
                *reinterpret_cast<float4 *>(gb_u1 + base + i0) = a1;
                *reinterpret_cast<float4 *>(gb_u2 + base + i0) = a2;
            }
        }
        __syncthreads();
        // z = (L(x) u1 - L(w) u2) / x_0, scattered to the owners; same split
        for (int t0 = 0; t0 < totw; t0 += DCT_T) {
            const int t = t0 + threadIdx.x;
            const bool act = t < totw;
            const int qi = t >> qsh, part = t & (QT - 1);
            float4 z1 = make_float4(0.f, 0.f, 0.f, 0.f), z2 = z1;
            int b = b0, i0 = 0, L = 0, base = 0;
            if (act) {
                while (b + 1 < b1 && ob.q[b + 1] <= qi) ++b;
                L = ob.len[b];
                i0 = 4 * (qi - ob.q[b]);
                base = ob.off[b] + 8;
                const float *xb = gb_x + base, *wb = gb_w + base;
                const float *u1b = gb_u1 + base + i0, *u2b = gb_u2 + base + i0;
                for (int s0 = 4 * part; s0 <= i0; s0 += 4 * QT) {
                    const float4 xs = *reinterpret_cast<const float4 *>(xb + s0);
                    const float4 ws = *reinterpret_cast<const float4 *>(wb + s0);
                    const float4 ua = *reinterpret_cast<const float4 *>(u1b - s0);      // u[i0 - s0 ..]
                    const float4 va = *reinterpret_cast<const float4 *>(u2b - s0);
                    const float4 ub = *reinterpret_cast<const float4 *>(u1b - s0 - 4);
                    const float4 vb = *reinterpret_cast<const float4 *>(u2b - s0 - 4);
                    z1.x = fmaf(xs.x, ua.x, fmaf(xs.y, ub.w, fmaf(xs.z, ub.z, fmaf(xs.w, ub.y, z1.x))));
                    z1.y = fmaf(xs.x, ua.y, fmaf(xs.y, ua.x, fmaf(xs.z, ub.w, fmaf(xs.w, ub.z, z1.y))));
                    z1.z = fmaf(xs.x, ua.z, fmaf(xs.y, ua.y, fmaf(xs.z, ua.x, fmaf(xs.w, ub.w, z1.z))));
                    z1.w = fmaf(xs.x, ua.w, fmaf(xs.y, ua.z, fmaf(xs.z, ua.y, fmaf(xs.w, ua.x, z1.w))));
                    z2.x = fmaf(ws.x, va.x, fmaf(ws.y, vb.w, fmaf(ws.z, vb.z, fmaf(ws.w, vb.y, z2.x))));
                    z2.y = fmaf(ws.x, va.y, fmaf(ws.y, va.x, fmaf(ws.z, vb.w, fmaf(ws.w, vb.z, z2.y))));
                    z2.z = fmaf(ws.x, va.z, fmaf(ws.y, va.y, fmaf(ws.z, va.x, fmaf(ws.w, vb.w, z2.z))));
                    z2.w = fmaf(ws.x, va.w, fmaf(ws.y, va.z, fmaf(ws.z, va.y, fmaf(ws.w, va.x, z2.w))));
                }
            }
            for (int ofs = 1; ofs < QT; ofs <<= 1) {
                z1.x += __shfl_xor_sync(0xffffffffu, z1.x, ofs); z1.y += __shfl_xor_sync(0xffffffffu, z1.y, ofs);
                z1.z += __shfl_xor_sync(0xffffffffu, z1.z, ofs); z1.w += __shfl_xor_sync(0xffffffffu, z1.w, ofs);
                z2.x += __shfl_xor_sync(0xffffffffu, z2.x, ofs); z2.y += __shfl_xor_sync(0xffffffffu, z2.y, ofs);
                z2.z += __shfl_xor_sync(0xffffffffu, z2.z, ofs); z2.w += __shfl_xor_sync(0xffffffffu, z2.w, ofs);
            }
            if (act && part == 0) {
                const float inv = 1.0f / gb_x[base];
                const float zz[4] = {z1.x - z2.x, z1.y - z2.y, z1.z - z2.z, z1.w - z2.w};
#pragma unroll
                for (int j = 0; j < 4; ++j)
                    if (i0 + j < L) {
                        const float zj = zz[j] * inv;
                        *rank_elem(cl, c_z, kper, ob.rank[b] + i0 + j) = zj;
                        acc_add_prod(rz, gb_r[base + i0 + j], zj);
                    }
            }
        }
        __syncthreads();     // the gb arrays are reused by the next round
    }
    cluster_sum_publish(rr_part, rz, s_red, s_part, parity);
    cl.sync();     // every scatter into every CTA's c_z is done, and every slot is published
}

// The orthonormal DCT-II coefficients of this CTA's modes of the draw,
// diag(beta) (acc.xy + alp acc.zw), into spec in mode order (spec[k], k of
// the detscan); out of line, for callers that asked for the spectra.
__device__ __noinline__ void write_spectrum(const Ctx &XS, float *__restrict__ spec, const float4 *acc,
                                            const float4 *wt, float alp)
{
    const Geo X = XS;
    const int n = X.n, m = X.m, m2 = X.m2, m2p = X.m2p, m1 = X.m1, p0 = X.p0;
    const int total = X.npl * m2;
    for (int e = threadIdx.x; e < total; e += DCT_T) {
        const int pl = fdiv(e, X.f_m2), k2 = e - pl * m2;
        const int p = p0 + pl;
        const int cnt = (p == 0) ? (m2 / 2 + 1) : ((2 * p == m1) ? (m2 + 1) / 2 : m2);
        if (k2 >= cnt) continue;
        int ib, q1, q2;
        if (p == 0) { q1 = 0; q2 = (k2 == 0) ? 0 : m2 - k2; ib = 2 * pl * m2p + q2; }
        else { q1 = m1 - p; q2 = m2 - 1 - k2; ib = ((q1 == p) ? 2 * pl : 2 * pl + 1) * m2p + q2; }
        const int ia = 2 * pl * m2p + k2;
        const int ka = p + m1 * k2, kb = q1 + m1 * q2;
        {
            const float4 A = acc[ia], w = wt[ia];
            spec[ka] = fmaf(alp, A.z, A.x) * w.x;
            spec[ka == 0 ? m : n - ka] = fmaf(alp, A.w, A.y) * w.y;
        }
        if (ib != ia && !(p == 0 && k2 == 0)) {
            const float4 A = acc[ib], w = wt[ib];
            spec[kb] = fmaf(alp, A.z, A.x) * w.x;
            spec[n - kb] = fmaf(alp, A.w, A.y) * w.y;
        }
    }
}

struct NcorrArgs {
    const float *d, *s;
    const double *gain;
    const uint32_t *flags;
    const double *psd;
    const int64_t *off;
    const DctPlan *plans;
    const int32_t *q_plan;
    const float2 *tw;
    const int32_t *work;
    int work_begin, work_count;
    int ndet;
    double fsamp;
    tod_rng rng;
    int mode;
    float tol;
    int maxit;
    float *x_out;
    int32_t *iters;
    int32_t *status;
    float4 *wscratch;
    float *spec_out;          // spectra of the draws in mode order (NULL: not written)
    const float *xtab;       // Toeplitz inverses' first columns per detector (NULL: no preconditioner)
    const int32_t *lvalid;
    int sz, m1max, m2max, twsz;
};

__global__ void __launch_bounds__(DCT_T, 1) k_ncorr(NcorrArgs a)
{
    extern __shared__ __align__(16) float2 smem_raw[];
    __shared__ Ctx sX;
    __shared__ DetScal s_sc;
    __shared__ double2 s_red[DCT_T / 32 + 1];
    __shared__ double2 s_part[2];
    __shared__ int3 s_wscan[DCT_T / 32 + 1];
    __shared__ int s_nown, s_ovf;
    __shared__ int g_beg[GAP_CAP], g_end[GAP_CAP];
    __shared__ int s_blen[GAP_CAP], s_brank[GAP_CAP], s_bord[GAP_CAP];   // gap blocks (thread 0)
    __shared__ OwnBlocks ob;
    cg::cluster_group cl = cg::this_cluster();
    const int C = static_cast<int>(cl.num_blocks()), c = static_cast<int>(cl.block_rank());
    const int cid = blockIdx.x / C, ncl = gridDim.x / C;
    Smem sm = carve(smem_raw, a.sz, a.twsz);
    // CG vectors and preconditioner work areas after the two buffers
    int *c_loc = reinterpret_cast<int *>(sm.tail);
    float *c_y = reinterpret_cast<float *>(c_loc + CG_KCAP);
    float *c_r = c_y + CG_KCAP;
    float *c_p = c_r + CG_KCAP;
    float *c_q = c_p + CG_KCAP;
    float *c_z = c_q + CG_KCAP;
    float *gb_r = c_z + CG_KCAP;        // five GB_CAP arrays of the preconditioner
    int parity = 0;
    int cur_pi = -1;      // plan staged in shared memory
    for (int w = cid; w < a.work_count; w += ncl) {
        const int q = a.work[a.work_begin + w];
        const int det = q % a.ndet;
        const int64_t o = a.off[q];
        load_plan(&sX, a.plans, a.q_plan[q], a.tw, sm, c, C, cur_pi);
        if (threadIdx.x == 0) { s_nown = 0; ob.nrnd = 0; }
        const Ctx &X = sX;     // read from shared memory: registers are scarce here
        const int n = X.n, m = X.m;
        const DetScal sc = det_scalars(&s_sc, a.psd, det, n, a.fsamp, a.gain, q);
        const float fscale = sc.fscale, alpha = sc.alpha, s2 = sc.s2;
        const float inv_s2 = sc.inv_s2, inv_s = sc.inv_s, g = sc.g;
        const bool draw = a.mode == TOD_MODE_DRAW;
        const float *dq = a.d + o, *sq = a.s + o;
        const uint32_t *fl = a.flags;
        const tod_rng rng = a.rng;
        const uint64_t gi = rng.gibbs_iter_dev ? *rng.gibbs_iter_dev : rng.gibbs_iter;
        float *xq = a.x_out + o;
        // per-CTA scratch: filter weights, then the CG spectral accumulators
        float4 *wt = a.wscratch + (static_cast<int64_t>(cid) * C + c) * (NCORR_SCRATCH_F4 * a.sz);
        float4 *acc = wt + a.sz;
        float2 *cur = sm.U0, *oth = sm.U1;
        // right-hand side, time-domain part: M (r/s2 + w1/s)
        ncorr_rhs(sX, cur, dq, sq, fl, o, g, inv_s2, inv_s, draw, q, gi, rng.seed, rng.band);
        if (dct_forward_pre(sX, cur, oth, cl)) { float2 *t_ = cur; cur = oth; oth = t_; }
        // prior term sqrt(phi) w2 in the packed layout into the free buffer
        // oth, filter weights of this detscan into wt
        ncorr_weights(sX, oth, wt, fscale, alpha, s2, inv_s2, draw, q, gi, rng.seed, rng.band);
        // (C b + prior term) times beta, between the two halves of the split
        split_roundtrip(X, cur, [&](int e, int, float2 Y) {
            const float4 w = wt[e];
            const float2 nu = oth[e];
            const float2 cb = make_float2(Y.x + nu.x, Y.y + nu.y);
            acc[e] = make_float4(cb.x, cb.y, 0.f, 0.f);       // x0 = C^T diag(beta) cb
            return make_float2(cb.x * w.x, cb.y * w.y);
        });

        if (dct_inverse_post(sX, cur, oth, cl)) { float2 *t_ = cur; cur = oth; oth = t_; }      // cur = x0 (time layout)
        // Flagged samples of the detscan, ranked in time order.  The CG
        // vectors are spread evenly over the cluster: CTA c holds ranks
        // [c kper, (c+1) kper), each entry with the (owner CTA, element) of
        // its sample in the transform layout (E and E^T go through DSMEM).
        // Gaps (runs of flagged samples) are listed in time order.
        const int64_t wb0 = o >> 5, wb1 = (o + n - 1) >> 5;
        const int nw = static_cast<int>(wb1 - wb0 + 1);
        const int per = (nw + DCT_T - 1) / DCT_T;
        // bits of word wi restricted to this detscan
        auto word_bits = [&](int wi) -> uint32_t {
            if (wi < 0 || wi >= nw) return 0u;
            uint32_t bits = fl[wb0 + wi];
            const int64_t base = ((wb0 + wi) << 5) - o;             // sample of bit 0
            if (base < 0) bits &= ~0u << static_cast<int>(-base);
            if (base + 32 > n) bits &= (n - base >= 32) ? ~0u : ((1u << static_cast<int>(n - base)) - 1u);
            return bits;
        };
        // per-word flagged counts, then their exclusive prefix, in the free
        // transform buffer (oth: nothing reads it until the CG scatters)
        int *wpre = reinterpret_cast<int *>(oth);
        int3 mine = make_int3(0, 0, 0);     // flagged samples, gap starts, gap ends
        for (int i = 0; i < per; ++i) {
            const int wi = threadIdx.x * per + i;
            if (wi >= nw) break;
            const uint32_t bits = word_bits(wi);
            const uint32_t prev = word_bits(wi - 1) >> 31;
            const uint32_t next = word_bits(wi + 1) & 1u;
            wpre[wi] = __popc(bits);
            mine.x += __popc(bits);
            mine.y += __popc(bits & ~((bits << 1) | prev));
            mine.z += __popc(bits & ~((bits >> 1) | (next << 31)));
        }
        int3 tot3;
        const int3 ex = block_exscan3(mine, s_wscan, tot3);
        const int kc_all = tot3.x, ngap = tot3.y;
        const int kper = (kc_all + C - 1) / C;
        const int k0 = min(kc_all, c * kper);
        const int kc = min(kc_all, k0 + kper) - k0;     // entries held by this CTA
        const bool cap_ovf = kper > CG_KCAP;
        if (kc_all == 0 || cap_ovf) {
            // x = x0 (no flagged sample, or too many for the CG buffers)
            const int tot = X.m1 * X.ncolmax;
            for (int e = threadIdx.x; e < tot; e += DCT_T) {
                int t0, t1;
                bool valid;
                elem_samples(X, e, t0, t1, valid);
                if (!valid) continue;
                const float2 v = cur[e];
                xq[t0] = v.x;
                xq[t1] = v.y;
            }
        }
        {
            int pos = ex.x, gpos = ex.y, epos = ex.z;
            for (int i = 0; i < per; ++i) {
                const int wi = threadIdx.x * per + i;
                if (wi >= nw) break;
                const uint32_t bits = word_bits(wi);
                const uint32_t prev = word_bits(wi - 1) >> 31;
                const uint32_t next = word_bits(wi + 1) & 1u;
                uint32_t st = bits & ~((bits << 1) | prev);
                uint32_t en = bits & ~((bits >> 1) | (next << 31));
                const int64_t base = ((wb0 + wi) << 5) - o;
                while (st) {
                    const int b = __popc((st & (0u - st)) - 1u);     // index of the lowest set bit
                    st &= st - 1;
                    if (gpos < GAP_CAP) g_beg[gpos] = static_cast<int>(base + b);
                    ++gpos;
                }
                while (en) {
                    const int b = __popc((en & (0u - en)) - 1u);
                    en &= en - 1;
                    if (epos < GAP_CAP) g_end[epos] = static_cast<int>(base + b + 1);
                    ++epos;
                }
                const int cnt = wpre[wi];
                wpre[wi] = pos;
                pos += cnt;
            }
        }
        __syncthreads();
        // own ranks [k0, k0 + kc): the word holding rank k is the last one whose
        // prefix is <= k (a word without flags shares its prefix with the next)
        if (!cap_ovf) {
            for (int k = k0 + threadIdx.x; k < k0 + kc; k += DCT_T) {
                int lo = 0, hi = nw - 1;
                while (lo < hi) {
                    const int mid = (lo + hi + 1) >> 1;
                    if (wpre[mid] <= k) lo = mid; else hi = mid - 1;
                }
                uint32_t bits = word_bits(lo);
                for (int r = k - wpre[lo]; r > 0; --r) bits &= bits - 1;
                const int b = __popc((bits & (0u - bits)) - 1u);
                int ow, loc;
                sample_loc(X, static_cast<int>(((wb0 + lo) << 5) - o + b), ow, loc);
                c_loc[k - k0] = (ow << 20) | loc;
            }
        }
        __syncthreads();
        // a gap that starts in one thread's words and ends in another's is
        // matched by index: starts and ends alternate in sample order
        const bool prec = a.xtab != nullptr && ngap <= GAP_CAP;
        if (prec && threadIdx.x == 0) {
            const int lmax = max(1, min(TOEP_LMAX, a.lvalid[det]));
            const int nb = assign_gap_blocks(ob, s_nown, g_beg, g_end, ngap, lmax, C, c, s_blen, s_brank, s_bord);
            s_ovf = nb > GAP_CAP;      // the same in every CTA
        }
        if (!prec && threadIdx.x == 0) s_ovf = 1;
        __syncthreads();
        const bool use_prec = s_ovf == 0;
        int it = 0;
        bool conv = true;
        float alp_spec = 0.f;      // the draw's spectrum is diag(beta) (acc.xy + alp_spec acc.zw)
        if (kc_all > 0 && cap_ovf) {
            conv = false;      // too many flagged samples for the CG buffers: left as x0
            set_status(a.status, q, TOD_ERR_NOT_CONVERGED);
        } else if (kc_all > 0) {
            const float *xt_det = a.xtab ? a.xtab + static_cast<int64_t>(det) * (TOEP_LMAX * (TOEP_LMAX + 1) / 2)
                                         : nullptr;
            // z = M^{-1} r (Gohberg-Semencul per own block, scattered to
            // owners) and the cluster sums (rr_part summed, r.z): returns
            // (sum rr_part, sum r z) with z complete in every CTA
            // With clear non-null, the transform buffer is zeroed after every
            // earlier remote read of it and before the closing barrier.
            const int tot = X.m1 * X.ncolmax;
            auto precond = [&](Acc2 rr_part, float2 *clear) -> double2 {
                if (!use_prec) {
                    Acc2 rz_loc = {0.f, 0.f};
                    for (int i = threadIdx.x; i < kc; i += DCT_T) {
                        c_z[i] = c_r[i];
                        acc_add_prod(rz_loc, c_r[i], c_r[i]);
                    }
                    if (clear) {
                        cl.sync();
                        for (int e = threadIdx.x; e < tot; e += DCT_T) clear[e] = make_float2(0.f, 0.f);
                    }
                    return cluster_sum_acc(rr_part, rz_loc, s_red, s_part, parity, cl);
                }
                apply_gap_precond(ob, c_r, c_z, gb_r, xt_det, kper, cl, rr_part, s_red, s_part, parity, clear, tot);
                return cluster_sum_collect(s_red, s_part, parity, cl);
            };
            // rhs = E^T x0 ; y = 0 ; r = rhs ; z = M^{-1} r ; p = z
            cl.sync();         // x0 is complete in every CTA before the gathers
            Acc2 rr_loc = {0.f, 0.f};
            for (int i = threadIdx.x; i < kc; i += DCT_T) {
                const float v = *cg_elem(cl, cur, c_loc, i);
                c_r[i] = v;
                acc_add_prod(rr_loc, v, v);
            }
            __syncthreads();
            // z = M^{-1} r, (r.r, r.z); x0's buffer is cleared for the first scatter
            const double2 rr2 = precond(rr_loc, cur);
            for (int i = threadIdx.x; i < kc; i += DCT_T) c_p[i] = c_z[i];
            double rz = rr2.y;
            const double stop = static_cast<double>(a.tol) * a.tol * rr2.x;
            conv = rr2.x == 0.0;
            // y = sum_i alpha_i p_i is never formed: x = x0 + B^{-1} E y
            // = C^T diag(beta) (cb + sum_i alpha_i C E p_i), with cb the
            // spectrum of x0 before the filter and C E p_i the spectra the
            // iterations compute anyway, accumulated per packed slot in acc
            // (x, y: cb plus the sum so far; z, w: the latest spectrum, whose
            // step length is known one iteration later)
            float alp_prev = 0.f;
            while (!conv && it < a.maxit) {
                // cur <- C^T diag(gamma) C E p (cur is zero in every CTA)
                for (int i = threadIdx.x; i < kc; i += DCT_T) *cg_elem(cl, cur, c_loc, i) = c_p[i];
                cl.sync();     // every scatter has landed
                if (dct_forward_pre(sX, cur, oth, cl)) { float2 *t_ = cur; cur = oth; oth = t_; }
                split_roundtrip(X, cur, [&](int e, int, float2 Y) {
                    const float4 w = wt[e];
                    const float4 A = acc[e];          // (z, w) = 0 and alp_prev = 0 at the first
                    acc[e] = make_float4(fmaf(alp_prev, A.z, A.x), fmaf(alp_prev, A.w, A.y), Y.x, Y.y);
                    return make_float2(Y.x * w.z, Y.y * w.w);
                });
                if (dct_inverse_post(sX, cur, oth, cl)) { float2 *t_ = cur; cur = oth; oth = t_; }
                cl.sync();     // every CTA's result is complete before the gathers
                Acc2 pq_loc = {0.f, 0.f};
                for (int i = threadIdx.x; i < kc; i += DCT_T) {
                    const float v = *cg_elem(cl, cur, c_loc, i);
                    c_q[i] = v;
                    acc_add_prod(pq_loc, c_p[i], v);
                }
                const double pq = cluster_sum_acc(pq_loc, Acc2{0.f, 0.f}, s_red, s_part, parity, cl).x;
                // the gathers ended before that cluster barrier: clear the buffer
                // for the next scatter (ordered by the barriers below)
                for (int e = threadIdx.x; e < tot; e += DCT_T) cur[e] = make_float2(0.f, 0.f);
                // step lengths in FP32 (the vectors are FP32); FP64 division
                // by every thread would cost more than the update itself
                const float alp = static_cast<float>(rz) / static_cast<float>(pq);
                alp_prev = alp;
                for (int i = threadIdx.x; i < kc; i += DCT_T) c_r[i] = fmaf(-alp, c_q[i], c_r[i]);
                Acc2 rn_loc = {0.f, 0.f};
                for (int i = threadIdx.x; i < kc; i += DCT_T) acc_add_prod(rn_loc, c_r[i], c_r[i]);
                __syncthreads();
                ++it;
                const double2 rn2 = precond(rn_loc, nullptr);     // (r.r, r.z)
                if (rn2.x <= stop) { conv = true; break; }
                const float beta = static_cast<float>(rn2.y) / static_cast<float>(rz);
                for (int i = threadIdx.x; i < kc; i += DCT_T) c_p[i] = fmaf(beta, c_p[i], c_z[i]);
                __syncthreads();
                rz = rn2.y;
            }
            // x from the accumulated spectrum, filtered by beta: one inverse
            // transform, written once
            split_inverse_from(X, cur, [&](int e, int) {
                const float4 A = acc[e], w = wt[e];
                return make_float2(fmaf(alp_prev, A.z, A.x) * w.x, fmaf(alp_prev, A.w, A.y) * w.y);
            });
            alp_spec = alp_prev;
            if (dct_inverse_post(sX, cur, oth, cl)) { float2 *t_ = cur; cur = oth; oth = t_; }
            for (int e = threadIdx.x; e < tot; e += DCT_T) {
                int t0, t1;
                bool valid;
                elem_samples(X, e, t0, t1, valid);
                if (!valid) continue;
                const float2 v = cur[e];
                xq[t0] = v.x;
                xq[t1] = v.y;
            }
            if (!conv) set_status(a.status, q, TOD_ERR_NOT_CONVERGED);
        }
        if (a.spec_out) write_spectrum(sX, a.spec_out + o, acc, wt, alp_spec);
        if (a.iters && c == 0 && threadIdx.x == 0) a.iters[q] = it;
        // No barrier here: every remote access of this detscan (transposes,
        // CG gathers and scatters, preconditioner) is followed by a cluster
        // barrier before it ends, and the cluster sums alternate their slot.
    }
    cl.sync();     // no CTA leaves while a sibling may still read its shared memory
}

// ---------------------------------------------------------------------------
// A8: TOD chi^2 with n_corr marginalised and its gradients.  Per detscan,
// rhat = C(M(d - g s)); L = 1/2 sum_{k>=1} [rhat^2/P + ln P];
// v = M C^T(rhat/P) (written out: dL/ds = -g v, so the map gradient is
// -P^T(g v), a binning); dL/dg = -<M s, v>; dL/dtheta for the PSD
// parameters from sum_k 1/2 (1/P - rhat^2/P^2) dP/dtheta.
// ---------------------------------------------------------------------------
struct Chi2Args {
    const float *d, *s;
    const double *gain;
    const uint32_t *flags;
    const double *psd;
    const int64_t *off;
    const DctPlan *plans;
    const int32_t *q_plan;
    const float2 *tw;
    const int32_t *work;
    int work_count;
    int ndet;
    double fsamp;
    double *chi2, *dgain, *dpsd;
    float *v_out;
    int sz, twsz;
};

__global__ void __launch_bounds__(DCT_T, 1) k_chi2(Chi2Args a)
{
    extern __shared__ __align__(16) float2 smem_raw[];
    __shared__ Ctx sX;
    __shared__ DetScal s_sc;
    __shared__ double2 s_red[DCT_T / 32 + 1];
    __shared__ double2 s_part[2];
    cg::cluster_group cl = cg::this_cluster();
    const int C = static_cast<int>(cl.num_blocks()), c = static_cast<int>(cl.block_rank());
    const int cid = blockIdx.x / C, ncl = gridDim.x / C;
    Smem sm = carve(smem_raw, a.sz, a.twsz);
    int parity = 0;
    int cur_pi = -1;      // plan staged in shared memory
    for (int w = cid; w < a.work_count; w += ncl) {
        const int q = a.work[w];
        const int det = q % a.ndet;
        const int64_t o = a.off[q];
        load_plan(&sX, a.plans, a.q_plan[q], a.tw, sm, c, C, cur_pi);
        const Ctx &X = sX;     // shared-memory copy (a register copy would live on the stack)
        const int n = X.n, m = X.m;
        const float *sq = a.s + o, *dq = a.d + o;
        const uint32_t *fl = a.flags;
        const DetScal sc = det_scalars(&s_sc, a.psd, det, n, a.fsamp, a.gain, q);
        const float fscale = sc.fscale, alpha = sc.alpha, s2 = sc.s2, g = sc.g;
        float2 *cur = sm.U0, *oth = sm.U1;
        load_time(X, cur, [&](int j) {
            const int t0 = vpos_t(2 * j, n, m), t1 = vpos_t(2 * j + 1, n, m);
            const float d0 = __ldg(dq + t0), d1 = __ldg(dq + t1), s0v = __ldg(sq + t0), s1v = __ldg(sq + t1);
            return make_float2(flagged(fl, o + t0) ? 0.f : d0 - g * s0v, flagged(fl, o + t1) ? 0.f : d1 - g * s1v);
        });
        if (dct_forward(sX, cur, oth, X.tw1, X.tw2, cl)) { float2 *t_ = cur; cur = oth; oth = t_; }
        // per mode: rhat^2/P, ln(1+x), and the f_knee / alpha gradient terms
        Acc2 aq = {0.f, 0.f}, al1 = {0.f, 0.f}, afk = {0.f, 0.f}, aal = {0.f, 0.f};
        {
            const int total = 2 * X.npl * X.m2;
            for (int e0 = threadIdx.x; e0 < total; e0 += DCT_T) {
                const int slot = fdiv(e0, X.f_m2), k2 = e0 - slot * X.m2;
                const int e = slot * X.m2p + k2;
                const int k1 = slot_row(X, slot);
                if (k1 < 0) continue;
                const int k = k1 + X.m1 * k2;
                float2 v = cur[e];
                float wv[2];
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int kap = h ? ((k == 0) ? m : n - k) : k;
                    const float rh = h ? v.y : v.x;
                    if (kap == 0) { wv[h] = 0.f; continue; }
                    const float lf = log2f(static_cast<float>(kap) * fscale);     // log2(f/fk)
                    const float x = exp2f(alpha * lf);
                    const float P = s2 * (1.0f + x);
                    const float q2 = rh * rh / P;                                    // rhat^2 / P
                    acc_add(aq, q2);
                    acc_add(al1, log1pf(x));
                    // 1/2 (1/P - rhat^2/P^2) dP/dtheta = 1/2 (1 - q2) (dP/dtheta) / P
                    const float cpre = 0.5f * (1.0f - q2) * s2 * x / P;
                    acc_add(afk, -cpre * alpha);                                     // times 1/fk on the host side
                    acc_add(aal, cpre * lf * 0.69314718055994531f);
                    wv[h] = rh / P;
                }
                cur[e] = make_float2(wv[0], wv[1]);
            }
            __syncthreads();
        }
        if (dct_inverse(sX, cur, oth, X.tw1, X.tw2, cl)) { float2 *t_ = cur; cur = oth; oth = t_; }
        Acc2 ag = {0.f, 0.f};
        {
            const int tot = X.m1 * X.ncolmax;
            float *vq = a.v_out ? a.v_out + o : nullptr;
            for (int e = threadIdx.x; e < tot; e += DCT_T) {
                int t0, t1;
                bool valid;
                elem_samples(X, e, t0, t1, valid);
                if (!valid) continue;
                const float2 v = cur[e];
                const bool f0 = flagged(fl, o + t0), f1 = flagged(fl, o + t1);
                const float v0 = f0 ? 0.f : v.x, v1 = f1 ? 0.f : v.y;
                if (vq) { vq[t0] = v0; vq[t1] = v1; }
                acc_add_prod(ag, __ldg(sq + t0), v0);
                acc_add_prod(ag, __ldg(sq + t1), v1);
            }
        }
        const double2 r1 = cluster_sum_acc(aq, al1, s_red, s_part, parity, cl);
        const double2 r2 = cluster_sum_acc(afk, aal, s_red, s_part, parity, cl);
        const double2 r3 = cluster_sum_acc(ag, Acc2{0.f, 0.f}, s_red, s_part, parity, cl);
        if (c == 0 && threadIdx.x == 0) {
            const double sig0 = a.psd[3 * det], fk = a.psd[3 * det + 1];
            const double nm1 = static_cast<double>(n - 1);
            a.chi2[q] = 0.5 * (r1.x + r1.y + nm1 * log(sig0 * sig0));
            a.dgain[q] = -r3.x;
            a.dpsd[3 * q + 0] = (nm1 - r1.x) / sig0;
            a.dpsd[3 * q + 1] = r2.x / fk;
            a.dpsd[3 * q + 2] = r2.y;
        }
    }
    cl.sync();     // no CTA leaves while a sibling may still read its cluster-sum slot
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
static size_t smem_bytes(const Plan &p, bool ncorr)
{
    size_t b = sizeof(float2) * (2 * static_cast<size_t>(p.sz) + p.twsz);
    if (ncorr) b += static_cast<size_t>(CG_KCAP) * (sizeof(int) + 5 * sizeof(float)) +
                    sizeof(float) * 5 * GB_CAP;
    return b;
}

static cudaError_t launch_cluster(const void *fn, void *args, int C, int nclusters, size_t smem,
                                  cudaStream_t st)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(static_cast<unsigned>(nclusters * C));
    cfg.blockDim = dim3(DCT_T);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = C;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    void *argv[1] = {args};
    return cudaLaunchKernelExC(&cfg, fn, argv);
}

static cudaError_t max_clusters(const void *fn, int C, size_t smem, int *out)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(static_cast<unsigned>(C * 64));
    cfg.blockDim = dim3(DCT_T);
    cfg.dynamicSmemBytes = smem;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = C;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int n = 0;
    cudaError_t e = cudaOccupancyMaxActiveClusters(&n, fn, &cfg);
    *out = n > 0 ? n : 1;
    return e;
}

// Function attributes that do not depend on a plan: the largest dynamic
// shared memory the device allows next to each kernel's static part, and
// cluster sizes above the portable 8.  Set for the current device.
static cudaError_t init_transform_kernels()
{
    int dev = 0, optin = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e != cudaSuccess) return e;
    const void *fns[3] = {reinterpret_cast<const void *>(k_gain), reinterpret_cast<const void *>(k_ncorr),
                          reinterpret_cast<const void *>(k_chi2)};
    for (const void *fn : fns) {
        cudaFuncAttributes fa;
        e = cudaFuncGetAttributes(&fa, fn);
        if (e != cudaSuccess) return e;
        e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 optin - static_cast<int>(fa.sharedSizeBytes));
        if (e != cudaSuccess) return e;
        e = cudaFuncSetAttribute(fn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

cudaError_t transform_cluster_occupancy(int C, size_t smem_dyn, int *nclusters)
{
    cudaError_t e = init_transform_kernels();
    if (e != cudaSuccess) return e;
    *nclusters = 0;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(static_cast<unsigned>(C * 64));
    cfg.blockDim = dim3(DCT_T);
    cfg.dynamicSmemBytes = smem_dyn;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = C;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaOccupancyMaxActiveClusters(nclusters, reinterpret_cast<const void *>(k_ncorr), &cfg);
}

cudaError_t setup_dct_kernels(Plan &p)
{
    p.smem_gain = smem_bytes(p, false);
    p.smem_ncorr = smem_bytes(p, true);
    cudaError_t e = init_transform_kernels();
    if (e != cudaSuccess) return e;
    e = max_clusters(reinterpret_cast<const void *>(k_gain), p.C, p.smem_gain, &p.nclusters_gain);
    if (e != cudaSuccess) return e;
    e = max_clusters(reinterpret_cast<const void *>(k_ncorr), p.C, p.smem_ncorr, &p.nclusters_ncorr);
    return e;
}

cudaError_t launch_gain(const Plan &p, const float *d, const float *s, const uint32_t *flags,
                        const double *psd, tod_rng rng, int mode, double *g, double *mu,
                        double *sig, cudaStream_t st, int work_begin, int work_count)
{
    if (work_count <= 0) return cudaSuccess;
    GainArgs a;
    a.d = d; a.s = s; a.flags = flags; a.psd = psd; a.off = p.off; a.plans = p.plans;
    a.q_plan = p.q_plan; a.tw = p.tw; a.work = p.work; a.work_begin = work_begin;
    a.work_count = work_count; a.ndet = p.ndet; a.fsamp = p.fsamp; a.rng = rng; a.mode = mode;
    a.ab_out = p.gain_ab; a.sz = p.sz;
    a.m1max = p.m1max; a.m2max = p.m2max; a.twsz = p.twsz;
    cudaError_t e = cudaSuccess;
    if (p.schedule == TOD_SCHED_PER_SCAN) {
        for (int w = 0; w < work_count && e == cudaSuccess; ++w) {
            a.work_begin = work_begin + w;
            a.work_count = 1;
            e = launch_cluster(reinterpret_cast<const void *>(k_gain), &a, p.C, 1, p.smem_gain, st);
        }
    } else {
        const int ncl = std::min(work_count, p.nclusters_gain);
        e = launch_cluster(reinterpret_cast<const void *>(k_gain), &a, p.C, ncl, p.smem_gain, st);
    }
    if (e != cudaSuccess) return e;
    k_gain_draw<<<(work_count + 255) / 256, 256, 0, st>>>(p.gain_ab, p.work, work_begin, work_count, rng, mode, g,
                                                          mu, sig, p.status);
    return cudaGetLastError();
}

cudaError_t launch_ncorr(const Plan &p, const float *d, const float *s, const double *gain,
                         const uint32_t *flags, const double *psd, tod_rng rng, int mode,
                         float tol, int maxit, float *x, int32_t *iters, cudaStream_t st,
                         int work_begin, int work_count, bool prepare)
{
    return launch_ncorr_scratch(p, d, s, gain, flags, psd, rng, mode, tol, maxit, x, iters, st,
                                work_begin, work_count, p.wscratch, p.nclusters_ncorr, prepare);
}

cudaError_t launch_ncorr_scratch(const Plan &p, const float *d, const float *s, const double *gain,
                                 const uint32_t *flags, const double *psd, tod_rng rng, int mode,
                                 float tol, int maxit, float *x, int32_t *iters, cudaStream_t st,
                                 int work_begin, int work_count, float4 *scratch, int nclusters_max,
                                 bool prepare)
{
    if (work_count <= 0) return cudaSuccess;
    if (nclusters_max < 1) return cudaErrorInvalidValue;
    NcorrArgs a;
    a.d = d; a.s = s; a.gain = gain; a.flags = flags; a.psd = psd; a.off = p.off; a.plans = p.plans;
    a.q_plan = p.q_plan; a.tw = p.tw; a.work = p.work; a.work_begin = work_begin;
    a.work_count = work_count; a.ndet = p.ndet; a.fsamp = p.fsamp; a.rng = rng; a.mode = mode;
    a.tol = tol; a.maxit = maxit; a.x_out = x; a.iters = iters; a.status = p.status; a.sz = p.sz;
    a.wscratch = scratch;
    a.spec_out = p.spec_out;
    const void *kfn = reinterpret_cast<const void *>(k_ncorr);
    a.xtab = p.use_prec ? p.xtab : nullptr;
    a.lvalid = p.lvalid;
    if (p.use_prec && prepare) {
        cudaError_t e = launch_toeplitz_prep(p, psd, st);
        if (e != cudaSuccess) return e;
    }
    a.m1max = p.m1max; a.m2max = p.m2max; a.twsz = p.twsz;
    if (p.schedule == TOD_SCHED_PER_SCAN) {
        for (int w = 0; w < work_count; ++w) {
            a.work_begin = work_begin + w;
            a.work_count = 1;
            cudaError_t e = launch_cluster(kfn, &a, p.C, 1, p.smem_ncorr, st);
            if (e != cudaSuccess) return e;
        }
        return cudaSuccess;
    }
    const int ncl = std::min(work_count, std::min(p.nclusters_ncorr, nclusters_max));
    return launch_cluster(kfn, &a, p.C, ncl, p.smem_ncorr, st);
}

}  // namespace tg

namespace tg {

cudaError_t launch_chi2(const Plan &p, const float *d, const float *s, const double *gain,
                        const uint32_t *flags, const double *psd, double *chi2, double *dgain,
                        double *dpsd, float *v, cudaStream_t st)
{
    if (p.nq == 0) return cudaSuccess;
    static_assert(sizeof(Chi2Args) < 4096, "kernel parameters");
    Chi2Args a;
    a.d = d; a.s = s; a.gain = gain; a.flags = flags; a.psd = psd; a.off = p.off; a.plans = p.plans;
    a.q_plan = p.q_plan; a.tw = p.tw; a.work = p.work; a.work_count = p.nq; a.ndet = p.ndet;
    a.fsamp = p.fsamp; a.chi2 = chi2; a.dgain = dgain; a.dpsd = dpsd; a.v_out = v; a.sz = p.sz;
    a.twsz = p.twsz;
    const int ncl = std::min(p.nq, p.nclusters_gain);
    return launch_cluster(reinterpret_cast<const void *>(k_chi2), &a, p.C, ncl, p.smem_gain, st);
}

}  // namespace tg
