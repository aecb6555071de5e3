// A3 batched DCT-II (the mirrored FFT of paper Sect. 4.2), A4 gain draw and
// A5 correlated-noise draw (Eq. `gibbsstart`, lines 1-2; Sect. 5 CG gap
// filling), as persistent thread-block-cluster kernels.
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
// Column FFTs (length m1) and row FFTs (length m2) are mixed-radix (2,3,4,5)
// Stockham passes in shared memory with butterflies in registers; the
// transpose between them reads the other CTAs' shared memory (DSMEM) into
// registers, applies the four-step twiddle, and writes back into the same
// buffer after a cluster barrier, so one buffer of ~m/C complex values per
// CTA holds a transform.  Nothing of a transform touches HBM.
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

// One Stockham radix-R pass (Govindaraju et al. 2008 formulation) over nvec
// vectors of length L held in shared memory (element stride es, vector
// stride vs).  All reads complete before the barrier, all writes follow it,
// so the pass is in place.  vfast: consecutive threads take consecutive
// vectors (column FFTs) instead of consecutive elements (row FFTs).
template <int R, bool INV>
__device__ __noinline__ void fft_pass(float2 *__restrict__ buf, int L, int Ns, int nvec, int es,
                                         int vs, bool vfast, const float2 *__restrict__ tw)
{
    constexpr int NB = DCT_EMAX / R;
    const int LR = L / R;
    const int total = nvec * LR;
    float2 v[NB][R];
#pragma unroll
    for (int b = 0; b < NB; ++b) {
        const int w = threadIdx.x + b * DCT_T;
        if (w < total) {
            int vec, j;
            if (vfast) { j = w / nvec; vec = w - j * nvec; }
            else { vec = w / LR; j = w - vec * LR; }
            const float2 *p = buf + vec * vs + j * es;
#pragma unroll
            for (int r = 0; r < R; ++r) v[b][r] = p[r * LR * es];
        }
    }
    __syncthreads();
    const int tstep = L / (Ns * R);
#pragma unroll
    for (int b = 0; b < NB; ++b) {
        const int w = threadIdx.x + b * DCT_T;
        if (w < total) {
            int vec, j;
            if (vfast) { j = w / nvec; vec = w - j * nvec; }
            else { vec = w / LR; j = w - vec * LR; }
            const int k = j % Ns;
#pragma unroll
            for (int r = 1; r < R; ++r) {
                float2 t = tw[r * k * tstep];
                if (INV) t.y = -t.y;
                v[b][r] = cmul(v[b][r], t);
            }
            Dft<R, INV>::run(v[b]);
            const int idxD = (j / Ns) * Ns * R + k;
            float2 *p = buf + vec * vs + idxD * es;
#pragma unroll
            for (int r = 0; r < R; ++r) p[r * Ns * es] = v[b][r];
        }
    }
    __syncthreads();
}

template <bool INV>
__device__ void fft_smem(float2 *buf, int L, const int8_t *rad, int nr, int nvec, int es, int vs,
                         bool vfast, const float2 *tw)
{
    int Ns = 1;
    for (int s = 0; s < nr; ++s) {
        const int R = rad[s];
        if (R == 4) fft_pass<4, INV>(buf, L, Ns, nvec, es, vs, vfast, tw);
        else if (R == 2) fft_pass<2, INV>(buf, L, Ns, nvec, es, vs, vfast, tw);
        else if (R == 3) fft_pass<3, INV>(buf, L, Ns, nvec, es, vs, vfast, tw);
        else fft_pass<5, INV>(buf, L, Ns, nvec, es, vs, vfast, tw);
        Ns *= R;
    }
}

// ---------------------------------------------------------------------------
// per-detscan transform context (shared memory copy of the plan + this CTA's
// share of it)
// ---------------------------------------------------------------------------
struct Ctx {
    int n, m, m1, m2, ncolmax, npmax, P;
    int nr1, nr2;
    int c, C;
    int ncol;    // valid local columns
    int p0, npl; // local row pairs
    int8_t r1[DCT_MAXR], r2[DCT_MAXR];
};

__device__ __forceinline__ int slot_row(const Ctx &X, int slot) {
    const int p = X.p0 + (slot >> 1);
    if (p >= X.P) return -1;
    if ((slot & 1) == 0) return p;
    const int r = X.m1 - p;
    if (p == 0 || r == p) return -1;
    return r;
}

// sample index of position i of the even/odd-reordered sequence v
__device__ __forceinline__ int vpos_t(int i, int n, int m) { return i < m ? 2 * i : 2 * n - 1 - 2 * i; }

// Forward half-split: packed orthonormal coefficients of slot k from Z_k, Z_{m-k}.
__device__ __forceinline__ float2 split_fwd_one(float2 a, float2 b, int k, int n, float sq) {
    const float2 cb = cconj(b);
    const float2 A = cscale(cadd(a, cb), 0.5f);
    const float2 d = csub(a, cb);
    const float2 Bv = make_float2(0.5f * d.y, -0.5f * d.x);                     // -i/2 (a - conj b)
    const float xk = static_cast<float>(k) / static_cast<float>(2 * n);
    const float2 e1 = cexpi_pi(-xk), e5 = cexpi_pi(-5.0f * xk);
    const float2 W = cadd(cmul(e1, A), cmul(e5, Bv));
    return make_float2(sq * W.x, -sq * W.y);
}
// Inverse of the half-split: Z_k from the packed slots k and m-k.
__device__ __forceinline__ float2 split_inv_one(float2 yk, float2 yp, int k, int kp, int n, float sq) {
    // V_k = sqrt(n/2) e^{i pi k/2n} conj(Y_k)   (sq carries sqrt(n/2)/m)
    const float2 Vk = cscale(cmul(cexpi_pi(static_cast<float>(k) / static_cast<float>(2 * n)), cconj(yk)), sq);
    const float2 Vp = cscale(cmul(cexpi_pi(static_cast<float>(kp) / static_cast<float>(2 * n)), cconj(yp)), sq);
    const float2 cVp = cconj(Vp);
    const float2 A = cscale(cadd(Vk, cVp), 0.5f);
    const float2 Bv = cscale(cmul(cexpi_pi(static_cast<float>(2 * k) / static_cast<float>(n)), csub(Vk, cVp)), 0.5f);
    return make_float2(A.x - Bv.y, A.y + Bv.x);                                 // A + i B
}

// Real split over this CTA's row pairs, in place (forward or inverse).
template <bool INV>
__device__ __noinline__ void split_pass(const Ctx &X, float2 *U)
{
    const int m2 = X.m2, m1 = X.m1, m = X.m, n = X.n;
    const float sq = INV ? static_cast<float>(sqrt(0.5 * n) / m) : static_cast<float>(sqrt(2.0 / n));
    const float s0 = INV ? static_cast<float>(sqrt(static_cast<double>(n)) / m)
                         : static_cast<float>(1.0 / sqrt(static_cast<double>(n)));
    const int total = X.npl * m2;
    for (int e = threadIdx.x; e < total; e += DCT_T) {
        const int pl = e / m2, k2 = e - pl * m2;
        const int p = X.p0 + pl;
        const int cnt = (p == 0) ? (m2 / 2 + 1) : ((2 * p == m1) ? (m2 + 1) / 2 : m2);
        if (k2 >= cnt) continue;
        const int k = p + m1 * k2;
        int ib, k2p;
        if (p == 0) { k2p = (m2 - k2) % m2; ib = 2 * pl * m2 + k2p; }
        else { k2p = m2 - 1 - k2; ib = ((m1 - p == p) ? 2 * pl : 2 * pl + 1) * m2 + k2p; }
        const int ia = 2 * pl * m2 + k2;
        const int kp = (m - k) % m;
        const float2 Za = U[ia], Zb = U[ib];
        if (k == 0) {
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
            const float2 Ya = split_fwd_one(Za, Zb, k, n, sq);
            if (ib != ia) U[ib] = split_fwd_one(Zb, Za, kp, n, sq);
            U[ia] = Ya;
        } else {
            const float2 Ya = split_inv_one(Za, Zb, k, kp, n, sq);
            if (ib != ia) U[ib] = split_inv_one(Zb, Za, kp, k, n, sq);
            U[ia] = Ya;
        }
    }
    __syncthreads();
}

// Time layout -> freq layout (forward) or back (inverse) through registers:
// remote reads, cluster barrier, local writes.  The four-step twiddle
// W_m^{-+ j2 k1} is applied on the way.
template <bool INV>
__device__ __noinline__ void transpose(const Ctx &X, float2 *U, cg::cluster_group &cl)
{
    constexpr int NE = DCT_EMAX;
    float2 tmp[NE];
    cl.sync();   // every CTA finished its local passes
    const float inv_m = 2.0f / static_cast<float>(X.m);
    if (!INV) {
        const int total = 2 * X.npl * X.m2;
#pragma unroll
        for (int b = 0; b < NE; ++b) {
            const int e = threadIdx.x + b * DCT_T;
            float2 v = make_float2(0.f, 0.f);
            if (e < total) {
                const int slot = e / X.m2, j2 = e - slot * X.m2;
                const int k1 = slot_row(X, slot);
                if (k1 >= 0) {
                    const int o = j2 / X.ncolmax, lc = j2 - o * X.ncolmax;
                    const float2 *rT = cl.map_shared_rank(U, o);
                    v = cmul(rT[k1 * X.ncolmax + lc], cexpi_pi(-static_cast<float>(j2 * k1) * inv_m));
                }
            }
            tmp[b] = v;
        }
        cl.sync();   // all remote reads done before anyone overwrites
#pragma unroll
        for (int b = 0; b < NE; ++b) {
            const int e = threadIdx.x + b * DCT_T;
            if (e < total) U[e] = tmp[b];
        }
    } else {
        const int total = X.m1 * X.ncolmax;
#pragma unroll
        for (int b = 0; b < NE; ++b) {
            const int e = threadIdx.x + b * DCT_T;
            float2 v = make_float2(0.f, 0.f);
            if (e < total) {
                const int k1 = e / X.ncolmax, lc = e - k1 * X.ncolmax;
                if (lc < X.ncol) {
                    const int j2 = X.c * X.ncolmax + lc;
                    const int p = min(k1, X.m1 - k1);
                    const int o = p / X.npmax;
                    const int slot = 2 * (p - o * X.npmax) + (k1 == p ? 0 : 1);
                    const float2 *rF = cl.map_shared_rank(U, o);
                    v = cmul(rF[slot * X.m2 + j2], cexpi_pi(static_cast<float>(j2 * k1) * inv_m));
                }
            }
            tmp[b] = v;
        }
        cl.sync();
#pragma unroll
        for (int b = 0; b < NE; ++b) {
            const int e = threadIdx.x + b * DCT_T;
            if (e < total) U[e] = tmp[b];
        }
    }
    __syncthreads();
}

// Forward DCT of the time-layout data already in U (packed spectrum -> U).
__device__ __noinline__ void dct_forward_inplace(const Ctx &X, float2 *U, const float2 *tw1, const float2 *tw2,
                                    cg::cluster_group &cl)
{
    fft_smem<false>(U, X.m1, X.r1, X.nr1, X.ncol, X.ncolmax, 1, true, tw1);
    transpose<false>(X, U, cl);
    fft_smem<false>(U, X.m2, X.r2, X.nr2, 2 * X.npl, 1, X.m2, false, tw2);
    split_pass<false>(X, U);
}
// Inverse (transpose of the orthonormal DCT-II): packed spectrum in U ->
// time layout in U, scaled.
__device__ __noinline__ void dct_inverse_inplace(const Ctx &X, float2 *U, const float2 *tw1, const float2 *tw2,
                                    cg::cluster_group &cl)
{
    split_pass<true>(X, U);
    fft_smem<true>(U, X.m2, X.r2, X.nr2, 2 * X.npl, 1, X.m2, false, tw2);
    transpose<true>(X, U, cl);
    fft_smem<true>(U, X.m1, X.r1, X.nr1, X.ncol, X.ncolmax, 1, true, tw1);
}

// Fill U (time layout) with f(j) = (x_{t(2j)}, x_{t(2j+1)}) for own columns.
template <class F>
__device__ void load_time(const Ctx &X, float2 *U, F f)
{
    const int total = X.m1 * X.ncolmax;
    for (int e = threadIdx.x; e < total; e += DCT_T) {
        const int j1 = e / X.ncolmax, lc = e - j1 * X.ncolmax;
        float2 z = make_float2(0.f, 0.f);
        if (lc < X.ncol) z = f(j1 * X.m2 + X.c * X.ncolmax + lc);
        U[e] = z;
    }
    __syncthreads();
}

// Cluster-wide sum of two doubles in a fixed order (identical in every CTA).
__device__ double2 cluster_sum2(double2 v, double2 *s_red, double2 *s_part, int &parity,
                                cg::cluster_group &cl)
{
#pragma unroll
    for (int o = 16; o; o >>= 1) {
        v.x += __shfl_xor_sync(0xffffffffu, v.x, o);
        v.y += __shfl_xor_sync(0xffffffffu, v.y, o);
    }
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) s_red[warp] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double2 t = make_double2(0.0, 0.0);
        for (int w = 0; w < DCT_T / 32; ++w) { t.x += s_red[w].x; t.y += s_red[w].y; }
        s_part[parity] = t;
    }
    cl.sync();
    double2 tot = make_double2(0.0, 0.0);
    for (int r = 0; r < static_cast<int>(cl.num_blocks()); ++r) {
        const double2 pr = *cl.map_shared_rank(&s_part[parity], r);
        tot.x += pr.x;
        tot.y += pr.y;
    }
    parity ^= 1;
    return tot;
}

__device__ void load_ctx(Ctx &X, const DctPlan &P, int c, int C)
{
    X.n = P.n; X.m = P.m; X.m1 = P.m1; X.m2 = P.m2; X.ncolmax = P.ncolmax; X.npmax = P.npmax;
    X.P = P.P; X.nr1 = P.nr1; X.nr2 = P.nr2; X.c = c; X.C = C;
    X.ncol = max(0, min(P.ncolmax, P.m2 - c * P.ncolmax));
    X.p0 = c * P.npmax;
    X.npl = max(0, min(P.npmax, P.P - X.p0));
    for (int i = 0; i < DCT_MAXR; ++i) { X.r1[i] = P.r1[i]; X.r2[i] = P.r2[i]; }
}

__device__ __forceinline__ bool flagged(const uint32_t *flags, int64_t t) {
    return (flags[t >> 5] >> (t & 31)) & 1u;
}

// (f/fknee)^alpha at DCT mode kappa, FP32
__device__ __forceinline__ float fratio_pow(int kappa, float fscale, float alpha) {
    return exp2f(alpha * log2f(static_cast<float>(kappa) * fscale));
}

// shared-memory carve-up common to both kernels
struct Smem {
    float2 *U0, *U1, *tw1, *tw2;
};
__device__ __forceinline__ Smem carve(void *raw, int sz, int m1max, int m2max)
{
    Smem s;
    float2 *p = static_cast<float2 *>(raw);
    s.U0 = p; p += sz;
    s.U1 = p; p += sz;
    s.tw1 = p; p += m1max;
    s.tw2 = p; p += m2max;
    return s;
}

__device__ void load_plan(Ctx *sX, const DctPlan *plans, int pi, const float2 *tw,
                          float2 *tw1, float2 *tw2, int c, int C)
{
    __syncthreads();      // previous users of sX are done
    if (threadIdx.x == 0) load_ctx(*sX, plans[pi], c, C);
    __syncthreads();
    const Ctx &X = *sX;
    const DctPlan &P = plans[pi];
    for (int i = threadIdx.x; i < X.m1; i += DCT_T) tw1[i] = tw[P.tw1 + i];
    for (int i = threadIdx.x; i < X.m2; i += DCT_T) tw2[i] = tw[P.tw2 + i];
    __syncthreads();
}

// ---------------------------------------------------------------------------
// A4: gain.  shat = C(M s) in U0, dhat = C(M d) in U1, sums over k >= 1.
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
    double *g_out, *mu_out, *sig_out;
    int32_t *status;
    int sz, m1max, m2max;
};

__global__ void __launch_bounds__(DCT_T, 1) k_gain(GainArgs a)
{
    extern __shared__ __align__(16) float2 smem_raw[];
    __shared__ Ctx sX;
    __shared__ double2 s_red[DCT_T / 32];
    __shared__ double2 s_part[2];
    cg::cluster_group cl = cg::this_cluster();
    const int C = static_cast<int>(cl.num_blocks()), c = static_cast<int>(cl.block_rank());
    const int cid = blockIdx.x / C, ncl = gridDim.x / C;
    Smem sm = carve(smem_raw, a.sz, a.m1max, a.m2max);
    int parity = 0;
    for (int w = cid; w < a.work_count; w += ncl) {
        const int q = a.work[a.work_begin + w];
        const int det = q % a.ndet;
        const int64_t o = a.off[q];
        load_plan(&sX, a.plans, a.q_plan[q], a.tw, sm.tw1, sm.tw2, c, C);
        const Ctx &X = sX;
        const int n = X.n, m = X.m;
        const float *sq = a.s + o, *dq = a.d + o;
        const uint32_t *fl = a.flags;
        load_time(X, sm.U0, [&](int j) {
            const int t0 = vpos_t(2 * j, n, m), t1 = vpos_t(2 * j + 1, n, m);
            return make_float2(flagged(fl, o + t0) ? 0.f : sq[t0], flagged(fl, o + t1) ? 0.f : sq[t1]);
        });
        dct_forward_inplace(X, sm.U0, sm.tw1, sm.tw2, cl);
        load_time(X, sm.U1, [&](int j) {
            const int t0 = vpos_t(2 * j, n, m), t1 = vpos_t(2 * j + 1, n, m);
            return make_float2(flagged(fl, o + t0) ? 0.f : dq[t0], flagged(fl, o + t1) ? 0.f : dq[t1]);
        });
        dct_forward_inplace(X, sm.U1, sm.tw1, sm.tw2, cl);
        // sums over this CTA's packed coefficients
        const double sig0 = a.psd[3 * det], fk = a.psd[3 * det + 1], al = a.psd[3 * det + 2];
        const float fscale = static_cast<float>(a.fsamp / (2.0 * n * fk));
        const float alpha = static_cast<float>(al);
        const float inv_s2 = static_cast<float>(1.0 / (sig0 * sig0));
        Acc2 sa = {0.f, 0.f}, sb = {0.f, 0.f};
        const int total = 2 * X.npl * X.m2;
        for (int e = threadIdx.x; e < total; e += DCT_T) {
            const int slot = e / X.m2, k2 = e - slot * X.m2;
            const int k1 = slot_row(X, slot);
            if (k1 < 0) continue;
            const int k = k1 + X.m1 * k2;
            const float2 S = sm.U0[e], D = sm.U1[e];
            const int ka = k, kb = (k == 0) ? m : n - k;
            if (ka != 0) {
                const float wa = inv_s2 / (1.0f + fratio_pow(ka, fscale, alpha));
                acc_add(sa, S.x * S.x * wa);
                acc_add(sb, S.x * D.x * wa);
            }
            const float wb = inv_s2 / (1.0f + fratio_pow(kb, fscale, alpha));
            acc_add(sa, S.y * S.y * wb);
            acc_add(sb, S.y * D.y * wb);
        }
        const double2 ab = cluster_sum2(make_double2(acc_value(sa), acc_value(sb)), s_red, s_part,
                                        parity, cl);
        if (c == 0 && threadIdx.x == 0) {
            const double A = ab.x, B = ab.y;
            if (!(A > 0.0)) {
                set_status(a.status, q, TOD_ERR_ARG);
                a.g_out[q] = 0.0;
                if (a.mu_out) a.mu_out[q] = 0.0;
                if (a.sig_out) a.sig_out[q] = 0.0;
            } else {
                const double mu = B / A, sg = 1.0 / sqrt(A);
                double z = 0.0;
                if (a.mode == TOD_MODE_DRAW) {
                    const uint64_t it = a.rng.gibbs_iter_dev ? *a.rng.gibbs_iter_dev : a.rng.gibbs_iter;
                    const u64x4 wv = philox4x64(0, static_cast<uint64_t>(q), 0, it,
                                                a.rng.seed, a.rng.band);
                    const double u1 = (static_cast<double>(wv.x[0] >> 11) + 0.5) * 1.1102230246251565e-16;
                    const double u2 = (static_cast<double>(wv.x[1] >> 11) + 0.5) * 1.1102230246251565e-16;
                    z = sqrt(-2.0 * log(u1)) * cospi(2.0 * u2);
                }
                a.g_out[q] = mu + z * sg;
                if (a.mu_out) a.mu_out[q] = mu;
                if (a.sig_out) a.sig_out[q] = sg;
            }
        }
    }
}

// ---------------------------------------------------------------------------
// A5: correlated noise.  x0 = B^{-1} b (B = C^T diag(phi + 1/sigma0^2) C) in
// U1; flagged detscans then solve the Schur complement
//   S y = E^T x0,  S = sigma0^2 I - E^T B^{-1} E = E^T C^T diag(gamma) C E
// (E: flagged samples; C^T C = I) by CG and add B^{-1} E y (Woodbury):
// x = A^{-1} b exactly, A = B - E E^T / sigma0^2.
// ---------------------------------------------------------------------------
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
    int sz, m1max, m2max;
};

// Multiply the packed spectrum in U by a per-mode weight:
//   beta_kappa  = 1/(phi_kappa + 1/sigma0^2) = s2/(1 + r)          (hp = false)
//   gamma_kappa = sigma0^2 - beta_kappa     = s2 r/(1 + r)         (hp = true)
// with r = sigma0^2 phi = (f/f_knee)^-alpha (r = 0 at kappa = 0).  gamma is
// evaluated directly, so the Schur operator sigma0^2 I - E^T B^{-1} E =
// E^T C^T diag(gamma) C E carries no FP32 cancellation on its small modes.
__device__ __noinline__ void apply_filter(const Ctx &X, float2 *U, float fscale, float alpha, float s2,
                                          bool hp)
{
    const int total = 2 * X.npl * X.m2;
    for (int e = threadIdx.x; e < total; e += DCT_T) {
        const int slot = e / X.m2, k2 = e - slot * X.m2;
        const int k1 = slot_row(X, slot);
        if (k1 < 0) continue;
        const int k = k1 + X.m1 * k2;
        const int ka = k, kb = (k == 0) ? X.m : X.n - k;
        const float ra = (ka == 0) ? 0.f : fratio_pow(ka, fscale, -alpha);
        const float rb = fratio_pow(kb, fscale, -alpha);
        const float wa = hp ? s2 * ra / (1.0f + ra) : s2 / (1.0f + ra);
        const float wb = hp ? s2 * rb / (1.0f + rb) : s2 / (1.0f + rb);
        float2 v = U[e];
        v.x *= wa;
        v.y *= wb;
        U[e] = v;
    }
    __syncthreads();
}

// element e of the time layout -> (t0, t1) samples
__device__ __forceinline__ void elem_samples(const Ctx &X, int e, int &t0, int &t1, bool &valid)
{
    const int j1 = e / X.ncolmax, lc = e - j1 * X.ncolmax;
    valid = lc < X.ncol;
    const int j = j1 * X.m2 + X.c * X.ncolmax + lc;
    t0 = vpos_t(2 * j, X.n, X.m);
    t1 = vpos_t(2 * j + 1, X.n, X.m);
}
// sample t -> (owner CTA, element, part)
__device__ __forceinline__ void sample_loc(const Ctx &X, int t, int &owner, int &loc)
{
    // position of sample t in the even-then-reversed-odd order: t/2 for even
    // t, n-1-(t-1)/2 = n-1-floor(t/2) for odd t
    const int h = t >> 1;
    const int i = (t & 1) ? (X.n - 1) - h : h;
    const int j = i >> 1;
    const int j1 = j / X.m2, j2 = j - j1 * X.m2;
    owner = j2 / X.ncolmax;
    const int lc = j2 - owner * X.ncolmax;
    loc = 2 * (j1 * X.ncolmax + lc) + (i & 1);
}

__global__ void __launch_bounds__(DCT_T, 1) k_ncorr(NcorrArgs a)
{
    extern __shared__ __align__(16) float2 smem_raw[];
    __shared__ Ctx sX;
    __shared__ double2 s_red[DCT_T / 32];
    __shared__ double2 s_part[2];
    __shared__ int s_scan[DCT_T];
    cg::cluster_group cl = cg::this_cluster();
    const int C = static_cast<int>(cl.num_blocks()), c = static_cast<int>(cl.block_rank());
    const int cid = blockIdx.x / C, ncl = gridDim.x / C;
    Smem sm = carve(smem_raw, a.sz, a.m1max, a.m2max);
    // CG vectors after the twiddle tables
    int *c_loc = reinterpret_cast<int *>(sm.tw2 + a.m2max);
    float *c_y = reinterpret_cast<float *>(c_loc + CG_KCAP);
    float *c_r = c_y + CG_KCAP;
    float *c_p = c_r + CG_KCAP;
    float *c_q = c_p + CG_KCAP;
    int parity = 0;
    for (int w = cid; w < a.work_count; w += ncl) {
        const int q = a.work[a.work_begin + w];
        const int det = q % a.ndet;
        const int64_t o = a.off[q];
        load_plan(&sX, a.plans, a.q_plan[q], a.tw, sm.tw1, sm.tw2, c, C);
        const Ctx &X = sX;
        const int n = X.n, m = X.m;
        const double sig0 = a.psd[3 * det], fk = a.psd[3 * det + 1], al = a.psd[3 * det + 2];
        const float fscale = static_cast<float>(a.fsamp / (2.0 * n * fk));
        const float alpha = static_cast<float>(al);
        const float s2 = static_cast<float>(sig0 * sig0);
        const float inv_s2 = static_cast<float>(1.0 / (sig0 * sig0));
        const float inv_s = static_cast<float>(1.0 / sig0);
        const float g = static_cast<float>(a.gain[q]);
        const bool draw = a.mode == TOD_MODE_DRAW;
        const float *dq = a.d + o, *sq = a.s + o;
        const uint32_t *fl = a.flags;
        const tod_rng rng = a.rng;
        const uint64_t gi = rng.gibbs_iter_dev ? *rng.gibbs_iter_dev : rng.gibbs_iter;
        // right-hand side, time-domain part: M (r/s2 + w1/s)
        load_time(X, sm.U1, [&](int j) {
            const int t0 = vpos_t(2 * j, n, m), t1 = vpos_t(2 * j + 1, n, m);
            float2 w1 = make_float2(0.f, 0.f);
            if (draw) w1 = stream_normal_pair(rng.seed, rng.band, q, 1, gi, 2 * j);
            const float r0 = flagged(fl, o + t0) ? 0.f
                                                  : fmaf(dq[t0] - g * sq[t0], inv_s2, w1.x * inv_s);
            const float r1 = flagged(fl, o + t1) ? 0.f
                                                  : fmaf(dq[t1] - g * sq[t1], inv_s2, w1.y * inv_s);
            return make_float2(r0, r1);
        });
        dct_forward_inplace(X, sm.U1, sm.tw1, sm.tw2, cl);
        // + sqrt(phi) w2, times beta
        {
            const int total = 2 * X.npl * X.m2;
            for (int e = threadIdx.x; e < total; e += DCT_T) {
                const int slot = e / X.m2, k2 = e - slot * X.m2;
                const int k1 = slot_row(X, slot);
                if (k1 < 0) continue;
                const int k = k1 + X.m1 * k2;
                const int ka = k, kb = (k == 0) ? m : n - k;
                const float pa = (ka == 0) ? 0.f : fratio_pow(ka, fscale, -alpha) * inv_s2;  // phi
                const float pb = fratio_pow(kb, fscale, -alpha) * inv_s2;
                float2 v = sm.U1[e];
                if (draw) {
                    const float2 w2 = stream_normal_pair(rng.seed, rng.band, q, 2, gi, 2 * k);
                    v.x += sqrtf(pa) * w2.x;
                    v.y += sqrtf(pb) * w2.y;
                }
                v.x /= (pa + inv_s2);
                v.y /= (pb + inv_s2);
                sm.U1[e] = v;
            }
            __syncthreads();
        }
        dct_inverse_inplace(X, sm.U1, sm.tw1, sm.tw2, cl);      // U1 = x0 (time layout)

        // flagged samples owned by this CTA, in sample order (deterministic)
        const int64_t wb0 = o >> 5, wb1 = (o + n - 1) >> 5;
        const int nw = static_cast<int>(wb1 - wb0 + 1);
        const int per = (nw + DCT_T - 1) / DCT_T;
        int mycnt = 0;
        for (int i = 0; i < per; ++i) {
            const int wi = threadIdx.x * per + i;
            if (wi >= nw) break;
            uint32_t bits = fl[wb0 + wi];
            while (bits) {
                const int b = __popc((bits & (0u - bits)) - 1u);   // index of the lowest set bit
                bits &= bits - 1;
                const int64_t tl = ((wb0 + wi) << 5) + b - o;
                if (tl < 0 || tl >= n) continue;
                int ow, loc;
                sample_loc(X, static_cast<int>(tl), ow, loc);
                if (ow == c) ++mycnt;
            }
        }
        s_scan[threadIdx.x] = mycnt;
        __syncthreads();
        if (threadIdx.x == 0) {
            int acc = 0;
            for (int i = 0; i < DCT_T; ++i) { const int v = s_scan[i]; s_scan[i] = acc; acc += v; }
            s_red[0].x = static_cast<double>(acc);
        }
        __syncthreads();
        const int kc = static_cast<int>(s_red[0].x);
        int pos = s_scan[threadIdx.x];
        __syncthreads();
        for (int i = 0; i < per; ++i) {
            const int wi = threadIdx.x * per + i;
            if (wi >= nw) break;
            uint32_t bits = fl[wb0 + wi];
            while (bits) {
                const int b = __popc((bits & (0u - bits)) - 1u);   // index of the lowest set bit
                bits &= bits - 1;
                const int64_t tl = ((wb0 + wi) << 5) + b - o;
                if (tl < 0 || tl >= n) continue;
                int ow, loc;
                sample_loc(X, static_cast<int>(tl), ow, loc);
                if (ow == c) {
                    if (pos < CG_KCAP) c_loc[pos] = loc;
                    ++pos;
                }
            }
        }
        __syncthreads();
        const double2 kt = cluster_sum2(make_double2(static_cast<double>(kc),
                                                     kc > CG_KCAP ? 1.0 : 0.0), s_red, s_part, parity, cl);
        int it = 0;
        bool conv = true;
        if (kt.x > 0.0 && kt.y > 0.0) {
            conv = false;      // too many flagged samples for the CG buffers: left as x0
            set_status(a.status, q, TOD_ERR_NOT_CONVERGED);
        } else if (kt.x > 0.0) {
            float *U1f = reinterpret_cast<float *>(sm.U1);
            float *U0f = reinterpret_cast<float *>(sm.U0);
            // rhs = E^T x0 ; y = 0 ; r = p = rhs
            double rr_loc = 0.0;
            for (int i = threadIdx.x; i < kc; i += DCT_T) {
                const float v = U1f[c_loc[i]];
                c_y[i] = 0.f; c_r[i] = v; c_p[i] = v;
                rr_loc += static_cast<double>(v) * v;
            }
            double rr = cluster_sum2(make_double2(rr_loc, 0.0), s_red, s_part, parity, cl).x;
            const double stop = static_cast<double>(a.tol) * a.tol * rr;
            conv = rr == 0.0;
            while (!conv && it < a.maxit) {
                // U0 <- E p ; U0 <- B^{-1} U0
                const int tot = X.m1 * X.ncolmax;
                for (int e = threadIdx.x; e < tot; e += DCT_T) sm.U0[e] = make_float2(0.f, 0.f);
                __syncthreads();
                for (int i = threadIdx.x; i < kc; i += DCT_T) U0f[c_loc[i]] = c_p[i];
                __syncthreads();
                dct_forward_inplace(X, sm.U0, sm.tw1, sm.tw2, cl);
                apply_filter(X, sm.U0, fscale, alpha, s2, true);
                dct_inverse_inplace(X, sm.U0, sm.tw1, sm.tw2, cl);
                double pq_loc = 0.0;
                for (int i = threadIdx.x; i < kc; i += DCT_T) {
                    const float v = U0f[c_loc[i]];
                    c_q[i] = v;
                    pq_loc += static_cast<double>(c_p[i]) * v;
                }
                const double pq = cluster_sum2(make_double2(pq_loc, 0.0), s_red, s_part, parity, cl).x;
                const float alp = static_cast<float>(rr / pq);
                double rn_loc = 0.0;
                for (int i = threadIdx.x; i < kc; i += DCT_T) {
                    c_y[i] = fmaf(alp, c_p[i], c_y[i]);
                    const float rv = fmaf(-alp, c_q[i], c_r[i]);
                    c_r[i] = rv;
                    rn_loc += static_cast<double>(rv) * rv;
                }
                const double rn = cluster_sum2(make_double2(rn_loc, 0.0), s_red, s_part, parity, cl).x;
                ++it;
                if (rn <= stop) { conv = true; break; }
                const float beta = static_cast<float>(rn / rr);
                for (int i = threadIdx.x; i < kc; i += DCT_T) c_p[i] = fmaf(beta, c_p[i], c_r[i]);
                __syncthreads();
                rr = rn;
            }
            // x = x0 + B^{-1} E y
            const int tot = X.m1 * X.ncolmax;
            for (int e = threadIdx.x; e < tot; e += DCT_T) sm.U0[e] = make_float2(0.f, 0.f);
            __syncthreads();
            for (int i = threadIdx.x; i < kc; i += DCT_T) U0f[c_loc[i]] = c_y[i];
            __syncthreads();
            dct_forward_inplace(X, sm.U0, sm.tw1, sm.tw2, cl);
            apply_filter(X, sm.U0, fscale, alpha, s2, false);
            dct_inverse_inplace(X, sm.U0, sm.tw1, sm.tw2, cl);
            for (int e = threadIdx.x; e < tot; e += DCT_T)
                sm.U1[e] = cadd(sm.U1[e], sm.U0[e]);
            __syncthreads();
            if (!conv) set_status(a.status, q, TOD_ERR_NOT_CONVERGED);
        }
        // store x (time layout -> samples)
        {
            const int tot = X.m1 * X.ncolmax;
            float *xq = a.x_out + o;
            for (int e = threadIdx.x; e < tot; e += DCT_T) {
                int t0, t1;
                bool valid;
                elem_samples(X, e, t0, t1, valid);
                if (!valid) continue;
                const float2 v = sm.U1[e];
                xq[t0] = v.x;
                xq[t1] = v.y;
            }
        }
        if (a.iters && c == 0 && threadIdx.x == 0) a.iters[q] = it;
        // U0/U1 of this CTA may still be read remotely by the last transpose of
        // a sibling: the next detscan starts with load_plan + local writes only
        // after this barrier.
        cl.sync();
    }
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
static size_t smem_bytes(const Plan &p, bool ncorr)
{
    size_t b = sizeof(float2) * (2 * static_cast<size_t>(p.sz) + p.m1max + p.m2max);
    if (ncorr) b += static_cast<size_t>(CG_KCAP) * (sizeof(int) + 4 * sizeof(float));
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

cudaError_t setup_dct_kernels(Plan &p)
{
    p.smem_gain = smem_bytes(p, false);
    p.smem_ncorr = smem_bytes(p, true);
    cudaError_t e;
    e = cudaFuncSetAttribute(k_gain, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(p.smem_gain));
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(k_ncorr, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(p.smem_ncorr));
    if (e != cudaSuccess) return e;
    if (p.C > 8) {
        e = cudaFuncSetAttribute(k_gain, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
        if (e != cudaSuccess) return e;
        e = cudaFuncSetAttribute(k_ncorr, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
        if (e != cudaSuccess) return e;
    }
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
    a.g_out = g; a.mu_out = mu; a.sig_out = sig; a.status = p.status; a.sz = p.sz;
    a.m1max = p.m1max; a.m2max = p.m2max;
    if (p.schedule == TOD_SCHED_PER_SCAN) {
        for (int w = 0; w < work_count; ++w) {
            a.work_begin = work_begin + w;
            a.work_count = 1;
            cudaError_t e = launch_cluster(reinterpret_cast<const void *>(k_gain), &a, p.C, 1, p.smem_gain, st);
            if (e != cudaSuccess) return e;
        }
        return cudaSuccess;
    }
    const int ncl = std::min(work_count, p.nclusters_gain);
    return launch_cluster(reinterpret_cast<const void *>(k_gain), &a, p.C, ncl, p.smem_gain, st);
}

cudaError_t launch_ncorr(const Plan &p, const float *d, const float *s, const double *gain,
                         const uint32_t *flags, const double *psd, tod_rng rng, int mode,
                         float tol, int maxit, float *x, int32_t *iters, cudaStream_t st,
                         int work_begin, int work_count)
{
    if (work_count <= 0) return cudaSuccess;
    NcorrArgs a;
    a.d = d; a.s = s; a.gain = gain; a.flags = flags; a.psd = psd; a.off = p.off; a.plans = p.plans;
    a.q_plan = p.q_plan; a.tw = p.tw; a.work = p.work; a.work_begin = work_begin;
    a.work_count = work_count; a.ndet = p.ndet; a.fsamp = p.fsamp; a.rng = rng; a.mode = mode;
    a.tol = tol; a.maxit = maxit; a.x_out = x; a.iters = iters; a.status = p.status; a.sz = p.sz;
    a.m1max = p.m1max; a.m2max = p.m2max;
    if (p.schedule == TOD_SCHED_PER_SCAN) {
        for (int w = 0; w < work_count; ++w) {
            a.work_begin = work_begin + w;
            a.work_count = 1;
            cudaError_t e = launch_cluster(reinterpret_cast<const void *>(k_ncorr), &a, p.C, 1, p.smem_ncorr, st);
            if (e != cudaSuccess) return e;
        }
        return cudaSuccess;
    }
    const int ncl = std::min(work_count, p.nclusters_ncorr);
    return launch_cluster(reinterpret_cast<const void *>(k_ncorr), &a, p.C, ncl, p.smem_ncorr, st);
}

}  // namespace tg
