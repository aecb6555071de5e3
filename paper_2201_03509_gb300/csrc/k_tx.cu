// A3 batched DCT-II (the mirrored FFT of Sect. 4.2) as passes through
// memory, and on it A4 (gain draw), A5 (correlated-noise draw with CG gap
// filling; Eq. `gibbsstart`, Sect. 5) and A8 (TOD chi^2 and gradients).
//
// A length-n real DCT-II is an m = n/2 complex FFT of the even/odd-packed,
// reversed-odd sequence z_j = (v_{2j}, v_{2j+1}), v_i = x_{2i} (i < m),
// x_{2n-1-2i} (i >= m) (Makhoul 1980), plus a real split.  The FFT is
// four-step, m = m1 x m2, with j = j1 m2 + j2 and k = k1 + m1 k2:
//   column pass: for a tile of column pairs {c, m2-1-c}: FFTs of length m1
//     along j1, times W_m^{c k1}, written row-major to the intermediate Y;
//     z_j and z_{m-1-j} together are the four samples x_{4j..4j+3}, so the
//     tile reads and writes whole runs of samples;
//   row pass: for a tile of row pairs {k1, m1-k1}: FFTs of length m2 along
//     k2, the real split (Z_k with Z_{m-k}) into packed orthonormal
//     coefficients (X_k, X_{n-k}) (slot 0: (X_0, X_m)), a per-mode filter,
//     the inverse split and inverse FFTs, written back to Y;
//   inverse column pass: times W_m^{-c k1}, inverse FFTs, samples out.
// Every tile is independent: a CTA holds one tile in shared memory, passes
// are separate grid-wide phases, and the intermediate goes through L2/HBM.
#include <cooperative_groups.h>
#include "fft_reg.cuh"

namespace cgrp = cooperative_groups;

namespace tg {

// ---------------------------------------------------------------------------
// per-item context
// ---------------------------------------------------------------------------
struct TxCtx {
    TxLen L;
    float s2, inv_s2, inv_s, fscale, alpha, g;   // detector noise, detscan gain
    int q, blk, det;
    int mode;                                    // CgState mode of the detscan (n_corr)
    int64_t o;                                   // first sample of the detscan
    int64_t yb;                                  // first complex value of its Y block
    int64_t koff;                                // first flagged rank (n_corr)
};

// Copy the length plan of item (q, blk) into shared memory (skipped when the
// previous item had the same length) and set the detscan scalars.  All
// threads call it; it ends with a barrier.
__device__ __forceinline__ void tx_begin(TxCtx &X, const TxLen *__restrict__ txl, const int32_t *__restrict__ q_tx,
                                         const int64_t *__restrict__ off, int q, int blk, int64_t obase, int ndet,
                                         double fsamp, const double *psd, const double *gain, int &cur,
                                         const float4 *__restrict__ qsc = nullptr)
{
    __syncthreads();                 // earlier readers of X are done
    const int li = q_tx[q];
    if (li != cur) {
        const int4 *src = reinterpret_cast<const int4 *>(txl + li);
        int4 *dst = reinterpret_cast<int4 *>(&X.L);
        for (int i = threadIdx.x; i < static_cast<int>(sizeof(TxLen) / 16); i += blockDim.x) dst[i] = src[i];
    }
    if (threadIdx.x == 0) {
        X.q = q;
        X.blk = blk;
        X.det = q % ndet;
        X.o = off[q];
        X.yb = (off[q] - obase) >> 1;
        if (qsc) {          // precomputed for this call: (s2, 1/s2, 1/s, fscale), (alpha, g, -, -)
            const float4 a0 = qsc[2 * q], a1 = qsc[2 * q + 1];
            X.s2 = a0.x; X.inv_s2 = a0.y; X.inv_s = a0.z; X.fscale = a0.w;
            X.alpha = a1.x;
            X.g = a1.y;
        } else if (psd) {
            const double sig0 = psd[3 * X.det], fk = psd[3 * X.det + 1], al = psd[3 * X.det + 2];
            const int n = static_cast<int>(off[q + 1] - off[q]);
            X.s2 = static_cast<float>(sig0 * sig0);
            X.inv_s2 = static_cast<float>(1.0 / (sig0 * sig0));
            X.inv_s = static_cast<float>(1.0 / sig0);
            X.fscale = static_cast<float>(fsamp / (2.0 * n * fk));
            X.alpha = static_cast<float>(al);
        }
        if (!qsc) X.g = gain ? static_cast<float>(gain[q]) : 1.0f;
    }
    cur = li;
    __syncthreads();
}

// The FP32 scalars of every detscan of a call, from the FP64 noise
// parameters (and gains): (sigma0^2, 1/sigma0^2, 1/sigma0, fsamp/(2 n f_knee)),
// (alpha, g, 0, 0).  Computed once per call instead of in every tile.
__device__ __forceinline__ void det_scalars_q(const double *psd, const double *gain, const int64_t *off, int ndet,
                                              double fsamp, int q, float4 *qsc)
{
    const int det = q % ndet;
    const double sig0 = psd[3 * det], fk = psd[3 * det + 1], al = psd[3 * det + 2];
    const double n = static_cast<double>(off[q + 1] - off[q]);
    qsc[2 * q] = make_float4(static_cast<float>(sig0 * sig0), static_cast<float>(1.0 / (sig0 * sig0)),
                             static_cast<float>(1.0 / sig0), static_cast<float>(fsamp / (2.0 * n * fk)));
    qsc[2 * q + 1] = make_float4(static_cast<float>(al), gain ? static_cast<float>(gain[q]) : 1.0f, 0.f, 0.f);
}
__global__ void k_det_scalars(const double *__restrict__ psd, const double *__restrict__ gain,
                              const int64_t *__restrict__ off, int ndet, double fsamp, int q0, int q1,
                              float4 *__restrict__ qsc)
{
    const int q = q0 + blockIdx.x * blockDim.x + threadIdx.x;
    if (q < q1) det_scalars_q(psd, gain, off, ndet, fsamp, q, qsc);
}

// This CTA's contiguous share [i0, i1) of nitems work items: consecutive
// items of a CTA are mostly tiles of one detscan (same length: the plan
// copy and the twiddles stay hot).
__device__ __forceinline__ void cta_share(int nitems, int &i0, int &i1) {
    const int per = (nitems + gridDim.x - 1) / gridDim.x;
    i0 = min(nitems, static_cast<int>(blockIdx.x) * per);
    i1 = min(nitems, i0 + per);
}

// The SFU's approximate base-2 logarithm and exponential and reciprocal
// (PTX lg2/ex2/rcp.approx: absolute error about 2^-22 in the logarithm,
// relative about 2^-22 in the others).  Used for the per-mode noise weights,
// where their error (below 1e-6 relative in a weight) is far inside the
// transforms' FP32 budget.
__device__ __forceinline__ float sfu_lg2(float x) {
    float y;
    asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float sfu_ex2(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float sfu_rcp(float x) {
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// (f_k / f_knee)^alpha at DCT mode k >= 1, FP32 (fscale = fsamp / (2 n f_knee))
__device__ __forceinline__ float tx_fpow(int k, float fscale, float alpha) {
    return sfu_ex2(alpha * sfu_lg2(static_cast<float>(k) * fscale));
}

// twiddle block of a length: W_m1^i, W_m2^i, W_4n^{k1}, W_4n^{m1 k2},
// W_4n^{5 k1}, W_4n^{5 m1 k2}, W_m^{64 i}, W_m^i (i < 64)
template <class V> struct TwB {
    const V *tw1, *tw2, *sa1, *sb1, *sa5, *sb5, *t4hi, *t4lo;
    __device__ __forceinline__ TwB(const V *base, const TxLen &L) {
        tw1 = base;
        tw2 = tw1 + L.m1;
        sa1 = tw2 + L.m2;
        sb1 = sa1 + L.m1;
        sa5 = sb1 + L.m2;
        sb5 = sa5 + L.m1;
        t4hi = sb5 + L.m2;
        t4lo = t4hi + L.m / 64 + 1;
    }
    __device__ __forceinline__ V w4(int r) const { return vmul(vld(t4hi + (r >> 6)), vld(t4lo + (r & 63))); }
};

// ---------------------------------------------------------------------------
// column tiles: pairs p in [p0, p0 + np), tile column lc = side * TP + i
// (side 0: column p0 + i; side 1: column m2-1-p0-i, absent when it is the
// middle column already held by side 0); element (j1, lc) at j1 * W + lc.
// ---------------------------------------------------------------------------
struct ColGeo {
    int n, m, m1, m2, P2, TP, W, p0, np, m1h;
    __device__ __forceinline__ ColGeo(const TxLen &L, int blk) {
        n = L.n; m = L.m; m1 = L.m1; m2 = L.m2; P2 = L.P2; TP = L.TP; W = 2 * L.TP;
        p0 = blk * TP;
        np = min(TP, P2 - p0);
        m1h = (m1 + 1) >> 1;
    }
    __device__ __forceinline__ int col(int lc) const {     // -1: no column
        const int side = lc >= TP, i = lc - side * TP;
        if (i >= np) return -1;
        const int p = p0 + i;
        if (!side) return p;
        const int c = m2 - 1 - p;
        return c == p ? -1 : c;
    }
    __device__ __forceinline__ int lcol(int c) const { return c < P2 ? c - p0 : TP + (m2 - 1 - c - p0); }
};

// flagged-sample mask (bit u: sample t + u) of samples t..t+cnt-1, cnt <= 4
__device__ __forceinline__ uint32_t flag_bits(const uint32_t *__restrict__ fl, int64_t t, int cnt) {
    const int64_t w = t >> 5;
    const int b = static_cast<int>(t & 31);
    uint32_t v = __ldg(fl + w) >> b;
    if (b + cnt > 32) v |= __ldg(fl + w + 1) << (32 - b);
    return v & ((1u << cnt) - 1u);
}

// The four samples of unit j (x_{4j..4j+3}; two at the centre j = m-1-j):
// load them as z_j = (x0, x2), z_{m-1-j} = (x3, x1).
__device__ __forceinline__ float4 ld4(const float *__restrict__ x, int64_t t, bool centre) {
    const float2 a = __ldg(reinterpret_cast<const float2 *>(x + t));
    if (centre) return make_float4(a.x, a.y, 0.f, 0.f);
    const float2 b = __ldg(reinterpret_cast<const float2 *>(x + t + 2));
    return make_float4(a.x, a.y, b.x, b.y);
}

// Asynchronous global -> shared copies (cp.async, Ampere and later): every
// copy of a tile is in flight at once; cp_wait ends them (a barrier must
// follow before other threads read the tile).
__device__ __forceinline__ void cp_async(float2 *dst, const float2 *src) {
    const uint32_t d = static_cast<uint32_t>(__cvta_generic_to_shared(dst));
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async(double2 *dst, const double2 *src) {
    const uint32_t d = static_cast<uint32_t>(__cvta_generic_to_shared(dst));
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_wait() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

constexpr int TX_UNR = 4;     // units per thread whose loads are issued together

// Column tiles have 2 TP = W columns with W a power of two dividing TX_T:
// thread t keeps column lc = t mod W and takes rows t / W, t / W + TX_T / W,
// ..., so a column's index arithmetic is done once per thread.
struct ColThread {
    int lc, c, r0, rstep, cpart, lpart;   // own column, its index, first row, row step; partner column and slot
    __device__ __forceinline__ ColThread(const ColGeo &G) {
        lc = threadIdx.x & (G.W - 1);
        r0 = threadIdx.x / G.W;
        rstep = TX_T / G.W;
        c = G.col(lc);
        cpart = c < 0 ? -1 : G.m2 - 1 - c;
        lpart = c < 0 ? -1 : G.lcol(cpart);
    }
};

// The flag bits of a thread's units, loaded ahead of the transform (all
// loads in flight together): bit 4i + u is sample u of the thread's i-th
// unit (rows r0, r0 + rstep, ..; at most TX_TILE / 512 <= 8 units).  Zero
// without flags (fl null) or for a thread without a column.
__device__ __forceinline__ uint32_t unit_flags(const ColGeo &G, const ColThread &C, const uint32_t *__restrict__ fl,
                                               int64_t o)
{
    uint32_t nib = 0;
    if (!fl || C.c < 0) return nib;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const int j1 = C.r0 + i * C.rstep;
        const int j = j1 * G.m2 + C.c;
        if (j1 < G.m1h && j <= G.m - 1 - j)
            nib |= flag_bits(fl, o + 4 * static_cast<int64_t>(j), j == G.m - 1 - j ? 2 : 4) << (4 * i);
    }
    return nib;
}

// Forward column pass.  For every unit j <= m-1-j of the tile (the four
// samples x_{4j..4j+3}, two at the centre j = m-1-j): D = ld(j, centre, fb)
// issues the unit's loads (TX_UNR units per thread at a time; fb: the
// unit's flag bits, from fl at sample o + 4j, read ahead), then
// put(D, ea, eb, j, jm, tile, fb) writes z_j at tile element ea = (j1, lc) and
// z_{m-1-j} at eb = (m1-1-j1, lcol(m2-1-c)).  pre(tile) runs first (after the columns a
// ragged tile lacks are zeroed), with a barrier before the units.  Then
// the column FFTs, the twiddle, and the tile out to Y.
template <class V, class Pre, class Ld, class Put>
__device__ __forceinline__ void col_forward(const TxCtx &X, V *b0, V *b1, V *__restrict__ Y, const V *__restrict__ twb,
                                            const uint32_t *__restrict__ fl, Pre pre, Ld ld, Put put)
{
    const ColGeo G(X.L, X.blk);
    const ColThread C(G);
    const int W = G.W, m1 = G.m1, m2 = G.m2;
    if (C.c < 0)
        for (int j1 = C.r0; j1 < m1; j1 += C.rstep) b0[j1 * W + C.lc] = vzero<V>();
    pre(b0);
    const uint32_t fnib = unit_flags(G, C, fl, X.o);
    __syncthreads();
    if (C.c >= 0) {
        for (int j10 = C.r0, i0 = 0; j10 < G.m1h; j10 += TX_UNR * C.rstep, i0 += TX_UNR) {
            decltype(ld(0, false, 0u)) D[TX_UNR];
            bool ok[TX_UNR];
#pragma unroll
            for (int k = 0; k < TX_UNR; ++k) {
                const int j1 = j10 + k * C.rstep;
                const int j = j1 * m2 + C.c;
                ok[k] = j1 < G.m1h && j <= G.m - 1 - j;
                if (ok[k]) D[k] = ld(j, j == G.m - 1 - j, (fnib >> (4 * (i0 + k))) & 15u);
            }
#pragma unroll
            for (int k = 0; k < TX_UNR; ++k) {
                if (!ok[k]) continue;
                const int j1 = j10 + k * C.rstep;
                const int j = j1 * m2 + C.c;
                put(D[k], j1 * W + C.lc, (m1 - 1 - j1) * W + C.lpart, j, G.m - 1 - j, b0,
                    (fnib >> (4 * (i0 + k))) & 15u);
            }
        }
    }
    __syncthreads();
    const TwB<V> T(twb, X.L);
    V *R = sp_transform<false, TX_T, true>(b0, b1, m1, X.L.s1, X.L.nr1, X.L.lgW, 0, T.tw1);
    if (C.c < 0) return;
    V *Yq = Y + X.yb + C.c;
    // W_m^{c k1} from the table at the first row of every TX_UNR rows, then
    // by steps of W_m^{c rstep} (at most TX_UNR - 1 products from an exact value)
    const V wstep = C.rstep < m1 ? T.w4(C.c * C.rstep) : vzero<V>();
    for (int k10 = C.r0; k10 < m1; k10 += TX_UNR * C.rstep) {
        V w = T.w4(C.c * k10);
#pragma unroll
        for (int k = 0; k < TX_UNR; ++k) {
            const int k1 = k10 + k * C.rstep;
            if (k1 < m1) Yq[static_cast<int64_t>(k1) * m2] = vmul(R[k1 * W + C.lc], w);
            if (k + 1 < TX_UNR) w = vmul(w, wstep);
        }
    }
}

// Inverse column pass: the tile's Y values copied in asynchronously,
// twiddled in place, inverse FFT of the columns; then for every unit
// j <= m-1-j: D = ld(j, centre, fb) (issued TX_UNR units at a time) and
// out(D, ea, eb, j, jm, tile, fb) with ea, eb, fb as for the forward pass
// (the flag bits are read while the tile loads).
template <class V, class Ld, class Out>
__device__ __forceinline__ void col_inverse(const TxCtx &X, V *b0, V *b1, const V *__restrict__ Y,
                                            const V *__restrict__ twb, const uint32_t *__restrict__ fl, Ld ld,
                                            Out out)
{
    const ColGeo G(X.L, X.blk);
    const ColThread C(G);
    const int W = G.W, m1 = G.m1, m2 = G.m2;
    const TwB<V> T(twb, X.L);
    uint32_t fnib = 0;
    if (C.c < 0) {
        for (int k1 = C.r0; k1 < m1; k1 += C.rstep) b0[k1 * W + C.lc] = vzero<V>();
    } else {
        const V *Yq = Y + X.yb + C.c;
        for (int k1 = C.r0; k1 < m1; k1 += C.rstep) cp_async(b0 + k1 * W + C.lc, Yq + static_cast<int64_t>(k1) * m2);
        fnib = unit_flags(G, C, fl, X.o);
        cp_wait();
        // the conjugate four-step twiddle, stepped as in the forward pass
        const V wstep = C.rstep < m1 ? T.w4(C.c * C.rstep) : vzero<V>();
        for (int k10 = C.r0; k10 < m1; k10 += TX_UNR * C.rstep) {
            V w = T.w4(C.c * k10);
#pragma unroll
            for (int k = 0; k < TX_UNR; ++k) {
                const int k1 = k10 + k * C.rstep;
                if (k1 < m1) b0[k1 * W + C.lc] = vmulc(b0[k1 * W + C.lc], w);
                if (k + 1 < TX_UNR) w = vmul(w, wstep);
            }
        }
    }
    __syncthreads();
    V *R = sp_transform<true, TX_T, true>(b0, b1, m1, X.L.s1, X.L.nr1, X.L.lgW, 0, T.tw1);
    if (C.c < 0) return;
    for (int j10 = C.r0, i0 = 0; j10 < G.m1h; j10 += TX_UNR * C.rstep, i0 += TX_UNR) {
        decltype(ld(0, false, 0u)) D[TX_UNR];
        bool ok[TX_UNR];
#pragma unroll
        for (int k = 0; k < TX_UNR; ++k) {
            const int j1 = j10 + k * C.rstep;
            const int j = j1 * m2 + C.c;
            ok[k] = j1 < G.m1h && j <= G.m - 1 - j;
            if (ok[k]) D[k] = ld(j, j == G.m - 1 - j, (fnib >> (4 * (i0 + k))) & 15u);
        }
#pragma unroll
        for (int k = 0; k < TX_UNR; ++k) {
            if (!ok[k]) continue;
            const int j1 = j10 + k * C.rstep;
            const int j = j1 * m2 + C.c;
            out(D[k], j1 * W + C.lc, (m1 - 1 - j1) * W + C.lpart, j, G.m - 1 - j, R, (fnib >> (4 * (i0 + k))) & 15u);
        }
    }
}

// ---------------------------------------------------------------------------
// row tiles: row pairs p in [r0, r0 + nr); slot 2i is row r0 + i, slot
// 2i+1 row m1 - r0 - i (unused when that row is the same, or r0 + i = 0);
// element (slot, k2) at slot * m2p + k2.
// ---------------------------------------------------------------------------
struct RowGeo {
    int n, m, m1, m2, m2p, r0, nr, TR;
    __device__ __forceinline__ RowGeo(const TxLen &L, int blk) {
        n = L.n; m = L.m; m1 = L.m1; m2 = L.m2; m2p = L.m2p; TR = L.TR;
        r0 = blk * TR;
        nr = min(TR, L.P1 - r0);
    }
    __device__ __forceinline__ int row(int slot) const {   // -1: unused
        const int i = slot >> 1;
        if (i >= nr) return -1;
        const int p = r0 + i;
        if (!(slot & 1)) return p;
        const int r = m1 - p;
        return (p == 0 || r == p) ? -1 : r;
    }
};

// The split's twiddles of mode k: e1 = W_4n^k, e5 = W_4n^{5k} (for
// k = k1 + m1 k2 the products of a per-row and a per-column table entry).
template <class V> struct SplitTw { V e1, e5; };
// Packed orthonormal coefficients of slot k from Z_k, Z_{m-k} (forward
// half-split): W = e^{-i pi k/2n} A + e^{-i 5 pi k/2n} B.
template <class V>
__device__ __forceinline__ V split_f(const SplitTw<V> &w, V a, V b, typename VecT<V>::S sq) {
    typedef typename VecT<V>::S S;
    const V cb = vconj(b);
    const V A = vscale(vadd(a, cb), static_cast<S>(0.5));
    const V d = vsub(a, cb);
    const V Bv = vmake<V>(static_cast<S>(0.5) * d.y, static_cast<S>(-0.5) * d.x);
    const V Wv = vadd(vmul(w.e1, A), vmul(w.e5, Bv));
    return vmake<V>(sq * Wv.x, -sq * Wv.y);
}
// Z_k from the packed slots k and m-k (inverse half-split; sq includes 1/m).
template <class V>
__device__ __forceinline__ V split_i(const SplitTw<V> &wk, const SplitTw<V> &wp, V yk, V yp,
                                     typename VecT<V>::S sq) {
    typedef typename VecT<V>::S S;
    const V Vk = vscale(vmulc(vconj(yk), wk.e1), sq);
    const V Vp = vscale(vmulc(vconj(yp), wp.e1), sq);
    const V cVp = vconj(Vp);
    const V A = vscale(vadd(Vk, cVp), static_cast<S>(0.5));
    const V e4 = vmulc(wk.e5, wk.e1);                                   // W_4n^{4k} = e^{-2 pi i k/n}
    const V Bv = vscale(vmulc(vsub(Vk, cVp), e4), static_cast<S>(0.5));
    return vmake<V>(A.x - Bv.y, A.y + Bv.x);
}

// Row pass.  Loads the tile's rows from Y, forward row FFTs, then
// pre(nubuf) (a second tile-sized buffer, or null when pre needs none; a
// barrier follows), then for every packed slot:
// Y' = f(e, k, Y) (e: tile element, k: slot, Y = (X_k, X_{n-k}) or (X_0, X_m));
// with INV_BACK the inverse split and inverse row FFTs follow and the rows go
// back to Y.  Rows are taken one at a time (their index is uniform over
// the CTA), the threads over k2.
template <class V, bool INV_BACK, class Pre, class F>
__device__ __forceinline__ void row_pass(const TxCtx &X, V *b0, V *b1, V *__restrict__ Y, const V *__restrict__ twb,
                                         Pre pre, F f)
{
    typedef typename VecT<V>::S S;
    const RowGeo G(X.L, X.blk);
    const int m1 = G.m1, m2 = G.m2, m2p = G.m2p;
    const int nslot = 2 * G.TR;
    const int tid = threadIdx.x;
    V *Yq = Y + X.yb;
    for (int sl = 0; sl < nslot; ++sl) {
        const int r = G.row(sl);
        V *dst = b0 + sl * m2p;
        if (r < 0) {
            for (int k2 = tid; k2 < m2; k2 += TX_T) dst[k2] = vzero<V>();
        } else {
            const V *src = Yq + static_cast<int64_t>(r) * m2;
            for (int k2 = tid; k2 < m2; k2 += TX_T) cp_async(dst + k2, src + k2);
        }
    }
    cp_wait();
    __syncthreads();
    const TwB<V> T(twb, X.L);
    V *R = sp_transform<false, TX_T, false>(b0, b1, m2, X.L.s2, X.L.nr2, X.L.lgS, m2p, T.tw2);
    V *Fr = R == b0 ? b1 : b0;
    pre(Fr);
    __syncthreads();
    const S sqf = static_cast<S>(X.L.sq_fwd), s0f = static_cast<S>(X.L.s0_fwd);
    const S sqi = static_cast<S>(X.L.sq_inv), s0i = static_cast<S>(X.L.s0_inv);
    for (int pl = 0; pl < G.nr; ++pl) {
        const int p = G.r0 + pl;
        const bool mid = 2 * p == m1;                 // the row pairs with itself
        // elements (pl, k2) for k2 < cnt; each pairs with mode m - k
        const int cnt = (p == 0) ? (m2 / 2 + 1) : (mid ? (m2 + 1) / 2 : m2);
        const int rowa = 2 * pl * m2p, rowb = (p == 0 || mid) ? rowa : rowa + m2p;
        const V a1 = vld(T.sa1 + p), a5 = vld(T.sa5 + p);
        for (int k2 = tid; k2 < cnt; k2 += TX_T) {
            const int q2 = (p == 0) ? (k2 == 0 ? 0 : m2 - k2) : m2 - 1 - k2;
            const int ia = rowa + k2, ib = rowb + q2;
            const V Za = R[ia], Zb = R[ib];
            const int ka = p + m1 * k2;
            if (ka == 0) {
                V Yv = vmake<V>((Za.x + Za.y) * s0f, (Za.x - Za.y) * s0f);
                Yv = f(ia, 0, Yv);
                if (INV_BACK) {
                    const S V0 = Yv.x * s0i, Vm = Yv.y * s0i;
                    R[ia] = vmake<V>(static_cast<S>(0.5) * (V0 + Vm), static_cast<S>(0.5) * (V0 - Vm));
                }
                continue;
            }
            SplitTw<V> wa;
            wa.e1 = vmul(a1, vld(T.sb1 + k2));
            wa.e5 = vmul(a5, vld(T.sb5 + k2));
            if (ib == ia) {                           // the mode pairs with itself
                V Ya = split_f(wa, Za, Zb, sqf);
                Ya = f(ia, ka, Ya);
                if (INV_BACK) R[ia] = split_i(wa, wa, Ya, Ya, sqi);
                continue;
            }
            // Both slots of the pair at once (modes k and m - k, whose split
            // twiddles are e1' = w conj(e1), e5' = -w conj(e5), w = e^{-i pi/4}):
            // with P = e1 (Za + conj Zb), Q = e5 (-i)(Za - conj Zb),
            // Y_k = (sq/2) conj(P + Q) and Y_{m-k} = (sq/2) conj(w) (P - Q).
            const V sum = vmake<V>(Za.x + Zb.x, Za.y - Zb.y), dif = vmake<V>(Za.x - Zb.x, Za.y + Zb.y);
            const V P = vmul(wa.e1, sum), Q = vmul(wa.e5, vmake<V>(dif.y, -dif.x));
            const S hq = static_cast<S>(0.5) * sqf;
            const S h = static_cast<S>(0.70710678118654752440);
            const V pm = vsub(P, Q);
            V Ya = vmake<V>(hq * (P.x + Q.x), -hq * (P.y + Q.y));
            V Yb = vmake<V>(hq * h * (pm.x - pm.y), hq * h * (pm.x + pm.y));
            Ya = f(ia, ka, Ya);
            Yb = f(ib, G.m - ka, Yb);
            if (INV_BACK) {
                // U_a = (sqi/2) conj(Y_k) conj(e1), U_b = (sqi/2) conj(Y_{m-k}) conj(w) e1;
                // S = U_a + conj(U_b), G = (U_a - conj(U_b)) conj(e4), e4 = e5 conj(e1);
                // Z_k = S + i G, Z_{m-k} = conj(S) + i conj(G)
                const S hi = static_cast<S>(0.5) * sqi;
                const V Ua = vscale(vmulc(vconj(Ya), wa.e1), hi);
                const V cb = vmul(vconj(Yb), wa.e1);
                const V Ub = vscale(vmake<V>(h * (cb.x - cb.y), h * (cb.x + cb.y)), hi);
                const V Sv = vmake<V>(Ua.x + Ub.x, Ua.y - Ub.y);
                const V Dv = vmake<V>(Ua.x - Ub.x, Ua.y + Ub.y);
                const V Gv = vmulc(Dv, vmulc(wa.e5, wa.e1));
                R[ia] = vmake<V>(Sv.x - Gv.y, Sv.y + Gv.x);
                R[ib] = vmake<V>(Sv.x + Gv.y, Gv.x - Sv.y);
            }
        }
    }
    if (!INV_BACK) return;
    __syncthreads();
    V *Ri = sp_transform<true, TX_T, false>(R, Fr, m2, X.L.s2, X.L.nr2, X.L.lgS, m2p, T.tw2);
    for (int sl = 0; sl < nslot; ++sl) {
        const int r = G.row(sl);
        if (r < 0) continue;
        const V *src = Ri + sl * m2p;
        V *dst = Yq + static_cast<int64_t>(r) * m2;
        for (int k2 = tid; k2 < m2; k2 += TX_T) dst[k2] = src[k2];
    }
}

// ---------------------------------------------------------------------------
// CTA reductions: FP32 double-word partials, warps merged by shuffles, the
// warp results added in FP64 in a fixed order by thread 0.
// ---------------------------------------------------------------------------
__device__ __forceinline__ Acc2 acc_merge_tx(const Acc2 &a, const Acc2 &b) {
    Acc2 r = a;
    acc_add(r, b.s);
    r.c = __fadd_rn(r.c, b.c);
    return r;
}
__device__ __forceinline__ Acc2 warp_acc(Acc2 x) {
#pragma unroll
    for (int o = 16; o; o >>= 1) {
        Acc2 y;
        y.s = __shfl_xor_sync(0xffffffffu, x.s, o);
        y.c = __shfl_xor_sync(0xffffffffu, x.c, o);
        x = acc_merge_tx(x, y);
    }
    return x;
}
// NV values per thread summed over the CTA; the totals land in out[0..NV)
// (shared) for every thread after the call.  s_red holds NV * TX_T/32.
template <int NV>
__device__ __forceinline__ void block_sums(const Acc2 (&a)[NV], double *s_red, double *out) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
    for (int v = 0; v < NV; ++v) {
        const Acc2 w = warp_acc(a[v]);
        if (lane == 0) s_red[v * (TX_T / 32) + warp] = acc_value(w);
    }
    __syncthreads();
    if (threadIdx.x < NV) {
        double t = 0.0;
        for (int w = 0; w < TX_T / 32; ++w) t += s_red[threadIdx.x * (TX_T / 32) + w];
        out[threadIdx.x] = t;
    }
    __syncthreads();
}
template <int NV>
__device__ __forceinline__ void block_sums_d(const double (&a)[NV], double *s_red, double *out) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
    for (int v = 0; v < NV; ++v) {
        double x = a[v];
#pragma unroll
        for (int o = 16; o; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
        if (lane == 0) s_red[v * (TX_T / 32) + warp] = x;
    }
    __syncthreads();
    if (threadIdx.x < NV) {
        double t = 0.0;
        for (int w = 0; w < TX_T / 32; ++w) t += s_red[threadIdx.x * (TX_T / 32) + w];
        out[threadIdx.x] = t;
    }
    __syncthreads();
}

// ===========================================================================
// A4: gain.  a = sum_{k>=1} shat_k^2 / P_k (row pass), u = C^T(shat / P) and
// b = sum_t M_t d_t u_t (inverse column pass): b = sum_k shat_k dhat_k / P_k.
// ===========================================================================
struct GainTx {
    const float *d, *s;
    const uint32_t *flags;
    const double *psd;
    const int64_t *off;
    const TxLen *txl;
    const int32_t *q_tx;
    const float2 *tw;
    const int2 *items;
    int item0, nitems;
    int ndet;
    double fsamp;
    int64_t obase;
    float2 *Y;
    double *part;                 // [item][4]
    const float4 *qsc;            // per-detscan FP32 scalars of the call
};

__global__ void __launch_bounds__(TX_T, 3) k_gain_cols(GainTx a)
{
    extern __shared__ __align__(16) float2 tx_smem[];
    __shared__ TxCtx X;
    float2 *b0 = tx_smem, *b1 = tx_smem + TX_TILE;
    int cur = -1;
    int i0, i1;
    cta_share(a.nitems, i0, i1);
    for (int it = i0; it < i1; ++it) {
        const int2 w = a.items[a.item0 + it];
        tx_begin(X, a.txl, a.q_tx, a.off, w.x, w.y, a.obase, a.ndet, a.fsamp, nullptr, nullptr, cur);
        const float *sq = a.s + X.o;
        col_forward(X, b0, b1, a.Y, a.tw + X.L.twb, a.flags, [](float2 *) {},
                    [&](int j, bool ctr, uint32_t) { return ld4(sq, 4 * static_cast<int64_t>(j), ctr); },
                    [&](const float4 &v, int ea, int eb, int j, int jm, float2 *U, uint32_t fb) {
                        const float x0 = (fb & 1) ? 0.f : v.x, x1 = (fb & 2) ? 0.f : v.y;
                        const float x2 = (fb & 4) ? 0.f : v.z, x3 = (fb & 8) ? 0.f : v.w;
                        if (j == jm) { U[ea] = make_float2(x0, x1); return; }
                        U[ea] = make_float2(x0, x2);
                        U[eb] = make_float2(x3, x1);
                    });
    }
}

__global__ void __launch_bounds__(TX_T, 3) k_gain_rows(GainTx a)
{
    extern __shared__ __align__(16) float2 tx_smem[];
    __shared__ TxCtx X;
    __shared__ double s_red[TX_T / 32], s_out[1];
    float2 *b0 = tx_smem, *b1 = tx_smem + TX_TILE;
    int cur = -1;
    int i0, i1;
    cta_share(a.nitems, i0, i1);
    for (int it = i0; it < i1; ++it) {
        const int2 w = a.items[a.item0 + it];
        tx_begin(X, a.txl, a.q_tx, a.off, w.x, w.y, a.obase, a.ndet, a.fsamp, a.psd, nullptr, cur, a.qsc);
        const float fscale = X.fscale, alpha = X.alpha, s2 = X.s2;
        const int n = X.L.n, m = X.L.m;
        Acc2 sa[1] = {{0.f, 0.f}};
        row_pass<float2, true>(X, b0, b1, a.Y, a.tw + X.L.twb, [](float2 *) {}, [&](int, int k, float2 S) {
            const int ka = k, kb = (k == 0) ? m : n - k;
            const float wa = ka == 0 ? 0.f : sfu_rcp(s2 * (1.0f + tx_fpow(ka, fscale, alpha)));
            const float wb = sfu_rcp(s2 * (1.0f + tx_fpow(kb, fscale, alpha)));
            const float2 Wv = make_float2(S.x * wa, S.y * wb);
            acc_add_prod(sa[0], S.x, Wv.x);
            acc_add_prod(sa[0], S.y, Wv.y);
            return Wv;
        });
        block_sums<1>(sa, s_red, s_out);
        if (threadIdx.x == 0) a.part[4 * static_cast<int64_t>(a.item0 + it)] = s_out[0];
    }
}

__global__ void __launch_bounds__(TX_T, 3) k_gain_colsinv(GainTx a)
{
    extern __shared__ __align__(16) float2 tx_smem[];
    __shared__ TxCtx X;
    __shared__ double s_red[TX_T / 32], s_out[1];
    float2 *b0 = tx_smem, *b1 = tx_smem + TX_TILE;
    int cur = -1;
    int i0, i1;
    cta_share(a.nitems, i0, i1);
    for (int it = i0; it < i1; ++it) {
        const int2 w = a.items[a.item0 + it];
        tx_begin(X, a.txl, a.q_tx, a.off, w.x, w.y, a.obase, a.ndet, a.fsamp, nullptr, nullptr, cur);
        const float *dq = a.d + X.o;
        Acc2 sb[1] = {{0.f, 0.f}};
        col_inverse(X, b0, b1, a.Y, a.tw + X.L.twb, a.flags, [&](int j, bool ctr, uint32_t) {
            return ld4(dq, 4 * static_cast<int64_t>(j), ctr);
        }, [&](const float4 &dv, int ea, int eb, int j, int jm, const float2 *U, uint32_t fb) {
            const bool ctr = j == jm;
            const float2 za = U[ea];
            if (ctr) {
                acc_add_prod(sb[0], (fb & 1) ? 0.f : dv.x, za.x);
                acc_add_prod(sb[0], (fb & 2) ? 0.f : dv.y, za.y);
                return;
            }
            const float2 zb = U[eb];
            acc_add_prod(sb[0], (fb & 1) ? 0.f : dv.x, za.x);
            acc_add_prod(sb[0], (fb & 2) ? 0.f : dv.y, zb.y);
            acc_add_prod(sb[0], (fb & 4) ? 0.f : dv.z, za.y);
            acc_add_prod(sb[0], (fb & 8) ? 0.f : dv.w, zb.x);
        });
        block_sums<1>(sb, s_red, s_out);
        if (threadIdx.x == 0) a.part[4 * static_cast<int64_t>(a.item0 + it) + 1] = s_out[0];
    }
}

// Per detscan: a and b summed over its row and column items in item order,
// then the draw g ~ N(b/a, 1/a); a <= 0 (no usable sample) or a non-finite
// sum gives g = 0 and TOD_ERR_ARG.  One thread per detscan.
__global__ void __launch_bounds__(256) k_gain_fin(const double *__restrict__ rpart, const double *__restrict__ cpart,
                                                  const int32_t *__restrict__ row_off,
                                                  const int32_t *__restrict__ col_off, int q0, int q1,
                                                  int rbase, int cbase, tod_rng rng, int mode, double *g_out,
                                                  double *mu_out, double *sig_out, int32_t *status)
{
    const int q = q0 + blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= q1) return;
    double A = 0.0, B = 0.0;
    for (int i = row_off[q]; i < row_off[q + 1]; ++i) A += rpart[4 * static_cast<int64_t>(i - rbase)];
    for (int i = col_off[q]; i < col_off[q + 1]; ++i) B += cpart[4 * static_cast<int64_t>(i - cbase) + 1];
    if (!(A > 0.0) || !isfinite(A) || !isfinite(B)) {
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

// ===========================================================================
// A8: chi^2 with n_corr marginalised and its gradients, FP32 or FP64
// transforms.  rhat = C(M(d - g s)); L = 1/2 sum_{k>=1} [rhat^2/P + ln P];
// dL/dtheta = 1/2 sum_k (1/P - rhat^2/P^2) dP/dtheta (row pass);
// v = M C^T(rhat / P), dL/dg = -<M s, v> (inverse column pass).
// ===========================================================================
// the samples of unit j of s in the pass's precision (float or double s)
template <class S>
__device__ __forceinline__ void ld4s(const void *x, int64_t t, bool centre, S (&v)[4]) {
    if constexpr (sizeof(S) == sizeof(float)) {
        const float4 a = ld4(static_cast<const float *>(x), t, centre);
        v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
    } else {
        const double *p = static_cast<const double *>(x) + t;     // t even: 16-byte aligned
        const double2 a = __ldg(reinterpret_cast<const double2 *>(p));
        v[0] = a.x; v[1] = a.y; v[2] = 0.0; v[3] = 0.0;
        if (!centre) {
            const double2 b = __ldg(reinterpret_cast<const double2 *>(p + 2));
            v[2] = b.x; v[3] = b.y;
        }
    }
}

template <class V> struct Chi2Tx {
    const float *d;
    const void *s;                // float or double [N] as V
    const double *gain;
    const uint32_t *flags;
    const double *psd;
    const int64_t *off;
    const TxLen *txl;
    const int32_t *q_tx;
    const V *tw;
    const int2 *items;
    int item0, nitems;
    int ndet;
    double fsamp;
    int64_t obase;
    V *Y;
    double *part;                 // [item][4]
    void *v_out;                  // float or double [N] (global sample index), or null
};

template <class V>
__global__ void __launch_bounds__(TX_T) k_chi2_cols(Chi2Tx<V> a)
{
    typedef typename VecT<V>::S S;
    extern __shared__ __align__(16) double2 tx_smem64[];
    __shared__ TxCtx X;
    V *b0 = reinterpret_cast<V *>(tx_smem64), *b1 = b0 + TX_TILE;
    int cur = -1;
    int i0, i1;
    cta_share(a.nitems, i0, i1);
    for (int it = i0; it < i1; ++it) {
        const int2 w = a.items[a.item0 + it];
        tx_begin(X, a.txl, a.q_tx, a.off, w.x, w.y, a.obase, a.ndet, a.fsamp, nullptr, nullptr, cur);
        const double gq = a.gain[X.q];
        const float *dq = a.d + X.o;
        const int64_t o = X.o;
        struct U4 { float4 dv; S sx[4]; };
        col_forward(X, b0, b1, a.Y, a.tw + X.L.twb, a.flags, [](V *) {},
                    [&](int j, bool ctr, uint32_t) {
                        const int64_t t = 4 * static_cast<int64_t>(j);
                        U4 D;
                        D.dv = ld4(dq, t, ctr);
                        ld4s<S>(a.s, o + t, ctr, D.sx);
                        return D;
                    },
                    [&](const U4 &D, int ea, int eb, int j, int jm, V *U, uint32_t fb) {
                        const bool ctr = j == jm;
                        const float4 dv = D.dv;
                        const struct { S x, y, z, w; } sv = {D.sx[0], D.sx[1], D.sx[2], D.sx[3]};
                        const S g = static_cast<S>(gq);
                        const S r0 = (fb & 1) ? S(0) : static_cast<S>(dv.x) - g * static_cast<S>(sv.x);
                        const S r1 = (fb & 2) ? S(0) : static_cast<S>(dv.y) - g * static_cast<S>(sv.y);
                        const S r2 = (fb & 4) ? S(0) : static_cast<S>(dv.z) - g * static_cast<S>(sv.z);
                        const S r3 = (fb & 8) ? S(0) : static_cast<S>(dv.w) - g * static_cast<S>(sv.w);
                        if (ctr) { U[ea] = vmake<V>(r0, r1); return; }
                        U[ea] = vmake<V>(r0, r2);
                        U[eb] = vmake<V>(r3, r1);
                    });
    }
}

// FP64 per-mode quantities of the chi^2 row pass: the weights and the
// gradient factors are formed in the pass's precision from the FP64 PSD.
template <class V>
__global__ void __launch_bounds__(TX_T) k_chi2_rows(Chi2Tx<V> a)
{
    typedef typename VecT<V>::S S;
    extern __shared__ __align__(16) double2 tx_smem64[];
    __shared__ TxCtx X;
    __shared__ double s_red[4 * (TX_T / 32)], s_out[4];
    __shared__ double s_par[4];       // sigma0^2, ln(fsamp/(2 n f_knee)), alpha, f_knee
    V *b0 = reinterpret_cast<V *>(tx_smem64), *b1 = b0 + TX_TILE;
    int cur = -1;
    int i0, i1;
    cta_share(a.nitems, i0, i1);
    for (int it = i0; it < i1; ++it) {
        const int2 w = a.items[a.item0 + it];
        tx_begin(X, a.txl, a.q_tx, a.off, w.x, w.y, a.obase, a.ndet, a.fsamp, a.psd, nullptr, cur);
        if (threadIdx.x == 0) {
            const double sig0 = a.psd[3 * X.det], fk = a.psd[3 * X.det + 1], al = a.psd[3 * X.det + 2];
            s_par[0] = sig0;
            s_par[1] = log(a.fsamp / (2.0 * X.L.n * fk));
            s_par[2] = al;
            s_par[3] = fk;
        }
        __syncthreads();
        const S sig0 = static_cast<S>(s_par[0]), lfs = static_cast<S>(s_par[1]), al = static_cast<S>(s_par[2]);
        const S fk = static_cast<S>(s_par[3]);
        const S s2 = sig0 * sig0;
        const int n = X.L.n, m = X.L.m;
        // sums: L, dL/dsigma0, dL/dfknee, dL/dalpha (FP64 per thread, as the
        // FP64 path needs; the FP32 path adds FP32 terms into FP64)
        double acc[4] = {0.0, 0.0, 0.0, 0.0};
        auto mode_terms = [&](int k, S r) -> S {
            // ln(f/fk) = ln k + ln(fsamp/(2 n fk)); P = s2 (1 + e^{alpha ln(f/fk)})
            const S lr = log(static_cast<S>(k)) + lfs;
            const S pw = exp(al * lr);
            const S P = s2 * (S(1) + pw);
            const S iP = S(1) / P;
            const S r2P = r * r * iP;
            acc[0] += 0.5 * (static_cast<double>(r2P) + static_cast<double>(log(P)));
            const S h = S(0.5) * (iP - r2P * iP);             // 1/2 (1/P - r^2/P^2)
            acc[1] += static_cast<double>(h * S(2) * P / sig0);
            acc[2] += static_cast<double>(h * (-s2 * al * pw / fk));
            acc[3] += static_cast<double>(h * s2 * pw * lr);
            return r * iP;
        };
        row_pass<V, true>(X, b0, b1, a.Y, a.tw + X.L.twb, [](V *) {}, [&](int, int k, V Rv) {
            const int ka = k, kb = (k == 0) ? m : n - k;
            const S wa = ka == 0 ? S(0) : mode_terms(ka, Rv.x);
            const S wb = mode_terms(kb, Rv.y);
            return vmake<V>(ka == 0 ? S(0) : wa, wb);
        });
        block_sums_d<4>(acc, s_red, s_out);
        if (threadIdx.x < 4) a.part[4 * static_cast<int64_t>(a.item0 + it) + threadIdx.x] = s_out[threadIdx.x];
    }
}

template <class V>
__global__ void __launch_bounds__(TX_T) k_chi2_colsinv(Chi2Tx<V> a)
{
    typedef typename VecT<V>::S S;
    extern __shared__ __align__(16) double2 tx_smem64[];
    __shared__ TxCtx X;
    __shared__ double s_red[TX_T / 32], s_out[1];
    V *b0 = reinterpret_cast<V *>(tx_smem64), *b1 = b0 + TX_TILE;
    int cur = -1;
    int i0, i1;
    cta_share(a.nitems, i0, i1);
    for (int it = i0; it < i1; ++it) {
        const int2 w = a.items[a.item0 + it];
        tx_begin(X, a.txl, a.q_tx, a.off, w.x, w.y, a.obase, a.ndet, a.fsamp, nullptr, nullptr, cur);
        const int64_t o = X.o;
        double acc[1] = {0.0};
        struct U4 { S sx[4]; };
        col_inverse(X, b0, b1, a.Y, a.tw + X.L.twb, a.flags, [&](int j, bool ctr, uint32_t) {
            U4 D;
            ld4s<S>(a.s, o + 4 * static_cast<int64_t>(j), ctr, D.sx);
            return D;
        }, [&](const U4 &D, int ea, int eb, int j, int jm, const V *U, uint32_t fb) {
            const bool ctr = j == jm;
            const int64_t t = 4 * static_cast<int64_t>(j);
            const S *sx = D.sx;
            const V za = U[ea];
            const V zb = ctr ? za : U[eb];
            S v[4] = {(fb & 1) ? S(0) : za.x, (fb & 2) ? S(0) : (ctr ? za.y : zb.y),
                      (fb & 4) ? S(0) : za.y, (fb & 8) ? S(0) : zb.x};
            const int cnt = ctr ? 2 : 4;
            for (int u = 0; u < cnt; ++u) acc[0] -= static_cast<double>(sx[u] * v[u]);
            if (a.v_out) {
                S *vo = static_cast<S *>(a.v_out) + o + t;
                for (int u = 0; u < cnt; ++u) vo[u] = v[u];
            }
        });
        block_sums_d<1>(acc, s_red, s_out);
        if (threadIdx.x == 0) a.part[4 * static_cast<int64_t>(a.item0 + it) + 1] = s_out[0];
    }
}

// Per detscan: chi^2 and its PSD-parameter terms from the row items, the
// gain derivative from the column items (item order).
__global__ void __launch_bounds__(256) k_chi2_fin(const double *__restrict__ rpart, const double *__restrict__ cpart,
                                                  const int32_t *__restrict__ row_off,
                                                  const int32_t *__restrict__ col_off, int q0, int q1, int rbase,
                                                  int cbase, double *chi2_q, double *dgain, double *dpsd_q)
{
    const int q = q0 + blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= q1) return;
    double s[4] = {0.0, 0.0, 0.0, 0.0};
    for (int i = row_off[q]; i < row_off[q + 1]; ++i)
        for (int k = 0; k < 4; ++k) s[k] += rpart[4 * static_cast<int64_t>(i - rbase) + k];
    double g = 0.0;
    for (int i = col_off[q]; i < col_off[q + 1]; ++i) g += cpart[4 * static_cast<int64_t>(i - cbase) + 1];
    chi2_q[q] = s[0];
    dgain[q] = g;
    for (int k = 0; k < 3; ++k) dpsd_q[3 * static_cast<int64_t>(q) + k] = s[k + 1];
}

// Band totals in detscan order (one thread): chi^2 and the PSD gradient of
// every detector.
__global__ void k_chi2_total(const double *__restrict__ chi2_q, const double *__restrict__ dpsd_q, int nq, int ndet,
                             double *total, double *dpsd_det)
{
    if (blockIdx.x != 0 || threadIdx.x != 0) return;
    double t = 0.0;
    for (int q = 0; q < nq; ++q) t += chi2_q[q];
    total[0] = t;
    for (int det = 0; det < ndet; ++det)
        for (int k = 0; k < 3; ++k) {
            double s = 0.0;
            for (int q = det; q < nq; q += ndet) s += dpsd_q[3 * static_cast<int64_t>(q) + k];
            dpsd_det[3 * det + k] = s;
        }
}

// ===========================================================================
// A5: correlated noise.  x0 = B^{-1} b with B = C^T diag(phi + 1/sigma0^2) C
// is the draw of a gap-free detscan; flagged detscans then solve the Schur
// complement S y = E^T x0, S = sigma0^2 I - E^T B^{-1} E
// = E^T C^T diag(gamma) C E (E: flagged samples), by CG preconditioned with
// the exact inverse of each gap's Toeplitz block, and x = x0 + B^{-1} E y
// (Woodbury): x = A^{-1} b, A = B - E E^T / sigma0^2.  A detscan with every
// sample flagged has A = C^T diag(phi) C: x is its exact spectral solution
// (the offset mode, unconstrained, set to zero).
//
// One cooperative launch: phases separated by grid barriers.
// ===========================================================================
struct NcorrTx {
    const float *d, *s;
    const double *gain;
    const uint32_t *flags;
    const double *psd;
    const int64_t *off;
    const TxLen *txl;
    const int32_t *q_tx;
    const float2 *tw;
    const int2 *colitems, *rowitems;
    const int32_t *col_off, *row_off;
    int q0, q1;                   // detscan range of this launch
    int ndet;
    double fsamp;
    tod_rng rng;
    int mode;
    float tol;
    int maxit;
    float *x_out;
    int32_t *iters;
    int32_t *status;
    float *spec_out;
    const float *xtab;            // Toeplitz inverses' first columns per detector (null: no preconditioner)
    const int32_t *lvalid;
    // coarse correction (null czsz: none)
    const float4 *cztab;          // [ndet][href + 1] prefix sums of the gap kernel
    int href;
    int32_t *gbpos;               // [nq][TX_GBMAX] first sample of each block
    float *czsz;                  // [czcap][TX_CZJ] S Z rows by flagged rank
    int64_t czcap;
    float *czl;                   // [nq][2 TX_CBMAX][TX_CZB + 1] factor of E
    // scratch
    float2 *Y;                    // launch-range intermediate
    int64_t *wpre;                // [range words + 1]
    int64_t *chunk;               // [gridDim + 1]
    CgState *cgs;                 // [nq]
    int2 *gblk;                   // [nq][TX_GBMAX]
    int32_t *gnb;                 // [nq]
    float *cgv;                   // [5][cgcap]
    int64_t cgcap;
    int32_t *count;               // [2]
    float4 *qsc;                  // [nq][2] per-detscan FP32 scalars, written in the index phase
    // the detscans a CG pass works on, in order, with the running counts of
    // their column and row items: list[0] = n, then q[nq], col[nq + 1], row[nq + 1]
    int32_t *list;
};
__device__ __forceinline__ int32_t *nl_q(const NcorrTx &a) { return a.list + 1; }
__device__ __forceinline__ int32_t *nl_col(const NcorrTx &a) { return a.list + 1 + (a.q1 - a.q0); }
__device__ __forceinline__ int32_t *nl_row(const NcorrTx &a) { return a.list + 2 + 2 * (a.q1 - a.q0); }

struct CgVec { float *y, *r, *p, *q, *z; };
__device__ __forceinline__ CgVec cg_vecs(const NcorrTx &a) {
    CgVec v;
    v.y = a.cgv; v.r = v.y + a.cgcap; v.p = v.r + a.cgcap; v.q = v.p + a.cgcap; v.z = v.q + a.cgcap;
    return v;
}

// flagged samples of the launch range before sample t (global index)
__device__ __forceinline__ int64_t flag_rank(const uint32_t *__restrict__ fl, const int64_t *__restrict__ wpre,
                                             int64_t w_lo, int64_t obase, int64_t t) {
    const int64_t w = t >> 5;
    uint32_t bits = __ldg(fl + w) & ((1u << (t & 31)) - 1u);
    if (w == w_lo) bits &= ~((1u << (obase & 31)) - 1u);
    return wpre[w - w_lo] + __popc(bits);
}

// Shared memory of the n_corr kernel besides the tiles.
struct NcShared {
    TxCtx X;
    double red[4 * (TX_T / 32)];
    double out[4];
    int3 scan[TX_T / 32 + 1];
    int gbeg[TX_GBMAX], gend[TX_GBMAX];
    int blen[TX_GBMAX], brank[TX_GBMAX], boff[TX_GBMAX], bq[TX_GBMAX];
    int rnd[TX_GBMAX + 1];
    int nrnd, nb;
    int64_t i64[2];
    double d64[4];
    int flag;
};

// Exclusive scan of one int3 per thread over the CTA; total gets the sum.
__device__ int3 cta_exscan3(int3 v, int3 *s_w, int3 &total)
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
        constexpr int NW = TX_T / 32;
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
    total = s_w[TX_T / 32];
    __syncthreads();
    return make_int3(b.x + inc.x - v.x, b.y + inc.y - v.y, b.z + inc.z - v.z);
}

// Flagged-sample prefix over the range's flag words, in chunks of words per
// CTA: count (chunk totals), scan (one thread), write (per-word prefix).
struct FlagChunk {
    int64_t w_lo, nw, c0, c1, t0, per, obase, oend;
};
__device__ __forceinline__ FlagChunk flag_chunk(const NcorrTx &a) {
    FlagChunk f;
    f.obase = a.off[a.q0];
    f.oend = a.off[a.q1];
    f.w_lo = f.obase >> 5;
    f.nw = ((f.oend + 31) >> 5) - f.w_lo;
    const int64_t cw = (f.nw + gridDim.x - 1) / gridDim.x;
    f.c0 = min(f.nw, static_cast<int64_t>(blockIdx.x) * cw);
    f.c1 = min(f.nw, f.c0 + cw);
    f.per = (f.c1 - f.c0 + TX_T - 1) / TX_T;
    f.t0 = f.c0 + threadIdx.x * f.per;
    return f;
}
// word w_lo + i restricted to the range
__device__ __forceinline__ uint32_t flag_word(const NcorrTx &a, const FlagChunk &f, int64_t i) {
    const int64_t w = f.w_lo + i;
    uint32_t b = __ldg(a.flags + w);
    const int64_t base = w << 5;
    if (base < f.obase) b &= ~0u << static_cast<int>(f.obase - base);
    if (base + 32 > f.oend) b &= (f.oend - base >= 32) ? ~0u : ((1u << static_cast<int>(f.oend - base)) - 1u);
    return b;
}
__device__ void nc_flag_count(const NcorrTx &a, NcShared &S)
{
    const FlagChunk f = flag_chunk(a);
    int mine = 0;
    for (int64_t i = f.t0; i < min(f.c1, f.t0 + f.per); ++i) mine += __popc(flag_word(a, f, i));
    int3 tot3;
    cta_exscan3(make_int3(mine, 0, 0), S.scan, tot3);
    if (threadIdx.x == 0) a.chunk[blockIdx.x] = tot3.x;
}
__device__ void nc_flag_write(const NcorrTx &a, NcShared &S)
{
    const FlagChunk f = flag_chunk(a);
    int mine = 0;
    for (int64_t i = f.t0; i < min(f.c1, f.t0 + f.per); ++i) mine += __popc(flag_word(a, f, i));
    int3 tot3;
    const int3 ex = cta_exscan3(make_int3(mine, 0, 0), S.scan, tot3);
    int64_t run = a.chunk[blockIdx.x] + ex.x;
    for (int64_t i = f.t0; i < min(f.c1, f.t0 + f.per); ++i) {
        a.wpre[i] = run;
        run += __popc(flag_word(a, f, i));
    }
    if (blockIdx.x == gridDim.x - 1 && threadIdx.x == 0) a.wpre[f.nw] = a.chunk[gridDim.x];
}

// Phase 2 (per detscan): flagged count and rank offset, CG mode, and the
// gap blocks of the preconditioner (gaps split into blocks of at most lmax).
__device__ void nc_detscan_index(const NcorrTx &a, NcShared &S, int q)
{
    const int64_t obase = a.off[a.q0];
    const int64_t w_lo = obase >> 5;
    const int64_t o = a.off[q], n = a.off[q + 1] - o;
    const int det = q % a.ndet;
    if (threadIdx.x == 0) {
        const int64_t k0 = flag_rank(a.flags, a.wpre, w_lo, obase, o);
        const int64_t k1 = (a.off[q + 1] == a.off[a.q1] && ((a.off[q + 1] & 31) == 0))
                               ? a.wpre[((a.off[q + 1]) >> 5) - w_lo]
                               : flag_rank(a.flags, a.wpre, w_lo, obase, a.off[q + 1]);
        S.i64[0] = k0;
        S.i64[1] = k1 - k0;
    }
    __syncthreads();
    const int64_t koff = S.i64[0];
    const int K = static_cast<int>(S.i64[1]);
    // gaps: runs of flagged samples
    const int64_t wb0 = o >> 5, wb1 = (o + n - 1) >> 5;
    const int nw = static_cast<int>(wb1 - wb0 + 1);
    const int per = (nw + TX_T - 1) / TX_T;
    auto wbits = [&](int wi) -> uint32_t {
        if (wi < 0 || wi >= nw) return 0u;
        uint32_t bits = __ldg(a.flags + wb0 + wi);
        const int64_t base = ((wb0 + wi) << 5) - o;
        if (base < 0) bits &= ~0u << static_cast<int>(-base);
        if (base + 32 > n) bits &= (n - base >= 32) ? ~0u : ((1u << static_cast<int>(n - base)) - 1u);
        return bits;
    };
    int3 mine = make_int3(0, 0, 0);
    for (int i = 0; i < per; ++i) {
        const int wi = threadIdx.x * per + i;
        if (wi >= nw) break;
        const uint32_t bits = wbits(wi), prev = wbits(wi - 1) >> 31, next = wbits(wi + 1) & 1u;
        mine.y += __popc(bits & ~((bits << 1) | prev));
        mine.z += __popc(bits & ~((bits >> 1) | (next << 31)));
    }
    int3 tot3;
    const int3 ex = cta_exscan3(mine, S.scan, tot3);
    const int ngap = tot3.y;
    if (ngap <= TX_GBMAX) {
        int gpos = ex.y, epos = ex.z;
        for (int i = 0; i < per; ++i) {
            const int wi = threadIdx.x * per + i;
            if (wi >= nw) break;
            const uint32_t bits = wbits(wi), prev = wbits(wi - 1) >> 31, next = wbits(wi + 1) & 1u;
            uint32_t st = bits & ~((bits << 1) | prev), en = bits & ~((bits >> 1) | (next << 31));
            const int base = static_cast<int>(((wb0 + wi) << 5) - o);
            while (st) { S.gbeg[gpos++] = base + __ffs(st) - 1; st &= st - 1; }
            while (en) { S.gend[epos++] = base + __ffs(en); en &= en - 1; }
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        det_scalars_q(a.psd, a.gain, a.off, a.ndet, a.fsamp, q, a.qsc);
        CgState cs;
        cs.rz = 0.0; cs.stop = 0.0; cs.koff = koff; cs.K = K; cs.it = 0; cs.ncz = 0;
        if (K == 0) cs.mode = CG_NONE;
        else if (K == n) cs.mode = CG_ALLFLAG;
        else if (koff + K > a.cgcap) cs.mode = CG_OVER;
        else cs.mode = CG_ACTIVE;
        a.cgs[q] = cs;
        // preconditioner blocks (rank within the detscan, length)
        int nb = 0;
        const int lmax = (a.xtab && a.lvalid) ? min(TOEP_LMAX, a.lvalid[det]) : 0;
        if (cs.mode == CG_ACTIVE && ngap <= TX_GBMAX && lmax >= 1) {
            int rank = 0;
            for (int g = 0; g < ngap && nb >= 0; ++g)
                for (int b0 = S.gbeg[g]; b0 < S.gend[g]; b0 += lmax) {
                    const int len = min(lmax, S.gend[g] - b0);
                    if (nb >= TX_GBMAX) { nb = -1; break; }
                    a.gblk[static_cast<int64_t>(q) * TX_GBMAX + nb] = make_int2(rank, len);
                    if (a.gbpos) a.gbpos[static_cast<int64_t>(q) * TX_GBMAX + nb] = b0;
                    ++nb;
                    rank += len;
                }
        } else {
            nb = -1;
        }
        a.gnb[q] = nb;
    }
}

// Phase 3, column pass of the right-hand side: M (r/sigma0^2 + w1/sigma0),
// r = d - g s; w1 of z_j is normal pair j of the NC_W1 stream (pair j mod 4
// of Philox block j/4).
__device__ void nc_rhs_cols(const NcorrTx &a, const TxCtx &X, float2 *b0, float2 *b1, uint64_t gi)
{
    const bool draw = a.mode == TOD_MODE_DRAW;
    const float *dq = a.d + X.o, *sq = a.s + X.o;
    const float g = X.g, inv_s2 = X.inv_s2, inv_s = X.inv_s;
    const uint64_t q = static_cast<uint64_t>(X.q);
    const ColGeo G(X.L, X.blk);
    struct U8 { float4 dv, sv; };
    col_forward(X, b0, b1, a.Y, a.tw + X.L.twb, a.flags,
                [&](float2 *U) {
                    // the tile's normals: one Philox block per thread, its four
                    // pairs to the tile elements whose index j falls in it
                    const ColGeo G(X.L, X.blk);
                    if (!draw) {
                        for (int e = threadIdx.x; e < G.m1 * G.W; e += TX_T) U[e] = make_float2(0.f, 0.f);
                        return;
                    }
                    const int nbk = (G.np + 3) / 4 + 1;          // blocks touching a side's j range of a row
                    const int total = G.m1 * 2 * nbk;
                    for (int w = threadIdx.x; w < total; w += TX_T) {
                        const int j1 = w / (2 * nbk), rest = w - j1 * 2 * nbk;
                        const int side = rest / nbk, bi = rest - side * nbk;
                        // j range of this row and side: [ja, jb)
                        int ja, jb;
                        if (side == 0) { ja = j1 * G.m2 + G.p0; jb = ja + G.np; }
                        else { jb = j1 * G.m2 + G.m2 - G.p0; ja = jb - G.np; }
                        const int bk = (ja >> 2) + bi;
                        if (4 * bk >= jb) continue;
                        const u64x4 rw = philox4x64(static_cast<uint64_t>(bk), q, 1, gi, a.rng.seed, a.rng.band);
#pragma unroll
                        for (int u = 0; u < 4; ++u) {
                            const int j = 4 * bk + u;
                            if (j < ja || j >= jb) continue;
                            const int c = j - j1 * G.m2;
                            const int lc = side == 0 ? c - G.p0 : G.TP + (G.m2 - 1 - c - G.p0);
                            if (G.col(lc) < 0) continue;      // the middle column's duplicate
                            U[j1 * G.W + lc] = philox_normal_pair(rw, u);
                        }
                    }
                },
                [&](int j, bool ctr, uint32_t) {
                    const int64_t t = 4 * static_cast<int64_t>(j);
                    return U8{ld4(dq, t, ctr), ld4(sq, t, ctr)};
                },
                [&](const U8 &D, int ea, int eb, int j, int jm, float2 *U, uint32_t fb) {
                    const bool ctr = j == jm;
                    const float4 dv = D.dv, sv = D.sv;
                    const float2 wa = U[ea];
                    if (ctr) {
                        U[ea] = make_float2((fb & 1) ? 0.f : fmaf(dv.x - g * sv.x, inv_s2, wa.x * inv_s),
                                            (fb & 2) ? 0.f : fmaf(dv.y - g * sv.y, inv_s2, wa.y * inv_s));
                        return;
                    }
                    const float2 wb = U[eb];
                    // samples 4j, 4j+2 -> z_j = (v_{2j}, v_{2j+1}); 4j+3, 4j+1 -> z_{m-1-j}
                    U[ea] = make_float2((fb & 1) ? 0.f : fmaf(dv.x - g * sv.x, inv_s2, wa.x * inv_s),
                                        (fb & 4) ? 0.f : fmaf(dv.z - g * sv.z, inv_s2, wa.y * inv_s));
                    U[eb] = make_float2((fb & 8) ? 0.f : fmaf(dv.w - g * sv.w, inv_s2, wb.x * inv_s),
                                        (fb & 2) ? 0.f : fmaf(dv.y - g * sv.y, inv_s2, wb.y * inv_s));
                });
}

// Filter weights of the packed slot pair: beta = 1/(phi + 1/sigma0^2) =
// sigma0^2/(1 + r), gamma = sigma0^2 r/(1 + r) with r = sigma0^2 phi =
// (f/f_knee)^-alpha (r = 0 at mode 0).  With every sample flagged beta is
// 1/phi = sigma0^2 / r (0 at mode 0).
__device__ __forceinline__ float nc_r(int k, const TxCtx &X) {
    return k == 0 ? 0.f : tx_fpow(k, X.fscale, -X.alpha);
}

// Phase 3, row pass of the right-hand side: + sqrt(phi) w2 (mode pair k of
// the NC_W2 stream), times beta; the spectrum beta (C b + prior term) is
// written when asked for.
__device__ void nc_rhs_rows(const NcorrTx &a, const TxCtx &X, float2 *b0, float2 *b1, uint64_t gi)
{
    const bool draw = a.mode == TOD_MODE_DRAW;
    const bool allf = X.mode == CG_ALLFLAG;
    const uint64_t q = static_cast<uint64_t>(X.q);
    const float s2 = X.s2, inv_s2 = X.inv_s2;
    const int n = X.L.n, m = X.L.m;
    float *spec = a.spec_out ? a.spec_out + X.o : nullptr;
    float2 *nu = nullptr;
    row_pass<float2, true>(X, b0, b1, a.Y, a.tw + X.L.twb,
        [&](float2 *Fr) {
            nu = Fr;
            const RowGeo G(X.L, X.blk);
            const int npl = G.nr, m1 = G.m1, m2 = G.m2, p0 = G.r0;
            if (!draw) {
                for (int e = threadIdx.x; e < 2 * G.TR * G.m2p; e += TX_T) Fr[e] = make_float2(0.f, 0.f);
                return;
            }
            // for a fixed k2 the even slots hold k = p0 + pl + m1 k2 and the
            // odd ones k = m1 - p0 - pl + m1 k2: one Philox block per thread
            // for up to four consecutive modes of a parity
            const int nbk = (npl + 3) / 4 + 1;
            const int items = 2 * nbk * m2;
            for (int w = threadIdx.x; w < items; w += TX_T) {
                const int rest = fdiv(w, X.L.f_m2), k2 = w - rest * m2;
                const int par = rest / nbk, bi = rest - par * nbk;
                const int kbase = (par == 0 ? p0 : m1 - p0 - (npl - 1)) + m1 * k2;
                const int bk = (kbase >> 2) + bi;
                if (npl <= 0 || 4 * bk >= kbase + npl) continue;
                const u64x4 rw = philox4x64(static_cast<uint64_t>(bk), q, 2, gi, a.rng.seed, a.rng.band);
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int k = 4 * bk + u;
                    if (k < kbase || k >= kbase + npl) continue;
                    const int pl = par == 0 ? k - kbase : (npl - 1) - (k - kbase);
                    const int p = p0 + pl;
                    const int e = (2 * pl + par) * G.m2p + k2;
                    if (par == 1 && (p == 0 || m1 - p == p)) { Fr[e] = make_float2(0.f, 0.f); continue; }
                    const int ka = k, kb = (k == 0) ? m : n - k;
                    const float ra = nc_r(ka, X), rb = nc_r(kb, X);
                    const float2 w2 = philox_normal_pair(rw, u);
                    Fr[e] = make_float2(sqrtf(ra * inv_s2) * w2.x, sqrtf(rb * inv_s2) * w2.y);
                }
            }
        },
        [&](int e, int k, float2 Yv) {
            const int ka = k, kb = (k == 0) ? m : n - k;
            const float ra = nc_r(ka, X), rb = nc_r(kb, X);
            float ba, bb;
            if (allf) { ba = ka == 0 ? 0.f : s2 * sfu_rcp(ra); bb = s2 * sfu_rcp(rb); }
            else { ba = s2 * sfu_rcp(1.0f + ra); bb = s2 * sfu_rcp(1.0f + rb); }
            const float2 cb = make_float2(Yv.x + nu[e].x, Yv.y + nu[e].y);
            const float2 xs = make_float2(cb.x * ba, cb.y * bb);
            if (spec) { spec[ka] = xs.x; spec[kb] = xs.y; }
            return xs;
        });
}

// Phase 3, inverse column pass: x0 out; its flagged samples are the CG
// right-hand side E^T x0.
__device__ void nc_x0_cols(const NcorrTx &a, const TxCtx &X, float2 *b0, float2 *b1)
{
    const bool cg = X.mode == CG_ACTIVE;
    float *xq = a.x_out + X.o;
    const int64_t o = X.o, obase = a.off[a.q0], w_lo = obase >> 5;
    float *r = a.cgv + a.cgcap;
    const ColGeo G(X.L, X.blk);
    col_inverse(X, b0, b1, a.Y, a.tw + X.L.twb, cg ? a.flags : nullptr, [&](int, bool, uint32_t) { return 0; },
                [&](int, int ea, int eb, int j, int jm, const float2 *U, uint32_t fbits) {
        const bool ctr = j == jm;
        const int64_t t = 4 * static_cast<int64_t>(j);
        const float2 za = U[ea];
        float v[4];
        if (ctr) { v[0] = za.x; v[1] = za.y; }
        else {
            const float2 zb = U[eb];
            v[0] = za.x; v[1] = zb.y; v[2] = za.y; v[3] = zb.x;
        }
        reinterpret_cast<float2 *>(xq + t)[0] = make_float2(v[0], v[1]);
        if (!ctr) reinterpret_cast<float2 *>(xq + t + 2)[0] = make_float2(v[2], v[3]);
        if (cg) {
            uint32_t fb = fbits;
            while (fb) {
                const int u = __ffs(fb) - 1;
                fb &= fb - 1;
                r[flag_rank(a.flags, a.wpre, w_lo, obase, o + t + u)] = v[u];
            }
        }
    });
}

// CG column pass: z = E vec (the flagged samples' entries of vec, zero
// elsewhere), forward columns.
__device__ void nc_scatter_cols(const NcorrTx &a, const TxCtx &X, float2 *b0, float2 *b1, const float *vec)
{
    const int64_t o = X.o, obase = a.off[a.q0], w_lo = obase >> 5;
    const ColGeo G(X.L, X.blk);
    col_forward(X, b0, b1, a.Y, a.tw + X.L.twb, a.flags, [](float2 *) {},
                [&](int j, bool, uint32_t fb) {
                    // the unit's flagged entries of vec (a rank lookup only where flagged)
                    const int64_t t = 4 * static_cast<int64_t>(j);
                    float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
                    while (fb) {
                        const int u = __ffs(fb) - 1;
                        fb &= fb - 1;
                        const float val = vec[flag_rank(a.flags, a.wpre, w_lo, obase, o + t + u)];
                        if (u == 0) v.x = val; else if (u == 1) v.y = val; else if (u == 2) v.z = val; else v.w = val;
                    }
                    return v;
                },
                [&](const float4 &D, int ea, int eb, int j, int jm, float2 *U, uint32_t) {
                    const float v[4] = {D.x, D.y, D.z, D.w};
                    if (j == jm) { U[ea] = make_float2(v[0], v[1]); return; }
                    U[ea] = make_float2(v[0], v[2]);
                    U[eb] = make_float2(v[3], v[1]);
                });
}

// CG row pass: times gamma (apply S), or times beta (the final B^{-1} E y,
// whose spectrum is added to the one written at the right-hand side).
template <bool BETA>
__device__ void nc_filter_rows(const NcorrTx &a, const TxCtx &X, float2 *b0, float2 *b1)
{
    const float s2 = X.s2;
    const int n = X.L.n, m = X.L.m;
    float *spec = (BETA && a.spec_out) ? a.spec_out + X.o : nullptr;
    row_pass<float2, true>(X, b0, b1, a.Y, a.tw + X.L.twb, [](float2 *) {}, [&](int, int k, float2 Yv) {
        const int ka = k, kb = (k == 0) ? m : n - k;
        const float ra = nc_r(ka, X), rb = nc_r(kb, X);
        float2 r;
        const float ia = sfu_rcp(1.0f + ra), ib = sfu_rcp(1.0f + rb);
        if (BETA) {
            r = make_float2(Yv.x * (s2 * ia), Yv.y * (s2 * ib));
            if (spec) { spec[ka] += r.x; spec[kb] += r.y; }
        } else {
            r = make_float2(Yv.x * (s2 * ra * ia), Yv.y * (s2 * rb * ib));
        }
        return r;
    });
}

// CG inverse column pass: q = E^T (...) (gather), or x += (...) (final).
template <bool ADD>
__device__ void nc_gather_cols(const NcorrTx &a, const TxCtx &X, float2 *b0, float2 *b1, float *qv)
{
    const int64_t o = X.o, obase = a.off[a.q0], w_lo = obase >> 5;
    float *xq = a.x_out + X.o;
    col_inverse(X, b0, b1, a.Y, a.tw + X.L.twb, ADD ? nullptr : a.flags, [&](int j, bool ctr, uint32_t) {
        // ADD: the unit's x0 (written earlier in this launch: coherent loads,
        // not the read-only path); the gather needs only the flag bits
        float4 x = make_float4(0.f, 0.f, 0.f, 0.f);
        if (ADD) {
            const int64_t t = 4 * static_cast<int64_t>(j);
            const float2 a01 = reinterpret_cast<const float2 *>(xq + t)[0];
            const float2 a23 = ctr ? make_float2(0.f, 0.f) : reinterpret_cast<const float2 *>(xq + t + 2)[0];
            x = make_float4(a01.x, a01.y, a23.x, a23.y);
        }
        return x;
    }, [&](const float4 &x0, int ea, int eb, int j, int jm, const float2 *U, uint32_t fbits) {
        if (!ADD && fbits == 0) return;          // no flagged sample in the unit
        const bool ctr = j == jm;
        const int64_t t = 4 * static_cast<int64_t>(j);
        const float2 za = U[ea];
        float v[4];
        if (ctr) { v[0] = za.x; v[1] = za.y; }
        else {
            const float2 zb = U[eb];
            v[0] = za.x; v[1] = zb.y; v[2] = za.y; v[3] = zb.x;
        }
        if (ADD) {
            float2 *p = reinterpret_cast<float2 *>(xq + t);
            p[0] = make_float2(x0.x + v[0], x0.y + v[1]);
            if (!ctr) p[1] = make_float2(x0.z + v[2], x0.w + v[3]);
        } else {
            uint32_t fb = fbits;
            while (fb) {
                const int u = __ffs(fb) - 1;
                fb &= fb - 1;
                qv[flag_rank(a.flags, a.wpre, w_lo, obase, o + t + u)] = v[u];
            }
        }
    });
}

// z = M^{-1} r over the detscan's gap blocks: T_L^{-1} = (L(x) L(x)^T -
// L(w) L(w)^T) / x_0 (Gohberg-Semencul; x = T_L^{-1} e_1 from the Durbin
// tables, w = (0, x_{L-1}, .., x_1)), blocks staged in rounds of at most
// TX_GBCAP padded floats.  Returns r.z (CTA total, every thread).  gb: five
// TX_GBCAP float arrays.
__device__ double nc_precond_m1(const NcorrTx &a, NcShared &S, int q, const float *r, float *z, float *gb)
{
    const int nb = a.gnb[q];
    const CgState &cs = a.cgs[q];
    const int K = cs.K;
    Acc2 rz[1] = {{0.f, 0.f}};
    if (nb < 0) {             // no preconditioner: z = r
        for (int i = threadIdx.x; i < K; i += TX_T) {
            const float v = r[i];
            z[i] = v;
            acc_add_prod(rz[0], v, v);
        }
        block_sums<1>(rz, S.red, S.out);
        return S.out[0];
    }
    const int det = q % a.ndet;
    const float *xt_det = a.xtab + static_cast<int64_t>(det) * (TOEP_LMAX * (TOEP_LMAX + 1) / 2);
    if (threadIdx.x == 0) {
        int nrnd = 0, len = 0, rq = 0;
        for (int b = 0; b < nb; ++b) {
            const int2 bl = a.gblk[static_cast<int64_t>(q) * TX_GBMAX + b];
            const int reg = ((bl.y + 3) & ~3) + 16;
            if (b == 0 || len + reg > TX_GBCAP) { S.rnd[nrnd++] = b; len = 0; rq = 0; }
            S.brank[b] = bl.x; S.blen[b] = bl.y; S.boff[b] = len; S.bq[b] = rq;
            len += reg;
            rq += (bl.y + 3) >> 2;
        }
        S.rnd[nrnd] = nb;
        S.nrnd = nrnd;
    }
    __syncthreads();
    float *gb_r = gb, *gb_x = gb + TX_GBCAP, *gb_w = gb + 2 * TX_GBCAP;
    float *gb_u1 = gb + 3 * TX_GBCAP, *gb_u2 = gb + 4 * TX_GBCAP;
    for (int rd = 0; rd < S.nrnd; ++rd) {
        const int b0 = S.rnd[rd], b1 = S.rnd[rd + 1];
        const int Ll = S.blen[b1 - 1];
        const int tot = S.boff[b1 - 1] + ((Ll + 3) & ~3) + 16;
        const int totq = S.bq[b1 - 1] + ((Ll + 3) >> 2);
        for (int f = threadIdx.x; f < tot; f += TX_T) {
            int b = b0;
            while (b + 1 < b1 && S.boff[b + 1] <= f) ++b;
            const int L = S.blen[b], li = f - S.boff[b] - 8;
            float rv = 0.f, xv = 0.f, wv = 0.f;
            if (li >= 0 && li < L) {
                const float *xt = xt_det + static_cast<int64_t>(L) * (L - 1) / 2;
                rv = r[S.brank[b] + li];
                xv = xt[li];
                wv = li == 0 ? 0.f : xt[L - li];
            }
            gb_r[f] = rv; gb_x[f] = xv; gb_w[f] = wv; gb_u1[f] = 0.f; gb_u2[f] = 0.f;
        }
        __syncthreads();
        // u1 = L(x)^T r, u2 = L(w)^T r: four outputs per group of QT threads
        const int QT = (totq * 4 <= TX_T) ? 4 : (totq * 2 <= TX_T) ? 2 : 1;
        const int qsh = QT == 4 ? 2 : QT == 2 ? 1 : 0;
        const int totw = totq << qsh;
        for (int t0 = 0; t0 < totw; t0 += TX_T) {
            const int t = t0 + threadIdx.x;
            const bool act = t < totw;
            const int qi = t >> qsh, part = t & (QT - 1);
            float4 a1 = make_float4(0.f, 0.f, 0.f, 0.f), a2 = a1;
            int base = 0, i0 = 0;
            if (act) {
                int b = b0;
                while (b + 1 < b1 && S.bq[b + 1] <= qi) ++b;
                const int L = S.blen[b];
                i0 = 4 * (qi - S.bq[b]);
                base = S.boff[b] + 8;
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
            for (int ofs = 1; ofs < QT; ofs <<= 1) {
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
        // z = (L(x) u1 - L(w) u2) / x_0
        for (int t0 = 0; t0 < totw; t0 += TX_T) {
            const int t = t0 + threadIdx.x;
            const bool act = t < totw;
            const int qi = t >> qsh, part = t & (QT - 1);
            float4 z1 = make_float4(0.f, 0.f, 0.f, 0.f), z2 = z1;
            int b = b0, i0 = 0, L = 0, base = 0;
            if (act) {
                while (b + 1 < b1 && S.bq[b + 1] <= qi) ++b;
                L = S.blen[b];
                i0 = 4 * (qi - S.bq[b]);
                base = S.boff[b] + 8;
                const float *xb = gb_x + base, *wb = gb_w + base;
                const float *u1b = gb_u1 + base + i0, *u2b = gb_u2 + base + i0;
                for (int s0 = 4 * part; s0 <= i0; s0 += 4 * QT) {
                    const float4 xs = *reinterpret_cast<const float4 *>(xb + s0);
                    const float4 ws = *reinterpret_cast<const float4 *>(wb + s0);
                    const float4 ua = *reinterpret_cast<const float4 *>(u1b - s0);
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
                for (int jj = 0; jj < 4; ++jj)
                    if (i0 + jj < L) {
                        const float zj = zz[jj] * inv;
                        z[S.brank[b] + i0 + jj] = zj;
                        acc_add_prod(rz[0], gb_r[base + i0 + jj], zj);
                    }
            }
        }
        __syncthreads();
    }
    block_sums<1>(rz, S.red, S.out);
    return S.out[0];
}

// ---------------------------------------------------------------------------
// Coarse correction (two-level preconditioner, balancing form):
//   M r = P^T M1 P r + Z E^{-1} Z^T r,  P = I - S Z E^{-1} Z^T,  E = Z^T S Z,
// with M1 the gap-block inverses above and Z two vectors per gap block: its
// indicator and its centred ramp (z(l) = (l - c) / c, c = (L - 1) / 2, over
// the block's L samples; zero for L = 1).  M is symmetric positive definite
// for any S Z and E^{-1} used consistently, so the CG converges to the same
// solution; the correction takes out the smooth modes spread over several
// gaps, which the block inverses leave to the iterations.  S Z is taken from
// the Toeplitz kernel alone, (S Z)_{i,(b,s)} = sum_{j in b} h(|p_i - p_j|)
// z_{b,s}(j), and only for the TX_CZW blocks either side of the row's own
// block (farther terms dropped), so E is banded (half-bandwidth TX_CZB in
// scalar rows) and one banded Cholesky factor per detscan applies E^{-1}.
// The sums over a block come from prefix sums of h:
//   sum_{delta=lo..hi} h(|delta|)       from H(x) = sum_{d<x} h(d),
//   sum_{delta=lo..hi} delta h(|delta|) from G(x) = sum_{d<x} d h(d),
// held as FP32 pairs and differenced in pair arithmetic (the differences of
// far blocks cancel most of the prefix values).
// ---------------------------------------------------------------------------
constexpr int CZ_LROW = TX_CZB + 1;                   // factor row: 1 / L_ii, then L_{i,i-k}, k = 1..TX_CZB
constexpr int CZ_FLOATS = 2 * TX_CBMAX * CZ_LROW + 3 * 2 * TX_CBMAX + TX_CBMAX * TX_CZJ + CZ_LROW * TX_CZB;

__device__ __forceinline__ float cz_ramp(int l, int L) {
    if (L < 2) return 0.f;
    const float c = 0.5f * static_cast<float>(L - 1);
    return (static_cast<float>(l) - c) * (1.0f / c);
}

// FP32 pair (hi + lo) arithmetic: Knuth's two-sum and an FMA two-product.
struct F2 { float h, l; };
__device__ __forceinline__ F2 f2_add(F2 x, F2 y) {
    const float s = x.h + y.h;
    const float bp = s - x.h;
    float e = (x.h - (s - bp)) + (y.h - bp);
    e += x.l + y.l;
    const float h = s + e;
    return {h, e - (h - s)};
}
__device__ __forceinline__ F2 f2_mulf(F2 x, float f) {
    const float p = __fmul_rn(x.h, f);        // not contracted into the sum below
    float e = fmaf(x.h, f, -p);
    e = fmaf(x.l, f, e);
    const float h = p + e;
    return {h, e - (h - p)};
}

// (S Z) entries of the row at sample p for a block of L samples from s:
// the indicator's sum over delta = p - j, and the ramp's.  Each table
// entry holds (H, G) at one x, loaded once.
__device__ __forceinline__ float2 cz_entry(const float4 *__restrict__ t, int p, int s, int L) {
    const int lo = p - (s + L - 1), hi = p - s;
    F2 I, Mo;
    if (lo >= 0) {
        const float4 A = __ldg(t + hi + 1), B = __ldg(t + lo);
        I = f2_add(F2{A.x, A.y}, F2{-B.x, -B.y});
        Mo = f2_add(F2{A.z, A.w}, F2{-B.z, -B.w});
    } else if (hi < 0) {
        const float4 A = __ldg(t + 1 - lo), B = __ldg(t - hi);
        I = f2_add(F2{A.x, A.y}, F2{-B.x, -B.y});
        Mo = f2_add(F2{B.z, B.w}, F2{-A.z, -A.w});
    } else {
        const float4 A = __ldg(t + hi + 1), B = __ldg(t + 1 - lo), C = __ldg(t + 1);
        I = f2_add(f2_add(F2{A.x, A.y}, F2{B.x, B.y}), F2{-C.x, -C.y});
        Mo = f2_add(F2{A.z, A.w}, F2{-B.z, -B.w});
    }
    float ramp = 0.f;
    if (L > 1) {
        // sum_j (j - c_b) h = (p - c_b) I - Mo, c_b = s + (L - 1)/2
        const float pc = 0.5f * static_cast<float>(2 * (p - s) - (L - 1));
        const F2 v = f2_add(f2_mulf(I, pc), F2{-Mo.h, -Mo.l});
        ramp = (v.h + v.l) * (1.0f / (0.5f * static_cast<float>(L - 1)));
    }
    return make_float2(I.h + I.l, ramp);
}

// Builds the coarse correction of detscan q (after the index phase): S Z
// rows, E, its banded Cholesky factor.  On success cgs[q].ncz = blocks.
__device__ void nc_coarse_setup(const NcorrTx &a, int q)
{
    __shared__ int s_rank[TX_CBMAX], s_len[TX_CBMAX], s_pos[TX_CBMAX];
    __shared__ float s_E[TX_CBMAX][4 * (2 * TX_CZW + 1)];
    __shared__ float s_L[2 * TX_CBMAX][CZ_LROW];
    __shared__ int s_ok;
    const CgState cs = a.cgs[q];
    const int nb = a.gnb[q];
    if (cs.mode != CG_ACTIVE || nb < 1 || nb > TX_CBMAX || !a.czsz || cs.koff + cs.K > a.czcap) return;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int det = q % a.ndet;
    const float4 *tab = a.cztab + static_cast<int64_t>(det) * (a.href + 1);
    for (int b = threadIdx.x; b < nb; b += TX_T) {
        const int2 bl = a.gblk[static_cast<int64_t>(q) * TX_GBMAX + b];
        s_rank[b] = bl.x;
        s_len[b] = bl.y;
        s_pos[b] = a.gbpos[static_cast<int64_t>(q) * TX_GBMAX + b];
    }
    __syncthreads();
    float *sz = a.czsz + cs.koff * TX_CZJ;
    // S Z rows, one warp per block, with the block's rows of E: for the
    // neighbour j and the row/column vector kinds (s', s), sum over the
    // block's samples of z_{s'} (S Z)_s
    for (int b = warp; b < nb; b += TX_T / 32) {
        const int L = s_len[b];
        float e[4 * (2 * TX_CZW + 1)];
#pragma unroll
        for (int k = 0; k < 4 * (2 * TX_CZW + 1); ++k) e[k] = 0.f;
        for (int l = lane; l < L; l += 32) {
            const int i = s_rank[b] + l, p = s_pos[b] + l;
            const float zr = cz_ramp(l, L);
            float2 *row = reinterpret_cast<float2 *>(sz + static_cast<int64_t>(i) * TX_CZJ);
#pragma unroll
            for (int j = 0; j < 2 * TX_CZW + 1; ++j) {
                const int c = b - TX_CZW + j;
                float2 v = make_float2(0.f, 0.f);
                if (c >= 0 && c < nb) v = cz_entry(tab, p, s_pos[c], s_len[c]);
                row[j] = v;
                e[4 * j + 0] += v.x;
                e[4 * j + 1] += v.y;
                e[4 * j + 2] = fmaf(zr, v.x, e[4 * j + 2]);
                e[4 * j + 3] = fmaf(zr, v.y, e[4 * j + 3]);
            }
        }
#pragma unroll
        for (int k = 0; k < 4 * (2 * TX_CZW + 1); ++k) {
            float v = e[k];
            for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
            if (lane == 0) s_E[b][k] = v;
        }
    }
    __syncthreads();
    // E's lower band, s_L[x][k] = E(x, x - k), x = 2b + s', y = 2c + s: from
    // block b's rows s_E[b][4 (c - b + W) + 2 s' + s], averaged with block
    // c's; a ramp of a one-sample block is zero (its row of E set to the
    // identity's)
    const int nc = 2 * nb;
    for (int i = threadIdx.x; i < nc * CZ_LROW; i += TX_T) {
        const int x = i / CZ_LROW, k = i % CZ_LROW, y = x - k;
        float v = 0.f;
        if (y >= 0) {
            const int b = x >> 1, sp = x & 1, c = y >> 1, sc = y & 1;
            if ((sp && s_len[b] < 2) || (sc && s_len[c] < 2)) v = x == y ? 1.f : 0.f;
            else if (b - c <= TX_CZW)
                v = 0.5f * (s_E[b][4 * (c - b + TX_CZW) + 2 * sp + sc] + s_E[c][4 * (b - c + TX_CZW) + 2 * sc + sp]);
        }
        s_L[x][k] = v;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        // banded Cholesky in place (FP32: E is a small, well-conditioned
        // Gram matrix of smooth vectors); s_L[x][0] becomes 1 / L_xx
        int ok = 1;
        for (int x = 0; x < nc && ok; ++x) {
            const float exx = s_L[x][0];
            float dsum = exx;
            for (int k = TX_CZB; k >= 1; --k) {
                const int y = x - k;
                float v = 0.f;
                if (y >= 0) {
                    v = s_L[x][k];
                    // sum over m < y of L(x, m) L(y, m), both within the band
                    for (int m = max(0, x - TX_CZB); m < y; ++m) v = fmaf(-s_L[x][x - m], s_L[y][y - m], v);
                    v *= s_L[y][0];
                }
                s_L[x][k] = v;
                dsum = fmaf(-v, v, dsum);
            }
            if (!(dsum > 1e-5f * fabsf(exx))) ok = 0;
            else s_L[x][0] = rsqrtf(dsum);
        }
        s_ok = ok;
        if (ok) a.cgs[q].ncz = nb;
    }
    __syncthreads();
    if (s_ok) {
        float *Lq = a.czl + static_cast<int64_t>(q) * (2 * TX_CBMAX * CZ_LROW);
        for (int i = threadIdx.x; i < nc * CZ_LROW; i += TX_T) Lq[i] = s_L[i / CZ_LROW][i % CZ_LROW];
    }
    __syncthreads();
}

// t = E^{-1} u with the banded factor staged in shared memory (rows of
// CZ_LROW; rows nc .. nc + TX_CZB - 1 zero).  One thread.
__device__ __forceinline__ void cz_solve(const float *L, int nc, const float *u, float *t)
{
    float w[TX_CZB];
#pragma unroll
    for (int k = 0; k < TX_CZB; ++k) w[k] = 0.f;
    for (int x = 0; x < nc; ++x) {
        const float *l = L + x * CZ_LROW;
        float v = u[x];
#pragma unroll
        for (int k = 1; k <= TX_CZB; ++k) v = fmaf(-l[k], w[k - 1], v);
        v *= l[0];
#pragma unroll
        for (int k = TX_CZB - 1; k > 0; --k) w[k] = w[k - 1];
        w[0] = v;
        t[x] = v;
    }
#pragma unroll
    for (int k = 0; k < TX_CZB; ++k) w[k] = 0.f;
    for (int x = nc - 1; x >= 0; --x) {
        float v = t[x];
#pragma unroll
        for (int k = 1; k <= TX_CZB; ++k) v = fmaf(-L[(x + k) * CZ_LROW + k], w[k - 1], v);
        v *= L[x * CZ_LROW];
#pragma unroll
        for (int k = TX_CZB - 1; k > 0; --k) w[k] = w[k - 1];
        w[0] = v;
        t[x] = v;
    }
}

// z = M r (two-level when the detscan has a coarse correction, else the
// block inverses alone).  Returns r.z (CTA total, every thread).  gb: the
// five TX_GBCAP arrays of the block inverses, then CZ_FLOATS for the
// coarse vectors.
__device__ double nc_precond(const NcorrTx &a, NcShared &S, int q, const float *r, float *z, float *gb)
{
    const CgState cs = a.cgs[q];
    const int nb = cs.ncz;
    if (nb <= 0) return nc_precond_m1(a, S, q, r, z, gb);
    const int nc = 2 * nb;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    float *cL = gb + 5 * TX_GBCAP;                      // [(nc + TX_CZB) rows][CZ_LROW]
    float *ct = cL + (2 * TX_CBMAX + TX_CZB) * CZ_LROW;  // t = E^{-1} Z^T r
    float *cu = ct + 2 * TX_CBMAX;                      // Z^T r, then (S Z)^T z1
    float *cs2 = cu + 2 * TX_CBMAX;                     // t - E^{-1} (S Z)^T z1
    float *cP = cs2 + 2 * TX_CBMAX;                     // [nb][TX_CZJ] per-block partial sums
    const int2 *gbl = a.gblk + static_cast<int64_t>(q) * TX_GBMAX;
    const float *Lq = a.czl + static_cast<int64_t>(q) * (2 * TX_CBMAX * CZ_LROW);
    const float *sz = a.czsz + cs.koff * TX_CZJ;
    for (int i = threadIdx.x; i < (nc + TX_CZB) * CZ_LROW; i += TX_T) cL[i] = i < nc * CZ_LROW ? Lq[i] : 0.f;
    // Z^T r: one warp per block
    for (int b = warp; b < nb; b += TX_T / 32) {
        const int2 bl = gbl[b];
        float s0 = 0.f, s1 = 0.f;
        for (int l = lane; l < bl.y; l += 32) {
            const float v = r[bl.x + l];
            s0 += v;
            s1 = fmaf(cz_ramp(l, bl.y), v, s1);
        }
        for (int o = 16; o; o >>= 1) {
            s0 += __shfl_xor_sync(0xffffffffu, s0, o);
            s1 += __shfl_xor_sync(0xffffffffu, s1, o);
        }
        if (lane == 0) { cu[2 * b] = s0; cu[2 * b + 1] = s1; }
    }
    __syncthreads();
    if (threadIdx.x == 0) cz_solve(cL, nc, cu, ct);
    __syncthreads();
    // w = r - (S Z) t, into z
    for (int b = warp; b < nb; b += TX_T / 32) {
        const int2 bl = gbl[b];
        for (int l = lane; l < bl.y; l += 32) {
            const int i = bl.x + l;
            const float2 *row = reinterpret_cast<const float2 *>(sz + static_cast<int64_t>(i) * TX_CZJ);
            float v = r[i];
#pragma unroll
            for (int j = 0; j < 2 * TX_CZW + 1; ++j) {
                const int c = b - TX_CZW + j;
                if (c >= 0 && c < nb) {
                    const float2 e = row[j];
                    v = fmaf(-e.x, ct[2 * c], v);
                    v = fmaf(-e.y, ct[2 * c + 1], v);
                }
            }
            z[i] = v;
        }
    }
    __syncthreads();
    // z1 = M1 w, in place
    nc_precond_m1(a, S, q, z, z, gb);
    __syncthreads();
    // (S Z)^T z1: per block the sums over its rows of each stored column
    for (int b = warp; b < nb; b += TX_T / 32) {
        const int2 bl = gbl[b];
        float e[TX_CZJ];
#pragma unroll
        for (int k = 0; k < TX_CZJ; ++k) e[k] = 0.f;
        for (int l = lane; l < bl.y; l += 32) {
            const int i = bl.x + l;
            const float2 *row = reinterpret_cast<const float2 *>(sz + static_cast<int64_t>(i) * TX_CZJ);
            const float zi = z[i];
#pragma unroll
            for (int j = 0; j < 2 * TX_CZW + 1; ++j) {
                const float2 v = row[j];
                e[2 * j] = fmaf(v.x, zi, e[2 * j]);
                e[2 * j + 1] = fmaf(v.y, zi, e[2 * j + 1]);
            }
        }
#pragma unroll
        for (int k = 0; k < TX_CZJ; ++k) {
            float v = e[k];
            for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
            if (lane == 0) cP[b * TX_CZJ + k] = v;
        }
    }
    __syncthreads();
    for (int x = threadIdx.x; x < nc; x += TX_T) {
        const int c = x >> 1, sc = x & 1;
        float v = 0.f;
        for (int bp = max(0, c - TX_CZW); bp <= min(nb - 1, c + TX_CZW); ++bp)
            v += cP[bp * TX_CZJ + 2 * (c - bp + TX_CZW) + sc];
        cu[x] = v;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        cz_solve(cL, nc, cu, cs2);
        for (int x = 0; x < nc; ++x) cs2[x] = ct[x] - cs2[x];
    }
    __syncthreads();
    // z = z1 + Z (t - E^{-1} (S Z)^T z1);  r.z
    Acc2 rz[1] = {{0.f, 0.f}};
    for (int b = warp; b < nb; b += TX_T / 32) {
        const int2 bl = gbl[b];
        const float c0 = cs2[2 * b], c1 = cs2[2 * b + 1];
        for (int l = lane; l < bl.y; l += 32) {
            const int i = bl.x + l;
            const float zi = z[i] + fmaf(c1, cz_ramp(l, bl.y), c0);
            z[i] = zi;
            acc_add_prod(rz[0], r[i], zi);
        }
    }
    block_sums<1>(rz, S.red, S.out);
    return S.out[0];
}

// CG start of detscan q: r = E^T x0 (already gathered), y = 0, z = M^{-1} r,
// p = z, (r.r, r.z); nothing to do when r = 0.
__device__ void nc_cg_init(const NcorrTx &a, NcShared &S, int q, float *gb)
{
    CgState cs = a.cgs[q];
    if (cs.mode != CG_ACTIVE) return;
    const CgVec V = cg_vecs(a);
    const int64_t k0 = cs.koff;
    const int K = cs.K;
    Acc2 rr[1] = {{0.f, 0.f}};
    for (int i = threadIdx.x; i < K; i += TX_T) {
        const float v = V.r[k0 + i];
        V.y[k0 + i] = 0.f;
        acc_add_prod(rr[0], v, v);
    }
    block_sums<1>(rr, S.red, S.out);
    const double rr0 = S.out[0];
    const double rz = nc_precond(a, S, q, V.r + k0, V.z + k0, gb);
    for (int i = threadIdx.x; i < K; i += TX_T) V.p[k0 + i] = V.z[k0 + i];
    if (threadIdx.x == 0) {
        cs.rz = rz;
        cs.stop = static_cast<double>(a.tol) * a.tol * rr0;
        cs.it = 0;
        if (rr0 == 0.0) cs.mode = CG_DONE;
        a.cgs[q] = cs;
        if (cs.mode == CG_ACTIVE) atomicAdd(a.count, 1);
    }
}

// One CG iteration of detscan q after q = S p is gathered.
__device__ void nc_cg_update(const NcorrTx &a, NcShared &S, int q, float *gb, int32_t *count_next)
{
    CgState cs = a.cgs[q];
    if (cs.mode != CG_ACTIVE) return;
    const CgVec V = cg_vecs(a);
    const int64_t k0 = cs.koff;
    const int K = cs.K;
    Acc2 pq[1] = {{0.f, 0.f}};
    for (int i = threadIdx.x; i < K; i += TX_T) acc_add_prod(pq[0], V.p[k0 + i], V.q[k0 + i]);
    block_sums<1>(pq, S.red, S.out);
    const float alp = static_cast<float>(cs.rz / S.out[0]);
    Acc2 rr[1] = {{0.f, 0.f}};
    for (int i = threadIdx.x; i < K; i += TX_T) {
        V.y[k0 + i] = fmaf(alp, V.p[k0 + i], V.y[k0 + i]);
        const float rn = fmaf(-alp, V.q[k0 + i], V.r[k0 + i]);
        V.r[k0 + i] = rn;
        acc_add_prod(rr[0], rn, rn);
    }
    block_sums<1>(rr, S.red, S.out);
    const double rrn = S.out[0];
    ++cs.it;
    bool cont = true;
    if (rrn <= cs.stop) { cs.mode = CG_DONE; cont = false; }
    else if (cs.it >= a.maxit || !(rrn == rrn)) {
        cs.mode = CG_DONE;
        cont = false;
        if (threadIdx.x == 0) set_status(a.status, q, TOD_ERR_NOT_CONVERGED);
    }
    if (cont) {
        const double rzn = nc_precond(a, S, q, V.r + k0, V.z + k0, gb);
        const float beta = static_cast<float>(rzn / cs.rz);
        for (int i = threadIdx.x; i < K; i += TX_T) V.p[k0 + i] = fmaf(beta, V.p[k0 + i], V.z[k0 + i]);
        cs.rz = rzn;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        a.cgs[q] = cs;
        if (cs.mode == CG_ACTIVE) atomicAdd(count_next, 1);
    }
}

// ---------------------------------------------------------------------------
// The n_corr kernels.  Each pass is its own launch over the tiles of the
// launch range, or of the detscans a CG pass concerns (a list rebuilt after
// every CG update); the CG runs a fixed number of iterations as launches of
// their own (each returns at once when no detscan is iterating), and a
// cooperative tail kernel finishes any detscan still iterating (grid
// barriers between its passes; it returns at once when none is).
// ---------------------------------------------------------------------------
// Every work item of the launch range, a contiguous share per CTA (tiles of
// one length together).
template <class Fn>
__device__ __forceinline__ void nc_items(const NcorrTx &a, TxCtx &X, bool rows, int &cur, Fn fn)
{
    const int2 *items = rows ? a.rowitems : a.colitems;
    const int j0 = rows ? a.row_off[a.q0] : a.col_off[a.q0];
    const int j1 = rows ? a.row_off[a.q1] : a.col_off[a.q1];
    int i0, i1;
    cta_share(j1 - j0, i0, i1);
    for (int it = j0 + i0; it < j0 + i1; ++it) {
        const int2 w = items[it];
        tx_begin(X, a.txl, a.q_tx, a.off, w.x, w.y, a.off[a.q0], a.ndet, a.fsamp, a.psd, a.gain, cur, a.qsc);
        if (threadIdx.x == 0) { X.mode = a.cgs[w.x].mode; X.koff = a.cgs[w.x].koff; }
        __syncthreads();
        fn();
    }
}

// The list of the launch range's detscans in CG mode `want` (ascending),
// with exclusive running counts of their column and row items.  One CTA
// (any multiple of 32 threads up to 1024) builds it.
__device__ void nc_build_list(const NcorrTx &a, int want)
{
    __shared__ int s_w[32][3];
    __shared__ int s_base[3], s_tot[3];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    if (threadIdx.x == 0) { s_base[0] = 0; s_base[1] = 0; s_base[2] = 0; }
    __syncthreads();
    int32_t *lq = nl_q(a), *lc = nl_col(a), *lr = nl_row(a);
    for (int c0 = a.q0; c0 < a.q1; c0 += blockDim.x) {
        const int q = c0 + threadIdx.x;
        const bool in = q < a.q1 && a.cgs[q].mode == want;
        int v[3] = {in ? 1 : 0, in ? a.col_off[q + 1] - a.col_off[q] : 0, in ? a.row_off[q + 1] - a.row_off[q] : 0};
        int x[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            int t = v[k];
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int u = __shfl_up_sync(0xffffffffu, t, o);
                if (lane >= o) t += u;
            }
            x[k] = t - v[k];                       // exclusive within the warp
            if (lane == 31) s_w[warp][k] = t;
        }
        __syncthreads();
        if (threadIdx.x < 3) {                     // warp totals -> exclusive warp offsets
            int acc = 0;
            for (int w = 0; w < nw; ++w) { const int t = s_w[w][threadIdx.x]; s_w[w][threadIdx.x] = acc; acc += t; }
            s_tot[threadIdx.x] = acc;
        }
        __syncthreads();
        if (in) {
            const int i = s_base[0] + s_w[warp][0] + x[0];
            lq[i] = q;
            lc[i] = s_base[1] + s_w[warp][1] + x[1];
            lr[i] = s_base[2] + s_w[warp][2] + x[2];
        }
        __syncthreads();
        if (threadIdx.x < 3) s_base[threadIdx.x] += s_tot[threadIdx.x];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        a.list[0] = s_base[0];
        lc[s_base[0]] = s_base[1];
        lr[s_base[0]] = s_base[2];
    }
}
__global__ void __launch_bounds__(1024) k_nc_list(NcorrTx a, int want, int par)
{
    if (par >= 0 && *reinterpret_cast<volatile const int32_t *>(a.count + par) == 0) return;
    nc_build_list(a, want);
}

// The listed detscans' column (or row) items, a contiguous share per CTA:
// consecutive items of a CTA are mostly tiles of one detscan.
template <class Fn>
__device__ __forceinline__ void nc_list_items(const NcorrTx &a, TxCtx &X, bool rows, int &cur, Fn fn)
{
    const int n = *reinterpret_cast<volatile const int32_t *>(a.list);
    if (n <= 0) return;
    const int32_t *lq = nl_q(a), *lo = rows ? nl_row(a) : nl_col(a);
    int i0, i1;
    cta_share(lo[n], i0, i1);
    if (i0 >= i1) return;
    int pos = 0, hi = n - 1;                      // last detscan whose items start at or before i0
    while (pos < hi) {
        const int mid = (pos + hi + 1) >> 1;
        if (lo[mid] <= i0) pos = mid; else hi = mid - 1;
    }
    for (int ii = i0; ii < i1; ++ii) {
        while (lo[pos + 1] <= ii) ++pos;
        const int q = lq[pos];
        tx_begin(X, a.txl, a.q_tx, a.off, q, ii - lo[pos], a.off[a.q0], a.ndet, a.fsamp, a.psd, a.gain, cur, a.qsc);
        if (threadIdx.x == 0) { X.mode = a.cgs[q].mode; X.koff = a.cgs[q].koff; }
        __syncthreads();
        fn();
    }
}


__global__ void __launch_bounds__(TX_T) k_nc_flag_count(NcorrTx a)
{
    __shared__ NcShared S;
    nc_flag_count(a, S);
}
__global__ void k_nc_flag_scan(NcorrTx a, int G)
{
    if (blockIdx.x != 0 || threadIdx.x != 0) return;
    int64_t acc = 0;
    for (int c = 0; c < G; ++c) { const int64_t v = a.chunk[c]; a.chunk[c] = acc; acc += v; }
    a.chunk[G] = acc;
}
__global__ void __launch_bounds__(TX_T) k_nc_flag_write(NcorrTx a)
{
    __shared__ NcShared S;
    nc_flag_write(a, S);
}
__global__ void __launch_bounds__(TX_T) k_nc_index(NcorrTx a)
{
    __shared__ NcShared S;
    if (blockIdx.x == 0 && threadIdx.x == 0) { a.count[0] = 0; a.count[1] = 0; }
    for (int q = a.q0 + blockIdx.x; q < a.q1; q += gridDim.x) {
        nc_detscan_index(a, S, q);
        __syncthreads();
    }
}
__global__ void __launch_bounds__(TX_T) k_nc_coarse(NcorrTx a)
{
    for (int q = a.q0 + blockIdx.x; q < a.q1; q += gridDim.x) nc_coarse_setup(a, q);
}
__global__ void __launch_bounds__(TX_T, 3) k_nc_rhs_cols(NcorrTx a)
{
    extern __shared__ __align__(16) float2 tx_smem[];
    __shared__ TxCtx X;
    const uint64_t gi = a.rng.gibbs_iter_dev ? *a.rng.gibbs_iter_dev : a.rng.gibbs_iter;
    int cur = -1;
    nc_items(a, X, false, cur, [&] { nc_rhs_cols(a, X, tx_smem, tx_smem + TX_TILE, gi); });
}
__global__ void __launch_bounds__(TX_T, 3) k_nc_rhs_rows(NcorrTx a)
{
    extern __shared__ __align__(16) float2 tx_smem[];
    __shared__ TxCtx X;
    const uint64_t gi = a.rng.gibbs_iter_dev ? *a.rng.gibbs_iter_dev : a.rng.gibbs_iter;
    int cur = -1;
    nc_items(a, X, true, cur, [&] { nc_rhs_rows(a, X, tx_smem, tx_smem + TX_TILE, gi); });
}
__global__ void __launch_bounds__(TX_T, 3) k_nc_x0_cols(NcorrTx a)
{
    extern __shared__ __align__(16) float2 tx_smem[];
    __shared__ TxCtx X;
    int cur = -1;
    nc_items(a, X, false, cur, [&] { nc_x0_cols(a, X, tx_smem, tx_smem + TX_TILE); });
}
__global__ void __launch_bounds__(TX_T, 3) k_nc_cg_init(NcorrTx a)
{
    extern __shared__ __align__(16) float2 tx_smem[];
    __shared__ NcShared S;
    for (int q = a.q0 + blockIdx.x; q < a.q1; q += gridDim.x) {
        __syncthreads();
        nc_cg_init(a, S, q, reinterpret_cast<float *>(tx_smem));
    }
}
// One CG iteration (parity par: count[par] active detscans going in, the
// update counts into count[par ^ 1]), or with FINAL the correction B^{-1} E y.
template <bool FINAL>
__global__ void __launch_bounds__(TX_T, 3) k_nc_scatter(NcorrTx a, int par)
{
    extern __shared__ __align__(16) float2 tx_smem[];
    __shared__ TxCtx X;
    if (!FINAL) {
        if (blockIdx.x == 0 && threadIdx.x == 0) a.count[par ^ 1] = 0;
        if (*reinterpret_cast<volatile const int32_t *>(a.count + par) == 0) return;
    }
    const CgVec V = cg_vecs(a);
    int cur = -1;
    nc_list_items(a, X, false, cur, [&] { nc_scatter_cols(a, X, tx_smem, tx_smem + TX_TILE, FINAL ? V.y : V.p); });
}
template <bool FINAL>
__global__ void __launch_bounds__(TX_T, 3) k_nc_filter(NcorrTx a, int par)
{
    extern __shared__ __align__(16) float2 tx_smem[];
    __shared__ TxCtx X;
    if (!FINAL && *reinterpret_cast<volatile const int32_t *>(a.count + par) == 0) return;
    int cur = -1;
    nc_list_items(a, X, true, cur, [&] { nc_filter_rows<FINAL>(a, X, tx_smem, tx_smem + TX_TILE); });
}
template <bool FINAL>
__global__ void __launch_bounds__(TX_T, 3) k_nc_gather(NcorrTx a, int par)
{
    extern __shared__ __align__(16) float2 tx_smem[];
    __shared__ TxCtx X;
    if (!FINAL && *reinterpret_cast<volatile const int32_t *>(a.count + par) == 0) return;
    const CgVec V = cg_vecs(a);
    int cur = -1;
    nc_list_items(a, X, false, cur,
                  [&] { nc_gather_cols<FINAL>(a, X, tx_smem, tx_smem + TX_TILE, FINAL ? nullptr : V.q); });
}
// the listed (iterating) detscans' CG update
__device__ __forceinline__ void nc_update_listed(const NcorrTx &a, NcShared &S, float *gb, int32_t *count_next)
{
    const int n = *reinterpret_cast<volatile const int32_t *>(a.list);
    for (int i = blockIdx.x; i < n; i += gridDim.x) {
        __syncthreads();
        nc_cg_update(a, S, nl_q(a)[i], gb, count_next);
    }
}
__global__ void __launch_bounds__(TX_T, 3) k_nc_update(NcorrTx a, int par)
{
    extern __shared__ __align__(16) float2 tx_smem[];
    __shared__ NcShared S;
    if (*reinterpret_cast<volatile const int32_t *>(a.count + par) == 0) return;
    nc_update_listed(a, S, reinterpret_cast<float *>(tx_smem), a.count + (par ^ 1));
}
// The iterations left after the launched ones, in one cooperative launch:
// the passes over the listed detscans with grid barriers between them, the
// list rebuilt by CTA 0 after each update.
__global__ void __launch_bounds__(TX_T, 2) k_nc_tail(NcorrTx a, int par)
{
    extern __shared__ __align__(16) float2 tx_smem[];
    __shared__ NcShared S;
    cgrp::grid_group grid = cgrp::this_grid();
    const CgVec V = cg_vecs(a);
    int cur = -1;
    for (;;) {
        if (*reinterpret_cast<volatile const int32_t *>(a.count + par) == 0) break;
        if (blockIdx.x == 0) nc_build_list(a, CG_ACTIVE);
        grid.sync();
        if (blockIdx.x == 0 && threadIdx.x == 0) a.count[par ^ 1] = 0;
        nc_list_items(a, S.X, false, cur, [&] { nc_scatter_cols(a, S.X, tx_smem, tx_smem + TX_TILE, V.p); });
        grid.sync();
        nc_list_items(a, S.X, true, cur, [&] { nc_filter_rows<false>(a, S.X, tx_smem, tx_smem + TX_TILE); });
        grid.sync();
        nc_list_items(a, S.X, false, cur, [&] { nc_gather_cols<false>(a, S.X, tx_smem, tx_smem + TX_TILE, V.q); });
        grid.sync();
        nc_update_listed(a, S, reinterpret_cast<float *>(tx_smem), a.count + (par ^ 1));
        grid.sync();
        par ^= 1;
    }
}
// Iteration counts; detscans left at x0 for want of CG room are reported.
__global__ void k_nc_finish(NcorrTx a)
{
    const int q = a.q0 + blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= a.q1) return;
    const CgState cs = a.cgs[q];
    if (a.iters) a.iters[q] = cs.it;
    if (cs.mode == CG_OVER) set_status(a.status, q, TOD_ERR_NOT_CONVERGED);
}

// ===========================================================================
// launchers
// ===========================================================================
static size_t tx_smem_bytes(bool fp64) { return (fp64 ? sizeof(double2) : sizeof(float2)) * 2 * TX_TILE; }
constexpr size_t kGbBytes = (5 * TX_GBCAP + CZ_FLOATS) * sizeof(float);   // preconditioner staging
static_assert(kGbBytes <= sizeof(float2) * 2 * TX_TILE, "the preconditioner staging fits the tile buffers");
constexpr int NC_LAUNCHED_ITERS = 8;                                // CG iterations as separate launches

template <class K>
static cudaError_t smem_attr(K k, size_t bytes) {
    return cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(bytes));
}

cudaError_t setup_tx_kernels(Plan &p)
{
    cudaError_t e;
    const size_t s32 = tx_smem_bytes(false), s64 = tx_smem_bytes(true);
    const size_t sgb = std::max(s32, kGbBytes);
    if ((e = smem_attr(k_gain_cols, s32)) || (e = smem_attr(k_gain_rows, s32)) || (e = smem_attr(k_gain_colsinv, s32)))
        return e;
    if ((e = smem_attr(k_chi2_cols<float2>, s32)) || (e = smem_attr(k_chi2_rows<float2>, s32)) ||
        (e = smem_attr(k_chi2_colsinv<float2>, s32)))
        return e;
    if ((e = smem_attr(k_chi2_cols<double2>, s64)) || (e = smem_attr(k_chi2_rows<double2>, s64)) ||
        (e = smem_attr(k_chi2_colsinv<double2>, s64)))
        return e;
    if ((e = smem_attr(k_nc_rhs_cols, s32)) || (e = smem_attr(k_nc_rhs_rows, s32)) ||
        (e = smem_attr(k_nc_x0_cols, s32)) || (e = smem_attr(k_nc_cg_init, sgb)) ||
        (e = smem_attr(k_nc_scatter<false>, s32)) || (e = smem_attr(k_nc_scatter<true>, s32)) ||
        (e = smem_attr(k_nc_filter<false>, s32)) || (e = smem_attr(k_nc_filter<true>, s32)) ||
        (e = smem_attr(k_nc_gather<false>, s32)) || (e = smem_attr(k_nc_gather<true>, s32)) ||
        (e = smem_attr(k_nc_update, sgb)) || (e = smem_attr(k_nc_tail, sgb)))
        return e;
    int dev = 0, nsm = 0, per = 0;
    if ((e = cudaGetDevice(&dev))) return e;
    if ((e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev))) return e;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_nc_tail, TX_T, sgb))) return e;
    p.coop_grid = std::max(1, per) * nsm;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_gain_rows, TX_T, s32))) return e;
    p.pass_grid = std::max(1, per) * nsm;
    return cudaSuccess;
}

static int grid_for(const Plan &p, int nitems) { return std::max(1, std::min(nitems, p.pass_grid)); }

cudaError_t launch_tx_gain(const Plan &p, const float *d, const float *s, const uint32_t *flags, const double *psd,
                           tod_rng rng, int mode, double *g, double *mu, double *sig, cudaStream_t st, int q0, int q1)
{
    if (q1 <= q0) return cudaSuccess;
    GainTx a = {};
    a.d = d; a.s = s; a.flags = flags; a.psd = psd; a.off = p.off; a.txl = p.txl; a.q_tx = p.q_tx; a.tw = p.txtw;
    a.ndet = p.ndet; a.fsamp = p.fsamp; a.obase = p.h_off[q0]; a.Y = p.ybuf; a.part = p.part; a.qsc = p.qsc;
    const int c0 = p.h_col_off[q0], c1 = p.h_col_off[q1], r0 = p.h_row_off[q0], r1 = p.h_row_off[q1];
    const size_t sm = tx_smem_bytes(false);
    {
        KTIME(TOD_KT_DET_SCALARS);
        k_det_scalars<<<(q1 - q0 + 127) / 128, 128, 0, st>>>(psd, nullptr, p.off, p.ndet, p.fsamp, q0, q1, p.qsc);
    }
    // column items' partials at part[4 c], row items' at part[4 (ncol + r)]
    double *cpart = p.part;
    double *rpart = p.part + 4 * static_cast<int64_t>(p.h_col_off[p.nq]);
    a.items = p.colitems; a.item0 = c0; a.nitems = c1 - c0; a.part = cpart;
    {
        KTIME(TOD_KT_GAIN_COLS);
        k_gain_cols<<<grid_for(p, a.nitems), TX_T, sm, st>>>(a);
    }
    a.items = p.rowitems; a.item0 = r0; a.nitems = r1 - r0; a.part = rpart;
    {
        KTIME(TOD_KT_GAIN_ROWS);
        k_gain_rows<<<grid_for(p, a.nitems), TX_T, sm, st>>>(a);
    }
    a.items = p.colitems; a.item0 = c0; a.nitems = c1 - c0; a.part = cpart;
    {
        KTIME(TOD_KT_GAIN_COLSINV);
        k_gain_colsinv<<<grid_for(p, a.nitems), TX_T, sm, st>>>(a);
    }
    {
        KTIME(TOD_KT_GAIN_FIN);
        k_gain_fin<<<(q1 - q0 + 255) / 256, 256, 0, st>>>(rpart, cpart, p.row_off, p.col_off, q0, q1, 0, 0, rng, mode,
                                                          g, mu, sig, p.status);
    }
    return cudaGetLastError();
}

template <class V>
static cudaError_t chi2_range(const Plan &p, const float *d, const void *s, const double *gain,
                              const uint32_t *flags, const double *psd, double *chi2_q, double *dgain, double *dpsd_q,
                              void *v_out, cudaStream_t st, int q0, int q1)
{
    Chi2Tx<V> a = {};
    a.d = d; a.s = s; a.gain = gain; a.flags = flags; a.psd = psd; a.off = p.off; a.txl = p.txl; a.q_tx = p.q_tx;
    a.tw = reinterpret_cast<const V *>(sizeof(V) == sizeof(float2) ? static_cast<const void *>(p.txtw)
                                                                     : static_cast<const void *>(p.txtw64));
    a.ndet = p.ndet; a.fsamp = p.fsamp; a.obase = p.h_off[q0];
    a.Y = reinterpret_cast<V *>(p.ybuf);
    a.v_out = v_out;
    const size_t sm = tx_smem_bytes(sizeof(V) != sizeof(float2));
    const int c0 = p.h_col_off[q0], c1 = p.h_col_off[q1], r0 = p.h_row_off[q0], r1 = p.h_row_off[q1];
    double *cpart = p.part;
    double *rpart = p.part + 4 * static_cast<int64_t>(p.h_col_off[p.nq]);
    a.items = p.colitems; a.item0 = c0; a.nitems = c1 - c0; a.part = cpart;
    {
        KTIME(TOD_KT_CHI2_COLS);
        k_chi2_cols<V><<<grid_for(p, a.nitems), TX_T, sm, st>>>(a);
    }
    a.items = p.rowitems; a.item0 = r0; a.nitems = r1 - r0; a.part = rpart;
    {
        KTIME(TOD_KT_CHI2_ROWS);
        k_chi2_rows<V><<<grid_for(p, a.nitems), TX_T, sm, st>>>(a);
    }
    a.items = p.colitems; a.item0 = c0; a.nitems = c1 - c0; a.part = cpart;
    {
        KTIME(TOD_KT_CHI2_COLSINV);
        k_chi2_colsinv<V><<<grid_for(p, a.nitems), TX_T, sm, st>>>(a);
    }
    {
        KTIME(TOD_KT_CHI2_FIN);
        k_chi2_fin<<<(q1 - q0 + 255) / 256, 256, 0, st>>>(rpart, cpart, p.row_off, p.col_off, q0, q1, 0, 0, chi2_q, dgain,
                                                           dpsd_q);
    }
    return cudaGetLastError();
}

cudaError_t launch_tx_chi2(const Plan &p, bool fp64, const float *d, const void *s, const double *gain,
                           const uint32_t *flags, const double *psd, double *chi2_q, double *dgain, double *dpsd_q,
                           double *total, double *dpsd_det, void *v_out, cudaStream_t st)
{
    cudaError_t e = cudaSuccess;
    if (!fp64) {
        e = chi2_range<float2>(p, d, s, gain, flags, psd, chi2_q, dgain, dpsd_q, v_out, st, 0, p.nq);
    } else {
        // the intermediate holds ybuf_floats / 4 double2: waves of detscans of
        // at most ybuf_floats / 2 samples (a whole detscan always fits)
        int q = 0;
        while (q < p.nq && e == cudaSuccess) {
            int q1 = q + 1;
            while (q1 < p.nq && p.h_off[q1 + 1] - p.h_off[q] <= p.ybuf_floats / 2) ++q1;
            e = chi2_range<double2>(p, d, s, gain, flags, psd, chi2_q, dgain, dpsd_q, v_out, st, q, q1);
            q = q1;
        }
    }
    if (e != cudaSuccess) return e;
    {
        KTIME(TOD_KT_CHI2_FIN);
        k_chi2_total<<<1, 1, 0, st>>>(chi2_q, dpsd_q, p.nq, p.ndet, total, dpsd_det);
    }
    return cudaGetLastError();
}

cudaError_t launch_tx_ncorr(const Plan &p, const float *d, const float *s, const double *gain,
                            const uint32_t *flags, const double *psd, tod_rng rng, int mode, float tol, int maxit,
                            float *x, int32_t *iters, cudaStream_t st, int q0, int q1, const TxNcorrScratch &sc,
                            int grid)
{
    if (q1 <= q0) return cudaSuccess;
    NcorrTx a = {};
    a.d = d; a.s = s; a.gain = gain; a.flags = flags; a.psd = psd; a.off = p.off; a.txl = p.txl; a.q_tx = p.q_tx;
    a.tw = p.txtw; a.colitems = p.colitems; a.rowitems = p.rowitems; a.col_off = p.col_off; a.row_off = p.row_off;
    a.q0 = q0; a.q1 = q1; a.ndet = p.ndet; a.fsamp = p.fsamp; a.rng = rng; a.mode = mode; a.tol = tol;
    a.maxit = maxit; a.x_out = x; a.iters = iters; a.status = p.status; a.spec_out = p.spec_out;
    a.xtab = p.use_prec ? p.xtab : nullptr; a.lvalid = p.lvalid;
    a.cztab = p.cztab; a.href = p.cz_href; a.gbpos = p.gbpos; a.czsz = (p.use_prec && p.use_coarse) ? p.czsz : nullptr;
    a.czcap = p.czcap; a.czl = p.czl;
    a.Y = sc.Y; a.wpre = sc.wpre; a.chunk = p.chunk; a.cgs = p.cgs; a.gblk = p.gblk; a.gnb = p.gnb;
    a.cgv = sc.cgv; a.cgcap = sc.cgcap; a.count = p.cg_count; a.qsc = p.qsc; a.list = p.nclist;
    const size_t s32 = tx_smem_bytes(false), sgb = std::max(s32, kGbBytes);
    const int nq = q1 - q0;
    const int ncol = p.h_col_off[q1] - p.h_col_off[q0], nrow = p.h_row_off[q1] - p.h_row_off[q0];
    const int gc = std::min(grid_for(p, ncol), grid), gr = std::min(grid_for(p, nrow), grid);
    const int gq = std::min(nq, std::max(1, grid));
    // flag index (the chunked scan uses the same grid for count and write)
    const int gf = std::max(1, std::min(p.pass_grid, grid));
    {
        KTIME(TOD_KT_NC_FLAG_COUNT);
        k_nc_flag_count<<<gf, TX_T, 0, st>>>(a);
    }
    {
        KTIME(TOD_KT_NC_FLAG_SCAN);
        k_nc_flag_scan<<<1, 1, 0, st>>>(a, gf);
    }
    {
        KTIME(TOD_KT_NC_FLAG_WRITE);
        k_nc_flag_write<<<gf, TX_T, 0, st>>>(a);
    }
    {
        KTIME(TOD_KT_NC_INDEX);
        k_nc_index<<<gq, TX_T, 0, st>>>(a);
    }
    {
        KTIME(TOD_KT_NC_COARSE);
        k_nc_coarse<<<gq, TX_T, 0, st>>>(a);
    }
    // x0 = B^{-1} b
    {
        KTIME(TOD_KT_NC_RHS_COLS);
        k_nc_rhs_cols<<<gc, TX_T, s32, st>>>(a);
    }
    {
        KTIME(TOD_KT_NC_RHS_ROWS);
        k_nc_rhs_rows<<<gr, TX_T, s32, st>>>(a);
    }
    {
        KTIME(TOD_KT_NC_X0_COLS);
        k_nc_x0_cols<<<gc, TX_T, s32, st>>>(a);
    }
    // CG on the Schur complement
    {
        KTIME(TOD_KT_NC_CG_INIT);
        k_nc_cg_init<<<gq, TX_T, sgb, st>>>(a);
    }
    int par = 0;
    {
        KTIME(TOD_KT_NC_LIST);
        k_nc_list<<<1, 1024, 0, st>>>(a, CG_ACTIVE, par);
    }
    for (int it = 0; it < NC_LAUNCHED_ITERS; ++it, par ^= 1) {
        {
            KTIME(TOD_KT_NC_SCATTER);
            k_nc_scatter<false><<<gc, TX_T, s32, st>>>(a, par);
        }
        {
            KTIME(TOD_KT_NC_FILTER);
            k_nc_filter<false><<<gr, TX_T, s32, st>>>(a, par);
        }
        {
            KTIME(TOD_KT_NC_GATHER);
            k_nc_gather<false><<<gc, TX_T, s32, st>>>(a, par);
        }
        {
            KTIME(TOD_KT_NC_UPDATE);
            k_nc_update<<<gq, TX_T, sgb, st>>>(a, par);
        }
        {
            KTIME(TOD_KT_NC_LIST);
            k_nc_list<<<1, 1024, 0, st>>>(a, CG_ACTIVE, par ^ 1);
        }
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    int tail_par = par;
    void *args[] = {&a, &tail_par};
    {
        KTIME(TOD_KT_NC_TAIL);
        e = cudaLaunchCooperativeKernel(reinterpret_cast<const void *>(k_nc_tail),
                                        dim3(std::max(1, std::min(grid, p.coop_grid))), dim3(TX_T), args, sgb, st);
    }
    if (e != cudaSuccess) return e;
    {
        KTIME(TOD_KT_NC_LIST);
        k_nc_list<<<1, 1024, 0, st>>>(a, CG_DONE, -1);
    }
    // x = x0 + B^{-1} E y for every detscan that ran the CG
    {
        KTIME(TOD_KT_NC_SCATTER_FINAL);
        k_nc_scatter<true><<<gc, TX_T, s32, st>>>(a, 0);
    }
    {
        KTIME(TOD_KT_NC_FILTER_FINAL);
        k_nc_filter<true><<<gr, TX_T, s32, st>>>(a, 0);
    }
    {
        KTIME(TOD_KT_NC_GATHER_FINAL);
        k_nc_gather<true><<<gc, TX_T, s32, st>>>(a, 0);
    }
    {
        KTIME(TOD_KT_NC_FINISH);
        k_nc_finish<<<(nq + 255) / 256, 256, 0, st>>>(a);
    }
    return cudaGetLastError();
}

}  // namespace tg
