// A6 binning into per-pixel normal equations and A7 per-pixel 3x3 solve
// (paper Sect. 5 table rows "TOD binning" and "Map solution (Ax=b for each
// pixel)"; Sect. 2.4: coadded on the fly, synchronised once).
//
// Binning is a deterministic two-level segmented reduction.  The plan holds,
// for every detscan, its pixel-sorted order (stable in time), the runs of
// equal pixel ("pairs" of detscan and pixel) ranked over the band by (pixel,
// detscan), and tiles of consecutive whole runs of one detscan (at most
// BIN_TILE samples, or one longer run alone).
//   k_bin:    one CTA per tile gathers the tile's data, residual and
//             psi/flag words in sorted order into shared memory (the
//             detscan's samples stay in L2 while its tiles run), then one
//             thread sums each run.  Products of FP32 values are formed
//             exactly and summed as FP32 double-words (FP64 accuracy at FP32
//             issue rate), the residual d - x taken exactly as a
//             double-word; each run's sums are scaled by the detscan's
//             g^2/sigma0^2, g/sigma0^2 in FP64 and written at the run's rank.
//             A run longer than a tile is summed by the whole CTA with a
//             fixed-order tree.
//   k_reduce: one thread per pixel adds its contiguous runs in FP64, in
//             ascending detscan order.
#include <algorithm>
#include "common.cuh"
#include "internal.cuh"


namespace tg {

constexpr int BIN_T = 256;

struct BinArgs {
    const uint16_t *psi;
    const float *d, *x;
    const double *gain;
    const uint32_t *flags;
    const double *psd;
    const int64_t *off;
    const uint32_t *ld_t;         // load order -> time index within the detscan
    const uint16_t *ld_pos;       // load order -> run-major position within the tile
    const int64_t *pair_start;
    const int32_t *pair_len, *pair_slot;
    const int32_t *tile_q, *tile_r0;
    const float2 *trig;
    int ndet;
    double *rec;
    // adjoint of the projection: no mask (flags null), weights 0 and g, and,
    // when y64 is set, the FP64 input y = hi + lo read as d = hi, x = -lo
    bool adjoint;
    const double *y64;
};

// sum of two double-words (two-sum on the heads, tails added)
__device__ __forceinline__ Acc2 acc_merge(const Acc2 &a, const Acc2 &b) {
    Acc2 r = a;
    acc_add(r, b.s);
    r.c = __fadd_rn(r.c, b.c);
    return r;
}

// the per-run sums: 1 (as hits), c, s, cc, cs, ss, r, cr, sr with r = d - x
// (taken exactly as a double-word: its head and tail)
constexpr int NSUM = 8;
struct RunSums {
    Acc2 a[NSUM];
    int hits;
};
__device__ __forceinline__ void sums_zero(RunSums &r) {
#pragma unroll
    for (int i = 0; i < NSUM; ++i) r.a[i] = Acc2{0.f, 0.f};
    r.hits = 0;
}
__device__ __forceinline__ void sums_add(RunSums &r, float2 cs, float dv, float xv) {
    ++r.hits;
    acc_add(r.a[0], cs.x);
    acc_add(r.a[1], cs.y);
    acc_add_prod(r.a[2], cs.x, cs.x);
    acc_add_prod(r.a[3], cs.x, cs.y);
    acc_add_prod(r.a[4], cs.y, cs.y);
    // r = d - x exactly: head rh (rounded difference) and tail rl (two-sum)
    const float rh = __fsub_rn(dv, xv);
    const float bb = __fsub_rn(rh, dv);
    const float rl = __fadd_rn(__fsub_rn(dv, __fsub_rn(rh, bb)), __fsub_rn(-xv, bb));
    acc_add(r.a[5], rh);
    r.a[5].c = __fadd_rn(r.a[5].c, rl);
    // c r and s r: exact products of the heads, the tails' products (below
    // 2^-24 of them) added to the compensation words
    acc_add_prod(r.a[6], cs.x, rh);
    r.a[6].c = __fmaf_rn(cs.x, rl, r.a[6].c);
    acc_add_prod(r.a[7], cs.y, rh);
    r.a[7].c = __fmaf_rn(cs.y, rl, r.a[7].c);
}
__device__ __forceinline__ void sums_store(const RunSums &r, double wA, double wb, double *rr) {
    rr[0] = wA * r.hits;
    rr[1] = wA * acc_value(r.a[0]);
    rr[2] = wA * acc_value(r.a[1]);
    rr[3] = wA * acc_value(r.a[2]);
    rr[4] = wA * acc_value(r.a[3]);
    rr[5] = wA * acc_value(r.a[4]);
    rr[6] = wb * acc_value(r.a[5]);
    rr[7] = wb * acc_value(r.a[6]);
    rr[8] = wb * acc_value(r.a[7]);
    rr[9] = static_cast<double>(r.hits);
}

__device__ __forceinline__ uint16_t psi_flag(const BinArgs &a, int64_t tg) {
    const uint32_t fb = a.flags ? (__ldg(a.flags + (tg >> 5)) >> (tg & 31)) & 1u : 0u;
    return static_cast<uint16_t>((__ldg(a.psi + tg) & 0x0FFF) | (fb << 15));
}

// data and residual of sample tg (the adjoint's input: y, or the head and
// negated tail of the FP64 y, whose difference is y to FP64 accuracy)
__device__ __forceinline__ void load_dx(const BinArgs &a, int64_t tg, float &dv, float &xv) {
    if (a.y64) {
        const double y = __ldg(a.y64 + tg);
        const float hi = static_cast<float>(y);
        dv = hi;
        xv = -static_cast<float>(y - static_cast<double>(hi));
    } else {
        dv = __ldg(a.d + tg);
        xv = a.x ? __ldg(a.x + tg) : 0.f;
    }
}

__global__ void __launch_bounds__(BIN_T) k_bin(BinArgs a)
{
    __shared__ float s_d[BIN_TILE], s_x[BIN_TILE];
    __shared__ float2 s_cs[BIN_TILE];
    __shared__ Acc2 s_red[BIN_T / 32][NSUM];
    __shared__ int s_hits[BIN_T / 32];
    __shared__ Acc2 s_out[BIN_T / 4][10];          // a quad's ten run outputs as double-words
    const int tile = blockIdx.x;
    const int q = a.tile_q[tile];
    const int r0 = a.tile_r0[tile], nr = a.tile_r0[tile + 1] - r0;
    const int64_t o = a.off[q];
    const int64_t s0 = a.pair_start[r0];
    const int cnt = static_cast<int>(a.pair_start[r0 + nr - 1] + a.pair_len[r0 + nr - 1] - s0);
    // the detscan's weights g^2/sigma0^2 and g/sigma0^2: FP64 divisions once,
    // by thread 0 (FP64 issues at 1/64 of the FP32 rate on this part)
    __shared__ double s_w[2];
    if (threadIdx.x == 0) {
        const double gq = a.gain[q];
        if (a.adjoint) {
            s_w[0] = 0.0;
            s_w[1] = gq;
        } else {
            const double sig0 = a.psd[3 * (q % a.ndet)];
            s_w[0] = gq * gq / (sig0 * sig0);
            s_w[1] = gq / (sig0 * sig0);
        }
    }
    __syncthreads();
    const double wA = s_w[0], wb = s_w[1];

    if (cnt > BIN_TILE) {
        // one run longer than a tile: strided partial sums, then a fixed-order tree
        RunSums r;
        sums_zero(r);
        for (int i = threadIdx.x; i < cnt; i += BIN_T) {
            const int64_t tg = o + __ldg(a.ld_t + s0 + i);     // a single run: run order
            const uint16_t pf = psi_flag(a, tg);
            if (pf >> 15) continue;
            float dv, xv;
            load_dx(a, tg, dv, xv);
            sums_add(r, __ldg(a.trig + (pf & 0x0FFF)), dv, xv);
        }
#pragma unroll
        for (int ofs = 16; ofs; ofs >>= 1) {
#pragma unroll
            for (int k = 0; k < NSUM; ++k) {
                Acc2 o2;
                o2.s = __shfl_down_sync(0xffffffffu, r.a[k].s, ofs);
                o2.c = __shfl_down_sync(0xffffffffu, r.a[k].c, ofs);
                r.a[k] = acc_merge(r.a[k], o2);
            }
            r.hits += __shfl_down_sync(0xffffffffu, r.hits, ofs);
        }
        const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
        if (lane == 0) {
#pragma unroll
            for (int k = 0; k < NSUM; ++k) s_red[warp][k] = r.a[k];
            s_hits[warp] = r.hits;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            for (int w = 1; w < BIN_T / 32; ++w) {
#pragma unroll
                for (int k = 0; k < NSUM; ++k) r.a[k] = acc_merge(r.a[k], s_red[w][k]);
                r.hits += s_hits[w];
            }
            sums_store(r, wA, wb, a.rec + static_cast<int64_t>(a.pair_slot[r0]) * 10);
        }
        return;
    }

    // gather in the tile's load order (the k-th sample of each run, k = 0,
    // 1, ..: a warp's 32 samples are close in time, so they share sectors):
    // the positions first, then every value load of the thread in flight
    // together, each value into its run-major slot; cos 2psi and sin 2psi
    // are staged with the data, and a flagged sample is marked by cos = 2
    constexpr int PER = BIN_TILE / BIN_T;
    int idx[PER], pos[PER];
#pragma unroll
    for (int u = 0; u < PER; ++u) {
        const int i = threadIdx.x + u * BIN_T;
        idx[u] = -1;
        pos[u] = 0;
        if (i < cnt) {
            idx[u] = static_cast<int>(__ldg(a.ld_t + s0 + i));
            pos[u] = __ldg(a.ld_pos + s0 + i);
        }
    }
#pragma unroll
    for (int u = 0; u < PER; ++u) {
        if (idx[u] < 0) continue;
        const int64_t tg = o + idx[u];
        const uint16_t pf = psi_flag(a, tg);
        float2 cs = __ldg(a.trig + (pf & 0x0FFF));
        if (pf >> 15) cs.x = 2.0f;
        const int i = pos[u];
        s_cs[i] = cs;
        load_dx(a, tg, s_d[i], s_x[i]);
    }
    __syncthreads();
    // four lanes per run: lane j of the quad takes samples j, j+4, ...; the
    // quad's partial sums are merged in a fixed order (deterministic)
    const int quad = threadIdx.x >> 2, ql = threadIdx.x & 3;
    for (int rb = 0; rb < nr; rb += BIN_T / 4) {
        const int r = rb + quad;
        RunSums rs;
        sums_zero(rs);
        int pr = -1;
        if (r < nr) {
            pr = r0 + r;
            const int st = static_cast<int>(a.pair_start[pr] - s0);
            const int len = a.pair_len[pr];
            for (int i = st + ql; i < st + len; i += 4) {
                const float2 cs = s_cs[i];
                if (cs.x > 1.5f) continue;
                sums_add(rs, cs, s_d[i], s_x[i]);
            }
        }
#pragma unroll
        for (int ofs = 1; ofs <= 2; ofs <<= 1) {
#pragma unroll
            for (int k = 0; k < NSUM; ++k) {
                Acc2 o2;
                o2.s = __shfl_xor_sync(0xffffffffu, rs.a[k].s, ofs);
                o2.c = __shfl_xor_sync(0xffffffffu, rs.a[k].c, ofs);
                rs.a[k] = (ql & ofs) ? acc_merge(o2, rs.a[k]) : acc_merge(rs.a[k], o2);
            }
            rs.hits += __shfl_xor_sync(0xffffffffu, rs.hits, ofs);
        }
        // the ten outputs in FP64, spread over the quad's lanes (lane ql takes
        // outputs ql, ql + 4, ql + 8: FP64 issues slowly on this part, so every
        // lane of its warp instructions works)
        if (pr >= 0 && ql == 0) {
            Acc2 *o = s_out[quad];
            o[0] = Acc2{static_cast<float>(rs.hits), 0.f};      // hits <= BIN_TILE: exact
#pragma unroll
            for (int k = 0; k < 5; ++k) o[1 + k] = rs.a[k];
#pragma unroll
            for (int k = 0; k < 3; ++k) o[6 + k] = rs.a[5 + k];
            o[9] = o[0];
        }
        __syncwarp();
        if (pr >= 0) {
            double *rr = a.rec + static_cast<int64_t>(a.pair_slot[pr]) * 10;
            for (int i = ql; i < 10; i += 4) {
                const Acc2 v = s_out[quad][i];
                const double w = i == 9 ? 1.0 : (i <= 5 ? wA : wb);
                rr[i] = w * acc_value(v);
            }
        }
        __syncwarp();
    }
}

// Per pixel, its runs added in ascending detscan order as a double-double
// (Knuth two-sum: hi + lo carries the sum to about 2^-104 of its size), then
// rounded once.  The rounded total is the sum of the runs correctly rounded
// but for sums within ~2^-104 of a rounding tie, whatever the grouping: the
// normal equations of a band split into scan ranges and combined with
// tod_combine_partials equal those of the whole band.
struct DD { double hi, lo; };
__device__ __forceinline__ void dd_add(DD &a, double x) {
    const double s = a.hi + x;
    const double bb = s - a.hi;
    const double e = (a.hi - (s - bb)) + (x - bb);
    a.hi = s;
    a.lo += e;
}
__device__ __forceinline__ void dd_add_dd(DD &a, const DD &b) {
    dd_add(a, b.hi);
    a.lo += b.lo;
}

__global__ void __launch_bounds__(256)
k_reduce(const double *__restrict__ rec, const int64_t *__restrict__ pix_slot_off, int npix,
         double *__restrict__ A, double *__restrict__ b, int32_t *__restrict__ hits, double *__restrict__ part)
{
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= npix) return;
    DD s[10];
#pragma unroll
    for (int i = 0; i < 9; ++i) s[i] = DD{0.0, 0.0};
    int nh = 0;                          // hits: an integer count, summed exactly as one
    for (int64_t k = pix_slot_off[p]; k < pix_slot_off[p + 1]; ++k) {
        const double *r = rec + k * 10;
#pragma unroll
        for (int i = 0; i < 9; ++i) dd_add(s[i], r[i]);
        nh += static_cast<int>(r[9]);
    }
    s[9] = DD{static_cast<double>(nh), 0.0};
    if (part) {          // the unrounded pairs (hi, lo) of the ten sums
        double *o = part + static_cast<int64_t>(p) * 20;
#pragma unroll
        for (int i = 0; i < 10; ++i) { o[2 * i] = s[i].hi; o[2 * i + 1] = s[i].lo; }
        return;
    }
    if (A) {
#pragma unroll
        for (int i = 0; i < 6; ++i) A[static_cast<int64_t>(p) * 6 + i] = s[i].hi + s[i].lo;
    }
#pragma unroll
    for (int i = 0; i < 3; ++i) b[static_cast<int64_t>(p) * 3 + i] = s[6 + i].hi + s[6 + i].lo;
    if (hits) hits[p] = static_cast<int32_t>(s[9].hi + s[9].lo);
}

// Shards' pairs of pixels [0, np) added in rank order as double-doubles,
// rounded once: parts [nparts][np][20] -> A [np][6], b [np][3], hits [np].
__global__ void __launch_bounds__(256)
k_combine(const double *__restrict__ parts, int nparts, int64_t np, double *__restrict__ A, double *__restrict__ b,
          int32_t *__restrict__ hits)
{
    const int64_t p = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (p >= np) return;
    DD s[10];
#pragma unroll
    for (int i = 0; i < 10; ++i) s[i] = DD{0.0, 0.0};
    for (int r = 0; r < nparts; ++r) {
        const double *o = parts + (static_cast<int64_t>(r) * np + p) * 20;
#pragma unroll
        for (int i = 0; i < 10; ++i) dd_add_dd(s[i], DD{o[2 * i], o[2 * i + 1]});
    }
#pragma unroll
    for (int i = 0; i < 6; ++i) A[p * 6 + i] = s[i].hi + s[i].lo;
#pragma unroll
    for (int i = 0; i < 3; ++i) b[p * 3 + i] = s[6 + i].hi + s[6 + i].lo;
    hits[p] = static_cast<int32_t>(s[9].hi + s[9].lo);
}

// ---------------------------------------------------------------------------
// A7: FP64 3x3 Cholesky per pixel, validity by hits and Hadamard ratio.
// ---------------------------------------------------------------------------
// Pixels [0, npix) of A, b, hits (a whole map, or one range of it: the
// outputs are indexed like the inputs).
__global__ void __launch_bounds__(256)
k_solve(const double *__restrict__ A, const double *__restrict__ b, const int32_t *__restrict__ hits,
        int npix, double rcond_min, double *__restrict__ map, float4 *__restrict__ map32,
        double *__restrict__ rcond, uint8_t *__restrict__ valid)
{
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= npix) return;
    const double *a = A + static_cast<int64_t>(p) * 6;
    const double a00 = a[0], a01 = a[1], a02 = a[2], a11 = a[3], a12 = a[4], a22 = a[5];
    const double det = a00 * (a11 * a22 - a12 * a12) - a01 * (a01 * a22 - a12 * a02)
                     + a02 * (a01 * a12 - a11 * a02);
    const double dp = a00 * a11 * a22;
    const double had = dp > 0.0 ? det / dp : 0.0;
    const bool ok = hits[p] >= 3 && had >= rcond_min && a00 > 0.0 && a11 > 0.0 && a22 > 0.0;
    double x0 = 0.0, x1 = 0.0, x2 = 0.0;
    if (ok) {
        const double l00 = sqrt(a00);
        const double l10 = a01 / l00, l20 = a02 / l00;
        const double l11 = sqrt(a11 - l10 * l10);
        const double l21 = (a12 - l20 * l10) / l11;
        const double l22 = sqrt(a22 - l20 * l20 - l21 * l21);
        const double *bb = b + static_cast<int64_t>(p) * 3;
        const double y0 = bb[0] / l00;
        const double y1 = (bb[1] - l10 * y0) / l11;
        const double y2 = (bb[2] - l20 * y0 - l21 * y1) / l22;
        x2 = y2 / l22;
        x1 = (y1 - l21 * x2) / l11;
        x0 = (y0 - l10 * x1 - l20 * x2) / l00;
    }
    map[p] = x0;
    map[npix + p] = x1;
    map[2 * static_cast<int64_t>(npix) + p] = x2;
    if (map32) map32[p] = make_float4(static_cast<float>(x0), static_cast<float>(x1), static_cast<float>(x2), 0.f);
    if (rcond) rcond[p] = had;
    if (valid) valid[p] = ok ? 1 : 0;
}

cudaError_t setup_bin_kernel(Plan &)
{
    return cudaSuccess;
}

cudaError_t launch_bin(const Plan &p, const uint16_t *psi, const float *d, const float *ncorr,
                       const double *gain, const uint32_t *flags, const double *psd, double *A,
                       double *b, int32_t *hits, double *part, cudaStream_t st)
{
    if (p.nq == 0) return cudaSuccess;
    BinArgs a;
    a.psi = psi; a.d = d; a.x = ncorr; a.gain = gain; a.flags = flags; a.psd = psd; a.off = p.off;
    a.ld_t = p.ld_t; a.ld_pos = p.ld_pos; a.pair_start = p.pair_start; a.pair_len = p.pair_len; a.pair_slot = p.pair_slot;
    a.tile_q = p.bin_tile_q; a.tile_r0 = p.bin_tile_r0; a.trig = p.trig; a.ndet = p.ndet; a.rec = p.rec;
    a.adjoint = false; a.y64 = nullptr;
    if (p.nbin_tiles > 0) {
        KTIME(TOD_KT_BIN);
        k_bin<<<p.nbin_tiles, BIN_T, 0, st>>>(a);
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const int nb = (p.npix + 255) / 256;
    {
        KTIME(TOD_KT_REDUCE);
        k_reduce<<<nb, 256, 0, st>>>(p.rec, p.pix_slot_off, p.npix, A, b, hits, part);
    }
    return cudaGetLastError();
}

cudaError_t launch_combine(const double *parts, int nparts, int64_t np, double *A, double *b, int32_t *hits,
                           cudaStream_t st)
{
    if (np <= 0) return cudaSuccess;
    k_combine<<<static_cast<unsigned>((np + 255) / 256), 256, 0, st>>>(parts, nparts, np, A, b, hits);
    return cudaGetLastError();
}

cudaError_t launch_project_adjoint(const Plan &p, const uint16_t *psi, const void *y, bool fp64, const double *gain,
                                   double *out, cudaStream_t st)
{
    if (p.nq == 0) return cudaSuccess;
    BinArgs a;
    a.psi = psi; a.d = fp64 ? nullptr : static_cast<const float *>(y); a.x = nullptr; a.gain = gain;
    a.flags = nullptr; a.psd = nullptr; a.off = p.off;
    a.ld_t = p.ld_t; a.ld_pos = p.ld_pos; a.pair_start = p.pair_start; a.pair_len = p.pair_len; a.pair_slot = p.pair_slot;
    a.tile_q = p.bin_tile_q; a.tile_r0 = p.bin_tile_r0; a.trig = p.trig; a.ndet = p.ndet; a.rec = p.rec;
    a.adjoint = true; a.y64 = fp64 ? static_cast<const double *>(y) : nullptr;
    if (p.nbin_tiles > 0) {
        KTIME(TOD_KT_BIN);
        k_bin<<<p.nbin_tiles, BIN_T, 0, st>>>(a);
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const int nb = (p.npix + 255) / 256;
    {
        KTIME(TOD_KT_REDUCE);
        k_reduce<<<nb, 256, 0, st>>>(p.rec, p.pix_slot_off, p.npix, nullptr, out, nullptr, nullptr);
    }
    return cudaGetLastError();
}

cudaError_t launch_solve(const Plan &p, const double *A, const double *b, const int32_t *hits,
                         double rcond_min, double *map, float4 *map32, double *rcond,
                         uint8_t *valid, cudaStream_t st)
{
    KTIME(TOD_KT_SOLVE);
    return launch_solve_n(p.npix, A, b, hits, rcond_min, map, map32, rcond, valid, st);
}

cudaError_t launch_solve_n(int64_t npix, const double *A, const double *b, const int32_t *hits, double rcond_min,
                           double *map, float4 *map32, double *rcond, uint8_t *valid, cudaStream_t st)
{
    if (npix <= 0) return cudaSuccess;
    const int nb = static_cast<int>((npix + 255) / 256);
    k_solve<<<nb, 256, 0, st>>>(A, b, hits, static_cast<int>(npix), rcond_min, map, map32, rcond, valid);
    return cudaGetLastError();
}

}  // namespace tg
