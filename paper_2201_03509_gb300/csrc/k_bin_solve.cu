// A6 binning into per-pixel normal equations and A7 per-pixel 3x3 solve
// (paper Sect. 5 table rows "TOD binning" and "Map solution (Ax=b for each
// pixel)"; Sect. 2.4: coadded on the fly, synchronised once).
//
// Binning is a deterministic two-level segmented reduction.  The plan holds,
// for every detscan, its samples sorted by pixel (stable in time) and the
// runs of equal pixel ("pairs" of detscan and pixel); the runs of the whole
// band are ranked by (pixel, detscan).
//   k_bin:    one cluster per detscan stages the detscan's data, residual and
//             psi/flag words in distributed shared memory (coalesced HBM
//             reads), then each thread sums whole runs, gathering from DSMEM.
//             Products of FP32 values are formed exactly and summed as FP32
//             double-words (FP64 accuracy at FP32 issue rate); each run's
//             sums are scaled by the detscan's g^2/sigma0^2, g/sigma0^2 in
//             FP64 and written at the run's rank.
//   k_reduce: one thread per pixel adds its contiguous runs in FP64, in
//             ascending detscan order.
#include <algorithm>
#include <cooperative_groups.h>
#include "common.cuh"
#include "internal.cuh"

namespace cg = cooperative_groups;

namespace tg {

constexpr int BIN_T = 512;

struct BinArgs {
    const uint16_t *psi;
    const float *d, *x;
    const double *gain;
    const uint32_t *flags;
    const double *psd;
    const int64_t *off;
    const uint32_t *inv;          // sample -> position in the detscan's pixel-sorted order
    const int64_t *pair_off, *pair_start;
    const int32_t *pair_len, *pair_slot;
    const float2 *trig;
    const int32_t *work;
    int nq, ndet;
    int chunk_cap;     // samples staged per CTA
    double *rec;
    int32_t *status;
};

// sum of two double-words (two-sum on the heads, tails added)
__device__ __forceinline__ Acc2 acc_merge(const Acc2 &a, const Acc2 &b) {
    Acc2 r = a;
    acc_add(r, b.s);
    r.c = __fadd_rn(r.c, b.c);
    return r;
}
__device__ __forceinline__ Acc2 acc_shfl_down(const Acc2 &a, int o) {
    Acc2 r;
    r.s = __shfl_down_sync(0xffffffffu, a.s, o);
    r.c = __shfl_down_sync(0xffffffffu, a.c, o);
    return r;
}

__global__ void __launch_bounds__(BIN_T, 1) k_bin(BinArgs a)
{
    extern __shared__ __align__(16) unsigned char bin_raw[];
    __shared__ FastDiv s_fchunk;
    __shared__ int s_ra, s_rb;
    cg::cluster_group cl = cg::this_cluster();
    const int C = static_cast<int>(cl.num_blocks()), c = static_cast<int>(cl.block_rank());
    const int cid = blockIdx.x / C, ncl = gridDim.x / C;
    float *s_d = reinterpret_cast<float *>(bin_raw);
    float *s_x = s_d + a.chunk_cap;
    uint16_t *s_pf = reinterpret_cast<uint16_t *>(s_x + a.chunk_cap);   // psi | flag << 15
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    for (int w = cid; w < a.nq; w += ncl) {
        const int q = a.work[w];
        const int64_t o = a.off[q];
        const int n = static_cast<int>(a.off[q + 1] - o);
        const int chunk = (n + C - 1) / C;
        if (chunk > a.chunk_cap) {                   // plan guarantees this never happens
            if (c == 0 && threadIdx.x == 0) set_status(a.status, q, TOD_ERR_ARG);
            cl.sync();
            continue;
        }
        const int64_t pr0 = a.pair_off[q], pr1 = a.pair_off[q + 1];
        if (threadIdx.x == 0) {
            s_fchunk = make_fastdiv_dev(static_cast<uint32_t>(chunk));
            // runs whose first sorted position lies in this CTA's chunk
            int64_t lo = pr0, hi = pr1;
            while (lo < hi) { const int64_t mid = (lo + hi) >> 1; if (a.pair_start[mid] - o < static_cast<int64_t>(c) * chunk) lo = mid + 1; else hi = mid; }
            s_ra = static_cast<int>(lo - pr0);
            lo = pr0; hi = pr1;
            while (lo < hi) { const int64_t mid = (lo + hi) >> 1; if (a.pair_start[mid] - o < static_cast<int64_t>(c + 1) * chunk) lo = mid + 1; else hi = mid; }
            s_rb = static_cast<int>(lo - pr0);
        }
        __syncthreads();
        const FastDiv fch = s_fchunk;
        // stage: coalesced reads in time order, stores to the sorted position
        const int t0 = c * chunk, t1 = min(n, t0 + chunk);
        for (int t = t0 + threadIdx.x; t < t1; t += BIN_T) {
            const int64_t tg = o + t;
            const int sp = static_cast<int>(a.inv[tg]);
            const int ow = fdiv(sp, fch), ls = sp - ow * chunk;
            const uint32_t fb = (a.flags[tg >> 5] >> (tg & 31)) & 1u;
            *cl.map_shared_rank(s_d + ls, ow) = a.d[tg];
            *cl.map_shared_rank(s_x + ls, ow) = a.x[tg];
            *cl.map_shared_rank(s_pf + ls, ow) = static_cast<uint16_t>((a.psi[tg] & 0x0FFF) | (fb << 15));
        }
        cl.sync();
        const int det = q % a.ndet;
        const double sig0 = a.psd[3 * det];
        const double gq = a.gain[q];
        const double wA = gq * gq / (sig0 * sig0), wb = gq / (sig0 * sig0);
        for (int r = s_ra + warp; r < s_rb; r += BIN_T / 32) {
            const int64_t pr = pr0 + r;
            const int st = static_cast<int>(a.pair_start[pr] - o);
            const int len = a.pair_len[pr];
            Acc2 acc[11];
#pragma unroll
            for (int i = 0; i < 11; ++i) acc[i] = Acc2{0.f, 0.f};
            int hits = 0;
            for (int i = lane; i < len; i += 32) {
                const int sp = st + i;
                const int ow = fdiv(sp, fch), ls = sp - ow * chunk;
                uint16_t pf;
                float dv, xv;
                if (ow == c) { pf = s_pf[ls]; dv = s_d[ls]; xv = s_x[ls]; }
                else {
                    pf = *cl.map_shared_rank(s_pf + ls, ow);
                    dv = *cl.map_shared_rank(s_d + ls, ow);
                    xv = *cl.map_shared_rank(s_x + ls, ow);
                }
                if (pf >> 15) continue;
                const float2 cs = __ldg(a.trig + (pf & 0x0FFF));
                ++hits;
                acc_add(acc[0], cs.x);
                acc_add(acc[1], cs.y);
                acc_add_prod(acc[2], cs.x, cs.x);
                acc_add_prod(acc[3], cs.x, cs.y);
                acc_add_prod(acc[4], cs.y, cs.y);
                acc_add(acc[5], dv);
                acc_add_prod(acc[6], cs.x, dv);
                acc_add_prod(acc[7], cs.y, dv);
                acc_add(acc[8], xv);
                acc_add_prod(acc[9], cs.x, xv);
                acc_add_prod(acc[10], cs.y, xv);
            }
            // warp tree in a fixed order (deterministic)
#pragma unroll
            for (int ofs = 16; ofs; ofs >>= 1) {
#pragma unroll
                for (int i = 0; i < 11; ++i) acc[i] = acc_merge(acc[i], acc_shfl_down(acc[i], ofs));
                hits += __shfl_down_sync(0xffffffffu, hits, ofs);
            }
            if (lane == 0) {
                double *rr = a.rec + static_cast<int64_t>(a.pair_slot[pr]) * 10;
                rr[0] = wA * hits;
                rr[1] = wA * acc_value(acc[0]);
                rr[2] = wA * acc_value(acc[1]);
                rr[3] = wA * acc_value(acc[2]);
                rr[4] = wA * acc_value(acc[3]);
                rr[5] = wA * acc_value(acc[4]);
                rr[6] = wb * (acc_value(acc[5]) - acc_value(acc[8]));
                rr[7] = wb * (acc_value(acc[6]) - acc_value(acc[9]));
                rr[8] = wb * (acc_value(acc[7]) - acc_value(acc[10]));
                rr[9] = static_cast<double>(hits);
            }
        }
        cl.sync();      // staging buffers are reused by the next detscan
    }
}

__global__ void __launch_bounds__(256)
k_reduce(const double *__restrict__ rec, const int64_t *__restrict__ pix_slot_off, int npix,
         double *__restrict__ A, double *__restrict__ b, int32_t *__restrict__ hits)
{
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= npix) return;
    double s[10];
#pragma unroll
    for (int i = 0; i < 10; ++i) s[i] = 0.0;
    for (int64_t k = pix_slot_off[p]; k < pix_slot_off[p + 1]; ++k) {
        const double *r = rec + k * 10;
#pragma unroll
        for (int i = 0; i < 10; ++i) s[i] += r[i];
    }
#pragma unroll
    for (int i = 0; i < 6; ++i) A[static_cast<int64_t>(p) * 6 + i] = s[i];
#pragma unroll
    for (int i = 0; i < 3; ++i) b[static_cast<int64_t>(p) * 3 + i] = s[6 + i];
    hits[p] = static_cast<int32_t>(s[9]);
}

// ---------------------------------------------------------------------------
// A7: FP64 3x3 Cholesky per pixel, validity by hits and Hadamard ratio.
// ---------------------------------------------------------------------------
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

// ---------------------------------------------------------------------------
// Cluster size and staging capacity are fixed at plan creation (the longest
// detscan over the cluster, <= 200 KB per CTA), so tod_bin only launches.
cudaError_t setup_bin_kernel(Plan &p)
{
    int64_t nmax = 0;
    for (int q = 0; q < p.nq; ++q) nmax = std::max<int64_t>(nmax, p.h_off[q + 1] - p.h_off[q]);
    int C = 1;
    while (C < 16 && (nmax + C - 1) / C * 10 > 200 * 1024) C *= 2;
    p.bin_C = C;
    p.bin_cap = static_cast<int>((nmax + C - 1) / C);
    p.smem_bin = static_cast<size_t>(p.bin_cap) * 10 + 16;
    cudaError_t e = cudaFuncSetAttribute(k_bin, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         static_cast<int>(p.smem_bin));
    if (e != cudaSuccess) return e;
    if (C > 8) {
        e = cudaFuncSetAttribute(k_bin, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
        if (e != cudaSuccess) return e;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(static_cast<unsigned>(C * 64));
    cfg.blockDim = dim3(BIN_T);
    cfg.dynamicSmemBytes = p.smem_bin;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = C; attr[0].val.clusterDim.y = 1; attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr; cfg.numAttrs = 1;
    int ncl = 0;
    e = cudaOccupancyMaxActiveClusters(&ncl, k_bin, &cfg);
    if (e != cudaSuccess) return e;
    p.bin_nclusters = std::max(1, std::min(ncl, p.nq));
    return cudaSuccess;
}

cudaError_t launch_bin(const Plan &p, const uint16_t *psi, const float *d, const float *ncorr,
                       const double *gain, const uint32_t *flags, const double *psd, double *A,
                       double *b, int32_t *hits, cudaStream_t st)
{
    if (p.nq == 0) return cudaSuccess;
    BinArgs a;
    a.psi = psi; a.d = d; a.x = ncorr; a.gain = gain; a.flags = flags; a.psd = psd; a.off = p.off;
    a.inv = p.lp; a.pair_off = p.pair_off; a.pair_start = p.pair_start; a.pair_len = p.pair_len;
    a.pair_slot = p.pair_slot; a.trig = p.trig; a.work = p.work; a.nq = p.nq; a.ndet = p.ndet;
    a.chunk_cap = p.bin_cap; a.rec = p.rec; a.status = p.status;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(static_cast<unsigned>(p.bin_nclusters * p.bin_C));
    cfg.blockDim = dim3(BIN_T);
    cfg.dynamicSmemBytes = p.smem_bin;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = p.bin_C; attr[0].val.clusterDim.y = 1; attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr; cfg.numAttrs = 1;
    void *argv[1] = {&a};
    cudaError_t e = cudaLaunchKernelExC(&cfg, reinterpret_cast<const void *>(k_bin), argv);
    if (e != cudaSuccess) return e;
    const int nb = (p.npix + 255) / 256;
    k_reduce<<<nb, 256, 0, st>>>(p.rec, p.pix_slot_off, p.npix, A, b, hits);
    return cudaGetLastError();
}

cudaError_t launch_solve(const Plan &p, const double *A, const double *b, const int32_t *hits,
                         double rcond_min, double *map, float4 *map32, double *rcond,
                         uint8_t *valid, cudaStream_t st)
{
    const int nb = (p.npix + 255) / 256;
    k_solve<<<nb, 256, 0, st>>>(A, b, hits, p.npix, rcond_min, map, map32, rcond, valid);
    return cudaGetLastError();
}

}  // namespace tg
