// Preconditioner of the correlated-noise gap filling: block-Jacobi over the
// gaps of the Schur operator S = E^T C^T diag(gamma) C E.  Within a gap of
// L consecutive flagged samples S is (away from the detscan ends) the
// symmetric Toeplitz matrix T_ij = h(|i-j|) with
//   h(d) = (1/n) sum_{k>=1} gamma_k cos(pi k d / n),
//   gamma_k = sigma0^2 r/(1+r),  r = (f_k/f_knee)^-alpha,  f_k = k f_samp/(2n).
// The kernel is evaluated per detector at a reference length H (cz_href, a
// power of two at least the longest detscan; the preconditioner only has to
// be symmetric positive definite, and a kernel shared by all detscans of a
// detector is close enough), at every lag d < H at once: h(d) is the real
// part of the length-2H DFT of the even sequence a_k = gamma_k (k < H),
// a_{2H-k} = gamma_k, a_H = 0, divided by 2H.  One FP32 Stockham FFT per
// detector gives it; a scan then stores, for the coarse correction, the
// prefix sums H(x) = sum_{d<x} h(d) and G(x) = sum_{d<x} d h(d) (FP64 sums
// kept as FP32 pairs), and the first TOEP_LMAX lags for the gap blocks.
// A second kernel runs the Durbin recursion (Golub & Van Loan, Algorithm
// 4.7.1) in FP64 and stores, for every order L, the first column
// x = T_L^{-1} e_1.  The CG then applies T_L^{-1} by the Gohberg-Semencul
// formula T^{-1} = (L(x) L(x)^T - L(w) L(w)^T) / x_0, w = (0, x_{L-1}, ..,
// x_1), L(v) the lower-triangular Toeplitz matrix with first column v.
#include "common.cuh"
#include "internal.cuh"

namespace tg {

constexpr int CZ_FT = 256;      // threads per CTA of the fill and FFT passes
constexpr int CZ_ST = 256;      // threads of the prefix-table kernels

// a_k for k < 2H (gamma at f_k = k f_samp / (2H); a_0 = a_H = 0)
__global__ void __launch_bounds__(CZ_FT)
k_cz_fill(const double *__restrict__ psd, int href, double fsamp, float2 *__restrict__ a)
{
    const int det = blockIdx.y;
    const int M = 2 * href;
    const int k = blockIdx.x * CZ_FT + threadIdx.x;
    if (k >= M) return;
    const double sig0 = psd[3 * det], fk = psd[3 * det + 1], al = psd[3 * det + 2];
    const float s2 = static_cast<float>(sig0 * sig0);
    const float fscale = static_cast<float>(fsamp / (2.0 * href * fk));
    const float mal = static_cast<float>(-al);
    const int kk = k <= href ? k : M - k;
    float g = 0.f;
    if (kk > 0 && kk < href) {
        const float r = exp2f(mal * log2f(static_cast<float>(kk) * fscale));
        g = s2 / (1.0f + 1.0f / r);           // sigma0^2 r / (1 + r), also for r = 0 or inf
    }
    a[static_cast<int64_t>(det) * M + k] = make_float2(g, 0.f);
}

// One radix-R Stockham pass (forward DFT) over every detector's length-M
// sequence, Ns points of each sub-transform already done (Ns, M powers of
// two).  Thread j < M/R reads x[j + r M/R], twiddles by exp(-2 pi i r k /
// (Ns R)), k = j mod Ns, and writes the R outputs to (j - k) R + k + r Ns.
template <int R>
__global__ void __launch_bounds__(CZ_FT)
k_cz_fft(const float2 *__restrict__ src, float2 *__restrict__ dst, int M, int Ns)
{
    const int det = blockIdx.y;
    const int MR = M / R;
    const int j = blockIdx.x * CZ_FT + threadIdx.x;
    if (j >= MR) return;
    const float2 *x = src + static_cast<int64_t>(det) * M;
    float2 *y = dst + static_cast<int64_t>(det) * M;
    const int k = j & (Ns - 1);
    float2 v[R];
#pragma unroll
    for (int r = 0; r < R; ++r) v[r] = x[j + r * MR];
    if (Ns > 1) {
#pragma unroll
        for (int r = 1; r < R; ++r) {
            float sn, cs;
            sincospif(-2.0f * static_cast<float>(r * k) / static_cast<float>(Ns * R), &sn, &cs);
            v[r] = make_float2(v[r].x * cs - v[r].y * sn, v[r].x * sn + v[r].y * cs);
        }
    }
    float2 o[R];
    if constexpr (R == 2) {
        o[0] = make_float2(v[0].x + v[1].x, v[0].y + v[1].y);
        o[1] = make_float2(v[0].x - v[1].x, v[0].y - v[1].y);
    } else {
        const float2 a0 = make_float2(v[0].x + v[2].x, v[0].y + v[2].y);
        const float2 a1 = make_float2(v[0].x - v[2].x, v[0].y - v[2].y);
        const float2 a2 = make_float2(v[1].x + v[3].x, v[1].y + v[3].y);
        const float2 a3 = make_float2(v[1].y - v[3].y, v[3].x - v[1].x);     // (v1 - v3) (-i)
        o[0] = make_float2(a0.x + a2.x, a0.y + a2.y);
        o[1] = make_float2(a1.x + a3.x, a1.y + a3.y);
        o[2] = make_float2(a0.x - a2.x, a0.y - a2.y);
        o[3] = make_float2(a1.x - a3.x, a1.y - a3.y);
    }
    const int base = (j - k) * R + k;
#pragma unroll
    for (int r = 0; r < R; ++r) y[base + r * Ns] = o[r];
}

__device__ __forceinline__ float4 cz_pack(double H, double G) {
    const float hh = __double2float_rn(H), gh = __double2float_rn(G);
    return make_float4(hh, __double2float_rn(H - static_cast<double>(hh)), gh,
                       __double2float_rn(G - static_cast<double>(gh)));
}

// h(d) = Re X_d / 2H for d < H; tab[x] = (H(x), G(x)) for x <= H (FP64 sums
// of the FP32 h values, as FP32 pairs); htab = the first TOEP_LMAX lags.
// The lags of a detector are cut into chunks of CZ_ST threads x cz_per(H)
// lags, one CTA each: k_cz_sums adds up every chunk, k_cz_tables scans
// within its chunk from the sum of the chunks before it.
__host__ __device__ __forceinline__ int cz_per(int href) { return href >= 64 * CZ_ST ? 64 : href / CZ_ST; }

__device__ __forceinline__ void cz_stretch(const float2 *__restrict__ x, int d0, int per, float inv, double &sh,
                                           double &sg) {
    sh = 0.0;
    sg = 0.0;
    for (int i = 0; i < per; ++i) {
        const double h = static_cast<double>(x[d0 + i].x * inv);
        sh += h;
        sg += static_cast<double>(d0 + i) * h;
    }
}

__global__ void __launch_bounds__(CZ_ST)
k_cz_sums(const float2 *__restrict__ X, int href, double2 *__restrict__ csum)
{
    const int det = blockIdx.y, nch = gridDim.x;
    const int per = cz_per(href);
    const float2 *x = X + static_cast<int64_t>(det) * 2 * href;
    const float inv = 1.0f / static_cast<float>(2 * href);      // exact: a power of two
    double sh, sg;
    cz_stretch(x, (blockIdx.x * CZ_ST + threadIdx.x) * per, per, inv, sh, sg);
    for (int o = 16; o; o >>= 1) {
        sh += __shfl_xor_sync(0xffffffffu, sh, o);
        sg += __shfl_xor_sync(0xffffffffu, sg, o);
    }
    __shared__ double wh[CZ_ST / 32], wg[CZ_ST / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) { wh[warp] = sh; wg[warp] = sg; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double th = 0.0, tg_ = 0.0;
        for (int w = 0; w < CZ_ST / 32; ++w) { th += wh[w]; tg_ += wg[w]; }
        csum[det * nch + blockIdx.x] = make_double2(th, tg_);
    }
}

__global__ void __launch_bounds__(CZ_ST)
k_cz_tables(const float2 *__restrict__ X, int href, const double2 *__restrict__ csum, float *__restrict__ htab,
            float4 *__restrict__ tab)
{
    const int det = blockIdx.y, ch = blockIdx.x, nch = gridDim.x;
    const int per = cz_per(href);
    const float2 *x = X + static_cast<int64_t>(det) * 2 * href;
    float4 *t = tab + static_cast<int64_t>(det) * (href + 1);
    const float inv = 1.0f / static_cast<float>(2 * href);
    const int d0 = (ch * CZ_ST + threadIdx.x) * per;
    double sh, sg;
    cz_stretch(x, d0, per, inv, sh, sg);
    // exclusive scan of (sh, sg) over the CTA, offset by the earlier chunks
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    double ih = sh, ig = sg;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const double uh = __shfl_up_sync(0xffffffffu, ih, o), ug = __shfl_up_sync(0xffffffffu, ig, o);
        if (lane >= o) { ih += uh; ig += ug; }
    }
    __shared__ double wh[CZ_ST / 32], wg[CZ_ST / 32];
    __shared__ double base[2];
    if (lane == 31) { wh[warp] = ih; wg[warp] = ig; }
    if (threadIdx.x == 0) {
        double bh = 0.0, bg = 0.0;
        for (int c = 0; c < ch; ++c) { const double2 v = csum[det * nch + c]; bh += v.x; bg += v.y; }
        base[0] = bh;
        base[1] = bg;
    }
    __syncthreads();
    if (warp == 0) {
        constexpr int NW = CZ_ST / 32;
        const double ownh = lane < NW ? wh[lane] : 0.0, owng = lane < NW ? wg[lane] : 0.0;
        double vh = ownh, vg = owng;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const double uh = __shfl_up_sync(0xffffffffu, vh, o), ug = __shfl_up_sync(0xffffffffu, vg, o);
            if (lane >= o) { vh += uh; vg += ug; }
        }
        if (lane < NW) {
            wh[lane] = vh - ownh;              // exclusive over the warps
            wg[lane] = vg - owng;
        }
    }
    __syncthreads();
    double Hc = base[0] + wh[warp] + (ih - sh), Gc = base[1] + wg[warp] + (ig - sg);
    for (int i = 0; i < per; ++i) {
        const int d = d0 + i;
        const float h32 = x[d].x * inv;
        if (d < TOEP_LMAX) htab[det * TOEP_LMAX + d] = h32;
        t[d] = cz_pack(Hc, Gc);
        Hc += static_cast<double>(h32);
        Gc += static_cast<double>(d) * static_cast<double>(h32);
    }
    if (ch == nch - 1 && threadIdx.x == CZ_ST - 1) t[href] = cz_pack(Hc, Gc);
}

// One CTA per detector (FP64 issue is the bound, so the dot products use
// all four SM sub-partitions).  xtab[det] holds, at offset L(L-1)/2, the L
// values of T_L^{-1} e_1 for L = 1..TOEP_LMAX; lvalid[det] is the largest
// order the recursion reached with a positive pivot.
constexpr int DT = 256;

__global__ void __launch_bounds__(DT)
k_toep_durbin(const float *__restrict__ htab, float *__restrict__ xtab, int32_t *__restrict__ lvalid)
{
    const int det = blockIdx.x;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    __shared__ double y[TOEP_LMAX];
    __shared__ double r[TOEP_LMAX];
    __shared__ double2 part[2][DT / 32];
    const float *h = htab + det * TOEP_LMAX;
    float *xt = xtab + static_cast<int64_t>(det) * (TOEP_LMAX * (TOEP_LMAX + 1) / 2);
    const double t0 = h[0];
    if (!(t0 > 0.0)) { if (tid == 0) lvalid[det] = 0; return; }
    for (int i = tid; i < TOEP_LMAX; i += DT) r[i] = (i + 1 < TOEP_LMAX ? h[i + 1] : 0.0f) / t0;
    __syncthreads();
    // order 1
    if (tid == 0) { xt[0] = static_cast<float>(1.0 / t0); y[0] = -r[0]; }
    __syncthreads();
    double beta = 1.0, alpha = -r[0];
    int valid = 1;
    for (int k = 1; k < TOEP_LMAX; ++k) {
        // with y^(k) (length k): D1 = r[0..k) . y, D2 = sum_j r[k-1-j] y[j]
        double d1 = 0.0, d2 = 0.0;
        for (int j = tid; j < k; j += DT) {
            const double yj = y[j];
            d1 += r[j] * yj;
            d2 += r[k - 1 - j] * yj;
        }
        for (int o = 16; o; o >>= 1) {
            d1 += __shfl_xor_sync(0xffffffffu, d1, o);
            d2 += __shfl_xor_sync(0xffffffffu, d2, o);
        }
        if (lane == 0) part[k & 1][warp] = make_double2(d1, d2);
        __syncthreads();
        double D1 = 0.0, D2 = 0.0;
        for (int w = 0; w < DT / 32; ++w) { D1 += part[k & 1][w].x; D2 += part[k & 1][w].y; }
        // x for order k+1: gamma = 1/(1 + D1), x = gamma (1, y) / t0
        const double gam = 1.0 / (1.0 + D1);
        if (!(gam > 0.0) || !isfinite(gam)) break;
        float *xk = xt + static_cast<int64_t>(k + 1) * k / 2;       // order L = k+1
        if (tid == 0) xk[0] = static_cast<float>(gam / t0);
        for (int i = tid; i < k; i += DT) xk[i + 1] = static_cast<float>(gam * y[i] / t0);
        valid = k + 1;
        if (k + 1 >= TOEP_LMAX) break;
        // Durbin step to y^(k+1)
        beta = (1.0 - alpha * alpha) * beta;
        if (!(beta > 0.0)) break;
        alpha = -(r[k] + D2) / beta;
        __syncthreads();      // every read of y^(k) is done
        // y[i] += alpha y[k-1-i] for i < k, pairs (i, k-1-i) by one thread
        for (int i = tid; i < (k + 1) / 2; i += DT) {
            const int jj = k - 1 - i;
            const double yi = y[i], yj = y[jj];
            y[i] = yi + alpha * yj;
            if (jj != i) y[jj] = yj + alpha * yi;
        }
        if (tid == 0) y[k] = alpha;
        __syncthreads();
    }
    if (tid == 0) lvalid[det] = valid;
}

cudaError_t launch_toeplitz_prep(const Plan &p, const double *psd, cudaStream_t st)
{
    const int M = 2 * p.cz_href;
    float2 *buf[2] = {p.czfft, p.czfft + static_cast<int64_t>(p.ndet) * M};
    {
        KTIME(TOD_KT_TOEP_KERNEL);
        k_cz_fill<<<dim3((M + CZ_FT - 1) / CZ_FT, p.ndet), CZ_FT, 0, st>>>(psd, p.cz_href, p.fsamp, buf[0]);
    }
    int cur = 0, Ns = 1, lg = 0;
    while ((1 << lg) < M) ++lg;
    if (lg & 1) {
        KTIME(TOD_KT_TOEP_KERNEL);
        k_cz_fft<2><<<dim3((M / 2 + CZ_FT - 1) / CZ_FT, p.ndet), CZ_FT, 0, st>>>(buf[cur], buf[cur ^ 1], M, Ns);
        cur ^= 1;
        Ns *= 2;
    }
    while (Ns < M) {
        KTIME(TOD_KT_TOEP_KERNEL);
        k_cz_fft<4><<<dim3((M / 4 + CZ_FT - 1) / CZ_FT, p.ndet), CZ_FT, 0, st>>>(buf[cur], buf[cur ^ 1], M, Ns);
        cur ^= 1;
        Ns *= 4;
    }
    // chunk sums into the other FFT buffer (free after the last pass)
    const int nch = p.cz_href / (CZ_ST * cz_per(p.cz_href));
    double2 *csum = reinterpret_cast<double2 *>(buf[cur ^ 1]);
    {
        KTIME(TOD_KT_TOEP_KERNEL);
        k_cz_sums<<<dim3(nch, p.ndet), CZ_ST, 0, st>>>(buf[cur], p.cz_href, csum);
    }
    {
        KTIME(TOD_KT_TOEP_KERNEL);
        k_cz_tables<<<dim3(nch, p.ndet), CZ_ST, 0, st>>>(buf[cur], p.cz_href, csum, p.htab, p.cztab);
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    {
        KTIME(TOD_KT_TOEP_DURBIN);
        k_toep_durbin<<<p.ndet, DT, 0, st>>>(p.htab, p.xtab, p.lvalid);
    }
    return cudaGetLastError();
}

}  // namespace tg
