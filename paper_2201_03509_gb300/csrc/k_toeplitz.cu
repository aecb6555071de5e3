// Preconditioner of the correlated-noise gap filling: block-Jacobi over the
// gaps of the Schur operator S = E^T C^T diag(gamma) C E.  Within a gap of
// L consecutive flagged samples S is (away from the detscan ends) the
// symmetric Toeplitz matrix T_ij = h(|i-j|) with
//   h(d) = (1/n) sum_{k>=1} gamma_k cos(pi k d / n),
//   gamma_k = sigma0^2 r/(1+r),  r = (f_k/f_knee)^-alpha,  f_k = k f_samp/(2n).
// One kernel evaluates h(d), d < TOEP_LMAX, per detector at a reference
// length (the preconditioner only has to be symmetric positive definite; a
// kernel shared by all detscans of a detector is close enough for 2-4 CG
// iterations); a second runs the Durbin recursion (Golub & Van Loan,
// Algorithm 4.7.1) in FP64 and stores, for every order L, the first column
// x = T_L^{-1} e_1.  The CG then applies T_L^{-1} by the Gohberg-Semencul
// formula T^{-1} = (L(x) L(x)^T - L(w) L(w)^T) / x_0, w = (0, x_{L-1}, ..,
// x_1), L(v) the lower-triangular Toeplitz matrix with first column v.
#include "common.cuh"
#include "internal.cuh"

namespace tg {

constexpr int HT = 256;     // threads per h block
constexpr int HD = 8;       // lags per h block

__global__ void __launch_bounds__(HT)
k_toep_h(const double *__restrict__ psd, int ndet, int nref, double fsamp, float *__restrict__ htab)
{
    const int det = blockIdx.y;
    const int d0 = blockIdx.x * HD;
    const double sig0 = psd[3 * det], fk = psd[3 * det + 1], al = psd[3 * det + 2];
    const float s2 = static_cast<float>(sig0 * sig0);
    const float fscale = static_cast<float>(fsamp / (2.0 * nref * fk));
    const float mal = static_cast<float>(-al);
    float acc[HD];
#pragma unroll
    for (int i = 0; i < HD; ++i) acc[i] = 0.f;
    const int two_n = 2 * nref;
    for (int k = 1 + threadIdx.x; k < nref; k += HT) {
        const float r = exp2f(mal * log2f(static_cast<float>(k) * fscale));
        const float g = s2 * r / (1.0f + r);
#pragma unroll
        for (int i = 0; i < HD; ++i) {
            const int d = d0 + i;
            const int ph = static_cast<int>((static_cast<int64_t>(k) * d) % two_n);  // k d mod 2n
            acc[i] = fmaf(g, cospif(static_cast<float>(ph) / static_cast<float>(nref)), acc[i]);
        }
    }
    __shared__ float red[HT / 32][HD];
#pragma unroll
    for (int i = 0; i < HD; ++i) {
        float v = acc[i];
        for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5][i] = v;
    }
    __syncthreads();
    if (threadIdx.x < HD) {
        float v = 0.f;
        for (int w = 0; w < HT / 32; ++w) v += red[w][threadIdx.x];
        htab[det * TOEP_LMAX + d0 + threadIdx.x] = v / static_cast<float>(nref);
    }
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
    dim3 g(TOEP_LMAX / HD, p.ndet);
    {
        KTIME(TOD_KT_TOEP_H);
        k_toep_h<<<g, HT, 0, st>>>(psd, p.ndet, p.toep_nref, p.fsamp, p.htab);
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
