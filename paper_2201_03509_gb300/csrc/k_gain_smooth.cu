// A12 joint gain draw of all scans of one detector under a smooth prior
// (the per-detscan gain conditional of Eq. `gibbsstart` as likelihood; the
// paper defers the gain model to its calibration companion paper, so the
// prior is a reading): precision diagonal in the orthonormal DCT-II basis
// of the scan index, lambda_0 = 0 (mean gain free), lambda_k = 1 /
// (sigma_g^2 k^alpha_g).  With a_s = 1/sigma_s^2, b_s = mu_s/sigma_s^2:
//   A g = b + a^(1/2) w1 + C^T (lambda^(1/2) w2),  A = diag(a) + C^T diag(lambda) C.
// One CTA per detector solves it by preconditioned CG for the fluctuation
// x = g - g_ref about the weighted mean g_ref = sum b / sum a (A g_ref =
// a g_ref: the prior does not see a constant), scaled by the mean of a, in
// the DCT domain, where the preconditioner diag(1 / (1 + lambda/abar)) is
// (C A C^T)^-1 exactly when every scan has the same a.  Transforms are direct sums over a shared
// quarter-wave cosine table (a detector has at most a few thousand scans),
// FP32 products in double-word sums, dot products in FP64, every sum in a
// fixed order: deterministic.  The table is padded by one word every 32
// (entry m at m + m/32) so that the inverse transform's even lane strides
// do not all fall in one shared-memory bank.
#include "common.cuh"
#include "internal.cuh"

namespace tg {

namespace {

constexpr int GS_T = 1024;
constexpr int GS_CHUNK = 16;          // terms summed in FP32 before entering the double-word sum

__host__ __device__ __forceinline__ int cpad(int m) { return m + (m >> 5); }

// FP64 block sum of two per-thread values, fixed order (warp trees, then a
// tree over the warps in warp 0); every thread gets both sums.  s_red holds
// GS_T / 32 + 1 entries.  (GB300 issues FP64 at a low rate: the sum over the
// warps is done once, not by every thread.)
__device__ double2 block_sum2(double u, double v, double2 *s_red)
{
#pragma unroll
    for (int o = 16; o; o >>= 1) {
        u += __shfl_xor_sync(0xffffffffu, u, o);
        v += __shfl_xor_sync(0xffffffffu, v, o);
    }
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    __syncthreads();                            // s_red free from the previous use
    if (lane == 0) s_red[w] = make_double2(u, v);
    __syncthreads();
    if (w == 0) {
        static_assert(GS_T / 32 == 32, "one partial per lane of warp 0");
        double su = s_red[lane].x, sv = s_red[lane].y;
#pragma unroll
        for (int o = 16; o; o >>= 1) {
            su += __shfl_xor_sync(0xffffffffu, su, o);
            sv += __shfl_xor_sync(0xffffffffu, sv, o);
        }
        if (lane == 0) s_red[GS_T / 32] = make_double2(su, sv);
    }
    __syncthreads();
    return s_red[GS_T / 32];
}

// sum_j v_j cos(pi m_j / (2S)) over j = 0..S-1 with m_j = (m0 + j step) mod 4S:
// four interleaved chains (j = 4i + c), each summing GS_CHUNK terms in FP32
// before its double-word sum; the chains are merged in a fixed order
__device__ __forceinline__ double cos_sum(const float *v, int m0, int step, const float *cosT, int S)
{
    const int S4 = 4 * S;
    const int step4 = static_cast<int>((4ll * step) % S4);
    int m[4];
    Acc2 acc[4];
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        m[c] = static_cast<int>((static_cast<long long>(m0) + static_cast<long long>(c) * step) % S4);
        acc[c] = Acc2{0.f, 0.f};
    }
    const int S4q = S & ~3;
    for (int j0 = 0; j0 < S4q; j0 += 4 * GS_CHUNK) {
        const int j1 = min(j0 + 4 * GS_CHUNK, S4q);
        float part[4] = {0.f, 0.f, 0.f, 0.f};
        for (int j = j0; j < j1; j += 4) {
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                part[c] = fmaf(v[j + c], cosT[cpad(m[c])], part[c]);
                m[c] += step4;
                if (m[c] >= S4) m[c] -= S4;
            }
        }
#pragma unroll
        for (int c = 0; c < 4; ++c) acc_add(acc[c], part[c]);
    }
#pragma unroll
    for (int c = 0; c < 3; ++c)                                   // the last S mod 4 terms
        if (S4q + c < S) acc_add(acc[c], v[S4q + c] * cosT[cpad(m[c])]);
#pragma unroll
    for (int c = 1; c < 4; ++c) {
        acc_add(acc[0], acc[c].s);
        acc[0].c = __fadd_rn(acc[0].c, acc[c].c);
    }
    return acc_value(acc[0]);
}

// y_k = c_k sum_q x_q cos(pi k (2q+1) / (2S)), c_0 = sqrt(1/S), c_k = sqrt(2/S)
// (c = (c_0, c_k), computed once per CTA)
__device__ void dct_fwd(const float *x, float *y, const float *cosT, int S, double2 c)
{
    for (int k = threadIdx.x; k < S; k += GS_T)
        y[k] = static_cast<float>(cos_sum(x, k, 2 * k, cosT, S) * (k ? c.y : c.x));
}

// x_q = sum_k c_k y_k cos(pi k (2q+1) / (2S)); ys holds c_k y_k
__device__ void dct_inv(const float *ys, float *x, const float *cosT, int S)
{
    for (int q = threadIdx.x; q < S; q += GS_T) x[q] = static_cast<float>(cos_sum(ys, 0, 2 * q + 1, cosT, S));
}

__global__ void __launch_bounds__(GS_T) k_gain_smooth(GainSmoothArgs g)
{
    extern __shared__ float sm[];
    __shared__ double2 s_red[GS_T / 32 + 1];
    __shared__ double2 s_c;
    const int S = g.nscan, det = blockIdx.x;
    float *cosT = sm;                  // [cpad(4S)] cos(pi m / (2S)) at cpad(m)
    float *ah = cosT + cpad(4 * S);    // a / abar
    float *lh = ah + S;                // lambda / abar
    float *ph = lh + S;                // 1 / (1 + lambda / abar)
    float *x = ph + S, *r = x + S, *z = r + S, *p = z + S, *q = p + S, *t = q + S;
    const int tid = threadIdx.x;

    // the detector's prior: sigma_g > 0 (also after rounding to FP32, where
    // the prior precision is held) and alpha_g finite, else every detscan of
    // the detector is marked TOD_ERR_ARG and its gain set to 0
    {
        const double sgp = g.prior[2 * det], alp = g.prior[2 * det + 1];
        const float sgf = static_cast<float>(sgp);
        if (!(sgp > 0.0) || !isfinite(sgp) || !isfinite(alp) || !(sgf * sgf > 0.0f) || !isfinite(sgf * sgf)) {
            for (int s = tid; s < S; s += GS_T) {
                set_status(g.status, s * g.ndet + det, TOD_ERR_ARG);
                g.gain_out[static_cast<int64_t>(s) * g.ndet + det] = 0.0;
            }
            if (tid == 0 && g.iters_out) g.iters_out[det] = 0;
            return;
        }
    }

    // quarter wave in FP64 (m <= S), the rest by symmetry; the normalisation once
    for (int m = tid; m <= S; m += GS_T)
        cosT[cpad(m)] = static_cast<float>(cospi(static_cast<double>(m) / (2.0 * S)));
    if (tid == 0) s_c = make_double2(sqrt(1.0 / S), sqrt(2.0 / S));
    __syncthreads();
    for (int m = S + 1 + tid; m < 4 * S; m += GS_T) {
        float v;
        if (m <= 2 * S) v = -cosT[cpad(2 * S - m)];
        else if (m <= 3 * S) v = -cosT[cpad(m - 2 * S)];
        else v = cosT[cpad(4 * S - m)];
        cosT[cpad(m)] = v;
    }
    const double2 cn = s_c;
    // sums of a and b (FP64), bad inputs flagged
    double sa = 0.0, sb = 0.0;
    for (int s = tid; s < S; s += GS_T) {
        const double sg = g.sigma[static_cast<int64_t>(s) * g.ndet + det];
        const double mu = g.mu[static_cast<int64_t>(s) * g.ndet + det];
        if (!(sg > 0.0) || !isfinite(sg) || !isfinite(mu)) {
            set_status(g.status, s * g.ndet + det, TOD_ERR_ARG);
            continue;
        }
        const double a = 1.0 / (sg * sg);
        sa += a;
        sb += a * mu;
    }
    const double2 ssum = block_sum2(sa, sb, s_red);
    if (!(ssum.x > 0.0)) return;                                  // uniform: nothing to solve
    const double gref = ssum.y / ssum.x, abar = ssum.x / S;
    const float sgpf = static_cast<float>(g.prior[2 * det]), alpf = static_cast<float>(g.prior[2 * det + 1]);
    const float sg2f = sgpf * sgpf, abarf = static_cast<float>(abar);
    const uint64_t it = g.rng.gibbs_iter_dev ? *g.rng.gibbs_iter_dev : g.rng.gibbs_iter;
    // The solve runs in the DCT domain (hats: C v): there the prior and the
    // preconditioner are diagonal, C A C^T v^ = C (a o C^T v^) + lambda o v^,
    // so an iteration takes two transforms.  Scaled by 1/abar throughout.
    // Right-hand side: C ((b - a g_ref + a^(1/2) w1) / abar) + lambda^(1/2) w2 / abar.
    for (int s = tid; s < S; s += GS_T) {
        const double sg = g.sigma[static_cast<int64_t>(s) * g.ndet + det];
        const double mu = g.mu[static_cast<int64_t>(s) * g.ndet + det];
        const double a = (sg > 0.0 && isfinite(sg) && isfinite(mu)) ? 1.0 / (sg * sg) : 0.0;
        double rhs = a * (mu - gref);
        // lambda_k / abar in FP32 (it is stored in FP32)
        const float lam = s ? exp2f(-alpf * log2f(static_cast<float>(s))) / sg2f : 0.0f;
        const float lamh = lam / abarf;
        ah[s] = static_cast<float>(a / abar);
        lh[s] = lamh;
        ph[s] = 1.0f / (1.0f + lamh);
        t[s] = 0.0f;
        if (g.mode == TOD_MODE_DRAW) {
            const u64x4 w = philox4x64(static_cast<uint64_t>(s), static_cast<uint64_t>(det),
                                       TOD_PURPOSE_GAIN_SMOOTH, it, g.rng.seed, g.rng.band);
            double u[4];
#pragma unroll
            for (int j = 0; j < 4; ++j) u[j] = (static_cast<double>(w.x[j] >> 11) + 0.5) * 1.1102230246251565e-16;
            const double w1 = sqrt(-2.0 * log(u[0])) * cospi(2.0 * u[1]);
            const double w2 = sqrt(-2.0 * log(u[2])) * cospi(2.0 * u[3]);
            rhs += sqrt(a) * w1;
            t[s] = sqrtf(lam) / abarf * static_cast<float>(w2);      // prior term, mode s of the DCT
        }
        z[s] = static_cast<float>(rhs / abar);
        x[s] = 0.0f;
    }
    __syncthreads();
    dct_fwd(z, r, cosT, S, cn);
    __syncthreads();
    // r^ (with the prior term), z^ = M^-1 r^ = ph o r^, p^ = z^
    double rz = 0.0, rr = 0.0;
    for (int k = tid; k < S; k += GS_T) {
        const float rk = r[k] + t[k];
        const float zk = ph[k] * rk;
        r[k] = rk;
        z[k] = zk;
        p[k] = zk;
        rz += static_cast<double>(rk) * zk;
        rr += static_cast<double>(rk) * rk;
    }
    double2 d2 = block_sum2(rz, rr, s_red);
    rz = d2.x;
    rr = d2.y;
    const double tol2 = static_cast<double>(g.tol) * g.tol * rr;
    int iter = 0;
    while (rr > tol2 && iter < g.maxiter) {
        // q^ = C (ah o C^T p^) + lh o p^   (z is free here: it is rebuilt below)
        for (int k = tid; k < S; k += GS_T)
            t[k] = static_cast<float>(static_cast<double>(p[k]) * (k ? cn.y : cn.x));
        __syncthreads();
        dct_inv(t, z, cosT, S);
        __syncthreads();
        for (int s = tid; s < S; s += GS_T) z[s] *= ah[s];
        __syncthreads();
        dct_fwd(z, q, cosT, S, cn);
        __syncthreads();
        double pq = 0.0;
        for (int k = tid; k < S; k += GS_T) {
            q[k] = fmaf(lh[k], p[k], q[k]);
            pq += static_cast<double>(p[k]) * q[k];
        }
        pq = block_sum2(pq, 0.0, s_red).x;
        if (!(pq > 0.0)) break;
        const double al = rz / pq;
        double rz1 = 0.0, rr1 = 0.0;
        for (int k = tid; k < S; k += GS_T) {
            x[k] = static_cast<float>(x[k] + al * p[k]);
            const float rk = static_cast<float>(r[k] - al * q[k]);
            const float zk = ph[k] * rk;
            r[k] = rk;
            z[k] = zk;
            rz1 += static_cast<double>(rk) * zk;
            rr1 += static_cast<double>(rk) * rk;
        }
        d2 = block_sum2(rz1, rr1, s_red);
        const double be = d2.x / rz;
        rz = d2.x;
        rr = d2.y;
        for (int k = tid; k < S; k += GS_T) p[k] = static_cast<float>(z[k] + be * p[k]);
        __syncthreads();
        ++iter;
    }
    // back to the scan domain: x = C^T x^
    for (int k = tid; k < S; k += GS_T) t[k] = static_cast<float>(static_cast<double>(x[k]) * (k ? cn.y : cn.x));
    __syncthreads();
    dct_inv(t, z, cosT, S);
    __syncthreads();
    for (int s = tid; s < S; s += GS_T)
        g.gain_out[static_cast<int64_t>(s) * g.ndet + det] = gref + static_cast<double>(z[s]);
    if (tid == 0) {
        if (g.iters_out) g.iters_out[det] = iter;
        if (rr > tol2) set_status(g.status, det, TOD_ERR_NOT_CONVERGED);
    }
}

}  // namespace

size_t gain_smooth_smem(int nscan)
{
    return sizeof(float) * (static_cast<size_t>(cpad(4 * nscan)) + 9u * static_cast<size_t>(nscan));
}

// once per plan (outside any stream capture): room for the largest scan count
cudaError_t setup_gain_smooth_kernel()
{
    return cudaFuncSetAttribute(k_gain_smooth, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                static_cast<int>(gain_smooth_smem(TOD_GAIN_SMOOTH_MAX_SCANS)));
}

cudaError_t launch_gain_smooth(const GainSmoothArgs &a, cudaStream_t st)
{
    k_gain_smooth<<<a.ndet, GS_T, gain_smooth_smem(a.nscan), st>>>(a);
    return cudaGetLastError();
}

}  // namespace tg
