// A10 noise PSD step: random-walk Metropolis on (ln f_knee, alpha) of every
// detector, from the DCT spectra of the n_corr draws (the paper lists the
// noise PSD step among the TOD steps of Sect. 5 and defers its sampler to
// the noise companion paper; the reading taken is the Gaussian density of
// n_corr under its 1/f prior, sigma0 fixed, flat prior on a box).
//
// With L = ln f_knee, a = alpha, N the detector's modes k >= 1 and
// f_{q,k} = k fsamp / (2 n_q) = k e^{c_q}:
//   ln L(L, a) = -1/2 [ e^{a L} / sigma0^2 S(a) + N ln sigma0^2
//                       + a (sum ln f - N L) ],
//   S(a) = sum_q e^{-a c_q} sum_{k>=1} xhat_{q,k}^2 k^{-a}.
// One evaluation is one pass over the spectra (k_psd_sums, one CTA per
// element tile of a detscan, partial sums per tile) and a fixed-order
// reduction per detector (k_psd_step), which also takes the Metropolis
// decision and draws the next proposal.  Deterministic.
#include "common.cuh"
#include "internal.cuh"

namespace tg {

namespace {

constexpr int PSD_T = 256;
// state per detector: ln f_knee, alpha, ln L, proposal (ln f_knee, alpha,
// in box), accepted count
constexpr int PS_LNFK = 0, PS_AL = 1, PS_LOGL = 2, PS_PLNFK = 3, PS_PAL = 4, PS_PVALID = 5, PS_ACC = 6;

__device__ __forceinline__ bool psd_in_box(double lnfk, double al) {
    return lnfk >= TOD_PSD_LNFK_MIN && lnfk <= TOD_PSD_LNFK_MAX && al >= TOD_PSD_ALPHA_MIN &&
           al <= TOD_PSD_ALPHA_MAX;
}

// The numbers of Metropolis step `step` of detector det: 53-bit uniforms
// from words 0 and 1 (Box-Muller pair of the proposal), word 2 (acceptance).
__device__ void psd_numbers(const tod_rng &rng, uint64_t it, int det, int step, double &z1, double &z2,
                            double &ua)
{
    const u64x4 w = philox4x64(static_cast<uint64_t>(step), static_cast<uint64_t>(det), TOD_PURPOSE_PSD, it,
                               rng.seed, rng.band);
    const double u1 = (static_cast<double>(w.x[0] >> 11) + 0.5) * 1.1102230246251565e-16;
    const double u2 = (static_cast<double>(w.x[1] >> 11) + 0.5) * 1.1102230246251565e-16;
    ua = (static_cast<double>(w.x[2] >> 11) + 0.5) * 1.1102230246251565e-16;
    const double r = sqrt(-2.0 * log(u1));
    z1 = r * cospi(2.0 * u2);
    z2 = r * sinpi(2.0 * u2);
}

__global__ void k_psd_begin(const double *__restrict__ psd_in, double *state, int ndet, double *psd_out,
                            int32_t *acc_out)
{
    const int det = blockIdx.x * blockDim.x + threadIdx.x;
    if (det >= ndet) return;
    const double fk = psd_in[3 * det + 1], al = psd_in[3 * det + 2];
    double *st = state + 8 * det;
    st[PS_LNFK] = log(fk);
    st[PS_AL] = al;
    st[PS_LOGL] = 0.0;
    st[PS_PLNFK] = st[PS_LNFK];        // the first evaluation is at the current state
    st[PS_PAL] = al;
    st[PS_PVALID] = 1.0;
    st[PS_ACC] = 0.0;
    psd_out[3 * det] = psd_in[3 * det];
    psd_out[3 * det + 1] = fk;
    psd_out[3 * det + 2] = al;
    if (acc_out) acc_out[det] = 0;
}

// partial S(alpha') of one element tile (one detscan's samples t0..t1)
__global__ void __launch_bounds__(PSD_T) k_psd_sums(const float *__restrict__ spec, const int64_t *__restrict__ off,
                                                    const int32_t *__restrict__ tile_q,
                                                    const int64_t *__restrict__ tile_t0,
                                                    const double *__restrict__ lnfs, const float2 *__restrict__ lnk,
                                                    const double *__restrict__ state, int ndet,
                                                    double *__restrict__ part)
{
    __shared__ double s_w[PSD_T / 32];
    const int q = tile_q[blockIdx.x];
    const int det = q % ndet;
    const double *st = state + 8 * det;
    if (st[PS_PVALID] == 0.0) {                       // proposal outside the box: rejected anyway
        if (threadIdx.x == 0) part[blockIdx.x] = 0.0;
        return;
    }
    const double al = st[PS_PAL];
    const float na = static_cast<float>(-al);
    const float na_lo = static_cast<float>(-al - static_cast<double>(na));
    const int64_t o = off[q], t0 = tile_t0[blockIdx.x];
    const int64_t t1 = (t0 + ELEM_TILE < off[q + 1]) ? t0 + ELEM_TILE : off[q + 1];
    // four modes per thread and round, every load in flight, four
    // accumulators merged in a fixed order
    constexpr int U = 4;
    Acc2 acc[U];
#pragma unroll
    for (int u = 0; u < U; ++u) acc[u] = Acc2{0.f, 0.f};
    for (int64_t tb = t0 + threadIdx.x; tb < t1; tb += U * PSD_T) {
        float x[U];
        float2 l[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int64_t t = tb + u * PSD_T;
            const int k = static_cast<int>(t - o);
            x[u] = 0.f;                                // the offset mode (k = 0) does not enter
            l[u] = make_float2(0.f, 0.f);
            if (t < t1 && k > 0) { x[u] = __ldg(spec + t); l[u] = __ldg(lnk + k); }   // ln k = l.x + l.y
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            // -alpha ln k as a double-float (p + e), then k^-alpha = e^p (1 + e)
            const float p = na * l[u].x;
            const float e = fmaf(na, l[u].x, -p) + fmaf(na, l[u].y, na_lo * l[u].x);
            const float w = expf(p) * (1.0f + e);
            acc_add_prod(acc[u], x[u] * x[u], w);
        }
    }
#pragma unroll
    for (int u = 1; u < U; ++u) {
        acc_add(acc[0], acc[u].s);
        acc[0].c = __fadd_rn(acc[0].c, acc[u].c);
    }
    // fixed-order reduction: warp trees, then the warps in order (thread 0, FP64)
#pragma unroll
    for (int ofs = 16; ofs; ofs >>= 1) {
        Acc2 o2;
        o2.s = __shfl_xor_sync(0xffffffffu, acc[0].s, ofs);
        o2.c = __shfl_xor_sync(0xffffffffu, acc[0].c, ofs);
        acc_add(acc[0], o2.s);
        acc[0].c = __fadd_rn(acc[0].c, o2.c);
    }
    if ((threadIdx.x & 31) == 0) s_w[threadIdx.x >> 5] = acc_value(acc[0]);
    __syncthreads();
    if (threadIdx.x == 0) {
        double sum = 0.0;
        for (int w = 0; w < PSD_T / 32; ++w) sum += s_w[w];
        part[blockIdx.x] = exp(-al * lnfs[q]) * sum;
    }
}

// One CTA per detector: S from the tiles' partials in a fixed order, ln L of
// the proposal, the Metropolis decision (step >= 0) or the first evaluation
// (step < 0), then the proposal of the next step and the outputs.
__global__ void __launch_bounds__(PSD_T) k_psd_step(int step, int nsteps, const double *__restrict__ part,
                                                    const int32_t *__restrict__ tile_q, int ntile, int ndet,
                                                    double *state, const double *__restrict__ psd_in,
                                                    const double *__restrict__ nmodes,
                                                    const double *__restrict__ sumlnf, tod_rng rng,
                                                    double step_lnfk, double step_al, double *psd_out,
                                                    int32_t *acc_out, double *loglike_out)
{
    __shared__ double s_r[PSD_T];
    const int det = blockIdx.x;
    double sum = 0.0;
    for (int i = threadIdx.x; i < ntile; i += PSD_T)
        if (tile_q[i] % ndet == det) sum += part[i];
    s_r[threadIdx.x] = sum;
    __syncthreads();
    for (int h = PSD_T / 2; h; h >>= 1) {
        if (threadIdx.x < h) s_r[threadIdx.x] += s_r[threadIdx.x + h];
        __syncthreads();
    }
    if (threadIdx.x != 0) return;
    double *st = state + 8 * det;
    const double S = s_r[0];
    const double s0 = psd_in[3 * det], ls2 = log(s0 * s0);
    const double N = nmodes[det];
    const double L = st[PS_PLNFK], a = st[PS_PAL];
    const double ll = -0.5 * (exp(a * L) / (s0 * s0) * S + N * ls2 + a * (sumlnf[det] - N * L));
    const uint64_t it = rng.gibbs_iter_dev ? *rng.gibbs_iter_dev : rng.gibbs_iter;
    if (step < 0) {
        st[PS_LOGL] = ll;
    } else {
        double z1, z2, ua;
        psd_numbers(rng, it, det, step, z1, z2, ua);
        if (st[PS_PVALID] != 0.0 && log(ua) < ll - st[PS_LOGL]) {
            st[PS_LNFK] = L;
            st[PS_AL] = a;
            st[PS_LOGL] = ll;
            st[PS_ACC] += 1.0;
        }
    }
    if (step + 1 < nsteps) {
        double z1, z2, ua;
        psd_numbers(rng, it, det, step + 1, z1, z2, ua);
        const double lp = st[PS_LNFK] + step_lnfk * z1, ap = st[PS_AL] + step_al * z2;
        st[PS_PLNFK] = lp;
        st[PS_PAL] = ap;
        st[PS_PVALID] = psd_in_box(lp, ap) ? 1.0 : 0.0;
    }
    psd_out[3 * det] = s0;
    psd_out[3 * det + 1] = exp(st[PS_LNFK]);
    psd_out[3 * det + 2] = st[PS_AL];
    if (acc_out) acc_out[det] = static_cast<int32_t>(st[PS_ACC]);
    if (loglike_out) loglike_out[det] = st[PS_LOGL];
}

}  // namespace

cudaError_t launch_noise_psd(const Plan &p, const float *spec, const double *psd_in, tod_rng rng, int nsteps,
                             double step_lnfk, double step_al, double *psd_out, int32_t *acc_out,
                             double *loglike_out, cudaStream_t st)
{
    {
        KTIME(TOD_KT_PSD_STEP);
        k_psd_begin<<<(p.ndet + 31) / 32, 32, 0, st>>>(psd_in, p.psd_state, p.ndet, psd_out, acc_out);
    }
    cudaError_t e = cudaGetLastError();
    for (int s = -1; s < nsteps && e == cudaSuccess; ++s) {
        if (p.ntile > 0)
            {
                KTIME(TOD_KT_PSD_SUMS);
                k_psd_sums<<<p.ntile, PSD_T, 0, st>>>(spec, p.off, p.tile_q, p.tile_t0, p.lnfs, p.lnk, p.psd_state,
                                                      p.ndet, p.psd_part);
            }
        {
            KTIME(TOD_KT_PSD_STEP);
            k_psd_step<<<p.ndet, PSD_T, 0, st>>>(s, nsteps, p.psd_part, p.tile_q, p.ntile, p.ndet, p.psd_state,
                                                 psd_in, p.psd_nmodes, p.psd_sumlnf, rng, step_lnfk, step_al,
                                                 psd_out, acc_out, loglike_out);
        }
        e = cudaGetLastError();
    }
    return e;
}

}  // namespace tg
