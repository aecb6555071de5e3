// tod_sample_ncorr_static: the correlated-noise draw of tod_sample_ncorr with
// its working memory (the transforms' complex intermediate, the flag-word
// prefix and the CG vectors) in a fixed device array compiled into the
// library, so the call itself allocates nothing.
//
// The array is one file-scope __device__ array per device of
// TOD_NCORR_STATIC_SCRATCH_BYTES.  Host code cannot use the array's name as
// a device address: tod_ncorr_static_setup looks the address up with
// cudaGetSymbolAddress (with the plan's device current) and caches it per
// device; the draw refuses to run on a device where that has not happened.
// The draw takes the band in waves of consecutive detscans whose working
// memory fits the array; each wave writes everything it reads, so no part
// of the array has to start at zero.  All calls on one device share the
// array: calls that may run at the same time on the device race on it.
#include <algorithm>
#include <mutex>
#include "internal.cuh"

namespace tg {

constexpr size_t kStaticF4 = TOD_NCORR_STATIC_SCRATCH_BYTES / sizeof(float4);

static __device__ __align__(256) float4 g_ncorr_static_scratch[kStaticF4];

constexpr int kMaxDevices = 64;
static std::mutex g_static_mu;
static float4 *g_static_addr[kMaxDevices] = {};

// Working memory of a wave of S samples: the intermediate (S/2 complex
// values), the flag prefix ((S/32 + 3) words of 8 bytes) and five CG vectors
// of S/4 floats, each area 256-byte aligned.
struct WaveCarve {
    int64_t y_bytes, w_bytes, v_bytes;
};
static WaveCarve carve(int64_t S) {
    auto al = [](int64_t b) { return (b + 255) & ~int64_t(255); };
    WaveCarve c;
    c.y_bytes = al(4 * S);
    c.w_bytes = al(8 * (S / 32 + 3));
    c.v_bytes = al(4 * 5 * std::max<int64_t>(1, S / 4));
    return c;
}
static int64_t wave_bytes(int64_t S) {
    const WaveCarve c = carve(S);
    return c.y_bytes + c.w_bytes + c.v_bytes;
}
// largest wave (samples) that fits the array
static int64_t max_wave_samples() {
    int64_t lo = 0, hi = TOD_NCORR_STATIC_SCRATCH_BYTES;
    while (lo < hi) {
        const int64_t mid = (lo + hi + 1) / 2;
        if (wave_bytes(mid) <= static_cast<int64_t>(TOD_NCORR_STATIC_SCRATCH_BYTES)) lo = mid; else hi = mid - 1;
    }
    return lo;
}

}  // namespace tg

using namespace tg;

extern "C" {

tod_status tod_ncorr_static_setup(tod_plan *pl, int64_t *max_wave_samples_out)
{
    if (!pl) return TOD_ERR_ARG;
    Plan *p = reinterpret_cast<Plan *>(pl);
    if (p->device < 0 || p->device >= kMaxDevices) return TOD_ERR_ARG;
    int prev = 0;
    if (cudaGetDevice(&prev) != cudaSuccess) return TOD_ERR_CUDA;
    if (prev != p->device && cudaSetDevice(p->device) != cudaSuccess) return TOD_ERR_CUDA;
    void *ptr = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&ptr, g_ncorr_static_scratch);
    if (prev != p->device) cudaSetDevice(prev);
    if (e != cudaSuccess) return TOD_ERR_CUDA;
    {
        std::lock_guard<std::mutex> lock(g_static_mu);
        g_static_addr[p->device] = static_cast<float4 *>(ptr);      // refreshed on every call
    }
    const int64_t S = max_wave_samples();
    if (max_wave_samples_out) max_wave_samples_out[0] = S;
    int64_t longest = 0;
    for (int q = 0; q < p->nq; ++q) longest = std::max<int64_t>(longest, p->h_off[q + 1] - p->h_off[q]);
    return longest > S ? TOD_ERR_SCRATCH : TOD_OK;
}

tod_status tod_sample_ncorr_static(tod_plan *pl, const float *d, const float *s, const double *gain,
                                   const uint32_t *flags, const double *psd, tod_rng rng, int32_t mode,
                                   double cg_tol, int32_t cg_maxiter, float *ncorr_out,
                                   int32_t *cg_iters_out, cudaStream_t stream)
{
    if (!pl || !d || !s || !gain || !flags || !psd || !ncorr_out) return TOD_ERR_ARG;
    if (mode != TOD_MODE_DRAW && mode != TOD_MODE_MEAN) return TOD_ERR_ARG;
    Plan *p = reinterpret_cast<Plan *>(pl);
    if (p->device < 0 || p->device >= kMaxDevices) return TOD_ERR_ARG;
    float4 *base = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_static_mu);
        base = g_static_addr[p->device];
    }
    if (!base) return TOD_ERR_ARG;              // tod_ncorr_static_setup has not run on this device
    const int64_t S = max_wave_samples();
    for (int q = 0; q < p->nq; ++q)
        if (p->h_off[q + 1] - p->h_off[q] > S) return TOD_ERR_SCRATCH;
    int prev = 0;
    if (cudaGetDevice(&prev) != cudaSuccess) return TOD_ERR_CUDA;
    if (prev != p->device && cudaSetDevice(p->device) != cudaSuccess) return TOD_ERR_CUDA;
    const float tol = cg_tol > 0 ? static_cast<float>(cg_tol) : 1e-6f;
    const int maxit = cg_maxiter > 0 ? cg_maxiter : 500;
    cudaError_t e = p->use_prec ? launch_toeplitz_prep(*p, psd, stream) : cudaSuccess;
    for (int q0 = 0; q0 < p->nq && e == cudaSuccess;) {
        int q1 = q0 + 1;
        while (q1 < p->nq && p->h_off[q1 + 1] - p->h_off[q0] <= S) ++q1;
        const int64_t Sw = p->h_off[q1] - p->h_off[q0];
        const WaveCarve c = carve(Sw);
        char *b = reinterpret_cast<char *>(base);
        TxNcorrScratch sc;
        sc.Y = reinterpret_cast<float2 *>(b);
        sc.wpre = reinterpret_cast<int64_t *>(b + c.y_bytes);
        sc.cgv = reinterpret_cast<float *>(b + c.y_bytes + c.w_bytes);
        sc.cgcap = std::max<int64_t>(1, Sw / 4);
        int items = 0;
        for (int q = q0; q < q1; ++q)
            items = std::max(items, std::max(p->h_col_off[q + 1] - p->h_col_off[q], p->h_row_off[q + 1] - p->h_row_off[q]));
        const int grid = std::min(p->pass_grid, std::max(1, (p->h_col_off[q1] - p->h_col_off[q0])));
        e = launch_tx_ncorr(*p, d, s, gain, flags, psd, rng, mode, tol, maxit, ncorr_out, cg_iters_out, stream, q0,
                            q1, sc, std::max(1, std::min(p->pass_grid, std::max(grid, items))));
        q0 = q1;
    }
    if (prev != p->device) cudaSetDevice(prev);
    if (e == cudaSuccess) return TOD_OK;
    return e == cudaErrorMemoryAllocation ? TOD_ERR_OOM : TOD_ERR_CUDA;
}

}  // extern "C"
