// tod_sample_ncorr_static: the correlated-noise draw of tod_sample_ncorr with
// its per-cluster scratch (filter weights, CG spectra) in a fixed device
// array compiled into the library, so the call itself allocates nothing.
//
// The scratch is one file-scope __device__ array per device of
// TOD_NCORR_STATIC_SCRATCH_BYTES.  Its device address is looked up once per
// device (with that device current) by cudaGetSymbolAddress and cached.  Each
// cluster of the draw writes its scratch before it reads it, so no
// part of the array has to start at zero.  All calls on one device share the
// array: two calls that may run at the same time (other streams, other
// plans, other host threads) race on it.
#include <algorithm>
#include <mutex>
#include "internal.cuh"

namespace tg {

constexpr size_t kNcorrStaticFloat4 = TOD_NCORR_STATIC_SCRATCH_BYTES / sizeof(float4);

static __device__ __align__(256) float4 g_ncorr_static_scratch[kNcorrStaticFloat4];

constexpr int kMaxDevices = 64;
static std::mutex g_static_mu;
static float4 *g_static_addr[kMaxDevices] = {};

// Device address of the static scratch on `dev` (made current by the caller).
static cudaError_t static_scratch(int dev, float4 **out)
{
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_static_mu);
    if (!g_static_addr[dev]) {
        void *ptr = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&ptr, g_ncorr_static_scratch);
        if (e != cudaSuccess) return e;
        g_static_addr[dev] = static_cast<float4 *>(ptr);
    }
    *out = g_static_addr[dev];
    return cudaSuccess;
}

}  // namespace tg

using namespace tg;

extern "C" {

tod_status tod_ncorr_static_setup(tod_plan *pl, int32_t *max_clusters_out)
{
    if (!pl) return TOD_ERR_ARG;
    Plan *p = reinterpret_cast<Plan *>(pl);
    int prev = 0;
    if (cudaGetDevice(&prev) != cudaSuccess) return TOD_ERR_CUDA;
    if (prev != p->device && cudaSetDevice(p->device) != cudaSuccess) return TOD_ERR_CUDA;
    float4 *scratch = nullptr;
    const cudaError_t e = static_scratch(p->device, &scratch);
    if (prev != p->device) cudaSetDevice(prev);
    if (e != cudaSuccess) return TOD_ERR_CUDA;
    const int64_t per_cluster = static_cast<int64_t>(p->C) * p->sz * NCORR_SCRATCH_F4;     // float4 per cluster
    const int64_t fit = static_cast<int64_t>(kNcorrStaticFloat4) / std::max<int64_t>(1, per_cluster);
    if (max_clusters_out) max_clusters_out[0] = static_cast<int32_t>(std::min<int64_t>(fit, p->nclusters_ncorr));
    return fit < 1 ? TOD_ERR_SCRATCH : TOD_OK;
}

tod_status tod_sample_ncorr_static(tod_plan *pl, const float *d, const float *s, const double *gain,
                                   const uint32_t *flags, const double *psd, tod_rng rng, int32_t mode,
                                   double cg_tol, int32_t cg_maxiter, float *ncorr_out,
                                   int32_t *cg_iters_out, cudaStream_t stream)
{
    if (!pl || !d || !s || !gain || !flags || !psd || !ncorr_out) return TOD_ERR_ARG;
    if (mode != TOD_MODE_DRAW && mode != TOD_MODE_MEAN) return TOD_ERR_ARG;
    Plan *p = reinterpret_cast<Plan *>(pl);
    const int64_t per_cluster = static_cast<int64_t>(p->C) * p->sz * NCORR_SCRATCH_F4;
    const int64_t fit = static_cast<int64_t>(kNcorrStaticFloat4) / std::max<int64_t>(1, per_cluster);
    if (fit < 1) return TOD_ERR_SCRATCH;          // one cluster's weights exceed the array
    int prev = 0;
    if (cudaGetDevice(&prev) != cudaSuccess) return TOD_ERR_CUDA;
    if (prev != p->device && cudaSetDevice(p->device) != cudaSuccess) return TOD_ERR_CUDA;
    float4 *scratch = nullptr;
    cudaError_t e = static_scratch(p->device, &scratch);
    if (e == cudaSuccess) {
        const float tol = cg_tol > 0 ? static_cast<float>(cg_tol) : 1e-6f;
        const int maxit = cg_maxiter > 0 ? cg_maxiter : 500;
        e = launch_ncorr_scratch(*p, d, s, gain, flags, psd, rng, mode, tol, maxit, ncorr_out,
                                 cg_iters_out, stream, 0, p->nq, scratch, static_cast<int>(fit));
    }
    if (prev != p->device) cudaSetDevice(prev);
    if (e == cudaSuccess) return TOD_OK;
    return e == cudaErrorMemoryAllocation ? TOD_ERR_OOM : TOD_ERR_CUDA;
}

}  // extern "C"
