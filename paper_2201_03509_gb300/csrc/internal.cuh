// Internal plan layout and kernel-launcher prototypes of libtodgibbs.
#pragma once
#include <cstdint>
#include <vector>
#include <cuda_runtime.h>
#include "../../include/todgibbs.h"
#include "common.cuh"

namespace tg {

constexpr int DEC_LUTB = 13;          // first-level decode table: 2^13 packed 32-bit entries
constexpr int32_t DEC_WIDE = -(1 << 26);   // table value: symbol too wide for the entry, read canonically
constexpr int DEC_T = 512;
constexpr int NCORR_SCRATCH_F4 = 2;   // float4 per packed slot of the n_corr scratch: filter weights, CG spectra            // decode threads per CTA (one checkpoint block each)
constexpr int DEC_ROUND = 16;         // symbols staged per thread before a coalesced write
// what a decoded value becomes: itself (pointing), the FP32 TOD, a flag bit
enum : int { DEC_VALUE = 0, DEC_TOD = 1, DEC_FLAG = 2 };
constexpr int ELEM_TILE = 4096;       // samples per tile of the element-wise kernels
constexpr int DCT_T = 512;            // threads per CTA of the cluster transform kernels
constexpr int DCT_SZ_MAX = 11776;     // complex values per CTA buffer (two buffers + CG fit in 227 KB)
constexpr int DCT_MAXR = 20;          // maximum number of radix stages per sub-transform
constexpr int CG_KCAP = 768;          // flagged samples per CTA held by the CG
constexpr int TOEP_LMAX = 512;        // longest gap block of the Toeplitz preconditioner
constexpr int GB_CAP = 1024;          // preconditioner elements applied per round in one CTA
constexpr int BIN_TILE = 2048;        // sorted samples staged per binning tile
constexpr int GAP_CAP = 256;          // gap blocks per detscan handled by the preconditioner

// Compressed stream kind, device copy + decode tables.
struct HuffDev {
    uint32_t *words = nullptr;       // + 2 zero pad words
    int64_t *word_off = nullptr;     // [nq+1]
    int64_t *nbits = nullptr;        // [nq]
    int64_t *blk_off = nullptr;      // [nq+1]
    uint32_t *ckpt_bit = nullptr;    // [nblk]
    int32_t *ckpt_val = nullptr;     // [nblk]
    int32_t *blk_q = nullptr;        // [nblk] detscan of each block
    int32_t *lut = nullptr;          // [nscan][1<<DEC_LUTB] value << 5 | length; length 0 = long code
    unsigned long long *lim = nullptr;  // [nscan][26] left-justified limits, index = length
    int32_t *base = nullptr;         // [nscan][26]
    int32_t *canon_off = nullptr;    // [nscan+1]
    int32_t *canon_vals = nullptr;   // symbols in canonical order
    int32_t *cta_scan = nullptr;     // decode work list: one entry per CTA
    int64_t *cta_blk0 = nullptr;
    int32_t *cta_nblk = nullptr;
    int32_t ncta = 0;
    int32_t max_canon = 0;           // largest code of any scan (symbols)
    int64_t nblk = 0;
};

// One Stockham pass of a sub-transform: radix R after Ns points are done.
struct DctStage {
    int32_t R, Ns;
    FastDiv fLR, fNs;                // divisions by L/R and Ns
};

// Per-length transform plan (real DCT-II of length n via an m = n/2 complex
// FFT split as m1 x m2 across a cluster of C CTAs).
struct DctPlan {
    int32_t n, m, m1, m2, ncolmax, npmax, P;
    int32_t m2p;                     // row stride of the frequency layout: m2 made odd
    int32_t nr1, nr2;
    int32_t tw1, tw2;                // offsets of the W_{m1}^i and W_{m2}^i tables
    int32_t twb;                     // offset of this length's twiddle block (see k_dct.cu)
    FastDiv f_ncolmax, f_m2, f_npmax;
    float sq_fwd, s0_fwd, sq_inv, s0_inv;   // real-split scales (FP64-computed on the host)
    DctStage s1[DCT_MAXR], s2[DCT_MAXR];
};

struct Plan {
    int device = 0;
    int32_t nside = 0, npix = 0, ndet = 0, nscan = 0, nq = 0;
    double fsamp = 0;
    int64_t N = 0;
    std::vector<int64_t> h_off;      // host copy of offsets
    int64_t *off = nullptr;          // [nq+1] device
    int32_t *status = nullptr;       // [nq] device
    HuffDev hpix, hpsi;
    // compressed TOD (ADC counts) and flag words, when attached
    HuffDev htod, hflag;
    bool has_tod = false, has_flag = false;
    double *tod_scale = nullptr;     // [nq] ADC quantum per detscan
    uint32_t flag_select = 0;        // flag-word bits that exclude a sample
    // element-wise tiles
    int32_t ntile = 0;
    int32_t *tile_q = nullptr;
    int64_t *tile_t0 = nullptr;
    float2 *trig = nullptr;          // [TOD_N_PSI] (cos 2psi, sin 2psi) at bin centres, FP32
    // transforms
    int32_t C = 1;                   // CTAs per cluster
    int32_t sz = 0;                  // complex values per CTA buffer (max over plans)
    int32_t twsz = 0;                // complex values of the largest twiddle block
    int32_t m1max = 0, m2max = 0;
    int32_t nplans = 0;
    DctPlan *plans = nullptr;        // device
    int32_t *q_plan = nullptr;       // [nq] plan index of each detscan
    float2 *tw = nullptr;            // twiddle tables
    int32_t *work = nullptr;         // [nq] detscans sorted by decreasing length
    int32_t nclusters_gain = 1, nclusters_ncorr = 1;
    float4 *wscratch = nullptr;      // per-CTA filter weights (beta, gamma) and CG spectra, packed layout
    float *htab = nullptr;           // [ndet][TOEP_LMAX] gap-kernel h(d)
    float *xtab = nullptr;           // [ndet][TOEP_LMAX (TOEP_LMAX+1)/2] T_L^{-1} e_1 per order
    int32_t *lvalid = nullptr;       // [ndet]
    int32_t toep_nref = 0;
    bool use_prec = true;
    int64_t wscratch_per_cluster = 0;
    int32_t schedule = TOD_SCHED_PERSISTENT;
    int32_t nbin_tiles = 0;          // binning tiles (whole runs of one detscan)
    double2 *gain_ab = nullptr;      // [nq] (a, b) of each detscan's gain conditional (scratch)
    // noise PSD step
    float *spec_out = nullptr;       // caller's buffer for the n_corr spectra (NULL: not written)
    float2 *lnk = nullptr;           // [longest detscan] ln k as an FP32 pair (hi, lo)
    double *lnfs = nullptr;          // [nq] ln(fsamp / (2 n_q))
    double *psd_nmodes = nullptr;    // [ndet] modes k >= 1 of the detector's detscans
    double *psd_sumlnf = nullptr;    // [ndet] sum of ln f_k over them
    double *psd_part = nullptr;      // [ntile] partial sums of one evaluation
    double *psd_state = nullptr;     // [ndet][8] chain state
    size_t smem_gain = 0, smem_ncorr = 0;
    // binning
    // Runs: the samples of one (detscan, pixel), in time order; a detscan's
    // runs ordered by their first sample, stored run-major.  A tile's samples
    // are loaded k-major (the k-th sample of each of its runs, k = 0, 1, ..):
    uint32_t *ld_t = nullptr;        // [N] time index within the detscan, in load order
    uint16_t *ld_pos = nullptr;      // [N] run-major position within the tile, in load order
    int32_t *bin_tile_q = nullptr;   // [nbin_tiles] detscan of the tile
    int32_t *bin_tile_r0 = nullptr;  // [nbin_tiles + 1] first run (global run index); last entry = npairs
    int64_t npairs = 0;
    int64_t *pair_off = nullptr;     // [nq+1] runs of each detscan
    int64_t *pair_start = nullptr;   // [npairs] run-major position (global) of the run's first sample
    int32_t *pair_len = nullptr;     // [npairs]
    int32_t *pair_slot = nullptr;    // [npairs] the run's slot among its pixel's runs (detscan order)
    int64_t *pix_slot_off = nullptr; // [npix+1]
    double *rec = nullptr;           // [npairs][10] per-run partial sums (scratch)
    int64_t device_bytes = 0;
    std::vector<void *> allocs;
};

// launchers (return cudaError_t of the launch)
cudaError_t setup_decode_kernel();
cudaError_t launch_decode(const Plan &p, const HuffDev &h, int32_t *pix_out, uint16_t *psi_out,
                          cudaStream_t st);
cudaError_t launch_decode_tod(const Plan &p, float *d_out, cudaStream_t st);

// joint gain draw under the smooth prior across scans (one CTA per detector)
struct GainSmoothArgs {
    const double *mu, *sigma;    // [nq] per-detscan gain conditionals, q = scan * ndet + det
    const double *prior;         // [ndet][2] sigma_g, alpha_g
    int32_t nscan, ndet;
    tod_rng rng;
    int32_t mode;
    float tol;
    int32_t maxiter;
    double *gain_out;            // [nq]
    int32_t *iters_out;          // [ndet] or null
    int32_t *status;
};
size_t gain_smooth_smem(int nscan);
cudaError_t setup_gain_smooth_kernel();
cudaError_t launch_gain_smooth(const GainSmoothArgs &a, cudaStream_t st);
cudaError_t launch_decode_flags(const Plan &p, uint32_t *flags_out, cudaStream_t st);
cudaError_t launch_project(const Plan &p, const float4 *map, const int32_t *pix, const uint16_t *psi,
                           const double *gain, float *s_out, cudaStream_t st);
cudaError_t setup_dct_kernels(Plan &p);
// co-resident clusters of C CTAs of the n_corr kernel with smem_dyn bytes of
// dynamic shared memory each (0 if none fits)
cudaError_t transform_cluster_occupancy(int C, size_t smem_dyn, int *nclusters);
cudaError_t launch_gain(const Plan &p, const float *d, const float *s, const uint32_t *flags,
                        const double *psd, tod_rng rng, int mode, double *g, double *mu,
                        double *sig, cudaStream_t st, int work_begin, int work_count);
cudaError_t launch_ncorr(const Plan &p, const float *d, const float *s, const double *gain,
                         const uint32_t *flags, const double *psd, tod_rng rng, int mode,
                         float tol, int maxit, float *x, int32_t *iters, cudaStream_t st,
                         int work_begin, int work_count, bool prepare = true);
// the same draw with caller-provided filter-weight scratch: at most
// nclusters_max clusters, each using C x sz float4 of it
cudaError_t launch_ncorr_scratch(const Plan &p, const float *d, const float *s, const double *gain,
                                 const uint32_t *flags, const double *psd, tod_rng rng, int mode,
                                 float tol, int maxit, float *x, int32_t *iters, cudaStream_t st,
                                 int work_begin, int work_count, float4 *scratch, int nclusters_max,
                                 bool prepare = true);
cudaError_t launch_chi2(const Plan &p, const float *d, const float *s, const double *gain,
                        const uint32_t *flags, const double *psd, double *chi2, double *dgain,
                        double *dpsd, float *v, cudaStream_t st);
cudaError_t setup_bin_kernel(Plan &p);
cudaError_t launch_toeplitz_prep(const Plan &p, const double *psd, cudaStream_t st);
cudaError_t launch_noise_psd(const Plan &p, const float *spec, const double *psd_in, tod_rng rng, int nsteps,
                             double step_lnfk, double step_al, double *psd_out, int32_t *acc_out,
                             double *loglike_out, cudaStream_t st);
cudaError_t launch_bin(const Plan &p, const uint16_t *psi, const float *d, const float *ncorr,
                       const double *gain, const uint32_t *flags, const double *psd, double *A,
                       double *b, int32_t *hits, cudaStream_t st);
cudaError_t launch_solve(const Plan &p, const double *A, const double *b, const int32_t *hits,
                         double rcond_min, double *map, float4 *map32, double *rcond,
                         uint8_t *valid, cudaStream_t st);

}  // namespace tg
