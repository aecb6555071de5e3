/*
 * todgibbs.h -- C ABI of the GB300 Gibbs TOD step library (libtodgibbs.so).
 *
 * The library implements the data-parallel per-scan time-ordered-data (TOD)
 * step of the Commander3 Gibbs sampler (BeyondPlanck, arXiv 2201.03509):
 * Huffman decode of the pointing streams (Sect. 4.1), projection of the TQU
 * sky (Eq. `todmodel`), the gain and correlated-noise conditionals
 * (Eq. `gibbsstart`, first two lines; Sect. 5 on CG gap filling), binning
 * into per-pixel normal equations and their solution (Sect. 5 table, rows
 * "TOD binning" and "Map solution").
 *
 * Conventions for every entry point
 *  - A band holds ndet detectors x nscan scans.  A "detscan" q = scan*ndet+det
 *    owns samples [off[q], off[q+1]) of every per-sample array (the
 *    comm_scan / comm_detscan hierarchy of Listing `tod`).
 *  - Sample counts are FFT lengths: even 2^a 3^b 5^c numbers (Sect. 4.2);
 *    use tod_fft_length() when ingesting.
 *  - Unless stated otherwise, array arguments of compute calls are DEVICE
 *    pointers owned by the caller; the library never frees them.  Calls are
 *    asynchronous on the given stream (0 = legacy default stream), return
 *    after enqueueing, and only argument errors are reported immediately.
 *    Faults found on the device (a data stream that does not decode, CG not
 *    converged, a detscan without usable samples or with non-finite sums)
 *    are recorded per detscan and read with tod_plan_status() after the
 *    stream is synchronised.  No call traps the GPU.  Non-finite detector
 *    data are not checked sample by sample: they surface as TOD_ERR_ARG
 *    from the gain draw (non-finite sums) and TOD_ERR_NOT_CONVERGED from
 *    the gap filling of flagged detscans.
 *  - flags: bit (t & 31) of word (t >> 5) is 1 when sample t (global index)
 *    is flagged (excluded: M_t = 0).
 *  - psd: double[ndet][3] = (sigma0 [data units], f_knee [Hz], alpha < 0).
 *    Noise model P(f) = sigma0^2 (1 + (f/f_knee)^alpha) at DCT frequencies
 *    f_k = k f_samp / (2 n) (the mirrored array of Sect. 4.2 has period 2n).
 *  - Not thread-safe per plan: calls on one plan must not run concurrently
 *    from several host threads.  Calls on one plan in different streams race.
 */
#ifndef TODGIBBS_H
#define TODGIBBS_H

#include <stdint.h>
#include <cuda_runtime_api.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int32_t tod_status;

#define TOD_OK                 0
#define TOD_ERR_ARG           -1   /* bad argument; nothing was enqueued */
#define TOD_ERR_CORRUPT_STREAM -2  /* a Huffman stream did not decode */
#define TOD_ERR_NOT_CONVERGED -3   /* CG gap filling hit its iteration cap */
#define TOD_ERR_TIMEOUT       -4   /* reserved: no call of this library waits on the device */
#define TOD_ERR_CUDA          -5   /* a CUDA runtime call failed */
#define TOD_ERR_OOM           -6   /* device or host allocation failed */
#define TOD_ERR_UNIMPLEMENTED -7
#define TOD_ERR_SCRATCH       -8   /* the plan needs more scratch than a fixed array holds */

#define TOD_MODE_DRAW 0   /* sample from the conditional */
#define TOD_MODE_MEAN 1   /* conditional mean: all normals set to zero */

#define TOD_N_PSI 4096    /* polarisation-angle bins over [0, 2pi) (Sect. 4.1) */
#define TOD_CKPT_BLOCK 512
#define TOD_HUFF_MAXLEN 24

/* Short, static description of a status code.  Never NULL. */
const char *tod_status_string(tod_status s);

/* Largest even 2^a 3^b 5^c not above n (0 if n < 2).  Sect. 4.2: chunks are
 * truncated at read-in to lengths that are cheap to transform; a detscan
 * keeps its first tod_fft_length(n) samples. */
int64_t tod_fft_length(int64_t n);

/* ---------------------------------------------------------------------------
 * Compressed pointing stream of one kind (HEALPix RING pixel, or psi bin) for
 * a whole band (Sect. 4.1: samples differenced, x(i) - x(i-1) with x(-1) = 0,
 * then Huffman coded; Listing `tod`: pix/psi stored as bytes).  Format:
 *   - one canonical Huffman code per (scan, kind), shared by the scan's
 *     detectors; code lengths <= TOD_HUFF_MAXLEN; symbols of each code listed
 *     in ascending value with their lengths (codes follow canonically:
 *     ordered by (length, value), consecutive, first code all zeros);
 *   - bits most-significant first in 32-bit words; each detscan's stream
 *     starts on a word boundary;
 *   - a checkpoint every TOD_CKPT_BLOCK samples: the bit offset of the block
 *     (relative to the detscan's first word) and the value preceding it.
 * All pointers HOST, read during the call only.
 * ------------------------------------------------------------------------- */
typedef struct {
    const uint32_t *words;      int64_t nwords;
    const int64_t  *word_off;   /* [ndetscan+1] first word of each detscan  */
    const int64_t  *nbits;      /* [ndetscan]   payload bits per detscan    */
    const int64_t  *blk_off;    /* [ndetscan+1] first checkpoint per detscan */
    const uint32_t *ckpt_bit;   /* [nblk] */
    const int32_t  *ckpt_val;   /* [nblk] */
    int64_t         nblk;
    const int64_t  *sym_off;    /* [nscan+1] first symbol of each scan's code */
    const int32_t  *sym_vals;   /* [nsym] ascending per scan */
    const uint8_t  *sym_len;    /* [nsym] */
    int64_t         nsym;
} tod_huff_streams;

/* Library-allocated output of tod_huff_encode (host memory). */
typedef struct {
    uint32_t *words;    int64_t nwords;
    int64_t  *word_off; int64_t *nbits; int64_t *blk_off;
    uint32_t *ckpt_bit; int32_t *ckpt_val; int64_t nblk;
    int64_t  *sym_off;  int32_t *sym_vals; uint8_t *sym_len; int64_t nsym;
} tod_huff_buffers;

/* Ingest (host, not on the per-step path): compress one stream kind of a
 * band.  values: HOST int32[offsets[ndetscan]] (pixel indices, psi bins,
 * ADC counts or flag words); every difference of consecutive values of a
 * detscan must fit in int32 (TOD_ERR_ARG otherwise).
 * offsets: HOST int64[ndet*nscan+1].  Fills *out with malloc'd arrays that
 * the caller releases with tod_huff_free.  Tie rules of the Huffman build:
 * leaves ordered by (count, value); two-queue merge taking the leaf on equal
 * counts; lengths above TOD_HUFF_MAXLEN trigger count halving ((c+1)/2) and
 * a rebuild.  A code with one symbol gets the 1-bit code 0.  Uses host
 * threads.  Returns TOD_ERR_ARG on bad sizes, TOD_ERR_OOM on allocation
 * failure. */
tod_status tod_huff_encode(int32_t ndet, int32_t nscan, const int64_t *offsets,
                           const int32_t *values, tod_huff_buffers *out);
void tod_huff_free(tod_huff_buffers *b);

/* ---------------------------------------------------------------------------
 * Plan = the band's TOD object (Listing `tod`: comm_tod -> comm_scan ->
 * comm_detscan): device copies of the compressed pointing streams, decode
 * tables, the per-detscan transform plans, the pixel-sorted binning
 * structure (pointing is fixed during the run, Sect. 2.1, so it is built
 * once) and scratch.  tod_plan_create decodes the pointing on the host to
 * build the binning structure.
 * ------------------------------------------------------------------------- */
typedef struct tod_plan tod_plan;

typedef struct {
    int32_t nside;          /* HEALPix Nside; npix = 12 nside^2 */
    int32_t ndet;
    int32_t nscan;
    int32_t n_psi;          /* must be TOD_N_PSI */
    double  fsamp;          /* sample rate [Hz] */
    const int64_t *offsets; /* HOST [ndet*nscan+1]; every length an FFT length */
    tod_huff_streams pix;   /* HOST compressed pixel stream */
    tod_huff_streams psi;   /* HOST compressed psi-bin stream */
    int32_t tile_pairs;     /* column pairs per tile of the transforms' column passes: 0 = the
                               widest tile that fits, else a cap 1..64 (the tile takes the
                               largest power of two not above it) */
    int32_t device;         /* CUDA device ordinal the plan lives on */
    int32_t max_radix;      /* largest Stockham radix of the transforms: 0 = 16; else 2..16 */
} tod_band_desc;

/* Counter-based random streams: Philox4x64-10 (Salmon et al. 2011) with key
 * (seed, band) and counter (block, detscan, purpose, gibbs_iter); purposes
 * 0 = gain, 1 = white-noise term, 2 = prior term of the n_corr draw. */
typedef struct {
    uint64_t seed;
    uint64_t band;
    uint64_t gibbs_iter;
    /* Optional DEVICE pointer: when non-NULL the kernels read the Gibbs
     * iteration from this word when they run (gibbs_iter is ignored), so a
     * captured CUDA graph replays with a new iteration after the caller
     * updates the word. */
    const uint64_t *gibbs_iter_dev;
} tod_rng;

tod_status tod_plan_create(tod_plan **out, const tod_band_desc *band);
tod_status tod_plan_destroy(tod_plan *p);
/* Sizes of the plan (host scalars; any pointer may be NULL). */
tod_status tod_plan_info(const tod_plan *p, int64_t *nsamples, int32_t *ndetscan,
                         int32_t *npix, int32_t *tile_pairs, int64_t *device_bytes);
/* Sizes of the plan's binning structure (host scalars; any pointer may be
 * NULL): runs (the samples of one (detscan, pixel) pair; one record of 80
 * bytes each per binning) and binning tiles. */
tod_status tod_plan_binning_info(const tod_plan *p, int64_t *nruns, int32_t *ntiles);
/* Synchronises the device, copies the per-detscan status words
 * (TOD_OK or an error code) into HOST int32[ndetscan] (may be NULL), clears
 * them, and returns the first error found (TOD_OK if none). */
tod_status tod_plan_status(tod_plan *p, int32_t *detscan_status);

/* Launch schedule of the transform stages (gain, n_corr):
 * TOD_SCHED_PERSISTENT (default): every pass of a stage is one launch over
 * the tiles of all detscans (the n_corr draw: a fixed sequence of pass
 * launches, its CG iterations past the eighth in one cooperative launch);
 * TOD_SCHED_PER_SCAN: the same kernels launched once per detscan (the
 * plain per-scan path, kept for comparison).  Results are identical: each
 * detscan's arithmetic does not depend on the others or on the launch. */
#define TOD_SCHED_PERSISTENT 0
#define TOD_SCHED_PER_SCAN   1
tod_status tod_plan_set_schedule(tod_plan *p, int32_t schedule);

/* Preconditioner of the n_corr CG (the Schur-complement solve of
 * tod_sample_ncorr; the paper fills the gaps with FFTs inside a CG solver,
 * Sect. 5, and states no preconditioner, so this is an implementation
 * choice): TOD_PREC_NONE;
 * TOD_PREC_BLOCKS, the exact inverses of
 * the gap blocks' Toeplitz matrices; TOD_PREC_TWO_LEVEL (default), those
 * plus a coarse correction over two vectors per gap block (indicator and
 * ramp) in the balancing form.  The solution is the same to the CG
 * tolerance; only the iteration count changes.  TOD_ERR_ARG for other
 * values. */
#define TOD_PREC_NONE      0
#define TOD_PREC_BLOCKS    1
#define TOD_PREC_TWO_LEVEL 2
tod_status tod_plan_set_preconditioner(tod_plan *p, int32_t levels);

/* Per-kernel timing (no counterpart in the paper; for measurement).  While
 * on, every kernel launch of this plan's calls is bracketed by two CUDA
 * events on the call's stream, recorded with the kernel's class below.
 * tod_plan_set_kernel_timing(p, 1) clears the records and starts timing,
 * (p, 0) stops it (records are kept).  tod_plan_kernel_times synchronises
 * on the recorded events and writes, per class, the summed milliseconds
 * (HOST double[TOD_KT_COUNT], may be NULL) and the number of launches (HOST
 * int32[TOD_KT_COUNT], may be NULL).  The events cost a few microseconds
 * per launch: time the headline separately.  Calls on one plan must not
 * overlap while timing is on.  tod_kernel_name gives a class's kernel name
 * (NULL outside [0, TOD_KT_COUNT)). */
enum {
    TOD_KT_DECODE = 0,        /* k_decode of the pointing (pix and psi: two launches) */
    TOD_KT_DECODE_TOD,        /* k_decode of the compressed TOD */
    TOD_KT_DECODE_FLAGS,      /* k_decode of the compressed flag words */
    TOD_KT_PROJECT,           /* k_project */
    TOD_KT_PROJECT64,         /* k_project64 */
    TOD_KT_DET_SCALARS,       /* k_det_scalars */
    TOD_KT_GAIN_COLS,         /* k_gain_cols */
    TOD_KT_GAIN_ROWS,         /* k_gain_rows */
    TOD_KT_GAIN_COLSINV,      /* k_gain_colsinv */
    TOD_KT_GAIN_FIN,          /* k_gain_fin */
    TOD_KT_TOEP_KERNEL,       /* the gap kernel h(d) and its prefix sums: k_cz_fill, the k_cz_fft
                                 passes (log2 of twice the reference length, halved, rounded up),
                                 k_cz_sums, k_cz_tables */
    TOD_KT_TOEP_DURBIN,       /* k_toep_durbin */
    TOD_KT_NC_FLAG_COUNT,     /* k_nc_flag_count */
    TOD_KT_NC_FLAG_SCAN,      /* k_nc_flag_scan */
    TOD_KT_NC_FLAG_WRITE,     /* k_nc_flag_write */
    TOD_KT_NC_INDEX,          /* k_nc_index */
    TOD_KT_NC_COARSE,         /* k_nc_coarse (the coarse correction of the preconditioner) */
    TOD_KT_NC_RHS_COLS,       /* k_nc_rhs_cols */
    TOD_KT_NC_RHS_ROWS,       /* k_nc_rhs_rows */
    TOD_KT_NC_X0_COLS,        /* k_nc_x0_cols */
    TOD_KT_NC_CG_INIT,        /* k_nc_cg_init */
    TOD_KT_NC_SCATTER,        /* k_nc_scatter of a CG iteration */
    TOD_KT_NC_FILTER,         /* k_nc_filter of a CG iteration */
    TOD_KT_NC_GATHER,         /* k_nc_gather of a CG iteration */
    TOD_KT_NC_UPDATE,         /* k_nc_update */
    TOD_KT_NC_LIST,           /* k_nc_list (the detscans a CG pass works on) */
    TOD_KT_NC_TAIL,           /* k_nc_tail (cooperative: the remaining CG iterations) */
    TOD_KT_NC_SCATTER_FINAL,  /* k_nc_scatter of the correction x = x0 + B^-1 E y */
    TOD_KT_NC_FILTER_FINAL,   /* k_nc_filter of the correction */
    TOD_KT_NC_GATHER_FINAL,   /* k_nc_gather of the correction */
    TOD_KT_NC_FINISH,         /* k_nc_finish */
    TOD_KT_BIN,               /* k_bin */
    TOD_KT_REDUCE,            /* k_reduce */
    TOD_KT_COMBINE,           /* k_combine */
    TOD_KT_SOLVE,             /* k_solve */
    TOD_KT_CHI2_COLS,         /* k_chi2_cols */
    TOD_KT_CHI2_ROWS,         /* k_chi2_rows */
    TOD_KT_CHI2_COLSINV,      /* k_chi2_colsinv */
    TOD_KT_CHI2_FIN,          /* k_chi2_fin and k_chi2_total */
    TOD_KT_PSD_SUMS,          /* k_psd_sums */
    TOD_KT_PSD_STEP,          /* k_psd_begin and k_psd_step */
    TOD_KT_COUNT
};
const char *tod_kernel_name(int32_t id);
tod_status tod_plan_set_kernel_timing(tod_plan *p, int32_t on);
tod_status tod_plan_kernel_times(tod_plan *p, double *ms_out, int32_t *launches_out);

/* A1 -- Huffman decode + undo differencing (Sect. 4.1).
 * pix_out int32[N], psi_out uint16[N] (device).  Bit-exact.  The pointing
 * streams are decoded once on the host by tod_plan_create (to build the
 * binning order), which rejects a stream that does not decode, so the
 * device-side check (TOD_ERR_CORRUPT_STREAM) cannot fire here. */
tod_status tod_decode(tod_plan *p, int32_t *pix_out, uint16_t *psi_out, cudaStream_t stream);

/* ---------------------------------------------------------------------------
 * Joint gain draw of every detector's scans under a smooth prior across
 * scans (the gain conditional of Eq. `gibbsstart` per detscan as the
 * likelihood; the paper defers the gain model to its calibration companion
 * paper, so the prior is this library's reading).  Per detector, with S
 * scans, a_s = 1/sigma_s^2 and b_s = mu_s/sigma_s^2 from the per-detscan
 * conditionals N(mu_s, sigma_s^2) (tod_sample_gain's mu_out, sigma_out):
 *   prior precision C^T diag(lambda) C, C the orthonormal DCT-II over the
 *   scan index, lambda_0 = 0 (mean gain free),
 *   lambda_k = 1 / (sigma_g^2 k^alpha_g) for k >= 1;
 *   A g = b + a^(1/2) w1 + C^T (lambda^(1/2) w2),
 *   A = diag(a) + C^T diag(lambda) C (noise terms dropped in TOD_MODE_MEAN).
 * w1_s, w2_s: Philox block (s, det, TOD_PURPOSE_GAIN_SMOOTH, iteration),
 * 53-bit uniforms from words 0, 1 (w1) and 2, 3 (w2), Box-Muller cosine
 * branch in FP64.  Preconditioned CG in FP32 (double-word transform sums,
 * FP64 dot products) to relative residual cg_tol, at most cg_maxiter
 * iterations; a detector that does not converge marks detscan det
 * TOD_ERR_NOT_CONVERGED, a sigma_s <= 0 or non-finite input marks its
 * detscan TOD_ERR_ARG.
 *   mu, sigma: DEVICE double[ndetscan]; prior: DEVICE double[ndet][2]
 *   (sigma_g > 0, alpha_g); gain_out: DEVICE double[ndetscan];
 *   cg_iters_out: DEVICE int32[ndet] or NULL.
 * TOD_ERR_ARG (host) when nscan > TOD_GAIN_SMOOTH_MAX_SCANS.  A detector
 * whose prior has sigma_g not > 0 (or zero once squared in FP32), or a
 * non-finite sigma_g or alpha_g, gets TOD_ERR_ARG in the status word of
 * each of its detscans and gains of 0; the other detectors are drawn.
 * ------------------------------------------------------------------------- */
#define TOD_GAIN_SMOOTH_MAX_SCANS 4096
tod_status tod_sample_gain_smooth(tod_plan *p, const double *mu, const double *sigma, const double *prior,
                                  tod_rng rng, int32_t mode, double cg_tol, int32_t cg_maxiter,
                                  double *gain_out, int32_t *cg_iters_out, cudaStream_t stream);

/* ---------------------------------------------------------------------------
 * Compressed TOD and quality flags (Sect. 4.1: the ADC integers and the flag
 * words are differenced and Huffman coded like the pointing; Listing `tod`:
 * comm_detscan holds tod and flag as compressed bytes).  Both streams use
 * the tod_huff_streams format above over the plan's offsets.
 *   tod:   ADC counts c_t (int32); the detector data are
 *          d_t = fl32(scale_q * c_t), the product in FP64, rounded once.
 *   flag:  flag words w_t (int32, read as uint32); sample t is flagged
 *          (M_t = 0) when (w_t & flag_select) != 0.
 * ------------------------------------------------------------------------- */
typedef struct {
    tod_huff_streams tod;       /* HOST compressed ADC counts */
    const double *tod_scale;    /* HOST [ndetscan] ADC quantum of each detscan (> 0, finite) */
    tod_huff_streams flag;      /* HOST compressed flag words */
    uint32_t flag_select;       /* flag-word bits that exclude a sample */
} tod_data_desc;

/* Ingest: copies both streams and their decode tables to the device (once
 * per plan; TOD_ERR_ARG if already attached or a stream is malformed). */
tod_status tod_plan_attach_data(tod_plan *p, const tod_data_desc *data);

/* A1 for the data streams: d_out float32[N] (d_t above), flags_out
 * uint32[(N+31)/32] (the flags layout of this header, fully rewritten:
 * zeroed, then the flagged bits set).  Either may be NULL, not both.
 * Bit-exact; TOD_ERR_ARG when nothing is attached; a stream that does not
 * decode marks its detscan TOD_ERR_CORRUPT_STREAM. */
tod_status tod_decode_data(tod_plan *p, float *d_out, uint32_t *flags_out, cudaStream_t stream);

/* A2 -- projection (Eq. `todmodel`, the g P m term):
 * s_t = g_q (T_p + Q_p cos 2psi_t + U_p sin 2psi_t), p = pix_t,
 * psi_t = (bin + 1/2) 2pi / TOD_N_PSI, cos/sin tabulated in FP32.
 * map_tqu: float4[npix] (T, Q, U, unused).  gain: double[ndetscan] or NULL
 * for unit gain.  s_out float32[N].  FP32 arithmetic. */
tod_status tod_project(tod_plan *p, const void *map_tqu, const int32_t *pix,
                       const uint16_t *psi, const double *gain, float *s_out,
                       cudaStream_t stream);
/* tod_project in FP64: map double[3][npix] (rows T, Q, U, the layout of
 * tod_solve_maps), the same tabulated cos 2psi, sin 2psi values, s_out
 * double[N]; for the FP64 chi^2 and its finite-difference checks. */
tod_status tod_project_f64(tod_plan *p, const double *map, const int32_t *pix, const uint16_t *psi,
                           const double *gain, double *s_out, cudaStream_t stream);

/* A4 -- gain draw (the gain conditional of Eq. `gibbsstart`; n_corr marginalised, so
 * the full noise PSD weights the fit).  Per detscan, with shat = C(M s),
 * dhat = C(M d) the orthonormal DCT-II (the mirrored FFT of Sect. 4.2):
 *   a = sum_{k>=1} shat_k^2 / P_k,  b = sum_{k>=1} shat_k dhat_k / P_k,
 *   mu = b/a, sigma = a^(-1/2), g = mu + z sigma (z = 0 in TOD_MODE_MEAN).
 * d, s: float32[N] (s at unit gain).  Outputs double[ndetscan].
 * Transforms in FP32, sums in FP64. */
tod_status tod_sample_gain(tod_plan *p, const float *d, const float *s,
                           const uint32_t *flags, const double *psd, tod_rng rng,
                           int32_t mode, double *gain_out, double *mu_out,
                           double *sigma_out, cudaStream_t stream);

/* A5 -- correlated-noise draw with flagged samples inpainted (Eq.
 * `gibbsstart`, the n_corr conditional; Sect. 5: CG gap filling).  Per detscan,
 * r = d - g s and x solves
 *   (C^T diag(phi) C + M / sigma0^2) x = M r / sigma0^2 + M w1 / sigma0
 *                                        + C^T (sqrt(phi) w2),
 * phi_k = 1 / (sigma0^2 (f_k/f_knee)^alpha) for k >= 1, phi_0 = 0.
 * w1[t] is normal i(t) of the NC_W1 stream (i(t) = t/2 for even t,
 * n-1-(t-1)/2 for odd t); w2[k] is normal 2k (k < n/2), 2(n-k)+1 (k > n/2),
 * 0 (k = 0) or 1 (k = n/2) of the NC_W2 stream.  Gap-free detscans are solved
 * exactly in the DCT basis; flagged ones by conjugate gradients on the
 * flagged samples (Woodbury form; preconditioner: tod_plan_set_preconditioner),
 * stopping at relative residual cg_tol
 * (<= 0: 1e-6) or cg_maxiter (<= 0: 500) iterations (then
 * TOD_ERR_NOT_CONVERGED).  ncorr_out float32[N]; cg_iters_out int32[ndetscan]
 * or NULL. */
tod_status tod_sample_ncorr(tod_plan *p, const float *d, const float *s,
                            const double *gain, const uint32_t *flags,
                            const double *psd, tod_rng rng, int32_t mode,
                            double cg_tol, int32_t cg_maxiter,
                            float *ncorr_out, int32_t *cg_iters_out,
                            cudaStream_t stream);

/* tod_ncorr_prepare / tod_sample_ncorr_prepared -- tod_sample_ncorr in two
 * calls, so that the first can run on another stream while earlier stages
 * of the step run.  The paper has no counterpart (its preconditioning is
 * not described): a scheduling convenience.  tod_sample_ncorr is exactly
 * tod_ncorr_prepare followed by tod_sample_ncorr_prepared on one stream.
 *   tod_ncorr_prepare builds, from psd (double[ndet][3], device), the
 *   per-detector gap preconditioner tables the plan holds (the Toeplitz
 *   autocovariance of the CG operator at every lag of a power-of-two
 *   reference length, by one FFT per detector, its prefix sums for the
 *   coarse correction, and the Durbin solutions of its first 512 lags),
 *   overwriting the previous ones.
 *   tod_sample_ncorr_prepared is tod_sample_ncorr (same arguments, results
 *   and errors) using those tables; psd must be the array they were built
 *   from.
 * Ordering is the caller's: the prepared draw must be queued after the
 * preparation has completed (an event), and a new preparation only after
 * every draw that reads the old tables has completed.  Two plans do not
 * share tables. */
tod_status tod_ncorr_prepare(tod_plan *p, const double *psd, cudaStream_t stream);
tod_status tod_sample_ncorr_prepared(tod_plan *p, const float *d, const float *s,
                                     const double *gain, const uint32_t *flags,
                                     const double *psd, tod_rng rng, int32_t mode,
                                     double cg_tol, int32_t cg_maxiter,
                                     float *ncorr_out, int32_t *cg_iters_out,
                                     cudaStream_t stream);

/* tod_sample_ncorr_static -- tod_sample_ncorr with nothing allocated.
 * The paper has no counterpart: it is a library convenience.  Same
 * arguments, results and errors as tod_sample_ncorr, except that the draw's
 * working memory (the transforms' complex intermediate, the flag-word
 * prefix and the CG vectors) comes from one fixed device array compiled into
 * the library (TOD_NCORR_STATIC_SCRATCH_BYTES per device) instead of the
 * plan's buffers.  It is for callers that must not allocate device memory
 * once they run: a process whose free device memory is all held by another
 * allocator's pool (so a new allocation fails or forces that pool to
 * release), or a pipeline whose policy forbids allocation after start-up.
 *   Set-up: call tod_ncorr_static_setup once per device, with a plan of that
 *   device, on the host before the first draw and before any stream
 *   capture.  It looks up the array's device address (cudaGetSymbolAddress
 *   with the plan's device current) and caches it; that lookup is what
 *   loads the array's module and so backs the array with device memory
 *   (with CUDA_MODULE_LOADING=EAGER every process that loads the library
 *   backs it at context creation, used or not).  A draw on a device where
 *   set-up has not run returns TOD_ERR_ARG and enqueues nothing; the draw
 *   itself calls no allocating routine.  After a device reset (a new primary
 *   context) call set-up again: it always refreshes the cached address.
 *   Size: the draw takes the band in waves of consecutive detscans of at
 *   most *max_wave_samples_out samples (about 7.2 million: the intermediate
 *   takes 4 bytes per sample, the CG vectors 20 bytes per flagged sample
 *   for up to a quarter of the wave's samples), one cooperative launch per
 *   wave, so it is slower than tod_sample_ncorr.  Set-up and draw return
 *   TOD_ERR_SCRATCH (the draw enqueuing nothing) when a single detscan is
 *   longer than a wave; detscans of a wave whose flagged samples exceed the
 *   quarter are left at the gap-free solution with TOD_ERR_NOT_CONVERGED.
 *   Contents: every wave writes the parts of the array it reads, so no part
 *   has to start at zero.
 *   Concurrency: all plans and streams on one device share the array; two
 *   calls that can overlap on the device (different streams, or host
 *   threads without ordering) race on it and give wrong results.  Serialise
 *   them on one stream. */
#define TOD_NCORR_STATIC_SCRATCH_BYTES (64u << 20)
tod_status tod_ncorr_static_setup(tod_plan *p, int64_t *max_wave_samples_out);
tod_status tod_sample_ncorr_static(tod_plan *p, const float *d, const float *s,
                                   const double *gain, const uint32_t *flags,
                                   const double *psd, tod_rng rng, int32_t mode,
                                   double cg_tol, int32_t cg_maxiter,
                                   float *ncorr_out, int32_t *cg_iters_out,
                                   cudaStream_t stream);

/* A6 -- binning (Sect. 5 table, "TOD binning"; Sect. 2.4: coadded during
 * the pass over chunks).  With r'_t = d_t - ncorr_t, w_t = M_t / sigma0^2:
 *   A_p = sum_t w_t g_q^2 u_t u_t^T,  b_p = sum_t w_t g_q u_t r'_t,
 *   u_t = (1, cos 2psi_t, sin 2psi_t),  hits_p = sum_t M_t.
 * A_out double[npix][6] (TT,TQ,TU,QQ,QU,UU), b_out double[npix][3],
 * hits_out int32[npix]; all overwritten.  Deterministic: samples are summed
 * per (detscan, pixel) run of the pixel-sorted order fixed at plan
 * creation, runs in ascending detscan order, with products and partial sums
 * carried at FP64 accuracy. */
tod_status tod_bin(tod_plan *p, const uint16_t *psi, const float *d,
                   const float *ncorr, const double *gain, const uint32_t *flags,
                   const double *psd, double *A_out, double *b_out,
                   int32_t *hits_out, cudaStream_t stream);

/* A6 for a band split over several processes (Sect. 2.3-2.4: the TOD is
 * distributed in chunks, coadded locally, and the maps synchronised once
 * per sweep).  tod_bin_partial is tod_bin (same arguments) writing, per
 * pixel, the ten sums (A 6, b 3, hits) unrounded as double-double pairs
 * (hi, lo): part_out double[npix][20] (value i at [2i], [2i+1]).  tod_bin
 * itself adds a pixel's runs the same way and rounds once.
 * tod_combine_partials adds nparts such arrays of npix_range pixels
 * ([nparts][npix_range][20], DEVICE, consecutive by rank) in rank order, as
 * double-doubles, and rounds once into A_out [npix_range][6],
 * b_out [npix_range][3], hits_out [npix_range]: the normal equations of
 * contiguous scan ranges combined this way equal tod_bin of the whole band
 * bit for bit (but for sums within ~2^-104 of a rounding tie).  No
 * counterpart in the paper's arithmetic (its coaddition order is MPI's). */
tod_status tod_bin_partial(tod_plan *p, const uint16_t *psi, const float *d, const float *ncorr,
                           const double *gain, const uint32_t *flags, const double *psd, double *part_out,
                           cudaStream_t stream);
tod_status tod_combine_partials(const double *parts, int32_t nparts, int64_t npix_range, double *A_out,
                                double *b_out, int32_t *hits_out, cudaStream_t stream);
/* A7 on a range of npix_range pixels held by this process (the solve after
 * the reduction above): the arithmetic and validity rule of tod_solve_maps,
 * with every array of the range alone: A [npix_range][6], b [npix_range][3],
 * hits [npix_range] in; map_out double[3][npix_range], map_f32_out
 * float4[npix_range] or NULL, rcond_out, valid_out [npix_range] or NULL. */
tod_status tod_solve_range(int64_t npix_range, const double *A, const double *b, const int32_t *hits, double rcond_min,
                           double *map_out, void *map_f32_out, double *rcond_out, uint8_t *valid_out,
                           cudaStream_t stream);

/* A7 -- per-pixel solve (Sect. 5 table, "Map solution (Ax=b for each
 * pixel)"): m_p = A_p^{-1} b_p by FP64 3x3 Cholesky.  A pixel is valid iff
 * hits_p >= 3 and its Hadamard ratio det(A_p)/(A_TT A_QQ A_UU) >= rcond_min;
 * invalid pixels get m_p = 0.  map_out double[3][npix]; map_f32_out
 * float4[npix] (T,Q,U,0) or NULL (next step's projection input);
 * rcond_out double[npix] (the Hadamard ratio) or NULL; valid_out
 * uint8[npix] or NULL. */
tod_status tod_solve_maps(tod_plan *p, const double *A, const double *b,
                          const int32_t *hits, double rcond_min, double *map_out,
                          void *map_f32_out, double *rcond_out, uint8_t *valid_out,
                          cudaStream_t stream);

/* A8 -- TOD chi^2 with the correlated noise marginalised, and its
 * gradients (the likelihood of the gain conditional of Eq. `gibbsstart`,
 * as a function of map, gains and noise parameters).  Per detscan, with
 * rhat = C(M(d - g s)) and P_k the noise PSD:
 *   chi2_out[q]  = 1/2 sum_{k>=1} [ rhat_k^2 / P_k + ln P_k ],
 *   dgain_out[q] = dL/dg_q = -<M s, v>,
 *   v[t] = M_t (C^T(rhat/P))_t, so dL/ds = -g v and dL/dm = -P^T(g v)
 *          (tod_project_adjoint of v),
 * and for the band total_out[0] = sum_q chi2_out[q] and
 * dpsd_out[det][3] = dL/d(sigma0, f_knee, alpha) of the detector, summed
 * over its detscans in detscan order.  s is the unit-gain projection, float[N]
 * (tod_project) with TOD_PREC_F32, double[N] (tod_project_f64) with
 * TOD_PREC_F64.  precision: TOD_PREC_F32 (FP32 transforms) or TOD_PREC_F64
 * (FP64 transforms and per-mode terms); sums in FP64 either way.  v_out: float[N]
 * (F32) or double[N] (F64), or NULL.  Outputs device memory; chi2_out,
 * dgain_out double[ndetscan], total_out double[1], dpsd_out double[ndet][3]. */
#define TOD_PREC_F32 0
#define TOD_PREC_F64 1
tod_status tod_chi2(tod_plan *p, const float *d, const void *s, const double *gain,
                    const uint32_t *flags, const double *psd, int32_t precision,
                    double *chi2_out, double *dgain_out, double *total_out, double *dpsd_out,
                    void *v_out, cudaStream_t stream);

/* Adjoint of tod_project (the transpose of the g P m term of Eq. `todmodel`):
 *   out_p = sum over samples t of pixel p of g_q y_t (1, cos 2psi_t, sin 2psi_t),
 * out double[npix][3] (T, Q, U), overwritten.  y: float[N] (TOD_PREC_F32) or
 * double[N] (TOD_PREC_F64, summed to FP64 accuracy); every sample counts
 * (mask y first).  Deterministic, in the binning order of tod_bin. */
tod_status tod_project_adjoint(tod_plan *p, const uint16_t *psi, const void *y, int32_t precision,
                               const double *gain, double *out, cudaStream_t stream);

/* A10 -- noise PSD step (Sect. 5 lists it among the TOD steps; the paper
 * defers the sampler to its noise companion paper, so this is a reading):
 * with sigma0 held fixed, nsteps random-walk Metropolis steps on
 * (ln f_knee, alpha) of every detector, targeting
 *   ln L = -1/2 sum_{q of the detector} sum_{k>=1} [ xhat_{q,k}^2 / Pc_{q,k}
 *                                                    + ln Pc_{q,k} ],
 *   Pc_{q,k} = sigma0^2 (f_{q,k} / f_knee)^alpha,  f_{q,k} = k fsamp / (2 n_q),
 * (the Gaussian density of the n_corr draw xhat = C n_corr under its 1/f
 * prior, offset mode excluded) times a flat prior on the box
 * [TOD_PSD_LNFK_MIN, TOD_PSD_LNFK_MAX] x [TOD_PSD_ALPHA_MIN, TOD_PSD_ALPHA_MAX].
 * Step s proposes (ln f_knee + step_lnfknee z1, alpha + step_alpha z2) and
 * accepts iff the proposal is in the box and ln u < ln L(proposal) - ln L(current);
 * z1, z2, u come from Philox block (s, det, TOD_PURPOSE_PSD, iteration) with
 * key (seed, band): 53-bit uniforms of words 0 and 1 give the Box-Muller
 * pair (cos, sin), word 2 the uniform u.
 *   spec: float32[N] (device), each detscan's orthonormal DCT-II coefficients
 *   of its n_corr draw in mode order (spec[off_q + k] = xhat_{q,k}), as the
 *   n_corr draws write them once tod_plan_set_ncorr_spectrum is set.
 *   psd_in, psd_out: double[ndet][3] (sigma0, f_knee, alpha), device, distinct.
 *   accepted_out: int32[ndet] or NULL; loglike_out: double[ndet] (ln L of the
 *   final state) or NULL.  nsteps >= 0 (0: psd_out = psd_in).
 * ln L from FP32 products summed as FP32 double-words and FP64 per tile;
 * the decisions in FP64.  Deterministic.  The plan holds the chain's state:
 * calls on one plan must not overlap. */
#define TOD_PURPOSE_PSD 3
#define TOD_PURPOSE_GAIN_SMOOTH 4
#define TOD_PSD_LNFK_MIN (-9.2103403719761836)   /* ln 1e-4 (f_knee in Hz) */
#define TOD_PSD_LNFK_MAX 2.3025850929940457      /* ln 10 */
#define TOD_PSD_ALPHA_MIN (-4.0)
#define TOD_PSD_ALPHA_MAX (-0.25)
tod_status tod_sample_noise_psd(tod_plan *p, const float *spec, const double *psd_in, tod_rng rng,
                                int32_t nsteps, double step_lnfknee, double step_alpha,
                                double *psd_out, int32_t *accepted_out, double *loglike_out,
                                cudaStream_t stream);
/* The buffer (device float32[N], or NULL to stop) into which every
 * following n_corr draw of this plan (tod_sample_ncorr and its variants)
 * also writes the orthonormal DCT-II coefficients of its draw, in mode
 * order per detscan; no counterpart in the paper (it feeds A10). */
tod_status tod_plan_set_ncorr_spectrum(tod_plan *p, float *spec_out);

#ifdef __cplusplus
}
#endif
#endif /* TODGIBBS_H */
