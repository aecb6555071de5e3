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
constexpr int DEC_T = 512;            // decode threads per CTA (one checkpoint block each)
constexpr int DEC_ROUND = 16;         // symbols staged per thread before a coalesced write
// what a decoded value becomes: itself (pointing), the FP32 TOD, a flag bit
enum : int { DEC_VALUE = 0, DEC_TOD = 1, DEC_FLAG = 2 };
constexpr int ELEM_TILE = 4096;       // samples per tile of the element-wise kernels
constexpr int TOEP_LMAX = 512;        // longest gap block of the Toeplitz preconditioner
constexpr int BIN_TILE = 2048;        // sorted samples staged per binning tile

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

// ---------------------------------------------------------------------------
// Multi-pass batched DCT-II (k_tx.cu).  A length-n transform is an m = n/2
// complex FFT split m = m1 x m2: a column pass (FFTs of length m1 over
// tiles of column pairs {c, m2-1-c}, four-step twiddle, written row-major
// to an intermediate in memory), a row pass (FFTs of length m2 over tiles of
// row pairs {k1, m1-k1}, where the real split and any per-mode filter run,
// then the inverse row FFTs), and an inverse column pass.
// ---------------------------------------------------------------------------
constexpr int TX_T = 256;             // threads per CTA of the pass kernels
constexpr int TX_TILE = 4096;         // complex values per tile buffer (two buffers per CTA)
constexpr int TX_MAXR = 20;           // radix stages per sub-transform
constexpr int TX_GBMAX = 256;         // preconditioner gap blocks per detscan
constexpr int TX_GBCAP = 2048;        // padded preconditioner elements staged per round
// Coarse correction of the preconditioner (two-level, balancing form): two
// vectors per gap block (its indicator and its centred ramp); S Z kept for
// the TX_CZW neighbouring blocks on either side of each block.
constexpr int TX_CZW = 2;
constexpr int TX_CZB = 2 * TX_CZW + 1;            // half-bandwidth of E = Z^T S Z (scalar rows)
constexpr int TX_CZJ = 2 * (2 * TX_CZW + 1);      // S Z entries stored per flagged sample
constexpr int TX_CBMAX = 64;                      // most blocks of a detscan with the coarse correction

struct alignas(16) TxLen {
    int32_t n, m, m1, m2, m2p;        // m2p: row stride of a row tile (>= m2, chosen against bank conflicts)
    int32_t P1, P2;                   // row pairs m1/2 + 1, column pairs (m2 + 1)/2
    int32_t TP, TR;                   // column pairs per column tile, row pairs per row tile
    int32_t nr1, nr2;                 // radix stages of the column and row FFTs
    int16_t lgW, lgS;                 // log2 of the column tile's 2 TP columns and the row tile's 2 TR rows
    int64_t twb;                      // offset of this length's twiddle block
    FastDiv f_m2, f_W, f_2TR;         // divisions by m2, 2 TP, 2 TR
    int32_t pad1;
    double sq_fwd, s0_fwd, sq_inv, s0_inv;   // real-split scales
    DctStage s1[TX_MAXR], s2[TX_MAXR];
};

// Per-detscan state of the CG gap filling (device).
struct CgState {
    double rz, stop;                  // r.z, stopping threshold tol^2 |r0|^2
    int64_t koff;                     // first flagged rank of the detscan in the launch range
    int32_t K;                        // flagged samples
    int32_t it;                       // iterations done
    int32_t mode;                     // CG_* below
    int32_t ncz;                      // blocks of the coarse correction (0: one-level preconditioner)
};
enum : int32_t { CG_NONE = 0, CG_ACTIVE = 1, CG_DONE = 2, CG_ALLFLAG = 3, CG_OVER = 4 };

// Per-kernel timing (tod_plan_set_kernel_timing): while on, every launch of
// the plan's kernels is bracketed by two events on its stream, recorded with
// the kernel's class (TOD_KT_*); tod_plan_kernel_times adds them up.
struct KTimer {
    bool on = false;
    std::vector<cudaEvent_t> pool;   // created on demand, reused after a reset
    size_t used = 0;                 // events of the pool in use
    std::vector<int32_t> ids;        // class of record i, events pool[2i], pool[2i+1]
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
    // correlated-noise preconditioner (k_toeplitz.cu)
    float *htab = nullptr;           // [ndet][TOEP_LMAX] gap-kernel h(d)
    float *xtab = nullptr;           // [ndet][TOEP_LMAX (TOEP_LMAX+1)/2] T_L^{-1} e_1 per order
    int32_t *lvalid = nullptr;       // [ndet]
    // coarse correction: the kernel h(d) at every lag below cz_href (a power
    // of two >= the longest detscan), from one FFT of length 2 cz_href per
    // detector, and its prefix sums
    int32_t cz_href = 0;
    float2 *czfft = nullptr;         // [2][ndet][2 cz_href] FFT work
    float4 *cztab = nullptr;         // [ndet][cz_href + 1] (H, G) as FP32 pairs: H(x) = sum_{d<x} h(d), G: d h(d)
    int32_t *gbpos = nullptr;        // [nq][TX_GBMAX] first sample (within the detscan) of each block
    float *czsz = nullptr;           // [czcap][TX_CZJ] S Z entries by flagged rank
    int64_t czcap = 0;
    float *czl = nullptr;            // [nq][2 TX_CBMAX][TX_CZB + 1] banded Cholesky factor of E
    bool use_prec = true;            // gap-block inverses (TOD_PREC_BLOCKS)
    bool use_coarse = true;          // and the coarse correction (TOD_PREC_TWO_LEVEL)
    int32_t schedule = TOD_SCHED_PERSISTENT;
    int32_t nbin_tiles = 0;          // binning tiles (whole runs of one detscan)
    // noise PSD step
    float *spec_out = nullptr;       // caller's buffer for the n_corr spectra (NULL: not written)
    float2 *lnk = nullptr;           // [longest detscan] ln k as an FP32 pair (hi, lo)
    double *lnfs = nullptr;          // [nq] ln(fsamp / (2 n_q))
    double *psd_nmodes = nullptr;    // [ndet] modes k >= 1 of the detector's detscans
    double *psd_sumlnf = nullptr;    // [ndet] sum of ln f_k over them
    double *psd_part = nullptr;      // [ntile] partial sums of one evaluation
    double *psd_state = nullptr;     // [ndet][8] chain state
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
    // multi-pass transforms (k_tx.cu)
    int32_t ntx = 0;                 // distinct lengths
    TxLen *txl = nullptr;            // [ntx] device
    std::vector<TxLen> h_txl;
    int32_t *q_tx = nullptr;         // [nq] length index of each detscan
    std::vector<int32_t> h_q_tx;
    float2 *txtw = nullptr;          // twiddle blocks, FP32
    double2 *txtw64 = nullptr;       // the same, FP64
    int2 *colitems = nullptr, *rowitems = nullptr;   // (detscan, tile) work items, detscan-major
    int32_t *col_off = nullptr, *row_off = nullptr;  // [nq+1] first item of each detscan
    std::vector<int32_t> h_col_off, h_row_off;
    float2 *ybuf = nullptr;          // complex intermediate (FP64 calls use it as double2)
    int64_t ybuf_floats = 0;         // its size in floats: max(N, 2 x longest detscan)
    double *part = nullptr;          // [max items][4] per-item partial sums
    int64_t *wpre = nullptr;         // [N/32 + 3] flagged samples before each flag word (range-relative)
    int64_t *chunk = nullptr;        // [grid + 1] word-chunk counts of the flag scan
    CgState *cgs = nullptr;          // [nq]
    int2 *gblk = nullptr;            // [nq][TX_GBMAX] preconditioner blocks (rank in detscan, length)
    int32_t *gnb = nullptr;          // [nq] blocks (-1: too many, no preconditioner)
    float *cgv = nullptr;            // [5][cgcap] CG vectors y, r, p, q, z by flagged rank
    int64_t cgcap = 0;
    int32_t *cg_count = nullptr;     // [2] active detscans (alternating)
    int32_t *nclist = nullptr;       // [3 nq + 3] detscans of a CG pass with their item counts
    double *chi2_dpsd = nullptr;     // [nq][3] per-detscan PSD terms of the chi^2 gradient
    float4 *qsc = nullptr;           // [nq][2] per-detscan FP32 noise scalars of the current call
    int32_t coop_grid = 0;           // co-resident CTAs of the cooperative n_corr kernel
    int32_t pass_grid = 0;           // persistent grid of the other pass kernels
    int32_t tile_pairs = 0;          // requested column pairs per tile (0 = choose)
    int64_t device_bytes = 0;
    std::vector<void *> allocs;
    mutable KTimer kt;
};

// Brackets one launch on stream st with the class id's events while the
// plan's timing is on (a no-op otherwise).
class KScope {
public:
    KScope(const Plan &p, int32_t id, cudaStream_t st);
    ~KScope();
    KScope(const KScope &) = delete;
    KScope &operator=(const KScope &) = delete;
private:
    cudaStream_t st_;
    cudaEvent_t stop_ = nullptr;
};
#define TG_KT_CAT2(a, b) a##b
#define TG_KT_CAT(a, b) TG_KT_CAT2(a, b)
// the launch that follows in the same scope is timed as class id (needs p and st)
#define KTIME(id) ::tg::KScope TG_KT_CAT(kt_scope_, __LINE__)(p, (id), st)

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
cudaError_t launch_project64(const Plan &p, const double *map, const int32_t *pix, const uint16_t *psi,
                             const double *gain, double *s_out, cudaStream_t st);
// multi-pass transform stages (k_tx.cu)
struct TxNcorrScratch {
    float2 *Y;          // complex intermediate of the launch's detscans
    int64_t *wpre;      // flag-word prefix: (launch samples)/32 + 3 entries
    float *cgv;         // CG vectors, 5 x cgcap
    int64_t cgcap;      // flagged samples the vectors hold
};
cudaError_t setup_tx_kernels(Plan &p);
cudaError_t launch_tx_gain(const Plan &p, const float *d, const float *s, const uint32_t *flags, const double *psd,
                           tod_rng rng, int mode, double *g, double *mu, double *sig, cudaStream_t st, int q0, int q1);
// the draw over detscans [q0, q1): pass kernels with at most `grid` CTAs
// (at most p.pass_grid), the cooperative tail with at most p.coop_grid
cudaError_t launch_tx_ncorr(const Plan &p, const float *d, const float *s, const double *gain,
                            const uint32_t *flags, const double *psd, tod_rng rng, int mode, float tol, int maxit,
                            float *x, int32_t *iters, cudaStream_t st, int q0, int q1, const TxNcorrScratch &sc,
                            int grid);
cudaError_t launch_tx_chi2(const Plan &p, bool fp64, const float *d, const void *s, const double *gain,
                           const uint32_t *flags, const double *psd, double *chi2_q, double *dgain, double *dpsd_q,
                           double *total, double *dpsd_det, void *v_out, cudaStream_t st);
cudaError_t setup_bin_kernel(Plan &p);
cudaError_t launch_toeplitz_prep(const Plan &p, const double *psd, cudaStream_t st);
cudaError_t launch_noise_psd(const Plan &p, const float *spec, const double *psd_in, tod_rng rng, int nsteps,
                             double step_lnfk, double step_al, double *psd_out, int32_t *acc_out,
                             double *loglike_out, cudaStream_t st);
// with part non-null the per-pixel double-double pairs go there ([npix][20])
// instead of A, b, hits
cudaError_t launch_bin(const Plan &p, const uint16_t *psi, const float *d, const float *ncorr,
                       const double *gain, const uint32_t *flags, const double *psd, double *A,
                       double *b, int32_t *hits, double *part, cudaStream_t st);
cudaError_t launch_combine(const double *parts, int nparts, int64_t np, double *A, double *b, int32_t *hits,
                           cudaStream_t st);
// P^T (g y): out_p = sum over the samples of pixel p of g_q y_t (1, cos 2psi, sin 2psi)
cudaError_t launch_project_adjoint(const Plan &p, const uint16_t *psi, const void *y, bool fp64, const double *gain,
                                   double *out, cudaStream_t st);
// the solve of npix pixels (map as [3][npix], outputs indexed like the inputs)
cudaError_t launch_solve_n(int64_t npix, const double *A, const double *b, const int32_t *hits, double rcond_min,
                           double *map, float4 *map32, double *rcond, uint8_t *valid, cudaStream_t st);
cudaError_t launch_solve(const Plan &p, const double *A, const double *b, const int32_t *hits,
                         double rcond_min, double *map, float4 *map32, double *rcond,
                         uint8_t *valid, cudaStream_t st);

}  // namespace tg
