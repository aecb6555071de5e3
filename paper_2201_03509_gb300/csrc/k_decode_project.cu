// A1 Huffman decode (paper Sect. 4.1) and A2 projection (Eq. `todmodel`).
//
// Decode: every checkpoint block (TOD_CKPT_BLOCK symbols of one detscan) is
// decoded by one thread, starting from the block's bit offset and the value
// preceding it, so a band's ~10^6 blocks decode in parallel.  One CTA takes
// up to DEC_T consecutive blocks of one scan and stages that scan's code
// (a 2^DEC_LUTB-entry first-level table, per-length limits for the long
// codes) in shared memory; the rare long codes read their symbol through
// the cache.  Each thread's decode is one long dependency chain, so the
// CTA is large (the table is staged once for more threads) and three fit
// on an SM.  Values are undone
// from their differences on the fly and staged DEC_ROUND at a time per
// thread in shared memory, then written with coalesced stores.
//
// The same decoder serves the TOD and quality-flag streams (Sect. 4.1:
// the ADC integers and flag words are differenced and coded like the
// pointing; Listing `tod`: tod and flag held as compressed bytes).  What a
// decoded value becomes is the kernel's KIND: the value itself (pointing),
// the FP32 TOD d = fl32(scale_q * count) (one FP64 product, one rounding),
// or the flag bit (word & select) != 0, packed into the sample bitmask with
// one warp vote and at most two atomic ORs per DEC_ROUND samples.
#include <type_traits>

#include "common.cuh"
#include "internal.cuh"

namespace tg {

static_assert(DEC_ROUND == 16, "the flag packing takes two runs of 16 samples per warp");

template <typename OutT, int KIND>
__global__ void __launch_bounds__(DEC_T)
k_decode(const uint32_t *__restrict__ words, const int64_t *__restrict__ word_off,
         const int64_t *__restrict__ nbits, const int64_t *__restrict__ blk_off,
         const uint32_t *__restrict__ ckpt_bit, const int32_t *__restrict__ ckpt_val,
         const int32_t *__restrict__ blk_q, const int32_t *__restrict__ lut,
         const unsigned long long *__restrict__ lim_g, const int32_t *__restrict__ base_g,
         const int32_t *__restrict__ canon_off, const int32_t *__restrict__ canon_vals,
         const int32_t *__restrict__ cta_scan, const int64_t *__restrict__ cta_blk0,
         const int32_t *__restrict__ cta_nblk, const int64_t *__restrict__ off,
         const double *__restrict__ scale, uint32_t select, OutT *__restrict__ out, int32_t *status)
{
    using StageT = typename std::conditional<KIND == DEC_FLAG, uint8_t, OutT>::type;
    extern __shared__ int32_t s_lut[];                     // [1 << DEC_LUTB]
    __shared__ unsigned long long s_lim[26];
    __shared__ int32_t s_base[26];
    __shared__ StageT s_tile[DEC_T][DEC_ROUND + 1];
    __shared__ int64_t s_out0[DEC_T];
    __shared__ int32_t s_cnt[DEC_T];

    const int tid = threadIdx.x;
    const int scan = cta_scan[blockIdx.x];
    const int64_t b0 = cta_blk0[blockIdx.x];
    const int nb = cta_nblk[blockIdx.x];

    for (int i = tid; i < (1 << DEC_LUTB); i += DEC_T) s_lut[i] = lut[(int64_t)scan * (1 << DEC_LUTB) + i];
    if (tid < 26) { s_lim[tid] = lim_g[scan * 26 + tid]; s_base[tid] = base_g[scan * 26 + tid]; }
    // symbols of long codes (longer than DEC_LUTB bits: rare) through the cache
    const int c0 = canon_off[scan], nc = canon_off[scan + 1] - c0;

    // this thread's block
    const bool active = tid < nb;
    int q = 0, cnt = 0;
    int64_t pos = 0, end = 0, wptr = 0;
    int32_t x = 0;
    double sc = 0.0;                    // DEC_TOD: the detscan's ADC quantum
    unsigned long long buf = 0;
    int have = 0;                       // valid bits in buf (left-aligned)
    bool ok = true;
    if (active) {
        const int64_t b = b0 + tid;
        q = blk_q[b];
        const int64_t j = b - blk_off[q];
        const int64_t n = off[q + 1] - off[q];
        cnt = static_cast<int>((n - j * TOD_CKPT_BLOCK < TOD_CKPT_BLOCK ? n - j * TOD_CKPT_BLOCK : TOD_CKPT_BLOCK));
        s_out0[tid] = off[q] + j * TOD_CKPT_BLOCK;
        s_cnt[tid] = cnt;
        const int64_t w0 = word_off[q];
        pos = w0 * 32 + ckpt_bit[b];
        end = w0 * 32 + nbits[q];
        x = ckpt_val[b];
        if constexpr (KIND == DEC_TOD) sc = scale[q];
        wptr = pos >> 5;
        const int sh = static_cast<int>(pos & 31);
        buf = ((static_cast<unsigned long long>(words[wptr]) << 32) | words[wptr + 1]) << sh;
        have = 64 - sh;
        wptr += 2;
    } else {
        s_cnt[tid] = 0;
        s_out0[tid] = 0;
    }
    __syncthreads();

    for (int round = 0; round < TOD_CKPT_BLOCK / DEC_ROUND; ++round) {
#pragma unroll 4
        for (int i = 0; i < DEC_ROUND; ++i) {
            const int idx = round * DEC_ROUND + i;
            if (active && ok && idx < cnt) {
                const uint32_t peek = static_cast<uint32_t>(buf >> 32);
                const int32_t e = s_lut[peek >> (32 - DEC_LUTB)];
                int len = e & 31;
                int32_t v = e >> 5;
                if (len == 0 || v == DEC_WIDE) {
                    // a code longer than the table (its length found from the
                    // canonical limits above DEC_LUTB), or a value too wide for
                    // the packed entry (length known)
                    int L = len;
                    if (len == 0) {
                        L = DEC_LUTB + 1;
                        while (L <= TOD_HUFF_MAXLEN && static_cast<unsigned long long>(peek) >= s_lim[L]) ++L;
                    }
                    if (L > TOD_HUFF_MAXLEN) { ok = false; len = 1; v = 0; }
                    else {
                        const int ci = s_base[L] + static_cast<int>(peek >> (32 - L));
                        if (ci < 0 || ci >= nc) { ok = false; v = 0; }
                        else v = __ldg(canon_vals + c0 + ci);
                        len = L;
                    }
                }
                x += v;
                buf <<= len;
                have -= len;
                pos += len;
                if (pos > end) ok = false;       // never read past the stream (+pad)
                if (ok && have < 32) {
                    buf |= static_cast<unsigned long long>(words[wptr]) << (32 - have);
                    ++wptr;
                    have += 32;
                }
                if constexpr (KIND == DEC_TOD)
                    s_tile[tid][i] = __double2float_rn(static_cast<double>(x) * sc);
                else if constexpr (KIND == DEC_FLAG)
                    s_tile[tid][i] = (static_cast<uint32_t>(x) & select) != 0u;
                else
                    s_tile[tid][i] = static_cast<OutT>(x);
            }
        }
        __syncthreads();
        // coalesced write-out: consecutive threads take consecutive values of a block
        for (int e = tid; e < DEC_T * DEC_ROUND; e += DEC_T) {
            const int bl = e / DEC_ROUND, i = e % DEC_ROUND;
            const int idx = round * DEC_ROUND + i;
            if constexpr (KIND == DEC_FLAG) {
                // lanes 0-15 and 16-31 each hold DEC_ROUND consecutive samples
                // of one block; their flagged bits are ORed into the bitmask
                // (bit t & 31 of word t >> 5; the words start zeroed)
                const uint32_t vote =
                    __ballot_sync(0xffffffffu, idx < s_cnt[bl] && s_tile[bl][i] != 0);
                const uint32_t mine = (vote >> (tid & 31 & ~(DEC_ROUND - 1))) & 0xffffu;
                if (i == 0 && mine) {
                    const int64_t g0 = s_out0[bl] + round * DEC_ROUND;
                    const unsigned long long v = static_cast<unsigned long long>(mine) << (g0 & 31);
                    atomicOr(out + (g0 >> 5), static_cast<uint32_t>(v));
                    if (v >> 32) atomicOr(out + (g0 >> 5) + 1, static_cast<uint32_t>(v >> 32));
                }
            } else {
                if (idx < s_cnt[bl]) out[s_out0[bl] + idx] = s_tile[bl][i];
            }
        }
        __syncthreads();
    }
    if (active && (!ok || pos > end)) set_status(status, q, TOD_ERR_CORRUPT_STREAM);
}

cudaError_t setup_decode_kernel()
{
    const int smem = static_cast<int>(sizeof(int32_t) * (1 << DEC_LUTB));
    cudaError_t e = cudaFuncSetAttribute(k_decode<int32_t, DEC_VALUE>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_decode<uint16_t, DEC_VALUE>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_decode<float, DEC_TOD>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_decode<uint32_t, DEC_FLAG>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    return e;
}

namespace {

template <int KIND> constexpr int32_t kind_id() {
    return KIND == DEC_TOD ? TOD_KT_DECODE_TOD : KIND == DEC_FLAG ? TOD_KT_DECODE_FLAGS : TOD_KT_DECODE;
}

template <typename OutT, int KIND>
cudaError_t decode_into(const Plan &p, const HuffDev &h, const double *scale, uint32_t select, OutT *out,
                        cudaStream_t st)
{
    if (h.ncta == 0) return cudaSuccess;
    const size_t smem = sizeof(int32_t) * (1 << DEC_LUTB);
    {
        KTIME(kind_id<KIND>());
        k_decode<OutT, KIND><<<h.ncta, DEC_T, smem, st>>>(
            h.words, h.word_off, h.nbits, h.blk_off, h.ckpt_bit, h.ckpt_val, h.blk_q, h.lut, h.lim, h.base,
            h.canon_off, h.canon_vals, h.cta_scan, h.cta_blk0, h.cta_nblk, p.off, scale, select, out, p.status);
    }
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_decode(const Plan &p, const HuffDev &h, int32_t *pix_out, uint16_t *psi_out,
                          cudaStream_t st)
{
    if (pix_out) return decode_into<int32_t, DEC_VALUE>(p, h, nullptr, 0u, pix_out, st);
    return decode_into<uint16_t, DEC_VALUE>(p, h, nullptr, 0u, psi_out, st);
}

cudaError_t launch_decode_tod(const Plan &p, float *d_out, cudaStream_t st)
{
    return decode_into<float, DEC_TOD>(p, p.htod, p.tod_scale, 0u, d_out, st);
}

cudaError_t launch_decode_flags(const Plan &p, uint32_t *flags_out, cudaStream_t st)
{
    cudaError_t e = cudaMemsetAsync(flags_out, 0, sizeof(uint32_t) * ((p.N + 31) / 32), st);
    if (e != cudaSuccess) return e;
    return decode_into<uint32_t, DEC_FLAG>(p, p.hflag, nullptr, p.flag_select, flags_out, st);
}

// ---------------------------------------------------------------------------
// A2 projection: one 16-byte map gather per sample, psi angle from the FP32
// table (L1-resident), gain per detscan.  Tiles of ELEM_TILE samples never
// cross a detscan.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256)
k_project(const float4 *__restrict__ map, const int32_t *__restrict__ pix,
          const uint16_t *__restrict__ psi, const double *__restrict__ gain,
          const float2 *__restrict__ trig, const int32_t *__restrict__ tile_q,
          const int64_t *__restrict__ tile_t0, const int64_t *__restrict__ off,
          int32_t npix, float *__restrict__ s_out, int32_t *status)
{
    const int q = tile_q[blockIdx.x];
    const int64_t t0 = tile_t0[blockIdx.x];
    const int64_t t1 = (t0 + ELEM_TILE < off[q + 1]) ? t0 + ELEM_TILE : off[q + 1];
    const float g = gain ? static_cast<float>(gain[q]) : 1.0f;
    for (int64_t t = t0 + threadIdx.x; t < t1; t += blockDim.x) {
        const int32_t pp = pix[t];
        const uint32_t b = psi[t];
        if (static_cast<uint32_t>(pp) >= static_cast<uint32_t>(npix) || b >= TOD_N_PSI) {
            set_status(status, q, TOD_ERR_ARG);      // out-of-range pointing: no gather
            s_out[t] = 0.0f;
            continue;
        }
        const float4 m = __ldg(map + pp);
        const float2 cs = __ldg(trig + b);
        s_out[t] = g * fmaf(m.z, cs.y, fmaf(m.y, cs.x, m.x));
    }
}

// The same in FP64: map double[3][npix] (rows T, Q, U), the FP32 table
// values read as FP64, s in FP64.
__global__ void __launch_bounds__(256)
k_project64(const double *__restrict__ map, const int32_t *__restrict__ pix,
            const uint16_t *__restrict__ psi, const double *__restrict__ gain,
            const float2 *__restrict__ trig, const int32_t *__restrict__ tile_q,
            const int64_t *__restrict__ tile_t0, const int64_t *__restrict__ off,
            int32_t npix, double *__restrict__ s_out, int32_t *status)
{
    const int q = tile_q[blockIdx.x];
    const int64_t t0 = tile_t0[blockIdx.x];
    const int64_t t1 = (t0 + ELEM_TILE < off[q + 1]) ? t0 + ELEM_TILE : off[q + 1];
    const double g = gain ? gain[q] : 1.0;
    for (int64_t t = t0 + threadIdx.x; t < t1; t += blockDim.x) {
        const int32_t pp = pix[t];
        const uint32_t b = psi[t];
        if (static_cast<uint32_t>(pp) >= static_cast<uint32_t>(npix) || b >= TOD_N_PSI) {
            set_status(status, q, TOD_ERR_ARG);
            s_out[t] = 0.0;
            continue;
        }
        const float2 cs = __ldg(trig + b);
        const double T = __ldg(map + pp), Q = __ldg(map + npix + pp), U = __ldg(map + 2 * static_cast<int64_t>(npix) + pp);
        s_out[t] = g * (T + Q * static_cast<double>(cs.x) + U * static_cast<double>(cs.y));
    }
}

cudaError_t launch_project64(const Plan &p, const double *map, const int32_t *pix, const uint16_t *psi,
                             const double *gain, double *s_out, cudaStream_t st)
{
    if (p.ntile == 0) return cudaSuccess;
    {
        KTIME(TOD_KT_PROJECT64);
        k_project64<<<p.ntile, 256, 0, st>>>(map, pix, psi, gain, p.trig, p.tile_q, p.tile_t0, p.off, p.npix,
                                             s_out, p.status);
    }
    return cudaGetLastError();
}

// One sample of the projection (out-of-range pointing: status, zero).
__device__ __forceinline__ float project_one(const float4 *__restrict__ map, const float2 *__restrict__ trig,
                                             int32_t pp, uint32_t b, int32_t npix, float g, int32_t *status, int q)
{
    if (static_cast<uint32_t>(pp) >= static_cast<uint32_t>(npix) || b >= TOD_N_PSI) {
        set_status(status, q, TOD_ERR_ARG);
        return 0.0f;
    }
    const float4 m = __ldg(map + pp);
    const float2 cs = __ldg(trig + b);
    return g * fmaf(m.z, cs.y, fmaf(m.y, cs.x, m.x));
}

// The same, four samples per thread: 16-byte pixel loads, 8-byte angle
// loads and 16-byte stores on the tile's aligned body (global sample index a
// multiple of 4; the caller checks the base pointers), its up to three head
// and tail samples one per thread.  Four map gathers in flight per thread.
__global__ void __launch_bounds__(256)
k_project4(const float4 *__restrict__ map, const int32_t *__restrict__ pix,
           const uint16_t *__restrict__ psi, const double *__restrict__ gain,
           const float2 *__restrict__ trig, const int32_t *__restrict__ tile_q,
           const int64_t *__restrict__ tile_t0, const int64_t *__restrict__ off,
           int32_t npix, float *__restrict__ s_out, int32_t *status)
{
    const int q = tile_q[blockIdx.x];
    const int64_t t0 = tile_t0[blockIdx.x];
    const int64_t t1 = (t0 + ELEM_TILE < off[q + 1]) ? t0 + ELEM_TILE : off[q + 1];
    const float g = gain ? static_cast<float>(gain[q]) : 1.0f;
    const int64_t a0 = min(t1, (t0 + 3) & ~static_cast<int64_t>(3));
    const int64_t a1 = max(a0, t1 & ~static_cast<int64_t>(3));
    if (threadIdx.x < a0 - t0) {
        const int64_t t = t0 + threadIdx.x;
        s_out[t] = project_one(map, trig, pix[t], psi[t], npix, g, status, q);
    }
    if (threadIdx.x < t1 - a1) {
        const int64_t t = a1 + threadIdx.x;
        s_out[t] = project_one(map, trig, pix[t], psi[t], npix, g, status, q);
    }
    for (int64_t t = a0 + 4 * static_cast<int64_t>(threadIdx.x); t < a1; t += 4 * blockDim.x) {
        const int4 p4 = *reinterpret_cast<const int4 *>(pix + t);
        const uint2 b4 = *reinterpret_cast<const uint2 *>(psi + t);
        float4 o;
        o.x = project_one(map, trig, p4.x, b4.x & 0xFFFFu, npix, g, status, q);
        o.y = project_one(map, trig, p4.y, b4.x >> 16, npix, g, status, q);
        o.z = project_one(map, trig, p4.z, b4.y & 0xFFFFu, npix, g, status, q);
        o.w = project_one(map, trig, p4.w, b4.y >> 16, npix, g, status, q);
        *reinterpret_cast<float4 *>(s_out + t) = o;
    }
}

cudaError_t launch_project(const Plan &p, const float4 *map, const int32_t *pix, const uint16_t *psi,
                           const double *gain, float *s_out, cudaStream_t st)
{
    if (p.ntile == 0) return cudaSuccess;
    const bool vec = (reinterpret_cast<uintptr_t>(pix) & 15u) == 0 && (reinterpret_cast<uintptr_t>(psi) & 7u) == 0 &&
                     (reinterpret_cast<uintptr_t>(s_out) & 15u) == 0;
    {
        KTIME(TOD_KT_PROJECT);
        if (vec)
            k_project4<<<p.ntile, 256, 0, st>>>(map, pix, psi, gain, p.trig, p.tile_q, p.tile_t0, p.off, p.npix,
                                                s_out, p.status);
        else
            k_project<<<p.ntile, 256, 0, st>>>(map, pix, psi, gain, p.trig, p.tile_q, p.tile_t0, p.off, p.npix,
                                               s_out, p.status);
    }
    return cudaGetLastError();
}

}  // namespace tg
