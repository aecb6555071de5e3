// C ABI of libtodgibbs: ingest (FFT lengths, Huffman encoding), plan
// construction (the band's TOD object) and the six step entry points.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <functional>
#include <map>
#include <mutex>
#include <new>
#include <numeric>
#include <thread>
#include <vector>

#include "internal.cuh"

using namespace tg;

namespace tg {

KScope::KScope(const Plan &p, int32_t id, cudaStream_t st) : st_(st)
{
    KTimer &k = p.kt;
    if (!k.on) return;
    while (k.pool.size() < k.used + 2) {
        cudaEvent_t ev = nullptr;
        if (cudaEventCreate(&ev) != cudaSuccess) return;     // untimed, never an error of the launch
        k.pool.push_back(ev);
    }
    cudaEvent_t start = k.pool[k.used];
    stop_ = k.pool[k.used + 1];
    k.used += 2;
    k.ids.push_back(id);
    cudaEventRecord(start, st_);
}

KScope::~KScope()
{
    if (stop_) cudaEventRecord(stop_, st_);
}

}  // namespace tg

namespace {

constexpr double kPi = 3.14159265358979323846;

// ---------------------------------------------------------------------------
// host helpers
// ---------------------------------------------------------------------------
void parallel_for(int64_t n, const std::function<void(int64_t, int64_t)> &f)
{
    unsigned hw = std::thread::hardware_concurrency();
    int64_t nt = std::max<int64_t>(1, std::min<int64_t>(hw ? hw : 4, 64));
    nt = std::min<int64_t>(nt, std::max<int64_t>(1, n));
    if (nt <= 1) { f(0, n); return; }
    std::vector<std::thread> th;
    std::atomic<int64_t> next(0);
    const int64_t grain = std::max<int64_t>(1, n / (nt * 8));
    for (int64_t i = 0; i < nt; ++i)
        th.emplace_back([&]() {
            for (;;) {
                const int64_t a = next.fetch_add(grain);
                if (a >= n) break;
                f(a, std::min(n, a + grain));
            }
        });
    for (auto &t : th) t.join();
}

// Code lengths of symbols (ascending value) from counts: two-queue Huffman
// merge over leaves ordered by (count, value), a leaf winning ties against a
// merged node; lengths over TOD_HUFF_MAXLEN halve every count ((c+1)/2) and
// rebuild.  The format (and so these rules) is shared with every reader of
// the streams.
std::vector<uint8_t> huffman_lengths(const std::vector<int64_t> &counts_in)
{
    const size_t k = counts_in.size();
    std::vector<uint8_t> len(k, 0);
    if (k == 1) { len[0] = 1; return len; }
    std::vector<int64_t> cnt(counts_in);
    for (auto &c : cnt) c = std::max<int64_t>(c, 1);
    for (;;) {
        std::vector<uint32_t> order(k);
        std::iota(order.begin(), order.end(), 0u);
        std::stable_sort(order.begin(), order.end(),
                         [&](uint32_t a, uint32_t b) { return cnt[a] < cnt[b]; });
        // node weights: [0,k) leaves in 'order', [k, 2k-1) merged nodes
        std::vector<int64_t> wt(2 * k - 1);
        std::vector<int32_t> up(2 * k - 1, -1);
        for (size_t i = 0; i < k; ++i) wt[i] = cnt[order[i]];
        size_t leaf = 0, mhead = k, mtail = k;
        auto pop = [&]() -> size_t {
            const bool use_leaf = leaf < k && (mhead == mtail || wt[leaf] <= wt[mhead]);
            return use_leaf ? leaf++ : mhead++;
        };
        while (mtail < 2 * k - 1) {
            const size_t a = pop(), b = pop();
            wt[mtail] = wt[a] + wt[b];
            up[a] = static_cast<int32_t>(mtail);
            up[b] = static_cast<int32_t>(mtail);
            ++mtail;
        }
        // depths top-down: a parent is always created after its children
        std::vector<int32_t> depth(2 * k - 1, 0);
        for (size_t i = 2 * k - 2; i-- > 0;) depth[i] = depth[up[i]] + 1;
        int maxd = 0;
        for (size_t i = 0; i < k; ++i) {
            len[order[i]] = static_cast<uint8_t>(std::min(depth[i], 255));
            maxd = std::max(maxd, depth[i]);
        }
        if (maxd <= TOD_HUFF_MAXLEN) break;
        for (auto &c : cnt) c = (c + 1) / 2;
    }
    return len;
}

// Canonical code words: ordered by (length, value), consecutive, shifted at
// each length increase.
std::vector<uint32_t> canonical_codes(const std::vector<uint8_t> &len)
{
    const size_t k = len.size();
    std::vector<uint32_t> idx(k), code(k, 0);
    std::iota(idx.begin(), idx.end(), 0u);
    std::stable_sort(idx.begin(), idx.end(), [&](uint32_t a, uint32_t b) { return len[a] < len[b]; });
    uint32_t c = 0;
    for (size_t i = 0; i < k; ++i) {
        if (i) c = (c + 1) << (len[idx[i]] - len[idx[i - 1]]);
        code[idx[i]] = c;
    }
    return code;
}

// A first-level decode entry in 32 bits: value << 5 | code length.  A value
// outside (DEC_WIDE, 2^26) is stored as DEC_WIDE with its length (the decoder
// reads the symbol from the canonical list); an entry 0 (length 0) means a
// code longer than DEC_LUTB bits, found from the canonical limits.
int32_t dec_lut_entry(int32_t value, int L)
{
    if (value <= DEC_WIDE || value >= (1 << 26)) value = DEC_WIDE;     // symbol read canonically, length known
    return static_cast<int32_t>((static_cast<uint32_t>(value) << 5) | static_cast<uint32_t>(L));
}

// canonical decode tables of one code (symbols ascending with lengths)
struct DecTab {
    std::vector<int32_t> lut;               // 1 << DEC_LUTB packed entries (see dec_lut_entry)
    unsigned long long lim[26];
    int32_t base[26];
    std::vector<int32_t> canon;
};

DecTab build_dectab(const int32_t *vals, const uint8_t *len, int64_t k)
{
    DecTab t;
    std::vector<int64_t> count(33, 0);
    for (int64_t i = 0; i < k; ++i) count[len[i]]++;
    // canonical order
    std::vector<int64_t> idx(k);
    std::iota(idx.begin(), idx.end(), 0);
    std::stable_sort(idx.begin(), idx.end(), [&](int64_t a, int64_t b) { return len[a] < len[b]; });
    t.canon.resize(k);
    for (int64_t i = 0; i < k; ++i) t.canon[i] = vals[idx[i]];
    uint64_t first = 0;
    int64_t index = 0;
    for (int L = 0; L < 26; ++L) { t.lim[L] = 0; t.base[L] = 0; }
    for (int L = 1; L <= TOD_HUFF_MAXLEN; ++L) {
        if (L > 1) first = (first + count[L - 1]) << 1;
        t.base[L] = static_cast<int32_t>(index - static_cast<int64_t>(first));
        t.lim[L] = (first + count[L]) << (32 - L);
        index += count[L];
    }
    t.lim[25] = ~0ull;
    t.lut.assign(1 << DEC_LUTB, 0);
    for (uint32_t v = 0; v < (1u << DEC_LUTB); ++v) {
        const uint64_t peek = static_cast<uint64_t>(v) << (32 - DEC_LUTB);
        for (int L = 1; L <= DEC_LUTB; ++L) {
            if (peek < t.lim[L]) {
                const int64_t ci = t.base[L] + static_cast<int64_t>(peek >> (32 - L));
                if (ci >= 0 && ci < k) t.lut[v] = dec_lut_entry(t.canon[ci], L);
                break;
            }
        }
    }
    return t;
}

// decode one detscan on the host (plan construction only)
bool host_decode(const tod_huff_streams &h, const DecTab &t, int64_t q, int64_t n, int32_t *out)
{
    const int64_t w0 = h.word_off[q], w1 = h.word_off[q + 1];
    const int64_t nb = h.nbits[q];
    int64_t pos = 0;
    int32_t x = 0;
    auto bit_window = [&](int64_t p) -> uint32_t {   // 32 bits starting at p (zero past the end)
        const int64_t w = p >> 5;
        const int sh = static_cast<int>(p & 31);
        const uint64_t a = (w0 + w < w1) ? h.words[w0 + w] : 0u;
        const uint64_t b = (w0 + w + 1 < w1) ? h.words[w0 + w + 1] : 0u;
        return static_cast<uint32_t>((((a << 32) | b) << sh) >> 32);
    };
    const int64_t k = static_cast<int64_t>(t.canon.size());
    for (int64_t i = 0; i < n; ++i) {
        const uint32_t peek = bit_window(pos);
        int L = 1;
        while (L <= TOD_HUFF_MAXLEN && static_cast<uint64_t>(peek) >= t.lim[L]) ++L;
        if (L > TOD_HUFF_MAXLEN) return false;
        const int64_t ci = t.base[L] + static_cast<int64_t>(peek >> (32 - L));
        if (ci < 0 || ci >= k) return false;
        x += t.canon[ci];
        out[i] = x;
        pos += L;
        if (pos > nb) return false;
    }
    return pos == nb;
}

template <class T>
cudaError_t dev_upload(Plan &p, T *&dst, const T *src, size_t count)
{
    dst = nullptr;
    if (count == 0) count = 1;
    cudaError_t e = cudaMalloc(reinterpret_cast<void **>(&dst), count * sizeof(T));
    if (e != cudaSuccess) return e;
    p.allocs.push_back(dst);
    p.device_bytes += static_cast<int64_t>(count * sizeof(T));
    if (src) return cudaMemcpy(dst, src, count * sizeof(T), cudaMemcpyHostToDevice);
    return cudaMemset(dst, 0, count * sizeof(T));
}

void free_plan(Plan *p)
{
    if (!p) return;
    int cur = 0;
    cudaGetDevice(&cur);
    cudaSetDevice(p->device);
    for (void *a : p->allocs) cudaFree(a);
    for (cudaEvent_t ev : p->kt.pool) cudaEventDestroy(ev);
    cudaSetDevice(cur);
    delete p;
}

int64_t fft_length_impl(int64_t n)
{
    if (n < 2) return 0;
    int64_t best = 0;
    for (int64_t a = 2; a <= n; a *= 2)
        for (int64_t b = a; b <= n; b *= 3)
            for (int64_t c = b; c <= n; c *= 5) best = std::max(best, c);
    return best;
}

// Stockham radices of a sub-transform of length L: repeatedly the largest
// register DFT up to rmax (16, 10, 9, 8, 6, 5, 4, 3, 2) that divides what is
// left (empty for L = 1).  A thread of the in-place passes holds the inputs
// of ceil(16/R) butterflies: at most 20 values with these radices.
std::vector<int8_t> radix_plan(int L, int rmax)
{
    static const int kRadix[] = {16, 10, 9, 8, 6, 5, 4, 3, 2};
    std::vector<int8_t> r;
    while (L > 1) {
        int pick = 0;
        for (int R : kRadix)
            if (R <= rmax && L % R == 0) { pick = R; break; }
        if (!pick) { r.clear(); return r; }
        r.push_back(static_cast<int8_t>(pick));
        L /= pick;
    }
    std::reverse(r.begin(), r.end());
    return r;
}

void fill_stages(DctStage *st, const std::vector<int8_t> &r, int L)
{
    int Ns = 1;
    for (size_t i = 0; i < r.size(); ++i) {
        st[i].R = r[i];
        st[i].Ns = Ns;
        st[i].fLR = make_fastdiv(static_cast<uint32_t>(L / r[i]));
        st[i].fNs = make_fastdiv(static_cast<uint32_t>(Ns));
        Ns *= r[i];
    }
}

// Column pairs per column tile: the largest power of two (at most 64, so
// that the 2 TP columns divide the CTA's threads) with 2 TP m1 <= TX_TILE,
// capped by tile_pairs when given.
int tile_width(int P2, int m1, int tile_pairs)
{
    int cap = std::min(64, TX_TILE / (2 * m1));
    if (tile_pairs > 0) cap = std::min(cap, tile_pairs);
    int tp = 1;
    while (2 * tp <= cap && tp < P2) tp *= 2;
    return tp;
}

// Shared-memory bank conflicts of the row FFTs of a row tile with nslot
// rows at stride m2p: butterfly w of a Stockham pass (radix R after Ns
// points) works on row w mod nslot, index j = w / nslot, reading elements
// j + r L/R and writing (j / Ns) Ns R + j mod Ns + r Ns.  Returned: the mean
// number of extra 8-byte wavefronts per half-warp access, over the first
// eight warps' first two reads and writes of every pass.
double row_bank_cost(int m2, int m2p, int nslot, const std::vector<int8_t> &radices)
{
    int Ns = 1;
    double extra = 0.0;
    int count = 0;
    for (int R : radices) {
        const int LR = m2 / R, total = nslot * LR;
        for (int w0 = 0; w0 < std::min(total, TX_T); w0 += 32)
            for (int half = 0; half < 32; half += 16)
                for (int rd = 0; rd < 2; ++rd)
                    for (int r = 0; r < 2; ++r) {
                        int hits[16] = {0};
                        int used = 0, worst = 0;
                        for (int i = 0; i < 16; ++i) {
                            const int w = w0 + half + i;
                            if (w >= total) break;
                            const int j = w / nslot, vec = w - j * nslot;
                            int e;
                            if (rd) e = j + r * LR;
                            else { const int jq = j / Ns, k = j - jq * Ns; e = jq * Ns * R + k + r * Ns; }
                            const int b = (vec * m2p + e) & 15;
                            worst = std::max(worst, ++hits[b]);
                            ++used;
                        }
                        if (used) { extra += worst - 1; ++count; }
                    }
        Ns *= R;
    }
    return count ? extra / count : 0.0;
}

// Row tile shape for row FFTs of length m2: TR row pairs, a power of two
// (so a warp's butterflies spread evenly over the rows), and the row
// stride m2p in [m2, m2 + 16] with the fewest bank conflicts; more row
// pairs win unless they cost more than a quarter wavefront per access.
void row_shape(int m2, int P1, const std::vector<int8_t> &radices, int &TR, int &m2p)
{
    // the shape depends on (m2, P1 up to 64) alone: remembered across lengths
    static std::mutex mu;
    static std::map<std::pair<int, int>, std::pair<int, int>> seen;
    const std::pair<int, int> key(m2, std::min(P1, 65));
    {
        std::lock_guard<std::mutex> lk(mu);
        const auto it = seen.find(key);
        if (it != seen.end()) { TR = it->second.first; m2p = it->second.second; return; }
    }
    double best = 1e30;
    TR = 1;
    m2p = m2 | 1;
    for (int tr = 1; tr <= 64 && 2 * tr * m2 <= TX_TILE; tr *= 2) {
        if (tr > 1 && tr / 2 >= P1) break;          // more row pairs than the transform has
        for (int p = m2; p <= m2 + 16 && 2 * tr * p <= TX_TILE; ++p) {
            const double score = row_bank_cost(m2, p, 2 * tr, radices) - 0.25 * std::log2(static_cast<double>(tr));
            if (score < best - 1e-12) { best = score; TR = tr; m2p = p; }
        }
    }
    std::lock_guard<std::mutex> lk(mu);
    seen[key] = std::make_pair(TR, m2p);
}

// Split m = n/2 = m1 x m2 for the multi-pass transform.  A column tile holds
// m1 rows of 2 TP columns and a row tile 2 TR rows of m2 (made odd), each at
// most TX_TILE values.  Wide column tiles (TP up to 16: sample runs of 64
// floats) and several row pairs (TR up to 4: fewer Philox blocks per mode)
// score highest, then m2 / m1 nearest 2.5.  tile_pairs > 0 caps TP.
bool choose_tx_split(int n, int rmax, int tile_pairs, TxLen &out)
{
    const int m = n / 2;
    double best = -1.0;
    int bm1 = 0;
    for (int m1 = 1; m1 <= m; ++m1) {
        if (m % m1) continue;
        const int m2 = m / m1;
        const auto r1 = radix_plan(m1, rmax), r2 = radix_plan(m2, rmax);
        if ((m1 > 1 && r1.empty()) || (m2 > 1 && r2.empty())) continue;
        if (r1.size() > TX_MAXR || r2.size() > TX_MAXR) continue;
        const int m2p = m2 | 1;
        if (2 * m1 > TX_TILE || 2 * m2p > TX_TILE) continue;
        const int P1 = m1 / 2 + 1, P2 = (m2 + 1) / 2;
        const int TP = tile_width(P2, m1, tile_pairs);
        const int TR = std::min(P1, TX_TILE / (2 * m2p));
        const double score = std::min(TP, 16) / 16.0 + std::min(TR, 4) / 4.0 -
                             1e-3 * std::fabs(std::log(static_cast<double>(m2) / m1 / 2.5));
        if (score > best) { best = score; bm1 = m1; }
    }
    if (bm1 == 0) return false;
    const int m1 = bm1, m2 = m / m1;
    const auto r1 = radix_plan(m1, rmax), r2 = radix_plan(m2, rmax);
    std::memset(&out, 0, sizeof(out));
    out.n = n; out.m = m; out.m1 = m1; out.m2 = m2;
    out.P1 = m1 / 2 + 1;
    out.P2 = (m2 + 1) / 2;
    out.TP = tile_width(out.P2, m1, tile_pairs);
    row_shape(m2, out.P1, r2, out.TR, out.m2p);
    out.nr1 = static_cast<int32_t>(r1.size());
    out.nr2 = static_cast<int32_t>(r2.size());
    fill_stages(out.s1, r1, m1);
    fill_stages(out.s2, r2, m2);
    out.f_m2 = make_fastdiv(static_cast<uint32_t>(m2));
    out.f_W = make_fastdiv(static_cast<uint32_t>(2 * out.TP));
    out.lgW = 0;
    while ((2 << out.lgW) <= 2 * out.TP) ++out.lgW;
    out.lgS = 0;
    while ((2 << out.lgS) <= 2 * out.TR) ++out.lgS;
    out.f_2TR = make_fastdiv(static_cast<uint32_t>(2 * out.TR));
    out.sq_fwd = std::sqrt(2.0 / n);
    out.s0_fwd = 1.0 / std::sqrt(static_cast<double>(n));
    out.sq_inv = std::sqrt(0.5 * n) / m;
    out.s0_inv = std::sqrt(static_cast<double>(n)) / m;
    return true;
}

tod_status to_status(cudaError_t e)
{
    if (e == cudaSuccess) return TOD_OK;
    if (e == cudaErrorMemoryAllocation) return TOD_ERR_OOM;
    return TOD_ERR_CUDA;
}

struct DeviceGuard {
    int prev = 0;
    explicit DeviceGuard(int dev) { cudaGetDevice(&prev); if (prev != dev) cudaSetDevice(dev); }
    ~DeviceGuard() { int cur = 0; cudaGetDevice(&cur); if (cur != prev) cudaSetDevice(prev); }
};

bool valid_streams(const tod_huff_streams &h, int64_t nq, int64_t nscan, const std::vector<int64_t> &off)
{
    if (!h.words || !h.word_off || !h.nbits || !h.blk_off || !h.ckpt_bit || !h.ckpt_val ||
        !h.sym_off || !h.sym_vals || !h.sym_len)
        return false;
    if (h.word_off[0] != 0 || h.word_off[nq] != h.nwords || h.blk_off[0] != 0 || h.blk_off[nq] != h.nblk)
        return false;
    if (h.sym_off[0] != 0 || h.sym_off[nscan] != h.nsym) return false;
    for (int64_t q = 0; q < nq; ++q) {
        const int64_t n = off[q + 1] - off[q];
        if (h.word_off[q + 1] < h.word_off[q]) return false;
        if (h.nbits[q] < 0 || h.nbits[q] > 32 * (h.word_off[q + 1] - h.word_off[q])) return false;
        if (h.blk_off[q + 1] - h.blk_off[q] != (n + TOD_CKPT_BLOCK - 1) / TOD_CKPT_BLOCK) return false;
        for (int64_t b = h.blk_off[q]; b < h.blk_off[q + 1]; ++b)
            if (static_cast<int64_t>(h.ckpt_bit[b]) > h.nbits[q]) return false;
    }
    for (int64_t s = 0; s < nscan; ++s) {
        if (h.sym_off[s + 1] <= h.sym_off[s]) return false;
        for (int64_t i = h.sym_off[s]; i < h.sym_off[s + 1]; ++i)
            if (h.sym_len[i] < 1 || h.sym_len[i] > TOD_HUFF_MAXLEN) return false;
    }
    return true;
}

cudaError_t build_huff(Plan &p, HuffDev &d, const tod_huff_streams &h)
{
    cudaError_t e;
    std::vector<uint32_t> words(h.nwords + 4, 0u);
    std::memcpy(words.data(), h.words, sizeof(uint32_t) * h.nwords);
    if ((e = dev_upload(p, d.words, words.data(), words.size()))) return e;
    if ((e = dev_upload(p, d.word_off, h.word_off, p.nq + 1))) return e;
    if ((e = dev_upload(p, d.nbits, h.nbits, p.nq))) return e;
    if ((e = dev_upload(p, d.blk_off, h.blk_off, p.nq + 1))) return e;
    if ((e = dev_upload(p, d.ckpt_bit, h.ckpt_bit, h.nblk))) return e;
    if ((e = dev_upload(p, d.ckpt_val, h.ckpt_val, h.nblk))) return e;
    std::vector<int32_t> blk_q(h.nblk);
    for (int64_t q = 0; q < p.nq; ++q)
        for (int64_t b = h.blk_off[q]; b < h.blk_off[q + 1]; ++b) blk_q[b] = static_cast<int32_t>(q);
    if ((e = dev_upload(p, d.blk_q, blk_q.data(), blk_q.size()))) return e;
    d.nblk = h.nblk;
    std::vector<int32_t> lut(static_cast<size_t>(p.nscan) << DEC_LUTB);
    std::vector<unsigned long long> lim(static_cast<size_t>(p.nscan) * 26);
    std::vector<int32_t> base(static_cast<size_t>(p.nscan) * 26);
    std::vector<int32_t> canon_off(p.nscan + 1, 0), canon;
    std::vector<int32_t> cta_scan;
    std::vector<int64_t> cta_blk0;
    std::vector<int32_t> cta_nblk;
    for (int s = 0; s < p.nscan; ++s) {
        const int64_t a = h.sym_off[s], k = h.sym_off[s + 1] - a;
        DecTab t = build_dectab(h.sym_vals + a, h.sym_len + a, k);
        std::copy(t.lut.begin(), t.lut.end(), lut.begin() + (static_cast<size_t>(s) << DEC_LUTB));
        for (int L = 0; L < 26; ++L) { lim[s * 26 + L] = t.lim[L]; base[s * 26 + L] = t.base[L]; }
        canon.insert(canon.end(), t.canon.begin(), t.canon.end());
        canon_off[s + 1] = static_cast<int32_t>(canon.size());
        d.max_canon = std::max<int32_t>(d.max_canon, static_cast<int32_t>(k));
        const int64_t b0 = h.blk_off[static_cast<int64_t>(s) * p.ndet];
        const int64_t b1 = h.blk_off[static_cast<int64_t>(s + 1) * p.ndet];
        for (int64_t b = b0; b < b1; b += DEC_T) {
            cta_scan.push_back(s);
            cta_blk0.push_back(b);
            cta_nblk.push_back(static_cast<int32_t>(std::min<int64_t>(DEC_T, b1 - b)));
        }
    }
    if ((e = dev_upload(p, d.lut, lut.data(), lut.size()))) return e;
    if ((e = dev_upload(p, d.lim, lim.data(), lim.size()))) return e;
    if ((e = dev_upload(p, d.base, base.data(), base.size()))) return e;
    if ((e = dev_upload(p, d.canon_off, canon_off.data(), canon_off.size()))) return e;
    if ((e = dev_upload(p, d.canon_vals, canon.data(), canon.size()))) return e;
    if ((e = dev_upload(p, d.cta_scan, cta_scan.data(), cta_scan.size()))) return e;
    if ((e = dev_upload(p, d.cta_blk0, cta_blk0.data(), cta_blk0.size()))) return e;
    if ((e = dev_upload(p, d.cta_nblk, cta_nblk.data(), cta_nblk.size()))) return e;
    d.ncta = static_cast<int32_t>(cta_scan.size());
    return cudaSuccess;
}

// The n_corr draw over the whole band (each pass one launch over every
// detscan's tiles) or, with the per-scan schedule, one launch sequence per
// detscan.
cudaError_t ncorr_draw(const Plan &p, const float *d, const float *s, const double *gain, const uint32_t *flags,
                       const double *psd, tod_rng rng, int mode, float tol, int maxit, float *x, int32_t *iters,
                       cudaStream_t st)
{
    const TxNcorrScratch sc = {p.ybuf, p.wpre, p.cgv, p.cgcap};
    if (p.schedule != TOD_SCHED_PER_SCAN)
        return launch_tx_ncorr(p, d, s, gain, flags, psd, rng, mode, tol, maxit, x, iters, st, 0, p.nq, sc,
                               p.pass_grid);
    cudaError_t e = cudaSuccess;
    for (int q = 0; q < p.nq && e == cudaSuccess; ++q) {
        const int items = std::max(p.h_col_off[q + 1] - p.h_col_off[q], p.h_row_off[q + 1] - p.h_row_off[q]);
        e = launch_tx_ncorr(p, d, s, gain, flags, psd, rng, mode, tol, maxit, x, iters, st, q, q + 1, sc,
                            std::min(p.pass_grid, std::max(1, items)));
    }
    return e;
}

}  // namespace

// ===========================================================================
// C ABI
// ===========================================================================
extern "C" {

const char *tod_status_string(tod_status s)
{
    switch (s) {
    case TOD_OK: return "ok";
    case TOD_ERR_ARG: return "invalid argument";
    case TOD_ERR_CORRUPT_STREAM: return "corrupt Huffman stream";
    case TOD_ERR_NOT_CONVERGED: return "conjugate gradients did not converge";
    case TOD_ERR_TIMEOUT: return "bounded device wait timed out";
    case TOD_ERR_CUDA: return "CUDA runtime error";
    case TOD_ERR_OOM: return "out of memory";
    case TOD_ERR_UNIMPLEMENTED: return "not implemented";
    case TOD_ERR_SCRATCH: return "fixed scratch array too small for this plan";
    default: return "unknown status";
    }
}

int64_t tod_fft_length(int64_t n) { return fft_length_impl(n); }

void tod_huff_free(tod_huff_buffers *b)
{
    if (!b) return;
    std::free(b->words); std::free(b->word_off); std::free(b->nbits); std::free(b->blk_off);
    std::free(b->ckpt_bit); std::free(b->ckpt_val); std::free(b->sym_off); std::free(b->sym_vals);
    std::free(b->sym_len);
    std::memset(b, 0, sizeof(*b));
}

tod_status tod_huff_encode(int32_t ndet, int32_t nscan, const int64_t *offsets, const int32_t *values,
                           tod_huff_buffers *out)
{
    if (!out || !offsets || ndet <= 0 || nscan <= 0) return TOD_ERR_ARG;
    std::memset(out, 0, sizeof(*out));
    const int64_t nq = static_cast<int64_t>(ndet) * nscan;
    for (int64_t q = 0; q < nq; ++q)
        if (offsets[q + 1] < offsets[q]) return TOD_ERR_ARG;
    if (offsets[0] != 0 || (offsets[nq] > 0 && !values)) return TOD_ERR_ARG;
    for (int64_t q = 0; q < nq; ++q) {          // every difference must be an int32 symbol
        int64_t prev = 0;
        for (int64_t t = offsets[q]; t < offsets[q + 1]; ++t) {
            const int64_t dv = static_cast<int64_t>(values[t]) - prev;
            if (dv < INT32_MIN || dv > INT32_MAX) return TOD_ERR_ARG;
            prev = values[t];
        }
    }
    try {
        // per scan: code over the deltas of all its detectors
        std::vector<std::vector<int32_t>> svals(nscan);
        std::vector<std::vector<uint8_t>> slen(nscan);
        std::vector<std::vector<uint32_t>> scode(nscan);
        parallel_for(nscan, [&](int64_t a, int64_t b) {
            for (int64_t s = a; s < b; ++s) {
                std::vector<int32_t> dl;
                for (int64_t q = s * ndet; q < (s + 1) * ndet; ++q) {
                    int32_t prev = 0;
                    for (int64_t t = offsets[q]; t < offsets[q + 1]; ++t) {
                        dl.push_back(values[t] - prev);
                        prev = values[t];
                    }
                }
                std::sort(dl.begin(), dl.end());
                std::vector<int32_t> v;
                std::vector<int64_t> c;
                for (size_t i = 0; i < dl.size();) {
                    size_t j = i;
                    while (j < dl.size() && dl[j] == dl[i]) ++j;
                    v.push_back(dl[i]);
                    c.push_back(static_cast<int64_t>(j - i));
                    i = j;
                }
                if (v.empty()) { v.push_back(0); c.push_back(1); }
                slen[s] = huffman_lengths(c);
                scode[s] = canonical_codes(slen[s]);
                svals[s] = std::move(v);
            }
        });
        // bit lengths per detscan
        std::vector<int64_t> nbits(nq, 0), nblk(nq, 0);
        parallel_for(nq, [&](int64_t a, int64_t b) {
            for (int64_t q = a; q < b; ++q) {
                const auto &v = svals[q / ndet];
                const auto &L = slen[q / ndet];
                int32_t prev = 0;
                int64_t bits = 0;
                for (int64_t t = offsets[q]; t < offsets[q + 1]; ++t) {
                    const int32_t dv = values[t] - prev;
                    prev = values[t];
                    bits += L[std::lower_bound(v.begin(), v.end(), dv) - v.begin()];
                }
                nbits[q] = bits;
                nblk[q] = (offsets[q + 1] - offsets[q] + TOD_CKPT_BLOCK - 1) / TOD_CKPT_BLOCK;
            }
        });
        const auto alloc = [](size_t bytes) { void *p = std::calloc(bytes ? bytes : 1, 1); if (!p) throw std::bad_alloc(); return p; };
        out->word_off = static_cast<int64_t *>(alloc(sizeof(int64_t) * (nq + 1)));
        out->nbits = static_cast<int64_t *>(alloc(sizeof(int64_t) * nq));
        out->blk_off = static_cast<int64_t *>(alloc(sizeof(int64_t) * (nq + 1)));
        for (int64_t q = 0; q < nq; ++q) {
            out->word_off[q + 1] = out->word_off[q] + (nbits[q] + 31) / 32;
            out->blk_off[q + 1] = out->blk_off[q] + nblk[q];
            out->nbits[q] = nbits[q];
        }
        out->nwords = out->word_off[nq];
        out->nblk = out->blk_off[nq];
        out->words = static_cast<uint32_t *>(alloc(sizeof(uint32_t) * out->nwords));
        out->ckpt_bit = static_cast<uint32_t *>(alloc(sizeof(uint32_t) * out->nblk));
        out->ckpt_val = static_cast<int32_t *>(alloc(sizeof(int32_t) * out->nblk));
        parallel_for(nq, [&](int64_t a, int64_t b) {
            for (int64_t q = a; q < b; ++q) {
                const auto &v = svals[q / ndet];
                const auto &L = slen[q / ndet];
                const auto &cw = scode[q / ndet];
                uint32_t *w = out->words + out->word_off[q];
                uint64_t acc = 0;          // pending bits, left-aligned in the low 'fill' bits
                int fill = 0;
                int64_t wi = 0, bitpos = 0;
                int32_t prev = 0;
                for (int64_t t = offsets[q], i = 0; t < offsets[q + 1]; ++t, ++i) {
                    if (i % TOD_CKPT_BLOCK == 0) {
                        const int64_t blk = out->blk_off[q] + i / TOD_CKPT_BLOCK;
                        out->ckpt_bit[blk] = static_cast<uint32_t>(bitpos);
                        out->ckpt_val[blk] = prev;
                    }
                    const int32_t dv = values[t] - prev;
                    prev = values[t];
                    const size_t si = std::lower_bound(v.begin(), v.end(), dv) - v.begin();
                    const int l = L[si];
                    acc = (acc << l) | cw[si];
                    fill += l;
                    bitpos += l;
                    while (fill >= 32) {
                        w[wi++] = static_cast<uint32_t>(acc >> (fill - 32));
                        fill -= 32;
                    }
                }
                if (fill > 0) w[wi++] = static_cast<uint32_t>(acc << (32 - fill));
            }
        });
        // code tables
        int64_t nsym = 0;
        for (int s = 0; s < nscan; ++s) nsym += static_cast<int64_t>(svals[s].size());
        out->nsym = nsym;
        out->sym_off = static_cast<int64_t *>(alloc(sizeof(int64_t) * (nscan + 1)));
        out->sym_vals = static_cast<int32_t *>(alloc(sizeof(int32_t) * nsym));
        out->sym_len = static_cast<uint8_t *>(alloc(nsym));
        for (int s = 0; s < nscan; ++s) {
            out->sym_off[s + 1] = out->sym_off[s] + static_cast<int64_t>(svals[s].size());
            std::copy(svals[s].begin(), svals[s].end(), out->sym_vals + out->sym_off[s]);
            std::copy(slen[s].begin(), slen[s].end(), out->sym_len + out->sym_off[s]);
        }
    } catch (const std::bad_alloc &) {
        tod_huff_free(out);
        return TOD_ERR_OOM;
    }
    return TOD_OK;
}

tod_status tod_plan_create(tod_plan **out, const tod_band_desc *band)
{
    if (!out || !band) return TOD_ERR_ARG;
    *out = nullptr;
    if (band->nside <= 0 || band->nside > 8192 || band->ndet <= 0 || band->nscan <= 0 ||
        band->n_psi != TOD_N_PSI || !(band->fsamp > 0) || !band->offsets)
        return TOD_ERR_ARG;
    const int tile_pairs = band->tile_pairs;
    if (tile_pairs < 0 || tile_pairs > 64) return TOD_ERR_ARG;
    const int rmax = band->max_radix > 0 ? band->max_radix : 16;
    if (rmax < 2 || rmax > 16) return TOD_ERR_ARG;
    Plan *p = new (std::nothrow) Plan();
    if (!p) return TOD_ERR_OOM;
    p->device = band->device;
    DeviceGuard dg(p->device);
    p->nside = band->nside;
    p->npix = 12 * band->nside * band->nside;
    p->ndet = band->ndet;
    p->nscan = band->nscan;
    p->nq = band->ndet * band->nscan;
    p->fsamp = band->fsamp;
    p->tile_pairs = tile_pairs;
    p->h_off.assign(band->offsets, band->offsets + p->nq + 1);
    if (p->h_off[0] != 0) { delete p; return TOD_ERR_ARG; }
    for (int q = 0; q < p->nq; ++q) {
        const int64_t n = p->h_off[q + 1] - p->h_off[q];
        if (n < 4 || n != fft_length_impl(n) || n > (int64_t(1) << 24)) { delete p; return TOD_ERR_ARG; }
        if (q % p->ndet && n != p->h_off[q] - p->h_off[q - 1]) { delete p; return TOD_ERR_ARG; }
    }
    p->N = p->h_off[p->nq];
    if (p->N >= (int64_t(1) << 40)) { delete p; return TOD_ERR_ARG; }
    if (!valid_streams(band->pix, p->nq, p->nscan, p->h_off) ||
        !valid_streams(band->psi, p->nq, p->nscan, p->h_off)) {
        delete p;
        return TOD_ERR_ARG;
    }
    cudaError_t e = cudaSetDevice(p->device);
    if (e != cudaSuccess) { delete p; return TOD_ERR_CUDA; }
    const auto fail = [&](cudaError_t err) { const tod_status s = to_status(err); free_plan(p); return s; };

    if ((e = dev_upload(*p, p->off, p->h_off.data(), p->h_off.size()))) return fail(e);
    if ((e = dev_upload(*p, p->status, static_cast<int32_t *>(nullptr), p->nq))) return fail(e);
    if ((e = setup_decode_kernel())) return fail(e);
    if ((e = setup_gain_smooth_kernel())) return fail(e);
    if ((e = build_huff(*p, p->hpix, band->pix))) return fail(e);
    if ((e = build_huff(*p, p->hpsi, band->psi))) return fail(e);

    // element-wise tiles
    {
        std::vector<int32_t> tq;
        std::vector<int64_t> t0;
        for (int q = 0; q < p->nq; ++q)
            for (int64_t t = p->h_off[q]; t < p->h_off[q + 1]; t += ELEM_TILE) { tq.push_back(q); t0.push_back(t); }
        p->ntile = static_cast<int32_t>(tq.size());
        if ((e = dev_upload(*p, p->tile_q, tq.data(), tq.size()))) return fail(e);
        if ((e = dev_upload(*p, p->tile_t0, t0.data(), t0.size()))) return fail(e);
    }
    // noise PSD step: ln k as FP32 pairs, ln(fsamp / (2 n_q)), and per
    // detector the mode count and sum of ln f_k (k >= 1), all from FP64
    {
        int64_t kmax = 1;
        for (int q = 0; q < p->nq; ++q) kmax = std::max<int64_t>(kmax, p->h_off[q + 1] - p->h_off[q]);
        std::vector<float2> lnk(static_cast<size_t>(kmax));
        for (int64_t k = 0; k < kmax; ++k) {
            const double l = k > 0 ? std::log(static_cast<double>(k)) : 0.0;
            const float hi = static_cast<float>(l);
            lnk[k] = make_float2(hi, static_cast<float>(l - static_cast<double>(hi)));
        }
        std::vector<double> lnfs(p->nq), nmodes(p->ndet, 0.0), sumlnf(p->ndet, 0.0);
        for (int q = 0; q < p->nq; ++q) {
            const int64_t n = p->h_off[q + 1] - p->h_off[q];
            lnfs[q] = n > 0 ? std::log(p->fsamp / (2.0 * static_cast<double>(n))) : 0.0;
            if (n < 2) continue;
            nmodes[q % p->ndet] += static_cast<double>(n - 1);
            sumlnf[q % p->ndet] += std::lgamma(static_cast<double>(n)) + static_cast<double>(n - 1) * lnfs[q];
        }
        if ((e = dev_upload(*p, p->lnk, lnk.data(), lnk.size()))) return fail(e);
        if ((e = dev_upload(*p, p->lnfs, lnfs.data(), lnfs.size()))) return fail(e);
        if ((e = dev_upload(*p, p->psd_nmodes, nmodes.data(), nmodes.size()))) return fail(e);
        if ((e = dev_upload(*p, p->psd_sumlnf, sumlnf.data(), sumlnf.size()))) return fail(e);
        if ((e = dev_upload(*p, p->psd_part, static_cast<double *>(nullptr), static_cast<size_t>(p->ntile))))
            return fail(e);
        if ((e = dev_upload(*p, p->psd_state, static_cast<double *>(nullptr), static_cast<size_t>(p->ndet) * 8)))
            return fail(e);
    }
    // psi table: FP32 values of cos 2psi, sin 2psi at the bin centres
    {
        std::vector<float2> trig(TOD_N_PSI);
        for (int b = 0; b < TOD_N_PSI; ++b) {
            const double psi = (b + 0.5) * (2.0 * kPi / TOD_N_PSI);
            trig[b] = make_float2(static_cast<float>(std::cos(2.0 * psi)), static_cast<float>(std::sin(2.0 * psi)));
        }
        if ((e = dev_upload(*p, p->trig, trig.data(), trig.size()))) return fail(e);
    }
    // transform plans of the multi-pass DCT (k_tx.cu): one per distinct length
    {
        std::vector<int> lens(p->nq);
        int maxlen = 0;
        for (int q = 0; q < p->nq; ++q) {
            lens[q] = static_cast<int>(p->h_off[q + 1] - p->h_off[q]);
            maxlen = std::max(maxlen, lens[q]);
        }
        std::vector<int> uniq(lens);
        std::sort(uniq.begin(), uniq.end());
        uniq.erase(std::unique(uniq.begin(), uniq.end()), uniq.end());
        std::vector<TxLen> tl;
        for (int n : uniq) {
            TxLen L;
            if (!choose_tx_split(n, rmax, tile_pairs, L)) { free_plan(p); return TOD_ERR_ARG; }
            tl.push_back(L);
        }
        // twiddle block per length, FP64-generated: W_m1^i (m1), W_m2^i (m2),
        // W_4n^{k1} (m1), W_4n^{m1 k2} (m2), W_4n^{5 k1} (m1),
        // W_4n^{5 m1 k2} (m2), W_m^{64 i} (m/64 + 1), W_m^i (64)
        std::vector<double2> tw;
        const auto push_w = [&](int64_t Lp, int64_t i) {
            const double ang = -2.0 * kPi * static_cast<double>(i % Lp) / static_cast<double>(Lp);
            tw.push_back(make_double2(std::cos(ang), std::sin(ang)));
        };
        for (auto &L : tl) {
            L.twb = static_cast<int64_t>(tw.size());
            const int64_t n4 = 4 * static_cast<int64_t>(L.n);
            for (int i = 0; i < L.m1; ++i) push_w(L.m1, i);
            for (int i = 0; i < L.m2; ++i) push_w(L.m2, i);
            for (int i = 0; i < L.m1; ++i) push_w(n4, i);
            for (int i = 0; i < L.m2; ++i) push_w(n4, static_cast<int64_t>(L.m1) * i);
            for (int i = 0; i < L.m1; ++i) push_w(n4, 5 * static_cast<int64_t>(i));
            for (int i = 0; i < L.m2; ++i) push_w(n4, 5 * static_cast<int64_t>(L.m1) * i);
            for (int i = 0; i <= L.m / 64; ++i) push_w(L.m, 64 * static_cast<int64_t>(i));
            for (int i = 0; i < 64; ++i) push_w(L.m, i);
        }
        std::vector<float2> tw32(tw.size());
        for (size_t i = 0; i < tw.size(); ++i)
            tw32[i] = make_float2(static_cast<float>(tw[i].x), static_cast<float>(tw[i].y));
        // work items, detscan-major
        std::vector<int32_t> qtx(p->nq);
        std::vector<int2> ci, ri;
        p->h_col_off.assign(p->nq + 1, 0);
        p->h_row_off.assign(p->nq + 1, 0);
        for (int q = 0; q < p->nq; ++q) {
            qtx[q] = static_cast<int32_t>(std::lower_bound(uniq.begin(), uniq.end(), lens[q]) - uniq.begin());
            const TxLen &L = tl[qtx[q]];
            for (int b = 0; b * L.TP < L.P2; ++b) ci.push_back(make_int2(q, b));
            for (int b = 0; b * L.TR < L.P1; ++b) ri.push_back(make_int2(q, b));
            p->h_col_off[q + 1] = static_cast<int32_t>(ci.size());
            p->h_row_off[q + 1] = static_cast<int32_t>(ri.size());
        }
        p->ntx = static_cast<int32_t>(tl.size());
        p->h_txl = tl;
        p->h_q_tx = qtx;
        if ((e = dev_upload(*p, p->txl, tl.data(), tl.size()))) return fail(e);
        if ((e = dev_upload(*p, p->q_tx, qtx.data(), qtx.size()))) return fail(e);
        if ((e = dev_upload(*p, p->txtw, tw32.data(), tw32.size()))) return fail(e);
        if ((e = dev_upload(*p, p->txtw64, tw.data(), tw.size()))) return fail(e);
        if ((e = dev_upload(*p, p->colitems, ci.data(), ci.size()))) return fail(e);
        if ((e = dev_upload(*p, p->rowitems, ri.data(), ri.size()))) return fail(e);
        if ((e = dev_upload(*p, p->col_off, p->h_col_off.data(), p->h_col_off.size()))) return fail(e);
        if ((e = dev_upload(*p, p->row_off, p->h_row_off.data(), p->h_row_off.size()))) return fail(e);
        if ((e = setup_tx_kernels(*p))) return fail(e);
        // scratch: the complex intermediate (room for one whole detscan in FP64
        // too), per-item partial sums, the flag prefix, CG state and vectors
        p->ybuf_floats = std::max<int64_t>(p->N, 2 * static_cast<int64_t>(maxlen));
        if ((e = dev_upload(*p, p->ybuf, static_cast<float2 *>(nullptr), static_cast<size_t>(p->ybuf_floats / 2))))
            return fail(e);
        if ((e = dev_upload(*p, p->part, static_cast<double *>(nullptr), 4 * (ci.size() + ri.size()))))
            return fail(e);
        if ((e = dev_upload(*p, p->wpre, static_cast<int64_t *>(nullptr), static_cast<size_t>(p->N / 32 + 3))))
            return fail(e);
        if ((e = dev_upload(*p, p->chunk, static_cast<int64_t *>(nullptr), static_cast<size_t>(std::max(p->coop_grid, p->pass_grid) + 1))))
            return fail(e);
        if ((e = dev_upload(*p, p->cgs, static_cast<CgState *>(nullptr), static_cast<size_t>(p->nq)))) return fail(e);
        if ((e = dev_upload(*p, p->gblk, static_cast<int2 *>(nullptr), static_cast<size_t>(p->nq) * TX_GBMAX)))
            return fail(e);
        if ((e = dev_upload(*p, p->gnb, static_cast<int32_t *>(nullptr), static_cast<size_t>(p->nq)))) return fail(e);
        p->cgcap = std::max<int64_t>(p->N / 16, 2 * static_cast<int64_t>(maxlen));
        if ((e = dev_upload(*p, p->cgv, static_cast<float *>(nullptr), static_cast<size_t>(5 * p->cgcap))))
            return fail(e);
        if ((e = dev_upload(*p, p->cg_count, static_cast<int32_t *>(nullptr), 2))) return fail(e);
        if ((e = dev_upload(*p, p->nclist, static_cast<int32_t *>(nullptr), 3 * static_cast<size_t>(p->nq) + 3)))
            return fail(e);
        if ((e = dev_upload(*p, p->chi2_dpsd, static_cast<double *>(nullptr), 3 * static_cast<size_t>(p->nq))))
            return fail(e);
        if ((e = dev_upload(*p, p->qsc, static_cast<float4 *>(nullptr), 2 * static_cast<size_t>(p->nq))))
            return fail(e);
        // Toeplitz preconditioner tables (per detector): the gap kernel at a
        // power-of-two reference length covering every lag of every detscan
        p->cz_href = 1024;
        while (p->cz_href < maxlen) p->cz_href *= 2;
        const size_t M2 = 2 * static_cast<size_t>(p->cz_href);
        if ((e = dev_upload(*p, p->czfft, static_cast<float2 *>(nullptr), 2 * static_cast<size_t>(p->ndet) * M2)))
            return fail(e);
        if ((e = dev_upload(*p, p->cztab, static_cast<float4 *>(nullptr),
                            static_cast<size_t>(p->ndet) * (static_cast<size_t>(p->cz_href) + 1))))
            return fail(e);
        // coarse correction: block positions, S Z rows for up to czcap
        // flagged samples (3 % of the band; detscans past it run the
        // one-level preconditioner), the factor of E per detscan
        if ((e = dev_upload(*p, p->gbpos, static_cast<int32_t *>(nullptr), static_cast<size_t>(p->nq) * TX_GBMAX)))
            return fail(e);
        p->czcap = std::max<int64_t>(p->N / 32, 2 * static_cast<int64_t>(maxlen));
        if ((e = dev_upload(*p, p->czsz, static_cast<float *>(nullptr), static_cast<size_t>(p->czcap) * TX_CZJ)))
            return fail(e);
        if ((e = dev_upload(*p, p->czl, static_cast<float *>(nullptr),
                            static_cast<size_t>(p->nq) * 2 * TX_CBMAX * (TX_CZB + 1))))
            return fail(e);
        if ((e = dev_upload(*p, p->htab, static_cast<float *>(nullptr), static_cast<size_t>(p->ndet) * TOEP_LMAX)))
            return fail(e);
        if ((e = dev_upload(*p, p->xtab, static_cast<float *>(nullptr),
                            static_cast<size_t>(p->ndet) * (TOEP_LMAX * (TOEP_LMAX + 1) / 2))))
            return fail(e);
        if ((e = dev_upload(*p, p->lvalid, static_cast<int32_t *>(nullptr), static_cast<size_t>(p->ndet))))
            return fail(e);
    }
    // binning structure from the pointing (fixed during the run)
    {
        std::vector<int32_t> pix(p->N);
        std::vector<DecTab> tabs(p->nscan);
        for (int s = 0; s < p->nscan; ++s) {
            const int64_t a = band->pix.sym_off[s];
            tabs[s] = build_dectab(band->pix.sym_vals + a, band->pix.sym_len + a, band->pix.sym_off[s + 1] - a);
        }
        std::atomic<bool> bad(false);
        std::vector<uint32_t> srt(p->N);
        std::vector<std::vector<int32_t>> rpix(p->nq), rlen(p->nq);
        std::vector<std::vector<int64_t>> rstart(p->nq);
        parallel_for(p->nq, [&](int64_t a, int64_t b) {
            std::vector<uint64_t> key;
            for (int64_t q = a; q < b; ++q) {
                const int64_t o = p->h_off[q], n = p->h_off[q + 1] - o;
                if (!host_decode(band->pix, tabs[q / p->ndet], q, n, pix.data() + o)) { bad = true; continue; }
                key.resize(n);
                for (int64_t t = 0; t < n; ++t) {
                    const int32_t px = pix[o + t];
                    if (px < 0 || px >= p->npix) { bad = true; break; }
                    key[t] = (static_cast<uint64_t>(px) << 32) | static_cast<uint64_t>(t);
                }
                if (bad) continue;
                std::sort(key.begin(), key.end());
                // runs (one per pixel, samples in time order), then ordered by
                // their first sample: neighbouring runs are neighbours on the
                // scan ring, so a tile's samples lie in a few stretches of
                // consecutive time per revolution
                std::vector<int64_t> rb;            // run starts in key
                for (int64_t i = 0; i < n; ++i)
                    if (i == 0 || (key[i] >> 32) != (key[i - 1] >> 32)) rb.push_back(i);
                rb.push_back(n);
                const size_t nrun = rb.size() - 1;
                std::vector<int32_t> ord(nrun);
                for (size_t r = 0; r < nrun; ++r) ord[r] = static_cast<int32_t>(r);
                std::sort(ord.begin(), ord.end(), [&](int32_t x, int32_t y) {
                    return (key[rb[x]] & 0xFFFFFFFFu) < (key[rb[y]] & 0xFFFFFFFFu);
                });
                int64_t pos = o;
                for (size_t k = 0; k < nrun; ++k) {
                    const int32_t r = ord[k];
                    rpix[q].push_back(static_cast<int32_t>(key[rb[r]] >> 32));
                    rstart[q].push_back(pos);
                    rlen[q].push_back(static_cast<int32_t>(rb[r + 1] - rb[r]));
                    for (int64_t i = rb[r]; i < rb[r + 1]; ++i)   // run-major position -> time index
                        srt[pos++] = static_cast<uint32_t>(key[i] & 0xFFFFFFFFu);
                }
            }
        });
        if (bad) { free_plan(p); return TOD_ERR_CORRUPT_STREAM; }
        std::vector<int64_t> pair_off(p->nq + 1, 0);
        for (int q = 0; q < p->nq; ++q) pair_off[q + 1] = pair_off[q] + static_cast<int64_t>(rpix[q].size());
        p->npairs = pair_off[p->nq];
        std::vector<int64_t> pstart(p->npairs), pslot_off(static_cast<size_t>(p->npix) + 1, 0);
        std::vector<int32_t> plen(p->npairs), pslot(p->npairs);
        for (int q = 0; q < p->nq; ++q)
            for (size_t i = 0; i < rpix[q].size(); ++i) pslot_off[rpix[q][i] + 1]++;
        for (int px = 0; px < p->npix; ++px) pslot_off[px + 1] += pslot_off[px];
        std::vector<int64_t> fillc(pslot_off.begin(), pslot_off.end() - 1);
        for (int q = 0; q < p->nq; ++q)
            for (size_t i = 0; i < rpix[q].size(); ++i) {
                const int64_t pr = pair_off[q] + static_cast<int64_t>(i);
                pstart[pr] = rstart[q][i];
                plen[pr] = rlen[q][i];
                pslot[pr] = static_cast<int32_t>(fillc[rpix[q][i]]++);
            }
        if (p->npairs >= (int64_t(1) << 31)) { free_plan(p); return TOD_ERR_ARG; }
        // binning tiles: consecutive whole runs of one detscan, at most
        // BIN_TILE samples, or a single longer run on its own
        std::vector<int32_t> tq, tr0;
        for (int q = 0; q < p->nq; ++q) {
            int64_t cnt = 0;
            for (int64_t pr = pair_off[q]; pr < pair_off[q + 1]; ++pr) {
                const int64_t len = plen[pr];
                if (pr == pair_off[q] || cnt + len > BIN_TILE) {
                    tq.push_back(q);
                    tr0.push_back(static_cast<int32_t>(pr));
                    cnt = 0;
                }
                cnt += len;
            }
        }
        tr0.push_back(static_cast<int32_t>(p->npairs));
        p->nbin_tiles = static_cast<int32_t>(tq.size());
        // load order of each tile: the k-th sample of every run of the tile,
        // k = 0, 1, ... (consecutive runs' k-th samples are close in time, so
        // a warp's loads share sectors); ld_pos is the sample's run-major
        // position in the tile, where the sums read it
        std::vector<uint32_t> ld_t(p->N);
        std::vector<uint16_t> ld_pos(p->N, 0);
        parallel_for(p->nbin_tiles, [&](int64_t a, int64_t b) {
            for (int64_t tl = a; tl < b; ++tl) {
                const int64_t r0 = tr0[tl], r1 = tr0[tl + 1];
                const int64_t s0 = pstart[r0];
                int32_t lmax = 0;
                for (int64_t r = r0; r < r1; ++r) lmax = std::max(lmax, plen[r]);
                if (r1 - r0 == 1) {          // one run (possibly longer than a tile): its own order
                    for (int32_t k = 0; k < plen[r0]; ++k) {
                        ld_t[s0 + k] = srt[s0 + k];
                        ld_pos[s0 + k] = static_cast<uint16_t>(std::min<int32_t>(k, 0xFFFF));
                    }
                    continue;
                }
                int64_t i = s0;
                for (int32_t k = 0; k < lmax; ++k)
                    for (int64_t r = r0; r < r1; ++r)
                        if (k < plen[r]) {
                            const int64_t pos = pstart[r] + k;
                            ld_t[i] = srt[pos];
                            ld_pos[i] = static_cast<uint16_t>(pos - s0);
                            ++i;
                        }
            }
        });
        if ((e = dev_upload(*p, p->ld_t, ld_t.data(), ld_t.size()))) return fail(e);
        if ((e = dev_upload(*p, p->ld_pos, ld_pos.data(), ld_pos.size()))) return fail(e);
        if ((e = dev_upload(*p, p->bin_tile_q, tq.data(), tq.size()))) return fail(e);
        if ((e = dev_upload(*p, p->bin_tile_r0, tr0.data(), tr0.size()))) return fail(e);
        if ((e = dev_upload(*p, p->pair_off, pair_off.data(), pair_off.size()))) return fail(e);
        if ((e = dev_upload(*p, p->pair_start, pstart.data(), pstart.size()))) return fail(e);
        if ((e = dev_upload(*p, p->pair_len, plen.data(), plen.size()))) return fail(e);
        if ((e = dev_upload(*p, p->pair_slot, pslot.data(), pslot.size()))) return fail(e);
        if ((e = dev_upload(*p, p->pix_slot_off, pslot_off.data(), pslot_off.size()))) return fail(e);
        if ((e = dev_upload(*p, p->rec, static_cast<double *>(nullptr), static_cast<size_t>(p->npairs) * 10))) return fail(e);
        if ((e = setup_bin_kernel(*p))) return fail(e);
    }
    if ((e = cudaDeviceSynchronize())) return fail(e);
    *out = reinterpret_cast<tod_plan *>(p);
    return TOD_OK;
}

tod_status tod_plan_destroy(tod_plan *pl)
{
    if (!pl) return TOD_ERR_ARG;
    free_plan(reinterpret_cast<Plan *>(pl));
    return TOD_OK;
}

static const char *const kKernelNames[TOD_KT_COUNT] = {
    "k_decode", "k_decode_tod", "k_decode_flags", "k_project", "k_project64", "k_det_scalars",
    "k_gain_cols", "k_gain_rows", "k_gain_colsinv", "k_gain_fin", "k_toep_kernel", "k_toep_durbin",
    "k_nc_flag_count", "k_nc_flag_scan", "k_nc_flag_write", "k_nc_index", "k_nc_coarse", "k_nc_rhs_cols", "k_nc_rhs_rows",
    "k_nc_x0_cols", "k_nc_cg_init", "k_nc_scatter", "k_nc_filter", "k_nc_gather", "k_nc_update", "k_nc_list", "k_nc_tail",
    "k_nc_scatter_final", "k_nc_filter_final", "k_nc_gather_final", "k_nc_finish", "k_bin", "k_reduce",
    "k_combine", "k_solve", "k_chi2_cols", "k_chi2_rows", "k_chi2_colsinv", "k_chi2_fin", "k_psd_sums",
    "k_psd_step"};

const char *tod_kernel_name(int32_t id)
{
    return (id >= 0 && id < TOD_KT_COUNT) ? kKernelNames[id] : nullptr;
}

tod_status tod_plan_set_kernel_timing(tod_plan *pl, int32_t on)
{
    if (!pl || (on != 0 && on != 1)) return TOD_ERR_ARG;
    Plan *p = reinterpret_cast<Plan *>(pl);
    if (on) {
        p->kt.used = 0;
        p->kt.ids.clear();
    }
    p->kt.on = on != 0;
    return TOD_OK;
}

tod_status tod_plan_kernel_times(tod_plan *pl, double *ms_out, int32_t *launches_out)
{
    if (!pl) return TOD_ERR_ARG;
    Plan *p = reinterpret_cast<Plan *>(pl);
    DeviceGuard dg(p->device);
    std::vector<double> ms(TOD_KT_COUNT, 0.0);
    std::vector<int32_t> n(TOD_KT_COUNT, 0);
    for (size_t i = 0; i < p->kt.ids.size(); ++i) {
        cudaEvent_t a = p->kt.pool[2 * i], b = p->kt.pool[2 * i + 1];
        cudaError_t e = cudaEventSynchronize(b);
        float t = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&t, a, b);
        if (e != cudaSuccess) return to_status(e);
        const int32_t id = p->kt.ids[i];
        if (id < 0 || id >= TOD_KT_COUNT) continue;
        ms[id] += t;
        ++n[id];
    }
    for (int i = 0; i < TOD_KT_COUNT; ++i) {
        if (ms_out) ms_out[i] = ms[i];
        if (launches_out) launches_out[i] = n[i];
    }
    return TOD_OK;
}

tod_status tod_plan_binning_info(const tod_plan *pl, int64_t *nruns, int32_t *ntiles)
{
    if (!pl) return TOD_ERR_ARG;
    const Plan *p = reinterpret_cast<const Plan *>(pl);
    if (nruns) *nruns = p->npairs;
    if (ntiles) *ntiles = p->nbin_tiles;
    return TOD_OK;
}

tod_status tod_plan_info(const tod_plan *pl, int64_t *nsamples, int32_t *ndetscan, int32_t *npix,
                         int32_t *tile_pairs, int64_t *device_bytes)
{
    if (!pl) return TOD_ERR_ARG;
    const Plan *p = reinterpret_cast<const Plan *>(pl);
    if (nsamples) *nsamples = p->N;
    if (ndetscan) *ndetscan = p->nq;
    if (npix) *npix = p->npix;
    if (tile_pairs) *tile_pairs = p->tile_pairs;
    if (device_bytes) *device_bytes = p->device_bytes;
    return TOD_OK;
}

tod_status tod_plan_status(tod_plan *pl, int32_t *detscan_status)
{
    if (!pl) return TOD_ERR_ARG;
    Plan *p = reinterpret_cast<Plan *>(pl);
    DeviceGuard dg(p->device);
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return TOD_ERR_CUDA;
    std::vector<int32_t> st(p->nq);
    e = cudaMemcpy(st.data(), p->status, sizeof(int32_t) * p->nq, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return TOD_ERR_CUDA;
    e = cudaMemset(p->status, 0, sizeof(int32_t) * p->nq);
    if (e != cudaSuccess) return TOD_ERR_CUDA;
    if (detscan_status) std::memcpy(detscan_status, st.data(), sizeof(int32_t) * p->nq);
    for (int32_t s : st)
        if (s != TOD_OK) return s;
    return TOD_OK;
}

tod_status tod_plan_set_schedule(tod_plan *pl, int32_t schedule)
{
    if (!pl || (schedule != TOD_SCHED_PERSISTENT && schedule != TOD_SCHED_PER_SCAN)) return TOD_ERR_ARG;
    reinterpret_cast<Plan *>(pl)->schedule = schedule;
    return TOD_OK;
}

tod_status tod_plan_set_preconditioner(tod_plan *pl, int32_t levels)
{
    if (!pl || levels < TOD_PREC_NONE || levels > TOD_PREC_TWO_LEVEL) return TOD_ERR_ARG;
    Plan *p = reinterpret_cast<Plan *>(pl);
    p->use_prec = levels >= TOD_PREC_BLOCKS;
    p->use_coarse = levels >= TOD_PREC_TWO_LEVEL;
    return TOD_OK;
}

tod_status tod_decode(tod_plan *pl, int32_t *pix_out, uint16_t *psi_out, cudaStream_t stream)
{
    if (!pl || (!pix_out && !psi_out)) return TOD_ERR_ARG;
    Plan *p = reinterpret_cast<Plan *>(pl);
    DeviceGuard dg(p->device);
    cudaError_t e = cudaSuccess;
    if (pix_out) e = launch_decode(*p, p->hpix, pix_out, nullptr, stream);
    if (e == cudaSuccess && psi_out) e = launch_decode(*p, p->hpsi, nullptr, psi_out, stream);
    return to_status(e);
}

tod_status tod_plan_attach_data(tod_plan *pl, const tod_data_desc *data)
{
    if (!pl || !data) return TOD_ERR_ARG;
    Plan *p = reinterpret_cast<Plan *>(pl);
    if (p->has_tod || p->has_flag || !data->tod_scale) return TOD_ERR_ARG;
    if (!valid_streams(data->tod, p->nq, p->nscan, p->h_off) ||
        !valid_streams(data->flag, p->nq, p->nscan, p->h_off))
        return TOD_ERR_ARG;
    for (int q = 0; q < p->nq; ++q)
        if (!(data->tod_scale[q] > 0.0) || !std::isfinite(data->tod_scale[q])) return TOD_ERR_ARG;
    DeviceGuard dg(p->device);
    cudaError_t e;
    if ((e = build_huff(*p, p->htod, data->tod))) return to_status(e);
    if ((e = dev_upload(*p, p->tod_scale, data->tod_scale, p->nq))) return to_status(e);
    p->has_tod = true;
    if ((e = build_huff(*p, p->hflag, data->flag))) return to_status(e);
    p->flag_select = data->flag_select;
    p->has_flag = true;
    return TOD_OK;
}

tod_status tod_sample_gain_smooth(tod_plan *pl, const double *mu, const double *sigma, const double *prior,
                                  tod_rng rng, int32_t mode, double cg_tol, int32_t cg_maxiter,
                                  double *gain_out, int32_t *cg_iters_out, cudaStream_t stream)
{
    if (!pl || !mu || !sigma || !prior || !gain_out) return TOD_ERR_ARG;
    if ((mode != TOD_MODE_DRAW && mode != TOD_MODE_MEAN) || !(cg_tol > 0.0) || cg_maxiter < 0) return TOD_ERR_ARG;
    Plan *p = reinterpret_cast<Plan *>(pl);
    if (p->nscan > TOD_GAIN_SMOOTH_MAX_SCANS) return TOD_ERR_ARG;
    DeviceGuard dg(p->device);
    GainSmoothArgs a{};
    a.mu = mu;
    a.sigma = sigma;
    a.prior = prior;
    a.nscan = p->nscan;
    a.ndet = p->ndet;
    a.rng = rng;
    a.mode = mode;
    a.tol = static_cast<float>(cg_tol);
    a.maxiter = cg_maxiter;
    a.gain_out = gain_out;
    a.iters_out = cg_iters_out;
    a.status = p->status;
    return to_status(launch_gain_smooth(a, stream));
}

tod_status tod_decode_data(tod_plan *pl, float *d_out, uint32_t *flags_out, cudaStream_t stream)
{
    if (!pl || (!d_out && !flags_out)) return TOD_ERR_ARG;
    Plan *p = reinterpret_cast<Plan *>(pl);
    if (!p->has_tod || !p->has_flag) return TOD_ERR_ARG;
    DeviceGuard dg(p->device);
    cudaError_t e = cudaSuccess;
    if (d_out) e = launch_decode_tod(*p, d_out, stream);
    if (e == cudaSuccess && flags_out) e = launch_decode_flags(*p, flags_out, stream);
    return to_status(e);
}

tod_status tod_project(tod_plan *pl, const void *map_tqu, const int32_t *pix, const uint16_t *psi,
                       const double *gain, float *s_out, cudaStream_t stream)
{
    if (!pl || !map_tqu || !pix || !psi || !s_out) return TOD_ERR_ARG;
    Plan *p = reinterpret_cast<Plan *>(pl);
    DeviceGuard dg(p->device);
    return to_status(launch_project(*p, static_cast<const float4 *>(map_tqu), pix, psi, gain, s_out, stream));
}

tod_status tod_project_f64(tod_plan *pl, const double *map, const int32_t *pix, const uint16_t *psi,
                           const double *gain, double *s_out, cudaStream_t stream)
{
    if (!pl || !map || !pix || !psi || !s_out) return TOD_ERR_ARG;
    Plan *p = reinterpret_cast<Plan *>(pl);
    DeviceGuard dg(p->device);
    return to_status(launch_project64(*p, map, pix, psi, gain, s_out, stream));
}

tod_status tod_sample_gain(tod_plan *pl, const float *d, const float *s, const uint32_t *flags,
                           const double *psd, tod_rng rng, int32_t mode, double *gain_out,
                           double *mu_out, double *sigma_out, cudaStream_t stream)
{
    if (!pl || !d || !s || !flags || !psd || !gain_out) return TOD_ERR_ARG;
    if (mode != TOD_MODE_DRAW && mode != TOD_MODE_MEAN) return TOD_ERR_ARG;
    Plan *p = reinterpret_cast<Plan *>(pl);
    DeviceGuard dg(p->device);
    cudaError_t e = cudaSuccess;
    if (p->schedule == TOD_SCHED_PER_SCAN) {
        for (int q = 0; q < p->nq && e == cudaSuccess; ++q)
            e = launch_tx_gain(*p, d, s, flags, psd, rng, mode, gain_out, mu_out, sigma_out, stream, q, q + 1);
    } else {
        e = launch_tx_gain(*p, d, s, flags, psd, rng, mode, gain_out, mu_out, sigma_out, stream, 0, p->nq);
    }
    return to_status(e);
}

tod_status tod_sample_ncorr(tod_plan *pl, const float *d, const float *s, const double *gain,
                            const uint32_t *flags, const double *psd, tod_rng rng, int32_t mode,
                            double cg_tol, int32_t cg_maxiter, float *ncorr_out, int32_t *cg_iters_out,
                            cudaStream_t stream)
{
    if (!pl || !d || !s || !gain || !flags || !psd || !ncorr_out) return TOD_ERR_ARG;
    if (mode != TOD_MODE_DRAW && mode != TOD_MODE_MEAN) return TOD_ERR_ARG;
    Plan *p = reinterpret_cast<Plan *>(pl);
    DeviceGuard dg(p->device);
    const float tol = cg_tol > 0 ? static_cast<float>(cg_tol) : 1e-6f;
    const int maxit = cg_maxiter > 0 ? cg_maxiter : 500;
    cudaError_t e = p->use_prec ? launch_toeplitz_prep(*p, psd, stream) : cudaSuccess;
    if (e == cudaSuccess) e = ncorr_draw(*p, d, s, gain, flags, psd, rng, mode, tol, maxit, ncorr_out, cg_iters_out, stream);
    return to_status(e);
}

tod_status tod_ncorr_prepare(tod_plan *pl, const double *psd, cudaStream_t stream)
{
    if (!pl || !psd) return TOD_ERR_ARG;
    Plan *p = reinterpret_cast<Plan *>(pl);
    DeviceGuard dg(p->device);
    if (!p->use_prec) return TOD_OK;
    return to_status(launch_toeplitz_prep(*p, psd, stream));
}

tod_status tod_sample_ncorr_prepared(tod_plan *pl, const float *d, const float *s, const double *gain,
                                     const uint32_t *flags, const double *psd, tod_rng rng, int32_t mode,
                                     double cg_tol, int32_t cg_maxiter, float *ncorr_out,
                                     int32_t *cg_iters_out, cudaStream_t stream)
{
    if (!pl || !d || !s || !gain || !flags || !psd || !ncorr_out) return TOD_ERR_ARG;
    if (mode != TOD_MODE_DRAW && mode != TOD_MODE_MEAN) return TOD_ERR_ARG;
    Plan *p = reinterpret_cast<Plan *>(pl);
    DeviceGuard dg(p->device);
    const float tol = cg_tol > 0 ? static_cast<float>(cg_tol) : 1e-6f;
    const int maxit = cg_maxiter > 0 ? cg_maxiter : 500;
    return to_status(ncorr_draw(*p, d, s, gain, flags, psd, rng, mode, tol, maxit, ncorr_out, cg_iters_out,
                                stream));
}

tod_status tod_plan_set_ncorr_spectrum(tod_plan *pl, float *spec_out)
{
    if (!pl) return TOD_ERR_ARG;
    reinterpret_cast<Plan *>(pl)->spec_out = spec_out;
    return TOD_OK;
}

tod_status tod_sample_noise_psd(tod_plan *pl, const float *spec, const double *psd_in, tod_rng rng,
                                int32_t nsteps, double step_lnfknee, double step_alpha, double *psd_out,
                                int32_t *accepted_out, double *loglike_out, cudaStream_t stream)
{
    if (!pl || !spec || !psd_in || !psd_out || psd_out == psd_in || nsteps < 0) return TOD_ERR_ARG;
    if (!(step_lnfknee >= 0.0) || !(step_alpha >= 0.0)) return TOD_ERR_ARG;
    Plan *p = reinterpret_cast<Plan *>(pl);
    DeviceGuard dg(p->device);
    return to_status(launch_noise_psd(*p, spec, psd_in, rng, nsteps, step_lnfknee, step_alpha, psd_out,
                                      accepted_out, loglike_out, stream));
}

tod_status tod_bin(tod_plan *pl, const uint16_t *psi, const float *d, const float *ncorr,
                   const double *gain, const uint32_t *flags, const double *psd, double *A_out,
                   double *b_out, int32_t *hits_out, cudaStream_t stream)
{
    if (!pl || !psi || !d || !ncorr || !gain || !flags || !psd || !A_out || !b_out || !hits_out)
        return TOD_ERR_ARG;
    Plan *p = reinterpret_cast<Plan *>(pl);
    DeviceGuard dg(p->device);
    return to_status(launch_bin(*p, psi, d, ncorr, gain, flags, psd, A_out, b_out, hits_out, nullptr, stream));
}

tod_status tod_bin_partial(tod_plan *pl, const uint16_t *psi, const float *d, const float *ncorr,
                           const double *gain, const uint32_t *flags, const double *psd, double *part_out,
                           cudaStream_t stream)
{
    if (!pl || !psi || !d || !ncorr || !gain || !flags || !psd || !part_out) return TOD_ERR_ARG;
    Plan *p = reinterpret_cast<Plan *>(pl);
    DeviceGuard dg(p->device);
    return to_status(launch_bin(*p, psi, d, ncorr, gain, flags, psd, nullptr, nullptr, nullptr, part_out, stream));
}

tod_status tod_combine_partials(const double *parts, int32_t nparts, int64_t npix_range, double *A_out,
                                double *b_out, int32_t *hits_out, cudaStream_t stream)
{
    if (!parts || nparts < 1 || npix_range < 0 || !A_out || !b_out || !hits_out) return TOD_ERR_ARG;
    return to_status(launch_combine(parts, nparts, npix_range, A_out, b_out, hits_out, stream));
}

tod_status tod_solve_range(int64_t npix_range, const double *A, const double *b, const int32_t *hits, double rcond_min,
                           double *map_out, void *map_f32_out, double *rcond_out, uint8_t *valid_out,
                           cudaStream_t stream)
{
    if (npix_range < 0 || npix_range >= (int64_t(1) << 31) || !A || !b || !hits || !map_out) return TOD_ERR_ARG;
    return to_status(launch_solve_n(npix_range, A, b, hits, rcond_min, map_out, static_cast<float4 *>(map_f32_out),
                                    rcond_out, valid_out, stream));
}

tod_status tod_chi2(tod_plan *pl, const float *d, const void *s, const double *gain, const uint32_t *flags,
                    const double *psd, int32_t precision, double *chi2_out, double *dgain_out, double *total_out,
                    double *dpsd_out, void *v_out, cudaStream_t stream)
{
    if (!pl || !d || !s || !gain || !flags || !psd || !chi2_out || !dgain_out || !total_out || !dpsd_out)
        return TOD_ERR_ARG;
    if (precision != TOD_PREC_F32 && precision != TOD_PREC_F64) return TOD_ERR_ARG;
    Plan *p = reinterpret_cast<Plan *>(pl);
    DeviceGuard dg(p->device);
    return to_status(launch_tx_chi2(*p, precision == TOD_PREC_F64, d, s, gain, flags, psd, chi2_out, dgain_out,
                                    p->chi2_dpsd, total_out, dpsd_out, v_out, stream));
}

tod_status tod_project_adjoint(tod_plan *pl, const uint16_t *psi, const void *y, int32_t precision,
                               const double *gain, double *out, cudaStream_t stream)
{
    if (!pl || !psi || !y || !gain || !out) return TOD_ERR_ARG;
    if (precision != TOD_PREC_F32 && precision != TOD_PREC_F64) return TOD_ERR_ARG;
    Plan *p = reinterpret_cast<Plan *>(pl);
    DeviceGuard dg(p->device);
    return to_status(launch_project_adjoint(*p, psi, y, precision == TOD_PREC_F64, gain, out, stream));
}

tod_status tod_solve_maps(tod_plan *pl, const double *A, const double *b, const int32_t *hits,
                          double rcond_min, double *map_out, void *map_f32_out, double *rcond_out,
                          uint8_t *valid_out, cudaStream_t stream)
{
    if (!pl || !A || !b || !hits || !map_out) return TOD_ERR_ARG;
    Plan *p = reinterpret_cast<Plan *>(pl);
    DeviceGuard dg(p->device);
    return to_status(launch_solve(*p, A, b, hits, rcond_min, map_out, static_cast<float4 *>(map_f32_out),
                                  rcond_out, valid_out, stream));
}

}  // extern "C"
