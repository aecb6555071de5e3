/*
 * Oracle: Huffman coding of differenced integer streams, plain C.
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * CPU-baseline leg of bench.py may load this file's library.
 *
 * Follows paper Sect. 4.1 (in-memory compression): integer streams are
 * differenced sample by sample (d(i) - d(i-1)) and each data segment gets its
 * own Huffman code (Huffman 1952), frequent symbols getting short codes.
 * The concrete format (one canonical code per scan and stream kind, MSB-first
 * 32-bit words, length limit, tie rules) is this project's reading; it is
 * stated once, in words, next to the product encoder and here:
 *
 *   - leaves ordered by (count, symbol value) ascending;
 *   - two-queue Huffman merge: always take the smaller of the heads of the
 *     leaf queue and the merged-node queue, preferring the leaf queue on a
 *     tie of counts;
 *   - if the longest code exceeds maxlen, every count c becomes (c+1)/2 and
 *     the tree is rebuilt, until it fits;
 *   - one distinct symbol gets the 1-bit code "0";
 *   - canonical codes: symbols ordered by (length, value); the first gets the
 *     all-zero code, each next one the previous code plus one, shifted left
 *     by the length increase;
 *   - bits are written most-significant-bit first into 32-bit words.
 *
 * Decoding walks the stream one bit at a time and stops as soon as the bits
 * read so far form a code word: the definition of prefix-code decoding.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct { int64_t count; int32_t order; } qitem;

/* Code lengths of nsym symbols (given sorted by value) from their counts.
 * Returns 0 on success, -1 on bad input. */
int oracle_huff_lengths(const int64_t *counts_in, int32_t nsym, int32_t maxlen,
                        uint8_t *lengths)
{
    if (nsym <= 0 || maxlen < 1 || maxlen > 31) return -1;
    if (nsym == 1) { lengths[0] = 1; return 0; }
    int64_t *counts = (int64_t *)malloc(sizeof(int64_t) * nsym);
    int32_t *leaf = (int32_t *)malloc(sizeof(int32_t) * nsym);      /* leaf order -> symbol */
    int32_t *parent = (int32_t *)malloc(sizeof(int32_t) * 2 * nsym); /* node -> parent node */
    int64_t *ncount = (int64_t *)malloc(sizeof(int64_t) * 2 * nsym);
    for (int32_t i = 0; i < nsym; ++i) counts[i] = counts_in[i] < 1 ? 1 : counts_in[i];
    for (;;) {
        /* order leaves by (count, value): insertion sort, stable on value */
        for (int32_t i = 0; i < nsym; ++i) leaf[i] = i;
        for (int32_t i = 1; i < nsym; ++i) {
            int32_t v = leaf[i]; int32_t j = i - 1;
            while (j >= 0 && counts[leaf[j]] > counts[v]) { leaf[j + 1] = leaf[j]; --j; }
            leaf[j + 1] = v;
        }
        /* nodes 0..nsym-1 are leaves in leaf order, nsym.. merged nodes */
        for (int32_t i = 0; i < nsym; ++i) ncount[i] = counts[leaf[i]];
        int32_t lh = 0, mh = nsym, mt = nsym;   /* leaf head, merged head, merged tail */
        while ((nsym - lh) + (mt - mh) > 1) {
            int32_t pick[2];
            for (int k = 0; k < 2; ++k) {
                int take_leaf;
                if (lh >= nsym) take_leaf = 0;
                else if (mh >= mt) take_leaf = 1;
                else take_leaf = ncount[lh] <= ncount[mh];
                pick[k] = take_leaf ? lh++ : mh++;
            }
            ncount[mt] = ncount[pick[0]] + ncount[pick[1]];
            parent[pick[0]] = mt; parent[pick[1]] = mt;
            ++mt;
        }
        int32_t root = mt - 1;
        int32_t longest = 0;
        for (int32_t i = 0; i < nsym; ++i) {
            int32_t depth = 0, node = i;
            while (node != root) { node = parent[node]; ++depth; }
            lengths[leaf[i]] = (uint8_t)(depth > 255 ? 255 : depth);
            if (depth > longest) longest = depth;
        }
        if (longest <= maxlen) break;
        for (int32_t i = 0; i < nsym; ++i) counts[i] = (counts[i] + 1) / 2;
    }
    free(counts); free(leaf); free(parent); free(ncount);
    return 0;
}

/* Canonical code words for symbols sorted by value with the given lengths. */
int oracle_huff_canonical(const uint8_t *lengths, int32_t nsym, uint32_t *codes)
{
    int32_t *ord = (int32_t *)malloc(sizeof(int32_t) * nsym);
    for (int32_t i = 0; i < nsym; ++i) ord[i] = i;
    /* stable insertion sort by length (values already ascending) */
    for (int32_t i = 1; i < nsym; ++i) {
        int32_t v = ord[i]; int32_t j = i - 1;
        while (j >= 0 && lengths[ord[j]] > lengths[v]) { ord[j + 1] = ord[j]; --j; }
        ord[j + 1] = v;
    }
    uint32_t code = 0; int prev = lengths[ord[0]];
    codes[ord[0]] = 0;
    for (int32_t i = 1; i < nsym; ++i) {
        int L = lengths[ord[i]];
        code = (code + 1) << (L - prev);
        codes[ord[i]] = code;
        prev = L;
    }
    free(ord);
    return 0;
}

static int32_t find_symbol(const int32_t *vals, int32_t nsym, int32_t v)
{
    int32_t lo = 0, hi = nsym - 1;
    while (lo <= hi) {
        int32_t mid = (lo + hi) / 2;
        if (vals[mid] == v) return mid;
        if (vals[mid] < v) lo = mid + 1; else hi = mid - 1;
    }
    return -1;
}

/* Append n symbols to a zero-initialised word buffer, starting at bit
 * position *bitpos (MSB-first).  Returns 0, or -1 on an unknown symbol or
 * buffer overflow. */
int oracle_huff_encode(const int32_t *syms, int64_t n, const int32_t *vals,
                       const uint32_t *codes, const uint8_t *lengths, int32_t nsym,
                       uint32_t *words, int64_t nwords, int64_t *bitpos)
{
    int64_t pos = *bitpos;
    for (int64_t i = 0; i < n; ++i) {
        int32_t s = find_symbol(vals, nsym, syms[i]);
        if (s < 0) return -1;
        int L = lengths[s]; uint32_t c = codes[s];
        for (int b = L - 1; b >= 0; --b) {          /* one bit at a time */
            int64_t w = pos >> 5;
            if (w >= nwords) return -1;
            if ((c >> b) & 1u) words[w] |= 1u << (31 - (pos & 31));
            ++pos;
        }
    }
    *bitpos = pos;
    return 0;
}

/* Decode n symbols starting at bit position bitpos; writes symbol values.
 * Returns the bit position after the last symbol, or -1 if the stream ends or
 * holds a bit string that is no code word. */
int64_t oracle_huff_decode(const uint32_t *words, int64_t nbits, int64_t bitpos,
                           const int32_t *vals, const uint32_t *codes, const uint8_t *lengths,
                           int32_t nsym, int32_t *out, int64_t n)
{
    /* per-length first code, count and first index in (length, value) order */
    int32_t count[33] = {0};
    for (int32_t i = 0; i < nsym; ++i) count[lengths[i]]++;
    int32_t *ord = (int32_t *)malloc(sizeof(int32_t) * nsym);
    int32_t k = 0;
    for (int L = 1; L <= 32; ++L)
        for (int32_t i = 0; i < nsym; ++i)
            if (lengths[i] == L) ord[k++] = i;
    uint32_t first[33] = {0}; int32_t index[33] = {0};
    {
        int32_t idx = 0;
        for (int L = 1; L <= 32; ++L) {
            index[L] = idx;
            first[L] = count[L] ? codes[ord[idx]] : 0;
            idx += count[L];
        }
    }
    int64_t pos = bitpos;
    for (int64_t i = 0; i < n; ++i) {
        uint32_t code = 0; int L = 0; int found = 0;
        while (L < 32) {
            if (pos >= nbits) { free(ord); return -1; }
            uint32_t bit = (words[pos >> 5] >> (31 - (pos & 31))) & 1u;
            ++pos; ++L;
            code = (code << 1) | bit;
            if (count[L] && code >= first[L] && code - first[L] < (uint32_t)count[L]) {
                out[i] = vals[ord[index[L] + (int32_t)(code - first[L])]];
                found = 1;
                break;
            }
        }
        if (!found) { free(ord); return -1; }
    }
    free(ord);
    return pos;
}
