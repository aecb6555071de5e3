// Device helpers shared by the library's kernels: status words, the Philox
// counter RNG, FP32 Box-Muller normals, FP32 double-word accumulation and
// small complex arithmetic.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace tg {

// ---------------------------------------------------------------------------
// division by a runtime constant: q = (umulhi(x, mul) + x) >> shift, exact for
// 0 <= x < 2^31 (round-up multiplier method, Granlund & Montgomery 1994)
// ---------------------------------------------------------------------------
struct FastDiv {
    uint32_t d, mul, shift;
};
inline FastDiv make_fastdiv(uint32_t d) {
    FastDiv f;
    f.d = d;
    uint32_t s = 0;
    while ((1ull << s) < d) ++s;
    f.shift = s;
    f.mul = static_cast<uint32_t>((((1ull << 32) * ((1ull << s) - d)) / d) + 1);
    return f;
}
__device__ __forceinline__ FastDiv make_fastdiv_dev(uint32_t d) {
    FastDiv f;
    f.d = d;
    uint32_t s = 0;
    while ((1ull << s) < d) ++s;
    f.shift = s;
    f.mul = static_cast<uint32_t>((((1ull << 32) * ((1ull << s) - d)) / d) + 1);
    return f;
}
__device__ __forceinline__ int fdiv(int x, const FastDiv &f) {
    const uint32_t ux = static_cast<uint32_t>(x);
    return static_cast<int>((__umulhi(ux, f.mul) + ux) >> f.shift);
}

// ---------------------------------------------------------------------------
// per-detscan status words (device): first error wins, never a trap
// ---------------------------------------------------------------------------
__device__ __forceinline__ void set_status(int32_t *status, int q, int32_t code) {
    if (status) atomicCAS(reinterpret_cast<int *>(status + q), 0, code);
}

// ---------------------------------------------------------------------------
// Philox4x64-10 (Salmon, Moraes, Dror, Shaw, SC'11): 10 rounds of
// multiply-hi/lo with two Weyl-sequence key bumps.
// ---------------------------------------------------------------------------
struct u64x4 { uint64_t x[4]; };

__device__ __forceinline__ u64x4 philox4x64(uint64_t c0, uint64_t c1, uint64_t c2, uint64_t c3,
                                             uint64_t k0, uint64_t k1) {
    const uint64_t M0 = 0xD2E7470EE14C6C93ull, M1 = 0xCA5A826395121157ull;
    const uint64_t W0 = 0x9E3779B97F4A7C15ull, W1 = 0xBB67AE8584CAA73Bull;
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r) { k0 += W0; k1 += W1; }
        const uint64_t hi0 = __umul64hi(M0, c0), lo0 = M0 * c0;
        const uint64_t hi1 = __umul64hi(M1, c2), lo1 = M1 * c2;
        const uint64_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
        c0 = n0; c1 = lo1; c2 = n2; c3 = lo0;
    }
    u64x4 o; o.x[0] = c0; o.x[1] = c1; o.x[2] = c2; o.x[3] = c3;
    return o;
}

// Normals 2j, 2j+1 (j = 0..3) of a Philox block: 32-bit halves h (low half
// of each word first) give uniforms u = ((h >> 9) + 1/2) 2^-23 (exact in
// FP32), and the pair is sqrt(-2 ln u1) (cos 2 pi u2, sin 2 pi u2).
// FP32 on the SFU: ln u1 from lg2.approx (absolute error about 2^-22.6 in
// log2 u1), or for 1 - u1 = v < 2^-10 from -v - v^2/2 (v exact, truncation
// below 3e-7 relative), where a fixed absolute error would dominate;
// sqrt(t) = t rsqrt.approx(t); the angle 2 pi u2 = pi + 2 pi (u2 - 1/2)
// reduced to [-pi, pi) for sin/cos.approx (absolute error about 2^-20.9).
// A normal's error stays near 1e-6 absolute, far inside the draws' FP32
// transform budget.
__device__ __forceinline__ float2 philox_normal_pair(const u64x4 &w, int j) {
    const uint64_t word = w.x[j];
    const uint32_t h0 = static_cast<uint32_t>(word), h1 = static_cast<uint32_t>(word >> 32);
    const float u1 = (static_cast<float>(h0 >> 9) + 0.5f) * 1.1920928955078125e-07f;  // 2^-23
    const float v1 = (static_cast<float>(0x7FFFFFu - (h0 >> 9)) + 0.5f) * 1.1920928955078125e-07f;  // 1 - u1
    const float u2 = (static_cast<float>(h1 >> 9) + 0.5f) * 1.1920928955078125e-07f;
    float lg;
    asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(lg) : "f"(u1));
    const float lnu = v1 < 9.765625e-4f ? -v1 * fmaf(0.5f, v1, 1.0f) : 0.69314718055994531f * lg;
    const float t = -2.0f * lnu;                       // > 0
    float rs;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(rs) : "f"(t));
    const float r = t * rs;
    const float ang = 6.28318530717958648f * (u2 - 0.5f);
    float sn, cs;
    asm("sin.approx.ftz.f32 %0, %1;" : "=f"(sn) : "f"(ang));
    asm("cos.approx.ftz.f32 %0, %1;" : "=f"(cs) : "f"(ang));
    return make_float2(-r * cs, -r * sn);
}

// The pair of normals (2i', 2i'+1) with i' = idx/2 of stream (q, purpose, it);
// idx must be even.
__device__ __forceinline__ float2 stream_normal_pair(uint64_t seed, uint64_t band, uint64_t q,
                                                     uint64_t purpose, uint64_t it, int64_t idx) {
    const u64x4 w = philox4x64(static_cast<uint64_t>(idx >> 3), q, purpose, it, seed, band);
    return philox_normal_pair(w, static_cast<int>((idx & 7) >> 1));
}

// ---------------------------------------------------------------------------
// FP32 double-word accumulation (Dekker 1971 / Knuth two-sum): sums of exact
// FP32 values and exact FP32 products with ~2^-44 relative error, for FP64-
// accurate pixel sums at FP32 issue rate.
// ---------------------------------------------------------------------------
struct Acc2 { float s, c; };

__device__ __forceinline__ void acc_add(Acc2 &a, float v) {
    const float s = __fadd_rn(a.s, v);
    const float bb = __fsub_rn(s, a.s);
    const float e = __fadd_rn(__fsub_rn(a.s, __fsub_rn(s, bb)), __fsub_rn(v, bb));
    a.s = s;
    a.c = __fadd_rn(a.c, e);
}
// add the exact product x*y
__device__ __forceinline__ void acc_add_prod(Acc2 &a, float x, float y) {
    const float p = __fmul_rn(x, y);
    const float e = __fmaf_rn(x, y, -p);
    acc_add(a, p);
    a.c = __fadd_rn(a.c, e);
}
__device__ __forceinline__ double acc_value(const Acc2 &a) {
    return static_cast<double>(a.s) + static_cast<double>(a.c);
}

// ---------------------------------------------------------------------------
// complex
// ---------------------------------------------------------------------------
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ float2 cmulc(float2 a, float2 b) {  // a * conj(b)
    return make_float2(a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y);
}
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cconj(float2 a) { return make_float2(a.x, -a.y); }
__device__ __forceinline__ float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }
// e^{i pi x}
__device__ __forceinline__ float2 cexpi_pi(float x) {
    float s, c;
    sincospif(x, &s, &c);
    return make_float2(c, s);
}

}  // namespace tg
