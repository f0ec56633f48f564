// Register-blocked 1-D Gaussian passes and async-copy helpers shared by the FP32 kernels.
//
// Both passes are the real 1-D Gaussian smoothing S * g of the paper's decomposition
// (Eq. 5-6 along rows, Eq. 7-9 along columns): a thread produces 8 consecutive outputs,
// walks the taps in chunks of 8 (taps zero-padded to a multiple of 8) and keeps a 16-sample
// window in two register banks used in ping-pong order, so every shared-memory load feeds 8
// FMAs per signal and no register is copied.
#pragma once

#include <cuda_runtime.h>
#include <cstdint>

namespace gb {

// Two independent round-to-nearest FMAs in one packed FP32x2 instruction (sm_100+): the same
// results as two fmaf calls, half the issue slots.  The compiler intrinsic lets register
// allocation keep operand pairs in place (no packing moves).
__device__ __forceinline__ float2 ffma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }

__device__ __forceinline__ float4 fmav(float4 w, float t, float4 a)
{
    const float2 tt = make_float2(t, t);
    const float2 lo = ffma2(make_float2(w.x, w.y), tt, make_float2(a.x, a.y));
    const float2 hi = ffma2(make_float2(w.z, w.w), tt, make_float2(a.z, a.w));
    return make_float4(lo.x, lo.y, hi.x, hi.y);
}
__device__ __forceinline__ float2 fmav(float2 w, float t, float2 a)
{
    return ffma2(w, make_float2(t, t), a);
}

// acc[j] += sum_d win[j + d] * t[d] for the 8 taps of one chunk; win = lo[0..7] ++ hi[0..7].
// The products that only need `lo` come first, so the loads of `hi` (issued just before the
// call) have 36 FMA groups of slack; j runs innermost so consecutive FMAs are independent.
template <typename V>
__device__ __forceinline__ void conv_step(const V (&lo)[8], const V (&hi)[8], const float4 t0, const float4 t1,
                                          V (&acc)[8])
{
    const float t[8] = {t0.x, t0.y, t0.z, t0.w, t1.x, t1.y, t1.z, t1.w};
#pragma unroll
    for (int d = 0; d < 8; ++d)
#pragma unroll
        for (int j = 0; j < 8 - d; ++j) acc[j] = fmav(lo[j + d], t[d], acc[j]);
#pragma unroll
    for (int d = 1; d < 8; ++d)
#pragma unroll
        for (int j = 8 - d; j < 8; ++j) acc[j] = fmav(hi[j + d - 8], t[d], acc[j]);
}

// Contiguous source (row pass): out[j] = sum_t src[j + t] * taps[t], j < 8.
// Reads src[0 .. 8 * nchunks + 7].  Window and taps of the next chunk are loaded one chunk
// ahead; two register banks alternate (no copies).  tail: one more tap, taps[8 nchunks]
// (filters of 8 k + 1 taps), applied to the window bank already loaded.
template <typename V>
__device__ __forceinline__ void conv8_linear(const V *__restrict__ src, const float4 *__restrict__ taps4,
                                             int nchunks, V (&acc)[8], bool tail = false)
{
    V wa[8], wb[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) wa[i] = src[i];
    float4 t0 = taps4[0], t1 = taps4[1];
    int c = 0;
    for (; c + 2 <= nchunks; c += 2) {
#pragma unroll
        for (int i = 0; i < 8; ++i) wb[i] = src[8 * (c + 1) + i];
        const float4 u0 = taps4[2 * c + 2], u1 = taps4[2 * c + 3];
        conv_step(wa, wb, t0, t1, acc);
#pragma unroll
        for (int i = 0; i < 8; ++i) wa[i] = src[8 * (c + 2) + i];
        t0 = taps4[2 * c + 4];
        t1 = taps4[2 * c + 5];
        conv_step(wb, wa, u0, u1, acc);
    }
    if (c < nchunks) {
#pragma unroll
        for (int i = 0; i < 8; ++i) wb[i] = src[8 * (c + 1) + i];
        conv_step(wa, wb, t0, t1, acc);
    }
    if (tail) {
        const float t = reinterpret_cast<const float *>(taps4)[8 * nchunks];
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[j] = fmav((nchunks & 1) ? wb[j] : wa[j], t, acc[j]);
    }
}

// Ring source (column pass): row r of the window is ring[slot(r) * STRIDE], slots advance
// by 8 per chunk modulo RS.  slot0 and RS are multiples of 8, so a chunk never wraps.  STRIDE
// is a compile-time constant so the 8 loads of a chunk use immediate offsets.  tail: as in
// conv8_linear.
template <typename V, int STRIDE>
__device__ __forceinline__ void conv8_ring(const V *__restrict__ ring, int RS, int slot0,
                                           const float4 *__restrict__ taps4, int nchunks, V (&acc)[8],
                                           bool tail = false)
{
    V wa[8], wb[8];
    int s = slot0;
    auto adv = [&]() {
        s += 8;
        if (s >= RS) s -= RS;
    };
    const V *p = ring + s * STRIDE;
#pragma unroll
    for (int i = 0; i < 8; ++i) wa[i] = p[i * STRIDE];
    float4 t0 = taps4[0], t1 = taps4[1];
    int c = 0;
    for (; c + 2 <= nchunks; c += 2) {
        adv();
        p = ring + s * STRIDE;
#pragma unroll
        for (int i = 0; i < 8; ++i) wb[i] = p[i * STRIDE];
        const float4 u0 = taps4[2 * c + 2], u1 = taps4[2 * c + 3];
        conv_step(wa, wb, t0, t1, acc);
        adv();
        p = ring + s * STRIDE;
#pragma unroll
        for (int i = 0; i < 8; ++i) wa[i] = p[i * STRIDE];
        t0 = taps4[2 * c + 4];
        t1 = taps4[2 * c + 5];
        conv_step(wb, wa, u0, u1, acc);
    }
    if (c < nchunks) {
        adv();
        p = ring + s * STRIDE;
#pragma unroll
        for (int i = 0; i < 8; ++i) wb[i] = p[i * STRIDE];
        conv_step(wa, wb, t0, t1, acc);
    }
    if (tail) {
        const float t = reinterpret_cast<const float *>(taps4)[8 * nchunks];
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[j] = fmav((nchunks & 1) ? wb[j] : wa[j], t, acc[j]);
    }
}

// Complex taps over a real window (the row pass in modulated-tap form): acc[j] += win[j + d] g[d]
// for the 8 complex taps of one chunk, win = lo[0..7] ++ hi[0..7]; one packed FMA per product.
__device__ __forceinline__ void conv_step_ct(const float (&lo)[8], const float (&hi)[8], const float2 (&g)[8],
                                             float2 (&acc)[8])
{
#pragma unroll
    for (int d = 0; d < 8; ++d)
#pragma unroll
        for (int j = 0; j < 8 - d; ++j) acc[j] = ffma2(g[d], make_float2(lo[j + d], lo[j + d]), acc[j]);
#pragma unroll
    for (int d = 1; d < 8; ++d)
#pragma unroll
        for (int j = 8 - d; j < 8; ++j) acc[j] = ffma2(g[d], make_float2(hi[j + d - 8], hi[j + d - 8]), acc[j]);
}

__device__ __forceinline__ void load_ctaps(float2 (&g)[8], const float4 *__restrict__ g4)
{
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const float4 v = g4[i];
        g[2 * i] = make_float2(v.x, v.y);
        g[2 * i + 1] = make_float2(v.z, v.w);
    }
}

// Contiguous real source, complex taps: out[j] = sum_t src[j + t] g[t], j < 8.  Reads
// src[0 .. 8 * nchunks + 7] and g[0 .. 8 * nchunks + 7] (g4: two complex taps per float4).
// tail: as in conv8_linear.
__device__ __forceinline__ void conv8_linear_ct(const float *__restrict__ src, const float4 *__restrict__ g4,
                                                int nchunks, float2 (&acc)[8], bool tail = false)
{
    float wa[8], wb[8];
    float2 ga[8], gb[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) wa[i] = src[i];
    load_ctaps(ga, g4);
    int c = 0;
    for (; c + 2 <= nchunks; c += 2) {
#pragma unroll
        for (int i = 0; i < 8; ++i) wb[i] = src[8 * (c + 1) + i];
        load_ctaps(gb, g4 + 4 * (c + 1));
        conv_step_ct(wa, wb, ga, acc);
#pragma unroll
        for (int i = 0; i < 8; ++i) wa[i] = src[8 * (c + 2) + i];
        load_ctaps(ga, g4 + 4 * (c + 2));
        conv_step_ct(wb, wa, gb, acc);
    }
    if (c < nchunks) {
#pragma unroll
        for (int i = 0; i < 8; ++i) wb[i] = src[8 * (c + 1) + i];
        conv_step_ct(wa, wb, ga, acc);
    }
    if (tail) {   // one more tap, g[8 nchunks] (filters of 8 k + 1 taps), on the loaded bank
        const float2 g = reinterpret_cast<const float2 *>(g4)[8 * nchunks];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const float w = (nchunks & 1) ? wb[j] : wa[j];
            acc[j] = ffma2(g, make_float2(w, w), acc[j]);
        }
    }
}

// conv8_linear_ct with the window read as float4 (src 16-byte aligned): two 16-byte loads per
// 8 samples instead of eight 4-byte ones.  Rows of the source that are = 4 (mod 32) floats
// apart keep the loads of 8 lanes on 8 different rows conflict-free.  Same arithmetic, same order.
__device__ __forceinline__ void load8(float (&w)[8], const float *__restrict__ p)
{
    const float4 a = reinterpret_cast<const float4 *>(p)[0], b = reinterpret_cast<const float4 *>(p)[1];
    w[0] = a.x; w[1] = a.y; w[2] = a.z; w[3] = a.w;
    w[4] = b.x; w[5] = b.y; w[6] = b.z; w[7] = b.w;
}
__device__ __forceinline__ void conv8_linear_ct4(const float *__restrict__ src, const float4 *__restrict__ g4,
                                                 int nchunks, float2 (&acc)[8], bool tail = false)
{
    float wa[8], wb[8];
    float2 ga[8], gb[8];
    load8(wa, src);
    load_ctaps(ga, g4);
    int c = 0;
    for (; c + 2 <= nchunks; c += 2) {
        load8(wb, src + 8 * (c + 1));
        load_ctaps(gb, g4 + 4 * (c + 1));
        conv_step_ct(wa, wb, ga, acc);
        load8(wa, src + 8 * (c + 2));
        load_ctaps(ga, g4 + 4 * (c + 2));
        conv_step_ct(wb, wa, gb, acc);
    }
    if (c < nchunks) {
        load8(wb, src + 8 * (c + 1));
        conv_step_ct(wa, wb, ga, acc);
    }
    if (tail) {
        const float2 g = reinterpret_cast<const float2 *>(g4)[8 * nchunks];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const float w = (nchunks & 1) ? wb[j] : wa[j];
            acc[j] = ffma2(g, make_float2(w, w), acc[j]);
        }
    }
}

// Complex taps over a ring of complex rows J (the SDFT column pass in modulated-tap form), for
// 8 consecutive outputs: with taps g = (Gr, Gi, Gi, Gr),
//   ac[j] += (Gr Jr, Gi Jr),  bd[j] += (Gi Ji, Gr Ji)
// so that sum g J = (ac.x - bd.x, ac.y + bd.y) and sum g conj(J) = (ac.x + bd.x, ac.y - bd.y).
__device__ __forceinline__ void conv_step_cc(const float2 (&lo)[8], const float2 (&hi)[8],
                                             const float4 *__restrict__ g4, float2 (&ac)[8], float2 (&bd)[8])
{
#pragma unroll
    for (int d = 0; d < 8; ++d) {
        const float4 g = g4[d];
        const float2 gri = make_float2(g.x, g.y), gir = make_float2(g.z, g.w);
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const float2 w = j + d < 8 ? lo[j + d] : hi[j + d - 8];
            ac[j] = ffma2(gri, make_float2(w.x, w.x), ac[j]);
            bd[j] = ffma2(gir, make_float2(w.y, w.y), bd[j]);
        }
    }
}

// Ring source of complex rows (see conv8_ring): out = the four real sums of conv_step_cc over
// 8 * nchunks taps; reads g4[0 .. 8 * nchunks - 1].
template <int STRIDE>
__device__ __forceinline__ void conv8_ring_cc(const float2 *__restrict__ ring, int RS, int slot0,
                                              const float4 *__restrict__ g4, int nchunks, float2 (&ac)[8],
                                              float2 (&bd)[8])
{
    float2 wa[8], wb[8];
    int s = slot0;
    auto adv = [&]() {
        s += 8;
        if (s >= RS) s -= RS;
    };
    const float2 *p = ring + s * STRIDE;
#pragma unroll
    for (int i = 0; i < 8; ++i) wa[i] = p[i * STRIDE];
    int c = 0;
    for (; c + 2 <= nchunks; c += 2) {
        adv();
        p = ring + s * STRIDE;
#pragma unroll
        for (int i = 0; i < 8; ++i) wb[i] = p[i * STRIDE];
        conv_step_cc(wa, wb, g4 + 8 * c, ac, bd);
        adv();
        p = ring + s * STRIDE;
#pragma unroll
        for (int i = 0; i < 8; ++i) wa[i] = p[i * STRIDE];
        conv_step_cc(wb, wa, g4 + 8 * (c + 1), ac, bd);
    }
    if (c < nchunks) {
        adv();
        p = ring + s * STRIDE;
#pragma unroll
        for (int i = 0; i < 8; ++i) wb[i] = p[i * STRIDE];
        conv_step_cc(wa, wb, g4 + 8 * c, ac, bd);
    }
}

// 4-byte global -> shared async copy; src_bytes = 0 writes a zero without reading.
__device__ __forceinline__ void cp_async4(void *smem, const void *gmem, int src_bytes)
{
    const unsigned s = static_cast<unsigned>(__cvta_generic_to_shared(smem));
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(s), "l"(gmem), "r"(src_bytes)
                 : "memory");
}
// 16-byte global -> shared async copy (both addresses 16-byte aligned).
__device__ __forceinline__ void cp_async16(void *smem, const void *gmem)
{
    const unsigned s = static_cast<unsigned>(__cvta_generic_to_shared(smem));
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}

__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

__host__ __device__ constexpr int round_up(int a, int b) { return (a + b - 1) / b * b; }

// Staging row width: at least need float2, and = 1 (mod 16) so that the 8 rows x 2 column
// groups of a half-warp fall on distinct bank pairs.
__host__ __device__ constexpr int stage_width(int need) { return round_up(need - 1, 16) + 1; }

}  // namespace gb
