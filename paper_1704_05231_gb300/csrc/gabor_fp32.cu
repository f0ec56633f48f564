// Fused FP32 Gabor filter-bank kernel (K1 + K2): Algorithm 1 of arXiv 1704.05231 for one
// frequency omega_s, all orientations, on FP32 CUDA cores.
//
// A CTA owns one horizontal pass ("unit": orientation theta_a and, when present, its
// mirror pi - theta_a), one strip of 32 image columns and one segment of rows.  It walks
// down the segment in chunks of TH rows:
//
//   row pass  (Eq. 5-6)   stage f * (cos, sin)(omega^c k) for the chunk's rows and the
//                         strip's columns plus an R-wide halo; smooth both signals with the
//                         real Gaussian S (8 outputs x 8 taps register blocks); remodulate
//                         into J_theta (Eq. 5-6) and immediately demodulate by
//                         (cos, sin)(omega^s y) into the column signals of Eq. 10:
//                             f_cr + f_si, f_sr - f_ci            (theta_a,   Eq. 7-9)
//                             f_cr - f_si, f_sr + f_ci            (pi - theta_a, Eq. 15-16)
//                         which go into a ring buffer of rows in shared memory.  J never
//                         leaves the chip; J_{pi-theta} = J*_theta (Eq. 13) costs nothing.
//   column pass (Eq. 7-9) smooth the ring's signals along y with S, remodulate by
//                         (cos, sin)(omega^s y) and store F_theta_a (and F_{pi-theta_a}).
//
// The ring keeps the 2R rows of vertical halo between chunks, so every row's horizontal pass
// is computed once per segment (plus 2R rows of prologue per segment).
#include "internal.h"
#include "conv_fp32.cuh"

namespace gb {

namespace {

struct Smem {
    float4 *ring4;
    float2 *ring2;
    float2 *stage;
    float2 *phx;
    float *taps;
};

__device__ __forceinline__ Smem carve(unsigned char *raw, const GaborArgs &a)
{
    Smem s;
    s.ring4 = reinterpret_cast<float4 *>(raw);
    s.ring2 = reinterpret_cast<float2 *>(raw);
    s.stage = reinterpret_cast<float2 *>(s.ring4 + (size_t)a.RS * (kStripW + 1));
    s.phx = s.stage + (size_t)a.TH * a.SW;
    s.taps = reinterpret_cast<float *>(s.phx + a.SW + 1);
    return s;
}

}  // namespace

size_t gabor_fp32_smem_bytes(int TH, int RS, int SW, int Tpad)
{
    return (size_t)RS * (kStripW + 1) * sizeof(float4) + (size_t)TH * SW * sizeof(float2) +
           (size_t)(SW + 1) * sizeof(float2) + (size_t)(Tpad + 8) * sizeof(float);
}

__global__ void __launch_bounds__(kThreads) k_gabor_fp32(const GaborArgs a)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const UnitDev u = a.units[blockIdx.z];
    const bool paired = u.plane_b >= 0;
    const int x0 = blockIdx.x * kStripW;
    const int ys = blockIdx.y * a.seg_len;
    if (ys >= a.H) return;
    const int ye = min(a.H, ys + a.seg_len);
    const int tid = threadIdx.x;
    const int stride = kStripW + 1;
    const Smem sm = carve(smem_raw, a);
    const float4 *taps4 = reinterpret_cast<const float4 *>(sm.taps);
    const int nchunks = a.Tpad / 8;

    for (int i = tid; i < a.Tpad + 8; i += kThreads) sm.taps[i] = i < a.Tpad ? a.taps[i] : 0.f;
    for (int j = tid; j <= a.SW; j += kThreads) {
        const int gx = x0 - a.R + j;
        sm.phx[j] = (j < a.SW && gx >= 0 && gx < a.W) ? u.phx[gx] : make_float2(0.f, 0.f);
    }
    for (int i = tid; i < a.RS * stride; i += kThreads) sm.ring4[i] = make_float4(0.f, 0.f, 0.f, 0.f);
    __syncthreads();

    const int ring_origin = ys - a.R;   // absolute row of ring slot 0
    const int ncols = kStripW + a.T - 1;

    // Horizontal pass for rows [r0, r0 + nrows), nrows <= TH.
    auto row_block = [&](int r0, int nrows) {
        const int warp = tid >> 5, lane = tid & 31;
        for (int r = warp; r < nrows; r += kThreads / 32) {
            const int y = r0 + r;
            const bool yin = y >= 0 && y < a.H;
            const float *src = a.img + (int64_t)(yin ? y : 0) * a.pitch;
            float2 *dst = sm.stage + (size_t)r * a.SW;
            for (int j = lane; j < a.SW; j += 32) {
                const int gx = x0 - a.R + j;
                float v = 0.f;
                if (yin && j < ncols && gx >= 0 && gx < a.W) v = __ldg(src + gx);
                const float2 ph = sm.phx[j];
                dst[j] = make_float2(v * ph.x, v * ph.y);   // f_c, f_s of Eq. 5
            }
        }
        __syncthreads();
        const int r = (tid & 7) | ((tid >> 5) << 3);
        const int q = (tid >> 3) & 3;
        if (r < nrows) {
            float2 acc[8];
#pragma unroll
            for (int j = 0; j < 8; ++j) acc[j] = make_float2(0.f, 0.f);
            row_conv8(sm.stage + (size_t)r * a.SW + 8 * q, taps4, nchunks, acc);
            const int y = r0 + r;
            const int slot = (y - ring_origin) % a.RS;
            const int base = slot * stride + 8 * q;
            const bool yin = y >= 0 && y < a.H;
            const float2 cy = yin ? u.phy[y] : make_float2(0.f, 0.f);
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const float2 px = sm.phx[a.R + 8 * q + j];
                const float A = acc[j].x, B = acc[j].y;
                // Eq. 5-6: Re J = cos A + sin B, Im J = sin A - cos B
                const float jr = fmaf(px.x, A, px.y * B);
                const float ji = fmaf(px.y, A, -px.x * B);
                // Eq. 10: f_cr, f_sr, f_ci, f_si
                const float fcr = jr * cy.x, fsr = jr * cy.y, fci = ji * cy.x, fsi = ji * cy.y;
                if (paired)
                    sm.ring4[base + j] = make_float4(fcr + fsi, fsr - fci, fcr - fsi, fsr + fci);
                else
                    sm.ring2[base + j] = make_float2(fcr + fsi, fsr - fci);
            }
        }
        __syncthreads();
    };

    // Vertical pass for output rows [c, c + nout).
    auto col_pass = [&](int c, int nout) {
        const int xl = tid & 31, yg = tid >> 5;
        const int x = x0 + xl;
        for (int yb = 8 * yg; yb < nout; yb += 8 * (kThreads / 32)) {
            const int slot0 = (c - ys + yb) % a.RS;
            if (paired) {
                float4 acc[8];
#pragma unroll
                for (int j = 0; j < 8; ++j) acc[j] = make_float4(0.f, 0.f, 0.f, 0.f);
                col_conv8<float4>(sm.ring4 + xl, stride, a.RS, slot0, taps4, nchunks, acc);
                if (x < a.W) {
                    float2 *oa = a.out + (int64_t)u.plane_a * a.plane + x;
                    float2 *ob = a.out + (int64_t)u.plane_b * a.plane + x;
#pragma unroll
                    for (int j = 0; j < 8; ++j) {
                        const int y = c + yb + j;
                        if (y < c + nout && y < a.H) {
                            const float2 cy = u.phy[y];
                            const float P = acc[j].x, Q = acc[j].y, P2 = acc[j].z, Q2 = acc[j].w;
                            // Eq. 7-8 and Eq. 15-16
                            __stcs(oa + (int64_t)y * a.W,
                                   make_float2(fmaf(cy.x, P, cy.y * Q), fmaf(cy.y, P, -cy.x * Q)));
                            __stcs(ob + (int64_t)y * a.W,
                                   make_float2(fmaf(cy.x, P2, cy.y * Q2), fmaf(cy.y, P2, -cy.x * Q2)));
                        }
                    }
                }
            } else {
                float2 acc[8];
#pragma unroll
                for (int j = 0; j < 8; ++j) acc[j] = make_float2(0.f, 0.f);
                col_conv8<float2>(sm.ring2 + xl, stride, a.RS, slot0, taps4, nchunks, acc);
                if (x < a.W) {
                    float2 *oa = a.out + (int64_t)u.plane_a * a.plane + x;
#pragma unroll
                    for (int j = 0; j < 8; ++j) {
                        const int y = c + yb + j;
                        if (y < c + nout && y < a.H) {
                            const float2 cy = u.phy[y];
                            const float P = acc[j].x, Q = acc[j].y;
                            __stcs(oa + (int64_t)y * a.W,
                                   make_float2(fmaf(cy.x, P, cy.y * Q), fmaf(cy.y, P, -cy.x * Q)));
                        }
                    }
                }
            }
        }
    };

    int next = ring_origin;
    for (int c = ys; c < ye; c += a.TH) {
        const int nout = min(a.TH, ye - c);
        const int need = c + nout + a.R;
        while (next < need) {
            const int n = min(a.TH, need - next);
            row_block(next, n);
            next += n;
        }
        col_pass(c, nout);
        __syncthreads();
    }
}

GaborLaunchCfg gabor_fp32_config(int H, int W, int R, int Tpad, int nunits, int tile_rows,
                                 int segments, int sm_count)
{
    GaborLaunchCfg cfg;
    const int T = 2 * R + 1;
    int TH = tile_rows > 0 ? tile_rows : (R <= 64 ? 64 : 32);
    for (;;) {
        cfg.TH = TH;
        cfg.RS = round_up(TH + T - 1, 8);
        cfg.SW = stage_width(kStripW + Tpad);
        cfg.smem = gabor_fp32_smem_bytes(TH, cfg.RS, cfg.SW, Tpad);
        if (cfg.smem <= (size_t)kSmemLimit || TH <= 8) break;
        TH /= 2;
    }
    const int cps = std::max(1, std::min(8, (int)(kSmemLimit / (cfg.smem + 1024))));
    const int nstrips = (W + kStripW - 1) / kStripW;
    const int64_t base = (int64_t)nstrips * nunits;
    int nseg = 1;
    if (segments > 0) {
        nseg = segments;
    } else {
        const int64_t target = 2LL * sm_count * cps;
        const int min_len = std::max(TH, 2 * (T - 1));
        while (base * nseg < target && H / (nseg + 1) >= min_len) ++nseg;
    }
    nseg = std::max(1, std::min(nseg, H));
    cfg.seg_len = (H + nseg - 1) / nseg;
    cfg.nseg = (H + cfg.seg_len - 1) / cfg.seg_len;
    return cfg;
}

cudaError_t gabor_fp32_prepare()
{
    return cudaFuncSetAttribute(k_gabor_fp32, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                kSmemLimit);
}

cudaError_t launch_gabor_fp32(const GaborArgs &a0, int nunits, const GaborLaunchCfg &cfg,
                              cudaStream_t st)
{
    GaborArgs a = a0;
    a.TH = cfg.TH;
    a.seg_len = cfg.seg_len;
    a.RS = cfg.RS;
    a.SW = cfg.SW;
    const dim3 grid((a.W + kStripW - 1) / kStripW, cfg.nseg, nunits);
    k_gabor_fp32<<<grid, kThreads, cfg.smem, st>>>(a);
    return cudaGetLastError();
}

}  // namespace gb
