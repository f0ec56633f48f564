// FP32 localized sliding DFT (K3 + K4): Algorithm 2 of arXiv 1704.05231 on CUDA cores.
//
// A CTA owns one horizontal frequency u in [0, Mx/2], one strip of 32 columns and one
// segment of rows, and walks down the segment in chunks of TH rows:
//
//   row pass (Eq. 19, 21-22)  J_u(x) = exp(i w0 u xhat) [S * f_c - i S * f_s](x) with
//                             f_c, f_s = f(m) (cos, sin)(w0 u m); twiddle indices are the
//                             exact integers (u m) mod Mx.  J_u goes to a ring of rows.
//   for each v in [0, My/2]   (J_u is reused for every v, Sec. III-B)
//     demodulate (Eq. 23-24) J_u(x, n) by (cos, sin)(w0 v n) into the four signals of the
//                             pair (u, Mx - u): J_{Mx-u} = J*_u (Eq. 25-26);
//     column pass             smooth them with S along y, remodulate by
//                             exp(i w0 v yhat) and store F_{u,v}, F_{Mx-u,v};
//     conjugate fill          F_{(Mx-u)%Mx, My-v} = F*_{u,v} and F_{u, My-v} = F*_{Mx-u,v}
//                             for 0 < v < My/2 (Algorithm 2, last loop).
//
// With the FIR passes used here each demodulate / smooth / remodulate triple is one
// convolution with modulated taps: J_u(x) = sum_a S(a - Mx/2) e^{-i w0 u a} f(xhat + a) and
// F_{u,v}(y) = sum_b S(b - My/2) e^{-i w0 v b} J_u(yhat + b), F_{Mx-u,v} the same sum over
// J*_u (twiddles from the exact integers (u a) mod Mx, (v b) mod My).  That form (the
// default) reads J_u straight from its ring for every v, with no demodulated copy of the
// window and no barrier between the v passes; the step-by-step form is kept as an option.
//
// No-reuse ablation (GB_OPT_SDFT_REUSE = 0): the reuse of Sec. III-B switched off.  Every
// (u, v) with u in [0, Mx) and v in [0, My/2] gets its own CTAs, which compute the row pass
// J_u for that v alone and derive nothing from J*_u; the conjugate fill of the v > My/2 half
// (F_{u,v} = F*_{Mx-u,My-v}) stays, as in the paper's own comparison (Table III).
//
// Filter order (Sec. III-B): the pass over the first axis runs for M/2 + 1 frequencies, the
// second for all M of the first times M/2 + 1 of its own.  With the FIR passes used here the
// first pass needs fewer FMAs along the longer window side; on request (vertical first) the
// host runs this kernel on the transposed image and the stores transpose back.
#include "internal.h"
#include "conv_fp32.cuh"

namespace gb {

namespace {

__device__ __forceinline__ int pmod(int a, int m)
{
    const int r = a % m;
    return r < 0 ? r + m : r;
}

size_t sdft_smem_bytes(int TH, int RS, int SW, int RW, int TpadX, int TpadY, int My)
{
    return (size_t)RS * (kStripW + 1) * (sizeof(float2) + sizeof(float4)) +
           (size_t)TH * SW * sizeof(float2) + (size_t)2 * TH * RW * sizeof(float) +
           (size_t)(SW + 1) * sizeof(float2) + (size_t)(TpadX + 8 + TpadY + 8) * sizeof(float) +
           (size_t)(My / 2 + 1) * My * sizeof(float2) + (size_t)round_up(RS, 4) * sizeof(int);
}

// Modulated-tap form: J ring, raw rows, row taps (complex), column taps per v as
// (Gr, Gi, Gi, Gr).  Every region starts on a 16-byte boundary.
size_t sdft_mt_smem_bytes(int TH, int RS, int RW, int TpadX, int TpadY, int My)
{
    return (size_t)RS * (kStripW + 1) * sizeof(float2) + (size_t)2 * TH * RW * sizeof(float) +
           (size_t)(TpadX + 8) * sizeof(float2) + (size_t)(My / 2 + 1) * (TpadY + 8) * sizeof(float4);
}

}  // namespace

// Step-by-step form: demodulate, smooth with the real Gaussian, remodulate, in both passes.
__device__ __forceinline__ void sdft_demod_form(const SdftArgs &a, unsigned char *smem_raw)
{
    const int Mx = a.Mx, My = a.My;
    const int nvz = My / 2 + 1;
    // u in 0 .. Mx/2 (reuse), or the (u, v) of this CTA in the no-reuse ablation
    const int u = a.noreuse ? (int)blockIdx.z / nvz : (int)blockIdx.z;
    const int v_lo = a.noreuse ? (int)blockIdx.z % nvz : 0, v_hi = a.noreuse ? v_lo + 1 : nvz;
    // J_0 and J_{Mx/2} are real; without reuse F_{Mx-u,v} has CTAs of its own
    const bool paired = !a.noreuse && u > 0 && 2 * u < Mx;
    const int x0 = blockIdx.x * kStripW;
    const int ys = blockIdx.y * a.seg_len;
    if (ys >= a.H) return;
    const int ye = min(a.H, ys + a.seg_len);
    const int tid = threadIdx.x;
    const int stride = kStripW + 1;

    float4 *sig = reinterpret_cast<float4 *>(smem_raw);
    float2 *jring = reinterpret_cast<float2 *>(sig + (size_t)a.RS * stride);
    float2 *stage = jring + (size_t)a.RS * stride;
    float *raw = reinterpret_cast<float *>(stage + (size_t)a.TH * a.SW);
    float2 *phx = reinterpret_cast<float2 *>(raw + (size_t)2 * a.TH * a.RW);
    float *tx = reinterpret_cast<float *>(phx + a.SW + 1);
    float *ty = tx + a.TpadX + 8;
    // tw2[v][m] = (cos, sin)(2 pi v m / My): demodulation / remodulation twiddles, v <= My/2
    float2 *tw2 = reinterpret_cast<float2 *>(ty + a.TpadY + 8);
    int *nmod = reinterpret_cast<int *>(tw2 + (My / 2 + 1) * My);   // ring slot -> row mod My
    const float4 *tx4 = reinterpret_cast<const float4 *>(tx);
    const float4 *ty4 = reinterpret_cast<const float4 *>(ty);

    for (int i = tid; i < a.TpadX + 8; i += kThreads) tx[i] = i < a.TpadX ? a.taps_x[i] : 0.f;
    for (int i = tid; i < a.TpadY + 8; i += kThreads) ty[i] = i < a.TpadY ? a.taps_y[i] : 0.f;
    for (int i = tid; i < (My / 2 + 1) * My; i += kThreads) {
        const int v = i / My, m = i % My;
        tw2[i] = a.tw_y[(v * m) % My];
    }
    // Row demodulation phase of staged column j, m = x0 - Mx/2 + j: (cos, sin)(w0 u m).
    for (int j = tid; j <= a.SW; j += kThreads) {
        const int m = x0 - Mx / 2 + j;
        phx[j] = a.tw_x[pmod(u * m, Mx)];
    }
    for (int i = tid; i < a.RS * stride; i += kThreads) {
        sig[i] = make_float4(0.f, 0.f, 0.f, 0.f);
        jring[i] = make_float2(0.f, 0.f);
    }
    __syncthreads();

    const int ring_origin = ys - My / 2;
    const int ncols = kStripW + Mx - 1;

    const int warp = tid >> 5, lane = tid & 31;
    const int TH = a.TH;
    const int need0 = min(ys + TH, ye) + My / 2 - 1;
    const int npro = (need0 - ring_origin + TH - 1) / TH;
    const int nch = (ye - ys + TH - 1) / TH;
    const int nblocks = npro + nch - 1;
    // Row blocks: the prologue [ys - My/2, need_0), then [need_{k-1}, need_k) per chunk k,
    // need_k = min(ys + (k+1) TH, ye) + My/2 - 1 (rows y - My/2 .. y + My/2 - 1).
    auto block_rows = [&](int b, int &start, int &n) {
        if (b < npro) {
            start = ring_origin + b * TH;
            n = min(TH, need0 - start);
        } else {
            const int k = b - npro + 1;
            start = min(ys + k * TH, ye) + My / 2 - 1;
            n = min(ys + (k + 1) * TH, ye) + My / 2 - 1 - start;
        }
    };
    auto issue = [&](int b) {
        int start, n;
        block_rows(b, start, n);
        float *dst = raw + (size_t)(b & 1) * TH * a.RW;
        if (a.bmode == kBoundaryZero) {
            for (int r = warp; r < n; r += kThreads / 32) {
                const int y = start + r;
                const bool yin = y >= 0 && y < a.H;
                const float *src = a.img + (int64_t)(yin ? y : 0) * a.pitch;
                for (int j = lane; j < ncols; j += 32) {
                    const int gx = x0 - Mx / 2 + j;
                    const bool ok = yin && gx >= 0 && gx < a.W;
                    cp_async4(dst + (size_t)r * a.RW + j, ok ? (const void *)(src + gx) : (const void *)a.img,
                              ok ? 4 : 0);
                }
            }
        } else {
            for (int r = warp; r < n; r += kThreads / 32) {
                const float *src = a.img + (int64_t)ext_coord(start + r, a.H, a.bmode) * a.pitch;
                for (int j = lane; j < ncols; j += 32)
                    cp_async4(dst + (size_t)r * a.RW + j, src + ext_coord(x0 - Mx / 2 + j, a.W, a.bmode), 4);
            }
        }
        cp_async_commit();
    };
    // Row pass of block b (Eq. 19, 21-22): demodulate, smooth, remodulate into J_u.
    auto row_pass = [&](int b) {
        int start, n;
        block_rows(b, start, n);
        const float *rawb = raw + (size_t)(b & 1) * TH * a.RW;
        for (int r = warp; r < n; r += kThreads / 32) {
            float2 *dst = stage + (size_t)r * a.SW;
            const float *src = rawb + (size_t)r * a.RW;
            for (int j = lane; j < a.SW; j += 32) {
                const float v = j < ncols ? src[j] : 0.f;
                const float2 ph = phx[j];
                dst[j] = make_float2(v * ph.x, v * ph.y);
            }
        }
        __syncthreads();
        const int r = (tid & 7) | ((tid >> 5) << 3);
        const int q = (tid >> 3) & 3;
        if (r < n) {
            float2 acc[8];
#pragma unroll
            for (int j = 0; j < 8; ++j) acc[j] = make_float2(0.f, 0.f);
            conv8_linear<float2>(stage + (size_t)r * a.SW + 8 * q, tx4, a.TpadX / 8, acc);
            const int y = start + r;
            const int slot = (y - ring_origin) % a.RS;
            const bool yin = a.bmode != kBoundaryZero || (y >= 0 && y < a.H);
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                // remodulation by exp(i w0 u xhat), xhat = x - Mx/2 = staged column 8q + j
                const float2 px = phx[8 * q + j];
                const float A = acc[j].x, B = acc[j].y;
                const float jr = fmaf(px.x, A, px.y * B);
                const float ji = fmaf(px.y, A, -px.x * B);
                jring[slot * stride + 8 * q + j] = yin ? make_float2(jr, ji) : make_float2(0.f, 0.f);
            }
        }
    };

    const int nv = My / 2 + 1;
    const int64_t plane = a.plane;
    // Output addressing: the kernel's (u, v, y, x), or for a transposed problem (the vertical
    // pass first, run on the transposed image) the original bin (u, v) -> (v, u) and pixel
    // (x, y) -> (y, x) of an H' = W, W' = H original.
    const int64_t step_y = a.trans ? 1 : a.W, step_x = a.trans ? a.H : 1;
    auto plane_of = [&](int uu, int vv) -> int64_t { return a.trans ? (int64_t)uu * My + vv : (int64_t)vv * Mx + uu; };
    auto col_pass = [&](int c, int nout) {
        const int xl = tid & 31, yg = tid >> 5;
        const int x = x0 + xl;
        const int base_row = c - My / 2;                     // absolute row of the window start
        const int base_off = pmod(base_row - ring_origin, a.RS);
        for (int s = tid; s < a.RS; s += kThreads) nmod[s] = pmod(base_row + pmod(s - base_off, a.RS), My);
        __syncthreads();
        for (int v = v_lo; v < v_hi; ++v) {
            const float2 *twv = tw2 + v * My;
            // Demodulate every ring slot by (cos, sin)(w0 v n) (Eq. 23-24 / 10).
            for (int i = tid; i < a.RS * kStripW; i += kThreads) {
                const int s = i >> 5, xx = i & 31;
                const float2 t = twv[nmod[s]];
                const float2 J = jring[s * stride + xx];
                const float fcr = J.x * t.x, fsr = J.x * t.y, fci = J.y * t.x, fsi = J.y * t.y;
                sig[s * stride + xx] = make_float4(fcr + fsi, fsr - fci, fcr - fsi, fsr + fci);
            }
            __syncthreads();
            for (int yb = 8 * yg; yb < nout; yb += 8 * (kThreads / 32)) {
                const int slot0 = (c - ys + yb) % a.RS;
                float4 acc[8];
#pragma unroll
                for (int j = 0; j < 8; ++j) acc[j] = make_float4(0.f, 0.f, 0.f, 0.f);
                conv8_ring<float4, kStripW + 1>(sig + xl, a.RS, slot0, ty4, a.TpadY / 8, acc);
                if (x < a.W) {
                    const int um = (Mx - u) % Mx, vm = (My - v) % My;
                    const bool fill = !a.half && v > 0 && 2 * v < My;
                    float2 *o_uv = a.out + plane_of(u, v) * plane + x * step_x;
                    float2 *o_mv = a.out + plane_of(um, v) * plane + x * step_x;
                    float2 *o_mm = a.out + plane_of(um, vm) * plane + x * step_x;
                    float2 *o_um = a.out + plane_of(u, vm) * plane + x * step_x;
#pragma unroll
                    for (int j = 0; j < 8; ++j) {
                        const int y = c + yb + j;
                        if (y < c + nout) {
                            // remodulation by exp(i w0 v yhat), yhat = y - My/2: the first window
                            // row of output y sits in ring slot slot0 + j
                            const float2 t = twv[nmod[slot0 + j]];
                            const float P = acc[j].x, Q = acc[j].y, P2 = acc[j].z, Q2 = acc[j].w;
                            const float2 Fa = make_float2(fmaf(t.x, P, t.y * Q), fmaf(t.y, P, -t.x * Q));
                            const int64_t off = (int64_t)y * step_y;
                            __stcs(o_uv + off, Fa);
                            if (fill) __stcs(o_mm + off, make_float2(Fa.x, -Fa.y));
                            if (paired) {
                                const float2 Fb = make_float2(fmaf(t.x, P2, t.y * Q2), fmaf(t.y, P2, -t.x * Q2));
                                __stcs(o_mv + off, Fb);
                                if (fill) __stcs(o_um + off, make_float2(Fb.x, -Fb.y));
                            }
                        }
                    }
                }
            }
            __syncthreads();
        }
    };

    issue(0);
    int b = 0;
    for (int k = 0; k < nch; ++k) {
        const int last = (k == 0) ? npro : npro + k;
        for (; b < last; ++b) {
            if (b + 1 < nblocks) {
                issue(b + 1);
                cp_async_wait<1>();
            } else {
                cp_async_wait<0>();
            }
            __syncthreads();
            row_pass(b);
        }
        __syncthreads();
        const int c = ys + k * TH;
        col_pass(c, min(TH, ye - c));
    }
}

// Modulated-tap form (see the head of this file).
__device__ __forceinline__ void sdft_mt_form(const SdftArgs &a, unsigned char *smem_raw)
{
    const int Mx = a.Mx, My = a.My;
    const int nvz = My / 2 + 1;
    // u in 0 .. Mx/2 (reuse), or the (u, v) of this CTA in the no-reuse ablation
    const int u = a.noreuse ? (int)blockIdx.z / nvz : (int)blockIdx.z;
    const int v_lo = a.noreuse ? (int)blockIdx.z % nvz : 0, v_hi = a.noreuse ? v_lo + 1 : nvz;
    // J_0 and J_{Mx/2} are real; without reuse F_{Mx-u,v} has CTAs of its own
    const bool paired = !a.noreuse && u > 0 && 2 * u < Mx;
    const int x0 = blockIdx.x * kStripW;
    const int ys = blockIdx.y * a.seg_len;
    if (ys >= a.H) return;
    const int ye = min(a.H, ys + a.seg_len);
    const int tid = threadIdx.x;
    const int stride = kStripW + 1;
    const int TH = a.TH, RS = a.RS, RW = a.RW;
    const int nv = My / 2 + 1;

    float2 *jring = reinterpret_cast<float2 *>(smem_raw);
    float *raw = reinterpret_cast<float *>(jring + (size_t)RS * stride);
    float2 *gx = reinterpret_cast<float2 *>(raw + (size_t)2 * TH * RW);      // TpadX + 8 row taps
    float4 *gy = reinterpret_cast<float4 *>(gx + a.TpadX + 8);              // [nv][TpadY + 8]
    const float4 *gx4 = reinterpret_cast<const float4 *>(gx);

    // G_u(a) = S(a - Mx/2) e^{-i w0 u a};  G_v(b) = S(b - My/2) e^{-i w0 v b}
    for (int i = tid; i < a.TpadX + 8; i += kThreads) {
        const float t = i < a.TpadX ? a.taps_x[i] : 0.f;
        const float2 w = i < Mx ? a.tw_x[(u * i) % Mx] : make_float2(0.f, 0.f);
        gx[i] = make_float2(t * w.x, -(t * w.y));
    }
    for (int i = tid; i < nv * (a.TpadY + 8); i += kThreads) {
        const int v = i / (a.TpadY + 8), b = i % (a.TpadY + 8);
        const float t = b < a.TpadY ? a.taps_y[b] : 0.f;
        const float2 w = b < My ? a.tw_y[(v * b) % My] : make_float2(0.f, 0.f);
        const float gr = t * w.x, gi = -(t * w.y);
        gy[i] = make_float4(gr, gi, gi, gr);
    }
    for (int i = tid; i < RS * stride; i += kThreads) jring[i] = make_float2(0.f, 0.f);
    const int ncols = kStripW + Mx - 1;
    // raw columns past the window are read (by zero taps) and never copied: zero them
    const int tail = RW - ncols;
    for (int i = tid; i < 2 * TH * tail; i += kThreads) raw[(size_t)(i / tail) * RW + ncols + i % tail] = 0.f;

    const int ring_origin = ys - My / 2;
    const int warp = tid >> 5, lane = tid & 31;
    const int need0 = min(ys + TH, ye) + My / 2 - 1;
    const int npro = (need0 - ring_origin + TH - 1) / TH;
    const int nch = (ye - ys + TH - 1) / TH;
    const int nblocks = npro + nch - 1;
    // Row blocks: the prologue [ys - My/2, need_0), then [need_{k-1}, need_k) per chunk k,
    // need_k = min(ys + (k+1) TH, ye) + My/2 - 1 (rows y - My/2 .. y + My/2 - 1).
    auto block_rows = [&](int b, int &start, int &n) {
        if (b < npro) {
            start = ring_origin + b * TH;
            n = min(TH, need0 - start);
        } else {
            const int k = b - npro + 1;
            start = min(ys + k * TH, ye) + My / 2 - 1;
            n = min(ys + (k + 1) * TH, ye) + My / 2 - 1 - start;
        }
    };
    auto issue = [&](int b) {
        int start, n;
        block_rows(b, start, n);
        float *dst = raw + (size_t)(b & 1) * TH * RW;
        if (a.bmode == kBoundaryZero) {
            for (int r = warp; r < n; r += kThreads / 32) {
                const int y = start + r;
                const bool yin = y >= 0 && y < a.H;
                const float *src = a.img + (int64_t)(yin ? y : 0) * a.pitch;
                for (int j = lane; j < ncols; j += 32) {
                    const int gxx = x0 - Mx / 2 + j;
                    const bool ok = yin && gxx >= 0 && gxx < a.W;
                    cp_async4(dst + (size_t)r * RW + j, ok ? (const void *)(src + gxx) : (const void *)a.img,
                              ok ? 4 : 0);
                }
            }
        } else {
            for (int r = warp; r < n; r += kThreads / 32) {
                const float *src = a.img + (int64_t)ext_coord(start + r, a.H, a.bmode) * a.pitch;
                for (int j = lane; j < ncols; j += 32)
                    cp_async4(dst + (size_t)r * RW + j, src + ext_coord(x0 - Mx / 2 + j, a.W, a.bmode), 4);
            }
        }
        cp_async_commit();
    };
    // Row pass of block b (Eq. 19, 21-22 as one complex-tap convolution of the raw rows):
    // thread = (row r, 8-column group q); a warp covers 8 rows x 4 groups (RW = 4 mod 32:
    // the 16-byte window loads of a quarter warp hit distinct banks).
    auto row_pass = [&](int b) {
        int start, n;
        block_rows(b, start, n);
        const float *rawb = raw + (size_t)(b & 1) * TH * RW;
        const int r = (tid & 7) | ((tid >> 5) << 3);
        const int q = (tid >> 3) & 3;
        if (r < n) {
            float2 acc[8];
#pragma unroll
            for (int j = 0; j < 8; ++j) acc[j] = make_float2(0.f, 0.f);
            conv8_linear_ct4(rawb + (size_t)r * RW + 8 * q, gx4, a.TpadX / 8, acc);
            const int y = start + r;
            const int slot = (y - ring_origin) % RS;
            const bool yin = a.bmode != kBoundaryZero || (y >= 0 && y < a.H);
#pragma unroll
            for (int j = 0; j < 8; ++j) jring[slot * stride + 8 * q + j] = yin ? acc[j] : make_float2(0.f, 0.f);
        }
    };

    const int64_t plane = a.plane;
    const int64_t step_y = a.trans ? 1 : a.W, step_x = a.trans ? a.H : 1;
    auto plane_of = [&](int uu, int vv) -> int64_t { return a.trans ? (int64_t)uu * My + vv : (int64_t)vv * Mx + uu; };
    // Column pass for output rows [c, c + nout): every v reads the same J ring.
    auto col_pass = [&](int c, int nout) {
        const int xl = tid & 31, yg = tid >> 5;
        const int x = x0 + xl;
        const int um = (Mx - u) % Mx;
        for (int v = v_lo; v < v_hi; ++v) {
            const float4 *gv = gy + v * (a.TpadY + 8);
            const int vm = (My - v) % My;
            const bool fill = !a.half && v > 0 && 2 * v < My;
            for (int yb = 8 * yg; yb < nout; yb += 8 * (kThreads / 32)) {
                const int slot0 = (c - ys + yb) % RS;
                float2 ac[8], bd[8];
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    ac[j] = make_float2(0.f, 0.f);
                    bd[j] = make_float2(0.f, 0.f);
                }
                conv8_ring_cc<kStripW + 1>(jring + xl, RS, slot0, gv, a.TpadY / 8, ac, bd);
                if (x < a.W) {
                    float2 *o_uv = a.out + plane_of(u, v) * plane + x * step_x;
                    float2 *o_mv = a.out + plane_of(um, v) * plane + x * step_x;
                    float2 *o_mm = a.out + plane_of(um, vm) * plane + x * step_x;
                    float2 *o_um = a.out + plane_of(u, vm) * plane + x * step_x;
#pragma unroll
                    for (int j = 0; j < 8; ++j) {
                        const int y = c + yb + j;
                        if (y < c + nout) {
                            // F_{u,v} = sum G_v J_u,  F_{Mx-u,v} = sum G_v J*_u (Eq. 25-26)
                            const float2 Fa = make_float2(ac[j].x - bd[j].x, ac[j].y + bd[j].y);
                            const int64_t off = (int64_t)y * step_y;
                            __stcs(o_uv + off, Fa);
                            if (fill) __stcs(o_mm + off, make_float2(Fa.x, -Fa.y));
                            if (paired) {
                                const float2 Fb = make_float2(ac[j].x + bd[j].x, ac[j].y - bd[j].y);
                                __stcs(o_mv + off, Fb);
                                if (fill) __stcs(o_um + off, make_float2(Fb.x, -Fb.y));
                            }
                        }
                    }
                }
            }
        }
    };

    // The row pass reads raw rows to its end, so block b + 1 (which refills the buffer of
    // block b - 1) is issued after the barrier that ends the row pass of block b - 1.
    issue(0);
    int b = 0;
    for (int k = 0; k < nch; ++k) {
        const int last = (k == 0) ? npro : npro + k;
        for (; b < last; ++b) {
            cp_async_wait<0>();
            __syncthreads();   // raw block b visible; the row pass of block b - 1 and the column
                               // pass of the previous chunk are done
            if (b + 1 < nblocks) issue(b + 1);
            row_pass(b);
        }
        __syncthreads();       // ring rows of chunk k complete
        const int c = ys + k * TH;
        col_pass(c, min(TH, ye - c));
    }
}

// The modulated-tap form is bounded to 80 registers so that three CTAs share an SM (its
// shared memory allows it; measured 10% faster than two at 16 x 16, a few bytes spilled);
// the step-by-step form to 128, so that two do.
template <bool MT>
__global__ void __launch_bounds__(kThreads, MT ? 3 : 2) k_sdft_fp32(const SdftArgs a)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    if constexpr (MT)
        sdft_mt_form(a, smem_raw);
    else
        sdft_demod_form(a, smem_raw);
}

// dst[x][y] = src[y][x] for an H x W image (32 x 32 tiles through shared memory).
__global__ void k_transpose(const float *__restrict__ src, int64_t pitch, int H, int W, float *__restrict__ dst)
{
    __shared__ float t[32][33];
    const int bx = blockIdx.x * 32, by = blockIdx.y * 32;
    for (int r = threadIdx.y; r < 32; r += blockDim.y) {
        const int y = by + r, x = bx + threadIdx.x;
        if (y < H && x < W) t[r][threadIdx.x] = src[(int64_t)y * pitch + x];
    }
    __syncthreads();
    for (int r = threadIdx.y; r < 32; r += blockDim.y) {
        const int x = bx + r, y = by + threadIdx.x;
        if (x < W && y < H) dst[(int64_t)x * H + y] = t[threadIdx.x][r];
    }
}

cudaError_t launch_transpose(const float *src, int64_t pitch, int H, int W, float *dst, cudaStream_t st)
{
    const dim3 grid((W + 31) / 32, (H + 31) / 32);
    k_transpose<<<grid, dim3(32, 8), 0, st>>>(src, pitch, H, W, dst);
    return cudaGetLastError();
}

cudaError_t sdft_fp32_prepare()
{
    cudaError_t e = cudaFuncSetAttribute(k_sdft_fp32<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemLimit);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(k_sdft_fp32<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemLimit);
}

cudaError_t launch_sdft_fp32(SdftArgs a, int sm_count, cudaStream_t st)
{
    const bool mt = !a.demod_form;
    a.TpadX = round_up(a.Mx, 8);
    a.TpadY = round_up(a.My, 8);
    a.SW = mt ? 0 : stage_width(kStripW + a.TpadX);
    // modulated taps: raw rows hold every tap window of the strip (zero tail), 4 mod 32 floats
    // apart (16-byte window loads, conflict-free over the 8 rows of a quarter warp)
    a.RW = mt ? round_up(kStripW + a.TpadX - 1, 32) + 4 : round_up(kStripW + a.Mx - 1, 4);
    int TH = 64;
    size_t smem;
    for (;;) {
        a.TH = TH;
        a.RS = round_up(TH + a.My - 1, 8);
        smem = mt ? sdft_mt_smem_bytes(TH, a.RS, a.RW, a.TpadX, a.TpadY, a.My)
                  : sdft_smem_bytes(TH, a.RS, a.SW, a.RW, a.TpadX, a.TpadY, a.My);
        if (smem <= (size_t)kSmemLimit || TH <= 8) break;
        TH /= 2;
    }
    const int cps = std::max(1, std::min(8, (int)(kSmemLimit / (smem + 1024))));
    const int nstrips = (a.W + kStripW - 1) / kStripW;
    const int nu = a.noreuse ? a.Mx * (a.My / 2 + 1) : a.Mx / 2 + 1;
    const int64_t base = (int64_t)nstrips * nu;
    int nseg = 1;
    const int64_t target = 2LL * sm_count * cps;
    const int min_len = std::max(TH, 2 * a.My);
    while (base * nseg < target && a.H / (nseg + 1) >= min_len) ++nseg;
    a.seg_len = (a.H + nseg - 1) / nseg;
    nseg = (a.H + a.seg_len - 1) / a.seg_len;
    const dim3 grid(nstrips, nseg, nu);
    if (mt)
        k_sdft_fp32<true><<<grid, kThreads, smem, st>>>(a);
    else
        k_sdft_fp32<false><<<grid, kThreads, smem, st>>>(a);
    return cudaGetLastError();
}

}  // namespace gb
