// Recursive-Gaussian variant of the FP32 bank (GB_SMOOTHER_IIR): Algorithm 1 with both 1-D
// Gaussian passes replaced by the third-order forward / backward recursion of Young and van
// Vliet (Signal Processing, 1995), the smoother Sec. II adopts.  Its cost per output does not
// depend on sigma; it approximates S_sigma (Sec. IV-C assesses it by SER against the FIR bank).
//
//   row kernel     one lane per (unit, image row), 32 rows per warp.  Rows are staged through
//                  32 x 32 shared-memory tiles so that global loads and stores stay coalesced
//                  while every lane runs its row's recursion: forward over f_c, f_s (Eq. 5)
//                  into a scratch buffer, then backward, remodulation into J (Eq. 5-6) and the
//                  column signals of Eq. 10 for theta and pi - theta (Eq. 15-16).
//   column kernel  one thread per (unit, image column, column signal): forward recursion of
//                  the signal down the column into scratch, backward recursion upward; the
//                  two signals of an orientation meet by shuffle for the remodulation by
//                  (cos, sin)(w^s y) (Eq. 7-8, 15-16) and the output stores.
//
// Every signal is extended by P_s = ceil(12 sigma_s) + 32 samples on each side (zeros under
// the zero rule, whose forward passes can start at the first image sample), and each
// recursion starts from zero state at the ends of its extended range.
#include <algorithm>

#include "internal.h"

namespace gb {

namespace {

constexpr int kIirWarps = 4;   // warps per row-kernel CTA (32 rows each)

struct IirRowSmem {
    float2 out[32][33];        // forward outputs, then backward inputs
    float sig[4][32][33];      // column signals (sig[0] doubles as the input tile)
};

}  // namespace

__global__ void __launch_bounds__(32 * kIirWarps) k_iir_rows(const IirArgs a)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    IirRowSmem &S = reinterpret_cast<IirRowSmem *>(smem_raw)[warp];
    const int u = blockIdx.y;
    const UnitDev un = a.units[u];
    const IirFreq fq = a.freqs[un.s];
    const bool paired = un.plane_b >= 0;
    const bool ext = a.bmode != kBoundaryZero;
    const int Pl = ext ? fq.P : 0;                 // extension before x = 0
    const int Wx = Pl + a.W + fq.P;                // extended row length
    const int r0 = (blockIdx.x * kIirWarps + warp) * 32;
    if (r0 >= a.Hr) return;
    const int r = r0 + lane;                       // this lane's row (y = r - Py)
    const int y = r - a.Py;
    float2 *tmp = a.tmp + (int64_t)u * a.Hr * a.Wxmax;
    const float c0 = fq.c[0], c1 = fq.c[1], c2 = fq.c[2], c3 = fq.c[3];

    // ---- forward: w = c0 x + c1 w[-1] + c2 w[-2] + c3 w[-3] over f_c and f_s
    float wc1 = 0.f, wc2 = 0.f, wc3 = 0.f, ws1 = 0.f, ws2 = 0.f, ws3 = 0.f;
    // the next 32 x 32 input tile, prefetched into registers (lane = column, index = row)
    float nxt[32];
    auto load_tile = [&](int i0) {
        const int xx = ext_coord(i0 + lane - Pl, a.W, a.bmode);
#pragma unroll
        for (int rr = 0; rr < 32; ++rr) {
            const int yy = ext_coord(r0 + rr - a.Py, a.H, a.bmode);
            const bool ok = r0 + rr < a.Hr && i0 + lane < Wx && yy >= 0 && xx >= 0;
            nxt[rr] = ok ? __ldg(a.img + (int64_t)yy * a.pitch + xx) : 0.f;
        }
    };
    load_tile(0);
    for (int i0 = 0; i0 < Wx; i0 += 32) {
#pragma unroll
        for (int rr = 0; rr < 32; ++rr) S.sig[0][rr][lane] = nxt[rr];
        if (i0 + 32 < Wx) load_tile(i0 + 32);
        __syncwarp();
#pragma unroll 4
        for (int c = 0; c < 32; ++c) {
            const float2 ph = un.phx[i0 + c - Pl];   // the same position for every lane
            const float v = S.sig[0][lane][c];
            const float wc = fmaf(c0, v * ph.x, fmaf(c1, wc1, fmaf(c2, wc2, c3 * wc3)));
            const float ws = fmaf(c0, v * ph.y, fmaf(c1, ws1, fmaf(c2, ws2, c3 * ws3)));
            wc3 = wc2; wc2 = wc1; wc1 = wc;
            ws3 = ws2; ws2 = ws1; ws1 = ws;
            S.out[lane][c] = make_float2(wc, ws);
        }
        __syncwarp();
        for (int rr = 0; rr < 32; ++rr)
            if (r0 + rr < a.Hr && i0 + lane < Wx) tmp[(int64_t)(r0 + rr) * a.Wxmax + i0 + lane] = S.out[rr][lane];
        __syncwarp();
    }
    // ---- backward, then J (Eq. 5-6) and the column signals (Eq. 10, 15-16)
    const bool yok = r < a.Hr && (ext || (y >= 0 && y < a.H));
    const float2 cy = yok ? un.phy[y] : make_float2(0.f, 0.f);
    float ac1 = 0.f, ac2 = 0.f, ac3 = 0.f, as1 = 0.f, as2 = 0.f, as3 = 0.f;
    const int nsig = paired ? 4 : 2;
    const int64_t plane = (int64_t)a.Hr * a.W;
    float *sig0 = a.sig + un.sig * plane;          // the unit's first column signal
    float2 nb[32];
    auto load_back = [&](int i0) {
#pragma unroll
        for (int rr = 0; rr < 32; ++rr)
            nb[rr] = (r0 + rr < a.Hr && i0 + lane < Wx) ? tmp[(int64_t)(r0 + rr) * a.Wxmax + i0 + lane]
                                                       : make_float2(0.f, 0.f);
    };
    load_back((Wx - 1) / 32 * 32);
    for (int i0 = (Wx - 1) / 32 * 32; i0 >= 0; i0 -= 32) {
#pragma unroll
        for (int rr = 0; rr < 32; ++rr) S.out[rr][lane] = nb[rr];
        if (i0 >= 32) load_back(i0 - 32);
        __syncwarp();
#pragma unroll 4
        for (int c = 31; c >= 0; --c) {
            const float2 w = S.out[lane][c];
            const float A = fmaf(c0, w.x, fmaf(c1, ac1, fmaf(c2, ac2, c3 * ac3)));
            const float B = fmaf(c0, w.y, fmaf(c1, as1, fmaf(c2, as2, c3 * as3)));
            ac3 = ac2; ac2 = ac1; ac1 = A;
            as3 = as2; as2 = as1; as1 = B;
            const int x = i0 + c - Pl;
            if (x >= 0 && x < a.W) {
                const float2 px = un.phx[x];
                // Eq. 5-6: Re J = cos A + sin B, Im J = sin A - cos B
                const float jr = fmaf(px.x, A, px.y * B), ji = fmaf(px.y, A, -px.x * B);
                const float fcr = jr * cy.x, fsr = jr * cy.y, fci = ji * cy.x, fsi = ji * cy.y;
                S.sig[0][lane][c] = fcr + fsi;
                S.sig[1][lane][c] = fsr - fci;
                if (paired) {
                    S.sig[2][lane][c] = fcr - fsi;
                    S.sig[3][lane][c] = fsr + fci;
                }
            }
        }
        __syncwarp();
        const int x = i0 + lane - Pl;
        if (x >= 0 && x < a.W)
            for (int rr = 0; rr < 32; ++rr)
                if (r0 + rr < a.Hr)
                    for (int k = 0; k < nsig; ++k) sig0[k * plane + (int64_t)(r0 + rr) * a.W + x] = S.sig[k][rr][lane];
        __syncwarp();
    }
}

// Rows per block of the column recursion: the block's loads are issued together, ahead of its
// recursion steps, so one memory latency covers kIirRows steps.
constexpr int kIirRows = 16;
constexpr int kIirColThreads = 128;   // 64 columns x 2 signals of one pair per CTA

// Thread = (column, one column signal of a pair): lane = 2 (column) + s, s = 0 for the P signal
// and 1 for Q; blockIdx.z picks the pair (0: theta_a, 1: pi - theta_a of a paired unit).  The
// two signals of an output meet by one shuffle.  (One thread per signal rather than per unit
// column: the recursion is sequential along the column, so parallelism comes from lanes.)
__global__ void __launch_bounds__(kIirColThreads) k_iir_cols(const IirArgs a)
{
    const int u = blockIdx.y, pair = blockIdx.z;
    const UnitDev un = a.units[u];
    const bool paired = un.plane_b >= 0;
    if (pair == 1 && !paired) return;
    const int sgn = threadIdx.x & 1;
    const int x = blockIdx.x * (kIirColThreads / 2) + (threadIdx.x >> 1);
    const bool xin = x < a.W;
    const IirFreq fq = a.freqs[un.s];
    const bool ext = a.bmode != kBoundaryZero;
    const int Pyl = ext ? fq.P : 0;                // extension above y = 0
    const int Hc = Pyl + a.H + fq.P;
    const float c0 = fq.c[0], c1 = fq.c[1], c2 = fq.c[2], c3 = fq.c[3];
    const int64_t plane = (int64_t)a.Hr * a.W;
    const int k = 2 * pair + sgn;                  // the unit's column signal of this thread
    const float *sig = a.sig + (un.sig + k) * plane;
    const int64_t tplane = (int64_t)a.Hcmax * a.W;
    float *tmp = reinterpret_cast<float *>(a.tmp) + (un.sig + k) * tplane;
    const int xc = xin ? x : 0;

    float w1 = 0.f, w2 = 0.f, w3 = 0.f;
    for (int j0 = 0; j0 < Hc; j0 += kIirRows) {
        float v[kIirRows];
#pragma unroll
        for (int t = 0; t < kIirRows; ++t) {
            const int rr = j0 + t - Pyl + a.Py;   // row of the signal buffer
            v[t] = (xin && j0 + t < Hc && rr >= 0 && rr < a.Hr) ? sig[(int64_t)rr * a.W + xc] : 0.f;
        }
#pragma unroll
        for (int t = 0; t < kIirRows; ++t) {
            if (j0 + t >= Hc) break;
            const float w = fmaf(c0, v[t], fmaf(c1, w1, fmaf(c2, w2, c3 * w3)));
            w3 = w2; w2 = w1; w1 = w;
            if (xin) tmp[(int64_t)(j0 + t) * a.W + x] = w;
        }
    }
    float s1 = 0.f, s2 = 0.f, s3 = 0.f;
    const int64_t oplane = (int64_t)a.H * a.W;
    const int oplane_idx = pair ? un.plane_b : un.plane_a;
    for (int j1 = Hc - 1; j1 >= 0; j1 -= kIirRows) {
        float v[kIirRows];
#pragma unroll
        for (int t = 0; t < kIirRows; ++t) v[t] = (xin && j1 - t >= 0) ? tmp[(int64_t)(j1 - t) * a.W + x] : 0.f;
#pragma unroll
        for (int t = 0; t < kIirRows; ++t) {
            const int j = j1 - t;
            if (j < 0) break;   // uniform across the warp
            const float sv = fmaf(c0, v[t], fmaf(c1, s1, fmaf(c2, s2, c3 * s3)));
            s3 = s2; s2 = s1; s1 = sv;
            const float q = __shfl_xor_sync(0xffffffffu, sv, 1);   // the pair's other signal
            const int y = j - Pyl;
            if (sgn == 0 && xin && y >= 0 && y < a.H) {
                const float2 cy = un.phy[y];
                // Eq. 7-8 (theta) or Eq. 15-16 (pi - theta)
                const int64_t pix = (int64_t)y * a.W + x;
                const int64_t o = a.layout ? pix * a.nplanes + oplane_idx : (int64_t)oplane_idx * oplane + pix;
                __stcs(a.out + o, make_float2(fmaf(cy.x, sv, cy.y * q), fmaf(cy.y, sv, -cy.x * q)));
            }
        }
    }
}

cudaError_t gabor_iir_prepare()
{
    return cudaFuncSetAttribute(k_iir_rows, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)(kIirWarps * sizeof(IirRowSmem)));
}

cudaError_t launch_gabor_iir(const IirArgs &a, int nunits, cudaStream_t st)
{
    if (nunits == 0) return cudaSuccess;
    const dim3 gr((a.Hr + 32 * kIirWarps - 1) / (32 * kIirWarps), nunits);
    k_iir_rows<<<gr, 32 * kIirWarps, kIirWarps * sizeof(IirRowSmem), st>>>(a);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const dim3 gc((a.W + kIirColThreads / 2 - 1) / (kIirColThreads / 2), nunits, 2);
    k_iir_cols<<<gc, kIirColThreads, 0, st>>>(a);
    return cudaGetLastError();
}

}  // namespace gb
