// Recursive-Gaussian variant of the FP32 bank (GB_SMOOTHER_IIR): Algorithm 1 with both 1-D
// Gaussian passes replaced by the third-order forward / backward recursion of Young and van
// Vliet (Signal Processing, 1995), the smoother Sec. II adopts.  Its cost per output does not
// depend on sigma; it approximates S_sigma (Sec. IV-C assesses it by SER against the FIR bank).
//
// The recursion runs in difference form (IirFreq): its state is the last output and the last two
// first differences, so that each step's rounding error is relative to a difference instead of
// to the output; in FP32 the direct form loses accuracy as sigma^3 (the feedback coefficients
// sum to 1 - c0 with c0 ~ 1 / sigma^3), the difference form stays near 1e-6 up to sigma 32.
// Every line carries two real signals with the same recursion (f_c and f_s of Eq. 5 in the row
// pass, P and Q of Eq. 10 in the column pass), which one thread runs together in packed
// FP32x2 arithmetic.
//
// Both passes are chunk-parallel (block-parallel recursive filtering in the manner of Nehab,
// Maximo, Lima and Hoppe, SIGGRAPH Asia 2011): a line is cut into chunks of 16 samples, one per
// thread.  A chunk run from zero state gives its end state L_j; the true end states then follow
// from S_j = A^16 S_{j-1} + L_j (A the zero-input state matrix), an inclusive scan evaluated
// Kogge-Stone fashion with the precomputed powers A^(16 * 2^i).  Lines longer than one scan
// group are walked in super-chunks with the state carried between them: a forward sweep keeps
// every chunk's true start state; a backward sweep re-runs each chunk forward from it, runs it
// backward from zero, scans those states from the end of the line, and re-runs it backward
// from its true state.
//
//   row kernel     one warp per (extended image row, horizontal pass), 32 chunks per
//                  super-chunk, warp shuffles for the scans.  Input and phases of the next
//                  super-chunk arrive by async copies into the other half of a double buffer
//                  (coalesced copies, conflict-free chunk reads from a padded layout); the
//                  output J = e^{i w^c x} (S*f_c - i S*f_s) (Eq. 5-6) is staged in shared
//                  memory and stored row-major per pass.
//   column kernel  one CTA per (horizontal pass, orientation of the pair, 32 image columns):
//                  8 warps hold 8 consecutive chunks of 16 rows of the same columns, so every
//                  load and store is a full row segment; the column signals P, Q (Eq. 10:
//                  J e^{-i w^s y} = P - i Q for theta, the same of J* for pi - theta,
//                  Eq. 13-16) are formed on load, the scans run through shared memory (one
//                  warp holds 4 columns x 8 chunks), the forward sweep's start states wait in a
//                  global scratch buffer, and F = e^{i w^s y} (P' - i Q') (Eq. 7-8, 15-16) is
//                  stored as complex64.
//
// Every signal is extended by P_s = ceil(12 sigma_s) + 32 samples on each side (zeros under
// the zero rule, whose forward passes can start at the first image sample), and each
// recursion starts from zero state at the ends of its extended range.
#include <algorithm>

#include "conv_fp32.cuh"
#include "internal.h"

namespace gb {

namespace {

constexpr int kK = kIirChunk;                        // samples per thread chunk
constexpr int kSC = 32 * kK;                         // samples per row super-chunk
constexpr int kSCp = kSC + kSC / kK;                 // padded: one slot after every chunk
constexpr int kColWarps = 8;                         // chunks per column super-chunk
constexpr int kColSC = kColWarps * kK;               // rows per column super-chunk
constexpr int kColCols = 32;                         // image columns per column CTA
constexpr int kStateStride = 6 * 32 + 4;             // floats per chunk of 32 two-signal states
constexpr size_t kMaxDynSmem = 220 * 1024;

// The padded shared-memory slot of super-chunk sample q: chunk j's samples sit at 17 j + n,
// so the 32 chunks' sample n fall on distinct banks.
__device__ __forceinline__ int ipad(int q) { return q + q / kK; }

__device__ __forceinline__ float2 f2(float a) { return make_float2(a, a); }

// State of two signals run together: last output, its last two first differences.
struct St3 {
    float2 w, d1, d2;
};
__device__ __forceinline__ St3 zero3() { return St3{f2(0.f), f2(0.f), f2(0.f)}; }

// Packed coefficients of the step below.
struct Coef {
    float2 c0, mce, mc3;
};
__device__ __forceinline__ Coef coef_of(const IirFreq &f) { return Coef{f2(f.c0), f2(-f.ce), f2(-f.c3)}; }

// One step of the difference form, D = c0 (x - w1) - e1 d1 - c3 d2, written with
// w1 = w2 + d1 as D = c0 (x - w2) - c3 d2 - ce d1 (ce = c0 + e1, w2 the output before w1), so
// that one FMA lies on the step-to-step dependence through d1.
struct Run {
    float2 w1, w2, d1, d2;
};
__device__ __forceinline__ Run run_from(const St3 &s)
{
    return Run{s.w, __ffma2_rn(s.d1, f2(-1.f), s.w), s.d1, s.d2};
}
__device__ __forceinline__ St3 state_of(const Run &r) { return St3{r.w1, r.d1, r.d2}; }
__device__ __forceinline__ void dstep(Run &s, float2 x, const Coef &c)
{
    const float2 xm = __ffma2_rn(s.w2, f2(-1.f), x);
    const float2 t = __ffma2_rn(c.c0, xm, __fmul2_rn(c.mc3, s.d2));
    const float2 D = __ffma2_rn(c.mce, s.d1, t);
    s.w2 = s.w1;
    s.w1 = __fadd2_rn(s.w1, D);
    s.d2 = s.d1;
    s.d1 = D;
}

// A chunk run from state s, forward or backward (REV); OUT: the outputs replace the inputs.
// s becomes the chunk's end state.
template <bool OUT, bool REV>
__device__ __forceinline__ void run_chunk(St3 &s, float2 (&x)[kK], const Coef &c)
{
    Run r = run_from(s);
#pragma unroll
    for (int k = 0; k < kK; ++k) {
        const int n = REV ? kK - 1 - k : k;
        dstep(r, x[n], c);
        if (OUT) x[n] = r.w1;
    }
    s = state_of(r);
}

// e += M s (M row-major 3 x 3, the same for both signals)
__device__ __forceinline__ void madd(St3 &e, const float *M, const St3 &s)
{
    e.w = __ffma2_rn(f2(M[0]), s.w, __ffma2_rn(f2(M[1]), s.d1, __ffma2_rn(f2(M[2]), s.d2, e.w)));
    e.d1 = __ffma2_rn(f2(M[3]), s.w, __ffma2_rn(f2(M[4]), s.d1, __ffma2_rn(f2(M[5]), s.d2, e.d1)));
    e.d2 = __ffma2_rn(f2(M[6]), s.w, __ffma2_rn(f2(M[7]), s.d1, __ffma2_rn(f2(M[8]), s.d2, e.d2)));
}

__device__ __forceinline__ float2 shfl_up2(float2 v, int d, int width)
{
    return make_float2(__shfl_up_sync(0xffffffffu, v.x, d, width), __shfl_up_sync(0xffffffffu, v.y, d, width));
}
__device__ __forceinline__ float2 shfl_down2(float2 v, int d, int width)
{
    return make_float2(__shfl_down_sync(0xffffffffu, v.x, d, width), __shfl_down_sync(0xffffffffu, v.y, d, width));
}
__device__ __forceinline__ float2 shfl_idx2(float2 v, int src, int width)
{
    return make_float2(__shfl_sync(0xffffffffu, v.x, src, width), __shfl_sync(0xffffffffu, v.y, src, width));
}
__device__ __forceinline__ St3 shfl_up3(const St3 &s, int d, int w)
{
    return St3{shfl_up2(s.w, d, w), shfl_up2(s.d1, d, w), shfl_up2(s.d2, d, w)};
}
__device__ __forceinline__ St3 shfl_down3(const St3 &s, int d, int w)
{
    return St3{shfl_down2(s.w, d, w), shfl_down2(s.d1, d, w), shfl_down2(s.d2, d, w)};
}
__device__ __forceinline__ St3 shfl_idx3(const St3 &s, int src, int w)
{
    return St3{shfl_idx2(s.w, src, w), shfl_idx2(s.d1, src, w), shfl_idx2(s.d2, src, w)};
}

// Inclusive scans S_j = A^16 S_{j-1} + L_j over the `width` lanes of a group (j = lane index in
// the group); the reverse form runs S_j = A^16 S_{j+1} + L_j.
template <int LEVELS>
__device__ __forceinline__ void scan_up(St3 &a, const IirFreq &f, int j, int width)
{
#pragma unroll
    for (int i = 0; i < LEVELS; ++i) {
        const int d = 1 << i;
        const St3 o = shfl_up3(a, d, width);
        if (j >= d) madd(a, f.m[i], o);
    }
}
template <int LEVELS>
__device__ __forceinline__ void scan_down(St3 &a, const IirFreq &f, int j, int width)
{
#pragma unroll
    for (int i = 0; i < LEVELS; ++i) {
        const int d = 1 << i;
        const St3 o = shfl_down3(a, d, width);
        if (j + d < width) madd(a, f.m[i], o);
    }
}

// A two-signal state as six floats 32 apart (thread idx of 32)
__device__ __forceinline__ void put3(float *p, int idx, const St3 &a)
{
    p[idx] = a.w.x;
    p[32 + idx] = a.w.y;
    p[64 + idx] = a.d1.x;
    p[96 + idx] = a.d1.y;
    p[128 + idx] = a.d2.x;
    p[160 + idx] = a.d2.y;
}
__device__ __forceinline__ St3 get3(const float *p, int idx)
{
    return St3{make_float2(p[idx], p[32 + idx]), make_float2(p[64 + idx], p[96 + idx]),
               make_float2(p[128 + idx], p[160 + idx])};
}

__device__ __forceinline__ void load_freq(IirFreq &dst, const IirFreq *src)
{
    constexpr int n = (int)(sizeof(IirFreq) / 4);
    for (int i = threadIdx.x; i < n; i += blockDim.x)
        reinterpret_cast<float *>(&dst)[i] = reinterpret_cast<const float *>(src)[i];
}

// Row kernel: the CTA's phase row (one pass, every row of the CTA), then per warp two input
// stage buffers, a J stage buffer and the start states [super-chunk][192].
__host__ __device__ inline size_t row_smem_cta(int nsc) { return (size_t)nsc * kSCp * sizeof(float2); }
__host__ __device__ inline size_t row_smem_per_warp(int nsc)
{
    return (size_t)kSCp * (2 * sizeof(float) + sizeof(float2)) + (size_t)nsc * 192 * sizeof(float);
}
// Column kernel: two scan buffers of end states and one of start states, [chunk][kStateStride].
constexpr size_t kColSmem = (size_t)3 * kColWarps * kStateStride * sizeof(float);
// Column kernel scratch per CTA: the start states [super-chunk][chunk][192].
__host__ __device__ inline size_t col_scratch_floats(int nsc) { return (size_t)nsc * kColWarps * 192; }

}  // namespace

size_t gabor_iir_col_scratch_floats(int col_nsc) { return col_scratch_floats(col_nsc); }

__global__ void __launch_bounds__(256, 2) k_iir_rows(const IirArgs a)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ IirFreq fq;
    const int nw = (int)(blockDim.x >> 5), warp = (int)(threadIdx.x >> 5), lane = (int)(threadIdx.x & 31);
    const int u = blockIdx.y;
    const UnitDev un = a.units[u];
    load_freq(fq, a.freqs + un.s);
    __syncthreads();
    const bool ext = a.bmode != kBoundaryZero;
    const int P = fq.P, Pl = ext ? P : 0;
    const int Wx = Pl + a.W + P;                 // extended row: position i is x = i - Pl
    const int nsc = (Wx + kSC - 1) / kSC;
    // the pass's phases (cos, sin)(w^c x) over the extended row, shared by the CTA's rows
    float2 *sph = reinterpret_cast<float2 *>(smem_raw);
    for (int i = (int)threadIdx.x; i < nsc * kSC; i += (int)blockDim.x)
        sph[ipad(i)] = i < Wx ? __ldg(un.phx + (i - Pl)) : f2(0.f);
    __syncthreads();
    const int r = blockIdx.x * nw + warp;
    if (r >= a.Hr) return;
    const int y = r - a.Py;
    if (ext && (y < -P || y >= a.H + P)) return;   // rows this pass's column recursion never reads
    const int yy = ext_coord(y, a.H, a.bmode);
    const float *row = a.img + (int64_t)yy * a.pitch;
    const Coef cf = coef_of(fq);

    unsigned char *ws = smem_raw + row_smem_cta(a.row_nsc) + (size_t)warp * row_smem_per_warp(a.row_nsc);
    float2 *sJ = reinterpret_cast<float2 *>(ws);                                   // J stage
    float *starts = reinterpret_cast<float *>(ws + kSCp * (sizeof(float2) + 2 * sizeof(float)));   // [t][192]
    auto sin_of = [&](int t) { return reinterpret_cast<float *>(ws + kSCp * sizeof(float2)) + (t & 1) * kSCp; };
    float2 *Jrow = a.J + ((int64_t)u * a.Hr + r) * a.W;

    // the input of super-chunk t into stage buffer t & 1 (32 consecutive samples per copy)
    auto stage = [&](int t) {
        float *si = sin_of(t);
#pragma unroll 4
        for (int m = 0; m < kK; ++m) {
            const int q = 32 * m + lane;
            const int i = t * kSC + q;
            const int xx = i < Wx ? ext_coord(i - Pl, a.W, a.bmode) : -1;
            cp_async4(si + ipad(q), xx >= 0 ? row + xx : row, xx >= 0 ? 4 : 0);
        }
        cp_async_commit();
    };
    // this lane's chunk of super-chunk t, demodulated (Eq. 5): (f cos(w^c x), f sin(w^c x))
    float2 v[kK];
    auto demod = [&](int t) {
        const float *si = sin_of(t);
        const float2 *sp = sph + t * kSCp;
#pragma unroll
        for (int n = 0; n < kK; ++n) {
            const int q = (kK + 1) * lane + n;
            v[n] = __fmul2_rn(f2(si[q]), sp[q]);
        }
    };

    // ---- forward sweep: the true start state of every chunk
    St3 carry = zero3();   // state before the super-chunk (the same in every lane)
    stage(0);
    for (int t = 0; t < nsc; ++t) {
        if (t + 1 < nsc) {
            stage(t + 1);
            cp_async_wait<1>();
        } else {
            cp_async_wait<0>();
        }
        __syncwarp();
        demod(t);
        St3 l = zero3();
        run_chunk<false, false>(l, v, cf);
        if (lane == 0) madd(l, fq.m[0], carry);
        scan_up<5>(l, fq, lane, 32);
        St3 st = shfl_up3(l, 1, 32);
        if (lane == 0) st = carry;
        put3(starts + t * 192, lane, st);
        carry = shfl_idx3(l, 31, 32);
        __syncwarp();
    }
    // ---- backward sweep, then J (Eq. 5-6); super-chunk nsc - 1 is still staged
    St3 bcarry = zero3();   // state after the super-chunk
    for (int t = nsc - 1; t >= 0; --t) {
        if (t > 0) {
            stage(t - 1);
            cp_async_wait<1>();
        } else {
            cp_async_wait<0>();
        }
        __syncwarp();
        demod(t);
        St3 f = get3(starts + t * 192, lane);
        run_chunk<true, false>(f, v, cf);
        const int i0 = t * kSC + kK * lane;
#pragma unroll
        for (int n = 0; n < kK; ++n)
            if (i0 + n >= Wx) v[n] = f2(0.f);     // the backward recursion starts at the range's end
        St3 l = zero3();
        run_chunk<false, true>(l, v, cf);
        if (lane == 31) madd(l, fq.m[0], bcarry);
        scan_down<5>(l, fq, lane, 32);
        St3 rs = shfl_down3(l, 1, 32);
        if (lane == 31) rs = bcarry;
        bcarry = shfl_idx3(l, 0, 32);
        run_chunk<true, true>(rs, v, cf);
        // J = e^{i w^c x} (A - i B) = (cos A + sin B, sin A - cos B), (A, B) = v[n]
        const float2 *sp = sph + t * kSCp;
#pragma unroll
        for (int n = 0; n < kK; ++n) {
            const int q = (kK + 1) * lane + n;
            const float2 ph = sp[q];
            sJ[q] = __ffma2_rn(ph, f2(v[n].x), __fmul2_rn(make_float2(ph.y, -ph.x), f2(v[n].y)));
        }
        __syncwarp();
#pragma unroll 4
        for (int m = 0; m < kK; ++m) {
            const int q = 32 * m + lane;
            const int x = t * kSC + q - Pl;
            if (x >= 0 && x < a.W) Jrow[x] = sJ[ipad(q)];
        }
        __syncwarp();
    }
}

__global__ void __launch_bounds__(32 * kColWarps, 2) k_iir_cols(const IirArgs a)
{
    extern __shared__ __align__(16) float csm[];
    __shared__ IirFreq fq;
    const int pair = (int)(blockIdx.x & 1), g = (int)(blockIdx.x >> 1), u = blockIdx.y;
    const UnitDev un = a.units[u];
    if (pair == 1 && un.plane_b < 0) return;      // uniform across the CTA
    load_freq(fq, a.freqs + un.s);
    __syncthreads();
    const int warp = (int)(threadIdx.x >> 5), lane = (int)(threadIdx.x & 31);
    const int x = g * kColCols + lane;
    const bool xin = x < a.W;
    const bool ext = a.bmode != kBoundaryZero;
    const int P = fq.P, Pyl = ext ? P : 0;
    const int Hc = Pyl + a.H + P;                 // extended column: position j is y = j - Pyl
    const int nsc = (Hc + kColSC - 1) / kColSC;
    const Coef cf = coef_of(fq);
    constexpr int kBuf = kColWarps * kStateStride;
    float *Ls0 = csm, *Ls1 = csm + kBuf, *Ss = csm + 2 * kBuf;
    // the forward sweep's start states of this CTA: [t][chunk][192]
    float *starts = a.col_scratch + ((int64_t)blockIdx.y * gridDim.x + blockIdx.x) * col_scratch_floats(a.col_nsc);
    // the scan thread: 4 columns x 8 chunks per warp
    const int sc = 4 * warp + (lane >> 3), sj = lane & 7;
    const float2 *Jc = a.J + (int64_t)u * a.Hr * a.W + (xin ? x : 0);
    const float2 *phy = un.phy;
    // theta: J e^{-i w^s y} = P - i Q; pi - theta: the same of J* (Eq. 10, 13-16)
    const float sgn = pair ? -1.f : 1.f;
    const int plane = pair ? un.plane_b : un.plane_a;

    float2 v[kK];
    // (P, Q) = Re J (cos, sin) + s Im J (sin, -cos)
    auto sig_of = [&](float2 J, float2 cy) {
        return __ffma2_rn(f2(J.x), cy, __fmul2_rn(f2(sgn * J.y), make_float2(cy.y, -cy.x)));
    };
    auto load_sig = [&](int t) {
        const int j0 = t * kColSC + kK * warp;
        if (j0 + kK <= Hc && (ext || j0 + kK - Pyl <= a.H)) {   // every row of the chunk is a signal row
            const float2 *jp = Jc + (int64_t)(j0 - Pyl + a.Py) * a.W;
            const float2 *pp = phy + (j0 - Pyl);
#pragma unroll
            for (int n = 0; n < kK; ++n) {
                const float2 J = xin ? jp[(int64_t)n * a.W] : f2(0.f);
                v[n] = sig_of(J, __ldg(pp + n));
            }
        } else {
#pragma unroll
            for (int n = 0; n < kK; ++n) {
                const int jj = j0 + n, yv = jj - Pyl;
                float2 J = f2(0.f), cy = make_float2(1.f, 0.f);
                if (xin && jj < Hc && (ext || yv < a.H)) {
                    J = Jc[(int64_t)(yv + a.Py) * a.W];
                    cy = __ldg(phy + yv);
                }
                v[n] = sig_of(J, cy);
            }
        }
    };

    // ---- forward sweep: the true start state of every chunk
    St3 carry = zero3();   // held by the scan threads of a column
    for (int t = 0; t < nsc; ++t) {
        load_sig(t);
        St3 l = zero3();
        run_chunk<false, false>(l, v, cf);
        float *L = (t & 1) ? Ls1 : Ls0;
        put3(L + warp * kStateStride, lane, l);
        __syncthreads();
        St3 e = get3(L + sj * kStateStride, sc);
        if (sj == 0) madd(e, fq.m[0], carry);
        scan_up<3>(e, fq, sj, 8);
        St3 st = shfl_up3(e, 1, 8);
        if (sj == 0) st = carry;
        put3(starts + (t * kColWarps + sj) * 192, sc, st);
        carry = shfl_idx3(e, 7, 8);
    }
    __syncthreads();
    // ---- backward sweep and the output (Eq. 7-8, 15-16)
    St3 bcarry = zero3();   // state below the super-chunk, held by the scan threads
    const int64_t oplane = (int64_t)a.H * a.W;
    for (int t = nsc - 1; t >= 0; --t) {
        load_sig(t);
        St3 f = get3(starts + (t * kColWarps + warp) * 192, lane);
        run_chunk<true, false>(f, v, cf);
        const int j0 = t * kColSC + kK * warp;
#pragma unroll
        for (int n = 0; n < kK; ++n)
            if (j0 + n >= Hc) v[n] = f2(0.f);
        St3 l = zero3();
        run_chunk<false, true>(l, v, cf);
        put3(Ls0 + warp * kStateStride, lane, l);
        __syncthreads();
        {
            St3 e = get3(Ls0 + sj * kStateStride, sc);
            if (sj == 7) madd(e, fq.m[0], bcarry);
            scan_down<3>(e, fq, sj, 8);
            St3 rs = shfl_down3(e, 1, 8);
            if (sj == 7) rs = bcarry;
            put3(Ss + sj * kStateStride, sc, rs);
            bcarry = shfl_idx3(e, 0, 8);
        }
        __syncthreads();
        St3 rs = get3(Ss + warp * kStateStride, lane);
        run_chunk<true, true>(rs, v, cf);
        // F = e^{i w^s y} (P' - i Q') = P' (cos, sin) + Q' (sin, -cos)
        auto out_of = [&](float2 pq, float2 cy) {
            return __ffma2_rn(f2(pq.x), cy, __fmul2_rn(f2(pq.y), make_float2(cy.y, -cy.x)));
        };
        const int y0 = j0 - Pyl;
        if (!a.layout && y0 >= 0 && y0 + kK <= a.H) {   // every row of the chunk is an image row
            float2 *op = a.out + (int64_t)plane * oplane + (int64_t)y0 * a.W + x;
            const float2 *pp = phy + y0;
#pragma unroll
            for (int n = 0; n < kK; ++n)
                if (xin) __stcs(op + (int64_t)n * a.W, out_of(v[n], __ldg(pp + n)));
        } else {
#pragma unroll
            for (int n = 0; n < kK; ++n) {
                const int yv = y0 + n;
                if (xin && yv >= 0 && yv < a.H) {
                    const int64_t pix = (int64_t)yv * a.W + x;
                    const int64_t o = a.layout ? pix * a.nplanes + plane : (int64_t)plane * oplane + pix;
                    __stcs(a.out + o, out_of(v[n], __ldg(phy + yv)));
                }
            }
        }
    }
}

bool gabor_iir_fits(int row_nsc, int col_nsc)
{
    (void)col_nsc;
    return row_smem_cta(row_nsc) + row_smem_per_warp(row_nsc) <= kMaxDynSmem;
}

cudaError_t gabor_iir_prepare()
{
    cudaError_t e = cudaFuncSetAttribute(k_iir_rows, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kMaxDynSmem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_iir_cols, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kColSmem);
    return e;
}

int gabor_iir_col_ctas(int W, int nunits) { return 2 * ((W + kColCols - 1) / kColCols) * nunits; }

cudaError_t launch_gabor_iir(const IirArgs &a, cudaStream_t st)
{
    if (a.nunits == 0) return cudaSuccess;
    if (!gabor_iir_fits(a.row_nsc, a.col_nsc)) return cudaErrorInvalidValue;
    int nw = 8;
    auto smem = [&](int n) { return row_smem_cta(a.row_nsc) + (size_t)n * row_smem_per_warp(a.row_nsc); };
    while (nw > 1 && smem(nw) > kMaxDynSmem) nw >>= 1;
    const dim3 gr((a.Hr + nw - 1) / nw, a.nunits);
    k_iir_rows<<<gr, 32 * nw, smem(nw), st>>>(a);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const dim3 gc(2 * ((a.W + kColCols - 1) / kColCols), a.nunits);
    k_iir_cols<<<gc, 32 * kColWarps, kColSmem, st>>>(a);
    return cudaGetLastError();
}

}  // namespace gb
