// Internal declarations of the gaborbank library (not part of the C ABI).
#pragma once

#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>
#include <cstdint>
#include <string>
#include <map>
#include <utility>
#include <vector>

#include "gaborbank.h"

namespace gb {

constexpr int kStripW = 32;        // image columns per CTA strip (one warp wide)
constexpr int kThreads = 256;      // threads per CTA of the FP32 kernels
constexpr int kMaxRadius = 160;    // largest Gaussian radius of the fused FP32 bank kernel
constexpr int kMaxSdftM = 64;      // largest SDFT window side
constexpr int kSmemLimit = 227 * 1024;
constexpr int kStaticSmemReserve = 256;   // static shared memory kept free next to the dynamic part
constexpr int kSmemPerSm = 228 * 1024;    // shared memory of one SM
constexpr int kSmemCtaReserve = 1024;     // taken by the system from every resident CTA

// Boundary rules for the image beyond its edges.
enum BoundaryMode { kBoundaryZero = 0, kBoundaryReplicate = 1, kBoundaryMirror = 2 };

// The image row / column that position i (of n) reads: i itself inside [0, n); outside, the
// edge sample (replicate) or the sample mirrored about the pixel edges, f(-1) = f(0),
// f(n) = f(n - 1), period 2n (mirror); -1 (a zero sample) for the zero rule.
__host__ __device__ inline int ext_coord(int i, int n, int mode)
{
    if (i >= 0 && i < n) return i;
    if (mode == kBoundaryReplicate) return i < 0 ? 0 : n - 1;
    if (mode == kBoundaryMirror) {
        const int p = 2 * n;
        int m = i % p;
        if (m < 0) m += p;
        return m < n ? m : p - 1 - m;
    }
    return -1;
}

// Device view of one horizontal pass ("row unit") of the bank: the pass of orientation
// theta_a at frequency omega_s, and the orientation pi - theta_a that reuses it (Eq. 13-16).
struct UnitDev {
    const float2 *phx;  // (cos, sin)(omega cos(theta_a) x), x in [-mg, Wcap + mg)
    const float2 *phy;  // (cos, sin)(omega sin(theta_a) y), y in [-mg, Hcap + mg)
    int s;              // frequency index
    int plane_a;        // output plane of theta_a  (s * n_theta + k)
    int plane_b;        // output plane of pi - theta_a, or -1 when unpaired
    int twin;           // FP32 bank, modulated-tap row pass: the unpaired unit that shares this
                        // unit's work items, or -1
    int pad_[2];
};

// Device view of one frequency: Gaussian taps and the FP32 kernel's tile geometry.
struct FreqDev {
    const float *taps;  // Tpad taps S(t - R), zero beyond T
    int R, T, Tpad;
    int TH;             // rows per streamed chunk (multiple of 8, <= 64)
    int RS;             // ring rows (multiple of 8, >= TH + T - 1)
    int SW;             // staging row width in float2 (>= kStripW + Tpad, = 1 mod 16)
    int RW;             // raw staging row width in floats (demodulation form: >= kStripW + T - 1,
                        // multiple of 4; modulated taps: >= kStripW + Tpr, = 4 mod 32)
    int mtaps;          // row pass form: 1 modulated taps, 0 demodulate / smooth / remodulate
    // row pass window: input columns x0 - Rw .. x0 + 31 + R of a strip, Tr = Rw + R + 1 taps
    // (Tpr padded to 8), the first Rw - R of them zero.  Modulated taps: Rw = R rounded up to 4,
    // so that the window starts on a 16-byte boundary; demodulation form: Rw = R.
    int Rw, Tr, Tpr;
    int pad_;
};

// One image of a launch.
struct ImageDev {
    const float *img;
    int64_t pitch;
    float2 *out;
    int H, W;
};

// One CTA's work: a unit, a strip of 32 columns and a row segment of one image.
struct WorkItem {
    int img, unit, strip, y0, y1;
};

// A run of work items of one image that share a frequency and a pairing: `nunits` units
// from u0 on, each cut into nstrips strips x nseg row segments of seg_len rows.  Item
// first + ((q * nstrips) + strip) * nseg + seg is unit u0 + q, that strip and segment.
struct ItemGroup {
    int first, u0, nstrips, nseg, seg_len;
    int ustride;        // units between consecutive items' units (2: twin items)
};
constexpr int kMaxGroups = 64;
constexpr int kMaxRawMaps = 8;   // frequencies whose FP32 row loads can go by TMA

// Arguments of the fused FP32 bank kernel (one launch covers every frequency).  Work items
// come from a device list (`items`, batches) or, for one image, are decoded from `groups`
// (largest item cost first), so that a single-image call needs no per-shape device data.
struct BankArgs {
    ImageDev img0;            // the image when imgs == nullptr
    const ImageDev *imgs;     // batch images (device), or nullptr
    const FreqDev *freqs;
    const UnitDev *units;
    const WorkItem *items;    // nullptr: decode from groups
    int *counter;             // work-queue head (zeroed before each launch)
    int nitems;
    int ngroups;
    int bmode;                // BoundaryMode
    int layout;               // 0: out[plane][y][x], 1: out[y][x][plane]
    int nplanes;              // n_freq * n_theta
    int *status;              // device status word (pipelined variant's bounded waits)
    int pipelined;            // 1: warp-specialised row / column pipeline (host-side choice)
    int mtaps;                // 1: row pass with modulated taps (host-side choice)
    int ctas;                 // CTAs per SM: 1 (16 warps each) or 2 (8 warps each)
    // Modulated-tap row loads by TMA (one image, zero rule, schedule without warp specialisation):
    // bit s of raw_mask set = frequency s loads its row blocks as boxes of RW columns x TH rows
    // of the FP32 image through raw_map[s] (zeros outside the image); clear = async copies.
    unsigned raw_mask;
    ItemGroup groups[kMaxGroups];
    CUtensorMap raw_map[kMaxRawMaps];
};

// ---- tensor-core bank (gabor_tc.cu) ----
struct TcFreqDev {
    const uint16_t *Brow;  // [64][Krow] Toeplitz S(k - x - R), FP16/BF16, K-major SW128
    const uint16_t *Bcol;  // [64][Kcol] Toeplitz S(l - y - R8)
    int R, R8, Krow, Kcol;
    float unscale_row, unscale_col;   // 2^-sB of the B operands
    int u0;                // first unit of the frequency
    int Kmt;               // K of the modulated-tap row pass: 64 + 2R rounded to 64
};
struct TcUnitDev {
    const float2 *phx, *phy;
    int s, plane_a, plane_b, pad_;
    int64_t sig_idx;       // first signal of the unit; its block starts at sig_idx * W * Hp
    const uint16_t *Am;    // modulated-tap row operand: strip of 128 rows x Kmt (FP16 core matrices)
    const uint16_t *Gm;    // modulated-tap column operand: strip of 2 col_mt_ty rows x Kcol
};
// One image of a tensor-core batch (gabor_bank_filter_batch): its input, output, intermediate
// ([signal][Hp / 8][W][8], image row y at Lpad + y) and F[1] tables.
struct TcImgDev {
    const float *img;
    int64_t pitch;
    int H, W;
    int Wq, pad_q;         // modulated-tap intermediate: columns per 8-row block (W rounded up to 16)
    float2 *out;
    int64_t plane;         // H * W
    uint16_t *sig;
    int64_t Hp;
    const float2 *onesA;   // [unit][W]
    const float2 *onesB;   // [unit][H]
    uint16_t *corrA;       // [unit][(W + 63) / 64] and [unit][(H + TYC - 1) / TYC] blocks of
    uint16_t *corrB;       // kCorrBlockHalfs: the correction operands (TcBankArgs)
    uint16_t *pimg;        // the row pass's operand image (TcBankArgs), pq elements per row
    int64_t pq;
};
constexpr int kMmParts = 64;   // partial min / max words per image of a batch (k_minmax)
constexpr int kCorrBlockHalfs = 2048;   // one correction operand block: 128 rows x 16 K, 4 KB
struct TcBankArgs {
    const float *img;
    int64_t pitch;
    int H, W;
    float2 *out;
    int64_t plane;
    // intermediate, image row y at Lpad + y: [signal][Hp / 8][W][8] (step-by-step form) or
    // [plane][Hp / 8][Wq][part][8] (modulated taps: plane = unit, or 2 unit + {hi, lo} under
    // BF16; part = Re J, Im J interleaved, so 16 columns x both parts x 8 rows are 512
    // contiguous bytes)
    uint16_t *sig;
    int64_t Hp;
    int Lpad, Wq;
    const TcFreqDev *freqs;
    const TcUnitDev *units;
    int *status;
    int row_kmax, row_pwmax, col_kmax, row_ty;
    unsigned *minmax;      // device words: ~(min key) and max key of the image (k_minmax)
    // F[1] = A(x) B(y), the bank's response to the image indicator (or to the constant 1 under
    // a non-zero boundary rule): the passes filter f - c and add c A(x) B(y) back.
    const float2 *onesA;   // [unit][W]
    const float2 *onesB;   // [unit][H]
    const double2 *ones_pre;   // [unit][2][2 Rmax + 2] prefix sums of S(d) exp(i w^{c|s} d)
    int ones_stride;           // 2 Rmax + 2
    // The modulated-tap column pass adds c A(x) B(y) by one extra K = 16 MMA per job; its
    // operands (written by k_ones once the centre c is known) in the shared-memory image the
    // MMA reads: per unit, one block of 128 rows x 16 K (FP16 or BF16, no-swizzle K-major core
    // matrices, kCorrBlockHalfs elements) per 64 image columns (rows 2 x + {Re, Im} of
    // c A(x) 2^(sB - t)) and per TYC image rows (rows 2 (TYC - 1 - y) + {Re, Im} of B(y) 2^t).
    uint16_t *corrA;
    uint16_t *corrB;
    int col_mt_ty;             // modulated-tap column pass: output rows per job (64, or 32 for large K)
    // Work items, decoded from the image shape: frequencies in the order forder[] (largest
    // radius first); every frequency has nu_f units, the first np_f of them paired.
    const int *forder;
    int nf, nu_f, np_f;
    int row_nx, row_cnt;   // row pass: 128-column tiles per tile row, items per frequency
    int col_ny, col_nx32, col_nx64, col_cnt;   // column pass: 64-row tiles, x tiles, items per frequency
    int col_nst;           // A-operand buffers of the column kernel (set by the launcher)
    int bmode;             // BoundaryMode
    int layout;            // 0: out[plane][y][x], 1: out[y][x][plane]
    int nplanes;           // n_freq * n_theta
    int row_y0;            // first image row of the row pass (< 0: halo rows for non-zero rules)
    int row_mt;            // 1: the modulated-tap kernels (intermediate = Re J, Im J per unit)
    // TMA maps of the intermediate (dimensions 8 rows of a block x W x signals x Hp / 8 blocks,
    // FP16, no swizzle) for the column pass's A operand: boxes of 8 x 32 columns x 4 signals x
    // 8 blocks (paired units) and 8 x 64 x 2 x 8 (unpaired units)
    CUtensorMap tmA[2];
    // Batches (modulated-tap kernels only): per-image views and TMA maps of their intermediates
    // in device memory, (centre, exponent) per image written by k_ones, kMmParts partial
    // (~min, max) key pairs per image, and explicit item lists; all nullptr for one image.
    const TcImgDev *imgs;
    const CUtensorMap *tmaps;
    float2 *img_ce;
    unsigned *mm_part;
    const int4 *row_list;  // {image, frequency, y0, x0}
    const int4 *col_list;  // {image, unit, x0, y0}
    int n_row, n_col, nimg;
    int split;             // 1: BF16 operands as hi + lo pairs (modulated-tap kernels)
    int col_mt_nst;        // operand stages of the modulated-tap column kernel (1 or 2)
    // p_tma = 1 (modulated taps, zero rule): k_ones writes the row pass's operand image
    // P = (f - c) 2^-e as FP16 (BF16 hi rows, then lo rows: H rows of pq elements each) and the
    // row kernel loads its tiles by TMA (map tmA[1], or tmaps[nimg + i] for image i of a batch,
    // 128-byte swizzle, zeros outside the image); p_tma = 0: the row kernel's producer warps
    // build P from the image.
    int p_tma;
    uint16_t *pimg;
    int64_t pq;
};
struct TcGeometry {
    int R, R8, Krow, Kcol, PW;
    size_t smem_rows, smem_cols;
};

// ---- recursive-Gaussian bank (gabor_iir.cu) ----
// Young-van Vliet recursion of one frequency, w[n] = c0 x[n] + c1 w[n-1] + c2 w[n-2] +
// c3 w[n-3] (and the same backward), evaluated in difference form: with the state
// (w1, d1, d2) = (w[n-1], w[n-1] - w[n-2], w[n-2] - w[n-3]) one step is
//   D = c0 (x[n] - w1) - e1 d1 - c3 d2,  w[n] = w1 + D,  (w1, d1, d2) <- (w[n], D, d1),
// e1 = c2 + c3 (the same recursion, since c1 + c2 + c3 = 1 - c0); the kernels use
// ce = c0 + e1.  m[i] is the 3 x 3 state matrix of kIirChunk << i zero-input steps
// (row-major), for the chunk-parallel scans.  P is the extension on each side of a signal.
constexpr int kIirChunk = 16;   // samples per thread chunk of the chunk-parallel recursions
constexpr int kIirLevels = 5;   // m[i] = A^(16 * 2^i), i < 5
struct IirFreq {
    float c0, ce, c3;
    int P;
    float m[kIirLevels][9];
    float pad_[3];
};
struct IirArgs {
    const float *img;
    int64_t pitch;
    int H, W;
    float2 *out;
    int layout, nplanes, bmode, nunits;
    const UnitDev *units;
    const IirFreq *freqs;
    float2 *J;             // row-pass outputs J [unit][Hr][W], row r at y = r - Py
    int Hr, Py;
    int row_nsc;           // super-chunks of the longest extended row (512 samples each)
    int col_nsc;           // super-chunks of the longest extended column (128 rows each)
    float *col_scratch;    // the column kernel's forward start states, gabor_iir_col_scratch_floats
                           // (col_nsc) floats per column CTA
};
// Arguments of the FP32 localized-SDFT kernel (Algorithm 2).
struct SdftArgs {
    const float *img;
    int64_t pitch;
    int H, W;
    float2 *out;
    int64_t plane;
    int Mx, My;
    int half;            // 1: only v <= My/2 planes
    const float *taps_x; // TpadX taps S(i - Mx/2), i < Mx
    const float *taps_y; // TpadY taps S(i - My/2), i < My
    const float2 *tw_x;  // (cos, sin)(2 pi j / Mx), j < Mx
    const float2 *tw_y;  // (cos, sin)(2 pi j / My), j < My
    int TpadX, TpadY;
    int TH, seg_len, RS, SW, RW;
    int bmode;           // BoundaryMode
    int trans;           // 1: a transposed problem (vertical pass first); outputs are written back transposed
    int demod_form;      // 1: demodulate / smooth / remodulate step by step; 0: modulated taps
    int noreuse;         // 1: the no-reuse ablation, one CTA per (u in [0, Mx), v in [0, My/2]) that
                         // recomputes J_u for its single v (no J_{Mx-u} = J*_u)
};

// One frequency of the plan.
struct Freq {
    double omega, sigma;
    int R, T, Tpad;
    int u0, u1;          // its units [u0, u1)
};

// One horizontal pass of the plan (host side).
struct Unit {
    int s;
    int k_a, k_b;        // orientation indices (k_b = -1: unpaired)
    double wc, ws;       // omega cos(theta_a), omega sin(theta_a)
};

// Kernel launchers (defined in the .cu files).
// Phase tables for positions -mg .. cap + mg - 1 (rows of cap + 2 mg entries per unit).
cudaError_t launch_build_gabor_tables(const double *d_unit_w, int nunits, int Wcap, int Hcap, int mg,
                                      float2 *phx, float2 *phy, cudaStream_t st);
cudaError_t launch_build_taps(const double *d_sigma, const int *d_lo, const int *d_T, int nfreq,
                              int tpad_max, float *taps, cudaStream_t st);
cudaError_t launch_build_twiddles(int M, float2 *tw, cudaStream_t st);
// Taps and twiddles of both SDFT window axes from by-value parameters: taps[2][tap_stride]
// (S(t - M/2), zero from t = M on), tw[2][tw_stride] ((cos, sin)(2 pi j / M), j < M).
cudaError_t launch_build_sdft_tables(double sigma, int Mx, int My, int tap_stride, int tw_stride, float *taps,
                                     float2 *tw, cudaStream_t st);
// Tile geometry of the FP32 bank kernel for radius R (tile_rows = 0: automatic).
FreqDev gabor_fp32_geometry(int R, int tile_rows, bool pipelined, bool mtaps, int ctas);
size_t gabor_fp32_smem_budget(int ctas);
size_t gabor_fp32_smem_bytes(const FreqDev &f);
cudaError_t launch_gabor_fp32(const BankArgs &a, int nitems, size_t smem, int sm_count, cudaStream_t st);
cudaError_t gabor_fp32_prepare();
cudaError_t launch_sdft_fp32(SdftArgs a, int sm_count, cudaStream_t st);
cudaError_t sdft_fp32_prepare();
// dst (W x H) = the transpose of an H x W image with row pitch `pitch`.
cudaError_t launch_transpose(const float *src, int64_t pitch, int H, int W, float *dst, cudaStream_t st);
// Tensor-core bank.
TcGeometry gabor_tc_geometry(int R);
bool gabor_tc_supported(int R);
// Modulated-tap row pass: tile geometry and the per-unit operand builder.
int gabor_tc_mt_tile_x();
int gabor_tc_mt_k(int R);
int gabor_tc_mt_pw(int R);
// split = 1: BF16 operands as hi + lo pairs (three products per K step).
int gabor_tc_mt_tile_y(int Kmax, int PWmax, int split);
size_t gabor_tc_smem_rows_mt(int Kmax, int PWmax, int TY, int split);
cudaError_t build_gabor_tc_am(uint16_t *Am, int R, double sigma, double wc, int split, cudaStream_t st);
cudaError_t build_gabor_tc_gm(uint16_t *Gm, int R, double sigma, double ws, int col_ty, int split, cudaStream_t st);
// 16-bit elements of one unit's modulated-tap operand strips (row pass; column pass of col_ty
// rows), both hi and lo under split.
int gabor_tc_mt_am_elems(int R, int split);
int gabor_tc_mt_gm_elems(int R, int col_ty, int split);
int gabor_tc_mt_col_stages(int col_kmax, int col_ty, int split);
bool gabor_tc_mt_fits(int row_kmax, int row_pwmax, int col_kmax, int split);
int gabor_tc_mt_col_ty(int col_kmax, int split);
cudaError_t build_gabor_tc_b(uint16_t *Brow, uint16_t *Bcol, int R, double sigma, int bf16, float *unscale,
                             cudaStream_t st);
cudaError_t gabor_tc_prepare();
cudaError_t launch_gabor_tc(const TcBankArgs &a, int sm_count, cudaStream_t st);
// The modulated-tap bank over a batch (a.imgs != nullptr): k_minmax, k_ones, the row and the
// column kernel, four launches for every image of the batch.
cudaError_t launch_gabor_tc_batch(const TcBankArgs &a, int sm_count, cudaStream_t st);
// Prefix sums of S(d) exp(i w^c d) and S(d) exp(i w^s d), d = -R .. R, per unit (FP64).
cudaError_t build_gabor_tc_prefix(const double *unit_w, const TcUnitDev *units, const TcFreqDev *freqs,
                                  const double *sigma, int nunits, int stride, double2 *pre, cudaStream_t st);
int gabor_tc_row_tile_x();
int gabor_tc_row_tile_y(int Rmax);
int gabor_tc_col_tile_y();
// Recursive-Gaussian bank (gabor_iir.cu).
cudaError_t gabor_iir_prepare();
bool gabor_iir_fits(int row_nsc, int col_nsc);   // the kernels' shared memory fits
size_t gabor_iir_col_scratch_floats(int col_nsc);
int gabor_iir_col_ctas(int W, int nunits);
cudaError_t launch_gabor_iir(const IirArgs &a, cudaStream_t st);
// FP32 FMA throughput probe (peak.cu).
cudaError_t launch_fma_peak(float *out, int blocks, int iters, int packed, cudaStream_t st);
cudaError_t launch_store_pattern(float2 *out, int64_t nplanes, int H, int W, int ctas, cudaStream_t st);
// Bounded-wait self-test (selftest.cu).
cudaError_t launch_wait_selftest(int *status, int signal, unsigned long long limit_ns, cudaStream_t st);
// Sets the message returned by gabor_bank_last_error() on the calling host thread.
void set_last_error(const char *msg);
// Argument checks shared by the entry points that take one image and one output (GB_OK or
// GB_ERR_INVALID_ARG with the message set), and the check for a CUDA error left by earlier
// work (GB_ERR_CUDA, cleared).
gb_status validate_image(const void *img, int H, int W, int64_t pitch, const void *out);
gb_status check_sticky();
// Tensor-core SDFT (windowed-DFT contraction on tcgen05).
bool sdft_tc_supported(int Mx, int My);
int sdft_tc_b_bytes(int Mx, int My);
cudaError_t build_sdft_tc_b(void *Bdev, double sigma, int Mx, int My, int bf16, float *b_unscale, cudaStream_t st);
cudaError_t sdft_tc_prepare();
// TMA-fed kernel (Mx in {8, 16, 32, 64}, Mx * My a multiple of 64): its workspace holds the
// row-unfolded image; other windows build A in shared memory from a staged patch.
bool sdft_tc_tma_ok(int Mx, int My);
int64_t sdft_tc_ws_bytes(int H, int W, int Mx, int My);
// ws: sdft_tc_ws_bytes() bytes (16-byte aligned) when sdft_tc_tma_ok(), else unused (may be NULL).
cudaError_t launch_sdft_tc(const float *img, int64_t pitch, int H, int W, float2 *out, int Mx, int My, int half,
                           const void *Bdev, float b_unscale, int bf16, int bmode, int *status, int sm_count,
                           void *ws, cudaStream_t st);
// The driver's tensor-map encoder (fetched once through the runtime).
PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder();

}  // namespace gb

// The opaque handle.
struct gabor_bank {
    int device = 0;
    int sm_count = 152;
    gb_precision prec = GB_FP32;
    double rf = 3.0;
    std::vector<double> theta, omega, sigma;
    std::vector<gb::Freq> freqs;
    std::vector<gb::Unit> units;
    int tpad_max = 8;
    // options
    int reuse = 1;
    int tile_rows = 0;
    int segments = 0;
    int boundary = 0;                         // gb::BoundaryMode
    int smoother = 0;                         // 0 truncated Gaussian (FIR), 1 recursive Gaussian (IIR)
    int fp32_pipeline = 0;                    // GB_OPT_PIPELINE (0 automatic, 1 phased, 2 pipelined)
    bool fp32_pipelined = false;              // schedule of the current tables
    int fp32_row_form = 0;                    // GB_OPT_ROW_PASS (0 automatic, 1 demodulation, 2 modulated taps)
    int fp32_ctas_opt = 0;                    // GB_OPT_BANK_CTAS (0 automatic, 1, 2)
    int fp32_ctas = 1;                        // CTAs per SM of the current tables
    int sdft_form = 0;                        // GB_OPT_SDFT_FORM (0 automatic, 1 step by step, 2 modulated taps)
    int sdft_reuse = 1;                       // GB_OPT_SDFT_REUSE (1 reuse J_u, 0 the no-reuse ablation)
    int sdft_order = 0;                       // 0 automatic, 1 horizontal pass first, 2 vertical first
    float *d_transp = nullptr;                // transposed image for the vertical-first SDFT
    size_t transp_elems = 0;
    int layout = 0;                           // 0 plane-major, 1 pixel-major bank output
    int ph_margin = 0;                        // phase-table entries before 0 and after the capacity
    std::vector<int> ftile_rows, fsegments;   // per-frequency overrides (0 = global / automatic)
    int *d_counter = nullptr;                 // work-queue head of the FP32 bank kernel
    std::vector<gb::ImageDev> last_imgs;      // batch descriptors last uploaded
    // device tables
    double *d_unit_w = nullptr;  // [nunits][2] (omega cos / pi, omega sin / pi)
    double *d_sigma = nullptr;
    int *d_lo = nullptr, *d_T = nullptr;
    float *d_taps = nullptr;     // [n_freq][tpad_max]
    float2 *d_phx = nullptr;     // [nunits][Wcap + 2 ph_margin], position x at ph_margin + x
    float2 *d_phy = nullptr;     // [nunits][Hcap + 2 ph_margin]
    gb::UnitDev *d_unitdev = nullptr;
    gb::FreqDev *d_freqdev = nullptr;
    std::vector<gb::FreqDev> freqdev;       // host copy (taps pointers into d_taps)
    // TMA maps of the FP32 row loads, encoded for the image and geometry in raw_key (the
    // encoding costs host time every call would pay otherwise)
    std::vector<int64_t> raw_key;
    unsigned raw_mask = 0;
    CUtensorMap raw_maps[gb::kMaxRawMaps];
    // work lists of the FP32 bank kernel, keyed by the image shapes of a launch
    std::map<std::vector<int64_t>, std::pair<gb::WorkItem *, int>> worklists;
    size_t max_smem = 0;
    int Wcap = 0, Hcap = 0;
    bool tables_ready = false;
    // SDFT tables (rebuilt when sigma / M change)
    float *d_sdft_taps = nullptr;   // [2][kMaxSdftM + 8]
    float2 *d_sdft_tw = nullptr;    // [2][kMaxSdftM]
    double sdft_sigma = -1.0;
    int sdft_Mx = 0, sdft_My = 0;
    // tensor-core SDFT operand B (pre-swizzled FP16 / BF16), keyed by (sigma, Mx, My)
    void *d_sdft_B = nullptr;
    size_t sdft_B_bytes = 0;
    float sdft_B_unscale = 1.f;
    void *d_sdft_ws = nullptr;      // tensor-core SDFT workspace (max |f|, unfolded image)
    size_t sdft_ws_bytes = 0;
    double sdftB_sigma = -1.0;
    int sdftB_Mx = 0, sdftB_My = 0;
    // tensor-core bank: B operands per frequency, unit descriptors, intermediate signals
    uint16_t *d_tcB = nullptr;
    uint16_t *d_tcAm = nullptr;               // modulated-tap row operands, one per unit
    gb::TcFreqDev *d_tcfreq = nullptr;
    gb::TcUnitDev *d_tcunit = nullptr;
    uint16_t *d_tcsig = nullptr;    // library-owned intermediate (when no workspace is attached)
    size_t tcsig_elems = 0;
    uint16_t *ws_ptr = nullptr;     // caller-owned workspace (gabor_bank_set_workspace), or nullptr
    size_t ws_bytes = 0;
    int *d_tcforder = nullptr;      // frequencies, largest radius first
    int tc_nsig = 0;                // column signals of all units
    int tc_nu_f = 0, tc_np_f = 0;   // units per frequency, paired units per frequency
    int tc_row_kmax = 0, tc_row_pwmax = 0, tc_col_kmax = 0;
    unsigned *d_tcminmax = nullptr;   // [2] image min / max keys
    double2 *d_tcpre = nullptr;       // prefix sums of the kernel taps per unit (F[1] tables)
    int tc_pre_stride = 0;
    int tc_row_ty = 64;
    int tc_mt_kmax = 0, tc_mt_pwmax = 0, tc_mt_ty = 64;   // modulated-tap row pass geometry
    bool tc_mt_ok = false;                    // the modulated-tap kernels fit every frequency
    int tc_row_ty_opt = 0, tc_col_ty_opt = 0; // GB_OPT_TC_TILES (0 automatic, 32, 64)
    uint16_t *d_tcGm = nullptr;               // modulated-tap column operands, one per unit
    int tc_H = 0, tc_W = 0, tc_Lpad = 0;
    int tc_zero_mt = -1;   // the intermediate layout whose halo was last zeroed (1: modulated taps)
    int64_t tc_Hp = 0;
    bool tc_ready = false;
    size_t tc_smem_rows = 0, tc_smem_cols = 0;
    // recursive-Gaussian path: coefficients per frequency and a library-owned workspace
    gb::IirFreq *d_iirfreq = nullptr;
    unsigned char *d_iirws = nullptr;
    size_t iirws_bytes = 0;
    // device status word (bounded waits)
    int *d_status = nullptr;
    // batch image descriptors
    gb::ImageDev *d_imgs = nullptr;
    int imgs_cap = 0;
    // host-buffer staging
    float *d_stage_img = nullptr;
    size_t stage_img_bytes = 0;
    void *d_stage_out = nullptr;
    size_t stage_out_bytes = 0;
    // tensor-core batches (modulated-tap kernels): workspace (intermediates, F[1] tables,
    // partial min / max keys, per-image centres), device image views, TMA maps and item lists,
    // with the key of the batch they were built for
    unsigned char *d_tcb_ws = nullptr;
    size_t tcb_ws_bytes = 0;
    gb::TcImgDev *d_tcb_imgs = nullptr;
    CUtensorMap *d_tcb_maps = nullptr;
    int tcb_cap = 0;
    int4 *d_tcb_rows = nullptr, *d_tcb_cols = nullptr;
    size_t tcb_rows_cap = 0, tcb_cols_cap = 0;
    int tcb_nrow = 0, tcb_ncol = 0;
    std::vector<int64_t> tcb_key;
    cudaStream_t copy_stream = nullptr;       // device-to-host copies of finished frequencies
    std::vector<cudaEvent_t> freq_done;       // one per frequency, plus one for the call's start
};
