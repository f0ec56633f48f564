// C ABI of the gaborbank library: argument validation, plan construction (Algorithm 1's
// orientation pairing), table management, dispatch to the kernels.  See include/gaborbank.h
// for the contract of every entry point.
#include <algorithm>
#include <cmath>
#include <mutex>

#include <cudaTypedefs.h>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>

#include "internal.h"

using namespace gb;

namespace {

thread_local std::string g_err;

gb_status fail(gb_status s, const std::string &msg)
{
    g_err = msg;
    return s;
}

#define GB_CU(call)                                                                          \
    do {                                                                                     \
        cudaError_t e_ = (call);                                                             \
        if (e_ != cudaSuccess)                                                               \
            return fail(GB_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_));    \
    } while (0)

#define GB_TRY(call)                                                                         \
    do {                                                                                     \
        gb_status s_ = (call);                                                               \
        if (s_ != GB_OK) return s_;                                                          \
    } while (0)

// Makes the handle's device current for the duration of a call and restores the caller's.
struct DeviceGuard {
    int prev = -1;
    bool ok = true;
    explicit DeviceGuard(int dev)
    {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (prev != dev) ok = cudaSetDevice(dev) == cudaSuccess;
    }
    ~DeviceGuard()
    {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

template <typename T>
gb_status dalloc(T **p, size_t n)
{
    *p = nullptr;
    if (n == 0) return GB_OK;
    cudaError_t e = cudaMalloc(reinterpret_cast<void **>(p), n * sizeof(T));
    if (e != cudaSuccess) {
        *p = nullptr;
        cudaGetLastError();
        return fail(GB_ERR_OUT_OF_MEMORY, std::string("cudaMalloc: ") + cudaGetErrorString(e));
    }
    return GB_OK;
}

template <typename T>
void dfree(T *&p)
{
    if (p) cudaFree(p);
    p = nullptr;
}

int radius_of(double sigma, double rf) { return (int)std::ceil(rf * sigma - 1e-9); }

// Samples a recursive pass extends a signal by on each side.
int iir_pad(double sigma) { return (int)std::ceil(12.0 * sigma) + 32; }

// Young and van Vliet's recursive Gaussian (Signal Processing 44, 1995): q from sigma (two
// fitted branches), the third-order coefficients b0..b3 and the gain B, for
// w[n] = B x[n] + (b1 w[n-1] + b2 w[n-2] + b3 w[n-3]) / b0; stored for the difference form
// (c0 = B, e1 = (b2 + b3) / b0, c3 = b3 / b0, kept as ce = c0 + e1) with the powers
// A^(16 * 2^i) of its zero-input state matrix, all in FP64 before rounding.
IirFreq iir_coefficients(double sigma)
{
    const double q = sigma >= 2.5 ? 0.98711 * sigma - 0.96330 : 3.97156 - 4.14554 * std::sqrt(1.0 - 0.26891 * sigma);
    const double q2 = q * q, q3 = q2 * q;
    const double b0 = 1.57825 + 2.44413 * q + 1.4281 * q2 + 0.422205 * q3;
    const double b1 = 2.44413 * q + 2.85619 * q2 + 1.26661 * q3;
    const double b2 = -(1.4281 * q2 + 1.26661 * q3);
    const double b3 = 0.422205 * q3;
    const double c0 = 1.0 - (b1 + b2 + b3) / b0, e1 = (b2 + b3) / b0, c3 = b3 / b0;
    IirFreq f{};
    f.c0 = (float)c0;
    f.ce = (float)(c0 + e1);
    f.c3 = (float)c3;
    f.P = iir_pad(sigma);
    // state (w1, d1, d2); one zero-input step: D = -c0 w1 - e1 d1 - c3 d2, (w1 + D, D, d1)
    double A[9] = {1.0 - c0, -e1, -c3, -c0, -e1, -c3, 0.0, 1.0, 0.0};
    auto mul = [](const double *x, const double *y, double *z) {
        double t[9];
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j)
                t[3 * i + j] = x[3 * i] * y[j] + x[3 * i + 1] * y[3 + j] + x[3 * i + 2] * y[6 + j];
        std::copy(t, t + 9, z);
    };
    double M[9] = {1, 0, 0, 0, 1, 0, 0, 0, 1};
    for (int k = 0; k < kIirChunk; ++k) mul(M, A, M);
    for (int l = 0; l < kIirLevels; ++l) {
        for (int i = 0; i < 9; ++i) f.m[l][i] = (float)M[i];
        mul(M, M, M);
    }
    return f;
}

// Pairs theta with pi - theta (Algorithm 1: J_{pi - theta} = J*_theta) and lays out the
// units of every frequency: paired units first, then unpaired ones, each in theta order.
void build_plan(gabor_bank *h)
{
    h->freqs.clear();
    h->units.clear();
    h->tpad_max = 8;
    const int K = (int)h->theta.size();
    for (int s = 0; s < (int)h->omega.size(); ++s) {
        Freq f;
        f.omega = h->omega[s];
        f.sigma = h->sigma[s];
        f.R = radius_of(f.sigma, h->rf);
        f.T = 2 * f.R + 1;
        f.Tpad = (f.T + 7) / 8 * 8;
        h->tpad_max = std::max(h->tpad_max, f.Tpad);
        f.u0 = (int)h->units.size();
        std::vector<char> used(K, 0);
        std::vector<Unit> fu;
        for (int k = 0; k < K; ++k) {
            if (used[k]) continue;
            used[k] = 1;
            Unit u;
            u.s = s;
            u.k_a = k;
            u.k_b = -1;
            if (h->reuse) {
                for (int j = 0; j < K; ++j) {
                    if (!used[j] && std::fabs(h->theta[k] + h->theta[j] - M_PI) < 1e-9) {
                        u.k_b = j;
                        used[j] = 1;
                        break;
                    }
                }
            }
            u.wc = f.omega * std::cos(h->theta[k]);
            u.ws = f.omega * std::sin(h->theta[k]);
            fu.push_back(u);
        }
        std::stable_partition(fu.begin(), fu.end(), [](const Unit &u) { return u.k_b >= 0; });
        h->units.insert(h->units.end(), fu.begin(), fu.end());
        f.u1 = (int)h->units.size();
        h->freqs.push_back(f);
    }
    // Phase tables also cover the positions a non-zero boundary rule reads beyond the image:
    // up to R + 128 columns (a 128-column tensor-core tile plus its halo) and rows.
    int rmax = 0;
    for (const Freq &f : h->freqs) rmax = std::max(rmax, std::max(f.R, iir_pad(f.sigma)));
    h->ph_margin = (rmax + 63) / 64 * 64 + 128;
}

void free_tables(gabor_bank *h)
{
    dfree(h->d_unit_w);
    dfree(h->d_sigma);
    dfree(h->d_lo);
    dfree(h->d_T);
    dfree(h->d_taps);
    dfree(h->d_phx);
    dfree(h->d_phy);
    dfree(h->d_unitdev);
    dfree(h->d_freqdev);
    for (auto &kv : h->worklists) cudaFree(kv.second.first);
    h->worklists.clear();
    h->freqdev.clear();
    h->Wcap = h->Hcap = 0;
    h->tables_ready = false;
    h->tc_H = h->tc_W = 0;   // the tensor-core intermediate's halo is re-zeroed on next use
}

// Device tables of the plan: taps per frequency, phase tables per unit (K0, FP64).
int twin_of(const gabor_bank *h, int ui);

gb_status ensure_tables(gabor_bank *h, int H, int W, cudaStream_t st)
{
    const int nu = (int)h->units.size();
    const int nf = (int)h->freqs.size();
    if (nu == 0) return GB_OK;
    if (h->tables_ready && W <= h->Wcap && H <= h->Hcap) return GB_OK;
    // Tables may be in use by earlier work on any stream.
    GB_CU(cudaDeviceSynchronize());
    const int Wcap = std::max(W, h->Wcap), Hcap = std::max(H, h->Hcap);
    free_tables(h);
    GB_TRY(dalloc(&h->d_unit_w, 2 * (size_t)nu));
    GB_TRY(dalloc(&h->d_sigma, (size_t)nf));
    GB_TRY(dalloc(&h->d_lo, (size_t)nf));
    GB_TRY(dalloc(&h->d_T, (size_t)nf));
    GB_TRY(dalloc(&h->d_taps, (size_t)nf * h->tpad_max));
    const int mg = h->ph_margin;
    GB_TRY(dalloc(&h->d_phx, (size_t)nu * (Wcap + 2 * mg)));
    GB_TRY(dalloc(&h->d_phy, (size_t)nu * (Hcap + 2 * mg)));
    GB_TRY(dalloc(&h->d_unitdev, (size_t)nu));
    GB_TRY(dalloc(&h->d_freqdev, (size_t)nf));
    std::vector<double> w(2 * nu), sg(nf);
    std::vector<int> lo(nf), T(nf);
    std::vector<UnitDev> ud(nu);
    for (int i = 0; i < nu; ++i) {
        w[2 * i] = h->units[i].wc / M_PI;
        w[2 * i + 1] = h->units[i].ws / M_PI;
        const int K = (int)h->theta.size();
        ud[i].phx = h->d_phx + (size_t)i * (Wcap + 2 * mg) + mg;
        ud[i].phy = h->d_phy + (size_t)i * (Hcap + 2 * mg) + mg;
        ud[i].s = h->units[i].s;
        ud[i].twin = twin_of(h, i);
        ud[i].plane_a = h->units[i].s * K + h->units[i].k_a;
        ud[i].plane_b = h->units[i].k_b >= 0 ? h->units[i].s * K + h->units[i].k_b : -1;
    }
    for (int s = 0; s < nf; ++s) {
        sg[s] = h->freqs[s].sigma;
        lo[s] = h->freqs[s].R;
        T[s] = h->freqs[s].T;
    }
    GB_CU(cudaMemcpy(h->d_unit_w, w.data(), w.size() * sizeof(double), cudaMemcpyHostToDevice));
    GB_CU(cudaMemcpy(h->d_sigma, sg.data(), nf * sizeof(double), cudaMemcpyHostToDevice));
    GB_CU(cudaMemcpy(h->d_lo, lo.data(), nf * sizeof(int), cudaMemcpyHostToDevice));
    GB_CU(cudaMemcpy(h->d_T, T.data(), nf * sizeof(int), cudaMemcpyHostToDevice));
    GB_CU(cudaMemcpy(h->d_unitdev, ud.data(), nu * sizeof(UnitDev), cudaMemcpyHostToDevice));
    h->freqdev.resize(nf);
    // the pipelined schedule where every frequency's geometry fits, else the phased one; two
    // CTAs per SM where every frequency's geometry fits in half of the SM's shared memory
    h->fp32_pipelined = h->fp32_pipeline == 2;
    h->fp32_ctas = (!h->fp32_pipelined && h->fp32_ctas_opt == 2) ? 2 : 1;
    for (int pass = 0; pass < 3; ++pass) {
        h->max_smem = 0;
        for (int s = 0; s < nf; ++s) {
            const int tr = (s < (int)h->ftile_rows.size() && h->ftile_rows[s] > 0) ? h->ftile_rows[s] : h->tile_rows;
            FreqDev fd = gabor_fp32_geometry(h->freqs[s].R, tr, h->fp32_pipelined, h->fp32_row_form != 1, h->fp32_ctas);
            fd.taps = h->d_taps + (size_t)s * h->tpad_max;
            h->freqdev[s] = fd;
            h->max_smem = std::max(h->max_smem, gabor_fp32_smem_bytes(fd));
        }
        if (h->max_smem <= gabor_fp32_smem_budget(h->fp32_ctas)) break;
        if (h->fp32_pipelined)
            h->fp32_pipelined = false;
        else
            h->fp32_ctas = 1;
    }
    GB_CU(cudaMemcpy(h->d_freqdev, h->freqdev.data(), nf * sizeof(FreqDev), cudaMemcpyHostToDevice));
    GB_CU(launch_build_taps(h->d_sigma, h->d_lo, h->d_T, nf, h->tpad_max, h->d_taps, st));
    GB_CU(launch_build_gabor_tables(h->d_unit_w, nu, Wcap, Hcap, mg, h->d_phx, h->d_phy, st));
    h->Wcap = Wcap;
    h->Hcap = Hcap;
    h->tables_ready = true;
    return GB_OK;
}

gb_status ensure_sdft_tables(gabor_bank *h, double sigma, int My, int Mx, cudaStream_t st)
{
    if (h->sdft_sigma == sigma && h->sdft_Mx == Mx && h->sdft_My == My) return GB_OK;
    GB_CU(cudaStreamSynchronize(st));
    if (!h->d_sdft_taps) GB_TRY(dalloc(&h->d_sdft_taps, 2 * (size_t)(kMaxSdftM + 8)));
    if (!h->d_sdft_tw) GB_TRY(dalloc(&h->d_sdft_tw, 2 * (size_t)kMaxSdftM));
    double *d_sg = nullptr;
    int *d_lo = nullptr;
    GB_TRY(dalloc(&d_sg, 2));
    gb_status s = dalloc(&d_lo, 4);
    if (s != GB_OK) { dfree(d_sg); return s; }
    const double sg[2] = {sigma, sigma};
    const int lo[4] = {Mx / 2, My / 2, Mx, My};   // lo[0..1], then T[0..1]
    cudaError_t e = cudaMemcpy(d_sg, sg, sizeof(sg), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(d_lo, lo, sizeof(lo), cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = launch_build_taps(d_sg, d_lo, d_lo + 2, 2, kMaxSdftM + 8, h->d_sdft_taps, st);
    if (e == cudaSuccess) e = launch_build_twiddles(Mx, h->d_sdft_tw, st);
    if (e == cudaSuccess) e = launch_build_twiddles(My, h->d_sdft_tw + kMaxSdftM, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    dfree(d_sg);
    dfree(d_lo);
    if (e != cudaSuccess) return fail(GB_ERR_CUDA, std::string("sdft tables: ") + cudaGetErrorString(e));
    h->sdft_sigma = sigma;
    h->sdft_Mx = Mx;
    h->sdft_My = My;
    return GB_OK;
}

// FP32 bank items take two unpaired units of a frequency together ("twins") under the
// modulated-tap row pass: two row passes, and column passes that fill both halves of a CTA.
// Units of a frequency are ordered paired first; unpaired ones are twinned in order.
bool twins_on(const gabor_bank *h) { return h->fp32_row_form != 1; }

int paired_count(const gabor_bank *h, int s)
{
    int np = 0;
    for (int u = h->freqs[s].u0; u < h->freqs[s].u1; ++u) np += h->units[u].k_b >= 0;
    return np;
}

// The second unit of the twin item that unit ui leads, or -1.
int twin_of(const gabor_bank *h, int ui)
{
    const Unit &u = h->units[ui];
    if (!twins_on(h) || u.k_b >= 0) return -1;
    const Freq &f = h->freqs[u.s];
    const int k = ui - (f.u0 + paired_count(h, u.s));
    return (k % 2 == 0 && ui + 1 < f.u1) ? ui + 1 : -1;
}

// Unit ui is the second unit of a twin item (it has no items of its own).
bool twinned(const gabor_bank *h, int ui)
{
    const Unit &u = h->units[ui];
    if (!twins_on(h) || u.k_b >= 0) return false;
    return (ui - (h->freqs[u.s].u0 + paired_count(h, u.s))) % 2 == 1;
}

// Cost of one work item in FMA lanes: `rows` output rows of a 32-column strip, plus the
// 2R-row prologue of its horizontal pass (`planes` column planes, `rowpasses` row passes).
double item_cost(const FreqDev &f, int planes, int rowpasses, double rows)
{
    return 32.0 * f.Tpad * (rows * 2 * planes + (rows + 2 * f.R) * 2 * rowpasses);
}
double item_cost(const gabor_bank *h, int ui, double rows)
{
    const FreqDev &f = h->freqdev[h->units[ui].s];
    if (h->units[ui].k_b >= 0) return item_cost(f, 2, 1, rows);
    return twin_of(h, ui) >= 0 ? item_cost(f, 2, 2, rows) : item_cost(f, 1, 1, rows);
}

// Row segments per column strip of frequency s on an Hh-row image: the per-frequency
// override, else as many as keep one item under `cap` (and segments at least max(TH, 2R)
// rows long).
int segments_of(const gabor_bank *h, int s, int Hh, double cap)
{
    const FreqDev &f = h->freqdev[s];
    const int fseg = (s < (int)h->fsegments.size() && h->fsegments[s] > 0) ? h->fsegments[s] : h->segments;
    int nseg = fseg > 0 ? fseg : 1;
    if (fseg <= 0) {
        const int min_len = std::max(f.TH, 2 * f.R);
        while (item_cost(f, 2, 1, (double)Hh / nseg) > cap && Hh / (nseg + 1) >= min_len) ++nseg;
    }
    return std::max(1, std::min(nseg, Hh));
}

// Item-size cap of a launch over `shapes` (of frequency only_s, or of all when -1): a third of
// one resident CTA's share of the launch.
double item_cap(const gabor_bank *h, const std::vector<int64_t> &shapes, int only_s = -1)
{
    double total = 0;
    for (size_t i = 0; i + 1 < shapes.size(); i += 2) {
        const int nstrips = (int)((shapes[i + 1] + kStripW - 1) / kStripW);
        for (int u = 0; u < (int)h->units.size(); ++u)
            if (!twinned(h, u) && (only_s < 0 || h->units[u].s == only_s))
                total += nstrips * item_cost(h, u, (double)shapes[i]);
    }
    return total / std::max(1, h->sm_count * h->fp32_ctas) / 3.0;
}

// Work items of a single-image launch as groups decoded by the kernel (no device list):
// one group per (frequency, pairing), largest item first; only frequency only_s when >= 0.
// Returns false when the plan has more groups than the kernel arguments hold.
bool single_image_groups(const gabor_bank *h, int H, int W, BankArgs &a, int *nitems, int only_s = -1)
{
    const double cap = item_cap(h, {H, W}, only_s);
    const int nstrips = (W + kStripW - 1) / kStripW;
    struct G { double cost; ItemGroup g; int n; };
    std::vector<G> gs;
    for (int s = 0; s < (int)h->freqs.size(); ++s) {
        if (only_s >= 0 && s != only_s) continue;
        const int nseg = segments_of(h, s, H, cap);
        const int seg_len = (H + nseg - 1) / nseg;
        const int nseg_used = (H + seg_len - 1) / seg_len;
        const int np = paired_count(h, s);
        const int nu = h->freqs[s].u1 - h->freqs[s].u0;
        // paired units; twin items of unpaired units; an unpaired unit left over
        const int nun = nu - np, ntw = twins_on(h) ? nun / 2 : 0;
        const int u0 = h->freqs[s].u0;
        const int cnt[3] = {np, ntw, nun - 2 * ntw};
        const int first_unit[3] = {u0, u0 + np, u0 + np + 2 * ntw};
        for (int pass = 0; pass < 3; ++pass) {
            if (cnt[pass] == 0) continue;
            G g;
            g.cost = item_cost(h, first_unit[pass], seg_len);
            g.g = ItemGroup{0, first_unit[pass], nstrips, nseg_used, seg_len, pass == 1 ? 2 : 1};
            g.n = cnt[pass] * nstrips * nseg_used;
            gs.push_back(g);
        }
    }
    if (gs.size() > (size_t)kMaxGroups) return false;
    std::stable_sort(gs.begin(), gs.end(), [](const G &p, const G &q) { return p.cost > q.cost; });
    int first = 0;
    for (size_t i = 0; i < gs.size(); ++i) {
        a.groups[i] = gs[i].g;
        a.groups[i].first = first;
        first += gs[i].n;
    }
    a.ngroups = (int)gs.size();
    *nitems = first;
    return true;
}

// Work list of one launch over `shapes` (H, W pairs): every (image, unit, strip, segment),
// most expensive first.  Segments are cut so that no item exceeds ~1/3 of an SM's share.
gb_status get_worklist(gabor_bank *h, const std::vector<int64_t> &shapes, WorkItem **items, int *n)
{
    auto itr = h->worklists.find(shapes);
    if (itr != h->worklists.end()) {
        *items = itr->second.first;
        *n = itr->second.second;
        return GB_OK;
    }
    const int nimg = (int)shapes.size() / 2;
    struct Cand { double cost; WorkItem w; };
    std::vector<Cand> cands;
    const double cap = item_cap(h, shapes);
    for (int i = 0; i < nimg; ++i) {
        const int Hh = (int)shapes[2 * i], Ww = (int)shapes[2 * i + 1];
        const int nstrips = (Ww + kStripW - 1) / kStripW;
        for (int s = 0; s < (int)h->freqs.size(); ++s) {
            const int seg_len = (Hh + segments_of(h, s, Hh, cap) - 1) / segments_of(h, s, Hh, cap);
            for (int ui = h->freqs[s].u0; ui < h->freqs[s].u1; ++ui) {
                if (twinned(h, ui)) continue;   // covered by the items of its twin
                for (int st = 0; st < nstrips; ++st)
                    for (int y0 = 0; y0 < Hh; y0 += seg_len) {
                        Cand c;
                        c.w = WorkItem{i, ui, st, y0, std::min(Hh, y0 + seg_len)};
                        c.cost = item_cost(h, ui, c.w.y1 - c.w.y0);
                        cands.push_back(c);
                    }
            }
        }
    }
    std::stable_sort(cands.begin(), cands.end(), [](const Cand &a, const Cand &b) { return a.cost > b.cost; });
    std::vector<WorkItem> w(cands.size());
    for (size_t k = 0; k < cands.size(); ++k) w[k] = cands[k].w;
    WorkItem *d = nullptr;
    GB_TRY(dalloc(&d, w.size()));
    GB_CU(cudaMemcpy(d, w.data(), w.size() * sizeof(WorkItem), cudaMemcpyHostToDevice));
    h->worklists[shapes] = {d, (int)w.size()};
    *items = d;
    *n = (int)w.size();
    return GB_OK;
}

// Tensor-core bank state: B operands, frequency and unit descriptors (once per plan; unit
// descriptors again when the phase tables move) and the library-owned intermediate.
void free_tc_batch(gabor_bank *h)
{
    dfree(h->d_tcb_ws);
    h->tcb_ws_bytes = 0;
    dfree(h->d_tcb_imgs);
    dfree(h->d_tcb_maps);
    h->tcb_cap = 0;
    dfree(h->d_tcb_rows);
    dfree(h->d_tcb_cols);
    h->tcb_rows_cap = h->tcb_cols_cap = 0;
    h->tcb_key.clear();
}

void free_tc(gabor_bank *h)
{
    free_tc_batch(h);
    dfree(h->d_tcB);
    dfree(h->d_tcAm);
    dfree(h->d_tcGm);
    dfree(h->d_tcfreq);
    dfree(h->d_tcunit);
    dfree(h->d_tcsig);
    dfree(h->d_tcforder);
    dfree(h->d_tcminmax);
    dfree(h->d_tcpre);
    h->tcsig_elems = 0;
    h->tc_H = h->tc_W = 0;
    h->tc_ready = false;
}

// Lpad (rows of zero halo above the image in the intermediate) of the plan.
int tc_lpad(const gabor_bank *h)
{
    int rmax = 0;
    for (const Freq &f : h->freqs) rmax = std::max(rmax, f.R);
    return ((rmax + 64) + 63) / 64 * 64;
}

// Output rows per column job of the modulated-tap column kernel: the GB_OPT_TC_TILES choice
// where it fits, else the largest that fits.
int tc_col_ty(const gabor_bank *h)
{
    const int split = h->prec == GB_BF16_TC;
    const int auto_ty = gabor_tc_mt_col_ty(h->tc_col_kmax, split);
    return (h->tc_col_ty_opt == 32 || (h->tc_col_ty_opt == 64 && auto_ty == 64)) ? h->tc_col_ty_opt : auto_ty;
}

// Elements of the intermediate for an H x W image: every column signal of every unit, one
// column of Hp = round64(H) + 2 Lpad rows per image column.
int tc_wq(int W) { return (W + 15) / 16 * 16; }
int64_t tc_sig_elems(const gabor_bank *h, int H, int W)
{
    const int64_t Hp = (int64_t)(H + 63) / 64 * 64 + 2 * tc_lpad(h);
    int64_t nsig = 0;
    for (const Unit &u : h->units) nsig += u.k_b >= 0 ? 4 : 2;
    // modulated taps: a plane of Re J, Im J per unit (two, hi and lo, under BF16), Wq columns
    const int64_t mt = (int64_t)(h->prec == GB_BF16_TC ? 2 : 1) * (int64_t)h->units.size() * 2 * tc_wq(W) * Hp;
    return std::max(nsig * W * Hp, mt);
}

// Workspace bytes of a tensor-core call: the intermediate signals, then the F[1] tables A, B.
int64_t tc_sig_bytes(const gabor_bank *h, int H, int W) { return (tc_sig_elems(h, H, W) * 2 + 255) / 256 * 256; }
// F[1] tables: A(x), B(y) of every unit (float2), 256-byte aligned
int64_t tc_ones_bytes(const gabor_bank *h, int H, int W)
{
    return ((int64_t)h->units.size() * ((int64_t)W + H) * (int64_t)sizeof(float2) + 255) / 256 * 256;
}
// the column pass's correction operands: per unit one block per 64 columns and per 32 rows
// (enough for either column-job height)
int64_t tc_corr_bytes(const gabor_bank *h, int H, int W)
{
    return (int64_t)h->units.size() * (((int64_t)W + 63) / 64 + ((int64_t)H + 31) / 32) * kCorrBlockHalfs * 2;
}
// the row pass's operand image (modulated taps under the zero rule): H rows of W rounded up
// to 8 FP16 elements, twice (hi, lo) under BF16
int64_t tc_pimg_pitch(int W) { return (W + 7) / 8 * 8; }
int64_t tc_pimg_bytes(const gabor_bank *h, int H, int W)
{
    return ((int64_t)(h->prec == GB_BF16_TC ? 2 : 1) * H * tc_pimg_pitch(W) * 2 + 255) / 256 * 256;
}
int64_t tc_ws_bytes(const gabor_bank *h, int H, int W)
{
    return tc_sig_bytes(h, H, W) + tc_ones_bytes(h, H, W) + tc_corr_bytes(h, H, W) + tc_pimg_bytes(h, H, W);
}

gb_status ensure_tc(gabor_bank *h, cudaStream_t st)
{
    const int nf = (int)h->freqs.size(), nu = (int)h->units.size();
    const int bf16 = h->prec == GB_BF16_TC;
    const int split = bf16;   // BF16: the modulated-tap operands as hi + lo pairs
    if (h->tc_ready) return GB_OK;
    size_t total = 0;
    std::vector<size_t> off_r(nf), off_c(nf);
    h->tc_row_kmax = h->tc_row_pwmax = h->tc_col_kmax = 0;
    int rmax = 0;
    for (int s = 0; s < nf; ++s) {
        const TcGeometry g = gabor_tc_geometry(h->freqs[s].R);
        off_r[s] = total;
        total += (size_t)gabor_tc_row_tile_x() * g.Krow;
        off_c[s] = total;
        total += (size_t)gabor_tc_col_tile_y() * g.Kcol;
        h->tc_row_kmax = std::max(h->tc_row_kmax, g.Krow);
        h->tc_row_pwmax = std::max(h->tc_row_pwmax, g.PW);
        h->tc_col_kmax = std::max(h->tc_col_kmax, g.Kcol);
        rmax = std::max(rmax, h->freqs[s].R);
    }
    h->tc_row_ty = gabor_tc_row_tile_y(rmax);
    // every frequency has the same units (the pairing depends on theta only)
    h->tc_nu_f = nf > 0 ? h->freqs[0].u1 - h->freqs[0].u0 : 0;
    h->tc_np_f = 0;
    for (int u = 0; u < h->tc_nu_f; ++u) h->tc_np_f += h->units[u].k_b >= 0;
    h->tc_nsig = 0;
    for (const Unit &u : h->units) h->tc_nsig += u.k_b >= 0 ? 4 : 2;
    GB_TRY(dalloc(&h->d_tcB, total));
    GB_TRY(dalloc(&h->d_tcfreq, (size_t)nf));
    GB_TRY(dalloc(&h->d_tcforder, (size_t)nf));
    GB_TRY(dalloc(&h->d_tcminmax, (size_t)2));
    GB_TRY(dalloc(&h->d_tcunit, (size_t)nu));
    std::vector<TcFreqDev> fd(nf);
    for (int s = 0; s < nf; ++s) {
        const TcGeometry g = gabor_tc_geometry(h->freqs[s].R);
        float unscale = 1.f;
        GB_CU(build_gabor_tc_b(h->d_tcB + off_r[s], h->d_tcB + off_c[s], g.R, h->freqs[s].sigma, bf16, &unscale, st));
        fd[s] = TcFreqDev{h->d_tcB + off_r[s], h->d_tcB + off_c[s], g.R, g.R8, g.Krow, g.Kcol, unscale, unscale,
                          h->freqs[s].u0, gabor_tc_mt_k(g.R)};
    }
    std::vector<int> order(nf);
    for (int s = 0; s < nf; ++s) order[s] = s;
    std::stable_sort(order.begin(), order.end(), [&](int p, int q) { return h->freqs[p].R > h->freqs[q].R; });
    // modulated-tap row operands: one [128][Kmt] block per unit
    std::vector<size_t> off_am(nu);
    size_t am_total = 0;
    h->tc_mt_kmax = h->tc_mt_pwmax = 0;
    for (int i = 0; i < nu; ++i) {
        const int R = h->freqs[h->units[i].s].R;
        off_am[i] = am_total;
        am_total += ((size_t)gabor_tc_mt_am_elems(R, split) + 127) / 128 * 128;   // 256-byte aligned strips
        h->tc_mt_kmax = std::max(h->tc_mt_kmax, gabor_tc_mt_k(R));
        h->tc_mt_pwmax = std::max(h->tc_mt_pwmax, gabor_tc_mt_pw(R));
    }
    h->tc_mt_ty = gabor_tc_mt_tile_y(h->tc_mt_kmax, h->tc_mt_pwmax, split);
    if (h->tc_row_ty_opt == 32) h->tc_mt_ty = 32;   // 64 only where it fits
    h->tc_mt_ok = gabor_tc_mt_fits(h->tc_mt_kmax, h->tc_mt_pwmax, h->tc_col_kmax, split);
    GB_TRY(dalloc(&h->d_tcAm, std::max<size_t>(am_total, 1)));
    std::vector<size_t> off_gm(nu);
    size_t gm_total = 0;
    const int col_ty = tc_col_ty(h);
    for (int i = 0; i < nu; ++i) {
        off_gm[i] = gm_total;
        gm_total += ((size_t)gabor_tc_mt_gm_elems(h->freqs[h->units[i].s].R, col_ty, split) + 127) / 128 * 128;
    }
    GB_TRY(dalloc(&h->d_tcGm, std::max<size_t>(gm_total, 1)));
    for (int i = 0; i < nu; ++i) {
        const Freq &fq = h->freqs[h->units[i].s];
        GB_CU(build_gabor_tc_am(h->d_tcAm + off_am[i], fq.R, fq.sigma, h->units[i].wc, split, st));
        GB_CU(build_gabor_tc_gm(h->d_tcGm + off_gm[i], fq.R, fq.sigma, h->units[i].ws, col_ty, split, st));
    }
    std::vector<TcUnitDev> ud(nu);
    const int K = (int)h->theta.size();
    int64_t sig = 0;
    for (int i = 0; i < nu; ++i) {
        const Unit &un = h->units[i];
        const bool paired = un.k_b >= 0;
        ud[i].phx = h->d_phx + (size_t)i * (h->Wcap + 2 * h->ph_margin) + h->ph_margin;
        ud[i].phy = h->d_phy + (size_t)i * (h->Hcap + 2 * h->ph_margin) + h->ph_margin;
        ud[i].s = un.s;
        ud[i].plane_a = un.s * K + un.k_a;
        ud[i].plane_b = paired ? un.s * K + un.k_b : -1;
        ud[i].pad_ = 0;
        ud[i].sig_idx = sig;
        ud[i].Am = h->d_tcAm + off_am[i];
        ud[i].Gm = h->d_tcGm + off_gm[i];
        sig += paired ? 4 : 2;
    }
    GB_CU(cudaMemcpy(h->d_tcfreq, fd.data(), nf * sizeof(TcFreqDev), cudaMemcpyHostToDevice));
    GB_CU(cudaMemcpy(h->d_tcforder, order.data(), nf * sizeof(int), cudaMemcpyHostToDevice));
    GB_CU(cudaMemcpy(h->d_tcunit, ud.data(), nu * sizeof(TcUnitDev), cudaMemcpyHostToDevice));
    h->tc_pre_stride = 2 * rmax + 2;
    GB_TRY(dalloc(&h->d_tcpre, (size_t)nu * 2 * h->tc_pre_stride));
    GB_CU(build_gabor_tc_prefix(h->d_unit_w, h->d_tcunit, h->d_tcfreq, h->d_sigma, nu, h->tc_pre_stride,
                                h->d_tcpre, st));
    h->tc_ready = true;
    return GB_OK;
}


// TMA map of the row pass's operand image (p_tma): W x H x (1, or 2 for hi and lo) 16-bit
// elements, boxes of 64 columns (128 bytes) x TY rows x 1 with the 128-byte swizzle (they land
// as the SW128 K-major P blocks the MMA reads), zeros outside the image.
gb_status encode_pimg_map(CUtensorMap *m, const uint16_t *pimg, int H, int W, int64_t pq, int split, int ty)
{
    PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
    if (!enc) return fail(GB_ERR_CUDA, "cuTensorMapEncodeTiled is not available from the driver");
    const cuuint64_t dims[3] = {(cuuint64_t)W, (cuuint64_t)H, (cuuint64_t)(split ? 2 : 1)};
    const cuuint64_t strides[2] = {(cuuint64_t)pq * 2, (cuuint64_t)pq * 2 * H};
    const cuuint32_t box[3] = {64, (cuuint32_t)ty, 1}, elem[3] = {1, 1, 1};
    const CUresult r = enc(m, split ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 3,
                           const_cast<uint16_t *>(pimg), dims, strides, box, elem, CU_TENSOR_MAP_INTERLEAVE_NONE,
                           CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                           CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return fail(GB_ERR_CUDA, "cuTensorMapEncodeTiled failed for the row operand image");
    return GB_OK;
}

// TMA maps of the blocked intermediate [signal][Hp / 8][W][8] for the column pass, as a 4-D
// tensor (8 rows of a block, W columns, signals, Hp / 8 blocks; FP16): boxes of 8 x 32 x 4 x 8
// and 8 x 64 x 2 x 8, no swizzle (they land as the MMA's K-major core matrices), zeros beyond
// the image width.
gb_status encode_tc_maps(TcBankArgs &a, int nsig, bool mt)
{
    PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
    if (!enc) return fail(GB_ERR_CUDA, "cuTensorMapEncodeTiled is not available from the driver");
    const cuuint64_t dims[4] = {8, (cuuint64_t)a.W, (cuuint64_t)nsig, (cuuint64_t)(a.Hp / 8)};
    const cuuint64_t strides[3] = {16, (cuuint64_t)a.Hp * a.W * 2, (cuuint64_t)a.W * 16};
    const cuuint32_t elem[4] = {1, 1, 1, 1};
    const cuuint32_t boxes[2][4] = {{8, 32, 4, 8}, {8, 64, 2, 8}};
    if (mt) {
        // modulated taps: nsig planes of [Hp / 8][Wq][part][8]; a box of 256 elements (16
        // columns x both parts x 8 rows, 512 contiguous bytes) x 4 column groups x 8 blocks lands
        // with operand row n = 2 x + part, K-group b 2048 bytes apart
        const cuuint64_t mdims[3] = {256, (cuuint64_t)(a.Wq / 16), (cuuint64_t)(a.Hp / 8) * nsig};
        const cuuint64_t mstrides[2] = {512, (cuuint64_t)a.Wq * 32};
        const cuuint32_t mbox[3] = {256, 4, 8};
        const CUresult r = enc(&a.tmA[0], CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 3, a.sig, mdims, mstrides, mbox, elem,
                               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                               CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r != CUDA_SUCCESS) return fail(GB_ERR_CUDA, "cuTensorMapEncodeTiled failed for the intermediate");
        if (a.p_tma) return encode_pimg_map(&a.tmA[1], a.pimg, a.H, a.W, a.pq, a.split, a.row_ty);
        return GB_OK;
    }
    for (int k = 0; k < 2; ++k) {
        const CUresult r = enc(&a.tmA[k], CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 4, a.sig, dims, strides, boxes[k], elem,
                               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                               CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r != CUDA_SUCCESS) return fail(GB_ERR_CUDA, "cuTensorMapEncodeTiled failed for the intermediate");
    }
    return GB_OK;
}

gb_status filter_device_tc(gabor_bank *h, const float *d_img, int H, int W, int64_t pitch, void *d_out,
                           cudaStream_t st)
{
    for (const Freq &f : h->freqs)
        if (!gabor_tc_supported(f.R))
            return fail(GB_ERR_UNSUPPORTED, "tensor-core bank supports radii up to 96 px");
    const int nf = (int)h->freqs.size();
    const int split = h->prec == GB_BF16_TC;
    const int64_t ny64 = (H + 63) / 64, nx32 = (W + 31) / 32, nx64 = (W + 63) / 64;
    // the unit descriptors point into the phase tables: (re)build them with the tables
    const bool tables_move = !(h->tables_ready && W <= h->Wcap && H <= h->Hcap);
    GB_TRY(ensure_tables(h, H, W, st));
    if (tables_move) free_tc(h);
    GB_TRY(ensure_tc(h, st));
    // both passes with modulated taps (64-column row tiles, J as the intermediate) unless
    // GB_OPT_ROW_PASS asks for the steps or a radius does not fit the kernels
    const bool row_mt = h->fp32_row_form != 1 && h->tc_mt_ok;
    if (split && !row_mt)
        return fail(GB_ERR_UNSUPPORTED,
                    "the BF16 bank (hi + lo operand pairs) runs with the modulated-tap kernels only: not under "
                    "GB_OPT_ROW_PASS = 1, nor when a radius does not fit them");
    const int ty = row_mt ? h->tc_mt_ty : h->tc_row_ty;
    const int tile_x = row_mt ? gabor_tc_mt_tile_x() : gabor_tc_row_tile_x();
    // Non-zero boundary rules: the row pass also produces the halo rows [-R, 0) and
    // [H, H + R) of the column signals, from the extended image.
    int rmax = 0;
    for (const Freq &f : h->freqs) rmax = std::max(rmax, f.R);
    const int ypad = h->boundary == kBoundaryZero ? 0 : (rmax + ty - 1) / ty * ty;
    const int64_t row_cnt = (int64_t)((H + 2 * ypad + ty - 1) / ty) * ((W + tile_x - 1) / tile_x);
    const int col_ty = tc_col_ty(h);   // modulated-tap column rows per job
    const int64_t ny_mt = (H + col_ty - 1) / col_ty;
    const int64_t col_cnt = row_mt ? ny_mt * h->tc_nu_f * nx64
                                   : ny64 * (h->tc_np_f * nx32 + (h->tc_nu_f - h->tc_np_f) * nx64);
    if ((int64_t)nf * std::max(row_cnt, col_cnt) > (int64_t)1 << 30)
        return fail(GB_ERR_UNSUPPORTED, "image too large for the tensor-core bank");
    const int Lpad = tc_lpad(h);
    const int64_t Hp = ny64 * 64 + 2 * Lpad;
    const int64_t need_bytes = tc_ws_bytes(h, H, W);
    const int64_t need = (need_bytes + 1) / 2;   // in 16-bit elements
    uint16_t *sig = h->ws_ptr;
    bool zero_halo = true;   // a caller-owned workspace may hold anything
    if (!sig) {
        if ((size_t)need > h->tcsig_elems) {
            // earlier work of this handle (on `st`) may still read the old buffer
            GB_CU(cudaStreamSynchronize(st));
            dfree(h->d_tcsig);
            h->tcsig_elems = 0;
            h->tc_H = h->tc_W = 0;
            GB_TRY(dalloc(&h->d_tcsig, (size_t)need));
            h->tcsig_elems = (size_t)need;
        }
        sig = h->d_tcsig;
        zero_halo = h->tc_H != H || h->tc_W != W || h->tc_zero_mt != (row_mt ? 1 : 0);
    } else if ((size_t)need_bytes > h->ws_bytes) {
        return fail(GB_ERR_BUDGET, "workspace too small: this image needs " + std::to_string(need_bytes) + " bytes");
    }
    float2 *onesA = reinterpret_cast<float2 *>(reinterpret_cast<char *>(sig) + tc_sig_bytes(h, H, W));
    float2 *onesB = onesA + (int64_t)h->units.size() * W;
    uint16_t *corrA = reinterpret_cast<uint16_t *>(reinterpret_cast<char *>(onesA) + tc_ones_bytes(h, H, W));
    uint16_t *corrB = corrA + (int64_t)h->units.size() * ((W + 63) / 64) * kCorrBlockHalfs;
    uint16_t *pimg = reinterpret_cast<uint16_t *>(reinterpret_cast<char *>(corrA) + tc_corr_bytes(h, H, W));
    if (zero_halo && need > 0) {
        // Layout [signal][Hp / 8][W][8].  The row pass writes rows [Lpad, Lpad + round_up(H, TY))
        // of every signal (zeros below row H); the column pass reads up to R8 rows beyond, so
        // the blocks of rows [0, Lpad) and [Lpad + round_up(H, 8), Hp) must be zero.
        // every signal either form uses (the modulated-tap form: 2 per unit, 4 as BF16 hi + lo)
        // (modulated taps: planes of Wq columns x both parts per 8-row block)
        const int64_t back = (Lpad + ((int64_t)H + 7) / 8 * 8) / 8;
        const size_t sig_bytes = row_mt ? (size_t)Hp * tc_wq(W) * 4 : (size_t)Hp * W * 2;
        const size_t blk = row_mt ? (size_t)tc_wq(W) * 32 : (size_t)W * 16;
        const size_t nsig_z = row_mt ? (size_t)(split ? 2 : 1) * h->units.size() : (size_t)h->tc_nsig;
        GB_CU(cudaMemset2DAsync(sig, sig_bytes, 0, (size_t)(Lpad / 8) * blk, nsig_z, st));
        GB_CU(cudaMemset2DAsync(reinterpret_cast<char *>(sig) + back * blk, sig_bytes, 0,
                                (size_t)(Hp / 8 - back) * blk, nsig_z, st));
    }
    h->tc_zero_mt = row_mt ? 1 : 0;
    h->tc_H = h->ws_ptr ? 0 : H;
    h->tc_W = h->ws_ptr ? 0 : W;
    TcBankArgs a{};
    a.img = d_img;
    a.pitch = pitch;
    a.H = H;
    a.W = W;
    a.out = reinterpret_cast<float2 *>(d_out);
    a.plane = (int64_t)H * W;
    a.sig = sig;
    a.Hp = Hp;
    a.Lpad = Lpad;
    a.Wq = tc_wq(W);
    a.freqs = h->d_tcfreq;
    a.units = h->d_tcunit;
    a.status = h->d_status;
    a.row_kmax = row_mt ? h->tc_mt_kmax : h->tc_row_kmax;
    a.row_pwmax = row_mt ? h->tc_mt_pwmax : h->tc_row_pwmax;
    a.row_mt = row_mt ? 1 : 0;
    a.col_kmax = h->tc_col_kmax;
    a.minmax = h->d_tcminmax;
    a.onesA = onesA;
    a.onesB = onesB;
    a.corrA = corrA;
    a.corrB = corrB;
    a.ones_pre = h->d_tcpre;
    a.ones_stride = h->tc_pre_stride;
    a.row_ty = ty;
    a.forder = h->d_tcforder;
    a.nf = nf;
    a.nu_f = h->tc_nu_f;
    a.np_f = h->tc_np_f;
    a.row_nx = (W + tile_x - 1) / tile_x;
    a.row_cnt = (int)row_cnt;
    a.col_ny = (int)(row_mt ? ny_mt : ny64);
    a.col_mt_ty = col_ty;
    a.col_nx32 = (int)nx32;
    a.col_nx64 = (int)nx64;
    a.col_cnt = (int)col_cnt;
    a.bmode = h->boundary;
    a.layout = h->layout;
    a.nplanes = (int)(h->omega.size() * h->theta.size());
    a.row_y0 = -ypad;
    a.split = split;
    a.p_tma = row_mt && h->boundary == kBoundaryZero ? 1 : 0;
    a.pimg = pimg;
    a.pq = tc_pimg_pitch(W);
    GB_TRY(encode_tc_maps(a, row_mt ? (split ? 2 : 1) * (int)h->units.size() : h->tc_nsig, row_mt));
    GB_CU(launch_gabor_tc(a, h->sm_count, st));
    return GB_OK;
}

// A batch on a tensor-core handle with the modulated-tap kernels: every image's row and column
// items in one launch each (after one k_minmax and one k_ones launch).  *done = false when the
// plan needs the step-by-step kernels (the caller then runs one bank pass per image).
gb_status filter_batch_tc(gabor_bank *h, int n, const float *const *d_imgs, const int *H, const int *W,
                          const int64_t *pitch, void *const *d_outs, cudaStream_t st, bool *done)
{
    *done = false;
    const int split = h->prec == GB_BF16_TC;
    for (const Freq &f : h->freqs)
        if (!gabor_tc_supported(f.R)) return fail(GB_ERR_UNSUPPORTED, "tensor-core bank supports radii up to 96 px");
    int Hm = 0, Wm = 0;
    for (int i = 0; i < n; ++i) {
        Hm = std::max(Hm, H[i]);
        Wm = std::max(Wm, W[i]);
    }
    const bool tables_move = !(h->tables_ready && Wm <= h->Wcap && Hm <= h->Hcap);
    GB_TRY(ensure_tables(h, Hm, Wm, st));
    if (tables_move) free_tc(h);
    GB_TRY(ensure_tc(h, st));
    if (h->fp32_row_form == 1 || !h->tc_mt_ok) return GB_OK;
    const int nf = (int)h->freqs.size(), nu = (int)h->units.size();
    const int ty = h->tc_mt_ty, tile_x = gabor_tc_mt_tile_x();
    const int col_ty = tc_col_ty(h);
    int rmax = 0;
    for (const Freq &f : h->freqs) rmax = std::max(rmax, f.R);
    const int ypad = h->boundary == kBoundaryZero ? 0 : (rmax + ty - 1) / ty * ty;
    const int Lpad = tc_lpad(h);
    const int nplane = (split ? 2 : 1) * nu;   // a plane of Re J, Im J per unit (hi and lo under BF16)
    // workspace: intermediates, F[1] tables, partial keys, centres (each 256-byte aligned)
    auto al = [](int64_t b) { return (b + 255) / 256 * 256; };
    std::vector<int64_t> off_sig(n), off_ones(n), off_corr(n), off_pimg(n), Hp(n);
    int64_t total = 0;
    for (int i = 0; i < n; ++i) {
        Hp[i] = (int64_t)(H[i] + 63) / 64 * 64 + 2 * Lpad;
        off_sig[i] = total;
        total += al((int64_t)nplane * tc_wq(W[i]) * Hp[i] * 4);
    }
    for (int i = 0; i < n; ++i) {
        off_ones[i] = total;
        total += al((int64_t)nu * ((int64_t)W[i] + H[i]) * (int64_t)sizeof(float2));
    }
    for (int i = 0; i < n; ++i) {
        off_corr[i] = total;
        total += al((int64_t)nu * (((int64_t)W[i] + 63) / 64 + ((int64_t)H[i] + 31) / 32) * kCorrBlockHalfs * 2);
    }
    const bool p_tma = h->boundary == kBoundaryZero;
    for (int i = 0; i < n; ++i) {
        off_pimg[i] = total;
        if (p_tma) total += tc_pimg_bytes(h, H[i], W[i]);
    }
    const int64_t off_parts = total;
    total += al((int64_t)n * kMmParts * 2 * sizeof(unsigned));
    const int64_t off_ce = total;
    total += al((int64_t)n * sizeof(float2));
    // the batch key: every pointer and shape, and the options the layout depends on
    std::vector<int64_t> key;
    key.reserve(5 * (size_t)n + 3);
    key.push_back(h->boundary);
    key.push_back(h->layout);
    key.push_back(total);
    for (int i = 0; i < n; ++i) {
        key.push_back((int64_t)reinterpret_cast<uintptr_t>(d_imgs[i]));
        key.push_back(pitch[i]);
        key.push_back(H[i]);
        key.push_back(W[i]);
        key.push_back((int64_t)reinterpret_cast<uintptr_t>(d_outs[i]));
    }
    if (key != h->tcb_key) {
        GB_CU(cudaStreamSynchronize(st));   // earlier batches of this handle may still use the buffers
        h->tcb_key.clear();
        if ((size_t)total > h->tcb_ws_bytes) {
            dfree(h->d_tcb_ws);
            h->tcb_ws_bytes = 0;
            GB_TRY(dalloc(&h->d_tcb_ws, (size_t)total));
            h->tcb_ws_bytes = (size_t)total;
        }
        if (n > h->tcb_cap) {
            dfree(h->d_tcb_imgs);
            dfree(h->d_tcb_maps);
            h->tcb_cap = 0;
            GB_TRY(dalloc(&h->d_tcb_imgs, (size_t)n));
            GB_TRY(dalloc(&h->d_tcb_maps, (size_t)2 * n));   // intermediates, then operand images
            h->tcb_cap = n;
        }
        unsigned char *ws = h->d_tcb_ws;
        std::vector<TcImgDev> imgs(n);
        std::vector<CUtensorMap> maps(2 * (size_t)n);
        PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
        if (!enc) return fail(GB_ERR_CUDA, "cuTensorMapEncodeTiled is not available from the driver");
        for (int i = 0; i < n; ++i) {
            TcImgDev &d = imgs[i];
            d.img = d_imgs[i];
            d.pitch = pitch[i];
            d.H = H[i];
            d.W = W[i];
            d.out = reinterpret_cast<float2 *>(d_outs[i]);
            d.plane = (int64_t)H[i] * W[i];
            d.sig = reinterpret_cast<uint16_t *>(ws + off_sig[i]);
            d.Hp = Hp[i];
            d.onesA = reinterpret_cast<const float2 *>(ws + off_ones[i]);
            d.onesB = d.onesA + (int64_t)nu * W[i];
            d.corrA = reinterpret_cast<uint16_t *>(ws + off_corr[i]);
            d.corrB = d.corrA + (int64_t)nu * ((W[i] + 63) / 64) * kCorrBlockHalfs;
            d.pimg = reinterpret_cast<uint16_t *>(ws + off_pimg[i]);
            d.pq = tc_pimg_pitch(W[i]);
            if (p_tma) GB_TRY(encode_pimg_map(&maps[n + i], d.pimg, H[i], W[i], d.pq, split, ty));
            // the intermediate's planes as in the single-image call: boxes of 256 elements (16
            // columns x both parts x 8 rows) x 4 column groups x 8 blocks
            d.Wq = tc_wq(W[i]);
            const cuuint64_t dims[3] = {256, (cuuint64_t)(d.Wq / 16), (cuuint64_t)(Hp[i] / 8) * nplane};
            const cuuint64_t strides[2] = {512, (cuuint64_t)d.Wq * 32};
            const cuuint32_t box[3] = {256, 4, 8}, elem[3] = {1, 1, 1};
            const CUresult r = enc(&maps[i], CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 3, d.sig, dims, strides, box, elem,
                                   CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                                   CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
            if (r != CUDA_SUCCESS) return fail(GB_ERR_CUDA, "cuTensorMapEncodeTiled failed for a batch intermediate");
        }
        // items: frequencies largest radius first (the row pass of frequency s covers every
        // unit of s), then images, then tiles
        std::vector<int> order(nf);
        for (int s2 = 0; s2 < nf; ++s2) order[s2] = s2;
        std::stable_sort(order.begin(), order.end(), [&](int p, int q) { return h->freqs[p].R > h->freqs[q].R; });
        std::vector<int4> rows, cols;
        for (int s2 : order)
            for (int i = 0; i < n; ++i) {
                const int nty = (H[i] + 2 * ypad + ty - 1) / ty, ntx = (W[i] + tile_x - 1) / tile_x;
                for (int r = 0; r < nty; ++r)
                    for (int c = 0; c < ntx; ++c) rows.push_back(make_int4(i, s2, -ypad + r * ty, c * tile_x));
            }
        for (int s2 : order)
            for (int i = 0; i < n; ++i) {
                const int ny = (H[i] + col_ty - 1) / col_ty, nx = (W[i] + 63) / 64;
                for (int u = h->freqs[s2].u0; u < h->freqs[s2].u1; ++u)
                    for (int r = 0; r < ny; ++r)
                        for (int c = 0; c < nx; ++c) cols.push_back(make_int4(i, u, c * 64, r * col_ty));
            }
        if (rows.size() > ((size_t)1 << 30) || cols.size() > ((size_t)1 << 30))
            return fail(GB_ERR_UNSUPPORTED, "batch too large for the tensor-core bank");
        if (rows.size() > h->tcb_rows_cap) {
            dfree(h->d_tcb_rows);
            h->tcb_rows_cap = 0;
            GB_TRY(dalloc(&h->d_tcb_rows, rows.size()));
            h->tcb_rows_cap = rows.size();
        }
        if (cols.size() > h->tcb_cols_cap) {
            dfree(h->d_tcb_cols);
            h->tcb_cols_cap = 0;
            GB_TRY(dalloc(&h->d_tcb_cols, cols.size()));
            h->tcb_cols_cap = cols.size();
        }
        GB_CU(cudaMemcpy(h->d_tcb_imgs, imgs.data(), n * sizeof(TcImgDev), cudaMemcpyHostToDevice));
        GB_CU(cudaMemcpy(h->d_tcb_maps, maps.data(), 2 * (size_t)n * sizeof(CUtensorMap), cudaMemcpyHostToDevice));
        if (!rows.empty())
            GB_CU(cudaMemcpy(h->d_tcb_rows, rows.data(), rows.size() * sizeof(int4), cudaMemcpyHostToDevice));
        if (!cols.empty())
            GB_CU(cudaMemcpy(h->d_tcb_cols, cols.data(), cols.size() * sizeof(int4), cudaMemcpyHostToDevice));
        // the intermediates' halo rows (above the image and below its last row tile) are read as
        // zeros and never written: clear the intermediates once per batch layout
        GB_CU(cudaMemsetAsync(h->d_tcb_ws, 0, (size_t)off_ones[0], st));
        GB_CU(cudaStreamSynchronize(st));
        h->tcb_nrow = (int)rows.size();
        h->tcb_ncol = (int)cols.size();
        h->tcb_key = key;
    }
    TcBankArgs a{};
    a.freqs = h->d_tcfreq;
    a.units = h->d_tcunit;
    a.status = h->d_status;
    a.row_kmax = h->tc_mt_kmax;
    a.row_pwmax = h->tc_mt_pwmax;
    a.row_mt = 1;
    a.col_kmax = h->tc_col_kmax;
    a.ones_pre = h->d_tcpre;
    a.ones_stride = h->tc_pre_stride;
    a.row_ty = ty;
    a.forder = h->d_tcforder;
    a.nf = nf;
    a.nu_f = h->tc_nu_f;
    a.np_f = h->tc_np_f;
    a.col_mt_ty = col_ty;
    a.bmode = h->boundary;
    a.layout = h->layout;
    a.nplanes = (int)(h->omega.size() * h->theta.size());
    a.row_y0 = -ypad;
    a.Lpad = Lpad;
    a.imgs = h->d_tcb_imgs;
    a.tmaps = h->d_tcb_maps;
    a.mm_part = reinterpret_cast<unsigned *>(h->d_tcb_ws + off_parts);
    a.img_ce = reinterpret_cast<float2 *>(h->d_tcb_ws + off_ce);
    a.row_list = h->d_tcb_rows;
    a.col_list = h->d_tcb_cols;
    a.n_row = h->tcb_nrow;
    a.n_col = h->tcb_ncol;
    a.nimg = n;
    a.split = split;
    a.p_tma = p_tma ? 1 : 0;
    GB_CU(launch_gabor_tc_batch(a, h->sm_count, st));
    *done = true;
    return GB_OK;
}

// The bank with the recursive Gaussian (GB_SMOOTHER_IIR): the row recursions write J into a
// library-owned workspace, the column recursions read it and write the bank.
gb_status filter_device_iir(gabor_bank *h, const float *d_img, int H, int W, int64_t pitch, void *d_out,
                            cudaStream_t st)
{
    if (h->prec != GB_FP32)
        return fail(GB_ERR_UNSUPPORTED, "the recursive Gaussian runs on the FP32 path only");
    for (const Freq &f : h->freqs)
        if (f.sigma < 0.5) return fail(GB_ERR_UNSUPPORTED, "the recursive Gaussian needs sigma >= 0.5");
    GB_TRY(ensure_tables(h, H, W, st));
    const int nf = (int)h->freqs.size();
    if (!h->d_iirfreq) {
        std::vector<IirFreq> fq(nf);
        for (int s = 0; s < nf; ++s) fq[s] = iir_coefficients(h->freqs[s].sigma);
        GB_TRY(dalloc(&h->d_iirfreq, (size_t)nf));
        GB_CU(cudaMemcpy(h->d_iirfreq, fq.data(), nf * sizeof(IirFreq), cudaMemcpyHostToDevice));
    }
    const bool ext = h->boundary != kBoundaryZero;
    int pmax = 0, wxmax = 0, hcmax = 0;
    for (const Freq &f : h->freqs) {
        const int P = iir_pad(f.sigma);
        pmax = std::max(pmax, P);
        wxmax = std::max(wxmax, (ext ? P : 0) + W + P);
        hcmax = std::max(hcmax, (ext ? P : 0) + H + P);
    }
    IirArgs a{};
    a.img = d_img;
    a.pitch = pitch;
    a.H = H;
    a.W = W;
    a.out = reinterpret_cast<float2 *>(d_out);
    a.layout = h->layout;
    a.nplanes = (int)(h->omega.size() * h->theta.size());
    a.bmode = h->boundary;
    a.nunits = (int)h->units.size();
    a.units = h->d_unitdev;
    a.freqs = h->d_iirfreq;
    a.Py = ext ? pmax : 0;
    a.Hr = H + 2 * a.Py;
    a.row_nsc = (wxmax + 511) / 512;
    a.col_nsc = (hcmax + 127) / 128;
    if (!gabor_iir_fits(a.row_nsc, a.col_nsc))
        return fail(GB_ERR_UNSUPPORTED, "the recursive Gaussian's extended rows or columns exceed its shared-memory plan");
    const size_t j_bytes = ((size_t)h->units.size() * a.Hr * W * sizeof(float2) + 255) / 256 * 256;
    const size_t need = j_bytes + (size_t)gabor_iir_col_ctas(W, (int)h->units.size()) *
                                      gabor_iir_col_scratch_floats(a.col_nsc) * sizeof(float);
    if (need > h->iirws_bytes) {
        GB_CU(cudaStreamSynchronize(st));   // earlier work of this handle may still use it
        dfree(h->d_iirws);
        h->iirws_bytes = 0;
        GB_TRY(dalloc(&h->d_iirws, need));
        h->iirws_bytes = need;
    }
    a.J = reinterpret_cast<float2 *>(h->d_iirws);
    a.col_scratch = reinterpret_cast<float *>(h->d_iirws + j_bytes);
    GB_CU(launch_gabor_iir(a, st));
    return GB_OK;
}

// TMA maps for the FP32 kernel's modulated-tap row loads of one image under the zero rule: per
// frequency a 2-D map of the image (W x H floats) with boxes of RW x TH (its raw buffer
// exactly).  Frequencies whose box exceeds the copy unit's 256 x 256 limit, images whose base
// or row pitch is not 16-byte aligned, and the other schedules keep the async copies.
gb_status encode_raw_maps(gabor_bank *h, BankArgs &a, const float *d_img, int H, int W, int64_t pitch)
{
    a.raw_mask = 0;
    const int nf = (int)h->freqs.size();
    if (!a.mtaps || a.pipelined || a.bmode != kBoundaryZero || nf > kMaxRawMaps) return GB_OK;
    if ((reinterpret_cast<uintptr_t>(d_img) & 15) != 0 || (pitch * 4) % 16 != 0) return GB_OK;
    std::vector<int64_t> key = {(int64_t)reinterpret_cast<uintptr_t>(d_img), H, W, pitch};
    for (int s = 0; s < nf; ++s) {
        key.push_back(h->freqdev[s].RW);
        key.push_back(h->freqdev[s].TH);
        key.push_back(h->freqdev[s].mtaps);
    }
    if (key != h->raw_key) {
        PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
        if (!enc) return GB_OK;
        h->raw_mask = 0;
        for (int s = 0; s < nf; ++s) {
            const FreqDev &f = h->freqdev[s];
            if (!f.mtaps || f.RW > 256 || f.TH > 256) continue;
            const cuuint64_t dims[2] = {(cuuint64_t)W, (cuuint64_t)H};
            const cuuint64_t strides[1] = {(cuuint64_t)pitch * 4};
            const cuuint32_t box[2] = {(cuuint32_t)f.RW, (cuuint32_t)f.TH}, elem[2] = {1, 1};
            const CUresult r = enc(&h->raw_maps[s], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float *>(d_img),
                                   dims, strides, box, elem, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                                   CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
            if (r == CUDA_SUCCESS) h->raw_mask |= 1u << s;
        }
        h->raw_key = key;
    }
    a.raw_mask = h->raw_mask;
    for (int s = 0; s < nf; ++s)
        if ((a.raw_mask >> s) & 1u) a.raw_map[s] = h->raw_maps[s];
    return GB_OK;
}

// The bank on one device image; only_s >= 0 (FP32 FIR path, plane-major layout, a plan with
// few enough groups) limits the launch to frequency only_s, whose planes it writes in place.
gb_status filter_device(gabor_bank *h, const float *d_img, int H, int W, int64_t pitch,
                        void *d_out, cudaStream_t st, int only_s = -1)
{
    if (h->smoother == GB_SMOOTHER_IIR) return filter_device_iir(h, d_img, H, W, pitch, d_out, st);
    if (h->prec != GB_FP32) return filter_device_tc(h, d_img, H, W, pitch, d_out, st);
    GB_TRY(ensure_tables(h, H, W, st));
    BankArgs a{};
    int n = 0;
    if (!single_image_groups(h, H, W, a, &n, only_s)) {
        if (only_s >= 0) return fail(GB_ERR_UNSUPPORTED, "per-frequency launch needs the decoded work groups");
        a.ngroups = 0;
        GB_TRY(get_worklist(h, {H, W}, const_cast<WorkItem **>(&a.items), &n));
    }
    a.img0 = ImageDev{d_img, pitch, reinterpret_cast<float2 *>(d_out), H, W};
    a.imgs = nullptr;
    a.freqs = h->d_freqdev;
    a.units = h->d_unitdev;
    a.counter = h->d_counter;
    a.bmode = h->boundary;
    a.layout = h->layout;
    a.nplanes = (int)(h->omega.size() * h->theta.size());
    a.status = h->d_status;
    a.pipelined = h->fp32_pipelined ? 1 : 0;
    a.mtaps = h->fp32_row_form != 1 ? 1 : 0;
    a.ctas = h->fp32_ctas;
    GB_TRY(encode_raw_maps(h, a, d_img, H, W, pitch));
    GB_CU(launch_gabor_fp32(a, n, h->max_smem, h->sm_count, st));
    return GB_OK;
}

}  // namespace

namespace gb {
// Records the message returned by gabor_bank_last_error() on this host thread.
void set_last_error(const char *msg) { g_err = msg; }

gb_status check_sticky()
{
    cudaError_t e = cudaPeekAtLastError();
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(GB_ERR_CUDA, std::string("earlier CUDA error: ") + cudaGetErrorString(e));
    }
    return GB_OK;
}

gb_status validate_image(const void *img, int H, int W, int64_t pitch, const void *out)
{
    if (!img || !out) return fail(GB_ERR_INVALID_ARG, "NULL image or output pointer");
    if (H <= 0 || W <= 0) return fail(GB_ERR_INVALID_ARG, "H and W must be positive");
    if (pitch < W) return fail(GB_ERR_INVALID_ARG, "pitch must be >= W");
    if ((int64_t)H * pitch > (int64_t)1 << 40) return fail(GB_ERR_INVALID_ARG, "image too large");
    if (reinterpret_cast<uintptr_t>(img) % 4) return fail(GB_ERR_INVALID_ARG, "image not 4-byte aligned");
    if (reinterpret_cast<uintptr_t>(out) % 8) return fail(GB_ERR_INVALID_ARG, "output not 8-byte aligned");
    return GB_OK;
}

// The driver's tensor-map encoder, fetched once through the runtime (no link against the
// driver library).
PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder()
{
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPoint("cuTensorMapEncodeTiled", &p, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    });
    return fn;
}
}  // namespace gb

extern "C" {

gb_status gabor_bank_create(gabor_bank_t *out, const double *theta, int n_theta,
                            const double *omega, const double *sigma, int n_freq,
                            double radius_factor, gb_precision prec, int max_H, int max_W)
{
    if (!out) return fail(GB_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (n_theta < 0 || n_freq < 0) return fail(GB_ERR_INVALID_ARG, "negative count");
    if ((n_theta == 0) != (n_freq == 0))
        return fail(GB_ERR_INVALID_ARG, "n_theta and n_freq must both be positive, or both 0");
    if (n_theta > 0 && (!theta || !omega || !sigma))
        return fail(GB_ERR_INVALID_ARG, "NULL theta/omega/sigma");
    if (n_theta > 4096 || n_freq > 4096) return fail(GB_ERR_INVALID_ARG, "too many filters");
    if (radius_factor == 0.0) radius_factor = 3.0;
    if (!std::isfinite(radius_factor) || radius_factor <= 0.0)
        return fail(GB_ERR_INVALID_ARG, "radius_factor must be positive and finite");
    if (prec != GB_FP32 && prec != GB_FP16_TC && prec != GB_BF16_TC)
        return fail(GB_ERR_INVALID_ARG, "unknown precision");
    if (max_H < 0 || max_W < 0) return fail(GB_ERR_INVALID_ARG, "negative max size");
    for (int k = 0; k < n_theta; ++k)
        if (!std::isfinite(theta[k])) return fail(GB_ERR_INVALID_ARG, "non-finite theta");
    for (int s = 0; s < n_freq; ++s) {
        if (!std::isfinite(omega[s])) return fail(GB_ERR_INVALID_ARG, "non-finite omega");
        if (!std::isfinite(sigma[s]) || sigma[s] <= 0.0)
            return fail(GB_ERR_INVALID_ARG, "sigma must be positive and finite");
        const double r = radius_factor * sigma[s];
        if (r > kMaxRadius || radius_of(sigma[s], radius_factor) > kMaxRadius)
            return fail(GB_ERR_UNSUPPORTED, "Gaussian radius above " + std::to_string(kMaxRadius) + " px");
    }
    gabor_bank *h = new (std::nothrow) gabor_bank();
    if (!h) return fail(GB_ERR_OUT_OF_MEMORY, "host allocation failed");
    h->prec = prec;
    h->rf = radius_factor;
    h->theta.assign(theta, theta + n_theta);
    h->omega.assign(omega, omega + n_freq);
    h->sigma.assign(sigma, sigma + n_freq);
    cudaError_t e = cudaGetDevice(&h->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&h->sm_count, cudaDevAttrMultiProcessorCount, h->device);
    if (e == cudaSuccess) e = gabor_fp32_prepare();
    if (e == cudaSuccess) e = sdft_fp32_prepare();
    if (e == cudaSuccess) e = sdft_tc_prepare();
    if (e == cudaSuccess) e = gabor_tc_prepare();
    if (e == cudaSuccess) e = gabor_iir_prepare();
    if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void **>(&h->d_status), sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(h->d_status, 0, sizeof(int));
    if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void **>(&h->d_counter), sizeof(int));
    if (e != cudaSuccess) {
        cudaGetLastError();
        dfree(h->d_status);
        dfree(h->d_counter);
        delete h;
        return fail(GB_ERR_CUDA, std::string("create: ") + cudaGetErrorString(e));
    }
    build_plan(h);
    if (max_H > 0 && max_W > 0 && !h->units.empty()) {
        gb_status s = ensure_tables(h, max_H, max_W, nullptr);
        if (s != GB_OK) {
            gabor_bank_destroy(h);
            return s;
        }
    }
    *out = h;
    return GB_OK;
}

gb_status gabor_bank_destroy(gabor_bank_t h)
{
    if (!h) return GB_OK;
    DeviceGuard g(h->device);
    cudaDeviceSynchronize();
    free_tables(h);
    dfree(h->d_sdft_taps);
    dfree(h->d_sdft_tw);
    dfree(h->d_status);
    dfree(h->d_counter);
    dfree(h->d_stage_img);
    dfree(h->d_imgs);
    dfree(h->d_iirfreq);
    dfree(h->d_iirws);
    dfree(h->d_transp);
    free_tc(h);
    if (h->d_sdft_B) cudaFree(h->d_sdft_B);
    h->d_sdft_B = nullptr;
    if (h->d_sdft_ws) cudaFree(h->d_sdft_ws);
    h->d_sdft_ws = nullptr;
    if (h->d_stage_out) cudaFree(h->d_stage_out);
    h->d_stage_out = nullptr;
    for (cudaEvent_t ev : h->freq_done) cudaEventDestroy(ev);
    if (h->copy_stream) cudaStreamDestroy(h->copy_stream);
    delete h;
    return GB_OK;
}

gb_status gabor_bank_filter(gabor_bank_t h, const float *d_img, int H, int W, int64_t pitch,
                            void *d_out, void *stream)
{
    if (!h) return fail(GB_ERR_INVALID_ARG, "NULL handle");
    GB_TRY(validate_image(d_img, H, W, pitch, d_out));
    if (h->units.empty()) return fail(GB_ERR_INVALID_ARG, "handle has no filter bank (SDFT-only)");
    DeviceGuard g(h->device);
    if (!g.ok) return fail(GB_ERR_CUDA, "cannot select the handle's device");
    GB_TRY(check_sticky());
    return filter_device(h, d_img, H, W, pitch, d_out, static_cast<cudaStream_t>(stream));
}

gb_status gabor_bank_filter_host(gabor_bank_t h, const float *h_img, int H, int W,
                                 int64_t pitch, void *h_out, void *stream)
{
    if (!h) return fail(GB_ERR_INVALID_ARG, "NULL handle");
    GB_TRY(validate_image(h_img, H, W, pitch, h_out));
    if (h->units.empty()) return fail(GB_ERR_INVALID_ARG, "handle has no filter bank (SDFT-only)");
    DeviceGuard g(h->device);
    if (!g.ok) return fail(GB_ERR_CUDA, "cannot select the handle's device");
    GB_TRY(check_sticky());
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const size_t img_bytes = (size_t)H * W * sizeof(float);
    const size_t out_bytes = (size_t)gabor_bank_output_elems(h, H, W) * 8;
    if (img_bytes > h->stage_img_bytes) {
        GB_CU(cudaStreamSynchronize(st));
        dfree(h->d_stage_img);
        h->stage_img_bytes = 0;
        GB_TRY(dalloc(&h->d_stage_img, (size_t)H * W));
        h->stage_img_bytes = img_bytes;
    }
    if (out_bytes > h->stage_out_bytes) {
        GB_CU(cudaStreamSynchronize(st));
        if (h->d_stage_out) cudaFree(h->d_stage_out);
        h->d_stage_out = nullptr;
        h->stage_out_bytes = 0;
        float2 *p = nullptr;
        GB_TRY(dalloc(&p, out_bytes / 8));
        h->d_stage_out = p;
        h->stage_out_bytes = out_bytes;
    }
    GB_CU(cudaMemcpy2DAsync(h->d_stage_img, (size_t)W * sizeof(float), h_img,
                            (size_t)pitch * sizeof(float), (size_t)W * sizeof(float), H,
                            cudaMemcpyHostToDevice, st));
    const int nf = (int)h->freqs.size();
    BankArgs probe{};
    int nprobe = 0;
    const bool chunked = nf > 1 && h->prec == GB_FP32 && h->smoother == GB_SMOOTHER_FIR &&
                         h->layout == GB_LAYOUT_PLANES && single_image_groups(h, H, W, probe, &nprobe);
    if (!chunked) {
        GB_TRY(filter_device(h, h->d_stage_img, H, W, W, h->d_stage_out, st));
        GB_CU(cudaMemcpyAsync(h_out, h->d_stage_out, out_bytes, cudaMemcpyDeviceToHost, st));
        GB_CU(cudaStreamSynchronize(st));
        return GB_OK;
    }
    // One launch per frequency, cheapest first; the planes of a finished frequency go back
    // to the host on a second stream (one copy per frequency) while the next ones compute.
    GB_TRY(ensure_tables(h, H, W, st));
    if (!h->copy_stream) GB_CU(cudaStreamCreateWithFlags(&h->copy_stream, cudaStreamNonBlocking));
    while ((int)h->freq_done.size() < nf + 1) {
        cudaEvent_t ev = nullptr;
        GB_CU(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
        h->freq_done.push_back(ev);
    }
    std::vector<int> order(nf);
    for (int s = 0; s < nf; ++s) order[s] = s;
    std::stable_sort(order.begin(), order.end(), [&](int p, int q) { return h->freqs[p].T < h->freqs[q].T; });
    const size_t freq_bytes = (size_t)h->theta.size() * H * W * sizeof(float2);
    // the copy stream must not overtake earlier work on `st` that reads or writes h_out
    GB_CU(cudaEventRecord(h->freq_done[nf], st));
    GB_CU(cudaStreamWaitEvent(h->copy_stream, h->freq_done[nf], 0));
    // every launch is queued before the first copy: a copy to pageable memory returns only
    // when it is done, and must not hold back the launches behind it
    for (int s : order) {
        GB_TRY(filter_device(h, h->d_stage_img, H, W, W, h->d_stage_out, st, s));
        GB_CU(cudaEventRecord(h->freq_done[s], st));
    }
    for (int s : order) {
        GB_CU(cudaStreamWaitEvent(h->copy_stream, h->freq_done[s], 0));
        GB_CU(cudaMemcpyAsync(static_cast<char *>(h_out) + s * freq_bytes,
                              reinterpret_cast<char *>(h->d_stage_out) + s * freq_bytes, freq_bytes,
                              cudaMemcpyDeviceToHost, h->copy_stream));
    }
    GB_CU(cudaStreamSynchronize(h->copy_stream));
    GB_CU(cudaStreamSynchronize(st));
    return GB_OK;
}

gb_status gabor_bank_sdft(gabor_bank_t h, const float *d_img, int H, int W, int64_t pitch,
                          double sigma, int My, int Mx, int half_spectrum, void *d_out,
                          void *stream)
{
    if (!h) return fail(GB_ERR_INVALID_ARG, "NULL handle");
    GB_TRY(validate_image(d_img, H, W, pitch, d_out));
    if (!std::isfinite(sigma) || sigma <= 0.0) return fail(GB_ERR_INVALID_ARG, "sigma must be positive");
    if (My < 2 || Mx < 2) return fail(GB_ERR_INVALID_ARG, "window sides must be >= 2");
    if ((My & 1) || (Mx & 1)) return fail(GB_ERR_UNSUPPORTED, "odd window sizes are not supported");
    if (My > kMaxSdftM || Mx > kMaxSdftM) return fail(GB_ERR_UNSUPPORTED, "window side above 64");
    if (half_spectrum != 0 && half_spectrum != 1) return fail(GB_ERR_INVALID_ARG, "half_spectrum must be 0 or 1");
    DeviceGuard g(h->device);
    if (!g.ok) return fail(GB_ERR_CUDA, "cannot select the handle's device");
    GB_TRY(check_sticky());
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    GB_TRY(ensure_sdft_tables(h, sigma, My, Mx, st));
    SdftArgs a{};
    a.img = d_img;
    a.pitch = pitch;
    a.H = H;
    a.W = W;
    a.out = reinterpret_cast<float2 *>(d_out);
    a.plane = (int64_t)H * W;
    a.Mx = Mx;
    a.My = My;
    a.half = half_spectrum;
    a.bmode = h->boundary;
    a.taps_x = h->d_sdft_taps;
    a.taps_y = h->d_sdft_taps + (kMaxSdftM + 8);
    a.tw_x = h->d_sdft_tw;
    a.tw_y = h->d_sdft_tw + kMaxSdftM;
    a.demod_form = h->sdft_form == 1 ? 1 : 0;
    a.noreuse = h->sdft_reuse ? 0 : 1;
    if (h->prec == GB_FP32) {
        // Filter order (Sec. III-B).  Vertical first (a transposed problem) saves FMAs when
        // My > Mx (the first FIR pass along the longer side), but its stores run across the
        // output rows; the kernel is bound by its stores, so the automatic order is
        // horizontal first and vertical first is taken only on request.
        const bool yfirst = !half_spectrum && h->sdft_order == 2;
        if (yfirst) {
            if ((size_t)H * W > h->transp_elems) {
                GB_CU(cudaStreamSynchronize(st));   // earlier work of this handle may still read it
                dfree(h->d_transp);
                h->transp_elems = 0;
                GB_TRY(dalloc(&h->d_transp, (size_t)H * W));
                h->transp_elems = (size_t)H * W;
            }
            GB_CU(launch_transpose(d_img, pitch, H, W, h->d_transp, st));
            SdftArgs t = a;
            t.img = h->d_transp;
            t.pitch = H;
            t.H = W;
            t.W = H;
            t.Mx = My;
            t.My = Mx;
            t.taps_x = a.taps_y;
            t.taps_y = a.taps_x;
            t.tw_x = a.tw_y;
            t.tw_y = a.tw_x;
            t.trans = 1;
            GB_CU(launch_sdft_fp32(t, h->sm_count, st));
            return GB_OK;
        }
        GB_CU(launch_sdft_fp32(a, h->sm_count, st));
        return GB_OK;
    }
    if (!sdft_tc_supported(Mx, My))
        return fail(GB_ERR_UNSUPPORTED, "tensor-core SDFT: the window's operands do not fit in shared memory "
                                        "(Mx * My <= 256 and (My / 2 + 1) * Mx bins within the limit)");
    const int bf16 = h->prec == GB_BF16_TC;
    if (h->sdftB_sigma != sigma || h->sdftB_Mx != Mx || h->sdftB_My != My) {
        const size_t bytes = (size_t)sdft_tc_b_bytes(Mx, My);
        if (bytes > h->sdft_B_bytes) {
            GB_CU(cudaStreamSynchronize(st));
            if (h->d_sdft_B) cudaFree(h->d_sdft_B);
            h->d_sdft_B = nullptr;
            h->sdft_B_bytes = 0;
            uint4 *p = nullptr;
            GB_TRY(dalloc(&p, bytes / 16));
            h->d_sdft_B = p;
            h->sdft_B_bytes = bytes;
        }
        GB_CU(build_sdft_tc_b(h->d_sdft_B, sigma, Mx, My, bf16, &h->sdft_B_unscale, st));
        h->sdftB_sigma = sigma;
        h->sdftB_Mx = Mx;
        h->sdftB_My = My;
    }
    const size_t ws_bytes = (size_t)sdft_tc_ws_bytes(H, W, Mx, My);
    if (ws_bytes > h->sdft_ws_bytes) {
        GB_CU(cudaStreamSynchronize(st));   // earlier work of this handle may still read it
        if (h->d_sdft_ws) cudaFree(h->d_sdft_ws);
        h->d_sdft_ws = nullptr;
        h->sdft_ws_bytes = 0;
        uint4 *p = nullptr;
        GB_TRY(dalloc(&p, (ws_bytes + 15) / 16));
        h->d_sdft_ws = p;
        h->sdft_ws_bytes = ws_bytes;
    }
    GB_CU(launch_sdft_tc(d_img, pitch, H, W, reinterpret_cast<float2 *>(d_out), Mx, My, half_spectrum,
                         h->d_sdft_B, h->sdft_B_unscale, bf16, h->boundary, h->d_status, h->sm_count,
                         ws_bytes ? h->d_sdft_ws : nullptr, st));
    return GB_OK;
}

gb_status gabor_bank_filter_batch(gabor_bank_t h, int n, const float *const *d_imgs,
                                  const int *H, const int *W, const int64_t *pitch,
                                  void *const *d_outs, void *stream)
{
    if (!h) return fail(GB_ERR_INVALID_ARG, "NULL handle");
    if (n < 0 || (n > 0 && (!d_imgs || !H || !W || !pitch || !d_outs)))
        return fail(GB_ERR_INVALID_ARG, "bad batch arrays");
    for (int i = 0; i < n; ++i) GB_TRY(validate_image(d_imgs[i], H[i], W[i], pitch[i], d_outs[i]));
    if (h->units.empty()) return fail(GB_ERR_INVALID_ARG, "handle has no filter bank (SDFT-only)");
    DeviceGuard g(h->device);
    if (!g.ok) return fail(GB_ERR_CUDA, "cannot select the handle's device");
    GB_TRY(check_sticky());
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (n == 0) return GB_OK;
    if (h->prec != GB_FP32 && h->smoother == GB_SMOOTHER_FIR) {
        // tensor-core handles: the whole batch in four launches (modulated-tap kernels), else
        // one bank pass per image
        bool done = false;
        GB_TRY(filter_batch_tc(h, n, d_imgs, H, W, pitch, d_outs, st, &done));
        if (done) return GB_OK;
    }
    if (h->prec != GB_FP32 || h->smoother == GB_SMOOTHER_IIR) {
        // the recursive smoother, and tensor-core plans that need the step-by-step kernels: one
        // bank pass per image
        for (int i = 0; i < n; ++i) GB_TRY(filter_device(h, d_imgs[i], H[i], W[i], pitch[i], d_outs[i], st));
        return GB_OK;
    }
    int Hm = 0, Wm = 0;
    for (int i = 0; i < n; ++i) {
        Hm = std::max(Hm, H[i]);
        Wm = std::max(Wm, W[i]);
    }
    GB_TRY(ensure_tables(h, Hm, Wm, st));
    // One launch over every image: upload the image descriptors, then the shared work list.
    if (n > h->imgs_cap) {
        GB_CU(cudaStreamSynchronize(st));
        dfree(h->d_imgs);
        h->imgs_cap = 0;
        GB_TRY(dalloc(&h->d_imgs, (size_t)n));
        h->imgs_cap = n;
        h->last_imgs.clear();
    }
    std::vector<ImageDev> imgs(n);
    std::vector<int64_t> shapes(2 * (size_t)n);
    for (int i = 0; i < n; ++i) {
        imgs[i] = ImageDev{d_imgs[i], pitch[i], reinterpret_cast<float2 *>(d_outs[i]), H[i], W[i]};
        shapes[2 * i] = H[i];
        shapes[2 * i + 1] = W[i];
    }
    // Upload the descriptors only when they changed since the last batch call, so that a
    // repeated call (for example under CUDA graph capture) issues no host-to-device copy.
    bool same = h->last_imgs.size() == (size_t)n;
    for (int i = 0; same && i < n; ++i)
        same = std::memcmp(&h->last_imgs[i], &imgs[i], sizeof(ImageDev)) == 0;
    if (!same) {
        // Pageable source: the copy is complete (staged) when the call returns.
        GB_CU(cudaMemcpyAsync(h->d_imgs, imgs.data(), n * sizeof(ImageDev), cudaMemcpyHostToDevice, st));
        h->last_imgs = imgs;
    }
    WorkItem *items = nullptr;
    int nitems = 0;
    GB_TRY(get_worklist(h, shapes, &items, &nitems));
    BankArgs a{};
    a.imgs = h->d_imgs;
    a.freqs = h->d_freqdev;
    a.units = h->d_unitdev;
    a.items = items;
    a.counter = h->d_counter;
    a.bmode = h->boundary;
    a.layout = h->layout;
    a.nplanes = (int)(h->omega.size() * h->theta.size());
    a.status = h->d_status;
    a.pipelined = h->fp32_pipelined ? 1 : 0;
    a.mtaps = h->fp32_row_form != 1 ? 1 : 0;
    a.ctas = h->fp32_ctas;
    GB_CU(launch_gabor_fp32(a, nitems, h->max_smem, h->sm_count, st));
    return GB_OK;
}

gb_status gabor_bank_set_option(gabor_bank_t h, int key, int64_t value)
{
    if (!h) return fail(GB_ERR_INVALID_ARG, "NULL handle");
    switch (key) {
    case GB_OPT_REUSE:
        if (value != 0 && value != 1) return fail(GB_ERR_INVALID_ARG, "GB_OPT_REUSE takes 0 or 1");
        if (h->reuse != (int)value) {
            DeviceGuard g(h->device);
            cudaDeviceSynchronize();
            h->reuse = (int)value;
            free_tables(h);
            free_tc(h);
            build_plan(h);
        }
        return GB_OK;
    case GB_OPT_TILE_ROWS:
        if (value != 0 && value != 8 && value != 16 && value != 32 && value != 64)
            return fail(GB_ERR_INVALID_ARG, "GB_OPT_TILE_ROWS takes 0, 8, 16, 32 or 64");
        if (h->tile_rows != (int)value) {
            DeviceGuard g(h->device);
            cudaDeviceSynchronize();
            h->tile_rows = (int)value;
            free_tables(h);
        }
        return GB_OK;
    case GB_OPT_PIPELINE:
        if (value < 0 || value > 2) return fail(GB_ERR_INVALID_ARG, "GB_OPT_PIPELINE takes 0, 1 or 2");
        if (h->fp32_pipeline != (int)value) {
            DeviceGuard g(h->device);
            cudaDeviceSynchronize();
            h->fp32_pipeline = (int)value;
            free_tables(h);
        }
        return GB_OK;
    case GB_OPT_ROW_PASS:
        if (value < 0 || value > 2) return fail(GB_ERR_INVALID_ARG, "GB_OPT_ROW_PASS takes 0, 1 or 2");
        if (h->fp32_row_form != (int)value) {
            DeviceGuard g(h->device);
            cudaDeviceSynchronize();
            h->fp32_row_form = (int)value;
            free_tables(h);
        }
        return GB_OK;
    case GB_OPT_BANK_CTAS:
        if (value < 0 || value > 2) return fail(GB_ERR_INVALID_ARG, "GB_OPT_BANK_CTAS takes 0, 1 or 2");
        if (h->fp32_ctas_opt != (int)value) {
            DeviceGuard g(h->device);
            cudaDeviceSynchronize();
            h->fp32_ctas_opt = (int)value;
            free_tables(h);
        }
        return GB_OK;
    case GB_OPT_SDFT_FORM:
        if (value < 0 || value > 2) return fail(GB_ERR_INVALID_ARG, "GB_OPT_SDFT_FORM takes 0, 1 or 2");
        h->sdft_form = (int)value;
        return GB_OK;
    case GB_OPT_TC_TILES: {
        const int r = (int)(value & 255), c = (int)(value >> 8);
        if (value < 0 || (r != 0 && r != 32 && r != 64) || (c != 0 && c != 32 && c != 64))
            return fail(GB_ERR_INVALID_ARG, "GB_OPT_TC_TILES takes row + 256 * column, each 0, 32 or 64");
        if (r != h->tc_row_ty_opt || c != h->tc_col_ty_opt) {
            DeviceGuard g(h->device);
            cudaDeviceSynchronize();
            h->tc_row_ty_opt = r;
            h->tc_col_ty_opt = c;
            free_tc(h);   // the column operand strips depend on the job rows
        }
        return GB_OK;
    }
    case GB_OPT_SDFT_REUSE:
        if (value != 0 && value != 1) return fail(GB_ERR_INVALID_ARG, "GB_OPT_SDFT_REUSE takes 0 or 1");
        h->sdft_reuse = (int)value;
        return GB_OK;
    case GB_OPT_BOUNDARY:
        if (value < GB_BOUNDARY_ZERO || value > GB_BOUNDARY_MIRROR)
            return fail(GB_ERR_INVALID_ARG, "GB_OPT_BOUNDARY takes GB_BOUNDARY_ZERO, _REPLICATE or _MIRROR");
        h->boundary = (int)value;
        h->tc_H = h->tc_W = 0;   // the tensor-core intermediate's halo rows change meaning
        return GB_OK;
    case GB_OPT_SDFT_ORDER:
        if (value < 0 || value > 2) return fail(GB_ERR_INVALID_ARG, "GB_OPT_SDFT_ORDER takes 0, 1 or 2");
        h->sdft_order = (int)value;
        return GB_OK;
    case GB_OPT_SMOOTHER:
        if (value != GB_SMOOTHER_FIR && value != GB_SMOOTHER_IIR)
            return fail(GB_ERR_INVALID_ARG, "GB_OPT_SMOOTHER takes GB_SMOOTHER_FIR or GB_SMOOTHER_IIR");
        h->smoother = (int)value;
        return GB_OK;
    case GB_OPT_LAYOUT:
        if (value != GB_LAYOUT_PLANES && value != GB_LAYOUT_PIXELS)
            return fail(GB_ERR_INVALID_ARG, "GB_OPT_LAYOUT takes GB_LAYOUT_PLANES or GB_LAYOUT_PIXELS");
        h->layout = (int)value;
        return GB_OK;
    case GB_OPT_SEGMENTS:
        if (value < 0 || value > 64) return fail(GB_ERR_INVALID_ARG, "GB_OPT_SEGMENTS takes 0 .. 64");
        if (h->segments != (int)value) {
            DeviceGuard g(h->device);
            cudaDeviceSynchronize();
            h->segments = (int)value;
            for (auto &kv : h->worklists) cudaFree(kv.second.first);
            h->worklists.clear();
        }
        return GB_OK;
    default:
        return fail(GB_ERR_INVALID_ARG, "unknown option");
    }
}

gb_status gabor_bank_set_tiling(gabor_bank_t h, int s, int tile_rows, int segments)
{
    if (!h) return fail(GB_ERR_INVALID_ARG, "NULL handle");
    const int nf = (int)h->freqs.size();
    if (s < -1 || s >= nf) return fail(GB_ERR_INVALID_ARG, "frequency index out of range");
    if (tile_rows != 0 && tile_rows != 8 && tile_rows != 16 && tile_rows != 32 && tile_rows != 64)
        return fail(GB_ERR_INVALID_ARG, "tile_rows takes 0, 8, 16, 32 or 64");
    if (segments < 0 || segments > 64) return fail(GB_ERR_INVALID_ARG, "segments takes 0 .. 64");
    DeviceGuard g(h->device);
    cudaDeviceSynchronize();
    h->ftile_rows.resize(nf, 0);
    h->fsegments.resize(nf, 0);
    for (int i = 0; i < nf; ++i) {
        if (s != -1 && i != s) continue;
        h->ftile_rows[i] = tile_rows;
        h->fsegments[i] = segments;
    }
    free_tables(h);   // tile geometry and work lists are rebuilt on the next call
    return GB_OK;
}

gb_status gabor_bank_device_status(gabor_bank_t h, void *stream)
{
    if (!h) return fail(GB_ERR_INVALID_ARG, "NULL handle");
    DeviceGuard g(h->device);
    GB_CU(cudaStreamSynchronize(static_cast<cudaStream_t>(stream)));
    int v = 0;
    GB_CU(cudaMemcpy(&v, h->d_status, sizeof(int), cudaMemcpyDeviceToHost));
    GB_CU(cudaMemset(h->d_status, 0, sizeof(int)));
    if (v == 60)
        return fail(GB_ERR_UNSUPPORTED, "an image's centre level |c| exceeds the FP16 tensor-core bank's range "
                                        "(|c| 2^sB >= 2^29, sB the column operand's scale exponent); use GB_BF16_TC");
    if (v != 0) return fail(GB_ERR_TIMEOUT, "a bounded device wait gave up (code " + std::to_string(v) + ")");
    return GB_OK;
}

gb_status gabor_fp32_fma_probe(void *d_out, int blocks, int iters, int packed, void *stream)
{
    if (!d_out || blocks <= 0 || iters <= 0 || (packed != 0 && packed != 1))
        return fail(GB_ERR_INVALID_ARG, "bad probe arguments");
    GB_TRY(check_sticky());
    GB_CU(launch_fma_peak(static_cast<float *>(d_out), blocks, iters, packed, static_cast<cudaStream_t>(stream)));
    return GB_OK;
}

gb_status gabor_store_probe(void *d_out, int64_t nplanes, int H, int W, int ctas, void *stream)
{
    if (!d_out || nplanes <= 0 || H <= 0 || W <= 0 || W % 128 != 0 || ctas <= 0)
        return fail(GB_ERR_INVALID_ARG, "bad probe arguments (W must be a positive multiple of 128)");
    if ((int64_t)H * W > (int64_t)1 << 40 || nplanes > ((int64_t)1 << 40) / ((int64_t)H * W))
        return fail(GB_ERR_INVALID_ARG, "probe output too large");
    GB_TRY(check_sticky());
    GB_CU(launch_store_pattern(static_cast<float2 *>(d_out), nplanes, H, W, ctas, static_cast<cudaStream_t>(stream)));
    return GB_OK;
}

gb_status gabor_bank_selftest_wait(gabor_bank_t h, int signal, double limit_ms, void *stream)
{
    if (!h) return fail(GB_ERR_INVALID_ARG, "NULL handle");
    if (signal != 0 && signal != 1) return fail(GB_ERR_INVALID_ARG, "signal must be 0 or 1");
    if (!(limit_ms > 0.0 && limit_ms <= 2000.0)) return fail(GB_ERR_INVALID_ARG, "limit_ms must be in (0, 2000]");
    DeviceGuard g(h->device);
    if (!g.ok) return fail(GB_ERR_CUDA, "cannot select the handle's device");
    GB_TRY(check_sticky());
    GB_CU(launch_wait_selftest(h->d_status, signal, (unsigned long long)(limit_ms * 1e6),
                               static_cast<cudaStream_t>(stream)));
    return GB_OK;
}

int64_t gabor_bank_workspace_bytes(gabor_bank_t h, int H, int W)
{
    if (!h || H <= 0 || W <= 0) return 0;
    if (h->prec == GB_FP32 || h->units.empty()) return 0;
    return tc_ws_bytes(h, H, W);
}

gb_status gabor_bank_set_workspace(gabor_bank_t h, void *d_ws, int64_t bytes)
{
    if (!h) return fail(GB_ERR_INVALID_ARG, "NULL handle");
    if (d_ws == nullptr) {
        if (bytes != 0) return fail(GB_ERR_INVALID_ARG, "NULL workspace with a non-zero size");
    } else {
        if (bytes <= 0) return fail(GB_ERR_INVALID_ARG, "workspace size must be positive");
        if (reinterpret_cast<uintptr_t>(d_ws) % 16) return fail(GB_ERR_INVALID_ARG, "workspace not 16-byte aligned");
    }
    h->ws_ptr = static_cast<uint16_t *>(d_ws);
    h->ws_bytes = d_ws ? (size_t)bytes : 0;
    h->tc_H = h->tc_W = 0;
    return GB_OK;
}

int64_t gabor_bank_output_elems(gabor_bank_t h, int H, int W)
{
    if (!h || H <= 0 || W <= 0) return 0;
    return (int64_t)h->omega.size() * (int64_t)h->theta.size() * H * W;
}

const char *gabor_bank_last_error(void) { return g_err.c_str(); }

const char *gabor_bank_version(void) { return "gaborbank 0.1 (sm_103a)"; }

}  // extern "C"
