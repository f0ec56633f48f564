// gabor_sdft_noalloc: the FP32 localized sliding DFT for callers that cannot allocate device
// memory, such as code running inside a memory pool or allocator that forbids cudaMalloc, or
// an application that fixes its device-memory budget before it starts.
//
// The FP32 SDFT kernel reads small tables (Gaussian taps and twiddles of both window axes).
// Here they live in one file-scope __device__ array, g_noalloc_scratch, instead of in memory
// owned by a gabor_bank handle, and the entry point needs no handle.  The array is kNoallocBytes
// (2 KiB) on every GPU that loads the library, for the life of the process.  Each call
// rewrites the whole table before its kernel runs; calls that overlap on the GPU (for example
// on two streams) race on it.
#include <cmath>
#include <mutex>

#include "internal.h"

namespace gb {

namespace {

constexpr int kNoallocMaxDevices = 64;
constexpr int kNoallocTap = kMaxSdftM + 8;   // taps per axis (zero-padded)
constexpr size_t kNoallocBytes = 2048;

// Layout: taps_x, taps_y (kNoallocTap floats each), twiddles x, y (kMaxSdftM float2 each),
// sigma x, y (double), lo x, y and T x, y (int).
constexpr size_t kOffTaps = 0;
constexpr size_t kOffTw = kOffTaps + 2 * kNoallocTap * sizeof(float);        // 576
constexpr size_t kOffSigma = kOffTw + 2 * kMaxSdftM * sizeof(float2);        // 1600
constexpr size_t kOffInts = kOffSigma + 2 * sizeof(double);                  // 1616
static_assert(kOffInts + 4 * sizeof(int) <= kNoallocBytes, "scratch too small");

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocBytes];

struct DeviceSetup {
    unsigned char *scratch = nullptr;   // device address of g_noalloc_scratch
    int sm_count = 0;
    bool ready = false;
};

DeviceSetup g_setup[kNoallocMaxDevices];
std::mutex g_setup_mutex;

// Once per device, with that device current: the device address of the scratch array (the
// host-side name is only a stand-in) and the kernel attributes.
gb_status setup_device(int dev, DeviceSetup *out)
{
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    DeviceSetup &d = g_setup[dev];
    if (!d.ready) {
        void *ptr = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&d.sm_count, cudaDevAttrMultiProcessorCount, dev);
        if (e == cudaSuccess) e = sdft_fp32_prepare();
        if (e != cudaSuccess) {
            cudaGetLastError();
            set_last_error((std::string("gabor_sdft_noalloc set-up: ") + cudaGetErrorString(e)).c_str());
            return GB_ERR_CUDA;
        }
        d.scratch = static_cast<unsigned char *>(ptr);
        d.ready = true;
    }
    *out = d;
    return GB_OK;
}

gb_status fail_arg(gb_status s, const char *msg)
{
    set_last_error(msg);
    return s;
}

}  // namespace

}  // namespace gb

using namespace gb;

extern "C" gb_status gabor_sdft_noalloc(const float *d_img, int H, int W, int64_t pitch, double sigma,
                                         int My, int Mx, int half_spectrum, void *d_out, void *stream)
{
    if (!d_img || !d_out) return fail_arg(GB_ERR_INVALID_ARG, "NULL image or output pointer");
    if (H <= 0 || W <= 0) return fail_arg(GB_ERR_INVALID_ARG, "H and W must be positive");
    if (pitch < W) return fail_arg(GB_ERR_INVALID_ARG, "pitch must be >= W");
    if (reinterpret_cast<uintptr_t>(d_img) % 4) return fail_arg(GB_ERR_INVALID_ARG, "image not 4-byte aligned");
    if (reinterpret_cast<uintptr_t>(d_out) % 8) return fail_arg(GB_ERR_INVALID_ARG, "output not 8-byte aligned");
    if (!std::isfinite(sigma) || sigma <= 0.0) return fail_arg(GB_ERR_INVALID_ARG, "sigma must be positive");
    if (My < 2 || Mx < 2) return fail_arg(GB_ERR_INVALID_ARG, "window sides must be >= 2");
    if ((My & 1) || (Mx & 1)) return fail_arg(GB_ERR_UNSUPPORTED, "odd window sizes are not supported");
    if (My > kMaxSdftM || Mx > kMaxSdftM)
        return fail_arg(GB_ERR_UNSUPPORTED, "window side above 64: beyond the fixed scratch table of gabor_sdft_noalloc");
    if (half_spectrum != 0 && half_spectrum != 1) return fail_arg(GB_ERR_INVALID_ARG, "half_spectrum must be 0 or 1");
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess || dev < 0 || dev >= kNoallocMaxDevices) {
        cudaGetLastError();
        return fail_arg(GB_ERR_CUDA, "gabor_sdft_noalloc: no usable current device");
    }
    DeviceSetup d;
    gb_status s = setup_device(dev, &d);
    if (s != GB_OK) return s;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    float *taps = reinterpret_cast<float *>(d.scratch + kOffTaps);
    float2 *tw = reinterpret_cast<float2 *>(d.scratch + kOffTw);
    double *d_sigma = reinterpret_cast<double *>(d.scratch + kOffSigma);
    int *d_ints = reinterpret_cast<int *>(d.scratch + kOffInts);
    // Parameters of this call (pageable source: staged before the call returns).
    const double sg[2] = {sigma, sigma};
    const int ints[4] = {Mx / 2, My / 2, Mx, My};   // lo x, lo y, T x, T y
    e = cudaMemcpyAsync(d_sigma, sg, sizeof(sg), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_ints, ints, sizeof(ints), cudaMemcpyHostToDevice, st);
    // Every table entry is rewritten: taps beyond T are written as zeros.
    if (e == cudaSuccess) e = launch_build_taps(d_sigma, d_ints, d_ints + 2, 2, kNoallocTap, taps, st);
    if (e == cudaSuccess) e = launch_build_twiddles(Mx, tw, st);
    if (e == cudaSuccess) e = launch_build_twiddles(My, tw + kMaxSdftM, st);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail_arg(GB_ERR_CUDA, "gabor_sdft_noalloc: table build failed");
    }
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
    a.taps_x = taps;
    a.taps_y = taps + kNoallocTap;
    a.tw_x = tw;
    a.tw_y = tw + kMaxSdftM;
    e = launch_sdft_fp32(a, d.sm_count, st);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail_arg(GB_ERR_CUDA, "gabor_sdft_noalloc: kernel launch failed");
    }
    return GB_OK;
}
