// gabor_sdft_noalloc: the FP32 localized sliding DFT for callers that cannot allocate device
// memory, such as code running inside a memory pool or allocator that forbids cudaMalloc, or
// an application that fixes its device-memory budget before it starts.
//
// The FP32 SDFT kernel reads small tables (Gaussian taps and twiddles of both window axes).
// Here they live in one file-scope __device__ array, g_noalloc_scratch, instead of in memory
// owned by a gabor_bank handle, and the entry point needs no handle.  The array is kNoallocBytes
// (2 KiB) on every GPU that loads the library, for the life of the process.  Each call
// rewrites the whole table with one small kernel before the SDFT kernel runs (two launches per
// call, no host-to-device copy); calls that overlap on the GPU (for example on two streams)
// race on it.
#include <atomic>
#include <cmath>
#include <mutex>

#include "internal.h"

namespace gb {

namespace {

constexpr int kNoallocMaxDevices = 64;
constexpr int kNoallocTap = kMaxSdftM + 8;   // taps per axis (zero-padded)
constexpr size_t kNoallocBytes = 2048;

// Layout: taps_x, taps_y (kNoallocTap floats each), then the twiddles of x and y (kMaxSdftM
// float2 each).  Every call writes all of it from by-value parameters.
constexpr size_t kOffTaps = 0;
constexpr size_t kOffTw = kOffTaps + 2 * kNoallocTap * sizeof(float);        // 576
static_assert(kOffTw + 2 * kMaxSdftM * sizeof(float2) <= kNoallocBytes, "scratch too small");

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocBytes];

struct DeviceSetup {
    unsigned char *scratch = nullptr;   // device address of g_noalloc_scratch
    int sm_count = 0;
};

DeviceSetup g_setup[kNoallocMaxDevices];
std::atomic<bool> g_ready[kNoallocMaxDevices];
std::mutex g_setup_mutex;

// Once per device, with that device current: the device address of the scratch array (the
// host-side name is only a stand-in) and the kernel attributes.  The first call on a device
// takes a process-wide mutex; later calls read the recorded set-up without locking.
gb_status setup_device(int dev, DeviceSetup *out)
{
    if (!g_ready[dev].load(std::memory_order_acquire)) {
        std::lock_guard<std::mutex> lock(g_setup_mutex);
        if (!g_ready[dev].load(std::memory_order_relaxed)) {
            DeviceSetup d;
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
            g_setup[dev] = d;
            g_ready[dev].store(true, std::memory_order_release);
        }
    }
    *out = g_setup[dev];
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
    // the same argument checks, in the same order and with the same messages, as gabor_bank_sdft
    gb_status s = validate_image(d_img, H, W, pitch, d_out);
    if (s != GB_OK) return s;
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
    s = check_sticky();
    if (s != GB_OK) return s;
    DeviceSetup d;
    s = setup_device(dev, &d);
    if (s != GB_OK) return s;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    float *taps = reinterpret_cast<float *>(d.scratch + kOffTaps);
    float2 *tw = reinterpret_cast<float2 *>(d.scratch + kOffTw);
    // One small kernel rewrites the whole table (1600 bytes) from by-value parameters: no host
    // copy, nothing left over from an earlier call with another window.
    e = launch_build_sdft_tables(sigma, Mx, My, kNoallocTap, kMaxSdftM, taps, tw, st);
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
