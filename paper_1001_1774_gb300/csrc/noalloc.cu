// tvcs_apply_noalloc: the fused products r = A x - y, g = A^T r for callers
// that cannot allocate device memory.
//
// Some applications may not call cudaMalloc at the point where they need the
// products: for example programs that reserve all device memory in their own
// pool at start-up, programs running under a hard device-memory cap, or
// latency-critical loops where the implicit synchronisation of a device
// allocation is not acceptable.  The regular entry points allocate their work
// buffers at tvcs_create; this one allocates nothing.  Its only work memory
// is the file-scope array below, of a fixed maximum size, which every GPU that
// loads this library holds until the process exits.
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <mutex>

#include "common.cuh"
#include "kernels.h"
#include "tvcs.h"

namespace tvcs {
// Defined in tvcs_api.cu: sets the calling thread's last-error message.
tvcs_status set_last_error(tvcs_status s, const char* fmt, ...);
}

using namespace tvcs;

namespace {

constexpr size_t kScratchBytes = 12u << 20;   // 12 MiB per device
constexpr int kMaxDevices = 64;

// Work memory of tvcs_apply_noalloc: per-block partial sums of A^T r, per-block
// double-single partials of ||r||^2 and a control block for the last-block ticket.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

std::mutex g_setup_mutex;
void* g_scratch_ptr[kMaxDevices] = {};
int g_num_sms[kMaxDevices] = {};

size_t round256(size_t b) { return (b + 255) & ~(size_t)255; }

// One-time set-up on the current device: device address of the scratch
// array (host code may not use the array's name as a device address) and the
// shared-memory limit of every product kernel shape.
tvcs_status setup_device(int dev)
{
    std::lock_guard<std::mutex> lk(g_setup_mutex);
    if (g_scratch_ptr[dev]) return TVCS_OK;
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p)
        return set_last_error(TVCS_ERR_CUDA, "cudaGetSymbolAddress of the scratch array: %s",
                              cudaGetErrorString(e));
    int sms = 0;
    e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess)
        return set_last_error(TVCS_ERR_CUDA, "cudaDeviceGetAttribute: %s", cudaGetErrorString(e));
    for (int n : {16, 32, 48, 64, 96, 128}) {
        if (!prod_supported(n)) continue;
        e = prod_configure(n);
        if (e != cudaSuccess)
            return set_last_error(TVCS_ERR_CUDA, "configuring the product kernel: %s",
                                  cudaGetErrorString(e));
    }
    g_num_sms[dev] = sms;
    g_scratch_ptr[dev] = p;
    return TVCS_OK;
}

// True when p is device memory of device `dev` or managed memory (which any
// device may access).  Device memory of another GPU is rejected: the kernels run
// on `dev`, and without peer access a load from another GPU's memory faults.
bool is_device_pointer_on(const void* p, int dev)
{
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    if (at.type == cudaMemoryTypeManaged) return true;
    return at.type == cudaMemoryTypeDevice && at.device == dev;
}

}  // namespace

extern "C" tvcs_status tvcs_apply_noalloc(const float* A, int m, int n, const float* x,
                                          const float* y, float* r, float* g, void* stream)
{
    if (!A || !x || !r || !g)
        return set_last_error(TVCS_ERR_INVALID_ARG, "A, x, r and g must be non-NULL");
    if (m < 1 || m > (1 << 24))
        return set_last_error(TVCS_ERR_INVALID_ARG, "m = %d outside [1, 2^24]", m);
    if (!prod_supported(n))
        return set_last_error(TVCS_ERR_INVALID_ARG,
                              "n = %d not supported (16, 32, 48, 64, 96, 128)", n);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    // The call reads an error word back to the host and synchronises the stream,
    // neither of which a stream capture can record: reject a capturing stream
    // (or a legacy-stream call while another capture forbids it) before any work.
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    cudaError_t e = cudaStreamIsCapturing(s, &cap);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return set_last_error(TVCS_ERR_INVALID_ARG,
                              "tvcs_apply_noalloc cannot run while a stream capture is active "
                              "(cudaStreamIsCapturing: %s)", cudaGetErrorString(e));
    }
    if (cap != cudaStreamCaptureStatusNone)
        return set_last_error(TVCS_ERR_INVALID_ARG,
                              "tvcs_apply_noalloc cannot be captured into a CUDA graph "
                              "(the stream is capturing)");
    int dev = 0;
    e = cudaGetDevice(&dev);
    if (e != cudaSuccess || dev < 0 || dev >= kMaxDevices)
        return set_last_error(TVCS_ERR_CUDA, "cudaGetDevice: %s", cudaGetErrorString(e));
    if (!is_device_pointer_on(A, dev) || !is_device_pointer_on(x, dev) ||
        !is_device_pointer_on(r, dev) || !is_device_pointer_on(g, dev) ||
        (y && !is_device_pointer_on(y, dev)))
        return set_last_error(TVCS_ERR_INVALID_ARG,
                              "all arrays must be device memory of the current device (%d)", dev);
    tvcs_status st = setup_device(dev);
    if (st != TVCS_OK) return st;

    const int N = n * n;
    const int P = prod_grid(n, m, g_num_sms[dev]);
    const size_t b_gpart = round256((size_t)P * N * sizeof(float));
    const size_t b_r2 = round256((size_t)P * sizeof(float2));
    const size_t b_ctrl = round256(sizeof(Ctrl));
    if (b_gpart + b_r2 + b_ctrl > kScratchBytes)
        return set_last_error(TVCS_ERR_INVALID_ARG,
                              "m = %d, n = %d need %zu bytes of scratch; the no-allocation "
                              "limit is %zu bytes",
                              m, n, b_gpart + b_r2 + b_ctrl, kScratchBytes);
    unsigned char* base = static_cast<unsigned char*>(g_scratch_ptr[dev]);
    float* gpart = reinterpret_cast<float*>(base);
    float2* r2part = reinterpret_cast<float2*>(base + b_gpart);
    Ctrl* ctrl = reinterpret_cast<Ctrl*>(base + b_gpart + b_r2);

    // The array keeps the previous call's contents: the control block (tickets,
    // error word) must start at zero; the partials are fully overwritten.
    e = cudaMemsetAsync(ctrl, 0, sizeof(Ctrl), s);
    if (e != cudaSuccess)
        return set_last_error(TVCS_ERR_CUDA, "cudaMemsetAsync: %s", cudaGetErrorString(e));
    ProdArgs a{};
    a.A = A;
    a.m = m;
    a.x = x;
    a.y = y;
    a.r = r;
    a.gpart = gpart;
    a.r2part = r2part;
    a.ctrl = ctrl;
    a.mode = MODE_PLAIN;
    a.budget = 1LL << 31;
    // Launch failures are this call's own: each launcher returns its launch status.
    e = launch_products(n, P, a, s);
    if (e == cudaSuccess) e = launch_greduce(gpart, P, N, g, ctrl, MODE_PLAIN, s);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return set_last_error(TVCS_ERR_CUDA, "tvcs_apply_noalloc: launch failed: %s",
                              cudaGetErrorString(e));
    }
    int err_word = 0;
    e = cudaMemcpyAsync(&err_word, &ctrl->error, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess)
        return set_last_error(TVCS_ERR_CUDA, "tvcs_apply_noalloc: %s", cudaGetErrorString(e));
    if (err_word == ERR_TIMEOUT)
        return set_last_error(TVCS_ERR_TIMEOUT, "a bounded device wait gave up");
    return TVCS_OK;
}
