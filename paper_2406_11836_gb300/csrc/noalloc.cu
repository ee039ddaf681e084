// Forward render for callers that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc (or any allocating routine) around a render: a
// real-time thread that must not block on the allocator (cudaMalloc can take a lock and
// wait for the device), or a host program that hands all device memory out from its own
// pool and so has none left to give a render.  rgs_render_fwd_noalloc serves them: it
// does the same work as rgs_render_fwd but takes its workspace from a fixed array in
// this file instead of from the caller, and allocates nothing itself.  Like
// rgs_render_fwd it synchronises its stream once, after the projection, to size the
// instance buffers.
//
// The array (kScratchBytes) is a file-scope __device__ variable: every GPU that loads the
// library holds it until the process exits.  In host code its name is only a host-side
// stand-in, so the device address is looked up once per device with
// cudaGetSymbolAddress, by the first call on that device (with the device current); make
// that first call before any stream capture.  All calls share the array and it keeps the
// previous call's contents: the render clears what has to start at zero (counters, tile
// ranges) itself, and calls that overlap on the GPU (several streams, several host
// threads) race on the array — serialise them.
#include <cstdio>
#include <mutex>

#include "rgs_internal.cuh"

namespace {

constexpr size_t kScratchBytes = size_t(64) << 20;   // 64 MiB
constexpr int kMaxDevices = 64;

__device__ __align__(256) unsigned char g_scratch[kScratchBytes];

std::mutex g_mu;
void* g_scratch_ptr[kMaxDevices] = {};

}  // namespace

extern "C" int rgs_render_fwd_noalloc(const rgs_kd* kd, const rgs_gaussians* g, const rgs_camera* cam,
                                      const rgs_render_opts* opts, float* partial_C, float* partial_T, float* image,
                                      float* T_final, float* tile_depth, void* stream) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) {
        rgs::set_error("render_fwd_noalloc: cudaGetDevice: %s", cudaGetErrorString(e));
        return RGS_ECUDA;
    }
    if (dev < 0 || dev >= kMaxDevices) {
        rgs::set_error("render_fwd_noalloc: device %d beyond the %d supported", dev, kMaxDevices);
        return RGS_EINVAL;
    }
    void* scratch = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_mu);
        if (!g_scratch_ptr[dev]) {
            e = cudaGetSymbolAddress(&scratch, g_scratch);
            if (e != cudaSuccess) {
                rgs::set_error("render_fwd_noalloc: cudaGetSymbolAddress: %s", cudaGetErrorString(e));
                return RGS_ECUDA;
            }
            g_scratch_ptr[dev] = scratch;
        }
        scratch = g_scratch_ptr[dev];
    }
    unsigned long long counts[2] = {0, 0};   // host copy of the instance counts (no pinned buffer)
    rgs::set_required_workspace(0);          // set again only when the scratch is what was too small
    rgs::prof_suppress(true);                // tracing would create CUDA events
    const int rc = rgs::render_fwd_into(kd, g, cam, opts, partial_C, partial_T, image, T_final, tile_depth, scratch,
                                        kScratchBytes, (cudaStream_t)stream, counts, false);
    rgs::prof_suppress(false);
    if (rc == RGS_EOVERFLOW && rgs_last_required_workspace() > kScratchBytes) {
        // keep the render's own reason (before or after binning) and say what to do
        char why[384];
        snprintf(why, sizeof why, "%s", rgs_last_error());
        rgs::set_error("render_fwd_noalloc: the fixed scratch of %zu bytes is too small (%s); "
                       "use rgs_render_fwd with a caller workspace", kScratchBytes, why);
    }
    return rc;
}
