// itc_noalloc.cu -- itc_fields_noalloc: the fields of one image without any caller-provided or
// library-allocated scratch.
//
// Some callers cannot allocate device memory at the point where they need the fields: a host
// that hands the library only its input and output buffers and forbids allocation during
// processing (a plugin or real-time host with a fixed memory budget), or code that must not call
// cudaMalloc while other work is being recorded.  For them the per-tile S_XX partial sums live in
// a fixed array in this file, sized once at load time; nothing is allocated per call.
#include <mutex>

#include "itc_internal.cuh"

namespace {

// Scratch of itc_fields_noalloc, laid out as itc_fields' workspace: the call's status word in
// the first 256 bytes, then one double per fields tile (ITC_NOALLOC_MAX_TILES doubles, 512 KiB).
// Every device that loads the library keeps it until the process exits.
static __device__ __align__(256) double g_noalloc_partials[32 + ITC_NOALLOC_MAX_TILES];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
void* g_scratch_of_device[kMaxDevices] = {};

// Device address of the scratch array on the current device, looked up once per device.
// Host code cannot use the array's name as a device address; cudaGetSymbolAddress gives it.
int scratch_address(void** out) {
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return ITC_ERR_CUDA;
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_of_device[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_partials) != cudaSuccess || !p) return ITC_ERR_CUDA;
        g_scratch_of_device[dev] = p;
    }
    *out = g_scratch_of_device[dev];
    return ITC_OK;
}

}  // namespace

extern "C" int itc_fields_noalloc(const itc_image* img, const itc_params* p, float* fields, double* sxx,
                                  void* stream) {
    const size_t need = itc_fields_workspace_bytes(img);   // status slot + one double per tile, 0 if invalid
    if (need == 0) return ITC_ERR_INVALID_ARG;
    if (need > sizeof(g_noalloc_partials)) return ITC_ERR_UNSUPPORTED;   // beyond the fixed scratch
    void* scratch = nullptr;
    const int rc = scratch_address(&scratch);
    if (rc) return rc;
    // The fields pass overwrites one partial per tile before the reduction reads them, and the
    // call clears the status word itself, so nothing else in the shared array needs clearing.
    return itc_fields(img, p, fields, sxx, scratch, sizeof(g_noalloc_partials), stream);
}
