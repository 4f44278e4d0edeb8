// ccl_noalloc.cu -- ccl_label_static: the single-image labelling path with its
// scratch memory in a fixed device array that lives in this library, for
// callers that cannot allocate device memory (see include/ccl.h).
//
// The scratch is a file-scope __device__ array of CCL_STATIC_SCRATCH_BYTES.
// Host code must not use the array's name as a device address (on the host it
// is only a stand-in symbol); its device address is fetched once per device
// with cudaGetSymbolAddress, with that device current, on the first call made
// on that device, and cached.
#include <atomic>

#include "ccl_internal.h"

namespace ccl {

static __device__ __align__(256) unsigned char g_static_scratch[CCL_STATIC_SCRATCH_BYTES];

namespace {
constexpr int kMaxDevices = 64;
std::atomic<void *> g_static_ptr[kMaxDevices];   // zero-initialised (static storage)
}  // namespace

// Device address of this device's copy of the scratch array (nullptr on error).
// Lock-free after the first call on a device; two first calls racing both look
// the address up and store the same value.
static void *static_scratch_address(int dev) {
    if (dev < 0 || dev >= kMaxDevices) return nullptr;
    void *p = g_static_ptr[dev].load(std::memory_order_acquire);
    if (p) return p;
    if (cudaGetSymbolAddress(&p, g_static_scratch) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    g_static_ptr[dev].store(p, std::memory_order_release);
    return p;
}

// Forget the cached addresses (a reset device gets new ones).
void forget_static_scratch() {
    for (auto &p : g_static_ptr) p.store(nullptr, std::memory_order_release);
}

}  // namespace ccl

extern "C" ccl_status ccl_label_static(const uint8_t *d_img, int32_t *d_labels, int height,
                                       int width, int connectivity, ccl_stream stream) {
    if (!d_img || !d_labels || !ccl::valid_image_dims(height, width) ||
        !ccl::valid_conn(connectivity))
        return CCL_ERR_INVALID_ARG;
    const size_t need = ccl_workspace_bytes(height, width, connectivity);
    if (need == 0 || need > (size_t)CCL_STATIC_SCRATCH_BYTES) return CCL_ERR_INVALID_ARG;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return CCL_ERR_CUDA;
    }
    void *scratch = ccl::static_scratch_address(dev);
    if (!scratch) return CCL_ERR_CUDA;
    // Every workspace word the kernels read is written earlier in the same
    // call (bit image, per-tile records), so nothing needs clearing here.
    return ccl::enqueue_label(d_img, d_labels, height, width, connectivity, 0, 0u, scratch,
                              (size_t)CCL_STATIC_SCRATCH_BYTES,
                              reinterpret_cast<cudaStream_t>(stream));
}
