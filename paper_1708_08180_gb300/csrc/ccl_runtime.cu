// ccl_runtime.cu -- status strings, the device error word, library-owned
// workspaces, ccl_sync / ccl_shutdown and host-only seam arithmetic.
#include <atomic>
#include <map>
#include <mutex>
#include <utility>

#include "ccl_core.cuh"
#include "ccl_internal.h"

namespace ccl {

// Device-side failures (a bounded loop that ran out) are OR-ed in here.
__device__ int g_ccl_error_word;

namespace {
// failure injection for tests (ccl_set_hop_budget, ccl_inject_alloc_failures)
std::atomic<int> g_hops_smem{kSmemHopBudget};
std::atomic<int> g_hops_glob{kGlobHopBudget};
std::atomic<int> g_fail_allocs{0};
std::mutex g_mu;
constexpr int kMaxDevices = 64;
std::atomic<int *> g_err_ptr[kMaxDevices];                        // device -> address
std::map<std::pair<int, cudaStream_t>, std::pair<void *, size_t>> g_ws;  // library workspaces
}  // namespace

int *device_error_word() {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return nullptr;
    int *p = g_err_ptr[dev].load(std::memory_order_acquire);
    if (p) return p;
    if (cudaGetSymbolAddress(reinterpret_cast<void **>(&p), g_ccl_error_word) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    g_err_ptr[dev].store(p, std::memory_order_release);
    return p;
}

int hop_budget_smem() { return g_hops_smem.load(std::memory_order_relaxed); }
int hop_budget_glob() { return g_hops_glob.load(std::memory_order_relaxed); }

// Consumes one injected allocation failure, if any is pending.
static bool take_injected_failure() {
    int c = g_fail_allocs.load();
    while (c > 0 && !g_fail_allocs.compare_exchange_weak(c, c - 1)) {
    }
    return c > 0;
}

void *library_workspace(cudaStream_t stream, size_t bytes, ccl_status *st) {
    if (take_injected_failure()) { *st = CCL_ERR_OOM; return nullptr; }
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) { *st = CCL_ERR_CUDA; return nullptr; }
    std::lock_guard<std::mutex> lk(g_mu);
    auto &slot = g_ws[{dev, stream}];
    if (slot.second >= bytes && slot.first) { *st = CCL_OK; return slot.first; }
    if (slot.first) {
        // the old buffer may still be in use by work queued on this stream
        if (cudaStreamSynchronize(stream) != cudaSuccess) { *st = CCL_ERR_CUDA; return nullptr; }
        cudaFree(slot.first);
        slot = {nullptr, 0};
    }
    void *p = nullptr;
    size_t want = bytes + bytes / 4 + 256;
    if (cudaMalloc(&p, want) != cudaSuccess) {
        cudaGetLastError();
        *st = CCL_ERR_OOM;
        return nullptr;
    }
    slot = {p, want};
    *st = CCL_OK;
    return p;
}

void free_library_workspaces() {
    std::lock_guard<std::mutex> lk(g_mu);
    int cur = 0;
    cudaGetDevice(&cur);
    for (auto &kv : g_ws) {
        if (!kv.second.first) continue;
        cudaSetDevice(kv.first.first);
        cudaDeviceSynchronize();
        cudaFree(kv.second.first);
    }
    g_ws.clear();
    cudaSetDevice(cur);
}

bool valid_image_dims(int height, int width) {
    if (height < 1 || width < 1) return false;
    return (long long)height * (long long)width <= 2147483646LL;
}

}  // namespace ccl

extern "C" const char *ccl_status_string(int status) {
    switch (status) {
        case CCL_OK: return "CCL_OK";
        case CCL_ERR_INVALID_ARG: return "CCL_ERR_INVALID_ARG";
        case CCL_ERR_CUDA: return "CCL_ERR_CUDA";
        case CCL_ERR_OOM: return "CCL_ERR_OOM";
        case CCL_ERR_TIMEOUT: return "CCL_ERR_TIMEOUT";
        case CCL_ERR_REJECTED: return "CCL_ERR_REJECTED";
        case CCL_ERR_SHUTDOWN: return "CCL_ERR_SHUTDOWN";
        case CCL_ERR_NOT_FOUND: return "CCL_ERR_NOT_FOUND";
        case CCL_ERR_PENDING: return "CCL_ERR_PENDING";
        default: return "CCL_ERR_UNKNOWN";
    }
}

extern "C" ccl_status ccl_sync(ccl_stream stream) {
    if (cudaStreamSynchronize(reinterpret_cast<cudaStream_t>(stream)) != cudaSuccess) {
        cudaGetLastError();
        return CCL_ERR_CUDA;
    }
    int *p = ccl::device_error_word();
    if (!p) return CCL_ERR_CUDA;
    int v = 0;
    if (cudaMemcpy(&v, p, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return CCL_ERR_CUDA;
    if (v != 0) {
        const int zero = 0;
        if (cudaMemcpy(p, &zero, sizeof(int), cudaMemcpyHostToDevice) != cudaSuccess)
            return CCL_ERR_CUDA;
        return CCL_ERR_TIMEOUT;
    }
    return CCL_OK;
}

extern "C" ccl_status ccl_set_hop_budget(int smem_hops, int global_hops) {
    if (smem_hops < 0 || global_hops < 0) return CCL_ERR_INVALID_ARG;
    ccl::g_hops_smem.store(smem_hops ? smem_hops : ccl::kSmemHopBudget);
    ccl::g_hops_glob.store(global_hops ? global_hops : ccl::kGlobHopBudget);
    return CCL_OK;
}

extern "C" ccl_status ccl_inject_alloc_failures(int count) {
    if (count < 0) return CCL_ERR_INVALID_ARG;
    ccl::g_fail_allocs.store(count);
    return CCL_OK;
}

extern "C" ccl_status ccl_shutdown(void) {
    ccl::free_library_workspaces();
    ccl::free_batched_state();
    ccl::forget_static_scratch();
    for (auto &p : ccl::g_err_ptr) p.store(nullptr, std::memory_order_release);
    return CCL_OK;
}

// Cross-tile neighbour pairs: all neighbour pairs of the image minus the ones
// inside a single tile (4-neighbour pairs of an a x b block: a(b-1) + b(a-1);
// diagonal pairs: 2(a-1)(b-1)).
extern "C" long long ccl_seam_pair_count(int height, int width, int connectivity, int tile_w,
                                         int tile_h) {
    if (!ccl::valid_image_dims(height, width) || !ccl::valid_conn(connectivity) || tile_w < 1 ||
        tile_h < 1)
        return -1;
    auto pairs4 = [](long long a, long long b) { return a * (b - 1) + b * (a - 1); };
    auto diag = [](long long a, long long b) { return 2 * (a - 1) * (b - 1); };
    const long long H = height, W = width;
    const long long fy = H / tile_h, ry = H % tile_h, fx = W / tile_w, rx = W % tile_w;
    // tile heights: fy of tile_h (+ one of ry); widths: fx of tile_w (+ one of rx)
    long long inside4 = 0, insided = 0;
    const long long hs[2] = {tile_h, ry}, hc[2] = {fy, ry ? 1 : 0};
    const long long ws[2] = {tile_w, rx}, wc[2] = {fx, rx ? 1 : 0};
    for (int i = 0; i < 2; ++i)
        for (int j = 0; j < 2; ++j) {
            if (!hc[i] || !wc[j]) continue;
            inside4 += hc[i] * wc[j] * pairs4(hs[i], ws[j]);
            insided += hc[i] * wc[j] * diag(hs[i], ws[j]);
        }
    long long n = pairs4(H, W) - inside4;
    if (connectivity == 8) n += diag(H, W) - insided;
    return n;
}
