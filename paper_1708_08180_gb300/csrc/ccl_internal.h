// ccl_internal.h -- host-side helpers shared by the library's translation
// units (not part of the public C ABI).
#pragma once

#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>
#include <utility>

#include "../../include/ccl.h"

namespace ccl {

// Device address of the current device's error word (set up once per device).
int *device_error_word();

// Forget the cached device addresses of the allocation-free scratch array.
void forget_static_scratch();

// Library-owned workspace for (current device, stream), grown to >= bytes.
void *library_workspace(cudaStream_t stream, size_t bytes, ccl_status *st);

// Release every library-owned workspace.
void free_library_workspaces();

// Hop budgets the 2-D kernels are launched with (ccl_set_hop_budget).
int hop_budget_smem();
int hop_budget_glob();

// Argument checks shared by the entry points.
bool valid_image_dims(int height, int width);
inline bool valid_conn(int conn) { return conn == 4 || conn == 8; }
inline bool valid_tile_w(int tw) { return tw == 32 || tw == 64 || tw == 128 || tw == 256; }

// Size-class table: tile width for an image (the autotuned default).
constexpr int kTileClasses = 7;   // extents <= 64, 128, 256, 512, 1024, 2048, > 2048
int tile_class(int extent);
int default_tile_width(int height, int width, int conn);
void set_tile_table_entry(int conn, int hc, int wc, int tile_w);

// Launch with programmatic stream serialisation: the grid may start once
// every block of the previous grid on the stream has called
// griddepcontrol.launch_dependents (or exited); it must griddepcontrol.wait
// before reading that grid's results.
template <typename... P, typename... A>
inline cudaError_t launch_pdl_smem(void (*kernel)(P...), unsigned grid, unsigned block,
                                   size_t smem, cudaStream_t s, A &&...args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(block);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, std::forward<A>(args)...);
}

template <typename... P, typename... A>
inline cudaError_t launch_pdl(void (*kernel)(P...), unsigned grid, unsigned block, cudaStream_t s,
                              A &&...args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(block);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, std::forward<A>(args)...);
}

// Release batched-path state.
void free_batched_state();

// Component-statistics outputs of ccl_label_with_stats.
struct StatsOut {
    void *comps;     // ccl_component records
    int max_comps;
    int32_t *ncomps;
};

// Enqueue the three single-image kernels with the given workspace (ccl_plain.cu).
// level < 0: foreground = nonzero byte, else byte == level; merge_out: the
// link phase writes only this pass's foreground pixels; so: also gather the
// statistics of every component (a fourth kernel packs the border ones).
ccl_status enqueue_label(const uint8_t *d_img, int32_t *d_labels, int height, int width,
                         int conn, int tile_w, unsigned flags, void *d_ws, size_t ws_bytes,
                         cudaStream_t stream, int level = -1, bool merge_out = false,
                         const StatsOut *so = nullptr);

}  // namespace ccl
