// ccl_autotune.cu -- measures the tile width of every size class on this GPU
// and installs the fastest in the table that ccl_label and the batched path
// consult when no tile width is given.
//
// For each (height class, width class) a synthetic image of the class's
// representative size is generated on the device (i.i.d. foreground with
// probability 1/2 from a SplitMix64-style integer hash of the pixel index,
// Steele, Lea and Flood, OOPSLA 2014), every supported tile width is timed with
// CUDA events (median of `reps` runs after one warm-up), and the fastest wins.
#include <algorithm>
#include <vector>

#include "ccl_internal.h"

namespace ccl {

__global__ void k_tune_fill(uint8_t *img, long long n, unsigned long long seed) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        unsigned long long z = seed + (unsigned long long)i * 0x9E3779B97F4A7C15ull;
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        z ^= z >> 31;
        img[i] = (uint8_t)(z >> 63);
    }
}

static int class_extent(int c) { return c < kTileClasses - 1 ? (64 << c) : 4096; }

}  // namespace ccl

extern "C" ccl_status ccl_get_tile_table(int connectivity, int *widths) {
    if (!ccl::valid_conn(connectivity) || !widths) return CCL_ERR_INVALID_ARG;
    for (int hc = 0; hc < ccl::kTileClasses; ++hc)
        for (int wc = 0; wc < ccl::kTileClasses; ++wc)
            widths[hc * ccl::kTileClasses + wc] =
                ccl::default_tile_width(ccl::class_extent(hc), ccl::class_extent(wc), connectivity);
    return CCL_OK;
}

extern "C" ccl_status ccl_set_tile_table(int connectivity, const int *widths) {
    if (!ccl::valid_conn(connectivity) || !widths) return CCL_ERR_INVALID_ARG;
    for (int k = 0; k < ccl::kTileClasses * ccl::kTileClasses; ++k)
        if (!ccl::valid_tile_w(widths[k])) return CCL_ERR_INVALID_ARG;
    for (int hc = 0; hc < ccl::kTileClasses; ++hc)
        for (int wc = 0; wc < ccl::kTileClasses; ++wc)
            ccl::set_tile_table_entry(connectivity, hc, wc,
                                      widths[hc * ccl::kTileClasses + wc]);
    return CCL_OK;
}

extern "C" ccl_status ccl_autotune(int connectivity, int reps, ccl_stream stream) {
    if (!ccl::valid_conn(connectivity) || reps < 1) return CCL_ERR_INVALID_ARG;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const int maxe = ccl::class_extent(ccl::kTileClasses - 1);
    const size_t npx = (size_t)maxe * maxe;
    size_t ws_bytes = ccl_workspace_bytes(maxe, maxe, connectivity);
    uint8_t *img = nullptr;
    int32_t *lab = nullptr;
    void *ws = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    ccl_status st = CCL_OK;
    if (cudaMalloc(&img, npx) != cudaSuccess || cudaMalloc(&lab, npx * 4) != cudaSuccess ||
        cudaMalloc(&ws, ws_bytes) != cudaSuccess) {
        cudaGetLastError();
        st = CCL_ERR_OOM;
    }
    if (st == CCL_OK && (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess))
        st = CCL_ERR_CUDA;
    std::vector<int> table(ccl::kTileClasses * ccl::kTileClasses, 256);
    for (int hc = 0; hc < ccl::kTileClasses && st == CCL_OK; ++hc) {
        for (int wc = 0; wc < ccl::kTileClasses && st == CCL_OK; ++wc) {
            const int H = ccl::class_extent(hc), W = ccl::class_extent(wc);
            ccl::k_tune_fill<<<1024, 256, 0, s>>>(img, (long long)H * W,
                                                 0x5EEDull + 131ull * (hc * 16 + wc));
            float best = 1e30f;
            int best_tw = 256;
            int cap = 32;   // never wider than the image needs
            while (cap < W && cap < 256) cap <<= 1;
            for (int tw = 32; tw <= cap && st == CCL_OK; tw <<= 1) {
                std::vector<float> t;
                for (int r = 0; r <= reps && st == CCL_OK; ++r) {
                    cudaEventRecord(e0, s);
                    st = ccl_label_tiled(img, lab, H, W, connectivity, tw, 0u, ws, ws_bytes, stream);
                    cudaEventRecord(e1, s);
                    if (st != CCL_OK) break;
                    if (cudaEventSynchronize(e1) != cudaSuccess) { st = CCL_ERR_CUDA; break; }
                    float ms = 0.f;
                    cudaEventElapsedTime(&ms, e0, e1);
                    if (r > 0) t.push_back(ms);
                }
                if (st != CCL_OK || t.empty()) break;
                std::nth_element(t.begin(), t.begin() + t.size() / 2, t.end());
                const float med = t[t.size() / 2];
                if (med < best) { best = med; best_tw = tw; }
            }
            table[hc * ccl::kTileClasses + wc] = best_tw;
        }
    }
    if (st == CCL_OK) st = ccl_sync(stream);
    if (st == CCL_OK) st = ccl_set_tile_table(connectivity, table.data());
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (img) cudaFree(img);
    if (lab) cudaFree(lab);
    if (ws) cudaFree(ws);
    return st;
}
