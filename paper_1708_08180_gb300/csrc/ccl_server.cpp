// ccl_server.cpp -- continuous-batching request server over ccl_label_batched.
//
// Requests (host buffers) enter a FIFO.  max_inflight worker threads each own
// a CUDA stream; whenever a worker is free it takes every queued request that
// fits (up to max_batch images and the free part of the HBM budget), so
// requests that arrive while other batches are on the GPU join the next batch
// as soon as a slot and memory free up.  A batch is: stream-ordered allocation
// from a private memory pool, one host-to-device copy per image, one batched
// labelling launch, one device-to-host copy per image, free, stream sync.
// Batches of different workers overlap on the device (copies of one with
// kernels of another).
//
// Admission: a request's footprint is its image (1 B/px) + labels (4 B/px) +
// labelling scratch; a request whose footprint exceeds the whole budget is
// rejected at submit, others wait until the budget has room.  Batch formation
// takes queued requests in FIFO order and may look past one that does not fit
// the free budget (at most kLookAhead queue entries), so a large request does
// not hold back smaller ones behind it; a request passed over kMaxPassOvers
// times stops the look-ahead until it is admitted, so it cannot starve.
//
// Timing: each batch records CUDA events around its host-to-device copies,
// its labelling launch and its device-to-host copies; ccl_server_timing
// reports their mean durations per batch.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "../../include/ccl.h"

namespace {

using Clock = std::chrono::steady_clock;

constexpr int kLookAhead = 32;      // queue entries examined past one that does not fit
constexpr int kMaxPassOvers = 8;    // then strict FIFO until that request is admitted

struct Request {
    int passed_over = 0;            // batches formed while it waited at or near the head
    uint64_t id = 0;
    const uint8_t *h_img = nullptr;
    int32_t *h_out = nullptr;
    int h = 0, w = 0;
    size_t footprint = 0;
    Clock::time_point t_submit;
    bool done = false;
    ccl_status status = CCL_ERR_PENDING;
};

size_t align256(size_t v) { return (v + 255u) & ~(size_t)255u; }

}  // namespace

struct ccl_server {
    ccl_server_config cfg{};
    cudaMemPool_t pool = nullptr;
    std::mutex mu;
    std::condition_variable cv_work;   // workers: new requests / budget freed / stop
    std::condition_variable cv_done;   // waiters: a request finished
    std::deque<Request *> pending;
    std::unordered_map<uint64_t, Request *> reqs;
    uint64_t next_id = 1;
    size_t in_use = 0;
    bool stopping = false;
    std::vector<std::thread> workers;
    // statistics
    double t_h2d_ms = 0.0, t_label_ms = 0.0, t_d2h_ms = 0.0;
    uint64_t timed_batches = 0;
    std::vector<double> lat_ms;
    uint64_t completed = 0, rejected = 0;
    double pixels = 0.0;
    bool any = false;
    Clock::time_point t_first, t_last;

    void worker_main(int slot);
    ccl_status run_batch(cudaStream_t s, cudaEvent_t *ev, std::vector<Request *> &batch);
    bool take_batch(std::vector<Request *> &batch, size_t &bytes);
};

static size_t request_footprint(int h, int w, int conn) {
    const size_t px = (size_t)h * (size_t)w;
    ccl_image im{reinterpret_cast<const uint8_t *>(256), reinterpret_cast<int32_t *>(256), h, w};
    return align256(px) + align256(px * 4) + ccl_batched_workspace_bytes(&im, 1, conn);
}

ccl_status ccl_server::run_batch(cudaStream_t s, cudaEvent_t *ev, std::vector<Request *> &batch) {
    const int n = (int)batch.size();
    std::vector<ccl_image> ims(n);
    std::vector<size_t> img_off(n), lab_off(n);
    size_t off = 0;
    for (int k = 0; k < n; ++k) {
        const size_t px = (size_t)batch[k]->h * batch[k]->w;
        img_off[k] = off;
        off += align256(px);
        lab_off[k] = off;
        off += align256(px * 4);
    }
    // scratch sized with the real pointers' alignment (the arena is 256-aligned)
    for (int k = 0; k < n; ++k)
        ims[k] = {reinterpret_cast<const uint8_t *>(256), reinterpret_cast<int32_t *>(256),
                  batch[k]->h, batch[k]->w};
    const size_t ws_bytes = ccl_batched_workspace_bytes(ims.data(), n, cfg.connectivity);
    const size_t ws_off = off;
    off += align256(ws_bytes);

    void *arena = nullptr;
    if (cudaMallocFromPoolAsync(&arena, off, pool, s) != cudaSuccess) {
        cudaGetLastError();
        return CCL_ERR_OOM;
    }
    char *base = static_cast<char *>(arena);
    ccl_status st = CCL_OK;
    if (ev) cudaEventRecord(ev[0], s);
    for (int k = 0; k < n && st == CCL_OK; ++k) {
        const size_t px = (size_t)batch[k]->h * batch[k]->w;
        ims[k].d_img = reinterpret_cast<const uint8_t *>(base + img_off[k]);
        ims[k].d_labels = reinterpret_cast<int32_t *>(base + lab_off[k]);
        if (cudaMemcpyAsync(base + img_off[k], batch[k]->h_img, px, cudaMemcpyHostToDevice, s) !=
            cudaSuccess)
            st = CCL_ERR_CUDA;
    }
    if (ev) cudaEventRecord(ev[1], s);
    if (st == CCL_OK)
        st = ccl_label_batched(ims.data(), n, cfg.connectivity, base + ws_off, ws_bytes, s);
    if (ev) cudaEventRecord(ev[2], s);
    for (int k = 0; k < n && st == CCL_OK; ++k) {
        const size_t px = (size_t)batch[k]->h * batch[k]->w;
        if (cudaMemcpyAsync(batch[k]->h_out, ims[k].d_labels, px * 4, cudaMemcpyDeviceToHost, s) !=
            cudaSuccess)
            st = CCL_ERR_CUDA;
    }
    if (ev) cudaEventRecord(ev[3], s);
    cudaFreeAsync(arena, s);
    if (cudaStreamSynchronize(s) != cudaSuccess) {
        cudaGetLastError();
        st = CCL_ERR_CUDA;
    }
    if (ev && st == CCL_OK) {
        float a = 0.f, b = 0.f, c = 0.f;
        if (cudaEventElapsedTime(&a, ev[0], ev[1]) == cudaSuccess &&
            cudaEventElapsedTime(&b, ev[1], ev[2]) == cudaSuccess &&
            cudaEventElapsedTime(&c, ev[2], ev[3]) == cudaSuccess) {
            std::lock_guard<std::mutex> lk(mu);
            t_h2d_ms += a;
            t_label_ms += b;
            t_d2h_ms += c;
            ++timed_batches;
        } else {
            cudaGetLastError();
        }
    }
    return st;
}

// Called with mu held: move the next batch out of the queue.  FIFO among the
// requests that fit; the scan looks at most kLookAhead entries past the first
// one that does not fit, and not past one that was passed over too often.
bool ccl_server::take_batch(std::vector<Request *> &batch, size_t &bytes) {
    int skipped = 0;
    for (auto it = pending.begin(); it != pending.end() && (int)batch.size() < cfg.max_batch;) {
        Request *r = *it;
        if (in_use + bytes + r->footprint <= cfg.hbm_budget_bytes) {
            batch.push_back(r);
            bytes += r->footprint;
            it = pending.erase(it);
            continue;
        }
        if (r->passed_over >= kMaxPassOvers || ++skipped > kLookAhead) break;
        ++it;
    }
    if (batch.empty()) return false;
    // every request still queued ahead of an admitted one was passed over
    const uint64_t last = batch.back()->id;
    for (Request *r : pending) {
        if (r->id > last) break;
        ++r->passed_over;
    }
    return true;
}

void ccl_server::worker_main(int slot) {
    (void)slot;
    cudaSetDevice(cfg.device);
    cudaStream_t s = nullptr;
    const bool stream_ok = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) == cudaSuccess;
    cudaEvent_t ev[4] = {};
    bool ev_ok = stream_ok;
    for (auto &e : ev)
        if (ev_ok && cudaEventCreate(&e) != cudaSuccess) { cudaGetLastError(); ev_ok = false; }
    for (;;) {
        std::vector<Request *> batch;
        size_t bytes = 0;
        {
            std::unique_lock<std::mutex> lk(mu);
            for (;;) {
                if (!pending.empty() && take_batch(batch, bytes)) break;
                if (pending.empty() && stopping) break;
                cv_work.wait(lk);
            }
            if (batch.empty()) break;   // stopping and nothing left
            in_use += bytes;
        }
        const ccl_status st = stream_ok ? run_batch(s, ev_ok ? ev : nullptr, batch) : CCL_ERR_CUDA;
        const auto now = Clock::now();
        {
            std::lock_guard<std::mutex> lk(mu);
            in_use -= bytes;
            for (Request *r : batch) {
                r->status = st;
                r->done = true;
                if (st == CCL_OK) {
                    lat_ms.push_back(
                        std::chrono::duration<double, std::milli>(now - r->t_submit).count());
                    ++completed;
                    pixels += (double)r->h * r->w;
                }
            }
            t_last = now;
        }
        cv_done.notify_all();
        cv_work.notify_all();
    }
    for (auto &e : ev)
        if (e) cudaEventDestroy(e);
    if (s) cudaStreamDestroy(s);
}

extern "C" ccl_status ccl_server_create(const ccl_server_config *cfg, ccl_server **out) {
    if (!cfg || !out) return CCL_ERR_INVALID_ARG;
    *out = nullptr;
    if (cfg->connectivity != 4 && cfg->connectivity != 8) return CCL_ERR_INVALID_ARG;
    if (cfg->max_batch < 0 || cfg->max_inflight < 0) return CCL_ERR_INVALID_ARG;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess) { cudaGetLastError(); return CCL_ERR_CUDA; }
    if (cfg->device < 0 || cfg->device >= ndev) return CCL_ERR_INVALID_ARG;
    ccl_server *srv = new (std::nothrow) ccl_server();
    if (!srv) return CCL_ERR_OOM;
    srv->cfg = *cfg;
    if (srv->cfg.hbm_budget_bytes == 0) srv->cfg.hbm_budget_bytes = (size_t)40 << 30;
    if (srv->cfg.max_batch == 0) srv->cfg.max_batch = 256;
    if (srv->cfg.max_inflight == 0) srv->cfg.max_inflight = 2;
    if (cudaSetDevice(cfg->device) != cudaSuccess) { delete srv; return CCL_ERR_CUDA; }
    cudaMemPoolProps props{};
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = cfg->device;
    if (cudaMemPoolCreate(&srv->pool, &props) != cudaSuccess) {
        cudaGetLastError();
        delete srv;
        return CCL_ERR_CUDA;
    }
    // keep freed blocks cached in the pool up to the budget
    uint64_t keep = srv->cfg.hbm_budget_bytes;
    cudaMemPoolSetAttribute(srv->pool, cudaMemPoolAttrReleaseThreshold, &keep);
    for (int k = 0; k < srv->cfg.max_inflight; ++k)
        srv->workers.emplace_back(&ccl_server::worker_main, srv, k);
    *out = srv;
    return CCL_OK;
}

extern "C" ccl_status ccl_server_submit(ccl_server *srv, const uint8_t *h_img, int height,
                                        int width, int32_t *h_labels_out, uint64_t *req_id_out) {
    if (!srv || !h_img || !h_labels_out || !req_id_out) return CCL_ERR_INVALID_ARG;
    if (height < 1 || width < 1 || (long long)height * width > 2147483646LL)
        return CCL_ERR_INVALID_ARG;
    const size_t fp = request_footprint(height, width, srv->cfg.connectivity);
    Request *r = new (std::nothrow) Request();
    if (!r) return CCL_ERR_OOM;
    r->h_img = h_img;
    r->h_out = h_labels_out;
    r->h = height;
    r->w = width;
    r->footprint = fp;
    r->t_submit = Clock::now();
    {
        std::lock_guard<std::mutex> lk(srv->mu);
        if (srv->stopping) { delete r; return CCL_ERR_SHUTDOWN; }
        if (fp > srv->cfg.hbm_budget_bytes) {
            ++srv->rejected;
            delete r;
            return CCL_ERR_REJECTED;
        }
        r->id = srv->next_id++;
        if (!srv->any) { srv->any = true; srv->t_first = r->t_submit; }
        srv->reqs[r->id] = r;
        srv->pending.push_back(r);
        *req_id_out = r->id;
    }
    srv->cv_work.notify_one();
    return CCL_OK;
}

static ccl_status take_finished(ccl_server *srv, uint64_t id, Request *r) {
    const ccl_status st = r->status;
    srv->reqs.erase(id);
    delete r;
    return st;
}

extern "C" ccl_status ccl_server_wait(ccl_server *srv, uint64_t req_id, int timeout_ms) {
    if (!srv) return CCL_ERR_INVALID_ARG;
    std::unique_lock<std::mutex> lk(srv->mu);
    auto it = srv->reqs.find(req_id);
    if (it == srv->reqs.end()) return CCL_ERR_NOT_FOUND;
    Request *r = it->second;
    if (timeout_ms < 0) {
        srv->cv_done.wait(lk, [&] { return r->done; });
    } else if (!srv->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms),
                                      [&] { return r->done; })) {
        return CCL_ERR_TIMEOUT;
    }
    return take_finished(srv, req_id, r);
}

extern "C" ccl_status ccl_server_poll(ccl_server *srv, uint64_t req_id) {
    if (!srv) return CCL_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(srv->mu);
    auto it = srv->reqs.find(req_id);
    if (it == srv->reqs.end()) return CCL_ERR_NOT_FOUND;
    if (!it->second->done) return CCL_ERR_PENDING;
    return take_finished(srv, req_id, it->second);
}

extern "C" ccl_status ccl_server_stats(ccl_server *srv, double *p50_ms, double *p99_ms,
                                       double *gpix_per_s, uint64_t *completed,
                                       uint64_t *rejected) {
    if (!srv) return CCL_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(srv->mu);
    std::vector<double> v = srv->lat_ms;
    auto pct = [&](double q) -> double {
        if (v.empty()) return 0.0;
        const size_t k = std::min(v.size() - 1, (size_t)(q * (double)(v.size() - 1) + 0.5));
        std::nth_element(v.begin(), v.begin() + k, v.end());
        return v[k];
    };
    if (p50_ms) *p50_ms = pct(0.50);
    if (p99_ms) *p99_ms = pct(0.99);
    if (gpix_per_s) {
        const double secs =
            srv->completed ? std::chrono::duration<double>(srv->t_last - srv->t_first).count() : 0.0;
        *gpix_per_s = secs > 0 ? srv->pixels / secs / 1e9 : 0.0;
    }
    if (completed) *completed = srv->completed;
    if (rejected) *rejected = srv->rejected;
    return CCL_OK;
}

extern "C" ccl_status ccl_server_timing(ccl_server *srv, double *h2d_ms, double *label_ms,
                                        double *d2h_ms, uint64_t *batches) {
    if (!srv) return CCL_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(srv->mu);
    const double n = srv->timed_batches ? (double)srv->timed_batches : 1.0;
    if (h2d_ms) *h2d_ms = srv->t_h2d_ms / n;
    if (label_ms) *label_ms = srv->t_label_ms / n;
    if (d2h_ms) *d2h_ms = srv->t_d2h_ms / n;
    if (batches) *batches = srv->timed_batches;
    return CCL_OK;
}

extern "C" ccl_status ccl_server_destroy(ccl_server *srv) {
    if (!srv) return CCL_ERR_INVALID_ARG;
    {
        std::lock_guard<std::mutex> lk(srv->mu);
        srv->stopping = true;
    }
    srv->cv_work.notify_all();
    for (auto &t : srv->workers) t.join();
    for (auto &kv : srv->reqs) delete kv.second;
    srv->reqs.clear();
    cudaSetDevice(srv->cfg.device);
    if (srv->pool) cudaMemPoolDestroy(srv->pool);
    delete srv;
    return CCL_OK;
}
