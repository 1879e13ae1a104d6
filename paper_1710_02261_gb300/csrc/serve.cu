// serve.cu -- continuous-batching fold-in server.
//
// A request is a new slice of mode `mode`: its observed entries give a new row
// by the row update of Eq. (rowupdate) with G and the other factors fixed
// (Theorem 1), and the row predicts the request's query coordinates by
// Eq. (recon2).  A worker thread keeps up to `slots` batches on the GPU at
// once, each on its own stream and context: while one batch runs, the next is
// formed from the requests that have arrived since, admitted in arrival order
// while the device bytes of the batches in flight stay under the memory cap.
//
// Each request's observed entries start at a multiple of the Gram tile, the
// gap up to the next request being padding (mode column -1, no contribution),
// so a request's arithmetic -- delta per entry, the Gram sums in their fixed
// order, the FP64 solve, each prediction -- is the same whatever batch it
// lands in: results are bit-identical alone and in a mix.
#include "common.cuh"

#include <chrono>
#include <condition_variable>
#include <deque>
#include <mutex>
#include <new>
#include <thread>
#include <unordered_map>
#include <vector>

namespace ptk {
namespace {

using Clock = std::chrono::steady_clock;

struct ServeRequest {
    uint64_t ticket = 0;
    std::vector<int32_t> obs_idx;    // [m][order]
    std::vector<uint8_t> obs_vals;   // [m] model dtype
    std::vector<int32_t> query_idx;  // [q][order]
    int64_t m = 0, q = 0;
    int64_t bytes = 0;               // device bytes while in flight
    Clock::time_point arrival, done_at;
    std::vector<uint8_t> row, preds;  // results
    bool done = false;
};

struct BatchSlot {
    cudaStream_t stream = nullptr;
    cudaEvent_t event = nullptr;
    ptk_ctx* ctx = nullptr;
    // pinned host staging
    uint8_t* h_in = nullptr;
    uint8_t* h_out = nullptr;
    size_t in_bytes = 0, out_bytes = 0;
    // device buffers
    uint8_t* d_in = nullptr;
    uint8_t* d_out = nullptr;
    std::vector<uint64_t> tickets;
    int64_t bytes = 0;
    bool busy = false;
    // layout of the packed batch
    int64_t count = 0, total_obs = 0, total_q = 0;
};

}  // namespace
}  // namespace ptk

struct ptk_server {
    ptk_model model{};
    ptk_server_opts opts{};
    int device = 0;
    int tile = 1;
    size_t esz = 4;
    std::vector<ptk::BatchSlot> slots;
    std::mutex mu;
    std::condition_variable cv;
    std::deque<uint64_t> queue;
    std::unordered_map<uint64_t, ptk::ServeRequest> reqs;
    uint64_t next_ticket = 1;
    int64_t inflight_bytes = 0;
    ptk_server_stats stats{};
    bool stop = false;
    ptk_status worker_status = PTK_OK;
    char worker_error[256] = "";
    std::thread worker;
};

namespace ptk {
namespace {

int64_t padded_obs(const ptk_server* s, int64_t m) { return (m + s->tile - 1) / s->tile * s->tile; }

// bytes a request occupies on the device while its batch is in flight
int64_t request_bytes(const ptk_server* s, int64_t m, int64_t q) {
    const int N = s->model.order;
    const int ld = delta_out_ld(s->model.J[s->opts.mode]);
    const int64_t mp = std::max<int64_t>(padded_obs(s, m), s->tile);
    return mp * (int64_t)(4 * N + s->esz + s->esz * ld + 4) + q * (int64_t)(4 * N + s->esz + s->esz * ld + 4) +
           (int64_t)gram_nout(s->model.J[s->opts.mode]) * 8 + 64;
}

// layout of a slot's packed input: obs_idx | obs_vals | obs_ptr | query_idx | query_ptr
struct Layout {
    size_t obs_idx, obs_vals, obs_ptr, query_idx, query_ptr, total;
};
Layout layout(const ptk_server* s, int64_t obs, int64_t q, int64_t count) {
    auto al = [](size_t x) { return (x + 255) / 256 * 256; };
    Layout L;
    const int N = s->model.order;
    L.obs_idx = 0;
    L.obs_vals = al(L.obs_idx + sizeof(int32_t) * N * obs);
    L.obs_ptr = al(L.obs_vals + s->esz * obs);
    L.query_idx = al(L.obs_ptr + sizeof(int64_t) * (count + 1));
    L.query_ptr = al(L.query_idx + sizeof(int32_t) * N * q);
    L.total = al(L.query_ptr + sizeof(int64_t) * (count + 1));
    return L;
}

ptk_status launch_batch(ptk_server* s, BatchSlot& sl, std::vector<ServeRequest*>& batch) {
    const int N = s->model.order;
    const int mode = s->opts.mode;
    const int J = s->model.J[mode];
    int64_t obs = 0, q = 0;
    for (ServeRequest* r : batch) {
        obs += padded_obs(s, r->m);
        q += r->q;
    }
    const int64_t count = (int64_t)batch.size();
    const Layout L = layout(s, obs, q, count);
    int32_t* oi = (int32_t*)(sl.h_in + L.obs_idx);
    uint8_t* ov = sl.h_in + L.obs_vals;
    int64_t* op = (int64_t*)(sl.h_in + L.obs_ptr);
    int32_t* qi = (int32_t*)(sl.h_in + L.query_idx);
    int64_t* qp = (int64_t*)(sl.h_in + L.query_ptr);
    int64_t eo = 0, eq = 0;
    for (int64_t r = 0; r < count; ++r) {
        ServeRequest* rq = batch[r];
        op[r] = eo;
        qp[r] = eq;
        std::memcpy(oi + eo * N, rq->obs_idx.data(), sizeof(int32_t) * N * rq->m);
        for (int64_t e = 0; e < rq->m; ++e) oi[(eo + e) * N + mode] = 0;
        std::memcpy(ov + eo * s->esz, rq->obs_vals.data(), s->esz * rq->m);
        const int64_t mp = padded_obs(s, rq->m);
        for (int64_t e = rq->m; e < mp; ++e) {  // padding: contributes nothing
            for (int k = 0; k < N; ++k) oi[(eo + e) * N + k] = 0;
            oi[(eo + e) * N + mode] = -1;
            std::memset(ov + (eo + e) * s->esz, 0, s->esz);
        }
        std::memcpy(qi + eq * N, rq->query_idx.data(), sizeof(int32_t) * N * rq->q);
        for (int64_t e = 0; e < rq->q; ++e) qi[(eq + e) * N + mode] = 0;
        eo += mp;
        eq += rq->q;
    }
    op[count] = eo;
    qp[count] = eq;
    PTK_CUDA(cudaMemcpyAsync(sl.d_in, sl.h_in, L.total, cudaMemcpyHostToDevice, sl.stream));
    ptk_foldin_batch b{};
    b.count = (int32_t)count;
    b.obs_ptr = (const int64_t*)(sl.d_in + L.obs_ptr);
    b.obs_idx = (const int32_t*)(sl.d_in + L.obs_idx);
    b.obs_vals = sl.d_in + L.obs_vals;
    b.query_ptr = (const int64_t*)(sl.d_in + L.query_ptr);
    b.query_idx = (const int32_t*)(sl.d_in + L.query_idx);
    b.rows_out = sl.d_out;
    const size_t rows_bytes = (s->esz * count * J + 255) / 256 * 256;
    b.preds_out = sl.d_out + rows_bytes;
    b.total_obs = eo;
    b.total_query = eq;
    PTK_TRY(ptk_foldin(sl.ctx, &s->model, mode, &b, s->opts.lambda, s->opts.precision, sl.stream));
    PTK_CUDA(cudaMemcpyAsync(sl.h_out, sl.d_out, rows_bytes + s->esz * std::max<int64_t>(eq, 1),
                             cudaMemcpyDeviceToHost, sl.stream));
    PTK_CUDA(cudaEventRecord(sl.event, sl.stream));
    sl.count = count;
    sl.total_obs = eo;
    sl.total_q = eq;
    sl.busy = true;
    return PTK_OK;
}

void finish_batch(ptk_server* s, BatchSlot& sl) {
    const int J = s->model.J[s->opts.mode];
    const size_t rows_bytes = (s->esz * sl.count * J + 255) / 256 * 256;
    const auto now = Clock::now();
    std::lock_guard<std::mutex> lock(s->mu);
    int64_t eq = 0;
    for (size_t r = 0; r < sl.tickets.size(); ++r) {
        auto it = s->reqs.find(sl.tickets[r]);
        if (it == s->reqs.end()) continue;
        ServeRequest& rq = it->second;
        rq.row.assign(sl.h_out + r * s->esz * J, sl.h_out + (r + 1) * s->esz * J);
        rq.preds.assign(sl.h_out + rows_bytes + eq * s->esz, sl.h_out + rows_bytes + (eq + rq.q) * s->esz);
        eq += rq.q;
        rq.done = true;
        rq.done_at = now;
        s->stats.completed += 1;
    }
    s->inflight_bytes -= sl.bytes;
    sl.tickets.clear();
    sl.bytes = 0;
    sl.busy = false;
    s->cv.notify_all();
}

void worker_main(ptk_server* s) {
    cudaSetDevice(s->device);
    while (true) {
        bool progressed = false;
        // completions
        for (BatchSlot& sl : s->slots) {
            if (sl.busy && cudaEventQuery(sl.event) == cudaSuccess) {
                finish_batch(s, sl);
                progressed = true;
            }
        }
        // form and launch a batch on a free slot
        BatchSlot* free_slot = nullptr;
        for (BatchSlot& sl : s->slots)
            if (!sl.busy) {
                free_slot = &sl;
                break;
            }
        if (free_slot) {
            std::vector<ServeRequest*> batch;
            int64_t obs = 0, q = 0, bytes = 0;
            {
                std::lock_guard<std::mutex> lock(s->mu);
                while (!s->queue.empty() && (int64_t)batch.size() < s->opts.max_batch_requests) {
                    ServeRequest& r = s->reqs[s->queue.front()];
                    const int64_t mp = padded_obs(s, r.m);
                    if (!batch.empty() && (obs + mp > s->opts.max_batch_entries || q + r.q > s->opts.max_batch_queries))
                        break;
                    if (s->inflight_bytes + bytes + r.bytes > s->opts.memory_cap_bytes) break;  // admission
                    batch.push_back(&r);
                    obs += mp;
                    q += r.q;
                    bytes += r.bytes;
                    s->queue.pop_front();
                }
                if (!batch.empty()) {
                    s->inflight_bytes += bytes;
                    s->stats.max_inflight_bytes = std::max(s->stats.max_inflight_bytes, s->inflight_bytes);
                    s->stats.batches += 1;
                }
            }
            if (!batch.empty()) {
                free_slot->tickets.clear();
                for (ServeRequest* r : batch) free_slot->tickets.push_back(r->ticket);
                free_slot->bytes = bytes;
                ptk_status rc = launch_batch(s, *free_slot, batch);
                if (rc != PTK_OK) {
                    std::lock_guard<std::mutex> lock(s->mu);
                    s->worker_status = rc;
                    std::snprintf(s->worker_error, sizeof s->worker_error, "%s", get_error());
                    s->stop = true;
                    s->cv.notify_all();
                    return;
                }
                progressed = true;
            }
        }
        std::unique_lock<std::mutex> lock(s->mu);
        if (s->stop) {
            bool any_busy = false;
            for (BatchSlot& sl : s->slots) any_busy = any_busy || sl.busy;
            if (!any_busy) return;
        }
        if (!progressed) {
            // poll: a batch in flight finishes on the GPU without waking us
            s->cv.wait_for(lock, std::chrono::microseconds(20));
        }
    }
}

}  // namespace
}  // namespace ptk

using namespace ptk;

extern "C" {

ptk_status ptk_server_create(const ptk_model* m, int device, const ptk_server_opts* o, ptk_server** out) {
    PTK_CHECK_ARG(m && o && out, "null argument");
    *out = nullptr;
    PTK_TRY(check_model(m));
    PTK_CHECK_ARG(o->mode >= 0 && o->mode < m->order, "mode out of range");
    PTK_CHECK_ARG(o->lambda > 0, "lambda must be > 0");
    PTK_CHECK_ARG(o->slots >= 1 && o->slots <= 8, "slots out of [1, 8]");
    PTK_CHECK_ARG(o->max_batch_requests >= 1 && o->max_batch_entries >= 1 && o->max_batch_queries >= 1,
                  "batch limits must be >= 1");
    PTK_CHECK_ARG(o->memory_cap_bytes > 0 && o->max_queue >= 1, "memory cap and queue length must be > 0");
    PTK_CUDA(cudaSetDevice(device));
    ptk_server* s = new (std::nothrow) ptk_server();
    if (!s) return PTK_ERR_OUT_OF_MEMORY;
    s->model = *m;
    s->opts = *o;
    s->device = device;
    s->esz = dtype_size(m->dtype);
    s->tile = gram_tile_entries(m->J[o->mode], m->dtype);
    const int J = m->J[o->mode];
    const int64_t max_obs = o->max_batch_entries + (int64_t)o->max_batch_requests * s->tile;
    const Layout L = layout(s, max_obs, o->max_batch_queries, o->max_batch_requests);
    const size_t out_bytes = (s->esz * o->max_batch_requests * J + 255) / 256 * 256 + s->esz * o->max_batch_queries + 256;
    s->slots.resize(o->slots);
    ptk_status rc = PTK_OK;
    for (BatchSlot& sl : s->slots) {
        if (cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&sl.event, cudaEventDisableTiming) != cudaSuccess ||
            cudaMallocHost(&sl.h_in, L.total) != cudaSuccess || cudaMallocHost(&sl.h_out, out_bytes) != cudaSuccess ||
            cudaMalloc(&sl.d_in, L.total) != cudaSuccess || cudaMalloc(&sl.d_out, out_bytes) != cudaSuccess) {
            cudaGetLastError();
            set_error("ptk_server_create: allocation of the batch buffers failed");
            rc = PTK_ERR_OUT_OF_MEMORY;
            break;
        }
        sl.in_bytes = L.total;
        sl.out_bytes = out_bytes;
        rc = ptk_create(&sl.ctx, device);
        if (rc != PTK_OK) break;
    }
    // warm-up: one full-size batch per slot grows each context's scratch now,
    // not on the first requests
    for (BatchSlot& sl : s->slots) {
        if (rc != PTK_OK) break;
        const int64_t count = o->max_batch_requests;
        const int64_t obs = std::max<int64_t>(max_obs / s->tile, 1) * s->tile, q = o->max_batch_queries;
        const Layout W = layout(s, obs, q, count);
        std::memset(sl.h_in, 0, W.total);
        int64_t* op = (int64_t*)(sl.h_in + W.obs_ptr);
        int64_t* qp = (int64_t*)(sl.h_in + W.query_ptr);
        for (int64_t r = 0; r <= count; ++r) {
            op[r] = std::min(obs, (obs / count + s->tile) / s->tile * s->tile * r);
            qp[r] = q * r / count;
        }
        op[count] = obs;
        if (cudaMemcpy(sl.d_in, sl.h_in, W.total, cudaMemcpyHostToDevice) != cudaSuccess) {
            set_error("ptk_server_create: warm-up copy failed");
            rc = PTK_ERR_CUDA;
            break;
        }
        ptk_foldin_batch b{};
        b.count = (int32_t)count;
        b.obs_ptr = (const int64_t*)(sl.d_in + W.obs_ptr);
        b.obs_idx = (const int32_t*)(sl.d_in + W.obs_idx);
        b.obs_vals = sl.d_in + W.obs_vals;
        b.query_ptr = (const int64_t*)(sl.d_in + W.query_ptr);
        b.query_idx = (const int32_t*)(sl.d_in + W.query_idx);
        b.rows_out = sl.d_out;
        b.preds_out = sl.d_out + (s->esz * count * J + 255) / 256 * 256;
        b.total_obs = obs;
        b.total_query = q;
        rc = ptk_foldin(sl.ctx, &s->model, o->mode, &b, o->lambda, o->precision, sl.stream);
        if (rc == PTK_OK && cudaStreamSynchronize(sl.stream) != cudaSuccess) {
            set_error("ptk_server_create: warm-up batch failed");
            rc = PTK_ERR_CUDA;
        }
    }
    if (rc != PTK_OK) {
        ptk_server_destroy(s);
        return rc;
    }
    s->worker = std::thread(worker_main, s);
    *out = s;
    return PTK_OK;
}

ptk_status ptk_server_submit(ptk_server* s, const int32_t* obs_idx_h, const void* obs_vals_h, int64_t m,
                             const int32_t* query_idx_h, int64_t q, uint64_t* ticket) {
    PTK_CHECK_ARG(s && ticket, "null argument");
    PTK_CHECK_ARG(m >= 0 && q >= 0, "negative sizes");
    PTK_CHECK_ARG((m == 0 || (obs_idx_h && obs_vals_h)) && (q == 0 || query_idx_h), "null arrays");
    const int N = s->model.order;
    PTK_CHECK_ARG(padded_obs(s, m) <= s->opts.max_batch_entries + s->tile && q <= s->opts.max_batch_queries,
                  "request larger than one batch");
    for (int64_t e = 0; e < m; ++e)
        for (int k = 0; k < N; ++k)
            if (k != s->opts.mode && (obs_idx_h[e * N + k] < 0 || obs_idx_h[e * N + k] >= s->model.dims[k])) {
                set_error("observed coordinate out of range");
                return PTK_ERR_INVALID_ARG;
            }
    for (int64_t e = 0; e < q; ++e)
        for (int k = 0; k < N; ++k)
            if (k != s->opts.mode && (query_idx_h[e * N + k] < 0 || query_idx_h[e * N + k] >= s->model.dims[k])) {
                set_error("query coordinate out of range");
                return PTK_ERR_INVALID_ARG;
            }
    const int64_t bytes = request_bytes(s, m, q);
    std::lock_guard<std::mutex> lock(s->mu);
    if (s->worker_status != PTK_OK) {
        set_error("server stopped: %s", s->worker_error);
        return s->worker_status;
    }
    if (bytes > s->opts.memory_cap_bytes || (int64_t)s->queue.size() >= s->opts.max_queue) {
        s->stats.rejected += 1;
        set_error(bytes > s->opts.memory_cap_bytes ? "request exceeds the memory cap" : "queue full");
        return PTK_ERR_BUSY;
    }
    const uint64_t t = s->next_ticket++;
    ServeRequest& r = s->reqs[t];
    r.ticket = t;
    r.m = m;
    r.q = q;
    r.bytes = bytes;
    r.obs_idx.assign(obs_idx_h, obs_idx_h + m * N);
    r.obs_vals.assign((const uint8_t*)obs_vals_h, (const uint8_t*)obs_vals_h + m * s->esz);
    r.query_idx.assign(query_idx_h, query_idx_h + q * N);
    r.arrival = Clock::now();
    s->queue.push_back(t);
    s->stats.submitted += 1;
    s->cv.notify_all();
    *ticket = t;
    return PTK_OK;
}

ptk_status ptk_server_poll(ptk_server* s, uint64_t ticket, void* row_h, void* preds_h, int32_t* done,
                           double* latency_ms) {
    PTK_CHECK_ARG(s && done, "null argument");
    std::lock_guard<std::mutex> lock(s->mu);
    *done = 0;
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end()) {
        set_error("unknown ticket %llu", (unsigned long long)ticket);
        return PTK_ERR_INVALID_ARG;
    }
    if (!it->second.done) {
        if (s->worker_status != PTK_OK) {
            set_error("server stopped: %s", s->worker_error);
            return s->worker_status;
        }
        return PTK_OK;
    }
    ServeRequest& r = it->second;
    if (row_h) std::memcpy(row_h, r.row.data(), r.row.size());
    if (preds_h && !r.preds.empty()) std::memcpy(preds_h, r.preds.data(), r.preds.size());
    if (latency_ms) latency_ms[0] = std::chrono::duration<double, std::milli>(r.done_at - r.arrival).count();
    *done = 1;
    s->reqs.erase(it);
    return PTK_OK;
}

ptk_status ptk_server_read_stats(ptk_server* s, ptk_server_stats* out) {
    PTK_CHECK_ARG(s && out, "null argument");
    std::lock_guard<std::mutex> lock(s->mu);
    *out = s->stats;
    out->queued = (int64_t)s->queue.size();
    out->inflight_bytes = s->inflight_bytes;
    return PTK_OK;
}

void ptk_server_destroy(ptk_server* s) {
    if (!s) return;
    {
        std::lock_guard<std::mutex> lock(s->mu);
        s->stop = true;
        s->queue.clear();
        s->cv.notify_all();
    }
    if (s->worker.joinable()) s->worker.join();
    cudaSetDevice(s->device);
    for (BatchSlot& sl : s->slots) {
        if (sl.stream) cudaStreamSynchronize(sl.stream);
        if (sl.ctx) ptk_destroy(sl.ctx);
        if (sl.event) cudaEventDestroy(sl.event);
        if (sl.stream) cudaStreamDestroy(sl.stream);
        if (sl.h_in) cudaFreeHost(sl.h_in);
        if (sl.h_out) cudaFreeHost(sl.h_out);
        if (sl.d_in) cudaFree(sl.d_in);
        if (sl.d_out) cudaFree(sl.d_out);
    }
    delete s;
}

}  // extern "C"
