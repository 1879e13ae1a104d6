// serve_dev.cu -- fold-in server with a device-resident request loop.
//
// A request is a new slice of mode `mode` (Theorem 1 with G and the other
// factors fixed): its m observed entries give the new row
//     a = c (B + lambda I)^{-1},  B = sum delta delta^T,  c = sum x delta
// (Eqs. rowupdate, rowB, rowC, delta) and the row predicts the request's q
// query coordinates (Eq. recon2).
//
// The loop lives on the GPU: `workers` persistent CTAs poll a ring of request
// descriptors in host-mapped pinned memory, claim the next published request
// with a compare-and-swap on a head counter in device memory, and each runs
// its request to the end: delta of every entry (the core permuted for the mode
// in shared memory, the entry's factor rows beside it), the row sums in
// double-float (FP32 model) or FP64 over tiles of 256 entries in a fixed
// order, an FP64 Cholesky solve with one refinement step, the predictions,
// and the results written back to mapped memory before a done word.  While
// some CTAs work on long requests, others take the requests that arrive
// meanwhile: requests of any size are served as they come, each by one CTA,
// so a request's arithmetic, and its result bits, do not depend on what else
// is in flight.
//
// The host side admits requests in arrival order into an arena of request
// data (pinned, mapped) and into the ring while the arena's bytes and the
// ring's slots allow, publishes each with a release store of the ring's tail,
// and collects done words.  Every device wait is bounded: a CTA that finds no
// work for `idle_ms` (measured on globaltimer) leaves, and when the last one
// has left the kernel ends; a host thread relaunches it when requests are
// waiting.  A stop word ends the loop at destruction.
#include "common.cuh"

#include <atomic>
#include <chrono>
#include <deque>
#include <mutex>
#include <new>
#include <thread>
#include <unordered_map>
#include <vector>

namespace ptk {
namespace {

constexpr int DS_T = 256;  // threads per worker CTA; entries per row-sum tile

// one request in the ring (host-mapped; written by the host before the tail
// moves past it)
struct DsDesc {
    int64_t seq;      // the request's sequence number
    int64_t m, q;     // observed entries, query coordinates
    int64_t obs_off;  // arena offsets (bytes): obs_idx [m][N] int32, obs_vals [m] T, query_idx [q][N] int32
    int64_t val_off;
    int64_t qry_off;
    int64_t res_off;  // result offset (bytes) in the result area: row [J] T, preds [q] T
};

struct DsCtrl {
    volatile unsigned long long tail;  // requests published (host writes)
    volatile int stop;                 // 1: leave now
    int pad;
};

struct DsParams {
    int order, mode, J;                 // J = J[mode]
    int others[PTK_MAX_ORDER];          // the other modes in order; the last one is innermost
    int Jo[PTK_MAX_ORDER];
    const void* factors[PTK_MAX_ORDER];
    int64_t ld[PTK_MAX_ORDER];
    int sr;                             // row-buffer stride per thread (elements, odd)
    int rowoff[PTK_MAX_ORDER];          // offset of each other mode's row in a thread's buffer
    int64_t R;                          // |G| / J
    const void* Gp;                     // core permuted: [J][R], the other modes in order
    double lambda;
    int64_t ring;
    const DsCtrl* ctrl;                 // mapped
    const DsDesc* desc;                 // mapped [ring]
    unsigned long long* done;           // mapped [ring]: seq + 1 when done
    const uint8_t* arena;               // mapped
    uint8_t* results;                   // mapped
    unsigned long long* head;           // device: requests claimed
    int* flags;                         // device: [0] CTAs that left idle, [1] requests served, [2] rows not PD
    long long idle_ns;
};

__device__ __forceinline__ unsigned long long gtimer() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
__device__ __forceinline__ unsigned long long ld_acquire_sys(const volatile unsigned long long* p) {
    unsigned long long v;
    asm volatile("ld.acquire.sys.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

// double-float sum for the FP32 model's row sums (Dot2, Ogita, Rump, Oishi)
struct DsAccF {
    float s = 0.f, lo = 0.f;
    __device__ __forceinline__ void add_prod(float a, float b) {
        const float p = __fmul_rn(a, b);
        const float e = fmaf(a, b, -p);
        const float t = __fadd_rn(s, p);
        const float bb = __fsub_rn(t, s);
        const float q = __fadd_rn(__fsub_rn(s, __fsub_rn(t, bb)), __fsub_rn(p, bb));
        s = t;
        lo = __fadd_rn(lo, __fadd_rn(q, e));
    }
    __device__ __forceinline__ double value() const { return (double)s + (double)lo; }
};
struct DsAccD {
    double s = 0.0;
    __device__ __forceinline__ void add_prod(double a, double b) { s = fma(a, b, s); }
    __device__ __forceinline__ double value() const { return s; }
};
template <typename T>
struct DsAcc;
template <>
struct DsAcc<float> {
    using A = DsAccF;
};
template <>
struct DsAcc<double> {
    using A = DsAccD;
};

// delta of one coordinate for the free mode: the thread's factor rows are in
// rows[]; the innermost other mode L is walked inside each combination of the
// outer ones (its product prefix computed once)
template <typename T, int JM>
__device__ __forceinline__ void ds_delta(const DsParams& p, const T* __restrict__ Gp, const T* __restrict__ rows,
                                         T (&d)[JM]) {
#pragma unroll
    for (int j = 0; j < JM; ++j) d[j] = T(0);
    const int no = p.order - 1;
    const int JL = p.Jo[no - 1];
    const T* rl = rows + p.rowoff[no - 1];
    const int64_t outer = p.R / JL;
    int idx[PTK_MAX_ORDER] = {};
    for (int64_t o = 0; o < outer; ++o) {
        T w = T(1);
        for (int k = 0; k < no - 1; ++k) w *= rows[p.rowoff[k] + idx[k]];
        const T* g = Gp + o * JL;
        for (int l = 0; l < JL; ++l) {
            const T t = w * rl[l];
#pragma unroll
            for (int j = 0; j < JM; ++j) d[j] = fma(g[(int64_t)j * p.R + l], t, d[j]);
        }
        for (int k = no - 2; k >= 0; --k) {  // odometer over the outer modes, last fastest
            if (++idx[k] < p.Jo[k]) break;
            idx[k] = 0;
        }
    }
}

// copies the factor rows of a coordinate (other modes) into the thread's buffer
template <typename T>
__device__ __forceinline__ void ds_rows(const DsParams& p, const int32_t* co, T* rows) {
    for (int k = 0; k < p.order - 1; ++k) {
        const int mk = p.others[k];
        const T* a = (const T*)p.factors[mk] + (int64_t)co[mk] * p.ld[mk];
        for (int j = 0; j < p.Jo[k]; ++j) rows[p.rowoff[k] + j] = a[j];
    }
}

// FP64 Cholesky solve of (B + lambda I) a = c with one refinement step (J <= 16);
// B packed upper row-major, c after it.  Returns false when not positive definite.
template <int JM>
__device__ bool ds_solve(const double* __restrict__ sums, double lambda, double* a) {
    constexpr int NT = JM * (JM + 1) / 2;
    double M[JM][JM], L[JM][JM], c[JM], y[JM], r[JM], dx[JM];
    int g = 0;
    for (int i = 0; i < JM; ++i)
        for (int k = i; k < JM; ++k, ++g) {
            M[i][k] = sums[g] + (i == k ? lambda : 0.0);
            M[k][i] = M[i][k];
        }
    for (int i = 0; i < JM; ++i) c[i] = sums[NT + i];
    for (int i = 0; i < JM; ++i) {
        for (int k = 0; k <= i; ++k) {
            double s = M[i][k];
            for (int t = 0; t < k; ++t) s -= L[i][t] * L[k][t];
            if (i == k) {
                if (!(s > 0.0)) return false;
                L[i][i] = sqrt(s);
            } else {
                L[i][k] = s / L[k][k];
            }
        }
    }
    auto solve = [&](const double* rhs, double* x) {
        for (int i = 0; i < JM; ++i) {
            double s = rhs[i];
            for (int t = 0; t < i; ++t) s -= L[i][t] * y[t];
            y[i] = s / L[i][i];
        }
        for (int i = JM - 1; i >= 0; --i) {
            double s = y[i];
            for (int t = i + 1; t < JM; ++t) s -= L[t][i] * x[t];
            x[i] = s / L[i][i];
        }
    };
    solve(c, a);
    for (int i = 0; i < JM; ++i) {
        double s = c[i];
        for (int k = 0; k < JM; ++k) s -= M[i][k] * a[k];
        r[i] = s;
    }
    solve(r, dx);
    for (int i = 0; i < JM; ++i) a[i] += dx[i];
    for (int i = 0; i < JM; ++i)
        if (!isfinite(a[i])) return false;
    return true;
}

template <typename T, int JM>
__global__ void __launch_bounds__(DS_T, 1) dserve_kernel(const DsParams p) {
    using A = typename DsAcc<T>::A;
    constexpr int NT = JM * (JM + 1) / 2, NOUT = NT + JM, DL = JM + 1;
    extern __shared__ __align__(16) uint8_t smem[];
    T* Gs = reinterpret_cast<T*>(smem);                                   // [JM][R]
    T* rows = Gs + (size_t)JM * p.R;                                      // [DS_T][sr]
    float* tileD = reinterpret_cast<float*>(rows + (size_t)DS_T * p.sr); // [DS_T][DL] (FP32 model)
    T* tileT = reinterpret_cast<T*>(tileD);                               // (FP64 model: T)
    __shared__ double sums[NOUT];
    __shared__ double arow[JM];
    __shared__ long long claimed;
    __shared__ int leave;
    const int tid = threadIdx.x;
    for (int64_t i = tid; i < (int64_t)JM * p.R; i += DS_T) Gs[i] = ((const T*)p.Gp)[i];
    T* myrows = rows + (size_t)tid * p.sr;
    const int N = p.order, mode = p.mode;
    unsigned long long last = gtimer();
    __syncthreads();
    for (;;) {
        __syncthreads();  // every thread has read the last iteration's claim before it is replaced
        if (tid == 0) {
            claimed = -1;
            leave = 0;
            if (p.ctrl->stop) {
                leave = 1;
            } else {
                const unsigned long long t = ld_acquire_sys(&p.ctrl->tail);
                const unsigned long long h = atomicAdd(p.head, 0ull);
                if (h < t && atomicCAS(p.head, h, h + 1) == h) {
                    claimed = (long long)h;
                    last = gtimer();
                } else if (h >= t) {
                    if ((long long)(gtimer() - last) > p.idle_ns) {
                        leave = 1;  // no work for idle_ns: leave (the host relaunches when work comes)
                        atomicAdd(&p.flags[0], 1);
                    } else {
                        __nanosleep(2000);
                    }
                }
            }
        }
        __syncthreads();
        if (leave) break;
        if (claimed < 0) continue;
        // ---- one request --------------------------------------------------
        const DsDesc* dd = p.desc + claimed % p.ring;
        const int64_t m = dd->m, q = dd->q;
        const int32_t* oi = reinterpret_cast<const int32_t*>(p.arena + dd->obs_off);
        const T* ov = reinterpret_cast<const T*>(p.arena + dd->val_off);
        const int32_t* qi = reinterpret_cast<const int32_t*>(p.arena + dd->qry_off);
        T* out = reinterpret_cast<T*>(p.results + dd->res_off);
        // row sums over tiles of DS_T entries, each output summed by one thread in entry order
        int oj = -1, ok_ = -1;  // this thread's output (j, k); k == JM: c_j = sum x delta_j
        if (tid < NOUT) {
            if (tid < NT) {
                int a = 0, first = 0;
                while (tid >= first + (JM - a)) {
                    first += JM - a;
                    ++a;
                }
                oj = a;
                ok_ = a + (tid - first);
            } else {
                oj = tid - NT;
                ok_ = JM;
            }
        }
        A acc;
        for (int64_t t0 = 0; t0 < m; t0 += DS_T) {
            const int64_t e = t0 + tid;
            T d[JM];
            T x = T(0);
            if (e < m) {
                ds_rows<T>(p, oi + e * N, myrows);
                ds_delta<T, JM>(p, Gs, myrows, d);
                x = ov[e];
            } else {
#pragma unroll
                for (int j = 0; j < JM; ++j) d[j] = T(0);
            }
#pragma unroll
            for (int j = 0; j < JM; ++j) tileT[tid * DL + j] = d[j];
            tileT[tid * DL + JM] = x;
            __syncthreads();
            if (oj >= 0) {
                const int64_t ne = m - t0 < DS_T ? m - t0 : DS_T;
                for (int i = 0; i < ne; ++i) acc.add_prod(tileT[i * DL + oj], tileT[i * DL + ok_]);
            }
            __syncthreads();
        }
        if (oj >= 0) sums[tid] = acc.value();
        __syncthreads();
        if (tid == 0) {
            double a[JM];
            if (m == 0 || !ds_solve<JM>(sums, p.lambda, a)) {
                for (int j = 0; j < JM; ++j) a[j] = 0.0;  // no entries: the zero row; not PD: zeroed and counted
                if (m > 0) atomicAdd(&p.flags[2], 1);
            }
            for (int j = 0; j < JM; ++j) {
                arow[j] = a[j];
                out[j] = (T)a[j];
            }
        }
        __syncthreads();
        // predictions: delta of the query coordinate for the mode, dotted with the new row
        T ar[JM];
#pragma unroll
        for (int j = 0; j < JM; ++j) ar[j] = (T)arow[j];
        for (int64_t e = tid; e < q; e += DS_T) {
            T d[JM];
            ds_rows<T>(p, qi + e * N, myrows);
            ds_delta<T, JM>(p, Gs, myrows, d);
            T s = T(0);
#pragma unroll
            for (int j = 0; j < JM; ++j) s = fma(ar[j], d[j], s);
            out[JM + e] = s;
        }
        __threadfence_system();  // results reach host memory before the done word
        __syncthreads();
        if (tid == 0) {
            atomicAdd(&p.flags[1], 1);
            *(volatile unsigned long long*)(p.done + claimed % p.ring) = (unsigned long long)claimed + 1;
            __threadfence_system();
        }
        (void)mode;
    }
}

}  // namespace
}  // namespace ptk

namespace ptk {
namespace {

using DsClock = std::chrono::steady_clock;

struct DsReq {
    uint64_t ticket = 0;
    int64_t m = 0, q = 0;
    std::vector<int32_t> obs_idx, query_idx;
    std::vector<uint8_t> obs_vals;
    DsClock::time_point arrival;
    int64_t seq = -1;            // ring sequence once admitted
    int64_t arena_off = 0, arena_bytes = 0;
    bool done = false;
    double latency_ms = 0.0;
    std::vector<uint8_t> row, preds;
};

}  // namespace
}  // namespace ptk

struct ptk_dserver {
    ptk_model model{};
    ptk_dserver_opts opts{};
    int device = 0;
    size_t esz = 4;
    int J = 0;
    int workers = 0;
    size_t smem = 0;
    // device
    void* Gp = nullptr;
    unsigned long long* head = nullptr;
    int* flags = nullptr;
    cudaStream_t stream = nullptr;
    cudaEvent_t ev = nullptr;
    bool launched = false;
    // mapped pinned host memory
    ptk::DsCtrl* ctrl = nullptr;
    ptk::DsDesc* desc = nullptr;
    unsigned long long* done = nullptr;
    uint8_t* arena = nullptr;
    uint8_t* results = nullptr;
    ptk::DsParams params{};
    // host bookkeeping
    std::mutex mu;
    std::deque<uint64_t> pending;                        // admitted later, in arrival order
    std::deque<uint64_t> inflight;                       // in ring order
    std::unordered_map<uint64_t, ptk::DsReq> reqs;
    uint64_t next_ticket = 1;
    int64_t published = 0;                               // == tail
    int64_t arena_head = 0, arena_tail = 0;              // byte ring [tail, head)
    int64_t max_q = 0;
    ptk_dserver_stats stats{};
    std::atomic<bool> stop{false};
    std::thread poller;
    ptk_status status = PTK_OK;
    char error[256] = "";
};

namespace ptk {
namespace {

int64_t ds_align(int64_t x) { return (x + 255) / 256 * 256; }

int64_t ds_bytes(const ptk_dserver* s, int64_t m, int64_t q) {
    const int N = s->model.order;
    return ds_align(sizeof(int32_t) * N * m) + ds_align((int64_t)s->esz * m) + ds_align(sizeof(int32_t) * N * q);
}

template <typename T, int JM>
ptk_status ds_launch_t(ptk_dserver* s) {
    auto kern = dserve_kernel<T, JM>;
    PTK_CUDA(cudaFuncSetAttribute((const void*)kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)s->smem));
    kern<<<s->workers, DS_T, s->smem, s->stream>>>(s->params);
    note_launch();
    PTK_CUDA(cudaGetLastError());
    PTK_CUDA(cudaEventRecord(s->ev, s->stream));
    s->launched = true;
    s->stats.launches += 1;
    return PTK_OK;
}

template <typename T>
ptk_status ds_launch_j(ptk_dserver* s) {
    switch (s->J) {
#define PTK_CASE(JJ) \
    case JJ:         \
        return ds_launch_t<T, JJ>(s);
        PTK_CASE(1) PTK_CASE(2) PTK_CASE(3) PTK_CASE(4) PTK_CASE(5) PTK_CASE(6) PTK_CASE(7) PTK_CASE(8)
        PTK_CASE(9) PTK_CASE(10) PTK_CASE(11) PTK_CASE(12) PTK_CASE(13) PTK_CASE(14) PTK_CASE(15) PTK_CASE(16)
#undef PTK_CASE
        default:
            set_error("device-loop server: J=%d unsupported", s->J);
            return PTK_ERR_UNSUPPORTED;
    }
}

// the loop is running or has been relaunched (caller holds s->mu)
ptk_status ds_ensure_running(ptk_dserver* s) {
    if (s->launched) {
        const cudaError_t e = cudaEventQuery(s->ev);
        if (e == cudaErrorNotReady) return PTK_OK;
        if (e != cudaSuccess) {
            set_error("device-loop server: %s", cudaGetErrorString(e));
            return PTK_ERR_CUDA;
        }
        s->launched = false;
    }
    return s->model.dtype == PTK_F64 ? ds_launch_j<double>(s) : ds_launch_j<float>(s);
}

// admits pending requests in arrival order while the ring and the arena have
// room, and publishes them (caller holds s->mu)
void ds_admit(ptk_dserver* s) {
    const int N = s->model.order;
    const int64_t cap = s->opts.arena_bytes;
    bool any = false;
    while (!s->pending.empty()) {
        DsReq& r = s->reqs[s->pending.front()];
        if (s->published - (int64_t)s->stats.completed >= s->opts.ring) break;  // ring full
        const int64_t need = ds_bytes(s, r.m, r.q);
        // arena ring [arena_tail, arena_head): take the next need bytes, wrapping to 0 if the end is short
        int64_t off = s->arena_head % cap;
        int64_t skip = 0;
        if (off + need > cap) {
            skip = cap - off;
            off = 0;
        }
        if (s->arena_head + skip + need - s->arena_tail > cap) break;  // not enough free bytes yet
        r.arena_off = s->arena_head + skip;
        r.arena_bytes = need + skip;
        s->arena_head += skip + need;
        uint8_t* base = s->arena + off;
        const int64_t oi = 0, ov = ds_align(sizeof(int32_t) * N * r.m), qi = ov + ds_align((int64_t)s->esz * r.m);
        std::memcpy(base + oi, r.obs_idx.data(), sizeof(int32_t) * N * r.m);
        std::memcpy(base + ov, r.obs_vals.data(), s->esz * r.m);
        std::memcpy(base + qi, r.query_idx.data(), sizeof(int32_t) * N * r.q);
        r.seq = s->published;
        DsDesc& d = s->desc[r.seq % s->opts.ring];
        d.seq = r.seq;
        d.m = r.m;
        d.q = r.q;
        d.obs_off = off + oi;
        d.val_off = off + ov;
        d.qry_off = off + qi;
        d.res_off = (r.seq % s->opts.ring) * (int64_t)ds_align((int64_t)s->esz * (s->J + s->max_q));
        s->done[r.seq % s->opts.ring] = 0;
        s->inflight.push_back(r.ticket);
        s->pending.pop_front();
        s->published += 1;
        any = true;
    }
    if (any) {
        std::atomic_thread_fence(std::memory_order_seq_cst);  // request data and descriptors before the tail
        s->ctrl->tail = (unsigned long long)s->published;
        std::atomic_thread_fence(std::memory_order_seq_cst);
    }
}

// collects finished requests (in ring order: the arena is freed in order)
void ds_collect(ptk_dserver* s) {
    const int64_t rb = ds_align((int64_t)s->esz * (s->J + s->max_q));
    while (!s->inflight.empty()) {
        DsReq& r = s->reqs[s->inflight.front()];
        const unsigned long long w = *(volatile unsigned long long*)(s->done + r.seq % s->opts.ring);
        if (w != (unsigned long long)r.seq + 1) break;
        std::atomic_thread_fence(std::memory_order_acquire);
        const uint8_t* res = s->results + (r.seq % s->opts.ring) * rb;
        r.row.assign(res, res + s->esz * s->J);
        r.preds.assign(res + s->esz * s->J, res + s->esz * (s->J + r.q));
        r.done = true;
        r.latency_ms = std::chrono::duration<double, std::milli>(DsClock::now() - r.arrival).count();
        s->arena_tail = r.arena_off + ds_bytes(s, r.m, r.q);  // freed in publication order
        s->stats.completed += 1;
        s->inflight.pop_front();
    }
}

void ds_poller(ptk_dserver* s) {
    cudaSetDevice(s->device);
    while (!s->stop.load()) {
        {
            std::lock_guard<std::mutex> lock(s->mu);
            ds_collect(s);
            ds_admit(s);
            if ((int64_t)s->stats.completed < s->published && s->status == PTK_OK) {
                const ptk_status rc = ds_ensure_running(s);
                if (rc != PTK_OK) {
                    s->status = rc;
                    std::snprintf(s->error, sizeof(s->error), "%s", get_error());
                }
            }
        }
        std::this_thread::sleep_for(std::chrono::microseconds(5));
    }
}

}  // namespace
}  // namespace ptk

using namespace ptk;

static void ds_free(ptk_dserver* s) {
    if (!s) return;
    cudaSetDevice(s->device);
    if (s->poller.joinable()) {
        s->stop.store(true);
        s->poller.join();
    }
    if (s->ctrl) s->ctrl->stop = 1;
    if (s->stream) cudaStreamSynchronize(s->stream);  // the loop leaves at its next poll
    if (s->ev) cudaEventDestroy(s->ev);
    if (s->stream) cudaStreamDestroy(s->stream);
    cudaFree(s->Gp);
    cudaFree(s->head);
    cudaFree(s->flags);
    if (s->ctrl) cudaFreeHost(s->ctrl);
    if (s->desc) cudaFreeHost(s->desc);
    if (s->done) cudaFreeHost(s->done);
    if (s->arena) cudaFreeHost(s->arena);
    if (s->results) cudaFreeHost(s->results);
    delete s;
}

namespace {
// the core permuted for the mode: Gp[j][r], r over the other modes in C order
template <typename T>
void ds_permute(const ptk_model* m, int mode, const std::vector<T>& G, std::vector<T>& Gp) {
    const int N = m->order;
    int64_t size = 1;
    for (int k = 0; k < N; ++k) size *= m->J[k];
    const int64_t R = size / m->J[mode];
    Gp.assign(size, T(0));
    std::vector<int> idx(N, 0);
    for (int64_t b = 0; b < size; ++b) {
        int64_t r = 0;
        for (int k = 0; k < N; ++k)
            if (k != mode) r = r * m->J[k] + idx[k];
        Gp[(int64_t)idx[mode] * R + r] = G[b];
        for (int k = N - 1; k >= 0; --k) {
            if (++idx[k] < m->J[k]) break;
            idx[k] = 0;
        }
    }
}
}  // namespace

extern "C" ptk_status ptk_dserver_create(const ptk_model* m, int device, const ptk_dserver_opts* o,
                                         ptk_dserver** out) {
    PTK_CHECK_ARG(m && o && out, "null argument");
    *out = nullptr;
    PTK_TRY(check_model(m));
    PTK_CHECK_ARG(o->mode >= 0 && o->mode < m->order, "mode out of range");
    PTK_CHECK_ARG(m->order >= 2, "order must be >= 2");
    PTK_CHECK_ARG(o->lambda > 0.0, "lambda must be > 0");
    PTK_CHECK_ARG(o->ring >= 1 && o->ring <= (1 << 16), "ring out of [1, 65536]");
    PTK_CHECK_ARG(o->arena_bytes >= 4096, "arena too small");
    PTK_CHECK_ARG(o->max_queries >= 0 && o->max_queries <= (1 << 20), "max_queries out of range");
    PTK_CHECK_ARG(o->idle_ms > 0.0 && o->idle_ms <= 60000.0, "idle_ms out of (0, 60000]");
    PTK_CUDA(cudaSetDevice(device));
    ptk_dserver* s = new (std::nothrow) ptk_dserver();
    if (!s) {
        set_error("out of host memory");
        return PTK_ERR_OUT_OF_MEMORY;
    }
    s->model = *m;
    s->opts = *o;
    s->device = device;
    s->esz = dtype_size(m->dtype);
    s->J = m->J[o->mode];
    s->max_q = o->max_queries;
    auto fail = [&](ptk_status rc) {
        ds_free(s);
        return rc;
    };
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) return fail(PTK_ERR_CUDA);
    s->workers = o->workers > 0 ? std::min(o->workers, sms) : sms;
    // shared memory: permuted core, a row buffer per thread, a tile of delta rows
    const int N = m->order, mode = o->mode;
    int64_t size = 1;
    for (int k = 0; k < N; ++k) size *= m->J[k];
    DsParams& p = s->params;
    p.order = N;
    p.mode = mode;
    p.J = s->J;
    int sr = 0, no = 0;
    for (int k = 0; k < N; ++k) {
        if (k == mode) continue;
        p.others[no] = k;
        p.Jo[no] = m->J[k];
        p.factors[k] = m->factors[k];
        p.ld[k] = m->ld[k];
        p.rowoff[no] = sr;
        sr += m->J[k];
        ++no;
    }
    p.sr = sr | 1;
    p.R = size / s->J;
    s->smem = s->esz * ((size_t)size + (size_t)DS_T * p.sr + (size_t)DS_T * (s->J + 1));
    int optin = 0;
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, device);
    if (s->smem + 4096 > (size_t)optin) {
        set_error("device-loop server: the core and row buffers need %zu bytes of shared memory", s->smem);
        return fail(PTK_ERR_UNSUPPORTED);
    }
    // permuted core
    std::vector<uint8_t> Gh(size * s->esz);
    if (cudaMemcpy(Gh.data(), m->core, Gh.size(), cudaMemcpyDeviceToHost) != cudaSuccess) return fail(PTK_ERR_CUDA);
    std::vector<uint8_t> Gph(Gh.size());
    if (m->dtype == PTK_F64) {
        std::vector<double> G(size), Gp;
        std::memcpy(G.data(), Gh.data(), Gh.size());
        ds_permute<double>(m, mode, G, Gp);
        std::memcpy(Gph.data(), Gp.data(), Gph.size());
    } else {
        std::vector<float> G(size), Gp;
        std::memcpy(G.data(), Gh.data(), Gh.size());
        ds_permute<float>(m, mode, G, Gp);
        std::memcpy(Gph.data(), Gp.data(), Gph.size());
    }
    if (cudaMalloc(&s->Gp, Gph.size()) != cudaSuccess || cudaMalloc(&s->head, sizeof(unsigned long long)) != cudaSuccess ||
        cudaMalloc(&s->flags, sizeof(int) * 4) != cudaSuccess) {
        cudaGetLastError();
        set_error("device-loop server: device allocation failed");
        return fail(PTK_ERR_OUT_OF_MEMORY);
    }
    if (cudaMemcpy(s->Gp, Gph.data(), Gph.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemset(s->head, 0, sizeof(unsigned long long)) != cudaSuccess ||
        cudaMemset(s->flags, 0, sizeof(int) * 4) != cudaSuccess)
        return fail(PTK_ERR_CUDA);
    // mapped pinned host memory: control words, ring, done words, arena, results
    const size_t rb = (size_t)ds_align((int64_t)s->esz * (s->J + s->max_q));
    auto host = [&](void** ptr, size_t bytes) -> bool {
        if (cudaHostAlloc(ptr, bytes, cudaHostAllocMapped) != cudaSuccess) {
            cudaGetLastError();
            return false;
        }
        std::memset(*ptr, 0, bytes);
        return true;
    };
    if (!host((void**)&s->ctrl, sizeof(DsCtrl)) || !host((void**)&s->desc, sizeof(DsDesc) * o->ring) ||
        !host((void**)&s->done, sizeof(unsigned long long) * o->ring) ||
        !host((void**)&s->arena, (size_t)o->arena_bytes) || !host((void**)&s->results, rb * o->ring)) {
        set_error("device-loop server: pinned host allocation failed");
        return fail(PTK_ERR_OUT_OF_MEMORY);
    }
    void *dctrl, *ddesc, *ddone, *darena, *dres;
    if (cudaHostGetDevicePointer(&dctrl, s->ctrl, 0) != cudaSuccess ||
        cudaHostGetDevicePointer(&ddesc, s->desc, 0) != cudaSuccess ||
        cudaHostGetDevicePointer(&ddone, s->done, 0) != cudaSuccess ||
        cudaHostGetDevicePointer(&darena, s->arena, 0) != cudaSuccess ||
        cudaHostGetDevicePointer(&dres, s->results, 0) != cudaSuccess)
        return fail(PTK_ERR_CUDA);
    p.Gp = s->Gp;
    p.lambda = o->lambda;
    p.ring = o->ring;
    p.ctrl = (const DsCtrl*)dctrl;
    p.desc = (const DsDesc*)ddesc;
    p.done = (unsigned long long*)ddone;
    p.arena = (const uint8_t*)darena;
    p.results = (uint8_t*)dres;
    p.head = s->head;
    p.flags = s->flags;
    p.idle_ns = (long long)(o->idle_ms * 1e6);
    if (cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&s->ev, cudaEventDisableTiming) != cudaSuccess)
        return fail(PTK_ERR_CUDA);
    s->poller = std::thread(ds_poller, s);
    *out = s;
    return PTK_OK;
}

extern "C" ptk_status ptk_dserver_submit(ptk_dserver* s, const int32_t* obs_idx_h, const void* obs_vals_h, int64_t m,
                                         const int32_t* query_idx_h, int64_t q, double arrival_s, uint64_t* ticket) {
    PTK_CHECK_ARG(s && ticket, "null argument");
    PTK_CHECK_ARG(m >= 0 && q >= 0 && q <= s->max_q, "q out of [0, max_queries]");
    PTK_CHECK_ARG(m == 0 || (obs_idx_h && obs_vals_h), "null observed arrays");
    PTK_CHECK_ARG(q == 0 || query_idx_h, "null query array");
    const int N = s->model.order;
    for (int64_t e = 0; e < m; ++e)
        for (int k = 0; k < N; ++k)
            if (k != s->opts.mode)
                PTK_CHECK_ARG(obs_idx_h[e * N + k] >= 0 && obs_idx_h[e * N + k] < s->model.dims[k],
                              "observed coordinate out of range");
    for (int64_t e = 0; e < q; ++e)
        for (int k = 0; k < N; ++k)
            if (k != s->opts.mode)
                PTK_CHECK_ARG(query_idx_h[e * N + k] >= 0 && query_idx_h[e * N + k] < s->model.dims[k],
                              "query coordinate out of range");
    if (ds_bytes(s, m, q) > s->opts.arena_bytes) {
        set_error("request of %lld bytes exceeds the arena", (long long)ds_bytes(s, m, q));
        return PTK_ERR_BUSY;
    }
    std::lock_guard<std::mutex> lock(s->mu);
    if (s->status != PTK_OK) {
        set_error("%s", s->error);
        return s->status;
    }
    if ((int64_t)s->pending.size() >= s->opts.max_pending) {
        s->stats.rejected += 1;
        set_error("pending queue full");
        return PTK_ERR_BUSY;
    }
    DsReq r;
    r.ticket = s->next_ticket++;
    r.m = m;
    r.q = q;
    r.obs_idx.assign(obs_idx_h, obs_idx_h + N * m);
    r.obs_vals.assign((const uint8_t*)obs_vals_h, (const uint8_t*)obs_vals_h + s->esz * m);
    r.query_idx.assign(query_idx_h, query_idx_h + N * q);
    // the request's arrival: now, or the caller's time on the same steady clock (seconds)
    r.arrival = arrival_s > 0.0 ? DsClock::time_point(std::chrono::duration_cast<DsClock::duration>(
                                      std::chrono::duration<double>(arrival_s)))
                                : DsClock::now();
    *ticket = r.ticket;
    s->pending.push_back(r.ticket);
    s->reqs.emplace(r.ticket, std::move(r));
    s->stats.submitted += 1;
    ds_admit(s);
    return PTK_OK;
}

extern "C" ptk_status ptk_dserver_poll(ptk_dserver* s, uint64_t ticket, void* row_h, void* preds_h, int32_t* done,
                                       double* latency_ms) {
    PTK_CHECK_ARG(s && done, "null argument");
    std::lock_guard<std::mutex> lock(s->mu);
    auto it = s->reqs.find(ticket);
    PTK_CHECK_ARG(it != s->reqs.end(), "unknown ticket");
    DsReq& r = it->second;
    if (!r.done) {
        *done = 0;
        if (s->status != PTK_OK) {
            set_error("%s", s->error);
            return s->status;
        }
        return PTK_OK;
    }
    if (row_h) std::memcpy(row_h, r.row.data(), r.row.size());
    if (preds_h && !r.preds.empty()) std::memcpy(preds_h, r.preds.data(), r.preds.size());
    if (latency_ms) *latency_ms = r.latency_ms;
    *done = 1;
    s->reqs.erase(it);
    return PTK_OK;
}

extern "C" double ptk_clock_seconds(void) {
    return std::chrono::duration<double>(DsClock::now().time_since_epoch()).count();
}

extern "C" ptk_status ptk_dserver_read_stats(ptk_dserver* s, ptk_dserver_stats* out_h) {
    PTK_CHECK_ARG(s && out_h, "null argument");
    int f[4] = {0, 0, 0, 0};
    std::lock_guard<std::mutex> lock(s->mu);
    PTK_CUDA(cudaMemcpy(f, s->flags, sizeof(f), cudaMemcpyDeviceToHost));
    s->stats.idle_exits = f[0];
    s->stats.served_on_device = f[1];
    s->stats.bad_rows = f[2];
    s->stats.pending = (int64_t)s->pending.size();
    s->stats.inflight = (int64_t)s->inflight.size();
    s->stats.running = s->launched && cudaEventQuery(s->ev) == cudaErrorNotReady ? 1 : 0;
    cudaGetLastError();
    *out_h = s->stats;
    return PTK_OK;
}

extern "C" void ptk_dserver_destroy(ptk_dserver* s) { ds_free(s); }
