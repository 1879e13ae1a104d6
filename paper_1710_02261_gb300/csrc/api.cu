// api.cu -- the C ABI of libptk (declared in include/ptk.h): argument checks,
// scratch management and the order of kernel launches for each call.
#include "common.cuh"

#include <new>

namespace ptk {

static thread_local char g_err[512] = "";
std::atomic<int64_t> g_launches{0};

void set_error(const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof g_err, fmt, ap);
    va_end(ap);
}
const char* get_error() { return g_err; }

void* scratch(ptk_ctx* ctx, int slot, size_t bytes) {
    bytes += 256;  // slack: bulk copies round their sizes up to 16 bytes
    if (ctx->slot_bytes[slot] >= bytes) return ctx->slot_ptr[slot];
    if (ctx->in_capture) {  // the uncaptured run before a capture sizes every slot
        set_error("scratch slot %d would grow during graph capture", slot);
        return nullptr;
    }
    if (ctx->slot_ptr[slot]) {
        cudaFree(ctx->slot_ptr[slot]);  // synchronises: no launch still uses it
        ctx->slot_ptr[slot] = nullptr;
        ctx->slot_bytes[slot] = 0;
    }
    size_t want = bytes + bytes / 8;
    void* p = nullptr;
    if (cudaMalloc(&p, want) != cudaSuccess) {
        cudaGetLastError();
        set_error("scratch allocation of %zu bytes failed", want);
        return nullptr;
    }
    ctx->slot_ptr[slot] = p;
    ctx->slot_bytes[slot] = want;
    return p;
}

ptk_status check_model(const ptk_model* m) {
    PTK_CHECK_ARG(m != nullptr, "model is null");
    PTK_CHECK_ARG(m->order >= 2 && m->order <= PTK_MAX_ORDER, "order %d out of [2, %d]", m->order, PTK_MAX_ORDER);
    PTK_CHECK_ARG(m->dtype == PTK_F32 || m->dtype == PTK_F64, "bad model dtype");
    PTK_CHECK_ARG(m->core != nullptr, "core is null");
    for (int n = 0; n < m->order; ++n) {
        PTK_CHECK_ARG(m->J[n] >= 1 && m->J[n] <= PTK_MAX_RANK, "J[%d]=%d out of [1, %d]", n, m->J[n], PTK_MAX_RANK);
        PTK_CHECK_ARG(m->dims[n] >= 1 && m->dims[n] < (1ll << 31), "dims[%d] out of range", n);
        PTK_CHECK_ARG(m->ld[n] >= m->J[n], "ld[%d] < J[%d]", n, n);
        PTK_CHECK_ARG(m->factors[n] != nullptr, "factor %d is null", n);
    }
    return PTK_OK;
}

ptk_status check_coo(const ptk_coo* x, const ptk_model* m) {
    PTK_CHECK_ARG(x != nullptr, "coo is null");
    PTK_CHECK_ARG(x->order == m->order, "coo order %d != model order %d", x->order, m->order);
    PTK_CHECK_ARG(x->nnz >= 0 && x->nnz < (1ll << 31), "nnz out of range");
    PTK_CHECK_ARG(x->nnz == 0 || (x->idx && x->vals), "coo arrays are null");
    for (int n = 0; n < x->order; ++n) PTK_CHECK_ARG(x->dims[n] == m->dims[n], "dims[%d] differ", n);
    return PTK_OK;
}

static int64_t core_size(const ptk_model* m) {
    int64_t s = 1;
    for (int n = 0; n < m->order; ++n) s *= m->J[n];
    return s;
}

static ptk_status read_flags(ptk_ctx* ctx, cudaStream_t st, int* flags_h) {
    PTK_CUDA(cudaMemcpyAsync(flags_h, ctx->d_flags, sizeof(int) * FLAG_COUNT, cudaMemcpyDeviceToHost, st));
    PTK_CUDA(cudaStreamSynchronize(st));
    return PTK_OK;
}

// Copies the device-side results of the last sweep's error pass to the host
// (synchronises `st`) and turns the status words into a status code.
static ptk_status read_last_stats(ptk_ctx* ctx, ptk_sweep_stats* stats, cudaStream_t st) {
    PTK_CUDA(cudaMemcpyAsync(ctx->h_stats, ctx->d_stats, sizeof(double) * 16, cudaMemcpyDeviceToHost, st));
    PTK_TRY(read_flags(ctx, st, ctx->h_flags));
    const double* h = ctx->h_stats;
    double reg = 0.0;
    for (int n = 0; n < ctx->last_order; ++n) reg += h[1 + n];
    const int64_t E = ctx->last_nnz;
    stats->sse = h[0];
    stats->error = sqrt(h[0]);
    stats->rmse = E > 0 ? sqrt(h[0] / (double)E) : 0.0;
    stats->loss = h[0] + ctx->last_lambda * reg;
    stats->core_nnz = (int64_t)h[12];
    stats->bad_rows = ctx->h_flags[FLAG_BAD_ROWS];
    if (ctx->h_flags[FLAG_TIMEOUT]) {
        set_error("a bounded device wait gave up (%d)", ctx->h_flags[FLAG_TIMEOUT]);
        return PTK_ERR_TIMEOUT;
    }
    if (ctx->h_flags[FLAG_SPARSE]) {
        set_error("the core's non-zeros changed between their count and the sparse delta");
        return PTK_ERR_INVALID_ARG;
    }
    if (stats->bad_rows) {
        set_error("%lld row systems were not positive definite", (long long)stats->bad_rows);
        return PTK_ERR_NUMERIC;
    }
    return PTK_OK;
}

// Values of `x` in the compute type; converts into scratch when they differ.
static ptk_status vals_as(ptk_ctx* ctx, const ptk_coo* x, ptk_dtype want, int slot, const void** out,
                          cudaStream_t st);

__global__ void convert_vals(const void* in, int in_f64, void* out, int out_f64, int64_t n) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
        double v = in_f64 ? ((const double*)in)[e] : (double)((const float*)in)[e];
        if (out_f64)
            ((double*)out)[e] = v;
        else
            ((float*)out)[e] = (float)v;
    }
}

static ptk_status vals_as(ptk_ctx* ctx, const ptk_coo* x, ptk_dtype want, int slot, const void** out,
                          cudaStream_t st) {
    if (x->dtype == want) {
        *out = x->vals;
        return PTK_OK;
    }
    void* buf = scratch(ctx, slot, dtype_size(want) * (size_t)x->nnz);
    if (!buf) return PTK_ERR_OUT_OF_MEMORY;
    int g = (int)std::min<int64_t>(ceil_div(std::max<int64_t>(x->nnz, 1), 256), ctx->sm_count * 16);
    { convert_vals<<<g, 256, 0, st>>>(x->vals, x->dtype == PTK_F64, buf, want == PTK_F64, x->nnz); ::ptk::note_launch(); }
    PTK_LAUNCH_CHECK();
    *out = buf;
    return PTK_OK;
}

DeltaJob make_job(const ptk_model* m, int mode, int64_t n) {
    DeltaJob j;
    j.n = n;
    j.order = m->order;
    j.mode = mode;
    for (int k = 0; k < m->order; ++k) {
        j.factors[k] = m->factors[k];
        j.ld[k] = m->ld[k];
        j.J[k] = m->J[k];
    }
    j.core = m->core;
    j.dtype = m->dtype;
    j.out_ld = delta_out_ld(m->J[mode]);
    return j;
}

// Fold-in padding: an observed entry whose mode column is -1 contributes
// nothing, so its Delta row (delta and x) is zeroed.
__global__ void zero_pad_rows(void* delta, int ld, int f64, const int32_t* __restrict__ idx, int order, int mode,
                              int64_t n) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
        if (idx[e * order + mode] != -1) continue;
        for (int j = 0; j < ld; ++j) {
            if (f64)
                ((double*)delta)[e * ld + j] = 0.0;
            else
                ((float*)delta)[e * ld + j] = 0.f;
        }
    }
}

// rid[e] = request r with ptr[r] <= e < ptr[r+1] (binary search)
__global__ void rid_from_ptr(const int64_t* __restrict__ ptr, int count, int64_t n, int32_t* __restrict__ rid) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
        int lo = 0, hi = count - 1;
        while (lo < hi) {
            int mid = (lo + hi + 1) >> 1;
            if (ptr[mid] <= e)
                lo = mid;
            else
                hi = mid - 1;
        }
        rid[e] = lo;
    }
}

}  // namespace ptk

using namespace ptk;

namespace {
template <typename T>
__global__ void count_nonzero(const T* __restrict__ g, int64_t n, unsigned long long* __restrict__ out) {
    unsigned long long c = 0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        c += g[i] != T(0);
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) c += __shfl_down_sync(0xffffffffu, c, off);
    if ((threadIdx.x & 31) == 0 && c) atomicAdd(out, c);
}
}  // namespace

extern "C" {

const char* ptk_last_error(void) { return get_error(); }
const char* ptk_version(void) { return "ptk 0.1 (sm_103a)"; }

int64_t ptk_launch_count(void) { return g_launches.load(); }

ptk_status ptk_set_timing(ptk_ctx* ctx, int32_t enable) {
    PTK_CHECK_ARG(ctx != nullptr, "null context");
    ctx->timing = enable ? 1 : 0;
    return PTK_OK;
}

ptk_status ptk_read_timers(ptk_ctx* ctx, double* ms_h, int64_t* launches_h, int64_t* groups_h) {
    PTK_CHECK_ARG(ctx != nullptr, "null context");
    PTK_CUDA(cudaSetDevice(ctx->device));
    for (auto& r : ctx->pending) {
        float ms = 0.f;
        if (cudaEventSynchronize(r.e1) == cudaSuccess && cudaEventElapsedTime(&ms, r.e0, r.e1) == cudaSuccess) {
            ctx->acc_ms[r.id] += ms;
            ctx->acc_groups[r.id] += 1;
        }
        cudaEventDestroy(r.e0);
        cudaEventDestroy(r.e1);
    }
    ctx->pending.clear();
    for (int i = 0; i < PTK_T_COUNT; ++i) {
        if (ms_h) ms_h[i] = ctx->acc_ms[i];
        if (launches_h) launches_h[i] = ctx->acc_launch[i];
        if (groups_h) groups_h[i] = ctx->acc_groups[i];
        ctx->acc_ms[i] = 0.0;
        ctx->acc_launch[i] = 0;
        ctx->acc_groups[i] = 0;
    }
    return PTK_OK;
}

ptk_status ptk_create(ptk_ctx** out, int device) {
    PTK_CHECK_ARG(out != nullptr, "ptk_create: out is null");
    *out = nullptr;
    int ndev = 0;
    PTK_CUDA(cudaGetDeviceCount(&ndev));
    PTK_CHECK_ARG(device >= 0 && device < ndev, "device %d not present (%d devices)", device, ndev);
    PTK_CUDA(cudaSetDevice(device));
    ptk_ctx* c = new (std::nothrow) ptk_ctx();
    if (!c) {
        set_error("out of host memory");
        return PTK_ERR_OUT_OF_MEMORY;
    }
    c->device = device;
    cudaDeviceProp prop;
    PTK_CUDA(cudaGetDeviceProperties(&prop, device));
    c->sm_count = prop.multiProcessorCount;
    c->smem_optin = prop.sharedMemPerBlockOptin;
    if (prop.major < 10) {
        delete c;
        set_error("libptk needs a Blackwell GPU (sm_103a); device %d is sm_%d%d", device, prop.major, prop.minor);
        return PTK_ERR_UNSUPPORTED;
    }
    PTK_CUDA(cudaMalloc(&c->d_flags, sizeof(int) * FLAG_COUNT));
    PTK_CUDA(cudaMemset(c->d_flags, 0, sizeof(int) * FLAG_COUNT));
    PTK_CUDA(cudaMalloc(&c->d_stats, sizeof(double) * 32));
    PTK_CUDA(cudaMallocHost(&c->h_stats, sizeof(double) * 32));
    PTK_CUDA(cudaMallocHost(&c->h_flags, sizeof(int) * FLAG_COUNT));
    // side stream for kernels that run beside the main one (forked and joined with events)
    PTK_CUDA(cudaStreamCreateWithFlags(&c->side, cudaStreamNonBlocking));
    PTK_CUDA(cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming));
    PTK_CUDA(cudaEventCreateWithFlags(&c->ev_join, cudaEventDisableTiming));
    {
        cudaMemPoolProps props;
        std::memset(&props, 0, sizeof props);
        props.allocType = cudaMemAllocationTypePinned;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = device;
        if (cudaMemPoolCreate(&c->pool, &props) == cudaSuccess) {
            uint64_t keep = ~0ull;  // never hand cached blocks back to the driver on its own
            cudaMemPoolSetAttribute(c->pool, cudaMemPoolAttrReleaseThreshold, &keep);
        } else {
            cudaGetLastError();
            c->pool = nullptr;  // slice arrays then use plain allocations
        }
    }
    *out = c;
    return PTK_OK;
}

void ptk_destroy(ptk_ctx* c) {
    if (!c) return;
    cudaSetDevice(c->device);
    cudaDeviceSynchronize();
    for (auto& l : c->lanes) {
        ptk_destroy(l.second);
        cudaStreamDestroy(l.first);
    }
    for (int s = 0; s < SLOT_COUNT; ++s)
        if (c->slot_ptr[s]) cudaFree(c->slot_ptr[s]);
    // blocks still held by live slice layouts keep the pool alive until freed
    if (c->pool) cudaMemPoolDestroy(c->pool);
    cudaFree(c->d_flags);
    cudaFree(c->d_stats);
    cudaFreeHost(c->h_stats);
    cudaFreeHost(c->h_flags);
    if (c->ev_fork) cudaEventDestroy(c->ev_fork);
    if (c->ev_join) cudaEventDestroy(c->ev_join);
    if (c->side) cudaStreamDestroy(c->side);
    delete c;
}

ptk_status ptk_build_mode_slices(ptk_ctx* ctx, const ptk_coo* x, int32_t mode, ptk_dtype compute, ptk_slices** out,
                                 ptk_stream_t stream) {
    PTK_CHECK_ARG(ctx && x && out, "null argument");
    *out = nullptr;
    PTK_CHECK_ARG(x->order >= 2 && x->order <= PTK_MAX_ORDER, "order out of range");
    PTK_CHECK_ARG(mode >= 0 && mode < x->order, "mode %d out of range", mode);
    PTK_CHECK_ARG(x->nnz >= 0 && x->nnz < (1ll << 31), "nnz out of range");
    PTK_CHECK_ARG(x->nnz == 0 || (x->idx && x->vals), "coo arrays are null");
    PTK_CHECK_ARG(compute == PTK_F32 || compute == PTK_F64, "bad compute dtype");
    for (int k = 0; k < x->order; ++k) PTK_CHECK_ARG(x->dims[k] >= 1 && x->dims[k] < (1ll << 31), "bad dims");
    PTK_CUDA(cudaSetDevice(ctx->device));
    ptk_slices* s = new (std::nothrow) ptk_slices();
    if (!s) return PTK_ERR_OUT_OF_MEMORY;
    s->device = ctx->device;
    ptk_status rc;
    {
        TimerScope ts(ctx, PTK_T_SLICES, (cudaStream_t)stream);
        rc = build_slices_impl(ctx, x, mode, compute, s, (cudaStream_t)stream);
    }
    if (rc != PTK_OK) {
        ptk_slices_destroy(s);
        return rc;
    }
    *out = s;
    return PTK_OK;
}

void ptk_slices_destroy(ptk_slices* s) {
    if (!s) return;
    cudaSetDevice(s->device);
    if (s->pooled) {
        // no launch may still use the arrays (as with cudaFree); the blocks go
        // back to the context's pool for the next layout
        cudaDeviceSynchronize();
        void* ps[4 + PTK_MAX_ORDER] = {s->perm, s->row_ptr, s->vals, s->tc_plan};
        for (int k = 0; k < PTK_MAX_ORDER; ++k) ps[4 + k] = s->cols[k];
        for (void* p : ps)
            if (p) cudaFreeAsync(p, nullptr);
    } else {
        cudaFree(s->perm);
        cudaFree(s->row_ptr);
        for (int k = 0; k < PTK_MAX_ORDER; ++k) cudaFree(s->cols[k]);
        cudaFree(s->vals);
        cudaFree(s->tc_plan);
    }
    delete s;
}

ptk_status ptk_slices_view(const ptk_slices* s, const int32_t** perm, const int64_t** row_ptr, const int32_t** rid,
                           int64_t* nnz, int64_t* rows) {
    PTK_CHECK_ARG(s != nullptr, "slices is null");
    if (perm) *perm = s->perm;
    if (row_ptr) *row_ptr = s->row_ptr;
    if (rid) *rid = s->cols[s->mode];
    if (nnz) *nnz = s->nnz;
    if (rows) *rows = s->rows;
    return PTK_OK;
}

ptk_status ptk_slices_export(const ptk_slices* s, int32_t* perm_out, int64_t* row_ptr_out, ptk_stream_t stream) {
    PTK_CHECK_ARG(s != nullptr, "slices is null");
    PTK_CUDA(cudaSetDevice(s->device));
    if (perm_out && s->nnz > 0)
        PTK_CUDA(cudaMemcpyAsync(perm_out, s->perm, sizeof(int32_t) * (size_t)s->nnz, cudaMemcpyDeviceToDevice,
                                 (cudaStream_t)stream));
    if (row_ptr_out)
        PTK_CUDA(cudaMemcpyAsync(row_ptr_out, s->row_ptr, sizeof(int64_t) * (size_t)(s->rows + 1),
                                 cudaMemcpyDeviceToDevice, (cudaStream_t)stream));
    return PTK_OK;
}

// Alg. 3 for one mode n: delta of every entry of x (slice layout s of mode
// n), the row sums, and the solve of rows [row_lo, row_hi) of A^(n) (rows
// outside the range keep their values).  *delta_out / *ld_out: the Delta array.

// nnz(G) on the host (one small read; the core changes only between sweeps)
static ptk_status core_nonzeros(ptk_ctx* ctx, const ptk_model* m, cudaStream_t st, int64_t* nnz) {
    const int64_t n = core_size(m);
    auto* d = (unsigned long long*)scratch(ctx, SLOT_SPARSE, 64);
    if (!d) return PTK_ERR_OUT_OF_MEMORY;
    PTK_CUDA(cudaMemsetAsync(d, 0, sizeof(unsigned long long), st));
    const int g = (int)std::max<int64_t>(1, std::min<int64_t>(ceil_div(n, 256), (int64_t)ctx->sm_count * 4));
    if (m->dtype == PTK_F64)
        { count_nonzero<double><<<g, 256, 0, st>>>((const double*)m->core, n, d); ::ptk::note_launch(); }
    else
        { count_nonzero<float><<<g, 256, 0, st>>>((const float*)m->core, n, d); ::ptk::note_launch(); }
    PTK_LAUNCH_CHECK();
    unsigned long long h = 0;
    PTK_CUDA(cudaMemcpyAsync(&h, d, sizeof h, cudaMemcpyDeviceToHost, st));
    PTK_CUDA(cudaStreamSynchronize(st));
    *nnz = (int64_t)h;
    return PTK_OK;
}

// core_nnz: nnz(G) when known (Approx sweeps; the CUDA-core delta then walks
// the non-zeros where that is shorter), else -1
static ptk_status update_mode(ptk_ctx* ctx, const ptk_coo* x, const ptk_slices* s, ptk_model* m, int n,
                              const ptk_als_opts* o, float* pres, int64_t row_lo, int64_t row_hi, cudaStream_t st,
                              void** delta_out, int* ld_out, int64_t core_nnz = -1) {
    const int N = m->order;
    const int64_t E = x->nnz;
    const ptk_dtype dt = m->dtype;
    const size_t ts = dtype_size(dt);
    const int Jn = m->J[n];
    DeltaJob job = make_job(m, n, E);
    for (int k = 0; k < N; ++k) job.col[k] = s->cols[k];
    job.cstride = 1;
    job.vals = s->vals;
    job.padded = true;  // slice arrays are allocated with 16 bytes of slack
    job.core_nnz = core_nnz;
    void* delta = scratch(ctx, SLOT_DELTA, ts * (size_t)E * job.out_ld);
    if (!delta) return PTK_ERR_OUT_OF_MEMORY;
    job.out = delta;
    *delta_out = delta;
    *ld_out = job.out_ld;
    {
        TimerScope tdelta(ctx, o->variant == PTK_CACHE ? PTK_T_CACHE : PTK_T_DELTA, st);
        if (o->variant == PTK_CACHE) {
            PTK_TRY(cache_delta(ctx, x, s, m, pres, delta, job.out_ld, st));
        } else {
            PTK_TRY(delta_run(ctx, job, o->precision, st));
        }
    }
    const int nout = gram_nout(Jn);
    void* rowbuf = scratch(ctx, SLOT_ROWBUF, 8 * (size_t)m->dims[n] * nout);  // FP64 or (s, lo) FP32 pairs
    if (!rowbuf) return PTK_ERR_OUT_OF_MEMORY;
    GramJob gj;
    gj.n = E;
    gj.rows = m->dims[n];
    gj.J = Jn;
    gj.delta = delta;
    gj.ld = job.out_ld;
    gj.rid = s->cols[n];
    gj.row_ptr = s->row_ptr;
    gj.rowbuf = rowbuf;
    gj.dtype = dt;
    gj.schedule = o->schedule;
    gj.max_row = s->max_row;
    gj.tc_plan = s->tc_plan;
    gj.tc_nchunks = s->tc_nchunks;
    gj.tc_long_entries = s->tc_long_entries;
    // deltas from tensor-core products carry errors of 2^-16 (BF16x3) or more:
    // 21-bit digits suffice; FP32 deltas keep 28 bits
    const bool tc_prec = o->precision == PTK_PREC_TF32 || o->precision == PTK_PREC_BF16 ||
                         o->precision == PTK_PREC_BF16X3;
    gj.digits = tc_prec && o->variant != PTK_CACHE ? 3 : 4;
    int sums_f64 = dt == PTK_F64 ? 1 : 0;
    gj.wrote_f64 = &sums_f64;
    {
        TimerScope tg(ctx, PTK_T_GRAM, st);
        PTK_TRY(gram(ctx, gj, st));
    }
    void* aold = nullptr;
    if (o->variant == PTK_CACHE) {
        aold = scratch(ctx, SLOT_AOLD, ts * (size_t)m->dims[n] * m->ld[n]);
        if (!aold) return PTK_ERR_OUT_OF_MEMORY;
        PTK_CUDA(cudaMemcpyAsync(aold, m->factors[n], ts * (size_t)m->dims[n] * m->ld[n], cudaMemcpyDeviceToDevice,
                                 st));
    }
    if (row_hi > row_lo) {
        SolveJob sj;
        sj.rows = row_hi - row_lo;
        sj.J = Jn;
        sj.rowbuf = (const char*)rowbuf + 8 * (size_t)row_lo * nout;
        sj.buf_dtype = sums_f64 ? PTK_F64 : PTK_F32;
        sj.row_ptr = s->row_ptr + row_lo;
        sj.lambda = o->lambda;
        sj.out = (char*)m->factors[n] + ts * (size_t)row_lo * m->ld[n];
        sj.ld = m->ld[n];
        sj.out_dtype = dt;
        TimerScope tsv(ctx, PTK_T_SOLVE, st);
        PTK_TRY(solve_rows(ctx, sj, st));
    }
    if (o->variant == PTK_CACHE) {
        TimerScope tc(ctx, PTK_T_CACHE, st);
        PTK_TRY(cache_rescale(ctx, x, m, n, aold, pres, st));
    }
    return PTK_OK;
}

ptk_status ptk_als_sweep(ptk_ctx* ctx, const ptk_coo* x, ptk_slices* const* slices, ptk_model* m,
                         const ptk_als_opts* o, ptk_sweep_stats* stats, ptk_stream_t stream) {
    PTK_CHECK_ARG(ctx && x && slices && m && o, "null argument");
    PTK_TRY(check_model(m));
    PTK_TRY(check_coo(x, m));
    PTK_CHECK_ARG(o->lambda > 0.0, "lambda must be > 0");
    PTK_CHECK_ARG(o->variant >= PTK_PLAIN && o->variant <= PTK_APPROX, "bad variant");
    PTK_CHECK_ARG(o->precision >= PTK_PREC_FP64 && o->precision <= PTK_PREC_BF16X3, "bad precision");
    PTK_CHECK_ARG(o->schedule >= PTK_SCHED_AUTO && o->schedule <= PTK_SCHED_TENSOR, "bad schedule");
    if (o->precision == PTK_PREC_FP64 && m->dtype != PTK_F64) {
        set_error("PTK_PREC_FP64 needs a PTK_F64 model");
        return PTK_ERR_UNSUPPORTED;
    }
    if (o->precision != PTK_PREC_FP64 && m->dtype != PTK_F32) {
        set_error("FP32/TF32/BF16 precision needs a PTK_F32 model");
        return PTK_ERR_UNSUPPORTED;
    }
    if (o->variant == PTK_APPROX) PTK_CHECK_ARG(o->trunc_rate > 0.0 && o->trunc_rate < 1.0, "trunc_rate not in (0,1)");
    cudaStream_t st = (cudaStream_t)stream;
    PTK_CUDA(cudaSetDevice(ctx->device));
    const int N = m->order;
    const int64_t E = x->nnz;
    const ptk_dtype dt = m->dtype;
    const size_t ts = dtype_size(dt);
    for (int n = 0; n < N; ++n) {
        PTK_CHECK_ARG(slices[n] != nullptr, "slices[%d] is null", n);
        PTK_CHECK_ARG(slices[n]->mode == n && slices[n]->nnz == E && slices[n]->rows == m->dims[n],
                      "slices[%d] does not match the tensor", n);
        PTK_CHECK_ARG(slices[n]->dtype == dt, "slices[%d] were built for another dtype", n);
    }
    PTK_CUDA(cudaMemsetAsync(ctx->d_flags, 0, sizeof(int) * FLAG_COUNT, st));

    float* pres = nullptr;
    if (o->variant == PTK_CACHE) {
        if (dt != PTK_F32) {
            set_error("P-Tucker-Cache is implemented for the FP32 model only");
            return PTK_ERR_UNSUPPORTED;
        }
        size_t bytes = sizeof(float) * (size_t)E * (size_t)core_size(m);
        pres = (float*)scratch(ctx, SLOT_PRES, bytes);
        if (!pres) return PTK_ERR_OUT_OF_MEMORY;
        TimerScope tc(ctx, PTK_T_CACHE, st);
        PTK_TRY(cache_build(ctx, x, m, pres, st));
    }

    void* delta = nullptr;
    int last_ld = 0;
    int64_t core_nnz = -1;  // Approx truncates the core between sweeps: its non-zeros steer the delta
    if (o->variant == PTK_APPROX) PTK_TRY(core_nonzeros(ctx, m, st, &core_nnz));
    for (int n = 0; n < N; ++n)
        PTK_TRY(update_mode(ctx, x, slices[n], m, n, o, pres, 0, m->dims[n], st, &delta, &last_ld, core_nnz));

    const bool want_stats = stats != nullptr && o->error_pass;
    if (o->error_pass) {
        TimerScope te(ctx, PTK_T_ERROR, st);
        const ptk_slices* s = slices[N - 1];
        PTK_TRY(error_from_delta(ctx, delta, last_ld, m->J[N - 1], s->cols[N - 1], 1, E, m->factors[N - 1],
                                 m->ld[N - 1], dt, ctx->d_stats + 0, st));
        PTK_TRY(sumsq_factors(ctx, m, ctx->d_stats + 1, st));
    }
    if (o->variant == PTK_APPROX) {
        TimerScope ta(ctx, PTK_T_APPROX, st);
        UVSource src;  // residuals from the last mode's Delta (slice order), as the error pass took them
        src.delta = (const float*)delta;
        src.ld = last_ld;
        src.dmode = N - 1;
        for (int k = 0; k < N; ++k) src.col[k] = slices[N - 1]->cols[k];
        src.cstride = 1;
        // reused only when Delta was taken in FP32 on CUDA cores, as a fresh pass would be
        const bool fp32_delta = dt == PTK_F32 && o->variant != PTK_CACHE && o->precision == PTK_PREC_FP32;
        PTK_TRY(approx_truncate(ctx, x, m, o->trunc_rate, o->trunc_rule, st, fp32_delta ? &src : nullptr,
                                core_nnz));
    }
    if (o->error_pass) {
        TimerScope te(ctx, PTK_T_ERROR, st);
        PTK_TRY(count_nonzero(ctx, m->core, core_size(m), dt, ctx->d_stats + 12, st));
    }
    ctx->last_order = N;
    ctx->last_nnz = E;
    ctx->last_lambda = o->lambda;
    if (want_stats) return read_last_stats(ctx, stats, st);
    return PTK_OK;
}

ptk_status ptk_als_mode(ptk_ctx* ctx, const ptk_coo* x, const ptk_slices* s, ptk_model* m, int32_t mode,
                        int64_t row_lo, int64_t row_hi, const ptk_als_opts* o, ptk_stream_t stream) {
    PTK_CHECK_ARG(ctx && x && s && m && o, "null argument");
    PTK_TRY(check_model(m));
    PTK_TRY(check_coo(x, m));
    PTK_CHECK_ARG(mode >= 0 && mode < m->order, "mode out of range");
    PTK_CHECK_ARG(0 <= row_lo && row_lo <= row_hi && row_hi <= m->dims[mode], "row range out of [0, dims[mode]]");
    PTK_CHECK_ARG(o->lambda > 0.0, "lambda must be > 0");
    PTK_CHECK_ARG(o->precision >= PTK_PREC_FP64 && o->precision <= PTK_PREC_BF16X3, "bad precision");
    PTK_CHECK_ARG(o->schedule >= PTK_SCHED_AUTO && o->schedule <= PTK_SCHED_TENSOR, "bad schedule");
    PTK_CHECK_ARG(s->mode == mode && s->nnz == x->nnz && s->rows == m->dims[mode] && s->dtype == m->dtype,
                  "slices do not match the entries");
    if (o->variant != PTK_PLAIN) {
        set_error("ptk_als_mode: only the plain variant (Cache keys Pres by entry across modes; Approx is a "
                  "whole-sweep step)");
        return PTK_ERR_UNSUPPORTED;
    }
    if ((o->precision == PTK_PREC_FP64) != (m->dtype == PTK_F64)) {
        set_error("PTK_PREC_FP64 goes with a PTK_F64 model, the other precisions with PTK_F32");
        return PTK_ERR_UNSUPPORTED;
    }
    cudaStream_t st = (cudaStream_t)stream;
    PTK_CUDA(cudaSetDevice(ctx->device));
    PTK_CUDA(cudaMemsetAsync(ctx->d_flags, 0, sizeof(int) * FLAG_COUNT, st));
    void* delta = nullptr;
    int ld = 0;
    return update_mode(ctx, x, s, m, mode, o, nullptr, row_lo, row_hi, st, &delta, &ld);
}

ptk_status ptk_sweep_stats_read(ptk_ctx* ctx, ptk_sweep_stats* stats, ptk_stream_t stream) {
    PTK_CHECK_ARG(ctx && stats, "null argument");
    PTK_CUDA(cudaSetDevice(ctx->device));
    return read_last_stats(ctx, stats, (cudaStream_t)stream);
}

ptk_status ptk_error(ptk_ctx* ctx, const ptk_coo* x, const ptk_model* m, double lambda, ptk_sweep_stats* stats,
                     ptk_stream_t stream) {
    PTK_CHECK_ARG(ctx && x && m && stats, "null argument");
    PTK_TRY(check_model(m));
    PTK_TRY(check_coo(x, m));
    cudaStream_t st = (cudaStream_t)stream;
    PTK_CUDA(cudaSetDevice(ctx->device));
    const int N = m->order;
    const int64_t E = x->nnz;
    const size_t ts = dtype_size(m->dtype);
    const void* vals = nullptr;
    if (E > 0) {
        PTK_TRY(vals_as(ctx, x, m->dtype, SLOT_FOLD1, &vals, st));
        DeltaJob job = make_job(m, 0, E);
        for (int k = 0; k < N; ++k) job.col[k] = x->idx + k;
        job.cstride = N;
        job.vals = vals;
        void* delta = scratch(ctx, SLOT_DELTA, ts * (size_t)E * job.out_ld);
        if (!delta) return PTK_ERR_OUT_OF_MEMORY;
        job.out = delta;
        PTK_TRY(delta_simt(ctx, job, st));
        PTK_TRY(error_from_delta(ctx, delta, job.out_ld, m->J[0], x->idx, N, E, m->factors[0], m->ld[0], m->dtype,
                                 ctx->d_stats + 0, st));
    } else {
        PTK_CUDA(cudaMemsetAsync(ctx->d_stats, 0, sizeof(double), st));
    }
    PTK_TRY(sumsq_factors(ctx, m, ctx->d_stats + 1, st));
    PTK_CUDA(cudaMemcpyAsync(ctx->h_stats, ctx->d_stats, sizeof(double) * 16, cudaMemcpyDeviceToHost, st));
    PTK_CUDA(cudaStreamSynchronize(st));
    const double* h = ctx->h_stats;
    double reg = 0.0;
    for (int n = 0; n < N; ++n) reg += h[1 + n];
    stats->sse = h[0];
    stats->error = sqrt(h[0]);
    stats->rmse = E > 0 ? sqrt(h[0] / (double)E) : 0.0;
    stats->loss = h[0] + lambda * reg;
    stats->core_nnz = -1;
    stats->bad_rows = 0;
    return PTK_OK;
}

ptk_status ptk_delta(ptk_ctx* ctx, const ptk_model* m, int32_t mode, const int32_t* coords, int64_t n,
                     ptk_precision prec, void* out, ptk_stream_t stream) {
    PTK_CHECK_ARG(ctx && m, "null argument");
    PTK_TRY(check_model(m));
    PTK_CHECK_ARG(mode >= 0 && mode < m->order, "mode out of range");
    PTK_CHECK_ARG(n >= 0 && n < (1ll << 31), "n out of range");
    PTK_CHECK_ARG(prec >= PTK_PREC_FP64 && prec <= PTK_PREC_BF16X3, "bad precision");
    if (n == 0) return PTK_OK;
    PTK_CHECK_ARG(coords && out, "null arrays");
    if ((prec == PTK_PREC_FP64) != (m->dtype == PTK_F64)) {
        set_error("PTK_PREC_FP64 goes with a PTK_F64 model, the other precisions with PTK_F32");
        return PTK_ERR_UNSUPPORTED;
    }
    cudaStream_t st = (cudaStream_t)stream;
    PTK_CUDA(cudaSetDevice(ctx->device));
    DeltaJob job = make_job(m, mode, n);
    for (int k = 0; k < m->order; ++k) job.col[k] = coords + k;
    job.cstride = m->order;
    job.out = out;
    job.out_ld = m->J[mode];
    TimerScope td(ctx, PTK_T_DELTA, st);
    return delta_run(ctx, job, prec, st);
}

namespace {
// double-float (s, lo) pairs of the FP32 entry-tile sums -> FP64
__global__ void pairs_to_f64(const float2* __restrict__ in, double* __restrict__ out, int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = (double)in[i].x + (double)in[i].y;
}
}  // namespace

ptk_status ptk_row_sums(ptk_ctx* ctx, const void* delta, ptk_dtype dtype, int32_t ld, int32_t J, const int64_t* row_ptr,
                        const int32_t* rid, int64_t rows, int64_t nnz, ptk_schedule schedule, int32_t digits,
                        double* out, ptk_stream_t stream) {
    PTK_CHECK_ARG(ctx != nullptr, "null context");
    PTK_CHECK_ARG(dtype == PTK_F32 || dtype == PTK_F64, "bad dtype");
    PTK_CHECK_ARG(J >= 1 && J <= PTK_MAX_RANK, "J out of range");
    PTK_CHECK_ARG(ld == delta_out_ld(J), "ld must be J + 1 rounded up to an odd number (%d)", delta_out_ld(J));
    PTK_CHECK_ARG(rows >= 1 && rows < (1ll << 31) && nnz >= 0 && nnz < (1ll << 31), "sizes out of range");
    PTK_CHECK_ARG(schedule >= PTK_SCHED_AUTO && schedule <= PTK_SCHED_TENSOR, "bad schedule");
    PTK_CHECK_ARG(row_ptr && out && (nnz == 0 || (delta && rid)), "null arrays");
    PTK_CHECK_ARG(digits == 0 || digits == 3 || digits == 4, "digits must be 0 (4), 3 or 4");
    cudaStream_t st = (cudaStream_t)stream;
    PTK_CUDA(cudaSetDevice(ctx->device));
    const int nout = gram_nout(J);
    PTK_CUDA(cudaMemsetAsync(out, 0, sizeof(double) * (size_t)rows * nout, st));
    if (nnz == 0) {
        PTK_CUDA(cudaStreamSynchronize(st));
        return PTK_OK;
    }
    // the kernels' bulk copies read up to a few rows past the end: work on
    // copies in context scratch (which keeps slack past every buffer)
    const size_t dbytes = dtype_size(dtype) * (size_t)nnz * ld;
    void* dcopy = scratch(ctx, SLOT_DELTA, dbytes);
    int32_t* rcopy = (int32_t*)scratch(ctx, SLOT_FOLD1, sizeof(int32_t) * (size_t)nnz);
    if (!dcopy || !rcopy) return PTK_ERR_OUT_OF_MEMORY;
    PTK_CUDA(cudaMemcpyAsync(dcopy, delta, dbytes, cudaMemcpyDeviceToDevice, st));
    PTK_CUDA(cudaMemcpyAsync(rcopy, rid, sizeof(int32_t) * (size_t)nnz, cudaMemcpyDeviceToDevice, st));
    GramJob gj;
    gj.n = nnz;
    gj.rows = rows;
    gj.J = J;
    gj.delta = dcopy;
    gj.ld = ld;
    gj.rid = rcopy;
    gj.row_ptr = row_ptr;
    gj.dtype = dtype;
    gj.schedule = schedule;
    gj.digits = digits == 3 ? 3 : 4;
    int64_t mx = 0;
    {
        // the longest row (the automatic schedule reads it)
        std::vector<int64_t> rp((size_t)rows + 1);
        PTK_CUDA(cudaMemcpyAsync(rp.data(), row_ptr, sizeof(int64_t) * (size_t)(rows + 1), cudaMemcpyDeviceToHost, st));
        PTK_CUDA(cudaStreamSynchronize(st));
        for (int64_t r = 0; r < rows; ++r) mx = std::max<int64_t>(mx, rp[r + 1] - rp[r]);
        PTK_CHECK_ARG(rp[0] == 0 && rp[rows] == nnz, "row_ptr must run from 0 to nnz");
    }
    gj.max_row = mx;
    if (dtype == PTK_F32 && (schedule == PTK_SCHED_AUTO || schedule == PTK_SCHED_TENSOR)) {
        int4* plan = (int4*)scratch(ctx, SLOT_TC_PLAN, sizeof(int4) * (size_t)gram_tc_plan_capacity(nnz));
        if (!plan) return PTK_ERR_OUT_OF_MEMORY;
        PTK_TRY(gram_tc_plan(ctx, row_ptr, rows, nnz, plan, &gj.tc_nchunks, &gj.tc_long_entries, st));
        gj.tc_plan = plan;
    }
    int f64 = dtype == PTK_F64 ? 1 : 0;
    gj.wrote_f64 = &f64;
    void* buf = out;
    if (dtype == PTK_F32) {  // entry tiles keep (s, lo) pairs: sums go to scratch, converted below
        buf = scratch(ctx, SLOT_ROWBUF, 8 * (size_t)rows * nout);
        if (!buf) return PTK_ERR_OUT_OF_MEMORY;
        PTK_CUDA(cudaMemsetAsync(buf, 0, 8 * (size_t)rows * nout, st));
    }
    gj.rowbuf = buf;
    PTK_CUDA(cudaMemsetAsync(ctx->d_flags, 0, sizeof(int) * FLAG_COUNT, st));
    {
        TimerScope tg(ctx, PTK_T_GRAM, st);
        PTK_TRY(gram(ctx, gj, st));
    }
    if (buf != out) {
        const int64_t n = rows * nout;
        const int g = (int)std::min<int64_t>(ceil_div(n, 256), (int64_t)ctx->sm_count * 8);
        if (f64)
            PTK_CUDA(cudaMemcpyAsync(out, buf, sizeof(double) * (size_t)n, cudaMemcpyDeviceToDevice, st));
        else
            { pairs_to_f64<<<g, 256, 0, st>>>((const float2*)buf, out, n); ::ptk::note_launch(); }
        PTK_LAUNCH_CHECK();
    }
    int h_flags[FLAG_COUNT];
    PTK_CUDA(cudaMemcpyAsync(h_flags, ctx->d_flags, sizeof(h_flags), cudaMemcpyDeviceToHost, st));
    PTK_CUDA(cudaStreamSynchronize(st));
    if (h_flags[FLAG_TIMEOUT]) {
        set_error("a bounded device wait gave up (%d)", h_flags[FLAG_TIMEOUT]);
        return PTK_ERR_TIMEOUT;
    }
    return PTK_OK;
}

ptk_status ptk_predict(ptk_ctx* ctx, const ptk_model* m, const int32_t* coords, int64_t n, void* out,
                       ptk_stream_t stream) {
    PTK_CHECK_ARG(ctx && m, "null argument");
    PTK_TRY(check_model(m));
    PTK_CHECK_ARG(n >= 0 && n < (1ll << 31), "n out of range");
    if (n == 0) return PTK_OK;
    PTK_CHECK_ARG(coords && out, "null arrays");
    cudaStream_t st = (cudaStream_t)stream;
    PTK_CUDA(cudaSetDevice(ctx->device));
    const int N = m->order;
    DeltaJob job = make_job(m, 0, n);
    for (int k = 0; k < N; ++k) job.col[k] = coords + k;
    job.cstride = N;
    void* delta = scratch(ctx, SLOT_FOLD0, dtype_size(m->dtype) * (size_t)n * job.out_ld);
    if (!delta) return PTK_ERR_OUT_OF_MEMORY;
    job.out = delta;
    PTK_TRY(delta_simt(ctx, job, st));
    return dot_rows(ctx, delta, job.out_ld, m->J[0], nullptr, coords, N, n, m->factors[0], m->ld[0], m->dtype, out,
                    st);
}

ptk_status ptk_foldin(ptk_ctx* ctx, const ptk_model* m, int32_t mode, const ptk_foldin_batch* b, double lambda,
                      ptk_precision prec, ptk_stream_t stream) {
    PTK_CHECK_ARG(ctx && m && b, "null argument");
    PTK_TRY(check_model(m));
    PTK_CHECK_ARG(mode >= 0 && mode < m->order, "mode out of range");
    PTK_CHECK_ARG(lambda > 0.0, "lambda must be > 0");
    PTK_CHECK_ARG(b->count >= 0, "count < 0");
    PTK_CHECK_ARG(b->total_obs >= 0 && b->total_obs < (1ll << 31) && b->total_query >= 0, "bad totals");
    if (b->count == 0) return PTK_OK;
    PTK_CHECK_ARG(b->obs_ptr && b->rows_out, "null arrays");
    cudaStream_t st = (cudaStream_t)stream;
    PTK_CUDA(cudaSetDevice(ctx->device));
    const int N = m->order;
    const int Jn = m->J[mode];
    const size_t ts = dtype_size(m->dtype);
    const int64_t no = b->total_obs;
    // rows: delta over the observed entries, Gram per request, FP64 solve
    DeltaJob job = make_job(m, mode, no);
    for (int k = 0; k < N; ++k) job.col[k] = b->obs_idx + k;
    job.cstride = N;
    job.vals = b->obs_vals;
    const int ld = job.out_ld;
    void* delta = scratch(ctx, SLOT_FOLD0, ts * (size_t)std::max<int64_t>(no, 1) * ld);
    int32_t* rid = (int32_t*)scratch(ctx, SLOT_FOLD1, sizeof(int32_t) * (size_t)std::max<int64_t>(no, 1));
    const int nout = gram_nout(Jn);
    void* rowbuf = scratch(ctx, SLOT_ROWBUF, 8 * (size_t)b->count * nout);
    if (!delta || !rid || !rowbuf) return PTK_ERR_OUT_OF_MEMORY;
    job.out = delta;
    if (no > 0) {
        PTK_TRY(delta_run(ctx, job, m->dtype == PTK_F32 ? prec : PTK_PREC_FP64, st));
        int g = (int)std::min<int64_t>(ceil_div(no, 256), ctx->sm_count * 16);
        { zero_pad_rows<<<g, 256, 0, st>>>(delta, ld, m->dtype == PTK_F64, b->obs_idx, N, mode, no); ::ptk::note_launch(); }
        { rid_from_ptr<<<g, 256, 0, st>>>(b->obs_ptr, b->count, no, rid); ::ptk::note_launch(); }
        PTK_LAUNCH_CHECK();
        GramJob gj;
        gj.n = no;
        gj.rows = b->count;
        gj.J = Jn;
        gj.delta = delta;
        gj.ld = ld;
        gj.rid = rid;
        gj.row_ptr = b->obs_ptr;
        gj.rowbuf = rowbuf;
        gj.dtype = m->dtype;
        PTK_TRY(gram(ctx, gj, st));
    }
    SolveJob sj;
    sj.rows = b->count;
    sj.J = Jn;
    sj.rowbuf = rowbuf;
    sj.buf_dtype = m->dtype;
    sj.row_ptr = b->obs_ptr;
    sj.lambda = lambda;
    sj.out = b->rows_out;
    sj.ld = Jn;
    sj.out_dtype = m->dtype;
    PTK_TRY(solve_rows(ctx, sj, st));
    // predictions of the query coordinates with the new rows, Eq. (recon2)
    const int64_t nq = b->total_query;
    if (nq > 0) {
        PTK_CHECK_ARG(b->query_ptr && b->query_idx && b->preds_out, "null query arrays");
        DeltaJob qj = make_job(m, mode, nq);
        for (int k = 0; k < N; ++k) qj.col[k] = b->query_idx + k;
        qj.cstride = N;
        void* qd = scratch(ctx, SLOT_DELTA, ts * (size_t)nq * qj.out_ld);
        int32_t* qrid = (int32_t*)scratch(ctx, SLOT_MISC, sizeof(int32_t) * (size_t)nq);
        if (!qd || !qrid) return PTK_ERR_OUT_OF_MEMORY;
        qj.out = qd;
        PTK_TRY(delta_simt(ctx, qj, st));
        int g = (int)std::min<int64_t>(ceil_div(nq, 256), ctx->sm_count * 16);
        { rid_from_ptr<<<g, 256, 0, st>>>(b->query_ptr, b->count, nq, qrid); ::ptk::note_launch(); }
        PTK_LAUNCH_CHECK();
        PTK_TRY(dot_rows(ctx, qd, qj.out_ld, Jn, qrid, nullptr, 0, nq, b->rows_out, Jn, m->dtype, b->preds_out, st));
    }
    return PTK_OK;
}

// Self-test of the bounded waits: one block waits on an mbarrier phase that
// nothing completes, gives up after `limit` polls, records FLAG_TIMEOUT and
// returns; the host turns the flag into PTK_ERR_TIMEOUT.  The context stays
// usable.
__global__ void wait_selftest(int* flags, long long limit) {
    __shared__ uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        fence_mbar_init();
        mbar_wait_bounded(&bar, 0, flags, limit);  // no arrival ever comes
    }
}

ptk_status ptk_selftest_wait(ptk_ctx* ctx, int64_t limit, ptk_stream_t stream) {
    PTK_CHECK_ARG(ctx && limit >= 1 && limit <= (1ll << 20), "bad argument");
    cudaStream_t st = (cudaStream_t)stream;
    PTK_CUDA(cudaSetDevice(ctx->device));
    PTK_CUDA(cudaMemsetAsync(ctx->d_flags, 0, sizeof(int) * FLAG_COUNT, st));
    { wait_selftest<<<1, 32, 0, st>>>(ctx->d_flags, (long long)limit); ::ptk::note_launch(); }
    PTK_LAUNCH_CHECK();
    PTK_TRY(read_flags(ctx, st, ctx->h_flags));
    if (ctx->h_flags[FLAG_TIMEOUT]) {
        set_error("a bounded device wait gave up (%d)", ctx->h_flags[FLAG_TIMEOUT]);
        return PTK_ERR_TIMEOUT;
    }
    return PTK_OK;
}

ptk_status ptk_partial_error(ptk_ctx* ctx, const ptk_coo* x, const ptk_model* m, double* R_out,
                             ptk_stream_t stream) {
    PTK_CHECK_ARG(ctx && x && m && R_out, "null argument");
    PTK_TRY(check_model(m));
    PTK_TRY(check_coo(x, m));
    if (m->dtype != PTK_F32 || x->dtype != PTK_F32) {
        set_error("ptk_partial_error needs an FP32 model and FP32 values");
        return PTK_ERR_UNSUPPORTED;
    }
    PTK_CUDA(cudaSetDevice(ctx->device));
    return partial_error_impl(ctx, x, m, (const float*)x->vals, R_out, (cudaStream_t)stream);
}

ptk_status ptk_qr_finalize(ptk_ctx* ctx, ptk_model* m, ptk_stream_t stream) {
    PTK_CHECK_ARG(ctx && m, "null argument");
    PTK_TRY(check_model(m));
    for (int n = 0; n < m->order; ++n) PTK_CHECK_ARG(m->dims[n] >= m->J[n], "QR needs I_n >= J_n (mode %d)", n);
    PTK_CUDA(cudaSetDevice(ctx->device));
    return qr_finalize_impl(ctx, m, (cudaStream_t)stream);
}

}  // extern "C"
