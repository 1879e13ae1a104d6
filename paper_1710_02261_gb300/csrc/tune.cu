// tune.cu -- launch-shape autotuner for the delta contraction.
//
// The fastest way to evaluate Eq. (delta) depends on the problem's shape: the
// tensor-core kernel needs J_n * J_L <= 128 and a middle-mode Kronecker width
// <= 256 and loses to the CUDA cores on small cores; a core larger than shared
// memory is streamed through it in chunks whose best size depends on the
// ranks; and when many problems share the GPU (batched fits), fewer resident
// blocks per launch can beat the occupancy limit.  The tuner times each
// candidate on a prefix of a real problem's entries and keeps the fastest per
// class (model dtype, precision, order, ranks) in the context's table, which
// every later delta launch of that class uses (the lanes of a batched fit
// share it).  A candidate never lowers the requested precision: the CUDA-core
// kernel computes in FP32 or FP64, at least what TF32/BF16 requests give.
#include "common.cuh"

namespace ptk {

uint64_t tune_key(const DeltaJob& job, ptk_precision prec) {
    uint64_t k = (uint64_t)(job.dtype == PTK_F64) | ((uint64_t)prec << 1) | ((uint64_t)job.order << 4);
    for (int n = 0; n < job.order; ++n) k |= (uint64_t)(job.J[n] & 31) << (7 + 5 * n);
    return k;
}

ptk_status delta_run(ptk_ctx* ctx, DeltaJob job, ptk_precision prec, cudaStream_t st) {
    const bool tc_ok = delta_tc_supported(job, prec);
    int backend = tc_ok ? TUNE_TC : TUNE_SIMT;
    if (ctx->tune && !ctx->tune->empty()) {
        auto it = ctx->tune->find(tune_key(job, prec));
        if (it != ctx->tune->end()) {
            const TuneCfg& c = it->second;
            if (c.backend == TUNE_SIMT || (c.backend == TUNE_TC && tc_ok)) backend = c.backend;
            job.chunk_kb = c.chunk_kb;
            job.ctas_per_sm = c.ctas_per_sm;
            job.dent = c.dent;
        }
    }
    if (backend == TUNE_TC) return delta_tc(ctx, job, prec, st);
    return delta_simt(ctx, job, st);
}

}  // namespace ptk

using namespace ptk;

extern "C" ptk_status ptk_autotune_delta(ptk_ctx* ctx, const ptk_slices* s, const ptk_model* m, ptk_precision prec,
                                         int64_t max_entries, int32_t reps, ptk_tune_report* out_h,
                                         ptk_stream_t stream) {
    PTK_CHECK_ARG(ctx && s && m, "null argument");
    PTK_TRY(check_model(m));
    PTK_CHECK_ARG(s->order == m->order && s->rows == m->dims[s->mode], "slices do not match the model");
    PTK_CHECK_ARG(s->dtype == m->dtype, "slices were built for another dtype");
    PTK_CHECK_ARG((prec == PTK_PREC_FP64) == (m->dtype == PTK_F64), "precision does not match the model dtype");
    PTK_CHECK_ARG(reps >= 1 && reps <= 100, "reps out of [1, 100]");
    cudaStream_t st = (cudaStream_t)stream;
    PTK_CUDA(cudaSetDevice(ctx->device));
    const int n = s->mode;
    DeltaJob job = make_job(m, n, std::min<int64_t>(s->nnz, max_entries > 0 ? max_entries : s->nnz));
    for (int k = 0; k < m->order; ++k) job.col[k] = s->cols[k];
    job.cstride = 1;
    job.vals = s->vals;
    job.padded = true;
    void* out = scratch(ctx, SLOT_DELTA, dtype_size(m->dtype) * (size_t)std::max<int64_t>(job.n, 1) * job.out_ld);
    if (!out) return PTK_ERR_OUT_OF_MEMORY;
    job.out = out;

    std::vector<TuneCfg> cand;
    if (delta_tc_supported(job, prec)) {
        TuneCfg c;
        c.backend = TUNE_TC;
        cand.push_back(c);
    }
    int64_t G = 1;
    for (int k = 0; k < m->order; ++k) G *= m->J[k];
    const bool streamed = (size_t)G * dtype_size(m->dtype) > std::min<size_t>(ctx->smem_optin, 100 * 1024);
    const int chunks[] = {16, 32, 48, 96};
    const int ctas[] = {0, 1};
    const int dents[] = {2, 4};
    for (int ch : chunks) {
        if (!streamed && ch != 48) continue;
        for (int ct : ctas)
            for (int dn : dents) {
                if (dn == 4 && m->dtype == PTK_F64) continue;  // FP64 runs two entries per thread
                TuneCfg c;
                c.backend = TUNE_SIMT;
                c.chunk_kb = streamed ? ch : 0;
                c.ctas_per_sm = ct;
                c.dent = dn;
                cand.push_back(c);
            }
    }
    PTK_CHECK_ARG((int)cand.size() <= PTK_TUNE_MAX, "too many candidates");
    cudaEvent_t e0, e1;
    PTK_CUDA(cudaEventCreate(&e0));
    PTK_CUDA(cudaEventCreate(&e1));
    ptk_status rc = PTK_OK;
    std::vector<float> ms(cand.size(), 0.f);
    for (size_t i = 0; i < cand.size() && rc == PTK_OK; ++i) {
        DeltaJob j = job;
        j.chunk_kb = cand[i].chunk_kb;
        j.ctas_per_sm = cand[i].ctas_per_sm;
        j.dent = cand[i].dent;
        auto launch = [&]() {
            return cand[i].backend == TUNE_TC ? delta_tc(ctx, j, prec, st) : delta_simt(ctx, j, st);
        };
        rc = launch();  // warm-up
        if (rc != PTK_OK) break;
        if (cudaEventRecord(e0, st) != cudaSuccess) rc = PTK_ERR_CUDA;
        for (int r = 0; r < reps && rc == PTK_OK; ++r) rc = launch();
        if (rc == PTK_OK && (cudaEventRecord(e1, st) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
                             cudaEventElapsedTime(&ms[i], e0, e1) != cudaSuccess)) {
            set_error("autotune: timing failed");
            rc = PTK_ERR_CUDA;
        }
        ms[i] /= (float)reps;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc != PTK_OK) return rc;
    size_t best = 0;
    for (size_t i = 1; i < cand.size(); ++i)
        if (ms[i] < ms[best]) best = i;
    (*ctx->tune)[tune_key(job, prec)] = cand[best];
    if (out_h) {
        std::memset(out_h, 0, sizeof *out_h);
        out_h->candidates = (int32_t)cand.size();
        out_h->best = (int32_t)best;
        out_h->entries = job.n;
        for (size_t i = 0; i < cand.size(); ++i) {
            out_h->backend[i] = cand[i].backend;
            out_h->chunk_kb[i] = cand[i].chunk_kb;
            out_h->ctas_per_sm[i] = cand[i].ctas_per_sm;
            out_h->entries_per_thread[i] = cand[i].backend == TUNE_SIMT ? cand[i].dent : 0;
            out_h->ms[i] = ms[i];
        }
    }
    return PTK_OK;
}

extern "C" void ptk_autotune_clear(ptk_ctx* ctx) {
    if (ctx && ctx->tune) ctx->tune->clear();
}
