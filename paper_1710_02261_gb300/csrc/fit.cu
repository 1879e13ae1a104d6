// fit.cu -- Alg. 2's driver over one or many independent problems.
//
// Each problem is a whole P-Tucker factorisation (its own tensor, slices,
// core and factors).  Problems are spread over lanes: a lane is a CUDA stream
// with a child context (its own scratch and status words), so the kernels of
// different problems run on the GPU at the same time and small problems fill
// the SMs together.  Problems go to lanes largest first, each to the lane
// with the least work so far (longest-processing-time order).
//
// Per problem, the first sweep runs eagerly: it sizes the lane's scratch and
// sets the kernels' attributes.  The remaining sweeps are one CUDA graph:
//
//     arm  ->  WHILE (h) { sweep ; record }
//
// `record` writes the sweep's error (Eq. reconfull), counts the sweep and sets
// the loop condition h from the stopping rule (sweep budget, relative error
// change below tol, a bounded wait that gave up); `arm` sets h from the first
// sweep's record.  The loop runs on the device: no host round trip between
// sweeps.
#include "common.cuh"

#include <cmath>
#include <numeric>

namespace ptk {
namespace {

struct FitDev {
    double* errors;   // [count][max_sweeps]
    int32_t* sweeps;  // [count] sweeps done
    int32_t* cont;    // [count] 1 while the problem keeps iterating
    int32_t* status;  // [count] bit 0: a bounded wait gave up
};

// One sweep's bookkeeping (one thread).  stats[0] is the sweep's SSE.
__global__ void fit_record(const double* __restrict__ stats, const int* __restrict__ flags, FitDev d, int p,
                           int max_sweeps, double tol, cudaGraphConditionalHandle h, int set_handle) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    const int s = d.sweeps[p];
    const double err = sqrt(stats[0]);
    double* e = d.errors + (int64_t)p * max_sweeps;
    if (s < max_sweeps) e[s] = err;
    const int done = s + 1;
    d.sweeps[p] = done;
    bool cont = done < max_sweeps;
    if (tol > 0.0 && s >= 1) {
        const double prev = e[s - 1];
        if (prev > 0.0 && fabs(err - prev) / prev < tol) cont = false;
    }
    if (flags[FLAG_TIMEOUT]) {
        d.status[p] |= 1;
        cont = false;
    }
    d.cont[p] = cont ? 1 : 0;
    if (set_handle) cudaGraphSetConditional(h, cont ? 1u : 0u);
}

__global__ void fit_arm(const int32_t* __restrict__ cont, cudaGraphConditionalHandle h) {
    if (threadIdx.x == 0 && blockIdx.x == 0) cudaGraphSetConditional(h, cont[0] ? 1u : 0u);
}

int64_t core_elems(const ptk_model& m) {
    int64_t g = 1;
    for (int n = 0; n < m.order; ++n) g *= m.J[n];
    return g;
}

// Work estimate of one sweep: delta (2|G| per entry and mode) plus Gram and
// solve terms; only the order of magnitude matters for the lane balance.
double sweep_cost(const ptk_problem& p) {
    const double G = (double)core_elems(p.model);
    double c = 0.0;
    for (int n = 0; n < p.model.order; ++n)
        c += (double)p.x.nnz * (2.0 * G + (double)p.model.J[n] * p.model.J[n]) +
             (double)p.model.dims[n] * std::pow((double)p.model.J[n], 3.0);
    return c;
}

ptk_status ensure_lanes(ptk_ctx* ctx, int L) {
    while ((int)ctx->lanes.size() < L) {
        cudaStream_t st = nullptr;
        PTK_CUDA(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
        ptk_ctx* child = nullptr;
        ptk_status rc = ptk_create(&child, ctx->device);
        if (rc != PTK_OK) {
            cudaStreamDestroy(st);
            return rc;
        }
        child->tune = ctx->tune;  // the lanes use the parent's tuned launch shapes
        ctx->lanes.emplace_back(st, child);
    }
    return PTK_OK;
}

struct GraphRec {
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    int problem = 0;
    int64_t body_launches = 0;  // launches of one loop iteration (counted once at capture)
};

// Captures  arm -> WHILE { sweep ; record }  for problem p on lane (st, lc).
ptk_status build_loop(ptk_ctx* lc, cudaStream_t st, ptk_problem* pr, const ptk_als_opts* ao, const FitDev& d, int p,
                      int max_sweeps, double tol, GraphRec* out) {
    cudaGraph_t g = nullptr;
    PTK_CUDA(cudaGraphCreate(&g, 0));
    out->graph = g;
    cudaGraphConditionalHandle h;
    PTK_CUDA(cudaGraphConditionalHandleCreate(&h, g, 0, 0));
    // arm node
    PTK_CUDA(cudaStreamBeginCaptureToGraph(st, g, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
    fit_arm<<<1, 32, 0, st>>>(d.cont + p, h);
    note_launch();
    cudaError_t le = cudaGetLastError();
    cudaGraph_t g2 = nullptr;
    cudaError_t ce = cudaStreamEndCapture(st, &g2);
    if (le != cudaSuccess || ce != cudaSuccess) {
        set_error("fit: capturing the loop's arm kernel failed: %s",
                  cudaGetErrorString(le != cudaSuccess ? le : ce));
        return PTK_ERR_CUDA;
    }
    cudaGraphNode_t arm = nullptr;
    size_t nn = 1;
    PTK_CUDA(cudaGraphGetNodes(g, &arm, &nn));
    if (nn != 1) {
        set_error("fit: the arm graph holds %zu nodes", nn);
        return PTK_ERR_CUDA;
    }
    // WHILE node and its body
    cudaGraphNodeParams cp = {cudaGraphNodeTypeConditional};  // the rest zero-initialised
    cp.conditional.handle = h;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    cudaGraphNode_t loop = nullptr;
    PTK_CUDA(cudaGraphAddNode(&loop, g, &arm, nullptr, 1, &cp));
    cudaGraph_t body = cp.conditional.phGraph_out[0];
    PTK_CUDA(cudaStreamBeginCaptureToGraph(st, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
    lc->in_capture = true;
    const int64_t l0 = g_launches.load();
    ptk_status rc = ptk_als_sweep(lc, &pr->x, pr->slices, &pr->model, ao, nullptr, st);
    if (rc == PTK_OK) {
        fit_record<<<1, 32, 0, st>>>(lc->d_stats, lc->d_flags, d, p, max_sweeps, tol, h, 1);
        note_launch();
        if (cudaGetLastError() != cudaSuccess) {
            set_error("fit: launching the record kernel into the loop body failed");
            rc = PTK_ERR_CUDA;
        }
    }
    out->body_launches = g_launches.load() - l0;
    lc->in_capture = false;
    cudaGraph_t b2 = nullptr;
    ce = cudaStreamEndCapture(st, &b2);
    if (rc != PTK_OK) return rc;
    if (ce != cudaSuccess) {
        set_error("fit: capturing the sweep into the loop body failed: %s", cudaGetErrorString(ce));
        return PTK_ERR_CUDA;
    }
    PTK_CUDA(cudaGraphInstantiate(&out->exec, g, 0));
    return PTK_OK;
}

}  // namespace
}  // namespace ptk

using namespace ptk;

extern "C" ptk_status ptk_fit(ptk_ctx* ctx, ptk_problem* probs, int32_t count, const ptk_fit_opts* o,
                              double* errors_h, int32_t* sweeps_h, ptk_stream_t stream) {
    PTK_CHECK_ARG(ctx && o && count >= 0 && (probs || count == 0), "null argument");
    PTK_CHECK_ARG(o->max_sweeps >= 0, "max_sweeps < 0");
    PTK_CHECK_ARG(o->lanes <= 16, "lanes > 16");
    if (count == 0) return PTK_OK;
    for (int p = 0; p < count; ++p) {
        PTK_TRY(check_model(&probs[p].model));
        PTK_TRY(check_coo(&probs[p].x, &probs[p].model));
    }
    PTK_CUDA(cudaSetDevice(ctx->device));
    cudaStream_t caller = (cudaStream_t)stream;
    const int S = o->max_sweeps;
    const int L = std::max(1, std::min<int>(count, o->lanes > 0 ? o->lanes : 8));
    PTK_TRY(ensure_lanes(ctx, L));

    // device bookkeeping
    const size_t eb = sizeof(double) * (size_t)count * std::max(S, 1);
    char* dmem = nullptr;
    PTK_CUDA(cudaMalloc(&dmem, eb + 3 * sizeof(int32_t) * (size_t)count + 256));
    FitDev d;
    d.errors = (double*)dmem;
    d.sweeps = (int32_t*)(dmem + eb);
    d.cont = d.sweeps + count;
    d.status = d.cont + count;
    std::vector<GraphRec> graphs;
    std::vector<cudaEvent_t> events;
    ptk_status rc = PTK_OK;
    auto fail = [&](ptk_status r) {
        if (rc == PTK_OK) rc = r;
    };
    do {
        if (cudaMemsetAsync(dmem, 0, eb + 3 * sizeof(int32_t) * (size_t)count, caller) != cudaSuccess) {
            set_error("fit: clearing the bookkeeping failed");
            fail(PTK_ERR_CUDA);
            break;
        }
        // lanes start after the caller's stream
        cudaEvent_t start;
        if (cudaEventCreateWithFlags(&start, cudaEventDisableTiming) != cudaSuccess) {
            fail(PTK_ERR_CUDA);
            break;
        }
        events.push_back(start);
        cudaEventRecord(start, caller);
        for (int l = 0; l < L; ++l) cudaStreamWaitEvent(ctx->lanes[l].first, start, 0);

        // largest first, each to the least-loaded lane
        std::vector<int> order(count);
        std::iota(order.begin(), order.end(), 0);
        std::vector<double> cost(count);
        for (int p = 0; p < count; ++p) cost[p] = sweep_cost(probs[p]);
        std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return cost[a] > cost[b]; });
        if (o->autotune) {
            // one tuning per untuned class, on its largest problem (the first met)
            for (int p : order) {
                ptk_problem* pr = &probs[p];
                if (pr->x.nnz == 0 || !pr->slices[0]) continue;
                DeltaJob key = make_job(&pr->model, 0, 0);
                if (ctx->tune->count(tune_key(key, o->als.precision))) continue;
                ptk_status r = ptk_autotune_delta(ctx, pr->slices[0], &pr->model, o->als.precision, 1 << 18, 2,
                                                  nullptr, caller);
                if (r != PTK_OK) {
                    fail(r);
                    break;
                }
            }
            if (rc != PTK_OK) break;
        }
        std::vector<double> load(L, 0.0);
        ptk_als_opts ao = o->als;
        ao.error_pass = 1;
        for (int p : order) {
            const int l = (int)(std::min_element(load.begin(), load.end()) - load.begin());
            load[l] += cost[p];
            cudaStream_t ls = ctx->lanes[l].first;
            ptk_ctx* lc = ctx->lanes[l].second;
            ptk_problem* pr = &probs[p];
            if (S >= 1) {
                ptk_status r = ptk_als_sweep(lc, &pr->x, pr->slices, &pr->model, &ao, nullptr, ls);
                if (r != PTK_OK) {
                    fail(r);
                    break;
                }
                { fit_record<<<1, 32, 0, ls>>>(lc->d_stats, lc->d_flags, d, p, S, o->tol, 0, 0); note_launch(); }
                if (cudaGetLastError() != cudaSuccess) {
                    set_error("fit: record kernel launch failed");
                    fail(PTK_ERR_CUDA);
                    break;
                }
            }
            if (S >= 2 && o->graphs) {
                GraphRec g;
                g.problem = p;
                ptk_status r = build_loop(lc, ls, pr, &ao, d, p, S, o->tol, &g);
                graphs.push_back(g);
                if (r != PTK_OK) {
                    fail(r);
                    break;
                }
                if (cudaGraphLaunch(g.exec, ls) != cudaSuccess) {
                    set_error("fit: graph launch failed");
                    fail(PTK_ERR_CUDA);
                    break;
                }
            } else if (S >= 2) {
                // eager: every sweep is enqueued; with a tolerance the host reads
                // the loop flag after each sweep
                for (int s = 1; s < S; ++s) {
                    if (o->tol > 0.0) {
                        int32_t c = 0;
                        if (cudaMemcpyAsync(&c, d.cont + p, sizeof c, cudaMemcpyDeviceToHost, ls) != cudaSuccess ||
                            cudaStreamSynchronize(ls) != cudaSuccess) {
                            set_error("fit: reading the loop flag failed");
                            fail(PTK_ERR_CUDA);
                            break;
                        }
                        if (!c) break;
                    }
                    ptk_status r = ptk_als_sweep(lc, &pr->x, pr->slices, &pr->model, &ao, nullptr, ls);
                    if (r != PTK_OK) {
                        fail(r);
                        break;
                    }
                    { fit_record<<<1, 32, 0, ls>>>(lc->d_stats, lc->d_flags, d, p, S, o->tol, 0, 0); note_launch(); }
                }
                if (rc != PTK_OK) break;
            }
            if (o->finalize_qr) {
                ptk_status r = ptk_qr_finalize(lc, &pr->model, ls);
                if (r != PTK_OK) {
                    fail(r);
                    break;
                }
            }
        }
        // the caller's stream waits for every lane
        for (int l = 0; l < L; ++l) {
            cudaEvent_t e;
            if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) continue;
            events.push_back(e);
            cudaEventRecord(e, ctx->lanes[l].first);
            cudaStreamWaitEvent(caller, e, 0);
        }
    } while (0);

    // wait for everything enqueued (also on failure: nothing may still run
    // when the bookkeeping is freed)
    for (int l = 0; l < L; ++l) cudaStreamSynchronize(ctx->lanes[l].first);
    cudaError_t se = cudaStreamSynchronize(caller);
    if (se != cudaSuccess) {
        set_error("fit: %s", cudaGetErrorString(se));
        fail(PTK_ERR_CUDA);
    }
    std::vector<int32_t> sweeps(count, 0), status(count, 0);
    if (rc == PTK_OK) {
        if (cudaMemcpy(sweeps.data(), d.sweeps, sizeof(int32_t) * count, cudaMemcpyDeviceToHost) != cudaSuccess ||
            cudaMemcpy(status.data(), d.status, sizeof(int32_t) * count, cudaMemcpyDeviceToHost) != cudaSuccess ||
            (errors_h && S > 0 && cudaMemcpy(errors_h, d.errors, eb, cudaMemcpyDeviceToHost) != cudaSuccess)) {
            set_error("fit: reading the results failed");
            fail(PTK_ERR_CUDA);
        }
    }
    if (rc == PTK_OK) {
        // launches inside the loops: one arm, then (sweeps - 1) loop bodies; one
        // arm and one body were counted when they were captured
        for (const GraphRec& g : graphs) g_launches.fetch_add((int64_t)(sweeps[g.problem] - 2) * g.body_launches);
        if (sweeps_h) std::memcpy(sweeps_h, sweeps.data(), sizeof(int32_t) * count);
        for (int p = 0; p < count; ++p)
            if (status[p] & 1) {
                set_error("fit: a bounded device wait gave up in problem %d", p);
                fail(PTK_ERR_TIMEOUT);
                break;
            }
    }
    for (GraphRec& g : graphs) {
        if (g.exec) cudaGraphExecDestroy(g.exec);
        if (g.graph) cudaGraphDestroy(g.graph);
    }
    for (cudaEvent_t e : events) cudaEventDestroy(e);
    cudaFree(dmem);
    return rc;
}
