// sort.cu -- slice layout (Omega^(n)_{i_n}, Table 1 / Alg. 3): a stable LSD
// radix sort of entry ids by their mode-n index, row boundaries, and the
// slice-ordered copies of coordinates and values.  Also the stable u64 key sort
// used by the Approx selection (Alg. 4, "sort R(beta) in descending order").
#include "common.cuh"

namespace ptk {
namespace {

constexpr int RS_T = 256;                 // threads per block
constexpr int RS_ITEMS = 16;              // rounds per tile
constexpr int RS_TILE = RS_T * RS_ITEMS;  // keys per block
constexpr int RS_WARPS = RS_T / 32;

// ---- device-wide exclusive scan of uint32 (chunks of 2048) ----------------
constexpr int SC_T = 256, SC_ITEMS = 8, SC_CH = SC_T * SC_ITEMS;

__device__ uint32_t block_excl_scan_256(uint32_t v, uint32_t* s_warp, uint32_t* total) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    uint32_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) s_warp[w] = x;
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t run = 0;
        for (int i = 0; i < SC_T / 32; ++i) {
            uint32_t t = s_warp[i];
            s_warp[i] = run;
            run += t;
        }
        s_warp[SC_T / 32] = run;
    }
    __syncthreads();
    uint32_t r = x - v + s_warp[w];
    *total = s_warp[SC_T / 32];
    __syncthreads();
    return r;
}

__global__ void scan_reduce(const uint32_t* __restrict__ in, int64_t n, uint32_t* __restrict__ sums) {
    __shared__ uint32_t s_warp[SC_T / 32 + 1];
    int64_t base = (int64_t)blockIdx.x * SC_CH;
    uint32_t acc = 0;
    for (int i = threadIdx.x; i < SC_CH; i += SC_T) {
        int64_t e = base + i;
        if (e < n) acc += in[e];
    }
    uint32_t tot;
    block_excl_scan_256(acc, s_warp, &tot);
    if (threadIdx.x == 0) sums[blockIdx.x] = tot;
}

__global__ void scan_top(uint32_t* __restrict__ sums, int64_t nb) {
    __shared__ uint32_t s_warp[SC_T / 32 + 1];
    uint32_t carry = 0;
    for (int64_t b = 0; b < nb; b += SC_T) {
        int64_t i = b + threadIdx.x;
        uint32_t v = i < nb ? sums[i] : 0u;
        uint32_t tot;
        uint32_t ex = block_excl_scan_256(v, s_warp, &tot);
        if (i < nb) sums[i] = ex + carry;
        carry += tot;
    }
}

__global__ void scan_apply(const uint32_t* __restrict__ in, uint32_t* __restrict__ out, int64_t n,
                           const uint32_t* __restrict__ sums) {
    __shared__ uint32_t s_warp[SC_T / 32 + 1];
    int64_t base = (int64_t)blockIdx.x * SC_CH + (int64_t)threadIdx.x * SC_ITEMS;
    uint32_t v[SC_ITEMS];
    uint32_t acc = 0;
#pragma unroll
    for (int i = 0; i < SC_ITEMS; ++i) {
        int64_t e = base + i;
        v[i] = e < n ? in[e] : 0u;
        acc += v[i];
    }
    uint32_t tot;
    uint32_t ex = block_excl_scan_256(acc, s_warp, &tot) + sums[blockIdx.x];
#pragma unroll
    for (int i = 0; i < SC_ITEMS; ++i) {
        int64_t e = base + i;
        if (e < n) out[e] = ex;
        ex += v[i];
    }
}

}  // namespace

ptk_status excl_scan_u32(ptk_ctx* ctx, const uint32_t* in, uint32_t* out, int64_t n, cudaStream_t st) {
    if (n <= 0) return PTK_OK;
    int64_t nb = ceil_div(n, SC_CH);
    uint32_t* sums = (uint32_t*)scratch(ctx, SLOT_SCAN, sizeof(uint32_t) * (size_t)nb);
    if (!sums) return PTK_ERR_OUT_OF_MEMORY;
    { scan_reduce<<<(unsigned)nb, SC_T, 0, st>>>(in, n, sums); ::ptk::note_launch(); }
    { scan_top<<<1, SC_T, 0, st>>>(sums, nb); ::ptk::note_launch(); }
    { scan_apply<<<(unsigned)nb, SC_T, 0, st>>>(in, out, n, sums); ::ptk::note_launch(); }
    PTK_LAUNCH_CHECK();
    return PTK_OK;
}

namespace {

// ---- radix sort passes -------------------------------------------------------
template <typename K>
__global__ void rs_hist(const K* __restrict__ keys, int64_t n, int shift, uint32_t* __restrict__ counts,
                        int64_t nblk) {
    __shared__ uint32_t h[256];
    h[threadIdx.x] = 0;
    __syncthreads();
    int64_t base = (int64_t)blockIdx.x * RS_TILE;
    for (int i = threadIdx.x; i < RS_TILE; i += RS_T) {
        int64_t e = base + i;
        if (e < n) atomicAdd(&h[(unsigned)(keys[e] >> shift) & 255u], 1u);
    }
    __syncthreads();
    counts[(int64_t)threadIdx.x * nblk + blockIdx.x] = h[threadIdx.x];
}

// Stable scatter: keys of a tile keep their relative order within a digit.
// Tile order = round-major, warp-major, lane-minor, i.e. input order.
template <typename K>
__global__ void rs_scatter(const K* __restrict__ kin, const uint32_t* __restrict__ vin, K* __restrict__ kout,
                           uint32_t* __restrict__ vout, int64_t n, int shift, const uint32_t* __restrict__ offs,
                           int64_t nblk) {
    __shared__ uint32_t base[256];
    __shared__ uint32_t wcnt[RS_WARPS][257];
    const int t = threadIdx.x, lane = t & 31, w = t >> 5;
    base[t] = offs[(int64_t)t * nblk + blockIdx.x];
    for (int i = 0; i < RS_WARPS; ++i) wcnt[i][t] = 0;
    if (t == 0)
        for (int i = 0; i < RS_WARPS; ++i) wcnt[i][256] = 0;
    __syncthreads();
    const unsigned lt = (1u << lane) - 1u;
    int64_t tile = (int64_t)blockIdx.x * RS_TILE;
    for (int r = 0; r < RS_ITEMS; ++r) {
        int64_t e = tile + (int64_t)r * RS_T + t;
        bool valid = e < n;
        K key = valid ? kin[e] : K(0);
        uint32_t val = valid ? vin[e] : 0u;
        unsigned d = valid ? ((unsigned)(key >> shift) & 255u) : 256u;
        unsigned peers = __match_any_sync(0xffffffffu, d);
        unsigned rank = __popc(peers & lt);
        bool leader = (__ffs(peers) - 1) == lane;
        if (leader) wcnt[w][d] = __popc(peers);
        __syncthreads();
        uint32_t pos = 0;
        if (valid) {
            uint32_t pre = 0;
            for (int i = 0; i < w; ++i) pre += wcnt[i][d];
            pos = base[d] + pre + rank;
        }
        __syncthreads();
        {
            uint32_t tot = 0;
            for (int i = 0; i < RS_WARPS; ++i) {
                tot += wcnt[i][t];
                wcnt[i][t] = 0;
            }
            base[t] += tot;
            if (t == 0)
                for (int i = 0; i < RS_WARPS; ++i) wcnt[i][256] = 0;
        }
        if (valid) {
            kout[pos] = key;
            vout[pos] = val;
        }
        __syncthreads();
    }
}

template <typename K>
ptk_status radix_sort_pairs(ptk_ctx* ctx, K* keys, uint32_t* vals, K* keys_tmp, uint32_t* vals_tmp, int64_t n,
                            int bits, cudaStream_t st, K** keys_out, uint32_t** vals_out) {
    *keys_out = keys;
    *vals_out = vals;
    if (n <= 1 || bits <= 0) return PTK_OK;
    int64_t nblk = ceil_div(n, RS_TILE);
    int64_t ncount = 256 * nblk;
    uint32_t* counts = (uint32_t*)scratch(ctx, SLOT_SORT2, sizeof(uint32_t) * (size_t)ncount);
    if (!counts) return PTK_ERR_OUT_OF_MEMORY;
    K* ka = keys;
    uint32_t* va = vals;
    K* kb = keys_tmp;
    uint32_t* vb = vals_tmp;
    for (int shift = 0; shift < bits; shift += 8) {
        { rs_hist<K><<<(unsigned)nblk, RS_T, 0, st>>>(ka, n, shift, counts, nblk); ::ptk::note_launch(); }
        PTK_LAUNCH_CHECK();
        PTK_TRY(excl_scan_u32(ctx, counts, counts, ncount, st));
        { rs_scatter<K><<<(unsigned)nblk, RS_T, 0, st>>>(ka, va, kb, vb, n, shift, counts, nblk); ::ptk::note_launch(); }
        PTK_LAUNCH_CHECK();
        K* tk = ka; ka = kb; kb = tk;
        uint32_t* tv = va; va = vb; vb = tv;
    }
    *keys_out = ka;
    *vals_out = va;
    return PTK_OK;
}

// ---- slice layout kernels ---------------------------------------------------
__global__ void slices_init(const int32_t* __restrict__ idx, int order, int mode, int64_t n, int64_t I,
                            uint32_t* __restrict__ keys, uint32_t* __restrict__ vals, int* flags) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
        int32_t i = idx[e * order + mode];
        if (i < 0 || i >= I) {
            atomicAdd(&flags[FLAG_BAD_INDEX], 1);
            i = 0;
        }
        keys[e] = (uint32_t)i;
        vals[e] = (uint32_t)e;
    }
}

__global__ void check_cols(const int32_t* __restrict__ idx, int order, int64_t n, const int64_t* __restrict__ dims,
                           int* flags) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
        for (int k = 0; k < order; ++k) {
            int32_t i = idx[e * order + k];
            if (i < 0 || i >= dims[k]) atomicAdd(&flags[FLAG_BAD_INDEX], 1);
        }
    }
}

// row_ptr[r] = first slice position whose row is >= r
__global__ void slices_rowptr(const uint32_t* __restrict__ keys, int64_t n, int64_t I, int64_t* __restrict__ row_ptr) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e <= n; e += (int64_t)gridDim.x * blockDim.x) {
        int64_t lo = e == 0 ? -1 : (int64_t)keys[e - 1];
        int64_t hi = e == n ? I : (int64_t)keys[e];
        for (int64_t r = lo + 1; r <= hi; ++r) row_ptr[r] = e;
    }
}

// longest row (entries) over all rows, folded into *out with atomicMax
__global__ void slices_maxrow(const int64_t* __restrict__ row_ptr, int64_t I, unsigned long long* out) {
    unsigned long long m = 0;
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < I; r += (int64_t)gridDim.x * blockDim.x)
        m = max(m, (unsigned long long)(row_ptr[r + 1] - row_ptr[r]));
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, off));
    if ((threadIdx.x & 31) == 0 && m > 0) atomicMax(out, m);
}

// Slice-ordered copies: entry e of the layout is input entry perm_in[e].  Each
// thread takes GU entries at once (their loads in flight together); with
// four modes a coordinate row is one 16-byte load.
template <typename TO, bool ROW4>
__global__ void slices_gather(const int32_t* __restrict__ idx, const void* __restrict__ vals_in, int in_f64,
                              int order, int mode, int64_t n, const uint32_t* __restrict__ keys,
                              const uint32_t* __restrict__ perm_in, int32_t* __restrict__ perm,
                              int32_t* const* __restrict__ cols, TO* __restrict__ vals) {
    constexpr int GU = 4;
    int32_t* c[PTK_MAX_ORDER];
    for (int k = 0; k < order; ++k) c[k] = cols[k];
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t e0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e0 < n; e0 += stride * GU) {
        uint32_t p[GU];
#pragma unroll
        for (int u = 0; u < GU; ++u) p[u] = e0 + u * stride < n ? perm_in[e0 + u * stride] : 0u;
        if constexpr (ROW4) {
            int4 r[GU];
            TO v[GU];
#pragma unroll
            for (int u = 0; u < GU; ++u) {
                r[u] = reinterpret_cast<const int4*>(idx)[p[u]];
                v[u] = in_f64 ? (TO)((const double*)vals_in)[p[u]] : (TO)((const float*)vals_in)[p[u]];
            }
#pragma unroll
            for (int u = 0; u < GU; ++u) {
                const int64_t e = e0 + u * stride;
                if (e >= n) break;
                perm[e] = (int32_t)p[u];
                c[0][e] = r[u].x;
                c[1][e] = r[u].y;
                c[2][e] = r[u].z;
                c[3][e] = r[u].w;
                c[mode][e] = (int32_t)keys[e];
                vals[e] = v[u];
            }
        } else {
#pragma unroll
            for (int u = 0; u < GU; ++u) {
                const int64_t e = e0 + u * stride;
                if (e >= n) break;
                perm[e] = (int32_t)p[u];
                for (int k = 0; k < order; ++k) c[k][e] = k == mode ? (int32_t)keys[e] : idx[(int64_t)p[u] * order + k];
                vals[e] = in_f64 ? (TO)((const double*)vals_in)[p[u]] : (TO)((const float*)vals_in)[p[u]];
            }
        }
    }
}

int grid_for(ptk_ctx* ctx, int64_t n, int threads) {
    int64_t g = ceil_div(n > 0 ? n : 1, threads);
    int64_t cap = (int64_t)ctx->sm_count * 16;
    return (int)(g < cap ? g : cap);
}

}  // namespace

ptk_status build_slices_impl(ptk_ctx* ctx, const ptk_coo* x, int mode, ptk_dtype compute, ptk_slices* s,
                             cudaStream_t st) {
    const int64_t n = x->nnz;
    const int64_t I = x->dims[mode];
    const int N = x->order;
    s->mode = mode;
    s->order = N;
    s->nnz = n;
    s->rows = I;
    s->dtype = compute;
    const size_t vs = dtype_size(compute);
    // owned buffers: from the context's stream-ordered pool (reused across
    // calls), else plain allocations
    s->pooled = ctx->pool != nullptr;
    auto alloc = [&](void** p, size_t bytes) -> ptk_status {
        if (s->pooled) {
            PTK_CUDA(cudaMallocFromPoolAsync(p, bytes, ctx->pool, st));
        } else {
            PTK_CUDA(cudaMalloc(p, bytes));
        }
        return PTK_OK;
    };
    PTK_TRY(alloc((void**)&s->row_ptr, sizeof(int64_t) * (size_t)(I + 1)));
    if (n > 0) {
        PTK_TRY(alloc((void**)&s->perm, sizeof(int32_t) * (size_t)n));
        PTK_TRY(alloc(&s->vals, vs * (size_t)n + 16));
        for (int k = 0; k < N; ++k) PTK_TRY(alloc((void**)&s->cols[k], sizeof(int32_t) * (size_t)n + 16));
    }
    PTK_CUDA(cudaMemsetAsync(ctx->d_flags, 0, sizeof(int) * FLAG_COUNT, st));
    if (n > 0) {
        uint32_t* k0 = (uint32_t*)scratch(ctx, SLOT_SORT0, sizeof(uint32_t) * (size_t)n);
        uint32_t* v0 = (uint32_t*)scratch(ctx, SLOT_SORT1, sizeof(uint32_t) * (size_t)n);
        uint32_t* k1 = (uint32_t*)scratch(ctx, SLOT_SORT3, sizeof(uint32_t) * (size_t)n * 2);
        if (!k0 || !v0 || !k1) return PTK_ERR_OUT_OF_MEMORY;
        uint32_t* v1 = k1 + n;
        // dims, then the longest row
        int64_t* d_dims = (int64_t*)scratch(ctx, SLOT_MISC, sizeof(int64_t) * (PTK_MAX_ORDER + 1));
        if (!d_dims) return PTK_ERR_OUT_OF_MEMORY;
        PTK_CUDA(cudaMemcpyAsync(d_dims, x->dims, sizeof(int64_t) * N, cudaMemcpyHostToDevice, st));
        int g = grid_for(ctx, n, 256);
        { check_cols<<<g, 256, 0, st>>>(x->idx, N, n, d_dims, ctx->d_flags); ::ptk::note_launch(); }
        { slices_init<<<g, 256, 0, st>>>(x->idx, N, mode, n, I, k0, v0, ctx->d_flags); ::ptk::note_launch(); }
        PTK_LAUNCH_CHECK();
        int bits = 0;
        while (bits < 32 && ((int64_t)1 << bits) < I) ++bits;
        uint32_t *ks, *vs_;
        PTK_TRY(radix_sort_pairs<uint32_t>(ctx, k0, v0, k1, v1, n, bits, st, &ks, &vs_));
        { slices_rowptr<<<grid_for(ctx, n + 1, 256), 256, 0, st>>>(ks, n, I, s->row_ptr); ::ptk::note_launch(); }
        auto* d_maxrow = reinterpret_cast<unsigned long long*>(d_dims + PTK_MAX_ORDER);
        PTK_CUDA(cudaMemsetAsync(d_maxrow, 0, sizeof(unsigned long long), st));
        { slices_maxrow<<<grid_for(ctx, I, 256), 256, 0, st>>>(s->row_ptr, I, d_maxrow); ::ptk::note_launch(); }
        PTK_CUDA(cudaMemcpyAsync(&s->max_row, d_maxrow, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
        int32_t** d_cols = (int32_t**)scratch(ctx, SLOT_QR, sizeof(int32_t*) * PTK_MAX_ORDER);
        if (!d_cols) return PTK_ERR_OUT_OF_MEMORY;
        PTK_CUDA(cudaMemcpyAsync(d_cols, s->cols, sizeof(int32_t*) * PTK_MAX_ORDER, cudaMemcpyHostToDevice, st));
        int in_f64 = x->dtype == PTK_F64;
        // four modes and a 16-byte aligned coordinate array: one vector load per row
        const bool row4 = N == 4 && ((uintptr_t)x->idx & 15) == 0;
        const int gg = grid_for(ctx, ceil_div(n, 4), 256);
        if (compute == PTK_F64) {
            if (row4)
                slices_gather<double, true><<<gg, 256, 0, st>>>(x->idx, x->vals, in_f64, N, mode, n, ks, vs_, s->perm,
                                                                d_cols, (double*)s->vals);
            else
                slices_gather<double, false><<<gg, 256, 0, st>>>(x->idx, x->vals, in_f64, N, mode, n, ks, vs_, s->perm,
                                                                 d_cols, (double*)s->vals);
        } else {
            if (row4)
                slices_gather<float, true><<<gg, 256, 0, st>>>(x->idx, x->vals, in_f64, N, mode, n, ks, vs_, s->perm,
                                                               d_cols, (float*)s->vals);
            else
                slices_gather<float, false><<<gg, 256, 0, st>>>(x->idx, x->vals, in_f64, N, mode, n, ks, vs_, s->perm,
                                                                d_cols, (float*)s->vals);
        }
        ::ptk::note_launch();
        PTK_LAUNCH_CHECK();
        if (compute == PTK_F32) {
            // chunks of the long rows for the tensor-core Gram (synchronous)
            PTK_TRY(alloc((void**)&s->tc_plan, sizeof(int4) * (size_t)gram_tc_plan_capacity(n)));
            PTK_TRY(gram_tc_plan(ctx, s->row_ptr, I, n, s->tc_plan, &s->tc_nchunks, &s->tc_long_entries, st));
        }
    } else {
        PTK_CUDA(cudaMemsetAsync(s->row_ptr, 0, sizeof(int64_t) * (size_t)(I + 1), st));
    }
    int h_flags[FLAG_COUNT];
    PTK_CUDA(cudaMemcpyAsync(h_flags, ctx->d_flags, sizeof(h_flags), cudaMemcpyDeviceToHost, st));
    PTK_CUDA(cudaStreamSynchronize(st));
    if (h_flags[FLAG_BAD_INDEX]) {
        set_error("ptk_build_mode_slices: %d coordinates out of range", h_flags[FLAG_BAD_INDEX]);
        return PTK_ERR_INVALID_ARG;
    }
    return PTK_OK;
}

// Stable ascending sort of u64 keys with u32 payloads (in place, via scratch).
ptk_status radix_sort_u64_desc_stable(ptk_ctx* ctx, uint64_t* keys, uint32_t* vals, int64_t n, cudaStream_t st) {
    if (n <= 1) return PTK_OK;
    uint64_t* kt = (uint64_t*)scratch(ctx, SLOT_SORT0, sizeof(uint64_t) * (size_t)n);
    uint32_t* vt = (uint32_t*)scratch(ctx, SLOT_SORT1, sizeof(uint32_t) * (size_t)n);
    if (!kt || !vt) return PTK_ERR_OUT_OF_MEMORY;
    uint64_t* ko;
    uint32_t* vo;
    PTK_TRY(radix_sort_pairs<uint64_t>(ctx, keys, vals, kt, vt, n, 64, st, &ko, &vo));
    if (ko != keys) {
        PTK_CUDA(cudaMemcpyAsync(keys, ko, sizeof(uint64_t) * (size_t)n, cudaMemcpyDeviceToDevice, st));
        PTK_CUDA(cudaMemcpyAsync(vals, vo, sizeof(uint32_t) * (size_t)n, cudaMemcpyDeviceToDevice, st));
    }
    return PTK_OK;
}

}  // namespace ptk
