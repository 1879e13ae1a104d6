// gram.cu -- Eqs. (rowB) and (rowC): for every row i of mode n,
//     B_i = sum_{alpha in Omega_i} delta_alpha delta_alpha^T   (upper triangle)
//     c_i = sum_{alpha in Omega_i} x_alpha delta_alpha
// over the slice-ordered Delta rows [delta_0..delta_{J-1}, x] written by the
// delta kernels.  Slices are uneven (Zipf heads hold >10^6 entries, the
// smallest rows one), so the work is split by ENTRIES, not rows -- the GPU
// counterpart of the paper's dynamic scheduling over rows (Sec. 3.4):
//   * a block owns a tile of TILE consecutive entries, copied into shared
//     memory by the TMA engine (cp.async.bulk, double buffered);
//   * each thread walks RUN consecutive entries, keeping the J(J+1)/2 + J sums
//     of the current row in registers; a row that is complete inside the run
//     is written straight to the row buffer;
//   * pieces of rows that cross run boundaries are combined per block by a
//     column-parallel ordered scan (compensated FP32 sums), and pieces that
//     cross tile boundaries by a second kernel in FP64.
// Every sum is taken in a fixed order, so results are deterministic.
#include "common.cuh"

namespace ptk {

int gram_nout(int J) { return J * (J + 1) / 2 + J; }

namespace {

template <typename T, int J>
struct Cfg {
    static constexpr int NOUT = J * (J + 1) / 2 + J;
    static constexpr int LD = ((J + 1) & 1) ? (J + 1) : (J + 2);
    static constexpr int RUN_MIN = (2 * NOUT + LD - 1) / LD;
    static constexpr int RUN0 = RUN_MIN > 15 ? RUN_MIN : 15;
    static constexpr int RUN = (RUN0 & 1) ? RUN0 : RUN0 + 1;
    // shared memory for NT threads: two staged tiles + one slot per thread
    static constexpr int smem_for(int nt) {
        return 2 * ((nt * RUN * LD * (int)sizeof(T) + nt * RUN * 4 + 127) / 128 * 128) + nt * NOUT * (int)sizeof(T) + 256;
    }
    static constexpr int BUDGET = 220 * 1024;
    static constexpr int NT = smem_for(128) <= BUDGET ? 128 : (smem_for(64) <= BUDGET ? 64 : 32);
    static constexpr int TILE = NT * RUN;
    static constexpr int DELTA_BYTES = TILE * LD * (int)sizeof(T);
    static constexpr int RID_BYTES = TILE * 4;
    static constexpr int STAGE_BYTES = (DELTA_BYTES + RID_BYTES + 127) / 128 * 128;
    static constexpr int LSLOT_BYTES = NT * NOUT * (int)sizeof(T);
    static constexpr int SMEM = 2 * STAGE_BYTES + LSLOT_BYTES + 256;
    static_assert(SMEM <= BUDGET, "gram tile does not fit in shared memory");
    static_assert(NOUT <= RUN * LD, "right slots must fit in a consumed tile");
};

struct GramOut {
    void* rowbuf;
    void* blkL;        // [ntiles][NOUT]
    void* blkR;        // [ntiles][NOUT]
    int* blkLrow;      // [ntiles] row of the left partial, -1 if none
    int* blkLpass;     // [ntiles] 1 if the left row passes through the whole tile
    int* blkRrow;      // [ntiles]
};

template <typename T>
__device__ __forceinline__ void kahan_add(T& s, T& c, T v) {
    T y = v - c;
    T t = s + y;
    c = (t - s) - y;
    s = t;
}

template <typename T, int J>
__global__ void __launch_bounds__(Cfg<T, J>::NT) gram_kernel(const T* __restrict__ delta, const int32_t* __restrict__ rid,
                                                             int64_t n, int64_t ntiles, GramOut out, int* flags) {
    using C = Cfg<T, J>;
    constexpr int NOUT = C::NOUT, LD = C::LD, RUN = C::RUN, NT = C::NT, TILE = C::TILE;
    constexpr int NTRI = J * (J + 1) / 2;
    extern __shared__ __align__(128) unsigned char smem[];
    T* sLslot = reinterpret_cast<T*>(smem + 2 * C::STAGE_BYTES);               // [NT][NOUT]
    __shared__ uint64_t bar[2];
    __shared__ int sHasL[NT], sHasR[NT], sLrow[NT], sRrow[NT], sLpass[NT];
    __shared__ int sAbort;
    const int tid = threadIdx.x;
    T* rowbuf = reinterpret_cast<T*>(out.rowbuf);

    auto stage_delta = [&](int s) { return reinterpret_cast<T*>(smem + s * C::STAGE_BYTES); };
    auto stage_rid = [&](int s) { return reinterpret_cast<int32_t*>(smem + s * C::STAGE_BYTES + C::DELTA_BYTES); };
    auto issue = [&](int s, int64_t tile) {
        int64_t e0 = tile * TILE;
        int64_t nv = n - e0 < TILE ? n - e0 : TILE;
        unsigned db = (unsigned)((nv * LD * (int64_t)sizeof(T) + 15) / 16 * 16);
        unsigned rb = (unsigned)((nv * 4 + 15) / 16 * 16);
        mbar_expect_tx(&bar[s], db + rb);
        bulk_g2s(stage_delta(s), delta + e0 * LD, db, &bar[s]);
        bulk_g2s(stage_rid(s), rid + e0, rb, &bar[s]);
    };

    if (tid == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        fence_mbar_init();
        sAbort = 0;
    }
    __syncthreads();
    const int64_t t0 = blockIdx.x;
    const int64_t gs = gridDim.x;
    if (tid == 0) {
        if (t0 < ntiles) issue(0, t0);
        if (t0 + gs < ntiles) issue(1, t0 + gs);
    }
    int k = 0;
    for (int64_t tile = t0; tile < ntiles; tile += gs, ++k) {
        const int s = k & 1;
        const unsigned parity = (k >> 1) & 1;
        if (!mbar_wait_bounded(&bar[s], parity, flags)) sAbort = 1;
        __syncthreads();
        if (sAbort) break;
        const T* sd = stage_delta(s);
        const int32_t* sr = stage_rid(s);
        const int64_t e0 = tile * TILE;
        const int nvalid = (int)(n - e0 < TILE ? n - e0 : TILE);
        const int prev = e0 > 0 ? rid[e0 - 1] : -1;
        const int next = e0 + nvalid < n ? rid[e0 + nvalid] : -1;

        // ---- phase 1: per-thread runs -------------------------------------
        const int r0 = tid * RUN;
        const int r1 = r0 + RUN < nvalid ? r0 + RUN : nvalid;
        T acc[NOUT];
        int hasL = 0, hasR = 0, Lrow = -1, Rrow = -1, Lpass = 0;
        if (r0 < nvalid) {
            const int before_row = r0 == 0 ? prev : sr[r0 - 1];
            const int after_row = r1 == nvalid ? next : sr[r1];
#pragma unroll
            for (int q = 0; q < NOUT; ++q) acc[q] = T(0);
            int cur = sr[r0];
            int ps = r0;
            auto flush = [&](int pe) {
                const bool bf = (ps == r0) && (cur == before_row);
                const bool af = (pe == r1) && (cur == after_row);
                if (!bf && !af) {
                    T* dst = rowbuf + (int64_t)cur * NOUT;
#pragma unroll
                    for (int q = 0; q < NOUT; ++q) dst[q] = acc[q];
                } else if (bf) {
                    hasL = 1;
                    Lrow = cur;
                    Lpass = af ? 1 : 0;
#pragma unroll
                    for (int q = 0; q < NOUT; ++q) sLslot[tid * NOUT + q] = acc[q];
                } else {
                    hasR = 1;
                    Rrow = cur;
                }
            };
            for (int i = r0; i < r1; ++i) {
                const int row = sr[i];
                if (row != cur) {
                    flush(i);
#pragma unroll
                    for (int q = 0; q < NOUT; ++q) acc[q] = T(0);
                    cur = row;
                    ps = i;
                }
                T d[J];
#pragma unroll
                for (int j = 0; j < J; ++j) d[j] = sd[i * LD + j];
                const T x = sd[i * LD + J];
                int q = 0;
#pragma unroll
                for (int j = 0; j < J; ++j) {
#pragma unroll
                    for (int kk = j; kk < J; ++kk) {
                        acc[q] = fma(d[j], d[kk], acc[q]);
                        ++q;
                    }
                }
#pragma unroll
                for (int j = 0; j < J; ++j) acc[NTRI + j] = fma(x, d[j], acc[NTRI + j]);
            }
            flush(r1);
        }
        sHasL[tid] = hasL;
        sHasR[tid] = hasR;
        sLrow[tid] = Lrow;
        sRrow[tid] = Rrow;
        sLpass[tid] = Lpass;
        __syncthreads();  // every thread is done reading stage s
        T* sRslot = stage_delta(s);  // reuse the consumed tile for the right pieces
        if (hasR) {
#pragma unroll
            for (int q = 0; q < NOUT; ++q) sRslot[tid * NOUT + q] = acc[q];
        }
        __syncthreads();

        // ---- phase 2: ordered combine of run-crossing pieces ---------------
        for (int p = tid; p < NOUT; p += NT) {
            T cs = T(0), cc = T(0);
            int active = 0, before = 0, crow = -1;
            for (int t = 0; t < NT; ++t) {
                if (sHasL[t]) {
                    if (!active) {
                        active = 1;
                        before = 1;
                        cs = T(0);
                        cc = T(0);
                        crow = sLrow[t];
                    }
                    kahan_add(cs, cc, sLslot[t * NOUT + p]);
                    if (!sLpass[t]) {
                        if (before)
                            reinterpret_cast<T*>(out.blkL)[tile * NOUT + p] = cs;
                        else
                            rowbuf[(int64_t)crow * NOUT + p] = cs;
                        active = 0;
                    }
                }
                if (sHasR[t]) {
                    active = 1;
                    before = 0;
                    cs = sRslot[t * NOUT + p];
                    cc = T(0);
                    crow = sRrow[t];
                }
            }
            if (active) {
                if (before)
                    reinterpret_cast<T*>(out.blkL)[tile * NOUT + p] = cs;
                else
                    reinterpret_cast<T*>(out.blkR)[tile * NOUT + p] = cs;
            }
        }
        if (tid == 0) {
            // tile-level edge rows (same walk over the flags only)
            int active = 0, before = 0, crow = -1, lrow = -1, lpass = 0, rrow = -1;
            for (int t = 0; t < NT; ++t) {
                if (sHasL[t]) {
                    if (!active) {
                        active = 1;
                        before = 1;
                        crow = sLrow[t];
                    }
                    if (!sLpass[t]) {
                        if (before) {
                            lrow = crow;
                            lpass = 0;
                        }
                        active = 0;
                    }
                }
                if (sHasR[t]) {
                    active = 1;
                    before = 0;
                    crow = sRrow[t];
                }
            }
            if (active) {
                if (before) {
                    lrow = crow;
                    lpass = 1;
                } else {
                    rrow = crow;
                }
            }
            out.blkLrow[tile] = lrow;
            out.blkLpass[tile] = lpass;
            out.blkRrow[tile] = rrow;
        }
        __syncthreads();  // stage s (and its right slots) is free again
        if (tid == 0 && tile + 2 * gs < ntiles) issue(s, tile + 2 * gs);
    }
    if (sAbort && tid == 0) {
        // drain whatever is still in flight before leaving (bounded)
        mbar_wait_bounded(&bar[0], 0, nullptr, 1 << 20);
        mbar_wait_bounded(&bar[1], 0, nullptr, 1 << 20);
    }
}

// Rows that cross tile boundaries: right piece of the first tile plus the
// left pieces of the following tiles, summed in FP64 in tile order.
template <typename T>
__global__ void gram_fixup(GramOut out, const int64_t* __restrict__ row_ptr, int64_t ntiles, int tile_entries,
                           int nout) {
    const int64_t b = blockIdx.x;
    const int r = out.blkLrow[b];
    if (r < 0 || out.blkLpass[b]) return;
    const int64_t b0 = row_ptr[r] / tile_entries;
    const T* L = reinterpret_cast<const T*>(out.blkL);
    const T* R = reinterpret_cast<const T*>(out.blkR);
    T* rowbuf = reinterpret_cast<T*>(out.rowbuf);
    for (int p = threadIdx.x; p < nout; p += blockDim.x) {
        double s = (double)R[b0 * nout + p];
        for (int64_t bb = b0 + 1; bb <= b; ++bb) s += (double)L[bb * nout + p];
        rowbuf[(int64_t)r * nout + p] = (T)s;
    }
}

template <typename T, int J>
ptk_status launch(ptk_ctx* ctx, const GramJob& job, cudaStream_t st) {
    using C = Cfg<T, J>;
    if (job.ld != C::LD) {
        set_error("gram: Delta row length %d, expected %d", job.ld, C::LD);
        return PTK_ERR_INVALID_ARG;
    }
    const int64_t ntiles = ceil_div(job.n, C::TILE);
    const int nout = C::NOUT;
    size_t part_bytes = sizeof(T) * (size_t)ntiles * nout;
    char* part = (char*)scratch(ctx, SLOT_PARTIAL, 2 * part_bytes + 64);
    int* prow = (int*)scratch(ctx, SLOT_PARTIAL_ROW, sizeof(int) * 3 * (size_t)ntiles + 64);
    if (!part || !prow) return PTK_ERR_OUT_OF_MEMORY;
    GramOut o;
    o.rowbuf = job.rowbuf;
    o.blkL = part;
    o.blkR = part + part_bytes;
    o.blkLrow = prow;
    o.blkLpass = prow + ntiles;
    o.blkRrow = prow + 2 * ntiles;
    auto kern = gram_kernel<T, J>;
    PTK_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, C::SMEM));
    int per_sm = 1;
    PTK_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, C::NT, C::SMEM));
    if (per_sm < 1) per_sm = 1;
    int64_t grid = std::min<int64_t>(ntiles, (int64_t)ctx->sm_count * per_sm);
    { kern<<<(unsigned)grid, C::NT, C::SMEM, st>>>((const T*)job.delta, job.rid, job.n, ntiles, o, ctx->d_flags); ::ptk::note_launch(); }
    PTK_LAUNCH_CHECK();
    { gram_fixup<T><<<(unsigned)ntiles, 128, 0, st>>>(o, job.row_ptr, ntiles, C::TILE, nout); ::ptk::note_launch(); }
    PTK_LAUNCH_CHECK();
    return PTK_OK;
}

template <typename T>
ptk_status dispatch(ptk_ctx* ctx, const GramJob& job, cudaStream_t st) {
    switch (job.J) {
#define PTK_CASE(J) \
    case J:         \
        return launch<T, J>(ctx, job, st);
        PTK_CASE(1) PTK_CASE(2) PTK_CASE(3) PTK_CASE(4) PTK_CASE(5) PTK_CASE(6) PTK_CASE(7) PTK_CASE(8)
        PTK_CASE(9) PTK_CASE(10) PTK_CASE(11) PTK_CASE(12) PTK_CASE(13) PTK_CASE(14) PTK_CASE(15) PTK_CASE(16)
#undef PTK_CASE
        default:
            set_error("gram: J=%d unsupported", job.J);
            return PTK_ERR_UNSUPPORTED;
    }
}

}  // namespace

ptk_status gram(ptk_ctx* ctx, const GramJob& job, cudaStream_t st) {
    if (job.n == 0) return PTK_OK;
    if (job.dtype == PTK_F64) return dispatch<double>(ctx, job, st);
    return dispatch<float>(ctx, job, st);
}

}  // namespace ptk
