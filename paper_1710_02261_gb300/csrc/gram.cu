// gram.cu -- Eqs. (rowB) and (rowC): for every row i of mode n,
//     B_i = sum_{alpha in Omega_i} delta_alpha delta_alpha^T   (upper triangle)
//     c_i = sum_{alpha in Omega_i} x_alpha delta_alpha
// over the slice-ordered Delta rows [delta_0..delta_{J-1}, x] written by the
// delta kernels.
//
// Accuracy.  lambda (0.01 in the paper) is tiny next to ||B_i|| when delta is
// large, and rows with fewer than J entries have a rank-deficient B_i, so a
// plain FP32 sum (error ~ eps * ||B_i||) can swamp lambda and make B_i + lambda I
// indefinite.  FP32 sums are therefore kept in double-float form: each product
// is split into its rounded value and exact error (TwoProduct with an FMA), each
// addition into its rounded sum and exact error (TwoSum), and the errors are
// gathered in a low word, so a sum is a pair (s, lo) with value s + lo and an
// error of order eps^2 * sum|terms| (as if summed in twice the precision).  The
// FP64 path (model dtype double) accumulates in plain FP64.
//
// Work split.  Slices are uneven (Zipf heads hold >10^6 entries, the smallest
// rows one), so the work is split by ENTRIES, not rows -- the GPU counterpart of
// the paper's dynamic scheduling over rows (Sec. 3.4):
//   * a block owns a tile of TILE consecutive entries, copied into shared
//     memory by the TMA engine (cp.async.bulk, double buffered);
//   * four threads walk the same RUN consecutive entries, each keeping its
//     share of the current row's sums in registers and updating them in
//     pairs with packed FP32x2 instructions (gram_plan.cuh); a row complete
//     inside the run is written straight to the row buffer;
//   * pieces of rows that cross run boundaries go to per-block slots and are
//     merged by a column-parallel ordered scan (a plain ordered sum for tiles
//     inside one row); pieces that cross tile boundaries are merged by a
//     second kernel.
// Every sum is taken in a fixed order, so results are deterministic.
//
// gram_rows is the row-per-warp mapping of Sec. 3.4's scheduling: taken for
// modes whose rows are all short next to a warp's share of the entries
// (PTK_SCHED_AUTO), and selectable for measurement (ptk_schedule).
#include <type_traits>

#include "common.cuh"
#include "gram_plan.cuh"

namespace ptk {

int gram_nout(int J) { return J * (J + 1) / 2 + J; }

namespace {

// ---- accumulators --------------------------------------------------------
struct AccF {  // double-float sum: value = s + lo (Dot2 of Ogita, Rump and Oishi, 2005)
    float s, lo;
    __device__ __forceinline__ void zero() {
        s = 0.f;
        lo = 0.f;
    }
    // The _rn intrinsics keep nvcc from contracting a product and a sum into
    // one FMA, which would break the error-free transformations.
    __device__ __forceinline__ void add_prod(float a, float b) {
        const float p = __fmul_rn(a, b);
        const float e = fmaf(a, b, -p);  // TwoProduct: a*b = p + e exactly
        const float t = __fadd_rn(s, p);  // TwoSum: s + p = t + q exactly
        const float bb = __fsub_rn(t, s);
        const float q = __fadd_rn(__fsub_rn(s, __fsub_rn(t, bb)), __fsub_rn(p, bb));
        s = t;
        lo = __fadd_rn(lo, __fadd_rn(q, e));
    }
    __device__ __forceinline__ void shfl_up(const AccF& v, int off) {
        s = __shfl_up_sync(0xffffffffu, v.s, off);
        lo = __shfl_up_sync(0xffffffffu, v.lo, off);
    }
    __device__ __forceinline__ void shfl_down(const AccF& v, int off) {
        s = __shfl_down_sync(0xffffffffu, v.s, off);
        lo = __shfl_down_sync(0xffffffffu, v.lo, off);
    }
    __device__ __forceinline__ void add(const AccF& o) {
        const float t = __fadd_rn(s, o.s);
        const float bb = __fsub_rn(t, s);
        const float q = __fadd_rn(__fsub_rn(s, __fsub_rn(t, bb)), __fsub_rn(o.s, bb));
        s = t;
        lo = __fadd_rn(lo, __fadd_rn(o.lo, q));
    }
};

struct AccD {
    double s;
    __device__ __forceinline__ void zero() { s = 0.0; }
    __device__ __forceinline__ void add_prod(double a, double b) { s = fma(a, b, s); }
    __device__ __forceinline__ void add(const AccD& o) { s += o.s; }
    __device__ __forceinline__ void shfl_up(const AccD& v, int off) { s = __shfl_up_sync(0xffffffffu, v.s, off); }
    __device__ __forceinline__ void shfl_down(const AccD& v, int off) { s = __shfl_down_sync(0xffffffffu, v.s, off); }
};

// A finished sum as an FP64 value: s + lo rounded once.
__device__ __forceinline__ double to_f64(const AccF& a) { return (double)a.s + (double)a.lo; }
__device__ __forceinline__ double to_f64(const AccD& a) { return a.s; }

template <typename T>
struct AccOf;
template <>
struct AccOf<float> {
    using A = AccF;
};
template <>
struct AccOf<double> {
    using A = AccD;
};

// Two double-float sums updated together by the packed FP32x2 instructions
// (FMUL2 / FFMA2 / FADD2): each lane is rounded exactly as the scalar AccF
// update, so results are identical to it, with half the instructions.
__device__ __forceinline__ float2 neg2(float2 v) { return make_float2(-v.x, -v.y); }
struct AccF2 {
    float2 s, lo;
    __device__ __forceinline__ void zero() {
        s = make_float2(0.f, 0.f);
        lo = make_float2(0.f, 0.f);
    }
    __device__ __forceinline__ void add_prod(float2 a, float2 b) {
        const float2 p = __fmul2_rn(a, b);
        const float2 e = __ffma2_rn(a, b, neg2(p));
        const float2 t = __fadd2_rn(s, p);
        const float2 bb = __fadd2_rn(t, neg2(s));
        const float2 q = __fadd2_rn(__fadd2_rn(s, neg2(__fadd2_rn(t, neg2(bb)))), __fadd2_rn(p, neg2(bb)));
        s = t;
        lo = __fadd2_rn(lo, __fadd2_rn(q, e));
    }
    __device__ __forceinline__ AccF lane(int y) const {
        AccF r;
        r.s = y ? s.y : s.x;
        r.lo = y ? lo.y : lo.x;
        return r;
    }
};

// The sums one thread keeps for a run: FP32 as packed double-float pairs
// (PackPlan), FP64 as one plain sum per output of the thread's chunk.
template <typename T, int J, int PART>
struct RunSums;

template <int J, int PART>
struct RunSums<float, J, PART> {
    static constexpr int NP = PackPlan<J>().np[PART];
    AccF2 acc[NP > 0 ? NP : 1];
    __device__ __forceinline__ void zero() {
#pragma unroll
        for (int q = 0; q < NP; ++q) acc[q].zero();
    }
    __device__ __forceinline__ void add(const float* d) {  // d[0..J-1] = delta, d[J] = x
        constexpr PackPlan<J> plan{};
#pragma unroll
        for (int q = 0; q < NP; ++q)
            acc[q].add_prod(make_float2(d[plan.a0[PART][q]], d[plan.a1[PART][q]]),
                            make_float2(d[plan.b0[PART][q]], d[plan.b1[PART][q]]));
    }
    // out[g * stride] = sum of output g, for this thread's outputs
    __device__ __forceinline__ void store(AccF* out, int64_t stride) const {
        constexpr PackPlan<J> plan{};
#pragma unroll
        for (int q = 0; q < NP; ++q) {
            out[plan.g0[PART][q] * stride] = acc[q].lane(0);
            if (plan.g1[PART][q] >= 0) out[plan.g1[PART][q] * stride] = acc[q].lane(1);
        }
    }
};

template <int J, int PART>
struct RunSums<double, J, PART> {
    static constexpr int NOUT = J * (J + 1) / 2 + J, NTRI = J * (J + 1) / 2;
    static constexpr int CH = (NOUT + 3) / 4;
    AccD acc[CH];
    __device__ __forceinline__ void zero() {
#pragma unroll
        for (int q = 0; q < CH; ++q) acc[q].zero();
    }
    __device__ __forceinline__ void add(const double* d) {
        constexpr Tri<J> tri;
#pragma unroll
        for (int q = 0; q < CH; ++q) {
            const int g = PART * CH + q;
            if (g < NTRI)
                acc[q].add_prod(d[tri.j[g]], d[tri.k[g]]);
            else if (g < NOUT)
                acc[q].add_prod(d[J], d[g - NTRI]);
        }
    }
    __device__ __forceinline__ void store(AccD* out, int64_t stride) const {
#pragma unroll
        for (int q = 0; q < CH; ++q)
            if (PART * CH + q < NOUT) out[(PART * CH + q) * stride] = acc[q];
    }
};

// ---- configuration ----------------------------------------------------------
template <typename T, int J>
struct Cfg {
    using A = typename AccOf<T>::A;
    static constexpr int NOUT = J * (J + 1) / 2 + J;
    static constexpr int NTRI = J * (J + 1) / 2;
    static constexpr int LD = ((J + 1) & 1) ? (J + 1) : (J + 2);
    static constexpr int RUN = 15;  // odd: conflict-free per-thread row walks
    static constexpr int S = 4;     // threads per run, each with a share of the NOUT sums
    static constexpr int stage_for(int nrun) {
        return (nrun * RUN * LD * (int)sizeof(T) + nrun * RUN * 4 + 127) / 128 * 128;
    }
    static constexpr int BUDGET = 200 * 1024;
    static constexpr int NRUN = 2 * stage_for(64) <= BUDGET ? 64 : 32;  // runs per tile
    static constexpr int RPL = NRUN / 32;                               // runs per lane in the merge
    static constexpr int NTH = NRUN * S;
    static constexpr int TILE = NRUN * RUN;
    static constexpr int DELTA_BYTES = TILE * LD * (int)sizeof(T);
    static constexpr int STAGE_BYTES = stage_for(NRUN);
    static constexpr int SMEM = 2 * STAGE_BYTES;
    static_assert(SMEM <= BUDGET, "gram tile does not fit in shared memory");
    static_assert((TILE * LD * (int)sizeof(T)) % 16 == 0, "bulk copies need 16-byte multiples");
    static_assert(TILE % 4 == 0, "tile starts must stay 16-byte aligned");
};

struct GramOut {
    void* rowbuf;      // [rows][NOUT] accumulators
    void* blkL;        // [ntiles][NOUT] accumulators
    void* blkR;        // [ntiles][NOUT]
    int* blkLrow;      // [ntiles] row of the left partial, -1 if none
    int* blkLpass;     // [ntiles] 1 if the left row passes through the whole tile
    int* blkRrow;      // [ntiles]
    void* slots;       // [grid][2][NOUT][NRUN] accumulators (run-crossing pieces)
};

// Phase 1 for a thread of chunk PART: walk the run's entries in order,
// keeping the sums of the current row; a row complete inside the run goes to
// the row buffer, pieces that touch the run's ends to the block's slots.
template <typename T, int J, int PART>
__device__ __forceinline__ void walk_run(const T* sd, const int32_t* sr, int r0, int r1, int before_row,
                                         int after_row, typename Cfg<T, J>::A* rowbuf,
                                         typename Cfg<T, J>::A* slotL, typename Cfg<T, J>::A* slotR, int run,
                                         int& hasL, int& hasR, int& Lrow, int& Rrow, int& Lpass) {
    using C = Cfg<T, J>;
    constexpr int NOUT = C::NOUT, LD = C::LD, NRUN = C::NRUN;
    RunSums<T, J, PART> acc;
    acc.zero();
    int cur = sr[r0];
    int ps = r0;
    auto flush = [&](int pe) {
        const bool bf = (ps == r0) && (cur == before_row);
        const bool af = (pe == r1) && (cur == after_row);
        if (!bf && !af) {
            acc.store(rowbuf + (int64_t)cur * NOUT, 1);
        } else if (bf) {
            hasL = 1;
            Lrow = cur;
            Lpass = af ? 1 : 0;
            acc.store(slotL + run, NRUN);
        } else {
            hasR = 1;
            Rrow = cur;
        }
    };
    for (int i = r0; i < r1; ++i) {
        const int row = sr[i];
        if (row != cur) {
            flush(i);
            acc.zero();
            cur = row;
            ps = i;
        }
        T d[J + 1];  // delta, then x
#pragma unroll
        for (int j = 0; j <= J; ++j) d[j] = sd[i * LD + j];
        acc.add(d);
    }
    flush(r1);
    if (hasR) acc.store(slotR + run, NRUN);
}

template <typename T, int J>
__global__ void __launch_bounds__(Cfg<T, J>::NTH) gram_kernel(const T* __restrict__ delta,
                                                              const int32_t* __restrict__ rid, int64_t n,
                                                              int64_t ntiles, GramOut out, int* flags) {
    using C = Cfg<T, J>;
    using A = typename C::A;
    constexpr int NOUT = C::NOUT, LD = C::LD, RUN = C::RUN, NRUN = C::NRUN, TILE = C::TILE;
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ uint64_t bar[2];
    __shared__ int sHasL[NRUN], sHasR[NRUN], sLrow[NRUN], sRrow[NRUN], sLpass[NRUN];
    __shared__ int sAbort;
    __shared__ int sTileL, sTilePass, sTileR;
    const int tid = threadIdx.x;
    const int run = tid % NRUN;   // entries [run*RUN, run*RUN+RUN) of the tile
    const int part = tid / NRUN;  // which of the run's four threads (its outputs: RunSums)
    A* rowbuf = reinterpret_cast<A*>(out.rowbuf);
    A* slotL = reinterpret_cast<A*>(out.slots) + (int64_t)blockIdx.x * 2 * NOUT * NRUN;  // [NOUT][NRUN]
    A* slotR = slotL + NOUT * NRUN;

    auto stage_delta = [&](int s) { return reinterpret_cast<T*>(smem + s * C::STAGE_BYTES); };
    auto stage_rid = [&](int s) { return reinterpret_cast<int32_t*>(smem + s * C::STAGE_BYTES + C::DELTA_BYTES); };
    auto issue = [&](int s, int64_t tile) {
        const int64_t e0 = tile * TILE;
        const int64_t nv = n - e0 < TILE ? n - e0 : TILE;
        const unsigned db = (unsigned)((nv * LD * (int64_t)sizeof(T) + 15) / 16 * 16);
        const unsigned rb = (unsigned)((nv * 4 + 15) / 16 * 16);
        mbar_expect_tx(&bar[s], db + rb);
        bulk_g2s(stage_delta(s), delta + e0 * LD, db, &bar[s]);
        bulk_g2s(stage_rid(s), rid + e0, rb, &bar[s]);
    };

    if (tid == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        fence_mbar_init();
        sAbort = 0;
        sTileL = -1;
        sTilePass = 0;
        sTileR = 0;
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
        const int64_t e0 = tile * TILE;
        const int nvalid = (int)(n - e0 < TILE ? n - e0 : TILE);
        // neighbouring row ids (issued before the wait so their latency overlaps it)
        const int prev = e0 > 0 ? __ldg(rid + e0 - 1) : -1;
        const int next = e0 + nvalid < n ? __ldg(rid + e0 + nvalid) : -1;
        if (!mbar_wait_bounded(&bar[s], parity, flags)) sAbort = 1;
        __syncthreads();
        if (sAbort) break;
        const T* sd = stage_delta(s);
        const int32_t* sr = stage_rid(s);
        // a tile strictly inside one row (the row began before it and goes on
        // after it): every run's piece passes through, and phase 2 is a plain
        // ordered sum of the runs (rows are sorted, so equal ends mean one row)
        const int row0 = sr[0];
        const bool interior = prev == row0 && next == row0 && sr[nvalid - 1] == row0;

        // ---- phase 1: per-thread runs -------------------------------------
        const int r0 = run * RUN;
        const int r1 = r0 + RUN < nvalid ? r0 + RUN : nvalid;
        int hasL = 0, hasR = 0, Lrow = -1, Rrow = -1, Lpass = 0;
        if (r0 < nvalid) {
            const int before_row = r0 == 0 ? prev : sr[r0 - 1];
            const int after_row = r1 == nvalid ? next : sr[r1];
            switch (part) {
#define PTK_WALK(PP)                                                                                            \
    case PP:                                                                                                    \
        walk_run<T, J, PP>(sd, sr, r0, r1, before_row, after_row, rowbuf, slotL, slotR, run, hasL, hasR, Lrow, \
                           Rrow, Lpass);                                                                        \
        break;
                PTK_WALK(0) PTK_WALK(1) PTK_WALK(2) PTK_WALK(3)
#undef PTK_WALK
            }
        }
        if (part == 0) {
            sHasL[run] = hasL;
            sHasR[run] = hasR;
            sLrow[run] = Lrow;
            sRrow[run] = Rrow;
            sLpass[run] = Lpass;
        }
        __syncthreads();  // stage s consumed; slots and flags written
        if (tid == 0 && tile + 2 * gs < ntiles) issue(s, tile + 2 * gs);

        // ---- phase 2: merge of run-crossing pieces -------------------------
        // One warp per column p.  Lane l folds its RPL runs in order into a
        // (head, tail) summary; the open segment carried across lanes follows
        // the associative rule  carry_out = reset ? b : carry_in + b,  taken as
        // a warp scan (Kogge-Stone) in fixed order.  Interior tiles need only
        // the sum of all runs: lane folds, then a shuffle tree (fixed order).
        if (interior) {
            const int lane = tid & 31, warp = tid >> 5;
            A nv[C::RPL];
            auto load_runs = [&](int pp) {
#pragma unroll
                for (int q = 0; q < C::RPL; ++q) nv[q] = slotL[pp * NRUN + lane * C::RPL + q];
            };
            if (warp < NOUT) load_runs(warp);
            for (int p = warp; p < NOUT; p += C::NTH / 32) {
                A v;
                v.zero();
#pragma unroll
                for (int q = 0; q < C::RPL; ++q) v.add(nv[q]);
                if (p + C::NTH / 32 < NOUT) load_runs(p + C::NTH / 32);
#pragma unroll
                for (int off = 16; off > 0; off >>= 1) {
                    A o;
                    o.shfl_down(v, off);
                    if (lane < off) v.add(o);
                }
                if (lane == 0) reinterpret_cast<A*>(out.blkL)[tile * NOUT + p] = v;
            }
            if (tid == 0) {
                sTileL = row0;
                sTilePass = 1;
            }
        } else {
            const int lane = tid & 31, warp = tid >> 5;
            const bool open0 = sHasL[0] != 0;  // a row that started before the tile
            // slot values of the next column are loaded while this one is scanned
            A nL[C::RPL], nR[C::RPL];
            auto load_slots = [&](int pp) {
#pragma unroll
                for (int q = 0; q < C::RPL; ++q) {
                    const int t = lane * C::RPL + q;
                    if (sHasL[t]) nL[q] = slotL[pp * NRUN + t];
                    if (sHasR[t]) nR[q] = slotR[pp * NRUN + t];
                }
            };
            if (warp < NOUT) load_slots(warp);
            for (int p = warp; p < NOUT; p += C::NTH / 32) {
                A vL[C::RPL], vR[C::RPL];
#pragma unroll
                for (int q = 0; q < C::RPL; ++q) {
                    vL[q] = nL[q];
                    vR[q] = nR[q];
                }
                if (p + C::NTH / 32 < NOUT) load_slots(p + C::NTH / 32);
                A head, tail;
                head.zero();
                tail.zero();
                bool has_end = false, open = false;
                int end_row = -1, open_row = -1;
#pragma unroll
                for (int q = 0; q < C::RPL; ++q) {
                    const int t = lane * C::RPL + q;
                    if (sHasL[t]) {
                        const A v = vL[q];
                        if (!open) {
                            head.add(v);
                            if (!sLpass[t]) {
                                has_end = true;
                                end_row = sLrow[t];
                            }
                        } else {
                            tail.add(v);
                            if (!sLpass[t]) {  // opened and closed inside this lane
                                rowbuf[(int64_t)open_row * NOUT + p] = tail;
                                open = false;
                                tail.zero();
                            }
                        }
                    }
                    if (sHasR[t]) {
                        open = true;
                        open_row = sRrow[t];
                        tail = vR[q];
                    }
                }
                // scan element: reset lanes restart the carry with b
                A b = open ? tail : head;
                if (has_end && !open) b.zero();
                int r = (has_end || open) ? 1 : 0;
                int o = open ? 1 : 0;
#pragma unroll
                for (int off = 1; off < 32; off <<= 1) {
                    A pb;
                    pb.shfl_up(b, off);
                    const int pr = __shfl_up_sync(0xffffffffu, r, off);
                    const int po = __shfl_up_sync(0xffffffffu, o, off);
                    if (lane >= off && !r) {
                        pb.add(b);
                        b = pb;
                        r = pr;
                        o = po;
                    }
                }
                // exclusive carry into this lane; lane 0 starts from the tile start
                A cin;
                cin.shfl_up(b, 1);
                int rin = __shfl_up_sync(0xffffffffu, r, 1);
                if (lane == 0) {
                    cin.zero();
                    rin = 0;
                }
                if (has_end) {
                    A tot = cin;
                    tot.add(head);
                    if (!rin)  // the carried segment began before this tile
                        reinterpret_cast<A*>(out.blkL)[tile * NOUT + p] = tot;
                    else
                        rowbuf[(int64_t)end_row * NOUT + p] = tot;
                    if (p == 0 && !rin) {
                        sTileL = end_row;
                        sTilePass = 0;
                    }
                }
                // state after the whole tile (lane 31, combined with the tile start)
                if (lane == 31) {
                    const A fin = b;
                    const int fr = r;
                    const int fo = fr ? o : (open0 ? 1 : 0);  // no reset: the tile-start state
                    if (fo) {
                        if (fr) {
                            reinterpret_cast<A*>(out.blkR)[tile * NOUT + p] = fin;
                            if (p == 0) sTileR = 1;
                        } else {
                            reinterpret_cast<A*>(out.blkL)[tile * NOUT + p] = fin;
                            if (p == 0) {
                                sTileL = sLrow[0];
                                sTilePass = 1;
                            }
                        }
                    }
                }
            }
        }
        __syncthreads();
        if (tid == 0) {
            // the open segment at the tile end was opened by the last right piece
            int rrow = -1;
            if (sTileR)
                for (int t = NRUN - 1; t >= 0; --t)
                    if (sHasR[t]) {
                        rrow = sRrow[t];
                        break;
                    }
            out.blkLrow[tile] = sTileL;
            out.blkLpass[tile] = sTilePass;
            out.blkRrow[tile] = rrow;
            sTileL = -1;
            sTilePass = 0;
            sTileR = 0;
        }
        __syncthreads();  // slots and flags free for the next tile
    }
    if (sAbort && tid == 0) {
        // let whatever is still in flight land before leaving (bounded)
        mbar_wait_bounded(&bar[0], 0, nullptr, 1 << 20);
        mbar_wait_bounded(&bar[1], 0, nullptr, 1 << 20);
    }
}

// Rows that cross tile boundaries: right piece of the first tile plus the left
// pieces of the following tiles.  Four threads per column take every fourth
// piece (16 loads issued back to back), then the four partials are added in order.
template <typename T, int J>
__global__ void __launch_bounds__(256) gram_fixup(GramOut out, const int64_t* __restrict__ row_ptr, int64_t ntiles) {
    using C = Cfg<T, J>;
    using A = typename C::A;
    __shared__ A part[4][C::NOUT];
    const int64_t b = blockIdx.x;
    const int r = out.blkLrow[b];
    if (r < 0 || out.blkLpass[b]) return;
    const int64_t b0 = row_ptr[r] / C::TILE;
    const int64_t m = b - b0 + 1;  // pieces: R[b0], L[b0+1], ..., L[b]
    const A* L = reinterpret_cast<const A*>(out.blkL);
    const A* R = reinterpret_cast<const A*>(out.blkR);
    A* rowbuf = reinterpret_cast<A*>(out.rowbuf);
    for (int t = threadIdx.x; t < 4 * C::NOUT; t += blockDim.x) {
        const int p = t % C::NOUT, q = t / C::NOUT;
        A s;
        s.zero();
        int64_t i = q;
        constexpr int U = 16;  // pieces in flight per thread (a Zipf head row spans > 10^3 tiles)
        for (; i + 4 * (U - 1) < m; i += 4 * U) {
            A v[U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int64_t k = i + 4 * u;
                v[u] = k == 0 ? R[b0 * C::NOUT + p] : L[(b0 + k) * C::NOUT + p];
            }
#pragma unroll
            for (int u = 0; u < U; ++u) s.add(v[u]);
        }
        for (; i < m; i += 4) s.add(i == 0 ? R[b0 * C::NOUT + p] : L[(b0 + i) * C::NOUT + p]);
        part[q][p] = s;
    }
    __syncthreads();
    for (int p = threadIdx.x; p < C::NOUT; p += blockDim.x) {
        A s = part[0][p];
        s.add(part[1][p]);
        s.add(part[2][p]);
        s.add(part[3][p]);
        rowbuf[(int64_t)r * C::NOUT + p] = s;
    }
}

// ---- row schedules ------------------------------------------------------------
// Sec. 3.4 hands whole rows to threads (dynamic scheduling, because slice sizes
// are uneven).  These kernels are that mapping on a GPU, kept to measure it
// against the entry split above: one warp owns a row, lane l keeps the sums of
// outputs l, l+32, ..., and the row's entries are walked in slice order, UNR at
// a time: lane k < LD loads element k of each entry's Delta row and every lane
// takes its two operands by shuffles.  Rows go to warps in turn (row r to warp
// r mod W) or, with DYN, from a counter in global memory.  Every sum is stored
// finished, as its FP64 value (the solve then reads FP64 without converting;
// here the conversions run with all lanes together, once per row).
template <typename T, int J, bool DYN>
__global__ void __launch_bounds__(256) gram_rows(const T* __restrict__ delta, const int64_t* __restrict__ row_ptr,
                                                 int64_t rows, double* __restrict__ rowbuf,
                                                 unsigned long long* __restrict__ next_row, int64_t below) {
    using C = Cfg<T, J>;
    using A = typename C::A;
    constexpr int NOUT = C::NOUT, NTRI = C::NTRI, LD = C::LD;
    constexpr int PER = (NOUT + 31) / 32;
    constexpr int UNR = 4;
    static_assert(LD <= 32, "a Delta row must fit in one warp");
    const int lane = threadIdx.x & 31;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    int oa[PER], ob[PER];  // operand positions in the Delta row (x sits at J)
#pragma unroll
    for (int q = 0; q < PER; ++q) {
        const int g = lane + 32 * q;
        oa[q] = 0;
        ob[q] = 0;
        if (g < NTRI) {
            int a = 0, first = 0;
            while (g >= first + (J - a)) {
                first += J - a;
                ++a;
            }
            oa[q] = a;
            ob[q] = a + (g - first);
        } else if (g < NOUT) {
            oa[q] = J;
            ob[q] = g - NTRI;
        }
    }
    auto take = [&]() -> int64_t {
        unsigned long long v = 0;
        if (lane == 0) v = atomicAdd(next_row, 1ull);
        return (int64_t)__shfl_sync(0xffffffffu, v, 0);
    };
    int64_t r = DYN ? take() : ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    while (r < rows) {
        const int64_t b = row_ptr[r], e = row_ptr[r + 1];
        if (e > b && (below <= 0 || e - b < below)) {  // rows of `below` entries or more: tensor-core Gram
            // FP32: outputs q and q+1 of a lane are updated together by the packed
            // FP32x2 form (lanes without a valid output compute on index 0 and
            // never store)
            constexpr bool PK = std::is_same<T, float>::value;
            constexpr int NPK = PK ? PER / 2 : 0;  // packed pairs (outputs 2m, 2m+1)
            AccF2 acc2[NPK > 0 ? NPK : 1];
            A acc[PER];
#pragma unroll
            for (int m = 0; m < NPK; ++m) acc2[m].zero();
#pragma unroll
            for (int q = 2 * NPK; q < PER; ++q) acc[q].zero();
            for (int64_t i = b; i < e; i += UNR) {
                T v[UNR];
#pragma unroll
                for (int u = 0; u < UNR; ++u) v[u] = (lane < LD && i + u < e) ? delta[(i + u) * LD + lane] : T(0);
#pragma unroll
                for (int u = 0; u < UNR; ++u) {
                    if (i + u >= e) break;  // the same for the whole warp
#pragma unroll
                    for (int m = 0; m < NPK; ++m) {
                        const float x0 = __shfl_sync(0xffffffffu, (float)v[u], oa[2 * m]);
                        const float x1 = __shfl_sync(0xffffffffu, (float)v[u], oa[2 * m + 1]);
                        const float y0 = __shfl_sync(0xffffffffu, (float)v[u], ob[2 * m]);
                        const float y1 = __shfl_sync(0xffffffffu, (float)v[u], ob[2 * m + 1]);
                        acc2[m].add_prod(make_float2(x0, x1), make_float2(y0, y1));
                    }
#pragma unroll
                    for (int q = 2 * NPK; q < PER; ++q) {
                        const T x = __shfl_sync(0xffffffffu, v[u], oa[q]);
                        const T y = __shfl_sync(0xffffffffu, v[u], ob[q]);
                        if (lane + 32 * q < NOUT) acc[q].add_prod(x, y);
                    }
                }
            }
            if constexpr (PK) {
#pragma unroll
                for (int m = 0; m < NPK; ++m)
#pragma unroll
                    for (int y = 0; y < 2; ++y)
                        if (lane + 32 * (2 * m + y) < NOUT)
                            rowbuf[r * NOUT + lane + 32 * (2 * m + y)] = to_f64(acc2[m].lane(y));
            }
#pragma unroll
            for (int q = 2 * NPK; q < PER; ++q)
                if (lane + 32 * q < NOUT) rowbuf[r * NOUT + lane + 32 * q] = to_f64(acc[q]);
        }
        r = DYN ? take() : r + nwarps;
    }
}

template <typename T, int J>
int64_t rows_grid(ptk_ctx* ctx, const GramJob& job, bool dyn) {
    int per_sm = 1;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, dyn ? gram_rows<T, J, true> : gram_rows<T, J, false>,
                                                      256, 0) != cudaSuccess || per_sm < 1)
        per_sm = 1;
    return std::max<int64_t>(1, std::min<int64_t>(ceil_div(job.rows, 8), (int64_t)ctx->sm_count * per_sm));
}

template <typename T, int J>
ptk_status launch_rows(ptk_ctx* ctx, const GramJob& job, cudaStream_t st) {
    using A = typename Cfg<T, J>::A;
    const bool dyn = job.schedule == PTK_SCHED_ROWS_DYNAMIC;
    auto kern = dyn ? gram_rows<T, J, true> : gram_rows<T, J, false>;
    const int64_t grid = rows_grid<T, J>(ctx, job, dyn);
    auto* next_row = (unsigned long long*)scratch(ctx, SLOT_PARTIAL_ROW, 64);
    if (!next_row) return PTK_ERR_OUT_OF_MEMORY;
    if (dyn) PTK_CUDA(cudaMemsetAsync(next_row, 0, sizeof(unsigned long long), st));
    { kern<<<(unsigned)grid, 256, 0, st>>>((const T*)job.delta, job.row_ptr, job.rows, (double*)job.rowbuf, next_row,
                                           job.rows_below); ::ptk::note_launch(); }
    PTK_LAUNCH_CHECK();
    if (job.wrote_f64) *job.wrote_f64 = 1;
    return PTK_OK;
}

template <typename T, int J>
ptk_status launch(ptk_ctx* ctx, const GramJob& job, cudaStream_t st) {
    using C = Cfg<T, J>;
    using A = typename C::A;
    if (job.ld != C::LD) {
        set_error("gram: Delta row length %d, expected %d", job.ld, C::LD);
        return PTK_ERR_INVALID_ARG;
    }
    // automatic: the tensor cores when at least half of the entries sit in rows
    // long enough for them (a few long rows among short ones stay on the row kernel)
    const bool tc_auto = gram_tc_supported(job) && 2 * job.tc_long_entries >= job.n;
    if (job.schedule == PTK_SCHED_TENSOR || (job.schedule == PTK_SCHED_AUTO && tc_auto)) {
        // long rows on the tensor cores, the others one per warp
        if (!gram_tc_supported(job)) {
            set_error("gram: the tensor-core schedule needs FP32 sums, J <= 15 and rows of >= %d entries",
                      gram_tc_min_row());
            return PTK_ERR_UNSUPPORTED;
        }
        // the short rows run on the context's side stream beside the tensor-core
        // kernel (which leaves most of each SM's issue slots free)
        const bool fork = job.tc_long_entries < job.n;
        if (fork) {
            PTK_CUDA(cudaEventRecord(ctx->ev_fork, st));
            PTK_CUDA(cudaStreamWaitEvent(ctx->side, ctx->ev_fork, 0));
            GramJob j = job;
            j.schedule = PTK_SCHED_ROWS_STATIC;
            j.rows_below = gram_tc_min_row();
            PTK_TRY(launch_rows<T, J>(ctx, j, ctx->side));
            PTK_CUDA(cudaEventRecord(ctx->ev_join, ctx->side));
        }
        const ptk_status rc = gram_tc(ctx, job, st);
        if (fork) PTK_CUDA(cudaStreamWaitEvent(st, ctx->ev_join, 0));  // joined even if the launch failed
        PTK_TRY(rc);
        if (job.wrote_f64) *job.wrote_f64 = 1;
        return PTK_OK;
    }
    if (job.schedule == PTK_SCHED_AUTO) {
        // whole rows per warp when the longest row is at most a quarter of a
        // warp's even share of the entries (the warps of a full static grid)
        GramJob j = job;
        const int64_t warps = rows_grid<T, J>(ctx, job, false) * 8;
        j.schedule = job.max_row > 0 && job.max_row * 4 * warps <= job.n ? PTK_SCHED_ROWS_STATIC : PTK_SCHED_ENTRIES;
        return launch<T, J>(ctx, j, st);
    }
    if (job.schedule != PTK_SCHED_ENTRIES) return launch_rows<T, J>(ctx, job, st);
    const int64_t ntiles = ceil_div(job.n, C::TILE);
    auto kern = gram_kernel<T, J>;
    PTK_TRY(smem_attr((const void*)kern, C::SMEM, st, true));
    int per_sm = 1;
    PTK_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, C::NTH, C::SMEM));
    if (per_sm < 1) per_sm = 1;
    const int64_t grid = std::min<int64_t>(ntiles, (int64_t)ctx->sm_count * per_sm);
    const size_t part_bytes = sizeof(A) * (size_t)ntiles * C::NOUT;
    const size_t slot_bytes = sizeof(A) * (size_t)grid * 2 * C::NOUT * C::NRUN;
    char* part = (char*)scratch(ctx, SLOT_PARTIAL, 2 * part_bytes + slot_bytes + 64);
    int* prow = (int*)scratch(ctx, SLOT_PARTIAL_ROW, sizeof(int) * 3 * (size_t)ntiles + 64);
    if (!part || !prow) return PTK_ERR_OUT_OF_MEMORY;
    GramOut o;
    o.rowbuf = job.rowbuf;
    o.blkL = part;
    o.blkR = part + part_bytes;
    o.slots = part + 2 * part_bytes;
    o.blkLrow = prow;
    o.blkLpass = prow + ntiles;
    o.blkRrow = prow + 2 * ntiles;
    { kern<<<(unsigned)grid, C::NTH, C::SMEM, st>>>((const T*)job.delta, job.rid, job.n, ntiles, o, ctx->d_flags); ::ptk::note_launch(); }
    PTK_LAUNCH_CHECK();
    { gram_fixup<T, J><<<(unsigned)ntiles, 256, 0, st>>>(o, job.row_ptr, ntiles); ::ptk::note_launch(); }
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

namespace {
template <typename T>
int tile_of(int J) {
    switch (J) {
#define PTK_CASE(JJ) \
    case JJ:         \
        return Cfg<T, JJ>::TILE;
        PTK_CASE(1) PTK_CASE(2) PTK_CASE(3) PTK_CASE(4) PTK_CASE(5) PTK_CASE(6) PTK_CASE(7) PTK_CASE(8)
        PTK_CASE(9) PTK_CASE(10) PTK_CASE(11) PTK_CASE(12) PTK_CASE(13) PTK_CASE(14) PTK_CASE(15) PTK_CASE(16)
#undef PTK_CASE
        default:
            return 1;
    }
}
}  // namespace

int gram_tile_entries(int J, ptk_dtype dtype) { return dtype == PTK_F64 ? tile_of<double>(J) : tile_of<float>(J); }

ptk_status gram(ptk_ctx* ctx, const GramJob& job, cudaStream_t st) {
    if (job.n == 0) return PTK_OK;
    if (job.dtype == PTK_F64) return dispatch<double>(ctx, job, st);
    return dispatch<float>(ctx, job, st);
}

}  // namespace ptk
