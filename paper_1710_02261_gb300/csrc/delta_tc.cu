// delta_tc.cu -- Eq. (delta) on the 5th-generation tensor cores (tcgen05).
//
// For the free mode n, split the other modes into a Kronecker group K (all of
// them but the last) and the last other mode L.  Then
//     delta_e(j_n) = sum_{j_L} a^(L)_{i_L j_L} * D_e(j_n, j_L),
//     D_e(j_n, j_L) = sum_k A_e(k) Gb((j_n, j_L), k),
// where A_e(k) = prod_{m in K} a^(m)_{i_m k_m} is the Kronecker product of the
// entry's K-group factor rows and Gb is the core reshaped to [(j_n, j_L)][k].
// D = A Gb^T is a dense contraction: a 128-entry tile is one
// tcgen05.mma (M = 128, N = J_n*J_L padded to 16, K = prod_{m in K} J_m
// padded to the instruction K) with BF16 or TF32 operands and FP32
// accumulation in tensor memory.  CUDA cores build A (one entry per thread,
// written straight into shared memory in the canonical K-major no-swizzle
// layout) and contract D with the L-mode row after tcgen05.ld.
//
// Pipeline (warp-specialised, persistent): a producer warpgroup gathers the
// entries' factor rows (one tile ahead) and writes A tiles into a ring of
// shared-memory stages; one thread issues the MMAs into four TMEM
// accumulators; two epilogue warpgroups drain them, alternate tiles each.  Gb is
// copied to shared memory once per CTA.  Every wait is bounded: on timeout the
// kernel records FLAG_TIMEOUT, lets issued MMAs land, frees its TMEM and
// returns.
#include "common.cuh"
#include "tc_ptx.cuh"

namespace ptk {
namespace {

constexpr int TC_M = 128;          // entries per tile (MMA M)

__device__ __forceinline__ int64_t ceil_div_dev(int64_t a, int64_t b) { return (a + b - 1) / b; }

using namespace ::ptk::tc;

// ---- shapes -----------------------------------------------------------------
// Layout of a K-major operand with R rows: 16-byte chunks of KPG elements;
// chunk (row, kc) at (row/8)*SBO + kc*128 + (row%8)*16 with SBO = KCH*128.
template <bool TF32>
struct Elt {
    static constexpr int ESZ = TF32 ? 4 : 2;
    static constexpr int KPG = 16 / ESZ;      // elements per 16-byte chunk
    static constexpr int MMA_K = TF32 ? 8 : 16;
};

struct TcParams {
    int64_t n;
    const int32_t* col_k[3];     // coordinate columns of the K-group modes (SoA, 16-byte aligned)
    const float* f_k[3];
    int64_t ld_k[3];
    const int32_t* col_l;        // coordinate column of the L mode
    const float* f_l;
    int64_t ld_l;
    const float* vals;           // x per entry (SoA, 16-byte aligned), or null
    float* out;
    int out_ld;
    const uint8_t* b_image;      // Gb in the shared-memory layout
    int b_bytes;
    int* flags;
    int bulk_out;                // 1: Delta tiles leave through shared memory with bulk copies
};

// shared memory of the kernel for rank J, Kronecker order NK, NS A stages
constexpr int TC_NC = 8;  // coordinate stages (must exceed NS + 2)
constexpr int tc_smem_bytes(int J, int NK, bool tf32, int ns, bool x3 = false) {
    const int esz = tf32 ? 4 : 2, mk = tf32 ? 8 : 16;
    const int parts = x3 ? 2 : 1;  // BF16x3: high and low BF16 parts of A and B
    const int K = NK == 1 ? J : (NK == 2 ? J * J : J * J * J);
    const int KP = (K + mk - 1) / mk * mk;
    const int NP = (J * J + 15) / 16 * 16;
    const int coords = TC_NC * (NK + 2) * TC_M * 4;
    const int outst = 4 * TC_M * (J + 2) * 4;  // Delta tiles staged for bulk stores (two per epilogue group)
    return parts * (NP * KP * esz + ns * (TC_M * KP * esz)) + coords + outst + 128;
}
constexpr int TC_SMEM_BUDGET = 220 * 1024;
constexpr bool tc_fits(int J, int NK, bool tf32, bool x3 = false) {
    return tc_smem_bytes(J, NK, tf32, 2, x3) <= TC_SMEM_BUDGET;
}

template <int J, int NK, bool TF32, bool X3 = false>
struct TcCfg {
    using E = Elt<TF32>;
    static constexpr int K = NK == 1 ? J : (NK == 2 ? J * J : J * J * J);
    static constexpr int KP = (K + E::MMA_K - 1) / E::MMA_K * E::MMA_K;
    static constexpr int KCH = KP / E::KPG;            // 16-byte chunks per row
    static constexpr int NN = J * J;                   // (j_n, j_L) pairs
    static constexpr int NP = (NN + 15) / 16 * 16;     // MMA N
    static constexpr int NCOL = NP <= 32 ? 32 : (NP <= 64 ? 64 : 128);  // TMEM columns per accumulator
    static constexpr int NACC = 4;  // accumulators in TMEM (4 x 128 columns at most = all 512)
    static constexpr int SBO = KCH * 128;
    static constexpr int A_BYTES = TC_M * KP * E::ESZ;
    static constexpr int B_BYTES = NP * KP * E::ESZ;
    static constexpr int CSTAGE = (NK + 2) * TC_M * 4;  // coordinate columns + values of one tile
    static constexpr int NPART = X3 ? 2 : 1;           // BF16x3: A and B held as high and low BF16 parts
    static constexpr int B_TOTAL = NPART * B_BYTES;
    static constexpr int A_STAGE = NPART * A_BYTES;
    static constexpr int NS = tc_smem_bytes(J, NK, TF32, 4, X3) <= TC_SMEM_BUDGET
                                  ? 4
                                  : (tc_smem_bytes(J, NK, TF32, 3, X3) <= TC_SMEM_BUDGET ? 3 : 2);  // A stages
    static constexpr int OUT_BYTES = TC_M * (J + 2) * 4;  // one staged Delta tile (row length <= J + 2)
    static constexpr int SMEM = B_TOTAL + NS * A_STAGE + TC_NC * CSTAGE + 4 * OUT_BYTES + 128;
    static constexpr int KSTEPS = KP / E::MMA_K;
    static_assert(NP <= 128, "accumulator wider than 128 columns");
    static_assert(TC_NC > NS + 2, "coordinate ring too short for the pipeline depth");
    static_assert(SMEM == tc_smem_bytes(J, NK, TF32, NS, X3) && SMEM <= TC_SMEM_BUDGET, "tile does not fit");
    static_assert(!(X3 && TF32), "BF16x3 splits FP32 into BF16 parts");
};

// Roles (14 warps): warps 0-3 are the producer warpgroup (gathers of the
// K-group rows, Kronecker rows, conversion into the A ring); warps 4-7 and
// 8-11 are two epilogue warpgroups taking alternate tiles (L-mode row gather,
// contraction, Delta stores); warp 12 issues the MMAs; warp 13 owns TMEM and
// streams each tile's coordinate columns and values into a ring with 1-D bulk
// copies.  Named barriers 1-4 belong to the epilogue groups (two each).
// Barriers (all waits bounded):
//   cfull[c] / cempty[c]  loader <-> producers + epilogue (256 arrivals)
//   full[s]  / empty[s]   producer <-> MMA (128 arrivals / tcgen05.commit)
//   tfull[a] / tempty[a]  MMA <-> epilogue (tcgen05.commit / 128 arrivals), NACC accumulators
constexpr int TC_ROLE_THREADS = 448;

template <int J, bool VEC>
__device__ __forceinline__ void load_row(const float* __restrict__ r, float* v) {
    if constexpr (VEC) {
#pragma unroll
        for (int q = 0; q < (J + 3) / 4; ++q) {
            const float4 t = __ldg(reinterpret_cast<const float4*>(r) + q);
            if (4 * q + 0 < J) v[4 * q + 0] = t.x;
            if (4 * q + 1 < J) v[4 * q + 1] = t.y;
            if (4 * q + 2 < J) v[4 * q + 2] = t.z;
            if (4 * q + 3 < J) v[4 * q + 3] = t.w;
        }
    } else {
#pragma unroll
        for (int j = 0; j < J; ++j) v[j] = __ldg(r + j);
    }
}

template <int J, int NK, bool TF32, bool VEC, bool X3>
__global__ void __launch_bounds__(TC_ROLE_THREADS, 1) delta_tc_kernel(const TcParams p) {
    using C = TcCfg<J, NK, TF32, X3>;
    using E = typename C::E;
    constexpr int NS = C::NS, NC = TC_NC;
    extern __shared__ __align__(128) uint8_t smem[];
    uint8_t* sB = smem;
    auto sA = [&](int s) { return smem + C::B_TOTAL + s * C::A_STAGE; };  // high part; low part + A_BYTES
    auto sCol = [&](int c, int m) {  // m < NK: K-group columns, NK: L column, NK+1: values
        return reinterpret_cast<int32_t*>(smem + C::B_TOTAL + NS * C::A_STAGE + c * C::CSTAGE + m * TC_M * 4);
    };
    constexpr int NACC = C::NACC;
    __shared__ uint64_t cfull[NC], cempty[NC], full[NS], empty[NS], tfull[NACC], tempty[NACC];
    __shared__ uint32_t tmem_base_s;
    __shared__ int abort_s;

    const int tid = threadIdx.x;
    const int warp = tid >> 5;

    for (int i = tid * 16; i < p.b_bytes; i += TC_ROLE_THREADS * 16)
        *reinterpret_cast<uint4*>(sB + i) = *reinterpret_cast<const uint4*>(p.b_image + i);
    if (tid == 0) {
        for (int c = 0; c < NC; ++c) {
            mbar_init(&cfull[c], 1);
            mbar_init(&cempty[c], 2 * TC_M);
        }
        for (int s = 0; s < NS; ++s) {
            mbar_init(&full[s], TC_M);
            mbar_init(&empty[s], 1);
        }
        for (int a = 0; a < NACC; ++a) {
            mbar_init(&tfull[a], 1);
            mbar_init(&tempty[a], TC_M);
        }
        fence_mbar_init();
        abort_s = 0;
    }
    if (warp == 13) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base_s)),
                     "r"(NACC * C::NCOL)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    fence_proxy_async_smem();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();

    const int64_t ntiles = ceil_div_dev(p.n, TC_M);
    const int64_t t0 = blockIdx.x, ts = gridDim.x;
    const int64_t my_tiles = t0 < ntiles ? (ntiles - 1 - t0) / ts + 1 : 0;
    auto tile_start = [&](int64_t k) { return (t0 + k * ts) * TC_M; };
    auto tile_valid = [&](int64_t k) {
        const int64_t nv = p.n - tile_start(k);
        return (int)(nv < TC_M ? nv : TC_M);
    };

    if (warp < 4) {
        // ---------------- producers ----------------
        const int r = tid & 127;     // row of the tile
        // factor rows of two tiles: tile k's rows are in use while tile k+1's
        // loads are in flight (the two buffers alternate, no copies between them)
        float rk0[NK * J], rk1[NK * J];
        auto gather = [&](int64_t k, float* dst) -> bool {
            const int c = (int)(k % NC);
            if (!mbar_wait_bounded(&cfull[c], (unsigned)((k / NC) & 1), p.flags, 1ll << 24)) return false;
            const bool valid = r < tile_valid(k);
            int32_t co[NK];
#pragma unroll
            for (int m = 0; m < NK; ++m) co[m] = valid ? sCol(c, m)[r] : 0;
            mbar_arrive(&cempty[c]);
#pragma unroll
            for (int m = 0; m < NK; ++m) {
                if (valid)
                    load_row<J, VEC>(p.f_k[m] + (int64_t)co[m] * p.ld_k[m], dst + m * J);
                else
#pragma unroll
                    for (int j = 0; j < J; ++j) dst[m * J + j] = 0.f;
            }
            return true;
        };
        auto build = [&](int64_t k, const float* rk) -> bool {
            const int s = (int)(k % NS);
            if (!mbar_wait_bounded(&empty[s], (unsigned)(((k / NS) & 1) ^ 1), p.flags, 1ll << 24)) return false;
            uint8_t* arow = sA(s) + (r >> 3) * C::SBO + (r & 7) * 16;
#pragma unroll
            for (int kc = 0; kc < C::KCH; ++kc) {
                float v[E::KPG];
#pragma unroll
                for (int t = 0; t < E::KPG; ++t) {
                    const int kk = kc * E::KPG + t;
                    float a = 0.f;
                    if (kk < C::K) {
                        if constexpr (NK == 1) {
                            a = rk[kk];
                        } else if constexpr (NK == 2) {
                            a = rk[kk / J] * rk[J + kk % J];
                        } else {
                            a = rk[kk / (J * J)] * rk[J + (kk / J) % J] * rk[2 * J + kk % J];
                        }
                    }
                    v[t] = a;
                }
                uint4 w;
                if constexpr (TF32) {
                    w = make_uint4(to_tf32(v[0]), to_tf32(v[1]), to_tf32(v[2]), to_tf32(v[3]));
                } else {
                    w = make_uint4(pack_bf16(v[0], v[1]), pack_bf16(v[2], v[3]), pack_bf16(v[4], v[5]),
                                   pack_bf16(v[6], v[7]));
                }
                *reinterpret_cast<uint4*>(arow + kc * 128) = w;
                if constexpr (X3) {
                    // low part: the rounding remainder of the high part, again in BF16
                    float lo[E::KPG];
#pragma unroll
                    for (int t = 0; t < E::KPG; ++t) lo[t] = v[t] - bf16_value(v[t]);
                    *reinterpret_cast<uint4*>(arow + C::A_BYTES + kc * 128) =
                        make_uint4(pack_bf16(lo[0], lo[1]), pack_bf16(lo[2], lo[3]), pack_bf16(lo[4], lo[5]),
                                   pack_bf16(lo[6], lo[7]));
                }
            }
            fence_proxy_async_smem();
            mbar_arrive(&full[s]);
            return true;
        };
        bool ok = my_tiles == 0 || gather(0, rk0);
        for (int64_t k = 0; ok && k < my_tiles; k += 2) {
            if (k + 1 < my_tiles) ok = gather(k + 1, rk1);
            ok = ok && build(k, rk0);
            if (!ok || k + 1 >= my_tiles) break;
            if (k + 2 < my_tiles) ok = gather(k + 2, rk0);
            ok = ok && build(k + 1, rk1);
        }
        if (!ok) abort_s = 1;
    } else if (warp < 12) {
        // ---------------- epilogue ----------------
        // Two warpgroups take alternate tiles (group g: tiles g, g + 2, ...),
        // so one group's waits on tensor memory, the L-mode rows and the
        // stores overlap the other's.  Warp w reads TMEM lanes 32 (w % 4).
        const int eg = (warp - 4) >> 2;  // 0 (warps 4-7) or 1 (warps 8-11)
        const int r = (tid - 128) & 127;
        const int bar_leave = 1 + 2 * eg, bar_stage = 2 + 2 * eg;  // named barriers of this group
        const uint32_t lane_off = (uint32_t)((warp & 3) * 32) << 16;
        // Delta rows of a full tile are contiguous in global memory
        // (128 * out_ld floats): they are written to a shared-memory tile and
        // leave in one bulk copy, instead of 4-byte stores that each cost an L2
        // sector write.  Each group alternates two staging tiles; before one is
        // rewritten, the copy that read it (the group's copy before last) has
        // finished reading.
        float* const sOut = reinterpret_cast<float*>(smem + C::B_TOTAL + NS * C::A_STAGE + NC * C::CSTAGE) +
                            eg * 2 * (C::OUT_BYTES / 4);
        for (int64_t k = eg; k < my_tiles; k += 2) {
            const int c = (int)(k % NC);
            const int a = (int)(k % NACC);     // accumulator
            const int ob = (int)((k >> 1) & 1);  // staged output tile of this group
            bool ok = mbar_wait_bounded(&cfull[c], (unsigned)((k / NC) & 1), p.flags, 1ll << 24);
            const bool valid = ok && r < tile_valid(k);
            int32_t cl = 0;
            float x = 0.f;
            if (valid) {
                cl = sCol(c, NK)[r];
                if (p.vals) x = reinterpret_cast<const float*>(sCol(c, NK + 1))[r];
            }
            if (ok) mbar_arrive(&cempty[c]);
            float al[J];
            if (valid)
                load_row<J, VEC>(p.f_l + (int64_t)cl * p.ld_l, al);
            else
#pragma unroll
                for (int j = 0; j < J; ++j) al[j] = 0.f;
            ok = ok && mbar_wait_bounded(&tfull[a], (unsigned)((k / NACC) & 1), p.flags, 1ll << 24);
            if (named_bar_or(bar_leave, 128, !ok)) {  // leave together
                abort_s = 1;
                break;
            }
            tc_fence_after();
            float dl[J];
#pragma unroll
            for (int jn = 0; jn < J; ++jn) dl[jn] = 0.f;
            const uint32_t taddr = tmem_base_s + lane_off + (uint32_t)(a * C::NCOL);
#pragma unroll
            for (int c0 = 0; c0 < C::NP; c0 += 16) {
                float d[16];
                tmem_ld16(taddr + c0, d);
                tmem_ld_wait();
#pragma unroll
                for (int t = 0; t < 16; ++t) {
                    const int cc = c0 + t;  // column (j_n, j_L) = (cc / J, cc % J)
                    if (cc < J * J) dl[cc / J] = fmaf(d[t], al[cc % J], dl[cc / J]);
                }
            }
            tc_fence_before();
            mbar_arrive(&tempty[a]);
            const bool full_tile = tile_valid(k) == TC_M;
            if (p.bulk_out && full_tile) {
                float* so = sOut + ob * (C::OUT_BYTES / 4);
                named_bar_or(bar_stage, 128, false);  // the copy that last read this tile has finished (see below)
                float* o = so + r * p.out_ld;
#pragma unroll
                for (int jn = 0; jn < J; ++jn) o[jn] = dl[jn];
                if (p.vals) o[J] = x;
                fence_proxy_async_smem();
                named_bar_or(bar_stage, 128, false);  // the whole tile is in shared memory
                if (r == 0) {
                    bulk_s2g(p.out + tile_start(k) * p.out_ld, so, (unsigned)(TC_M * p.out_ld * 4));
                    bulk_commit();
                    bulk_wait_read<1>();  // the copy issued before this one has read its tile
                }
            } else if (valid) {
                float* o = p.out + (tile_start(k) + r) * p.out_ld;
#pragma unroll
                for (int jn = 0; jn < J; ++jn) o[jn] = dl[jn];
                if (p.vals) o[J] = x;
            }
        }
        if (r == 0) bulk_wait_all();  // every Delta tile has reached global memory
    } else if (tid == 12 * 32) {
        // ---------------- MMA issue ----------------
        const uint32_t idesc = instr_desc(TF32 ? 2 : 1, TC_M, C::NP);
        for (int64_t k = 0; k < my_tiles; ++k) {
            const int s = (int)(k % NS);
            const int a = (int)(k % NACC);
            if (!mbar_wait_bounded(&full[s], (unsigned)((k / NS) & 1), p.flags, 1ll << 24) ||
                !mbar_wait_bounded(&tempty[a], (unsigned)(((k / NACC) & 1) ^ 1), p.flags, 1ll << 24)) {
                abort_s = 1;
                break;
            }
            tc_fence_after();
            const uint32_t tmem = tmem_base_s + (uint32_t)(a * C::NCOL);
#pragma unroll
            for (int ks = 0; ks < C::KSTEPS; ++ks) {
                const uint64_t ad = smem_desc(sA(s) + ks * 256, 128, C::SBO);
                const uint64_t bd = smem_desc(sB + ks * 256, 128, C::SBO);
                mma<TF32>(tmem, ad, bd, idesc, ks > 0);
            }
            if constexpr (X3) {
                // + A_hi B_lo + A_lo B_hi (the A_lo B_lo term is below FP32 rounding)
#pragma unroll
                for (int ks = 0; ks < C::KSTEPS; ++ks) {
                    const uint64_t ad = smem_desc(sA(s) + ks * 256, 128, C::SBO);
                    const uint64_t bd = smem_desc(sB + C::B_BYTES + ks * 256, 128, C::SBO);
                    mma<TF32>(tmem, ad, bd, idesc, 1);
                }
#pragma unroll
                for (int ks = 0; ks < C::KSTEPS; ++ks) {
                    const uint64_t ad = smem_desc(sA(s) + C::A_BYTES + ks * 256, 128, C::SBO);
                    const uint64_t bd = smem_desc(sB + ks * 256, 128, C::SBO);
                    mma<TF32>(tmem, ad, bd, idesc, 1);
                }
            }
            mma_commit(&tfull[a]);
            mma_commit(&empty[s]);
        }
    } else if (tid == 13 * 32) {
        // ---------------- coordinate loader ----------------
        for (int64_t k = 0; k < my_tiles; ++k) {
            const int c = (int)(k % NC);
            if (!mbar_wait_bounded(&cempty[c], (unsigned)(((k / NC) & 1) ^ 1), p.flags, 1ll << 24)) {
                abort_s = 1;
                break;
            }
            const int64_t e0 = tile_start(k);
            const unsigned bytes = (unsigned)((tile_valid(k) * 4 + 15) / 16 * 16);
            const int ncol = NK + 1 + (p.vals ? 1 : 0);
            mbar_expect_tx(&cfull[c], bytes * ncol);
#pragma unroll
            for (int m = 0; m < NK; ++m) bulk_g2s(sCol(c, m), p.col_k[m] + e0, bytes, &cfull[c]);
            bulk_g2s(sCol(c, NK), p.col_l + e0, bytes, &cfull[c]);
            if (p.vals) bulk_g2s(sCol(c, NK + 1), p.vals + e0, bytes, &cfull[c]);
        }
    }
    __syncthreads();
    if (warp == 13) {
        if (abort_s) {
            // let issued MMAs and copies land before the columns are freed (bounded)
            for (int a = 0; a < NACC; ++a) mbar_wait_bounded(&tfull[a], 0, nullptr, 1 << 20);
        }
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base_s), "r"(NACC * C::NCOL)
                     : "memory");
    }
}

// The same contraction with the roles split the other way: warps 0-3 and 4-7
// are two producer warpgroups taking alternate tiles, warps 8-11 one epilogue
// warpgroup (named barriers 1 and 2), warps 12 and 13 as above.  TF32 and
// BF16x3 tiles cost the producers twice the shared-memory stores (and BF16x3
// the low parts' conversions), so for them the second producer group is worth
// more than a second epilogue group; BF16 takes the split above.
template <int J, int NK, bool TF32, bool VEC, bool X3>
__global__ void __launch_bounds__(TC_ROLE_THREADS, 1) delta_tc_kernel_2p(const TcParams p) {
    using C = TcCfg<J, NK, TF32, X3>;
    using E = typename C::E;
    constexpr int NS = C::NS, NC = TC_NC;
    extern __shared__ __align__(128) uint8_t smem[];
    uint8_t* sB = smem;
    auto sA = [&](int s) { return smem + C::B_TOTAL + s * C::A_STAGE; };  // high part; low part + A_BYTES
    auto sCol = [&](int c, int m) {  // m < NK: K-group columns, NK: L column, NK+1: values
        return reinterpret_cast<int32_t*>(smem + C::B_TOTAL + NS * C::A_STAGE + c * C::CSTAGE + m * TC_M * 4);
    };
    constexpr int NACC = C::NACC;
    __shared__ uint64_t cfull[NC], cempty[NC], full[NS], empty[NS], tfull[NACC], tempty[NACC];
    __shared__ uint32_t tmem_base_s;
    __shared__ int abort_s;

    const int tid = threadIdx.x;
    const int warp = tid >> 5;

    for (int i = tid * 16; i < p.b_bytes; i += TC_ROLE_THREADS * 16)
        *reinterpret_cast<uint4*>(sB + i) = *reinterpret_cast<const uint4*>(p.b_image + i);
    if (tid == 0) {
        for (int c = 0; c < NC; ++c) {
            mbar_init(&cfull[c], 1);
            mbar_init(&cempty[c], 2 * TC_M);
        }
        for (int s = 0; s < NS; ++s) {
            mbar_init(&full[s], TC_M);
            mbar_init(&empty[s], 1);
        }
        for (int a = 0; a < NACC; ++a) {
            mbar_init(&tfull[a], 1);
            mbar_init(&tempty[a], TC_M);
        }
        fence_mbar_init();
        abort_s = 0;
    }
    if (warp == 13) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base_s)),
                     "r"(NACC * C::NCOL)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    fence_proxy_async_smem();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();

    const int64_t ntiles = ceil_div_dev(p.n, TC_M);
    const int64_t t0 = blockIdx.x, ts = gridDim.x;
    const int64_t my_tiles = t0 < ntiles ? (ntiles - 1 - t0) / ts + 1 : 0;
    auto tile_start = [&](int64_t k) { return (t0 + k * ts) * TC_M; };
    auto tile_valid = [&](int64_t k) {
        const int64_t nv = p.n - tile_start(k);
        return (int)(nv < TC_M ? nv : TC_M);
    };

    if (warp < 8) {
        // ---------------- producers ----------------
        const int grp = warp >> 2;   // producer group: tiles k = grp, grp + 2, ...
        const int r = tid & 127;     // row of the tile
        float rk[NK * J], rkn[NK * J];
        auto gather = [&](int64_t k, float* dst) -> bool {
            const int c = (int)(k % NC);
            if (!mbar_wait_bounded(&cfull[c], (unsigned)((k / NC) & 1), p.flags, 1ll << 24)) return false;
            const bool valid = r < tile_valid(k);
            int32_t co[NK];
#pragma unroll
            for (int m = 0; m < NK; ++m) co[m] = valid ? sCol(c, m)[r] : 0;
            mbar_arrive(&cempty[c]);
#pragma unroll
            for (int m = 0; m < NK; ++m) {
                if (valid)
                    load_row<J, VEC>(p.f_k[m] + (int64_t)co[m] * p.ld_k[m], dst + m * J);
                else
#pragma unroll
                    for (int j = 0; j < J; ++j) dst[m * J + j] = 0.f;
            }
            return true;
        };
        bool ok = true;
        if (grp < my_tiles) ok = gather(grp, rk);
        for (int64_t k = grp; ok && k < my_tiles; k += 2) {
            if (k + 2 < my_tiles && !gather(k + 2, rkn)) {
                ok = false;
                break;
            }
            const int s = (int)(k % NS);
            if (!mbar_wait_bounded(&empty[s], (unsigned)(((k / NS) & 1) ^ 1), p.flags, 1ll << 24)) {
                ok = false;
                break;
            }
            uint8_t* arow = sA(s) + (r >> 3) * C::SBO + (r & 7) * 16;
#pragma unroll
            for (int kc = 0; kc < C::KCH; ++kc) {
                float v[E::KPG];
#pragma unroll
                for (int t = 0; t < E::KPG; ++t) {
                    const int kk = kc * E::KPG + t;
                    float a = 0.f;
                    if (kk < C::K) {
                        if constexpr (NK == 1) {
                            a = rk[kk];
                        } else if constexpr (NK == 2) {
                            a = rk[kk / J] * rk[J + kk % J];
                        } else {
                            a = rk[kk / (J * J)] * rk[J + (kk / J) % J] * rk[2 * J + kk % J];
                        }
                    }
                    v[t] = a;
                }
                uint4 w;
                if constexpr (TF32) {
                    w = make_uint4(to_tf32(v[0]), to_tf32(v[1]), to_tf32(v[2]), to_tf32(v[3]));
                } else {
                    w = make_uint4(pack_bf16(v[0], v[1]), pack_bf16(v[2], v[3]), pack_bf16(v[4], v[5]),
                                   pack_bf16(v[6], v[7]));
                }
                *reinterpret_cast<uint4*>(arow + kc * 128) = w;
                if constexpr (X3) {
                    // low part: the rounding remainder of the high part, again in BF16
                    float lo[E::KPG];
#pragma unroll
                    for (int t = 0; t < E::KPG; ++t) lo[t] = v[t] - bf16_value(v[t]);
                    *reinterpret_cast<uint4*>(arow + C::A_BYTES + kc * 128) =
                        make_uint4(pack_bf16(lo[0], lo[1]), pack_bf16(lo[2], lo[3]), pack_bf16(lo[4], lo[5]),
                                   pack_bf16(lo[6], lo[7]));
                }
            }
            fence_proxy_async_smem();
            mbar_arrive(&full[s]);
#pragma unroll
            for (int q = 0; q < NK * J; ++q) rk[q] = rkn[q];
        }
        if (!ok) abort_s = 1;
    } else if (warp < 12) {
        // ---------------- epilogue ----------------
        const int r = tid - 256;
        const uint32_t lane_off = (uint32_t)((warp & 3) * 32) << 16;
        // Delta rows of a full tile are contiguous in global memory
        // (128 * out_ld floats): they are written to a shared-memory tile and
        // leave in one bulk copy, instead of 4-byte stores that each cost an L2
        // sector write.  Two tiles alternate; before a tile is rewritten, the
        // copy that read it two tiles ago has finished reading.
        float* const sOut = reinterpret_cast<float*>(smem + C::B_TOTAL + NS * C::A_STAGE + NC * C::CSTAGE);
        for (int64_t k = 0; k < my_tiles; ++k) {
            const int c = (int)(k % NC);
            const int a = (int)(k % NACC);  // accumulator
            const int ob = (int)(k & 1);     // staged output tile
            bool ok = mbar_wait_bounded(&cfull[c], (unsigned)((k / NC) & 1), p.flags, 1ll << 24);
            const bool valid = ok && r < tile_valid(k);
            int32_t cl = 0;
            float x = 0.f;
            if (valid) {
                cl = sCol(c, NK)[r];
                if (p.vals) x = reinterpret_cast<const float*>(sCol(c, NK + 1))[r];
            }
            if (ok) mbar_arrive(&cempty[c]);
            float al[J];
            if (valid)
                load_row<J, VEC>(p.f_l + (int64_t)cl * p.ld_l, al);
            else
#pragma unroll
                for (int j = 0; j < J; ++j) al[j] = 0.f;
            ok = ok && mbar_wait_bounded(&tfull[a], (unsigned)((k / NACC) & 1), p.flags, 1ll << 24);
            if (named_bar_or(1, 128, !ok)) {  // leave together
                abort_s = 1;
                break;
            }
            tc_fence_after();
            float dl[J];
#pragma unroll
            for (int jn = 0; jn < J; ++jn) dl[jn] = 0.f;
            const uint32_t taddr = tmem_base_s + lane_off + (uint32_t)(a * C::NCOL);
#pragma unroll
            for (int c0 = 0; c0 < C::NP; c0 += 16) {
                float d[16];
                tmem_ld16(taddr + c0, d);
                tmem_ld_wait();
#pragma unroll
                for (int t = 0; t < 16; ++t) {
                    const int cc = c0 + t;  // column (j_n, j_L) = (cc / J, cc % J)
                    if (cc < J * J) dl[cc / J] = fmaf(d[t], al[cc % J], dl[cc / J]);
                }
            }
            tc_fence_before();
            mbar_arrive(&tempty[a]);
            const bool full_tile = tile_valid(k) == TC_M;
            if (p.bulk_out && full_tile) {
                float* so = sOut + ob * (C::OUT_BYTES / 4);
                named_bar_or(2, 128, false);  // the copy that last read this tile has finished (see below)
                float* o = so + r * p.out_ld;
#pragma unroll
                for (int jn = 0; jn < J; ++jn) o[jn] = dl[jn];
                if (p.vals) o[J] = x;
                fence_proxy_async_smem();
                named_bar_or(2, 128, false);  // the whole tile is in shared memory
                if (r == 0) {
                    bulk_s2g(p.out + tile_start(k) * p.out_ld, so, (unsigned)(TC_M * p.out_ld * 4));
                    bulk_commit();
                    bulk_wait_read<1>();  // the copy issued before this one has read its tile
                }
            } else if (valid) {
                float* o = p.out + (tile_start(k) + r) * p.out_ld;
#pragma unroll
                for (int jn = 0; jn < J; ++jn) o[jn] = dl[jn];
                if (p.vals) o[J] = x;
            }
        }
        if (r == 0) bulk_wait_all();  // every Delta tile has reached global memory
    } else if (tid == 12 * 32) {
        // ---------------- MMA issue ----------------
        const uint32_t idesc = instr_desc(TF32 ? 2 : 1, TC_M, C::NP);
        for (int64_t k = 0; k < my_tiles; ++k) {
            const int s = (int)(k % NS);
            const int a = (int)(k % NACC);
            if (!mbar_wait_bounded(&full[s], (unsigned)((k / NS) & 1), p.flags, 1ll << 24) ||
                !mbar_wait_bounded(&tempty[a], (unsigned)(((k / NACC) & 1) ^ 1), p.flags, 1ll << 24)) {
                abort_s = 1;
                break;
            }
            tc_fence_after();
            const uint32_t tmem = tmem_base_s + (uint32_t)(a * C::NCOL);
#pragma unroll
            for (int ks = 0; ks < C::KSTEPS; ++ks) {
                const uint64_t ad = smem_desc(sA(s) + ks * 256, 128, C::SBO);
                const uint64_t bd = smem_desc(sB + ks * 256, 128, C::SBO);
                mma<TF32>(tmem, ad, bd, idesc, ks > 0);
            }
            if constexpr (X3) {
                // + A_hi B_lo + A_lo B_hi (the A_lo B_lo term is below FP32 rounding)
#pragma unroll
                for (int ks = 0; ks < C::KSTEPS; ++ks) {
                    const uint64_t ad = smem_desc(sA(s) + ks * 256, 128, C::SBO);
                    const uint64_t bd = smem_desc(sB + C::B_BYTES + ks * 256, 128, C::SBO);
                    mma<TF32>(tmem, ad, bd, idesc, 1);
                }
#pragma unroll
                for (int ks = 0; ks < C::KSTEPS; ++ks) {
                    const uint64_t ad = smem_desc(sA(s) + C::A_BYTES + ks * 256, 128, C::SBO);
                    const uint64_t bd = smem_desc(sB + ks * 256, 128, C::SBO);
                    mma<TF32>(tmem, ad, bd, idesc, 1);
                }
            }
            mma_commit(&tfull[a]);
            mma_commit(&empty[s]);
        }
    } else if (tid == 13 * 32) {
        // ---------------- coordinate loader ----------------
        for (int64_t k = 0; k < my_tiles; ++k) {
            const int c = (int)(k % NC);
            if (!mbar_wait_bounded(&cempty[c], (unsigned)(((k / NC) & 1) ^ 1), p.flags, 1ll << 24)) {
                abort_s = 1;
                break;
            }
            const int64_t e0 = tile_start(k);
            const unsigned bytes = (unsigned)((tile_valid(k) * 4 + 15) / 16 * 16);
            const int ncol = NK + 1 + (p.vals ? 1 : 0);
            mbar_expect_tx(&cfull[c], bytes * ncol);
#pragma unroll
            for (int m = 0; m < NK; ++m) bulk_g2s(sCol(c, m), p.col_k[m] + e0, bytes, &cfull[c]);
            bulk_g2s(sCol(c, NK), p.col_l + e0, bytes, &cfull[c]);
            if (p.vals) bulk_g2s(sCol(c, NK + 1), p.vals + e0, bytes, &cfull[c]);
        }
    }
    __syncthreads();
    if (warp == 13) {
        if (abort_s) {
            // let issued MMAs and copies land before the columns are freed (bounded)
            for (int a = 0; a < NACC; ++a) mbar_wait_bounded(&tfull[a], 0, nullptr, 1 << 20);
        }
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base_s), "r"(NACC * C::NCOL)
                     : "memory");
    }
}

// ---- A in tensor memory ---------------------------------------------------
// The tensor cores may read A from tensor memory instead of shared memory.
// Here each producer thread writes its Kronecker row straight from registers
// into its own TMEM lane (tcgen05.st), so neither the producers' row writes
// nor the MMAs' re-reads of A (once per K step and, with BF16x3, twice for
// the high part) go through shared memory, which then carries only Gb: per
// 128-entry tile at J = 10, NK = 2 and BF16x3 that is about 74 KB of operand
// reads instead of about 215 KB of reads and writes.  Tensor memory (512
// columns) holds two accumulators (columns 0-255) and two A stages
// (256-511, one per producer group): the shapes whose A stage fits 128
// columns (KP elements of 16 bits two to a column, or of 32 bits one).
template <int J, int NK, bool TF32, bool X3>
struct TmCfg {
    using C = TcCfg<J, NK, TF32, X3>;
    static constexpr int APART = C::KP * C::E::ESZ / 4;  // TMEM columns of one A part
    static constexpr int ACOLS = C::NPART * APART;
    static constexpr int ACC0 = 0, A0 = 256;             // first accumulator / A stage column
    static constexpr int SMEM = C::B_TOTAL + TC_NC * C::CSTAGE + 2 * C::OUT_BYTES + 128;
};
constexpr bool tm_fits(int J, int NK, bool tf32, bool x3) {
    const int mk = tf32 ? 8 : 16;
    const int K = NK == 1 ? J : (NK == 2 ? J * J : J * J * J);
    const int KP = (K + mk - 1) / mk * mk;
    return (x3 ? 2 : 1) * KP * (tf32 ? 4 : 2) / 4 <= 128;
}

// Roles: warps 0-3 and 4-7 are two producer groups (tiles k = group,
// group + 2, ...; group g fills A stage g), warps 8-11 the epilogue, warp 12
// issues the MMAs, warp 13 owns TMEM and streams the coordinate columns.
// Barriers (all waits bounded):
//   cfull[c] / cempty[c]  loader <-> producers + epilogue (256 arrivals)
//   full[s]  / empty[s]   producer group s <-> MMA (128 arrivals / tcgen05.commit)
//   tfull[a] / tempty[a]  MMA <-> epilogue (tcgen05.commit / 128 arrivals)
template <int J, int NK, bool TF32, bool VEC, bool X3>
__global__ void __launch_bounds__(TC_ROLE_THREADS, 1) delta_tc_kernel_tm(const TcParams p) {
    using C = TcCfg<J, NK, TF32, X3>;
    using T = TmCfg<J, NK, TF32, X3>;
    using E = typename C::E;
    constexpr int NC = TC_NC;
    extern __shared__ __align__(128) uint8_t smem[];
    uint8_t* sB = smem;
    auto sCol = [&](int c, int m) {  // m < NK: K-group columns, NK: L column, NK+1: values
        return reinterpret_cast<int32_t*>(smem + C::B_TOTAL + c * C::CSTAGE + m * TC_M * 4);
    };
    __shared__ uint64_t cfull[NC], cempty[NC], full[2], empty[2], tfull[2], tempty[2];
    __shared__ uint32_t tmem_base_s;
    __shared__ int abort_s;

    const int tid = threadIdx.x;
    const int warp = tid >> 5;

    for (int i = tid * 16; i < p.b_bytes; i += TC_ROLE_THREADS * 16)
        *reinterpret_cast<uint4*>(sB + i) = *reinterpret_cast<const uint4*>(p.b_image + i);
    if (tid == 0) {
        for (int c = 0; c < NC; ++c) {
            mbar_init(&cfull[c], 1);
            mbar_init(&cempty[c], 2 * TC_M);
        }
        for (int s = 0; s < 2; ++s) {
            mbar_init(&full[s], TC_M);
            mbar_init(&empty[s], 1);
            mbar_init(&tfull[s], 1);
            mbar_init(&tempty[s], TC_M);
        }
        fence_mbar_init();
        abort_s = 0;
    }
    if (warp == 13) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base_s)),
                     "r"(512)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    fence_proxy_async_smem();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();

    const int64_t ntiles = ceil_div_dev(p.n, TC_M);
    const int64_t t0 = blockIdx.x, ts = gridDim.x;
    const int64_t my_tiles = t0 < ntiles ? (ntiles - 1 - t0) / ts + 1 : 0;
    auto tile_start = [&](int64_t k) { return (t0 + k * ts) * TC_M; };
    auto tile_valid = [&](int64_t k) {
        const int64_t nv = p.n - tile_start(k);
        return (int)(nv < TC_M ? nv : TC_M);
    };
    const uint32_t lane_off = (uint32_t)((warp & 3) * 32) << 16;

    if (warp < 8) {
        // ---------------- producers ----------------
        const int grp = warp >> 2;   // producer group: tiles k = grp, grp + 2, ...; A stage grp
        const int r = tid & 127;     // row of the tile = TMEM lane
        float rk[NK * J], rkn[NK * J];
        auto gather = [&](int64_t k, float* dst) -> bool {
            const int c = (int)(k % NC);
            if (!mbar_wait_bounded(&cfull[c], (unsigned)((k / NC) & 1), p.flags, 1ll << 24)) return false;
            const bool valid = r < tile_valid(k);
            int32_t co[NK];
#pragma unroll
            for (int m = 0; m < NK; ++m) co[m] = valid ? sCol(c, m)[r] : 0;
            mbar_arrive(&cempty[c]);
#pragma unroll
            for (int m = 0; m < NK; ++m) {
                if (valid)
                    load_row<J, VEC>(p.f_k[m] + (int64_t)co[m] * p.ld_k[m], dst + m * J);
                else
#pragma unroll
                    for (int j = 0; j < J; ++j) dst[m * J + j] = 0.f;
            }
            return true;
        };
        // the four 32-bit words of 16-byte chunk kc (and of its low part)
        auto chunk = [&](int kc, uint32_t* w, uint32_t* wl) {
            float v[E::KPG];
#pragma unroll
            for (int t = 0; t < E::KPG; ++t) {
                const int kk = kc * E::KPG + t;
                float a = 0.f;
                if (kk < C::K) {
                    if constexpr (NK == 1) {
                        a = rk[kk];
                    } else if constexpr (NK == 2) {
                        a = rk[kk / J] * rk[J + kk % J];
                    } else {
                        a = rk[kk / (J * J)] * rk[J + (kk / J) % J] * rk[2 * J + kk % J];
                    }
                }
                v[t] = a;
            }
            if constexpr (TF32) {
#pragma unroll
                for (int t = 0; t < 4; ++t) w[t] = to_tf32(v[t]);
            } else {
#pragma unroll
                for (int t = 0; t < 4; ++t) w[t] = pack_bf16(v[2 * t], v[2 * t + 1]);
                if constexpr (X3) {
                    // low part: the rounding remainder of the high part, again in BF16
#pragma unroll
                    for (int t = 0; t < 4; ++t)
                        wl[t] = pack_bf16(v[2 * t] - bf16_value(v[2 * t]), v[2 * t + 1] - bf16_value(v[2 * t + 1]));
                }
            }
        };
        // the whole row into A stage grp: pairs of chunks (eight columns) per store
        const uint32_t arow = tmem_base_s + lane_off + (uint32_t)(T::A0 + grp * 128);
        bool ok = true;
        if (grp < my_tiles) ok = gather(grp, rk);
        for (int64_t k = grp; ok && k < my_tiles; k += 2) {
            if (k + 2 < my_tiles && !gather(k + 2, rkn)) {
                ok = false;
                break;
            }
            if (!mbar_wait_bounded(&empty[grp], (unsigned)(((k >> 1) & 1) ^ 1), p.flags, 1ll << 24)) {
                ok = false;
                break;
            }
            tc_fence_after();
#pragma unroll
            for (int kc = 0; kc < C::KCH; kc += 2) {
                uint32_t w[8], wl[8];
                chunk(kc, w, wl);
                chunk(kc + 1, w + 4, wl + 4);
                tmem_st8(arow + (uint32_t)(kc * 4), w);
                if constexpr (X3) tmem_st8(arow + (uint32_t)(T::APART + kc * 4), wl);
            }
            tmem_st_wait();
            tc_fence_before();
            mbar_arrive(&full[grp]);
#pragma unroll
            for (int q = 0; q < NK * J; ++q) rk[q] = rkn[q];
        }
        if (!ok) abort_s = 1;
    } else if (warp < 12) {
        // ---------------- epilogue ----------------
        // Each warp drains its 32 rows on its own (no barrier across the
        // group): the Delta rows of a full tile's warp (32 * out_ld floats,
        // contiguous in global memory) are staged in shared memory and leave
        // in one bulk copy; two staged buffers per warp alternate, and before
        // one is rewritten the copy that read it two tiles ago has finished
        // reading (lane 0 waits for it right after issuing the next copy).
        const int r = tid - 256;
        const int lane = tid & 31, wq = warp & 3;
        float* const sOut = reinterpret_cast<float*>(smem + C::B_TOTAL + NC * C::CSTAGE);
        for (int64_t k = 0; k < my_tiles; ++k) {
            const int c = (int)(k % NC);
            const int a = (int)(k & 1);   // accumulator
            const int ob = (int)(k & 1);  // staged buffer
            bool ok = mbar_wait_bounded(&cfull[c], (unsigned)((k / NC) & 1), p.flags, 1ll << 24);
            const bool valid = ok && r < tile_valid(k);
            int32_t cl = 0;
            float x = 0.f;
            if (valid) {
                cl = sCol(c, NK)[r];
                if (p.vals) x = reinterpret_cast<const float*>(sCol(c, NK + 1))[r];
            }
            if (ok) mbar_arrive(&cempty[c]);
            float al[J];
            if (valid)
                load_row<J, VEC>(p.f_l + (int64_t)cl * p.ld_l, al);
            else
#pragma unroll
                for (int j = 0; j < J; ++j) al[j] = 0.f;
            ok = ok && mbar_wait_bounded(&tfull[a], (unsigned)((k >> 1) & 1), p.flags, 1ll << 24);
            if (__any_sync(0xffffffffu, !ok)) {  // the warp leaves together
                abort_s = 1;
                break;
            }
            tc_fence_after();
            float dl[J];
#pragma unroll
            for (int jn = 0; jn < J; ++jn) dl[jn] = 0.f;
            const uint32_t taddr = tmem_base_s + lane_off + (uint32_t)(T::ACC0 + a * 128);
#pragma unroll
            for (int c0 = 0; c0 < C::NP; c0 += 16) {
                float d[16];
                tmem_ld16(taddr + c0, d);
                tmem_ld_wait();
#pragma unroll
                for (int t = 0; t < 16; ++t) {
                    const int cc = c0 + t;  // column (j_n, j_L) = (cc / J, cc % J)
                    if (cc < J * J) dl[cc / J] = fmaf(d[t], al[cc % J], dl[cc / J]);
                }
            }
            tc_fence_before();
            mbar_arrive(&tempty[a]);
            const bool full_tile = tile_valid(k) == TC_M;
            if (p.bulk_out && full_tile) {
                float* so = sOut + ob * (C::OUT_BYTES / 4) + wq * 32 * p.out_ld;
                __syncwarp();  // lane 0 has seen the copy that last read this buffer finish
                float* o = so + lane * p.out_ld;
#pragma unroll
                for (int jn = 0; jn < J; ++jn) o[jn] = dl[jn];
                if (p.vals) o[J] = x;
                fence_proxy_async_smem();
                __syncwarp();  // the warp's rows are in shared memory
                if (lane == 0) {
                    bulk_s2g(p.out + (tile_start(k) + wq * 32) * p.out_ld, so, (unsigned)(32 * p.out_ld * 4));
                    bulk_commit();
                    bulk_wait_read<1>();  // the copy issued before this one has read its buffer
                }
            } else if (valid) {
                float* o = p.out + (tile_start(k) + r) * p.out_ld;
#pragma unroll
                for (int jn = 0; jn < J; ++jn) o[jn] = dl[jn];
                if (p.vals) o[J] = x;
            }
        }
        if (lane == 0) bulk_wait_all();  // every Delta row has reached global memory
    } else if (tid == 12 * 32) {
        // ---------------- MMA issue ----------------
        const uint32_t idesc = instr_desc(TF32 ? 2 : 1, TC_M, C::NP);
        for (int64_t k = 0; k < my_tiles; ++k) {
            const int s = (int)(k & 1);  // A stage of tile k
            const int a = (int)(k & 1);
            const unsigned ph = (unsigned)((k >> 1) & 1);
            if (!mbar_wait_bounded(&full[s], ph, p.flags, 1ll << 24) ||
                !mbar_wait_bounded(&tempty[a], ph ^ 1, p.flags, 1ll << 24)) {
                abort_s = 1;
                break;
            }
            tc_fence_after();
            const uint32_t tmem = tmem_base_s + (uint32_t)(T::ACC0 + a * 128);
            const uint32_t ta = tmem_base_s + (uint32_t)(T::A0 + s * 128);
#pragma unroll
            for (int ks = 0; ks < C::KSTEPS; ++ks)
                mma_ts<TF32>(tmem, ta + ks * 8, smem_desc(sB + ks * 256, 128, C::SBO), idesc, ks > 0);
            if constexpr (X3) {
                // + A_hi B_lo + A_lo B_hi (the A_lo B_lo term is below FP32 rounding)
#pragma unroll
                for (int ks = 0; ks < C::KSTEPS; ++ks)
                    mma_ts<TF32>(tmem, ta + ks * 8, smem_desc(sB + C::B_BYTES + ks * 256, 128, C::SBO), idesc, 1);
#pragma unroll
                for (int ks = 0; ks < C::KSTEPS; ++ks)
                    mma_ts<TF32>(tmem, ta + T::APART + ks * 8, smem_desc(sB + ks * 256, 128, C::SBO), idesc, 1);
            }
            mma_commit(&tfull[a]);
            mma_commit(&empty[s]);
        }
    } else if (tid == 13 * 32) {
        // ---------------- coordinate loader ----------------
        for (int64_t k = 0; k < my_tiles; ++k) {
            const int c = (int)(k % NC);
            if (!mbar_wait_bounded(&cempty[c], (unsigned)(((k / NC) & 1) ^ 1), p.flags, 1ll << 24)) {
                abort_s = 1;
                break;
            }
            const int64_t e0 = tile_start(k);
            const unsigned bytes = (unsigned)((tile_valid(k) * 4 + 15) / 16 * 16);
            const int ncol = NK + 1 + (p.vals ? 1 : 0);
            mbar_expect_tx(&cfull[c], bytes * ncol);
#pragma unroll
            for (int m = 0; m < NK; ++m) bulk_g2s(sCol(c, m), p.col_k[m] + e0, bytes, &cfull[c]);
            bulk_g2s(sCol(c, NK), p.col_l + e0, bytes, &cfull[c]);
            if (p.vals) bulk_g2s(sCol(c, NK + 1), p.vals + e0, bytes, &cfull[c]);
        }
    }
    __syncthreads();
    if (warp == 13) {
        if (abort_s) {
            // let issued MMAs and copies land before the columns are freed (bounded)
            for (int a = 0; a < 2; ++a) mbar_wait_bounded(&tfull[a], 0, nullptr, 1 << 20);
        }
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base_s), "r"(512) : "memory");
    }
}

// Coordinate columns as 16-byte aligned SoA arrays for the bulk copies:
// column m of entry e goes to out[m * stride + e], taken from base[e * cstride + sel[m]].
struct Sel4 {
    int m[4];
};
__global__ void to_soa(const int32_t* __restrict__ base, int64_t cstride, int ncol, Sel4 sel, int64_t n, int64_t stride,
                       int32_t* __restrict__ out) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
        for (int m = 0; m < ncol; ++m) out[m * stride + e] = base[e * cstride + sel.m[m]];
}

// Gb in the layout above: row r = j_n * J + j_L, column k over the K-group
// modes (C order), zero padded.
// With X3 the image holds the BF16 high parts, then (B_BYTES further) the
// BF16 low parts: G = hi + lo up to 2^-16 relative.
template <bool TF32, bool X3>
__global__ void build_b_image(const float* __restrict__ G, int order, int mode, int lmode, int J, int NK,
                              const int* __restrict__ kmodes_unused, int K, int NP, int KP, uint8_t* __restrict__ img) {
    using E = Elt<TF32>;
    const int KCH = KP / E::KPG;
    const int SBO = KCH * 128;
    const int total = NP * KP;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < total; t += gridDim.x * blockDim.x) {
        const int r = t / KP, k = t % KP;
        float v = 0.f;
        if (r < J * J && k < K) {
            const int jn = r / J, jl = r % J;
            int jj[PTK_MAX_ORDER];
            jj[mode] = jn;
            jj[lmode] = jl;
            // K-group modes in increasing order, the last one fastest in k
            int rem = k;
            for (int m = order - 1; m >= 0; --m) {
                if (m == mode || m == lmode) continue;
                jj[m] = rem % J;
                rem /= J;
            }
            int src = 0;
            for (int m = 0; m < order; ++m) src = src * J + jj[m];
            v = G[src];
        }
        const int off = (r >> 3) * SBO + (k / E::KPG) * 128 + (r & 7) * 16 + (k % E::KPG) * E::ESZ;
        if constexpr (TF32) {
            uint32_t u;
            asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(u) : "f"(v));
            *reinterpret_cast<uint32_t*>(img + off) = u;
        } else {
            const __nv_bfloat16 hi = __float2bfloat16_rn(v);
            *reinterpret_cast<__nv_bfloat16*>(img + off) = hi;
            if constexpr (X3)
                *reinterpret_cast<__nv_bfloat16*>(img + (size_t)NP * KP * E::ESZ + off) =
                    __float2bfloat16_rn(v - __bfloat162float(hi));
        }
    }
}

struct Shape {
    bool ok = false;
    int J = 0, NK = 0;
    int kmodes[3] = {};
    int lmode = -1;
};

Shape shape_of(const DeltaJob& job) {
    Shape s;
    const int N = job.order;
    if (job.dtype != PTK_F32 || N < 3 || N > 5) return s;
    const int J = job.J[0];
    for (int k = 0; k < N; ++k)
        if (job.J[k] != J) return s;
    if (J * J > 128 || J < 2) return s;
    s.J = J;
    s.NK = N - 2;
    int o = 0;
    for (int k = 0; k < N; ++k) {
        if (k == job.mode) continue;
        if (o < s.NK)
            s.kmodes[o] = k;
        else
            s.lmode = k;
        ++o;
    }
    // the K extent must fit the shared-memory budget (A double buffer + Gb)
    int K = 1;
    for (int m = 0; m < s.NK; ++m) K *= J;
    if (K > 256) return s;
    s.ok = true;
    return s;
}

template <int J, int NK, bool TF32, bool X3>
ptk_status launch_tc(ptk_ctx* ctx, const DeltaJob& job, const Shape& sh, cudaStream_t st) {
    using C = TcCfg<J, NK, TF32, X3>;
    uint8_t* img = (uint8_t*)scratch(ctx, SLOT_GPERM_TC, C::B_TOTAL);
    if (!img) return PTK_ERR_OUT_OF_MEMORY;
    {
        const int total = C::NP * C::KP;
        build_b_image<TF32, X3><<<(total + 255) / 256, 256, 0, st>>>((const float*)job.core, job.order, job.mode,
                                                                     sh.lmode, J, NK, nullptr, C::K, C::NP, C::KP,
                                                                     img);
        ::ptk::note_launch();
    }
    PTK_LAUNCH_CHECK();
    TcParams p{};
    p.n = job.n;
    for (int m = 0; m < NK; ++m) {
        p.col_k[m] = job.col[sh.kmodes[m]];
        p.f_k[m] = (const float*)job.factors[sh.kmodes[m]];
        p.ld_k[m] = job.ld[sh.kmodes[m]];
    }
    p.col_l = job.col[sh.lmode];
    p.f_l = (const float*)job.factors[sh.lmode];
    p.ld_l = job.ld[sh.lmode];
    p.vals = (const float*)job.vals;
    // the loader bulk-copies coordinate columns: they must be SoA and 16-byte aligned
    // (and, unless the arrays carry slack, a multiple of 4 entries: the last tile's
    // copy is rounded up to 16 bytes)
    bool soa = job.cstride == 1 && (uintptr_t)p.col_l % 16 == 0 && (uintptr_t)p.vals % 16 == 0 &&
               (job.padded || job.n % 4 == 0);
    for (int m = 0; m < NK; ++m) soa = soa && (uintptr_t)p.col_k[m] % 16 == 0;
    if (!soa) {
        const int64_t stride = (job.n + 3) / 4 * 4 + 4;  // 16-byte aligned columns with slack
        int32_t* buf = (int32_t*)scratch(ctx, SLOT_TC_COORDS, sizeof(int32_t) * (size_t)stride * (NK + 2));
        if (!buf) return PTK_ERR_OUT_OF_MEMORY;
        // job.col[k] = base + k for interleaved rows, or separate columns
        Sel4 sel{};
        const int32_t* base = job.col[0];
        bool interleaved = job.cstride > 1;
        for (int m = 0; m < NK; ++m) sel.m[m] = sh.kmodes[m];
        sel.m[NK] = sh.lmode;
        const int g = (int)std::min<int64_t>(ceil_div(job.n, 256), (int64_t)ctx->sm_count * 8);
        if (interleaved) {
            { to_soa<<<g, 256, 0, st>>>(base, job.cstride, NK + 1, sel, job.n, stride, buf); ::ptk::note_launch(); }
        } else {
            for (int m = 0; m <= NK; ++m)
                PTK_CUDA(cudaMemcpyAsync(buf + m * stride, job.col[sel.m[m]], sizeof(int32_t) * (size_t)job.n,
                                         cudaMemcpyDeviceToDevice, st));
        }
        PTK_LAUNCH_CHECK();
        for (int m = 0; m < NK; ++m) p.col_k[m] = buf + m * stride;
        p.col_l = buf + NK * stride;
        if (p.vals) {
            float* vb = reinterpret_cast<float*>(buf + (NK + 1) * stride);
            PTK_CUDA(cudaMemcpyAsync(vb, p.vals, sizeof(float) * (size_t)job.n, cudaMemcpyDeviceToDevice, st));
            p.vals = vb;
        }
    }
    p.out = (float*)job.out;
    p.out_ld = job.out_ld;
    // bulk stores need 16-byte aligned tile starts (128 * out_ld * 4 bytes apart)
    p.bulk_out = ((uintptr_t)p.out % 16 == 0 && p.out_ld <= J + 2) ? 1 : 0;
    p.b_image = img;
    p.b_bytes = C::B_TOTAL;
    p.flags = ctx->d_flags;
    bool vec = true;  // 16-byte row loads need 16-byte aligned rows
    for (int m = 0; m < NK; ++m) vec = vec && (p.ld_k[m] % 4 == 0) && ((uintptr_t)p.f_k[m] % 16 == 0);
    vec = vec && (p.ld_l % 4 == 0) && ((uintptr_t)p.f_l % 16 == 0);
    const int64_t tiles = ceil_div(job.n, TC_M);
    if constexpr ((TF32 || X3) && tm_fits(J, NK, TF32, X3)) {
        // TF32 and BF16x3: A in tensor memory, which the CTA takes whole (one per SM)
        using T = TmCfg<J, NK, TF32, X3>;
        auto kern = vec ? delta_tc_kernel_tm<J, NK, TF32, true, X3> : delta_tc_kernel_tm<J, NK, TF32, false, X3>;
        PTK_TRY(smem_attr((const void*)kern, T::SMEM, st, true));
        const int64_t grid = std::max<int64_t>(1, std::min<int64_t>(tiles, (int64_t)ctx->sm_count));
        { kern<<<(unsigned)grid, TC_ROLE_THREADS, T::SMEM, st>>>(p); ::ptk::note_launch(); }
        PTK_LAUNCH_CHECK();
        return PTK_OK;
    } else {
    // TF32 and BF16x3: two producer warpgroups; BF16: two epilogue warpgroups
    auto pick = [vec]() {
        if constexpr (TF32 || X3)
            return vec ? delta_tc_kernel_2p<J, NK, TF32, true, X3> : delta_tc_kernel_2p<J, NK, TF32, false, X3>;
        else
            return vec ? delta_tc_kernel<J, NK, TF32, true, X3> : delta_tc_kernel<J, NK, TF32, false, X3>;
    };
    auto kern = pick();
    PTK_TRY(smem_attr((const void*)kern, C::SMEM, st, true));
    int per_sm = 1;
    PTK_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, TC_ROLE_THREADS, C::SMEM));
    per_sm = std::max(1, std::min(per_sm, 512 / (C::NACC * C::NCOL)));  // TMEM: 512 columns per SM
    const int64_t grid = std::max<int64_t>(1, std::min<int64_t>(tiles, (int64_t)ctx->sm_count * per_sm));
    { kern<<<(unsigned)grid, TC_ROLE_THREADS, C::SMEM, st>>>(p); ::ptk::note_launch(); }
    PTK_LAUNCH_CHECK();
    return PTK_OK;
    }
}

template <bool TF32, bool X3>
ptk_status dispatch_tc(ptk_ctx* ctx, const DeltaJob& job, const Shape& sh, cudaStream_t st) {
#define PTK_TC(JJ, KK)                                           \
    if constexpr (tc_fits(JJ, KK, TF32, X3))                     \
        if (sh.J == JJ && sh.NK == KK) return launch_tc<JJ, KK, TF32, X3>(ctx, job, sh, st);
    PTK_TC(10, 2) PTK_TC(10, 1) PTK_TC(5, 1) PTK_TC(5, 2) PTK_TC(5, 3)
    PTK_TC(2, 1) PTK_TC(3, 1) PTK_TC(4, 1) PTK_TC(6, 1) PTK_TC(7, 1) PTK_TC(8, 1) PTK_TC(9, 1) PTK_TC(11, 1)
    PTK_TC(2, 2) PTK_TC(3, 2) PTK_TC(4, 2) PTK_TC(6, 2) PTK_TC(7, 2) PTK_TC(8, 2) PTK_TC(9, 2) PTK_TC(11, 2)
    PTK_TC(2, 3) PTK_TC(3, 3) PTK_TC(4, 3) PTK_TC(6, 3)
#undef PTK_TC
    set_error("tensor-core delta: no kernel for J=%d, order %d", sh.J, sh.NK + 2);
    return PTK_ERR_UNSUPPORTED;
}

}  // namespace

bool delta_tc_supported(const DeltaJob& job, ptk_precision prec) {
    if (prec != PTK_PREC_BF16 && prec != PTK_PREC_TF32 && prec != PTK_PREC_BF16X3) return false;
    Shape s = shape_of(job);
    if (!s.ok) return false;
    if (s.NK == 3 && s.J > 6) return false;  // order-5 kernels exist for J <= 6
    return tc_fits(s.J, s.NK, prec == PTK_PREC_TF32, prec == PTK_PREC_BF16X3);
}

ptk_status delta_tc(ptk_ctx* ctx, const DeltaJob& job, ptk_precision prec, cudaStream_t st) {
    Shape s = shape_of(job);
    if (!s.ok || !delta_tc_supported(job, prec)) {
        set_error("tensor-core delta is not available for this shape");
        return PTK_ERR_UNSUPPORTED;
    }
    if (job.n == 0) return PTK_OK;
    if (prec == PTK_PREC_TF32) return dispatch_tc<true, false>(ctx, job, s, st);
    if (prec == PTK_PREC_BF16X3) return dispatch_tc<false, true>(ctx, job, s, st);
    return dispatch_tc<false, false>(ctx, job, s, st);
}

}  // namespace ptk

extern "C" int ptk_delta_tc_supported(const ptk_model* m, int32_t mode, ptk_precision prec) {
    if (!m || mode < 0 || mode >= m->order) return 0;
    ptk::DeltaJob j;
    j.order = m->order;
    j.mode = mode;
    for (int k = 0; k < m->order; ++k) j.J[k] = m->J[k];
    j.dtype = m->dtype;
    return ptk::delta_tc_supported(j, prec) ? 1 : 0;
}
