// gemm_tc.cu -- trailing update of the mixed-precision LU on the 5th-generation
// tensor cores (tcgen05, sm_103a):
//     C[r0+i, c0+j] -= sum_k L[r0+i, k0+k] U[k0+k, c0+j],   i < M, j < N, k < Kd
// on the column-major FP32 S^K of every element (batched over elements).
//
// 1. pack: L (M x Kd) and U (Kd x N) are copied into K-major operand panels
//    in the operand type (TF32 rounded to nearest, or BF16), zero-padded in K
//    to whole 128-byte rows (or taken from panels that earlier kernels wrote:
//    the TRSM product's copy of U12, a merged pair's multipliers);
// 2. MMA: a persistent kernel, one CTA per SM, walks the 128 x BN tiles of C
//    (BN = 256 for split-BF16 updates at least 256 wide, else 128, or 32/64
//    for narrow updates) of all elements.  Warp 0 (one lane) streams 128-byte
//    K-chunks of both panels into a shared-memory ring with TMA (128B
//    swizzle, mbarrier transaction counts); warp 1 (one lane) issues
//    tcgen05.mma (kind::tf32 or kind::f16) into one of two TMEM accumulators
//    and releases each ring slot with tcgen05.commit;
// 3. epilogue: sixteen warps, four per TMEM lane quarter (32 rows), each on
//    32 columns (two such groups at BN = 256): C is read before the
//    accumulator is ready, then C - D is written in place (32 consecutive rows
//    per warp and column: coalesced 128-byte accesses).  The epilogue of one
//    tile runs while the MMAs of the next tile fill the other accumulator.
// The TRSM product (store mode) writes the product instead of C - D, and two
// more warps split its FP32 B operand into TF32 hi and lo in shared memory.
// Every mbarrier wait is bounded; on timeout the element's status becomes
// MEHDG_ETIMEOUT, the loops end and TMEM is still released.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>
#include <algorithm>
#include <cstdlib>
#include <cstring>
#include "lu_internal.cuh"
#include "prof.cuh"

namespace {

constexpr int TM = 128;           // rows of a C tile (TMEM lanes)
constexpr int CHUNK_BYTES = 128;  // K bytes per TMA box / swizzle row

__device__ __forceinline__ uint32_t s_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* b, uint32_t cnt) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(s_addr(b)), "r"(cnt) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* b, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(s_addr(b)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try(uint64_t* b, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok) : "r"(s_addr(b)), "r"(parity) : "memory");
    return ok != 0;
}
// bounded wait (about a second at most); false on timeout
__device__ __forceinline__ bool mbar_wait(uint64_t* b, uint32_t parity) {
    for (uint32_t i = 0; i < (1u << 23); ++i) {
        if (mbar_try(b, parity)) return true;
        if (i > 32) __nanosleep(64);
    }
    return false;
}
__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, uint64_t* bar, int x, int y, int z) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4, %5}], [%2];"
        ::"r"(s_addr(dst)), "l"(reinterpret_cast<uint64_t>(map)), "r"(s_addr(bar)), "r"(x), "r"(y), "r"(z)
        : "memory");
}
// shared-memory matrix descriptor: K-major, 128B swizzle, 8-row groups 1024 B apart
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
    d |= (uint64_t)1u << 16;                 // leading byte offset (unused for swizzled K-major)
    d |= (uint64_t)(1024u >> 4) << 32;       // stride byte offset
    d |= (uint64_t)1u << 46;                 // descriptor version
    d |= (uint64_t)2u << 61;                 // 128-byte swizzle
    return d;
}
// instruction descriptor: D = F32, A/B format, K-major A and B, N>>3, M>>4
__host__ __device__ constexpr uint32_t idesc(int M, int N, uint32_t fmt) {
    return (1u << 4) | (fmt << 7) | (fmt << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}
template <bool BF16>
__device__ __forceinline__ void umma(uint32_t d, uint64_t a, uint64_t b, uint32_t id, uint32_t acc) {
    if constexpr (BF16)
        asm volatile("{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                     " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n"
                     ::"r"(d), "l"(a), "l"(b), "r"(id), "r"(acc));
    else
        asm volatile("{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                     " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n"
                     ::"r"(d), "l"(a), "l"(b), "r"(id), "r"(acc));
}
__device__ __forceinline__ void umma_commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                 ::"r"(s_addr(bar)) : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// round to TF32 (nearest, ties away), kept in FP32 storage
__device__ __forceinline__ float tf32_rn(float x) {
    uint32_t y;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(y) : "f"(x));
    return __uint_as_float(y);
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t* r) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// ---------------------------------------------------------------- streaming kernel
// Persistent form of the update: one CTA per SM walks the tiles
// (element-major, then column tiles, then row tiles) with eighteen warps
// (twenty in store mode):
//   warp 0 (one lane)  TMA: operand chunks into the ring (up to 6 slots; 3 in
//                      the split modes, 2 at BN = 256);
//   warp 1 (one lane)  tcgen05.mma into one of two TMEM accumulators (2 x BN
//                      columns); the whole warp owns the TMEM allocation;
//   warps 2-17         epilogue: four warps per TMEM lane quarter, each on
//                      32 of the tile's columns (BN / 32 groups; a warp takes
//                      two at BN = 256).  A warp fetches its C values for the
//                      next tile before it waits for that tile's accumulator,
//                      so the C reads (32 per thread in flight) overlap the
//                      MMAs, and the stores of one tile overlap the MMAs of
//                      the next;
//   warps 18-19        store mode only: split each B chunk in shared memory.
// Every mbarrier wait is bounded; a warp that times out records
// MEHDG_ETIMEOUT and leaves its loop, the others time out in turn, and TMEM
// is released after the final barrier.
constexpr int EPI_WARPS = 16;
constexpr int RING_BYTES = 192 * 1024;   // operand ring budget

__device__ __forceinline__ void mbar_arrive(uint64_t* b) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(s_addr(b)) : "memory");
}

// a ring slot holds one K-chunk of A and of B, each as hi (and lo when split)
template <int BN, bool SPLIT>
constexpr int stage_bytes() { return (SPLIT ? 2 : 1) * (TM + BN) * CHUNK_BYTES; }
template <int BN, bool SPLIT>
constexpr int n_stages() { return RING_BYTES / stage_bytes<BN, SPLIT>() < 6 ? RING_BYTES / stage_bytes<BN, SPLIT>() : 6; }
template <int BN, bool SPLIT>
constexpr size_t stream_smem_bytes() { return (size_t)n_stages<BN, SPLIT>() * stage_bytes<BN, SPLIT>() + 1024; }

// SPLIT: the panels hold [hi | lo] (lo at K offset kpa in A, kpb in B); each
// chunk is loaded once per part and takes the three products hi hi, hi lo, lo hi.
// STORE (the TRSM product, split TF32): B arrives as plain FP32 rows and two
// more warps split each chunk in shared memory (hi in place, lo beside it)
// before the MMAs take it.
constexpr int CONV_WARPS = 2;
template <bool STORE> constexpr int stream_threads() { return 64 + 32 * EPI_WARPS + (STORE ? 32 * CONV_WARPS : 0); }
template <int BN, bool BF16, bool STORE, bool SPLIT>
__global__ void __launch_bounds__(stream_threads<STORE>(), 1)
tc_stream_kernel(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB,
                 float* __restrict__ Sall, int64_t ld, int r0, int c0, int M, int N, int nchunk, int kpa, int kpb,
                 int tiles_m, int tiles_n, int64_t ntiles, int32_t* status, BqOut bo) {
    constexpr int A_BYTES = TM * CHUNK_BYTES;
    constexpr int B_BYTES = BN * CHUNK_BYTES;
    constexpr int NP = SPLIT ? 2 : 1;
    constexpr int STG = stage_bytes<BN, SPLIT>();
    constexpr int SSTAGES = n_stages<BN, SPLIT>();
    constexpr int CHUNK_K = BF16 ? 64 : 32;
    constexpr uint32_t ID = idesc(TM, BN, BF16 ? 1u : 2u);
    constexpr int NH = BN / 32;                    // column groups per lane quarter
    constexpr int W = 32;                          // columns per epilogue warp
    constexpr bool CONVB = STORE;                  // B split in shared memory
    static_assert(!CONVB || (SPLIT && !BF16), "the TRSM product is split TF32");
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char* smem = reinterpret_cast<unsigned char*>(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    // slot s: [A hi | A lo | B hi | B lo] (lo parts only when split)
    __shared__ uint64_t full[SSTAGES], empty[SSTAGES], conv[SSTAGES], acc_full[2], acc_empty[2];
    __shared__ uint32_t tmem_slot;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int tiles_e = tiles_m * tiles_n;

    if (threadIdx.x == 0) {
        for (int s = 0; s < SSTAGES; ++s) { mbar_init(&full[s], 1); mbar_init(&empty[s], 1); mbar_init(&conv[s], CONV_WARPS); }
        for (int b = 0; b < 2; ++b) { mbar_init(&acc_full[b], 1); mbar_init(&acc_empty[b], EPI_WARPS); }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     ::"r"(s_addr(&tmem_slot)), "r"((uint32_t)(2 * BN)) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_slot;

    if (warp == 0) {
        if (lane == 0) {
            uint32_t g = 0;
            for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
                const int K = (int)(t / tiles_e), rem = (int)(t % tiles_e);
                const int tm = rem % tiles_m, tn = rem / tiles_m;
                bool ok = true;
                for (int c = 0; c < nchunk; ++c, ++g) {
                    const int s = (int)(g % SSTAGES);
                    if (g >= SSTAGES && !mbar_wait(&empty[s], ((g / SSTAGES) - 1) & 1)) { ok = false; break; }
                    unsigned char* slot = smem + (size_t)s * STG;
                    mbar_expect_tx(&full[s], CONVB ? STG - B_BYTES : STG);
                    tma_load_3d(slot, &mapA, &full[s], c * CHUNK_K, tm * TM, K);
                    tma_load_3d(slot + NP * A_BYTES, &mapB, &full[s], c * CHUNK_K, tn * BN, K);
                    if (SPLIT) {
                        tma_load_3d(slot + A_BYTES, &mapA, &full[s], kpa + c * CHUNK_K, tm * TM, K);
                        if (!CONVB)
                            tma_load_3d(slot + NP * A_BYTES + B_BYTES, &mapB, &full[s], kpb + c * CHUNK_K, tn * BN, K);
                    }
                }
                if (!ok) { if (status) status[K] = MEHDG_ETIMEOUT; break; }
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            uint32_t g = 0;
            int i = 0;
            for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x, ++i) {
                const int K = (int)(t / tiles_e), b = i & 1;
                bool ok = !(i >= 2 && !mbar_wait(&acc_empty[b], ((i >> 1) - 1) & 1));
                tc_fence_after();
                const uint32_t d = tmem + (uint32_t)(b * BN);
                for (int c = 0; ok && c < nchunk; ++c, ++g) {
                    const int s = (int)(g % SSTAGES);
                    if (!mbar_wait(CONVB ? &conv[s] : &full[s], (g / SSTAGES) & 1)) { ok = false; break; }
                    tc_fence_after();
                    unsigned char* slot = smem + (size_t)s * STG;
                    const uint64_t da = sdesc(s_addr(slot));
                    const uint64_t db = sdesc(s_addr(slot + NP * A_BYTES));
#pragma unroll
                    for (int j = 0; j < CHUNK_BYTES / 32; ++j) {
                        umma<BF16>(d, da + (uint64_t)(j * 2), db + (uint64_t)(j * 2), ID, (c | j) != 0);
                        if (SPLIT) {
                            const uint64_t dal = sdesc(s_addr(slot + A_BYTES));
                            const uint64_t dbl = sdesc(s_addr(slot + NP * A_BYTES + B_BYTES));
                            umma<BF16>(d, da + (uint64_t)(j * 2), dbl + (uint64_t)(j * 2), ID, 1u);
                            umma<BF16>(d, dal + (uint64_t)(j * 2), db + (uint64_t)(j * 2), ID, 1u);
                        }
                    }
                    umma_commit(&empty[s]);
                }
                if (!ok) { if (status) status[K] = MEHDG_ETIMEOUT; break; }
                umma_commit(&acc_full[b]);
            }
        }
    } else if (CONVB && warp >= 2 + EPI_WARPS) {
        // the B chunk of each slot, FP32 as loaded, into hi (in place) and lo
        // (the next B_BYTES): the same offsets, so the swizzled layout carries over
        const int ct = (warp - 2 - EPI_WARPS) * 32 + lane;
        uint32_t g = 0;
        for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
            const int K = (int)(t / tiles_e);
            bool ok = true;
            for (int c = 0; c < nchunk; ++c, ++g) {
                const int s = (int)(g % SSTAGES);
                if (!mbar_wait(&full[s], (g / SSTAGES) & 1)) { ok = false; break; }
                float4* hb = reinterpret_cast<float4*>(smem + (size_t)s * STG + NP * A_BYTES);
                float4* lb = reinterpret_cast<float4*>(smem + (size_t)s * STG + NP * A_BYTES + B_BYTES);
#pragma unroll 4
                for (int i = ct; i < B_BYTES / 16; i += 32 * CONV_WARPS) {
                    const float4 v = hb[i];
                    float4 h, l;
                    h.x = tf32_rn(v.x); l.x = tf32_rn(v.x - h.x);
                    h.y = tf32_rn(v.y); l.y = tf32_rn(v.y - h.y);
                    h.z = tf32_rn(v.z); l.z = tf32_rn(v.z - h.z);
                    h.w = tf32_rn(v.w); l.w = tf32_rn(v.w - h.w);
                    hb[i] = h;
                    lb[i] = l;
                }
                // the tensor cores read shared memory through the async proxy
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                __syncwarp();
                if (lane == 0) mbar_arrive(&conv[s]);
            }
            if (!ok) { if (lane == 0 && status) status[K] = MEHDG_ETIMEOUT; break; }
        }
    } else {
        // lane quarter q, column group h (and h + 4 when BN = 256: the second
        // group's C is read after the first group's stores, which keeps the
        // registers of one group)
        const int ew = warp - 2, q = warp & 3, h = ew >> 2;
        constexpr int GPW = BN > 128 ? BN / 128 : 1;      // column groups per warp
        float* S0 = Sall;
        int i = 0;
        for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x, ++i) {
            const int K = (int)(t / tiles_e), rem = (int)(t % tiles_e);
            const int tm = rem % tiles_m, tn = rem / tiles_m, b = i & 1;
            const int row = tm * TM + 32 * q + lane;
            int hh = h, col0 = tn * BN + hh * W;
            // columns of this warp's slice inside the update (0 for rows past M)
            int nc = (hh < NH && row < M) ? min(W, N - col0) : 0;
            float* Cp = S0 + (size_t)K * ld * ld + (size_t)(r0 + row) + (size_t)(c0 + col0) * ld;
            float cv[W];
            if (!STORE) {
                const float* p = Cp;
#pragma unroll
                for (int j = 0; j < W; ++j) { cv[j] = j < nc ? __ldcs(p) : 0.f; p += ld; }
            }
            const bool ok = __all_sync(0xffffffffu, mbar_wait(&acc_full[b], (i >> 1) & 1));
            if (!ok) { if (lane == 0 && status) status[K] = MEHDG_ETIMEOUT; break; }
            tc_fence_after();
#pragma unroll 1
            for (int gs = 0; gs < GPW; ++gs) {
                if (gs > 0) {
                    hh = h + 4 * gs;
                    col0 = tn * BN + hh * W;
                    nc = (hh < NH && row < M) ? min(W, N - col0) : 0;
                    Cp = S0 + (size_t)K * ld * ld + (size_t)(r0 + row) + (size_t)(c0 + col0) * ld;
                    if (!STORE) {
                        const float* p = Cp;
#pragma unroll
                        for (int j = 0; j < W; ++j) { cv[j] = j < nc ? __ldcs(p) : 0.f; p += ld; }
                    }
                }
                if (hh < NH && !STORE && bo.p) {
                    // an update whose result is the next TRSM's B operand: C - D as FP32
                    // rows of kp entries (row = its K index), S left as it is
                    uint32_t r[32];
                    tmem_ld32(tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(b * BN + hh * W), r);
                    float* qf = reinterpret_cast<float*>(bo.p) +
                                ((size_t)K * bo.nc + bo.c0 + col0) * (size_t)bo.kp + bo.k0 + row;
#pragma unroll
                    for (int j = 0; j < W; ++j) {
                        if (j < nc) qf[0] = cv[j] - __uint_as_float(r[j]);
                        qf += bo.kp;
                    }
                } else if (hh < NH) {
                    uint32_t r[32];
                    tmem_ld32(tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(b * BN + hh * W), r);
                    // a fresh copy of the base pointer, so that the 32 store addresses are
                    // recomputed instead of being kept live from the loads
                    float* p;
                    asm volatile("mov.b64 %0, %1;" : "=l"(p) : "l"(Cp));
#pragma unroll
                    for (int j = 0; j < W; ++j) {
                        if (j < nc) __stcs(p, STORE ? __uint_as_float(r[j]) : cv[j] - __uint_as_float(r[j]));
                        p += ld;
                    }
                    if (STORE && bo.p) {
                        // the same product as the next update's split-BF16 B operand
                        // (row = its K index, column = its N index): [hi | lo] rows
                        __nv_bfloat16* qb = reinterpret_cast<__nv_bfloat16*>(bo.p) +
                                            ((size_t)K * bo.nc + bo.c0 + col0) * (size_t)(2 * bo.kp) + bo.k0 + row;
#pragma unroll
                        for (int j = 0; j < W; ++j) {
                            if (j < nc) {
                                const float v = __uint_as_float(r[j]);
                                const __nv_bfloat16 hi = __float2bfloat16_rn(v);
                                qb[0] = hi;
                                qb[bo.kp] = __float2bfloat16_rn(v - __bfloat162float(hi));
                            }
                            qb += 2 * bo.kp;
                        }
                    }
                }
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&acc_empty[b]);
        }
    }
    __syncwarp();
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"((uint32_t)(2 * BN)) : "memory");
    }
}

// ---------------------------------------------------------------- packing
// Operand rounding: TF32 (round to nearest on 10 mantissa bits, kept in FP32
// storage) or BF16.  With split precision a product a b is taken as
// a_hi b_hi + a_hi b_lo + a_lo b_hi (hi = round(x), lo = round(x - hi)): both
// panels hold the two K-segments [hi | lo] and the MMA issuer takes the three
// products from one ring slot.
template <bool BF16>
__device__ __forceinline__ float op_round(float x) {
    if constexpr (BF16) return __bfloat162float(__float2bfloat16_rn(x));
    else return tf32_rn(x);
}
template <bool BF16>
__device__ __forceinline__ void op_store(void* out, size_t o, float x) {
    if constexpr (BF16) reinterpret_cast<__nv_bfloat16*>(out)[o] = __float2bfloat16_rn(x);
    else reinterpret_cast<float*>(out)[o] = x;     // already TF32-rounded
}
// write x into the nseg K-segments [hi (| lo)] of a row
template <bool BF16>
__device__ __forceinline__ void op_put(void* out, size_t row_base, int Kp, int k, int nseg, float x) {
    const float hi = op_round<BF16>(x);
    op_store<BF16>(out, row_base + k, hi);
    if (nseg == 2) op_store<BF16>(out, row_base + Kp + k, op_round<BF16>(x - hi));
}

// eight consecutive K entries of one packed row, as 16-byte stores
template <bool BF16>
__device__ __forceinline__ void op_store8(void* out, size_t o, const float (&x)[8]) {
    if constexpr (BF16) {
        uint4 u;
        uint32_t* w = reinterpret_cast<uint32_t*>(&u);
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            __nv_bfloat162 h = __floats2bfloat162_rn(x[2 * j], x[2 * j + 1]);
            w[j] = *reinterpret_cast<uint32_t*>(&h);
        }
        *reinterpret_cast<uint4*>(reinterpret_cast<__nv_bfloat16*>(out) + o) = u;
    } else {
        float4* d = reinterpret_cast<float4*>(reinterpret_cast<float*>(out) + o);
        d[0] = make_float4(x[0], x[1], x[2], x[3]);
        d[1] = make_float4(x[4], x[5], x[6], x[7]);
    }
}
// write x[0..8) (K entries k..k+7, k a multiple of 8) into the nseg K-segments [hi (| lo)] of a row
template <bool BF16>
__device__ __forceinline__ void op_put8(void* out, size_t row_base, int Kp, int k, int nseg, const float (&x)[8]) {
    float hi[8], lo[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) { hi[j] = op_round<BF16>(x[j]); lo[j] = op_round<BF16>(x[j] - hi[j]); }
    op_store8<BF16>(out, row_base + k, hi);
    if (nseg == 2) op_store8<BF16>(out, row_base + Kp + k, lo);
}

// A panel: Ap[K][m][seg*Kp + kout + k] = L[r0+m][k0+k] (k < Kd, else 0), elements
// erows rows apart.  A 64 (m) x 32 (k) tile is transposed through shared
// memory; each thread then writes 8 consecutive k of one row per segment.
// Kp and kout are multiples of 32; grid.y covers the k blocks written.
template <bool BF16>
__global__ void __launch_bounds__(256)
pack_A_kernel(const float* __restrict__ Sall, int64_t ld, int r0, int k0, int M, int Kd, int Kp,
              int nseg, int erows, int kout, void* __restrict__ out) {
    const int K = blockIdx.z;
    const float* S = Sall + (size_t)K * ld * ld;
    __shared__ float t[32][65];
    const int m0 = blockIdx.x * 64, kk0 = blockIdx.y * 32;
    {
        const int tx = threadIdx.x & 63, ty = threadIdx.x >> 6;
        const int m = m0 + tx;
#pragma unroll
        for (int i = ty; i < 32; i += 4) {
            const int k = kk0 + i;
            t[i][tx] = (k < Kd && m < M) ? S[(size_t)(r0 + m) + (size_t)(k0 + k) * ld] : 0.f;
        }
    }
    __syncthreads();
    const int ml = threadIdx.x >> 2, kq = (threadIdx.x & 3) * 8;
    const int m = m0 + ml;
    if (m >= M) return;
    float x[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) x[j] = t[kq + j][ml];
    op_put8<BF16>(out, ((size_t)K * erows + m) * (size_t)(nseg * Kp), Kp, kout + kk0 + kq, nseg, x);
}
// B panel: Bp[K][n][seg*Kp + k] = U[k0+k][c0+n] (contiguous in k on both sides);
// one warp per column n, 8 consecutive k per lane.  k0 is a multiple of 4 and
// ld of 256, so the 16-byte loads are aligned; Kp is a multiple of 8.
template <bool BF16>
__global__ void __launch_bounds__(256)
pack_B_kernel(const float* __restrict__ Sall, int64_t ld, int k0, int c0, int N, int Kd, int Kp,
              int nseg, void* __restrict__ out) {
    const int K = blockIdx.z;
    const float* S = Sall + (size_t)K * ld * ld;
    const int n = blockIdx.x * 8 + (threadIdx.x >> 5);
    if (n >= N) return;
    const float* col = S + (size_t)k0 + (size_t)(c0 + n) * ld;
    for (int k = (threadIdx.x & 31) * 8; k < Kp; k += 256) {
        float x[8];
        if (k + 8 <= Kd) {
            const float4 a = __ldg(reinterpret_cast<const float4*>(col + k));
            const float4 b = __ldg(reinterpret_cast<const float4*>(col + k + 4));
            x[0] = a.x; x[1] = a.y; x[2] = a.z; x[3] = a.w; x[4] = b.x; x[5] = b.y; x[6] = b.z; x[7] = b.w;
        } else {
#pragma unroll
            for (int j = 0; j < 8; ++j) x[j] = k + j < Kd ? col[k + j] : 0.f;
        }
        op_put8<BF16>(out, ((size_t)K * N + n) * (size_t)(nseg * Kp), Kp, k, nseg, x);
    }
}

// Gathered rows of an A panel (split BF16): slot i in [i0, min(i1, nr)) of
// the net permutation perm with cont[i] != i gives packed row rows[i] - r0
// the values S[rows[cont[i]]][k0 + k] for k < kn (the rest of the row stays
// as packed).  One warp per slot; the source row is read along its columns.
__global__ void __launch_bounds__(256)
pack_A_gather_kernel(const float* __restrict__ Sall, int64_t ld, const int32_t* __restrict__ perm, int i0, int i1,
                     int r0, int M, int k0, int kn, int Kp, void* __restrict__ out) {
    const int K = blockIdx.y;
    const float* S = Sall + (size_t)K * ld * ld;
    const int32_t* pl = perm + (size_t)K * LU_PW;
    const int nr = pl[0];
    const int32_t* rows = pl + 1;
    const int32_t* cont = rows + 2 * LU_NB;
    const int i = i0 + blockIdx.x * 8 + (threadIdx.x >> 5), lane = threadIdx.x & 31;
    if (i >= i1 || i >= nr) return;
    const int ci = cont[i];
    if (ci == i) return;
    const int m = rows[i] - r0, src = rows[ci];
    if (m < 0 || m >= M || src < 0 || src >= ld) return;
    const size_t base = ((size_t)K * M + m) * (size_t)(2 * Kp);
    for (int k = lane; k < kn; k += 32) op_put<true>(out, base, Kp, k, 2, S[(size_t)src + (size_t)(k0 + k) * ld]);
}

PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;

bool encoder() {
    if (g_encode) return true;
    cudaDriverEntryPointQueryResult q;
    void* fn = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess || !fn)
        return false;
    g_encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
    return true;
}

// 3-D map over packed panels [nK][rows][Kp] (elements elem_rows rows apart,
// default rows), box = 128 bytes of K x box_rows
bool make_map(CUtensorMap* map, const void* base, bool bf16, int Kp, int rows, int64_t nK, int box_rows,
              int elem_rows = 0) {
    const int es = bf16 ? 2 : 4;
    if (elem_rows <= 0) elem_rows = rows;
    cuuint64_t dims[3] = {(cuuint64_t)Kp, (cuuint64_t)rows, (cuuint64_t)nK};
    cuuint64_t strides[2] = {(cuuint64_t)Kp * es, (cuuint64_t)Kp * es * elem_rows};
    cuuint32_t box[3] = {(cuuint32_t)(CHUNK_BYTES / es), (cuuint32_t)box_rows, 1};
    cuuint32_t estr[3] = {1, 1, 1};
    CUresult r = g_encode(map, bf16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3,
                          const_cast<void*>(base),
                          dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                          CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

bool wide_tiles() {
    const char* f = std::getenv("MEHDG_TC_BN");
    return !(f && std::atoi(f) == 128);
}

int sm_count() {
    static int n = 0;
    if (n == 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        if (n <= 0) n = 1;
    }
    return n;
}

// one operand panel: ld rows x (2 segments x 256) FP32 per element
size_t panel_bytes(int64_t nK, int64_t ld) {
    size_t b = (size_t)nK * ld * 2 * LU_NB * 4;
    return (b + 255) & ~(size_t)255;
}

template <int BN, bool BF16, bool STORE, bool SPLIT>
cudaError_t launch_stream(const CUtensorMap& a, const CUtensorMap& b, const LUPlan& P, int r0, int c0, int M, int N,
                          int nchunk, int kpa, int kpb, cudaStream_t st, BqOut bo = BqOut()) {
    const int tiles_m = (M + TM - 1) / TM, tiles_n = (N + BN - 1) / BN;
    const int64_t ntiles = (int64_t)tiles_m * tiles_n * P.nK;
    constexpr size_t sm = stream_smem_bytes<BN, SPLIT>();
    auto kern = tc_stream_kernel<BN, BF16, STORE, SPLIT>;
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    const int64_t grid = std::min<int64_t>(ntiles, (int64_t)sm_count());
    kern<<<(unsigned)grid, stream_threads<STORE>(), sm, st>>>(a, b, (float*)P.S, P.ld, r0, c0, M, N, nchunk, kpa, kpb,
                                                         tiles_m, tiles_n, ntiles, P.status, bo);
    MEHDG_COUNT(1);
    return cudaGetLastError();
}

// one update / solve product with the operand panels already packed
template <bool BF16, bool STORE, bool SPLIT>
cudaError_t launch_stream_bn(int BN, const CUtensorMap& a, const CUtensorMap& b, const LUPlan& P, int r0, int c0,
                             int M, int N, int nchunk, int kpa, int kpb, cudaStream_t st, BqOut bo = BqOut()) {
    if constexpr (BF16 && !STORE && SPLIT)
        if (BN == 256) return launch_stream<256, BF16, STORE, SPLIT>(a, b, P, r0, c0, M, N, nchunk, kpa, kpb, st, bo);
    if (BN == 128) return launch_stream<128, BF16, STORE, SPLIT>(a, b, P, r0, c0, M, N, nchunk, kpa, kpb, st, bo);
    if (BN == 64) return launch_stream<64, BF16, STORE, SPLIT>(a, b, P, r0, c0, M, N, nchunk, kpa, kpb, st, bo);
    return launch_stream<32, BF16, STORE, SPLIT>(a, b, P, r0, c0, M, N, nchunk, kpa, kpb, st, bo);
}


// Inverse X = L^-1 of the unit-lower 256 x 256 diagonal block L of every
// element, written as the K-major operand panel Ap[K][m][k] = X[m][k] (TF32
// rounded, split into [hi | lo] when nseg = 2).  One CTA per (32-column block
// jb of X, element), by block forward substitution over the 32-row blocks ib:
//   X[ib] = L[ib][ib]^-1 (E[ib] - sum_{jb <= kb < ib} L[ib][kb] X[kb]),
// E the identity's block.  The 32 x 32 products run from shared memory (each
// thread 4 outputs), the next block of L is fetched into registers while the
// current one is used, and the unit-lower diagonal solves are done by the
// warps, 4 columns each, with shuffles.
template <bool BF16>
__global__ void __launch_bounds__(256)
trtri256_kernel(const float* __restrict__ Sall, int64_t ld, int c0, int nseg, void* __restrict__ Ap) {
    constexpr int T = 256, NB = T / 32;
    const int K = blockIdx.y, jb = blockIdx.x;
    const float* L = Sall + (size_t)K * ld * ld + (size_t)c0 + (size_t)c0 * ld;   // L[i][k] = L[i + k ld]
    __shared__ float Xs[NB][32][33];
    __shared__ float Lb[2][32][33];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int r = tid >> 3, c4 = (tid & 7) * 4;       // product layout: row r, columns c4..c4+3
    // block sequence: for ib = jb..7: (ib, jb), (ib, jb+1), ..., (ib, ib)
    int total = 0;
    for (int ib = jb; ib < NB; ++ib) total += ib - jb + 1;
    auto fetch = [&](int ib, int kb, float (&v)[4]) {
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int e = tid + 256 * u, i = e & 31, k = e >> 5;
            v[u] = L[(size_t)(32 * ib + i) + (size_t)(32 * kb + k) * ld];
        }
    };
    float acc[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) acc[q] = (r == c4 + q) ? 1.f : 0.f;   // E block of ib = jb
    float nxt[4];
    fetch(jb, jb, nxt);
    int ib = jb, kb = jb;
    for (int n = 0; n < total; ++n) {
        float (*lb)[33] = Lb[n & 1];
#pragma unroll
        for (int u = 0; u < 4; ++u) { const int e = tid + 256 * u; lb[e & 31][e >> 5] = nxt[u]; }
        __syncthreads();
        const int ib2 = kb < ib ? ib : ib + 1, kb2 = kb < ib ? kb + 1 : jb;
        if (n + 1 < total) fetch(ib2, kb2, nxt);
        if (kb < ib) {
#pragma unroll 8
            for (int k = 0; k < 32; ++k) {
                const float l = lb[r][k];
#pragma unroll
                for (int q = 0; q < 4; ++q) acc[q] -= l * Xs[kb][k][c4 + q];
            }
        } else {
#pragma unroll
            for (int q = 0; q < 4; ++q) Xs[ib][r][c4 + q] = acc[q];
            __syncthreads();
#pragma unroll
            for (int cc = 0; cc < 4; ++cc) {
                const int col = 4 * warp + cc;
                float x = Xs[ib][lane][col];
#pragma unroll
                for (int k = 0; k < 32; ++k) {
                    const float xk = __shfl_sync(0xffffffffu, x, k);
                    if (lane > k) x -= lb[lane][k] * xk;
                }
                Xs[ib][lane][col] = x;
            }
#pragma unroll
            for (int q = 0; q < 4; ++q) acc[q] = 0.f;
        }
        ib = ib2; kb = kb2;
    }
    __syncthreads();
    for (int m = warp; m < T; m += 8) {
        const int mb = m >> 5;
        const float x = mb < jb ? 0.f : Xs[mb][m & 31][lane];
        op_put<BF16>(Ap, ((size_t)K * T + m) * (size_t)(nseg * T), T, 32 * jb + lane, nseg, x);
    }
}

// Row exchanges of the outer panel c0 on the trailing columns, fused with the
// packing of the TRSM's B operand: one warp per column gathers the rows of
// the net permutation (the 256 block rows and the rows below that take
// part), writes the rows below that change, and writes the new block rows
// to the FP32 panel Bp[K][n][256] (the TRSM product splits them in shared
// memory).  The block rows of S are not written back: the TRSM product
// overwrites them.
__global__ void __launch_bounds__(256)
laswp_pack_kernel(float* __restrict__ Sall, int64_t ld, const int32_t* __restrict__ perm, int j0, int N,
                  float* __restrict__ Bp) {
    const int K = blockIdx.y;
    float* S = Sall + (size_t)K * ld * ld;
    const int32_t* pl = perm + (size_t)K * LU_PW;
    const int nr = pl[0];
    const int32_t* rows = pl + 1;
    const int32_t* cont = rows + 2 * LU_NB;
    __shared__ float buf[8][2 * LU_NB];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int n = blockIdx.x * 8 + warp;
    if (n >= N) return;
    float* Sc = S + (size_t)(j0 + n) * ld;
    float* b = buf[warp];
    // gather, four rows per lane and iteration so that their loads overlap
    for (int i0 = lane; i0 < nr; i0 += 128) {
        float v[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int i = i0 + 32 * u;
            v[u] = i < nr ? Sc[rows[i]] : 0.f;
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) { const int i = i0 + 32 * u; if (i < nr) b[i] = v[u]; }
    }
    __syncwarp();
    float* out = Bp + ((size_t)K * N + n) * (size_t)LU_NB;
    for (int i = lane; i < nr; i += 32) {
        const int ci = cont[i];
        const float v = b[ci];
        if (i < LU_NB) out[i] = v;
        else if (ci != i) Sc[rows[i]] = v;
    }
}

}  // namespace

// Rows [c0, c0+256) of the columns [j0, j1): U12 = L11^-1 A12 on the tensor
// cores, through the explicit inverse of the unit-lower block L11.
namespace {
// the TRSM product with B = rows [c0, c0+256) of the columns [j0, j0+N), FP32 in Bp
cudaError_t trsm256_product(const LUPlan& P, int c0, int j0, int N, void* Ap, void* Bp, const BqOut* bq,
                            cudaStream_t st) {
    const int Kd = LU_NB, nseg = 2, nchunk = Kd / (CHUNK_BYTES / 4);
    {
        dim3 gt(LU_NB / 32, (unsigned)P.nK);
        trtri256_kernel<false><<<gt, 256, 0, st>>>((const float*)P.S, P.ld, c0, nseg, Ap);
        MEHDG_COUNT(1);
    }
    const int BN = N >= 128 ? 128 : (N >= 64 ? 64 : 32);
    CUtensorMap ma, mb;
    // B: plain FP32 rows of 256 (split by the kernel's converter warps)
    if (!make_map(&ma, Ap, false, nseg * Kd, 256, P.nK, TM) || !make_map(&mb, Bp, false, Kd, N, P.nK, BN))
        return cudaErrorInvalidValue;
    return launch_stream_bn<false, true, true>(BN, ma, mb, P, c0, j0, 256, N, nchunk, Kd, Kd, st,
                                               bq ? *bq : BqOut());
}

// the three operand panels of the workspace: A, B, and the next update's B (split BF16)
unsigned char* panel_base(const LUPlan& P) {
    return reinterpret_cast<unsigned char*>(P.work) + lu_perm_bytes(P.nK, P.ld);
}
}  // namespace

void* gemm_tc_bq_panel(const LUPlan& P) { return panel_base(P) + 2 * panel_bytes(P.nK, P.ld); }
void* gemm_tc_bp_panel(const LUPlan& P) { return panel_base(P) + panel_bytes(P.nK, P.ld); }

// The outer step right of panel c0: row exchanges of the columns [c0+256, ld)
// by the panel's net permutation, fused with the packing of B, then the TRSM
// U12 = L11^-1 A12 of their rows [c0, c0+256) on the tensor cores in split
// TF32 (every mixed mode: the explicit inverse of L11 amplifies operand
// rounding, and one-pass TF32 or BF16 here leaves the factors too inexact for
// the FP64 refinement).
cudaError_t gemm_tc_swap_trsm256(const LUPlan& P, const int32_t* perm, int c0, cudaStream_t st, const BqOut* bq) {
    const int j0 = c0 + LU_NB, N = (int)P.ld - j0;
    if (N <= 0) return cudaSuccess;
    if (!encoder()) return cudaErrorNotSupported;
    unsigned char* w = panel_base(P);
    const size_t pan = panel_bytes(P.nK, P.ld);
    void* Ap = w;
    float* Bp = reinterpret_cast<float*>(w + pan);
    dim3 gb((unsigned)((N + 7) / 8), (unsigned)P.nK);
    laswp_pack_kernel<<<gb, 256, 0, st>>>((float*)P.S, P.ld, perm, j0, N, Bp);
    MEHDG_COUNT(1);
    return trsm256_product(P, c0, j0, N, Ap, Bp, bq, st);
}

// The TRSM product alone, with its B operand (rows [c0, c0+256) of the
// columns right of them) already in the FP32 B panel
cudaError_t gemm_tc_trsm256(const LUPlan& P, int c0, cudaStream_t st, const BqOut* bq) {
    const int j0 = c0 + LU_NB, N = (int)P.ld - j0;
    if (N <= 0) return cudaSuccess;
    if (!encoder()) return cudaErrorNotSupported;
    return trsm256_product(P, c0, j0, N, panel_base(P), gemm_tc_bp_panel(P), bq, st);
}

size_t gemm_tc_work_bytes(int64_t nK, int64_t ld, int prec) {
    // panels of ld rows x 2 KB per element: split FP32/TF32 operands of depth
    // 256 or split BF16 of depth 512 (A, B, and the next update's B written by
    // the TRSM products); split BF16 adds the multipliers of a pair of outer
    // panels, kept from one update to the next
    return (prec == MEHDG_MIXED_BF16X3 ? 4 : 3) * panel_bytes(nK, ld);
}

void* gemm_tc_a2_panel(const LUPlan& P) { return panel_base(P) + 3 * panel_bytes(P.nK, P.ld); }

cudaError_t gemm_tc_pack_a2(const LUPlan& P, int erows, int row0, int kp, int kout, int r0, int k0, int M, int Kd,
                            cudaStream_t st) {
    if (M <= 0) return cudaSuccess;
    if (P.prec != MEHDG_MIXED_BF16X3 || Kd % 32 || kout % 32 || kout + Kd > kp || row0 < 0 || row0 + M > erows ||
        (size_t)erows * 4 * kp > (size_t)P.ld * 2 * LU_NB * 4)
        return cudaErrorInvalidValue;
    __nv_bfloat16* out = reinterpret_cast<__nv_bfloat16*>(gemm_tc_a2_panel(P)) + (size_t)row0 * 2 * kp;
    dim3 g3((unsigned)((M + 63) / 64), (unsigned)(Kd / 32), (unsigned)P.nK);
    pack_A_kernel<true><<<g3, 256, 0, st>>>((const float*)P.S, P.ld, r0, k0, M, Kd, kp, 2, erows, kout, out);
    MEHDG_COUNT(1);
    return cudaGetLastError();
}

cudaError_t gemm_tc_gather_a2(const LUPlan& P, int erows, int kp, int r0, int k0, const AGather& g, cudaStream_t st) {
    if (g.i1 <= g.i0) return cudaSuccess;
    if (P.prec != MEHDG_MIXED_BF16X3 || g.kn > kp || (size_t)erows * 4 * kp > (size_t)P.ld * 2 * LU_NB * 4)
        return cudaErrorInvalidValue;
    dim3 gg((unsigned)((g.i1 - g.i0 + 7) / 8), (unsigned)P.nK);
    pack_A_gather_kernel<<<gg, 256, 0, st>>>((const float*)P.S, P.ld, g.perm, g.i0, g.i1, r0, erows, k0, g.kn, kp,
                                             gemm_tc_a2_panel(P));
    MEHDG_COUNT(1);
    return cudaGetLastError();
}

cudaError_t gemm_tc_update(const LUPlan& P, int r0, int c0, int k0, int M, int N, int Kd, cudaStream_t st,
                           int ph_pack, int ph_gemm, double flops, const PackedB* b, const AGather* g,
                           const BqOut* out, const PackedA* a) {
    if (M <= 0 || N <= 0) return cudaSuccess;
    const bool bf16 = P.prec == MEHDG_MIXED_BF16 || P.prec == MEHDG_MIXED_BF16X3;
    const bool split = P.prec == MEHDG_MIXED_TF32X3 || P.prec == MEHDG_MIXED_BF16X3;
    // split BF16 only, whole row tiles; a packed A takes no gathers here
    if ((b || g || out || a) && (!(bf16 && split) || M < TM || (a && g))) return cudaErrorInvalidValue;
    if (M < TM) return gemm_simt_update_f32(P, r0, c0, k0, M, N, Kd, st);   // a few tiny inner updates
    if (!encoder()) return cudaErrorNotSupported;
    const int nseg = split ? 2 : 1;
    const int es = bf16 ? 2 : 4;
    const int chunk_k = CHUNK_BYTES / es;
    const int Kp = (Kd + chunk_k - 1) / chunk_k * chunk_k;
    const int nchunk = Kp / chunk_k;
    // each operand panel holds ld rows x 2 KB per element
    if ((size_t)std::max(M, N) * nseg * Kp * es > (size_t)P.ld * 2 * LU_NB * 4) return cudaErrorInvalidValue;
    unsigned char* w = panel_base(P);
    const size_t pan = panel_bytes(P.nK, P.ld);
    void* Ap = w;
    void* Bp = w + pan;
    // pack
    {
        const int ev = ph_pack >= 0 ? prof_begin(P.prof, ph_pack, st) : -1;
        dim3 g3((unsigned)((M + 63) / 64), (unsigned)(Kp / 32), (unsigned)P.nK);
        if (!a) {
            if (bf16) pack_A_kernel<true><<<g3, 256, 0, st>>>((const float*)P.S, P.ld, r0, k0, M, Kd, Kp, nseg, M, 0, Ap);
            else pack_A_kernel<false><<<g3, 256, 0, st>>>((const float*)P.S, P.ld, r0, k0, M, Kd, Kp, nseg, M, 0, Ap);
            MEHDG_COUNT(1);
        }
        if (!a && g && g->i1 > g->i0) {
            dim3 gg((unsigned)((g->i1 - g->i0 + 7) / 8), (unsigned)P.nK);
            pack_A_gather_kernel<<<gg, 256, 0, st>>>((const float*)P.S, P.ld, g->perm, g->i0, g->i1, r0, M, k0,
                                                     std::min(g->kn, Kd), Kp, Ap);
            MEHDG_COUNT(1);
        }
        if (!b) {
            dim3 gb((unsigned)((N + 7) / 8), 1, (unsigned)P.nK);
            if (bf16) pack_B_kernel<true><<<gb, 256, 0, st>>>((const float*)P.S, P.ld, k0, c0, N, Kd, Kp, nseg, Bp);
            else pack_B_kernel<false><<<gb, 256, 0, st>>>((const float*)P.S, P.ld, k0, c0, N, Kd, Kp, nseg, Bp);
            MEHDG_COUNT(1);
        }
        if (ev >= 0) prof_end(P.prof, ev, st, 0.0);
    }
    // split BF16 updates at least 256 wide take 128 x 256 tiles: their MMAs read
    // a quarter fewer shared-memory bytes per flop (MEHDG_TC_BN=128 keeps
    // 128 x 128 tiles)
    int BN = N >= 128 ? 128 : (N >= 64 ? 64 : 32);
    if (bf16 && split && N >= 256 && wide_tiles()) BN = 256;
    CUtensorMap ma, mb;
    bool ok;
    int kpa = Kp, kpb = Kp;
    if (a) {
        // rows row0.. of the packed A panel
        if (a->kp < Kp || a->row0 < 0 || a->row0 + M > a->erows) return cudaErrorInvalidValue;
        const void* base = reinterpret_cast<const __nv_bfloat16*>(a->p) + (size_t)a->row0 * 2 * a->kp;
        ok = make_map(&ma, base, true, 2 * a->kp, M, P.nK, TM, a->erows);
        kpa = a->kp;
    } else {
        ok = make_map(&ma, Ap, bf16, nseg * Kp, M, P.nK, TM);
    }
    if (b) {
        // rows c0.. of the packed panel; a K chunk of this update never reaches the lo segment
        if (b->kp < Kp || b->c0 < 0 || b->c0 + N > b->nc) return cudaErrorInvalidValue;
        const void* base = reinterpret_cast<const __nv_bfloat16*>(b->p) + (size_t)b->c0 * 2 * b->kp;
        ok = ok && make_map(&mb, base, true, 2 * b->kp, N, P.nK, BN, b->nc);
        kpb = b->kp;
    } else {
        ok = ok && make_map(&mb, Bp, bf16, nseg * Kp, N, P.nK, BN);
    }
    if (!ok) return cudaErrorInvalidValue;
    const int ev = ph_gemm >= 0 ? prof_begin(P.prof, ph_gemm, st) : -1;
    cudaError_t e;
    if (bf16) e = split ? launch_stream_bn<true, false, true>(BN, ma, mb, P, r0, c0, M, N, nchunk, kpa, kpb, st,
                                                              out ? *out : BqOut())
                        : launch_stream_bn<true, false, false>(BN, ma, mb, P, r0, c0, M, N, nchunk, Kp, kpb, st);
    else e = split ? launch_stream_bn<false, false, true>(BN, ma, mb, P, r0, c0, M, N, nchunk, Kp, kpb, st)
                   : launch_stream_bn<false, false, false>(BN, ma, mb, P, r0, c0, M, N, nchunk, Kp, kpb, st);
    if (ev >= 0) prof_end(P.prof, ev, st, flops);
    return e;
}

// test hook: one trailing update on caller-owned FP32 column-major matrices
extern "C" int mehdg_test_trailing_update(int64_t nK, int64_t ld, float* S, int r0, int c0, int k0, int M, int N,
                                          int Kd, int prec, void* work, void* stream) {
    LUPlan P;
    std::memset(&P, 0, sizeof(P));
    P.nK = nK; P.ld = ld; P.N = ld; P.fp64 = false; P.prec = prec; P.S = S; P.work = work;
    cudaError_t e = gemm_tc_update(P, r0, c0, k0, M, N, Kd, (cudaStream_t)stream);
    return e == cudaSuccess ? MEHDG_OK : MEHDG_ECUDA;
}

extern "C" size_t mehdg_test_trailing_work_bytes(int64_t nK, int64_t ld) {
    return lu_perm_bytes(nK, ld) + gemm_tc_work_bytes(nK, ld, 1);
}
