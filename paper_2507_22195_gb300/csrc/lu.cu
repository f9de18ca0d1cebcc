// lu.cu -- batched dense LU with partial pivoting of every S^K, and solves.
//
// S^K is column-major with a padded size ld (multiple of 256; the padding is
// an identity block, so pivots never leave the true rows).  The factorisation
// is right-looking over outer panels of NB = 256 columns; each outer panel is
// factored recursively (halves, down to 32-column leaves):
//   leaf   : one CTA per element factors the (ld-c) x 32 panel, the whole
//            leaf or 8 (or fewer) columns at a time in shared memory with
//            partial pivoting (largest |a|, ties to the lowest row),
//            left-looking between the sub-panels, and applies its row
//            exchanges to the other 224 columns of the outer panel;
//   inner  : TRSM with the unit-lower triangle, trailing update of the right
//            half (width 32 in FP32 on the SIMT pipe, 64 and 128 on the tensor
//            cores), recursion on the right half;
//   outer  : row swaps and TRSM of the rows right of the panel, then the
//            trailing update C -= L21 U12 with depth 256.
// Rows left of an outer panel are not swapped again (LINPACK order); the
// forward solve replays each outer panel's swaps before its block column.
// The trailing updates run on the tensor cores for the mixed precisions
// (gemm_tc.cu) and on the FP64 pipe for MEHDG_FP64.
#include <cstdio>
#include <cstdlib>
#include <type_traits>
#include "common.cuh"
#include "kernels.cuh"
#include "lu_internal.cuh"

namespace {

constexpr int LEAF = 32;
constexpr int PANEL_THREADS = 512;

__device__ __forceinline__ float tabs(float x) { return fabsf(x); }
__device__ __forceinline__ double tabs(double x) { return fabs(x); }

// ---------------------------------------------------------------- leaf panel
// One CTA per element; the IB columns of a sub-panel live in shared memory.
// Row ownership is fixed (row r belongs to thread r mod PANEL_THREADS), so a
// pivot column costs two barriers: one to publish the per-warp maxima, one
// after every thread has read the old pivot row and row cc.  The search for
// the next pivot runs on the values the update has just produced.
// one FP32 CTA per SM (fewer elements than SMs): 1024 threads; four per SM
// (small leaves of many elements): 256; otherwise 512 (FP64 keeps 512 so that
// its registers do not spill)
template <class TS, int MINB> constexpr int panel_threads() {
    return (MINB == 1 && sizeof(TS) == 4) ? 2 * PANEL_THREADS : MINB == 4 ? PANEL_THREADS / 2 : PANEL_THREADS;
}

template <class TS, int IB, int MINB>
__global__ void __launch_bounds__(panel_threads<TS, MINB>(), MINB)
panel_kernel(TS* __restrict__ Sall, int64_t ld, int c, int32_t* __restrict__ pivall, int32_t* status) {
    constexpr int nth = panel_threads<TS, MINB>(), NW = nth / 32;
    const int K = blockIdx.x;
    TS* S = Sall + (size_t)K * ld * ld;
    int32_t* piv = pivall + (size_t)K * ld;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int R0 = (int)(ld - c);                  // rows of the panel
    TS* X = reinterpret_cast<TS*>(smem_raw);       // [IB][R0] column-major sub-panel
    constexpr int UT = IB < LEAF ? LEAF : 1;      // left-looking staging, only with several sub-panels
    __shared__ TS Utop[UT][IB];
    __shared__ TS Lt[UT][UT + 1];
    __shared__ TS s_swap[UT][2 * IB];
    __shared__ TS red_v[2][NW];
    __shared__ int red_i[2][NW];
    __shared__ int s_piv[IB];
    __shared__ TS s_prow[2][IB], s_crow[2][IB];
    __shared__ int s_rows[2 * IB], s_cont[2 * IB], s_nr;
    __shared__ int s_pall[LEAF];                   // the leaf's pivots, relative to c
    __shared__ int s_lrows[2 * LEAF], s_lcont[2 * LEAF], s_lnr;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    bool singular = false;
    for (int jb = 0; jb < LEAF; jb += IB) {
        const int R = R0 - jb;                     // rows of this sub-panel, starting at c + jb
        // (a) left-looking update with the earlier sub-panels of this leaf
        bool staged = false;
        if constexpr (IB < LEAF) if (jb > 0) {
            staged = true;
            // U part: rows c..c+jb-1 of the sub-panel columns, unit-lower forward
            // substitution with the jb x jb block of L staged in shared memory
            for (int i = tid; i < jb * jb; i += nth) Lt[i % jb][i / jb] = S[(size_t)(c + i % jb) + (size_t)(c + i / jb) * ld];
            for (int i = tid; i < jb * IB; i += nth) Utop[i % jb][i / jb] = S[(size_t)(c + i % jb) + (size_t)(c + jb + i / jb) * ld];
            __syncthreads();
            if (tid < IB)
                for (int i = 1; i < jb; ++i) {
                    TS s = Utop[i][tid];
                    for (int t = 0; t < i; ++t) s -= Lt[i][t] * Utop[t][tid];
                    Utop[i][tid] = s;
                }
            __syncthreads();
            for (int i = tid; i < jb * IB; i += nth) S[(size_t)(c + i % jb) + (size_t)(c + jb + i / jb) * ld] = Utop[i % jb][i / jb];
            // L part into shared memory: X[cc][r] = A[c+jb+r][col] - sum_t L[c+jb+r][c+t] U[t][cc];
            // two rows per thread and iteration, IB loads of each row at a time
            constexpr int RB = 2;
            for (int rb = tid; rb < R; rb += nth * RB) {
                TS acc[RB][IB];
#pragma unroll
                for (int u = 0; u < RB; ++u) {
                    const int r = rb + u * nth;
                    const TS* row = S + (size_t)(c + jb + (r < R ? r : 0));
#pragma unroll
                    for (int cc = 0; cc < IB; ++cc) acc[u][cc] = r < R ? row[(size_t)(c + jb + cc) * ld] : (TS)0;
                }
                for (int t0 = 0; t0 < jb; t0 += IB) {
                    TS l[RB][IB];
#pragma unroll
                    for (int u = 0; u < RB; ++u) {
                        const int r = rb + u * nth;
                        const TS* row = S + (size_t)(c + jb + (r < R ? r : 0));
#pragma unroll
                        for (int tt = 0; tt < IB; ++tt) l[u][tt] = r < R ? row[(size_t)(c + t0 + tt) * ld] : (TS)0;
                    }
#pragma unroll
                    for (int u = 0; u < RB; ++u)
#pragma unroll
                        for (int tt = 0; tt < IB; ++tt)
#pragma unroll
                            for (int cc = 0; cc < IB; ++cc) acc[u][cc] -= l[u][tt] * Utop[t0 + tt][cc];
                }
#pragma unroll
                for (int u = 0; u < RB; ++u) {
                    const int r = rb + u * nth;
                    if (r < R) {
#pragma unroll
                        for (int cc = 0; cc < IB; ++cc) X[cc * R0 + r] = acc[u][cc];
                    }
                }
            }
        }
        if (!staged) {
            // several rows per thread and iteration, so 32 loads are in flight
            constexpr int RB = IB >= 32 ? 1 : 32 / IB;
            for (int rb = tid; rb < R; rb += nth * RB) {
                TS v[RB][IB];
#pragma unroll
                for (int u = 0; u < RB; ++u) {
                    const int r = rb + u * nth;
                    const TS* row = S + (size_t)(c + (r < R ? r : 0));
#pragma unroll
                    for (int cc = 0; cc < IB; ++cc) v[u][cc] = r < R ? row[(size_t)(c + cc) * ld] : (TS)0;
                }
#pragma unroll
                for (int u = 0; u < RB; ++u) {
                    const int r = rb + u * nth;
                    if (r < R) {
#pragma unroll
                        for (int cc = 0; cc < IB; ++cc) X[cc * R0 + r] = v[u][cc];
                    }
                }
            }
        }
        // (b) partial pivoting factorisation of the IB columns in shared memory;
        // every thread reads and writes only its own rows, except for the two
        // rows copied to s_prow / s_crow between the barriers of a column.
        // (magnitudes compared in the storage precision: the order is that of
        // their exact FP64 promotions, and it keeps the FP64 pipe free)
        TS best = (TS)-1; int bi = 0x7fffffff;
        for (int r = tid; r < R; r += nth) {
            const TS a = tabs(X[r]);
            if (a > best) { best = a; bi = r; }          // increasing r: ties keep the lowest
        }
#pragma unroll
        for (int cc = 0; cc < IB; ++cc) {
            for (int o = 16; o > 0; o >>= 1) {
                TS ob = __shfl_xor_sync(0xffffffffu, best, o);
                int oi = __shfl_xor_sync(0xffffffffu, bi, o);
                if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
            }
            if (lane == 0) { red_v[cc & 1][wid] = best; red_i[cc & 1][wid] = bi; }
            __syncthreads();
            best = lane < NW ? red_v[cc & 1][lane] : (TS)-1;
            bi = lane < NW ? red_i[cc & 1][lane] : 0x7fffffff;
            for (int o = 16; o > 0; o >>= 1) {
                TS ob = __shfl_xor_sync(0xffffffffu, best, o);
                int oi = __shfl_xor_sync(0xffffffffu, bi, o);
                if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
            }
            // no finite candidate (all zero or NaN): keep the row, report singular
            if (bi >= R || !(best > (TS)0)) { bi = cc; best = (TS)0; }
            const int pr = bi;
            if (best == (TS)0) singular = true;
            if (tid < IB) { s_prow[cc & 1][tid] = X[tid * R0 + pr]; s_crow[cc & 1][tid] = X[tid * R0 + cc]; }
            if (tid == 0) s_piv[cc] = pr;
            __syncthreads();
            // narrow sub-panels: the pivot row and the old row cc in registers (the
            // row loop stores to X, which the compiler cannot tell apart from s_prow)
            constexpr int HR = IB <= 8 ? IB : 1;
            TS prow_r[HR], crow_r[HR];
            if constexpr (IB <= 8) {
#pragma unroll
                for (int q = 0; q < IB; ++q) { prow_r[q] = s_prow[cc & 1][q]; crow_r[q] = s_crow[cc & 1][q]; }
            }
            const TS* prow = IB <= 8 ? prow_r : s_prow[cc & 1];
            const TS* crow = IB <= 8 ? crow_r : s_crow[cc & 1];
            const TS pivv = prow[cc];
            const TS inv = pivv != (TS)0 ? (TS)1 / pivv : (TS)0;
            best = (TS)-1; bi = 0x7fffffff;
            int r = tid;
            if (r == cc) {                         // row cc takes the pivot row
                if (pr != cc) {
#pragma unroll
                    for (int q = 0; q < IB; ++q) X[q * R0 + r] = prow[q];
                }
                r += nth;
            } else if (r < cc) {
                r += nth;
            }
            for (; r < R; r += nth) {
                if (r == pr) {                     // row pr takes the old row cc
#pragma unroll
                    for (int q = 0; q < cc; ++q) X[q * R0 + r] = crow[q];
                    const TS l = crow[cc] * inv;
                    X[cc * R0 + r] = l;
#pragma unroll
                    for (int q = cc + 1; q < IB; ++q) {
                        const TS nv = crow[q] - l * prow[q];
                        X[q * R0 + r] = nv;
                        if (q == cc + 1) { const TS a = tabs(nv); if (a > best) { best = a; bi = r; } }
                    }
                } else {
                    const TS l = X[cc * R0 + r] * inv;
                    X[cc * R0 + r] = l;
#pragma unroll
                    for (int q = cc + 1; q < IB; ++q) {
                        const TS nv = X[q * R0 + r] - l * prow[q];
                        X[q * R0 + r] = nv;
                        if (q == cc + 1) { const TS a = tabs(nv); if (a > best) { best = a; bi = r; } }
                    }
                }
            }
        }
        // (c) write back the own rows, record pivots
        for (int r = tid; r < R; r += nth) {
            TS* row = S + (size_t)(c + jb + r);
#pragma unroll
            for (int cc = 0; cc < IB; ++cc) row[(size_t)(c + jb + cc) * ld] = X[cc * R0 + r];
        }
        if (tid < IB) { piv[c + jb + tid] = c + jb + s_piv[tid]; s_pall[jb + tid] = jb + s_piv[tid]; }
        if constexpr (IB < LEAF) {
            // (d) apply the IB swaps to the other columns of the leaf as one net
            // permutation: slot i (row s_rows[i]) takes the old content of slot s_cont[i]
            if (tid == 0) {
                int nr = IB;
                for (int i = 0; i < IB; ++i) { s_rows[i] = jb + i; s_cont[i] = i; }
                for (int i = 0; i < IB; ++i) {
                    const int b = jb + s_piv[i];
                    if (b == jb + i) continue;
                    int sb = -1;
                    if (b < jb + IB) sb = b - jb;
                    else {
                        for (int j = IB; j < nr; ++j) if (s_rows[j] == b) { sb = j; break; }
                        if (sb < 0) { sb = nr++; s_rows[sb] = b; s_cont[sb] = sb; }
                    }
                    const int t = s_cont[i]; s_cont[i] = s_cont[sb]; s_cont[sb] = t;
                }
                s_nr = nr;
            }
            __syncthreads();
            const int nr = s_nr;
            for (int e = tid; e < LEAF * 2 * IB; e += nth) {
                const int t = e / (2 * IB), i = e % (2 * IB);
                if (i < nr && (t < jb || t >= jb + IB)) s_swap[t][i] = S[(size_t)(c + s_rows[i]) + (size_t)(c + t) * ld];
            }
            __syncthreads();
            for (int e = tid; e < LEAF * 2 * IB; e += nth) {
                const int t = e / (2 * IB), i = e % (2 * IB);
                if (i < nr && (t < jb || t >= jb + IB) && s_cont[i] != i)
                    S[(size_t)(c + s_rows[i]) + (size_t)(c + t) * ld] = s_swap[t][s_cont[i]];
            }
            __syncthreads();
        }
    }
    // (e) the leaf's row exchanges on the other columns of its outer panel, as
    // one net permutation of at most 64 rows (slot i, row c + s_lrows[i], takes
    // the old content of slot s_lcont[i]); one warp per column, the values in
    // registers and exchanged by shuffles
    __syncthreads();
    if (wid == 0) {
        for (int i = lane; i < 2 * LEAF; i += 32) { s_lrows[i] = i; s_lcont[i] = i; }
        __syncwarp();
        int nr = LEAF;
        for (int i = 0; i < LEAF; ++i) {
            const int b = s_pall[i];
            if (b == i) continue;
            int sb;
            if (b < LEAF) sb = b;
            else {
                const unsigned hit = __ballot_sync(0xffffffffu, LEAF + lane < nr && s_lrows[LEAF + lane] == b);
                if (hit) sb = LEAF + __ffs(hit) - 1;
                else {
                    sb = nr++;
                    if (lane == 0) s_lrows[sb] = b;
                }
            }
            __syncwarp();
            if (lane == 0) { const int t = s_lcont[i]; s_lcont[i] = s_lcont[sb]; s_lcont[sb] = t; }
            __syncwarp();
        }
        if (lane == 0) s_lnr = nr;
    }
    __syncthreads();
    {
        const int nr = s_lnr;
        const int c0 = (c / LU_NB) * LU_NB, nleft = c - c0;
        const int r0 = s_lrows[lane], r1 = s_lrows[lane + 32];
        const int q0 = s_lcont[lane], q1 = s_lcont[lane + 32];
        const bool w0 = lane < nr && q0 != lane, w1 = lane + 32 < nr && q1 != lane + 32;
        // four columns per warp and iteration: their loads are in flight together
        constexpr int CU = 4;
        const int nw = nth / 32;
        for (int j0 = wid * CU; j0 < LU_NB - LEAF; j0 += nw * CU) {
            TS v0[CU], v1[CU];
            TS* Sc[CU];
#pragma unroll
            for (int u = 0; u < CU; ++u) {
                const int j = j0 + u;
                const int col = j < nleft ? c0 + j : c + j - nleft + LEAF;
                Sc[u] = S + (size_t)col * ld + c;
                const bool in = j < LU_NB - LEAF;
                v0[u] = in && lane < nr ? Sc[u][r0] : (TS)0;
                v1[u] = in && lane + 32 < nr ? Sc[u][r1] : (TS)0;
            }
#pragma unroll
            for (int u = 0; u < CU; ++u) {
                const TS a0 = __shfl_sync(0xffffffffu, v0[u], q0 & 31), b0 = __shfl_sync(0xffffffffu, v1[u], q0 & 31);
                const TS a1 = __shfl_sync(0xffffffffu, v0[u], q1 & 31), b1 = __shfl_sync(0xffffffffu, v1[u], q1 & 31);
                if (j0 + u < LU_NB - LEAF) {
                    if (w0) Sc[u][r0] = q0 < 32 ? a0 : b0;
                    if (w1) Sc[u][r1] = q1 < 32 ? a1 : b1;
                }
            }
        }
    }
    if (singular && tid == 0 && status) status[K] = MEHDG_ESINGULAR;
}

// ---------------------------------------------------------------- row swaps
// Net permutation of the swap sequence piv[c0 .. c0+w): slots 0..w-1 are the
// rows c0..c0+w-1, further slots the rows below the block that take part;
// after the sequence, slot i holds the old content of slot cont[i].  One warp
// per element: rows/cont live in shared memory, the search for a row below
// the block is done by the 32 lanes at once.
__global__ void __launch_bounds__(128)
perm_build_kernel(const int32_t* __restrict__ pivall, int64_t ld, int c0, int w,
                  int32_t* __restrict__ perm /*[nK][1 + 4w]*/, int nK) {
    extern __shared__ int32_t sp[];               // per warp: rows[2w], cont[2w]
    const int wl = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int K = blockIdx.x * 4 + wl;
    if (K >= nK) return;
    const int32_t* piv = pivall + (size_t)K * ld;
    int32_t* rows = sp + wl * 4 * w;
    int32_t* cont = rows + 2 * w;
    for (int i = lane; i < w; i += 32) { rows[i] = c0 + i; cont[i] = i; }
    __syncwarp();
    int nr = w;
    for (int i = 0; i < w; ++i) {
        const int b = piv[c0 + i];
        if (b == c0 + i) continue;
        int sb;
        if (b < c0 + w) sb = b - c0;
        else {
            sb = -1;
            for (int j0 = w; j0 < nr && sb < 0; j0 += 32) {
                int j = j0 + lane;
                unsigned hit = __ballot_sync(0xffffffffu, j < nr && rows[j] == b);
                if (hit) sb = j0 + __ffs(hit) - 1;
            }
            if (sb < 0) {
                sb = nr++;
                if (lane == 0) { rows[sb] = b; cont[sb] = sb; }
            }
        }
        __syncwarp();
        if (lane == 0) { int t = cont[i]; cont[i] = cont[sb]; cont[sb] = t; }
        __syncwarp();
    }
    int32_t* out = perm + (size_t)K * (1 + 4 * w);
    for (int i = lane; i < nr; i += 32) { out[1 + i] = rows[i]; out[1 + 2 * w + i] = cont[i]; }
    if (lane == 0) out[0] = nr;
}

// Row exchanges of the columns [j0, j1): new row rows[i] = old row rows[cont[i]].
// One warp per column; the block rows [c0, c0+w) are read contiguously.
template <class TS>
__global__ void __launch_bounds__(256)
laswp_kernel(TS* __restrict__ Sall, int64_t ld, const int32_t* __restrict__ perm, int w, int j0, int j1) {
    const int K = blockIdx.y;
    TS* S = Sall + (size_t)K * ld * ld;
    const int32_t* pl = perm + (size_t)K * (1 + 4 * w);
    const int nr = pl[0];
    const int32_t* rows = pl + 1;
    const int32_t* cont = rows + 2 * w;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    TS* buf = reinterpret_cast<TS*>(smem_raw) + (size_t)warp * 2 * w;
    const int col = j0 + blockIdx.x * 8 + warp;
    if (col >= j1) return;
    TS* Sc = S + (size_t)col * ld;
    for (int i = lane; i < nr; i += 32) buf[i] = Sc[rows[i]];
    __syncwarp();
    for (int i = lane; i < nr; i += 32) {
        const int src = cont[i];
        if (src != i) Sc[rows[i]] = buf[src];
    }
}

// ---------------------------------------------------------------- TRSM
// X = L^-1 X for X = rows [c0, c0+t) of columns [j0, j1), L = unit-lower
// S[c0:c0+t, c0:c0+t].  One CTA per 32 columns; 256 threads = 32 cols x 8.
// Loads and stores of X and of the diagonal blocks run with consecutive
// threads on consecutive rows of a column (coalesced in column-major S); X
// and the blocks are padded to 33 columns in shared memory.
constexpr int TRSM_XS = 33;
template <class TS>
__global__ void __launch_bounds__(256)
trsm_kernel(TS* __restrict__ Sall, int64_t ld, int c0, int t, int j0, int j1) {
    const int K = blockIdx.y;
    TS* S = Sall + (size_t)K * ld * ld;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    TS* X = reinterpret_cast<TS*>(smem_raw);        // [t][33]
    TS* Lo = X + (size_t)t * TRSM_XS;                // [t - 32][33]: L below the diagonal block
    __shared__ TS Lb[32][33];
    const int tc = threadIdx.x & 31, tr = threadIdx.x >> 5;
    const int cb = j0 + blockIdx.x * 32;             // first column of this CTA
    for (int e = threadIdx.x; e < t * 32; e += 256) {
        const int i = e % t, cc = e / t;
        X[i * TRSM_XS + cc] = cb + cc < j1 ? S[(size_t)(c0 + i) + (size_t)(cb + cc) * ld] : (TS)0;
    }
    __syncthreads();
    for (int rb = 0; rb < t; rb += 32) {
        for (int e = threadIdx.x; e < 32 * 32; e += 256) {
            const int i = e & 31, q = e >> 5;
            Lb[i][q] = S[(size_t)(c0 + rb + i) + (size_t)(c0 + rb + q) * ld];
        }
        // the L rows below the block, staged with coalesced loads (lane = row)
        for (int i0 = rb + 32; i0 < t; i0 += 32)
            for (int q = tr; q < 32; q += 8)
                if (i0 + tc < t) Lo[(i0 + tc - 32) * 33 + q] = S[(size_t)(c0 + i0 + tc) + (size_t)(c0 + rb + q) * ld];
        __syncthreads();
        if (tr == 0) {
            // the 32 x 32 unit-lower block, one column per lane, in registers:
            // once x[q] is final every later row takes its term (the same
            // subtraction order per entry as the row-by-row form, but 31 - q
            // independent updates per step instead of one dependent chain)
            TS x[32];
#pragma unroll
            for (int i = 0; i < 32; ++i) x[i] = X[(rb + i) * TRSM_XS + tc];
#pragma unroll
            for (int q = 0; q < 31; ++q)
#pragma unroll
                for (int i = q + 1; i < 32; ++i) x[i] -= Lb[i][q] * x[q];
#pragma unroll
            for (int i = 1; i < 32; ++i) X[(rb + i) * TRSM_XS + tc] = x[i];
        }
        __syncthreads();
        for (int i = rb + 32 + tr; i < t; i += 8) {
            TS s = X[i * TRSM_XS + tc];
            const TS* Lr = Lo + (i - 32) * 33;
#pragma unroll 8
            for (int q = 0; q < 32; ++q) s -= Lr[q] * X[(rb + q) * TRSM_XS + tc];
            X[i * TRSM_XS + tc] = s;
        }
        __syncthreads();
    }
    for (int e = threadIdx.x; e < t * 32; e += 256) {
        const int i = e % t, cc = e / t;
        if (cb + cc < j1) S[(size_t)(c0 + i) + (size_t)(cb + cc) * ld] = X[i * TRSM_XS + cc];
    }
}

// ---------------------------------------------------------------- SIMT GEMM
// C[r0.., c0..] -= A[r0.., k0..] * B[k0.., c0..] (M x N, depth Kd), col-major
// blocks of the same S^K.  64x64 tile, 256 threads, 4x4 per thread.
template <class TS>
__global__ void __launch_bounds__(256)
gemm_simt_kernel(TS* __restrict__ Sall, int64_t ld, int r0, int c0, int k0, int M, int N, int Kd) {
    const int K = blockIdx.z;
    TS* S = Sall + (size_t)K * ld * ld;
    const int tm = blockIdx.x * 64, tn = blockIdx.y * 64;
    __shared__ TS As[16][64 + 1];
    __shared__ TS Bs[16][64 + 1];
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    TS acc[4][4] = {};
    for (int kk = 0; kk < Kd; kk += 16) {
        for (int i = threadIdx.x; i < 16 * 64; i += 256) {
            int a_m = i % 64, a_k = i / 64;
            int gm = tm + a_m;
            As[a_k][a_m] = (gm < M) ? S[(size_t)(r0 + gm) + (size_t)(k0 + kk + a_k) * ld] : (TS)0;
            int b_k = i % 16, b_n = i / 16;
            int gn = tn + b_n;
            Bs[b_k][b_n] = (gn < N) ? S[(size_t)(k0 + kk + b_k) + (size_t)(c0 + gn) * ld] : (TS)0;
        }
        __syncthreads();
#pragma unroll
        for (int q = 0; q < 16; ++q) {
            TS a[4], b[4];
            for (int i = 0; i < 4; ++i) { a[i] = As[q][tx + 16 * i]; b[i] = Bs[q][ty + 16 * i]; }
            for (int i = 0; i < 4; ++i)
                for (int j = 0; j < 4; ++j) acc[i][j] += a[i] * b[j];
        }
        __syncthreads();
    }
    for (int i = 0; i < 4; ++i)
        for (int j = 0; j < 4; ++j) {
            int gm = tm + tx + 16 * i, gn = tn + ty + 16 * j;
            if (gm < M && gn < N) S[(size_t)(r0 + gm) + (size_t)(c0 + gn) * ld] -= acc[i][j];
        }
}

// ---------------------------------------------------------------- solve
// CL CTAs (one thread-block cluster) per element.  The 32-row blocks of the
// right-hand side are owned cyclically (block b by rank b mod CL, and inside
// it by warp (b / CL) mod 16); y lives in each CTA's shared memory, and an
// owned block holds working values while every other block receives the final
// values its owner broadcasts into the CTA (distributed shared memory).
// Forward (unit-lower L, LINPACK order): at each outer panel the net
// permutation kept by the factorisation is applied (gather through
// distributed shared memory between full cluster barriers); then, block by
// block, the owning warp of block s+1 first applies block s to its rows,
// solves its 32 x 32 triangle, broadcasts the result and arrives on the
// cluster barrier, while the other warps arrive at once and apply block s to
// their rows.  Backward with U the same way from the last block.  One cluster
// barrier phase per block; the factors are read once per solve.
// Arithmetic in the factor precision; r scaled by its max norm.
__device__ __forceinline__ uint32_t cl_rank() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}
__device__ __forceinline__ void cl_arrive() { asm volatile("barrier.cluster.arrive.release.aligned;" ::: "memory"); }
__device__ __forceinline__ void cl_wait() { asm volatile("barrier.cluster.wait.acquire.aligned;" ::: "memory"); }
__device__ __forceinline__ void cl_sync() { cl_arrive(); cl_wait(); }
__device__ __forceinline__ uint32_t cl_map(const void* p, uint32_t rank) {
    uint32_t a;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;"
                 : "=r"(a) : "r"((uint32_t)__cvta_generic_to_shared(p)), "r"(rank));
    return a;
}
__device__ __forceinline__ void cl_st(uint32_t a, float v) { asm volatile("st.shared::cluster.f32 [%0], %1;" ::"r"(a), "f"(v) : "memory"); }
__device__ __forceinline__ void cl_st(uint32_t a, double v) { asm volatile("st.shared::cluster.f64 [%0], %1;" ::"r"(a), "d"(v) : "memory"); }
__device__ __forceinline__ float cl_ld(uint32_t a, float) {
    float v;
    asm volatile("ld.shared::cluster.f32 %0, [%1];" : "=f"(v) : "r"(a) : "memory");
    return v;
}
__device__ __forceinline__ double cl_ld(uint32_t a, double) {
    double v;
    asm volatile("ld.shared::cluster.f64 %0, [%1];" : "=d"(v) : "r"(a) : "memory");
    return v;
}

constexpr int SOLVE_THREADS = 512;
constexpr int SOLVE_WARPS = SOLVE_THREADS / 32;

template <class TS, int CL>
__global__ void __cluster_dims__(CL, 1, 1) __launch_bounds__(SOLVE_THREADS)
solve_kernel(const TS* __restrict__ Sall, int64_t ld, const int32_t* __restrict__ perms, int64_t nK,
             const double* __restrict__ rall, double* __restrict__ xall, const int32_t* skip) {
    constexpr int BPP = LU_NB / 32;                // 32-row blocks per outer panel
    const int K = blockIdx.x / CL;
    if (skip && skip[K]) return;                   // the whole cluster leaves together
    const int rank = CL > 1 ? (int)cl_rank() : 0;
    const TS* S = Sall + (size_t)K * ld * ld;
    const double* r = rall + (size_t)K * ld;
    double* x = xall + (size_t)K * ld;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    TS* y = reinterpret_cast<TS*>(smem_raw);        // [ld]
    TS* tmp = y + ld;                                // [2 NB] permutation gather
    __shared__ double red[SOLVE_WARPS];
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const int nb = (int)(ld / 32);
    auto owner = [](int b) { return b % CL; };
    auto wslot = [](int b) { return (b / CL) % SOLVE_WARPS; };
    // the first block this warp owns above (dir > 0) or below (dir < 0) block s
    auto first_mine = [&](int s, int dir) {
        // owned blocks of this warp: b = rank + CL (wid + SOLVE_WARPS u)
        const int step = CL * SOLVE_WARPS, b0 = rank + CL * wid;
        if (dir > 0) {
            if (b0 > s) return b0;
            return b0 + ((s - b0) / step + 1) * step;
        }
        if (b0 >= s) return -1;
        return b0 + ((s - 1 - b0) / step) * step;
    };
    auto broadcast = [&](int b, TS v) {
        for (int rk = 0; rk < CL; ++rk)
            if (rk != rank) cl_st(cl_map(&y[32 * b + lane], (uint32_t)rk), v);
    };
    // row block b -= (L or U)[block b, block s] * y_block(s)
    auto apply = [&](int b, int s) {
        const TS* col = S + (size_t)(32 * b + lane) + (size_t)(32 * s) * ld;
        TS l[32];
#pragma unroll
        for (int j = 0; j < 32; ++j) l[j] = col[(size_t)j * ld];
        TS acc = y[32 * b + lane];
#pragma unroll
        for (int j = 0; j < 32; ++j) acc -= l[j] * y[32 * s + j];
        y[32 * b + lane] = acc;
    };
    auto tri_lower = [&](int s) {
        const TS* col = S + (size_t)(32 * s + lane) + (size_t)(32 * s) * ld;
        TS l[32];
#pragma unroll
        for (int j = 0; j < 32; ++j) l[j] = col[(size_t)j * ld];
        TS yl = y[32 * s + lane];
#pragma unroll
        for (int i = 0; i < 32; ++i) {
            const TS yi = __shfl_sync(0xffffffffu, yl, i);
            if (lane > i) yl -= l[i] * yi;
        }
        y[32 * s + lane] = yl;
        broadcast(s, yl);
    };
    auto tri_upper = [&](int s) {
        const TS* col = S + (size_t)(32 * s + lane) + (size_t)(32 * s) * ld;
        TS u[32];
#pragma unroll
        for (int j = 0; j < 32; ++j) u[j] = col[(size_t)j * ld];
        TS yl = y[32 * s + lane];
#pragma unroll
        for (int i = 31; i >= 0; --i) {
            if (lane == i) yl = yl / u[i];
            const TS yi = __shfl_sync(0xffffffffu, yl, i);
            if (lane < i) yl -= u[i] * yi;
        }
        y[32 * s + lane] = yl;
        broadcast(s, yl);
    };

    // scale by the max norm of r (every CTA of the cluster computes it)
    double mx = 0.0;
    for (int i = tid; i < ld; i += SOLVE_THREADS) mx = fmax(mx, fabs(r[i]));
    for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if (lane == 0) red[wid] = mx;
    __syncthreads();
    mx = 0.0;
    for (int i = 0; i < SOLVE_WARPS; ++i) mx = fmax(mx, red[i]);
    const double sc = mx > 0.0 ? 1.0 / mx : 1.0;
    for (int i = tid; i < ld; i += SOLVE_THREADS)
        if (owner(i >> 5) == rank) y[i] = (TS)(r[i] * sc);

    // forward
    for (int s = 0; s < nb; ++s) {
        if (s % BPP == 0) {
            cl_sync();                              // every row below is up to date
            const int32_t* pl = perms + ((size_t)(s / BPP) * nK + K) * LU_PW;
            const int nr = pl[0];
            const int32_t* rows = pl + 1;
            const int32_t* cont = rows + 2 * LU_NB;
            for (int i = tid; i < nr; i += SOLVE_THREADS) {
                const int row = rows[i], ci = cont[i];
                if (ci != i && owner(row >> 5) == rank) {
                    const int src = rows[ci], os = owner(src >> 5);
                    tmp[i] = os == rank ? y[src] : cl_ld(cl_map(&y[src], (uint32_t)os), (TS)0);
                }
            }
            cl_sync();
            for (int i = tid; i < nr; i += SOLVE_THREADS) {
                const int row = rows[i];
                if (cont[i] != i && owner(row >> 5) == rank) y[row] = tmp[i];
            }
            cl_sync();
            if (owner(s) == rank && wid == wslot(s)) tri_lower(s);
            cl_sync();
        } else {
            cl_wait();
        }
        const bool next_regular = s + 1 < nb && (s + 1) % BPP != 0;
        const bool crit = next_regular && owner(s + 1) == rank && wid == wslot(s + 1);
        if (next_regular) {
            if (crit) { apply(s + 1, s); tri_lower(s + 1); }
            cl_arrive();
        }
        for (int b = first_mine(s, 1); b < nb; b += CL * SOLVE_WARPS)
            if (!(crit && b == s + 1)) apply(b, s);
    }
    // backward
    for (int s = nb - 1; s >= 0; --s) {
        if (s == nb - 1) {
            cl_sync();
            if (owner(s) == rank && wid == wslot(s)) tri_upper(s);
            cl_sync();
        } else {
            cl_wait();
        }
        const bool crit = s >= 1 && owner(s - 1) == rank && wid == wslot(s - 1);
        if (s >= 1) {
            if (crit) { apply(s - 1, s); tri_upper(s - 1); }
            cl_arrive();
        }
        for (int b = first_mine(s, -1); b >= 0; b -= CL * SOLVE_WARPS)
            if (!(crit && b == s - 1)) apply(b, s);
    }
    cl_sync();                                      // no CTA leaves while its y may still be read
    for (int i = tid; i < ld; i += SOLVE_THREADS)
        if (owner(i >> 5) == rank) x[i] = (double)y[i] * mx;
}

// sub-panel width: the whole leaf when its (ld - c) x 32 block fits in the
// shared-memory budget of one CTA (ctas per SM: 1, 2 or 4), else the widest
// of 8, 4, 2, 1 that fits (16 would need more registers than the left-looking
// step can hold)
template <class TS>
int pick_ib(int64_t rows, int ctas) {
    // with more elements than SMs, two CTAs per SM (the leaf is latency-bound:
    // a second element's leaf hides the barriers of the first) as long as the
    // sub-panel stays >= 4 wide; otherwise the widest sub-panel that fits
    // (four per SM: 47 KB, so that four CTAs with their up to 8.4 KB of static
    // shared memory and the 1 KB each that the driver keeps fit in 228 KB)
    const size_t budget1 = 200 * 1024, budget = ctas == 4 ? 47 * 1024 : ctas == 2 ? 100 * 1024 : budget1;
    if ((size_t)LEAF * rows * sizeof(TS) <= budget) return LEAF;
    int ib = 8;
    while (ib > 4 && (size_t)ib * rows * sizeof(TS) > budget) ib >>= 1;
    while (ib > 1 && (size_t)ib * rows * sizeof(TS) > budget1) ib >>= 1;
    return ib;
}

// Leaf CTAs per SM: 1 (1024 threads, up to 200 KB), 2 (512 threads, 100 KB)
// or 4 (256 threads, 47 KB: with more than two elements per SM a leaf launch
// then runs in one wave instead of two, for the FP32 leaves whose sub-panel of
// at least 8 columns fits -- at most 1504 rows; taller ones take 2, since
// 4-column sub-panels there measured slower than two CTAs with 8).  leaf_ctas
// 0 chooses from the element count; MEHDG_LEAF_CTAS_PER_SM (1, 2 or 4)
// overrides it.
template <class TS>
cudaError_t launch_panel(TS* S, int64_t ld, int c, int32_t* piv, int32_t* status, int64_t nK, int leaf_ctas,
                         cudaStream_t st) {
    int dev = 0, nsm = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    int ctas = (leaf_ctas == 1 || leaf_ctas == 2 || leaf_ctas == 4) ? leaf_ctas
             : nK > 2 * nsm ? 4 : nK > nsm ? 2 : 1;
    if (const char* f = std::getenv("MEHDG_LEAF_CTAS_PER_SM")) {
        const int v = std::atoi(f);
        if (v == 1 || v == 2 || v == 4) ctas = v;
    }
    if (ctas == 4 && (sizeof(TS) != 4 || pick_ib<TS>(ld - c, 4) < 8)) ctas = 2;
    const int ib = pick_ib<TS>(ld - c, ctas);
    size_t sm = (size_t)ib * (ld - c) * sizeof(TS);
    if (sm < 16) sm = 16;
    // registers: 64 per thread with two or four CTAs per SM, up to 128 with one
#define LP2(IB, MB) do { cudaFuncSetAttribute(panel_kernel<TS, IB, MB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm); \
                         panel_kernel<TS, IB, MB><<<(unsigned)nK, panel_threads<TS, MB>(), sm, st>>>(S, ld, c, piv, status); } while (0)
#define LP(IB) do { if (ctas == 2) LP2(IB, 2); else LP2(IB, 1); } while (0)
    if constexpr (sizeof(TS) == 4) {
        if (ctas == 4) {
            switch (ib) {
            case 32: LP2(32, 4); break;
            case 8: LP2(8, 4); break;
            default: LP2(4, 4); break;
            }
            MEHDG_COUNT(1);
            return cudaGetLastError();
        }
    }
    {
        switch (ib) {
        case 32: LP(32); break;
        case 8: LP(8); break;
        case 4: LP(4); break;
        case 2: LP(2); break;
        default: LP(1); break;
        }
    }
#undef LP
#undef LP2
    MEHDG_COUNT(1);
    return cudaGetLastError();
}

// net permutation of the swaps piv[c0 .. c0+w) of every element into perm ([nK][LU_PW])
cudaError_t launch_perm_build(const LUPlan& P, int c0, int w, int32_t* perm, cudaStream_t st) {
    perm_build_kernel<<<(unsigned)((P.nK + 3) / 4), 128, 4 * 4 * w * sizeof(int32_t), st>>>(P.piv, P.ld, c0, w,
                                                                                           perm, (int)P.nK);
    MEHDG_COUNT(1);
    return cudaGetLastError();
}

// outer panel c0's permutation, kept in the workspace for the solves
int32_t* panel_perm(const LUPlan& P, int c0) {
    return reinterpret_cast<int32_t*>(reinterpret_cast<unsigned char*>(P.work) + lu_perm_scratch_bytes(P.nK)) +
           (size_t)(c0 / LU_NB) * P.nK * LU_PW;
}

// row exchanges of the columns [j0, j1) by a permutation built with width w
template <class TS>
cudaError_t launch_laswp_perm(const LUPlan& P, const int32_t* perm, int w, int j0, int j1, cudaStream_t st) {
    if (j1 <= j0) return cudaSuccess;
    size_t sm = (size_t)8 * 2 * w * sizeof(TS);
    cudaFuncSetAttribute(laswp_kernel<TS>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    dim3 g((unsigned)((j1 - j0 + 7) / 8), (unsigned)P.nK);
    laswp_kernel<TS><<<g, 256, sm, st>>>((TS*)P.S, P.ld, perm, w, j0, j1);
    MEHDG_COUNT(1);
    return cudaGetLastError();
}


template <class TS>
cudaError_t launch_trsm(const LUPlan& P, int c0, int t, int j0, int j1, cudaStream_t st) {
    if (j1 <= j0) return cudaSuccess;
    size_t sm = ((size_t)t * TRSM_XS + (size_t)(t > 32 ? t - 32 : 0) * 33) * sizeof(TS);
    cudaFuncSetAttribute(trsm_kernel<TS>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    dim3 g((unsigned)((j1 - j0 + 31) / 32), (unsigned)P.nK);
    trsm_kernel<TS><<<g, 256, sm, st>>>((TS*)P.S, P.ld, c0, t, j0, j1);
    MEHDG_COUNT(1);
    return cudaGetLastError();
}

template <class TS>
cudaError_t launch_gemm_simt(const LUPlan& P, int r0, int c0, int k0, int M, int N, int Kd, cudaStream_t st) {
    if (M <= 0 || N <= 0) return cudaSuccess;
    dim3 g((unsigned)((M + 63) / 64), (unsigned)((N + 63) / 64), (unsigned)P.nK);
    gemm_simt_kernel<TS><<<g, 256, 0, st>>>((TS*)P.S, P.ld, r0, c0, k0, M, N, Kd);
    MEHDG_COUNT(1);
    return cudaGetLastError();
}

// The 32-wide inner update of the mixed-precision LU in exact FP32 on the
// SIMT pipe: C[r0+i, c0+j] -= sum_k L[r0+i, k0+k] U[k0+k, c0+j], j, k < 32.
// One thread per row, its 32 L and 32 C values loaded together (64 loads in
// flight), U staged in shared memory and read as broadcast float4; 32
// independent accumulators.  (The tensor-core path would pack both operands
// for a K = 32 product first.)
__global__ void __launch_bounds__(128)
update32_kernel(float* __restrict__ Sall, int64_t ld, int r0, int c0, int k0, int M) {
    const int K = blockIdx.y;
    float* S = Sall + (size_t)K * ld * ld;
    __shared__ __align__(16) float U[32][32];
    for (int i = threadIdx.x; i < 32 * 32; i += blockDim.x) {
        const int k = i & 31, j = i >> 5;
        U[k][j] = S[(size_t)(k0 + k) + (size_t)(c0 + j) * ld];
    }
    __syncthreads();
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= M) return;
    const float* pl = S + (size_t)(r0 + r) + (size_t)k0 * ld;
    const float* pc = S + (size_t)(r0 + r) + (size_t)c0 * ld;
    float l[32], acc[32];
#pragma unroll
    for (int k = 0; k < 32; ++k) { l[k] = pl[0]; pl += ld; }
#pragma unroll
    for (int j = 0; j < 32; ++j) { acc[j] = pc[0]; pc += ld; }
#pragma unroll
    for (int k = 0; k < 32; ++k) {
#pragma unroll
        for (int j = 0; j < 32; j += 4) {
            const float4 u = *reinterpret_cast<const float4*>(&U[k][j]);
            acc[j] = fmaf(-l[k], u.x, acc[j]);
            acc[j + 1] = fmaf(-l[k], u.y, acc[j + 1]);
            acc[j + 2] = fmaf(-l[k], u.z, acc[j + 2]);
            acc[j + 3] = fmaf(-l[k], u.w, acc[j + 3]);
        }
    }
    float* q = S + (size_t)(r0 + r) + (size_t)c0 * ld;
#pragma unroll
    for (int j = 0; j < 32; ++j) { q[0] = acc[j]; q += ld; }
}

cudaError_t launch_update32(const LUPlan& P, int r0, int c0, int k0, int M, cudaStream_t st) {
    if (M <= 0) return cudaSuccess;
    dim3 g((unsigned)((M + 127) / 128), (unsigned)P.nK);
    update32_kernel<<<g, 128, 0, st>>>((float*)P.S, P.ld, r0, c0, k0, M);
    MEHDG_COUNT(1);
    return cudaGetLastError();
}

template <class TS>
cudaError_t trailing_update(const LUPlan& P, int r0, int c0, int k0, int M, int N, int Kd, cudaStream_t st,
                            int ph_pack = -1, int ph_gemm = -1, double flops = 0.0, const PackedB* b = nullptr,
                            const AGather* g = nullptr, const BqOut* out = nullptr, const PackedA* a = nullptr) {
    if constexpr (std::is_same<TS, double>::value) {
        const int ev = ph_gemm >= 0 ? prof_begin(P.prof, ph_gemm, st) : -1;
        cudaError_t e = launch_gemm_simt<double>(P, r0, c0, k0, M, N, Kd, st);
        if (ev >= 0) prof_end(P.prof, ev, st, flops);
        return e;
    } else {
        if (N == 32 && Kd == 32 && !b && !g && !out && !a) return launch_update32(P, r0, c0, k0, M, st);
        return gemm_tc_update(P, r0, c0, k0, M, N, Kd, st, ph_pack, ph_gemm, flops, b, g, out, a);
    }
}

template <class TS>
cudaError_t rec_panel(const LUPlan& P, int c, int w, cudaStream_t st) {
    cudaError_t e;
    if (w == LEAF) return launch_panel<TS>((TS*)P.S, P.ld, c, P.piv, P.status, P.nK, P.leaf_ctas, st);
    // (every leaf applies its row exchanges to all columns of the outer panel,
    // so the halves need no separate exchange passes)
    int h = w / 2;
    if ((e = rec_panel<TS>(P, c, h, st)) != cudaSuccess) return e;
    if ((e = launch_trsm<TS>(P, c, h, c + h, c + w, st)) != cudaSuccess) return e;
    if ((e = trailing_update<TS>(P, c + h, c + h, c, (int)P.ld - (c + h), h, h, st)) != cudaSuccess) return e;
    return rec_panel<TS>(P, c + h, h, st);
}

// outer panel c0 factored, and its net permutation built (kept for the solves)
template <class TS>
cudaError_t outer_panel(const LUPlan& P, int c0, cudaStream_t st, int32_t** pp) {
    cudaError_t e;
    if ((e = rec_panel<TS>(P, c0, LU_NB, st)) != cudaSuccess) return e;
    *pp = panel_perm(P, c0);
    return launch_perm_build(P, c0, LU_NB, *pp, st);
}

inline double upd_flops(const LUPlan& P, int M, int N, int Kd) { return 2.0 * M * (double)N * Kd * (double)P.nK; }

template <class TS>
cudaError_t factor_t(const LUPlan& P, cudaStream_t st) {
    cudaError_t e;
    const int ld = (int)P.ld;
    for (int c0 = 0; c0 < ld; c0 += LU_NB) {
        int ev = prof_begin(P.prof, PH_LU_PANELS, st);
        int32_t* pp = nullptr;
        if ((e = outer_panel<TS>(P, c0, st, &pp)) != cudaSuccess) return e;
        const int j0 = c0 + LU_NB, rest = ld - j0;
        BqOut bo;
        if (rest > 0) {
            if constexpr (std::is_same<TS, double>::value) {
                if ((e = launch_laswp_perm<TS>(P, pp, LU_NB, j0, ld, st)) != cudaSuccess) return e;
                e = launch_trsm<TS>(P, c0, LU_NB, j0, ld, st);
            } else {
                // split BF16: the product also writes the update's B panel
                if (P.prec == MEHDG_MIXED_BF16X3) bo = BqOut{gemm_tc_bq_panel(P), rest, 0, 0, LU_NB};
                e = gemm_tc_swap_trsm256(P, pp, c0, st, bo.p ? &bo : nullptr);
            }
            if (e != cudaSuccess) return e;
        }
        prof_end(P.prof, ev, st, 0.0);
        if (rest > 0) {
            const PackedB pb{bo.p, bo.nc, 0, bo.kp};
            if ((e = trailing_update<TS>(P, j0, j0, c0, rest, rest, LU_NB, st, PH_PACK_OUTER, PH_GEMM_OUTER,
                                         upd_flops(P, rest, rest, LU_NB), bo.p ? &pb : nullptr)) != cudaSuccess)
                return e;
        }
    }
    return cudaSuccess;
}

// Split BF16 with the outer updates of two panels merged.  For the pair of
// outer panels a = [c0, c0+256) and b = [c0+256, c0+512), with R the columns
// right of b:
//   1. factor a; exchange the rows of all columns right of a by a's
//      permutation P_a and take U_a = L_aa^-1 A of their rows in a (TRSM
//      product, which also writes U_a as the B operand, K entries 0..255);
//   2. update only b's 256 columns by a (depth 256), and factor b;
//   3. on R: exchange rows by P_b (block rows written back); the block rows
//      of b then hold rows of A not yet updated by a: subtract their part
//      L_a(src) U_a, with the multipliers L_a of the rows they came from (a's
//      columns are not exchanged by P_b), the result going straight to the
//      TRSM's B operand;
//   4. U_b = L_bb^-1 (those rows) by the TRSM product (K entries 256..511 of
//      the same B operand);
//   5. one update of R's rows below b with depth 512: [L_a | L_b] [U_a; U_b],
//      L_a gathered through P_b for the rows that P_b moved.
// L_a of the rows below a is packed once, into a fourth operand panel that
// the three updates of the pair share (b's multipliers join it for step 5).
// The factors and the permutations kept for the solves are those of the
// one-panel form (rows left of a panel are never exchanged again); only the
// order of the roundings in the trailing matrix differs, and its C is
// streamed once per pair instead of twice.
cudaError_t factor_pairs(const LUPlan& P, cudaStream_t st) {
    cudaError_t e;
    const int ld = (int)P.ld;
    void* bq = gemm_tc_bq_panel(P);
    for (int ca = 0; ca < ld; ca += 2 * LU_NB) {
        const int cb = ca + LU_NB, jr = cb + LU_NB;
        int ev = prof_begin(P.prof, PH_LU_PANELS, st);
        int32_t *pa = nullptr, *pb = nullptr;
        if ((e = outer_panel<float>(P, ca, st, &pa)) != cudaSuccess) return e;
        if (cb >= ld) { prof_end(P.prof, ev, st, 0.0); break; }
        const int n1 = ld - cb;                       // columns right of a (b's and R's)
        const BqOut ba{bq, n1, 0, 0, 2 * LU_NB};
        if ((e = gemm_tc_swap_trsm256(P, pa, ca, st, &ba)) != cudaSuccess) return e;
        prof_end(P.prof, ev, st, 0.0);
        // a's multipliers of every row below a, packed once into the pair's A
        // panel (rows cb.., segment 512) for the three updates of the pair
        constexpr int KP2 = 2 * LU_NB;
        {
            const int evp = prof_begin(P.prof, PH_PACK_OUTER, st);
            if ((e = gemm_tc_pack_a2(P, n1, 0, KP2, 0, cb, ca, n1, LU_NB, st)) != cudaSuccess) return e;
            prof_end(P.prof, evp, st, 0.0);
            const PackedB b{bq, n1, 0, KP2};
            const PackedA a2{gemm_tc_a2_panel(P), n1, 0, KP2};
            if ((e = trailing_update<float>(P, cb, cb, ca, n1, LU_NB, LU_NB, st, PH_PACK_OUTER, PH_GEMM_OUTER,
                                            upd_flops(P, n1, LU_NB, LU_NB), &b, nullptr, nullptr, &a2)) != cudaSuccess)
                return e;
        }
        ev = prof_begin(P.prof, PH_LU_PANELS, st);
        if ((e = outer_panel<float>(P, cb, st, &pb)) != cudaSuccess) return e;
        const int nr = ld - jr;                       // columns of R
        if (nr <= 0) { prof_end(P.prof, ev, st, 0.0); break; }
        if ((e = launch_laswp_perm<float>(P, pb, LU_NB, jr, ld, st)) != cudaSuccess) return e;
        prof_end(P.prof, ev, st, 0.0);
        const PackedB b{bq, n1, LU_NB, KP2};
        {
            // the block rows of b (a's multipliers of the rows they came from),
            // corrected and written as the TRSM's FP32 B operand
            const int evp = prof_begin(P.prof, PH_PACK_OUTER, st);
            if ((e = gemm_tc_gather_a2(P, n1, KP2, cb, ca, AGather{pb, LU_NB, 0, LU_NB}, st)) != cudaSuccess)
                return e;
            prof_end(P.prof, evp, st, 0.0);
            const PackedA a2{gemm_tc_a2_panel(P), n1, 0, KP2};
            const BqOut bp{gemm_tc_bp_panel(P), nr, 0, 0, LU_NB};
            if ((e = trailing_update<float>(P, cb, jr, ca, LU_NB, nr, LU_NB, st, PH_PACK_OUTER, PH_GEMM_OUTER,
                                            upd_flops(P, LU_NB, nr, LU_NB), &b, nullptr, &bp, &a2)) != cudaSuccess)
                return e;
        }
        ev = prof_begin(P.prof, PH_LU_PANELS, st);
        const BqOut bb{bq, n1, LU_NB, LU_NB, 2 * LU_NB};
        if ((e = gemm_tc_trsm256(P, cb, st, &bb)) != cudaSuccess) return e;
        prof_end(P.prof, ev, st, 0.0);
        {
            // rows below b: b's multipliers beside a's (K entries 256..511), and a's
            // multipliers of the rows that P_b moved taken from their source rows
            const int evp = prof_begin(P.prof, PH_PACK_OUTER, st);
            if ((e = gemm_tc_pack_a2(P, n1, LU_NB, KP2, LU_NB, jr, cb, nr, LU_NB, st)) != cudaSuccess) return e;
            if ((e = gemm_tc_gather_a2(P, n1, KP2, cb, ca, AGather{pb, LU_NB, LU_NB, 2 * LU_NB}, st)) != cudaSuccess)
                return e;
            prof_end(P.prof, evp, st, 0.0);
            const PackedA a2{gemm_tc_a2_panel(P), n1, LU_NB, KP2};
            if ((e = trailing_update<float>(P, jr, jr, ca, nr, nr, 2 * LU_NB, st, PH_PACK_OUTER, PH_GEMM_OUTER,
                                            upd_flops(P, nr, nr, 2 * LU_NB), &b, nullptr, nullptr, &a2)) != cudaSuccess)
                return e;
        }
    }
    return cudaSuccess;
}

// merged pairs of outer updates: split BF16 only (the mode whose TRSM product
// writes the B operand); MEHDG_LU_PAIRS=0 selects the one-panel form
bool use_pairs(const LUPlan& P) {
    if (P.fp64 || P.prec != MEHDG_MIXED_BF16X3) return false;
    if (const char* f = std::getenv("MEHDG_LU_PAIRS")) return std::atoi(f) != 0;
    return true;
}

}  // namespace

cudaError_t gemm_simt_update_f32(const LUPlan& P, int r0, int c0, int k0, int M, int N, int Kd, cudaStream_t st) {
    return launch_gemm_simt<float>(P, r0, c0, k0, M, N, Kd, st);
}

size_t lu_work_bytes(int64_t nK, int64_t ld, bool fp64, int prec) {
    return lu_perm_bytes(nK, ld) + (fp64 ? 0 : gemm_tc_work_bytes(nK, ld, prec));
}

cudaError_t lu_factor(const LUPlan& P, cudaStream_t st) {
    if (P.fp64) return factor_t<double>(P, st);
    if (use_pairs(P)) return factor_pairs(P, st);
    return factor_t<float>(P, st);
}

namespace {
template <class TS, int CL>
cudaError_t launch_solve(const LUPlan& P, const int32_t* perms, const double* r, double* x, const int32_t* skip,
                         cudaStream_t st) {
    const size_t sm = sizeof(TS) * ((size_t)P.ld + 2 * LU_NB);
    cudaFuncSetAttribute(solve_kernel<TS, CL>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    solve_kernel<TS, CL><<<(unsigned)(P.nK * CL), SOLVE_THREADS, sm, st>>>((const TS*)P.S, P.ld, perms, P.nK, r, x,
                                                                         skip);
    MEHDG_COUNT(1);
    return cudaGetLastError();
}
template <class TS>
cudaError_t solve_t(const LUPlan& P, const int32_t* perms, const double* r, double* x, const int32_t* skip,
                    cudaStream_t st) {
    // CTAs per element: enough clusters to give every SM two CTAs, at most 8
    int dev = 0, nsm = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    int cl = 1;
    while (cl < 8 && P.nK * cl < 2 * (int64_t)nsm) cl *= 2;
    if (P.solve_ctas == 1 || P.solve_ctas == 2 || P.solve_ctas == 4 || P.solve_ctas == 8) cl = P.solve_ctas;
    // MEHDG_SOLVE_CTAS (1, 2, 4 or 8) overrides the choice, e.g. to test every variant
    if (const char* f = std::getenv("MEHDG_SOLVE_CTAS")) {
        const int v = std::atoi(f);
        if (v == 1 || v == 2 || v == 4 || v == 8) cl = v;
    }
    switch (cl) {
    case 8: return launch_solve<TS, 8>(P, perms, r, x, skip, st);
    case 4: return launch_solve<TS, 4>(P, perms, r, x, skip, st);
    case 2: return launch_solve<TS, 2>(P, perms, r, x, skip, st);
    default: return launch_solve<TS, 1>(P, perms, r, x, skip, st);
    }
}
}  // namespace

namespace {
// Transposed solve S^T x = r with the same factors.  The forward solve
// applies, block column by block column, the panel's row permutation (at the
// first block of each outer panel) and the elimination with the unit-lower
// block column, then the backward substitution with U: S^-1 = U^-1 T_last
// ... T_0.  Hence S^-T = T_0^T ... T_last^T U^-T: a forward substitution
// with U^T (dot products down U's columns, contiguous in column-major
// storage), then, from the last block column to the first, the transposed
// elimination (dots down L's columns below the block, then the unit-upper
// L_ss^T solve) and the inverse row permutation.  One CTA per element, x in
// shared memory in FP64 (the factors in their storage precision).
template <class TS>
__global__ void __launch_bounds__(512)
solve_T_kernel(const TS* __restrict__ Sall, int64_t ld, const int32_t* __restrict__ perms, int64_t nK,
               const double* __restrict__ rall, double* __restrict__ xall, const int32_t* skip) {
    constexpr int BPP = LU_NB / 32;
    const int K = blockIdx.x;
    if (skip && skip[K]) return;
    const TS* S = Sall + (size_t)K * ld * ld;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    double* z = reinterpret_cast<double*>(smem_raw);     // [ld]
    double* tmp = z + ld;                                 // [2 NB]
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5, nw = blockDim.x >> 5;
    const int nb = (int)(ld / 32);
    for (int i = tid; i < ld; i += blockDim.x) z[i] = rall[(size_t)K * ld + i];
    __syncthreads();
    // z = U^-T z
    for (int s = 0; s < nb; ++s) {
        const int r1 = 32 * s;
        for (int j = wid; j < 32; j += nw) {
            const TS* col = S + (size_t)(r1 + j) * ld;
            double acc = 0.0;
            for (int i = lane; i < r1; i += 32) acc += (double)col[i] * z[i];
            for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
            if (lane == 0) z[r1 + j] -= acc;
        }
        __syncthreads();
        if (wid == 0) {
            const TS* col = S + (size_t)(r1 + lane) * ld + r1;    // column lane of U_ss
            double u[32];
#pragma unroll
            for (int k = 0; k < 32; ++k) u[k] = (double)col[k];
            double y = z[r1 + lane];
#pragma unroll
            for (int i = 0; i < 32; ++i) {
                if (lane == i) y = y / u[i];
                const double yi = __shfl_sync(0xffffffffu, y, i);
                if (lane > i) y -= u[i] * yi;
            }
            z[r1 + lane] = y;
        }
        __syncthreads();
    }
    // z = T_0^T ... T_last^T z
    for (int s = nb - 1; s >= 0; --s) {
        const int r1 = 32 * s, below = r1 + 32;
        for (int j = wid; j < 32; j += nw) {
            const TS* col = S + (size_t)(r1 + j) * ld;
            double acc = 0.0;
            for (int i = below + lane; i < ld; i += 32) acc += (double)col[i] * z[i];
            for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
            if (lane == 0) z[r1 + j] -= acc;
        }
        __syncthreads();
        if (wid == 0) {
            const TS* col = S + (size_t)(r1 + lane) * ld + r1;    // column lane of L_ss (below its diagonal)
            double l[32];
#pragma unroll
            for (int k = 0; k < 32; ++k) l[k] = k > lane ? (double)col[k] : 0.0;
            double y = z[r1 + lane];
#pragma unroll
            for (int i = 31; i >= 0; --i) {
                const double yi = __shfl_sync(0xffffffffu, y, i);
                if (lane < i) y -= l[i] * yi;
            }
            z[r1 + lane] = y;
        }
        __syncthreads();
        if (s % BPP == 0) {
            // inverse of the panel's row exchange (new row rows[i] = old row rows[cont[i]])
            const int32_t* pl = perms + ((size_t)(s / BPP) * nK + K) * LU_PW;
            const int nr = pl[0];
            const int32_t* rows = pl + 1;
            const int32_t* cont = rows + 2 * LU_NB;
            for (int i = tid; i < nr; i += blockDim.x) tmp[i] = z[rows[i]];
            __syncthreads();
            for (int i = tid; i < nr; i += blockDim.x) z[rows[cont[i]]] = tmp[i];
            __syncthreads();
        }
    }
    for (int i = tid; i < ld; i += blockDim.x) xall[(size_t)K * ld + i] = z[i];
}

template <class TS>
cudaError_t solve_T_t(const LUPlan& P, const int32_t* perms, const double* r, double* x, const int32_t* skip,
                      cudaStream_t st) {
    const size_t sm = sizeof(double) * ((size_t)P.ld + 2 * LU_NB);
    cudaFuncSetAttribute(solve_T_kernel<TS>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    solve_T_kernel<TS><<<(unsigned)P.nK, 512, sm, st>>>((const TS*)P.S, P.ld, perms, P.nK, r, x, skip);
    MEHDG_COUNT(1);
    return cudaGetLastError();
}
}  // namespace

cudaError_t lu_solve_T(const LUPlan& P, const double* r, double* x, const int32_t* skip, cudaStream_t st) {
    const int32_t* perms = panel_perm(P, 0);
    if (P.fp64) return solve_T_t<double>(P, perms, r, x, skip, st);
    return solve_T_t<float>(P, perms, r, x, skip, st);
}

cudaError_t lu_solve(const LUPlan& P, const double* r, double* x, const int32_t* skip, cudaStream_t st) {
    const int32_t* perms = panel_perm(P, 0);
    if (P.fp64) return solve_t<double>(P, perms, r, x, skip, st);
    return solve_t<float>(P, perms, r, x, skip, st);
}
