// Additive Schwarz preconditioner (2D): patch geometry, the per-context plan
// (local maps, scalings and inverse factors of every active patch) and the
// device helpers shared by the single-system and the batched solvers.
#pragma once
#include <cstdint>
#include <cuda_fp16.h>
#include "internal.cuh"
#include "ctx.cuh"

namespace stk {

constexpr int PB = 4;               // patch core (slots per side)
constexpr int PR = PB + 2;          // with the one-slot ring
constexpr int PMAX = 3 * PR * PR;   // unknowns per patch at most (2D: 108)
constexpr int PMAX8 = (PMAX + 7) / 8 * 8;   // local vectors padded to blocks of 8
// Stored factor of one patch: X = L^-1 of the unit-diagonal patch matrix,
// each row r scaled by rho_r = max_c |X[r][c]|, kept as FP16 (X~ = X / rho_r
// in [-1, 1]) with rho_r^2 in FP32; the operator is X~^T diag(rho^2) X~.
// Layout: PMAX FP32 row factors rho_r^2 (432 bytes), then the packed lower
// triangle of X~ by bands of 8 rows: band m (rows 8m .. 8m+7, of which an
// n-row patch keeps k = min(8, n - 8m)) holds 8(m+1) columns, stored as
// m + 1 blocks of 8 columns, each block with the band's k rows one after
// another (16 bytes per row).  The 8 rows of an 8 x 8 block are then one
// contiguous 128-byte run, which ldmatrix reads without bank conflicts.
// Band m starts at 32 m (m+1) halves; tri8_off(r) is where row r would end
// the stored triangle (the first r rows take tri8_off(r) halves).
__host__ __device__ constexpr int tri8_off(int r) { return 32 * (r / 8) * (r / 8 + 1) + (r - 8 * (r / 8)) * 8 * (r / 8 + 1); }
// Offset (halves) of entry (r, c), c < 8 (r / 8 + 1), in an n-row patch.
__host__ __device__ constexpr int sw_fac_off(int r, int c, int n) {
    return 32 * (r / 8) * (r / 8 + 1) + (c / 8) * 8 * (n - 8 * (r / 8) < 8 ? n - 8 * (r / 8) : 8) + (r % 8) * 8 +
           c % 8;
}
constexpr int SW_RS_BYTES = PMAX * (int)sizeof(float);                       // 432
constexpr int SW_FAC_BYTES = SW_RS_BYTES + tri8_off(PMAX) * 2;               // 12,976 bytes per patch
// Bytes of a patch's stored factor with n unknowns (a multiple of 16).
__host__ __device__ constexpr uint32_t sw_patch_bytes(int n) { return (uint32_t)(SW_RS_BYTES + tri8_off(n) * 2); }

struct SchwarzPlan {
    int npx, npy;                   // patch grid over slots [0, nx] x [0, ny]
    int* pid;                       // [npy * npx] compact patch id or -1
    int* corner;                    // [np] packed (I, J)
    int* nloc;                      // [np] active unknowns per patch
    short* lmap;                    // [np * PMAX] local index of (f, jj, ii) or -1
    uint8_t* fac;                   // [np * SW_FAC_BYTES] stored factor of each patch (layout above)
    float* scale;                   // [np * PMAX] D^-1/2 of each patch, by position (f, jj, ii)
    float* ybuf;                    // [npy * npx * PMAX] local results by grid patch and position
                                    // (f, jj, ii); zero for inactive patches and positions
    int np;
    int evict_first;                // the factors (of this plan, or of a whole batch) exceed half of
                                    // L2: load them with an evict-first L2 policy
};

// Whether the unknown of field f (0 tau_xx at a cell, 1 tau_xy at a node,
// 2 p at a cell) at sample (i, j) exists and is active; act_cell / act_node
// are the activity masks in slot layout.
__device__ __forceinline__ bool unknown_active(const uint8_t* act_cell, const uint8_t* act_node, const Layout& L,
                                               int f, int i, int j) {
    if (i < 0 || j < 0 || i > L.nx || j > L.ny) return false;
    if (f != 1 && (i >= L.nx || j >= L.ny)) return false;
    return (f == 1 ? act_node : act_cell)[L.off(i + 1, j + 1, 0)] != 0;
}
__device__ __forceinline__ bool unknown_active(const DevArrays& D, const Layout& L, int f, int i, int j) {
    return unknown_active(D.act[0], D.act[1], L, f, i, j);
}

// Shared-memory address of a pointer (for mbarrier and bulk-copy operands).
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// Polls of the bulk copy's mbarrier before a local solve gives up (each
// try_wait itself blocks for a while); the copy of 13 KB takes microseconds.
constexpr long long SW_WAIT_POLLS = 1LL << 22;
// Polls of the test hook's wait (options.wait_test): a copy that is never
// issued, so the wait gives up after about a millisecond.
constexpr long long SW_TEST_POLLS = 1024;

// Wait for phase `parity` of an mbarrier, at most `polls` polls.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, long long polls = SW_WAIT_POLLS) {
    for (long long i = 0; i < polls; ++i) {
        uint32_t ok;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(ok)
            : "r"(bar), "r"(parity)
            : "memory");
        if (ok) return true;
    }
    return false;
}

// Start the bulk (TMA) copy of one packed factor into shared memory,
// completing on mbarrier `bar` (one thread).  The factors are read once per
// CG iteration; when they do not fit in L2 (evict_first) they are loaded
// with an evict-first L2 policy, so that the solver's vectors and
// coefficients stay in L2 instead of being evicted by the stream; when they
// fit, the default policy keeps them resident from one iteration to the next.
__device__ __forceinline__ void sw_issue(uint32_t bar, void* dst, const void* src, uint32_t bytes,
                                         bool evict_first) {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
    if (bytes == 0) return;
    if (evict_first) {
        uint64_t pol;
        asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
        asm volatile(
            "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1], %2, [%3], "
            "%4;" ::"r"(smem_u32(dst)),
            "l"(src), "r"(bytes), "r"(bar), "l"(pol)
            : "memory");
    } else {
        asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                         smem_u32(dst)),
                     "l"(src), "r"(bytes), "r"(bar)
                     : "memory");
    }
}

// Whether factor bytes exceed half of this device's L2 (host).
inline bool sw_factors_exceed_l2(size_t bytes) {
    int dev = 0, l2 = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, dev);
    return l2 > 0 && bytes > (size_t)l2 / 2;
}

// ---- the two triangular products on the tensor cores ---------------------
// mma.sync m16n8k16, FP16 operands, FP32 accumulation.  The FP32 vector is
// scaled by a power of two (largest magnitude into [2^13, 2^14)) and split
// into FP16 hi + lo parts, which fill columns 0 and 1 of the B operand:
// products of FP16 numbers are exact in FP32, so X~ (v_hi + v_lo) carries
// the vector to about 2^-22 of its largest entry, as the FP32 path did.
__device__ __forceinline__ void mma_f16_16816(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}
__device__ __forceinline__ void ldsm_x4(uint32_t (&a)[4], uint32_t addr) {
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];"
                 : "=r"(a[0]), "=r"(a[1]), "=r"(a[2]), "=r"(a[3])
                 : "r"(addr));
}
__device__ __forceinline__ void ldsm_x4_trans(uint32_t (&a)[4], uint32_t addr) {
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];"
                 : "=r"(a[0]), "=r"(a[1]), "=r"(a[2]), "=r"(a[3])
                 : "r"(addr));
}

// Power of two putting a largest magnitude m into [2^13, 2^14) (shift
// clamped to +-120): v * sc is split into FP16 hi + lo, results are scaled
// back by inv = 1 / sc.
__device__ __forceinline__ void sw_hl_scale(float m, float& sc, float& inv) {
    const int e = m > 0.f ? ((__float_as_int(m) >> 23) & 0xff) - 127 : 0;
    const int k = max(-120, min(120, 13 - e));
    sc = __int_as_float((127 + k) << 23);
    inv = __int_as_float((127 - k) << 23);
}

// Split of the vector v (n entries, scaled by sc) into FP16 hi + lo parts,
// one entry per thread (threads 0..111), into hb[0][.] and hb[1][.]; entries
// from n to 111 are zero.
__device__ __forceinline__ void sw_split(const float* v, int n, float sc, __half* hb) {
    const int t = threadIdx.x;
    if (t < 16 * 7) {
        const float x = t < n ? v[t] * sc : 0.f;
        const __half hi = __float2half_rn(x);
        hb[t] = hi;
        hb[16 * 7 + t] = __float2half_rn(x - __half2float(hi));
    }
}

// Shared scratch of sw_factor_products, in halves: the split vector (hi,
// lo), the row table (one 32-bit word per stored row) and the four warps'
// largest magnitudes (one word each).
constexpr int SW_HB_HALVES = 2 * 16 * 7 + 2 * 16 * 7 + 2 * 4;

// Largest |v[k]| over k < n (up to 128 entries), every thread of warps 0..3
// taking one entry: a warp reduction, the four warps' results through wm,
// one barrier (every thread of the CTA must call it).
__device__ __forceinline__ float sw_cta_absmax(const float* v, int n, unsigned* wm) {
    const int t = threadIdx.x, warp = t >> 5;
    if (warp < 4) {
        const unsigned m = __reduce_max_sync(0xffffffffu, t < n ? __float_as_uint(fabsf(v[t])) : 0u);
        if ((t & 31) == 0) wm[warp] = m;
    }
    __syncthreads();
    const uint4 a = *reinterpret_cast<const uint4*>(wm);
    return __uint_as_float(max(max(a.x, a.y), max(a.z, a.w)));
}

// y = X~ s for the row tiles MA and MB (MB < MA; MB < 0: none) of one warp:
// row tile m costs m + 1 tile products (k-tiles 0..m), the two chains
// interleaved.  hbw: the split vector as words (lane's B fragment of k-tile
// kt at hbw[lb + 8 kt] and hbw[lb + 8 kt + 4]); rowtab: the row table.
template <int MA, int MB>
__device__ __forceinline__ void sw_rows(uint32_t X, int ntile, int lane, const uint32_t* hbw, int lb,
                                        const uint32_t* rowtab, float (&dA)[4], float (&dB)[4]) {
    const int li = lane >> 3, lj = lane & 7;      // ldmatrix: matrix li, its row lj
    const bool onA = MA < ntile, onB = MB >= 0 && MB < ntile;
    const uint32_t eA = rowtab[16 * MA + (li & 1) * 8 + lj], sA = eA >> 16;
    const uint32_t aA = X + (eA & 0xffffu) + (uint32_t)(li >> 1) * (sA >> 1);
    uint32_t aB = 0, sB = 0;
    if (MB >= 0) {
        const uint32_t eB = rowtab[16 * (MB < 0 ? 0 : MB) + (li & 1) * 8 + lj];
        sB = eB >> 16;
        aB = X + (eB & 0xffffu) + (uint32_t)(li >> 1) * (sB >> 1);
    }
#pragma unroll
    for (int kt = 0; kt <= MA; ++kt) {
        if (kt >= ntile) break;                          // no chain reaches this k-tile
        const uint32_t b0 = hbw[lb + 8 * kt], b1 = hbw[lb + 8 * kt + 4];
        uint32_t a[4];
        if (onA) {
            ldsm_x4(a, aA + sA * kt);
            if (kt == MA) a[2] = 0u;                     // upper 8 x 8 block of the diagonal tile
            mma_f16_16816(dA, a, b0, b1);
        }
        if (kt <= MB && onB) {
            ldsm_x4(a, aB + sB * kt);
            if (kt == MB) a[2] = 0u;
            mma_f16_16816(dB, a, b0, b1);
        }
    }
}

// z = X~^T v for the column tiles CA and CB (CA < CB; CB > 6: none) of one
// warp: column tile c costs 7 - c tile products (row tiles c..6, the
// transposed tiles by ldmatrix.trans), the two chains interleaved.
template <int CA, int CB>
__device__ __forceinline__ void sw_cols(uint32_t X, int ntile, int lane, const uint32_t* hbw, int lb,
                                        const uint32_t* rowtab, float (&dA)[4], float (&dB)[4]) {
    const int li = lane >> 3, lj = lane & 7;
#pragma unroll
    for (int rt = CA; rt < 7; ++rt) {
        if (rt >= ntile) break;
        const uint32_t e = rowtab[16 * rt + (li >> 1) * 8 + lj], st = e >> 16;
        const uint32_t addr = X + (e & 0xffffu) + (uint32_t)(li & 1) * (st >> 1);
        const uint32_t b0 = hbw[lb + 8 * rt], b1 = hbw[lb + 8 * rt + 4];
        uint32_t a[4];
        ldsm_x4_trans(a, addr + st * CA);
        if (rt == CA) a[1] = 0u;                         // upper 8 x 8 block of the diagonal tile
        mma_f16_16816(dA, a, b0, b1);
        if (CB <= 6 && rt >= CB) {
            ldsm_x4_trans(a, addr + st * (CB <= 6 ? CB : 0));
            if (rt == CB) a[1] = 0u;
            mma_f16_16816(dB, a, b0, b1);
        }
    }
}

// s <- X~^T diag(rho^2) X~ s for the stored factor F of an n-unknown patch in
// shared memory, by warps 0-3 of the CTA (every thread of the CTA must call
// it, with at least 112 threads).  X~ is cut into 16 x 16 tiles (rows and
// columns up to 112); tiles wholly above the diagonal are skipped and the
// upper 8 x 8 block of each diagonal tile (not stored: rows of the first
// half hold 8 columns fewer) is zeroed in the fragment.  y = X~ s: output
// tile m costs m + 1 tile products, so warps 0..3 take tiles {6}, {5, 0},
// {4, 1}, {3, 2} (7 each, the two chains of a warp interleaved); z = X~^T
// (rho^2 y): output tile c costs 7 - c, so {0}, {1, 6}, {2, 5}, {3, 4}.
// Each warp runs its own tile lists unrolled at compile time (one code path
// per warp) and takes its tile addresses from a row table built once per
// patch (byte offset of the row's first column block and the step to the
// next 16 columns; rows at or past n point at row 0, whose data is finite:
// their outputs are dropped in the first product and meet zero vector
// entries in the second), so a tile costs its ldmatrix, its mma and one
// address add.  Each vector is split into FP16 hi + lo once, one entry per
// thread.  hb: SW_HB_HALVES halves of shared memory (16-byte aligned); s
// holds PMAX8 floats (entries from n on are not read); y holds PMAX8 floats
// of scratch and may be s itself (s is not read once split).  Ends after a
// barrier with z in s[0, n) (entries from n to the last tile's end hold
// finite values that callers do not read).
__device__ __forceinline__ void sw_factor_products(const uint8_t* F, int n, float* s, float* y, __half* hb) {
    const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
    const float* rs = reinterpret_cast<const float*>(F);
    const uint32_t X = smem_u32(F + SW_RS_BYTES);
    uint32_t* rowtab = reinterpret_cast<uint32_t*>(hb + 2 * 16 * 7);
    unsigned* wm = reinterpret_cast<unsigned*>(hb + 4 * 16 * 7);
    const uint32_t* hbw = reinterpret_cast<const uint32_t*>(hb);
    const int g = lane >> 2, tq = lane & 3;
    // word of the lane's B fragment: columns 0 (hi) and 1 (lo) are the split
    // vector; columns 2..7 repeat them, and their outputs are not read
    const int lb = 56 * (g & 1) + tq;
    const int ntile = (n + 15) >> 4;
    if (t < 16 * 7) {
        const int row = t < n ? t : 0;
        const uint32_t R = (uint32_t)row >> 3, w = (uint32_t)min(8, n - 8 * (int)R);
        rowtab[t] = (2u * (32u * R * (R + 1u) + (uint32_t)(row & 7) * 8u)) | ((32u * w) << 16);
    }
    float sc, inv;
    sw_hl_scale(sw_cta_absmax(s, n, wm), sc, inv);
    sw_split(s, n, sc, hb);
    __syncthreads();
    if (warp < 4) {
        float dA[4] = {0.f, 0.f, 0.f, 0.f}, dB[4] = {0.f, 0.f, 0.f, 0.f};
        switch (warp) {
            case 0: sw_rows<6, -1>(X, ntile, lane, hbw, lb, rowtab, dA, dB); break;
            case 1: sw_rows<5, 0>(X, ntile, lane, hbw, lb, rowtab, dA, dB); break;
            case 2: sw_rows<4, 1>(X, ntile, lane, hbw, lb, rowtab, dA, dB); break;
            default: sw_rows<3, 2>(X, ntile, lane, hbw, lb, rowtab, dA, dB); break;
        }
        if (tq == 0) {
            const int mA = 6 - warp, mB = warp - 1;
            // rows from n to the tile's end get finite values that are not read
            if (mA < ntile) {
                const int r0 = 16 * mA + g, r1 = r0 + 8;
                y[r0] = (dA[0] + dA[1]) * inv * rs[r0];
                y[r1] = (dA[2] + dA[3]) * inv * rs[r1];
            }
            if (mB >= 0 && mB < ntile) {
                const int r0 = 16 * mB + g, r1 = r0 + 8;
                y[r0] = (dB[0] + dB[1]) * inv * rs[r0];
                y[r1] = (dB[2] + dB[3]) * inv * rs[r1];
            }
        }
    }
    __syncthreads();
    sw_hl_scale(sw_cta_absmax(y, n, wm), sc, inv);
    sw_split(y, n, sc, hb);          // hb of the first product is no longer read
    __syncthreads();
    if (warp < 4) {
        float dA[4] = {0.f, 0.f, 0.f, 0.f}, dB[4] = {0.f, 0.f, 0.f, 0.f};
        switch (warp) {
            case 0: sw_cols<0, 7>(X, ntile, lane, hbw, lb, rowtab, dA, dB); break;
            case 1: sw_cols<1, 6>(X, ntile, lane, hbw, lb, rowtab, dA, dB); break;
            case 2: sw_cols<2, 5>(X, ntile, lane, hbw, lb, rowtab, dA, dB); break;
            default: sw_cols<3, 4>(X, ntile, lane, hbw, lb, rowtab, dA, dB); break;
        }
        if (tq == 0) {
            // s is no longer read (it was split into hb before the first barrier)
            const int cA = warp, cB = 7 - warp;
            if (cA < ntile) {
                const int c0 = 16 * cA + g, c1 = c0 + 8;
                s[c0] = (dA[0] + dA[1]) * inv;
                s[c1] = (dA[2] + dA[3]) * inv;
            }
            if (cB <= 6 && cB < ntile) {
                const int c0 = 16 * cB + g, c1 = c0 + 8;
                s[c0] = (dB[0] + dB[1]) * inv;
                s[c1] = (dB[2] + dB[3]) * inv;
            }
        }
    }
    __syncthreads();
}

}  // namespace stk
