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
// triangle of X~ with every row padded to a multiple of 8 entries, so rows
// start on 16-byte boundaries: row r (group m = r / 8, rows of group m hold
// 8(m+1) entries) starts at 32 m (m+1) + (r - 8m) 8 (m+1) halves.
__host__ __device__ constexpr int tri8_off(int r) { return 32 * (r / 8) * (r / 8 + 1) + (r - 8 * (r / 8)) * 8 * (r / 8 + 1); }
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

// s <- X~^T diag(rho^2) X~ s for the stored factor F of an n-unknown patch in
// shared memory (at least 128 threads).  y = X~ s: thread t takes row t, 16-byte loads
// of eight FP16 entries; y_t *= rho_t^2; z = X~^T y: eight threads per block
// of eight columns, each taking every eighth row, joined by shuffles.  s
// holds PMAX8 floats, zero from n up to the next multiple of 8; y holds PMAX
// floats of scratch.  Ends after a barrier with z in s[0, n).
__device__ __forceinline__ void sw_factor_products(const uint8_t* F, int n, float* s, float* y) {
    const int t = threadIdx.x;
    const float* rs = reinterpret_cast<const float*>(F);
    const __half* X = reinterpret_cast<const __half*>(F + SW_RS_BYTES);
    if (t < n) {
        const uint4* xr = reinterpret_cast<const uint4*>(X + tri8_off(t));
        const float4* s4 = reinterpret_cast<const float4*>(s);
        float acc = 0.f;
        for (int j = 0; j <= t / 8; ++j) {
            const uint4 a = xr[j];
            const float4 b0 = s4[2 * j], b1 = s4[2 * j + 1];
            float2 f = __half22float2(*reinterpret_cast<const __half2*>(&a.x));
            acc = fmaf(f.x, b0.x, acc);
            acc = fmaf(f.y, b0.y, acc);
            f = __half22float2(*reinterpret_cast<const __half2*>(&a.y));
            acc = fmaf(f.x, b0.z, acc);
            acc = fmaf(f.y, b0.w, acc);
            f = __half22float2(*reinterpret_cast<const __half2*>(&a.z));
            acc = fmaf(f.x, b1.x, acc);
            acc = fmaf(f.y, b1.y, acc);
            f = __half22float2(*reinterpret_cast<const __half2*>(&a.w));
            acc = fmaf(f.x, b1.z, acc);
            acc = fmaf(f.y, b1.w, acc);
        }
        y[t] = acc * rs[t];
    }
    __syncthreads();
    const int cb = t >> 3, q = t & 7;
    float z[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) z[k] = 0.f;
    if (8 * cb < n)
        for (int row = 8 * cb + q; row < n; row += 8) {
            const uint4 a = *reinterpret_cast<const uint4*>(X + tri8_off(row) + 8 * cb);
            const float yr = y[row];
            const uint32_t w[4] = {a.x, a.y, a.z, a.w};
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const float2 f = __half22float2(*reinterpret_cast<const __half2*>(&w[k]));
                z[2 * k] = fmaf(f.x, yr, z[2 * k]);
                z[2 * k + 1] = fmaf(f.y, yr, z[2 * k + 1]);
            }
        }
#pragma unroll
    for (int o = 1; o <= 4; o <<= 1)
#pragma unroll
        for (int k = 0; k < 8; ++k) z[k] += __shfl_xor_sync(0xffffffffu, z[k], o);
    // s is no longer read (y = X~ s ended at the barrier above)
    if (q == 0 && 8 * cb < n) {
        reinterpret_cast<float4*>(s)[2 * cb] = make_float4(z[0], z[1], z[2], z[3]);
        reinterpret_cast<float4*>(s)[2 * cb + 1] = make_float4(z[4], z[5], z[6], z[7]);
    }
    __syncthreads();
}

}  // namespace stk
