// Additive Schwarz preconditioner (2D): patch geometry, the per-context plan
// (local maps, scalings and inverse factors of every active patch) and the
// device helpers shared by the single-system and the batched solvers.
#pragma once
#include <cstdint>
#include "internal.cuh"
#include "ctx.cuh"

namespace stk {

constexpr int PB = 4;               // patch core (slots per side)
constexpr int PR = PB + 2;          // with the one-slot ring
constexpr int PMAX = 3 * PR * PR;   // unknowns per patch at most (2D: 108)
// Packed lower triangle with every row padded to a multiple of 4 entries, so
// rows start on 16-byte boundaries: row r (group m = r / 4, rows of group m
// hold 4(m+1) entries) starts at 8 m (m+1) + (r - 4m) 4 (m+1).
__host__ __device__ constexpr int tri4_off(int r) { return 8 * (r / 4) * (r / 4 + 1) + (r - 4 * (r / 4)) * 4 * (r / 4 + 1); }
constexpr int PFAC = tri4_off(PMAX);                          // 6048 floats per patch

struct SchwarzPlan {
    int npx, npy;                   // patch grid over slots [0, nx] x [0, ny]
    int* pid;                       // [npy * npx] compact patch id or -1
    int* corner;                    // [np] packed (I, J)
    int* nloc;                      // [np] active unknowns per patch
    short* lmap;                    // [np * PMAX] local index of (f, jj, ii) or -1
    float* inv;                     // [np * PFAC] X = L^-1 of each scaled patch matrix, packed rows
                                    // padded to 16 bytes
    float* scale;                   // [np * PMAX] D^-1/2 of each patch, by position (f, jj, ii)
    float* ybuf;                    // [npy * npx * PMAX] local results by grid patch and position
                                    // (f, jj, ii); zero for inactive patches and positions
    int np;
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
// try_wait itself blocks for a while); the copy of 23 KB takes microseconds.
constexpr long long SW_WAIT_POLLS = 1LL << 22;

// Wait for phase `parity` of an mbarrier, at most SW_WAIT_POLLS polls.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
    for (long long i = 0; i < SW_WAIT_POLLS; ++i) {
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
// completing on mbarrier `bar` (one thread).
__device__ __forceinline__ void sw_issue(uint32_t bar, void* dst, const void* src, uint32_t bytes) {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
    if (bytes > 0)
        asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                         smem_u32(dst)),
                     "l"(src), "r"(bytes), "r"(bar)
                     : "memory");
}

}  // namespace stk
