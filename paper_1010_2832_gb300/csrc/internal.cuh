// Internal types shared by the libstokes translation units.
#pragma once
#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>
#include <string>
#include "../../include/stokes.h"

namespace stk {

// Padded storage of one field.  Padded coordinates (c, r, q): sample
// (i, j, k) sits at (i + 1, j + 1, k + 1) (2D: q = 0).  Pad columns, rows and
// planes hold zeros; a guard of zeros before and after the data keeps every
// +-1 halo access of a tile in bounds.
struct Layout {
    int dim, nx, ny, nz;
    int P, R, Q;          // pitch, rows, planes (Q = 1 in 2D)
    int64_t guard;        // zeros before the data
    int64_t stride;       // elements per field, guards included
    int ntx, nty, ntz;    // tiles per axis over the padded domain
    __host__ __device__ int64_t off(int c, int r, int q) const {
        return guard + ((int64_t)q * R + r) * P + c;
    }
};

// Tile shape over padded coordinates.
constexpr int TX = 32;
constexpr int TY2 = 8;                 // 2D: 32 x 8 slots, one per thread
constexpr int TY3 = 4, TZ3 = 4;        // 3D: 32 x 4 x 4 slots, 2 per thread
// 3D apply unit: 32 x 8 slots streamed over zt tile layers of 4 planes
// (2 x zt tiles of the tile grid, zt = 1..4), bit dy + 2 dz of its mask for
// tile (.., 2 uy + dy, zt uz + dz)
constexpr int UY3 = 2 * TY3, ZT_MAX = 4;
__host__ __device__ inline int units_y(int nty) { return (nty + 1) / 2; }
__host__ __device__ inline int units_z(int ntz, int zt) { return (ntz + zt - 1) / zt; }

// Face flags (one byte per face).
enum : uint8_t { F_LIVE = 1, F_BAD = 2, F_INVALID = 4, F_WALL = 8, F_EXISTS = 16 };

// Coefficients of the matrix-free operator in one precision (slot layout).
// 2D fields: a_c, a_n, d_c, d_n, K_u, K_v.
// 3D fields: a_c, a_xy, a_xz, a_yz, d_c, d_xy, d_xz, d_yz, K_u, K_v, K_w.
// a = W_L / h on active unknowns (0 otherwise); d = W_L W_F / mu on active
// stress unknowns, 1 on inactive ones; K = dt W_F / (rho W_L) on live faces.
// 2D BF16 coefficients are also stored in pairs, one 32-bit word per slot
// (first coefficient in the low half): (a_c, a_n), (d_c, d_n), (K_u, K_v),
// so that one 16-byte load brings two coefficients of four slots; 3D BF16
// coefficients also in fours, 8 bytes per slot (first in the low half of
// .x): (a_c, a_xy, a_xz, a_yz) and (d_c, d_xy, d_xz, d_yz), so that a slot's
// row weights or diagonal are one load (nullptr where not stored).
template <class C> struct Coef {
    const C* f[11];
    const uint32_t* pr[3];
    const uint2* qd[2];
};

// Device-resident scalars of one CG solve.
struct CgScalars {
    double rz, pq, rr, rr0, alpha, beta;
    double tol2;            // (tol_rel)^2 * rr0 for the recurrence test
    double scale;           // inner right-hand side = scale * outer residual
    double tol_rel;         // relative recurrence tolerance of this solve
    int iter, done, status, max_iter;
    int wait_test;          // test hook: the local solves wait for a copy never issued
};

enum { MODE_PLAIN = 0, MODE_RESID = 1, MODE_CG = 2 };

struct ApplyArgs {
    const void* b;       // RESID: right-hand side (same type as x)
    const void* pold;    // CG: previous direction
    void* pnew;          // CG: new direction (output)
    double* partial;
    unsigned* counter;
    CgScalars* sc;
    // 3D: the units to apply (nullptr: every unit of the grid, every tile
    // in the grid active, ZT_MAX layers deep), their tile masks and depth
    const int* units;
    const uint8_t* umask;
    int nunits;
    int zt;
};

struct Ctx;   // defined in api.cu

// ---- host helpers implemented across translation units --------------------
void set_error(Ctx* c, const std::string& m);

// weights.cu
cudaError_t launch_build_weights(Ctx* c, const double* phiL, const double* phiS, const double* const* rho,
                                 const double* const* mu, const double* const* ubc);
// rhs_recover.cu
cudaError_t launch_rhs(Ctx* c, const double* const* ustar, double* b);
cudaError_t launch_recover(Ctx* c, const double* const* ustar, const double* x, double* const* uout);
cudaError_t launch_slots_fields(Ctx* c, const double* src, double* dst, int to_fields);
// pcg.cu
stokes_status solve_system(Ctx* c, const double* b, double* x, const stokes_options* o, stokes_stats* st);

// Field-layout index of sample (i, j[, k]) of a kind (x fastest).
// Kinds 2D: 0 cell, 1 node, 2 u, 3 v.  3D: 0 cell, 1 u, 2 v, 3 w, 4 exy, 5 exz, 6 eyz.
__host__ __device__ __forceinline__ int64_t fidx2(int kind, int i, int j, int nx, int ny) {
    int w = (kind == 1 || kind == 2) ? nx + 1 : nx;
    (void)ny;
    return (int64_t)j * w + i;
}
__host__ __device__ __forceinline__ int64_t fidx3(int kind, int i, int j, int k, int nx, int ny, int nz) {
    int wx = (kind == 1 || kind == 4 || kind == 5) ? nx + 1 : nx;
    int wy = (kind == 2 || kind == 4 || kind == 6) ? ny + 1 : ny;
    (void)nz;
    return ((int64_t)k * wy + j) * wx + i;
}

// reduction helpers --------------------------------------------------------
__device__ __forceinline__ double warp_sum(double v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Error-free float addition (Knuth TwoSum): s + e == a + b exactly.
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
    s = a + b;
    float bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}

// Warp sum of float-float values (hi, lo), returned as a double.  Used to
// keep FP32 dot products accurate to ~2^-44 relative without FP64 adds.
__device__ __forceinline__ double warp_sum_ff(float hi, float lo) {
    for (int o = 16; o > 0; o >>= 1) {
        float oh = __shfl_xor_sync(0xffffffffu, hi, o);
        float ol = __shfl_xor_sync(0xffffffffu, lo, o);
        float s, e;
        two_sum(hi, oh, s, e);
        e += lo + ol;
        hi = s + e;
        lo = e - (hi - s);
    }
    return (double)hi + (double)lo;
}

}  // namespace stk
