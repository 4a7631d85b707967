// Additive Schwarz preconditioner (2D) for the SPD pressure-stress system.
//
// The paper solved its systems with CG and an overlapping Schwarz domain
// decomposition (Section 9); this is a GPU form of that idea with many small
// overlapping patches and exact local solves:
//
//   M^-1 r = sum_p R_p^T A_p^-1 R_p r,
//
// where patch p covers the slots of a 4x4 core plus a one-slot ring
// (6x6 slots, up to 108 unknowns), R_p restricts to its active unknowns and
// A_p = R_p A R_p^T.  Setup (once per weight build), one CTA per patch:
//   1. index the patch's active unknowns (fixed order: field, row, column);
//   2. assemble A_p from the operator coefficients, C on the stress diagonal
//      plus K_f beta_f beta_f^T for every face touching the patch, faces in a
//      fixed order (the local matrices are reproducible bit for bit);
//   3. scale to unit diagonal, Cholesky, solve for the inverse column by
//      column, scale back, store in BF16.
// Apply (every CG step): one CTA per patch computes y_p = A_p^-1 r_p (FP32
// accumulation); a gather kernel sums, for every unknown, the contributions
// of the (at most four) patches covering it in a fixed order, so the
// preconditioner is symmetric and deterministic.  Inactive unknowns get z = r.
#include <cmath>
#include <vector>
#include "internal.cuh"
#include "ctx.cuh"

namespace stk {

constexpr int PB = 4;               // patch core (slots per side)
constexpr int PR = PB + 2;          // with the one-slot ring
constexpr int PMAX = 3 * PR * PR;   // unknowns per patch at most (2D: 108)

struct SchwarzPlan {
    int npx, npy;                   // patch grid over slots [0, nx] x [0, ny]
    int* pid;                       // [npy * npx] compact patch id or -1
    int* corner;                    // [np] packed (I, J)
    int* nloc;                      // [np] active unknowns per patch
    short* lmap;                    // [np * PMAX] local index of (f, jj, ii) or -1
    __nv_bfloat16* inv;             // [np * PMAX * PMAX] local inverses
    float* ybuf;                    // [np * PMAX]
    int np;
};

// slot (i, j) of a patch position; f = field (0 txx cell, 1 txy node, 2 p cell)
__device__ __forceinline__ bool unknown_active(const DevArrays& D, const Layout& L, int f, int i, int j) {
    if (i < 0 || j < 0 || i > L.nx || j > L.ny) return false;
    if (f != 1 && (i >= L.nx || j >= L.ny)) return false;
    return D.act[f == 1 ? 1 : 0][L.off(i + 1, j + 1, 0)] != 0;
}

__global__ void k_schwarz_mark(Layout L, DevArrays D, int npx, int npy, int* flag) {
    int I = blockIdx.x * blockDim.x + threadIdx.x, J = blockIdx.y;
    if (I >= npx || J >= npy) return;
    int any = 0;
    for (int f = 0; f < 3; ++f)
        for (int jj = 0; jj < PB; ++jj)
            for (int ii = 0; ii < PB; ++ii) any |= unknown_active(D, L, f, PB * I + ii, PB * J + jj);
    flag[J * npx + I] = any;
}

// one CTA (256 threads) per active patch; dynamic smem: A (PMAX^2 floats),
// X (PMAX^2 floats), diag scale, map
__global__ void __launch_bounds__(256) k_schwarz_setup(Layout L, DevArrays D, const float* coef, SchwarzPlan P) {
    extern __shared__ __align__(16) float sm[];
    float* A = sm;                       // n x n (row-major, stride PMAX)
    float* X = A + PMAX * PMAX;          // inverse columns
    float* sc = X + PMAX * PMAX;         // 1/sqrt(diag)
    __shared__ short map[PMAX];
    __shared__ int n_s;
    const int p = blockIdx.x;
    const int I = P.corner[p] & 0xffff, J = P.corner[p] >> 16;
    const int a0 = PB * I - 1, b0 = PB * J - 1;       // ring origin (slot coords)
    const int t = threadIdx.x;
    const int64_t S = L.stride;
    const float *a_c = coef, *a_n = coef + S, *d_c = coef + 2 * S, *d_n = coef + 3 * S, *K_u = coef + 4 * S,
                *K_v = coef + 5 * S;
    // 1. local indices in fixed order (thread 0: 108 positions)
    if (t == 0) {
        int n = 0;
        for (int f = 0; f < 3; ++f)
            for (int jj = 0; jj < PR; ++jj)
                for (int ii = 0; ii < PR; ++ii) {
                    int pos = (f * PR + jj) * PR + ii;
                    map[pos] = unknown_active(D, L, f, a0 + ii, b0 + jj) ? (short)n++ : (short)-1;
                }
        n_s = n;
        P.nloc[p] = n;
    }
    __syncthreads();
    const int n = n_s;
    for (int e = t; e < PMAX; e += 256) P.lmap[(int64_t)p * PMAX + e] = map[e];
    for (int e = t; e < n * PMAX; e += 256) A[e] = 0.f;
    __syncthreads();
    auto lidx = [&](int f, int i, int j) -> int {
        int ii = i - a0, jj = j - b0;
        if (ii < 0 || jj < 0 || ii >= PR || jj >= PR) return -1;
        return map[(f * PR + jj) * PR + ii];
    };
    // 2. stress diagonal C
    for (int e = t; e < 2 * PR * PR; e += 256) {
        int f = e / (PR * PR), rem = e % (PR * PR), jj = rem / PR, ii = rem % PR;
        int k = map[(f * PR + jj) * PR + ii];
        if (k >= 0) {
            int64_t o = L.off(a0 + ii + 1, b0 + jj + 1, 0);
            A[k * PMAX + k] += (f == 0 ? d_c : d_n)[o];
        }
    }
    __syncthreads();
    // faces touching the patch, one warp, faces in a fixed order; lanes own
    // distinct (row, column) pairs of one face's 6x6 outer product
    if (t < 32) {
        for (int dir = 0; dir < 2; ++dir) {
            // u faces i in [a0+1, a0+PR], j in [b0-1, b0+PR-1]; v faces transposed
            for (int jj = -1; jj <= PR; ++jj)
                for (int ii = -1; ii <= PR; ++ii) {
                    int i = a0 + ii, j = b0 + jj;
                    int ku_ok = dir == 0 ? (i >= 0 && i <= L.nx && j >= 0 && j < L.ny)
                                         : (i >= 0 && i < L.nx && j >= 0 && j <= L.ny);
                    if (!ku_ok) continue;
                    int64_t o = L.off(i + 1, j + 1, 0);
                    float K = (dir == 0 ? K_u : K_v)[o];
                    if (K == 0.f) continue;
                    int idx[6];
                    float b[6];
                    if (dir == 0) {
                        float am = a_c[L.off(i, j + 1, 0)], ap = a_c[o];
                        idx[0] = lidx(0, i - 1, j); b[0] = am;       // txx(i-1): +a
                        idx[1] = lidx(2, i - 1, j); b[1] = -am;      // p(i-1):   -a
                        idx[2] = lidx(0, i, j);     b[2] = -ap;      // txx(i):   -a
                        idx[3] = lidx(2, i, j);     b[3] = ap;       // p(i):     +a
                        idx[4] = lidx(1, i, j);     b[4] = a_n[o];                     // txy(i, j)
                        idx[5] = lidx(1, i, j + 1); b[5] = -a_n[L.off(i + 1, j + 2, 0)];  // txy(i, j+1)
                    } else {
                        float am = a_c[L.off(i + 1, j, 0)], ap = a_c[o];
                        idx[0] = lidx(0, i, j - 1); b[0] = -am;      // txx(j-1): -a
                        idx[1] = lidx(2, i, j - 1); b[1] = -am;      // p(j-1):   -a
                        idx[2] = lidx(0, i, j);     b[2] = ap;       // txx(j):   +a
                        idx[3] = lidx(2, i, j);     b[3] = ap;       // p(j):     +a
                        idx[4] = lidx(1, i, j);     b[4] = a_n[o];                     // txy(i, j)
                        idx[5] = lidx(1, i + 1, j); b[5] = -a_n[L.off(i + 2, j + 1, 0)];  // txy(i+1, j)
                    }
                    for (int q = t; q < 36; q += 32) {
                        int r = q / 6, c = q % 6;
                        if (idx[r] >= 0 && idx[c] >= 0) A[idx[r] * PMAX + idx[c]] += K * b[r] * b[c];
                    }
                    __syncwarp();
                }
        }
    }
    __syncthreads();
    // 3. unit-diagonal scaling, Cholesky (lower, in place), inverse
    for (int k = t; k < n; k += 256) sc[k] = A[k * PMAX + k] > 0.f ? rsqrtf(A[k * PMAX + k]) : 1.f;
    __syncthreads();
    for (int e = t; e < n * n; e += 256) {
        int r = e / n, c = e % n;
        A[r * PMAX + c] *= sc[r] * sc[c];
    }
    __syncthreads();
    for (int k = 0; k < n; ++k) {
        if (t == 0) {
            float d = A[k * PMAX + k];
            A[k * PMAX + k] = d > 1e-12f ? sqrtf(d) : 1.f;    // a vanishing pivot is replaced (robust, still SPD)
        }
        __syncthreads();
        float piv = A[k * PMAX + k];
        for (int r = k + 1 + t; r < n; r += 256) A[r * PMAX + k] /= piv;
        __syncthreads();
        int m = n - k - 1;
        for (int e = t; e < m * m; e += 256) {
            int r = k + 1 + e / m, c = k + 1 + e % m;
            if (c <= r) A[r * PMAX + c] -= A[r * PMAX + k] * A[c * PMAX + k];
        }
        __syncthreads();
    }
    // column c of the inverse: L y = e_c, L^T x = y (thread c, column in X)
    for (int c = t; c < n; c += 256) {
        for (int r = 0; r < n; ++r) X[r * PMAX + c] = 0.f;
        for (int r = c; r < n; ++r) {
            float s = r == c ? 1.f : 0.f;
            for (int q = c; q < r; ++q) s -= A[r * PMAX + q] * X[q * PMAX + c];
            X[r * PMAX + c] = s / A[r * PMAX + r];
        }
        for (int r = n - 1; r >= 0; --r) {
            float s = X[r * PMAX + c];
            for (int q = r + 1; q < n; ++q) s -= A[q * PMAX + r] * X[q * PMAX + c];
            X[r * PMAX + c] = s / A[r * PMAX + r];
        }
    }
    __syncthreads();
    __nv_bfloat16* out = P.inv + (int64_t)p * PMAX * PMAX;
    for (int e = t; e < n * n; e += 256) {
        int r = e / n, c = e % n;
        out[e] = __float2bfloat16(X[r * PMAX + c] * sc[r] * sc[c]);
    }
}

// y_p = A_p^-1 r_p, one CTA (128 threads) per patch; a warp per row
__global__ void __launch_bounds__(128) k_schwarz_gemv(Layout L, SchwarzPlan P, const float* __restrict__ r,
                                                      const CgScalars* sc) {
    __shared__ float rp[PMAX];
    if (sc->done) return;
    const int p = blockIdx.x;
    const int n = P.nloc[p];
    const int I = P.corner[p] & 0xffff, J = P.corner[p] >> 16;
    const int a0 = PB * I - 1, b0 = PB * J - 1;
    const short* map = P.lmap + (int64_t)p * PMAX;
    for (int e = threadIdx.x; e < PMAX; e += 128) {
        int k = map[e];
        if (k >= 0) {
            int f = e / (PR * PR), rem = e % (PR * PR), jj = rem / PR, ii = rem % PR;
            rp[k] = r[(int64_t)f * L.stride + L.off(a0 + ii + 1, b0 + jj + 1, 0)];
        }
    }
    __syncthreads();
    const __nv_bfloat16* M = P.inv + (int64_t)p * PMAX * PMAX;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int row = w; row < n; row += 4) {
        float s = 0.f;
        for (int c = lane; c < n; c += 32) s = fmaf(__bfloat162float(M[row * n + c]), rp[c], s);
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0) P.ybuf[(int64_t)p * PMAX + row] = s;
    }
}

// z = sum over covering patches (fixed order) for active unknowns, z = r on
// inactive ones.  Returns this thread's (r.z, r.r) over the slot's fields.
__device__ __forceinline__ void schwarz_gather_slot(const Layout& L, const DevArrays& D, const SchwarzPlan& P,
                                                    const float* __restrict__ r, float* __restrict__ z, int c,
                                                    int rr, double& rz, double& r2) {
    const int i = c - 1, j = rr - 1;
    const int64_t o = L.off(c, rr, 0);
    for (int f = 0; f < 3; ++f) {
        const int64_t of = (int64_t)f * L.stride + o;
        const float rv = r[of];
        float zv;
        if (!unknown_active(D, L, f, i, j)) {
            zv = (i >= 0 && j >= 0 && i <= L.nx && j <= L.ny) ? rv : 0.f;
        } else {
            float s = 0.f;
            // patch I's ring covers slots [PB I - 1, PB I + PB]:
            // I from ceil(i / PB) - 1 to floor((i + 1) / PB)   (i >= 0)
            const int ilo = (i + PB - 1) / PB - 1, ihi = (i + 1) / PB;
            const int jlo = (j + PB - 1) / PB - 1, jhi = (j + 1) / PB;
            for (int J = max(jlo, 0); J <= min(jhi, P.npy - 1); ++J)
                for (int I = max(ilo, 0); I <= min(ihi, P.npx - 1); ++I) {
                    const int q = P.pid[J * P.npx + I];
                    if (q < 0) continue;
                    const int ii = i - (PB * I - 1), jj = j - (PB * J - 1);
                    const int k = P.lmap[(int64_t)q * PMAX + (f * PR + jj) * PR + ii];
                    if (k >= 0) s += P.ybuf[(int64_t)q * PMAX + k];
                }
            zv = s;
        }
        z[of] = zv;
        rz += (double)rv * zv;
        r2 += (double)rv * rv;
    }
}

// x += alpha p, r -= alpha q (FP32), no preconditioning
__global__ void __launch_bounds__(256) k_cg_xr(Layout L, const int* __restrict__ tiles, int nf, CgWork<float> w,
                                               const float* __restrict__ p, const CgScalars* sc) {
    if (sc->done) return;
    const int tile = tiles[blockIdx.x];
    const int c0 = (tile % L.ntx) * TX, r0 = (tile / L.ntx) * TY2;
    const int64_t o = L.off(c0 + (threadIdx.x & 31), r0 + (threadIdx.x >> 5), 0);
    const float alpha = (float)sc->alpha;
    float* __restrict__ X = w.x;
    float* __restrict__ R = w.r;
    const float* __restrict__ Q = w.q;
    float pv[3], xv[3], rv[3], qv[3];
#pragma unroll
    for (int f = 0; f < 3; ++f) {
        const int64_t of = (int64_t)f * L.stride + o;
        pv[f] = __ldg(p + of); xv[f] = X[of]; rv[f] = R[of]; qv[f] = __ldg(Q + of);
    }
#pragma unroll
    for (int f = 0; f < 3; ++f) {
        const int64_t of = (int64_t)f * L.stride + o;
        X[of] = xv[f] + alpha * pv[f];
        R[of] = rv[f] - alpha * qv[f];
    }
}

}  // namespace stk
