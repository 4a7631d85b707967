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
//   3. rotate every cell's (tau_xx, p) pair to (tau_xx + p, tau_xx - p)/sqrt2
//      (u faces couple only tau_xx - p, v faces only tau_xx + p, so a cell
//      whose faces in one direction are nearly dead has one combination
//      held only by the tiny stress block C: in the original basis that is
//      an eigenvalue near 1e-8 after diagonal scaling, which FP32 cannot
//      factor; after the rotation the diagonal scaling absorbs it);
//   4. scale to unit diagonal (D^-1/2 Q A_p Q D^-1/2 = L L^T), Cholesky, invert
//      the factor (X = L^-1) and store it in FP32 (BF16 loses the small-
//      eigenvalue directions of the worst-conditioned patches, and those
//      then cost many CG iterations on large grids).
// Apply (every CG step): one CTA per patch computes
// z_p = Q D^-1/2 X^T X D^-1/2 Q r_p (FP32 accumulation), symmetric positive
// definite whatever the rounding of X; a gather kernel sums, for every
// unknown, the contributions of the (at most four) patches covering it in a
// fixed order, so the preconditioner is symmetric and deterministic.
// Inactive unknowns get z = r.
#include <cmath>
#include <vector>
#include "schwarz_plan.cuh"

namespace stk {

__global__ void k_schwarz_mark(Layout L, DevArrays D, int npx, int npy, int* flag) {
    int I = blockIdx.x * blockDim.x + threadIdx.x, J = blockIdx.y;
    if (I >= npx || J >= npy) return;
    int any = 0;
    for (int f = 0; f < 3; ++f)
        for (int jj = 0; jj < PB; ++jj)
            for (int ii = 0; ii < PB; ++ii) any |= unknown_active(D, L, f, PB * I + ii, PB * J + jj);
    flag[J * npx + I] = any;
}

// one CTA (256 threads) per active patch.  The local matrix is assembled in
// FP64 from the FP64 operator coefficients: in FP32 the cancellation between
// face terms leaves some patch matrices indefinite.  Only the unit-diagonal
// matrix is rounded to FP32 for the factorisation.  Every global load is
// issued in parallel (activity flags, then the coefficients of the faces
// touching the patch, staged in shared memory); each thread accumulates one
// row, faces in a fixed order, so the local matrices are reproducible bit for
// bit.  Dynamic smem: the FP64 matrix (PMAX^2 doubles), whose upper half
// later holds the scaled FP32 matrix and whose lower half the inverse factor
// X = L^-1, then the diagonal scaling: about 94 KB, two CTAs per SM.
constexpr int SW_NFACE = 2 * (PR + 2) * (PR + 2);   // faces of both directions around a patch
constexpr int SW_SETUP_SMEM = PMAX * PMAX * 8 + PMAX * 4;
__global__ void __launch_bounds__(256) k_schwarz_setup(Layout L, DevArrays D, const double* coef, SchwarzPlan P) {
    extern __shared__ __align__(16) double smd[];
    double* Ad = smd;                                        // n x n (row-major, stride PMAX), FP64
    float* A = reinterpret_cast<float*>(smd) + PMAX * PMAX;  // upper half: scaled copy, FP32
    float* X = reinterpret_cast<float*>(smd);                // lower half: L^-1
    float* sc = reinterpret_cast<float*>(smd + PMAX * PMAX); // 1/sqrt(diag)
    __shared__ short map[PMAX];
    __shared__ unsigned ballots[4];
    __shared__ double dd[PMAX];                              // 1/sqrt(diag) in FP64, 0 if not positive
    __shared__ double fK[SW_NFACE], fb[SW_NFACE][6];
    __shared__ short fidx[SW_NFACE][6];
    const int p = blockIdx.x;
    const int I = P.corner[p] & 0xffff, J = P.corner[p] >> 16;
    const int a0 = PB * I - 1, b0 = PB * J - 1;       // ring origin (slot coords)
    const int t = threadIdx.x, lane = t & 31, w = t >> 5;
    const int64_t S = L.stride;
    const double *a_c = coef, *a_n = coef + S, *d_c = coef + 2 * S, *d_n = coef + 3 * S, *K_u = coef + 4 * S,
                 *K_v = coef + 5 * S;
    // 1. local indices in fixed order (field, row, column): a ballot scan
    bool act = false;
    if (t < PMAX) {
        const int f = t / (PR * PR), rem = t % (PR * PR), jj = rem / PR, ii = rem % PR;
        act = unknown_active(D, L, f, a0 + ii, b0 + jj);
    }
    if (w < 4) {
        const unsigned m = __ballot_sync(0xffffffffu, act);
        if (lane == 0) ballots[w] = m;
    }
    __syncthreads();
    int n = 0;
    for (int q = 0; q < 4; ++q) n += __popc(ballots[q]);
    if (t < PMAX) {
        int before = 0;
        for (int q = 0; q < w; ++q) before += __popc(ballots[q]);
        before += __popc(ballots[w] & ((1u << lane) - 1u));
        map[t] = act ? (short)before : (short)-1;
        P.lmap[(int64_t)p * PMAX + t] = map[t];
    }
    if (t == 0) P.nloc[p] = n;
    for (int e = t; e < n * PMAX; e += 256) Ad[e] = 0.0;
    __syncthreads();
    auto lidx = [&](int f, int i, int j) -> int {
        int ii = i - a0, jj = j - b0;
        if (ii < 0 || jj < 0 || ii >= PR || jj >= PR) return -1;
        return map[(f * PR + jj) * PR + ii];
    };
    // 2. stage the faces touching the patch (u faces, then v faces; rows
    // b0-1 .. b0+PR, columns a0-1 .. a0+PR): K, the six coefficients of
    // B^T's row and the local indices they multiply; K = 0 marks no face
    if (t < SW_NFACE) {
        const int dir = t / ((PR + 2) * (PR + 2)), rem = t % ((PR + 2) * (PR + 2));
        const int i = a0 + rem % (PR + 2) - 1, j = b0 + rem / (PR + 2) - 1;
        const bool ok = dir == 0 ? (i >= 0 && i <= L.nx && j >= 0 && j < L.ny)
                                 : (i >= 0 && i < L.nx && j >= 0 && j <= L.ny);
        double K = 0.0;
        if (ok) {
            const int64_t o = L.off(i + 1, j + 1, 0);
            K = (dir == 0 ? K_u : K_v)[o];
            if (K != 0.0) {
                if (dir == 0) {
                    const double am = a_c[L.off(i, j + 1, 0)], ap = a_c[o];
                    fidx[t][0] = lidx(0, i - 1, j); fb[t][0] = am;       // txx(i-1): +a
                    fidx[t][1] = lidx(2, i - 1, j); fb[t][1] = -am;      // p(i-1):   -a
                    fidx[t][2] = lidx(0, i, j);     fb[t][2] = -ap;      // txx(i):   -a
                    fidx[t][3] = lidx(2, i, j);     fb[t][3] = ap;       // p(i):     +a
                    fidx[t][4] = lidx(1, i, j);     fb[t][4] = a_n[o];                     // txy(i, j)
                    fidx[t][5] = lidx(1, i, j + 1); fb[t][5] = -a_n[L.off(i + 1, j + 2, 0)];  // txy(i, j+1)
                } else {
                    const double am = a_c[L.off(i + 1, j, 0)], ap = a_c[o];
                    fidx[t][0] = lidx(0, i, j - 1); fb[t][0] = -am;      // txx(j-1): -a
                    fidx[t][1] = lidx(2, i, j - 1); fb[t][1] = -am;      // p(j-1):   -a
                    fidx[t][2] = lidx(0, i, j);     fb[t][2] = ap;       // txx(j):   +a
                    fidx[t][3] = lidx(2, i, j);     fb[t][3] = ap;       // p(j):     +a
                    fidx[t][4] = lidx(1, i, j);     fb[t][4] = a_n[o];                     // txy(i, j)
                    fidx[t][5] = lidx(1, i + 1, j); fb[t][5] = -a_n[L.off(i + 2, j + 1, 0)];  // txy(i+1, j)
                }
            }
        }
        fK[t] = K;
    }
    __syncthreads();
    // 3. row r of A_p by thread r: the stress diagonal C, then K_f b_f b_f^T
    // of every face containing r, faces in order (each entry sums the same
    // terms in the same order whichever thread owns it: reproducible bit for
    // bit)
    if (t < n) {
        double* row = Ad + (int64_t)t * PMAX;
        int pos = -1;                     // position (field, ring row, ring column) of unknown t
        for (int e = 0; e < PMAX; ++e)
            if (map[e] == t) { pos = e; break; }
        const int f = pos / (PR * PR), cell = pos % (PR * PR);
        if (f < 2) row[t] += (f == 0 ? d_c : d_n)[L.off(a0 + cell % PR + 1, b0 + cell / PR + 1, 0)];
        for (int fc = 0; fc < SW_NFACE; ++fc) {
            const double K = fK[fc];
            if (K == 0.0) continue;
            for (int q = 0; q < 6; ++q) {
                if (fidx[fc][q] != t) continue;
                const double kb = K * fb[fc][q];
                for (int c = 0; c < 6; ++c) {
                    const int ic = fidx[fc][c];
                    if (ic >= 0) row[ic] += kb * fb[fc][c];
                }
            }
        }
    }
    __syncthreads();
    // 5. Q A_p Q with Q the symmetric orthogonal pair rotation (rows, then columns)
    constexpr double H = 0.70710678118654752440;
    for (int e = t; e < PR * PR * n; e += 256) {
        int cell = e / n, c = e % n;
        int kt = map[cell], kp = map[2 * PR * PR + cell];
        if (kt < 0 || kp < 0) continue;
        double a = Ad[kt * PMAX + c], b = Ad[kp * PMAX + c];
        Ad[kt * PMAX + c] = (a + b) * H;
        Ad[kp * PMAX + c] = (a - b) * H;
    }
    __syncthreads();
    for (int e = t; e < PR * PR * n; e += 256) {
        int cell = e / n, r = e % n;
        int kt = map[cell], kp = map[2 * PR * PR + cell];
        if (kt < 0 || kp < 0) continue;
        double a = Ad[r * PMAX + kt], b = Ad[r * PMAX + kp];
        Ad[r * PMAX + kt] = (a + b) * H;
        Ad[r * PMAX + kp] = (a - b) * H;
    }
    __syncthreads();
    // 6. unit-diagonal scaling (FP64, then rounded to FP32).  The FP32 row r
    // lands on FP64 rows >= r of the same buffer, so rows are converted from
    // the last down, a block of rows at a time (read all, barrier, write all).
    // (FP64 divisions and square roots are slow on this part: one per row)
    for (int k = t; k < n; k += 256) {
        const double d = Ad[k * PMAX + k];
        dd[k] = d > 0.0 ? 1.0 / sqrt(d) : 0.0;
        sc[k] = d > 0.0 ? (float)dd[k] : 1.f;
    }
    __syncthreads();
    constexpr int CONV_ROWS = 16;
    for (int r1 = n; r1 > 0; r1 -= CONV_ROWS) {
        const int r0 = max(r1 - CONV_ROWS, 0);
        float v[(CONV_ROWS * PMAX + 255) / 256];
#pragma unroll
        for (int q = 0; q < (CONV_ROWS * PMAX + 255) / 256; ++q) {
            const int e = t + 256 * q, r = r0 + e / PMAX, c = e % PMAX;
            v[q] = 0.f;
            if (r < r1 && c < n) {
                const double sr = dd[r], scc = dd[c];
                v[q] = (sr > 0.0 && scc > 0.0) ? (float)(Ad[r * PMAX + c] * sr * scc) : (r == c ? 1.f : 0.f);
            }
        }
        __syncthreads();
#pragma unroll
        for (int q = 0; q < (CONV_ROWS * PMAX + 255) / 256; ++q) {
            const int e = t + 256 * q, r = r0 + e / PMAX, c = e % PMAX;
            if (r < r1 && c < n) A[r * PMAX + c] = v[q];
        }
        __syncthreads();
    }
    // 7. Cholesky (lower, in place, FP32).  Column k is copied to colk once
    // scaled; the trailing update runs on a 16 x 16 thread grid (thread
    // (tr, tc): rows k+1+tr+16i, columns k+1+tc+16j <= row), lower triangle only
    __shared__ float colk[PMAX];
    const int tr = t >> 4, tc = t & 15;
    for (int k = 0; k < n; ++k) {
        if (t == 0) {
            float d = A[k * PMAX + k];
            A[k * PMAX + k] = d > 1e-12f ? sqrtf(d) : 1.f;    // a vanishing pivot is replaced (robust, still SPD)
        }
        __syncthreads();
        const float piv = A[k * PMAX + k];
        for (int r = k + 1 + t; r < n; r += 256) {
            const float v = A[r * PMAX + k] / piv;
            A[r * PMAX + k] = v;
            colk[r] = v;
        }
        __syncthreads();
        for (int r = k + 1 + tr; r < n; r += 16) {
            const float lr = colk[r];
            float* Ar = A + r * PMAX;
            for (int c = k + 1 + tc; c <= r; c += 16) Ar[c] -= lr * colk[c];
        }
        __syncthreads();
    }
    // 8. X = L^-1 by forward elimination on the identity, all columns at
    // once: row k is final once divided by L_kk, then eliminated from the
    // rows below (thread (tr, tc): rows k+1+tr+16i, columns tc+16j <= k)
    for (int e = t; e < n * PMAX; e += 256) {
        const int r = e / PMAX, c = e - r * PMAX;
        if (c < n) X[e] = r == c ? 1.f : 0.f;
    }
    __syncthreads();
    for (int k = 0; k < n; ++k) {
        const float inv = 1.f / A[k * PMAX + k];
        for (int c = t; c <= k; c += 256) X[k * PMAX + c] *= inv;
        __syncthreads();
        const float* Xk = X + k * PMAX;
        for (int r = k + 1 + tr; r < n; r += 16) {
            const float lr = A[r * PMAX + k];
            float* Xr = X + r * PMAX;
            for (int c = tc; c <= k; c += 16) Xr[c] -= lr * Xk[c];
        }
        __syncthreads();
    }
    // stored factor: row factors rho_r^2 and the packed FP16 rows X[r][0..r] /
    // rho_r (padded to 16 bytes), and the scaling by position.  The patch
    // operator D^-1/2 X~^T diag(rho^2) X~ D^-1/2 is symmetric positive
    // definite whatever the rounding of X~ (it stays triangular with a
    // positive diagonal: |X[r][r]| >= 1 and rho_r <= sqrt(cond)).
    __shared__ float rho_inv[PMAX];
    uint8_t* F = P.fac + (int64_t)p * SW_FAC_BYTES;
    if (t < PMAX) {
        float m = 0.f;
        if (t < n)
            for (int c = 0; c <= t; ++c) m = fmaxf(m, fabsf(X[t * PMAX + c]));
        rho_inv[t] = m > 0.f ? 1.f / m : 0.f;
        reinterpret_cast<float*>(F)[t] = m * m;
    }
    __syncthreads();
    __half* Xh = reinterpret_cast<__half*>(F + SW_RS_BYTES);
    const int n8 = (n + 7) / 8 * 8;
    for (int e = t; e < n * n8; e += 256) {
        const int r = e / n8, c = e % n8;
        if (c < (r / 8 + 1) * 8) Xh[sw_fac_off(r, c, n)] = __float2half_rn(c <= r ? X[r * PMAX + c] * rho_inv[r] : 0.f);
    }
    for (int e = t; e < PMAX; e += 256) P.scale[(int64_t)p * PMAX + e] = map[e] >= 0 ? sc[map[e]] : 0.f;
}

// z_p = Q D^-1/2 X~^T diag(rho^2) X~ D^-1/2 Q r_p, one CTA (128 threads) per
// active patch.  Thread 0 starts a bulk (TMA) copy of the stored factor
// (13 KB at most) into shared memory, completing on an mbarrier; meanwhile
// the threads gather, rotate and scale r_p into s.  Then the two triangular
// products on the tensor cores (sw_factor_products); rotate back and store
// by position.  A copy
// that never completes (bounded wait) marks the solve STOKES_ERR_TIMEOUT and
// ends it.  With the test hook (sc->wait_test) no copy is issued, so the
// wait runs out after SW_TEST_POLLS polls and nothing is left in flight.
// Given q, the residual read is r - alpha q (alpha of this CG step): the
// step's update of r is written later by the gather, for every slot once.
__global__ void __launch_bounds__(128, 15) k_schwarz_gemv(Layout L, SchwarzPlan P, const float* __restrict__ r,
                                                      const float* __restrict__ q, CgScalars* sc) {
    extern __shared__ __align__(128) uint8_t Fs[];             // SW_FAC_BYTES
    __shared__ __align__(16) float s[PMAX8];            // r_p, then (as y) X~ r_p, then z_p
    __shared__ __align__(16) __half hb[SW_HB_HALVES];
    __shared__ __align__(8) unsigned long long bar;
    __shared__ int ok_s;
    const int t = threadIdx.x;
    const int p = blockIdx.x;
    const uint32_t b_addr = smem_u32(&bar);
    // the patch's size and corner and the solve's scalars are loaded together
    // (one memory round trip before the copy starts)
    const int n = P.nloc[p], cw = P.corner[p];
    const int done = sc->done;
    const bool stall = sc->wait_test != 0;
    const float alpha = q ? (float)sc->alpha : 0.f;
    if (done) return;
    if (t == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(b_addr), "r"(1) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        if (!stall) sw_issue(b_addr, Fs, P.fac + (int64_t)p * SW_FAC_BYTES, sw_patch_bytes(n), P.evict_first != 0);
    }
    constexpr float H = 0.70710678118654752f;
    const int I = cw & 0xffff, J = cw >> 16;
    const int a0 = PB * I - 1, b0 = PB * J - 1;
    const short* map = P.lmap + (int64_t)p * PMAX;
    const float* scl = P.scale + (int64_t)p * PMAX;
    // gather, rotate and scale: position e < PR^2 handles the cell's
    // (tau_xx, p) pair, e in [PR^2, 2 PR^2) the node's tau_xy.  All loads
    // are independent (r is zero on inactive unknowns and outside the grid,
    // the scaling is stored by position), so they are in flight together.
    int kk = -1, kp = -1;
    float sa = 0.f, sb = 0.f;
    if (t < 2 * PR * PR) {
        const int e = t;
        const int rem = e % (PR * PR), jj = rem / PR, ii = rem % PR;
        const int64_t o = L.off(a0 + ii + 1, b0 + jj + 1, 0);
        kk = map[e];
        sa = scl[e];
        if (e >= PR * PR) {
            const float rv = q ? r[L.stride + o] - alpha * q[L.stride + o] : r[L.stride + o];
            if (kk >= 0) s[kk] = rv * sa;
        } else {
            kp = map[2 * PR * PR + e];
            sb = scl[2 * PR * PR + e];
            const float rt = q ? r[o] - alpha * q[o] : r[o];
            const float rp = q ? r[2 * L.stride + o] - alpha * q[2 * L.stride + o] : r[2 * L.stride + o];
            // the scaling belongs to the rotated unknowns: rotate, then scale
            if (kk >= 0 && kp >= 0) {
                s[kk] = (rt + rp) * H * sa;
                s[kp] = (rt - rp) * H * sb;
            } else if (kk >= 0) {
                s[kk] = rt * sa;
            } else if (kp >= 0) {
                s[kp] = rp * sb;
            }
        }
    }
    if (t >= n && t < (n + 7) / 8 * 8) s[t] = 0.f;    // the padded last block
    if (t == 0) ok_s = mbar_wait(b_addr, 0, stall ? SW_TEST_POLLS : SW_WAIT_POLLS) ? 1 : 0;
    __syncthreads();
    if (!ok_s) {
        // give an issued copy one more bounded wait before the CTA leaves
        if (t == 0) {
            if (!stall) mbar_wait(b_addr, 0);
            sc->status = STOKES_ERR_TIMEOUT;
            sc->done = 1;
        }
        return;
    }
    sw_factor_products(Fs, n, s, s, hb);
    // scale, rotate back and store by position
    float* out = P.ybuf + (int64_t)(J * P.npx + I) * PMAX;
    if (t < 2 * PR * PR) {
        const int e = t;
        if (e >= PR * PR) {
            if (kk >= 0) out[e] = s[kk] * sa;
        } else if (kk >= 0 && kp >= 0) {
            const float a = s[kk] * sa, b = s[kp] * sb;     // scale, then rotate back
            out[e] = (a + b) * H;
            out[2 * PR * PR + e] = (a - b) * H;
        } else if (kk >= 0) {
            out[e] = s[kk] * sa;
        } else if (kp >= 0) {
            out[2 * PR * PR + e] = s[kp] * sb;
        }
    }
}

// dynamic shared memory of k_schwarz_gemv: the stored factor
constexpr int SW_GEMV_SMEM = SW_FAC_BYTES;

static inline void launch_schwarz_gemv(const Layout& L, const SchwarzPlan& P, const float* r, CgScalars* sc,
                                       cudaStream_t s, const float* q = nullptr) {
    if (P.np) k_schwarz_gemv<<<P.np, 128, SW_GEMV_SMEM, s>>>(L, P, r, q, sc);
}

// z at one slot (c, rr) from the patches' local results, in two parts so
// that a thread can issue the loads of several slots before using any:
// sw_gather_load issues every load (the residual, the activity flags and a
// fixed 2 x 2 window of patches' results), sw_gather_finish sums, writes z
// and accumulates r.z and r.r.  Inactive unknowns take z = r (zero outside
// the grid).
struct SwGather {
    float rv[3], v[3][4];
    bool act[3], use[4], real;
    int64_t o;
};
// The CG update fused into the gather (x += alpha p, r -= alpha q for the
// slot itself): the slot's q, x and p.
struct SwUpdate {
    float qv[3], xv[3], pv[3];
};

__device__ __forceinline__ void sw_update_load(const Layout& L, const CgWork<float>& w, const float* __restrict__ p,
                                               int64_t o, SwUpdate& u) {
#pragma unroll
    for (int f = 0; f < 3; ++f) {
        const int64_t of = (int64_t)f * L.stride + o;
        u.qv[f] = __ldg(w.q + of);
        u.xv[f] = w.x[of];
        u.pv[f] = __ldg(p + of);
    }
}

__device__ __forceinline__ void sw_gather_load(const Layout& L, const DevArrays& D, const SchwarzPlan& P,
                                               const float* __restrict__ r, int c, int rr, SwGather& g) {
    const int i = c - 1, j = rr - 1;
    g.o = L.off(c, rr, 0);
    // patch I's ring covers slots [PB I - 1, PB I + PB]:
    // I from ceil(i / PB) - 1 to floor((i + 1) / PB)   (i >= 0)
    const int ilo = max((i + PB - 1) / PB - 1, 0), ihi = min((i + 1) / PB, P.npx - 1);
    const int jlo = max((j + PB - 1) / PB - 1, 0), jhi = min((j + 1) / PB, P.npy - 1);
    g.real = i >= 0 && j >= 0 && i <= L.nx && j <= L.ny;
    // a fixed 2 x 2 window of patches (ilo.., jlo..); the ones outside
    // [ilo, ihi] x [jlo, jhi] (which may lie past the patch grid) are masked
    // and read element 0 instead.  Inside the ranges the ring position is in
    // [0, PR) (PB I - 1 <= i <= PB I + PB).  The local results are zero for
    // inactive patches and unknowns, so they are summed unconditionally.
    // (The results hold npy npx PMAX floats, far below 2^31.)
    int base[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int I = ilo + (q & 1), J = jlo + (q >> 1);
        g.use[q] = I <= ihi && J <= jhi;
        const int ii = i - (PB * I - 1), jj = j - (PB * J - 1);
        base[q] = g.use[q] ? (J * P.npx + I) * PMAX + jj * PR + ii : 0;
    }
#pragma unroll
    for (int f = 0; f < 3; ++f) {
        g.rv[f] = r[(int64_t)f * L.stride + g.o];
        g.act[f] = unknown_active(D, L, f, i, j);
#pragma unroll
        for (int q = 0; q < 4; ++q) g.v[f][q] = P.ybuf[g.use[q] ? base[q] + f * PR * PR : 0];
    }
}

// With an update u (and alpha): r -= alpha q and x += alpha p are written
// first, and z, r.z, r.r use the new r.
__device__ __forceinline__ void sw_gather_finish(const Layout& L, SwGather& g, float* __restrict__ z,
                                                 AccT<float>& rz, AccT<float>& r2, const SwUpdate* u = nullptr,
                                                 float alpha = 0.f, float* __restrict__ r = nullptr,
                                                 float* __restrict__ x = nullptr) {
#pragma unroll
    for (int f = 0; f < 3; ++f) {
        if (u) {
            const int64_t of = (int64_t)f * L.stride + g.o;
            g.rv[f] = g.rv[f] - alpha * u->qv[f];
            r[of] = g.rv[f];
            x[of] = u->xv[f] + alpha * u->pv[f];
        }
        float s = 0.f;
#pragma unroll
        for (int q = 0; q < 4; ++q) s += g.use[q] ? g.v[f][q] : 0.f;
        const float zv = g.act[f] ? s : (g.real ? g.rv[f] : 0.f);
        z[(int64_t)f * L.stride + g.o] = zv;
        rz.add(g.rv[f], zv);          // float-float: FP64 arithmetic is slow on this part
        r2.add(g.rv[f], g.rv[f]);
    }
}

}  // namespace stk
