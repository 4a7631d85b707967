// One 2D tile of the matrix-free apply (shared by the per-tile kernels and the
// persistent batched solver).  See apply.cu for the method and the modes.
#pragma once
#include "internal.cuh"

namespace stk {

template <class T> struct Acc;
template <> struct Acc<double> {
    double s = 0.0;
    __device__ void add(double a, double b) { s = fma(a, b, s); }
    __device__ double warp() { return warp_sum(s); }
};
// FP32 vectors: products and sums kept as float-float pairs (TwoProd via FMA,
// TwoSum) so the partial is accurate to ~2^-44 relative without FP64 math.
template <> struct Acc<float> {
    float hi = 0.f, lo = 0.f;
    __device__ void add(float a, float b) {
        float p = a * b;
        float e = fmaf(a, b, -p);
        float s, t;
        two_sum(hi, p, s, t);
        lo += t + e;
        hi = s;
    }
    __device__ double warp() { return warp_sum_ff(hi, lo); }
};

template <class T, class C> __device__ __forceinline__ T ld(const C* p, int64_t o);
template <> __device__ __forceinline__ double ld<double, double>(const double* p, int64_t o) { return __ldg(p + o); }
template <> __device__ __forceinline__ float ld<float, float>(const float* p, int64_t o) { return __ldg(p + o); }
template <> __device__ __forceinline__ float ld<float, __nv_bfloat16>(const __nv_bfloat16* p, int64_t o) {
    return __bfloat162float(__ldg(p + o));      // read-only path, as for the FP32 and FP64 coefficients
}

template <class T, int MODE>
__device__ __forceinline__ T stage_val(const T* x, const T* pold, T beta, int64_t o) {
    if (MODE == MODE_CG) return x[o] + beta * pold[o];
    return x[o];
}

template <class T, int TY> struct Smem2 {
    T U[TY + 2][TX + 2], V[TY + 2][TX + 2], N[TY + 2][TX + 2];
    T Zu[TY + 1][TX + 1], Zv[TY + 1][TX + 1];
    T own[3][TY][TX];   // the tile's own unknowns (after the direction update)
};

// Apply on the tile whose lower corner is (c0, r0) in padded coordinates.
// x: input (CG mode: z, with p = z + beta pold written to pnew); y: output;
// b: RESID right-hand side.  Returns the warp sum of this warp's partial dot
// (x.y in CG mode, y.y in RESID mode); the caller combines warps.
template <class T, class C, int MODE, int TY, int NT>
__device__ double apply2d_tile(const Layout& L, int c0, int r0, const Coef<C>& cf, const T* __restrict__ x,
                               T* __restrict__ y, const T* __restrict__ pold, T* __restrict__ pnew, T beta,
                               const T* __restrict__ b, Smem2<T, TY>& sm) {
    const int64_t S = L.stride;
    const C *a_c = cf.f[0], *a_n = cf.f[1], *d_c = cf.f[2], *d_n = cf.f[3], *K_u = cf.f[4], *K_v = cf.f[5];
    const int t = threadIdx.x;
    // Every global load of the tile is issued up front (face coefficients and
    // the own slots' coefficients into registers), so one CTA waits for one
    // memory round trip rather than three.
    constexpr int NFACE = ((TY + 1) * (TX + 1) + NT - 1) / NT;
    constexpr int NOWN = (TY * TX + NT - 1) / NT;
    T ku[NFACE], kv[NFACE];
#pragma unroll
    for (int q = 0; q < NFACE; ++q) {
        int e = t + q * NT;
        if (e < (TY + 1) * (TX + 1)) {
            int jj = e / (TX + 1), ii = e - jj * (TX + 1);
            ku[q] = ld<T, C>(K_u, L.off(c0 + ii, r0 - 1 + jj, 0));
            kv[q] = ld<T, C>(K_v, L.off(c0 - 1 + ii, r0 + jj, 0));
        }
    }
    T oac[NOWN], oan[NOWN], odc[NOWN], odn[NOWN];
#pragma unroll
    for (int q = 0; q < NOWN; ++q) {
        int e = t + q * NT;
        if (e < TY * TX) {
            const int64_t o = L.off(c0 + (e & (TX - 1)), r0 + e / TX, 0);
            oac[q] = ld<T, C>(a_c, o); oan[q] = ld<T, C>(a_n, o);
            odc[q] = ld<T, C>(d_c, o); odn[q] = ld<T, C>(d_n, o);
        }
    }
    for (int e = t; e < (TY + 2) * (TX + 2); e += NT) {
        int jj = e / (TX + 2), ii = e - jj * (TX + 2);
        int64_t o = L.off(c0 - 1 + ii, r0 - 1 + jj, 0);
        T ac = ld<T, C>(a_c, o), an = ld<T, C>(a_n, o);
        T txx = stage_val<T, MODE>(x, pold, beta, o);
        T txy = stage_val<T, MODE>(x + S, pold + S, beta, o);
        T p = stage_val<T, MODE>(x + 2 * S, pold + 2 * S, beta, o);
        if (ii >= 1 && ii <= TX && jj >= 1 && jj <= TY) {
            if (MODE == MODE_CG) { pnew[o] = txx; pnew[S + o] = txy; pnew[2 * S + o] = p; }
            sm.own[0][jj - 1][ii - 1] = txx;
            sm.own[1][jj - 1][ii - 1] = txy;
            sm.own[2][jj - 1][ii - 1] = p;
        }
        sm.U[jj][ii] = ac * (p - txx);
        sm.V[jj][ii] = ac * (p + txx);
        sm.N[jj][ii] = an * txy;
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < NFACE; ++q) {
        int e = t + q * NT;
        if (e < (TY + 1) * (TX + 1)) {
            int jj = e / (TX + 1), ii = e - jj * (TX + 1);
            sm.Zu[jj][ii] = ku[q] * ((sm.U[jj][ii + 1] - sm.U[jj][ii]) + (sm.N[jj][ii + 1] - sm.N[jj + 1][ii + 1]));
            sm.Zv[jj][ii] = kv[q] * ((sm.V[jj + 1][ii] - sm.V[jj][ii]) + (sm.N[jj + 1][ii] - sm.N[jj + 1][ii + 1]));
        }
    }
    __syncthreads();
    Acc<T> acc;
#pragma unroll
    for (int q = 0; q < NOWN; ++q) {
        const int e = t + q * NT;
        if (e >= TY * TX) break;
        const int tx = e & (TX - 1), ty = e / TX;
        const int64_t o = L.off(c0 + tx, r0 + ty, 0);
        T ac = oac[q], an = oan[q], dc = odc[q], dn = odn[q];
        T txx = sm.own[0][ty][tx], txy = sm.own[1][ty][tx], p_ = sm.own[2][ty][tx];
        T zu = sm.Zu[ty + 1][tx], zur = sm.Zu[ty + 1][tx + 1], zud = sm.Zu[ty][tx];
        T zv = sm.Zv[ty][tx + 1], zvu = sm.Zv[ty + 1][tx + 1], zvl = sm.Zv[ty][tx];
        T yp, yxx;
        if (ac != T(0)) {
            yp = ac * ((zu - zur) + (zv - zvu));
            yxx = dc * txx + ac * ((zur - zu) + (zv - zvu));
        } else {
            yp = p_;
            yxx = txx;
        }
        T yxy = dn * txy + an * ((zu - zud) + (zv - zvl));
        if (MODE == MODE_RESID) {
            yxx = b[o] - yxx; yxy = b[S + o] - yxy; yp = b[2 * S + o] - yp;
        }
        y[o] = yxx; y[S + o] = yxy; y[2 * S + o] = yp;
        if (MODE == MODE_RESID) { acc.add(yxx, yxx); acc.add(yxy, yxy); acc.add(yp, yp); }
        else if (MODE == MODE_CG) { acc.add(txx, yxx); acc.add(txy, yxy); acc.add(p_, yp); }
    }
    return MODE == MODE_PLAIN ? 0.0 : acc.warp();
}

}  // namespace stk
