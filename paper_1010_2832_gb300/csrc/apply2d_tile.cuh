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
    return __bfloat162float(p[o]);
}

template <class T, int MODE>
__device__ __forceinline__ T stage_val(const T* x, const T* pold, T beta, int64_t o) {
    if (MODE == MODE_CG) return x[o] + beta * pold[o];
    return x[o];
}

template <class T, int TY> struct Smem2 {
    T U[TY + 2][TX + 2], V[TY + 2][TX + 2], N[TY + 2][TX + 2];
    T Zu[TY + 1][TX + 1], Zv[TY + 1][TX + 1];
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
    for (int e = t; e < (TY + 2) * (TX + 2); e += NT) {
        int jj = e / (TX + 2), ii = e - jj * (TX + 2);
        int64_t o = L.off(c0 - 1 + ii, r0 - 1 + jj, 0);
        T ac = ld<T, C>(a_c, o), an = ld<T, C>(a_n, o);
        T txx = stage_val<T, MODE>(x, pold, beta, o);
        T txy = stage_val<T, MODE>(x + S, pold + S, beta, o);
        T p = stage_val<T, MODE>(x + 2 * S, pold + 2 * S, beta, o);
        if (MODE == MODE_CG && ii >= 1 && ii <= TX && jj >= 1 && jj <= TY) {
            pnew[o] = txx; pnew[S + o] = txy; pnew[2 * S + o] = p;
        }
        sm.U[jj][ii] = ac * (p - txx);
        sm.V[jj][ii] = ac * (p + txx);
        sm.N[jj][ii] = an * txy;
    }
    __syncthreads();
    for (int e = t; e < (TY + 1) * (TX + 1); e += NT) {
        int jj = e / (TX + 1), ii = e - jj * (TX + 1);
        T ku = ld<T, C>(K_u, L.off(c0 + ii, r0 - 1 + jj, 0));
        T kv = ld<T, C>(K_v, L.off(c0 - 1 + ii, r0 + jj, 0));
        sm.Zu[jj][ii] = ku * ((sm.U[jj][ii + 1] - sm.U[jj][ii]) + (sm.N[jj][ii + 1] - sm.N[jj + 1][ii + 1]));
        sm.Zv[jj][ii] = kv * ((sm.V[jj + 1][ii] - sm.V[jj][ii]) + (sm.N[jj + 1][ii] - sm.N[jj + 1][ii + 1]));
    }
    __syncthreads();
    Acc<T> acc;
    for (int e = t; e < TY * TX; e += NT) {
        const int tx = e & (TX - 1), ty = e / TX;
        const int64_t o = L.off(c0 + tx, r0 + ty, 0);
        T ac = ld<T, C>(a_c, o), an = ld<T, C>(a_n, o), dc = ld<T, C>(d_c, o), dn = ld<T, C>(d_n, o);
        T p_, txx, txy;
        if (MODE == MODE_CG) {
            txx = pnew[o]; txy = pnew[S + o]; p_ = pnew[2 * S + o];
        } else {
            txx = x[o]; txy = x[S + o]; p_ = x[2 * S + o];
        }
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
