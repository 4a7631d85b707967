// Matrix-free apply of the SPD pressure-stress operator, eq. stokesmixedsystemspd,
// in the factored form of Section 7: y = C x + B (K (B^T x)).
//
// Tiles of the padded slot lattice: 2D 32x8 slots, taken by persistent,
// software-pipelined CTAs (the next tile's loads are in flight while the
// current tile is computed); 3D 32x4x4, one CTA per tile.
// Phase 1 stages, for the tile plus a one-slot halo, the row-weighted
// unknowns that each face sees (for a u face: a_c (p - tau_xx) of the cells
// on both sides and a_n tau_xy of the nodes above and below, ...).
// Phase 2 forms the face values z_f = K_f (B^T x)_f for every face the tile
// needs.  Phase 3 gathers y = C x + B z for the tile's own slots.
//
// Modes:  PLAIN  y = A x
//         RESID  y = b - A x, block partial of ||y||^2
//         CG     x := z + beta p_old (written to p_new for the tile), y = A x,
//                block partial of x . y  (the CG search-direction update fused
//                with the operator and the p.Ap dot)
// Block partials are summed by the last block to finish (fixed order, so
// the result is deterministic) which then updates the CG scalars.
#include <algorithm>
#include <cstdlib>
#include "internal.cuh"
#include "ctx.cuh"
#include "apply2d_tile.cuh"

namespace stk {

// Block reduction of one double per thread into partial[blockIdx.x], then the
// last block sums all partials (index order) and calls fin(total).
template <int NT, class Fin>
__device__ void block_partial_and_finish(double v, double* partial, unsigned* counter, int nblocks, Fin fin) {
    __shared__ double red[NT / 32];
    __shared__ bool last;
    v = warp_sum(v);
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) red[w] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int q = 0; q < NT / 32; ++q) s += red[q];
        partial[blockIdx.x] = s;
        __threadfence();
        unsigned prev = atomicAdd(counter, 1u);
        last = (prev == (unsigned)nblocks - 1u);
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    double s = 0.0;
    for (int b = threadIdx.x; b < nblocks; b += NT) s += ((volatile double*)partial)[b];
    s = warp_sum(s);
    if (lane == 0) red[w] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double tot = 0.0;
        for (int q = 0; q < NT / 32; ++q) tot += red[q];
        fin(tot);
        *counter = 0u;
    }
}

// ------------------------------- 2D -----------------------------------------
// Everything one thread loads for one 2D tile (32 x 8 slots, 256 threads):
// two staging positions of the (8+2) x (32+2) halo region, two face
// coefficients of each direction, the own slot's four coefficients.
template <class T> struct Tile2Loads {
    T sx[2][3], sp[2][3], sac[2], san[2];
    T ku[2], kv[2];
    T oac, oan, odc, odn;
};

constexpr int ST2 = (TY2 + 2) * (TX + 2);     // staged positions (340)
constexpr int FC2 = (TY2 + 1) * (TX + 1);     // faces of each direction (297)

template <class T, class C, int MODE>
__device__ __forceinline__ void tile2_load(const Layout& L, int c0, int r0, const Coef<C>& cf, const T* __restrict__ x,
                                           const T* __restrict__ pold, Tile2Loads<T>& d) {
    const int t = threadIdx.x;
    const int64_t S = L.stride;
#pragma unroll
    for (int q = 0; q < 2; ++q) {
        const int e = t + q * 256;
        if (e < ST2) {
            const int jj = e / (TX + 2), ii = e - jj * (TX + 2);
            const int64_t o = L.off(c0 - 1 + ii, r0 - 1 + jj, 0);
            d.sac[q] = ld<T, C>(cf.f[0], o);
            d.san[q] = ld<T, C>(cf.f[1], o);
#pragma unroll
            for (int f = 0; f < 3; ++f) {
                d.sx[q][f] = __ldg(x + f * S + o);
                if (MODE == MODE_CG) d.sp[q][f] = __ldg(pold + f * S + o);
            }
        }
        if (e < FC2) {
            const int jj = e / (TX + 1), ii = e - jj * (TX + 1);
            d.ku[q] = ld<T, C>(cf.f[4], L.off(c0 + ii, r0 - 1 + jj, 0));
            d.kv[q] = ld<T, C>(cf.f[5], L.off(c0 - 1 + ii, r0 + jj, 0));
        }
    }
    const int64_t o = L.off(c0 + (t & (TX - 1)), r0 + t / TX, 0);
    d.oac = ld<T, C>(cf.f[0], o);
    d.oan = ld<T, C>(cf.f[1], o);
    d.odc = ld<T, C>(cf.f[2], o);
    d.odn = ld<T, C>(cf.f[3], o);
}

// 2D apply, persistent over the tile list and software-pipelined: while a
// CTA forms the faces and outputs of one tile, the loads of its next tile are
// already in flight (registers), and the tile index after that too.  One
// block reduction per CTA.  Same arithmetic, in the same order, as
// apply2d_tile.
template <class T, class C, int MODE, int MINB>
__global__ void __launch_bounds__(256, MINB) k_apply2d(Layout L, const int* __restrict__ tiles, Coef<C> cf,
                                                       const T* __restrict__ x, T* __restrict__ y, ApplyArgs args,
                                                       int ntiles) {
    __shared__ Smem2<T, TY2> sm;
    if (MODE == MODE_CG && args.sc->done) return;
    const T beta = MODE == MODE_CG ? (T)args.sc->beta : T(0);
    const T* __restrict__ pold = (const T*)args.pold;
    T* __restrict__ pnew = (T*)args.pnew;
    const T* __restrict__ b = (const T*)args.b;
    const int64_t S = L.stride;
    const int t = threadIdx.x;
    const int G = gridDim.x;
    auto tile_at = [&](int k) { return tiles ? tiles[k] : k; };
    Acc<T> acc;
    int k = blockIdx.x;
    Tile2Loads<T> d;
    int tile = k < ntiles ? tile_at(k) : 0;
    int tile_next = k + G < ntiles ? tile_at(k + G) : 0;
    if (k < ntiles) tile2_load<T, C, MODE>(L, (tile % L.ntx) * TX, (tile / L.ntx) * TY2, cf, x, pold, d);
    for (; k < ntiles; k += G) {
        const int c0 = (tile % L.ntx) * TX, r0 = (tile / L.ntx) * TY2;
        // 1. stage this tile (p = z + beta p_old in CG mode)
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            const int e = t + q * 256;
            if (e < ST2) {
                const int jj = e / (TX + 2), ii = e - jj * (TX + 2);
                T v[3];
#pragma unroll
                for (int f = 0; f < 3; ++f) v[f] = MODE == MODE_CG ? d.sx[q][f] + beta * d.sp[q][f] : d.sx[q][f];
                if (ii >= 1 && ii <= TX && jj >= 1 && jj <= TY2) {
                    if (MODE == MODE_CG) {
                        const int64_t o = L.off(c0 - 1 + ii, r0 - 1 + jj, 0);
                        pnew[o] = v[0]; pnew[S + o] = v[1]; pnew[2 * S + o] = v[2];
                    }
                    sm.own[0][jj - 1][ii - 1] = v[0];
                    sm.own[1][jj - 1][ii - 1] = v[1];
                    sm.own[2][jj - 1][ii - 1] = v[2];
                }
                sm.U[jj][ii] = d.sac[q] * (v[2] - v[0]);
                sm.V[jj][ii] = d.sac[q] * (v[2] + v[0]);
                sm.N[jj][ii] = d.san[q] * v[1];
            }
        }
        const T ku0 = d.ku[0], ku1 = d.ku[1], kv0 = d.kv[0], kv1 = d.kv[1];
        const T ac = d.oac, an = d.oan, dc = d.odc, dn = d.odn;
        // 2. prefetch the next tile and the tile index after it
        const int kn = k + G;
        const int tile_cur = tile;
        tile = tile_next;
        if (kn < ntiles) {
            tile_next = kn + G < ntiles ? tile_at(kn + G) : 0;
            tile2_load<T, C, MODE>(L, (tile % L.ntx) * TX, (tile / L.ntx) * TY2, cf, x, pold, d);
        }
        (void)tile_cur;
        __syncthreads();
        // 3. face values z_f = K_f (B^T x)_f
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            const int e = t + q * 256;
            if (e < FC2) {
                const int jj = e / (TX + 1), ii = e - jj * (TX + 1);
                const T ku = q == 0 ? ku0 : ku1, kv = q == 0 ? kv0 : kv1;
                sm.Zu[jj][ii] = ku * ((sm.U[jj][ii + 1] - sm.U[jj][ii]) + (sm.N[jj][ii + 1] - sm.N[jj + 1][ii + 1]));
                sm.Zv[jj][ii] = kv * ((sm.V[jj + 1][ii] - sm.V[jj][ii]) + (sm.N[jj + 1][ii] - sm.N[jj + 1][ii + 1]));
            }
        }
        __syncthreads();
        // 4. y = C x + B z on the own slot
        {
            const int tx = t & (TX - 1), ty = t / TX;
            const int64_t o = L.off(c0 + tx, r0 + ty, 0);
            const T txx = sm.own[0][ty][tx], txy = sm.own[1][ty][tx], p_ = sm.own[2][ty][tx];
            const T zu = sm.Zu[ty + 1][tx], zur = sm.Zu[ty + 1][tx + 1], zud = sm.Zu[ty][tx];
            const T zv = sm.Zv[ty][tx + 1], zvu = sm.Zv[ty + 1][tx + 1], zvl = sm.Zv[ty][tx];
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
        __syncthreads();                         // the next tile's staging reuses shared memory
    }
    if (MODE != MODE_PLAIN) {
        double v = acc.warp();
        if ((t & 31) != 0) v = 0.0;
        CgScalars* sc = args.sc;
        block_partial_and_finish<256>(v, args.partial, args.counter, gridDim.x, [&](double tot) {
            if (MODE == MODE_RESID) { sc->rr = tot; return; }
            sc->pq = tot;
            if (!(tot > 0.0) || !isfinite(tot)) { sc->done = 1; sc->status = (isfinite(tot) ? STOKES_ERR_BREAKDOWN : STOKES_ERR_NONFINITE); }
            else sc->alpha = sc->rz / tot;
        });
    }
}

// 2D apply with FP32 vectors, four slots per thread: a CTA of 256 threads
// is four groups of 64, each working on its own 32 x 8 tile of the list
// (persistent: group g of CTA b takes tiles 4 b + g, 4 b + g + 4 G, ...)
// and synchronising on its own named barrier.  Every load of a row's 32
// slots is one 16-byte load per field for the vectors and FP32 coefficients,
// and per pair of fields for BF16 coefficients (the pair arrays of Coef),
// plus scalar loads for the two halo columns: about 5 load instructions per
// slot against 17 with one slot per thread.
// Every load of a tile is issued before any is used (one memory round trip
// per tile; 127 registers, two CTAs = eight tiles in flight per SM): FP32 on
// a 4096^2 box 0.77 of the measured HBM bandwidth (one slot per thread,
// software-pipelined: 0.69; this layout with a round trip per phase: 0.63).
// The arithmetic of each slot is that of apply2d_tile, in the same order.
// Four consecutive coefficients of one field as loaded (R: float4) and as
// FP32.  The kernel reads BF16 coefficients from the pair arrays instead;
// V4<__nv_bfloat16> only types its field-by-field branch, unused for BF16.
template <class C> struct V4;
template <> struct V4<float> {
    using R = float4;
    static __device__ __forceinline__ R ld(const float* p, int64_t o) {
        return __ldg(reinterpret_cast<const float4*>(p + o));
    }
    static __device__ __forceinline__ float4 f(const R& r) { return r; }
};
template <> struct V4<__nv_bfloat16> {
    using R = uint2;
    static __device__ __forceinline__ R ld(const __nv_bfloat16* p, int64_t o) {
        return __ldg(reinterpret_cast<const uint2*>(p + o));
    }
    static __device__ __forceinline__ float4 f(const R& w) {
        return make_float4(__uint_as_float(w.x << 16), __uint_as_float(w.x & 0xffff0000u), __uint_as_float(w.y << 16),
                           __uint_as_float(w.y & 0xffff0000u));
    }
};
__device__ __forceinline__ float f4(const float4& v, int i) { return i == 0 ? v.x : i == 1 ? v.y : i == 2 ? v.z : v.w; }
// a pair word of the BF16 pair arrays: first coefficient (low half), second
__device__ __forceinline__ float plo(uint32_t w) { return __uint_as_float(w << 16); }
__device__ __forceinline__ float phi(uint32_t w) { return __uint_as_float(w & 0xffff0000u); }
__device__ __forceinline__ float4 plo4(const uint4& q) { return make_float4(plo(q.x), plo(q.y), plo(q.z), plo(q.w)); }
__device__ __forceinline__ float4 phi4(const uint4& q) { return make_float4(phi(q.x), phi(q.y), phi(q.z), phi(q.w)); }
__device__ __forceinline__ uint32_t u4(const uint4& q, int i) { return i == 0 ? q.x : i == 1 ? q.y : i == 2 ? q.z : q.w; }

struct Smem2v {
    float U[TY2 + 2][TX + 2], V[TY2 + 2][TX + 2], N[TY2 + 2][TX + 2];
    float Zu[TY2 + 1][TX + 1], Zv[TY2 + 1][TX + 1];
    float own[3][TY2][TX];
};

template <class C, int MODE>
__global__ void __launch_bounds__(256, 2) k_apply2d_v4(Layout L, const int* __restrict__ tiles, Coef<C> cf,
                                                       const float* __restrict__ x, float* __restrict__ y,
                                                       ApplyArgs args, int ntiles) {
    __shared__ __align__(16) Smem2v smg[4];
    if (MODE == MODE_CG && args.sc->done) return;
    const float beta = MODE == MODE_CG ? (float)args.sc->beta : 0.f;
    const float* __restrict__ pold = (const float*)args.pold;
    float* __restrict__ pnew = (float*)args.pnew;
    const float* __restrict__ b = (const float*)args.b;
    const int64_t S = L.stride;
    const int g = threadIdx.x >> 6, l = threadIdx.x & 63;
    Smem2v& sm = smg[g];
    const C *a_c = cf.f[0], *a_n = cf.f[1], *d_c = cf.f[2], *d_n = cf.f[3], *K_u = cf.f[4], *K_v = cf.f[5];
    auto gsync = [&]() { asm volatile("bar.sync %0, 64;" ::"r"(1 + g) : "memory"); };
    // the thread's items of one tile: a staged quad (row l/8 of rows 0..7),
    // a second staged quad (rows 8, 9) or a halo-column pair of values, up to
    // three face quads or leftover faces, and its own output quad
    constexpr int NFQ = 2 * (TY2 + 1) * 8 + 2 * (TY2 + 1);   // 144 face quads + 18 single faces
    using CR = typename V4<C>::R;
    // BF16 coefficients come from the pair arrays: the staged and own quads'
    // (a_c, a_n) and (d_c, d_n) in one 16-byte load each, and the faces as
    // (K_u, K_v) quads of the ten rows r0-1 .. r0+8 (row r0-1+jr gives the
    // u faces of row jr and the v faces of row jr-1): 80 face loads a tile
    // instead of 144
    constexpr bool PAIR = sizeof(C) == 2;
    constexpr int NKQ = (TY2 + 2) * 8;                       // 80 pair quads
    const uint32_t* __restrict__ pac = cf.pr[0];
    const uint32_t* __restrict__ pdc = cf.pr[1];
    const uint32_t* __restrict__ pku = cf.pr[2];
    struct Loads {
        float4 xa[3], pa[3];
        CR aca, ana;                       // staged quad A
        float4 xb[3], pb[3];
        CR acb, anb;                       // staged quad B (l < 16)
        float hac, han;                    // or halo values (l < 36: .x of xb, pb)
        CR kf[3];                          // face coefficients (quads)
        float kf1[3];                      // or single faces
        CR oac, oan, odc, odn;             // own quad
        float4 ob[3];
        uint4 ppa, ppb, kq[2], opa, opd;   // pair form (BF16)
        uint32_t hp, ks;
    };
    auto load_tile = [&](int c0, int r0, Loads& d) {
        {
            const int64_t o = L.off(c0 + 4 * (l & 7), r0 - 1 + (l >> 3), 0);
#pragma unroll
            for (int f = 0; f < 3; ++f) {
                d.xa[f] = __ldg(reinterpret_cast<const float4*>(x + f * S + o));
                if (MODE == MODE_CG) d.pa[f] = __ldg(reinterpret_cast<const float4*>(pold + f * S + o));
            }
            if constexpr (PAIR) {
                d.ppa = __ldg(reinterpret_cast<const uint4*>(pac + o));
            } else {
                d.aca = V4<C>::ld(a_c, o);
                d.ana = V4<C>::ld(a_n, o);
            }
        }
        if (l < 16) {
            const int64_t o = L.off(c0 + 4 * (l & 7), r0 + 7 + (l >> 3), 0);
#pragma unroll
            for (int f = 0; f < 3; ++f) {
                d.xb[f] = __ldg(reinterpret_cast<const float4*>(x + f * S + o));
                if (MODE == MODE_CG) d.pb[f] = __ldg(reinterpret_cast<const float4*>(pold + f * S + o));
            }
            if constexpr (PAIR) {
                d.ppb = __ldg(reinterpret_cast<const uint4*>(pac + o));
            } else {
                d.acb = V4<C>::ld(a_c, o);
                d.anb = V4<C>::ld(a_n, o);
            }
        } else if (l < 16 + 2 * (TY2 + 2)) {
            const int e = l - 16, jj = e >> 1, ii = (e & 1) ? TX + 1 : 0;
            const int64_t o = L.off(c0 - 1 + ii, r0 - 1 + jj, 0);
#pragma unroll
            for (int f = 0; f < 3; ++f) {
                d.xb[f].x = __ldg(x + f * S + o);
                if (MODE == MODE_CG) d.pb[f].x = __ldg(pold + f * S + o);
            }
            if constexpr (PAIR) {
                d.hp = __ldg(pac + o);
            } else {
                d.hac = ld<float, C>(a_c, o);
                d.han = ld<float, C>(a_n, o);
            }
        }
        if constexpr (PAIR) {
#pragma unroll
            for (int u = 0; u < 2; ++u) {
                const int it = l + 64 * u;
                if (it < NKQ) {
                    d.kq[u] = __ldg(reinterpret_cast<const uint4*>(pku + L.off(c0 + 4 * (it & 7), r0 - 1 + (it >> 3), 0)));
                } else if (it < NKQ + 2 * (TY2 + 1)) {
                    const int e = it - NKQ, jj = e >> 1;
                    d.ks = (e & 1) ? __ldg(pku + L.off(c0 + TX, r0 - 1 + jj, 0)) : __ldg(pku + L.off(c0 - 1, r0 + jj, 0));
                }
            }
        } else {
#pragma unroll
        for (int u = 0; u < 3; ++u) {
            const int it = l + 64 * u;
            if (it < 2 * (TY2 + 1) * 8) {
                const int dir = it / ((TY2 + 1) * 8), rem = it - dir * ((TY2 + 1) * 8), jj = rem >> 3, qd = rem & 7;
                d.kf[u] = dir == 0 ? V4<C>::ld(K_u, L.off(c0 + 4 * qd, r0 - 1 + jj, 0))
                                   : V4<C>::ld(K_v, L.off(c0 + 4 * qd, r0 + jj, 0));
            } else if (it < NFQ) {
                const int e = it - 2 * (TY2 + 1) * 8, jj = e >> 1;
                d.kf1[u] = (e & 1) ? ld<float, C>(K_u, L.off(c0 + TX, r0 - 1 + jj, 0))
                                   : ld<float, C>(K_v, L.off(c0 - 1, r0 + jj, 0));
            }
        }
        }
        {
            const int64_t o = L.off(c0 + 4 * (l & 7), r0 + (l >> 3), 0);
            if constexpr (PAIR) {
                d.opa = __ldg(reinterpret_cast<const uint4*>(pac + o));
                d.opd = __ldg(reinterpret_cast<const uint4*>(pdc + o));
            } else {
                d.oac = V4<C>::ld(a_c, o);
                d.oan = V4<C>::ld(a_n, o);
                d.odc = V4<C>::ld(d_c, o);
                d.odn = V4<C>::ld(d_n, o);
            }
            if (MODE == MODE_RESID) {
#pragma unroll
                for (int f = 0; f < 3; ++f) d.ob[f] = __ldg(reinterpret_cast<const float4*>(b + f * S + o));
            }
        }
    };
    // staged quad at staged row jj, columns ii..ii+3 (ii = 1 + 4 qd)
    auto stage_quad = [&](int c0, int r0, int jj, int qd, float4 (&vx)[3], const float4 (&po)[3], const float4 ac,
                          const float4 an) {
        const int ii = 1 + 4 * qd;
        if (MODE == MODE_CG) {
#pragma unroll
            for (int f = 0; f < 3; ++f) {
                vx[f].x += beta * po[f].x; vx[f].y += beta * po[f].y;
                vx[f].z += beta * po[f].z; vx[f].w += beta * po[f].w;
            }
        }
        if (jj >= 1 && jj <= TY2) {
            if (MODE == MODE_CG) {
                const int64_t o = L.off(c0 + 4 * qd, r0 - 1 + jj, 0);
#pragma unroll
                for (int f = 0; f < 3; ++f) *reinterpret_cast<float4*>(pnew + f * S + o) = vx[f];
            }
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                sm.own[0][jj - 1][ii - 1 + i] = f4(vx[0], i);
                sm.own[1][jj - 1][ii - 1 + i] = f4(vx[1], i);
                sm.own[2][jj - 1][ii - 1 + i] = f4(vx[2], i);
            }
        }
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const float txx = f4(vx[0], i), txy = f4(vx[1], i), p = f4(vx[2], i);
            sm.U[jj][ii + i] = f4(ac, i) * (p - txx);
            sm.V[jj][ii + i] = f4(ac, i) * (p + txx);
            sm.N[jj][ii + i] = f4(an, i) * txy;
        }
    };
    Acc<float> acc;
    for (int k = blockIdx.x * 4 + g; k < ntiles; k += gridDim.x * 4) {
        const int tile = tiles ? tiles[k] : k;
        const int c0 = (tile % L.ntx) * TX, r0 = (tile / L.ntx) * TY2;
        // every global load of the tile is issued first: one memory round trip
        Loads d;
        load_tile(c0, r0, d);
        // 1. stage (p = z + beta p_old in CG mode)
        if constexpr (PAIR) stage_quad(c0, r0, l >> 3, l & 7, d.xa, d.pa, plo4(d.ppa), phi4(d.ppa));
        else stage_quad(c0, r0, l >> 3, l & 7, d.xa, d.pa, V4<C>::f(d.aca), V4<C>::f(d.ana));
        if (l < 16) {
            if constexpr (PAIR) stage_quad(c0, r0, 8 + (l >> 3), l & 7, d.xb, d.pb, plo4(d.ppb), phi4(d.ppb));
            else stage_quad(c0, r0, 8 + (l >> 3), l & 7, d.xb, d.pb, V4<C>::f(d.acb), V4<C>::f(d.anb));
        } else if (l < 16 + 2 * (TY2 + 2)) {
            const int e = l - 16, jj = e >> 1, ii = (e & 1) ? TX + 1 : 0;
            float v[3];
#pragma unroll
            for (int f = 0; f < 3; ++f) v[f] = MODE == MODE_CG ? d.xb[f].x + beta * d.pb[f].x : d.xb[f].x;
            const float hac = PAIR ? plo(d.hp) : d.hac, han = PAIR ? phi(d.hp) : d.han;
            sm.U[jj][ii] = hac * (v[2] - v[0]);
            sm.V[jj][ii] = hac * (v[2] + v[0]);
            sm.N[jj][ii] = han * v[1];
        }
        gsync();
        // 2. faces z_u (ii = 0..32 at columns c0 + ii) and z_v (ii = 0..32 at
        // columns c0 - 1 + ii), rows jj = 0..8: quads of four, and the one
        // face left over in each row (z_u: ii = 32; z_v: ii = 0)
        if constexpr (PAIR) {
#pragma unroll
            for (int u = 0; u < 2; ++u) {
                const int it = l + 64 * u;
                if (it < NKQ) {
                    const int jr = it >> 3, qd = it & 7;
                    if (jr <= TY2) {
                        const int jj = jr, ii = 4 * qd;
#pragma unroll
                        for (int i = 0; i < 4; ++i)
                            sm.Zu[jj][ii + i] = plo(u4(d.kq[u], i)) * ((sm.U[jj][ii + i + 1] - sm.U[jj][ii + i]) +
                                                                       (sm.N[jj][ii + i + 1] - sm.N[jj + 1][ii + i + 1]));
                    }
                    if (jr >= 1) {
                        const int jj = jr - 1, ii = 1 + 4 * qd;
#pragma unroll
                        for (int i = 0; i < 4; ++i)
                            sm.Zv[jj][ii + i] = phi(u4(d.kq[u], i)) * ((sm.V[jj + 1][ii + i] - sm.V[jj][ii + i]) +
                                                                       (sm.N[jj + 1][ii + i] - sm.N[jj + 1][ii + i + 1]));
                    }
                } else if (it < NKQ + 2 * (TY2 + 1)) {
                    const int e = it - NKQ, jj = e >> 1;
                    if (e & 1)
                        sm.Zu[jj][TX] = plo(d.ks) * ((sm.U[jj][TX + 1] - sm.U[jj][TX]) +
                                                     (sm.N[jj][TX + 1] - sm.N[jj + 1][TX + 1]));
                    else
                        sm.Zv[jj][0] = phi(d.ks) * ((sm.V[jj + 1][0] - sm.V[jj][0]) + (sm.N[jj + 1][0] - sm.N[jj + 1][1]));
                }
            }
        } else {
#pragma unroll
        for (int u = 0; u < 3; ++u) {
            const int it = l + 64 * u;
            if (it < 2 * (TY2 + 1) * 8) {
                const int dir = it / ((TY2 + 1) * 8), rem = it - dir * ((TY2 + 1) * 8), jj = rem >> 3, qd = rem & 7;
                const float4 k4 = V4<C>::f(d.kf[u]);
                if (dir == 0) {
                    const int ii = 4 * qd;
#pragma unroll
                    for (int i = 0; i < 4; ++i)
                        sm.Zu[jj][ii + i] = f4(k4, i) * ((sm.U[jj][ii + i + 1] - sm.U[jj][ii + i]) +
                                                         (sm.N[jj][ii + i + 1] - sm.N[jj + 1][ii + i + 1]));
                } else {
                    const int ii = 1 + 4 * qd;
#pragma unroll
                    for (int i = 0; i < 4; ++i)
                        sm.Zv[jj][ii + i] = f4(k4, i) * ((sm.V[jj + 1][ii + i] - sm.V[jj][ii + i]) +
                                                         (sm.N[jj + 1][ii + i] - sm.N[jj + 1][ii + i + 1]));
                }
            } else if (it < NFQ) {
                const int e = it - 2 * (TY2 + 1) * 8, jj = e >> 1;
                if (e & 1)
                    sm.Zu[jj][TX] = d.kf1[u] * ((sm.U[jj][TX + 1] - sm.U[jj][TX]) +
                                                (sm.N[jj][TX + 1] - sm.N[jj + 1][TX + 1]));
                else
                    sm.Zv[jj][0] = d.kf1[u] * ((sm.V[jj + 1][0] - sm.V[jj][0]) + (sm.N[jj + 1][0] - sm.N[jj + 1][1]));
            }
        }
        }
        gsync();
        // 3. y = C x + B z on the thread's own quad (row ty, columns 4 qd..4 qd+3)
        {
            const int ty = l >> 3, qd = l & 7;
            const int64_t o = L.off(c0 + 4 * qd, r0 + ty, 0);
            float yo[3][4];
            const float4 oac = PAIR ? plo4(d.opa) : V4<C>::f(d.oac), oan = PAIR ? phi4(d.opa) : V4<C>::f(d.oan);
            const float4 odc = PAIR ? plo4(d.opd) : V4<C>::f(d.odc), odn = PAIR ? phi4(d.opd) : V4<C>::f(d.odn);
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const int tx = 4 * qd + i;
                const float ac = f4(oac, i), an = f4(oan, i), dc = f4(odc, i), dn = f4(odn, i);
                const float txx = sm.own[0][ty][tx], txy = sm.own[1][ty][tx], p_ = sm.own[2][ty][tx];
                const float zu = sm.Zu[ty + 1][tx], zur = sm.Zu[ty + 1][tx + 1], zud = sm.Zu[ty][tx];
                const float zv = sm.Zv[ty][tx + 1], zvu = sm.Zv[ty + 1][tx + 1], zvl = sm.Zv[ty][tx];
                float yp, yxx;
                if (ac != 0.f) {
                    yp = ac * ((zu - zur) + (zv - zvu));
                    yxx = dc * txx + ac * ((zur - zu) + (zv - zvu));
                } else {
                    yp = p_;
                    yxx = txx;
                }
                float yxy = dn * txy + an * ((zu - zud) + (zv - zvl));
                if (MODE == MODE_RESID) {
                    yxx = f4(d.ob[0], i) - yxx; yxy = f4(d.ob[1], i) - yxy; yp = f4(d.ob[2], i) - yp;
                }
                yo[0][i] = yxx; yo[1][i] = yxy; yo[2][i] = yp;
                if (MODE == MODE_RESID) { acc.add(yxx, yxx); acc.add(yxy, yxy); acc.add(yp, yp); }
                else if (MODE == MODE_CG) { acc.add(txx, yxx); acc.add(txy, yxy); acc.add(p_, yp); }
            }
#pragma unroll
            for (int f = 0; f < 3; ++f)
                *reinterpret_cast<float4*>(y + f * S + o) = make_float4(yo[f][0], yo[f][1], yo[f][2], yo[f][3]);
        }
        gsync();                                 // the next tile's staging reuses the group's shared memory
    }
    if (MODE != MODE_PLAIN) {
        double v = acc.warp();
        if ((threadIdx.x & 31) != 0) v = 0.0;
        CgScalars* sc = args.sc;
        block_partial_and_finish<256>(v, args.partial, args.counter, gridDim.x, [&](double tot) {
            if (MODE == MODE_RESID) { sc->rr = tot; return; }
            sc->pq = tot;
            if (!(tot > 0.0) || !isfinite(tot)) { sc->done = 1; sc->status = (isfinite(tot) ? STOKES_ERR_BREAKDOWN : STOKES_ERR_NONFINITE); }
            else sc->alpha = sc->rz / tot;
        });
    }
}

// ------------------------------- 3D -----------------------------------------
// Staged helpers per slot (tile + halo):
//   Uc = a_c (p - txx), Vc = a_c (p - tyy), Wc = a_c (p + txx + tyy)
//   Nxy = a_xy txy, Nxz = a_xz txz, Nyz = a_yz tyz
// Face values:
//   z_u = K_u [Uc(c) - Uc(c-1) + Nxy(r) - Nxy(r+1) + Nxz(q) - Nxz(q+1)]
//   z_v = K_v [Vc(r) - Vc(r-1) + Nxy(c) - Nxy(c+1) + Nyz(q) - Nyz(q+1)]
//   z_w = K_w [Wc(q) - Wc(q-1) + Nxz(c) - Nxz(c+1) + Nyz(r) - Nyz(r+1)]
// Gather:
//   y_p   = a_c [z_u(c) - z_u(c+1) + z_v(r) - z_v(r+1) + z_w(q) - z_w(q+1)]
//   y_txx = d_c (txx + tyy/2) + a_c [z_u(c+1) - z_u(c) + z_w(q) - z_w(q+1)]
//   y_tyy = d_c (tyy + txx/2) + a_c [z_v(r+1) - z_v(r) + z_w(q) - z_w(q+1)]
//   y_txy = d_xy txy + a_xy [z_u(r) - z_u(r-1) + z_v(c) - z_v(c-1)]
//   y_txz = d_xz txz + a_xz [z_u(q) - z_u(q-1) + z_w(c) - z_w(c-1)]
//   y_tyz = d_yz tyz + a_yz [z_v(q) - z_v(q-1) + z_w(r) - z_w(r-1)]
//
// The kernel streams along z: a CTA (256 threads) owns a unit of 32 x 8
// slots and zt tile layers (16 planes; 4 where the active tiles are too few
// to fill the device with deep units) and walks its planes in order, keeping two staged
// planes (34 x 10 positions) and two planes of each face direction in
// shared memory.  Every staged value is loaded once per unit (halo 1.33x in
// x and y, 1.13x in z), against 2.4 staged positions per output for a
// 32 x 4 x 4 tile holding all its planes at once (FP32 on a 256^3 box: 0.63
// of the measured HBM bandwidth against 0.49).  Issuing a plane's own-value
// and coefficient loads before its staging (one memory round trip per
// plane, 64 registers, 4 CTAs per SM) measured 0.63 for FP32 and lost for
// BF16 coefficients (0.47 against 0.57) and FP64; 8 CTAs per SM at 32
// registers lost too (0.58).  For output plane q the step
//   1. stages plane q+1 (in CG mode p = z + beta p_old, written to p_new on
//      the unit's own slots of active tiles),
//   2. forms z_u(q), z_v(q) (staged planes q, q+1) and z_w(q+1) (planes q,
//      q+1),
//   3. writes y on plane q from z_u(q-1..q), z_v(q-1..q), z_w(q..q+1) and the
//      own values (re-read from p_new, or x), for slots of active tiles.
// (On the thin 3D liquid column the 16-plane units were too few: its apply
// ran slower than with 32 x 4 x 4 tiles until units of one layer were used
// for sparse grids.)
template <class T> struct Smem3 {
    static constexpr int SX = TX + 2, SY = UY3 + 2, NS = SX * SY;   // staged plane: 34 x 10
    static constexpr int FX = TX + 1, FY = UY3 + 1, NF = FX * FY;   // faces per plane: 33 x 9
    T st[2][6][NS];        // staged planes by parity: U, V, W, Nxy, Nxz, Nyz
    T fz[3][2][NF];        // z_u, z_v, z_w by plane parity
};

template <class T, class C, int MODE>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? 6 : 3) k_apply3d(Layout L, Coef<C> cf, const T* __restrict__ x,
                                                                          T* __restrict__ y, ApplyArgs args) {
    using SM = Smem3<T>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    SM& sm = *reinterpret_cast<SM*>(smem_raw);
    if (MODE == MODE_CG && args.sc->done) return;
    const int t = threadIdx.x;
    const int nuy = units_y(L.nty);
    const int u = args.units ? args.units[blockIdx.x] : blockIdx.x;
    const int zt = args.units ? args.zt : ZT_MAX;   // tile layers per unit
    unsigned mask;
    const int ux = u % L.ntx, urest = u / L.ntx, uy = urest % nuy, uz = urest / nuy;
    if (args.umask) {
        mask = args.umask[u];
    } else {                                  // every tile of the grid
        mask = 0;
        for (int dz = 0; dz < zt; ++dz)
            for (int dy = 0; dy < 2; ++dy)
                if (2 * uy + dy < L.nty && zt * uz + dz < L.ntz) mask |= 1u << (dy + 2 * dz);
    }
    const int c0 = ux * TX, r0 = uy * UY3, q0 = uz * zt * TZ3;
    const int64_t S = L.stride;
    const C *a_c = cf.f[0], *a_xy = cf.f[1], *a_xz = cf.f[2], *a_yz = cf.f[3];
    const C *d_c = cf.f[4], *d_xy = cf.f[5], *d_xz = cf.f[6], *d_yz = cf.f[7];
    const C *K_u = cf.f[8], *K_v = cf.f[9], *K_w = cf.f[10];
    // BF16: a slot's row weights and its diagonal from the arrays in fours
    // (one 8-byte load each), the face coefficients through L2 only (a warp's
    // 2-byte loads cover half of a 128-byte line)
    constexpr bool QD = sizeof(C) == 2;
    const uint2* __restrict__ qa = cf.qd[0];
    const uint2* __restrict__ qdg = cf.qd[1];
    auto ldk = [&](const C* p, int64_t o) -> T {
        if constexpr (QD) return T(__uint_as_float((uint32_t)__ldcg(reinterpret_cast<const unsigned short*>(p + o)) << 16));
        else return ld<T, C>(p, o);
    };
    const T* pold = (const T*)args.pold;
    T* pnew = (T*)args.pnew;
    const T beta = MODE == MODE_CG ? (T)args.sc->beta : T(0);
    // whether slot row r (padded) of plane q belongs to an active tile of the unit
    auto active = [&](int r, int q) -> bool {
        const int dy = (r - r0) / TY3, dz = (q - q0) / TZ3;
        return (mask >> (dy + 2 * dz)) & 1u;
    };
    // unknown fields: 0 txx, 1 tyy, 2 txy, 3 txz, 4 tyz, 5 p.  Staged rows past
    // the padded rows (row R is the next plane's pad row; later rows are only
    // read for the outputs and faces of inactive tile rows past the grid)
    // are zero, so every read stays inside the guards.
    auto stage = [&](int q) {
        T(*st)[SM::NS] = sm.st[q & 1];
        const bool own_plane = q >= q0 && q < q0 + zt * TZ3;
        for (int e = t; e < SM::NS; e += 256) {
            const int ii = e % SM::SX, jj = e / SM::SX;
            if (r0 - 1 + jj > L.R) {
#pragma unroll
                for (int f = 0; f < 6; ++f) st[f][e] = T(0);
                continue;
            }
            const int64_t o = L.off(c0 - 1 + ii, r0 - 1 + jj, q);
            T v[6];
#pragma unroll
            for (int f = 0; f < 6; ++f) v[f] = stage_val<T, MODE>(x + f * S, pold + f * S, beta, o);
            if (MODE == MODE_CG && own_plane && ii >= 1 && ii <= TX && jj >= 1 && jj <= UY3 &&
                active(r0 - 1 + jj, q)) {
#pragma unroll
                for (int f = 0; f < 6; ++f) pnew[f * S + o] = v[f];
            }
            T ac, axy, axz, ayz;
            if constexpr (QD) {
                const uint2 w = __ldg(qa + o);
                ac = T(plo(w.x)); axy = T(phi(w.x)); axz = T(plo(w.y)); ayz = T(phi(w.y));
            } else {
                ac = ld<T, C>(a_c, o); axy = ld<T, C>(a_xy, o); axz = ld<T, C>(a_xz, o); ayz = ld<T, C>(a_yz, o);
            }
            st[0][e] = ac * (v[5] - v[0]);
            st[1][e] = ac * (v[5] - v[1]);
            st[2][e] = ac * (v[5] + v[0] + v[1]);
            st[3][e] = axy * v[2];
            st[4][e] = axz * v[3];
            st[5][e] = ayz * v[4];
        }
    };
    // face coefficients of z_u(q), z_v(q), z_w(q+1) at face position e (zero
    // past the padded rows, see stage)
    constexpr int FPT = (SM::NF + 255) / 256;     // face positions per thread (2)
    auto face_k = [&](int q, T (&k)[FPT][3]) {
#pragma unroll
        for (int it = 0; it < FPT; ++it) {
            const int e = t + 256 * it;
            k[it][0] = k[it][1] = k[it][2] = T(0);
            if (e < SM::NF) {
                const int ii = e % SM::FX, jj = e / SM::FX;
                if (r0 + jj <= L.R) {
                    k[it][0] = ldk(K_u, L.off(c0 + ii, r0 - 1 + jj, q));
                    k[it][1] = ldk(K_v, L.off(c0 - 1 + ii, r0 + jj, q));
                    k[it][2] = ldk(K_w, L.off(c0 - 1 + ii, r0 - 1 + jj, q + 1));
                }
            }
        }
    };
    // z_u(q), z_v(q) from staged planes q and q+1; z_w(q+1) from planes q and q+1
    auto faces = [&](int q, const T (&k)[FPT][3]) {
        const T(*A)[SM::NS] = sm.st[q & 1];
        const T(*B)[SM::NS] = sm.st[(q + 1) & 1];
#pragma unroll
        for (int it = 0; it < FPT; ++it) {
            const int e = t + 256 * it;
            if (e >= SM::NF) break;
            const int ii = e % SM::FX, jj = e / SM::FX;
            if (r0 + jj > L.R) {
                sm.fz[0][q & 1][e] = sm.fz[1][q & 1][e] = sm.fz[2][(q + 1) & 1][e] = T(0);
                continue;
            }
            // z_u at (c0+ii, r0-1+jj, q): staged (ii+1, jj)
            const int su = jj * SM::SX + ii + 1;
            sm.fz[0][q & 1][e] = k[it][0] * ((A[0][su] - A[0][su - 1]) + (A[3][su] - A[3][su + SM::SX]) +
                                             (A[4][su] - B[4][su]));
            // z_v at (c0-1+ii, r0+jj, q): staged (ii, jj+1)
            const int sv = (jj + 1) * SM::SX + ii;
            sm.fz[1][q & 1][e] = k[it][1] * ((A[1][sv] - A[1][sv - SM::SX]) + (A[3][sv] - A[3][sv + 1]) +
                                             (A[5][sv] - B[5][sv]));
            // z_w at (c0-1+ii, r0-1+jj, q+1): staged (ii, jj) of planes q+1 and q
            const int sw = jj * SM::SX + ii;
            sm.fz[2][(q + 1) & 1][e] = k[it][2] * ((B[2][sw] - A[2][sw]) + (B[4][sw] - B[4][sw + 1]) +
                                                   (B[5][sw] - B[5][sw + SM::SX]));
        }
    };
    Acc<T> acc;
    // planes up to the last tile layer holding an active tile (all inside
    // the padded planes: staging reaches plane q_end <= Q, the trailing pad)
    int dz_end = 0;
    for (int dz = 0; dz < zt; ++dz)
        if ((mask >> (2 * dz)) & 3u) dz_end = dz + 1;
    const int q_end = q0 + TZ3 * dz_end;
    if (q_end > q0) {
    // prologue: planes q0-1 and q0; z_u(q0-1), z_v(q0-1); z_w(q0)
    stage(q0 - 1);
    stage(q0);
    __syncthreads();
    T k0[FPT][3];
    face_k(q0 - 1, k0);
    faces(q0 - 1, k0);
    __syncthreads();
    }
    const int tx = t & (TX - 1), ty = t >> 5;
    auto fi = [](int ii, int jj) { return jj * SM::FX + ii; };
    for (int q = q0; q < q_end; ++q) {
        stage(q + 1);
        __syncthreads();
        {
            T kq[FPT][3];
            face_k(q, kq);
            faces(q, kq);
        }
        __syncthreads();
        const int r = r0 + ty;
        if (active(r, q)) {
            const int64_t o = L.off(c0 + tx, r, q);
            T v[6];
#pragma unroll
            for (int f = 0; f < 6; ++f) v[f] = MODE == MODE_CG ? pnew[f * S + o] : x[f * S + o];
            const T* zu_q = sm.fz[0][q & 1];
            const T* zu_m = sm.fz[0][(q - 1) & 1];
            const T* zv_q = sm.fz[1][q & 1];
            const T* zv_m = sm.fz[1][(q - 1) & 1];
            const T* zw_q = sm.fz[2][q & 1];
            const T* zw_p = sm.fz[2][(q + 1) & 1];
            // z_u(c, r, q): face (tx, ty+1); z_v(c, r, q): (tx+1, ty); z_w(c, r, q): (tx+1, ty+1)
            const T zu = zu_q[fi(tx, ty + 1)], zu_cp = zu_q[fi(tx + 1, ty + 1)];
            const T zu_rm = zu_q[fi(tx, ty)], zu_qm = zu_m[fi(tx, ty + 1)];
            const T zv = zv_q[fi(tx + 1, ty)], zv_rp = zv_q[fi(tx + 1, ty + 1)];
            const T zv_cm = zv_q[fi(tx, ty)], zv_qm = zv_m[fi(tx + 1, ty)];
            const T zw = zw_q[fi(tx + 1, ty + 1)], zw_qp = zw_p[fi(tx + 1, ty + 1)];
            const T zw_cm = zw_q[fi(tx, ty + 1)], zw_rm = zw_q[fi(tx + 1, ty)];
            T ac, axy, axz, ayz, dc, dxy, dxz, dyz;
            if constexpr (QD) {
                const uint2 wa = __ldg(qa + o), wd = __ldg(qdg + o);
                ac = T(plo(wa.x)); axy = T(phi(wa.x)); axz = T(plo(wa.y)); ayz = T(phi(wa.y));
                dc = T(plo(wd.x)); dxy = T(phi(wd.x)); dxz = T(plo(wd.y)); dyz = T(phi(wd.y));
            } else {
                ac = ld<T, C>(a_c, o); axy = ld<T, C>(a_xy, o); axz = ld<T, C>(a_xz, o); ayz = ld<T, C>(a_yz, o);
                dc = ld<T, C>(d_c, o); dxy = ld<T, C>(d_xy, o); dxz = ld<T, C>(d_xz, o); dyz = ld<T, C>(d_yz, o);
            }
            T yv[6];
            if (ac != T(0)) {
                const T ww = zw - zw_qp;
                yv[5] = ac * ((zu - zu_cp) + (zv - zv_rp) + ww);
                yv[0] = dc * (v[0] + T(0.5) * v[1]) + ac * ((zu_cp - zu) + ww);
                yv[1] = dc * (v[1] + T(0.5) * v[0]) + ac * ((zv_rp - zv) + ww);
            } else {
                yv[5] = v[5]; yv[0] = v[0]; yv[1] = v[1];
            }
            yv[2] = dxy * v[2] + axy * ((zu - zu_rm) + (zv - zv_cm));
            yv[3] = dxz * v[3] + axz * ((zu - zu_qm) + (zw - zw_cm));
            yv[4] = dyz * v[4] + ayz * ((zv - zv_qm) + (zw - zw_rm));
            if (MODE == MODE_RESID) {
                const T* b = (const T*)args.b;
#pragma unroll
                for (int f = 0; f < 6; ++f) yv[f] = b[f * S + o] - yv[f];
            }
#pragma unroll
            for (int f = 0; f < 6; ++f) y[f * S + o] = yv[f];
            if (MODE == MODE_RESID) {
#pragma unroll
                for (int f = 0; f < 6; ++f) acc.add(yv[f], yv[f]);
            } else if (MODE == MODE_CG) {
#pragma unroll
                for (int f = 0; f < 6; ++f) acc.add(v[f], yv[f]);
            }
        }
        // the next step's staging overwrites the staged plane q (read by the
        // faces above, before the barrier); its faces overwrite z_u(q-1),
        // z_v(q-1) and z_w(q), read here: the barrier after its staging
        // orders them
    }
    if (MODE != MODE_PLAIN) {
        double v = acc.warp();
        if ((threadIdx.x & 31) != 0) v = 0.0;
        CgScalars* sc = args.sc;
        block_partial_and_finish<256>(v, args.partial, args.counter, gridDim.x, [&](double tot) {
            if (MODE == MODE_RESID) { sc->rr = tot; return; }
            sc->pq = tot;
            if (!(tot > 0.0) || !isfinite(tot)) { sc->done = 1; sc->status = (isfinite(tot) ? STOKES_ERR_BREAKDOWN : STOKES_ERR_NONFINITE); }
            else sc->alpha = sc->rz / tot;
        });
    }
}

// CTAs that fit on the device at once for a kernel (cached per device): the
// persistent kernels launch min(tiles, this) CTAs.
static int resident_ctas(const void* fn, int threads, size_t smem, int* cache) {
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 16) dev = 0;
    if (cache[dev] <= 0) {
        int sms = 0, per = 0;
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, fn, threads, smem);
        cache[dev] = std::max(1, sms) * std::max(1, per);
    }
    return cache[dev];
}

template <class T, class C, int MODE>
static cudaError_t launch_mode(const Layout& L, const int* tiles, int ntiles, const Coef<C>& cf, const T* x, T* y,
                               const ApplyArgs& a, cudaStream_t s) {
    if (ntiles <= 0) return cudaSuccess;
    static int cache2[16], cache3[16];
    if (L.dim == 2) {
        // FP64 vectors: one slot per thread, software-pipelined over the tiles
        // (bound by the FP64 pipe; the unconstrained build is faster)
        // FP32 vectors: four slots per thread, four tiles per CTA, 16-byte
        // loads and stores of the vectors, which callers' arrays (a view at
        // an odd offset) need not allow: those take one slot per thread
        const bool aligned = (((uintptr_t)x | (uintptr_t)y | (uintptr_t)a.pold | (uintptr_t)a.pnew |
                               (uintptr_t)a.b) & 15u) == 0;
        if constexpr (sizeof(T) == 4) {
            if (aligned && (sizeof(C) == 4 || cf.pr[0])) {
                const int grid =
                    std::min((ntiles + 3) / 4, resident_ctas((const void*)k_apply2d_v4<C, MODE>, 256, 0, cache2));
                k_apply2d_v4<C, MODE><<<grid, 256, 0, s>>>(L, tiles, cf, x, y, a, ntiles);
            } else {
                static int cache1[16];
                constexpr int MINB = sizeof(C) == 2 ? 5 : 4;
                const int grid =
                    std::min(ntiles, resident_ctas((const void*)k_apply2d<T, C, MODE, MINB>, 256, 0, cache1));
                k_apply2d<T, C, MODE, MINB><<<grid, 256, 0, s>>>(L, tiles, cf, x, y, a, ntiles);
            }
        } else {
            constexpr int MINB = 1;
            const int grid = std::min(ntiles, resident_ctas((const void*)k_apply2d<T, C, MODE, MINB>, 256, 0, cache2));
            k_apply2d<T, C, MODE, MINB><<<grid, 256, 0, s>>>(L, tiles, cf, x, y, a, ntiles);
        }
    } else {
        // 3D: one CTA per unit (32 x 8 slots, 16 planes), over the active
        // units (an apply over the active tiles needs the unit list) or all
        (void)cache3;
        if (tiles && !a.units) return cudaErrorInvalidValue;
        if (sizeof(C) == 2 && !cf.qd[0]) return cudaErrorInvalidValue;   // BF16 reads the arrays in fours
        const int nu = tiles ? a.nunits : L.ntx * units_y(L.nty) * units_z(L.ntz, ZT_MAX);
        if (nu > 0) k_apply3d<T, C, MODE><<<nu, 256, sizeof(Smem3<T>), s>>>(L, cf, x, y, a);
    }
    return cudaGetLastError();
}

template <class T, class C>
cudaError_t launch_apply_mode(const Layout& L, const int* tiles, int ntiles, const Coef<C>& cf, const T* x, T* y,
                              int mode, const ApplyArgs& a, cudaStream_t s) {
    switch (mode) {
        case MODE_PLAIN: return launch_mode<T, C, MODE_PLAIN>(L, tiles, ntiles, cf, x, y, a, s);
        case MODE_RESID: return launch_mode<T, C, MODE_RESID>(L, tiles, ntiles, cf, x, y, a, s);
        default: return launch_mode<T, C, MODE_CG>(L, tiles, ntiles, cf, x, y, a, s);
    }
}

template <class T, class C>
static void set_attr3() {
    int sm = (int)sizeof(Smem3<T>);
    cudaFuncSetAttribute(k_apply3d<T, C, MODE_PLAIN>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
    cudaFuncSetAttribute(k_apply3d<T, C, MODE_RESID>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
    cudaFuncSetAttribute(k_apply3d<T, C, MODE_CG>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
}

// Opt the 3D kernels into more than 48 KB of dynamic shared memory (once per
// process and device, before any launch or graph capture).
void apply_set_attributes() {
    set_attr3<double, double>();
    set_attr3<float, float>();
    set_attr3<float, __nv_bfloat16>();
}

template cudaError_t launch_apply_mode<double, double>(const Layout&, const int*, int, const Coef<double>&,
                                                       const double*, double*, int, const ApplyArgs&, cudaStream_t);
template cudaError_t launch_apply_mode<float, float>(const Layout&, const int*, int, const Coef<float>&, const float*,
                                                     float*, int, const ApplyArgs&, cudaStream_t);
template cudaError_t launch_apply_mode<float, __nv_bfloat16>(const Layout&, const int*, int,
                                                             const Coef<__nv_bfloat16>&, const float*, float*, int,
                                                             const ApplyArgs&, cudaStream_t);

}  // namespace stk
