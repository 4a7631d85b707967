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
            const T ac = ld<T, C>(a_c, o);
            st[0][e] = ac * (v[5] - v[0]);
            st[1][e] = ac * (v[5] - v[1]);
            st[2][e] = ac * (v[5] + v[0] + v[1]);
            st[3][e] = ld<T, C>(a_xy, o) * v[2];
            st[4][e] = ld<T, C>(a_xz, o) * v[3];
            st[5][e] = ld<T, C>(a_yz, o) * v[4];
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
                    k[it][0] = ld<T, C>(K_u, L.off(c0 + ii, r0 - 1 + jj, q));
                    k[it][1] = ld<T, C>(K_v, L.off(c0 - 1 + ii, r0 + jj, q));
                    k[it][2] = ld<T, C>(K_w, L.off(c0 - 1 + ii, r0 - 1 + jj, q + 1));
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
            const T ac = ld<T, C>(a_c, o), dc = ld<T, C>(d_c, o);
            T yv[6];
            if (ac != T(0)) {
                const T ww = zw - zw_qp;
                yv[5] = ac * ((zu - zu_cp) + (zv - zv_rp) + ww);
                yv[0] = dc * (v[0] + T(0.5) * v[1]) + ac * ((zu_cp - zu) + ww);
                yv[1] = dc * (v[1] + T(0.5) * v[0]) + ac * ((zv_rp - zv) + ww);
            } else {
                yv[5] = v[5]; yv[0] = v[0]; yv[1] = v[1];
            }
            yv[2] = ld<T, C>(d_xy, o) * v[2] + ld<T, C>(a_xy, o) * ((zu - zu_rm) + (zv - zv_cm));
            yv[3] = ld<T, C>(d_xz, o) * v[3] + ld<T, C>(a_xz, o) * ((zu - zu_qm) + (zw - zw_cm));
            yv[4] = ld<T, C>(d_yz, o) * v[4] + ld<T, C>(a_yz, o) * ((zv - zv_qm) + (zw - zw_rm));
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
        // FP32 vectors: at most 64 registers, four CTAs per SM (measured 70% of
        // HBM at 4096^2, against 54% with 96 registers and three CTAs, 67% with
        // five); BF16 coefficients: five CTAs per SM (44% against 38% with
        // four); FP64 is bound by the FP64 pipe, where the unconstrained build
        // is faster
        constexpr int MINB = sizeof(C) == 2 ? 5 : (sizeof(T) == 4 ? 4 : 1);
        const int grid = std::min(ntiles, resident_ctas((const void*)k_apply2d<T, C, MODE, MINB>, 256, 0, cache2));
        k_apply2d<T, C, MODE, MINB><<<grid, 256, 0, s>>>(L, tiles, cf, x, y, a, ntiles);
    } else {
        // 3D: one CTA per unit (32 x 8 slots, 16 planes), over the active
        // units (an apply over the active tiles needs the unit list) or all
        (void)cache3;
        if (tiles && !a.units) return cudaErrorInvalidValue;
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
