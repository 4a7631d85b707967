// Preconditioned conjugate gradients on the SPD pressure-stress system and
// the FP64 iterative-refinement driver around it.
//
// Inner solve (precision T of the vectors, C of the coefficients), Jacobi
// preconditioner M^-1 = diag(A)^-1:
//   init      r = T(scale * r64), z = M^-1 r, x = 0, p_old = 0, rho = r.z
//   iterate   [apply, CG mode]  p = z + beta p_old, q = A p, alpha = rho / p.q
//             [update]          x += alpha p, r -= alpha q, z = M^-1 r,
//                               rho' = r.z, beta = rho'/rho, stop on r.r <= tol2
// The loop runs on the device as a CUDA graph with a conditional while node
// whose condition the update kernel clears when the solve is done, so the
// host is involved once per inner solve.
//
// Outer loop (FP64): x64 += d / scale, r64 = b - A64 x64 recomputed from
// scratch with the FP64 operator; stop when ||r64|| <= tol ||b||.  In FP64
// mode the inner solve is FP64 CG and normally one outer step suffices.
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>
#include "internal.cuh"
#include "ctx.cuh"

namespace stk {

cudaError_t run_inner_fpcg(Ctx* c, stokes_net_s* net, double scale, double tol_rel, int max_iter, int* iters,
                           int* jacobi_steps);

// Walk the slots of one tile: 2D 8 rows of 32, 3D 16 rows of 32.
__device__ __forceinline__ int tile_rows(const Layout& L) { return L.dim == 2 ? TY2 : TY3 * TZ3; }

__device__ __forceinline__ int64_t tile_row_off(const Layout& L, int tile, int row) {
    int tcx = tile % L.ntx;
    if (L.dim == 2) {
        int tr = tile / L.ntx;
        return L.off(tcx * TX, tr * TY2 + row, 0);
    }
    int rest = tile / L.ntx;
    int tr = rest % L.nty, tq = rest / L.nty;
    return L.off(tcx * TX, tr * TY3 + row % TY3, tq * TZ3 + row / TY3);
}

template <class T> struct AccT;
template <> struct AccT<double> {
    double s = 0.0;
    __device__ void add(double a, double b) { s = fma(a, b, s); }
    __device__ double warp() { return warp_sum(s); }
};
template <> struct AccT<float> {
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

// Two partial sums per block; the last block to finish reduces both.
template <class Fin>
__device__ void block_partial2(double v0, double v1, double* partial, unsigned* counter, int nblocks, Fin fin) {
    __shared__ double red[2][8];
    __shared__ bool last;
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) { red[0][w] = v0; red[1][w] = v1; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double s0 = 0.0, s1 = 0.0;
        for (int q = 0; q < 8; ++q) { s0 += red[0][q]; s1 += red[1][q]; }
        partial[2 * blockIdx.x] = s0;
        partial[2 * blockIdx.x + 1] = s1;
        __threadfence();
        unsigned prev = atomicAdd(counter, 1u);
        last = (prev == (unsigned)nblocks - 1u);
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    double s0 = 0.0, s1 = 0.0;
    for (int b = threadIdx.x; b < nblocks; b += 256) {
        s0 += ((volatile double*)partial)[2 * b];
        s1 += ((volatile double*)partial)[2 * b + 1];
    }
    s0 = warp_sum(s0);
    s1 = warp_sum(s1);
    __syncthreads();
    if (lane == 0) { red[0][w] = s0; red[1][w] = s1; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double t0 = 0.0, t1 = 0.0;
        for (int q = 0; q < 8; ++q) { t0 += red[0][q]; t1 += red[1][q]; }
        fin(t0, t1);
        *counter = 0u;
    }
}

// init: r = T(scale * r64), z = minv r, x = 0, p0 = 0; rho = r.z, rr0 = r.r
template <class T>
__global__ void __launch_bounds__(256) k_cg_init(Layout L, const int* __restrict__ tiles, int nf, const double* r64,
                                                 const T* __restrict__ minv, CgWork<T> w, CgScalars* sc,
                                                 double* partial, unsigned* counter, int nblocks,
                                                 cudaGraphConditionalHandle h, int use_cond) {
    const int tile = tiles[blockIdx.x];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const T scale = (T)sc->scale;
    AccT<T> rz, rr;
    const int nrow = tile_rows(L);
    for (int row = warp; row < nrow; row += 8) {
        int64_t o = tile_row_off(L, tile, row) + lane;
        for (int f = 0; f < nf; ++f) {
            int64_t of = (int64_t)f * L.stride + o;
            T r = (T)(r64[of] * (double)scale);
            T z = minv[of] * r;
            w.r[of] = r; w.z[of] = z; w.x[of] = T(0); w.p[0][of] = T(0);
            rz.add(r, z); rr.add(r, r);
        }
    }
    double a = rz.warp(), b = rr.warp();
    block_partial2(a, b, partial, counter, nblocks, [&](double trz, double trr) {
        sc->rz = trz; sc->rr = trr; sc->rr0 = trr;
        sc->tol2 = sc->tol_rel * sc->tol_rel * trr;
        sc->beta = 0.0; sc->iter = 0; sc->status = 0;
        sc->done = (trr <= sc->tol2 || trr == 0.0) ? 1 : 0;
        if (!isfinite(trr)) { sc->done = 1; sc->status = STOKES_ERR_NONFINITE; }
        if (use_cond) cudaGraphSetConditional(h, sc->done ? 0u : 1u);
    });
}

// update: x += alpha p, r -= alpha q, z = minv r; rho' = r.z, r.r
template <class T>
__global__ void __launch_bounds__(256) k_cg_update(Layout L, const int* __restrict__ tiles, int nf,
                                                   const T* __restrict__ minv, CgWork<T> w, const T* __restrict__ p,
                                                   CgScalars* sc, double* partial, unsigned* counter, int ntiles,
                                                   cudaGraphConditionalHandle h, int use_cond) {
    if (sc->done) {
        if (use_cond && blockIdx.x == 0 && threadIdx.x == 0) cudaGraphSetConditional(h, 0u);
        return;
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const T alpha = (T)sc->alpha;
    AccT<T> rz, rr;
    const int nrow = tile_rows(L);
    T* __restrict__ X = w.x;
    T* __restrict__ Rr = w.r;
    T* __restrict__ Z = w.z;
    const T* __restrict__ Q = w.q;
    // persistent over the tile list: one block reduction per CTA
    for (int k = blockIdx.x; k < ntiles; k += gridDim.x) {
    const int tile = tiles[k];
    for (int row = warp; row < nrow; row += 8) {
        const int64_t o = tile_row_off(L, tile, row) + lane;
        // issue every load of the slot's fields before any store
        T pv[6], xv[6], rv[6], qv[6], mv[6];
#pragma unroll
        for (int f = 0; f < 6; ++f) {
            if (f < nf) {
                const int64_t of = (int64_t)f * L.stride + o;
                pv[f] = __ldg(p + of); xv[f] = X[of]; rv[f] = Rr[of]; qv[f] = __ldg(Q + of); mv[f] = __ldg(minv + of);
            }
        }
#pragma unroll
        for (int f = 0; f < 6; ++f) {
            if (f < nf) {
                const int64_t of = (int64_t)f * L.stride + o;
                T r = rv[f] - alpha * qv[f];
                T z = mv[f] * r;
                X[of] = xv[f] + alpha * pv[f];
                Rr[of] = r; Z[of] = z;
                rz.add(r, z); rr.add(r, r);
            }
        }
    }
    }
    double a = rz.warp(), b = rr.warp();
    block_partial2(a, b, partial, counter, gridDim.x, [&](double trz, double trr) {
        sc->rr = trr;
        sc->iter += 1;
        if (!isfinite(trr) || !isfinite(trz)) { sc->done = 1; sc->status = STOKES_ERR_NONFINITE; }
        else if (trr <= sc->tol2) { sc->done = 1; }
        else if (!(trz > 0.0)) { sc->done = 1; sc->status = STOKES_ERR_BREAKDOWN; }
        else if (sc->iter >= sc->max_iter) { sc->done = 1; sc->status = STOKES_ERR_NOT_CONVERGED; }
        sc->beta = trz / sc->rz;
        sc->rz = trz;
        if (use_cond) cudaGraphSetConditional(h, sc->done ? 0u : 1u);
    });
}

}  // namespace stk
#include "schwarz.cuh"
namespace stk {

__global__ void k_jacobi_apply(int64_t n, const float* r, const float* minv, float* z) {
    int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e < n) z[e] = minv[e] * r[e];
}

// Schwarz-preconditioned CG (2D, FP32 vectors).  init: r = scale r64, x = 0,
// p_old = 0 (z follows from the patch solves); finish: gather z, r.z, r.r and
// the CG bookkeeping (INIT: start values; else as in k_cg_update).
__global__ void __launch_bounds__(256) k_sw_init(Layout L, const int* __restrict__ tiles, const double* r64,
                                                 CgWork<float> w, const CgScalars* sc) {
    const int tile = tiles[blockIdx.x];
    const int c0 = (tile % L.ntx) * TX, r0 = (tile / L.ntx) * TY2;
    const int64_t o = L.off(c0 + (threadIdx.x & 31), r0 + (threadIdx.x >> 5), 0);
    const double scale = sc->scale;
    for (int f = 0; f < 3; ++f) {
        const int64_t of = (int64_t)f * L.stride + o;
        w.r[of] = (float)(r64[of] * scale);
        w.x[of] = 0.f;
        w.p[0][of] = 0.f;
    }
}

// (five CTAs share an SM, each taking two tiles per round, so up to 1,520
// active tiles are one wave; the dots are float-float, not FP64, whose
// arithmetic is slow on this part).  UPD: the CG step's x += alpha p,
// r -= alpha q is done here for every slot of the tile (the local solves
// read r - alpha q), so no separate update kernel runs.
template <int INIT, int UPD = 0>
__global__ void __launch_bounds__(256, UPD ? 3 : 5) k_sw_finish(Layout L, const int* __restrict__ tiles, DevArrays D,
                                                   SchwarzPlan P, CgWork<float> w, CgScalars* sc, double* partial,
                                                   unsigned* counter, int ntiles, cudaGraphConditionalHandle h,
                                                   int use_cond, const float* __restrict__ pdir = nullptr) {
    if (!INIT && sc->done) {
        if (use_cond && blockIdx.x == 0 && threadIdx.x == 0) cudaGraphSetConditional(h, 0u);
        return;
    }
    AccT<float> rz, rr;
    // persistent over the tile list, two tiles per round (tile k and tile
    // k + gridDim.x): the loads of both slots are issued before either is
    // summed; one block reduction per CTA
    for (int k = blockIdx.x; k < ntiles; k += 2 * gridDim.x) {
        const int k2 = k + gridDim.x;
        SwGather g0, g1;
        SwUpdate u0, u1;
        const int t0 = tiles[k];
        sw_gather_load(L, D, P, w.r, (t0 % L.ntx) * TX + (threadIdx.x & 31), (t0 / L.ntx) * TY2 + (threadIdx.x >> 5),
                       g0);
        if (UPD) sw_update_load(L, w, pdir, g0.o, u0);
        if (k2 < ntiles) {
            const int t1 = tiles[k2];
            sw_gather_load(L, D, P, w.r, (t1 % L.ntx) * TX + (threadIdx.x & 31),
                           (t1 / L.ntx) * TY2 + (threadIdx.x >> 5), g1);
            if (UPD) sw_update_load(L, w, pdir, g1.o, u1);
        }
        const float alpha = UPD ? (float)sc->alpha : 0.f;
        sw_gather_finish(L, g0, w.z, rz, rr, UPD ? &u0 : nullptr, alpha, w.r, w.x);
        if (k2 < ntiles) sw_gather_finish(L, g1, w.z, rz, rr, UPD ? &u1 : nullptr, alpha, w.r, w.x);
    }
    block_partial2(rz.warp(), rr.warp(), partial, counter, gridDim.x, [&](double trz, double trr) {
        if (INIT) {
            const bool timed_out = sc->status == STOKES_ERR_TIMEOUT;   // set by a local solve
            sc->rz = trz; sc->rr = trr; sc->rr0 = trr;
            sc->tol2 = sc->tol_rel * sc->tol_rel * trr;
            sc->beta = 0.0; sc->iter = 0; sc->status = 0;
            sc->done = (trr <= sc->tol2 || trr == 0.0) ? 1 : 0;
            if (!isfinite(trr)) { sc->done = 1; sc->status = STOKES_ERR_NONFINITE; }
            if (timed_out) { sc->done = 1; sc->status = STOKES_ERR_TIMEOUT; }
        } else {
            sc->rr = trr;
            sc->iter += 1;
            if (!isfinite(trr) || !isfinite(trz)) { sc->done = 1; sc->status = STOKES_ERR_NONFINITE; }
            else if (trr <= sc->tol2) { sc->done = 1; }
            else if (!(trz > 0.0)) { sc->done = 1; sc->status = STOKES_ERR_BREAKDOWN; }
            else if (sc->iter >= sc->max_iter) { sc->done = 1; sc->status = STOKES_ERR_NOT_CONVERGED; }
            sc->beta = trz / sc->rz;
            sc->rz = trz;
        }
        if (use_cond) cudaGraphSetConditional(h, sc->done ? 0u : 1u);
    });
}

// Patch plan and local inverses (after every weight build, on first use).
static cudaError_t schwarz_build(Ctx* c) {
    const Layout& L = c->L;
    cudaError_t e;
    for (void* p : c->sw_allocs) cudaFree(p);
    c->sw_allocs.clear();
    ++c->sw_epoch;
    if (!c->sw) c->sw = new SchwarzPlan();
    SchwarzPlan& P = *c->sw;
    P.npx = (L.nx + 1 + PB - 1) / PB;
    P.npy = (L.ny + 1 + PB - 1) / PB;
    const int ng = P.npx * P.npy;
    auto al = [&](void** p, size_t bytes) -> cudaError_t {
        cudaError_t r = cudaMalloc(p, bytes ? bytes : 16);
        if (r == cudaSuccess) c->sw_allocs.push_back(*p);
        return r;
    };
    int* dflag = nullptr;
    if ((e = al((void**)&dflag, sizeof(int) * ng)) != cudaSuccess) return e;
    k_schwarz_mark<<<dim3((P.npx + 127) / 128, P.npy), 128, 0, c->stream>>>(L, c->A, P.npx, P.npy, dflag);
    std::vector<int> flag(ng), pid(ng, -1), corner;
    if ((e = cudaMemcpyAsync(flag.data(), dflag, sizeof(int) * ng, cudaMemcpyDeviceToHost, c->stream)) != cudaSuccess)
        return e;
    if ((e = cudaStreamSynchronize(c->stream)) != cudaSuccess) return e;
    for (int J = 0; J < P.npy; ++J)
        for (int I = 0; I < P.npx; ++I)
            if (flag[J * P.npx + I]) { pid[J * P.npx + I] = (int)corner.size(); corner.push_back(I | (J << 16)); }
    P.np = (int)corner.size();
    P.evict_first = sw_factors_exceed_l2((size_t)P.np * SW_FAC_BYTES) ? 1 : 0;
    const size_t np = std::max(1, P.np);
    if ((e = al((void**)&P.pid, sizeof(int) * ng)) != cudaSuccess) return e;
    if ((e = al((void**)&P.corner, sizeof(int) * np)) != cudaSuccess) return e;
    if ((e = al((void**)&P.nloc, sizeof(int) * np)) != cudaSuccess) return e;
    if ((e = al((void**)&P.lmap, sizeof(short) * np * PMAX)) != cudaSuccess) return e;
    // FP16 factors with a FP32 scale per row (BF16 storage needed 4.4x the CG
    // iterations on the 1024^2 bump workload; FP16 about 1.02x)
    if ((e = al((void**)&P.fac, (size_t)SW_FAC_BYTES * np)) != cudaSuccess) return e;
    if ((e = al((void**)&P.scale, sizeof(float) * np * PMAX)) != cudaSuccess) return e;
    if ((e = al((void**)&P.ybuf, sizeof(float) * ng * PMAX)) != cudaSuccess) return e;
    cudaMemcpyAsync(P.pid, pid.data(), sizeof(int) * ng, cudaMemcpyHostToDevice, c->stream);
    if (P.np) cudaMemcpyAsync(P.corner, corner.data(), sizeof(int) * P.np, cudaMemcpyHostToDevice, c->stream);
    cudaMemsetAsync(P.ybuf, 0, sizeof(float) * ng * PMAX, c->stream);
    const int smem = SW_SETUP_SMEM;
    cudaFuncSetAttribute(k_schwarz_setup, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    cudaFuncSetAttribute(k_schwarz_gemv, cudaFuncAttributeMaxDynamicSharedMemorySize, SW_GEMV_SMEM);
    cudaEvent_t a, b;
    cudaEventCreate(&a); cudaEventCreate(&b);
    cudaEventRecord(a, c->stream);
    if (P.np) k_schwarz_setup<<<P.np, 256, smem, c->stream>>>(L, c->A, c->A.coef64, P);
    cudaEventRecord(b, c->stream);
    if ((e = cudaEventSynchronize(b)) != cudaSuccess) return e;
    float ms = 0;
    cudaEventElapsedTime(&ms, a, b);
    cudaEventDestroy(a); cudaEventDestroy(b);
    c->sw_setup_ms = ms;
    c->sw_ready = true;
    return cudaGetLastError();
}

// CTAs of a persistent tile kernel: min(tiles, the CTAs resident on the
// device at once), cached per kernel.
static int persist_grid(const void* fn, int ntiles, size_t smem = 0) {
    static std::mutex mu;
    static std::vector<std::pair<const void*, int>> cache;
    int res = 0;
    {
        std::lock_guard<std::mutex> g(mu);
        for (auto& kv : cache)
            if (kv.first == fn) res = kv.second;
        if (!res) {
            int dev = 0, sms = 0, per = 0;
            cudaGetDevice(&dev);
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, fn, 256, smem);
            res = std::max(1, sms) * std::max(1, per);
            cache.push_back({fn, res});
        }
    }
    return std::max(1, std::min(ntiles, res));
}

static void schwarz_body(Ctx* c, cudaStream_t s, cudaGraphConditionalHandle h, int use_cond, int parity) {
    const Layout& L = c->L;
    const int nb = c->ntiles_active;
    CgWork<float>& w = c->w32;
    ApplyArgs a = c->apply_args();
    a.pold = w.p[parity];
    a.pnew = w.p[parity ^ 1];
    a.partial = c->partial;
    a.counter = c->counter;
    a.sc = c->sc;
    launch_apply_mode<float, float>(L, c->tiles, nb, c->coef<float>(), w.z, w.q, MODE_CG, a, s);
    // the step's x += alpha p, r -= alpha q: the local solves read r - alpha q
    // and the gather writes both for every slot
    launch_schwarz_gemv(L, *c->sw, w.r, c->sc, s, w.q);
    k_sw_finish<0, 1><<<persist_grid((const void*)k_sw_finish<0, 1>, (nb + 1) / 2), 256, 0, s>>>(
        L, c->tiles, c->A, *c->sw, w, c->sc, c->partial, c->counter, nb, h, use_cond, w.p[parity ^ 1]);
}

static void schwarz_start(Ctx* c, cudaStream_t s, cudaGraphConditionalHandle h, int use_cond) {
    const Layout& L = c->L;
    const int nb = c->ntiles_active;
    CgWork<float>& w = c->w32;
    k_sw_init<<<nb, 256, 0, s>>>(L, c->tiles, c->w64.r, w, c->sc);
    launch_schwarz_gemv(L, *c->sw, w.r, c->sc, s);
    k_sw_finish<1><<<persist_grid((const void*)k_sw_finish<1>, (nb + 1) / 2), 256, 0, s>>>(L, c->tiles, c->A, *c->sw, w, c->sc,
                                                                               c->partial, c->counter, nb, h, use_cond);
}

// x64 += sign * d / scale (refinement update; sign = -1 undoes it), over active tiles
template <class T>
__global__ void __launch_bounds__(256) k_ir_update(Layout L, const int* __restrict__ tiles, int nf, double* x64,
                                                   const T* __restrict__ d, const CgScalars* sc, double sign) {
    const int tile = tiles[blockIdx.x];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const double inv = sign / sc->scale;
    const int nrow = tile_rows(L);
    for (int row = warp; row < nrow; row += 8) {
        int64_t o = tile_row_off(L, tile, row) + lane;
        for (int f = 0; f < nf; ++f) {
            int64_t of = (int64_t)f * L.stride + o;
            x64[of] += (double)d[of] * inv;
        }
    }
}

// r64 = b, x64 = 0 over active tiles; rr = b.b (FP64)
__global__ void __launch_bounds__(256) k_outer_init(Layout L, const int* __restrict__ tiles, int nf, const double* b,
                                                    double* x64, double* r64, CgScalars* so, double* partial,
                                                    unsigned* counter, int nblocks) {
    const int tile = tiles[blockIdx.x];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    double s = 0.0;
    const int nrow = tile_rows(L);
    for (int row = warp; row < nrow; row += 8) {
        int64_t o = tile_row_off(L, tile, row) + lane;
        for (int f = 0; f < nf; ++f) {
            int64_t of = (int64_t)f * L.stride + o;
            double v = b[of];
            r64[of] = v; x64[of] = 0.0;
            s = fma(v, v, s);
        }
    }
    double a = warp_sum(s);
    block_partial2(a, 0.0, partial, counter, nblocks, [&](double t0, double) {
        so->rr = t0; so->rr0 = t0; so->iter = 0; so->status = 0; so->done = 0;
    });
}

// Build the inner-solve graph for one precision: init kernel, then a
// conditional while node whose body runs two CG iterations (the search
// direction alternates between p[0] and p[1]).
template <class T, class C>
static cudaError_t build_inner_graph(Ctx* c, CgWork<T>& w, const T* minv, const Coef<C>& cf, CgScalars* sc,
                                     cudaGraphExec_t* out) {
    const Layout& L = c->L;
    cudaStream_t s = c->stream;
    const int nb = c->ntiles_active;
    double* part = c->partial;
    unsigned* cnt = c->counter;
    cudaError_t e;
    cudaGraph_t g = nullptr;
    if ((e = cudaGraphCreate(&g, 0)) != cudaSuccess) return e;
    cudaGraphConditionalHandle h;
    if ((e = cudaGraphConditionalHandleCreate(&h, g, 1u, cudaGraphCondAssignDefault)) != cudaSuccess) return e;
    // init node by capture into g
    if ((e = cudaStreamBeginCaptureToGraph(s, g, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed)) != cudaSuccess)
        return e;
    k_cg_init<T><<<nb, 256, 0, s>>>(L, c->tiles, c->nf, c->w64.r, minv, w, sc, part, cnt, nb, h, 1);
    cudaGraph_t captured = nullptr;
    if ((e = cudaStreamEndCapture(s, &captured)) != cudaSuccess) return e;
    // find the init node (the graph's only node so far)
    size_t nn = 0;
    cudaGraphGetNodes(g, nullptr, &nn);
    std::vector<cudaGraphNode_t> nodes(nn);
    cudaGraphGetNodes(g, nodes.data(), &nn);
    cudaGraphNodeParams cp = {};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = h;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    cudaGraphNode_t cond;
    if ((e = cudaGraphAddNode(&cond, g, nodes.data(), nullptr, nn, &cp)) != cudaSuccess) return e;
    cudaGraph_t body = cp.conditional.phGraph_out[0];
    if ((e = cudaStreamBeginCaptureToGraph(s, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed)) != cudaSuccess)
        return e;
    for (int k = 0; k < 2; ++k) {
        ApplyArgs a = c->apply_args();
        a.pold = w.p[k];
        a.pnew = w.p[k ^ 1];
        a.partial = part;
        a.counter = cnt;
        a.sc = sc;
        launch_apply_mode<T, C>(L, c->tiles, nb, cf, w.z, w.q, MODE_CG, a, s);
        k_cg_update<T><<<persist_grid((const void*)k_cg_update<T>, nb), 256, 0, s>>>(L, c->tiles, c->nf, minv, w,
                                                                                   w.p[k ^ 1], sc, part, cnt, nb, h, 1);
    }
    cudaGraph_t cap2 = nullptr;
    if ((e = cudaStreamEndCapture(s, &cap2)) != cudaSuccess) return e;
    e = cudaGraphInstantiate(out, g, 0);
    cudaGraphDestroy(g);
    return e;
}

static cudaError_t fetch_scalars(Ctx* c) {
    cudaError_t e = cudaMemcpyAsync(c->h_sc, c->sc, 2 * sizeof(CgScalars), cudaMemcpyDeviceToHost, c->stream);
    if (e != cudaSuccess) return e;
    return cudaStreamSynchronize(c->stream);
}

// One inner solve.  use_graph: the device-side graph (one launch); else
// chunks of ``chunk`` iterations launched kernel by kernel, the host reading
// the done flag between chunks (kernels after "done" return at once).
template <class T, class C>
static cudaError_t run_inner(Ctx* c, int prec_slot, CgWork<T>& w, const T* minv, const Coef<C>& cf, int use_graph,
                             int chunk) {
    cudaError_t e;
    if (use_graph) {
        cudaGraphExec_t& ge = c->graph[prec_slot];
        if (!ge) {
            if ((e = build_inner_graph<T, C>(c, w, minv, cf, c->sc, &ge)) != cudaSuccess) return e;
        }
        return cudaGraphLaunch(ge, c->stream);
    }
    const Layout& L = c->L;
    cudaStream_t s = c->stream;
    const int nb = c->ntiles_active;
    cudaGraphConditionalHandle h0 = 0;
    k_cg_init<T><<<nb, 256, 0, s>>>(L, c->tiles, c->nf, c->w64.r, minv, w, c->sc, c->partial, c->counter, nb, h0, 0);
    chunk = chunk < 2 ? 2 : (chunk + 1) & ~1;   // even: p[0]/p[1] parity restarts each chunk
    for (long it = 0;; it += chunk) {
        for (int k = 0; k < chunk; ++k) {
            ApplyArgs a = c->apply_args();
            a.pold = w.p[k & 1];
            a.pnew = w.p[(k & 1) ^ 1];
            a.partial = c->partial;
            a.counter = c->counter;
            a.sc = c->sc;
            if ((e = launch_apply_mode<T, C>(L, c->tiles, nb, cf, w.z, w.q, MODE_CG, a, s)) != cudaSuccess) return e;
            k_cg_update<T><<<persist_grid((const void*)k_cg_update<T>, nb), 256, 0, s>>>(L, c->tiles, c->nf, minv, w,
                                                                                       w.p[(k & 1) ^ 1], c->sc, c->partial,
                                              c->counter, nb, h0, 0);
        }
        if ((e = fetch_scalars(c)) != cudaSuccess) return e;
        if (c->h_sc[0].done) break;
    }
    return cudaGetLastError();
}

// Inner Schwarz-preconditioned CG solve (FP32 vectors): graph with a
// conditional while node, or host-driven chunks.
static cudaError_t run_inner_schwarz(Ctx* c, int use_graph, int chunk) {
    cudaError_t e;
    if (!c->sw_ready && (e = schwarz_build(c)) != cudaSuccess) return e;
    cudaStream_t s = c->stream;
    if (use_graph) {
        cudaGraphExec_t& ge = c->graph[3];
        if (!ge) {
            cudaGraph_t g = nullptr;
            if ((e = cudaGraphCreate(&g, 0)) != cudaSuccess) return e;
            cudaGraphConditionalHandle h;
            if ((e = cudaGraphConditionalHandleCreate(&h, g, 1u, cudaGraphCondAssignDefault)) != cudaSuccess) return e;
            if ((e = cudaStreamBeginCaptureToGraph(s, g, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed)) !=
                cudaSuccess)
                return e;
            schwarz_start(c, s, h, 1);
            cudaGraph_t cap = nullptr;
            if ((e = cudaStreamEndCapture(s, &cap)) != cudaSuccess) return e;
            // the conditional node follows every node without dependents
            size_t na = 0;
            cudaGraphGetNodes(g, nullptr, &na);
            std::vector<cudaGraphNode_t> all(na), leaves;
            cudaGraphGetNodes(g, all.data(), &na);
            for (auto nd : all) {
                size_t nd_out = 0;
                cudaGraphNodeGetDependentNodes(nd, nullptr, nullptr, &nd_out);
                if (nd_out == 0) leaves.push_back(nd);
            }
            size_t nn = leaves.size();
            cudaGraphNodeParams cp = {};
            cp.type = cudaGraphNodeTypeConditional;
            cp.conditional.handle = h;
            cp.conditional.type = cudaGraphCondTypeWhile;
            cp.conditional.size = 1;
            cudaGraphNode_t cond;
            if ((e = cudaGraphAddNode(&cond, g, leaves.data(), nullptr, nn, &cp)) != cudaSuccess) return e;
            cudaGraph_t body = cp.conditional.phGraph_out[0];
            if ((e = cudaStreamBeginCaptureToGraph(s, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed)) !=
                cudaSuccess)
                return e;
            schwarz_body(c, s, h, 1, 0);
            schwarz_body(c, s, h, 1, 1);
            cudaGraph_t cap2 = nullptr;
            if ((e = cudaStreamEndCapture(s, &cap2)) != cudaSuccess) return e;
            e = cudaGraphInstantiate(&ge, g, 0);
            cudaGraphDestroy(g);
            if (e != cudaSuccess) return e;
        }
        return cudaGraphLaunch(ge, s);
    }
    cudaGraphConditionalHandle h0 = 0;
    schwarz_start(c, s, h0, 0);
    chunk = chunk < 2 ? 2 : (chunk + 1) & ~1;
    for (;;) {
        for (int k = 0; k < chunk; ++k) schwarz_body(c, s, h0, 0, k & 1);
        if ((e = fetch_scalars(c)) != cudaSuccess) return e;
        if (c->h_sc[0].done) break;
    }
    return cudaGetLastError();
}

static cudaError_t push_inner_params(Ctx* c, double scale, double tol_rel, int max_iter) {
    CgScalars& h = c->h_sc[0];
    std::memset(&h, 0, sizeof(h));
    h.scale = scale;
    h.tol_rel = tol_rel;
    h.max_iter = max_iter;
    h.wait_test = c->wait_test;
    return cudaMemcpyAsync(c->sc, &h, sizeof(CgScalars), cudaMemcpyHostToDevice, c->stream);
}

stokes_status solve_system(Ctx* c, const double* b, double* x, const stokes_options* o, stokes_stats* st) {
    const Layout& L = c->L;
    cudaStream_t s = c->stream;
    const int nb = c->ntiles_active;
    cudaError_t e = cudaSuccess;
    int total_iter = 0, outer = 0;
    int status = STOKES_OK;
    double rel = 0.0;
#define CK(...)                                                                \
    do {                                                                       \
        if ((e = (__VA_ARGS__)) != cudaSuccess) {                              \
            set_error(c, std::string("CUDA error in solve: ") + cudaGetErrorString(e)); \
            return STOKES_ERR_CUDA;                                            \
        }                                                                      \
    } while (0)
    if (nb == 0) {
        if (st) { st->iterations = 0; st->outer = 0; st->rel_residual = 0.0; st->status = 0; }
        return STOKES_OK;
    }
    // the wait test hook holds for this solve only
    struct WaitTestScope {
        int& v;
        ~WaitTestScope() { v = 0; }
    } wait_scope{c->wait_test};
    c->wait_test = o->wait_test;
    CgScalars* so = c->sc + 1;
    k_outer_init<<<nb, 256, 0, s>>>(L, c->tiles, c->nf, b, x, c->w64.r, so, c->partial, c->counter, nb);
    CK(cudaGetLastError());
    CK(fetch_scalars(c));
    const double bb = c->h_sc[1].rr0;
    if (bb == 0.0) {
        if (st) { st->iterations = 0; st->outer = 0; st->rel_residual = 0.0; st->status = 0; }
        return STOKES_OK;
    }
    if (!std::isfinite(bb)) {
        set_error(c, "non-finite right-hand side");
        return STOKES_ERR_NONFINITE;
    }
    double rr = bb;
    int mode = o->mode;
    const int use_graph = o->use_graph;
    ApplyArgs ra = c->apply_args();
    ra.b = b;
    ra.partial = c->partial;
    ra.counter = c->counter;
    ra.sc = so;
    auto residual = [&]() -> cudaError_t {   // r64 = b - A64 x, ||r64||^2 -> so->rr
        return launch_apply_mode<double, double>(L, c->tiles, nb, c->coef<double>(), x, c->w64.r, MODE_RESID, ra, s);
    };
    auto update = [&](double sign) {
        if (mode == STOKES_FP64) k_ir_update<double><<<nb, 256, 0, s>>>(L, c->tiles, c->nf, x, c->w64.x, c->sc, sign);
        else k_ir_update<float><<<nb, 256, 0, s>>>(L, c->tiles, c->nf, x, c->w32.x, c->sc, sign);
    };
    for (outer = 0; outer < o->max_outer; ++outer) {
        rel = std::sqrt(rr / bb);
        if (rel <= o->tol) break;
        int remaining = o->max_iter - total_iter;
        if (remaining <= 0) { status = STOKES_ERR_NOT_CONVERGED; break; }
        // inner tolerance: loose in mixed mode, the final target in FP64 mode
        double target = 0.5 * o->tol / rel;   // relative to the current residual
        double tol_rel = mode == STOKES_FP64 ? target : std::fmax(o->inner_tol, target);
        double scale = 1.0 / std::sqrt(rr);
        CK(push_inner_params(c, scale, tol_rel, remaining));
        if (o->precond == 2 && L.dim == 2 && mode != STOKES_FP64) {
            // additive Schwarz preconditioner, FP32 inner CG
            CK(run_inner_schwarz(c, use_graph, o->check_every));
            mode = STOKES_FP32;
        } else if (o->precond == 1 && c->learned.net && mode != STOKES_FP64) {
            // learned preconditioner: flexible CG in FP32 (both FP32 and BF16 modes)
            int its = 0, jac = 0;
            CK(run_inner_fpcg(c, c->learned.net, scale, tol_rel, remaining, &its, &jac));
            c->learned_jacobi_steps += jac;
            mode = STOKES_FP32;
        } else if (mode == STOKES_FP64)
            CK(run_inner<double, double>(c, 0, c->w64, c->A.minv64, c->coef<double>(), use_graph, o->check_every));
        else if (mode == STOKES_FP32)
            CK(run_inner<float, float>(c, 1, c->w32, c->A.minv32, c->coef<float>(), use_graph, o->check_every));
        else
            CK(run_inner<float, __nv_bfloat16>(c, 2, c->w32, c->A.minv32, c->coef<__nv_bfloat16>(), use_graph,
                                               o->check_every));
        update(1.0);
        CK(cudaGetLastError());
        CK(residual());
        CK(fetch_scalars(c));
        total_iter += c->h_sc[0].iter;
        double rr_new = c->h_sc[1].rr;
        int ist = c->h_sc[0].status;
        if (std::getenv("STOKES_VERBOSE"))
            std::fprintf(stderr, "[stokes] outer %d mode %d precond %d inner iters %d status %d rel %.3e -> %.3e\n",
                         outer, mode, o->precond, c->h_sc[0].iter, ist, std::sqrt(rr / bb), std::sqrt(rr_new / bb));
        if (ist == STOKES_ERR_TIMEOUT) { status = ist; break; }   // a bounded device wait ran out
        if (!(rr_new <= 4.0 * rr) || !std::isfinite(rr_new)) {
            // the step made the FP64 residual grow (refinement diverging at
            // this inner precision): undo it and move the inner solve up one
            // precision (BF16 -> FP32 -> FP64).  A step that merely stalls is
            // kept: later steps usually recover.
            update(-1.0);
            CK(residual());
            CK(fetch_scalars(c));
            rr = c->h_sc[1].rr;
            if (mode == STOKES_FP64) {
                status = (ist == STOKES_OK || ist == STOKES_ERR_NOT_CONVERGED) ? STOKES_ERR_NOT_CONVERGED : ist;
                break;
            }
            mode = mode == STOKES_BF16 ? STOKES_FP32 : STOKES_FP64;
            continue;
        }
        rr = rr_new;
        if ((ist == STOKES_ERR_NONFINITE || ist == STOKES_ERR_BREAKDOWN) && std::sqrt(rr / bb) > o->tol) {
            if (mode == STOKES_FP64) { status = ist; break; }
            mode = mode == STOKES_BF16 ? STOKES_FP32 : STOKES_FP64;
        }
    }
    rel = std::sqrt(rr / bb);
    if (status == STOKES_OK && rel > o->tol) status = STOKES_ERR_NOT_CONVERGED;
    if (st) {
        st->iterations = total_iter;
        st->outer = outer;
        st->rel_residual = rel;
        st->status = status;
        st->precision_used = mode;
    }
    if (status != STOKES_OK) set_error(c, "solve stopped with status " + std::to_string(status) +
                                              " at relative residual " + std::to_string(rel));
    return (stokes_status)status;
#undef CK
}

// z = M^-1 r for a FP32 slot-layout r: Jacobi (0) or additive Schwarz (2, 2D).
cudaError_t apply_preconditioner(Ctx* c, int which, const float* r, float* z) {
    const Layout& L = c->L;
    cudaStream_t s = c->stream;
    const int64_t V = c->vec_elems();
    cudaError_t e;
    if (which == 0) {
        k_jacobi_apply<<<(unsigned)((V + 255) / 256), 256, 0, s>>>(V, r, c->A.minv32, z);
        return cudaGetLastError();
    }
    if (L.dim != 2) return cudaErrorInvalidValue;
    if (!c->sw_ready && (e = schwarz_build(c)) != cudaSuccess) return e;
    if ((e = push_inner_params(c, 1.0, 0.0, 1)) != cudaSuccess) return e;
    // inactive tiles: identity on real slots (r is zero on padding)
    if ((e = cudaMemcpyAsync(z, r, sizeof(float) * V, cudaMemcpyDeviceToDevice, s)) != cudaSuccess) return e;
    CgWork<float> w{};
    w.r = (float*)r;
    w.z = z;
    const int nb = c->ntiles_active;
    launch_schwarz_gemv(L, *c->sw, r, c->sc, s);
    if (nb)
        k_sw_finish<1><<<persist_grid((const void*)k_sw_finish<1>, (nb + 1) / 2), 256, 0, s>>>(L, c->tiles, c->A, *c->sw, w, c->sc,
                                                                                   c->partial, c->counter, nb, 0, 0);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if ((e = fetch_scalars(c)) != cudaSuccess) return e;
    return c->h_sc[0].status == STOKES_ERR_TIMEOUT ? cudaErrorLaunchTimeout : cudaSuccess;
}

double schwarz_setup_ms(Ctx* c) { return c->sw_ready ? c->sw_setup_ms : -1.0; }

// The context's Schwarz plan for its current weights, built if needed.
cudaError_t schwarz_ensure(Ctx* c, const SchwarzPlan** plan) {
    cudaError_t e = cudaSuccess;
    if (!c->sw_ready) e = schwarz_build(c);
    if (plan) *plan = c->sw;
    return e;
}

// ---------------------------------------------------------------------------
// Allocation-free additive Schwarz apply.  For callers that cannot allocate
// device memory while they run: a process whose device memory is reserved up
// front by its own pool allocator (cudaMalloc would fail or break its budget),
// or a real-time loop that cannot accept the implicit device-wide
// synchronisation of cudaMalloc/cudaFree.  It runs the same kernels as
// apply_preconditioner(which = 2) with their scratch (the per-patch local
// results, the block partials, the reduction counter and the CG scalars) in
// the file-scope device array below instead of context memory, and allocates
// nothing, host or device.  The patch factors themselves are the context's
// (built by an earlier Schwarz apply or solve).
//
// The array's device address is looked up once per device, on the first call
// on it, with the context's device current; a call made while another device
// is current is refused.  Each call reads the solve status back and
// synchronises the context's stream.  Every call uses the same array: calls
// that overlap on the GPU (other streams, other contexts, other threads) race
// and give wrong results.
constexpr size_t NOALLOC_SCRATCH_BYTES = size_t(8) << 20;   // 8 MiB: 2D grids up to 555^2
static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_SCRATCH_BYTES];
constexpr int NOALLOC_MAX_DEVICES = 64;
static void* g_noalloc_ptr[NOALLOC_MAX_DEVICES];
static std::mutex g_noalloc_mu;

static size_t round256(size_t b) { return (b + 255) / 256 * 256; }

// byte offsets of the scratch parts for this context: scalars, counter,
// partials, local results
struct NoallocLayout { size_t sc, counter, partial, ybuf, total; };
static NoallocLayout noalloc_layout(const Ctx* c) {
    NoallocLayout o;
    const size_t ng = (size_t)c->sw->npx * c->sw->npy;
    o.sc = 0;
    o.counter = round256(2 * sizeof(CgScalars));
    o.partial = o.counter + 256;
    o.ybuf = o.partial + round256(sizeof(double) * 2 * ((size_t)c->ntiles_active + 32));
    o.total = o.ybuf + round256(sizeof(float) * ng * PMAX);
    return o;
}

cudaError_t apply_schwarz_noalloc(Ctx* c, const float* r, float* z, std::string* why) {
    const Layout& L = c->L;
    if (L.dim != 2) { *why = "the Schwarz preconditioner is 2D only"; return cudaErrorInvalidValue; }
    if (!c->sw_ready || !c->sw) {
        *why = "no Schwarz plan for these weights: call stokes_apply_preconditioner(which = 2) or a solve with "
               "precond = 2 first (that call builds it and may allocate)";
        return cudaErrorNotReady;
    }
    const NoallocLayout lo = noalloc_layout(c);
    if (lo.total > NOALLOC_SCRATCH_BYTES) {
        *why = "grid too large for the allocation-free scratch: needs " + std::to_string(lo.total) +
               " bytes, the fixed maximum is " + std::to_string(NOALLOC_SCRATCH_BYTES) +
               " (2D grids up to 555^2); use stokes_apply_preconditioner";
        return cudaErrorInvalidValue;
    }
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    // the symbol's address is per device, and the kernels run on the
    // context's stream: both need the context's device current
    if (dev != c->device) {
        *why = "the context's device (" + std::to_string(c->device) + ") is not the current device (" +
               std::to_string(dev) + "): make it current first";
        return cudaErrorInvalidValue;
    }
    if (dev < 0 || dev >= NOALLOC_MAX_DEVICES) { *why = "device index out of range"; return cudaErrorInvalidDevice; }
    unsigned char* base = nullptr;
    {
        std::lock_guard<std::mutex> g(g_noalloc_mu);
        if (!g_noalloc_ptr[dev]) {
            void* p = nullptr;
            e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
            if (e != cudaSuccess) { *why = "cudaGetSymbolAddress failed"; return e; }
            g_noalloc_ptr[dev] = p;
        }
        base = static_cast<unsigned char*>(g_noalloc_ptr[dev]);
    }
    CgScalars* sc = reinterpret_cast<CgScalars*>(base + lo.sc);
    unsigned* counter = reinterpret_cast<unsigned*>(base + lo.counter);
    double* partial = reinterpret_cast<double*>(base + lo.partial);
    SchwarzPlan P = *c->sw;
    P.ybuf = reinterpret_cast<float*>(base + lo.ybuf);
    cudaStream_t s = c->stream;
    const int64_t V = c->vec_elems();
    // what must start at zero: the scalars (done, status), the counter and
    // the local results (inactive patches and positions are summed as zeros).
    // The scalars stay zero apart from what the kernels write: this call
    // defines only z (the r.z and r.r the gather also forms are not returned),
    // so it needs none of the CG parameters the existing entry point uploads.
    // The kernels, their order and their inputs are those of that entry point,
    // so z is bit-identical to its result.
    if ((e = cudaMemsetAsync(base, 0, lo.total, s)) != cudaSuccess) return e;
    // inactive tiles: identity on real slots (r is zero on padding)
    if ((e = cudaMemcpyAsync(z, r, sizeof(float) * V, cudaMemcpyDeviceToDevice, s)) != cudaSuccess) return e;
    CgWork<float> w{};
    w.r = (float*)r;
    w.z = z;
    const int nb = c->ntiles_active;
    launch_schwarz_gemv(L, P, r, sc, s);
    if (nb)
        k_sw_finish<1><<<persist_grid((const void*)k_sw_finish<1>, (nb + 1) / 2), 256, 0, s>>>(L, c->tiles, c->A, P, w, sc, partial,
                                                                                   counter, nb, 0, 0);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    int status = 0;
    if ((e = cudaMemcpyAsync(&status, &sc->status, sizeof(int), cudaMemcpyDeviceToHost, s)) != cudaSuccess) return e;
    if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return e;
    if (status == STOKES_ERR_TIMEOUT) { *why = "a local solve's copy wait timed out"; return cudaErrorLaunchTimeout; }
    return cudaSuccess;
}

// Time real CG iterations kernel by kernel: r = b (the last right-hand side),
// then ``launches`` x [apply in CG mode, update] with CUDA events around each
// launch on the context's stream.  Averages in ms per launch.
template <class T, class C>
static cudaError_t bench_impl(Ctx* c, CgWork<T>& w, const T* minv, const Coef<C>& cf, int launches, double* ms_apply,
                              double* ms_update) {
    const Layout& L = c->L;
    cudaStream_t s = c->stream;
    const int nb = c->ntiles_active;
    cudaError_t e;
    if ((e = push_inner_params(c, 1.0, 0.0, 1 << 30)) != cudaSuccess) return e;
    cudaGraphConditionalHandle h0 = 0;
    k_cg_init<T><<<nb, 256, 0, s>>>(L, c->tiles, c->nf, c->b64, minv, w, c->sc, c->partial, c->counter, nb, h0, 0);
    std::vector<cudaEvent_t> ev(2 * launches + 1);
    for (auto& x : ev) cudaEventCreate(&x);
    // two untimed iterations first: the first launch of a kernel in a process
    // can wait on the host (module loading), which the events would count
    for (int k = -2; k < 0; ++k) {
        ApplyArgs a = c->apply_args();
        a.pold = w.p[k & 1];
        a.pnew = w.p[(k & 1) ^ 1];
        a.partial = c->partial;
        a.counter = c->counter;
        a.sc = c->sc;
        launch_apply_mode<T, C>(L, c->tiles, nb, cf, w.z, w.q, MODE_CG, a, s);
        k_cg_update<T><<<persist_grid((const void*)k_cg_update<T>, nb), 256, 0, s>>>(L, c->tiles, c->nf, minv, w,
                                                                                   w.p[(k & 1) ^ 1], c->sc, c->partial,
                                                                                   c->counter, nb, h0, 0);
    }
    if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return e;
    cudaEventRecord(ev[0], s);
    for (int k = 0; k < launches; ++k) {
        ApplyArgs a = c->apply_args();
        a.pold = w.p[k & 1];
        a.pnew = w.p[(k & 1) ^ 1];
        a.partial = c->partial;
        a.counter = c->counter;
        a.sc = c->sc;
        launch_apply_mode<T, C>(L, c->tiles, nb, cf, w.z, w.q, MODE_CG, a, s);
        cudaEventRecord(ev[2 * k + 1], s);
        k_cg_update<T><<<persist_grid((const void*)k_cg_update<T>, nb), 256, 0, s>>>(L, c->tiles, c->nf, minv, w,
                                                                                   w.p[(k & 1) ^ 1], c->sc, c->partial,
                                          c->counter, nb, h0, 0);
        cudaEventRecord(ev[2 * k + 2], s);
    }
    if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return e;
    double ta = 0, tu = 0;
    for (int k = 0; k < launches; ++k) {
        float a = 0, u = 0;
        cudaEventElapsedTime(&a, ev[2 * k], ev[2 * k + 1]);
        cudaEventElapsedTime(&u, ev[2 * k + 1], ev[2 * k + 2]);
        ta += a; tu += u;
    }
    for (auto& x : ev) cudaEventDestroy(x);
    *ms_apply = ta / launches;
    *ms_update = tu / launches;
    if ((e = fetch_scalars(c)) != cudaSuccess) return e;
    if (c->h_sc[0].done) return cudaErrorInvalidValue;  // the loop stopped early: timings invalid
    return cudaGetLastError();
}

// Time the Schwarz kernels of a CG iteration launch by launch (local patch
// solves, then the gather with its dots), CUDA events around each on the
// context's stream, r = the last right-hand side.  bytes_local: algorithmic
// bytes of one local-solve launch (every patch's factor, its residual gather
// by position, scaling and local map, its results).
cudaError_t bench_schwarz_kernels(Ctx* c, int launches, double* ms_local, double* ms_gather, double* bytes_local) {
    const Layout& L = c->L;
    cudaStream_t s = c->stream;
    cudaError_t e;
    if (L.dim != 2) return cudaErrorInvalidValue;
    if (!c->sw_ready && (e = schwarz_build(c)) != cudaSuccess) return e;
    const SchwarzPlan& P = *c->sw;
    std::vector<int> nloc(std::max(1, P.np));
    if (P.np && (e = cudaMemcpy(nloc.data(), P.nloc, sizeof(int) * P.np, cudaMemcpyDeviceToHost)) != cudaSuccess)
        return e;
    double by = 0.0;
    for (int q = 0; q < P.np; ++q)
        by += (double)sw_patch_bytes(nloc[q]) + PMAX * (sizeof(float) + sizeof(float) + sizeof(float) + sizeof(short)) +
              2 * PR * PR * sizeof(float) + 2 * sizeof(int);   // factor; r, q, scaling, map; results; corner, count
    *bytes_local = by;
    if ((e = push_inner_params(c, 1.0, 0.0, 1 << 30)) != cudaSuccess) return e;
    CgWork<float>& w = c->w32;
    const int nb = c->ntiles_active;
    k_sw_init<<<nb, 256, 0, s>>>(L, c->tiles, c->b64, w, c->sc);
    launch_schwarz_gemv(L, P, w.r, c->sc, s);
    k_sw_finish<1><<<persist_grid((const void*)k_sw_finish<1>, (nb + 1) / 2), 256, 0, s>>>(L, c->tiles, c->A, P, w, c->sc,
                                                                               c->partial, c->counter, nb, 0, 0);
    std::vector<cudaEvent_t> ev(2 * launches + 1);
    for (auto& x : ev) cudaEventCreate(&x);
    // two untimed iterations first: the first launch of a kernel in a process
    // can wait on the host (module loading), which the events would count
    // the kernels as the CG loop runs them (alpha = 0 here: r and x keep their values)
    for (int k = 0; k < 2; ++k) {
        launch_schwarz_gemv(L, P, w.r, c->sc, s, w.q);
        k_sw_finish<0, 1><<<persist_grid((const void*)k_sw_finish<0, 1>, (nb + 1) / 2), 256, 0, s>>>(
            L, c->tiles, c->A, P, w, c->sc, c->partial, c->counter, nb, 0, 0, w.p[0]);
    }
    if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return e;
    cudaEventRecord(ev[0], s);
    for (int k = 0; k < launches; ++k) {
        launch_schwarz_gemv(L, P, w.r, c->sc, s, w.q);
        cudaEventRecord(ev[2 * k + 1], s);
        k_sw_finish<0, 1><<<persist_grid((const void*)k_sw_finish<0, 1>, (nb + 1) / 2), 256, 0, s>>>(
            L, c->tiles, c->A, P, w, c->sc, c->partial, c->counter, nb, 0, 0, w.p[0]);
        cudaEventRecord(ev[2 * k + 2], s);
    }
    if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return e;
    double ta = 0, tg = 0;
    for (int k = 0; k < launches; ++k) {
        float a = 0, g = 0;
        cudaEventElapsedTime(&a, ev[2 * k], ev[2 * k + 1]);
        cudaEventElapsedTime(&g, ev[2 * k + 1], ev[2 * k + 2]);
        ta += a; tg += g;
    }
    for (auto& x : ev) cudaEventDestroy(x);
    *ms_local = ta / launches;
    *ms_gather = tg / launches;
    if ((e = fetch_scalars(c)) != cudaSuccess) return e;
    if (c->h_sc[0].done) return cudaErrorInvalidValue;  // the kernels returned early: timings invalid
    return cudaGetLastError();
}

cudaError_t bench_cg_kernels(Ctx* c, int precision, int launches, double* ms_apply, double* ms_update) {
    if (precision == STOKES_FP64)
        return bench_impl<double, double>(c, c->w64, c->A.minv64, c->coef<double>(), launches, ms_apply, ms_update);
    if (precision == STOKES_FP32)
        return bench_impl<float, float>(c, c->w32, c->A.minv32, c->coef<float>(), launches, ms_apply, ms_update);
    return bench_impl<float, __nv_bfloat16>(c, c->w32, c->A.minv32, c->coef<__nv_bfloat16>(), launches, ms_apply,
                                            ms_update);
}

}  // namespace stk
