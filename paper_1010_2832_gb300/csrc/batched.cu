// Batched solve of many independent 2D systems (eq. stokesmixedsystemspd,
// one per context) in one persistent cooperative kernel.
//
// Work list: the active tiles of every instance, concatenated (instance i
// owns the contiguous range [tb_i, te_i)); with the Schwarz preconditioner
// also every instance's active patches.  Each CTA walks the lists with a
// grid stride.  Per CG iteration, phases separated by grid barriers:
//   A  CG instances: p = z + beta p_old, q = A p, p.q   -> alpha
//      CHECK instances: r = b - A x (true FP64 residual)
//   C  (Schwarz only) local patch solves on r - alpha q (r in CHECK mode)
//   D  CG instances: x += alpha p, r -= alpha q; every instance:
//      z = M^-1 r (Jacobi, or the gather of the local results), r.z, r.r
// The CTA that reports an instance's last tile of a phase reduces that
// instance's per-tile partials in list order (deterministic) and updates
// its scalars: CG -> CHECK when the recurrence residual meets the
// tolerance; CHECK -> done if the true residual meets it, else CG restarts
// from the true residual.  Instances retire independently; the kernel ends
// when all have.  Every grid barrier is a bounded wait: after ~2^24 polls
// it records STOKES_ERR_TIMEOUT and every CTA returns.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <fstream>
#include <map>
#include <sstream>
#include <string>
#include <vector>
#include "internal.cuh"
#include "ctx.cuh"
#include "apply2d_tile.cuh"
#include "schwarz_plan.cuh"

namespace stk {
cudaError_t schwarz_ensure(Ctx* c, const SchwarzPlan** plan);
cudaError_t launch_rhs(Ctx* c, const double* const* ustar, double* b);
cudaError_t launch_recover(Ctx* c, const double* const* ustar, const double* x, double* const* uout);
cudaError_t launch_unpack(Ctx* c, const double* slots, double* const* fields, int to_fields);
}  // namespace stk

using namespace stk;

namespace {

struct BInst {
    Layout L;
    Coef<double> cf;
    const double* minv;
    const double* b;
    double *x, *r, *z, *q;
    double* p[2];
    int tb, te;
    int use_sw;                     // additive Schwarz preconditioner (else Jacobi)
    SchwarzPlan sw;
    const uint8_t* act_cell;
    const uint8_t* act_node;
};

struct BState {
    double rz, rr, alpha, beta, tol2, bb;
    int mode;      // 0 CG, 1 CHECK (true residual), 2 START (Schwarz: first z = M^-1 b pending)
    int parity, iter, done, status;
    unsigned cnt;
};

struct BGlobal {
    unsigned bar_count, bar_gen;
    int ndone, err;
};

__device__ bool grid_sync(BGlobal* g, unsigned nblocks) {
    __shared__ int ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        ok = 1;
        volatile unsigned* genp = &g->bar_gen;
        volatile int* errp = &g->err;
        unsigned gen = *genp;
        __threadfence();
        unsigned arrived = atomicAdd(&g->bar_count, 1u) + 1u;
        if (arrived == nblocks) {
            g->bar_count = 0u;
            __threadfence();
            atomicAdd(&g->bar_gen, 1u);
        } else {
            long long spins = 0;
            while (*genp == gen) {
                if (*errp) { ok = 0; break; }
                if (++spins > (1LL << 24)) { atomicExch(&g->err, (int)STOKES_ERR_TIMEOUT); ok = 0; break; }
                __nanosleep(64);
            }
        }
        __threadfence();
    }
    __syncthreads();
    return ok && !((volatile int*)&g->err)[0];
}

// Block-reduce two warp partials, store them for tile w, and let the CTA that
// completes instance i's phase reduce all of i's tiles; fin(s0, s1) runs on
// thread 0 of that CTA.
template <class Fin>
__device__ void tile_report(double v0, double v1, double* part, int w, BState* st, const BInst& I, Fin fin) {
    __shared__ double red[2][8];
    __shared__ bool last;
    int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
    if (lane == 0) { red[0][wp] = v0; red[1][wp] = v1; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double s0 = 0.0, s1 = 0.0;
        for (int q = 0; q < 8; ++q) { s0 += red[0][q]; s1 += red[1][q]; }
        part[2 * w] = s0;
        part[2 * w + 1] = s1;
        __threadfence();
        unsigned prev = atomicAdd(&st->cnt, 1u);
        last = (prev == (unsigned)(I.te - I.tb) - 1u);
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    double s0 = 0.0, s1 = 0.0;
    for (int k = I.tb + threadIdx.x; k < I.te; k += 256) {
        s0 += ((volatile double*)part)[2 * k];
        s1 += ((volatile double*)part)[2 * k + 1];
    }
    s0 = warp_sum(s0);
    s1 = warp_sum(s1);
    __syncthreads();
    if (lane == 0) { red[0][wp] = s0; red[1][wp] = s1; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double t0 = 0.0, t1 = 0.0;
        for (int q = 0; q < 8; ++q) { t0 += red[0][q]; t1 += red[1][q]; }
        fin(t0, t1);
        st->cnt = 0u;
        __threadfence();
    }
    __syncthreads();
}

// Additive Schwarz local solve of patch p of instance I, by the whole CTA
// (256 threads; the triangular products use 128): the same arithmetic as
// the single-system kernel k_schwarz_gemv, on r_eff = r - alpha q read in
// FP64 (alpha = 0 outside a CG step).  Thread 0 starts the bulk copy of the
// factor and waits on the CTA's mbarrier (phase parity = uses & 1, bounded);
// a copy that never completes sets the batch's error flag.
__device__ void batched_local_solve(const BInst& I, int p, double alpha, uint8_t* Fs, float* s, float* y, __half* hb,
                                    unsigned long long* bar, uint32_t& uses, int& ok_s, BGlobal* g) {
    const SchwarzPlan& P = I.sw;
    const Layout& L = I.L;
    const int t = threadIdx.x;
    // after an error (a copy that timed out) start no further copies; the
    // decision is the same for the whole CTA
    if (t == 0) ok_s = ((volatile int*)&g->err)[0] == 0;
    __syncthreads();
    if (!ok_s) return;
    const int n = P.nloc[p];
    const uint32_t b_addr = smem_u32(bar);
    if (t == 0) sw_issue(b_addr, Fs, P.fac + (int64_t)p * SW_FAC_BYTES, sw_patch_bytes(n), P.evict_first != 0);
    constexpr float H = 0.70710678118654752f;
    const int CI = P.corner[p] & 0xffff, CJ = P.corner[p] >> 16;
    const int a0 = PB * CI - 1, b0 = PB * CJ - 1;
    const short* map = P.lmap + (int64_t)p * PMAX;
    const float* scl = P.scale + (int64_t)p * PMAX;
    int kk = -1, kp = -1;
    float sa = 0.f, sb = 0.f;
    if (t < 2 * PR * PR) {
        const int e = t;
        const int rem = e % (PR * PR), jj = rem / PR, ii = rem % PR;
        const int64_t o = L.off(a0 + ii + 1, b0 + jj + 1, 0);
        kk = map[e];
        sa = scl[e];
        if (e >= PR * PR) {
            const float rv = (float)(I.r[L.stride + o] - alpha * I.q[L.stride + o]);
            if (kk >= 0) s[kk] = rv * sa;
        } else {
            kp = map[2 * PR * PR + e];
            sb = scl[2 * PR * PR + e];
            const float rt = (float)(I.r[o] - alpha * I.q[o]);
            const float rp = (float)(I.r[2 * L.stride + o] - alpha * I.q[2 * L.stride + o]);
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
    if (t >= n && t < (n + 7) / 8 * 8) s[t] = 0.f;
    if (t == 0) {
        ok_s = mbar_wait(b_addr, uses & 1u) ? 1 : 0;
        ++uses;
    }
    __syncthreads();
    if (!ok_s) {
        if (t == 0) {
            mbar_wait(b_addr, (uses - 1u) & 1u);
            atomicExch(&g->err, (int)STOKES_ERR_TIMEOUT);
        }
        __syncthreads();
        return;
    }
    sw_factor_products(Fs, n, s, y, hb);
    float* out = P.ybuf + (int64_t)(CJ * P.npx + CI) * PMAX;
    if (t < 2 * PR * PR) {
        const int e = t;
        if (e >= PR * PR) {
            if (kk >= 0) out[e] = s[kk] * sa;
        } else if (kk >= 0 && kp >= 0) {
            const float a = s[kk] * sa, b = s[kp] * sb;
            out[e] = (a + b) * H;
            out[2 * PR * PR + e] = (a - b) * H;
        } else if (kk >= 0) {
            out[e] = s[kk] * sa;
        } else if (kp >= 0) {
            out[2 * PR * PR + e] = s[kp] * sb;
        }
    }
    __syncthreads();                             // the next patch reuses shared memory
}

// z of field f at sample (i, j) from the patches' local results (the
// single-system gather schwarz_gather_slot, in FP64 out).
__device__ __forceinline__ double batched_gather(const BInst& I, int f, int i, int j, double r) {
    const Layout& L = I.L;
    if (!unknown_active(I.act_cell, I.act_node, L, f, i, j))
        return (i >= 0 && j >= 0 && i <= L.nx && j <= L.ny) ? r : 0.0;
    const SchwarzPlan& P = I.sw;
    const int ilo = max((i + PB - 1) / PB - 1, 0), ihi = min((i + 1) / PB, P.npx - 1);
    const int jlo = max((j + PB - 1) / PB - 1, 0), jhi = min((j + 1) / PB, P.npy - 1);
    // (a loop over the patches in range: a fixed, masked 2 x 2 window as in
    // the single-system gather needs more registers here, which costs this
    // persistent kernel a CTA per SM)
    float s = 0.f;
    for (int J = jlo; J <= jhi; ++J)
        for (int Ip = ilo; Ip <= ihi; ++Ip) {
            const int ii = i - (PB * Ip - 1), jj = j - (PB * J - 1);
            s += P.ybuf[(int64_t)(J * P.npx + Ip) * PMAX + (f * PR + jj) * PR + ii];
        }
    return (double)s;
}

template <int TY, bool SW>
struct BatchedSmem {
    static constexpr int APPLY = (int)sizeof(Smem2<double, TY>);
    static constexpr int LOCAL = SW ? SW_FAC_BYTES : 0;
    static constexpr int BYTES = APPLY > LOCAL ? APPLY : LOCAL;
};

template <int TY, bool SW>
__global__ void __launch_bounds__(256) k_batched(const BInst* __restrict__ inst, BState* st,
                                                 const int* __restrict__ wl_inst, const int* __restrict__ wl_c0,
                                                 const int* __restrict__ wl_r0, int nwork,
                                                 const int* __restrict__ pl_inst, const int* __restrict__ pl_patch,
                                                 int npatch, double* part, BGlobal* g, int ninst, int max_iter,
                                                 double tol) {
    // shared memory: the apply's staging (phase A) and the local solves'
    // factor (phase C) never live at the same time
    __shared__ __align__(128) unsigned char smraw[BatchedSmem<TY, SW>::BYTES];
    Smem2<double, TY>& sm = *reinterpret_cast<Smem2<double, TY>*>(smraw);
    uint8_t* Fs = reinterpret_cast<uint8_t*>(smraw);
    __shared__ __align__(16) float ls[SW ? PMAX8 : 4];
    __shared__ __align__(16) __half lhb[SW ? SW_HB_HALVES : 8];
    __shared__ __align__(8) unsigned long long lbar;
    __shared__ int lok;
    uint32_t uses = 0;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const unsigned nb = gridDim.x;
    if (SW && threadIdx.x == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&lbar)), "r"(1) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    // ---- init: r = b, x = 0, p = 0; Jacobi: z = M^-1 r (Schwarz: later) --
    for (int w = blockIdx.x; w < nwork; w += nb) {
        const int i = wl_inst[w];
        const BInst& I = inst[i];
        const bool swi = SW && I.use_sw;
        const int64_t S = I.L.stride;
        double rz = 0.0, rr = 0.0;
        for (int row = warp; row < TY; row += 8) {
            int64_t o = I.L.off(wl_c0[w] + lane, wl_r0[w] + row, 0);
            for (int f = 0; f < 3; ++f) {
                int64_t of = f * S + o;
                double r = I.b[of], z = swi ? 0.0 : I.minv[of] * r;
                I.r[of] = r; I.z[of] = z; I.x[of] = 0.0; I.p[0][of] = 0.0; I.p[1][of] = 0.0;
                rz = fma(r, z, rz); rr = fma(r, r, rr);
            }
        }
        BState* s = st + i;
        tile_report(warp_sum(rz), warp_sum(rr), part, w, s, I, [&](double trz, double trr) {
            s->rz = trz; s->rr = trr; s->bb = trr; s->tol2 = tol * tol * trr;
            s->mode = swi ? 2 : 0; s->parity = 0; s->iter = 0; s->beta = 0.0; s->status = 0; s->alpha = 0.0;
            s->done = trr == 0.0 ? 1 : 0;
            if (!isfinite(trr)) { s->done = 1; s->status = STOKES_ERR_NONFINITE; }
            if (s->done) atomicAdd(&g->ndone, 1);
        });
    }
    if (!grid_sync(g, nb)) return;
    for (;;) {
        if (((volatile int*)&g->ndone)[0] >= ninst) return;
        // ---- phase A: CG: p = z + beta p_old, q = A p, p.q; CHECK: r = b - A x
        for (int w = blockIdx.x; w < nwork; w += nb) {
            const int i = wl_inst[w];
            volatile BState* vs = st + i;
            if (vs->done || vs->mode == 2) continue;
            const BInst& I = inst[i];
            BState* s = st + i;
            double v;
            if (vs->mode == 0) {
                int par = vs->parity;
                v = apply2d_tile<double, double, MODE_CG, TY, 256>(I.L, wl_c0[w], wl_r0[w], I.cf, I.z, I.q,
                                                                   I.p[par], I.p[par ^ 1], vs->beta, nullptr, sm);
                tile_report(v, 0.0, part, w, s, I, [&](double pq, double) {
                    if (!(pq > 0.0) || !isfinite(pq)) {
                        s->done = 1;
                        s->status = isfinite(pq) ? STOKES_ERR_BREAKDOWN : STOKES_ERR_NONFINITE;
                        atomicAdd(&g->ndone, 1);
                    } else {
                        s->alpha = s->rz / pq;
                    }
                });
            } else {
                v = apply2d_tile<double, double, MODE_RESID, TY, 256>(I.L, wl_c0[w], wl_r0[w], I.cf, I.x, I.r,
                                                                      nullptr, nullptr, 0.0, I.b, sm);
                tile_report(v, 0.0, part, w, s, I, [&](double, double) {});
            }
            __syncthreads();
        }
        if (!grid_sync(g, nb)) return;
        // ---- phase C (Schwarz): local solves on r_eff = r - alpha q ----------
        if (SW) {
            for (int k = blockIdx.x; k < npatch; k += nb) {
                const int i = pl_inst[k];
                volatile BState* vs = st + i;
                if (vs->done) continue;
                const double alpha = vs->mode == 0 ? vs->alpha : 0.0;
                batched_local_solve(inst[i], pl_patch[k], alpha, Fs, ls, ls, lhb, &lbar, uses, lok, g);
            }
            if (!grid_sync(g, nb)) return;
        }
        // ---- phase D: CG: x += alpha p, r -= alpha q; z = M^-1 r; r.z, r.r ---
        for (int w = blockIdx.x; w < nwork; w += nb) {
            const int i = wl_inst[w];
            volatile BState* vs = st + i;
            if (vs->done) continue;
            const BInst& I = inst[i];
            const bool swi = SW && I.use_sw;
            BState* s = st + i;
            const int64_t S = I.L.stride;
            const int mode = vs->mode;
            const double alpha = vs->alpha;
            const double* pn = I.p[vs->parity ^ 1];
            double rz = 0.0, rr = 0.0;
            for (int row = warp; row < TY; row += 8) {
                const int c = wl_c0[w] + lane, rw = wl_r0[w] + row;
                int64_t o = I.L.off(c, rw, 0);
                for (int f = 0; f < 3; ++f) {
                    int64_t of = f * S + o;
                    double r;
                    if (mode == 0) {
                        I.x[of] += alpha * pn[of];
                        r = I.r[of] - alpha * I.q[of];
                        I.r[of] = r;
                    } else {
                        r = I.r[of];
                    }
                    double z = swi ? batched_gather(I, f, c - 1, rw - 1, r) : I.minv[of] * r;
                    I.z[of] = z;
                    rz = fma(r, z, rz); rr = fma(r, r, rr);
                }
            }
            tile_report(warp_sum(rz), warp_sum(rr), part, w, s, I, [&](double trz, double trr) {
                s->rr = trr;
                if (!isfinite(trr) || !isfinite(trz)) {
                    s->done = 1; s->status = STOKES_ERR_NONFINITE; atomicAdd(&g->ndone, 1); return;
                }
                if (mode == 2) {                           // first preconditioned residual
                    if (!(trz > 0.0)) {
                        s->done = 1; s->status = STOKES_ERR_BREAKDOWN; atomicAdd(&g->ndone, 1);
                    } else {
                        s->rz = trz; s->mode = 0; s->beta = 0.0;
                    }
                } else if (mode == 0) {
                    s->iter += 1;
                    if (trr <= s->tol2) {
                        s->mode = 1;                       // verify with the true residual
                    } else if (!(trz > 0.0)) {
                        s->done = 1; s->status = STOKES_ERR_BREAKDOWN; atomicAdd(&g->ndone, 1);
                    } else {
                        s->beta = trz / s->rz; s->rz = trz; s->parity ^= 1;
                    }
                    if (!s->done && s->iter >= max_iter) {
                        s->done = 1; s->status = STOKES_ERR_NOT_CONVERGED; atomicAdd(&g->ndone, 1);
                    }
                } else {
                    if (trr <= s->tol2) {
                        s->done = 1; atomicAdd(&g->ndone, 1);
                    } else {                               // restart from the true residual
                        s->mode = 0; s->beta = 0.0; s->rz = trz;
                    }
                }
            });
            __syncthreads();
        }
        if (!grid_sync(g, nb)) return;
    }
}

}  // namespace

// ---------------------------------------------------------------------------
// Host side: plan (work lists per tile height), autotuner, graph.
// ---------------------------------------------------------------------------
struct stokes_batch_s {
    std::vector<stokes_ctx> ctx;
    std::vector<Ctx*> c;
    int n = 0;
    bool sw = false;            // additive Schwarz preconditioner for every instance
    int* d_pl = nullptr;        // [2][pl_cap]: instance, patch
    int npatch = 0, pl_cap = 0;
    std::vector<unsigned> plan_epoch;     // each instance's plan build count when its plan was uploaded
    stokes_options opt{};
    cudaStream_t s = nullptr;
    int ty = 8, cps = 1;        // chosen tile height and CTAs per SM
    double tuned_us = -1.0;
    std::string err;
    // device
    BInst* d_inst = nullptr;
    BState* d_st = nullptr;
    BState* d_st0 = nullptr;    // initial states (empty instances already retired)
    BGlobal* d_g0 = nullptr;
    bool use_graph = true;
    BGlobal* d_g = nullptr;
    int* d_wl = nullptr;        // [3][wl_cap]: instance, first column, first row of each work tile
    double* d_part = nullptr;   // [2 wl_cap] per-tile partial sums
    size_t wl_cap = 0;
    int nwork = 0;
    int grid = 0;
    std::vector<BState> h_st;
    cudaGraphExec_t graph = nullptr;
    std::vector<const void*> io_key;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
};

static int num_sms() {
    int dev = 0, n = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    return n;
}

template <int TY, bool SW> static void* kernel_ptr() { return (void*)k_batched<TY, SW>; }
static void* kernel_for(int ty, bool sw) {
    if (sw) return ty == 4 ? kernel_ptr<4, true>() : ty == 16 ? kernel_ptr<16, true>() : kernel_ptr<8, true>();
    return ty == 4 ? kernel_ptr<4, false>() : ty == 16 ? kernel_ptr<16, false>() : kernel_ptr<8, false>();
}

static int max_ctas_per_sm(int ty, bool sw) {
    int nb = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kernel_for(ty, sw), 256, 0);
    return nb;
}

// active tiles of height ty (from the 32x4 activity flags of each context)
static cudaError_t build_worklist(stokes_batch b, int ty, std::vector<int>& wi, std::vector<int>& wc,
                                  std::vector<int>& wr, std::vector<BInst>& insts) {
    wi.clear(); wc.clear(); wr.clear();
    insts.resize(b->n);
    for (int i = 0; i < b->n; ++i) {
        Ctx* c = b->c[i];
        const Layout& L = c->L;
        int n4 = L.R / 4;
        std::vector<uint8_t> f4((size_t)L.ntx * n4);
        cudaError_t e = cudaMemcpy(f4.data(), c->A.tile_flag4, f4.size(), cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) return e;
        BInst& I = insts[i];
        I.L = L;
        I.cf = c->coef<double>();
        I.minv = c->A.minv64;
        I.b = c->b64;
        I.x = c->x64;
        I.r = c->w64.r; I.z = c->w64.z; I.q = c->w64.q;
        I.p[0] = c->w64.p[0]; I.p[1] = c->w64.p[1];
        I.use_sw = b->sw ? 1 : 0;
        I.act_cell = c->A.act[0];
        I.act_node = c->A.act[1];
        std::memset(&I.sw, 0, sizeof(I.sw));
        if (b->sw) {
            const SchwarzPlan* P = nullptr;
            if ((e = schwarz_ensure(c, &P)) != cudaSuccess) return e;
            I.sw = *P;
        }
        I.tb = (int)wi.size();
        int per = ty / 4;
        for (int tr = 0; tr < L.R / ty; ++tr)
            for (int tx = 0; tx < L.ntx; ++tx) {
                bool a = false;
                for (int q = 0; q < per; ++q) a |= f4[(size_t)(tr * per + q) * L.ntx + tx] != 0;
                if (a) { wi.push_back(i); wc.push_back(tx * TX); wr.push_back(tr * ty); }
            }
        I.te = (int)wi.size();
    }
    return cudaSuccess;
}

// Patch list of the Schwarz phase (instance, patch), in instance order; a
// larger list than the last one reallocates (and so needs a new graph).
static cudaError_t upload_patches(stokes_batch b, const std::vector<BInst>& insts) {
    b->plan_epoch.assign(b->n, 0u);
    if (!b->sw) { b->npatch = 0; return cudaSuccess; }
    std::vector<int> pi, pp;
    for (int i = 0; i < b->n; ++i) {
        b->plan_epoch[i] = b->c[i]->sw_epoch;
        if (insts[i].te == insts[i].tb) continue;        // no active tile: retired at once
        for (int q = 0; q < insts[i].sw.np; ++q) { pi.push_back(i); pp.push_back(q); }
    }
    const int np = (int)pi.size();
    cudaError_t e;
    if (np > b->pl_cap || !b->d_pl) {
        if (b->d_pl) cudaFree(b->d_pl);
        b->d_pl = nullptr;
        b->pl_cap = std::max(np, 1);
        if ((e = cudaMalloc(&b->d_pl, 2 * (size_t)b->pl_cap * sizeof(int))) != cudaSuccess) return e;
        if (b->graph) { cudaGraphExecDestroy(b->graph); b->graph = nullptr; }
    }
    if (np != b->npatch && b->graph) { cudaGraphExecDestroy(b->graph); b->graph = nullptr; }
    b->npatch = np;
    if (np) {
        if ((e = cudaMemcpy(b->d_pl, pi.data(), np * sizeof(int), cudaMemcpyHostToDevice)) != cudaSuccess) return e;
        if ((e = cudaMemcpy(b->d_pl + b->pl_cap, pp.data(), np * sizeof(int), cudaMemcpyHostToDevice)) != cudaSuccess)
            return e;
    }
    return cudaSuccess;
}

static cudaError_t upload_plan(stokes_batch b, int ty) {
    std::vector<int> wi, wc, wr;
    std::vector<BInst> insts;
    cudaError_t e = build_worklist(b, ty, wi, wc, wr, insts);
    if (e != cudaSuccess) return e;
    if (b->sw) {
        // the batch's factors stream through L2 together: the evict-first
        // policy applies when all of them together exceed half of L2
        size_t tot = 0;
        for (const BInst& I : insts) tot += (size_t)I.sw.np * SW_FAC_BYTES;
        const int ef = sw_factors_exceed_l2(tot) ? 1 : 0;
        for (BInst& I : insts) I.sw.evict_first = ef;
    }
    const int old_nwork = b->nwork;
    b->nwork = (int)wi.size();
    std::vector<BState> st0(b->n);
    std::memset(st0.data(), 0, st0.size() * sizeof(BState));
    BGlobal g0{};
    for (int i = 0; i < b->n; ++i)
        if (insts[i].te == insts[i].tb) { st0[i].done = 1; g0.ndone += 1; }
    if ((e = cudaMemcpy(b->d_st0, st0.data(), st0.size() * sizeof(BState), cudaMemcpyHostToDevice)) != cudaSuccess)
        return e;
    if ((e = cudaMemcpy(b->d_g0, &g0, sizeof(g0), cudaMemcpyHostToDevice)) != cudaSuccess) return e;
    // A captured graph holds the work-list and partial-sum pointers, the work
    // count and the grid by value: it is dropped whenever any of them changes
    // (the next solve captures again).  The buffers keep their capacity.
    const size_t need = std::max(1, b->nwork);
    if (!b->d_wl || need > b->wl_cap) {
        if (b->graph) { cudaGraphExecDestroy(b->graph); b->graph = nullptr; }
        if (b->d_wl) { cudaFree(b->d_wl); b->d_wl = nullptr; }
        if (b->d_part) { cudaFree(b->d_part); b->d_part = nullptr; }
        b->wl_cap = need;
        if ((e = cudaMalloc(&b->d_wl, 3 * b->wl_cap * sizeof(int))) != cudaSuccess) return e;
        if ((e = cudaMalloc(&b->d_part, 2 * b->wl_cap * sizeof(double))) != cudaSuccess) return e;
    }
    if (b->nwork != old_nwork && b->graph) { cudaGraphExecDestroy(b->graph); b->graph = nullptr; }
    if (b->nwork) {
        const size_t nw = b->wl_cap;
        if ((e = cudaMemcpy(b->d_wl, wi.data(), wi.size() * sizeof(int), cudaMemcpyHostToDevice)) != cudaSuccess ||
            (e = cudaMemcpy(b->d_wl + nw, wc.data(), wc.size() * sizeof(int), cudaMemcpyHostToDevice)) != cudaSuccess ||
            (e = cudaMemcpy(b->d_wl + 2 * nw, wr.data(), wr.size() * sizeof(int), cudaMemcpyHostToDevice)) !=
                cudaSuccess)
            return e;
    }
    if ((e = upload_patches(b, insts)) != cudaSuccess) return e;
    return cudaMemcpy(b->d_inst, insts.data(), insts.size() * sizeof(BInst), cudaMemcpyHostToDevice);
}

static cudaError_t launch_persistent(stokes_batch b, int ty, int grid, int max_iter, double tol) {
    cudaError_t e;
    if ((e = cudaMemcpyAsync(b->d_g, b->d_g0, sizeof(BGlobal), cudaMemcpyDeviceToDevice, b->s)) != cudaSuccess)
        return e;
    if ((e = cudaMemcpyAsync(b->d_st, b->d_st0, b->n * sizeof(BState), cudaMemcpyDeviceToDevice, b->s)) != cudaSuccess)
        return e;
    const size_t nw = b->wl_cap;
    const int* wi = b->d_wl;
    const int* wc = b->d_wl + nw;
    const int* wr = b->d_wl + 2 * nw;
    const int* pli = b->d_pl;
    const int* plp = b->d_pl ? b->d_pl + b->pl_cap : nullptr;
    void* args[] = {(void*)&b->d_inst, (void*)&b->d_st, (void*)&wi, (void*)&wc, (void*)&wr, (void*)&b->nwork,
                    (void*)&pli, (void*)&plp, (void*)&b->npatch,
                    (void*)&b->d_part, (void*)&b->d_g, (void*)&b->n, (void*)&max_iter, (void*)&tol};
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(256);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = b->s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelExC(&cfg, kernel_for(ty, b->sw), args);
}

static std::string cache_path(const char* given) {
    if (given && *given) return given;
    const char* env = std::getenv("STOKES_AUTOTUNE_CACHE");
    if (env && *env) return env;
    const char* home = std::getenv("HOME");
    return std::string(home ? home : ".") + "/.cache/libstokes_autotune.txt";
}

// Cache file: one line per key, "key ty cps us_per_iter".
static bool cache_lookup(const std::string& path, const std::string& key, int& ty, int& cps, double& us) {
    std::ifstream f(path);
    std::string line;
    while (std::getline(f, line)) {
        std::istringstream is(line);
        std::string k;
        int a, c;
        double u;
        if (is >> k >> a >> c >> u && k == key && (a == 4 || a == 8 || a == 16) && c >= 1) {
            ty = a; cps = c; us = u;
            return true;
        }
    }
    return false;
}

static void cache_store(const std::string& path, const std::string& key, int ty, int cps, double us) {
    std::vector<std::string> keep;
    {
        std::ifstream f(path);
        std::string line;
        while (std::getline(f, line))
            if (line.compare(0, key.size() + 1, key + " ") != 0) keep.push_back(line);
    }
    std::string dir = path.substr(0, path.find_last_of('/'));
    if (!dir.empty() && dir != path) { std::string cmd = "mkdir -p '" + dir + "' 2>/dev/null"; (void)!system(cmd.c_str()); }
    std::ofstream f(path, std::ios::trunc);
    for (auto& l : keep) f << l << "\n";
    f << key << " " << ty << " " << cps << " " << us << "\n";
}

static std::string tune_key(stokes_batch b) {
    long long slots = 0;
    for (auto* c : b->c) slots += (long long)c->L.P * c->L.R;
    int lg = 0;
    while ((1LL << (lg + 1)) <= slots) ++lg;
    cudaDeviceProp p{};
    int dev = 0;
    cudaGetDevice(&dev);
    cudaGetDeviceProperties(&p, dev);
    std::string gpu = p.name;
    for (auto& ch : gpu) if (ch == ' ') ch = '_';
    return std::string(b->sw ? "batch2d_fp64_schwarz_n" : "batch2d_fp64_n") + std::to_string(b->n) + "_slots2^" +
           std::to_string(lg) + "_" + gpu;
}

static cudaError_t autotune(stokes_batch b, const char* cache) {
    std::string path = cache_path(cache), key = tune_key(b);
    int ty, cps;
    double us;
    if (cache_lookup(path, key, ty, cps, us) && cps <= max_ctas_per_sm(ty, b->sw)) {
        b->ty = ty; b->cps = cps; b->tuned_us = us;
        return upload_plan(b, ty);
    }
    const int sms = num_sms();
    const int iters = 24;
    double best = 1e30;
    int bt = 8, bc = 1;
    for (int t : {4, 8, 16}) {
        cudaError_t e = upload_plan(b, t);
        if (e != cudaSuccess) return e;
        int mx = max_ctas_per_sm(t, b->sw);
        for (int c = 1; c <= std::min(mx, 4); ++c) {
            int grid = std::min(sms * c, std::max(1, b->nwork));
            // warm run, then a timed run of a fixed number of iterations
            if ((e = launch_persistent(b, t, grid, 4, 0.0)) != cudaSuccess) return e;
            cudaEventRecord(b->ev0, b->s);
            if ((e = launch_persistent(b, t, grid, iters, 0.0)) != cudaSuccess) return e;
            cudaEventRecord(b->ev1, b->s);
            if ((e = cudaEventSynchronize(b->ev1)) != cudaSuccess) return e;
            float ms = 0.f;
            cudaEventElapsedTime(&ms, b->ev0, b->ev1);
            double per = 1000.0 * ms / iters;
            if (per < best) { best = per; bt = t; bc = c; }
        }
    }
    b->ty = bt; b->cps = bc; b->tuned_us = best;
    cache_store(path, key, bt, bc, best);
    return upload_plan(b, bt);
}

// right-hand sides, the persistent solve, recovery and unpacking, on b->s
static cudaError_t enqueue(stokes_batch b, const stokes_batch_io* io) {
    for (int i = 0; i < b->n; ++i) {
        Ctx* c = b->c[i];
        cudaStream_t keep = c->stream;
        c->stream = b->s;
        launch_rhs(c, io[i].u_star, c->b64);
        c->stream = keep;
    }
    launch_persistent(b, b->ty, b->grid, b->opt.max_iter, b->opt.tol);
    for (int i = 0; i < b->n; ++i) {
        Ctx* c = b->c[i];
        cudaStream_t keep = c->stream;
        c->stream = b->s;
        launch_recover(c, io[i].u_star, c->x64, io[i].u_out);
        double* outs[6];
        for (int f = 0; f < c->nf - 1; ++f) outs[f] = io[i].tau_out[f];
        outs[c->nf - 1] = io[i].p_out;
        launch_unpack(c, c->x64, outs, 1);
        c->stream = keep;
    }
    return cudaGetLastError();
}

// Capture enqueue() into a CUDA graph; if the cooperative launch cannot be
// captured, fall back to enqueueing directly on every solve.
static cudaError_t capture(stokes_batch b, const stokes_batch_io* io) {
    cudaError_t e;
    if (b->graph) { cudaGraphExecDestroy(b->graph); b->graph = nullptr; }
    const int sms = num_sms();
    b->grid = std::min(sms * b->cps, std::max(1, b->nwork));
    if ((e = cudaStreamBeginCapture(b->s, cudaStreamCaptureModeRelaxed)) != cudaSuccess) return e;
    cudaError_t ee = enqueue(b, io);
    cudaGraph_t g = nullptr;
    e = cudaStreamEndCapture(b->s, &g);
    if (ee == cudaSuccess && e == cudaSuccess) e = cudaGraphInstantiate(&b->graph, g, 0);
    if (g) cudaGraphDestroy(g);
    if (ee != cudaSuccess || e != cudaSuccess) {
        cudaGetLastError();
        b->use_graph = false;
        b->graph = nullptr;
    }
    return cudaSuccess;
}

static std::vector<const void*> io_pointers(const stokes_batch_io* io, int n) {
    std::vector<const void*> v;
    for (int i = 0; i < n; ++i) {
        for (int d = 0; d < 2; ++d) { v.push_back(io[i].u_star[d]); v.push_back(io[i].u_out[d]); }
        for (int f = 0; f < 2; ++f) v.push_back(io[i].tau_out[f]);
        v.push_back(io[i].p_out);
    }
    return v;
}

extern "C" {

stokes_status stokes_batch_destroy(stokes_batch b) {
    if (!b) return STOKES_OK;
    if (b->graph) cudaGraphExecDestroy(b->graph);
    cudaFree(b->d_inst); cudaFree(b->d_st); cudaFree(b->d_g); cudaFree(b->d_wl); cudaFree(b->d_part);
    cudaFree(b->d_st0); cudaFree(b->d_g0);
    if (b->d_pl) cudaFree(b->d_pl);
    if (b->ev0) cudaEventDestroy(b->ev0);
    if (b->ev1) cudaEventDestroy(b->ev1);
    if (b->s) cudaStreamDestroy(b->s);
    delete b;
    return STOKES_OK;
}

stokes_status stokes_batch_create(stokes_batch* out, int n, const stokes_ctx* ctxs, const stokes_options* opt,
                                  const char* tune_cache) {
    if (!out || n < 1 || !ctxs || !opt) return STOKES_ERR_ARG;
    *out = nullptr;
    auto* b = new stokes_batch_s();
    b->n = n;
    b->opt = *opt;
    b->sw = opt->precond == 2;
    for (int i = 0; i < n; ++i) {
        if (!ctxs[i] || ctxs[i]->c.L.dim != 2 || !ctxs[i]->c.have_weights) {
            delete b;
            return STOKES_ERR_ARG;
        }
        b->ctx.push_back(ctxs[i]);
        b->c.push_back(&ctxs[i]->c);
        cudaStreamSynchronize(ctxs[i]->c.stream);
    }
    cudaError_t e = cudaStreamCreate(&b->s);
    if (e == cudaSuccess) e = cudaMalloc(&b->d_inst, n * sizeof(BInst));
    if (e == cudaSuccess) e = cudaMalloc(&b->d_st, n * sizeof(BState));
    if (e == cudaSuccess) e = cudaMalloc(&b->d_g, sizeof(BGlobal));
    if (e == cudaSuccess) e = cudaEventCreate(&b->ev0);
    if (e == cudaSuccess) e = cudaEventCreate(&b->ev1);
    if (e == cudaSuccess) e = cudaMalloc(&b->d_st0, n * sizeof(BState));
    if (e == cudaSuccess) e = cudaMalloc(&b->d_g0, sizeof(BGlobal));
    // tuning runs real CG iterations: give every instance a nonzero
    // right-hand side (the Jacobi diagonal; every solve overwrites it)
    for (int i = 0; i < n && e == cudaSuccess; ++i)
        e = cudaMemcpyAsync(b->c[i]->b64, b->c[i]->A.minv64, sizeof(double) * b->c[i]->vec_elems(),
                            cudaMemcpyDeviceToDevice, b->s);
    if (e == cudaSuccess) e = autotune(b, tune_cache);
    // the tuning runs may have covered slots (inactive ones in coarser tiles)
    // that the chosen work list never initialises: clear every vector they
    // wrote, so the unpacked solution is zero on inactive unknowns
    for (int i = 0; i < n && e == cudaSuccess; ++i) {
        Ctx* c = b->c[i];
        const size_t bytes = sizeof(double) * c->vec_elems();
        double* vs[] = {c->x64, c->b64, c->w64.r, c->w64.z, c->w64.q, c->w64.p[0], c->w64.p[1]};
        for (double* v : vs)
            if (e == cudaSuccess) e = cudaMemsetAsync(v, 0, bytes, b->s);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->s);
    if (e != cudaSuccess) {
        if (std::getenv("STOKES_VERBOSE")) std::fprintf(stderr, "stokes_batch_create: %s\n", cudaGetErrorString(e));
        cudaGetLastError();   // leave no pending error for later calls
        stokes_batch_destroy(b);
        return STOKES_ERR_CUDA;
    }
    b->h_st.resize(n);
    *out = b;
    return STOKES_OK;
}

stokes_status stokes_batch_tuning(stokes_batch b, int* tile_rows, int* ctas_per_sm, double* us_per_iter,
                                  int* graph_captured) {
    if (!b) return STOKES_ERR_ARG;
    if (graph_captured) *graph_captured = b->use_graph && b->graph ? 1 : 0;
    if (tile_rows) *tile_rows = b->ty;
    if (ctas_per_sm) *ctas_per_sm = b->cps;
    if (us_per_iter) *us_per_iter = b->tuned_us;
    return STOKES_OK;
}

stokes_status stokes_batch_solve(stokes_batch b, const stokes_batch_io* io, stokes_stats* stats, double* ms) {
    if (!b || !io) return STOKES_ERR_ARG;
    for (int i = 0; i < b->n; ++i) {
        if (!io[i].u_star[0] || !io[i].u_star[1] || !io[i].u_out[0] || !io[i].u_out[1] || !io[i].tau_out[0] ||
            !io[i].tau_out[1] || !io[i].p_out)
            return STOKES_ERR_ARG;
        cudaStreamSynchronize(b->c[i]->stream);
    }
    cudaError_t e = cudaSuccess;
    if (b->sw) {
        // the contexts' Schwarz plans are rebuilt (all their buffers
        // reallocated) after every weight build: refresh the instance table
        // and patch list when any plan was rebuilt since the last upload.
        // (Comparing one buffer's address is not enough: the allocator may
        // hand that one back at the same address and move the others.)
        bool moved = false;
        for (int i = 0; i < b->n; ++i) {
            const SchwarzPlan* P = nullptr;
            if ((e = schwarz_ensure(b->c[i], &P)) != cudaSuccess) return STOKES_ERR_CUDA;
            moved |= (int)b->plan_epoch.size() != b->n || b->c[i]->sw_epoch != b->plan_epoch[i];
        }
        if (moved && (e = upload_plan(b, b->ty)) != cudaSuccess) return STOKES_ERR_CUDA;
    }
    auto key = io_pointers(io, b->n);
    if (b->use_graph && (!b->graph || key != b->io_key)) {
        e = capture(b, io);
        if (e != cudaSuccess) return STOKES_ERR_CUDA;
        b->io_key = key;
    }
    if (!b->use_graph) b->grid = std::min(num_sms() * b->cps, std::max(1, b->nwork));
    cudaEventRecord(b->ev0, b->s);
    e = b->use_graph ? cudaGraphLaunch(b->graph, b->s) : enqueue(b, io);
    cudaEventRecord(b->ev1, b->s);
    if (e == cudaSuccess) e = cudaEventSynchronize(b->ev1);
    if (e != cudaSuccess) return STOKES_ERR_CUDA;
    float t = 0.f;
    cudaEventElapsedTime(&t, b->ev0, b->ev1);
    if (ms) *ms = t;
    BGlobal g{};
    cudaMemcpy(&g, b->d_g, sizeof(g), cudaMemcpyDeviceToHost);
    cudaMemcpy(b->h_st.data(), b->d_st, b->n * sizeof(BState), cudaMemcpyDeviceToHost);
    int worst = STOKES_OK;
    for (int i = 0; i < b->n; ++i) {
        const BState& s = b->h_st[i];
        if (stats) {
            stokes_stats& o = stats[i];
            std::memset(&o, 0, sizeof(o));
            o.status = g.err ? g.err : s.status;
            o.iterations = s.iter;
            o.outer = 1;
            o.rel_residual = s.bb > 0 ? std::sqrt(s.rr / s.bb) : 0.0;
            o.ms_solve = t;
            o.precision_used = STOKES_FP64;
        }
        if (s.status != STOKES_OK && worst == STOKES_OK) worst = s.status;
    }
    if (g.err) return (stokes_status)g.err;
    return (stokes_status)worst;
}

stokes_status stokes_solve_batched(int n, const stokes_ctx* ctxs, const stokes_batch_io* io, const stokes_options* opt,
                                   stokes_stats* stats) {
    stokes_batch b = nullptr;
    stokes_status s = stokes_batch_create(&b, n, ctxs, opt, nullptr);
    if (s != STOKES_OK) return s;
    s = stokes_batch_solve(b, io, stats, nullptr);
    stokes_batch_destroy(b);
    return s;
}

}  // extern "C"
