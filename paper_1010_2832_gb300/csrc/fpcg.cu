// Flexible preconditioned CG with the learned network as preconditioner.
//
// Network input at slot (i, j[, k]) -> voxel (k, j, i), channels:
//   [ s * sqrt(m_f) r_f  for each unknown field f ]  (Jacobi-scaled residual,
//                                                     unit RMS over the grid)
//   [ log(m_f) / 16      for each unknown field f ]  (operator information)
//   zero channels up to the network's cin;
// m_f is the Jacobi inverse diagonal (1 on inactive unknowns, 0 on padding).
// The network corrects the Jacobi step: output channel f gives
// z_f = m_f r_f + sqrt(m_f) out_f / s on active unknowns (a zero network is
// plain Jacobi); an inactive unknown keeps z = r (its row is the identity).
// Training targets are therefore the part of the error that the Jacobi step
// misses, e - M_J A e, in the same scaling.
//
// Flexible CG (Polak-Ribiere): beta = r_{k+1}.(z_{k+1} - z_k) / r_k.z_k, so a
// preconditioner that is not a fixed linear operator still gives a
// convergent method; if the network direction fails r.z > 0 the iteration
// falls back to the Jacobi direction for that step, and if the residual norm
// does not halve within 100 iterations the rest of the inner solve is plain
// Jacobi-PCG.  Vectors are FP32; the
// refinement loop around it (pcg.cu) recomputes the true residual in FP64.
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <vector>
#include "internal.cuh"
#include "ctx.cuh"

#include <algorithm>

namespace stk {

struct NetGrid { int D, H, W, cin, cout; };

__device__ __forceinline__ void slot_of(const Layout& L, int64_t v, const NetGrid& g, int& i, int& j, int& k) {
    i = v % g.W; j = (v / g.W) % g.H; k = v / ((int64_t)g.W * g.H);
}

// sum over active real slots of m_f r_f^2 (for the RMS scaling)
__global__ void k_feat_norm(Layout L, int nf, const float* r, const float* minv, NetGrid g, double* out) {
    int64_t nv = (int64_t)g.D * g.H * g.W;
    double s = 0.0;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < nv; v += (int64_t)gridDim.x * blockDim.x) {
        int i, j, k;
        slot_of(L, v, g, i, j, k);
        if (i > L.nx || j > L.ny || k > (L.dim == 3 ? L.nz : 0)) continue;
        int64_t o = L.off(i + 1, j + 1, L.dim == 3 ? k + 1 : 0);
        for (int f = 0; f < nf; ++f) {
            float m = minv[(int64_t)f * L.stride + o], x = r[(int64_t)f * L.stride + o];
            s += (double)m * x * x;
        }
    }
    s = warp_sum(s);
    if ((threadIdx.x & 31) == 0) atomicAdd(out, s);
}

template <class Tin>
__global__ void k_features(Layout L, int nf, const Tin* r, const float* minv, NetGrid g, const double* norm,
                           double count, float* x) {
    int64_t nv = (int64_t)g.D * g.H * g.W;
    int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= nv) return;
    double rms = sqrt(*norm / fmax(count, 1.0));
    float s = rms > 0 ? (float)(1.0 / rms) : 0.f;
    int i, j, k;
    slot_of(L, v, g, i, j, k);
    float* xo = x + v * g.cin;
    bool real = i <= L.nx && j <= L.ny && k <= (L.dim == 3 ? L.nz : 0);
    int64_t o = real ? L.off(i + 1, j + 1, L.dim == 3 ? k + 1 : 0) : 0;
    for (int c = 0; c < g.cin; ++c) {
        float val = 0.f;
        if (real && c < nf) {
            float m = minv[(int64_t)c * L.stride + o];
            val = s * sqrtf(m) * (float)r[(int64_t)c * L.stride + o];
        } else if (real && c < 2 * nf) {
            float m = minv[(int64_t)(c - nf) * L.stride + o];
            val = m > 0.f ? logf(m) / 16.f : 0.f;
        }
        xo[c] = val;
    }
}

// z from the network output (active unknowns), z = r on inactive unknowns
__global__ void k_unfeatures(Layout L, int nf, const float* out, const float* r, const float* minv,
                             const uint8_t* const* act_site, NetGrid g, const double* norm, double count, float* z) {
    int64_t nv = (int64_t)g.D * g.H * g.W;
    int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= nv) return;
    int i, j, k;
    slot_of(L, v, g, i, j, k);
    if (i > L.nx || j > L.ny || k > (L.dim == 3 ? L.nz : 0)) return;
    double rms = sqrt(*norm / fmax(count, 1.0));
    float inv_s = (float)rms;
    int64_t o = L.off(i + 1, j + 1, L.dim == 3 ? k + 1 : 0);
    for (int f = 0; f < nf; ++f) {
        int site = L.dim == 2 ? (f == 1 ? 1 : 0) : (f <= 1 || f == 5 ? 0 : f - 1);
        int64_t of = (int64_t)f * L.stride + o;
        float m = minv[of];
        float zz;
        if (act_site[site][o]) zz = m * r[of] + sqrtf(m) * out[v * g.cout + f] * inv_s;
        else zz = m > 0.f ? r[of] : 0.f;
        z[of] = zz;
    }
}

__global__ void k_scaled_copy(Layout L, int nf, const float* in, float s, float* out, int64_t n) {
    int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e < n) out[e] = in[e] * s;
}

// dots over active tiles: r.a, r.b, r.r  (three partials, last block reduces)
__global__ void __launch_bounds__(256) k_dots3(Layout L, const int* __restrict__ tiles, int nf, const float* r,
                                               const float* a, const float* b, double* partial, unsigned* counter,
                                               int nblocks, double* out3) {
    const int tile = tiles[blockIdx.x];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    double s0 = 0, s1 = 0, s2 = 0;
    const int nrow = L.dim == 2 ? TY2 : TY3 * TZ3;
    for (int row = warp; row < nrow; row += 8) {
        int tcx = tile % L.ntx;
        int64_t o;
        if (L.dim == 2) o = L.off(tcx * TX, (tile / L.ntx) * TY2 + row, 0);
        else {
            int rest = tile / L.ntx;
            o = L.off(tcx * TX, (rest % L.nty) * TY3 + row % TY3, (rest / L.nty) * TZ3 + row / TY3);
        }
        o += lane;
        for (int f = 0; f < nf; ++f) {
            int64_t of = (int64_t)f * L.stride + o;
            double rv = r[of];
            s0 += rv * a[of]; s1 += rv * b[of]; s2 += rv * rv;
        }
    }
    __shared__ double red[3][8];
    __shared__ bool last;
    s0 = warp_sum(s0); s1 = warp_sum(s1); s2 = warp_sum(s2);
    if (lane == 0) { red[0][warp] = s0; red[1][warp] = s1; red[2][warp] = s2; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double t0 = 0, t1 = 0, t2 = 0;
        for (int q = 0; q < 8; ++q) { t0 += red[0][q]; t1 += red[1][q]; t2 += red[2][q]; }
        partial[3 * blockIdx.x] = t0; partial[3 * blockIdx.x + 1] = t1; partial[3 * blockIdx.x + 2] = t2;
        __threadfence();
        last = atomicAdd(counter, 1u) == (unsigned)nblocks - 1u;
    }
    __syncthreads();
    if (!last) return;
    if (threadIdx.x == 0) {
        __threadfence();
        double t0 = 0, t1 = 0, t2 = 0;
        for (int q = 0; q < nblocks; ++q) {
            t0 += ((volatile double*)partial)[3 * q];
            t1 += ((volatile double*)partial)[3 * q + 1];
            t2 += ((volatile double*)partial)[3 * q + 2];
        }
        out3[0] = t0; out3[1] = t1; out3[2] = t2;
        *counter = 0u;
    }
}

// x += alpha p, r -= alpha q  (no preconditioning)
__global__ void __launch_bounds__(256) k_xr_update(Layout L, const int* __restrict__ tiles, int nf, float* x, float* r,
                                                   const float* p, const float* q, const CgScalars* sc) {
    const int tile = tiles[blockIdx.x];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const float alpha = (float)sc->alpha;
    const int nrow = L.dim == 2 ? TY2 : TY3 * TZ3;
    for (int row = warp; row < nrow; row += 8) {
        int tcx = tile % L.ntx;
        int64_t o;
        if (L.dim == 2) o = L.off(tcx * TX, (tile / L.ntx) * TY2 + row, 0);
        else {
            int rest = tile / L.ntx;
            o = L.off(tcx * TX, (rest % L.nty) * TY3 + row % TY3, (rest / L.nty) * TZ3 + row / TY3);
        }
        o += lane;
        for (int f = 0; f < nf; ++f) {
            int64_t of = (int64_t)f * L.stride + o;
            x[of] += alpha * p[of];
            r[of] -= alpha * q[of];
        }
    }
}

__global__ void k_jacobi_dir(int64_t n, const float* r, const float* minv, float* z) {
    int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e < n) z[e] = minv[e] * r[e];
}

// r32 = scale * r64 on every element (pads are zero in both)
__global__ void k_narrow(int64_t n, const double* r64, double scale, float* r32) {
    int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e < n) r32[e] = (float)(r64[e] * scale);
}

static unsigned nb256(int64_t n) { return (unsigned)((n + 255) / 256); }

NetGrid net_grid(Ctx* c) {
    const Layout& L = c->L;
    NetGrid g;
    auto up4 = [](int v) { return (v + 3) / 4 * 4; };
    g.W = up4(L.nx + 1);
    g.H = up4(L.ny + 1);
    g.D = L.dim == 3 ? up4(L.nz + 1) : 1;
    g.cin = L.dim == 2 ? 8 : 12;
    g.cout = L.dim == 2 ? 4 : 8;
    return g;
}

// z = P(r) with the network; returns the count used for the RMS
static cudaError_t precondition(Ctx* c, stokes_net_s* net, const float* r, float* z) {
    const Layout& L = c->L;
    NetGrid g = net_grid(c);
    int64_t nv = (int64_t)g.D * g.H * g.W;
    cudaError_t e;
    double* norm = c->learned.norm;
    if ((e = cudaMemsetAsync(norm, 0, sizeof(double), c->stream)) != cudaSuccess) return e;
    k_feat_norm<<<std::min<int64_t>(nb256(nv), 4096), 256, 0, c->stream>>>(L, c->nf, r, c->A.minv32, g, norm);
    double count = (double)c->learned.n_active;
    k_features<float><<<nb256(nv), 256, 0, c->stream>>>(L, c->nf, r, c->A.minv32, g, norm, count, c->learned.feat);
    // the network runs on its own stream: order it after our work
    if ((e = cudaStreamSynchronize(c->stream)) != cudaSuccess) return e;
    if (stokes_net_forward(net, 1, g.D, g.H, g.W, c->learned.feat, c->learned.out) != STOKES_OK)
        return cudaErrorLaunchFailure;
    const uint8_t* const* act = c->learned.d_act;
    k_unfeatures<<<nb256(nv), 256, 0, c->stream>>>(L, c->nf, c->learned.out, r, c->A.minv32, act, g, norm, count, z);
    return cudaGetLastError();
}

// One inner flexible-CG solve on A32 d = scale * r64 with the learned
// preconditioner; host-driven (the network is several launches per step).
cudaError_t run_inner_fpcg(Ctx* c, stokes_net_s* net, double scale, double tol_rel, int max_iter, int* iters,
                           int* jacobi_steps) {
    const Layout& L = c->L;
    cudaStream_t s = c->stream;
    const int nb = c->ntiles_active;
    const int64_t V = c->vec_elems();
    CgWork<float>& w = c->w32;
    float* zold = c->learned.zold;
    double* d3 = c->learned.dots;
    double h3[3];
    cudaError_t e;
    k_narrow<<<nb256(V), 256, 0, s>>>(V, c->w64.r, scale, w.r);
    cudaMemsetAsync(w.x, 0, sizeof(float) * V, s);
    cudaMemsetAsync(w.p[0], 0, sizeof(float) * V, s);
    if ((e = precondition(c, net, w.r, w.z)) != cudaSuccess) return e;
    k_dots3<<<nb, 256, 0, s>>>(L, c->tiles, c->nf, w.r, w.z, w.z, c->partial, c->counter, nb, d3);
    cudaMemcpyAsync(h3, d3, sizeof(h3), cudaMemcpyDeviceToHost, s);
    if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return e;
    double rr0 = h3[2], rz = h3[0];
    int jac = 0;
    if (!(rz > 0)) {
        k_jacobi_dir<<<nb256(V), 256, 0, s>>>(V, w.r, c->A.minv32, w.z);
        k_dots3<<<nb, 256, 0, s>>>(L, c->tiles, c->nf, w.r, w.z, w.z, c->partial, c->counter, nb, d3);
        cudaMemcpyAsync(h3, d3, sizeof(h3), cudaMemcpyDeviceToHost, s);
        cudaStreamSynchronize(s);
        rz = h3[0];
        ++jac;
    }
    CgScalars hs{};
    hs.beta = 0.0;
    hs.rz = rz;
    hs.max_iter = max_iter;
    int it = 0;
    const double tol2 = tol_rel * tol_rel * rr0;
    double rr = rr0;
    // progress check: every FPCG_WINDOW iterations the residual norm must at
    // least halve, else the rest of this solve uses the Jacobi direction
    // (plain PCG), so a poor network costs at most one window
    constexpr int FPCG_WINDOW = 100;
    bool jacobi_only = false;
    int win_it = 0;
    double win_rr = rr0;
    while (it < max_iter && rr > tol2 && rr0 > 0) {
        // p = z + beta p_old, q = A p, alpha = rz / p.q
        cudaMemcpyAsync(c->sc, &hs, sizeof(CgScalars), cudaMemcpyHostToDevice, s);
        ApplyArgs a = c->apply_args();
        a.pold = w.p[it & 1];
        a.pnew = w.p[(it & 1) ^ 1];
        a.partial = c->partial;
        a.counter = c->counter;
        a.sc = c->sc;
        if ((e = launch_apply_mode<float, float>(L, c->tiles, nb, c->coef<float>(), w.z, w.q, MODE_CG, a, s)) !=
            cudaSuccess)
            return e;
        k_xr_update<<<nb, 256, 0, s>>>(L, c->tiles, c->nf, w.x, w.r, w.p[(it & 1) ^ 1], w.q, c->sc);
        cudaMemcpyAsync(zold, w.z, sizeof(float) * V, cudaMemcpyDeviceToDevice, s);
        if (jacobi_only) {
            k_jacobi_dir<<<nb256(V), 256, 0, s>>>(V, w.r, c->A.minv32, w.z);
            ++jac;
        } else if ((e = precondition(c, net, w.r, w.z)) != cudaSuccess) {
            return e;
        }
        k_dots3<<<nb, 256, 0, s>>>(L, c->tiles, c->nf, w.r, w.z, zold, c->partial, c->counter, nb, d3);
        cudaMemcpyAsync(h3, d3, sizeof(h3), cudaMemcpyDeviceToHost, s);
        CgScalars back{};
        cudaMemcpyAsync(&back, c->sc, sizeof(CgScalars), cudaMemcpyDeviceToHost, s);
        if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return e;
        ++it;
        const bool verbose = std::getenv("STOKES_VERBOSE") != nullptr;
        if (verbose && (it <= 5 || it % 100 == 0 || back.done))
            std::fprintf(stderr, "[stokes] fpcg it %d rr/rr0 %.3e r.z %.3e r.zold %.3e alpha %.3e pq %.3e done %d\n", it,
                         h3[2] / rr0, h3[0], h3[1], back.alpha, back.pq, back.done);
        if (back.done) break;   // p.Ap <= 0: breakdown
        rr = h3[2];
        double rz_new = h3[0], rz_old = h3[1];
        if (!(rz_new > 0)) {
            k_jacobi_dir<<<nb256(V), 256, 0, s>>>(V, w.r, c->A.minv32, w.z);
            k_dots3<<<nb, 256, 0, s>>>(L, c->tiles, c->nf, w.r, w.z, zold, c->partial, c->counter, nb, d3);
            cudaMemcpyAsync(h3, d3, sizeof(h3), cudaMemcpyDeviceToHost, s);
            cudaStreamSynchronize(s);
            rz_new = h3[0]; rz_old = h3[1];
            ++jac;
        }
        hs.beta = std::fmax(0.0, (rz_new - rz_old) / hs.rz);
        hs.rz = rz_new;
        hs.done = 0;
        if (!jacobi_only && it - win_it >= FPCG_WINDOW) {
            if (rr > 0.25 * win_rr) {
                jacobi_only = true;
                if (verbose) std::fprintf(stderr, "[stokes] fpcg it %d: residual fell %.2fx in %d steps, Jacobi from here\n",
                                          it, std::sqrt(win_rr / rr), FPCG_WINDOW);
            }
            win_it = it;
            win_rr = rr;
        }
    }
    // hand the result to the refinement loop like the Jacobi path does
    CgScalars res{};
    res.scale = scale;
    res.iter = it;
    res.status = STOKES_OK;
    cudaMemcpyAsync(c->sc, &res, sizeof(CgScalars), cudaMemcpyHostToDevice, s);
    *iters = it;
    *jacobi_steps = jac;
    return cudaStreamSynchronize(s);
}

// training targets: y_f = e_f / (sqrt(m_f) rms) on active unknowns, else 0
__global__ void k_targets(Layout L, int nf, const double* e, const float* minv, const uint8_t* const* act_site,
                          NetGrid g, double rms, float* y) {
    int64_t nv = (int64_t)g.D * g.H * g.W;
    int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= nv) return;
    int i, j, k;
    slot_of(L, v, g, i, j, k);
    bool real = i <= L.nx && j <= L.ny && k <= (L.dim == 3 ? L.nz : 0);
    int64_t o = real ? L.off(i + 1, j + 1, L.dim == 3 ? k + 1 : 0) : 0;
    for (int c = 0; c < g.cout; ++c) {
        float val = 0.f;
        if (real && c < nf) {
            int site = L.dim == 2 ? (c == 1 ? 1 : 0) : (c <= 1 || c == 5 ? 0 : c - 1);
            float m = minv[(int64_t)c * L.stride + o];
            if (act_site[site][o] && m > 0.f && rms > 0) val = (float)(e[(int64_t)c * L.stride + o] / (sqrt((double)m) * rms));
        }
        y[v * g.cout + c] = val;
    }
}

}  // namespace stk

using namespace stk;

extern "C" {

stokes_status stokes_learned_grid(stokes_ctx h, int* D, int* H, int* W, int* cin, int* cout) {
    if (!h) return STOKES_ERR_ARG;
    NetGrid g = net_grid(&h->c);
    if (D) *D = g.D;
    if (H) *H = g.H;
    if (W) *W = g.W;
    if (cin) *cin = g.cin;
    if (cout) *cout = g.cout;
    return STOKES_OK;
}

// Attach a network as the learned preconditioner of a context (weights must
// be built; re-attach after every stokes_build_weights).  NULL detaches.
stokes_status stokes_set_learned_preconditioner(stokes_ctx h, stokes_net_s* net) {
    if (!h) return STOKES_ERR_ARG;
    Ctx& c = h->c;
    if (!net) { c.learned.net = nullptr; return STOKES_OK; }
    if (!c.have_weights) { c.err = "stokes_build_weights has not run"; return STOKES_ERR_STATE; }
    NetGrid g = net_grid(&c);
    int64_t nv = (int64_t)g.D * g.H * g.W;
    auto alloc = [&](void** p, size_t bytes) -> cudaError_t {
        cudaError_t e = cudaMalloc(p, bytes);
        if (e == cudaSuccess) { c.allocs.push_back(*p); e = cudaMemset(*p, 0, bytes); }
        return e;
    };
    cudaError_t e = cudaSuccess;
    if (!c.learned.feat) {
        e = alloc((void**)&c.learned.feat, sizeof(float) * nv * g.cin);
        if (e == cudaSuccess) e = alloc((void**)&c.learned.out, sizeof(float) * nv * g.cout);
        if (e == cudaSuccess) e = alloc((void**)&c.learned.zold, sizeof(float) * c.vec_elems());
        if (e == cudaSuccess) e = alloc((void**)&c.learned.norm, sizeof(double) * 4);
        if (e == cudaSuccess) e = alloc((void**)&c.learned.dots, sizeof(double) * 4);
        if (e == cudaSuccess) e = alloc((void**)&c.learned.d_act, sizeof(uint8_t*) * 4);
    }
    if (e != cudaSuccess) { c.err = "allocation for the learned preconditioner failed"; return STOKES_ERR_CUDA; }
    const uint8_t* acts[4] = {c.A.act[0], c.A.act[1], c.nsite > 2 ? c.A.act[2] : nullptr,
                              c.nsite > 3 ? c.A.act[3] : nullptr};
    cudaMemcpy((void*)c.learned.d_act, acts, sizeof(acts), cudaMemcpyHostToDevice);
    // number of active unknowns (normalises the residual RMS)
    int64_t n = stokes_export_size(h, 3);
    std::vector<uint8_t> a(n);
    uint8_t* d = nullptr;
    if (cudaMalloc(&d, n) != cudaSuccess) return STOKES_ERR_CUDA;
    stokes_export(h, 3, d);
    cudaMemcpy(a.data(), d, n, cudaMemcpyDeviceToHost);
    cudaFree(d);
    int64_t cnt = 0;
    for (auto v : a) cnt += v != 0;
    c.learned.n_active = cnt;
    c.learned.net = net;
    return STOKES_OK;
}

// Network input for an FP64 residual in slot layout (device), and the RMS
// used to normalise it.
stokes_status stokes_learned_features(stokes_ctx h, const double* r, float* x, double* rms) {
    if (!h || !r || !x) return STOKES_ERR_ARG;
    Ctx& c = h->c;
    if (!c.learned.norm) { c.err = "attach a network first"; return STOKES_ERR_STATE; }
    NetGrid g = net_grid(&c);
    int64_t nv = (int64_t)g.D * g.H * g.W;
    // the norm kernel reads FP32: narrow r into the FP32 work vector
    int64_t V = c.vec_elems();
    k_narrow<<<nb256(V), 256, 0, c.stream>>>(V, r, 1.0, c.w32.q);
    cudaMemsetAsync(c.learned.norm, 0, sizeof(double), c.stream);
    k_feat_norm<<<std::min<int64_t>(nb256(nv), 4096), 256, 0, c.stream>>>(c.L, c.nf, c.w32.q, c.A.minv32, g,
                                                                         c.learned.norm);
    k_features<double><<<nb256(nv), 256, 0, c.stream>>>(c.L, c.nf, r, c.A.minv32, g, c.learned.norm,
                                                        (double)c.learned.n_active, x);
    double nrm = 0;
    cudaMemcpyAsync(&nrm, c.learned.norm, sizeof(double), cudaMemcpyDeviceToHost, c.stream);
    if (cudaStreamSynchronize(c.stream) != cudaSuccess) return STOKES_ERR_CUDA;
    if (rms) *rms = std::sqrt(nrm / std::fmax((double)c.learned.n_active, 1.0));
    return STOKES_OK;
}

stokes_status stokes_learned_targets(stokes_ctx h, const double* e, double rms, float* y) {
    if (!h || !e || !y) return STOKES_ERR_ARG;
    Ctx& c = h->c;
    if (!c.learned.d_act) { c.err = "attach a network first"; return STOKES_ERR_STATE; }
    NetGrid g = net_grid(&c);
    int64_t nv = (int64_t)g.D * g.H * g.W;
    k_targets<<<nb256(nv), 256, 0, c.stream>>>(c.L, c.nf, e, c.A.minv32, c.learned.d_act, g, rms, y);
    return cudaStreamSynchronize(c.stream) == cudaSuccess ? STOKES_OK : STOKES_ERR_CUDA;
}

long stokes_learned_jacobi_steps(stokes_ctx h) { return h ? h->c.learned_jacobi_steps : -1; }

}  // extern "C"
