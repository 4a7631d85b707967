// Context of one grid: layout, device arrays and solver work space.
#pragma once
#include <string>
#include <vector>
#include "internal.cuh"

namespace stk {

struct Ptr3 { const double* p[3]; };
struct Ptr4 { const double* p[4]; };

// Device pointers handed to the build kernels (plain struct, passed by value).
struct DevArrays {
    double* WL[7];
    double* WF[7];
    uint8_t* fflag[3];
    double* effWF[3];
    double* K64[3];
    double* rec[3];       // dt / (rho W_L) on live faces (velocity recovery)
    double* ubc[3];
    uint8_t* act[4];      // activity of unknown sites: cell, then stress sites
    double* coef64;
    float* coef32;
    __nv_bfloat16* coef16;
    uint32_t* pair16;     // 2D: coef16 in pairs (see Coef)
    uint2* quad16;        // 3D: coef16 in fours (see Coef)
    double* minv64;
    float* minv32;
    uint8_t* tile_flag;
    uint8_t* tile_flag4;  // 2D: activity of 32 x 4 tiles (batched solver plans)
    uint8_t* unit_mask;   // 3D: active tiles of each apply unit (bit mask, see UY3)
};

// Learned-preconditioner state of a context (fpcg.cu).
struct LearnedState {
    struct stokes_net_s* net = nullptr;
    float* feat = nullptr;     // network input (D, H, W, cin)
    float* out = nullptr;      // network output (D, H, W, cout)
    float* zold = nullptr;     // previous preconditioned residual
    double* norm = nullptr;
    double* dots = nullptr;
    int64_t n_active = 0;
    const uint8_t** d_act = nullptr;   // device copy of the activity pointers
};

// Work vectors of one precision.
template <class T> struct CgWork {
    T *x = nullptr, *r = nullptr, *z = nullptr, *p[2] = {nullptr, nullptr}, *q = nullptr;
};

struct Ctx {
    stokes_grid g{};
    Layout L{};
    cudaStream_t stream = nullptr;
    int device = 0;
    std::string err;
    int nf = 0;        // unknown fields
    int nk = 0;        // sample kinds
    int nd = 0;        // face kinds
    int nsite = 0;     // unknown sites (cell + stress sites)
    int ncoef = 0;
    int ntiles_all = 0;
    int ntiles_active = 0;
    int* tiles = nullptr;       // active tile list (device)
    int* d_ntiles = nullptr;
    int nunits_all = 0;         // 3D apply units of the grid at depth 1 (the most there can be)
    int unit_zt = ZT_MAX;       // depth of the current units (tile layers), chosen at weight build
    int nunits_active = 0;
    int* units = nullptr;       // active unit list (device, 3D)
    int* d_nunits = nullptr;
    bool have_weights = false;
    double min_face_liquid = 0.0;   // floor of the live faces' mass fraction (next weight build)
    bool own_stream = false;
    std::vector<void*> allocs;
    DevArrays A{};
    void* weight_block = nullptr;
    size_t weight_bytes = 0;
    // solver state
    CgScalars* sc = nullptr;     // [0] inner/plain CG, [1] outer
    CgScalars* h_sc = nullptr;   // pinned host mirror
    double* partial = nullptr;   // per-block partials (2 arrays)
    unsigned* counter = nullptr;
    CgWork<double> w64;
    CgWork<float> w32;
    double* b64 = nullptr;       // rhs (solve_step)
    double* x64 = nullptr;       // solution (solve_step)
    double* y64 = nullptr;       // scratch
    cudaEvent_t ev[4]{};
    double last_apply_ms = -1.0;
    cudaGraphExec_t graph[4] = {nullptr, nullptr, nullptr, nullptr};  // inner solve per precision (+ Schwarz)
    LearnedState learned;
    long learned_jacobi_steps = 0;
    int wait_test = 0;          // options.wait_test of the solve in progress (0 outside a solve)
    // additive Schwarz preconditioner (2D), rebuilt lazily after each weight build
    struct SchwarzPlan* sw = nullptr;
    std::vector<void*> sw_allocs;
    bool sw_ready = false;
    unsigned sw_epoch = 0;       // incremented by every plan build (its buffers are reallocated)
    double sw_setup_ms = 0.0;
    // transport step (advect.cu): staged velocity and validity, allocated on first use
    void* adv_scratch = nullptr;

    DevArrays dev_arrays() const { return A; }
    // arguments of an apply over the active tiles (3D: the active units)
    ApplyArgs apply_args() const {
        ApplyArgs a{};
        a.units = units;
        a.umask = A.unit_mask;
        a.nunits = nunits_active;
        a.zt = unit_zt;
        return a;
    }
    cudaError_t zero_weights() { return cudaMemsetAsync(weight_block, 0, weight_bytes, stream); }
    template <class C> Coef<C> coef() const;
    int64_t vec_elems() const { return (int64_t)nf * L.stride; }
};

template <> inline Coef<double> Ctx::coef<double>() const {
    Coef<double> c{};
    for (int f = 0; f < ncoef; ++f) c.f[f] = A.coef64 + (int64_t)f * L.stride;
    return c;
}
template <> inline Coef<float> Ctx::coef<float>() const {
    Coef<float> c{};
    for (int f = 0; f < ncoef; ++f) c.f[f] = A.coef32 + (int64_t)f * L.stride;
    return c;
}
template <> inline Coef<__nv_bfloat16> Ctx::coef<__nv_bfloat16>() const {
    Coef<__nv_bfloat16> c{};
    for (int f = 0; f < ncoef; ++f) c.f[f] = A.coef16 + (int64_t)f * L.stride;
    if (L.dim == 2 && A.pair16)
        for (int k = 0; k < 3; ++k) c.pr[k] = A.pair16 + (int64_t)k * L.stride;
    if (L.dim == 3 && A.quad16)
        for (int k = 0; k < 2; ++k) c.qd[k] = A.quad16 + (int64_t)k * L.stride;
    return c;
}

template <class T, class C>
cudaError_t launch_apply_mode(const Layout& L, const int* tiles, int ntiles, const Coef<C>& cf, const T* x, T* y,
                              int mode, const ApplyArgs& a, cudaStream_t s);

}  // namespace stk

struct stokes_ctx_s {
    stk::Ctx c;
};
