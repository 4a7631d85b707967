// C-ABI entry points of libstokes (declared in include/stokes.h).
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include "internal.cuh"
#include "ctx.cuh"

using namespace stk;


namespace stk {
void set_error(Ctx* c, const std::string& m) { c->err = m; }
cudaError_t launch_unpack(Ctx* c, const double* slots, double* const* fields, int to_fields);
cudaError_t launch_traction(Ctx* c, const double* const* bc_fields, const double* const* ustar, double* const* uout);
void apply_set_attributes();
cudaError_t bench_cg_kernels(Ctx* c, int precision, int launches, double* ms_apply, double* ms_update);
cudaError_t bench_schwarz_kernels(Ctx* c, int launches, double* ms_local, double* ms_gather, double* bytes_local);
cudaError_t apply_preconditioner(Ctx* c, int which, const float* r, float* z);
cudaError_t apply_schwarz_noalloc(Ctx* c, const float* r, float* z, std::string* why);
double schwarz_setup_ms(Ctx* c);
size_t advect_scratch_bytes(const Layout& L);
cudaError_t launch_advect2d(Ctx* c, void* scratch, const double* const* u_in, const double* phi_in, const double* g,
                            int passes, const uint8_t* valid, const double* phi_union, double* const* u_out,
                            double* phi_out);
}  // namespace stk

extern "C" stokes_status stokes_apply_preconditioner(stokes_ctx h, int which, const float* r, float* z) {
    if (!h || !r || !z || r == z || (which != 0 && which != 2)) return STOKES_ERR_ARG;
    Ctx& c = h->c;
    if (!c.have_weights) { c.err = "stokes_build_weights has not run"; return STOKES_ERR_STATE; }
    if (which == 2 && c.L.dim != 2) { c.err = "the Schwarz preconditioner is 2D only"; return STOKES_ERR_ARG; }
    cudaError_t e = apply_preconditioner(&c, which, r, z);
    if (e != cudaSuccess) { c.err = std::string("preconditioner failed: ") + cudaGetErrorString(e); return STOKES_ERR_CUDA; }
    return STOKES_OK;
}

extern "C" double stokes_schwarz_setup_ms(stokes_ctx h) { return h ? schwarz_setup_ms(&h->c) : -1.0; }

// Allocation-free variant of stokes_apply_preconditioner(which = 2); the
// scratch lives in a fixed device array (see apply_schwarz_noalloc).
extern "C" stokes_status stokes_apply_schwarz_noalloc(stokes_ctx h, const float* r, float* z) {
    if (!h || !r || !z || r == z) return STOKES_ERR_ARG;
    Ctx& c = h->c;
    if (!c.have_weights) { c.err = "stokes_build_weights has not run"; return STOKES_ERR_STATE; }
    std::string why;
    cudaError_t e = apply_schwarz_noalloc(&c, r, z, &why);
    if (e == cudaSuccess) return STOKES_OK;
    if (e == cudaErrorNotReady) { c.err = why; return STOKES_ERR_STATE; }
    if (e == cudaErrorInvalidValue) { c.err = why; return STOKES_ERR_ARG; }
    if (e == cudaErrorLaunchTimeout) { c.err = why; return STOKES_ERR_TIMEOUT; }
    c.err = std::string("allocation-free Schwarz apply failed: ") + (why.empty() ? "" : why + ": ") +
            cudaGetErrorString(e);
    return STOKES_ERR_CUDA;
}

extern "C" stokes_status stokes_bench_schwarz_kernels(stokes_ctx h, int launches, double* ms_local,
                                                      double* ms_gather, double* bytes_local) {
    if (!h || !ms_local || !ms_gather || !bytes_local || launches < 1) return STOKES_ERR_ARG;
    Ctx& c = h->c;
    if (!c.have_weights) { c.err = "stokes_build_weights has not run"; return STOKES_ERR_STATE; }
    if (c.L.dim != 2) { c.err = "the Schwarz preconditioner is 2D only"; return STOKES_ERR_ARG; }
    if (c.ntiles_active == 0) { c.err = "no active unknowns"; return STOKES_ERR_STATE; }
    cudaError_t e = bench_schwarz_kernels(&c, launches, ms_local, ms_gather, bytes_local);
    if (e != cudaSuccess) { c.err = std::string("Schwarz kernel timing failed: ") + cudaGetErrorString(e); return STOKES_ERR_CUDA; }
    return STOKES_OK;
}

extern "C" stokes_status stokes_bench_cg_kernels(stokes_ctx h, int precision, int launches, double* ms_apply,
                                                 double* ms_update) {
    if (!h || !ms_apply || !ms_update || launches < 1 || precision < 0 || precision > 2) return STOKES_ERR_ARG;
    Ctx& c = h->c;
    if (!c.have_weights) { c.err = "stokes_build_weights has not run"; return STOKES_ERR_STATE; }
    if (c.ntiles_active == 0) { c.err = "no active unknowns"; return STOKES_ERR_STATE; }
    cudaError_t e = bench_cg_kernels(&c, precision, launches, ms_apply, ms_update);
    if (e != cudaSuccess) {
        c.err = std::string("kernel timing failed: ") + cudaGetErrorString(e);
        return STOKES_ERR_CUDA;
    }
    return STOKES_OK;
}

extern "C" int stokes_active_tiles(stokes_ctx h) { return h ? h->c.ntiles_active : -1; }

static thread_local std::string g_create_error;

static int64_t round_up(int64_t v, int64_t m) { return (v + m - 1) / m * m; }

#define API_CHECK_CUDA(ctx, call)                                                          \
    do {                                                                                   \
        cudaError_t e__ = (call);                                                          \
        if (e__ != cudaSuccess) {                                                          \
            (ctx)->c.err = std::string(#call " failed: ") + cudaGetErrorString(e__);       \
            return STOKES_ERR_CUDA;                                                        \
        }                                                                                  \
    } while (0)

static cudaError_t dalloc(Ctx& c, void** p, size_t bytes) {
    cudaError_t e = cudaMalloc(p, bytes);
    if (e == cudaSuccess) {
        c.allocs.push_back(*p);
        e = cudaMemset(*p, 0, bytes);
    }
    return e;
}

extern "C" {

void stokes_default_options(stokes_options* o) {
    if (!o) return;
    o->mode = STOKES_FP64;
    o->tol = 1e-8;
    o->max_iter = 200000;
    o->inner_tol = 1e-4;
    o->max_outer = 40;
    o->check_every = 64;
    o->precond = 0;
    o->use_graph = 1;
    o->wait_test = 0;
}

const char* stokes_last_error(stokes_ctx ctx) {
    if (!ctx) return g_create_error.c_str();
    return ctx->c.err.c_str();
}

stokes_status stokes_create(stokes_ctx* out, const stokes_grid* g, void* stream) {
    if (!out || !g) { g_create_error = "null argument"; return STOKES_ERR_ARG; }
    *out = nullptr;
    if (g->dim != 2 && g->dim != 3) { g_create_error = "dim must be 2 or 3"; return STOKES_ERR_ARG; }
    if (g->nx < 1 || g->ny < 1 || (g->dim == 3 && g->nz < 1)) { g_create_error = "grid sizes must be >= 1"; return STOKES_ERR_ARG; }
    if (!(g->h > 0) || !(g->dt > 0) || !std::isfinite(g->h) || !std::isfinite(g->dt)) {
        g_create_error = "h and dt must be positive and finite";
        return STOKES_ERR_ARG;
    }
    int64_t slots = (int64_t)(g->nx + 1) * (g->ny + 1) * (g->dim == 3 ? (g->nz + 1) : 1);
    if (slots > (int64_t)1 << 31) { g_create_error = "grid too large for 32-bit tile indices"; return STOKES_ERR_ARG; }
    stokes_ctx h = new (std::nothrow) stokes_ctx_s();
    if (!h) { g_create_error = "out of host memory"; return STOKES_ERR_ARG; }
    Ctx& c = h->c;
    c.g = *g;
    c.stream = (cudaStream_t)stream;
    cudaGetDevice(&c.device);
    if (!c.stream) {
        // the legacy default stream cannot be captured into a graph: use an
        // own blocking stream, which is ordered with the legacy stream
        if (cudaStreamCreate(&c.stream) != cudaSuccess) {
            g_create_error = "cudaStreamCreate failed";
            delete h;
            return STOKES_ERR_CUDA;
        }
        c.own_stream = true;
    }
    Layout& L = c.L;
    L.dim = g->dim; L.nx = g->nx; L.ny = g->ny; L.nz = g->dim == 3 ? g->nz : 0;
    L.P = (int)round_up(g->nx + 3, TX);
    if (g->dim == 2) {
        L.R = (int)round_up(g->ny + 3, 16);   // tile heights 4, 8 and 16 all divide R
        L.Q = 1;
        L.guard = round_up(L.P + 1, 32);
        L.ntx = L.P / TX; L.nty = L.R / TY2; L.ntz = 1;
    } else {
        L.R = (int)round_up(g->ny + 3, TY3);
        L.Q = (int)round_up(g->nz + 3, TZ3);
        L.guard = round_up((int64_t)L.P * L.R + L.P + 1, 32);
        L.ntx = L.P / TX; L.nty = L.R / TY3; L.ntz = L.Q / TZ3;
    }
    L.stride = round_up(2 * L.guard + (int64_t)L.P * L.R * L.Q, 64);
    c.nf = g->dim == 2 ? 3 : 6;
    c.nk = g->dim == 2 ? 4 : 7;
    c.nd = g->dim == 2 ? 2 : 3;
    c.nsite = g->dim == 2 ? 2 : 4;
    c.ncoef = g->dim == 2 ? 6 : 11;
    c.ntiles_all = L.ntx * L.nty * L.ntz;
    const int64_t S = L.stride;
    // one block for everything stokes_build_weights writes (zeroed per build)
    size_t wb = 0;
    auto add = [&](size_t bytes) { size_t o = wb; wb += round_up((int64_t)bytes, 256); return o; };
    size_t oWL = add(sizeof(double) * S * c.nk), oWF = add(sizeof(double) * S * c.nk);
    size_t oFF = add(S * c.nd), oEW = add(sizeof(double) * S * c.nd), oK = add(sizeof(double) * S * c.nd);
    size_t oRec = add(sizeof(double) * S * c.nd), oUbc = add(sizeof(double) * S * c.nd);
    size_t oAct = add(S * c.nsite);
    size_t oC64 = add(sizeof(double) * S * c.ncoef), oC32 = add(sizeof(float) * S * c.ncoef);
    size_t oC16 = add(sizeof(__nv_bfloat16) * S * c.ncoef);
    size_t oP16 = add(g->dim == 2 ? sizeof(uint32_t) * S * 3 : 4);
    size_t oQ16 = add(g->dim == 3 ? sizeof(uint2) * S * 2 : 8);
    size_t oM64 = add(sizeof(double) * S * c.nf), oM32 = add(sizeof(float) * S * c.nf);
    size_t oTF = add(c.ntiles_all);
    size_t oTF4 = add(g->dim == 2 ? (size_t)L.ntx * (L.R / 4) : 1);
    c.nunits_all = g->dim == 3 ? L.ntx * units_y(L.nty) * units_z(L.ntz, 1) : 0;
    size_t oUM = add(std::max(c.nunits_all, 1));
    c.weight_bytes = wb;
    cudaError_t e = dalloc(c, &c.weight_block, wb);
    char* base = (char*)c.weight_block;
    if (e == cudaSuccess) {
        DevArrays& A = c.A;
        for (int k = 0; k < c.nk; ++k) {
            A.WL[k] = (double*)(base + oWL) + k * S;
            A.WF[k] = (double*)(base + oWF) + k * S;
        }
        for (int d = 0; d < c.nd; ++d) {
            A.fflag[d] = (uint8_t*)(base + oFF) + d * S;
            A.effWF[d] = (double*)(base + oEW) + d * S;
            A.K64[d] = (double*)(base + oK) + d * S;
            A.rec[d] = (double*)(base + oRec) + d * S;
            A.ubc[d] = (double*)(base + oUbc) + d * S;
        }
        for (int s = 0; s < c.nsite; ++s) A.act[s] = (uint8_t*)(base + oAct) + s * S;
        A.coef64 = (double*)(base + oC64);
        A.coef32 = (float*)(base + oC32);
        A.coef16 = (__nv_bfloat16*)(base + oC16);
        A.pair16 = g->dim == 2 ? (uint32_t*)(base + oP16) : nullptr;
        A.quad16 = g->dim == 3 ? (uint2*)(base + oQ16) : nullptr;
        A.minv64 = (double*)(base + oM64);
        A.minv32 = (float*)(base + oM32);
        A.tile_flag = (uint8_t*)(base + oTF);
        A.tile_flag4 = (uint8_t*)(base + oTF4);
        A.unit_mask = (uint8_t*)(base + oUM);
    }
    const int64_t V = (int64_t)c.nf * S;
    if (e == cudaSuccess) e = dalloc(c, (void**)&c.tiles, sizeof(int) * c.ntiles_all);
    if (e == cudaSuccess) e = dalloc(c, (void**)&c.d_ntiles, sizeof(int));
    if (e == cudaSuccess) e = dalloc(c, (void**)&c.units, sizeof(int) * std::max(c.nunits_all, 1));
    if (e == cudaSuccess) e = dalloc(c, (void**)&c.d_nunits, sizeof(int));
    if (e == cudaSuccess) e = dalloc(c, (void**)&c.sc, 2 * sizeof(CgScalars));
    if (e == cudaSuccess) e = dalloc(c, (void**)&c.partial, sizeof(double) * 2 * (c.ntiles_all + 32));
    if (e == cudaSuccess) e = dalloc(c, (void**)&c.counter, sizeof(unsigned) * 4);
    if (e == cudaSuccess) e = cudaMallocHost((void**)&c.h_sc, 2 * sizeof(CgScalars));
    double** v64[] = {&c.w64.x, &c.w64.r, &c.w64.z, &c.w64.p[0], &c.w64.p[1], &c.w64.q, &c.b64, &c.x64, &c.y64};
    for (double** p : v64)
        if (e == cudaSuccess) e = dalloc(c, (void**)p, sizeof(double) * V);
    float** v32[] = {&c.w32.x, &c.w32.r, &c.w32.z, &c.w32.p[0], &c.w32.p[1], &c.w32.q};
    for (float** p : v32)
        if (e == cudaSuccess) e = dalloc(c, (void**)p, sizeof(float) * V);
    for (int i = 0; i < 4 && e == cudaSuccess; ++i) e = cudaEventCreate(&c.ev[i]);
    if (e == cudaSuccess && g->dim == 3) apply_set_attributes();
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) {
        g_create_error = std::string("device allocation failed: ") + cudaGetErrorString(e);
        stokes_destroy(h);
        return STOKES_ERR_CUDA;
    }
    *out = h;
    return STOKES_OK;
}

stokes_status stokes_destroy(stokes_ctx h) {
    if (!h) return STOKES_OK;
    Ctx& c = h->c;
    for (auto& ge : c.graph)
        if (ge) cudaGraphExecDestroy(ge);
    for (void* p : c.allocs) cudaFree(p);
    for (void* p : c.sw_allocs) cudaFree(p);
    delete c.sw;
    if (c.h_sc) cudaFreeHost(c.h_sc);
    for (auto& ev : c.ev)
        if (ev) cudaEventDestroy(ev);
    if (c.own_stream && c.stream) cudaStreamDestroy(c.stream);
    delete h;
    return STOKES_OK;
}

stokes_status stokes_vector_layout(stokes_ctx h, stokes_layout* out) {
    if (!h || !out) return STOKES_ERR_ARG;
    const Layout& L = h->c.L;
    out->nfields = h->c.nf;
    out->field_stride = L.stride;
    out->base = L.guard;
    out->pitch = L.P;
    out->rows = L.R;
    out->planes = L.Q;
    out->total = (int64_t)h->c.nf * L.stride;
    return STOKES_OK;
}

stokes_status stokes_set_min_face_liquid(stokes_ctx h, double eps) {
    if (!h) return STOKES_ERR_ARG;
    if (!(eps >= 0.0 && eps <= 1.0)) { h->c.err = "min_face_liquid must lie in [0, 1]"; return STOKES_ERR_ARG; }
    h->c.min_face_liquid = eps;
    return STOKES_OK;
}

stokes_status stokes_build_weights(stokes_ctx h, const double* phiL, const double* phiS, const double* const* rho,
                                   const double* const* mu, const double* const* ubc) {
    if (!h) return STOKES_ERR_ARG;
    Ctx& c = h->c;
    if (!phiL || !phiS || !rho || !mu || !ubc) { c.err = "null argument"; return STOKES_ERR_ARG; }
    for (int d = 0; d < c.nd; ++d)
        if (!rho[d] || !ubc[d]) { c.err = "null face array"; return STOKES_ERR_ARG; }
    for (int s = 0; s < c.nsite; ++s)
        if (!mu[s]) { c.err = "null viscosity array"; return STOKES_ERR_ARG; }
    for (auto& ge : c.graph)
        if (ge) { cudaGraphExecDestroy(ge); ge = nullptr; }
    c.sw_ready = false;
    c.learned.net = nullptr;
    cudaError_t e = launch_build_weights(&c, phiL, phiS, rho, mu, ubc);
    if (e != cudaSuccess) {
        c.err = std::string("weight build failed: ") + cudaGetErrorString(e);
        c.have_weights = false;
        return STOKES_ERR_CUDA;
    }
    c.have_weights = true;
    return STOKES_OK;
}

stokes_status stokes_apply(stokes_ctx h, const void* x, void* y, int precision) {
    if (!h) return STOKES_ERR_ARG;
    Ctx& c = h->c;
    if (!x || !y || x == y) { c.err = "x and y must be distinct non-null device vectors"; return STOKES_ERR_ARG; }
    if (!c.have_weights) { c.err = "stokes_build_weights has not run"; return STOKES_ERR_STATE; }
    ApplyArgs a{};
    cudaError_t e;
    API_CHECK_CUDA(h, cudaEventRecord(c.ev[0], c.stream));
    // every tile: inactive unknowns outside active tiles must also map x -> x
    if (precision == STOKES_FP64)
        e = launch_apply_mode<double, double>(c.L, nullptr, c.ntiles_all, c.coef<double>(), (const double*)x,
                                              (double*)y, MODE_PLAIN, a, c.stream);
    else if (precision == STOKES_FP32)
        e = launch_apply_mode<float, float>(c.L, nullptr, c.ntiles_all, c.coef<float>(), (const float*)x, (float*)y,
                                            MODE_PLAIN, a, c.stream);
    else if (precision == STOKES_BF16)
        e = launch_apply_mode<float, __nv_bfloat16>(c.L, nullptr, c.ntiles_all, c.coef<__nv_bfloat16>(),
                                                    (const float*)x, (float*)y, MODE_PLAIN, a, c.stream);
    else { c.err = "unknown precision"; return STOKES_ERR_ARG; }
    if (e != cudaSuccess) { c.err = std::string("apply failed: ") + cudaGetErrorString(e); return STOKES_ERR_CUDA; }
    API_CHECK_CUDA(h, cudaEventRecord(c.ev[1], c.stream));
    return STOKES_OK;
}

double stokes_last_apply_ms(stokes_ctx h) {
    if (!h) return -1.0;
    float ms = -1.f;
    if (cudaEventSynchronize(h->c.ev[1]) != cudaSuccess) return -1.0;
    if (cudaEventElapsedTime(&ms, h->c.ev[0], h->c.ev[1]) != cudaSuccess) return -1.0;
    return ms;
}

stokes_status stokes_rhs(stokes_ctx h, const double* const* u_star, double* b) {
    if (!h) return STOKES_ERR_ARG;
    Ctx& c = h->c;
    if (!u_star || !b) { c.err = "null argument"; return STOKES_ERR_ARG; }
    for (int d = 0; d < c.nd; ++d)
        if (!u_star[d]) { c.err = "null u_star component"; return STOKES_ERR_ARG; }
    if (!c.have_weights) { c.err = "stokes_build_weights has not run"; return STOKES_ERR_STATE; }
    API_CHECK_CUDA(h, launch_rhs(&c, u_star, b));
    return STOKES_OK;
}

stokes_status stokes_recover(stokes_ctx h, const double* const* u_star, const double* x, double* const* u_out) {
    if (!h) return STOKES_ERR_ARG;
    Ctx& c = h->c;
    if (!u_star || !x || !u_out) { c.err = "null argument"; return STOKES_ERR_ARG; }
    for (int d = 0; d < c.nd; ++d)
        if (!u_star[d] || !u_out[d]) { c.err = "null face component"; return STOKES_ERR_ARG; }
    if (!c.have_weights) { c.err = "stokes_build_weights has not run"; return STOKES_ERR_STATE; }
    API_CHECK_CUDA(h, launch_recover(&c, u_star, x, u_out));
    return STOKES_OK;
}

static stokes_status check_opts(Ctx& c, const stokes_options* o) {
    if (!o) { c.err = "null options"; return STOKES_ERR_ARG; }
    if (o->mode < 0 || o->mode > 2) { c.err = "bad mode"; return STOKES_ERR_ARG; }
    if (!(o->tol > 0) || o->max_iter < 1 || o->max_outer < 1 || !(o->inner_tol > 0)) {
        c.err = "bad tolerances or caps";
        return STOKES_ERR_ARG;
    }
    if (o->wait_test != 0 && o->wait_test != 1) { c.err = "wait_test must be 0 or 1"; return STOKES_ERR_ARG; }
    if (!c.have_weights) { c.err = "stokes_build_weights has not run"; return STOKES_ERR_STATE; }
    return STOKES_OK;
}

stokes_status stokes_solve_system(stokes_ctx h, const double* b, double* x, const stokes_options* o,
                                  stokes_stats* st) {
    if (!h) return STOKES_ERR_ARG;
    Ctx& c = h->c;
    if (!b || !x || b == x) { c.err = "b and x must be distinct non-null device vectors"; return STOKES_ERR_ARG; }
    stokes_status s = check_opts(c, o);
    if (s != STOKES_OK) return s;
    API_CHECK_CUDA(h, cudaEventRecord(c.ev[0], c.stream));
    s = solve_system(&c, b, x, o, st);
    cudaEventRecord(c.ev[1], c.stream);
    if (st) {
        float ms = 0.f;
        cudaEventSynchronize(c.ev[1]);
        cudaEventElapsedTime(&ms, c.ev[0], c.ev[1]);
        st->ms_solve = ms;
        st->ms_rhs = st->ms_recover = 0.0;
    }
    return s;
}

stokes_status stokes_traction_u_star(stokes_ctx h, const double* const* tau_bc, const double* p_bc,
                                     const double* const* u_star, double* const* u_star_out) {
    if (!h) return STOKES_ERR_ARG;
    Ctx& c = h->c;
    if (!tau_bc || !p_bc || !u_star || !u_star_out) { c.err = "null argument"; return STOKES_ERR_ARG; }
    for (int d = 0; d < c.nd; ++d)
        if (!u_star[d] || !u_star_out[d]) { c.err = "null face component"; return STOKES_ERR_ARG; }
    const double* fields[6];
    for (int f = 0; f < c.nf - 1; ++f) {
        if (!tau_bc[f]) { c.err = "null stress component"; return STOKES_ERR_ARG; }
        fields[f] = tau_bc[f];
    }
    fields[c.nf - 1] = p_bc;
    if (!c.have_weights) { c.err = "stokes_build_weights has not run"; return STOKES_ERR_STATE; }
    API_CHECK_CUDA(h, launch_traction(&c, fields, u_star, u_star_out));
    return STOKES_OK;
}

stokes_status stokes_advect(stokes_ctx h, const double* const* u_in, const double* phi_in, const double* gravity,
                            int ext_passes, const uint8_t* valid, const double* phi_union, double* const* u_out,
                            double* phi_out) {
    if (!h) return STOKES_ERR_ARG;
    Ctx& c = h->c;
    if (c.L.dim != 2) { c.err = "stokes_advect is 2D only"; return STOKES_ERR_ARG; }
    if (c.L.nx < 2 || c.L.ny < 2) { c.err = "stokes_advect needs nx, ny >= 2"; return STOKES_ERR_ARG; }
    if (!u_in || !u_out || !gravity || ext_passes < 0) { c.err = "null argument or negative pass count"; return STOKES_ERR_ARG; }
    for (int d = 0; d < 2; ++d)
        if (!u_in[d] || !u_out[d]) { c.err = "null face component"; return STOKES_ERR_ARG; }
    if (phi_in && (!phi_out || phi_out == phi_in)) {
        c.err = "phi_out must be a device array distinct from phi_in";
        return STOKES_ERR_ARG;
    }
    if (!valid && !c.have_weights) { c.err = "no validity mask and stokes_build_weights has not run"; return STOKES_ERR_STATE; }
    if (!c.adv_scratch) API_CHECK_CUDA(h, dalloc(c, &c.adv_scratch, advect_scratch_bytes(c.L)));
    API_CHECK_CUDA(h, launch_advect2d(&c, c.adv_scratch, u_in, phi_in, gravity, ext_passes, valid, phi_union, u_out,
                                      phi_out));
    return STOKES_OK;
}

stokes_status stokes_solve_step(stokes_ctx h, const double* const* u_star, double* const* u_out,
                                double* const* tau_out, double* p_out, const stokes_options* o, stokes_stats* st) {
    if (!h) return STOKES_ERR_ARG;
    Ctx& c = h->c;
    if (!u_star || !u_out || !tau_out || !p_out) { c.err = "null argument"; return STOKES_ERR_ARG; }
    for (int d = 0; d < c.nd; ++d)
        if (!u_star[d] || !u_out[d]) { c.err = "null face component"; return STOKES_ERR_ARG; }
    for (int f = 0; f < c.nf - 1; ++f)
        if (!tau_out[f]) { c.err = "null stress component"; return STOKES_ERR_ARG; }
    stokes_status s = check_opts(c, o);
    if (s != STOKES_OK) return s;
    API_CHECK_CUDA(h, cudaEventRecord(c.ev[0], c.stream));
    API_CHECK_CUDA(h, launch_rhs(&c, u_star, c.b64));
    API_CHECK_CUDA(h, cudaEventRecord(c.ev[1], c.stream));
    stokes_stats local{};
    s = solve_system(&c, c.b64, c.x64, o, &local);
    if (s == STOKES_ERR_CUDA || s == STOKES_ERR_ARG) return s;
    API_CHECK_CUDA(h, cudaEventRecord(c.ev[2], c.stream));
    API_CHECK_CUDA(h, launch_recover(&c, u_star, c.x64, u_out));
    double* outs[6];
    for (int f = 0; f < c.nf - 1; ++f) outs[f] = tau_out[f];
    outs[c.nf - 1] = p_out;
    API_CHECK_CUDA(h, launch_unpack(&c, c.x64, outs, 1));
    API_CHECK_CUDA(h, cudaEventRecord(c.ev[3], c.stream));
    API_CHECK_CUDA(h, cudaEventSynchronize(c.ev[3]));
    if (st) {
        *st = local;
        float a = 0, b = 0, d = 0;
        cudaEventElapsedTime(&a, c.ev[0], c.ev[1]);
        cudaEventElapsedTime(&b, c.ev[1], c.ev[2]);
        cudaEventElapsedTime(&d, c.ev[2], c.ev[3]);
        st->ms_rhs = a; st->ms_solve = b; st->ms_recover = d;
    }
    return s;
}

int64_t stokes_export_size(stokes_ctx h, int what) {
    if (!h) return -1;
    Ctx& c = h->c;
    const Layout& L = c.L;
    int nx = L.nx, ny = L.ny, nz = L.nz;
    auto kind_count = [&](int kind) -> int64_t {
        if (L.dim == 2) {
            int wx = (kind == 1 || kind == 2) ? nx + 1 : nx, wy = (kind == 1 || kind == 3) ? ny + 1 : ny;
            return (int64_t)wx * wy;
        }
        int wx = (kind == 1 || kind == 4 || kind == 5) ? nx + 1 : nx;
        int wy = (kind == 2 || kind == 4 || kind == 6) ? ny + 1 : ny;
        int wz = (kind == 3 || kind == 5 || kind == 6) ? nz + 1 : nz;
        return (int64_t)wx * wy * wz;
    };
    int64_t n = 0;
    switch (what) {
        case 0:
        case 1:
            for (int k = 0; k < c.nk; ++k) n += kind_count(k);
            return n * (int64_t)sizeof(double);
        case 2:
            for (int d = 0; d < c.nd; ++d) n += kind_count(L.dim == 2 ? 2 + d : 1 + d);
            return n;
        case 3:
            if (L.dim == 2) return kind_count(0) * 2 + kind_count(1);
            return kind_count(0) * 3 + kind_count(4) + kind_count(5) + kind_count(6);
        default:
            return -1;
    }
}

}  // extern "C"

namespace stk {
// per-kind slot array -> field layout (double or byte)
template <class T>
__global__ void k_export(Layout L, int kind, const T* src, T* dst) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    int j = blockIdx.y * blockDim.y + threadIdx.y;
    int k = blockIdx.z;
    if (L.dim == 2) {
        int wx = (kind == 1 || kind == 2) ? L.nx + 1 : L.nx, wy = (kind == 1 || kind == 3) ? L.ny + 1 : L.ny;
        if (i >= wx || j >= wy) return;
        dst[fidx2(kind, i, j, L.nx, L.ny)] = src[L.off(i + 1, j + 1, 0)];
    } else {
        int wx = (kind == 1 || kind == 4 || kind == 5) ? L.nx + 1 : L.nx;
        int wy = (kind == 2 || kind == 4 || kind == 6) ? L.ny + 1 : L.ny;
        int wz = (kind == 3 || kind == 5 || kind == 6) ? L.nz + 1 : L.nz;
        if (i >= wx || j >= wy || k >= wz) return;
        dst[fidx3(kind, i, j, k, L.nx, L.ny, L.nz)] = src[L.off(i + 1, j + 1, k + 1)];
    }
}
}  // namespace stk

extern "C" stokes_status stokes_export(stokes_ctx h, int what, void* out) {
    if (!h || !out) return STOKES_ERR_ARG;
    Ctx& c = h->c;
    if (!c.have_weights) { c.err = "stokes_build_weights has not run"; return STOKES_ERR_STATE; }
    const Layout& L = c.L;
    dim3 blk(32, 8), grd((L.nx + 2 + 31) / 32, (L.ny + 2 + 7) / 8, L.dim == 2 ? 1 : L.nz + 1);
    char* o = (char*)out;
    auto count = [&](int kind) -> int64_t {
        int nx = L.nx, ny = L.ny, nz = L.nz;
        if (L.dim == 2) {
            int wx = (kind == 1 || kind == 2) ? nx + 1 : nx, wy = (kind == 1 || kind == 3) ? ny + 1 : ny;
            return (int64_t)wx * wy;
        }
        int wx = (kind == 1 || kind == 4 || kind == 5) ? nx + 1 : nx;
        int wy = (kind == 2 || kind == 4 || kind == 6) ? ny + 1 : ny;
        int wz = (kind == 3 || kind == 5 || kind == 6) ? nz + 1 : nz;
        return (int64_t)wx * wy * wz;
    };
    if (what == 0 || what == 1) {
        for (int k = 0; k < c.nk; ++k) {
            k_export<double><<<grd, blk, 0, c.stream>>>(L, k, what == 0 ? c.A.WL[k] : c.A.WF[k], (double*)o);
            o += count(k) * sizeof(double);
        }
    } else if (what == 2) {
        for (int d = 0; d < c.nd; ++d) {
            int kind = L.dim == 2 ? 2 + d : 1 + d;
            k_export<uint8_t><<<grd, blk, 0, c.stream>>>(L, kind, c.A.fflag[d], (uint8_t*)o);
            o += count(kind);
        }
    } else if (what == 3) {
        // unknown order: 2D tau_xx(cell) tau_xy(node) p(cell); 3D txx tyy (cell) exy exz eyz, p(cell)
        if (L.dim == 2) {
            int site[3] = {0, 1, 0}, kind[3] = {0, 1, 0};
            for (int u = 0; u < 3; ++u) {
                k_export<uint8_t><<<grd, blk, 0, c.stream>>>(L, kind[u], c.A.act[site[u]], (uint8_t*)o);
                o += count(kind[u]);
            }
        } else {
            int site[6] = {0, 0, 1, 2, 3, 0}, kind[6] = {0, 0, 4, 5, 6, 0};
            for (int u = 0; u < 6; ++u) {
                k_export<uint8_t><<<grd, blk, 0, c.stream>>>(L, kind[u], c.A.act[site[u]], (uint8_t*)o);
                o += count(kind[u]);
            }
        }
    } else {
        c.err = "unknown export selector";
        return STOKES_ERR_ARG;
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) { c.err = std::string("export failed: ") + cudaGetErrorString(e); return STOKES_ERR_CUDA; }
    return STOKES_OK;
}

extern "C" stokes_status stokes_slots_to_fields(stokes_ctx h, const double* slots, double* fields) {
    if (!h || !slots || !fields) return STOKES_ERR_ARG;
    Ctx& c = h->c;
    double* outs[6];
    // fields are concatenated in unknown order
    int64_t off = 0;
    const Layout& L = c.L;
    for (int f = 0; f < c.nf; ++f) {
        outs[f] = fields + off;
        int kind;
        if (L.dim == 2) kind = f == 1 ? 1 : 0;
        else kind = (f <= 1 || f == 5) ? 0 : (f == 2 ? 4 : f == 3 ? 5 : 6);
        int64_t n;
        if (L.dim == 2) n = kind == 0 ? (int64_t)L.nx * L.ny : (int64_t)(L.nx + 1) * (L.ny + 1);
        else {
            int wx = (kind == 4 || kind == 5) ? L.nx + 1 : L.nx;
            int wy = (kind == 4 || kind == 6) ? L.ny + 1 : L.ny;
            int wz = (kind == 5 || kind == 6) ? L.nz + 1 : L.nz;
            n = (int64_t)wx * wy * wz;
        }
        off += n;
    }
    API_CHECK_CUDA(h, launch_unpack(&c, slots, outs, 1));
    return STOKES_OK;
}

extern "C" stokes_status stokes_fields_to_slots(stokes_ctx h, const double* fields, double* slots) {
    if (!h || !slots || !fields) return STOKES_ERR_ARG;
    Ctx& c = h->c;
    double* ins[6];
    int64_t off = 0;
    const Layout& L = c.L;
    for (int f = 0; f < c.nf; ++f) {
        ins[f] = (double*)fields + off;
        int kind;
        if (L.dim == 2) kind = f == 1 ? 1 : 0;
        else kind = (f <= 1 || f == 5) ? 0 : (f == 2 ? 4 : f == 3 ? 5 : 6);
        int64_t n;
        if (L.dim == 2) n = kind == 0 ? (int64_t)L.nx * L.ny : (int64_t)(L.nx + 1) * (L.ny + 1);
        else {
            int wx = (kind == 4 || kind == 5) ? L.nx + 1 : L.nx;
            int wy = (kind == 4 || kind == 6) ? L.ny + 1 : L.ny;
            int wz = (kind == 5 || kind == 6) ? L.nz + 1 : L.nz;
            n = (int64_t)wx * wy * wz;
        }
        off += n;
    }
    API_CHECK_CUDA(h, launch_unpack(&c, slots, ins, 0));
    return STOKES_OK;
}
