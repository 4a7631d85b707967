// Transport around the Stokes step (Section "Application to Viscous Jet
// Buckling", 2D): extension of the velocity into fluid faces that carry no
// liquid, first-order semi-Lagrangian advection of the MAC velocity with
// bilinear interpolation plus the body force, and semi-Lagrangian advection
// of the liquid level set on the half lattice.
//
// Positions are in grid units X = (x - origin) / h: u face (i, j) at
// (i, j + 1/2), v face (i, j) at (i + 1/2, j), lattice point (a, b) at
// ((a - 1)/2, (b - 1)/2).  A field is interpolated bilinearly between its
// samples and clamped onto their box outside it.  Every product and sum is an
// explicitly rounded FP64 operation in a fixed order, so the departure cells
// (a floor of an FP64 coordinate) and the interpolated values do not depend
// on contraction into fused multiply-adds.
#include "ctx.cuh"

namespace stk {

namespace {

__device__ __forceinline__ double lerp_rn(double a, double b, double t) {
    return __dadd_rn(__dmul_rn(a, __dsub_rn(1.0, t)), __dmul_rn(b, t));
}

// Bilinear interpolation of a row-major (ny_s, nx_s) array at sample
// coordinates (fx, fy); nx_s, ny_s >= 2.
__device__ double bilerp(const double* __restrict__ f, int nx_s, int ny_s, double fx, double fy) {
    fx = fmin(fmax(fx, 0.0), (double)(nx_s - 1));
    fy = fmin(fmax(fy, 0.0), (double)(ny_s - 1));
    int i0 = min((int)floor(fx), nx_s - 2);
    int j0 = min((int)floor(fy), ny_s - 2);
    double tx = __dsub_rn(fx, (double)i0), ty = __dsub_rn(fy, (double)j0);
    const double* r0 = f + (int64_t)j0 * nx_s + i0;
    const double* r1 = r0 + nx_s;
    return lerp_rn(lerp_rn(r0[0], r0[1], tx), lerp_rn(r1[0], r1[1], tx), ty);
}

struct Vel2 {
    const double* u;   // (ny, nx+1)
    const double* v;   // (ny+1, nx)
    int nx, ny;
    __device__ double at_u(double X, double Y) const { return bilerp(u, nx + 1, ny, X, __dsub_rn(Y, 0.5)); }
    __device__ double at_v(double X, double Y) const { return bilerp(v, nx, ny + 1, __dsub_rn(X, 0.5), Y); }
};

// Stage u_in into buffer 0 and mark the faces whose value is kept: those the
// caller flags valid, else those that are not fluid-without-liquid ("bad")
// in the context's weights.
__global__ void k_ext_init(Layout L, const double* __restrict__ u_in, const double* __restrict__ v_in,
                           const uint8_t* __restrict__ valid, const uint8_t* __restrict__ flag_u,
                           const uint8_t* __restrict__ flag_v, double* __restrict__ f, uint8_t* __restrict__ ok) {
    const int nu = (L.nx + 1) * L.ny, nv = L.nx * (L.ny + 1);
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < nu + nv; t += gridDim.x * blockDim.x) {
        bool keep;
        if (valid) {
            keep = valid[t] != 0;
        } else if (t < nu) {
            int i = t % (L.nx + 1), j = t / (L.nx + 1);
            keep = (flag_u[L.off(i + 1, j + 1, 0)] & F_BAD) == 0;
        } else {
            int s = t - nu, i = s % L.nx, j = s / L.nx;
            keep = (flag_v[L.off(i + 1, j + 1, 0)] & F_BAD) == 0;
        }
        f[t] = t < nu ? u_in[t] : v_in[t - nu];
        ok[t] = keep;
    }
}

// One Jacobi sweep: a face not yet valid with valid 4-neighbours of its own
// component takes their mean (left, right, below, above summed in that order).
__global__ void k_ext_pass(int nx, int ny, const double* __restrict__ f, const uint8_t* __restrict__ ok,
                           double* __restrict__ g, uint8_t* __restrict__ ok_out) {
    const int nu = (nx + 1) * ny, nv = nx * (ny + 1);
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < nu + nv; t += gridDim.x * blockDim.x) {
        if (ok[t]) {
            g[t] = f[t];
            ok_out[t] = 1;
            continue;
        }
        int W, H, base, s;
        if (t < nu) { W = nx + 1; H = ny; base = 0; s = t; }
        else        { W = nx; H = ny + 1; base = nu; s = t - nu; }
        int i = s % W, j = s / W;
        double sum = 0.0;
        int c = 0;
        const int nb[4][2] = {{-1, 0}, {1, 0}, {0, -1}, {0, 1}};
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            int ii = i + nb[q][0], jj = j + nb[q][1];
            if (ii < 0 || ii >= W || jj < 0 || jj >= H) continue;
            int64_t o = base + (int64_t)jj * W + ii;
            if (ok[o]) { sum = __dadd_rn(sum, f[o]); ++c; }
        }
        g[t] = c > 0 ? __ddiv_rn(sum, (double)c) : f[t];
        ok_out[t] = c > 0;
    }
}

// u* = (advected u) + dt g on every u and v face.
__global__ void k_adv_velocity(Vel2 V, double c, double dtg_x, double dtg_y, double* __restrict__ u_out,
                               double* __restrict__ v_out) {
    const int nx = V.nx, ny = V.ny;
    const int nu = (nx + 1) * ny, nv = nx * (ny + 1);
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < nu + nv; t += gridDim.x * blockDim.x) {
        if (t < nu) {
            int i = t % (nx + 1), j = t / (nx + 1);
            double X = (double)i, Y = (double)j + 0.5;
            double vy = V.at_v(X, Y);
            double Xd = __dsub_rn(X, __dmul_rn(c, V.u[t])), Yd = __dsub_rn(Y, __dmul_rn(c, vy));
            u_out[t] = __dadd_rn(V.at_u(Xd, Yd), dtg_x);
        } else {
            int s = t - nu, i = s % nx, j = s / nx;
            double X = (double)i + 0.5, Y = (double)j;
            double ux = V.at_u(X, Y);
            double Xd = __dsub_rn(X, __dmul_rn(c, ux)), Yd = __dsub_rn(Y, __dmul_rn(c, V.v[s]));
            v_out[s] = __dadd_rn(V.at_v(Xd, Yd), dtg_y);
        }
    }
}

// phi^{n+1} at every half-lattice point; optionally the union with a source
// region (phi_out = min(phi_out, phi_union)).
__global__ void k_adv_levelset(Vel2 V, double c, const double* __restrict__ phi, const double* __restrict__ phi_union,
                               double* __restrict__ phi_out) {
    const int La = 2 * V.nx + 3, Lb = 2 * V.ny + 3;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < La * Lb; t += gridDim.x * blockDim.x) {
        int a = t % La, b = t / La;
        double X = (double)(a - 1) * 0.5, Y = (double)(b - 1) * 0.5;
        double Xd = __dsub_rn(X, __dmul_rn(c, V.at_u(X, Y)));
        double Yd = __dsub_rn(Y, __dmul_rn(c, V.at_v(X, Y)));
        double r = bilerp(phi, La, Lb, __dadd_rn(__dmul_rn(2.0, Xd), 1.0), __dadd_rn(__dmul_rn(2.0, Yd), 1.0));
        if (phi_union) r = fmin(r, phi_union[t]);
        phi_out[t] = r;
    }
}

int grid_for(int64_t n, int block) {
    int64_t b = (n + block - 1) / block;
    return (int)(b < 1 ? 1 : (b > 152 * 16 ? 152 * 16 : b));
}

}  // namespace

// scratch: 2 (nu + nv) doubles then 2 (nu + nv) bytes
size_t advect_scratch_bytes(const Layout& L) {
    size_t nf = (size_t)(L.nx + 1) * L.ny + (size_t)L.nx * (L.ny + 1);
    return nf * (2 * sizeof(double) + 2);
}

cudaError_t launch_advect2d(Ctx* c, void* scratch, const double* const* u_in, const double* phi_in, const double* g,
                            int passes, const uint8_t* valid, const double* phi_union, double* const* u_out,
                            double* phi_out) {
    const Layout& L = c->L;
    const int nu = (L.nx + 1) * L.ny, nv = L.nx * (L.ny + 1), nf = nu + nv;
    double* f[2] = {(double*)scratch, (double*)scratch + nf};
    uint8_t* ok[2] = {(uint8_t*)(f[1] + nf), (uint8_t*)(f[1] + nf) + nf};
    const int B = 256;
    k_ext_init<<<grid_for(nf, B), B, 0, c->stream>>>(L, u_in[0], u_in[1], valid, c->A.fflag[0], c->A.fflag[1], f[0],
                                                     ok[0]);
    int cur = 0;
    for (int p = 0; p < passes; ++p) {
        k_ext_pass<<<grid_for(nf, B), B, 0, c->stream>>>(L.nx, L.ny, f[cur], ok[cur], f[1 - cur], ok[1 - cur]);
        cur = 1 - cur;
    }
    const double cfl = c->g.dt / c->g.h;
    Vel2 V{f[cur], f[cur] + nu, L.nx, L.ny};
    if (phi_in) {
        int64_t nl = (int64_t)(2 * L.nx + 3) * (2 * L.ny + 3);
        k_adv_levelset<<<grid_for(nl, B), B, 0, c->stream>>>(V, cfl, phi_in, phi_union, phi_out);
    }
    k_adv_velocity<<<grid_for(nf, B), B, 0, c->stream>>>(V, cfl, c->g.dt * g[0], c->g.dt * g[1], u_out[0], u_out[1]);
    return cudaGetLastError();
}

}  // namespace stk
