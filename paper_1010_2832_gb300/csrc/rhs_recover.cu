// Right-hand side (eq. stokesmixedsystemspd with the prescribed-velocity terms
// of Section 6.2), velocity recovery (first block row of eq.
// stokesmixedsystem) and conversions between slot and field layouts.
//
// Right-hand side of an unknown s with row operator R (a row of D or G^T):
//   b_s = a_s [ sum_f R_sf v_f - W_S^s sum_f R_sf u_BC,f ],
//   v_f = W_F,f u*_f + (1 - W_F,f) u_BC,f   (effective face fluid weight),
// with a_s = W_L^s / h on active unknowns and R_sf = +-1.  Faces outside the
// grid carry v = u_BC = 0.
#include "internal.cuh"
#include "ctx.cuh"

namespace stk {

struct FacePtrs { const double* p[3]; };
struct FaceOut { double* p[3]; };

// v_f and u_BC,f of face kind d at padded position (c, r, q); zero outside.
__device__ __forceinline__ void face_vals(const Layout& L, const DevArrays& D, const FacePtrs& us, int d, int c,
                                          int r, int q, double& v, double& ub) {
    int i = c - 1, j = r - 1, k = q - 1;
    bool ex;
    if (L.dim == 2) {
        ex = i >= 0 && j >= 0 && i <= L.nx && j <= L.ny && (d == 0 ? j < L.ny : i < L.nx);
    } else {
        ex = i >= 0 && j >= 0 && k >= 0 && i <= L.nx && j <= L.ny && k <= L.nz &&
             (d == 0 ? (j < L.ny && k < L.nz) : d == 1 ? (i < L.nx && k < L.nz) : (i < L.nx && j < L.ny));
    }
    if (!ex) { v = 0.0; ub = 0.0; return; }
    int64_t o = L.off(c, r, L.dim == 2 ? 0 : q);
    double wf = D.effWF[d][o];
    ub = D.ubc[d][o];
    int64_t fi = L.dim == 2 ? fidx2(2 + d, i, j, L.nx, L.ny) : fidx3(1 + d, i, j, k, L.nx, L.ny, L.nz);
    v = wf * us.p[d][fi] + (1.0 - wf) * ub;
}

__global__ void k_rhs2d(Layout L, DevArrays D, FacePtrs us, double* b) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    int j = blockIdx.y * blockDim.y + threadIdx.y;
    if (i > L.nx || j > L.ny) return;
    int c = i + 1, r = j + 1;
    int64_t o = L.off(c, r, 0);
    const int64_t S = L.stride;
    const double* a_c = D.coef64;
    const double* a_n = D.coef64 + S;
    if (i < L.nx && j < L.ny) {
        double vl, ul, vr, ur, vb, ubb, vt, ut;
        face_vals(L, D, us, 0, c, r, 0, vl, ul);
        face_vals(L, D, us, 0, c + 1, r, 0, vr, ur);
        face_vals(L, D, us, 1, c, r, 0, vb, ubb);
        face_vals(L, D, us, 1, c, r + 1, 0, vt, ut);
        double ws = 1.0 - D.WF[0][o];
        double a = a_c[o];
        // p: G^T = (u_l - u_r) + (v_b - v_t);  tau_xx: (u_r - u_l) - (v_t - v_b)
        double gp = (vl - vr) + (vb - vt), gpb = (ul - ur) + (ubb - ut);
        double dx = (vr - vl) - (vt - vb), dxb = (ur - ul) - (ut - ubb);
        b[2 * S + o] = a * (gp - ws * gpb);
        b[o] = a * (dx - ws * dxb);
    }
    {
        // tau_xy at node: (u(i,j) - u(i,j-1)) + (v(i,j) - v(i-1,j))
        double vu, uu, vd, ud, vr, ur, vl, ul;
        face_vals(L, D, us, 0, c, r, 0, vu, uu);
        face_vals(L, D, us, 0, c, r - 1, 0, vd, ud);
        face_vals(L, D, us, 1, c, r, 0, vr, ur);
        face_vals(L, D, us, 1, c - 1, r, 0, vl, ul);
        double ws = 1.0 - D.WF[1][o];
        double dxy = (vu - vd) + (vr - vl), dxyb = (uu - ud) + (ur - ul);
        b[S + o] = a_n[o] * (dxy - ws * dxyb);
    }
}

__global__ void k_rhs3d(Layout L, DevArrays D, FacePtrs us, double* b) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    int j = blockIdx.y * blockDim.y + threadIdx.y;
    int k = blockIdx.z;
    if (i > L.nx || j > L.ny || k > L.nz) return;
    int c = i + 1, r = j + 1, q = k + 1;
    int64_t o = L.off(c, r, q);
    const int64_t S = L.stride;
    auto A = [&](int f) { return D.coef64[(int64_t)f * S + o]; };
    // fields: 0 txx, 1 tyy, 2 txy, 3 txz, 4 tyz, 5 p
    if (i < L.nx && j < L.ny && k < L.nz) {
        double v0, u0, v1, u1, w0, wb0, v2, u2, v3, u3, w1, wb1;
        double ul_, ur_, vb_, vt_, wd_, wu_;
        face_vals(L, D, us, 0, c, r, q, v0, ul_);
        face_vals(L, D, us, 0, c + 1, r, q, v1, ur_);
        face_vals(L, D, us, 1, c, r, q, v2, vb_);
        face_vals(L, D, us, 1, c, r + 1, q, v3, vt_);
        face_vals(L, D, us, 2, c, r, q, w0, wd_);
        face_vals(L, D, us, 2, c, r, q + 1, w1, wu_);
        (void)u0; (void)u1; (void)wb0; (void)u2; (void)u3; (void)wb1;
        double ws = 1.0 - D.WF[0][o];
        double a = A(0);
        double dux = v1 - v0, dvy = v3 - v2, dwz = w1 - w0;
        double bux = ur_ - ul_, bvy = vt_ - vb_, bwz = wu_ - wd_;
        b[5 * S + o] = a * (-(dux + dvy + dwz) - ws * (-(bux + bvy + bwz)));
        b[0 * S + o] = a * ((dux - dwz) - ws * (bux - bwz));
        b[1 * S + o] = a * ((dvy - dwz) - ws * (bvy - bwz));
    }
    if (k < L.nz) {  // txy on z-edge: (u(j) - u(j-1)) + (v(i) - v(i-1))
        double a1, b1, a2, b2, a3, b3, a4, b4;
        face_vals(L, D, us, 0, c, r, q, a1, b1);
        face_vals(L, D, us, 0, c, r - 1, q, a2, b2);
        face_vals(L, D, us, 1, c, r, q, a3, b3);
        face_vals(L, D, us, 1, c - 1, r, q, a4, b4);
        double ws = 1.0 - D.WF[4][o];
        b[2 * S + o] = A(1) * (((a1 - a2) + (a3 - a4)) - ws * ((b1 - b2) + (b3 - b4)));
    }
    if (j < L.ny) {  // txz on y-edge: (u(k) - u(k-1)) + (w(i) - w(i-1))
        double a1, b1, a2, b2, a3, b3, a4, b4;
        face_vals(L, D, us, 0, c, r, q, a1, b1);
        face_vals(L, D, us, 0, c, r, q - 1, a2, b2);
        face_vals(L, D, us, 2, c, r, q, a3, b3);
        face_vals(L, D, us, 2, c - 1, r, q, a4, b4);
        double ws = 1.0 - D.WF[5][o];
        b[3 * S + o] = A(2) * (((a1 - a2) + (a3 - a4)) - ws * ((b1 - b2) + (b3 - b4)));
    }
    if (i < L.nx) {  // tyz on x-edge: (v(k) - v(k-1)) + (w(j) - w(j-1))
        double a1, b1, a2, b2, a3, b3, a4, b4;
        face_vals(L, D, us, 1, c, r, q, a1, b1);
        face_vals(L, D, us, 1, c, r, q - 1, a2, b2);
        face_vals(L, D, us, 2, c, r, q, a3, b3);
        face_vals(L, D, us, 2, c, r - 1, q, a4, b4);
        double ws = 1.0 - D.WF[6][o];
        b[4 * S + o] = A(3) * (((a1 - a2) + (a3 - a4)) - ws * ((b1 - b2) + (b3 - b4)));
    }
}

// (B^T x)_f at one face: the same bracket as the apply's face value.
__global__ void k_recover2d(Layout L, DevArrays D, FacePtrs us, const double* x, FaceOut out) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    int j = blockIdx.y * blockDim.y + threadIdx.y;
    if (i > L.nx || j > L.ny) return;
    const int64_t S = L.stride;
    const double* a_c = D.coef64;
    const double* a_n = D.coef64 + S;
    int c = i + 1, r = j + 1;
    int64_t o = L.off(c, r, 0);
    auto U = [&](int64_t oo) { return a_c[oo] * (x[2 * S + oo] - x[oo]); };
    auto V = [&](int64_t oo) { return a_c[oo] * (x[2 * S + oo] + x[oo]); };
    auto N = [&](int64_t oo) { return a_n[oo] * x[S + oo]; };
    for (int d = 0; d < 2; ++d) {
        if (d == 0 && j >= L.ny) continue;
        if (d == 1 && i >= L.nx) continue;
        uint8_t fl = D.fflag[d][o];
        int64_t fi = fidx2(2 + d, i, j, L.nx, L.ny);
        double us_ = us.p[d][fi];
        double u;
        if (fl & F_LIVE) {
            double btx = d == 0 ? (U(o) - U(L.off(c - 1, r, 0))) + (N(o) - N(L.off(c, r + 1, 0)))
                                : (V(o) - V(L.off(c, r - 1, 0))) + (N(o) - N(L.off(c + 1, r, 0)));
            u = us_ - D.rec[d][o] * btx;
        } else if (D.effWF[d][o] == 0.0) {
            u = D.ubc[d][o];
        } else {
            u = us_;
        }
        out.p[d][fi] = u;
    }
}

__global__ void k_recover3d(Layout L, DevArrays D, FacePtrs us, const double* x, FaceOut out) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    int j = blockIdx.y * blockDim.y + threadIdx.y;
    int k = blockIdx.z;
    if (i > L.nx || j > L.ny || k > L.nz) return;
    const int64_t S = L.stride;
    int c = i + 1, r = j + 1, q = k + 1;
    int64_t o = L.off(c, r, q);
    const double* cf = D.coef64;
    auto Uc = [&](int64_t oo) { return cf[oo] * (x[5 * S + oo] - x[oo]); };
    auto Vc = [&](int64_t oo) { return cf[oo] * (x[5 * S + oo] - x[S + oo]); };
    auto Wc = [&](int64_t oo) { return cf[oo] * (x[5 * S + oo] + x[oo] + x[S + oo]); };
    auto Nxy = [&](int64_t oo) { return cf[S + oo] * x[2 * S + oo]; };
    auto Nxz = [&](int64_t oo) { return cf[2 * S + oo] * x[3 * S + oo]; };
    auto Nyz = [&](int64_t oo) { return cf[3 * S + oo] * x[4 * S + oo]; };
    for (int d = 0; d < 3; ++d) {
        bool ex = d == 0 ? (j < L.ny && k < L.nz) : d == 1 ? (i < L.nx && k < L.nz) : (i < L.nx && j < L.ny);
        if (!ex) continue;
        uint8_t fl = D.fflag[d][o];
        int64_t fi = fidx3(1 + d, i, j, k, L.nx, L.ny, L.nz);
        double us_ = us.p[d][fi];
        double u;
        if (fl & F_LIVE) {
            double btx;
            if (d == 0)
                btx = (Uc(o) - Uc(L.off(c - 1, r, q))) + (Nxy(o) - Nxy(L.off(c, r + 1, q))) +
                      (Nxz(o) - Nxz(L.off(c, r, q + 1)));
            else if (d == 1)
                btx = (Vc(o) - Vc(L.off(c, r - 1, q))) + (Nxy(o) - Nxy(L.off(c + 1, r, q))) +
                      (Nyz(o) - Nyz(L.off(c, r, q + 1)));
            else
                btx = (Wc(o) - Wc(L.off(c, r, q - 1))) + (Nxz(o) - Nxz(L.off(c + 1, r, q))) +
                      (Nyz(o) - Nyz(L.off(c, r + 1, q)));
            u = us_ - D.rec[d][o] * btx;
        } else if (D.effWF[d][o] == 0.0) {
            u = D.ubc[d][o];
        } else {
            u = us_;
        }
        out.p[d][fi] = u;
    }
}

// slot field f <-> field-layout array of its site kind
struct FieldMap { double* p[6]; };
__global__ void k_slots_fields(Layout L, const double* src, double* dst, int to_fields, int nf, int64_t f_off0,
                               FieldMap fm, int copy_mode) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    int j = blockIdx.y * blockDim.y + threadIdx.y;
    int k = blockIdx.z;
    if (i > L.nx || j > L.ny || (L.dim == 3 && k > L.nz)) return;
    int64_t o = L.off(i + 1, j + 1, L.dim == 2 ? 0 : k + 1);
    for (int f = 0; f < nf; ++f) {
        int kind;
        if (L.dim == 2) kind = (f == 1) ? 1 : 0;
        else kind = (f <= 1 || f == 5) ? 0 : (f == 2 ? 4 : f == 3 ? 5 : 6);
        bool ex;
        int64_t fi;
        if (L.dim == 2) {
            ex = kind == 0 ? (i < L.nx && j < L.ny) : true;
            fi = fidx2(kind, i, j, L.nx, L.ny);
        } else {
            ex = kind == 0 ? (i < L.nx && j < L.ny && k < L.nz)
                           : kind == 4 ? k < L.nz : kind == 5 ? j < L.ny : i < L.nx;
            fi = fidx3(kind, i, j, k, L.nx, L.ny, L.nz);
        }
        if (!ex) continue;
        double* fp = fm.p[f];
        if (to_fields) fp[fi] = src[(int64_t)f * L.stride + o];
        else dst[(int64_t)f * L.stride + o] = fp[fi];
    }
    (void)f_off0; (void)copy_mode;
}

static dim3 slot_grid(const Layout& L) {
    return dim3((L.nx + 1 + 31) / 32, (L.ny + 1 + 7) / 8, L.dim == 2 ? 1 : L.nz + 1);
}

cudaError_t launch_rhs(Ctx* c, const double* const* ustar, double* b) {
    const Layout& L = c->L;
    FacePtrs us{{ustar[0], ustar[1], L.dim == 3 ? ustar[2] : nullptr}};
    cudaError_t e = cudaMemsetAsync(b, 0, sizeof(double) * c->vec_elems(), c->stream);
    if (e != cudaSuccess) return e;
    if (L.dim == 2) k_rhs2d<<<slot_grid(L), dim3(32, 8), 0, c->stream>>>(L, c->A, us, b);
    else k_rhs3d<<<slot_grid(L), dim3(32, 8), 0, c->stream>>>(L, c->A, us, b);
    return cudaGetLastError();
}

cudaError_t launch_recover(Ctx* c, const double* const* ustar, const double* x, double* const* uout) {
    const Layout& L = c->L;
    FacePtrs us{{ustar[0], ustar[1], L.dim == 3 ? ustar[2] : nullptr}};
    FaceOut out{{uout[0], uout[1], L.dim == 3 ? uout[2] : nullptr}};
    if (L.dim == 2) k_recover2d<<<slot_grid(L), dim3(32, 8), 0, c->stream>>>(L, c->A, us, x, out);
    else k_recover3d<<<slot_grid(L), dim3(32, 8), 0, c->stream>>>(L, c->A, us, x, out);
    return cudaGetLastError();
}

// Unknown vector <-> separate field-layout arrays (one per unknown field).
cudaError_t launch_unpack(Ctx* c, const double* slots, double* const* fields, int to_fields) {
    const Layout& L = c->L;
    FieldMap fm{};
    for (int f = 0; f < c->nf; ++f) fm.p[f] = fields[f];
    if (!to_fields) {
        cudaError_t e = cudaMemsetAsync((void*)slots, 0, sizeof(double) * c->vec_elems(), c->stream);
        if (e != cudaSuccess) return e;
    }
    k_slots_fields<<<slot_grid(L), dim3(32, 8), 0, c->stream>>>(L, slots, (double*)slots, to_fields, c->nf, 0, fm, 0);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Prescribed traction (Section 6.1): the face force
//   f = W_A^u (M^T x_BC) - M^T (W_A^x x_BC),  W_A = 1 - W_L (1 on eliminated
//   unknowns), M^T = [D^T | G],
// enters the first block row weighted like the mass term, so it shifts u* on
// live faces by dt/(rho W_L^u) f (the recovery coefficient).  The section
// prints the force with the opposite sign, which would give a liquid under a
// uniform surface pressure P0 the pressure -P0; this sign gives +P0.
// ---------------------------------------------------------------------------

// xa = W_A * xb per unknown field, on every slot (xb is zero where no sample
// exists)
__global__ void k_air_weight(Layout L, DevArrays D, int nf, const double* xb, double* xa) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    int j = blockIdx.y * blockDim.y + threadIdx.y;
    int k = blockIdx.z;
    if (i > L.nx || j > L.ny || (L.dim == 3 && k > L.nz)) return;
    const int64_t o = L.off(i + 1, j + 1, L.dim == 2 ? 0 : k + 1);
    for (int f = 0; f < nf; ++f) {
        // W_L kind and activity site of unknown field f
        int kind, site;
        if (L.dim == 2) { kind = f == 1 ? 1 : 0; site = f == 1 ? 1 : 0; }
        else if (f <= 1 || f == 5) { kind = 0; site = 0; }
        else { kind = f + 2; site = f - 1; }
        const double wl = D.act[site][o] ? D.WL[kind][o] : 0.0;
        xa[(int64_t)f * L.stride + o] = (1.0 - wl) * xb[(int64_t)f * L.stride + o];
    }
}

__global__ void k_traction2d(Layout L, DevArrays D, const double* xa, const double* xb, FacePtrs us, FaceOut out,
                             double inv_h) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    int j = blockIdx.y * blockDim.y + threadIdx.y;
    if (i > L.nx || j > L.ny) return;
    const int64_t S = L.stride;
    int c = i + 1, r = j + 1;
    int64_t o = L.off(c, r, 0);
    for (int d = 0; d < 2; ++d) {
        if (d == 0 && j >= L.ny) continue;
        if (d == 1 && i >= L.nx) continue;
        const int64_t fi = fidx2(2 + d, i, j, L.nx, L.ny);
        double u = us.p[d][fi];
        if (D.fflag[d][o] & F_LIVE) {
            // (M^T v) on this face for v = xa and v = xb
            auto mt = [&](const double* x) {
                auto U = [&](int64_t oo) { return x[2 * S + oo] - x[oo]; };
                auto V = [&](int64_t oo) { return x[2 * S + oo] + x[oo]; };
                auto N = [&](int64_t oo) { return x[S + oo]; };
                return d == 0 ? (U(o) - U(L.off(c - 1, r, 0))) + (N(o) - N(L.off(c, r + 1, 0)))
                              : (V(o) - V(L.off(c, r - 1, 0))) + (N(o) - N(L.off(c + 1, r, 0)));
            };
            const double wa = 1.0 - D.WL[2 + d][o];
            const double f = inv_h * (wa * mt(xb) - mt(xa));
            u += D.rec[d][o] * f;
        }
        out.p[d][fi] = u;
    }
}

__global__ void k_traction3d(Layout L, DevArrays D, const double* xa, const double* xb, FacePtrs us, FaceOut out,
                             double inv_h) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    int j = blockIdx.y * blockDim.y + threadIdx.y;
    int k = blockIdx.z;
    if (i > L.nx || j > L.ny || k > L.nz) return;
    const int64_t S = L.stride;
    int c = i + 1, r = j + 1, q = k + 1;
    int64_t o = L.off(c, r, q);
    for (int d = 0; d < 3; ++d) {
        bool ex = d == 0 ? (j < L.ny && k < L.nz) : d == 1 ? (i < L.nx && k < L.nz) : (i < L.nx && j < L.ny);
        if (!ex) continue;
        const int64_t fi = fidx3(1 + d, i, j, k, L.nx, L.ny, L.nz);
        double u = us.p[d][fi];
        if (D.fflag[d][o] & F_LIVE) {
            auto mt = [&](const double* x) {
                auto Uc = [&](int64_t oo) { return x[5 * S + oo] - x[oo]; };
                auto Vc = [&](int64_t oo) { return x[5 * S + oo] - x[S + oo]; };
                auto Wc = [&](int64_t oo) { return x[5 * S + oo] + x[oo] + x[S + oo]; };
                auto Nxy = [&](int64_t oo) { return x[2 * S + oo]; };
                auto Nxz = [&](int64_t oo) { return x[3 * S + oo]; };
                auto Nyz = [&](int64_t oo) { return x[4 * S + oo]; };
                if (d == 0)
                    return (Uc(o) - Uc(L.off(c - 1, r, q))) + (Nxy(o) - Nxy(L.off(c, r + 1, q))) +
                           (Nxz(o) - Nxz(L.off(c, r, q + 1)));
                if (d == 1)
                    return (Vc(o) - Vc(L.off(c, r - 1, q))) + (Nxy(o) - Nxy(L.off(c + 1, r, q))) +
                           (Nyz(o) - Nyz(L.off(c, r, q + 1)));
                return (Wc(o) - Wc(L.off(c, r, q - 1))) + (Nxz(o) - Nxz(L.off(c + 1, r, q))) +
                       (Nyz(o) - Nyz(L.off(c, r + 1, q)));
            };
            const double wa = 1.0 - D.WL[1 + d][o];
            const double f = inv_h * (wa * mt(xb) - mt(xa));
            u += D.rec[d][o] * f;
        }
        out.p[d][fi] = u;
    }
}

// u*_out = u* + dt/(rho W_L^u) f on live faces, u* elsewhere.  The prescribed
// fields (tau_BC fields then p_BC, field layout) go through two of the
// solver's work vectors.
cudaError_t launch_traction(Ctx* c, const double* const* bc_fields, const double* const* ustar, double* const* uout) {
    const Layout& L = c->L;
    double* xb = c->w64.z;
    double* xa = c->w64.q;
    cudaError_t e = launch_unpack(c, xb, (double* const*)bc_fields, 0);
    if (e != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(xa, 0, sizeof(double) * c->vec_elems(), c->stream)) != cudaSuccess) return e;
    k_air_weight<<<slot_grid(L), dim3(32, 8), 0, c->stream>>>(L, c->A, c->nf, xb, xa);
    FacePtrs us{{ustar[0], ustar[1], L.dim == 3 ? ustar[2] : nullptr}};
    FaceOut out{{uout[0], uout[1], L.dim == 3 ? uout[2] : nullptr}};
    if (L.dim == 2) k_traction2d<<<slot_grid(L), dim3(32, 8), 0, c->stream>>>(L, c->A, xa, xb, us, out, 1.0 / c->g.h);
    else k_traction3d<<<slot_grid(L), dim3(32, 8), 0, c->stream>>>(L, c->A, xa, xb, us, out, 1.0 / c->g.h);
    return cudaGetLastError();
}

}  // namespace stk
