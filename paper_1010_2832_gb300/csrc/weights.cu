// Weight build (stokes_build_weights): volume fractions of every sample's
// control volume (Section 5), face status and the null-space elimination of
// Section 8, operator coefficients, the Jacobi diagonal and the list of
// tiles that hold an active unknown.  One thread per slot of the padded
// vertex lattice; everything in FP64.
#include <algorithm>
#include "internal.cuh"
#include "ctx.cuh"

namespace stk {

// ---------------------------------------------------------------------------
// Fractions of {phi < 0} of the piecewise-linear interpolant on a simplex.
// Closed forms by the count k of negative vertices (sorted values s):
//   triangle  k=1: s0^2/((s0-s1)(s0-s2))       k=2: 1 - s2^2/((s2-s0)(s2-s1))
//   tetra     k=1: s0^3/((s0-s1)(s0-s2)(s0-s3)) k=3: 1 - s3^3/(...)
//             k=2: [x^2y^2 - (p+q)xy(x+y) + pq(x^2+xy+y^2)] / [(x-p)(x-q)(y-p)(y-q)]
// (the two-negative tetrahedron written without cancellation).
// ---------------------------------------------------------------------------
// Sign tests and ordering on the IEEE bit patterns (integer ALU; FP64
// compares and min/max run on the FP64 pipe, which is slow on this part).
// For finite values they decide exactly as v < 0, v > 0 and <= do
// (-0 is neither negative nor positive and orders with +0).
__device__ __forceinline__ bool dneg(double v) {
    const long long b = __double_as_longlong(v);
    return b < 0 && b != (long long)0x8000000000000000ULL;
}
__device__ __forceinline__ bool dpos(double v) { return __double_as_longlong(v) > 0; }
__device__ __forceinline__ long long dkey(double v) {
    const long long b = __double_as_longlong(v);
    return b ^ ((b >> 63) & 0x7FFFFFFFFFFFFFFFLL);
}
__device__ __forceinline__ void cswap(double& a, double& b) {
    if (dkey(b) < dkey(a)) {
        const double t = a;
        a = b;
        b = t;
    }
}

__device__ double tri_frac(double a, double b, double c) {
    cswap(a, b); cswap(b, c); cswap(a, b);
    int k = dneg(a) + dneg(b) + dneg(c);
    if (k == 0) return 0.0;
    if (k == 3) return 1.0;
    if (k == 1) return __dmul_rn(a, a) / __dmul_rn(__dsub_rn(a, b), __dsub_rn(a, c));
    return 1.0 - __dmul_rn(c, c) / __dmul_rn(__dsub_rn(c, a), __dsub_rn(c, b));
}

__device__ double tet_frac(double a, double b, double c, double d) {
    cswap(a, b); cswap(c, d); cswap(a, c); cswap(b, d); cswap(b, c);
    int k = dneg(a) + dneg(b) + dneg(c) + dneg(d);
    if (k == 0) return 0.0;
    if (k == 4) return 1.0;
    if (k == 1) {
        double num = __dmul_rn(__dmul_rn(a, a), a);
        double den = __dmul_rn(__dmul_rn(__dsub_rn(a, b), __dsub_rn(a, c)), __dsub_rn(a, d));
        return num / den;
    }
    if (k == 3) {
        double num = __dmul_rn(__dmul_rn(d, d), d);
        double den = __dmul_rn(__dmul_rn(__dsub_rn(d, a), __dsub_rn(d, b)), __dsub_rn(d, c));
        return 1.0 - num / den;
    }
    // evaluation order (left to right, no fused multiply-add):
    //   ((x x) y) y - (((p + q) x) y)(x + y) + (p q)((x x + x y) + y y)
    //   over (((x - p)(x - q))(y - p))(y - q)
    double x = a, y = b, p = c, q = d;
    double xx = __dmul_rn(x, x), yy = __dmul_rn(y, y), xy = __dmul_rn(x, y);
    double t1 = __dmul_rn(__dmul_rn(xx, y), y);
    double t2 = __dmul_rn(__dmul_rn(__dmul_rn(__dadd_rn(p, q), x), y), __dadd_rn(x, y));
    double t3 = __dmul_rn(__dmul_rn(p, q), __dadd_rn(__dadd_rn(xx, xy), yy));
    double num = __dadd_rn(__dsub_rn(t1, t2), t3);
    double den = __dmul_rn(__dmul_rn(__dmul_rn(__dsub_rn(x, p), __dsub_rn(x, q)), __dsub_rn(y, p)), __dsub_rn(y, q));
    return num / den;
}

// A CV whose lattice values have one sign is exactly 0 or 1 (the simplex
// formulas give the same; the test only skips work).  Mixed CVs keep the
// computed value.  Every operation above is rounded separately and in the
// same order as in the FP64 reference, so the values, and every W > 0 test
// on them, are reproducible bit for bit.
__device__ __forceinline__ double clamp_open(double f) { return f; }

// 2D CV centred at lattice (a, b); lattice row length Lx.  8 triangles
// (centre, edge midpoint, corner).
__device__ double cv_frac_2d(const double* phi, int Lx, int a, int b) {
    double v[9];
    int n = 0;
    // ring order E, NE, N, NW, W, SW, S, SE
    const int da[8] = {1, 1, 0, -1, -1, -1, 0, 1};
    const int db[8] = {0, 1, 1, 1, 0, -1, -1, -1};
    double c = phi[(int64_t)b * Lx + a];
    int neg = dneg(c), pos = dpos(c);
    for (int t = 0; t < 8; ++t) {
        v[t] = phi[(int64_t)(b + db[t]) * Lx + (a + da[t])];
        neg |= dneg(v[t]); pos |= dpos(v[t]);
    }
    (void)n;
    if (!neg) return 0.0;
    if (!pos) return 1.0;
    double s = 0.0;
    for (int t = 0; t < 8; ++t) s += tri_frac(c, v[t], v[(t + 1) & 7]);
    return clamp_open(s / 8.0);
}

// 3D CV centred at lattice (a, b, c).  24 tetrahedra (centre, face centre,
// two consecutive corners of that face), faces in the order -x, +x, -y, +y,
// -z, +z and corners cycling (-,-), (+,-), (+,+), (-,+) over the two other
// axes in increasing axis order.
__device__ double cv_frac_3d(const double* phi, int Lx, int Ly, int a, int b, int c) {
    auto P = [&](int da, int db, int dc) -> double {
        return phi[((int64_t)(c + dc) * Ly + (b + db)) * Lx + (a + da)];
    };
    int neg = 0, pos = 0;
    for (int dc = -1; dc <= 1; ++dc)
        for (int db = -1; db <= 1; ++db)
            for (int da = -1; da <= 1; ++da) {
                double v = P(da, db, dc);
                neg |= dneg(v); pos |= dpos(v);
            }
    if (!neg) return 0.0;
    if (!pos) return 1.0;
    double centre = P(0, 0, 0);
    const int lu[4] = {-1, 1, 1, -1}, lv[4] = {-1, -1, 1, 1};
    double s = 0.0;
    for (int axis = 0; axis < 3; ++axis) {
        for (int sg = -1; sg <= 1; sg += 2) {
            int o[3] = {0, 0, 0};
            o[axis] = sg;
            double fc = P(o[0], o[1], o[2]);
            int ua = axis == 0 ? 1 : 0, va = axis == 2 ? 1 : 2;
            double cr[4];
            for (int t = 0; t < 4; ++t) {
                int q[3] = {o[0], o[1], o[2]};
                q[ua] = lu[t]; q[va] = lv[t];
                cr[t] = P(q[0], q[1], q[2]);
            }
            for (int t = 0; t < 4; ++t) s += tet_frac(centre, fc, cr[t], cr[(t + 1) & 3]);
        }
    }
    return clamp_open(s / 24.0);
}

// Sample kinds.  2D: 0 cell, 1 node, 2 u, 3 v.  3D: 0 cell, 1 u, 2 v, 3 w,
// 4 exy, 5 exz, 6 eyz.  Lattice offset per axis (a = 2 i + off).
__constant__ int c_off2[4][2] = {{2, 2}, {1, 1}, {1, 2}, {2, 1}};
__constant__ int c_off3[7][3] = {{2, 2, 2}, {1, 2, 2}, {2, 1, 2}, {2, 2, 1}, {1, 1, 2}, {1, 2, 1}, {2, 1, 1}};

__host__ __device__ __forceinline__ bool exists2(int kind, int i, int j, int nx, int ny) {
    if (i < 0 || j < 0 || i > nx || j > ny) return false;
    switch (kind) {
        case 0: return i < nx && j < ny;
        case 1: return true;
        case 2: return j < ny;
        default: return i < nx;
    }
}

__host__ __device__ __forceinline__ bool exists3(int kind, int i, int j, int k, int nx, int ny, int nz) {
    if (i < 0 || j < 0 || k < 0 || i > nx || j > ny || k > nz) return false;
    switch (kind) {
        case 0: return i < nx && j < ny && k < nz;
        case 1: return j < ny && k < nz;
        case 2: return i < nx && k < nz;
        case 3: return i < nx && j < ny;
        case 4: return k < nz;
        case 5: return j < ny;
        default: return i < nx;
    }
}

// ---- kernel 1: fractions ----------------------------------------------------
// 2D form of block_sign3: the block [2i, 2i+3]^2, clipped to the lattice.
__device__ __forceinline__ int block_sign2(const double* phi, int Lx, int Ly, int i, int j) {
    int neg = 0, nonneg = 0;
    const int ea = min(4, Lx - 2 * i), eb = min(4, Ly - 2 * j);
    for (int db = 0; db < eb; ++db)
        for (int da = 0; da < ea; ++da) {
            const int n = dneg(phi[(int64_t)(2 * j + db) * Lx + (2 * i + da)]);
            neg |= n;
            nonneg |= !n;
        }
    return !neg ? 0 : (!nonneg ? 1 : -1);
}

__global__ void k_fractions2d(Layout L, const double* phiL, const double* phiS, DevArrays D) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    int j = blockIdx.y * blockDim.y + threadIdx.y;
    if (i > L.nx || j > L.ny) return;
    int Lx = 2 * L.nx + 3, Ly = 2 * L.ny + 3;
    int64_t o = L.off(i + 1, j + 1, 0);
    const int bl = block_sign2(phiL, Lx, Ly, i, j), bs = block_sign2(phiS, Lx, Ly, i, j);
    for (int kd = 0; kd < 4; ++kd) {
        if (!exists2(kd, i, j, L.nx, L.ny)) continue;
        int a = 2 * i + c_off2[kd][0], b = 2 * j + c_off2[kd][1];
        D.WL[kd][o] = bl >= 0 ? (double)bl : cv_frac_2d(phiL, Lx, a, b);
        D.WF[kd][o] = bs >= 0 ? 1.0 - (double)bs : 1.0 - cv_frac_2d(phiS, Lx, a, b);
    }
}

// Sign summary of the lattice block [2i, 2i+3]^3 (clipped to the lattice,
// whose last index per axis is 2n+2) that holds the control volumes of all
// seven sample kinds of slot (i, j, k) that exist (at i = nx only kinds
// centred at 2i+1 exist, and their points end at 2nx+2): 0 if the block has
// no negative value (every fraction is 0), 1 if every value is negative
// (every fraction is 1), -1 otherwise (evaluate each kind).
__device__ __forceinline__ int block_sign3(const double* phi, int Lx, int Ly, int Lz, int i, int j, int k) {
    int neg = 0, nonneg = 0;
    const int ea = min(4, Lx - 2 * i), eb = min(4, Ly - 2 * j), ec = min(4, Lz - 2 * k);
    for (int dc = 0; dc < ec; ++dc)
        for (int db = 0; db < eb; ++db)
            for (int da = 0; da < ea; ++da) {
                const double v = phi[((int64_t)(2 * k + dc) * Ly + (2 * j + db)) * Lx + (2 * i + da)];
                const int n = dneg(v);
                neg |= n;
                nonneg |= !n;
            }
    return !neg ? 0 : (!nonneg ? 1 : -1);
}

// Fraction of the CV centred at lattice (a, b, c) computed by a whole warp
// (every lane must call it with the same arguments): lanes 0..26 test the 27
// lattice values for one sign; otherwise lane l < 24 evaluates tetrahedron l
// (faces -x, +x, -y, +y, -z, +z, four per face, as in cv_frac_3d) and the 24
// values are added in that order, so the result is cv_frac_3d's bit for bit.
__device__ double cv_frac_3d_warp(const double* phi, int Lx, int Ly, int a, int b, int c) {
    const int lane = threadIdx.x & 31;
    auto P = [&](int da, int db, int dc) -> double {
        return phi[((int64_t)(c + dc) * Ly + (b + db)) * Lx + (a + da)];
    };
    int isneg = 0, ispos = 0;
    if (lane < 27) {
        const double v = P(lane % 3 - 1, (lane / 3) % 3 - 1, lane / 9 - 1);
        isneg = dneg(v);
        ispos = dpos(v);
    }
    const unsigned neg = __ballot_sync(0xffffffffu, isneg), pos = __ballot_sync(0xffffffffu, ispos);
    if (!neg) return 0.0;
    if (!pos) return 1.0;
    double tv = 0.0;
    if (lane < 24) {
        const int face = lane >> 2, t = lane & 3;
        const int axis = face >> 1, sg = (face & 1) ? 1 : -1;
        int o[3] = {0, 0, 0};
        o[axis] = sg;
        const int ua = axis == 0 ? 1 : 0, va = axis == 2 ? 1 : 2;
        const int lu[4] = {-1, 1, 1, -1}, lv[4] = {-1, -1, 1, 1};
        int q0[3] = {o[0], o[1], o[2]}, q1[3] = {o[0], o[1], o[2]};
        q0[ua] = lu[t]; q0[va] = lv[t];
        q1[ua] = lu[(t + 1) & 3]; q1[va] = lv[(t + 1) & 3];
        tv = tet_frac(P(0, 0, 0), P(o[0], o[1], o[2]), P(q0[0], q0[1], q0[2]), P(q1[0], q1[1], q1[2]));
    }
    double sum = 0.0;
    for (int l = 0; l < 24; ++l) sum += __shfl_sync(0xffffffffu, tv, l);
    return clamp_open(sum / 24.0);
}

// One thread per slot decides, from a sign scan of its lattice block, which
// of its fractions are 0 or 1 outright; the control volumes cut by an
// interface are then evaluated by the whole warp, one at a time (the
// interfaces are thin, so most warps hold few of them, and a serial
// per-thread evaluation would leave the other lanes idle on the slow FP64
// pipe).
__global__ void k_fractions3d(Layout L, const double* phiL, const double* phiS, DevArrays D) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    int j = blockIdx.y * blockDim.y + threadIdx.y;
    int k = blockIdx.z;
    const bool inside = i <= L.nx && j <= L.ny && k <= L.nz;
    int Lx = 2 * L.nx + 3, Ly = 2 * L.ny + 3, Lz = 2 * L.nz + 3;
    int64_t o = inside ? L.off(i + 1, j + 1, k + 1) : 0;
    unsigned need = 0;                          // bit kd: W_L of kind kd, bit 7 + kd: W_F
    if (inside) {
        // the seven CVs lie in a 4x4x4 block of the (padded) lattice: one
        // sign scan of it settles every kind away from the interfaces
        const int bl = block_sign3(phiL, Lx, Ly, Lz, i, j, k), bs = block_sign3(phiS, Lx, Ly, Lz, i, j, k);
        for (int kd = 0; kd < 7; ++kd) {
            if (!exists3(kd, i, j, k, L.nx, L.ny, L.nz)) continue;
            if (bl >= 0) D.WL[kd][o] = (double)bl; else need |= 1u << kd;
            if (bs >= 0) D.WF[kd][o] = 1.0 - (double)bs; else need |= 1u << (7 + kd);
        }
    }
    unsigned todo = __ballot_sync(0xffffffffu, need != 0);
    while (todo) {
        const int src = __ffs(todo) - 1;
        todo &= todo - 1;
        const unsigned nd = __shfl_sync(0xffffffffu, need, src);
        const int si = __shfl_sync(0xffffffffu, i, src), sj = __shfl_sync(0xffffffffu, j, src);
        const long long so = __shfl_sync(0xffffffffu, (long long)o, src);
        for (int bit = 0; bit < 14; ++bit) {
            if (!(nd & (1u << bit))) continue;
            const int kd = bit % 7;
            const int a = 2 * si + c_off3[kd][0], b = 2 * sj + c_off3[kd][1], c = 2 * k + c_off3[kd][2];
            if (bit < 7) {
                const double f = cv_frac_3d_warp(phiL, Lx, Ly, a, b, c);
                if ((threadIdx.x & 31) == src) D.WL[kd][so] = f;
            } else {
                const double f = cv_frac_3d_warp(phiS, Lx, Ly, a, b, c);
                if ((threadIdx.x & 31) == src) D.WF[kd][so] = 1.0 - f;
            }
        }
    }
}

// zero-fluid-weight multiplier: W_L > 0 and W_F == 0 (Section 8, solid side)
__device__ __forceinline__ bool zwm(const DevArrays& D, int kind, int64_t o) {
    return D.WL[kind][o] > 0.0 && D.WF[kind][o] == 0.0;
}

// ---- kernel 2: faces ----------------------------------------------------------
// Adjacent multiplier samples of each face (through D and G^T):
//   2D u(i,j): cells (i-1,j),(i,j); nodes (i,j),(i,j+1)
//   2D v(i,j): cells (i,j-1),(i,j); nodes (i,j),(i+1,j)
//   3D u: cells (i-1),(i); exy (i,j),(i,j+1); exz (i,j,k),(i,j,k+1)
//   3D v: cells (j-1),(j); exy (i,j),(i+1,j); eyz (i,j,k),(i,j,k+1)
//   3D w: cells (k-1),(k); exz (i,j,k),(i+1,j,k); eyz (i,j,k),(i,j+1,k)
// wl_min floors the liquid fraction of live faces where it is their mass
// (K and the recovery coefficient); 0 keeps the fractions as computed.
__global__ void k_faces2d(Layout L, double dt, double wl_min, const double* rho_u, const double* rho_v,
                          const double* ubc_u, const double* ubc_v, DevArrays D) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    int j = blockIdx.y * blockDim.y + threadIdx.y;
    if (i > L.nx || j > L.ny) return;
    for (int d = 0; d < 2; ++d) {
        int kind = 2 + d;
        if (!exists2(kind, i, j, L.nx, L.ny)) continue;
        int64_t o = L.off(i + 1, j + 1, 0);
        uint8_t fl = F_EXISTS;
        double wf = D.WF[kind][o], wl = D.WL[kind][o];
        bool wall = d == 0 ? (i == 0 || i == L.nx) : (j == 0 || j == L.ny);
        if (wall) { fl |= F_WALL; wf = 0.0; }
        if (wf > 0.0) {
            bool inval;
            if (d == 0)
                inval = (i > 0 && zwm(D, 0, L.off(i, j + 1, 0))) || (i < L.nx && zwm(D, 0, o)) ||
                        zwm(D, 1, o) || zwm(D, 1, L.off(i + 1, j + 2, 0));
            else
                inval = (j > 0 && zwm(D, 0, L.off(i + 1, j, 0))) || (j < L.ny && zwm(D, 0, o)) ||
                        zwm(D, 1, o) || zwm(D, 1, L.off(i + 2, j + 1, 0));
            if (inval) { fl |= F_INVALID; wf = 0.0; }
        }
        double K = 0.0, rec = 0.0;
        if (wf > 0.0 && wl > 0.0) {
            fl |= F_LIVE;
            double rho = (d == 0 ? rho_u : rho_v)[fidx2(kind, i, j, L.nx, L.ny)];
            double wm = fmax(wl, wl_min);
            K = (dt * wf) / (rho * wm);
            rec = dt / (rho * wm);
        } else if (wf > 0.0) {
            fl |= F_BAD;
        }
        D.fflag[d][o] = fl;
        D.effWF[d][o] = wf;
        D.K64[d][o] = K;
        D.rec[d][o] = rec;
        D.ubc[d][o] = (d == 0 ? ubc_u : ubc_v)[fidx2(kind, i, j, L.nx, L.ny)];
    }
}

__global__ void k_faces3d(Layout L, double dt, double wl_min, Ptr3 rho, Ptr3 ubc, DevArrays D) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    int j = blockIdx.y * blockDim.y + threadIdx.y;
    int k = blockIdx.z;
    if (i > L.nx || j > L.ny || k > L.nz) return;
    int64_t o = L.off(i + 1, j + 1, k + 1);
    for (int d = 0; d < 3; ++d) {
        int kind = 1 + d;
        if (!exists3(kind, i, j, k, L.nx, L.ny, L.nz)) continue;
        uint8_t fl = F_EXISTS;
        double wf = D.WF[kind][o], wl = D.WL[kind][o];
        bool wall = d == 0 ? (i == 0 || i == L.nx) : d == 1 ? (j == 0 || j == L.ny) : (k == 0 || k == L.nz);
        if (wall) { fl |= F_WALL; wf = 0.0; }
        if (wf > 0.0) {
            bool inval = false;
            // cells on both sides along d (interior faces: both exist)
            int64_t om = d == 0 ? L.off(i, j + 1, k + 1) : d == 1 ? L.off(i + 1, j, k + 1) : L.off(i + 1, j + 1, k);
            inval |= zwm(D, 0, om) || zwm(D, 0, o);
            if (d == 0) {
                inval |= zwm(D, 4, o) || zwm(D, 4, L.off(i + 1, j + 2, k + 1));
                inval |= zwm(D, 5, o) || zwm(D, 5, L.off(i + 1, j + 1, k + 2));
            } else if (d == 1) {
                inval |= zwm(D, 4, o) || zwm(D, 4, L.off(i + 2, j + 1, k + 1));
                inval |= zwm(D, 6, o) || zwm(D, 6, L.off(i + 1, j + 1, k + 2));
            } else {
                inval |= zwm(D, 5, o) || zwm(D, 5, L.off(i + 2, j + 1, k + 1));
                inval |= zwm(D, 6, o) || zwm(D, 6, L.off(i + 1, j + 2, k + 1));
            }
            if (inval) { fl |= F_INVALID; wf = 0.0; }
        }
        double K = 0.0, rec = 0.0;
        int64_t fi = fidx3(kind, i, j, k, L.nx, L.ny, L.nz);
        if (wf > 0.0 && wl > 0.0) {
            fl |= F_LIVE;
            double r = rho.p[d][fi];
            double wm = fmax(wl, wl_min);
            K = (dt * wf) / (r * wm);
            rec = dt / (r * wm);
        } else if (wf > 0.0) {
            fl |= F_BAD;
        }
        D.fflag[d][o] = fl;
        D.effWF[d][o] = wf;
        D.K64[d][o] = K;
        D.rec[d][o] = rec;
        D.ubc[d][o] = ubc.p[d][fi];
    }
}

// ---- kernel 3: unknown validity and coefficients -------------------------------
__device__ __forceinline__ void face_state(const DevArrays& D, int d, int64_t o, bool& bad, bool& live) {
    uint8_t f = D.fflag[d][o];
    bad |= (f & F_BAD) != 0;
    live |= (f & F_LIVE) != 0;
}

__global__ void k_unknowns2d(Layout L, double inv_h, const double* mu_c, const double* mu_n, DevArrays D) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    int j = blockIdx.y * blockDim.y + threadIdx.y;
    if (i > L.nx || j > L.ny) return;
    int64_t o = L.off(i + 1, j + 1, 0);
    double* a_c = D.coef64 + 0 * L.stride;
    double* a_n = D.coef64 + 1 * L.stride;
    double* d_c = D.coef64 + 2 * L.stride;
    double* d_n = D.coef64 + 3 * L.stride;
    // cell: faces u(i), u(i+1), v(j), v(j+1)
    if (i < L.nx && j < L.ny) {
        bool bad = false, live = false;
        face_state(D, 0, o, bad, live);
        face_state(D, 0, L.off(i + 2, j + 1, 0), bad, live);
        face_state(D, 1, o, bad, live);
        face_state(D, 1, L.off(i + 1, j + 2, 0), bad, live);
        double wl = D.WL[0][o], wf = D.WF[0][o];
        bool act = wl > 0.0 && !bad && live;
        a_c[o] = act ? wl * inv_h : 0.0;
        d_c[o] = act ? (wl * wf) / mu_c[fidx2(0, i, j, L.nx, L.ny)] : 1.0;
        D.act[0][o] = act;
    }
    // node: faces u(i, j-1), u(i, j), v(i-1, j), v(i, j)
    {
        bool bad = false, live = false;
        if (j > 0) face_state(D, 0, L.off(i + 1, j, 0), bad, live);
        if (j < L.ny) face_state(D, 0, o, bad, live);
        if (i > 0) face_state(D, 1, L.off(i, j + 1, 0), bad, live);
        if (i < L.nx) face_state(D, 1, o, bad, live);
        double wl = D.WL[1][o], wf = D.WF[1][o];
        bool act = wl > 0.0 && !bad && (wf > 0.0 || live);
        a_n[o] = act ? wl * inv_h : 0.0;
        d_n[o] = act ? (wl * wf) / mu_n[fidx2(1, i, j, L.nx, L.ny)] : 1.0;
        D.act[1][o] = act;
    }
}

__global__ void k_unknowns3d(Layout L, double inv_h, Ptr4 mu, DevArrays D) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    int j = blockIdx.y * blockDim.y + threadIdx.y;
    int k = blockIdx.z;
    if (i > L.nx || j > L.ny || k > L.nz) return;
    int64_t o = L.off(i + 1, j + 1, k + 1);
    // coefficient fields: 0 a_c, 1 a_xy, 2 a_xz, 3 a_yz, 4 d_c, 5 d_xy, 6 d_xz, 7 d_yz
    auto A = [&](int f) { return D.coef64 + (int64_t)f * L.stride; };
    int64_t ox = L.off(i + 2, j + 1, k + 1), oy = L.off(i + 1, j + 2, k + 1), oz = L.off(i + 1, j + 1, k + 2);
    int64_t mx = L.off(i, j + 1, k + 1), my = L.off(i + 1, j, k + 1), mz = L.off(i + 1, j + 1, k);
    if (i < L.nx && j < L.ny && k < L.nz) {
        bool bad = false, live = false;
        face_state(D, 0, o, bad, live); face_state(D, 0, ox, bad, live);
        face_state(D, 1, o, bad, live); face_state(D, 1, oy, bad, live);
        face_state(D, 2, o, bad, live); face_state(D, 2, oz, bad, live);
        double wl = D.WL[0][o], wf = D.WF[0][o];
        bool act = wl > 0.0 && !bad && live;
        A(0)[o] = act ? wl * inv_h : 0.0;
        A(4)[o] = act ? (wl * wf) / mu.p[0][fidx3(0, i, j, k, L.nx, L.ny, L.nz)] : 1.0;
        D.act[0][o] = act;
    }
    // exy (z-edge): u(i,j-1,k), u(i,j,k), v(i-1,j,k), v(i,j,k)
    if (k < L.nz) {
        bool bad = false, live = false;
        if (j > 0) face_state(D, 0, my, bad, live);
        if (j < L.ny) face_state(D, 0, o, bad, live);
        if (i > 0) face_state(D, 1, mx, bad, live);
        if (i < L.nx) face_state(D, 1, o, bad, live);
        double wl = D.WL[4][o], wf = D.WF[4][o];
        bool act = wl > 0.0 && !bad && (wf > 0.0 || live);
        A(1)[o] = act ? wl * inv_h : 0.0;
        A(5)[o] = act ? (wl * wf) / mu.p[1][fidx3(4, i, j, k, L.nx, L.ny, L.nz)] : 1.0;
        D.act[1][o] = act;
    }
    // exz (y-edge): u(i,j,k-1), u(i,j,k), w(i-1,j,k), w(i,j,k)
    if (j < L.ny) {
        bool bad = false, live = false;
        if (k > 0) face_state(D, 0, mz, bad, live);
        if (k < L.nz) face_state(D, 0, o, bad, live);
        if (i > 0) face_state(D, 2, mx, bad, live);
        if (i < L.nx) face_state(D, 2, o, bad, live);
        double wl = D.WL[5][o], wf = D.WF[5][o];
        bool act = wl > 0.0 && !bad && (wf > 0.0 || live);
        A(2)[o] = act ? wl * inv_h : 0.0;
        A(6)[o] = act ? (wl * wf) / mu.p[2][fidx3(5, i, j, k, L.nx, L.ny, L.nz)] : 1.0;
        D.act[2][o] = act;
    }
    // eyz (x-edge): v(i,j,k-1), v(i,j,k), w(i,j-1,k), w(i,j,k)
    if (i < L.nx) {
        bool bad = false, live = false;
        if (k > 0) face_state(D, 1, mz, bad, live);
        if (k < L.nz) face_state(D, 1, o, bad, live);
        if (j > 0) face_state(D, 2, my, bad, live);
        if (j < L.ny) face_state(D, 2, o, bad, live);
        double wl = D.WL[6][o], wf = D.WF[6][o];
        bool act = wl > 0.0 && !bad && (wf > 0.0 || live);
        A(3)[o] = act ? wl * inv_h : 0.0;
        A(7)[o] = act ? (wl * wf) / mu.p[3][fidx3(6, i, j, k, L.nx, L.ny, L.nz)] : 1.0;
        D.act[3][o] = act;
    }
}

// ---- kernel 4: Jacobi inverse diagonal, reduced-precision copies, tile flags
__global__ void k_finish2d(Layout L, DevArrays D) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    int j = blockIdx.y * blockDim.y + threadIdx.y;
    if (i > L.nx || j > L.ny) return;
    int64_t o = L.off(i + 1, j + 1, 0);
    const double* Ku = D.K64[0];
    const double* Kv = D.K64[1];
    const double* cf = D.coef64;
    double ac = cf[o], an = cf[L.stride + o], dc = cf[2 * L.stride + o], dn = cf[3 * L.stride + o];
    bool tile_act = false;
    if (i < L.nx && j < L.ny) {
        double sK = Ku[o] + Ku[L.off(i + 2, j + 1, 0)] + Kv[o] + Kv[L.off(i + 1, j + 2, 0)];
        bool act = D.act[0][o];
        D.minv64[0 * L.stride + o] = act ? 1.0 / (dc + ac * ac * sK) : 1.0;
        D.minv64[2 * L.stride + o] = act ? 1.0 / (ac * ac * sK) : 1.0;
        tile_act |= act;
    }
    {
        double sK = Ku[o] + Ku[L.off(i + 1, j, 0)] + Kv[o] + Kv[L.off(i, j + 1, 0)];
        bool act = D.act[1][o];
        D.minv64[1 * L.stride + o] = act ? 1.0 / (dn + an * an * sK) : 1.0;
        tile_act |= act;
    }
    // K fields live in the coefficient array as fields 4 and 5
    D.coef64[4 * L.stride + o] = Ku[o];
    D.coef64[5 * L.stride + o] = Kv[o];
    uint32_t h[6];
    for (int f = 0; f < 6; ++f) {
        double v = D.coef64[(int64_t)f * L.stride + o];
        D.coef32[(int64_t)f * L.stride + o] = (float)v;
        const __nv_bfloat16 b = __double2bfloat16(v);
        D.coef16[(int64_t)f * L.stride + o] = b;
        h[f] = __bfloat16_as_ushort(b);
    }
    // the same BF16 values in pairs (a_c, a_n), (d_c, d_n), (K_u, K_v)
    for (int k = 0; k < 3; ++k) D.pair16[(int64_t)k * L.stride + o] = h[2 * k] | (h[2 * k + 1] << 16);
    for (int f = 0; f < 3; ++f) D.minv32[(int64_t)f * L.stride + o] = (float)D.minv64[(int64_t)f * L.stride + o];
    if (tile_act) {
        int c = i + 1, r = j + 1;
        D.tile_flag[(r / TY2) * L.ntx + c / TX] = 1;
        D.tile_flag4[(r / 4) * L.ntx + c / TX] = 1;
    }
}

__global__ void k_finish3d(Layout L, DevArrays D) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    int j = blockIdx.y * blockDim.y + threadIdx.y;
    int k = blockIdx.z;
    if (i > L.nx || j > L.ny || k > L.nz) return;
    int64_t o = L.off(i + 1, j + 1, k + 1);
    int64_t S = L.stride;
    const double *Ku = D.K64[0], *Kv = D.K64[1], *Kw = D.K64[2];
    const double* cf = D.coef64;
    int64_t ox = L.off(i + 2, j + 1, k + 1), oy = L.off(i + 1, j + 2, k + 1), oz = L.off(i + 1, j + 1, k + 2);
    int64_t mx = L.off(i, j + 1, k + 1), my = L.off(i + 1, j, k + 1), mz = L.off(i + 1, j + 1, k);
    bool tile_act = false;
    // unknown fields: 0 txx, 1 tyy, 2 txy, 3 txz, 4 tyz, 5 p
    if (i < L.nx && j < L.ny && k < L.nz) {
        double ac = cf[o], dc = cf[4 * S + o];
        double su = Ku[o] + Ku[ox], sv = Kv[o] + Kv[oy], sw = Kw[o] + Kw[oz];
        bool act = D.act[0][o];
        double a2 = ac * ac;
        D.minv64[0 * S + o] = act ? 1.0 / (dc + a2 * (su + sw)) : 1.0;
        D.minv64[1 * S + o] = act ? 1.0 / (dc + a2 * (sv + sw)) : 1.0;
        D.minv64[5 * S + o] = act ? 1.0 / (a2 * (su + sv + sw)) : 1.0;
        tile_act |= act;
    }
    if (k < L.nz) {
        double a = cf[1 * S + o], d = cf[5 * S + o];
        double s = Ku[my] + Ku[o] + Kv[mx] + Kv[o];
        bool act = D.act[1][o];
        D.minv64[2 * S + o] = act ? 1.0 / (d + a * a * s) : 1.0;
        tile_act |= act;
    }
    if (j < L.ny) {
        double a = cf[2 * S + o], d = cf[6 * S + o];
        double s = Ku[mz] + Ku[o] + Kw[mx] + Kw[o];
        bool act = D.act[2][o];
        D.minv64[3 * S + o] = act ? 1.0 / (d + a * a * s) : 1.0;
        tile_act |= act;
    }
    if (i < L.nx) {
        double a = cf[3 * S + o], d = cf[7 * S + o];
        double s = Kv[mz] + Kv[o] + Kw[my] + Kw[o];
        bool act = D.act[3][o];
        D.minv64[4 * S + o] = act ? 1.0 / (d + a * a * s) : 1.0;
        tile_act |= act;
    }
    D.coef64[8 * S + o] = Ku[o];
    D.coef64[9 * S + o] = Kv[o];
    D.coef64[10 * S + o] = Kw[o];
    uint32_t h[8];
    for (int f = 0; f < 11; ++f) {
        double v = D.coef64[(int64_t)f * S + o];
        D.coef32[(int64_t)f * S + o] = (float)v;
        const __nv_bfloat16 b = __double2bfloat16(v);
        D.coef16[(int64_t)f * S + o] = b;
        if (f < 8) h[f] = __bfloat16_as_ushort(b);
    }
    // the same BF16 values in fours: (a_c, a_xy, a_xz, a_yz), (d_c, d_xy, d_xz, d_yz)
    for (int k = 0; k < 2; ++k)
        D.quad16[(int64_t)k * S + o] = make_uint2(h[4 * k] | (h[4 * k + 1] << 16), h[4 * k + 2] | (h[4 * k + 3] << 16));
    for (int f = 0; f < 6; ++f) D.minv32[(int64_t)f * S + o] = (float)D.minv64[(int64_t)f * S + o];
    if (tile_act) {
        int c = i + 1, r = j + 1, q = k + 1;
        D.tile_flag[((int64_t)(q / TZ3) * L.nty + r / TY3) * L.ntx + c / TX] = 1;
    }
}

// Tile mask of every 3D apply unit (32 x 8 slots x zt tile layers; bit
// dy + 2 dz), tiles past the tile grid counted inactive.
__global__ void k_unit_masks(Layout L, int zt, const uint8_t* __restrict__ tflag, uint8_t* __restrict__ umask,
                             int nunits) {
    const int u = blockIdx.x * blockDim.x + threadIdx.x;
    if (u >= nunits) return;
    const int nuy = units_y(L.nty);
    const int ux = u % L.ntx, rest = u / L.ntx, uy = rest % nuy, uz = rest / nuy;
    unsigned m = 0;
    for (int dz = 0; dz < zt; ++dz)
        for (int dy = 0; dy < 2; ++dy) {
            const int ty = 2 * uy + dy, tz = zt * uz + dz;
            if (ty < L.nty && tz < L.ntz && tflag[((int64_t)tz * L.nty + ty) * L.ntx + ux]) m |= 1u << (dy + 2 * dz);
        }
    umask[u] = (uint8_t)m;
}

// Ordered compaction of the tile flags (one block; tile counts are small).
__global__ void k_compact_tiles(const uint8_t* flag, int n, int* list, int* count) {
    __shared__ int warp_tot[32];
    __shared__ int base;
    if (threadIdx.x == 0) base = 0;
    __syncthreads();
    for (int start = 0; start < n; start += blockDim.x) {
        int t = start + threadIdx.x;
        int f = (t < n && flag[t]) ? 1 : 0;
        unsigned m = __ballot_sync(0xffffffffu, f);
        int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
        int before = __popc(m & ((1u << lane) - 1u));
        if (lane == 0) warp_tot[w] = __popc(m);
        __syncthreads();
        int off = 0;
        for (int q = 0; q < w; ++q) off += warp_tot[q];
        if (f) list[base + off + before] = t;
        __syncthreads();
        if (threadIdx.x == 0) {
            int tot = 0;
            for (int q = 0; q < (int)(blockDim.x >> 5); ++q) tot += warp_tot[q];
            base += tot;
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) *count = base;
}

cudaError_t launch_build_weights(Ctx* c, const double* phiL, const double* phiS, const double* const* rho,
                                 const double* const* mu, const double* const* ubc) {
    const Layout& L = c->L;
    cudaStream_t s = c->stream;
    DevArrays D = c->dev_arrays();
    cudaError_t e;
    cudaGetLastError();   // a stale, non-sticky error from earlier work is not this call's
    // pads and guards must read as zero; coefficients of inactive real
    // unknowns are written below
    if ((e = c->zero_weights()) != cudaSuccess) return e;
    dim3 blk(32, 8);
    if (L.dim == 2) {
        dim3 grd((L.nx + 1 + 31) / 32, (L.ny + 1 + 7) / 8);
        k_fractions2d<<<grd, blk, 0, s>>>(L, phiL, phiS, D);
        k_faces2d<<<grd, blk, 0, s>>>(L, c->g.dt, c->min_face_liquid, rho[0], rho[1], ubc[0], ubc[1], D);
        k_unknowns2d<<<grd, blk, 0, s>>>(L, 1.0 / c->g.h, mu[0], mu[1], D);
        k_finish2d<<<grd, blk, 0, s>>>(L, D);
    } else {
        dim3 grd((L.nx + 1 + 31) / 32, (L.ny + 1 + 7) / 8, L.nz + 1);
        Ptr3 r3{{rho[0], rho[1], rho[2]}}, u3{{ubc[0], ubc[1], ubc[2]}};
        Ptr4 m4{{mu[0], mu[1], mu[2], mu[3]}};
        k_fractions3d<<<grd, blk, 0, s>>>(L, phiL, phiS, D);
        k_faces3d<<<grd, blk, 0, s>>>(L, c->g.dt, c->min_face_liquid, r3, u3, D);
        k_unknowns3d<<<grd, blk, 0, s>>>(L, 1.0 / c->g.h, m4, D);
        k_finish3d<<<grd, blk, 0, s>>>(L, D);
    }
    k_compact_tiles<<<1, 1024, 0, s>>>(D.tile_flag, c->ntiles_all, c->tiles, c->d_ntiles);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if ((e = cudaMemcpyAsync(&c->ntiles_active, c->d_ntiles, sizeof(int), cudaMemcpyDeviceToHost, s)) != cudaSuccess)
        return e;
    if (L.dim == 3) {
        // units of 4 tile layers (16 planes) when there are enough of them to
        // fill the device a few times over, else of one layer: a thin liquid
        // region has too few deep units to keep every SM busy
        if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return e;
        int dev = 0, sms = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        // (deep units hold 2 ZT_MAX tiles; six CTAs per SM; two waves)
        c->unit_zt = c->ntiles_active >= 2 * (2 * ZT_MAX) * 6 * std::max(sms, 1) ? ZT_MAX : 1;
        const int nu = L.ntx * units_y(L.nty) * units_z(L.ntz, c->unit_zt);
        k_unit_masks<<<(nu + 255) / 256, 256, 0, s>>>(L, c->unit_zt, D.tile_flag, D.unit_mask, nu);
        k_compact_tiles<<<1, 1024, 0, s>>>(D.unit_mask, nu, c->units, c->d_nunits);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        if ((e = cudaMemcpyAsync(&c->nunits_active, c->d_nunits, sizeof(int), cudaMemcpyDeviceToHost, s)) !=
            cudaSuccess)
            return e;
    }
    return cudaStreamSynchronize(s);
}

}  // namespace stk
