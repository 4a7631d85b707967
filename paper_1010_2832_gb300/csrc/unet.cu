// Learned preconditioner network: a three-level U-Net on the slot lattice.
//
// Tensors are channel-last, (B, D, H, W, C); activations are stored in BF16,
// every sum is accumulated in FP32, master weights and gradients are FP32.
// Weight layout per convolution: W[tap][cin][cout] (tap = (dz*KY + dy)*KX + dx
// with dz in 0..KZ-1), then bias[cout].  Layer order and widths:
//   enc0a cin->8, enc0b 8->8, enc1a 8->16, enc1b 16->16, enc2a 16->32,
//   enc2b 32->32, dec1a (32+16)->16, dec1b 16->16, dec0a (16+8)->8,
//   dec0b 8->8, out 8->cout (1x1)
// 3x3(x3) convolutions with zero padding 1 and ReLU; 2x average-pool down,
// nearest-neighbour up, concatenation [upsampled, skip].  In 2D, KZ = 1 and
// D = 1.
//
// Kernels: direct convolution (one output voxel per thread, the input halo
// staged in shared memory as BF16, warp-uniform weight loads), the same
// kernel for the data gradient (with flipped, transposed weights), a weight
// gradient kernel that reduces over a tile in registers then adds to global
// FP32 with atomics, pooling/upsampling and their adjoints, the normalised
// squared-error loss and Adam.
#include <cmath>
#include <cstring>
#include <string>
#include <vector>
#include "internal.cuh"
#include "ctx.cuh"

using stk::warp_sum;

namespace {

struct Shape { int B, D, H, W; };
__host__ __device__ inline int64_t vox(const Shape& s) { return (int64_t)s.B * s.D * s.H * s.W; }

constexpr int CT_X = 8, CT_Y = 8, CT_Z3 = 4;     // 3D tile 8x8x4 = 256 voxels
constexpr int CT2_X = 16, CT2_Y = 16;           // 2D tile 16x16

__device__ __forceinline__ float to_f(__nv_bfloat16 v) { return __bfloat162float(v); }
__device__ __forceinline__ float to_f(float v) { return v; }
template <class T> __device__ __forceinline__ T zero_of();
template <> __device__ __forceinline__ __nv_bfloat16 zero_of<__nv_bfloat16>() { return __float2bfloat16(0.f); }
template <> __device__ __forceinline__ float zero_of<float>() { return 0.f; }

// ---- convolution (forward on BF16 activations; data gradient on FP32 ------
// gradients with prepared weights)
template <class TIN, int KZ, int COUT>
__global__ void __launch_bounds__(256) k_conv(const TIN* __restrict__ X, Shape s, int cin,
                                              const float* __restrict__ Wt, const float* __restrict__ bias,
                                              int relu, __nv_bfloat16* __restrict__ Yb, float* __restrict__ Yf,
                                              int ksize) {
    extern __shared__ __align__(16) unsigned char smraw[];
    TIN* sx = reinterpret_cast<TIN*>(smraw);
    const int TXc = KZ == 3 ? CT_X : CT2_X, TYc = KZ == 3 ? CT_Y : CT2_Y, TZc = KZ == 3 ? CT_Z3 : 1;
    const int R = ksize / 2;                 // halo radius (1 for 3x3, 0 for 1x1)
    const int kz = KZ == 3 ? ksize : 1;
    const int HX = TXc + 2 * R, HY = TYc + 2 * R, HZ = TZc + (KZ == 3 ? 2 * R : 0);
    const int ntx = (s.W + TXc - 1) / TXc, nty = (s.H + TYc - 1) / TYc, ntz = (s.D + TZc - 1) / TZc;
    int bid = blockIdx.x;
    const int bx = bid % ntx; bid /= ntx;
    const int by = bid % nty; bid /= nty;
    const int bz = bid % ntz; const int b = bid / ntz;
    const int x0 = bx * TXc, y0 = by * TYc, z0 = bz * TZc;
    const int zr = KZ == 3 ? R : 0;
    // stage the input halo
    const int nh = HX * HY * HZ;
    for (int e = threadIdx.x; e < nh * cin; e += 256) {
        int c = e % cin, v = e / cin;
        int hx = v % HX, hy = (v / HX) % HY, hz = v / (HX * HY);
        int gx = x0 + hx - R, gy = y0 + hy - R, gz = z0 + hz - zr;
        TIN val = zero_of<TIN>();
        if (gx >= 0 && gx < s.W && gy >= 0 && gy < s.H && gz >= 0 && gz < s.D)
            val = X[((((int64_t)b * s.D + gz) * s.H + gy) * s.W + gx) * cin + c];
        sx[v * cin + c] = val;
    }
    __syncthreads();
    const int tx = threadIdx.x % TXc, ty = (threadIdx.x / TXc) % TYc, tz = threadIdx.x / (TXc * TYc);
    const int gx = x0 + tx, gy = y0 + ty, gz = z0 + tz;
    if (gx >= s.W || gy >= s.H || gz >= s.D) return;
    float acc[COUT];
#pragma unroll
    for (int c = 0; c < COUT; ++c) acc[c] = bias ? bias[c] : 0.f;
    int tap = 0;
    for (int dz = 0; dz < kz; ++dz)
        for (int dy = 0; dy < ksize; ++dy)
            for (int dx = 0; dx < ksize; ++dx, ++tap) {
                const TIN* xin = sx + (((tz + dz) * HY + (ty + dy)) * HX + (tx + dx)) * cin;
                const float* w = Wt + (int64_t)tap * cin * COUT;
                for (int ci = 0; ci < cin; ++ci) {
                    float v = to_f(xin[ci]);
                    const float4* w4 = reinterpret_cast<const float4*>(w + ci * COUT);
#pragma unroll
                    for (int q = 0; q < COUT / 4; ++q) {
                        float4 ww = __ldg(w4 + q);
                        acc[4 * q] = fmaf(v, ww.x, acc[4 * q]);
                        acc[4 * q + 1] = fmaf(v, ww.y, acc[4 * q + 1]);
                        acc[4 * q + 2] = fmaf(v, ww.z, acc[4 * q + 2]);
                        acc[4 * q + 3] = fmaf(v, ww.w, acc[4 * q + 3]);
                    }
                }
            }
    int64_t o = ((((int64_t)b * s.D + gz) * s.H + gy) * s.W + gx) * COUT;
#pragma unroll
    for (int c = 0; c < COUT; ++c) {
        float v = relu ? fmaxf(acc[c], 0.f) : acc[c];
        if (Yb) Yb[o + c] = __float2bfloat16(v);
        if (Yf) Yf[o + c] = v;
    }
}

// ---- weight gradient: dW[tap][ci][co] += sum_v X[v + tap][ci] dY[v][co] -----
template <int KZ>
__global__ void __launch_bounds__(256) k_conv_wgrad(const __nv_bfloat16* __restrict__ X, Shape s, int cin,
                                                    const float* __restrict__ dY, int cout, int ksize,
                                                    float* __restrict__ dW, float* __restrict__ db) {
    extern __shared__ __align__(16) unsigned char smraw[];
    const int TXc = KZ == 3 ? CT_X : CT2_X, TYc = KZ == 3 ? CT_Y : CT2_Y, TZc = KZ == 3 ? CT_Z3 : 1;
    const int R = ksize / 2, kz = KZ == 3 ? ksize : 1, zr = KZ == 3 ? R : 0;
    const int HX = TXc + 2 * R, HY = TYc + 2 * R, HZ = TZc + 2 * zr;
    float* sdy = reinterpret_cast<float*>(smraw);                               // 256 x cout
    __nv_bfloat16* sx = reinterpret_cast<__nv_bfloat16*>(sdy + 256 * cout);     // halo x cin
    const int ntx = (s.W + TXc - 1) / TXc, nty = (s.H + TYc - 1) / TYc, ntz = (s.D + TZc - 1) / TZc;
    int bid = blockIdx.x;
    const int bx = bid % ntx; bid /= ntx;
    const int by = bid % nty; bid /= nty;
    const int bz = bid % ntz; const int b = bid / ntz;
    const int x0 = bx * TXc, y0 = by * TYc, z0 = bz * TZc;
    const int nh = HX * HY * HZ;
    for (int e = threadIdx.x; e < nh * cin; e += 256) {
        int c = e % cin, v = e / cin;
        int hx = v % HX, hy = (v / HX) % HY, hz = v / (HX * HY);
        int gx = x0 + hx - R, gy = y0 + hy - R, gz = z0 + hz - zr;
        __nv_bfloat16 val = __float2bfloat16(0.f);
        if (gx >= 0 && gx < s.W && gy >= 0 && gy < s.H && gz >= 0 && gz < s.D)
            val = X[((((int64_t)b * s.D + gz) * s.H + gy) * s.W + gx) * cin + c];
        sx[v * cin + c] = val;
    }
    for (int e = threadIdx.x; e < 256 * cout; e += 256) {
        int c = e % cout, v = e / cout;
        int tx = v % TXc, ty = (v / TXc) % TYc, tz = v / (TXc * TYc);
        int gx = x0 + tx, gy = y0 + ty, gz = z0 + tz;
        float val = 0.f;
        if (gx < s.W && gy < s.H && gz < s.D) val = dY[((((int64_t)b * s.D + gz) * s.H + gy) * s.W + gx) * cout + c];
        sdy[e] = val;
    }
    __syncthreads();
    const int taps = kz * ksize * ksize;
    const int E = taps * cin * cout;
    for (int e = threadIdx.x; e < E; e += 256) {
        int co = e % cout, ci = (e / cout) % cin, tap = e / (cout * cin);
        int dx = tap % ksize, dy = (tap / ksize) % ksize, dz = tap / (ksize * ksize);
        float sum = 0.f;
        for (int v = 0; v < 256; ++v) {
            int tx = v % TXc, ty = (v / TXc) % TYc, tz = v / (TXc * TYc);
            float xv = __bfloat162float(sx[(((tz + dz) * HY + (ty + dy)) * HX + (tx + dx)) * cin + ci]);
            sum = fmaf(xv, sdy[v * cout + co], sum);
        }
        atomicAdd(dW + e, sum);
    }
    if (threadIdx.x < cout) {
        float sum = 0.f;
        for (int v = 0; v < 256; ++v) sum += sdy[v * cout + threadIdx.x];
        atomicAdd(db + threadIdx.x, sum);
    }
}

// Data-gradient weights: W'[tap'][co][ci] = W[flip(tap')][ci][co]
__global__ void k_flip_weights(const float* W, int taps, int cin, int cout, float* Wb) {
    int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= taps * cin * cout) return;
    int ci = e % cin, co = (e / cin) % cout, tp = e / (cin * cout);
    Wb[e] = W[((int64_t)(taps - 1 - tp) * cin + ci) * cout + co];
}

// 2x average pooling (and its adjoint: nearest up-spread divided by 2^d)
__global__ void k_pool(const __nv_bfloat16* X, Shape s, int c, int pz, __nv_bfloat16* Y) {
    Shape o{s.B, pz ? s.D / 2 : s.D, s.H / 2, s.W / 2};
    int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= vox(o) * c) return;
    int ch = e % c;
    int64_t v = e / c;
    int x = v % o.W, y = (v / o.W) % o.H, z = (v / ((int64_t)o.W * o.H)) % o.D, b = v / ((int64_t)o.W * o.H * o.D);
    float sum = 0.f;
    int nz = pz ? 2 : 1;
    for (int dz = 0; dz < nz; ++dz)
        for (int dy = 0; dy < 2; ++dy)
            for (int dx = 0; dx < 2; ++dx) {
                int zz = pz ? 2 * z + dz : z;
                sum += __bfloat162float(X[((((int64_t)b * s.D + zz) * s.H + 2 * y + dy) * s.W + 2 * x + dx) * c + ch]);
            }
    Y[e] = __float2bfloat16(sum / (nz * 4));
}

__global__ void k_pool_adj(const float* dY, Shape s, int c, int pz, float* dX) {  // s: fine shape
    int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= vox(s) * c) return;
    int ch = e % c;
    int64_t v = e / c;
    int x = v % s.W, y = (v / s.W) % s.H, z = (v / ((int64_t)s.W * s.H)) % s.D, b = v / ((int64_t)s.W * s.H * s.D);
    Shape o{s.B, pz ? s.D / 2 : s.D, s.H / 2, s.W / 2};
    int zc = pz ? z / 2 : z;
    dX[e] += dY[((((int64_t)b * o.D + zc) * o.H + y / 2) * o.W + x / 2) * c + ch] / ((pz ? 2 : 1) * 4);
}

// nearest 2x upsampling of X (coarse) into channels [0, c) of Y (fine, cy channels)
__global__ void k_up_concat(const __nv_bfloat16* Xc, const __nv_bfloat16* skip, Shape s, int c, int cs, int pz,
                            __nv_bfloat16* Y) {
    int cy = c + cs;
    int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= vox(s) * cy) return;
    int ch = e % cy;
    int64_t v = e / cy;
    if (ch < c) {
        int x = v % s.W, y = (v / s.W) % s.H, z = (v / ((int64_t)s.W * s.H)) % s.D, b = v / ((int64_t)s.W * s.H * s.D);
        Shape o{s.B, pz ? s.D / 2 : s.D, s.H / 2, s.W / 2};
        int zc = pz ? z / 2 : z;
        Y[e] = Xc[((((int64_t)b * o.D + zc) * o.H + y / 2) * o.W + x / 2) * c + ch];
    } else {
        Y[e] = skip[v * cs + (ch - c)];
    }
}

// adjoint of k_up_concat: coarse gradient (sum over the 2^d children) and
// skip gradient (added)
__global__ void k_up_concat_adj(const float* dY, Shape s, int c, int cs, int pz, float* dXc, float* dskip) {
    int cy = c + cs;
    Shape o{s.B, pz ? s.D / 2 : s.D, s.H / 2, s.W / 2};
    int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int64_t nco = vox(o) * c, nsk = vox(s) * cs;
    if (e < nco) {
        int ch = e % c;
        int64_t v = e / c;
        int x = v % o.W, y = (v / o.W) % o.H, z = (v / ((int64_t)o.W * o.H)) % o.D, b = v / ((int64_t)o.W * o.H * o.D);
        float sum = 0.f;
        int nz = pz ? 2 : 1;
        for (int dz = 0; dz < nz; ++dz)
            for (int dy = 0; dy < 2; ++dy)
                for (int dx = 0; dx < 2; ++dx) {
                    int zz = pz ? 2 * z + dz : z;
                    sum += dY[((((int64_t)b * s.D + zz) * s.H + 2 * y + dy) * s.W + 2 * x + dx) * cy + ch];
                }
        dXc[e] = sum;
    }
    if (e < nsk) {
        int ch = e % cs;
        int64_t v = e / cs;
        dskip[e] += dY[v * cy + c + ch];
    }
}

// gradient through ReLU: g *= (y > 0); g may be FP32 accumulated from several paths
__global__ void k_relu_bwd(float* g, const __nv_bfloat16* y, int64_t n) {
    int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e < n && !(__bfloat162float(y[e]) > 0.f)) g[e] = 0.f;
}

__global__ void k_to_bf16(const float* x, __nv_bfloat16* y, int64_t n) {
    int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e < n) y[e] = __float2bfloat16(x[e]);
}

// loss = mean_b ||out_b - y_b||^2 / ||y_b||^2; g = d loss / d out
__global__ void k_loss_sums(const float* out, const float* y, int64_t per, double* sums) {
    int b = blockIdx.y;
    double num = 0.0, den = 0.0;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < per; e += (int64_t)gridDim.x * blockDim.x) {
        float d = out[b * per + e] - y[b * per + e];
        num += (double)d * d;
        den += (double)y[b * per + e] * y[b * per + e];
    }
    num = warp_sum(num);
    den = warp_sum(den);
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(sums + 2 * b, num);
        atomicAdd(sums + 2 * b + 1, den);
    }
}

__global__ void k_loss_grad(const float* out, const float* y, int64_t per, int B, const double* sums, float* g) {
    int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= per * B) return;
    int b = e / per;
    double den = fmax(sums[2 * b + 1], 1e-300);
    g[e] = (float)(2.0 * (out[e] - y[e]) / den / B);
}

__global__ void k_adam(float* th, const float* g, float* m, float* v, int64_t n, float lr, float b1, float b2,
                       float eps, float c1, float c2) {
    int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n) return;
    float gg = g[e];
    float mm = b1 * m[e] + (1.f - b1) * gg;
    float vv = b2 * v[e] + (1.f - b2) * gg * gg;
    m[e] = mm; v[e] = vv;
    th[e] -= lr * (mm / c1) / (sqrtf(vv / c2) + eps);
}

inline unsigned nblk(int64_t n) { return (unsigned)((n + 255) / 256); }

}  // namespace

// ---------------------------------------------------------------------------
struct Conv {
    int cin, cout, ks;
    int64_t w_off, b_off, nw;
};

struct stokes_net_s {
    int dim = 3, cin = 0, cout = 0;
    int KZ = 3;
    int64_t max_vox = 0;
    std::vector<Conv> L;
    int64_t np = 0;
    float *theta = nullptr, *grad = nullptr, *m = nullptr, *v = nullptr, *wflip = nullptr;
    int adam_t = 0;
    // activations (BF16) and gradients (FP32)
    __nv_bfloat16 *xin = nullptr, *e0a = nullptr, *e0 = nullptr, *p0 = nullptr, *e1a = nullptr, *e1 = nullptr,
                  *p1 = nullptr, *e2a = nullptr, *e2 = nullptr, *c1 = nullptr, *d1a = nullptr, *d1 = nullptr,
                  *c0 = nullptr, *d0a = nullptr, *d0 = nullptr;
    float* out = nullptr;
    float *g_a = nullptr, *g_b = nullptr, *g_skip0 = nullptr, *g_skip1 = nullptr, *g_c = nullptr;
    double* sums = nullptr;
    std::vector<void*> allocs;
    cudaStream_t s = nullptr;
    std::string err;
};

namespace {

int conv_cout_template_ok(int c) { return c == 4 || c == 8 || c == 12 || c == 16 || c == 24 || c == 32 || c == 48; }

template <int KZ, class TIN>
cudaError_t conv_launch(stokes_net_s* n, const TIN* X, Shape s, int cin, const float* W, const float* b,
                        int relu, __nv_bfloat16* Yb, float* Yf, int cout, int ks) {
    const int TXc = KZ == 3 ? CT_X : CT2_X, TYc = KZ == 3 ? CT_Y : CT2_Y, TZc = KZ == 3 ? CT_Z3 : 1;
    const int R = ks / 2;
    size_t smem = (size_t)(TXc + 2 * R) * (TYc + 2 * R) * (TZc + (KZ == 3 ? 2 * R : 0)) * cin * sizeof(TIN);
    unsigned grid = (unsigned)((int64_t)s.B * ((s.D + TZc - 1) / TZc) * ((s.H + TYc - 1) / TYc) * ((s.W + TXc - 1) / TXc));
#define CASE(C)                                                                                             \
    case C:                                                                                                 \
        cudaFuncSetAttribute(k_conv<TIN, KZ, C>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);   \
        k_conv<TIN, KZ, C><<<grid, 256, smem, n->s>>>(X, s, cin, W, b, relu, Yb, Yf, ks);                   \
        break;
    switch (cout) {
        CASE(4) CASE(8) CASE(12) CASE(16) CASE(24) CASE(32) CASE(48)
        default: return cudaErrorInvalidValue;
    }
#undef CASE
    return cudaGetLastError();
}

template <int KZ>
cudaError_t wgrad_launch(stokes_net_s* n, const __nv_bfloat16* X, Shape s, int cin, const float* dY, int cout, int ks,
                         float* dW, float* db) {
    const int TXc = KZ == 3 ? CT_X : CT2_X, TYc = KZ == 3 ? CT_Y : CT2_Y, TZc = KZ == 3 ? CT_Z3 : 1;
    const int R = ks / 2;
    size_t smem = 256 * cout * 4 + (size_t)(TXc + 2 * R) * (TYc + 2 * R) * (TZc + (KZ == 3 ? 2 * R : 0)) * cin * 2;
    unsigned grid = (unsigned)((int64_t)s.B * ((s.D + TZc - 1) / TZc) * ((s.H + TYc - 1) / TYc) * ((s.W + TXc - 1) / TXc));
    cudaFuncSetAttribute(k_conv_wgrad<KZ>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_conv_wgrad<KZ><<<grid, 256, smem, n->s>>>(X, s, cin, dY, cout, ks, dW, db);
    return cudaGetLastError();
}

cudaError_t conv(stokes_net_s* n, int li, const __nv_bfloat16* X, Shape s, int relu, __nv_bfloat16* Yb, float* Yf) {
    const Conv& c = n->L[li];
    if (n->KZ == 3)
        return conv_launch<3, __nv_bfloat16>(n, X, s, c.cin, n->theta + c.w_off, n->theta + c.b_off, relu, Yb, Yf,
                                             c.cout, c.ks);
    return conv_launch<1, __nv_bfloat16>(n, X, s, c.cin, n->theta + c.w_off, n->theta + c.b_off, relu, Yb, Yf,
                                         c.cout, c.ks);
}

// data gradient of layer li: dX = conv(dY, flipped W) (no bias, no ReLU)
cudaError_t conv_dgrad(stokes_net_s* n, int li, const float* dY, Shape s, float* dX) {
    const Conv& c = n->L[li];
    int taps = (n->KZ == 3 ? c.ks : 1) * c.ks * c.ks;
    k_flip_weights<<<nblk(c.nw), 256, 0, n->s>>>(n->theta + c.w_off, taps, c.cin, c.cout, n->wflip);
    // gradients stay FP32 (staged as FP32 in shared memory)
    if (n->KZ == 3) return conv_launch<3, float>(n, dY, s, c.cout, n->wflip, nullptr, 0, nullptr, dX, c.cin, c.ks);
    return conv_launch<1, float>(n, dY, s, c.cout, n->wflip, nullptr, 0, nullptr, dX, c.cin, c.ks);
}

cudaError_t conv_wgrad(stokes_net_s* n, int li, const __nv_bfloat16* X, Shape s, const float* dY) {
    const Conv& c = n->L[li];
    if (n->KZ == 3) return wgrad_launch<3>(n, X, s, c.cin, dY, c.cout, c.ks, n->grad + c.w_off, n->grad + c.b_off);
    return wgrad_launch<1>(n, X, s, c.cin, dY, c.cout, c.ks, n->grad + c.w_off, n->grad + c.b_off);
}

Shape half(const Shape& s, int pz) { return Shape{s.B, pz ? s.D / 2 : s.D, s.H / 2, s.W / 2}; }

cudaError_t forward(stokes_net_s* n, Shape s) {
    const int pz = n->KZ == 3;
    Shape s1 = half(s, pz), s2 = half(s1, pz);
    cudaError_t e;
    if ((e = conv(n, 0, n->xin, s, 1, n->e0a, nullptr))) return e;
    if ((e = conv(n, 1, n->e0a, s, 1, n->e0, nullptr))) return e;
    k_pool<<<nblk(vox(s1) * 8), 256, 0, n->s>>>(n->e0, s, 8, pz, n->p0);
    if ((e = conv(n, 2, n->p0, s1, 1, n->e1a, nullptr))) return e;
    if ((e = conv(n, 3, n->e1a, s1, 1, n->e1, nullptr))) return e;
    k_pool<<<nblk(vox(s2) * 16), 256, 0, n->s>>>(n->e1, s1, 16, pz, n->p1);
    if ((e = conv(n, 4, n->p1, s2, 1, n->e2a, nullptr))) return e;
    if ((e = conv(n, 5, n->e2a, s2, 1, n->e2, nullptr))) return e;
    k_up_concat<<<nblk(vox(s1) * 48), 256, 0, n->s>>>(n->e2, n->e1, s1, 32, 16, pz, n->c1);
    if ((e = conv(n, 6, n->c1, s1, 1, n->d1a, nullptr))) return e;
    if ((e = conv(n, 7, n->d1a, s1, 1, n->d1, nullptr))) return e;
    k_up_concat<<<nblk(vox(s) * 24), 256, 0, n->s>>>(n->d1, n->e0, s, 16, 8, pz, n->c0);
    if ((e = conv(n, 8, n->c0, s, 1, n->d0a, nullptr))) return e;
    if ((e = conv(n, 9, n->d0a, s, 1, n->d0, nullptr))) return e;
    return conv(n, 10, n->d0, s, 0, nullptr, n->out);
}

// backward from dL/dout (in g_a), accumulating parameter gradients in grad
cudaError_t backward(stokes_net_s* n, Shape s) {
    const int pz = n->KZ == 3;
    Shape s1 = half(s, pz), s2 = half(s1, pz);
    cudaError_t e;
    float *ga = n->g_a, *gb = n->g_b;
    auto relu_b = [&](float* g, const __nv_bfloat16* y, int64_t nel) { k_relu_bwd<<<nblk(nel), 256, 0, n->s>>>(g, y, nel); };
    // out (1x1, no ReLU): input d0
    if ((e = conv_wgrad(n, 10, n->d0, s, ga))) return e;
    if ((e = conv_dgrad(n, 10, ga, s, gb))) return e;                  // gb = d d0
    relu_b(gb, n->d0, vox(s) * 8);
    if ((e = conv_wgrad(n, 9, n->d0a, s, gb))) return e;
    if ((e = conv_dgrad(n, 9, gb, s, ga))) return e;                   // ga = d d0a
    relu_b(ga, n->d0a, vox(s) * 8);
    if ((e = conv_wgrad(n, 8, n->c0, s, ga))) return e;
    if ((e = conv_dgrad(n, 8, ga, s, gb))) return e;                   // gb = d c0 (24 ch)
    cudaMemsetAsync(n->g_skip0, 0, sizeof(float) * vox(s) * 8, n->s);
    k_up_concat_adj<<<nblk(std::max(vox(s1) * 16, vox(s) * 8)), 256, 0, n->s>>>(gb, s, 16, 8, pz, ga, n->g_skip0);
    // ga = d d1 (16 ch at s1)
    relu_b(ga, n->d1, vox(s1) * 16);
    if ((e = conv_wgrad(n, 7, n->d1a, s1, ga))) return e;
    if ((e = conv_dgrad(n, 7, ga, s1, gb))) return e;                  // gb = d d1a
    relu_b(gb, n->d1a, vox(s1) * 16);
    if ((e = conv_wgrad(n, 6, n->c1, s1, gb))) return e;
    if ((e = conv_dgrad(n, 6, gb, s1, ga))) return e;                  // ga = d c1 (48 ch at s1)
    cudaMemsetAsync(n->g_skip1, 0, sizeof(float) * vox(s1) * 16, n->s);
    k_up_concat_adj<<<nblk(std::max(vox(s2) * 32, vox(s1) * 16)), 256, 0, n->s>>>(ga, s1, 32, 16, pz, gb, n->g_skip1);
    // gb = d e2 (32 ch at s2)
    relu_b(gb, n->e2, vox(s2) * 32);
    if ((e = conv_wgrad(n, 5, n->e2a, s2, gb))) return e;
    if ((e = conv_dgrad(n, 5, gb, s2, ga))) return e;                  // ga = d e2a
    relu_b(ga, n->e2a, vox(s2) * 32);
    if ((e = conv_wgrad(n, 4, n->p1, s2, ga))) return e;
    if ((e = conv_dgrad(n, 4, ga, s2, gb))) return e;                  // gb = d p1 (16 ch at s2)
    k_pool_adj<<<nblk(vox(s1) * 16), 256, 0, n->s>>>(gb, s1, 16, pz, n->g_skip1);   // += into d e1
    relu_b(n->g_skip1, n->e1, vox(s1) * 16);
    if ((e = conv_wgrad(n, 3, n->e1a, s1, n->g_skip1))) return e;
    if ((e = conv_dgrad(n, 3, n->g_skip1, s1, ga))) return e;          // ga = d e1a
    relu_b(ga, n->e1a, vox(s1) * 16);
    if ((e = conv_wgrad(n, 2, n->p0, s1, ga))) return e;
    if ((e = conv_dgrad(n, 2, ga, s1, gb))) return e;                  // gb = d p0 (8 ch at s1)
    k_pool_adj<<<nblk(vox(s) * 8), 256, 0, n->s>>>(gb, s, 8, pz, n->g_skip0);      // += into d e0
    relu_b(n->g_skip0, n->e0, vox(s) * 8);
    if ((e = conv_wgrad(n, 1, n->e0a, s, n->g_skip0))) return e;
    if ((e = conv_dgrad(n, 1, n->g_skip0, s, ga))) return e;           // ga = d e0a
    relu_b(ga, n->e0a, vox(s) * 8);
    return conv_wgrad(n, 0, n->xin, s, ga);
}

}  // namespace

extern "C" {

stokes_status stokes_net_destroy(stokes_net n) {
    if (!n) return STOKES_OK;
    for (void* p : n->allocs) cudaFree(p);
    if (n->s) cudaStreamDestroy(n->s);
    delete n;
    return STOKES_OK;
}

stokes_status stokes_net_create(stokes_net* out, int dim, int cin, int cout, int64_t max_voxels) {
    if (!out || (dim != 2 && dim != 3) || cin < 1 || cin > 48 || !conv_cout_template_ok(cin) ||
        !conv_cout_template_ok(cout) || max_voxels < 1)
        return STOKES_ERR_ARG;
    auto* n = new stokes_net_s();
    n->dim = dim; n->cin = cin; n->cout = cout; n->KZ = dim == 3 ? 3 : 1;
    n->max_vox = max_voxels;
    int sizes[11][3] = {{cin, 8, 3}, {8, 8, 3}, {8, 16, 3}, {16, 16, 3}, {16, 32, 3}, {32, 32, 3},
                        {48, 16, 3}, {16, 16, 3}, {24, 8, 3}, {8, 8, 3}, {8, cout, 1}};
    int64_t off = 0;
    for (auto& q : sizes) {
        Conv c;
        c.cin = q[0]; c.cout = q[1]; c.ks = q[2];
        int taps = (dim == 3 && c.ks == 3 ? 3 : 1) * c.ks * c.ks;
        c.nw = (int64_t)taps * c.cin * c.cout;
        c.w_off = off; off += c.nw;
        c.b_off = off; off += c.cout;
        off = (off + 3) & ~3LL;       // float4-aligned weight blocks
        n->L.push_back(c);
    }
    n->np = off;
    cudaError_t e = cudaStreamCreate(&n->s);
    auto A = [&](void** p, size_t bytes) {
        if (e != cudaSuccess) return;
        e = cudaMalloc(p, bytes);
        if (e == cudaSuccess) { n->allocs.push_back(*p); e = cudaMemset(*p, 0, bytes); }
    };
    int64_t V = max_voxels;
    A((void**)&n->theta, 4 * off); A((void**)&n->grad, 4 * off); A((void**)&n->m, 4 * off); A((void**)&n->v, 4 * off);
    A((void**)&n->wflip, 4 * 27 * 48 * 48);
    A((void**)&n->xin, 2 * V * cin);
    __nv_bfloat16** full8[] = {&n->e0a, &n->e0, &n->d0a, &n->d0};
    for (auto p : full8) A((void**)p, 2 * V * 8);
    A((void**)&n->c0, 2 * V * 24);
    __nv_bfloat16** half16[] = {&n->p0, &n->e1a, &n->e1, &n->d1a, &n->d1};
    for (auto p : half16) A((void**)p, 2 * V * 16);          // generous (V/4 or V/8 needed)
    A((void**)&n->c1, 2 * V * 48 / 2);
    A((void**)&n->p1, 2 * V * 16); A((void**)&n->e2a, 2 * V * 32 / 4); A((void**)&n->e2, 2 * V * 32 / 4);
    A((void**)&n->out, 4 * V * cout);
    A((void**)&n->g_a, 4 * V * 48); A((void**)&n->g_b, 4 * V * 48); A((void**)&n->g_c, 4 * V * 48);
    A((void**)&n->g_skip0, 4 * V * 8); A((void**)&n->g_skip1, 4 * V * 16);
    A((void**)&n->sums, 16 * 1024);
    if (e != cudaSuccess) { stokes_net_destroy(n); return STOKES_ERR_CUDA; }
    *out = n;
    return STOKES_OK;
}

int64_t stokes_net_param_count(stokes_net n) { return n ? n->np : -1; }

stokes_status stokes_net_set_params(stokes_net n, const float* host) {
    if (!n || !host) return STOKES_ERR_ARG;
    if (cudaMemcpy(n->theta, host, 4 * n->np, cudaMemcpyHostToDevice) != cudaSuccess) return STOKES_ERR_CUDA;
    cudaMemset(n->m, 0, 4 * n->np);
    cudaMemset(n->v, 0, 4 * n->np);
    n->adam_t = 0;
    return STOKES_OK;
}

stokes_status stokes_net_get_params(stokes_net n, float* host) {
    if (!n || !host) return STOKES_ERR_ARG;
    return cudaMemcpy(host, n->theta, 4 * n->np, cudaMemcpyDeviceToHost) == cudaSuccess ? STOKES_OK : STOKES_ERR_CUDA;
}

static bool shape_ok(stokes_net n, int B, int D, int H, int W) {
    int m = n->dim == 3 ? 4 : 1;
    return B >= 1 && D >= 1 && H >= 4 && W >= 4 && H % 4 == 0 && W % 4 == 0 && D % m == 0 &&
           (n->dim == 3 || D == 1) && (int64_t)B * D * H * W <= n->max_vox;
}

// x: FP32 device (B, D, H, W, cin) channel-last; y: FP32 device (.., cout)
stokes_status stokes_net_forward(stokes_net n, int B, int D, int H, int W, const float* x, float* y) {
    if (!n || !x || !y || !shape_ok(n, B, D, H, W)) return STOKES_ERR_ARG;
    Shape s{B, D, H, W};
    k_to_bf16<<<nblk(vox(s) * n->cin), 256, 0, n->s>>>(x, n->xin, vox(s) * n->cin);
    if (forward(n, s) != cudaSuccess) return STOKES_ERR_CUDA;
    if (cudaMemcpyAsync(y, n->out, 4 * vox(s) * n->cout, cudaMemcpyDeviceToDevice, n->s) != cudaSuccess)
        return STOKES_ERR_CUDA;
    return cudaStreamSynchronize(n->s) == cudaSuccess ? STOKES_OK : STOKES_ERR_CUDA;
}

// Loss (mean over samples of ||N(x) - y||^2 / ||y||^2) and its parameter
// gradient (left in the network; copied to grad_host if not NULL).
stokes_status stokes_net_gradient(stokes_net n, int B, int D, int H, int W, const float* x, const float* y,
                                  double* loss, float* grad_host) {
    if (!n || !x || !y || !shape_ok(n, B, D, H, W) || B > 1024) return STOKES_ERR_ARG;
    Shape s{B, D, H, W};
    k_to_bf16<<<nblk(vox(s) * n->cin), 256, 0, n->s>>>(x, n->xin, vox(s) * n->cin);
    if (forward(n, s) != cudaSuccess) return STOKES_ERR_CUDA;
    int64_t per = (int64_t)D * H * W * n->cout;
    cudaMemsetAsync(n->sums, 0, 16 * B, n->s);
    k_loss_sums<<<dim3(64, B), 256, 0, n->s>>>(n->out, y, per, n->sums);
    k_loss_grad<<<nblk(per * B), 256, 0, n->s>>>(n->out, y, per, B, n->sums, n->g_a);
    cudaMemsetAsync(n->grad, 0, 4 * n->np, n->s);
    if (backward(n, s) != cudaSuccess) return STOKES_ERR_CUDA;
    std::vector<double> sums(2 * B);
    cudaMemcpyAsync(sums.data(), n->sums, 16 * B, cudaMemcpyDeviceToHost, n->s);
    if (cudaStreamSynchronize(n->s) != cudaSuccess) return STOKES_ERR_CUDA;
    if (loss) {
        double L = 0;
        for (int b = 0; b < B; ++b) L += sums[2 * b] / std::fmax(sums[2 * b + 1], 1e-300);
        *loss = L / B;
    }
    if (grad_host && cudaMemcpy(grad_host, n->grad, 4 * n->np, cudaMemcpyDeviceToHost) != cudaSuccess)
        return STOKES_ERR_CUDA;
    return STOKES_OK;
}

stokes_status stokes_net_train_step(stokes_net n, int B, int D, int H, int W, const float* x, const float* y, float lr,
                                    double* loss) {
    stokes_status st = stokes_net_gradient(n, B, D, H, W, x, y, loss, nullptr);
    if (st != STOKES_OK) return st;
    n->adam_t += 1;
    const float b1 = 0.9f, b2 = 0.999f;
    float c1 = 1.f - std::pow(b1, (float)n->adam_t), c2 = 1.f - std::pow(b2, (float)n->adam_t);
    k_adam<<<nblk(n->np), 256, 0, n->s>>>(n->theta, n->grad, n->m, n->v, n->np, lr, b1, b2, 1e-8f, c1, c2);
    return cudaStreamSynchronize(n->s) == cudaSuccess ? STOKES_OK : STOKES_ERR_CUDA;
}

// Per layer (cin, cout, kernel size, weight offset, bias offset) in the flat
// parameter vector, for host-side conversion between layouts.
stokes_status stokes_net_layer(stokes_net n, int i, int* cin, int* cout, int* ks, int64_t* w_off, int64_t* b_off) {
    if (!n || i < 0 || i >= (int)n->L.size()) return STOKES_ERR_ARG;
    const Conv& c = n->L[i];
    *cin = c.cin; *cout = c.cout; *ks = c.ks; *w_off = c.w_off; *b_off = c.b_off;
    return STOKES_OK;
}

}  // extern "C"
