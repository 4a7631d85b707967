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
// Convolutions run on the tensor cores (unet_tc.cuh: implicit GEMM with
// mma.sync, BF16 operands, FP32 accumulation; activations and output
// gradients are staged channel-last with the channel count padded to a
// multiple of 8).  The data gradient is the forward kernel on the output
// gradient (rounded to BF16) with flipped, transposed weights; the weight
// gradient reduces per-CTA partials in a fixed order (no atomics), so a
// gradient is bit-reproducible.  Pooling/upsampling and their adjoints, the
// normalised squared-error loss and Adam are plain elementwise kernels.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>
#include "internal.cuh"
#include "ctx.cuh"
#include "unet_tc.cuh"

using stk::warp_sum;

namespace {

struct Shape { int B, D, H, W; };
__host__ __device__ inline int64_t vox(const Shape& s) { return (int64_t)s.B * s.D * s.H * s.W; }


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

// loss = mean_b ||out_b - y_b||^2 / ||y_b||^2; g = d loss / d out.  The two
// sums per sample are reduced deterministically: per-block partials (warp
// shuffles, then warps in order), then the blocks in order.
constexpr int LOSS_BLOCKS = 64;
__global__ void k_loss_partials(const float* out, const float* y, int64_t per, double* part) {
    __shared__ double red[2][8];
    const int b = blockIdx.y;
    double num = 0.0, den = 0.0;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < per; e += (int64_t)gridDim.x * blockDim.x) {
        float d = out[b * per + e] - y[b * per + e];
        num += (double)d * d;
        den += (double)y[b * per + e] * y[b * per + e];
    }
    num = warp_sum(num);
    den = warp_sum(den);
    const int w = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0) { red[0][w] = num; red[1][w] = den; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0.0, c = 0.0;
        for (int q = 0; q < (int)(blockDim.x >> 5); ++q) { a += red[0][q]; c += red[1][q]; }
        part[2 * (b * LOSS_BLOCKS + blockIdx.x)] = a;
        part[2 * (b * LOSS_BLOCKS + blockIdx.x) + 1] = c;
    }
}

__global__ void k_loss_finish(const double* part, int B, double* sums) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= B) return;
    double a = 0.0, c = 0.0;
    for (int q = 0; q < LOSS_BLOCKS; ++q) { a += part[2 * (b * LOSS_BLOCKS + q)]; c += part[2 * (b * LOSS_BLOCKS + q) + 1]; }
    sums[2 * b] = a;
    sums[2 * b + 1] = c;
}

__global__ void k_loss_grad(const float* out, const float* y, int64_t per, int B, const double* sums, float* g) {
    int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= per * B) return;
    int b = e / per;
    // a sample whose target is zero contributes nothing (no gradient)
    if (!(sums[2 * b + 1] > 0.0)) { g[e] = 0.f; return; }
    double den = sums[2 * b + 1];
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
    float *theta = nullptr, *grad = nullptr, *m = nullptr, *v = nullptr;
    // packed BF16 weights per layer: forward [cp(cout)][taps cp(cin)], data
    // gradient [cp(cin)][taps cp(cout)]; the forward ones are repacked after
    // every change of the parameters
    std::vector<__nv_bfloat16*> wf, wg;
    bool wf_valid = false;
    __nv_bfloat16* g16 = nullptr;   // output gradient of the layer in BF16 (cp(cout) channels)
    float* part = nullptr;          // weight-gradient partials, part_ctas x part_stride floats
    int part_ctas = 0, sms = 0;
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

using unet_tc::cp8;
// (cin, cout) the network supports: the tensor-core kernels are instantiated
// for input channels padded to 8 or 16 and output channels padded to 8 or 16
bool io_channels_ok(int c) { return c == 4 || c == 8 || c == 12 || c == 16; }
constexpr int PART_STRIDE = 27 * 32 * 32 + 32;     // largest taps x cp(cin) x cp(cout) + cp(cout)

int taps_of(const stokes_net_s* n, const Conv& c) { return (n->KZ == 3 && c.ks == 3 ? 3 : 1) * c.ks * c.ks; }

template <int KZ, int KS, int CP, int COUTP>
cudaError_t launch_conv_tc(stokes_net_s* n, const __nv_bfloat16* X, Shape s, const __nv_bfloat16* Wp,
                           const float* bias, int cout, int relu, __nv_bfloat16* Yb, float* Yf) {
    using C = unet_tc::ConvCfg<KZ, KS, CP, COUTP>;
    auto k = unet_tc::k_conv_tc<KZ, KS, CP, COUTP>;
    cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::SMEM);
    const unet_tc::TShape ts{s.B, s.D, s.H, s.W};
    k<<<C::G::tiles(ts), 256, C::SMEM, n->s>>>(X, ts, Wp, bias, cout, relu, Yb, Yf);
    return cudaGetLastError();
}

// one convolution on the tensor cores: input X with cp channels, packed
// weights Wp with coutp rows
cudaError_t conv_tc(stokes_net_s* n, int ks, int cp, int coutp, const __nv_bfloat16* X, Shape s,
                    const __nv_bfloat16* Wp, const float* bias, int cout, int relu, __nv_bfloat16* Yb, float* Yf) {
#define CONV_CASE(KZ_, KS_, CP_, CO_)                                                                      \
    if (n->KZ == KZ_ && ks == KS_ && cp == CP_ && coutp == CO_)                                            \
        return launch_conv_tc<KZ_, KS_, CP_, CO_>(n, X, s, Wp, bias, cout, relu, Yb, Yf);
#define CONV_CASES(KZ_)                                                                                    \
    CONV_CASE(KZ_, 3, 8, 8) CONV_CASE(KZ_, 3, 16, 8) CONV_CASE(KZ_, 3, 8, 16) CONV_CASE(KZ_, 3, 16, 16)   \
    CONV_CASE(KZ_, 3, 16, 32) CONV_CASE(KZ_, 3, 32, 32) CONV_CASE(KZ_, 3, 48, 16) CONV_CASE(KZ_, 3, 24, 8) \
    CONV_CASE(KZ_, 3, 8, 24) CONV_CASE(KZ_, 3, 16, 48) CONV_CASE(KZ_, 3, 32, 16)                           \
    CONV_CASE(KZ_, 1, 8, 8) CONV_CASE(KZ_, 1, 8, 16) CONV_CASE(KZ_, 1, 16, 8)
    CONV_CASES(3)
    CONV_CASES(1)
#undef CONV_CASES
#undef CONV_CASE
    return cudaErrorInvalidValue;
}

template <int KZ, int KS, int CP, int COUTP>
cudaError_t launch_wgrad_tc(stokes_net_s* n, const __nv_bfloat16* X, Shape s, const __nv_bfloat16* g16, int cin,
                            int cout, float* dW, float* db) {
    using C = unet_tc::WgCfg<KZ, KS, CP, COUTP>;
    static_assert(C::E + COUTP <= PART_STRIDE, "partial buffer too small");
    auto k = unet_tc::k_wgrad_tc<KZ, KS, CP, COUTP>;
    cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::SMEM);
    int per = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k, 256, (int)C::SMEM);
    const unet_tc::TShape ts{s.B, s.D, s.H, s.W};
    const int G = std::min({C::G::tiles(ts), n->sms * std::max(per, 1), n->part_ctas});
    k<<<G, 256, C::SMEM, n->s>>>(X, ts, g16, n->part);
    const int tot = C::E + COUTP;
    unet_tc::k_wgrad_reduce<<<(tot + 255) / 256, 256, 0, n->s>>>(n->part, G, C::G::TAPS, CP, COUTP, cin, cout, dW,
                                                                  db);
    return cudaGetLastError();
}

cudaError_t wgrad_tc(stokes_net_s* n, int ks, int cp, int coutp, const __nv_bfloat16* X, Shape s,
                     const __nv_bfloat16* g16, int cin, int cout, float* dW, float* db) {
#define WG_CASE(KZ_, KS_, CP_, CO_)                                                                        \
    if (n->KZ == KZ_ && ks == KS_ && cp == CP_ && coutp == CO_)                                            \
        return launch_wgrad_tc<KZ_, KS_, CP_, CO_>(n, X, s, g16, cin, cout, dW, db);
#define WG_CASES(KZ_)                                                                                      \
    WG_CASE(KZ_, 3, 8, 8) WG_CASE(KZ_, 3, 16, 8) WG_CASE(KZ_, 3, 8, 16) WG_CASE(KZ_, 3, 16, 16)           \
    WG_CASE(KZ_, 3, 16, 32) WG_CASE(KZ_, 3, 32, 32) WG_CASE(KZ_, 3, 48, 16) WG_CASE(KZ_, 3, 24, 8)         \
    WG_CASE(KZ_, 1, 8, 8) WG_CASE(KZ_, 1, 8, 16)
    WG_CASES(3)
    WG_CASES(1)
#undef WG_CASES
#undef WG_CASE
    return cudaErrorInvalidValue;
}

// pack the forward (and, for training, data-gradient) weights of every layer
cudaError_t pack_weights(stokes_net_s* n, bool grad) {
    for (size_t li = 0; li < n->L.size(); ++li) {
        const Conv& c = n->L[li];
        const int taps = taps_of(n, c);
        if (!n->wf_valid) {
            const int rows = cp8(c.cout), tot = rows * taps * cp8(c.cin);
            unet_tc::k_pack_weights<<<nblk(tot), 256, 0, n->s>>>(n->theta + c.w_off, taps, c.cin, c.cout, rows,
                                                                  cp8(c.cin), 0, n->wf[li]);
        }
        if (grad) {
            const int rows = cp8(c.cin), tot = rows * taps * cp8(c.cout);
            unet_tc::k_pack_weights<<<nblk(tot), 256, 0, n->s>>>(n->theta + c.w_off, taps, c.cin, c.cout, rows,
                                                                  cp8(c.cout), 1, n->wg[li]);
        }
    }
    n->wf_valid = true;
    return cudaGetLastError();
}

cudaError_t conv(stokes_net_s* n, int li, const __nv_bfloat16* X, Shape s, int relu, __nv_bfloat16* Yb, float* Yf) {
    const Conv& c = n->L[li];
    return conv_tc(n, c.ks, cp8(c.cin), cp8(c.cout), X, s, n->wf[li], n->theta + c.b_off, c.cout, relu, Yb, Yf);
}

// gradient step of layer li: dY (FP32, cout channels; the ReLU mask already
// applied) -> BF16; weight and bias gradient from the layer input X; data
// gradient into dX (FP32, cin channels) unless dX is null
cudaError_t conv_backward(stokes_net_s* n, int li, const __nv_bfloat16* X, Shape s, const float* dY, float* dX) {
    const Conv& c = n->L[li];
    unet_tc::k_to_bf16_pad<<<nblk(vox(s) * cp8(c.cout)), 256, 0, n->s>>>(dY, vox(s), c.cout, cp8(c.cout), n->g16);
    cudaError_t e = wgrad_tc(n, c.ks, cp8(c.cin), cp8(c.cout), X, s, n->g16, c.cin, c.cout, n->grad + c.w_off,
                             n->grad + c.b_off);
    if (e != cudaSuccess || !dX) return e;
    return conv_tc(n, c.ks, cp8(c.cout), cp8(c.cin), n->g16, s, n->wg[li], nullptr, c.cin, 0, nullptr, dX);
}

Shape half(const Shape& s, int pz) { return Shape{s.B, pz ? s.D / 2 : s.D, s.H / 2, s.W / 2}; }

cudaError_t forward(stokes_net_s* n, Shape s) {
    const int pz = n->KZ == 3;
    if (!n->wf_valid && pack_weights(n, false) != cudaSuccess) return cudaGetLastError();
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
    if (pack_weights(n, true) != cudaSuccess) return cudaGetLastError();
    Shape s1 = half(s, pz), s2 = half(s1, pz);
    cudaError_t e;
    float *ga = n->g_a, *gb = n->g_b;
    auto relu_b = [&](float* g, const __nv_bfloat16* y, int64_t nel) { k_relu_bwd<<<nblk(nel), 256, 0, n->s>>>(g, y, nel); };
    // out (1x1, no ReLU): input d0
    if ((e = conv_backward(n, 10, n->d0, s, ga, gb))) return e;                  // gb = d d0
    relu_b(gb, n->d0, vox(s) * 8);
    if ((e = conv_backward(n, 9, n->d0a, s, gb, ga))) return e;                   // ga = d d0a
    relu_b(ga, n->d0a, vox(s) * 8);
    if ((e = conv_backward(n, 8, n->c0, s, ga, gb))) return e;                   // gb = d c0 (24 ch)
    cudaMemsetAsync(n->g_skip0, 0, sizeof(float) * vox(s) * 8, n->s);
    k_up_concat_adj<<<nblk(std::max(vox(s1) * 16, vox(s) * 8)), 256, 0, n->s>>>(gb, s, 16, 8, pz, ga, n->g_skip0);
    // ga = d d1 (16 ch at s1)
    relu_b(ga, n->d1, vox(s1) * 16);
    if ((e = conv_backward(n, 7, n->d1a, s1, ga, gb))) return e;                  // gb = d d1a
    relu_b(gb, n->d1a, vox(s1) * 16);
    if ((e = conv_backward(n, 6, n->c1, s1, gb, ga))) return e;                  // ga = d c1 (48 ch at s1)
    cudaMemsetAsync(n->g_skip1, 0, sizeof(float) * vox(s1) * 16, n->s);
    k_up_concat_adj<<<nblk(std::max(vox(s2) * 32, vox(s1) * 16)), 256, 0, n->s>>>(ga, s1, 32, 16, pz, gb, n->g_skip1);
    // gb = d e2 (32 ch at s2)
    relu_b(gb, n->e2, vox(s2) * 32);
    if ((e = conv_backward(n, 5, n->e2a, s2, gb, ga))) return e;                  // ga = d e2a
    relu_b(ga, n->e2a, vox(s2) * 32);
    if ((e = conv_backward(n, 4, n->p1, s2, ga, gb))) return e;                  // gb = d p1 (16 ch at s2)
    k_pool_adj<<<nblk(vox(s1) * 16), 256, 0, n->s>>>(gb, s1, 16, pz, n->g_skip1);   // += into d e1
    relu_b(n->g_skip1, n->e1, vox(s1) * 16);
    if ((e = conv_backward(n, 3, n->e1a, s1, n->g_skip1, ga))) return e;          // ga = d e1a
    relu_b(ga, n->e1a, vox(s1) * 16);
    if ((e = conv_backward(n, 2, n->p0, s1, ga, gb))) return e;                  // gb = d p0 (8 ch at s1)
    k_pool_adj<<<nblk(vox(s) * 8), 256, 0, n->s>>>(gb, s, 8, pz, n->g_skip0);      // += into d e0
    relu_b(n->g_skip0, n->e0, vox(s) * 8);
    if ((e = conv_backward(n, 1, n->e0a, s, n->g_skip0, ga))) return e;           // ga = d e0a
    relu_b(ga, n->e0a, vox(s) * 8);
    return conv_backward(n, 0, n->xin, s, ga, nullptr);
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
    if (!out || (dim != 2 && dim != 3) || !io_channels_ok(cin) || !io_channels_ok(cout) || max_voxels < 1)
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
    for (const Conv& c : n->L) {
        const int64_t taps = (dim == 3 && c.ks == 3 ? 3 : 1) * c.ks * c.ks;
        n->wf.push_back(nullptr);
        n->wg.push_back(nullptr);
        A((void**)&n->wf.back(), 2 * taps * cp8(c.cin) * cp8(c.cout));
        A((void**)&n->wg.back(), 2 * taps * cp8(c.cin) * cp8(c.cout));
    }
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n->sms, cudaDevAttrMultiProcessorCount, dev);
    n->part_ctas = 2 * std::max(n->sms, 1);
    A((void**)&n->part, 4 * (size_t)n->part_ctas * PART_STRIDE);
    A((void**)&n->g16, 2 * V * 8);
    A((void**)&n->xin, 2 * V * cp8(cin));
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
    A((void**)&n->sums, 16 * 1024 + 16 * 1024 * LOSS_BLOCKS);   // sums, then the per-block partials
    if (e != cudaSuccess) { stokes_net_destroy(n); return STOKES_ERR_CUDA; }
    *out = n;
    return STOKES_OK;
}

int64_t stokes_net_param_count(stokes_net n) { return n ? n->np : -1; }

stokes_status stokes_net_set_params(stokes_net n, const float* host) {
    if (!n || !host) return STOKES_ERR_ARG;
    if (cudaMemcpy(n->theta, host, 4 * n->np, cudaMemcpyHostToDevice) != cudaSuccess) return STOKES_ERR_CUDA;
    n->wf_valid = false;
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
    unet_tc::k_to_bf16_pad<<<nblk(vox(s) * cp8(n->cin)), 256, 0, n->s>>>(x, vox(s), n->cin, cp8(n->cin), n->xin);
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
    unet_tc::k_to_bf16_pad<<<nblk(vox(s) * cp8(n->cin)), 256, 0, n->s>>>(x, vox(s), n->cin, cp8(n->cin), n->xin);
    if (forward(n, s) != cudaSuccess) return STOKES_ERR_CUDA;
    int64_t per = (int64_t)D * H * W * n->cout;
    k_loss_partials<<<dim3(LOSS_BLOCKS, B), 256, 0, n->s>>>(n->out, y, per, n->sums + 2 * 1024);
    k_loss_finish<<<(B + 127) / 128, 128, 0, n->s>>>(n->sums + 2 * 1024, B, n->sums);
    k_loss_grad<<<nblk(per * B), 256, 0, n->s>>>(n->out, y, per, B, n->sums, n->g_a);
    cudaMemsetAsync(n->grad, 0, 4 * n->np, n->s);
    if (backward(n, s) != cudaSuccess) return STOKES_ERR_CUDA;
    std::vector<double> sums(2 * B);
    cudaMemcpyAsync(sums.data(), n->sums, 16 * B, cudaMemcpyDeviceToHost, n->s);
    if (cudaStreamSynchronize(n->s) != cudaSuccess) return STOKES_ERR_CUDA;
    if (loss) {
        double L = 0;
        for (int b = 0; b < B; ++b) L += sums[2 * b + 1] > 0.0 ? sums[2 * b] / sums[2 * b + 1] : 0.0;
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
    n->wf_valid = false;
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
