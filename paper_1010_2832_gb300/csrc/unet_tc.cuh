// Tensor-core convolutions of the learned preconditioner's U-Net (implicit
// GEMM on mma.sync m16n8k16 / m16n8k8, BF16 operands, FP32 accumulation).
//
// Layout: activations are channel-last BF16 with the channel count padded to
// a multiple of 8 (cp(c)), so that every voxel's channels start on a 16-byte
// boundary and 8 channels form one ldmatrix row.  A CTA of 256 threads
// (8 warps) owns a tile of 256 output voxels (3D 8 x 8 x 4, 2D 16 x 16) and
// stages its input halo in shared memory (voxel stride cp + 8 halves, which
// spreads the ldmatrix rows over the banks).
//
// * Forward / data gradient (k_conv_tc): out[v][co] = sum over taps and input
//   channels of in[v + tap][ci] W[co][tap][ci].  GEMM M = voxels (each warp
//   two 16-voxel m-tiles), N = output channels (n-tiles of 8), K = taps x
//   channels in chunks of 16 (one ldmatrix.x4 per m-tile: matrices 0 and 1
//   are rows 0-7 / 8-15 at channels 0-7 of the chunk, 2 and 3 at channels
//   8-15), with one k8 step for a channel count of 8 mod 16.  The packed
//   weights Wp[co][tap * cp + ci] (row stride K + 8 halves) sit in shared
//   memory; B fragments are 32-bit loads.  The epilogue adds the bias,
//   applies ReLU and stores BF16 and/or FP32.  The data gradient is the same
//   kernel on the output gradient with the flipped, transposed weights.
// * Weight gradient (k_wgrad_tc): dW[tap][ci][co] = sum over voxels
//   in[v + tap][ci] dY[v][co].  GEMM M = input channels (16-channel tiles),
//   N = output channels, K = voxels (16 per step), both operands by
//   ldmatrix.trans from the staged halo and output-gradient tile.  Work
//   units (tap, channel tile) are dealt to warps; each warp adds its
//   accumulators to the CTA's FP32 partial in shared memory (every entry has
//   one owner, so the sum order is fixed).  A persistent grid walks the
//   tiles; every CTA writes its partial, and k_wgrad_reduce sums the
//   partials in CTA order: deterministic, no atomics.
#pragma once
#include <cstdint>
#include <cuda_bf16.h>

namespace unet_tc {

__host__ __device__ constexpr int cp8(int c) { return (c + 7) / 8 * 8; }

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void ldsm4(uint32_t (&a)[4], uint32_t addr) {
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];"
                 : "=r"(a[0]), "=r"(a[1]), "=r"(a[2]), "=r"(a[3])
                 : "r"(addr));
}
__device__ __forceinline__ void ldsm2(uint32_t (&a)[2], uint32_t addr) {
    asm volatile("ldmatrix.sync.aligned.m8n8.x2.shared.b16 {%0,%1}, [%2];" : "=r"(a[0]), "=r"(a[1]) : "r"(addr));
}
__device__ __forceinline__ void ldsm4t(uint32_t (&a)[4], uint32_t addr) {
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];"
                 : "=r"(a[0]), "=r"(a[1]), "=r"(a[2]), "=r"(a[3])
                 : "r"(addr));
}
__device__ __forceinline__ void ldsm2t(uint32_t (&a)[2], uint32_t addr) {
    asm volatile("ldmatrix.sync.aligned.m8n8.x2.trans.shared.b16 {%0,%1}, [%2];" : "=r"(a[0]), "=r"(a[1]) : "r"(addr));
}
__device__ __forceinline__ void mma16(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}
__device__ __forceinline__ void mma8(float (&d)[4], const uint32_t (&a)[2], uint32_t b0) {
    asm volatile(
        "mma.sync.aligned.m16n8k8.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5}, {%6}, {%0,%1,%2,%3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(b0));
}

struct TShape { int B, D, H, W; };

// tile geometry: 3D 8 x 8 x 4 (KZ = 3), 2D 16 x 16 (KZ = 1); R = halo radius
template <int KZ, int KS>
struct Geo {
    static constexpr int TX = KZ == 3 ? 8 : 16, TY = KZ == 3 ? 8 : 16, TZ = KZ == 3 ? 4 : 1;
    static constexpr int R = KS / 2;
    static constexpr int RZ = KZ == 3 ? R : 0;
    static constexpr int HX = TX + 2 * R, HY = TY + 2 * R, HZ = TZ + 2 * RZ;
    static constexpr int NH = HX * HY * HZ;
    static constexpr int TAPS = (KZ == 3 ? KS : 1) * KS * KS;
    __host__ __device__ static int tiles(const TShape& s) {
        return s.B * ((s.D + TZ - 1) / TZ) * ((s.H + TY - 1) / TY) * ((s.W + TX - 1) / TX);
    }
    // tile t -> batch and origin
    __device__ static void origin(const TShape& s, int t, int& b, int& x0, int& y0, int& z0) {
        const int ntx = (s.W + TX - 1) / TX, nty = (s.H + TY - 1) / TY, ntz = (s.D + TZ - 1) / TZ;
        x0 = (t % ntx) * TX; t /= ntx;
        y0 = (t % nty) * TY; t /= nty;
        z0 = (t % ntz) * TZ; b = t / ntz;
    }
    // tap k -> offset in halo voxels
    __device__ static int tap_off(int k) {
        const int dx = k % KS, dy = (k / KS) % KS, dz = k / (KS * KS);
        return ((dz - RZ) * HY + (dy - R)) * HX + (dx - R);
    }
    // output voxel v of the tile -> its halo index (tap offset 0)
    __device__ static int halo_of(int v) {
        const int x = v % TX, y = (v / TX) % TY, z = v / (TX * TY);
        return ((z + RZ) * HY + (y + R)) * HX + (x + R);
    }
};

// Stage the input halo of one tile: CP channels (multiple of 8) per voxel
// from global (channel-last, CP channels), zero outside the grid; smem voxel
// stride CPS halves.
template <int KZ, int KS, int CP, int CPS>
__device__ __forceinline__ void stage_halo(const __nv_bfloat16* __restrict__ X, const TShape& s, int b, int x0, int y0,
                                           int z0, __nv_bfloat16* sx) {
    using G = Geo<KZ, KS>;
    constexpr int NG = CP / 8;
    for (int e = threadIdx.x; e < G::NH * NG; e += blockDim.x) {
        const int gq = e % NG, v = e / NG;
        const int hx = v % G::HX, hy = (v / G::HX) % G::HY, hz = v / (G::HX * G::HY);
        const int gx = x0 + hx - G::R, gy = y0 + hy - G::R, gz = z0 + hz - G::RZ;
        uint4 val = make_uint4(0u, 0u, 0u, 0u);
        if (gx >= 0 && gx < s.W && gy >= 0 && gy < s.H && gz >= 0 && gz < s.D)
            val = *reinterpret_cast<const uint4*>(X + ((((int64_t)b * s.D + gz) * s.H + gy) * s.W + gx) * CP + 8 * gq);
        *reinterpret_cast<uint4*>(sx + v * CPS + 8 * gq) = val;
    }
}

// ---- forward / data gradient ------------------------------------------------
// Wp: packed BF16 weights [COUTP][K] (K = TAPS * CP), read into shared
// memory with row stride K + 8.  bias: FP32 [cout] or null.  Outputs: Yb
// (BF16, COUTP channels, the padded channels written as zero) and/or Yf
// (FP32, cout channels).
template <int KZ, int KS, int CP, int COUTP>
struct ConvCfg {
    using G = Geo<KZ, KS>;
    static constexpr int CPS = CP + 8;
    static constexpr int K = G::TAPS * CP;
    static constexpr int KW = K + 8;
    static constexpr int NT = COUTP / 8;
    static constexpr size_t SMEM = (size_t)G::NH * CPS * 2 + (size_t)COUTP * KW * 2;
};

template <int KZ, int KS, int CP, int COUTP>
__global__ void __launch_bounds__(256) k_conv_tc(const __nv_bfloat16* __restrict__ X, TShape s,
                                                 const __nv_bfloat16* __restrict__ Wp, const float* __restrict__ bias,
                                                 int cout, int relu, __nv_bfloat16* __restrict__ Yb,
                                                 float* __restrict__ Yf) {
    using C = ConvCfg<KZ, KS, CP, COUTP>;
    using G = typename C::G;
    extern __shared__ __align__(16) unsigned char smraw[];
    __nv_bfloat16* sx = reinterpret_cast<__nv_bfloat16*>(smraw);
    __nv_bfloat16* sw = sx + G::NH * C::CPS;
    // weights: [COUTP][K] -> stride KW, 16-byte pieces
    for (int e = threadIdx.x; e < COUTP * (C::K / 8); e += blockDim.x) {
        const int n = e / (C::K / 8), q = e % (C::K / 8);
        *reinterpret_cast<uint4*>(sw + n * C::KW + 8 * q) =
            *reinterpret_cast<const uint4*>(Wp + (int64_t)n * C::K + 8 * q);
    }
    int b, x0, y0, z0;
    G::origin(s, blockIdx.x, b, x0, y0, z0);
    stage_halo<KZ, KS, CP, C::CPS>(X, s, b, x0, y0, z0, sx);
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int g = lane >> 2, t = lane & 3;
    const int li = lane >> 3, lj = lane & 7;
    // ldmatrix rows: voxel (li & 1) * 8 + lj of each m-tile, channel half li >> 1
    int hrow[2];
#pragma unroll
    for (int m = 0; m < 2; ++m) hrow[m] = G::halo_of(32 * warp + 16 * m + (li & 1) * 8 + lj);
    const uint32_t sxa = smem_addr(sx), swa = smem_addr(sw);
    float acc[2][C::NT][4];
#pragma unroll
    for (int m = 0; m < 2; ++m)
#pragma unroll
        for (int nt = 0; nt < C::NT; ++nt)
#pragma unroll
            for (int q = 0; q < 4; ++q) acc[m][nt][q] = 0.f;
    for (int tap = 0; tap < G::TAPS; ++tap) {
        const int toff = G::tap_off(tap);
        const int kbase = tap * CP;
#pragma unroll
        for (int c16 = 0; c16 < CP / 16; ++c16) {
            uint32_t a[2][4];
#pragma unroll
            for (int m = 0; m < 2; ++m)
                ldsm4(a[m], sxa + 2u * (uint32_t)((hrow[m] + toff) * C::CPS + 16 * c16 + (li >> 1) * 8));
#pragma unroll
            for (int nt = 0; nt < C::NT; ++nt) {
                const uint32_t wa = swa + 2u * (uint32_t)((8 * nt + g) * C::KW + kbase + 16 * c16 + 2 * t);
                uint32_t b0, b1;
                asm volatile("ld.shared.b32 %0, [%1];" : "=r"(b0) : "r"(wa));
                asm volatile("ld.shared.b32 %0, [%1];" : "=r"(b1) : "r"(wa + 16u));
#pragma unroll
                for (int m = 0; m < 2; ++m) mma16(acc[m][nt], a[m], b0, b1);
            }
        }
        if constexpr (CP % 16 == 8) {
            uint32_t a[2][2];
#pragma unroll
            for (int m = 0; m < 2; ++m)
                ldsm2(a[m], sxa + 2u * (uint32_t)((hrow[m] + toff) * C::CPS + CP - 8));
#pragma unroll
            for (int nt = 0; nt < C::NT; ++nt) {
                const uint32_t wa = swa + 2u * (uint32_t)((8 * nt + g) * C::KW + kbase + CP - 8 + 2 * t);
                uint32_t b0;
                asm volatile("ld.shared.b32 %0, [%1];" : "=r"(b0) : "r"(wa));
#pragma unroll
                for (int m = 0; m < 2; ++m) mma8(acc[m][nt], a[m], b0);
            }
        }
    }
    // epilogue: D[row][col] = acc[..][q]: rows g (q 0, 1) and g + 8 (q 2, 3), columns 2t, 2t + 1
#pragma unroll
    for (int m = 0; m < 2; ++m)
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int v = 32 * warp + 16 * m + g + 8 * h;
            const int x = x0 + v % G::TX, y = y0 + (v / G::TX) % G::TY, z = z0 + v / (G::TX * G::TY);
            if (x >= s.W || y >= s.H || z >= s.D) continue;
            const int64_t o = (((int64_t)b * s.D + z) * s.H + y) * s.W + x;
#pragma unroll
            for (int nt = 0; nt < C::NT; ++nt) {
                const int c = 8 * nt + 2 * t;
                float v0 = acc[m][nt][2 * h], v1 = acc[m][nt][2 * h + 1];
                if (bias) {
                    v0 += c < cout ? bias[c] : 0.f;
                    v1 += c + 1 < cout ? bias[c + 1] : 0.f;
                }
                if (relu) { v0 = fmaxf(v0, 0.f); v1 = fmaxf(v1, 0.f); }
                if (c >= cout) v0 = 0.f;
                if (c + 1 >= cout) v1 = 0.f;
                if (Yb) *reinterpret_cast<__nv_bfloat162*>(Yb + o * COUTP + c) = __floats2bfloat162_rn(v0, v1);
                if (Yf) {
                    if (c < cout) Yf[o * cout + c] = v0;
                    if (c + 1 < cout) Yf[o * cout + c + 1] = v1;
                }
            }
        }
}

// ---- weight gradient ----------------------------------------------------------
// X: layer input (BF16, CP channels), dY: output gradient (BF16, COUTP
// channels).  part: FP32 [gridDim.x][TAPS * CP * COUTP + COUTP] partials
// (weights as [tap][ci][co], then the bias gradient).
template <int KZ, int KS, int CP, int COUTP>
struct WgCfg {
    using G = Geo<KZ, KS>;
    static constexpr int CPS = CP + 8;
    static constexpr int COS = COUTP + 8;
    static constexpr int MT = (CP + 15) / 16;                 // 16-channel tiles of the input
    static constexpr int NT = COUTP / 8;
    static constexpr int E = G::TAPS * CP * COUTP;
    static constexpr int UNITS = G::TAPS * MT;
    static constexpr size_t SMEM = (size_t)G::NH * CPS * 2 + (size_t)256 * COS * 2 + (size_t)(E + COUTP) * 4;
};

template <int KZ, int KS, int CP, int COUTP>
__global__ void __launch_bounds__(256) k_wgrad_tc(const __nv_bfloat16* __restrict__ X, TShape s,
                                                  const __nv_bfloat16* __restrict__ dY, float* __restrict__ part) {
    using C = WgCfg<KZ, KS, CP, COUTP>;
    using G = typename C::G;
    extern __shared__ __align__(16) unsigned char smraw[];
    __nv_bfloat16* sx = reinterpret_cast<__nv_bfloat16*>(smraw);
    __nv_bfloat16* sy = sx + G::NH * C::CPS;
    float* dw = reinterpret_cast<float*>(sy + 256 * C::COS);     // [E] then [COUTP]
    for (int e = threadIdx.x; e < C::E + COUTP; e += blockDim.x) dw[e] = 0.f;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int g = lane >> 2, t = lane & 3;
    const int li = lane >> 3, lj = lane & 7;
    const uint32_t sxa = smem_addr(sx), sya = smem_addr(sy);
    const int ntiles = G::tiles(s);
    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        int b, x0, y0, z0;
        G::origin(s, tile, b, x0, y0, z0);
        __syncthreads();                                  // the previous tile's operands are no longer read
        stage_halo<KZ, KS, CP, C::CPS>(X, s, b, x0, y0, z0, sx);
        for (int e = threadIdx.x; e < 256 * (COUTP / 8); e += blockDim.x) {
            const int q = e % (COUTP / 8), v = e / (COUTP / 8);
            const int x = x0 + v % G::TX, y = y0 + (v / G::TX) % G::TY, z = z0 + v / (G::TX * G::TY);
            uint4 val = make_uint4(0u, 0u, 0u, 0u);
            if (x < s.W && y < s.H && z < s.D)
                val = *reinterpret_cast<const uint4*>(dY + ((((int64_t)b * s.D + z) * s.H + y) * s.W + x) * COUTP +
                                                      8 * q);
            *reinterpret_cast<uint4*>(sy + v * C::COS + 8 * q) = val;
        }
        __syncthreads();
        // bias gradient: thread co sums the tile's 256 voxels in order
        if (threadIdx.x < COUTP) {
            float acc = 0.f;
            for (int v = 0; v < 256; ++v) acc += __bfloat162float(sy[v * C::COS + threadIdx.x]);
            dw[C::E + threadIdx.x] += acc;
        }
        for (int u = warp; u < C::UNITS; u += 8) {
            const int tap = u / C::MT, mt = u % C::MT;
            const int toff = G::tap_off(tap);
            const bool half = CP - 16 * mt == 8;          // the tile's upper 8 channels do not exist
            float acc[C::NT][4];
#pragma unroll
            for (int nt = 0; nt < C::NT; ++nt)
#pragma unroll
                for (int q = 0; q < 4; ++q) acc[nt][q] = 0.f;
            for (int c = 0; c < 16; ++c) {
                // A = X^T: matrix li holds channels (li & 1) * 8 + 0..7 of voxels (li >> 1) * 8 + 0..7
                uint32_t a[4];
                const int va = 16 * c + (li >> 1) * 8 + lj;
                const int cha = 16 * mt + (half ? 0 : (li & 1) * 8);
                ldsm4t(a, sxa + 2u * (uint32_t)((G::halo_of(va) + toff) * C::CPS + cha));
                if (half) { a[1] = 0u; a[3] = 0u; }
                const int vb = 16 * c + (li & 1) * 8 + lj;
#pragma unroll
                for (int nt = 0; nt + 1 < C::NT; nt += 2) {
                    uint32_t bb[4];
                    ldsm4t(bb, sya + 2u * (uint32_t)(vb * C::COS + 8 * (nt + (li >> 1))));
                    mma16(acc[nt], a, bb[0], bb[1]);
                    mma16(acc[nt + 1], a, bb[2], bb[3]);
                }
                if constexpr (C::NT % 2 == 1) {
                    uint32_t bb[2];
                    ldsm2t(bb, sya + 2u * (uint32_t)(vb * C::COS + 8 * (C::NT - 1)));
                    mma16(acc[C::NT - 1], a, bb[0], bb[1]);
                }
            }
            // D[m = channel][n = out channel]: rows g, g + 8; columns 2t, 2t + 1
#pragma unroll
            for (int nt = 0; nt < C::NT; ++nt)
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int ci = 16 * mt + g + 8 * h;
                    if (ci >= CP) continue;
                    float* d = dw + ((int64_t)tap * CP + ci) * COUTP + 8 * nt + 2 * t;
                    d[0] += acc[nt][2 * h];
                    d[1] += acc[nt][2 * h + 1];
                }
        }
    }
    __syncthreads();
    float* o = part + (int64_t)blockIdx.x * (C::E + COUTP);
    for (int e = threadIdx.x; e < C::E + COUTP; e += blockDim.x) o[e] = dw[e];
}

// dW[tap][ci][co] (ci < cin, co < cout) and db[co] from the partials of
// nparts CTAs, summed in CTA order.
__global__ void k_wgrad_reduce(const float* __restrict__ part, int nparts, int taps, int cp, int coutp, int cin,
                               int cout, float* __restrict__ dW, float* __restrict__ db) {
    const int E = taps * cp * coutp;
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= E + coutp) return;
    float acc = 0.f;
    for (int q = 0; q < nparts; ++q) acc += part[(int64_t)q * (E + coutp) + e];
    if (e >= E) {
        const int co = e - E;
        if (co < cout) db[co] = acc;
        return;
    }
    const int co = e % coutp, ci = (e / coutp) % cp, tap = e / (coutp * cp);
    if (ci < cin && co < cout) dW[((int64_t)tap * cin + ci) * cout + co] = acc;
}

// Packed BF16 weights for k_conv_tc from the FP32 master W[tap][cin][cout]:
// forward  Wp[co][tap * cp + ci] = W[tap][ci][co];
// gradient Wp[ci][tap * cpo + co] = W[taps - 1 - tap][ci][co] (the data
//          gradient as a convolution of the output gradient).
// Padded rows and columns are zero.
__global__ void k_pack_weights(const float* __restrict__ W, int taps, int cin, int cout, int rows, int cpk, int grad,
                               __nv_bfloat16* __restrict__ Wp) {
    const int K = taps * cpk;
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= rows * K) return;
    const int n = e / K, k = e % K, tap = k / cpk, c = k % cpk;
    float v = 0.f;
    if (!grad) {
        if (n < cout && c < cin) v = W[((int64_t)tap * cin + c) * cout + n];
    } else {
        if (n < cin && c < cout) v = W[((int64_t)(taps - 1 - tap) * cin + n) * cout + c];
    }
    Wp[e] = __float2bfloat16(v);
}

// FP32 channel-last (c channels) -> BF16 with cp channels (zero padded)
__global__ void k_to_bf16_pad(const float* __restrict__ x, int64_t nvox, int c, int cp, __nv_bfloat16* __restrict__ y) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= nvox * cp) return;
    const int ch = e % cp;
    const int64_t v = e / cp;
    y[e] = __float2bfloat16(ch < c ? x[v * c + ch] : 0.f);
}

}  // namespace unet_tc
