// Warm-start U-Net on the tensor cores: forward, backward and Adam.
//
// Convolutions are implicit GEMMs on channels-last BF16 activations
// [voxel][channel] with mma.sync m16n8k16 (BF16 in, FP32 accumulate):
//   forward      y[v][co] = b[co] + sum_t sum_ci x[v + off(t)][ci] W[t][co][ci]
//                (M = 16 voxels per warp, N = all output channels, K = 27 taps x Cin)
//   data grad    dx = forward(dy) with the taps flipped and W transposed,
//                because the adjoint of a zero-padded correlation is the
//                correlation with the mirrored kernel
//   weight grad  dW[t][co][ci] = sum_v dy[v][co] x[v + off(t)][ci]
//                (M = 16 output channels, N = input channels, K = voxels;
//                partial sums of voxel chunks are added with atomics)
// Pooling (2x2x2 mean), nearest upsampling, channel concatenation, ReLU
// masks, the mean-squared-error loss and Adam are elementwise kernels.
// Master weights and Adam moments are FP32; the tensor cores see BF16 copies.
#include "unet.cuh"
#include "ops.cuh"
#include "../../include/cdi.h"

#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

namespace cdi {
namespace {

using bf16 = __nv_bfloat16;

struct CG {
    int nx, ny, nz, N;
};

constexpr int kLayers = 8;
// name order e0, e1, e2, b, d2, d1, d0, head: Cin, Cout, taps
constexpr int kCin[kLayers] = {2, 16, 32, 64, 192, 96, 48, 16};
constexpr int kCout[kLayers] = {16, 32, 64, 128, 64, 32, 16, 1};
constexpr int kTaps[kLayers] = {27, 27, 27, 27, 27, 27, 27, 1};

inline int pad16(int c) { return (c + 15) / 16 * 16; }

__device__ __forceinline__ unsigned ld_pair(const bf16* p) { return *reinterpret_cast<const unsigned*>(p); }
__device__ __forceinline__ unsigned pack2(bf16 lo, bf16 hi) {
    return (unsigned)__bfloat16_as_ushort(lo) | ((unsigned)__bfloat16_as_ushort(hi) << 16);
}
__device__ __forceinline__ void mma_bf16(float* c, unsigned a0, unsigned a1, unsigned a2, unsigned a3, unsigned b0,
                                         unsigned b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

// tap t = (dz+1)*9 + (dy+1)*3 + (dx+1); a 1-tap layer is the centre only
__device__ __forceinline__ void tap_off(int tap, int ntaps, int& dz, int& dy, int& dx) {
    if (ntaps == 1) {
        dz = dy = dx = 0;
        return;
    }
    dz = tap / 9 - 1;
    dy = (tap / 3) % 3 - 1;
    dx = tap % 3 - 1;
}

struct Vox {
    int x, y, z;
    bool in;
};
__device__ __forceinline__ Vox vox(const CG& g, int v) {
    Vox o;
    o.in = v < g.N;
    const int vv = o.in ? v : 0;
    o.x = vv % g.nx;
    const int r = vv / g.nx;
    o.y = r % g.ny;
    o.z = r / g.ny;
    return o;
}
// neighbour index or -1 (zero padding)
__device__ __forceinline__ int nbr(const CG& g, const Vox& p, int dz, int dy, int dx) {
    const int x = p.x + dx, y = p.y + dy, z = p.z + dz;
    if (!p.in || x < 0 || x >= g.nx || y < 0 || y >= g.ny || z < 0 || z >= g.nz) return -1;
    return x + g.nx * (y + g.ny * z);
}

// forward convolution (also the data gradient with flipped, transposed W)
template <int NF, bool OUTF32>
__global__ void __launch_bounds__(128) k_conv(CG g, const bf16* __restrict__ in, int cin_pad,
                                              const bf16* __restrict__ w, int cout_pad, const float* __restrict__ bias,
                                              int cout, void* out, int out_stride, int out_off, int relu, int ntaps) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, gid = lane >> 2, tig = lane & 3;
    const int r0 = (blockIdx.x * 4 + warp) * 16 + gid, r1 = r0 + 8;
    const Vox v0 = vox(g, r0), v1 = vox(g, r1);
    float acc[NF][4];
#pragma unroll
    for (int j = 0; j < NF; ++j) acc[j][0] = acc[j][1] = acc[j][2] = acc[j][3] = 0.f;
    for (int tap = 0; tap < ntaps; ++tap) {
        int dz, dy, dx;
        tap_off(tap, ntaps, dz, dy, dx);
        const int n0 = nbr(g, v0, dz, dy, dx), n1 = nbr(g, v1, dz, dy, dx);
        const bf16* p0 = in + (size_t)(n0 < 0 ? 0 : n0) * cin_pad + 2 * tig;
        const bf16* p1 = in + (size_t)(n1 < 0 ? 0 : n1) * cin_pad + 2 * tig;
        const bf16* wt = w + ((size_t)tap * cout_pad + gid) * cin_pad + 2 * tig;
        for (int k0 = 0; k0 < cin_pad; k0 += 16) {
            const unsigned a0 = n0 >= 0 ? ld_pair(p0 + k0) : 0u;
            const unsigned a1 = n1 >= 0 ? ld_pair(p1 + k0) : 0u;
            const unsigned a2 = n0 >= 0 ? ld_pair(p0 + k0 + 8) : 0u;
            const unsigned a3 = n1 >= 0 ? ld_pair(p1 + k0 + 8) : 0u;
#pragma unroll
            for (int j = 0; j < NF; ++j) {
                const bf16* wj = wt + (size_t)j * 8 * cin_pad + k0;
                mma_bf16(acc[j], a0, a1, a2, a3, ld_pair(wj), ld_pair(wj + 8));
            }
        }
    }
#pragma unroll
    for (int j = 0; j < NF; ++j)
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int r = h ? r1 : r0;
            if (r >= g.N) continue;
#pragma unroll
            for (int e = 0; e < 2; ++e) {
                const int co = j * 8 + 2 * tig + e;
                if (co >= cout) continue;
                float v = acc[j][2 * h + e] + (bias ? bias[co] : 0.f);
                if (relu) v = fmaxf(v, 0.f);
                const size_t o = (size_t)r * out_stride + out_off + co;
                if (OUTF32) reinterpret_cast<float*>(out)[o] = v;
                else reinterpret_cast<bf16*>(out)[o] = __float2bfloat16(v);
            }
        }
}

// weight gradient: dW[t][co][ci] += sum over a voxel chunk of dy[v][co] x[v+off(t)][ci]
template <int NF>
__global__ void __launch_bounds__(128) k_wgrad(CG g, const bf16* __restrict__ in, int cin_pad,
                                               const bf16* __restrict__ dyv, int cout_pad, float* dW, int cout, int cin,
                                               int ntaps, int chunk) {
    const int tap = blockIdx.x, co0 = blockIdx.y * 16;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, gid = lane >> 2, tig = lane & 3;
    int dz, dy, dx;
    tap_off(tap, ntaps, dz, dy, dx);
    float acc[NF][4];
#pragma unroll
    for (int j = 0; j < NF; ++j) acc[j][0] = acc[j][1] = acc[j][2] = acc[j][3] = 0.f;
    const int per_warp = chunk / 4;
    const int vbeg = blockIdx.z * chunk + warp * per_warp;
    const int vend = min(vbeg + per_warp, g.N);
    const bf16 zero = __float2bfloat16(0.f);
    auto dyat = [&](int v, int co) { return (v < g.N && co < cout_pad) ? dyv[(size_t)v * cout_pad + co] : zero; };
    for (int vb = vbeg; vb < vend; vb += 16) {
        const int vk[4] = {vb + 2 * tig, vb + 2 * tig + 1, vb + 2 * tig + 8, vb + 2 * tig + 9};
        const int ca = co0 + gid, cb = co0 + gid + 8;
        const unsigned a0 = pack2(dyat(vk[0], ca), dyat(vk[1], ca));
        const unsigned a1 = pack2(dyat(vk[0], cb), dyat(vk[1], cb));
        const unsigned a2 = pack2(dyat(vk[2], ca), dyat(vk[3], ca));
        const unsigned a3 = pack2(dyat(vk[2], cb), dyat(vk[3], cb));
        int nb[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) nb[i] = (vk[i] < vend) ? nbr(g, vox(g, vk[i]), dz, dy, dx) : -1;
#pragma unroll
        for (int j = 0; j < NF; ++j) {
            const int ci = j * 8 + gid;
            auto xin = [&](int n) { return n >= 0 ? in[(size_t)n * cin_pad + ci] : zero; };
            mma_bf16(acc[j], a0, a1, a2, a3, pack2(xin(nb[0]), xin(nb[1])), pack2(xin(nb[2]), xin(nb[3])));
        }
    }
#pragma unroll
    for (int j = 0; j < NF; ++j)
#pragma unroll
        for (int h = 0; h < 2; ++h)
#pragma unroll
            for (int e = 0; e < 2; ++e) {
                const int co = co0 + gid + 8 * h, ci = j * 8 + 2 * tig + e;
                if (co < cout && ci < cin) atomicAdd(&dW[((size_t)tap * cout + co) * cin + ci], acc[j][2 * h + e]);
            }
}

__global__ void k_bias_grad(int N, const bf16* dy, int stride, int C, float* db) {
    const int c = blockIdx.y;
    float s = 0.f;
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < N; v += gridDim.x * blockDim.x)
        s += __bfloat162float(dy[(size_t)v * stride + c]);
    __shared__ float sh[256];
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) atomicAdd(&db[c], sh[0]);
}

// 2x2x2 mean of the fine grid gf into the coarse grid; 8 channels (16 bytes) per thread
__global__ void k_pool(CG gf, const bf16* in, int C, bf16* out) {
    const int Nc = gf.N / 8, C8 = C / 8;
    const long t = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (long)Nc * C8) return;
    const int g8 = (int)(t % C8), V = (int)(t / C8);
    const int cx = gf.nx / 2, cy = gf.ny / 2;
    const int X = V % cx, Y = (V / cx) % cy, Z = V / (cx * cy);
    float s[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    for (int k = 0; k < 2; ++k)
        for (int j = 0; j < 2; ++j)
            for (int i = 0; i < 2; ++i) {
                const size_t v = (size_t)((2 * X + i) + gf.nx * ((2 * Y + j) + gf.ny * (2 * Z + k)));
                const uint4 q = *reinterpret_cast<const uint4*>(in + v * C + 8 * g8);
                const bf16* h = reinterpret_cast<const bf16*>(&q);
#pragma unroll
                for (int e = 0; e < 8; ++e) s[e] += __bfloat162float(h[e]);
            }
    __align__(16) bf16 o[8];
#pragma unroll
    for (int e = 0; e < 8; ++e) o[e] = __float2bfloat16(0.125f * s[e]);
    *reinterpret_cast<uint4*>(out + (size_t)V * C + 8 * g8) = *reinterpret_cast<const uint4*>(o);
}

// din[v][off+c] += dout[parent(v)][c] / 8 on the fine grid gf
__global__ void k_pool_bwd_add(CG gf, const bf16* dout, int C, bf16* din, int stride, int off) {
    const long t = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (long)gf.N * C) return;
    const int c = (int)(t % C), v = (int)(t / C);
    const int x = v % gf.nx, y = (v / gf.nx) % gf.ny, z = v / (gf.nx * gf.ny);
    const int P = (x / 2) + (gf.nx / 2) * ((y / 2) + (gf.ny / 2) * (z / 2));
    const size_t o = (size_t)v * stride + off + c;
    din[o] = __float2bfloat16(__bfloat162float(din[o]) + 0.125f * __bfloat162float(dout[(size_t)P * C + c]));
}

// nearest upsampling of the coarse input into channels [off, off+C) of the fine output; 8 channels per thread
__global__ void k_up(CG gf, const bf16* in, int C, bf16* out, int stride, int off) {
    const int C8 = C / 8;
    const long t = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (long)gf.N * C8) return;
    const int g8 = (int)(t % C8), v = (int)(t / C8);
    const int x = v % gf.nx, y = (v / gf.nx) % gf.ny, z = v / (gf.nx * gf.ny);
    const int P = (x / 2) + (gf.nx / 2) * ((y / 2) + (gf.ny / 2) * (z / 2));
    *reinterpret_cast<uint4*>(out + (size_t)v * stride + off + 8 * g8) =
        *reinterpret_cast<const uint4*>(in + (size_t)P * C + 8 * g8);
}

// adjoint of k_up: din[V][c] = sum of the 8 children dout[child][off+c]
__global__ void k_up_bwd(CG gf, const bf16* dout, int stride, int off, int C, bf16* din) {
    const int Nc = gf.N / 8;
    const long t = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (long)Nc * C) return;
    const int c = (int)(t % C), V = (int)(t / C);
    const int cx = gf.nx / 2, cy = gf.ny / 2;
    const int X = V % cx, Y = (V / cx) % cy, Z = V / (cx * cy);
    float s = 0.f;
    for (int k = 0; k < 2; ++k)
        for (int j = 0; j < 2; ++j)
            for (int i = 0; i < 2; ++i)
                s += __bfloat162float(
                    dout[(size_t)((2 * X + i) + gf.nx * ((2 * Y + j) + gf.ny * (2 * Z + k))) * stride + off + c]);
    din[t] = __float2bfloat16(s);
}

// channel block copy, 8 channels (16 bytes) per thread; strides, offsets and C multiples of 8
__global__ void k_copy_ch(int N, const bf16* src, int sstride, int soff, bf16* dst, int dstride, int doff, int C) {
    const int C8 = C / 8;
    const long t = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (long)N * C8) return;
    const int g8 = (int)(t % C8), v = (int)(t / C8);
    *reinterpret_cast<uint4*>(dst + (size_t)v * dstride + doff + 8 * g8) =
        *reinterpret_cast<const uint4*>(src + (size_t)v * sstride + soff + 8 * g8);
}

// g *= (y > 0) (ReLU backward), both [N][C] contiguous
__global__ void k_relu_mask(long n, bf16* g, const bf16* y) {
    const long t = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t < n && !(__bfloat162float(y[t]) > 0.f)) g[t] = __float2bfloat16(0.f);
}

// mean squared error: partial sums of (y-t)^2 and the BF16 gradient 2(y-t)/N in channel 0 of 16
__global__ void k_loss(int N, const float* y, const float* t, bf16* gy, float* part) {
    float s = 0.f;
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < N; v += gridDim.x * blockDim.x) {
        const float d = y[v] - t[v];
        s += d * d;
        gy[(size_t)v * 16] = __float2bfloat16(2.f * d / (float)N);
    }
    __shared__ float sh[256];
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) atomicAdd(part, sh[0]);
}

// Adam (Kingma and Ba, 2015) with bias corrections bc1 = 1 - b1^t, bc2 = 1 - b2^t
__global__ void k_adam(long n, float* w, const float* g, float* m, float* v, float lr, float b1, float b2, float eps,
                       float bc1, float bc2) {
    const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    w[i] -= lr * (mi / bc1) / (sqrtf(vi / bc2) + eps);
}

// BF16 copies: wb[t][co_pad][ci_pad] = W[t][co][ci]; wt[t][ci_pad][co_pad] = W[T-1-t][co][ci]
__global__ void k_weights_bf16(const float* W, int taps, int cout, int cin, int co_pad, int ci_pad, bf16* wb,
                               bf16* wt) {
    const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
    const long n = (long)taps * co_pad * ci_pad;
    if (i >= n) return;
    const int ci = (int)(i % ci_pad), co = (int)((i / ci_pad) % co_pad), t = (int)(i / ((long)ci_pad * co_pad));
    const float val = (co < cout && ci < cin) ? W[((size_t)t * cout + co) * cin + ci] : 0.f;
    wb[i] = __float2bfloat16(val);
    const int tf = taps - 1 - t;
    wt[((size_t)tf * ci_pad + ci) * co_pad + co] = __float2bfloat16(val);
}

__global__ void k_input_host(int N, const double* x2, bf16* x) {  // x2: [N][2] from the host
    const long t = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (long)N * 16) return;
    const int c = (int)(t % 16), v = (int)(t / 16);
    x[t] = __float2bfloat16(c < 2 ? (float)x2[(size_t)v * 2 + c] : 0.f);
}

__global__ void k_input_dev(int N, const float* x2, bf16* x) {  // x2: [N][2] on the device
    const long t = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (long)N * 16) return;
    const int c = (int)(t % 16), v = (int)(t / 16);
    x[t] = __float2bfloat16(c < 2 ? x2[(size_t)v * 2 + c] : 0.f);
}

// scales of one prediction from ||f||_2 (one thread): sd = {1/rms(f), rms(f) max(rho) h^2}
// in FP64 and sf the same in FP32; a zero right-hand side gives a zero guess
__global__ void k_solver_scales(const double* fnorm, int N, double rho_h2, double* sd, float* sf) {
    const double rms = *fnorm / sqrt((double)N);
    sd[0] = rms > 0.0 ? 1.0 / rms : 0.0;
    sd[1] = rms * rho_h2;
    sf[0] = (float)sd[0];
    sf[1] = (float)sd[1];
}

// network input from the solver's f (its mean already removed in the FP64
// form; removed here with the double-float mean in the FP32-mixed form) and phi
template <typename T>
__global__ void k_input_solver(int N, const FT<T>* f, const float* fmean_df, const T* phi, float drho, float rho2,
                               float inv_rmax, const double* sd, const float* sf, bf16* x) {
    const long t = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (long)N * 16) return;
    const int c = (int)(t % 16), v = (int)(t / 16);
    float val = 0.f;
    if (c == 0) {
        if constexpr (sizeof(T) == 8) val = (float)(f[v] * sd[0]);
        else val = ((f[v] - fmean_df[0]) - fmean_df[1]) * sf[0];
    } else if (c == 1) {
        val = (drho * (float)phi[v] + rho2) * inv_rmax;
    }
    x[t] = __float2bfloat16(val);
}

template <typename T>
__global__ void k_output_solver(int N, const float* y, const double* sd, const float* sf, PT<T>* p) {
    const long v = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= N) return;
    if constexpr (sizeof(T) == 8) p[v] = (double)y[v] * sd[1];
    else p[v] = make_float2(y[v] * sf[1], 0.f);
}

unsigned blocks(long n, int t = 256) { return (unsigned)((n + t - 1) / t); }

// ---------------------------------------------------------------------------
// 3x3x3 convolution on the 5th-generation tensor cores (tcgen05).
//
// One CTA of 128 threads computes output tiles of 8 (x) x 16 (y) x 2 (z)
// voxels for all N output channels: two M = 128 GEMMs (one per z plane) whose
// FP32 accumulators D[128][N] live side by side in tensor memory (TMEM lane m
// = voxel m of the plane, column zp N + n = channel n).  The work of a tile is
// a sequence of steps (16-input-channel block cb, nine taps t0 .. t0+8).  For
// each channel block the CTA stages the input tile with a one-voxel halo
// (10 x 18 x 4 voxels) in shared memory once, and every tap of both planes
// reads its A operand from it: tap (dz, dy, dx) is the tile shifted by whole
// 16-byte rows, so it only changes the start address of the shared-memory
// matrix descriptor.  Halo tiles and weight blocks are double-buffered and
// filled with cp.async while the tensor core works on the previous step; one
// thread issues the MMAs (tcgen05.mma.cta_group::1.kind::f16: BF16 A and B,
// FP32 D, M = 128, K = 16) and commits them to the step's mbarrier, and a
// buffer is refilled only after the MMAs that read it have completed.
// Operands use the canonical K-major layout without swizzling: a core matrix
// is 8 rows of 16 bytes (8 channels) stored contiguously; the descriptor's
// leading offset steps to the next 8 channels, its stride offset to the next
// 8 rows.
// ---------------------------------------------------------------------------
constexpr int kTcThreads = 128;
constexpr int kTileX = 8, kTileY = 16, kTileZ = 2;
constexpr int kHX = kTileX + 2, kHY = kTileY + 2, kHZ = kTileZ + 2, kKC = 2;  // halo; 16 channels = 2 x 8
constexpr int kHaloUnits = kHZ * kHY * kKC * kHX;                            // 16-byte units
constexpr int kHaloBytes = kHaloUnits * 16;
constexpr int kGuardBytes = 4096;
constexpr int kTapsPerIter = 9;

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ unsigned long long tc_globaltimer() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
// wait (at most about one second) for the phase of the given parity to complete
// Wait for phase `parity` of an mbarrier.  It gives up only after 1 s of
// wall time AND 2^20 polls: a context switched out by time slicing does not
// poll, so a long preemption alone cannot end the wait.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity) {
    const unsigned long long t0 = tc_globaltimer();
    long polls = 0;
    while (!mbar_try_wait(bar, parity))
        if (++polls > (1L << 20) && tc_globaltimer() - t0 > 1000000000ull) return false;
    return true;
}
// A second wait for a phase whose first wait gave up, bounded by polls only
// (2^22 polls with a 1 us back-off, about 4 s of running time); true once
// the phase completed.
__device__ __forceinline__ bool mbar_drain(uint64_t* bar, uint32_t parity) {
    for (long it = 0; it < (1L << 22); ++it) {
        if (mbar_try_wait(bar, parity)) return true;
        __nanosleep(1000);
    }
    return false;
}
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// shared-memory matrix descriptor: start address, leading byte offset (next 8
// channels), stride byte offset (next 8 rows), descriptor version 1, no swizzle
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = (uint64_t)((saddr >> 4) & 0x3FFFu);
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;
    return d;
}
// instruction descriptor of kind::f16: FP32 D, BF16 A and B, both K-major, M x N
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void tc_mma(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                       uint32_t accumulate) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}
__device__ __forceinline__ void tc_commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}
// 8 consecutive FP32 columns of this thread's TMEM lane
__device__ __forceinline__ void tmem_ld8(uint32_t taddr, float* v) {
    uint32_t r[8];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
                 : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 8; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ void cp_async16(uint32_t saddr, const void* g, bool valid) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(saddr), "l"(g), "r"(valid ? 16 : 0)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

// tcgen05 convolution: out[v][co] = act(bias[co] + sum_t sum_ci in[v + off(t)][ci] w[t][co][ci]) for
// co < cout (BF16 out, row stride out_stride); cin and N multiples of 16, N <= 256; ncols: TMEM
// columns (a power of two >= max(32, 2N)).  With up != NULL the input is the concatenation
// [nearest upsampling of up (cup channels, on the grid of half the extents), in (cin - cup channels)],
// gathered while staging instead of being stored.  On a wait that runs out, *err is set to 1 and
// the CTA stops.  Tensor memory is released only once every MMA the CTA committed has been seen
// complete: a barrier whose wait gave up is waited for again (poll-bounded) before the dealloc;
// if an MMA is still unconfirmed then, *err is set to 2 (the CTA must still release its columns
// before it exits, so their contents are not to be trusted by any later kernel of the context).
__global__ void __launch_bounds__(kTcThreads) k_conv_tc(CG g, const bf16* __restrict__ in, int cin,
                                                        const bf16* __restrict__ up, int cup,
                                                        const bf16* __restrict__ w, int N,
                                                        const float* __restrict__ bias, int cout, bf16* out,
                                                        int out_stride, int relu, int ncols, int* err) {
    extern __shared__ __align__(1024) unsigned char smem[];
    __shared__ __align__(8) uint64_t mbar[2];
    __shared__ uint32_t s_tmem;
    __shared__ int s_abort;
    const int bunits = kTapsPerIter * 2 * N;  // 16-byte units of one weight buffer
    const uint32_t halo_addr = smem_u32(smem);                                   // 2 halo buffers
    const uint32_t b_addr = smem_u32(smem + 2 * kHaloBytes + kGuardBytes);       // 2 weight buffers
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&s_tmem)),
                     "r"(ncols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        mbar_init(&mbar[0], 1);
        mbar_init(&mbar[1], 1);
        s_abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = s_tmem;
    const uint32_t idesc = idesc_bf16(128, N);

    const int tiles_x = (g.nx + kTileX - 1) / kTileX, tiles_y = (g.ny + kTileY - 1) / kTileY;
    const int tiles_z = (g.nz + kTileZ - 1) / kTileZ;
    const long ntiles = (long)tiles_x * tiles_y * tiles_z;
    const int ncb = cin / 16, steps_per_cb = 27 / kTapsPerIter;
    const int steps_per_tile = ncb * steps_per_cb;
    // this CTA's tiles: blockIdx.x, blockIdx.x + gridDim.x, ...; its steps are numbered 0, 1, ...
    const long my_tiles = blockIdx.x < ntiles ? (ntiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;
    const long nsteps = my_tiles * steps_per_tile;
    uint32_t phase[2] = {0u, 0u};
    bool pending[2] = {false, false};
    bool unconfirmed[2] = {false, false};   // a wait on this barrier gave up (phase uphase[b])
    uint32_t uphase[2] = {0u, 0u};

    auto tile_origin = [&](long k, int& x0, int& y0, int& z0) {
        const long tile = blockIdx.x + k * gridDim.x;
        const long tz = tile / ((long)tiles_x * tiles_y);
        const int rem = (int)(tile - tz * tiles_x * tiles_y);
        z0 = (int)tz * kTileZ;
        y0 = (rem / tiles_x) * kTileY;
        x0 = (rem % tiles_x) * kTileX;
    };
    // wait for the MMAs committed to mbarrier b (every thread; a wait that runs out sets s_abort)
    auto wait_mma = [&](int b) {
        if (pending[b]) {
            if (!mbar_wait_bounded(&mbar[b], phase[b])) {
                s_abort = 1;
                atomicExch(err, 1);
                unconfirmed[b] = true;
                uphase[b] = phase[b];
            }
            phase[b] ^= 1u;
            pending[b] = false;
        }
    };
    // issue the cp.async loads of step s: the halo tile when s starts a channel block, and the weights
    auto load_step = [&](long s) {
        const long k = s / steps_per_tile;
        const int r = (int)(s - k * steps_per_tile), cbi = r / steps_per_cb, t0 = (r % steps_per_cb) * kTapsPerIter;
        const int cb = cbi * 16;
        if (t0 == 0) {
            int x0, y0, z0;
            tile_origin(k, x0, y0, z0);
            const uint32_t hbase = halo_addr + (uint32_t)(((k * ncb + cbi) & 1) * kHaloBytes);
            for (int u = tid; u < kHaloUnits; u += kTcThreads) {
                const int hx = u % kHX, r1 = u / kHX, kc = r1 % kKC, r2 = r1 / kKC, hy = r2 % kHY, hz = r2 / kHY;
                const int gx = x0 + hx - 1, gy = y0 + hy - 1, gz = z0 + hz - 1;
                const bool ok = gx >= 0 && gx < g.nx && gy >= 0 && gy < g.ny && gz >= 0 && gz < g.nz;
                const int c = cb + kc * 8;
                const bf16* src = in;
                if (ok) {
                    if (c < cup)
                        src = up + ((size_t)((long)(gz >> 1) * (g.ny >> 1) + (gy >> 1)) * (g.nx >> 1) + (gx >> 1)) * cup +
                              c;
                    else
                        src = in + ((size_t)((long)gz * g.ny + gy) * g.nx + gx) * (cin - cup) + (c - cup);
                }
                cp_async16(hbase + (uint32_t)u * 16u, src, ok);
            }
        }
        const uint32_t bbase = b_addr + (uint32_t)((s & 1) * bunits * 16);
        for (int u = tid; u < bunits; u += kTcThreads) {
            const int t = u / (2 * N), rr = u - t * 2 * N;
            const int ng = rr >> 4, kc = (rr >> 3) & 1, n = ng * 8 + (rr & 7);
            cp_async16(bbase + (uint32_t)u * 16u, w + ((size_t)(t0 + t) * N + n) * cin + cb + kc * 8, true);
        }
        cp_async_commit();
    };

    if (nsteps > 0) load_step(0);
    for (long s = 0; s < nsteps; ++s) {
        const long k = s / steps_per_tile;
        const int r = (int)(s - k * steps_per_tile), cbi = r / steps_per_cb, t0 = (r % steps_per_cb) * kTapsPerIter;
        // operands of step s are in shared memory
        cp_async_wait_all();
        fence_proxy_async();
        __syncthreads();
        if (s_abort) break;
        if (tid == 0) {
            tc_fence_after();
            const uint32_t hbase = halo_addr + (uint32_t)(((k * ncb + cbi) & 1) * kHaloBytes);
            const uint32_t bbase = b_addr + (uint32_t)((s & 1) * bunits * 16);
#pragma unroll 1
            for (int t = 0; t < kTapsPerIter; ++t) {
                const int tap = t0 + t;
                const int dz = tap / 9 - 1, dy = (tap / 3) % 3 - 1, dx = tap % 3 - 1;
                const uint64_t bd = smem_desc(bbase + (uint32_t)(t * 2 * N) * 16u, 8 * 16, kKC * 8 * 16);
#pragma unroll
                for (int zp = 0; zp < kTileZ; ++zp) {
                    const int u0 = ((zp + 1 + dz) * kHY + (1 + dy)) * kKC * kHX + (1 + dx);
                    const uint64_t ad = smem_desc(hbase + (uint32_t)u0 * 16u, kHX * 16, kKC * kHX * 16);
                    tc_mma(tmem + (uint32_t)(zp * N), ad, bd, idesc, (r == 0 && t == 0) ? 0u : 1u);
                }
            }
            tc_commit(&mbar[s & 1]);
        }
        pending[s & 1] = true;
        // the buffers of step s+1 were last read by step s-1: wait for it, then prefetch step s+1
        wait_mma((int)((s + 1) & 1));
        if (s + 1 < nsteps) load_step(s + 1);
        if (r == steps_per_tile - 1) {
            // last step of the tile: accumulators complete once step s's MMAs are
            wait_mma((int)(s & 1));
            __syncthreads();
            if (s_abort) break;
            tc_fence_after();
            int x0, y0, z0;
            tile_origin(k, x0, y0, z0);
            const int m = warp * 32 + lane;
            const int gx = x0 + (m & 7), gy = y0 + (m >> 3);
            for (int zp = 0; zp < kTileZ; ++zp) {
                const int gz = z0 + zp;
                const bool inside = gx < g.nx && gy < g.ny && gz < g.nz;
                bf16* orow =
                    out + ((size_t)((long)(inside ? gz : 0) * g.ny + (inside ? gy : 0)) * g.nx + (inside ? gx : 0)) *
                              out_stride;
                for (int c0 = 0; c0 < N; c0 += 8) {
                    float v[8];
                    tmem_ld8(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(zp * N + c0), v);
                    if (inside && c0 + 8 <= cout) {
                        __align__(16) bf16 o[8];
#pragma unroll
                        for (int e = 0; e < 8; ++e) {
                            float a = v[e] + (bias ? bias[c0 + e] : 0.f);
                            if (relu) a = fmaxf(a, 0.f);
                            o[e] = __float2bfloat16(a);
                        }
                        *reinterpret_cast<uint4*>(orow + c0) = *reinterpret_cast<const uint4*>(o);
                    }
                }
            }
            tc_fence_before();
        }
    }
    // outstanding copies and MMAs (bounded) before TMEM is released; a phase
    // whose wait gave up must be seen complete before the dealloc
    cp_async_wait_all();
    for (int b = 0; b < 2; ++b) wait_mma(b);
    for (int b = 0; b < 2; ++b)
        if (unconfirmed[b] && !mbar_drain(&mbar[b], uphase[b])) atomicMax(err, 2);
    tc_fence_before();
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(ncols) : "memory");
}

// ---------------------------------------------------------------------------
// Weight and bias gradients on the tcgen05 tensor cores.
//
// dW[t][co][ci] = sum_v x[v + off(t)][ci] dy[v][co] and dB[co] = sum_v dy[v][co]
// form one GEMM D[m][n] = sum_k A[m][k] B[n][k]: rows m = t Cin_pad + ci
// (taps x padded input channels), then one row of ones (m = R = taps
// Cin_pad) whose product is the bias gradient, further rows zero; columns n =
// output channels (N = Cout_pad); K = voxels.  A CTA takes a block of 128
// rows and a contiguous range of voxel chunks (a K split), accumulates
// D[128][N] in tensor memory over chunks of kWgK voxels (eight MMAs of K =
// 16 each, M = 128) and stores it as FP32 partial sums; k_wgrad_reduce adds
// the splits in a fixed order, so no atomics are involved.  The operands
// arrive channels-last, so staging transposes them into the canonical K-major
// layout without swizzling (a core matrix is 8 rows of 16 bytes: 8 voxels of
// one row): a thread loads the 16-byte 8-channel groups of 8 voxels and
// stores eight 16-byte core-matrix rows, one per channel, after an 8 x 8
// transpose in registers.  Core matrices of consecutive row groups are
// kWgSbo = 272 bytes apart (not 256), so the eight threads of a store phase
// hit different bank groups.  Chunks are double-buffered: the MMAs of one
// chunk run while the next one is staged.  Waits are bounded and tensor
// memory is released under the same rules as in k_conv_tc.
// ---------------------------------------------------------------------------
constexpr int kWgK = 128;        // voxels per chunk
constexpr int kWgThreads = 128;
constexpr int kWgSbo = 272;      // bytes between the core matrices of consecutive 8-row groups
constexpr int kWgAStep = 16 * kWgSbo;   // bytes of one K = 16 step of A (16 row groups)
constexpr int kWgABytes = (kWgK / 16) * kWgAStep;
constexpr int kWgMaxCtas = 304;  // row blocks x splits of a launch (about two per SM)

__host__ __device__ constexpr int wg_bstep(int N) { return (N / 8) * kWgSbo; }
__host__ __device__ constexpr int wg_buf_bytes(int N) { return kWgABytes + (kWgK / 16) * wg_bstep(N); }

// 8 x 8 transpose of BF16 values: in[e] holds channels 0..7 of voxel e, out[j]
// voxels 0..7 of channel j (element i of a 16-byte group in bytes 2i, 2i+1)
__device__ __forceinline__ void transpose8(const uint4* in, uint4* out) {
    const uint32_t* w = reinterpret_cast<const uint32_t*>(in);  // w[4 e + k]: channels 2k (low), 2k+1 of voxel e
    uint32_t* o = reinterpret_cast<uint32_t*>(out);              // o[4 j + m]: voxels 2m (low), 2m+1 of channel j
#pragma unroll
    for (int k = 0; k < 4; ++k)
#pragma unroll
        for (int m = 0; m < 4; ++m) {
            const uint32_t a = w[4 * (2 * m) + k], b = w[4 * (2 * m + 1) + k];
            o[4 * (2 * k) + m] = __byte_perm(a, b, 0x5410);
            o[4 * (2 * k + 1) + m] = __byte_perm(a, b, 0x7632);
        }
}

// Partial GEMM of row block blockIdx.x over voxel chunks [blockIdx.y cps,
// (blockIdx.y + 1) cps) into part[(split nrb + rb) 128 + row][N] (FP32).
// x: [voxel][cin_pad], dy: [voxel][N]; N a multiple of 16 in [16, 128].
__global__ void __launch_bounds__(kWgThreads) k_wgrad_tc(CG g, const bf16* __restrict__ x, int cin_pad, int ntaps,
                                                         const bf16* __restrict__ dy, int N, int cps,
                                                         float* __restrict__ part, int ncols, int* err) {
    extern __shared__ __align__(1024) unsigned char smem[];
    __shared__ __align__(8) uint64_t mbar[2];
    __shared__ uint32_t s_tmem;
    __shared__ int s_abort;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int rb = blockIdx.x, nrb = gridDim.x;
    const int bstep = wg_bstep(N), bufb = wg_buf_bytes(N);

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&s_tmem)),
                     "r"(ncols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        mbar_init(&mbar[0], 1);
        mbar_init(&mbar[1], 1);
        s_abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = s_tmem;
    const uint32_t idesc = idesc_bf16(128, N);

    const int R = ntaps * cin_pad;  // weight rows; row R is the row of ones
    const int nchunks = (g.N + kWgK - 1) / kWgK;
    const int ch0 = blockIdx.y * cps, nch = max(0, min(ch0 + cps, nchunks) - ch0);
    uint32_t phase[2] = {0u, 0u};
    bool pending[2] = {false, false};
    bool unconfirmed[2] = {false, false};
    uint32_t uphase[2] = {0u, 0u};
    auto wait_mma = [&](int b) {
        if (pending[b]) {
            if (!mbar_wait_bounded(&mbar[b], phase[b])) {
                s_abort = 1;
                atomicExch(err, 1);
                unconfirmed[b] = true;
                uphase[b] = phase[b];
            }
            phase[b] ^= 1u;
            pending[b] = false;
        }
    };
    const uint4 zero4 = make_uint4(0u, 0u, 0u, 0u);
    // stage chunk ch0 + c into buffer b
    auto stage = [&](int c, int b) {
        unsigned char* A = smem + b * bufb;
        unsigned char* B = A + kWgABytes;
        const int vbase = (ch0 + c) * kWgK;
        // A: 16 row groups x kWgK / 8 voxel octets (consecutive threads: consecutive row groups)
        for (int u = tid; u < 16 * (kWgK / 8); u += kWgThreads) {
            const int gq = u & 15, o = u >> 4;
            const int row0 = rb * 128 + gq * 8;
            uint4 in[8];
            if (row0 < R) {
                const int tap = row0 / cin_pad, ci0 = row0 - tap * cin_pad;
                int dz, dyy, dx;
                tap_off(tap, ntaps, dz, dyy, dx);
#pragma unroll
                for (int e = 0; e < 8; ++e) {
                    const int n = nbr(g, vox(g, vbase + 8 * o + e), dz, dyy, dx);
                    in[e] = n >= 0 ? __ldg(reinterpret_cast<const uint4*>(x + (size_t)n * cin_pad + ci0)) : zero4;
                }
            } else {
                // the row of ones (channel 0 of the group starting at row R), then zeros
#pragma unroll
                for (int e = 0; e < 8; ++e) {
                    in[e] = zero4;
                    if (row0 == R && vbase + 8 * o + e < g.N) in[e].x = 0x3F80u;  // BF16 1.0 in element 0
                }
            }
            uint4 out[8];
            transpose8(in, out);
            unsigned char* dst = A + (o >> 1) * kWgAStep + gq * kWgSbo + (o & 1) * 128;
#pragma unroll
            for (int j = 0; j < 8; ++j) *reinterpret_cast<uint4*>(dst + j * 16) = out[j];
        }
        // B: N / 8 column groups x kWgK / 8 voxel octets
        const int ng = N >> 3;
        for (int u = tid; u < ng * (kWgK / 8); u += kWgThreads) {
            const int gq = u % ng, o = u / ng;
            uint4 in[8];
#pragma unroll
            for (int e = 0; e < 8; ++e) {
                const int v = vbase + 8 * o + e;
                in[e] = v < g.N ? __ldg(reinterpret_cast<const uint4*>(dy + (size_t)v * N + gq * 8)) : zero4;
            }
            uint4 out[8];
            transpose8(in, out);
            unsigned char* dst = B + (o >> 1) * bstep + gq * kWgSbo + (o & 1) * 128;
#pragma unroll
            for (int j = 0; j < 8; ++j) *reinterpret_cast<uint4*>(dst + j * 16) = out[j];
        }
    };

    for (int c = 0; c < nch; ++c) {
        const int b = c & 1;
        wait_mma(b);  // the MMAs of chunk c - 2 read this buffer
        stage(c, b);
        fence_proxy_async();
        __syncthreads();
        if (s_abort) break;
        if (tid == 0) {
            tc_fence_after();
            const uint32_t a0 = smem_u32(smem + b * bufb), b0 = a0 + kWgABytes;
#pragma unroll
            for (int q = 0; q < kWgK / 16; ++q) {
                const uint64_t ad = smem_desc(a0 + (uint32_t)(q * kWgAStep), 128, kWgSbo);
                const uint64_t bd = smem_desc(b0 + (uint32_t)(q * bstep), 128, kWgSbo);
                tc_mma(tmem, ad, bd, idesc, (c == 0 && q == 0) ? 0u : 1u);
            }
            tc_commit(&mbar[b]);
        }
        pending[b] = true;
    }
    for (int b = 0; b < 2; ++b) wait_mma(b);
    __syncthreads();
    if (!s_abort && nch > 0) {
        tc_fence_after();
        const int row = warp * 32 + lane;
        float* dst = part + ((size_t)(blockIdx.y * nrb + rb) * 128 + row) * N;
        for (int c0 = 0; c0 < N; c0 += 8) {
            float v[8];
            tmem_ld8(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, v);
            *reinterpret_cast<float4*>(dst + c0) = make_float4(v[0], v[1], v[2], v[3]);
            *reinterpret_cast<float4*>(dst + c0 + 4) = make_float4(v[4], v[5], v[6], v[7]);
        }
    }
    // a phase whose wait gave up must be seen complete before the dealloc
    for (int b = 0; b < 2; ++b)
        if (unconfirmed[b] && !mbar_drain(&mbar[b], uphase[b])) atomicMax(err, 2);
    tc_fence_before();
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(ncols) : "memory");
}

// dW[t][co][ci] (ci < cin, co < cout) and dB[co] from the partial sums of the
// nsplit voxel splits, added in split order
__global__ void k_wgrad_reduce(const float* __restrict__ part, int nsplit, int nrb, int N, int ntaps, int cin_pad,
                               int cin, int cout, float* __restrict__ dW, float* __restrict__ dB) {
    const long t = (long)blockIdx.x * blockDim.x + threadIdx.x;
    const int R = ntaps * cin_pad;
    if (t >= (long)(R + 1) * cout) return;
    const int n = (int)(t % cout);
    const int m = (int)(t / cout);  // row, 0 .. R
    const int rb = m >> 7, row = m & 127;
    float s = 0.f;
    for (int k = 0; k < nsplit; ++k) s += part[((size_t)(k * nrb + rb) * 128 + row) * N + n];
    if (m == R) {
        dB[n] = s;
        return;
    }
    const int tap = m / cin_pad, ci = m - tap * cin_pad;
    if (ci < cin) dW[((size_t)tap * cout + n) * cin + ci] = s;
}

}  // namespace
}  // namespace cdi

using namespace cdi;

struct cdi_unet {
    int n[3] = {0, 0, 0};
    CG g[4];  // levels 0..3
    char* ws = nullptr;
    size_t ws_bytes = 0;
    cudaStream_t stream = nullptr;
    // parameters
    float *W[kLayers], *B[kLayers], *gW[kLayers], *gB[kLayers];
    float *mW[kLayers], *vW[kLayers], *mB[kLayers], *vB[kLayers];
    bf16 *Wb[kLayers], *Wt[kLayers];
    int ci_pad[kLayers], co_pad[kLayers];
    // activations and gradients (BF16, channels last)
    bf16 *x, *e0, *p0, *e1, *p1, *e2, *p2, *b, *c2, *d2, *c1, *d1, *c0, *d0;
    bf16 *gy, *gd0, *gc0, *gd1, *gc1, *gd2, *gc2, *gb, *gp2, *ge2, *gp1, *ge1, *gp0, *ge0;
    float *y, *t, *part;
    float* wpart;  // FP32 partial sums of the tcgen05 weight gradients (voxel splits x rows x columns)
    double* x2;  // host-input staging [N][2]
    double* sd;  // prediction scales (FP64 and FP32 copies)
    float* sf;
    int* tc_err;          // set by a tcgen05 convolution whose bounded wait ran out
    bool use_tc = true;   // 3x3x3 convolutions on tcgen05 (else mma.sync)
    bool wgrad_tc = true; // weight and bias gradients on tcgen05 (else mma.sync with FP32 atomics)
    long adam_t = 0;
    bool weights_ready = false;
    std::string err;
};

namespace {

std::string g_unet_error;

cdi_status ufail(cdi_unet* u, cdi_status st, const std::string& m) {
    if (u) u->err = m;
    else g_unet_error = m;
    return st;
}

struct UCarver {
    char* base;
    size_t off = 0;
    void* take(size_t bytes) {
        off = (off + 255) & ~size_t(255);
        void* p = base ? base + off : nullptr;
        off += bytes;
        return p;
    }
};

// level of the grid each layer works on (e0 e1 e2 b d2 d1 d0 head)
constexpr int kLevelOf[kLayers] = {0, 1, 2, 3, 2, 1, 0, 0};

// work split of the tcgen05 weight gradient of one layer: row blocks of 128
// (taps x padded input channels, plus the row of ones), voxel splits of cps
// chunks each (every split holds at least one chunk), about kWgMaxCtas CTAs
struct WgPlan {
    int nrb, nsplit, cps;
};
WgPlan wg_plan(int l, long nvox, int ci_pad) {
    WgPlan p;
    p.nrb = (kTaps[l] * ci_pad + 1 + 127) / 128;
    const int nchunks = (int)std::max(1L, (nvox + kWgK - 1) / kWgK);
    const int s = std::max(1, std::min(nchunks, (kWgMaxCtas + p.nrb - 1) / p.nrb));
    p.cps = (nchunks + s - 1) / s;
    p.nsplit = (nchunks + p.cps - 1) / p.cps;
    return p;
}

void unet_carve(cdi_unet* u, char* base, size_t* total) {
    UCarver cv{base};
    for (int l = 0; l < kLayers; ++l) {
        const size_t nw = (size_t)kTaps[l] * kCout[l] * kCin[l], nb = kCout[l];
        u->ci_pad[l] = pad16(kCin[l]);
        u->co_pad[l] = pad16(kCout[l]);
        u->W[l] = (float*)cv.take(nw * 4);
        u->B[l] = (float*)cv.take(nb * 4);
        u->gW[l] = (float*)cv.take(nw * 4);
        u->gB[l] = (float*)cv.take(nb * 4);
        u->mW[l] = (float*)cv.take(nw * 4);
        u->vW[l] = (float*)cv.take(nw * 4);
        u->mB[l] = (float*)cv.take(nb * 4);
        u->vB[l] = (float*)cv.take(nb * 4);
        const size_t np = (size_t)kTaps[l] * u->ci_pad[l] * u->co_pad[l];
        u->Wb[l] = (bf16*)cv.take(np * 2);
        u->Wt[l] = (bf16*)cv.take(np * 2);
    }
    const long N0 = u->g[0].N, N1 = u->g[1].N, N2 = u->g[2].N, N3 = u->g[3].N;
    auto act = [&](long n, int c) { return (bf16*)cv.take((size_t)n * c * 2); };
    u->x = act(N0, 16);
    u->e0 = act(N0, 16);
    u->p0 = act(N1, 16);
    u->e1 = act(N1, 32);
    u->p1 = act(N2, 32);
    u->e2 = act(N2, 64);
    u->p2 = act(N3, 64);
    u->b = act(N3, 128);
    u->c2 = act(N2, 192);
    u->d2 = act(N2, 64);
    u->c1 = act(N1, 96);
    u->d1 = act(N1, 32);
    u->c0 = act(N0, 48);
    u->d0 = act(N0, 16);
    u->gy = act(N0, 16);
    u->gd0 = act(N0, 16);
    u->gc0 = act(N0, 48);
    u->gd1 = act(N1, 32);
    u->gc1 = act(N1, 96);
    u->gd2 = act(N2, 64);
    u->gc2 = act(N2, 192);
    u->gb = act(N3, 128);
    u->gp2 = act(N3, 64);
    u->ge2 = act(N2, 64);
    u->gp1 = act(N2, 32);
    u->ge1 = act(N1, 32);
    u->gp0 = act(N1, 16);
    u->ge0 = act(N0, 16);
    u->y = (float*)cv.take((size_t)N0 * 4);
    u->t = (float*)cv.take((size_t)N0 * 4);
    u->part = (float*)cv.take(256);
    size_t wp = 0;
    for (int l = 0; l < kLayers; ++l) {
        const WgPlan p = wg_plan(l, u->g[kLevelOf[l]].N, pad16(kCin[l]));
        wp = std::max(wp, (size_t)p.nsplit * p.nrb * 128 * pad16(kCout[l]));
    }
    u->wpart = (float*)cv.take(wp * 4);
    u->sd = (double*)cv.take(4 * sizeof(double));
    u->sf = (float*)cv.take(4 * sizeof(float));
    u->tc_err = (int*)cv.take(sizeof(int));
    u->x2 = (double*)cv.take((size_t)N0 * 2 * 8);
    *total = cv.off + 256;
}

// tcgen05 convolution launch: a persistent grid of as many CTAs as fit at once (shared memory
// bounds the CTAs per SM below what the TMEM columns allow, so no TMEM allocation ever waits)
void conv_tc(cdi_unet* u, const CG& gl, const bf16* in, int cin, const bf16* w, int N, const float* bias, int cout,
             bf16* out, int out_stride, bool relu, const bf16* up = nullptr, int cup = 0) {
    static int nsm = 0, smem_sm = 0;
    static bool attr = false;
    const int ncols = 2 * N <= 32 ? 32 : 2 * N <= 64 ? 64 : 2 * N <= 128 ? 128 : 2 * N <= 256 ? 256 : 512;
    const size_t smem = 2 * (size_t)kHaloBytes + kGuardBytes + 2 * (size_t)kTapsPerIter * 2 * N * 16;
    if (!attr) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
        cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
        cudaFuncSetAttribute(k_conv_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
        cudaFuncSetAttribute(k_conv_tc, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
        attr = true;
    }
    // CTAs per SM: shared memory (1 KB reserved per CTA, plus the static 1 KB), threads, TMEM columns
    int per = (int)((size_t)smem_sm / (smem + 2048));
    per = std::max(1, std::min({per, 2048 / kTcThreads, 512 / ncols}));
    const long tiles = (long)((gl.nx + kTileX - 1) / kTileX) * ((gl.ny + kTileY - 1) / kTileY) *
                       ((gl.nz + kTileZ - 1) / kTileZ);
    const unsigned grid = (unsigned)std::max(1L, std::min(tiles, (long)nsm * per));
    k_conv_tc<<<grid, kTcThreads, smem, u->stream>>>(gl, in, cin, up, cup, w, N, bias, cout, out, out_stride,
                                                     relu ? 1 : 0, ncols, u->tc_err);
}

// y = conv(in) for layer l on level grid gl into out (stride, offset)
template <bool OUTF32>
void conv_fwd(cdi_unet* u, int l, const CG& gl, const bf16* in, void* out, int stride, int off, bool relu) {
    if (!OUTF32 && kTaps[l] == 27 && u->use_tc && off == 0 && stride == u->co_pad[l]) {
        conv_tc(u, gl, in, u->ci_pad[l], u->Wb[l], u->co_pad[l], u->B[l], u->co_pad[l], (bf16*)out, stride, relu);
        return;
    }
    const unsigned gb = (unsigned)((gl.N + 63) / 64);
    const int nf = u->co_pad[l] / 8;
    const int cin = u->ci_pad[l], cop = u->co_pad[l];
    cudaStream_t s = u->stream;
#define CONV_CASE(NFV)                                                                                          \
    case NFV:                                                                                                   \
        k_conv<NFV, OUTF32><<<gb, 128, 0, s>>>(gl, in, cin, u->Wb[l], cop, u->B[l], kCout[l], out, stride, off, \
                                                relu ? 1 : 0, kTaps[l]);                                        \
        break;
    switch (nf) {
        CONV_CASE(2)
        CONV_CASE(4)
        CONV_CASE(8)
        CONV_CASE(16)
        default: break;
    }
#undef CONV_CASE
}

// dx (BF16 [N][ci_pad]) = adjoint of layer l applied to dy (BF16 [N][co_pad])
void conv_dgrad(cdi_unet* u, int l, const CG& gl, const bf16* dy, bf16* dx) {
    if (kTaps[l] == 27 && u->use_tc) {
        conv_tc(u, gl, dy, u->co_pad[l], u->Wt[l], u->ci_pad[l], nullptr, u->ci_pad[l], dx, u->ci_pad[l], false);
        return;
    }
    const unsigned gb = (unsigned)((gl.N + 63) / 64);
    const int nf = u->ci_pad[l] / 8;
    cudaStream_t s = u->stream;
#define DG_CASE(NFV)                                                                                              \
    case NFV:                                                                                                     \
        k_conv<NFV, false><<<gb, 128, 0, s>>>(gl, dy, u->co_pad[l], u->Wt[l], u->ci_pad[l], nullptr,             \
                                               u->ci_pad[l], dx, u->ci_pad[l], 0, 0, kTaps[l]);                   \
        break;
    switch (nf) {
        DG_CASE(2)
        DG_CASE(4)
        DG_CASE(6)
        DG_CASE(8)
        DG_CASE(12)
        DG_CASE(24)
        default: break;
    }
#undef DG_CASE
}

// weight and bias gradients of layer l on the tcgen05 tensor cores (no atomics)
void wgrad_tc(cdi_unet* u, int l, const CG& gl, const bf16* in, const bf16* dy) {
    static bool attr = false;
    if (!attr) {
        cudaFuncSetAttribute(k_wgrad_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, 2 * wg_buf_bytes(128));
        attr = true;
    }
    const int N = u->co_pad[l];
    const WgPlan p = wg_plan(l, gl.N, u->ci_pad[l]);
    const int ncols = N <= 32 ? 32 : N <= 64 ? 64 : 128;
    k_wgrad_tc<<<dim3((unsigned)p.nrb, (unsigned)p.nsplit), kWgThreads, 2 * (size_t)wg_buf_bytes(N), u->stream>>>(
        gl, in, u->ci_pad[l], kTaps[l], dy, N, p.cps, u->wpart, ncols, u->tc_err);
    const long nt = (long)(kTaps[l] * u->ci_pad[l] + 1) * kCout[l];
    k_wgrad_reduce<<<blocks(nt), 256, 0, u->stream>>>(u->wpart, p.nsplit, p.nrb, N, kTaps[l], u->ci_pad[l], kCin[l],
                                                      kCout[l], u->gW[l], u->gB[l]);
}

void conv_wgrad(cdi_unet* u, int l, const CG& gl, const bf16* in, const bf16* dy) {
    if (u->wgrad_tc) {
        wgrad_tc(u, l, gl, in, dy);
        return;
    }
    const int chunk = 1024;
    dim3 grid((unsigned)kTaps[l], (unsigned)((u->co_pad[l] + 15) / 16), (unsigned)((gl.N + chunk - 1) / chunk));
    const int nf = u->ci_pad[l] / 8;
    cudaStream_t s = u->stream;
#define WG_CASE(NFV)                                                                                                \
    case NFV:                                                                                                       \
        k_wgrad<NFV><<<grid, 128, 0, s>>>(gl, in, u->ci_pad[l], dy, u->co_pad[l], u->gW[l], kCout[l], kCin[l],     \
                                           kTaps[l], chunk);                                                        \
        break;
    switch (nf) {
        WG_CASE(2)
        WG_CASE(4)
        WG_CASE(6)
        WG_CASE(8)
        WG_CASE(12)
        WG_CASE(24)
        default: break;
    }
#undef WG_CASE
    k_bias_grad<<<dim3(64, (unsigned)kCout[l]), 256, 0, s>>>(gl.N, dy, u->co_pad[l], kCout[l], u->gB[l]);
}

void refresh_weights(cdi_unet* u) {
    for (int l = 0; l < kLayers; ++l) {
        const long n = (long)kTaps[l] * u->co_pad[l] * u->ci_pad[l];
        k_weights_bf16<<<blocks(n), 256, 0, u->stream>>>(u->W[l], kTaps[l], kCout[l], kCin[l], u->co_pad[l],
                                                          u->ci_pad[l], u->Wb[l], u->Wt[l]);
    }
    u->weights_ready = true;
}

// forward pass from u->x to u->y (FP32).  With keep_concat the decoder inputs
// [up(coarser), skip] are stored (the weight gradients read them); otherwise the
// tcgen05 convolution gathers them while staging its input tiles.
void forward(cdi_unet* u, bool keep_concat = true) {
    const CG* g = u->g;
    cudaStream_t s = u->stream;
    const bool fuse = !keep_concat && u->use_tc;
    conv_fwd<false>(u, 0, g[0], u->x, u->e0, 16, 0, true);
    k_pool<<<blocks(g[1].N * 2L), 256, 0, s>>>(g[0], u->e0, 16, u->p0);
    conv_fwd<false>(u, 1, g[1], u->p0, u->e1, 32, 0, true);
    k_pool<<<blocks(g[2].N * 4L), 256, 0, s>>>(g[1], u->e1, 32, u->p1);
    conv_fwd<false>(u, 2, g[2], u->p1, u->e2, 64, 0, true);
    k_pool<<<blocks(g[3].N * 8L), 256, 0, s>>>(g[2], u->e2, 64, u->p2);
    conv_fwd<false>(u, 3, g[3], u->p2, u->b, 128, 0, true);
    g_launches += 7;
    if (fuse) {
        conv_tc(u, g[2], u->e2, 192, u->Wb[4], 64, u->B[4], 64, u->d2, 64, true, u->b, 128);
        conv_tc(u, g[1], u->e1, 96, u->Wb[5], 32, u->B[5], 32, u->d1, 32, true, u->d2, 64);
        conv_tc(u, g[0], u->e0, 48, u->Wb[6], 16, u->B[6], 16, u->d0, 16, true, u->d1, 32);
        g_launches += 3;
    } else {
        k_up<<<blocks(g[2].N * 16L), 256, 0, s>>>(g[2], u->b, 128, u->c2, 192, 0);
        k_copy_ch<<<blocks(g[2].N * 8L), 256, 0, s>>>(g[2].N, u->e2, 64, 0, u->c2, 192, 128, 64);
        conv_fwd<false>(u, 4, g[2], u->c2, u->d2, 64, 0, true);
        k_up<<<blocks(g[1].N * 8L), 256, 0, s>>>(g[1], u->d2, 64, u->c1, 96, 0);
        k_copy_ch<<<blocks(g[1].N * 4L), 256, 0, s>>>(g[1].N, u->e1, 32, 0, u->c1, 96, 64, 32);
        conv_fwd<false>(u, 5, g[1], u->c1, u->d1, 32, 0, true);
        k_up<<<blocks(g[0].N * 4L), 256, 0, s>>>(g[0], u->d1, 32, u->c0, 48, 0);
        k_copy_ch<<<blocks(g[0].N * 2L), 256, 0, s>>>(g[0].N, u->e0, 16, 0, u->c0, 48, 32, 16);
        conv_fwd<false>(u, 6, g[0], u->c0, u->d0, 16, 0, true);
        g_launches += 9;
    }
    conv_fwd<true>(u, 7, g[0], u->d0, u->y, 1, 0, false);
    g_launches += 1;
}

// gradients of the mean squared error (u->y against u->t) into gW, gB
void backward(cdi_unet* u) {
    const CG* g = u->g;
    cudaStream_t s = u->stream;
    for (int l = 0; l < kLayers; ++l) {
        cudaMemsetAsync(u->gW[l], 0, (size_t)kTaps[l] * kCout[l] * kCin[l] * 4, s);
        cudaMemsetAsync(u->gB[l], 0, (size_t)kCout[l] * 4, s);
    }
    cudaMemsetAsync(u->gy, 0, (size_t)g[0].N * 16 * 2, s);
    cudaMemsetAsync(u->part, 0, 4, s);
    k_loss<<<256, 256, 0, s>>>(g[0].N, u->y, u->t, u->gy, u->part);
    // head and d0
    conv_wgrad(u, 7, g[0], u->d0, u->gy);
    conv_dgrad(u, 7, g[0], u->gy, u->gd0);
    k_relu_mask<<<blocks(g[0].N * 16L), 256, 0, s>>>(g[0].N * 16L, u->gd0, u->d0);
    conv_wgrad(u, 6, g[0], u->c0, u->gd0);
    conv_dgrad(u, 6, g[0], u->gd0, u->gc0);
    k_up_bwd<<<blocks(g[1].N * 32L), 256, 0, s>>>(g[0], u->gc0, 48, 0, 32, u->gd1);
    k_relu_mask<<<blocks(g[1].N * 32L), 256, 0, s>>>(g[1].N * 32L, u->gd1, u->d1);
    k_copy_ch<<<blocks(g[0].N * 2L), 256, 0, s>>>(g[0].N, u->gc0, 48, 32, u->ge0, 16, 0, 16);
    // d1
    conv_wgrad(u, 5, g[1], u->c1, u->gd1);
    conv_dgrad(u, 5, g[1], u->gd1, u->gc1);
    k_up_bwd<<<blocks(g[2].N * 64L), 256, 0, s>>>(g[1], u->gc1, 96, 0, 64, u->gd2);
    k_relu_mask<<<blocks(g[2].N * 64L), 256, 0, s>>>(g[2].N * 64L, u->gd2, u->d2);
    k_copy_ch<<<blocks(g[1].N * 4L), 256, 0, s>>>(g[1].N, u->gc1, 96, 64, u->ge1, 32, 0, 32);
    // d2
    conv_wgrad(u, 4, g[2], u->c2, u->gd2);
    conv_dgrad(u, 4, g[2], u->gd2, u->gc2);
    k_up_bwd<<<blocks(g[3].N * 128L), 256, 0, s>>>(g[2], u->gc2, 192, 0, 128, u->gb);
    k_relu_mask<<<blocks(g[3].N * 128L), 256, 0, s>>>(g[3].N * 128L, u->gb, u->b);
    k_copy_ch<<<blocks(g[2].N * 8L), 256, 0, s>>>(g[2].N, u->gc2, 192, 128, u->ge2, 64, 0, 64);
    // bottleneck
    conv_wgrad(u, 3, g[3], u->p2, u->gb);
    conv_dgrad(u, 3, g[3], u->gb, u->gp2);
    k_pool_bwd_add<<<blocks(g[2].N * 64L), 256, 0, s>>>(g[2], u->gp2, 64, u->ge2, 64, 0);
    k_relu_mask<<<blocks(g[2].N * 64L), 256, 0, s>>>(g[2].N * 64L, u->ge2, u->e2);
    // e2
    conv_wgrad(u, 2, g[2], u->p1, u->ge2);
    conv_dgrad(u, 2, g[2], u->ge2, u->gp1);
    k_pool_bwd_add<<<blocks(g[1].N * 32L), 256, 0, s>>>(g[1], u->gp1, 32, u->ge1, 32, 0);
    k_relu_mask<<<blocks(g[1].N * 32L), 256, 0, s>>>(g[1].N * 32L, u->ge1, u->e1);
    // e1
    conv_wgrad(u, 1, g[1], u->p0, u->ge1);
    conv_dgrad(u, 1, g[1], u->ge1, u->gp0);
    k_pool_bwd_add<<<blocks(g[0].N * 16L), 256, 0, s>>>(g[0], u->gp0, 16, u->ge0, 16, 0);
    k_relu_mask<<<blocks(g[0].N * 16L), 256, 0, s>>>(g[0].N * 16L, u->ge0, u->e0);
    // e0
    conv_wgrad(u, 0, g[0], u->x, u->ge0);
    g_launches += 50;
}

void adam(cdi_unet* u, double lr) {
    ++u->adam_t;
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    const float bc1 = (float)(1.0 - std::pow(0.9, (double)u->adam_t));
    const float bc2 = (float)(1.0 - std::pow(0.999, (double)u->adam_t));
    for (int l = 0; l < kLayers; ++l) {
        const long nw = (long)kTaps[l] * kCout[l] * kCin[l];
        k_adam<<<blocks(nw), 256, 0, u->stream>>>(nw, u->W[l], u->gW[l], u->mW[l], u->vW[l], (float)lr, b1, b2, eps,
                                                   bc1, bc2);
        k_adam<<<blocks(kCout[l]), 256, 0, u->stream>>>(kCout[l], u->B[l], u->gB[l], u->mB[l], u->vB[l], (float)lr,
                                                         b1, b2, eps, bc1, bc2);
    }
    refresh_weights(u);
}

size_t param_count() {
    size_t n = 0;
    for (int l = 0; l < kLayers; ++l) n += (size_t)kTaps[l] * kCout[l] * kCin[l] + kCout[l];
    return n;
}

// after a synchronisation: did a tcgen05 convolution give up on a wait?
cdi_status check_tc(cdi_unet* u) {
    int e = 0;
    if (cudaMemcpy(&e, u->tc_err, sizeof e, cudaMemcpyDeviceToHost) != cudaSuccess)
        return ufail(u, CDI_ECUDA, "error flag read failed");
    if (e) {
        cudaMemset(u->tc_err, 0, sizeof(int));
        return ufail(u, CDI_ETIMEOUT,
                     e == 1 ? "a tensor-core convolution timed out waiting for its MMAs"
                            : "a tensor-core convolution released tensor memory with an MMA still unconfirmed "
                              "after its waits ran out: treat the device state as unknown");
    }
    return CDI_OK;
}

cdi_status upload_x(cdi_unet* u, const double* x_host) {
    const long N = u->g[0].N;
    if (cudaMemcpyAsync(u->x2, x_host, (size_t)N * 2 * 8, cudaMemcpyHostToDevice, u->stream) != cudaSuccess)
        return ufail(u, CDI_ECUDA, "input upload failed");
    k_input_host<<<blocks(N * 16), 256, 0, u->stream>>>((int)N, u->x2, u->x);
    return CDI_OK;
}

}  // namespace

namespace cdi {

template <typename T>
cudaError_t unet_predict_device(cdi_unet* u, const MG& mg, const T* phi_dev, double rho1, double rho2, double h,
                                cudaStream_t s) {
    cudaStream_t keep = u->stream;
    u->stream = s;
    if (!u->weights_ready) refresh_weights(u);
    const long N = u->g[0].N;
    const double rmax = fmax(rho1, rho2);
    k_solver_scales<<<1, 1, 0, s>>>(mg.scal + S_FNORM, (int)N, rmax * h * h, u->sd, u->sf);
    k_input_solver<T><<<blocks(N * 16), 256, 0, s>>>((int)N, ops::fbuf<T>(mg.lv[0]), mg.scalf + SF_FMEAN_HI,
                                                     phi_dev, (float)(rho1 - rho2), (float)rho2, (float)(1.0 / rmax),
                                                     u->sd, u->sf, u->x);
    forward(u, false);
    k_output_solver<T><<<blocks(N), 256, 0, s>>>((int)N, u->y, u->sd, u->sf, ops::pbuf<T>(mg.lv[0]));
    g_launches += 3;
    u->stream = keep;
    return cudaGetLastError();
}

void unet_extents(const cdi_unet* u, int* n) {
    n[0] = u->n[0];
    n[1] = u->n[1];
    n[2] = u->n[2];
}

template cudaError_t unet_predict_device<double>(cdi_unet*, const MG&, const double*, double, double, double,
                                                 cudaStream_t);
template cudaError_t unet_predict_device<float>(cdi_unet*, const MG&, const float*, double, double, double,
                                                cudaStream_t);

}  // namespace cdi

extern "C" {

cdi_status cdi_unet_create(cdi_unet** out, int nx, int ny, int nz) {
    if (!out) return ufail(nullptr, CDI_EINVAL, "out is NULL");
    *out = nullptr;
    if (nx < 8 || ny < 8 || nz < 8 || nx % 8 || ny % 8 || nz % 8)
        return ufail(nullptr, CDI_EINVAL, "network extents must be multiples of 8 (three 2x2x2 poolings)");
    if ((long)nx * ny * nz > (1L << 28)) return ufail(nullptr, CDI_EINVAL, "grid too large for the network");
    cdi_unet* u = new (std::nothrow) cdi_unet();
    if (!u) return ufail(nullptr, CDI_EINVAL, "out of host memory");
    u->n[0] = nx;
    u->n[1] = ny;
    u->n[2] = nz;
    for (int l = 0; l < 4; ++l) {
        u->g[l].nx = nx >> l;
        u->g[l].ny = ny >> l;
        u->g[l].nz = nz >> l;
        u->g[l].N = u->g[l].nx * u->g[l].ny * u->g[l].nz;
    }
    size_t total = 0;
    unet_carve(u, nullptr, &total);
    u->ws_bytes = total;
    *out = u;
    return CDI_OK;
}

cdi_status cdi_unet_workspace_bytes(const cdi_unet* u, size_t* bytes) {
    if (!u || !bytes) return ufail(nullptr, CDI_EINVAL, "null argument");
    *bytes = u->ws_bytes;
    return CDI_OK;
}

cdi_status cdi_unet_bind_workspace(cdi_unet* u, void* dev_ptr, size_t bytes, void* stream) {
    if (!u) return ufail(nullptr, CDI_EINVAL, "null network");
    if (!dev_ptr || bytes < u->ws_bytes) return ufail(u, CDI_EINVAL, "workspace missing or too small");
    if (((uintptr_t)dev_ptr) & 255u) return ufail(u, CDI_EINVAL, "workspace must be 256-byte aligned");
    u->ws = (char*)dev_ptr;
    u->stream = (cudaStream_t)stream;
    size_t total = 0;
    unet_carve(u, u->ws, &total);
    if (cudaMemsetAsync(u->ws, 0, u->ws_bytes - 256, u->stream) != cudaSuccess ||
        cudaStreamSynchronize(u->stream) != cudaSuccess)
        return ufail(u, CDI_ECUDA, "workspace clear failed");
    u->adam_t = 0;
    u->weights_ready = false;
    return CDI_OK;
}

cdi_status cdi_unet_param_count(size_t* n) {
    if (!n) return ufail(nullptr, CDI_EINVAL, "null argument");
    *n = param_count();
    return CDI_OK;
}

// flat parameter order: for each layer (e0, e1, e2, b, d2, d1, d0, head) the
// weights [taps][Cout][Cin] then the biases [Cout]
cdi_status cdi_unet_set_params(cdi_unet* u, const double* host, size_t n) {
    if (!u || !u->ws) return ufail(u, CDI_ESTATE, "network workspace not bound");
    if (!host || n != param_count()) return ufail(u, CDI_EINVAL, "parameter array has the wrong length");
    std::vector<float> tmp(host, host + n);
    size_t o = 0;
    for (int l = 0; l < kLayers; ++l) {
        const size_t nw = (size_t)kTaps[l] * kCout[l] * kCin[l];
        cudaMemcpyAsync(u->W[l], tmp.data() + o, nw * 4, cudaMemcpyHostToDevice, u->stream);
        o += nw;
        cudaMemcpyAsync(u->B[l], tmp.data() + o, (size_t)kCout[l] * 4, cudaMemcpyHostToDevice, u->stream);
        o += kCout[l];
        cudaMemsetAsync(u->mW[l], 0, nw * 4, u->stream);
        cudaMemsetAsync(u->vW[l], 0, nw * 4, u->stream);
        cudaMemsetAsync(u->mB[l], 0, (size_t)kCout[l] * 4, u->stream);
        cudaMemsetAsync(u->vB[l], 0, (size_t)kCout[l] * 4, u->stream);
    }
    u->adam_t = 0;
    refresh_weights(u);
    if (cudaStreamSynchronize(u->stream) != cudaSuccess) return ufail(u, CDI_ECUDA, "parameter upload failed");
    return CDI_OK;
}

cdi_status cdi_unet_get_params(cdi_unet* u, double* host, size_t n) {
    if (!u || !u->ws) return ufail(u, CDI_ESTATE, "network workspace not bound");
    if (!host || n != param_count()) return ufail(u, CDI_EINVAL, "parameter array has the wrong length");
    std::vector<float> tmp(n);
    size_t o = 0;
    for (int l = 0; l < kLayers; ++l) {
        const size_t nw = (size_t)kTaps[l] * kCout[l] * kCin[l];
        cudaMemcpyAsync(tmp.data() + o, u->W[l], nw * 4, cudaMemcpyDeviceToHost, u->stream);
        o += nw;
        cudaMemcpyAsync(tmp.data() + o, u->B[l], (size_t)kCout[l] * 4, cudaMemcpyDeviceToHost, u->stream);
        o += kCout[l];
    }
    if (cudaStreamSynchronize(u->stream) != cudaSuccess) return ufail(u, CDI_ECUDA, "parameter download failed");
    for (size_t i = 0; i < n; ++i) host[i] = tmp[i];
    return CDI_OK;
}

// x_host: [N][2] (channels last), y_host: [N]
cdi_status cdi_unet_forward(cdi_unet* u, const double* x_host, double* y_host) {
    if (!u || !u->ws) return ufail(u, CDI_ESTATE, "network workspace not bound");
    if (!x_host || !y_host) return ufail(u, CDI_EINVAL, "null array");
    if (!u->weights_ready) refresh_weights(u);
    cdi_status st = upload_x(u, x_host);
    if (st) return st;
    forward(u, false);
    const long N = u->g[0].N;
    std::vector<float> y(N);
    if (cudaMemcpyAsync(y.data(), u->y, (size_t)N * 4, cudaMemcpyDeviceToHost, u->stream) != cudaSuccess ||
        cudaStreamSynchronize(u->stream) != cudaSuccess)
        return ufail(u, CDI_ECUDA, std::string("forward: ") + cudaGetErrorString(cudaGetLastError()));
    for (long i = 0; i < N; ++i) y_host[i] = y[i];
    return check_tc(u);
}

// forward pass on device arrays (FP32 [N][2] -> FP32 [N]), stream-ordered, no host copies
cdi_status cdi_unet_forward_device(cdi_unet* u, const float* x_dev, float* y_dev) {
    if (!u || !u->ws) return ufail(u, CDI_ESTATE, "network workspace not bound");
    if (!x_dev || !y_dev) return ufail(u, CDI_EINVAL, "null array");
    if (!u->weights_ready) refresh_weights(u);
    const long N = u->g[0].N;
    k_input_dev<<<blocks(N * 16), 256, 0, u->stream>>>((int)N, x_dev, u->x);
    forward(u, false);
    g_launches += 1;
    if (cudaMemcpyAsync(y_dev, u->y, (size_t)N * 4, cudaMemcpyDeviceToDevice, u->stream) != cudaSuccess)
        return ufail(u, CDI_ECUDA, "output copy failed");
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return ufail(u, CDI_ECUDA, std::string("forward_device: ") + cudaGetErrorString(e));
    return CDI_OK;
}

// one training step on (x, target): loss before the update; grads (FP32,
// flat parameter order) if grads_host is not NULL; Adam update if lr > 0
cdi_status cdi_unet_train_step(cdi_unet* u, const double* x_host, const double* t_host, double lr, double* loss,
                               double* grads_host) {
    if (!u || !u->ws) return ufail(u, CDI_ESTATE, "network workspace not bound");
    if (!x_host || !t_host) return ufail(u, CDI_EINVAL, "null array");
    if (!(lr >= 0.0) || !std::isfinite(lr)) return ufail(u, CDI_EINVAL, "lr must be >= 0");
    if (!u->weights_ready) refresh_weights(u);
    const long N = u->g[0].N;
    cdi_status st = upload_x(u, x_host);
    if (st) return st;
    std::vector<float> t(t_host, t_host + N);
    cudaMemcpyAsync(u->t, t.data(), (size_t)N * 4, cudaMemcpyHostToDevice, u->stream);
    forward(u);
    backward(u);
    float part = 0.f;
    cudaMemcpyAsync(&part, u->part, 4, cudaMemcpyDeviceToHost, u->stream);
    if (grads_host) {
        std::vector<float> g(param_count());
        size_t o = 0;
        for (int l = 0; l < kLayers; ++l) {
            const size_t nw = (size_t)kTaps[l] * kCout[l] * kCin[l];
            cudaMemcpyAsync(g.data() + o, u->gW[l], nw * 4, cudaMemcpyDeviceToHost, u->stream);
            o += nw;
            cudaMemcpyAsync(g.data() + o, u->gB[l], (size_t)kCout[l] * 4, cudaMemcpyDeviceToHost, u->stream);
            o += kCout[l];
        }
        if (cudaStreamSynchronize(u->stream) != cudaSuccess) return ufail(u, CDI_ECUDA, "gradient download failed");
        for (size_t i = 0; i < g.size(); ++i) grads_host[i] = g[i];
    }
    if (lr > 0.0) adam(u, lr);
    if (cudaStreamSynchronize(u->stream) != cudaSuccess)
        return ufail(u, CDI_ECUDA, std::string("train step: ") + cudaGetErrorString(cudaGetLastError()));
    if (loss) *loss = (double)part / (double)N;
    return check_tc(u);
}

cdi_status cdi_unet_set_conv_kernel(cdi_unet* u, int tensor_core) {
    if (!u) return ufail(nullptr, CDI_EINVAL, "null network");
    if (tensor_core < 0 || tensor_core > 2) return ufail(u, CDI_EINVAL, "tensor_core must be 0, 1 or 2");
    u->use_tc = tensor_core != 0;
    u->wgrad_tc = tensor_core == 1;
    return CDI_OK;
}

const char* cdi_unet_last_error(const cdi_unet* u) { return u ? u->err.c_str() : g_unet_error.c_str(); }

void cdi_unet_destroy(cdi_unet* u) { delete u; }

}  // extern "C"
