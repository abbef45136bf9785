// Defect-correction residual of the FP32-mixed form on a 3D finest level,
// tiled: r = (f - mean f) - A p with p a double-float, accumulated in
// double-float, and |r|^2 (the pressure solve's convergence measure, Sec. 4:
// the projection's Poisson equation, Eq. NS_incompressibility).  Every cell's
// arithmetic is that of ops::resid_df_at (terms x-, x+, y-, y+, z-, z+ through
// ops::df_acc_term, then ops::resid_df_finish), so r is bit-identical to the
// per-cell kernel's; what changes is the access pattern.
//
// A CTA owns a 64 x 16 tile of the x-y plane and marches along a chunk of z.
// Planes are staged in shared memory by 16-byte cp.async copies one plane
// ahead of use: p (double-floats) with a one-cell halo in y and two cells in
// x (whole 16-byte quads), and f and the three face-coefficient arrays over
// the tile plus one column and one row (the x+ and y+ faces of the tile's
// last column and row); halos wrap around the periodic x and y axes.  A
// cell's six neighbours and faces then come from shared memory at fixed
// offsets, so no index is recovered by division and every global access is a
// whole coalesced quad.  The z- face of a plane is the z+ face of the plane
// below, staged once, and its flux is that plane's z+ flux negated (the flux
// is odd in its two pressures, so the sum is unchanged to the bit).
//
// Threads: 512 (16 warps); warp w computes tile row w, lane l the cells
// x0 + l and x0 + 32 + l (32 consecutive double-floats a warp access: free of
// bank conflicts).
#include "ops.cuh"
#include "stage.cuh"

#include <cmath>

namespace cdi {

namespace {

using namespace stage;

constexpr int kQX = 64, kQY = 16;              // tile of cells in x, y
constexpr int kQThreads = 512;
constexpr int kPW = kQX + 4;                   // staged p row: cells x0-2 .. x0+65
constexpr int kPR = kQY + 2;                   // staged p rows: y0-1 .. y0+16
constexpr int kPPlaneF = 2 * kPW * kPR;        // floats of a staged p plane (2448)
constexpr int kPQuads = kPPlaneF / 4;          // 16-byte quads of a p plane (612)
constexpr int kCW = kQX + 4, kCR = kQY + 1;    // staged f / coefficient rows: x0 .. x0+67, y0 .. y0+16
constexpr int kCPlane = kCW * kCR;             // floats (1156)
constexpr int kCQuads = kCPlane / 4;           // 289
// ring slots: p planes k-1, k, k+1 in use and k+2 in flight (six slots: the z
// loop unrolls by six and every slot index is a constant); f, b0, b1 of plane
// k in use and k+1 in flight; b2 (z faces) planes k, k+1 in use and k+2 in flight
constexpr int kPSlots = 6, kCSlots = 2, kZSlots = 3;
constexpr int kOffF = kPSlots * kPPlaneF;
constexpr int kOffB0 = kOffF + kCSlots * kCPlane;
constexpr int kOffB1 = kOffB0 + kCSlots * kCPlane;
constexpr int kOffB2 = kOffB1 + kCSlots * kCPlane;
constexpr int kResidFloats = kOffB2 + kZSlots * kCPlane;
constexpr size_t kResidSmem = (size_t)kResidFloats * sizeof(float);
constexpr int kResidPerSM = 2;                 // resident CTAs an SM (shared memory)
static_assert(kPQuads <= 2 * kQThreads && kCQuads <= kQThreads, "at most two p quads and one f quad a thread");
static_assert(kPPlaneF % 4 == 0 && kCPlane % 4 == 0 && kOffF % 4 == 0, "16-byte aligned slots");

template <int V>
struct IC {
    static constexpr int value = V;
};

__device__ double tile_block_sum(double v) {
    __shared__ double sh[kQThreads / 32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) sh[wid] = v;
    __syncthreads();
    v = (wid == 0 && lane < kQThreads / 32) ? sh[lane] : 0.0;
    if (wid == 0)
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__global__ void __launch_bounds__(kQThreads, kResidPerSM)
    k_resid_tile(Geom g, const float2* __restrict__ p, const float* __restrict__ f, const float* __restrict__ b0,
                 const float* __restrict__ b1, const float* __restrict__ b2, float* __restrict__ r,
                 const float* __restrict__ fmean_df, double* __restrict__ part, int zchunk) {
    extern __shared__ __align__(128) float smr[];
    const float2 fmean = make_float2(fmean_df[0], fmean_df[1]);
    const int nx = g.n[0], ny = g.n[1], nz = g.n[2];
    const long NP = g.NP;
    const int x0 = blockIdx.x * kQX, y0 = blockIdx.y * kQY;
    const int z0 = blockIdx.z * zchunk;
    const int z1 = min(z0 + zchunk, nz);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const float* pf = reinterpret_cast<const float*>(p);

    // staging jobs of this thread, the same for every plane (offsets within
    // a plane, wrapped around x and y): p quads tid and tid + 512 (two cells
    // each), and quad tid of f / b0 / b1 / b2
    auto wrap = [](int v, int n) { return v < 0 ? v + n : (v >= n ? v - n : v); };
    int pg[2] = {0, 0}, ps[2] = {0, 0};
    const bool has_p1 = tid + kQThreads < kPQuads;
#pragma unroll
    for (int m = 0; m < 2; ++m) {
        const int q = tid + m * kQThreads;
        const int row = q / (kPW / 2), qq = q - row * (kPW / 2);
        const int x = wrap(x0 - 2 + 2 * qq, nx), y = wrap(y0 - 1 + row, ny);
        pg[m] = 2 * (x + nx * y);
        ps[m] = row * (2 * kPW) + 4 * qq;
    }
    const bool has_c = tid < kCQuads;
    int cg = 0, cs = 0;
    {
        const int row = tid / (kCW / 4), qq = tid - row * (kCW / 4);
        cg = wrap(x0 + 4 * qq, nx) + nx * wrap(y0 + row, ny);
        cs = row * kCW + 4 * qq;
    }
    // p plane zp into p slot sp (skipped beyond the walls and beyond what the
    // chunk reads)
    auto stage_p = [&](int zp, int sp) {
        if (zp < 0 || zp >= nz || zp > z1) return;
        const float* src = pf + (long)zp * (2 * NP);
        float* dst = smr + sp * kPPlaneF;
        cp_async16(dst + ps[0], src + pg[0]);
        if (has_p1) cp_async16(dst + ps[1], src + pg[1]);
    };
    // f, b0, b1 of plane zc into slot sc
    auto stage_c = [&](int zc, int sc) {
        if (zc >= z1 || !has_c) return;
        const long o = (long)zc * NP + cg;
        cp_async16(smr + kOffF + sc * kCPlane + cs, f + o);
        cp_async16(smr + kOffB0 + sc * kCPlane + cs, b0 + o);
        cp_async16(smr + kOffB1 + sc * kCPlane + cs, b1 + o);
    };
    // b2 (the low z face of every cell; plane nz holds the high wall) of plane zb into slot sz
    auto stage_z = [&](int zb, int sz) {
        if (zb > z1 || !has_c) return;
        cp_async16(smr + kOffB2 + sz * kCPlane + cs, b2 + (long)zb * NP + cg);
    };
    // prologue: p planes z0-1, z0 (slots 0, 1) and b2 plane z0 (slot 0); then
    // the group of plane z0: p plane z0+1, f / b0 / b1 plane z0, b2 plane z0+1
    stage_p(z0 - 1, 0);
    stage_p(z0, 1);
    stage_z(z0, 0);
    cp_async_commit();
    stage_p(z0 + 1, 2);
    stage_c(z0, 0);
    stage_z(z0 + 1, 1);
    cp_async_commit();

    const int ip = (warp + 1) * kPW + lane + 2;  // staged p index (double-floats) of the first cell
    const int ic = warp * kCW + lane;            // staged f / coefficient index of the first cell
    float* rout = r + (long)z0 * NP + (long)nx * (y0 + warp) + x0 + lane;
    const float ih2 = g.ih2f;
    float acc = 0.f;
    float zt[2] = {0.f, 0.f}, zte[2] = {0.f, 0.f};  // z+ flux of the previous plane, per cell

    // plane k = z0 + 6 m + u: p plane k + j in slot (u + j + 1) mod 6, f / b0 /
    // b1 plane k in slot u mod 2, b2 plane k + j in slot (u + j) mod 3
    auto plane = [&](auto uc, int k) {
        constexpr int u = decltype(uc)::value;
        constexpr int sPm = u % kPSlots, sP0 = (u + 1) % kPSlots, sPp = (u + 2) % kPSlots;
        constexpr int sC = u % kCSlots, sZ0 = u % kZSlots, sZ1 = (u + 1) % kZSlots;
        cp_async_wait<0>();
        __syncthreads();  // plane k's group has landed; plane k-1 is done with its slots
        stage_p(k + 2, (u + 3) % kPSlots);
        stage_c(k + 1, (u + 1) % kCSlots);
        stage_z(k + 2, (u + 2) % kZSlots);
        cp_async_commit();
        const float2* P0 = reinterpret_cast<const float2*>(smr + sP0 * kPPlaneF);
        const float2* Pm = reinterpret_cast<const float2*>(smr + sPm * kPPlaneF);
        const float2* Pp = reinterpret_cast<const float2*>(smr + sPp * kPPlaneF);
        const float* F = smr + kOffF + sC * kCPlane;
        const float* B0 = smr + kOffB0 + sC * kCPlane;
        const float* B1 = smr + kOffB1 + sC * kCPlane;
        const float* Z0 = smr + kOffB2 + sZ0 * kCPlane;
        const float* Z1 = smr + kOffB2 + sZ1 * kCPlane;
        const bool lo = k > 0, hi = k < nz - 1;
#pragma unroll
        for (int i = 0; i < 2; ++i) {
            const int jp = ip + 32 * i, jc = ic + 32 * i;
            const float2 pc = P0[jp];
            float Sh = 0.f, Sl = 0.f;
            ops::df_acc_term(B0[jc], P0[jp - 1], pc, Sh, Sl);
            ops::df_acc_term(B0[jc + 1], P0[jp + 1], pc, Sh, Sl);
            ops::df_acc_term(B1[jc], P0[jp - kPW], pc, Sh, Sl);
            ops::df_acc_term(B1[jc + kCW], P0[jp + kPW], pc, Sh, Sl);
            // the z- flux is the z+ flux of the plane below with its sign
            // flipped (exactly: the flux is odd in its two pressures), except
            // on the chunk's first plane
            float t, te;
            if (k == z0) {
                ops::df_term(Z0[jc], lo ? Pm[jp] : pc, pc, t, te);
            } else {
                t = -zt[i];
                te = -zte[i];
            }
            ops::df_acc(t, te, Sh, Sl);
            ops::df_term(Z1[jc], hi ? Pp[jp] : pc, pc, zt[i], zte[i]);
            ops::df_acc(zt[i], zte[i], Sh, Sl);
            const float v = ops::resid_df_finish(Sh, Sl, ih2, F[jc], fmean);
            rout[32 * i] = v;
            acc += v * v;
        }
        rout += NP;
    };
    for (int kb = z0; kb < z1; kb += kPSlots) {
        plane(IC<0>{}, kb);
        if (kb + 1 >= z1) break;
        plane(IC<1>{}, kb + 1);
        if (kb + 2 >= z1) break;
        plane(IC<2>{}, kb + 2);
        if (kb + 3 >= z1) break;
        plane(IC<3>{}, kb + 3);
        if (kb + 4 >= z1) break;
        plane(IC<4>{}, kb + 4);
        if (kb + 5 >= z1) break;
        plane(IC<5>{}, kb + 5);
    }
    cp_async_wait<0>();  // the last group stages nothing, but leave no copy in flight
    const double a = tile_block_sum((double)acc);
    if (tid == 0) part[blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z)] = a;
}

int sm_count() {
    static int n = 0;
    if (!n) {
        int dev = 0, v = 0;
        if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) !=
                                                      cudaSuccess) {
            cudaGetLastError();
            v = 152;
        }
        n = v;
    }
    return n;
}

// planes per z chunk: the chunk count maximises the fill of the last wave of
// resident CTAs times the share of staged p planes that are not re-read halo
// (two per chunk), with at most kMaxParts CTAs (one partial sum each)
int resid_zchunk(const Geom& g, int max_parts) {
    const long tiles = (long)(g.n[0] / kQX) * (g.n[1] / kQY);
    const double wave = (double)kResidPerSM * sm_count();
    const int nz = g.n[2];
    int best = nz;
    double best_score = -1.0;
    for (int c = 1; c <= nz && tiles * c <= max_parts; ++c) {
        const int ch = (nz + c - 1) / c;
        const int nc = (nz + ch - 1) / ch;
        const double waves = tiles * nc / wave;
        const double fill = waves / std::ceil(waves);
        const double score = fill * (1.0 - 2.0 / (ch + 2.0));
        if (score > best_score + 1e-9) {
            best_score = score;
            best = ch;
        }
    }
    return best;
}

}  // namespace

bool resid_tile_supported(const Geom& g, int max_parts) {
    return g.D == 3 && g.n[0] % kQX == 0 && g.n[1] % kQY == 0 && g.n[2] >= 2 &&
           (long)(g.n[0] / kQX) * (g.n[1] / kQY) <= max_parts && g.N < (1L << 31);
}

cudaError_t resid_tile_prepare() {
    return cudaFuncSetAttribute((const void*)k_resid_tile, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)kResidSmem);
}

// r and the partial sums of |r|^2 (one a CTA) of the FP32-mixed form's level
// 0; returns the number of partials
unsigned launch_resid_tile(const MGLevel& L0, const float* fmean_df, double* part, int max_parts, cudaStream_t s) {
    const Geom& g = L0.g;
    const int zchunk = resid_zchunk(g, max_parts);
    const dim3 grid((unsigned)(g.n[0] / kQX), (unsigned)(g.n[1] / kQY), (unsigned)((g.n[2] + zchunk - 1) / zchunk));
    k_resid_tile<<<grid, kQThreads, kResidSmem, s>>>(g, reinterpret_cast<const float2*>(L0.p),
                                                     reinterpret_cast<const float*>(L0.f), L0.bf[0], L0.bf[1],
                                                     L0.bf[2], L0.r, fmean_df, part, zchunk);
    return grid.x * grid.y * grid.z;
}

}  // namespace cdi
