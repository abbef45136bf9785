// Pressure projection, geometric multigrid and fixed-order reductions as
// standalone kernels (the launch-per-kernel path and the stage-level C-ABI
// calls).  The arithmetic lives in ops.cuh.
//
//   k_div            f = div u* / (c dt)                                   Eq. (NS_incompressibility)
//   k_sub_mean_sq    remove the mean of f (the walls and periodic sides
//                    carry no net flux), accumulate |f|^2 (FP64 form; the
//                    FP32-mixed form keeps f and removes the mean in k_resid)
//   k_coef0          face coefficients 1/rho_f, rho_f the mean of the two  Sec. 2 (rho linear in phi)
//                    adjacent cells, zero on the walls
//   k_resid          residual r = f - A p in the form's precision, |r|^2,
//                    FP32 copy of r
//   k_rbgs_rows      FP32 red-black Gauss-Seidel colour pass of A e = r on a
//                    coarse level (row-mapped; level 0: k_rbgs0, or the
//                    one-pass sweep of k_sweep.cu)
//   k_resid_restrict FP32 residual and its restriction (mean of the 2^D children)
//   k_prolong        FP32 cell-centred (bi/tri)linear prolongation (3D grids of
//                    32 x 8 columns: k_prolong0_3)
//   k_coarse         FP64 dense solve of the coarsest level in one CTA
//   k_update         p += e (FP64, or double-float in the FP32-mixed form) where
//                    the V-cycle's last level-0 sweep does not add it
//   k_project        u = u* - c dt grad p / rho_f on every interior face     Eq. (no-penetration BC)
//   k_mass, k_umax, k_contact_line: FP64 reductions                          Sec. 2, 3.1, 5.1
//
// Every sum is deterministic: a fixed grid of at most kPartials blocks, a
// fixed per-thread stride, a warp-shuffle tree per block and one final block.
#include "ops.cuh"

#include <algorithm>
#include <cmath>
#include <mutex>
#include <unordered_map>

namespace cdi {

namespace {

constexpr int kThreads = 256;
using Ld = ops::LdPlain;
inline unsigned blocks_for(long n) { return (unsigned)((n + kThreads - 1) / kThreads); }
// Grid of a grid-stride reduction kernel: at most kPartials blocks, at most one
// cell per thread, and no more blocks than the device holds at once (a second,
// partial wave would leave most SMs idle while it runs).  The grid depends only
// on the kernel and the device, so every sum keeps its fixed order.
unsigned red_blocks(const void* kernel, long n) {
    static std::mutex mu;
    static std::unordered_map<const void*, long> resident;
    long res;
    {
        std::lock_guard<std::mutex> lk(mu);
        auto it = resident.find(kernel);
        if (it == resident.end()) {
            int dev = 0, nsm = 0, per = 0;
            if (cudaGetDevice(&dev) != cudaSuccess ||
                cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
                cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kernel, kThreads, 0) != cudaSuccess) {
                cudaGetLastError();
                nsm = 1;
                per = kPartials;
            }
            it = resident.emplace(kernel, std::max(1L, (long)nsm * per)).first;
        }
        res = it->second;
    }
    return (unsigned)std::max(1L, std::min({(long)kPartials, res, (n + kThreads - 1) / kThreads}));
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_down_sync(0xffffffffu, v, o));
    return v;
}
// block-wide sum, valid in thread 0
__device__ double block_sum(double v) {
    __shared__ double sh[32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    v = warp_sum(v);
    __syncthreads();
    if (lane == 0) sh[wid] = v;
    __syncthreads();
    const int nw = (blockDim.x + 31) >> 5;
    v = (wid == 0 && lane < nw) ? sh[lane] : 0.0;
    if (wid == 0) v = warp_sum(v);
    return v;
}
__device__ double block_max(double v) {
    __shared__ double sh[32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    v = warp_max(v);
    __syncthreads();
    if (lane == 0) sh[wid] = v;
    __syncthreads();
    const int nw = (blockDim.x + 31) >> 5;
    v = (wid == 0 && lane < nw) ? sh[lane] : 0.0;
    if (wid == 0) v = warp_max(v);
    return v;
}

// out = mean as a double-float, from the FP64 mean (one thread)
__global__ void k_mean_df(const double* mean, float* out) {
    const float2 m = ops::dfl::from_double(*mean);
    out[0] = m.x;
    out[1] = m.y;
}

// final pass of a sum: out = scale * sum(partials[0..np))
__global__ void k_final_sum(const double* part, int np, double scale, double* out, int do_sqrt) {
    double v = 0.0;
    for (int t = threadIdx.x; t < np; t += blockDim.x) v += part[t];
    v = block_sum(v);
    if (threadIdx.x == 0) {
        double r = v * scale;
        *out = do_sqrt ? sqrt(r) : r;
    }
}

template <typename T, int DIM>
__global__ void k_div(Geom g, const T* u0, const T* u1, const T* u2, T inv_cdt, FT<T>* f, double* part) {
    const T* us[3] = {u0, u1, u2};
    const T ih = g_ih<T>(g);
    ops::SumAcc<T> acc;
    const long stride = (long)gridDim.x * blockDim.x;
    for (long c = (long)blockIdx.x * blockDim.x + threadIdx.x; c < g.N; c += stride) {
        const T v = ops::div_at<Ld, T, DIM>(g, us, ih, inv_cdt, c);
        f[c] = v;
        acc.add(v);
    }
    const double a = block_sum(acc.value());
    if (threadIdx.x == 0) part[blockIdx.x] = a;
}

// k_div on FP32 3D grids with nx a multiple of 4: four cells of one x row an
// iteration on float4 words (the x+ face of the fourth is the next quad's
// first word, or the row's first across the periodic seam), the terms of
// div_at in its order; the same fixed grid and per-block sums
__global__ void k_div4(Geom g, const float* __restrict__ u0, const float* __restrict__ u1,
                       const float* __restrict__ u2, float inv_cdt, float* __restrict__ f, double* part) {
    const float ih = g.ihf;
    const int nx = g.n[0], ny = g.n[1];
    const long nq = g.N / 4;
    ops::SumAcc<float> acc;
    const long stride = (long)gridDim.x * blockDim.x;
    for (long t = (long)blockIdx.x * blockDim.x + threadIdx.x; t < nq; t += stride) {
        const long c = 4 * t;
        const long line = c / nx;
        const int i0 = (int)(c - line * nx);
        const int j = (int)(line % ny);
        const long row = line * nx;
        const float4 a0 = __ldg(reinterpret_cast<const float4*>(u0 + c));
        const float xe = __ldg(u0 + (i0 + 4 == nx ? row : c + 4));
        const long yp = (j == ny - 1) ? c - (long)(ny - 1) * nx : c + nx;
        const float4 b0 = __ldg(reinterpret_cast<const float4*>(u1 + c));
        const float4 b1 = __ldg(reinterpret_cast<const float4*>(u1 + yp));
        const float4 z0 = __ldg(reinterpret_cast<const float4*>(u2 + c));
        const float4 z1 = __ldg(reinterpret_cast<const float4*>(u2 + c + g.NP));
        const float ax[5] = {a0.x, a0.y, a0.z, a0.w, xe};
        const float by0[4] = {b0.x, b0.y, b0.z, b0.w}, by1[4] = {b1.x, b1.y, b1.z, b1.w};
        const float zz0[4] = {z0.x, z0.y, z0.z, z0.w}, zz1[4] = {z1.x, z1.y, z1.z, z1.w};
        float o[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            float div = 0.f;
            div += ax[e + 1] - ax[e];
            div += by1[e] - by0[e];
            div += zz1[e] - zz0[e];
            o[e] = div * ih * inv_cdt;
            acc.add(o[e]);
        }
        *reinterpret_cast<float4*>(f + c) = make_float4(o[0], o[1], o[2], o[3]);
    }
    const double a = block_sum(acc.value());
    if (threadIdx.x == 0) part[blockIdx.x] = a;
}

// FP64 form: f -= mean, |f|^2
__global__ void k_sub_mean_sq(long N, double* f, const double* mean_p, double* part) {
    const double mean = *mean_p;
    double acc = 0.0;
    const long stride = (long)gridDim.x * blockDim.x;
    for (long c = (long)blockIdx.x * blockDim.x + threadIdx.x; c < N; c += stride) {
        const double v = f[c] - mean;
        f[c] = v;
        acc += v * v;
    }
    acc = block_sum(acc);
    if (threadIdx.x == 0) part[blockIdx.x] = acc;
}

// FP32-mixed form: |f - mean|^2 with the double-float mean, f unchanged
__global__ void k_fnorm_df(long N, const float* f, const float* mean_df, double* part) {
    const float mh = mean_df[0], ml = mean_df[1];
    float acc = 0.f;
    const long stride = (long)gridDim.x * blockDim.x;
    for (long c = (long)blockIdx.x * blockDim.x + threadIdx.x; c < N; c += stride) {
        const float v = (f[c] - mh) - ml;
        acc += v * v;
    }
    const double a = block_sum((double)acc);
    if (threadIdx.x == 0) part[blockIdx.x] = a;
}

template <typename T, int DIM>
__global__ void k_coef0(Geom g, PhysDev ph, const T* phi, double* b0, double* b1, double* b2, float* f0, float* f1,
                        float* f2, float* rho0) {
    double* bs[3] = {b0, b1, b2};
    float* bf[3] = {f0, f1, f2};
    long t = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t < g.N + g.NP) ops::coef0_at<Ld, T, DIM>(g, ph, phi, bs, bf, rho0, t);
}

// k_coef0 of the FP32-mixed form on 3D grids with nx a multiple of 4: four
// cells of one x row a thread on float4 words (64 x-quads x 4 rows of one z
// plane a block), the arithmetic of coef0_at term for term; the top plane's
// threads also clear the high wall's faces above them
constexpr int kCoefX = 64, kCoefY = 4;
__global__ void __launch_bounds__(kCoefX * kCoefY)
    k_coef0_4(Geom g, PhysDev ph, const float* __restrict__ phi, float* f0, float* f1, float* f2, float* rho0) {
    const int q = blockIdx.x * kCoefX + threadIdx.x, j = blockIdx.y * kCoefY + threadIdx.y;
    const int nx = g.n[0], ny = g.n[1], k = blockIdx.z;
    if (4 * q >= nx || j >= ny) return;
    const long row = (long)nx * ((long)j + (long)ny * k);
    const long c = row + 4L * q;
    const float dr = phys<float>(ph).drho, rho2 = phys<float>(ph).rho2;
    const float4 pc4 = __ldg(reinterpret_cast<const float4*>(phi + c));
    const float pc[4] = {pc4.x, pc4.y, pc4.z, pc4.w};
    *reinterpret_cast<float4*>(rho0 + c) =
        make_float4(dr * pc[0] + rho2, dr * pc[1] + rho2, dr * pc[2] + rho2, dr * pc[3] + rho2);
    float* bf[3] = {f0, f1, f2};
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        if (a == 2 && k == 0) {  // low wall faces
            *reinterpret_cast<float4*>(f2 + c) = make_float4(0.f, 0.f, 0.f, 0.f);
            continue;
        }
        float pl[4];
        if (a == 0) {
            pl[0] = __ldg(phi + (q == 0 ? row + nx - 1 : c - 1));
            pl[1] = pc[0];
            pl[2] = pc[1];
            pl[3] = pc[2];
        } else {
            const long cL = a == 1 ? ((j == 0) ? c + (long)(ny - 1) * nx : c - nx) : c - g.NP;
            const float4 l4 = __ldg(reinterpret_cast<const float4*>(phi + cL));
            pl[0] = l4.x;
            pl[1] = l4.y;
            pl[2] = l4.z;
            pl[3] = l4.w;
        }
        float o[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const float rf = 0.5f * ((dr * pl[e] + rho2) + (dr * pc[e] + rho2));
            o[e] = 1.f / rf;
        }
        *reinterpret_cast<float4*>(bf[a] + c) = make_float4(o[0], o[1], o[2], o[3]);
    }
    if (k == g.n[2] - 1)  // high wall faces
        *reinterpret_cast<float4*>(f2 + c + g.NP) = make_float4(0.f, 0.f, 0.f, 0.f);
}

template <int DIM>
__global__ void k_coef_restrict(Geom gf, Geom gc, const float* f0, const float* f1, const float* f2, float* c0,
                                float* c1, float* c2) {
    const float* fb[3] = {f0, f1, f2};
    float* cb[3] = {c0, c1, c2};
    long t = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t < gc.N + gc.NP) ops::coef_restrict_at<Ld, float, DIM>(gf, gc, fb, cb, t);
}

template <typename T, int DIM>
__global__ void k_resid(MGLevel L0, const float* fmean_df, double* part) {
    const PT<T>* p = ops::pbuf<T>(L0);
    const FT<T>* f = ops::fbuf<T>(L0);
    const float2 fmean = fmean_df ? make_float2(fmean_df[0], fmean_df[1]) : make_float2(0.f, 0.f);
    T acc = T(0);
    const long stride = (long)gridDim.x * blockDim.x;
    for (long c = (long)blockIdx.x * blockDim.x + threadIdx.x; c < L0.g.N; c += stride) {
        const T r = ops::resid_form_at<Ld, DIM>(L0, p, f, fmean, c);
        L0.r[c] = (float)r;
        acc += r * r;
    }
    const double a = block_sum((double)acc);
    if (threadIdx.x == 0) part[blockIdx.x] = a;
}

// row-mapped colour passes (k_rbgs_rows, k_rbgs0): blocks of 64 pairs x 4 rows
constexpr int kSweepX = 64, kSweepY = 4;

// One colour of a coarse level's red-black sweep with the arithmetic of
// ops::rbgs_at (stencil_L's terms x, y, z with the stored face coefficients,
// then step_div) on the row-mapped thread grid of k_rbgs0: thread (ix, j, k)
// updates cell 2 ix + ((colour + j + k) & 1) of row (j, k), so no index is
// decoded.
template <int DIM>
__global__ void __launch_bounds__(kSweepX * kSweepY)
    k_rbgs_rows(Geom g, const float* __restrict__ b0, const float* __restrict__ b1, const float* __restrict__ b2,
                float* __restrict__ e, const float* __restrict__ r, int colour) {
    const int nx = g.n[0], ny = g.n[1];
    const int ix = blockIdx.x * kSweepX + threadIdx.x;
    const int j = blockIdx.y * kSweepY + threadIdx.y;
    const int k = (DIM == 3) ? (int)blockIdx.z : 0;
    if (2 * ix >= nx || j >= ny) return;
    const int i = 2 * ix + ((colour + j + k) & 1);
    const long row = (long)nx * ((long)j + (long)ny * k);
    const long c = row + i;
    const float ih2 = g.ih2f;
    float diag = 0.f, off = 0.f;
    {  // x (periodic)
        const long lo = row + (i == 0 ? nx - 1 : i - 1), hi = row + (i == nx - 1 ? 0 : i + 1);
        const float bm = b0[c], bp = b0[hi];
        diag += (bm + bp) * ih2;
        off += (bm * e[lo] + bp * e[hi]) * ih2;
    }
    if (DIM == 3) {  // y (periodic), then z (walls)
        const long lo = (j == 0) ? c + (long)(ny - 1) * nx : c - nx;
        const long hi = (j == ny - 1) ? c - (long)(ny - 1) * nx : c + nx;
        const float bm = b1[c], bp = b1[hi];
        diag += (bm + bp) * ih2;
        off += (bm * e[lo] + bp * e[hi]) * ih2;
        const long np = g.NP;
        const bool wlo = k == 0, whi = k == g.n[2] - 1;
        const float bmz = b2[c], bpz = b2[c + np];
        const float pm = wlo ? 0.f : e[c - np], pp = whi ? 0.f : e[c + np];
        diag += (bmz + bpz) * ih2;
        off += (bmz * pm + bpz * pp) * ih2;
    } else {  // y (walls)
        const bool wlo = j == 0, whi = j == ny - 1;
        const float bm = b1[c], bp = b1[c + nx];
        const float pm = wlo ? 0.f : e[c - nx], pp = whi ? 0.f : e[c + nx];
        diag += (bm + bp) * ih2;
        off += (bm * pm + bp * pp) * ih2;
    }
    e[c] = ops::step_div(off - r[c], diag);
}

// Level-0 red-black sweep of one colour on a (x/2, y, z) thread grid: thread
// (ix, j, k) updates cell i = 2 ix + ((colour + j + k) & 1) of row (j, k), so
// no index is recovered by division.  Coefficients b = 2 / (rho_c + rho_nb)
// from the FP32 cell densities, zero through the walls (the last axis); the
// update e_c = (sum b e_nb - r h^2) / sum b (the Gauss-Seidel step of
// apply_L_rho) is formed with the half coefficients b' = 1 / (rho_c + rho_nb)
// as (sum b' e_nb - r h^2 / 2) / sum b', reciprocals by ops::rcp_approx: the
// arithmetic, term for term, of the one-pass sweep (k_sweep.cu).
// kSweepFromZero: the first red pass of a V-cycle, whose neighbours are all
// zero (e is not cleared beforehand: every cell of e is written before it is
// read).  kSweepUpdate: the last black pass, which also adds the now final
// correction of both cells of the thread's pair (2 ix, 2 ix + 1) to p.
template <typename T, int DIM, int MODE>
__global__ void __launch_bounds__(kSweepX * kSweepY) k_rbgs0(Geom g, const float* __restrict__ rho,
                                                             float* __restrict__ e, const float* __restrict__ r,
                                                             int colour, float h2h, float omega, int own_zero,
                                                             PT<T>* __restrict__ p) {
    const int nx = g.n[0], ny = g.n[1];
    const int ix = blockIdx.x * kSweepX + threadIdx.x;
    const int j = blockIdx.y * kSweepY + threadIdx.y;
    const int k = (DIM == 3) ? (int)blockIdx.z : 0;
    if (2 * ix >= nx || j >= ny) return;
    const int i = 2 * ix + ((colour + j + k) & 1);
    const long row = (long)nx * ((long)j + (long)ny * k);
    const long c = row + i;
    const float rc = rho[c];
    // e of a neighbour (zero in the first pass: the loads are not issued)
    auto en = [&](long n) { return MODE == kSweepFromZero ? 0.f : e[n]; };
    const long xm = row + (i == 0 ? nx - 1 : i - 1), xp = row + (i == nx - 1 ? 0 : i + 1);
    float bsum, off;
    {
        const float b0 = ops::rcp_approx(rc + rho[xm]), b1 = ops::rcp_approx(rc + rho[xp]);
        bsum = b0 + b1;
        off = b0 * en(xm) + b1 * en(xp);
    }
    if (DIM == 2) {  // y is the wall axis
        if (j > 0) {
            const float b = ops::rcp_approx(rc + rho[c - nx]);
            bsum += b;
            off += b * en(c - nx);
        }
        if (j < ny - 1) {
            const float b = ops::rcp_approx(rc + rho[c + nx]);
            bsum += b;
            off += b * en(c + nx);
        }
    } else {
        const long ym = (j == 0) ? c + (long)(ny - 1) * nx : c - nx;
        const long yp = (j == ny - 1) ? c - (long)(ny - 1) * nx : c + nx;
        const float b2 = ops::rcp_approx(rc + rho[ym]), b3 = ops::rcp_approx(rc + rho[yp]);
        bsum += b2 + b3;
        off += b2 * en(ym) + b3 * en(yp);
        const long np = g.NP;
        if (k > 0) {
            const float b = ops::rcp_approx(rc + rho[c - np]);
            bsum += b;
            off += b * en(c - np);
        }
        if (k < g.n[2] - 1) {
            const float b = ops::rcp_approx(rc + rho[c + np]);
            bsum += b;
            off += b * en(c + np);
        }
    }
    float ec = __fmul_rn(off - r[c] * h2h, ops::rcp_approx(bsum));
    // over-relaxation from the cell's old value (zero in the first sweep of a V-cycle)
    if (omega != 1.f) ec = ops::relax(MODE == kSweepFromZero || own_zero ? 0.f : e[c], ec, omega);
    e[c] = ec;
    if (MODE == kSweepUpdate) {
        const long co = c ^ 1;  // the pair's other cell (row starts are even: nx is even)
        p[c] = ops::p_add(p[c], ec);
        p[co] = ops::p_add(p[co], e[co]);
    }
}

template <int DIM>
__global__ void k_resid_restrict0(Geom gf, Geom gc, const float* rho0, const float* e, const float* r, float* rc,
                                  float* ec) {
    long t = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t < gc.N) ops::resid_restrict_rho_at<Ld, DIM>(gf, gc, rho0, e, r, rc, ec, t);
}

// Level-0 -> level-1 restriction of the residual of 3D grids in the order of
// ops::resid_restrict_rho_at (children in the order z, y, x; each child's
// stencil x, y, z) with the finest-level smoother's coefficients: half
// coefficients b' = 1 / (rho_c + rho_nb) by ops::rcp_approx against 2 / h^2,
// so the coarse correction targets the operator the one-pass sweep and the
// colour passes smooth.  One thread per coarse (x, y) column marching over a
// z chunk, the fine neighbour offsets formed once.  r_c = mean of the
// children's f - A e, e_c = 0.  Coarse blocks of 32 x 8 columns.
constexpr int kRestrictZ = 4;
__global__ void __launch_bounds__(256) k_restrict0_3(Geom gf, Geom gc, const float* __restrict__ rho,
                                                     const float* __restrict__ e, const float* __restrict__ r,
                                                     float* __restrict__ rc, float* __restrict__ ec) {
    const int I = blockIdx.x * 32 + threadIdx.x, J = blockIdx.y * 8 + threadIdx.y;
    const int nx = gf.n[0], ny = gf.n[1], nz = gf.n[2];
    const long NP = gf.NP;
    const float ih2 = 2.f * gf.ih2f;  // half coefficients b' = b / 2: 2 / h^2
    // offsets of the x and y neighbours of the children 2I + t0, 2J + t1
    long xm[2], xp[2], ym[2], yp[2];
    xm[0] = 2 * I == 0 ? nx - 1 : -1;
    xp[0] = 1;
    xm[1] = -1;
    xp[1] = 2 * I + 1 == nx - 1 ? -(long)(nx - 1) : 1;
    ym[0] = 2 * J == 0 ? (long)(ny - 1) * nx : -(long)nx;
    yp[0] = nx;
    ym[1] = -(long)nx;
    yp[1] = 2 * J + 1 == ny - 1 ? -(long)(ny - 1) * nx : (long)nx;
    const long cbase = 2L * I + (long)nx * (2L * J);
    const long tbase = (long)I + (long)gc.n[0] * J;
    const int K0 = blockIdx.z * kRestrictZ, K1 = min(K0 + kRestrictZ, gc.n[2]);
    for (int K = K0; K < K1; ++K) {
        float s = 0.f;
#pragma unroll
        for (int t2 = 0; t2 < 2; ++t2)
#pragma unroll
            for (int t1 = 0; t1 < 2; ++t1)
#pragma unroll
                for (int t0 = 0; t0 < 2; ++t0) {
                    const int k = 2 * K + t2;
                    const long c = cbase + t0 + (long)nx * t1 + (long)k * NP;
                    const float rcen = __ldg(rho + c);
                    float diag = 0.f, off = 0.f;
                    {
                        const long lo = c + xm[t0], hi = c + xp[t0];
                        const float bm = ops::rcp_approx(rcen + __ldg(rho + lo));
                        const float bp = ops::rcp_approx(rcen + __ldg(rho + hi));
                        diag += (bm + bp) * ih2;
                        off += (bm * __ldg(e + lo) + bp * __ldg(e + hi)) * ih2;
                    }
                    {
                        const long lo = c + ym[t1], hi = c + yp[t1];
                        const float bm = ops::rcp_approx(rcen + __ldg(rho + lo));
                        const float bp = ops::rcp_approx(rcen + __ldg(rho + hi));
                        diag += (bm + bp) * ih2;
                        off += (bm * __ldg(e + lo) + bp * __ldg(e + hi)) * ih2;
                    }
                    {
                        const bool wlo = k == 0, whi = k == nz - 1;
                        const long lo = wlo ? c : c - NP, hi = whi ? c : c + NP;
                        const float bm = (wlo ? 0.f : 1.f) * ops::rcp_approx(rcen + __ldg(rho + lo));
                        const float bp = (whi ? 0.f : 1.f) * ops::rcp_approx(rcen + __ldg(rho + hi));
                        const float pm = wlo ? 0.f : __ldg(e + lo);
                        const float pp = whi ? 0.f : __ldg(e + hi);
                        diag += (bm + bp) * ih2;
                        off += (bm * pm + bp * pp) * ih2;
                    }
                    const float Lp = off - diag * __ldg(e + c);
                    s += __ldg(r + c) - Lp;
                }
        const long t = tbase + (long)K * gc.NP;
        rc[t] = s * (1.f / 8.f);
        ec[t] = 0.f;
    }
}

// Residual restriction of a coarse 3D level (stored face coefficients) with
// the arithmetic of ops::resid_restrict_at (children in the order z, y, x;
// each child's stencil_L terms x, y, z), one thread per coarse (x, y) column
// marching over a z chunk with the fine neighbour offsets formed once:
// r_c = mean of the children's r - A e, e_c = 0.  Coarse blocks of 32 x 8.
__global__ void __launch_bounds__(256) k_restrict_bf3(Geom gf, Geom gc, const float* __restrict__ b0,
                                                      const float* __restrict__ b1, const float* __restrict__ b2,
                                                      const float* __restrict__ e, const float* __restrict__ r,
                                                      float* __restrict__ rc, float* __restrict__ ec) {
    const int I = blockIdx.x * 32 + threadIdx.x, J = blockIdx.y * 8 + threadIdx.y;
    const int nx = gf.n[0], ny = gf.n[1], nz = gf.n[2];
    const long NP = gf.NP;
    const float ih2 = gf.ih2f;
    // offsets of the x and y neighbours of the children 2I + t0, 2J + t1
    long xm[2], xp[2], ym[2], yp[2];
    xm[0] = 2 * I == 0 ? nx - 1 : -1;
    xp[0] = 1;
    xm[1] = -1;
    xp[1] = 2 * I + 1 == nx - 1 ? -(long)(nx - 1) : 1;
    ym[0] = 2 * J == 0 ? (long)(ny - 1) * nx : -(long)nx;
    yp[0] = nx;
    ym[1] = -(long)nx;
    yp[1] = 2 * J + 1 == ny - 1 ? -(long)(ny - 1) * nx : (long)nx;
    const long cbase = 2L * I + (long)nx * (2L * J);
    const long tbase = (long)I + (long)gc.n[0] * J;
    const int K0 = blockIdx.z * kRestrictZ, K1 = min(K0 + kRestrictZ, gc.n[2]);
    for (int K = K0; K < K1; ++K) {
        float s = 0.f;
#pragma unroll
        for (int t2 = 0; t2 < 2; ++t2)
#pragma unroll
            for (int t1 = 0; t1 < 2; ++t1)
#pragma unroll
                for (int t0 = 0; t0 < 2; ++t0) {
                    const int k = 2 * K + t2;
                    const long c = cbase + t0 + (long)nx * t1 + (long)k * NP;
                    float diag = 0.f, off = 0.f;
                    {
                        const long lo = c + xm[t0], hi = c + xp[t0];
                        const float bm = __ldg(b0 + c), bp = __ldg(b0 + hi);
                        diag += (bm + bp) * ih2;
                        off += (bm * __ldg(e + lo) + bp * __ldg(e + hi)) * ih2;
                    }
                    {
                        const long lo = c + ym[t1], hi = c + yp[t1];
                        const float bm = __ldg(b1 + c), bp = __ldg(b1 + hi);
                        diag += (bm + bp) * ih2;
                        off += (bm * __ldg(e + lo) + bp * __ldg(e + hi)) * ih2;
                    }
                    {
                        const bool wlo = k == 0, whi = k == nz - 1;
                        const float bm = __ldg(b2 + c), bp = __ldg(b2 + c + NP);
                        const float pm = wlo ? 0.f : __ldg(e + c - NP);
                        const float pp = whi ? 0.f : __ldg(e + c + NP);
                        diag += (bm + bp) * ih2;
                        off += (bm * pm + bp * pp) * ih2;
                    }
                    const float Lp = off - diag * __ldg(e + c);
                    s += __ldg(r + c) - Lp;
                }
        const long t = tbase + (long)K * gc.NP;
        rc[t] = s * (1.f / 8.f);
        ec[t] = 0.f;
    }
}

// Level-1 -> level-0 prolongation of 3D grids with the arithmetic of
// ops::prolong_val (trilinear weights 3/4, 1/4; coarse neighbours in the order
// z, y, x), one thread per fine (x, y) column marching over a z chunk: the
// four coarse columns' values of coarse planes K-1 .. K+2 are held in
// registers (fine planes 2K and 2K+1 use K with K-1 and with K+1), so each
// coarse value is loaded once per thread, and the fine values of four planes
// are loaded together: e += P e_c.  Fine blocks of 32 x 8.
constexpr int kProlongZ = 16;  // fine planes a thread (even)
__global__ void __launch_bounds__(256) k_prolong0_3(Geom gf, Geom gc, const float* __restrict__ ecoarse,
                                                    float* __restrict__ e) {
    const int i = blockIdx.x * 32 + threadIdx.x, j = blockIdx.y * 8 + threadIdx.y;
    const int ncx = gc.n[0], ncy = gc.n[1], ncz = gc.n[2];
    int Ix[2], Iy[2];
    Ix[0] = i >> 1;
    Ix[1] = (i & 1) ? Ix[0] + 1 : Ix[0] - 1;
    if (Ix[1] < 0) Ix[1] += ncx;
    else if (Ix[1] >= ncx) Ix[1] -= ncx;
    Iy[0] = j >> 1;
    Iy[1] = (j & 1) ? Iy[0] + 1 : Iy[0] - 1;
    if (Iy[1] < 0) Iy[1] += ncy;
    else if (Iy[1] >= ncy) Iy[1] -= ncy;
    const float w[2] = {0.75f, 0.25f};
    long col[4];  // coarse column (t1, t0) at index 2 t1 + t0
#pragma unroll
    for (int t1 = 0; t1 < 2; ++t1)
#pragma unroll
        for (int t0 = 0; t0 < 2; ++t0) col[2 * t1 + t0] = (long)Ix[t0] + (long)ncx * Iy[t1];
    const long ncp = gc.NP;
    // the four columns' values of coarse plane K (clamped to the grid: the
    // prolongation's wall rule)
    auto load = [&](int K, float* v) {
        const long o = (long)min(max(K, 0), ncz - 1) * ncp;
#pragma unroll
        for (int q = 0; q < 4; ++q) v[q] = __ldg(ecoarse + col[q] + o);
    };
    float* ef = e + (long)i + (long)gf.n[0] * j;
    // correction of a fine cell from coarse planes Iz0 = k / 2 (va) and Iz1 (vb)
    auto corr = [&](const float* va, const float* vb) {
        float s = 0.f;
#pragma unroll
        for (int t2 = 0; t2 < 2; ++t2) {
            const float* vv = t2 == 0 ? va : vb;
#pragma unroll
            for (int t1 = 0; t1 < 2; ++t1)
#pragma unroll
                for (int t0 = 0; t0 < 2; ++t0) s += w[t0] * w[t1] * w[t2] * vv[2 * t1 + t0];
        }
        return s;
    };
    // four fine planes 2K .. 2K+3 an iteration (their e loads issued together):
    // coarse planes K-1 .. K+2 in vm, v0, vp, vq
    const int k0 = blockIdx.z * kProlongZ, k1 = min(k0 + kProlongZ, gf.n[2]);
    const long NP = gf.NP;
    float vm[4], v0[4], vp[4], vq[4];
    load((k0 >> 1) - 1, vm);
    load(k0 >> 1, v0);
    load((k0 >> 1) + 1, vp);
    load((k0 >> 1) + 2, vq);
    for (int k = k0; k < k1; k += 4) {
        float* c = ef + (long)k * NP;
        const int nq = min(4, k1 - k);  // 2 or 4 (every extent of a coarsened grid is even)
        float o[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) o[q] = q < nq ? c[q * NP] : 0.f;
        o[0] += corr(v0, vm);  // plane 2K: K and K-1
        o[1] += corr(v0, vp);  // 2K+1: K and K+1
        o[2] += corr(vp, v0);  // 2K+2: K+1 and K
        o[3] += corr(vp, vq);  // 2K+3: K+1 and K+2
#pragma unroll
        for (int q = 0; q < 4; ++q)
            if (q < nq) c[q * NP] = o[q];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            vm[q] = vp[q];
            v0[q] = vq[q];
        }
        load((k >> 1) + 3, vp);
        load((k >> 1) + 4, vq);
    }
}

template <int DIM>
__global__ void k_resid_restrict(Geom gf, Geom gc, const float* b0, const float* b1, const float* b2, const float* e,
                                 const float* r, float* rc, float* ec) {
    const float* beta[3] = {b0, b1, b2};
    long t = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t < gc.N) ops::resid_restrict_at<Ld, float, DIM>(gf, gc, beta, e, r, rc, ec, t);
}

template <int DIM>
__global__ void k_prolong(Geom gf, Geom gc, const float* ec, float* e) {
    long c = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (c < gf.N) ops::prolong_at<Ld, float, DIM>(gf, gc, ec, e, c);
}

// inverse of the coarsest level's shifted matrix, once per solve (one block)
template <int DIM>
__global__ void k_coarse_invert(Geom g, const float* b0, const float* b1, const float* b2, float* ainv) {
    const float* beta[3] = {b0, b1, b2};
    __shared__ float A[kMaxCoarse * kMaxCoarse + 1];
    __shared__ float fct[kMaxCoarse];
    __shared__ float sh;
    ops::coarse_invert_block<Ld, float, DIM>(g, beta, A, fct, &sh);
    const int n = (int)g.N;
    for (int t = threadIdx.x; t <= n * n; t += blockDim.x) ainv[t] = A[t];  // inverse and shift
}

// coarsest-level correction: the FP64 solve of A e = r (every V-cycle)
template <int DIM>
__global__ void k_coarse(Geom g, const float* b0, const float* b1, const float* b2, const float* ainv,
                         const float* r, float* e) {
    const float* beta[3] = {b0, b1, b2};
    __shared__ double rd[kMaxCoarse], ed[kMaxCoarse], rr[kMaxCoarse];
    ops::coarse_apply_block<Ld, float, DIM>(g, beta, ainv, r, e, rd, ed, rr);
}

template <typename T>
__global__ void k_update(long N, PT<T>* p, const float* e) {
    long c = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (c < N) p[c] = ops::p_add(p[c], e[c]);
}

template <typename X>
__global__ void k_partial_sum(long N, const X* x, double* part) {
    ops::SumAcc<X> acc;
    const long stride = (long)gridDim.x * blockDim.x;
    for (long c = (long)blockIdx.x * blockDim.x + threadIdx.x; c < N; c += stride) acc.add(x[c]);
    const double a = block_sum(acc.value());
    if (threadIdx.x == 0) part[blockIdx.x] = a;
}

__global__ void k_partial_sum_df(long N, const float2* x, double* part) {
    float2 acc = make_float2(0.f, 0.f);
    const long stride = (long)gridDim.x * blockDim.x;
    for (long c = (long)blockIdx.x * blockDim.x + threadIdx.x; c < N; c += stride) acc = ops::dfl::add(acc, x[c]);
    const double a = block_sum(ops::dfl::to_double(acc));
    if (threadIdx.x == 0) part[blockIdx.x] = a;
}

// p -= mean (mean: the FP64 value, or its double-float copy in the FP32-mixed form)
template <typename T>
__global__ void k_sub_mean_p(long N, PT<T>* p, const double* mean, const float* mean_df) {
    long c = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= N) return;
    if constexpr (sizeof(T) == 8) p[c] = p[c] - *mean;
    else p[c] = ops::dfl::sub(p[c], make_float2(mean_df[0], mean_df[1]));
}

// the FP32-mixed form's p -= mean on 16-byte words (two double-float cells a
// thread; N even)
__global__ void k_sub_mean_p2(long N2, float4* p, const float* mean_df) {
    long t = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= N2) return;
    const float2 m = make_float2(mean_df[0], mean_df[1]);
    const float4 v = p[t];
    const float2 a = ops::dfl::sub(make_float2(v.x, v.y), m), b = ops::dfl::sub(make_float2(v.z, v.w), m);
    p[t] = make_float4(a.x, a.y, b.x, b.y);
}

template <typename T>
__global__ void k_p_extrap(long N, PT<T>* p, const PT<T>* hnew, const PT<T>* hold) {
    long c = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (c < N) p[c] = ops::p_extrap(hnew[c], hold[c]);
}

// host-side conversions of the FP32-mixed level-0 arrays through an FP64 buffer
__global__ void k_p_to_double(long N, const float2* p, double* x) {
    long c = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (c < N) x[c] = ops::dfl::to_double(p[c]);
}
__global__ void k_p_from_double(long N, float2* p, const double* x) {
    long c = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (c < N) p[c] = ops::dfl::from_double(x[c]);
}
__global__ void k_f_to_double(long N, const float* f, const float* mean_df, double* x) {
    long c = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (c < N) x[c] = (double)f[c] - ops::dfl::to_double(make_float2(mean_df[0], mean_df[1]));
}
__global__ void k_f_from_double(long N, float* f, const double* x) {
    long c = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (c < N) f[c] = (float)x[c];
}

template <typename T, int DIM>
__global__ void k_project(Geom g, PhysDev ph, const T* phi, T* u0, T* u1, T* u2, T cdt, const PT<T>* p) {
    T* us[3] = {u0, u1, u2};
    long c = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (c < g.N) ops::project_at<Ld, T, DIM>(g, ph, phi, us, cdt, p, c);
}

// 3D projection with the arithmetic of ops::project_at (faces of x, y, z in
// that order; the wall face of z stays zero): one thread per (x, y) column
// marching over kProjectZ planes, neighbour offsets formed once.
constexpr int kProjectZ = 8;
template <typename T>
__global__ void __launch_bounds__(256) k_project3(Geom g, PhysDev ph, const T* __restrict__ phi, T* u0, T* u1,
                                                  T* u2, T cdt, const PT<T>* __restrict__ p) {
    T* us[3] = {u0, u1, u2};
    const int i = blockIdx.x * 32 + threadIdx.x, j = blockIdx.y * 8 + threadIdx.y;
    const int nx = g.n[0], ny = g.n[1], nz = g.n[2];
    const long NP = g.NP;
    const long dm[3] = {i == 0 ? nx - 1 : -1, j == 0 ? (long)(ny - 1) * nx : -(long)nx, -NP};
    const T ih = g_ih<T>(g), dr = phys<T>(ph).drho, rho2 = phys<T>(ph).rho2;
    const long pidx = (long)i + (long)nx * j;
    const int k0 = blockIdx.z * kProjectZ, k1 = min(k0 + kProjectZ, nz);
    // the cell below (the z face's other side): the previous plane's values
    T phib = k0 > 0 ? __ldg(phi + pidx + (long)(k0 - 1) * NP) : T(0);
    PT<T> pb = k0 > 0 ? __ldg(p + pidx + (long)(k0 - 1) * NP) : PT<T>{};
    for (int k = k0; k < k1; ++k) {
        const long c = pidx + (long)k * NP;
        const T phic = __ldg(phi + c);
        const PT<T> pc = __ldg(p + c);
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            if (a == 2 && k == 0) continue;  // wall face stays zero
            const long cL = c + dm[a];
            const T phiL = a == 2 ? phib : __ldg(phi + cL);
            const PT<T> pL = a == 2 ? pb : __ldg(p + cL);
            const T rf = T(0.5) * ((dr * phiL + rho2) + (dr * phic + rho2));
            const T beta = T(1) / rf;
            const T dpv = ops::p_diff(pc, pL) * ih;
            us[a][c] = us[a][c] - cdt * beta * dpv;
        }
        phib = phic;
        pb = pc;
    }
}

// k_project3 of the FP32-mixed form with nx a multiple of 4: four cells of one
// x row a thread on float4 words (double-float p: two float4 words), the
// arithmetic of project_at term for term; 64 x-quads x 4 rows of one z plane
// a block (kCoefX x kCoefY)
__global__ void __launch_bounds__(kCoefX * kCoefY)
    k_project4(Geom g, PhysDev ph, const float* __restrict__ phi, float* u0, float* u1, float* u2, float cdt,
               const float2* __restrict__ p) {
    const int q = blockIdx.x * kCoefX + threadIdx.x, j = blockIdx.y * kCoefY + threadIdx.y;
    const int nx = g.n[0], ny = g.n[1], k = blockIdx.z;
    if (4 * q >= nx || j >= ny) return;
    const long row = (long)nx * ((long)j + (long)ny * k);
    const long c = row + 4L * q;
    const float ih = g.ihf, dr = phys<float>(ph).drho, rho2 = phys<float>(ph).rho2;
    auto ld4 = [](const float* a, long i, float* v) {
        const float4 w = __ldg(reinterpret_cast<const float4*>(a + i));
        v[0] = w.x;
        v[1] = w.y;
        v[2] = w.z;
        v[3] = w.w;
    };
    auto ldp4 = [](const float2* a, long i, float2* v) {
        const float4 w0 = __ldg(reinterpret_cast<const float4*>(a + i));
        const float4 w1 = __ldg(reinterpret_cast<const float4*>(a + i + 2));
        v[0] = make_float2(w0.x, w0.y);
        v[1] = make_float2(w0.z, w0.w);
        v[2] = make_float2(w1.x, w1.y);
        v[3] = make_float2(w1.z, w1.w);
    };
    float phic[4];
    float2 pc[4];
    ld4(phi, c, phic);
    ldp4(p, c, pc);
    float* us[3] = {u0, u1, u2};
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        if (a == 2 && k == 0) continue;  // wall face stays zero
        float phiL[4];
        float2 pL[4];
        if (a == 0) {
            const long xm = q == 0 ? row + nx - 1 : c - 1;
            phiL[0] = __ldg(phi + xm);
            pL[0] = __ldg(p + xm);
#pragma unroll
            for (int e = 1; e < 4; ++e) {
                phiL[e] = phic[e - 1];
                pL[e] = pc[e - 1];
            }
        } else {
            const long cL = a == 1 ? ((j == 0) ? c + (long)(ny - 1) * nx : c - nx) : c - g.NP;
            ld4(phi, cL, phiL);
            ldp4(p, cL, pL);
        }
        float4 u = *reinterpret_cast<const float4*>(us[a] + c);
        float uv[4] = {u.x, u.y, u.z, u.w};
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const float rf = 0.5f * ((dr * phiL[e] + rho2) + (dr * phic[e] + rho2));
            const float beta = 1.f / rf;
            const float dpv = ops::p_diff(pc[e], pL[e]) * ih;
            uv[e] = uv[e] - cdt * beta * dpv;
        }
        *reinterpret_cast<float4*>(us[a] + c) = make_float4(uv[0], uv[1], uv[2], uv[3]);
    }
}

template <typename T>
__global__ void k_mass_partial(long N, const T* phi, double* part) {
    double acc = 0.0;
    const long stride = (long)gridDim.x * blockDim.x;
    for (long c = (long)blockIdx.x * blockDim.x + threadIdx.x; c < N; c += stride) acc += (double)phi[c];
    acc = block_sum(acc);
    if (threadIdx.x == 0) part[blockIdx.x] = acc;
}

template <typename T>
__global__ void k_umax_partial(long n0, long n1, long n2, const T* u0, const T* u1, const T* u2, double* part) {
    T m = T(0);
    const long stride = (long)gridDim.x * blockDim.x;
    for (long c = (long)blockIdx.x * blockDim.x + threadIdx.x; c < n0; c += stride) m = fmax(m, fabs(u0[c]));
    for (long c = (long)blockIdx.x * blockDim.x + threadIdx.x; c < n1; c += stride) m = fmax(m, fabs(u1[c]));
    for (long c = (long)blockIdx.x * blockDim.x + threadIdx.x; c < n2; c += stride) m = fmax(m, fabs(u2[c]));
    const double a = block_max((double)m);
    if (threadIdx.x == 0) part[blockIdx.x] = a;
}

__global__ void k_gamma_final(const double* part, int np, double floor_gamma, double* umax, double* gamma,
                              float* gammaf) {
    double v = 0.0;
    for (int t = threadIdx.x; t < np; t += blockDim.x) v = fmax(v, part[t]);
    v = block_max(v);
    if (threadIdx.x == 0) {
        *umax = v;
        *gamma = fmax(2.5 * v, floor_gamma);
        *gammaf = (float)*gamma;
    }
}

// contact line on one wall from the wall-column arrays (phi_w, psi_w, d_n psi_w)
__global__ void k_contact_line(int D, int nx, int nlines, double h, const double* cols, long NP, double* theta_out,
                               double* wetted_out) {
    const double* phw = cols;
    const double* psw = cols + NP;
    const double* dnw = cols + 2 * NP;
    double th_sum = 0.0, cnt = 0.0, len_sum = 0.0;
    for (int line = threadIdx.x; line < nlines; line += blockDim.x) {
        const long base = (long)line * nx;
        // the neighbouring lines (3D: the y derivative of the wall psi)
        const long bup = (long)((line + 1) % nlines) * nx, bdn = (long)((line + nlines - 1) % nlines) * nx;
        auto wrapi = [&](int i) { i %= nx; return i < 0 ? i + nx : i; };
        int i0 = 0;
        for (int i = 1; i < nx; ++i)
            if (phw[base + i] < phw[base + i0]) i0 = i;
        double xl = 0.0, xr = 0.0, thl = 0.0, thr = 0.0;
        bool have_l = false, have_r = false;
        for (int kk = 1; kk <= nx && !have_r; ++kk) {
            const int ip = i0 + kk - 1, ic = i0 + kk;
            const double a0 = phw[base + wrapi(ip)], a1 = phw[base + wrapi(ic)];
            const bool crossing = (!have_l) ? (a0 < 0.5 && a1 >= 0.5) : (a0 >= 0.5 && a1 < 0.5);
            if (!crossing) continue;
            const double t = (0.5 - a0) / (a1 - a0);
            const double x = ((double)ip + 0.5 + t) * h;
            const double gn0 = dnw[base + wrapi(ip)], gn1 = dnw[base + wrapi(ic)];
            const double gt0 = (psw[base + wrapi(ip + 1)] - psw[base + wrapi(ip - 1)]) / (2.0 * h);
            const double gt1 = (psw[base + wrapi(ic + 1)] - psw[base + wrapi(ic - 1)]) / (2.0 * h);
            const double gn = gn0 + t * (gn1 - gn0), gt = gt0 + t * (gt1 - gt0);
            // theta = acos(-d_n psi / |grad psi|) with the whole wall gradient
            double gm;
            if (D == 3) {
                const double gy0 = (psw[bup + wrapi(ip)] - psw[bdn + wrapi(ip)]) / (2.0 * h);
                const double gy1 = (psw[bup + wrapi(ic)] - psw[bdn + wrapi(ic)]) / (2.0 * h);
                const double gy = gy0 + t * (gy1 - gy0);
                gm = sqrt(gn * gn + gt * gt + gy * gy);
            } else {
                gm = sqrt(gn * gn + gt * gt);
            }
            double cv = -gn / gm;
            cv = fmin(fmax(cv, -1.0), 1.0);
            const double th = acos(cv);
            if (!have_l) { xl = x; thl = th; have_l = true; }
            else { xr = x; thr = th; have_r = true; }
        }
        if (have_l && have_r) {
            th_sum += thl + thr;
            cnt += 2.0;
            len_sum += (D == 3) ? (xr - xl) * h : (xr - xl);
        }
    }
    th_sum = block_sum(th_sum);
    __syncthreads();
    cnt = block_sum(cnt);
    __syncthreads();
    len_sum = block_sum(len_sum);
    if (threadIdx.x == 0) {
        if (cnt == 0.0) {
            *theta_out = nan("");
            *wetted_out = 0.0;
        } else {
            *theta_out = th_sum / cnt;
            *wetted_out = (D == 2) ? len_sum : 2.0 * sqrt(len_sum / 3.14159265358979323846);
        }
    }
}

}  // namespace

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
template <typename T>
void launch_div(const Geom& g, const T* const* us, double inv_cdt, MG& mg, cudaStream_t s) {
    const bool on = prof_before(KC_DIV, s);
    FT<T>* f = ops::fbuf<T>(mg.lv[0]);
    if constexpr (sizeof(T) == 4) {
        if (g.D == 3 && g.n[0] % 4 == 0) {
            const unsigned G4 = red_blocks((const void*)k_div4, g.N / 4);
            k_div4<<<G4, kThreads, 0, s>>>(g, us[0], us[1], us[2], (float)inv_cdt, f, mg.partials);
            prof_after(on, s);
            k_final_sum<<<1, 1024, 0, s>>>(mg.partials, (int)G4, 1.0 / (double)g.N, mg.scal + S_MEAN, 0);
            g_launches += 2;
            return;
        }
    }
    const unsigned G = red_blocks(g.D == 2 ? (const void*)k_div<T, 2> : (const void*)k_div<T, 3>, g.N);
    if (g.D == 2)
        k_div<T, 2><<<G, kThreads, 0, s>>>(g, us[0], us[1], nullptr, (T)inv_cdt, f, mg.partials);
    else
        k_div<T, 3><<<G, kThreads, 0, s>>>(g, us[0], us[1], us[2], (T)inv_cdt, f, mg.partials);
    prof_after(on, s);
    k_final_sum<<<1, 1024, 0, s>>>(mg.partials, (int)G, 1.0 / (double)g.N, mg.scal + S_MEAN, 0);
    g_launches += 2;
}

template <typename T>
void launch_sum_f(const Geom& g, MG& mg, cudaStream_t s) {
    const unsigned G = red_blocks((const void*)k_partial_sum<FT<T>>, g.N);
    k_partial_sum<FT<T>><<<G, kThreads, 0, s>>>(g.N, ops::fbuf<T>(mg.lv[0]), mg.partials);
    k_final_sum<<<1, 1024, 0, s>>>(mg.partials, (int)G, 1.0 / (double)g.N, mg.scal + S_MEAN, 0);
    g_launches += 2;
}

// S_MEAN holds the mean of f: the FP64 form centres f, the FP32-mixed form
// keeps a double-float copy of the mean for its residual; then ||f - mean||
template <typename T>
void launch_sub_mean_and_norm(const Geom& g, MG& mg, cudaStream_t s) {
    const unsigned G =
        red_blocks(sizeof(T) == 8 ? (const void*)k_sub_mean_sq : (const void*)k_fnorm_df, g.N);
    if constexpr (sizeof(T) == 8) {
        k_sub_mean_sq<<<G, kThreads, 0, s>>>(g.N, mg.lv[0].f, mg.scal + S_MEAN, mg.partials);
    } else {
        k_mean_df<<<1, 1, 0, s>>>(mg.scal + S_MEAN, mg.scalf + SF_FMEAN_HI);
        k_fnorm_df<<<G, kThreads, 0, s>>>(g.N, ops::fbuf<float>(mg.lv[0]), mg.scalf + SF_FMEAN_HI, mg.partials);
        ++g_launches;
    }
    k_final_sum<<<1, 1024, 0, s>>>(mg.partials, (int)G, 1.0, mg.scal + S_FNORM, 1);
    g_launches += 2;
}

template <typename T>
void launch_mg_coef(const Geom& g, const PhysDev& ph, const T* phi, MG& mg, cudaStream_t s) {
    MGLevel& L0 = mg.lv[0];
    bool vec = false;
    if constexpr (sizeof(T) == 4) vec = g.D == 3 && g.n[0] % 4 == 0;
    if (vec)
        k_coef0_4<<<dim3((unsigned)((g.n[0] / 4 + kCoefX - 1) / kCoefX), (unsigned)((g.n[1] + kCoefY - 1) / kCoefY),
                         (unsigned)g.n[2]),
                    dim3(kCoefX, kCoefY), 0, s>>>(g, ph, (const float*)phi, L0.bf[0], L0.bf[1], L0.bf[2], L0.rho0);
    else if (g.D == 2)
        k_coef0<T, 2><<<blocks_for(g.N + g.NP), kThreads, 0, s>>>(g, ph, phi, L0.beta[0], L0.beta[1],
                                                                  nullptr, L0.bf[0], L0.bf[1], nullptr, L0.rho0);
    else
        k_coef0<T, 3><<<blocks_for(g.N + g.NP), kThreads, 0, s>>>(g, ph, phi, L0.beta[0], L0.beta[1],
                                                                  L0.beta[2], L0.bf[0], L0.bf[1], L0.bf[2], L0.rho0);
    ++g_launches;
    for (int l = 1; l < mg.nlev; ++l) {
        const MGLevel& F = mg.lv[l - 1];
        MGLevel& C = mg.lv[l];
        const unsigned nb = blocks_for(C.g.N + C.g.NP);
        if (g.D == 2)
            k_coef_restrict<2><<<nb, kThreads, 0, s>>>(F.g, C.g, F.bf[0], F.bf[1], nullptr, C.bf[0], C.bf[1], nullptr);
        else
            k_coef_restrict<3><<<nb, kThreads, 0, s>>>(F.g, C.g, F.bf[0], F.bf[1], F.bf[2], C.bf[0], C.bf[1], C.bf[2]);
        ++g_launches;
    }
    const MGLevel& Lc = mg.lv[mg.nlev - 1];
    if (g.D == 2) k_coarse_invert<2><<<1, 256, 0, s>>>(Lc.g, Lc.bf[0], Lc.bf[1], nullptr, mg.ainv);
    else k_coarse_invert<3><<<1, 256, 0, s>>>(Lc.g, Lc.bf[0], Lc.bf[1], Lc.bf[2], mg.ainv);
    ++g_launches;
}

// level-0 restriction and prolongation: the column-marching 3D kernels where
// the block shape fits, else one thread per cell
template <int DIM>
static void launch_restrict0(const MGLevel& L, MGLevel& C, const float* e, cudaStream_t s) {
    if (DIM == 3 && C.g.n[0] % 32 == 0 && C.g.n[1] % 8 == 0) {
        const dim3 grid((unsigned)(C.g.n[0] / 32), (unsigned)(C.g.n[1] / 8),
                        (unsigned)((C.g.n[2] + kRestrictZ - 1) / kRestrictZ));
        CDI_PROF(KC_RESTRICT0, s, (k_restrict0_3<<<grid, dim3(32, 8), 0, s>>>(L.g, C.g, L.rho0, e, L.r, C.r, C.e)));
    } else {
        CDI_PROF(KC_RESTRICT0, s,
                 (k_resid_restrict0<DIM><<<blocks_for(C.g.N), kThreads, 0, s>>>(L.g, C.g, L.rho0, e, L.r, C.r, C.e)));
    }
    ++g_launches;
}
template <int DIM>
static void launch_prolong0(const MGLevel& L, const MGLevel& C, float* e, cudaStream_t s) {
    // the column kernel where its grid fills the GPU (smaller levels: one thread a cell)
    if (DIM == 3 && L.g.n[0] % 32 == 0 && L.g.n[1] % 8 == 0 && L.g.N >= (1L << 21)) {
        const dim3 grid((unsigned)(L.g.n[0] / 32), (unsigned)(L.g.n[1] / 8),
                        (unsigned)((L.g.n[2] + kProlongZ - 1) / kProlongZ));
        CDI_PROF(KC_PROLONG0, s, (k_prolong0_3<<<grid, dim3(32, 8), 0, s>>>(L.g, C.g, C.e, e)));
    } else {
        CDI_PROF(KC_PROLONG0, s, (k_prolong<DIM><<<blocks_for(L.g.N), kThreads, 0, s>>>(L.g, C.g, C.e, e)));
    }
    ++g_launches;
}

// One V-cycle from level l.  On level 0 (when the single-CTA tail does not
// take it) the first sweep starts from e = 0 and the last one adds e to p;
// returns whether p has been updated.
template <typename T, int DIM>
static bool vcycle_rec(MG& mg, PT<T>* p, int l, int npre, int npost, cudaStream_t s) {
    MGLevel& L = mg.lv[l];
    if (mg.tail_args && l == mg.tail_lt) {
        CDI_PROF(KC_COARSE, s, launch_tail(mg.tail_args, DIM, mg.tail_smem, s));
        ++g_launches;
        return false;
    }
    if (l == mg.nlev - 1) {
        CDI_PROF(KC_COARSE, s, (k_coarse<DIM><<<1, 64, 0, s>>>(L.g, L.bf[0], L.bf[1], L.bf[2], mg.ainv, L.r, L.e)));
        ++g_launches;
        return false;
    }
    const unsigned nb = blocks_for(L.g.N);
    const unsigned nbh = blocks_for(L.g.N / 2);
    const int kc_rbgs = (l == 0) ? KC_RBGS0 : KC_RBGS;
    if (DIM == 3 && l == 0 && L.e2 &&
        (mg.sweep_mode == 1 || mg.sweep_mode == 3 || (mg.sweep_mode == 0 && sweep0_auto(L.g)))) {
        // one-pass sweeps (k_sweep.cu), alternating between the two correction
        // buffers: the first starts from e = 0, the last adds e to p
        float* buf[2] = {L.e, L.e2};
        const SweepMaps* maps = mg.sweep_mode == 3 ? nullptr : mg.maps;
        double* err = mg.scal + S_TMAERR;
        int cur = -1;
        for (int it = 0; it < npre; ++it) {
            const int out = cur == 0 ? 1 : 0;
            CDI_PROF(KC_RBGS0, s,
                     launch_sweep0<T>(L, maps, cur < 0 ? nullptr : buf[cur], buf[out],
                                      cur < 0 ? kSweepFromZero : kSweepPlain, mg.omega, p, err, s));
            ++g_launches;
            cur = out;
        }
        MGLevel& C = mg.lv[1];
        launch_restrict0<DIM>(L, C, buf[cur], s);
        vcycle_rec<T, DIM>(mg, p, 1, npre, npost, s);
        launch_prolong0<DIM>(L, C, buf[cur], s);
        for (int it = 0; it < npost; ++it) {
            const int out = 1 - cur;
            CDI_PROF(KC_RBGS0, s,
                     launch_sweep0<T>(L, maps, buf[cur], buf[out], it == npost - 1 ? kSweepUpdate : kSweepPlain,
                                      mg.omega, p, err, s));
            ++g_launches;
            cur = out;
        }
        return true;
    }
    // one red-black sweep; level 0 forms its coefficients from the cell densities
    const dim3 sweep_grid((unsigned)((L.g.n[0] / 2 + kSweepX - 1) / kSweepX),
                          (unsigned)((L.g.n[1] + kSweepY - 1) / kSweepY), (unsigned)(DIM == 3 ? L.g.n[2] : 1));
    const dim3 sweep_block(kSweepX, kSweepY);
    const float h2h = 0.5f * (float)(L.g.h * L.g.h);
    // first: a pass of the V-cycle's first sweep, whose old correction is zero
    auto sweep = [&](int col, int mode, int first = 0) {
        if (l == 0) {
            if (mode == kSweepFromZero)
                CDI_PROF(kc_rbgs, s,
                         (k_rbgs0<T, DIM, kSweepFromZero><<<sweep_grid, sweep_block, 0, s>>>(L.g, L.rho0, L.e, L.r,
                                                                                              col, h2h, mg.omega, first, p)));
            else if (mode == kSweepUpdate)
                CDI_PROF(kc_rbgs, s,
                         (k_rbgs0<T, DIM, kSweepUpdate><<<sweep_grid, sweep_block, 0, s>>>(L.g, L.rho0, L.e, L.r,
                                                                                            col, h2h, mg.omega, first, p)));
            else
                CDI_PROF(kc_rbgs, s,
                         (k_rbgs0<T, DIM, kSweepPlain><<<sweep_grid, sweep_block, 0, s>>>(L.g, L.rho0, L.e, L.r,
                                                                                           col, h2h, mg.omega, first, p)));
        } else {
            CDI_PROF(kc_rbgs, s,
                     (k_rbgs_rows<DIM><<<sweep_grid, sweep_block, 0, s>>>(L.g, L.bf[0], L.bf[1], L.bf[2], L.e, L.r,
                                                                           col)));
        }
        ++g_launches;
    };
    // the coarser levels' own counts, when set
    const int lpre = (l > 0 && mg.cpre >= 0) ? mg.cpre : npre;
    const int lpost = (l > 0 && mg.cpost >= 0) ? mg.cpost : npost;
    for (int it = 0; it < lpre; ++it)
        for (int col = 0; col < 2; ++col)
            sweep(col, (l == 0 && it == 0 && col == 0) ? kSweepFromZero : kSweepPlain, l == 0 && it == 0);
    MGLevel& C = mg.lv[l + 1];
    if (l == 0) {
        launch_restrict0<DIM>(L, C, L.e, s);
    } else {
        if (DIM == 3 && C.g.n[0] % 32 == 0 && C.g.n[1] % 8 == 0 && L.g.N >= (1L << 21))
            k_restrict_bf3<<<dim3((unsigned)(C.g.n[0] / 32), (unsigned)(C.g.n[1] / 8),
                                  (unsigned)((C.g.n[2] + kRestrictZ - 1) / kRestrictZ)),
                             dim3(32, 8), 0, s>>>(L.g, C.g, L.bf[0], L.bf[1], L.bf[2], L.e, L.r, C.r, C.e);
        else
            k_resid_restrict<DIM><<<blocks_for(C.g.N), kThreads, 0, s>>>(L.g, C.g, L.bf[0], L.bf[1], L.bf[2], L.e,
                                                                         L.r, C.r, C.e);
        ++g_launches;
    }
    vcycle_rec<T, DIM>(mg, p, l + 1, npre, npost, s);
    launch_prolong0<DIM>(L, C, L.e, s);  // any level: the column kernel where the shape fits
    for (int it = 0; it < lpost; ++it)
        for (int col = 0; col < 2; ++col)
            sweep(col, (l == 0 && it == lpost - 1 && col == 1) ? kSweepUpdate : kSweepPlain);
    return l == 0;
}

// one V-cycle on A e = r and p += e (npre, npost >= 1)
template <typename T>
void launch_vcycle(const Geom& g, MG& mg, int npre, int npost, cudaStream_t s) {
    PT<T>* p = ops::pbuf<T>(mg.lv[0]);
    const bool updated = (g.D == 2) ? vcycle_rec<T, 2>(mg, p, 0, npre, npost, s)
                                    : vcycle_rec<T, 3>(mg, p, 0, npre, npost, s);
    if (!updated) {
        k_update<T><<<blocks_for(g.N), kThreads, 0, s>>>(g.N, p, mg.lv[0].e);
        ++g_launches;
    }
}

// residual and |r|^2 partials: the tiled kernel (k_resid.cu) for the
// FP32-mixed form on 3D grids of 64 x 16 tiles (not with the colour-pass
// smoother, which keeps the per-cell kernel: the two are compared bit for bit),
// else one thread a cell
template <typename T>
void launch_resid_norm(const Geom& g, MG& mg, cudaStream_t s) {
    const float* fm = sizeof(T) == 8 ? nullptr : mg.scalf + SF_FMEAN_HI;
    unsigned G;
    const bool on = prof_before(KC_RESID, s);
    if (sizeof(T) == 4 && mg.sweep_mode != 2 && resid_tile_supported(g, kPartials)) {
        G = launch_resid_tile(mg.lv[0], fm, mg.partials, kPartials, s);
    } else {
        G = red_blocks(g.D == 2 ? (const void*)k_resid<T, 2> : (const void*)k_resid<T, 3>, g.N);
        if (g.D == 2) k_resid<T, 2><<<G, kThreads, 0, s>>>(mg.lv[0], fm, mg.partials);
        else k_resid<T, 3><<<G, kThreads, 0, s>>>(mg.lv[0], fm, mg.partials);
    }
    prof_after(on, s);
    k_final_sum<<<1, 1024, 0, s>>>(mg.partials, (int)G, 1.0, mg.scal + S_RNORM, 1);
    g_launches += 2;
}

template <typename T>
void launch_p_mean_remove(const Geom& g, MG& mg, cudaStream_t s) {
    const unsigned G =
        red_blocks(sizeof(T) == 8 ? (const void*)k_partial_sum<double> : (const void*)k_partial_sum_df, g.N);
    if constexpr (sizeof(T) == 8) {
        k_partial_sum<double><<<G, kThreads, 0, s>>>(g.N, mg.lv[0].p, mg.partials);
    } else {
        k_partial_sum_df<<<G, kThreads, 0, s>>>(g.N, ops::pbuf<float>(mg.lv[0]), mg.partials);
    }
    k_final_sum<<<1, 1024, 0, s>>>(mg.partials, (int)G, 1.0 / (double)g.N, mg.scal + S_MEAN, 0);
    if constexpr (sizeof(T) == 4) {
        k_mean_df<<<1, 1, 0, s>>>(mg.scal + S_MEAN, mg.scalf + SF_PMEAN_HI);
        ++g_launches;
    }
    if (sizeof(T) == 4 && g.N % 2 == 0)
        k_sub_mean_p2<<<blocks_for(g.N / 2), kThreads, 0, s>>>(g.N / 2, reinterpret_cast<float4*>(mg.lv[0].p),
                                                                mg.scalf + SF_PMEAN_HI);
    else
        k_sub_mean_p<T><<<blocks_for(g.N), kThreads, 0, s>>>(g.N, ops::pbuf<T>(mg.lv[0]), mg.scal + S_MEAN,
                                                            mg.scalf + SF_PMEAN_HI);
    g_launches += 3;
}

template <typename T>
void launch_p_extrap(const Geom& g, MG& mg, const double* hnew, const double* hold, cudaStream_t s) {
    k_p_extrap<T><<<blocks_for(g.N), kThreads, 0, s>>>(g.N, ops::pbuf<T>(mg.lv[0]),
                                                      reinterpret_cast<const PT<T>*>(hnew),
                                                      reinterpret_cast<const PT<T>*>(hold));
    ++g_launches;
}
template void launch_p_extrap<double>(const Geom&, MG&, const double*, const double*, cudaStream_t);
template void launch_p_extrap<float>(const Geom&, MG&, const double*, const double*, cudaStream_t);

void launch_p_to_double(const Geom& g, const MG& mg, double* x, cudaStream_t s) {
    k_p_to_double<<<blocks_for(g.N), kThreads, 0, s>>>(g.N, ops::pbuf<float>(mg.lv[0]), x);
    ++g_launches;
}
void launch_p_from_double(const Geom& g, MG& mg, const double* x, cudaStream_t s) {
    k_p_from_double<<<blocks_for(g.N), kThreads, 0, s>>>(g.N, ops::pbuf<float>(mg.lv[0]), x);
    ++g_launches;
}
void launch_f_to_double(const Geom& g, const MG& mg, double* x, cudaStream_t s) {
    k_f_to_double<<<blocks_for(g.N), kThreads, 0, s>>>(g.N, ops::fbuf<float>(mg.lv[0]), mg.scalf + SF_FMEAN_HI, x);
    ++g_launches;
}
void launch_f_from_double(const Geom& g, MG& mg, const double* x, cudaStream_t s) {
    k_f_from_double<<<blocks_for(g.N), kThreads, 0, s>>>(g.N, ops::fbuf<float>(mg.lv[0]), x);
    ++g_launches;
}

template <typename T>
void launch_project(const Geom& g, const PhysDev& ph, const T* phi, T* const* us, double cdt, const double* p,
                    cudaStream_t s) {
    const bool on = prof_before(KC_PROJECT, s);
    const PT<T>* pp = reinterpret_cast<const PT<T>*>(p);
    bool vec = false;
    if constexpr (sizeof(T) == 4) vec = g.D == 3 && g.n[0] % 4 == 0;
    if (vec)
        k_project4<<<dim3((unsigned)((g.n[0] / 4 + kCoefX - 1) / kCoefX), (unsigned)((g.n[1] + kCoefY - 1) / kCoefY),
                          (unsigned)g.n[2]),
                     dim3(kCoefX, kCoefY), 0, s>>>(g, ph, (const float*)phi, (float*)us[0], (float*)us[1],
                                                   (float*)us[2], (float)cdt, (const float2*)pp);
    else if (g.D == 2)
        k_project<T, 2><<<blocks_for(g.N), kThreads, 0, s>>>(g, ph, phi, us[0], us[1], nullptr, (T)cdt, pp);
    else if (g.n[0] % 32 == 0 && g.n[1] % 8 == 0)
        k_project3<T><<<dim3((unsigned)(g.n[0] / 32), (unsigned)(g.n[1] / 8), (unsigned)((g.n[2] + kProjectZ - 1) / kProjectZ)),
                        dim3(32, 8), 0, s>>>(g, ph, phi, us[0], us[1], us[2], (T)cdt, pp);
    else
        k_project<T, 3><<<blocks_for(g.N), kThreads, 0, s>>>(g, ph, phi, us[0], us[1], us[2], (T)cdt, pp);
    prof_after(on, s);
    ++g_launches;
}

template <typename T>
void launch_mass(const Geom& g, const T* phi, MG& mg, cudaStream_t s) {
    const unsigned G = red_blocks((const void*)k_mass_partial<T>, g.N);
    k_mass_partial<T><<<G, kThreads, 0, s>>>(g.N, phi, mg.partials);
    double dv = (g.D == 2) ? g.h * g.h : g.h * g.h * g.h;
    k_final_sum<<<1, 1024, 0, s>>>(mg.partials, (int)G, dv, mg.scal + S_MASS, 0);
    g_launches += 2;
}

template <typename T>
void launch_gamma(const Geom& g, const T* const* u, double gamma_param, MG& mg, cudaStream_t s) {
    const unsigned G = red_blocks((const void*)k_umax_partial<T>, g.N + g.NP);
    long n2 = (g.D == 3) ? g.N + g.NP : 0;
    long n1 = (g.D == 2) ? g.N + g.NP : g.N;
    k_umax_partial<T><<<G, kThreads, 0, s>>>(g.N, n1, n2, u[0], u[1], g.D == 3 ? u[2] : u[1], mg.partials);
    k_gamma_final<<<1, 1024, 0, s>>>(mg.partials, (int)G, -gamma_param, mg.scal + S_UMAX, mg.scal + S_GAMMA,
                                     mg.scalf + SF_GAMMA);
    g_launches += 2;
}

void launch_contact_line(const Geom& g, int wall, const double* cols, MG& mg, cudaStream_t s) {
    const int nlines = (g.D == 3) ? g.n[1] : 1;
    k_contact_line<<<1, 256, 0, s>>>(g.D, g.n[0], nlines, g.h, cols + (long)wall * 3 * g.NP, g.NP, mg.scal + S_THETA,
                                     mg.scal + S_WETTED);
    ++g_launches;
}

template void launch_sum_f<double>(const Geom&, MG&, cudaStream_t);
template void launch_sum_f<float>(const Geom&, MG&, cudaStream_t);
template void launch_sub_mean_and_norm<double>(const Geom&, MG&, cudaStream_t);
template void launch_sub_mean_and_norm<float>(const Geom&, MG&, cudaStream_t);
template void launch_vcycle<double>(const Geom&, MG&, int, int, cudaStream_t);
template void launch_vcycle<float>(const Geom&, MG&, int, int, cudaStream_t);
template void launch_resid_norm<double>(const Geom&, MG&, cudaStream_t);
template void launch_resid_norm<float>(const Geom&, MG&, cudaStream_t);
template void launch_p_mean_remove<double>(const Geom&, MG&, cudaStream_t);
template void launch_p_mean_remove<float>(const Geom&, MG&, cudaStream_t);
template void launch_div<double>(const Geom&, const double* const*, double, MG&, cudaStream_t);
template void launch_div<float>(const Geom&, const float* const*, double, MG&, cudaStream_t);
template void launch_mg_coef<double>(const Geom&, const PhysDev&, const double*, MG&, cudaStream_t);
template void launch_mg_coef<float>(const Geom&, const PhysDev&, const float*, MG&, cudaStream_t);
template void launch_project<double>(const Geom&, const PhysDev&, const double*, double* const*, double, const double*,
                                     cudaStream_t);
template void launch_project<float>(const Geom&, const PhysDev&, const float*, float* const*, double, const double*,
                                    cudaStream_t);
template void launch_mass<double>(const Geom&, const double*, MG&, cudaStream_t);
template void launch_mass<float>(const Geom&, const float*, MG&, cudaStream_t);
template void launch_gamma<double>(const Geom&, const double* const*, double, MG&, cudaStream_t);
template void launch_gamma<float>(const Geom&, const float* const*, double, MG&, cudaStream_t);

}  // namespace cdi
