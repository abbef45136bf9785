// Standalone kernels of one right-hand-side evaluation and of the RK4 stage
// update (one thread per cell or wall-plane position).  The arithmetic lives
// in ops.cuh; these kernels serve the stage-level C-ABI calls (cdi_eval_rhs,
// cdi_eval_wall, cdi_contact_angle) and the launch-per-kernel step path.
//
//   k_psi        psi = eps ln(phi/(1-phi))                                     Eq. (psi)
//   k_cell       grad psi, lap psi, normal, chemical potential                 Eqs. (chemical potential),
//                                                                               (curvature), Sec. 4
//   k_wall       wall rows: extrapolation, GNBC slip u^Y, ghost velocity        Eqs. (slip BC), (u_slip_v),
//                                                                               (u_slip_Y), Sec. 3, Sec. 4
//   k_phi_rhs    phi flux, its divergence, consistent mass flux                 Eqs. (CDI), (no-flux BC)
//   k_mom        momentum right-hand side                                      Eqs. (NS_momentum), (EB)
//   k_stage_*    RK4 stage values of phi and rho_f u, stage velocity u*        Sec. 4
//
// No ghost value of phi is ever formed: wall-normal stencils and
// extrapolations read interior rows only (Sec. 4).
#include "ops.cuh"

namespace cdi {

thread_local long g_launches = 0;
thread_local Profiler g_prof;
const char* const kKernelClassNames[KC_COUNT] = {"psi", "cell", "wall", "phi_rhs", "mom", "stage_phi", "stage_mom",
                                                 "div", "rbgs0", "rbgs", "resid_restrict0", "prolong0", "coarse",
                                                 "resid", "project", "step"};

namespace {

constexpr int kThreads = 256;
inline unsigned blocks_for(long n) { return (unsigned)((n + kThreads - 1) / kThreads); }
using Ld = ops::LdPlain;

template <typename T>
__global__ void k_psi(Geom g, PhysDev ph, const T* phi, T* psi) {
    long c = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (c < g.N) ops::psi_at<Ld>(g, ph, phi, psi, c);
}

template <typename T, int DIM>
__global__ void k_cell(Geom g, PhysDev ph, const T* phi, const T* psi, T* nh0, T* nh1, T* nh2, T* muc) {
    long c = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (c < g.N) ops::cell_at<Ld, T, DIM>(g, ph, phi, psi, nh0, nh1, nh2, muc, c);
}

template <typename T, int DIM>
__global__ void k_wall(Geom g, PhysDev ph, const T* phi, const T* psi, const T* u0, const T* u1, T* wuY, T* wghost,
                       T* wmuw) {
    long t = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t < 2 * g.NP) ops::wall_at<Ld, T, DIM>(g, ph, phi, psi, u0, u1, wuY, wghost, wmuw, t);
}

// column quantities (phi_w, psi_w, d_n psi_w) for the contact line
template <typename T, int DIM>
__global__ void k_wall_cols(Geom g, PhysDev ph, const T* phi, const T* psi, double* cols) {
    long t = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= 2 * g.NP) return;
    const int s = (int)(t / g.NP);
    const long pidx = t - s * g.NP;
    const int i = (int)(pidx % g.n[0]);
    const int j = (DIM == 3) ? (int)(pidx / g.n[0]) : 0;
    const ops::ColQ<T> q = ops::wall_column<Ld, T, DIM>(g, ph, phi, psi, s, i, j);
    double* base = cols + (long)s * 3 * g.NP;
    base[pidx] = (double)q.phiw;
    base[g.NP + pidx] = (double)q.psiw;
    base[2 * g.NP + pidx] = (double)q.dnw;
}

// gamma of the step in the kernel's type (the FP32 copy in FP32 kernels)
__device__ __forceinline__ double stage_gamma(const StageFields<double>& f) { return *f.gamma; }
__device__ __forceinline__ float stage_gamma(const StageFields<float>& f) { return *f.gammaf; }

template <typename T, int DIM>
__global__ void k_phi_rhs(Geom g, PhysDev ph, StageFields<T> f) {
    long c = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (c < g.N) ops::phi_rhs_at<Ld, T, DIM>(g, ph, f, stage_gamma(f), c);
}

template <typename T, int DIM>
__global__ void k_mom(Geom g, PhysDev ph, StageFields<T> f) {
    long c = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (c < g.N) ops::mom_at<Ld, T, DIM>(g, ph, f, c);
}

// 3D cell-centre quantities with the arithmetic of ops::cell_at (the same
// terms in the same order: derivatives along x, y, z; central inside, the
// second-order one-sided wall-normal stencils in the first and last rows,
// Sec. 4): one thread per (x, y) column marching over kCellZ planes, the
// in-plane neighbour offsets (periodic wraps) formed once.  Blocks of 32 x 8
// columns; nx a multiple of 32 and ny of 8.
constexpr int kCellZ = 8;
template <typename T>
__global__ void __launch_bounds__(256) k_cell3(Geom g, PhysDev ph, const T* __restrict__ phi,
                                               const T* __restrict__ psi, T* __restrict__ nh0, T* __restrict__ nh1,
                                               T* __restrict__ nh2, T* __restrict__ muc) {
    const int i = blockIdx.x * 32 + threadIdx.x, j = blockIdx.y * 8 + threadIdx.y;
    const int nx = g.n[0], ny = g.n[1], nz = g.n[2];
    const long NP = g.NP;
    const long dxm = i == 0 ? nx - 1 : -1, dxp = i == nx - 1 ? -(long)(nx - 1) : 1;
    const long dym = j == 0 ? (long)(ny - 1) * nx : -(long)nx, dyp = j == ny - 1 ? -(long)(ny - 1) * nx : (long)nx;
    const T ih = g_ih<T>(g);
    const T half_ih = T(0.5) * ih, ih2 = ih * ih;
    const PhysT<T>& Q = phys<T>(ph);
    const T delta = Q.delta, eps = Q.eps;
    const long pidx = (long)i + (long)nx * j;
    const int k0 = blockIdx.z * kCellZ, k1 = min(k0 + kCellZ, nz);
    for (int k = k0; k < k1; ++k) {
        const long c = pidx + (long)k * NP;
        const T s0 = __ldg(psi + c);
        T gb[3], grad2 = T(0), lap = T(0);
        {  // x
            const T sm = __ldg(psi + c + dxm), sp = __ldg(psi + c + dxp);
            const T d1 = (sp - sm) * half_ih, d2 = (sp - T(2) * s0 + sm) * ih2;
            gb[0] = d1;
            grad2 += d1 * d1;
            lap += d2;
        }
        {  // y
            const T sm = __ldg(psi + c + dym), sp = __ldg(psi + c + dyp);
            const T d1 = (sp - sm) * half_ih, d2 = (sp - T(2) * s0 + sm) * ih2;
            gb[1] = d1;
            grad2 += d1 * d1;
            lap += d2;
        }
        {  // z: the wall axis
            T d1, d2;
            if (k == 0) {
                const T s1 = __ldg(psi + c + NP), s2 = __ldg(psi + c + 2 * NP), s3 = __ldg(psi + c + 3 * NP);
                d1 = (T(-3) * s0 + T(4) * s1 - s2) * half_ih;
                d2 = (T(2) * s0 - T(5) * s1 + T(4) * s2 - s3) * ih2;
            } else if (k == nz - 1) {
                const T s1 = __ldg(psi + c - NP), s2 = __ldg(psi + c - 2 * NP), s3 = __ldg(psi + c - 3 * NP);
                d1 = (T(3) * s0 - T(4) * s1 + s2) * half_ih;
                d2 = (T(2) * s0 - T(5) * s1 + T(4) * s2 - s3) * ih2;
            } else {
                const T sm = __ldg(psi + c - NP), sp = __ldg(psi + c + NP);
                d1 = (sp - sm) * half_ih;
                d2 = (sp - T(2) * s0 + sm) * ih2;
            }
            gb[2] = d1;
            grad2 += d1 * d1;
            lap += d2;
        }
        T pt = clampv(__ldg(phi + c), delta, T(1) - delta);
        T P = pt * (T(1) - pt);
        muc[c] = T(6) * Q.sigma * (P * (T(1) - T(2) * pt) * (T(1) - grad2) / eps - P * lap);
        const T igm = T(1) / (sqrt(grad2) + Q.tau);
        nh0[c] = gb[0] * igm;
        nh1[c] = gb[1] * igm;
        nh2[c] = gb[2] * igm;
    }
}

// 3D phi right-hand side and mass flux with the arithmetic of ops::phi_rhs_at
// (faces of axes x, y, z in that order; the low face flux and the high face
// flux from ops::phi_flux, zero on the walls): one thread per (x, y) column
// marching over kCellZ planes, neighbour offsets formed once.
template <typename T>
__global__ void __launch_bounds__(256) k_phi_rhs3(Geom g, PhysDev ph, StageFields<T> f) {
    using Ld = ops::LdPlain;
    const int i = blockIdx.x * 32 + threadIdx.x, j = blockIdx.y * 8 + threadIdx.y;
    const int nx = g.n[0], ny = g.n[1], nz = g.n[2];
    const long NP = g.NP;
    const long dm[2] = {i == 0 ? nx - 1 : -1, j == 0 ? (long)(ny - 1) * nx : -(long)nx};
    const long dp[2] = {i == nx - 1 ? -(long)(nx - 1) : 1, j == ny - 1 ? -(long)(ny - 1) * nx : (long)nx};
    const T ih = g_ih<T>(g);
    const PhysT<T>& Q = phys<T>(ph);
    const T eps = Q.eps, delta = Q.delta, drho = Q.drho, rho2 = Q.rho2;
    const T gamma = stage_gamma(f);
    const long pidx = (long)i + (long)nx * j;
    const int k0 = blockIdx.z * kCellZ, k1 = min(k0 + kCellZ, nz);
    for (int k = k0; k < k1; ++k) {
        const long c = pidx + (long)k * NP;
        T div = T(0);
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const T* ua = f.u[a];
            const T* na = f.nh[a];
            T Flo = T(0), Fhi = T(0);
            const T ulo = __ldg(ua + c);
            const bool wlo = a == 2 && k == 0, whi = a == 2 && k == nz - 1;
            const long cL = a < 2 ? c + dm[a] : c - NP, cR = a < 2 ? c + dp[a] : c + NP;
            if (!wlo) Flo = ops::phi_flux<Ld>(f.phi, na, cL, c, ulo, gamma, eps, ih, delta);
            if (!whi) Fhi = ops::phi_flux<Ld>(f.phi, na, c, cR, __ldg(ua + cR), gamma, eps, ih, delta);
            div += Fhi - Flo;
            f.m[a][c] = wlo ? T(0) : drho * Flo + rho2 * ulo;
        }
        f.rphi[c] = -div * ih;
    }
}

template <typename T>
__global__ void k_stage_phi(long N, T b, T cdt, T dt, int first, int last, const T* phi0, const T* rphi, T* acc,
                            T* phik) {
    long c = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (c < N) ops::stage_phi_at<Ld>(b, cdt, dt, first, last, phi0, rphi, acc, phik, c);
}

template <typename T>
struct Ptr3 {
    T* p[3];
};

template <typename T, int DIM>
__global__ void k_stage_mom(Geom g, PhysDev ph, T b, T cdt, T dt, int first, int last, const T* phi0, const T* phik,
                            Ptr3<const T> u0, Ptr3<const T> rm, Ptr3<T> acc, Ptr3<T> uk) {
    long c = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (c < g.N) ops::stage_mom_at<Ld, T, DIM>(g, ph, b, cdt, dt, first, last, phi0, phik, u0.p, rm.p, acc.p, uk.p, c);
}

// FP32 3D grids with nx a multiple of 4: the elementwise stage kernels on
// float4 words (four cells of one x row a thread, 16-byte loads and stores),
// with the arithmetic of psi_at, stage_phi_at and stage_mom_at term for term.
// Thread block: 64 x-quads x 4 rows of one z plane, so no index is decoded.
constexpr int kVecX = 64, kVecY = 4;
__device__ __forceinline__ float v4(const float4& a, int e) { return e == 0 ? a.x : e == 1 ? a.y : e == 2 ? a.z : a.w; }

__global__ void __launch_bounds__(kVecX * kVecY) k_psi4(Geom g, PhysDev ph, const float* __restrict__ phi,
                                                        float* __restrict__ psi) {
    const int q = blockIdx.x * kVecX + threadIdx.x, j = blockIdx.y * kVecY + threadIdx.y;
    if (4 * q >= g.n[0] || j >= g.n[1]) return;
    const long c = 4L * q + (long)g.n[0] * ((long)j + (long)g.n[1] * blockIdx.z);
    const PhysT<float>& P = phys<float>(ph);
    const float4 f = __ldg(reinterpret_cast<const float4*>(phi + c));
    float o[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) {
        const float pt = clampv(v4(f, e), P.delta, 1.f - P.delta);
        o[e] = P.eps * log(pt / (1.f - pt));
    }
    *reinterpret_cast<float4*>(psi + c) = make_float4(o[0], o[1], o[2], o[3]);
}

__global__ void __launch_bounds__(kVecX * kVecY) k_stage_phi4(Geom g, float b, float cdt, float dt, int first,
                                                              int last, const float* __restrict__ phi0,
                                                              const float* __restrict__ rphi, float* acc,
                                                              float* phik) {
    const int q = blockIdx.x * kVecX + threadIdx.x, j = blockIdx.y * kVecY + threadIdx.y;
    if (4 * q >= g.n[0] || j >= g.n[1]) return;
    const long c = 4L * q + (long)g.n[0] * ((long)j + (long)g.n[1] * blockIdx.z);
    const float4 k4 = __ldg(reinterpret_cast<const float4*>(rphi + c));
    const float4 p4 = __ldg(reinterpret_cast<const float4*>(phi0 + c));
    const float4 a4 = first ? make_float4(0.f, 0.f, 0.f, 0.f) : *reinterpret_cast<const float4*>(acc + c);
    float ao[4], po[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) {
        const float k = v4(k4, e);
        const float a = first ? b * k : v4(a4, e) + b * k;
        ao[e] = a;
        po[e] = last ? v4(p4, e) + dt * a : v4(p4, e) + cdt * k;
    }
    *reinterpret_cast<float4*>(acc + c) = make_float4(ao[0], ao[1], ao[2], ao[3]);
    *reinterpret_cast<float4*>(phik + c) = make_float4(po[0], po[1], po[2], po[3]);
}

// the three faces of four cells: the low neighbours' phi (x: the word before,
// or the row's last cell across the periodic seam; y, z: the quads one row and
// one plane back, y periodic, z skipped on the wall plane)
__global__ void __launch_bounds__(kVecX * kVecY)
    k_stage_mom4(Geom g, PhysDev ph, float b, float cdt, float dt, int first, int last,
                 const float* __restrict__ phi0, const float* __restrict__ phik, Ptr3<const float> u0,
                 Ptr3<const float> rm, Ptr3<float> acc, Ptr3<float> uk) {
    const int q = blockIdx.x * kVecX + threadIdx.x, j = blockIdx.y * kVecY + threadIdx.y;
    const int nx = g.n[0], ny = g.n[1], k = blockIdx.z;
    if (4 * q >= nx || j >= ny) return;
    const long row = (long)nx * ((long)j + (long)ny * k);
    const long c = row + 4L * q;
    const float drho = phys<float>(ph).drho, rho2 = phys<float>(ph).rho2;
    const long xm = (q == 0) ? row + nx - 1 : c - 1;
    const long ym = (j == 0) ? c + (long)(ny - 1) * nx : c - nx;
    const float4 p0c = __ldg(reinterpret_cast<const float4*>(phi0 + c));
    const float4 pkc = __ldg(reinterpret_cast<const float4*>(phik + c));
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        float* ua = uk.p[a];
        float* aa = acc.p[a];
        if (a == 2 && k == 0) {  // the wall face
            *reinterpret_cast<float4*>(ua + c) = make_float4(0.f, 0.f, 0.f, 0.f);
            *reinterpret_cast<float4*>(aa + c) = make_float4(0.f, 0.f, 0.f, 0.f);
            continue;
        }
        float p0L[4], pkL[4];
        if (a == 0) {
            p0L[0] = __ldg(phi0 + xm);
            pkL[0] = __ldg(phik + xm);
#pragma unroll
            for (int e = 1; e < 4; ++e) {
                p0L[e] = v4(p0c, e - 1);
                pkL[e] = v4(pkc, e - 1);
            }
        } else {
            const long cL = a == 1 ? ym : c - g.NP;
            const float4 x0 = __ldg(reinterpret_cast<const float4*>(phi0 + cL));
            const float4 xk = __ldg(reinterpret_cast<const float4*>(phik + cL));
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                p0L[e] = v4(x0, e);
                pkL[e] = v4(xk, e);
            }
        }
        const float4 uo = __ldg(reinterpret_cast<const float4*>(u0.p[a] + c));
        const float4 kk = __ldg(reinterpret_cast<const float4*>(rm.p[a] + c));
        const float4 ao = first ? make_float4(0.f, 0.f, 0.f, 0.f) : *reinterpret_cast<const float4*>(aa + c);
        float an[4], un[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const float rf0 = 0.5f * ((drho * p0L[e] + rho2) + (drho * v4(p0c, e) + rho2));
            const float M0 = rf0 * v4(uo, e);
            const float kv = v4(kk, e);
            const float ac = first ? b * kv : v4(ao, e) + b * kv;
            an[e] = ac;
            const float Mv = last ? M0 + dt * ac : M0 + cdt * kv;
            const float rfk = 0.5f * ((drho * pkL[e] + rho2) + (drho * v4(pkc, e) + rho2));
            un[e] = Mv / rfk;
        }
        *reinterpret_cast<float4*>(aa + c) = make_float4(an[0], an[1], an[2], an[3]);
        *reinterpret_cast<float4*>(ua + c) = make_float4(un[0], un[1], un[2], un[3]);
    }
}

__device__ __forceinline__ void ld4(const float* a, long i, float* v) {
    const float4 w = __ldg(reinterpret_cast<const float4*>(a + i));
    v[0] = w.x;
    v[1] = w.y;
    v[2] = w.z;
    v[3] = w.w;
}
__device__ __forceinline__ void st4(float* a, long i, const float* v) {
    *reinterpret_cast<float4*>(a + i) = make_float4(v[0], v[1], v[2], v[3]);
}

// k_cell3 on float4 words: four cells of one x row a thread (the x
// neighbours of the end cells are the words before and after the quad, across
// the periodic seam at the row ends), the terms of k_cell3 in its order
__global__ void __launch_bounds__(kVecX * kVecY)
    k_cell4(Geom g, PhysDev ph, const float* __restrict__ phi, const float* __restrict__ psi, float* __restrict__ nh0,
            float* __restrict__ nh1, float* __restrict__ nh2, float* __restrict__ muc) {
    const int q = blockIdx.x * kVecX + threadIdx.x, j = blockIdx.y * kVecY + threadIdx.y;
    const int nx = g.n[0], ny = g.n[1], nz = g.n[2], k = blockIdx.z;
    if (4 * q >= nx || j >= ny) return;
    const long NP = g.NP;
    const long row = (long)nx * ((long)j + (long)ny * k);
    const long c = row + 4L * q;
    const float ih = g.ihf;
    const float half_ih = 0.5f * ih, ih2 = ih * ih;
    const PhysT<float>& Q = phys<float>(ph);
    const float delta = Q.delta, eps = Q.eps;
    float s0[4], sx[6], ym[4], yp[4], z1[4], z2[4], z3[4], ph4[4];
    ld4(psi, c, s0);
    sx[0] = __ldg(psi + (q == 0 ? row + nx - 1 : c - 1));
    sx[5] = __ldg(psi + (4 * q + 4 == nx ? row : c + 4));
#pragma unroll
    for (int e = 0; e < 4; ++e) sx[e + 1] = s0[e];
    ld4(psi, (j == 0) ? c + (long)(ny - 1) * nx : c - nx, ym);
    ld4(psi, (j == ny - 1) ? c - (long)(ny - 1) * nx : c + nx, yp);
    if (k == 0) {
        ld4(psi, c + NP, z1);
        ld4(psi, c + 2 * NP, z2);
        ld4(psi, c + 3 * NP, z3);
    } else if (k == nz - 1) {
        ld4(psi, c - NP, z1);
        ld4(psi, c - 2 * NP, z2);
        ld4(psi, c - 3 * NP, z3);
    } else {
        ld4(psi, c - NP, z1);  // below
        ld4(psi, c + NP, z2);  // above
    }
    ld4(phi, c, ph4);
    float o0[4], o1[4], o2[4], om[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) {
        float gb[3], grad2 = 0.f, lap = 0.f;
        {  // x
            const float sm = sx[e], sp = sx[e + 2];
            const float d1 = (sp - sm) * half_ih, d2 = (sp - 2.f * s0[e] + sm) * ih2;
            gb[0] = d1;
            grad2 += d1 * d1;
            lap += d2;
        }
        {  // y
            const float sm = ym[e], sp = yp[e];
            const float d1 = (sp - sm) * half_ih, d2 = (sp - 2.f * s0[e] + sm) * ih2;
            gb[1] = d1;
            grad2 += d1 * d1;
            lap += d2;
        }
        {  // z: the wall axis
            float d1, d2;
            if (k == 0) {
                d1 = (-3.f * s0[e] + 4.f * z1[e] - z2[e]) * half_ih;
                d2 = (2.f * s0[e] - 5.f * z1[e] + 4.f * z2[e] - z3[e]) * ih2;
            } else if (k == nz - 1) {
                d1 = (3.f * s0[e] - 4.f * z1[e] + z2[e]) * half_ih;
                d2 = (2.f * s0[e] - 5.f * z1[e] + 4.f * z2[e] - z3[e]) * ih2;
            } else {
                const float sm = z1[e], sp = z2[e];
                d1 = (sp - sm) * half_ih;
                d2 = (sp - 2.f * s0[e] + sm) * ih2;
            }
            gb[2] = d1;
            grad2 += d1 * d1;
            lap += d2;
        }
        const float pt = clampv(ph4[e], delta, 1.f - delta);
        const float P = pt * (1.f - pt);
        om[e] = 6.f * Q.sigma * (P * (1.f - 2.f * pt) * (1.f - grad2) / eps - P * lap);
        const float igm = 1.f / (sqrtf(grad2) + Q.tau);
        o0[e] = gb[0] * igm;
        o1[e] = gb[1] * igm;
        o2[e] = gb[2] * igm;
    }
    st4(muc, c, om);
    st4(nh0, c, o0);
    st4(nh1, c, o1);
    st4(nh2, c, o2);
}

// k_phi_rhs3 on float4 words: four cells of one x row a thread; the five x
// faces of the quad are formed once each (the high face of one cell is the
// low face of the next), each face by ops::phi_flux_v, the terms of
// k_phi_rhs3 in its order
__global__ void __launch_bounds__(kVecX * kVecY) k_phi_rhs4(Geom g, PhysDev ph, StageFields<float> f) {
    const int q = blockIdx.x * kVecX + threadIdx.x, j = blockIdx.y * kVecY + threadIdx.y;
    const int nx = g.n[0], ny = g.n[1], nz = g.n[2], k = blockIdx.z;
    if (4 * q >= nx || j >= ny) return;
    const long NP = g.NP;
    const long row = (long)nx * ((long)j + (long)ny * k);
    const long c = row + 4L * q;
    const float ih = g.ihf;
    const PhysT<float>& Q = phys<float>(ph);
    const float eps = Q.eps, delta = Q.delta, drho = Q.drho, rho2 = Q.rho2;
    const float gamma = stage_gamma(f);
    const long xm = q == 0 ? row + nx - 1 : c - 1, xp = 4 * q + 4 == nx ? row : c + 4;
    float pc[4], nc[4], ul[4];
    ld4(f.phi, c, pc);
    float div[4] = {0.f, 0.f, 0.f, 0.f};
    {  // x: faces e = 0..4 between cells e-1 and e of the quad
        float fx[6], nx6[6], F[5];
        ld4(f.nh[0], c, nc);
        ld4(f.u[0], c, ul);
        fx[0] = __ldg(f.phi + xm);
        nx6[0] = __ldg(f.nh[0] + xm);
        fx[5] = __ldg(f.phi + xp);
        nx6[5] = __ldg(f.nh[0] + xp);
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            fx[e + 1] = pc[e];
            nx6[e + 1] = nc[e];
        }
        const float u4 = __ldg(f.u[0] + xp);
#pragma unroll
        for (int e = 0; e < 5; ++e)
            F[e] = ops::phi_flux_v(fx[e], fx[e + 1], nx6[e], nx6[e + 1], e < 4 ? ul[e] : u4, gamma, eps, ih, delta);
        float m[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            div[e] += F[e + 1] - F[e];
            m[e] = drho * F[e] + rho2 * ul[e];
        }
        st4(f.m[0], c, m);
    }
    {  // y (periodic)
        const long cL = (j == 0) ? c + (long)(ny - 1) * nx : c - nx;
        const long cR = (j == ny - 1) ? c - (long)(ny - 1) * nx : c + nx;
        float fL[4], fR[4], nL[4], nR[4], uR[4], m[4];
        ld4(f.nh[1], c, nc);
        ld4(f.u[1], c, ul);
        ld4(f.phi, cL, fL);
        ld4(f.nh[1], cL, nL);
        ld4(f.phi, cR, fR);
        ld4(f.nh[1], cR, nR);
        ld4(f.u[1], cR, uR);
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const float Flo = ops::phi_flux_v(fL[e], pc[e], nL[e], nc[e], ul[e], gamma, eps, ih, delta);
            const float Fhi = ops::phi_flux_v(pc[e], fR[e], nc[e], nR[e], uR[e], gamma, eps, ih, delta);
            div[e] += Fhi - Flo;
            m[e] = drho * Flo + rho2 * ul[e];
        }
        st4(f.m[1], c, m);
    }
    {  // z (walls: no flux through the wall faces)
        const bool wlo = k == 0, whi = k == nz - 1;
        float fL[4], fR[4], nL[4], nR[4], uR[4], m[4];
        ld4(f.nh[2], c, nc);
        ld4(f.u[2], c, ul);
        if (!wlo) {
            ld4(f.phi, c - NP, fL);
            ld4(f.nh[2], c - NP, nL);
        }
        if (!whi) {
            ld4(f.phi, c + NP, fR);
            ld4(f.nh[2], c + NP, nR);
            ld4(f.u[2], c + NP, uR);
        }
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            float Flo = 0.f, Fhi = 0.f;
            if (!wlo) Flo = ops::phi_flux_v(fL[e], pc[e], nL[e], nc[e], ul[e], gamma, eps, ih, delta);
            if (!whi) Fhi = ops::phi_flux_v(pc[e], fR[e], nc[e], nR[e], uR[e], gamma, eps, ih, delta);
            div[e] += Fhi - Flo;
            m[e] = wlo ? 0.f : drho * Flo + rho2 * ul[e];
        }
        st4(f.m[2], c, m);
    }
    float r[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) r[e] = -div[e] * ih;
    st4(f.rphi, c, r);
}

template <typename T>
inline bool vec4_ok(const Geom& g) {
    return sizeof(T) == 4 && g.D == 3 && g.n[0] % 4 == 0;
}
inline dim3 vec4_grid(const Geom& g) {
    return dim3((unsigned)((g.n[0] / 4 + kVecX - 1) / kVecX), (unsigned)((g.n[1] + kVecY - 1) / kVecY),
                (unsigned)g.n[2]);
}

}  // namespace

// wall columns are FP64-heavy and few: small blocks spread them over the SMs
constexpr int kWallThreads = 64;
inline unsigned wall_blocks(const Geom& g) { return (unsigned)((2 * g.NP + kWallThreads - 1) / kWallThreads); }

template <typename T>
void launch_rhs(const Geom& g, const PhysDev& ph, const StageFields<T>& f, cudaStream_t s) {
    const unsigned nb = blocks_for(g.N);
    if constexpr (sizeof(T) == 4) {
        if (vec4_ok<T>(g))
            CDI_PROF(KC_PSI, s, (k_psi4<<<vec4_grid(g), dim3(kVecX, kVecY), 0, s>>>(g, ph, f.phi, f.psi)));
        else
            CDI_PROF(KC_PSI, s, (k_psi<T><<<nb, kThreads, 0, s>>>(g, ph, f.phi, f.psi)));
    } else {
        CDI_PROF(KC_PSI, s, (k_psi<T><<<nb, kThreads, 0, s>>>(g, ph, f.phi, f.psi)));
    }
    if (g.D == 2) {
        CDI_PROF(KC_CELL, s,
                 (k_cell<T, 2><<<nb, kThreads, 0, s>>>(g, ph, f.phi, f.psi, f.nh[0], f.nh[1], nullptr, f.muc)));
        CDI_PROF(KC_WALL, s, (k_wall<T, 2><<<wall_blocks(g), kWallThreads, 0, s>>>(
                                 g, ph, f.phi, f.psi, f.u[0], nullptr, f.wuY, f.wghost, f.wmuw)));
        CDI_PROF(KC_PHI_RHS, s, (k_phi_rhs<T, 2><<<nb, kThreads, 0, s>>>(g, ph, f)));
        CDI_PROF(KC_MOM, s, (k_mom<T, 2><<<nb, kThreads, 0, s>>>(g, ph, f)));
    } else {
        bool vec = false;
        if constexpr (sizeof(T) == 4) vec = vec4_ok<T>(g);
        if (vec) {
            CDI_PROF(KC_CELL, s,
                     (k_cell4<<<vec4_grid(g), dim3(kVecX, kVecY), 0, s>>>(
                         g, ph, (const float*)f.phi, (const float*)f.psi, (float*)f.nh[0], (float*)f.nh[1],
                         (float*)f.nh[2], (float*)f.muc)));
        } else if (g.n[0] % 32 == 0 && g.n[1] % 8 == 0) {
            const dim3 grid((unsigned)(g.n[0] / 32), (unsigned)(g.n[1] / 8), (unsigned)((g.n[2] + kCellZ - 1) / kCellZ));
            CDI_PROF(KC_CELL, s,
                     (k_cell3<T><<<grid, dim3(32, 8), 0, s>>>(g, ph, f.phi, f.psi, f.nh[0], f.nh[1], f.nh[2], f.muc)));
        } else {
            CDI_PROF(KC_CELL, s,
                     (k_cell<T, 3><<<nb, kThreads, 0, s>>>(g, ph, f.phi, f.psi, f.nh[0], f.nh[1], f.nh[2], f.muc)));
        }
        CDI_PROF(KC_WALL, s, (k_wall<T, 3><<<wall_blocks(g), kWallThreads, 0, s>>>(
                                 g, ph, f.phi, f.psi, f.u[0], f.u[1], f.wuY, f.wghost, f.wmuw)));
        if constexpr (sizeof(T) == 4) {
            if (vec) CDI_PROF(KC_PHI_RHS, s, (k_phi_rhs4<<<vec4_grid(g), dim3(kVecX, kVecY), 0, s>>>(g, ph, f)));
        }
        if (!vec) {
            if (g.n[0] % 32 == 0 && g.n[1] % 8 == 0) {
                const dim3 grid((unsigned)(g.n[0] / 32), (unsigned)(g.n[1] / 8),
                                (unsigned)((g.n[2] + kCellZ - 1) / kCellZ));
                CDI_PROF(KC_PHI_RHS, s, (k_phi_rhs3<T><<<grid, dim3(32, 8), 0, s>>>(g, ph, f)));
            } else {
                CDI_PROF(KC_PHI_RHS, s, (k_phi_rhs<T, 3><<<nb, kThreads, 0, s>>>(g, ph, f)));
            }
        }
        if (mom_tile_supported(g)) {
            CDI_PROF(KC_MOM, s, launch_mom_tile<T>(g, ph, f, s));
        } else {
            CDI_PROF(KC_MOM, s, (k_mom<T, 3><<<nb, kThreads, 0, s>>>(g, ph, f)));
        }
    }
    g_launches += 5;
}

template <typename T>
void launch_stage_update(const Geom& g, const PhysDev& ph, int stage, double dt, const T* phi0, const T* const* u0,
                         const T* rphi, const T* const* rm, T* accphi, T* const* accm, T* phik, T* const* uk,
                         cudaStream_t s) {
    static const double ck[4] = {0.0, 0.5, 0.5, 1.0};
    static const double bk[4] = {1.0 / 6.0, 1.0 / 3.0, 1.0 / 3.0, 1.0 / 6.0};
    const int first = stage == 0, last = stage == 3;
    const double cn = last ? 1.0 : ck[stage + 1];
    const unsigned nb = blocks_for(g.N);
    Ptr3<const T> pu0{{u0[0], u0[1], u0[2]}}, prm{{rm[0], rm[1], rm[2]}};
    Ptr3<T> pacc{{accm[0], accm[1], accm[2]}}, puk{{uk[0], uk[1], uk[2]}};
    if constexpr (sizeof(T) == 4) {
        if (vec4_ok<T>(g)) {
            const dim3 grid = vec4_grid(g), block(kVecX, kVecY);
            CDI_PROF(KC_STAGE_PHI, s, (k_stage_phi4<<<grid, block, 0, s>>>(g, (T)bk[stage], (T)(cn * dt), (T)dt,
                                                                            first, last, phi0, rphi, accphi, phik)));
            CDI_PROF(KC_STAGE_MOM, s, (k_stage_mom4<<<grid, block, 0, s>>>(g, ph, (T)bk[stage], (T)(cn * dt), (T)dt,
                                                                            first, last, phi0, phik, pu0, prm, pacc,
                                                                            puk)));
            g_launches += 2;
            return;
        }
    }
    CDI_PROF(KC_STAGE_PHI, s, (k_stage_phi<T><<<nb, kThreads, 0, s>>>(g.N, (T)bk[stage], (T)(cn * dt), (T)dt, first,
                                                                       last, phi0, rphi, accphi, phik)));
    if (g.D == 2)
        CDI_PROF(KC_STAGE_MOM, s, (k_stage_mom<T, 2><<<nb, kThreads, 0, s>>>(
                                      g, ph, (T)bk[stage], (T)(cn * dt), (T)dt, first, last, phi0, phik, pu0, prm,
                                      pacc, puk)));
    else
        CDI_PROF(KC_STAGE_MOM, s, (k_stage_mom<T, 3><<<nb, kThreads, 0, s>>>(
                                      g, ph, (T)bk[stage], (T)(cn * dt), (T)dt, first, last, phi0, phik, pu0, prm,
                                      pacc, puk)));
    g_launches += 2;
}

template <typename T>
void launch_wall_columns(const Geom& g, const PhysDev& ph, const T* phi, T* psi, double* cols, cudaStream_t s) {
    k_psi<T><<<blocks_for(g.N), kThreads, 0, s>>>(g, ph, phi, psi);
    if (g.D == 2) k_wall_cols<T, 2><<<blocks_for(2 * g.NP), kThreads, 0, s>>>(g, ph, phi, psi, cols);
    else k_wall_cols<T, 3><<<blocks_for(2 * g.NP), kThreads, 0, s>>>(g, ph, phi, psi, cols);
    g_launches += 2;
}

template void launch_rhs<double>(const Geom&, const PhysDev&, const StageFields<double>&, cudaStream_t);
template void launch_rhs<float>(const Geom&, const PhysDev&, const StageFields<float>&, cudaStream_t);
template void launch_stage_update<double>(const Geom&, const PhysDev&, int, double, const double*,
                                          const double* const*, const double*, const double* const*, double*,
                                          double* const*, double*, double* const*, cudaStream_t);
template void launch_stage_update<float>(const Geom&, const PhysDev&, int, double, const float*, const float* const*,
                                         const float*, const float* const*, float*, float* const*, float*,
                                         float* const*, cudaStream_t);
template void launch_wall_columns<double>(const Geom&, const PhysDev&, const double*, double*, double*, cudaStream_t);
template void launch_wall_columns<float>(const Geom&, const PhysDev&, const float*, float*, double*, cudaStream_t);

}  // namespace cdi
