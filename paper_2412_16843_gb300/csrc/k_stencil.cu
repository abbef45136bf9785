// Stencil kernels of one right-hand-side evaluation and the RK4 stage update.
//
//   k_psi        psi = eps ln(phi/(1-phi)), phi clamped to [delta, 1-delta]   Eq. (psi)
//   k_cell       grad psi, lap psi, normal n = grad psi/|grad psi|, chemical
//                potential mu_c                                             Eqs. (chemical potential),
//                (second-order central inside, second-order one-sided       (curvature), Sec. 4
//                wall-normal stencils in the first and last rows)
//   k_wall       wall rows: first-order linear extrapolation of phi, psi,
//                d_n psi, kappa_p to the wall, GNBC slip u^Y (Model 4A or    Eqs. (slip BC), (u_slip_v),
//                another model of Sec. 3) and the ghost velocity that        (u_slip_Y), (Model 1A..4B),
//                imposes the slip condition                                 Sec. 4
//   k_phi_rhs    phi flux u phi - R on every face (zero on the walls),      Eqs. (CDI), (no-flux BC),
//                its divergence, and the mass flux (rho1-rho2)F + rho2 u     (NS_momentum)
//   k_mom        momentum right-hand side on every velocity face:
//                -div(m u) + div(mu (grad u + grad u^T)) + mu_c grad phi      Eqs. (NS_momentum), (EB)
//   k_stage_*    classical RK4 stage values of phi and of the face
//                momentum rho_f u, and the stage velocity u* = (rho u)/rho_f  Sec. 4
//
// One thread per cell (or wall-plane position).  The wall-normal stencils and
// extrapolations read interior rows only: no ghost value of phi is ever
// formed (Sec. 4).
#include "cdi_internal.cuh"

namespace cdi {

thread_local long g_launches = 0;

namespace {

constexpr int kThreads = 256;

inline unsigned blocks_for(long n) { return (unsigned)((n + kThreads - 1) / kThreads); }

// first and second derivative of s along axis b at cell q (index c)
template <typename T>
__device__ __forceinline__ void d12(const Geom& g, const T* __restrict__ s, const IJK& q, long c, int b,
                                    T ih, T& d1, T& d2) {
    const T half_ih = T(0.5) * ih, ih2 = ih * ih;
    if (b == g.W) {
        const int r = coord(q, b);
        const long st = g.NP;
        if (r == 0) {
            T s0 = s[c], s1 = s[c + st], s2 = s[c + 2 * st], s3 = s[c + 3 * st];
            d1 = (T(-3) * s0 + T(4) * s1 - s2) * half_ih;
            d2 = (T(2) * s0 - T(5) * s1 + T(4) * s2 - s3) * ih2;
            return;
        }
        if (r == g.n[b] - 1) {
            T s0 = s[c], s1 = s[c - st], s2 = s[c - 2 * st], s3 = s[c - 3 * st];
            d1 = (T(3) * s0 - T(4) * s1 + s2) * half_ih;
            d2 = (T(2) * s0 - T(5) * s1 + T(4) * s2 - s3) * ih2;
            return;
        }
        T sm = s[c - st], s0 = s[c], sp = s[c + st];
        d1 = (sp - sm) * half_ih;
        d2 = (sp - T(2) * s0 + sm) * ih2;
        return;
    }
    T sm = s[idx(g, shift(g, q, b, -1))], s0 = s[c], sp = s[idx(g, shift(g, q, b, 1))];
    d1 = (sp - sm) * half_ih;
    d2 = (sp - T(2) * s0 + sm) * ih2;
}

template <typename T>
__global__ void k_psi(Geom g, PhysDev ph, const T* __restrict__ phi, T* __restrict__ psi) {
    long c = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= g.N) return;
    const T delta = (T)ph.delta;
    T pt = clampv(phi[c], delta, T(1) - delta);
    psi[c] = (T)ph.eps * log(pt / (T(1) - pt));
}

template <typename T, int DIM>
__global__ void k_cell(Geom g, PhysDev ph, const T* __restrict__ phi, const T* __restrict__ psi,
                       T* __restrict__ nh0, T* __restrict__ nh1, T* __restrict__ nh2, T* __restrict__ muc) {
    long c = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= g.N) return;
    const IJK q = decode(g, c);
    const T ih = T(1) / (T)g.h;
    T gb[3], grad2 = T(0), lap = T(0);
#pragma unroll
    for (int b = 0; b < DIM; ++b) {
        T d1, d2;
        d12(g, psi, q, c, b, ih, d1, d2);
        gb[b] = d1;
        grad2 += d1 * d1;
        lap += d2;
    }
    const T delta = (T)ph.delta, eps = (T)ph.eps;
    T pt = clampv(phi[c], delta, T(1) - delta);
    T P = pt * (T(1) - pt);
    muc[c] = T(6) * (T)ph.sigma * (P * (T(1) - T(2) * pt) * (T(1) - grad2) / eps - P * lap);
    T gm = sqrt(grad2) + (T)ph.tau;
    nh0[c] = gb[0] / gm;
    nh1[c] = gb[1] / gm;
    if (DIM == 3) nh2[c] = gb[2] / gm;
}

// Wall-column quantities: values extrapolated to the wall from the first two
// cell centres, q_w = (3 q_0 - q_1)/2 (first-order linear extrapolation, Sec. 4).
template <typename T>
struct ColQ {
    T phiw, psiw, dnw, kpw, dnphiw;
    T gt[2], gtphi[2];
};

template <typename T, int DIM>
__device__ ColQ<T> wall_column(const Geom& g, const PhysDev& ph, const T* __restrict__ phi,
                               const T* __restrict__ psi, int s, int i, int j) {
    const int W = DIM - 1, nW = g.n[W];
    const int r0 = s == 0 ? 0 : nW - 1, r1 = s == 0 ? 1 : nW - 2;
    const T sgn = s == 0 ? T(1) : T(-1);  // inward wall normal
    const T ih = T(1) / (T)g.h;
    const T delta = (T)ph.delta, eps = (T)ph.eps, tau = (T)ph.tau;
    T kp[2], dn[2], dnph[2], gtv[2][2], gtp[2][2], phv[2], psv[2];
#pragma unroll
    for (int rr = 0; rr < 2; ++rr) {
        IJK q;
        q.i = i;
        if (DIM == 2) { q.j = rr == 0 ? r0 : r1; q.k = 0; }
        else { q.j = j; q.k = rr == 0 ? r0 : r1; }
        const long c = idx(g, q);
        T gb[3], grad2 = T(0), lap = T(0), dph[3];
#pragma unroll
        for (int b = 0; b < DIM; ++b) {
            T d1, d2;
            d12(g, psi, q, c, b, ih, d1, d2);
            gb[b] = d1;
            grad2 += d1 * d1;
            lap += d2;
            T e1, e2;
            d12(g, phi, q, c, b, ih, e1, e2);
            dph[b] = e1;
        }
        T pt = clampv(phi[c], delta, T(1) - delta);
        T kap = (T(1) - T(2) * pt) * (T(1) - grad2) / eps - lap;
        if (DIM == 3) {
            // in-plane curvature: subtract the normal curvature along the
            // contact-line direction s = n_phi x n_wall (purely tangential)
            const T ih2 = ih * ih;
            const T p0 = psi[c];
            T pxx = (psi[idx(g, shift(g, q, 0, 1))] - T(2) * p0 + psi[idx(g, shift(g, q, 0, -1))]) * ih2;
            T pyy = (psi[idx(g, shift(g, q, 1, 1))] - T(2) * p0 + psi[idx(g, shift(g, q, 1, -1))]) * ih2;
            IJK qpp = shift(g, shift(g, q, 0, 1), 1, 1), qpm = shift(g, shift(g, q, 0, 1), 1, -1);
            IJK qmp = shift(g, shift(g, q, 0, -1), 1, 1), qmm = shift(g, shift(g, q, 0, -1), 1, -1);
            T pxy = (psi[idx(g, qpp)] - psi[idx(g, qpm)] - psi[idx(g, qmp)] + psi[idx(g, qmm)]) * (T(0.25) * ih2);
            T px = gb[0], py = gb[1];
            T gm = sqrt(grad2);
            T t2 = px * px + py * py;
            T num = py * py * pxx - T(2) * px * py * pxy + px * px * pyy;
            T ks = -num / ((t2 + tau * tau) * (gm + tau));
            kap -= ks;
        }
        kp[rr] = kap;
        dn[rr] = sgn * gb[W];
        dnph[rr] = sgn * dph[W];
        gtv[rr][0] = gb[0];
        gtp[rr][0] = dph[0];
        if (DIM == 3) { gtv[rr][1] = gb[1]; gtp[rr][1] = dph[1]; }
        phv[rr] = phi[c];
        psv[rr] = psi[c];
    }
    ColQ<T> o;
    o.phiw = clampv(T(0.5) * (T(3) * phv[0] - phv[1]), T(0), T(1));
    o.psiw = T(0.5) * (T(3) * psv[0] - psv[1]);
    o.dnw = T(0.5) * (T(3) * dn[0] - dn[1]);
    o.kpw = T(0.5) * (T(3) * kp[0] - kp[1]);
    o.dnphiw = T(0.5) * (T(3) * dnph[0] - dnph[1]);
    o.gt[0] = T(0.5) * (T(3) * gtv[0][0] - gtv[1][0]);
    o.gtphi[0] = T(0.5) * (T(3) * gtp[0][0] - gtp[1][0]);
    if (DIM == 3) {
        o.gt[1] = T(0.5) * (T(3) * gtv[0][1] - gtv[1][1]);
        o.gtphi[1] = T(0.5) * (T(3) * gtp[0][1] - gtp[1][1]);
    } else {
        o.gt[1] = T(0);
        o.gtphi[1] = T(0);
    }
    return o;
}

// u^Y of the slip models of Sec. 3: -(6 sigma/beta) [A + B cos(theta_eq)] T
template <typename T>
__device__ __forceinline__ T slip_model(int model, T sigma, T eps, T beta, T costh, T P, T dnpsi, T dtpsi,
                                        T gpsi, T dnphi, T dtphi, T gphi, T kp, T psiw) {
    const bool corr = (model == M3A || model == M3B || model == M4A || model == M4B);
    const T cc = corr ? (T(1) + kp * psiw) : T(1);
    T A, B, Tt;
    switch (model) {
        case M1A: case M3A: A = eps * dnphi; B = P * cc; Tt = dtphi; break;
        case M1B: case M3B: A = eps * dnphi; B = eps * gphi * cc; Tt = dtphi; break;
        case M2A: case M4A: A = P * dnpsi; B = P * cc; Tt = P / eps * dtpsi; break;
        default:            A = P * dnpsi; B = P * gpsi * cc; Tt = P / eps * dtpsi; break;
    }
    return -(T(6) * sigma / beta) * (A + B * costh) * Tt;
}

// one thread per (wall, wall-plane position): slip velocity, ghost value and
// wall viscosity for every tangential component at this face position
template <typename T, int DIM>
__global__ void k_wall(Geom g, PhysDev ph, const T* __restrict__ phi, const T* __restrict__ psi,
                       const T* __restrict__ u0, const T* __restrict__ u1, T* __restrict__ wuY,
                       T* __restrict__ wghost, T* __restrict__ wmuw) {
    long t = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= 2 * g.NP) return;
    const int s = (int)(t / g.NP);
    const long pidx = t - s * g.NP;
    const int i = (int)(pidx % g.n[0]);
    const int j = (DIM == 3) ? (int)(pidx / g.n[0]) : 0;
    const int W = DIM - 1;
    const int r0 = s == 0 ? 0 : g.n[W] - 1;
    const T h = (T)g.h, ih = T(1) / h;
    const WallDev& wp = ph.wall[s];
    const ColQ<T> cR = wall_column<T, DIM>(g, ph, phi, psi, s, i, j);
#pragma unroll
    for (int a = 0; a < DIM - 1; ++a) {
        int iL = i, jL = j;
        if (a == 0) iL = (i == 0) ? g.n[0] - 1 : i - 1;
        else jL = (j == 0) ? g.n[1] - 1 : j - 1;
        const ColQ<T> cL = wall_column<T, DIM>(g, ph, phi, psi, s, iL, jL);
        const T pb = T(0.5) * (cL.phiw + cR.phiw);
        const T P = pb * (T(1) - pb);
        const T psb = T(0.5) * (cL.psiw + cR.psiw);
        const T dnb = T(0.5) * (cL.dnw + cR.dnw);
        const T kb = T(0.5) * (cL.kpw + cR.kpw);
        const T dtau = (cR.psiw - cL.psiw) * ih;
        const T dnphi = T(0.5) * (cL.dnphiw + cR.dnphiw);
        const T dtphi = (cR.phiw - cL.phiw) * ih;
        T gs = dnb * dnb, gf = dnphi * dnphi;
#pragma unroll
        for (int tt = 0; tt < DIM - 1; ++tt) {
            T gt = (tt == a) ? dtau : T(0.5) * (cL.gt[tt] + cR.gt[tt]);
            T gtf = (tt == a) ? dtphi : T(0.5) * (cL.gtphi[tt] + cR.gtphi[tt]);
            gs += gt * gt;
            gf += gtf * gtf;
        }
        const T muw = (T)(ph.mu1 - ph.mu2) * pb + (T)ph.mu2;
        T uY = T(0), lw = T(0);
        if (!wp.noslip) {
            const T beta = (T)(wp.beta1 - wp.beta2) * pb + (T)wp.beta2;
            uY = slip_model<T>(ph.model, (T)ph.sigma, (T)ph.eps, beta, (T)wp.costh, P, dnb, dtau, sqrt(gs), dnphi,
                               dtphi, sqrt(gf), kb, psb);
            lw = muw / beta;
        }
        // tangential velocity in the first row of cells next to this wall
        const long cq = (DIM == 2) ? encode(g, i, r0, 0) : encode(g, i, j, r0);
        const T uf = (a == 0) ? u0[cq] : u1[cq];
        // ghost value: u_w = (u0+ug)/2, d_n u = (u0-ug)/h, u_w - U = l_w d_n u + u^Y
        const T lwh = lw * ih;
        const T ug = ((T)wp.U[a] + uY - uf * (T(0.5) - lwh)) / (T(0.5) + lwh);
        const long o = ((long)s * (DIM - 1) + a) * g.NP + pidx;
        wuY[o] = uY;
        wghost[o] = ug;
        wmuw[o] = muw;
    }
}

// column quantities only (phi_w, psi_w, d_n psi_w) for the contact line
template <typename T, int DIM>
__global__ void k_wall_cols(Geom g, PhysDev ph, const T* __restrict__ phi, const T* __restrict__ psi,
                            double* __restrict__ cols) {
    long t = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= 2 * g.NP) return;
    const int s = (int)(t / g.NP);
    const long pidx = t - s * g.NP;
    const int i = (int)(pidx % g.n[0]);
    const int j = (DIM == 3) ? (int)(pidx / g.n[0]) : 0;
    const ColQ<T> q = wall_column<T, DIM>(g, ph, phi, psi, s, i, j);
    double* base = cols + (long)s * 3 * g.NP;
    base[pidx] = (double)q.phiw;
    base[g.NP + pidx] = (double)q.psiw;
    base[2 * g.NP + pidx] = (double)q.dnw;
}

// total phi flux u phi - R across the face between cells cL and cR (Eq. CDI)
template <typename T>
__device__ __forceinline__ T phi_flux(const T* __restrict__ phi, const T* __restrict__ nh, long cL, long cR, T uf,
                                      T gamma, T eps, T ih, T delta) {
    const T fL = phi[cL], fR = phi[cR];
    const T pb = T(0.5) * (fL + fR);
    const T pc = clampv(pb, delta, T(1) - delta);
    const T nb = T(0.5) * (nh[cL] + nh[cR]);
    return uf * pb - gamma * (eps * (fR - fL) * ih - pc * (T(1) - pc) * nb);
}

template <typename T, int DIM>
__global__ void k_phi_rhs(Geom g, PhysDev ph, StageFields<T> f) {
    long c = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= g.N) return;
    const IJK q = decode(g, c);
    const int W = DIM - 1;
    const T ih = T(1) / (T)g.h;
    const T gamma = (T)(*f.gamma), eps = (T)ph.eps, delta = (T)ph.delta;
    const T drho = (T)(ph.rho1 - ph.rho2), rho2 = (T)ph.rho2;
    T div = T(0);
#pragma unroll
    for (int a = 0; a < DIM; ++a) {
        const T* __restrict__ ua = f.u[a];
        const T* __restrict__ na = f.nh[a];
        const int r = coord(q, a);
        T Flo = T(0), Fhi = T(0);
        if (!(a == W && r == 0)) {
            long cL = idx(g, shift(g, q, a, -1));
            Flo = phi_flux(f.phi, na, cL, c, ua[c], gamma, eps, ih, delta);
        }
        if (!(a == W && r == g.n[W] - 1)) {
            long cR = idx(g, shift(g, q, a, 1));
            long fi = (a == W) ? c + g.NP : cR;
            Fhi = phi_flux(f.phi, na, c, cR, ua[fi], gamma, eps, ih, delta);
        }
        div += Fhi - Flo;
        // consistent mass flux of the momentum equation on the low face
        f.m[a][c] = (a == W && r == 0) ? T(0) : drho * Flo + rho2 * ua[c];
    }
    f.rphi[c] = -div * ih;
}

template <typename T, int DIM>
__global__ void k_mom(Geom g, PhysDev ph, StageFields<T> f) {
    long c = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= g.N) return;
    const IJK q = decode(g, c);
    const int W = DIM - 1, nW = g.n[W];
    const T ih = T(1) / (T)g.h;
    const T dmu = (T)(ph.mu1 - ph.mu2), mu2 = (T)ph.mu2;
    const T* __restrict__ phi = f.phi;
    auto mu = [&](long cc) { return dmu * phi[cc] + mu2; };
    // position of this column in the wall plane
    const long pidx = (DIM == 2) ? (long)q.i : (long)q.i + (long)g.n[0] * q.j;
#pragma unroll
    for (int a = 0; a < DIM; ++a) {
        const T* __restrict__ ua = f.u[a];
        if (a == W && coord(q, W) == 0) { f.rm[a][c] = T(0); continue; }  // wall face
        const long cR = c;
        const IJK qL = shift(g, q, a, -1);
        const long cL = idx(g, qL);
        T adv = T(0), vis = T(0);
#pragma unroll
        for (int b = 0; b < DIM; ++b) {
            if (b == a) {
                // fluxes at the cell centres cL (low) and cR (high)
                const long fRlo = c, fRhi = (a == W) ? c + g.NP : idx(g, shift(g, q, a, 1));
                const long fLlo = cL, fLhi = c;
                const T* __restrict__ ma = f.m[a];
                T mbR = T(0.5) * (ma[fRlo] + ma[fRhi]), ubR = T(0.5) * (ua[fRlo] + ua[fRhi]);
                T mbL = T(0.5) * (ma[fLlo] + ma[fLhi]), ubL = T(0.5) * (ua[fLlo] + ua[fLhi]);
                T tR = T(2) * mu(cR) * (ua[fRhi] - ua[fRlo]) * ih;
                T tL = T(2) * mu(cL) * (ua[fLhi] - ua[fLlo]) * ih;
                adv -= (mbR * ubR - mbL * ubL) * ih;
                vis += (tR - tL) * ih;
            } else {
                T conv[2], tau[2];
#pragma unroll
                for (int side = 0; side < 2; ++side) {
                    const int eb = coord(q, b) + side;
                    if (b == W && (eb == 0 || eb == nW)) {
                        const int s = eb == 0 ? 0 : 1;
                        const long o = ((long)s * (DIM - 1) + a) * g.NP + pidx;
                        const T ug = f.wghost[o], muw = f.wmuw[o];
                        const T u0 = ua[c];
                        conv[side] = T(0);
                        tau[side] = (s == 0) ? muw * (u0 - ug) * ih : muw * (ug - u0) * ih;
                        continue;
                    }
                    IJK qhi = q;
                    setc(qhi, b, eb);
                    if (b != W && eb == g.n[b]) setc(qhi, b, 0);
                    const IJK qlo = shift(g, qhi, b, -1);
                    const long chi = idx(g, qhi), clo = idx(g, qlo);
                    const long chiA = idx(g, shift(g, qhi, a, -1)), cloA = idx(g, shift(g, qlo, a, -1));
                    const T ub = T(0.5) * (ua[clo] + ua[chi]);
                    const T mb = T(0.5) * (f.m[b][chi] + f.m[b][chiA]);
                    conv[side] = mb * ub;
                    const T me = T(0.25) * (mu(chi) + mu(chiA) + mu(clo) + mu(cloA));
                    const T dub = (ua[chi] - ua[clo]) * ih;
                    const T dua = (f.u[b][chi] - f.u[b][chiA]) * ih;
                    tau[side] = me * (dub + dua);
                }
                adv -= (conv[1] - conv[0]) * ih;
                vis += (tau[1] - tau[0]) * ih;
            }
        }
        // energy-based surface tension on the face (Eq. EB)
        const T st = T(0.5) * (f.muc[cL] + f.muc[cR]) * (phi[cR] - phi[cL]) * ih;
        f.rm[a][c] = adv + vis + st;
    }
}

// RK4 stage update of phi: acc += b_k k; next = phi0 + c dt k (or the final value)
template <typename T>
__global__ void k_stage_phi(long N, T b, T cdt, T dt, int first, int last, const T* __restrict__ phi0,
                            const T* __restrict__ rphi, T* __restrict__ acc, T* __restrict__ phik) {
    long c = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= N) return;
    const T k = rphi[c];
    const T a = first ? b * k : acc[c] + b * k;
    acc[c] = a;
    phik[c] = last ? phi0[c] + dt * a : phi0[c] + cdt * k;
}

// RK4 stage update of the face momentum and the stage velocity u* = M/rho_f
template <typename T, int DIM>
__global__ void k_stage_mom(Geom g, PhysDev ph, T b, T cdt, T dt, int first, int last,
                            const T* __restrict__ phi0, const T* __restrict__ phik, StageFields<T> f,
                            const T* __restrict__ u00, const T* __restrict__ u01, const T* __restrict__ u02,
                            T* __restrict__ acc0, T* __restrict__ acc1, T* __restrict__ acc2, T* __restrict__ uk0,
                            T* __restrict__ uk1, T* __restrict__ uk2) {
    long c = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= g.N) return;
    const IJK q = decode(g, c);
    const int W = DIM - 1;
    const T drho = (T)(ph.rho1 - ph.rho2), rho2 = (T)ph.rho2;
    const T* u0s[3] = {u00, u01, u02};
    T* accs[3] = {acc0, acc1, acc2};
    T* uks[3] = {uk0, uk1, uk2};
#pragma unroll
    for (int a = 0; a < DIM; ++a) {
        if (a == W && coord(q, W) == 0) { uks[a][c] = T(0); accs[a][c] = T(0); continue; }
        const long cL = idx(g, shift(g, q, a, -1));
        const T rf0 = T(0.5) * ((drho * phi0[cL] + rho2) + (drho * phi0[c] + rho2));
        const T M0 = rf0 * u0s[a][c];
        const T k = f.rm[a][c];
        const T ac = first ? b * k : accs[a][c] + b * k;
        accs[a][c] = ac;
        const T Mv = last ? M0 + dt * ac : M0 + cdt * k;
        const T rfk = T(0.5) * ((drho * phik[cL] + rho2) + (drho * phik[c] + rho2));
        uks[a][c] = Mv / rfk;
    }
}

}  // namespace

template <typename T>
void launch_rhs(const Geom& g, const PhysDev& ph, const StageFields<T>& f, cudaStream_t s) {
    const unsigned nb = blocks_for(g.N);
    k_psi<T><<<nb, kThreads, 0, s>>>(g, ph, f.phi, f.psi);
    if (g.D == 2) {
        k_cell<T, 2><<<nb, kThreads, 0, s>>>(g, ph, f.phi, f.psi, f.nh[0], f.nh[1], nullptr, f.muc);
        k_wall<T, 2><<<blocks_for(2 * g.NP), kThreads, 0, s>>>(g, ph, f.phi, f.psi, f.u[0], nullptr, f.wuY,
                                                              f.wghost, f.wmuw);
        k_phi_rhs<T, 2><<<nb, kThreads, 0, s>>>(g, ph, f);
        k_mom<T, 2><<<nb, kThreads, 0, s>>>(g, ph, f);
    } else {
        k_cell<T, 3><<<nb, kThreads, 0, s>>>(g, ph, f.phi, f.psi, f.nh[0], f.nh[1], f.nh[2], f.muc);
        k_wall<T, 3><<<blocks_for(2 * g.NP), kThreads, 0, s>>>(g, ph, f.phi, f.psi, f.u[0], f.u[1], f.wuY,
                                                              f.wghost, f.wmuw);
        k_phi_rhs<T, 3><<<nb, kThreads, 0, s>>>(g, ph, f);
        k_mom<T, 3><<<nb, kThreads, 0, s>>>(g, ph, f);
    }
    g_launches += 5;
}

template <typename T>
void launch_stage_update(const Geom& g, const PhysDev& ph, int stage, double dt, const T* phi0,
                         const T* const* u0, const T* rphi, const T* const* rm, T* accphi, T* const* accm,
                         T* phik, T* const* uk, cudaStream_t s) {
    static const double ck[4] = {0.0, 0.5, 0.5, 1.0};
    static const double bk[4] = {1.0 / 6.0, 1.0 / 3.0, 1.0 / 3.0, 1.0 / 6.0};
    const int first = stage == 0, last = stage == 3;
    const double cn = last ? 1.0 : ck[stage + 1];
    const unsigned nb = blocks_for(g.N);
    k_stage_phi<T><<<nb, kThreads, 0, s>>>(g.N, (T)bk[stage], (T)(cn * dt), (T)dt, first, last, phi0, rphi,
                                           accphi, phik);
    StageFields<T> f{};
    for (int a = 0; a < 3; ++a) f.rm[a] = const_cast<T*>(rm[a]);
    if (g.D == 2)
        k_stage_mom<T, 2><<<nb, kThreads, 0, s>>>(g, ph, (T)bk[stage], (T)(cn * dt), (T)dt, first, last, phi0,
                                                  phik, f, u0[0], u0[1], nullptr, accm[0], accm[1], nullptr,
                                                  uk[0], uk[1], nullptr);
    else
        k_stage_mom<T, 3><<<nb, kThreads, 0, s>>>(g, ph, (T)bk[stage], (T)(cn * dt), (T)dt, first, last, phi0,
                                                  phik, f, u0[0], u0[1], u0[2], accm[0], accm[1], accm[2],
                                                  uk[0], uk[1], uk[2]);
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
template void launch_stage_update<float>(const Geom&, const PhysDev&, int, double, const float*,
                                         const float* const*, const float*, const float* const*, float*,
                                         float* const*, float*, float* const*, cudaStream_t);
template void launch_wall_columns<double>(const Geom&, const PhysDev&, const double*, double*, double*,
                                          cudaStream_t);
template void launch_wall_columns<float>(const Geom&, const PhysDev&, const float*, float*, double*,
                                         cudaStream_t);

}  // namespace cdi
