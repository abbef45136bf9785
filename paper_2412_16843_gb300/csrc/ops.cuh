// Per-element device operations of the time step.  The standalone kernels
// (k_stencil.cu, k_mg.cu) and the persistent step kernel (k_persist.cu) both
// call these, so the two execution paths share one copy of the arithmetic.
//
// The load policy L decides how fields are read: LdPlain is an ordinary
// global load; LdCG reads through L2 only (ld.global.cg), which the persistent
// kernel uses for every field another block may have written before the last
// grid barrier.
//
// Formulas (paper sections and equations):
//   psi_at          Eq. (psi), phi clamped to [delta, 1-delta]
//   cell_at         Eqs. (chemical potential), (curvature); normal grad psi/|grad psi|;
//                   central differences inside, one-sided in the wall rows (Sec. 4)
//   wall_at         Eqs. (slip BC), (u_slip_v), (u_slip_Y) and Models 1A..4B (Sec. 3);
//                   wall values by first-order linear extrapolation (Sec. 4)
//   phi_rhs_at      Eqs. (CDI), (no-flux BC): u phi - R on faces, zero on walls;
//                   mass flux (rho1-rho2)(u phi - R) + rho2 u of Eq. (NS_momentum)
//   mom_at          Eq. (NS_momentum) without the pressure; Eq. (EB surface tension)
//   stage_*_at      classical RK4 (Sec. 4) on phi and on the face momentum rho_f u
//   div/coef/rbgs/resid/restrict/prolong/project: projection onto div u = 0
//                   (Eq. NS_incompressibility) by geometric multigrid
#pragma once

#include "cdi_internal.cuh"

namespace cdi {
namespace ops {

struct LdPlain {
    template <typename T>
    __device__ __forceinline__ static T ld(const T* p) { return *p; }
};
struct LdCG {
    template <typename T>
    __device__ __forceinline__ static T ld(const T* p) { return __ldcg(p); }
};

// ---------------------------------------------------------------------------
// a1: psi and cell-centre derivatives
// ---------------------------------------------------------------------------
template <class L, typename T>
__device__ __forceinline__ void d12(const Geom& g, const T* s, const IJK& q, long c, int b, T ih, T& d1, T& d2) {
    const T half_ih = T(0.5) * ih, ih2 = ih * ih;
    if (b == g.W) {
        const int r = coord(q, b);
        const long st = g.NP;
        if (r == 0) {
            T s0 = L::ld(s + c), s1 = L::ld(s + c + st), s2 = L::ld(s + c + 2 * st), s3 = L::ld(s + c + 3 * st);
            d1 = (T(-3) * s0 + T(4) * s1 - s2) * half_ih;
            d2 = (T(2) * s0 - T(5) * s1 + T(4) * s2 - s3) * ih2;
            return;
        }
        if (r == g.n[b] - 1) {
            T s0 = L::ld(s + c), s1 = L::ld(s + c - st), s2 = L::ld(s + c - 2 * st), s3 = L::ld(s + c - 3 * st);
            d1 = (T(3) * s0 - T(4) * s1 + s2) * half_ih;
            d2 = (T(2) * s0 - T(5) * s1 + T(4) * s2 - s3) * ih2;
            return;
        }
        T sm = L::ld(s + c - st), s0 = L::ld(s + c), sp = L::ld(s + c + st);
        d1 = (sp - sm) * half_ih;
        d2 = (sp - T(2) * s0 + sm) * ih2;
        return;
    }
    T sm = L::ld(s + idx(g, shift(g, q, b, -1))), s0 = L::ld(s + c), sp = L::ld(s + idx(g, shift(g, q, b, 1)));
    d1 = (sp - sm) * half_ih;
    d2 = (sp - T(2) * s0 + sm) * ih2;
}

template <class L, typename T>
__device__ __forceinline__ void psi_at(const Geom& g, const PhysDev& ph, const T* phi, T* psi, long c) {
    const PhysT<T>& P = phys<T>(ph);
    T pt = clampv(L::ld(phi + c), P.delta, T(1) - P.delta);
    psi[c] = P.eps * log(pt / (T(1) - pt));
}

template <class L, typename T, int DIM>
__device__ __forceinline__ void cell_at(const Geom& g, const PhysDev& ph, const T* phi, const T* psi, T* nh0,
                                        T* nh1, T* nh2, T* muc, long c) {
    const IJK q = decode(g, c);
    const T ih = g_ih<T>(g);
    T gb[3], grad2 = T(0), lap = T(0);
#pragma unroll
    for (int b = 0; b < DIM; ++b) {
        T d1, d2;
        d12<L>(g, psi, q, c, b, ih, d1, d2);
        gb[b] = d1;
        grad2 += d1 * d1;
        lap += d2;
    }
    const PhysT<T>& Q = phys<T>(ph);
    const T delta = Q.delta, eps = Q.eps;
    T pt = clampv(L::ld(phi + c), delta, T(1) - delta);
    T P = pt * (T(1) - pt);
    muc[c] = T(6) * Q.sigma * (P * (T(1) - T(2) * pt) * (T(1) - grad2) / eps - P * lap);
    const T igm = T(1) / (sqrt(grad2) + Q.tau);  // one division (FP64 is scarce on this part)
    nh0[c] = gb[0] * igm;
    nh1[c] = gb[1] * igm;
    if (DIM == 3) nh2[c] = gb[2] * igm;
}

// ---------------------------------------------------------------------------
// a2: wall rows
// ---------------------------------------------------------------------------
template <typename T>
struct ColQ {
    T phiw, psiw, dnw, kpw, dnphiw;
    T gt[2], gtphi[2];
};

// values extrapolated to wall s from the first two cell centres of column (i, j):
// q_w = (3 q_0 - q_1)/2 (first-order linear extrapolation, Sec. 4)
template <class L, typename T, int DIM>
__device__ ColQ<T> wall_column(const Geom& g, const PhysDev& ph, const T* phi, const T* psi, int s, int i, int j) {
    const int W = DIM - 1, nW = g.n[W];
    const int r0 = s == 0 ? 0 : nW - 1, r1 = s == 0 ? 1 : nW - 2;
    const T sgn = s == 0 ? T(1) : T(-1);  // inward wall normal
    const T ih = g_ih<T>(g);
    const T delta = phys<T>(ph).delta, eps = phys<T>(ph).eps, tau = phys<T>(ph).tau;
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
            d12<L>(g, psi, q, c, b, ih, d1, d2);
            gb[b] = d1;
            grad2 += d1 * d1;
            lap += d2;
            T e1, e2;
            d12<L>(g, phi, q, c, b, ih, e1, e2);
            dph[b] = e1;
        }
        const T phic = L::ld(phi + c), psic = L::ld(psi + c);
        T pt = clampv(phic, delta, T(1) - delta);
        T kap = (T(1) - T(2) * pt) * (T(1) - grad2) / eps - lap;
        if (DIM == 3) {
            // in-plane curvature: subtract the normal curvature along the
            // contact-line direction s = n_phi x n_wall (tangent to the wall)
            const T ih2 = ih * ih;
            T pxx = (L::ld(psi + idx(g, shift(g, q, 0, 1))) - T(2) * psic + L::ld(psi + idx(g, shift(g, q, 0, -1)))) *
                    ih2;
            T pyy = (L::ld(psi + idx(g, shift(g, q, 1, 1))) - T(2) * psic + L::ld(psi + idx(g, shift(g, q, 1, -1)))) *
                    ih2;
            IJK qpp = shift(g, shift(g, q, 0, 1), 1, 1), qpm = shift(g, shift(g, q, 0, 1), 1, -1);
            IJK qmp = shift(g, shift(g, q, 0, -1), 1, 1), qmm = shift(g, shift(g, q, 0, -1), 1, -1);
            T pxy = (L::ld(psi + idx(g, qpp)) - L::ld(psi + idx(g, qpm)) - L::ld(psi + idx(g, qmp)) +
                     L::ld(psi + idx(g, qmm))) *
                    (T(0.25) * ih2);
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
        gtv[rr][1] = (DIM == 3) ? gb[1] : T(0);
        gtp[rr][1] = (DIM == 3) ? dph[1] : T(0);
        phv[rr] = phic;
        psv[rr] = psic;
    }
    ColQ<T> o;
    o.phiw = clampv(T(0.5) * (T(3) * phv[0] - phv[1]), T(0), T(1));
    o.psiw = T(0.5) * (T(3) * psv[0] - psv[1]);
    o.dnw = T(0.5) * (T(3) * dn[0] - dn[1]);
    o.kpw = T(0.5) * (T(3) * kp[0] - kp[1]);
    o.dnphiw = T(0.5) * (T(3) * dnph[0] - dnph[1]);
    o.gt[0] = T(0.5) * (T(3) * gtv[0][0] - gtv[1][0]);
    o.gtphi[0] = T(0.5) * (T(3) * gtp[0][0] - gtp[1][0]);
    o.gt[1] = T(0.5) * (T(3) * gtv[0][1] - gtv[1][1]);
    o.gtphi[1] = T(0.5) * (T(3) * gtp[0][1] - gtp[1][1]);
    return o;
}

// u^Y of the slip models of Sec. 3: -(6 sigma/beta) [A + B cos(theta_eq)] T
template <typename T>
__device__ __forceinline__ T slip_model(int model, T sigma, T eps, T beta, T costh, T P, T dnpsi, T dtpsi, T gpsi,
                                        T dnphi, T dtphi, T gphi, T kp, T psiw) {
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

// slip velocity, ghost value and wall viscosity of tangential component a at
// position pidx = (i, j) of wall s, from the extrapolated quantities of the
// column (cR) and of its low neighbour along a (cL)
template <class L, typename T, int DIM>
__device__ __forceinline__ void wall_finish(const Geom& g, const PhysDev& ph, const ColQ<T>& cR, const ColQ<T>& cL,
                                            int a, int s, long pidx, int i, int j, const T* u0, const T* u1, T* wuY,
                                            T* wghost, T* wmuw) {
    const int W = DIM - 1;
    const int r0 = s == 0 ? 0 : g.n[W] - 1;
    const T ih = g_ih<T>(g);
    const WallDev& wp = ph.wall[s];
    const PhysT<T>& Q = phys<T>(ph);
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
    const T muw = Q.dmu * pb + Q.mu2;
    T uY = T(0), lw = T(0);
    if (!wp.noslip) {
        const T beta = Q.dbeta[s] * pb + Q.beta2[s];  // beta linear in phi
        uY = slip_model<T>(ph.model, Q.sigma, Q.eps, beta, Q.costh[s], P, dnb, dtau, sqrt(gs), dnphi, dtphi, sqrt(gf),
                           kb, psb);
        lw = muw / beta;
    }
    const long cq = (DIM == 2) ? encode(g, i, r0, 0) : encode(g, i, j, r0);
    const T uf = (a == 0) ? L::ld(u0 + cq) : L::ld(u1 + cq);
    // ghost value: u_w = (u0+ug)/2, d_n u = (u0-ug)/h, u_w - U = l_w d_n u + u^Y
    const T lwh = lw * ih;
    const T ug = (Q.U[s][a] + uY - uf * (T(0.5) - lwh)) / (T(0.5) + lwh);
    const long o = ((long)s * (DIM - 1) + a) * g.NP + pidx;
    wuY[o] = uY;
    wghost[o] = ug;
    wmuw[o] = muw;
}

// wall s = t / NP and wall-plane position t % NP of a thread index t in [0, 2 NP)
struct WallPos {
    int s, i, j;
    long pidx;
};
__device__ __forceinline__ WallPos wall_pos(const Geom& g, int dim, long t) {
    WallPos w;
    w.s = (int)(t / g.NP);
    w.pidx = t - w.s * g.NP;
    w.i = (int)(w.pidx % g.n[0]);
    w.j = (dim == 3) ? (int)(w.pidx / g.n[0]) : 0;
    return w;
}
// position of the low neighbour along tangential axis a (periodic)
__device__ __forceinline__ void wall_low(const Geom& g, int a, int i, int j, int& iL, int& jL) {
    iL = i;
    jL = j;
    if (a == 0) iL = (i == 0) ? g.n[0] - 1 : i - 1;
    else jL = (j == 0) ? g.n[1] - 1 : j - 1;
}

// thread t in [0, 2 NP): slip velocity, ghost value and wall viscosity of
// every tangential component, the column quantities formed here
template <class L, typename T, int DIM>
__device__ void wall_at(const Geom& g, const PhysDev& ph, const T* phi, const T* psi, const T* u0, const T* u1,
                        T* wuY, T* wghost, T* wmuw, long t) {
    const WallPos w = wall_pos(g, DIM, t);
    const ColQ<T> cR = wall_column<L, T, DIM>(g, ph, phi, psi, w.s, w.i, w.j);
#pragma unroll
    for (int a = 0; a < DIM - 1; ++a) {
        int iL, jL;
        wall_low(g, a, w.i, w.j, iL, jL);
        const ColQ<T> cL = wall_column<L, T, DIM>(g, ph, phi, psi, w.s, iL, jL);
        wall_finish<L, T, DIM>(g, ph, cR, cL, a, w.s, w.pidx, w.i, w.j, u0, u1, wuY, wghost, wmuw);
    }
}

// the column quantities of wall position t, once per column (stored in cq[t])
template <class L, typename T, int DIM>
__device__ __forceinline__ void wall_colq_at(const Geom& g, const PhysDev& ph, const T* phi, const T* psi, ColQ<T>* cq,
                                             long t) {
    const WallPos w = wall_pos(g, DIM, t);
    cq[t] = wall_column<L, T, DIM>(g, ph, phi, psi, w.s, w.i, w.j);
}

template <class L, typename T>
__device__ __forceinline__ ColQ<T> load_colq(const ColQ<T>* p) {
    ColQ<T> q;
    q.phiw = L::ld(&p->phiw);
    q.psiw = L::ld(&p->psiw);
    q.dnw = L::ld(&p->dnw);
    q.kpw = L::ld(&p->kpw);
    q.dnphiw = L::ld(&p->dnphiw);
    for (int k = 0; k < 2; ++k) {
        q.gt[k] = L::ld(&p->gt[k]);
        q.gtphi[k] = L::ld(&p->gtphi[k]);
    }
    return q;
}

// wall_at from the stored column quantities (wall_colq_at)
template <class L, typename T, int DIM>
__device__ void wall_from_colq_at(const Geom& g, const PhysDev& ph, const ColQ<T>* cq, const T* u0, const T* u1,
                                  T* wuY, T* wghost, T* wmuw, long t) {
    const WallPos w = wall_pos(g, DIM, t);
    const ColQ<T> cR = load_colq<L>(cq + t);
#pragma unroll
    for (int a = 0; a < DIM - 1; ++a) {
        int iL, jL;
        wall_low(g, a, w.i, w.j, iL, jL);
        const long tL = (long)w.s * g.NP + (DIM == 2 ? (long)iL : (long)iL + (long)g.n[0] * jL);
        const ColQ<T> cL = load_colq<L>(cq + tL);
        wall_finish<L, T, DIM>(g, ph, cR, cL, a, w.s, w.pidx, w.i, w.j, u0, u1, wuY, wghost, wmuw);
    }
}

// ---------------------------------------------------------------------------
// a3: phi flux and the consistent mass flux
// ---------------------------------------------------------------------------
// flux of the face between cells L and R from their phi, normal component and
// the face velocity
template <typename T>
__device__ __forceinline__ T phi_flux_v(T fL, T fR, T nL, T nR, T uf, T gamma, T eps, T ih, T delta) {
    const T pb = T(0.5) * (fL + fR);
    const T pc = clampv(pb, delta, T(1) - delta);
    const T nb = T(0.5) * (nL + nR);
    return uf * pb - gamma * (eps * (fR - fL) * ih - pc * (T(1) - pc) * nb);
}
template <class L, typename T>
__device__ __forceinline__ T phi_flux(const T* phi, const T* nh, long cL, long cR, T uf, T gamma, T eps, T ih,
                                      T delta) {
    return phi_flux_v(L::ld(phi + cL), L::ld(phi + cR), L::ld(nh + cL), L::ld(nh + cR), uf, gamma, eps, ih, delta);
}

template <class L, typename T, int DIM>
__device__ __forceinline__ void phi_rhs_at(const Geom& g, const PhysDev& ph, const StageFields<T>& f, T gamma,
                                           long c) {
    const IJK q = decode(g, c);
    const int W = DIM - 1;
    const T ih = g_ih<T>(g);
    const PhysT<T>& Q = phys<T>(ph);
    const T eps = Q.eps, delta = Q.delta;
    const T drho = Q.drho, rho2 = Q.rho2;
    T div = T(0);
#pragma unroll
    for (int a = 0; a < DIM; ++a) {
        const T* ua = f.u[a];
        const T* na = f.nh[a];
        const int r = coord(q, a);
        T Flo = T(0), Fhi = T(0);
        const T ulo = L::ld(ua + c);
        if (!(a == W && r == 0)) {
            long cL = idx(g, shift(g, q, a, -1));
            Flo = phi_flux<L>(f.phi, na, cL, c, ulo, gamma, eps, ih, delta);
        }
        if (!(a == W && r == g.n[W] - 1)) {
            long cR = idx(g, shift(g, q, a, 1));
            long fi = (a == W) ? c + g.NP : cR;
            Fhi = phi_flux<L>(f.phi, na, c, cR, L::ld(ua + fi), gamma, eps, ih, delta);
        }
        div += Fhi - Flo;
        f.m[a][c] = (a == W && r == 0) ? T(0) : drho * Flo + rho2 * ulo;
    }
    f.rphi[c] = -div * ih;
}

// ---------------------------------------------------------------------------
// a4: momentum right-hand side (all components on the low faces of cell c)
// ---------------------------------------------------------------------------
template <class L, typename T, int DIM>
__device__ void mom_at(const Geom& g, const PhysDev& ph, const StageFields<T>& f, long c) {
    const IJK q = decode(g, c);
    const int W = DIM - 1, nW = g.n[W];
    const T ih = g_ih<T>(g);
    const T dmu = phys<T>(ph).dmu, mu2 = phys<T>(ph).mu2;
    const T* phi = f.phi;
    auto mu = [&](long cc) { return dmu * L::ld(phi + cc) + mu2; };
    const long pidx = (DIM == 2) ? (long)q.i : (long)q.i + (long)g.n[0] * q.j;
#pragma unroll
    for (int a = 0; a < DIM; ++a) {
        const T* ua = f.u[a];
        if (a == W && coord(q, W) == 0) { f.rm[a][c] = T(0); continue; }  // wall face
        const long cR = c;
        const long cL = idx(g, shift(g, q, a, -1));
        T adv = T(0), vis = T(0);
#pragma unroll
        for (int b = 0; b < DIM; ++b) {
            if (b == a) {
                const long fRlo = c, fRhi = (a == W) ? c + g.NP : idx(g, shift(g, q, a, 1));
                const long fLlo = cL, fLhi = c;
                const T* ma = f.m[a];
                const T uRlo = L::ld(ua + fRlo), uRhi = L::ld(ua + fRhi), uLlo = L::ld(ua + fLlo);
                T mbR = T(0.5) * (L::ld(ma + fRlo) + L::ld(ma + fRhi)), ubR = T(0.5) * (uRlo + uRhi);
                T mbL = T(0.5) * (L::ld(ma + fLlo) + L::ld(ma + fLhi)), ubL = T(0.5) * (uLlo + uRlo);
                T tR = T(2) * mu(cR) * (uRhi - uRlo) * ih;
                T tL = T(2) * mu(cL) * (uRlo - uLlo) * ih;
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
                        const T ug = L::ld(f.wghost + o), muw = L::ld(f.wmuw + o);
                        const T u0 = L::ld(ua + c);
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
                    const T uhi = L::ld(ua + chi), ulo = L::ld(ua + clo);
                    const T ub = T(0.5) * (ulo + uhi);
                    const T mb = T(0.5) * (L::ld(f.m[b] + chi) + L::ld(f.m[b] + chiA));
                    conv[side] = mb * ub;
                    const T me = T(0.25) * (mu(chi) + mu(chiA) + mu(clo) + mu(cloA));
                    const T dub = (uhi - ulo) * ih;
                    const T dua = (L::ld(f.u[b] + chi) - L::ld(f.u[b] + chiA)) * ih;
                    tau[side] = me * (dub + dua);
                }
                adv -= (conv[1] - conv[0]) * ih;
                vis += (tau[1] - tau[0]) * ih;
            }
        }
        // energy-based surface tension on the face (Eq. EB)
        const T st = T(0.5) * (L::ld(f.muc + cL) + L::ld(f.muc + cR)) * (L::ld(phi + cR) - L::ld(phi + cL)) * ih;
        f.rm[a][c] = adv + vis + st;
    }
}

// ---------------------------------------------------------------------------
// a5: RK4 stage values
// ---------------------------------------------------------------------------
template <class L, typename T>
__device__ __forceinline__ void stage_phi_at(T b, T cdt, T dt, int first, int last, const T* phi0, const T* rphi,
                                             T* acc, T* phik, long c) {
    const T k = L::ld(rphi + c);
    const T a = first ? b * k : L::ld(acc + c) + b * k;
    acc[c] = a;
    phik[c] = last ? L::ld(phi0 + c) + dt * a : L::ld(phi0 + c) + cdt * k;
}

template <class L, typename T, int DIM>
__device__ __forceinline__ void stage_mom_at(const Geom& g, const PhysDev& ph, T b, T cdt, T dt, int first, int last,
                                             const T* phi0, const T* phik, const T* const* u0, const T* const* rm,
                                             T* const* acc, T* const* uk, long c) {
    const IJK q = decode(g, c);
    const int W = DIM - 1;
    const T drho = phys<T>(ph).drho, rho2 = phys<T>(ph).rho2;
#pragma unroll
    for (int a = 0; a < DIM; ++a) {
        if (a == W && coord(q, W) == 0) { uk[a][c] = T(0); acc[a][c] = T(0); continue; }
        const long cL = idx(g, shift(g, q, a, -1));
        const T rf0 = T(0.5) * ((drho * L::ld(phi0 + cL) + rho2) + (drho * L::ld(phi0 + c) + rho2));
        const T M0 = rf0 * L::ld(u0[a] + c);
        const T k = L::ld(rm[a] + c);
        const T ac = first ? b * k : L::ld(acc[a] + c) + b * k;
        acc[a][c] = ac;
        const T Mv = last ? M0 + dt * ac : M0 + cdt * k;
        const T rfk = T(0.5) * ((drho * L::ld(phik + cL) + rho2) + (drho * L::ld(phik + c) + rho2));
        uk[a][c] = Mv / rfk;
    }
}

// ---------------------------------------------------------------------------
// a6..a8: projection and multigrid
//
// The pressure solve is defect correction around an FP32 V-cycle: the
// residual r = f - A p, its norm and the update p += e are taken in the
// precision of the form (FP64; or double-float in the FP32-mixed form, see
// PForm), while the V-cycle that computes the correction e ~ A^-1 r runs in
// FP32 (M = float), except the dense solve of the coarsest level, which is
// FP64.  The iteration converges to a tolerance far below FP32 round-off
// because each V-cycle only has to reduce the error by a fixed factor.
// ---------------------------------------------------------------------------
template <class L, typename T, int DIM>
__device__ __forceinline__ T div_at(const Geom& g, const T* const* us, T ih, T inv_cdt, long c) {
    const IJK q = decode(g, c);
    T div = T(0);
#pragma unroll
    for (int a = 0; a < DIM; ++a) {
        const long hi = (a == DIM - 1) ? c + g.NP : idx(g, shift(g, q, a, 1));
        div += L::ld(us[a] + hi) - L::ld(us[a] + c);
    }
    return div * ih * inv_cdt;
}

// face coefficients 1/rho_f of level 0: FP32 (bsf) in both forms, and FP64
// (bs) in the FP64 form, where bsf is the rounded FP64 value; t in [0, N + NP)
// (the last NP are the high wall faces of the wall-normal component)
template <class L, typename T, int DIM>
__device__ __forceinline__ void coef0_at(const Geom& g, const PhysDev& ph, const T* phi, double* const* bs,
                                         float* const* bsf, float* rho0, long t) {
    constexpr bool f64 = sizeof(T) == 8;
    if (t >= g.N) {
        if (f64) bs[DIM - 1][t] = 0.0;
        bsf[DIM - 1][t] = 0.f;
        return;
    }
    const IJK q = decode(g, t);
    const T dr = phys<T>(ph).drho, rho2 = phys<T>(ph).rho2;
    rho0[t] = (float)(dr * L::ld(phi + t) + rho2);
#pragma unroll
    for (int a = 0; a < DIM; ++a) {
        if (a == DIM - 1 && coord(q, a) == 0) {
            if (f64) bs[a][t] = 0.0;
            bsf[a][t] = 0.f;
            continue;
        }
        const long cL = idx(g, shift(g, q, a, -1));
        const T rf = T(0.5) * ((dr * L::ld(phi + cL) + rho2) + (dr * L::ld(phi + t) + rho2));
        const T b = T(1) / rf;
        if (f64) bs[a][t] = (double)b;
        bsf[a][t] = (float)b;
    }
}

// coarse face coefficient = mean of the 2^(D-1) fine faces covering it; t in [0, Nc + NPc)
template <class L, typename M, int DIM>
__device__ __forceinline__ void coef_restrict_at(const Geom& gf, const Geom& gc, const M* const* fb, M* const* cb,
                                                 long t) {
    IJK q = decode(gc, t < gc.N ? t : t - gc.NP);
    if (t >= gc.N) setc(q, DIM - 1, gc.n[DIM - 1]);
#pragma unroll
    for (int a = 0; a < DIM; ++a) {
        if (t >= gc.N && a != DIM - 1) continue;
        int other[2] = {0, 0}, no = 0;
        for (int b = 0; b < DIM; ++b)
            if (b != a) other[no++] = b;
        const int o2 = (DIM == 3) ? 2 : 1;
        M sum = M(0);
        for (int t2 = 0; t2 < o2; ++t2)
            for (int t1 = 0; t1 < 2; ++t1) {
                IJK qf;
                qf.i = 2 * q.i;
                qf.j = 2 * q.j;
                qf.k = (DIM == 3) ? 2 * q.k : 0;
                setc(qf, other[0], coord(qf, other[0]) + t1);
                if (DIM == 3) setc(qf, other[1], coord(qf, other[1]) + t2);
                sum += L::ld(fb[a] + idx(gf, qf));
            }
        cb[a][idx(gc, q)] = sum * (M(1) / M(2 * o2));
    }
}

// (A p)_c pieces: diag = sum (beta- + beta+)/h^2, off = sum (beta- p- + beta+ p+)/h^2,
// the neighbour values p+- given by nv(index); zero coefficients on the walls
// (Neumann), where no neighbour value is taken (it may not exist yet)
template <class L, typename M, int DIM, class NV>
__device__ __forceinline__ void stencil_L(const Geom& g, const M* const* beta, const IJK& q, long c, M ih2, NV nv,
                                          M& diag, M& off) {
    diag = M(0);
    off = M(0);
#pragma unroll
    for (int a = 0; a < DIM; ++a) {
        long lo, hi;
        bool wlo = false, whi = false;
        if (a == DIM - 1) {
            const int r = coord(q, a);
            wlo = r == 0;
            whi = r == g.n[a] - 1;
            lo = wlo ? c : c - g.NP;
            hi = whi ? c : c + g.NP;
        } else {
            lo = idx(g, shift(g, q, a, -1));
            hi = idx(g, shift(g, q, a, 1));
        }
        const long fhi = (a == DIM - 1) ? c + g.NP : hi;
        const M bm = L::ld(beta[a] + c);
        const M bp = L::ld(beta[a] + fhi);
        const M pm = wlo ? M(0) : nv(lo);
        const M pp = whi ? M(0) : nv(hi);
        diag += (bm + bp) * ih2;
        off += (bm * pm + bp * pp) * ih2;
    }
}

// (A p)_c with the stored neighbour values; returns off - diag p_c
template <class L, typename M, int DIM>
__device__ __forceinline__ M apply_L(const Geom& g, const M* const* beta, const M* p, const IJK& q, long c, M ih2,
                                     M& diag, M& off) {
    stencil_L<L, M, DIM>(g, beta, q, c, ih2, [&](long n) { return L::ld(p + n); }, diag, off);
    return off - diag * L::ld(p + c);
}

// stencil_L on level 0 with the face coefficients formed from the FP32 cell
// densities, beta = 2 / (rho_L + rho_R) (coef0_at's 1 / mean density, by the
// fast FP32 division): one array read instead of D coefficient arrays.  Used
// by the level-0 smoother and residual restriction only; the defect-correction
// residual keeps the stored coefficients.  Walls carry a zero coefficient.
template <class L, int DIM, class NV>
__device__ __forceinline__ void stencil_L_rho(const Geom& g, const float* rho, const IJK& q, long c, float ih2, NV nv,
                                              float& diag, float& off) {
    diag = 0.f;
    off = 0.f;
    const float rc = L::ld(rho + c);
#pragma unroll
    for (int a = 0; a < DIM; ++a) {
        long lo, hi;
        bool wlo = false, whi = false;
        if (a == DIM - 1) {
            const int r = coord(q, a);
            wlo = r == 0;
            whi = r == g.n[a] - 1;
            lo = wlo ? c : c - g.NP;
            hi = whi ? c : c + g.NP;
        } else {
            lo = idx(g, shift(g, q, a, -1));
            hi = idx(g, shift(g, q, a, 1));
        }
        const float bm = (wlo ? 0.f : 1.f) * __fdividef(2.f, rc + L::ld(rho + lo));
        const float bp = (whi ? 0.f : 1.f) * __fdividef(2.f, rc + L::ld(rho + hi));
        const float pm = wlo ? 0.f : nv(lo);
        const float pp = whi ? 0.f : nv(hi);
        diag += (bm + bp) * ih2;
        off += (bm * pm + bp * pp) * ih2;
    }
}

template <class L, int DIM>
__device__ __forceinline__ float apply_L_rho(const Geom& g, const float* rho, const float* p, const IJK& q, long c,
                                             float ih2, float& diag, float& off) {
    stencil_L_rho<L, DIM>(g, rho, q, c, ih2, [&](long n) { return L::ld(p + n); }, diag, off);
    return off - diag * L::ld(p + c);
}

// k-th cell of one colour ((i+j+k) even or odd); every extent of a smoothed level is even
__device__ __forceinline__ long colour_cell(const Geom& g, int colour, long k) {
    const unsigned half = (unsigned)g.n[0] >> 1;
    const unsigned line = (unsigned)k / half;
    const unsigned m = (unsigned)k - line * half;
    const unsigned kk = g.fd1.div(line);
    const unsigned j = line - kk * (unsigned)g.n[1];
    const unsigned i = 2u * m + ((colour + j + kk) & 1u);
    return (long)(i + (unsigned)g.n[0] * line);
}

// Gauss-Seidel step p_c = (off - f_c) / diag of cell c; the variants take the
// neighbour values as zero (the first step of a V-cycle's smoothing, whose
// correction starts from zero) or as stored plus the prolongation of the
// coarse correction pc (the first step after the coarse-grid correction, which
// is then never stored: a Gauss-Seidel step does not read its own cell)
enum StepNb { kNbStored = 0, kNbZero = 1, kNbProlong = 2 };

// 1 / x by the hardware approximation (rcp.approx.ftz.f32: relative error
// below 2^-23, subnormals flushed), for the finest-level smoother's face
// coefficients, which only precondition (the defect correction iterates to the
// tolerance regardless)
__device__ __forceinline__ float rcp_approx(float x) {
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// over-relaxed update e + omega (e_gs - e) from the old value e, every
// rounding explicit (no contraction with the producer of e_gs)
__device__ __forceinline__ float relax(float e, float egs, float omega) {
    return __fmaf_rn(omega, __fsub_rn(egs, e), e);
}

// quotient of a smoothing step: the fast FP32 division (a preconditioner's
// arithmetic; the defect correction iterates to the tolerance regardless)
__device__ __forceinline__ float step_div(float a, float b) { return __fdividef(a, b); }
__device__ __forceinline__ double step_div(double a, double b) { return a / b; }

template <class L, typename M, int DIM>
__device__ __forceinline__ M prolong_val(const Geom& gf, const Geom& gc, const M* pc, long c);

// the new value of cell c (rbgs_at without the store)
template <class L, typename M, int DIM, int NB = kNbStored>
__device__ __forceinline__ M rbgs_val(const Geom& g, const M* const* beta, const M* p, const M* f, long c,
                                      const Geom* gc = nullptr, const M* pc = nullptr) {
    const IJK q = decode(g, c);
    const M ih2 = g_ih2<M>(g);
    M diag, off;
    stencil_L<L, M, DIM>(
        g, beta, q, c, ih2,
        [&](long n) -> M {
            if (NB == kNbZero) return M(0);
            if (NB == kNbProlong) return L::ld(p + n) + prolong_val<L, M, DIM>(g, *gc, pc, n);
            return L::ld(p + n);
        },
        diag, off);
    return step_div(off - L::ld(f + c), diag);
}

template <class L, typename M, int DIM, int NB = kNbStored>
__device__ __forceinline__ void rbgs_at(const Geom& g, const M* const* beta, M* p, const M* f, long c,
                                        const Geom* gc = nullptr, const M* pc = nullptr) {
    p[c] = rbgs_val<L, M, DIM, NB>(g, beta, p, f, c, gc, pc);
}

// level-0 smoothing value with density-formed coefficients (stencil_L_rho)
template <class L, int DIM, int NB = kNbStored>
__device__ __forceinline__ float rbgs_rho_val(const Geom& g, const float* rho, const float* p, const float* f, long c,
                                              const Geom* gc = nullptr, const float* pc = nullptr) {
    const IJK q = decode(g, c);
    float diag, off;
    stencil_L_rho<L, DIM>(
        g, rho, q, c, g.ih2f,
        [&](long n) -> float {
            if (NB == kNbZero) return 0.f;
            if (NB == kNbProlong) return L::ld(p + n) + prolong_val<L, float, DIM>(g, *gc, pc, n);
            return L::ld(p + n);
        },
        diag, off);
    return step_div(off - L::ld(f + c), diag);
}

template <class L, int DIM, int NB = kNbStored>
__device__ __forceinline__ void rbgs_rho_at(const Geom& g, const float* rho, float* p, const float* f, long c,
                                            const Geom* gc = nullptr, const float* pc = nullptr) {
    p[c] = rbgs_rho_val<L, DIM, NB>(g, rho, p, f, c, gc, pc);
}

// One colour of a red-black pass over the cells k0, k0 + stride, ... < half
// of that colour: two cells an iteration, both values formed (val(k, c))
// before either is stored (put(c, v)), so their loads overlap; cells of one
// colour do not depend on each other, so the result is the same.
template <class VAL, class PUT>
__device__ __forceinline__ void colour_pass(int k0, int half, int stride, VAL val, PUT put) {
    int k = k0;
    for (; k + stride < half; k += 2 * stride) {
        long c0, c1;
        const auto v0 = val(k, c0);
        const auto v1 = val(k + stride, c1);
        put(c0, v0);
        put(c1, v1);
    }
    if (k < half) {
        long c0;
        const auto v0 = val(k, c0);
        put(c0, v0);
    }
}

// FP64 residual f - A p of level 0
template <class L, int DIM>
__device__ __forceinline__ double resid64_at(const Geom& g, const double* const* beta, const double* p,
                                             const double* f, long c) {
    const IJK q = decode(g, c);
    const double ih2 = g.ih2;
    double diag, off;
    return L::ld(f + c) - apply_L<L, double, DIM>(g, beta, p, q, c, ih2, diag, off);
}

// ---------------------------------------------------------------------------
// Double-float arithmetic of the FP32-mixed form: a value is hi + lo with
// |lo| at most half an ulp of hi.  Built from error-free transformations:
// TwoSum (Knuth, TAOCP vol. 2, sec. 4.2.2: s + e = a + b exactly) and the
// product error by one FMA (a b - fl(a b) is exact in FP32).  The __f*_rn
// intrinsics keep the compiler from contracting or reordering them.
// ---------------------------------------------------------------------------
namespace dfl {
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}
__device__ __forceinline__ void two_prod(float a, float b, float& p, float& e) {
    p = __fmul_rn(a, b);
    e = __fmaf_rn(a, b, -p);
}
// renormalised (hi, lo) of s + e
__device__ __forceinline__ float2 norm2(float s, float e) {
    float hi, lo;
    two_sum(s, e, hi, lo);
    return make_float2(hi, lo);
}
// a + x
__device__ __forceinline__ float2 add(float2 a, float x) {
    float s, e;
    two_sum(a.x, x, s, e);
    return norm2(s, __fadd_rn(e, a.y));
}
// a + b
__device__ __forceinline__ float2 add(float2 a, float2 b) {
    float s, e;
    two_sum(a.x, b.x, s, e);
    return norm2(s, __fadd_rn(e, __fadd_rn(a.y, b.y)));
}
// a - b
__device__ __forceinline__ float2 sub(float2 a, float2 b) { return add(a, make_float2(-b.x, -b.y)); }
// the double-float nearest a double (host and device; the device use is per thread, not per cell)
__host__ __device__ __forceinline__ float2 from_double(double v) {
    const float hi = (float)v;
    return make_float2(hi, (float)(v - (double)hi));
}
__host__ __device__ __forceinline__ double to_double(float2 a) { return (double)a.x + (double)a.y; }
}  // namespace dfl

// Running sum of a form's values, accurate enough that the mean of f it
// yields leaves no constant component in the residual: FP64, or double-float
// for FP32 values.
template <typename T> struct SumAcc;
template <> struct SumAcc<double> {
    double s = 0.0;
    __device__ __forceinline__ void add(double v) { s += v; }
    __device__ __forceinline__ double value() const { return s; }
};
template <> struct SumAcc<float> {
    float2 s = make_float2(0.f, 0.f);
    __device__ __forceinline__ void add(float v) { s = dfl::add(s, v); }
    __device__ __forceinline__ double value() const { return dfl::to_double(s); }
};

// the flux b (x - y) for double-floats x, y and an FP32 coefficient b, as an
// unevaluated sum t + te (every step is odd in (x, y): swapping them negates t
// and te exactly)
__device__ __forceinline__ void df_term(float b, float2 x, float2 y, float& t, float& te) {
    float d, de;
    dfl::two_sum(x.x, -y.x, d, de);
    const float dl = __fadd_rn(de, __fsub_rn(x.y, y.y));
    dfl::two_prod(b, d, t, te);
    te = __fmaf_rn(b, dl, te);
}
// (Sh, Sl) += t + te
__device__ __forceinline__ void df_acc(float t, float te, float& Sh, float& Sl) {
    float s2, se;
    dfl::two_sum(Sh, t, s2, se);
    Sh = s2;
    Sl = __fadd_rn(Sl, __fadd_rn(se, te));
}
// S += b (x - y) into the double-float accumulator (Sh, Sl)
__device__ __forceinline__ void df_acc_term(float b, float2 x, float2 y, float& Sh, float& Sl) {
    float t, te;
    df_term(b, x, y, t, te);
    df_acc(t, te, Sh, Sl);
}

// (f - mean) - S / h^2 for the double-float flux sum S = (Sh, Sl), rounded to FP32
__device__ __forceinline__ float resid_df_finish(float Sh, float Sl, float ih2f, float fc, float2 fmean) {
    float ah, al;
    dfl::two_prod(Sh, ih2f, ah, al);
    al = __fmaf_rn(Sl, ih2f, al);
    float r1, e1, r2, e2;
    dfl::two_sum(fc, -fmean.x, r1, e1);
    dfl::two_sum(r1, -ah, r2, e2);
    return __fadd_rn(r2, __fadd_rn(__fsub_rn(e1, fmean.y), __fsub_rn(e2, al)));
}

// Residual (f - mean) - A p of the FP32-mixed form at cell c, with the FP32
// face coefficients bf and 1/h^2 of the V-cycles, accumulated in double-float
// (error about 2^-44 of the largest flux term, far below any tolerance a
// solve asks for); returned rounded to FP32.  Same stencil as apply_L.
template <class L, int DIM>
__device__ __forceinline__ float resid_df_at(const Geom& g, const float* const* bf, const float2* p, const float* f,
                                             float2 fmean, long c) {
    const IJK q = decode(g, c);
    const float2 pc = L::ld(p + c);
    float Sh = 0.f, Sl = 0.f;
#pragma unroll
    for (int a = 0; a < DIM; ++a) {
        long lo, hi;
        if (a == DIM - 1) {
            const int r = coord(q, a);
            lo = r > 0 ? c - g.NP : c;
            hi = r < g.n[a] - 1 ? c + g.NP : c;
        } else {
            lo = idx(g, shift(g, q, a, -1));
            hi = idx(g, shift(g, q, a, 1));
        }
        const long fhi = (a == DIM - 1) ? c + g.NP : hi;
        const float bm = L::ld(bf[a] + c);
        const float bp = L::ld(bf[a] + fhi);
        df_acc_term(bm, L::ld(p + lo), pc, Sh, Sl);
        df_acc_term(bp, L::ld(p + hi), pc, Sh, Sl);
    }
    return resid_df_finish(Sh, Sl, g.ih2f, L::ld(f + c), fmean);
}

// level-0 residual of either form (fmean: the mean of f, FP32-mixed form only)
template <class L, int DIM>
__device__ __forceinline__ double resid_form_at(const MGLevel& L0, const double* p, const double* f, float2, long c) {
    const double* b[3] = {L0.beta[0], L0.beta[1], L0.beta[2]};
    return resid64_at<L, DIM>(L0.g, b, p, f, c);
}
template <class L, int DIM>
__device__ __forceinline__ float resid_form_at(const MGLevel& L0, const float2* p, const float* f, float2 fmean,
                                               long c) {
    const float* b[3] = {L0.bf[0], L0.bf[1], L0.bf[2]};
    return resid_df_at<L, DIM>(L0.g, b, p, f, fmean, c);
}

// typed views of the level-0 pressure and right-hand side
template <typename T>
__host__ __device__ __forceinline__ PT<T>* pbuf(const MGLevel& L0) { return reinterpret_cast<PT<T>*>(L0.p); }
template <typename T>
__host__ __device__ __forceinline__ FT<T>* fbuf(const MGLevel& L0) { return reinterpret_cast<FT<T>*>(L0.f); }

// pressure updates of either form
__device__ __forceinline__ double p_add(double p, float e) { return p + (double)e; }
__device__ __forceinline__ float2 p_add(float2 p, float e) { return dfl::add(p, e); }
__device__ __forceinline__ double p_sub(double p, double m, float2) { return p - m; }
__device__ __forceinline__ float2 p_sub(float2 p, double, float2 m) { return dfl::sub(p, m); }
__device__ __forceinline__ double p_extrap(double pn, double po) { return 2.0 * pn - po; }
__device__ __forceinline__ float2 p_extrap(float2 pn, float2 po) {
    return dfl::sub(make_float2(2.f * pn.x, 2.f * pn.y), po);
}
template <typename T> __device__ __forceinline__ PT<T> p_zero();
template <> __device__ __forceinline__ double p_zero<double>() { return 0.0; }
template <> __device__ __forceinline__ float2 p_zero<float>() { return make_float2(0.f, 0.f); }
// difference of two pressures in the arithmetic type of the form
__device__ __forceinline__ double p_diff(double a, double b) { return a - b; }
__device__ __forceinline__ float p_diff(float2 a, float2 b) { return (a.x - b.x) + (a.y - b.y); }

// Coarse correction at coarse cell t after its right-hand side fc_t is known:
// zero (cb null: the level starts from zero elsewhere), or, on a red cell
// ((i + j + k) even: the colour smoothed first), the first Gauss-Seidel step
// from zero, -fc_t / diag (rbgs_at with kNbZero); black cells are left for the
// black half-sweep, which overwrites them without reading them.
template <class L, typename M, int DIM>
__device__ __forceinline__ void coarse_start(const Geom& gc, const M* const* cb, const IJK& Q, long t, M fct, M* pc) {
    if (!cb) {
        pc[t] = M(0);
        return;
    }
    if (((Q.i + Q.j + Q.k) & 1) != 0) return;
    M diag, off;
    stencil_L<L, M, DIM>(gc, cb, Q, t, g_ih2<M>(gc), [](long) { return M(0); }, diag, off);
    pc[t] = step_div(off - fct, diag);
}

// coarse cell t: mean of the 2^D fine residuals, then coarse_start
template <class L, typename M, int DIM>
__device__ __forceinline__ void resid_restrict_at(const Geom& gf, const Geom& gc, const M* const* beta, const M* p,
                                                  const M* f, M* fc, M* pc, long t, const M* const* cb = nullptr) {
    const IJK Q = decode(gc, t);
    const M ih2 = g_ih2<M>(gf);
    const int o2 = (DIM == 3) ? 2 : 1;
    M s = M(0);
    for (int t2 = 0; t2 < o2; ++t2)
        for (int t1 = 0; t1 < 2; ++t1)
            for (int t0 = 0; t0 < 2; ++t0) {
                IJK q;
                q.i = 2 * Q.i + t0;
                q.j = 2 * Q.j + t1;
                q.k = (DIM == 3) ? 2 * Q.k + t2 : 0;
                const long c = idx(gf, q);
                M diag, off;
                const M Lp = apply_L<L, M, DIM>(gf, beta, p, q, c, ih2, diag, off);
                s += L::ld(f + c) - Lp;
            }
    const M v = s * (M(1) / M(4 * o2));
    fc[t] = v;
    coarse_start<L, M, DIM>(gc, cb, Q, t, v, pc);
}

// resid_restrict_at on level 0 with density-formed coefficients (apply_L_rho)
template <class L, int DIM>
__device__ __forceinline__ void resid_restrict_rho_at(const Geom& gf, const Geom& gc, const float* rho, const float* p,
                                                      const float* f, float* fc, float* pc, long t,
                                                      const float* const* cb = nullptr) {
    const IJK Q = decode(gc, t);
    const int o2 = (DIM == 3) ? 2 : 1;
    float s = 0.f;
    for (int t2 = 0; t2 < o2; ++t2)
        for (int t1 = 0; t1 < 2; ++t1)
            for (int t0 = 0; t0 < 2; ++t0) {
                IJK q;
                q.i = 2 * Q.i + t0;
                q.j = 2 * Q.j + t1;
                q.k = (DIM == 3) ? 2 * Q.k + t2 : 0;
                const long c = idx(gf, q);
                float diag, off;
                const float Lp = apply_L_rho<L, DIM>(gf, rho, p, q, c, gf.ih2f, diag, off);
                s += L::ld(f + c) - Lp;
            }
    const float v = s * (1.f / (float)(4 * o2));
    fc[t] = v;
    coarse_start<L, float, DIM>(gc, cb, Q, t, v, pc);
}

// cell-centred (bi/tri)linear prolongation, weights 3/4 and 1/4 per axis;
// beyond a wall the coarse value is reflected (Neumann)
template <class L, typename M, int DIM>
__device__ __forceinline__ M prolong_val(const Geom& gf, const Geom& gc, const M* pc, long c) {
    const IJK q = decode(gf, c);
    int I[3][2];
    M w[3][2];
#pragma unroll
    for (int b = 0; b < 3; ++b) {
        if (b >= DIM) { I[b][0] = I[b][1] = 0; w[b][0] = M(1); w[b][1] = M(0); continue; }
        const int qb = coord(q, b);
        const int P = qb >> 1;
        int nb = (qb & 1) ? P + 1 : P - 1;
        if (b == DIM - 1) nb = min(max(nb, 0), gc.n[b] - 1);
        else { if (nb < 0) nb += gc.n[b]; else if (nb >= gc.n[b]) nb -= gc.n[b]; }
        I[b][0] = P;
        I[b][1] = nb;
        w[b][0] = M(0.75);
        w[b][1] = M(0.25);
    }
    M s = M(0);
#pragma unroll
    for (int t2 = 0; t2 < (DIM == 3 ? 2 : 1); ++t2)
#pragma unroll
        for (int t1 = 0; t1 < 2; ++t1)
#pragma unroll
            for (int t0 = 0; t0 < 2; ++t0)
                s += w[0][t0] * w[1][t1] * w[2][t2] * L::ld(pc + encode(gc, I[0][t0], I[1][t1], I[2][t2]));
    return s;
}

template <class L, typename M, int DIM>
__device__ __forceinline__ void prolong_at(const Geom& gf, const Geom& gc, const M* pc, M* p, long c) {
    p[c] = L::ld(p + c) + prolong_val<L, M, DIM>(gf, gc, pc, c);
}

// u = u* - c dt grad p / rho_f on the interior faces of cell c
template <class L, typename T, int DIM>
__device__ __forceinline__ void project_at(const Geom& g, const PhysDev& ph, const T* phi, T* const* us, T cdt,
                                           const PT<T>* p, long c) {
    const IJK q = decode(g, c);
    const T ih = g_ih<T>(g), dr = phys<T>(ph).drho, rho2 = phys<T>(ph).rho2;
#pragma unroll
    for (int a = 0; a < DIM; ++a) {
        if (a == DIM - 1 && coord(q, a) == 0) continue;  // wall face stays zero
        const long cL = idx(g, shift(g, q, a, -1));
        const T rf = T(0.5) * ((dr * L::ld(phi + cL) + rho2) + (dr * L::ld(phi + c) + rho2));
        const T beta = T(1) / rf;
        const T dp = p_diff(L::ld(p + c), L::ld(p + cL)) * ih;
        us[a][c] = L::ld(us[a] + c) - cdt * beta * dp;
    }
}

// ---------------------------------------------------------------------------
// Coarsest level (at most kMaxCoarse cells), solved by one thread block.
// The matrix A of the level plus the rank-one term c 1 1^T (c = -(mean
// diagonal magnitude) / n) is negative definite: A is negative semidefinite
// with the constants as its null space, and the rank-one term is negative on
// them.  Its coefficients are fixed during a pressure solve, so the block
// inverts it once per solve in FP32 (coarse_invert_block: in-place
// Gauss-Jordan elimination, which needs no pivoting for a definite matrix;
// the shift c is stored after the n x n inverse) and every V-cycle solves
// (A + c 1 1^T) e = r in FP64 (coarse_apply_block): e = Ainv r, then two
// steps of iterative refinement whose residuals r - (A + c 1 1^T) e are
// formed in FP64 from the level's coefficients, each corrected with the FP32
// inverse.  The FP32 inverse has a relative error of about 1e-7 cond(A), so
// two steps bring e to FP64 round-off for the condition numbers of these
// small levels; an FP64 inverse would cost n^3 FP64 operations on one SM per
// solve.  With a right-hand side summing to zero, the solution also solves
// A e = r with sum(e) = 0.
// ---------------------------------------------------------------------------
template <class L, typename M, int DIM>
__device__ void coarse_invert_block(const Geom& g, const M* const* beta, float* A, float* fct, float* shift_s) {
    const int n = (int)g.N;
    const float ih2 = g.ih2f;
    for (int t = threadIdx.x; t < n * n; t += blockDim.x) A[t] = 0.f;
    __syncthreads();
    for (int c = threadIdx.x; c < n; c += blockDim.x) {  // row c of A
        const IJK q = decode(g, c);
        float diag = 0.f;
        for (int a = 0; a < DIM; ++a) {
            const long hi = (a == DIM - 1) ? c + g.NP : idx(g, shift(g, q, a, 1));
            const float bm = (float)L::ld(beta[a] + c), bp = (float)L::ld(beta[a] + hi);
            diag -= (bm + bp) * ih2;
            if (bm != 0.f) A[c * n + idx(g, shift(g, q, a, -1))] += bm * ih2;
            if (bp != 0.f) A[c * n + hi] += bp * ih2;
        }
        A[c * n + c] += diag;
        fct[c] = -diag;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        float dsum = 0.f;
        for (int c = 0; c < n; ++c) dsum += fct[c];
        *shift_s = -dsum / ((float)n * (float)n);
    }
    __syncthreads();
    const float sh = *shift_s;
    for (int t = threadIdx.x; t < n * n; t += blockDim.x) A[t] += sh;
    __syncthreads();
    for (int k = 0; k < n; ++k) {
        const float piv = A[k * n + k];
        for (int i = threadIdx.x; i < n; i += blockDim.x) fct[i] = A[i * n + k];
        __syncthreads();
        for (int jj = threadIdx.x; jj < n; jj += blockDim.x) A[k * n + jj] = (jj == k ? 1.f : A[k * n + jj]) / piv;
        __syncthreads();
        for (int t = threadIdx.x; t < n * n; t += blockDim.x) {
            const int i = t / n, jj = t - i * n;
            if (i == k) continue;
            A[t] = (jj == k ? 0.f : A[t]) - fct[i] * A[k * n + jj];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) A[n * n] = sh;  // the shift, read by coarse_apply_block
    __syncthreads();
}

// x[c] += Ainv y on the coarsest level (Ainv symmetric up to rounding; thread
// c reads column c, so neighbouring threads read neighbouring words)
__device__ __forceinline__ void coarse_ainv_add(int n, const float* Ainv, const double* y, double* x, bool add) {
    for (int c = threadIdx.x; c < n; c += blockDim.x) {
        float s = 0.f;
        for (int t = 0; t < n; ++t) s += Ainv[t * n + c] * (float)y[t];
        x[c] = add ? x[c] + (double)s : (double)s;
    }
}

// e = (A + c 1 1^T)^-1 r in FP64 (see above); rd, ed, rr: 3 x n doubles of
// block-shared scratch; beta: the level's face coefficients
template <class L, typename M, int DIM>
__device__ void coarse_apply_block(const Geom& g, const M* const* beta, const float* Ainv, const M* r, M* e,
                                   double* rd, double* ed, double* rr) {
    const int n = (int)g.N;
    const double ih2 = g.ih2;
    const double sh = (double)Ainv[n * n];
    for (int c = threadIdx.x; c < n; c += blockDim.x) rd[c] = (double)L::ld(r + c);
    __syncthreads();
    coarse_ainv_add(n, Ainv, rd, ed, false);
    __syncthreads();
    for (int it = 0; it < 2; ++it) {
        for (int c = threadIdx.x; c < n; c += blockDim.x) {
            double esum = 0.0;
            for (int t = 0; t < n; ++t) esum += ed[t];
            const IJK q = decode(g, c);
            double Ae = 0.0;
            for (int a = 0; a < DIM; ++a) {
                const long hi = (a == DIM - 1) ? c + g.NP : idx(g, shift(g, q, a, 1));
                const double bm = (double)L::ld(beta[a] + c), bp = (double)L::ld(beta[a] + hi);
                if (bm != 0.0) Ae += bm * (ed[idx(g, shift(g, q, a, -1))] - ed[c]);
                if (bp != 0.0) Ae += bp * (ed[hi] - ed[c]);
            }
            rr[c] = rd[c] - (Ae * ih2 + sh * esum);
        }
        __syncthreads();
        coarse_ainv_add(n, Ainv, rr, ed, true);
        __syncthreads();
    }
    for (int c = threadIdx.x; c < n; c += blockDim.x) e[c] = (M)ed[c];
    __syncthreads();
}

}  // namespace ops
}  // namespace cdi
