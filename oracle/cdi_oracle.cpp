// Plain FP64 CPU oracle for one time step of the conservative diffuse interface
// (CDI) two-phase solver with the GNBC contact-line treatment of Brown,
// Mirjalili, Khanwale & Mani (arXiv 2412.16843).
//
// TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the bench's
// CPU-baseline leg load this library.  It shares no code, header, table or
// helper with the CUDA library; both receive their inputs from the seeded
// generators in paper_2412_16843_gb300/inputs.py.
//
// It is deliberately slow and literal: one loop per formula, no blocking, no
// fusion, no reordering beyond what the formulas state.  Compiled with
// -O2 -ffp-contract=off so x86 and Arm give the same bits.
//
// What each part follows (paper sections and equations):
//   psi, grad psi, lap psi, normal, curvature, chemical potential
//       Eq. (psi), Eq. (chemical potential), Eq. (curvature), Sec. 4
//       (second-order central differences inside, second-order one-sided
//       wall-normal stencils in the first and last cell rows)
//   phi flux and wall no-flux      Eq. (CDI), Eq. (no-flux BC), Eq. (no-penetration BC)
//   mass flux of the momentum eq.  Eq. (NS_momentum) with S = (rho1-rho2) R
//   surface tension                Eq. (EB surface tension)
//   GNBC slip, Model 4A            Eq. (slip BC), (u_slip_v), (u_slip_Y) = Model 4A,
//                                  beta linear in phi (Sec. 2), first-order linear
//                                  extrapolation of wall quantities (Sec. 4)
//   other slip models 1A..4B       Eqs. (Model 1A) .. (Model 4B), Sec. 3
//   time stepping                  classical RK4 (Sec. 4)
//   pressure projection            Eq. (NS_incompressibility); the linear solve is a
//                                  geometric multigrid (no solver is named in the paper)
//   mass, contact angle            Sec. 2 (conservation), Sec. 3.1 (angle of the
//                                  phi = 0.5 contour), Sec. 5.1 (wetted length)
//
// Readings where the paper is silent (discretisation details are deferred to
// references that are not part of the paper): the face values are arithmetic
// means of the two adjacent cells; the normal on a face is the mean of the two
// cell-centre normals; the velocity slip condition is imposed through a ghost
// value below the wall; every stage value of RK4 and the final value are
// projected; psi uses phi clamped to [delta, 1-delta] (delta = 1e-6, a clamp
// that FP32 arithmetic also represents, so both precisions share it).
//
// In 3D (an extension: the paper is 2D) the in-plane curvature kappa_p is the
// EB curvature minus the normal curvature along the contact-line direction
// s = n_phi x n_wall; it equals kappa exactly for data invariant along y.

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <vector>

namespace {

using vec = std::vector<double>;

enum { ORC_OK = 0, ORC_EINVAL = 1, ORC_ESTATE = 2, ORC_ENOCONV = 4, ORC_ENAN = 5 };

// Slip models of Sec. 3 (Eqs. Model 1A .. Model 4B).
enum { M1A = 0, M1B, M2A, M2B, M3A, M3B, M4A, M4B };

struct Grid {
    int D = 2;
    int n[3] = {1, 1, 1};
    double h = 1.0;
    int W = 1;  // wall axis: the last axis
    long N() const { return (long)n[0] * n[1] * n[2]; }
    // number of faces of velocity component a along axis b
    int fdim(int a, int b) const { return n[b] + ((a == W && b == W) ? 1 : 0); }
    long NF(int a) const { return (long)fdim(a, 0) * fdim(a, 1) * fdim(a, 2); }
};

struct Q { int v[3]; int& operator[](int i) { return v[i]; } int operator[](int i) const { return v[i]; } };

inline Q sh(Q q, int b, int s) { q[b] += s; return q; }

inline int wrap(int i, int n) { i %= n; return i < 0 ? i + n : i; }

// cell index; periodic wrap on every axis but the wall axis
inline long C(const Grid& g, Q q) {
    for (int b = 0; b < 3; ++b) if (b != g.W) q[b] = wrap(q[b], g.n[b]);
    return q[0] + (long)g.n[0] * (q[1] + (long)g.n[1] * q[2]);
}
// face index of component a; face q is the low face of cell q
inline long F(const Grid& g, int a, Q q) {
    for (int b = 0; b < 3; ++b) if (b != g.W) q[b] = wrap(q[b], g.n[b]);
    return q[0] + (long)g.fdim(a, 0) * (q[1] + (long)g.fdim(a, 1) * q[2]);
}

inline double clampd(double x, double lo, double hi) { return x < lo ? lo : (x > hi ? hi : x); }

struct WallParams {
    double theta = M_PI / 2;
    double beta1 = INFINITY, beta2 = INFINITY;  // infinite friction = no slip
    double U[2] = {0.0, 0.0};                     // tangential wall velocity (x, y)
};

struct Level {
    int n[3];
    double h;
    vec beta[3];  // face coefficients 1/rho_f, face layout as the velocity components
    vec p, f, r;
};

struct Solver {
    Grid g;
    double rho1 = 1, rho2 = 1, mu1 = 1, mu2 = 1, sigma = 0, eps = 1, gamma = 0;
    WallParams wall[2];
    int model = M4A;
    double delta = 1e-6, tau = 1e-6;  // clamp of phi for psi and phi(1-phi); floor of |grad psi|
    double tol = 1e-10;
    int maxcyc = 200;
    int warm = 1;           // 1: previous pressure as the first guess, 0: zero
    int npre = 2, npost = 2;
    int project_stages = 1; // 1: project every RK stage value and the final value
    vec phi, u[3], p;
    int last_cycles = 0, max_cycles_step = 0;
    double last_resid = 0;
    long total_cycles = 0;
    std::vector<Level> lv;
};

// ---------------------------------------------------------------------------
// a1: psi and its derivatives at cell centres
// ---------------------------------------------------------------------------
struct PsiOut {
    vec psi, g[3], lap, kappa, muc, nh[3];
};

// derivative along axis b at cell q: central inside, second-order one-sided in
// the first and last rows of the wall axis (Sec. 4)
static void d12(const Grid& g, const vec& s, Q q, int b, double& d1, double& d2) {
    const double h = g.h;
    const int nb = g.n[b];
    if (b == g.W && q[b] == 0) {
        double s0 = s[C(g, q)], s1 = s[C(g, sh(q, b, 1))], s2 = s[C(g, sh(q, b, 2))], s3 = s[C(g, sh(q, b, 3))];
        d1 = (-3.0 * s0 + 4.0 * s1 - s2) / (2.0 * h);
        d2 = (2.0 * s0 - 5.0 * s1 + 4.0 * s2 - s3) / (h * h);
    } else if (b == g.W && q[b] == nb - 1) {
        double s0 = s[C(g, q)], s1 = s[C(g, sh(q, b, -1))], s2 = s[C(g, sh(q, b, -2))], s3 = s[C(g, sh(q, b, -3))];
        d1 = (3.0 * s0 - 4.0 * s1 + s2) / (2.0 * h);
        d2 = (2.0 * s0 - 5.0 * s1 + 4.0 * s2 - s3) / (h * h);
    } else {
        double sm = s[C(g, sh(q, b, -1))], s0 = s[C(g, q)], sp = s[C(g, sh(q, b, 1))];
        d1 = (sp - sm) / (2.0 * h);
        d2 = (sp - 2.0 * s0 + sm) / (h * h);
    }
}

static void eval_psi(const Solver& S, const vec& phi, PsiOut& o) {
    const Grid& g = S.g;
    const long N = g.N();
    o.psi.assign(N, 0.0);
    o.lap.assign(N, 0.0);
    o.kappa.assign(N, 0.0);
    o.muc.assign(N, 0.0);
    for (int b = 0; b < 3; ++b) { o.g[b].assign(N, 0.0); o.nh[b].assign(N, 0.0); }
    // Eq. (psi) with phi clamped away from 0 and 1
    for (long c = 0; c < N; ++c) {
        double pt = clampd(phi[c], S.delta, 1.0 - S.delta);
        o.psi[c] = S.eps * std::log(pt / (1.0 - pt));
    }
    for (int k = 0; k < g.n[2]; ++k)
        for (int j = 0; j < g.n[1]; ++j)
            for (int i = 0; i < g.n[0]; ++i) {
                Q q{{i, j, k}};
                long c = C(g, q);
                double grad2 = 0.0, lap = 0.0;
                for (int b = 0; b < g.D; ++b) {
                    double d1, d2;
                    d12(g, o.psi, q, b, d1, d2);
                    o.g[b][c] = d1;
                    grad2 += d1 * d1;
                    lap += d2;
                }
                double pt = clampd(phi[c], S.delta, 1.0 - S.delta);
                // Eq. (curvature)
                o.kappa[c] = (1.0 - 2.0 * pt) * (1.0 - grad2) / S.eps - lap;
                // Eq. (chemical potential)
                o.muc[c] = 6.0 * S.sigma *
                           (pt * (1.0 - pt) * (1.0 - 2.0 * pt) * (1.0 - grad2) / S.eps - pt * (1.0 - pt) * lap);
                o.lap[c] = lap;
                double gm = std::sqrt(grad2);
                for (int b = 0; b < g.D; ++b) o.nh[b][c] = o.g[b][c] / (gm + S.tau);
            }
}

// ---------------------------------------------------------------------------
// a2: wall rows -- extrapolated wall quantities, GNBC slip, ghost velocity
// ---------------------------------------------------------------------------
struct WallOut {
    // per wall s, per tangential component a (< D-1), per face position in the
    // wall plane (nx in 2D, nx*ny in 3D)
    vec uY[2][2], ghost[2][2], muw[2][2];
    // per wall, per wall column (cell position in the wall plane)
    vec phiw[2], psiw[2], dnw[2], kpw[2], gtw[2][2], dnphiw[2], gtphiw[2][2];
};

static long plane_index(const Grid& g, Q q) {  // q[W] ignored
    int i = wrap(q[0], g.n[0]);
    if (g.D == 2) return i;
    int j = wrap(q[1], g.n[1]);
    return i + (long)g.n[0] * j;
}

// Face quantities entering the slip models (all at one tangential-velocity
// face position on the wall).
struct SlipIn {
    double P;       // phi(1-phi) of the wall phi
    double dnpsi;   // d psi / d n_wall
    double dtpsi;   // d psi / d tau_wall
    double gpsi;    // |grad psi|
    double dnphi;   // d phi / d n_wall
    double dtphi;   // d phi / d tau_wall
    double gphi;    // |grad phi|
    double kp;      // in-plane curvature kappa_p
    double psi;     // psi on the wall
};

// Eqs. (Model 1A) .. (Model 4B): u^Y = -(6 sigma / beta) [ A + B cos(theta_eq) ] T
static double slip_model(const Solver& S, int model, const SlipIn& x, double beta, double costh) {
    const double e = S.eps;
    const bool corr = (model == M3A || model == M3B || model == M4A || model == M4B);
    const double cc = corr ? (1.0 + x.kp * x.psi) : 1.0;
    double A, B, T;
    switch (model) {
        case M1A: case M3A:   // phi derivatives, equilibrium form
            A = e * x.dnphi; B = x.P * cc; T = x.dtphi; break;
        case M1B: case M3B:   // phi derivatives, eps |grad phi|
            A = e * x.dnphi; B = e * x.gphi * cc; T = x.dtphi; break;
        case M2A: case M4A:   // psi derivatives, equilibrium form
            A = x.P * x.dnpsi; B = x.P * cc; T = x.P / e * x.dtpsi; break;
        case M2B: case M4B: default:  // psi derivatives, |grad psi|
            A = x.P * x.dnpsi; B = x.P * x.gpsi * cc; T = x.P / e * x.dtpsi; break;
    }
    return -(6.0 * S.sigma / beta) * (A + B * costh) * T;
}

static void eval_wall(const Solver& S, const vec& phi, const vec* u, const PsiOut& ps, WallOut& w) {
    const Grid& g = S.g;
    const int W = g.W, nW = g.n[W];
    const long NP = (g.D == 2) ? g.n[0] : (long)g.n[0] * g.n[1];
    for (int s = 0; s < 2; ++s) {
        const int r0 = s == 0 ? 0 : nW - 1, r1 = s == 0 ? 1 : nW - 2;
        const double sgn = s == 0 ? 1.0 : -1.0;  // inward normal along +W (low) or -W (high)
        w.phiw[s].assign(NP, 0.0);
        w.psiw[s].assign(NP, 0.0);
        w.dnw[s].assign(NP, 0.0);
        w.kpw[s].assign(NP, 0.0);
        w.dnphiw[s].assign(NP, 0.0);
        for (int t = 0; t < 2; ++t) { w.gtw[s][t].assign(NP, 0.0); w.gtphiw[s][t].assign(NP, 0.0); }
        for (int j = 0; j < (g.D == 3 ? g.n[1] : 1); ++j)
            for (int i = 0; i < g.n[0]; ++i) {
                Q q0{{i, j, 0}}, q1{{i, j, 0}};
                q0[W] = r0;
                q1[W] = r1;
                if (g.D == 2) { q0[2] = 0; q1[2] = 0; }
                long c0 = C(g, q0), c1 = C(g, q1);
                long pi = plane_index(g, q0);
                // in-plane curvature kappa_p at the two rows
                double kp[2];
                long cc[2] = {c0, c1};
                Q qq[2] = {q0, q1};
                for (int r = 0; r < 2; ++r) {
                    double kap = ps.kappa[cc[r]];
                    if (g.D == 3) {
                        Q q = qq[r];
                        const double h = g.h;
                        double px = ps.g[0][cc[r]], py = ps.g[1][cc[r]];
                        double pxx = (ps.psi[C(g, sh(q, 0, 1))] - 2.0 * ps.psi[cc[r]] + ps.psi[C(g, sh(q, 0, -1))]) / (h * h);
                        double pyy = (ps.psi[C(g, sh(q, 1, 1))] - 2.0 * ps.psi[cc[r]] + ps.psi[C(g, sh(q, 1, -1))]) / (h * h);
                        double pxy = (ps.psi[C(g, sh(sh(q, 0, 1), 1, 1))] - ps.psi[C(g, sh(sh(q, 0, 1), 1, -1))] -
                                      ps.psi[C(g, sh(sh(q, 0, -1), 1, 1))] + ps.psi[C(g, sh(sh(q, 0, -1), 1, -1))]) /
                                     (4.0 * h * h);
                        double gm = std::sqrt(px * px + py * py + ps.g[2][cc[r]] * ps.g[2][cc[r]]);
                        double t2 = px * px + py * py;
                        double num = py * py * pxx - 2.0 * px * py * pxy + px * px * pyy;
                        double ks = -num / ((t2 + S.tau * S.tau) * (gm + S.tau));
                        kap -= ks;
                    }
                    kp[r] = kap;
                }
                // phi derivatives at the two rows (for the phi-based models only)
                double dphi[2][3];
                for (int r = 0; r < 2; ++r)
                    for (int b = 0; b < g.D; ++b) {
                        double d1, d2;
                        d12(g, phi, qq[r], b, d1, d2);
                        dphi[r][b] = d1;
                    }
                // first-order linear extrapolation from the two first cell centres
                w.phiw[s][pi] = clampd(0.5 * (3.0 * phi[c0] - phi[c1]), 0.0, 1.0);
                w.psiw[s][pi] = 0.5 * (3.0 * ps.psi[c0] - ps.psi[c1]);
                w.dnw[s][pi] = 0.5 * (3.0 * sgn * ps.g[W][c0] - sgn * ps.g[W][c1]);
                w.kpw[s][pi] = 0.5 * (3.0 * kp[0] - kp[1]);
                w.dnphiw[s][pi] = 0.5 * (3.0 * sgn * dphi[0][W] - sgn * dphi[1][W]);
                for (int t = 0; t < g.D - 1; ++t) {
                    w.gtw[s][t][pi] = 0.5 * (3.0 * ps.g[t][c0] - ps.g[t][c1]);
                    w.gtphiw[s][t][pi] = 0.5 * (3.0 * dphi[0][t] - dphi[1][t]);
                }
            }
        const WallParams& wp = S.wall[s];
        const bool noslip = std::isinf(wp.beta1) || std::isinf(wp.beta2);
        const double costh = std::cos(wp.theta);
        for (int a = 0; a < g.D - 1; ++a) {
            w.uY[s][a].assign(NP, 0.0);
            w.ghost[s][a].assign(NP, 0.0);
            w.muw[s][a].assign(NP, 0.0);
            for (int j = 0; j < (g.D == 3 ? g.n[1] : 1); ++j)
                for (int i = 0; i < g.n[0]; ++i) {
                    Q q{{i, j, 0}};
                    if (g.D == 2) q[2] = 0;
                    q[W] = r0;
                    long pR = plane_index(g, q), pL = plane_index(g, sh(q, a, -1));
                    // face values: means of the two adjacent wall columns, compact d_tau
                    double pb = 0.5 * (w.phiw[s][pL] + w.phiw[s][pR]);
                    SlipIn x;
                    x.P = pb * (1.0 - pb);
                    x.psi = 0.5 * (w.psiw[s][pL] + w.psiw[s][pR]);
                    x.dnpsi = 0.5 * (w.dnw[s][pL] + w.dnw[s][pR]);
                    x.kp = 0.5 * (w.kpw[s][pL] + w.kpw[s][pR]);
                    x.dtpsi = (w.psiw[s][pR] - w.psiw[s][pL]) / g.h;
                    x.dnphi = 0.5 * (w.dnphiw[s][pL] + w.dnphiw[s][pR]);
                    x.dtphi = (w.phiw[s][pR] - w.phiw[s][pL]) / g.h;
                    double gs = x.dnpsi * x.dnpsi, gf = x.dnphi * x.dnphi;
                    for (int t = 0; t < g.D - 1; ++t) {
                        double gt = (t == a) ? x.dtpsi : 0.5 * (w.gtw[s][t][pL] + w.gtw[s][t][pR]);
                        double gtf = (t == a) ? x.dtphi : 0.5 * (w.gtphiw[s][t][pL] + w.gtphiw[s][t][pR]);
                        gs += gt * gt;
                        gf += gtf * gtf;
                    }
                    x.gpsi = std::sqrt(gs);
                    x.gphi = std::sqrt(gf);
                    double muw = (S.mu1 - S.mu2) * pb + S.mu2;
                    double uY = 0.0, lw = 0.0;
                    if (!noslip) {
                        double beta = (wp.beta1 - wp.beta2) * pb + wp.beta2;  // beta linear in phi
                        uY = slip_model(S, S.model, x, beta, costh);
                        lw = muw / beta;
                    }
                    long f0 = F(g, a, q);
                    double u0 = u[a][f0];
                    // ghost: u_w = (u0 + ug)/2, d_n u = (u0 - ug)/h,
                    // u_w - U = (mu_w/beta_w) d_n u + u^Y   (Eqs. slip BC, u_slip_v)
                    double ug = (wp.U[a] + uY - u0 * (0.5 - lw / g.h)) / (0.5 + lw / g.h);
                    w.uY[s][a][pR] = uY;
                    w.ghost[s][a][pR] = ug;
                    w.muw[s][a][pR] = muw;
                }
        }
    }
}

// ---------------------------------------------------------------------------
// a3: phi flux, its divergence and the consistent mass flux
// ---------------------------------------------------------------------------
static void eval_phi_flux(const Solver& S, const vec& phi, const vec* u, const PsiOut& ps, double gamma,
                          vec& rhs, vec* m) {
    const Grid& g = S.g;
    const int W = g.W;
    vec Fx[3];
    for (int a = 0; a < g.D; ++a) {
        Fx[a].assign(g.NF(a), 0.0);
        m[a].assign(g.NF(a), 0.0);
        for (int k = 0; k < g.fdim(a, 2); ++k)
            for (int j = 0; j < g.fdim(a, 1); ++j)
                for (int i = 0; i < g.fdim(a, 0); ++i) {
                    Q q{{i, j, k}};
                    long f = F(g, a, q);
                    if (a == W && (q[W] == 0 || q[W] == g.n[W])) {  // wall face: no flux
                        Fx[a][f] = 0.0;
                        m[a][f] = 0.0;
                        continue;
                    }
                    long cR = C(g, q), cL = C(g, sh(q, a, -1));
                    double pb = 0.5 * (phi[cL] + phi[cR]);
                    double pc = clampd(pb, S.delta, 1.0 - S.delta);
                    double nb = 0.5 * (ps.nh[a][cL] + ps.nh[a][cR]);
                    // u phi - R with R = gamma [eps grad phi - phi(1-phi) n]  (Eq. CDI)
                    double flux = u[a][f] * pb - gamma * (S.eps * (phi[cR] - phi[cL]) / g.h - pc * (1.0 - pc) * nb);
                    Fx[a][f] = flux;
                    // rho u - S = (rho1 - rho2)(u phi - R) + rho2 u  (Eq. NS_momentum)
                    m[a][f] = (S.rho1 - S.rho2) * flux + S.rho2 * u[a][f];
                }
    }
    rhs.assign(g.N(), 0.0);
    for (int k = 0; k < g.n[2]; ++k)
        for (int j = 0; j < g.n[1]; ++j)
            for (int i = 0; i < g.n[0]; ++i) {
                Q q{{i, j, k}};
                double div = 0.0;
                for (int a = 0; a < g.D; ++a) div += Fx[a][F(g, a, sh(q, a, 1))] - Fx[a][F(g, a, q)];
                rhs[C(g, q)] = -div / g.h;
            }
}

// ---------------------------------------------------------------------------
// a4: momentum right-hand side on every velocity face (without pressure)
// ---------------------------------------------------------------------------
static void eval_mom(const Solver& S, const vec& phi, const vec* u, const vec* m, const PsiOut& ps,
                     const WallOut& w, vec* rhs) {
    const Grid& g = S.g;
    const int W = g.W, nW = g.n[W];
    const double h = g.h;
    auto mu = [&](long c) { return (S.mu1 - S.mu2) * phi[c] + S.mu2; };
    for (int a = 0; a < g.D; ++a) {
        rhs[a].assign(g.NF(a), 0.0);
        for (int k = 0; k < g.fdim(a, 2); ++k)
            for (int j = 0; j < g.fdim(a, 1); ++j)
                for (int i = 0; i < g.fdim(a, 0); ++i) {
                    Q q{{i, j, k}};
                    long f = F(g, a, q);
                    if (a == W && (q[W] == 0 || q[W] == nW)) { rhs[a][f] = 0.0; continue; }
                    long cR = C(g, q), cL = C(g, sh(q, a, -1));
                    double adv = 0.0, vis = 0.0;
                    for (int b = 0; b < g.D; ++b) {
                        if (b == a) {
                            // fluxes at the two cell centres bounding the momentum cell
                            auto cflux = [&](Q qc, double& conv, double& tau) {
                                long flo = F(g, a, qc), fhi = F(g, a, sh(qc, a, 1));
                                double mb = 0.5 * (m[a][flo] + m[a][fhi]);
                                double ub = 0.5 * (u[a][flo] + u[a][fhi]);
                                conv = mb * ub;
                                tau = 2.0 * mu(C(g, qc)) * (u[a][fhi] - u[a][flo]) / h;
                            };
                            double chi, thi, clo, tlo;
                            cflux(q, chi, thi);
                            cflux(sh(q, a, -1), clo, tlo);
                            adv -= (chi - clo) / h;
                            vis += (thi - tlo) / h;
                        } else {
                            // fluxes at the two edges (b-low and b-high) of the momentum cell
                            double conv[2], tau[2];
                            for (int side = 0; side < 2; ++side) {
                                int eb = q[b] + side;  // b-face index of the edge
                                if (b == W && (eb == 0 || eb == nW)) {
                                    int s = eb == 0 ? 0 : 1;
                                    Q qr = q;  // the momentum face in the row next to the wall
                                    long pi = plane_index(g, qr);
                                    double ug = w.ghost[s][a][pi];
                                    double u0 = u[a][F(g, a, qr)];
                                    conv[side] = 0.0;  // no mass flux through the wall
                                    // wall shear from the ghost value; d_a u_W = 0 on the wall
                                    tau[side] = (s == 0) ? w.muw[s][a][pi] * (u0 - ug) / h
                                                         : w.muw[s][a][pi] * (ug - u0) / h;
                                    continue;
                                }
                                Q qhi = q;
                                qhi[b] = eb;       // momentum face above the edge
                                Q qlo = sh(qhi, b, -1);
                                double ub = 0.5 * (u[a][F(g, a, qlo)] + u[a][F(g, a, qhi)]);
                                // mass flux m_b at b-face eb of the two cells adjacent along a
                                double mb = 0.5 * (m[b][F(g, b, qhi)] + m[b][F(g, b, sh(qhi, a, -1))]);
                                conv[side] = mb * ub;
                                double me = 0.25 * (mu(C(g, qhi)) + mu(C(g, sh(qhi, a, -1))) + mu(C(g, qlo)) +
                                                    mu(C(g, sh(qlo, a, -1))));
                                double dub = (u[a][F(g, a, qhi)] - u[a][F(g, a, qlo)]) / h;
                                double dua = (u[b][F(g, b, qhi)] - u[b][F(g, b, sh(qhi, a, -1))]) / h;
                                tau[side] = me * (dub + dua);
                            }
                            adv -= (conv[1] - conv[0]) / h;
                            vis += (tau[1] - tau[0]) / h;
                        }
                    }
                    // Eq. (EB surface tension) on the face
                    double st = 0.5 * (ps.muc[cL] + ps.muc[cR]) * (phi[cR] - phi[cL]) / h;
                    rhs[a][f] = adv + vis + st;
                }
    }
}

// ---------------------------------------------------------------------------
// a7: multigrid for div( (1/rho_f) grad p ) = f, periodic + Neumann at walls
// ---------------------------------------------------------------------------
static int L_fdim(const Grid& g, const Level& L, int a, int b) {
    return L.n[b] + ((a == g.W && b == g.W) ? 1 : 0);
}
static long LC(const Grid& g, const Level& L, Q q) {
    for (int b = 0; b < 3; ++b) if (b != g.W) q[b] = wrap(q[b], L.n[b]);
    return q[0] + (long)L.n[0] * (q[1] + (long)L.n[1] * q[2]);
}
static long LF(const Grid& g, const Level& L, int a, Q q) {
    for (int b = 0; b < 3; ++b) if (b != g.W) q[b] = wrap(q[b], L.n[b]);
    return q[0] + (long)L_fdim(g, L, a, 0) * (q[1] + (long)L_fdim(g, L, a, 1) * q[2]);
}
static long LN(const Level& L) { return (long)L.n[0] * L.n[1] * L.n[2]; }

static void build_levels(Solver& S) {
    const Grid& g = S.g;
    S.lv.clear();
    Level L0;
    for (int b = 0; b < 3; ++b) L0.n[b] = g.n[b];
    L0.h = g.h;
    S.lv.push_back(L0);
    for (;;) {
        const Level& L = S.lv.back();
        bool ok = true;
        for (int b = 0; b < g.D; ++b) if (L.n[b] % 2 != 0 || L.n[b] / 2 < 2) ok = false;
        if (!ok) break;
        Level Lc;
        for (int b = 0; b < 3; ++b) Lc.n[b] = (b < g.D) ? L.n[b] / 2 : 1;
        Lc.h = 2.0 * L.h;
        S.lv.push_back(Lc);
    }
    for (auto& L : S.lv) {
        long n = LN(L);
        L.p.assign(n, 0.0);
        L.f.assign(n, 0.0);
        L.r.assign(n, 0.0);
        for (int a = 0; a < g.D; ++a)
            L.beta[a].assign((long)L_fdim(g, L, a, 0) * L_fdim(g, L, a, 1) * L_fdim(g, L, a, 2), 0.0);
    }
}

static void set_coefficients(Solver& S, const vec& phi) {
    const Grid& g = S.g;
    auto rho = [&](long c) { return (S.rho1 - S.rho2) * phi[c] + S.rho2; };
    Level& L0 = S.lv[0];
    for (int a = 0; a < g.D; ++a)
        for (int k = 0; k < L_fdim(g, L0, a, 2); ++k)
            for (int j = 0; j < L_fdim(g, L0, a, 1); ++j)
                for (int i = 0; i < L_fdim(g, L0, a, 0); ++i) {
                    Q q{{i, j, k}};
                    long f = LF(g, L0, a, q);
                    if (a == g.W && (q[a] == 0 || q[a] == L0.n[a])) { L0.beta[a][f] = 0.0; continue; }
                    double rf = 0.5 * (rho(LC(g, L0, sh(q, a, -1))) + rho(LC(g, L0, q)));
                    L0.beta[a][f] = 1.0 / rf;
                }
    // coarse face coefficient = mean of the fine faces covering it
    for (size_t l = 1; l < S.lv.size(); ++l) {
        Level& Lf = S.lv[l - 1];
        Level& Lc = S.lv[l];
        for (int a = 0; a < g.D; ++a)
            for (int k = 0; k < L_fdim(g, Lc, a, 2); ++k)
                for (int j = 0; j < L_fdim(g, Lc, a, 1); ++j)
                    for (int i = 0; i < L_fdim(g, Lc, a, 0); ++i) {
                        Q q{{i, j, k}};
                        double sum = 0.0;
                        int cnt = 0;
                        int o1 = (g.D >= 2) ? 2 : 1, o2 = (g.D == 3) ? 2 : 1;
                        // children faces: index 2q along a, 2q and 2q+1 along the others
                        for (int t2 = 0; t2 < o2; ++t2)
                            for (int t1 = 0; t1 < o1; ++t1) {
                                Q qf{{2 * q[0], 2 * q[1], 2 * q[2]}};
                                if (g.D == 2) qf[2] = 0;
                                int other[2], no = 0;
                                for (int b = 0; b < g.D; ++b) if (b != a) other[no++] = b;
                                if (no > 0) qf[other[0]] += t1;
                                if (no > 1) qf[other[1]] += t2;
                                sum += Lf.beta[a][LF(g, Lf, a, qf)];
                                ++cnt;
                            }
                        Lc.beta[a][LF(g, Lc, a, q)] = sum / cnt;
                    }
    }
}

static double apply_L(const Solver& S, const Level& L, const vec& p, Q q, double* diag_out, double* off_out) {
    const Grid& g = S.g;
    long c = LC(g, L, q);
    double diag = 0.0, off = 0.0;
    for (int a = 0; a < g.D; ++a) {
        double bm = L.beta[a][LF(g, L, a, q)];
        double bp = L.beta[a][LF(g, L, a, sh(q, a, 1))];
        double pm = (bm != 0.0) ? p[LC(g, L, sh(q, a, -1))] : 0.0;
        double pp = (bp != 0.0) ? p[LC(g, L, sh(q, a, 1))] : 0.0;
        double ih2 = 1.0 / (L.h * L.h);
        diag += (bm + bp) * ih2;
        off += (bm * pm + bp * pp) * ih2;
    }
    if (diag_out) *diag_out = diag;
    if (off_out) *off_out = off;
    return off - diag * p[c];
}

static void residual(const Solver& S, Level& L) {
    const Grid& g = S.g;
    for (int k = 0; k < L.n[2]; ++k)
        for (int j = 0; j < L.n[1]; ++j)
            for (int i = 0; i < L.n[0]; ++i) {
                Q q{{i, j, k}};
                long c = LC(g, L, q);
                L.r[c] = L.f[c] - apply_L(S, L, L.p, q, nullptr, nullptr);
            }
}

static void rbgs(const Solver& S, Level& L) {
    const Grid& g = S.g;
    for (int colour = 0; colour < 2; ++colour)
        for (int k = 0; k < L.n[2]; ++k)
            for (int j = 0; j < L.n[1]; ++j)
                for (int i = 0; i < L.n[0]; ++i) {
                    if (((i + j + k) & 1) != colour) continue;
                    Q q{{i, j, k}};
                    double diag, off;
                    apply_L(S, L, L.p, q, &diag, &off);
                    L.p[LC(g, L, q)] = (off - L.f[LC(g, L, q)]) / diag;
                }
}

// direct solve of the (singular) coarse system: (L + c 1 1^T) p = f, Gaussian
// elimination with partial pivoting; c makes the constant mode nonsingular
static void dense_solve(const Solver& S, Level& L) {
    const Grid& g = S.g;
    const long n = LN(L);
    std::vector<double> A(n * n, 0.0), b(n);
    double dsum = 0.0;
    for (int k = 0; k < L.n[2]; ++k)
        for (int j = 0; j < L.n[1]; ++j)
            for (int i = 0; i < L.n[0]; ++i) {
                Q q{{i, j, k}};
                long c = LC(g, L, q);
                double ih2 = 1.0 / (L.h * L.h);
                for (int a = 0; a < g.D; ++a) {
                    double bm = L.beta[a][LF(g, L, a, q)];
                    double bp = L.beta[a][LF(g, L, a, sh(q, a, 1))];
                    A[c * n + c] -= (bm + bp) * ih2;
                    if (bm != 0.0) A[c * n + LC(g, L, sh(q, a, -1))] += bm * ih2;
                    if (bp != 0.0) A[c * n + LC(g, L, sh(q, a, 1))] += bp * ih2;
                }
                dsum += -A[c * n + c];
                b[c] = L.f[c];
            }
    const double shift = -dsum / ((double)n * (double)n);  // same sign as the diagonal
    for (long i = 0; i < n * n; ++i) A[i] += shift;
    for (long col = 0; col < n; ++col) {
        long piv = col;
        for (long r = col + 1; r < n; ++r)
            if (std::fabs(A[r * n + col]) > std::fabs(A[piv * n + col])) piv = r;
        if (piv != col) {
            for (long t = 0; t < n; ++t) std::swap(A[col * n + t], A[piv * n + t]);
            std::swap(b[col], b[piv]);
        }
        for (long r = col + 1; r < n; ++r) {
            double fct = A[r * n + col] / A[col * n + col];
            if (fct == 0.0) continue;
            for (long t = col; t < n; ++t) A[r * n + t] -= fct * A[col * n + t];
            b[r] -= fct * b[col];
        }
    }
    for (long r = n - 1; r >= 0; --r) {
        double s = b[r];
        for (long t = r + 1; t < n; ++t) s -= A[r * n + t] * L.p[t];
        L.p[r] = s / A[r * n + r];
    }
}

static void restrict_residual(const Solver& S, const Level& Lf, Level& Lc) {
    const Grid& g = S.g;
    const int o0 = 2, o1 = 2, o2 = (g.D == 3) ? 2 : 1;
    const double w = 1.0 / (o0 * o1 * o2);
    for (int k = 0; k < Lc.n[2]; ++k)
        for (int j = 0; j < Lc.n[1]; ++j)
            for (int i = 0; i < Lc.n[0]; ++i) {
                double s = 0.0;
                for (int t2 = 0; t2 < o2; ++t2)
                    for (int t1 = 0; t1 < o1; ++t1)
                        for (int t0 = 0; t0 < o0; ++t0) {
                            Q qf{{2 * i + t0, 2 * j + t1, (g.D == 3) ? 2 * k + t2 : 0}};
                            s += Lf.r[LC(g, Lf, qf)];
                        }
                Lc.f[LC(g, Lc, Q{{i, j, k}})] = s * w;
            }
}

// cell-centred (bi/tri)linear prolongation, weights 3/4 and 1/4 per axis;
// beyond a wall the coarse value is reflected (Neumann)
static void prolong_add(const Solver& S, const Level& Lc, Level& Lf) {
    const Grid& g = S.g;
    for (int k = 0; k < Lf.n[2]; ++k)
        for (int j = 0; j < Lf.n[1]; ++j)
            for (int i = 0; i < Lf.n[0]; ++i) {
                Q qf{{i, j, k}};
                int I[3][2];
                double wgt[3][2];
                for (int b = 0; b < 3; ++b) {
                    if (b >= g.D) { I[b][0] = I[b][1] = 0; wgt[b][0] = 1.0; wgt[b][1] = 0.0; continue; }
                    int pc = qf[b] / 2;
                    int nb = (qf[b] % 2 == 0) ? pc - 1 : pc + 1;
                    if (b == g.W) nb = std::min(std::max(nb, 0), Lc.n[b] - 1);
                    I[b][0] = pc;
                    I[b][1] = nb;
                    wgt[b][0] = 0.75;
                    wgt[b][1] = 0.25;
                }
                double s = 0.0;
                for (int t2 = 0; t2 < 2; ++t2)
                    for (int t1 = 0; t1 < 2; ++t1)
                        for (int t0 = 0; t0 < 2; ++t0) {
                            double wv = wgt[0][t0] * wgt[1][t1] * wgt[2][t2];
                            if (wv == 0.0) continue;
                            s += wv * Lc.p[LC(g, Lc, Q{{I[0][t0], I[1][t1], I[2][t2]}})];
                        }
                Lf.p[LC(g, Lf, qf)] += s;
            }
}

static void vcycle(Solver& S, size_t l) {
    Level& L = S.lv[l];
    if (l + 1 == S.lv.size()) { dense_solve(S, L); return; }
    for (int s = 0; s < S.npre; ++s) rbgs(S, L);
    residual(S, L);
    Level& Lc = S.lv[l + 1];
    restrict_residual(S, L, Lc);
    std::fill(Lc.p.begin(), Lc.p.end(), 0.0);
    vcycle(S, l + 1);
    prolong_add(S, Lc, L);
    for (int s = 0; s < S.npost; ++s) rbgs(S, L);
}

static double norm2(const vec& v) {
    double s = 0.0;
    for (double x : v) s += x * x;
    return std::sqrt(s);
}

// solve with f given on level 0 (mean already removed) and the first guess in lv[0].p
static int mg_solve(Solver& S, int* cycles, double* rel) {
    Level& L = S.lv[0];
    double fn = norm2(L.f);
    *cycles = 0;
    if (fn == 0.0) {
        std::fill(L.p.begin(), L.p.end(), 0.0);
        *rel = 0.0;
        return ORC_OK;
    }
    residual(S, L);
    double rn = norm2(L.r);
    while (rn > S.tol * fn && *cycles < S.maxcyc) {
        vcycle(S, 0);
        ++*cycles;
        residual(S, L);
        rn = norm2(L.r);
        if (!std::isfinite(rn)) return ORC_ENAN;
    }
    *rel = rn / fn;
    double mean = 0.0;
    for (double x : L.p) mean += x;
    mean /= (double)L.p.size();
    for (double& x : L.p) x -= mean;
    return (rn > S.tol * fn) ? ORC_ENOCONV : ORC_OK;
}

// a6 + a7 + a8: u = u* - c dt grad p / rho_f with div( grad p / rho_f ) = div u* / (c dt)
static int project(Solver& S, const vec& phi, vec* us, double cdt) {
    const Grid& g = S.g;
    set_coefficients(S, phi);
    Level& L = S.lv[0];
    for (int k = 0; k < g.n[2]; ++k)
        for (int j = 0; j < g.n[1]; ++j)
            for (int i = 0; i < g.n[0]; ++i) {
                Q q{{i, j, k}};
                double div = 0.0;
                for (int a = 0; a < g.D; ++a) div += us[a][F(g, a, sh(q, a, 1))] - us[a][F(g, a, q)];
                L.f[C(g, q)] = div / g.h / cdt;
            }
    double mean = 0.0;
    for (double x : L.f) mean += x;
    mean /= (double)L.f.size();
    for (double& x : L.f) x -= mean;
    if (S.warm && S.p.size() == L.p.size()) L.p = S.p;
    else std::fill(L.p.begin(), L.p.end(), 0.0);
    int cyc;
    double rel;
    int st = mg_solve(S, &cyc, &rel);
    S.last_cycles = cyc;
    S.last_resid = rel;
    S.total_cycles += cyc;
    S.max_cycles_step = std::max(S.max_cycles_step, cyc);
    if (st != ORC_OK) return st;
    S.p = L.p;
    for (int a = 0; a < g.D; ++a)
        for (int k = 0; k < g.fdim(a, 2); ++k)
            for (int j = 0; j < g.fdim(a, 1); ++j)
                for (int i = 0; i < g.fdim(a, 0); ++i) {
                    Q q{{i, j, k}};
                    if (a == g.W && (q[a] == 0 || q[a] == g.n[a])) continue;
                    long f = F(g, a, q);
                    double dp = (L.p[C(g, q)] - L.p[C(g, sh(q, a, -1))]) / g.h;
                    us[a][f] -= cdt * L.beta[a][f] * dp;
                }
    return ORC_OK;
}

// a1..a4 on a stage state
static void eval_rhs(const Solver& S, const vec& phi, const vec* u, double gamma, vec& rphi, vec* rmom,
                     PsiOut* ps_out = nullptr, WallOut* w_out = nullptr) {
    PsiOut ps;
    WallOut w;
    vec m[3];
    eval_psi(S, phi, ps);
    eval_wall(S, phi, u, ps, w);
    eval_phi_flux(S, phi, u, ps, gamma, rphi, m);
    eval_mom(S, phi, u, m, ps, w, rmom);
    if (ps_out) *ps_out = ps;
    if (w_out) *w_out = w;
}

static double umax(const Solver& S) {
    double mx = 0.0;
    for (int a = 0; a < S.g.D; ++a)
        for (double x : S.u[a]) mx = std::max(mx, std::fabs(x));
    return mx;
}

static double gamma_now(const Solver& S) {
    if (S.gamma >= 0.0) return S.gamma;
    return std::max(2.5 * umax(S), -S.gamma);  // gamma = 2.5 |u|_max, floored (Sec. 5.1)
}

// one RK4 step: stage states of phi and of the face momentum rho_f u,
// each stage velocity projected (a5)
static int step(Solver& S, double dt) {
    const Grid& g = S.g;
    const double ck[4] = {0.0, 0.5, 0.5, 1.0};
    const double bk[4] = {1.0 / 6.0, 1.0 / 3.0, 1.0 / 3.0, 1.0 / 6.0};
    const double gamma = gamma_now(S);
    auto rho = [&](const vec& ph, long c) { return (S.rho1 - S.rho2) * ph[c] + S.rho2; };
    auto rhof = [&](const vec& ph, int a, Q q) {
        return 0.5 * (rho(ph, C(g, sh(q, a, -1))) + rho(ph, C(g, q)));
    };
    const vec phi0 = S.phi;
    vec M0[3], accM[3], uk[3], Mk[3], rmom[3];
    for (int a = 0; a < g.D; ++a) {
        M0[a].assign(g.NF(a), 0.0);
        accM[a].assign(g.NF(a), 0.0);
        for (int k = 0; k < g.fdim(a, 2); ++k)
            for (int j = 0; j < g.fdim(a, 1); ++j)
                for (int i = 0; i < g.fdim(a, 0); ++i) {
                    Q q{{i, j, k}};
                    if (a == g.W && (q[a] == 0 || q[a] == g.n[a])) continue;
                    long f = F(g, a, q);
                    M0[a][f] = rhof(phi0, a, q) * S.u[a][f];
                }
        uk[a] = S.u[a];
    }
    vec accphi(g.N(), 0.0), phik = phi0, rphi;
    S.max_cycles_step = 0;
    for (int st = 0; st < 4; ++st) {
        eval_rhs(S, phik, uk, gamma, rphi, rmom);
        for (long c = 0; c < g.N(); ++c) accphi[c] += bk[st] * rphi[c];
        for (int a = 0; a < g.D; ++a)
            for (long f = 0; f < g.NF(a); ++f) accM[a][f] += bk[st] * rmom[a][f];
        const bool last = (st == 3);
        const double c = last ? 1.0 : ck[st + 1];
        // next stage value (or the final value)
        for (long cc = 0; cc < g.N(); ++cc)
            phik[cc] = last ? phi0[cc] + dt * accphi[cc] : phi0[cc] + c * dt * rphi[cc];
        for (int a = 0; a < g.D; ++a) {
            Mk[a].assign(g.NF(a), 0.0);
            for (int k = 0; k < g.fdim(a, 2); ++k)
                for (int j = 0; j < g.fdim(a, 1); ++j)
                    for (int i = 0; i < g.fdim(a, 0); ++i) {
                        Q q{{i, j, k}};
                        long f = F(g, a, q);
                        if (a == g.W && (q[a] == 0 || q[a] == g.n[a])) { uk[a][f] = 0.0; continue; }
                        double Mv = last ? M0[a][f] + dt * accM[a][f] : M0[a][f] + c * dt * rmom[a][f];
                        uk[a][f] = Mv / rhof(phik, a, q);
                    }
        }
        if (S.project_stages || last) {
            int stt = project(S, phik, uk, c * dt);
            if (stt != ORC_OK) return stt;
        }
    }
    S.phi = phik;
    for (int a = 0; a < g.D; ++a) S.u[a] = uk[a];
    for (double x : S.phi) if (!std::isfinite(x)) return ORC_ENAN;
    return ORC_OK;
}

// a9: contact angle and wetted length on one wall (2D: both crossings of the
// extrapolated phi_w = 0.5 level; 3D: every x line of the wall plane)
static void contact_line(const Solver& S, int s, double* theta, double* wetted) {
    const Grid& g = S.g;
    PsiOut ps;
    WallOut w;
    eval_psi(S, S.phi, ps);
    eval_wall(S, S.phi, S.u, ps, w);
    const int nx = g.n[0];
    const int nlines = (g.D == 3) ? g.n[1] : 1;
    double th_sum = 0.0;
    long th_cnt = 0;
    double len_sum = 0.0;
    const double h = g.h;
    for (int line = 0; line < nlines; ++line) {
        const long base = (long)line * nx;
        auto phw = [&](int i) { return w.phiw[s][base + wrap(i, nx)]; };
        // wall gradient of psi at column i: central in x (and, in 3D, in y
        // across the neighbouring lines), extrapolated normal part
        const long bup = (long)((line + 1) % nlines) * nx, bdn = (long)((line + nlines - 1) % nlines) * nx;
        auto grad_at = [&](int i, double& gn, double& gt, double& gy) {
            gn = w.dnw[s][base + wrap(i, nx)];
            gt = (w.psiw[s][base + wrap(i + 1, nx)] - w.psiw[s][base + wrap(i - 1, nx)]) / (2.0 * h);
            gy = (g.D == 3) ? (w.psiw[s][bup + wrap(i, nx)] - w.psiw[s][bdn + wrap(i, nx)]) / (2.0 * h) : 0.0;
        };
        int i0 = 0;
        for (int i = 1; i < nx; ++i) if (phw(i) < phw(i0)) i0 = i;
        double xl = 0.0, xr = 0.0;
        bool have_l = false, have_r = false;
        double thl = 0.0, thr = 0.0;
        for (int kk = 1; kk <= nx && !have_r; ++kk) {
            int ip = i0 + kk - 1, ic = i0 + kk;
            double a0 = phw(ip), a1 = phw(ic);
            bool crossing = (!have_l) ? (a0 < 0.5 && a1 >= 0.5) : (a0 >= 0.5 && a1 < 0.5);
            if (!crossing) continue;
            double t = (0.5 - a0) / (a1 - a0);
            double x = ((double)ip + 0.5 + t) * h;
            double gn0, gt0, gy0, gn1, gt1, gy1;
            grad_at(ip, gn0, gt0, gy0);
            grad_at(ic, gn1, gt1, gy1);
            double gn = gn0 + t * (gn1 - gn0), gt = gt0 + t * (gt1 - gt0), gy = gy0 + t * (gy1 - gy0);
            // theta = acos(-d_n psi / |grad psi|) with the whole wall gradient
            double gm = (g.D == 3) ? std::sqrt(gn * gn + gt * gt + gy * gy) : std::sqrt(gn * gn + gt * gt);
            double th = std::acos(clampd(-gn / gm, -1.0, 1.0));
            if (!have_l) { xl = x; thl = th; have_l = true; }
            else { xr = x; thr = th; have_r = true; }
        }
        if (have_l && have_r) {
            th_sum += thl + thr;
            th_cnt += 2;
            len_sum += (g.D == 3) ? (xr - xl) * h : (xr - xl);
        }
    }
    if (th_cnt == 0) { *theta = NAN; *wetted = 0.0; return; }
    *theta = th_sum / th_cnt;
    if (g.D == 2) *wetted = len_sum;
    else *wetted = 2.0 * std::sqrt(len_sum / M_PI);  // equivalent base diameter
}

// copy helpers between the solver's face layout and the caller's arrays (same layout)
static void copy_in(vec& dst, const double* src, long n) { dst.assign(src, src + n); }

}  // namespace

// ===========================================================================
// C API used by the Python test harness (ctypes)
// ===========================================================================
extern "C" {

void* orc_create(int dim, int nx, int ny, int nz, double Lx, double Ly, double Lz) {
    if (dim != 2 && dim != 3) return nullptr;
    if (nx < 2 || ny < 4 || (dim == 3 && nz < 4)) return nullptr;
    auto* S = new Solver();
    S->g.D = dim;
    S->g.n[0] = nx;
    S->g.n[1] = ny;
    S->g.n[2] = (dim == 3) ? nz : 1;
    S->g.W = dim - 1;
    S->g.h = Lx / nx;
    (void)Ly;
    (void)Lz;
    S->phi.assign(S->g.N(), 0.0);
    for (int a = 0; a < dim; ++a) S->u[a].assign(S->g.NF(a), 0.0);
    S->p.assign(S->g.N(), 0.0);
    build_levels(*S);
    return S;
}

void orc_destroy(void* h) { delete (Solver*)h; }

int orc_set_fluids(void* h, double rho1, double rho2, double mu1, double mu2, double sigma, double eps,
                   double gamma) {
    auto* S = (Solver*)h;
    S->rho1 = rho1; S->rho2 = rho2; S->mu1 = mu1; S->mu2 = mu2;
    S->sigma = sigma; S->eps = eps; S->gamma = gamma;
    return ORC_OK;
}

// wall: 0 low, 1 high, 2 both; beta = INFINITY means no slip
int orc_set_wall(void* h, int wall, double theta, double beta1, double beta2, double Ux, double Uy) {
    auto* S = (Solver*)h;
    for (int s = 0; s < 2; ++s) {
        if (wall != 2 && wall != s) continue;
        S->wall[s].theta = theta;
        S->wall[s].beta1 = beta1;
        S->wall[s].beta2 = beta2;
        S->wall[s].U[0] = Ux;
        S->wall[s].U[1] = Uy;
    }
    return ORC_OK;
}

int orc_set_model(void* h, int model) { ((Solver*)h)->model = model; return ORC_OK; }

int orc_set_solver(void* h, double tol, int maxcyc, int warm) {
    auto* S = (Solver*)h;
    S->tol = tol; S->maxcyc = maxcyc; S->warm = warm;
    return ORC_OK;
}

int orc_set_regularisation(void* h, double delta, double tau) {
    auto* S = (Solver*)h;
    S->delta = delta; S->tau = tau;
    return ORC_OK;
}

int orc_set_state(void* h, const double* phi, const double* u, const double* v, const double* w, const double* p) {
    auto* S = (Solver*)h;
    const Grid& g = S->g;
    copy_in(S->phi, phi, g.N());
    const double* comps[3] = {u, v, w};
    for (int a = 0; a < g.D; ++a) copy_in(S->u[a], comps[a], g.NF(a));
    if (p) copy_in(S->p, p, g.N());
    else S->p.assign(g.N(), 0.0);
    return ORC_OK;
}

int orc_get_state(void* h, double* phi, double* u, double* v, double* w, double* p) {
    auto* S = (Solver*)h;
    const Grid& g = S->g;
    if (phi) std::memcpy(phi, S->phi.data(), sizeof(double) * g.N());
    double* comps[3] = {u, v, w};
    for (int a = 0; a < g.D; ++a) if (comps[a]) std::memcpy(comps[a], S->u[a].data(), sizeof(double) * g.NF(a));
    if (p) std::memcpy(p, S->p.data(), sizeof(double) * g.N());
    return ORC_OK;
}

int orc_step(void* h, double dt, int nsteps) {
    auto* S = (Solver*)h;
    for (int n = 0; n < nsteps; ++n) {
        int st = step(*S, dt);
        if (st != ORC_OK) return st;
    }
    return ORC_OK;
}

int orc_project_final_only(void* h, int flag) { ((Solver*)h)->project_stages = flag ? 0 : 1; return ORC_OK; }

double orc_mass(void* h) {
    auto* S = (Solver*)h;
    const Grid& g = S->g;
    double dv = std::pow(g.h, g.D);
    // pairwise-free plain sum; the phi values are O(1)
    double s = 0.0;
    for (double x : S->phi) s += x;
    return s * dv;
}

int orc_contact_angle(void* h, int wall, double* theta, double* wetted) {
    contact_line(*(Solver*)h, wall, theta, wetted);
    return ORC_OK;
}

int orc_last_stats(void* h, int* cycles, double* resid, int* max_cycles_step, long* total) {
    auto* S = (Solver*)h;
    if (cycles) *cycles = S->last_cycles;
    if (resid) *resid = S->last_resid;
    if (max_cycles_step) *max_cycles_step = S->max_cycles_step;
    if (total) *total = S->total_cycles;
    return ORC_OK;
}

// a1 on a given phi: psi, grad psi (D arrays), lap psi, kappa, mu_c, normal (D arrays)
int orc_eval_psi(void* h, const double* phi_in, double* psi, double* gx, double* gy, double* gz, double* lap,
                 double* kappa, double* muc, double* nx, double* ny, double* nz) {
    auto* S = (Solver*)h;
    const Grid& g = S->g;
    vec phi(phi_in, phi_in + g.N());
    PsiOut o;
    eval_psi(*S, phi, o);
    long N = g.N();
    auto out = [&](double* d, const vec& s) { if (d) std::memcpy(d, s.data(), sizeof(double) * N); };
    out(psi, o.psi); out(gx, o.g[0]); out(gy, o.g[1]); if (g.D == 3) out(gz, o.g[2]);
    out(lap, o.lap); out(kappa, o.kappa); out(muc, o.muc);
    out(nx, o.nh[0]); out(ny, o.nh[1]); if (g.D == 3) out(nz, o.nh[2]);
    return ORC_OK;
}

// a2 on the current state: u^Y and ghost per wall and tangential component,
// layout [wall][comp][plane position]; phiw per wall column [wall][plane]
int orc_eval_wall(void* h, double* uY, double* ghost, double* phiw) {
    auto* S = (Solver*)h;
    const Grid& g = S->g;
    PsiOut ps;
    WallOut w;
    eval_psi(*S, S->phi, ps);
    eval_wall(*S, S->phi, S->u, ps, w);
    long NP = (g.D == 2) ? g.n[0] : (long)g.n[0] * g.n[1];
    for (int s = 0; s < 2; ++s) {
        for (int a = 0; a < g.D - 1; ++a) {
            if (uY) std::memcpy(uY + (s * (g.D - 1) + a) * NP, w.uY[s][a].data(), sizeof(double) * NP);
            if (ghost) std::memcpy(ghost + (s * (g.D - 1) + a) * NP, w.ghost[s][a].data(), sizeof(double) * NP);
        }
        if (phiw) std::memcpy(phiw + s * NP, w.phiw[s].data(), sizeof(double) * NP);
    }
    return ORC_OK;
}

// wall-column quantities of the current state, per wall and column of the wall
// plane: the extrapolated psi_w and in-plane curvature kappa_p (read-only view
// of eval_wall's intermediate values, for the closed-form pins)
int orc_eval_wall_columns(void* h, double* psiw, double* kpw) {
    auto* S = (Solver*)h;
    const Grid& g = S->g;
    PsiOut ps;
    WallOut w;
    eval_psi(*S, S->phi, ps);
    eval_wall(*S, S->phi, S->u, ps, w);
    long NP = (g.D == 2) ? g.n[0] : (long)g.n[0] * g.n[1];
    for (int s = 0; s < 2; ++s) {
        if (psiw) std::memcpy(psiw + s * NP, w.psiw[s].data(), sizeof(double) * NP);
        if (kpw) std::memcpy(kpw + s * NP, w.kpw[s].data(), sizeof(double) * NP);
    }
    return ORC_OK;
}

// a1..a4 on the current state with the given gamma (gamma < 0: the step's rule)
int orc_eval_rhs(void* h, double gamma, double* rphi, double* ru, double* rv, double* rw) {
    auto* S = (Solver*)h;
    const Grid& g = S->g;
    vec rp, rm[3];
    double gm = (gamma >= 0.0) ? gamma : gamma_now(*S);
    eval_rhs(*S, S->phi, S->u, gm, rp, rm);
    if (rphi) std::memcpy(rphi, rp.data(), sizeof(double) * g.N());
    double* outs[3] = {ru, rv, rw};
    for (int a = 0; a < g.D; ++a) if (outs[a]) std::memcpy(outs[a], rm[a].data(), sizeof(double) * g.NF(a));
    return ORC_OK;
}

// a7 alone: solve div(grad p / rho_f(phi)) = f (f's mean removed first) with the
// current phi; p is the first guess on entry and the mean-free solution on exit
int orc_poisson(void* h, const double* f, double* p, int* cycles, double* resid) {
    auto* S = (Solver*)h;
    const Grid& g = S->g;
    set_coefficients(*S, S->phi);
    Level& L = S->lv[0];
    L.f.assign(f, f + g.N());
    double mean = 0.0;
    for (double x : L.f) mean += x;
    mean /= (double)g.N();
    for (double& x : L.f) x -= mean;
    L.p.assign(p, p + g.N());
    int cyc = 0;
    double rel = 0.0;
    int st = mg_solve(*S, &cyc, &rel);
    if (cycles) *cycles = cyc;
    if (resid) *resid = rel;
    std::memcpy(p, L.p.data(), sizeof(double) * g.N());
    return st;
}

// direct dense solve of the same system on the fine grid (small grids only)
int orc_poisson_direct(void* h, const double* f, double* p) {
    auto* S = (Solver*)h;
    const Grid& g = S->g;
    if (g.N() > 4096) return ORC_EINVAL;
    set_coefficients(*S, S->phi);
    Level& L = S->lv[0];
    L.f.assign(f, f + g.N());
    double mean = 0.0;
    for (double x : L.f) mean += x;
    mean /= (double)g.N();
    for (double& x : L.f) x -= mean;
    dense_solve(*S, L);
    mean = 0.0;
    for (double x : L.p) mean += x;
    mean /= (double)g.N();
    for (long c = 0; c < g.N(); ++c) p[c] = L.p[c] - mean;
    return ORC_OK;
}

// apply the pressure operator (for residual checks in the tests)
int orc_apply_laplacian(void* h, const double* p, double* out) {
    auto* S = (Solver*)h;
    const Grid& g = S->g;
    set_coefficients(*S, S->phi);
    Level& L = S->lv[0];
    vec pv(p, p + g.N());
    for (int k = 0; k < g.n[2]; ++k)
        for (int j = 0; j < g.n[1]; ++j)
            for (int i = 0; i < g.n[0]; ++i) {
                Q q{{i, j, k}};
                out[C(g, q)] = apply_L(*S, L, pv, q, nullptr, nullptr);
            }
    return ORC_OK;
}

// divergence of the current velocity at cell centres
int orc_divergence(void* h, double* out) {
    auto* S = (Solver*)h;
    const Grid& g = S->g;
    for (int k = 0; k < g.n[2]; ++k)
        for (int j = 0; j < g.n[1]; ++j)
            for (int i = 0; i < g.n[0]; ++i) {
                Q q{{i, j, k}};
                double div = 0.0;
                for (int a = 0; a < g.D; ++a) div += S->u[a][F(g, a, sh(q, a, 1))] - S->u[a][F(g, a, q)];
                out[C(g, q)] = div / g.h;
            }
    return ORC_OK;
}

int orc_num_levels(void* h) { return (int)((Solver*)h)->lv.size(); }

}  // extern "C"
