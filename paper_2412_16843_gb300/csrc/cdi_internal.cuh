// Internal declarations of libcdi.so: grid geometry, the bundle of device
// field pointers, index helpers shared by the kernels, and the launchers.
//
// Layout in the workspace: every field is a flat array with x fastest.  Cell
// fields hold N = nx*ny(*nz) values.  Velocity component a holds its faces
// with the same linear index as the cell whose low face it is; the component
// normal to the walls (the last axis) has one extra plane of NP values
// (NP = cells in a wall plane) for the high wall.  So the low face of cell c
// is entry c of every component.
#pragma once

#include <cuda_runtime.h>
#include <cstddef>
#include <cstdint>

namespace cdi {

constexpr int kMaxLevels = 16;
constexpr int kMaxCoarse = 64;      // cells of the coarsest multigrid level
constexpr int kPartials = 1024;     // blocks of the fixed-order reductions

struct Geom {
    int D;        // 2 or 3
    int n[3];     // cells per axis, n[2] = 1 in 2D
    int W;        // wall axis = D-1
    long N;       // cells
    long NP;      // cells of one wall plane (= stride of the wall axis)
    double h;
};

// slip model ids (the CDI_MODEL_* values of cdi.h)
enum { M1A = 0, M1B, M2A, M2B, M3A, M3B, M4A, M4B };

struct WallDev {
    double costh;       // cos(theta_eq)
    double beta1, beta2;
    double U[2];        // tangential wall velocity (x, y)
    int noslip;         // beta infinite
};

struct PhysDev {
    double rho1, rho2, mu1, mu2, sigma, eps;
    double delta, tau;  // clamp of phi for psi; floor of |grad psi|
    int model;
    WallDev wall[2];
};

// Device pointers of one evaluation (stage state in, stage results out).
template <typename T>
struct StageFields {
    const T* phi;       // stage phi [N]
    const T* u[3];      // stage velocity components
    T* psi;             // [N]
    T* nh[3];           // cell-centre normal [N] per axis
    T* muc;             // chemical potential [N]
    T* m[3];            // face mass flux
    T* rphi;            // phi right-hand side [N]
    T* rm[3];           // face momentum right-hand side
    T* wuY;             // [2][D-1][NP]
    T* wghost;          // [2][D-1][NP]
    T* wmuw;            // [2][D-1][NP]
    const double* gamma;  // device scalar
};

// ---------------------------------------------------------------------------
// index helpers
// ---------------------------------------------------------------------------
struct IJK {
    int i, j, k;
};

__host__ __device__ inline IJK decode(const Geom& g, long c) {
    IJK q;
    q.i = (int)(c % g.n[0]);
    long r = c / g.n[0];
    q.j = (int)(r % g.n[1]);
    q.k = (int)(r / g.n[1]);
    return q;
}
__host__ __device__ inline long encode(const Geom& g, int i, int j, int k) {
    return (long)i + (long)g.n[0] * ((long)j + (long)g.n[1] * k);
}
__host__ __device__ inline int coord(const IJK& q, int a) { return a == 0 ? q.i : (a == 1 ? q.j : q.k); }
__host__ __device__ inline void setc(IJK& q, int a, int v) {
    if (a == 0) q.i = v; else if (a == 1) q.j = v; else q.k = v;
}
// shift by s along axis a; periodic axes wrap (|s| <= n), the wall axis does not
__host__ __device__ inline IJK shift(const Geom& g, IJK q, int a, int s) {
    int v = coord(q, a) + s;
    if (a != g.W) {
        if (v < 0) v += g.n[a];
        else if (v >= g.n[a]) v -= g.n[a];
    }
    setc(q, a, v);
    return q;
}
__host__ __device__ inline long idx(const Geom& g, const IJK& q) { return encode(g, q.i, q.j, q.k); }

template <typename T>
__host__ __device__ inline T clampv(T x, T lo, T hi) { return x < lo ? lo : (x > hi ? hi : x); }

// ---------------------------------------------------------------------------
// launchers (stencils: k_stencil.cu; multigrid and reductions: k_mg.cu)
// ---------------------------------------------------------------------------
template <typename T>
void launch_rhs(const Geom& g, const PhysDev& ph, const StageFields<T>& f, cudaStream_t s);

template <typename T>
void launch_stage_update(const Geom& g, const PhysDev& ph, int stage, double dt,
                         const T* phi0, const T* const* u0, const T* rphi, const T* const* rm,
                         T* accphi, T* const* accm, T* phik, T* const* uk, cudaStream_t s);

template <typename T>
void launch_wall_columns(const Geom& g, const PhysDev& ph, const T* phi, T* psi, double* cols,
                         cudaStream_t s);

// multigrid hierarchy, all arrays in double
struct MGLevel {
    int n[3];
    long N, NP;
    double h;
    double* p;
    double* f;
    double* beta[3];
};

struct MG {
    int nlev;
    MGLevel lv[kMaxLevels];
    double* partials;   // [kPartials]
    double* scal;       // device scalars
    double* host_scal;  // pinned host mirror (nullable)
};

// scalar slots in MG::scal
enum { S_MEAN = 0, S_FNORM = 1, S_RNORM = 2, S_MASS = 3, S_UMAX = 4, S_GAMMA = 5,
       S_THETA = 6, S_WETTED = 7, S_NSCAL = 16 };

template <typename T>
void launch_div(const Geom& g, const T* const* us, double inv_cdt, MG& mg, cudaStream_t s);
void launch_sum_f(const Geom& g, MG& mg, cudaStream_t s);
void launch_sub_mean_and_norm(const Geom& g, MG& mg, cudaStream_t s);
template <typename T>
void launch_mg_coef(const Geom& g, const PhysDev& ph, const T* phi, MG& mg, cudaStream_t s);
void launch_vcycle(const Geom& g, MG& mg, int npre, int npost, cudaStream_t s);
void launch_resid_norm(const Geom& g, MG& mg, cudaStream_t s);
void launch_p_mean_remove(const Geom& g, MG& mg, cudaStream_t s);
template <typename T>
void launch_project(const Geom& g, const PhysDev& ph, const T* phi, T* const* us, double cdt,
                    const double* p, cudaStream_t s);
template <typename T>
void launch_mass(const Geom& g, const T* phi, MG& mg, cudaStream_t s);
template <typename T>
void launch_gamma(const Geom& g, const T* const* u, double gamma_param, MG& mg, cudaStream_t s);
void launch_contact_line(const Geom& g, int wall, const double* cols, MG& mg, cudaStream_t s);

// number of kernel launches issued since the counter was reset (host side)
extern thread_local long g_launches;

}  // namespace cdi
