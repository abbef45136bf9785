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

#include <cuda.h>
#include <cuda_runtime.h>
#include <cstddef>
#include <cstdint>

namespace cdi {

constexpr int kMaxLevels = 16;
constexpr int kMaxCoarse = 64;      // cells of the coarsest multigrid level
constexpr int kPartials = 1024;     // blocks of the fixed-order reductions

// Division by a runtime constant d of an unsigned x < 2^31 with one
// multiply-high, an add and a shift: q = (umulhi(x, m) + x) >> s with
// s = ceil(log2 d) and m = floor(2^32 (2^s - d) / d) + 1 (the round-up method
// of Granlund and Montgomery, "Division by invariant integers using
// multiplication", 1994).
struct FastDiv {
    unsigned d, m;
    int s;
    __host__ void init(unsigned dv) {
        d = dv;
        s = 0;
        while ((1ull << s) < dv) ++s;
        m = (unsigned)((((1ull << 32) * ((1ull << s) - dv)) / dv) + 1);
    }
    __host__ __device__ __forceinline__ unsigned div(unsigned x) const {
#ifdef __CUDA_ARCH__
        return (__umulhi(x, m) + x) >> s;
#else
        return x / d;
#endif
    }
};

struct Geom {
    int D;        // 2 or 3
    int n[3];     // cells per axis, n[2] = 1 in 2D
    int W;        // wall axis = D-1
    long N;       // cells
    long NP;      // cells of one wall plane (= stride of the wall axis)
    double h;
    double ih, ih2;         // 1/h, 1/h^2
    float hf, ihf, ih2f;    // FP32 copies (1/h and 1/h^2 rounded from the FP32 h and h^2)
    FastDiv fd0, fd1;  // division by n[0] and by n[1]
};

// 1/h and 1/h^2 in the arithmetic type of a kernel.  On GB300 an FP64
// instruction (including a conversion from FP64) issues at a small fraction of
// the FP32 rate, so FP32 kernels take the FP32 copies made on the host.
template <typename T> __host__ __device__ __forceinline__ T g_ih(const Geom& g);
template <> __host__ __device__ __forceinline__ double g_ih<double>(const Geom& g) { return g.ih; }
template <> __host__ __device__ __forceinline__ float g_ih<float>(const Geom& g) { return g.ihf; }
template <typename T> __host__ __device__ __forceinline__ T g_ih2(const Geom& g);
template <> __host__ __device__ __forceinline__ double g_ih2<double>(const Geom& g) { return g.ih2; }
template <> __host__ __device__ __forceinline__ float g_ih2<float>(const Geom& g) { return g.ih2f; }

inline Geom make_geom(int D, const int n[3], double h) {
    Geom g{};
    g.D = D;
    for (int a = 0; a < 3; ++a) g.n[a] = n[a];
    g.W = D - 1;
    g.N = (long)n[0] * n[1] * n[2];
    g.NP = (D == 2) ? (long)n[0] : (long)n[0] * n[1];
    g.h = h;
    g.ih = 1.0 / h;
    g.ih2 = 1.0 / (h * h);
    g.hf = (float)h;
    g.ihf = 1.f / (float)h;
    g.ih2f = 1.f / (float)(h * h);
    g.fd0.init((unsigned)n[0]);
    g.fd1.init((unsigned)n[1]);
    return g;
}

// slip model ids (the CDI_MODEL_* values of cdi.h)
enum { M1A = 0, M1B, M2A, M2B, M3A, M3B, M4A, M4B };

struct WallDev {
    double costh;       // cos(theta_eq)
    double beta1, beta2;
    double U[2];        // tangential wall velocity (x, y)
    int noslip;         // beta infinite
};

// The parameters in one arithmetic type, with the differences the stencils use.
template <typename T>
struct PhysT {
    T rho1, rho2, mu1, mu2, sigma, eps, delta, tau;
    T drho, dmu;                       // rho1 - rho2, mu1 - mu2
    T costh[2], beta2[2], dbeta[2];    // per wall; dbeta = beta1 - beta2
    T U[2][2];                         // per wall, tangential components
};

struct PhysDev {
    double rho1, rho2, mu1, mu2, sigma, eps;
    double delta, tau;  // clamp of phi for psi; floor of |grad psi|
    int model;
    WallDev wall[2];
    PhysT<double> pd;   // copies in FP64 and FP32 (finalize_phys)
    PhysT<float> pf;
};

template <typename T>
inline void fill_phys(const PhysDev& ph, PhysT<T>& o) {
    o.rho1 = (T)ph.rho1; o.rho2 = (T)ph.rho2; o.mu1 = (T)ph.mu1; o.mu2 = (T)ph.mu2;
    o.sigma = (T)ph.sigma; o.eps = (T)ph.eps; o.delta = (T)ph.delta; o.tau = (T)ph.tau;
    o.drho = (T)(ph.rho1 - ph.rho2);
    o.dmu = (T)(ph.mu1 - ph.mu2);
    for (int s = 0; s < 2; ++s) {
        o.costh[s] = (T)ph.wall[s].costh;
        o.beta2[s] = (T)ph.wall[s].beta2;
        o.dbeta[s] = ph.wall[s].noslip ? T(0) : (T)(ph.wall[s].beta1 - ph.wall[s].beta2);
        o.U[s][0] = (T)ph.wall[s].U[0];
        o.U[s][1] = (T)ph.wall[s].U[1];
    }
}

// refresh the typed copies after any change of the FP64 parameters
inline void finalize_phys(PhysDev& ph) {
    fill_phys<double>(ph, ph.pd);
    fill_phys<float>(ph, ph.pf);
}

template <typename T> __host__ __device__ __forceinline__ const PhysT<T>& phys(const PhysDev& ph);
template <> __host__ __device__ __forceinline__ const PhysT<double>& phys<double>(const PhysDev& ph) { return ph.pd; }
template <> __host__ __device__ __forceinline__ const PhysT<float>& phys<float>(const PhysDev& ph) { return ph.pf; }

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
    const float* gammaf;  // its FP32 copy
};

// ---------------------------------------------------------------------------
// index helpers (grids hold fewer than 2^31 cells)
// ---------------------------------------------------------------------------
struct IJK {
    int i, j, k;
};

__host__ __device__ __forceinline__ IJK decode(const Geom& g, long c) {
    IJK q;
    const unsigned cc = (unsigned)c;
    const unsigned r = g.fd0.div(cc);
    q.i = (int)(cc - r * (unsigned)g.n[0]);
    const unsigned k = g.fd1.div(r);
    q.j = (int)(r - k * (unsigned)g.n[1]);
    q.k = (int)k;
    return q;
}
__host__ __device__ __forceinline__ long encode(const Geom& g, int i, int j, int k) {
    return (long)((unsigned)i + (unsigned)g.n[0] * ((unsigned)j + (unsigned)g.n[1] * (unsigned)k));
}
__host__ __device__ __forceinline__ int coord(const IJK& q, int a) { return a == 0 ? q.i : (a == 1 ? q.j : q.k); }
__host__ __device__ __forceinline__ void setc(IJK& q, int a, int v) {
    if (a == 0) q.i = v; else if (a == 1) q.j = v; else q.k = v;
}
// shift by s along axis a; periodic axes wrap (|s| <= n), the wall axis does not
__host__ __device__ __forceinline__ IJK shift(const Geom& g, IJK q, int a, int s) {
    int v = coord(q, a) + s;
    if (a != g.W) {
        if (v < 0) v += g.n[a];
        else if (v >= g.n[a]) v -= g.n[a];
    }
    setc(q, a, v);
    return q;
}
__host__ __device__ __forceinline__ long idx(const Geom& g, const IJK& q) { return encode(g, q.i, q.j, q.k); }

template <typename T>
__host__ __device__ __forceinline__ T clampv(T x, T lo, T hi) { return x < lo ? lo : (x > hi ? hi : x); }

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

// Multigrid hierarchy.  The pressure p and its right-hand side f live on
// level 0 in the storage of the precision form (PForm below); the FP64 form
// also keeps FP64 level-0 face coefficients beta for its residual.  Every
// level holds an FP32 correction e, right-hand side r and coefficients bf for
// the V-cycle.
struct MGLevel {
    Geom g;
    double* p;         // level 0 only (8 bytes per cell, typed by PForm)
    double* f;         // level 0 only (8 bytes per cell, typed by PForm)
    double* beta[3];   // level 0 only, FP64 form
    float* rho0;       // level 0 only: FP32 cell densities (the level-0 smoother's coefficients)
    float* e2;         // level 0 only: the second correction buffer of the one-pass 3D sweep
    float* e;
    float* r;
    float* bf[3];
};

struct MG {
    int nlev;
    MGLevel lv[kMaxLevels];
    double* partials;   // [2 * kPartials]
    double* scal;       // device scalars
    float* scalf;       // FP32 device scalars
    float* ainv;        // launch-per-kernel path: FP32 inverse of the coarsest level [n^2] and its shift
    // launch-per-kernel path: levels tail_lt .. nlev-1 of a V-cycle run as one
    // single-CTA launch in shared memory (tail_args: its descriptor in device
    // memory, an InstArgs<float>; null: every level as separate kernels)
    const void* tail_args;
    int tail_lt;
    size_t tail_smem;
    // launch-per-kernel path, 3D level 0: 0 one-pass sweeps where the grid
    // fills the GPU, 1 one-pass sweeps wherever the tile shape fits, 2 colour
    // passes, 3 one-pass sweeps staged by cp.async only
    int sweep_mode;
    // relaxation of the finest level's red-black sweeps on the launch-per-kernel
    // path: e <- e + omega (e_GS - e); 1 is Gauss-Seidel
    float omega;
    // launch-per-kernel path: sweeps before / after the coarse-grid correction
    // on the levels below the finest that run as separate launches (-1: the
    // finest level's counts)
    int cpre, cpost;
    // tensor maps of the one-pass sweep's level-0 arrays (host memory; null
    // or not encoded: cp.async staging)
    const struct SweepMaps* maps;
};

// TMA tensor maps of the level-0 arrays the one-pass 3D sweep stages: cell
// densities, both correction buffers and the residual, each an (nx, ny, nz)
// FP32 array, box of 72 cells x 20 rows (18 for r) of one z plane
struct SweepMaps {
    CUtensorMap rho, e, e2, r;
    bool ok;
};

// scalar slots in MG::scal
enum { S_MEAN = 0, S_FNORM = 1, S_RNORM = 2, S_MASS = 3, S_UMAX = 4, S_GAMMA = 5,
       S_THETA = 6, S_WETTED = 7, S_BADIN = 8 /* nonzero: an uploaded value was not finite */,
       S_TMAERR = 9 /* nonzero: a bounded wait for a staged copy ran out */,
       S_CYC = 10 /* V-cycles of the device-controlled solve */,
       S_SOLVE = 11 /* how the device-controlled solve ended (SolveEnd) */, S_NSCAL = 16 };
// S_SOLVE values: the loop ran (converged or out of cycles: the host compares
// the residual), f was zero, f or the residual was not finite, a staged copy
// of the one-pass sweep timed out
enum SolveEnd { kSolveRan = 0, kSolveZeroF = 1, kSolveNanF = 2, kSolveNanR = 3, kSolveTma = 4 };
// slots in MG::scalf: the means of f and p as double-floats (FP32-mixed form) and gamma
enum { SF_FMEAN_HI = 0, SF_FMEAN_LO = 1, SF_GAMMA = 2, SF_PMEAN_HI = 4, SF_PMEAN_LO = 5, SF_NSCAL = 8 };

// ---------------------------------------------------------------------------
// Level-0 pressure p and right-hand side f of the two precision forms.
// FP64 form: p and f FP64, f stored with its mean removed, residual with the
// FP64 face coefficients.  FP32-mixed form: p is a double-float (hi, lo)
// pair, about 48 significant bits; f is the FP32 divergence as computed, its
// mean kept apart as a double-float and removed inside the residual, which
// uses the FP32 face coefficients of the V-cycles in double-float arithmetic
// and so issues no FP64 instruction.
// ---------------------------------------------------------------------------
template <typename T> struct PForm;
template <> struct PForm<double> { using P = double; using F = double; };
template <> struct PForm<float> { using P = float2; using F = float; };
template <typename T> using PT = typename PForm<T>::P;
template <typename T> using FT = typename PForm<T>::F;

template <typename T>
void launch_div(const Geom& g, const T* const* us, double inv_cdt, MG& mg, cudaStream_t s);
template <typename T>
void launch_sum_f(const Geom& g, MG& mg, cudaStream_t s);
template <typename T>
void launch_sub_mean_and_norm(const Geom& g, MG& mg, cudaStream_t s);
template <typename T>
void launch_mg_coef(const Geom& g, const PhysDev& ph, const T* phi, MG& mg, cudaStream_t s);
template <typename T>
void launch_resid_norm(const Geom& g, MG& mg, cudaStream_t s);   // residual, its norm, r0 and e0 = 0
template <typename T>
void launch_vcycle(const Geom& g, MG& mg, int npre, int npost, cudaStream_t s);  // FP32 V-cycle, p += e0
template <typename T>
void launch_p_mean_remove(const Geom& g, MG& mg, cudaStream_t s);
// p = 2 hnew - hold (extrapolated first guess; history arrays in the form's p storage)
template <typename T>
void launch_p_extrap(const Geom& g, MG& mg, const double* hnew, const double* hold, cudaStream_t s);
// level-0 smoothing modes: plain; the first sweep of a V-cycle, whose old
// correction is zero (not read); the last, which also adds the correction to p
enum SweepMode { kSweepPlain = 0, kSweepFromZero = 1, kSweepUpdate = 2 };
// one-pass red-black sweep of the 3D level 0 (k_sweep.cu): ein -> eout in one
// launch (ein unused from zero; the update mode adds the new e to p instead
// of writing eout)
bool sweep0_supported(const Geom& g);  // the tile shape fits the grid
bool sweep0_auto(const Geom& g);       // it fits and the grid fills the GPU
cudaError_t sweep0_prepare();
void sweep0_encode_maps(const MGLevel& L0, SweepMaps* maps);  // maps->ok false if TMA is unavailable
template <typename T>
void launch_sweep0(const MGLevel& L0, const SweepMaps* maps, const float* ein, float* eout, int mode, float omega,
                   PT<T>* p, double* err, cudaStream_t s);
// tiled 3D momentum right-hand side (k_mom.cu): nx a multiple of 32, ny of 8;
// mom_tile_prepare sets its shared-memory size (once per process and device)
bool mom_tile_supported(const Geom& g);
cudaError_t mom_tile_prepare();
template <typename T>
void launch_mom_tile(const Geom& g, const PhysDev& ph, const StageFields<T>& f, cudaStream_t s);
// tiled level-0 residual of the FP32-mixed form on 3D grids (k_resid.cu): r
// and one |r|^2 partial a CTA (at most max_parts); returns the partial count
bool resid_tile_supported(const Geom& g, int max_parts);
cudaError_t resid_tile_prepare();
unsigned launch_resid_tile(const MGLevel& L0, const float* fmean_df, double* part, int max_parts, cudaStream_t s);
// the single-CTA shared-memory tail of a V-cycle as its own launch (k_persist.cu)
cudaError_t tail_prepare(int dim, size_t smem);
cudaError_t launch_tail(const void* inst_args, int dim, size_t smem, cudaStream_t s);
// host <-> level-0 p / f conversions of the FP32-mixed form (FP64 staging buffer x)
void launch_p_to_double(const Geom& g, const MG& mg, double* x, cudaStream_t s);
void launch_p_from_double(const Geom& g, MG& mg, const double* x, cudaStream_t s);
void launch_f_to_double(const Geom& g, const MG& mg, double* x, cudaStream_t s);
void launch_f_from_double(const Geom& g, MG& mg, const double* x, cudaStream_t s);
template <typename T>
void launch_project(const Geom& g, const PhysDev& ph, const T* phi, T* const* us, double cdt,
                    const double* p, cudaStream_t s);
template <typename T>
void launch_mass(const Geom& g, const T* phi, MG& mg, cudaStream_t s);
template <typename T>
void launch_gamma(const Geom& g, const T* const* u, double gamma_param, MG& mg, cudaStream_t s);
void launch_contact_line(const Geom& g, int wall, const double* cols, MG& mg, cudaStream_t s);

// ---------------------------------------------------------------------------
// persistent step kernel (k_persist.cu)
// ---------------------------------------------------------------------------
constexpr int kPersistThreads = 512;

// per-instance outcome of one launch (zeroed before every launch)
struct InstStats {
    int status;        // CDI_OK or the cdi_status that ended the instance's steps
    int max_cycles;    // largest V-cycle count of one solve in this launch
    int last_cycles;
    int total_cycles;  // V-cycles of all solves in this launch
    int steps_done;
    int pad;
    double last_resid;
};

// control block of the single-grid persistent kernel in the workspace
struct PersistCtl {
    // grid-barrier arrivals since the launch (zeroed by the host before it);
    // bit kBarError set (atomic OR) when a CTA gives up waiting
    unsigned long long bar;
    InstStats st;
};
constexpr unsigned long long kBarError = 1ull << 62;

// offsets (in floats) of the FP32 multigrid tail levels in dynamic shared
// memory, and of the FP64 scratch of the coarsest dense solve (in doubles,
// from the 8-byte aligned end of the float part)
struct PersistLayout {
    long sm_e[kMaxLevels], sm_r[kMaxLevels], sm_b[kMaxLevels][3];
    long sm_dbl;   // float offset where the double scratch starts
    long sm_A, sm_bb, sm_fct;
};

// everything one instance's steps need (copied by value into the kernel
// parameters, or into shared memory by the batched kernel)
template <typename T>
struct __align__(16) InstArgs : PersistLayout {
    Geom g;
    PhysDev ph;
    T *phi_s, *phi_k, *acc_phi, *rphi, *psi, *muc, *wuY, *wghost, *wmuw;
    T *u_s[3], *u_k[3], *acc_m[3], *rm[3], *nh[3], *m[3];
    MGLevel lv[kMaxLevels];
    int nlev, lt;        // levels lt.. are solved by one CTA in shared memory
    double tol;
    int max_vcycles, warm, npre, npost;
    double gamma_param, dt;
    // first guess by extrapolation in time (CDI_WARM_EXTRAP): the pressure of
    // RK stage k of the last two steps, hist[k][s & 1] written at step s
    double* hist[4][2];
    long hist_step0;   // steps stored before this launch
    const float* ainv; // coarsest-level inverse in global memory (launch-per-kernel tail), or null:
                       // the tail inverts in shared memory at the first V-cycle of each solve
    void* colq;        // extrapolated wall-column quantities, [2 NP] (ops::ColQ<T>)
    int tail_bf_stored;  // nonzero: the tail's top level's coefficients are in lv[lt].bf already
};

template <typename T>
struct PersistArgs {
    InstArgs<T> I;
    PersistCtl* ctl;
    double* partials;    // 2 * kPartials doubles
    int nsteps;
    long spin_limit;     // barrier timeout in nanoseconds
};

template <typename T>
struct BatchArgs {
    const InstArgs<T>* insts;  // sorted by decreasing cell count
    InstStats* stats;
    int* counter;              // next instance to take (zeroed before the launch)
    int n_inst;
    int nsteps;
};

size_t persist_tail_layout(const Geom& g, const MG& mg, int lt, PersistLayout& L);
template <typename T>
cudaError_t persist_prepare(int dim, size_t smem, int* grid);
template <typename T>
cudaError_t launch_step_persist(PersistArgs<T>& A, size_t smem, int grid, cudaStream_t s);
template <typename T>
cudaError_t batch_prepare(int dim, int threads, size_t smem, int* grid);
template <typename T>
cudaError_t launch_batch_persist(BatchArgs<T>& B, int dim, int threads, size_t smem, int grid, cudaStream_t s);

// number of kernel launches issued since the counter was reset (host side)
extern thread_local long g_launches;

// Kernel classes that the launch profiler can bracket with CUDA events.
enum KClass { KC_PSI = 0, KC_CELL, KC_WALL, KC_PHI_RHS, KC_MOM, KC_STAGE_PHI, KC_STAGE_MOM, KC_DIV,
              KC_RBGS0, KC_RBGS, KC_RESTRICT0, KC_PROLONG0, KC_COARSE, KC_RESID, KC_PROJECT, KC_STEP, KC_COUNT };
extern const char* const kKernelClassNames[KC_COUNT];

// Launch profiler: records an event pair around each launch of one kernel
// class on the launching stream, up to a fixed number of launches.
struct Profiler {
    int target = -1;
    int cap = 0;
    int used = 0;
    cudaEvent_t* ev = nullptr;  // 2 * cap events
};
extern thread_local Profiler g_prof;

inline bool prof_before(int kc, cudaStream_t s) {
    if (g_prof.target != kc || g_prof.used >= g_prof.cap) return false;
    cudaEventRecord(g_prof.ev[2 * g_prof.used], s);
    return true;
}
inline void prof_after(bool on, cudaStream_t s) {
    if (!on) return;
    cudaEventRecord(g_prof.ev[2 * g_prof.used + 1], s);
    ++g_prof.used;
}
#define CDI_PROF(kc, s, launch)              \
    do {                                     \
        const bool _on = prof_before(kc, s); \
        launch;                              \
        prof_after(_on, s);                  \
    } while (0)

}  // namespace cdi
