// C ABI of libcdi.so (declared in include/cdi.h): argument checking, the
// workspace layout, and the host-side driver of one RK4 time step.
//
// One step (Sec. 4: classical RK4; every stage value and the final value are
// projected, so four pressure solves per step):
//   for stage k = 1..4:
//       right-hand side on the stage state        (k_psi, k_cell, k_wall, k_phi_rhs, k_mom)
//       stage update of phi and rho_f u, u* = M/rho_f   (k_stage_phi, k_stage_mom)
//       projection: f = div u*/(c dt), multigrid, u = u* - c dt grad p/rho_f
// The new state lands in the stage buffers, whose role is then swapped with
// the state buffers.
#include "cdi_internal.cuh"
#include "unet.cuh"
#include "../../include/cdi.h"

#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>
#include <algorithm>

using namespace cdi;

struct cdi_ctx {
    Geom g{};
    double L[3] = {0, 0, 0};
    int precision = CDI_FP64;
    // physics
    PhysDev ph{};
    double gamma = 0.0;
    double wall_slip_length[2] = {-1.0, -1.0};
    bool fluids_set = false;
    // solver
    double tol = 1e-10;
    int max_vcycles = 100;
    int warm = CDI_WARM_PREV;
    cdi_unet* unet = nullptr;  // learned first guess (CDI_WARM_UNET)
    double* hist[4][2] = {{nullptr, nullptr}, {nullptr, nullptr}, {nullptr, nullptr}, {nullptr, nullptr}};
    long hist_steps = 0;  // steps whose stage pressures are in hist
    int npre = 2, npost = 2;
    // workspace
    char* ws = nullptr;
    size_t ws_bytes = 0;
    cudaStream_t stream = nullptr;
    bool bound = false;
    // fields (element type double or float, see precision)
    void* phi_s = nullptr;
    void* u_s[3] = {nullptr, nullptr, nullptr};
    void* phi_k = nullptr;
    void* u_k[3] = {nullptr, nullptr, nullptr};
    void* acc_phi = nullptr;
    void* acc_m[3] = {nullptr, nullptr, nullptr};
    void* rphi = nullptr;
    void* rm[3] = {nullptr, nullptr, nullptr};
    void* psi = nullptr;
    void* nh[3] = {nullptr, nullptr, nullptr};
    void* muc = nullptr;
    void* m[3] = {nullptr, nullptr, nullptr};
    void* wuY = nullptr;
    void* wghost = nullptr;
    void* wmuw = nullptr;
    void* colq = nullptr;  // persistent mode: extrapolated wall-column quantities (9 values a column)
    double* cols = nullptr;
    double* xfer = nullptr;  // FP64 staging of one face field for host copies
    MG mg{};
    double* host_scal = nullptr;
    // execution of cdi_step: one persistent cooperative launch, or one launch per kernel
    int exec = CDI_EXEC_AUTO;
    PersistCtl* ctl = nullptr;
    bool persist_ready = false;
    void* tail_dev = nullptr;  // launch-per-kernel path: descriptor of the V-cycle's shared-memory tail
    bool tail_ready = false;
    SweepMaps smaps{};         // tensor maps of the one-pass sweep (encoded with the tail)
    // launch-per-kernel path: one V-cycle plus its residual norm as a CUDA graph per form
    cudaStream_t cap_stream = nullptr;
    cudaGraphExec_t vc_exec[2] = {nullptr, nullptr};
    long vc_nodes[2] = {0, 0};
    bool vc_graph_failed = false;
    // launch-per-kernel path: a whole pressure solve (first residual, the
    // V-cycles in a conditional while node, the zero right-hand side guard) as
    // one CUDA graph per form; tolerance and cycle limit are baked into its
    // kernels
    cudaGraphExec_t solve_exec[2] = {nullptr, nullptr};
    long solve_nodes[2][3] = {{0, 0, 0}, {0, 0, 0}};  // before, per V-cycle, after the loop
    double solve_tol[2] = {0.0, 0.0};
    int solve_max[2] = {0, 0};
    bool solve_graph_failed = false;
    // launch-per-kernel path: the level-0 pressure still carries the constant
    // its V-cycles added (removed when p is read out)
    bool p_mean_pending = false;
    PersistLayout playout{};
    int persist_lt = 0;
    size_t persist_smem = 0;
    int persist_grid = 0;
    long spin_limit_ns = 2000000000L;
    // statistics
    int last_cycles = 0;
    double last_resid = 0.0;
    int max_cycles_step = 0;
    int total_cycles_call = 0;
    long launches_per_step = 0;
    std::string err;
};

namespace {

std::string g_init_error;

cdi_status fail(cdi_ctx* c, cdi_status st, const std::string& msg) {
    if (c) c->err = msg;
    else g_init_error = msg;
    return st;
}

cdi_status cuda_check(cdi_ctx* c, cudaError_t e, const char* what) {
    if (e == cudaSuccess) return CDI_OK;
    return fail(c, CDI_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

// The cached CUDA graphs hold kernel arguments (sweep counts, relaxation,
// sweep form, tolerance, buffers): dropped whenever one of them changes.
void drop_graphs(cdi_ctx* c) {
    for (int k = 0; k < 2; ++k) {
        if (c->vc_exec[k]) {
            cudaGraphExecDestroy(c->vc_exec[k]);
            c->vc_exec[k] = nullptr;
        }
        if (c->solve_exec[k]) {
            cudaGraphExecDestroy(c->solve_exec[k]);
            c->solve_exec[k] = nullptr;
        }
    }
}

size_t esize(const cdi_ctx* c) { return c->precision == CDI_FP64 ? sizeof(double) : sizeof(float); }

long nface(const Geom& g, int a) { return g.N + (a == g.W ? g.NP : 0); }

// Fixed-order carving of the workspace; the same walk computes the size.
struct Carver {
    char* base;
    size_t off = 0;
    void* take(size_t bytes) {
        off = (off + 255) & ~size_t(255);
        void* p = base ? base + off : nullptr;
        off += bytes;
        return p;
    }
};

void carve(cdi_ctx* c, char* base, size_t* total) {
    Carver cv{base};
    const Geom& g = c->g;
    const size_t es = esize(c);
    auto cell = [&]() { return cv.take(g.N * es); };
    auto face = [&](int a) { return cv.take(nface(g, a) * es); };
    c->phi_s = cell();
    c->phi_k = cell();
    c->acc_phi = cell();
    c->rphi = cell();
    c->psi = cell();
    c->muc = cell();
    for (int a = 0; a < 3; ++a) {
        bool on = a < g.D;
        c->u_s[a] = on ? face(a) : nullptr;
        c->u_k[a] = on ? face(a) : nullptr;
        c->acc_m[a] = on ? face(a) : nullptr;
        c->rm[a] = on ? face(a) : nullptr;
        c->m[a] = on ? face(a) : nullptr;
        c->nh[a] = on ? cell() : nullptr;
    }
    const size_t nw = (size_t)2 * (g.D - 1) * g.NP;
    c->wuY = cv.take(nw * es);
    c->wghost = cv.take(nw * es);
    c->wmuw = cv.take(nw * es);
    c->colq = cv.take((size_t)2 * g.NP * 9 * es);
    c->cols = (double*)cv.take((size_t)2 * 3 * g.NP * sizeof(double));
    c->xfer = (double*)cv.take((size_t)(g.N + g.NP) * sizeof(double));
    MG& mg = c->mg;
    for (int l = 0; l < mg.nlev; ++l) {
        MGLevel& L = mg.lv[l];
        const long nl = L.g.N, np = L.g.NP;
        if (l == 0) {  // pressure, right-hand side (8 bytes a cell in both forms) and FP64 coefficients
            L.p = (double*)cv.take(nl * sizeof(double));
            L.f = (double*)cv.take(nl * sizeof(double));
            const bool f64 = c->precision == CDI_FP64;
            for (int a = 0; a < 3; ++a)
                L.beta[a] = (f64 && a < g.D) ? (double*)cv.take((nl + (a == g.W ? np : 0)) * sizeof(double))
                                             : nullptr;
            L.rho0 = (float*)cv.take(nl * sizeof(float));
            L.e2 = sweep0_supported(g) ? (float*)cv.take(nl * sizeof(float)) : nullptr;
        } else {
            L.p = nullptr;
            L.f = nullptr;
            L.rho0 = nullptr;
            L.e2 = nullptr;
            for (int a = 0; a < 3; ++a) L.beta[a] = nullptr;
        }
        L.e = (float*)cv.take(nl * sizeof(float));
        L.r = (float*)cv.take(nl * sizeof(float));
        for (int a = 0; a < 3; ++a)
            L.bf[a] = (a < g.D) ? (float*)cv.take((nl + (a == g.W ? np : 0)) * sizeof(float)) : nullptr;
    }
    mg.partials = (double*)cv.take(2 * kPartials * sizeof(double));
    mg.scal = (double*)cv.take(S_NSCAL * sizeof(double));
    mg.scalf = (float*)cv.take(SF_NSCAL * sizeof(float));
    mg.ainv = (float*)cv.take(((size_t)kMaxCoarse * kMaxCoarse + 1) * sizeof(float));  // inverse, then the shift
    c->ctl = (PersistCtl*)cv.take(sizeof(PersistCtl));
    c->tail_dev = cv.take(sizeof(InstArgs<float>));
    for (int k = 0; k < 4; ++k)
        for (int j = 0; j < 2; ++j) c->hist[k][j] = (double*)cv.take((size_t)g.N * sizeof(double));
    *total = cv.off + 256;
}

template <typename T>
__global__ void k_to_double(long n, const T* __restrict__ src, double* __restrict__ dst) {
    long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) dst[i] = (double)src[i];
}
// dst = src in the field's type; *bad = 1 where a value is not finite (every
// writer stores the same value)
template <typename T>
__global__ void k_from_double(long n, const double* __restrict__ src, T* __restrict__ dst, double* bad) {
    long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) {
        const double v = src[i];
        if (!isfinite(v)) *bad = 1.0;
        dst[i] = (T)v;
    }
}
__global__ void k_check_finite(long n, const double* __restrict__ x, double* bad) {
    long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n && !isfinite(x[i])) *bad = 1.0;
}
__global__ void k_set_gamma(double* p, float* pf, double v) {
    *p = v;
    *pf = (float)v;
}
template <typename T>
__global__ void k_zero_wall_planes(long N, long NP, T* __restrict__ w) {
    long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < NP) {
        w[i] = T(0);
        w[N + i] = T(0);
    }
}

unsigned nblk(long n) { return (unsigned)((n + 255) / 256); }

// copy a host double array into a device field of the context's precision;
// a value that is not finite (found on the device while converting or by a
// check of the copy) returns CDI_ENAN, leaving the field undefined
// Device address of a host buffer that kernels may read and write directly
// (page-locked and mapped into the device's address space, e.g. from
// cudaHostAlloc or a pinned torch tensor), or null for pageable memory, which
// is copied through the staging buffer instead.
const void* host_alias(const void* p) {
    cudaPointerAttributes a{};
    if (!p || cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return a.type == cudaMemoryTypeHost ? a.devicePointer : nullptr;
}

cdi_status upload(cdi_ctx* c, void* dst, const double* src, long n, const char* what) {
    double* bad = c->mg.scal + S_BADIN;
    cdi_status st = cuda_check(c, cudaMemsetAsync(bad, 0, sizeof(double), c->stream), "cudaMemsetAsync");
    if (st) return st;
    // mapped host memory: one pass that reads the host array over the link,
    // checks it and stores it in the field's type
    const double* hs = static_cast<const double*>(host_alias(src));
    if (hs) {
        if (c->precision == CDI_FP64) k_from_double<double><<<nblk(n), 256, 0, c->stream>>>(n, hs, (double*)dst, bad);
        else k_from_double<float><<<nblk(n), 256, 0, c->stream>>>(n, hs, (float*)dst, bad);
    } else if (c->precision == CDI_FP64) {
        st = cuda_check(c, cudaMemcpyAsync(dst, src, n * sizeof(double), cudaMemcpyHostToDevice, c->stream),
                        "cudaMemcpyAsync(H2D)");
        if (st) return st;
        k_check_finite<<<nblk(n), 256, 0, c->stream>>>(n, (const double*)dst, bad);
    } else {
        st = cuda_check(c, cudaMemcpyAsync(c->xfer, src, n * sizeof(double), cudaMemcpyHostToDevice, c->stream),
                        "cudaMemcpyAsync(H2D)");
        if (st) return st;
        k_from_double<float><<<nblk(n), 256, 0, c->stream>>>(n, c->xfer, (float*)dst, bad);
    }
    st = cuda_check(c, cudaMemcpyAsync(c->host_scal + S_BADIN, bad, sizeof(double), cudaMemcpyDeviceToHost,
                                       c->stream), "cudaMemcpyAsync(D2H)");
    if (st) return st;
    st = cuda_check(c, cudaStreamSynchronize(c->stream), "upload");
    if (st) return st;
    if (c->host_scal[S_BADIN] != 0.0) return fail(c, CDI_ENAN, std::string(what) + " holds a non-finite value");
    return CDI_OK;
}

cdi_status download(cdi_ctx* c, double* dst, const void* src, long n) {
    if (!dst) return CDI_OK;
    double* hd = static_cast<double*>(const_cast<void*>(host_alias(dst)));
    if (hd && c->precision != CDI_FP64) {  // mapped host memory: convert straight into it
        k_to_double<float><<<nblk(n), 256, 0, c->stream>>>(n, (const float*)src, hd);
    } else if (c->precision == CDI_FP64) {
        cdi_status st = cuda_check(c, cudaMemcpyAsync(dst, src, n * sizeof(double), cudaMemcpyDeviceToHost, c->stream),
                                   "cudaMemcpyAsync(D2H)");
        if (st) return st;
    } else {
        k_to_double<float><<<nblk(n), 256, 0, c->stream>>>(n, (const float*)src, c->xfer);
        cdi_status st = cuda_check(c, cudaMemcpyAsync(dst, c->xfer, n * sizeof(double), cudaMemcpyDeviceToHost,
                                                      c->stream), "cudaMemcpyAsync(D2H)");
        if (st) return st;
    }
    return cuda_check(c, cudaStreamSynchronize(c->stream), "download");
}

// level-0 pressure, or right-hand side with its mean removed, to host FP64
// (the FP32-mixed form converts through the staging buffer)
cdi_status download_level0(cdi_ctx* c, double* dst, bool pressure) {
    const Geom& g = c->g;
    if (pressure && c->p_mean_pending) {
        if (c->precision == CDI_FP64) launch_p_mean_remove<double>(g, c->mg, c->stream);
        else launch_p_mean_remove<float>(g, c->mg, c->stream);
        c->p_mean_pending = false;
    }
    const double* src = pressure ? c->mg.lv[0].p : c->mg.lv[0].f;
    double* hd = static_cast<double*>(const_cast<void*>(host_alias(dst)));
    if (c->precision != CDI_FP64) {
        double* to = hd ? hd : c->xfer;  // mapped host memory: convert straight into it
        if (pressure) launch_p_to_double(g, c->mg, to, c->stream);
        else launch_f_to_double(g, c->mg, to, c->stream);
        src = c->xfer;
    }
    if (!hd || c->precision == CDI_FP64) {
        cdi_status st = cuda_check(
            c, cudaMemcpyAsync(dst, src, g.N * sizeof(double), cudaMemcpyDeviceToHost, c->stream), "cudaMemcpyAsync(D2H)");
        if (st) return st;
    }
    return cuda_check(c, cudaStreamSynchronize(c->stream), "download");
}

// host FP64 pressure or right-hand side into level 0
cdi_status upload_level0(cdi_ctx* c, const double* src, bool pressure) {
    const Geom& g = c->g;
    double* dst = c->precision == CDI_FP64 ? (pressure ? c->mg.lv[0].p : c->mg.lv[0].f) : c->xfer;
    cdi_status st = cuda_check(c, cudaMemcpyAsync(dst, src, g.N * sizeof(double), cudaMemcpyHostToDevice, c->stream),
                               "cudaMemcpyAsync(H2D)");
    if (st) return st;
    if (c->precision != CDI_FP64) {
        if (pressure) launch_p_from_double(g, c->mg, c->xfer, c->stream);
        else launch_f_from_double(g, c->mg, c->xfer, c->stream);
    }
    return cuda_check(c, cudaStreamSynchronize(c->stream), "upload");
}

cdi_status read_scalars(cdi_ctx* c) {
    cdi_status st = cuda_check(c, cudaMemcpyAsync(c->host_scal, c->mg.scal, S_NSCAL * sizeof(double),
                                                  cudaMemcpyDeviceToHost, c->stream), "cudaMemcpyAsync(scalars)");
    if (st) return st;
    return cuda_check(c, cudaStreamSynchronize(c->stream), "cudaStreamSynchronize");
}

cdi_status need_bound(cdi_ctx* c) {
    if (!c) return fail(nullptr, CDI_EINVAL, "null context");
    if (!c->bound) return fail(c, CDI_ESTATE, "no workspace bound");
    return CDI_OK;
}

// Multigrid solve of div(beta grad p) = f on level 0 (f already mean-free,
// its norm in S_FNORM, coefficients set); p holds the first guess.
size_t pick_tail(const cdi_ctx* c, size_t budget, int* lt_out, PersistLayout* L, long max_cells = 1L << 40);
// launch-per-kernel path: the largest level the single-CTA tail takes.  One CTA
// sweeping 8192 cells (32 x 16 x 16 on the 512x256x256 grid) took 77 us a
// V-cycle; such a level runs faster as grid-wide launches.
constexpr long kTailMaxCells = 2048;
cdi_status smem_optin(cdi_ctx* c, size_t* bytes);

// Launch-per-kernel path: the coarse levels of every V-cycle that fit in one
// CTA's shared memory run as a single launch (k_tail) instead of one launch
// per sweep; set up once per bound workspace.
cdi_status kernels_tail_setup(cdi_ctx* c) {
    if (c->tail_ready) return CDI_OK;
    size_t optin = 0;
    cdi_status st = smem_optin(c, &optin);
    if (st) return st;
    c->mg.maps = nullptr;
    st = cuda_check(c, resid_tile_prepare(), "tiled residual setup");
    if (st) return st;
    if (c->mg.lv[0].e2) {
        st = cuda_check(c, sweep0_prepare(), "one-pass sweep setup");
        if (st) return st;
        sweep0_encode_maps(c->mg.lv[0], &c->smaps);
        if (c->smaps.ok) c->mg.maps = &c->smaps;
    }
    const size_t budget = optin > 8192 ? optin - 4096 : 0;
    int lt = 0;
    PersistLayout lay{};
    const size_t sm = pick_tail(c, budget, &lt, &lay, kTailMaxCells);
    c->mg.tail_args = nullptr;
    if (sm <= budget) {
        InstArgs<float> A{};
        static_cast<PersistLayout&>(A) = lay;
        A.g = c->g;
        for (int l = 0; l < kMaxLevels; ++l) A.lv[l] = c->mg.lv[l];
        A.nlev = c->mg.nlev;
        A.lt = lt;
        A.npre = c->npre;
        A.npost = c->npost;
        A.ainv = c->mg.ainv;
        A.tail_bf_stored = 1;  // launch_mg_coef restricts the coefficients of every level once per solve
        st = cuda_check(c, cudaMemcpyAsync(c->tail_dev, &A, sizeof A, cudaMemcpyHostToDevice, c->stream),
                        "cudaMemcpyAsync(tail)");
        if (st) return st;
        st = cuda_check(c, cudaStreamSynchronize(c->stream), "tail setup");
        if (st) return st;
        st = cuda_check(c, tail_prepare(c->g.D, sm), "tail kernel setup");
        if (st) return st;
        c->mg.tail_args = c->tail_dev;
        c->mg.tail_lt = lt;
        c->mg.tail_smem = sm;
    }
    c->tail_ready = true;
    return CDI_OK;
}

// One V-cycle and the residual norm after it.  Outside the event profiler the
// sequence (about 50 launches, most of them on small coarse levels) is
// captured once into a CUDA graph on a private stream and replayed on the
// context's stream, which removes the per-launch latency.
template <typename T>
void vcycle_and_residual(cdi_ctx* c) {
    const Geom& g = c->g;
    MG& mg = c->mg;
    const int k = sizeof(T) == 8 ? 0 : 1;
    if (g_prof.target < 0 && !c->vc_graph_failed) {
        if (!c->vc_exec[k]) {
            bool ok = c->cap_stream || cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking) == cudaSuccess;
            cudaGraph_t gr = nullptr;
            const long l0 = g_launches;
            if (ok) ok = cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
            if (ok) {
                launch_vcycle<T>(g, mg, c->npre, c->npost, c->cap_stream);
                launch_resid_norm<T>(g, mg, c->cap_stream);
                ok = cudaStreamEndCapture(c->cap_stream, &gr) == cudaSuccess && gr;
            }
            c->vc_nodes[k] = g_launches - l0;
            g_launches = l0;
            if (ok) ok = cudaGraphInstantiate(&c->vc_exec[k], gr, 0) == cudaSuccess;
            if (gr) cudaGraphDestroy(gr);
            if (!ok) {
                cudaGetLastError();
                c->vc_exec[k] = nullptr;
                c->vc_graph_failed = true;
            }
        }
        if (c->vc_exec[k] && cudaGraphLaunch(c->vc_exec[k], c->stream) == cudaSuccess) {
            g_launches += c->vc_nodes[k];
            return;
        }
        cudaGetLastError();
        c->vc_graph_failed = true;
    }
    launch_vcycle<T>(g, mg, c->npre, c->npost, c->stream);
    launch_resid_norm<T>(g, mg, c->stream);
}

// Device-side control of the V-cycle loop: the tests of the host loop in
// mg_solve (f finite and nonzero, residual above tol |f|, staged-copy
// timeout, finite residual, cycle limit), in the same order and the same FP64
// arithmetic, set the condition of the solve graph's while node.
__global__ void k_solve_begin(double* scal, cudaGraphConditionalHandle h, double tol, int max_cycles) {
    const double fn = scal[S_FNORM], rn = scal[S_RNORM];
    unsigned go = 0;
    double end = kSolveRan;
    if (!isfinite(fn) || !isfinite(rn)) end = kSolveNanF;
    else if (fn == 0.0) end = kSolveZeroF;
    else go = (rn > tol * fn && 0 < max_cycles) ? 1u : 0u;
    scal[S_CYC] = 0.0;
    scal[S_SOLVE] = end;
    cudaGraphSetConditional(h, go);
}

__global__ void k_solve_next(double* scal, cudaGraphConditionalHandle h, double tol, int max_cycles) {
    const double fn = scal[S_FNORM], rn = scal[S_RNORM];
    const double cyc = scal[S_CYC] + 1.0;
    unsigned go = 0;
    if (scal[S_TMAERR] != 0.0) scal[S_SOLVE] = kSolveTma;
    else if (!isfinite(rn)) scal[S_SOLVE] = kSolveNanR;
    else go = (rn > tol * fn && cyc < (double)max_cycles) ? 1u : 0u;
    scal[S_CYC] = cyc;
    cudaGraphSetConditional(h, go);
}

// a zero right-hand side has the constant solutions: p = 0 (both forms keep 8
// bytes a cell, and all-zero bytes are zero in both)
__global__ void k_zero_p_if_zero_f(long n, double* p, const double* scal) {
    if (scal[S_SOLVE] != (double)kSolveZeroF) return;
    for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) p[i] = 0.0;
}

// The whole pressure solve as one CUDA graph: the first guess's residual norm
// and the loop's first test, a conditional while node whose body is one
// V-cycle, the residual norm after it and the next test, then p = 0 for a zero
// f.  The host waits once per solve instead of once per V-cycle.  Returns
// false when the graph could not be built (the caller then drives the loop
// from the host).
template <typename T>
bool build_solve_graph(cdi_ctx* c, int k) {
    const Geom& g = c->g;
    MG& mg = c->mg;
    if (!c->cap_stream && cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking) != cudaSuccess) return false;
    cudaStream_t cs = c->cap_stream;
    const long l0 = g_launches;
    long n_before = 0, n_body = 0, n_after = 0;
    cudaGraph_t G = nullptr, body = nullptr;
    cudaGraphConditionalHandle h = 0;
    bool ok = cudaGraphCreate(&G, 0) == cudaSuccess;
    ok = ok && cudaGraphConditionalHandleCreate(&h, G, 0, cudaGraphCondAssignDefault) == cudaSuccess;
    if (ok) ok = cudaStreamBeginCaptureToGraph(cs, G, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
    if (ok) {
        launch_resid_norm<T>(g, mg, cs);
        k_solve_begin<<<1, 1, 0, cs>>>(mg.scal, h, c->tol, c->max_vcycles);
        ++g_launches;
        n_before = g_launches - l0;
        cudaStreamCaptureStatus cst = cudaStreamCaptureStatusNone;
        cudaGraph_t cg = nullptr;
        const cudaGraphNode_t* deps = nullptr;
        size_t nd = 0;
        bool node_ok = cudaStreamGetCaptureInfo(cs, &cst, nullptr, &cg, &deps, nullptr, &nd) == cudaSuccess &&
                       cst == cudaStreamCaptureStatusActive;
        cudaGraphNodeParams np{};
        np.type = cudaGraphNodeTypeConditional;
        np.conditional.handle = h;
        np.conditional.type = cudaGraphCondTypeWhile;
        np.conditional.size = 1;
        cudaGraphNode_t wn = nullptr;
        node_ok = node_ok && cudaGraphAddNode(&wn, cg, deps, nullptr, nd, &np) == cudaSuccess;
        node_ok = node_ok && cudaStreamUpdateCaptureDependencies(cs, &wn, nullptr, 1,
                                                                 cudaStreamSetCaptureDependencies) == cudaSuccess;
        if (node_ok) body = np.conditional.phGraph_out[0];
        const long l1 = g_launches;
        k_zero_p_if_zero_f<<<2 * 152, 256, 0, cs>>>(g.N, mg.lv[0].p, mg.scal);
        ++g_launches;
        n_after = g_launches - l1;
        cudaGraph_t out = nullptr;
        ok = cudaStreamEndCapture(cs, &out) == cudaSuccess && node_ok && body;
    }
    if (ok) {
        const long l2 = g_launches;
        ok = cudaStreamBeginCaptureToGraph(cs, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal) ==
             cudaSuccess;
        if (ok) {
            launch_vcycle<T>(g, mg, c->npre, c->npost, cs);
            launch_resid_norm<T>(g, mg, cs);
            k_solve_next<<<1, 1, 0, cs>>>(mg.scal, h, c->tol, c->max_vcycles);
            ++g_launches;
            cudaGraph_t out = nullptr;
            ok = cudaStreamEndCapture(cs, &out) == cudaSuccess;
        }
        n_body = g_launches - l2;
    }
    g_launches = l0;
    cudaGraphExec_t ex = nullptr;
    if (ok) ok = cudaGraphInstantiate(&ex, G, 0) == cudaSuccess;
    if (G) cudaGraphDestroy(G);
    if (!ok) {
        cudaGetLastError();
        if (ex) cudaGraphExecDestroy(ex);
        return false;
    }
    c->solve_exec[k] = ex;
    c->solve_nodes[k][0] = n_before;
    c->solve_nodes[k][1] = n_body;
    c->solve_nodes[k][2] = n_after;
    c->solve_tol[k] = c->tol;
    c->solve_max[k] = c->max_vcycles;
    return true;
}

// Outcome of a solve-graph launch: one wait, then the statuses and statistics
// of the host loop.
cdi_status finish_solve_graph(cdi_ctx* c, int k) {
    cdi_status st = read_scalars(c);
    if (st) return st;
    const double* hs = c->host_scal;
    const double fn = hs[S_FNORM], rn = hs[S_RNORM];
    const int cyc = (int)hs[S_CYC];
    const int end = (int)hs[S_SOLVE];
    g_launches += c->solve_nodes[k][0] + (long)cyc * c->solve_nodes[k][1] + c->solve_nodes[k][2];
    if (end == kSolveNanF) return fail(c, CDI_ENAN, "non-finite pressure right-hand side");
    if (end == kSolveZeroF) {
        c->last_cycles = 0;
        c->last_resid = 0.0;
        return CDI_OK;
    }
    if (end == kSolveTma) {
        cudaMemsetAsync(c->mg.scal + S_TMAERR, 0, sizeof(double), c->stream);
        return fail(c, CDI_ETIMEOUT, "one-pass sweep: a staged copy did not complete within its bounded wait");
    }
    if (end == kSolveNanR) return fail(c, CDI_ENAN, "non-finite pressure residual");
    c->p_mean_pending = true;
    c->last_cycles = cyc;
    c->last_resid = rn / fn;
    if (cyc > c->max_cycles_step) c->max_cycles_step = cyc;
    c->total_cycles_call += cyc;
    if (rn > c->tol * fn) {
        char b[160];
        snprintf(b, sizeof b, "pressure solve: %d V-cycles left relative residual %.3e > tol %.3e", cyc, rn / fn,
                 c->tol);
        return fail(c, CDI_ENOCONV, b);
    }
    return CDI_OK;
}

template <typename T>
cdi_status mg_solve(cdi_ctx* c) {
    const Geom& g = c->g;
    cudaStream_t s = c->stream;
    MG& mg = c->mg;
    cdi_status st0 = kernels_tail_setup(c);
    if (st0) return st0;
    const int k = sizeof(T) == 8 ? 0 : 1;
    if (g_prof.target < 0 && !c->solve_graph_failed) {
        if (c->solve_exec[k] && (c->solve_tol[k] != c->tol || c->solve_max[k] != c->max_vcycles)) {
            cudaGraphExecDestroy(c->solve_exec[k]);
            c->solve_exec[k] = nullptr;
        }
        if (!c->solve_exec[k] && !build_solve_graph<T>(c, k)) c->solve_graph_failed = true;
        if (c->solve_exec[k]) {
            if (cudaGraphLaunch(c->solve_exec[k], s) == cudaSuccess) return finish_solve_graph(c, k);
            cudaGetLastError();
            c->solve_graph_failed = true;
        }
    }
    launch_resid_norm<T>(g, mg, s);
    cdi_status st = read_scalars(c);
    if (st) return st;
    const double fn = c->host_scal[S_FNORM];
    double rn = c->host_scal[S_RNORM];
    int cyc = 0;
    if (!std::isfinite(fn) || !std::isfinite(rn)) return fail(c, CDI_ENAN, "non-finite pressure right-hand side");
    if (fn == 0.0) {
        cudaMemsetAsync(mg.lv[0].p, 0, g.N * sizeof(double), s);
        c->last_cycles = 0;
        c->last_resid = 0.0;
        return CDI_OK;
    }
    while (rn > c->tol * fn && cyc < c->max_vcycles) {
        vcycle_and_residual<T>(c);
        st = read_scalars(c);
        if (st) return st;
        if (c->host_scal[S_TMAERR] != 0.0) {
            cudaMemsetAsync(mg.scal + S_TMAERR, 0, sizeof(double), s);
            return fail(c, CDI_ETIMEOUT, "one-pass sweep: a staged copy did not complete within its bounded wait");
        }
        rn = c->host_scal[S_RNORM];
        ++cyc;
        if (!std::isfinite(rn)) return fail(c, CDI_ENAN, "non-finite pressure residual");
    }
    c->last_cycles = cyc;
    c->last_resid = rn / fn;
    if (cyc > c->max_cycles_step) c->max_cycles_step = cyc;
    c->total_cycles_call += cyc;
    if (rn > c->tol * fn) {
        char b[160];
        snprintf(b, sizeof b, "pressure solve: %d V-cycles left relative residual %.3e > tol %.3e", cyc, rn / fn,
                 c->tol);
        return fail(c, CDI_ENOCONV, b);
    }
    // p is determined up to a constant (periodic axes, Neumann walls) and
    // nothing in the step reads more than its differences, so the zero-mean
    // normalisation waits until p is read out (download_level0)
    c->p_mean_pending = true;
    return CDI_OK;
}

template <typename T>
cdi_status project(cdi_ctx* c, const T* phi, T* const* u, double cdt, int stage) {
    const Geom& g = c->g;
    cudaStream_t s = c->stream;
    const T* uc[3] = {u[0], u[1], u[2]};
    launch_div<T>(g, uc, 1.0 / cdt, c->mg, s);
    launch_sub_mean_and_norm<T>(g, c->mg, s);
    launch_mg_coef<T>(g, c->ph, phi, c->mg, s);
    // first guess: zero, the last solve's pressure, the same RK stage of the
    // last two steps extrapolated linearly in time, or the network's prediction
    const bool extrap = c->warm == CDI_WARM_EXTRAP;
    const long sg = c->hist_steps;
    if (c->warm == CDI_WARM_ZERO) cudaMemsetAsync(c->mg.lv[0].p, 0, g.N * sizeof(double), s);
    if (extrap && sg >= 2) launch_p_extrap<T>(g, c->mg, c->hist[stage][(sg - 1) & 1], c->hist[stage][sg & 1], s);
    if (c->warm == CDI_WARM_UNET) {
        const cudaError_t e = unet_predict_device<T>(c->unet, c->mg, phi, c->ph.rho1, c->ph.rho2, c->g.h, s);
        if (e != cudaSuccess) return cuda_check(c, e, "network first guess");
    }
    cdi_status st = mg_solve<T>(c);
    if (st) return st;
    if (extrap) {
        st = cuda_check(c, cudaMemcpyAsync(c->hist[stage][sg & 1], c->mg.lv[0].p, g.N * sizeof(double),
                                           cudaMemcpyDeviceToDevice, s), "cudaMemcpyAsync(history)");
        if (st) return st;
    }
    launch_project<T>(g, c->ph, phi, u, cdt, c->mg.lv[0].p, s);
    return CDI_OK;
}

template <typename T>
StageFields<T> stage_fields(cdi_ctx* c, const void* phi, void* const* u) {
    StageFields<T> f{};
    f.phi = (const T*)phi;
    for (int a = 0; a < 3; ++a) {
        f.u[a] = (const T*)u[a];
        f.nh[a] = (T*)c->nh[a];
        f.m[a] = (T*)c->m[a];
        f.rm[a] = (T*)c->rm[a];
    }
    f.psi = (T*)c->psi;
    f.muc = (T*)c->muc;
    f.rphi = (T*)c->rphi;
    f.wuY = (T*)c->wuY;
    f.wghost = (T*)c->wghost;
    f.wmuw = (T*)c->wmuw;
    f.gamma = c->mg.scal + S_GAMMA;
    f.gammaf = c->mg.scalf + SF_GAMMA;
    return f;
}

template <typename T>
void set_gamma(cdi_ctx* c, const void* const* u, double gamma_arg) {
    if (gamma_arg >= 0.0) {
        k_set_gamma<<<1, 1, 0, c->stream>>>(c->mg.scal + S_GAMMA, c->mg.scalf + SF_GAMMA, gamma_arg);
        ++g_launches;
    } else {
        const T* uc[3] = {(const T*)u[0], (const T*)u[1], (const T*)u[2]};
        launch_gamma<T>(c->g, uc, gamma_arg, c->mg, c->stream);
    }
}

template <typename T>
cdi_status step_once(cdi_ctx* c, double dt) {
    const Geom& g = c->g;
    cudaStream_t s = c->stream;
    set_gamma<T>(c, c->u_s, c->gamma);
    const double ck[4] = {0.0, 0.5, 0.5, 1.0};
    for (int st = 0; st < 4; ++st) {
        const void* phi = st == 0 ? c->phi_s : c->phi_k;
        void* const* u = st == 0 ? c->u_s : c->u_k;
        StageFields<T> f = stage_fields<T>(c, phi, u);
        launch_rhs<T>(g, c->ph, f, s);
        const T* u0[3] = {(const T*)c->u_s[0], (const T*)c->u_s[1], (const T*)c->u_s[2]};
        const T* rmc[3] = {(const T*)c->rm[0], (const T*)c->rm[1], (const T*)c->rm[2]};
        T* accm[3] = {(T*)c->acc_m[0], (T*)c->acc_m[1], (T*)c->acc_m[2]};
        T* uk[3] = {(T*)c->u_k[0], (T*)c->u_k[1], (T*)c->u_k[2]};
        launch_stage_update<T>(g, c->ph, st, dt, (const T*)c->phi_s, u0, (const T*)c->rphi, rmc, (T*)c->acc_phi, accm,
                               (T*)c->phi_k, uk, s);
        const double cdt = (st == 3 ? 1.0 : ck[st + 1]) * dt;
        cdi_status stt = project<T>(c, (const T*)c->phi_k, uk, cdt, st);
        if (stt) return stt;
    }
    ++c->hist_steps;
    std::swap(c->phi_s, c->phi_k);
    for (int a = 0; a < 3; ++a) std::swap(c->u_s[a], c->u_k[a]);
    return cuda_check(c, cudaGetLastError(), "kernel launch");
}

// First multigrid level that one CTA solves in shared memory (the largest
// FP32 tail that fits the budget) and its layout.
size_t pick_tail(const cdi_ctx* c, size_t budget, int* lt_out, PersistLayout* L, long max_cells) {
    int lt = c->mg.nlev - 1;
    for (int l = 0; l < c->mg.nlev; ++l) {
        PersistLayout t{};
        if (c->mg.lv[l].g.N <= max_cells && persist_tail_layout(c->g, c->mg, l, t) <= budget) {
            lt = l;
            break;
        }
    }
    *lt_out = lt;
    return persist_tail_layout(c->g, c->mg, lt, *L);
}

cdi_status smem_optin(cdi_ctx* c, size_t* bytes) {
    int dev = 0, optin = 0;
    cdi_status st = cuda_check(c, cudaGetDevice(&dev), "cudaGetDevice");
    if (st) return st;
    st = cuda_check(c, cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev),
                    "cudaDeviceGetAttribute");
    if (st) return st;
    *bytes = (size_t)optin;
    return CDI_OK;
}

template <typename T>
cdi_status persist_setup(cdi_ctx* c) {
    if (c->persist_ready) return CDI_OK;
    size_t optin = 0;
    cdi_status st = smem_optin(c, &optin);
    if (st) return st;
    const size_t budget = optin > 8192 ? optin - 4096 : 0;
    c->persist_smem = pick_tail(c, budget, &c->persist_lt, &c->playout);
    st = cuda_check(c, persist_prepare<T>(c->g.D, c->persist_smem, &c->persist_grid), "persistent kernel setup");
    if (st) return st;
    c->persist_ready = true;
    return CDI_OK;
}

// the descriptor of this context's next steps (current state pointers)
template <typename T>
void fill_inst(const cdi_ctx* c, InstArgs<T>& A, int lt, const PersistLayout& lay, double dt) {
    static_cast<PersistLayout&>(A) = lay;
    A.g = c->g;
    A.ph = c->ph;
    A.phi_s = (T*)c->phi_s;
    A.phi_k = (T*)c->phi_k;
    A.acc_phi = (T*)c->acc_phi;
    A.rphi = (T*)c->rphi;
    A.psi = (T*)c->psi;
    A.muc = (T*)c->muc;
    A.wuY = (T*)c->wuY;
    A.wghost = (T*)c->wghost;
    A.wmuw = (T*)c->wmuw;
    A.colq = c->colq;
    for (int a = 0; a < 3; ++a) {
        A.u_s[a] = (T*)c->u_s[a];
        A.u_k[a] = (T*)c->u_k[a];
        A.acc_m[a] = (T*)c->acc_m[a];
        A.rm[a] = (T*)c->rm[a];
        A.nh[a] = (T*)c->nh[a];
        A.m[a] = (T*)c->m[a];
    }
    for (int l = 0; l < kMaxLevels; ++l) A.lv[l] = c->mg.lv[l];
    A.nlev = c->mg.nlev;
    A.lt = lt;
    A.tol = c->tol;
    A.max_vcycles = c->max_vcycles;
    A.warm = c->warm;
    A.npre = c->npre;
    A.npost = c->npost;
    A.gamma_param = c->gamma;
    A.dt = dt;
    for (int k = 0; k < 4; ++k)
        for (int j = 0; j < 2; ++j) A.hist[k][j] = c->hist[k][j];
    A.hist_step0 = c->hist_steps;
    A.ainv = nullptr;  // the shared-memory tail inverts the coarsest level itself
}

// record one launch's outcome on the context; the kernel swapped the state
// and stage buffers once per finished step
cdi_status apply_stats(cdi_ctx* c, const InstStats& h, const char* who) {
    c->last_cycles = h.last_cycles;
    c->last_resid = h.last_resid;
    c->max_cycles_step = h.max_cycles;
    c->total_cycles_call = h.total_cycles;
    c->hist_steps += h.steps_done;
    for (int s = 0; s < h.steps_done; ++s) {
        std::swap(c->phi_s, c->phi_k);
        for (int a = 0; a < 3; ++a) std::swap(c->u_s[a], c->u_k[a]);
    }
    if (h.status == CDI_OK) return CDI_OK;
    char b[240];
    if (h.status == CDI_ENOCONV)
        snprintf(b, sizeof b, "%spressure solve: %d V-cycles left relative residual %.3e > tol %.3e (step %d)", who,
                 h.last_cycles, h.last_resid, c->tol, h.steps_done);
    else if (h.status == CDI_ETIMEOUT)
        snprintf(b, sizeof b, "%sa grid barrier of the persistent step kernel timed out (step %d)", who, h.steps_done);
    else
        snprintf(b, sizeof b, "%snon-finite value in the pressure solve (step %d)", who, h.steps_done);
    return fail(c, (cdi_status)h.status, b);
}

template <typename T>
cdi_status step_persist(cdi_ctx* c, double dt, int nsteps) {
    cdi_status st = persist_setup<T>(c);
    if (st) return st;
    PersistArgs<T> A{};
    fill_inst<T>(c, A.I, c->persist_lt, c->playout, dt);
    A.partials = c->mg.partials;
    A.ctl = c->ctl;
    A.nsteps = nsteps;
    A.spin_limit = c->spin_limit_ns;
    st = cuda_check(c, cudaMemsetAsync(c->ctl, 0, sizeof(PersistCtl), c->stream), "cudaMemsetAsync(ctl)");
    if (st) return st;
    const bool on = prof_before(KC_STEP, c->stream);
    st = cuda_check(c, launch_step_persist<T>(A, c->persist_smem, c->persist_grid, c->stream),
                    "cudaLaunchCooperativeKernel");
    prof_after(on, c->stream);
    if (st) return st;
    ++g_launches;
    PersistCtl h{};
    st = cuda_check(c, cudaMemcpyAsync(&h, c->ctl, sizeof h, cudaMemcpyDeviceToHost, c->stream), "read ctl");
    if (st) return st;
    st = cuda_check(c, cudaStreamSynchronize(c->stream), "persistent step");
    if (st) return st;
    c->p_mean_pending = false;  // the persistent kernel leaves p zero-mean after every solve
    return apply_stats(c, h.st, "");
}

cdi_status check_wall(cdi_ctx* c, int wall) {
    if (!c) return fail(nullptr, CDI_EINVAL, "null context");
    if (wall < 0 || wall > 2) return fail(c, CDI_EINVAL, "wall must be CDI_WALL_LO, CDI_WALL_HI or CDI_WALL_BOTH");
    return CDI_OK;
}

}  // namespace

// ===========================================================================
extern "C" {

cdi_status cdi_init_grid(cdi_ctx** out, int dim, int nx, int ny, int nz, double Lx, double Ly, double Lz,
                         unsigned wall_mask, int precision) {
    if (!out) return fail(nullptr, CDI_EINVAL, "out is NULL");
    *out = nullptr;
    if (dim != 2 && dim != 3) return fail(nullptr, CDI_EINVAL, "dim must be 2 or 3");
    if (wall_mask != 3u) return fail(nullptr, CDI_EINVAL, "wall_mask must be 3 (walls on both ends of the last axis)");
    if (precision != CDI_FP64 && precision != CDI_FP32_MIXED) return fail(nullptr, CDI_EINVAL, "bad precision");
    int n[3] = {nx, ny, dim == 3 ? nz : 1};
    double L[3] = {Lx, Ly, dim == 3 ? Lz : 0.0};
    const int W = dim - 1;
    for (int a = 0; a < dim; ++a) {
        if (a == W) {
            if (n[a] < 4) return fail(nullptr, CDI_EINVAL, "the wall axis needs at least 4 cells");
        } else if (n[a] < 2 || n[a] % 2) {
            return fail(nullptr, CDI_EINVAL, "periodic extents must be even and >= 2");
        }
        if (!(L[a] > 0.0) || !std::isfinite(L[a])) return fail(nullptr, CDI_EINVAL, "domain lengths must be > 0");
    }
    const double h = Lx / nx;
    for (int a = 1; a < dim; ++a)
        if (std::fabs(L[a] / n[a] - h) > 1e-12 * h) return fail(nullptr, CDI_EINVAL, "the spacing must be uniform");
    const long N = (long)n[0] * n[1] * n[2];
    if (N > (1L << 31)) return fail(nullptr, CDI_EINVAL, "grid too large");
    cdi_ctx* c = new (std::nothrow) cdi_ctx();
    if (!c) return fail(nullptr, CDI_EINVAL, "out of host memory");
    c->g = make_geom(dim, n, h);
    for (int a = 0; a < 3; ++a) c->L[a] = L[a];
    c->precision = precision;
    // V(1,1) in 2D, where the small grids are bound by the barriers of each sweep; V(2,2) in 3D
    // measured fastest a step: V(1,1) on single 2D grids, V(1,2) on 3D grids
    c->npre = 1;
    c->npost = (dim == 2) ? 1 : 2;
    // 3D: over-relaxed finest-level sweeps, measured 4 % fewer V-cycles a step
    // on the 512x256x256 drop for omega 1.1 .. 1.3 (1.4: more)
    c->mg.omega = (dim == 3) ? 1.15f : 1.f;
    c->mg.cpre = -1;
    c->mg.cpost = -1;
    // one clamp rule for both precisions, representable in FP32 (1 - delta
    // must differ from 1): phi in [1e-6, 1 - 1e-6] for psi and every phi(1-phi)
    // factor, |grad psi| floored at 1e-6
    c->ph.delta = 1e-6;
    c->ph.tau = 1e-6;
    c->ph.model = M4A;
    for (int s = 0; s < 2; ++s) {
        c->ph.wall[s].costh = 0.0;
        c->ph.wall[s].beta1 = c->ph.wall[s].beta2 = INFINITY;
        c->ph.wall[s].noslip = 1;
    }
    finalize_phys(c->ph);
    // multigrid hierarchy: halve every axis while all extents stay even and >= 2
    MG& mg = c->mg;
    mg.nlev = 1;
    int ln[3] = {n[0], n[1], n[2]};
    double lh = h;
    auto set_level = [&](int l) { mg.lv[l].g = make_geom(dim, ln, lh); };
    set_level(0);
    for (;;) {
        bool ok = mg.nlev < kMaxLevels;
        for (int a = 0; a < dim; ++a)
            if (ln[a] % 2 || ln[a] / 2 < 2) ok = false;
        if (!ok) break;
        for (int a = 0; a < dim; ++a) ln[a] /= 2;
        lh *= 2.0;
        set_level(mg.nlev++);
    }
    if (mg.lv[mg.nlev - 1].g.N > kMaxCoarse) {
        delete c;
        return fail(nullptr, CDI_EINVAL, "the coarsest multigrid level has more than 64 cells; use extents with more "
                                         "factors of two");
    }
    size_t total = 0;
    carve(c, nullptr, &total);
    c->ws_bytes = total;
    *out = c;
    return CDI_OK;
}

cdi_status cdi_workspace_bytes(const cdi_ctx* c, size_t* bytes) {
    if (!c || !bytes) return fail(nullptr, CDI_EINVAL, "null argument");
    *bytes = c->ws_bytes;
    return CDI_OK;
}

cdi_status cdi_bind_workspace(cdi_ctx* c, void* dev_ptr, size_t bytes, void* stream) {
    if (!c) return fail(nullptr, CDI_EINVAL, "null context");
    if (!dev_ptr) return fail(c, CDI_EINVAL, "workspace pointer is NULL");
    if (bytes < c->ws_bytes) return fail(c, CDI_EINVAL, "workspace too small");
    if (((uintptr_t)dev_ptr) & 255u) return fail(c, CDI_EINVAL, "workspace must be 256-byte aligned");
    cudaPointerAttributes attr;
    if (cudaPointerGetAttributes(&attr, dev_ptr) != cudaSuccess || attr.type != cudaMemoryTypeDevice) {
        cudaGetLastError();
        return fail(c, CDI_EINVAL, "workspace is not device memory");
    }
    c->ws = (char*)dev_ptr;
    c->stream = (cudaStream_t)stream;
    size_t total = 0;
    carve(c, c->ws, &total);
    c->mg.tail_args = nullptr;
    c->tail_ready = false;
    drop_graphs(c);
    if (!c->host_scal) {
        cdi_status st = cuda_check(c, cudaMallocHost((void**)&c->host_scal, S_NSCAL * sizeof(double)),
                                   "cudaMallocHost");
        if (st) return st;
    }
    if (mom_tile_supported(c->g)) {
        cdi_status st = cuda_check(c, mom_tile_prepare(), "tiled momentum setup");
        if (st) return st;
    }
    cdi_status st = cuda_check(c, cudaMemsetAsync(c->ws, 0, c->ws_bytes - 256, c->stream), "cudaMemsetAsync");
    if (st) return st;
    st = cuda_check(c, cudaStreamSynchronize(c->stream), "bind");
    if (st) return st;
    c->bound = true;
    return CDI_OK;
}

cdi_status cdi_set_fluids(cdi_ctx* c, double rho1, double rho2, double mu1, double mu2, double sigma, double eps,
                          double gamma) {
    if (!c) return fail(nullptr, CDI_EINVAL, "null context");
    double v[7] = {rho1, rho2, mu1, mu2, sigma, eps, gamma};
    for (double x : v)
        if (!std::isfinite(x)) return fail(c, CDI_EINVAL, "fluid parameters must be finite");
    if (!(rho1 > 0) || !(rho2 > 0)) return fail(c, CDI_EINVAL, "densities must be > 0");
    if (mu1 < 0 || mu2 < 0) return fail(c, CDI_EINVAL, "viscosities must be >= 0");
    if (!(eps > 0)) return fail(c, CDI_EINVAL, "eps must be > 0");
    c->ph.rho1 = rho1; c->ph.rho2 = rho2; c->ph.mu1 = mu1; c->ph.mu2 = mu2;
    c->ph.sigma = sigma; c->ph.eps = eps;
    c->gamma = gamma;
    c->fluids_set = true;
    for (int s = 0; s < 2; ++s)
        if (c->wall_slip_length[s] > 0.0) {
            c->ph.wall[s].beta1 = mu1 / c->wall_slip_length[s];
            c->ph.wall[s].beta2 = mu2 / c->wall_slip_length[s];
        }
    finalize_phys(c->ph);
    return CDI_OK;
}

cdi_status cdi_set_wall(cdi_ctx* c, int wall, double theta_eq, double slip_length, double U_wall) {
    cdi_status st = check_wall(c, wall);
    if (st) return st;
    if (!(theta_eq > 0.0 && theta_eq < M_PI)) return fail(c, CDI_EINVAL, "theta_eq must lie in (0, pi)");
    if (!(slip_length >= 0.0) || !std::isfinite(slip_length)) return fail(c, CDI_EINVAL, "slip length must be >= 0");
    if (!std::isfinite(U_wall)) return fail(c, CDI_EINVAL, "wall velocity must be finite");
    if (!c->fluids_set) return fail(c, CDI_ESTATE, "call cdi_set_fluids before cdi_set_wall");
    for (int s = 0; s < 2; ++s) {
        if (wall != 2 && wall != s) continue;
        WallDev& w = c->ph.wall[s];
        w.costh = std::cos(theta_eq);
        w.U[0] = U_wall;
        c->wall_slip_length[s] = slip_length;
        if (slip_length == 0.0) {
            w.noslip = 1;
            w.beta1 = w.beta2 = INFINITY;
        } else {
            w.noslip = 0;
            w.beta1 = c->ph.mu1 / slip_length;
            w.beta2 = c->ph.mu2 / slip_length;
            if (!(w.beta1 > 0) || !(w.beta2 > 0)) {
                finalize_phys(c->ph);
                return fail(c, CDI_EINVAL, "slip length form needs mu1, mu2 > 0 (use cdi_set_wall_beta)");
            }
        }
    }
    finalize_phys(c->ph);
    return CDI_OK;
}

cdi_status cdi_set_wall_beta(cdi_ctx* c, int wall, double beta1, double beta2) {
    cdi_status st = check_wall(c, wall);
    if (st) return st;
    const bool inf1 = std::isinf(beta1) && beta1 > 0, inf2 = std::isinf(beta2) && beta2 > 0;
    if (inf1 != inf2) return fail(c, CDI_EINVAL, "beta1 and beta2 must both be finite or both +inf");
    if (!inf1 && (!(beta1 > 0) || !(beta2 > 0) || !std::isfinite(beta1) || !std::isfinite(beta2)))
        return fail(c, CDI_EINVAL, "beta must be > 0");
    for (int s = 0; s < 2; ++s) {
        if (wall != 2 && wall != s) continue;
        WallDev& w = c->ph.wall[s];
        w.beta1 = beta1;
        w.beta2 = beta2;
        w.noslip = inf1 ? 1 : 0;
        c->wall_slip_length[s] = -1.0;
    }
    finalize_phys(c->ph);
    return CDI_OK;
}

cdi_status cdi_set_wall_velocity(cdi_ctx* c, int wall, double Ux, double Uy) {
    cdi_status st = check_wall(c, wall);
    if (st) return st;
    if (!std::isfinite(Ux) || !std::isfinite(Uy)) return fail(c, CDI_EINVAL, "wall velocity must be finite");
    for (int s = 0; s < 2; ++s) {
        if (wall != 2 && wall != s) continue;
        c->ph.wall[s].U[0] = Ux;
        c->ph.wall[s].U[1] = Uy;
    }
    finalize_phys(c->ph);
    return CDI_OK;
}

cdi_status cdi_set_model(cdi_ctx* c, int model) {
    if (!c) return fail(nullptr, CDI_EINVAL, "null context");
    if (model < CDI_MODEL_1A || model > CDI_MODEL_4B) return fail(c, CDI_EINVAL, "unknown slip model");
    c->ph.model = model;
    finalize_phys(c->ph);
    return CDI_OK;
}

cdi_status cdi_set_phi(cdi_ctx* c, const double* phi) {
    cdi_status st = need_bound(c);
    if (st) return st;
    if (!phi) return fail(c, CDI_EINVAL, "phi is NULL");
    c->hist_steps = 0;
    return upload(c, c->phi_s, phi, c->g.N, "phi");
}

cdi_status cdi_set_velocity(cdi_ctx* c, const double* u, const double* v, const double* w) {
    cdi_status st = need_bound(c);
    if (st) return st;
    const double* comps[3] = {u, v, w};
    for (int a = 0; a < c->g.D; ++a) {
        if (!comps[a]) return fail(c, CDI_EINVAL, "velocity component is NULL");
        st = upload(c, c->u_s[a], comps[a], nface(c->g, a), "velocity");
        if (st) return st;
    }
    c->hist_steps = 0;
    // no penetration: the wall planes of the wall-normal component are zero
    void* wn = c->u_s[c->g.W];
    if (c->precision == CDI_FP64)
        k_zero_wall_planes<double><<<nblk(c->g.NP), 256, 0, c->stream>>>(c->g.N, c->g.NP, (double*)wn);
    else
        k_zero_wall_planes<float><<<nblk(c->g.NP), 256, 0, c->stream>>>(c->g.N, c->g.NP, (float*)wn);
    return cuda_check(c, cudaStreamSynchronize(c->stream), "set_velocity");
}

cdi_status cdi_set_solver(cdi_ctx* c, double tol, int max_vcycles, int warm) {
    if (!c) return fail(nullptr, CDI_EINVAL, "null context");
    if (!(tol > 0.0) || !std::isfinite(tol)) return fail(c, CDI_EINVAL, "tol must be > 0");
    if (max_vcycles < 1) return fail(c, CDI_EINVAL, "max_vcycles must be >= 1");
    if (warm != CDI_WARM_PREV && warm != CDI_WARM_ZERO && warm != CDI_WARM_EXTRAP && warm != CDI_WARM_UNET)
        return fail(c, CDI_EINVAL, "bad warm-start mode");
    c->tol = tol;
    c->max_vcycles = max_vcycles;
    c->warm = warm;
    c->hist_steps = 0;
    return CDI_OK;
}

cdi_status cdi_step(cdi_ctx* c, double dt, int nsteps) {
    cdi_status st = need_bound(c);
    if (st) return st;
    if (!(dt > 0.0) || !std::isfinite(dt)) return fail(c, CDI_EINVAL, "dt must be > 0");
    if (nsteps < 0) return fail(c, CDI_EINVAL, "nsteps must be >= 0");
    if (!c->fluids_set) return fail(c, CDI_ESTATE, "fluids not set");
    c->max_cycles_step = 0;
    c->total_cycles_call = 0;
    if (nsteps == 0) return CDI_OK;
    if (c->warm == CDI_WARM_UNET && !c->unet) return fail(c, CDI_ESTATE, "CDI_WARM_UNET without an attached network");
    const long l0 = g_launches;
    const bool persistent =
        c->exec == CDI_EXEC_PERSISTENT || (c->exec == CDI_EXEC_AUTO && c->g.N <= (1L << 20));
    if (persistent && c->warm != CDI_WARM_UNET) {
        st = (c->precision == CDI_FP64) ? step_persist<double>(c, dt, nsteps) : step_persist<float>(c, dt, nsteps);
        if (st) return st;
    } else {
        for (int n = 0; n < nsteps; ++n) {
            st = (c->precision == CDI_FP64) ? step_once<double>(c, dt) : step_once<float>(c, dt);
            if (st) return st;
        }
    }
    c->launches_per_step = (g_launches - l0 + nsteps - 1) / nsteps;   // rounded up: 1 for a persistent call
    return cuda_check(c, cudaStreamSynchronize(c->stream), "cdi_step");
}

cdi_status cdi_set_warm_unet(cdi_ctx* c, cdi_unet* net) {
    if (!c) return fail(nullptr, CDI_EINVAL, "null context");
    if (net) {
        if (c->g.D != 3) return fail(c, CDI_EINVAL, "the network needs a 3D grid");
        int n[3];
        unet_extents(net, n);
        if (n[0] != c->g.n[0] || n[1] != c->g.n[1] || n[2] != c->g.n[2])
            return fail(c, CDI_EINVAL, "network extents differ from the grid");
    }
    c->unet = net;
    return CDI_OK;
}

cdi_status cdi_last_pressure(cdi_ctx* c, double* f, double* p) {
    cdi_status st = need_bound(c);
    if (st) return st;
    if (f) {
        st = download_level0(c, f, false);
        if (st) return st;
    }
    if (p) st = download_level0(c, p, true);
    return st;
}

cdi_status cdi_set_relaxation(cdi_ctx* c, double omega) {
    if (!c) return fail(nullptr, CDI_EINVAL, "null context");
    if (!(omega > 0.0 && omega < 2.0)) return fail(c, CDI_EINVAL, "relaxation must lie in (0, 2)");
    c->mg.omega = (float)omega;
    // the V-cycle graphs hold the kernels' arguments
    drop_graphs(c);
    return CDI_OK;
}

cdi_status cdi_set_smoothing(cdi_ctx* c, int npre, int npost) {
    if (!c) return fail(nullptr, CDI_EINVAL, "null context");
    if (npre < 1 || npre > 4 || npost < 1 || npost > 4) return fail(c, CDI_EINVAL, "sweeps must lie in [1, 4]");
    c->npre = npre;
    c->npost = npost;
    // the launch-per-kernel tail descriptor and V-cycle graphs hold the sweep counts
    c->tail_ready = false;
    c->mg.tail_args = nullptr;
    drop_graphs(c);
    return CDI_OK;
}

cdi_status cdi_set_coarse_smoothing(cdi_ctx* c, int npre, int npost) {
    if (!c) return fail(nullptr, CDI_EINVAL, "null context");
    const bool dflt = npre == -1 && npost == -1;
    if (!dflt && (npre < 0 || npre > 4 || npost < 0 || npost > 4 || npre + npost < 1))
        return fail(c, CDI_EINVAL, "coarse sweeps must lie in [0, 4] with at least one, or both be -1");
    c->mg.cpre = npre;
    c->mg.cpost = npost;
    drop_graphs(c);  // the graphs hold the launches of the previous counts
    return CDI_OK;
}

cdi_status cdi_set_level0_sweep(cdi_ctx* c, int mode) {
    if (!c) return fail(nullptr, CDI_EINVAL, "null context");
    if (mode != CDI_SWEEP_AUTO && mode != CDI_SWEEP_ONEPASS && mode != CDI_SWEEP_COLOUR &&
        mode != CDI_SWEEP_ONEPASS_CPASYNC)
        return fail(c, CDI_EINVAL,
                    "sweep mode must be CDI_SWEEP_AUTO, CDI_SWEEP_ONEPASS, CDI_SWEEP_COLOUR or "
                    "CDI_SWEEP_ONEPASS_CPASYNC");
    c->mg.sweep_mode = mode;
    // the V-cycle graphs hold the launches of the previous choice
    drop_graphs(c);
    return CDI_OK;
}

cdi_status cdi_set_barrier_timeout(cdi_ctx* c, long long ns) {
    if (!c) return fail(nullptr, CDI_EINVAL, "null context");
    if (ns < 0 || ns > 60000000000LL) return fail(c, CDI_EINVAL, "barrier timeout must lie in [0, 60 s]");
    c->spin_limit_ns = (long)ns;
    return CDI_OK;
}

cdi_status cdi_set_exec(cdi_ctx* c, int mode) {
    if (!c) return fail(nullptr, CDI_EINVAL, "null context");
    if (mode != CDI_EXEC_PERSISTENT && mode != CDI_EXEC_KERNELS && mode != CDI_EXEC_AUTO)
        return fail(c, CDI_EINVAL, "unknown exec mode");
    c->exec = mode;
    return CDI_OK;
}

cdi_status cdi_mass(cdi_ctx* c, double* mass_out) {
    cdi_status st = need_bound(c);
    if (st) return st;
    if (!mass_out) return fail(c, CDI_EINVAL, "mass_out is NULL");
    if (c->precision == CDI_FP64) launch_mass<double>(c->g, (const double*)c->phi_s, c->mg, c->stream);
    else launch_mass<float>(c->g, (const float*)c->phi_s, c->mg, c->stream);
    st = read_scalars(c);
    if (st) return st;
    *mass_out = c->host_scal[S_MASS];
    return CDI_OK;
}

cdi_status cdi_contact_angle(cdi_ctx* c, int wall, double* theta, double* wetted) {
    cdi_status st = need_bound(c);
    if (st) return st;
    if (wall != 0 && wall != 1) return fail(c, CDI_EINVAL, "wall must be CDI_WALL_LO or CDI_WALL_HI");
    if (!theta || !wetted) return fail(c, CDI_EINVAL, "null output");
    if (c->precision == CDI_FP64)
        launch_wall_columns<double>(c->g, c->ph, (const double*)c->phi_s, (double*)c->psi, c->cols, c->stream);
    else
        launch_wall_columns<float>(c->g, c->ph, (const float*)c->phi_s, (float*)c->psi, c->cols, c->stream);
    launch_contact_line(c->g, wall, c->cols, c->mg, c->stream);
    st = read_scalars(c);
    if (st) return st;
    *theta = c->host_scal[S_THETA];
    *wetted = c->host_scal[S_WETTED];
    return CDI_OK;
}

cdi_status cdi_get_fields(cdi_ctx* c, double* phi, double* u, double* v, double* w, double* p) {
    cdi_status st = need_bound(c);
    if (st) return st;
    st = download(c, phi, c->phi_s, c->g.N);
    if (st) return st;
    double* comps[3] = {u, v, w};
    for (int a = 0; a < c->g.D; ++a) {
        st = download(c, comps[a], c->u_s[a], nface(c->g, a));
        if (st) return st;
    }
    if (p) st = download_level0(c, p, true);
    return st;
}

cdi_status cdi_eval_rhs(cdi_ctx* c, double gamma, double* rphi, double* ru, double* rv, double* rw) {
    cdi_status st = need_bound(c);
    if (st) return st;
    if (c->precision == CDI_FP64) {
        set_gamma<double>(c, c->u_s, gamma >= 0 ? gamma : c->gamma);
        launch_rhs<double>(c->g, c->ph, stage_fields<double>(c, c->phi_s, c->u_s), c->stream);
    } else {
        set_gamma<float>(c, c->u_s, gamma >= 0 ? gamma : c->gamma);
        launch_rhs<float>(c->g, c->ph, stage_fields<float>(c, c->phi_s, c->u_s), c->stream);
    }
    st = cuda_check(c, cudaGetLastError(), "eval_rhs launch");
    if (st) return st;
    st = download(c, rphi, c->rphi, c->g.N);
    if (st) return st;
    double* comps[3] = {ru, rv, rw};
    for (int a = 0; a < c->g.D; ++a) {
        st = download(c, comps[a], c->rm[a], nface(c->g, a));
        if (st) return st;
    }
    return CDI_OK;
}

cdi_status cdi_eval_wall(cdi_ctx* c, double* uY, double* ghost) {
    cdi_status st = need_bound(c);
    if (st) return st;
    if (c->precision == CDI_FP64) {
        set_gamma<double>(c, c->u_s, c->gamma >= 0 ? c->gamma : 0.0);
        launch_rhs<double>(c->g, c->ph, stage_fields<double>(c, c->phi_s, c->u_s), c->stream);
    } else {
        set_gamma<float>(c, c->u_s, c->gamma >= 0 ? c->gamma : 0.0);
        launch_rhs<float>(c->g, c->ph, stage_fields<float>(c, c->phi_s, c->u_s), c->stream);
    }
    const long nw = 2L * (c->g.D - 1) * c->g.NP;
    st = download(c, uY, c->wuY, nw);
    if (st) return st;
    return download(c, ghost, c->wghost, nw);
}

cdi_status cdi_solve_pressure(cdi_ctx* c, const double* f, double* p) {
    cdi_status st = need_bound(c);
    if (st) return st;
    if (!f || !p) return fail(c, CDI_EINVAL, "null array");
    const Geom& g = c->g;
    MG& mg = c->mg;
    cudaStream_t s = c->stream;
    st = upload_level0(c, f, false);
    if (st) return st;
    st = upload_level0(c, p, true);
    if (st) return st;
    if (c->precision == CDI_FP64) {
        launch_sum_f<double>(g, mg, s);
        launch_sub_mean_and_norm<double>(g, mg, s);
        launch_mg_coef<double>(g, c->ph, (const double*)c->phi_s, mg, s);
        st = mg_solve<double>(c);
    } else {
        launch_sum_f<float>(g, mg, s);
        launch_sub_mean_and_norm<float>(g, mg, s);
        launch_mg_coef<float>(g, c->ph, (const float*)c->phi_s, mg, s);
        st = mg_solve<float>(c);
    }
    if (st) return st;
    return download_level0(c, p, true);
}

cdi_status cdi_profile_start(cdi_ctx* c, const char* kernel, int max_launches) {
    if (!c || !kernel) return fail(c, CDI_EINVAL, "null argument");
    if (max_launches < 1 || max_launches > (1 << 20)) return fail(c, CDI_EINVAL, "max_launches out of range");
    int kc = -1;
    for (int i = 0; i < KC_COUNT; ++i)
        if (std::strcmp(kernel, kKernelClassNames[i]) == 0) kc = i;
    if (kc < 0) return fail(c, CDI_EINVAL, std::string("unknown kernel class ") + kernel);
    Profiler& P = g_prof;
    if (P.ev) {
        for (int i = 0; i < 2 * P.cap; ++i) cudaEventDestroy(P.ev[i]);
        delete[] P.ev;
        P.ev = nullptr;
    }
    P.ev = new (std::nothrow) cudaEvent_t[2 * max_launches];
    if (!P.ev) return fail(c, CDI_EINVAL, "out of host memory");
    for (int i = 0; i < 2 * max_launches; ++i) {
        cdi_status st = cuda_check(c, cudaEventCreate(&P.ev[i]), "cudaEventCreate");
        if (st) {
            for (int j = 0; j < i; ++j) cudaEventDestroy(P.ev[j]);
            delete[] P.ev;
            P.ev = nullptr;
            return st;
        }
    }
    P.cap = max_launches;
    P.used = 0;
    P.target = kc;
    return CDI_OK;
}

cdi_status cdi_profile_stop(cdi_ctx* c, double* total_ms, long* launches) {
    if (!c) return fail(nullptr, CDI_EINVAL, "null context");
    Profiler& P = g_prof;
    cdi_status st = cuda_check(c, cudaStreamSynchronize(c->stream), "profile sync");
    if (st) return st;
    double tot = 0.0;
    for (int i = 0; i < P.used; ++i) {
        float ms = 0.f;
        st = cuda_check(c, cudaEventElapsedTime(&ms, P.ev[2 * i], P.ev[2 * i + 1]), "cudaEventElapsedTime");
        if (st) return st;
        tot += ms;
    }
    if (total_ms) *total_ms = tot;
    if (launches) *launches = P.used;
    for (int i = 0; i < 2 * P.cap; ++i) cudaEventDestroy(P.ev[i]);
    delete[] P.ev;
    P.ev = nullptr;
    P.cap = 0;
    P.used = 0;
    P.target = -1;
    return CDI_OK;
}

cdi_status cdi_last_stats(cdi_ctx* c, int* vcycles, double* resid, int* max_vcycles_step,
                          int* total_vcycles_call) {
    if (!c) return fail(nullptr, CDI_EINVAL, "null context");
    if (vcycles) *vcycles = c->last_cycles;
    if (resid) *resid = c->last_resid;
    if (max_vcycles_step) *max_vcycles_step = c->max_cycles_step;
    if (total_vcycles_call) *total_vcycles_call = c->total_cycles_call;
    return CDI_OK;
}

cdi_status cdi_launches_per_step(cdi_ctx* c, long* launches) {
    if (!c || !launches) return fail(c, CDI_EINVAL, "null argument");
    *launches = c->launches_per_step;
    return CDI_OK;
}

const char* cdi_last_error(const cdi_ctx* c) {
    if (!c) return g_init_error.c_str();
    return c->err.c_str();
}

void cdi_destroy(cdi_ctx* c) {
    if (!c) return;
    drop_graphs(c);
    if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
    if (c->host_scal) cudaFreeHost(c->host_scal);
    delete c;
}

}  // extern "C"

// ===========================================================================
// Batched sweep: many independent contexts advanced by one launch
// ===========================================================================
struct cdi_batch {
    int n = 0;
    int dim = 2;
    int precision = CDI_FP64;
    std::vector<cdi_ctx*> inst;
    std::vector<int> order;        // instance indices by decreasing cell count
    std::vector<int> lt;           // per instance: first level solved in shared memory
    std::vector<PersistLayout> lay;
    size_t smem = 0;               // dynamic shared memory of the launch
    size_t tail_budget = 0;        // shared-memory budget of one CTA's multigrid tail
    int threads = 512;
    int grid = 0;
    bool prepared = false;
    char* ws = nullptr;
    size_t ws_bytes = 0;
    cudaStream_t stream = nullptr;
    void* d_insts = nullptr;
    InstStats* d_stats = nullptr;
    int* d_counter = nullptr;
    std::vector<InstStats> stats;  // last launch, caller's order
    float last_ms = 0.f;
    std::string err;
};

namespace {

std::string g_batch_error;

cdi_status bfail(cdi_batch* b, cdi_status st, const std::string& msg) {
    if (b) b->err = msg;
    else g_batch_error = msg;
    return st;
}

size_t inst_bytes(int precision) {
    return precision == CDI_FP64 ? sizeof(InstArgs<double>) : sizeof(InstArgs<float>);
}

void batch_carve(cdi_batch* b, char* base, size_t* total) {
    Carver cv{base};
    b->d_insts = cv.take((size_t)b->n * inst_bytes(b->precision));
    b->d_stats = (InstStats*)cv.take((size_t)b->n * sizeof(InstStats));
    b->d_counter = (int*)cv.take(sizeof(int));
    *total = cv.off + 256;
}

template <typename T>
cdi_status batch_launch(cdi_batch* b, const double* dt, int nsteps, float* ms) {
    cdi_status st;
    if (!b->prepared) {
        cudaError_t e = batch_prepare<T>(b->dim, b->threads, b->smem, &b->grid);
        if (e != cudaSuccess) return bfail(b, CDI_ECUDA, std::string("batched kernel setup: ") + cudaGetErrorString(e));
        b->prepared = true;
    }
    std::vector<InstArgs<T>> h(b->n);
    for (int k = 0; k < b->n; ++k) {
        const int i = b->order[k];
        fill_inst<T>(b->inst[i], h[k], b->lt[i], b->lay[i], dt[i]);
    }
    cudaStream_t s = b->stream;
    cudaError_t e = cudaMemcpyAsync(b->d_insts, h.data(), h.size() * sizeof(InstArgs<T>), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(b->d_stats, 0, (size_t)b->n * sizeof(InstStats), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(b->d_counter, 0, sizeof(int), s);
    if (e != cudaSuccess) return bfail(b, CDI_ECUDA, std::string("batch upload: ") + cudaGetErrorString(e));
    BatchArgs<T> B{(const InstArgs<T>*)b->d_insts, b->d_stats, b->d_counter, b->n, nsteps};
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (ms) {
        cudaEventCreate(&e0);
        cudaEventCreate(&e1);
        cudaEventRecord(e0, s);
    }
    const bool on = prof_before(KC_STEP, s);
    e = launch_batch_persist<T>(B, b->dim, b->threads, b->smem, b->grid, s);
    prof_after(on, s);
    if (ms) cudaEventRecord(e1, s);
    if (e != cudaSuccess) return bfail(b, CDI_ECUDA, std::string("batched launch: ") + cudaGetErrorString(e));
    ++g_launches;
    std::vector<InstStats> hs(b->n);
    e = cudaMemcpyAsync(hs.data(), b->d_stats, hs.size() * sizeof(InstStats), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return bfail(b, CDI_ECUDA, std::string("batched step: ") + cudaGetErrorString(e));
    if (ms) {
        cudaEventElapsedTime(ms, e0, e1);
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
    }
    cdi_status first = CDI_OK;
    for (int k = 0; k < b->n; ++k) {
        const int i = b->order[k];
        b->stats[i] = hs[k];
        char who[48];
        snprintf(who, sizeof who, "instance %d: ", i);
        st = apply_stats(b->inst[i], hs[k], who);
        if (st && first == CDI_OK) {
            first = st;
            b->err = b->inst[i]->err;
        }
    }
    return first;
}

}  // namespace

extern "C" {

// levels of every instance solved in one CTA's shared memory under a budget
// (bytes a CTA); the launch takes the largest instance's need
void batch_tail_layout(cdi_batch* b, size_t budget) {
    b->tail_budget = budget;
    b->smem = 0;
    for (int i = 0; i < b->n; ++i) {
        const size_t sm = pick_tail(b->inst[i], budget, &b->lt[i], &b->lay[i]);
        b->smem = std::max(b->smem, sm);
    }
    b->prepared = false;
}

cdi_status cdi_batch_create(cdi_batch** out, int n, cdi_ctx* const* instances) {
    if (!out) return bfail(nullptr, CDI_EINVAL, "out is NULL");
    *out = nullptr;
    if (n < 1 || !instances) return bfail(nullptr, CDI_EINVAL, "need at least one instance");
    cdi_batch* b = new (std::nothrow) cdi_batch();
    if (!b) return bfail(nullptr, CDI_EINVAL, "out of host memory");
    b->n = n;
    b->inst.assign(instances, instances + n);
    for (int i = 0; i < n; ++i) {
        cdi_ctx* c = b->inst[i];
        if (!c || !c->bound || !c->fluids_set) {
            delete b;
            return bfail(nullptr, CDI_ESTATE, "every instance must be initialised, bound and have its fluids set");
        }
        if (c->precision != b->inst[0]->precision || c->g.D != b->inst[0]->g.D) {
            delete b;
            return bfail(nullptr, CDI_EINVAL, "all instances need the same dimension and precision");
        }
        for (int j = 0; j < i; ++j)
            if (b->inst[j] == c) {
                delete b;
                return bfail(nullptr, CDI_EINVAL, "an instance appears twice");
            }
    }
    b->dim = b->inst[0]->g.D;
    b->precision = b->inst[0]->precision;
    b->stream = b->inst[0]->stream;
    b->order.resize(n);
    for (int i = 0; i < n; ++i) b->order[i] = i;
    std::stable_sort(b->order.begin(), b->order.end(),
                     [&](int x, int y) { return b->inst[x]->g.N > b->inst[y]->g.N; });
    // shared-memory tail per instance under a budget that leaves room for two
    // CTAs per SM; the launch uses the largest
    size_t optin = 0;
    cdi_status st = smem_optin(b->inst[0], &optin);
    if (st) {
        delete b;
        return bfail(nullptr, st, "cannot query the device");
    }
    b->lt.resize(n);
    b->lay.resize(n);
    b->stats.assign(n, InstStats{});
    batch_tail_layout(b, std::min<size_t>(optin > 8192 ? optin - 4096 : 0, 100 * 1024));
    size_t total = 0;
    batch_carve(b, nullptr, &total);
    b->ws_bytes = total;
    *out = b;
    return CDI_OK;
}

cdi_status cdi_batch_workspace_bytes(const cdi_batch* b, size_t* bytes) {
    if (!b || !bytes) return bfail(nullptr, CDI_EINVAL, "null argument");
    *bytes = b->ws_bytes;
    return CDI_OK;
}

cdi_status cdi_batch_bind_workspace(cdi_batch* b, void* dev_ptr, size_t bytes, void* stream) {
    if (!b) return bfail(nullptr, CDI_EINVAL, "null batch");
    if (!dev_ptr || bytes < b->ws_bytes) return bfail(b, CDI_EINVAL, "workspace missing or too small");
    if (((uintptr_t)dev_ptr) & 255u) return bfail(b, CDI_EINVAL, "workspace must be 256-byte aligned");
    b->ws = (char*)dev_ptr;
    b->stream = (cudaStream_t)stream;
    size_t total = 0;
    batch_carve(b, b->ws, &total);
    return CDI_OK;
}

cdi_status cdi_batch_set_threads(cdi_batch* b, int threads) {
    if (!b) return bfail(nullptr, CDI_EINVAL, "null batch");
    if (threads != 256 && threads != 512 && threads != 1024) return bfail(b, CDI_EINVAL, "threads must be 256, 512 or 1024");
    if (threads != b->threads) b->prepared = false;
    b->threads = threads;
    return CDI_OK;
}

cdi_status cdi_batch_step(cdi_batch* b, const double* dt, int nsteps) {
    if (!b) return bfail(nullptr, CDI_EINVAL, "null batch");
    if (!b->ws) return bfail(b, CDI_ESTATE, "no workspace bound");
    if (!dt) return bfail(b, CDI_EINVAL, "dt is NULL");
    if (nsteps < 0) return bfail(b, CDI_EINVAL, "nsteps must be >= 0");
    for (int i = 0; i < b->n; ++i) {
        if (!(dt[i] > 0.0) || !std::isfinite(dt[i])) return bfail(b, CDI_EINVAL, "every dt must be > 0");
        if (b->inst[i]->warm == CDI_WARM_UNET)
            return bfail(b, CDI_EINVAL, "CDI_WARM_UNET is not available in batched execution");
    }
    if (nsteps == 0) return CDI_OK;
    return b->precision == CDI_FP64 ? batch_launch<double>(b, dt, nsteps, &b->last_ms)
                                    : batch_launch<float>(b, dt, nsteps, &b->last_ms);
}

cdi_status cdi_batch_set_tail_budget(cdi_batch* b, size_t bytes) {
    if (!b) return bfail(nullptr, CDI_EINVAL, "null batch");
    size_t optin = 0;
    cdi_status st = smem_optin(b->inst[0], &optin);
    if (st) return bfail(b, st, "cannot query the device");
    if (bytes < 8192 || bytes + 4096 > optin) return bfail(b, CDI_EINVAL, "tail budget outside [8 KiB, opt-in limit - 4 KiB]");
    batch_tail_layout(b, bytes);
    return CDI_OK;
}

cdi_status cdi_batch_autotune(cdi_batch* b, const double* dt, int trial_steps, int* threads_out,
                              size_t* tail_bytes_out, double* ms_out) {
    if (!b) return bfail(nullptr, CDI_EINVAL, "null batch");
    if (trial_steps < 1) return bfail(b, CDI_EINVAL, "trial_steps must be >= 1");
    size_t optin = 0;
    cdi_status st = smem_optin(b->inst[0], &optin);
    if (st) return bfail(b, st, "cannot query the device");
    const int cand[3] = {256, 512, 1024};
    const size_t budgets[4] = {32 * 1024, 64 * 1024, 100 * 1024, optin > 8192 ? optin - 4096 : 0};
    int best = b->threads;
    size_t best_budget = b->tail_budget;
    float best_ms = 1e30f;
    for (int u = 0; u < 4; ++u) {
        batch_tail_layout(b, budgets[u]);
        for (int k = 0; k < 3; ++k) {
            if (ms_out) ms_out[u * 3 + k] = -1.0;
            st = cdi_batch_set_threads(b, cand[k]);
            if (st) return st;
            {  // the candidate must fit one CTA per SM with this shared memory
                int grid = 0;
                cudaError_t e = b->precision == CDI_FP64 ? batch_prepare<double>(b->dim, cand[k], b->smem, &grid)
                                                         : batch_prepare<float>(b->dim, cand[k], b->smem, &grid);
                if (e != cudaSuccess || grid < 1) {
                    cudaGetLastError();
                    continue;
                }
            }
            st = cdi_batch_step(b, dt, trial_steps);
            if (st) return st;
            if (ms_out) ms_out[u * 3 + k] = b->last_ms;
            if (b->last_ms < best_ms) {
                best_ms = b->last_ms;
                best = cand[k];
                best_budget = budgets[u];
            }
        }
    }
    batch_tail_layout(b, best_budget);
    cdi_batch_set_threads(b, best);
    if (threads_out) *threads_out = best;
    if (tail_bytes_out) *tail_bytes_out = best_budget;
    return CDI_OK;
}

cdi_status cdi_batch_stats(cdi_batch* b, int i, int* status, int* max_vcycles, int* total_vcycles, float* last_ms) {
    if (!b) return bfail(nullptr, CDI_EINVAL, "null batch");
    if (i < 0 || i >= b->n) return bfail(b, CDI_EINVAL, "instance index out of range");
    if (status) *status = b->stats[i].status;
    if (max_vcycles) *max_vcycles = b->stats[i].max_cycles;
    if (total_vcycles) *total_vcycles = b->stats[i].total_cycles;
    if (last_ms) *last_ms = b->last_ms;
    return CDI_OK;
}

const char* cdi_batch_last_error(const cdi_batch* b) {
    if (!b) return g_batch_error.c_str();
    return b->err.c_str();
}

void cdi_batch_destroy(cdi_batch* b) { delete b; }

}  // extern "C"
