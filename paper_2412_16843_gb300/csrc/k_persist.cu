// Persistent time-step kernels.
//
// k_step_persist: nsteps full RK4 steps (Sec. 4) of ONE grid in one
//   cooperative launch with one CTA per SM.  Every phase (the right-hand side
//   of Eqs. CDI and NS_momentum, the RK4 stage update, each projection with its
//   multigrid V-cycles and convergence test) is a grid-stride loop between
//   grid barriers.  Barriers wait a bounded time, then set CDI_ETIMEOUT and
//   every CTA returns.  Reductions are deterministic: each CTA writes one
//   partial and every CTA sums the partials in the same order, so all take the
//   same convergence decision.  Data another CTA wrote before the last barrier
//   is read with ld.global.cg (L2), never from a possibly stale L1 line.
//
// k_batch_persist: many independent grids (a parameter sweep) in one launch.
//   Each CTA takes the largest instance not yet taken (atomic counter over a
//   size-sorted descriptor array) and runs all its steps alone, so every
//   barrier is a __syncthreads and no CTA ever waits for another.
//
// Both run the same step code, written once against an executor X that
// supplies the thread range, the barrier and the reductions.  In both, the
// multigrid levels that fit in shared memory are solved by one CTA there.
#include "ops.cuh"
#include "../../include/cdi.h"

namespace cdi {

namespace {

using LG = ops::LdCG;
using LP = ops::LdPlain;

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
// block-wide sum or max, returned to every thread of the block
template <bool MAX>
__device__ double block_reduce_all(double v) {
    __shared__ double sh[32];
    __shared__ double res;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    v = MAX ? warp_max(v) : warp_sum(v);
    __syncthreads();
    if (lane == 0) sh[wid] = v;
    __syncthreads();
    if (wid == 0) {
        const int nw = (blockDim.x + 31) >> 5;
        double x = lane < nw ? sh[lane] : 0.0;
        x = MAX ? warp_max(x) : warp_sum(x);
        if (lane == 0) res = x;
    }
    __syncthreads();
    return res;
}

__device__ __forceinline__ unsigned long long globaltimer() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// ---------------------------------------------------------------------------
// executors
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned long long atom_add_acq_rel(unsigned long long* a, unsigned long long v) {
    unsigned long long old;
    asm volatile("atom.acq_rel.gpu.global.add.u64 %0, [%1], %2;" : "=l"(old) : "l"(a), "l"(v) : "memory");
    return old;
}
__device__ __forceinline__ unsigned long long ld_acquire(const unsigned long long* a) {
    unsigned long long v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(a) : "memory");
    return v;
}

struct GridX {
    PersistCtl* ctl;
    double* partials;  // 2 * kPartials
    long limit;        // barrier timeout, ns
    int red;
    unsigned long long epoch;  // barriers passed by this CTA
    using Ld = LG;
    __device__ int tid() const { return blockIdx.x * blockDim.x + threadIdx.x; }
    __device__ int nth() const { return gridDim.x * blockDim.x; }
    // the thread's first index of a loop with stride nth() whose consecutive
    // indices go to consecutive CTAs
    __device__ int spread() const { return threadIdx.x * gridDim.x + blockIdx.x; }
    __device__ bool tail_cta() const { return blockIdx.x == 0; }
    __device__ bool leader() const { return blockIdx.x == 0 && threadIdx.x == 0; }
    // Grid barrier on one arrival counter that only grows: barrier number m
    // is passed once the counter reaches m x gridDim.x.  Thread 0 arrives with
    // one acquire-release atomic (publishing the CTA's writes, ordered before
    // it by __syncthreads) and polls with acquire loads.  A wait longer than
    // `limit` ns (or 2^31 polls) sets CDI_ETIMEOUT and sets the bit kBarError
    // of the counter with an atomic OR (idempotent, so CTAs that give up at
    // the same time cannot carry it out of the word; arrivals never reach
    // that bit), which releases every waiter of this and every later barrier
    // with false.  Returns false when the launch is ending.
    __device__ bool sync() {
        __shared__ int ok;
        __syncthreads();  // the CTA's writes of this phase are done
        ++epoch;
        if (threadIdx.x == 0) {
            const unsigned long long target = epoch * gridDim.x;
            unsigned long long v = atom_add_acq_rel(&ctl->bar, 1ull) + 1ull;
            if (v < target) {
                const unsigned long long t0 = globaltimer();
                long it = 0;
                do {
                    __nanosleep(20);
                    v = ld_acquire(&ctl->bar);
                    if (v < target && (++it > (1L << 31) || globaltimer() - t0 > (unsigned long long)limit)) {
                        atomicCAS(&ctl->st.status, 0, (int)CDI_ETIMEOUT);
                        atomicOr(&ctl->bar, kBarError);
                        v = kBarError;
                    }
                } while (v < target);
            }
            ok = v < kBarError;
        }
        __syncthreads();
        return ok != 0;
    }
    template <bool MAX>
    __device__ bool reduce(double v, double& out) {
        double* part = partials + (red++ & 1) * kPartials;
        v = block_reduce_all<MAX>(v);
        if (threadIdx.x == 0) part[blockIdx.x] = v;
        if (!sync()) return false;
        double s = 0.0;
        for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x)
            s = MAX ? fmax(s, __ldcg(part + b)) : s + __ldcg(part + b);
        out = block_reduce_all<MAX>(s);
        return true;
    }
};

struct BlockX {
    using Ld = LP;  // one CTA owns the instance: its own writes are visible after __syncthreads
    __device__ int tid() const { return threadIdx.x; }
    __device__ int nth() const { return blockDim.x; }
    __device__ int spread() const { return threadIdx.x; }
    __device__ bool tail_cta() const { return true; }
    __device__ bool leader() const { return threadIdx.x == 0; }
    __device__ bool sync() {
        __syncthreads();
        return true;
    }
    template <bool MAX>
    __device__ bool reduce(double v, double& out) {
        out = block_reduce_all<MAX>(v);
        return true;
    }
};

// ---------------------------------------------------------------------------
// multigrid tail: FP32 levels lt .. nlev-1 by one CTA in shared memory.
// Input: the right-hand side r of level lt (global); output: its correction e.
// Level geometry and shared-memory offsets are copied into registers per
// level, so no per-thread array is indexed at run time.
// ---------------------------------------------------------------------------
struct SmLevel {
    Geom g;
    float* e;
    float* r;
    float* b[3];
};

template <typename T, int DIM>
__device__ __forceinline__ SmLevel sm_level(const InstArgs<T>& A, float* sm, int l) {
    SmLevel s;
    s.g = A.lv[l].g;
    s.e = sm + A.sm_e[l];
    s.r = sm + A.sm_r[l];
#pragma unroll
    for (int a = 0; a < 3; ++a) s.b[a] = (a < DIM) ? sm + A.sm_b[l][a] : nullptr;
    return s;
}

// one colour of a smoothing pass of a shared-memory level of the tail
template <int DIM>
__device__ __forceinline__ void tail_pass(const SmLevel& L, const float* const* bl, int col, int t0, int nt,
                                          int half) {
    ops::colour_pass(
        t0, half, nt,
        [&](int k, long& c) {
            c = ops::colour_cell(L.g, col, k);
            return ops::rbgs_val<LP, float, DIM>(L.g, bl, L.e, L.r, c);
        },
        [&](long c, float v) { L.e[c] = v; });
}

template <typename T, int DIM>
__device__ void tail_vcycle(const InstArgs<T>& A, bool first, float* sm) {
    const int lt = A.lt, nl = A.nlev;
    const int nt = blockDim.x, t0 = threadIdx.x;
    double* sd = reinterpret_cast<double*>(sm + A.sm_dbl);
    if (first) {
        // coefficients of the tail levels (constant during one solve)
        const SmLevel top = sm_level<T, DIM>(A, sm, lt);
        const int ntop = (int)(top.g.N + top.g.NP);
        if (lt == 0 || A.tail_bf_stored) {
            // stored by an earlier phase or kernel of this solve: copied in
            for (int a = 0; a < DIM; ++a) {
                const int nf = (int)(top.g.N + (a == DIM - 1 ? top.g.NP : 0));
                const float* src = A.lv[lt].bf[a];
                constexpr int U = 4;  // loads in flight per thread before the stores
                for (int c0 = t0; c0 < nf; c0 += U * nt) {
                    float v[U];
#pragma unroll
                    for (int u = 0; u < U; ++u) v[u] = (c0 + u * nt < nf) ? __ldcg(src + c0 + u * nt) : 0.f;
#pragma unroll
                    for (int u = 0; u < U; ++u)
                        if (c0 + u * nt < nf) top.b[a][c0 + u * nt] = v[u];
                }
            }
        } else {
            const MGLevel F = A.lv[lt - 1];
            const float* fb[3] = {F.bf[0], F.bf[1], F.bf[2]};
            for (int t = t0; t < ntop; t += nt) ops::coef_restrict_at<LG, float, DIM>(F.g, top.g, fb, top.b, t);
        }
        __syncthreads();
        for (int l = lt + 1; l < nl; ++l) {
            const SmLevel f = sm_level<T, DIM>(A, sm, l - 1), c = sm_level<T, DIM>(A, sm, l);
            const float* fb[3] = {f.b[0], f.b[1], f.b[2]};
            const int n = (int)(c.g.N + c.g.NP);
            for (int t = t0; t < n; t += nt) ops::coef_restrict_at<LP, float, DIM>(f.g, c.g, fb, c.b, t);
            __syncthreads();
        }
    }
    // As in the grid-wide levels, a smoothed level starts with its red cells at
    // their first step from zero, written with its r (here on copying it in,
    // below by the restriction).  (The coarsest level is solved directly.)
    {
        const SmLevel top = sm_level<T, DIM>(A, sm, lt);
        const float* bt[3] = {top.b[0], top.b[1], top.b[2]};
        const float* src = A.lv[lt].r;
        const bool seed = lt < nl - 1;
        const int n = (int)top.g.N;
        constexpr int U = 8;  // loads in flight per thread before the first store
        for (int c0 = t0; c0 < n; c0 += U * nt) {
            float rv[U];
#pragma unroll
            for (int u = 0; u < U; ++u) rv[u] = (c0 + u * nt < n) ? __ldcg(src + c0 + u * nt) : 0.f;
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int c = c0 + u * nt;
                if (c < n) {
                    top.r[c] = rv[u];
                    if (seed) ops::coarse_start<LP, float, DIM>(top.g, bt, decode(top.g, c), c, rv[u], top.e);
                }
            }
        }
        __syncthreads();
    }
    for (int l = lt; l < nl - 1; ++l) {  // down
        const SmLevel L = sm_level<T, DIM>(A, sm, l), C = sm_level<T, DIM>(A, sm, l + 1);
        const float* bl[3] = {L.b[0], L.b[1], L.b[2]};
        const float* bc[3] = {C.b[0], C.b[1], C.b[2]};
        const int half = (int)(L.g.N / 2);
        for (int it = 0; it < A.npre; ++it)
            for (int col = 0; col < 2; ++col) {
                if (it == 0 && col == 0) continue;
                tail_pass<DIM>(L, bl, col, t0, nt, half);
                __syncthreads();
            }
        const float* const* cbp = (l + 1 < nl - 1) ? bc : nullptr;
        for (int t = t0; t < (int)C.g.N; t += nt)
            ops::resid_restrict_at<LP, float, DIM>(L.g, C.g, bl, L.e, L.r, C.r, C.e, t, cbp);
        __syncthreads();
    }
    {
        const SmLevel C = sm_level<T, DIM>(A, sm, nl - 1);
        const float* bc[3] = {C.b[0], C.b[1], C.b[2]};
        float* Asm = reinterpret_cast<float*>(sd + A.sm_A);
        if (!A.ainv && first) {
            __shared__ float shv;
            ops::coarse_invert_block<LP, float, DIM>(C.g, bc, Asm, reinterpret_cast<float*>(sd + A.sm_fct), &shv);
        }
        double* cs = sd + A.sm_bb;  // FP64 scratch of the solve: 3 x kMaxCoarse doubles (sm_bb, then sm_fct)
        ops::coarse_apply_block<LP, float, DIM>(C.g, bc, A.ainv ? A.ainv : Asm, C.r, C.e, cs, cs + kMaxCoarse,
                                                sd + A.sm_fct);
    }
    // up: in shared memory a separate prolongation pass is cheaper than
    // prolonging the neighbours of every red cell on the fly
    for (int l = nl - 2; l >= lt; --l) {
        const SmLevel L = sm_level<T, DIM>(A, sm, l), C = sm_level<T, DIM>(A, sm, l + 1);
        const float* bl[3] = {L.b[0], L.b[1], L.b[2]};
        const int half = (int)(L.g.N / 2);
        for (int c = t0; c < (int)L.g.N; c += nt) ops::prolong_at<LP, float, DIM>(L.g, C.g, C.e, L.e, c);
        __syncthreads();
        for (int it = 0; it < A.npost; ++it)
            for (int col = 0; col < 2; ++col) {
                tail_pass<DIM>(L, bl, col, t0, nt, half);
                __syncthreads();
            }
    }
    {
        const SmLevel top = sm_level<T, DIM>(A, sm, lt);
        float* dst = A.lv[lt].e;
        for (int c = t0; c < (int)top.g.N; c += nt) dst[c] = top.e[c];
    }
}

// One FP32 V-cycle on the correction equation A e = r from level 0 (levels
// 0 .. lt-1 by the executor's threads, the tail by one CTA), ending with
// p += e.  Every grid-wide level starts with its red cells already at their
// first smoothing step from zero (written with r: by resid_local on level 0,
// by the restriction above), and the first smoothing step after the
// coarse-grid correction reads the black neighbours with the prolongation
// added on the fly, so neither e = 0 nor the prolonged e is ever stored: two
// grid barriers fewer per level.
template <typename T, int DIM, class X>
__device__ bool vcycle(const InstArgs<T>& A, X& x, bool first, float* sm) {
    using L_ = typename X::Ld;
    const int tid = x.tid(), nth = x.nth();
    for (int l = 0; l < A.lt; ++l) {
        const MGLevel L = A.lv[l];
        const MGLevel C = A.lv[l + 1];
        const float* bl[3] = {L.bf[0], L.bf[1], L.bf[2]};
        const int half = (int)(L.g.N / 2);
        for (int it = 0; it < A.npre; ++it)
            for (int col = 0; col < 2; ++col) {
                if (it == 0 && col == 0) continue;  // written with this level's r
                ops::colour_pass(
                    tid, half, nth,
                    [&](int k, long& c) {
                        c = ops::colour_cell(L.g, col, k);
                        return l == 0 ? ops::rbgs_rho_val<L_, DIM>(L.g, L.rho0, L.e, L.r, c)
                                      : ops::rbgs_val<L_, float, DIM>(L.g, bl, L.e, L.r, c);
                    },
                    [&](long c, float v) { L.e[c] = v; });
                if (!x.sync()) return false;
            }
        // the tail starts its top level from zero itself
        const float* cb[3] = {C.bf[0], C.bf[1], C.bf[2]};
        const float* const* cbp = (l + 1 < A.lt) ? cb : nullptr;
        for (int t = tid; t < (int)C.g.N; t += nth) {
            if (l == 0) ops::resid_restrict_rho_at<L_, DIM>(L.g, C.g, L.rho0, L.e, L.r, C.r, C.e, t, cbp);
            else ops::resid_restrict_at<L_, float, DIM>(L.g, C.g, bl, L.e, L.r, C.r, C.e, t, cbp);
        }
        if (!x.sync()) return false;
    }
    if (x.tail_cta()) tail_vcycle<T, DIM>(A, first, sm);
    if (!x.sync()) return false;
    const MGLevel L0 = A.lv[0];
    PT<T>* P0 = ops::pbuf<T>(L0);
    bool updated = false;
    for (int l = A.lt - 1; l >= 0; --l) {
        const MGLevel L = A.lv[l];
        const MGLevel C = A.lv[l + 1];
        const float* bl[3] = {L.bf[0], L.bf[1], L.bf[2]};
        const int half = (int)(L.g.N / 2);
        for (int it = 0; it < A.npost; ++it)
            for (int col = 0; col < 2; ++col) {
                const bool last = (l == 0 && it == A.npost - 1 && col == 1);
                const bool pro = (it == 0 && col == 0);
                ops::colour_pass(
                    tid, half, nth,
                    [&](int k, long& c) {
                        c = ops::colour_cell(L.g, col, k);
                        if (pro)
                            return l == 0 ? ops::rbgs_rho_val<L_, DIM, ops::kNbProlong>(L.g, L.rho0, L.e, L.r, c,
                                                                                      &C.g, C.e)
                                          : ops::rbgs_val<L_, float, DIM, ops::kNbProlong>(L.g, bl, L.e, L.r, c,
                                                                                         &C.g, C.e);
                        return l == 0 ? ops::rbgs_rho_val<L_, DIM>(L.g, L.rho0, L.e, L.r, c)
                                      : ops::rbgs_val<L_, float, DIM>(L.g, bl, L.e, L.r, c);
                    },
                    [&](long c, float v) {
                        L.e[c] = v;
                        if (last) P0[c] = ops::p_add(L_::ld(P0 + c), v);
                    });
                if (last) {  // the other colour is final already
                    for (int k = tid; k < half; k += nth) {
                        const long c = ops::colour_cell(L.g, 0, k);
                        P0[c] = ops::p_add(L_::ld(P0 + c), L_::ld(L.e + c));
                    }
                    updated = true;
                }
                if (!x.sync()) return false;
            }
    }
    if (!updated) {
        for (int c = tid; c < (int)L0.g.N; c += nth) P0[c] = ops::p_add(L_::ld(P0 + c), L_::ld(L0.e + c));
        if (!x.sync()) return false;
    }
    return true;
}

// residual of level 0 in the form's precision: this thread's part of its
// squared norm, the FP32 copy r, and on the red cells the first smoothing
// step of the next V-cycle from zero (rbgs_rho_at with kNbZero)
template <class Ld, typename T, int DIM>
__device__ double resid_local(const MGLevel& L0, float2 fmean, int tid, int nth) {
    const PT<T>* p = ops::pbuf<T>(L0);
    const FT<T>* f = ops::fbuf<T>(L0);
    T acc = T(0);
    for (int c = tid; c < (int)L0.g.N; c += nth) {
        const T r = ops::resid_form_at<Ld, DIM>(L0, p, f, fmean, c);
        const float rf = (float)r;
        L0.r[c] = rf;
        const IJK q = decode(L0.g, c);
        if (((q.i + q.j + q.k) & 1) == 0) {
            float diag, off;
            ops::stencil_L_rho<Ld, DIM>(L0.g, L0.rho0, q, c, L0.g.ih2f, [](long) { return 0.f; }, diag, off);
            L0.e[c] = ops::step_div(off - rf, diag);
        }
        acc += r * r;
    }
    return (double)acc;
}

template <class X>
__device__ void set_status(X& x, InstStats* S, int st) {
    if (x.leader()) atomicCAS(&S->status, 0, st);
}

// projection: f = div u*/(c dt) - mean, defect correction to tol,
// u = u* - c dt grad p / rho_f
template <typename T, int DIM, class X>
__device__ bool project(const InstArgs<T>& A, X& x, InstStats* S, const T* phi, T* const* u, double cdt, float* sm,
                        int stage, long sg) {
    using L_ = typename X::Ld;
    const Geom& g = A.g;
    const int tid = x.tid(), nth = x.nth();
    const MGLevel L0 = A.lv[0];
    PT<T>* P0 = ops::pbuf<T>(L0);
    FT<T>* F0 = ops::fbuf<T>(L0);
    const T ih = g_ih<T>(g), inv_cdt = (T)(1.0 / cdt);
    const T* uc[3] = {u[0], u[1], u[2]};
    ops::SumAcc<T> s;
    for (int c = tid; c < (int)g.N; c += nth) {
        const T v = ops::div_at<L_, T, DIM>(g, uc, ih, inv_cdt, c);
        F0[c] = v;
        s.add(v);
    }
    double sum;
    if (!x.template reduce<false>(s.value(), sum)) return false;
    const double mean = sum / (double)g.N;
    // FP64 form: f is centred in place; FP32-mixed form: the residual removes the mean
    const float2 fmean = ops::dfl::from_double(mean);
    T s2 = T(0);
    // first guess: zero, the last solve's pressure, or the same RK stage of the
    // last two steps extrapolated linearly in time (2 p_(n-1) - p_(n-2))
    const bool extrap = (A.warm == CDI_WARM_EXTRAP);
    const PT<T>* hnew = extrap ? reinterpret_cast<const PT<T>*>(A.hist[stage][(sg - 1) & 1]) : nullptr;
    const PT<T>* hold = extrap ? reinterpret_cast<const PT<T>*>(A.hist[stage][sg & 1]) : nullptr;
    for (int c = tid; c < (int)g.N; c += nth) {
        T v;
        if constexpr (sizeof(T) == 8) {
            v = L_::ld(F0 + c) - mean;
            F0[c] = v;
        } else {
            v = (L_::ld(F0 + c) - fmean.x) - fmean.y;
        }
        s2 += v * v;
        if (A.warm == CDI_WARM_ZERO) P0[c] = ops::p_zero<T>();
        else if (extrap && sg >= 2) P0[c] = ops::p_extrap(L_::ld(hnew + c), L_::ld(hold + c));
    }
    for (int t = tid; t < (int)(g.N + g.NP); t += nth)
        ops::coef0_at<L_, T, DIM>(g, A.ph, phi, L0.beta, L0.bf, L0.rho0, t);
    double fsq;
    if (!x.template reduce<false>((double)s2, fsq)) return false;
    const double fn = sqrt(fsq);
    for (int l = 1; l < A.lt; ++l) {
        const MGLevel F = A.lv[l - 1];
        const MGLevel C = A.lv[l];
        const float* fb[3] = {F.bf[0], F.bf[1], F.bf[2]};
        for (int t = tid; t < (int)(C.g.N + C.g.NP); t += nth)
            ops::coef_restrict_at<L_, float, DIM>(F.g, C.g, fb, C.bf, t);
        if (!x.sync()) return false;
    }
    double rsq;
    if (!x.template reduce<false>(resid_local<L_, T, DIM>(L0, fmean, tid, nth), rsq)) return false;
    double rn = sqrt(rsq);
    if (!isfinite(fn) || !isfinite(rn)) {
        set_status(x, S, CDI_ENAN);
        return false;
    }
    int cyc = 0;
    PT<T>* hput = extrap ? reinterpret_cast<PT<T>*>(A.hist[stage][sg & 1]) : nullptr;
    if (fn == 0.0) {
        for (int c = tid; c < (int)g.N; c += nth) {
            P0[c] = ops::p_zero<T>();
            if (extrap) hput[c] = ops::p_zero<T>();
        }
        if (!x.sync()) return false;
    } else {
        bool first = true;
        while (rn > A.tol * fn && cyc < A.max_vcycles) {
            if (!vcycle<T, DIM>(A, x, first, sm)) return false;
            first = false;
            if (!x.template reduce<false>(resid_local<L_, T, DIM>(L0, fmean, tid, nth), rsq)) return false;
            rn = sqrt(rsq);
            ++cyc;
            if (!isfinite(rn)) {
                set_status(x, S, CDI_ENAN);
                return false;
            }
        }
        if (rn > A.tol * fn) {
            set_status(x, S, CDI_ENOCONV);
            if (x.leader()) {
                S->last_cycles = cyc;
                S->last_resid = rn / fn;
            }
            return false;
        }
        double ps;
        if constexpr (sizeof(T) == 8) {
            ps = 0.0;
            for (int c = tid; c < (int)g.N; c += nth) ps += L_::ld(P0 + c);
        } else {
            float2 a = make_float2(0.f, 0.f);
            for (int c = tid; c < (int)g.N; c += nth) a = ops::dfl::add(a, L_::ld(P0 + c));
            ps = ops::dfl::to_double(a);
        }
        double psum;
        if (!x.template reduce<false>(ps, psum)) return false;
        const double pmean = psum / (double)g.N;
        const float2 pm2 = ops::dfl::from_double(pmean);
        for (int c = tid; c < (int)g.N; c += nth) {
            const PT<T> v = ops::p_sub(L_::ld(P0 + c), pmean, pm2);
            P0[c] = v;
            if (extrap) hput[c] = v;
        }
        if (!x.sync()) return false;
    }
    if (x.leader()) {
        S->last_cycles = cyc;
        S->last_resid = fn == 0.0 ? 0.0 : rn / fn;
        S->total_cycles += cyc;
        if (cyc > S->max_cycles) S->max_cycles = cyc;
    }
    for (int c = tid; c < (int)g.N; c += nth) ops::project_at<L_, T, DIM>(g, A.ph, phi, u, (T)cdt, P0, c);
    return x.sync();
}

// nsteps RK4 steps of one instance; the state pointers swap once per step
template <typename T, int DIM, class X>
__device__ void run_steps(const InstArgs<T>& A, X& x, int nsteps, InstStats* S, float* sm) {
    using L_ = typename X::Ld;
    const Geom& g = A.g;
    const int tid = x.tid(), nth = x.nth();
    T* phi_s = A.phi_s;
    T* phi_k = A.phi_k;
    T* u_s[3] = {A.u_s[0], A.u_s[1], A.u_s[2]};
    T* u_k[3] = {A.u_k[0], A.u_k[1], A.u_k[2]};
    const double ck[4] = {0.0, 0.5, 0.5, 1.0};
    const double bk[4] = {1.0 / 6.0, 1.0 / 3.0, 1.0 / 3.0, 1.0 / 6.0};
    for (int step = 0; step < nsteps; ++step) {
        double gamma = A.gamma_param;
        if (gamma < 0.0) {  // gamma = 2.5 |u|_max, floored (Sec. 5.1)
            T mx = T(0);
            for (int a = 0; a < DIM; ++a) {
                const int nf = (int)(g.N + (a == DIM - 1 ? g.NP : 0));
                for (int c = tid; c < nf; c += nth) mx = fmax(mx, fabs(L_::ld(u_s[a] + c)));
            }
            double umax;
            if (!x.template reduce<true>((double)mx, umax)) return;
            gamma = fmax(2.5 * umax, -A.gamma_param);
        }
        for (int st = 0; st < 4; ++st) {
            T* phi = st == 0 ? phi_s : phi_k;
            T* const* u = st == 0 ? u_s : u_k;
            StageFields<T> f{};
            f.phi = phi;
            for (int a = 0; a < 3; ++a) {
                f.u[a] = u[a];
                f.nh[a] = A.nh[a];
                f.m[a] = A.m[a];
                f.rm[a] = A.rm[a];
            }
            f.psi = A.psi;
            f.muc = A.muc;
            f.rphi = A.rphi;
            f.wuY = A.wuY;
            f.wghost = A.wghost;
            f.wmuw = A.wmuw;
            for (int c = tid; c < (int)g.N; c += nth) ops::psi_at<L_>(g, A.ph, phi, A.psi, c);
            if (!x.sync()) return;
            // Wall columns are spread over the CTAs (column w on CTA w mod CTAs: each
            // is FP64-heavy, and a grid-stride loop would give them all to the first
            // CTAs); their extrapolated quantities are formed once per column here,
            // and the slip and ghost values, which two adjacent columns combine into,
            // in the next phase (phi_rhs does not read them).
            ops::ColQ<T>* colq = reinterpret_cast<ops::ColQ<T>*>(A.colq);
            for (int c = tid; c < (int)g.N; c += nth)
                ops::cell_at<L_, T, DIM>(g, A.ph, phi, A.psi, A.nh[0], A.nh[1], A.nh[2], A.muc, c);
            for (int t = x.spread(); t < (int)(2 * g.NP); t += nth)
                ops::wall_colq_at<L_, T, DIM>(g, A.ph, phi, A.psi, colq, t);
            if (!x.sync()) return;
            for (int c = tid; c < (int)g.N; c += nth) ops::phi_rhs_at<L_, T, DIM>(g, A.ph, f, (T)gamma, c);
            for (int t = x.spread(); t < (int)(2 * g.NP); t += nth)
                ops::wall_from_colq_at<L_, T, DIM>(g, A.ph, colq, u[0], u[1], A.wuY, A.wghost, A.wmuw, t);
            if (!x.sync()) return;
            for (int c = tid; c < (int)g.N; c += nth) ops::mom_at<L_, T, DIM>(g, A.ph, f, c);
            if (!x.sync()) return;
            const int first = st == 0, last = st == 3;
            const double cn = last ? 1.0 : ck[st + 1];
            const T b = (T)bk[st], cdt = (T)(cn * A.dt), dt = (T)A.dt;
            for (int c = tid; c < (int)g.N; c += nth)
                ops::stage_phi_at<L_>(b, cdt, dt, first, last, phi_s, A.rphi, A.acc_phi, phi_k, c);
            if (!x.sync()) return;
            const T* u0c[3] = {u_s[0], u_s[1], u_s[2]};
            const T* rmc[3] = {A.rm[0], A.rm[1], A.rm[2]};
            T* accm[3] = {A.acc_m[0], A.acc_m[1], A.acc_m[2]};
            for (int c = tid; c < (int)g.N; c += nth)
                ops::stage_mom_at<L_, T, DIM>(g, A.ph, b, cdt, dt, first, last, phi_s, phi_k, u0c, rmc, accm, u_k, c);
            if (!x.sync()) return;
            if (!project<T, DIM>(A, x, S, phi_k, u_k, cn * A.dt, sm, st, A.hist_step0 + step)) return;
        }
        T* tp = phi_s;
        phi_s = phi_k;
        phi_k = tp;
        for (int a = 0; a < 3; ++a) {
            T* tu = u_s[a];
            u_s[a] = u_k[a];
            u_k[a] = tu;
        }
        if (x.leader()) S->steps_done = step + 1;
    }
}

template <typename T, int DIM>
__global__ void __launch_bounds__(kPersistThreads, 1) k_step_persist(PersistArgs<T> P) {
    extern __shared__ double smd[];
    float* sm = reinterpret_cast<float*>(smd);
    GridX x{P.ctl, P.partials, P.spin_limit, 0, 0ull};
    run_steps<T, DIM>(P.I, x, P.nsteps, &P.ctl->st, sm);
}

template <typename T, int DIM, int NT>
__global__ void __launch_bounds__(NT, 1) k_batch_persist(BatchArgs<T> B) {
    extern __shared__ double smd[];
    float* sm = reinterpret_cast<float*>(smd);
    __shared__ int s_inst;
    __shared__ __align__(16) InstArgs<T> sA;
    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) s_inst = atomicAdd(B.counter, 1);
        __syncthreads();
        const int i = s_inst;
        if (i >= B.n_inst) return;
        // the instance descriptor into shared memory (16-byte words)
        const int4* src = reinterpret_cast<const int4*>(B.insts + i);
        int4* dst = reinterpret_cast<int4*>(&sA);
        for (int w = threadIdx.x; w < (int)(sizeof(InstArgs<T>) / sizeof(int4)); w += blockDim.x) dst[w] = src[w];
        __syncthreads();
        BlockX x;
        run_steps<T, DIM>(sA, x, B.nsteps, B.stats + i, sm);
    }
}

}  // namespace

// shared-memory layout of the FP32 tail levels and the FP64 dense-solve scratch; returns bytes
size_t persist_tail_layout(const Geom& g, const MG& mg, int lt, PersistLayout& L) {
    long off = 0;  // floats
    for (int l = lt; l < mg.nlev; ++l) {
        const Geom& v = mg.lv[l].g;
        L.sm_e[l] = off;
        off += v.N;
        L.sm_r[l] = off;
        off += v.N;
        for (int a = 0; a < 3; ++a) {
            L.sm_b[l][a] = off;
            if (a < g.D) off += v.N + (a == g.W ? v.NP : 0);
        }
    }
    off = (off + 1) & ~1L;  // 8-byte alignment for the double scratch
    L.sm_dbl = off;
    long d = 0;  // doubles
    L.sm_A = d;
    d += (long)kMaxCoarse * kMaxCoarse;
    L.sm_bb = d;
    d += 2 * kMaxCoarse;
    L.sm_fct = d;
    d += kMaxCoarse;
    return (size_t)off * sizeof(float) + (size_t)d * sizeof(double);
}

// One V-cycle's shared-memory tail as its own single-CTA launch (the
// launch-per-kernel path): levels lt .. nlev-1 of the descriptor, the tail
// coefficients restricted afresh each launch (shared memory does not outlive it)
template <int DIM>
__global__ void __launch_bounds__(kPersistThreads, 1) k_tail(const InstArgs<float>* A) {
    extern __shared__ double smd[];
    tail_vcycle<float, DIM>(*A, true, reinterpret_cast<float*>(smd));
}

cudaError_t tail_prepare(int dim, size_t smem) {
    const void* fn = (dim == 2) ? (const void*)k_tail<2> : (const void*)k_tail<3>;
    return cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}

cudaError_t launch_tail(const void* inst_args, int dim, size_t smem, cudaStream_t s) {
    const InstArgs<float>* A = static_cast<const InstArgs<float>*>(inst_args);
    if (dim == 2) k_tail<2><<<1, kPersistThreads, smem, s>>>(A);
    else k_tail<3><<<1, kPersistThreads, smem, s>>>(A);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_step_persist(PersistArgs<T>& A, size_t smem, int grid, cudaStream_t s) {
    void* args[] = {&A};
    const void* fn = (A.I.g.D == 2) ? (const void*)k_step_persist<T, 2> : (const void*)k_step_persist<T, 3>;
    return cudaLaunchCooperativeKernel(fn, dim3(grid), dim3(kPersistThreads), args, smem, s);
}

template <typename T>
cudaError_t persist_prepare(int dim, size_t smem, int* grid) {
    const void* fn = (dim == 2) ? (const void*)k_step_persist<T, 2> : (const void*)k_step_persist<T, 3>;
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int dev = 0, nsm = 0, per = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, fn, kPersistThreads, smem)) != cudaSuccess) return e;
    if (per < 1) return cudaErrorInvalidConfiguration;
    *grid = nsm;  // one CTA per SM
    return cudaSuccess;
}

template <typename T, int NT>
static const void* batch_fn(int dim) {
    return (dim == 2) ? (const void*)k_batch_persist<T, 2, NT> : (const void*)k_batch_persist<T, 3, NT>;
}
template <typename T>
static const void* batch_fn_threads(int dim, int threads) {
    switch (threads) {
        case 256: return batch_fn<T, 256>(dim);
        case 1024: return batch_fn<T, 1024>(dim);
        default: return batch_fn<T, 512>(dim);
    }
}

template <typename T>
cudaError_t batch_prepare(int dim, int threads, size_t smem, int* grid) {
    const void* fn = batch_fn_threads<T>(dim, threads);
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int dev = 0, nsm = 0, per = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, fn, threads, smem)) != cudaSuccess) return e;
    if (per < 1) return cudaErrorInvalidConfiguration;
    *grid = nsm * per;
    return cudaSuccess;
}

template <typename T>
cudaError_t launch_batch_persist(BatchArgs<T>& B, int dim, int threads, size_t smem, int grid, cudaStream_t s) {
    void* args[] = {&B};
    return cudaLaunchKernel(batch_fn_threads<T>(dim, threads), dim3(grid), dim3(threads), args, smem, s);
}

template cudaError_t launch_step_persist<double>(PersistArgs<double>&, size_t, int, cudaStream_t);
template cudaError_t launch_step_persist<float>(PersistArgs<float>&, size_t, int, cudaStream_t);
template cudaError_t persist_prepare<double>(int, size_t, int*);
template cudaError_t persist_prepare<float>(int, size_t, int*);
template cudaError_t batch_prepare<double>(int, int, size_t, int*);
template cudaError_t batch_prepare<float>(int, int, size_t, int*);
template cudaError_t launch_batch_persist<double>(BatchArgs<double>&, int, int, size_t, int, cudaStream_t);
template cudaError_t launch_batch_persist<float>(BatchArgs<float>&, int, int, size_t, int, cudaStream_t);

}  // namespace cdi
