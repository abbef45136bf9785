// Pressure projection, geometric multigrid and fixed-order reductions.
//
//   k_div            f = div u* / (c dt)                                   Eq. (NS_incompressibility)
//   k_sub_mean_sq    remove the mean of f (compatibility with the walls' and
//                    periodic sides' zero net flux), accumulate |f|^2
//   k_coef0          face coefficients 1/rho_f, rho_f the mean of the two   Sec. 2 (rho linear in phi)
//                    adjacent cells, zero on the walls (Neumann)
//   k_rbgs           red-black Gauss-Seidel sweep of div(beta grad p) = f
//   k_resid_restrict residual and its restriction (mean of the 2^D children)
//   k_prolong        cell-centred (bi/tri)linear prolongation, wall reflection
//   k_coarse         dense direct solve of the coarsest level in one CTA
//   k_project        u = u* - c dt grad p / rho_f on every interior face     Eq. (no-penetration BC)
//   k_mass, k_umax, k_contact_line: FP64 reductions                          Sec. 2, 3.1, 5.1
//
// Every sum is deterministic: a fixed grid of at most kPartials blocks, a
// fixed per-thread stride, a warp-shuffle tree per block and one final block.
#include "cdi_internal.cuh"

#include <algorithm>
#include <cmath>

namespace cdi {

namespace {

constexpr int kThreads = 256;
inline unsigned blocks_for(long n) { return (unsigned)((n + kThreads - 1) / kThreads); }
inline unsigned red_blocks(long n) { return (unsigned)std::max(1L, std::min((long)kPartials, (n + kThreads - 1) / kThreads)); }

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

Geom level_geom(const Geom& g, const MGLevel& L) {
    Geom lg = g;
    for (int b = 0; b < 3; ++b) lg.n[b] = L.n[b];
    lg.N = L.N;
    lg.NP = L.NP;
    lg.h = L.h;
    return lg;
}

// final pass of a sum: out = scale * sum(partials[0..np))
__global__ void k_final_sum(const double* __restrict__ part, int np, double scale, double* __restrict__ out,
                            int do_sqrt) {
    double v = 0.0;
    for (int t = threadIdx.x; t < np; t += blockDim.x) v += part[t];
    v = block_sum(v);
    if (threadIdx.x == 0) {
        double r = v * scale;
        *out = do_sqrt ? sqrt(r) : r;
    }
}

template <typename T, int DIM>
__global__ void k_div(Geom g, const T* __restrict__ u0, const T* __restrict__ u1, const T* __restrict__ u2,
                      double inv_cdt, double* __restrict__ f, double* __restrict__ part) {
    const T* us[3] = {u0, u1, u2};
    const double ih = 1.0 / g.h;
    double acc = 0.0;
    const long stride = (long)gridDim.x * blockDim.x;
    for (long c = (long)blockIdx.x * blockDim.x + threadIdx.x; c < g.N; c += stride) {
        const IJK q = decode(g, c);
        double div = 0.0;
#pragma unroll
        for (int a = 0; a < DIM; ++a) {
            const long hi = (a == DIM - 1) ? c + g.NP : idx(g, shift(g, q, a, 1));
            div += (double)us[a][hi] - (double)us[a][c];
        }
        const double v = div * ih * inv_cdt;
        f[c] = v;
        acc += v;
    }
    acc = block_sum(acc);
    if (threadIdx.x == 0) part[blockIdx.x] = acc;
}

__global__ void k_sub_mean_sq(long N, double* __restrict__ f, const double* __restrict__ sum,
                              double* __restrict__ part) {
    const double mean = *sum / (double)N;
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

template <typename T, int DIM>
__global__ void k_coef0(Geom g, double rho1, double rho2, const T* __restrict__ phi, double* __restrict__ b0,
                        double* __restrict__ b1, double* __restrict__ b2) {
    double* bs[3] = {b0, b1, b2};
    long c = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= g.N + g.NP) return;
    if (c >= g.N) {  // top wall plane of the wall-normal coefficients
        bs[DIM - 1][c] = 0.0;
        return;
    }
    const IJK q = decode(g, c);
    const double dr = rho1 - rho2;
#pragma unroll
    for (int a = 0; a < DIM; ++a) {
        if (a == DIM - 1 && coord(q, a) == 0) { bs[a][c] = 0.0; continue; }
        const long cL = idx(g, shift(g, q, a, -1));
        const double rf = 0.5 * ((dr * (double)phi[cL] + rho2) + (dr * (double)phi[c] + rho2));
        bs[a][c] = 1.0 / rf;
    }
}

// coarse face coefficient = mean of the 2^(D-1) fine faces covering it
template <int DIM>
__global__ void k_coef_restrict(Geom gf, Geom gc, const double* __restrict__ f0, const double* __restrict__ f1,
                                const double* __restrict__ f2, double* __restrict__ c0, double* __restrict__ c1,
                                double* __restrict__ c2) {
    const double* fb[3] = {f0, f1, f2};
    double* cb[3] = {c0, c1, c2};
    long t = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= gc.N + gc.NP) return;
    // faces of every component at this linear index (the wall-normal one has an extra plane)
    IJK q = decode(gc, t < gc.N ? t : t - gc.NP);
    if (t >= gc.N) setc(q, DIM - 1, gc.n[DIM - 1]);
#pragma unroll
    for (int a = 0; a < DIM; ++a) {
        if (t >= gc.N && a != DIM - 1) continue;
        int other[2], no = 0;
        for (int b = 0; b < DIM; ++b)
            if (b != a) other[no++] = b;
        const int o2 = (DIM == 3) ? 2 : 1;
        double sum = 0.0;
        int cnt = 0;
        for (int t2 = 0; t2 < o2; ++t2)
            for (int t1 = 0; t1 < 2; ++t1) {
                IJK qf;
                qf.i = 2 * q.i;
                qf.j = 2 * q.j;
                qf.k = (DIM == 3) ? 2 * q.k : 0;
                setc(qf, other[0], coord(qf, other[0]) + t1);
                if (DIM == 3) setc(qf, other[1], coord(qf, other[1]) + t2);
                sum += fb[a][idx(gf, qf)];
                ++cnt;
            }
        cb[a][idx(gc, q)] = sum / cnt;
    }
}

template <int DIM>
__device__ __forceinline__ double apply_L(const Geom& g, const double* const* beta, const double* __restrict__ p,
                                          const IJK& q, long c, double ih2, double& diag, double& off) {
    diag = 0.0;
    off = 0.0;
#pragma unroll
    for (int a = 0; a < DIM; ++a) {
        const long hi = (a == DIM - 1) ? c + g.NP : idx(g, shift(g, q, a, 1));
        const double bm = beta[a][c];
        const double bp = beta[a][hi];
        const double pm = (bm != 0.0) ? p[idx(g, shift(g, q, a, -1))] : 0.0;
        const double pp = (bp != 0.0) ? p[(a == DIM - 1) ? c + g.NP : hi] : 0.0;
        diag += (bm + bp) * ih2;
        off += (bm * pm + bp * pp) * ih2;
    }
    return off - diag * p[c];
}

template <int DIM>
__global__ void k_rbgs(Geom g, const double* __restrict__ b0, const double* __restrict__ b1,
                       const double* __restrict__ b2, double* __restrict__ p, const double* __restrict__ f,
                       int colour) {
    const double* beta[3] = {b0, b1, b2};
    long c = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= g.N) return;
    const IJK q = decode(g, c);
    if (((q.i + q.j + q.k) & 1) != colour) return;
    const double ih2 = 1.0 / (g.h * g.h);
    double diag, off;
    apply_L<DIM>(g, beta, p, q, c, ih2, diag, off);
    p[c] = (off - f[c]) / diag;
}

template <int DIM>
__global__ void k_resid_restrict(Geom gf, Geom gc, const double* __restrict__ b0, const double* __restrict__ b1,
                                 const double* __restrict__ b2, const double* __restrict__ p,
                                 const double* __restrict__ f, double* __restrict__ fc, double* __restrict__ pc) {
    const double* beta[3] = {b0, b1, b2};
    long t = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= gc.N) return;
    const IJK Q = decode(gc, t);
    const double ih2 = 1.0 / (gf.h * gf.h);
    const int o2 = (DIM == 3) ? 2 : 1;
    double s = 0.0;
    for (int t2 = 0; t2 < o2; ++t2)
        for (int t1 = 0; t1 < 2; ++t1)
            for (int t0 = 0; t0 < 2; ++t0) {
                IJK q;
                q.i = 2 * Q.i + t0;
                q.j = 2 * Q.j + t1;
                q.k = (DIM == 3) ? 2 * Q.k + t2 : 0;
                const long c = idx(gf, q);
                double diag, off;
                const double Lp = apply_L<DIM>(gf, beta, p, q, c, ih2, diag, off);
                s += f[c] - Lp;
            }
    fc[t] = s * (1.0 / (4 * o2));
    pc[t] = 0.0;
}

template <int DIM>
__global__ void k_prolong(Geom gf, Geom gc, const double* __restrict__ pc, double* __restrict__ p) {
    long c = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= gf.N) return;
    const IJK q = decode(gf, c);
    int I[3][2];
    double w[3][2];
#pragma unroll
    for (int b = 0; b < 3; ++b) {
        if (b >= DIM) { I[b][0] = I[b][1] = 0; w[b][0] = 1.0; w[b][1] = 0.0; continue; }
        const int qb = coord(q, b);
        const int P = qb / 2;
        int nb = (qb % 2 == 0) ? P - 1 : P + 1;
        if (b == DIM - 1) nb = min(max(nb, 0), gc.n[b] - 1);
        else { if (nb < 0) nb += gc.n[b]; else if (nb >= gc.n[b]) nb -= gc.n[b]; }
        I[b][0] = P;
        I[b][1] = nb;
        w[b][0] = 0.75;
        w[b][1] = 0.25;
    }
    double s = 0.0;
    for (int t2 = 0; t2 < 2; ++t2)
        for (int t1 = 0; t1 < 2; ++t1)
            for (int t0 = 0; t0 < 2; ++t0) {
                const double wv = w[0][t0] * w[1][t1] * w[2][t2];
                if (wv == 0.0) continue;
                s += wv * pc[encode(gc, I[0][t0], I[1][t1], I[2][t2])];
            }
    p[c] += s;
}

// Dense direct solve of (L + c 1 1^T) p = f on the coarsest level (at most
// kMaxCoarse cells): Gaussian elimination with partial pivoting in one CTA.
template <int DIM>
__global__ void k_coarse(Geom g, const double* __restrict__ b0, const double* __restrict__ b1,
                         const double* __restrict__ b2, const double* __restrict__ f, double* __restrict__ p) {
    const double* beta[3] = {b0, b1, b2};
    __shared__ double A[kMaxCoarse * kMaxCoarse];
    __shared__ double bb[kMaxCoarse];
    __shared__ double diagv[kMaxCoarse];
    __shared__ int piv_s;
    __shared__ double shift_s;
    const int n = (int)g.N;
    const double ih2 = 1.0 / (g.h * g.h);
    for (int t = threadIdx.x; t < n * n; t += blockDim.x) A[t] = 0.0;
    __syncthreads();
    if (threadIdx.x == 0) {
        // rows in cell order (neighbours of a periodic extent 2 coincide and add up)
        double dsum = 0.0;
        for (int c = 0; c < n; ++c) {
            const IJK q = decode(g, c);
            for (int a = 0; a < DIM; ++a) {
                const long hi = (a == DIM - 1) ? c + g.NP : idx(g, shift(g, q, a, 1));
                const double bm = beta[a][c], bp = beta[a][hi];
                A[c * n + c] -= (bm + bp) * ih2;
                if (bm != 0.0) A[c * n + idx(g, shift(g, q, a, -1))] += bm * ih2;
                if (bp != 0.0) A[c * n + ((a == DIM - 1) ? c + g.NP : hi)] += bp * ih2;
            }
            dsum += -A[c * n + c];
            bb[c] = f[c];
        }
        shift_s = -dsum / ((double)n * (double)n);
    }
    __syncthreads();
    for (int t = threadIdx.x; t < n * n; t += blockDim.x) A[t] += shift_s;
    __syncthreads();
    for (int col = 0; col < n; ++col) {
        if (threadIdx.x == 0) {
            int pv = col;
            for (int r = col + 1; r < n; ++r)
                if (fabs(A[r * n + col]) > fabs(A[pv * n + col])) pv = r;
            piv_s = pv;
        }
        __syncthreads();
        const int pv = piv_s;
        if (pv != col) {
            for (int t = threadIdx.x; t < n; t += blockDim.x) {
                double tmp = A[col * n + t];
                A[col * n + t] = A[pv * n + t];
                A[pv * n + t] = tmp;
            }
            if (threadIdx.x == 0) {
                double tmp = bb[col];
                bb[col] = bb[pv];
                bb[pv] = tmp;
            }
        }
        __syncthreads();
        for (int r = col + 1 + threadIdx.x; r < n; r += blockDim.x) {
            const double fct = A[r * n + col] / A[col * n + col];
            diagv[r] = fct;
        }
        __syncthreads();
        for (int r = col + 1 + threadIdx.x; r < n; r += blockDim.x) {
            const double fct = diagv[r];
            if (fct == 0.0) continue;
            for (int t = col; t < n; ++t) A[r * n + t] -= fct * A[col * n + t];
            bb[r] -= fct * bb[col];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        for (int r = n - 1; r >= 0; --r) {
            double s = bb[r];
            for (int t = r + 1; t < n; ++t) s -= A[r * n + t] * p[t];
            p[r] = s / A[r * n + r];
        }
    }
}

template <int DIM>
__global__ void k_resid_sq(Geom g, const double* __restrict__ b0, const double* __restrict__ b1,
                           const double* __restrict__ b2, const double* __restrict__ p,
                           const double* __restrict__ f, double* __restrict__ part) {
    const double* beta[3] = {b0, b1, b2};
    const double ih2 = 1.0 / (g.h * g.h);
    double acc = 0.0;
    const long stride = (long)gridDim.x * blockDim.x;
    for (long c = (long)blockIdx.x * blockDim.x + threadIdx.x; c < g.N; c += stride) {
        const IJK q = decode(g, c);
        double diag, off;
        const double r = f[c] - apply_L<DIM>(g, beta, p, q, c, ih2, diag, off);
        acc += r * r;
    }
    acc = block_sum(acc);
    if (threadIdx.x == 0) part[blockIdx.x] = acc;
}

__global__ void k_partial_sum(long N, const double* __restrict__ x, double* __restrict__ part) {
    double acc = 0.0;
    const long stride = (long)gridDim.x * blockDim.x;
    for (long c = (long)blockIdx.x * blockDim.x + threadIdx.x; c < N; c += stride) acc += x[c];
    acc = block_sum(acc);
    if (threadIdx.x == 0) part[blockIdx.x] = acc;
}

__global__ void k_sub_scalar(long N, double* __restrict__ x, const double* __restrict__ sum) {
    const double mean = *sum / (double)N;
    long c = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (c < N) x[c] -= mean;
}

template <typename T, int DIM>
__global__ void k_project(Geom g, double rho1, double rho2, const T* __restrict__ phi, T* __restrict__ u0,
                          T* __restrict__ u1, T* __restrict__ u2, double cdt, const double* __restrict__ p) {
    T* us[3] = {u0, u1, u2};
    long c = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= g.N) return;
    const IJK q = decode(g, c);
    const double ih = 1.0 / g.h, dr = rho1 - rho2;
#pragma unroll
    for (int a = 0; a < DIM; ++a) {
        if (a == DIM - 1 && coord(q, a) == 0) continue;  // wall face stays zero
        const long cL = idx(g, shift(g, q, a, -1));
        const double rf = 0.5 * ((dr * (double)phi[cL] + rho2) + (dr * (double)phi[c] + rho2));
        const double beta = 1.0 / rf;
        const double dp = (p[c] - p[cL]) * ih;
        us[a][c] = (T)((double)us[a][c] - cdt * beta * dp);
    }
}

template <typename T>
__global__ void k_mass_partial(long N, const T* __restrict__ phi, double* __restrict__ part) {
    double acc = 0.0;
    const long stride = (long)gridDim.x * blockDim.x;
    for (long c = (long)blockIdx.x * blockDim.x + threadIdx.x; c < N; c += stride) acc += (double)phi[c];
    acc = block_sum(acc);
    if (threadIdx.x == 0) part[blockIdx.x] = acc;
}

template <typename T>
__global__ void k_umax_partial(long n0, long n1, long n2, const T* __restrict__ u0, const T* __restrict__ u1,
                               const T* __restrict__ u2, double* __restrict__ part) {
    double m = 0.0;
    const long stride = (long)gridDim.x * blockDim.x;
    for (long c = (long)blockIdx.x * blockDim.x + threadIdx.x; c < n0; c += stride) m = fmax(m, fabs((double)u0[c]));
    for (long c = (long)blockIdx.x * blockDim.x + threadIdx.x; c < n1; c += stride) m = fmax(m, fabs((double)u1[c]));
    for (long c = (long)blockIdx.x * blockDim.x + threadIdx.x; c < n2; c += stride) m = fmax(m, fabs((double)u2[c]));
    m = block_max(m);
    if (threadIdx.x == 0) part[blockIdx.x] = m;
}

__global__ void k_gamma_final(const double* __restrict__ part, int np, double floor_gamma,
                              double* __restrict__ umax, double* __restrict__ gamma) {
    double v = 0.0;
    for (int t = threadIdx.x; t < np; t += blockDim.x) v = fmax(v, part[t]);
    v = block_max(v);
    if (threadIdx.x == 0) {
        *umax = v;
        *gamma = fmax(2.5 * v, floor_gamma);
    }
}

// contact line on one wall from the wall-column arrays (phi_w, psi_w, d_n psi_w)
__global__ void k_contact_line(int D, int nx, int nlines, double h, const double* __restrict__ cols, long NP,
                               double* __restrict__ theta_out, double* __restrict__ wetted_out) {
    const double* phw = cols;
    const double* psw = cols + NP;
    const double* dnw = cols + 2 * NP;
    double th_sum = 0.0, cnt = 0.0, len_sum = 0.0;
    for (int line = threadIdx.x; line < nlines; line += blockDim.x) {
        const long base = (long)line * nx;
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
            double cv = -gn / sqrt(gn * gn + gt * gt);
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
    const unsigned G = red_blocks(g.N);
    if (g.D == 2)
        k_div<T, 2><<<G, kThreads, 0, s>>>(g, us[0], us[1], nullptr, inv_cdt, mg.lv[0].f, mg.partials);
    else
        k_div<T, 3><<<G, kThreads, 0, s>>>(g, us[0], us[1], us[2], inv_cdt, mg.lv[0].f, mg.partials);
    k_final_sum<<<1, 1024, 0, s>>>(mg.partials, (int)G, 1.0, mg.scal + S_MEAN, 0);
    g_launches += 2;
}

void launch_sum_f(const Geom& g, MG& mg, cudaStream_t s) {
    const unsigned G = red_blocks(g.N);
    k_partial_sum<<<G, kThreads, 0, s>>>(g.N, mg.lv[0].f, mg.partials);
    k_final_sum<<<1, 1024, 0, s>>>(mg.partials, (int)G, 1.0, mg.scal + S_MEAN, 0);
    g_launches += 2;
}

void launch_sub_mean_and_norm(const Geom& g, MG& mg, cudaStream_t s) {
    const unsigned G = red_blocks(g.N);
    k_sub_mean_sq<<<G, kThreads, 0, s>>>(g.N, mg.lv[0].f, mg.scal + S_MEAN, mg.partials);
    k_final_sum<<<1, 1024, 0, s>>>(mg.partials, (int)G, 1.0, mg.scal + S_FNORM, 1);
    g_launches += 2;
}

template <typename T>
void launch_mg_coef(const Geom& g, const PhysDev& ph, const T* phi, MG& mg, cudaStream_t s) {
    MGLevel& L0 = mg.lv[0];
    if (g.D == 2)
        k_coef0<T, 2><<<blocks_for(g.N + g.NP), kThreads, 0, s>>>(g, ph.rho1, ph.rho2, phi, L0.beta[0], L0.beta[1],
                                                                  nullptr);
    else
        k_coef0<T, 3><<<blocks_for(g.N + g.NP), kThreads, 0, s>>>(g, ph.rho1, ph.rho2, phi, L0.beta[0], L0.beta[1],
                                                                  L0.beta[2]);
    ++g_launches;
    for (int l = 1; l < mg.nlev; ++l) {
        Geom gf = level_geom(g, mg.lv[l - 1]), gc = level_geom(g, mg.lv[l]);
        MGLevel& Lf = mg.lv[l - 1];
        MGLevel& Lc = mg.lv[l];
        if (g.D == 2)
            k_coef_restrict<2><<<blocks_for(gc.N + gc.NP), kThreads, 0, s>>>(gf, gc, Lf.beta[0], Lf.beta[1], nullptr,
                                                                            Lc.beta[0], Lc.beta[1], nullptr);
        else
            k_coef_restrict<3><<<blocks_for(gc.N + gc.NP), kThreads, 0, s>>>(gf, gc, Lf.beta[0], Lf.beta[1],
                                                                            Lf.beta[2], Lc.beta[0], Lc.beta[1],
                                                                            Lc.beta[2]);
        ++g_launches;
    }
}

template <int DIM>
static void vcycle_rec(const Geom& g, MG& mg, int l, int npre, int npost, cudaStream_t s) {
    MGLevel& L = mg.lv[l];
    Geom lg = level_geom(g, L);
    if (l == mg.nlev - 1) {
        k_coarse<DIM><<<1, 64, 0, s>>>(lg, L.beta[0], L.beta[1], L.beta[2], L.f, L.p);
        ++g_launches;
        return;
    }
    const unsigned nb = blocks_for(L.N);
    for (int it = 0; it < npre; ++it)
        for (int col = 0; col < 2; ++col) {
            k_rbgs<DIM><<<nb, kThreads, 0, s>>>(lg, L.beta[0], L.beta[1], L.beta[2], L.p, L.f, col);
            ++g_launches;
        }
    MGLevel& C = mg.lv[l + 1];
    Geom cg = level_geom(g, C);
    k_resid_restrict<DIM><<<blocks_for(C.N), kThreads, 0, s>>>(lg, cg, L.beta[0], L.beta[1], L.beta[2], L.p, L.f,
                                                              C.f, C.p);
    ++g_launches;
    vcycle_rec<DIM>(g, mg, l + 1, npre, npost, s);
    k_prolong<DIM><<<nb, kThreads, 0, s>>>(lg, cg, C.p, L.p);
    ++g_launches;
    for (int it = 0; it < npost; ++it)
        for (int col = 0; col < 2; ++col) {
            k_rbgs<DIM><<<nb, kThreads, 0, s>>>(lg, L.beta[0], L.beta[1], L.beta[2], L.p, L.f, col);
            ++g_launches;
        }
}

void launch_vcycle(const Geom& g, MG& mg, int npre, int npost, cudaStream_t s) {
    if (g.D == 2) vcycle_rec<2>(g, mg, 0, npre, npost, s);
    else vcycle_rec<3>(g, mg, 0, npre, npost, s);
}

void launch_resid_norm(const Geom& g, MG& mg, cudaStream_t s) {
    MGLevel& L = mg.lv[0];
    const unsigned G = red_blocks(g.N);
    if (g.D == 2)
        k_resid_sq<2><<<G, kThreads, 0, s>>>(g, L.beta[0], L.beta[1], L.beta[2], L.p, L.f, mg.partials);
    else
        k_resid_sq<3><<<G, kThreads, 0, s>>>(g, L.beta[0], L.beta[1], L.beta[2], L.p, L.f, mg.partials);
    k_final_sum<<<1, 1024, 0, s>>>(mg.partials, (int)G, 1.0, mg.scal + S_RNORM, 1);
    g_launches += 2;
}

void launch_p_mean_remove(const Geom& g, MG& mg, cudaStream_t s) {
    const unsigned G = red_blocks(g.N);
    k_partial_sum<<<G, kThreads, 0, s>>>(g.N, mg.lv[0].p, mg.partials);
    k_final_sum<<<1, 1024, 0, s>>>(mg.partials, (int)G, 1.0, mg.scal + S_MEAN, 0);
    k_sub_scalar<<<blocks_for(g.N), kThreads, 0, s>>>(g.N, mg.lv[0].p, mg.scal + S_MEAN);
    g_launches += 3;
}

template <typename T>
void launch_project(const Geom& g, const PhysDev& ph, const T* phi, T* const* us, double cdt, const double* p,
                    cudaStream_t s) {
    if (g.D == 2)
        k_project<T, 2><<<blocks_for(g.N), kThreads, 0, s>>>(g, ph.rho1, ph.rho2, phi, us[0], us[1], nullptr, cdt, p);
    else
        k_project<T, 3><<<blocks_for(g.N), kThreads, 0, s>>>(g, ph.rho1, ph.rho2, phi, us[0], us[1], us[2], cdt, p);
    ++g_launches;
}

template <typename T>
void launch_mass(const Geom& g, const T* phi, MG& mg, cudaStream_t s) {
    const unsigned G = red_blocks(g.N);
    k_mass_partial<T><<<G, kThreads, 0, s>>>(g.N, phi, mg.partials);
    double dv = (g.D == 2) ? g.h * g.h : g.h * g.h * g.h;
    k_final_sum<<<1, 1024, 0, s>>>(mg.partials, (int)G, dv, mg.scal + S_MASS, 0);
    g_launches += 2;
}

template <typename T>
void launch_gamma(const Geom& g, const T* const* u, double gamma_param, MG& mg, cudaStream_t s) {
    const unsigned G = red_blocks(g.N + g.NP);
    long n2 = (g.D == 3) ? g.N + g.NP : 0;
    long n1 = (g.D == 2) ? g.N + g.NP : g.N;
    k_umax_partial<T><<<G, kThreads, 0, s>>>(g.N, n1, n2, u[0], u[1], g.D == 3 ? u[2] : u[1], mg.partials);
    k_gamma_final<<<1, 1024, 0, s>>>(mg.partials, (int)G, -gamma_param, mg.scal + S_UMAX, mg.scal + S_GAMMA);
    g_launches += 2;
}

void launch_contact_line(const Geom& g, int wall, const double* cols, MG& mg, cudaStream_t s) {
    const int nlines = (g.D == 3) ? g.n[1] : 1;
    k_contact_line<<<1, 256, 0, s>>>(g.D, g.n[0], nlines, g.h, cols + (long)wall * 3 * g.NP, g.NP,
                                     mg.scal + S_THETA, mg.scal + S_WETTED);
    ++g_launches;
}

template void launch_div<double>(const Geom&, const double* const*, double, MG&, cudaStream_t);
template void launch_div<float>(const Geom&, const float* const*, double, MG&, cudaStream_t);
template void launch_mg_coef<double>(const Geom&, const PhysDev&, const double*, MG&, cudaStream_t);
template void launch_mg_coef<float>(const Geom&, const PhysDev&, const float*, MG&, cudaStream_t);
template void launch_project<double>(const Geom&, const PhysDev&, const double*, double* const*, double,
                                     const double*, cudaStream_t);
template void launch_project<float>(const Geom&, const PhysDev&, const float*, float* const*, double,
                                    const double*, cudaStream_t);
template void launch_mass<double>(const Geom&, const double*, MG&, cudaStream_t);
template void launch_mass<float>(const Geom&, const float*, MG&, cudaStream_t);
template void launch_gamma<double>(const Geom&, const double* const*, double, MG&, cudaStream_t);
template void launch_gamma<float>(const Geom&, const float* const*, double, MG&, cudaStream_t);

}  // namespace cdi
