// Momentum right-hand side of 3D grids, tiled (Eq. NS_momentum without the
// pressure, Eq. EB surface tension): every component on the low faces of
// every cell, with the arithmetic, terms and order of terms of ops::mom_at
// (advection of the mass flux, the viscous stress mu (grad u + grad u^T) on
// cell centres and edges, the wall-edge stress from the wall rows, the
// energy-based surface tension); what changes is where the operands come from.
//
// A CTA owns a 32 x 8 tile of the x-y plane and marches along a chunk of z.
// The eight arrays a face's terms read (the three velocity components, the
// three mass fluxes, phi and mu_c) are staged in shared memory one plane ahead
// by 16-byte cp.async copies, each with a one-cell halo in y and a one-quad
// halo in x (wrapped around the periodic axes), in a ring of four planes
// (k-1, k, k+1 in use, k+2 in flight).  Each thread computes the three faces
// of one cell; every operand is then a shared-memory word at a constant
// offset from the thread's own, instead of a global gather with its own
// 64-bit index (the column-marching form issued about 150 such gathers a
// cell and waited on them).  Warp w stages array w.
#include "ops.cuh"
#include "stage.cuh"

#include <cmath>

namespace cdi {

namespace {

using namespace stage;

constexpr int kMX = 32, kMY = 8;          // tile of cells in x, y
constexpr int kMThreads = kMX * kMY;      // one cell (its three faces) a thread
constexpr int kMArrays = 8;               // u0 u1 u2 m0 m1 m2 phi mu_c (array w staged by warp w)
constexpr int kMSlots = 4;                // planes k-1, k, k+1 in use, k+2 in flight
template <typename T>
constexpr int mom_per_sm() { return sizeof(T) == 4 ? 3 : 2; }  // resident CTAs an SM (registers)
static_assert(kMArrays == kMThreads / 32, "one staging warp an array");

template <typename T>
struct MomTile {
    static constexpr int QE = 16 / (int)sizeof(T);  // elements of a 16-byte quad
    static constexpr int RW = kMX + 2 * QE;          // staged row: x0-QE .. x0+kMX+QE-1
    static constexpr int RH = kMY + 2;               // staged rows: y0-1 .. y0+kMY
    static constexpr int PL = RW * RH;               // elements of one array's staged plane
    static constexpr int QR = RW / QE;               // quads a staged row
    static constexpr int QP = QR * RH;               // quads of one array's staged plane
    static constexpr int QM = (QP + 31) / 32;        // staging rounds of a warp
    static constexpr int SLOT = kMArrays * PL;       // elements of one staged plane of every array
    static constexpr size_t SMEM = (size_t)kMSlots * SLOT * sizeof(T);
};

template <int V>
struct IC {
    static constexpr int value = V;
};

template <typename T>
__global__ void __launch_bounds__(kMThreads, mom_per_sm<T>())
    k_mom_tile(Geom g, PhysDev ph, StageFields<T> f, int zchunk) {
    using M = MomTile<T>;
    extern __shared__ __align__(128) unsigned char smm_raw[];
    T* sm = reinterpret_cast<T*>(smm_raw);
    const int nx = g.n[0], ny = g.n[1], nz = g.n[2];
    const long NP = g.NP;
    const int tx = threadIdx.x, ty = threadIdx.y, lane = tx;
    const int x0 = blockIdx.x * kMX, y0 = blockIdx.y * kMY;
    const int z0 = blockIdx.z * zchunk, z1 = min(z0 + zchunk, nz);
    const T ih = g_ih<T>(g);
    const T dmu = phys<T>(ph).dmu, mu2 = phys<T>(ph).mu2;

    // staging: warp ty copies array ty, quads lane + 32 m (offsets within a
    // plane formed once, wrapped around x and y); the face arrays u2, m2
    // have a plane for the high wall (nz + 1 planes)
    const T* src = ty == 0 ? f.u[0] : ty == 1 ? f.u[1] : ty == 2 ? f.u[2] : ty == 3 ? f.m[0] : ty == 4 ? f.m[1]
                 : ty == 5 ? f.m[2] : ty == 6 ? f.phi : f.muc;
    const int planes = (ty == 2 || ty == 5) ? nz + 1 : nz;
    int qg[M::QM], qs[M::QM];
#pragma unroll
    for (int m = 0; m < M::QM; ++m) {
        const int q = lane + 32 * m;
        const int row = q / M::QR, qq = q - row * M::QR;
        int x = x0 - M::QE + M::QE * qq, y = y0 - 1 + row;
        x = x < 0 ? x + nx : (x >= nx ? x - nx : x);
        y = y < 0 ? y + ny : (y >= ny ? y - ny : y);
        qg[m] = q < M::QP ? x + nx * y : -1;
        qs[m] = ty * M::PL + row * M::RW + M::QE * qq;
    }
    auto stage_plane = [&](int z, int slot) {
        if (z >= 0 && z < planes && z <= z1) {
            const T* s = src + (long)z * NP;
            T* d = sm + slot * M::SLOT;
#pragma unroll
            for (int m = 0; m < M::QM; ++m)
                if (qg[m] >= 0) cp_async16(d + qs[m], s + qg[m]);
        }
        cp_async_commit();
    };
    // prologue: planes z0-1, z0 (slots 0, 1), then z0+1 (slot 2); plane z
    // sits in slot (z - z0 + 1) mod 4
    stage_plane(z0 - 1, 0);
    stage_plane(z0, 1);
    stage_plane(z0 + 1, 2);

    const int base = (ty + 1) * M::RW + tx + M::QE;  // the thread's cell in a staged array plane
    const long pidx = (long)(x0 + tx) + (long)nx * (y0 + ty);
    T* rm0 = f.rm[0] + pidx;
    T* rm1 = f.rm[1] + pidx;
    T* rm2 = f.rm[2] + pidx;

    // the faces of plane k = z0 + 4 m + u (its planes k-1, k, k+1 in slots
    // u, u+1, u+2 mod 4)
    auto plane = [&](auto uc, int k) {
        constexpr int u = decltype(uc)::value;
        cp_async_wait<0>();
        __syncthreads();  // plane k+1 has landed; plane k-1 is done with slot u+3
        stage_plane(k + 2, (u + 3) % kMSlots);
        // value of array `arr` at the cell offset (dx, dy, dz) from this thread's
        auto V = [&](int arr, int dx, int dy, int dz) -> T {
            const int slot = (u + 1 + dz + kMSlots) % kMSlots;
            return sm[slot * M::SLOT + arr * M::PL + base + dy * M::RW + dx];
        };
        auto mu = [&](int dx, int dy, int dz) { return dmu * V(6, dx, dy, dz) + mu2; };
        const long c = (long)k * NP;
        T out[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const int ax = a == 0, ay = a == 1, az = a == 2;  // e_a
            if (a == 2 && k == 0) {  // wall face
                out[a] = T(0);
                continue;
            }
            T adv = T(0), vis = T(0);
#pragma unroll
            for (int b = 0; b < 3; ++b) {
                if (b == a) {
                    const T uRlo = V(a, 0, 0, 0), uRhi = V(a, ax, ay, az), uLlo = V(a, -ax, -ay, -az);
                    T mbR = T(0.5) * (V(3 + a, 0, 0, 0) + V(3 + a, ax, ay, az)), ubR = T(0.5) * (uRlo + uRhi);
                    T mbL = T(0.5) * (V(3 + a, -ax, -ay, -az) + V(3 + a, 0, 0, 0)), ubL = T(0.5) * (uLlo + uRlo);
                    T tR = T(2) * mu(0, 0, 0) * (uRhi - uRlo) * ih;
                    T tL = T(2) * mu(-ax, -ay, -az) * (uRlo - uLlo) * ih;
                    adv -= (mbR * ubR - mbL * ubL) * ih;
                    vis += (tR - tL) * ih;
                } else {
                    const int bx = b == 0, by = b == 1, bz = b == 2;  // e_b
                    T conv[2], tau[2];
#pragma unroll
                    for (int side = 0; side < 2; ++side) {
                        if (b == 2 && ((side == 0 && k == 0) || (side == 1 && k == nz - 1))) {
                            const int s = side;  // the edge lies on wall s
                            const long o = ((long)s * 2 + a) * NP + pidx;
                            const T ug = __ldg(f.wghost + o), muw = __ldg(f.wmuw + o);
                            const T u0 = V(a, 0, 0, 0);
                            conv[side] = T(0);
                            tau[side] = (s == 0) ? muw * (u0 - ug) * ih : muw * (ug - u0) * ih;
                            continue;
                        }
                        // chi = c + side e_b, clo = chi - e_b, chiA = chi - e_a, cloA = clo - e_a
                        const int hx = side * bx, hy = side * by, hz = side * bz;
                        const T uhi = V(a, hx, hy, hz), ulo = V(a, hx - bx, hy - by, hz - bz);
                        const T ub = T(0.5) * (ulo + uhi);
                        const T mb = T(0.5) * (V(3 + b, hx, hy, hz) + V(3 + b, hx - ax, hy - ay, hz - az));
                        conv[side] = mb * ub;
                        const T me = T(0.25) * (mu(hx, hy, hz) + mu(hx - ax, hy - ay, hz - az) +
                                                mu(hx - bx, hy - by, hz - bz) +
                                                mu(hx - bx - ax, hy - by - ay, hz - bz - az));
                        const T dub = (uhi - ulo) * ih;
                        const T dua = (V(b, hx, hy, hz) - V(b, hx - ax, hy - ay, hz - az)) * ih;
                        tau[side] = me * (dub + dua);
                    }
                    adv -= (conv[1] - conv[0]) * ih;
                    vis += (tau[1] - tau[0]) * ih;
                }
            }
            // energy-based surface tension on the face (Eq. EB)
            const T st = T(0.5) * (V(7, -ax, -ay, -az) + V(7, 0, 0, 0)) * (V(6, 0, 0, 0) - V(6, -ax, -ay, -az)) * ih;
            out[a] = adv + vis + st;
        }
        rm0[c] = out[0];
        rm1[c] = out[1];
        rm2[c] = out[2];
    };
    for (int kb = z0; kb < z1; kb += kMSlots) {
        plane(IC<0>{}, kb);
        if (kb + 1 >= z1) break;
        plane(IC<1>{}, kb + 1);
        if (kb + 2 >= z1) break;
        plane(IC<2>{}, kb + 2);
        if (kb + 3 >= z1) break;
        plane(IC<3>{}, kb + 3);
    }
    cp_async_wait<0>();  // the last groups stage nothing, but leave no copy in flight
}

int sm_count() {
    static int n = 0;
    if (!n) {
        int dev = 0, v = 0;
        if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) !=
                                                      cudaSuccess) {
            cudaGetLastError();
            v = 152;
        }
        n = v;
    }
    return n;
}

// planes per z chunk: the chunk count maximises the fill of the last wave of
// resident CTAs times the share of staged planes that are not halo (two a chunk)
int mom_zchunk(const Geom& g, int per_sm) {
    const long tiles = (long)(g.n[0] / kMX) * (g.n[1] / kMY);
    const double wave = (double)per_sm * sm_count();
    const int nz = g.n[2];
    int best = nz;
    double best_score = -1.0;
    for (int c = 1; c <= nz; ++c) {
        const int ch = (nz + c - 1) / c;
        const int nc = (nz + ch - 1) / ch;
        const double waves = tiles * nc / wave;
        const double fill = waves / std::ceil(waves);
        const double score = fill * (1.0 - 2.0 / (ch + 2.0));
        if (score > best_score + 1e-9) {
            best_score = score;
            best = ch;
        }
    }
    return best;
}

}  // namespace

bool mom_tile_supported(const Geom& g) { return g.D == 3 && g.n[0] % kMX == 0 && g.n[1] % kMY == 0; }

cudaError_t mom_tile_prepare() {
    cudaError_t e = cudaFuncSetAttribute((const void*)k_mom_tile<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)MomTile<double>::SMEM);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute((const void*)k_mom_tile<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)MomTile<float>::SMEM);
    return e;
}

template <typename T>
void launch_mom_tile(const Geom& g, const PhysDev& ph, const StageFields<T>& f, cudaStream_t s) {
    const int zchunk = mom_zchunk(g, mom_per_sm<T>());
    const dim3 grid((unsigned)(g.n[0] / kMX), (unsigned)(g.n[1] / kMY), (unsigned)((g.n[2] + zchunk - 1) / zchunk));
    k_mom_tile<T><<<grid, dim3(kMX, kMY), MomTile<T>::SMEM, s>>>(g, ph, f, zchunk);
}

template void launch_mom_tile<double>(const Geom&, const PhysDev&, const StageFields<double>&, cudaStream_t);
template void launch_mom_tile<float>(const Geom&, const PhysDev&, const StageFields<float>&, cudaStream_t);

}  // namespace cdi
