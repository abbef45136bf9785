// Level-0 red-black Gauss-Seidel sweep of the 3D pressure multigrid in ONE
// pass: both colours of a sweep of A e = r (the FP32 V-cycle's smoother,
// coefficients 2 / (rho_c + rho_nb) from the FP32 cell densities, zero
// through the walls on z) read e from one buffer and write the new e to
// another, so that every array moves through HBM once per sweep in whole
// sectors: rho, r and the old e read, the new e written (16 bytes a cell).
// The two colour passes it replaces each touched half of every sector of e
// and r (about 2 x 20 bytes a cell of DRAM traffic per sweep).
//
// A CTA owns a 64 x 16 tile of the x-y plane and marches along a chunk of z.
// At step k it updates the red cells of plane k+1 and then the black cells of
// plane k: a black cell needs the new red values of its six neighbours (the
// in-plane ones at plane k, made at step k-1, and the ones at k-1 and k+1),
// and a red cell the old black values.  The red cells are also updated on a
// one-cell ring around the tile (the values the tile's black cells need from
// outside it), so no CTA waits for another.  Planes of rho and the old e
// (with a two-cell halo) and of r (one-cell halo) are staged in shared
// memory by 16-byte cp.async copies two planes ahead of use; a red value,
// once made, replaces the old e of its cell in the staged plane.  Staged
// planes are addressed as floats, so a cell's x neighbours are always the
// words just before and after it and its y neighbours one staged row away,
// whatever its colour.  The arithmetic of each update, and its order of
// terms, are those of k_rbgs0 (x-, x+, y-, y+, z-, z+), so the result equals
// a red pass followed by a black pass.
//
// Threads: a thread owns a cell pair (2p, 2p+1) of one tile row (each pair
// holds one red and one black cell of a plane).  A warp covers 16 pairs of
// two adjacent rows: the colour of the pair's red cell flips from one row to
// the next and a staged row is 72 words long, so the two half-warps read
// even and odd banks, free of conflicts.  Warps 0..15 cover tile rows 0..15
// (red and black updates), warps 16..17 the ring rows -1 and 16 (red only),
// warp 18 the red ring cell of each row left or right of the tile.
#include "ops.cuh"

#include <cmath>

namespace cdi {

namespace {

constexpr int kTX = 64, kTY = 16;                  // tile of cells in x, y
constexpr int kTP = kTX / 2;                       // pairs in x (32 = warp width)
constexpr int kEP = kTP + 4;                       // staged pairs per row: -2..33 (16-byte aligned quads)
constexpr int kEQ = kEP / 2;                       // staged quads (4 cells) per row
constexpr int kER = kTY + 4;                       // staged e / rho rows: -2..kTY+1
constexpr int kRR = kTY + 2;                       // staged r rows: -1..kTY
constexpr int kEPlane = 2 * kEP * kER;             // floats per staged e or rho plane
constexpr int kRPlane = 2 * kEP * kRR;
constexpr int kRowF = 2 * kEP;                     // floats per staged row
constexpr int kESlots = 6, kRSlots = 4;            // ring buffers (planes k-1..k+2 in use, two in flight)
constexpr int kPD = 2;                             // planes loaded ahead of use
constexpr int kSweepWarps = kTY + 3;               // 19
constexpr int kSweepThreads = kSweepWarps * 32;    // 608
constexpr size_t kSweepSmem = (size_t)(2 * kESlots * kEPlane + kRSlots * kRPlane) * sizeof(float);
static_assert(kEQ * kER <= kSweepThreads && kEQ * kRR <= kSweepThreads, "one staged quad per thread");

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N)); }

// Gauss-Seidel value of the staged cell at float index fi of plane (E, H)
// (old or new e, rho), with the planes below / above (null through a wall)
// and the cell's r: e = (sum_nb b e_nb - r h^2) / sum_nb b, b = 2 / (rho_c +
// rho_nb), terms in the order x-, x+, y-, y+, z-, z+
__device__ __forceinline__ float cell_update(const float* E, const float* H, const float* Em, const float* Hm,
                                             const float* Ep, const float* Hp, int fi, float rcen, float h2) {
    const float rc = H[fi];
    const float b0 = __fdividef(2.f, rc + H[fi - 1]), b1 = __fdividef(2.f, rc + H[fi + 1]);
    float bsum = b0 + b1;
    float off = b0 * E[fi - 1] + b1 * E[fi + 1];
    const float b2 = __fdividef(2.f, rc + H[fi - kRowF]), b3 = __fdividef(2.f, rc + H[fi + kRowF]);
    bsum += b2 + b3;
    off += b2 * E[fi - kRowF] + b3 * E[fi + kRowF];
    if (Em) {
        const float b = __fdividef(2.f, rc + Hm[fi]);
        bsum += b;
        off += b * Em[fi];
    }
    if (Ep) {
        const float b = __fdividef(2.f, rc + Hp[fi]);
        bsum += b;
        off += b * Ep[fi];
    }
    return __fdividef(off - rcen * h2, bsum);
}

// p[0] += e.x, p[1] += e.y for two cells of a pair (16-byte aligned)
__device__ __forceinline__ void p_add_pair(double* p, float2 e) {
    double2 v = *reinterpret_cast<double2*>(p);
    v.x += (double)e.x;
    v.y += (double)e.y;
    *reinterpret_cast<double2*>(p) = v;
}
__device__ __forceinline__ void p_add_pair(float2* p, float2 e) {
    float4 v = *reinterpret_cast<float4*>(p);
    const float2 a = ops::p_add(make_float2(v.x, v.y), e.x), b = ops::p_add(make_float2(v.z, v.w), e.y);
    *reinterpret_cast<float4*>(p) = make_float4(a.x, a.y, b.x, b.y);
}

__device__ __forceinline__ int next_slot(int s, int n) { return s + 1 == n ? 0 : s + 1; }

template <typename T, int MODE>
__global__ void __launch_bounds__(kSweepThreads, 2)
    k_sweep0(Geom g, const float* __restrict__ rho, const float* __restrict__ ein, float* __restrict__ eout,
             const float* __restrict__ r, float h2, PT<T>* __restrict__ p, int zchunk) {
    extern __shared__ float smf[];
    float* Es = smf;                                 // [kESlots][kER][kEP][2] old e, then new red values
    float* Rh = Es + kESlots * kEPlane;              // [kESlots][kER][kEP][2] rho
    float* Rs = Rh + kESlots * kEPlane;              // [kRSlots][kRR][kEP][2] r
    const int nx = g.n[0], ny = g.n[1], nz = g.n[2];
    const long NP = g.NP;
    const int x0 = blockIdx.x * kTX, y0 = blockIdx.y * kTY;
    const int z0 = blockIdx.z * zchunk;
    const int z1 = min(z0 + zchunk, nz);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    // ring-buffer slots: plane z sits in slot (z - (z0 - 2)) mod kESlots (e, rho)
    // and (z - (z0 - 2)) mod kRSlots (r)
    auto eslot = [&](int z) { return (z - z0 + 2) % kESlots; };
    auto rslot = [&](int z) { return (z - z0 + 2) % kRSlots; };

    // The staging pattern of every plane is the same: thread tid copies at most
    // one quad (4 cells, 16 bytes) of the e / rho grid (rows -2..kTY+1, pairs
    // -2..33) and one of the r grid (rows -1..kTY); its offsets within a z
    // plane (periodic in x and y) are formed once.
    auto quad_off = [&](int q, int row_rel) -> int {
        int x = x0 + 4 * q - 4;
        if (x < 0) x += nx;
        else if (x >= nx) x -= nx;
        int y = y0 + row_rel;
        if (y < 0) y += ny;
        else if (y >= ny) y -= ny;
        return x + nx * y;
    };
    const bool has_e = tid < kEQ * kER, has_r = tid < kEQ * kRR;
    int e_off = 0, e_sm = 0, r_off = 0, r_sm = 0;
    if (has_e) {
        const int row = tid / kEQ, q = tid - row * kEQ;
        e_off = quad_off(q, row - 2);
        e_sm = row * kRowF + 4 * q;
    }
    if (has_r) {
        const int row = tid / kEQ, q = tid - row * kEQ;
        r_off = quad_off(q, row - 1);
        r_sm = row * kRowF + 4 * q;
    }
    // stage e / rho plane z and r plane zr (planes outside the wall-bounded
    // domain, or beyond what this chunk reads, are skipped); one commit group
    // per call, possibly empty
    auto issue = [&](int z, int zr) {
        if (has_e && z >= 0 && z < nz && z <= z1 + 1) {
            const int sl = eslot(z);
            const long o = (long)z * NP + e_off;
            cp_async16(Rh + sl * kEPlane + e_sm, rho + o);
            if (MODE == kSweepFromZero)
                *reinterpret_cast<float4*>(Es + sl * kEPlane + e_sm) = make_float4(0.f, 0.f, 0.f, 0.f);
            else
                cp_async16(Es + sl * kEPlane + e_sm, ein + o);
        }
        if (has_r && zr >= 0 && zr < nz && zr <= z1) cp_async16(Rs + rslot(zr) * kRPlane + r_sm, r + (long)zr * NP + r_off);
        cp_async_commit();
    };
    // prologue: e / rho planes z0-2 and z0-1, then group m (m = 0, 1, ...) holds
    // e / rho plane z0+m and r plane z0-1+m; step k = z0-2+m reads groups <= m
    issue(z0 - 2, -1);
    issue(z0 - 1, -1);
    for (int m = 0; m < kPD; ++m) issue(z0 + m, z0 - 1 + m);

    // this thread's pair: red update on rows -1..kTY (warps 0..kTY+1), black
    // update on rows 0..kTY-1 (warps 2..kTY+1); warp kTY+2: the ring cells
    const int half = lane >> 4, sub = lane & 15;
    int red_row = -1, pc = 0;   // staged r row (tile row + 1) and staged pair (tile pair + 2)
    if (warp < kTY) {           // tile rows 0..kTY-1: red and black updates
        red_row = 2 * (warp >> 1) + half + 1;
        pc = 16 * (warp & 1) + sub + 2;
    } else if (warp < kTY + 2) {  // ring rows -1 and kTY (opposite colours: conflict-free too)
        red_row = half ? kTY + 1 : 0;
        pc = 16 * (warp & 1) + sub + 2;
    } else if (lane < kTY + 2) {  // ring columns
        red_row = lane;
    }
    const bool black_thread = warp < kTY;
    const int jrel = red_row - 1;  // tile row of the pair
    // slots of planes k-1, k, k+1 (e / rho) and of r planes k, k+1 at the
    // current step, and the slots the step's loads fill (e / rho plane k+4, r
    // plane k+3); global offsets of those planes
    int sm1 = eslot(z0 - 3 + kESlots), s0 = eslot(z0 - 2), sp1 = eslot(z0 - 1);
    int r0 = rslot(z0 - 2 + kRSlots), rp1 = rslot(z0 - 1);
    for (int k = z0 - 2; k < z1; ++k) {
        cp_async_wait<kPD - 1>();
        __syncthreads();  // e / rho planes <= k+2 and r planes <= k+1 are staged
        // e / rho plane k-2 and r plane k-1 were last read by step k-1's black
        // update: their slots take the planes two steps ahead
        issue(k + 2 + kPD, k + 1 + kPD);
        const int sp2 = next_slot(sp1, kESlots);
        // red cells of plane kr = k+1 on the tile and its one-cell ring
        const int kr = k + 1;
        if (kr >= 0 && kr < nz && red_row >= 0) {
            const int y = y0 + red_row - 1;
            int pcr = pc, t;
            if (warp < kTY + 2) {
                t = (y + kr) & 1;
            } else {
                // the red one of cells x0-1 (pair -1, second cell) and x0+kTX (pair kTP, first cell)
                const bool left = ((y + kr) & 1) != 0;
                pcr = left ? 1 : kTP + 2;
                t = left ? 1 : 0;
            }
            const int fi = (red_row + 1) * kRowF + 2 * pcr + t;
            const float* E = Es + sp1 * kEPlane;
            const float* H = Rh + sp1 * kEPlane;
            const float rcen = Rs[rp1 * kRPlane + red_row * kRowF + 2 * pcr + t];
            const float v = cell_update(E, H, kr > 0 ? Es + s0 * kEPlane : nullptr, Rh + s0 * kEPlane,
                                        kr < nz - 1 ? Es + sp2 * kEPlane : nullptr, Rh + sp2 * kEPlane, fi, rcen,
                                        h2);
            Es[sp1 * kEPlane + fi] = v;
        }
        __syncthreads();  // the red values of plane k+1 are visible
        // black cells of plane k on the tile, written out with their red partners
        if (k >= z0 && black_thread) {
            const int t = (y0 + jrel + k + 1) & 1;
            const int fb = (jrel + 2) * kRowF + 2 * pc;
            const float* E = Es + s0 * kEPlane;
            const float* H = Rh + s0 * kEPlane;
            const float rcen = Rs[r0 * kRPlane + (jrel + 1) * kRowF + 2 * pc + t];
            const float v = cell_update(E, H, k > 0 ? Es + sm1 * kEPlane : nullptr, Rh + sm1 * kEPlane,
                                        k < nz - 1 ? Es + sp1 * kEPlane : nullptr, Rh + sp1 * kEPlane, fb + t, rcen,
                                        h2);
            const float red = E[fb + 1 - t];  // the pair's red value is in place
            const float2 out = t == 0 ? make_float2(v, red) : make_float2(red, v);
            const long c = (long)k * NP + (long)(x0 + 2 * (pc - 2)) + (long)nx * (y0 + jrel);
            reinterpret_cast<float2*>(eout)[c >> 1] = out;
            if (MODE == kSweepUpdate) p_add_pair(p + c, out);
        }
        sm1 = s0;
        s0 = sp1;
        sp1 = sp2;
        r0 = rp1;
        rp1 = next_slot(rp1, kRSlots);
    }
    cp_async_wait<0>();
}

}  // namespace

bool sweep0_supported(const Geom& g) {
    return g.D == 3 && g.n[0] % kTX == 0 && g.n[1] % kTY == 0 && g.n[2] >= 4 && (g.N / 2) < (1L << 31);
}

namespace {
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
// planes per z chunk: the chunk count c maximises the fill of the last wave
// of resident CTAs (kSweepPerSM per SM) times the share of staged planes
// that are not re-read halo (each chunk stages four extra e / rho planes);
// chunks hold at least 8 planes
constexpr int kSweepPerSM = 2;
int sweep0_zchunk(const Geom& g) {
    const long tiles = (long)(g.n[0] / kTX) * (g.n[1] / kTY);
    const double wave = (double)kSweepPerSM * sm_count();
    const int nz = g.n[2];
    int best = nz;
    double best_score = -1.0;
    for (int c = 1; (nz + c - 1) / c >= 8 || c == 1; ++c) {
        const int ch = (nz + c - 1) / c;
        const int nc = (nz + ch - 1) / ch;
        const double waves = tiles * nc / wave;
        const double fill = waves / std::ceil(waves);
        const double score = fill * (1.0 - 2.0 / ch);
        if (score > best_score + 1e-9) {
            best_score = score;
            best = ch;
        }
    }
    return best;
}
}  // namespace

bool sweep0_auto(const Geom& g) {
    if (!sweep0_supported(g)) return false;
    const long tiles = (long)(g.n[0] / kTX) * (g.n[1] / kTY);
    const int ch = sweep0_zchunk(g);
    return tiles * ((g.n[2] + ch - 1) / ch) >= (long)kSweepPerSM * sm_count();  // at least one full wave
}

cudaError_t sweep0_prepare() {
    const void* fns[] = {(const void*)k_sweep0<double, kSweepFromZero>, (const void*)k_sweep0<double, kSweepPlain>,
                         (const void*)k_sweep0<double, kSweepUpdate>,   (const void*)k_sweep0<float, kSweepFromZero>,
                         (const void*)k_sweep0<float, kSweepPlain>,     (const void*)k_sweep0<float, kSweepUpdate>};
    for (const void* f : fns) {
        const cudaError_t e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSweepSmem);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

// one full red-black sweep of level 0: ein -> eout (ein unused when from_zero),
// and p += eout when update
template <typename T>
void launch_sweep0(const Geom& g, const float* rho, const float* ein, float* eout, const float* r, int mode, PT<T>* p,
                   cudaStream_t s) {
    const int zchunk = sweep0_zchunk(g);
    const dim3 grid((unsigned)(g.n[0] / kTX), (unsigned)(g.n[1] / kTY), (unsigned)((g.n[2] + zchunk - 1) / zchunk));
    const float h2 = (float)(g.h * g.h);
    if (mode == kSweepFromZero)
        k_sweep0<T, kSweepFromZero><<<grid, kSweepThreads, kSweepSmem, s>>>(g, rho, ein, eout, r, h2, p, zchunk);
    else if (mode == kSweepUpdate)
        k_sweep0<T, kSweepUpdate><<<grid, kSweepThreads, kSweepSmem, s>>>(g, rho, ein, eout, r, h2, p, zchunk);
    else
        k_sweep0<T, kSweepPlain><<<grid, kSweepThreads, kSweepSmem, s>>>(g, rho, ein, eout, r, h2, p, zchunk);
}

template void launch_sweep0<double>(const Geom&, const float*, const float*, float*, const float*, int, double*,
                                    cudaStream_t);
template void launch_sweep0<float>(const Geom&, const float*, const float*, float*, const float*, int, float2*,
                                   cudaStream_t);

}  // namespace cdi
