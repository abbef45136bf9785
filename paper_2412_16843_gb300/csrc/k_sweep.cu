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
// Staging.  Tiles whose halo lies inside the grid (every tile but those on
// the periodic seams of x and y) load each staged plane with one TMA copy per
// array (cp.async.bulk.tensor of a 72 x 20 box of rho and the old e, a 72 x 18
// box of r, issued by one thread and completed on the plane's mbarrier, every
// wait bounded); the box lands in shared memory in exactly the layout below,
// so both stagings feed the same arithmetic.  Seam tiles, whose halo wraps
// around the grid, keep the per-thread 16-byte cp.async copies.
//
// Threads: a thread owns a cell pair (2p, 2p+1) of one tile row (each pair
// holds one red and one black cell of a plane).  A warp covers 16 pairs of
// two adjacent rows: the colour of the pair's red cell flips from one row to
// the next and a staged row is 72 words long, so the two half-warps read
// even and odd banks, free of conflicts.  Warps 0..15 cover tile rows 0..15
// (red and black updates), warps 16..17 the ring rows -1 and 16 (red only),
// warp 18 the red ring cell of each row left or right of the tile.
#include "ops.cuh"
#include "stage.cuh"

#include <cudaTypedefs.h>

#include <cmath>

namespace cdi {

namespace {

using namespace stage;

constexpr int kTX = 64, kTY = 16;                  // tile of cells in x, y
constexpr int kTP = kTX / 2;                       // pairs in x (32 = warp width)
constexpr int kEP = kTP + 4;                       // staged pairs per row: -2..33 (16-byte aligned quads)
constexpr int kEQ = kEP / 2;                       // staged quads (4 cells) per row
constexpr int kER = kTY + 4;                       // staged e / rho rows: -2..kTY+1
constexpr int kRR = kTY + 2;                       // staged r rows: -1..kTY
constexpr int kEPlane = 2 * kEP * kER;             // floats per staged e or rho plane
constexpr int kRPlane = 2 * kEP * kRR;
constexpr int kRowF = 2 * kEP;                     // floats per staged row
// ring buffers: e / rho planes k-1..k+2 in use and two in flight; r planes k,
// k+1 in use and two in flight.  Both rings have six slots, so the z loop
// unrolls by six and every slot index is a compile-time constant.
constexpr int kESlots = 6, kRSlots = 6;
constexpr int kPD = 2;                             // planes loaded ahead of use
constexpr int kSweepWarps = kTY + 3;               // 19
constexpr int kSweepThreads = kSweepWarps * 32;    // 608
// an r slot padded to a multiple of 128 bytes (TMA destinations are 128-byte aligned)
constexpr int kRSlotF = (kRPlane * 4 + 127) / 128 * 32;
constexpr int kSlotsF = 2 * kESlots * kEPlane + kRSlots * kRSlotF;   // floats of the staged planes
constexpr size_t kSweepSmem = (size_t)kSlotsF * sizeof(float) + kESlots * sizeof(unsigned long long);
constexpr unsigned kEBoxBytes = kEPlane * 4, kRBoxBytes = kRPlane * 4;   // one TMA box of e / rho, of r
static_assert(kEQ * kER <= kSweepThreads && kEQ * kRR <= kSweepThreads, "one staged quad per thread");
static_assert(kEPlane * 4 % 128 == 0 && kRSlotF * 4 % 128 == 0, "slots start on 128-byte boundaries");

// Gauss-Seidel value of the staged cell at float index fi of the e plane E
// (old or new e; its rho plane lies kESlots e planes further on), with the
// cell's rho rc, the rho and e of the cells below (hm, em) and above (hp, ep)
// (taken when lo / hi: not through a wall) and the cell's r: e = (sum_nb b e_nb - r h^2) / sum_nb b with b = 2 /
// (rho_c + rho_nb), formed as (sum_nb b' e_nb - r h^2 / 2) / sum_nb b' with
// b' = b / 2 = 1 / (rho_c + rho_nb) (ops::rcp_approx), terms in the order x-,
// x+, y-, y+, z-, z+; h2h = h^2 / 2
__device__ __forceinline__ float cell_update(const float* E, int fi, float rc, bool lo, float hm, float em, bool hi,
                                             float hp, float ep, float rcen, float h2h) {
    constexpr int HO = kESlots * kEPlane;
    const float b0 = ops::rcp_approx(rc + E[HO + fi - 1]), b1 = ops::rcp_approx(rc + E[HO + fi + 1]);
    float bsum = b0 + b1;
    float off = b0 * E[fi - 1] + b1 * E[fi + 1];
    const float b2 = ops::rcp_approx(rc + E[HO + fi - kRowF]), b3 = ops::rcp_approx(rc + E[HO + fi + kRowF]);
    bsum += b2 + b3;
    off += b2 * E[fi - kRowF] + b3 * E[fi + kRowF];
    if (lo) {
        const float b = ops::rcp_approx(rc + hm);
        bsum += b;
        off += b * em;
    }
    if (hi) {
        const float b = ops::rcp_approx(rc + hp);
        bsum += b;
        off += b * ep;
    }
    return __fmul_rn(off - rcen * h2h, ops::rcp_approx(bsum));
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

template <int V>
struct IC {
    static constexpr int value = V;
};

template <typename T, int MODE>
__global__ void __launch_bounds__(kSweepThreads, 2)
    k_sweep0(Geom g, const float* __restrict__ rho, const float* __restrict__ ein, float* __restrict__ eout,
             const float* __restrict__ r, float h2h, float omega, PT<T>* __restrict__ p, int zchunk,
             const __grid_constant__ CUtensorMap tm_rho, const __grid_constant__ CUtensorMap tm_e,
             const __grid_constant__ CUtensorMap tm_r, int use_tma, double* __restrict__ err) {
    extern __shared__ __align__(128) float smf[];
    float* Es = smf;                                 // [kESlots][kER][kEP][2] old e, then new red values
    float* Rh = Es + kESlots * kEPlane;              // [kESlots][kER][kEP][2] rho
    float* Rs = Rh + kESlots * kEPlane;              // [kRSlots][kRR][kEP][2] r (slots kRSlotF floats apart)
    const unsigned bar0 = smem_u32(smf + kSlotsF);   // [kESlots] mbarriers, one per e / rho slot
    const int nx = g.n[0], ny = g.n[1], nz = g.n[2];
    const long NP = g.NP;
    const int x0 = blockIdx.x * kTX, y0 = blockIdx.y * kTY;
    const int z0 = blockIdx.z * zchunk;
    const int z1 = min(z0 + zchunk, nz);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    // TMA staging: the tile's halo boxes lie inside the grid (no periodic wrap)
    const bool tma = use_tma && x0 >= 4 && x0 + kTX + 4 <= nx && y0 >= 2 && y0 + kTY + 2 <= ny &&
                     (smem_u32(smf) & 127u) == 0;
    if (tma && tid == 0) {
        for (int i = 0; i < kESlots; ++i) mbar_init(bar0 + 8u * i, 1);
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
        fence_proxy_async();
    }
    __syncthreads();
    bool timed_out = false;

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
    // Stage e / rho plane z into e slot es and r plane zr into r slot rs
    // (planes outside the wall-bounded domain, or beyond what this chunk
    // reads, are skipped).  Plane z sits in slot (z - z0 + 2) mod 6, and so
    // does r plane zr.  cp.async: one commit group per call, possibly empty.
    // TMA: thread 0 arms mbarrier es with the bytes of the call's boxes and
    // issues them (an empty call just arrives).
    auto issue = [&](int z, int zr, int es, int rs) {
        const bool ce = z >= 0 && z < nz && z <= z1 + 1, cr = zr >= 0 && zr < nz && zr <= z1;
        if (MODE == kSweepFromZero && ce && has_e)
            *reinterpret_cast<float4*>(Es + es * kEPlane + e_sm) = make_float4(0.f, 0.f, 0.f, 0.f);
        if (tma) {
            if (tid == 0) {
                const unsigned bar = bar0 + 8u * es;
                mbar_arrive_tx(bar, (ce ? (MODE == kSweepFromZero ? 1u : 2u) * kEBoxBytes : 0u) + (cr ? kRBoxBytes : 0u));
                if (ce) {
                    tma_plane(smem_u32(Rh + es * kEPlane), &tm_rho, x0 - 4, y0 - 2, z, bar);
                    if (MODE != kSweepFromZero) tma_plane(smem_u32(Es + es * kEPlane), &tm_e, x0 - 4, y0 - 2, z, bar);
                }
                if (cr) tma_plane(smem_u32(Rs + rs * kRSlotF), &tm_r, x0 - 4, y0 - 1, zr, bar);
            }
            return;
        }
        if (has_e && ce) {
            const long o = (long)z * NP + e_off;
            cp_async16(Rh + es * kEPlane + e_sm, rho + o);
            if (MODE != kSweepFromZero) cp_async16(Es + es * kEPlane + e_sm, ein + o);
        }
        if (has_r && cr) cp_async16(Rs + rs * kRSlotF + r_sm, r + (long)zr * NP + r_off);
        cp_async_commit();
    };
    // prologue: e / rho planes z0-2 .. z0+1 (slots 0..3) and r planes z0-1, z0
    // (slots 1, 2); with TMA the first step's planes z0-2, z0-1 are waited for here
    issue(z0 - 2, -1, 0, 0);
    issue(z0 - 1, -1, 1, 0);
    issue(z0, z0 - 1, 2, 1);
    issue(z0 + 1, z0, 3, 2);
    if (tma)
        for (int j = 0; j < 2; ++j)
            if (!mbar_wait_bounded(bar0 + 8u * j, 0u)) timed_out = true;

    // this thread's pair: red update on rows -1..kTY (warps 0..kTY+1), black
    // update on rows 0..kTY-1 (warps 0..kTY-1); warp kTY+2: the ring cells
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
    // The colour of a cell flips from one plane to the next, so the thread's
    // red cell (staged float index fr, r index rr) and the parity tb of its
    // black cell take one value on the even steps of the z march and another
    // on the odd ones.
    int fr[2] = {0, 0}, rr[2] = {0, 0}, tb[2] = {0, 0};
    if (red_row >= 0) {
        const int y = y0 + red_row - 1;
#pragma unroll
        for (int par = 0; par < 2; ++par) {
            const int kr = z0 - 1 + par;  // red plane of the first (par 0) or second step
            int pcr = pc, t;
            if (warp < kTY + 2) {
                t = (y + kr) & 1;
            } else {
                // the red one of cells x0-1 (pair -1, second cell) and x0+kTX (pair kTP, first cell)
                const bool left = ((y + kr) & 1) != 0;
                pcr = left ? 1 : kTP + 2;
                t = left ? 1 : 0;
            }
            fr[par] = (red_row + 1) * kRowF + 2 * pcr + t;
            rr[par] = red_row * kRowF + 2 * pcr + t;
            tb[par] = (y0 + jrel + kr) & 1;
        }
    }
    const int fb = (jrel + 2) * kRowF + 2 * pc;  // staged float index of the pair
    const int rb = (jrel + 1) * kRowF + 2 * pc;
    // this thread's output pair of plane z0 (black threads); advanced by one
    // plane per black update
    const long cb = (long)z0 * NP + (long)(x0 + 2 * (pc - 2)) + (long)nx * (y0 + jrel);
    float2* o2 = reinterpret_cast<float2*>(eout) + (black_thread ? cb >> 1 : 0);
    PT<T>* pp = p + (black_thread && MODE == kSweepUpdate ? cb : 0);
    const long NPh = NP >> 1;

    // Step k = z0 - 2 + 6 m + u of the march: red cells of plane k + 1, then
    // black cells of plane k.  e / rho plane k + j sits in slot (u + j) mod 6
    // and r plane k + j in slot (u + j) mod 6.  With TMA, plane k + 2 is call
    // 6 m + u + 2 of mbarrier (u + 2) mod 6, phase m + (u >= 4).
    float prev_red = 0.f;  // this thread's red value of the previous step
    auto step = [&](auto uc, int k, unsigned ph) {
        constexpr int u = decltype(uc)::value;
        constexpr int sM = (u + 5) % 6, s0 = u, s1 = (u + 1) % 6, s2 = (u + 2) % 6;
        if (tma) {
            if (!mbar_wait_bounded(bar0 + 8u * s2, ph ^ (u >= 4 ? 1u : 0u))) timed_out = true;
        } else {
            cp_async_wait<kPD - 1>();
        }
        __syncthreads();  // e / rho planes <= k+2 and r planes <= k+1 are staged
        // e / rho plane k-2 and r plane k-3 were last read before this step:
        // their slots take the planes two steps ahead
        issue(k + 2 + kPD, k + 1 + kPD, (u + 4) % 6, (u + 3) % 6);
        // red cells of plane kr = k+1 on the tile and its one-cell ring.  A
        // tile thread's black cell of plane k lies in the same column (x, y) as
        // its red cell of plane k+1, and the pair's red cell of plane k is the
        // one it updated in the previous step: those values pass in registers.
        constexpr int HO = kESlots * kEPlane;
        const int kr = k + 1;
        float v_red = 0.f, rc_red = 0.f, hm_red = 0.f;
        const bool red_here = kr >= 0 && kr < nz;
        if (red_here && red_row >= 0) {
            const int fi = fr[u & 1];
            const float* E = Es + s1 * kEPlane;
            const bool lo = kr > 0, hi = kr < nz - 1;
            rc_red = E[HO + fi];
            hm_red = lo ? Es[HO + s0 * kEPlane + fi] : 0.f;
            const float em = lo ? Es[s0 * kEPlane + fi] : 0.f;
            const float hp = hi ? Es[HO + s2 * kEPlane + fi] : 0.f;
            const float ep = hi ? Es[s2 * kEPlane + fi] : 0.f;
            const float rcen = Rs[s1 * kRSlotF + rr[u & 1]];
            v_red = cell_update(E, fi, rc_red, lo, hm_red, em, hi, hp, ep, rcen, h2h);
            if (omega != 1.f) v_red = ops::relax(E[fi], v_red, omega);  // over-relaxation from the old value
            Es[s1 * kEPlane + fi] = v_red;
            // the slot is refilled by TMA later on: order this generic write before it
            if (MODE != kSweepFromZero && tma) fence_proxy_async();
        }
        __syncthreads();  // the red values of plane k+1 are visible
        // black cells of plane k on the tile, written out with their red partners
        if (k >= z0 && black_thread) {
            const int t = tb[u & 1];
            const int fi = fb + t;  // = fr[u & 1]
            const float* E = Es + s0 * kEPlane;
            const bool lo = k > 0, hi = k < nz - 1;  // hi: the red update of plane k+1 ran
            const float rc = red_here ? hm_red : E[HO + fi];
            const float hm = lo ? Es[HO + sM * kEPlane + fi] : 0.f;
            const float em = lo ? Es[sM * kEPlane + fi] : 0.f;
            const float rcen = Rs[s0 * kRSlotF + rb + t];
            float v = cell_update(E, fi, rc, lo, hm, em, hi, rc_red, v_red, rcen, h2h);
            if (omega != 1.f) v = ops::relax(E[fi], v, omega);
            const float red = prev_red;  // the pair's red value of plane k
            const float2 out = t == 0 ? make_float2(v, red) : make_float2(red, v);
            if (MODE == kSweepUpdate) {  // the V-cycle's last sweep: e is not read again
                p_add_pair(pp, out);
                pp += NP;
            } else {
                *o2 = out;
                o2 += NPh;
            }
        }
        prev_red = v_red;
    };
    unsigned ph = 0;
    for (int kb = z0 - 2; kb < z1; kb += 6, ph ^= 1u) {
        step(IC<0>{}, kb, ph);
        if (kb + 1 >= z1) break;
        step(IC<1>{}, kb + 1, ph);
        if (kb + 2 >= z1) break;
        step(IC<2>{}, kb + 2, ph);
        if (kb + 3 >= z1) break;
        step(IC<3>{}, kb + 3, ph);
        if (kb + 4 >= z1) break;
        step(IC<4>{}, kb + 4, ph);
        if (kb + 5 >= z1) break;
        step(IC<5>{}, kb + 5, ph);
    }
    // every call that staged bytes was waited for above (the calls after the
    // last wait stage nothing: their planes lie beyond z1 + 1)
    if (!tma) cp_async_wait<0>();
    if (timed_out) *err = 1.0;
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

namespace {
// cuTensorMapEncodeTiled from the driver, through the runtime's entry-point
// query (no link against the driver library); null if unavailable
PFN_cuTensorMapEncodeTiled_v12000 encode_tiled() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        void* f = nullptr;
        cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess && f)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(f);
        else
            cudaGetLastError();
    }
    return fn;
}
// (nx, ny, nz) FP32 array, x fastest; box kRowF x rows x 1, no swizzle (the
// box lands row after row, kRowF floats a row), zero fill outside the grid
bool encode_plane_map(CUtensorMap* m, const float* base, const Geom& g, int rows) {
    PFN_cuTensorMapEncodeTiled_v12000 fn = encode_tiled();
    if (!fn || !base) return false;
    const cuuint64_t dims[3] = {(cuuint64_t)g.n[0], (cuuint64_t)g.n[1], (cuuint64_t)g.n[2]};
    const cuuint64_t strides[2] = {(cuuint64_t)g.n[0] * sizeof(float), (cuuint64_t)g.NP * sizeof(float)};
    const cuuint32_t box[3] = {(cuuint32_t)kRowF, (cuuint32_t)rows, 1u};
    const cuuint32_t estr[3] = {1u, 1u, 1u};
    return fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<float*>(base), dims, strides, box, estr,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}
}  // namespace

void sweep0_encode_maps(const MGLevel& L, SweepMaps* m) {
    *m = SweepMaps{};
    if (!sweep0_supported(L.g) || !L.e2) return;
    m->ok = encode_plane_map(&m->rho, L.rho0, L.g, kER) && encode_plane_map(&m->e, L.e, L.g, kER) &&
            encode_plane_map(&m->e2, L.e2, L.g, kER) && encode_plane_map(&m->r, L.r, L.g, kRR);
}

// one full red-black sweep of level 0: ein -> eout (ein unused when from_zero),
// or, in update mode, p += the new e (eout not written: nothing reads it); interior tiles stage with TMA when maps is
// non-null and encoded, a wait that runs out sets *err
template <typename T>
void launch_sweep0(const MGLevel& L, const SweepMaps* maps, const float* ein, float* eout, int mode, float omega,
                   PT<T>* p, double* err, cudaStream_t s) {
    const Geom& g = L.g;
    const int zchunk = sweep0_zchunk(g);
    const dim3 grid((unsigned)(g.n[0] / kTX), (unsigned)(g.n[1] / kTY), (unsigned)((g.n[2] + zchunk - 1) / zchunk));
    const float h2h = 0.5f * (float)(g.h * g.h);
    static const SweepMaps none{};
    const bool tma = maps && maps->ok;
    const SweepMaps& m = tma ? *maps : none;
    const CUtensorMap& me = (ein == L.e2) ? m.e2 : m.e;
    const int ut = tma ? 1 : 0;
    if (mode == kSweepFromZero)
        k_sweep0<T, kSweepFromZero><<<grid, kSweepThreads, kSweepSmem, s>>>(g, L.rho0, ein, eout, L.r, h2h, omega, p, zchunk,
                                                                            m.rho, me, m.r, ut, err);
    else if (mode == kSweepUpdate)
        k_sweep0<T, kSweepUpdate><<<grid, kSweepThreads, kSweepSmem, s>>>(g, L.rho0, ein, eout, L.r, h2h, omega, p, zchunk,
                                                                          m.rho, me, m.r, ut, err);
    else
        k_sweep0<T, kSweepPlain><<<grid, kSweepThreads, kSweepSmem, s>>>(g, L.rho0, ein, eout, L.r, h2h, omega, p, zchunk,
                                                                         m.rho, me, m.r, ut, err);
}

template void launch_sweep0<double>(const MGLevel&, const SweepMaps*, const float*, float*, int, float, double*,
                                    double*, cudaStream_t);
template void launch_sweep0<float>(const MGLevel&, const SweepMaps*, const float*, float*, int, float, float2*,
                                   double*, cudaStream_t);

}  // namespace cdi
