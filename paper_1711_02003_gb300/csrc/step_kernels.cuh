// step_kernels.cuh -- the fused per-site, per-step update (arXiv:1711.02003, Eqs. 1-11):
// device code, kernels and launchers, instantiated once per storage format by step_f64.cu,
// step_f32.cu, step_f32dev.cu and step_f16.cu (four translation units compiled in parallel).
//
// One launch performs, for every fluid site x:
//   pull streaming f_i^k(x) <- f_i^k(x - c_i) with halfway bounce-back (Eq. 1),
//   densities, momentum and psi = (rho_R - rho_B)/rho (Eqs. 2-3),
//   the colour gradient F = 3 sum_i w_i psi(x + c_i) c_i (Sec. II),
//   the regularized collision at the mixture relaxation time (Eqs. 5, 6, 11),
//   the perturbation (Eq. 9) and recolouring (Eq. 10),
// reading buffer A (post-collision state of step t) and writing buffer B.
//
// The colour gradient needs psi of the neighbours AFTER streaming, i.e. the
// streamed densities of a one-site ring around each tile.  The kernels recompute
// that ring from A (the ring loads are shared with neighbouring tiles and mostly
// hit L2), so each step reads A once and writes B once from HBM:
//   D2Q9 : one warp owns a strip of 30 sites in x (lanes 1..30; lanes 0 and 31 are
//          the ring) and marches along y.  psi of rows y-1, y, y+1 sits in
//          registers; x-neighbours come from warp shuffles.  No shared memory, no
//          block barrier.
//   D3Q19: one block owns 30 x (WY-2) sites in x-y (ring lanes and ring warps)
//          and marches along z; psi of four z-planes is staged in shared memory.
//
// Element offsets are 32-bit when all 2Q planes fit below 2^31 elements (IDX = int),
// 64-bit otherwise.  Upstream offsets are site-index differences precomputed per
// lane (x), row (y) and plane (z), so periodic wrap costs nothing per direction.
#pragma once
#include <cuda.h>
#include <cudaTypedefs.h>

#include <type_traits>

#include "lbcg_device.cuh"

namespace lbcg {

// Site coordinate along one axis for a lane/row/plane that may sit one beyond the
// box: returns false when the site is outside a closed axis.
__device__ __forceinline__ bool wrap_coord(int v, int n, int per, int& vs)
{
    if (v >= 0 && v < n) {
        vs = v;
        return true;
    }
    if (per) {
        vs = v < 0 ? v + n : v - n;
        return vs >= 0 && vs < n;
    }
    vs = 0;
    return false;
}

// offsets (in sites along this axis) to the upstream neighbours vs-1 and vs+1; a
// neighbour outside a closed axis is clamped to vs (reached only through a
// bounce-back link, so never read)
__device__ __forceinline__ void nbr_off(int vs, int n, int per, int& dm, int& dp)
{
    dm = vs - 1 >= 0 ? -1 : (per ? n - 1 : 0);
    dp = vs + 1 < n ? 1 : (per ? -(n - 1) : 0);
}

// site-index offsets of the upstream neighbours: *m for c_axis = +1 (pull from the
// minus side), *p for c_axis = -1
struct Up {
    int xm, xp;
    long long ym, yp;
    long long zm, zp;
};

template <int LAT, typename IDX>
__device__ __forceinline__ IDX up_off(const Up& u, int i)
{
    using L = Lat<LAT>;
    IDX d = 0;
    if (L::cx(i) > 0) d += (IDX)u.xm;
    if (L::cx(i) < 0) d += (IDX)u.xp;
    if (L::cy(i) > 0) d += (IDX)u.ym;
    if (L::cy(i) < 0) d += (IDX)u.yp;
    if (L::cz(i) > 0) d += (IDX)u.zm;
    if (L::cz(i) < 0) d += (IDX)u.zp;
    return d;
}

// Streamed populations (pull, Eq. 1) of the fluid site s into r/g; returns its psi.
template <int LAT, int PREC, typename IDX>
__device__ __forceinline__ typename Store<PREC>::T pull_fluid(const KParams& P,
                                                              const typename Store<PREC>::S* __restrict__ A, IDX s,
                                                              const Up& u, uint32_t lk,
                                                              typename Store<PREC>::T (&r)[Lat<LAT>::Q],
                                                              typename Store<PREC>::T (&g)[Lat<LAT>::Q])
{
    using L = Lat<LAT>;
    using SP = Store<PREC>;
    using T = typename SP::T;
    constexpr int Q = L::Q;
    const IDX np = (IDX)P.np;
    const Phys<T>& ph = phys<T>(P);
    constexpr uint32_t qmask = (1u << Q) - 1u;
    if ((lk & qmask) == 0u) {
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            const IDX ir = (IDX)i * np + s + up_off<LAT, IDX>(u, i);
            load_pop<PREC, IDX>(P, A, ir, ir + (IDX)Q * np, ph, L::cls(i), r[i], g[i]);
        }
    } else {
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            const bool bounce = (lk >> i) & 1u;
            const IDX ir = bounce ? (IDX)L::opp(i) * np + s : (IDX)i * np + s + up_off<LAT, IDX>(u, i);
            load_pop<PREC, IDX>(P, A, ir, ir + (IDX)Q * np, ph, L::cls(i), r[i], g[i]);
        }
    }
    T rr = r[0], sg = g[0];
#pragma unroll
    for (int i = 1; i < Q; ++i) {
        rr += r[i];
        sg += g[i];
    }
    const T rho = ph.rho0 + sg;
    return (rr - (rho - rr)) / rho;
}

template <int LAT, int PREC, typename IDX>
__device__ __forceinline__ void store_site(const KParams& P, typename Store<PREC>::S* __restrict__ B, IDX s,
                                           const typename Store<PREC>::T (&r)[Lat<LAT>::Q],
                                           const typename Store<PREC>::T (&g)[Lat<LAT>::Q])
{
    using L = Lat<LAT>;
    using T = typename Store<PREC>::T;
    const IDX np = (IDX)P.np;
#pragma unroll
    for (int i = 0; i < L::Q; ++i) {
        const IDX ir = (IDX)i * np + s;
        store_pop<PREC, IDX>(P, B, ir, ir + (IDX)L::Q * np, phys<T>(P), L::cls(i), r[i], g[i]);
    }
}

// Tiles with at least one fluid site, when the geometry has walls: the launch covers only
// those (P.ntiles entries of `tiles`: D2Q9, the linear index of a strip; D3Q19, two ints
// per block tile, the linear index of its x-y column and its z-range z0 | z1 << 16, cut to
// the runs of planes of the column that hold fluid); without a list every tile of the box
// is launched, the z-range of block z being [z * rows, min(z * rows + rows, nz)).
__device__ __forceinline__ bool strip_of(const KParams& P, const int* __restrict__ tiles, int gw, int& sxi, int& syi)
{
    int t = gw;
    if (tiles) {
        if (gw >= P.ntiles) return false;
        t = tiles[gw];
    } else if (gw >= P.nsx * P.nsy) {
        return false;
    }
    sxi = t % P.nsx;
    syi = t / P.nsx;
    return true;
}

__device__ __forceinline__ void block_of(const KParams& P, const int* __restrict__ tiles, int& bx, int& by, int& z0,
                                         int& z1)
{
    if (tiles) {
        const int t = tiles[2 * blockIdx.x];
        const int zr = tiles[2 * blockIdx.x + 1];
        bx = t % P.nsx;
        by = t / P.nsx;
        z0 = zr & 0xffff;
        z1 = zr >> 16;
    } else {
        bx = blockIdx.x;
        by = blockIdx.y;
        z0 = (int)blockIdx.z * P.rows;
        z1 = min(z0 + P.rows, P.nz);
    }
}

// psi-ring access through the bounds checks (ring of 4 planes x the block's threads)
template <typename T>
__device__ __forceinline__ void ring_put(const KParams& P, T* ring, int i, T v)
{
    if (in_bounds(P, i, 4LL * blockDim.x * blockDim.y)) ring[i] = v;
}
template <typename T>
__device__ __forceinline__ T ring_get(const KParams& P, const T* ring, int i)
{
    return in_bounds(P, i, 4LL * blockDim.x * blockDim.y) ? ring[i] : T(0);
}

// port tables of a fused refill (D3Q19 tiles, D2Q9 strips) and the ghost-psi tables of the
// input and output buffers (the refill and its tables are described with refill_tile_ports)
struct PortTab {
    const int* tab;     // ghost table [4][ng] (site, inward neighbour, port, kind) or nullptr
    const double* gu;   // [5][ng] inlet velocity, port density, port psi
    int ng;
    const int* gstart;  // [ntiles + 1] first row in grow of each tile
    const int* grow;    // ghost-table rows grouped by tile
    const void* gpsi_in;  // ghost-psi table of the input buffer (compute type) or nullptr
    void* gpsi_out;       // of the output buffer, written by the refill, or nullptr
};

// psi of the port site s (link word lk) from the input buffer's ghost-psi table, else from
// the ghost's populations
template <int LAT, int PREC, typename IDX>
__device__ __forceinline__ typename Store<PREC>::T port_psi(const KParams& P,
                                                            const typename Store<PREC>::S* __restrict__ A, IDX s,
                                                            uint32_t lk, const typename Store<PREC>::T* gpsi, int ng)
{
    if (gpsi) {
        const int t = (int)(lk & kGhostMask);
        if (in_bounds(P, t, ng)) return gpsi[t];
    }
    return ghost_psi<LAT, PREC, IDX>(P, A, s);
}

// ------------------------------------------------------------------------ D2Q9
// one warp: the strip (sxi, syi) of 30 x rows sites
template <int PREC, typename IDX>
__device__ __forceinline__ void strip_d2q9(const KParams& P, const typename Store<PREC>::S* __restrict__ A,
                                           typename Store<PREC>::S* __restrict__ B, const uint32_t* __restrict__ link,
                                           int sxi, int syi, const typename Store<PREC>::T* __restrict__ gpsi_in,
                                           int gpsi_n)
{
    using T = typename Store<PREC>::T;
    using L = Lat<0>;
    constexpr int Q = 9;
    const int lane = threadIdx.x & 31;
    const int nx = P.nx, ny = P.ny;
    const int x = sxi * 30 + lane - 1;
    int xs;
    const bool xok = wrap_coord(x, nx, P.per[0], xs) && x <= nx;
    const bool xint = lane >= 1 && lane <= 30 && x < nx;
    Up u;
    nbr_off(xs, nx, P.per[0], u.xm, u.xp);
    u.zm = u.zp = 0;
    const int y0 = syi * P.rows;
    const int y1 = min(y0 + P.rows, ny);
    const T psi_wall = phys<T>(P).psi_wall;

    T psi_a = psi_wall, psi_b = psi_wall;  // rows yy-2, yy-1
    T rb[Q], gb[Q];                        // populations of row yy-1
    bool coll_b = false;
    IDX s_b = 0;
#pragma unroll
    for (int i = 0; i < Q; ++i) rb[i] = gb[i] = T(0);

#pragma unroll 2
    for (int yy = y0 - 1; yy <= y1; ++yy) {
        int ys;
        const bool yok = wrap_coord(yy, ny, P.per[1], ys);
        int dym, dyp;
        nbr_off(ys, ny, P.per[1], dym, dyp);
        u.ym = (long long)dym * nx;
        u.yp = (long long)dyp * nx;
        T rn[Q], gn[Q];  // set for fluid sites, the only ones collided
        T psi_n = psi_wall;
        bool fluid_n = false;
        const IDX s = (IDX)xs + (IDX)nx * (IDX)ys;
        if (xok && yok) {
            const uint32_t lk = load_link(P, link, s);
            const uint32_t type = (lk >> kTypeShift) & 3u;
            if (type == kTypeFluid) {
                psi_n = pull_fluid<0, PREC, IDX>(P, A, s, u, lk, rn, gn);
                fluid_n = true;
            } else if (type == kTypePort) {
                psi_n = port_psi<0, PREC, IDX>(P, A, s, lk, gpsi_in, gpsi_n);
            }
        }
        if (yy - 1 >= y0) {  // warp-uniform: collide row yy-1
            const T am = __shfl_up_sync(0xffffffffu, psi_a, 1), ap = __shfl_down_sync(0xffffffffu, psi_a, 1);
            const T bm = __shfl_up_sync(0xffffffffu, psi_b, 1), bp = __shfl_down_sync(0xffffffffu, psi_b, 1);
            const T nm = __shfl_up_sync(0xffffffffu, psi_n, 1), np_ = __shfl_down_sync(0xffffffffu, psi_n, 1);
            if (coll_b) {
                // F = 3 sum_p w_p (psi(x + c_p) - psi(x - c_p)) c_p; rows by cy: -1 a, 0 b, +1 n
                auto nb = [&](int cx, int cy) -> T {
                    return cy < 0 ? (cx < 0 ? am : (cx > 0 ? ap : psi_a))
                         : cy > 0 ? (cx < 0 ? nm : (cx > 0 ? np_ : psi_n))
                                  : (cx < 0 ? bm : (cx > 0 ? bp : psi_b));
                };
                T F[3] = {T(0), T(0), T(0)};
#pragma unroll
                for (int k = 0; k < L::NP; ++k) {
                    const int p = L::rep(k);
                    const int cx = L::cx(p), cy = L::cy(p);
                    const T d = (T)L::w(p) * (nb(cx, cy) - nb(-cx, -cy));
                    if (cx) F[0] += cx > 0 ? d : -d;
                    if (cy) F[1] += cy > 0 ? d : -d;
                }
                F[0] *= T(3);
                F[1] *= T(3);
                collide_site<0, T>(P, phys<T>(P), rb, gb, F);
                store_site<0, PREC, IDX>(P, B, s_b, rb, gb);
            }
        }
        psi_a = psi_b;
        psi_b = psi_n;
        coll_b = fluid_n && xint && yy >= y0 && yy < y1;
        s_b = s;
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            rb[i] = rn[i];
            gb[i] = gn[i];
        }
    }
}

// Fused port refill of a D2Q9 strip march: the ghosts whose inward neighbour x' lies in strip
// `strip` of the active list (rows gstart[strip] .. gstart[strip + 1] - 1 of grow), rebuilt
// by the warp that has just written every x' of the strip, one lane per ghost
template <int PREC>
__device__ __forceinline__ void refill_strip_ports(const KParams& P, typename Store<PREC>::S* B, const PortTab& pt,
                                                   int strip)
{
    const int g0 = pt.gstart[strip], g1 = pt.gstart[strip + 1];
    if (g0 >= g1) return;  // warp-uniform
    __syncwarp();          // the populations of every x' of the strip are written
    for (int e = g0 + (int)(threadIdx.x & 31); e < g1; e += 32)
        fill_one<0, PREC>(P, B, pt.tab, pt.gu, pt.ng, pt.grow[e], (typename Store<PREC>::T*)pt.gpsi_out);
}

// PORTS: compiled with the fused port refill (launched for boxes with ports)
template <int PREC, typename IDX, bool PORTS>
__global__ void __launch_bounds__(256) k_step_d2q9(const KParams P, const typename Store<PREC>::S* __restrict__ A,
                                                   typename Store<PREC>::S* __restrict__ B,
                                                   const uint32_t* __restrict__ link, const int* __restrict__ tiles,
                                                   const PortTab pt)
{
    const int gw = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    int sxi, syi;
    if (!strip_of(P, tiles, gw, sxi, syi)) return;  // warp-uniform
    strip_d2q9<PREC, IDX>(P, A, B, link, sxi, syi, (const typename Store<PREC>::T*)pt.gpsi_in, pt.ng);
    if (PORTS && pt.tab) refill_strip_ports<PREC>(P, B, pt, gw);
}

// ----------------------------------------------------------------------- D3Q19
// blockDim = (32, WY); warp w owns row y = by*(WY-2) + w - 1; rows 1..WY-2 collide.
// one block: the tile (bx, by) of 30 x (WY-2) sites over the planes [z0, z1); psi_s holds
// 4 * WY * 32 values of shared memory
template <int PREC, bool KEEP, typename IDX>
__device__ __forceinline__ void tile_d3q19(const KParams& P, const typename Store<PREC>::S* __restrict__ A,
                                           typename Store<PREC>::S* __restrict__ B, const uint32_t* __restrict__ link,
                                           int bx, int by, int z0, int z1, typename Store<PREC>::T* psi_s)
{
    using T = typename Store<PREC>::T;
    using L = Lat<1>;
    constexpr int Q = 19;
    const int lane = threadIdx.x;
    const int w = threadIdx.y;
    const int WY = blockDim.y;
    const int nx = P.nx, ny = P.ny, nz = P.nz;
    const long long nxy = (long long)nx * ny;
    const int x = bx * 30 + lane - 1;
    const int y = by * (WY - 2) + w - 1;
    int xs, ys;
    const bool xok = wrap_coord(x, nx, P.per[0], xs) && x <= nx;
    const bool yok = wrap_coord(y, ny, P.per[1], ys) && y <= ny;
    const bool inner = lane >= 1 && lane <= 30 && x < nx && w >= 1 && w <= WY - 2 && y < ny;
    Up u;
    {
        int a, b;
        nbr_off(xs, nx, P.per[0], u.xm, u.xp);
        nbr_off(ys, ny, P.per[1], a, b);
        u.ym = (long long)a * nx;
        u.yp = (long long)b * nx;
    }
    const IDX sxy = (IDX)xs + (IDX)nx * (IDX)ys;
    const T psi_wall = phys<T>(P).psi_wall;

    T rb[Q], gb[Q];
    bool coll_b = false;
#pragma unroll
    for (int i = 0; i < Q; ++i) rb[i] = gb[i] = T(0);

#pragma unroll 2
    for (int zz = z0 - 1; zz <= z1; ++zz) {
        int zs;
        const bool zok = wrap_coord(zz, nz, P.per[2], zs);
        {
            int a, b;
            nbr_off(zs, nz, P.per[2], a, b);
            u.zm = (long long)a * nxy;
            u.zp = (long long)b * nxy;
        }
        T rn[Q], gn[Q];  // set for fluid sites, the only ones collided
        T psi_n = psi_wall;
        bool fluid_n = false;
        const IDX s = sxy + (IDX)nxy * (IDX)zs;
        if (xok && yok && zok) {
            const uint32_t lk = load_link(P, link, s);
            const uint32_t type = (lk >> kTypeShift) & 3u;
            if (type == kTypeFluid) {
                psi_n = pull_fluid<1, PREC, IDX>(P, A, s, u, lk, rn, gn);
                fluid_n = true;
            } else if (type == kTypePort) {
                psi_n = ghost_psi<1, PREC, IDX>(P, A, s);
            }
        }
        const int slot_n = (zz - z0 + 1) & 3;
        ring_put(P, psi_s, (slot_n * WY + w) * 32 + lane, psi_n);
        __syncthreads();
        if (zz - 1 >= z0 && coll_b) {
            const int zc = zz - 1;
            const IDX sc = sxy + (IDX)nxy * (IDX)zc;
            if (!KEEP) {
                int a, b;
                nbr_off(zc, nz, P.per[2], a, b);
                Up uc = u;
                uc.zm = (long long)a * nxy;
                uc.zp = (long long)b * nxy;
                const uint32_t lk = load_link(P, link, sc);
                pull_fluid<1, PREC, IDX>(P, A, sc, uc, lk, rb, gb);
            }
            auto nb = [&](int cx, int cy, int cz) -> T {
                const int slot = (zc + cz - z0 + 1) & 3;
                return ring_get(P, psi_s, (slot * WY + (w + cy)) * 32 + (lane + cx));
            };
            T F[3] = {T(0), T(0), T(0)};
#pragma unroll
            for (int k = 0; k < L::NP; ++k) {
                const int p = L::rep(k);
                const int cx = L::cx(p), cy = L::cy(p), cz = L::cz(p);
                const T d = (T)L::w(p) * (nb(cx, cy, cz) - nb(-cx, -cy, -cz));
                if (cx) F[0] += cx > 0 ? d : -d;
                if (cy) F[1] += cy > 0 ? d : -d;
                if (cz) F[2] += cz > 0 ? d : -d;
            }
            F[0] *= T(3);
            F[1] *= T(3);
            F[2] *= T(3);
            collide_site<1, T>(P, phys<T>(P), rb, gb, F);
            store_site<1, PREC, IDX>(P, B, sc, rb, gb);
        }
        coll_b = fluid_n && inner && zz >= z0 && zz < z1;
        if (KEEP) {
#pragma unroll
            for (int i = 0; i < Q; ++i) {
                rb[i] = rn[i];
                gb[i] = gn[i];
            }
        }
    }
}

template <int PREC, bool KEEP, typename IDX>
__global__ void __launch_bounds__(256, 2) k_step_d3q19(const KParams P,
                                                       const typename Store<PREC>::S* __restrict__ A,
                                                       typename Store<PREC>::S* __restrict__ B,
                                                       const uint32_t* __restrict__ link, const int* __restrict__ tiles)
{
    extern __shared__ unsigned char smem_raw[];
    int bx, by, z0, z1;
    block_of(P, tiles, bx, by, z0, z1);
    tile_d3q19<PREC, KEEP, IDX>(P, A, B, link, bx, by, z0, z1, reinterpret_cast<typename Store<PREC>::T*>(smem_raw));
}

// variant 5: re-read variant compiled for three resident blocks per SM (<= 85 registers)
template <int PREC, typename IDX>
__global__ void __launch_bounds__(256, 3) k_step_d3q19_occ(const KParams P,
                                                           const typename Store<PREC>::S* __restrict__ A,
                                                           typename Store<PREC>::S* __restrict__ B,
                                                           const uint32_t* __restrict__ link, const int* __restrict__ tiles)
{
    extern __shared__ unsigned char smem_raw[];
    int bx, by, z0, z1;
    block_of(P, tiles, bx, by, z0, z1);
    tile_d3q19<PREC, false, IDX>(P, A, B, link, bx, by, z0, z1, reinterpret_cast<typename Store<PREC>::T*>(smem_raw));
}

// ------------------------------------------------------------ fused port refill
// A step kernel that refills port ghosts itself: the host assigns every ghost to the block
// tile that collides its inward neighbour x' (rows gstart[t] .. gstart[t+1]-1 of grow are the
// ghost-table rows of tile t).  After its tile, a block holding such ghosts rebuilds them in
// the output buffer from the populations of x' its threads have just written there (fill_one,
// the rule of the separate refill, one thread per ghost), so the next step finds them
// refilled without a refill launch.
//
// Ghost-psi table: the refill also stores each ghost's psi (computed from the values it has
// just written, in compute precision) in a per-buffer table, and the link word of a port site
// carries its ghost-table row.  A port lane of the march then reads one value instead of
// pulling the ghost's 2Q populations in a branch of its own, which the fluid lanes of the same
// warp would wait through.


template <int PREC>
__device__ __forceinline__ void refill_tile_ports(const KParams& P, typename Store<PREC>::S* B, const PortTab& pt,
                                                  int tile)
{
    const int g0 = pt.gstart[tile], g1 = pt.gstart[tile + 1];
    if (g0 >= g1) return;  // block-uniform
    __syncthreads();       // the populations of every x' of the tile are written
    const int nt = blockDim.x * blockDim.y;
    for (int e = g0 + threadIdx.y * blockDim.x + threadIdx.x; e < g1; e += nt)
        fill_one<1, PREC>(P, B, pt.tab, pt.gu, pt.ng, pt.grow[e], (typename Store<PREC>::T*)pt.gpsi_out);
}

// ---------------------------------------------------------- neighbour-only plane barrier
// Warp w of a march reads the psi rows of warps w - 1 and w + 1 only, so instead of a block
// barrier per plane the warps exchange signals with their two neighbours through named
// barriers of 64 threads: B_w (id 1 + w) carries w's "psi written" to w + 1, A_w (id WY + w)
// carries w + 1's to w.  Each warp signals up, waits on the warp below, signals down, waits
// on the warp above: no warp's signal depends on another warp's wait (no chain), and a warp
// signals a barrier again only after its partner has consumed the previous generation.  A
// warp runs at most one plane ahead of its neighbours, which the four-slot psi ring allows.
// Needs 2 (WY - 1) <= 15 barriers: WY <= 8.
__device__ __forceinline__ void bar_arrive(int id, int n)
{
    asm volatile("bar.arrive %0, %1;" ::"r"(id), "r"(n) : "memory");
}
__device__ __forceinline__ void bar_sync_n(int id, int n)
{
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(n) : "memory");
}
__device__ __forceinline__ void neighbour_sync(int w, int WY)
{
    if (w < WY - 1) bar_arrive(1 + w, 64);        // psi of w written: tell w + 1
    if (w > 0) bar_sync_n(w, 64);                 // w - 1 has written
    if (w > 0) bar_arrive(WY + w - 1, 64);        // tell w - 1
    if (w < WY - 1) bar_sync_n(WY + w, 64);       // w + 1 has written
}

// ------------------------------------------------- moment march (variants 6, 7; regularized)
template <typename T>
__device__ __forceinline__ void mom_put(const SiteMom<T>& m, T* p, int st)
{
    p[0] = m.rr;
    p[st] = m.sg;
    p[2 * st] = m.jx;
    p[3 * st] = m.jy;
    p[4 * st] = m.jz;
    p[5 * st] = m.pxx;
    p[6 * st] = m.pyy;
    p[7 * st] = m.pzz;
    p[8 * st] = m.pxy;
    p[9 * st] = m.pxz;
    p[10 * st] = m.pyz;
}

template <typename T>
__device__ __forceinline__ void mom_get(SiteMom<T>& m, const T* p, int st)
{
    m.rr = p[0];
    m.sg = p[st];
    m.jx = p[2 * st];
    m.jy = p[3 * st];
    m.jz = p[4 * st];
    m.pxx = p[5 * st];
    m.pyy = p[6 * st];
    m.pzz = p[7 * st];
    m.pxy = p[8 * st];
    m.pxz = p[9 * st];
    m.pyz = p[10 * st];
}

// Streamed populations of one fluid site summed into the moments of the regularized
// collision as they arrive (pull, Eq. 1, halfway bounce-back on the link bits); returns
// psi.  FULL = false: only rho_R and rho (psi of a ring site).
template <int LAT, int PREC, typename IDX, bool FULL>
__device__ __forceinline__ typename Store<PREC>::T pull_moments(const KParams& P,
                                                                const typename Store<PREC>::S* __restrict__ A, IDX s,
                                                                const Up& u, uint32_t lk,
                                                                SiteMom<typename Store<PREC>::T>& m)
{
    using L = Lat<LAT>;
    using SP = Store<PREC>;
    using T = typename SP::T;
    constexpr int Q = L::Q;
    const IDX np = (IDX)P.np;
    const Phys<T>& ph = phys<T>(P);
    constexpr uint32_t qmask = (1u << Q) - 1u;
    auto body = [&](auto walls) {
        constexpr bool WALLS = decltype(walls)::value;
        auto ld = [&](int i, T& r, T& g) {
            IDX ir = (IDX)i * np + s + up_off<LAT, IDX>(u, i);
            if (WALLS && ((lk >> i) & 1u)) ir = (IDX)L::opp(i) * np + s;
            load_pop<PREC, IDX>(P, A, ir, ir + (IDX)Q * np, ph, L::cls(i), r, g);
        };
        T r0, g0;
        ld(0, r0, g0);
        m.rr = r0;
        m.sg = g0;
#pragma unroll
        for (int k = 0; k < L::NP; ++k) {
            const int p = L::rep(k);
            T rp, gp, rq, gq;
            ld(p, rp, gp);
            ld(L::opp(p), rq, gq);
            mom_add_pair<LAT, FULL>(m, k, rp, gp, rq, gq);
        }
    };
    // one body per warp: the bounce-back body is right for every site, so a warp with any
    // bounced link takes it for all its lanes instead of running both bodies one after the other
    if (!__any_sync(__activemask(), (lk & qmask) != 0u))
        body(std::false_type{});
    else
        body(std::true_type{});
    const T rho = ph.rho0 + m.sg;
    return (m.rr - (rho - m.rr)) / rho;
}

// The block tile of tile_d3q19, marching along z, with the waiting plane held as its
// 11 moments: plane z+1 is pulled and summed (psi to the shared ring), then plane z
// is collided from its moments and written.  No population is read twice from the
// memory system and no population array lives in registers.  Regularized collision
// only (the BGK update needs the individual populations).  MSMEM parks the waiting
// moments in a thread-private shared-memory slot (two slots, alternating by plane)
// instead of registers, for a smaller register budget.
template <int PREC, typename IDX, bool MSMEM, bool PAIR = false>
__device__ __forceinline__ void tile_d3q19_mom(const KParams& P, const typename Store<PREC>::S* __restrict__ A,
                                               typename Store<PREC>::S* __restrict__ B,
                                               const uint32_t* __restrict__ link, int bx, int by, int z0, int z1,
                                               typename Store<PREC>::T* psi_s,
                                               const typename Store<PREC>::T* __restrict__ gpsi_in, int gpsi_n)
{
    using T = typename Store<PREC>::T;
    using SP = Store<PREC>;
    using L = Lat<1>;
    constexpr int Q = 19;
    const int lane = threadIdx.x;
    const int w = threadIdx.y;
    const int WY = blockDim.y;
    const int nx = P.nx, ny = P.ny, nz = P.nz;
    const long long nxy = (long long)nx * ny;
    const int x = bx * 30 + lane - 1;
    const int y = by * (WY - 2) + w - 1;
    int xs, ys;
    const bool xok = wrap_coord(x, nx, P.per[0], xs) && x <= nx;
    const bool yok = wrap_coord(y, ny, P.per[1], ys) && y <= ny;
    const bool row_in = w >= 1 && w <= WY - 2 && y < ny;  // warp-uniform
    const bool inner = row_in && lane >= 1 && lane <= 30 && x < nx;
    Up u;
    {
        int a, b;
        nbr_off(xs, nx, P.per[0], u.xm, u.xp);
        nbr_off(ys, ny, P.per[1], a, b);
        u.ym = (long long)a * nx;
        u.yp = (long long)b * nx;
    }
    const IDX sxy = (IDX)xs + (IDX)nx * (IDX)ys;
    const IDX np = (IDX)P.np;
    const Phys<T>& ph = phys<T>(P);
    const T psi_wall = ph.psi_wall;

    SiteMom<T> mb;
    mom_zero(mb);
    bool coll_b = false;
    T* const mom_s = psi_s + 4 * WY * 32 + (w * 32 + lane);  // [slot][11][WY * 32]
    const int mstride = WY * 32;

#pragma unroll 1
    for (int zz = z0 - 1; zz <= z1; ++zz) {
        int zs;
        const bool zok = wrap_coord(zz, nz, P.per[2], zs);
        {
            int a, b;
            nbr_off(zs, nz, P.per[2], a, b);
            u.zm = (long long)a * nxy;
            u.zp = (long long)b * nxy;
        }
        SiteMom<T> mn;
        mom_zero(mn);
        T psi_n = psi_wall;
        bool fluid_n = false;
        const IDX s = sxy + (IDX)nxy * (IDX)zs;
        const bool full = row_in && zz >= z0 && zz < z1;  // block-uniform in z, warp-uniform in y
        if (xok && yok && zok) {
            const uint32_t lk = load_link(P, link, s);
            const uint32_t type = (lk >> kTypeShift) & 3u;
            if (type == kTypeFluid) {
                psi_n = full ? pull_moments<1, PREC, IDX, true>(P, A, s, u, lk, mn)
                             : pull_moments<1, PREC, IDX, false>(P, A, s, u, lk, mn);
                fluid_n = true;
            } else if (type == kTypePort) {
                psi_n = port_psi<1, PREC, IDX>(P, A, s, lk, gpsi_in, gpsi_n);
            }
        }
        const int slot_n = (zz - z0 + 1) & 3;
        ring_put(P, psi_s, (slot_n * WY + w) * 32 + lane, psi_n);
        if (MSMEM && fluid_n && full) mom_put(mn, mom_s + (zz & 1) * 11 * mstride, mstride);
        if (PAIR && WY <= 8)
            neighbour_sync(w, WY);
        else
            __syncthreads();
        if (zz - 1 >= z0 && coll_b) {
            const int zc = zz - 1;
            const IDX sc = sxy + (IDX)nxy * (IDX)zc;
            auto nb = [&](int cx, int cy, int cz) -> T {
                const int slot = (zc + cz - z0 + 1) & 3;
                return ring_get(P, psi_s, (slot * WY + (w + cy)) * 32 + (lane + cx));
            };
            T F[3] = {T(0), T(0), T(0)};
#pragma unroll
            for (int k = 0; k < L::NP; ++k) {
                const int p = L::rep(k);
                const int cx = L::cx(p), cy = L::cy(p), cz = L::cz(p);
                const T d = (T)L::w(p) * (nb(cx, cy, cz) - nb(-cx, -cy, -cz));
                if (cx) F[0] += cx > 0 ? d : -d;
                if (cy) F[1] += cy > 0 ? d : -d;
                if (cz) F[2] += cz > 0 ? d : -d;
            }
            F[0] *= T(3);
            F[1] *= T(3);
            F[2] *= T(3);
            if (MSMEM) mom_get(mb, mom_s + (zc & 1) * 11 * mstride, mstride);
            collide_moments<1, T>(ph, mb, F, [&](int i, T r, T g) {
                const IDX ir = (IDX)i * np + sc;
                store_pop<PREC, IDX>(P, B, ir, ir + (IDX)Q * np, ph, L::cls(i), r, g);
            });
        }
        coll_b = fluid_n && inner && zz >= z0 && zz < z1;
        if (!MSMEM) mb = mn;
    }
}

// PORTS: compiled with the fused port refill (launched for boxes with ports; without, the
// kernel carries no refill code and keeps the march's register allocation to itself)
// variant 6: moments in registers; three blocks per SM (FP64: two, at 128 registers).  With
// per-tile ghost lists the kernel refills the port ghosts itself (refill_tile_ports).
template <int PREC, typename IDX, bool PORTS>
__global__ void __launch_bounds__(256, PREC == LBCG_FP64 ? 2 : 3) k_step_d3q19_mom(const KParams P,
                                                           const typename Store<PREC>::S* __restrict__ A,
                                                           typename Store<PREC>::S* __restrict__ B,
                                                           const uint32_t* __restrict__ link, const int* __restrict__ tiles,
                                                           const PortTab pt)
{
    extern __shared__ unsigned char smem_raw[];
    int bx, by, z0, z1;
    block_of(P, tiles, bx, by, z0, z1);
    tile_d3q19_mom<PREC, IDX, false>(P, A, B, link, bx, by, z0, z1, reinterpret_cast<typename Store<PREC>::T*>(smem_raw),
                                     (const typename Store<PREC>::T*)pt.gpsi_in, pt.ng);
    if (PORTS && pt.tab) refill_tile_ports<PREC>(P, B, pt, (int)blockIdx.x);
}

// variant 9: variant 6 with neighbour-only plane barriers
template <int PREC, typename IDX, bool PORTS>
__global__ void __launch_bounds__(256, PREC == LBCG_FP64 ? 2 : 3) k_step_d3q19_momn(const KParams P,
                                                           const typename Store<PREC>::S* __restrict__ A,
                                                           typename Store<PREC>::S* __restrict__ B,
                                                           const uint32_t* __restrict__ link, const int* __restrict__ tiles,
                                                           const PortTab pt)
{
    extern __shared__ unsigned char smem_raw[];
    int bx, by, z0, z1;
    block_of(P, tiles, bx, by, z0, z1);
    tile_d3q19_mom<PREC, IDX, false, true>(P, A, B, link, bx, by, z0, z1,
                                           reinterpret_cast<typename Store<PREC>::T*>(smem_raw),
                                           (const typename Store<PREC>::T*)pt.gpsi_in, pt.ng);
    if (PORTS && pt.tab) refill_tile_ports<PREC>(P, B, pt, (int)blockIdx.x);
}

// variant 7: the moment march with the waiting moments in shared memory; 64 registers, so
// four blocks of 8 warps or two of 16 per SM; refills port ghosts like variant 6
template <int PREC, typename IDX, bool PORTS>
__global__ void __launch_bounds__(512, 2) k_step_d3q19_moms(const KParams P,
                                                                const typename Store<PREC>::S* __restrict__ A,
                                                                typename Store<PREC>::S* __restrict__ B,
                                                                const uint32_t* __restrict__ link,
                                                                const int* __restrict__ tiles, const PortTab pt)
{
    extern __shared__ unsigned char smem_raw[];
    int bx, by, z0, z1;
    block_of(P, tiles, bx, by, z0, z1);
    tile_d3q19_mom<PREC, IDX, true>(P, A, B, link, bx, by, z0, z1, reinterpret_cast<typename Store<PREC>::T*>(smem_raw),
                                    (const typename Store<PREC>::T*)pt.gpsi_in, pt.ng);
    if (PORTS && pt.tab) refill_tile_ports<PREC>(P, B, pt, (int)blockIdx.x);
}

// ------------------------------------------------ D2Q9 moment march (2D variant 6)
// strip_d2q9 with the waiting row held as the moments of the regularized collision (7 numbers
// in 2D) instead of its 2Q populations; regularized collision only.
template <int PREC, typename IDX>
__device__ __forceinline__ void strip_d2q9_mom(const KParams& P, const typename Store<PREC>::S* __restrict__ A,
                                               typename Store<PREC>::S* __restrict__ B,
                                               const uint32_t* __restrict__ link, int sxi, int syi,
                                               const typename Store<PREC>::T* __restrict__ gpsi_in, int gpsi_n)
{
    using T = typename Store<PREC>::T;
    using SP = Store<PREC>;
    using L = Lat<0>;
    constexpr int Q = 9;
    const int lane = threadIdx.x & 31;
    const int nx = P.nx, ny = P.ny;
    const int x = sxi * 30 + lane - 1;
    int xs;
    const bool xok = wrap_coord(x, nx, P.per[0], xs) && x <= nx;
    const bool xint = lane >= 1 && lane <= 30 && x < nx;
    Up u;
    nbr_off(xs, nx, P.per[0], u.xm, u.xp);
    u.zm = u.zp = 0;
    const int y0 = syi * P.rows;
    const int y1 = min(y0 + P.rows, ny);
    const IDX np = (IDX)P.np;
    const Phys<T>& ph = phys<T>(P);
    const T psi_wall = ph.psi_wall;

    T psi_a = psi_wall, psi_b = psi_wall;  // rows yy-2, yy-1
    SiteMom<T> mb;                         // moments of row yy-1
    mom_zero(mb);
    bool coll_b = false;
    IDX s_b = 0;

#pragma unroll 1
    for (int yy = y0 - 1; yy <= y1; ++yy) {
        int ys;
        const bool yok = wrap_coord(yy, ny, P.per[1], ys);
        int dym, dyp;
        nbr_off(ys, ny, P.per[1], dym, dyp);
        u.ym = (long long)dym * nx;
        u.yp = (long long)dyp * nx;
        SiteMom<T> mn;
        mom_zero(mn);
        T psi_n = psi_wall;
        bool fluid_n = false;
        const IDX s = (IDX)xs + (IDX)nx * (IDX)ys;
        if (xok && yok) {
            const uint32_t lk = load_link(P, link, s);
            const uint32_t type = (lk >> kTypeShift) & 3u;
            if (type == kTypeFluid) {
                psi_n = pull_moments<0, PREC, IDX, true>(P, A, s, u, lk, mn);
                fluid_n = true;
            } else if (type == kTypePort) {
                psi_n = port_psi<0, PREC, IDX>(P, A, s, lk, gpsi_in, gpsi_n);
            }
        }
        if (yy - 1 >= y0) {  // warp-uniform: collide row yy-1
            const T am = __shfl_up_sync(0xffffffffu, psi_a, 1), ap = __shfl_down_sync(0xffffffffu, psi_a, 1);
            const T bm = __shfl_up_sync(0xffffffffu, psi_b, 1), bp = __shfl_down_sync(0xffffffffu, psi_b, 1);
            const T nm = __shfl_up_sync(0xffffffffu, psi_n, 1), np_ = __shfl_down_sync(0xffffffffu, psi_n, 1);
            if (coll_b) {
                auto nb = [&](int cx, int cy) -> T {
                    return cy < 0 ? (cx < 0 ? am : (cx > 0 ? ap : psi_a))
                         : cy > 0 ? (cx < 0 ? nm : (cx > 0 ? np_ : psi_n))
                                  : (cx < 0 ? bm : (cx > 0 ? bp : psi_b));
                };
                T F[3] = {T(0), T(0), T(0)};
#pragma unroll
                for (int k = 0; k < L::NP; ++k) {
                    const int p = L::rep(k);
                    const int cx = L::cx(p), cy = L::cy(p);
                    const T d = (T)L::w(p) * (nb(cx, cy) - nb(-cx, -cy));
                    if (cx) F[0] += cx > 0 ? d : -d;
                    if (cy) F[1] += cy > 0 ? d : -d;
                }
                F[0] *= T(3);
                F[1] *= T(3);
                collide_moments<0, T>(ph, mb, F, [&](int i, T r, T g) {
                    const IDX ir = (IDX)i * np + s_b;
                    store_pop<PREC, IDX>(P, B, ir, ir + (IDX)Q * np, ph, L::cls(i), r, g);
                });
            }
        }
        psi_a = psi_b;
        psi_b = psi_n;
        coll_b = fluid_n && xint && yy >= y0 && yy < y1;
        s_b = s;
        mb = mn;
    }
}

template <int PREC, typename IDX, bool PORTS>
__global__ void __launch_bounds__(256) k_step_d2q9_mom(const KParams P, const typename Store<PREC>::S* __restrict__ A,
                                                       typename Store<PREC>::S* __restrict__ B,
                                                       const uint32_t* __restrict__ link,
                                                       const int* __restrict__ tiles, const PortTab pt)
{
    const int gw = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    int sxi, syi;
    if (!strip_of(P, tiles, gw, sxi, syi)) return;  // warp-uniform
    strip_d2q9_mom<PREC, IDX>(P, A, B, link, sxi, syi, (const typename Store<PREC>::T*)pt.gpsi_in, pt.ng);
    if (PORTS && pt.tab) refill_strip_ports<PREC>(P, B, pt, gw);
}

// ------------------------------------------- TMA-staged moment march (variant 8)
// The moment march of tile_d3q19_mom with its pulls served from shared memory.  For every
// pulled plane, warp 0 of the block asks the tensor memory accelerator for Q boxes, one
// per direction holding both of its arrays: the 36 x WY floats the block's threads pull,
// the rows and the plane already shifted by the direction's c_y and c_z, the x-range
// starting at the 16-byte boundary at or below the shifted first lane.  Two stages: the boxes of
// plane z+2 load while plane z+1 is summed and plane z collided.  A thread reads its 2Q
// pulled values at fixed shared-memory offsets: no per-load address arithmetic and no
// global-load latency of its own.  Global loads remain only where a box cannot serve the
// pull: bounce-back links (the site's own opposite population) and upstream sites across
// a periodic x or y edge (a box does not wrap; its out-of-range part is zero-filled and
// never read).  Every pipeline wait is bounded: on timeout the block records it in the
// status word, waits (bounded) for its copies in flight and returns.  Requirements: 4-byte
// storage, regularized collision, nx a multiple of 4 (row stride a multiple of 16 bytes),
// 32-bit element offsets.

constexpr int kTmaBoxX = 36;            // floats per staged row: 32 lanes + up to 3 of shift
constexpr int kTmaWaitLimit = 1 << 22;  // mbarrier polls before a wait gives up
constexpr int kTmaStallLimit = 1 << 12; // the same in the failure-path test

template <int WY>
struct TmaLayout {
    static constexpr int ROWS = kTmaBoxX * WY;             // floats of one array's rows
    static constexpr int BOX = 2 * ROWS * 4;               // bytes of one box: both arrays
    static constexpr int SLOT = (BOX + 127) / 128 * 128;   // 128-byte aligned box slot
    static constexpr int SLOTF = SLOT / 4;                 // floats per slot
    static constexpr int STAGE = 19 * SLOT;                // the Q boxes of one plane
    static constexpr int PSI = 4 * WY * 32 * 4;            // psi ring
    static constexpr int BYTES = 2 * STAGE + PSI + 16;     // + two mbarriers
};

__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0u;
}

// count `bytes` of the current phase's expected transaction bytes as arrived
__device__ __forceinline__ void mbar_complete_tx(uint64_t* bar, uint32_t bytes)
{
    asm volatile("mbarrier.complete_tx.relaxed.cta.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}

// bounded wait for the phase with the given parity to complete; false after `limit` polls
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, int limit)
{
    for (int k = 0; k < limit; ++k)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}

__device__ __forceinline__ void tma_load_5d(void* dst, const CUtensorMap* map, uint64_t* bar, int x, int y, int z,
                                            int i, int k)
{
    asm volatile(
        "cp.async.bulk.tensor.5d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, "
        "%5, %6}], [%7];" ::"r"(smem_addr(dst)),
        "l"(map), "r"(x), "r"(y), "r"(z), "r"(i), "r"(k), "r"(smem_addr(bar))
        : "memory");
}

// Pulled populations of one fluid site from the staged boxes (global loads where a box
// cannot serve the pull), summed into the moments as in pull_moments; returns psi.
template <int PREC, int WY, bool FULL>
__device__ __forceinline__ float pull_staged(const KParams& P, const float* __restrict__ box,
                                             const typename Store<PREC>::S* __restrict__ A, int s, const Up& u,
                                             uint32_t lk, bool edge, int x, int y, const int (&sh)[3], int boff,
                                             SiteMom<float>& m)
{
    using L = Lat<1>;
    using SP = Store<PREC>;
    constexpr int Q = 19;
    constexpr int SF = TmaLayout<WY>::SLOTF;
    const int np = (int)P.np;
    const Phys<float>& ph = phys<float>(P);
    constexpr uint32_t qmask = (1u << Q) - 1u;
    auto body = [&](auto careful) {
        constexpr bool CAREFUL = decltype(careful)::value;
        auto ld = [&](int i, float& r, float& g) {
            if (CAREFUL) {
                const bool bounce = (lk >> i) & 1u;
                const bool wrap = (P.per[0] && (unsigned)(x - L::cx(i)) >= (unsigned)P.nx) ||
                                  (P.per[1] && (unsigned)(y - L::cy(i)) >= (unsigned)P.ny);
                if (bounce || wrap) {
                    const int ir = bounce ? L::opp(i) * np + s : i * np + s + up_off<1, int>(u, i);
                    load_pop<PREC, int>(P, A, ir, ir + Q * np, ph, L::cls(i), r, g);
                    return;
                }
            }
            const int o = i * SF + sh[L::cx(i) + 1];  // from the box start, which lies boff into the stage
            if (!in_bounds(P, boff + o, SF * Q - TmaLayout<WY>::ROWS)) {
                r = g = 0.f;
                return;
            }
            SP::decode(box[o], box[o + TmaLayout<WY>::ROWS], ph, L::cls(i), r, g);
        };
        float r0, g0;
        ld(0, r0, g0);
        m.rr = r0;
        m.sg = g0;
#pragma unroll
        for (int k = 0; k < L::NP; ++k) {
            const int p = L::rep(k);
            float rp, gp, rq, gq;
            ld(p, rp, gp);
            ld(L::opp(p), rq, gq);
            mom_add_pair<1, FULL>(m, k, rp, gp, rq, gq);
        }
    };
    if ((lk & qmask) == 0u && !edge)
        body(std::false_type{});
    else
        body(std::true_type{});
    const float rho = ph.rho0 + m.sg;
    return (m.rr - (rho - m.rr)) / rho;
}

template <int PREC, int WY>
__device__ __forceinline__ void tile_d3q19_tma(const KParams& P, const CUtensorMap* map,
                                               const typename Store<PREC>::S* __restrict__ A,
                                               typename Store<PREC>::S* __restrict__ B,
                                               const uint32_t* __restrict__ link, int bx, int by, int z0, int z1,
                                               unsigned char* smem, int* status, const float* __restrict__ gpsi_in,
                                               int gpsi_n)
{
    using T = float;
    using SP = Store<PREC>;
    using L = Lat<1>;
    using Lay = TmaLayout<WY>;
    constexpr int Q = 19;
    const int lane = threadIdx.x;
    const int w = threadIdx.y;
    const int nx = P.nx, ny = P.ny, nz = P.nz;
    const int nxy = nx * ny;
    const int x0 = bx * 30 - 1, y0 = by * (WY - 2) - 1;  // lane 0 / warp 0 coordinates
    const int x = x0 + lane, y = y0 + w;
    int xs, ys;
    const bool xok = wrap_coord(x, nx, P.per[0], xs) && x <= nx;
    const bool yok = wrap_coord(y, ny, P.per[1], ys) && y <= ny;
    const bool row_in = w >= 1 && w <= WY - 2 && y < ny;  // warp-uniform
    const bool inner = row_in && lane >= 1 && lane <= 30 && x < nx;
    const bool edge = (P.per[0] && (x <= 0 || x >= nx - 1)) || (P.per[1] && (y <= 0 || y >= ny - 1));
    Up u;
    {
        int a, b;
        nbr_off(xs, nx, P.per[0], u.xm, u.xp);
        nbr_off(ys, ny, P.per[1], a, b);
        u.ym = (long long)a * nx;
        u.yp = (long long)b * nx;
    }
    const int sxy = xs + nx * ys;
    const int np = (int)P.np;
    const int nplanes = z1 - z0 + 2;  // pulled planes z0-1 .. z1
    const Phys<T>& ph = phys<T>(P);
    const T psi_wall = ph.psi_wall;
    // column shift of a lane's pull inside a box, by c_x (box start: 16-byte boundary)
    int sh[3];
#pragma unroll
    for (int c = -1; c <= 1; ++c) sh[c + 1] = (x0 - c) - ((x0 - c) & ~3);

    T* psi_s = reinterpret_cast<T*>(smem + 2 * Lay::STAGE);
    uint64_t* bar = reinterpret_cast<uint64_t*>(smem + 2 * Lay::STAGE + Lay::PSI);
    if (lane == 0 && w == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();

    // failure-path test: every phase expects 16 bytes that never come, so each wait runs out
    const int wait_limit = P.stall_test ? kTmaStallLimit : kTmaWaitLimit;
    const uint32_t extra_tx = P.stall_test ? 16u : 0u;
    // warp 0: the Q boxes (both arrays of a direction each) of pulled plane p into stage k
    auto issue = [&](int p, int k) {
        if (lane == 0) mbar_expect_tx(&bar[k], Q * Lay::BOX + extra_tx);
        __syncwarp();
        if (lane < Q) {
            const int i = lane;
            const int cx = L::cx(i), cy = L::cy(i), cz = L::cz(i);
            int zsrc = p - cz;
            if (P.per[2]) zsrc = zsrc < 0 ? zsrc + nz : (zsrc >= nz ? zsrc - nz : zsrc);
            tma_load_5d(smem + k * Lay::STAGE + i * Lay::SLOT, map, &bar[k], (x0 - cx) & ~3, y0 - cy, zsrc, i, 0);
        }
    };
    if (w == 0) {
        issue(z0 - 1, 0);
        issue(z0, 1);
    }

    SiteMom<T> mb;
    mom_zero(mb);
    bool coll_b = false;
#pragma unroll 1
    for (int k = 0; k < nplanes; ++k) {
        const int zz = z0 - 1 + k;
        const int stg = k & 1;
        const bool got = mbar_wait(&bar[stg], (uint32_t)((k >> 1) & 1), wait_limit);
        int zs;
        const bool zok = wrap_coord(zz, nz, P.per[2], zs);
        {
            int a, b;
            nbr_off(zs, nz, P.per[2], a, b);
            u.zm = (long long)a * nxy;
            u.zp = (long long)b * nxy;
        }
        SiteMom<T> mn;
        mom_zero(mn);
        T psi_n = psi_wall;
        bool fluid_n = false;
        const int s = sxy + nxy * zs;
        const bool full = row_in && zz >= z0 && zz < z1;
        if (got && xok && yok && zok) {
            const uint32_t lk = load_link(P, link, s);
            const uint32_t type = (lk >> kTypeShift) & 3u;
            if (type == kTypeFluid) {
                const float* box = reinterpret_cast<const float*>(smem + stg * Lay::STAGE) + w * kTmaBoxX + lane;
                const int boff = w * kTmaBoxX + lane;
                psi_n = full ? pull_staged<PREC, WY, true>(P, box, A, s, u, lk, edge, x, y, sh, boff, mn)
                             : pull_staged<PREC, WY, false>(P, box, A, s, u, lk, edge, x, y, sh, boff, mn);
                fluid_n = true;
            } else if (type == kTypePort) {
                psi_n = port_psi<1, PREC, int>(P, A, s, lk, gpsi_in, gpsi_n);
            }
        }
        ring_put(P, psi_s, (((k & 3) * WY) + w) * 32 + lane, psi_n);
        if (__syncthreads_or(!got)) {
            // a phase did not complete: record it, then wait (bounded) until the copies still
            // in flight into this block's shared memory have landed before the block exits.
            // In the failure-path test the phases of planes k and k + 1 (both outstanding)
            // miss only the 16 extra bytes nobody sends: count those as arrived, so each phase
            // completes exactly when its real copies have landed.  On a real timeout the
            // missing bytes are unknown and the waits below just run out.
            if (lane == 0 && w == 0) {
                atomicExch(status, 1);
                if (P.stall_test) {
                    mbar_complete_tx(&bar[stg], extra_tx);
                    if (k + 1 < nplanes) mbar_complete_tx(&bar[stg ^ 1], extra_tx);
                }
            }
            __syncthreads();
            mbar_wait(&bar[stg], (uint32_t)((k >> 1) & 1), kTmaWaitLimit);
            if (k + 1 < nplanes) mbar_wait(&bar[stg ^ 1], (uint32_t)(((k + 1) >> 1) & 1), kTmaWaitLimit);
            return;
        }
        // every thread is done with stage stg: refill it with plane zz + 2
        if (w == 0 && k + 2 < nplanes) {
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            issue(zz + 2, stg);
        }
        if (k >= 2 && coll_b) {
            const int zc = zz - 1;
            const int sc = sxy + nxy * zc;
            auto nb = [&](int cx, int cy, int cz) -> T {
                const int slot = (k - 1 + cz) & 3;
                return ring_get(P, psi_s, (slot * WY + (w + cy)) * 32 + (lane + cx));
            };
            T F[3] = {T(0), T(0), T(0)};
#pragma unroll
            for (int kk = 0; kk < L::NP; ++kk) {
                const int p = L::rep(kk);
                const int cx = L::cx(p), cy = L::cy(p), cz = L::cz(p);
                const T d = (T)L::w(p) * (nb(cx, cy, cz) - nb(-cx, -cy, -cz));
                if (cx) F[0] += cx > 0 ? d : -d;
                if (cy) F[1] += cy > 0 ? d : -d;
                if (cz) F[2] += cz > 0 ? d : -d;
            }
            F[0] *= T(3);
            F[1] *= T(3);
            F[2] *= T(3);
            collide_moments<1, T>(ph, mb, F, [&](int i, T r, T g) {
                const int ir = i * np + sc;
                store_pop<PREC, int>(P, B, ir, ir + Q * np, ph, L::cls(i), r, g);
            });
        }
        coll_b = fluid_n && inner && full;
        mb = mn;
    }
}

template <int PREC, int WY>
__global__ void __launch_bounds__(32 * WY, WY <= 6 ? 3 : 2) k_step_d3q19_tma(const KParams P,
                                                                              const __grid_constant__ CUtensorMap tmA,
                                                                              const typename Store<PREC>::S* __restrict__ A,
                                                                              typename Store<PREC>::S* __restrict__ B,
                                                                              const uint32_t* __restrict__ link,
                                                                              const int* __restrict__ tiles, int* status,
                                                                              const float* __restrict__ gpsi_in,
                                                                              int gpsi_n)
{
    extern __shared__ __align__(1024) unsigned char smem_tma[];
    int bx, by, z0, z1;
    block_of(P, tiles, bx, by, z0, z1);
    tile_d3q19_tma<PREC, WY>(P, &tmA, A, B, link, bx, by, z0, z1, smem_tma, status, gpsi_in, gpsi_n);
}

// ------------------------------------------------------------- batched kernels
// Many instances advance in one launch: the blocks of a fixed (persistent) grid stride
// over the work items of all instances, stage the item's instance parameters in shared
// memory and run the same per-strip / per-tile code as the single-instance kernels, so
// every instance's result is bit-identical to its solo run.  Node k of a captured graph
// advances the instances with steps > k; even k reads buffer a, odd k reads buffer b.
__device__ __forceinline__ void stage_params(KParams& dst, const KParams& src)
{
    const int nt = blockDim.x * blockDim.y;
    const int t = threadIdx.y * blockDim.x + threadIdx.x;
    const int* s = reinterpret_cast<const int*>(&src);
    int* d = reinterpret_cast<int*>(&dst);
    for (int i = t; i < (int)(sizeof(KParams) / sizeof(int)); i += nt) d[i] = s[i];
}

template <int PREC>
__global__ void __launch_bounds__(256) k_batch_d2q9(const BatchSlot* __restrict__ slots,
                                                    const BatchItem* __restrict__ items,
                                                    const int* __restrict__ nitems, int k)
{
    using S = typename Store<PREC>::S;
    __shared__ KParams sP;
    const int n = *nitems;
    for (int w = blockIdx.x; w < n; w += gridDim.x) {
        const BatchItem it = items[w];
        const BatchSlot& sl = slots[it.slot];
        if (k >= sl.steps) continue;  // block-uniform
        __syncthreads();
        stage_params(sP, sl.kp);
        __syncthreads();
        const bool odd = k & 1;
        const S* src = (const S*)(odd ? sl.b : sl.a);
        S* dst = (S*)(odd ? sl.a : sl.b);
        const int wib = threadIdx.x >> 5;
        if (wib < it.y) {
            const int strip = it.x + wib;
            strip_d2q9<PREC, int>(sP, src, dst, sl.link, strip % sP.nsx, strip / sP.nsx,
                                  (const typename Store<PREC>::T*)(odd ? sl.gpsi_b : sl.gpsi_a), sl.nghost);
        }
    }
}

// Regularized instances take the moment march (moments in registers), BGK instances the
// re-read march; MINB resident blocks per SM (3; FP64 2)
template <int PREC, int MINB>
__global__ void __launch_bounds__(256, MINB) k_batch_d3q19(const BatchSlot* __restrict__ slots,
                                                           const BatchItem* __restrict__ items,
                                                           const int* __restrict__ nitems, int k)
{
    using S = typename Store<PREC>::S;
    using T = typename Store<PREC>::T;
    extern __shared__ unsigned char smem_raw[];
    __shared__ KParams sP;
    const int n = *nitems;
    for (int w = blockIdx.x; w < n; w += gridDim.x) {
        const BatchItem it = items[w];
        const BatchSlot& sl = slots[it.slot];
        if (k >= sl.steps) continue;  // block-uniform
        __syncthreads();
        stage_params(sP, sl.kp);
        __syncthreads();
        const bool odd = k & 1;
        const S* src = (const S*)(odd ? sl.b : sl.a);
        S* dst = (S*)(odd ? sl.a : sl.b);
        if (sP.collision == LBCG_REG)
            tile_d3q19_mom<PREC, int, false>(sP, src, dst, sl.link, it.x, it.y, it.z & 0xffff, it.z >> 16,
                                             reinterpret_cast<T*>(smem_raw),
                                             (const T*)(odd ? sl.gpsi_b : sl.gpsi_a), sl.nghost);
        else
            tile_d3q19<PREC, false, int>(sP, src, dst, sl.link, it.x, it.y, it.z & 0xffff, it.z >> 16, reinterpret_cast<T*>(smem_raw));
    }
}

// ---------------------------------------------------------------------- launchers

template <int PREC>
static cudaError_t launch_d2q9(lbcg_ctx* c, const void* a, void* b)
{
    using S = typename Store<PREC>::S;
    const KParams& P = c->kp;
    const int* tl = c->d_tiles;
    const long long warps = tl ? (long long)P.ntiles : (long long)P.nsx * P.nsy;
    const int threads = 256;
    const long long blocks = (warps * 32 + threads - 1) / threads;
    const uint32_t* lk = c->any_link ? c->d_link : nullptr;
    // with ports: the strips refill the ghosts of the output (and its ghost-psi table); the
    // input's table was written by the previous step or by the refill launch before this one
    const bool fuse = c->nghost > 0 && c->d_gstart && tl;
    const PortTab pt{fuse ? c->d_ghost : nullptr, c->d_ghost_u, c->nghost, c->d_gstart, c->d_grow,
                     gpsi_for(c, a), fuse ? gpsi_for(c, b) : nullptr};
    auto go = [&](auto kern) { kern<<<(unsigned)blocks, threads, 0, c->stream>>>(P, (const S*)a, (S*)b, lk, tl, pt); };
    if (effective_variant(c) == 6) {
        if (small_index(c))
            fuse ? go(k_step_d2q9_mom<PREC, int, true>) : go(k_step_d2q9_mom<PREC, int, false>);
        else
            fuse ? go(k_step_d2q9_mom<PREC, long long, true>) : go(k_step_d2q9_mom<PREC, long long, false>);
    } else {
        if (small_index(c))
            fuse ? go(k_step_d2q9<PREC, int, true>) : go(k_step_d2q9<PREC, int, false>);
        else
            fuse ? go(k_step_d2q9<PREC, long long, true>) : go(k_step_d2q9<PREC, long long, false>);
    }
    return cudaGetLastError();
}

// Tensor map of state buffer `buf` as a 5D float tensor (x, y, z, direction, red/second
// array) with boxes of kTmaBoxX x wy x 1 x 1 x 2; two cached (the context's two buffers)
static cudaError_t tma_map_for(lbcg_ctx* c, const void* buf, int wy, const CUtensorMap** out)
{
    for (int k = 0; k < 2; ++k)
        if (c->tmap_buf[k] == buf && c->tmap_wy[k] == wy) {
            *out = reinterpret_cast<const CUtensorMap*>(c->tmap[k]);
            return cudaSuccess;
        }
    const void* other = buf == c->A ? c->B : c->A;
    const int k = (c->tmap_buf[0] == other && c->tmap_wy[0] == wy) ? 1 : 0;
    const cuuint64_t dim[5] = {(cuuint64_t)c->dims[0], (cuuint64_t)c->dims[1], (cuuint64_t)c->dims[2],
                               (cuuint64_t)c->Q, 2};
    const cuuint64_t stride[4] = {(cuuint64_t)c->dims[0] * 4, (cuuint64_t)c->dims[0] * c->dims[1] * 4,
                                  (cuuint64_t)c->np * 4, (cuuint64_t)c->Q * c->np * 4};
    const cuuint32_t box[5] = {(cuuint32_t)kTmaBoxX, (cuuint32_t)wy, 1, 1, 2};
    const cuuint32_t estr[5] = {1, 1, 1, 1, 1};
    CUtensorMap* m = reinterpret_cast<CUtensorMap*>(c->tmap[k]);
    const CUresult r = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(tma_encode_entry())(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 5, const_cast<void*>(buf), dim, stride, box,
                                     estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                                     CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) {
        c->tmap_buf[k] = nullptr;
        return cudaErrorInvalidValue;
    }
    c->tmap_buf[k] = buf;
    c->tmap_wy[k] = wy;
    *out = m;
    return cudaSuccess;
}

template <int PREC>
static cudaError_t launch_d3q19_tma(lbcg_ctx* c, const void* a, void* b)
{
    using S = typename Store<PREC>::S;
    const KParams& P = c->kp;
    const int wy = c->block_rows;
    const CUtensorMap* m = nullptr;
    cudaError_t e = tma_map_for(c, a, wy, &m);
    if (e != cudaSuccess) return e;
    const int* tl = c->d_tiles;
    const dim3 grid = tl ? dim3((unsigned)P.ntiles) : dim3(P.nsx, P.nsy, P.nsz);
    const uint32_t* lk = c->any_link ? c->d_link : nullptr;
    const float* gp = (const float*)gpsi_for(c, a);
    auto go = [&](auto kern, int bytes, int rows) {
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
        kern<<<grid, dim3(32, rows), (size_t)bytes, c->stream>>>(P, *m, (const S*)a, (S*)b, lk, tl, c->d_status, gp,
                                                                   c->nghost);
    };
    if (wy == 8)
        go(k_step_d3q19_tma<PREC, 8>, TmaLayout<8>::BYTES, 8);
    else
        go(k_step_d3q19_tma<PREC, 6>, TmaLayout<6>::BYTES, 6);
    return cudaGetLastError();
}

template <int PREC, bool KEEP>
static cudaError_t launch_d3q19(lbcg_ctx* c, const void* a, void* b, int variant)
{
    using S = typename Store<PREC>::S;
    using T = typename Store<PREC>::T;
    const KParams& P = c->kp;
    const int wy = c->block_rows;
    const int* tl = c->d_tiles;
    dim3 block(32, wy);
    dim3 grid = tl ? dim3((unsigned)P.ntiles) : dim3(P.nsx, P.nsy, P.nsz);
    size_t smem = 4 * (size_t)wy * 32 * sizeof(T);
    const uint32_t* lk = c->any_link ? c->d_link : nullptr;
    const bool fuse = c->nghost > 0 && c->d_gstart && tl;
    const PortTab pt{fuse ? c->d_ghost : nullptr, c->d_ghost_u, c->nghost, c->d_gstart, c->d_grow,
                     gpsi_for(c, a), fuse ? gpsi_for(c, b) : nullptr};
    const bool ports = pt.tab != nullptr;
    if (variant == 7 && !KEEP) {
        const size_t smem7 = smem + 2 * 11 * (size_t)wy * 32 * sizeof(T);
        auto go = [&](auto kern) {
            cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem7);
            kern<<<grid, block, smem7, c->stream>>>(P, (const S*)a, (S*)b, lk, tl, pt);
        };
        if (small_index(c))
            ports ? go(k_step_d3q19_moms<PREC, int, true>) : go(k_step_d3q19_moms<PREC, int, false>);
        else
            ports ? go(k_step_d3q19_moms<PREC, long long, true>) : go(k_step_d3q19_moms<PREC, long long, false>);
        return cudaGetLastError();
    }
    if (variant == 9 && !KEEP) {
        auto go = [&](auto kern) { kern<<<grid, block, smem, c->stream>>>(P, (const S*)a, (S*)b, lk, tl, pt); };
        if (small_index(c))
            ports ? go(k_step_d3q19_momn<PREC, int, true>) : go(k_step_d3q19_momn<PREC, int, false>);
        else
            ports ? go(k_step_d3q19_momn<PREC, long long, true>) : go(k_step_d3q19_momn<PREC, long long, false>);
        return cudaGetLastError();
    }
    if (variant == 6 && !KEEP) {
        auto go = [&](auto kern) { kern<<<grid, block, smem, c->stream>>>(P, (const S*)a, (S*)b, lk, tl, pt); };
        if (small_index(c))
            ports ? go(k_step_d3q19_mom<PREC, int, true>) : go(k_step_d3q19_mom<PREC, int, false>);
        else
            ports ? go(k_step_d3q19_mom<PREC, long long, true>) : go(k_step_d3q19_mom<PREC, long long, false>);
        return cudaGetLastError();
    }
    if (variant == 5 && !KEEP) {
        if (small_index(c))
            k_step_d3q19_occ<PREC, int><<<grid, block, smem, c->stream>>>(P, (const S*)a, (S*)b, lk, tl);
        else
            k_step_d3q19_occ<PREC, long long><<<grid, block, smem, c->stream>>>(P, (const S*)a, (S*)b, lk, tl);
        return cudaGetLastError();
    }
    if (small_index(c))
        k_step_d3q19<PREC, KEEP, int><<<grid, block, smem, c->stream>>>(P, (const S*)a, (S*)b, lk, tl);
    else
        k_step_d3q19<PREC, KEEP, long long><<<grid, block, smem, c->stream>>>(P, (const S*)a, (S*)b, lk, tl);
    return cudaGetLastError();
}


// ------------------------------------------------------- per-storage-format entry points
// the batched step kernel of `lattice` for this format: f(kernel, threads per block, bytes of
// dynamic shared memory per block) for block height wy (D3Q19)
template <int PREC, typename F>
static cudaError_t with_batch_kernel(int lattice, int wy, F&& f)
{
    if (lattice == LBCG_D2Q9) return f(k_batch_d2q9<PREC>, 256, (size_t)0);
    const int threads = 32 * wy;
    return f(k_batch_d3q19<PREC, PREC == LBCG_FP64 ? 2 : 3>, threads,
             4 * (size_t)threads * sizeof(typename Store<PREC>::T));
}

template <int PREC>
int batch_resident_blocks_prec(int lattice, int wy)
{
    int per = 0;
    const cudaError_t e = with_batch_kernel<PREC>(lattice, wy, [&](auto kern, int threads, size_t smem) {
        return cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kern, threads, smem);
    });
    return e == cudaSuccess ? per : 0;
}

template <int PREC>
cudaError_t launch_batch_step_prec(int lattice, const BatchSlot* slots, const BatchItem* items, const int* nitems,
                                   int k, int grid, int wy, cudaStream_t st)
{
    return with_batch_kernel<PREC>(lattice, wy, [&](auto kern, int threads, size_t smem) {
        const dim3 block = lattice == LBCG_D2Q9 ? dim3(256) : dim3(32, wy);
        (void)threads;
        kern<<<(unsigned)grid, block, smem, st>>>(slots, items, nitems, k);
        return cudaGetLastError();
    });
}

template <int PREC>
cudaError_t launch_step_prec(lbcg_ctx* c, const void* a, void* b)
{
    if (c->p.lattice == LBCG_D2Q9) return launch_d2q9<PREC>(c, a, b);
    const int v = effective_variant(c);
    if constexpr (PREC == LBCG_FP32 || PREC == LBCG_FP32_DEV) {
        if (v == 8) return launch_d3q19_tma<PREC>(c, a, b);
    }
    return v == 1 ? launch_d3q19<PREC, true>(c, a, b, v) : launch_d3q19<PREC, false>(c, a, b, v);
}

#ifdef LBCG_STEP_PREC
template int batch_resident_blocks_prec<LBCG_STEP_PREC>(int, int);
template cudaError_t launch_batch_step_prec<LBCG_STEP_PREC>(int, const BatchSlot*, const BatchItem*, const int*, int,
                                                            int, int, cudaStream_t);
template cudaError_t launch_step_prec<LBCG_STEP_PREC>(lbcg_ctx*, const void*, void*);
#endif

}  // namespace lbcg
