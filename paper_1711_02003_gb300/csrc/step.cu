// step.cu -- the fused per-site, per-step update (arXiv:1711.02003, Eqs. 1-11).
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
#include <cuda.h>
#include <cudaTypedefs.h>

#include <mutex>
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
            SP::load(A, ir, ir + (IDX)Q * np, ph, L::cls(i), r[i], g[i]);
        }
    } else {
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            const bool bounce = (lk >> i) & 1u;
            const IDX ir = bounce ? (IDX)L::opp(i) * np + s : (IDX)i * np + s + up_off<LAT, IDX>(u, i);
            SP::load(A, ir, ir + (IDX)Q * np, ph, L::cls(i), r[i], g[i]);
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

// psi of a port ghost site from its own (already filled) populations
template <int LAT, int PREC, typename IDX>
__device__ __forceinline__ typename Store<PREC>::T ghost_psi(const KParams& P,
                                                             const typename Store<PREC>::S* __restrict__ A, IDX s)
{
    using L = Lat<LAT>;
    using SP = Store<PREC>;
    using T = typename SP::T;
    const IDX np = (IDX)P.np;
    T rr = 0, sg = 0;
#pragma unroll
    for (int i = 0; i < L::Q; ++i) {
        T r, g;
        const IDX ir = (IDX)i * np + s;
        SP::load(A, ir, ir + (IDX)L::Q * np, phys<T>(P), L::cls(i), r, g);
        rr += r;
        sg += g;
    }
    const T rho = phys<T>(P).rho0 + sg;
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
        Store<PREC>::store(B, ir, ir + (IDX)L::Q * np, phys<T>(P), L::cls(i), r[i], g[i]);
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

// ------------------------------------------------------------------------ D2Q9
// one warp: the strip (sxi, syi) of 30 x rows sites
template <int PREC, typename IDX>
__device__ __forceinline__ void strip_d2q9(const KParams& P, const typename Store<PREC>::S* __restrict__ A,
                                           typename Store<PREC>::S* __restrict__ B, const uint32_t* __restrict__ link,
                                           int sxi, int syi)
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
            const uint32_t lk = link ? __ldg(link + s) : 0u;
            const uint32_t type = (lk >> kTypeShift) & 3u;
            if (type == kTypeFluid) {
                psi_n = pull_fluid<0, PREC, IDX>(P, A, s, u, lk, rn, gn);
                fluid_n = true;
            } else if (type == kTypePort) {
                psi_n = ghost_psi<0, PREC, IDX>(P, A, s);
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

template <int PREC, typename IDX>
__global__ void __launch_bounds__(256) k_step_d2q9(const KParams P, const typename Store<PREC>::S* __restrict__ A,
                                                   typename Store<PREC>::S* __restrict__ B,
                                                   const uint32_t* __restrict__ link, const int* __restrict__ tiles)
{
    const int gw = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    int sxi, syi;
    if (!strip_of(P, tiles, gw, sxi, syi)) return;  // warp-uniform
    strip_d2q9<PREC, IDX>(P, A, B, link, sxi, syi);
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
            const uint32_t lk = link ? __ldg(link + s) : 0u;
            const uint32_t type = (lk >> kTypeShift) & 3u;
            if (type == kTypeFluid) {
                psi_n = pull_fluid<1, PREC, IDX>(P, A, s, u, lk, rn, gn);
                fluid_n = true;
            } else if (type == kTypePort) {
                psi_n = ghost_psi<1, PREC, IDX>(P, A, s);
            }
        }
        const int slot_n = (zz - z0 + 1) & 3;
        psi_s[(slot_n * WY + w) * 32 + lane] = psi_n;
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
                const uint32_t lk = link ? __ldg(link + sc) : 0u;
                pull_fluid<1, PREC, IDX>(P, A, sc, uc, lk, rb, gb);
            }
            auto nb = [&](int cx, int cy, int cz) -> T {
                const int slot = (zc + cz - z0 + 1) & 3;
                return psi_s[(slot * WY + (w + cy)) * 32 + (lane + cx)];
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
            SP::load(A, ir, ir + (IDX)Q * np, ph, L::cls(i), r, g);
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
    if ((lk & qmask) == 0u)
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
template <int PREC, typename IDX, bool MSMEM>
__device__ __forceinline__ void tile_d3q19_mom(const KParams& P, const typename Store<PREC>::S* __restrict__ A,
                                               typename Store<PREC>::S* __restrict__ B,
                                               const uint32_t* __restrict__ link, int bx, int by, int z0, int z1,
                                               typename Store<PREC>::T* psi_s)
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
            const uint32_t lk = link ? __ldg(link + s) : 0u;
            const uint32_t type = (lk >> kTypeShift) & 3u;
            if (type == kTypeFluid) {
                psi_n = full ? pull_moments<1, PREC, IDX, true>(P, A, s, u, lk, mn)
                             : pull_moments<1, PREC, IDX, false>(P, A, s, u, lk, mn);
                fluid_n = true;
            } else if (type == kTypePort) {
                psi_n = ghost_psi<1, PREC, IDX>(P, A, s);
            }
        }
        const int slot_n = (zz - z0 + 1) & 3;
        psi_s[(slot_n * WY + w) * 32 + lane] = psi_n;
        if (MSMEM && fluid_n && full) mom_put(mn, mom_s + (zz & 1) * 11 * mstride, mstride);
        __syncthreads();
        if (zz - 1 >= z0 && coll_b) {
            const int zc = zz - 1;
            const IDX sc = sxy + (IDX)nxy * (IDX)zc;
            auto nb = [&](int cx, int cy, int cz) -> T {
                const int slot = (zc + cz - z0 + 1) & 3;
                return psi_s[(slot * WY + (w + cy)) * 32 + (lane + cx)];
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
                SP::store(B, ir, ir + (IDX)Q * np, ph, L::cls(i), r, g);
            });
        }
        coll_b = fluid_n && inner && zz >= z0 && zz < z1;
        if (!MSMEM) mb = mn;
    }
}

// variant 6: moments in registers; three blocks per SM (FP64: two, at 128 registers)
template <int PREC, typename IDX>
__global__ void __launch_bounds__(256, PREC == LBCG_FP64 ? 2 : 3) k_step_d3q19_mom(const KParams P,
                                                           const typename Store<PREC>::S* __restrict__ A,
                                                           typename Store<PREC>::S* __restrict__ B,
                                                           const uint32_t* __restrict__ link, const int* __restrict__ tiles)
{
    extern __shared__ unsigned char smem_raw[];
    int bx, by, z0, z1;
    block_of(P, tiles, bx, by, z0, z1);
    tile_d3q19_mom<PREC, IDX, false>(P, A, B, link, bx, by, z0, z1, reinterpret_cast<typename Store<PREC>::T*>(smem_raw));
}

// variant 7: the moment march with the waiting moments in shared memory; 64 registers, so
// four blocks of 8 warps or two of 16 per SM
template <int PREC, typename IDX>
__global__ void __launch_bounds__(512, 2) k_step_d3q19_moms(const KParams P,
                                                                const typename Store<PREC>::S* __restrict__ A,
                                                                typename Store<PREC>::S* __restrict__ B,
                                                                const uint32_t* __restrict__ link,
                                                                const int* __restrict__ tiles)
{
    extern __shared__ unsigned char smem_raw[];
    int bx, by, z0, z1;
    block_of(P, tiles, bx, by, z0, z1);
    tile_d3q19_mom<PREC, IDX, true>(P, A, B, link, bx, by, z0, z1, reinterpret_cast<typename Store<PREC>::T*>(smem_raw));
}

// ------------------------------------------------ D2Q9 moment march (2D variant 6)
// strip_d2q9 with the waiting row held as the moments of the regularized collision (7 numbers
// in 2D) instead of its 2Q populations; regularized collision only.
template <int PREC, typename IDX>
__device__ __forceinline__ void strip_d2q9_mom(const KParams& P, const typename Store<PREC>::S* __restrict__ A,
                                               typename Store<PREC>::S* __restrict__ B,
                                               const uint32_t* __restrict__ link, int sxi, int syi)
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
            const uint32_t lk = link ? __ldg(link + s) : 0u;
            const uint32_t type = (lk >> kTypeShift) & 3u;
            if (type == kTypeFluid) {
                psi_n = pull_moments<0, PREC, IDX, true>(P, A, s, u, lk, mn);
                fluid_n = true;
            } else if (type == kTypePort) {
                psi_n = ghost_psi<0, PREC, IDX>(P, A, s);
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
                    SP::store(B, ir, ir + (IDX)Q * np, ph, L::cls(i), r, g);
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

template <int PREC, typename IDX>
__global__ void __launch_bounds__(256) k_step_d2q9_mom(const KParams P, const typename Store<PREC>::S* __restrict__ A,
                                                       typename Store<PREC>::S* __restrict__ B,
                                                       const uint32_t* __restrict__ link,
                                                       const int* __restrict__ tiles)
{
    const int gw = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    int sxi, syi;
    if (!strip_of(P, tiles, gw, sxi, syi)) return;  // warp-uniform
    strip_d2q9_mom<PREC, IDX>(P, A, B, link, sxi, syi);
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
                                             uint32_t lk, bool edge, int x, int y, const int (&sh)[3],
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
                    SP::load(A, ir, ir + Q * np, ph, L::cls(i), r, g);
                    return;
                }
            }
            const float* b = box + i * SF + sh[L::cx(i) + 1];
            SP::decode(b[0], b[TmaLayout<WY>::ROWS], ph, L::cls(i), r, g);
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
                                               unsigned char* smem, int* status)
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
            const uint32_t lk = link ? __ldg(link + s) : 0u;
            const uint32_t type = (lk >> kTypeShift) & 3u;
            if (type == kTypeFluid) {
                const float* box = reinterpret_cast<const float*>(smem + stg * Lay::STAGE) + w * kTmaBoxX + lane;
                psi_n = full ? pull_staged<PREC, WY, true>(P, box, A, s, u, lk, edge, x, y, sh, mn)
                             : pull_staged<PREC, WY, false>(P, box, A, s, u, lk, edge, x, y, sh, mn);
                fluid_n = true;
            } else if (type == kTypePort) {
                psi_n = ghost_psi<1, PREC, int>(P, A, s);
            }
        }
        psi_s[(((k & 3) * WY) + w) * 32 + lane] = psi_n;
        if (__syncthreads_or(!got)) {
            // a copy did not arrive: record it, wait (bounded) for both stages, give up
            if (lane == 0 && w == 0) atomicExch(status, 1);
            mbar_wait(&bar[stg], (uint32_t)((k >> 1) & 1), wait_limit);
            if (k + 1 < nplanes) mbar_wait(&bar[stg ^ 1], (uint32_t)(((k + 1) >> 1) & 1), wait_limit);
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
                return psi_s[(slot * WY + (w + cy)) * 32 + (lane + cx)];
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
                SP::store(B, ir, ir + Q * np, ph, L::cls(i), r, g);
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
                                                                              const int* __restrict__ tiles, int* status)
{
    extern __shared__ __align__(1024) unsigned char smem_tma[];
    int bx, by, z0, z1;
    block_of(P, tiles, bx, by, z0, z1);
    tile_d3q19_tma<PREC, WY>(P, &tmA, A, B, link, bx, by, z0, z1, smem_tma, status);
}

// --------------------------------------- psi-exchange moment march (variant 10)
// The psi ring of a block tile is the one quantity the tile cannot compute from its own
// sites; the other marches recompute it by pulling the ring sites' 2Q populations (32 x WY
// threads pull for 30 x (WY - 2) collided sites).  Here every thread owns an interior site
// (tiles of 32 x WY) and the tiles exchange psi instead: after summing plane z a tile
// publishes psi of its sites (per-site buffer, then its flag for that plane = the step's
// epoch), waits for the flags of its eight x-y neighbour tiles for the same plane and
// reads their edge psi from L2.  z-ring planes are still pulled (tiles of one x-y column
// are in different slabs).  Blocks are persistent and take tiles in list order (slab, then
// column); a tile is at most one plane ahead of its neighbours, so with more than
// (nsx + 2)(rows + 2) resident blocks the oldest tile always completes (checked on the
// host, else variant 6 runs).  Waits are bounded: on a timeout the status word is set,
// every other wait gives up at once, the step completes with an invalid state and the host
// reports LBCG_ERR_TIMEOUT.  The last block to finish resets the tile counter and advances
// the epoch, so replays of a captured graph need no host involvement.  Regularized
// collision, 4- and 2-byte storage, boxes closed in x and y.
struct XParams {
    int nsx, nsy, ntiles, rows;
    const int* tiles;  // [ntiles][2]: column bx + nsx * by, slab
    const int* map;    // [slab][column]: tile index or -1 (no fluid or port in its planes)
    float* psi;        // per-site psi of the current step (psi_wall where never written)
    int* flags;        // [ntiles][rows + 2]: epoch of the last publication of each plane
    int* ctl;          // [0] next tile, [1] blocks done, [2] epoch
    int* status;       // nonzero: a wait timed out (every later wait gives up)
};

constexpr int kXWaitLimit = 1 << 16;  // polls of a neighbour flag (32 ns sleeps) before giving up

template <int PREC>
__global__ void __launch_bounds__(256, 4) k_step_d3q19_xchg(const KParams P, const XParams X,
                                                            const typename Store<PREC>::S* __restrict__ A,
                                                            typename Store<PREC>::S* __restrict__ B,
                                                            const uint32_t* __restrict__ link)
{
    using T = typename Store<PREC>::T;
    using SP = Store<PREC>;
    using L = Lat<1>;
    constexpr int Q = 19;
    extern __shared__ unsigned char smem_raw[];
    T* const ring = reinterpret_cast<T*>(smem_raw);  // [8][WY + 2][34]
    __shared__ int s_tile;
    const int lane = threadIdx.x, w = threadIdx.y, WY = blockDim.y, tid = w * 32 + lane;
    const int RW = 34, RH = WY + 2;
    const int mstride = WY * 32;
    T* const mom = ring + 8 * RH * RW + tid;  // [plane mod 3][11][WY * 32], thread-private
    const int nx = P.nx, ny = P.ny, nz = P.nz;
    const int nxy = nx * ny;
    const int np = (int)P.np;
    const Phys<T>& ph = phys<T>(P);
    const T psi_wall = ph.psi_wall;
    const int epoch = *(volatile const int*)(X.ctl + 2);
    const int nplanes_max = X.rows + 2;

    for (;;) {
        if (tid == 0) s_tile = atomicAdd(X.ctl, 1);
        __syncthreads();
        const int t = s_tile;
        __syncthreads();
        if (t >= X.ntiles) break;
        const int col = X.tiles[2 * t], slab = X.tiles[2 * t + 1];
        const int bx = col % X.nsx, by = col / X.nsx;
        const int x0 = bx * 32, y0 = by * WY;
        const int x = x0 + lane, y = y0 + w;
        const bool inb = x < nx && y < ny;
        const int xs = inb ? x : 0, ys = inb ? y : 0;
        Up u;
        {
            int a, b;
            nbr_off(xs, nx, 0, u.xm, u.xp);
            nbr_off(ys, ny, 0, a, b);
            u.ym = (long long)a * nx;
            u.yp = (long long)b * nx;
        }
        const int sxy = xs + nx * ys;
        const int z0 = slab * X.rows, z1 = min(z0 + X.rows, nz);
        const int nplanes = z1 - z0 + 2;
        // waiter lanes 0..7 of the last warp: the eight x-y neighbour tiles of the same slab
        int nbt = -1;
        if (w == WY - 1 && lane < 8) {
            const int dx = lane < 3 ? lane - 1 : (lane == 3 ? -1 : (lane == 4 ? 1 : lane - 6));
            const int dy = lane < 3 ? -1 : (lane < 5 ? 0 : 1);
            const int nbx = bx + dx, nby = by + dy;
            if (nbx >= 0 && nbx < X.nsx && nby >= 0 && nby < X.nsy)
                nbt = X.map[(size_t)slab * X.nsx * X.nsy + nbx + X.nsx * nby];
        }

        // iteration k pulls plane z0 - 1 + k, publishes it, collides plane z0 - 3 + k (its
        // ring planes are complete) and only then waits for the neighbours' plane k and
        // fetches its ring edge: one barrier per plane, the wait overlapping the collision
        unsigned coll_bits = 0;  // bit k: plane z0 - 1 + k is collided by this thread
#pragma unroll 1
        for (int k = 0; k <= nplanes; ++k) {
            const int zz = z0 - 1 + k;
            const bool pulling = k < nplanes;
            int zs = 0;
            const bool zok = pulling && wrap_coord(zz, nz, P.per[2], zs);
            const int slot = k & 7;
            if (pulling) {
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
                const int site = sxy + nxy * zs;
                const bool full = zz >= z0 && zz < z1;
                if (inb && zok) {
                    const uint32_t lk = __ldg(link + site);
                    const uint32_t type = (lk >> kTypeShift) & 3u;
                    if (type == kTypeFluid) {
                        psi_n = full ? pull_moments<1, PREC, int, true>(P, A, site, u, lk, mn)
                                     : pull_moments<1, PREC, int, false>(P, A, site, u, lk, mn);
                        fluid_n = true;
                    } else if (type == kTypePort) {
                        psi_n = ghost_psi<1, PREC, int>(P, A, site);
                    }
                    X.psi[site] = (float)psi_n;
                }
                ring[(slot * RH + w + 1) * RW + lane + 1] = psi_n;
                if (fluid_n && inb && full) {
                    mom_put(mn, mom + (k % 3) * 11 * mstride, mstride);
                    coll_bits |= 1u << k;
                }
            }
            __syncthreads();
            if (pulling && tid == 0) {
                __threadfence();
                atomicExch(X.flags + (size_t)t * nplanes_max + k, epoch);
            }
            // collide plane z0 - 3 + k: psi of its planes z0 - 4 + k .. z0 - 2 + k is complete
            if (k >= 3 && (coll_bits >> (k - 2) & 1u)) {
                const int kc = k - 2;
                const int zc = z0 - 1 + kc;
                const int sc = sxy + nxy * zc;
                auto nb = [&](int cx, int cy, int cz) -> T {
                    return ring[(((kc + cz) & 7) * RH + (w + 1 + cy)) * RW + (lane + 1 + cx)];
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
                SiteMom<T> mb;
                mom_get(mb, mom + (kc % 3) * 11 * mstride, mstride);
                collide_moments<1, T>(ph, mb, F, [&](int i, T r, T g) {
                    const int ir = i * np + sc;
                    SP::store(B, ir, ir + Q * np, ph, L::cls(i), r, g);
                });
            }
            if (pulling && w == WY - 1) {
                // the last warp waits for the neighbours' plane k and fetches the ring edge
                bool ok = true;
                if (nbt >= 0) {
                    const volatile int* f = X.flags + (size_t)nbt * nplanes_max + k;
                    const int want = P.stall_test ? epoch + 1 : epoch;  // failure-path test: never published
                    int it = 0;
                    while (*f != want) {
                        if (*(volatile int*)X.status != 0 || ++it > kXWaitLimit) {
                            ok = false;
                            break;
                        }
                        __nanosleep(32);
                    }
                    __threadfence();
                }
                if (!ok) atomicExch(X.status, 2);
                __syncwarp();
                const int ncell = 2 * RW + 2 * WY;
                for (int c = lane; c < ncell; c += 32) {
                    int gx, gy, rr, rc;
                    if (c < 2 * RW) {
                        const int top = c < RW;
                        rc = top ? c : c - RW;
                        rr = top ? 0 : WY + 1;
                        gx = x0 - 1 + rc;
                        gy = top ? y0 - 1 : y0 + WY;
                    } else {
                        const int c2 = c - 2 * RW;
                        const int left = c2 < WY;
                        rr = (left ? c2 : c2 - WY) + 1;
                        rc = left ? 0 : RW - 1;
                        gx = left ? x0 - 1 : x0 + 32;
                        gy = y0 + rr - 1;
                    }
                    T v = psi_wall;
                    if (zok && gx >= 0 && gx < nx && gy >= 0 && gy < ny) v = (T)__ldcg(X.psi + gx + nx * gy + nxy * zs);
                    ring[(slot * RH + rr) * RW + rc] = v;
                }
            }
        }
        __syncthreads();  // the ring and moment slots are reused by the next tile
    }
    // the last block to finish rearms the tile counter and advances the epoch
    if (tid == 0) {
        __threadfence();
        const int d = atomicAdd(X.ctl + 1, 1);
        if (d == (int)gridDim.x - 1) {
            atomicExch(X.ctl, 0);
            atomicExch(X.ctl + 1, 0);
            __threadfence();
            atomicAdd(X.ctl + 2, 1);
        }
    }
}

// ------------------------------------------------- pipelined variants (variant 3)
// The collision of row/plane k needs psi of k+1, so a plain march waits for the loads of
// k+1 and only then computes.  The pipelined march collides k-2 while the loads of k are
// in flight: iteration k issues the pull of k, collides k-2 (its psi neighbours k-3..k-1
// are known), then finishes psi(k).  D2Q9 keeps three rows of populations in registers;
// D3Q19 parks the waiting plane's populations in a per-thread shared-memory stage.

template <int PREC, typename IDX>
__global__ void __launch_bounds__(256) k_step_d2q9_pipe(const KParams P,
                                                        const typename Store<PREC>::S* __restrict__ A,
                                                        typename Store<PREC>::S* __restrict__ B,
                                                        const uint32_t* __restrict__ link,
                                                        const int* __restrict__ tiles)
{
    using T = typename Store<PREC>::T;
    using L = Lat<0>;
    constexpr int Q = 9;
    const int lane = threadIdx.x & 31;
    const int gw = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    int sxi, syi;
    if (!strip_of(P, tiles, gw, sxi, syi)) return;  // warp-uniform
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

    T psi_a = psi_wall, psi_b = psi_wall, psi_c = psi_wall;  // rows k-3, k-2, k-1
    T r1[Q], g1[Q], r2[Q], g2[Q];                           // populations of rows k-1, k-2
    bool c1 = false, c2 = false;
    IDX s1 = 0, s2 = 0;
#pragma unroll
    for (int i = 0; i < Q; ++i) r1[i] = g1[i] = r2[i] = g2[i] = T(0);

    for (int yy = y0 - 1; yy <= y1 + 1; ++yy) {
        T rn[Q], gn[Q];
#pragma unroll
        for (int i = 0; i < Q; ++i) rn[i] = gn[i] = T(0);
        T psi_n = psi_wall;
        bool fluid_n = false;
        IDX s = 0;
        if (yy <= y1) {
            int ys;
            const bool yok = wrap_coord(yy, ny, P.per[1], ys);
            int dym, dyp;
            nbr_off(ys, ny, P.per[1], dym, dyp);
            u.ym = (long long)dym * nx;
            u.yp = (long long)dyp * nx;
            s = (IDX)xs + (IDX)nx * (IDX)ys;
            if (xok && yok) {
                const uint32_t lk = link ? __ldg(link + s) : 0u;
                const uint32_t type = (lk >> kTypeShift) & 3u;
                if (type == kTypeFluid) {
                    psi_n = pull_fluid<0, PREC, IDX>(P, A, s, u, lk, rn, gn);
                    fluid_n = true;
                } else if (type == kTypePort) {
                    psi_n = ghost_psi<0, PREC, IDX>(P, A, s);
                }
            }
        }
        if (yy - 2 >= y0) {  // warp-uniform: collide row yy-2 with psi rows a, b, c
            const T am = __shfl_up_sync(0xffffffffu, psi_a, 1), ap = __shfl_down_sync(0xffffffffu, psi_a, 1);
            const T bm = __shfl_up_sync(0xffffffffu, psi_b, 1), bp = __shfl_down_sync(0xffffffffu, psi_b, 1);
            const T cm = __shfl_up_sync(0xffffffffu, psi_c, 1), cp = __shfl_down_sync(0xffffffffu, psi_c, 1);
            if (c2) {
                auto nb = [&](int cx, int cy) -> T {
                    return cy < 0 ? (cx < 0 ? am : (cx > 0 ? ap : psi_a))
                         : cy > 0 ? (cx < 0 ? cm : (cx > 0 ? cp : psi_c))
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
                collide_site<0, T>(P, phys<T>(P), r2, g2, F);
                store_site<0, PREC, IDX>(P, B, s2, r2, g2);
            }
        }
        psi_a = psi_b;
        psi_b = psi_c;
        psi_c = psi_n;
        c2 = c1;
        s2 = s1;
        c1 = fluid_n && xint && yy >= y0 && yy < y1;
        s1 = s;
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            r2[i] = r1[i];
            g2[i] = g1[i];
            r1[i] = rn[i];
            g1[i] = gn[i];
        }
    }
}

// blockDim = (32, WY); smem: psi [4][WY][32], population stages [2][2Q][WY*32]
template <int PREC, typename IDX>
__global__ void __launch_bounds__(256, 2) k_step_d3q19_pipe(const KParams P,
                                                            const typename Store<PREC>::S* __restrict__ A,
                                                            typename Store<PREC>::S* __restrict__ B,
                                                            const uint32_t* __restrict__ link,
                                                            const int* __restrict__ tiles)
{
    int bx, by, z0, z1;
    block_of(P, tiles, bx, by, z0, z1);
    using T = typename Store<PREC>::T;
    using L = Lat<1>;
    constexpr int Q = 19;
    extern __shared__ unsigned char smem_raw[];
    const int lane = threadIdx.x;
    const int w = threadIdx.y;
    const int WY = blockDim.y;
    const int nthr = 32 * WY;
    const int tid = w * 32 + lane;
    T* psi_s = reinterpret_cast<T*>(smem_raw);  // [4][WY][32]
    T* stage = psi_s + 4 * nthr;                 // [2][2Q][nthr]
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
    bool c1 = false, c2 = false;  // planes k-1, k-2 collide here

    for (int zz = z0 - 1; zz <= z1 + 1; ++zz) {
        T rn[Q], gn[Q];
#pragma unroll
        for (int i = 0; i < Q; ++i) rn[i] = gn[i] = T(0);
        T psi_n = psi_wall;
        bool fluid_n = false;
        if (zz <= z1) {
            int zs;
            const bool zok = wrap_coord(zz, nz, P.per[2], zs);
            int a, b;
            nbr_off(zs, nz, P.per[2], a, b);
            u.zm = (long long)a * nxy;
            u.zp = (long long)b * nxy;
            const IDX s = sxy + (IDX)nxy * (IDX)zs;
            if (xok && yok && zok) {
                const uint32_t lk = link ? __ldg(link + s) : 0u;
                const uint32_t type = (lk >> kTypeShift) & 3u;
                if (type == kTypeFluid) {
                    psi_n = pull_fluid<1, PREC, IDX>(P, A, s, u, lk, rn, gn);
                    fluid_n = true;
                } else if (type == kTypePort) {
                    psi_n = ghost_psi<1, PREC, IDX>(P, A, s);
                }
            }
        }
        if (c2) {  // collide plane zc = zz-2 (psi of zc-1..zc+1 are in shared memory)
            const int zc = zz - 2;
            T* st = stage + (size_t)(zc & 1) * 2 * Q * nthr;
            T rc[Q], gc[Q];
#pragma unroll
            for (int i = 0; i < Q; ++i) {
                rc[i] = st[i * nthr + tid];
                gc[i] = st[(Q + i) * nthr + tid];
            }
            auto nb = [&](int cx, int cy, int cz) -> T {
                const int slot = (zc + cz - z0 + 1) & 3;
                return psi_s[(slot * WY + (w + cy)) * 32 + (lane + cx)];
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
            collide_site<1, T>(P, phys<T>(P), rc, gc, F);
            store_site<1, PREC, IDX>(P, B, sxy + (IDX)nxy * (IDX)zc, rc, gc);
        }
        c2 = c1;
        c1 = fluid_n && inner && zz >= z0 && zz < z1;
        if (c1) {  // park plane zz's populations (same slot as the plane just collided)
            T* st = stage + (size_t)(zz & 1) * 2 * Q * nthr;
#pragma unroll
            for (int i = 0; i < Q; ++i) {
                st[i * nthr + tid] = rn[i];
                st[(Q + i) * nthr + tid] = gn[i];
            }
        }
        if (zz <= z1) psi_s[(((zz - z0 + 1) & 3) * WY + w) * 32 + lane] = psi_n;
        __syncthreads();
    }
}

// ----------------------------------------------- asynchronous-copy variant (variant 4)
// D3Q19, 4-byte storage formats.  Each thread copies the pulled populations of its site
// for plane zz+2 into its own shared-memory stage with cp.async while it computes psi of
// plane zz and collides plane zz-1, so loads are in flight during the arithmetic instead of
// between it.  Stages: zz-1 (collided), zz (psi), zz+1, zz+2 (in flight) -> 4 per thread.
// The link word of a plane is read one iteration before its copies are issued.
__device__ __forceinline__ void cp_async4(void* smem, const void* gmem)
{
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait()
{
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

constexpr int kAsyncStages = 4;  // lookahead 2

template <int PREC, typename IDX>
__global__ void __launch_bounds__(256, 1) k_step_d3q19_async(const KParams P,
                                                             const typename Store<PREC>::S* __restrict__ A,
                                                             typename Store<PREC>::S* __restrict__ B,
                                                             const uint32_t* __restrict__ link,
                                                             const int* __restrict__ tiles)
{
    int bx, by, z0, z1;
    block_of(P, tiles, bx, by, z0, z1);
    using S = typename Store<PREC>::S;
    using T = typename Store<PREC>::T;
    using L = Lat<1>;
    constexpr int Q = 19;
    static_assert(sizeof(S) == 4, "4-byte storage only");
    extern __shared__ unsigned char smem_raw[];
    const int lane = threadIdx.x;
    const int w = threadIdx.y;
    const int WY = blockDim.y;
    const int nthr = 32 * WY;
    const int tid = w * 32 + lane;
    T* psi_s = reinterpret_cast<T*>(smem_raw);        // [4][WY][32]
    S* stage = reinterpret_cast<S*>(psi_s + 4 * nthr);  // [kAsyncStages][2Q][nthr]
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
    const IDX np = (IDX)P.np;
    const Phys<T>& ph = phys<T>(P);
    const T psi_wall = ph.psi_wall;
    // site kind of a plane for this thread: 0 outside/wall, 1 fluid, 2 port ghost
    auto kind_of = [&](int zz, uint32_t& lk, IDX& s, int& zs) -> int {
        lk = 0;
        s = 0;
        zs = 0;
        if (zz > z1) return 0;
        const bool zok = wrap_coord(zz, nz, P.per[2], zs);
        if (!(xok && yok && zok)) return 0;
        s = sxy + (IDX)nxy * (IDX)zs;
        lk = link ? __ldg(link + s) : 0u;
        const uint32_t type = (lk >> kTypeShift) & 3u;
        return type == kTypeFluid ? 1 : (type == kTypePort ? 2 : 0);
    };
    // issue the copies of plane zz (kind k) into its stage
    auto issue = [&](int zz, int k, uint32_t lk, IDX s, int zs) {
        S* st = stage + (size_t)((zz - z0 + 1) & (kAsyncStages - 1)) * 2 * Q * nthr;
        if (k == 1) {
            Up uu = u;
            int a, b;
            nbr_off(zs, nz, P.per[2], a, b);
            uu.zm = (long long)a * nxy;
            uu.zp = (long long)b * nxy;
#pragma unroll
            for (int i = 0; i < Q; ++i) {
                const bool bounce = (lk >> i) & 1u;
                const IDX ir = bounce ? (IDX)L::opp(i) * np + s : (IDX)i * np + s + up_off<1, IDX>(uu, i);
                cp_async4(st + i * nthr + tid, A + ir);
                cp_async4(st + (Q + i) * nthr + tid, A + ir + (IDX)Q * np);
            }
        } else if (k == 2) {
#pragma unroll
            for (int i = 0; i < Q; ++i) {
                const IDX ir = (IDX)i * np + s;
                cp_async4(st + i * nthr + tid, A + ir);
                cp_async4(st + (Q + i) * nthr + tid, A + ir + (IDX)Q * np);
            }
        }
        cp_async_commit();
    };
    auto read_stage = [&](int zz, T (&r)[Q], T (&g)[Q]) {
        const S* st = stage + (size_t)((zz - z0 + 1) & (kAsyncStages - 1)) * 2 * Q * nthr;
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            // decode exactly as a global load would (Store::load on the staged element)
            Store<PREC>::load(st, (IDX)(i * nthr + tid), (IDX)((Q + i) * nthr + tid), ph, L::cls(i), r[i], g[i]);
        }
    };

    // prologue: planes z0-1 and z0 in flight, link of z0+1 known
    int k_a, k_b, k_c, zs_a, zs_b, zs_c;
    uint32_t lk_a, lk_b, lk_c;
    IDX s_a, s_b, s_c;
    k_a = kind_of(z0 - 1, lk_a, s_a, zs_a);
    issue(z0 - 1, k_a, lk_a, s_a, zs_a);
    k_b = kind_of(z0, lk_b, s_b, zs_b);
    issue(z0, k_b, lk_b, s_b, zs_b);
    k_c = kind_of(z0 + 1, lk_c, s_c, zs_c);
    int kind_cur = k_a;       // kind of plane zz (for psi)
    int kind_next = k_b;      // kind of plane zz+1
    bool coll_b = false;      // plane zz-1 collides here
    IDX sc_prev = 0;

    for (int zz = z0 - 1; zz <= z1; ++zz) {
        // 1. issue plane zz+2 (its link word was read last iteration), read the link of zz+3
        issue(zz + 2, k_c, lk_c, s_c, zs_c);
        const int kind_2 = k_c;
        k_c = kind_of(zz + 3, lk_c, s_c, zs_c);
        // 2. plane zz has landed (two newer groups may still be in flight)
        cp_async_wait<2>();
        T psi_n = psi_wall;
        if (kind_cur != 0) {
            T r[Q], g[Q];
            read_stage(zz, r, g);
            T rr = r[0], sg = g[0];
#pragma unroll
            for (int i = 1; i < Q; ++i) {
                rr += r[i];
                sg += g[i];
            }
            const T rho = ph.rho0 + sg;
            psi_n = (rr - (rho - rr)) / rho;
        }
        psi_s[(((zz - z0 + 1) & 3) * WY + w) * 32 + lane] = psi_n;
        __syncthreads();
        // 3. collide plane zz-1
        if (zz - 1 >= z0 && coll_b) {
            const int zc = zz - 1;
            T r[Q], g[Q];
            read_stage(zc, r, g);
            auto nb = [&](int cx, int cy, int cz) -> T {
                const int slot = (zc + cz - z0 + 1) & 3;
                return psi_s[(slot * WY + (w + cy)) * 32 + (lane + cx)];
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
            collide_site<1, T>(P, ph, r, g, F);
            store_site<1, PREC, IDX>(P, B, sc_prev, r, g);
        }
        coll_b = kind_cur == 1 && inner && zz >= z0 && zz < z1;
        sc_prev = sxy + (IDX)nxy * (IDX)(zz < 0 ? 0 : (zz >= nz ? 0 : zz));
        kind_cur = kind_next;
        kind_next = kind_2;
    }
    cp_async_wait<0>();
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
            strip_d2q9<PREC, int>(sP, src, dst, sl.link, strip % sP.nsx, strip / sP.nsx);
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
            tile_d3q19_mom<PREC, int, false>(sP, src, dst, sl.link, it.x, it.y, it.z & 0xffff, it.z >> 16, reinterpret_cast<T*>(smem_raw));
        else
            tile_d3q19<PREC, false, int>(sP, src, dst, sl.link, it.x, it.y, it.z & 0xffff, it.z >> 16, reinterpret_cast<T*>(smem_raw));
    }
}

cudaError_t launch_batch_step(int lattice, int precision, const BatchSlot* slots, const BatchItem* items,
                              const int* nitems, int k, cudaStream_t st)
{
    const int sms = 152;
    if (lattice == LBCG_D2Q9) {
        const unsigned grid = sms * 3;
        switch (precision) {
            case LBCG_FP64: k_batch_d2q9<LBCG_FP64><<<grid, 256, 0, st>>>(slots, items, nitems, k); break;
            case LBCG_FP32: k_batch_d2q9<LBCG_FP32><<<grid, 256, 0, st>>>(slots, items, nitems, k); break;
            case LBCG_FP32_DEV: k_batch_d2q9<LBCG_FP32_DEV><<<grid, 256, 0, st>>>(slots, items, nitems, k); break;
            default: k_batch_d2q9<LBCG_FP16_SCALED><<<grid, 256, 0, st>>>(slots, items, nitems, k); break;
        }
    } else {
        const dim3 block(32, 8);
        const size_t sm4 = 4 * 8 * 32 * sizeof(float);
        switch (precision) {
            case LBCG_FP64:
                k_batch_d3q19<LBCG_FP64, 2><<<sms * 2, block, 4 * 8 * 32 * sizeof(double), st>>>(slots, items, nitems, k);
                break;
            case LBCG_FP32: k_batch_d3q19<LBCG_FP32, 3><<<sms * 3, block, sm4, st>>>(slots, items, nitems, k); break;
            case LBCG_FP32_DEV:
                k_batch_d3q19<LBCG_FP32_DEV, 3><<<sms * 3, block, sm4, st>>>(slots, items, nitems, k);
                break;
            default: k_batch_d3q19<LBCG_FP16_SCALED, 3><<<sms * 3, block, sm4, st>>>(slots, items, nitems, k); break;
        }
    }
    return cudaGetLastError();
}

// ---------------------------------------------------------------------- launchers
static bool small_index(const lbcg_ctx* c) { return (long long)2 * c->Q * (long long)c->np < (1LL << 31) - 1; }

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
    if (effective_variant(c) == 6) {
        if (small_index(c))
            k_step_d2q9_mom<PREC, int><<<(unsigned)blocks, threads, 0, c->stream>>>(P, (const S*)a, (S*)b, lk, tl);
        else
            k_step_d2q9_mom<PREC, long long><<<(unsigned)blocks, threads, 0, c->stream>>>(P, (const S*)a, (S*)b, lk, tl);
        return cudaGetLastError();
    }
    if (c->variant == 3) {
        if (small_index(c))
            k_step_d2q9_pipe<PREC, int><<<(unsigned)blocks, threads, 0, c->stream>>>(P, (const S*)a, (S*)b, lk, tl);
        else
            k_step_d2q9_pipe<PREC, long long><<<(unsigned)blocks, threads, 0, c->stream>>>(P, (const S*)a, (S*)b, lk, tl);
        return cudaGetLastError();
    }
    if (small_index(c))
        k_step_d2q9<PREC, int><<<(unsigned)blocks, threads, 0, c->stream>>>(P, (const S*)a, (S*)b, lk, tl);
    else
        k_step_d2q9<PREC, long long><<<(unsigned)blocks, threads, 0, c->stream>>>(P, (const S*)a, (S*)b, lk, tl);
    return cudaGetLastError();
}

// ------------------------------------------------------------- tensor maps (host)
static PFN_cuTensorMapEncodeTiled_v12000 tma_encoder()
{
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(f);
    });
    return fn;
}

bool tma_supported(const lbcg_ctx* c)
{
    const int prec = c->p.precision;
    return c->p.lattice == LBCG_D3Q19 && c->p.collision == LBCG_REG &&
           (prec == LBCG_FP32 || prec == LBCG_FP32_DEV) && c->dims[0] % 4 == 0 &&
           (c->block_rows == 6 || c->block_rows == 8) && small_index(c) && c->d_status != nullptr &&
           tma_encoder() != nullptr;
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
    const CUresult r = tma_encoder()(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 5, const_cast<void*>(buf), dim, stride, box,
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
    auto go = [&](auto kern, int bytes, int rows) {
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
        kern<<<grid, dim3(32, rows), (size_t)bytes, c->stream>>>(P, *m, (const S*)a, (S*)b, lk, tl, c->d_status);
    };
    if (wy == 8)
        go(k_step_d3q19_tma<PREC, 8>, TmaLayout<8>::BYTES, 8);
    else
        go(k_step_d3q19_tma<PREC, 6>, TmaLayout<6>::BYTES, 6);
    return cudaGetLastError();
}

// ----------------------------------------------------- psi-exchange march (host)
static size_t xchg_smem(int wy) { return (8 * (size_t)(wy + 2) * 34 + 3 * 11 * 32 * (size_t)wy) * sizeof(float); }

int xchg_resident_blocks(const lbcg_ctx* c)
{
    int dev = 0, sms = 0, per = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
    const int threads = 32 * c->block_rows;
    cudaError_t e;
    switch (c->p.precision) {
        case LBCG_FP32:
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_step_d3q19_xchg<LBCG_FP32>, threads,
                                                              xchg_smem(c->block_rows));
            break;
        case LBCG_FP32_DEV:
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_step_d3q19_xchg<LBCG_FP32_DEV>, threads,
                                                              xchg_smem(c->block_rows));
            break;
        case LBCG_FP16_SCALED:
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_step_d3q19_xchg<LBCG_FP16_SCALED>, threads,
                                                              xchg_smem(c->block_rows));
            break;
        default: return 0;
    }
    return e == cudaSuccess ? per * sms : 0;
}

// Tables built and the progress bound met: more resident blocks than a tile's neighbours
// span in list order (nsx + 2 columns) times the planes a tile can run ahead (rows + 2).
bool xchg_supported(const lbcg_ctx* c)
{
    return c->d_xtiles && c->xntiles > 0 && c->xwy == c->block_rows && c->xrows == c->kp.rows &&
           (long long)c->xgrid >= (long long)(c->xnsx + 2) * (c->xrows + 2) + 32 && small_index(c);
}

template <int PREC>
static cudaError_t launch_d3q19_xchg(lbcg_ctx* c, const void* a, void* b)
{
    using S = typename Store<PREC>::S;
    XParams X;
    X.nsx = c->xnsx;
    X.nsy = c->xnsy;
    X.ntiles = c->xntiles;
    X.rows = c->xrows;
    X.tiles = c->d_xtiles;
    X.map = c->d_xmap;
    X.psi = c->d_psibuf;
    X.flags = c->d_xflags;
    X.ctl = c->d_xctl;
    X.status = c->d_status;
    k_step_d3q19_xchg<PREC><<<c->xgrid, dim3(32, c->block_rows), xchg_smem(c->block_rows), c->stream>>>(
        c->kp, X, (const S*)a, (S*)b, c->d_link);
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
    if constexpr (sizeof(S) == 4) {
        if (variant == 4) {
            const size_t smem4 = (4 * sizeof(T) + (size_t)kAsyncStages * 2 * 19 * sizeof(S)) * (size_t)wy * 32;
            if (small_index(c)) {
                cudaFuncSetAttribute(k_step_d3q19_async<PREC, int>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)smem4);
                k_step_d3q19_async<PREC, int><<<grid, block, smem4, c->stream>>>(P, (const S*)a, (S*)b, lk, tl);
            } else {
                cudaFuncSetAttribute(k_step_d3q19_async<PREC, long long>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)smem4);
                k_step_d3q19_async<PREC, long long><<<grid, block, smem4, c->stream>>>(P, (const S*)a, (S*)b, lk, tl);
            }
            return cudaGetLastError();
        }
    }
    if (variant == 7 && !KEEP) {
        const size_t smem7 = smem + 2 * 11 * (size_t)wy * 32 * sizeof(T);
        auto go = [&](auto kern) {
            cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem7);
            kern<<<grid, block, smem7, c->stream>>>(P, (const S*)a, (S*)b, lk, tl);
        };
        if (small_index(c))
            go(k_step_d3q19_moms<PREC, int>);
        else
            go(k_step_d3q19_moms<PREC, long long>);
        return cudaGetLastError();
    }
    if (variant == 6 && !KEEP) {
        if (small_index(c))
            k_step_d3q19_mom<PREC, int><<<grid, block, smem, c->stream>>>(P, (const S*)a, (S*)b, lk, tl);
        else
            k_step_d3q19_mom<PREC, long long><<<grid, block, smem, c->stream>>>(P, (const S*)a, (S*)b, lk, tl);
        return cudaGetLastError();
    }
    if (variant == 5 && !KEEP) {
        if (small_index(c))
            k_step_d3q19_occ<PREC, int><<<grid, block, smem, c->stream>>>(P, (const S*)a, (S*)b, lk, tl);
        else
            k_step_d3q19_occ<PREC, long long><<<grid, block, smem, c->stream>>>(P, (const S*)a, (S*)b, lk, tl);
        return cudaGetLastError();
    }
    if (variant == 3) {
        const size_t smem3 = (4 + 2 * 2 * 19) * (size_t)wy * 32 * sizeof(T);
        if (small_index(c)) {
            cudaFuncSetAttribute(k_step_d3q19_pipe<PREC, int>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem3);
            k_step_d3q19_pipe<PREC, int><<<grid, block, smem3, c->stream>>>(P, (const S*)a, (S*)b, lk, tl);
        } else {
            cudaFuncSetAttribute(k_step_d3q19_pipe<PREC, long long>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem3);
            k_step_d3q19_pipe<PREC, long long><<<grid, block, smem3, c->stream>>>(P, (const S*)a, (S*)b, lk, tl);
        }
        return cudaGetLastError();
    }
    if (small_index(c))
        k_step_d3q19<PREC, KEEP, int><<<grid, block, smem, c->stream>>>(P, (const S*)a, (S*)b, lk, tl);
    else
        k_step_d3q19<PREC, KEEP, long long><<<grid, block, smem, c->stream>>>(P, (const S*)a, (S*)b, lk, tl);
    return cudaGetLastError();
}

int effective_variant(const lbcg_ctx* c)
{
    const int prec = c->p.precision;
    // D2Q9: 3 the pipelined march; the moment march (6) by default for the regularized
    // collision (measured fastest on large boxes); every other value the plain march
    if (c->p.lattice == LBCG_D2Q9) {
        if (c->variant == 3) return 3;
        return (c->variant == 0 || c->variant == 6) && c->p.collision == LBCG_REG ? 6 : 0;
    }
    // default (measured fastest): the moment march with its moments in registers; the BGK
    // update needs the individual populations and re-reads them (three blocks per SM, FP64 two)
    const bool reg = c->p.collision == LBCG_REG;
    int v = c->variant != 0 ? c->variant : (reg ? 6 : (prec == LBCG_FP64 ? 2 : 5));
    if (v == 8 && !tma_supported(c)) v = prec == LBCG_FP64 ? 6 : 7;
    if (v == 10 && !xchg_supported(c)) v = 6;
    if ((v == 6 || v == 7) && !reg) v = prec == LBCG_FP64 ? 2 : 5;
    if (v == 4 && prec != LBCG_FP32 && prec != LBCG_FP32_DEV) v = 2;
    return v;
}

cudaError_t launch_step(lbcg_ctx* c, const void* a, void* b)
{
    const int prec = c->p.precision;
    if (c->p.lattice == LBCG_D2Q9) {
        switch (prec) {
            case LBCG_FP64: return launch_d2q9<LBCG_FP64>(c, a, b);
            case LBCG_FP32: return launch_d2q9<LBCG_FP32>(c, a, b);
            case LBCG_FP32_DEV: return launch_d2q9<LBCG_FP32_DEV>(c, a, b);
            case LBCG_FP16_SCALED: return launch_d2q9<LBCG_FP16_SCALED>(c, a, b);
        }
    } else {
        // default: 5 (re-read, three blocks per SM; measured fastest) for 4- and 2-byte storage;
        // FP64 re-reads with two blocks per SM (it spills at the three-block register budget)
        const int v = effective_variant(c);
        if (v == 10) {
            if (prec == LBCG_FP32) return launch_d3q19_xchg<LBCG_FP32>(c, a, b);
            if (prec == LBCG_FP32_DEV) return launch_d3q19_xchg<LBCG_FP32_DEV>(c, a, b);
            return launch_d3q19_xchg<LBCG_FP16_SCALED>(c, a, b);
        }
        if (v == 8) {
            if (prec == LBCG_FP32) return launch_d3q19_tma<LBCG_FP32>(c, a, b);
            return launch_d3q19_tma<LBCG_FP32_DEV>(c, a, b);
        }
        const bool keep = v == 1;
        switch (prec) {
            case LBCG_FP64:
                return keep ? launch_d3q19<LBCG_FP64, true>(c, a, b, v) : launch_d3q19<LBCG_FP64, false>(c, a, b, v);
            case LBCG_FP32:
                return keep ? launch_d3q19<LBCG_FP32, true>(c, a, b, v) : launch_d3q19<LBCG_FP32, false>(c, a, b, v);
            case LBCG_FP32_DEV:
                return keep ? launch_d3q19<LBCG_FP32_DEV, true>(c, a, b, v)
                            : launch_d3q19<LBCG_FP32_DEV, false>(c, a, b, v);
            case LBCG_FP16_SCALED:
                return keep ? launch_d3q19<LBCG_FP16_SCALED, true>(c, a, b, v)
                            : launch_d3q19<LBCG_FP16_SCALED, false>(c, a, b, v);
        }
    }
    return cudaErrorInvalidValue;
}

}  // namespace lbcg
