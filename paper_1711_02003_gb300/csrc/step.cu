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
//   D3Q19: one block owns 30 x (rows-2) sites in x-y (ring lanes and ring warps)
//          and marches along z; psi of four z-planes is staged in shared memory.
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

// upstream neighbours (x - 1, x + 1) clamped into the box; a clamped one is only
// reached through a bounce-back link, so its value is never used
__device__ __forceinline__ void nbrs(int vs, int n, int per, int& vm, int& vp)
{
    vm = vs - 1 >= 0 ? vs - 1 : (per ? n - 1 : 0);
    vp = vs + 1 < n ? vs + 1 : (per ? 0 : n - 1);
}

// Streamed populations (pull, Eq. 1) of the fluid site (xs, ys, zs) into r/g and
// its psi.  Upstream of direction i is x - c_i.
template <int LAT, int PREC>
__device__ __forceinline__ typename Store<PREC>::T pull_fluid(
    const KParams& P, const typename Store<PREC>::S* __restrict__ A, int xs, int xm, int xp, int ys, int ym,
    int yp, int zs, int zm, int zp, uint32_t lk, typename Store<PREC>::T (&r)[Lat<LAT>::Q],
    typename Store<PREC>::T (&g)[Lat<LAT>::Q])
{
    using L = Lat<LAT>;
    using SP = Store<PREC>;
    using T = typename SP::T;
    constexpr int Q = L::Q;
    const size_t self = (size_t)xs + (size_t)P.nx * ((size_t)ys + (size_t)P.ny * (size_t)zs);
    T rr = 0, sg = 0;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        const int sx = L::cx(i) > 0 ? xm : (L::cx(i) < 0 ? xp : xs);
        const int sy = L::cy(i) > 0 ? ym : (L::cy(i) < 0 ? yp : ys);
        const int sz = L::cz(i) > 0 ? zm : (L::cz(i) < 0 ? zp : zs);
        const size_t src = (size_t)sx + (size_t)P.nx * ((size_t)sy + (size_t)P.ny * (size_t)sz);
        const bool bounce = (lk >> i) & 1u;
        SP::load(A, P.np, Q, bounce ? L::opp(i) : i, bounce ? self : src, phys<T>(P), L::cls(i), r[i], g[i]);
        rr += r[i];
        sg += g[i];
    }
    const T rho = phys<T>(P).rho0 + sg;
    return (rr - (rho - rr)) / rho;
}

// psi of a port ghost site from its own (already filled) populations
template <int LAT, int PREC>
__device__ __forceinline__ typename Store<PREC>::T ghost_psi(const KParams& P,
                                                             const typename Store<PREC>::S* __restrict__ A,
                                                             size_t s)
{
    using L = Lat<LAT>;
    using SP = Store<PREC>;
    using T = typename SP::T;
    T rr = 0, sg = 0;
#pragma unroll
    for (int i = 0; i < L::Q; ++i) {
        T r, g;
        SP::load(A, P.np, L::Q, i, s, phys<T>(P), L::cls(i), r, g);
        rr += r;
        sg += g;
    }
    const T rho = phys<T>(P).rho0 + sg;
    return (rr - (rho - rr)) / rho;
}

template <int LAT, int PREC>
__device__ __forceinline__ void store_site(const KParams& P, typename Store<PREC>::S* __restrict__ B, size_t s,
                                           const typename Store<PREC>::T (&r)[Lat<LAT>::Q],
                                           const typename Store<PREC>::T (&g)[Lat<LAT>::Q])
{
    using L = Lat<LAT>;
    using T = typename Store<PREC>::T;
#pragma unroll
    for (int i = 0; i < L::Q; ++i) Store<PREC>::store(B, P.np, L::Q, i, s, phys<T>(P), L::cls(i), r[i], g[i]);
}

// ------------------------------------------------------------------------ D2Q9
template <int PREC>
__global__ void __launch_bounds__(256) k_step_d2q9(const KParams P, const typename Store<PREC>::S* __restrict__ A,
                                                   typename Store<PREC>::S* __restrict__ B,
                                                   const uint32_t* __restrict__ link)
{
    using T = typename Store<PREC>::T;
    using L = Lat<0>;
    constexpr int Q = 9;
    const int lane = threadIdx.x & 31;
    const int gw = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    if (gw >= P.nsx * P.nsy) return;  // warp-uniform
    const int sxi = gw % P.nsx, syi = gw / P.nsx;
    const int nx = P.nx, ny = P.ny;
    const int x = sxi * 30 + lane - 1;
    int xs;
    const bool xok = wrap_coord(x, nx, P.per[0], xs) && x <= nx;
    const bool xint = lane >= 1 && lane <= 30 && x < nx;
    int xm, xp;
    nbrs(xs, nx, P.per[0], xm, xp);
    const int y0 = syi * P.rows;
    const int y1 = min(y0 + P.rows, ny);
    const T psi_wall = phys<T>(P).psi_wall;

    T psi_a = psi_wall, psi_b = psi_wall;  // rows yy-2, yy-1
    T rb[Q], gb[Q];                        // populations of row yy-1
    bool coll_b = false;
#pragma unroll
    for (int i = 0; i < Q; ++i) rb[i] = gb[i] = T(0);

    for (int yy = y0 - 1; yy <= y1; ++yy) {
        int ys;
        const bool yok = wrap_coord(yy, ny, P.per[1], ys);
        int ym, yp;
        nbrs(ys, ny, P.per[1], ym, yp);
        T rn[Q], gn[Q];
#pragma unroll
        for (int i = 0; i < Q; ++i) rn[i] = gn[i] = T(0);
        T psi_n = psi_wall;
        bool fluid_n = false;
        if (xok && yok) {
            const size_t s = (size_t)xs + (size_t)nx * (size_t)ys;
            const uint32_t lk = link ? __ldg(link + s) : 0u;
            const uint32_t type = (lk >> kTypeShift) & 3u;
            if (type == kTypeFluid) {
                psi_n = pull_fluid<0, PREC>(P, A, xs, xm, xp, ys, ym, yp, 0, 0, 0, lk, rn, gn);
                fluid_n = true;
            } else if (type == kTypePort) {
                psi_n = ghost_psi<0, PREC>(P, A, s);
            }
        }
        if (yy - 1 >= y0) {  // warp-uniform: collide row yy-1
            const T am = __shfl_up_sync(0xffffffffu, psi_a, 1), ap = __shfl_down_sync(0xffffffffu, psi_a, 1);
            const T bm = __shfl_up_sync(0xffffffffu, psi_b, 1), bp = __shfl_down_sync(0xffffffffu, psi_b, 1);
            const T nm = __shfl_up_sync(0xffffffffu, psi_n, 1), np = __shfl_down_sync(0xffffffffu, psi_n, 1);
            if (coll_b) {
                // neighbour psi in direction order; the row index is cy: -1 -> a, 0 -> b, +1 -> n
                T F[3] = {T(0), T(0), T(0)};
#pragma unroll
                for (int i = 1; i < Q; ++i) {
                    const int cx = L::cx(i), cy = L::cy(i);
                    const T v = cy < 0 ? (cx < 0 ? am : (cx > 0 ? ap : psi_a))
                              : cy > 0 ? (cx < 0 ? nm : (cx > 0 ? np : psi_n))
                                       : (cx < 0 ? bm : (cx > 0 ? bp : psi_b));
                    const T wv = (T)L::w(i) * v;
                    if (cx) F[0] += cx > 0 ? wv : -wv;
                    if (cy) F[1] += cy > 0 ? wv : -wv;
                }
                F[0] *= T(3);
                F[1] *= T(3);
                collide_site<0, T>(P, phys<T>(P), rb, gb, F);
                int yc = yy - 1;
                store_site<0, PREC>(P, B, (size_t)xs + (size_t)nx * (size_t)yc, rb, gb);
            }
        }
        psi_a = psi_b;
        psi_b = psi_n;
        coll_b = fluid_n && xint && yy >= y0 && yy < y1;
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            rb[i] = rn[i];
            gb[i] = gn[i];
        }
    }
}

// ----------------------------------------------------------------------- D3Q19
// blockDim = (32, WY); warp w owns row y = by*(WY-2) + w - 1; rows 1..WY-2 collide.
template <int PREC, bool KEEP>
__global__ void __launch_bounds__(512) k_step_d3q19(const KParams P, const typename Store<PREC>::S* __restrict__ A,
                                                    typename Store<PREC>::S* __restrict__ B,
                                                    const uint32_t* __restrict__ link)
{
    using T = typename Store<PREC>::T;
    using L = Lat<1>;
    constexpr int Q = 19;
    extern __shared__ unsigned char smem_raw[];
    T* psi_s = reinterpret_cast<T*>(smem_raw);  // [4][WY][32]
    const int lane = threadIdx.x;
    const int w = threadIdx.y;
    const int WY = blockDim.y;
    const int nx = P.nx, ny = P.ny, nz = P.nz;
    const int x = blockIdx.x * 30 + lane - 1;
    const int y = blockIdx.y * (WY - 2) + w - 1;
    int xs, ys;
    const bool xok = wrap_coord(x, nx, P.per[0], xs) && x <= nx;
    const bool yok = wrap_coord(y, ny, P.per[1], ys) && y <= ny;
    const bool inner = lane >= 1 && lane <= 30 && x < nx && w >= 1 && w <= WY - 2 && y < ny;
    int xm, xp, ym, yp;
    nbrs(xs, nx, P.per[0], xm, xp);
    nbrs(ys, ny, P.per[1], ym, yp);
    const int z0 = blockIdx.z * P.rows;
    const int z1 = min(z0 + P.rows, nz);
    const T psi_wall = phys<T>(P).psi_wall;

    T rb[Q], gb[Q];
    bool coll_b = false;
#pragma unroll
    for (int i = 0; i < Q; ++i) rb[i] = gb[i] = T(0);

    for (int zz = z0 - 1; zz <= z1; ++zz) {
        int zs;
        const bool zok = wrap_coord(zz, nz, P.per[2], zs);
        int zm, zp;
        nbrs(zs, nz, P.per[2], zm, zp);
        T rn[Q], gn[Q];
#pragma unroll
        for (int i = 0; i < Q; ++i) rn[i] = gn[i] = T(0);
        T psi_n = psi_wall;
        bool fluid_n = false;
        if (xok && yok && zok) {
            const size_t s = (size_t)xs + (size_t)nx * ((size_t)ys + (size_t)ny * (size_t)zs);
            const uint32_t lk = link ? __ldg(link + s) : 0u;
            const uint32_t type = (lk >> kTypeShift) & 3u;
            if (type == kTypeFluid) {
                psi_n = pull_fluid<1, PREC>(P, A, xs, xm, xp, ys, ym, yp, zs, zm, zp, lk, rn, gn);
                fluid_n = true;
            } else if (type == kTypePort) {
                psi_n = ghost_psi<1, PREC>(P, A, s);
            }
        }
        const int slot_n = (zz - z0 + 1) & 3;
        psi_s[(slot_n * WY + w) * 32 + lane] = psi_n;
        __syncthreads();
        if (zz - 1 >= z0 && coll_b) {
            const int zc = zz - 1;
            int zcs = zc, zcm, zcp;
            nbrs(zcs, nz, P.per[2], zcm, zcp);
            if (!KEEP) {
                const size_t s = (size_t)xs + (size_t)nx * ((size_t)ys + (size_t)ny * (size_t)zcs);
                const uint32_t lk = link ? __ldg(link + s) : 0u;
                pull_fluid<1, PREC>(P, A, xs, xm, xp, ys, ym, yp, zcs, zcm, zcp, lk, rb, gb);
            }
            T F[3] = {T(0), T(0), T(0)};
#pragma unroll
            for (int i = 1; i < Q; ++i) {
                const int cx = L::cx(i), cy = L::cy(i), cz = L::cz(i);
                const int slot = (zc + cz - z0 + 1) & 3;
                const T v = psi_s[(slot * WY + (w + cy)) * 32 + (lane + cx)];
                const T wv = (T)L::w(i) * v;
                if (cx) F[0] += cx > 0 ? wv : -wv;
                if (cy) F[1] += cy > 0 ? wv : -wv;
                if (cz) F[2] += cz > 0 ? wv : -wv;
            }
            F[0] *= T(3);
            F[1] *= T(3);
            F[2] *= T(3);
            collide_site<1, T>(P, phys<T>(P), rb, gb, F);
            store_site<1, PREC>(P, B, (size_t)xs + (size_t)nx * ((size_t)ys + (size_t)ny * (size_t)zcs), rb, gb);
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

// ---------------------------------------------------------------------- launchers
template <int PREC>
static cudaError_t launch_d2q9(lbcg_ctx* c, const void* a, void* b)
{
    using S = typename Store<PREC>::S;
    const KParams& P = c->kp;
    const long long warps = (long long)P.nsx * P.nsy;
    const int threads = 256;
    const long long blocks = (warps * 32 + threads - 1) / threads;
    k_step_d2q9<PREC><<<(unsigned)blocks, threads, 0, c->stream>>>(P, (const S*)a, (S*)b,
                                                                    c->any_link ? c->d_link : nullptr);
    return cudaGetLastError();
}

template <int PREC, bool KEEP>
static cudaError_t launch_d3q19(lbcg_ctx* c, const void* a, void* b)
{
    using S = typename Store<PREC>::S;
    using T = typename Store<PREC>::T;
    const KParams& P = c->kp;
    const int wy = c->block_rows;
    dim3 block(32, wy);
    dim3 grid(P.nsx, P.nsy, P.nsz);
    size_t smem = 4 * (size_t)wy * 32 * sizeof(T);
    k_step_d3q19<PREC, KEEP><<<grid, block, smem, c->stream>>>(P, (const S*)a, (S*)b,
                                                                c->any_link ? c->d_link : nullptr);
    return cudaGetLastError();
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
        switch (prec) {
            case LBCG_FP64: return launch_d3q19<LBCG_FP64, false>(c, a, b);
            case LBCG_FP32: return launch_d3q19<LBCG_FP32, true>(c, a, b);
            case LBCG_FP32_DEV: return launch_d3q19<LBCG_FP32_DEV, true>(c, a, b);
            case LBCG_FP16_SCALED: return launch_d3q19<LBCG_FP16_SCALED, true>(c, a, b);
        }
    }
    return cudaErrorInvalidValue;
}

}  // namespace lbcg
