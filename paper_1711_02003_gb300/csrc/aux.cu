// aux.cu -- kernels around the fused step: port ghost refill, initial equilibrium,
// field and population read-back, FP64 observable reductions and droplet labelling
// (arXiv:1711.02003: Eqs. 2-3 moments, Eq. 6 equilibrium, Eq. 8 pressure; the
// observables follow the resting-droplet and droplet-size analyses of Secs. IV A-B).
#include "lbcg_device.cuh"

namespace lbcg {

// ----------------------------------------------------------------- helpers
template <int LAT, typename T>
__device__ __forceinline__ T feq_comp(const T (&phi)[3], T rho_k, T ux, T uy, T uz, int i)
{
    using L = Lat<LAT>;
    const T cu = (T)L::cx(i) * ux + (T)L::cy(i) * uy + (T)L::cz(i) * uz;
    const T usq = ux * ux + uy * uy + uz * uz;
    return rho_k * (phi[L::cls(i)] + (T)L::w(i) * (T(3) * cu + T(4.5) * cu * cu - T(1.5) * usq));
}

__device__ __forceinline__ void coords(long long s, int nx, int ny, int& x, int& y, int& z)
{
    x = (int)(s % nx);
    long long r = s / nx;
    y = (int)(r % ny);
    z = (int)(r / ny);
}

// red and blue populations of direction i at site s, decoded from any storage format
template <int LAT, int PREC>
__device__ __forceinline__ void load_rb(const KParams& P, const typename Store<PREC>::S* a, int i, size_t s,
                                        double& fr, double& fb)
{
    using SP = Store<PREC>;
    using T = typename SP::T;
    if constexpr (PREC == LBCG_FP64 || PREC == LBCG_FP32) {
        fr = (double)a[(size_t)i * P.np + s];
        fb = (double)a[(size_t)(Lat<LAT>::Q + i) * P.np + s];
    } else {
        T r, g;
        SP::load(a, (size_t)i * P.np + s, (size_t)(Lat<LAT>::Q + i) * P.np + s, phys<T>(P), Lat<LAT>::cls(i), r, g);
        fr = (double)r;
        fb = ((double)g + P.pd.wr0[Lat<LAT>::cls(i)]) - (double)r;
    }
}

// store red and blue populations of direction i at site s into any storage format
template <int LAT, int PREC>
__device__ __forceinline__ void store_rb(const KParams& P, typename Store<PREC>::S* a, int i, size_t s, double fr,
                                         double fb)
{
    using SP = Store<PREC>;
    using S = typename SP::S;
    using T = typename SP::T;
    if constexpr (PREC == LBCG_FP64 || PREC == LBCG_FP32) {
        a[(size_t)i * P.np + s] = (S)fr;
        a[(size_t)(Lat<LAT>::Q + i) * P.np + s] = (S)fb;
    } else {
        const int c = Lat<LAT>::cls(i);
        SP::store(a, (size_t)i * P.np + s, (size_t)(Lat<LAT>::Q + i) * P.np + s, phys<T>(P), c, (T)fr,
                  (T)((fr + fb) - P.pd.wr0[c]));
    }
}

// ------------------------------------------------------------ port ghost refill
// Ghost g of port m, inward neighbour x' (a fluid site):
//   velocity:      f^k = f^{k,eq}(chi^k rho', u_port) + chi^k (f(x') - f^eq(x'))
//   pressure:      f^k = f^{k,eq}(rho_port rho'^k / rho', u') + f^k(x') - f^{k,eq}(x')
//   zero-gradient: f^k = f^k(x')
// Arithmetic in FP64 (a few thousand sites per step).
template <int LAT, int PREC>
__global__ void k_fill_ports(const KParams P, typename Store<PREC>::S* __restrict__ a, const int* __restrict__ tab,
                             const double* __restrict__ gu, int ng)
{
    using L = Lat<LAT>;
    constexpr int Q = L::Q;
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= ng) return;
    const size_t g = (size_t)tab[t];
    const size_t xp = (size_t)tab[ng + t];
    const int kind = tab[3 * ng + t];
    double fr[Q], fb[Q];
#pragma unroll
    for (int i = 0; i < Q; ++i) load_rb<LAT, PREC>(P, a, i, xp, fr[i], fb[i]);
    if (kind == LBCG_PORT_ZERO_GRADIENT) {
#pragma unroll
        for (int i = 0; i < Q; ++i) store_rb<LAT, PREC>(P, a, i, g, fr[i], fb[i]);
        return;
    }
    double rr = 0, rb = 0, jx = 0, jy = 0, jz = 0;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        rr += fr[i];
        rb += fb[i];
        const double f = fr[i] + fb[i];
        jx += L::cx(i) * f;
        jy += L::cy(i) * f;
        jz += L::cz(i) * f;
    }
    const double rho = rr + rb;
    const double ux = jx / rho, uy = jy / rho, uz = jz / rho;
    const double(&phR)[3] = P.pd.phiR;
    const double(&phB)[3] = P.pd.phiB;
    if (kind == LBCG_PORT_VELOCITY) {
        const double vx = gu[t], vy = gu[ng + t], vz = gu[2 * ng + t];
        const double psi = gu[4 * ng + t];
        const double xr = (1.0 + psi) / 2.0, xb = (1.0 - psi) / 2.0;
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            const double fneq = (fr[i] + fb[i]) - (feq_comp<LAT, double>(phR, rr, ux, uy, uz, i) +
                                                   feq_comp<LAT, double>(phB, rb, ux, uy, uz, i));
            const double gr = feq_comp<LAT, double>(phR, xr * rho, vx, vy, vz, i) + xr * fneq;
            const double gb = feq_comp<LAT, double>(phB, xb * rho, vx, vy, vz, i) + xb * fneq;
            store_rb<LAT, PREC>(P, a, i, g, gr, gb);
        }
    } else {
        const double rho_out = gu[3 * ng + t];
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            const double gr = feq_comp<LAT, double>(phR, rho_out * rr / rho, ux, uy, uz, i) +
                              (fr[i] - feq_comp<LAT, double>(phR, rr, ux, uy, uz, i));
            const double gb = feq_comp<LAT, double>(phB, rho_out * rb / rho, ux, uy, uz, i) +
                              (fb[i] - feq_comp<LAT, double>(phB, rb, ux, uy, uz, i));
            store_rb<LAT, PREC>(P, a, i, g, gr, gb);
        }
    }
}

// ---------------------------------------------------------------- initial state
// f^k = f^{k,eq}(rho^k, u) (Eq. 6) at fluid sites, zero elsewhere.
template <int LAT, int PREC>
__global__ void k_init(const KParams P, const double* __restrict__ rr, const double* __restrict__ rb,
                       const double* __restrict__ u, const uint32_t* __restrict__ link, long long n,
                       typename Store<PREC>::S* __restrict__ a)
{
    using L = Lat<LAT>;
    for (long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x; s < n;
         s += (long long)gridDim.x * blockDim.x) {
        const bool fluid = link == nullptr || ((link[s] >> kTypeShift) & 3u) == kTypeFluid;
        const double r = fluid ? rr[s] : 0.0, b = fluid ? rb[s] : 0.0;
        double ux = 0, uy = 0, uz = 0;
        if (u) {
            ux = u[s];
            uy = u[n + s];
            if (L::D == 3) uz = u[2 * n + s];
        }
#pragma unroll
        for (int i = 0; i < L::Q; ++i)
            store_rb<LAT, PREC>(P, a, i, (size_t)s, feq_comp<LAT, double>(P.pd.phiR, r, ux, uy, uz, i),
                                feq_comp<LAT, double>(P.pd.phiB, b, ux, uy, uz, i));
    }
}

// --------------------------------------------------------------------- fields
template <int LAT, int PREC>
__global__ void k_fields(const KParams P, const typename Store<PREC>::S* __restrict__ a,
                         const uint32_t* __restrict__ link, long long n, double* __restrict__ orr,
                         double* __restrict__ orb, double* __restrict__ ou)
{
    using L = Lat<LAT>;
    for (long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x; s < n;
         s += (long long)gridDim.x * blockDim.x) {
        const bool fluid = link == nullptr || ((link[s] >> kTypeShift) & 3u) == kTypeFluid;
        double rr = 0, rb = 0, jx = 0, jy = 0, jz = 0;
        if (fluid) {
#pragma unroll
            for (int i = 0; i < L::Q; ++i) {
                double fr, fb;
                load_rb<LAT, PREC>(P, a, i, (size_t)s, fr, fb);
                rr += fr;
                rb += fb;
                const double f = fr + fb;
                jx += L::cx(i) * f;
                jy += L::cy(i) * f;
                jz += L::cz(i) * f;
            }
        }
        const double rho = rr + rb;
        orr[s] = rr;
        orb[s] = rb;
        ou[s] = rho > 0 ? jx / rho : 0.0;
        ou[n + s] = rho > 0 ? jy / rho : 0.0;
        if (L::D == 3) ou[2 * n + s] = rho > 0 ? jz / rho : 0.0;
    }
}

// ---------------------------------------------------------- population transfer
template <int LAT, int PREC>
__global__ void k_plane_to_f64(const KParams P, const typename Store<PREC>::S* __restrict__ a, int k, int i,
                               long long n, double* __restrict__ out)
{
    for (long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x; s < n;
         s += (long long)gridDim.x * blockDim.x) {
        double fr, fb;
        load_rb<LAT, PREC>(P, a, i, (size_t)s, fr, fb);
        out[s] = k == 0 ? fr : fb;
    }
}

// direction i from two staged FP64 planes (red, blue)
template <int LAT, int PREC>
__global__ void k_dir_from_f64(const KParams P, const double* __restrict__ fr, const double* __restrict__ fb,
                               int i, long long n, typename Store<PREC>::S* __restrict__ a)
{
    for (long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x; s < n;
         s += (long long)gridDim.x * blockDim.x)
        store_rb<LAT, PREC>(P, a, i, (size_t)s, fr[s], fb[s]);
}

// ------------------------------------------------------------------ reductions
// Deterministic two-level FP64 reductions: a fixed grid of kMaxPartials-or-fewer
// blocks, each thread strides over sites in a fixed order, warp shuffles then
// shared memory inside a block, per-block partials reduced by one block in index
// order.  Results do not depend on timing.

template <int NS>
__device__ __forceinline__ void block_reduce(double (&v)[NS], const bool (&is_max)[NS], double* out_row)
{
    __shared__ double sh[32][NS];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < NS; ++k)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const double t = __shfl_xor_sync(0xffffffffu, v[k], o);
            v[k] = is_max[k] ? fmax(v[k], t) : v[k] + t;
        }
    if (lane == 0)
#pragma unroll
        for (int k = 0; k < NS; ++k) sh[warp][k] = v[k];
    __syncthreads();
    if (warp == 0) {
        const int nw = blockDim.x >> 5;
#pragma unroll
        for (int k = 0; k < NS; ++k) {
            double t = lane < nw ? sh[lane][k] : (is_max[k] ? 0.0 : 0.0);
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                const double q = __shfl_xor_sync(0xffffffffu, t, o);
                t = is_max[k] ? fmax(t, q) : t + q;
            }
            if (lane == 0) out_row[k] = t;
        }
    }
}

constexpr int kS1 = 8;  // mass_r, mass_b, mom x, y, z, amount, umax, nonfinite
constexpr int kS2 = 4;  // p_in sum, n_in, p_out sum, n_out

template <int LAT, int PREC>
__global__ void __launch_bounds__(256) k_obs_pass1(const KParams P, const typename Store<PREC>::S* __restrict__ a,
                                                   const uint32_t* __restrict__ link, long long n,
                                                   double* __restrict__ partials)
{
    using L = Lat<LAT>;
    double v[kS1] = {0, 0, 0, 0, 0, 0, 0, 0};
    const bool mx[kS1] = {false, false, false, false, false, false, true, false};
    for (long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x; s < n;
         s += (long long)gridDim.x * blockDim.x) {
        if (link && ((link[s] >> kTypeShift) & 3u) != kTypeFluid) continue;
        double rr = 0, rb = 0, jx = 0, jy = 0, jz = 0;
#pragma unroll
        for (int i = 0; i < L::Q; ++i) {
            double fr, fb;
            load_rb<LAT, PREC>(P, a, i, (size_t)s, fr, fb);
            rr += fr;
            rb += fb;
            const double f = fr + fb;
            jx += L::cx(i) * f;
            jy += L::cy(i) * f;
            jz += L::cz(i) * f;
        }
        const double rho = rr + rb;
        if (!(rho > 0.0) || !isfinite(rho)) {
            v[7] += 1.0;
            continue;
        }
        v[0] += rr;
        v[1] += rb;
        v[2] += jx;
        v[3] += jy;
        v[4] += jz;
        v[5] += (1.0 + (rr - rb) / rho) / 2.0;
        v[6] = fmax(v[6], sqrt(jx * jx + jy * jy + jz * jz) / rho);
    }
    block_reduce<kS1>(v, mx, partials + (size_t)blockIdx.x * kObsSlots);
}

template <int LAT, int PREC>
__global__ void __launch_bounds__(256) k_obs_pass2(const KParams P, const typename Store<PREC>::S* __restrict__ a,
                                                   const uint32_t* __restrict__ link, long long n, double cx,
                                                   double cy, double cz, double kpr, double kpb,
                                                   const double* __restrict__ res, double* __restrict__ partials)
{
    using L = Lat<LAT>;
    const double r_in = res[9], r_out = res[10];
    double v[kS2] = {0, 0, 0, 0};
    const bool mx[kS2] = {false, false, false, false};
    for (long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x; s < n;
         s += (long long)gridDim.x * blockDim.x) {
        if (link && ((link[s] >> kTypeShift) & 3u) != kTypeFluid) continue;
        int x, y, z;
        coords(s, P.nx, P.ny, x, y, z);
        double d2 = 0.0;
        {
            double dd = fabs((double)x - cx);
            if (P.per[0] && P.nx - dd < dd) dd = P.nx - dd;
            d2 += dd * dd;
            dd = fabs((double)y - cy);
            if (P.per[1] && P.ny - dd < dd) dd = P.ny - dd;
            d2 += dd * dd;
            if (L::D == 3) {
                dd = fabs((double)z - cz);
                if (P.per[2] && P.nz - dd < dd) dd = P.nz - dd;
                d2 += dd * dd;
            }
        }
        const double r = sqrt(d2);
        if (r >= r_in && r <= r_out) continue;
        double rr = 0, rb = 0;
#pragma unroll
        for (int i = 0; i < L::Q; ++i) {
            double fr, fb;
            load_rb<LAT, PREC>(P, a, i, (size_t)s, fr, fb);
            rr += fr;
            rb += fb;
        }
        const double p = kpr * rr + kpb * rb;
        if (r < r_in) {
            v[0] += p;
            v[1] += 1.0;
        } else {
            v[2] += p;
            v[3] += 1.0;
        }
    }
    block_reduce<kS2>(v, mx, partials + (size_t)blockIdx.x * kObsSlots);
}

// one block: reduce nb partial rows of ns slots in block-index order into res[off..]
__global__ void k_obs_final(const double* __restrict__ partials, int nb, int ns, unsigned maxmask, int off,
                            double* __restrict__ res, int dim, double r_in, double r_out)
{
    // thread k reduces slot k sequentially over blocks: fixed order
    const int k = threadIdx.x;
    if (k < ns) {
        const bool is_max = (maxmask >> k) & 1u;
        double t = 0.0;
        for (int b = 0; b < nb; ++b) {
            const double q = partials[(size_t)b * kObsSlots + k];
            t = is_max ? fmax(t, q) : t + q;
        }
        res[off + k] = t;
    }
    __syncthreads();
    if (off == 0 && k == 0) {
        const double amount = res[5];
        const double pi = 3.14159265358979323846;
        const double reff = dim == 2 ? sqrt(amount / pi) : cbrt(3.0 * amount / (4.0 * pi));
        res[8] = reff;
        res[9] = r_in < 0.0 ? reff / 2.0 : r_in;
        res[10] = r_out < 0.0 ? reff + 5.0 : r_out;
    }
}

// ------------------------------------------------------------------- labelling
// Union-find over the face graph of droplet sites (rho_R > rho_B): every union
// links the larger root under the smaller with atomicMin and retries until it
// lands on a root (Playne and Hawick's GPU connected-component scheme), so each
// final root is the smallest index of its component.  Loops are bounded; a bound
// that is hit sets *flag.
__device__ __forceinline__ int find_root(volatile int* L, int a, int* flag)
{
    for (int it = 0; it < (1 << 28); ++it) {
        const int p = L[a];
        if (p == a) return a;
        a = p;
    }
    *flag = 1;
    return a;
}

__device__ __forceinline__ void unite(int* L, int a, int b, int* flag)
{
    for (int it = 0; it < (1 << 24); ++it) {
        a = find_root(L, a, flag);
        b = find_root(L, b, flag);
        if (a == b) return;
        if (a < b) {
            const int old = atomicMin(L + b, a);
            if (old == b) return;
            b = old;
        } else {
            const int old = atomicMin(L + a, b);
            if (old == a) return;
            a = old;
        }
    }
    *flag = 1;
}

template <int LAT, int PREC>
__global__ void k_label_init(const KParams P, const typename Store<PREC>::S* __restrict__ a,
                             const uint32_t* __restrict__ link, long long n, int* __restrict__ L,
                             double* __restrict__ half)
{
    for (long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x; s < n;
         s += (long long)gridDim.x * blockDim.x) {
        int lab = -1;
        double h = 0.0;
        if (!(link && ((link[s] >> kTypeShift) & 3u) != kTypeFluid)) {
            double rr = 0, rb = 0;
#pragma unroll
            for (int i = 0; i < Lat<LAT>::Q; ++i) {
                double fr, fb;
                load_rb<LAT, PREC>(P, a, i, (size_t)s, fr, fb);
                rr += fr;
                rb += fb;
            }
            if (rr > rb) lab = (int)s;
            h = (1.0 + (rr - rb) / (rr + rb)) / 2.0;
        }
        L[s] = lab;
        half[s] = h;
    }
}

__global__ void k_label_union(const KParams P, int dim, long long n, int* L, int* flag)
{
    for (long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x; s < n;
         s += (long long)gridDim.x * blockDim.x) {
        if (L[s] < 0) continue;
        int x, y, z;
        coords(s, P.nx, P.ny, x, y, z);
        const int dims[3] = {P.nx, P.ny, P.nz};
        for (int ax = 0; ax < dim; ++ax) {
            int v[3] = {x, y, z};
            v[ax] += 1;
            if (v[ax] == dims[ax]) {
                if (!P.per[ax]) continue;
                v[ax] = 0;
            }
            const long long t = (long long)v[0] + (long long)P.nx * ((long long)v[1] + (long long)P.ny * v[2]);
            if (t == s) continue;
            if (((volatile int*)L)[t] < 0) continue;
            unite(L, (int)s, (int)t, flag);
        }
    }
}

__global__ void k_label_flatten(long long n, int* L, int* flag)
{
    for (long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x; s < n;
         s += (long long)gridDim.x * blockDim.x) {
        if (L[s] < 0) continue;
        L[s] = find_root((volatile int*)L, (int)s, flag);
    }
}

// ---------------------------------------------------------------------- launchers
static unsigned grid_for(long long n, int threads = 256)
{
    long long b = (n + threads - 1) / threads;
    if (b > 152LL * 16) b = 152LL * 16;
    if (b < 1) b = 1;
    return (unsigned)b;
}

#define LBCG_DISPATCH(c, F)                                                    \
    do {                                                                       \
        const int lat_ = (c)->p.lattice, prec_ = (c)->p.precision;             \
        if (lat_ == LBCG_D2Q9) {                                               \
            if (prec_ == LBCG_FP64) { F(0, LBCG_FP64); }                       \
            else if (prec_ == LBCG_FP32) { F(0, LBCG_FP32); }                  \
            else if (prec_ == LBCG_FP32_DEV) { F(0, LBCG_FP32_DEV); }          \
            else { F(0, LBCG_FP16_SCALED); }                                   \
        } else {                                                               \
            if (prec_ == LBCG_FP64) { F(1, LBCG_FP64); }                       \
            else if (prec_ == LBCG_FP32) { F(1, LBCG_FP32); }                  \
            else if (prec_ == LBCG_FP32_DEV) { F(1, LBCG_FP32_DEV); }          \
            else { F(1, LBCG_FP16_SCALED); }                                   \
        }                                                                      \
    } while (0)

template <int PREC>
using SOf = typename Store<PREC>::S;

cudaError_t launch_fill_ports(lbcg_ctx* c, void* a)
{
    if (c->nghost == 0) return cudaSuccess;
    const unsigned blocks = (unsigned)((c->nghost + 127) / 128);
#define F_(LAT, PREC) \
    k_fill_ports<LAT, PREC><<<blocks, 128, 0, c->stream>>>(c->kp, (SOf<PREC>*)a, c->d_ghost, c->d_ghost_u, c->nghost)
    LBCG_DISPATCH(c, F_);
#undef F_
    return cudaGetLastError();
}

cudaError_t launch_init(lbcg_ctx* c, const double* rr, const double* rb, const double* u, void* a)
{
    const unsigned g = grid_for(c->n);
    const uint32_t* lk = c->any_link ? c->d_link : nullptr;
#define F_(LAT, PREC) k_init<LAT, PREC><<<g, 256, 0, c->stream>>>(c->kp, rr, rb, u, lk, c->n, (SOf<PREC>*)a)
    LBCG_DISPATCH(c, F_);
#undef F_
    return cudaGetLastError();
}

cudaError_t launch_fields(lbcg_ctx* c, const void* a, double* rr, double* rb, double* u)
{
    const unsigned g = grid_for(c->n);
    const uint32_t* lk = c->any_link ? c->d_link : nullptr;
#define F_(LAT, PREC) \
    k_fields<LAT, PREC><<<g, 256, 0, c->stream>>>(c->kp, (const SOf<PREC>*)a, lk, c->n, rr, rb, u)
    LBCG_DISPATCH(c, F_);
#undef F_
    return cudaGetLastError();
}

cudaError_t launch_pop_plane_to_f64(lbcg_ctx* c, const void* a, int k, int i, double* out)
{
    const unsigned g = grid_for(c->n);
#define F_(LAT, PREC) \
    k_plane_to_f64<LAT, PREC><<<g, 256, 0, c->stream>>>(c->kp, (const SOf<PREC>*)a, k, i, c->n, out)
    LBCG_DISPATCH(c, F_);
#undef F_
    return cudaGetLastError();
}

cudaError_t launch_pops_from_f64(lbcg_ctx* c, const double* f, void* a, int i)
{
    // f holds two staged planes: red then blue of direction i
    const unsigned g = grid_for(c->n);
#define F_(LAT, PREC) \
    k_dir_from_f64<LAT, PREC><<<g, 256, 0, c->stream>>>(c->kp, f, f + c->n, i, c->n, (SOf<PREC>*)a)
    LBCG_DISPATCH(c, F_);
#undef F_
    return cudaGetLastError();
}

cudaError_t launch_observables(lbcg_ctx* c, const void* a, const double centre[3], double r_in, double r_out,
                               double* d_partials, double* d_result)
{
    long long b = (c->n + 255) / 256;
    if (b > kMaxPartials) b = kMaxPartials;
    if (b < 1) b = 1;
    const unsigned nb = (unsigned)b;
    const uint32_t* lk = c->any_link ? c->d_link : nullptr;
    const int dim = c->D;
    const double ar = c->p.alpha_r, ab = c->p.alpha_b;
    const double kpr = dim == 2 ? 3.0 * (1.0 - ar) / 5.0 : (1.0 - ar) / 2.0;
    const double kpb = dim == 2 ? 3.0 * (1.0 - ab) / 5.0 : (1.0 - ab) / 2.0;
#define F_(LAT, PREC) \
    k_obs_pass1<LAT, PREC><<<nb, 256, 0, c->stream>>>(c->kp, (const SOf<PREC>*)a, lk, c->n, d_partials)
    LBCG_DISPATCH(c, F_);
#undef F_
    k_obs_final<<<1, 32, 0, c->stream>>>(d_partials, (int)nb, kS1, 1u << 6, 0, d_result, dim, r_in, r_out);
#define F_(LAT, PREC)                                                                                         \
    k_obs_pass2<LAT, PREC><<<nb, 256, 0, c->stream>>>(c->kp, (const SOf<PREC>*)a, lk, c->n, centre[0],      \
                                                       centre[1], centre[2], kpr, kpb, d_result, d_partials)
    LBCG_DISPATCH(c, F_);
#undef F_
    k_obs_final<<<1, 32, 0, c->stream>>>(d_partials, (int)nb, kS2, 0u, 11, d_result, dim, r_in, r_out);
    return cudaGetLastError();
}

cudaError_t launch_label(lbcg_ctx* c, const void* a, int32_t* L, double* half, int* d_flag)
{
    const unsigned g = grid_for(c->n);
    const uint32_t* lk = c->any_link ? c->d_link : nullptr;
#define F_(LAT, PREC) \
    k_label_init<LAT, PREC><<<g, 256, 0, c->stream>>>(c->kp, (const SOf<PREC>*)a, lk, c->n, L, half)
    LBCG_DISPATCH(c, F_);
#undef F_
    k_label_union<<<g, 256, 0, c->stream>>>(c->kp, c->D, c->n, L, d_flag);
    k_label_flatten<<<g, 256, 0, c->stream>>>(c->n, L, d_flag);
    return cudaGetLastError();
}

}  // namespace lbcg
