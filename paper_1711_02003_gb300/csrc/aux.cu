// aux.cu -- kernels around the fused step: port ghost refill, initial equilibrium,
// field and population read-back, FP64 observable reductions and droplet labelling
// (arXiv:1711.02003: Eqs. 2-3 moments, Eq. 6 equilibrium, Eq. 8 pressure; the
// observables follow the resting-droplet and droplet-size analyses of Secs. IV A-B).
#include "obs_kernels.cuh"

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

constexpr int kFillThreads = 64;

template <int LAT, int PREC>
__global__ void __launch_bounds__(kFillThreads) k_fill_ports(const KParams P, typename Store<PREC>::S* __restrict__ a,
                                                             const int* __restrict__ tab,
                                                             const double* __restrict__ gu, int ng,
                                                             typename Store<PREC>::T* __restrict__ gpsi)
{
    const int t = (int)(blockIdx.x * blockDim.x + threadIdx.x);
    if (t >= ng) return;
    fill_one<LAT, PREC>(P, a, tab, gu, ng, t, gpsi);
}

// batched refill: work item (slot, first ghost, count <= kFillThreads), one thread per
// ghost; node k refills the source buffer of step k of instances with steps > k
template <int LAT, int PREC>
__global__ void __launch_bounds__(kFillThreads) k_batch_fill(const BatchSlot* __restrict__ slots,
                                                             const BatchItem* __restrict__ items,
                                                             const int* __restrict__ nitems, int k)
{
    const int w = blockIdx.x;
    if (w >= *nitems) return;
    const BatchItem it = items[w];
    const BatchSlot& sl = slots[it.slot];
    if (k >= sl.steps) return;
    if ((int)threadIdx.x >= it.y) return;
    typename Store<PREC>::S* src = (typename Store<PREC>::S*)((k & 1) ? sl.b : sl.a);
    // the source buffer's ghost-psi table too, read by the batched march's port lanes
    fill_one<LAT, PREC>(sl.kp, src, sl.ghost, sl.ghost_u, sl.nghost, it.x + (int)threadIdx.x,
                        (typename Store<PREC>::T*)((k & 1) ? sl.gpsi_b : sl.gpsi_a));
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
    using T = typename Store<PREC>::T;
    for (long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x; s < n;
         s += (long long)gridDim.x * blockDim.x) {
        const bool fluid = link == nullptr || ((link[s] >> kTypeShift) & 3u) == kTypeFluid;
        T rr = 0, rb = 0, rho = 0, j[3] = {0, 0, 0};
        if (fluid) obs_site<LAT, PREC>(P, a, (size_t)s, rr, rb, rho, j);
        const bool ok = fluid && rho > T(0);
        orr[s] = fluid ? (double)rr : 0.0;
        orb[s] = fluid ? (double)rb : 0.0;
        ou[s] = ok ? (double)(j[0] / rho) : 0.0;
        ou[n + s] = ok ? (double)(j[1] / rho) : 0.0;
        if (L::D == 3) ou[2 * n + s] = ok ? (double)(j[2] / rho) : 0.0;
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
    const unsigned blocks = (unsigned)((c->nghost + kFillThreads - 1) / kFillThreads);  // a thread per ghost
    // the ghost-psi table of buffer a, read by the marches' port lanes
    void* gpsi = gpsi_for(c, a);
#define F_(LAT, PREC)                                                                                   \
    k_fill_ports<LAT, PREC><<<blocks, kFillThreads, 0, c->stream>>>(c->kp, (SOf<PREC>*)a, c->d_ghost, \
                                                                    c->d_ghost_u, c->nghost,          \
                                                                    (typename Store<PREC>::T*)gpsi)
    LBCG_DISPATCH(c, F_);
#undef F_
    return cudaGetLastError();
}

cudaError_t launch_batch_fill(int lattice, int precision, const BatchSlot* slots, const BatchItem* items,
                              const int* nitems, int cap, int k, cudaStream_t st)
{
    if (cap <= 0) return cudaSuccess;
#define BF_(LAT, PREC) k_batch_fill<LAT, PREC><<<(unsigned)cap, kFillThreads, 0, st>>>(slots, items, nitems, k)
    if (lattice == LBCG_D2Q9) {
        if (precision == LBCG_FP64) BF_(0, LBCG_FP64);
        else if (precision == LBCG_FP32) BF_(0, LBCG_FP32);
        else if (precision == LBCG_FP32_DEV) BF_(0, LBCG_FP32_DEV);
        else BF_(0, LBCG_FP16_SCALED);
    } else {
        if (precision == LBCG_FP64) BF_(1, LBCG_FP64);
        else if (precision == LBCG_FP32) BF_(1, LBCG_FP32);
        else if (precision == LBCG_FP32_DEV) BF_(1, LBCG_FP32_DEV);
        else BF_(1, LBCG_FP16_SCALED);
    }
#undef BF_
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
    return run_observables(*c, a, FluidLink{c->any_link ? c->d_link : nullptr}, centre, r_in, r_out, (int)b,
                           d_partials, d_result, c->stream);
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
