// noalloc.cu -- allocation-free observables reduction (lbcg_observables_noalloc).
//
// For callers that must not allocate device memory themselves or through the
// library: code that runs while a CUDA stream is being captured into a graph
// (cudaMalloc is not a capturable operation), plug-ins whose host application owns
// every device allocation through its own pool, and real-time loops that forbid
// allocation after start-up.  It computes what lbcg_observables computes, from a
// caller-owned state buffer and an optional caller-owned device mask, without a
// context; its reduction scratch is the file-scope array below.
#include <cstring>
#include <mutex>
#include <string>

#include "lbcg_device.cuh"

namespace lbcg {
namespace {

constexpr int kNaRows = 1024;                              // partial rows (one per block)
constexpr int kNaSlots = kObsSlots;                        // doubles per row
constexpr int kNaScratch = kNaRows * kNaSlots + 2 * kNaSlots;  // + result rows: 131,328 bytes

// Shared by every call in the process on this device; keeps the last call's contents.
static __device__ __align__(256) double g_noalloc_scratch[kNaScratch];

constexpr int kMaxDevices = 64;
std::mutex g_na_mutex;
double* g_na_ptr[kMaxDevices] = {nullptr};

template <int LAT, int PREC>
__device__ __forceinline__ void na_rb(const KParams& P, const typename Store<PREC>::S* a, int i, size_t s, double& fr,
                                      double& fb)
{
    using SP = Store<PREC>;
    using T = typename SP::T;
    const size_t ir = (size_t)i * P.np + s, ig = (size_t)(Lat<LAT>::Q + i) * P.np + s;
    if constexpr (PREC == LBCG_FP64 || PREC == LBCG_FP32) {
        fr = (double)a[ir];
        fb = (double)a[ig];
    } else {
        T r, g;
        SP::load(a, ir, ig, phys<T>(P), Lat<LAT>::cls(i), r, g);
        fr = (double)r;
        fb = ((double)g + P.pd.wr0[Lat<LAT>::cls(i)]) - (double)r;
    }
}

template <int NS>
__device__ __forceinline__ void na_block_reduce(double (&v)[NS], unsigned maxmask, double* out_row)
{
    __shared__ double sh[32][NS];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < NS; ++k)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const double t = __shfl_xor_sync(0xffffffffu, v[k], o);
            v[k] = ((maxmask >> k) & 1u) ? fmax(v[k], t) : v[k] + t;
        }
    if (lane == 0)
#pragma unroll
        for (int k = 0; k < NS; ++k) sh[warp][k] = v[k];
    __syncthreads();
    if (warp == 0) {
        const int nw = blockDim.x >> 5;
#pragma unroll
        for (int k = 0; k < NS; ++k) {
            double t = lane < nw ? sh[lane][k] : 0.0;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                const double q = __shfl_xor_sync(0xffffffffu, t, o);
                t = ((maxmask >> k) & 1u) ? fmax(t, q) : t + q;
            }
            if (lane == 0) out_row[k] = t;
        }
    }
}

// masses, momentum, red amount, max |u|, non-finite count (Eqs. 2-3)
template <int LAT, int PREC>
__global__ void __launch_bounds__(256) k_na_pass1(const KParams P, const typename Store<PREC>::S* __restrict__ a,
                                                  const uint8_t* __restrict__ mask, long long n, double* partials)
{
    using L = Lat<LAT>;
    double v[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    for (long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x; s < n;
         s += (long long)gridDim.x * blockDim.x) {
        if (mask && mask[s] != LBCG_MASK_FLUID) continue;
        double rr = 0, rb = 0, jx = 0, jy = 0, jz = 0;
#pragma unroll
        for (int i = 0; i < L::Q; ++i) {
            double fr, fb;
            na_rb<LAT, PREC>(P, a, i, (size_t)s, fr, fb);
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
    na_block_reduce<8>(v, 1u << 6, partials + (size_t)blockIdx.x * kNaSlots);
}

// pressure (Eq. 8) averaged inside r < r_in and outside r > r_out
template <int LAT, int PREC>
__global__ void __launch_bounds__(256) k_na_pass2(const KParams P, const typename Store<PREC>::S* __restrict__ a,
                                                  const uint8_t* __restrict__ mask, long long n, double cx, double cy,
                                                  double cz, double kpr, double kpb, const double* res,
                                                  double* partials)
{
    using L = Lat<LAT>;
    const double r_in = res[9], r_out = res[10];
    double v[4] = {0, 0, 0, 0};
    for (long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x; s < n;
         s += (long long)gridDim.x * blockDim.x) {
        if (mask && mask[s] != LBCG_MASK_FLUID) continue;
        const int x = (int)(s % P.nx);
        const int y = (int)((s / P.nx) % P.ny);
        const int z = (int)(s / ((long long)P.nx * P.ny));
        double d2 = 0.0, dd;
        dd = fabs((double)x - cx);
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
        const double r = sqrt(d2);
        if (r >= r_in && r <= r_out) continue;
        double rr = 0, rb = 0;
#pragma unroll
        for (int i = 0; i < L::Q; ++i) {
            double fr, fb;
            na_rb<LAT, PREC>(P, a, i, (size_t)s, fr, fb);
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
    na_block_reduce<4>(v, 0u, partials + (size_t)blockIdx.x * kNaSlots);
}

// one block: fixed-order reduction of nb partial rows into res[off..off+ns)
__global__ void k_na_final(const double* partials, int nb, int ns, unsigned maxmask, int off, double* res, int dim,
                           double r_in, double r_out)
{
    const int k = threadIdx.x;
    if (k < ns) {
        const bool is_max = (maxmask >> k) & 1u;
        double t = 0.0;
        for (int b = 0; b < nb; ++b) {
            const double q = partials[(size_t)b * kNaSlots + k];
            t = is_max ? fmax(t, q) : t + q;
        }
        res[off + k] = t;
    }
    __syncthreads();
    if (off == 0 && k == 0) {
        const double pi = 3.14159265358979323846;
        const double reff = dim == 2 ? sqrt(res[5] / pi) : cbrt(3.0 * res[5] / (4.0 * pi));
        res[8] = reff;
        res[9] = r_in < 0.0 ? reff / 2.0 : r_in;
        res[10] = r_out < 0.0 ? reff + 5.0 : r_out;
    }
}

// device address of the scratch array on the current device (set-up once per device)
cudaError_t na_scratch(double** out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_na_mutex);
    if (!g_na_ptr[dev]) {
        void* ptr = nullptr;
        e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_na_ptr[dev] = (double*)ptr;
    }
    *out = g_na_ptr[dev];
    return cudaSuccess;
}

}  // namespace

int noalloc_observables(const lbcg_params* p, const void* state, const uint8_t* mask, const double centre[3],
                        double r_in, double r_out, void* stream_ptr, lbcg_obs* out, std::string& err)
{
    // kernel parameters from a throw-away context description (host memory only)
    lbcg_ctx c;
    c.p = *p;
    if (c.p.lattice == LBCG_D2Q9) c.p.nz = 1;
    c.Q = c.p.lattice == LBCG_D2Q9 ? 9 : 19;
    c.D = c.p.lattice == LBCG_D2Q9 ? 2 : 3;
    c.dims[0] = c.p.nx;
    c.dims[1] = c.p.ny;
    c.dims[2] = c.p.nz;
    c.n = (long long)c.p.nx * c.p.ny * c.p.nz;
    c.np = (size_t)((c.n + 127) / 128 * 128);
    fill_kparams(&c);
    const cudaStream_t st = (cudaStream_t)stream_ptr;
    long long b = (c.n + 255) / 256;
    if (b > kNaRows) b = kNaRows;
    if (b < 1) b = 1;
    const int nb = (int)b;
    if (nb > kNaRows) {
        err = "lbcg_observables_noalloc: reduction needs more partial rows than the static scratch holds";
        return LBCG_ERR_CAPACITY;
    }
    double* scratch = nullptr;
    cudaError_t e = na_scratch(&scratch);
    if (e != cudaSuccess) {
        err = std::string("lbcg_observables_noalloc: cudaGetSymbolAddress: ") + cudaGetErrorString(e);
        return LBCG_ERR_CUDA;
    }
    double* partials = scratch;
    double* res = scratch + (size_t)kNaRows * kNaSlots;
    const int dim = c.D;
    const double kpr = dim == 2 ? 3.0 * (1.0 - p->alpha_r) / 5.0 : (1.0 - p->alpha_r) / 2.0;
    const double kpb = dim == 2 ? 3.0 * (1.0 - p->alpha_b) / 5.0 : (1.0 - p->alpha_b) / 2.0;
    const KParams& P = c.kp;
    const long long n = c.n;
#define NA_DISPATCH(F)                                                                           \
    do {                                                                                         \
        if (c.p.lattice == LBCG_D2Q9) {                                                          \
            if (c.p.precision == LBCG_FP64) F(0, LBCG_FP64);                                     \
            else if (c.p.precision == LBCG_FP32) F(0, LBCG_FP32);                                \
            else if (c.p.precision == LBCG_FP32_DEV) F(0, LBCG_FP32_DEV);                        \
            else F(0, LBCG_FP16_SCALED);                                                         \
        } else {                                                                                 \
            if (c.p.precision == LBCG_FP64) F(1, LBCG_FP64);                                     \
            else if (c.p.precision == LBCG_FP32) F(1, LBCG_FP32);                                \
            else if (c.p.precision == LBCG_FP32_DEV) F(1, LBCG_FP32_DEV);                        \
            else F(1, LBCG_FP16_SCALED);                                                         \
        }                                                                                        \
    } while (0)
#define F1_(LAT, PREC) \
    k_na_pass1<LAT, PREC><<<nb, 256, 0, st>>>(P, (const typename Store<PREC>::S*)state, mask, n, partials)
#define F2_(LAT, PREC)                                                                                    \
    k_na_pass2<LAT, PREC><<<nb, 256, 0, st>>>(P, (const typename Store<PREC>::S*)state, mask, n, centre[0], \
                                              centre[1], centre[2], kpr, kpb, res, partials)
    NA_DISPATCH(F1_);
    k_na_final<<<1, 32, 0, st>>>(partials, nb, 8, 1u << 6, 0, res, dim, r_in, r_out);
    NA_DISPATCH(F2_);
    k_na_final<<<1, 32, 0, st>>>(partials, nb, 4, 0u, 11, res, dim, r_in, r_out);
#undef F1_
#undef F2_
#undef NA_DISPATCH
    double h[2 * kNaSlots];
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(h, res, sizeof(h), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
        err = std::string("lbcg_observables_noalloc: ") + cudaGetErrorString(e);
        return LBCG_ERR_CUDA;
    }
    std::memset(out, 0, sizeof(*out));
    out->mass_r = h[0];
    out->mass_b = h[1];
    out->mom[0] = h[2];
    out->mom[1] = h[3];
    out->mom[2] = h[4];
    out->amount = h[5];
    out->umax = h[6];
    out->nonfinite = (int)h[7];
    out->r_eff = h[8];
    out->n_in = h[12];
    out->n_out = h[14];
    out->p_in = h[12] > 0 ? h[11] / h[12] : 0.0;
    out->p_out = h[14] > 0 ? h[13] / h[14] : 0.0;
    out->dp = out->p_in - out->p_out;
    out->step = -1;
    if (out->nonfinite > 0) {
        err = "non-finite or non-positive density at fluid sites";
        return LBCG_ERR_DIVERGED;
    }
    return LBCG_OK;
}

}  // namespace lbcg
