// noalloc.cu -- allocation-free observables reduction (lbcg_observables_noalloc).
//
// For callers that must not allocate device memory themselves or through the
// library: plug-ins whose host application owns every device allocation through its
// own pool, real-time loops that forbid allocation after start-up, and code running
// with the device memory budget fully committed.  It computes what lbcg_observables
// computes, from a caller-owned state buffer and an optional caller-owned device mask,
// without a context; its reduction scratch is the file-scope array below.  The call is
// synchronous (it reads the result back to the host), so it cannot be recorded into a
// CUDA graph: on a stream that is being captured it returns LBCG_ERR_STATE at once.
#include <algorithm>
#include <cstring>
#include <mutex>
#include <string>

#include "obs_kernels.cuh"

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
    // a synchronous read-back would invalidate a capture: refuse before touching the stream
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    cudaError_t e = cudaStreamIsCapturing(st, &cap);
    if (e != cudaSuccess || cap != cudaStreamCaptureStatusNone) {
        err = "lbcg_observables_noalloc: synchronous call on a stream that is being captured";
        return LBCG_ERR_STATE;
    }
    // one partial row per block; the grid strides over the sites, so every lattice fits
    const int nb = (int)std::min<long long>(kNaRows, std::max<long long>(1, (c.n + 255) / 256));
    double* scratch = nullptr;
    e = na_scratch(&scratch);
    if (e != cudaSuccess) {
        err = std::string("lbcg_observables_noalloc: cudaGetSymbolAddress: ") + cudaGetErrorString(e);
        return LBCG_ERR_CUDA;
    }
    double* partials = scratch;
    double* res = scratch + (size_t)kNaRows * kNaSlots;
    e = run_observables(c, state, FluidMask{mask}, centre, r_in, r_out, nb, partials, res, st);
    double h[2 * kNaSlots];
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
