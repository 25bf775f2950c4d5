// step.cu -- which step kernel runs, and the dispatch of the step launches to the
// translation unit of the storage format (step_kernels.cuh, instantiated by step_f64.cu,
// step_f32.cu, step_f32dev.cu and step_f16.cu).
#include <cuda.h>
#include <cudaTypedefs.h>

#include <mutex>

#include "lbcg_internal.h"

namespace lbcg {

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

void* tma_encode_entry() { return reinterpret_cast<void*>(tma_encoder()); }

int effective_variant(const lbcg_ctx* c)
{
    const int prec = c->p.precision;
    // D2Q9: the moment march (6) by default for the regularized collision (measured fastest
    // on large boxes); every other value the plain march
    if (c->p.lattice == LBCG_D2Q9) {
        return (c->variant == 0 || c->variant == 6) && c->p.collision == LBCG_REG ? 6 : 0;
    }
    // default (measured fastest): the moment march with its moments in registers, on boxes with
    // walls or ports with neighbour-only plane barriers (9; on a link-free periodic box the two
    // run alike); the BGK update needs the individual populations and re-reads them (three
    // blocks per SM, FP64 two)
    const bool reg = c->p.collision == LBCG_REG;
    const int dflt = reg ? (c->any_link && c->block_rows <= 8 ? 9 : 6) : (prec == LBCG_FP64 ? 2 : 5);
    int v = c->variant != 0 ? c->variant : dflt;
    if (v == 8 && !tma_supported(c)) v = prec == LBCG_FP64 ? 6 : 7;
    if ((v == 6 || v == 7 || v == 9) && !reg) v = prec == LBCG_FP64 ? 2 : 5;
    return v;
}

// the step kernel refills the port ghosts of its output itself (the D3Q19 moment marches and
// both D2Q9 strip marches)
bool step_fuses_ports(const lbcg_ctx* c)
{
    if (c->nghost == 0 || !c->d_gstart || !c->d_tiles) return false;
    if (c->p.lattice == LBCG_D2Q9) return true;
    const int v = effective_variant(c);
    return v == 6 || v == 7 || v == 9;
}

cudaError_t launch_step(lbcg_ctx* c, const void* a, void* b)
{
    switch (c->p.precision) {
        case LBCG_FP64: return launch_step_prec<LBCG_FP64>(c, a, b);
        case LBCG_FP32: return launch_step_prec<LBCG_FP32>(c, a, b);
        case LBCG_FP32_DEV: return launch_step_prec<LBCG_FP32_DEV>(c, a, b);
        case LBCG_FP16_SCALED: return launch_step_prec<LBCG_FP16_SCALED>(c, a, b);
    }
    return cudaErrorInvalidValue;
}

int batch_resident_blocks(int lattice, int precision, int wy)
{
    switch (precision) {
        case LBCG_FP64: return batch_resident_blocks_prec<LBCG_FP64>(lattice, wy);
        case LBCG_FP32: return batch_resident_blocks_prec<LBCG_FP32>(lattice, wy);
        case LBCG_FP32_DEV: return batch_resident_blocks_prec<LBCG_FP32_DEV>(lattice, wy);
        default: return batch_resident_blocks_prec<LBCG_FP16_SCALED>(lattice, wy);
    }
}

cudaError_t launch_batch_step(int lattice, int precision, const BatchSlot* slots, const BatchItem* items,
                              const int* nitems, int k, int grid, int wy, cudaStream_t st)
{
    switch (precision) {
        case LBCG_FP64: return launch_batch_step_prec<LBCG_FP64>(lattice, slots, items, nitems, k, grid, wy, st);
        case LBCG_FP32: return launch_batch_step_prec<LBCG_FP32>(lattice, slots, items, nitems, k, grid, wy, st);
        case LBCG_FP32_DEV:
            return launch_batch_step_prec<LBCG_FP32_DEV>(lattice, slots, items, nitems, k, grid, wy, st);
        default: return launch_batch_step_prec<LBCG_FP16_SCALED>(lattice, slots, items, nitems, k, grid, wy, st);
    }
}

}  // namespace lbcg
