// join_fp32.cu -- FP32-mixed instantiations of the diagonal-tile kernel:
// FP64 statistics and anchors, FP32 recurrence, correlation and compares.
#include "join_tile.cuh"

namespace mpgb {
namespace {

template <int D, int W, int RC>
struct V {
    using Sh = TileShape<TraitsF32, D, W, RC>;
    static void *fn() { return (void *)join_tile_kernel<TraitsF32, D, W, RC, 2>; }
    static cudaError_t launch(const Prob *probs, const Band *bands,
                              const unsigned long long *tp, Hdr *hdr, int tile_rows,
                              int anchor_every, int grid, cudaStream_t st)
    {
        join_tile_kernel<TraitsF32, D, W, RC, 2><<<grid, Sh::NT, Sh::SMEM, st>>>(
            probs, bands, tp, hdr, tile_rows, anchor_every);
        return cudaGetLastError();
    }
};

// variant table: {D, W, RC}
#define MPGB_F32_VARIANTS(X) X(0, 8, 4, 256) X(1, 4, 4, 256) X(2, 8, 2, 256) X(3, 16, 2, 256)

}  // namespace

int f32_variant_count() { return 4; }

bool f32_variant_info(int v, int *tile_diags, int *chunk_rows, int *threads, int *smem)
{
    switch (v) {
#define X(id, D, W, RC)                                              \
    case id:                                                         \
        *tile_diags = V<D, W, RC>::Sh::TD;                           \
        *chunk_rows = RC;                                            \
        *threads = V<D, W, RC>::Sh::NT;                              \
        *smem = V<D, W, RC>::Sh::SMEM;                               \
        return true;
        MPGB_F32_VARIANTS(X)
#undef X
    default:
        return false;
    }
}

int f32_blocks_per_sm(int v)
{
    int n = 0;
    switch (v) {
#define X(id, D, W, RC)                                                                       \
    case id:                                                                                  \
        cudaFuncSetAttribute(V<D, W, RC>::fn(), cudaFuncAttributeMaxDynamicSharedMemorySize,  \
                             V<D, W, RC>::Sh::SMEM);                                          \
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, V<D, W, RC>::fn(),              \
                                                          V<D, W, RC>::Sh::NT,                \
                                                          V<D, W, RC>::Sh::SMEM) != cudaSuccess) \
            n = 0;                                                                            \
        break;
        MPGB_F32_VARIANTS(X)
#undef X
    default:
        break;
    }
    return n;
}

cudaError_t launch_join_f32(int v, const Prob *probs, const Band *bands,
                            const unsigned long long *tile_prefix, Hdr *hdr, int tile_rows,
                            int anchor_every, int grid, cudaStream_t st)
{
    switch (v) {
#define X(id, D, W, RC) \
    case id:            \
        return V<D, W, RC>::launch(probs, bands, tile_prefix, hdr, tile_rows, anchor_every, grid, st);
        MPGB_F32_VARIANTS(X)
#undef X
    default:
        return cudaErrorInvalidValue;
    }
}

}  // namespace mpgb
