// join_fp64.cu -- all-FP64 instantiations of the diagonal-tile kernel
// (the comparison twin of the FP32-mixed kernel: every step in FP64).
#include "join_tile.cuh"

namespace mpgb {
namespace {

template <int D, int W, int RC, int MINB, bool RAW = false>
struct V {
    using Sh = TileShape<TraitsF64, D, W, RC>;
    static void *fn() { return (void *)join_tile_kernel<TraitsF64, D, W, RC, MINB, RAW>; }
    static cudaError_t launch(const Prob *probs, const Band *bands,
                              const unsigned long long *tp, Hdr *hdr, int tile_rows,
                              int anchor_every, int grid, cudaStream_t st)
    {
        join_tile_kernel<TraitsF64, D, W, RC, MINB, RAW><<<grid, Sh::NT, Sh::SMEM, st>>>(
            probs, bands, tp, hdr, tile_rows, anchor_every);
        return cudaGetLastError();
    }
};

// variant table: {id, D (diagonals per thread), W (warps per CTA), RC (rows per
// staged chunk), MINB (CTAs per SM the register budget must allow)}
#define MPGB_F64_VARIANTS(X) \
    X(0, 4, 4, 128, 2) X(1, 2, 4, 128, 2) X(2, 8, 2, 128, 2)

}  // namespace

int f64_variant_count() { return 3; }

bool f64_variant_info(int v, int *tile_diags, int *chunk_rows, int *threads, int *smem)
{
    switch (v) {
#define X(id, D, W, RC, MINB)                                              \
    case id:                                                         \
        *tile_diags = V<D, W, RC, MINB>::Sh::TD;                           \
        *chunk_rows = RC;                                            \
        *threads = V<D, W, RC, MINB>::Sh::NT;                              \
        *smem = V<D, W, RC, MINB>::Sh::SMEM;                               \
        return true;
        MPGB_F64_VARIANTS(X)
#undef X
    default:
        return false;
    }
}

int f64_blocks_per_sm(int v)
{
    int n = 0;
    switch (v) {
#define X(id, D, W, RC, MINB)                                                                       \
    case id:                                                                                  \
        cudaFuncSetAttribute(V<D, W, RC, MINB>::fn(), cudaFuncAttributeMaxDynamicSharedMemorySize,  \
                             V<D, W, RC, MINB>::Sh::SMEM);                                          \
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, V<D, W, RC, MINB>::fn(),              \
                                                          V<D, W, RC, MINB>::Sh::NT,                \
                                                          V<D, W, RC, MINB>::Sh::SMEM) != cudaSuccess) \
            n = 0;                                                                            \
        break;
        MPGB_F64_VARIANTS(X)
#undef X
    default:
        break;
    }
    return n;
}

cudaError_t launch_join_f64(int v, const Prob *probs, const Band *bands,
                            const unsigned long long *tile_prefix, Hdr *hdr, int tile_rows,
                            int anchor_every, int grid, cudaStream_t st)
{
    switch (v) {
#define X(id, D, W, RC, MINB) \
    case id:            \
        return V<D, W, RC, MINB>::launch(probs, bands, tile_prefix, hdr, tile_rows, anchor_every, grid, st);
        MPGB_F64_VARIANTS(X)
#undef X
    default:
        return cudaErrorInvalidValue;
    }
}

// the non-normalised distance (MP_FLAG_RAW) runs variant 0's shape only
int f64_raw_blocks_per_sm()
{
    using R = V<4, 4, 128, 2, true>;
    int n = 0;
    cudaFuncSetAttribute(R::fn(), cudaFuncAttributeMaxDynamicSharedMemorySize, R::Sh::SMEM);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, R::fn(), R::Sh::NT, R::Sh::SMEM) !=
        cudaSuccess)
        n = 0;
    return n;
}

cudaError_t launch_join_f64_raw(const Prob *probs, const Band *bands,
                                const unsigned long long *tile_prefix, Hdr *hdr, int tile_rows,
                                int anchor_every, int grid, cudaStream_t st)
{
    return V<4, 4, 128, 2, true>::launch(probs, bands, tile_prefix, hdr, tile_rows,
                                                 anchor_every, grid, st);
}

}  // namespace mpgb
