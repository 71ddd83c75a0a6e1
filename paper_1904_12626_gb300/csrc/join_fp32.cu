// join_fp32.cu -- FP32-mixed instantiations of the diagonal-tile kernel:
// FP64 statistics and anchors, FP32 recurrence, correlation and compares.
#include "join_tile.cuh"

namespace mpgb {
namespace {

template <int D, int W, int RC, int MINB, bool RAW = false>
struct V {
    using Sh = TileShape<TraitsF32, D, W, RC>;
    static void *fn() { return (void *)join_tile_kernel<TraitsF32, D, W, RC, MINB, RAW>; }
    static cudaError_t launch(const Prob *probs, const Band *bands,
                              const unsigned long long *tp, Hdr *hdr, int tile_rows,
                              int anchor_every, int grid, cudaStream_t st)
    {
        join_tile_kernel<TraitsF32, D, W, RC, MINB, RAW><<<grid, Sh::NT, Sh::SMEM, st>>>(
            probs, bands, tp, hdr, tile_rows, anchor_every);
        return cudaGetLastError();
    }
};

// variant table: {id, D (diagonals per thread), W (warps per CTA), RC (rows per
// staged chunk), MINB (CTAs per SM the register budget must allow)}
#define MPGB_F32_VARIANTS(X) \
    X(0, 8, 2, 512, 8) X(1, 8, 4, 512, 4) X(2, 8, 2, 512, 10) X(3, 8, 4, 256, 4) \
    X(4, 8, 1, 256, 16) X(5, 8, 2, 256, 12) X(6, 8, 2, 256, 10) X(7, 8, 4, 512, 5)
// (four warps with 1024-row chunks at 4 CTAs per SM was slower on every join
// family: self-join 106.3 ms against 102.8 for variant 7, AB 289 / 263,
// batched 1398 / 1298, pan 72.0 / 69.4, gradient input 1.71 / 1.36)

}  // namespace

int f32_variant_count() { return 8; }

bool f32_variant_info(int v, int *tile_diags, int *chunk_rows, int *threads, int *smem)
{
    switch (v) {
#define X(id, D, W, RC, MINB)                                              \
    case id:                                                         \
        *tile_diags = V<D, W, RC, MINB>::Sh::TD;                           \
        *chunk_rows = RC;                                            \
        *threads = V<D, W, RC, MINB>::Sh::NT;                              \
        *smem = V<D, W, RC, MINB>::Sh::SMEM;                               \
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
#define X(id, D, W, RC, MINB)                                                                       \
    case id:                                                                                  \
        cudaFuncSetAttribute(V<D, W, RC, MINB>::fn(), cudaFuncAttributeMaxDynamicSharedMemorySize,  \
                             V<D, W, RC, MINB>::Sh::SMEM);                                          \
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, V<D, W, RC, MINB>::fn(),              \
                                                          V<D, W, RC, MINB>::Sh::NT,                \
                                                          V<D, W, RC, MINB>::Sh::SMEM) != cudaSuccess) \
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
#define X(id, D, W, RC, MINB) \
    case id:            \
        return V<D, W, RC, MINB>::launch(probs, bands, tile_prefix, hdr, tile_rows, anchor_every, grid, st);
        MPGB_F32_VARIANTS(X)
#undef X
    default:
        return cudaErrorInvalidValue;
    }
}

// the non-normalised distance (MP_FLAG_RAW) runs variant 0's shape only
int f32_raw_blocks_per_sm()
{
    using R = V<8, 2, 512, 8, true>;
    int n = 0;
    cudaFuncSetAttribute(R::fn(), cudaFuncAttributeMaxDynamicSharedMemorySize, R::Sh::SMEM);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, R::fn(), R::Sh::NT, R::Sh::SMEM) !=
        cudaSuccess)
        n = 0;
    return n;
}

cudaError_t launch_join_f32_raw(const Prob *probs, const Band *bands,
                                const unsigned long long *tile_prefix, Hdr *hdr, int tile_rows,
                                int anchor_every, int grid, cudaStream_t st)
{
    return V<8, 2, 512, 8, true>::launch(probs, bands, tile_prefix, hdr, tile_rows,
                                                 anchor_every, grid, st);
}

}  // namespace mpgb
