// noalloc.cu -- a self-join entry point for callers that cannot allocate
// device memory.
//
// Some callers have no way to get a device workspace: code running where
// cudaMalloc is forbidden or unavailable (inside a region another framework
// is capturing into a CUDA graph, under an allocator that owns all device
// memory, or in a plugin host that hands over only its input and output
// buffers).  mp_selfjoin_noalloc serves them with scratch memory the library
// itself owns: one file-scope device array of kNoAllocScratchBytes (64 MiB),
// which every GPU that loads the library keeps until the process exits.
//
// The array's name is only a host-side stand-in in host code: its device
// address belongs to the CUDA context the library's device code is loaded
// in.  Every call therefore looks the address up with cudaGetSymbolAddress,
// on the device current at the call, instead of keeping one from an earlier
// call (a cached address would go stale after cudaDeviceReset or in another
// context).  The first call on a device also loads the library's device code
// there, so make that first call before any stream capture.  All calls on a
// device share the one array and it keeps whatever the last call left in it;
// the join clears what must start at zero (its header and keys) itself.
// Calls whose work overlaps on the GPU (different streams, or host threads,
// without ordering between them) race on the array and give wrong results:
// serialise them.
#include "internal.cuh"

namespace {

constexpr size_t kNoAllocScratchBytes = 64ull << 20;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

// device address of the scratch array in the current device's context
mp_status noalloc_scratch(void **out)
{
    void *p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || p == nullptr)
        return MP_ECUDA;
    *out = p;
    return MP_OK;
}

}  // namespace

extern "C" int64_t mp_selfjoin_noalloc_max_n(const mp_config *cfg)
{
    if (!cfg || cfg->m < 4) return 0;
    // the workspace grows with n: the largest n whose workspace fits
    int64_t lo = cfg->m, hi = (int64_t)1 << 31;
    const size_t first = mp_selfjoin_workspace_bytes(lo, cfg);
    if (first == 0 || first > kNoAllocScratchBytes) return 0;
    while (hi - lo > 1) {
        const int64_t mid = lo + (hi - lo) / 2;
        const size_t need = mp_selfjoin_workspace_bytes(mid, cfg);
        if (need != 0 && need <= kNoAllocScratchBytes) lo = mid; else hi = mid;
    }
    return lo;
}

extern "C" mp_status mp_selfjoin_noalloc(const void *x, int32_t dtype, int64_t n,
                                         const mp_config *cfg, double *mp, int64_t *pi,
                                         void *stream)
{
    if (!x || !mp || !pi || !cfg) return MP_EINVAL;
    const size_t need = mp_selfjoin_workspace_bytes(n, cfg);
    if (need == 0) return MP_EINVAL;
    if (need > kNoAllocScratchBytes) return MP_ENOMEM;     // series too long for the scratch
    void *ws = nullptr;
    const mp_status s = noalloc_scratch(&ws);
    if (s != MP_OK) return s;
    return mp_selfjoin(x, dtype, n, cfg, mp, pi, ws, kNoAllocScratchBytes, stream);
}

extern "C" mp_status mp_selfjoin_noalloc_device_status(void *stream)
{
    void *ws = nullptr;
    const mp_status s = noalloc_scratch(&ws);
    if (s != MP_OK) return s;
    return mp_get_device_status(ws, stream);
}
