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
// The array's name is only a host-side stand-in in host code, so the first
// call on each device (with that device current) looks up its device address
// with cudaGetSymbolAddress and caches it; that first call should therefore
// come before any stream capture.  All calls on a device share the one array
// and it keeps whatever the last call left in it; the join clears what must
// start at zero (its header and keys) itself.  Calls whose work overlaps on
// the GPU (different streams, or host threads, without ordering between
// them) race on the array and give wrong results: serialise them.
#include <mutex>

#include "internal.cuh"

namespace {

constexpr size_t kNoAllocScratchBytes = 64ull << 20;
constexpr int kNoAllocMaxDevices = 64;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

void *g_noalloc_ptr[kNoAllocMaxDevices] = {nullptr};
std::mutex g_noalloc_mu;

// device address of the scratch array on the current device (set up once)
mp_status noalloc_scratch(void **out)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return MP_ECUDA;
    if (dev < 0 || dev >= kNoAllocMaxDevices) return MP_EUNSUPPORTED;
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (g_noalloc_ptr[dev] == nullptr) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || p == nullptr)
            return MP_ECUDA;
        g_noalloc_ptr[dev] = p;
    }
    *out = g_noalloc_ptr[dev];
    return MP_OK;
}

}  // namespace

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
