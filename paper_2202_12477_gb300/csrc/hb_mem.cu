// Memory of meshes and solver state.
//
// Device arrays that a mesh allocates while it is built come from one memory
// pool per device that the library owns, through stream-ordered allocation
// (cudaMallocFromPoolAsync / cudaFreeAsync): neither call waits for the rest
// of the device, so a mesh can be built and released while other streams run
// (the server builds requests' meshes beside the rounds it launches). The
// pool keeps up to kKeepBytes of freed memory for reuse and returns the rest
// to the device at the next synchronisation; it never makes one stream wait
// for another's frees (internal dependencies are off), it grows instead.
//
// Small pinned host buffers (the CG state read-backs) are carved from pinned
// chunks that are allocated once and reused, so creating or destroying a mesh
// calls neither cudaMallocHost nor cudaFreeHost.
#include <mutex>
#include <vector>

#include "hb_internal.h"

namespace {

constexpr uint64_t kKeepBytes = 8ull << 30;
constexpr size_t kPinnedSlot = 256;   // bytes per pinned buffer
constexpr size_t kPinnedChunk = 256;  // buffers per pinned chunk

std::mutex g_mem_mu;
cudaMemPool_t g_pool[64] = {};
std::vector<void *> g_pinned_free;

cudaError_t pool_for(int dev, cudaMemPool_t *out)
{
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lk(g_mem_mu);
    if (!g_pool[dev]) {
        cudaMemPoolProps props{};
        props.allocType = cudaMemAllocationTypePinned;
        props.handleTypes = cudaMemHandleTypeNone;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = dev;
        cudaMemPool_t p = nullptr;
        cudaError_t e = cudaMemPoolCreate(&p, &props);
        if (e != cudaSuccess) return e;
        uint64_t keep = kKeepBytes;
        int no = 0;
        e = cudaMemPoolSetAttribute(p, cudaMemPoolAttrReleaseThreshold, &keep);
        if (e == cudaSuccess) e = cudaMemPoolSetAttribute(p, cudaMemPoolReuseAllowInternalDependencies, &no);
        if (e != cudaSuccess) {
            cudaMemPoolDestroy(p);
            return e;
        }
        g_pool[dev] = p;
    }
    *out = g_pool[dev];
    return cudaSuccess;
}

}  // namespace

cudaError_t hb_dev_alloc(void **p, size_t bytes, cudaStream_t s)
{
    *p = nullptr;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    cudaMemPool_t pool = nullptr;
    if (e == cudaSuccess) e = pool_for(dev, &pool);
    if (e == cudaSuccess) e = cudaMallocFromPoolAsync(p, bytes > 0 ? bytes : 16, pool, s);
    return e;
}

void hb_dev_free(void *p, cudaStream_t s)
{
    if (p) cudaFreeAsync(p, s);
}

cudaError_t hb_dev_keep(uint64_t bytes)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    cudaMemPool_t pool = nullptr;
    if (e == cudaSuccess) e = pool_for(dev, &pool);
    if (e == cudaSuccess) e = cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &bytes);
    return e;
}

uint64_t hb_dev_keep_default() { return kKeepBytes; }

void hb_dev_trim()
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return;
    std::lock_guard<std::mutex> lk(g_mem_mu);
    if (g_pool[dev]) cudaMemPoolTrimTo(g_pool[dev], 0);
}

cudaError_t hb_pinned_get(void **p, size_t bytes)
{
    *p = nullptr;
    if (bytes > kPinnedSlot) return cudaErrorInvalidValue;
    std::lock_guard<std::mutex> lk(g_mem_mu);
    if (g_pinned_free.empty()) {
        unsigned char *chunk = nullptr;
        cudaError_t e = cudaMallocHost((void **)&chunk, kPinnedSlot * kPinnedChunk);
        if (e != cudaSuccess) return e;
        for (size_t i = kPinnedChunk; i-- > 0;) g_pinned_free.push_back(chunk + i * kPinnedSlot);
    }
    *p = g_pinned_free.back();
    g_pinned_free.pop_back();
    return cudaSuccess;
}

void hb_pinned_put(void *p)
{
    if (!p) return;
    std::lock_guard<std::mutex> lk(g_mem_mu);
    g_pinned_free.push_back(p);
}
